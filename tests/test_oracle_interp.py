"""Pins of the oracle's interpolation and push-forward (Sec. 3.1, Eqs. 6-8)
against library routines, closed forms and brute force."""
import numpy as np
import pytest
from scipy import ndimage

from oracle.lagrangian import Grid, cell_centres, interpolate, scatter, scatter_gradient


def _grid(d):
    return Grid((7, 5, 4)[:d], lo=(-0.3, 0.1, 0.0)[:d], hi=(1.1, 0.9, 2.0)[:d])


@pytest.mark.parametrize("d", [2, 3])
def test_interpolate_matches_scipy_grid_constant(d):
    """Linear interpolation with zero extension is scipy's order-1
    map_coordinates in 'grid-constant' mode (data extended by cval = 0)."""
    g = _grid(d)
    rng = np.random.default_rng(1)
    F = rng.normal(size=g.shape)
    P = 400
    p = np.stack([rng.uniform(g.lo[a] - 2 * g.h[a], g.hi[a] + 2 * g.h[a], P) for a in range(d)])
    ours = interpolate(F, g, p)
    # continuous index per numpy axis (z, y, x)
    coords = np.stack([(p[a] - g.lo[a]) / g.h[a] - 0.5 for a in reversed(range(d))])
    ref = ndimage.map_coordinates(F, coords, order=1, mode="grid-constant", cval=0.0)
    np.testing.assert_allclose(ours, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_interpolate_reproduces_affine_and_its_gradient(d):
    g = _grid(d)
    rng = np.random.default_rng(2)
    a = rng.normal(size=d)
    b = 0.7
    xc = cell_centres(g)
    F = (b + a @ xc).reshape(g.shape)
    # points strictly inside the hull of the centres
    p = np.stack([rng.uniform(g.lo[k] + 0.5 * g.h[k], g.hi[k] - 0.5 * g.h[k], 300) for k in range(d)])
    val, grad = interpolate(F, g, p, gradient=True)
    np.testing.assert_allclose(val, b + a @ p, atol=1e-12)
    np.testing.assert_allclose(grad, np.repeat(a[:, None], p.shape[1], axis=1), atol=1e-11)


@pytest.mark.parametrize("d", [2, 3])
def test_interpolate_gradient_central_difference(d):
    g = _grid(d)
    rng = np.random.default_rng(3)
    F = rng.normal(size=g.shape)
    p = np.stack([rng.uniform(g.lo[k] - g.h[k], g.hi[k] + g.h[k], 200) for k in range(d)])
    _, grad = interpolate(F, g, p, gradient=True)
    eps = 1e-7
    for a in range(d):
        e = np.zeros((d, 1))
        e[a] = eps
        fd = (interpolate(F, g, p + e) - interpolate(F, g, p - e)) / (2 * eps)
        np.testing.assert_allclose(grad[a], fd, rtol=1e-5, atol=1e-5)


def test_gradient_at_nodes_takes_the_cell_to_the_right():
    """At a node the interpolant has a kink; the derivative is that of the
    cell to the right (floor), i.e. the forward difference, with zero beyond
    the last node.  The domain's h is not exact in binary, so (x - lo)/h - 1/2
    is not an exact integer at every node before it is snapped."""
    g = Grid((37, 29), lo=(-0.2, 0.0), hi=(1.1, 1.3))
    F = np.random.default_rng(5).normal(size=g.shape)      # [y][x]
    val, grad = interpolate(F, g, cell_centres(g), gradient=True)
    assert np.allclose(val.reshape(g.shape), F, rtol=0, atol=1e-12)
    Fp = np.concatenate([F, np.zeros((g.m[1], 1))], axis=1)
    fx = (Fp[:, 1:] - Fp[:, :-1]) / g.h[0]
    Fq = np.concatenate([F, np.zeros((1, g.m[0]))], axis=0)
    fy = (Fq[1:, :] - Fq[:-1, :]) / g.h[1]
    assert np.allclose(grad[0].reshape(g.shape), fx, rtol=0, atol=1e-9)
    assert np.allclose(grad[1].reshape(g.shape), fy, rtol=0, atol=1e-9)


def test_zero_extension_far_outside():
    g = _grid(2)
    F = np.ones(g.shape)
    p = np.array([[g.lo[0] - 3 * g.h[0], g.hi[0] + 5.0], [0.5, 0.5]])
    val, grad = interpolate(F, g, p, gradient=True)
    assert np.all(val == 0.0) and np.all(grad == 0.0)


@pytest.mark.parametrize("d", [2, 3])
def test_scatter_is_transpose_of_interpolate(d):
    """With particle width = cell size the push-forward matrix is the transpose
    of the linear interpolation matrix (Sec. 3.1, end of Step 2)."""
    g = _grid(d)
    rng = np.random.default_rng(4)
    P = 150
    p = np.stack([rng.uniform(g.lo[a] - g.h[a], g.hi[a] + g.h[a], P) for a in range(d)])
    w = rng.normal(size=P)
    F = rng.normal(size=g.shape)
    lhs = np.sum(scatter(w, g, p) * F)
    rhs = np.sum(w * interpolate(F, g, p))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("d", [2, 3])
def test_scatter_conserves_mass_inside(d):
    """Columns of F sum to one (Sec. 3.1): mass is conserved for particles whose
    stencil stays on the grid."""
    g = _grid(d)
    rng = np.random.default_rng(5)
    P = 300
    p = np.stack([rng.uniform(g.lo[a] + 0.5 * g.h[a], g.hi[a] - 0.5 * g.h[a], P) for a in range(d)])
    w = rng.uniform(0, 1, size=P)
    assert abs(scatter(w, g, p).sum() - w.sum()) <= 1e-12 * w.sum()


def test_scatter_weights_are_top_hat_cell_integrals_1d():
    """Brute force in 1D: the splat weight of a particle at y on cell i equals the
    integral over cell i of a unit-mass top-hat particle of width h centred at y
    (exact cell integration, Eq. 8, with width = cell size)."""
    g = Grid((9,), lo=(0.0,), hi=(1.0,))
    h = g.h[0]
    rng = np.random.default_rng(6)
    for y in rng.uniform(0.5 * h, 1 - 0.5 * h, 40):
        w = scatter(np.array([1.0]), g, np.array([[y]]))
        xs = (np.arange(9) + 0.5) * h
        # overlap length of [y - h/2, y + h/2] with [x_i - h/2, x_i + h/2], per unit h
        ov = np.clip(np.minimum(y + h / 2, xs + h / 2) - np.maximum(y - h / 2, xs - h / 2), 0, None) / h
        np.testing.assert_allclose(w, ov, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_scatter_gradient_is_derivative_of_scatter(d):
    g = _grid(d)
    rng = np.random.default_rng(7)
    P = 120
    p = np.stack([rng.uniform(g.lo[a], g.hi[a], P) for a in range(d)])
    dp = rng.normal(size=p.shape)
    w = rng.normal(size=P)
    eps = 1e-7
    fd = (scatter(w, g, p + eps * dp) - scatter(w, g, p - eps * dp)) / (2 * eps)
    np.testing.assert_allclose(scatter_gradient(w, dp, g, p), fd, rtol=1e-5, atol=1e-5)
