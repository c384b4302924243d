"""Pins of the oracle's general PIC push-forward (Eqs. 7-8 with any particle
half-width delta): the cell weights against the textbook quadratic B-spline at
delta = h and against brute-force quadrature of the particle over the cells at
other widths, the mass balance the paper states (columns of F sum to one), the
Dirac limit, and the derivatives against finite differences and the adjoint
identity."""
import numpy as np
import pytest

from oracle import lagrangian as L
from oracle import objective as O


def _bspline2(t):
    """Quadratic B-spline (the box convolved with the hat), textbook form."""
    t = np.abs(t)
    return np.where(t <= 0.5, 0.75 - t * t, np.where(t <= 1.5, 0.5 * (1.5 - t) ** 2, 0.0))


def _weights_1d(g, y, delta):
    """Dense F column for one particle at y on a 1D grid."""
    return L.scatter_hat(np.ones(1), g, np.array([[y]]), delta)


def test_width_h_is_the_quadratic_bspline():
    g = L.Grid((12,), (0.0,), (1.2,))
    h = g.h[0]
    rng = np.random.default_rng(0)
    for y in rng.uniform(0.3, 0.9, size=25):
        w = _weights_1d(g, y, h)
        xc = g.lo[0] + (np.arange(12) + 0.5) * h
        assert np.allclose(w, _bspline2((xc - y) / h), atol=1e-14)
    # a particle at a cell centre: 1/8, 3/4, 1/8
    w = _weights_1d(g, g.lo[0] + 5.5 * h, h)
    assert np.allclose(w[4:7], [0.125, 0.75, 0.125], atol=1e-14) and abs(w.sum() - 1) < 1e-14


@pytest.mark.parametrize("ratio", [0.3, 0.5, 1.0, 1.7, 2.5, 3.5])
def test_weights_match_quadrature_of_the_particle(ratio):
    g = L.Grid((16,), (0.0,), (1.0,))
    h = g.h[0]
    delta = ratio * h
    rng = np.random.default_rng(int(ratio * 10))
    for y in rng.uniform(0.2, 0.8, size=6):
        w = _weights_1d(g, y, delta)
        # midpoint rule with 4000 samples per cell of the hat density
        n = 4000
        ref = np.zeros(16)
        for i in range(16):
            x = (i + (np.arange(n) + 0.5) / n) * h
            ref[i] = np.sum(np.maximum(0.0, 1.0 - np.abs(x - y) / delta) / delta) * h / n
        assert np.max(np.abs(w - ref)) < 2e-7


def test_2d_weights_match_quadrature():
    g = L.Grid((6, 5), (0.0, 0.0), (1.2, 1.0))
    delta = 0.27
    p = np.array([[0.55], [0.47]])
    w = L.scatter_hat(np.ones(1), g, p, delta)
    n = 200
    ref = np.zeros(g.shape)
    for j in range(5):
        for i in range(6):
            x = g.lo[0] + (i + (np.arange(n) + 0.5) / n) * g.h[0]
            y = g.lo[1] + (j + (np.arange(n) + 0.5) / n) * g.h[1]
            X, Y = np.meshgrid(x, y, indexing="ij")
            dens = np.maximum(0, 1 - np.abs(X - p[0, 0]) / delta) * np.maximum(0, 1 - np.abs(Y - p[1, 0]) / delta)
            ref[j, i] = dens.sum() / delta ** 2 * g.cell_volume / n ** 2
    assert np.max(np.abs(w - ref)) < 1e-5
    assert abs(w.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("ratio", [0.4, 1.0, 2.2, 3.5])
def test_mass_is_preserved_for_any_width(ratio):
    g = L.Grid((20, 18, 9), (0.0, 0.0, 0.0), (1.0, 0.9, 0.45))
    rng = np.random.default_rng(1)
    P = 200
    p = np.stack([rng.uniform(0.25, 0.75, P), rng.uniform(0.25, 0.65, P), rng.uniform(0.2, 0.25, P)])
    m = rng.uniform(0.5, 2.0, P)
    out = L.scatter_hat(m, g, p, ratio * 0.05)
    assert abs(out.sum() - m.sum()) < 1e-12 * m.sum()
    # mass that reaches past the boundary leaves the grid
    q = np.array([[0.01], [0.45], [0.225]])
    assert L.scatter_hat(np.ones(1), g, q, 0.1).sum() < 1.0 - 1e-3


def test_narrow_particle_is_nearest_cell():
    g = L.Grid((10, 10))
    rng = np.random.default_rng(2)
    p = (np.floor(rng.uniform(1, 9, size=(2, 30))) + rng.uniform(0.3, 0.7, size=(2, 30))) * g.h[:, None]
    out = L.scatter_hat(np.ones(30), g, p, 0.2 * g.h[0])
    ref = np.zeros(g.shape)
    idx = np.floor(p / g.h[:, None]).astype(int)
    np.add.at(ref, (idx[1], idx[0]), 1.0)
    assert np.allclose(out, ref, atol=1e-14)


def test_scatter_gradient_and_gather_transpose():
    g = L.Grid((9, 11), (0.0, 0.0), (0.9, 1.1))
    rng = np.random.default_rng(3)
    P, delta = 40, 0.17
    p = rng.uniform(0.05, 0.95, size=(2, P))
    m = rng.uniform(0.5, 1.5, P)
    dp = rng.normal(size=(2, P))
    eps = 1e-6
    fd = (L.scatter_hat(m, g, p + eps * dp, delta) - L.scatter_hat(m, g, p - eps * dp, delta)) / (2 * eps)
    an = L.scatter_hat_gradient(m, dp, g, p, delta)
    assert np.max(np.abs(fd - an)) < 1e-7 * max(1.0, np.max(np.abs(an)))
    F = rng.normal(size=g.shape)
    val, grad = L.gather_hat(F, g, p, delta, gradient=True)
    assert abs(np.sum(L.scatter_hat(m, g, p, delta) * F) - np.sum(m * val)) < 1e-12
    assert abs(np.sum(an * F) - np.sum(m * np.sum(grad * dp, axis=0))) < 1e-11


def _problem(delta):
    ig = L.Grid((14, 12), (0.0, 0.0), (1.0, 0.9))
    vg = L.Grid((7, 6), (0.0, 0.0), (1.0, 0.9))
    return O.Problem(ig, vg, 2, 3, "continuity", "diffusion", 1e-3, 0.0, delta=delta)


def _fields(prob, seed=4):
    rng = np.random.default_rng(seed)
    X = L.cell_centres(prob.igrid)
    T = np.exp(-((X[0] - 0.5) ** 2 + (X[1] - 0.45) ** 2) / 0.02).reshape(prob.igrid.shape)
    T[:4], T[-4:], T[:, :4], T[:, -4:] = 0.0, 0.0, 0.0, 0.0    # no mass within reach of the boundary
    v = 0.02 * rng.normal(size=prob.vshape)
    dv = rng.normal(size=prob.vshape)
    r = rng.normal(size=prob.igrid.shape)
    return T, v, dv, r


@pytest.mark.parametrize("ratio", [0.6, 1.0, 2.0])
def test_model_derivatives_with_general_width(ratio):
    prob = _problem(ratio * 1.0 / 14)
    T, v, dv, r = _fields(prob)
    args = (prob.model, v, prob.vgrid, T, prob.igrid, prob.N)
    eps = 1e-5
    up, _ = L.final_state("continuity", v + eps * dv, prob.vgrid, T, prob.igrid, prob.N, prob.delta)
    dn, _ = L.final_state("continuity", v - eps * dv, prob.vgrid, T, prob.igrid, prob.N, prob.delta)
    J = L.jvp(*args, dv, prob.delta)
    assert np.linalg.norm((up - dn) / (2 * eps) - J) <= 1e-6 * np.linalg.norm(J)
    lhs = np.sum(J * r)
    rhs = np.sum(dv * L.jtvp(*args, r, prob.delta))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
    u1, _ = L.final_state(*args, prob.delta)
    assert abs(u1.sum() - T.sum()) <= 1e-12 * T.sum()


def test_objective_gradient_with_general_width():
    prob = _problem(1.5 / 14)
    T, v, dv, _ = _fields(prob, 5)
    R = np.roll(T, 1, axis=1)
    g = O.gradient(prob, v, T, R)
    eps = 1e-6
    fd = (O.objective(prob, v + eps * dv, T, R)[0] - O.objective(prob, v - eps * dv, T, R)[0]) / (2 * eps)
    assert abs(fd - np.sum(g * dv)) <= 1e-6 * abs(fd)
