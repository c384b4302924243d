"""Pins of the oracle's characteristics (Eq. 4, Alg. 1) and final states
(Eqs. 6-7) against closed forms and invariants."""
import numpy as np
import pytest

from oracle import lagrangian as L
from paper_1703_04446_gb300 import synth


def _vel_from(fun, vgrid, K):
    """Sample a velocity field fun(x_list, t) -> list of d arrays on the grid nodes."""
    xc = L.cell_centres(vgrid)
    v = np.zeros((K, vgrid.d) + vgrid.shape)
    for j in range(K):
        t = 0.0 if K == 1 else j / (K - 1)
        comps = fun([xc[a] for a in range(vgrid.d)], t)
        for c in range(vgrid.d):
            v[j, c] = np.asarray(comps[c]).reshape(vgrid.shape)
    return v


@pytest.mark.parametrize("model", ["transport", "continuity"])
@pytest.mark.parametrize("d,K", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_zero_velocity_is_identity(model, d, K):
    ig = L.Grid((6, 5, 4)[:d])
    vg = L.Grid((3, 3, 2)[:d])
    T = np.random.default_rng(0).normal(size=ig.shape)
    v = np.zeros((K, d) + vg.shape)
    u1, y = L.final_state(model, v, vg, T, ig, 4)
    assert np.array_equal(y, L.cell_centres(ig))
    # the cell-centre coordinates round-trip through the continuous index
    np.testing.assert_allclose(u1, T, rtol=0, atol=1e-13)


@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("d", [2, 3])
def test_constant_velocity_is_exact_shift(direction, d):
    """v = c in the interior: every RK4 stage sees c, so y = x + direction * c."""
    vg = L.Grid((12,) * d)
    c = np.array([0.07, -0.05, 0.03][:d])
    v = _vel_from(lambda x, t: [np.full_like(x[0], c[a]) for a in range(d)], vg, 1)
    rng = np.random.default_rng(1)
    x = rng.uniform(0.3, 0.7, size=(d, 50))
    y, _, _ = L.characteristics(v, vg, x, 5, direction)
    np.testing.assert_allclose(y, x + direction * c[:, None], atol=1e-14)


def test_constant_velocity_transport_is_grid_shift():
    """Transport with a constant displacement of whole image cells shifts T by
    that many cells (interior voxels)."""
    ig = L.Grid((16, 16))
    vg = L.Grid((16, 16))
    h = ig.h[0]
    c = np.array([2 * h, -1 * h])
    v = _vel_from(lambda x, t: [np.full_like(x[0], c[0]), np.full_like(x[0], c[1])], vg, 1)
    T = np.random.default_rng(2).normal(size=ig.shape)
    u1, _ = L.final_state("transport", v, vg, T, ig, 3)
    # u1(x) = T(x - c): voxel (iy, ix) takes T[iy + 1, ix - 2]
    np.testing.assert_allclose(u1[2:12, 4:12], T[3:13, 2:10], atol=1e-12)


def _rotation(d, omega, x0):
    if d == 2:
        return lambda x, t: [-omega * (x[1] - x0[1]), omega * (x[0] - x0[0])]
    return lambda x, t: [-omega * (x[1] - x0[1]), omega * (x[0] - x0[0]), np.zeros_like(x[0])]


def _rotate(x, x0, ang):
    out = x.copy()
    dx, dy = x[0] - x0[0], x[1] - x0[1]
    out[0] = x0[0] + np.cos(ang) * dx - np.sin(ang) * dy
    out[1] = x0[1] + np.sin(ang) * dx + np.cos(ang) * dy
    return out


def _order(errs, Ns):
    return np.polyfit(np.log(Ns), np.log(errs), 1)[0]


@pytest.mark.parametrize("d", [2, 3])
def test_rk4_is_fourth_order_on_rigid_rotation(d):
    """A rigid rotation is linear in x, so multilinear interpolation is exact
    inside the grid and only the RK4 error remains: slope -4 (Alg. 1)."""
    vg = L.Grid((20,) * d)
    x0 = np.full(d, 0.5)
    omega = 2.0
    v = _vel_from(_rotation(d, omega, x0), vg, 1)
    rng = np.random.default_rng(3)
    x = x0[:, None] + rng.uniform(-0.2, 0.2, size=(d, 40))
    Ns = np.array([4, 8, 16, 32])
    errs = []
    for N in Ns:
        y, _, _ = L.characteristics(v, vg, x, int(N), +1)
        errs.append(np.max(np.abs(y - _rotate(x, x0, omega))))
    assert abs(_order(errs, Ns) + 4.0) < 0.2, errs
    # backward map rotates the other way
    y, _, _ = L.characteristics(v, vg, x, 16, -1)
    assert np.max(np.abs(y - _rotate(x, x0, -omega))) < 1e-5


def test_euler_is_first_order_on_rigid_rotation():
    vg = L.Grid((20, 20))
    x0 = np.array([0.5, 0.5])
    v = _vel_from(_rotation(2, 1.0, x0), vg, 1)
    x = x0[:, None] + np.random.default_rng(4).uniform(-0.2, 0.2, size=(2, 20))
    Ns = np.array([16, 32, 64, 128])
    errs = [np.max(np.abs(L.euler_characteristics(v, vg, x, int(N), 1) - _rotate(x, x0, 1.0))) for N in Ns]
    assert abs(_order(errs, Ns) + 1.0) < 0.15


def test_printed_third_stage_would_be_first_order():
    """Reading of Alg. 1's third stage: with y3 = y + dt/2 v3 as printed, RK4
    loses its order; the standard y3 = y + dt v3 keeps fourth order."""
    vg = L.Grid((20, 20))
    x0 = np.array([0.5, 0.5])
    v = _vel_from(_rotation(2, 2.0, x0), vg, 1)
    x = x0[:, None] + np.random.default_rng(5).uniform(-0.2, 0.2, size=(2, 20))

    def printed(N):
        dt = 1.0 / N
        y = x.copy()
        for k in range(N):
            t = k * dt
            v1 = L.velocity(v, vg, y, t)
            v2 = L.velocity(v, vg, y + dt / 2 * v1, t + dt / 2)
            v3 = L.velocity(v, vg, y + dt / 2 * v2, t + dt / 2)
            v4 = L.velocity(v, vg, y + dt / 2 * v3, t + dt)
            y = y + dt / 6 * (v1 + 2 * v2 + 2 * v3 + v4)
        return y

    Ns = np.array([8, 16, 32, 64])
    errs = [np.max(np.abs(printed(int(N)) - _rotate(x, x0, 2.0))) for N in Ns]
    assert _order(errs, Ns) > -1.5


@pytest.mark.parametrize("direction", [-1, 1])
def test_time_linear_velocity_exact(direction):
    """v(x, t) = a + b t, uniform in space, on 3 time nodes: linear time
    interpolation and RK4 are exact; the displacement is the time integral."""
    d = 2
    vg = L.Grid((10, 10))
    a = np.array([0.05, -0.02])
    b = np.array([-0.04, 0.06])
    v = _vel_from(lambda x, t: [np.full_like(x[0], a[c] + b[c] * t) for c in range(d)], vg, 3)
    x = np.random.default_rng(6).uniform(0.35, 0.65, size=(d, 30))
    y, _, _ = L.characteristics(v, vg, x, 3, direction)
    np.testing.assert_allclose(y, x + direction * (a + b / 2)[:, None], atol=1e-14)


def test_forward_backward_compose_to_identity():
    """y(v, y(v, x, 0, 1), 1, 0) = x (Sec. 2), to RK4 accuracy, for a linear v."""
    vg = L.Grid((16, 16))
    x0 = np.array([0.5, 0.5])
    v = _vel_from(_rotation(2, 1.5, x0), vg, 1)
    x = x0[:, None] + np.random.default_rng(7).uniform(-0.2, 0.2, size=(2, 30))
    errs = []
    for N in (4, 8, 16):
        y1, _, _ = L.characteristics(v, vg, x, N, +1)
        back, _, _ = L.characteristics(v, vg, y1, N, -1)
        errs.append(np.max(np.abs(back - x)))
    # at least fourth order (the round trip can cancel further)
    assert errs[-1] < 1e-6 and _order(errs, [4, 8, 16]) < -3.8


def test_continuity_conserves_mass():
    """Discrete mass preservation of the PIC push-forward (Sec. 3.1)."""
    ig = L.Grid((32, 32))
    vg = L.Grid((16, 16))
    T = synth.gaussian_blobs(synth.centres(synth.GridSpec((32, 32), (0, 0), (1, 1))),
                             [(1.0, 0.08, (0.5, 0.5)), (0.5, 0.05, (0.4, 0.6))])
    T[:4, :] = T[-4:, :] = T[:, :4] = T[:, -4:] = 0.0   # no mass near the edge, none leaves
    v = synth.random_velocity(synth.GridSpec((16, 16), (0, 0), (1, 1)), 3, 0.1, 9)
    u1, _ = L.final_state("continuity", v, vg, T, ig, 6)
    assert abs(u1.sum() - T.sum()) <= 1e-12 * T.sum()


def test_transport_and_continuity_are_adjoint_for_fixed_points():
    """<F(y) T, R> = <T, P(y) R>: continuity mirrors transport (Sec. 3.1)."""
    ig = L.Grid((12, 10))
    rng = np.random.default_rng(10)
    y = rng.uniform(-0.1, 1.1, size=(2, ig.size))
    T = rng.normal(size=ig.size)
    R = rng.normal(size=ig.shape)
    lhs = np.sum(L.scatter(T, ig, y) * R)
    rhs = np.sum(T * L.interpolate(R, ig, y))
    assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))


@pytest.mark.parametrize("d", [2, 3])
def test_jacobian_determinant_of_affine_maps(d):
    """Finite differences are exact on affine maps: det grad (A x + b) = det A,
    also at the one-sided ends; the identity has determinant 1."""
    g = L.Grid((7, 6, 5)[:d], hi=(1.0, 1.4, 0.8)[:d])
    x = L.cell_centres(g)
    A = np.eye(d) + 0.3 * np.random.default_rng(3).normal(size=(d, d))
    y = A @ x + 0.2
    np.testing.assert_allclose(L.jacobian_determinant(y, g), np.linalg.det(A), rtol=1e-12)
    np.testing.assert_allclose(L.jacobian_determinant(x, g), 1.0, rtol=1e-12)


def test_jacobian_determinant_of_rotation_flow_is_one():
    """A rigid rotation preserves volume: det grad y = 1 up to RK4 error."""
    vg = L.Grid((20, 20))
    x0 = np.array([0.5, 0.5])
    v = _vel_from(_rotation(2, 1.0, x0), vg, 1)
    ig = L.Grid((10, 10), lo=(0.3, 0.3), hi=(0.7, 0.7))
    y, _, _ = L.characteristics(v, vg, L.cell_centres(ig), 16, -1)
    np.testing.assert_allclose(L.jacobian_determinant(y, ig), 1.0, atol=1e-6)
