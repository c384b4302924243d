"""Pins of the oracle's derivatives (Alg. 1 derivative recursion, Sec. 3.2):
J = d_v u1 against central differences of the forward map, J^T against J by
the adjoint identity, and the objective gradient against differences of J(v)."""
import numpy as np
import pytest

from oracle import lagrangian as L
from oracle.objective import Problem, gradient, objective, reg_operator, reg_value
from paper_1703_04446_gb300 import synth


def _case(d, K, model, seed=0):
    ig = L.Grid((10, 9, 8)[:d])
    vg = L.Grid((6, 5, 4)[:d])
    gs = synth.GridSpec(ig.m, tuple(ig.lo), tuple(ig.hi))
    rng = np.random.default_rng(seed)
    T = synth.gaussian_blobs(synth.centres(gs), [(1.0, 0.2, tuple(rng.uniform(0.35, 0.65, d))),
                                                 (0.6, 0.12, tuple(rng.uniform(0.3, 0.7, d)))])
    vs = synth.GridSpec(vg.m, tuple(vg.lo), tuple(vg.hi))
    v = synth.random_velocity(vs, K, 0.15, seed + 1)
    dv = synth.random_velocity(vs, K, 0.1, seed + 2) + 0.02 * rng.normal(size=v.shape)
    return ig, vg, T, v, dv


CASES = [(2, 1, "transport"), (2, 3, "transport"), (2, 1, "continuity"), (2, 2, "continuity"),
         (3, 1, "transport"), (3, 2, "continuity")]


@pytest.mark.parametrize("d,K,model", CASES)
def test_jvp_matches_central_difference(d, K, model):
    ig, vg, T, v, dv = _case(d, K, model)
    N = 3
    eps = 1e-7
    up, _ = L.final_state(model, v + eps * dv, vg, T, ig, N)
    dn, _ = L.final_state(model, v - eps * dv, vg, T, ig, N)
    fd = (up - dn) / (2 * eps)
    J = L.jvp(model, v, vg, T, ig, N, dv)
    assert np.linalg.norm(J - fd) <= 1e-6 * np.linalg.norm(fd)


@pytest.mark.parametrize("d,K,model", CASES)
def test_jtvp_is_adjoint_of_jvp(d, K, model):
    ig, vg, T, v, dv = _case(d, K, model, seed=3)
    N = 3
    r = np.random.default_rng(11).normal(size=ig.shape)
    lhs = np.sum(L.jvp(model, v, vg, T, ig, N, dv) * r)
    rhs = np.sum(dv * L.jtvp(model, v, vg, T, ig, N, r))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_characteristic_tangent_matches_difference_of_end_points():
    """(d_v y) dv from Alg. 1 against central differences of y(v) itself."""
    ig, vg, T, v, dv = _case(2, 3, "transport", seed=5)
    x = L.cell_centres(ig)
    eps = 1e-7
    _, dy, _ = L.characteristics(v, vg, x, 4, -1, dv=dv)
    yp, _, _ = L.characteristics(v + eps * dv, vg, x, 4, -1)
    ym, _, _ = L.characteristics(v - eps * dv, vg, x, 4, -1)
    np.testing.assert_allclose(dy, (yp - ym) / (2 * eps), rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("reg", ["diffusion", "curvature", "elastic"])
@pytest.mark.parametrize("model", ["transport", "continuity"])
def test_gradient_matches_difference_of_objective(reg, model):
    ig, vg, T, v, dv = _case(2, 2, model, seed=7)
    gs = synth.GridSpec(ig.m, tuple(ig.lo), tuple(ig.hi))
    R = synth.gaussian_blobs(synth.centres(gs), [(0.9, 0.18, (0.52, 0.47))])
    prob = Problem(ig, vg, K=2, N=3, model=model, reg=reg, alpha=0.05, gamma=0.0, mu=1.0, lam=0.5)
    g = gradient(prob, v, T, R)
    eps = 1e-6
    fd = (objective(prob, v + eps * dv, T, R)[0] - objective(prob, v - eps * dv, T, R)[0]) / (2 * eps)
    assert abs(np.sum(g * dv) - fd) <= 1e-6 * max(abs(fd), 1e-8)


@pytest.mark.parametrize("reg", ["diffusion", "curvature", "elastic"])
def test_regularizer_is_quadratic_form_of_its_operator(reg):
    """S(v) = 1/2 v^T (dt h^d A) v and A is symmetric."""
    _, vg, _, v, dv = _case(3, 2, "transport", seed=9)
    prob = Problem(L.Grid((10, 9, 8)), vg, K=2, N=2, reg=reg, alpha=1.0, mu=0.7, lam=0.4)
    assert abs(reg_value(prob, v) - 0.5 * np.sum(v * reg_operator(prob, v))) <= 1e-12 * reg_value(prob, v)
    assert abs(np.sum(dv * reg_operator(prob, v)) - np.sum(v * reg_operator(prob, dv))) <= 1e-10
