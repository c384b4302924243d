"""Pins of the oracle's multilevel continuation (Sec. 3.2): restriction by
averaging and prolongation by the interpolation of Sec. 3.1 against closed
forms, and a coarse-to-fine solve that lowers the objective on every level."""
import numpy as np
import pytest

from oracle import lagrangian as L
from oracle.objective import Problem
from oracle.solver import coarse_grid, level_problems, multilevel_gauss_newton, prolong_velocity, restrict_image
from paper_1703_04446_gb300 import synth


@pytest.mark.parametrize("d", [2, 3])
def test_restriction_of_affine_field_is_affine_and_keeps_the_integral(d):
    g = L.Grid((8, 6, 4)[:d], lo=(-0.5, 0.0, 0.2)[:d], hi=(1.5, 1.2, 1.0)[:d])
    cg = coarse_grid(g)
    a = np.array([0.3, -1.2, 0.7][:d])
    F = (0.4 + a @ L.cell_centres(g)).reshape(g.shape)
    Fc = restrict_image(F, g)
    np.testing.assert_allclose(Fc.ravel(), 0.4 + a @ L.cell_centres(cg), atol=1e-12)
    rnd = np.random.default_rng(0).normal(size=g.shape)
    assert abs(restrict_image(rnd, g).sum() * cg.cell_volume - rnd.sum() * g.cell_volume) < 1e-12


def test_prolongation_of_affine_field_is_exact_inside():
    cg = L.Grid((6, 5))
    fg = L.Grid((12, 10))
    a = np.array([0.8, -0.3])
    vc = np.zeros((2, 2) + cg.shape)
    for c in range(2):
        vc[:, c] = (0.1 * (c + 1) + a @ L.cell_centres(cg)).reshape(cg.shape)
    vf = prolong_velocity(vc, cg, fg)
    x = L.cell_centres(fg)
    inside = np.all([(x[k] > cg.lo[k] + 0.5 * cg.h[k]) & (x[k] < cg.hi[k] - 0.5 * cg.h[k]) for k in range(2)], axis=0)
    for c in range(2):
        exact = 0.1 * (c + 1) + a @ x
        np.testing.assert_allclose(vf[1, c].ravel()[inside], exact[inside], atol=1e-12)


def test_level_problems_halve_grids():
    p = Problem(L.Grid((32, 16)), L.Grid((16, 8)), K=2, N=3, alpha=0.1)
    ps = level_problems(p, 3)
    assert [q.igrid.m for q in ps] == [(8, 4), (16, 8), (32, 16)]
    assert [q.vgrid.m for q in ps] == [(4, 2), (8, 4), (16, 8)]
    with pytest.raises(ValueError):
        level_problems(Problem(L.Grid((6, 6)), L.Grid((3, 3)), K=1, N=2), 3)


def test_multilevel_solve_lowers_objective_on_each_level():
    ig, vg = L.Grid((32, 32)), L.Grid((16, 16))
    gs = synth.GridSpec(ig.m, (0.0, 0.0), (1.0, 1.0))
    blobs = [(1.0, 0.15, (0.45, 0.5)), (0.6, 0.08, (0.6, 0.4))]
    T = synth.gaussian_blobs(synth.centres(gs), blobs)
    R = synth.gaussian_blobs([c - 0.04 for c in synth.centres(gs)], blobs)
    prob = Problem(ig, vg, K=1, N=4, alpha=1e-2, gamma=0.0)
    v, reps = multilevel_gauss_newton(prob, T, R, 3, max_gn=6, gtol=1e-3, max_pcg=20, pcg_tol=0.1)
    assert len(reps) == 3 and v.shape == prob.vshape
    for rep in reps:
        assert rep["J"] <= rep["J0"]
    # the finest level starts from the prolonged coarse solution, already well below J(0)
    from oracle.objective import objective
    J_zero = objective(prob, np.zeros(prob.vshape), T, R)[0]
    assert reps[-1]["J0"] < 0.7 * J_zero


def test_level_problems_keep_the_particle_width_and_weights():
    """The coarse levels solve the same continuous problem: the PIC half-width
    (in domain units), K, N, model, regularizer and weights are the finest
    level's."""
    p = Problem(L.Grid((32, 32)), L.Grid((16, 16)), K=3, N=5, model="continuity", reg="elastic", alpha=0.2,
                gamma=1e-3, mu=0.7, lam=0.4, delta=0.05)
    for q in level_problems(p, 3):
        assert (q.K, q.N, q.model, q.reg, q.alpha, q.gamma, q.mu, q.lam, q.delta) == \
            (3, 5, "continuity", "elastic", 0.2, 1e-3, 0.7, 0.4, 0.05)
