"""Multilevel continuation on the GPU (restriction, prolongation, coarse-to-fine
Gauss-Newton) against the oracle's multilevel driver (Sec. 3.2)."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import Problem as OP, objective
from oracle.solver import coarse_grid, multilevel_gauss_newton, prolong_velocity, restrict_image
from paper_1703_04446_gb300 import synth
from tests._cases import rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [(16, 12), (8, 6, 10)])
def test_restriction_matches_oracle(m):
    from paper_1703_04446_gb300 import lgnk
    d = len(m)
    lo, hi = (-0.2, 0.0, 0.1)[:d], (1.0, 1.5, 0.9)[:d]
    F = np.random.default_rng(0).normal(size=tuple(reversed(m))).astype(np.float32)
    C = lgnk.lgnk_restrict_image(torch.from_numpy(F).cuda(), m, lo, hi)
    ref = restrict_image(F.astype(np.float64), L.Grid(m, lo, hi))
    assert rel(C.cpu().numpy(), ref) <= 1e-6


@pytest.mark.parametrize("cm,K", [((6, 5), 2), ((4, 5, 3), 1)])
def test_prolongation_matches_oracle(cm, K):
    from paper_1703_04446_gb300 import lgnk
    d = len(cm)
    fm = tuple(2 * a for a in cm)
    vc = np.random.default_rng(1).normal(size=(K, d) + tuple(reversed(cm))).astype(np.float32)
    vf = lgnk.lgnk_prolong_velocity(torch.from_numpy(vc).cuda(), cm, fm)
    ref = prolong_velocity(vc.astype(np.float64), L.Grid(cm), L.Grid(fm))
    assert rel(vf.cpu().numpy(), ref) <= 1e-6


def test_multilevel_solve_matches_oracle():
    from paper_1703_04446_gb300 import lgnk
    ig, vg = L.Grid((32, 32)), L.Grid((16, 16))
    gs = synth.GridSpec(ig.m, (0.0, 0.0), (1.0, 1.0))
    blobs = [(1.0, 0.15, (0.45, 0.5)), (0.6, 0.08, (0.6, 0.4))]
    T = synth.gaussian_blobs(synth.centres(gs), blobs).astype(np.float32)
    R = synth.gaussian_blobs([c - 0.04 for c in synth.centres(gs)], blobs).astype(np.float32)
    prob = OP(ig, vg, K=1, N=4, alpha=1e-2, gamma=0.0)
    vo, reps_o = multilevel_gauss_newton(prob, T.astype(np.float64), R.astype(np.float64), 3,
                                         max_gn=6, gtol=1e-3, max_pcg=20, pcg_tol=0.1)
    gp = lgnk.Problem(image_m=(32, 32), velocity_m=(16, 16), time_nodes=1, rk4_steps=4, alpha=1e-2)
    v, reps = lgnk.lgnk_solve_multilevel(gp, torch.from_numpy(T).cuda(), torch.from_numpy(R).cuda(), 3,
                                         max_gn=6, gn_grad_rtol=1e-3, max_pcg=20, pcg_rtol=0.1)
    assert len(reps) == 3
    # the coarsest level starts at v = 0 on the restricted images: identical objective
    assert abs(reps[0]["J0"] - reps_o[0]["J0"]) <= 1e-5 * reps_o[0]["J0"]
    for r, ro in zip(reps, reps_o):
        assert r["J"] <= r["J0"]
        assert abs(r["J"] - ro["J"]) <= 2e-2 * ro["J0"]
    # the returned fine velocity is the iterate of the finest report
    Jv = objective(prob, v.cpu().numpy().astype(np.float64), T.astype(np.float64), R.astype(np.float64))[0]
    assert abs(Jv - reps[-1]["J"]) <= 1e-4 * reps[-1]["J"]


def test_multilevel_rejects_indivisible_grids():
    from paper_1703_04446_gb300 import lgnk
    gp = lgnk.Problem(image_m=(30, 32), velocity_m=(15, 16), time_nodes=1, rk4_steps=2)
    T = torch.zeros(gp.image_shape, device="cuda")
    with pytest.raises(lgnk.LgnkError):
        lgnk.lgnk_solve_multilevel(gp, T, T.clone(), 3)
