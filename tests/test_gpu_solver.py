"""lgnk_solve (inexact Gauss-Newton-Krylov with Armijo, Eq. 11) against the
oracle's Gauss-Newton on the 2D transport workload (GN 10 outer / 20 inner)."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import Problem as OP, objective
from oracle.solver import gauss_newton
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(model="transport", K=1):
    from paper_1703_04446_gb300 import lgnk
    ins = synth.make_inputs("2d_transport_64", seed=3)
    wl = ins["workload"]
    prob = lgnk.Problem.from_workload(wl, model=model, time_nodes=K, gamma=1e-4)
    op = OP(L.Grid(wl.image.m), L.Grid(wl.velocity.m), K=K, N=wl.rk4_steps, model=model, reg=wl.regularizer,
            alpha=wl.alpha, gamma=1e-4)
    return lgnk, prob, op, ins


def test_first_gauss_newton_step_matches_oracle():
    """From v = 0 both sides take one GN step (PCG 20, tolerance 0.1, Armijo):
    the objective after it agrees to 1e-4 relative."""
    lgnk, prob, op, ins = _setup()
    ctx = lgnk.Context(prob)
    T, R = (torch.from_numpy(ins[k]).cuda() for k in ("T", "R"))
    v, rep = ctx.solve(T, R, None, max_gn=1, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=0.0)
    vo, repo = gauss_newton(op, ins["T"].astype(np.float64), ins["R"].astype(np.float64),
                            np.zeros(op.vshape), max_gn=1, gtol=0.0, max_pcg=20, pcg_tol=0.1)
    assert abs(rep["J0"] - repo["J0"]) <= 1e-5 * repo["J0"]
    assert abs(rep["J"] - repo["J"]) <= 1e-4 * repo["J"]
    assert rep["gn_iters"] == 1 and rep["pcg_iters"] == repo["pcg_iters"]
    # the returned v is the iterate whose objective was reported
    Jv = objective(op, v.cpu().numpy().astype(np.float64), ins["T"].astype(np.float64),
                   ins["R"].astype(np.float64))[0]
    assert abs(Jv - rep["J"]) <= 1e-4 * rep["J"]


@pytest.mark.parametrize("model,K", [("transport", 1), ("continuity", 2)])
def test_solve_decreases_objective_like_oracle(model, K):
    lgnk, prob, op, ins = _setup(model, K)
    ctx = lgnk.Context(prob)
    T, R = (torch.from_numpy(ins[k]).cuda() for k in ("T", "R"))
    v, rep = ctx.solve(T, R, None, max_gn=10, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=1e-3)
    _, repo = gauss_newton(op, ins["T"].astype(np.float64), ins["R"].astype(np.float64),
                           np.zeros(op.vshape), max_gn=10, gtol=1e-3, max_pcg=20, pcg_tol=0.1)
    assert rep["J"] < 0.5 * rep["J0"]
    assert rep["g"] < rep["g0"]
    # FP32 and FP64 Gauss-Newton paths may separate slowly; the minimum reached agrees
    assert abs(rep["J"] - repo["J"]) <= 2e-2 * repo["J0"]
    assert rep["status_name"] in ("ok", "not converged")


@pytest.mark.parametrize("matvec", [1, 0])
def test_first_gauss_newton_step_with_curvature_regularizer(matvec):
    """With a regularizer other than diffusion the PCG loop ends each product
    with the separate distribution, stencil and inner-product kernels: one GN
    step from v = 0 on the curvature case (three time nodes, a domain whose
    cell widths are not exact in binary), with the assembled J and matrix-free,
    against the oracle's (PCG 20, tolerance 0.1, Armijo).  At v = 0 every end
    point is an image node, where both sides take the derivative of the cell
    to the right."""
    from paper_1703_04446_gb300 import lgnk
    from tests._cases import make_case
    op, gp, a = make_case("2d_transport_ragged_K3")
    ctx = lgnk.Context(lgnk.Problem(**gp))
    T, R = (torch.from_numpy(a[k]).cuda() for k in ("T", "R"))
    _, rep = ctx.solve(T, R, None, max_gn=1, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=0.0, matvec=matvec)
    _, repo = gauss_newton(op, a["T"].astype(np.float64), a["R"].astype(np.float64), np.zeros(op.vshape),
                           max_gn=1, gtol=0.0, max_pcg=20, pcg_tol=0.1)
    assert abs(rep["J0"] - repo["J0"]) <= 1e-5 * repo["J0"]
    assert abs(rep["g0"] - repo["g0"]) <= 1e-5 * repo["g0"]
    assert abs(rep["J"] - repo["J"]) <= 1e-4 * repo["J"]
    assert rep["gn_iters"] == 1 and rep["pcg_iters"] == repo["pcg_iters"]


def test_nonfinite_input_is_reported():
    lgnk, prob, op, ins = _setup()
    ctx = lgnk.Context(prob)
    T = torch.from_numpy(ins["T"]).cuda()
    T[3, 4] = float("nan")
    R = torch.from_numpy(ins["R"]).cuda()
    with pytest.raises(lgnk.LgnkError) as e:
        ctx.objective(torch.zeros(prob.velocity_shape, device="cuda"), T, R)
    assert e.value.status == 4


@pytest.mark.parametrize("matvec", [0, 1])
def test_device_loop_and_direct_launches_agree(matvec):
    """The PCG loop as a device-side CUDA graph (the default) against direct
    launches with a host read per iteration (the path taken while the
    tracing kernels are profiled): the same iterations and the same minimum,
    up to the order of float atomics in the gradient scatter."""
    lgnk, prob, op, ins = _setup()
    ctx = lgnk.Context(prob)
    T, R = (torch.from_numpy(ins[k]).cuda() for k in ("T", "R"))
    v_g, rep_g = ctx.solve(T, R, None, max_gn=6, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=1e-3, matvec=matvec)
    ctx.profile(True)
    v_d, rep_d = ctx.solve(T, R, None, max_gn=6, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=1e-3, matvec=matvec)
    ms, traced, launches = ctx.profile_read()
    ctx.profile(False)
    assert traced > 0 and launches > traced
    assert rep_d["gn_iters"] == rep_g["gn_iters"]
    assert abs(rep_d["pcg_iters"] - rep_g["pcg_iters"]) <= 2
    assert abs(rep_d["J"] - rep_g["J"]) <= 1e-4 * rep_g["J"]
    assert float(torch.linalg.norm(v_d - v_g) / torch.linalg.norm(v_g)) <= 1e-3
