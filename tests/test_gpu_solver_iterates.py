"""Gauss-Newton iterates of lgnk_solve against the oracle, iterate by iterate.

The GN problem is non-convex and the FP32 GPU path and the FP64 oracle may
drift apart over many steps, so each GPU iterate is handed to the oracle and
both take the next step from that same point: the objective and gradient
norm at the iterate, the step, and the objective after the step are compared
(the GPU solve runs one GN iteration per call from the iterate it is given).
Tolerances: objectives and gradient norms 1e-5 at a given iterate, steps 0.1
(the test docstrings say why)."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import Problem as OP, gradient, hessvec, objective
from oracle.solver import apply_preconditioner, armijo, gauss_newton, pcg
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(name, seed=0):
    from paper_1703_04446_gb300 import lgnk
    ins = synth.make_inputs(name, seed=seed)
    wl = ins["workload"]
    prob = lgnk.Problem.from_workload(wl)
    op = OP(L.Grid(wl.image.m, wl.image.lo, wl.image.hi), L.Grid(wl.velocity.m, wl.velocity.lo, wl.velocity.hi),
            K=wl.time_nodes, N=wl.rk4_steps, model=wl.model, reg=wl.regularizer, alpha=wl.alpha, gamma=wl.gamma,
            mu=wl.extra.get("mu", 1.0), lam=wl.extra.get("lam", 0.0))
    ctx = lgnk.Context(prob)
    T64, R64 = ins["T"].astype(np.float64), ins["R"].astype(np.float64)
    tT, tR = (torch.from_numpy(ins[k]).cuda() for k in ("T", "R"))
    return ctx, op, T64, R64, tT, tR


@pytest.mark.parametrize("matvec", [1, 0])
def test_transport_64_iterates_follow_the_oracle(matvec):
    """2D intensity-preserving workload (64^2, 10 GN / 20 PCG): every GN step
    from the GPU's own iterate, with the assembled J and matrix-free.  The
    step is compared twice: against the oracle's step after the same number
    of CG iterations (when the two residual norms cross the 0.1 threshold one
    iteration apart, the oracle is run for the GPU's count), to 0.1 in the
    plain norm and in the norm of the Gauss-Newton Hessian H, and through
    the oracle's operator, where it must meet the PCG stopping test
    |H x + g| <= 0.1 |g| (5% slack for the FP32 recurrence) unless PCG hit
    its cap.  Why 0.1 for the step: CG amplifies rounding in its matrix
    products; on this workload the oracle's own FP64 step moves by up to 3e-2
    (plain norm) and 4.6e-2 (H norm) when each of its Hessian products
    carries a random relative error of 1e-6, the size of FP32 rounding in the
    GPU products.  The objective after the step is checked twice: the GPU's
    value against the oracle's objective at the GPU's new iterate (1e-5), and
    that objective against the one the oracle reaches with its own step,
    whose difference must stay within what the step difference e explains to
    second order, |g1 . e| + e^T H e (g1 the oracle's gradient after its own
    step; the factor 2 on the quadratic term covers the curvature that the
    Gauss-Newton H leaves out), plus 1e-5 of J."""
    ctx, op, T64, R64, tT, tR = _setup("2d_transport_64")
    v = torch.zeros(op.vshape, device="cuda")
    g_first = None
    rows = []
    for k in range(10):
        v_next, rep = ctx.solve(tT, tR, v, max_gn=1, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=0.0, matvec=matvec)
        v64 = v.cpu().numpy().astype(np.float64)
        vo, repo = gauss_newton(op, T64, R64, v64, max_gn=1, gtol=0.0, max_pcg=20, pcg_tol=0.1)
        h = repo["history"][0]
        g = gradient(op, v64, T64, R64)
        step = v_next.cpu().numpy().astype(np.float64) - v64
        x = step / rep["last_mu"] if rep["last_mu"] > 0 else step
        res = float(np.linalg.norm(hessvec(op, v64, T64, x) + g) / np.linalg.norm(g))
        ref_step, J_after, mu_o = h["mu"] * h["dv"], repo["J"], h["mu"]
        if rep["pcg_iters"] != h["pcg"]:
            # the two residual norms crossed the 0.1 threshold one iteration
            # apart: the oracle's step after the GPU's number of CG iterations
            dv, _, _ = pcg(lambda q: hessvec(op, v64, T64, q), -g, lambda r: apply_preconditioner(op, r), tol=0.0,
                           maxit=rep["pcg_iters"])
            mu_o, J_after = armijo(lambda w: objective(op, w, T64, R64)[0], v64, h["J"], g, dv)
            ref_step = mu_o * dv
        e = step - ref_step
        eHe = float(np.sum(e * hessvec(op, v64, T64, e)))
        stepH = float(np.sqrt(eHe / np.sum(ref_step * hessvec(op, v64, T64, ref_step))))
        J_gpu_point = objective(op, v64 + step, T64, R64)[0]
        g1 = gradient(op, v64 + ref_step, T64, R64)
        rows.append(dict(k=k, J0=abs(rep["J0"] - h["J"]) / h["J"], g0=abs(rep["g0"] - h["g"]) / h["g"],
                         pcg=(rep["pcg_iters"], h["pcg"]), mu=(rep["last_mu"], mu_o),
                         step=float(np.linalg.norm(e) / np.linalg.norm(ref_step)), stepH=stepH,
                         res=res, J=abs(rep["J"] - J_gpu_point) / J_gpu_point,
                         dJ=abs(J_gpu_point - J_after), dJ_bound=abs(float(np.sum(g1 * e))) + eHe + 1e-5 * J_after))
        g_first = g_first or h["g"]
        v = v_next
        if h["g"] <= 1e-3 * g_first:
            break
    print("\n".join(str(r) for r in rows))
    for r in rows:
        assert r["J0"] <= 1e-5 and r["g0"] <= 1e-5, r
        assert abs(r["pcg"][0] - r["pcg"][1]) <= 1, r
        assert r["stepH"] <= 1e-1 and r["step"] <= 1e-1, r
        if r["pcg"][0] < 20:
            assert r["res"] <= 0.1 * 1.05, r
        assert r["mu"][0] == r["mu"][1], r
        assert r["J"] <= 1e-5, r
        assert r["dJ"] <= r["dJ_bound"], r


def test_transport_64_final_objective_of_independent_solves():
    """Both solvers from v = 0 on their own (10 GN / 20 PCG, stop at a 1e-3
    gradient-norm drop): the final objectives agree to 1e-4."""
    ctx, op, T64, R64, tT, tR = _setup("2d_transport_64")
    _, rep = ctx.solve(tT, tR, None, max_gn=10, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=1e-3)
    _, repo = gauss_newton(op, T64, R64, np.zeros(op.vshape), max_gn=10, gtol=1e-3, max_pcg=20, pcg_tol=0.1)
    assert abs(rep["J0"] - repo["J0"]) <= 1e-5 * repo["J0"]
    assert abs(rep["J"] - repo["J"]) <= 1e-4 * repo["J"]


def test_continuity_256_iterates_under_the_oracle():
    """2D mass-preserving workload (256^2, 5 time nodes, N = 16, elastic):
    three GN steps from the GPU's iterates.  At each iterate the oracle's J and
    |g| match; the GPU's step is an inexact Newton step of the oracle's own
    system (|H x + g| <= 0.1 |g| unless PCG hit its cap, and x a descent
    direction); the objective after the step matches the oracle's objective at
    the GPU's new iterate.  (The oracle's PCG itself takes minutes here.)"""
    ctx, op, T64, R64, tT, tR = _setup("2d_continuity_256")
    v = torch.zeros(op.vshape, device="cuda")
    for k in range(3):
        v_next, rep = ctx.solve(tT, tR, v, max_gn=1, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=0.0)
        v64 = v.cpu().numpy().astype(np.float64)
        J = objective(op, v64, T64, R64)[0]
        g = gradient(op, v64, T64, R64)
        gn = float(np.linalg.norm(g))
        assert abs(rep["J0"] - J) <= 1e-5 * J, k
        # |g| to 5e-5: where a stage position lies within ~1e-7 cells of a cell
        # face, FP32 and FP64 take different cells (the kink of the linear
        # interpolant); with 65536 particles, 64 stages and the adjoint sweep a
        # handful of such particles per gradient is expected, and one run in
        # about ten saw 2e-5 after two GN steps (otherwise <= 2e-6)
        assert abs(rep["g0"] - gn) <= 5e-5 * gn, k
        assert rep["last_mu"] > 0.0, k
        vn64 = v_next.cpu().numpy().astype(np.float64)
        x = (vn64 - v64) / rep["last_mu"]
        res = np.linalg.norm(hessvec(op, v64, T64, x) + g)
        if rep["pcg_iters"] < 20:
            assert res <= 0.1 * gn * 1.05, k
        assert res < gn and float(np.sum(g * x)) < 0.0, k
        Jn = objective(op, vn64, T64, R64)[0]
        assert abs(rep["J"] - Jn) <= 1e-5 * Jn, k
        assert rep["J"] < rep["J0"], k
        v = v_next


def test_line_search_forced_to_fail_keeps_the_iterate():
    """A sufficient-decrease constant above one (c = 2) asks for more than the
    quadratic model gives, so every trial fails: the solve reports
    LGNK_LS_FAILED after one GN iteration and returns the iterate it was given,
    bit for bit, as the oracle's Gauss-Newton does."""
    ctx, op, T64, R64, tT, tR = _setup("2d_transport_64")
    v0 = torch.from_numpy(synth.random_velocity(synth.WORKLOADS["2d_transport_64"].velocity, 1, 0.01, 4)
                          .astype(np.float32)).cuda()
    v, rep = ctx.solve(tT, tR, v0, max_gn=3, max_pcg=20, pcg_rtol=0.1, gn_grad_rtol=1e-3, armijo_c=2.0)
    assert rep["status"] == 6 and rep["status_name"] == "line search failed"
    assert rep["gn_iters"] == 1 and rep["last_mu"] == 0.0
    assert torch.equal(v, v0)
    assert rep["J"] == rep["J0"]
    _, repo = gauss_newton(op, T64, R64, v0.cpu().numpy().astype(np.float64), max_gn=3, gtol=1e-3, max_pcg=20,
                           pcg_tol=0.1, armijo_c=2.0)
    assert repo["status"] == "line search failed" and repo["iters"] == 1
