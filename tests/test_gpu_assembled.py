"""The assembled J (lgnk_assemble and the *_assembled products) against the
oracle's J, J^T and Gauss-Newton products on every transport parity case, and
against the matrix-free kernels at the full 128^3 size; capacity overflow,
the solver's fallback and the error paths."""
import functools

import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import Problem as OProblem, hessvec
from paper_1703_04446_gb300 import synth
from tests._cases import CASES, make_case, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5
TRANSPORT = [n for n in CASES if CASES[n][6] == "transport"]


@functools.lru_cache(maxsize=None)
def _case(name):
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case(name)
    ctx = lgnk.Context(lgnk.Problem(**gp))
    t = {k: torch.from_numpy(v).cuda() for k, v in a.items()}
    ctx.assemble(t["v"], t["T"])
    f64 = {k: v.astype(np.float64) for k, v in a.items()}
    ref = dict(jvp=L.jvp(op.model, f64["v"], op.vgrid, f64["T"], op.igrid, op.N, f64["dv"]),
               jtvp=L.jtvp(op.model, f64["v"], op.vgrid, f64["T"], op.igrid, op.N, f64["r"]),
               hess=hessvec(op, f64["v"], f64["T"], f64["dv"]))
    return ctx, t, ref


def _np(x):
    return x.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", TRANSPORT)
def test_assembled_jvp(name):
    ctx, t, ref = _case(name)
    assert rel(_np(ctx.jvp_assembled(t["dv"])), ref["jvp"]) <= TOL


@pytest.mark.parametrize("name", TRANSPORT)
def test_assembled_jtvp(name):
    ctx, t, ref = _case(name)
    assert rel(_np(ctx.jtvp_assembled(t["r"])), ref["jtvp"]) <= TOL


@pytest.mark.parametrize("name", TRANSPORT)
def test_assembled_hessvec(name):
    ctx, t, ref = _case(name)
    got = _np(ctx.hessvec_assembled(t["dv"]))
    assert rel(got, ref["hess"]) <= TOL
    # the matrix-free kernel at the same point agrees to FP32 summation order
    mf = _np(ctx.hessvec(t["v"], t["T"], t["dv"]))
    assert rel(got, mf) <= 2e-6


def test_assembled_products_at_full_size():
    """128^3 image, 64^3 stationary velocity, N = 8: the configuration of the
    throughput benchmark; the assembled products against the matrix-free ones,
    and the adjoint identity of the assembled pair."""
    from paper_1703_04446_gb300 import lgnk
    ins = synth.make_inputs("3d_transport_128", seed=0)
    wl = ins["workload"]
    ctx = lgnk.Context(lgnk.Problem.from_workload(wl, gamma=1e-4))
    h = min(wl.image.h)
    dv = synth.random_velocity(wl.velocity, 1, 2 * h, 5).astype(np.float32)
    r = np.random.default_rng(4).normal(size=ins["T"].shape).astype(np.float32)
    v, T, dv, r = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (ins["v0"], ins["T"], dv, r))
    blocks = ctx.assemble(v, T)
    M = T.numel()
    assert M <= blocks <= 16 * M
    assert rel(_np(ctx.hessvec_assembled(dv)), _np(ctx.hessvec(v, T, dv))) <= 1e-5
    assert rel(_np(ctx.jvp_assembled(dv)), _np(ctx.jvp(v, T, dv))) <= 1e-5
    assert rel(_np(ctx.jtvp_assembled(r)), _np(ctx.jtvp(v, T, r))) <= 1e-5
    lhs = float((ctx.jvp_assembled(dv).double() * r.double()).sum())
    rhs = float((ctx.jtvp_assembled(r).double() * dv.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))
    ctx.close()
    torch.cuda.empty_cache()


def _overflow_case():
    """Many time slices and a large velocity: every characteristic meets more
    (slice, cell) blocks than a row holds."""
    from paper_1703_04446_gb300 import lgnk
    im, vm = (16, 16, 16), (8, 8, 8)
    prob = lgnk.Problem(image_m=im, velocity_m=vm, time_nodes=3, rk4_steps=12, model="transport")
    g = synth.GridSpec(vm, (0.0,) * 3, (1.0,) * 3)
    v = synth.random_velocity(g, 3, 0.3, 7).astype(np.float32)
    ig = synth.GridSpec(im, (0.0,) * 3, (1.0,) * 3)
    T = synth.gaussian_blobs(synth.centres(ig), [(1.0, 0.2, (0.5, 0.5, 0.5))]).astype(np.float32)
    R = synth.gaussian_blobs(synth.centres(ig), [(1.0, 0.2, (0.55, 0.5, 0.5))]).astype(np.float32)
    return lgnk.Context(prob), torch.from_numpy(v).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(R).cuda()


def test_capacity_overflow_is_reported_and_the_solver_falls_back():
    from paper_1703_04446_gb300 import lgnk
    ctx, v, T, R = _overflow_case()
    with pytest.raises(lgnk.LgnkError) as e:
        ctx.assemble(v, T)
    assert e.value.status == 8
    with pytest.raises(lgnk.LgnkError):
        ctx.hessvec_assembled(v)            # no valid J after a failed assembly
    _, rep_mf = ctx.solve(T, R, v, max_gn=3, matvec=0)
    _, rep_as = ctx.solve(T, R, v, max_gn=3, matvec=1)
    assert rep_as["assembled_gn"] == 0
    assert rep_as["gn_iters"] == rep_mf["gn_iters"]
    # the same solve twice: only the order of float atomics in the gradient scatter differs
    assert abs(rep_as["J"] - rep_mf["J"]) <= 1e-4 * abs(rep_mf["J"])


def test_matrix_free_product_where_rows_overflow():
    """Where the rows of J are too long to assemble (3 time nodes, 12 steps,
    large displacements), the solver falls back to the matrix-free product:
    it matches the oracle's Gauss-Newton product on that case."""
    from paper_1703_04446_gb300 import lgnk
    ctx, v, T, R = _overflow_case()
    with pytest.raises(lgnk.LgnkError) as e:
        ctx.assemble(v, T)               # the rows do not fit: the overflow path is taken
    assert e.value.status == 8
    im, vm = (16, 16, 16), (8, 8, 8)
    op = OProblem(L.Grid(im), L.Grid(vm), K=3, N=12, model="transport")
    g = synth.GridSpec(vm, (0.0,) * 3, (1.0,) * 3)
    dv = synth.random_velocity(g, 3, 0.05, 8).astype(np.float32)
    ref = hessvec(op, _np(v), _np(T), dv.astype(np.float64))
    got = _np(ctx.hessvec(v, T, torch.from_numpy(dv).cuda()))
    assert rel(got, ref) <= TOL


def test_solver_with_assembled_matvec_matches_matrix_free():
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case("2d_transport_64")
    ctx = lgnk.Context(lgnk.Problem(**gp))
    T, R = (torch.from_numpy(a[k]).cuda() for k in ("T", "R"))
    v_mf, rep_mf = ctx.solve(T, R, None, max_gn=8, matvec=0)
    v_as, rep_as = ctx.solve(T, R, None, max_gn=8)          # the default: assembled
    assert rep_as["assembled_gn"] == rep_as["gn_iters"] > 0
    assert rep_as["gn_iters"] == rep_mf["gn_iters"]
    assert abs(rep_as["J"] - rep_mf["J"]) <= 1e-5 * abs(rep_mf["J"])
    assert rel(_np(v_as), _np(v_mf)) <= 1e-4


def test_errors():
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case("2d_transport_64")
    ctx = lgnk.Context(lgnk.Problem(**gp))
    dv = torch.from_numpy(a["dv"]).cuda()
    with pytest.raises(lgnk.LgnkError, match="no assembled J"):
        ctx.jvp_assembled(dv)
    op, gp, a = make_case("2d_continuity_K5")
    cctx = lgnk.Context(lgnk.Problem(**gp))
    with pytest.raises(lgnk.LgnkError, match="transport model only"):
        cctx.assemble(torch.from_numpy(a["v"]).cuda(), torch.from_numpy(a["T"]).cuda())
