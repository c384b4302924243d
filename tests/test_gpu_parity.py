"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by
element on seeded inputs that span several tiles and ragged tails.

Tolerances (FP32 tracing against FP64): forward state and J / J^T / H
products <= 1e-5 relative L2; objective <= 1e-5 relative (the bar for the
final objective is 1e-4)."""
import functools

import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import gradient, hessvec, objective, reg_operator
from oracle.solver import apply_preconditioner
from paper_1703_04446_gb300 import synth
from tests._cases import CASES, make_case, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5


@functools.lru_cache(maxsize=None)
def _oracle(name):
    op, gp, a = make_case(name)
    f64 = {k: v.astype(np.float64) for k, v in a.items()}
    u1, y = L.final_state(op.model, f64["v"], op.vgrid, f64["T"], op.igrid, op.N, op.delta)
    out = dict(u1=u1, y=y,
               jvp=L.jvp(op.model, f64["v"], op.vgrid, f64["T"], op.igrid, op.N, f64["dv"], op.delta),
               jtvp=L.jtvp(op.model, f64["v"], op.vgrid, f64["T"], op.igrid, op.N, f64["r"], op.delta),
               hess=hessvec(op, f64["v"], f64["T"], f64["dv"]),
               obj=objective(op, f64["v"], f64["T"], f64["R"])[:3],
               grad=gradient(op, f64["v"], f64["T"], f64["R"]),
               prec=apply_preconditioner(op, f64["dv"]))
    return out


@functools.lru_cache(maxsize=None)
def _gpu(name):
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case(name)
    ctx = lgnk.Context(lgnk.Problem(**gp))
    t = {k: torch.from_numpy(v).cuda() for k, v in a.items()}
    return ctx, t


def _np(x):
    return x.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_forward_state(name):
    ctx, t = _gpu(name)
    u1, y = ctx.forward(t["v"], t["T"], return_y=True)
    o = _oracle(name)
    assert rel(_np(u1), o["u1"]) <= TOL
    assert rel(_np(y).reshape(len(ctx.problem.image_m), -1), o["y"]) <= 1e-6


@pytest.mark.parametrize("name", list(CASES))
def test_jvp(name):
    ctx, t = _gpu(name)
    assert rel(_np(ctx.jvp(t["v"], t["T"], t["dv"])), _oracle(name)["jvp"]) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_jtvp(name):
    ctx, t = _gpu(name)
    assert rel(_np(ctx.jtvp(t["v"], t["T"], t["r"])), _oracle(name)["jtvp"]) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_hessvec(name):
    ctx, t = _gpu(name)
    assert rel(_np(ctx.hessvec(t["v"], t["T"], t["dv"])), _oracle(name)["hess"]) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_objective_and_gradient(name):
    ctx, t = _gpu(name)
    J, D, S, g = ctx.objective(t["v"], t["T"], t["R"], grad=True)
    Jo, Do, So = _oracle(name)["obj"]
    assert abs(J - Jo) <= TOL * abs(Jo)
    assert abs(D - Do) <= TOL * abs(Do)
    assert abs(S - So) <= TOL * abs(So)
    assert rel(_np(g), _oracle(name)["grad"]) <= TOL
    # without the gradient: same objective up to FP32 residual/atomic ordering
    J2, D2, S2 = ctx.objective(t["v"], t["T"], t["R"])
    assert abs(J2 - J) <= 1e-6 * abs(J)


@pytest.mark.parametrize("name", list(CASES))
def test_preconditioner(name):
    ctx, t = _gpu(name)
    assert rel(_np(ctx.precond(t["dv"])), _oracle(name)["prec"]) <= TOL


@pytest.mark.parametrize("vm,K", [((130, 20), 2), ((40, 36, 129), 1), ((128, 128), 1), ((64, 64, 64), 1),
                                  ((64, 61, 33), 2), ((37, 64, 16), 1), ((65, 40, 20), 1),
                                  ((64, 61), 2), ((6, 64), 1), ((19, 15), 3)])
def test_preconditioner_axis_lengths(vm, K):
    """Axes of more than 128 cells take the untiled DCT kernel, the others the
    shared-memory tile (128 is the largest tiled length); 3D xy planes of at
    most 64 x 64 cells take the plane kernel (float4 stores when x is a
    multiple of 4, scalar ones otherwise), wider ones the per-axis tiles; 2D
    planes of at most 64 x 64 cells take the whole transform in one kernel."""
    from oracle import lagrangian as Lg
    from oracle.objective import Problem as OProblem
    from paper_1703_04446_gb300 import lgnk
    d = len(vm)
    im = tuple(2 * a for a in vm)
    op = OProblem(Lg.Grid(im), Lg.Grid(vm), K=K, N=2, alpha=1e-2, gamma=1e-3)
    ctx = lgnk.Context(lgnk.Problem(image_m=im, velocity_m=vm, time_nodes=K, rk4_steps=2, alpha=1e-2, gamma=1e-3))
    r = np.random.default_rng(3).normal(size=(K, d) + tuple(reversed(vm))).astype(np.float32)
    got = _np(ctx.precond(torch.from_numpy(r).cuda()))
    assert rel(got, apply_preconditioner(op, r.astype(np.float64))) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_identity_on_gpu(name):
    """<J dv, r> = <dv, J^T r> within FP32 accumulation error."""
    ctx, t = _gpu(name)
    lhs = float(torch.sum(ctx.jvp(t["v"], t["T"], t["dv"]).double() * t["r"].double()))
    rhs = float(torch.sum(ctx.jtvp(t["v"], t["T"], t["r"]).double() * t["dv"].double()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))


def test_dot_accumulates_beyond_fp32():
    """Inner products are summed in FP64 per element: a sum that FP32 alone
    would round is exact, and a random ragged case lands within 1e-12 of
    sum |a_i b_i| from the exactly rounded sum of the exact FP64 products
    (FP32 accumulation misses by about 3e-8 here)."""
    import math
    ctx, t = _gpu("2d_transport_64")
    a = torch.full((1 << 20,), 1.0 + 2.0 ** -20, device="cuda")
    b = torch.full((1 << 20,), 3.0, device="cuda")
    assert ctx.dot(a, b) == pytest.approx(3.0 * (1.0 + 2.0 ** -20) * (1 << 20), rel=1e-15)
    rng = np.random.default_rng(11)
    n = (1 << 20) + 123
    x = rng.normal(size=n).astype(np.float32) * np.exp(rng.uniform(-8, 8, size=n)).astype(np.float32)
    y = (-x * (1.0 + 1e-6 * rng.normal(size=n))).astype(np.float32)
    y[::7] = rng.normal(size=y[::7].size).astype(np.float32)
    prods = x.astype(np.float64) * y.astype(np.float64)        # exact
    ref = math.fsum(prods)
    got = ctx.dot(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    assert abs(got - ref) <= 1e-12 * float(np.abs(prods).sum())


@pytest.mark.parametrize("lo,hi", [(-20.0, -12.0), (-23.0, -19.0), (15.0, 20.0)])
def test_dot_keeps_fp64_range(lo, hi):
    """Entries of 1e-20 to 1e-12 (the size of residuals and directions late in
    a PCG solve on fine grids) have products of 1e-40 to 1e-24, below FP32's
    normal range; entries near 1e20 have products beyond FP32's largest value.
    Both sum to within 1e-12 of sum |a_i b_i| of math.fsum over the exact
    products, and the SSD of such images keeps its value too."""
    import math
    ctx, t = _gpu("2d_transport_64")
    rng = np.random.default_rng(12)
    n = (1 << 18) + 77
    x = (rng.normal(size=n) * 10.0 ** rng.uniform(lo, hi, size=n)).astype(np.float32)
    y = (rng.normal(size=n) * 10.0 ** rng.uniform(lo, hi, size=n)).astype(np.float32)
    prods = x.astype(np.float64) * y.astype(np.float64)
    ref = math.fsum(prods)
    got = ctx.dot(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda())
    assert abs(got - ref) <= 1e-12 * float(np.abs(prods).sum())
    assert ctx.dot(torch.from_numpy(x).cuda(), torch.from_numpy(x).cuda()) == \
        pytest.approx(math.fsum(x.astype(np.float64) ** 2), rel=1e-12)
    # SSD at v = 0, where u1 = T exactly (every characteristic ends on its node)
    T, R = x[:4096].reshape(64, 64), y[:4096].reshape(64, 64)
    _, D, _ = ctx.objective(torch.zeros((1, 2, 32, 32), device="cuda"), torch.from_numpy(T.copy()).cuda(),
                            torch.from_numpy(R.copy()).cuda())
    d = T.astype(np.float64) - R.astype(np.float64)
    assert D == pytest.approx(0.5 / 64 ** 2 * math.fsum((d * d).ravel()), rel=1e-12)


def test_zero_velocity_is_identity():
    for name in ("2d_transport_64", "3d_continuity_K2"):
        ctx, t = _gpu(name)
        u1 = ctx.forward(torch.zeros_like(t["v"]), t["T"])
        np.testing.assert_allclose(_np(u1), t["T"].cpu().numpy(), rtol=0, atol=1e-6 * float(t["T"].abs().max()))


def test_continuity_conserves_mass_on_gpu():
    ctx, t = _gpu("2d_continuity_K5")
    T = t["T"].clone()
    T[:6] = 0
    T[-6:] = 0
    T[:, :6] = 0
    T[:, -6:] = 0
    u1 = ctx.forward(t["v"], T)
    assert abs(float(u1.double().sum()) - float(T.double().sum())) <= 1e-6 * float(T.double().sum())


def test_particles_leaving_the_domain_match_oracle():
    """Large velocities push characteristics outside the grid: zero extension on
    gathers, dropped mass on splats, exactly as the oracle."""
    from paper_1703_04446_gb300 import lgnk
    for model in ("transport", "continuity"):
        op, gp, a = make_case("2d_transport_64")
        op.model = gp["model"] = model
        v = a["v"].copy()
        v[:, 0] += 0.25   # an unwindowed shift along x carries particles across the edges
        ctx = lgnk.Context(lgnk.Problem(**gp))
        u1 = ctx.forward(torch.from_numpy(v).cuda(), torch.from_numpy(a["T"]).cuda())
        ref, y = L.final_state(model, v.astype(np.float64), op.vgrid, a["T"].astype(np.float64), op.igrid, op.N)
        # zero-extended v stops characteristics about half a velocity cell outside
        assert (y < 0.0).any() or (y > 1.0).any()
        assert rel(_np(u1), ref) <= TOL


def test_max_steps_and_degenerate_axis():
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case("2d_transport_64")
    op.N = gp["rk4_steps"] = 64
    ctx = lgnk.Context(lgnk.Problem(**gp))
    tv, tT, tdv = (torch.from_numpy(a[k]).cuda() for k in ("v", "T", "dv"))
    H = ctx.hessvec(tv, tT, tdv)
    ref = hessvec(op, a["v"].astype(np.float64), a["T"].astype(np.float64), a["dv"].astype(np.float64))
    assert rel(_np(H), ref) <= TOL
    # a grid one cell thick along y
    gp2 = dict(gp, image_m=(24, 1), velocity_m=(12, 1), rk4_steps=3)
    from oracle.objective import Problem as OP
    op2 = OP(L.Grid((24, 1)), L.Grid((12, 1)), K=1, N=3, alpha=op.alpha, gamma=op.gamma)
    rng = np.random.default_rng(3)
    T = rng.uniform(size=(1, 24)).astype(np.float32)
    v = (0.02 * rng.normal(size=(1, 2, 1, 12))).astype(np.float32)
    dv = (0.02 * rng.normal(size=(1, 2, 1, 12))).astype(np.float32)
    ctx2 = lgnk.Context(lgnk.Problem(**gp2))
    u1 = ctx2.forward(torch.from_numpy(v).cuda(), torch.from_numpy(T).cuda())
    assert rel(_np(u1), L.final_state("transport", v.astype(np.float64), op2.vgrid, T.astype(np.float64),
                                      op2.igrid, 3)[0]) <= TOL
    H2 = ctx2.hessvec(torch.from_numpy(v).cuda(), torch.from_numpy(T).cuda(), torch.from_numpy(dv).cuda())
    assert rel(_np(H2), hessvec(op2, v.astype(np.float64), T.astype(np.float64), dv.astype(np.float64))) <= TOL


@pytest.mark.parametrize("model", ["transport", "continuity"])
def test_max_steps_3d_time_dependent(model):
    """N = 64 (the largest the kernels record) with three time nodes (129 time
    slices) on a ragged 3D grid: the longest stage record and the most slices."""
    from paper_1703_04446_gb300 import lgnk
    from oracle.objective import Problem as OP
    from oracle.objective import gradient as ograd
    im, vm = (13, 11, 9), (7, 6, 5)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 0.9, 0.8)
    op = OP(L.Grid(im, lo, hi), L.Grid(vm, lo, hi), K=3, N=64, model=model, alpha=1e-2, gamma=1e-3)
    ctx = lgnk.Context(lgnk.Problem(image_m=im, velocity_m=vm, time_nodes=3, rk4_steps=64, model=model, alpha=1e-2,
                                    gamma=1e-3, image_lo=lo, image_hi=hi))
    rng = np.random.default_rng(11)
    X = L.cell_centres(op.igrid)
    T = np.exp(-((X[0] - 0.5) ** 2 + (X[1] - 0.45) ** 2 + (X[2] - 0.4) ** 2) / 0.03).reshape(op.igrid.shape)
    R = np.roll(T, 1, axis=2)
    g = synth.GridSpec(vm, lo, hi)
    v = synth.random_velocity(g, 3, 0.15, 3)
    dv = synth.random_velocity(g, 3, 0.05, 4)
    r = rng.normal(size=T.shape)
    f32 = {k: np.ascontiguousarray(a, dtype=np.float32) for k, a in dict(T=T, R=R, v=v, dv=dv, r=r).items()}
    f64 = {k: a.astype(np.float64) for k, a in f32.items()}
    t = {k: torch.from_numpy(a).cuda() for k, a in f32.items()}
    args = (model, f64["v"], op.vgrid, f64["T"], op.igrid, 64)
    assert rel(_np(ctx.forward(t["v"], t["T"])), L.final_state(*args)[0]) <= TOL
    assert rel(_np(ctx.hessvec(t["v"], t["T"], t["dv"])), hessvec(op, f64["v"], f64["T"], f64["dv"])) <= TOL
    if model == "transport":
        assert rel(_np(ctx.jvp(t["v"], t["T"], t["dv"])), L.jvp(*args, f64["dv"])) <= TOL
        assert rel(_np(ctx.jtvp(t["v"], t["T"], t["r"])), L.jtvp(*args, f64["r"])) <= TOL
        _, _, _, gr = ctx.objective(t["v"], t["T"], t["R"], grad=True)
        assert rel(_np(gr), ograd(op, f64["v"], f64["T"], f64["R"])) <= TOL


def test_aliasing_and_shape_errors():
    from paper_1703_04446_gb300 import lgnk
    ctx, t = _gpu("2d_transport_64")
    with pytest.raises(lgnk.LgnkError):
        ctx.hessvec(t["v"], t["T"], t["dv"], out=t["dv"])
    with pytest.raises(ValueError):
        ctx.forward(t["v"][..., :-1].contiguous(), t["T"])
    with pytest.raises(ValueError):
        ctx.forward(t["v"].double(), t["T"])


def test_memory_budget_is_enforced():
    from paper_1703_04446_gb300 import lgnk
    op, gp, a = make_case("3d_transport_ragged")
    with pytest.raises(lgnk.LgnkError) as e:
        lgnk.Context(lgnk.Problem(**gp), mem_budget=1024)
    assert e.value.status == 2
    ctx = lgnk.Context(lgnk.Problem(**gp))
    assert ctx.scratch_bytes > 0


def test_regularizer_operator_through_hessvec_at_zero_image():
    """With T = 0 the data term vanishes and H dv = alpha dt h^d A dv + gamma dv."""
    for name in ("2d_transport_ragged_K3", "2d_continuity_K5", "3d_continuity_K2"):
        op, gp, a = make_case(name)
        ctx, t = _gpu(name)
        H = ctx.hessvec(t["v"], torch.zeros_like(t["T"]), t["dv"])
        ref = op.alpha * reg_operator(op, a["dv"].astype(np.float64)) + op.gamma * a["dv"].astype(np.float64)
        assert rel(_np(H), ref) <= TOL


@pytest.mark.parametrize("name", ["2d_transport_ragged_K3", "3d_transport_ragged", "3d_continuity_K2"])
def test_jacobian_determinant(name):
    """det grad y of the generated map against the oracle's finite differences of
    its own end points (Sec. 4 monitors its range)."""
    ctx, t = _gpu(name)
    op, gp, a = make_case(name)
    det, lo, hi = ctx.jacobian_determinant(t["v"], t["T"])
    ref = L.jacobian_determinant(_oracle(name)["y"], op.igrid)
    got = det.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    assert abs(lo - ref.min()) <= 1e-4 * abs(ref.min()) and abs(hi - ref.max()) <= 1e-4 * abs(ref.max())
    assert abs(lo - got.min()) <= 1e-6 * abs(lo) and abs(hi - got.max()) <= 1e-6 * abs(hi)
