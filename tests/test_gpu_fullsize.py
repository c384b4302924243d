"""Parity at the benchmark's full size (128^3 image, 64^3 x 3 velocity, N = 8,
the same context and calls that bench.py times).  The oracle cannot run the
whole grid in seconds, so per-voxel outputs are compared on sampled voxels
(characteristics are independent: the oracle traces exactly those start
points), and outputs that sum over all voxels are checked through identities
that hold at any size."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from oracle.objective import Problem as OP, reg_operator
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def full():
    from paper_1703_04446_gb300 import lgnk
    ins = synth.make_inputs("3d_transport_128", seed=0)
    wl = ins["workload"]
    dv = synth.random_velocity(wl.velocity, 1, 4.0 / 128, 11).astype(np.float32)
    r = np.random.default_rng(5).normal(size=ins["T"].shape).astype(np.float32)
    ctx = lgnk.Context(lgnk.Problem.from_workload(wl, gamma=1e-3))
    t = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda()
         for k, a in dict(v=ins["v0"], T=ins["T"], R=ins["R"], dv=dv, r=r).items()}
    ig = L.Grid(wl.image.m, wl.image.lo, wl.image.hi)
    vg = L.Grid(wl.velocity.m, wl.velocity.lo, wl.velocity.hi)
    sample = np.random.default_rng(9).choice(ig.size, size=3000, replace=False)
    return ctx, t, ins, dv, ig, vg, sample, wl


def test_forward_and_jvp_on_sampled_voxels(full):
    ctx, t, ins, dv, ig, vg, sample, wl = full
    u1 = ctx.forward(t["v"], t["T"]).cpu().numpy().ravel()[sample]
    du = ctx.jvp(t["v"], t["T"], t["dv"]).cpu().numpy().ravel()[sample]
    x = L.cell_centres(ig)[:, sample]
    v64, T64 = ins["v0"].astype(np.float64), ins["T"].astype(np.float64)
    y, dy, _ = L.characteristics(v64, vg, x, wl.rk4_steps, -1, dv=dv.astype(np.float64))
    val, gT = L.interpolate(T64, ig, y, gradient=True)
    ref_du = np.sum(gT * dy, axis=0)
    assert np.linalg.norm(u1 - val) <= TOL * np.linalg.norm(val)
    assert np.linalg.norm(du - ref_du) <= TOL * np.linalg.norm(ref_du)


def test_adjoint_identity_full_size(full):
    ctx, t, *_ = full
    lhs = float((ctx.jvp(t["v"], t["T"], t["dv"]).double() * t["r"].double()).sum())
    rhs = float((ctx.jtvp(t["v"], t["T"], t["r"]).double() * t["dv"].double()).sum())
    assert abs(lhs - rhs) <= TOL * (abs(lhs) + abs(rhs))


def test_hessian_symmetric_and_consistent_full_size(full):
    ctx, t, ins, dv, ig, vg, sample, wl = full
    p, q = t["dv"], t["v"].clone()
    Hp, Hq = ctx.hessvec(t["v"], t["T"], p), ctx.hessvec(t["v"], t["T"], q)
    a = float((q.double() * Hp.double()).sum())
    b = float((p.double() * Hq.double()).sum())
    assert abs(a - b) <= TOL * (abs(a) + abs(b))
    # <p, Hp> = h^d |J p|^2 + alpha p^T A p + gamma |p|^2
    Jp = ctx.jvp(t["v"], t["T"], p).double()
    op = OP(ig, vg, K=1, N=wl.rk4_steps, alpha=wl.alpha, gamma=1e-3)
    p64 = dv.astype(np.float64)
    ref = ig.cell_volume * float((Jp * Jp).sum()) + wl.alpha * float(np.sum(p64 * reg_operator(op, p64))) \
        + 1e-3 * float(np.sum(p64 * p64))
    got = float((p.double() * Hp.double()).sum())
    assert abs(got - ref) <= TOL * abs(ref)


def test_objective_gradient_consistency_full_size(full):
    """d/de J(v + e dv) at e = 0 from central differences of the GPU objective
    agrees with <grad, dv> (FP64 sums; e = 1e-2 relative keeps FP32 noise low)."""
    ctx, t, *_ = full
    J, D, S, g = ctx.objective(t["v"], t["T"], t["R"], grad=True)
    e = 1e-2
    Jp = ctx.objective((t["v"] + e * t["dv"]).contiguous(), t["T"], t["R"])[0]
    Jm = ctx.objective((t["v"] - e * t["dv"]).contiguous(), t["T"], t["R"])[0]
    fd = (Jp - Jm) / (2 * e)
    an = float((g.double() * t["dv"].double()).sum())
    assert abs(an - fd) <= 2e-3 * abs(an)


def test_jtvp_on_sampled_support(full):
    """J^T r element by element at full size: r is zero except on the 3000
    sampled voxels, so J^T r is the sum of exactly those characteristics'
    adjoint sweeps, which the oracle computes one by one."""
    ctx, t, ins, dv, ig, vg, sample, wl = full
    rng = np.random.default_rng(21)
    r = np.zeros(ig.size, dtype=np.float32)
    r[sample] = rng.normal(size=sample.size).astype(np.float32)
    gv = ctx.jtvp(t["v"], t["T"], torch.from_numpy(r.reshape(ig.shape)).cuda()).cpu().numpy().astype(np.float64)
    v64, T64 = ins["v0"].astype(np.float64), ins["T"].astype(np.float64)
    x = L.cell_centres(ig)[:, sample]
    y, _, hist = L.characteristics(v64, vg, x, wl.rk4_steps, -1, keep=True)
    _, gT = L.interpolate(T64, ig, y, gradient=True)
    ref = L.characteristics_adjoint(v64, vg, hist, wl.rk4_steps, -1, gT * r[sample].astype(np.float64))
    assert np.linalg.norm(gv - ref) <= TOL * np.linalg.norm(ref)


def _sparse_template(ins, ig, wl, n_spots=12, radius=2, seed=31):
    """The benchmark's template kept only in small balls around a few interior
    points (zero elsewhere), and the voxels whose characteristic can end where
    its interpolated gradient is nonzero: within the balls' radius, plus the
    largest displacement the velocity can make in unit time, plus one cell."""
    rng = np.random.default_rng(seed)
    m = np.array(ig.m)
    centres = rng.integers(16, m - 16, size=(n_spots, 3))
    z, y, x = np.meshgrid(*(np.arange(k) for k in reversed(ig.m)), indexing="ij")
    idx = np.stack([x, y, z])
    d2 = np.min([np.sum((idx - c.reshape(3, 1, 1, 1)) ** 2, axis=0) for c in centres], axis=0)
    T = np.where(d2 <= radius ** 2, ins["T"], 0.0).astype(np.float32)
    vmax = float(np.sqrt(np.sum(ins["v0"].astype(np.float64) ** 2, axis=1)).max())
    reach = radius + vmax / min(ig.h) + 2.0
    support = np.flatnonzero(d2.ravel() <= reach ** 2)
    return T, support


@pytest.mark.parametrize("assembled", [False, True])
def test_hessvec_on_sparse_template(full, assembled):
    """The fused matrix-free Gauss-Newton matvec (and the assembled one) at full
    size, element by element: with a template that is zero outside a few small
    balls, row i of J vanishes unless characteristic i ends next to a ball, so
    H dv = sum over those voxels of J_i^T h^d J_i dv + alpha A dv + gamma dv,
    which the oracle computes voxel by voxel."""
    ctx, t, ins, dv, ig, vg, sample, wl = full
    Ts, support = _sparse_template(ins, ig, wl)
    tTs = torch.from_numpy(Ts).cuda()
    if assembled:
        ctx.assemble(t["v"], tTs)
        Hp = ctx.hessvec_assembled(t["dv"])
    else:
        Hp = ctx.hessvec(t["v"], tTs, t["dv"])
    Hp = Hp.cpu().numpy().astype(np.float64)
    # rows outside the support are exactly zero on the GPU as well
    du = ctx.jvp(t["v"], tTs, t["dv"]).cpu().numpy().ravel()
    outside = np.ones(ig.size, dtype=bool)
    outside[support] = False
    assert not np.any(du[outside])
    v64, T64, dv64 = ins["v0"].astype(np.float64), Ts.astype(np.float64), dv.astype(np.float64)
    x = L.cell_centres(ig)[:, support]
    y, dy, hist = L.characteristics(v64, vg, x, wl.rk4_steps, -1, dv=dv64, keep=True)
    _, gT = L.interpolate(T64, ig, y, gradient=True)
    du_ref = np.sum(gT * dy, axis=0)
    g = L.characteristics_adjoint(v64, vg, hist, wl.rk4_steps, -1, ig.cell_volume * du_ref * gT)
    op = OP(ig, vg, K=1, N=wl.rk4_steps, alpha=wl.alpha, gamma=1e-3)
    ref = g + wl.alpha * reg_operator(op, dv64) + 1e-3 * dv64
    data = g
    assert np.linalg.norm(data) > 1e-3 * np.linalg.norm(ref)      # the data term is not negligible
    assert np.linalg.norm(Hp - ref) <= TOL * np.linalg.norm(ref)
    # the data term alone, against its own norm
    reg_only = wl.alpha * reg_operator(op, dv64) + 1e-3 * dv64
    assert np.linalg.norm((Hp - reg_only) - data) <= 1e-4 * np.linalg.norm(data)
