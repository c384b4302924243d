"""Parity at the full sizes of the mass-preserving workloads (2D 256^2 on 5 time
nodes, N = 16; 3D 192 x 224 x 160 on 9 time nodes, N = 16), in the contexts
bench.py runs them.  Characteristics are independent, so the end points of
sampled particles are compared with the oracle's one by one; the push-forward
and the derivative products sum over all particles and are checked through
identities that hold at any size."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", params=["2d_continuity_256", "3d_continuity_brain"])
def case(request):
    from paper_1703_04446_gb300 import lgnk
    name = request.param
    ins = synth.make_inputs(name, seed=0)
    wl = ins["workload"]
    ctx = lgnk.Context(lgnk.Problem.from_workload(wl, gamma=1e-4))
    h = min(wl.image.h)
    dv = synth.random_velocity(wl.velocity, wl.time_nodes, 2 * h, 5).astype(np.float32)
    p2 = synth.random_velocity(wl.velocity, wl.time_nodes, 2 * h, 6).astype(np.float32)
    r = np.random.default_rng(4).normal(size=ins["T"].shape).astype(np.float32)
    t = {k: torch.from_numpy(np.ascontiguousarray(a)).cuda()
         for k, a in dict(v=ins["v0"], T=ins["T"], dv=dv, p2=p2, r=r).items()}
    yield name, wl, ins, ctx, t
    ctx.close()
    torch.cuda.empty_cache()


def test_end_points_of_sampled_particles(case):
    name, wl, ins, ctx, t = case
    u1, y = ctx.forward(t["v"], t["T"], return_y=True)
    d = wl.image.d
    ig = L.Grid(wl.image.m, wl.image.lo, wl.image.hi)
    vg = L.Grid(wl.velocity.m, wl.velocity.lo, wl.velocity.hi)
    sample = np.random.default_rng(2).choice(ig.size, size=1500, replace=False)
    x = L.cell_centres(ig)[:, sample]
    ref, _, _ = L.characteristics(ins["v0"].astype(np.float64), vg, x, wl.rk4_steps, +1)
    got = y.reshape(d, -1).cpu().numpy()[:, sample].astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)
    # mass is conserved (the phantoms stay inside the grid)
    assert abs(float(u1.double().sum()) - float(t["T"].double().sum())) <= 1e-5 * float(t["T"].double().sum())


def test_adjoint_identity_full_size(case):
    name, wl, ins, ctx, t = case
    lhs = float((ctx.jvp(t["v"], t["T"], t["dv"]).double() * t["r"].double()).sum())
    rhs = float((ctx.jtvp(t["v"], t["T"], t["r"]).double() * t["dv"].double()).sum())
    assert abs(lhs - rhs) <= TOL * (abs(lhs) + abs(rhs))


def test_hessian_symmetry_full_size(case):
    name, wl, ins, ctx, t = case
    Hp = ctx.hessvec(t["v"], t["T"], t["dv"])
    Hq = ctx.hessvec(t["v"], t["T"], t["p2"])
    a = float((t["p2"].double() * Hp.double()).sum())
    b = float((t["dv"].double() * Hq.double()).sum())
    assert abs(a - b) <= TOL * (abs(a) + abs(b))


def _sampled_particles(wl, ins, n=1500, seed=12):
    """A template whose mass sits only on n sampled particles (zero elsewhere):
    the push-forward, its derivative and its transpose then involve exactly
    those characteristics, which the oracle traces one by one."""
    ig = L.Grid(wl.image.m, wl.image.lo, wl.image.hi)
    sample = np.random.default_rng(seed).choice(ig.size, size=n, replace=False)
    Ts = np.zeros(ig.size, dtype=np.float32)
    Ts[sample] = ins["T"].ravel()[sample] + np.float32(0.5 * ins["T"].max())
    return ig, sample, Ts


def test_products_on_sampled_particles(case):
    """u1, J dv and J^T r element by element at full size (the whole image and
    the whole velocity gradient), with the template's mass on sampled particles."""
    name, wl, ins, ctx, t = case
    ig, sample, Ts = _sampled_particles(wl, ins)
    vg = L.Grid(wl.velocity.m, wl.velocity.lo, wl.velocity.hi)
    tTs = torch.from_numpy(Ts.reshape(ig.shape)).cuda()
    u1 = ctx.forward(t["v"], tTs).cpu().numpy().astype(np.float64).ravel()
    du = ctx.jvp(t["v"], tTs, t["dv"]).cpu().numpy().astype(np.float64).ravel()
    gv = ctx.jtvp(t["v"], tTs, t["r"]).cpu().numpy().astype(np.float64)
    v64, dv64 = ins["v0"].astype(np.float64), t["dv"].cpu().numpy().astype(np.float64)
    x = L.cell_centres(ig)[:, sample]
    mass = Ts[sample].astype(np.float64)
    y, dy, _ = L.characteristics(v64, vg, x, wl.rk4_steps, +1, dv=dv64)
    u1_ref = L.scatter(mass, ig, y).ravel()
    du_ref = L.scatter_gradient(mass, dy, ig, y).ravel()
    assert np.linalg.norm(u1 - u1_ref) <= TOL * np.linalg.norm(u1_ref)
    assert np.linalg.norm(du - du_ref) <= TOL * np.linalg.norm(du_ref)
    _, _, hist = L.characteristics(v64, vg, x, wl.rk4_steps, +1, keep=True)
    _, gr = L.interpolate(t["r"].cpu().numpy().astype(np.float64), ig, y, gradient=True)
    gv_ref = L.characteristics_adjoint(v64, vg, hist, wl.rk4_steps, +1, gr * mass)
    assert np.linalg.norm(gv - gv_ref) <= TOL * np.linalg.norm(gv_ref)
