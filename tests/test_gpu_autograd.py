"""The Lagrangian forward map as a torch.autograd.Function (forward = lgnk_forward,
backward = the hand-written J^T kernel, trajectory recomputed): checked by
central finite differences (h = 1e-3) and against the oracle's J^T on 16^3
crops of the 3D transport workload."""
import numpy as np
import pytest
import torch

from oracle import lagrangian as L
from paper_1703_04446_gb300 import synth

pytestmark = pytest.mark.gpu


def _crop_problem(seed=0):
    from paper_1703_04446_gb300 import lgnk
    ins = synth.make_inputs("3d_transport_128", seed=seed)
    T = np.ascontiguousarray(ins["T"][40:56, 50:66, 30:46])       # 16^3 crop of the phantom
    R = np.ascontiguousarray(ins["R"][40:56, 50:66, 30:46])
    g = synth.GridSpec((16, 16, 16), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    vg = synth.GridSpec((8, 8, 8), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    v = synth.random_velocity(vg, 1, 3.0 / 16, seed + 3).astype(np.float32)
    prob = lgnk.Problem(image_m=(16, 16, 16), velocity_m=(8, 8, 8), time_nodes=1, rk4_steps=8, alpha=1e-3)
    return prob, g, vg, T, R, v


def test_backward_matches_central_differences():
    from paper_1703_04446_gb300 import lgnk
    prob, g, vg, T, R, v = _crop_problem()
    ctx = lgnk.Context(prob)
    tT, tR = torch.from_numpy(T).cuda(), torch.from_numpy(R).cuda()
    tv = torch.from_numpy(v).cuda().requires_grad_(True)

    def loss(vv):
        u1 = lgnk.lagrangian_forward(ctx, vv, tT)
        return 0.5 * ((u1 - tR) ** 2).sum()

    lo = loss(tv)
    lo.backward()
    grad = tv.grad.detach().double()
    rng = np.random.default_rng(7)
    h = 1e-3
    for _ in range(3):
        d = torch.from_numpy(rng.normal(size=v.shape).astype(np.float32)).cuda()
        d = d / d.norm() * float(tv.detach().norm())
        with torch.no_grad():
            fd = (loss(tv.detach() + h * d).double() - loss(tv.detach() - h * d).double()) / (2 * h)
        an = float((grad * d.double()).sum())
        assert abs(an - float(fd)) <= 2e-3 * max(abs(an), abs(float(fd))), (an, float(fd))


def test_backward_matches_oracle_jtvp():
    from paper_1703_04446_gb300 import lgnk
    prob, g, vg, T, R, v = _crop_problem(seed=1)
    ctx = lgnk.Context(prob)
    tT, tR = torch.from_numpy(T).cuda(), torch.from_numpy(R).cuda()
    tv = torch.from_numpy(v).cuda().requires_grad_(True)
    u1 = lgnk.lagrangian_forward(ctx, tv, tT)
    (u1 * tR).sum().backward()
    ig, og = L.Grid((16, 16, 16)), L.Grid((8, 8, 8))
    ref = L.jtvp("transport", v.astype(np.float64), og, T.astype(np.float64), ig, 8, R.astype(np.float64))
    got = tv.grad.detach().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_autograd_composes_with_torch_ops():
    """Gradients through u1 flow into the rest of a torch graph (T constant)."""
    from paper_1703_04446_gb300 import lgnk
    prob, g, vg, T, R, v = _crop_problem(seed=2)
    ctx = lgnk.Context(prob)
    tT = torch.from_numpy(T).cuda()
    w = torch.randn(prob.image_shape, device="cuda")
    tv = torch.from_numpy(v).cuda().requires_grad_(True)
    scale = torch.tensor(2.0, device="cuda", requires_grad=True)
    out = (scale * lgnk.lagrangian_forward(ctx, tv, tT) * w).sum()
    out.backward()
    gv = ctx.jtvp(tv.detach(), tT, (2.0 * w).contiguous())
    assert torch.allclose(tv.grad, gv, rtol=1e-5, atol=1e-7 * float(gv.abs().max()))
    assert scale.grad is not None
