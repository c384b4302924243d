"""The allocation-free transport forward (lgnk_forward_transport_static).

It serves callers that must not call cudaMalloc after start-up, such as a
latency-critical loop or a process whose device memory already belongs to
another allocator.  Its scratch is a fixed 32 MiB device array shared by all
calls.  Here it is called twice in a row through the C ABI on different
problems, and each result is compared with the context-based lgnk_forward and
the SSD of lgnk_objective.  The file sorts last, so a failure here does not
stop the other tests of a run that halts at the first failure."""
import ctypes

import numpy as np
import pytest
import torch

from tests._cases import make_case, rel

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _static_call(lib, prob_c, t, with_ssd=True):
    u1 = torch.empty_like(t["T"])
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    ptr = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else None
    st = lib.lgnk_forward_transport_static(ctypes.byref(prob_c), ptr(t["v"]), ptr(t["T"]),
                                           ptr(t["R"]) if with_ssd else None, ptr(u1),
                                           ptr(D) if with_ssd else None,
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, u1, D


def test_static_scratch_forward_matches_context_path_twice():
    from paper_1703_04446_gb300 import lgnk
    lib = lgnk.load_library()
    for name in ("3d_transport_ragged", "2d_transport_ragged_K3"):
        op, gp, a = make_case(name)
        prob = lgnk.Problem(**gp)
        t = {k: torch.from_numpy(v).cuda() for k, v in a.items()}
        st, u1, D = _static_call(lib, prob.to_c(), t)
        assert st == 0, lib.lgnk_last_error(None)
        ctx = lgnk.Context(prob)
        ref_u1 = ctx.forward(t["v"], t["T"])
        _, ref_D, _ = ctx.objective(t["v"], t["T"], t["R"])
        torch.cuda.synchronize()
        assert rel(u1.cpu().numpy(), ref_u1.cpu().numpy()) <= TOL
        assert abs(float(D.item()) - ref_D) <= TOL * abs(ref_D)
        ctx.close()


def test_static_scratch_without_ssd_and_size_limit():
    from paper_1703_04446_gb300 import lgnk
    lib = lgnk.load_library()
    op, gp, a = make_case("2d_transport_64")
    prob = lgnk.Problem(**gp)
    t = {k: torch.from_numpy(v).cuda() for k, v in a.items()}
    st, u1, _ = _static_call(lib, prob.to_c(), t, with_ssd=False)
    assert st == 0
    ref = lgnk.Context(prob).forward(t["v"], t["T"])
    torch.cuda.synchronize()
    assert rel(u1.cpu().numpy(), ref.cpu().numpy()) <= TOL
    # a 256^3 image alone needs more than the fixed scratch (the call is rejected
    # before the device is touched)
    big = lgnk.Problem(image_m=(256, 256, 256), velocity_m=(128, 128, 128), rk4_steps=2)
    tb = {"v": torch.zeros(big.velocity_shape, device="cuda"), "T": torch.zeros(big.image_shape, device="cuda"),
          "R": torch.zeros(big.image_shape, device="cuda")}
    st, _, _ = _static_call(lib, big.to_c(), tb)
    assert st == 1 and b"static maximum" in lib.lgnk_last_error(None)
    # continuity is not offered allocation-free
    cont = lgnk.Problem(**dict(gp, model="continuity"))
    st, _, _ = _static_call(lib, cont.to_c(), t)
    assert st == 1
