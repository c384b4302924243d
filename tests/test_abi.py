"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/lgnk.h declares, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lgnk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(lgnk_[a-z_]+)\s*\(", src))
    return sorted(n for n in names)


@pytest.fixture(scope="module")
def lib():
    from paper_1703_04446_gb300 import build, lgnk
    build.build()
    return lgnk.load_library()


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("lgnk_create", "lgnk_forward", "lgnk_jvp", "lgnk_jtvp", "lgnk_objective", "lgnk_hessvec",
              "lgnk_solve", "lgnk_destroy", "lgnk_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1703_04446_gb300 import lgnk
    assert set(_declared()) <= set(lgnk.EXPORTS), set(_declared()) - set(lgnk.EXPORTS)


def test_status_strings(lib):
    for s in range(9):
        assert lib.lgnk_status_string(s) != b"unknown status"
    assert lib.lgnk_status_string(99) == b"unknown status"


def _problem(**over):
    from paper_1703_04446_gb300 import lgnk
    p = lgnk.Problem(image_m=(16, 16), velocity_m=(8, 8), time_nodes=1, rk4_steps=4)
    for k, v in over.items():
        setattr(p, k, v)
    return p.to_c()


@pytest.mark.parametrize("field,value,msg", [
    ("rk4_steps", 0, b"rk4_steps"), ("rk4_steps", 65, b"rk4_steps"), ("time_nodes", 0, b"time_nodes"),
    ("model", 5, b"model"), ("regularizer", 9, b"regularizer"), ("alpha", -1.0, b"alpha"),
    ("gamma", float("nan"), b"gamma"), ("pic_delta", -0.1, b"pic_delta"), ("pic_delta", float("inf"), b"pic_delta"),
    ("pic_delta", 0.01, b"continuity model only"),
])
def test_create_rejects_invalid_problem_before_any_device_call(lib, field, value, msg):
    pc = _problem()
    setattr(pc, field, value)
    h = ctypes.c_void_p()
    st = lib.lgnk_create(ctypes.byref(pc), None, 0, ctypes.byref(h))
    assert st == 1 and not h.value
    assert msg in lib.lgnk_last_error(None)


def test_create_rejects_too_wide_pic_particles(lib):
    pc = _problem(model="continuity", pic_delta=3.6 / 16)
    h = ctypes.c_void_p()
    assert lib.lgnk_create(ctypes.byref(pc), None, 0, ctypes.byref(h)) == 1
    assert b"3.5 image cells" in lib.lgnk_last_error(None)


def test_create_rejects_bad_grids(lib):
    pc = _problem()
    pc.image.d = 4
    h = ctypes.c_void_p()
    assert lib.lgnk_create(ctypes.byref(pc), None, 0, ctypes.byref(h)) == 1
    pc = _problem()
    pc.velocity.hi[0] = pc.velocity.lo[0]
    assert lib.lgnk_create(ctypes.byref(pc), None, 0, ctypes.byref(h)) == 1
    pc = _problem()
    pc.velocity.d = 3
    assert lib.lgnk_create(ctypes.byref(pc), None, 0, ctypes.byref(h)) == 1
    assert lib.lgnk_create(None, None, 0, ctypes.byref(h)) == 1


def test_null_context_is_rejected(lib):
    for name in ("lgnk_forward", "lgnk_jvp", "lgnk_jtvp", "lgnk_hessvec"):
        assert getattr(lib, name)(None, None, None, None, None) == 1
    assert lib.lgnk_precond(None, None, None) == 1
    assert lib.lgnk_assemble(None, None, None, None) == 1
    for name in ("lgnk_jvp_assembled", "lgnk_jtvp_assembled", "lgnk_hessvec_assembled"):
        assert getattr(lib, name)(None, None, None) == 1
    lib.lgnk_destroy(None)
    assert lib.lgnk_scratch_bytes(None) == 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1703_04446_gb300 import lgnk
    saved = lgnk._lib
    lgnk._lib = None
    try:
        with pytest.raises(RuntimeError, match="not found"):
            lgnk.load_library(str(tmp_path / "missing.so"))
    finally:
        lgnk._lib = saved


@pytest.mark.parametrize("m,c,B,scale", [(12, 4, 1, 1.0), (4, 4, 1, 1.0), (16, 0, 1, 1.0), (16, 4, 0, 1.0),
                                         (16, 4, 1, 0.0), (16, 4, 1, -1.0), (16, 300, 1, 1.0)])
def test_warm_start_create_rejects_bad_shapes_before_any_device_call(lib, m, c, B, scale):
    h = ctypes.c_void_p()
    assert lib.lgnk_ws_create(m, c, B, ctypes.c_float(scale), None, ctypes.byref(h)) == 1
    assert not h.value


def test_warm_start_null_handle_is_rejected(lib):
    assert lib.lgnk_ws_create(16, 4, 1, ctypes.c_float(1.0), None, None) == 1
    assert lib.lgnk_ws_num_params(None) == 0
    assert lib.lgnk_ws_predict(None, 1, None, None, None) == 1
    assert lib.lgnk_ws_train_step(None, 1, None, None, None, ctypes.c_float(1e-3), None) == 1
    for name in ("lgnk_ws_set_params", "lgnk_ws_get_params", "lgnk_ws_get_grads"):
        assert getattr(lib, name)(None, None) == 1
    assert lib.lgnk_ws_last_error(None)
    lib.lgnk_ws_destroy(None)
