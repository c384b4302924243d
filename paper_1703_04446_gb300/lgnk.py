"""Thin ctypes binding of the lgnk C ABI (include/lgnk.h).

Argument marshalling only: every step of the hot path runs in the CUDA library
``liblgnk.so``.  Tensors are torch CUDA float32 and contiguous; the library
works on torch's current stream.  If the library is missing or cannot be
loaded, every call raises: there is no CPU fallback.

The functions keep the C names (``lgnk_forward`` ...) and take a ``Context``;
``Context`` also exposes them as methods.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np
import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblgnk.so")

TRANSPORT, CONTINUITY = 0, 1
SSD = 0
DIFFUSION, CURVATURE, ELASTIC = 0, 1, 2
_MODELS = {"transport": TRANSPORT, "continuity": CONTINUITY}
_REGS = {"diffusion": DIFFUSION, "curvature": CURVATURE, "elastic": ELASTIC}

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "non-finite value",
          5: "internal error", 6: "line search failed", 7: "not converged", 8: "capacity exceeded"}


class LgnkError(RuntimeError):
    def __init__(self, status, detail=""):
        super().__init__(f"lgnk: {STATUS.get(status, status)}" + (f": {detail}" if detail else ""))
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("m", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class _Problem(ctypes.Structure):
    _fields_ = [("image", _Grid), ("velocity", _Grid), ("time_nodes", ctypes.c_int),
                ("rk4_steps", ctypes.c_int), ("model", ctypes.c_int), ("distance", ctypes.c_int),
                ("regularizer", ctypes.c_int), ("alpha", ctypes.c_double), ("gamma", ctypes.c_double),
                ("mu_lame", ctypes.c_double), ("lambda_lame", ctypes.c_double), ("pic_delta", ctypes.c_double)]


class _SolveOpts(ctypes.Structure):
    _fields_ = [("max_gn", ctypes.c_int), ("gn_grad_rtol", ctypes.c_double), ("max_pcg", ctypes.c_int),
                ("pcg_rtol", ctypes.c_double), ("armijo_c", ctypes.c_double), ("max_ls", ctypes.c_int),
                ("precond", ctypes.c_int), ("verbosity", ctypes.c_int), ("gn_grad_atol", ctypes.c_double),
                ("matvec", ctypes.c_int)]


class _SolveReport(ctypes.Structure):
    _fields_ = [("gn_iters", ctypes.c_int), ("pcg_iters", ctypes.c_int), ("hessvecs", ctypes.c_int),
                ("objective_evals", ctypes.c_int), ("J0", ctypes.c_double), ("J", ctypes.c_double),
                ("D", ctypes.c_double), ("S", ctypes.c_double), ("g0", ctypes.c_double),
                ("g", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("assembled_gn", ctypes.c_int), ("last_mu", ctypes.c_double)]


EXPORTS = {
    # name: (restype, argtypes)
    "lgnk_create": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_void_p, ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "lgnk_destroy": (None, [ctypes.c_void_p]),
    "lgnk_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lgnk_scratch_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "lgnk_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lgnk_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lgnk_forward": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "lgnk_jvp": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "lgnk_jtvp": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "lgnk_objective": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.POINTER(ctypes.c_double)] * 3
                       + [ctypes.c_void_p]),
    "lgnk_hessvec": (ctypes.c_int, [ctypes.c_void_p] * 5),
    "lgnk_precond": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "lgnk_assemble": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.POINTER(ctypes.c_size_t)]),
    "lgnk_jvp_assembled": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "lgnk_jtvp_assembled": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "lgnk_hessvec_assembled": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "lgnk_jacobian_determinant": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.POINTER(ctypes.c_double)] * 2),
    "lgnk_dot": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)]),
    "lgnk_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lgnk_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "lgnk_forward_transport_static": (ctypes.c_int, [ctypes.POINTER(_Problem)] + [ctypes.c_void_p] * 6),
    "lgnk_restrict_image": (ctypes.c_int, [ctypes.POINTER(_Grid)] + [ctypes.c_void_p] * 3),
    "lgnk_prolong_velocity": (ctypes.c_int, [ctypes.POINTER(_Grid), ctypes.POINTER(_Grid), ctypes.c_int]
                              + [ctypes.c_void_p] * 3),
    "lgnk_solve_multilevel": (ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.POINTER(_SolveOpts), ctypes.c_void_p]),
    "lgnk_solve_opts_default": (None, [ctypes.POINTER(_SolveOpts)]),
    "lgnk_solve": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.POINTER(_SolveOpts),
                                                         ctypes.POINTER(_SolveReport)]),
    "lgnk_ws_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "lgnk_ws_destroy": (None, [ctypes.c_void_p]),
    "lgnk_ws_num_params": (ctypes.c_size_t, [ctypes.c_void_p]),
    "lgnk_ws_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lgnk_ws_set_params": (ctypes.c_int, [ctypes.c_void_p] * 2),
    "lgnk_ws_get_params": (ctypes.c_int, [ctypes.c_void_p] * 2),
    "lgnk_ws_get_grads": (ctypes.c_int, [ctypes.c_void_p] * 2),
    "lgnk_ws_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3),
    "lgnk_ws_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 3
                           + [ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblgnk.so (built by ``paper_1703_04446_gb300.build``) and declare its symbols."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"lgnk CUDA library not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


@dataclass
class Problem:
    """Eq. 9 with SSD on cell-centred grids (Sec. 3).  Grid tuples are in axis
    order (x, y[, z]); arrays use numpy order (z, y, x)."""
    image_m: tuple
    velocity_m: tuple
    time_nodes: int = 1
    rk4_steps: int = 4
    model: str = "transport"
    regularizer: str = "diffusion"
    alpha: float = 1e-2
    gamma: float = 0.0
    image_lo: tuple = None
    image_hi: tuple = None
    velocity_lo: tuple = None
    velocity_hi: tuple = None
    mu_lame: float = 1.0
    lambda_lame: float = 0.0
    pic_delta: float = 0.0      # continuity PIC half-width (domain units); 0: width = cell size
    extra: dict = field(default_factory=dict)

    def __post_init__(self):
        d = len(self.image_m)
        self.image_lo = tuple(self.image_lo or (0.0,) * d)
        self.image_hi = tuple(self.image_hi or (1.0,) * d)
        self.velocity_lo = tuple(self.velocity_lo or self.image_lo)
        self.velocity_hi = tuple(self.velocity_hi or self.image_hi)

    @property
    def d(self):
        return len(self.image_m)

    @property
    def image_shape(self):
        return tuple(reversed(self.image_m))

    @property
    def velocity_shape(self):
        return (self.time_nodes, self.d) + tuple(reversed(self.velocity_m))

    @classmethod
    def from_workload(cls, wl, **over):
        kw = dict(image_m=wl.image.m, velocity_m=wl.velocity.m, time_nodes=wl.time_nodes,
                  rk4_steps=wl.rk4_steps, model=wl.model, regularizer=wl.regularizer, alpha=wl.alpha,
                  gamma=wl.gamma, image_lo=wl.image.lo, image_hi=wl.image.hi, velocity_lo=wl.velocity.lo,
                  velocity_hi=wl.velocity.hi, mu_lame=wl.extra.get("mu", 1.0),
                  lambda_lame=wl.extra.get("lam", 0.0))
        kw.update(over)
        return cls(**kw)

    def to_c(self) -> _Problem:
        def grid(m, lo, hi):
            g = _Grid()
            g.d = len(m)
            for a in range(3):
                g.m[a] = int(m[a]) if a < len(m) else 1
                g.lo[a] = float(lo[a]) if a < len(m) else 0.0
                g.hi[a] = float(hi[a]) if a < len(m) else 1.0
            return g
        p = _Problem()
        p.image = grid(self.image_m, self.image_lo, self.image_hi)
        p.velocity = grid(self.velocity_m, self.velocity_lo, self.velocity_hi)
        p.time_nodes = int(self.time_nodes)
        p.rk4_steps = int(self.rk4_steps)
        p.model = _MODELS[self.model] if isinstance(self.model, str) else int(self.model)
        p.distance = SSD
        p.regularizer = _REGS[self.regularizer] if isinstance(self.regularizer, str) else int(self.regularizer)
        p.alpha = float(self.alpha)
        p.gamma = float(self.gamma)
        p.mu_lame = float(self.mu_lame)
        p.lambda_lame = float(self.lambda_lame)
        p.pic_delta = float(self.pic_delta)
        return p


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Context:
    """An lgnk context bound to one CUDA device; wraps lgnk_create/lgnk_destroy."""

    def __init__(self, problem: Problem, mem_budget: int = 0, device=None):
        self.lib = load_library()
        self.problem = problem
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        handle = ctypes.c_void_p()
        self._pc = problem.to_c()
        with torch.cuda.device(self.device):
            st = self.lib.lgnk_create(ctypes.byref(self._pc), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      ctypes.c_size_t(mem_budget), ctypes.byref(handle))
        if st != 0:
            raise LgnkError(st, self.lib.lgnk_last_error(None).decode())
        self.handle = handle

    # --------------------------------------------------------------- helpers
    def close(self):
        if getattr(self, "handle", None):
            self.lib.lgnk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        self.lib.lgnk_set_stream(self.handle, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def _check(self, st):
        if st != 0:
            raise LgnkError(st, self.lib.lgnk_last_error(self.handle).decode())

    def _arg(self, t, shape, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.device != self.device or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if t.numel() != int(torch.Size(shape).numel()):
            raise ValueError(f"{name} has {t.numel()} elements, expected shape {tuple(shape)}")
        return t

    def _img(self, t, name):
        return self._arg(t, self.problem.image_shape, name)

    def _vel(self, t, name):
        return self._arg(t, self.problem.velocity_shape, name)

    def _new_img(self):
        return torch.empty(self.problem.image_shape, device=self.device, dtype=torch.float32)

    def _new_vel(self):
        return torch.empty(self.problem.velocity_shape, device=self.device, dtype=torch.float32)

    @property
    def scratch_bytes(self):
        return int(self.lib.lgnk_scratch_bytes(self.handle))

    # ------------------------------------------------------------- the calls
    def forward(self, v, T, return_y=False):
        return lgnk_forward(self, v, T, return_y)

    def jvp(self, v, T, dv):
        return lgnk_jvp(self, v, T, dv)

    def jtvp(self, v, T, r):
        return lgnk_jtvp(self, v, T, r)

    def objective(self, v, T, R, grad=False):
        return lgnk_objective(self, v, T, R, grad)

    def hessvec(self, v, T, dv, out=None):
        return lgnk_hessvec(self, v, T, dv, out)

    def precond(self, r):
        return lgnk_precond(self, r)

    def assemble(self, v, T):
        return lgnk_assemble(self, v, T)

    def jvp_assembled(self, dv):
        return lgnk_jvp_assembled(self, dv)

    def jtvp_assembled(self, r):
        return lgnk_jtvp_assembled(self, r)

    def hessvec_assembled(self, dv, out=None):
        return lgnk_hessvec_assembled(self, dv, out)

    def jacobian_determinant(self, v, T, field=True):
        return lgnk_jacobian_determinant(self, v, T, field)

    def dot(self, a, b):
        return lgnk_dot(self, a, b)

    def solve(self, T, R, v0=None, **opts):
        return lgnk_solve(self, T, R, v0, **opts)

    def profile(self, enable=True):
        """Start (reset) or stop CUDA-event timing of the tracing kernels."""
        self._check(self.lib.lgnk_profile(self.handle, int(bool(enable))))

    def profile_read(self):
        """(tracing-kernel ms, tracing launches, all kernel launches) since profile(True)."""
        ms, nt, nk = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self.lib.lgnk_profile_read(self.handle, ctypes.byref(ms), ctypes.byref(nt), ctypes.byref(nk)))
        return ms.value, nt.value, nk.value


def lgnk_create(problem: Problem, mem_budget: int = 0, device=None) -> Context:
    return Context(problem, mem_budget, device)


def lgnk_destroy(ctx: Context):
    ctx.close()


def lgnk_forward(ctx: Context, v, T, return_y=False):
    """u1(v) (Eq. 6 / Eq. 7); with return_y also the characteristic end points [d][M]."""
    ctx._vel(v, "v"), ctx._img(T, "T")
    u1 = ctx._new_img()
    y = torch.empty((ctx.problem.d,) + ctx.problem.image_shape, device=ctx.device) if return_y else None
    ctx._stream()
    ctx._check(ctx.lib.lgnk_forward(ctx.handle, _ptr(v), _ptr(T), _ptr(u1), _ptr(y)))
    return (u1, y) if return_y else u1


def lgnk_jvp(ctx: Context, v, T, dv):
    """(d_v u1) dv (Sec. 3.2)."""
    ctx._vel(v, "v"), ctx._img(T, "T"), ctx._vel(dv, "dv")
    du = ctx._new_img()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_jvp(ctx.handle, _ptr(v), _ptr(T), _ptr(dv), _ptr(du)))
    return du


def lgnk_jtvp(ctx: Context, v, T, r):
    """(d_v u1)^T r (Sec. 3.2)."""
    ctx._vel(v, "v"), ctx._img(T, "T"), ctx._img(r, "r")
    gv = ctx._new_vel()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_jtvp(ctx.handle, _ptr(v), _ptr(T), _ptr(r), _ptr(gv)))
    return gv


def lgnk_objective(ctx: Context, v, T, R, grad=False):
    """(J, D, S) of Eq. 9-10, and the gradient when grad=True."""
    ctx._vel(v, "v"), ctx._img(T, "T"), ctx._img(R, "R")
    J, D, S = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    g = ctx._new_vel() if grad else None
    ctx._stream()
    ctx._check(ctx.lib.lgnk_objective(ctx.handle, _ptr(v), _ptr(T), _ptr(R), ctypes.byref(J),
                                      ctypes.byref(D), ctypes.byref(S), _ptr(g)))
    out = (J.value, D.value, S.value)
    return out + (g,) if grad else out


def lgnk_hessvec(ctx: Context, v, T, dv, out=None):
    """Gauss-Newton Hessian matvec H dv at v (Sec. 3.2)."""
    ctx._vel(v, "v"), ctx._img(T, "T"), ctx._vel(dv, "dv")
    out = ctx._new_vel() if out is None else ctx._vel(out, "out")
    ctx._stream()
    ctx._check(ctx.lib.lgnk_hessvec(ctx.handle, _ptr(v), _ptr(T), _ptr(dv), _ptr(out)))
    return out


def lgnk_assemble(ctx: Context, v, T):
    """Assemble J = d_v u1 at (v, T) (transport, Sec. 3.3) into the context.
    Returns the number of (time slice, velocity cell) blocks stored."""
    ctx._vel(v, "v"), ctx._img(T, "T")
    blocks = ctypes.c_size_t()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_assemble(ctx.handle, _ptr(v), _ptr(T), ctypes.byref(blocks)))
    return blocks.value


def lgnk_jvp_assembled(ctx: Context, dv):
    """J dv with the assembled J."""
    ctx._vel(dv, "dv")
    du = ctx._new_img()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_jvp_assembled(ctx.handle, _ptr(dv), _ptr(du)))
    return du


def lgnk_jtvp_assembled(ctx: Context, r):
    """J^T r with the assembled J."""
    ctx._img(r, "r")
    gv = ctx._new_vel()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_jtvp_assembled(ctx.handle, _ptr(r), _ptr(gv)))
    return gv


def lgnk_hessvec_assembled(ctx: Context, dv, out=None):
    """Gauss-Newton Hessian matvec with the assembled J (plus the regularizer)."""
    ctx._vel(dv, "dv")
    out = ctx._new_vel() if out is None else ctx._vel(out, "out")
    ctx._stream()
    ctx._check(ctx.lib.lgnk_hessvec_assembled(ctx.handle, _ptr(dv), _ptr(out)))
    return out


def lgnk_precond(ctx: Context, r):
    """Spectral (DCT) preconditioner applied to r (Sec. 3.2)."""
    ctx._vel(r, "r")
    z = ctx._new_vel()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_precond(ctx.handle, _ptr(r), _ptr(z)))
    return z


def lgnk_jacobian_determinant(ctx: Context, v, T, field=True):
    """(det grad y field or None, min, max) of the map generated by v."""
    ctx._vel(v, "v"), ctx._img(T, "T")
    det = ctx._new_img() if field else None
    lo, hi = ctypes.c_double(), ctypes.c_double()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_jacobian_determinant(ctx.handle, _ptr(v), _ptr(T), _ptr(det), ctypes.byref(lo),
                                                 ctypes.byref(hi)))
    return det, lo.value, hi.value


def lgnk_dot(ctx: Context, a, b):
    """Inner product of two float32 device tensors, summed in FP64 on the device, as a Python float."""
    if a.numel() != b.numel():
        raise ValueError("size mismatch")
    for t in (a, b):
        if t.device != ctx.device or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("dot operands must be contiguous float32 on the context's device")
    out = ctypes.c_double()
    ctx._stream()
    ctx._check(ctx.lib.lgnk_dot(ctx.handle, _ptr(a), _ptr(b), ctypes.c_size_t(a.numel()), ctypes.byref(out)))
    return out.value


def lgnk_solve(ctx: Context, T, R, v0=None, **opts):
    """Inexact Gauss-Newton-Krylov solve (Eq. 11).  Returns (v, report dict)."""
    ctx._img(T, "T"), ctx._img(R, "R")
    v = torch.zeros(ctx.problem.velocity_shape, device=ctx.device) if v0 is None else ctx._vel(v0, "v0").clone()
    o = _SolveOpts()
    ctx.lib.lgnk_solve_opts_default(ctypes.byref(o))
    for k, val in opts.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown solve option {k}")
        setattr(o, k, type(getattr(o, k))(val))
    rep = _SolveReport()
    ctx._stream()
    st = ctx.lib.lgnk_solve(ctx.handle, _ptr(T), _ptr(R), _ptr(v), ctypes.byref(o), ctypes.byref(rep))
    report = {f: getattr(rep, f) for f, _ in _SolveReport._fields_}
    report["status_name"] = STATUS.get(st, str(st))
    if st not in (0, 6, 7):
        raise LgnkError(st, ctx.lib.lgnk_last_error(ctx.handle).decode())
    return v, report


def _grid_c(m, lo, hi):
    g = _Grid()
    g.d = len(m)
    for a in range(3):
        g.m[a] = int(m[a]) if a < len(m) else 1
        g.lo[a] = float(lo[a]) if a < len(m) else 0.0
        g.hi[a] = float(hi[a]) if a < len(m) else 1.0
    return g


def _raise_free(lib, st):
    if st != 0:
        raise LgnkError(st, lib.lgnk_last_error(None).decode())


def lgnk_restrict_image(F, m, lo=None, hi=None):
    """Average of the 2^d fine cells tiling each coarse cell (m: fine cell counts, x first)."""
    lib = load_library()
    d = len(m)
    lo = lo or (0.0,) * d
    hi = hi or (1.0,) * d
    if F.dtype != torch.float32 or not F.is_cuda or not F.is_contiguous() or F.numel() != int(np.prod(m)):
        raise ValueError("F must be a contiguous float32 CUDA tensor with prod(m) elements")
    C = torch.empty(tuple(reversed([a // 2 for a in m])), device=F.device, dtype=torch.float32)
    g = _grid_c(m, lo, hi)
    _raise_free(lib, lib.lgnk_restrict_image(ctypes.byref(g), _ptr(F), _ptr(C),
                                             ctypes.c_void_p(torch.cuda.current_stream(F.device).cuda_stream)))
    return C


def lgnk_prolong_velocity(vc, coarse_m, fine_m, lo=None, hi=None):
    """Multilinear interpolation of the coarse velocity [K][d][...] at the fine cell centres."""
    lib = load_library()
    d = len(coarse_m)
    lo = lo or (0.0,) * d
    hi = hi or (1.0,) * d
    K = vc.shape[0]
    if vc.dtype != torch.float32 or not vc.is_cuda or not vc.is_contiguous():
        raise ValueError("vc must be a contiguous float32 CUDA tensor")
    vf = torch.empty((K, d) + tuple(reversed(fine_m)), device=vc.device, dtype=torch.float32)
    cg, fg = _grid_c(coarse_m, lo, hi), _grid_c(fine_m, lo, hi)
    _raise_free(lib, lib.lgnk_prolong_velocity(ctypes.byref(cg), ctypes.byref(fg), K, _ptr(vc), _ptr(vf),
                                               ctypes.c_void_p(torch.cuda.current_stream(vc.device).cuda_stream)))
    return vf


def lgnk_solve_multilevel(problem: Problem, T, R, levels, mem_budget=0, **opts):
    """Coarse-to-fine Gauss-Newton (Sec. 3.2).  Returns (v on the finest level,
    list of per-level report dicts, coarsest first)."""
    lib = load_library()
    dev = T.device
    for t, name in ((T, "T"), (R, "R")):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or \
                t.numel() != int(torch.Size(problem.image_shape).numel()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of the image shape")
    v = torch.empty(problem.velocity_shape, device=dev, dtype=torch.float32)
    o = _SolveOpts()
    lib.lgnk_solve_opts_default(ctypes.byref(o))
    for k, val in opts.items():
        if not hasattr(o, k):
            raise KeyError(f"unknown solve option {k}")
        setattr(o, k, type(getattr(o, k))(val))
    reps = (_SolveReport * levels)()
    pc = problem.to_c()
    st = lib.lgnk_solve_multilevel(ctypes.byref(pc), int(levels),
                                   ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream),
                                   ctypes.c_size_t(mem_budget), _ptr(T), _ptr(R), _ptr(v), ctypes.byref(o),
                                   ctypes.cast(reps, ctypes.c_void_p))
    if st not in (0, 6, 7):
        raise LgnkError(st, lib.lgnk_last_error(None).decode())
    out = []
    for r in reps:
        d = {f: getattr(r, f) for f, _ in _SolveReport._fields_}
        d["status_name"] = STATUS.get(d["status"], str(d["status"]))
        out.append(d)
    return v, out


class WarmStart:
    """The learned warm-start network (lgnk_ws_*): predicts a stationary 2D
    starting velocity [B][2][m/2][m/2] from image pairs T, R [B][m][m]."""

    def __init__(self, image_m: int, base_channels: int, max_batch: int, scale: float, device=None):
        self.lib = load_library()
        self.m, self.c, self.max_batch, self.scale = int(image_m), int(base_channels), int(max_batch), float(scale)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        handle = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = self.lib.lgnk_ws_create(self.m, self.c, self.max_batch, ctypes.c_float(self.scale),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                         ctypes.byref(handle))
        if st != 0:
            raise LgnkError(st, "lgnk_ws_create rejected its arguments or could not allocate")
        self.handle = handle
        self.num_params = int(self.lib.lgnk_ws_num_params(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.lgnk_ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise LgnkError(st, self.lib.lgnk_ws_last_error(self.handle).decode())

    def _t(self, t, numel, name):
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != torch.float32 \
                or not t.is_contiguous() or t.numel() != numel:
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device} with {numel} elements")
        return _ptr(t)

    def _pair(self, T, R):
        if T.dim() == 2:
            T, R = T[None], R[None]
        B = T.shape[0]
        if B < 1 or B > self.max_batch:
            raise ValueError(f"batch {B} outside [1, {self.max_batch}]")
        n = B * self.m * self.m
        return B, self._t(T, n, "T"), self._t(R, n, "R")

    def set_params(self, params):
        p = torch.as_tensor(params, dtype=torch.float32).to(self.device).contiguous()
        self._check(self.lib.lgnk_ws_set_params(self.handle, self._t(p, self.num_params, "params")))
        torch.cuda.current_stream(self.device).synchronize()

    def params(self):
        out = torch.empty(self.num_params, device=self.device, dtype=torch.float32)
        self._check(self.lib.lgnk_ws_get_params(self.handle, _ptr(out)))
        return out

    def grads(self):
        out = torch.empty(self.num_params, device=self.device, dtype=torch.float32)
        self._check(self.lib.lgnk_ws_get_grads(self.handle, _ptr(out)))
        return out

    def predict(self, T, R, out=None):
        B, pT, pR = self._pair(T, R)
        h = self.m // 2
        v = out if out is not None else torch.empty((B, 2, h, h), device=self.device, dtype=torch.float32)
        self._check(self.lib.lgnk_ws_predict(self.handle, B, pT, pR, self._t(v, B * 2 * h * h, "out")))
        return v

    def train_step(self, T, R, v_target, lr: float, return_loss=True):
        B, pT, pR = self._pair(T, R)
        h = self.m // 2
        loss = ctypes.c_double()
        self._check(self.lib.lgnk_ws_train_step(self.handle, B, pT, pR, self._t(v_target, B * 2 * h * h, "v_target"),
                                                ctypes.c_float(lr), ctypes.byref(loss) if return_loss else None))
        return loss.value if return_loss else None


class LagrangianForward(torch.autograd.Function):
    """u1(v) as an autograd function: forward is lgnk_forward, backward is the
    hand-written J^T kernel (lgnk_jtvp), which recomputes the trajectory
    instead of storing it.  T is treated as a constant."""

    @staticmethod
    def forward(fctx, v, T, lctx):
        fctx.lctx = lctx
        fctx.save_for_backward(v, T)
        return lgnk_forward(lctx, v.contiguous(), T.contiguous())

    @staticmethod
    def backward(fctx, grad_u1):
        v, T = fctx.saved_tensors
        gv = lgnk_jtvp(fctx.lctx, v.contiguous(), T.contiguous(), grad_u1.contiguous().float())
        return gv, None, None


def lagrangian_forward(lctx: Context, v, T):
    return LagrangianForward.apply(v, T, lctx)
