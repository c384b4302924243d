"""Seeded parity cases shared by the GPU tests: the same inputs go to the CUDA
path and to the oracle."""
import numpy as np

from oracle import lagrangian as L
from oracle.objective import Problem as OProblem
from paper_1703_04446_gb300 import synth

# name: (image m, velocity m, lo, hi, K, N, model, regularizer, v amplitude in image cells)
CASES = {
    "2d_transport_64": ((64, 64), (32, 32), (0, 0), (1, 1), 1, 4, "transport", "diffusion", 4.0),
    "2d_transport_ragged_K3": ((37, 29), (19, 15), (-0.2, 0.0), (1.1, 1.3), 3, 5, "transport", "curvature", 3.0),
    "2d_continuity_K5": ((48, 48), (24, 24), (0, 0), (1, 1), 5, 16, "continuity", "elastic", 3.0),
    "2d_transport_tiny": ((11, 9), (6, 5), (0, 0), (1.1, 0.9), 1, 3, "transport", "diffusion", 1.5),
    "3d_transport_ragged": ((20, 18, 17), (10, 9, 9), (0, 0, 0), (1, 1, 1), 1, 8, "transport", "diffusion", 2.5),
    "3d_transport_K2_N1": ((12, 12, 12), (6, 6, 6), (0, 0, 0), (1, 1, 1), 2, 1, "transport", "diffusion", 2.0),
    "3d_continuity_K2": ((16, 20, 12), (8, 10, 6), (0, 0, 0), (1.0, 1.25, 0.75), 2, 3, "continuity", "diffusion", 2.0),
    "2d_continuity_hat_K3": ((40, 36), (20, 18), (0, 0), (1.0, 0.9), 3, 6, "continuity", "diffusion", 2.5),
    "2d_continuity_hat_widest": ((32, 32), (16, 16), (0, 0), (1, 1), 1, 4, "continuity", "diffusion", 2.0),
    "3d_continuity_hat_K2": ((18, 16, 14), (9, 8, 7), (0, 0, 0), (1.0, 0.9, 0.8), 2, 3, "continuity", "diffusion", 2.0),
}

# general-width PIC cases: particle half-width delta in units of the smallest image cell
PIC_DELTA = {"2d_continuity_hat_K3": 1.7, "2d_continuity_hat_widest": 3.5, "3d_continuity_hat_K2": 0.6}


def make_case(name, seed=0, alpha=1e-2, gamma=1e-3):
    im, vm, lo, hi, K, N, model, reg, amp = CASES[name]
    d = len(im)
    lo = tuple(float(a) for a in lo)
    hi = tuple(float(a) for a in hi)
    ig = synth.GridSpec(im, lo, hi)
    vg = synth.GridSpec(vm, lo, hi)
    rng = np.random.default_rng(seed)
    coords = synth.centres(ig)
    ctr = [lo[a] + (hi[a] - lo[a]) * rng.uniform(0.35, 0.65) for a in range(d)]
    ext = min(hi[a] - lo[a] for a in range(d))
    blobs = [(1.0, 0.18 * ext, tuple(ctr)),
             (0.7, 0.08 * ext, tuple(c + 0.1 * ext for c in ctr)),
             (0.5, 0.12 * ext, tuple(c - 0.12 * ext for c in ctr))]
    T = synth.gaussian_blobs(coords, blobs)
    R = synth.gaussian_blobs([c - 0.03 * ext for c in coords], blobs)
    h = min(ig.h)
    v = synth.random_velocity(vg, K, amp * h, seed + 1)
    dv = synth.random_velocity(vg, K, 0.5 * amp * h, seed + 2) + 0.1 * amp * h * rng.normal(size=v.shape)
    r = rng.normal(size=T.shape)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    arrays = {k: f32(a) for k, a in dict(T=T, R=R, v=v, dv=dv, r=r).items()}
    delta = PIC_DELTA[name] * h if name in PIC_DELTA else None
    oprob = OProblem(L.Grid(im, lo, hi), L.Grid(vm, lo, hi), K=K, N=N, model=model, reg=reg, alpha=alpha,
                     gamma=gamma, mu=1.0, lam=0.5, delta=delta)
    gprob = dict(image_m=im, velocity_m=vm, time_nodes=K, rk4_steps=N, model=model, regularizer=reg, alpha=alpha,
                 gamma=gamma, image_lo=lo, image_hi=hi, velocity_lo=lo, velocity_hi=hi, mu_lame=1.0,
                 lambda_lame=0.5, pic_delta=delta or 0.0)
    return oprob, gprob, arrays


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
