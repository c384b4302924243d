"""Seeded synthetic inputs shaped like the registration problems of Sec. 4.

This module draws images and velocity fields and nothing else: it holds no
step of the registration method (no characteristic tracing, no grid
interpolation, no regularizer).  Reference images are made by evaluating the
analytic template at analytically displaced coordinates, so a reference never
comes from either implementation of the method.

Arrays follow the library's layout: an image on a grid with ``m = (m_x, m_y
[, m_z])`` cells is a float array of numpy shape ``(m_z, m_y, m_x)`` (x fastest);
a velocity with ``K`` time nodes is ``(K, d, m_z, m_y, m_x)``; component ``c``
is the velocity along axis ``c`` (x = 0).

Workloads (sizes from the paper's experiment classes, Sec. 4.2-4.5):

* ``2d_transport_64``   64^2 template of 6 Gaussian blobs on (0,1)^2, velocity
  32^2 x 2, stationary, N = 4 RK4 steps, diffusion alpha = 1e-2.
* ``2d_continuity_256`` 256^2 unit-mass density of 20 Gaussians, velocity
  128^2 x 2 on 5 time nodes, N = 16, elastic alpha = 1e-3, noise 0.01.
* ``3d_transport_128``  128^3 nested-ellipsoid phantom, noise 0.01, velocity
  64^3 x 3, stationary, N = 8, diffusion alpha = 1e-2; reference displaced by
  up to 8 voxels.
* ``3d_continuity_brain`` 192 x 224 x 160 shell phantom on
  (0,1.2) x (0,1.4) x (0,1), velocity 96 x 112 x 80 x 3 on 9 time nodes,
  N = 16, diffusion alpha = 1e-3, continuity.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "GridSpec", "Workload", "WORKLOADS", "centres", "gaussian_blobs",
    "smooth_field", "ellipsoid_phantom", "shell_phantom", "make_inputs",
    "random_velocity", "prior_velocity", "warmstart_init", "warmstart_pair",
]


@dataclass(frozen=True)
class GridSpec:
    """Cell-centred grid: ``m`` cells per axis (x first) on the box [lo, hi]."""
    m: tuple
    lo: tuple
    hi: tuple

    @property
    def d(self) -> int:
        return len(self.m)

    @property
    def shape(self) -> tuple:
        return tuple(reversed(self.m))

    @property
    def h(self) -> tuple:
        return tuple((b - a) / n for a, b, n in zip(self.lo, self.hi, self.m))


@dataclass(frozen=True)
class Workload:
    name: str
    image: GridSpec
    velocity: GridSpec
    time_nodes: int
    rk4_steps: int
    model: str            # "transport" | "continuity"
    regularizer: str      # "diffusion" | "curvature" | "elastic"
    alpha: float
    gamma: float = 0.0
    extra: dict = field(default_factory=dict)


def _box(m, lo=None, hi=None):
    d = len(m)
    lo = tuple([0.0] * d) if lo is None else tuple(lo)
    hi = tuple([1.0] * d) if hi is None else tuple(hi)
    return GridSpec(tuple(m), lo, hi)


WORKLOADS = {
    "2d_transport_64": Workload(
        "2d_transport_64", _box((64, 64)), _box((32, 32)), 1, 4,
        "transport", "diffusion", 1e-2, 0.0),
    "2d_continuity_256": Workload(
        "2d_continuity_256", _box((256, 256)), _box((128, 128)), 5, 16,
        "continuity", "elastic", 1e-3, 0.0, {"mu": 1.0, "lam": 0.0}),
    "3d_transport_128": Workload(
        "3d_transport_128", _box((128, 128, 128)), _box((64, 64, 64)), 1, 8,
        "transport", "diffusion", 1e-2, 0.0),
    "3d_continuity_brain": Workload(
        "3d_continuity_brain", _box((192, 224, 160), hi=(1.2, 1.4, 1.0)),
        _box((96, 112, 80), hi=(1.2, 1.4, 1.0)), 9, 16,
        "continuity", "diffusion", 1e-3, 0.0),
    # image pairs of the learned warm start (128^2 images, stationary 64^2 velocity)
    "2d_warmstart_128": Workload(
        "2d_warmstart_128", _box((128, 128)), _box((64, 64)), 1, 4,
        "transport", "diffusion", 1e-3, 0.0),
}

WARMSTART_MAX_DISP_PX = 10.0


def centres(g: GridSpec):
    """Coordinate arrays (x, y[, z]) of the cell centres, each of shape g.shape."""
    axes = [g.lo[a] + (np.arange(g.m[a]) + 0.5) * g.h[a] for a in range(g.d)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return list(reversed(mesh))


def _window(coords, lo, hi):
    w = 1.0
    for c, a, b in zip(coords, lo, hi):
        w = w * np.sin(np.pi * (c - a) / (b - a)) ** 2
    return w


def gaussian_blobs(coords, params):
    """Sum of isotropic Gaussians ``a exp(-|x-c|^2 / (2 s^2))`` at the given coordinates."""
    out = 0.0
    for amp, sig, ctr in params:
        r2 = sum((x - c) ** 2 for x, c in zip(coords, ctr))
        out = out + amp * np.exp(-r2 / (2.0 * sig * sig))
    return out


def _blob_params(rng, n, d, sigma, amp, lo, hi):
    ps = []
    for _ in range(n):
        ps.append((rng.uniform(*amp), rng.uniform(*sigma),
                   tuple(rng.uniform(lo, hi, size=d))))
    return ps


def _fourier_modes(rng, d, n_modes, kmax=3):
    modes = []
    for _ in range(n_modes):
        k = rng.integers(1, kmax + 1, size=d)
        phase = rng.uniform(0.0, 2.0 * np.pi)
        dirn = rng.normal(size=d)
        modes.append((k, phase, dirn))
    return modes


def smooth_field(coords, lo, hi, modes, window=True):
    """Vector field ``sum_j dir_j sin(2 pi k_j . xhat + phi_j)`` (xhat: box-normalised),
    optionally windowed by prod sin^2 so that it vanishes on the box boundary."""
    d = len(coords)
    xh = [(c - a) / (b - a) for c, a, b in zip(coords, lo, hi)]
    out = [np.zeros_like(coords[0]) for _ in range(d)]
    for k, phase, dirn in modes:
        s = np.sin(2.0 * np.pi * sum(kk * x for kk, x in zip(k, xh)) + phase)
        for c in range(d):
            out[c] = out[c] + dirn[c] * s
    if window:
        w = _window(coords, lo, hi)
        out = [o * w for o in out]
    return out


def _scale_to(field_list, amplitude):
    mag = np.sqrt(sum(f * f for f in field_list))
    mx = float(mag.max())
    if mx == 0.0:
        return field_list
    return [f * (amplitude / mx) for f in field_list]


def random_velocity(g: GridSpec, time_nodes: int, amplitude: float, seed: int,
                    n_modes: int = 4, dtype=np.float64):
    """Smooth windowed velocity of shape (K, d, *g.shape); each time node has its own
    modes blended linearly in time, max |v| = amplitude (physical units per unit time)."""
    rng = np.random.default_rng(seed)
    coords = centres(g)
    a = _fourier_modes(rng, g.d, n_modes)
    b = _fourier_modes(rng, g.d, n_modes)
    fa = _scale_to(smooth_field(coords, g.lo, g.hi, a), amplitude)
    fb = _scale_to(smooth_field(coords, g.lo, g.hi, b), amplitude)
    v = np.zeros((time_nodes, g.d) + g.shape)
    for j in range(time_nodes):
        s = 0.0 if time_nodes == 1 else j / (time_nodes - 1)
        for c in range(g.d):
            v[j, c] = (1.0 - s) * fa[c] + s * fb[c] if time_nodes > 1 else fa[c]
    return v.astype(dtype)


def ellipsoid_phantom(coords, rng, lo, hi):
    """Three nested ellipsoids with tanh-edged boundaries and smooth intensity ramps."""
    d = len(coords)
    ctr = [a + (b - a) * (0.5 + rng.uniform(-0.03, 0.03)) for a, b in zip(lo, hi)]
    out = np.zeros_like(coords[0])
    for level, (scale, inten) in enumerate(((0.38, 0.5), (0.26, 0.3), (0.14, 0.2))):
        radii = [(b - a) * scale * rng.uniform(0.85, 1.15) for a, b in zip(lo, hi)]
        r = np.sqrt(sum(((x - c) / rr) ** 2 for x, c, rr in zip(coords, ctr, radii)))
        ramp = 1.0 + 0.3 * (coords[0] - ctr[0]) / (hi[0] - lo[0])
        out = out + inten * ramp * 0.5 * (1.0 - np.tanh((r - 1.0) / 0.06))
    return out


def shell_phantom(coords, rng, lo, hi):
    """Brain-like phantom: ellipsoidal shells with smooth intensities, positive everywhere inside."""
    ctr = [a + 0.5 * (b - a) for a, b in zip(lo, hi)]
    out = np.zeros_like(coords[0])
    for scale, inten in ((0.42, 0.6), (0.33, 0.9), (0.22, 0.5), (0.12, 0.3)):
        radii = [(b - a) * scale * rng.uniform(0.9, 1.1) for a, b in zip(lo, hi)]
        r = np.sqrt(sum(((x - c) / rr) ** 2 for x, c, rr in zip(coords, ctr, radii)))
        out = out + inten * 0.5 * (1.0 - np.tanh((r - 1.0) / 0.05))
    return out


def make_inputs(name: str, seed: int = 0, dtype=np.float32):
    """Template T, reference R and a smooth velocity v0 (linearisation point for
    throughput runs, never the solution) for one named workload.

    The reference is the analytic template at displaced coordinates x - s(x)
    (transport) or the template's Gaussians moved by s (continuity), with s a
    windowed Fourier displacement; noise is added where the workload says so.
    """
    wl = WORKLOADS[name]
    g = wl.image
    rng = np.random.default_rng(seed)
    coords = centres(g)
    h = min(g.h)
    if name == "2d_transport_64":
        params = _blob_params(rng, 6, 2, (0.05, 0.15), (0.5, 1.0), 0.2, 0.8)
        T = gaussian_blobs(coords, params)
        s = _scale_to(smooth_field(coords, g.lo, g.hi, _fourier_modes(rng, 2, 4)), 0.1)
        R = gaussian_blobs([c - sc for c, sc in zip(coords, s)], params)
        vamp = 0.1
    elif name == "2d_continuity_256":
        params = _blob_params(rng, 20, 2, (0.03, 0.08), (0.2, 1.0), 0.25, 0.75)
        T = gaussian_blobs(coords, params)
        cell = float(np.prod(g.h))
        mass = T.sum() * cell
        T = T / mass
        modes = _fourier_modes(rng, 2, 4)
        ctrs = [np.array(p[2]) for p in params]
        cc = [np.array([c[a] for c in ctrs]) for a in range(2)]
        sc = _scale_to(smooth_field(cc, g.lo, g.hi, modes), 0.15)
        moved = [(amp, sig, tuple(ctrs[i] + np.array([sc[0][i], sc[1][i]])))
                 for i, (amp, sig, _) in enumerate(params)]
        R = gaussian_blobs(coords, moved) / mass + rng.normal(0.0, 0.01, size=T.shape)
        vamp = 0.15
    elif name == "3d_transport_128":
        T = ellipsoid_phantom(coords, np.random.default_rng(seed), g.lo, g.hi)
        s = _scale_to(smooth_field(coords, g.lo, g.hi, _fourier_modes(rng, 3, 4)), 8 * h)
        R = ellipsoid_phantom([c - sc for c, sc in zip(coords, s)],
                              np.random.default_rng(seed), g.lo, g.hi)
        T = T + rng.normal(0.0, 0.01, size=T.shape)
        R = R + rng.normal(0.0, 0.01, size=R.shape)
        vamp = 8 * h
    elif name == "3d_continuity_brain":
        T = shell_phantom(coords, np.random.default_rng(seed), g.lo, g.hi)
        s = _scale_to(smooth_field(coords, g.lo, g.hi, _fourier_modes(rng, 3, 4)), 6 * h)
        R = shell_phantom([c - sc for c, sc in zip(coords, s)],
                          np.random.default_rng(seed), g.lo, g.hi)
        cell = float(np.prod(g.h))
        mt, mr = T.sum() * cell, R.sum() * cell
        T, R = T / mt, R / mr
        vamp = 6 * h
    elif name == "2d_warmstart_128":
        T, v_true = warmstart_pair(0, seed)
        return {"workload": wl, "T": T.astype(dtype), "R": None, "v0": v_true.astype(dtype)}
    else:
        raise KeyError(name)
    v0 = random_velocity(wl.velocity, wl.time_nodes, vamp, seed + 7)
    return {
        "workload": wl,
        "T": np.ascontiguousarray(T, dtype=dtype),
        "R": np.ascontiguousarray(R, dtype=dtype),
        "v0": np.ascontiguousarray(v0, dtype=dtype),
    }


def warmstart_init(c: int, seed: int):
    """Seeded He-normal initial parameters (zero biases) of the warm-start
    encoder-decoder with c base channels, as one flat float32 vector in the
    layer order e0, e1, e2, e3, d2, d1, out (W [c_out][c_in][3][3], then b)."""
    shapes = [(2, c), (c, 2 * c), (2 * c, 4 * c), (4 * c, 8 * c), (8 * c, 4 * c), (4 * c, 2 * c), (2 * c, 2)]
    rng = np.random.default_rng(seed)
    out = []
    for ci, co in shapes:
        out.append(rng.normal(0.0, np.sqrt(2.0 / (9 * ci)), size=co * ci * 9))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def warmstart_pair(index: int, seed: int = 0):
    """Template and true velocity of image pair `index` for the learned warm
    start: T = 4 to 9 random Gaussian blobs on the 128^2 grid; v drawn from the
    diffusion prior (prior_velocity) with a maximum displacement of 10 pixels.
    The reference R = T moved by v is computed on the device by the forward map.
    Returns (T [128][128] float32, v [1][2][64][64] float32)."""
    wl = WORKLOADS["2d_warmstart_128"]
    rng = np.random.default_rng([seed, index])
    coords = centres(wl.image)
    params = _blob_params(rng, int(rng.integers(4, 10)), 2, (0.04, 0.12), (0.4, 1.0), 0.15, 0.85)
    T = gaussian_blobs(coords, params).astype(np.float32)
    v = prior_velocity(wl.velocity, wl.alpha, WARMSTART_MAX_DISP_PX * min(wl.image.h),
                       int(rng.integers(2 ** 31)))
    return T, v


def prior_velocity(g: GridSpec, alpha: float, max_disp: float, seed: int, eps: float = 1e-3):
    """Stationary velocity (1, d, *g.shape) drawn from the regularizer prior:
    white Gaussian noise filtered in Fourier space by 1 / (alpha |k|^2 + eps)
    (the inverse of a diffusion operator), windowed to vanish on the boundary
    and scaled to a maximum magnitude of max_disp."""
    rng = np.random.default_rng(seed)
    coords = centres(g)
    freqs = np.meshgrid(*[np.fft.fftfreq(n, d=h) for n, h in zip(reversed(g.m), reversed(g.h))], indexing="ij")
    k2 = sum((2 * np.pi * f) ** 2 for f in freqs)
    filt = 1.0 / (alpha * k2 + eps)
    comps = []
    for _ in range(g.d):
        noise = rng.normal(size=g.shape)
        comps.append(np.real(np.fft.ifftn(np.fft.fftn(noise) * filt)))
    w = _window(coords, g.lo, g.hi)
    comps = _scale_to([c * w for c in comps], max_disp)
    return np.stack(comps)[None].astype(np.float32)
