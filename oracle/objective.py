"""Discrete objective of the oracle (Sec. 3.2, Eq. 9): SSD distance (Eq. 10),
regularizers (Sec. 2.1), gradient and Gauss-Newton Hessian.  FP64, numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper taken here:
* ``B`` is the forward-difference gradient between neighbouring cell centres
  (interior faces only), so ``A = B^T B`` is the homogeneous-Neumann Laplacian,
  diagonalised by the DCT-II (Sec. 3.2, Toeplitz-plus-Hankel structure).
* The time weight ``dt`` in ``d_v S = dt h^d B^T B v`` is the time-cell width of
  the velocity grid, 1/(K-1), with every time node weighted equally; a
  stationary field (K = 1) has weight 1 (Sec. 2.1, time integral dropped).
  ``h^d`` is the velocity grid's cell volume for S and the image's for D.
* ``S = 1/2 dt h^d |B v|^2``, ``J = D + alpha S``; gamma enters only the Hessian.
* The Hessian of SSD is ``h^d`` times the identity on the image grid (the
  printed ``h^3 I_n`` is read as ``h^d I_M``).
* Elastic regularizer (Navier-Lame, mu |grad v|^2 + (lam + mu) (div v)^2, div by
  centred differences with mirrored ends): the paper names elastic models
  but never defines one; pinned by closed forms on linear fields and by the
  lam = -mu reduction to mu times diffusion.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lagrangian import Grid, final_state, jtvp, jvp


@dataclass
class Problem:
    """Eq. 9 with SSD: grids, K velocity time nodes, N RK4 steps, model flag,
    regularizer name and weights."""
    igrid: Grid
    vgrid: Grid
    K: int
    N: int
    model: str = "transport"        # "transport" (Eq. 2) | "continuity" (Eq. 3)
    reg: str = "diffusion"          # "diffusion" | "curvature" | "elastic"
    alpha: float = 1e-2
    gamma: float = 0.0
    mu: float = 1.0
    lam: float = 0.0
    delta: float = None             # PIC half-width (continuity); None: width = cell size

    @property
    def time_weight(self) -> float:
        return 1.0 if self.K == 1 else 1.0 / (self.K - 1)

    @property
    def vshape(self):
        return (self.K, self.vgrid.d) + self.vgrid.shape


# ---------------------------------------------------------------------------
# Difference operators on one scalar grid function
# ---------------------------------------------------------------------------

def _axis(grid: Grid, a: int) -> int:
    """numpy axis of grid axis a (arrays are stored (z, y, x))."""
    return grid.d - 1 - a


def grad_forward(x: np.ndarray, grid: Grid):
    """B x: forward differences between neighbouring cell centres, per axis."""
    return [np.diff(x, axis=_axis(grid, a)) / grid.h[a] for a in range(grid.d)]


def grad_forward_T(g, grid: Grid) -> np.ndarray:
    """B^T g for face values g (list per axis)."""
    out = np.zeros(grid.shape)
    for a in range(grid.d):
        ax = _axis(grid, a)
        ga = g[a] / grid.h[a]
        lo = [slice(None)] * grid.d
        hi = [slice(None)] * grid.d
        lo[ax] = slice(0, grid.m[a] - 1)
        hi[ax] = slice(1, grid.m[a])
        out[tuple(lo)] -= ga
        out[tuple(hi)] += ga
    return out


def laplacian_neumann(x: np.ndarray, grid: Grid) -> np.ndarray:
    """A x = B^T B x (positive semi-definite Neumann Laplacian)."""
    return grad_forward_T(grad_forward(x, grid), grid)


def div_centred(u, grid: Grid) -> np.ndarray:
    """Centred-difference divergence of the vector field u (list of d components),
    one-sided at the ends (mirrored ghost value)."""
    out = np.zeros(grid.shape)
    for a in range(grid.d):
        ax = _axis(grid, a)
        p = np.concatenate([np.take(u[a], [0], axis=ax), u[a], np.take(u[a], [-1], axis=ax)], axis=ax)
        n = grid.m[a]
        out += (np.take(p, np.arange(2, n + 2), axis=ax) - np.take(p, np.arange(0, n), axis=ax)) / (2 * grid.h[a])
    return out


def div_centred_T(s: np.ndarray, grid: Grid):
    """Transpose of ``div_centred``: returns the list of d component fields."""
    out = []
    for a in range(grid.d):
        ax = _axis(grid, a)
        n = grid.m[a]
        comp = np.zeros(grid.shape)
        c = s / (2 * grid.h[a])
        for i in range(n):
            src = np.take(c, [i], axis=ax)
            up, dn = min(i + 1, n - 1), max(i - 1, 0)
            sl_up = [slice(None)] * grid.d
            sl_dn = [slice(None)] * grid.d
            sl_up[ax] = slice(up, up + 1)
            sl_dn[ax] = slice(dn, dn + 1)
            comp[tuple(sl_up)] += src
            comp[tuple(sl_dn)] -= src
        out.append(comp)
    return out


# ---------------------------------------------------------------------------
# Regularizers (Sec. 2.1) on the full velocity (K, d, *grid)
# ---------------------------------------------------------------------------

def reg_value(prob: Problem, v: np.ndarray) -> float:
    """S(v) = 1/2 dt h^d |B v|^2 (diffusion), 1/2 dt h^d |A v|^2 (curvature),
    or the elastic form."""
    g = prob.vgrid
    w = prob.time_weight * g.cell_volume
    s = 0.0
    for j in range(prob.K):
        if prob.reg == "elastic":
            s += prob.mu * sum(np.sum(f ** 2) for c in range(g.d) for f in grad_forward(v[j, c], g))
            s += (prob.lam + prob.mu) * np.sum(div_centred([v[j, c] for c in range(g.d)], g) ** 2)
            continue
        for c in range(g.d):
            if prob.reg == "diffusion":
                s += sum(np.sum(f ** 2) for f in grad_forward(v[j, c], g))
            elif prob.reg == "curvature":
                s += np.sum(laplacian_neumann(v[j, c], g) ** 2)
            else:
                raise ValueError(prob.reg)
    return 0.5 * w * s


def reg_operator(prob: Problem, x: np.ndarray) -> np.ndarray:
    """dt h^d B^T B x (the Hessian of S; its gradient at x)."""
    g = prob.vgrid
    w = prob.time_weight * g.cell_volume
    out = np.zeros_like(x, dtype=np.float64)
    for j in range(prob.K):
        if prob.reg == "elastic":
            dv = div_centred_T(div_centred([x[j, c] for c in range(g.d)], g), g)
            for c in range(g.d):
                out[j, c] = prob.mu * laplacian_neumann(x[j, c], g) + (prob.lam + prob.mu) * dv[c]
            continue
        for c in range(g.d):
            if prob.reg == "diffusion":
                out[j, c] = laplacian_neumann(x[j, c], g)
            elif prob.reg == "curvature":
                out[j, c] = laplacian_neumann(laplacian_neumann(x[j, c], g), g)
            else:
                raise ValueError(prob.reg)
    return w * out


# ---------------------------------------------------------------------------
# Objective, gradient, Gauss-Newton Hessian (Sec. 3.2)
# ---------------------------------------------------------------------------

def ssd(u1: np.ndarray, R: np.ndarray, igrid: Grid) -> float:
    """Eq. 10: D = h^d/2 res^T res, res = u1 - R."""
    res = np.asarray(u1, dtype=np.float64) - np.asarray(R, dtype=np.float64)
    return 0.5 * igrid.cell_volume * float(np.sum(res * res))


def objective(prob: Problem, v, T, R):
    """J(v) = D(u1(v), R) + alpha S(v) (Eq. 9).  Returns (J, D, S, u1)."""
    u1, _ = final_state(prob.model, v, prob.vgrid, T, prob.igrid, prob.N, prob.delta)
    D = ssd(u1, R, prob.igrid)
    S = reg_value(prob, v)
    return D + prob.alpha * S, D, S, u1


def gradient(prob: Problem, v, T, R):
    """d_v J = (d_v u1)^T h^d res + alpha dt h^d B^T B v."""
    u1, _ = final_state(prob.model, v, prob.vgrid, T, prob.igrid, prob.N, prob.delta)
    res = u1 - np.asarray(R, dtype=np.float64)
    g = jtvp(prob.model, v, prob.vgrid, T, prob.igrid, prob.N, prob.igrid.cell_volume * res, prob.delta)
    return g + prob.alpha * reg_operator(prob, v)


def hessvec(prob: Problem, v, T, p):
    """H p = (d_v u1)^T h^d (d_v u1) p + alpha dt h^d B^T B p + gamma p."""
    du = jvp(prob.model, v, prob.vgrid, T, prob.igrid, prob.N, p, prob.delta)
    Hp = jtvp(prob.model, v, prob.vgrid, T, prob.igrid, prob.N, prob.igrid.cell_volume * du, prob.delta)
    return Hp + prob.alpha * reg_operator(prob, p) + prob.gamma * np.asarray(p, dtype=np.float64)
