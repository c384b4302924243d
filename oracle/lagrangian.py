"""Lagrangian forward maps of the oracle (Sec. 3.1): characteristics, final
states and their exact discrete derivatives.  FP64, numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions
-----------
* A grid has ``m = (m_x, m_y[, m_z])`` cells of width ``h_a = (hi_a - lo_a)/m_a``;
  its points are the cell centres ``lo_a + (i + 1/2) h_a`` (Sec. 3, "cell-centered
  points").  Grid arrays have numpy shape ``(m_z, m_y, m_x)`` (x fastest).
* Point sets are arrays ``(d, P)``; row ``a`` is the coordinate along axis ``a``.
* A velocity with ``K`` time nodes has shape ``(K, d, *grid.shape)``; node ``j``
  sits at ``t_j = j / (K - 1)``; ``K = 1`` is a stationary field.

Readings of the paper taken here (where it is silent or garbled):
* Interpolation extends grid data by zero outside the grid (images are
  compactly supported, Sec. 2); the cell of a point is ``floor`` of its
  continuous index, so derivatives at a cell face are those of the upper cell.
* Alg. 1's third stage: standard RK4 (``y3 = y + dt * v3``), the printed
  ``dt/2`` being a typo (its own derivative line uses ``dt * D3``).
* Transport traces backward from t = 1 (dt = -1/N), continuity forward from
  t = 0 (dt = +1/N); stage times t_k, t_k + dt/2, t_k + dt/2, t_k + dt.
* The push-forward matrix with particle width equal to the cell size is the
  transpose of the linear interpolation matrix (Sec. 3.1, end of Step 2).
* The general PIC kernel (Eqs. 7-8 with any width delta): each particle is the
  tensor product of normalised 1D hats of half-width delta (unit mass), and
  cell i receives the exact integral of the particle over the cell (Eq. 8), so
  the columns of F sum to one for any delta and h.  ``delta=None`` selects the
  width-equals-cell-size case above.
"""
from __future__ import annotations

import itertools

import numpy as np


class Grid:
    """Cell-centred regular grid (Sec. 3)."""

    def __init__(self, m, lo=None, hi=None):
        self.m = tuple(int(a) for a in m)
        self.d = len(self.m)
        self.lo = np.zeros(self.d) if lo is None else np.asarray(lo, dtype=np.float64)
        self.hi = np.ones(self.d) if hi is None else np.asarray(hi, dtype=np.float64)
        self.h = (self.hi - self.lo) / np.asarray(self.m, dtype=np.float64)

    @property
    def shape(self):
        return tuple(reversed(self.m))

    @property
    def size(self):
        return int(np.prod(self.m))

    @property
    def cell_volume(self):
        return float(np.prod(self.h))


def cell_centres(grid: Grid) -> np.ndarray:
    """Cell centres x_c as a (d, M) array, ordered like the flattened grid array."""
    axes = [grid.lo[a] + (np.arange(grid.m[a]) + 0.5) * grid.h[a] for a in range(grid.d)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return np.stack([mesh[grid.d - 1 - a].ravel() for a in range(grid.d)])


def _corners(grid: Grid, p: np.ndarray):
    """For each of the 2^d corners of the cell holding each point: the flat index
    (or -1 when the corner lies outside the grid), the multilinear weight, and
    the derivative of that weight along every axis."""
    d = grid.d
    xi = [(p[a] - grid.lo[a]) / grid.h[a] - 0.5 for a in range(d)]
    # a point on a node in exact arithmetic must take the cell to its right
    # (floor, Sec. 3.1 derivative of the interpolant); (p - lo) / h - 1/2 can
    # land a few ulps below the integer, so such values are snapped to it
    xi = [np.where(np.abs(x - np.rint(x)) <= 16.0 * np.finfo(np.float64).eps * np.maximum(1.0, np.abs(x)),
                   np.rint(x), x) for x in xi]
    base = [np.floor(x).astype(np.int64) for x in xi]
    frac = [x - b for x, b in zip(xi, base)]
    strides = [int(np.prod(grid.m[:a])) for a in range(d)]
    out = []
    for corner in itertools.product((0, 1), repeat=d):
        idx = [base[a] + corner[a] for a in range(d)]
        inside = np.ones(p.shape[1], dtype=bool)
        flat = np.zeros(p.shape[1], dtype=np.int64)
        for a in range(d):
            inside &= (idx[a] >= 0) & (idx[a] < grid.m[a])
            flat += idx[a] * strides[a]
        flat = np.where(inside, flat, -1)
        w1 = [frac[a] if corner[a] else 1.0 - frac[a] for a in range(d)]
        dw1 = [(1.0 if corner[a] else -1.0) / grid.h[a] for a in range(d)]
        w = np.prod(w1, axis=0)
        dw = []
        for a in range(d):
            g = np.full(p.shape[1], dw1[a])
            for b in range(d):
                if b != a:
                    g = g * w1[b]
            dw.append(g)
        out.append((flat, w, np.stack(dw)))
    return out


def interpolate(F: np.ndarray, grid: Grid, p: np.ndarray, gradient: bool = False):
    """Linear (bi/trilinear) interpolation T(y) of the grid function F at points p
    (Eq. 6 with the linear model of Sec. 3.1), and optionally its gradient
    grad T(y) (Sec. 3.2, derivative of the transport final state)."""
    f = F.reshape(-1)
    val = np.zeros(p.shape[1])
    grad = np.zeros(p.shape) if gradient else None
    for flat, w, dw in _corners(grid, p):
        inside = flat >= 0
        fv = np.where(inside, f[np.where(inside, flat, 0)], 0.0)
        val += w * fv
        if gradient:
            grad += dw * fv
    return (val, grad) if gradient else val


def scatter(values: np.ndarray, grid: Grid, p: np.ndarray) -> np.ndarray:
    """Transpose of ``interpolate``: out = P(p)^T values, dropping corners outside
    the grid.  Used as the PIC push-forward (Eqs. 7-8 with width = cell size)."""
    out = np.zeros(grid.size)
    for flat, w, _ in _corners(grid, p):
        inside = flat >= 0
        np.add.at(out, flat[inside], (w * values)[inside])
    return out.reshape(grid.shape)


def scatter_gradient(values: np.ndarray, dp: np.ndarray, grid: Grid, p: np.ndarray) -> np.ndarray:
    """out_i = sum_j values_j (d w_i / d y)(p_j) . dp_j: the derivative of
    ``scatter(values, grid, p)`` along the point displacement dp (Sec. 3.2,
    continuity derivative d_y(F(y) T))."""
    out = np.zeros(grid.size)
    for flat, _, dw in _corners(grid, p):
        inside = flat >= 0
        contrib = values * np.sum(dw * dp, axis=0)
        np.add.at(out, flat[inside], contrib[inside])
    return out.reshape(grid.shape)


def _hat_cdf(s):
    """Integral of the unit-mass hat max(0, 1 - |x|) from -inf to s."""
    s = np.clip(s, -1.0, 1.0)
    return np.where(s <= 0.0, 0.5 * (1.0 + s) ** 2, 1.0 - 0.5 * (1.0 - s) ** 2)


def _hat(s):
    return np.maximum(0.0, 1.0 - np.abs(s))


def _hat_cells(grid: Grid, p: np.ndarray, delta: float):
    """For every cell that the hat particle of half-width delta at each point can
    overlap: the flat index (-1 outside the grid), the mass fraction (Eq. 8,
    exact integral of the particle over the cell) and its derivative with
    respect to the particle position, per axis."""
    d = grid.d
    per_axis = []
    for a in range(d):
        lo = np.floor((p[a] - delta - grid.lo[a]) / grid.h[a]).astype(np.int64)
        hi = np.floor((p[a] + delta - grid.lo[a]) / grid.h[a]).astype(np.int64)
        n = int((hi - lo).max()) + 1 if p.shape[1] else 1
        cells = []
        for o in range(n):
            i = lo + o
            e0 = grid.lo[a] + i * grid.h[a]          # faces of cell i
            e1 = e0 + grid.h[a]
            w = _hat_cdf((e1 - p[a]) / delta) - _hat_cdf((e0 - p[a]) / delta)
            dw = (_hat((e0 - p[a]) / delta) - _hat((e1 - p[a]) / delta)) / delta
            cells.append((i, w, dw))
        per_axis.append(cells)
    strides = [int(np.prod(grid.m[:a])) for a in range(d)]
    out = []
    for combo in itertools.product(*per_axis):
        inside = np.ones(p.shape[1], dtype=bool)
        flat = np.zeros(p.shape[1], dtype=np.int64)
        for a, (i, _, _) in enumerate(combo):
            inside &= (i >= 0) & (i < grid.m[a])
            flat += i * strides[a]
        w = np.prod([c[1] for c in combo], axis=0)
        dw = []
        for a in range(d):
            g = combo[a][2].copy()
            for b in range(d):
                if b != a:
                    g = g * combo[b][1]
            dw.append(g)
        out.append((np.where(inside, flat, -1), w, np.stack(dw)))
    return out


def scatter_hat(values: np.ndarray, grid: Grid, p: np.ndarray, delta: float) -> np.ndarray:
    """PIC push-forward with hat particles of half-width delta (Eqs. 7-8):
    out_i = sum_j values_j F_ij, F_ij = integral over cell i of particle j."""
    out = np.zeros(grid.size)
    for flat, w, _ in _hat_cells(grid, p, delta):
        inside = flat >= 0
        np.add.at(out, flat[inside], (w * values)[inside])
    return out.reshape(grid.shape)


def scatter_hat_gradient(values: np.ndarray, dp: np.ndarray, grid: Grid, p: np.ndarray,
                         delta: float) -> np.ndarray:
    """Derivative of ``scatter_hat`` along the point displacement dp."""
    out = np.zeros(grid.size)
    for flat, _, dw in _hat_cells(grid, p, delta):
        inside = flat >= 0
        np.add.at(out, flat[inside], (values * np.sum(dw * dp, axis=0))[inside])
    return out.reshape(grid.shape)


def gather_hat(F: np.ndarray, grid: Grid, p: np.ndarray, delta: float, gradient: bool = False):
    """Transpose of ``scatter_hat``: sum_i F_ij F_i per point, and optionally its
    gradient with respect to the point (the continuity J^T seed)."""
    f = F.reshape(-1)
    val = np.zeros(p.shape[1])
    grad = np.zeros(p.shape) if gradient else None
    for flat, w, dw in _hat_cells(grid, p, delta):
        inside = flat >= 0
        fv = np.where(inside, f[np.where(inside, flat, 0)], 0.0)
        val += w * fv
        if gradient:
            grad += dw * fv
    return (val, grad) if gradient else val


def _time_nodes(K: int, t: float):
    """Linear interpolation in time between nodes t_j = j/(K-1); t clamped to [0, 1]."""
    if K == 1:
        return [(0, 1.0)]
    s = min(max(t, 0.0), 1.0) * (K - 1)
    j = min(int(np.floor(s)), K - 2)
    th = s - j
    return [(j, 1.0 - th), (j + 1, th)]


def velocity(v: np.ndarray, vgrid: Grid, p: np.ndarray, t: float, jacobian: bool = False):
    """I(v, y, t): space-time interpolation of the velocity at points p and time t
    (Sec. 3.1, Step 1: bi/trilinear in space, linear in time, per component).
    With ``jacobian`` also returns d_y I as an array (d, d, P): [c, a] = dV_c/dy_a."""
    d = vgrid.d
    V = np.zeros((d, p.shape[1]))
    J = np.zeros((d, d, p.shape[1])) if jacobian else None
    for j, wt in _time_nodes(v.shape[0], t):
        if wt == 0.0:
            continue
        for c in range(d):
            if jacobian:
                val, g = interpolate(v[j, c], vgrid, p, gradient=True)
                J[c] += wt * g
            else:
                val = interpolate(v[j, c], vgrid, p)
            V[c] += wt * val
    return (V, J) if jacobian else V


def scatter_velocity(gv: np.ndarray, vgrid: Grid, p: np.ndarray, t: float, mu: np.ndarray):
    """gv += (d_v I(v, p, t))^T mu: transpose of the velocity interpolation,
    accumulated into gv (shape of v)."""
    for j, wt in _time_nodes(gv.shape[0], t):
        if wt == 0.0:
            continue
        for c in range(vgrid.d):
            gv[j, c] += wt * scatter(mu[c], vgrid, p)


def _direction(model: str) -> int:
    return -1 if model == "transport" else +1


def characteristics(v, vgrid: Grid, x: np.ndarray, N: int, direction: int,
                    dv: np.ndarray | None = None, keep: bool = False):
    """Alg. 1: RK4 with N equal steps from x, returning the end points y, and when
    dv is given the directional derivative (d_v y) dv carried alongside.  With
    ``keep`` also the list of the step start points y_k (k = 0..N-1).
    direction = -1 traces y(v, x, 1, 0) (backward), +1 traces y(v, x, 0, 1)."""
    dt = direction / N
    t0 = 1.0 if direction < 0 else 0.0
    y = np.array(x, dtype=np.float64, copy=True)
    dy = np.zeros_like(y)
    hist = []
    for k in range(N):
        tk = t0 + k * dt
        if keep:
            hist.append(y.copy())
        v1 = velocity(v, vgrid, y, tk)
        y1 = y + (dt / 2) * v1
        v2 = velocity(v, vgrid, y1, tk + dt / 2)
        y2 = y + (dt / 2) * v2
        v3 = velocity(v, vgrid, y2, tk + dt / 2)
        y3 = y + dt * v3
        v4 = velocity(v, vgrid, y3, tk + dt)
        if dv is not None:
            _, J1 = velocity(v, vgrid, y, tk, jacobian=True)
            _, J2 = velocity(v, vgrid, y1, tk + dt / 2, jacobian=True)
            _, J3 = velocity(v, vgrid, y2, tk + dt / 2, jacobian=True)
            _, J4 = velocity(v, vgrid, y3, tk + dt, jacobian=True)
            D1 = velocity(dv, vgrid, y, tk) + _matvec(J1, dy)
            D2 = velocity(dv, vgrid, y1, tk + dt / 2) + _matvec(J2, dy + (dt / 2) * D1)
            D3 = velocity(dv, vgrid, y2, tk + dt / 2) + _matvec(J3, dy + (dt / 2) * D2)
            D4 = velocity(dv, vgrid, y3, tk + dt) + _matvec(J4, dy + dt * D3)
            dy = dy + (dt / 6) * (D1 + 2 * D2 + 2 * D3 + D4)
        y = y + (dt / 6) * (v1 + 2 * v2 + 2 * v3 + v4)
    return y, dy, hist


def _matvec(J, x):
    return np.einsum("cap,ap->cp", J, x)


def _rmatvec(J, x):
    return np.einsum("cap,cp->ap", J, x)


def characteristics_adjoint(v, vgrid: Grid, hist, N: int, direction: int, lam: np.ndarray):
    """Transpose of the derivative recursion of Alg. 1: given the adjoint seed lam
    on the end points, returns (d_v y)^T lam with the shape of v.  The step start
    points ``hist`` come from ``characteristics(..., keep=True)``."""
    dt = direction / N
    t0 = 1.0 if direction < 0 else 0.0
    gv = np.zeros_like(v, dtype=np.float64)
    lam = np.array(lam, dtype=np.float64, copy=True)
    for k in reversed(range(N)):
        tk = t0 + k * dt
        y = hist[k]
        v1, J1 = velocity(v, vgrid, y, tk, jacobian=True)
        y1 = y + (dt / 2) * v1
        v2, J2 = velocity(v, vgrid, y1, tk + dt / 2, jacobian=True)
        y2 = y + (dt / 2) * v2
        v3, J3 = velocity(v, vgrid, y2, tk + dt / 2, jacobian=True)
        y3 = y + dt * v3
        _, J4 = velocity(v, vgrid, y3, tk + dt, jacobian=True)
        # dy' = dy + dt/6 (D1 + 2 D2 + 2 D3 + D4), each D_s = I(dv, y_s) + J_s (stage offset)
        mu4 = (dt / 6) * lam
        scatter_velocity(gv, vgrid, y3, tk + dt, mu4)
        nu4 = _rmatvec(J4, mu4)
        mu3 = (dt / 3) * lam + dt * nu4
        scatter_velocity(gv, vgrid, y2, tk + dt / 2, mu3)
        nu3 = _rmatvec(J3, mu3)
        mu2 = (dt / 3) * lam + (dt / 2) * nu3
        scatter_velocity(gv, vgrid, y1, tk + dt / 2, mu2)
        nu2 = _rmatvec(J2, mu2)
        mu1 = (dt / 6) * lam + (dt / 2) * nu2
        scatter_velocity(gv, vgrid, y, tk, mu1)
        nu1 = _rmatvec(J1, mu1)
        lam = lam + nu1 + nu2 + nu3 + nu4
    return gv


def euler_characteristics(v, vgrid: Grid, x, N: int, direction: int):
    """Forward Euler characteristics (Eq. 5); first order, kept to contrast with RK4."""
    dt = direction / N
    t0 = 1.0 if direction < 0 else 0.0
    y = np.array(x, dtype=np.float64, copy=True)
    for k in range(N):
        y = y + dt * velocity(v, vgrid, y, t0 + k * dt)
    return y


# ---------------------------------------------------------------------------
# Final states u1(v) and their derivatives (Sec. 3.1 Step 2, Sec. 3.2)
# ---------------------------------------------------------------------------

def final_state(model: str, v, vgrid: Grid, T, igrid: Grid, N: int, delta=None):
    """u1(v): transport pull-back u1 = T(y(v, x_c, 1, 0)) (Eq. 6) or continuity
    push-forward u1 = F(y(v, x_c, 0, 1)) T(x_c) (Eq. 7; delta: PIC half-width,
    None for width = cell size).  Returns (u1, y)."""
    x = cell_centres(igrid)
    y, _, _ = characteristics(v, vgrid, x, N, _direction(model))
    if model == "transport":
        u1 = interpolate(T, igrid, y).reshape(igrid.shape)
    elif delta is None:
        u1 = scatter(np.asarray(T, dtype=np.float64).reshape(-1), igrid, y)
    else:
        u1 = scatter_hat(np.asarray(T, dtype=np.float64).reshape(-1), igrid, y, delta)
    return u1, y


def jvp(model: str, v, vgrid: Grid, T, igrid: Grid, N: int, dv, delta=None):
    """(d_v u1) dv.  Transport: grad T(y) . (d_v y) dv; continuity:
    d_y(F(y) T) (d_v y) dv (Sec. 3.2)."""
    x = cell_centres(igrid)
    y, dy, _ = characteristics(v, vgrid, x, N, _direction(model), dv=dv)
    if model == "transport":
        _, gT = interpolate(T, igrid, y, gradient=True)
        return np.sum(gT * dy, axis=0).reshape(igrid.shape)
    Tf = np.asarray(T, dtype=np.float64).reshape(-1)
    if delta is None:
        return scatter_gradient(Tf, dy, igrid, y)
    return scatter_hat_gradient(Tf, dy, igrid, y, delta)


def jtvp(model: str, v, vgrid: Grid, T, igrid: Grid, N: int, r, delta=None):
    """(d_v u1)^T r: the transpose of ``jvp``."""
    x = cell_centres(igrid)
    direction = _direction(model)
    y, _, hist = characteristics(v, vgrid, x, N, direction, keep=True)
    r = np.asarray(r, dtype=np.float64)
    if model == "transport":
        _, gT = interpolate(T, igrid, y, gradient=True)
        lam = gT * r.reshape(-1)
    else:
        if delta is None:
            _, gr = interpolate(r, igrid, y, gradient=True)
        else:
            _, gr = gather_hat(r, igrid, y, delta, gradient=True)
        lam = gr * np.asarray(T, dtype=np.float64).reshape(-1)
    return characteristics_adjoint(v, vgrid, hist, N, direction, lam)


def jacobian_determinant(y: np.ndarray, grid: Grid) -> np.ndarray:
    """det grad y of a map sampled at the cell centres (y: (d, M) end points),
    with central differences inside and one-sided differences at the ends
    (numpy.gradient, edge order 1).  The paper monitors it to check that the
    discrete transformation stays diffeomorphic (Sec. 4)."""
    d = grid.d
    comps = [y[a].reshape(grid.shape) for a in range(d)]
    J = np.zeros((d, d) + grid.shape)
    for a in range(d):
        for b in range(d):
            J[a, b] = np.gradient(comps[a], grid.h[b], axis=d - 1 - b, edge_order=1)
    if d == 2:
        return J[0, 0] * J[1, 1] - J[0, 1] * J[1, 0]
    return (J[0, 0] * (J[1, 1] * J[2, 2] - J[1, 2] * J[2, 1])
            - J[0, 1] * (J[1, 0] * J[2, 2] - J[1, 2] * J[2, 0])
            + J[0, 2] * (J[1, 0] * J[2, 1] - J[1, 1] * J[2, 0]))
