"""Inexact Gauss-Newton-Krylov solver of the oracle (Sec. 3.2, Eq. 11): spectral
(DCT) preconditioner, preconditioned CG, Armijo backtracking.  FP64, numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper taken here:
* The preconditioner is the regularizer's Hessian plus gamma, P = alpha dt h^d A +
  gamma I, applied through its DCT-II eigen-decomposition (Sec. 3.2: its
  pseudo-inverse via the DCT).  A zero eigenvalue (gamma = 0, the constant
  mode) is replaced by the smallest nonzero one, so P stays positive definite
  and scales its null space like the rest of its spectrum.  For the elastic
  model only its mu-Laplacian part is used.
* Stopping and line-search constants are the textbook ones (the paper defers
  to FAIR's defaults): PCG stops at relative residual 0.1 or 50 iterations
  (Sec. 4.1); Armijo starts at mu = 1, halves, c = 1e-4, at most 10 trials;
  Gauss-Newton stops when |g| <= gtol |g0|.
"""
from __future__ import annotations

import numpy as np
from scipy.fft import dctn, idctn

from .objective import Problem, gradient, hessvec, objective


def laplacian_eigenvalues(prob: Problem) -> np.ndarray:
    """Eigenvalues of the Neumann Laplacian A on the velocity grid, arranged like
    the DCT-II coefficients of one (z, y, x) block."""
    g = prob.vgrid
    lam = np.zeros(g.shape)
    for a in range(g.d):
        k = np.arange(g.m[a])
        e = (2.0 - 2.0 * np.cos(np.pi * k / g.m[a])) / g.h[a] ** 2
        shape = [1] * g.d
        shape[g.d - 1 - a] = g.m[a]
        lam = lam + e.reshape(shape)
    return lam


def preconditioner_eigenvalues(prob: Problem) -> np.ndarray:
    """Diagonal of P = alpha dt h^d A_reg + gamma I in the DCT-II basis, with zeros
    replaced by the smallest nonzero entry (1 if all are zero)."""
    lam = laplacian_eigenvalues(prob)
    if prob.reg == "curvature":
        lam = lam * lam
    elif prob.reg == "elastic":
        lam = prob.mu * lam
    p = prob.alpha * prob.time_weight * prob.vgrid.cell_volume * lam + prob.gamma
    pos = p[p > 0.0]
    fill = pos.min() if pos.size else 1.0
    return np.where(p == 0.0, fill, p)


def apply_preconditioner(prob: Problem, r: np.ndarray) -> np.ndarray:
    """P^+ r, block by block over time nodes and components (DCT-II, divide, DCT-III)."""
    ev = preconditioner_eigenvalues(prob)
    out = np.zeros_like(r, dtype=np.float64)
    for j in range(r.shape[0]):
        for c in range(r.shape[1]):
            out[j, c] = idctn(dctn(r[j, c], type=2, norm="ortho") / ev, type=2, norm="ortho")
    return out


def pcg(Hfun, b, Minv=None, tol=0.1, maxit=50):
    """Preconditioned conjugate gradients for H x = b from x0 = 0 (Hestenes-Stiefel).
    Stops when |r| <= tol |b| or after maxit iterations, or on non-positive
    curvature p^T H p <= 0.  The paper leaves the curvature test to its
    reference (Nocedal-Wright); read as their line-search Newton-CG: the
    iterate reached so far is returned, except when the very first direction
    has non-positive curvature, where the (preconditioned) steepest-descent
    direction z0 = M^-1 b is returned instead of x = 0, so that the
    Gauss-Newton step is never empty.  Returns (x, iterations, relative
    residual); iterations counts the accepted CG steps (0 in that case)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.sqrt(np.sum(b * b))
    if nb == 0.0:
        return x, 0, 0.0
    z = Minv(r) if Minv is not None else r.copy()
    p = z.copy()
    rz = np.sum(r * z)
    it = 0
    for it in range(1, maxit + 1):
        Hp = Hfun(p)
        pHp = np.sum(p * Hp)
        if pHp <= 0.0:
            if it == 1:
                x = z.copy()        # p = z0 = M^-1 b: preconditioned steepest descent
            it -= 1
            break
        a = rz / pHp
        x = x + a * p
        r = r - a * Hp
        if np.sqrt(np.sum(r * r)) <= tol * nb:
            break
        z = Minv(r) if Minv is not None else r.copy()
        rz_new = np.sum(r * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, float(np.sqrt(np.sum(r * r)) / nb)


def armijo(Jfun, v, J0, g, dv, c=1e-4, max_trials=10):
    """Backtracking line search: the first mu in 1, 1/2, 1/4, ... with
    J(v + mu dv) <= J0 + c mu g^T dv.  Returns (mu, J(v + mu dv)) or (0, J0)."""
    slope = float(np.sum(g * dv))
    mu = 1.0
    for _ in range(max_trials):
        Jt = Jfun(v + mu * dv)
        if Jt <= J0 + c * mu * slope:
            return mu, Jt
        mu *= 0.5
    return 0.0, J0


def gauss_newton(prob: Problem, T, R, v0, max_gn=10, gtol=1e-3, max_pcg=50,
                 pcg_tol=0.1, precond=True, log=None, armijo_c=1e-4, max_ls=10):
    """Inexact Gauss-Newton-Krylov with Armijo (Eq. 11).  Returns (v, report);
    the report's history holds, per GN iteration, J and |g| at the iterate, the
    PCG count, the step dv and the step length mu taken."""
    v = np.array(v0, dtype=np.float64, copy=True)
    J, D, S, _ = objective(prob, v, T, R)
    g = gradient(prob, v, T, R)
    g0 = float(np.sqrt(np.sum(g * g)))
    rep = {"J0": J, "g0": g0, "iters": 0, "pcg_iters": 0, "history": []}
    Minv = (lambda r: apply_preconditioner(prob, r)) if precond else None
    for it in range(max_gn):
        gn = float(np.sqrt(np.sum(g * g)))
        if gn <= gtol * g0:
            break
        dv, pit, rel = pcg(lambda p: hessvec(prob, v, T, p), -g, Minv, pcg_tol, max_pcg)
        mu, Jt = armijo(lambda w: objective(prob, w, T, R)[0], v, J, g, dv, c=armijo_c, max_trials=max_ls)
        rep["history"].append({"J": J, "g": gn, "pcg": pit, "relres": rel, "mu": mu, "dv": dv})
        rep["pcg_iters"] += pit
        rep["iters"] = it + 1
        if log:
            log(rep["history"][-1])
        if mu == 0.0:
            rep["status"] = "line search failed"
            break
        v = v + mu * dv
        J, D, S, _ = objective(prob, v, T, R)
        g = gradient(prob, v, T, R)
    rep.update({"J": J, "D": D, "S": S, "g": float(np.sqrt(np.sum(g * g)))})
    return v, rep


# ---------------------------------------------------------------------------
# Multilevel continuation (Sec. 3.2, last paragraph): solve on a coarse
# discretisation, refine the velocity and use it as the starting guess of the
# next level.
# ---------------------------------------------------------------------------

def coarse_grid(grid, factor=2):
    """The same box with every cell count divided by ``factor`` (cell counts must divide)."""
    from .lagrangian import Grid
    if any(m % factor for m in grid.m):
        raise ValueError("cell counts must be divisible by the coarsening factor")
    return Grid(tuple(m // factor for m in grid.m), grid.lo, grid.hi)


def restrict_image(F: np.ndarray, grid) -> np.ndarray:
    """Average of the 2^d fine cells that tile each coarse cell (keeps the integral
    of the image: mean value times cell volume)."""
    d = grid.d
    shape = []
    for a in reversed(range(d)):
        shape += [grid.m[a] // 2, 2]
    blocks = np.asarray(F, dtype=np.float64).reshape(shape)
    return blocks.mean(axis=tuple(range(1, 2 * d, 2)))


def prolong_velocity(vc: np.ndarray, cgrid, fgrid) -> np.ndarray:
    """Coarse velocity interpolated (Sec. 3.1, Step 1 interpolation) at the fine
    velocity grid's cell centres, per time node and component."""
    from .lagrangian import cell_centres, interpolate
    x = cell_centres(fgrid)
    out = np.zeros((vc.shape[0], vc.shape[1]) + fgrid.shape)
    for j in range(vc.shape[0]):
        for c in range(vc.shape[1]):
            out[j, c] = interpolate(vc[j, c], cgrid, x).reshape(fgrid.shape)
    return out


def level_problems(prob: Problem, levels: int):
    """Problems from coarsest to finest; level l halves both grids (levels - 1 - l) times.
    Every other field (K, N, model, regularizer and weights, the PIC half-width
    delta in domain units) is the finest problem's."""
    probs = [prob]
    for _ in range(levels - 1):
        p = probs[0]
        probs.insert(0, Problem(coarse_grid(p.igrid), coarse_grid(p.vgrid), K=p.K, N=p.N, model=p.model,
                                reg=p.reg, alpha=p.alpha, gamma=p.gamma, mu=p.mu, lam=p.lam, delta=p.delta))
    return probs


def multilevel_gauss_newton(prob: Problem, T, R, levels, **gn):
    """Coarse-to-fine Gauss-Newton: images restricted by averaging, each level
    started from the prolonged solution of the coarser one (zero on the coarsest).
    Returns (v on the finest level, list of per-level reports)."""
    probs = level_problems(prob, levels)
    Ts, Rs = [np.asarray(T, dtype=np.float64)], [np.asarray(R, dtype=np.float64)]
    for l in range(levels - 1, 0, -1):
        Ts.insert(0, restrict_image(Ts[0], probs[l].igrid))
        Rs.insert(0, restrict_image(Rs[0], probs[l].igrid))
    v = np.zeros(probs[0].vshape)
    reports = []
    for l, p in enumerate(probs):
        if l > 0:
            v = prolong_velocity(v, probs[l - 1].vgrid, p.vgrid)
        v, rep = gauss_newton(p, Ts[l], Rs[l], v, **gn)
        reports.append(rep)
    return v, reports
