"""Pins of the oracle's regularizer operators, spectral preconditioner, PCG and
Gauss-Newton (Sec. 3.2, Eq. 11) against dense linear algebra on tiny grids."""
import numpy as np
import pytest

from oracle import lagrangian as L
from oracle.objective import Problem, hessvec, objective, reg_operator
from oracle.solver import apply_preconditioner, armijo, gauss_newton, pcg, preconditioner_eigenvalues
from paper_1703_04446_gb300 import synth


def _neumann_1d(m, h):
    """Dense 1D Neumann second-difference matrix (positive semi-definite)."""
    A = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    A[0, 0] = A[-1, -1] = 1.0
    return A / h ** 2


def _dense_laplacian(grid):
    """Kronecker sum of 1D Neumann matrices, in the flattened (z, y, x) order."""
    mats = [_neumann_1d(grid.m[a], grid.h[a]) for a in range(grid.d)]
    eyes = [np.eye(grid.m[a]) for a in range(grid.d)]
    n = grid.size
    A = np.zeros((n, n))
    for a in range(grid.d):
        term = np.ones((1, 1))
        for b in reversed(range(grid.d)):   # numpy order z, y, x -> kron(z, y, x)
            term = np.kron(term, mats[b] if b == a else eyes[b])
        A += term
    return A


@pytest.mark.parametrize("reg", ["diffusion", "curvature"])
@pytest.mark.parametrize("d", [2, 3])
def test_regularizer_operator_matches_dense_kronecker_sum(reg, d):
    vg = L.Grid((5, 4, 3)[:d], hi=(1.0, 0.8, 1.5)[:d])
    prob = Problem(L.Grid(vg.m), vg, K=3, N=2, reg=reg, alpha=1.0)
    A = _dense_laplacian(vg)
    if reg == "curvature":
        A = A @ A
    x = np.random.default_rng(0).normal(size=prob.vshape)
    out = reg_operator(prob, x)
    w = prob.time_weight * vg.cell_volume
    for j in range(3):
        for c in range(d):
            np.testing.assert_allclose(out[j, c].ravel(), w * A @ x[j, c].ravel(), rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("reg,gamma", [("diffusion", 0.0), ("diffusion", 1e-2), ("curvature", 1e-2)])
def test_spectral_preconditioner_inverts_dense_operator(reg, gamma):
    """The DCT diagonalises the Neumann operator (Toeplitz-plus-Hankel structure,
    Sec. 3.2): P^+ (P x) = x off the null space."""
    vg = L.Grid((6, 5), hi=(1.0, 1.3))
    prob = Problem(L.Grid(vg.m), vg, K=1, N=2, reg=reg, alpha=0.3, gamma=gamma)
    x = np.random.default_rng(1).normal(size=prob.vshape)
    if gamma == 0.0:
        x -= x.mean(axis=(2, 3), keepdims=True)      # remove the constant (null) mode
    Px = prob.alpha * reg_operator(prob, x) + gamma * x
    np.testing.assert_allclose(apply_preconditioner(prob, Px), x, atol=1e-10)
    ev = np.sort(preconditioner_eigenvalues(prob).ravel())
    A = prob.alpha * prob.vgrid.cell_volume * _dense_laplacian(vg)
    if reg == "curvature":
        A = A @ A / (prob.alpha * prob.vgrid.cell_volume)
    dense_ev = np.sort(np.linalg.eigvalsh(A + gamma * np.eye(vg.size)))
    if gamma == 0.0:
        dense_ev[0] = dense_ev[1]     # the null-space eigenvalue takes the smallest nonzero one
    np.testing.assert_allclose(ev, dense_ev, rtol=1e-9, atol=1e-12)


def _tiny_problem(model, K=1):
    ig = L.Grid((8, 8))
    vg = L.Grid((4, 4))
    gs = synth.GridSpec(ig.m, (0.0, 0.0), (1.0, 1.0))
    T = synth.gaussian_blobs(synth.centres(gs), [(1.0, 0.18, (0.45, 0.5)), (0.5, 0.1, (0.6, 0.4))])
    R = synth.gaussian_blobs(synth.centres(gs), [(1.0, 0.18, (0.52, 0.47)), (0.5, 0.1, (0.62, 0.45))])
    prob = Problem(ig, vg, K=K, N=3, model=model, reg="diffusion", alpha=1e-3, gamma=1e-4)
    v = synth.random_velocity(synth.GridSpec(vg.m, (0.0, 0.0), (1.0, 1.0)), K, 0.05, 3)
    return prob, T, R, v


def _dense_hessian(prob, v, T):
    n = int(np.prod(prob.vshape))
    H = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        H[:, i] = hessvec(prob, v, T, e.reshape(prob.vshape)).ravel()
    return H


@pytest.mark.parametrize("model", ["transport", "continuity"])
def test_gauss_newton_hessian_is_symmetric_and_matches_jacobian(model):
    """H = J^T h^d J + alpha dt h^d A + gamma I with J assembled column by column."""
    prob, T, R, v = _tiny_problem(model)
    H = _dense_hessian(prob, v, T)
    np.testing.assert_allclose(H, H.T, atol=1e-12 * np.abs(H).max())
    n = H.shape[0]
    Jm = np.zeros((prob.igrid.size, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Jm[:, i] = L.jvp(model, v, prob.vgrid, T, prob.igrid, prob.N, e.reshape(prob.vshape)).ravel()
    Ar = np.stack([reg_operator(prob, np.eye(n)[i].reshape(prob.vshape)).ravel() for i in range(n)], axis=1)
    Hd = prob.igrid.cell_volume * Jm.T @ Jm + prob.alpha * Ar + prob.gamma * np.eye(n)
    np.testing.assert_allclose(H, Hd, atol=1e-12 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > 0.0


def test_pcg_step_equals_cholesky_step():
    """Run to convergence, PCG returns the Cholesky solution of Eq. 11."""
    prob, T, R, v = _tiny_problem("transport")
    H = _dense_hessian(prob, v, T)
    b = np.random.default_rng(2).normal(size=H.shape[0])
    c = np.linalg.cholesky(H)
    x_ref = np.linalg.solve(c.T, np.linalg.solve(c, b))
    Hf = lambda p: (H @ p.ravel()).reshape(p.shape)
    x, it, rel = pcg(Hf, b.reshape(prob.vshape), lambda r: apply_preconditioner(prob, r),
                     tol=1e-13, maxit=500)
    np.testing.assert_allclose(x.ravel(), x_ref, rtol=1e-8, atol=1e-10 * np.abs(x_ref).max())
    x0, _, _ = pcg(Hf, b.reshape(prob.vshape), None, tol=1e-13, maxit=500)
    np.testing.assert_allclose(x0.ravel(), x_ref, rtol=1e-8, atol=1e-10 * np.abs(x_ref).max())


@pytest.mark.parametrize("model,K", [("transport", 1), ("continuity", 2)])
def test_gauss_newton_decreases_objective(model, K):
    prob, T, R, _ = _tiny_problem(model, K)
    v0 = np.zeros(prob.vshape)
    v, rep = gauss_newton(prob, T, R, v0, max_gn=6, gtol=1e-3, max_pcg=20, pcg_tol=0.1)
    Js = [h["J"] for h in rep["history"]] + [rep["J"]]
    assert all(b <= a for a, b in zip(Js, Js[1:]))
    assert rep["J"] < 0.5 * rep["J0"]
    assert rep["g"] < rep["g0"]
    assert abs(objective(prob, v, T, R)[0] - rep["J"]) < 1e-14


def test_pcg_first_direction_with_nonpositive_curvature_returns_preconditioned_descent():
    """Line-search Newton-CG (Nocedal-Wright, the paper's reference for the
    Krylov and line-search settings): when the first direction already has
    non-positive curvature, the step is the preconditioned steepest-descent
    direction M^-1 b, not x = 0, and no CG step is counted."""
    b = np.array([[1.0, -2.0, 0.5], [0.25, 3.0, -1.0]])
    Minv = lambda r: r / np.array([2.0, 4.0, 8.0])
    for Hf in (lambda p: -p, lambda p: 0.0 * p):
        x, it, _ = pcg(Hf, b, Minv, tol=1e-8, maxit=10)
        assert it == 0
        np.testing.assert_array_equal(x, Minv(b))
        x, it, _ = pcg(Hf, b, None, tol=1e-8, maxit=10)
        assert it == 0
        np.testing.assert_array_equal(x, b)


def test_pcg_later_direction_with_negative_curvature_keeps_the_iterate():
    """H = diag(1, -1), b = (2, 1): the first direction has curvature 3 > 0,
    alpha = 5/3; the second direction (20/9, 40/9) has negative curvature, so
    PCG stops with x1 = (10/3, 5/3) after one step."""
    H = np.diag([1.0, -1.0])
    x, it, _ = pcg(lambda p: H @ p, np.array([2.0, 1.0]), None, tol=1e-8, maxit=10)
    assert it == 1
    np.testing.assert_allclose(x, [10.0 / 3.0, 5.0 / 3.0], rtol=1e-15)


def test_armijo_with_constant_above_one_rejects_every_step_of_a_convex_model():
    """With c > 1 the sufficient-decrease test asks for more than the linear
    model promises; on a convex quadratic no step length passes, the search
    reports mu = 0 and the Gauss-Newton loop stops with the iterate unchanged."""
    Jf = lambda w: float(np.sum((w - 1.0) ** 2))
    v = np.zeros(3)
    g = 2.0 * (v - 1.0)
    mu, Jt = armijo(Jf, v, Jf(v), g, -g / 2.0, c=2.0, max_trials=10)
    assert mu == 0.0 and Jt == Jf(v)
    prob, T, R, _ = _tiny_problem("transport")
    v0 = np.zeros(prob.vshape)
    v, rep = gauss_newton(prob, T, R, v0, max_gn=3, gtol=1e-3, max_pcg=20, pcg_tol=0.1, armijo_c=2.0)
    assert rep["status"] == "line search failed" and rep["iters"] == 1
    np.testing.assert_array_equal(v, v0)
    assert rep["J"] == rep["J0"]
