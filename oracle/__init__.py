"""Plain FP64 CPU oracle of the Lagrangian Gauss-Newton-Krylov method
(Mang & Ruthotto, "A Lagrangian Gauss-Newton-Krylov solver for mass- and
intensity-preserving diffeomorphic image registration", arXiv 1703.04446).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, the smoke check and the CPU-baseline leg of the benchmark call it.
It shares no code with the CUDA path: every step is re-derived from the paper
in numpy, vectorised over particles (the same scalar recursion applied to all
characteristics at once), with library primitives (floor, gather, add.at,
DCT) as single steps and no blocking or fusion.

Modules
-------
lagrangian  interpolation I(v, y, t), RK4 characteristics with the forward-mode
            derivative (Alg. 1), transport pull-back (Eq. 6), PIC push-forward
            (Eqs. 7-8), their J and J^T products.
objective   SSD (Eq. 10), regularizers (Sec. 2.1), objective, gradient,
            Gauss-Newton Hessian (Sec. 3.2).
solver      spectral (DCT) preconditioner, PCG, Armijo, Gauss-Newton (Eq. 11),
            multilevel continuation (Sec. 3.2).
warmstart   the learned warm-start network (an addition, not in the paper) in
            torch CPU FP64; imported on its own (needs torch).

Parity status: every function is pinned by a test against closed forms,
invariants, library routines or brute force.  The elastic regularizer, which
the paper names but does not define, is a reading of the Navier-Lame energy;
it is pinned by closed-form energies of fields that are linear in the cell
centres and by its reduction to mu times the diffusion regularizer when
lam + mu = 0.
"""
from . import lagrangian, objective, solver  # noqa: F401
