"""Plain, slow FP64 CPU oracle for the hp space-time multigrid Newton-Krylov method.

TEST INFRASTRUCTURE ONLY.  This package is the independent statement of what the
GPU path computes, written from the paper (Margenberg & Bause, "A monolithic hp
space-time multigrid preconditioned Newton-Krylov solver for space-time FEM applied
to the incompressible Navier-Stokes equations").  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import it.  The product path (``paper_2602_13841_gb300``) never
imports, calls or links anything here, and nothing here imports the product path.

Every function names the section / equation / algorithm of the paper it follows.
Where the paper is silent or garbled the oracle takes one documented reading; the
list of readings is kept in the repository's design notes.

Modules
-------
reference   quadrature rules, 1D bases, time matrices K, M, C (Appendix A, Sec. 3.1)
mesh        structured (optionally perturbed) quad/hex meshes, DoF maps (Sec. 2.2)
problems    analytic data: Taylor-Green and manufactured flows (Sec. 5)
forms       residual R_n, Jacobian J_n, mass-weighted norm (Problem 3.1, Eq. 3.11-3.12)
multigrid   transfers, Vanka smoother, V-cycle, coarse solve (Sec. 4.2-4.3)
krylov      FGMRES and inexact Newton with EW forcing and Armijo (Sec. 4.1, Alg. 1-2)
"""
