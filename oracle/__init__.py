"""FP64 CPU oracle for the generalized-Poisson pressure solve.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement in numpy/scipy (float64) of what the solver computes.  It shares
no code with the CUDA library and imports nothing from it.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the product path never does.

Modules
  poisson    the discrete operator A = c~ - div(kappa grad) (Eq. Poiss /
             GeneralizedPoisson with Eqs. cpoiss, kappapoiss), its assembly,
             and reference solves (dense Cholesky, sparse direct, Jacobi-PCG).
  multigrid  the geometric-multigrid V-cycle the GPU uses as preconditioner
             (coarsening, restriction, prolongation, red-black Gauss-Seidel),
             written level by level.
  unet       the learned warm start's network layers in float64 (forward and
             hand-derived backward).
  diffusion  the dissipative fourth-order second-derivative stencil of the
             viscous terms (Sec. 4, Eq. dissipativestencil4) in flux form,
             and the non-dissipative nine-point stencil it replaces.
  projection the steps either side of the solve (Sec. 2, steps (iv)-(viii)):
             right-hand side of Eq. fpoiss, dual-cell pressure gradient
             (Eqs. pbnd, nablaP), momentum, face-velocity and energy updates.
  fem        the operator in Q1 finite elements (Sec. 2.5): element
             matrices, harmonic-mean element kappa, lumped c~ term.
  fractional one whole fractional step around the solve (Sec. 2.4 steps
             (i)-(ix)): MUSCL-upwinded advection, the projection steps, the
             ideal-gas reset; the Gresho vortex's kinetic energy.

Pins (what fixes each function to something other than itself) live in
tests/test_oracle_*.py.  Functions whose result has no such pin say
"parity unpinned" in their docstring.
"""
