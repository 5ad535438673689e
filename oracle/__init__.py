"""Plain, slow FP64 CPU oracle for the inexact All-Floating IETI solver.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; the two meet only in the
seeded input generators of ``afi_workloads``.

Every function follows the paper's definitions written out directly
(Cox-de Boor recursion, quadrature sums, Kronecker products, the projectors
and the recovery formulas of Section 4, Algorithm 1, textbook MINRES), using
NumPy/SciPy primitives (eigh, splu, sparse products) as single steps.

Parity status per module:
  spline    pinned (partition of unity, Greville linear precision, p=1
            closed forms, 1D matrix identities)
  fd        pinned (dense Kronecker solve, eigen identities)
  assembly  pinned (rigid modes in kernel, constant-strain energy, Kronecker
            special case on axis-aligned boxes, manufactured-solution rates)
  ieti      pinned (conforming direct solve, projector identities, N_c counts)
  minres    pinned (dense solve on SPD-preconditioned systems)
  adjoint   pinned (closed forms and central finite differences)
"""
