"""CPU FP64 oracle for the modal DGSEM hot path (test infrastructure only).

A plain, slow, obviously correct NumPy implementation of what the GPU library
computes: the modal Galerkin weak form of the compressible Euler equations on
mixed hex/prism/pyramid/tet meshes (weak form Eq. 1 of the paper, Sec. 2),
collapsed (Duffy) quadrature, the projection of Algorithm 1, LSERK time
stepping, and the adjoint (vector-Jacobian products) of the right-hand side and
of K time steps.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with the CUDA library; the only common module
is the seeded input generator (dg_inputs), which holds none of the method's
arithmetic.

Parity status per function (see each module's header):
  basis / quadrature / mesh / rhs / lserk / adjoint / curved elements
  (oracle.curved): pinned by the tests in
  tests/test_oracle_*.py (closed forms, invariants, brute force).  The choice
  of modal space, quadrature and flux where the paper is silent is a reading,
  listed in the design notes; those readings are pinned for internal
  consistency only ("parity unpinned" against the paper's own solver).
"""
