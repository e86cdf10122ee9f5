"""FP64 CPU oracle for the LADMM compartment-mapping method (test infrastructure).

This package is the independent, slow, plainly written reference that the CUDA path
is checked against. It is test infrastructure only: the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library itself never
does, and it shares no code, tables or helpers with the CUDA path.

Modules:
  grid   -- the finite-difference operator D of Eq. 8 and the norm of D^T D
  ladmm  -- Algorithm 2 (low-rank f-step, Eq. 28) and its full-rank variant (Eq. 26),
            the objective of Eq. 7 and the stopping rule
  nnls   -- voxel-by-voxel NNLS (Eq. 6 with R = 0): Lawson-Hanson and brute force
  pg     -- an independent projected-gradient (FISTA) solver of Eq. 7
  admm   -- Algorithm 1, the three-split ADMM the paper compares against
  kkt    -- first-order optimality residuals of Eq. 7
  tune   -- the paper's beta heuristic: tune on a 3x3 patch (Sec. III-E)

Everything is float64 with numpy / scipy primitives (SVD, sparse matmul, dense
solves) as single steps; no blocking, fusion or reordering beyond what the paper's
equations state.
"""
