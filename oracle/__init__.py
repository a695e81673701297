"""Plain FP64 CPU oracle of the DNN-MG hot path (test infrastructure only).

This package is the slow, obviously correct statement of what the CUDA path
computes.  It is used by the tests, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg only; the product path never imports it.  It
shares no code with the CUDA path: element matrices are integrated here by
2x2 Gauss quadrature of the Q1 basis functions and assembled into global CSR
matrices, and every solver step works on those matrices.

Modules
  mesh    level hierarchy, obstacle, boundary masks (Sec. 2.1, Eq. 2)
  fem     Q1/Q1 + LPS element matrices and assembly (Eqs. 3-5)
  mg      transfers, cell-wise Vanka smoother, coarse LU, V-cycle (Sec. 2.2)
  krylov  flexible GMRES (Sec. 2.2)
  newton  Newton time step (Eq. 6, the Newton iteration of Algorithm 1)
  net     patch GRU + dense network, BPTT backward, loss (Eq. 7), Adam
  dnnmg   prolongation, network inputs, scatter, Rhs and restriction
          (the network correction of Algorithm 1)

Readings of the paper where it is silent or garbled are stated in each
module's docstring.  Pins that tie each function to the paper or to
mathematics live in tests/test_oracle_*.py.
"""
