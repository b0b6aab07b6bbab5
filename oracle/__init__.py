"""CPU FP64 oracle for the G-prox PDHG implicit-step solver (arxiv 2305.03945).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct numpy restatement
of the paper's method, used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it; the product
library (``paper_2305_03945_gb300``) never does, and shares no code with it.

Modules
  rd_oracle  the implicit scheme, residual map F, its adjoint Jacobian, the spectral
             preconditioner and the PDHG iteration of Algorithm 1 (numpy, library FFT / DCT)
  rd_oracle_cpp.cpp, cpp_oracle
             the same method as plain FP64 C++ with its own radix-2 FFT and a DCT-II by the
             2N-point even extension, optionally over OpenMP threads (the timed CPU baseline),
             behind a small C ABI and its ctypes binding
  dense      dense matrices written out from the paper's block forms (Section 2.1, Remark 1),
             dense Newton for the implicit step; used only as pins
  theory     closed forms of Theorem 1 / Corollary 1 / Appendix A
  adapt      the adaptive time step size of Section 2.2 on top of rd_oracle's implicit step

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (dense matrices, eigenmodes, closed-form iteration recurrences,
dense Newton, invariants, paper-printed iteration counts, the reaction terms against their PDEs
on uniform states and single modes); the C++ oracle by brute-force transforms, closed forms,
dense Newton, the reaction pins and element-wise equality with the numpy oracle.
"""
