"""FP64 CPU oracle for sCWatter (arXiv 2404.07293) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import, call or execute anything in this package.
The GPU library (``paper_2404_07293_gb300``) never calls it and shares no code
with it; the only thing both sides share is the seeded input generator in
``workloads`` (random draws and geometry, no coupled-wave arithmetic).

Contents
  cw     the coupled-wave solve of Sec. 2: orders (Eq. 6), s_z (Eq. 2), Fourier
         coefficients (Eq. 11-12), property matrix D (Eq. 21), eigenmodes
         (Sec. 2.5.3), top/bottom matrices and the connection equations
         (Eq. 24-29), the 6M linear system (Sec. 3.4), alpha recovery and the
         E-field rows W (Eq. 33, Sec. 4.1); plus the full block system that
         the connection equations reduce (brute-force cross-check).
  synth  field synthesis: per-plane spectrum (Eq. 9 outside, Eq. 30/34 inside)
         and recomposition by direct summation (Eq. 10); an FFT variant used
         only to cross-check the direct sum.
  fno    (surrogate) plain FP64 forward/backward of the Fourier neural operator.

Precision: complex128 / float64 everywhere.
Parity status per function is stated in each function's docstring; the
heterogeneous-sample field values themselves are "parity unpinned" beyond the
invariants listed there, because the paper prints no field values.
"""
