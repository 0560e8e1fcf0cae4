"""FP64 CPU oracle for the wFQ / wFQFmu linear-response solve (test infrastructure).

This package is the independent, slow, obviously-correct reference against
which the CUDA library is checked.  It is test infrastructure only: the
library, its Python binding and the timed GPU path never import it.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may use
it.  It shares no code with the CUDA path; both consume the same seeded inputs
from ``paper_2510_12731_gb300.structures``, which holds no arithmetic of the
method.

Modules
-------
model     dense assembly of K (Eq. 3), the Fermi damping (Eq. 4), Kbar (Eq. 2),
          the Gaussian kernels T^qq (Eq. 5) and their derivatives T^qmu,
          T^muq, T^mumu (Sec. 2.2), the shifts z_q (Eq. 6) and z_mu (Eq. 8),
          the right-hand sides of Eq. 1 / Eq. 7, the direct LU solve
          ("inversion" in Sec. Solvers) and the observables (Sec. Observables).
spectral  a second exact route for wFQ (Cholesky of T + symmetric eigensolve),
          used as a cross-check and for sizes where one LU per frequency is
          too slow.
calibrate the effective-area calibration that the parameter presets use.
fields    induced density, potential and field of a solved structure at probe points
          (the maps of Sec. "Post-process Analysis").
hetero    heterogeneous wFQFmu (Eq. 9, the frequency-dependent conductance block, and the
          per-atom interband polarisability of Eq. 10).

Pins: every function is checked in ``tests/test_oracle_*.py`` against values
fixed by the paper and by mathematics (closed forms, limits, brute force,
invariants), not against itself.
"""
