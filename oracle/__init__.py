"""Plain FP64 CPU oracle for the FMG-MLMC / MLQMC method (arXiv 1910.04727).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports,
links or runs anything here, and this package imports nothing from the
product.  The two sides share no code; only the seeded input generators in
``workloads.py`` (which hold none of the method's arithmetic) serve both.

Layout
  fmg_oracle.c  points (Philox4x64-10, Sobol', inverse normal CDF), finite
                volumes (Eq. 1, Table 1 Case II), RB-GS V-cycles, full
                multigrid with injected coefficients and the Q^c by-product
                (Sec. 2.5, Algorithm 3); compiled by ``build()``
  lib.py        ctypes wrappers of the C functions
  kl.py         Karhunen-Loeve basis of the exponential Matern field (Sec. 3.1)
                by the Nystrom method, and the field synthesis k = exp(g)
  mlmc.py       MLMC / MLQMC estimators and sample-size control (Sec. 2.2-2.4,
                Algorithms 1-3)
  mlp.py        FP64 surrogate network (forward, backward, Adam) used as a
                control-variate level
"""
from .build import build, library_path  # noqa: F401
