"""Workload descriptions and seeded synthetic inputs shared by the tests,
the benchmark and the oracle.

Holds parameters and seeded random generators only: none of the method's
arithmetic (no KL basis, no solver, no estimator) lives here.

The five workloads follow the paper's setting (unit square, Table 1 Case II
with p = 1 on the west edge and p = 0 on the east edge, lognormal field with
the exponential Matern covariance of Sec. 3.1) at the sizes the project is
measured on.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

DEFAULT_SEED = 1910047270


@dataclass
class Workload:
    name: str
    levels: List[int]          # finest grid n_l of each MLMC level
    M: int                     # KL modes
    sigma2: float
    lam: float
    eps: float                 # target RMSE
    n_pilot: int
    nu0: int = 2               # V-cycles per FMG stage
    nu1: int = 2
    nu2: int = 2
    pW: float = 1.0
    pE: float = 0.0
    n0: int = 4                # coarsest FMG grid
    n_shifts: int = 16         # QMC digital shifts
    kl_q: int = 0              # Nystrom quadrature grid (0: automatic)
    seed: int = DEFAULT_SEED
    extra: dict = field(default_factory=dict)

    @property
    def n_ref(self):
        return self.levels[-1]


WORKLOADS = {
    # single-level MC, 32x32, 64 KL modes, 256 samples, FMG 4x4..32x32
    "mc32": Workload("mc32", [32], 64, 1.0, 0.3, eps=0.0, n_pilot=256),
    # FMG-MLMC, five levels 16x16..256x256, 128 KL modes, RMSE 1e-3
    "fmg_mlmc5": Workload("fmg_mlmc5", [16, 32, 64, 128, 256], 128, 1.0, 0.3,
                          eps=1e-3, n_pilot=1000),
    # uneven batch: 4096 samples over 64x64..1024x1024, 256 modes
    "batched4096": Workload("batched4096", [64, 128, 256, 512, 1024], 256, 1.0, 0.3,
                            eps=1e-3, n_pilot=64),
    # surrogate level below the 16x16 level of fmg_mlmc5
    "surrogate5": Workload("surrogate5", [16, 32, 64, 128, 256], 128, 1.0, 0.3,
                           eps=1e-3, n_pilot=1000),
    # high contrast: 6 levels 64x64..2048x2048, sigma^2 = 2, lambda = 0.1, 1024 modes
    "contrast6": Workload("contrast6", [64, 128, 256, 512, 1024, 2048], 1024, 2.0, 0.1,
                          eps=5e-4, n_pilot=64),
}


def rng(seed=DEFAULT_SEED, tag=0):
    """numpy Generator for synthetic test inputs (not the method's own streams)."""
    return np.random.default_rng([seed, tag])


def lognormal_field(n, S=1, sigma=1.0, seed=DEFAULT_SEED, tag=1):
    """i.i.d. lognormal cell values [S][n][n]: a rough field for solver tests."""
    g = rng(seed, tag).standard_normal((S, n, n)) * sigma
    return np.exp(g)


def smooth_lognormal_field(n, S=1, sigma=1.0, modes=6, seed=DEFAULT_SEED, tag=2, kmax=4):
    """exp of a few random Fourier modes [S][n][n] (wave numbers below kmax):
    a smooth field for solver tests."""
    r = rng(seed, tag)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    g = np.zeros((S, n, n))
    for _ in range(modes):
        kx, ky = r.integers(0, kmax, size=2)
        a = r.standard_normal(S)[:, None, None] * sigma / np.sqrt(modes)
        ph = r.uniform(0, 2 * np.pi, size=S)[:, None, None]
        g += a * np.cos(np.pi * (kx * X + ky * Y)[None] + ph)
    return np.exp(g)


def normals(S, M, seed=DEFAULT_SEED, tag=3):
    """Standard normal KL coefficients [S][M] for tests that bypass the point sets."""
    return rng(seed, tag).standard_normal((S, M))
