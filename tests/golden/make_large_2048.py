"""Writes large_2048.json: converged FP64 oracle outfluxes (Q^f and the
1024 x 1024 stage's Q^c) of three 2048 x 2048 high-contrast test fields, with
the plain V-cycle and with the energy-optimal correction step.

The fields are workloads.smooth_lognormal_field(2048, S=3, sigma=sqrt(2),
modes=24, tag=3100, kmax=12): log-permeability variance 2 in short-wavelength
Fourier modes, the grid and variance of the large high-contrast case.  Only
the oracle computes the stored values (FMG with V-cycles to a relative
residual of 1e-14, Table 1 Case II boundary data).  Run from the repository
root: python tests/golden/make_large_2048.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import workloads as W  # noqa: E402
from oracle import lib as OL  # noqa: E402

FIELD = dict(n=2048, S=3, sigma=float(np.sqrt(2.0)), modes=24, tag=3100, kmax=12)


def main():
    K = W.smooth_lognormal_field(FIELD["n"], S=FIELD["S"], sigma=FIELD["sigma"], modes=FIELD["modes"],
                                 tag=FIELD["tag"], kmax=FIELD["kmax"])
    qf, qc, _, _ = OL.fmg_solve_batch(K, OL.params(converged=True, tol=1e-14, max_cycles=400), nthreads=3)
    # the same with the energy-optimal correction step, which converges on all three
    ef, ec, _, _ = OL.fmg_solve_batch(K, OL.params(converged=True, tol=1e-14, max_cycles=400, energy_step=True),
                                      nthreads=3)
    out = {"source": "oracle/lib.py fmg_solve_batch, converged FP64 (tol 1e-14), this script",
           "field": FIELD, "contrast": [float(k.max() / k.min()) for k in K],
           "qf": [float(x) for x in qf], "qc": [float(x) for x in qc],
           "qf_energy_step": [float(x) for x in ef], "qc_energy_step": [float(x) for x in ec]}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_2048.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
