"""Every smoother launch shape gives the same solve, bit for bit.

The column-strip wavefront, the staged and register-blocked tiles and the
one-launch-per-colour sweeps update each cell with the same expression in
the same order, so setting any of them for every grid of a hierarchy must
leave Q^f, Q^c and the fine-grid iterate unchanged, in FP64 and in the
mixed form, with fixed schedules and with converged stages (where samples
drop out of the sweeps at different cycles).  Grids from 16 x 16 to
512 x 512 and batches from one sample up make the strips overlap in columns
(ragged last strip) and, for small batches, split into row segments.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import lib as OL

pytestmark = pytest.mark.gpu

SHAPES = [(0, 0), (-1, 0), (32, 256), (32, 128), (16, 0), (32, 0)]
LEVELWISE = 1
CASES = [(16, 5), (32, 3), (64, 7), (128, 2), (256, 3), (256, 37), (512, 1)]


def _grids(n):
    return [4 << k for k in range(20) if (4 << k) <= n]


def _same(a, b):
    return np.array_equal(a.cpu().numpy(), b.cpu().numpy(), equal_nan=True)


@pytest.mark.parametrize("precision,converged", [(0, 0), (0, 1), (1, 1)])
def test_every_shape_gives_the_same_solve(precision, converged):
    import paper_1910_04727_gb300 as fm
    c = fm.Context(2, 16, 16, precision=precision, converged=converged, tol=1e-12, qtol=0.0, max_cycles=200)
    for n, S in CASES:
        K = torch.tensor(W.smooth_lognormal_field(n, S=S, tag=2000 + n + S), device="cuda")
        ref = None
        for tile, threads in SHAPES:
            for m in _grids(n):
                c.set_smoother_shape(m, tile, threads)
            # the level-wise schedule (small grids would otherwise run the resident kernel)
            qf, qc, p = c.fmg_solve_batch(K, want_p=True, kernel=LEVELWISE)
            if ref is None:
                ref = (qf, qc, p)
                continue
            assert _same(qf, ref[0]) and _same(qc, ref[1]) and _same(p, ref[2]), (n, S, tile, threads)
    for m in _grids(512):
        c.set_smoother_shape(m, -2)


def test_strip_shape_against_the_oracle():
    import paper_1910_04727_gb300 as fm
    c = fm.Context(2, 16, 16)
    for n, S in [(64, 3), (256, 2)]:
        K = W.smooth_lognormal_field(n, S=S, tag=2100 + n)
        for m in _grids(n):
            c.set_smoother_shape(m, -1)
        qf, qc, _ = c.fmg_solve_batch(torch.tensor(K, device="cuda"), kernel=LEVELWISE)
        of, oc, _, _ = OL.fmg_solve_batch(K, OL.params())
        assert np.max(np.abs(qf.cpu().numpy() - of) / np.abs(of)) < 1e-10
        assert np.max(np.abs(qc.cpu().numpy() - oc) / np.abs(oc)) < 1e-10


def test_shape_arguments_are_checked():
    import paper_1910_04727_gb300 as fm
    c = fm.Context(2, 16, 16)
    for args in [(24, 0, 0), (64, 48, 0), (64, -1, 128), (64, 0, 256), (64, 32, 64)]:
        with pytest.raises(fm.FmError):
            c.set_smoother_shape(*args)


@pytest.mark.parametrize("precision,converged,case,nc", [(0, 0, 2, 4), (0, 1, 2, 4), (1, 1, 2, 4), (1, 1, 1, 4),
                                                          (0, 0, 2, 2), (0, 1, 1, 3), (1, 1, 2, 3)])
def test_resident_vcycle_tail_changes_nothing(precision, converged, case, nc):
    """The V-cycle below 32 x 32 as one resident launch per cycle (the default)
    against grid-by-grid launches: every result bit for bit, on every shape of
    the grids above it, in both boundary cases, for coarsest grids of 2, 3 and
    4 cells a side (the tail's deepest and largest footprints)."""
    import paper_1910_04727_gb300 as fm
    c = fm.Context(2, nc * 4, 16, n_coarsest=nc, precision=precision, converged=converged, tol=1e-12, qtol=1e-10,
                   max_cycles=200, bc_case=case, pS=0.3, pN=0.7)
    for n, S in [(nc * 16, 7), (nc * 32, 3), (nc * 64, 2)]:
        K = torch.tensor(W.smooth_lognormal_field(n, S=S, tag=2300 + n), device="cuda")
        out = {}
        for tail in (32, 0, 16):
            c.set_vcycle_tail(tail)
            out[tail] = c.fmg_solve_batch(K, want_p=True, kernel=LEVELWISE)
        for tail in (0, 16):
            for a, b in zip(out[32], out[tail]):
                assert _same(a, b), (n, tail)
    c.set_vcycle_tail(32)
    with pytest.raises(fm.FmError):
        c.set_vcycle_tail(24)
