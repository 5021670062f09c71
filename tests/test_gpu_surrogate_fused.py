"""The fused MC inference kernel against the layer-by-layer path.

For inputs up to 256 wide, surrogate_eval_mc runs the whole network in one
kernel per 128 rows (inputs formed from the Philox words in shared memory,
the hidden layers back to back on the tensor cores, the output layer in the
same summation order).  It must give S bit for bit as the layer-by-layer
path does, for every row count (ragged last tile, one row, many tiles), for
input widths 128 and 256 (padded), and it must agree with the FP64 oracle
network on the same inputs.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kl as okl
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def _ctx(M, seed):
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(32, M, 1.0, 0.3, q=max(32, int(np.ceil(np.sqrt(8 * M)))))
    c = fm.Context(2, 16, M, sigma2=1.0, lam=0.3, seed=seed)
    c.kl_basis_set(basis.B_ref)
    r = W.rng(tag=900 + M)
    params = np.concatenate([np.concatenate([Wl.ravel(), bl.ravel()]) for Wl, bl in
                             omlp.init_params(M, lambda n: r.uniform(size=n))]).astype(np.float32)
    c.surrogate_set_params(params, mu=0.7, sd=0.4)
    return c


@pytest.mark.parametrize("M", [64, 128, 200])
def test_fused_equals_layer_by_layer(M):
    c = _ctx(M, 31 + M)
    try:
        for level, first, n in [(0, 0, 1), (0, 17, 127), (3, 5, 128), (12, 1 << 33, 129), (1, 999, 20000),
                                (12, 0, (1 << 18) + 5)]:
            c.surrogate_set_fused(True)
            a = c.surrogate_eval_mc(level, first, n).cpu().numpy()
            c.surrogate_set_fused(False)
            b = c.surrogate_eval_mc(level, first, n).cpu().numpy()
            assert np.array_equal(a, b), (M, level, first, n, np.max(np.abs(a - b)))
        c.surrogate_set_fused(True)
    finally:
        c.close()


def test_wide_inputs_take_the_layer_by_layer_path():
    """M = 300 pads to 384 input columns, beyond the fused kernel's 256: the
    switch changes nothing there."""
    c = _ctx(300, 7)
    try:
        a = c.surrogate_eval_mc(0, 3, 1000).cpu().numpy()
        c.surrogate_set_fused(False)
        b = c.surrogate_eval_mc(0, 3, 1000).cpu().numpy()
        assert np.array_equal(a, b)
    finally:
        c.close()


def test_fused_matches_the_oracle_network():
    M = 128
    c = _ctx(M, 5)
    try:
        n = 4096
        s = c.surrogate_eval_mc(0, 77, n).cpu().numpy()
        xi = c.mc_points(0, 77, n).cpu().numpy()
        r = W.rng(tag=900 + M)
        pairs = omlp.init_params(M, lambda k: r.uniform(size=k))
        pairs = [(Wl.astype(np.float32).astype(np.float64), bl.astype(np.float32).astype(np.float64))
                 for Wl, bl in pairs]
        out, _ = omlp.forward(pairs, xi, rounding=True)
        ref = 0.7 + 0.4 * out
        # the FP32 Philox-word inputs differ from the FP64 points in the odd
        # BF16 rounding; the rest is FP32 vs FP64 accumulation
        d = np.abs(s - ref)
        assert np.median(d) < 1e-5
        assert np.mean(d > 1e-3) < 0.01
    finally:
        c.close()
