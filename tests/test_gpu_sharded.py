"""The estimate shared between two ranks, on one GPU: two contexts driven by
two host threads, the level sums exchanged through a host barrier.  The
ranks only meet on the host between controller rounds, so their kernels
never wait on one another."""
import threading

import numpy as np
import pytest
import torch

from oracle import kl as okl

pytestmark = pytest.mark.gpu


class ThreadGather:
    def __init__(self, world):
        self.world = world
        self.slots = [None] * world
        self.bar = threading.Barrier(world)

    def for_rank(self, rank):
        def gather(data):
            self.slots[rank] = data
            self.bar.wait(timeout=120)
            out = b"".join(self.slots)
            self.bar.wait(timeout=120)
            return out
        return gather


def _ctx(fm, basis, surrogate=False):
    c = fm.Context(3, 16, 32, sigma2=1.0, lam=0.3, seed=31)
    c.kl_basis_set(basis.B_ref)
    return c


@pytest.mark.parametrize("qmc", [False, True])
def test_two_ranks_reproduce_one_rank(qmc):
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(64, 32, 1.0, 0.3, q=32)
    eps = 2e-3
    one = _ctx(fm, basis).mlmc_estimate(eps, qmc=qmc, n_pilot=128 if not qmc else 32)
    ctxs = [_ctx(fm, basis) for _ in range(2)]
    tg = ThreadGather(2)
    res = [None, None]

    def run(rank):
        res[rank] = ctxs[rank].mlmc_estimate(eps, qmc=qmc, n_pilot=128 if not qmc else 32,
                                             shard=(rank, 2, tg.for_rank(rank)))

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert res[0] is not None and res[1] is not None
    assert res[0]["estimate"] == res[1]["estimate"]
    assert list(res[0]["N"]) == list(one["N"]) and list(res[1]["N"]) == list(one["N"])
    assert abs(res[0]["estimate"] - one["estimate"]) <= 1e-13 * abs(one["estimate"])
    assert res[0]["var_estimator"] <= eps ** 2 / 2 * 1.0001
