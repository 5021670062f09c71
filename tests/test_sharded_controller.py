"""The sample-size controller shared among ranks (no GPU).

mlmc_estimate_core is the library's host controller: it asks for samples,
reads running sums and exchanges them between ranks.  Here its samples come
from the CPU oracle and the exchange from torch.distributed over gloo, with
two ranks in two processes; the schedule and the estimate must be those of
one rank, and the oracle's own controller (Sec. 2.3 rule) must agree.
"""
import math
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import workloads as W
from oracle import kl, mlmc

LEVELS = [8, 16, 32]
EPS = 6e-3


def test_shard_ranges_partition_every_request():
    import paper_1910_04727_gb300 as fm
    for first, n in [(0, 0), (0, 1), (5, 7), (1000, 1001), (3, 64)]:
        for world in (1, 2, 3, 8):
            parts = [fm.shard_range(first, n, r, world) for r in range(world)]
            assert parts[0][0] == first
            for (f0, n0), (f1, _) in zip(parts, parts[1:]):
                assert f0 + n0 == f1                      # contiguous, in rank order
            assert sum(c for _, c in parts) == n
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
    # a rank outside the group gets nothing
    assert fm.shard_range(0, 10, 2, 2)[1] == 0


def _basis():
    Bref, _ = kl.layered_basis_y(LEVELS[-1], 16, 1.0, 0.3, q=128)

    class Basis:
        def level_basis(self, n):
            return np.ascontiguousarray(Bref[kl.level_rows(n, LEVELS[-1])])
    return Basis()


def _neumaier(pair, x):
    s, c = pair[0], pair[1]
    t = s + x
    c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
    pair[0], pair[1] = t, c


class HostSampler:
    """Running level sums of the oracle sampler (samples in id order)."""

    def __init__(self, n_ext):
        from paper_1910_04727_gb300 import _lib
        self.s = mlmc.FMGSampler(LEVELS, _basis(), seed=23)
        self.sums = (_lib.FmLevelSums * n_ext)()
        self.drawn = [[] for _ in range(n_ext)]

    def enqueue(self, e, first, n, shift):
        y, qf, qc = self.s(e, first, n)
        cell = self.sums[e]
        for v, f, c in zip(y, qf, qc):
            _neumaier(cell.sum_y, float(v))
            _neumaier(cell.sum_y2, float(v) * float(v))
            _neumaier(cell.sum_qf, float(f))
            _neumaier(cell.sum_qc, float(c) if e > 0 else 0.0)
        cell.count += n
        self.drawn[e].append((first, n))

    def read(self):
        return list(self.sums)


def _cost():
    return mlmc.cost_model(np.array(LEVELS) ** 2)


def _run_rank(rank, world, port, out):
    import torch.distributed as dist

    import paper_1910_04727_gb300 as fm
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h = HostSampler(len(LEVELS))
        r = fm.estimate_core(_cost(), EPS, h.enqueue, h.read, gather=fm.allgather_over(),
                             n_pilot=64, rank=rank, world=world)
        out.put((rank, r["estimate"], r["var_estimator"], list(r["N"]), r["rounds"], h.drawn))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def single():
    import paper_1910_04727_gb300 as fm
    h = HostSampler(len(LEVELS))
    r = fm.estimate_core(_cost(), EPS, h.enqueue, h.read, n_pilot=64)
    return r, h


def test_core_follows_the_oracle_controller(single):
    """One rank: the library's controller and the oracle's (Sec. 2.3 rule with
    exact sums) reach the same sample sizes and the same estimate."""
    r, _ = single
    ref = mlmc.mlmc(mlmc.FMGSampler(LEVELS, _basis(), seed=23), len(LEVELS) - 1, EPS, 64, _cost())
    assert list(r["N"]) == list(ref["N"])
    assert math.isclose(r["estimate"], ref["estimate"], rel_tol=1e-12)
    assert math.isclose(r["var_estimator"], ref["var_estimator"], rel_tol=1e-9)
    assert r["var_estimator"] <= EPS ** 2 / 2


def test_two_gloo_ranks_reproduce_one_rank(single):
    r1, h1 = single
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_run_rank, args=(rank, 2, port, q)) for rank in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, est, var, N, rounds, drawn = q.get(timeout=600)
        res[rank] = (est, var, N, rounds, drawn)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks hold the same result
    assert res[0][:4] == res[1][:4]
    est, var, N, rounds, _ = res[0]
    assert N == list(r1["N"]) and rounds == r1["rounds"]
    # the same samples, summed in another order
    assert math.isclose(est, r1["estimate"], rel_tol=1e-13)
    assert math.isclose(var, r1["var_estimator"], rel_tol=1e-9)
    # the two ranks' requests tile each level's sample ids 0 .. N_l - 1 exactly
    for e, n_total in enumerate(N):
        ids = sorted(i for rank in (0, 1) for f, n in res[rank][4][e] for i in range(f, f + n))
        assert ids == list(range(n_total))


class HostQMCSampler(HostSampler):
    """Level sums per (level, shift) of the oracle's randomized-QMC sampler."""

    def __init__(self, n_ext, R):
        from paper_1910_04727_gb300 import _lib
        from oracle import lib as OL
        self.s = mlmc.FMGSampler(LEVELS, _basis(), seed=29, qmc_dirnums=OL.sobol_direction_numbers(16),
                                 n_shifts=R)
        self.R = R
        self.sums = (_lib.FmLevelSums * (n_ext * R))()
        self.drawn = [[] for _ in range(n_ext)]

    def enqueue(self, e, first, n, shift):
        y, qf, qc = self.s(e, first, n, shift)
        cell = self.sums[e * self.R + shift]
        for v, f, c in zip(y, qf, qc):
            _neumaier(cell.sum_y, float(v))
            _neumaier(cell.sum_y2, float(v) * float(v))
            _neumaier(cell.sum_qf, float(f))
            _neumaier(cell.sum_qc, float(c) if e > 0 else 0.0)
        cell.count += n


def test_core_follows_the_oracle_mlqmc_doubling_rule():
    """QMC (Algorithm 2): R shifted Sobol' point sets per level, the doubling
    rule on the level maximising V[Y^_l] / (N_l C_l); the native controller
    and the oracle reach the same N_l and estimate."""
    import paper_1910_04727_gb300 as fm
    R, eps = 4, 2e-3
    h = HostQMCSampler(len(LEVELS), R)
    r = fm.estimate_core(_cost(), eps, h.enqueue, h.read, qmc=True, n_shifts=R, n_pilot=8)
    from oracle import lib as OL
    ref_s = mlmc.FMGSampler(LEVELS, _basis(), seed=29, qmc_dirnums=OL.sobol_direction_numbers(16), n_shifts=R)
    ref = mlmc.mlqmc(ref_s, len(LEVELS) - 1, eps, 8, R, _cost())
    assert list(r["N"]) == list(ref["N"]) and r["rounds"] == ref["rounds"]
    assert math.isclose(r["estimate"], ref["estimate"], rel_tol=1e-12)
    assert r["var_estimator"] <= eps ** 2 / 2
