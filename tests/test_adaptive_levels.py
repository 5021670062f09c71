"""Growth of the finest level by the bias test (Algorithms 1-3), no GPU.

The oracle's adaptive estimators are pinned to a model whose level means
are known exactly: Q_l = Q - c 2^(-alpha l), so E[Y_l] = c (2^alpha - 1)
2^(-alpha l) for l >= 1 and the true weak error after level L is c
2^(-alpha L), which the Richardson estimate reproduces exactly.  Without
noise the run must stop at the first L whose true error is below
eps/sqrt(2); with noise, the mean squared error over many seeds must stay
near eps^2.  The library's controller must then make the oracle's
decisions (levels, sample sizes, rounds) on the same samples, in one
process and over two gloo ranks.
"""
import math
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest
from scipy.special import ndtri

from oracle import mlmc

Q_INF, C_BIAS = 1.25, 0.5


def _splitmix(x):
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(0xFFFFFFFFFFFFFFFF)
    return x ^ (x >> np.uint64(31))


def _normals(seed, e, r, first, n):
    """Standard normals of samples first .. first+n-1, one per sample id."""
    with np.errstate(over="ignore"):
        ids = np.arange(first, first + n, dtype=np.uint64)
        key = np.uint64((seed * 1000003 + e * 131 + (r + 1)) & 0xFFFFFFFF) << np.uint64(32)
        w = _splitmix(ids ^ key)
    u = ((w >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return ndtri(u)


class Model:
    """Extended levels e = 0 .. below + L_max: `below` base levels under MLMC
    level 0 (like the surrogate level), then Y_0 = Q_0 and Y_l = Q_l - Q_{l-1}
    with Q_l = Q_INF - C_BIAS 2^(-alpha l); noise sd s0 2^(-beta l / 2)."""

    def __init__(self, alpha, L_max, below=0, s0=0.0, beta=2.0, seed=1):
        self.alpha, self.below, self.s0, self.beta, self.seed = alpha, below, s0, beta, seed
        q = [Q_INF - C_BIAS * 2.0 ** (-alpha * l) for l in range(L_max + 1)]
        y = [q[0]] + [q[l] - q[l - 1] for l in range(1, L_max + 1)]
        base = [0.75, -0.25][:below]
        if below:
            y[0] -= sum(base)          # base levels plus level 0 still sum to Q_0
        self.mu = base + y
        self.sd = [s0] * below + [s0 * 2.0 ** (-beta * l / 2) for l in range(L_max + 1)]

    def true_value(self, L):
        return Q_INF - C_BIAS * 2.0 ** (-self.alpha * L)

    def __call__(self, e, first, n, r=None):
        y = self.mu[e] + (self.sd[e] * _normals(self.seed, e, -1 if r is None else r, first, n)
                          if self.sd[e] > 0 else np.zeros(n))
        return y, y, np.zeros(n)


def _cost(n_ext, below=0, gamma=2.0):
    return np.array([0.05] * below + [2.0 ** (gamma * l) for l in range(n_ext - below)])


# ------------------------------------------------------------------ oracle pins

@pytest.mark.parametrize("alpha", [0.75, 1.0, 2.0])
@pytest.mark.parametrize("given", [True, False])
def test_noiseless_run_stops_at_the_first_level_with_small_true_bias(alpha, given):
    L_start, L_max = 2, 9
    for x in np.linspace(1.0, 3.5, 41):
        eps = 10.0 ** -x
        m = Model(alpha, L_max)
        r = mlmc.mlmc_adaptive(m, L_start, L_max, eps, 4, _cost(L_max + 1), alpha=alpha if given else None)
        true_bias = [C_BIAS * 2.0 ** (-alpha * L) for L in range(L_max + 1)]
        ok = [L for L in range(L_start, L_max + 1) if true_bias[L] < eps / math.sqrt(2.0)]
        assert r["L"] == (ok[0] if ok else L_max), (eps, r["L"])
        assert r["bias_ok"] == bool(ok)
        assert abs(r["estimate"] - m.true_value(r["L"])) < 1e-14
        assert math.isclose(r["bias"], true_bias[r["L"]], rel_tol=1e-9)
        assert math.isclose(r["alpha_used"], alpha, rel_tol=1e-9)
        if ok:
            assert abs(r["estimate"] - Q_INF) < eps / math.sqrt(2.0)


def test_noiseless_mlqmc_stops_at_the_same_level():
    for x in np.linspace(1.0, 3.5, 21):
        eps = 10.0 ** -x
        m = Model(1.0, 9)
        a = mlmc.mlmc_adaptive(m, 2, 9, eps, 4, _cost(10))
        b = mlmc.mlqmc_adaptive(m, 2, 9, eps, 4, 4, _cost(10))
        assert a["L"] == b["L"] and a["bias_ok"] == b["bias_ok"]
        assert abs(a["estimate"] - b["estimate"]) < 1e-14


def test_a_shallow_fitted_rate_is_floored():
    """A fitted alpha below 1/2 is replaced by 1/2; a given alpha is used as is."""
    m = Model(0.3, 6)
    r = mlmc.mlmc_adaptive(m, 2, 6, 1e-2, 4, _cost(7))
    assert r["alpha_used"] == 0.5
    mu_L = C_BIAS * (2.0 ** 0.3 - 1.0) * 2.0 ** (-0.3 * r["L"])
    assert math.isclose(r["bias"], mu_L / (2.0 ** 0.5 - 1.0), rel_tol=1e-12)
    r2 = mlmc.mlmc_adaptive(m, 2, 6, 1e-2, 4, _cost(7), alpha=0.3)
    assert r2["alpha_used"] == 0.3 and r2["L"] >= r["L"]


@pytest.mark.parametrize("qmc", [False, True])
def test_noisy_runs_meet_the_mse_target(qmc):
    """Over 40 seeds the mean squared error against Q stays within 1.5 eps^2
    (variance <= eps^2/2 by the sample-size rule, bias^2 <= eps^2/2 by the
    test), and every run's own variance estimate meets its half."""
    eps, L_max = 1e-2, 9
    errs = []
    for seed in range(40):
        m = Model(1.0, L_max, s0=0.05, seed=seed)
        if qmc:
            r = mlmc.mlqmc_adaptive(m, 2, L_max, eps, 16, 8, _cost(L_max + 1))
        else:
            r = mlmc.mlmc_adaptive(m, 2, L_max, eps, 32, _cost(L_max + 1))
        assert r["var_estimator"] <= eps ** 2 / 2
        errs.append(r["estimate"] - Q_INF)
    mse = float(np.mean(np.square(errs)))
    assert mse < 1.5 * eps ** 2, (mse, eps ** 2)


# ------------------------------------------------------------------ native controller

def _neumaier(pair, x):
    s, c = pair[0], pair[1]
    t = s + x
    c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
    pair[0], pair[1] = t, c


class Sums:
    """Running level sums (samples added in request order) for the native controller."""

    def __init__(self, model, n_ext, R=1):
        from paper_1910_04727_gb300 import _lib
        self.m, self.R = model, R
        self.sums = (_lib.FmLevelSums * (n_ext * R))()

    def enqueue(self, e, first, n, shift):
        y, _, _ = self.m(e, first, n, None if shift < 0 else shift)
        cell = self.sums[e * self.R + max(shift, 0)]
        for v in y:
            _neumaier(cell.sum_y, float(v))
            _neumaier(cell.sum_y2, float(v) * float(v))
        cell.count += n

    def read(self):
        return list(self.sums)


# the run stops in the middle (bias test passed) or at the last level (failed)
CASES = [(1.0, 0, 2e-2), (1.0, 1, 1e-2), (2.0, 0, 5e-4), (0.6, 1, 4e-2), (1.0, 0, 2e-3)]


@pytest.mark.parametrize("alpha,below,eps", CASES)
@pytest.mark.parametrize("given", [False, True])
def test_native_core_makes_the_oracle_decisions(alpha, below, eps, given):
    import paper_1910_04727_gb300 as fm
    L_max, L_start = 8, 2
    m = Model(alpha, L_max, below=below, s0=0.05, seed=11)
    cost = _cost(below + L_max + 1, below)
    a = alpha if given else None
    ref = mlmc.mlmc_adaptive(m, L_start, L_max, eps, 32, cost, alpha=a, below=below)
    h = Sums(m, len(cost))
    r = fm.estimate_core(cost, eps, h.enqueue, h.read, n_pilot=32, level0=below,
                         adapt_from=below + L_start + 1, alpha=a or 0.0)
    assert r["n_ext_used"] == below + ref["L"] + 1
    assert list(r["N"]) == list(ref["N"]) and r["rounds"] == ref["rounds"]
    assert math.isclose(r["estimate"], ref["estimate"], rel_tol=1e-12)
    assert r["bias_ok"] == ref["bias_ok"]
    assert math.isclose(r["bias"], ref["bias"], rel_tol=1e-9)
    assert math.isclose(r["alpha_used"], ref["alpha_used"], rel_tol=1e-9)


@pytest.mark.parametrize("alpha,below,eps", CASES[:4])
def test_native_core_makes_the_oracle_mlqmc_decisions(alpha, below, eps):
    import paper_1910_04727_gb300 as fm
    L_max, L_start, R = 8, 2, 8
    m = Model(alpha, L_max, below=below, s0=0.05, seed=12)
    cost = _cost(below + L_max + 1, below)
    ref = mlmc.mlqmc_adaptive(m, L_start, L_max, eps, 16, R, cost, below=below)
    h = Sums(m, len(cost), R)
    r = fm.estimate_core(cost, eps, h.enqueue, h.read, qmc=True, n_shifts=R, n_pilot=16, level0=below,
                         adapt_from=below + L_start + 1)
    assert r["n_ext_used"] == below + ref["L"] + 1
    assert list(r["N"]) == list(ref["N"]) and r["rounds"] == ref["rounds"]
    assert math.isclose(r["estimate"], ref["estimate"], rel_tol=1e-12)
    assert r["bias_ok"] == ref["bias_ok"]


def test_starting_at_the_last_level_is_the_fixed_level_run():
    import paper_1910_04727_gb300 as fm
    m = Model(1.0, 4, s0=0.05, seed=13)
    cost = _cost(5)
    h1, h2 = Sums(m, 5), Sums(m, 5)
    a = fm.estimate_core(cost, 1e-3, h1.enqueue, h1.read, n_pilot=32)
    b = fm.estimate_core(cost, 1e-3, h2.enqueue, h2.read, n_pilot=32, adapt_from=5)
    assert list(a["N"]) == list(b["N"]) and a["estimate"] == b["estimate"] and a["rounds"] == b["rounds"]
    assert a["n_ext_used"] == 5 and math.isclose(a["bias"], b["bias"])


def test_fmg_sampler_grows_like_the_oracle():
    """The oracle FMG-MLMC sampler (8 x 8 .. 64 x 64, layered field): the
    native controller and the oracle's Algorithm 3 grow to the same level."""
    import paper_1910_04727_gb300 as fm
    from oracle import kl
    levels = [8, 16, 32, 64]
    Bref, _ = kl.layered_basis_y(levels[-1], 16, 1.0, 0.3, q=128)

    class Basis:
        def level_basis(self, n):
            return np.ascontiguousarray(Bref[kl.level_rows(n, levels[-1])])

    cost = mlmc.cost_model(np.array(levels) ** 2)
    ref = mlmc.mlmc_adaptive(mlmc.FMGSampler(levels, Basis(), seed=23), 1, 3, 6e-3, 64, cost)
    s = mlmc.FMGSampler(levels, Basis(), seed=23)

    class H(Sums):
        def enqueue(self, e, first, n, shift):
            y, _, _ = s(e, first, n)
            cell = self.sums[e]
            for v in y:
                _neumaier(cell.sum_y, float(v))
                _neumaier(cell.sum_y2, float(v) * float(v))
            cell.count += n

    h = H(None, len(levels))
    r = fm.estimate_core(cost, 6e-3, h.enqueue, h.read, n_pilot=64, adapt_from=2)
    assert r["n_ext_used"] == ref["L"] + 1
    assert list(r["N"]) == list(ref["N"])
    assert math.isclose(r["estimate"], ref["estimate"], rel_tol=1e-12)


# ------------------------------------------------------------------ two gloo ranks

def _run_rank(rank, world, port, out):
    import torch.distributed as dist

    import paper_1910_04727_gb300 as fm
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = Model(1.0, 8, below=1, s0=0.05, seed=14)
        cost = _cost(10, 1)
        h = Sums(m, len(cost))
        r = fm.estimate_core(cost, 1e-2, h.enqueue, h.read, gather=fm.allgather_over(), n_pilot=32,
                             rank=rank, world=world, level0=1, adapt_from=4)
        out.put((rank, r["n_ext_used"], list(r["N"]), r["rounds"], r["estimate"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_grow_like_one_rank():
    import paper_1910_04727_gb300 as fm
    m = Model(1.0, 8, below=1, s0=0.05, seed=14)
    cost = _cost(10, 1)
    h = Sums(m, len(cost))
    one = fm.estimate_core(cost, 1e-2, h.enqueue, h.read, n_pilot=32, level0=1, adapt_from=4)
    assert 4 < one["n_ext_used"] < 10 and one["bias_ok"]
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_run_rank, args=(rank, 2, port, q)) for rank in range(2)]
    for p in procs:
        p.start()
    res = dict((v[0], v[1:]) for v in (q.get(timeout=600) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][:3] == res[1][:3]
    E, N, rounds, est = res[0]
    assert E == one["n_ext_used"] and N == list(one["N"]) and rounds == one["rounds"]
    assert math.isclose(est, one["estimate"], rel_tol=1e-13)


def test_adaptive_options_are_checked():
    import paper_1910_04727_gb300 as fm
    m = Model(1.0, 4, below=1, s0=0.05, seed=15)
    cost = _cost(6, 1)
    for kw in (dict(level0=1, adapt_from=2),        # fewer than MLMC levels 0 and 1
               dict(level0=0, adapt_from=7),        # more than n_ext
               dict(level0=6, adapt_from=6)):       # level 0 outside the extended levels
        h = Sums(m, len(cost))
        with pytest.raises(fm.FmError):
            fm.estimate_core(cost, 1e-2, h.enqueue, h.read, n_pilot=32, **kw)
