"""MLMC / MLQMC / FMG-MLMC estimators and sample-size control (Sec. 2.2-2.5).

TEST INFRASTRUCTURE ONLY (see the oracle package docstring).

  * telescoping sum E[Q_L] = sum_l E[Y_l], Y_0 = Q_0, Y_l = Q^f_l - Q^c_l (Eq. 2-3),
    the same sample omega for both terms of a level, independent samples
    across levels (Eq. 5);
  * MSE split  sum_l V_l/N_l <= eps^2/2,  bias^2 <= eps^2/2 (Sec. 2.3);
  * optimal N_l minimising sum_l N_l C_l under the variance constraint (Sec.
    2.3 states the problem, not the answer): by Lagrange multipliers
    N_l = (2/eps^2) sqrt(V_l/C_l) sum_k sqrt(V_k C_k), rounded up;
  * Richardson bias estimate |E[Y_L]| / (2^alpha - 1) (Algorithm 1);
  * growth of the finest level (Algorithms 1-3): start at L = L_start; once
    the sample sizes are met (MC: no level needs extra samples; QMC:
    sum_l V[Y^_l] <= eps^2/2), stop if the bias estimate is below
    eps/sqrt(2), else add level L + 1 with a pilot set.  alpha is the
    caller's weak rate, or the fitted slope of -log2|Y^_l| over l = 1..L
    floored at 1/2 (a noisy two-point fit must not drive 2^alpha - 1 to 0);
  * MLQMC (Algorithm 2): R independently shifted point sets per level; the
    level estimate is the mean over shifts and its variance the sample
    variance of the R shift means divided by R; while sum_l V[Y^_l] > eps^2/2
    double N_l on the level maximising V[Y^_l] / (N_l C_l).

Sums are exact-rounded (math.fsum), the plainest correct reduction.
"""
import math

import numpy as np

from . import kl as _kl
from . import lib as _lib


def optimal_samples(V, C, eps):
    """N_l = ceil((2/eps^2) sqrt(V_l/C_l) sum_k sqrt(V_k C_k))."""
    V = np.asarray(V, float)
    C = np.asarray(C, float)
    total = float(np.sum(np.sqrt(V * C)))
    return np.ceil(2.0 / eps ** 2 * np.sqrt(V / C) * total).astype(np.int64)


def cost_model(n_cells):
    """Deterministic cost per sample: finest cells x 4/3 (all FMG grids)."""
    return np.asarray(n_cells, float) * 4.0 / 3.0


class LevelAccumulator:
    """Per-level sums of Y, Y^2, Q^f, Q^c over the samples seen so far."""

    def __init__(self, nlev):
        self.Y = [[] for _ in range(nlev)]
        self.Qf = [[] for _ in range(nlev)]
        self.Qc = [[] for _ in range(nlev)]

    def add(self, l, y, qf, qc):
        self.Y[l].extend(np.asarray(y).tolist())
        self.Qf[l].extend(np.asarray(qf).tolist())
        self.Qc[l].extend(np.asarray(qc).tolist())

    def N(self, l):
        return len(self.Y[l])

    def mean(self, l):
        return math.fsum(self.Y[l]) / len(self.Y[l])

    def var(self, l):
        n = len(self.Y[l])
        m = self.mean(l)
        return math.fsum((y - m) ** 2 for y in self.Y[l]) / (n - 1)


def fit_rate(values, start=1):
    """Least-squares slope of -log2|values_l| against l for l >= start."""
    l = np.arange(start, len(values))
    v = np.abs(np.asarray(values[start:], float))
    if len(l) < 2 or np.any(v <= 0):
        return float("nan")
    A = np.stack([l, np.ones_like(l)], axis=1).astype(float)
    slope = np.linalg.lstsq(A, np.log2(v), rcond=None)[0][0]
    return float(-slope)


def mlmc(sampler, L, eps, n_pilot, cost, max_rounds=50):
    """Algorithm 1 / 3 for a fixed finest level L.
    sampler(l, first, n) -> (Y, Qf, Qc) for samples first..first+n-1 of level l."""
    acc = LevelAccumulator(L + 1)
    dN = np.full(L + 1, n_pilot, np.int64)
    rounds = 0
    while np.any(dN > 0) and rounds < max_rounds:
        for l in range(L + 1):
            if dN[l] > 0:
                y, qf, qc = sampler(l, acc.N(l), int(dN[l]))
                acc.add(l, y, qf, qc)
        V = np.array([acc.var(l) for l in range(L + 1)])
        Nopt = optimal_samples(V, cost, eps)
        dN = np.maximum(0, Nopt - np.array([acc.N(l) for l in range(L + 1)]))
        rounds += 1
    return _report(acc, L, eps, cost, rounds)


def _report(acc, L, eps, cost, rounds):
    means = np.array([acc.mean(l) for l in range(L + 1)])
    V = np.array([acc.var(l) for l in range(L + 1)])
    N = np.array([acc.N(l) for l in range(L + 1)])
    alpha = fit_rate(means, 1)
    beta = fit_rate(V, 1)
    bias = abs(means[L]) / (2.0 ** alpha - 1.0) if np.isfinite(alpha) and alpha > 0 else float("nan")
    return dict(estimate=math.fsum(means), means=means, V=V, N=N,
                var_estimator=float(np.sum(V / N)), alpha=alpha, beta=beta,
                bias=bias, rounds=rounds, cost=float(np.sum(N * cost)), acc=acc)


def mlqmc(sampler, L, eps, n_pilot, R, cost, max_rounds=200):
    """Algorithm 2 for a fixed L.  sampler(l, first, n, r) -> (Y, Qf, Qc) for
    points first..first+n-1 of shift r on level l."""
    Ys = [[[] for _ in range(R)] for _ in range(L + 1)]
    N = np.full(L + 1, n_pilot, np.int64)
    for l in range(L + 1):
        for r in range(R):
            Ys[l][r].extend(np.asarray(sampler(l, 0, n_pilot, r)[0]).tolist())

    def level_stats(l):
        m = np.array([math.fsum(Ys[l][r]) / len(Ys[l][r]) for r in range(R)])
        mean = math.fsum(m) / R
        var_hat = math.fsum((m - mean) ** 2) / (R * (R - 1))
        return mean, var_hat

    rounds = 0
    while rounds < max_rounds:
        stats = [level_stats(l) for l in range(L + 1)]
        Vhat = np.array([s[1] for s in stats])
        if Vhat.sum() <= eps ** 2 / 2:
            break
        l = int(np.argmax(Vhat / (N * cost)))
        for r in range(R):
            Ys[l][r].extend(np.asarray(sampler(l, int(N[l]), int(N[l]), r)[0]).tolist())
        N[l] *= 2
        rounds += 1
    stats = [level_stats(l) for l in range(L + 1)]
    means = np.array([s[0] for s in stats])
    Vhat = np.array([s[1] for s in stats])
    alpha = fit_rate(means, 1)
    bias = abs(means[L]) / (2.0 ** alpha - 1.0) if np.isfinite(alpha) and alpha > 0 else float("nan")
    return dict(estimate=math.fsum(means), means=means, Vhat=Vhat, N=N,
                var_estimator=float(Vhat.sum()), alpha=alpha, bias=bias, rounds=rounds,
                cost=float(np.sum(N * R * cost)))


class FMGSampler:
    """Samples of one FMG-MLMC level: points -> KL field -> FMG -> (Q^f, Q^c).

    levels[l] = n_l (finest grid of level l); basis: a KLBasis (or anything
    with level_basis(n)); seed: the Philox key for MC points and QMC shifts."""

    def __init__(self, levels, basis, seed, prm=None, n0=4, qmc_dirnums=None,
                 n_shifts=0, nthreads=0, rule="shift", lattice_z=None, lattice_m=16):
        """rule (randomized QMC, Sec. 2.4): 'shift' Sobol' + digital shift,
        'owen' Sobol' + nested uniform scrambling (qmc_dirnums needed for
        both), 'lattice' the shifted lattice sequence with generating vector
        lattice_z over 2^lattice_m points."""
        self.levels, self.basis, self.seed = list(levels), basis, seed
        self.prm = prm or _lib.params()
        self.n0 = n0
        self.B = [basis.level_basis(n) for n in self.levels]
        self.V = qmc_dirnums
        self.rule, self.z, self.mz = rule, lattice_z, lattice_m
        self.shifts = None
        if qmc_dirnums is not None and rule == "shift":
            M = self.B[0].shape[1]
            self.shifts = [_lib.sobol_shifts(seed, l, n_shifts, M) for l in range(len(levels))]
        self.nthreads = nthreads
        self.solves = [0] * len(levels)

    def points(self, l, first, n, r=None):
        M = self.B[l].shape[1]
        if r is None:
            return _lib.mc_normals(self.seed, l, first, n, M)
        if self.rule == "owen":
            x = _lib.sobol_owen_points(self.V, self.seed, l, first, n, r, 1)[0]
        elif self.rule == "lattice":
            x = _lib.lattice_points(self.z, self.mz, self.seed, l, first, n, r, 1)[0]
        else:
            _, xi = _lib.sobol_points(self.V, first, n, self.shifts[l][r:r + 1], want_xi=True)
            return xi[0]
        return _lib.norminv((x.astype(np.float64) + 0.5) * 2.0 ** -32)

    def solve(self, l, xi):
        n = self.levels[l]
        K = _kl.synthesize(self.B[l], xi).reshape(-1, n, n)
        qf, qc, _, _ = _lib.fmg_solve_batch(K, self.prm, self.n0, nthreads=self.nthreads)
        self.solves[l] += len(qf)
        return qf, qc

    def __call__(self, l, first, n, r=None):
        qf, qc = self.solve(l, self.points(l, first, n, r))
        y = qf if l == 0 else qf - qc
        return y, qf, qc


class SurrogateLevels:
    """The control-variate level below the coarsest grid (north of the
    paper's Eq. 2): extended level 0 samples S(xi) on its own stream, extended
    level 1 samples Q_0(xi) - S(xi) on level 0's stream, extended level l+1 is
    level l of `sampler`.  E[S] + E[Q_0 - S] + sum_{l>=1} E[Y_l] = E[Q_L] for
    any S.  predict(xi [n][M]) -> S [n]; surrogate_stream is the Philox level
    id of extended level 0."""

    def __init__(self, sampler, predict, surrogate_stream=100):
        self.s, self.predict, self.stream = sampler, predict, surrogate_stream

    def __call__(self, l, first, n, r=None):
        if l == 0:
            M = self.s.B[0].shape[1]
            xi = _lib.mc_normals(self.s.seed, self.stream, first, n, M)
            y = self.predict(xi)
            return y, y, np.zeros_like(y)
        if l == 1:
            xi = self.s.points(0, first, n, r)
            qf, _ = self.s.solve(0, xi)
            return qf - self.predict(xi), qf, self.predict(xi)
        return self.s(l - 1, first, n, r)


ALPHA_MIN = 0.5


def richardson_bias(level_means, alpha=None):
    """Algorithm 1's weak-error estimate |E[Q_L - Q]| ~ |E[Y_L]| / (2^alpha - 1).
    level_means: the means of Y_1 .. Y_L.  Returns (bias, alpha used)."""
    if alpha is None or not alpha > 0:
        a = fit_rate(np.concatenate([[np.nan], level_means]), 1)
        alpha = max(a, ALPHA_MIN) if np.isfinite(a) else ALPHA_MIN
    return abs(level_means[-1]) / (2.0 ** alpha - 1.0), float(alpha)


def mlmc_adaptive(sampler, L_start, L_max, eps, n_pilot, cost, alpha=None, below=0, max_rounds=200):
    """Algorithm 1 (Algorithm 3 with an FMG sampler) with the finest level
    grown from L_start up to at most L_max.  Extended levels e = 0 ..
    below + L: `below` levels sit under MLMC level 0 (1 with the surrogate
    level), cost[e] is the cost of one sample of extended level e.  Each
    round evaluates the extra samples dN_e, then updates V_e and the optimal
    N_e; when no level needs more, the bias test decides between stopping
    and adding a level with n_pilot samples."""
    n_all = below + L_max + 1
    acc = LevelAccumulator(n_all)
    L = L_start
    dN = np.zeros(n_all, np.int64)
    dN[:below + L + 1] = n_pilot
    rounds = 0
    while rounds < max_rounds:
        E = below + L + 1
        for e in range(E):
            if dN[e] > 0:
                y, qf, qc = sampler(e, acc.N(e), int(dN[e]))
                acc.add(e, y, qf, qc)
        rounds += 1
        V = np.array([acc.var(e) for e in range(E)])
        Nopt = optimal_samples(V, cost[:E], eps)
        dN[:E] = np.maximum(0, Nopt - np.array([acc.N(e) for e in range(E)]))
        if np.any(dN[:E] > 0):
            continue
        bias, _ = richardson_bias(np.array([acc.mean(e) for e in range(below + 1, E)]), alpha)
        if bias < eps / math.sqrt(2.0) or L == L_max:
            break
        L += 1
        dN[below + L] = n_pilot
    E = below + L + 1
    means = np.array([acc.mean(e) for e in range(E)])
    V = np.array([acc.var(e) for e in range(E)])
    N = np.array([acc.N(e) for e in range(E)])
    bias, a_used = richardson_bias(means[below + 1:], alpha)
    return dict(estimate=math.fsum(means), means=means, V=V, N=N, var_estimator=float(np.sum(V / N)),
                L=L, bias=bias, alpha_used=a_used, bias_ok=bool(bias < eps / math.sqrt(2.0)), rounds=rounds,
                cost=float(np.sum(N * cost[:E])))


def mlqmc_adaptive(sampler, L_start, L_max, eps, n_pilot, R, cost, alpha=None, below=0, max_rounds=400):
    """Algorithm 2 with the finest level grown from L_start up to at most
    L_max: while sum_e V[Y^_e] > eps^2/2 double N_e on the level maximising
    V[Y^_e] / (N_e C_e); otherwise stop if the bias estimate is below
    eps/sqrt(2), else add a level with n_pilot points per shift.  Each
    doubling and each added level counts as a round."""
    n_all = below + L_max + 1
    Ys = [[[] for _ in range(R)] for _ in range(n_all)]
    N = np.zeros(n_all, np.int64)

    def draw(e, first, n):
        for r in range(R):
            Ys[e][r].extend(np.asarray(sampler(e, first, n, r)[0]).tolist())

    def level_stats(e):
        m = np.array([math.fsum(Ys[e][r]) / len(Ys[e][r]) for r in range(R)])
        mean = math.fsum(m) / R
        return mean, math.fsum((m - mean) ** 2) / (R * (R - 1))

    L = L_start
    for e in range(below + L + 1):
        draw(e, 0, n_pilot)
        N[e] = n_pilot
    rounds = 0
    while rounds < max_rounds:
        E = below + L + 1
        stats = [level_stats(e) for e in range(E)]
        Vhat = np.array([s[1] for s in stats])
        if Vhat.sum() > eps ** 2 / 2:
            e = int(np.argmax(Vhat / (N[:E] * cost[:E])))
            draw(e, int(N[e]), int(N[e]))
            N[e] *= 2
            rounds += 1
            continue
        bias, _ = richardson_bias(np.array([s[0] for s in stats[below + 1:]]), alpha)
        if bias < eps / math.sqrt(2.0) or L == L_max:
            break
        L += 1
        draw(below + L, 0, n_pilot)
        N[below + L] = n_pilot
        rounds += 1
    E = below + L + 1
    stats = [level_stats(e) for e in range(E)]
    means = np.array([s[0] for s in stats])
    Vhat = np.array([s[1] for s in stats])
    bias, a_used = richardson_bias(means[below + 1:], alpha)
    return dict(estimate=math.fsum(means), means=means, Vhat=Vhat, N=N[:E].copy(),
                var_estimator=float(Vhat.sum()), L=L, bias=bias, alpha_used=a_used,
                bias_ok=bool(bias < eps / math.sqrt(2.0)),
                rounds=rounds, cost=float(np.sum(N[:E] * R * cost[:E])))
