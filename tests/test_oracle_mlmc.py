"""Pins of the oracle's estimators (Sec. 2.2-2.5): the sample-size rule, the
telescoping identity under the FMG by-product, and closed-form expectations
of a layered field."""
import numpy as np
import pytest
import scipy.optimize

import workloads as W
from oracle import kl, lib as L, mlmc


def test_optimal_samples_solve_the_constrained_minimisation():
    """Minimise sum N_l C_l s.t. sum V_l/N_l = eps^2/2 (Sec. 2.3) numerically."""
    V = np.array([1e-1, 2e-2, 5e-3, 1e-3, 3e-4])
    C = np.array([1.0, 4.0, 16.0, 64.0, 256.0])
    eps = 1e-2
    N = mlmc.optimal_samples(V, C, eps)
    assert np.sum(V / N) <= eps ** 2 / 2 * (1 + 1e-12)
    res = scipy.optimize.minimize(
        lambda x: np.sum(np.exp(x) * C), np.log(np.full(5, 1e3)),
        constraints=[{"type": "eq", "fun": lambda x: np.sum(V / np.exp(x)) / (eps ** 2 / 2) - 1}],
        method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
    np.testing.assert_allclose(np.exp(res.x), N, rtol=1e-3, atol=1.0)


def _layered_setup(levels, M=16, sigma2=1.0, lam=0.3):
    n_ref = levels[-1]
    Bref, _ = kl.layered_basis_y(n_ref, M, sigma2, lam, q=128)

    class Basis:
        def level_basis(self, n):
            return np.ascontiguousarray(Bref[kl.level_rows(n, n_ref)])

    return Basis()


def _layered_expectation(basis, n):
    """E[Q] for K(y) = exp(g(y)): Q = sum_j K_j / n and E[exp(g)] = exp(Var g / 2)."""
    B = basis.level_basis(n).reshape(n, n, -1)[:, 0, :]    # one row per j
    return float(np.sum(np.exp(0.5 * np.sum(B * B, axis=1))) / n)


def test_per_sample_telescoping_with_fmg_by_product():
    """Same omega on every level: Q^c_l(omega) = Q^f_(l-1)(omega), so
    Q_0 + sum_l (Q^f_l - Q^c_l) = Q^f_L sample by sample (Eq. 2)."""
    levels = [8, 16, 32, 64]
    basis = kl.KLBasis(64, 32, 1.0, 0.3, q=24)
    s = mlmc.FMGSampler(levels, basis, seed=5)
    xi = W.normals(6, 32, tag=40)
    qf = [s.solve(l, xi)[0] for l in range(4)]
    qc = [s.solve(l, xi)[1] for l in range(4)]
    for l in range(1, 4):
        np.testing.assert_allclose(qc[l], qf[l - 1], rtol=1e-13, atol=0)
    tele = qf[0] + sum(qf[l] - qc[l] for l in range(1, 4))
    np.testing.assert_allclose(tele, qf[3], rtol=1e-13)


def test_mlmc_estimate_matches_layered_closed_form():
    levels = [8, 16, 32]
    basis = _layered_setup(levels)
    sampler = mlmc.FMGSampler(levels, basis, seed=7)
    cost = mlmc.cost_model(np.array(levels) ** 2)
    res = mlmc.mlmc(sampler, 2, 4e-3, 200, cost)
    exact = _layered_expectation(basis, levels[-1])
    assert res["var_estimator"] <= (4e-3) ** 2 / 2 * 1.05
    assert abs(res["estimate"] - exact) < 3 * np.sqrt(res["var_estimator"])
    # each level's mean estimates E[Q_l] - E[Q_(l-1)] of the same closed form
    e = [_layered_expectation(basis, n) for n in levels]
    for l in range(3):
        target = e[l] - (e[l - 1] if l else 0.0)
        sd = np.sqrt(res["V"][l] / res["N"][l])
        assert abs(res["means"][l] - target) < 4 * sd + 1e-14


def test_mlqmc_estimate_and_smaller_variance_than_mc():
    levels = [8, 16]
    basis = _layered_setup(levels, M=8)
    V = L.sobol_direction_numbers(8)
    qmc = mlmc.FMGSampler(levels, basis, seed=9, qmc_dirnums=V, n_shifts=8)
    cost = mlmc.cost_model(np.array(levels) ** 2)
    res = mlmc.mlqmc(qmc, 1, 2e-3, 32, 8, cost)
    exact = _layered_expectation(basis, levels[-1])
    assert res["var_estimator"] <= (2e-3) ** 2 / 2
    assert abs(res["estimate"] - exact) < 4 * np.sqrt(res["var_estimator"])
    # Sec. 3.2: QMC lowers the estimator variance at equal points
    N0 = int(res["N"][0]) * 8
    mc = mlmc.FMGSampler(levels, basis, seed=9)
    y = mc(0, 0, N0)[0]
    assert res["Vhat"][0] < np.var(y, ddof=1) / N0


def test_variance_of_corrections_decays_over_levels():
    levels = [8, 16, 32, 64]
    basis = kl.KLBasis(64, 32, 1.0, 0.3, q=24)
    s = mlmc.FMGSampler(levels, basis, seed=11)
    V = [np.var(s(l, 0, 200)[0], ddof=1) for l in range(4)]
    assert V[1] < V[0] and V[2] < V[1] and V[3] < V[2]
    assert mlmc.fit_rate(V, 1) > 0.5


def test_constant_surrogate_reduces_to_plain_mlmc():
    """S = c: extended level 0 averages c, extended level 1 averages Q_0 - c,
    so their sum is the plain level-0 mean sample for sample."""
    levels = [8, 16]
    basis = kl.KLBasis(16, 12, 1.0, 0.3, q=16)
    s = mlmc.FMGSampler(levels, basis, seed=13)
    sur = mlmc.SurrogateLevels(s, lambda xi: np.full(len(xi), 0.75))
    y0 = sur(0, 0, 50)[0]
    y1 = sur(1, 0, 200)[0]
    plain = s(0, 0, 200)[0]
    assert np.all(y0 == 0.75)
    np.testing.assert_allclose(np.mean(y0) + np.mean(y1), np.mean(plain), rtol=1e-14)


def test_bad_surrogate_keeps_the_estimator_unbiased():
    """A surrogate unrelated to Q still gives E[Q_L] within the estimator's RMSE."""
    levels = [8, 16, 32]
    basis = _layered_setup(levels)
    s = mlmc.FMGSampler(levels, basis, seed=17)
    sur = mlmc.SurrogateLevels(s, lambda xi: 1.0 + 0.5 * np.tanh(xi[:, 0] * xi[:, 1]))
    cost = np.concatenate([[1.0], mlmc.cost_model(np.array(levels) ** 2)])
    res = mlmc.mlmc(sur, 3, 5e-3, 100, cost)
    exact = _layered_expectation(basis, levels[-1])
    assert abs(res["estimate"] - exact) < 3 * np.sqrt(res["var_estimator"])
