"""The oracle's energy-optimal coarse-grid correction step (no GPU).

With energy_step the V-cycle adds alpha P e_c with alpha = (r, d) / (d, A d),
d = P e_c: the exact minimiser of the energy error along d for the symmetric
positive definite operator.  Red-black Gauss-Seidel sweeps never raise the
energy error either, so every cycle is monotone in the energy norm whatever
the coarse operators are.  Pinned here:
  * monotone energy error, cycle by cycle, against a dense direct solve on
    high-contrast 16 x 16 and 32 x 32 fields;
  * the step is the line minimum: perturbing alpha either way raises the
    energy error (checked through the same dense operator);
  * on high-contrast 128 x 128 fields where the plain V-cycle diverges
    (contraction factor above 1), the stepped cycle contracts;
  * converged FMG with and without the step reaches the same discrete
    solution on a benign field.
"""
import numpy as np
import pytest

import workloads as W
from oracle import lib as L


def _dense(K):
    n = K.shape[0]
    A = np.zeros((n * n, n * n))
    for c in range(n * n):
        e = np.zeros(n * n)
        e[c] = 1
        A[:, c] = L.apply_A(K, e.reshape(n, n)).ravel()
    return A


def _energy(A, x, xs):
    e = (x - xs).ravel()
    return float(e @ A @ e)


@pytest.mark.parametrize("n", [16, 32])
def test_energy_error_never_rises(n):
    K = W.smooth_lognormal_field(n, S=4, sigma=2.0, modes=24, tag=3200, kmax=12)
    rng = np.random.default_rng(n)
    for k in K:
        A = _dense(k)
        b = rng.standard_normal(n * n)
        xs = np.linalg.solve(A, b).reshape(n, n)
        x = np.zeros((n, n))
        prev = _energy(A, x, xs)
        for _ in range(12):
            x, _ = L.vcycle_solve(k, b.reshape(n, n), x, ncycles=1, energy_step=True)
            cur = _energy(A, x, xs)
            assert cur <= prev * (1 + 1e-12)
            prev = cur
        assert prev < 1e-4 * _energy(A, np.zeros((n, n)), xs)


def test_step_is_the_line_minimum():
    """One V(0, 0) cycle on 8 x 8 (two grids, exact coarse solve): the stepped
    result minus the plain one is (alpha - 1) d, and the energy error along
    that line is smallest at the stepped point."""
    n = 8
    k = W.smooth_lognormal_field(n, S=1, sigma=2.0, modes=12, tag=3300, kmax=6)[0]
    A = _dense(k)
    b = np.random.default_rng(3).standard_normal(n * n)
    xs = np.linalg.solve(A, b).reshape(n, n)
    x0 = np.zeros((n, n))
    xa, _ = L.vcycle_solve(k, b.reshape(n, n), x0, nu1=0, nu2=0, ncycles=1, energy_step=True)
    x1, _ = L.vcycle_solve(k, b.reshape(n, n), x0, nu1=0, nu2=0, ncycles=1, energy_step=False)
    d = x1 - x0                       # the plain cycle adds d = P e_c once
    ea = _energy(A, xa, xs)
    for t in (-0.05, 0.05):
        assert ea < _energy(A, xa + t * d, xs)
    # and (r, d) / (d, A d) from the dense operator gives the same point
    r = b - A @ x0.ravel()
    alpha = (r @ d.ravel()) / (d.ravel() @ A @ d.ravel())
    np.testing.assert_allclose(xa, x0 + alpha * d, rtol=1e-10, atol=1e-12)


def test_stepped_cycle_contracts_where_the_plain_one_diverges():
    n = 128
    K = W.smooth_lognormal_field(n, S=6, sigma=np.sqrt(2.0), modes=24, tag=3100, kmax=12)
    rng = np.random.default_rng(0)
    diverged = 0
    for k in K:
        b = rng.standard_normal((n, n))
        rates = []
        for es in (False, True):
            _, h = L.vcycle_solve(k, b, np.zeros((n, n)), ncycles=12, energy_step=es)
            rates.append((h[-1] / h[4]) ** (1 / 8))
        diverged += rates[0] > 1.0
        assert rates[1] < 0.7, (float(k.max() / k.min()), rates)
    assert diverged >= 1   # the set holds a field the plain cycle cannot solve


def test_stepped_fmg_reaches_the_same_solution():
    K = W.smooth_lognormal_field(64, S=3, sigma=1.0, tag=3400)
    a = L.fmg_solve_batch(K, L.params(converged=True, tol=1e-13, max_cycles=200))
    b = L.fmg_solve_batch(K, L.params(converged=True, tol=1e-13, max_cycles=200, energy_step=True))
    # both stop at a relative residual of 1e-13; the outflux error scales like n tol
    np.testing.assert_allclose(b[0], a[0], rtol=1e-10)
    np.testing.assert_allclose(b[1], a[1], rtol=1e-10)
