"""The oracle against the set-up the paper prints (tests/golden/paper_setup.json):
Table 1's Case II boundary data, Sec. 3.1's level grids and Table 2's
exponential (nu = 1/2) random fields with the KL trace identity."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import kl, lib as L

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_setup.json")))


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_case_ii_constant_field_outflow_is_the_pressure_drop(level):
    """K = 1 on the unit square with Table 1's Case II data: p = u_W (1 - x)
    exactly and the east outflow is u_W - u_E = 100, on every level grid."""
    c = GOLDEN["case_ii"]
    n = GOLDEN["level_grid"]["side_of_level"][level]
    assert n == 2 ** (level + 2)
    K = np.ones((1, n, n))
    prm = L.params(pW=c["u_west"], pE=c["u_east"], converged=True, tol=1e-14, max_cycles=200)
    qf, _, p, _ = L.fmg_solve_batch(K, prm, want_p=True)
    assert abs(qf[0] - (c["u_west"] - c["u_east"])) < 1e-10 * c["u_west"]
    x = (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(p[0], np.broadcast_to(c["u_west"] * (1 - x), (n, n)), atol=1e-9)


def test_case_ii_outflow_scales_with_the_boundary_data():
    """The problem is linear in the Dirichlet data: Table 1's u_W = 100 gives
    100 times the outflow of u_W = 1 (the default of the workloads) per sample."""
    c = GOLDEN["case_ii"]
    K = W.smooth_lognormal_field(32, S=4, tag=880)
    q1 = L.fmg_solve_batch(K, L.params(pW=1.0, pE=0.0))[0]
    q100 = L.fmg_solve_batch(K, L.params(pW=c["u_west"], pE=c["u_east"]))[0]
    np.testing.assert_allclose(q100, 100.0 * q1, rtol=1e-12)


@pytest.mark.parametrize("field", [0, 1])
def test_table2_exponential_fields_trace_and_capture(field):
    """Table 2's nu = 1/2 fields: the Nystrom spectrum sums to sigma^2 meas(Omega)
    (Sec. 3.1) and a finite number of modes captures 99% of it."""
    f = GOLDEN["random_fields"]["fields"][field]
    assert f["nu"] == 0.5
    theta, _, _, _, trace = kl.nystrom_eigs(24, 24 * 24, f["sigma2"], f["lambda"], all_modes=True)
    area = 1.0
    assert abs(np.sum(theta) - f["sigma2"] * area) < 1e-10
    assert abs(trace - GOLDEN["random_fields"]["trace_over_sigma2"] * f["sigma2"]) < 1e-10
    frac = np.cumsum(np.sort(theta)[::-1]) / np.sum(theta)
    m99 = int(np.searchsorted(frac, GOLDEN["random_fields"]["captured_fraction"]) + 1)
    assert 1 < m99 < theta.size
    # a longer correlation length concentrates the variance in fewer modes
    if field == 1:
        t0, _, _, _, _ = kl.nystrom_eigs(24, 24 * 24, 1.0, 0.5, all_modes=True)
        f0 = np.cumsum(np.sort(t0)[::-1]) / np.sum(t0)
        assert m99 <= int(np.searchsorted(f0, 0.99) + 1)
