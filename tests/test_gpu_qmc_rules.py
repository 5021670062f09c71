"""The randomized QMC rules of Sec. 2.4 on the GPU against the oracle: the
randomly shifted rank-1 lattice sequence (its generating vector from the
library's fast component-by-component construction) and nested uniform
(Owen) scrambling of Sobol' points.  Integer points bit-exact; normals
within 1e-13; per-sample QoIs within 1e-10; estimates within their error."""
import numpy as np
import pytest
import torch

from oracle import kl as okl
from oracle import lib as OL
from oracle import mlmc as omlmc

pytestmark = pytest.mark.gpu

M = 24
LATTICE_M = 10


@pytest.fixture(scope="module")
def ctxs():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(32, M, 1.0, 0.3, q=24)
    out = {}
    for rule in (1, 2):
        c = fm.Context(3, 8, M, seed=77, n_shifts=8, qmc_rule=rule, lattice_m=LATTICE_M)
        c.kl_basis_set(basis.B_ref)
        out[rule] = c
    return out, basis


def test_lattice_vector_is_the_oracle_construction(ctxs):
    c, _ = ctxs
    np.testing.assert_array_equal(c[2].lattice_generating_vector(), OL.lattice_cbc(M, 5, LATTICE_M))


def test_lattice_points_bit_exact(ctxs):
    c, _ = ctxs
    z = OL.lattice_cbc(M, 5, LATTICE_M)
    for level, first, n, s0, R in [(0, 0, 1 << LATTICE_M, 0, 2), (2, 77, 300, 3, 4)]:
        x, xi = c[2].qmc_points(2, level, first, n, s0, R)
        ref = OL.lattice_points(z, LATTICE_M, 77, level, first, n, s0, R)
        np.testing.assert_array_equal(x.cpu().numpy().view(np.uint32), ref)
        np.testing.assert_allclose(xi.cpu().numpy(), OL.norminv((ref.astype(np.float64) + 0.5) * 2.0 ** -32),
                                   rtol=1e-13, atol=1e-15)


def test_owen_points_bit_exact(ctxs):
    c, _ = ctxs
    V = OL.sobol_direction_numbers(M)
    for level, first, n, s0, R in [(0, 0, 512, 0, 2), (1, 12345, 97, 5, 3)]:
        x, xi = c[1].qmc_points(1, level, first, n, s0, R)
        ref = OL.sobol_owen_points(V, 77, level, first, n, s0, R)
        np.testing.assert_array_equal(x.cpu().numpy().view(np.uint32), ref)
        np.testing.assert_allclose(xi.cpu().numpy(), OL.norminv((ref.astype(np.float64) + 0.5) * 2.0 ** -32),
                                   rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("rule,name", [(1, "owen"), (2, "lattice")])
def test_sample_level_matches_oracle(ctxs, rule, name):
    c, basis = ctxs
    V = OL.sobol_direction_numbers(M)
    osamp = omlmc.FMGSampler([8, 16, 32], basis, seed=77, qmc_dirnums=V, rule=name,
                             lattice_z=OL.lattice_cbc(M, 5, LATTICE_M), lattice_m=LATTICE_M)
    for level in range(3):
        qf, qc = c[rule].mlmc_sample_level(level, 32, 64, 3, sums=c[rule].new_sums()[0], want_q=True)
        y, rf, rc = osamp(level, 32, 64, 3)
        assert np.max(np.abs(qf.cpu().numpy() - rf) / np.abs(rf)) < 1e-10
        if level > 0:
            assert np.max(np.abs(qc.cpu().numpy() - rc) / np.abs(rc)) < 1e-10


@pytest.mark.parametrize("rule", [1, 2])
def test_mlqmc_estimate_with_each_rule_agrees_with_mlmc(ctxs, rule):
    c, _ = ctxs
    eps = 6e-3
    mc = c[rule].mlmc_estimate(eps, n_pilot=64)
    q = c[rule].mlmc_estimate(eps, qmc=True, n_pilot=32)
    assert q["var_estimator"] <= eps ** 2 / 2 * 1.001
    assert abs(q["estimate"] - mc["estimate"]) < 4 * np.sqrt(q["var_estimator"] + mc["var_estimator"])
    # QMC needs fewer level-0 points than MC for the same variance target
    assert q["N"][0] * 8 < mc["N"][0]


def test_lattice_rule_limits_are_checked(ctxs):
    import paper_1910_04727_gb300 as fm
    c, _ = ctxs
    with pytest.raises(fm.FmError, match="lattice"):
        c[2].qmc_points(2, 0, (1 << LATTICE_M) - 4, 8)
    with pytest.raises(fm.FmError, match="lattice"):
        c[1].qmc_points(2, 0, 0, 8)
