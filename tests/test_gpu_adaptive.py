"""The estimator with the finest level grown by the bias test (Algorithms 1-3)
on the GPU, against the oracle's adaptive estimators on the same samples.

The FP64 fixed-schedule context draws the oracle sampler's points and
solves its problems to 1e-10, so both controllers see the same level
statistics and make the same decisions (levels, sample sizes, rounds).
"""
import math

import numpy as np
import pytest
import torch

from oracle import kl as okl
from oracle import lib as OL
from oracle import mlmc as omlmc

pytestmark = pytest.mark.gpu

LEVELS = [8, 16, 32, 64]
M, R, SEED = 32, 8, 51


@pytest.fixture(scope="module")
def setup():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(LEVELS[-1], M, 1.0, 0.3, q=32)
    ctx = fm.Context(len(LEVELS), LEVELS[0], M, sigma2=1.0, lam=0.3, seed=SEED, n_shifts=R)
    ctx.kl_basis_set(basis.B_ref)
    return fm, ctx, basis


def _cost():
    return omlmc.cost_model(np.array(LEVELS) ** 2)


def _same_decisions(res, ref, n_key="N"):
    assert res["L"] == ref["L"]
    N = np.asarray(res[n_key])[:ref["L"] + 1]
    if np.array_equal(N, ref["N"]):
        assert res["rounds"] == ref["rounds"]
        assert abs(res["estimate"] - ref["estimate"]) < 1e-9 * abs(ref["estimate"])
    else:   # a ceil at a tie may round one level's size differently
        assert np.max(np.abs(N - ref["N"]) / ref["N"]) < 0.01
    assert res["bias_ok"] == ref["bias_ok"]


def test_mc_growth_matches_oracle(setup):
    fm, ctx, basis = setup
    eps = 1e-2
    res = ctx.mlmc_estimate(eps, n_pilot=64, L_start=1)
    ref = omlmc.mlmc_adaptive(omlmc.FMGSampler(LEVELS, basis, seed=SEED), 1, 3, eps, 64, _cost())
    print("GPU", res["L"], res["N"], res["bias"], "oracle", ref["L"], ref["N"], ref["bias"])
    assert ref["L"] > 1                     # the level did grow
    _same_decisions(res, ref)
    assert math.isclose(res["bias"], ref["bias"], rel_tol=1e-6)
    assert res["var_estimator"] <= eps ** 2 / 2 * 1.001


def test_qmc_growth_matches_oracle(setup):
    fm, ctx, basis = setup
    eps = 3e-3
    res = ctx.mlmc_estimate(eps, qmc=True, n_pilot=16, L_start=1, alpha=1.0)
    samp = omlmc.FMGSampler(LEVELS, basis, seed=SEED, qmc_dirnums=OL.sobol_direction_numbers(M), n_shifts=R)
    ref = omlmc.mlqmc_adaptive(samp, 1, 3, eps, 16, R, _cost(), alpha=1.0)
    print("GPU", res["L"], res["N"], "oracle", ref["L"], ref["N"])
    assert ref["L"] > 1
    _same_decisions(res, ref)
    assert res["alpha_used"] == 1.0
    assert res["var_estimator"] <= eps ** 2 / 2


@pytest.mark.parametrize("qmc", [False, True])
def test_start_at_the_last_level_is_the_fixed_level_run(setup, qmc):
    fm, ctx, _ = setup
    kw = dict(qmc=qmc, n_pilot=16 if qmc else 64)
    a = ctx.mlmc_estimate(6e-3, **kw)
    b = ctx.mlmc_estimate(6e-3, L_start=len(LEVELS) - 1, **kw)
    assert list(a["N"]) == list(b["N"]) and a["rounds"] == b["rounds"] and a["estimate"] == b["estimate"]
    assert a["L"] == b["L"] == len(LEVELS) - 1
    assert a["bias"] == b["bias"] and a["bias_ok"] == b["bias_ok"]
    # the reported bias is the Richardson estimate of the last level in use
    assert math.isclose(a["bias"], abs(a["means"][-1]) / (2.0 ** a["alpha_used"] - 1.0), rel_tol=1e-12)


def test_batched_rounds_grow_the_same_way(setup):
    fm, ctx, _ = setup
    a = ctx.mlmc_estimate(1e-2, n_pilot=64, L_start=1)
    b = ctx.mlmc_estimate(1e-2, n_pilot=64, L_start=1, batched=True)
    assert a["L"] == b["L"] and list(a["N"]) == list(b["N"]) and a["rounds"] == b["rounds"]
    assert abs(a["estimate"] - b["estimate"]) <= 1e-14 * abs(a["estimate"])


def test_growth_with_the_surrogate_level(setup):
    """With the surrogate level below level 0 the bias test still reads the
    MLMC levels 1 .. L; the estimate agrees with the plain adaptive one."""
    fm, ctx, _ = setup
    ctx.surrogate_train(n_train=4096, epochs=20, lr=3e-3, seed=3, batch=512)
    eps = 1e-2
    plain = ctx.mlmc_estimate(eps, n_pilot=64, L_start=1)
    sur = ctx.mlmc_estimate(eps, n_pilot=64, L_start=1, surrogate=True, surrogate_cost=0.02)
    assert sur["L"] >= 1 and sur["N_s"] > 0
    assert sur["var_estimator"] <= eps ** 2 / 2 * 1.001
    assert math.isclose(sur["bias"], abs(sur["means"][sur["L"]]) / (2.0 ** sur["alpha_used"] - 1.0),
                        rel_tol=1e-12)
    assert abs(sur["estimate"] - plain["estimate"]) < 3 * math.sqrt(sur["var_estimator"] + plain["var_estimator"])


def test_bad_start_levels_are_rejected(setup):
    fm, ctx, _ = setup
    for L0 in (0, len(LEVELS)):
        with pytest.raises(fm.FmError):
            ctx.mlmc_estimate(1e-2, n_pilot=64, L_start=L0)
    torch.cuda.synchronize()
