"""Training the surrogate beside other work (fm_train_opts.async_run).

The training steps run on the network's own stream while the caller goes on
(an estimator round solving its levels, say); every use of the network waits
for the last step on the device.  The run must leave exactly the network a
synchronous run leaves, and an estimate started before the steps end must
equal, bit for bit, the one started after a synchronous run.
"""
import numpy as np
import pytest
import torch

from oracle import kl as okl

pytestmark = pytest.mark.gpu

M = 128
TRAIN = dict(n_train=4096, epochs=4, lr=3e-3, seed=11, batch=256)


@pytest.fixture(scope="module")
def ctx():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(64, M, 1.0, 0.3, q=32)
    c = fm.Context(3, 16, M, sigma2=1.0, lam=0.3, seed=77, precision=1, converged=True, tol=1e-12, qtol=1e-10,
                   max_cycles=200)
    c.kl_basis_set(basis.B_ref)
    yield c
    c.close()


def _estimate(c, batched):
    r = c.mlmc_estimate(4e-3, n_pilot=256, surrogate=True, surrogate_cost=0.01, batched=batched)
    return r["estimate"], r["var_estimator"], list(r["N"]), r["N_s"]


@pytest.mark.parametrize("batched", [True, False])
def test_estimate_beside_the_training_equals_the_synchronous_one(ctx, batched):
    rep_sync = ctx.surrogate_train(**TRAIN)
    p_sync = ctx.surrogate_get_params()
    est_sync = _estimate(ctx, batched)

    rep0 = ctx.surrogate_train(**TRAIN, async_run=True)
    # known at launch; the rest after the finish
    assert rep0["mu"] == rep_sync["mu"] and rep0["sd"] == rep_sync["sd"]
    assert rep0["steps"] == rep_sync["steps"]
    assert np.isnan(rep0["loss_last"]) and np.isnan(rep0["corr"])
    est_async = _estimate(ctx, batched)   # enqueued while the steps may still run
    rep = ctx.surrogate_train_finish()
    p_async = ctx.surrogate_get_params()

    assert np.array_equal(p_sync, p_async)
    assert est_async == est_sync
    for k in ("loss_first", "loss_last", "corr", "var_q", "var_residual"):
        assert rep[k] == rep_sync[k], k


def test_evaluation_waits_for_the_steps(ctx):
    import paper_1910_04727_gb300 as fm
    ctx.surrogate_train(**TRAIN)
    ref = ctx.surrogate_eval_mc(0, 5000, 20000).cpu().numpy()
    ctx.surrogate_train(**TRAIN, async_run=True)
    got = ctx.surrogate_eval_mc(0, 5000, 20000)   # ordered after the last step on the device
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)
    ctx.surrogate_train_finish()
    with pytest.raises(fm.FmError):
        ctx.surrogate_train_finish()   # nothing in flight
