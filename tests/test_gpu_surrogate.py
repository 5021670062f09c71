"""The surrogate control-variate level on the GPU against the FP64 oracle.

The oracle network rounds to BF16 where the tensor-core kernels hold BF16
operands, so the remaining differences are FP32 vs FP64 accumulation and
erff vs erf, plus the odd activation that lands on the other side of a BF16
rounding boundary: gradients agree to a few 1e-3 in norm per layer.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kl as okl
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

M = 128
DIMS = [(256, M), (256, 256), (256, 256), (1, 256)]


def _to_oracle(p):
    out, o = [], 0
    for r, c in DIMS:
        Wl = p[o:o + r * c].reshape(r, c).astype(np.float64)
        o += r * c
        bl = p[o:o + r].astype(np.float64)
        o += r
        out.append((Wl, bl))
    return out


def _flat(pairs):
    return np.concatenate([np.concatenate([Wl.ravel(), bl.ravel()]) for Wl, bl in pairs])


@pytest.fixture(scope="module")
def ctx():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(32, M, 1.0, 0.3, q=32)
    c = fm.Context(2, 16, M, sigma2=1.0, lam=0.3, seed=21)
    c.kl_basis_set(basis.B_ref)
    return c


def _random_params(seed):
    r = W.rng(tag=400 + seed)
    pairs = omlp.init_params(M, lambda n: r.uniform(size=n))
    return _flat(pairs).astype(np.float32)


def test_loss_and_gradients_match_oracle(ctx):
    p = _random_params(1)
    ctx.surrogate_set_params(p)
    xi = W.normals(256, M, tag=401)
    t = W.rng(tag=402).standard_normal(256).astype(np.float32)
    loss, g = ctx.surrogate_loss_grad(torch.tensor(xi, device="cuda"), torch.tensor(t, device="cuda"))
    params = _to_oracle(p)
    L, grads = omlp.mse_loss_and_grad(params, xi, t.astype(np.float64), rounding=True)
    assert abs(loss - L) < 1e-3 * L
    go = _flat(grads)
    o = 0
    for r, c in DIMS:
        for n in (r * c, r):
            a, b = g[o:o + n], go[o:o + n]
            assert np.linalg.norm(a - b) < 5e-3 * np.linalg.norm(b), (r, c, n)
            o += n


def test_eval_matches_oracle_forward(ctx):
    p = _random_params(2)
    ctx.surrogate_set_params(p, mu=1.1, sd=0.3)
    xi = W.normals(3000, M, tag=403)
    s = ctx.surrogate_eval(torch.tensor(xi, device="cuda")).cpu().numpy()
    out, _ = omlp.forward(_to_oracle(p), xi, rounding=True)
    ref = 1.1 + 0.3 * out
    assert np.max(np.abs(s - ref)) < 5e-3 * 0.3 * (1 + np.max(np.abs(out)))


def test_constant_surrogate_reduces_to_plain_level0(ctx):
    """S = c: the S level averages c exactly and level 0 averages Q_0 - c, so
    together they give the plain level-0 mean of the same samples."""
    p = np.zeros(ctx.surrogate_param_count(), np.float32)
    ctx.surrogate_set_params(p, mu=0.8125, sd=1.0)
    ctx.surrogate_enable(True)
    try:
        a, b = ctx.new_sums(), ctx.new_sums()
        ctx.mlmc_sample_level(-1, 0, 3000, -1, sums=a[0])
        ctx.mlmc_sample_level(0, 0, 700, -1, sums=b[0])
    finally:
        ctx.surrogate_enable(False)
    c = ctx.new_sums()
    ctx.mlmc_sample_level(0, 0, 700, -1, sums=c[0])
    torch.cuda.synchronize()
    ms = ctx.read_sums(a[0])[0]
    m0 = ctx.read_sums(b[0])[0]
    mp = ctx.read_sums(c[0])[0]
    assert ms == 0.8125
    assert abs(ms + m0 - mp) < 1e-13


def test_training_learns_the_level0_outflux(ctx):
    rep = ctx.surrogate_train(n_train=8192, epochs=25, lr=2e-3, seed=5)
    print("surrogate training:", rep)
    assert rep["loss_last"] < 0.5 * rep["loss_first"]
    assert rep["var_residual"] < 0.5 * rep["var_q"]
    assert rep["corr"] > 0.7


def test_loose_training_targets_give_the_same_network_quality(ctx):
    """target_tol: the training pairs' solves stop at a looser tolerance; the
    targets move by about that much, far below the network's own fit error,
    so the fit is as good and the standardisation nearly the same."""
    full = ctx.surrogate_train(n_train=8192, epochs=25, lr=2e-3, seed=5)
    loose = ctx.surrogate_train(n_train=8192, epochs=25, lr=2e-3, seed=5, target_tol=1e-6)
    assert abs(loose["mu"] - full["mu"]) < 1e-5 * abs(full["mu"])
    assert abs(loose["var_q"] - full["var_q"]) < 1e-4 * full["var_q"]
    assert abs(loose["corr"] - full["corr"]) < 2e-3
    assert abs(loose["var_residual"] - full["var_residual"]) < 0.05 * full["var_residual"]


def test_estimate_with_surrogate_agrees_with_plain_mlmc(ctx):
    if ctx.surrogate_param_count() <= 0:
        pytest.skip("no network")
    rep = ctx.surrogate_train(n_train=8192, epochs=25, lr=2e-3, seed=6)
    eps = 4e-3
    plain = ctx.mlmc_estimate(eps, n_pilot=256)
    sur = ctx.mlmc_estimate(eps, n_pilot=256, surrogate=True, surrogate_cost=0.01)
    print("plain", plain["estimate"], plain["N"], "surrogate", sur["estimate"], sur["N"], sur["N_s"])
    assert sur["var_estimator"] <= eps ** 2 / 2 * 1.01
    assert abs(sur["estimate"] - plain["estimate"]) < 3 * np.sqrt(sur["var_estimator"] + plain["var_estimator"])
    # the surrogate moves level-0 work onto cheap S samples
    assert sur["N"][0] < plain["N"][0]
    assert sur["N_s"] > sur["N"][0]


def test_philox_word_inputs_match_fp64_points(ctx):
    """The estimator evaluates S from the samples' Philox words (FP32 inverse
    normal, BF16 input); on the FP64 points of the same samples S differs only
    where the two inputs round to different BF16 values."""
    p = _random_params(3)
    ctx.surrogate_set_params(p, mu=0.5, sd=1.0)
    n = 20000
    a = ctx.surrogate_eval_mc(0, 1234, n).cpu().numpy()
    xi = ctx.mc_points(0, 1234, n)
    b = ctx.surrogate_eval(xi).cpu().numpy()
    d = np.abs(a - b)
    assert np.mean(d > 1e-6) < 0.05
    assert d.max() < 0.1
    # and the oracle network on the same FP64 points
    ref, _ = omlp.forward(_to_oracle(p), xi.cpu().numpy(), rounding=True)
    assert np.median(np.abs(a - (0.5 + ref))) < 1e-5


def test_surrogate_level_is_unbiased_over_many_seeds():
    """E[S] + E[Q_0 - S] = E[Q_0] holds only if the S level and level 0 apply
    the same map from a sample to S.  For 24 seeds (each its own Philox
    streams and its own trained network) the control-variate estimate of
    E[Q_0] is compared with a plain level-0 mean on disjoint samples of the
    same seed: the z-scores must average to 0 within 3/sqrt(24) and none
    may exceed 4."""
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(32, M, 1.0, 0.3, q=32)
    z = []
    for seed in range(24):
        c = fm.Context(2, 16, M, sigma2=1.0, lam=0.3, seed=1000 + seed)
        c.kl_basis_set(basis.B_ref)
        c.surrogate_train(n_train=4096, epochs=8, lr=3e-3, seed=seed, batch=256)
        c.surrogate_enable(True)
        s_sums, r_sums, p_sums = c.new_sums(), c.new_sums(), c.new_sums()
        c.mlmc_sample_level(-1, 0, 1 << 18, -1, sums=s_sums[0])
        c.mlmc_sample_level(0, 0, 16384, -1, sums=r_sums[0])
        c.surrogate_enable(False)
        # plain level-0 samples with ids disjoint from the ones above
        c.mlmc_sample_level(0, 1 << 30, 16384, -1, sums=p_sums[0])
        torch.cuda.synchronize()
        ms, vs, ns = c.read_sums(s_sums[0])[:3]
        mr, vr, nr = c.read_sums(r_sums[0])[:3]
        mp, vp, npl = c.read_sums(p_sums[0])[:3]
        z.append(((ms + mr) - mp) / np.sqrt(vs / ns + vr / nr + vp / npl))
        c.close()
    z = np.array(z)
    print("z-scores:", np.round(z, 2))
    assert abs(z.mean()) < 3.0 / np.sqrt(len(z))
    assert np.max(np.abs(z)) < 4.0
