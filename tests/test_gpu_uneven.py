"""Uneven batches (groups of different grid sizes in one CUDA graph) and the
smoother autotuner, against per-group solves and the FP64 oracle.

In the graph every group runs the kernels fmg_solve_batch runs, in the same
order, and the converged stages loop on the device with the tests of the
host loop, so every per-sample result must equal the per-group call's bit
for bit; the oracle bars are those of the per-group parity tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kl as okl
from oracle import lib as OL

pytestmark = pytest.mark.gpu

GRIDS = [(16, 70), (32, 33), (64, 9), (128, 5), (256, 3)]


@pytest.fixture(scope="module")
def ctx():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(32, 24, 1.0, 0.3, q=24)
    c = fm.Context(3, 8, 24, sigma2=1.0, lam=0.3, seed=5)
    c.kl_basis_set(basis.B_ref)
    return c


def _fields(tag0):
    return [W.smooth_lognormal_field(n, S=S, tag=tag0 + n) for n, S in GRIDS]


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def _same(a, b):
    return np.array_equal(a.cpu().numpy(), b.cpu().numpy(), equal_nan=True)


def test_fixed_schedule_matches_groups_and_oracle(ctx):
    Ks = [torch.tensor(K, device="cuda") for K in _fields(300)]
    outs = ctx.solve_uneven(Ks)
    for (n, S), K, (qf, qc, _) in zip(GRIDS, Ks, outs):
        rf, rc, _ = ctx.fmg_solve_batch(K)
        assert _same(qf, rf) and _same(qc, rc), n
        of, oc, _, _ = OL.fmg_solve_batch(K.cpu().numpy(), OL.params())
        assert _rel(qf.cpu().numpy(), of) < 1e-10
        assert _rel(qc.cpu().numpy(), oc) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_converged_device_loops_match_host_loops(ctx, precision):
    """Refined stages loop on the device (conditional graph nodes) and reach
    the per-group results bit for bit; the mixed form stays within its bar."""
    Ks = [torch.tensor(K, device="cuda") for K in _fields(400)]
    kw = dict(precision=precision, converged=1, tol=1e-12, qtol=0.0, max_cycles=400)
    outs = ctx.solve_uneven(Ks, want_status=True, **kw)
    for (n, S), K, (qf, qc, st) in zip(GRIDS, Ks, outs):
        rf, rc, _, rs = ctx.fmg_solve_batch(K, want_status=True, **kw)
        assert _same(qf, rf) and _same(qc, rc), n
        assert int(st.abs().sum()) == 0 and int(rs.abs().sum()) == 0
    for (n, S), K, (qf, qc, _) in zip(GRIDS[:3], Ks, outs):
        of, oc, _, _ = OL.fmg_solve_batch(K.cpu().numpy(), OL.params(converged=True, tol=1e-13, max_cycles=300))
        bar = 1e-8 if precision else 10 * n * 1e-12
        assert _rel(qf.cpu().numpy(), of) < bar and _rel(qc.cpu().numpy(), oc) < bar


@pytest.mark.parametrize("precision", [0, 1])
def test_converged_solves_without_qc(ctx, precision):
    """Without Q^c a converged solve leaves its coarse stage unrefined: the
    graph and the per-group call agree bit for bit, Q^f stays within the
    tolerance's reach of the solve that refines both stages, and a kept
    graph of the same grids with Q^c is not reused for it."""
    Ks = [torch.tensor(K, device="cuda") for K in _fields(450)]
    kw = dict(precision=precision, converged=1, tol=1e-12, qtol=0.0, max_cycles=400)
    with_qc = ctx.solve_uneven(Ks, **kw)
    before = ctx.uneven_stats()
    outs = ctx.solve_uneven(Ks, want_qc=False, **kw)
    after = ctx.uneven_stats()
    assert after["instantiations"] - before["instantiations"] == 1
    for (n, S), K, (qf, qc, _), (wf, _, _) in zip(GRIDS, Ks, outs, with_qc):
        assert qc is None
        rf, rqc, _ = ctx.fmg_solve_batch(K, want_qc=False, **kw)
        assert rqc is None and _same(qf, rf), n
        assert _rel(qf.cpu().numpy(), wf.cpu().numpy()) < 10 * n * 1e-12, n


def test_device_loop_reports_non_convergence(ctx):
    Ks = [torch.tensor(W.smooth_lognormal_field(n, S=4, tag=500 + n), device="cuda") for n in (32, 128)]
    outs = ctx.solve_uneven(Ks, want_status=True, converged=1, tol=1e-15, qtol=0.0, max_cycles=1)
    for qf, qc, st in outs:
        assert np.all(st.cpu().numpy() == 4)   # FM_ENOTCONV, the loop stopped at its bound
        assert np.all(np.isfinite(qf.cpu().numpy()))


def test_graph_is_reused_across_calls_of_one_shape(ctx):
    before = ctx.uneven_stats()
    res = []
    for tag in (600, 700):
        Ks = [torch.tensor(K, device="cuda") for K in _fields(tag)]
        res.append((Ks, ctx.solve_uneven(Ks, converged=1, tol=1e-10, max_cycles=200)))
    after = ctx.uneven_stats()
    assert after["launches"] - before["launches"] == 2
    assert (after["instantiations"] - before["instantiations"]) + (after["updates"] - before["updates"]) == 2
    for Ks, outs in res:   # the second launch ran the second set of fields
        for K, (qf, _, _) in zip(Ks, outs):
            rf, _, _ = ctx.fmg_solve_batch(K, converged=1, tol=1e-10, max_cycles=200)
            assert _same(qf, rf)


def test_empty_groups_and_argument_errors(ctx):
    import paper_1910_04727_gb300 as fm
    K = torch.tensor(W.smooth_lognormal_field(32, S=3, tag=800), device="cuda")
    empty = torch.empty((0, 64, 64), dtype=torch.float64, device="cuda")
    outs = ctx.solve_uneven([K, empty])
    rf, _, _ = ctx.fmg_solve_batch(K)
    assert _same(outs[0][0], rf) and outs[1][0].numel() == 0
    with pytest.raises(fm.FmError):
        ctx.solve_uneven([torch.zeros((2, 24, 24), dtype=torch.float64, device="cuda")])   # not 4 * 2^m


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_shapes_keep_every_result(ctx, precision):
    """Every launch shape computes the same sweeps: results before and after
    tuning are identical, and the tuner reports a time for each grid."""
    import paper_1910_04727_gb300 as fm
    Ks = [torch.tensor(K, device="cuda") for K in _fields(900)]
    kw = dict(precision=precision, converged=1, tol=1e-11, max_cycles=300)
    before = [ctx.fmg_solve_batch(K, **kw)[0] for K in Ks]
    rep = ctx.autotune(precision=precision, nsweeps=2, n_min=8, n_max=256)
    assert [e["n"] for e in rep] == [8, 16, 32, 64, 128, 256]
    assert all(e["ms_best"] > 0 and e["ms_best"] <= e["ms_default"] * 1.0001 for e in rep)
    after = [ctx.fmg_solve_batch(K, **kw)[0] for K in Ks]
    uneven = ctx.solve_uneven(Ks, **kw)
    for b, a, (u, _, _) in zip(before, after, uneven):
        assert _same(a, b) and _same(u, b)


def test_tile_smoother_is_deterministic_across_runs(ctx):
    """Many tiles per sample (256 x 256 in 32 x 32 tiles) and a converged mixed
    solve: two runs agree bit for bit whatever order the CTAs ran in."""
    K = torch.tensor(W.smooth_lognormal_field(256, S=24, tag=950), device="cuda")
    kw = dict(precision=1, converged=1, tol=1e-12, max_cycles=400)
    a = ctx.fmg_solve_batch(K, **kw)
    b = ctx.fmg_solve_batch(K, **kw)
    assert _same(a[0], b[0]) and _same(a[1], b[1])


@pytest.mark.parametrize("qmc", [False, True])
def test_batched_estimate_matches_per_level_estimate(qmc):
    """Each round's solves of all levels as one uneven batch: the same
    samples, the same per-sample results, so the same schedule and estimate."""
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(128, 32, 1.0, 0.3, q=32)
    c = fm.Context(4, 16, 32, sigma2=1.0, lam=0.3, seed=41, precision=1, converged=1, tol=1e-10,
                   qtol=1e-9, max_cycles=200, n_shifts=8)
    c.kl_basis_set(basis.B_ref)
    kw = dict(qmc=qmc, n_pilot=64 if not qmc else 16)
    a = c.mlmc_estimate(3e-3, **kw)
    b = c.mlmc_estimate(3e-3, batched=True, **kw)
    assert list(a["N"]) == list(b["N"]) and a["rounds"] == b["rounds"]
    assert abs(a["estimate"] - b["estimate"]) <= 1e-14 * abs(a["estimate"])
    assert b["batched_seconds"] > 0


def test_batched_estimate_with_surrogate_level():
    import paper_1910_04727_gb300 as fm
    basis = okl.KLBasis(64, 128, 1.0, 0.3, q=32)
    c = fm.Context(3, 16, 128, sigma2=1.0, lam=0.3, seed=43, precision=1, converged=1, tol=1e-10,
                   qtol=1e-9, max_cycles=200)
    c.kl_basis_set(basis.B_ref)
    c.surrogate_train(n_train=4096, epochs=20, lr=3e-3, seed=3, batch=512)
    kw = dict(n_pilot=128, surrogate=True, surrogate_cost=0.02)
    a = c.mlmc_estimate(4e-3, **kw)
    b = c.mlmc_estimate(4e-3, batched=True, **kw)
    assert list(a["N"]) == list(b["N"]) and a["N_s"] == b["N_s"]
    assert abs(a["estimate"] - b["estimate"]) <= 1e-14 * abs(a["estimate"])


def test_full_size_uneven_batch_sampled_against_oracle():
    """The benchmark's uneven batch at its grids (64 x 64 .. 1024 x 1024) and
    solver settings (FP32 smoothing, FP64 refinement to 1e-12 or an outflux
    change of 1e-10), fewer samples: per-group results bit for bit, and the
    first sample of every grid against the converged FP64 oracle (the mixed
    bar, 1e-8)."""
    import paper_1910_04727_gb300 as fm
    c = fm.Context(5, 64, 16, sigma2=1.0, lam=0.3, seed=47, precision=1, converged=1, tol=1e-12, qtol=1e-10,
                   max_cycles=200)
    counts = [5, 4, 3, 2, 1]
    Kn = [W.smooth_lognormal_field(64 << l, S=cnt, tag=1000 + l) for l, cnt in enumerate(counts)]
    Ks = [torch.tensor(K, device="cuda") for K in Kn]
    outs = c.solve_uneven(Ks)
    for K, (qf, qc, _) in zip(Ks, outs):
        rf, rc, _ = c.fmg_solve_batch(K)
        assert _same(qf, rf) and _same(qc, rc)
    errs = []
    for K, (qf, qc, _) in zip(Kn, outs):
        of, oc, _, _ = OL.fmg_solve_batch(K[:1], OL.params(converged=True, tol=1e-14, max_cycles=400))
        errs.append((K.shape[-1], _rel(qf.cpu().numpy()[:1], of), _rel(qc.cpu().numpy()[:1], oc)))
    print("outflux error against the converged oracle:", errs)
    assert all(ef < 1e-8 and ec < 1e-8 for _, ef, ec in errs)


@pytest.mark.parametrize("precision", [0, 1])
def test_energy_step_in_the_graph_equals_per_group_solves(ctx, precision):
    """The energy-optimal correction step inside the captured graph (device
    refinement loops, level-wise branches for every group): the same results
    as per-group fmg_solve_batch calls, bit for bit, and within the bars of
    the stepped oracle."""
    Ks = [torch.tensor(W.smooth_lognormal_field(n, S=S, sigma=1.4, tag=950 + n), device="cuda")
          for n, S in [(32, 11), (64, 6), (128, 3)]]
    # FP64: the residual test alone at 1e-13 (the stopping rule of the FP64 bar);
    # mixed: the benchmark's rule
    rule = dict(tol=1e-13, qtol=0.0) if precision == 0 else dict(tol=1e-12, qtol=1e-10)
    kw = dict(precision=precision, converged=1, max_cycles=300, energy_step=1, **rule)
    outs = ctx.solve_uneven(Ks, **kw)
    for K, (qf, qc, _) in zip(Ks, outs):
        a, b, _ = ctx.fmg_solve_batch(K, **kw)
        assert _same(a, qf) and _same(b, qc)
        rf, rc, _, _ = OL.fmg_solve_batch(K.cpu().numpy(), OL.params(converged=True, tol=1e-13, max_cycles=300,
                                                                     energy_step=True))
        bar = 1e-10 if precision == 0 else 1e-8
        assert _rel(qf.cpu().numpy(), rf) < bar
        assert _rel(qc.cpu().numpy(), rc) < bar
