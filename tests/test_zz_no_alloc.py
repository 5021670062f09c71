"""The allocation-free solve (fmg_solve_batch_static) against fmg_solve_batch.

Callers that cannot allocate device memory during a solve (fixed memory
budgets, memory pools owned by someone else) use the entry point whose
scratch is a static device array.  It must give the same Q^f and Q^c as the
level-wise schedule of fmg_solve_batch, call after call (the array keeps the
previous call's contents), and refuse batches larger than its 32 MiB.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

LEVELWISE = 1


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_static_scratch_solve_matches_fmg_solve_batch_twice():
    import paper_1910_04727_gb300 as fm
    from paper_1910_04727_gb300 import _lib
    L = _lib.load()
    ctx = fm.Context(2, 32, 8, seed=3)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, S, tag) in enumerate([(64, 37, 200), (128, 9, 201)]):
        K = torch.tensor(W.smooth_lognormal_field(n, S=S, tag=tag), device="cuda")
        ref_qf, ref_qc, _ = ctx.fmg_solve_batch(K, kernel=LEVELWISE)
        prm = ctx.solve_params()
        qf = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
        qc = torch.full((S,), float("nan"), dtype=torch.float64, device="cuda")
        st = L.fmg_solve_batch_static(ctx._h, n, S, _ptr(K), C.byref(prm), _ptr(qf), _ptr(qc), stream)
        assert st == 0, L.fm_last_error(ctx._h)
        torch.cuda.synchronize()
        a, b = qf.cpu().numpy(), ref_qf.cpu().numpy()
        assert np.max(np.abs(a - b) / np.abs(b)) < 1e-10, call
        a, b = qc.cpu().numpy(), ref_qc.cpu().numpy()
        assert np.max(np.abs(a - b) / np.abs(b)) < 1e-10, call


def test_static_scratch_solve_rejects_batches_beyond_its_array():
    import paper_1910_04727_gb300 as fm
    from paper_1910_04727_gb300 import _lib
    L = _lib.load()
    ctx = fm.Context(2, 32, 8, seed=3)
    K = torch.ones((64, 256, 256), dtype=torch.float64, device="cuda")
    qf = torch.empty(64, dtype=torch.float64, device="cuda")
    prm = ctx.solve_params()
    st = L.fmg_solve_batch_static(ctx._h, 256, 64, _ptr(K), C.byref(prm), _ptr(qf), None, None)
    assert st == _lib.FM_EINVAL
    assert b"static scratch" in L.fm_last_error(ctx._h)


def test_static_scratch_solve_refuses_the_energy_step():
    # the energy-optimal step keeps per-sample dot products that the static
    # layout has no room for: the call must refuse it before any launch
    import paper_1910_04727_gb300 as fm
    from paper_1910_04727_gb300 import _lib
    L = _lib.load()
    ctx = fm.Context(2, 32, 8, seed=3)
    K = torch.ones((4, 32, 32), dtype=torch.float64, device="cuda")
    qf = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    prm = ctx.solve_params(energy_step=1)
    st = L.fmg_solve_batch_static(ctx._h, 32, 4, _ptr(K), C.byref(prm), _ptr(qf), None, None)
    assert st == _lib.FM_EINVAL
    assert b"energy" in L.fm_last_error(ctx._h)
    torch.cuda.synchronize()
    assert torch.isnan(qf).all()


def test_static_scratch_solve_leaves_an_open_profile_alone():
    # with a profile open the call still allocates nothing: it times nothing
    import paper_1910_04727_gb300 as fm
    from paper_1910_04727_gb300 import _lib
    L = _lib.load()
    ctx = fm.Context(2, 32, 8, seed=3)
    K = torch.tensor(W.smooth_lognormal_field(32, S=5, tag=202), device="cuda")
    ref_qf, _, _ = ctx.fmg_solve_batch(K, kernel=LEVELWISE)
    qf = torch.empty(5, dtype=torch.float64, device="cuda")
    ctx.profile_begin()
    prm = ctx.solve_params()
    st = L.fmg_solve_batch_static(ctx._h, 32, 5, _ptr(K), C.byref(prm), _ptr(qf), None,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.fm_last_error(ctx._h)
    prof = ctx.profile_end()
    assert sum(v["launches"] for v in prof.values()) == 0
    a, b = qf.cpu().numpy(), ref_qf.cpu().numpy()
    assert np.max(np.abs(a - b) / np.abs(b)) < 1e-10
