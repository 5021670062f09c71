"""Failure detection on the device without a fault: a bounded wait that
nothing completes runs out, the kernel returns, and the host reads
FM_ETIMEOUT through fm_sync; the context keeps working afterwards."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def test_a_wait_that_nothing_completes_reports_a_timeout_and_the_context_survives():
    import paper_1910_04727_gb300 as fm
    from paper_1910_04727_gb300 import _lib
    L = _lib.load()
    ctx = fm.Context(1, 16, 8, seed=4)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    assert L.fm_wait_check(ctx._h, 20_000_000, stream) == 0       # 20 ms
    st = L.fm_sync(ctx._h)
    dt = time.perf_counter() - t0
    assert st == _lib.FM_ETIMEOUT, st
    assert b"ran out" in L.fm_last_error(ctx._h)
    assert 0.015 < dt < 5.0, dt
    # reported once; the context still solves
    assert L.fm_sync(ctx._h) == 0
    K = torch.tensor(W.smooth_lognormal_field(16, S=8, tag=300), device="cuda")
    qf, _, _ = ctx.fmg_solve_batch(K)
    ctx.sync()
    assert np.all(np.isfinite(qf.cpu().numpy()))
    assert L.fm_wait_check(ctx._h, -1, stream) == _lib.FM_EINVAL
    ctx.close()
