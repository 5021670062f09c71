"""GB300 full-multigrid multilevel (quasi-) Monte Carlo (arXiv 1910.04727).

A thin binding of the C ABI in include/fmgmlmc.h.  It only marshals
arguments: every step of the method runs in the library's CUDA kernels.
PyTorch provides device memory and the current stream.
"""
import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import FM_PREC_FP64, FM_PREC_MIXED, STATUS_NAMES

__all__ = ["Context", "FmError", "FM_PREC_FP64", "FM_PREC_MIXED", "load_library", "shard_range",
           "estimate_core", "allgather_over", "matern_covariance"]


class FmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


def load_library():
    return _lib.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def matern_covariance(d, nu, sigma2=1.0, lam=1.0):
    """The library's Matern covariance (fm_matern_covariance) at distances d (host)."""
    L = _lib.load()
    d = np.ascontiguousarray(d, dtype=np.float64)
    c = np.empty_like(d)
    st = L.fm_matern_covariance(nu, sigma2, lam, d.ctypes.data_as(C.c_void_p), d.size,
                                c.ctypes.data_as(C.c_void_p))
    if st != 0:
        raise FmError(st, "fm_matern_covariance")
    return c


def lattice_cbc(dim, m_min, m_max):
    """Generating vector of the embedded lattice sequence (fm_lattice_cbc, host)."""
    L = _lib.load()
    z = np.zeros(dim, np.uint32)
    st = L.fm_lattice_cbc(dim, m_min, m_max, z.ctypes.data_as(C.c_void_p))
    if st != 0:
        raise FmError(st, "fm_lattice_cbc")
    return z


def shard_range(first, n, rank, world):
    """(first, count) of rank `rank`'s contiguous share of samples first .. first+n-1."""
    L = _lib.load()
    a, b = C.c_uint64(), C.c_uint64()
    L.fm_shard_range(first, n, rank, world, C.byref(a), C.byref(b))
    return a.value, b.value


def allgather_over(group=None):
    """gather(local_bytes) -> bytes of every rank's buffer in rank order, over a
    torch.distributed group (gloo on the host, nccl through the GPU)."""
    import torch.distributed as dist

    def gather(data):
        world = dist.get_world_size(group)
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.frombuffer(bytearray(data), dtype=torch.uint8).to(dev)
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        return b"".join(p.cpu().numpy().tobytes() for p in parts)
    return gather


def _allgather_cb(gather):
    if gather is None:
        return _lib.ALLGATHER_FN()

    def cb(user, local, all_, nbytes):
        try:
            res = gather(C.string_at(local, nbytes))
            C.memmove(all_, res, len(res))
            return 0
        except Exception:
            return _lib.FM_EINVAL
    return _lib.ALLGATHER_FN(cb)


def estimate_core(cost, eps, enqueue, read, gather=None, qmc=False, n_shifts=0, n_pilot=1000,
                  max_rounds=100, rank=0, world=1, level0=0, adapt_from=None, alpha=0.0):
    """mlmc_estimate_core over Python callables: enqueue(ext_level, first, n, shift) queues
    samples on this rank; read() returns this rank's running sums as a sequence of
    FmLevelSums ([n_ext][R]); gather(bytes) -> bytes of all ranks (None for one rank).
    adapt_from = n: start with n extended levels and grow by the bias test."""
    L = _lib.load()
    n_ext = len(cost)
    costs = (C.c_double * n_ext)(*[float(c) for c in cost])
    opts = _lib.FmCoreOpts(n_ext, costs, eps, int(bool(qmc)), n_shifts, n_pilot, max_rounds, rank, world,
                           level0, int(adapt_from is not None), adapt_from or 0, alpha)

    def enq(user, e, first, n, shift):
        try:
            enqueue(int(e), int(first), int(n), int(shift))
            return 0
        except Exception:
            return _lib.FM_EINVAL

    def rd(user, local):
        try:
            sums = read()
            for i, v in enumerate(sums):
                local[i] = v
            return 0
        except Exception:
            return _lib.FM_EINVAL

    cb_e, cb_r, cb_g = _lib.ENQUEUE_FN(enq), _lib.READ_FN(rd), _allgather_cb(gather)
    res = _lib.FmCoreResult()
    err = C.create_string_buffer(512)
    st = L.mlmc_estimate_core(C.byref(opts), cb_e, cb_r, cb_g, None, C.byref(res), err, 512)
    if st != 0:
        raise FmError(st, err.value.decode())
    E = res.n_ext_used
    return dict(estimate=res.estimate, var_estimator=res.var_estimator, means=np.array(res.mean[:E]),
                V=np.array(res.var[:E]), N=np.array(res.N[:E]), rounds=res.rounds, n_ext_used=E,
                bias=res.bias, alpha_used=res.alpha_used, bias_ok=bool(res.bias_ok))


class Context:
    """One fm_ctx: the problem (levels, field, boundary data) and the solver settings."""

    def __init__(self, n_levels, n_level0, M, sigma2=1.0, lam=0.3, pW=1.0, pE=0.0, nu0=2, nu1=2,
                 nu2=2, n_coarsest=4, n_shifts=16, seed=1910047270, max_batch=0,
                 precision=FM_PREC_FP64, converged=False, tol=1e-10, qtol=0.0, max_cycles=100,
                 kl_mode=0, bc_case=_lib.FM_CASE_II, pS=0.0, pN=0.0, nu=0.5, qmc_rule=0, lattice_m=0,
                 ir_cycles=0, energy_step=False):
        """bc_case: Table 1's FM_CASE_II (no flow north / south, east outflux) or
        FM_CASE_I (Dirichlet pW, pE, pS, pN on all four edges, QoI u(0.5, 0.5)).
        nu: Matern smoothness of the field (0.5, 1, 1.5 or 2.5).
        qmc_rule: FM_QMC_SOBOL_SHIFT, FM_QMC_SOBOL_OWEN or FM_QMC_LATTICE (2^lattice_m points).
        ir_cycles: V-cycles between residual tests of converged stages (0: nu0).
        energy_step: the energy-optimal coarse-grid correction step in every solve."""
        self._L = _lib.load()
        cfg = _lib.FmConfig(n_levels, n_level0, n_coarsest, M, sigma2, lam, pW, pE, nu0, nu1, nu2,
                            precision, int(bool(converged)), tol, qtol, max_cycles, kl_mode, n_shifts,
                            seed, max_batch, bc_case, pS, pN, nu, qmc_rule, lattice_m, ir_cycles,
                            int(bool(energy_step)))
        h = C.c_void_p()
        st = self._L.fm_create(C.byref(cfg), C.byref(h))
        if st != 0:
            raise FmError(st, self._L.fm_last_error(None).decode())
        self._h = h
        self.cfg = cfg
        self.levels = [n_level0 << l for l in range(n_levels)]
        self.M = M

    def _check(self, st):
        if st != 0:
            raise FmError(st, self._L.fm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.fm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------- points
    def mc_points(self, level, first, n, dim=None, out=None):
        dim = dim or self.M
        out = out if out is not None else torch.empty((n, dim), dtype=torch.float64, device="cuda")
        self._check(self._L.mc_points(self._h, level, first, n, dim, _ptr(out), _stream()))
        return out

    def mc_words(self, level, first, n, dim=None):
        """The raw 64-bit Philox words behind mc_points, [n][dim] (int64 bit patterns)."""
        dim = dim or self.M
        out = torch.empty((n, dim), dtype=torch.int64, device="cuda")
        self._check(self._L.mc_words(self._h, level, first, n, dim, _ptr(out), _stream()))
        return out

    def sobol_points(self, level, first, n, first_shift=0, n_shifts=1, dim=None, want_x=True,
                     want_xi=True):
        dim = dim or self.M
        x = torch.empty((n_shifts, n, dim), dtype=torch.int32, device="cuda") if want_x else None
        xi = torch.empty((n_shifts, n, dim), dtype=torch.float64, device="cuda") if want_xi else None
        self._check(self._L.sobol_points(self._h, level, dim, first, n, first_shift, n_shifts,
                                         _ptr(x), _ptr(xi), _stream()))
        return x, xi

    def qmc_points(self, rule, level, first, n, first_shift=0, n_shifts=1, dim=None, want_x=True,
                   want_xi=True):
        """Randomized QMC points of an FM_QMC_* rule: (x uint32 bits as int32, xi) [n_shifts][n][dim]."""
        dim = dim or self.M
        x = torch.empty((n_shifts, n, dim), dtype=torch.int32, device="cuda") if want_x else None
        xi = torch.empty((n_shifts, n, dim), dtype=torch.float64, device="cuda") if want_xi else None
        self._check(self._L.qmc_points(self._h, rule, level, dim, first, n, first_shift, n_shifts,
                                       _ptr(x), _ptr(xi), _stream()))
        return x, xi

    def lattice_generating_vector(self):
        z = np.zeros(self.M, np.uint32)
        self._check(self._L.lattice_generating_vector(self._h, z.ctypes.data_as(C.c_void_p)))
        return z

    def sobol_direction_numbers(self):
        V = np.zeros((self.M, 32), np.uint32)
        self._check(self._L.sobol_direction_numbers(self._h, V.ctypes.data_as(C.c_void_p)))
        return V

    # ----------------------------------------------------------- KL field
    def kl_basis_set(self, B_ref):
        """B_ref: [n_ref^2][M] float64 (numpy array or CUDA tensor)."""
        if isinstance(B_ref, torch.Tensor):
            t = B_ref.to(device="cuda", dtype=torch.float64).contiguous()
            self._check(self._L.kl_basis_set(self._h, _ptr(t), 1))
            torch.cuda.synchronize()
        else:
            a = np.ascontiguousarray(B_ref, dtype=np.float64)
            self._check(self._L.kl_basis_set(self._h, a.ctypes.data_as(C.c_void_p), 0))

    def kl_basis_build(self, q=0, interp=0):
        """Nystrom KL basis on the GPU; interp: 0 auto, 1 FP64, 2 tensor cores (BF16x3)."""
        theta = np.zeros(self.M)
        cap = C.c_double()
        self._check(self._L.kl_basis_build_ex(self._h, q, interp, theta.ctypes.data_as(C.c_void_p),
                                              C.byref(cap)))
        return theta, cap.value

    def sync(self):
        """Synchronise and raise on device-side failures of earlier calls."""
        self._check(self._L.fm_sync(self._h))

    def kl_basis_get(self, out=None):
        """The installed finest-grid basis [n_ref^2][M] (CUDA tensor, or into a
        given CPU/CUDA float64 tensor)."""
        n = self.levels[-1]
        if out is None:
            out = torch.empty((n * n, self.M), dtype=torch.float64, device="cuda")
        on_dev = 1 if out.is_cuda else 0
        self._check(self._L.kl_basis_get(self._h, C.c_void_p(out.data_ptr()), on_dev))
        return out

    def kl_basis_set_host_ptr(self, ptr):
        """Install a basis from host memory at address ptr (e.g. pinned)."""
        self._check(self._L.kl_basis_set(self._h, C.c_void_p(ptr), 0))

    def kl_field_batch(self, level, xi, out=None):
        n = xi.shape[0]
        N = self.levels[level]
        out = out if out is not None else torch.empty((n, N, N), dtype=torch.float64, device="cuda")
        self._check(self._L.kl_field_batch(self._h, level, n, _ptr(xi), _ptr(out), _stream()))
        return out

    # ----------------------------------------------------------- solver
    def solve_params(self, **over):
        c = self.cfg
        p = _lib.FmSolveParams(c.pW, c.pE, c.n_coarsest, c.nu0, c.nu1, c.nu2, c.precision,
                               _lib.FM_KERNEL_AUTO, c.converged, c.tol, c.qtol, c.max_cycles, c.energy_step,
                               c.bc_case, c.pS, c.pN, c.ir_cycles)
        for k, v in over.items():
            setattr(p, k, v)
        return p

    def fmg_solve_batch(self, K, want_qc=True, want_p=False, want_status=False, **params):
        """K: CUDA float64 [S][n][n]. Returns (qf, qc or None, p or None[, status])."""
        S, n = K.shape[0], K.shape[-1]
        prm = self.solve_params(**params)
        qf = torch.empty(S, dtype=torch.float64, device="cuda")
        qc = torch.empty(S, dtype=torch.float64, device="cuda") if want_qc else None
        p = torch.empty((S, n, n), dtype=torch.float64, device="cuda") if want_p else None
        st = torch.empty(S, dtype=torch.int32, device="cuda") if want_status else None
        self._check(self._L.fmg_solve_batch(self._h, n, S, _ptr(K), C.byref(prm), _ptr(qf), _ptr(qc),
                                            _ptr(p), _ptr(st), _stream()))
        return (qf, qc, p, st) if want_status else (qf, qc, p)

    def solve_uneven(self, Ks, want_qc=True, want_status=False, **params):
        """One CUDA graph over groups of different grid sizes: Ks is a list of CUDA
        float64 tensors [count][n][n].  Returns [(qf, qc, status)] per group."""
        prm = self.solve_params(**params)
        groups = (_lib.FmBatchGroup * len(Ks))()
        outs = []
        for g, K in enumerate(Ks):
            S, n = K.shape[0], K.shape[1]
            qf = torch.empty(S, dtype=torch.float64, device="cuda")
            qc = torch.empty(S, dtype=torch.float64, device="cuda") if want_qc else None
            st = torch.zeros(S, dtype=torch.int32, device="cuda") if want_status else None
            groups[g] = _lib.FmBatchGroup(n, S, K.data_ptr(), qf.data_ptr(), qc.data_ptr() if want_qc else None,
                                          st.data_ptr() if want_status else None)
            outs.append((qf, qc, st))
        self._check(self._L.fmg_solve_uneven(self._h, len(Ks), groups, C.byref(prm), _stream()))
        return outs

    def uneven_stats(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.fmg_uneven_stats(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return dict(instantiations=a.value, updates=b.value, launches=c.value)

    def autotune(self, precision=None, nsweeps=None, n_min=8, n_max=None):
        """Times the smoother launch shapes per grid and keeps the fastest (fm_autotune)."""
        precision = self.cfg.precision if precision is None else precision
        nsweeps = self.cfg.nu1 if nsweeps is None else nsweeps
        n_max = n_max or self.levels[-1]
        out = (_lib.FmTuneEntry * 16)()
        cnt = C.c_int32()
        self._check(self._L.fm_autotune(self._h, precision, nsweeps, n_min, n_max, out, 16, C.byref(cnt)))
        return [{f: getattr(e, f) for f, _ in _lib.FmTuneEntry._fields_} for e in out[:cnt.value]]

    def set_vcycle_tail(self, n_max):
        """Level-wise V-cycles run the part below correction grids up to n_max as one resident
        launch (0: grid by grid); the results are the same either way."""
        self._check(self._L.fm_set_vcycle_tail(self._h, n_max))

    def set_smoother_shape(self, n, tile, threads=0, precision=None):
        """Smoother launch shape of grid n (fm_set_smoother_shape): tile 0 colour launches,
        -1 column strips, 8..64 tiles (threads 0 register-blocked, 128 / 256 staged),
        -2 back to the built-in default."""
        precision = self.cfg.precision if precision is None else precision
        self._check(self._L.fm_set_smoother_shape(self._h, precision, n, tile, threads))

    # ----------------------------------------------------------- MLMC
    @staticmethod
    def new_sums(count=1):
        return torch.zeros((count, 16), dtype=torch.float64, device="cuda")

    def mlmc_sample_level(self, level, first, n, shift=-1, sums=None, want_q=False):
        qf = torch.empty(n, dtype=torch.float64, device="cuda") if want_q else None
        qc = torch.empty(n, dtype=torch.float64, device="cuda") if want_q else None
        self._check(self._L.mlmc_sample_level(self._h, level, first, n, shift, _ptr(sums), _ptr(qf),
                                              _ptr(qc), _stream()))
        return qf, qc

    @staticmethod
    def read_sums(sums):
        """(mean, var, count, sum_qf, sum_qc) of one fm_level_sums row (fm_level_stats)."""
        L = _lib.load()
        raw = np.ascontiguousarray(sums.detach().cpu().numpy(), dtype=np.float64)
        cell = _lib.FmLevelSums.from_buffer_copy(raw.tobytes())
        st = _lib.FmLevelStat()
        rc = L.fm_level_stats(C.byref(cell), C.byref(st))
        if rc != 0:
            raise FmError(rc, "fm_level_stats")
        return st.mean, st.var, st.count, st.sum_qf, st.sum_qc

    # ----------------------------------------------------------- profiling
    def profile_begin(self, mask=0xFFFFFFFF):
        self._check(self._L.fm_profile_begin(self._h, mask))

    def profile_end(self):
        """{family name: dict(launches, ms, bytes, flops)} since profile_begin."""
        stats = (_lib.FmKernelStat * 32)()
        n = C.c_int32()
        self._check(self._L.fm_profile_end(self._h, stats, 32, C.byref(n)))
        out = {}
        for s in stats[:n.value]:
            out[self._L.fm_kernel_family_name(s.family).decode()] = dict(
                launches=s.launches, ms=s.ms, bytes=s.bytes, flops=s.flops, flops_fp64=s.flops_fp64)
        return out

    # ----------------------------------------------------------- surrogate
    def surrogate_param_count(self):
        return int(self._L.surrogate_param_count(self._h))

    def surrogate_get_params(self):
        p = np.zeros(self.surrogate_param_count(), np.float32)
        self._check(self._L.surrogate_params(self._h, p.ctypes.data_as(C.c_void_p), 0))
        return p

    def surrogate_set_params(self, params, mu=0.0, sd=1.0):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.surrogate_param_count()
        self._check(self._L.surrogate_params(self._h, p.ctypes.data_as(C.c_void_p), 1))
        self._check(self._L.surrogate_set_scale(self._h, mu, sd))

    def surrogate_loss_grad(self, xi, target):
        """xi: CUDA float64 [256][M]; target: CUDA float32 [256]. Returns (loss, grads)."""
        g = np.zeros(self.surrogate_param_count(), np.float32)
        loss = C.c_double()
        self._check(self._L.surrogate_loss_grad(self._h, _ptr(xi), _ptr(target),
                                                g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return loss.value, g

    def surrogate_train(self, n_train=20000, epochs=200, lr=1e-3, seed=7, batch=256, async_run=False,
                        target_tol=0.0):
        """async_run: return once the training steps are launched (the report's
        losses and fit are NaN until surrogate_train_finish).  target_tol > 0:
        tolerance of the training pairs' level-0 solves (else the context's)."""
        opts = _lib.FmTrainOpts(n_train, epochs, lr, seed, batch, int(bool(async_run)), float(target_tol))
        rep = _lib.FmTrainReport()
        self._check(self._L.surrogate_train(self._h, C.byref(opts), C.byref(rep)))
        return {f: getattr(rep, f) for f, _ in _lib.FmTrainReport._fields_}

    def surrogate_train_finish(self):
        rep = _lib.FmTrainReport()
        self._check(self._L.surrogate_train_finish(self._h, C.byref(rep)))
        return {f: getattr(rep, f) for f, _ in _lib.FmTrainReport._fields_}

    def surrogate_eval(self, xi):
        s = torch.empty(xi.shape[0], dtype=torch.float64, device="cuda")
        self._check(self._L.surrogate_eval(self._h, xi.shape[0], _ptr(xi), _ptr(s), _stream()))
        return s

    def surrogate_eval_mc(self, stream_level, first, n):
        """S for MC samples first..first+n-1 of a Philox stream, from the Philox words."""
        s = torch.empty(n, dtype=torch.float64, device="cuda")
        self._check(self._L.surrogate_eval_mc(self._h, stream_level, first, n, _ptr(s), _stream()))
        return s

    def surrogate_set_fused(self, on=True):
        self._check(self._L.surrogate_set_fused(self._h, int(bool(on))))

    def surrogate_enable(self, on=True):
        self._check(self._L.surrogate_enable(self._h, int(bool(on))))

    def mlmc_estimate(self, eps, qmc=False, n_pilot=1000, max_rounds=100, surrogate=False,
                      surrogate_cost=0.01, group=None, shard=None, batched=False, L_start=None, alpha=0.0):
        """With a torch.distributed `group` of several ranks (one context per rank, all
        with the same seed), or shard = (rank, world, gather) with gather(bytes) ->
        bytes of all ranks, every request is shared among the ranks and the level
        sums are exchanged once per round; all ranks return the same estimate.
        L_start: grow the finest level from L_start by the bias test (alpha > 0 fixes
        the weak rate, else it is fitted).  The library orders the estimate after
        earlier work of the legacy default stream; a surrogate training launched
        with async_run keeps running beside it."""
        opts = _lib.FmEstimateOpts(eps, int(bool(qmc)), n_pilot, max_rounds, int(bool(surrogate)),
                                   surrogate_cost, int(bool(batched)), int(L_start is not None),
                                   L_start or 0, alpha)
        res = _lib.FmResult()
        if group is not None:
            import torch.distributed as dist
            shard = (dist.get_rank(group), dist.get_world_size(group), allgather_over(group))
        if shard is None:
            self._check(self._L.mlmc_estimate(self._h, C.byref(opts), C.byref(res)))
        else:
            rank, world, gather = shard
            cb = _allgather_cb(gather)
            self._check(self._L.mlmc_estimate_sharded(self._h, C.byref(opts), rank, world, cb, None,
                                                      C.byref(res)))
        L = res.L + 1
        return dict(estimate=res.estimate, var_estimator=res.var_estimator, L=res.L, bias_ok=bool(res.bias_ok),
                    alpha_used=res.alpha_used,
                    means=np.array(res.mean[:L]), V=np.array(res.var[:L]),
                    N=np.array(res.N[:L]), alpha=res.alpha, beta=res.beta, bias=res.bias,
                    rounds=res.rounds, seconds=res.seconds, mean_s=res.mean_s, var_s=res.var_s,
                    N_s=res.N_s, level_seconds=np.array(res.level_seconds[:L]),
                    seconds_s=res.seconds_s, batched_seconds=res.batched_seconds)
