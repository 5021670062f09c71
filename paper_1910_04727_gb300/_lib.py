"""ctypes declarations of the C ABI in include/fmgmlmc.h.

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
import ctypes as C
import os

from .build import LIB_PATH

FM_OK, FM_EINVAL, FM_ENOMEM, FM_ECUDA, FM_ENOTCONV, FM_ETIMEOUT, FM_EUNSUPPORTED = range(7)
FM_MAX_LEVELS = 12
FM_PREC_FP64 = 0
FM_PREC_MIXED = 1
FM_KERNEL_AUTO, FM_KERNEL_LEVELWISE, FM_KERNEL_RESIDENT = 0, 1, 2
FM_KL_AUTO, FM_KL_FP64, FM_KL_BF16, FM_KL_BF16X3 = 0, 1, 2, 3
FM_CASE_I, FM_CASE_II = 1, 2
FM_QMC_SOBOL_SHIFT, FM_QMC_SOBOL_OWEN, FM_QMC_LATTICE = 0, 1, 2

STATUS_NAMES = {0: "FM_OK", 1: "FM_EINVAL", 2: "FM_ENOMEM", 3: "FM_ECUDA", 4: "FM_ENOTCONV",
                5: "FM_ETIMEOUT", 6: "FM_EUNSUPPORTED"}

# every entry point declared in include/fmgmlmc.h
EXPORTS = ["fm_create", "fm_destroy", "fm_last_error", "mc_points", "sobol_points",
           "sobol_direction_numbers", "kl_basis_set", "kl_basis_build", "kl_basis_get", "kl_field_batch",
           "fmg_solve_batch", "mlmc_sample_level", "mlmc_estimate", "fm_profile_begin",
           "fm_profile_end", "fm_kernel_family_name", "fm_sync", "fmg_solve_batch_static",
           "surrogate_param_count", "surrogate_params", "surrogate_set_scale", "surrogate_loss_grad",
           "surrogate_train", "surrogate_train_finish", "surrogate_set_fused", "surrogate_eval", "surrogate_enable", "surrogate_eval_mc", "fm_shard_range",
           "mlmc_estimate_core", "mlmc_estimate_sharded", "fm_autotune", "fmg_solve_uneven",
           "fmg_uneven_stats", "fm_set_smoother_shape", "mc_words", "fm_level_stats", "fm_wait_check", "fm_matern_covariance", "qmc_points",
           "fm_lattice_cbc", "lattice_generating_vector", "kl_basis_build_ex",
           "fm_set_vcycle_tail"]


class FmConfig(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_level0", C.c_int32), ("n_coarsest", C.c_int32),
                ("M", C.c_int32), ("sigma2", C.c_double), ("lambda_", C.c_double),
                ("pW", C.c_double), ("pE", C.c_double), ("nu0", C.c_int32), ("nu1", C.c_int32),
                ("nu2", C.c_int32), ("precision", C.c_int32), ("converged", C.c_int32),
                ("tol", C.c_double), ("qtol", C.c_double), ("max_cycles", C.c_int32),
                ("kl_mode", C.c_int32),
                ("n_shifts", C.c_int32), ("seed", C.c_uint64), ("max_batch", C.c_int64),
                ("bc_case", C.c_int32), ("pS", C.c_double), ("pN", C.c_double), ("nu", C.c_double),
                ("qmc_rule", C.c_int32), ("lattice_m", C.c_int32), ("ir_cycles", C.c_int32),
                ("energy_step", C.c_int32)]


class FmSolveParams(C.Structure):
    _fields_ = [("pW", C.c_double), ("pE", C.c_double), ("n_coarsest", C.c_int32),
                ("nu0", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("precision", C.c_int32), ("kernel", C.c_int32), ("converged", C.c_int32),
                ("tol", C.c_double), ("qtol", C.c_double), ("max_cycles", C.c_int32),
                ("energy_step", C.c_int32), ("bc_case", C.c_int32), ("pS", C.c_double), ("pN", C.c_double),
                ("ir_cycles", C.c_int32)]


class FmLevelSums(C.Structure):
    _fields_ = [("sum_y", C.c_double * 2), ("sum_y2", C.c_double * 2), ("sum_qf", C.c_double * 2),
                ("sum_qc", C.c_double * 2), ("count", C.c_double), ("pad", C.c_double * 7)]


class FmLevelStat(C.Structure):
    _fields_ = [("count", C.c_double), ("mean", C.c_double), ("var", C.c_double), ("sum_qf", C.c_double),
                ("sum_qc", C.c_double)]


class FmEstimateOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("qmc", C.c_int32), ("n_pilot", C.c_int64),
                ("max_rounds", C.c_int32), ("surrogate", C.c_int32), ("surrogate_cost", C.c_double),
                ("batched", C.c_int32), ("adapt_L", C.c_int32), ("L_start", C.c_int32), ("alpha", C.c_double)]


class FmKernelStat(C.Structure):
    _fields_ = [("family", C.c_int32), ("launches", C.c_int64), ("ms", C.c_double),
                ("bytes", C.c_double), ("flops", C.c_double), ("flops_fp64", C.c_double)]


class FmTrainOpts(C.Structure):
    _fields_ = [("n_train", C.c_int32), ("epochs", C.c_int32), ("lr", C.c_double), ("seed", C.c_uint64),
                ("batch", C.c_int32), ("async_run", C.c_int32), ("target_tol", C.c_double)]


class FmTrainReport(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("mu", C.c_double),
                ("sd", C.c_double), ("corr", C.c_double), ("var_q", C.c_double),
                ("var_residual", C.c_double), ("steps", C.c_int32), ("seconds", C.c_double)]


class FmResult(C.Structure):
    _fields_ = [("estimate", C.c_double), ("var_estimator", C.c_double),
                ("mean", C.c_double * FM_MAX_LEVELS), ("var", C.c_double * FM_MAX_LEVELS),
                ("N", C.c_int64 * FM_MAX_LEVELS), ("alpha", C.c_double), ("beta", C.c_double),
                ("bias", C.c_double), ("rounds", C.c_int32), ("seconds", C.c_double),
                ("mean_s", C.c_double), ("var_s", C.c_double), ("N_s", C.c_int64),
                ("level_seconds", C.c_double * FM_MAX_LEVELS), ("seconds_s", C.c_double),
                ("batched_seconds", C.c_double), ("L", C.c_int32), ("bias_ok", C.c_int32),
                ("alpha_used", C.c_double)]


class FmCoreOpts(C.Structure):
    _fields_ = [("n_ext", C.c_int32), ("cost", C.POINTER(C.c_double)), ("eps", C.c_double),
                ("qmc", C.c_int32), ("n_shifts", C.c_int32), ("n_pilot", C.c_int64),
                ("max_rounds", C.c_int32), ("rank", C.c_int32), ("world", C.c_int32),
                ("level0", C.c_int32), ("adapt", C.c_int32), ("n_ext_start", C.c_int32), ("alpha", C.c_double)]


class FmCoreResult(C.Structure):
    _fields_ = [("estimate", C.c_double), ("var_estimator", C.c_double),
                ("mean", C.c_double * (FM_MAX_LEVELS + 1)), ("var", C.c_double * (FM_MAX_LEVELS + 1)),
                ("N", C.c_int64 * (FM_MAX_LEVELS + 1)), ("rounds", C.c_int32), ("n_ext_used", C.c_int32),
                ("bias_ok", C.c_int32), ("bias", C.c_double), ("alpha_used", C.c_double)]


class FmTuneEntry(C.Structure):
    _fields_ = [("n", C.c_int32), ("tile", C.c_int32), ("threads", C.c_int32), ("ms_best", C.c_double),
                ("ms_default", C.c_double), ("samples", C.c_int64)]


class FmBatchGroup(C.Structure):
    _fields_ = [("n_fine", C.c_int32), ("count", C.c_uint32), ("d_K", C.c_void_p), ("d_qf", C.c_void_p),
                ("d_qc", C.c_void_p), ("d_status", C.c_void_p)]


ENQUEUE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int32, C.c_uint64, C.c_uint64, C.c_int32)
READ_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.POINTER(FmLevelSums))
ALLGATHER_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.POINTER(FmLevelSums), C.POINTER(FmLevelSums), C.c_size_t)

_lib = None


def load(path=None):
    """Load libfmgmlmc.so and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libfmgmlmc.so is not built (%s); run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    P, U32, U64, I32, I64, D = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_int64, C.c_double
    sig = {
        "fm_create": (I32, [C.POINTER(FmConfig), C.POINTER(P)]),
        "fm_destroy": (None, [P]),
        "fm_last_error": (C.c_char_p, [P]),
        "mc_points": (I32, [P, U32, U64, U32, U32, P, P]),
        "mc_words": (I32, [P, U32, U64, U32, U32, P, P]),
        "fm_level_stats": (I32, [P, C.POINTER(FmLevelStat)]),
        "sobol_points": (I32, [P, U32, U32, U64, U32, U32, U32, P, P, P]),
        "sobol_direction_numbers": (I32, [P, P]),
        "kl_basis_set": (I32, [P, P, I32]),
        "kl_basis_build": (I32, [P, I32, P, P]),
        "kl_basis_build_ex": (I32, [P, I32, I32, P, P]),
        "kl_basis_get": (I32, [P, P, I32]),
        "kl_field_batch": (I32, [P, I32, U32, P, P, P]),
        "fmg_solve_batch": (I32, [P, I32, U32, P, C.POINTER(FmSolveParams), P, P, P, P, P]),
        "mlmc_sample_level": (I32, [P, I32, U64, U32, I32, P, P, P, P]),
        "mlmc_estimate": (I32, [P, C.POINTER(FmEstimateOpts), C.POINTER(FmResult)]),
        "fm_profile_begin": (I32, [P, U32]),
        "fm_profile_end": (I32, [P, P, I32, C.POINTER(I32)]),
        "fm_kernel_family_name": (C.c_char_p, [I32]),
        "fm_sync": (I32, [P]),
        "fm_wait_check": (I32, [P, I64, P]),
        "fm_matern_covariance": (I32, [D, D, D, P, I64, P]),
        "qmc_points": (I32, [P, I32, U32, U32, U64, U32, U32, U32, P, P, P]),
        "fm_lattice_cbc": (I32, [U32, I32, I32, P]),
        "lattice_generating_vector": (I32, [P, P]),
        "fmg_solve_batch_static": (I32, [P, I32, U32, P, C.POINTER(FmSolveParams), P, P, P]),
        "surrogate_param_count": (I64, [P]),
        "surrogate_params": (I32, [P, P, I32]),
        "surrogate_set_scale": (I32, [P, D, D]),
        "surrogate_loss_grad": (I32, [P, P, P, P, P]),
        "surrogate_train": (I32, [P, C.POINTER(FmTrainOpts), C.POINTER(FmTrainReport)]),
        "surrogate_train_finish": (I32, [P, C.POINTER(FmTrainReport)]),
        "surrogate_set_fused": (I32, [P, I32]),
        "surrogate_eval": (I32, [P, U32, P, P, P]),
        "surrogate_enable": (I32, [P, I32]),
        "surrogate_eval_mc": (I32, [P, U32, U64, U32, P, P]),
        "fm_autotune": (I32, [P, I32, I32, I32, I32, P, I32, C.POINTER(I32)]),
        "fmg_solve_uneven": (I32, [P, I32, P, C.POINTER(FmSolveParams), P]),
        "fmg_uneven_stats": (I32, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
        "fm_set_smoother_shape": (I32, [P, I32, I32, I32, I32]),
        "fm_set_vcycle_tail": (I32, [P, I32]),
        "fm_shard_range": (None, [U64, U64, I32, I32, C.POINTER(U64), C.POINTER(U64)]),
        "mlmc_estimate_core": (I32, [C.POINTER(FmCoreOpts), ENQUEUE_FN, READ_FN, ALLGATHER_FN, P,
                                     C.POINTER(FmCoreResult), C.c_char_p, C.c_size_t]),
        "mlmc_estimate_sharded": (I32, [P, C.POINTER(FmEstimateOpts), I32, I32, ALLGATHER_FN, P,
                                        C.POINTER(FmResult)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L
