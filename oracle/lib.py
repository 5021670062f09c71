"""ctypes wrappers of the oracle's C functions (test infrastructure only).

Every wrapper takes and returns numpy arrays; all floating point is FP64.
"""
import ctypes as C

import numpy as np

from .build import build

_lib = None


class Params(C.Structure):
    """Solver parameters (mirrors ``or_params`` in fmg_oracle.c)."""
    _fields_ = [("pW", C.c_double), ("pE", C.c_double), ("nu0", C.c_int),
                ("nu1", C.c_int), ("nu2", C.c_int), ("converged", C.c_int),
                ("tol", C.c_double), ("max_cycles", C.c_int), ("coarse_op", C.c_int),
                ("energy_step", C.c_int), ("bc_case", C.c_int), ("pS", C.c_double), ("pN", C.c_double)]


def params(pW=1.0, pE=0.0, nu0=2, nu1=2, nu2=2, converged=False, tol=1e-12,
           max_cycles=100, coarse_op=1, energy_step=False, bc_case=2, pS=0.0, pN=0.0):
    """bc_case 2: Table 1 Case II (no flow north / south, outflux QoI);
    1: Case I (Dirichlet pS / pN on the south / north edges, QoI u(0.5, 0.5))."""
    return Params(pW, pE, nu0, nu1, nu2, int(bool(converged)), tol, max_cycles, coarse_op,
                  int(bool(energy_step)), bc_case, pS, pN)


def case1_params(**kw):
    """Table 1 Case I: u = 100 / 0 / 10 / 50 on the west / east / south / north edges."""
    kw.setdefault("pW", 100.0)
    kw.setdefault("pE", 0.0)
    kw.setdefault("pS", 10.0)
    kw.setdefault("pN", 50.0)
    return params(bc_case=1, **kw)


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.or_philox4x64_10.argtypes = [_U64, _U64, _U64]
        L.or_philox_word.argtypes = [C.c_uint64] * 4
        L.or_philox_word.restype = C.c_uint64
        L.or_norminv.argtypes = [C.c_double]
        L.or_norminv.restype = C.c_double
        L.or_mc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32,
                                    C.c_uint32, _D]
        L.or_mc_words.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32, _U64]
        L.or_lattice_cbc.argtypes = [C.c_uint32, C.c_int, C.c_int, _U32]
        L.or_lattice_e2.argtypes = [_U32, C.c_uint32, C.c_int]
        L.or_lattice_e2.restype = C.c_double
        L.or_lattice_points.argtypes = [_U32, C.c_uint32, C.c_int, C.c_uint64, C.c_uint32, C.c_uint64,
                                        C.c_uint32, C.c_uint32, C.c_uint32, _U32]
        L.or_owen_scramble.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.or_owen_scramble.restype = C.c_uint32
        L.or_sobol_owen_points.argtypes = [_U32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint32,
                                           C.c_uint32, C.c_uint32, _U32]
        L.or_gf2_is_primitive.argtypes = [C.c_uint64, C.c_int]
        L.or_primitive_polys.argtypes = [C.c_int, _U64, _I32]
        L.or_sobol_direction_numbers.argtypes = [C.c_uint32, _U32]
        L.or_sobol_shifts.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, _U32]
        L.or_sobol_points.argtypes = [_U32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_uint32,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_apply_A.argtypes = [C.c_int, _D, _D, _D]
        L.or_stage_rhs.argtypes = [C.c_int, _D, C.c_double, C.c_double, _D]
        L.or_rbgs_sweep.argtypes = [C.c_int, _D, _D, _D]
        L.or_residual.argtypes = [C.c_int, _D, _D, _D, _D]
        L.or_restrict_sum.argtypes = [C.c_int, _D, _D]
        L.or_prolong_add.argtypes = [C.c_int, _D, _D]
        L.or_fmg_interpolate.argtypes = [C.c_int, _D, C.c_double, C.c_double, _D]
        L.or_inject.argtypes = [C.c_int, _D, _D]
        L.or_geometric_children.argtypes = [C.c_int, _D, _D]
        L.or_exact_solve.argtypes = [C.c_int, _D, _D, _D]
        L.or_outflux.argtypes = [C.c_int, _D, _D, C.c_double]
        L.or_outflux.restype = C.c_double
        L.or_influx.argtypes = [C.c_int, _D, _D, C.c_double]
        L.or_influx.restype = C.c_double
        L.or_fmg_solve.argtypes = [C.c_int, C.c_int, _D, C.POINTER(Params), C.c_void_p,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_fmg_solve.restype = C.c_int
        L.or_vcycle_solve.argtypes = [C.c_int, C.c_int, _D, _D, _D, C.c_int, C.c_int,
                                      C.c_int, C.c_int, C.c_int, C.c_int, _D]
        L.or_apply_A_bc.argtypes = [C.c_int, _D, C.c_int, _D, _D]
        L.or_stage_rhs_bc.argtypes = [C.c_int, _D, _D, C.c_int, _D]
        L.or_prolong_add_bc.argtypes = [C.c_int, _D, C.c_int, _D]
        L.or_fmg_interpolate_bc.argtypes = [C.c_int, _D, _D, C.c_int, _D]
        L.or_exact_solve_bc.argtypes = [C.c_int, _D, C.c_int, _D, _D]
        L.or_centre_value.argtypes = [C.c_int, _D]
        L.or_centre_value.restype = C.c_double
        L.or_fmg_solve_batch.argtypes = [C.c_int, C.c_int, C.c_int, _D, C.POINTER(Params),
                                         C.c_void_p, _D, _D, C.c_int]
        L.or_fmg_solve_batch.restype = C.c_int
        _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- points
def philox4x64_10(ctr, key):
    out = np.zeros(4, np.uint64)
    lib().or_philox4x64_10(_c(ctr, np.uint64), _c(key, np.uint64), out)
    return out


def philox_word(key0, key1, index, w):
    return int(lib().or_philox_word(key0, key1, index, w))


def norminv(u):
    f = lib().or_norminv
    return np.array([f(float(x)) for x in np.ravel(u)]).reshape(np.shape(u))


def mc_normals(seed, level, first, n, dim):
    xi = np.zeros((n, dim))
    lib().or_mc_normals(seed, level, first, n, dim, xi)
    return xi


def mc_words(seed, level, first, n, dim):
    """The 64-bit Philox words behind mc_normals, [n][dim] uint64."""
    w = np.zeros((n, dim), np.uint64)
    lib().or_mc_words(seed, level, first, n, dim, w)
    return w


def lattice_cbc(dim, m_min, m_max):
    """Generating vector of the embedded lattice sequence (component by component)."""
    z = np.zeros(dim, np.uint32)
    assert lib().or_lattice_cbc(dim, m_min, m_max, z) == 0
    return z


def lattice_e2(z, m):
    """Shift-averaged squared worst-case error of the 2^m-point lattice."""
    z = np.ascontiguousarray(z, np.uint32)
    return lib().or_lattice_e2(z, len(z), m)


def lattice_points(z, m_max, seed, level, first, n, first_shift=0, n_shifts=1):
    """Randomly shifted lattice sequence, uint32 [n_shifts][n][dim]."""
    z = np.ascontiguousarray(z, np.uint32)
    x = np.zeros((n_shifts, n, len(z)), np.uint32)
    lib().or_lattice_points(z, len(z), m_max, seed, level, first, n, first_shift, n_shifts, x)
    return x


def owen_scramble(seed, level, r, d, x):
    return np.array([lib().or_owen_scramble(seed, level, r, d, int(v)) for v in np.ravel(x)],
                    np.uint32).reshape(np.shape(x))


def sobol_owen_points(V, seed, level, first, n, first_shift=0, n_shifts=1):
    """Owen-scrambled Sobol' points, uint32 [n_shifts][n][dim]."""
    V = np.ascontiguousarray(V, np.uint32)
    dim = V.shape[0]
    x = np.zeros((n_shifts, n, dim), np.uint32)
    lib().or_sobol_owen_points(V, dim, seed, level, first, n, first_shift, n_shifts, x)
    return x


def primitive_polys(count):
    p = np.zeros(count, np.uint64)
    d = np.zeros(count, np.int32)
    got = lib().or_primitive_polys(count, p, d)
    return p[:got], d[:got]


def is_primitive(p, deg):
    return bool(lib().or_gf2_is_primitive(p, deg))


def sobol_direction_numbers(dim):
    V = np.zeros((dim, 32), np.uint32)
    if lib().or_sobol_direction_numbers(dim, V) != 0:
        raise ValueError("not enough primitive polynomials")
    return V


def sobol_shifts(seed, level, n_shifts, dim):
    s = np.zeros((n_shifts, dim), np.uint32)
    lib().or_sobol_shifts(seed, level, n_shifts, dim, s)
    return s


def sobol_points(V, first, n, shifts=None, want_xi=False):
    """Returns (x uint32 [R][n][dim], xi float64 or None)."""
    V = _c(V, np.uint32)
    dim = V.shape[0]
    R = 1 if shifts is None else shifts.shape[0]
    out = np.zeros((R, n, dim), np.uint32)
    xi = np.zeros((R, n, dim)) if want_xi else None
    sh = None if shifts is None else _c(shifts, np.uint32)
    lib().or_sobol_points(V, dim, first, n, R,
                          None if sh is None else sh.ctypes.data,
                          out.ctypes.data, None if xi is None else xi.ctypes.data)
    return out, xi


# ----------------------------------------------------------------- solver
def apply_A(K, x):
    n = K.shape[0]
    y = np.zeros((n, n))
    lib().or_apply_A(n, _c(K), _c(x), y)
    return y


def stage_rhs(K, pW=1.0, pE=0.0):
    n = K.shape[0]
    b = np.zeros((n, n))
    lib().or_stage_rhs(n, _c(K), pW, pE, b)
    return b


def rbgs_sweep(K, b, x):
    x = _c(x).copy()
    lib().or_rbgs_sweep(K.shape[0], _c(K), _c(b), x)
    return x


def residual(K, b, x):
    r = np.zeros_like(_c(x))
    lib().or_residual(K.shape[0], _c(K), _c(b), _c(x), r)
    return r


def restrict_sum(rf):
    nc = rf.shape[0] // 2
    bc = np.zeros((nc, nc))
    lib().or_restrict_sum(nc, _c(rf), bc)
    return bc


def prolong_add(ec, xf):
    xf = _c(xf).copy()
    lib().or_prolong_add(ec.shape[0], _c(ec), xf)
    return xf


def fmg_interpolate(uc, pW=1.0, pE=0.0):
    nc = uc.shape[0]
    xf = np.zeros((2 * nc, 2 * nc))
    lib().or_fmg_interpolate(nc, _c(uc), pW, pE, xf)
    return xf


def inject(Kf):
    nc = Kf.shape[0] // 2
    Kc = np.zeros((nc, nc))
    lib().or_inject(nc, _c(Kf), Kc)
    return Kc


def geometric_children(Kf):
    """Coefficients of a correction grid: the geometric mean of each coarse
    cell's four children on the finer grid Kf."""
    nc = Kf.shape[0] // 2
    Kc = np.zeros((nc, nc))
    lib().or_geometric_children(nc, _c(Kf), Kc)
    return Kc


def exact_solve(K, b):
    x = np.zeros_like(_c(b))
    lib().or_exact_solve(K.shape[0], _c(K), _c(b), x)
    return x


def outflux(K, x, pE=0.0):
    return lib().or_outflux(K.shape[0], _c(K), _c(x), pE)


def influx(K, x, pW=1.0):
    return lib().or_influx(K.shape[0], _c(K), _c(x), pW)


def fmg_solve(K, prm=None, n0=4, want_p=False):
    """One FMG solve. Returns (qf, qc, p or None, cycles)."""
    prm = prm or params()
    K = _c(K)
    n = K.shape[0]
    p = np.zeros((n, n)) if want_p else None
    qf, qc = C.c_double(), C.c_double()
    cyc = lib().or_fmg_solve(n, n0, K, C.byref(prm),
                             None if p is None else p.ctypes.data,
                             C.byref(qf), C.byref(qc))
    return qf.value, qc.value, p, cyc


def vcycle_solve(K, b, x0, nu1=2, nu2=2, ncycles=10, n0=4, coarse_op=1, energy_step=False, ns=0):
    """V-cycles on A x = b (ns = 1: Dirichlet north / south edges, Case I);
    returns (x, residual norms before/after each cycle)."""
    x = _c(x0).copy()
    hist = np.zeros(ncycles + 1)
    lib().or_vcycle_solve(K.shape[0], n0, _c(K), _c(b), x, nu1, nu2, ncycles, coarse_op,
                          int(bool(energy_step)), int(ns), hist)
    return x, hist


# ----------------------------------------------------------------- Case I (all-Dirichlet)
def apply_A_bc(K, x, ns):
    y = np.zeros_like(_c(x))
    lib().or_apply_A_bc(K.shape[0], _c(K), int(ns), _c(x), y)
    return y


def stage_rhs_bc(K, g, ns):
    """g = (west, east, south, north) boundary values."""
    b = np.zeros_like(_c(K))
    lib().or_stage_rhs_bc(K.shape[0], _c(K), _c(g), int(ns), b)
    return b


def prolong_add_bc(ec, xf, ns):
    xf = _c(xf).copy()
    lib().or_prolong_add_bc(ec.shape[0], _c(ec), int(ns), xf)
    return xf


def fmg_interpolate_bc(uc, g, ns):
    nc = uc.shape[0]
    xf = np.zeros((2 * nc, 2 * nc))
    lib().or_fmg_interpolate_bc(nc, _c(uc), _c(g), int(ns), xf)
    return xf


def exact_solve_bc(K, b, ns):
    x = np.zeros_like(_c(b))
    lib().or_exact_solve_bc(K.shape[0], _c(K), int(ns), _c(b), x)
    return x


def centre_value(x):
    return lib().or_centre_value(x.shape[0], _c(x))


def fmg_solve_batch(K, prm=None, n0=4, want_p=False, nthreads=0):
    """Batch of FMG solves, K [S][n][n]. Returns (qf [S], qc [S], p or None, threads)."""
    prm = prm or params()
    K = _c(K)
    S, n = K.shape[0], K.shape[1]
    qf, qc = np.zeros(S), np.zeros(S)
    p = np.zeros((S, n, n)) if want_p else None
    used = lib().or_fmg_solve_batch(n, n0, S, K, C.byref(prm),
                                    None if p is None else p.ctypes.data, qf, qc,
                                    nthreads)
    return qf, qc, p, used
