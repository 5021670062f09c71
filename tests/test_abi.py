"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/fmgmlmc.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmgmlmc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?!typedef\b)(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1910_04727_gb300 import build
    return build.build()


def test_header_declares_the_method_entry_points():
    names = declared_functions()
    for required in ("mlmc_sample_level", "fmg_solve_batch", "kl_field_batch", "sobol_points",
                     "mlmc_estimate", "fm_create", "fm_destroy", "fm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_export(lib_path):
    from paper_1910_04727_gb300 import _lib
    assert sorted(_lib.EXPORTS) == declared_functions()
    L = _lib.load(lib_path)
    for n in _lib.EXPORTS:
        assert getattr(L, n).argtypes is not None or n == "fm_destroy"


def test_create_rejects_bad_config_without_touching_the_gpu(lib_path):
    from paper_1910_04727_gb300 import _lib
    L = _lib.load(lib_path)
    cfg = _lib.FmConfig(0, 16, 4, 8, 1.0, 0.3, 1.0, 0.0, 2, 2, 2, 0, 0, 1, 0)   # n_levels = 0
    h = ctypes.c_void_p()
    assert L.fm_create(ctypes.byref(cfg), ctypes.byref(h)) == _lib.FM_EINVAL
    assert b"n_levels" in L.fm_last_error(None)
    cfg = _lib.FmConfig(2, 12, 4, 8, 1.0, 0.3, 1.0, 0.0, 2, 2, 2, 0, 0, 1, 0)    # 12 != 4*2^m
    assert L.fm_create(ctypes.byref(cfg), ctypes.byref(h)) == _lib.FM_EINVAL
    assert not h.value


def _dd(x):
    """(hi, lo) doubles with hi + lo = the rational x to about 2^-106 relative."""
    hi = float(x)
    return hi, float(x - __import__("fractions").Fraction(hi))


@pytest.mark.parametrize("mean,sd", [(1.0, 0.5), (1e4, 1e-3), (-3e6, 0.5), (0.0, 1e-9)])
def test_level_stats_from_exact_sums(lib_path, mean, sd):
    """fm_level_stats (host only) on level sums holding the exact sums of Y
    and Y^2 as (sum, compensation) pairs: mean and Bessel-corrected variance
    agree with exact rational arithmetic, even with mean^2 / var near 1e14,
    where S2 - S1^2/n in plain doubles keeps about two digits."""
    from fractions import Fraction
    import numpy as np
    from paper_1910_04727_gb300 import _lib
    L = _lib.load(lib_path)
    y = mean + sd * np.random.default_rng(3).standard_normal(1000)
    s1 = sum(Fraction(v) for v in y)
    s2 = sum(Fraction(v) * Fraction(v) for v in y)
    n = len(y)
    cell = _lib.FmLevelSums()
    cell.sum_y[0], cell.sum_y[1] = _dd(s1)
    cell.sum_y2[0], cell.sum_y2[1] = _dd(s2)
    cell.count = n
    st = _lib.FmLevelStat()
    assert L.fm_level_stats(ctypes.byref(cell), ctypes.byref(st)) == 0
    want_var = (s2 - s1 * s1 / n) / (n - 1)
    assert abs(st.mean - float(s1 / n)) <= 1e-15 * abs(float(s1 / n)) + 1e-300
    assert abs(Fraction(st.var) - want_var) <= Fraction(1, 10 ** 12) * want_var
    assert L.fm_level_stats(None, ctypes.byref(st)) == _lib.FM_EINVAL


@pytest.mark.parametrize("dim,m_min,m_max", [(8, 3, 7), (32, 4, 10), (128, 5, 10), (16, 5, 12)])
def test_fast_lattice_construction_equals_the_plain_one(lib_path, dim, m_min, m_max):
    """fm_lattice_cbc (host only: FFTs over the odd residues, the minimum
    confirmed on plain sums) gives the oracle's plain component-by-component
    vector bit for bit."""
    import numpy as np
    from oracle import lib as OL
    from paper_1910_04727_gb300 import _lib
    L = _lib.load(lib_path)
    z = np.zeros(dim, np.uint32)
    assert L.fm_lattice_cbc(dim, m_min, m_max, z.ctypes.data_as(ctypes.c_void_p)) == 0
    np.testing.assert_array_equal(z, OL.lattice_cbc(dim, m_min, m_max))
    assert L.fm_lattice_cbc(dim, 6, 5, z.ctypes.data_as(ctypes.c_void_p)) == _lib.FM_EINVAL
