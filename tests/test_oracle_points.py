"""Pins of the oracle's point generators (Sec. 2.3 MC points, Sec. 2.4 / 3.1
randomized Sobol' points) against things other than the oracle itself."""
import math

import numpy as np
import pytest
import scipy.special
import scipy.stats

from oracle import lib as L


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((5, 7, 9, 11), (0x1234, 0xABCDEF)),
    ((2 ** 64 - 1, 3, 0, 0), (1, 2)),
    ((123456789, 2 ** 63 + 5, 77, 2 ** 64 - 2), (2 ** 64 - 1, 2 ** 40 + 3)),
])
def test_philox_matches_numpy_philox4x64_10(ctr, key):
    """numpy.random.Philox is Philox4x64-10; it bumps its counter by one
    before each block, so block `ctr` is numpy's first block at ctr - 1."""
    mine = L.philox4x64_10(np.array(ctr, np.uint64), np.array(key, np.uint64))
    v = sum(int(c) << (64 * i) for i, c in enumerate(ctr)) - 1
    prev = np.array([(v >> (64 * i)) & (2 ** 64 - 1) for i in range(4)], np.uint64)
    ref = np.random.Philox(counter=prev, key=np.array(key, np.uint64)).random_raw(4)
    assert [int(x) for x in mine] == [int(x) for x in ref]


def test_mc_uniforms_chi_square():
    words = np.array([L.philox_word(7, 1 << 32, s, k) for s in range(2048) for k in range(16)],
                     dtype=np.uint64)
    u = ((words >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    counts = np.histogram(u, bins=1024, range=(0, 1))[0]
    p = scipy.stats.chisquare(counts).pvalue
    assert 1e-4 < p


def test_mc_normals_moments_and_streams():
    xi = L.mc_normals(11, 0, 0, 4000, 8)
    assert abs(xi.mean()) < 0.05 and abs(xi.var() - 1) < 0.05
    # a different level is a different stream; a later first index continues it
    other = L.mc_normals(11, 1, 0, 10, 8)
    assert not np.allclose(other, xi[:10])
    np.testing.assert_array_equal(L.mc_normals(11, 0, 100, 5, 8), xi[100:105])


# ---------------------------------------------------------------- Phi^-1
def test_norminv_against_scipy_ndtri():
    u = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 2001), 2.0 ** -np.arange(2, 53),
                        1 - 2.0 ** -np.arange(2, 53)])
    mine = L.norminv(u)
    ref = scipy.special.ndtri(u)
    # a few ulp of the result, plus the conditioning of solving Phi(x) = u
    # with Phi rounded to ~ulp(u): dx = du / phi(x)
    pdf = np.exp(-0.5 * ref * ref) / np.sqrt(2 * np.pi)
    tol = 8 * np.spacing(np.abs(ref)) + 4 * np.spacing(np.minimum(u, 1 - u) + 0.0) / pdf \
        + 4 * np.spacing(np.maximum(u, 0.5)) * (np.abs(u - 0.5) < 0.25) / pdf
    bad = np.abs(mine - ref) > tol
    assert not bad.any(), (u[bad], mine[bad], ref[bad])


def test_norminv_symmetry_and_roundtrip():
    u = (np.arange(1, 4096) + 0.5) / 8192.0
    a, b = L.norminv(u), L.norminv(1 - u)
    np.testing.assert_array_equal(a, -b)
    np.testing.assert_allclose(scipy.special.ndtr(a), u, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- Sobol'
def _totient(n):
    result, m, q = n, n, 2
    while q * q <= m:
        if m % q == 0:
            while m % q == 0:
                m //= q
            result -= result // q
        q += 1
    if m > 1:
        result -= result // m
    return result


def test_primitive_polynomial_counts_closed_form():
    """There are phi(2^d - 1)/d primitive polynomials of degree d over GF(2)."""
    polys, degs = L.primitive_polys(1200)
    for d in range(1, 12):
        assert int(np.sum(degs == d)) == _totient(2 ** d - 1) // d


def test_primitive_vs_irreducible_not_primitive():
    # x^4+x+1 is primitive; x^4+x^3+x^2+x+1 is irreducible of order 5 only;
    # x^4+x^2+1 = (x^2+x+1)^2 is reducible
    assert L.is_primitive(0b10011, 4)
    assert not L.is_primitive(0b11111, 4)
    assert not L.is_primitive(0b10101, 4)
    assert L.is_primitive(0b11, 1) and L.is_primitive(0b111, 2)


def test_second_dimension_is_pascal_triangle_mod2():
    """With x + 1 the recurrence gives m_k = m_(k-1) XOR 2 m_(k-1), m_1 = 1:
    the bits of m_k are row k-1 of Pascal's triangle mod 2."""
    V = L.sobol_direction_numbers(2)
    for k in range(1, 33):
        m = int(V[1, k - 1]) >> (32 - k)
        expect = sum((math.comb(k - 1, i) % 2) << i for i in range(k))
        assert m == expect


def test_direction_numbers_valid():
    V = L.sobol_direction_numbers(300)
    for d in range(300):
        for k in range(1, 33):
            m = int(V[d, k - 1]) >> (32 - k)
            assert m % 2 == 1 and m < 2 ** k
            assert (int(V[d, k - 1]) & ((1 << (32 - k)) - 1)) == 0


def test_van_der_corput_first_points():
    V = L.sobol_direction_numbers(1)
    x, _ = L.sobol_points(V, 0, 4)
    # Gray-code order: 0, 1/2, 3/4, 1/4
    assert [int(v) for v in x[0, :, 0]] == [0, 2 ** 31, 3 * 2 ** 30, 2 ** 30]


@pytest.mark.parametrize("shifted", [False, True])
def test_one_dimensional_nets(shifted):
    """The first 2^m points of every coordinate are one point per interval of
    length 2^-m; a digital shift permutes those intervals."""
    dim = 128
    V = L.sobol_direction_numbers(dim)
    sh = L.sobol_shifts(5, 0, 1, dim) if shifted else None
    x, _ = L.sobol_points(V, 0, 4096, sh)
    for m in (1, 4, 8, 12):
        top = x[0, : 2 ** m, :] >> np.uint32(32 - m)
        for d in range(dim):
            assert len(np.unique(top[:, d])) == 2 ** m


def test_first_two_dimensions_form_a_02_net():
    V = L.sobol_direction_numbers(2)
    m = 8
    x, _ = L.sobol_points(V, 0, 2 ** m)
    pts = x[0]
    for a in range(m + 1):
        cx = pts[:, 0].astype(np.uint64) >> np.uint64(32 - a) if a else np.zeros(2 ** m, np.uint64)
        b = m - a
        cy = pts[:, 1].astype(np.uint64) >> np.uint64(32 - b) if b else np.zeros(2 ** m, np.uint64)
        boxes = cx * np.uint64(2 ** 20) + cy
        assert len(np.unique(boxes)) == 2 ** m


def test_gray_code_recurrence_equals_direct_index():
    """Antonov-Saleev: x_(n+1) = x_n XOR V[c], c = index of the lowest zero bit of n."""
    dim = 16
    V = L.sobol_direction_numbers(dim)
    x, _ = L.sobol_points(V, 0, 1000)
    cur = np.zeros(dim, np.uint32)
    for n in range(999):
        c = (~n & (n + 1)).bit_length() - 1
        cur = cur ^ V[:, c]
        np.testing.assert_array_equal(cur, x[0, n + 1])


def test_sobol_xi_is_norminv_of_midpoint():
    V = L.sobol_direction_numbers(4)
    sh = L.sobol_shifts(3, 2, 2, 4)
    x, xi = L.sobol_points(V, 10, 20, sh, want_xi=True)
    u = (x.astype(np.float64) + 0.5) * 2.0 ** -32
    np.testing.assert_allclose(xi, scipy.special.ndtri(u), rtol=1e-14, atol=1e-15)
