"""Pins of the oracle's randomized QMC rules (Sec. 2.4): the rank-1 lattice
sequence with a random shift, built component by component, and nested
uniform (Owen) scrambling of the Sobol' points.

- The shift-averaged worst-case error the construction minimises equals its
  dual-lattice series: B_2(x) = sum_{h != 0} e^{2 pi i h x} / (2 pi^2 h^2),
  so e^2 = sum over nonzero h with h.z = 0 (mod n) of prod_j r(h_j),
  r(0) = 1, r(h) = gamma_j / (2 pi^2 h^2).
- Each component is the minimiser of its criterion, recomputed from the
  error definition directly; the vector beats random odd vectors.
- The first 2^m points of the sequence are exactly the 2^m-point lattice.
- Owen scrambling keeps the one-dimensional (0, m, 1)-net property and the
  two-dimensional (0, m, 2)-net property of the Sobol' points, is a
  bijection, and two inputs with a common leading block of bits keep a
  common leading block of the same length and differ in the next bit.
"""
import numpy as np
import pytest

from oracle import lib as L


def test_worst_case_error_is_its_dual_lattice_series():
    """One dimension, z = 1: the dual lattice is h = l n, so
    e^2 = 2 sum_l 1 / (2 pi^2 l^2 n^2) = 1 / (6 n^2) exactly.  Two dimensions,
    z = (1, z_2), gamma = (1, 1/4): summing h_1 over each residue class in
    closed form (sum_l (a + l n)^-2 = (pi/n)^2 / sin^2(pi a / n)) leaves a
    series over h_2 whose tail beyond 2e6 is below 1e-9."""
    for m in (3, 6, 9):
        n = 1 << m
        # -1 + (1/n) sum (1 + omega) cancels: rounding of the sum is n eps at most
        assert abs(L.lattice_e2(np.array([1], np.uint32), m) - 1.0 / (6.0 * n * n)) < 4 * n * 2.0 ** -52
    m, n, z2 = 6, 64, 27
    H = 2_000_000
    h2 = np.arange(-H, H + 1, dtype=np.int64)
    a = (-h2 * z2) % n
    safe = np.where(a == 0, 1, a)
    inner = np.where(a == 0, 1.0 + 1.0 / (6.0 * n * n), 1.0 / (2.0 * n * n * np.sin(np.pi * safe / n) ** 2))
    r2 = np.where(h2 == 0, 1.0, 0.25 / (2.0 * np.pi ** 2 * np.where(h2 == 0, 1, h2).astype(float) ** 2))
    series = float(np.sum(r2 * inner)) - 1.0     # leave out h = 0
    e2 = L.lattice_e2(np.array([1, z2], np.uint32), m)
    assert abs(series - e2) < 1e-3 * e2


def test_each_component_minimises_its_criterion():
    """Recompute the criterion sum_m e^2_m(z_1..z_s) / e^2_m(z_1..z_(s-1)) from
    the error definition (a direct product over all components) for every
    odd candidate; the construction's choice attains the minimum."""
    m_min, m_max, dim = 3, 7, 5
    z = L.lattice_cbc(dim, m_min, m_max)
    assert z[0] == 1
    for s in range(1, dim):
        crit = {}
        for c in range(1, 1 << (m_max - 1), 2):
            zz = np.concatenate([z[:s], [c]]).astype(np.uint32)
            crit[c] = sum(L.lattice_e2(zz, m) / L.lattice_e2(z[:s], m) for m in range(m_min, m_max + 1))
        best = min(crit.values())
        assert crit[int(z[s])] <= best * (1 + 1e-12)
        assert int(z[s]) == min(c for c, v in crit.items() if v <= best * (1 + 1e-12))


def test_vector_beats_random_odd_vectors_at_every_size():
    m_min, m_max, dim = 4, 10, 16
    z = L.lattice_cbc(dim, m_min, m_max)
    rng = np.random.default_rng(7)
    vecs = [(2 * rng.integers(0, 1 << (m_max - 1), dim) + 1).astype(np.uint32) for _ in range(20)]
    for m in range(m_min, m_max + 1):
        rand = [L.lattice_e2(v, m) for v in vecs]
        # the criterion balances every size: better than a typical random
        # vector at all of them, better than the best of 20 above the smallest
        assert L.lattice_e2(z, m) < np.median(rand), m
        if m > m_min:
            assert L.lattice_e2(z, m) < min(rand), m


def test_first_points_of_the_sequence_are_the_lattice():
    m_max = 10
    z = L.lattice_cbc(6, 3, m_max)
    x = L.lattice_points(z, m_max, seed=5, level=2, first=0, n=1 << m_max, first_shift=3, n_shifts=1)[0]
    delta = x[0]                                  # point 0 is the origin shifted
    t = (x - delta) >> np.uint32(32 - m_max)      # undo the shift, back to the integer lattice
    for m in range(3, m_max + 1):
        n = 1 << m
        got = {tuple(r) for r in (t[:n] >> np.uint32(m_max - m))}
        want = {tuple((k * z.astype(np.int64)) % n) for k in range(n)}
        assert got == want, m
    # the shift: one random vector per (level, shift), the same for every point
    y = L.lattice_points(z, m_max, seed=5, level=2, first=17, n=5, first_shift=3, n_shifts=1)[0]
    np.testing.assert_array_equal(y, x[17:22])


def test_owen_scramble_keeps_the_net_property_and_is_a_bijection():
    V = L.sobol_direction_numbers(4)
    m = 10
    x = L.sobol_owen_points(V, seed=9, level=1, first=0, n=1 << m, first_shift=2, n_shifts=2)
    for r in range(2):
        for d in range(4):
            top = np.sort(x[r, :, d] >> np.uint32(32 - m))
            np.testing.assert_array_equal(top, np.arange(1 << m))
        # (0, m, 2)-net in the first two dimensions: every 2^a x 2^(m-a) box holds one point
        for a in range(m + 1):
            cells = (x[r, :, 0] >> np.uint32(32 - a)).astype(np.int64) * (1 << (m - a)) + \
                    (x[r, :, 1] >> np.uint32(32 - (m - a))).astype(np.int64)
            assert len(np.unique(cells)) == 1 << m
    ins = np.random.default_rng(3).integers(0, 1 << 32, 4000, dtype=np.uint64).astype(np.uint32)
    out = L.owen_scramble(9, 1, 0, 3, ins)
    assert len(np.unique(out)) == len(np.unique(ins))


def test_owen_scramble_is_nested():
    rng = np.random.default_rng(11)
    for _ in range(200):
        a = int(rng.integers(0, 1 << 32))
        k = int(rng.integers(0, 32))
        b = a ^ (1 << (31 - k))                    # same leading k bits, differ at bit k
        b ^= int(rng.integers(0, 1 << max(31 - k, 0))) if k < 31 else 0
        ya, yb = (int(v) for v in L.owen_scramble(4, 0, 1, 2, np.array([a, b], np.uint32)))
        if k > 0:
            assert (ya >> (32 - k)) == (yb >> (32 - k))
        assert ((ya >> (31 - k)) & 1) != ((yb >> (31 - k)) & 1)
    # across scrambles the leading bits of a fixed input are uniform
    tops = [int(L.owen_scramble(4, 0, r, 0, np.array([123456789], np.uint32))[0]) >> 28 for r in range(1600)]
    counts = np.bincount(tops, minlength=16)
    chi2 = np.sum((counts - 100.0) ** 2 / 100.0)
    assert chi2 < 45.0
