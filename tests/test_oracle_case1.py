"""Pins of the oracle's Case I (Table 1, row 1): Dirichlet data on all four
edges (west 100, east 0, south 10, north 50) and the point QoI u(0.5, 0.5),
read as the mean of the four cells that meet at the centre.

- Constant K: the discrete problem is the cell-centred Dirichlet Laplacian,
  diagonalised by the type-II discrete sine transform (sin(pi k (i+1/2)/n),
  eigenvalue 4 sin^2(pi k / 2n) per direction); scipy's DST solves it.
- Any K symmetric under the square's rotations and reflections: by
  superposition and symmetry the centre value is exactly the mean of the
  four edge values, 40 for Table 1's data.
- Equal data on every edge: u is that constant for any K.
- Reflection in y swaps the south and north data.
"""
import numpy as np
import pytest
import scipy.fft

import workloads as W
from oracle import lib as L

G = np.array([100.0, 0.0, 10.0, 50.0])   # west, east, south, north


def _dst_solve(n, g):
    """Cell-centred Dirichlet Laplacian with K = 1 (boundary faces 2, data g)."""
    b = np.zeros((n, n))   # [j][i]
    b[:, 0] += 2 * g[0]
    b[:, -1] += 2 * g[1]
    b[0, :] += 2 * g[2]
    b[-1, :] += 2 * g[3]
    k = np.arange(1, n + 1)
    lam = 4 * np.sin(np.pi * k / (2 * n)) ** 2
    bh = scipy.fft.dstn(b, type=2)
    uh = bh / (lam[:, None] + lam[None, :])
    return scipy.fft.idstn(uh, type=2)


@pytest.mark.parametrize("n", [4, 8, 32, 64])
def test_constant_k_matches_the_sine_transform_solution(n):
    K = np.ones((n, n))
    want = _dst_solve(n, G)
    prm = L.case1_params(converged=True, tol=1e-13, max_cycles=300)
    qf, qc, p, _ = L.fmg_solve(K, prm, want_p=True)
    np.testing.assert_allclose(p, want, rtol=0, atol=1e-10 * np.abs(want).max())
    h = n // 2
    assert abs(qf - want[h - 1:h + 1, h - 1:h + 1].mean()) < 1e-10 * 100
    # the dense exact solve of the small grids
    if n <= 8:
        x = L.exact_solve_bc(K, L.stage_rhs_bc(K, G, 1), 1)
        np.testing.assert_allclose(x, want, atol=1e-11 * 100)


def _d4_field(n, a=0.8, b=0.5):
    """A field invariant under the square's symmetry group, exactly: the value
    of a cell depends only on its sorted distances (in cells) to the nearest
    west/east and south/north edges."""
    d = np.minimum(np.arange(n), n - 1 - np.arange(n))
    DX, DY = np.meshgrid(d, d, indexing="xy")
    lo, hi = np.minimum(DX, DY), np.maximum(DX, DY)
    g = a * np.cos(0.7 * lo) + b * np.sin(0.3 * hi + 0.1 * lo * hi)
    return np.exp(g)


@pytest.mark.parametrize("n", [8, 16, 64])
def test_rotation_symmetric_field_gives_the_mean_of_the_edge_values(n):
    K = _d4_field(n)
    assert np.array_equal(K, K.T) and np.array_equal(K, K[::-1, :]) and np.array_equal(K, K[:, ::-1])
    prm = L.case1_params(converged=True, tol=1e-13, max_cycles=300)
    qf, qc, _, _ = L.fmg_solve(K, prm)
    assert abs(qf - G.mean()) < 1e-9 * 100
    # (Q^c is not pinned here: injection keeps the lower-left child, so the
    # coarse field is no longer symmetric)
    # the fixed schedule (2 V(2,2) per stage) is close but not exact
    q2 = L.fmg_solve(K, L.case1_params())[0]
    assert abs(q2 - G.mean()) < 2e-2 * 100


@pytest.mark.parametrize("n", [8, 32])
def test_equal_data_on_every_edge_gives_that_constant_for_any_field(n):
    K = W.smooth_lognormal_field(n, S=1, sigma=1.5, tag=610)[0]
    prm = L.case1_params(pW=7.0, pE=7.0, pS=7.0, pN=7.0)
    qf, qc, p, _ = L.fmg_solve(K, prm, want_p=True)
    np.testing.assert_allclose(p, 7.0, rtol=1e-13)
    assert abs(qf - 7.0) < 1e-12 and abs(qc - 7.0) < 1e-12


def test_reflection_in_y_swaps_south_and_north():
    n = 32
    K = W.smooth_lognormal_field(n, S=1, tag=611)[0]
    K = 0.5 * (K + K[::-1, :])   # symmetric in y
    prm = dict(converged=True, tol=1e-13, max_cycles=300)
    _, _, pa, _ = L.fmg_solve(K, L.case1_params(pW=0, pE=0, pS=0, pN=1, **prm), want_p=True)
    _, _, pb, _ = L.fmg_solve(K, L.case1_params(pW=0, pE=0, pS=1, pN=0, **prm), want_p=True)
    np.testing.assert_allclose(pa, pb[::-1, :], atol=1e-11)
    assert np.all(np.diff(pa, axis=0) > 0)   # rises towards the north edge


def test_operator_is_spd_and_mass_balanced():
    n = 8
    K = W.smooth_lognormal_field(n, S=1, tag=612)[0]
    A = np.stack([L.apply_A_bc(K, e.reshape(n, n), 1).ravel() for e in np.eye(n * n)], axis=1)
    np.testing.assert_allclose(A, A.T, atol=1e-14)
    assert np.linalg.eigvalsh(A).min() > 0
    # the rows sum to the boundary transmissibilities: A 1 = stage rhs of unit data
    np.testing.assert_allclose(A.sum(axis=1), L.stage_rhs_bc(K, np.ones(4), 1).ravel(), rtol=1e-13,
                               atol=1e-13 * K.max())


def test_prolongation_and_fmg_interpolation_of_linear_functions():
    """u = a + b x + c y: the bilinear interpolation reproduces it in the
    interior; with the face values of u as Dirichlet ghosts (2 g - u) the
    FMG interpolation reproduces it everywhere; the correction ghost -e
    makes P e vanish on a face where e is linear and zero."""
    nc = 8
    x = (np.arange(nc) + 0.5) / nc
    X, Y = np.meshgrid(x, x, indexing="xy")
    a, b, c = 0.3, 1.7, -0.9
    uc = a + b * X + c * Y
    xf = (np.arange(2 * nc) + 0.5) / (2 * nc)
    XF, YF = np.meshgrid(xf, xf, indexing="xy")
    want = a + b * XF + c * YF
    # face data along each edge vary linearly; a constant per edge is exact
    # only where the function is constant along the edge: take b = 0 for
    # the north/south faces and c = 0 for the west/east faces separately
    for bb, cc in ((b, 0.0), (0.0, c)):
        u = a + bb * X + cc * Y
        g = np.array([a + cc * 0.5, a + bb + cc * 0.5, a + bb * 0.5, a + bb * 0.5 + cc])
        if bb == 0.0:
            g = np.array([np.nan, np.nan, a, a + cc])
            got = L.fmg_interpolate_bc(u, np.nan_to_num(g), 1)
            np.testing.assert_allclose(got[:, 1:-1], (a + cc * YF)[:, 1:-1], atol=1e-14)
        else:
            g = np.array([a, a + bb, np.nan, np.nan])
            got = L.fmg_interpolate_bc(u, np.nan_to_num(g), 0)
            np.testing.assert_allclose(got, a + bb * XF, atol=1e-14)
    # interior of a general linear function
    got = L.prolong_add_bc(uc, np.zeros((2 * nc, 2 * nc)), 1)
    np.testing.assert_allclose(got[1:-1, 1:-1], want[1:-1, 1:-1], atol=1e-14)
    # correction of an error that vanishes on the south face: e = y
    e = Y.copy()
    got = L.prolong_add_bc(e, np.zeros((2 * nc, 2 * nc)), 1)
    np.testing.assert_allclose(got[:, 2:-2][:-1], YF[:, 2:-2][:-1], atol=1e-14)


@pytest.mark.parametrize("n", [32, 64])
def test_vcycle_contracts_on_dirichlet_problems(n):
    K = W.smooth_lognormal_field(n, S=1, sigma=1.0, tag=613)[0]
    for KK, bound in ((np.ones((n, n)), 0.15), (K, 0.3)):
        b = L.stage_rhs_bc(KK, G, 1)
        _, h = L.vcycle_solve(KK, b, np.zeros_like(b), ncycles=10, ns=1)
        rho = (h[10] / h[4]) ** (1 / 6)
        assert rho < bound, rho


@pytest.mark.parametrize("converged", [False, True])
def test_coarse_qoi_is_the_fine_qoi_of_the_injected_problem(converged):
    n = 64
    K = W.smooth_lognormal_field(n, S=1, tag=614)[0]
    prm = L.case1_params(converged=converged, tol=1e-12)
    qf, qc, _, _ = L.fmg_solve(K, prm)
    qf2, _, _, _ = L.fmg_solve(np.ascontiguousarray(K[::2, ::2]), prm)
    assert qc == qf2


def test_centre_value_is_linear_in_the_data():
    K = W.smooth_lognormal_field(16, S=1, tag=615)[0]
    prm = dict(converged=True, tol=1e-13)
    q = L.fmg_solve(K, L.case1_params(**prm))[0]
    q2 = L.fmg_solve(K, L.case1_params(pW=200.0, pE=0.0, pS=20.0, pN=100.0, **prm))[0]
    assert abs(q2 - 2 * q) < 1e-10 * abs(q)
