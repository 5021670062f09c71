"""Pins of the oracle's finite-volume discretisation (Eq. 1, Table 1 Case II)
and its full multigrid (Sec. 2.5) against closed forms, invariants, a dense
library solve and textbook multigrid behaviour."""
import numpy as np
import pytest

import workloads as W
from oracle import lib as L


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_constant_k_linear_pressure_unit_outflux(n):
    """K = 1, p_W = 1, p_E = 0: the discrete solution is p = 1 - x at the cell
    centres and the outflux is exactly 1; FMG interpolation reproduces it."""
    K = np.ones((n, n))
    qf, qc, p, _ = L.fmg_solve(K, want_p=True)
    x = (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(p, np.broadcast_to(1 - x, (n, n)), atol=1e-14)
    assert abs(qf - 1) < 1e-13
    if n > 4:
        assert abs(qc - 1) < 1e-13


def test_outflux_is_linear_in_boundary_data():
    K = W.smooth_lognormal_field(16)[0]
    prm = dict(converged=True, tol=1e-13)
    q1 = L.fmg_solve(K, L.params(pW=1.0, pE=0.0, **prm))[0]
    q100 = L.fmg_solve(K, L.params(pW=100.0, pE=0.0, **prm))[0]
    qshift = L.fmg_solve(K, L.params(pW=101.0, pE=1.0, **prm))[0]
    assert abs(q100 / q1 - 100) < 1e-9
    assert abs(qshift / q1 - 100) < 1e-9


@pytest.mark.parametrize("n", [8, 32])
def test_layered_in_x_series_harmonic_mean(n):
    """K varies with x only: each row is a series of resistances 1/K_i, so
    Q = n / sum_i (1/K_i)  (harmonic mean).  K is smooth at the grid scale,
    as a truncated KL field is: coarse operators built from injected K do not
    represent cell-to-cell jumps, and V-cycles on white-noise K can diverge."""
    x = (np.arange(n) + 0.5) / n
    kx = np.exp(1.5 * np.sin(2 * np.pi * x) + 0.5 * np.cos(6 * np.pi * x))
    K = np.broadcast_to(kx, (n, n)).copy()
    qf = L.fmg_solve(K, L.params(converged=True, tol=1e-14, max_cycles=200))[0]
    assert abs(qf - n / np.sum(1 / kx)) < 1e-11 * qf


@pytest.mark.parametrize("n", [8, 32])
def test_layered_in_y_parallel_arithmetic_mean(n):
    """K varies with y only: rows are parallel channels, p = 1 - x in every
    row, Q = sum_j K_j / n (arithmetic mean); already exact after FMG."""
    ky = np.exp(W.rng(tag=11).standard_normal(n))  # any K: rows do not interact
    K = np.broadcast_to(ky[:, None], (n, n)).copy()
    qf, qc, p, _ = L.fmg_solve(K, want_p=True)
    assert abs(qf - ky.sum() / n) < 1e-12 * qf
    x = (np.arange(n) + 0.5) / n
    np.testing.assert_allclose(p, np.broadcast_to(1 - x, (n, n)), atol=1e-13)


def _dense(K):
    n = K.shape[0]
    A = np.zeros((n * n, n * n))
    for c in range(n * n):
        e = np.zeros(n * n)
        e[c] = 1
        A[:, c] = L.apply_A(K, e.reshape(n, n)).ravel()
    return A


@pytest.mark.parametrize("n", [4, 8, 16])
def test_operator_symmetric_positive_definite(n):
    A = _dense(W.lognormal_field(n, tag=12)[0])
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-14 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    # zero row sums except where a Dirichlet face adds to the diagonal
    rs = A.sum(axis=1).reshape(n, n)
    assert np.allclose(rs[:, 1:-1], 0, atol=1e-12)


@pytest.mark.parametrize("n", [4, 8, 16])
def test_converged_fmg_matches_dense_direct_solve(n):
    """Brute force: numpy's LU solve of the assembled system."""
    K = W.smooth_lognormal_field(n, tag=13)[0]
    b = L.stage_rhs(K)
    x_direct = np.linalg.solve(_dense(K), b.ravel()).reshape(n, n)
    qf, _, p, _ = L.fmg_solve(K, L.params(converged=True, tol=1e-14, max_cycles=300),
                              want_p=True)
    np.testing.assert_allclose(p, x_direct, rtol=0, atol=1e-12)
    assert abs(qf - L.outflux(K, x_direct)) < 1e-12 * abs(qf)


def test_exact_coarsest_solve_matches_library():
    K = W.lognormal_field(4, tag=14)[0]
    b = W.rng(tag=15).standard_normal((4, 4))
    np.testing.assert_allclose(L.exact_solve(K, b),
                               np.linalg.solve(_dense(K), b.ravel()).reshape(4, 4),
                               rtol=0, atol=1e-13)


def test_mass_balance():
    K = W.smooth_lognormal_field(32, tag=16)[0]
    _, _, p, _ = L.fmg_solve(K, L.params(converged=True, tol=1e-13, max_cycles=500),
                             want_p=True)
    qin, qout = L.influx(K, p), L.outflux(K, p)
    assert abs(qin - qout) < 1e-9 * qout


def test_injection_takes_lower_left_child():
    n = 8
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    Kf = 1000.0 * j + i
    Kc = L.inject(Kf)
    J, I = np.meshgrid(np.arange(n // 2), np.arange(n // 2), indexing="ij")
    np.testing.assert_array_equal(Kc, 2000.0 * J + 2.0 * I)


def test_restriction_sums_children():
    rf = W.rng(tag=17).standard_normal((8, 8))
    bc = L.restrict_sum(rf)
    np.testing.assert_allclose(bc, rf.reshape(4, 2, 4, 2).sum(axis=(1, 3)), atol=1e-15)


def test_prolongation_reproduces_linear_functions_in_the_interior():
    nc = 8
    xc = (np.arange(nc) + 0.5) / nc
    xf = (np.arange(2 * nc) + 0.5) / (2 * nc)
    for fx, fy in [(1.0, 0.0), (0.0, 1.0), (0.7, -0.3)]:
        ec = fx * xc[None, :] + fy * xc[:, None] + 0.25
        out = L.prolong_add(ec, np.zeros((2 * nc, 2 * nc)))
        exact = fx * xf[None, :] + fy * xf[:, None] + 0.25
        np.testing.assert_allclose(out[1:-1, 1:-1], exact[1:-1, 1:-1], atol=1e-14)
    # an error linear in x and zero on the west face is exact up to that face
    ec = np.broadcast_to(xc, (nc, nc)).copy()
    out = L.prolong_add(ec, np.zeros((2 * nc, 2 * nc)))
    np.testing.assert_allclose(out[1:-1, :-1], np.broadcast_to(xf, (2 * nc, 2 * nc))[1:-1, :-1],
                               atol=1e-14)
    # a constant error is kept where no Dirichlet ghost enters, halved next to one
    out = L.prolong_add(np.ones((nc, nc)), np.zeros((2 * nc, 2 * nc)))
    np.testing.assert_allclose(out[:, 1:-1], 1.0, atol=1e-15)
    np.testing.assert_allclose(out[:, [0, -1]], 0.5, atol=1e-15)


def test_fmg_interpolation_of_linear_solution_is_exact():
    """The Dirichlet ghost 2 g - u is linear extrapolation to the ghost centre."""
    nc = 8
    xc = (np.arange(nc) + 0.5) / nc
    uc = np.broadcast_to(3.0 - 2.0 * xc, (nc, nc)).copy()      # g_W = 3, g_E = 1
    out = L.fmg_interpolate(uc, pW=3.0, pE=1.0)
    xf = (np.arange(2 * nc) + 0.5) / (2 * nc)
    np.testing.assert_allclose(out, np.broadcast_to(3.0 - 2.0 * xf, (2 * nc, 2 * nc)), atol=1e-14)


def test_vcycle_convergence_factor():
    """Textbook RB-GS V(2,2): per-cycle residual reduction well below 0.2 for
    the Laplacian, with either choice of correction coefficients (they agree
    for constant K)."""
    n = 64
    b = W.rng(tag=18).standard_normal((n, n))
    for op in (0, 1):
        _, hist = L.vcycle_solve(np.ones((n, n)), b, np.zeros((n, n)), ncycles=8, coarse_op=op)
        rho = (hist[8] / hist[3]) ** (1 / 5)
        assert rho < 0.15, rho


def test_correction_operators_from_child_means_keep_the_cycle_contracting():
    """Injected coefficients on the correction grids sample K up to half a
    coarse cell away from the cell centre on deep grids; on a field with
    contrast ~100 the cycle then diverges.  Geometric means of the children
    keep every field of the set contracting."""
    n = 32
    K = W.smooth_lognormal_field(n, S=23, tag=122)
    rho = {0: [], 1: []}
    for k in K:
        b = L.stage_rhs(k)
        for op in (0, 1):
            _, h = L.vcycle_solve(k, b, np.zeros_like(b), ncycles=12, coarse_op=op)
            rho[op].append((h[12] / h[4]) ** (1 / 8))
    assert max(rho[0]) > 1.0          # injection: at least one field diverges
    assert max(rho[1]) < 0.6          # child means: all contract


@pytest.mark.parametrize("nc", [2, 4, 16])
def test_child_geometric_mean_of_a_log_affine_field_is_its_value_at_the_parent_centre(nc):
    """K = exp(a + b x + c y) at the cell centres of grid 2 nc.  The four
    children of a coarse cell are placed symmetrically about its centre, so
    their geometric mean is exp(a + b X + c Y) at the coarse centre (X, Y),
    whatever a, b, c.  An arithmetic mean, a wrong set of children, or
    swapped row / column indices all miss this value."""
    nf = 2 * nc
    a, b, c = 0.3, 2.1, -1.4
    x = (np.arange(nf) + 0.5) / nf
    Kf = np.exp(a + b * x[None, :] + c * x[:, None])      # [j][i], x fastest
    X = (np.arange(nc) + 0.5) / nc
    want = np.exp(a + b * X[None, :] + c * X[:, None])
    got = L.geometric_children(Kf)
    np.testing.assert_allclose(got, want, rtol=2e-15, atol=0)
    # the children are the 2x2 block of the parent: a field constant on
    # each block (and different between blocks) passes through unchanged
    r = np.random.default_rng(5).uniform(0.5, 2.0, (nc, nc))
    np.testing.assert_allclose(L.geometric_children(np.kron(r, np.ones((2, 2)))), r, rtol=2e-15)


def test_fmg_two_vcycles_is_close_to_converged_for_smooth_fields():
    K = W.smooth_lognormal_field(64, S=1, sigma=1.0, tag=20)[0]
    q2 = L.fmg_solve(K)[0]
    qc = L.fmg_solve(K, L.params(converged=True, tol=1e-13, max_cycles=200))[0]
    assert abs(q2 - qc) < 2e-3 * abs(qc)


@pytest.mark.parametrize("converged", [False, True])
def test_coarse_qoi_is_the_fine_qoi_of_the_injected_problem(converged):
    """Algorithm 3: Q^c of a level-l solve is bitwise the Q^f of a solve one
    grid coarser on the injected coefficients (the FMG by-product)."""
    prm = L.params(converged=converged, tol=1e-12)
    for n in (8, 16, 64):
        K = W.lognormal_field(n, tag=21 + n)[0]
        _, qc, _, _ = L.fmg_solve(K, prm)
        qf_coarse, _, _, _ = L.fmg_solve(L.inject(K), prm)
        assert qc == qf_coarse


def test_batch_equals_single_solves():
    K = W.lognormal_field(16, S=5, tag=30)
    qf, qc, p, _ = L.fmg_solve_batch(K, want_p=True, nthreads=2)
    for s in range(5):
        a, b, ps, _ = L.fmg_solve(K[s], want_p=True)
        assert qf[s] == a and qc[s] == b
        np.testing.assert_array_equal(p[s], ps)
