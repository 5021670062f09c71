"""Pins of the oracle's KL basis (Sec. 3.1): the trace identity the paper
states, eigenvalues known in closed form, and the pointwise variance."""
import numpy as np
import pytest

from oracle import kl


def test_trace_identity_sum_of_all_eigenvalues_is_sigma2_area():
    """sum_i theta_i = sigma^2 meas(Omega) (Sec. 3.1), here with every mode."""
    theta, V, pts, w, trace = kl.nystrom_eigs(16, 256, 1.7, 0.3, all_modes=True)
    assert abs(theta.sum() - 1.7) < 1e-12
    assert abs(trace - 1.7) < 1e-12
    assert np.all(theta > 0)
    assert np.all(np.diff(theta) <= 1e-15)


def test_eigenvectors_orthonormal_and_eigen_residual():
    theta, V, pts, w, _ = kl.nystrom_eigs(20, 40, 1.0, 0.3)
    np.testing.assert_allclose(V.T @ V, np.eye(40), atol=1e-12)
    A = w * kl.covariance(pts, pts, 1.0, 0.3)
    np.testing.assert_allclose(A @ V, V * theta, atol=1e-13)


def test_one_dimensional_exponential_kernel_matches_closed_form():
    """Ghanem & Spanos eigenvalues of exp(-|x-y|/lambda) on [0,1]."""
    exact = kl.exp_kernel_1d_eigenvalues(10, 1.0, 0.3)
    approx, *_ = kl.nystrom_eigs(800, 10, 1.0, 0.3, dim=1)
    np.testing.assert_allclose(approx, exact, rtol=2e-4)
    coarse, *_ = kl.nystrom_eigs(200, 10, 1.0, 0.3, dim=1)
    # midpoint quadrature: the error shrinks about 4x per halving of h
    assert np.max(np.abs(coarse / exact - 1)) > 3 * np.max(np.abs(approx / exact - 1))


def test_two_dimensional_assembly_on_a_separable_kernel():
    """With the l1 distance the kernel factorises and the 2-D spectrum is the
    set of products of the 1-D spectrum (Kronecker structure)."""
    a, *_ = kl.nystrom_eigs(12, 144, 1.0, 0.5, dim=2, metric="l1", all_modes=True)
    b, *_ = kl.nystrom_eigs(12, 12, 1.0, 0.5, dim=1, all_modes=True)
    np.testing.assert_allclose(a, np.sort(np.outer(b, b).ravel())[::-1], atol=1e-14)


def test_pointwise_variance_with_all_modes_is_sigma2():
    """At a quadrature point with every mode kept, sum_k theta_k phi_k^2 = C(x,x)."""
    q = 12
    theta, V, pts, w, _ = kl.nystrom_eigs(q, q * q, 2.0, 0.4, all_modes=True)
    B = kl.nystrom_basis(pts, theta, V, pts, w, 2.0, 0.4)
    np.testing.assert_allclose(np.sum(B * B, axis=1), 2.0, rtol=1e-10)
    # and the Nystrom formula reproduces phi_k at the quadrature nodes
    np.testing.assert_allclose(B, V / np.sqrt(w) * np.sqrt(theta), atol=1e-10)


def test_covariance_reconstruction_improves_with_modes():
    q = 24
    theta, V, pts, w, _ = kl.nystrom_eigs(q, 200, 1.0, 0.3)
    x = kl.field_points(8, 8)
    C = kl.covariance(x, x, 1.0, 0.3)
    errs = []
    for M in (10, 50, 200):
        B = kl.nystrom_basis(x, theta[:M], V[:, :M], pts, w, 1.0, 0.3)
        errs.append(np.abs(B @ B.T - C).max())
    assert errs[0] > errs[1] > errs[2]


def test_nested_points_injection_maps_to_identical_points():
    """Cell (I,J) of grid n and cell (2I,2J) of grid 2n share one field point."""
    for n in (4, 8, 16):
        coarse = kl.field_points(n, 64)
        fine = kl.field_points(2 * n, 64).reshape(2 * n, 2 * n, 2)
        np.testing.assert_array_equal(coarse.reshape(n, n, 2), fine[::2, ::2])
    rows16 = kl.level_rows(16, 64).reshape(16, 16)
    rows32 = kl.level_rows(32, 64).reshape(32, 32)
    np.testing.assert_array_equal(rows16, rows32[::2, ::2])


def test_captured_fraction_of_the_workload_field():
    b = kl.KLBasis(32, 64, 1.0, 0.3, q=24)
    assert abs(b.trace - 1.0) < 1e-12
    assert 0.8 < b.captured < 1.0
    assert b.B_ref.shape == (32 * 32, 64)
