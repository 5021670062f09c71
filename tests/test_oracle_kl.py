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


# ---------------------------------------------------------------- Matern smoothness (Table 2)
@pytest.mark.parametrize("lam", [0.1, 0.5, 1.0])
def test_matern_general_formula_reduces_to_the_closed_forms(lam):
    """The paper's formula with K_nu: nu = 1/2 is sigma^2 exp(-d/lambda);
    nu = 3/2 is (1 + x) e^-x with x = sqrt(3) d / lambda; nu = 5/2 is
    (1 + x + x^2/3) e^-x with x = sqrt(5) d / lambda."""
    d = np.linspace(0.0, 2.0, 401)
    np.testing.assert_allclose(kl.matern(d, 1.3, lam, 0.5), 1.3 * np.exp(-d / lam), rtol=1e-13)
    x = np.sqrt(3.0) * d / lam
    np.testing.assert_allclose(kl.matern(d, 1.3, lam, 1.5), 1.3 * (1 + x) * np.exp(-x), rtol=1e-12)
    x = np.sqrt(5.0) * d / lam
    np.testing.assert_allclose(kl.matern(d, 1.3, lam, 2.5), 1.3 * (1 + x + x * x / 3) * np.exp(-x), rtol=1e-12)


@pytest.mark.parametrize("r", [0.03, 0.2, 0.7, 1.4])
def test_matern_nu1_is_the_hankel_transform_of_its_spectral_density(r):
    """In two dimensions the Matern covariance with nu = 1 has spectral
    density proportional to (a^2 + w^2)^-2, a = sqrt(2)/lambda, so
    C(r) / sigma^2 = 2 a^2 int_0^inf J_0(w r) w / (a^2 + w^2)^2 dw."""
    import scipy.integrate
    import scipy.special
    lam = 0.5
    a = np.sqrt(2.0) / lam
    f = lambda w: scipy.special.j0(w * r) * w / (a * a + w * w) ** 2
    total, cut = 0.0, 0.0
    step = 2 * np.pi / r
    while cut < 4000.0:
        total += scipy.integrate.quad(f, cut, cut + step, limit=200, epsabs=1e-16, epsrel=1e-13)[0]
        cut += step
    want = 2 * a * a * total
    assert abs(kl.matern(r, 1.0, lam, 1.0) - want) < 1e-8


def test_matern_nu1_spectrum_satisfies_the_trace_identity():
    theta, V, pts, w, trace = kl.nystrom_eigs(16, 256, 0.9, 0.5, all_modes=True, nu=1.0)
    assert abs(theta.sum() - 0.9) < 1e-12 and abs(trace - 0.9) < 1e-12
    assert np.all(theta > -1e-14)
    # a smoother field puts more variance in its first modes than nu = 1/2
    t05, *_ = kl.nystrom_eigs(16, 8, 0.9, 0.5, nu=0.5)
    assert theta[:8].sum() > t05.sum()


def test_library_covariance_matches_the_oracle():
    """fm_matern_covariance (the library's own x K_1(x): ascending series
    below 2, trapezoidal rule on its integral above) against the oracle's
    formula through scipy, for every smoothness the library builds."""
    import paper_1910_04727_gb300 as fm
    d = np.concatenate([[0.0, 1e-12, 1e-6], np.linspace(1e-4, 3.0, 3001)])
    for nu in (0.5, 1.0, 1.5, 2.5):
        for lam in (0.1, 0.5, 1.0):
            got = fm.matern_covariance(d, nu, 1.7, lam)
            want = kl.matern(d, 1.7, lam, nu)
            big = want > 1e-200
            np.testing.assert_allclose(got[big], want[big], rtol=5e-14, atol=0)
    with pytest.raises(fm.FmError):
        fm.matern_covariance(d, 0.75, 1.0, 1.0)
