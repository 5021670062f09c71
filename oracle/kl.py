"""Karhunen-Loeve expansion of the lognormal permeability (Sec. 3.1).

TEST INFRASTRUCTURE ONLY (see the oracle package docstring).

The Gaussian field g has the Matern covariance of Sec. 3.1,
C(d) = sigma^2 2^(1-nu) / Gamma(nu) (sqrt(2 nu) d / lambda)^nu K_nu(sqrt(2 nu) d / lambda),
C(0) = sigma^2, d the Euclidean distance (Table 2 uses nu = 1/2, the
exponential sigma^2 exp(-d / lambda), and nu = 1).
Its KL expansion g(x) = sum_k sqrt(theta_k) phi_k(x) xi_k, truncated to M
terms, is computed by the Nystrom method (the paper cites Ernst et al. for
the eigenproblem and states no method of its own):

  * midpoint quadrature on a q x q grid, equal weights w = 1/q^2;
  * the symmetric matrix A_ij = w C(x_i, x_j) has eigenpairs (theta_k, v_k),
    v_k orthonormal, and phi_k(x_j) = v_jk / sqrt(w);
  * phi_k at any point x by the Nystrom formula
    phi_k(x) = (1/theta_k) sum_j w C(x, x_j) phi_k(x_j).

The sum of all eigenvalues equals trace(A) = sigma^2 meas(Omega) exactly, the
identity the paper uses to define the captured-variability fraction.

Field points (the consistency reading of Sec. 2.5): the field of the n x n
grid is sampled at the points of the finest configured grid n_ref that
coarsening by injection keeps, i.e. cell (i, j) of grid n sits at
((s i + 1/2)/n_ref, (s j + 1/2)/n_ref), s = n_ref / n.  Injection
k^c[I][J] = k^f[2I][2J] then maps every coarse point onto the same physical
point, so K^c_l and K^f_(l-1) are the same random vector, not merely equal
in law.
"""
import numpy as np
import scipy.linalg
import scipy.optimize
import scipy.special


def quadrature_points(q, dim=2):
    """Midpoint grid of [0,1]^dim; 2-D points ordered j*q + i (x fastest)."""
    t = (np.arange(q) + 0.5) / q
    if dim == 1:
        return t[:, None]
    X, Y = np.meshgrid(t, t, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def matern(d, sigma2, lam, nu=0.5):
    """The Matern covariance of Sec. 3.1 at distances d, written as the paper
    states it (scipy's modified Bessel function K_nu); C(0) = sigma^2."""
    d = np.asarray(d, dtype=np.float64)
    x = np.sqrt(2.0 * nu) * d / lam
    with np.errstate(invalid="ignore", divide="ignore"):
        c = sigma2 * 2.0 ** (1.0 - nu) / scipy.special.gamma(nu) * x ** nu * scipy.special.kv(nu, x)
    return np.where(x == 0.0, sigma2, c)


def covariance(X, Y, sigma2, lam, metric="l2", nu=0.5):
    """Matern covariance (smoothness nu) between point sets X [a][d], Y [b][d].
    metric 'l1' (separable, nu = 1/2) exists only to pin the 2-D code against
    1-D results."""
    diff = X[:, None, :] - Y[None, :, :]
    if metric == "l2":
        d = np.sqrt(np.sum(diff * diff, axis=-1))
    elif metric == "l1":
        d = np.sum(np.abs(diff), axis=-1)
    else:
        raise ValueError(metric)
    if nu == 0.5:
        return sigma2 * np.exp(-d / lam)
    return matern(d, sigma2, lam, nu)


def nystrom_eigs(q, M, sigma2, lam, dim=2, metric="l2", all_modes=False, nu=0.5):
    """Top-M eigenpairs of the Nystrom matrix, eigenvalues descending.
    Returns (theta [M], V [q^dim][M] orthonormal columns, points, w, trace)."""
    pts = quadrature_points(q, dim)
    n = pts.shape[0]
    w = 1.0 / n
    A = w * covariance(pts, pts, sigma2, lam, metric, nu)
    if all_modes or M >= n:
        theta, V = scipy.linalg.eigh(A)
    else:
        theta, V = scipy.linalg.eigh(A, subset_by_index=[n - M, n - 1])
    order = np.argsort(theta)[::-1]
    theta, V = theta[order][:M], V[:, order][:, :M]
    # fix the sign of each eigenvector: its largest-magnitude entry positive
    idx = np.argmax(np.abs(V), axis=0)
    V = V * np.sign(V[idx, np.arange(V.shape[1])])
    return theta, V, pts, w, float(np.trace(A))


def nystrom_basis(points, theta, V, qpts, w, sigma2, lam, metric="l2", chunk=4096, nu=0.5):
    """B[x][k] = sqrt(theta_k) phi_k(x) = (1/sqrt(theta_k)) sum_j sqrt(w) C(x,x_j) v_jk."""
    B = np.empty((points.shape[0], theta.shape[0]))
    scale = np.sqrt(w) / np.sqrt(theta)
    for a in range(0, points.shape[0], chunk):
        Cx = covariance(points[a:a + chunk], qpts, sigma2, lam, metric, nu)
        B[a:a + chunk] = (Cx @ V) * scale
    return B


def field_points(n, n_ref):
    """Sample points of the n x n grid (nested reading), ordered j*n + i."""
    s = n_ref // n
    assert s * n == n_ref
    t = (s * np.arange(n) + 0.5) / n_ref
    X, Y = np.meshgrid(t, t, indexing="xy")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def level_rows(n, n_ref):
    """Row indices of the n_ref x n_ref basis that the n x n grid uses."""
    s = n_ref // n
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return ((s * j) * n_ref + s * i).ravel()


class KLBasis:
    """Truncated KL basis on the finest grid's points; coarser grids take rows."""

    def __init__(self, n_ref, M, sigma2, lam, q=None, metric="l2", nu=0.5):
        if q is None:
            q = max(32, int(np.ceil(np.sqrt(8 * M))))
        self.n_ref, self.M, self.sigma2, self.lam, self.q, self.nu = n_ref, M, sigma2, lam, q, nu
        theta, V, qpts, w, trace = nystrom_eigs(q, M, sigma2, lam, 2, metric, nu=nu)
        self.theta = theta
        self.trace = trace                           # = sigma^2 meas(Omega)
        self.captured = float(theta.sum() / trace)   # fraction of variability kept
        self.B_ref = nystrom_basis(field_points(n_ref, n_ref), theta, V, qpts, w,
                                   sigma2, lam, metric, nu=nu)

    def level_basis(self, n):
        """[n*n][M] rows of the basis for the n x n grid."""
        return np.ascontiguousarray(self.B_ref[level_rows(n, self.n_ref)])


def layered_basis_y(n_ref, M, sigma2, lam, q=256):
    """A field varying only in y (1-D KL in y on the nested points), as a
    [n_ref*n_ref][M] basis; used by the closed-form estimator checks."""
    theta, V, qpts, w, _ = nystrom_eigs(q, M, sigma2, lam, 1)
    y = ((np.arange(n_ref) + 0.5) / n_ref)[:, None]
    b = nystrom_basis(y, theta, V, qpts, w, sigma2, lam)     # [n_ref][M]
    return np.repeat(b, n_ref, axis=0), theta                # row j*n_ref+i -> b[j]


def synthesize(B, xi):
    """K = exp(g), g = B xi: B [cells][M], xi [S][M] -> K [S][cells]."""
    return np.exp(xi @ B.T)


def exp_kernel_1d_eigenvalues(M, sigma2, lam, length=1.0):
    """Exact eigenvalues of sigma^2 exp(-|x-y|/lam) on an interval of the given
    length (Ghanem & Spanos 1991, Sec. 2.3.3): with c = 1/lam, a = length/2,
    theta = 2 c sigma^2 / (w^2 + c^2), where w solves c - w tan(w a) = 0
    (even eigenfunctions) or w + c tan(w a) = 0 (odd ones)."""
    c, a = 1.0 / lam, 0.5 * length
    roots = []
    for m in range(M + 2):
        lo, hi = m * np.pi / a, (m + 0.5) * np.pi / a      # even root in each branch
        f = lambda w: c - w * np.tan(w * a)
        roots.append(scipy.optimize.brentq(f, lo + 1e-12, hi - 1e-12))
        lo, hi = (m + 0.5) * np.pi / a, (m + 1) * np.pi / a  # odd root
        g = lambda w: w + c * np.tan(w * a)
        roots.append(scipy.optimize.brentq(g, lo + 1e-12, hi - 1e-12))
    w = np.sort(np.array(roots))[:M]
    return 2 * c * sigma2 / (w * w + c * c)
