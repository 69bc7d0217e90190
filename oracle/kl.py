"""Karhunen-Loeve random fields for log K and phi (oracle; test infrastructure only).

The paper models porosity (and through it permeability) as random fields
driven by a few random variables (Sec. 2.2 and the abstract; future work on
richer fields, Sec. 5).  The configuration solved with random fields takes
log K and phi as Gaussian random fields with the squared-exponential
covariance C(r) = sigma^2 exp(-r^2 / (2 l^2)), l = 0.3 m, each truncated to
its 32 leading Karhunen-Loeve terms:

    log K(x) = log K_mean + sigma_K   sum_k sqrt(lam_k) theta_k   psi_k(x)
    phi(x)   = phi_mean   + sigma_phi sum_k sqrt(lam_k) theta'_k  psi_k(x),  clipped to [phi_lo, phi_hi]

with theta, theta' iid N(0, 1) passed in by the caller (they are the method's
random inputs), and q_in from a uniform xi as in the three-parameter model.

The covariance kernel separates, exp(-(dx^2 + dy^2)/(2 l^2)) =
exp(-dx^2/(2 l^2)) exp(-dy^2/(2 l^2)), so the 2-D eigenpairs are products of
1-D ones on [0, Lx] and [0, Ly]: lam = lam_x lam_y, psi = psi_x(x) psi_y(y).
Each 1-D eigenproblem is solved by the Nystrom method on an n-point
Gauss-Legendre rule (numpy's nodes, scipy's symmetric eigensolver): with
W = diag(w), the matrix W^1/2 K W^1/2 has eigenpairs (lam, W^1/2 u), u the
eigenfunction at the nodes normalised to sum_q w_q u_q^2 = 1, and
psi(x) = (1/lam) sum_q w_q k(x, x_q) u_q extends it to any x (the Nystrom
interpolant).  Conventions (needed for two independent implementations to
agree): each 1-D eigenfunction's sign makes sum_q w_q (q + 1) u_q positive;
the 2-D terms are the 32 largest products lam_x lam_y, ordered by decreasing
product, ties (relative difference below 1e-9) ordered by (i + j, i).
"""
import numpy as np
import scipy.linalg as sla

N_QUAD = 256
N_TERMS = 32
CORR_LEN = 0.3
N_1D = 40  # 1-D modes considered for the 2-D products


def gauss_legendre(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def kernel_1d(x, y, ell=CORR_LEN):
    return np.exp(-((x[:, None] - y[None, :]) ** 2) / (2.0 * ell * ell))


def nystrom_1d(L, n=N_QUAD, ell=CORR_LEN, m=N_1D):
    """Leading m eigenpairs of the 1-D SE kernel on [0, L]: (lam[m], nodes,
    weights, u[m][n]) with u normalised and sign-fixed as described above."""
    xq, wq = gauss_legendre(n, 0.0, L)
    sw = np.sqrt(wq)
    A = sw[:, None] * kernel_1d(xq, xq, ell) * sw[None, :]
    lam, V = sla.eigh(A)
    order = np.argsort(lam)[::-1][:m]
    lam = lam[order]
    U = (V[:, order] / sw[:, None]).T          # u_i(x_q): sum_q w_q u^2 = 1
    s = np.sign(U @ (wq * (np.arange(n) + 1.0)))
    U = U * s[:, None]
    return lam, xq, wq, U


def eval_1d(x, lam, xq, wq, U, ell=CORR_LEN):
    """psi_i(x) for the points x: (1/lam_i) sum_q w_q k(x, x_q) u_i(x_q) -> [m][len(x)]."""
    Kx = kernel_1d(np.asarray(x, dtype=np.float64), xq, ell)   # [len(x)][n]
    return (U * wq[None, :]) @ Kx.T / lam[:, None]


def term_pairs(lam_x, lam_y, n_terms=N_TERMS):
    """The n_terms (i, j) pairs with the largest lam_x[i] lam_y[j]."""
    cand = []
    for i in range(len(lam_x)):
        for j in range(len(lam_y)):
            cand.append((lam_x[i] * lam_y[j], i, j))
    cand.sort(key=lambda t: -t[0])
    top = cand[:n_terms + 8]
    # deterministic tie order: within relative 1e-9, by (i + j, i)
    out = []
    k = 0
    while k < len(top):
        grp = [top[k]]
        while k + len(grp) < len(top) and abs(top[k + len(grp)][0] - top[k][0]) <= 1e-9 * top[k][0]:
            grp.append(top[k + len(grp)])
        grp.sort(key=lambda t: (t[1] + t[2], t[1]))
        out += grp
        k += len(grp)
    return out[:n_terms]


class KLBasis:
    """The 2-D KL basis of the SE kernel on [0, Lx] x [0, Ly]."""

    def __init__(self, Lx=2.0, Ly=1.0, n_terms=N_TERMS, ell=CORR_LEN, n_quad=N_QUAD):
        self.ell = ell
        self.x1 = nystrom_1d(Lx, n_quad, ell)
        self.y1 = nystrom_1d(Ly, n_quad, ell)
        self.pairs = term_pairs(self.x1[0], self.y1[0], n_terms)
        self.lam = np.array([p[0] for p in self.pairs])

    def modes(self, xc, yc):
        """psi_k at the cell centres: [n_terms][len(yc)][len(xc)]."""
        px = eval_1d(xc, *self.x1, ell=self.ell)
        py = eval_1d(yc, *self.y1, ell=self.ell)
        return np.stack([py[j][:, None] * px[i][None, :] for _, i, j in self.pairs])

    def field(self, xc, yc, theta):
        """sum_k sqrt(lam_k) theta_k psi_k(x, y) on the (len(yc), len(xc)) grid."""
        M = self.modes(xc, yc)
        return np.tensordot(np.sqrt(self.lam) * np.asarray(theta, dtype=np.float64), M, axes=1)


_BASIS = {}


def default_basis(Lx=2.0, Ly=1.0):
    key = (Lx, Ly)
    if key not in _BASIS:
        _BASIS[key] = KLBasis(Lx, Ly)
    return _BASIS[key]


def coefficients_kl(prm, grid, inp, basis=None, sigma_logK=0.5, sigma_phi=0.1, phi_lo=0.05, phi_hi=0.65):
    """Per-cell phi and K fields and q_in for one sample of the random-field
    model; inp = (theta_K[32], theta_phi[32], xi3)."""
    from .henry import Coeffs
    basis = basis or default_basis(prm.Lx, prm.Ly)
    n = len(basis.pairs)
    inp = np.asarray(inp, dtype=complex if np.iscomplexobj(inp) else np.float64)
    xc = (np.arange(grid.nx) + 0.5) * grid.h
    yc = (np.arange(grid.ny) + 0.5) * grid.h
    M = basis.modes(xc, yc)
    sl = np.sqrt(basis.lam)
    gK = np.tensordot(sl * inp[:n], M, axes=1)
    gphi = np.tensordot(sl * inp[n:2 * n], M, axes=1)
    K = prm.K_mean * np.exp(sigma_logK * gK)
    phi = prm.phi_mean + sigma_phi * gphi
    if np.iscomplexobj(phi):  # complex-step derivatives: clip on the real part (derivative 0 when clipped)
        phi = np.where(phi.real < phi_lo, phi_lo, np.where(phi.real > phi_hi, phi_hi, phi))
    else:
        phi = np.clip(phi, phi_lo, phi_hi)
    qin = prm.qin_mean * (1.0 + prm.qin_amp * inp[2 * n])
    return Coeffs(phi=phi, K=K, qin=qin)
