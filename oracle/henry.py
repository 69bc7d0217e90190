"""Henry saltwater-intrusion scenario solve, plain FP64 (oracle; test infrastructure only).

What is computed, and where it comes from in arXiv 2302.07804:

* PDEs: fluid mass  d_t(phi rho) + div(rho q) = 0            (Eq. e_cont_eq)
        salt mass   d_t(phi rho c) + div(rho c q - rho D grad c) = 0   (Eq. e_tran_eq)
        Darcy       q = -(K/mu) (grad p - rho g),  g = (0, -g)        (Eq. e_Darcy_vel)
        density     rho(c) = rho0 + (rho1 - rho0) c, mu constant      (Eq. e_lin_density)
        dispersion  D = phi Dm I                                      (Eq. e_mol_diff)
  with isotropic K (Sec. 2.1).
* Boundary conditions (Sec. 2.1): seaside x = Lx: c = 1 and hydrostatic brine
  pressure; land side x = 0: c = 0 and a prescribed inflow of fresh water;
  top and bottom: no flux.  Initial state c = 0 (Sec. 2.1) with fresh-water
  hydrostatic pressure.
* Time: implicit Euler with a fixed step tau, r = T / tau steps; each step is
  solved by Newton's method (Sec. 2.3).  Here the Newton linear systems are
  solved directly (scipy's sparse LU), so the oracle reaches the discrete
  implicit-Euler solution without any multigrid.
* Space: the configuration solved here uses a cell-centred finite-volume
  discretisation with upwind advection on a uniform grid of square cells
  (the paper uses a vertex-centred scheme; the cell-centred reading is the
  one the solved configuration fixes).  Coordinates: x in [0, Lx], y in
  [0, Ly] pointing up, so the seaside pressure is rho1 g (Ly - y) (the paper's
  y in [-1, 0] shifted by +1).

Discrete equations (per cell P, volume V = h^2, face length h, every flux
outward from P, rho_P = rho(c_P)):

  R^m_P = phi_P (rho_P - rho_P^old) V / tau + sum_f F_f
  R^s_P = phi_P (rho_P c_P - rho_P^old c_P^old) V / tau + sum_f G_f

  interior face P|Nb:  rho_f = (rho_P + rho_Nb)/2,  K_f, (phi D)_f harmonic means
     horizontal: q_f = -(K_f/mu) (p_Nb - p_P)/h * s           (s = +1 east, -1 west)
     vertical:   q_f = -(K_f/mu) ((p_Nb - p_P)/h * s + rho_f g * s)   (s = +1 north, -1 south)
     F_f = rho_f q_f h
     G_f = F_f c_up - rho_f (phi D)_f (c_Nb - c_P)          c_up = c_P if F_f >= 0 else c_Nb
  x = 0:  F = -rho0 q_in h;  G = -rho_b (phi D)_P (0 - c_P) / (h/2) * h, rho_b = (rho_P + rho0)/2
  x = Lx: p_b = rho1 g (Ly - y_P), rho_b = (rho_P + rho1)/2,
          q = -(K_P/mu) (p_b - p_P)/(h/2),  F = rho_b q h,  c_up = c_P if F >= 0 else 1,
          G = F c_up - rho_b (phi D)_P (1 - c_P)/(h/2) * h
  y = 0, y = Ly: no flux.

Readings taken where the paper is silent (they match the CUDA path's):
the inflow q_in is a volumetric velocity into the domain (so rho q . n =
-rho0 q_in on x = 0); c = 0 at x = 0 acts on diffusion across a half cell;
face densities are arithmetic means and salt is upwinded by the sign of the
mass flux; the point QoI c(1.5, 0.25) is the mean of the four cells that meet
at that grid vertex.

Unknown ordering in the sparse Jacobian: index 2*cell + var, cell = iy*nx + ix,
var 0 = p, var 1 = c; equation 0 = fluid mass, 1 = salt mass.

``residual`` optionally adds manufactured sources and replaces the boundary
data by given functions; the manufactured-solution convergence test uses
this, the Henry solve never does.
"""
from dataclasses import dataclass, field, replace
import cmath
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass(frozen=True)
class Params:
    """Physics and discretisation constants in SI units (configuration values;
    the paper's Table tab:HenryParam lists 0.35, 18.8571e-6, 1.020408e-9, 9.8,
    1000, 1024.99, 1e-3)."""
    Lx: float = 2.0
    Ly: float = 1.0
    T: float = 7200.0
    rho0: float = 1000.0
    rho1: float = 1025.0
    mu: float = 1e-3
    g: float = 9.81
    Dm: float = 1.886e-5
    phi_mean: float = 0.35
    K_mean: float = 1.02e-9
    qin_mean: float = 6.6e-5
    phi_amp: float = 0.2
    logK_amp: float = 0.5
    qin_amp: float = 0.2
    nx0: int = 32
    ny0: int = 16
    steps0: int = 20
    # Newton stopping: scaled residual max-norm, scaled update max-norm, cap.
    newton_atol: float = 1e-11
    newton_dxtol: float = 1e-12
    newton_maxit: int = 30
    # a step that would change some mass fraction by more than this is scaled
    # down to it (0: full Newton steps)
    newton_dc_limit: float = 1.0


@dataclass(frozen=True)
class Grid:
    """Uniform grid of square cells at MLMC level ``level``: the spatial grid
    is refined regularly (cells x4 per level) and the time step halves
    (Sec. 2.3: tau_{l+1} = tau_l / 2, r_l = r_0 2^l)."""
    nx: int
    ny: int
    h: float
    tau: float
    steps: int

    @staticmethod
    def level(prm: Params, level: int) -> "Grid":
        nx = prm.nx0 << level
        ny = prm.ny0 << level
        steps = prm.steps0 << level
        return Grid(nx=nx, ny=ny, h=prm.Ly / ny, tau=prm.T / steps, steps=steps)

    @property
    def ncell(self):
        return self.nx * self.ny


@dataclass
class Coeffs:
    """Per-cell porosity and permeability fields and the scalar inflow."""
    phi: np.ndarray  # (ny, nx)
    K: np.ndarray    # (ny, nx)
    qin: float


def _exp(v):
    """exp of a real (libm) or complex (cmath) scalar: the coefficient models
    also accept complex inputs, for complex-step derivatives in the adjoint
    checks; real inputs take the same path as before."""
    return cmath.exp(v) if isinstance(v, complex) else math.exp(float(v))


def _scalar(v):
    return complex(v) if np.iscomplexobj(v) else float(v)


def coefficients(prm: Params, grid: Grid, xi) -> Coeffs:
    """Three-parameter random model of the solved configuration:
    phi = phi_mean (1 + phi_amp xi1), K = K_mean exp(logK_amp xi2),
    q_in = qin_mean (1 + qin_amp xi3), xi_i iid U[-1, 1] (the paper's model of
    Sec. 4 is a two-layer porosity field with Kozeny-Carman K; the configuration
    replaces it by these independent factors)."""
    xi1, xi2, xi3 = _scalar(xi[0]), _scalar(xi[1]), _scalar(xi[2])
    phi = prm.phi_mean * (1.0 + prm.phi_amp * xi1)
    K = prm.K_mean * _exp(prm.logK_amp * xi2)
    qin = prm.qin_mean * (1.0 + prm.qin_amp * xi3)
    shape = (grid.ny, grid.nx)
    return Coeffs(phi=np.full(shape, phi), K=np.full(shape, K), qin=qin)


def kozeny_carman_kappa(K_mean, phi_mean):
    """kappa_KC with K(E[phi]) = K_mean for K(phi) = kappa phi^3 / (1 - phi^2)
    (Eq. e_perm_Kozeny_Carman and the sentence after it)."""
    return K_mean * (1.0 - phi_mean ** 2) / phi_mean ** 3


def coefficients_two_layer(prm: Params, grid: Grid, xi) -> Coeffs:
    """The paper's random porosity, Eq. (poro_2levels): two horizontal layers,
    phi = phi_mean (1 + 0.15 (xi2 cos(pi x / 2) + xi2 sin(2 pi y) + xi1 cos(2 pi x))) C0(xi1),
    C0 = 1 + 0.2 xi1 below y = -0.75 and 1 - 0.2 xi1 above (paper coordinates,
    y in [-1, 0]: y_paper = y - Ly here), K = K(phi) by Kozeny-Carman, and the
    recharge q_in = qin_mean (1 + qin_amp xi3) (Sec. 4; xi2 appears twice and
    xi3 only in the recharge, as printed)."""
    xi1, xi2, xi3 = _scalar(xi[0]), _scalar(xi[1]), _scalar(xi[2])
    x = (np.arange(grid.nx) + 0.5) * grid.h
    yp = (np.arange(grid.ny) + 0.5) * grid.h - prm.Ly
    X, Y = np.meshgrid(x, yp)
    C0 = np.where(Y < -0.75, 1.0 + 0.2 * xi1, 1.0 - 0.2 * xi1)
    phi = prm.phi_mean * (1.0 + 0.15 * (xi2 * np.cos(np.pi * X / 2.0) + xi2 * np.sin(2.0 * np.pi * Y)
                                        + xi1 * np.cos(2.0 * np.pi * X))) * C0
    kappa = kozeny_carman_kappa(prm.K_mean, prm.phi_mean)
    K = kappa * phi ** 3 / (1.0 - phi ** 2)
    qin = prm.qin_mean * (1.0 + prm.qin_amp * xi3)
    return Coeffs(phi=phi, K=K, qin=qin)


def initial_state(prm: Params, grid: Grid):
    """c = 0 and fresh-water hydrostatic pressure p = rho0 g (Ly - y) at cell centres."""
    y = (np.arange(grid.ny) + 0.5) * grid.h
    p = np.repeat((prm.rho0 * prm.g * (prm.Ly - y))[:, None], grid.nx, axis=1)
    c = np.zeros((grid.ny, grid.nx))
    return p, c


def _harm(a, b):
    return 2.0 * a * b / (a + b)


@dataclass
class BoundaryData:
    """Boundary data; the defaults are the Henry problem's.  Each entry is a
    function of the face-centre coordinate along the boundary (y)."""
    left_mass_flux: object = None   # outward rho q.n on x=0, per unit length
    left_c: object = None           # Dirichlet c on x=0
    right_p: object = None          # Dirichlet p on x=Lx
    right_c: object = None          # Dirichlet c on x=Lx
    bottom_mass_flux: object = None  # outward rho q.n on y=0 (default 0)
    top_mass_flux: object = None     # outward rho q.n on y=Ly (default 0)
    bottom_salt_flux: object = None  # outward salt flux on y=0 (default 0)
    top_salt_flux: object = None


def residual(prm, grid, coef, p, c, p_old, c_old, src=None, bc=None):
    """Unscaled residuals (R^m, R^s), each (ny, nx), in kg / (m s) per unit depth.

    ``src`` = optional (S_m, S_s) volume sources in kg/(m^3 s), subtracted as
    S V; ``bc`` = optional BoundaryData (manufactured-solution tests only)."""
    h, tau = grid.h, grid.tau
    V = h * h
    drho = prm.rho1 - prm.rho0
    rho = prm.rho0 + drho * c
    rho_old = prm.rho0 + drho * c_old
    phi, K = coef.phi, coef.K
    PD = phi * prm.Dm

    Rm = phi * (rho - rho_old) * V / tau
    Rs = phi * (rho * c - rho_old * c_old) * V / tau

    # horizontal interior faces: L = [:, :-1], R = [:, 1:]
    Kf = _harm(K[:, :-1], K[:, 1:])
    PDf = _harm(PD[:, :-1], PD[:, 1:])
    rhof = 0.5 * (rho[:, :-1] + rho[:, 1:])
    q = -(Kf / prm.mu) * (p[:, 1:] - p[:, :-1]) / h
    F = rhof * q * h
    # upwind switches compare real parts (complex inputs: complex-step derivatives)
    cup = np.where(np.real(F) >= 0.0, c[:, :-1], c[:, 1:])
    G = F * cup - rhof * PDf * (c[:, 1:] - c[:, :-1])
    Rm[:, :-1] += F
    Rm[:, 1:] -= F
    Rs[:, :-1] += G
    Rs[:, 1:] -= G

    # vertical interior faces: B = [:-1, :], T = [1:, :]; flux from B up to T
    Kf = _harm(K[:-1, :], K[1:, :])
    PDf = _harm(PD[:-1, :], PD[1:, :])
    rhof = 0.5 * (rho[:-1, :] + rho[1:, :])
    q = -(Kf / prm.mu) * ((p[1:, :] - p[:-1, :]) / h + rhof * prm.g)
    F = rhof * q * h
    cup = np.where(np.real(F) >= 0.0, c[:-1, :], c[1:, :])
    G = F * cup - rhof * PDf * (c[1:, :] - c[:-1, :])
    Rm[:-1, :] += F
    Rm[1:, :] -= F
    Rs[:-1, :] += G
    Rs[1:, :] -= G

    yc = (np.arange(grid.ny) + 0.5) * h
    xc = (np.arange(grid.nx) + 0.5) * h

    # land side x = 0
    if bc is None or bc.left_mass_flux is None:
        Fl = np.full(grid.ny, -prm.rho0 * coef.qin * h)
    else:
        Fl = bc.left_mass_flux(yc) * h
    cl = np.zeros(grid.ny) if (bc is None or bc.left_c is None) else bc.left_c(yc)
    rhob = 0.5 * (rho[:, 0] + prm.rho0 + drho * cl)
    Rm[:, 0] += Fl
    # advective salt: inflow carries the boundary value, outflow the cell value
    cupl = np.where(np.real(Fl) >= 0.0, c[:, 0], cl)
    Rs[:, 0] += Fl * cupl - rhob * PD[:, 0] * (cl - c[:, 0]) / (0.5 * h) * h

    # seaside x = Lx
    pr = prm.rho1 * prm.g * (prm.Ly - yc) if (bc is None or bc.right_p is None) else bc.right_p(yc)
    cr = np.ones(grid.ny) if (bc is None or bc.right_c is None) else bc.right_c(yc)
    rhob = 0.5 * (rho[:, -1] + prm.rho0 + drho * cr)
    q = -(K[:, -1] / prm.mu) * (pr - p[:, -1]) / (0.5 * h)
    Fr = rhob * q * h
    cupr = np.where(np.real(Fr) >= 0.0, c[:, -1], cr)
    Rm[:, -1] += Fr
    Rs[:, -1] += Fr * cupr - rhob * PD[:, -1] * (cr - c[:, -1]) / (0.5 * h) * h

    # top / bottom: no flux for the Henry problem
    if bc is not None:
        if bc.bottom_mass_flux is not None:
            Rm[0, :] += bc.bottom_mass_flux(xc) * h
        if bc.top_mass_flux is not None:
            Rm[-1, :] += bc.top_mass_flux(xc) * h
        if bc.bottom_salt_flux is not None:
            Rs[0, :] += bc.bottom_salt_flux(xc) * h
        if bc.top_salt_flux is not None:
            Rs[-1, :] += bc.top_salt_flux(xc) * h

    if src is not None:
        Rm -= src[0] * V
        Rs -= src[1] * V
    return Rm, Rs


def jacobian(prm, grid, coef, p, c, p_old, c_old, bc=None):
    """Analytic Jacobian d(R^m, R^s)/d(p, c) of ``residual`` as a CSR matrix of
    size 2N x 2N (ordering in the module docstring).  Boundary data may depend
    on position but not on the unknowns."""
    nx, ny, h, tau = grid.nx, grid.ny, grid.h, grid.tau
    V = h * h
    drho = prm.rho1 - prm.rho0
    rho = prm.rho0 + drho * c
    phi, K = coef.phi, coef.K
    PD = phi * prm.Dm
    mu, g = prm.mu, prm.g
    cell = np.arange(nx * ny).reshape(ny, nx)
    rows, cols, vals = [], [], []

    def add(eq_cells, eq, var_cells, var, v):
        rows.append((2 * eq_cells + eq).ravel())
        cols.append((2 * var_cells + var).ravel())
        vals.append(np.broadcast_to(v, eq_cells.shape).ravel().astype(np.float64))

    # accumulation: d/dc of phi rho V/tau and phi rho c V/tau
    add(cell, 0, cell, 1, phi * drho * V / tau)
    add(cell, 1, cell, 1, phi * (drho * c + rho) * V / tau)

    def face(P, Nb, KP, KN, PDP, PDN, pP, pN, cP, cN, rhoP, rhoN, grav):
        """Derivatives of the flux (F, G) from P to Nb w.r.t. (p_P, c_P, p_Nb, c_Nb);
        ``grav`` = g for an upward face (Nb above P), 0 for a horizontal one."""
        Kf = _harm(KP, KN)
        PDf = _harm(PDP, PDN)
        rhof = 0.5 * (rhoP + rhoN)
        q = -(Kf / mu) * ((pN - pP) / h + rhof * grav)
        F = rhof * q * h
        upP = F >= 0.0
        cup = np.where(upP, cP, cN)
        dq_dc = -(Kf / mu) * 0.5 * drho * grav      # same for c_P and c_Nb
        dF_dpP = rhof * (Kf / mu)                    # rho_f * (K/(mu h)) * h
        dF_dpN = -dF_dpP
        dF_dc = 0.5 * drho * q * h + rhof * dq_dc * h
        dif = PDf * (cN - cP)                         # (phi D)_f (c_N - c_P)
        dG_dpP = dF_dpP * cup
        dG_dpN = dF_dpN * cup
        dG_dcP = dF_dc * cup + np.where(upP, F, 0.0) - (0.5 * drho * dif - rhof * PDf)
        dG_dcN = dF_dc * cup + np.where(upP, 0.0, F) - (0.5 * drho * dif + rhof * PDf)
        # residual of P gains +flux, residual of Nb gains -flux
        for sgn, E in ((1.0, P), (-1.0, Nb)):
            add(E, 0, P, 0, sgn * dF_dpP)
            add(E, 0, Nb, 0, sgn * dF_dpN)
            add(E, 0, P, 1, sgn * dF_dc)
            add(E, 0, Nb, 1, sgn * dF_dc)
            add(E, 1, P, 0, sgn * dG_dpP)
            add(E, 1, Nb, 0, sgn * dG_dpN)
            add(E, 1, P, 1, sgn * dG_dcP)
            add(E, 1, Nb, 1, sgn * dG_dcN)

    face(cell[:, :-1], cell[:, 1:], K[:, :-1], K[:, 1:], PD[:, :-1], PD[:, 1:],
         p[:, :-1], p[:, 1:], c[:, :-1], c[:, 1:], rho[:, :-1], rho[:, 1:], 0.0)
    face(cell[:-1, :], cell[1:, :], K[:-1, :], K[1:, :], PD[:-1, :], PD[1:, :],
         p[:-1, :], p[1:, :], c[:-1, :], c[1:, :], rho[:-1, :], rho[1:, :], g)

    yc = (np.arange(ny) + 0.5) * h
    # land side: mass flux fixed; salt = advective (fixed flux times upwind value) + diffusive
    L = cell[:, 0]
    if bc is None or bc.left_mass_flux is None:
        Fl = np.full(ny, -prm.rho0 * coef.qin * h)
    else:
        Fl = bc.left_mass_flux(yc) * h
    cl = np.zeros(ny) if (bc is None or bc.left_c is None) else bc.left_c(yc)
    rhob = 0.5 * (rho[:, 0] + prm.rho0 + drho * cl)
    difl = PD[:, 0] * (cl - c[:, 0]) * 2.0           # (phi D)(c_b - c_P)/(h/2)*h
    dGl = np.where(Fl >= 0.0, Fl, 0.0) - (0.5 * drho * difl - rhob * PD[:, 0] * 2.0)
    add(L, 1, L, 1, dGl)

    # seaside
    R = cell[:, -1]
    pr = prm.rho1 * g * (prm.Ly - yc) if (bc is None or bc.right_p is None) else bc.right_p(yc)
    cr = np.ones(ny) if (bc is None or bc.right_c is None) else bc.right_c(yc)
    rhob = 0.5 * (rho[:, -1] + prm.rho0 + drho * cr)
    KP = K[:, -1]
    q = -(KP / mu) * (pr - p[:, -1]) / (0.5 * h)
    F = rhob * q * h
    upP = F >= 0.0
    cup = np.where(upP, c[:, -1], cr)
    dF_dp = rhob * (KP / mu) * 2.0
    dF_dc = 0.5 * drho * q * h
    difr = PD[:, -1] * (cr - c[:, -1]) * 2.0
    add(R, 0, R, 0, dF_dp)
    add(R, 0, R, 1, dF_dc)
    add(R, 1, R, 0, dF_dp * cup)
    add(R, 1, R, 1, dF_dc * cup + np.where(upP, F, 0.0) - (0.5 * drho * difr - rhob * PD[:, -1] * 2.0))

    n = 2 * nx * ny
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    J.sum_duplicates()
    return J


def residual_scale(prm, grid):
    """Newton scales both residuals by rho0 V / tau (kg per cell per step)."""
    return prm.rho0 * grid.h * grid.h / grid.tau


def pack(p, c):
    """(ny, nx) fields -> interleaved vector, index 2*cell + var."""
    return np.stack([p.ravel(), c.ravel()], axis=1).ravel()


def unpack(v, grid):
    v = v.reshape(-1, 2)
    return v[:, 0].reshape(grid.ny, grid.nx), v[:, 1].reshape(grid.ny, grid.nx)


def newton_step(prm, grid, coef, p_old, c_old, src=None, bc=None, linsolve=None, stats=None):
    """One implicit-Euler step: Newton's method from the old state (Sec. 2.3)
    with a direct sparse solve of each linear system.

    Stops when the scaled residual max-norm is <= newton_atol, or right after
    an update whose scaled max-norm (p in units of rho0 g Ly) is <=
    newton_dxtol.  A step whose largest mass-fraction change exceeds
    newton_dc_limit is scaled down to it (c lies in [0, 1], so such a step
    overshoots; near convergence the steps are full Newton steps and the
    root is the same).  Returns (p, c, converged)."""
    s = residual_scale(prm, grid)
    pref = prm.rho0 * prm.g * prm.Ly
    p, c = p_old.copy(), c_old.copy()
    solve = linsolve or (lambda J, b: spla.spsolve(J.tocsc(), b))
    for it in range(prm.newton_maxit):
        Rm, Rs = residual(prm, grid, coef, p, c, p_old, c_old, src, bc)
        rnorm = max(np.abs(Rm).max(), np.abs(Rs).max()) / s
        if rnorm <= prm.newton_atol:
            if stats is not None:
                stats.append(it)
            return p, c, True
        J = jacobian(prm, grid, coef, p, c, p_old, c_old, bc)
        dx = solve(J, -pack(Rm, Rs))
        dp, dc = unpack(dx, grid)
        dcmax = np.abs(dc).max()
        theta = prm.newton_dc_limit / dcmax if (prm.newton_dc_limit > 0 and dcmax > prm.newton_dc_limit) else 1.0
        p = p + theta * dp
        c = c + theta * dc
        if max(np.abs(dp).max() / pref, dcmax) <= prm.newton_dxtol:
            if stats is not None:
                stats.append(it + 1)
            return p, c, True
    if stats is not None:
        stats.append(prm.newton_maxit)
    return p, c, False


def qoi(prm, grid, coef, p, c):
    """QoIs at the final time: total salt mass sum_P phi_P rho_P c_P h^2 (kg per
    metre of depth) and c at (1.5, 0.25), the mean of the four cells meeting at
    that vertex (the configuration's point; the paper's points are Eq. 12points)."""
    rho = prm.rho0 + (prm.rho1 - prm.rho0) * c
    mass = _scalar(np.sum(coef.phi * rho * c) * grid.h * grid.h)
    ix = int(round(1.5 / grid.h))
    iy = int(round(0.25 / grid.h))
    cpt = _scalar(0.25 * (c[iy - 1, ix - 1] + c[iy - 1, ix] + c[iy, ix - 1] + c[iy, ix]))
    return mass, cpt


# The paper's 12 observation points, Eq. (12points), in its coordinates
# (x in [0, 2], y in [-1, 0]); y here is y_paper + Ly.
POINTS_12 = [(x, y) for y in (-0.95, -0.75, -0.50) for x in (1.10, 1.35, 1.60, 1.85)]
C_FRESH = 0.012178  # Eq. (integral_fw): fresh water where c <= 0.012178


def point_value(prm, grid, c, x, y):
    """c at (x, y) (this domain's coordinates) by bilinear interpolation of
    the four surrounding cell-centre values (clamped stencil)."""
    tx = x * grid.nx / prm.Lx - 0.5
    ty = y * grid.ny / prm.Ly - 0.5
    # the 2 x 2 stencil stays on the grid: a point outside the hull of the cell
    # centres (only on coarse grids) is extrapolated linearly
    ix = min(max(int(math.floor(tx)), 0), grid.nx - 2)
    iy = min(max(int(math.floor(ty)), 0), grid.ny - 2)
    fx, fy = tx - ix, ty - iy
    return ((1 - fy) * ((1 - fx) * c[iy, ix] + fx * c[iy, ix + 1])
            + fy * ((1 - fx) * c[iy + 1, ix] + fx * c[iy + 1, ix + 1]))


def freshwater_area(grid, c):
    """Eq. (integral_fw) by the midpoint rule: the area of the cells whose
    mass fraction is at most 0.012178."""
    return float(np.count_nonzero(c <= C_FRESH)) * grid.h * grid.h


def field_level0(prm, grid, c):
    """c averaged over the cells of the level-0 grid (nx0 x ny0), row-major."""
    f = grid.nx // prm.nx0
    return c.reshape(prm.ny0, f, prm.nx0, f).mean(axis=(1, 3)).ravel()


def series_stride(prm, grid):
    """Fine steps per level-0 step (2^l at level l)."""
    return grid.steps // prm.steps0


def qoi_paper(prm, grid, coef, p, c, field=False):
    """The paper's QoIs at T (Sec. 2.2 and 4): salt mass and c(1.5, 0.25) as in
    ``qoi``, the freshwater integral Q_FW, c at the 12 points of Eq. (12points)
    and, with ``field``, the c field averaged to the level-0 grid (whose MLMC
    mean and variance are the paper's mean and variance fields)."""
    mass, cpt = qoi(prm, grid, coef, p, c)
    out = [mass, cpt, freshwater_area(grid, c)]
    out += [float(point_value(prm, grid, c, x, y + prm.Ly)) for x, y in POINTS_12]
    if field:
        out += list(field_level0(prm, grid, c))
    return np.array(out)


def paper_params(**kw):
    """The paper's variant of the problem (Table tab:HenryParam, Sec. 4):
    g = 9.8, rho1 = 1024.99, Dm = 18.8571e-6, K = 1.020408e-9, recharge
    amplitude 0.5, T = 6016 s in 188 steps at level 0 (tau = 32 s); used with
    the two-layer porosity model."""
    base = dict(g=9.8, rho1=1024.99, Dm=18.8571e-6, K_mean=1.020408e-9, qin_amp=0.5, T=6016.0, steps0=188)
    base.update(kw)
    return Params(**base)


def coefficient_model(model):
    """'uniform3' (default), 'kl' (oracle.kl) or 'two_layer'."""
    if model == "uniform3":
        return coefficients
    if model == "two_layer":
        return coefficients_two_layer
    if model == "kl":
        from . import kl
        return kl.coefficients_kl
    raise ValueError(model)


def solve_scenario(prm, level, xi, return_state=False, stats=None, model="uniform3", qoi_set=0):
    """All r_l implicit-Euler steps of one scenario at MLMC level ``level`` for
    random input ``xi``; returns the QoIs ((mass, c_point) for qoi_set 0,
    ``qoi_paper`` for 1, with the level-0 field for 2, with the freshwater
    integral after every level-0 time step for 3) and a convergence flag."""
    grid = Grid.level(prm, level)
    coef = coefficient_model(model)(prm, grid, xi)
    p, c = initial_state(prm, grid)
    ok = True
    series = []
    for n in range(grid.steps):
        p, c, conv = newton_step(prm, grid, coef, p, c, stats=stats)
        ok = ok and conv
        if qoi_set == 3 and (n + 1) % series_stride(prm, grid) == 0:
            series.append(freshwater_area(grid, c))  # Q_FW at the level-0 step times (Sec. 4)
    q = qoi(prm, grid, coef, p, c) if qoi_set == 0 else qoi_paper(prm, grid, coef, p, c, field=qoi_set == 2)
    if qoi_set == 3:
        q = np.concatenate([q, series])
    if return_state:
        return q, ok, (p, c)
    return q, ok


def solve_scenarios(prm, level, xis, stats=None, model="uniform3", qoi_set=0):
    """Sequential loop over samples: returns q[n][n_qoi] and ok[n]."""
    xis = np.asarray(xis, dtype=np.float64)
    rows, ok = [], np.empty(xis.shape[0], dtype=bool)
    for i, xi in enumerate(xis):
        q, o = solve_scenario(prm, level, xi, stats=stats, model=model, qoi_set=qoi_set)
        rows.append(np.asarray(q, dtype=np.float64))
        ok[i] = o
    return np.array(rows).reshape(xis.shape[0], -1), ok


def _solve_one(args):
    prm, level, xi = args
    q, ok = solve_scenario(prm, level, xi)
    return q, ok


def solve_scenarios_pool(prm, level, xis, processes):
    """Same as ``solve_scenarios`` with one sample per worker of a spawn-context
    process pool (spawn: safe after the parent has touched a GPU)."""
    import multiprocessing as mp
    xis = np.asarray(xis, dtype=np.float64)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes) as pool:
        res = pool.map(_solve_one, [(prm, level, xi) for xi in xis])
    out = np.array([r[0] for r in res], dtype=np.float64).reshape(-1, 2)
    ok = np.array([r[1] for r in res], dtype=bool)
    return out, ok
