"""Henry scenario solve with the paper's vertex-centred finite volumes, plain
FP64 (oracle; test infrastructure only).

The paper discretises Eqs. e_cont_eq and e_tran_eq with a vertex-centred
finite-volume scheme on quadrilaterals: two unknowns (p, c) per grid vertex,
so n_l = 2 (nx + 1)(ny + 1) degrees of freedom (Sec. 2.3 and Table
tab:adaptiveTS_times: 1122 at 32 x 16 elements), a "consistent velocity"
for Darcy's law and partial upwinding of the convective terms, implicit
Euler in time and Newton's method per step (Sec. 2.3).  The paper names
these ingredients and cites them; it does not write them out.  This module
fixes each one as follows, in the same coordinates as ``oracle.henry``
(x in [0, Lx], y in [0, Ly] pointing up; gravity -g e_y).

Grid and control volumes.  Vertices (j, i) at (i h, j h), i = 0..nx,
j = 0..ny; the elements are the squares of ``oracle.henry.Grid`` and carry
that module's per-element phi and K.  The control volume of a vertex is the
union of the quarter-squares of its elements (the dual "box" grid).  Inside
an element with corners v0 (bottom-left), v1 (bottom-right), v2 (top-left)
and v3 (top-right) and local coordinates (xi, eta) in [0, 1]^2, four
sub-control-volume faces of length h/2 join the element centre to the edge
midpoints:

    S_b: v0 -> v1, normal +e_x, integration point (1/2, 1/4)
    S_t: v2 -> v3, normal +e_x, integration point (1/2, 3/4)
    S_l: v0 -> v2, normal +e_y, integration point (1/4, 1/2)
    S_r: v1 -> v3, normal +e_y, integration point (3/4, 1/2)

Fields between vertices are bilinear; grad p and grad c at an integration
point are the gradients of the bilinear interpolants.

Consistent velocity (reading).  q.n = -(K_E / mu)(grad p . n + rho_g g n_y)
with the gravity density rho_g(xi) = (1 - xi)(rho_0 + rho_2)/2 +
xi (rho_1 + rho_3)/2: the mean density of each vertical element edge,
interpolated linearly in x.  A state in discrete hydrostatic balance along
the vertical edges, p_top - p_bottom = -g h (rho_top + rho_bottom)/2, then
has zero vertical Darcy flux at every integration point, whatever the
density field: the discrete gravity term is consistent with the discrete
pressure gradient, which is what the cited "consistent velocity" secures.

Fluxes.  Through a face from vertex a to vertex b: mass F = rho_ip (q.n) h/2
with rho_ip the bilinear density at the integration point; salt
G = F c_f - rho_ip phi_E Dm (grad c . n) h/2.

Partial upwind (reading).  c_f = (c_a + c_b)/2 + s sgn(F)(c_a - c_b)/2 with
s = max(0, 1 - rho_ip phi_E Dm / (2 |F|)): central differences where the
face Peclet number allows, and otherwise the smallest upwind share that
keeps each element's coupling coefficients of the salt equation
non-positive (on squares the bilinear diffusion couples a vertex to each of
the other three corners of an element with -rho phi Dm / 4).

Storage (lumped).  Fluid: sum_E phi_E h^2/4 (rho_v - rho_v^old)/tau; salt
the same with rho c.

Boundary conditions (Sec. 2.1).  x = Lx: the vertices carry the Dirichlet
values p = rho1 g (Ly - y), c = 1; x = 0: c = 0 at the vertices, and the
fluid equation of each vertex gains the inflow -rho0 q_in times its share
of the boundary (h, or h/2 at the corners); y = 0, Ly: no flux.  A
Dirichlet equation reads (value - boundary value) times the residual scale
(rho0 h^2/tau, with p measured in units of rho0 g Ly).

Initial state (reading).  c = 0 and fresh-water hydrostatic p, except at
the Dirichlet vertices, which hold their boundary values from t = 0.

QoIs.  Salt mass sum_v (sum_E phi_E h^2/4) rho_v c_v; c(1.5, 0.25) is the
value at that vertex (a grid vertex on every level).

Newton's Jacobian is the exact derivative of the residual by the complex
step (Squire and Trapp, SIAM Rev. 1998): the residual is written so that it
accepts complex states, and a 3 x 3 colouring of the vertices gives every
column from 18 residual evaluations.  The linear systems are solved by
scipy's sparse LU, so the discrete implicit-Euler solution is reached with
no multigrid.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import henry as cc

Params = cc.Params
Grid = cc.Grid

# Sub-control-volume faces: (a, b, normal, xi, eta), corners numbered
# 0 bottom-left, 1 bottom-right, 2 top-left, 3 top-right.
FACES = ((0, 1, "x", 0.5, 0.25), (2, 3, "x", 0.5, 0.75), (0, 2, "y", 0.25, 0.5), (1, 3, "y", 0.75, 0.5))
_CORNER = ((slice(None, -1), slice(None, -1)), (slice(None, -1), slice(1, None)),
           (slice(1, None), slice(None, -1)), (slice(1, None), slice(1, None)))


def n_dof(grid):
    """Two unknowns per vertex: n = 2 (nx + 1)(ny + 1)."""
    return 2 * (grid.nx + 1) * (grid.ny + 1)


def vertex_y(grid):
    return np.arange(grid.ny + 1) * grid.h


def initial_state(prm, grid):
    """c = 0 and p = rho0 g (Ly - y); the seaside column at its Dirichlet values."""
    y = vertex_y(grid)
    p = np.repeat((prm.rho0 * prm.g * (prm.Ly - y))[:, None], grid.nx + 1, axis=1)
    c = np.zeros((grid.ny + 1, grid.nx + 1))
    p[:, -1] = prm.rho1 * prm.g * (prm.Ly - y)
    c[:, -1] = 1.0
    return p, c


def density(prm, c):
    return prm.rho0 + (prm.rho1 - prm.rho0) * c


def storage_weights(grid, coef):
    """sum over a vertex's elements of phi_E h^2 / 4: the lumped phi |CV|."""
    w = np.zeros((grid.ny + 1, grid.nx + 1))
    for k in range(4):
        w[_CORNER[k]] += coef.phi
    return w * (grid.h * grid.h / 4.0)


def _corners(u):
    return [u[s] for s in _CORNER]


def face_fluxes(prm, grid, coef, p, c):
    """[(a, b, F, G)] for the four faces of every element: mass and salt
    fluxes from corner a to corner b, each an (ny, nx) array."""
    h = grid.h
    rho = density(prm, c)
    P, C, R = _corners(p), _corners(c), _corners(rho)
    out = []
    for a, b, normal, xi, eta in FACES:
        if normal == "x":
            dp = ((1 - eta) * (P[1] - P[0]) + eta * (P[3] - P[2])) / h
            dc = ((1 - eta) * (C[1] - C[0]) + eta * (C[3] - C[2])) / h
            grav = 0.0
        else:
            dp = ((1 - xi) * (P[2] - P[0]) + xi * (P[3] - P[1])) / h
            dc = ((1 - xi) * (C[2] - C[0]) + xi * (C[3] - C[1])) / h
            grav = ((1 - xi) * 0.5 * (R[0] + R[2]) + xi * 0.5 * (R[1] + R[3])) * prm.g
        qn = -(coef.K / prm.mu) * (dp + grav)
        rho_ip = (1 - xi) * (1 - eta) * R[0] + xi * (1 - eta) * R[1] + (1 - xi) * eta * R[2] + xi * eta * R[3]
        F = rho_ip * qn * (0.5 * h)
        Dc = rho_ip * coef.phi * prm.Dm
        pos = np.real(F) >= 0
        absF = np.where(pos, F, -F)
        upw = np.real(Dc) < 2.0 * np.real(absF)
        s = np.where(upw, 1.0 - Dc / (2.0 * np.where(upw, absF, 1.0)), 0.0)
        sg = np.where(pos, 1.0, -1.0)
        cf = 0.5 * (C[a] + C[b]) + 0.5 * s * sg * (C[a] - C[b])
        G = F * cf - Dc * dc * (0.5 * h)
        out.append((a, b, F, G))
    return out


def inflow_lengths(grid):
    """Each x = 0 vertex's share of the boundary: h, and h/2 at the corners."""
    L = np.full(grid.ny + 1, grid.h)
    L[0] = L[-1] = 0.5 * grid.h
    return L


def cv_areas(grid):
    """|CV| of every vertex: h^2 inside, h^2/2 on an edge, h^2/4 at a corner."""
    a = np.zeros((grid.ny + 1, grid.nx + 1))
    for k in range(4):
        a[_CORNER[k]] += 1.0
    return a * (grid.h * grid.h / 4.0)


def fv_residual(prm, grid, coef, p, c, p_old, c_old, inflow=True):
    """The finite-volume balances (R^m, R^s) of every vertex, (ny+1, nx+1)
    each, before the Dirichlet vertices' equations are replaced: storage
    plus outgoing face fluxes, plus (if ``inflow``) the inflow term at x = 0."""
    rho, rho_o = density(prm, c), density(prm, c_old)
    w = storage_weights(grid, coef)
    Rm = w * (rho - rho_o) / grid.tau
    Rs = w * (rho * c - rho_o * c_old) / grid.tau
    Rm = Rm + 0j if np.iscomplexobj(p) or np.iscomplexobj(c) else Rm
    Rs = Rs + 0j if np.iscomplexobj(Rm) else Rs
    for a, b, F, G in face_fluxes(prm, grid, coef, p, c):
        Rm[_CORNER[a]] += F
        Rm[_CORNER[b]] -= F
        Rs[_CORNER[a]] += G
        Rs[_CORNER[b]] -= G
    if inflow:
        Rm[:, 0] -= prm.rho0 * coef.qin * inflow_lengths(grid)
    return Rm, Rs


def residual_scale(prm, grid):
    return prm.rho0 * grid.h * grid.h / grid.tau


def residual(prm, grid, coef, p, c, p_old, c_old, src=None, dirichlet=None):
    """Newton's residual: the balances, with the Dirichlet vertices'
    equations replaced by (value - boundary value) x residual scale.

    For the manufactured-solution test only: ``src`` = vertex sources
    (S_m, S_s) in kg/(m^3 s), subtracted as S |CV|; ``dirichlet`` = vertex
    arrays (p_b, c_b) whose boundary entries replace the Henry boundary
    conditions by Dirichlet data for p and c on all four sides."""
    Rm, Rs = fv_residual(prm, grid, coef, p, c, p_old, c_old, inflow=dirichlet is None)
    s = residual_scale(prm, grid)
    pscale = prm.rho0 * prm.g * prm.Ly
    if src is not None:
        a = cv_areas(grid)
        Rm = Rm - src[0] * a
        Rs = Rs - src[1] * a
    if dirichlet is not None:
        edge = np.zeros((grid.ny + 1, grid.nx + 1), dtype=bool)
        edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
        Rm = np.where(edge, s * (p - dirichlet[0]) / pscale, Rm)
        Rs = np.where(edge, s * (c - dirichlet[1]), Rs)
        return Rm, Rs
    y = vertex_y(grid)
    Rm[:, -1] = s * (p[:, -1] - prm.rho1 * prm.g * (prm.Ly - y)) / pscale
    Rs[:, -1] = s * (c[:, -1] - 1.0)
    Rs[:, 0] = s * c[:, 0]
    return Rm, Rs


def pack(p, c):
    return np.stack([p.ravel(), c.ravel()], axis=1).ravel()


def unpack(v, grid):
    v = v.reshape(-1, 2)
    shape = (grid.ny + 1, grid.nx + 1)
    return v[:, 0].reshape(shape), v[:, 1].reshape(shape)


def jacobian(prm, grid, coef, p, c, p_old, c_old, src=None, dirichlet=None, step=1e-30):
    """d(R^m, R^s)/d(p, c) by the complex step: vertices coloured by (j mod 3,
    i mod 3) are perturbed together; a vertex couples only to the corners of
    its elements, so each row sees at most one perturbed vertex per colour."""
    ny1, nx1 = grid.ny + 1, grid.nx + 1
    J = np.arange(ny1)[:, None] + np.zeros((1, nx1), dtype=int)
    I = np.arange(nx1)[None, :] + np.zeros((ny1, 1), dtype=int)
    rows, cols, vals = [], [], []
    for var in (0, 1):
        for cj in range(3):
            for ci in range(3):
                mask = ((J % 3) == cj) & ((I % 3) == ci)
                pz = p.astype(complex)
                cz = c.astype(complex)
                if var == 0:
                    pz = pz + 1j * step * mask
                else:
                    cz = cz + 1j * step * mask
                Rm, Rs = residual(prm, grid, coef, pz, cz, p_old, c_old, src, dirichlet)
                dj = (cj - J) % 3
                di = (ci - I) % 3
                jp = J + np.where(dj == 2, -1, dj)
                ip = I + np.where(di == 2, -1, di)
                ok = (jp >= 0) & (jp < ny1) & (ip >= 0) & (ip < nx1)
                col = 2 * (jp * nx1 + ip) + var
                for eq, R in ((0, Rm), (1, Rs)):
                    d = R.imag / step
                    sel = ok & (d != 0)
                    rows.append((2 * (J * nx1 + I) + eq)[sel])
                    cols.append(col[sel])
                    vals.append(d[sel])
    n = 2 * ny1 * nx1
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def newton_step(prm, grid, coef, p_old, c_old, stats=None, src=None, dirichlet=None):
    """One implicit-Euler step by Newton's method with direct sparse solves;
    the stopping rule and the mass-fraction step limit of oracle.henry."""
    s = residual_scale(prm, grid)
    pref = prm.rho0 * prm.g * prm.Ly
    p, c = p_old.copy(), c_old.copy()
    for it in range(prm.newton_maxit):
        Rm, Rs = residual(prm, grid, coef, p, c, p_old, c_old, src, dirichlet)
        if max(np.abs(Rm).max(), np.abs(Rs).max()) / s <= prm.newton_atol:
            if stats is not None:
                stats.append(it)
            return p, c, True
        Jm = jacobian(prm, grid, coef, p, c, p_old, c_old, src, dirichlet)
        dp, dc = unpack(spla.spsolve(Jm.tocsc(), -pack(Rm, Rs)), grid)
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


def salt_mass(prm, grid, coef, c):
    return float(np.sum(storage_weights(grid, coef) * density(prm, c) * c))


def qoi(prm, grid, coef, p, c):
    """(salt mass, c at the vertex (1.5, 0.25))."""
    i = int(round(1.5 / grid.h))
    j = int(round(0.25 / grid.h))
    return salt_mass(prm, grid, coef, c), float(c[j, i])


def solve_scenario(prm, level, xi, return_state=False, stats=None, model="uniform3"):
    """All r_l steps of one scenario at MLMC level ``level``; returns the QoIs
    and a convergence flag (and the final state if asked)."""
    grid = Grid.level(prm, level)
    coef = cc.coefficient_model(model)(prm, grid, xi)
    p, c = initial_state(prm, grid)
    ok = True
    for _ in range(grid.steps):
        p, c, conv = newton_step(prm, grid, coef, p, c, stats=stats)
        ok = ok and conv
    q = qoi(prm, grid, coef, p, c)
    if return_state:
        return q, ok, (p, c)
    return q, ok
