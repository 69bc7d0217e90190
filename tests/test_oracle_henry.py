"""Pins of the oracle's Henry-problem solve against facts fixed by mathematics.

Each test pins a different part, so that a dropped term, a wrong sign or a
wrong index in ``oracle.henry`` fails at least one of them:

* Jacobian vs central differences of the residual            (analytic J)
* constant-density limit: closed-form pressure, and c equal to the
  one-dimensional implicit upwind scheme solved by the Thomas algorithm
  (boundary fluxes, advection, diffusion, accumulation)
* manufactured solution: observed order of convergence ~1 in (h, tau) jointly
  (all terms incl. gravity and density coupling); planted parameter
  mismatches make the order collapse
* bounds 0 <= c <= 1, discrete salt-mass conservation
* Newton with a brute-force finite-difference Jacobian and a dense solve
  reaches the same state (the solution is the root of the residual)
* mistakes planted in the oracle's source each fail one of the above
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import henry, philox
from paper_2302_07804_gb300 import inputs

PRM = henry.Params()


def _tiny(nx=8, ny=4, tau=90.0):
    return henry.Grid(nx=nx, ny=ny, h=PRM.Ly / ny, tau=tau, steps=1)


def _fd_jacobian(prm, grid, coef, p, c, po, co, eps_p=1e-3, eps_c=1e-7, bc=None):
    n = grid.ncell
    x0 = henry.pack(p, c)
    J = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        e = eps_p if j % 2 == 0 else eps_c
        xp = x0.copy()
        xm = x0.copy()
        xp[j] += e
        xm[j] -= e
        Rp = henry.pack(*henry.residual(prm, grid, coef, *henry.unpack(xp, grid), po, co, bc=bc))
        Rm = henry.pack(*henry.residual(prm, grid, coef, *henry.unpack(xm, grid), po, co, bc=bc))
        J[:, j] = (Rp - Rm) / (2 * e)
    return J


def _fluxes_away_from_zero(prm, grid, coef, p, c):
    """True when no face mass flux is so close to 0 that a finite-difference
    probe could flip its upwind direction."""
    rho = prm.rho0 + (prm.rho1 - prm.rho0) * c
    K = coef.K[0, 0]
    qh = -(K / prm.mu) * (p[:, 1:] - p[:, :-1]) / grid.h
    qv = -(K / prm.mu) * ((p[1:, :] - p[:-1, :]) / grid.h + 0.5 * (rho[1:, :] + rho[:-1, :]) * prm.g)
    return min(np.abs(qh).min(), np.abs(qv).min()) > 1e-9


@pytest.mark.parametrize("tag", [1, 2, 3])
def test_jacobian_matches_central_differences(tag):
    grid = _tiny()
    xi = inputs.uniform_xi(tag, 1)[0]
    coef = henry.coefficients(PRM, grid, xi)
    p, c = inputs.random_states(tag, 2, grid.ny, grid.nx, p_top=5e3, p_bottom=1e4, dp=400.0)
    assert _fluxes_away_from_zero(PRM, grid, coef, p[0], c[0])
    J = henry.jacobian(PRM, grid, coef, p[0], c[0], p[1], c[1]).toarray()
    Jfd = _fd_jacobian(PRM, grid, coef, p[0], c[0], p[1], c[1])
    scale = np.abs(J).max(axis=1, keepdims=True)
    assert np.abs(J - Jfd).max() / 1.0 <= 1e-6 * scale.max()
    np.testing.assert_allclose(J, Jfd, rtol=1e-5, atol=1e-7 * scale.max())


def test_jacobian_is_five_point_block_stencil():
    grid = _tiny()
    coef = henry.coefficients(PRM, grid, [0.1, -0.2, 0.3])
    p, c = inputs.random_states(7, 2, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    J = henry.jacobian(PRM, grid, coef, p[0], c[0], p[1], c[1]).tocoo()
    P, Q = J.row // 2, J.col // 2
    dy = Q // grid.nx - P // grid.nx
    dx = Q % grid.nx - P % grid.nx
    assert np.all(np.abs(dx) + np.abs(dy) <= 1)


def _thomas(a, b, c, d):
    """Tridiagonal solve, sub-diagonal a, diagonal b, super-diagonal c."""
    n = len(b)
    cp = np.zeros(n)
    dp = np.zeros(n)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        m = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / m if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m
    x = np.zeros(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def _one_d_step(c_old, phi, Dm, rho, q, h, tau):
    """Implicit Euler step of the 1-D upwind advection-diffusion scheme for
    rho phi c_t + (rho q c - rho phi Dm c_x)_x = 0 on n cells of width h (the
    y-independent problem per unit depth), with c = 0 across a half cell at
    the inflow x = 0 (where the flow carries no salt) and c = 1 across a half
    cell at the outflow x = Lx."""
    n = len(c_old)
    acc = phi * rho * h * h / tau
    u = rho * q * h
    d = rho * phi * Dm
    lo = np.full(n, -u - d)
    di = np.full(n, acc + u + 2 * d)
    up = np.full(n, -d)
    rhs = acc * c_old.copy()
    di[0] = acc + u + 3 * d
    di[-1] = acc + u + 3 * d
    rhs[-1] += 2 * d
    lo[0] = 0.0
    return _thomas(lo, di, up, rhs)


@pytest.mark.parametrize("qin", [6.6e-5, 0.0])
def test_constant_density_limit(qin):
    prm = henry.Params(rho1=1000.0)
    grid = henry.Grid.level(prm, 0)
    coef = henry.coefficients(prm, grid, [0.3, -0.4, 0.0])
    coef.qin = qin
    phi, K = coef.phi[0, 0], coef.K[0, 0]
    p, c = henry.initial_state(prm, grid)
    c1d = np.zeros(grid.nx)
    x = (np.arange(grid.nx) + 0.5) * grid.h
    y = (np.arange(grid.ny) + 0.5) * grid.h
    p_exact = prm.rho0 * prm.g * (prm.Ly - y)[:, None] + prm.mu * qin * (prm.Lx - x)[None, :] / K
    for _ in range(6):
        p, c, ok = henry.newton_step(prm, grid, coef, p, c)
        assert ok
        c1d = _one_d_step(c1d, phi, prm.Dm, prm.rho0, qin, grid.h, grid.tau)
        np.testing.assert_allclose(p, p_exact, rtol=1e-11, atol=1e-9)
        np.testing.assert_allclose(c, np.broadcast_to(c1d, c.shape), rtol=0, atol=1e-11)
    assert c.max() > 1e-3  # salt did enter


def _mms_errors(levels, prm_disc, T_end=600.0, steps0=4, K=2e-10, phi=0.35):
    """Max errors (c, p) at t = T_end of the discrete solution with sources and
    boundary data derived by sympy from a manufactured (p, c), using the
    physics of PRM, while the discrete scheme runs with ``prm_disc``."""
    sy = pytest.importorskip("sympy")
    x, y, t = sy.symbols("x y t")
    rho0, rho1, mu, g, Dm = PRM.rho0, PRM.rho1, PRM.mu, PRM.g, PRM.Dm
    c_ex = 0.5 + 0.3 * sy.sin(sy.pi * x / 2 + 0.3) * sy.cos(sy.pi * y) * sy.exp(-t / 3600)
    p_ex = rho0 * g * (1 - y) + 60 * (2 - x) + 30 * sy.cos(sy.pi * x / 2) * sy.cos(sy.pi * y) * (1 + t / 3600)
    rho = rho0 + (rho1 - rho0) * c_ex
    qx = -(K / mu) * sy.diff(p_ex, x)
    qy = -(K / mu) * (sy.diff(p_ex, y) + rho * g)
    fsx = rho * c_ex * qx - rho * phi * Dm * sy.diff(c_ex, x)
    fsy = rho * c_ex * qy - rho * phi * Dm * sy.diff(c_ex, y)
    Sm = sy.diff(phi * rho, t) + sy.diff(rho * qx, x) + sy.diff(rho * qy, y)
    Ss = sy.diff(phi * rho * c_ex, t) + sy.diff(fsx, x) + sy.diff(fsy, y)
    L = lambda e: sy.lambdify((x, y, t), e, "numpy")
    fSm, fSs, fc, fp, fmx, fmy, fsy_ = map(L, (Sm, Ss, c_ex, p_ex, rho * qx, rho * qy, fsy))
    out = []
    for lev in levels:
        gl = henry.Grid.level(prm_disc, lev)
        steps = steps0 << lev
        grid = henry.Grid(gl.nx, gl.ny, gl.h, T_end / steps, steps)
        shape = (grid.ny, grid.nx)
        coef = henry.Coeffs(phi=np.full(shape, phi), K=np.full(shape, K), qin=0.0)
        X, Y = np.meshgrid((np.arange(grid.nx) + 0.5) * grid.h, (np.arange(grid.ny) + 0.5) * grid.h)
        full = lambda f, a, b, tt: f(a, b, tt) + 0.0 * (a + b)
        p, c = full(fp, X, Y, 0.0), full(fc, X, Y, 0.0)
        for n in range(steps):
            tn = (n + 1) * grid.tau
            bc = henry.BoundaryData(
                left_mass_flux=lambda yy, tn=tn: -full(fmx, 0.0 * yy, yy, tn),
                left_c=lambda yy, tn=tn: full(fc, 0.0 * yy, yy, tn),
                right_p=lambda yy, tn=tn: full(fp, 2.0 + 0.0 * yy, yy, tn),
                right_c=lambda yy, tn=tn: full(fc, 2.0 + 0.0 * yy, yy, tn),
                bottom_mass_flux=lambda xx, tn=tn: -full(fmy, xx, 0.0 * xx, tn),
                top_mass_flux=lambda xx, tn=tn: full(fmy, xx, 1.0 + 0.0 * xx, tn),
                bottom_salt_flux=lambda xx, tn=tn: -full(fsy_, xx, 0.0 * xx, tn),
                top_salt_flux=lambda xx, tn=tn: full(fsy_, xx, 1.0 + 0.0 * xx, tn))
            src = (full(fSm, X, Y, tn), full(fSs, X, Y, tn))
            p, c, ok = henry.newton_step(prm_disc, grid, coef, p, c, src=src, bc=bc)
            assert ok
        out.append((np.abs(c - full(fc, X, Y, T_end)).max(), np.abs(p - full(fp, X, Y, T_end)).max()))
    return np.array(out)


def test_manufactured_solution_first_order():
    e = _mms_errors([0, 1, 2], PRM)
    order_c = np.log2(e[:-1, 0] / e[1:, 0])
    order_p = np.log2(e[:-1, 1] / e[1:, 1])
    # upwind advection + implicit Euler: first order (Sec. 2.3); pressure converges faster
    assert np.all(order_c > 0.75), order_c
    assert order_c[-1] > 0.85, order_c
    assert np.all(order_p > 1.2), order_p


@pytest.mark.parametrize("mutation", [dict(g=-9.81), dict(rho1=1000.0), dict(Dm=2 * 1.886e-5), dict(mu=0.5e-3)])
def test_manufactured_solution_detects_planted_mistake(mutation):
    """Running the scheme with a wrong constant (as a sign slip or a dropped
    term would) must destroy convergence to the manufactured solution."""
    good = _mms_errors([1, 2], PRM)
    bad = _mms_errors([1, 2], henry.Params(**mutation))
    assert bad[1, 0] > 3 * good[1, 0] or bad[1, 1] > 3 * good[1, 1]
    assert bad[1, 0] > 0.6 * bad[0, 0] or bad[1, 1] > 0.6 * bad[0, 1]


def test_bounds_and_salt_conservation():
    grid = henry.Grid.level(PRM, 0)
    for xi in philox.sample_xi(inputs.SEED, 0, 100, 3):
        coef = henry.coefficients(PRM, grid, xi)
        p, c = henry.initial_state(PRM, grid)
        for _ in range(grid.steps):
            po, co = p, c
            p, c, ok = henry.newton_step(PRM, grid, coef, po, co)
            assert ok
            assert c.min() >= -1e-10 and c.max() <= 1 + 1e-10
            # interior face fluxes cancel in the sum: the change of total salt
            # equals minus tau times the net outflow through x = 0 and x = Lx
            rho = PRM.rho0 + (PRM.rho1 - PRM.rho0) * c
            rho_o = PRM.rho0 + (PRM.rho1 - PRM.rho0) * co
            dM = np.sum(coef.phi * (rho * c - rho_o * co)) * grid.h ** 2
            phiD = coef.phi[0, 0] * PRM.Dm
            yc = (np.arange(grid.ny) + 0.5) * grid.h
            out_left = np.sum(0.5 * (rho[:, 0] + PRM.rho0) * phiD * c[:, 0] * 2.0)
            pb = PRM.rho1 * PRM.g * (PRM.Ly - yc)
            qr = -(coef.K[:, -1] / PRM.mu) * (pb - p[:, -1]) / (0.5 * grid.h)
            rb = 0.5 * (rho[:, -1] + PRM.rho1)
            Fr = rb * qr * grid.h
            out_right = np.sum(Fr * np.where(Fr >= 0, c[:, -1], 1.0) - rb * phiD * (1 - c[:, -1]) * 2.0)
            scale = PRM.rho0 * grid.h ** 2
            assert abs(dM + grid.tau * (out_left + out_right)) <= 1e-9 * scale * grid.ncell


def test_newton_with_finite_difference_jacobian_reaches_same_state():
    grid = _tiny(nx=8, ny=4, tau=300.0)
    coef = henry.coefficients(PRM, grid, [-0.3, 0.5, 0.2])
    p0, c0 = henry.initial_state(PRM, grid)
    p_a, c_a, ok = henry.newton_step(PRM, grid, coef, p0, c0)
    assert ok
    # brute force: dense FD Jacobian and numpy's dense solver
    p, c = p0.copy(), c0.copy()
    for _ in range(40):
        R = henry.pack(*henry.residual(PRM, grid, coef, p, c, p0, c0))
        J = _fd_jacobian(PRM, grid, coef, p, c, p0, c0, eps_p=1e-4, eps_c=1e-8)
        dx = np.linalg.solve(J, -R)
        dp, dc = henry.unpack(dx, grid)
        p, c = p + dp, c + dc
        if np.abs(dc).max() < 1e-13 and np.abs(dp).max() < 1e-9:
            break
    np.testing.assert_allclose(c, c_a, atol=1e-11)
    np.testing.assert_allclose(p, p_a, rtol=1e-12, atol=1e-8)


def test_qoi_point_is_mean_of_four_cells_at_vertex():
    for lev in (0, 1, 2):
        grid = henry.Grid.level(PRM, lev)
        coef = henry.coefficients(PRM, grid, [0, 0, 0])
        c = np.zeros((grid.ny, grid.nx))
        # cells whose centres are at distance h/2 from (1.5, 0.25) in x and y
        xc = (np.arange(grid.nx) + 0.5) * grid.h
        yc = (np.arange(grid.ny) + 0.5) * grid.h
        sel = (np.abs(np.abs(xc - 1.5) - grid.h / 2) < 1e-12)[None, :] & \
              (np.abs(np.abs(yc - 0.25) - grid.h / 2) < 1e-12)[:, None]
        assert sel.sum() == 4
        c[sel] = [0.1, 0.2, 0.3, 0.6]
        mass, cpt = henry.qoi(PRM, grid, coef, np.zeros_like(c), c)
        assert cpt == pytest.approx(0.3, abs=1e-15)
        phi = coef.phi[0, 0]
        rho = PRM.rho0 + (PRM.rho1 - PRM.rho0) * c
        assert mass == pytest.approx(float(np.sum(phi * rho * c)) * grid.h ** 2, rel=1e-14)


def test_salt_mass_closed_forms():
    """The salt-mass QoI against closed forms, not against its own formula.
    For uniform c the mass is phi rho(c) c Lx Ly.  For c = x / Lx the cell
    sum is the midpoint rule of a quadratic in x: the exact integral
    phi Ly Lx (rho0 / 2 + drho / 3) less phi Ly h^2 / 24 times the integral
    of the second derivative, 2 drho / Lx."""
    drho = PRM.rho1 - PRM.rho0
    for lev in (0, 2):
        grid = henry.Grid.level(PRM, lev)
        coef = henry.coefficients(PRM, grid, [0.4, -0.7, 0.1])
        phi = float(coef.phi[0, 0])
        area = PRM.Lx * PRM.Ly
        for cu in (0.0, 0.5, 1.0):
            c = np.full((grid.ny, grid.nx), cu)
            mass, _ = henry.qoi(PRM, grid, coef, np.zeros_like(c), c)
            assert mass == pytest.approx(phi * (PRM.rho0 + drho * cu) * cu * area, rel=1e-13, abs=1e-300)
        xc = (np.arange(grid.nx) + 0.5) * grid.h
        c = np.broadcast_to(xc / PRM.Lx, (grid.ny, grid.nx)).copy()
        mass, _ = henry.qoi(PRM, grid, coef, np.zeros_like(c), c)
        exact = phi * PRM.Ly * (PRM.Lx * (PRM.rho0 / 2 + drho / 3) - grid.h ** 2 / 24 * 2 * drho / PRM.Lx)
        assert mass == pytest.approx(exact, rel=1e-13)


def test_three_parameter_coefficients_ranges_and_separation():
    """The three-parameter model at the corners of [-1, 1]^3: the ranges the
    configuration states (phi in [0.28, 0.42], K in 1.02e-9 [e^-0.5, e^0.5],
    q_in in [5.28e-5, 7.92e-5]), means at xi = 0, each coefficient moved by
    its own xi component only, and log K affine in xi2."""
    grid = henry.Grid.level(PRM, 0)
    c0 = henry.coefficients(PRM, grid, [0.0, 0.0, 0.0])
    assert (c0.phi == 0.35).all() and (c0.K == 1.02e-9).all() and c0.qin == 6.6e-5
    lo = henry.coefficients(PRM, grid, [-1.0, -1.0, -1.0])
    hi = henry.coefficients(PRM, grid, [1.0, 1.0, 1.0])
    # abs=0: pytest's default absolute tolerance (1e-12) would swamp K ~ 1e-9
    assert lo.phi[0, 0] == pytest.approx(0.28, rel=1e-15, abs=0) and hi.phi[0, 0] == pytest.approx(0.42, rel=1e-15, abs=0)
    assert lo.K[0, 0] == pytest.approx(6.186613e-10, rel=1e-6, abs=0)
    assert hi.K[0, 0] == pytest.approx(1.681696e-9, rel=1e-6, abs=0)
    assert lo.qin == pytest.approx(5.28e-5, rel=1e-14, abs=0) and hi.qin == pytest.approx(7.92e-5, rel=1e-14, abs=0)
    for k in range(3):
        e = [0.0, 0.0, 0.0]
        e[k] = 0.7
        ck = henry.coefficients(PRM, grid, e)
        moved = [not np.array_equal(ck.phi, c0.phi), not np.array_equal(ck.K, c0.K), ck.qin != c0.qin]
        assert moved == [j == k for j in range(3)]
    logK = [np.log(henry.coefficients(PRM, grid, [0.0, t, 0.0]).K[0, 0]) for t in (-0.8, 0.1, 0.6)]
    assert (logK[2] - logK[1]) / 0.5 == pytest.approx((logK[1] - logK[0]) / 0.9, rel=1e-12)


def test_grid_hierarchy_counts():
    """N_l = 512 * 4^l cells, r_l = 20 * 2^l steps, tau_l = 360 / 2^l s
    (regular refinement and halved time step, Sec. 2.3)."""
    for lev in range(6):
        g = henry.Grid.level(PRM, lev)
        assert g.ncell == 512 * 4 ** lev
        assert g.steps == 20 * 2 ** lev
        assert g.tau == pytest.approx(360.0 / 2 ** lev)
        assert g.h == pytest.approx(1.0 / (16 * 2 ** lev))


# Mistakes planted in the oracle's source.  The planted copy gets a complex-
# step Jacobian of its own (planted) residual, so that Newton still converges
# to the planted scheme's solution and only the physics pins above can tell.
CC_MISTAKES = {
    "horizontal upwind reversed": ("cup = np.where(np.real(F) >= 0.0, c[:, :-1], c[:, 1:])",
                                   "cup = np.where(np.real(F) >= 0.0, c[:, 1:], c[:, :-1])"),
    "gravity with the reference density": ("((p[1:, :] - p[:-1, :]) / h + rhof * prm.g)",
                                           "((p[1:, :] - p[:-1, :]) / h + prm.rho0 * prm.g)"),
    "seaside distance h instead of h/2": ("q = -(K[:, -1] / prm.mu) * (pr - p[:, -1]) / (0.5 * h)",
                                          "q = -(K[:, -1] / prm.mu) * (pr - p[:, -1]) / h"),
    "salt scatter sign": ("    Rs[:, 1:] -= G\n", "    Rs[:, 1:] += G\n"),
    "land-side diffusion distance h": ("rhob * PD[:, 0] * (cl - c[:, 0]) / (0.5 * h) * h",
                                       "rhob * PD[:, 0] * (cl - c[:, 0]) / h * h"),
    "storage without porosity": ("Rs = phi * (rho * c - rho_old * c_old) * V / tau",
                                 "Rs = (rho * c - rho_old * c_old) * V / tau"),
}


def _planted_cc(name=None):
    """A copy of oracle.henry with the named mistake planted (None: no
    mistake) and a complex-step Jacobian."""
    import os
    import types
    import scipy.sparse as sp
    src = open(os.path.join(os.path.dirname(henry.__file__), "henry.py")).read()
    if name is not None:
        a, b = CC_MISTAKES[name]
        assert src.count(a) == 1, name
        src = src.replace(a, b)
    mod = types.ModuleType("oracle._henry_planted")
    mod.__package__ = "oracle"
    exec(compile(src, "henry_planted", "exec"), mod.__dict__)

    def cs_jacobian(prm, grid, coef, p, c, p_old, c_old, bc=None, step=1e-30):
        # 5-point coupling: colour (i + 2 j) mod 5 separates a cell from its four neighbours
        J_, I_ = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
        colour = (I_ + 2 * J_) % 5
        rows, cols, vals = [], [], []
        nbrs = [(0, 0), (0, 1), (0, -1), (1, 0), (-1, 0)]
        for var in (0, 1):
            for k in range(5):
                mask = colour == k
                pz, cz = p.astype(complex), c.astype(complex)
                if var == 0:
                    pz = pz + 1j * step * mask
                else:
                    cz = cz + 1j * step * mask
                Rm, Rs = mod.residual(prm, grid, coef, pz, cz, p_old, c_old, bc=bc)
                for dj, di in nbrs:
                    jn, inn = J_ + dj, I_ + di
                    ok = (jn >= 0) & (jn < grid.ny) & (inn >= 0) & (inn < grid.nx)
                    ok &= ((inn + 2 * jn) % 5) == k
                    for eq, R in ((0, Rm), (1, Rs)):
                        d = R.imag / step
                        sel = ok & (d != 0)
                        rows.append((2 * (J_ * grid.nx + I_) + eq)[sel])
                        cols.append((2 * (jn * grid.nx + inn) + var)[sel])
                        vals.append(d[sel])
        n = 2 * grid.ncell
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))

    mod.jacobian = cs_jacobian
    return mod


def test_planted_copy_without_a_mistake_passes_the_pins(monkeypatch):
    """The harness itself: an unplanted copy, with the complex-step Jacobian,
    passes the physics pins, so a failure below is the planted mistake's."""
    monkeypatch.setitem(globals(), "henry", _planted_cc())
    test_constant_density_limit(6.6e-5)
    test_bounds_and_salt_conservation()


@pytest.mark.parametrize("name", sorted(CC_MISTAKES))
def test_pins_detect_a_mistake_planted_in_the_source(name, monkeypatch):
    monkeypatch.setitem(globals(), "henry", _planted_cc(name))
    failed = []
    for label, check in (("constant density", lambda: test_constant_density_limit(6.6e-5)),
                         ("bounds and conservation", test_bounds_and_salt_conservation),
                         ("manufactured solution", test_manufactured_solution_first_order)):
        try:
            check()
        except AssertionError:
            failed.append(label)
            break
    assert failed, name
