"""Pins of the vertex-centred oracle (oracle.henry_vc) against what the paper
and the mathematics fix: the paper's degree-of-freedom counts, the discrete
hydrostatic consistency of the velocity, the pairwise cancellation of face
fluxes, a closed form in the constant-density limit with an independent
1-D scheme for c, the exactness of the complex-step Jacobian, bounds on c,
and agreement with the independent cell-centred discretisation as the grid
is refined."""
import numpy as np
import pytest
from dataclasses import replace

from conftest import golden_rows
from oracle import henry as cc
from oracle import henry_vc as vc
from oracle import philox
from paper_2302_07804_gb300 import inputs

PRM = vc.Params()


def test_dof_counts_match_the_paper_table():
    prm = cc.paper_params()
    for lev, n, r in golden_rows("paper_table_dofs.txt"):
        grid = vc.Grid.level(prm, int(lev))
        assert vc.n_dof(grid) == int(n)
        assert grid.steps == int(r)


def _random_state(grid, seed, hydrostatic=False):
    gen = inputs.rng(seed)
    c = gen.uniform(0.0, 1.0, (grid.ny + 1, grid.nx + 1))
    if hydrostatic:
        # trapezoidal discrete hydrostatics up every vertical grid line
        rho = vc.density(PRM, c)
        p = np.zeros_like(c)
        p[-1] = gen.uniform(0.0, 50.0, grid.nx + 1)
        for j in range(grid.ny - 1, -1, -1):
            p[j] = p[j + 1] + PRM.g * grid.h * 0.5 * (rho[j] + rho[j + 1])
    else:
        p = gen.uniform(0.0, 1.0e4, c.shape)
    return p, c


def _check_consistency(m):
    grid = m.Grid.level(PRM, 0)
    coef = cc.coefficients(PRM, grid, [0.2, -0.5, 0.1])
    p, c = _random_state(grid, 11, hydrostatic=True)
    fl = m.face_fluxes(PRM, grid, coef, p, c)
    scale = np.abs(fl[0][2]).max()
    assert scale > 0
    for (a, b, F, G), face in zip(fl, m.FACES):
        if face[2] == "y":
            assert np.abs(F).max() <= 1e-12 * scale
    p2, _ = _random_state(grid, 12)
    fl2 = m.face_fluxes(PRM, grid, coef, p2, c)
    assert np.abs(fl2[2][2]).max() > 1e3 * 1e-12 * scale


def test_consistent_velocity_has_no_vertical_flux_in_discrete_hydrostatic_balance():
    """Any density field: a pressure in trapezoidal hydrostatic balance along
    the vertical grid lines gives zero mass flux through every horizontal
    face (S_l, S_r); an arbitrary pressure does not."""
    _check_consistency(vc)


def _check_telescoping(m):
    grid = m.Grid.level(PRM, 1)
    gen = inputs.rng(21)
    coef = cc.Coeffs(phi=gen.uniform(0.2, 0.5, (grid.ny, grid.nx)), K=gen.uniform(5e-10, 2e-9, (grid.ny, grid.nx)),
                     qin=7.1e-5)
    p, c = _random_state(grid, 22)
    po, co = _random_state(grid, 23)
    Rm, Rs = m.fv_residual(PRM, grid, coef, p, c, po, co)
    w = m.storage_weights(grid, coef)
    rho, rho_o = m.density(PRM, c), m.density(PRM, co)
    sm = np.sum(w * (rho - rho_o)) / grid.tau - PRM.rho0 * coef.qin * PRM.Ly
    ss = np.sum(w * (rho * c - rho_o * co)) / grid.tau
    flux_scale = max(np.abs(F).max() for _, _, F, _ in m.face_fluxes(PRM, grid, coef, p, c))
    assert abs(Rm.sum() - sm) <= 1e-12 * flux_scale * Rm.size
    assert abs(Rs.sum() - ss) <= 1e-12 * flux_scale * Rs.size
    # the lumped volumes tile the domain
    ones = cc.Coeffs(phi=np.ones((grid.ny, grid.nx)), K=coef.K, qin=0.0)
    assert m.storage_weights(grid, ones).sum() == pytest.approx(PRM.Lx * PRM.Ly, rel=1e-14, abs=0)


def test_face_fluxes_cancel_in_the_sum_of_the_balances():
    """Every face flux leaves one control volume and enters its neighbour, so
    the balances of all vertices add up to the storage terms and the inflow
    through x = 0 alone (random states, random element fields)."""
    _check_telescoping(vc)


def _one_d_salt(prm, grid, phi, qin, steps):
    """Independent 1-D form of the vertex scheme for a y-independent salt
    field at constant density: vertices x_i = i h with c_0 = 0 and c_nx = 1
    fixed, face flux rho0 qin h c_f - rho0 phi Dm (c_{i+1} - c_i) with the
    central/upwind blend of the partial upwind rule, storage rho0 phi h^2;
    each implicit step is one tridiagonal (Thomas) solve."""
    n = grid.nx + 1
    h, tau, rho = grid.h, grid.tau, prm.rho0
    Fh = rho * qin * h / 2.0                        # one of the two half-height faces
    Dh = rho * phi * prm.Dm
    s = max(0.0, 1.0 - Dh / (2.0 * abs(Fh))) if Fh != 0 else 0.0
    wl, wr = 0.5 * (1 + s), 0.5 * (1 - s)            # c_f = wl c_i + wr c_{i+1} (flow to +x)
    F, D = 2 * Fh, Dh                                # a vertex row has two half-height faces per column gap
    acc = rho * phi * h * h / tau
    c = np.zeros(n)
    c[-1] = 1.0
    for _ in range(steps):
        m = n - 2
        lo, di, up, rhs = np.zeros(m), np.zeros(m), np.zeros(m), acc * c[1:-1].copy()
        for k in range(m):
            i = k + 1
            # + G_{i+1/2} = F (wl c_i + wr c_{i+1}) - D (c_{i+1} - c_i)
            # - G_{i-1/2} = -F (wl c_{i-1} + wr c_i) + D (c_i - c_{i-1})
            di[k] = acc + F * wl + D - F * wr + D
            up[k] = F * wr - D
            lo[k] = -F * wl - D
        rhs[0] -= lo[0] * c[0]
        rhs[-1] -= up[-1] * c[-1]
        # Thomas algorithm
        cp, dp = np.zeros(m), np.zeros(m)
        cp[0], dp[0] = up[0] / di[0], rhs[0] / di[0]
        for k in range(1, m):
            den = di[k] - lo[k] * cp[k - 1]
            cp[k] = up[k] / den
            dp[k] = (rhs[k] - lo[k] * dp[k - 1]) / den
        x = np.zeros(m)
        x[-1] = dp[-1]
        for k in range(m - 2, -1, -1):
            x[k] = dp[k] - cp[k] * x[k + 1]
        c[1:-1] = x
    return c


def _check_constant_density(m, qin):
    prm = replace(PRM, rho1=PRM.rho0)
    grid = m.Grid.level(prm, 0)
    coef = cc.coefficients(prm, grid, [0.0, 0.0, 0.0])
    coef = cc.Coeffs(phi=coef.phi, K=coef.K, qin=qin)
    K, phi = float(coef.K[0, 0]), float(coef.phi[0, 0])
    p, c = m.initial_state(prm, grid)
    steps = 12
    for _ in range(steps):
        p, c, ok = m.newton_step(prm, grid, coef, p, c)
        assert ok
    x = np.arange(grid.nx + 1) * grid.h
    y = m.vertex_y(grid)
    p_exact = prm.rho0 * prm.g * (prm.Ly - y)[:, None] + prm.mu * qin * (prm.Lx - x)[None, :] / K
    np.testing.assert_allclose(p, p_exact, rtol=0, atol=1e-9 * prm.rho0 * prm.g * prm.Ly)
    c1 = _one_d_salt(prm, grid, phi, qin, steps)
    np.testing.assert_allclose(c, np.broadcast_to(c1, c.shape), rtol=0, atol=1e-11)


@pytest.mark.parametrize("qin", [0.0, 6.6e-5, 1.0e-3])
def test_constant_density_limit(qin):
    """rho1 = rho0: the pressure is exactly rho0 g (Ly - y) + mu qin (Lx - x)/K
    (bilinear fields reproduce it, and the flow is uniform), and c stays
    y-independent and equal to the 1-D scheme; qin = 1e-3 m/s drives the
    partial upwinding (face Peclet number ~10 at level 0)."""
    _check_constant_density(vc, qin)


def test_complex_step_jacobian_matches_central_differences():
    grid = vc.Grid(nx=6, ny=3, h=1.0 / 3, tau=200.0, steps=1)
    prm = replace(PRM, Lx=2.0, Ly=1.0)
    coef = cc.coefficients(prm, grid, [0.3, 0.4, -0.2])
    coef = cc.Coeffs(phi=coef.phi, K=coef.K * 400.0, qin=coef.qin * 40.0)   # strong flow: partial upwind active
    p, c = _random_state(grid, 31)
    c = 0.1 + 0.8 * c
    po, co = _random_state(grid, 32)
    J = vc.jacobian(prm, grid, coef, p, c, po, co).toarray()
    x0 = vc.pack(p, c)
    n = x0.size
    fd = np.zeros((n, n))
    for k in range(n):
        e = 1e-2 if k % 2 == 0 else 1e-5
        xp, xm = x0.copy(), x0.copy()
        xp[k] += e
        xm[k] -= e
        rp = vc.pack(*vc.residual(prm, grid, coef, *vc.unpack(xp, grid), po, co))
        rm = vc.pack(*vc.residual(prm, grid, coef, *vc.unpack(xm, grid), po, co))
        fd[:, k] = (rp - rm) / (2 * e)
    for r in range(n):
        scale = np.abs(J[r]).max()
        np.testing.assert_allclose(J[r], fd[r], rtol=0, atol=1e-6 * scale)


def test_bounds_through_a_level0_solve():
    for xi in philox.sample_xi(inputs.SEED, 0, 500, 2):
        grid = vc.Grid.level(PRM, 0)
        coef = cc.coefficients(PRM, grid, xi)
        p, c = vc.initial_state(PRM, grid)
        for _ in range(grid.steps):
            p, c, ok = vc.newton_step(PRM, grid, coef, p, c)
            assert ok
            assert c.min() >= -1e-10 and c.max() <= 1 + 1e-10


def test_salt_mass_of_uniform_fields():
    grid = vc.Grid.level(PRM, 1)
    coef = cc.coefficients(PRM, grid, [-0.6, 0.2, 0.9])
    phi = float(coef.phi[0, 0])
    for cu in (0.25, 1.0):
        c = np.full((grid.ny + 1, grid.nx + 1), cu)
        m, cpt = vc.qoi(PRM, grid, coef, c, c)
        assert m == pytest.approx(phi * (PRM.rho0 + (PRM.rho1 - PRM.rho0) * cu) * cu * PRM.Lx * PRM.Ly, rel=1e-13, abs=0)
        assert cpt == cu


def test_agrees_with_the_cell_centred_scheme_as_the_grid_is_refined():
    """Two independent consistent discretisations of the same equations: the
    QoIs agree to within the first-order discretisation error, and the point
    value's difference shrinks from level 0 to level 1."""
    xi = [0.3, -0.4, 0.5]
    d = []
    for lev in (0, 1):
        qv, okv = vc.solve_scenario(PRM, lev, xi)
        qc, okc = cc.solve_scenario(PRM, lev, xi)
        assert okv and okc
        assert abs(qv[0] - qc[0]) <= 0.03 * qc[0]
        d.append(abs(qv[1] - qc[1]))
    assert d[0] < 1e-2 and d[1] < 0.75 * d[0]



def _mms_errors(levels, T_end=600.0, steps0=2, K=2e-10, phi=0.35):
    """Max errors (c, p) at t = T_end against a manufactured (p, c): sympy
    derives the vertex sources of the fluid and salt balances and the
    Dirichlet data on all four sides; grids of 8 x 4 elements times 2^l with
    tau proportional to h^2, so that the spatial order shows."""
    sy = pytest.importorskip("sympy")
    x, y, t = sy.symbols("x y t")
    rho0, rho1, mu, g, Dm = PRM.rho0, PRM.rho1, PRM.mu, PRM.g, PRM.Dm
    c_ex = 0.5 + 0.3 * sy.sin(sy.pi * x / 2 + 0.3) * sy.cos(sy.pi * y) * sy.exp(-t / 3600)
    p_ex = rho0 * g * (1 - y) + 60 * (2 - x) + 30 * sy.cos(sy.pi * x / 2) * sy.cos(sy.pi * y) * (1 + t / 3600)
    rho = rho0 + (rho1 - rho0) * c_ex
    qx = -(K / mu) * sy.diff(p_ex, x)
    qy = -(K / mu) * (sy.diff(p_ex, y) + rho * g)
    Sm = sy.diff(phi * rho, t) + sy.diff(rho * qx, x) + sy.diff(rho * qy, y)
    Ss = sy.diff(phi * rho * c_ex, t) + sy.diff(rho * c_ex * qx - rho * phi * Dm * sy.diff(c_ex, x), x) + \
        sy.diff(rho * c_ex * qy - rho * phi * Dm * sy.diff(c_ex, y), y)
    fSm, fSs, fc, fp = (sy.lambdify((x, y, t), e, "numpy") for e in (Sm, Ss, c_ex, p_ex))
    full = lambda f, a, b, tt: f(a, b, tt) + 0.0 * (a + b)
    out = []
    for lev in levels:
        nx, ny = 8 << lev, 4 << lev
        steps = steps0 * 4 ** lev
        grid = vc.Grid(nx, ny, 1.0 / ny, T_end / steps, steps)
        coef = cc.Coeffs(phi=np.full((ny, nx), phi), K=np.full((ny, nx), K), qin=0.0)
        X, Y = np.meshgrid(np.arange(nx + 1) * grid.h, np.arange(ny + 1) * grid.h)
        p, c = full(fp, X, Y, 0.0), full(fc, X, Y, 0.0)
        for n in range(steps):
            tn = (n + 1) * grid.tau
            p, c, ok = vc.newton_step(PRM, grid, coef, p, c, src=(full(fSm, X, Y, tn), full(fSs, X, Y, tn)),
                                      dirichlet=(full(fp, X, Y, tn), full(fc, X, Y, tn)))
            assert ok
        out.append((np.abs(c - full(fc, X, Y, T_end)).max(), np.abs(p - full(fp, X, Y, T_end)).max()))
    return np.array(out)


def test_manufactured_solution_second_order():
    """Bilinear fluxes on the box grid with central faces (the manufactured
    flow has face Peclet numbers below 2, so the partial upwind stays
    central) and tau ~ h^2: second order in h for c and p."""
    e = _mms_errors([0, 1, 2])
    order_c = np.log2(e[:-1, 0] / e[1:, 0])
    order_p = np.log2(e[:-1, 1] / e[1:, 1])
    assert np.all(order_c > 1.7), order_c
    assert np.all(order_p > 1.7), order_p

MISTAKES = {
    "gravity sign": ("grav = ((1 - xi)", "grav = -((1 - xi)"),
    "full upwind": ("s = np.where(upw, 1.0 - Dc / (2.0 * np.where(upw, absF, 1.0)), 0.0)", "s = 1.0 + 0.0 * absF"),
    "salt scatter sign": ("        Rs[_CORNER[b]] -= G", "        Rs[_CORNER[b]] += G"),
    "storage volume h^2/2": ("return w * (grid.h * grid.h / 4.0)", "return w * (grid.h * grid.h / 2.0)"),
    "inflow share": ("L[0] = L[-1] = 0.5 * grid.h", "L[0] = L[-1] = grid.h"),
    "y-gradient transposed": ("dc = ((1 - xi) * (C[2] - C[0]) + xi * (C[3] - C[1])) / h",
                              "dc = ((1 - xi) * (C[1] - C[0]) + xi * (C[3] - C[2])) / h"),
}


def _planted(name):
    """A copy of oracle.henry_vc with one mistake planted in its source."""
    import os
    import types
    a, b = MISTAKES[name]
    src = open(os.path.join(os.path.dirname(vc.__file__), "henry_vc.py")).read()
    assert src.count(a) == 1, name
    mod = types.ModuleType("oracle._henry_vc_planted")
    mod.__package__ = "oracle"
    exec(compile(src.replace(a, b), "henry_vc_planted", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_pins_detect_a_planted_mistake(name):
    """Each planted mistake fails at least one of the pins above."""
    m = _planted(name)
    failed = 0
    for check in (lambda: _check_consistency(m), lambda: _check_telescoping(m),
                  lambda: _check_constant_density(m, 6.6e-5), lambda: _check_constant_density(m, 1.0e-3)):
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed > 0, name
