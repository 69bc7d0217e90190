"""Pins of the oracle's Philox, MLMC and multigrid pieces.

* Philox4x32-10 against the known-answer vectors published with Random123
  (tests/golden/philox4x32_10_kat.txt); the xi map's exactness and symmetry.
* Eq. (M_ell) against every row of the paper's Table tab:M_ell
  (tests/golden/paper_table_M_ell.txt).
* Two-pass moments against numpy's variance; the telescoping identity of
  Eq. (EgL) with the same xi on every level (sum of Y_l = g_L per sample).
* Galerkin product against the explicit R A P; red-black sweep zeroes the
  residual on the swept colour; the 2-level V-cycle without smoothing is the
  exact coarse-grid correction P A_c^{-1} R; BiCGStab meets its tolerance and
  agrees with a direct solve.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from conftest import golden_rows
from oracle import henry, mg, mlmc, philox
from paper_2302_07804_gb300 import inputs

PRM = henry.Params()


def test_philox_known_answers():
    rows = golden_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(w, 16) for w in r]
        assert philox.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_xi_map_exact_odd_and_symmetric():
    gen = inputs.rng(11)
    for w0, w1 in gen.integers(0, 2 ** 32, size=(200, 2)):
        u = philox.words_to_unit(w0, w1)
        assert -1.0 < u < 1.0
        k = u * 2.0 ** 52
        assert k == math.floor(k) and int(k) % 2 != 0       # odd integer / 2^52, exact
        assert philox.words_to_unit(~int(w0) & 0xFFFFFFFF, ~int(w1) & 0xFFFFFFFF) == -u
    assert philox.words_to_unit(0, 0) == -1.0 + 2.0 ** -52
    assert philox.words_to_unit(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -52


def test_xi_moments_and_independence_of_levels():
    xi = philox.sample_xi(inputs.SEED, 0, 0, 3000)
    assert abs(xi.mean()) < 4 * math.sqrt(1 / 3 / xi.size)
    assert abs(xi.var() - 1 / 3) < 0.02
    xi1 = philox.sample_xi(inputs.SEED, 1, 0, 3000)
    assert abs(np.corrcoef(xi[:, 0], xi1[:, 0])[0, 1]) < 0.1
    # counters of a sample do not depend on the batch it is drawn in
    np.testing.assert_array_equal(philox.sample_xi(inputs.SEED, 2, 17, 3),
                                  philox.sample_xi(inputs.SEED, 2, 0, 20)[17:20])


def test_allocation_reproduces_paper_table():
    rows = golden_rows("paper_table_M_ell.txt")
    s = [float(v) for v in rows[0][1:]]
    V = [float(v) for v in rows[1][1:]]
    checked = 0
    for r in rows[2:]:
        eps2 = float(r[1])
        assert mlmc.allocate(V, s, eps2) == [int(v) for v in r[2:]]
        checked += 1
    assert checked == 4


def test_total_cost_formula():
    V, s = [1.4e-5, 2e-6], [1.156, 4.113]
    # two levels: the cost at the optimum m equals sum m_l s_l before rounding
    tot = sum(math.sqrt(v * c) for v, c in zip(V, s))
    m = [math.sqrt(v / c) * tot / 1e-6 for v, c in zip(V, s)]
    assert mlmc.total_cost(V, s, 1e-6) == pytest.approx(sum(mi * si for mi, si in zip(m, s)), rel=1e-12)
    assert sum(v / mi for v, mi in zip(V, m)) == pytest.approx(1e-6, rel=1e-12, abs=0)


def test_two_pass_moments_match_numpy():
    y = inputs.rng(5).normal(3.0, 2.0, size=(1000, 2))
    n, mean, m2 = mlmc.two_pass_moments(y)
    assert n == 1000
    np.testing.assert_allclose(mean, np.mean(y, axis=0), rtol=1e-14)
    np.testing.assert_allclose(m2 / (n - 1), np.var(y, axis=0, ddof=1), rtol=1e-12)


def test_telescoping_identity_same_xi():
    """With the same xi on every level, sum_l Y_l^(i) = g_L^(i) per sample."""
    L = 2
    xis = philox.sample_xi(inputs.SEED, 9, 0, 2)
    g = [henry.solve_scenarios(PRM, lev, xis)[0] for lev in range(L + 1)]
    ys = [mlmc.level_differences(g[0], None)] + [mlmc.level_differences(g[l], g[l - 1]) for l in range(1, L + 1)]
    np.testing.assert_allclose(sum(ys), g[L], rtol=1e-14, atol=1e-14)
    est, _ = mlmc.estimator([y for y in ys])
    np.testing.assert_allclose(est, g[L].mean(axis=0), rtol=1e-13)
    # the level differences shrink with the level (first-order scheme)
    assert np.abs(ys[2][:, 1]).max() < np.abs(ys[1][:, 1]).max() + 1e-3


def _henry_blocks(tag, level=0):
    grid = henry.Grid.level(PRM, level)
    coef = henry.coefficients(PRM, grid, inputs.uniform_xi(tag, 1)[0])
    p, c = inputs.random_states(tag, 2, grid.ny, grid.nx, 5e3, 1e4, 200.0)
    J = henry.jacobian(PRM, grid, coef, p[0], c[0], p[1], c[1])
    return grid, coef, p, c, J


def _piecewise_constant_P(nx, ny):
    rows, cols = [], []
    for iy in range(ny):
        for ix in range(nx):
            for v in range(2):
                rows.append(2 * (iy * nx + ix) + v)
                cols.append(2 * ((iy // 2) * (nx // 2) + ix // 2) + v)
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(2 * nx * ny, 2 * nx * ny // 4))


def test_blocks_roundtrip_and_apply():
    grid, coef, p, c, J = _henry_blocks(21)
    A = mg.blocks_from_csr(J, grid.nx, grid.ny)
    x = inputs.random_vectors(3, 1, grid.ny, grid.nx)[0]
    np.testing.assert_allclose(mg.apply(A, x).ravel(), J @ x.ravel(), rtol=1e-13, atol=1e-13 * np.abs(J).max())


def test_galerkin_is_RAP():
    grid, coef, p, c, J = _henry_blocks(22)
    A = mg.blocks_from_csr(J, grid.nx, grid.ny)
    P = _piecewise_constant_P(grid.nx, grid.ny)
    Ac_ref = (P.T @ J @ P).toarray()
    Ac = mg.dense(mg.galerkin(A))
    np.testing.assert_allclose(Ac, Ac_ref, rtol=1e-13, atol=1e-13 * np.abs(Ac_ref).max())


def test_rb_sweep_zeroes_residual_on_swept_colour():
    grid, coef, p, c, J = _henry_blocks(23)
    A = mg.blocks_from_csr(J, grid.nx, grid.ny)
    b = inputs.random_vectors(4, 1, grid.ny, grid.nx)[0]
    x = inputs.random_vectors(5, 1, grid.ny, grid.nx)[0]
    iy, ix = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
    for colour in (0, 1):
        mg.rb_sweep(A, x, b, colour)
        r = b - mg.apply(A, x)
        on = ((ix + iy) & 1) == colour
        assert np.abs(r[on]).max() <= 1e-12 * np.abs(b).max() * max(1.0, np.abs(A).max())
        assert np.abs(r[~on]).max() > 1e-6


def test_two_level_cycle_without_smoothing_is_coarse_correction():
    grid, coef, p, c, J = _henry_blocks(24)
    ops = mg.rediscretised_hierarchy(PRM, grid, coef, p[0], c[0], p[1], c[1])
    two = [ops[0], ops[1]]
    b = inputs.random_vectors(6, 1, grid.ny, grid.nx)[0]
    x = mg.vcycle(two, b, nu1=0, nu2=0)
    P = _piecewise_constant_P(grid.nx, grid.ny)
    xc = np.linalg.solve(mg.dense(ops[1]), P.T @ b.ravel())
    np.testing.assert_allclose(x.ravel(), P @ xc, rtol=1e-12)


def test_rediscretised_coarse_level_is_coarse_grid_jacobian():
    """Level-1 operator of the hierarchy = Jacobian of the scheme on the 2x
    coarser grid at the 2x2-averaged states, in the fine level's scaling."""
    grid, coef, p, c, J = _henry_blocks(25, level=1)
    ops = mg.rediscretised_hierarchy(PRM, grid, coef, p[0], c[0], p[1], c[1])
    g0 = henry.Grid.level(PRM, 0)
    gc = henry.Grid(g0.nx, g0.ny, g0.h, grid.tau, 1)
    avg = lambda f: f.reshape(gc.ny, 2, gc.nx, 2).mean(axis=(1, 3))
    coefc = henry.coefficients(PRM, gc, [0, 0, 0])
    coefc.phi[:] = coef.phi[0, 0]
    coefc.K[:] = coef.K[0, 0]
    coefc.qin = coef.qin
    Jc = henry.jacobian(PRM, gc, coefc, avg(p[0]), avg(c[0]), avg(p[1]), avg(c[1]))
    ref = mg.blocks_from_csr(Jc, gc.nx, gc.ny) / henry.residual_scale(PRM, grid)
    np.testing.assert_allclose(ops[1], ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
    assert ops[-1].shape[:2] == (1, 2)


def _trajectory_state(level, xi, steps):
    """State after ``steps`` implicit-Euler steps of a real scenario."""
    grid = henry.Grid.level(PRM, level)
    coef = henry.coefficients(PRM, grid, xi)
    p, c = henry.initial_state(PRM, grid)
    for _ in range(steps):
        p, c, ok = henry.newton_step(PRM, grid, coef, p, c)
        assert ok
    return grid, coef, p, c


@pytest.mark.parametrize("level", [0, 1])
def test_vcycle_iteration_converges_and_bicgstab_matches_direct(level):
    grid, coef, p, c = _trajectory_state(level, inputs.uniform_xi(26 + level, 1)[0], 3 << level)
    s = henry.residual_scale(PRM, grid)
    # first Newton system of the next step: Jacobian at the old state
    ops = mg.rediscretised_hierarchy(PRM, grid, coef, p, c, p, c)
    J = henry.jacobian(PRM, grid, coef, p, c, p, c)
    A = ops[0]
    b = inputs.random_vectors(8, 1, grid.ny, grid.nx)[0]
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(12):
        x = x + mg.vcycle(ops, b - mg.apply(A, x))
    assert np.linalg.norm(b - mg.apply(A, x)) < 1e-6 * r0
    xk, its, ok = mg.bicgstab(A, b, lambda v: mg.vcycle(ops, v), 1e-10)
    assert ok and its <= 15
    xd = spla.spsolve((J / s).tocsc(), b.ravel()).reshape(b.shape)
    assert np.linalg.norm(b - mg.apply(A, xk)) <= 1e-10 * r0
    np.testing.assert_allclose(xk, xd, rtol=0, atol=1e-7 * np.abs(xd).max())


def test_rates_recover_exact_geometric_sequences():
    """Theorem (costMLMC) rates from per-level statistics: exact power laws
    give exact slopes; level 0 (Y_0 = g_0, not a difference) lies off the
    line and must be excluded by first_level; two levels give the log2 ratio."""
    lev = np.arange(6)
    mean = 0.3 * 2.0 ** (-1.0 * lev) * (-1.0) ** lev
    mean[0] = 0.47                      # E[g_0]: not on the weak-error line
    V = 7e-4 * 2.0 ** (-2.0 * lev)
    V[0] = 0.03
    s = 1.5 * 8.0 ** lev
    a, b, g = mlmc.rates(mean, V, s, first_level=1)
    assert a == pytest.approx(1.0, rel=1e-12)
    assert b == pytest.approx(2.0, rel=1e-12)
    assert g == pytest.approx(3.0, rel=1e-12)
    a0, b0, _ = mlmc.rates(mean, V, s, first_level=0)
    assert abs(a0 - 1.0) > 0.05 and abs(b0 - 2.0) > 0.05
    a2, b2, g2 = mlmc.rates([9.0, 0.2, 0.05], [9.0, 0.1, 0.02], [1.0, 3.0, 20.0], first_level=1)
    assert a2 == pytest.approx(math.log2(0.2 / 0.05), rel=1e-12)
    assert b2 == pytest.approx(math.log2(0.1 / 0.02), rel=1e-12)
    assert g2 == pytest.approx(math.log2(20.0 / 3.0), rel=1e-12)


def test_bias_test_is_the_geometric_tail():
    """With E[Y_l] = c 2^(-alpha l) exactly, the bias of the level-L estimator
    is sum_{l > L} E[Y_l]; the test's estimate must equal that sum."""
    c, L = 0.01, 4
    for alpha in (0.5, 1.0, 2.0):
        means = [c * 2.0 ** (-alpha * l) for l in range(L + 1)]
        tail = sum(c * 2.0 ** (-alpha * l) for l in range(L + 1, 400))
        b, ok = mlmc.bias_test(means, alpha, 1.0)
        assert b == pytest.approx(tail, rel=1e-12, abs=0)
        assert ok
        assert mlmc.bias_test(means, alpha, math.sqrt(2.0) * tail * 0.999)[1] is False
        assert mlmc.bias_test(means, alpha, math.sqrt(2.0) * tail * 1.001)[1] is True


def test_fitted_bias_test_recovers_the_tail_and_smooths_noise():
    """The fitted variant: on exact power laws (level 0 off the line, as the
    level-0 mean is g_0 itself) it returns the exact geometric tail and the
    exact alpha; with multiplicative noise on the means it stays within the
    noise's spread of the tail, and a slope below alpha_min is floored."""
    c, L = 0.01, 5
    for alpha in (0.7, 1.0, 1.6):
        means = [0.45] + [c * 2.0 ** (-alpha * l) for l in range(1, L + 1)]
        tail = sum(c * 2.0 ** (-alpha * l) for l in range(L + 1, 400))
        b, ok, a = mlmc.bias_test_fit(means, 1.0)
        assert a == pytest.approx(alpha, rel=1e-12) and b == pytest.approx(tail, rel=1e-10)
        assert mlmc.bias_test_fit(means, math.sqrt(2.0) * tail * 0.999)[1] is False
        assert mlmc.bias_test_fit(means, math.sqrt(2.0) * tail * 1.001)[1] is True
    gen = np.random.default_rng(5)
    means = [0.45] + [c * 2.0 ** (-l) * (1 + 0.2 * gen.standard_normal()) for l in range(1, L + 1)]
    b, _, a = mlmc.bias_test_fit(means, 1.0)
    assert 0.7 < a < 1.3 and 0.5 * c * 2.0 ** -L < b < 2.0 * c * 2.0 ** -L
    flat = [0.45] + [c] * L
    assert mlmc.bias_test_fit(flat, 1.0, alpha_min=0.5)[2] == 0.5


def test_mlmc_with_independent_samples_agrees_with_plain_mc():
    """Eq. (A) with independent samples on each level (level 0: 40 samples,
    level 1: 12 fine/coarse pairs) estimates E[g_1]; plain Monte Carlo on
    level 1 (24 independent samples) estimates the same mean.  The two agree
    within 3 standard errors of their difference, for both QoIs.  (A
    16 x 8 base grid with 10 steps keeps the oracle quick; the property does
    not depend on the grid.)"""
    from dataclasses import replace
    prm = replace(PRM, nx0=16, ny0=8, steps0=10)
    x0 = philox.sample_xi(inputs.SEED, 0, 300, 40)
    x1 = philox.sample_xi(inputs.SEED, 1, 300, 12)
    xmc = philox.sample_xi(inputs.SEED, 7, 300, 24)
    g0, _ = henry.solve_scenarios(prm, 0, x0)
    f1, _ = henry.solve_scenarios(prm, 1, x1)
    c1, _ = henry.solve_scenarios(prm, 0, x1)
    mc, _ = henry.solve_scenarios(prm, 1, xmc)
    est, var = mlmc.estimator([mlmc.level_differences(g0, None), mlmc.level_differences(f1, c1)])
    n, mean, m2 = mlmc.two_pass_moments(mc)
    var_mc = m2 / (n - 1) / n
    assert np.all(np.abs(est - mean) <= 3.0 * np.sqrt(var + var_mc))
    assert np.all(var > 0) and np.all(var_mc > 0)
