"""Pins of the oracle's discrete adjoint (oracle.adjoint).

* Central differences of the full forward solve (Newton tightened to 1e-13 so
  that the differences resolve 1e-8): all three xi of the three-parameter
  model and six of the 65 inputs of the KL model (log K and phi coefficients,
  and xi3 of the recharge), and the two-layer model's three inputs, at
  level 0.
* The two structural facts the adjoint recursion relies on: the residual of
  a cell depends on the old state only through that cell's mass fraction
  (a cell-local, diagonal coupling), and not on the old pressure; the QoIs do
  not involve the pressure.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import adjoint, henry
from paper_2302_07804_gb300 import inputs

PRM = replace(henry.Params(), newton_atol=1e-13, newton_dxtol=1e-14)
W = (0.01, 1.0)


def test_adjoint_matches_central_differences_uniform3():
    for tag in (700, 702):
        xi = inputs.uniform_xi(tag, 1)[0]
        g, q, ok = adjoint.adjoint_gradient(PRM, 0, xi, W)
        assert ok
        fd = adjoint.finite_difference_gradient(PRM, 0, xi, W, delta=1e-5)
        np.testing.assert_allclose(g, fd, rtol=0, atol=1e-8 * np.abs(g).max())
        ref, _ = henry.solve_scenarios(PRM, 0, xi[None, :])
        np.testing.assert_allclose(q, ref[0], rtol=1e-13)


def test_adjoint_matches_central_differences_kl():
    gen = inputs.rng(701)
    th = np.concatenate([gen.standard_normal(64), gen.uniform(-1, 1, 1)])
    g, q, ok = adjoint.adjoint_gradient(PRM, 0, th, W, model="kl")
    assert ok and g.shape == (65,)
    which = [0, 5, 31, 32, 40, 64]
    fd = adjoint.finite_difference_gradient(PRM, 0, th, W, model="kl", delta=1e-5, which=which)
    np.testing.assert_allclose(g[which], fd, rtol=0, atol=1e-8 * np.abs(g).max())


def test_adjoint_matches_central_differences_two_layer():
    xi = np.array([0.3, -0.4, 0.2])
    g, q, ok = adjoint.adjoint_gradient(PRM, 0, xi, W, model="two_layer")
    assert ok
    fd = adjoint.finite_difference_gradient(PRM, 0, xi, W, model="two_layer", delta=1e-5)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-8 * np.abs(g).max())


def test_old_state_coupling_is_cell_local_and_pressure_free():
    grid = henry.Grid.level(PRM, 0)
    coef = henry.coefficients(PRM, grid, [0.3, -0.2, 0.5])
    p, c = inputs.random_states(710, 2, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    base = henry.residual(PRM, grid, coef, p[0], c[0], p[1], c[1])
    co = c[1].copy()
    co[5, 7] += 1e-3
    Rm, Rs = henry.residual(PRM, grid, coef, p[0], c[0], p[1], co)
    for R, R0 in ((Rm, base[0]), (Rs, base[1])):
        d = np.abs(R - R0)
        assert d[5, 7] > 0
        d[5, 7] = 0
        assert d.max() == 0.0
    Rm, Rs = henry.residual(PRM, grid, coef, p[0], c[0], p[1] + 123.0, c[1])
    assert np.array_equal(Rm, base[0]) and np.array_equal(Rs, base[1])
    assert henry.qoi(PRM, grid, coef, p[0] + 55.0, c[0]) == henry.qoi(PRM, grid, coef, p[0], c[0])
