"""Pins of the oracle's paper QoIs (Sec. 2.2 and 4).

* Q_FW of Eq. (integral_fw) on the initial state (c = 0 everywhere) is the
  whole domain, 2.0, the initial freshwater volume the paper prints (Sec. 4);
  for c = x / Lx it is the area of the columns whose centre lies left of
  x = 0.012178 Lx.
* Point values by bilinear interpolation reproduce a linear field exactly at
  the 12 points of Eq. (12points), equal the cell value at a cell centre, and
  at the vertex (1.5, 0.25) equal the four-cell mean of the c_point QoI.
* The level-0 field average is the identity at level 0, keeps constants, and
  preserves the integral of c.
* The paper preset's level-0 step is tau = 6016 / 188 = 32 s (Sec. 4).
"""
import math

import numpy as np
import pytest

from oracle import henry

PRM = henry.Params()


def test_freshwater_area_of_initial_state_is_the_domain():
    for level in (0, 2):
        grid = henry.Grid.level(PRM, level)
        p, c = henry.initial_state(PRM, grid)
        assert henry.freshwater_area(grid, c) == pytest.approx(2.0, rel=1e-15)
        xc = (np.arange(grid.nx) + 0.5) * grid.h
        cx = np.tile(xc / PRM.Lx, (grid.ny, 1))
        ncol = int(np.count_nonzero(xc / PRM.Lx <= henry.C_FRESH))
        assert henry.freshwater_area(grid, cx) == pytest.approx(ncol * grid.ny * grid.h * grid.h, rel=1e-15)


def test_point_values_reproduce_linear_fields():
    for level in (0, 1, 2):
        grid = henry.Grid.level(PRM, level)
        x = (np.arange(grid.nx) + 0.5) * grid.h
        y = (np.arange(grid.ny) + 0.5) * grid.h
        X, Y = np.meshgrid(x, y)
        c = 0.3 + 0.2 * X - 0.7 * Y
        for px, py in henry.POINTS_12:
            yy = py + PRM.Ly
            assert henry.point_value(PRM, grid, c, px, yy) == pytest.approx(0.3 + 0.2 * px - 0.7 * yy, abs=1e-14)
        rng = np.random.default_rng(3)
        r = rng.random((grid.ny, grid.nx))
        assert henry.point_value(PRM, grid, r, x[5], y[3]) == pytest.approx(r[3, 5], abs=1e-15)
        coef = henry.coefficients(PRM, grid, [0.0, 0.0, 0.0])
        assert henry.point_value(PRM, grid, r, 1.5, 0.25) == pytest.approx(henry.qoi(PRM, grid, coef, r, r)[1],
                                                                         abs=1e-15)


def test_level0_field_average():
    rng = np.random.default_rng(4)
    g0 = henry.Grid.level(PRM, 0)
    c0 = rng.random((g0.ny, g0.nx))
    np.testing.assert_array_equal(henry.field_level0(PRM, g0, c0), c0.ravel())
    g2 = henry.Grid.level(PRM, 2)
    c2 = rng.random((g2.ny, g2.nx))
    f = henry.field_level0(PRM, g2, c2)
    assert f.shape == (g0.nx * g0.ny,)
    assert f.sum() * g0.h ** 2 == pytest.approx(c2.sum() * g2.h ** 2, rel=1e-13)
    np.testing.assert_allclose(henry.field_level0(PRM, g2, np.full((g2.ny, g2.nx), 0.37)), 0.37, rtol=1e-15)


def test_paper_preset_and_solve():
    prm = henry.paper_params()
    grid = henry.Grid.level(prm, 0)
    assert grid.tau == pytest.approx(32.0) and grid.steps == 188 and prm.T == 6016.0
    q, ok = henry.solve_scenario(prm, 0, [-0.5898, -0.7257, -0.9616], model="two_layer", qoi_set=1)
    assert ok and q.shape == (15,)
    assert 0.0 < q[2] < 2.0                 # salt has entered: less fresh water than the whole domain
    assert np.all((q[3:] >= -1e-12) & (q[3:] <= 1 + 1e-12))
    assert q[6] > q[3]                      # closer to the sea, saltier (same row, y = -0.95)


def test_freshwater_series():
    """Q_FW after every level-0 step (qoi_set 3): starts below the initial
    2.0, ends at the final-time Q_FW, and at level 1 is recorded every second
    fine step, at the same instants."""
    xi = [0.2, -0.3, 0.4]
    q0, ok0 = henry.solve_scenario(PRM, 0, xi, qoi_set=3)
    q1, ok1 = henry.solve_scenario(PRM, 1, xi, qoi_set=3)
    assert ok0 and ok1 and q0.shape == (15 + 20,) and q1.shape == (15 + 20,)
    for q in (q0, q1):
        assert q[-1] == q[2]
        assert np.all(q[15:] <= 2.0) and q[15] < 2.0
    assert np.all(np.diff(q0[15:]) <= 1e-12)   # salt only advances in this scenario
