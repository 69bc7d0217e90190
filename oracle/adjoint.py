"""Discrete adjoint of the Henry scenario solve (oracle; test infrastructure only).

Quantity: the gradient of Q(theta) = w . qoi(x_N, theta) with respect to the
random inputs theta (xi of the three-parameter model, or the KL coefficients
and xi3 of the random-field model), where x_1 .. x_N are the implicit-Euler
states of Sec. 2.3, R_n(x_n, x_{n-1}, theta) = 0, from the fixed initial state
x_0.  Differentiating the constraints gives the adjoint (Lagrange multiplier)
recursion, written out directly:

    J_N^T lam_N = (dQ/dx_N)^T,
    J_n^T lam_n = -(dR_{n+1}/dx_n)^T lam_{n+1},          n = N-1 .. 1,
    dQ/dtheta   = dQ/dtheta|_x - sum_n lam_n^T dR_n/dtheta,

with J_n = dR_n/dx_n at the converged states (the oracle's analytic Jacobian,
itself pinned against central differences), each system solved by scipy's
sparse direct solver.  Every other partial derivative is taken by complex-step
differentiation (Squire and Trapp, SIAM Review 40, 1998): df/dt = Im f(t + i e)
/ e with e = 1e-30, exact to rounding for f analytic in t (the upwind switches
compare real parts, the porosity clip acts on the real part).  R_n depends on
the old state only through the accumulation terms of its own cell, and not on
the old pressure, so one complex perturbation of all old mass fractions gives
the whole (diagonal) old-state coupling; both facts are checked in the tests.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import henry

EPS_CS = 1e-30


def forward_states(prm, grid, coef):
    """States x_0 .. x_N of the implicit-Euler solve (oracle Newton); returns
    (list of (p, c), converged)."""
    p, c = henry.initial_state(prm, grid)
    states = [(p, c)]
    ok = True
    for _ in range(grid.steps):
        p, c, conv = henry.newton_step(prm, grid, coef, p, c)
        ok = ok and conv
        states.append((p, c))
    return states, ok


def _weighted_qoi(prm, grid, coef, p, c, w):
    m, cp = henry.qoi(prm, grid, coef, p, c)
    return w[0] * m + w[1] * cp


def adjoint_gradient(prm, level, theta, weights, model="uniform3"):
    """(dQ/dtheta, qoi(x_N), converged) for Q = weights[0] mass + weights[1] c_point."""
    grid = henry.Grid.level(prm, level)
    make = henry.coefficient_model(model)
    theta = np.asarray(theta, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    coef = make(prm, grid, theta)
    states, ok = forward_states(prm, grid, coef)
    pN, cN = states[-1]
    q = np.array(henry.qoi(prm, grid, coef, pN, cN), dtype=np.float64)
    nth = theta.size
    coef_cs = [make(prm, grid, theta + 1j * EPS_CS * np.eye(nth)[k]) for k in range(nth)]

    # dQ/dtheta at fixed state, and dQ/dc_N cell by cell (the QoIs do not involve p)
    grad = np.array([np.imag(_weighted_qoi(prm, grid, coef_cs[k], pN, cN, w)) / EPS_CS for k in range(nth)])
    dq_dc = np.zeros((grid.ny, grid.nx))
    for iy in range(grid.ny):
        for ix in range(grid.nx):
            cc = cN.astype(complex)
            cc[iy, ix] += 1j * EPS_CS
            dq_dc[iy, ix] = np.imag(_weighted_qoi(prm, grid, coef, pN, cc, w)) / EPS_CS
    rhs = henry.pack(np.zeros_like(dq_dc), dq_dc)

    for m in range(grid.steps, 0, -1):
        p, c = states[m]
        po, co = states[m - 1]
        J = henry.jacobian(prm, grid, coef, p, c, po, co)
        lam = spla.spsolve(J.T.tocsc(), rhs)
        for k in range(nth):
            Rm, Rs = henry.residual(prm, grid, coef_cs[k], p, c, po, co)
            grad[k] -= lam @ (henry.pack(np.imag(Rm), np.imag(Rs)) / EPS_CS)
        Rm, Rs = henry.residual(prm, grid, coef, p, c, po, co + 1j * EPS_CS)
        lm, ls = henry.unpack(lam, grid)
        rhs = henry.pack(np.zeros_like(lm), -(lm * np.imag(Rm) + ls * np.imag(Rs)) / EPS_CS)
    return grad, q, ok


def finite_difference_gradient(prm, level, theta, weights, model="uniform3", delta=1e-5, which=None):
    """Central differences (Q(theta + d e_k) - Q(theta - d e_k)) / (2 d) of the
    full forward solve for the components ``which`` (default: all)."""
    grid = henry.Grid.level(prm, level)
    make = henry.coefficient_model(model)
    theta = np.asarray(theta, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    which = range(theta.size) if which is None else which
    out = []
    for k in which:
        vals = []
        for sgn in (1.0, -1.0):
            t = theta.copy()
            t[k] += sgn * delta
            coef = make(prm, grid, t)
            states, _ = forward_states(prm, grid, coef)
            vals.append(float(_weighted_qoi(prm, grid, coef, *states[-1], w)))
        out.append((vals[0] - vals[1]) / (2.0 * delta))
    return np.array(out)
