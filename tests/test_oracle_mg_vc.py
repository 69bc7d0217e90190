"""Pins of the vertex-centred multigrid oracle (oracle.mg_vc): the block
operator equals the sparse Jacobian; prolongation is exact on bilinear
fields and restriction is its transpose; a sweep zeroes the residual on its
colour; a cycle without smoothing is the coarse-grid correction written with
explicit matrices; the V-cycle converges at a rate that does not grow with
refinement (the assumption of Sec. 2.3); BiCGStab with it matches a direct
solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import henry as cc
from oracle import henry_vc as vc
from oracle import mg
from oracle import mg_vc
from paper_2302_07804_gb300 import inputs

PRM = vc.Params()


def _newton_system(level, xi=(0.3, -0.2, 0.4), steps=3):
    """The Jacobian and residual of the first Newton iteration of a time step
    after a few real steps of the scheme."""
    grid = vc.Grid.level(PRM, level)
    coef = cc.coefficients(PRM, grid, list(xi))
    p, c = vc.initial_state(PRM, grid)
    for _ in range(steps):
        p, c, ok = vc.newton_step(PRM, grid, coef, p, c)
        assert ok
    return grid, coef, p, c


def test_block_operator_equals_the_sparse_jacobian():
    grid, coef, p, c = _newton_system(0)
    Jsp = vc.jacobian(PRM, grid, coef, p, c, p, c)
    A = mg_vc.blocks_from_csr(Jsp, grid)
    x = inputs.rng(3).standard_normal((grid.ny + 1, grid.nx + 1, 2))
    # rounding bound per row: summation order differs, rows can cancel
    bound = 1e-14 * (abs(Jsp) @ np.abs(x.ravel()))
    assert np.all(np.abs(mg_vc.apply(A, x).ravel() - Jsp @ x.ravel()) <= bound)
    np.testing.assert_allclose(mg_vc.dense(A), Jsp.toarray(), rtol=0, atol=0)


def test_prolongation_is_exact_on_bilinear_fields_and_restriction_is_its_transpose():
    nyc, nxc = 4, 8
    Yc, Xc = np.meshgrid(np.arange(nyc + 1) * 2.0, np.arange(nxc + 1) * 2.0, indexing="ij")
    Yf, Xf = np.meshgrid(np.arange(2 * nyc + 1), np.arange(2 * nxc + 1), indexing="ij")
    f = lambda X, Y: 0.3 + 1.7 * X - 0.4 * Y + 0.25 * X * Y
    xc = np.stack([f(Xc, Yc), -f(Xc, Yc)], axis=-1)
    np.testing.assert_allclose(mg_vc.prolong(xc), np.stack([f(Xf, Yf), -f(Xf, Yf)], axis=-1), rtol=1e-14, atol=1e-13)
    gen = inputs.rng(4)
    zc = gen.standard_normal((nyc + 1, nxc + 1, 2))
    r = gen.standard_normal((2 * nyc + 1, 2 * nxc + 1, 2))
    assert np.vdot(mg_vc.prolong(zc), r) == pytest.approx(np.vdot(zc, mg_vc.restrict(r)), rel=1e-13, abs=0)


def test_sweep_zeroes_the_residual_on_its_colour():
    grid, coef, p, c = _newton_system(0)
    A = mg_vc.blocks_from_csr(vc.jacobian(PRM, grid, coef, p, c, p, c), grid)
    gen = inputs.rng(5)
    b = gen.standard_normal((grid.ny + 1, grid.nx + 1, 2))
    x = gen.standard_normal(b.shape)
    for colour in range(4):
        x = mg_vc.sweep(A, x, b, colour)
        r = b - mg_vc.apply(A, x)
        sel = mg_vc.colour_of(grid.ny + 1, grid.nx + 1) == colour
        assert np.abs(r[sel]).max() <= 1e-12 * np.abs(b).max()
        assert np.abs(r[~sel]).max() > 1e-6


def test_cycle_without_smoothing_is_the_coarse_grid_correction():
    grid, coef, p, c = _newton_system(0)
    ops = mg_vc.hierarchy(PRM, grid, coef, p, c, p, c)[:2]
    b = inputs.rng(6).standard_normal((grid.ny + 1, grid.nx + 1, 2))
    x = mg_vc.vcycle(ops, b, nu1=0, nu2=0)
    # explicit matrices: P from prolongated unit vectors, the coarse Dirichlet entries removed from R b
    nyc1, nxc1 = ops[1].shape[:2]
    nc = 2 * nyc1 * nxc1
    P = np.stack([mg_vc.prolong(e.reshape(nyc1, nxc1, 2)).ravel() for e in np.eye(nc)], axis=1)
    keep = ~mg_vc.dirichlet_mask(nyc1, nxc1).ravel()
    rc = (P.T @ b.ravel()) * keep
    expected = P @ np.linalg.solve(mg_vc.dense(ops[1]), rc)
    np.testing.assert_allclose(x.ravel(), expected, rtol=0, atol=1e-12 * np.abs(expected).max())


def _vcycle_rate(level):
    grid, coef, p, c = _newton_system(level)
    ops = mg_vc.hierarchy(PRM, grid, coef, p, c, p, c)
    b = inputs.rng(7).standard_normal(ops[0].shape[:2] + (2,))
    b[mg_vc.dirichlet_mask(*b.shape[:2])] = 0.0
    x = np.zeros_like(b)
    norms = []
    for _ in range(6):
        r = b - mg_vc.apply(ops[0], x)
        norms.append(np.linalg.norm(r))
        x = x + mg_vc.vcycle(ops, r)
    return max(norms[k + 1] / norms[k] for k in range(2, len(norms) - 1))


def test_vcycle_rate_does_not_grow_with_refinement():
    r0, r1 = _vcycle_rate(0), _vcycle_rate(1)
    assert r0 < 0.15 and r1 < 0.15, (r0, r1)
    assert r1 < 2.0 * r0 + 0.05, (r0, r1)


def test_bicgstab_with_the_vcycle_matches_a_direct_solve():
    grid, coef, p, c = _newton_system(1)
    Jsp = vc.jacobian(PRM, grid, coef, p, c, p, c)
    ops = mg_vc.hierarchy(PRM, grid, coef, p, c, p, c)
    b = inputs.rng(8).standard_normal((grid.ny + 1, grid.nx + 1, 2))
    x, its, ok = mg.bicgstab(lambda z: mg_vc.apply(ops[0], z), b, lambda z: mg_vc.vcycle(ops, z), rtol=1e-12)
    assert ok and its <= 10, its
    ref = spla.spsolve(Jsp.tocsc(), b.ravel())
    np.testing.assert_allclose(x.ravel(), ref, rtol=0, atol=1e-9 * np.abs(ref).max())
