"""GPU parity on the widest grids: MLMC levels 4 (512 x 256 cells) and 5
(1024 x 512 cells), through the C ABI, against the FP64 oracle element by
element.

These levels run code that the narrower grids never reach:
* the fine assembly (and the rediscretised coarse operators wider than 256
  cells) is the 128 x 2-tile face-once kernel, with halo faces evaluated on
  the tiles' west and south edges (default ``tile_assembly = 1``);
* the BiCGStab dot products of a sample are reduced once per sample by the
  finalising kernel (nct = N / 256 = 512 and 2048 blocks per sample, at or
  above the default ``finalize_nct = 512``);
* the V-cycle descends through 9 and 10 multigrid levels.

Tolerances are those of the level 0-1 parity tests: residuals to 1e-12 of the
flux scale, Jacobian blocks to 1e-11 of each block entry's largest magnitude,
y = J x to 1e-12 of |J| |x|, a V-cycle to 1e-9 of its largest entry (rounding
amplified by the smoother), and the linear solve to its stated relative
residual measured with the oracle's own sparse Jacobian.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry
from oracle import mg as omg
from paper_2302_07804_gb300 import inputs

PRM = ohenry.Params()
DEV = "cuda"
LEVELS = [4, 5]


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


@pytest.fixture(scope="module")
def solver(hl):
    s = hl.Solver()
    assert s.cfg.tile_assembly == 1 and 0 < s.cfg.finalize_nct <= 512
    yield s
    s.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _case(tag, level, n):
    grid = ohenry.Grid.level(PRM, level)
    xi = inputs.uniform_xi(tag, n)
    p, c = inputs.random_states(tag, 2 * n, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    return grid, xi, p[:n], c[:n], p[n:], c[n:]


def _st(p, c):
    return np.stack([p, c], axis=-1)


def _wedge_states(grid, coef, shift):
    """A salt-wedge-like state: c a smooth front rising towards the sea, p in
    hydrostatic balance with rho(c) (a cell-centred column sum from the top),
    plus the constant-density inflow gradient mu q_in (Lx - x) / K and a
    smooth 20 Pa perturbation.  Random states with cell-scale noise in c give
    advection-dominated Jacobians on which the red-black smoother diverges;
    on states like this one (and on real trajectories) a V(2,2) cycle
    contracts by 0.01-0.05.  Without the perturbation the balance would be
    exact in the discrete sense, every vertical flux would be zero up to
    rounding, and the upwind choice on those faces (and with it the
    Jacobian's dG/dp = c_up dF/dp) would be decided by rounding on each side:
    two correct Jacobians, not one."""
    x = (np.arange(grid.nx) + 0.5) * grid.h
    y = (np.arange(grid.ny) + 0.5) * grid.h
    X, Y = np.meshgrid(x, y)
    c = 0.5 * (1.0 + np.tanh((X - 1.3 - 0.5 * Y + shift) / 0.15))
    rho = PRM.rho0 + (PRM.rho1 - PRM.rho0) * c
    col = np.cumsum(rho[::-1, :], axis=0)[::-1, :] * grid.h * PRM.g
    p = col - 0.5 * grid.h * PRM.g * rho + PRM.mu * coef.qin * (PRM.Lx - X) / coef.K
    p = p + 20.0 * np.sin(np.pi * X / 2 + shift) * np.cos(np.pi * Y + 0.3)
    return p, c


def _wedge_case(tag, level, n):
    grid = ohenry.Grid.level(PRM, level)
    xi = inputs.uniform_xi(tag, n)
    shifts = inputs.rng(tag).uniform(-0.2, 0.2, size=n)
    p, c, po, co = [], [], [], []
    for i in range(n):
        coef = ohenry.coefficients(PRM, grid, xi[i])
        a, b = _wedge_states(grid, coef, shifts[i])
        ao, bo = _wedge_states(grid, coef, shifts[i] + 0.02)
        p.append(a); c.append(b); po.append(ao); co.append(bo)
    return grid, xi, np.array(p), np.array(c), np.array(po), np.array(co)


@pytest.mark.parametrize("level", LEVELS)
def test_assemble_wide_grid_against_oracle(solver, level):
    grid, xi, p, c, po, co = _case(900 + level, level, 1)
    F, J = solver.assemble(level, _dev(xi), _dev(_st(p, c)), _dev(_st(po, co)))
    F, J = F.cpu().numpy()[0], J.cpu().numpy()[0]
    s = ohenry.residual_scale(PRM, grid)
    coef = ohenry.coefficients(PRM, grid, xi[0])
    Rm, Rs = ohenry.residual(PRM, grid, coef, p[0], c[0], po[0], co[0])
    Jo = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p[0], c[0], po[0], co[0]), grid.nx, grid.ny) / s
    Fo = np.stack([Rm, Rs], axis=-1) / s
    fscale = np.abs(Jo[..., 0, :, 0]).max() * 300.0 + 1.0
    np.testing.assert_allclose(F, Fo, rtol=0, atol=1e-12 * fscale)
    for k in range(5):          # centre, west, east, south, north
        for eq in range(2):
            for var in range(2):
                scale = np.abs(Jo[..., k, eq, var]).max()
                np.testing.assert_allclose(J[..., k, eq, var], Jo[..., k, eq, var], rtol=0,
                                           atol=1e-11 * max(scale, 1e-300))


@pytest.mark.parametrize("level", LEVELS)
def test_apply_jacobian_wide_grid_against_oracle(solver, level):
    grid, xi, p, c, po, co = _case(910 + level, level, 1)
    x = inputs.random_vectors(911 + level, 1, grid.ny, grid.nx)
    y = solver.apply_jacobian(level, _dev(xi), _dev(_st(p, c)), _dev(_st(po, co)), _dev(x)).cpu().numpy()[0]
    coef = ohenry.coefficients(PRM, grid, xi[0])
    J = ohenry.jacobian(PRM, grid, coef, p[0], c[0], po[0], co[0]) / ohenry.residual_scale(PRM, grid)
    yo = (J @ x[0].ravel()).reshape(grid.ny, grid.nx, 2)
    np.testing.assert_allclose(y, yo, rtol=0, atol=1e-12 * np.abs(J).max() * np.abs(x[0]).max())


@pytest.mark.parametrize("level", LEVELS)
def test_vcycle_wide_grid_against_oracle(solver, level):
    """One V(2,2) cycle on the rediscretised hierarchy (9 or 10 levels) built
    at the given states, against the textbook cycle of oracle.mg."""
    grid, xi, p, c, po, co = _wedge_case(920 + level, level, 1)
    b = inputs.random_vectors(921 + level, 1, grid.ny, grid.nx)
    z = solver.precondition(level, _dev(xi), _dev(_st(p, c)), _dev(_st(po, co)), _dev(b)).cpu().numpy()[0]
    coef = ohenry.coefficients(PRM, grid, xi[0])
    ops = omg.rediscretised_hierarchy(PRM, grid, coef, p[0], c[0], po[0], co[0])
    assert len(ops) == level + 5     # 32 x 16 * 2^l down to 2 x 1
    zo = omg.vcycle(ops, b[0], solver.cfg.nu1, solver.cfg.nu2)
    np.testing.assert_allclose(z, zo, rtol=0, atol=1e-9 * np.abs(zo).max())


@pytest.mark.parametrize("level", LEVELS)
def test_linear_solve_wide_grid_reaches_tolerance(hl, level):
    """BiCGStab with the finalised per-sample reductions: the returned x
    satisfies ||b - J x|| <= rtol ||b|| with J the oracle's sparse Jacobian."""
    rtol = 1e-8
    s = hl.Solver(lin_rtol=rtol, lin_maxit=40)
    assert s.cfg.finalize_nct <= (s.cfg.nx0 << level) * (s.cfg.ny0 << level) // 256
    grid, xi, p, c, po, co = _wedge_case(930 + level, level, 2)
    b = inputs.random_vectors(931 + level, 2, grid.ny, grid.nx)
    x, its = s.linear_solve(level, _dev(xi), _dev(_st(p, c)), _dev(_st(po, co)), _dev(b))
    x, its = x.cpu().numpy(), its.cpu().numpy()
    assert np.all(its > 0) and np.all(its <= 40), its
    for i in range(2):
        coef = ohenry.coefficients(PRM, grid, xi[i])
        J = ohenry.jacobian(PRM, grid, coef, p[i], c[i], po[i], co[i]) / ohenry.residual_scale(PRM, grid)
        r = b[i].ravel() - J @ x[i].ravel()
        assert np.linalg.norm(r) <= 1.5 * rtol * np.linalg.norm(b[i]), np.linalg.norm(r) / np.linalg.norm(b[i])
    s.close()


def test_kl_assemble_level4_against_oracle(hl):
    """The field model on the tile kernel's halo faces: per-cell phi, K and
    the harmonic face means of the KL fields at level 4."""
    from oracle import kl as okl
    level = 4
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    grid = ohenry.Grid.level(PRM, level)
    gen = inputs.rng(940)
    th = np.concatenate([gen.standard_normal((1, 64)), gen.uniform(-1, 1, (1, 1))], axis=1)
    p, c = inputs.random_states(941, 2, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    F, J = s.assemble(level, _dev(th), _dev(_st(p[:1], c[:1])), _dev(_st(p[1:], c[1:])))
    F, J = F.cpu().numpy()[0], J.cpu().numpy()[0]
    sc = ohenry.residual_scale(PRM, grid)
    coef = okl.coefficients_kl(PRM, grid, th[0])
    Rm, Rs = ohenry.residual(PRM, grid, coef, p[0], c[0], p[1], c[1])
    Jo = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p[0], c[0], p[1], c[1]), grid.nx, grid.ny) / sc
    Fo = np.stack([Rm, Rs], axis=-1) / sc
    fscale = np.abs(Jo[..., 0, :, 0]).max() * 300.0 + 1.0
    np.testing.assert_allclose(F, Fo, rtol=0, atol=1e-11 * fscale)
    for k in range(5):
        for eq in range(2):
            for var in range(2):
                scale = np.abs(Jo[..., k, eq, var]).max()
                np.testing.assert_allclose(J[..., k, eq, var], Jo[..., k, eq, var], rtol=0,
                                           atol=1e-11 * max(scale, 1e-300))
    s.close()


@pytest.mark.parametrize("level,tile_w", [(3, 32), (3, 256), (4, 32), (4, 64), (4, 256)])
def test_assembly_tile_shapes_give_identical_values(hl, level, tile_w):
    """Each tile shape (assembly_tile_w x 256 / assembly_tile_w cells)
    evaluates every face with the same source arithmetic as the default tiles
    (whole 256-cell rows at level 3, 128 x 2 at level 4), only in another CTA
    or thread, or on a tile edge instead of in shared memory: F is
    bit-identical, and every Jacobian block entry agrees to 1e-14 of that
    entry's largest magnitude (the compiler contracts multiply-adds into FMAs
    per call site, so the face derivatives evaluated on a tile edge may differ
    in the last bit), for the three-parameter and the KL model (per-cell
    fields and face means)."""
    grid, xi, p, c, po, co = _case(950 + level, level, 2)
    gen = inputs.rng(952 + level)
    th = _dev(np.concatenate([gen.standard_normal((2, 64)), gen.uniform(-1, 1, (2, 1))], axis=1))
    for model, x in ((hl.HENRY_MODEL_UNIFORM3, _dev(xi)), (hl.HENRY_MODEL_KL, th)):
        ref = hl.Solver(coef_model=model)
        alt = hl.Solver(coef_model=model, assembly_tile_w=tile_w)
        F0, J0 = ref.assemble(level, x, _dev(_st(p, c)), _dev(_st(po, co)))
        F1, J1 = alt.assemble(level, x, _dev(_st(p, c)), _dev(_st(po, co)))
        assert torch.equal(F1, F0), (model, tile_w)
        J0, J1 = J0.cpu().numpy(), J1.cpu().numpy()
        for k in range(J0.shape[-3]):
            for eq in range(2):
                for var in range(2):
                    scale = np.abs(J0[..., k, eq, var]).max()
                    np.testing.assert_allclose(J1[..., k, eq, var], J0[..., k, eq, var], rtol=0,
                                               atol=1e-14 * max(scale, 1e-300), err_msg=str((model, tile_w, k)))
        ref.close()
        alt.close()
