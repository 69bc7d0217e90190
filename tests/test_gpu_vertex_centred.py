"""GPU parity of the vertex-centred assembly (henry_vc_assemble, the paper's
own discretisation of Sec. 2.3) against the vertex-centred oracle: residuals
and 9-point Jacobian blocks, through the C ABI, at levels 0 and 1 and with a
flow strong enough for partial upwinding.  Tolerances as on the host build
of the same arithmetic: 1e-12 of the largest flux for residuals, 1e-11 of
each block column's largest entry for the Jacobian."""
import numpy as np
import pytest
from dataclasses import replace

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as cc
from oracle import henry_vc as vc
from paper_2302_07804_gb300 import inputs
from test_vc_assembly_host import blocks_from_sparse, random_states


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("level,n,scale", [(0, 3, 1.0), (1, 2, 1.0), (0, 2, 50.0)])
def test_vc_assembly_matches_oracle(hl, level, n, scale):
    prm = replace(vc.Params(), K_mean=1.02e-9 * scale, qin_mean=6.6e-5 * scale)
    s = hl.Solver(K_mean=prm.K_mean, qin_mean=prm.qin_mean)
    grid = vc.Grid.level(prm, level)
    xi = hl.sample_xi(inputs.SEED, level, 900, n)
    xs = xi.cpu().numpy()
    states = [random_states(grid, 60 + k, 300.0) for k in range(n)]
    olds = [random_states(grid, 70 + k, 300.0) for k in range(n)]
    st = _dev(np.stack([np.stack(a, axis=-1) for a in states]))
    so = _dev(np.stack([np.stack(a, axis=-1) for a in olds]))
    R, J = s.vc_assemble(level, xi, st, so)
    torch.cuda.synchronize()
    R, J = R.cpu().numpy(), J.cpu().numpy()
    for k in range(n):
        coef = cc.coefficients(prm, grid, xs[k])
        (p, c), (po, co) = states[k], olds[k]
        Rm, Rs = vc.residual(prm, grid, coef, p, c, po, co)
        Jo = blocks_from_sparse(vc.jacobian(prm, grid, coef, p, c, po, co), grid)
        fl = vc.face_fluxes(prm, grid, coef, p, c)
        sm = max(max(np.abs(F).max() for _, _, F, _ in fl), vc.residual_scale(prm, grid))
        ss = max(max(np.abs(G).max() for _, _, _, G in fl), vc.residual_scale(prm, grid))
        np.testing.assert_allclose(R[k, ..., 0], Rm, rtol=0, atol=1e-12 * sm)
        np.testing.assert_allclose(R[k, ..., 1], Rs, rtol=0, atol=1e-12 * ss)
        for eq in (0, 1):
            for var in (0, 1):
                sc = np.abs(Jo[..., eq, var]).max()
                np.testing.assert_allclose(J[k, ..., eq, var], Jo[..., eq, var], rtol=0, atol=1e-11 * sc)
    s.close()


def test_vc_assembly_rejects_field_models(hl):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    ny, nx = s.grid(0)
    xi = torch.zeros((1, s.n_xi), dtype=torch.float64, device="cuda")
    st = torch.zeros((1, ny + 1, nx + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hl.HenryError) as e:
        s.vc_assemble(0, xi, st, st)
    assert e.value.code == hl.HENRY_EINVAL
    s.close()


def test_vc_assembly_rejects_inputs_outside_the_model(hl):
    """xi1 = -6 gives phi = 0.35 (1 - 1.2) < 0: the call refuses the batch and
    names the sample instead of assembling from a negative porosity."""
    s = hl.Solver()
    ny, nx = s.grid(0)
    xi = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    xi[1, 0] = -6.0
    st = torch.zeros((3, ny + 1, nx + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hl.HenryError) as e:
        s.vc_assemble(0, xi, st, st)
    assert e.value.code == hl.HENRY_EINVAL and "sample 1" in str(e.value)
    xi[1, 0] = 0.0
    R, _ = s.vc_assemble(0, xi, st, st, with_jacobian=False)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(R).all())
    s.close()


# ---------------------------------------------------------------------------
# The vertex-centred solve (scheme = HENRY_SCHEME_VERTEX) against
# oracle.henry_vc and oracle.mg_vc.  Per-step results agree to rounding:
# J x to 1e-12 of |J| |x|, one V-cycle to 1e-9 of its largest entry; full
# solves' QoIs to relative 1e-10 (both sides stop Newton on the same scaled
# residual and update tests).


def _vc_trajectory_states(level, xi, steps):
    """(x, x_old) of step `steps` of an oracle trajectory: a real Newton
    system's states (p, c pairs, natural vertex order)."""
    prm = vc.Params()
    grid = vc.Grid.level(prm, level)
    coef = cc.coefficients(prm, grid, xi)
    p, c = vc.initial_state(prm, grid)
    for _ in range(steps):
        po, co = p, c
        p, c, ok = vc.newton_step(prm, grid, coef, p, c)
        assert ok
    # perturb the iterate so the system is a mid-Newton one
    j, i = np.meshgrid(np.arange(grid.ny + 1), np.arange(grid.nx + 1), indexing="ij")
    p1 = p + 3.0 * np.sin(0.7 * i + 0.3 * j)
    c1 = np.clip(c + 0.01 * np.cos(0.5 * i - 0.2 * j), 0.0, 1.0)
    p1[:, -1], c1[:, -1] = p[:, -1], c[:, -1]
    c1[:, 0] = 0.0
    return grid, coef, (p1, c1), (po, co)


def _vc_solver(hl, **kw):
    return hl.Solver(scheme=hl.HENRY_SCHEME_VERTEX, **kw)


@pytest.mark.parametrize("level", [0, 1])
def test_vc_apply_jacobian_matches_oracle(hl, level):
    s = _vc_solver(hl)
    prm = vc.Params()
    grid = vc.Grid.level(prm, level)
    xi = inputs.uniform_xi(960 + level, 2)
    states = [random_states(grid, 80 + k, 300.0) for k in range(2)]
    olds = [random_states(grid, 90 + k, 300.0) for k in range(2)]
    x = inputs.rng(961 + level).standard_normal((2, grid.ny + 1, grid.nx + 1, 2))
    y = s.apply_jacobian(level, _dev(xi), _dev(np.stack([np.stack(a, axis=-1) for a in states])),
                         _dev(np.stack([np.stack(a, axis=-1) for a in olds])), _dev(x)).cpu().numpy()
    sc = vc.residual_scale(prm, grid)
    for k in range(2):
        coef = cc.coefficients(prm, grid, xi[k])
        Jo = vc.jacobian(prm, grid, coef, *states[k], *olds[k]) / sc
        yo = (Jo @ x[k].reshape(-1)).reshape(x[k].shape)
        np.testing.assert_allclose(y[k], yo, rtol=0, atol=1e-12 * abs(Jo).max() * np.abs(x[k]).max())
    s.close()


@pytest.mark.parametrize("level,nu", [(0, (2, 2)), (1, (2, 2)), (1, (1, 0)), (0, (0, 1)), (2, (1, 2))])
def test_vc_vcycle_matches_oracle(hl, level, nu):
    """One V-cycle on the vertex hierarchy (four-colour sweeps, full
    weighting with Dirichlet entries zeroed, bilinear prolongation, dense
    coarsest solve) equals oracle.mg_vc.vcycle on the same operators (the
    library scales every level by the fine 1 / (rho0 h^2 / tau), which scales
    the cycle's output by rho0 h^2 / tau)."""
    from oracle import mg_vc
    s = _vc_solver(hl, nu1=nu[0], nu2=nu[1])
    prm = vc.Params()
    xi = inputs.uniform_xi(970 + level, 2)
    st, so, ops = [], [], []
    for k in range(2):
        grid, coef, (p, c), (po, co) = _vc_trajectory_states(level, xi[k], 2 + k)
        st.append(np.stack([p, c], axis=-1))
        so.append(np.stack([po, co], axis=-1))
        ops.append(mg_vc.hierarchy(prm, grid, coef, p, c, po, co))
    b = inputs.rng(971 + level).standard_normal((2, grid.ny + 1, grid.nx + 1, 2))
    z = s.precondition(level, _dev(xi), _dev(np.stack(st)), _dev(np.stack(so)), _dev(b)).cpu().numpy()
    sc = vc.residual_scale(prm, grid)
    for k in range(2):
        zo = sc * mg_vc.vcycle(ops[k], b[k], nu[0], nu[1])
        np.testing.assert_allclose(z[k], zo, rtol=0, atol=1e-9 * np.abs(zo).max())
    s.close()


@pytest.mark.parametrize("level", [1, 4])
def test_vc_linear_solve_reaches_tolerance(hl, level):
    """BiCGStab with the vertex V-cycle: ||b - J x|| <= rtol ||b|| with J the
    oracle's complex-step Jacobian (level 4: 513 x 257 vertices, finalised
    per-sample reductions)."""
    prm = vc.Params()
    grid = vc.Grid.level(prm, level)
    rtol = 1e-8
    s = _vc_solver(hl, lin_rtol=rtol)
    xi = inputs.uniform_xi(980 + level, 1)
    coef = cc.coefficients(prm, grid, xi[0])
    p, c = vc.initial_state(prm, grid)
    j, i = np.meshgrid(np.arange(grid.ny + 1), np.arange(grid.nx + 1), indexing="ij")
    c = np.clip(0.5 * (1 + np.tanh((i * grid.h - 1.4 - 0.4 * j * grid.h) / 0.2)), 0, 1)
    c[:, 0], c[:, -1] = 0.0, 1.0
    p = p + 10.0 * np.sin(np.pi * i * grid.h / 2) * np.cos(np.pi * j * grid.h)
    p[:, -1] = vc.initial_state(prm, grid)[0][:, -1]
    st = np.stack([p, c], axis=-1)[None]
    b = inputs.rng(981 + level).standard_normal((1, grid.ny + 1, grid.nx + 1, 2))
    x, its = s.linear_solve(level, _dev(xi), _dev(st), _dev(st), _dev(b))
    its = its.cpu().numpy()
    assert 0 < its[0] <= s.cfg.lin_maxit
    J = vc.jacobian(prm, grid, coef, p, c, p, c) / vc.residual_scale(prm, grid)
    r = b[0].reshape(-1) - J @ x.cpu().numpy()[0].reshape(-1)
    assert np.linalg.norm(r) <= 1.5 * rtol * np.linalg.norm(b[0])
    s.close()


def _qoi_close(q, ref):
    np.testing.assert_allclose(q[:, 0], ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(q[:, 1], ref[:, 1], rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("precision", [0, 1])
def test_vc_level0_solves_match_oracle(hl, precision):
    prm = vc.Params()
    s = _vc_solver(hl, precision=precision)
    xi = hl.sample_xi(inputs.SEED, 0, 7000, 4)
    q, _, st, stats = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0
    ref = np.array([vc.solve_scenario(prm, 0, x)[0] for x in xi.cpu().numpy()])
    _qoi_close(q.cpu().numpy(), ref)
    assert stats["cell_steps"] == 4 * 512 * 20
    s.close()


def test_vc_level1_with_coarse_partner_matches_oracle(hl):
    prm = vc.Params()
    s = _vc_solver(hl)
    xi = hl.sample_xi(inputs.SEED, 1, 7100, 2)
    qf, qc, st, _ = s.level_batch_solve(1, xi, with_coarse=True)
    assert int(st.abs().sum()) == 0
    x = xi.cpu().numpy()
    _qoi_close(qf.cpu().numpy(), np.array([vc.solve_scenario(prm, 1, v)[0] for v in x]))
    _qoi_close(qc.cpu().numpy(), np.array([vc.solve_scenario(prm, 0, v)[0] for v in x]))
    # the uneven-batch path gives the same bits
    qm, qcm, _, _ = s.batch_solve_mixed(np.array([1, 1], dtype=np.int32), xi, with_coarse=True)
    assert torch.equal(qm, qf) and torch.equal(qcm, qc)
    s.close()


def test_vc_graphs_and_plain_launches_agree(hl):
    xi = hl.sample_xi(inputs.SEED, 1, 7200, 3)
    out = []
    for g in (0, 1):
        s = _vc_solver(hl, cuda_graphs=g)
        out.append(s.level_batch_solve(1, xi)[0])
        s.close()
    assert torch.equal(out[0], out[1])


def test_vc_scheme_rejects_unsupported_settings(hl):
    with pytest.raises(hl.HenryError):
        _vc_solver(hl, coef_model=hl.HENRY_MODEL_KL)
    with pytest.raises(hl.HenryError):
        _vc_solver(hl, qoi_set=hl.HENRY_QOI_PAPER)
    s = _vc_solver(hl)
    xi = hl.sample_xi(inputs.SEED, 0, 0, 1)
    w = torch.tensor([[0.0, 1.0]], dtype=torch.float64, device="cuda")
    with pytest.raises(hl.HenryError):
        s.adjoint(0, xi, w)
    s.close()


def test_vc_residual_first_and_chord_newton(hl):
    """The vertex-centred Newton loop with the residual evaluated alone first
    (bit-identical iterates) and with chord Newton (the Jacobian every 2nd
    iteration; the same discrete solution, against the oracle at 1e-10)."""
    prm = vc.Params()
    xi = hl.sample_xi(inputs.SEED, 0, 7300, 3)
    out = []
    for rf in (-1, 0):
        s = _vc_solver(hl, newton_residual_first=rf)
        q, _, st, stats = s.level_batch_solve(0, xi)
        out.append((q, st, stats["newton_iters"], stats["linear_iters"]))
        s.close()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1]) and out[0][2:] == out[1][2:]
    ref = np.array([vc.solve_scenario(prm, 0, v)[0] for v in xi.cpu().numpy()])
    for kw in (dict(newton_jacobian_every=2, lin_rtol=1e-2), dict(newton_predictor_order=1)):
        s = _vc_solver(hl, **kw)  # chord Newton; the linear time predictor (the default is quadratic)
        q, _, st, _ = s.level_batch_solve(0, xi)
        assert int(st.abs().sum()) == 0
        _qoi_close(q.cpu().numpy(), ref)
        s.close()


def test_vc_level_tuning_applies_and_autotune_runs(hl):
    """A level's tuning (henry_set_tuning, henry_autotune) governs the
    vertex-centred solve as it does the cell-centred one: with lin_rtol 1e-2
    and the Jacobian every 2nd iteration set as level 0's tuning, the solve
    takes that path (fewer BiCGStab iterations than the configuration's
    settings) and still reaches the oracle's QoIs at 1e-10; the autotuner
    returns a setting that solves every trial sample."""
    prm = vc.Params()
    xi = hl.sample_xi(inputs.SEED, 0, 7400, 3)
    s = _vc_solver(hl)
    _, _, _, plain = s.level_batch_solve(0, xi)
    s.set_tuning(0, dict(s.tuning(0), lin_rtol=1e-2, newton_jacobian_every=2))
    q, _, st, tuned = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0
    assert tuned["linear_iters"] < plain["linear_iters"], (tuned, plain)
    _qoi_close(q.cpu().numpy(), np.array([vc.solve_scenario(prm, 0, v)[0] for v in xi.cpu().numpy()]))
    s.set_tuning(0, None)
    t = s.autotune(0, hl.sample_xi(inputs.SEED, 0, 7500, 64))
    assert t["cell_steps_per_s"] > 0 and t["mg_tail_cells"] == s.cfg.mg_tail_cells
    q, _, st, _ = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0
    _qoi_close(q.cpu().numpy(), np.array([vc.solve_scenario(prm, 0, v)[0] for v in xi.cpu().numpy()]))
    s.close()


@pytest.mark.parametrize("level", [0, 2])
def test_vc_face_once_assembly_matches_per_vertex_kernel_and_oracle(hl, level):
    """The face-once tile assembly (the default: each element face evaluated
    once by its source vertex and shared through shared memory, faces of
    neighbours outside the CTA's range evaluated again) against the
    one-thread-per-vertex kernel (tile_assembly = 0) and the oracle.  Level 2
    (129 x 65 vertices) has CTA ranges that cut rows, so both the shared and
    the re-evaluated neighbour faces are taken.  The two kernels add the same
    faces in the same order; the compiler may contract multiply-adds
    differently in each, so they are compared at 1e-14 of each quantity's
    scale, the oracle at the assembly tests' tolerances.  The residual alone
    (with_jacobian False) equals the residual assembled with the Jacobian."""
    prm = vc.Params()
    grid = vc.Grid.level(prm, level)
    xi = inputs.uniform_xi(990 + level, 3)
    states = [random_states(grid, 100 + k, 300.0) for k in range(3)]
    olds = [random_states(grid, 110 + k, 300.0) for k in range(3)]
    st = _dev(np.stack([np.stack(a, axis=-1) for a in states]))
    so = _dev(np.stack([np.stack(a, axis=-1) for a in olds]))
    a, b = _vc_solver(hl), _vc_solver(hl, tile_assembly=0)
    Fa, Ja = a.assemble(level, _dev(xi), st, so)
    Fb, Jb = b.assemble(level, _dev(xi), st, so)
    Fr, _ = a.assemble(level, _dev(xi), st, so, with_jacobian=False)
    assert torch.equal(Fr, Fa)
    Fa, Ja, Fb, Jb = (t.cpu().numpy() for t in (Fa, Ja, Fb, Jb))
    for eq in (0, 1):
        np.testing.assert_allclose(Fa[..., eq], Fb[..., eq], rtol=0, atol=1e-14 * np.abs(Fb[..., eq]).max())
    for q in range(9):
        for eq in (0, 1):
            for var in (0, 1):
                sc = np.abs(Jb[..., q, eq, var]).max()
                np.testing.assert_allclose(Ja[..., q, eq, var], Jb[..., q, eq, var], rtol=0,
                                           atol=1e-14 * max(sc, 1e-300))
    sc = vc.residual_scale(prm, grid)
    for k in range(3):
        coef = cc.coefficients(prm, grid, xi[k])
        (p, c), (po, co) = states[k], olds[k]
        Rm, Rs = vc.residual(prm, grid, coef, p, c, po, co)
        Jo = blocks_from_sparse(vc.jacobian(prm, grid, coef, p, c, po, co), grid) / sc
        fl = vc.face_fluxes(prm, grid, coef, p, c)
        sm = max(max(np.abs(F).max() for _, _, F, _ in fl), sc)
        ss = max(max(np.abs(G).max() for _, _, _, G in fl), sc)
        np.testing.assert_allclose(Fa[k, ..., 0], Rm / sc, rtol=0, atol=1e-12 * sm / sc)
        np.testing.assert_allclose(Fa[k, ..., 1], Rs / sc, rtol=0, atol=1e-12 * ss / sc)
        for eq in (0, 1):
            for var in (0, 1):
                scj = np.abs(Jo[..., eq, var]).max()
                np.testing.assert_allclose(Ja[k].reshape(Jo.shape)[..., eq, var], Jo[..., eq, var], rtol=0,
                                           atol=1e-11 * scj)
    a.close()
    b.close()
