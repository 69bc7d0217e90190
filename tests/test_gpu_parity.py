"""GPU parity: every step of the CUDA path, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances (FP64 path): per-step results agree to rounding (rtol 1e-11 on
residual/Jacobian entries relative to the entry scale of the block row;
1e-9 on a V-cycle, which multiplies rounding differences by the operator's
amplification); QoIs of full scenario solves agree to 1e-10 relative, both the salt mass
and c at the point (a 1e-14 absolute floor only guards values near zero,
which c(1.5, 0.25) never takes: over the input cube it stays above 0.1):
both sides converge every Newton solve to the stopping rule's 1e-11 /
1e-12, far below that.  Philox xi and all index work are bit-exact.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry
from oracle import mg as omg
from oracle import mlmc as omlmc
from oracle import philox as ophilox
from paper_2302_07804_gb300 import inputs

PRM = ohenry.Params()
DEV = "cuda"


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
    yield s
    s.close()


def _to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _states_np(p, c):
    return np.stack([p, c], axis=-1)


@pytest.mark.parametrize("level,first", [(0, 0), (3, 12345), (5, (1 << 32) - 3)])
def test_sample_xi_bit_exact(hl, level, first):
    n = 257
    xi = hl.sample_xi(inputs.SEED, level, first, n).cpu().numpy()
    ref = ophilox.sample_xi(inputs.SEED, level, first, n)
    assert np.array_equal(xi.view(np.uint64), ref.view(np.uint64))


def _random_case(tag, level, n):
    grid = ohenry.Grid.level(PRM, level)
    xi = inputs.uniform_xi(tag, n)
    p, c = inputs.random_states(tag, 2 * n, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    return grid, xi, p[:n], c[:n], p[n:], c[n:]


@pytest.mark.parametrize("level", [0, 1])
def test_assemble_residual_and_jacobian(solver, level):
    n = 3
    grid, xi, p, c, po, co = _random_case(100 + level, level, n)
    F, J = solver.assemble(level, _to_dev(xi), _to_dev(_states_np(p, c)), _to_dev(_states_np(po, co)))
    F, J = F.cpu().numpy(), J.cpu().numpy()
    s = ohenry.residual_scale(PRM, grid)
    for i in range(n):
        coef = ohenry.coefficients(PRM, grid, xi[i])
        Rm, Rs = ohenry.residual(PRM, grid, coef, p[i], c[i], po[i], co[i])
        Jo = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p[i], c[i], po[i], co[i]), grid.nx, grid.ny) / s
        Fo = np.stack([Rm, Rs], axis=-1) / s
        # residual: cancellation of O(1e2) face fluxes -> compare to the flux scale
        fscale = np.abs(Jo[..., 0, :, 0]).max() * 300.0 + 1.0
        np.testing.assert_allclose(F[i], Fo, rtol=0, atol=1e-12 * fscale)
        for eq in range(2):
            for var in range(2):
                row_scale = np.abs(Jo[..., eq, var]).max()
                np.testing.assert_allclose(J[i][..., eq, var], Jo[..., eq, var], rtol=0, atol=1e-11 * row_scale)


def test_assemble_mixed_precision_blocks(hl):
    s32 = hl.Solver(precision=hl.HENRY_MIXED)
    grid, xi, p, c, po, co = _random_case(120, 0, 2)
    F, J = s32.assemble(0, _to_dev(xi), _to_dev(_states_np(p, c)), _to_dev(_states_np(po, co)))
    s = ohenry.residual_scale(PRM, grid)
    coef = ohenry.coefficients(PRM, grid, xi[0])
    Jo = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p[0], c[0], po[0], co[0]), grid.nx, grid.ny) / s
    J = J.cpu().numpy()[0]
    for eq in range(2):
        for var in range(2):
            np.testing.assert_allclose(J[..., eq, var], Jo[..., eq, var], rtol=0,
                                       atol=1e-6 * np.abs(Jo[..., eq, var]).max())
    Fo = np.stack(ohenry.residual(PRM, grid, coef, p[0], c[0], po[0], co[0]), axis=-1) / s
    np.testing.assert_allclose(F.cpu().numpy()[0], Fo, rtol=0, atol=1e-9 * np.abs(Fo).max())  # F stays FP64
    s32.close()


@pytest.mark.parametrize("level", [0, 2])
def test_apply_jacobian(solver, level):
    n = 2
    grid, xi, p, c, po, co = _random_case(130 + level, level, n)
    x = inputs.random_vectors(131, n, grid.ny, grid.nx)
    y = solver.apply_jacobian(level, _to_dev(xi), _to_dev(_states_np(p, c)), _to_dev(_states_np(po, co)),
                              _to_dev(x)).cpu().numpy()
    s = ohenry.residual_scale(PRM, grid)
    for i in range(n):
        coef = ohenry.coefficients(PRM, grid, xi[i])
        J = ohenry.jacobian(PRM, grid, coef, p[i], c[i], po[i], co[i]) / s
        yo = (J @ x[i].ravel()).reshape(grid.ny, grid.nx, 2)
        scale = np.abs(J).max() * np.abs(x[i]).max()
        np.testing.assert_allclose(y[i], yo, rtol=0, atol=1e-12 * scale)


def _trajectory(level, xi, steps):
    grid = ohenry.Grid.level(PRM, level)
    coef = ohenry.coefficients(PRM, grid, xi)
    p, c = ohenry.initial_state(PRM, grid)
    for _ in range(steps):
        p, c, ok = ohenry.newton_step(PRM, grid, coef, p, c)
        assert ok
    return grid, coef, p, c


@pytest.mark.parametrize("level,coarse_op", [(0, 0), (1, 0), (0, 1)])
def test_vcycle_matches_oracle(hl, level, coarse_op):
    s = hl.Solver(coarse_op=coarse_op)
    xi = inputs.uniform_xi(140 + level, 2)
    states, olds, ops = [], [], []
    for i in range(2):
        grid, coef, p, c = _trajectory(level, xi[i], 2 + i)
        # Jacobian at a perturbed iterate of the next step
        p1 = p + 5.0 * np.sin(np.arange(p.size).reshape(p.shape))
        c1 = np.clip(c + 0.01, 0, 1)
        states.append(_states_np(p1, c1))
        olds.append(_states_np(p, c))
        if coarse_op == 0:
            ops.append(omg.rediscretised_hierarchy(PRM, grid, coef, p1, c1, p, c))
        else:
            A0 = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p1, c1, p, c), grid.nx, grid.ny)
            ops.append(omg.galerkin_hierarchy(A0 / ohenry.residual_scale(PRM, grid)))
    b = inputs.random_vectors(141, 2, grid.ny, grid.nx)
    z = s.precondition(level, _to_dev(xi), _to_dev(np.stack(states)), _to_dev(np.stack(olds)), _to_dev(b))
    z = z.cpu().numpy()
    for i in range(2):
        zo = omg.vcycle(ops[i], b[i], s.cfg.nu1, s.cfg.nu2)
        np.testing.assert_allclose(z[i], zo, rtol=0, atol=1e-9 * np.abs(zo).max())
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_linear_solve_reaches_tolerance(hl, precision):
    s = hl.Solver(precision=precision, lin_rtol=1e-8 if precision == 0 else 1e-5)
    level = 1
    xi = inputs.uniform_xi(150, 2)
    states, olds, Js = [], [], []
    for i in range(2):
        grid, coef, p, c = _trajectory(level, xi[i], 3)
        states.append(_states_np(p, c))
        olds.append(_states_np(p, c))
        Js.append(ohenry.jacobian(PRM, grid, coef, p, c, p, c) / ohenry.residual_scale(PRM, grid))
    b = inputs.random_vectors(151, 2, grid.ny, grid.nx)
    x, its = s.linear_solve(level, _to_dev(xi), _to_dev(np.stack(states)), _to_dev(np.stack(olds)), _to_dev(b))
    x, its = x.cpu().numpy(), its.cpu().numpy()
    assert np.all(its > 0) and np.all(its <= 20), its
    for i in range(2):
        r = b[i].ravel() - Js[i] @ x[i].ravel()
        rel = np.linalg.norm(r) / np.linalg.norm(b[i])
        assert rel <= (1.5e-8 if precision == 0 else 5e-5), rel
        xd = spla.spsolve(Js[i].tocsc(), b[i].ravel())
        assert np.abs(x[i].ravel() - xd).max() <= (1e-5 if precision == 0 else 1e-2) * np.abs(xd).max()
    s.close()


def _qoi_check(q_gpu, q_ref):
    np.testing.assert_allclose(q_gpu[:, 0], q_ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(q_gpu[:, 1], q_ref[:, 1], rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("fused,precision", [(2, 0), (0, 0), (1, 1), (0, 1)])
def test_level0_batch_solve_matches_oracle(hl, fused, precision):
    """Level 0 through the fused one-CTA-per-sample solver and through the
    multi-kernel path, in FP64 and mixed precision."""
    solver = hl.Solver(fused_small_grids=fused, precision=precision)
    n = 16
    xi_d = hl.sample_xi(inputs.SEED, 0, 0, n)
    qf, qc, st, stats = solver.level_batch_solve(0, xi_d)
    assert int(st.abs().sum()) == 0
    xi = xi_d.cpu().numpy()
    ref, ok = ohenry.solve_scenarios(PRM, 0, xi)
    assert ok.all()
    _qoi_check(qf.cpu().numpy(), ref)
    assert stats["cell_steps"] == n * 512 * 20
    assert stats["newton_iters"] >= n * 20 and stats["linear_iters"] > 0
    solver.close()


def test_fused_and_multikernel_paths_agree(hl):
    n = 40
    xi_d = hl.sample_xi(inputs.SEED, 0, 300, n)
    a = hl.Solver(fused_small_grids=2)
    b = hl.Solver(fused_small_grids=0)
    qa, _, sa, _ = a.level_batch_solve(0, xi_d)
    qb, _, sb, _ = b.level_batch_solve(0, xi_d)
    assert int(sa.abs().sum()) == 0 and int(sb.abs().sum()) == 0
    _qoi_check(qa.cpu().numpy(), qb.cpu().numpy())
    a.close()
    b.close()


def test_level1_with_coarse_partner(hl, solver):
    n = 3
    xi_d = hl.sample_xi(inputs.SEED, 1, 40, n)
    qf, qc, st, stats = solver.level_batch_solve(1, xi_d, with_coarse=True)
    assert int(st.abs().sum()) == 0
    xi = xi_d.cpu().numpy()
    ref1, _ = ohenry.solve_scenarios(PRM, 1, xi)
    ref0, _ = ohenry.solve_scenarios(PRM, 0, xi)
    _qoi_check(qf.cpu().numpy(), ref1)
    _qoi_check(qc.cpu().numpy(), ref0)
    # the coarse partner equals an independent level-0 solve of the same xi, bit for bit
    q0, _, _, _ = solver.level_batch_solve(0, xi_d)
    assert torch.equal(q0, qc)
    assert stats["cell_steps"] == n * (2048 * 40 + 512 * 20)


def test_mixed_precision_solve_matches_oracle(hl):
    s = hl.Solver(precision=hl.HENRY_MIXED, lin_rtol=1e-4)
    n = 8
    xi_d = hl.sample_xi(inputs.SEED, 0, 100, n)
    qf, _, st, _ = s.level_batch_solve(0, xi_d)
    assert int(st.abs().sum()) == 0
    ref, _ = ohenry.solve_scenarios(PRM, 0, xi_d.cpu().numpy())
    _qoi_check(qf.cpu().numpy(), ref)   # Newton on the FP64 residual reaches the same solution
    s.close()


def test_galerkin_option_solve_matches_oracle(hl):
    s = hl.Solver(coarse_op=hl.HENRY_COARSE_GALERKIN)
    xi_d = hl.sample_xi(inputs.SEED, 0, 200, 4)
    qf, _, st, _ = s.level_batch_solve(0, xi_d)
    assert int(st.abs().sum()) == 0
    ref, _ = ohenry.solve_scenarios(PRM, 0, xi_d.cpu().numpy())
    _qoi_check(qf.cpu().numpy(), ref)
    s.close()


def test_mlmc_accumulate_matches_two_pass(hl):
    gen = inputs.rng(160)
    qf = gen.normal(0.5, 0.1, size=(1000, 2))
    qc = qf + gen.normal(0.0, 0.01, size=(1000, 2))
    status = np.zeros(1000, dtype=np.int32)
    status[::97] = 1
    sums = torch.zeros((2, 2, 3), dtype=torch.float64, device=DEV)
    st = torch.as_tensor(status, device=DEV)
    # two batches merged must equal one two-pass computation over the union
    hl.mlmc_accumulate(1, _to_dev(qf[:600]), _to_dev(qc[:600]), st[:600], sums)
    hl.mlmc_accumulate(1, _to_dev(qf[600:]), _to_dev(qc[600:]), st[600:], sums)
    keep = status == 0
    y = omlmc.level_differences(qf[keep], qc[keep])
    n, mean, m2 = omlmc.two_pass_moments(y)
    S = sums.cpu().numpy()
    assert S[0, 0, 0] == n
    np.testing.assert_allclose(S[0, :, 1], mean, rtol=1e-13)
    np.testing.assert_allclose(S[0, :, 2], m2, rtol=1e-10)
    n1, mean1, m21 = omlmc.two_pass_moments(qf[keep])
    np.testing.assert_allclose(S[1, :, 1], mean1, rtol=1e-13)
    np.testing.assert_allclose(S[1, :, 2], m21, rtol=1e-10)


def test_nan_input_reports_nonfinite_status(hl, solver):
    xi = hl.sample_xi(inputs.SEED, 0, 0, 4)
    xi[2, 1] = float("nan")
    qf, _, st, stats = solver.level_batch_solve(0, xi, allow_failures=True)
    st = st.cpu().numpy()
    assert st[2] == hl.HENRY_SAMPLE_NONFINITE
    assert (st[[0, 1, 3]] == 0).all()
    assert stats["failed_samples"] == 1


def test_newton_cap_reports_newton_status(hl):
    s = hl.Solver(newton_maxit=1)
    xi = hl.sample_xi(inputs.SEED, 0, 0, 2)
    _, _, st, stats = s.level_batch_solve(0, xi, allow_failures=True)
    assert (st.cpu().numpy() == hl.HENRY_SAMPLE_NEWTON).all()
    with pytest.raises(hl.HenryError) as e:
        s.level_batch_solve(0, xi)
    assert e.value.code == hl.HENRY_ENOCONV
    s.close()


@pytest.mark.parametrize("level", [2, 3])
def test_full_size_batch_sampled_against_oracle(hl, solver, level):
    """Level-l batch of the MLMC workload's size in the same launch
    configuration; one sampled scenario is recomputed by the oracle."""
    n = {2: 64, 3: 32}[level]
    xi_d = hl.sample_xi(inputs.SEED, level, 0, n)
    qf, qc, st, _ = solver.level_batch_solve(level, xi_d, with_coarse=True)
    assert int(st.abs().sum()) == 0
    q = qf.cpu().numpy()
    qcn = qc.cpu().numpy()
    # properties that hold at any size
    assert np.all((q[:, 1] >= -1e-12) & (q[:, 1] <= 1 + 1e-12))
    assert np.all(q[:, 0] > 0)
    assert np.abs(q[:, 1] - qcn[:, 1]).max() < 0.1   # level differences are small
    i = n // 2
    ref, ok = ohenry.solve_scenarios(PRM, level, xi_d[i:i + 1].cpu().numpy())
    assert ok.all()
    _qoi_check(q[i:i + 1], ref)


def test_finalized_reductions_give_identical_results(hl):
    """The per-sample reduction kernel used on large grids sums the partials in
    the same order as the consumer kernels, so the QoIs are bit-identical."""
    xi_d = hl.sample_xi(inputs.SEED, 2, 700, 3)
    a = hl.Solver(finalize_nct=1)
    b = hl.Solver(finalize_nct=0)
    qa, _, sa, _ = a.level_batch_solve(2, xi_d)
    qb, _, sb, _ = b.level_batch_solve(2, xi_d)
    assert int(sa.abs().sum()) == 0 and int(sb.abs().sum()) == 0
    assert torch.equal(qa, qb)
    a.close()
    b.close()


def test_cuda_graphs_give_identical_results(hl):
    """The BiCGStab iteration body replayed from a captured CUDA graph runs
    the same kernels with the same arguments as plain launches: QoIs,
    statuses and adjoint gradients are bit-identical (FP64 with coarse
    partners, mixed precision on the multi-kernel path, KL inputs that need
    the fallback preconditioner, the adjoint's transposed solves)."""
    import os
    xi1 = hl.sample_xi(inputs.SEED, 1, 730, 5)
    xi0 = hl.sample_xi(inputs.SEED, 0, 731, 7)
    th = torch.as_tensor(np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "kl_hard_inputs.txt")),
                         dtype=torch.float64, device="cuda")
    w = torch.tensor([[0.01, 1.0]] * 7, dtype=torch.float64, device="cuda")
    cases = [({}, 1, xi1, True), ({"precision": 1, "fused_small_grids": 0}, 0, xi0, False),
             ({"coef_model": hl.HENRY_MODEL_KL}, 0, th, False)]
    for kw, level, xi, wc in cases:
        out = []
        for g in (0, 1):
            s = hl.Solver(cuda_graphs=g, **kw)
            qf, qc, st, _ = s.level_batch_solve(level, xi, with_coarse=wc)
            out.append((qf, qc, st))
            s.close()
        assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][2], out[1][2])
        if wc:
            assert torch.equal(out[0][1], out[1][1])
    grads = []
    for g in (0, 1):
        s = hl.Solver(cuda_graphs=g)
        grads.append(s.adjoint(0, xi0, w, checkpoint_every=6)[0])
        s.close()
    assert torch.equal(grads[0], grads[1])


@pytest.mark.parametrize("model", [0, 1])
def test_tile_assembly_equals_per_cell_assembly_on_wide_grids(hl, model):
    """Grids wider than 256 cells (level 4: 512 x 256) are assembled face-once
    in 128 x 2 tiles with halo faces on the tiles' west and south edges; the
    residual and every Jacobian block equal the per-cell form's to rounding,
    for the three-parameter and the KL model, and full solves agree."""
    level, n = 4, 2
    if model == 1:
        gen = inputs.rng(860)
        xi = torch.as_tensor(np.concatenate([gen.standard_normal((n, 64)), gen.uniform(-1, 1, (n, 1))], axis=1),
                             dtype=torch.float64, device="cuda")
    else:
        xi = hl.sample_xi(inputs.SEED, level, 860, n)
    grid = ohenry.Grid.level(PRM, level)
    p, c = inputs.random_states(861, 2 * n, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    st = torch.as_tensor(np.stack([p[:n], c[:n]], axis=-1), dtype=torch.float64, device="cuda")
    so = torch.as_tensor(np.stack([p[n:], c[n:]], axis=-1), dtype=torch.float64, device="cuda")
    out = []
    for tile in (1, 0):
        s = hl.Solver(coef_model=model, tile_assembly=tile)
        F, J = s.assemble(level, xi, st, so)
        out.append((F.cpu().numpy(), J.cpu().numpy()))
        s.close()
    (F1, J1), (F0, J0) = out
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-12 * np.abs(F0).max())
    for k in range(5):
        np.testing.assert_allclose(J1[..., k, :, :], J0[..., k, :, :], rtol=0,
                                   atol=1e-12 * np.abs(J0[..., k, :, :]).max())
    if model == 0:
        q = []
        for tile in (1, 0):
            s = hl.Solver(tile_assembly=tile)
            q.append(s.level_batch_solve(level, xi)[0].cpu().numpy())
            s.close()
        np.testing.assert_allclose(q[0][:, 0], q[1][:, 0], rtol=1e-11, atol=0)
        np.testing.assert_allclose(q[0][:, 1], q[1][:, 1], rtol=0, atol=1e-11)


@pytest.mark.parametrize("level,model,tile,precision", [(0, 0, 1, 0), (1, 1, 1, 0), (4, 0, 1, 0), (0, 0, 0, 0),
                                                        (2, 2, 1, 0), (1, 0, 1, 1)])
def test_residual_only_kernel_is_bit_identical(hl, level, model, tile, precision):
    """The residual-only assembly (the Newton test's first evaluation from
    iteration newton_residual_first on) gives the same bits as the residual
    assembled with the Jacobian: whole-row tiles, 128 x 2 tiles (level 4), the
    per-cell form, the KL and two-layer models, FP64 and mixed precision."""
    s = hl.Solver(coef_model=model, tile_assembly=tile, precision=precision)
    grid = ohenry.Grid.level(PRM, level)
    n = 3
    if model == hl.HENRY_MODEL_KL:
        gen = inputs.rng(870 + level)
        xi = np.concatenate([gen.standard_normal((n, 64)), gen.uniform(-1, 1, (n, 1))], axis=1)
    else:
        xi = inputs.uniform_xi(870 + level, n)
    p, c = inputs.random_states(871 + level, 2 * n, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    st, so = _to_dev(_states_np(p[:n], c[:n])), _to_dev(_states_np(p[n:], c[n:]))
    F1, J1 = s.assemble(level, _to_dev(xi), st, so, with_jacobian=True)
    F0, J0 = s.assemble(level, _to_dev(xi), st, so, with_jacobian=False)
    assert J0 is None and J1 is not None
    assert torch.equal(F0, F1)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_first_newton_gives_identical_solves(hl, precision):
    """Evaluating the residual alone before assembling the Jacobian changes
    no iterate: QoIs, statuses and iteration counts are bit-identical with
    the option on (from iteration 0, from 2) and off."""
    xi = hl.sample_xi(inputs.SEED, 1, 4400, 6)
    out = []
    for rf in (-1, 0, 2):
        s = hl.Solver(precision=precision, fused_small_grids=0, newton_residual_first=rf)
        qf, qc, st, stats = s.level_batch_solve(1, xi, with_coarse=True)
        out.append((qf, qc, st, stats["newton_iters"], stats["linear_iters"]))
        s.close()
    for o in out[1:]:
        assert torch.equal(o[0], out[0][0]) and torch.equal(o[1], out[0][1]) and torch.equal(o[2], out[0][2])
        assert o[3:] == out[0][3:]


@pytest.mark.parametrize("precision", [0, 1])
def test_fused_multigrid_tail_is_bit_identical(hl, precision):
    """The V-cycle's coarse levels run as one kernel per cycle (one CTA per
    sample, operators in shared memory) compute exactly what the level-by-
    level kernels compute: one V-cycle at levels 0, 2 and 4 and full solves
    with coarse partners are bit-identical with the tail on (from 4 x 2, 8 x
    4, 16 x 8 and 32 x 16 cells, and from 64 x 32 cells, whose block planes
    do not fit in shared memory beside the vectors and are read from global
    memory) and off."""
    for level in (0, 2, 4):
        n = 5 if level < 4 else 2
        grid, xi, p, c, po, co = _random_case(880 + level, level, n)
        b = inputs.random_vectors(881 + level, n, grid.ny, grid.nx)
        zs = []
        for tail in (0, 8, 32, 128, 512, 2048):
            s = hl.Solver(mg_tail_cells=tail, precision=precision)
            zs.append(s.precondition(level, _to_dev(xi), _to_dev(_states_np(p, c)), _to_dev(_states_np(po, co)),
                                     _to_dev(b)))
            s.close()
        for z in zs[1:]:
            assert torch.equal(z, zs[0]), level
    xi = hl.sample_xi(inputs.SEED, 2, 5100, 4)
    q = []
    for tail in (0, 32, 128, 2048):
        s = hl.Solver(mg_tail_cells=tail, precision=precision, fused_small_grids=0, mg_tail_batch_cells=0)
        qf, qc, st, stats = s.level_batch_solve(2, xi, with_coarse=True)
        q.append((qf, qc, st, stats["linear_iters"]))
        s.close()
    for o in q[1:]:
        assert torch.equal(q[0][0], o[0]) and torch.equal(q[0][1], o[1]) and torch.equal(q[0][2], o[2])
        assert q[0][3] == o[3]


@pytest.mark.parametrize("precision", [0, 1])
def test_multigrid_cta_size_and_tile_shape_are_bit_identical(hl, precision):
    """The smoother, restriction and prolongation kernels' CTA size
    (mg_threads) changes only which CTA and thread does a cell's arithmetic:
    one V-cycle at levels 1 and 3 and level-2 solves with coarse partners are
    bit-identical, with the setting in the configuration and as a level's
    tuning on one handle (so that BiCGStab graphs captured under one setting
    are not replayed under another).  The assembly tile (assembly_tile_w)
    evaluates each face with the same source arithmetic at another call site,
    where the compiler may contract multiply-adds into FMAs differently: its
    solves are compared at relative 1e-12 on the QoIs."""
    for level in (1, 3):
        grid, xi, p, c, po, co = _random_case(890 + level, level, 2)
        b = inputs.random_vectors(891 + level, 2, grid.ny, grid.nx)
        zs = []
        for nt in (0, 64, 128, 512):
            s = hl.Solver(mg_threads=nt, mg_tail_cells=0, precision=precision)
            zs.append(s.precondition(level, _to_dev(xi), _to_dev(_states_np(p, c)), _to_dev(_states_np(po, co)),
                                     _to_dev(b)))
            s.close()
        for z in zs[1:]:
            assert torch.equal(z, zs[0]), level
    xi = hl.sample_xi(inputs.SEED, 2, 5200, 4)

    def run(s):
        qf, qc, st, stats = s.level_batch_solve(2, xi, with_coarse=True)
        assert int(st.abs().sum()) == 0
        return qf, qc, stats["newton_iters"], stats["linear_iters"]

    def same(a, b, what, tiles):
        if tiles:
            for x, y in ((a[0], b[0]), (a[1], b[1])):
                assert torch.allclose(x, y, rtol=1e-12, atol=0), what
        else:
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and a[2:] == b[2:], what

    s = hl.Solver(precision=precision, fused_small_grids=0)
    ref = run(s)
    s.close()
    for kw in (dict(mg_threads=128), dict(mg_threads=64, mg_tail_cells=0), dict(mg_threads=512, assembly_tile_w=32),
               dict(assembly_tile_w=64, mg_tail_cells=0)):
        s = hl.Solver(precision=precision, fused_small_grids=0, **kw)
        same(run(s), ref, kw, "assembly_tile_w" in kw)
        s.close()
    s = hl.Solver(precision=precision, fused_small_grids=0)
    for kw in (dict(mg_threads=128), dict(mg_tail_cells=0), dict(mg_threads=512, assembly_tile_w=32)):
        for lv in (1, 2):
            s.set_tuning(lv, dict(s.tuning(lv), **kw))
        same(run(s), ref, ("tuning", kw), "assembly_tile_w" in s.tuning(2) and s.tuning(2)["assembly_tile_w"] > 0)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_linear_predictor_reaches_the_oracle_solution(hl, precision):
    """The default predictor of Newton's first iterate is quadratic in time
    (newton_predictor_order 2, which every other test runs); the linear one
    (order 1) converges to the same discrete solution: level-1 solves with
    coarse partners and level-0 solves (the fused small-grid solver in mixed
    precision) against the oracle at relative 1e-10, set in the
    configuration, and level-2 solves with it set as a level's tuning."""
    xi = hl.sample_xi(inputs.SEED, 1, 4700, 3)
    s = hl.Solver(newton_predictor_order=1, precision=precision)
    qf, qc, st, _ = s.level_batch_solve(1, xi, with_coarse=True)
    q0, _, st0, _ = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0 and int(st0.abs().sum()) == 0
    x = xi.cpu().numpy()
    ref1, _ = ohenry.solve_scenarios(PRM, 1, x)
    ref0, _ = ohenry.solve_scenarios(PRM, 0, x)
    _qoi_check(qf.cpu().numpy(), ref1)
    _qoi_check(qc.cpu().numpy(), ref0)
    _qoi_check(q0.cpu().numpy(), ref0)
    s.close()
    t = hl.Solver(precision=precision)
    for lv in (1, 2):
        t.set_tuning(lv, dict(t.tuning(lv), newton_predictor_order=1))
    xi2 = hl.sample_xi(inputs.SEED, 2, 4720, 2)
    q2, q1, st2, _ = t.level_batch_solve(2, xi2, with_coarse=True)
    assert int(st2.abs().sum()) == 0
    x2 = xi2.cpu().numpy()
    ref2, _ = ohenry.solve_scenarios(PRM, 2, x2)
    ref1b, _ = ohenry.solve_scenarios(PRM, 1, x2)
    _qoi_check(q2.cpu().numpy(), ref2)
    _qoi_check(q1.cpu().numpy(), ref1b)
    t.close()


@pytest.mark.parametrize("every,precision", [(2, 0), (3, 0), (2, 1)])
def test_chord_newton_reaches_the_oracle_solution(hl, every, precision):
    """Chord Newton (the Jacobian and coarse operators re-assembled every
    k-th iteration of a step, the residual alone in between) converges to the
    same discrete solution: level-1 solves with coarse partners against the
    oracle at relative 1e-10, FP64 and mixed precision (multi-kernel path)."""
    s = hl.Solver(newton_jacobian_every=every, precision=precision, fused_small_grids=0)
    xi = hl.sample_xi(inputs.SEED, 1, 4600, 3)
    qf, qc, st, stats = s.level_batch_solve(1, xi, with_coarse=True)
    assert int(st.abs().sum()) == 0
    x = xi.cpu().numpy()
    ref1, _ = ohenry.solve_scenarios(PRM, 1, x)
    ref0, _ = ohenry.solve_scenarios(PRM, 0, x)
    _qoi_check(qf.cpu().numpy(), ref1)
    _qoi_check(qc.cpu().numpy(), ref0)
    s.close()
