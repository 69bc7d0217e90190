"""The paper's QoIs on the GPU (qoi_set PAPER / PAPER_FIELD) against the
oracle: salt mass, c(1.5, 0.25), c at the 12 points of Eq. (12points) and the
level-0 c field at 1e-10; the freshwater integral Q_FW of Eq. (integral_fw)
exactly, up to one cell area per cell whose oracle mass fraction lies within
1e-9 of the threshold 0.012178 (the two sides' states differ by ~1e-12, so
only such cells can fall on different sides).  Also the paper's preset (T =
6016 s in 188 steps, two-layer porosity), MLMC accumulation of the 527 QoIs
(mean and variance fields), uneven batches and the adjoint with wider QoI rows."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry
from oracle import mlmc as omlmc
from paper_2302_07804_gb300 import inputs


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _check_paper_qois(q_gpu, prm, level, xis, model, qoi_set):
    grid = ohenry.Grid.level(prm, level)
    for i, xi in enumerate(xis):
        q_ref, ok, (p, c) = ohenry.solve_scenario(prm, level, xi, return_state=True, model=model, qoi_set=qoi_set)
        assert ok
        g = q_gpu[i]
        assert g.shape == q_ref.shape
        assert abs(g[0] - q_ref[0]) <= 1e-10 * abs(q_ref[0])
        np.testing.assert_allclose(g[1], q_ref[1], rtol=0, atol=1e-10)
        near = int(np.count_nonzero(np.abs(c - ohenry.C_FRESH) < 1e-9))
        assert abs(g[2] - q_ref[2]) <= near * grid.h * grid.h + 1e-15
        np.testing.assert_allclose(g[3:], q_ref[3:], rtol=0, atol=1e-10)


@pytest.mark.parametrize("level", [0, 1])
def test_paper_qoi_sets_match_oracle(hl, level):
    xi = hl.sample_xi(inputs.SEED, level, 640, 3)
    s2 = hl.Solver(qoi_set=hl.HENRY_QOI_PAPER_FIELD)
    q2, _, st, _ = s2.level_batch_solve(level, xi)
    assert int(st.abs().sum()) == 0 and q2.shape == (3, 15 + 512)
    _check_paper_qois(q2.cpu().numpy(), ohenry.Params(), level, xi.cpu().numpy(), "uniform3", 2)
    s0 = hl.Solver()
    q0, _, _, _ = s0.level_batch_solve(level, xi)
    assert torch.equal(q0, q2[:, :2])
    s1 = hl.Solver(qoi_set=hl.HENRY_QOI_PAPER)
    q1, _, _, _ = s1.level_batch_solve(level, xi)
    assert torch.equal(q1, q2[:, :15])
    for s in (s0, s1, s2):
        s.close()


def test_paper_preset_matches_oracle(hl):
    s = hl.Solver(**hl.paper_config())
    xi = hl.sample_xi(inputs.SEED, 0, 650, 3)
    q, _, st, _ = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0 and q.shape == (3, 15)
    _check_paper_qois(q.cpu().numpy(), ohenry.paper_params(), 0, xi.cpu().numpy(), "two_layer", 1)
    s.close()


def test_field_qois_accumulate_to_mean_and_variance_fields(hl):
    s = hl.Solver(qoi_set=hl.HENRY_QOI_PAPER_FIELD)
    xi = hl.sample_xi(inputs.SEED, 1, 660, 24)
    qf, qc, st, _ = s.level_batch_solve(1, xi, with_coarse=True)
    sums = torch.zeros((2, s.n_qoi, 3), dtype=torch.float64, device="cuda")
    hl.mlmc_accumulate(1, qf[:10], qc[:10], st[:10], sums)
    hl.mlmc_accumulate(1, qf[10:], qc[10:], st[10:], sums)
    y = (qf - qc).cpu().numpy()
    n, mean, m2 = omlmc.two_pass_moments(y)
    S = sums.cpu().numpy()
    assert np.all(S[0, :, 0] == n)
    np.testing.assert_allclose(S[0, :, 1], mean, rtol=0, atol=1e-13)
    np.testing.assert_allclose(S[0, :, 2], m2, rtol=1e-9, atol=1e-22)
    n1, mean1, _ = omlmc.two_pass_moments(qf.cpu().numpy())
    np.testing.assert_allclose(S[1, :, 1], mean1, rtol=0, atol=1e-13)
    s.close()


def test_uneven_batch_and_adjoint_with_wide_qoi_rows(hl):
    s = hl.Solver(qoi_set=hl.HENRY_QOI_PAPER)
    levels = np.array([1, 0, 2, 0, 1], dtype=np.int32)
    xi = torch.as_tensor(inputs.uniform_xi(670, 5), device="cuda")
    qf, qc, st, _ = s.batch_solve_mixed(levels, xi, with_coarse=True)
    assert int(st.abs().sum()) == 0
    for l in (0, 1, 2):
        idx = torch.as_tensor(np.nonzero(levels == l)[0], device="cuda")
        a, b, _, _ = s.level_batch_solve(l, xi[idx].contiguous(), with_coarse=l > 0)
        assert torch.equal(qf[idx], a)
        if l > 0:
            assert torch.equal(qc[idx], b)
        else:
            assert bool((qc[idx] == 0).all())
    w = torch.tensor([[0.01, 1.0]] * 2, dtype=torch.float64, device="cuda")
    x0 = xi[:2].contiguous()
    g1, q1, _ = s.adjoint(0, x0, w)
    s0 = hl.Solver()
    g0, q0, _ = s0.adjoint(0, x0, w)
    assert torch.equal(g1, g0) and torch.equal(q1[:, :2], q0)
    ref, _, _, _ = s.level_batch_solve(0, x0)
    assert torch.equal(q1, ref)
    s.close()
    s0.close()


@pytest.mark.parametrize("level", [0, 1])
def test_freshwater_series_matches_oracle(hl, level):
    """QoI set 3: Q_FW after every level-0 time step.  Each instant may differ
    from the oracle by at most one cell area (a cell within the states'
    ~1e-12 difference of the threshold); the last entry is the final Q_FW."""
    s = hl.Solver(qoi_set=hl.HENRY_QOI_PAPER_SERIES)
    xi = hl.sample_xi(inputs.SEED, level, 680, 2)
    q, _, st, _ = s.level_batch_solve(level, xi)
    assert int(st.abs().sum()) == 0 and q.shape == (2, 35)
    qn = q.cpu().numpy()
    grid = ohenry.Grid.level(ohenry.Params(), level)
    ref, ok = ohenry.solve_scenarios(ohenry.Params(), level, xi.cpu().numpy(), qoi_set=3)
    assert ok.all()
    assert np.all(np.abs(qn[:, 15:] - ref[:, 15:]) <= grid.h * grid.h + 1e-15)
    assert np.array_equal(qn[:, -1], qn[:, 2])
    np.testing.assert_allclose(qn[:, 3:15], ref[:, 3:15], rtol=0, atol=1e-10)
    w = torch.tensor([[0.01, 1.0]] * 2, dtype=torch.float64, device="cuda")
    _, qa, _ = s.adjoint(level, xi, w)
    assert torch.equal(qa, q)
    s.close()
