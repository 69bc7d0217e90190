"""Full sizes, in the launch configuration the bench uses.

* Level 0 with the bench's 81675 samples (the workspace budget splits the
  batch into chunks, as in the bench), FP64 and mixed precision: every status
  0 and every QoI in range; samples at the chunk boundaries, the first, the
  middle and the last recomputed by the oracle (1e-10).
* Level 5, the largest grid (1024 x 512 cells, 640 steps), two samples with
  coarse partners: the oracle cannot redo these in a test, so properties that
  hold at any size are checked: 0 <= c <= 1 at the point, positive salt mass,
  a small level difference, and the FP64 and mixed-precision solves (two
  different linear-algebra precisions driving the same FP64 Newton test)
  reaching the same discrete solution to 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry
from paper_2302_07804_gb300 import inputs

PRM = ohenry.Params()
N0 = 81675


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


@pytest.mark.parametrize("precision", [0, 1])
def test_level0_bench_batch_sampled_against_oracle(hl, precision):
    s = hl.Solver(precision=precision)
    xi = hl.sample_xi(inputs.SEED, 0, 10 ** 7, N0)
    q, _, st, stats = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0 and stats["failed_samples"] == 0
    qn = q.cpu().numpy()
    assert np.all((qn[:, 1] >= -1e-12) & (qn[:, 1] <= 1 + 1e-12)) and np.all(qn[:, 0] > 0)
    picks = sorted({0, 1, N0 // 2, N0 - 2, N0 - 1} | {k for k in (16401, 16402, 65273, 65274) if k < N0})
    ref, ok = ohenry.solve_scenarios(PRM, 0, xi[picks].cpu().numpy())
    assert ok.all()
    np.testing.assert_allclose(qn[picks, 0], ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(qn[picks, 1], ref[:, 1], rtol=1e-10, atol=1e-14)
    s.close()


def test_largest_grid_properties(hl):
    xi = hl.sample_xi(inputs.SEED, 5, 0, 2)
    out = []
    for precision in (0, 1):
        s = hl.Solver(precision=precision)
        qf, qc, st, _ = s.level_batch_solve(5, xi, with_coarse=True)
        assert int(st.abs().sum()) == 0
        out.append((qf.cpu().numpy(), qc.cpu().numpy()))
        s.close()
    (f64, c64), (f32, c32) = out
    assert np.all((f64[:, 1] >= -1e-12) & (f64[:, 1] <= 1 + 1e-12)) and np.all(f64[:, 0] > 0)
    assert np.abs(f64[:, 1] - c64[:, 1]).max() < 0.01
    np.testing.assert_allclose(f32[:, 0], f64[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(f32[:, 1], f64[:, 1], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(c32[:, 1], c64[:, 1], rtol=1e-10, atol=1e-14)
