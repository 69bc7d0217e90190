"""Degenerate inputs of the three-parameter model: the eight corners of the
input cube [-1, 1]^3 (the extremes of phi, K and q_in together; the Philox
map itself never returns +-1), solved through the C ABI and compared with
the oracle at the tolerances of the other full-solve parity tests (1e-10
relative salt mass and c at the point, with a 1e-14 absolute floor)."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry

PRM = ohenry.Params()
CORNERS = np.array(list(itertools.product((-1.0, 1.0), repeat=3)))


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


@pytest.fixture(scope="module")
def ref0():
    ref, ok = ohenry.solve_scenarios(PRM, 0, CORNERS)
    assert ok.all()
    return ref


def _check(q, ref):
    np.testing.assert_allclose(q[:, 0], ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(q[:, 1], ref[:, 1], rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("fused,precision", [(2, 0), (0, 0), (1, 1)])
def test_level0_corners_match_oracle(hl, ref0, fused, precision):
    s = hl.Solver(fused_small_grids=fused, precision=precision)
    xi = torch.as_tensor(CORNERS, dtype=torch.float64, device="cuda")
    qf, _, st, _ = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0
    _check(qf.cpu().numpy(), ref0)
    s.close()


def test_level1_corners_with_coarse_partner(hl, ref0):
    pick = [0, 7]                         # all inputs at -1, all at +1
    ref1, ok = ohenry.solve_scenarios(PRM, 1, CORNERS[pick])
    assert ok.all()
    s = hl.Solver()
    xi = torch.as_tensor(CORNERS[pick], dtype=torch.float64, device="cuda")
    qf, qc, st, _ = s.level_batch_solve(1, xi, with_coarse=True)
    assert int(st.abs().sum()) == 0
    _check(qf.cpu().numpy(), ref1)
    _check(qc.cpu().numpy(), ref0[pick])
    s.close()
