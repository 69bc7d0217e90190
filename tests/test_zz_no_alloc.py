"""The allocation-free batch solve (henry_level_batch_solve_static).

Some callers cannot call cudaMalloc at run time (their device memory belongs
to another allocator or pool, or they must not grow after loading), so the
library offers a variant of the batch solve whose workspace is a device array
compiled into the library.  This test calls it through the C ABI twice in a
row (different levels and batch shapes, so the second call reuses the array
the first one left behind) and checks each result against the ordinary entry
point, henry_level_batch_solve, within the QoI tolerance of the parity tests
(1e-10 relative on both QoIs).  It also
checks that a batch larger than the array is refused with a clear error.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _same(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    np.testing.assert_allclose(a[:, 0], b[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(a[:, 1], b[:, 1], rtol=1e-10, atol=1e-14)


def test_static_solve_matches_allocating_solve_twice(hl):
    from paper_2302_07804_gb300 import inputs
    cfg = hl.default_config()
    ref = hl.Solver()
    # call 1: level 1 with coarse partners
    xi1 = hl.sample_xi(inputs.SEED, 1, 500, 8)
    qf, qc, st = hl.level_batch_solve_static(cfg, 1, xi1, with_coarse=True)
    rf, rc_, rst, _ = ref.level_batch_solve(1, xi1, with_coarse=True)
    assert int(st.abs().sum()) == 0 and int(rst.abs().sum()) == 0
    _same(qf, rf)
    _same(qc, rc_)
    # call 2: a full 64-sample level-0 batch in the same array
    xi0 = hl.sample_xi(inputs.SEED, 0, 900, 64)
    qf2, qc2, st2 = hl.level_batch_solve_static(cfg, 0, xi0)
    rf2, _, rst2, _ = ref.level_batch_solve(0, xi0)
    assert qc2 is None
    assert int(st2.abs().sum()) == 0 and int(rst2.abs().sum()) == 0
    _same(qf2, rf2)
    ref.close()


def test_static_solve_mixed_precision_matches_allocating_solve(hl):
    """HENRY_MIXED lays out FP32 groups in the same array (other sizes and
    offsets than FP64): level 1 with coarse partners, then level 0, each
    against the allocating entry point in mixed precision."""
    from paper_2302_07804_gb300 import inputs
    cfg = hl.default_config(precision=hl.HENRY_MIXED)
    ref = hl.Solver(precision=hl.HENRY_MIXED)
    xi1 = hl.sample_xi(inputs.SEED, 1, 620, 6)
    qf, qc, st = hl.level_batch_solve_static(cfg, 1, xi1, with_coarse=True)
    rf, rc_, rst, _ = ref.level_batch_solve(1, xi1, with_coarse=True)
    assert int(st.abs().sum()) == 0 and int(rst.abs().sum()) == 0
    _same(qf, rf)
    _same(qc, rc_)
    xi0 = hl.sample_xi(inputs.SEED, 0, 640, 32)
    qf2, _, st2 = hl.level_batch_solve_static(cfg, 0, xi0)
    rf2, _, rst2, _ = ref.level_batch_solve(0, xi0)
    assert int(st2.abs().sum()) == 0 and int(rst2.abs().sum()) == 0
    _same(qf2, rf2)
    ref.close()


def test_static_solve_rejects_batches_beyond_the_array(hl):
    cfg = hl.default_config()
    xi = torch.zeros((1000, 3), dtype=torch.float64, device="cuda")
    out = torch.empty((1000, 2), dtype=torch.float64, device="cuda")
    st = torch.empty((1000,), dtype=torch.int32, device="cuda")
    L = hl.lib()
    rc = L.henry_level_batch_solve_static(ctypes.byref(cfg), 0, 0, ctypes.c_void_p(xi.data_ptr()), 1000,
                                          ctypes.c_void_p(out.data_ptr()), None, ctypes.c_void_p(st.data_ptr()),
                                          None)
    assert rc == hl.HENRY_EINVAL
    msg = L.henry_last_error().decode()
    assert "static scratch" in msg and "bytes" in msg
