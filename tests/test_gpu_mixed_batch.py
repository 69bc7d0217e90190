"""henry_batch_solve_mixed: an uneven batch over several MLMC levels in one
call (levels on concurrent streams and host threads).  Each sample's result
depends only on its own inputs, so it must be bit-identical to
henry_level_batch_solve on the same samples, in any input order; level-0
samples get zero coarse QoIs; per-level handles report to the profiler."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2302_07804_gb300 import inputs


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _per_level(hl, solver_kw, levels, xi, with_coarse):
    """QoIs of each sample from one henry_level_batch_solve per level."""
    s = hl.Solver(**solver_kw)
    n = len(levels)
    qf = torch.zeros((n, 2), dtype=torch.float64, device=xi.device)
    qc = torch.zeros((n, 2), dtype=torch.float64, device=xi.device)
    for l in sorted(set(levels.tolist())):
        idx = torch.as_tensor(np.nonzero(levels == l)[0], device=xi.device)
        a, b, st, _ = s.level_batch_solve(l, xi[idx].contiguous(), with_coarse=with_coarse and l > 0)
        assert int(st.abs().sum()) == 0
        qf[idx] = a
        if b is not None:
            qc[idx] = b
    s.close()
    return qf, qc


@pytest.mark.parametrize("shuffle", [False, True])
def test_mixed_batch_is_bit_identical_to_per_level_solves(hl, shuffle):
    counts = [7, 5, 3, 2]
    levels = np.concatenate([np.full(m, l, dtype=np.int32) for l, m in enumerate(counts)])
    if shuffle:
        levels = inputs.rng(610).permutation(levels).astype(np.int32)
    xi = torch.as_tensor(inputs.uniform_xi(611, len(levels)), device="cuda")
    s = hl.Solver()
    qf, qc, st, stats = s.batch_solve_mixed(levels, xi, with_coarse=True)
    assert int(st.abs().sum()) == 0 and stats["failed_samples"] == 0
    rf, rc = _per_level(hl, {}, levels, xi, True)
    assert torch.equal(qf, rf)
    assert torch.equal(qc, rc)
    assert bool((qc[torch.as_tensor(levels == 0, device="cuda")] == 0).all())
    cfg = s.cfg
    cs = sum(int(m) * (cfg.nx0 << l) * (cfg.ny0 << l) * (cfg.steps0 << l) for l, m in enumerate(counts)) + \
        sum(int(m) * (cfg.nx0 << (l - 1)) * (cfg.ny0 << (l - 1)) * (cfg.steps0 << (l - 1))
            for l, m in enumerate(counts) if l > 0)
    assert stats["cell_steps"] == cs
    # a second call reuses the child handles and the permutation buffer
    qf2, qc2, _, _ = s.batch_solve_mixed(levels, xi, with_coarse=True)
    assert torch.equal(qf2, qf) and torch.equal(qc2, qc)
    s.close()


def test_mixed_batch_kl_mixed_precision(hl):
    kw = dict(coef_model=hl.HENRY_MODEL_KL, precision=hl.HENRY_MIXED)
    levels = np.array([1, 0, 0, 1, 0, 2], dtype=np.int32)
    gen = inputs.rng(620)
    th = np.concatenate([gen.standard_normal((len(levels), 64)), gen.uniform(-1, 1, (len(levels), 1))], axis=1)
    xi = torch.as_tensor(th, device="cuda")
    s = hl.Solver(**kw)
    qf, _, st, _ = s.batch_solve_mixed(levels, xi)
    assert int(st.abs().sum()) == 0
    rf, _ = _per_level(hl, kw, levels, xi, False)
    assert torch.equal(qf, rf)
    s.close()


def test_mixed_batch_profiles_through_level_handles(hl):
    s = hl.Solver()
    levels = np.array([0, 1, 0, 1], dtype=np.int32)
    xi = torch.as_tensor(inputs.uniform_xi(630, 4), device="cuda")
    s.profile(True)
    s.batch_solve_mixed(levels, xi, with_coarse=True)
    prof = s.profile_read()
    assert prof["smooth"][1] > 0 and prof["assemble"][1] > 0
    s.profile(False)
    s.close()


def test_mixed_batch_rejects_bad_arguments(hl):
    s = hl.Solver()
    xi = torch.as_tensor(inputs.uniform_xi(640, 3), device="cuda")
    with pytest.raises(hl.HenryError) as e:
        s.batch_solve_mixed(np.array([0, 1, 6], dtype=np.int32), xi)
    assert e.value.code == hl.HENRY_EINVAL
    with pytest.raises(ValueError):
        s.batch_solve_mixed([0, 1], xi)
    s.close()
