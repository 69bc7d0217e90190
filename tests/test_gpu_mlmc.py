"""The MLMC driver on the GPU: the adaptive choice of the finest level by the
bias test, with the rates fitted by the library checked against the oracle's
fit of the same per-level statistics."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlmc as omlmc


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def test_adaptive_mlmc_bias_test_and_rates(hl):
    from paper_2302_07804_gb300 import mlmc
    s = hl.Solver()
    eps = 5e-3
    r = mlmc.run_mlmc_adaptive(s, eps=eps, L_start=2, L_max=3, pilot=(200, 50, 20, 10))
    means = [p["mean_Y"] for p in r["levels"]]
    var = [p["var_Y"] for p in r["levels"]]
    assert r["L"] in (2, 3) and len(means) == r["L"] + 1
    assert r["bias_ok"] or r["L"] == 3
    cost = [mlmc.level_cost_model(s.cfg, l) for l in range(r["L"] + 1)]
    a, b, g = omlmc.rates(means, var, cost, first_level=1)
    assert r["alpha"] == pytest.approx(a, rel=1e-10)
    assert r["beta"] == pytest.approx(b, rel=1e-10)
    assert r["gamma_d"] == pytest.approx(g, rel=1e-10)
    bias, ok = omlmc.bias_test(means, max(a, 0.5), eps)
    assert r["bias_est"] == pytest.approx(bias, rel=1e-10, abs=0) and r["bias_ok"] == ok
    assert r["estimate"] == pytest.approx(sum(means), rel=1e-13)
    assert r["variance"] <= 1.5 * 0.5 * eps * eps
    assert all(p["failed"] == 0 for p in r["levels"])
    s.close()


def test_concurrent_rounds_give_the_same_estimate(hl):
    """run_mlmc's rounds as one henry_batch_solve_mixed call over all levels
    solve the same samples (same Philox counters) and accumulate the same
    per-level batches as the level-by-level driver: identical sums."""
    from paper_2302_07804_gb300 import mlmc
    import json
    out = []
    for conc in (True, False):
        s = hl.Solver()
        r = mlmc.run_mlmc(s, eps=4e-3, max_level=2, pilot=(300, 60, 20), concurrent=conc)
        out.append(r)
        s.close()
    assert out[0]["estimate"] == out[1]["estimate"] and out[0]["alloc"] == out[1]["alloc"]
    a, b = json.loads(out[0]["checkpoint"]), json.loads(out[1]["checkpoint"])
    for la, lb in zip(a, b):
        assert la["sums"] == lb["sums"] and la["n_used"] == lb["n_used"] and la["cell_steps"] == lb["cell_steps"]


def test_resume_from_checkpoint_continues_identically(hl):
    """An MLMC run stopped after its first top-up round, serialised
    (per-level sums and Philox counter offsets) and resumed from the JSON,
    ends with exactly the sums of an uninterrupted run."""
    from paper_2302_07804_gb300 import mlmc
    import json
    kw = dict(eps=4e-3, max_level=2, pilot=(300, 60, 20))
    s = hl.Solver()
    full = mlmc.run_mlmc(s, **kw)
    part = mlmc.run_mlmc(s, max_rounds=1, **kw)
    dev = torch.device("cuda", torch.cuda.current_device())
    state = [mlmc.LevelState.from_json(d, dev) for d in json.loads(part["checkpoint"])]
    resumed = mlmc.run_mlmc(s, state=state, **kw)
    assert resumed["estimate"] == full["estimate"]
    for a, b in zip(json.loads(resumed["checkpoint"]), json.loads(full["checkpoint"])):
        assert a["sums"] == b["sums"] and a["n_used"] == b["n_used"]
    s.close()


@pytest.mark.parametrize("precision,level", [(0, 0), (1, 0), (0, 2)])
def test_autotune_picks_a_candidate_and_solves_stay_exact(hl, precision, level):
    """henry_autotune keeps one of its candidates for the level, and solves
    with it still reach the oracle's discrete solution (1e-10); an uneven
    batch's level handles inherit the tuning (bit-identical results)."""
    import numpy as np
    from oracle import henry as ohenry
    from paper_2302_07804_gb300 import inputs
    s = hl.Solver(precision=precision)
    trial = hl.sample_xi(inputs.SEED, level, 5000, 256 if level == 0 else 16)
    best = s.autotune(level, trial)
    assert best["lin_rtol"] in (1e-4, 1e-3, 1e-2) and (best["nu1"], best["nu2"]) in ((2, 2), (1, 2), (2, 1))
    assert best["mg_tail_cells"] in (-1, 0, 32, 128, 512, 2048) and best["newton_residual_first"] in (-1, 2, 3, 4)
    assert best["newton_jacobian_every"] in (1, 2, 3)
    assert best["cell_steps_per_s"] > 0 and s.tuning(level) == best
    xi = hl.sample_xi(inputs.SEED, level, 6000, 3)
    q, _, st, _ = s.level_batch_solve(level, xi)
    assert int(st.abs().sum()) == 0
    ref, ok = ohenry.solve_scenarios(ohenry.Params(), level, xi.cpu().numpy())
    assert ok.all()
    np.testing.assert_allclose(q.cpu().numpy()[:, 0], ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(q.cpu().numpy()[:, 1], ref[:, 1], rtol=1e-10, atol=1e-14)
    qm, _, _, _ = s.batch_solve_mixed(np.full(3, level, dtype=np.int32), xi)
    assert torch.equal(qm, q)
    s.close()
