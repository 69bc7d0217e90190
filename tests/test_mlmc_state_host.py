"""The MLMC driver's checkpoint format on the host: a level's state (sums
of Y and of the fine QoI, the Philox counter offset, cost and failure
counters) survives a JSON round trip unchanged."""
import json

import pytest

torch = pytest.importorskip("torch")


def test_level_state_json_round_trip():
    from paper_2302_07804_gb300 import mlmc
    st = mlmc.LevelState(2, "cpu", n_qoi=5)
    st.sums = torch.arange(30, dtype=torch.float64).reshape(2, 5, 3) / 7.0
    st.n_used, st.gpu_seconds, st.cell_steps, st.failed = 1234, 0.5, 9.9e8, 3
    back = mlmc.LevelState.from_json(json.loads(json.dumps(st.to_json())), "cpu")
    assert back.level == 2 and back.n_used == 1234 and back.failed == 3
    assert back.gpu_seconds == 0.5 and back.cell_steps == 9.9e8
    assert torch.equal(back.sums, st.sums) and back.sums.shape == (2, 5, 3)
    n, mean, var = back.moments()
    assert n == st.sums[0, 0, 0].item() and len(var) == 5


def test_run_mlmc_checks_its_arguments_before_any_device_work():
    from types import SimpleNamespace
    from paper_2302_07804_gb300 import mlmc
    solver = SimpleNamespace(cfg=SimpleNamespace(max_level=5, nx0=32, ny0=16, steps0=20), n_qoi=2)
    for kw, text in ((dict(max_level=6), "outside [0, 5]"), (dict(max_level=-1), "outside [0, 5]"),
                     (dict(max_level=4, pilot=(10, 10, 10)), "pilot gives 3 levels"),
                     (dict(max_level=1, state=[mlmc.LevelState(l, "cpu") for l in range(3)]), "state holds 3")):
        with pytest.raises(ValueError) as e:
            mlmc.run_mlmc(solver, **kw)
        assert text in str(e.value)
    with pytest.raises(ValueError):
        mlmc.run_level(solver, mlmc.LevelState(0, "cpu"), 5, 1, xi=torch.zeros((4, 3), dtype=torch.float64))
