"""henry_adjoint on the GPU: dQ/dtheta of the implicit-Euler solve against
the oracle's adjoint (direct solves, complex-step partials) for the three
models, against central differences of the GPU's own forward solve (h = 1e-6)
at level 1 and at the full 256 x 128, 200-step size, independence of the
checkpoint interval, the forward QoIs, and the torch.autograd wrapper.

Tolerances: both sides stop Newton at a scaled residual of 1e-11, which moves
the states (and so the gradients) by ~1e-10 relative; 1e-7 of the largest
component is used against the oracle.  Central differences of the GPU
forward resolve the gradient to ~1e-11 / 1e-6 = 1e-5 relative; 1e-4 is used."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adjoint as oadj
from oracle import henry as ohenry
from paper_2302_07804_gb300 import inputs

PRM = ohenry.Params()


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _kl_inputs(tag, n):
    gen = inputs.rng(tag)
    return np.concatenate([gen.standard_normal((n, 64)), gen.uniform(-1, 1, (n, 1))], axis=1)


W4 = np.array([[0.01, 1.0], [1.0, 0.0], [0.0, 1.0], [0.3, -2.0]])


@pytest.mark.parametrize("model", ["uniform3", "kl", "two_layer"])
def test_adjoint_matches_oracle_adjoint(hl, model):
    code = {"uniform3": hl.HENRY_MODEL_UNIFORM3, "kl": hl.HENRY_MODEL_KL, "two_layer": hl.HENRY_MODEL_TWO_LAYER}
    s = hl.Solver(coef_model=code[model])
    n = 4 if model != "kl" else 2
    if model == "kl":
        xi = _dev(_kl_inputs(800, n))
    else:
        xi = hl.sample_xi(inputs.SEED, 0, 500, n)
    w = _dev(W4[:n])
    grad, q, st = s.adjoint(0, xi, w, checkpoint_every=7)
    assert int(st.abs().sum()) == 0
    qf, _, _, _ = s.level_batch_solve(0, xi)
    assert torch.equal(q, qf)
    for i in range(n):
        g_ref, q_ref, ok = oadj.adjoint_gradient(PRM, 0, xi[i].cpu().numpy(), W4[i], model=model)
        assert ok
        np.testing.assert_allclose(grad[i].cpu().numpy(), g_ref, rtol=0, atol=1e-7 * np.abs(g_ref).max())
    s.close()


@pytest.mark.parametrize("order", [1, 2])
def test_adjoint_is_independent_of_the_checkpoint_interval(hl, order):
    """Recomputing each segment from its checkpoint (two states, three with
    the quadratic predictor) reproduces the forward states: gradients and
    QoIs bit-identical for every interval, and the forward QoIs equal the
    level solve's."""
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL, newton_predictor_order=order)
    xi = _dev(_kl_inputs(810, 3))
    w = _dev(W4[:3])
    ref = None
    for ck in (1, 3, 20, 1000):
        grad, q, st = s.adjoint(1, xi, w, checkpoint_every=ck)
        assert int(st.abs().sum()) == 0
        if ref is None:
            ref = (grad.clone(), q.clone())
        else:
            assert torch.equal(grad, ref[0]) and torch.equal(q, ref[1])
    qf, _, _, _ = s.level_batch_solve(1, xi)
    assert torch.equal(ref[1], qf)
    s.close()


def _fd_check(hl, s, level, xi, w, grad, comps, h=1e-6, tol=1e-4):
    """Central differences of the GPU forward solve for the (sample, component)
    pairs in comps, all perturbed inputs solved in one batch."""
    rows = []
    for i, k in comps:
        for sgn in (1.0, -1.0):
            x = xi[i].clone()
            x[k] += sgn * h
            rows.append(x)
    qf, _, st, _ = s.level_batch_solve(level, torch.stack(rows).contiguous())
    assert int(st.abs().sum()) == 0
    qf = qf.cpu().numpy()
    wn = w.cpu().numpy()
    g = grad.cpu().numpy()
    for j, (i, k) in enumerate(comps):
        fd = (wn[i] @ qf[2 * j] - wn[i] @ qf[2 * j + 1]) / (2 * h)
        assert abs(fd - g[i, k]) <= tol * np.abs(g[i]).max(), (i, k, fd, g[i, k])


def test_adjoint_matches_gpu_central_differences_level1(hl):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    xi = _dev(_kl_inputs(820, 2))
    w = _dev(W4[:2])
    grad, _, st = s.adjoint(1, xi, w)
    assert int(st.abs().sum()) == 0
    _fd_check(hl, s, 1, xi, w, grad, [(0, 0), (0, 33), (0, 64), (1, 7), (1, 40)])
    s.close()


def test_adjoint_full_size_256x128_200_steps(hl):
    """The adjoint workload's size: 256 x 128 cells, 200 implicit steps
    (level 3 with 25 steps at level 0), KL inputs, checkpoints every 20
    steps; a batch of 64, five components checked by central differences."""
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL, steps0=25)
    xi = _dev(_kl_inputs(830, 64))
    w = _dev(np.tile([0.01, 1.0], (64, 1)))
    grad, q, st = s.adjoint(3, xi, w, checkpoint_every=20)
    assert int(st.abs().sum()) == 0
    assert bool(torch.isfinite(grad).all())
    _fd_check(hl, s, 3, xi, w, grad, [(0, 0), (0, 32), (0, 64), (63, 3), (63, 50)])
    s.close()


def test_autograd_function_calls_the_adjoint(hl):
    s = hl.Solver()
    xi = hl.sample_xi(inputs.SEED, 1, 900, 3).clone().requires_grad_(True)
    w = _dev(W4[:3])
    q = hl.scenario_qoi(s, 1, xi, checkpoint_every=10)
    (q * w).sum().backward()
    g, _, _ = s.adjoint(1, xi.detach(), w, checkpoint_every=10)
    assert torch.equal(xi.grad, g)
    s.close()


def test_nonfinite_sample_is_isolated(hl):
    """A sample with a non-finite input fails alone: status 3 and a zero
    gradient for it, and every other sample bit-identical to a batch
    without it (adjoint and uneven batch)."""
    s = hl.Solver()
    xi = hl.sample_xi(inputs.SEED, 0, 840, 4).clone()
    xi[2, 1] = float("nan")
    w = _dev(W4)
    g, q, st = s.adjoint(0, xi, w, allow_failures=True)
    assert st.tolist() == [0, 0, 3, 0]
    assert bool((g[2] == 0).all())
    keep = torch.tensor([0, 1, 3], device="cuda")
    g2, q2, st2 = s.adjoint(0, xi[keep].contiguous(), w[keep].contiguous())
    assert torch.equal(g[keep], g2) and torch.equal(q[keep], q2)
    levels = np.array([0, 1, 0, 1], dtype=np.int32)
    qf, qc, stm, stats = s.batch_solve_mixed(levels, xi, with_coarse=True, allow_failures=True)
    assert stm.tolist() == [0, 0, 3, 0] and stats["failed_samples"] == 1
    a, _, _, _ = s.level_batch_solve(1, xi[[1, 3]].contiguous(), with_coarse=True)
    assert torch.equal(qf[[1, 3]], a)
    s.close()
