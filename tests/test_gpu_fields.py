"""GPU parity of the coefficient-field models against the oracle.

* KL random fields (log K and phi, 32 terms each; the caller supplies the
  Gaussian coefficients): per-step residual and Jacobian with per-cell
  coefficients and harmonic face means (rtol as in test_gpu_parity), and full
  scenario QoIs at levels 0 and 1 in FP64 and mixed precision (1e-10).
* The paper's two-layer porosity with Kozeny-Carman permeability: QoIs at
  level 0 (1e-10).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as ohenry
from oracle import kl as okl
from oracle import mg as omg
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


def _to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _kl_inputs(tag, n):
    gen = inputs.rng(tag)
    return np.concatenate([gen.standard_normal((n, 64)), gen.uniform(-1, 1, (n, 1))], axis=1)


def _qoi_check(q_gpu, q_ref):
    np.testing.assert_allclose(q_gpu[:, 0], q_ref[:, 0], rtol=1e-10, atol=0)
    np.testing.assert_allclose(q_gpu[:, 1], q_ref[:, 1], rtol=1e-10, atol=1e-14)


def test_kl_assemble_matches_oracle(hl):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    level, n = 1, 2
    grid = ohenry.Grid.level(PRM, level)
    th = _kl_inputs(500, n)
    p, c = inputs.random_states(501, 2 * n, grid.ny, grid.nx, 5e3, 1e4, 300.0)
    st = np.stack([p[:n], c[:n]], axis=-1)
    so = np.stack([p[n:], c[n:]], axis=-1)
    F, J = s.assemble(level, _to_dev(th), _to_dev(st), _to_dev(so))
    F, J = F.cpu().numpy(), J.cpu().numpy()
    sc = ohenry.residual_scale(PRM, grid)
    for i in range(n):
        coef = okl.coefficients_kl(PRM, grid, th[i])
        Rm, Rs = ohenry.residual(PRM, grid, coef, p[i], c[i], p[n + i], c[n + i])
        Jo = omg.blocks_from_csr(ohenry.jacobian(PRM, grid, coef, p[i], c[i], p[n + i], c[n + i]),
                                 grid.nx, grid.ny) / sc
        Fo = np.stack([Rm, Rs], axis=-1) / sc
        fscale = np.abs(Jo[..., 0, :, 0]).max() * 300.0 + 1.0
        np.testing.assert_allclose(F[i], Fo, rtol=0, atol=1e-11 * fscale)
        for eq in range(2):
            for var in range(2):
                np.testing.assert_allclose(J[i][..., eq, var], Jo[..., eq, var], rtol=0,
                                           atol=1e-11 * np.abs(Jo[..., eq, var]).max())
    s.close()


@pytest.mark.parametrize("level,precision", [(0, 0), (0, 1), (1, 0)])
def test_kl_solve_matches_oracle(hl, level, precision):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL, precision=precision)
    n = 4 if level == 0 else 2
    th = _kl_inputs(510 + level, n)
    qf, _, st, stats = s.level_batch_solve(level, _to_dev(th))
    assert int(st.abs().sum()) == 0
    ref, ok = ohenry.solve_scenarios(PRM, level, th, model="kl")
    assert ok.all()
    _qoi_check(qf.cpu().numpy(), ref)
    s.close()


def test_kl_coarse_partner(hl):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    th = _kl_inputs(520, 3)
    qf, qc, st, _ = s.level_batch_solve(1, _to_dev(th), with_coarse=True)
    assert int(st.abs().sum()) == 0
    ref0, _ = ohenry.solve_scenarios(PRM, 0, th, model="kl")
    _qoi_check(qc.cpu().numpy(), ref0)
    s.close()


def test_two_layer_paper_variant_matches_oracle(hl):
    # the paper's constants (Table tab:HenryParam) and recharge amplitude 0.5 (Sec. 4)
    prm = ohenry.Params(g=9.8, rho1=1024.99, Dm=18.8571e-6, K_mean=1.020408e-9, qin_amp=0.5)
    s = hl.Solver(coef_model=hl.HENRY_MODEL_TWO_LAYER, g=9.8, rho1=1024.99, Dm=18.8571e-6, K_mean=1.020408e-9,
                  qin_amp=0.5)
    xi = hl.sample_xi(inputs.SEED, 0, 0, 6)
    qf, _, st, _ = s.level_batch_solve(0, xi)
    assert int(st.abs().sum()) == 0
    ref, ok = ohenry.solve_scenarios(prm, 0, xi.cpu().numpy(), model="two_layer")
    assert ok.all()
    _qoi_check(qf.cpu().numpy(), ref)
    s.close()


def test_kl_hard_samples_converge_with_fallback(hl):
    """Inputs with strong permeability/porosity contrast for which one
    V-cycle preconditioner loses BiCGStab convergence (the same happens in
    the oracle's textbook V-cycle): the fallback V-cycle on the Jacobian
    without density derivatives and the Newton step limit let every sample
    converge, to the oracle's solution."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "kl_hard_inputs.txt")
    th = np.loadtxt(path)
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    qf, _, st, _ = s.level_batch_solve(0, _to_dev(th))
    assert int(st.abs().sum()) == 0
    ref, ok = ohenry.solve_scenarios(PRM, 0, th, model="kl")
    assert ok.all()
    _qoi_check(qf.cpu().numpy(), ref)
    s.close()
