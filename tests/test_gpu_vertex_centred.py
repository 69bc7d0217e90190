"""GPU parity of the vertex-centred assembly (henry_vc_assemble, the paper's
own discretisation of Sec. 2.3) against the vertex-centred oracle: residuals
and 9-point Jacobian blocks, through the C ABI, at levels 0 and 1 and with a
flow strong enough for partial upwinding.  Tolerances as on the host build
of the same arithmetic: 1e-12 of the largest flux for residuals, 1e-11 of
each block column's largest entry for the Jacobian."""
import numpy as np
import pytest
from dataclasses import replace

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import henry as cc
from oracle import henry_vc as vc
from paper_2302_07804_gb300 import inputs
from test_vc_assembly_host import blocks_from_sparse, random_states


@pytest.fixture(scope="module")
def hl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("level,n,scale", [(0, 3, 1.0), (1, 2, 1.0), (0, 2, 50.0)])
def test_vc_assembly_matches_oracle(hl, level, n, scale):
    prm = replace(vc.Params(), K_mean=1.02e-9 * scale, qin_mean=6.6e-5 * scale)
    s = hl.Solver(K_mean=prm.K_mean, qin_mean=prm.qin_mean)
    grid = vc.Grid.level(prm, level)
    xi = hl.sample_xi(inputs.SEED, level, 900, n)
    xs = xi.cpu().numpy()
    states = [random_states(grid, 60 + k, 300.0) for k in range(n)]
    olds = [random_states(grid, 70 + k, 300.0) for k in range(n)]
    st = _dev(np.stack([np.stack(a, axis=-1) for a in states]))
    so = _dev(np.stack([np.stack(a, axis=-1) for a in olds]))
    R, J = s.vc_assemble(level, xi, st, so)
    torch.cuda.synchronize()
    R, J = R.cpu().numpy(), J.cpu().numpy()
    for k in range(n):
        coef = cc.coefficients(prm, grid, xs[k])
        (p, c), (po, co) = states[k], olds[k]
        Rm, Rs = vc.residual(prm, grid, coef, p, c, po, co)
        Jo = blocks_from_sparse(vc.jacobian(prm, grid, coef, p, c, po, co), grid)
        fl = vc.face_fluxes(prm, grid, coef, p, c)
        sm = max(max(np.abs(F).max() for _, _, F, _ in fl), vc.residual_scale(prm, grid))
        ss = max(max(np.abs(G).max() for _, _, _, G in fl), vc.residual_scale(prm, grid))
        np.testing.assert_allclose(R[k, ..., 0], Rm, rtol=0, atol=1e-12 * sm)
        np.testing.assert_allclose(R[k, ..., 1], Rs, rtol=0, atol=1e-12 * ss)
        for eq in (0, 1):
            for var in (0, 1):
                sc = np.abs(Jo[..., eq, var]).max()
                np.testing.assert_allclose(J[k, ..., eq, var], Jo[..., eq, var], rtol=0, atol=1e-11 * sc)
    s.close()


def test_vc_assembly_rejects_field_models(hl):
    s = hl.Solver(coef_model=hl.HENRY_MODEL_KL)
    ny, nx = s.grid(0)
    xi = torch.zeros((1, s.n_xi), dtype=torch.float64, device="cuda")
    st = torch.zeros((1, ny + 1, nx + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hl.HenryError) as e:
        s.vc_assemble(0, xi, st, st)
    assert e.value.code == hl.HENRY_EINVAL
    s.close()


def test_vc_assembly_rejects_inputs_outside_the_model(hl):
    """xi1 = -6 gives phi = 0.35 (1 - 1.2) < 0: the call refuses the batch and
    names the sample instead of assembling from a negative porosity."""
    s = hl.Solver()
    ny, nx = s.grid(0)
    xi = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    xi[1, 0] = -6.0
    st = torch.zeros((3, ny + 1, nx + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(hl.HenryError) as e:
        s.vc_assemble(0, xi, st, st)
    assert e.value.code == hl.HENRY_EINVAL and "sample 1" in str(e.value)
    xi[1, 0] = 0.0
    R, _ = s.vc_assemble(0, xi, st, st, with_jacobian=False)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(R).all())
    s.close()
