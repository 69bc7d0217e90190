"""The vertex-centred assembly of the CUDA path (henry_vc.cuh), compiled for
the host from the same source the kernel uses, against the vertex-centred
oracle (oracle.henry_vc): residuals and 9-point Jacobian blocks on random
states, central and partial-upwind faces.  This checks the arithmetic of the
kernel without a GPU; the GPU test checks the kernel's launch and layout."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT
from oracle import henry as cc
from oracle import henry_vc as vc
from paper_2302_07804_gb300 import inputs

PRM = vc.Params()


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("vc") / "libvc_harness.so")
    src = os.path.join(ROOT, "tests", "vc_harness.cpp")
    subprocess.run([cxx, "-O2", "-shared", "-fPIC", "-std=c++17", src, "-o", out], check=True)
    L = ctypes.CDLL(out)
    D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    L.vc_assemble_host.argtypes = [I, I] + [D] * 10 + [P] * 4
    L.vc_assemble_host.restype = None
    return L


def blocks_from_sparse(Jsp, grid):
    """[ny+1][nx+1][3][3][2][2] blocks of a sparse vertex Jacobian."""
    ny1, nx1 = grid.ny + 1, grid.nx + 1
    Jd = Jsp.tocoo()
    out = np.zeros((ny1, nx1, 3, 3, 2, 2))
    for r, c, v in zip(Jd.row, Jd.col, Jd.data):
        vr, eq = divmod(r, 2)
        vcol, var = divmod(c, 2)
        j, i = divmod(vr, nx1)
        jc, ic = divmod(vcol, nx1)
        out[j, i, jc - j + 1, ic - i + 1, eq, var] += v
    return out


def host_assemble(L, prm, grid, coef, p, c, po, co):
    x = np.ascontiguousarray(np.stack([p, c], axis=-1))
    xo = np.ascontiguousarray(np.stack([po, co], axis=-1))
    R = np.zeros_like(x)
    J = np.zeros((grid.ny + 1, grid.nx + 1, 3, 3, 2, 2))
    phi, K = float(coef.phi[0, 0]), float(coef.K[0, 0])
    L.vc_assemble_host(grid.nx, grid.ny, grid.h, grid.tau, prm.rho0, prm.rho1, prm.g, prm.Ly, phi, K / prm.mu,
                       phi * prm.Dm, float(coef.qin), x.ctypes.data, xo.ctypes.data, R.ctypes.data, J.ctypes.data)
    return R, J


def random_states(grid, seed, spread):
    gen = inputs.rng(seed)
    shape = (grid.ny + 1, grid.nx + 1)
    y = vc.vertex_y(grid)
    p = PRM.rho0 * PRM.g * (PRM.Ly - y)[:, None] + gen.uniform(-spread, spread, shape)
    c = gen.uniform(0.0, 1.0, shape)
    return p, c


@pytest.mark.parametrize("level,xi,spread,qscale", [(0, [0.0, 0.0, 0.0], 20.0, 1.0),
                                                    (0, [0.7, -0.9, 0.4], 300.0, 1.0),
                                                    (1, [-0.5, 0.8, -0.3], 100.0, 1.0),
                                                    (0, [0.2, 0.9, 0.9], 2000.0, 50.0)])
def test_host_build_of_the_kernel_math_matches_the_oracle(harness, level, xi, spread, qscale):
    """The last case multiplies K and q_in by 50, so that many faces take the
    partial upwind branch."""
    grid = vc.Grid.level(PRM, level)
    coef = cc.coefficients(PRM, grid, xi)
    coef = cc.Coeffs(phi=coef.phi, K=coef.K * qscale, qin=coef.qin * qscale)
    p, c = random_states(grid, 40 + level, spread)
    po, co = random_states(grid, 50 + level, spread)
    R, J = host_assemble(harness, PRM, grid, coef, p, c, po, co)
    Rm, Rs = vc.residual(PRM, grid, coef, p, c, po, co)
    Jo = blocks_from_sparse(vc.jacobian(PRM, grid, coef, p, c, po, co), grid)
    # rounding: relative to the largest face flux or storage term
    fl = vc.face_fluxes(PRM, grid, coef, p, c)
    sm = max(max(np.abs(F).max() for _, _, F, _ in fl), vc.residual_scale(PRM, grid))
    ss = max(max(np.abs(G).max() for _, _, _, G in fl), vc.residual_scale(PRM, grid))
    np.testing.assert_allclose(R[..., 0], Rm, rtol=0, atol=1e-12 * sm)
    np.testing.assert_allclose(R[..., 1], Rs, rtol=0, atol=1e-12 * ss)
    for eq in (0, 1):
        for var in (0, 1):
            scale = np.abs(Jo[..., eq, var]).max()
            assert scale > 0
            np.testing.assert_allclose(J[..., eq, var], Jo[..., eq, var], rtol=0, atol=1e-11 * scale)
    if qscale > 1:
        up = sum(int(np.sum(np.abs(F) * 2 > (vc.density(PRM, 0.5) * coef.phi * PRM.Dm))) for _, _, F, _ in fl)
        assert up > 0


def _csr_from_blocks(J, grid):
    import scipy.sparse as sp
    ny1, nx1 = grid.ny + 1, grid.nx + 1
    rows, cols, vals = [], [], []
    Jg, Ig = np.meshgrid(np.arange(ny1), np.arange(nx1), indexing="ij")
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            jn, inb = Jg + dj, Ig + di
            ok = (jn >= 0) & (jn < ny1) & (inb >= 0) & (inb < nx1)
            for eq in (0, 1):
                for var in (0, 1):
                    rows.append((2 * (Jg * nx1 + Ig) + eq)[ok])
                    cols.append((2 * (jn * nx1 + inb) + var)[ok])
                    vals.append(J[..., dj + 1, di + 1, eq, var][ok])
    n = 2 * ny1 * nx1
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def test_scenario_solved_with_the_kernel_math_matches_the_oracle(harness):
    """A whole level-0 scenario (20 implicit steps): Newton on the residual and
    Jacobian of the host build of the kernel arithmetic, with sparse direct
    solves, against the oracle's own solve; the QoIs agree to 1e-10."""
    import scipy.sparse.linalg as spla
    xi = [0.4, -0.6, 0.3]
    grid = vc.Grid.level(PRM, 0)
    coef = cc.coefficients(PRM, grid, xi)
    p, c = vc.initial_state(PRM, grid)
    sc = vc.residual_scale(PRM, grid)
    for _ in range(grid.steps):
        po, co = p, c
        for it in range(PRM.newton_maxit):
            R, J = host_assemble(harness, PRM, grid, coef, p, c, po, co)
            if np.abs(R).max() / sc <= PRM.newton_atol:
                break
            dx = spla.spsolve(_csr_from_blocks(J, grid).tocsc(), -R.ravel()).reshape(R.shape)
            p, c = p + dx[..., 0], c + dx[..., 1]
        else:
            pytest.fail("Newton did not converge")
    q_kernel = vc.qoi(PRM, grid, coef, p, c)
    q_oracle, ok = vc.solve_scenario(PRM, 0, xi)
    assert ok
    assert q_kernel[0] == pytest.approx(q_oracle[0], rel=1e-10, abs=0)
    assert q_kernel[1] == pytest.approx(q_oracle[1], rel=0, abs=1e-10)
