"""C-ABI checks that need no GPU: the library builds, loads and exports every
function include/henry.h declares; host-only calls (mlmc_allocate, argument
validation) behave as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, golden_rows

HEADER = os.path.join(ROOT, "include", "henry.h")


@pytest.fixture(scope="module")
def L():
    from paper_2302_07804_gb300 import build, henry
    build.build()
    return henry.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("henry_create", "henry_destroy", "henry_sample_xi", "henry_level_batch_solve",
                     "mlmc_accumulate", "mlmc_allocate", "henry_last_error", "henry_assemble",
                     "henry_apply_jacobian", "henry_precondition", "henry_linear_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_mlmc_allocate_reproduces_paper_table(L):
    from paper_2302_07804_gb300 import henry
    rows = golden_rows("paper_table_M_ell.txt")
    s = [float(v) for v in rows[0][1:]]
    V = [float(v) for v in rows[1][1:]]
    for r in rows[2:]:
        assert henry.mlmc_allocate(V, s, float(r[1])) == [int(v) for v in r[2:]]


def test_mlmc_allocate_rejects_bad_input(L):
    from paper_2302_07804_gb300 import henry
    with pytest.raises(henry.HenryError) as e:
        henry.mlmc_allocate([1e-5, 1e-6], [1.0, 0.0], 1e-6)
    assert e.value.code == henry.HENRY_EINVAL
    with pytest.raises(henry.HenryError):
        henry.mlmc_allocate([1e-5], [1.0], 0.0)
    assert henry.mlmc_allocate([0.0, 1e-6], [1.0, 2.0], 1e-6)[0] == 0


def test_create_validates_config(L):
    from paper_2302_07804_gb300 import henry
    for bad in (dict(nx0=30), dict(ny0=12, nx0=24), dict(precision=7), dict(nu1=-1), dict(max_level=12),
                dict(Lx=3.0), dict(ny0=1 << 12, nx0=1 << 13, max_level=8), dict(ny0=1 << 29, nx0=1 << 30, max_level=0),
                dict(steps0=1 << 26, max_level=5), dict(qoi_set=4), dict(workspace_bytes=0.0),
                dict(assembly_tile_w=16), dict(assembly_tile_w=512), dict(mg_threads=96), dict(mg_threads=1024),
                dict(newton_predictor_order=3), dict(newton_predictor_order=0)):
        with pytest.raises(henry.HenryError) as e:
            henry.Solver(**bad)
        assert e.value.code == henry.HENRY_EINVAL
    with pytest.raises(henry.HenryError) as e:
        henry.Solver(ny0=1 << 12, nx0=1 << 13, max_level=8)
    assert "finest level too large" in str(e.value)
    henry.Solver(ny0=1 << 10, nx0=1 << 11, max_level=4, steps0=1 << 20)   # 2^29 cells, 2^24 steps: accepted


def test_static_entry_checks_the_config_before_any_device_call(L):
    from paper_2302_07804_gb300 import henry
    P = ctypes.c_void_p
    for bad, text in ((dict(ny0=1 << 12, nx0=1 << 13, max_level=8), b"finest level too large"),
                      (dict(nx0=30), b"grid must be"), (dict(qoi_set=1), b"qoi_set 0"),
                      (dict(coef_model=henry.HENRY_MODEL_KL), b"three-parameter model")):
        cfg = henry.default_config()
        for k, v in bad.items():
            setattr(cfg, k, v)
        rc = L.henry_level_batch_solve_static(ctypes.byref(cfg), 0, 0, P(16), 1, P(16), None, P(16), None)
        assert rc == henry.HENRY_EINVAL
        assert text in L.henry_last_error()
    cfg = henry.default_config()
    cfg.workspace_bytes = 0.0        # no workspace budget on this path: not an error by itself
    assert L.henry_level_batch_solve_static(ctypes.byref(cfg), 0, 1, P(16), 1, P(16), P(16), P(16), None) == \
        henry.HENRY_EINVAL
    assert b"no coarse partner" in L.henry_last_error()


def test_null_and_range_arguments_return_einval(L):
    from paper_2302_07804_gb300 import henry
    P = ctypes.c_void_p
    assert L.henry_level_batch_solve(None, 0, 0, None, 1, None, None, None, None, None) == henry.HENRY_EINVAL
    assert b"NULL" in L.henry_last_error()
    s = henry.Solver()
    assert L.henry_level_batch_solve(s._h, 9, 0, P(16), 1, P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert L.henry_level_batch_solve(s._h, 0, 0, P(16), 0, P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert L.henry_level_batch_solve(s._h, 0, 1, P(16), 4, P(16), P(16), P(16), None, None) == henry.HENRY_EINVAL
    assert L.henry_sample_xi(1, 0, 0, 0, P(16), None) == henry.HENRY_EINVAL
    assert L.mlmc_accumulate(0, 0, 2, P(16), None, None, P(16), None) == henry.HENRY_EINVAL
    assert L.henry_assemble(s._h, -1, P(16), 1, P(16), P(16), P(16), None, None) == henry.HENRY_EINVAL
    lv = (ctypes.c_int32 * 3)(0, 1, 9)
    mixed = L.henry_batch_solve_mixed
    assert mixed(s._h, lv, 3, 0, P(16), P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert b"levels_host[2]" in L.henry_last_error()
    assert mixed(s._h, lv, 0, 0, P(16), P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert mixed(s._h, lv, 2, 1, P(16), P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert mixed(s._h, None, 2, 0, P(16), P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    assert mixed(None, lv, 2, 0, P(16), P(16), None, P(16), None, None) == henry.HENRY_EINVAL
    s.close()


def test_mlmc_rates_and_bias_test_match_oracle(L):
    import numpy as np
    from oracle import mlmc as omlmc
    from paper_2302_07804_gb300 import henry
    rows = golden_rows("paper_table_M_ell.txt")
    s = [float(v) for v in rows[0][1:]]
    V = [float(v) for v in rows[1][1:]]
    gen = np.random.default_rng(5)
    means = list(0.02 * 2.0 ** -np.arange(6) * np.exp(0.3 * gen.standard_normal(6)))
    for first in (0, 1, 2):
        got = henry.mlmc_rates(means, V, s, first_level=first)
        ref = omlmc.rates(means, V, s, first_level=first)
        np.testing.assert_allclose(got, ref, rtol=1e-12)
    a, b, g = henry.mlmc_rates(None, V, None)
    assert a is None and g is None and b == pytest.approx(omlmc.rates(means, V, s)[1], rel=1e-12)
    for alpha, eps in ((1.0, 1e-3), (0.7, 1e-2), (2.0, 1e-5)):
        b, ok = henry.mlmc_bias_test(means, alpha, eps)
        rb, rok = omlmc.bias_test(means, alpha, eps)
        assert b == pytest.approx(rb, rel=1e-14, abs=0) and ok == rok


def test_mlmc_rates_reject_bad_input(L):
    from paper_2302_07804_gb300 import henry
    for args in (([1.0], [1.0], [1.0], 0), ([1.0, 0.5], [1.0, 0.5], [1.0, 2.0], 1),
                 ([1.0, 0.0, 0.1], [1.0, 0.5, 0.2], [1.0, 2.0, 4.0], 0),
                 ([1.0, 0.5, 0.1], [1.0, -0.5, 0.2], [1.0, 2.0, 4.0], 0)):
        with pytest.raises(henry.HenryError) as e:
            henry.mlmc_rates(*args[:3], first_level=args[3])
        assert e.value.code == henry.HENRY_EINVAL
    for args in (([1.0], 1.0, 1e-3), ([1.0, 0.5], 0.0, 1e-3), ([1.0, 0.5], 1.0, 0.0),
                 ([1.0, float("nan")], 1.0, 1e-3), ([1.0, 0.5], float("inf"), 1e-3),
                 ([1.0, 0.5], float("nan"), 1e-3), ([1.0, 0.5], 1.0, float("inf"))):
        with pytest.raises(henry.HenryError):
            henry.mlmc_bias_test(*args)


def test_qoi_sets_and_paper_config(L):
    from paper_2302_07804_gb300 import henry
    for qs, nq in ((0, 2), (1, 15), (2, 15 + 32 * 16), (3, 15 + 20)):
        cfg = henry.default_config(qoi_set=qs)
        assert L.henry_n_qoi(ctypes.byref(cfg)) == nq
    assert L.henry_n_qoi(ctypes.byref(henry.default_config(qoi_set=4))) == -henry.HENRY_EINVAL
    with pytest.raises(henry.HenryError) as e:
        henry.Solver(qoi_set=4)
    assert e.value.code == henry.HENRY_EINVAL
    kw = henry.paper_config()
    assert (kw["T"], kw["steps0"], kw["g"], kw["rho1"]) == (6016.0, 188, 9.8, 1024.99)
    assert kw["coef_model"] == henry.HENRY_MODEL_TWO_LAYER and kw["qoi_set"] == henry.HENRY_QOI_PAPER
    assert henry.Solver(**kw).n_qoi == 15


def test_adjoint_and_rates_arguments_return_einval(L):
    from paper_2302_07804_gb300 import henry
    P = ctypes.c_void_p
    s = henry.Solver()
    adj = L.henry_adjoint
    assert adj(None, 0, P(16), 1, P(16), P(16), P(16), 20, P(16), None) == henry.HENRY_EINVAL
    assert adj(s._h, 0, P(16), 1, P(16), P(16), P(16), 0, P(16), None) == henry.HENRY_EINVAL
    assert b"checkpoint_every" in L.henry_last_error()
    assert adj(s._h, 0, P(16), 0, P(16), P(16), P(16), 20, P(16), None) == henry.HENRY_EINVAL
    assert adj(s._h, 9, P(16), 1, P(16), P(16), P(16), 20, P(16), None) == henry.HENRY_EINVAL
    assert adj(s._h, 0, None, 1, P(16), P(16), P(16), 20, P(16), None) == henry.HENRY_EINVAL
    assert L.henry_n_qoi(None) == -henry.HENRY_EINVAL
    s.close()
    bad = henry.Solver(adj_rtol=0.0)
    assert adj(bad._h, 0, P(16), 1, P(16), P(16), P(16), 20, P(16), None) == henry.HENRY_EINVAL
    bad.close()


def test_kl_basis_matches_oracle(L):
    """The library's KL basis (its own cyclic-Jacobi Nystrom eigensolver, the
    one the solves use) against the oracle's (LAPACK through scipy): the same
    eigenvalues, term order and modes at the cell centres."""
    import numpy as np
    from oracle import henry as ohenry
    from oracle import kl as okl
    from paper_2302_07804_gb300 import henry
    basis = okl.KLBasis()
    for level in (0, 2):
        sl, modes = henry.kl_basis(level)
        grid = ohenry.Grid.level(ohenry.Params(), level)
        xc = (np.arange(grid.nx) + 0.5) * grid.h
        yc = (np.arange(grid.ny) + 0.5) * grid.h
        np.testing.assert_allclose(sl, np.sqrt(basis.lam), rtol=1e-10)
        np.testing.assert_allclose(modes, basis.modes(xc, yc), rtol=0, atol=1e-9)
    P = ctypes.c_void_p
    assert L.henry_kl_basis(None, 0, P(16), None) == henry.HENRY_EINVAL
    cfg = henry.default_config()
    assert L.henry_kl_basis(ctypes.byref(cfg), 9, P(16), None) == henry.HENRY_EINVAL


def test_autotune_arguments_return_einval(L):
    from paper_2302_07804_gb300 import henry
    P = ctypes.c_void_p
    s = henry.Solver()
    t = henry.HenryTuning()
    assert L.henry_autotune(None, 0, 0, P(16), 4, ctypes.byref(t), None) == henry.HENRY_EINVAL
    assert L.henry_autotune(s._h, 0, 0, P(16), 0, ctypes.byref(t), None) == henry.HENRY_EINVAL
    assert L.henry_autotune(s._h, 0, 1, P(16), 4, ctypes.byref(t), None) == henry.HENRY_EINVAL
    assert L.henry_autotune(s._h, 9, 0, P(16), 4, ctypes.byref(t), None) == henry.HENRY_EINVAL
    # without tuning, a level's settings are the configuration's
    assert s.tuning(2) == {"lin_rtol": 1e-3, "nu1": 2, "nu2": 2, "fused_small_grids": 1, "cell_steps_per_s": 0.0,
                           "mg_tail_cells": -1, "newton_residual_first": 2, "newton_jacobian_every": 1,
                           "assembly_tile_w": 0, "mg_threads": 0, "newton_predictor_order": 2}
    for bad in (dict(mg_tail_cells=-2), dict(assembly_tile_w=48), dict(mg_threads=32), dict(newton_jacobian_every=0),
                dict(newton_predictor_order=3)):
        with pytest.raises(henry.HenryError):
            s.set_tuning(2, dict(s.tuning(2), **bad))
    good = dict(s.tuning(2), assembly_tile_w=32, mg_threads=128)
    s.set_tuning(2, good)
    assert s.tuning(2) == good
    s.close()


def test_binding_checks_tensors_before_passing_pointers(L):
    """Every tensor the binding hands to the library as a raw pointer is
    checked for shape, dtype, contiguity and device first (checked in that
    order, so each check is reachable with CPU tensors)."""
    import torch
    from paper_2302_07804_gb300 import henry
    f64 = torch.zeros((4, 3), dtype=torch.float64)
    cases = [
        (lambda: henry._dev_f64(f64, (4, 2), "xi"), "xi: expected shape (4, 2)"),
        (lambda: henry._dev_f64(f64.float(), (4, 3), "xi"), "expected torch.float64"),
        (lambda: henry._dev_f64(f64.t(), (3, 4), "xi"), "contiguous"),
        (lambda: henry._dev_f64(f64, (4, 3), "xi"), "expected a CUDA tensor"),
        (lambda: henry._dev_i32(torch.zeros(4, dtype=torch.int64), (4,), "status"), "expected torch.int32"),
        (lambda: henry._dev_f64([0.0], None, "xi"), "expected a torch.Tensor"),
        (lambda: henry._outputs((torch.zeros((4, 2), dtype=torch.float64), None,
                                 torch.zeros(4, dtype=torch.int32)), 4, 15, False, "cpu"), "out[0] (qoi_fine)"),
        (lambda: henry.mlmc_accumulate(0, torch.zeros((4, 2), dtype=torch.float64), None,
                                       torch.zeros(5, dtype=torch.int32), torch.zeros((2, 2, 3), dtype=torch.float64)),
         "expected a CUDA tensor"),
        (lambda: henry.mlmc_accumulate(0, torch.zeros(4, dtype=torch.float64), None, None, None), "[n][n_qoi]"),
    ]
    for call, text in cases:
        with pytest.raises(ValueError) as e:
            call()
        assert text in str(e.value), (text, str(e.value))
    s = henry.Solver(coef_model=henry.HENRY_MODEL_KL)
    with pytest.raises(ValueError) as e:       # 3 inputs per sample where the KL model takes 2 kl_terms + 1
        s.level_batch_solve(0, f64)
    assert "expected shape (4, 65)" in str(e.value)
    with pytest.raises(ValueError) as e:       # xi of the step calls is checked too
        s.assemble(0, f64, torch.zeros((4, 16, 32, 2), dtype=torch.float64),
                   torch.zeros((4, 16, 32, 2), dtype=torch.float64))
    assert "xi: expected shape (4, 65)" in str(e.value)
    s.close()


def test_fitted_bias_test_matches_the_oracle(L):
    """mlmc_bias_test_fit against oracle.mlmc.bias_test_fit on noisy power
    laws (the bench's bias test), and its argument checks."""
    from oracle import mlmc as omlmc
    from paper_2302_07804_gb300 import henry
    gen = np.random.default_rng(11)
    for trial in range(20):
        L_ = int(gen.integers(2, 7))
        alpha = float(gen.uniform(0.3, 2.0))
        means = [0.45] + [0.01 * 2.0 ** (-alpha * l) * (1 + 0.3 * gen.standard_normal()) * gen.choice([-1, 1])
                          for l in range(1, L_ + 1)]
        eps = float(gen.uniform(1e-4, 1e-2))
        b, ok, a = henry.mlmc_bias_test_fit(means, eps)
        bo, oko, ao = omlmc.bias_test_fit(means, eps)
        assert a == pytest.approx(ao, rel=1e-12) and b == pytest.approx(bo, rel=1e-10) and ok == oko
    D = ctypes.c_double
    arr = (D * 3)(0.4, 0.0, 0.01)
    assert L.mlmc_bias_test_fit(3, 1, arr, 0.5, 1e-3, None, None, None) == henry.HENRY_EINVAL
    arr = (D * 3)(0.4, 0.02, 0.01)
    assert L.mlmc_bias_test_fit(3, 2, arr, 0.5, 1e-3, None, None, None) == henry.HENRY_EINVAL
    assert L.mlmc_bias_test_fit(3, 1, arr, 0.0, 1e-3, None, None, None) == henry.HENRY_EINVAL
    assert L.mlmc_bias_test_fit(3, 1, arr, 0.5, 1e-3, None, None, None) == henry.HENRY_OK

