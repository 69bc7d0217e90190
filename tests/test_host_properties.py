"""Property-based checks (hypothesis) of the host-side MLMC functions on
random inputs: the sample allocation of Eq. (M_ell), the host merge of
replica tables against the two-pass moments of the union, and the rate fit
of Theorem costMLMC on exact power laws.  Skipped where hypothesis is not
installed."""
import math

import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st

from oracle import mlmc as omlmc

pos = st.floats(min_value=1e-8, max_value=1e3, allow_nan=False, allow_infinity=False)


@pytest.fixture(scope="module")
def henry():
    from paper_2302_07804_gb300 import build, henry as h
    build.build()
    return h


@settings(max_examples=60, deadline=None)
@given(st.lists(st.tuples(pos, pos), min_size=1, max_size=7), st.floats(min_value=1e-9, max_value=1e-2))
def test_allocation_properties(henry, levels, budget):
    """m_l = ceil of the optimum of Eq. (M_ell): it meets the variance budget,
    stays within one sample of the real optimum per level, follows the
    oracle, and more samples go where V_l / s_l is larger."""
    V = [v for v, _ in levels]
    s = [c for _, c in levels]
    m = henry.mlmc_allocate(V, s, budget)
    assert m == omlmc.allocate(V, s, budget)
    tot = math.fsum(math.sqrt(v * c) for v, c in levels)
    for ml, v, c in zip(m, V, s):
        opt = math.sqrt(v / c) * tot / budget      # the real optimum, to a few ulps
        assert opt * (1 - 1e-14) <= ml < opt * (1 + 1e-14) + 1
    assert math.fsum(v / ml for v, ml in zip(V, m)) <= budget * (1 + 1e-12)
    for a in range(len(V)):
        for b in range(len(V)):
            if V[a] / s[a] > 1.01 * V[b] / s[b]:
                assert m[a] >= m[b]


@settings(max_examples=40, deadline=None)
@given(st.lists(st.integers(min_value=1, max_value=40), min_size=1, max_size=5), st.integers(0, 2 ** 31))
def test_merged_replica_tables_equal_two_pass_moments(sizes, seed):
    from paper_2302_07804_gb300 import mlmc
    gen = np.random.default_rng(seed)
    parts, data = [], []
    for n in sizes:
        y = gen.normal(gen.uniform(-5, 5), gen.uniform(0.01, 3.0), size=(n, 3))
        data.append(y)
        t = np.zeros((2, 3, 3))
        t[:, :, 0] = n
        t[:, :, 1] = y.mean(axis=0)
        t[:, :, 2] = ((y - y.mean(axis=0)) ** 2).sum(axis=0)
        parts.append(t)
    merged = mlmc.merge_sums(parts).numpy()
    allv = np.concatenate(data)
    n, mean, m2 = omlmc.two_pass_moments(allv)
    assert np.all(merged[0, :, 0] == n)
    np.testing.assert_allclose(merged[0, :, 1], mean, rtol=1e-12, atol=1e-12 * np.abs(allv).max())
    np.testing.assert_allclose(merged[0, :, 2], m2, rtol=1e-10, atol=1e-10 * max(1.0, m2.max()))


@settings(max_examples=40, deadline=None)
@given(st.floats(0.3, 3.0), st.floats(0.3, 4.0), st.floats(0.5, 4.0), st.floats(1e-4, 1.0),
       st.integers(3, 7), st.integers(0, 2))
def test_rates_recover_exact_power_laws(henry, alpha, beta, gamma, c0, n_levels, first):
    """|E Y_l| = c0 2^(-alpha l), V_l = c0 2^(-beta l), s_l = 2^(gamma l) give
    exactly (alpha, beta, gamma) from any first level; both sides agree."""
    if n_levels - first < 2:
        return
    l = np.arange(n_levels)
    means = list(c0 * 2.0 ** (-alpha * l))
    V = list(c0 * 2.0 ** (-beta * l))
    s = list(2.0 ** (gamma * l))
    a, b, g = henry.mlmc_rates(means, V, s, first_level=first)
    assert a == pytest.approx(alpha, rel=1e-9, abs=0) and b == pytest.approx(beta, rel=1e-9, abs=0)
    assert g == pytest.approx(gamma, rel=1e-9, abs=0)
    np.testing.assert_allclose((a, b, g), omlmc.rates(means, V, s, first_level=first), rtol=1e-12)


@settings(max_examples=8, deadline=None)
@given(st.floats(min_value=0.1, max_value=1.2), st.integers(min_value=1, max_value=64))
def test_kl_basis_agrees_with_the_oracle_to_its_conditioning(henry, ell, terms):
    """The library's KL basis (cyclic Jacobi) against the oracle's (LAPACK)
    for any correlation length and number of terms.  Eigenvalues far below
    the largest are fixed only to rounding of the largest, and so are their
    modes, so the comparison is absolute in lam_max: the eigenvalues to
    1e-13 lam_max, the field contributions sqrt(lam_k) psi_k of the terms
    with lam_k >= 1e-12 lam_max to 1e-9 sqrt(lam_max), and those of the
    terms below, whose eigenvalues lie within rounding of zero (long
    correlation lengths with many terms, e.g. 1.125 with 56), to
    1e-6 sqrt(lam_max) = sqrt(1e-12 lam_max) times the modes' unit scale."""
    from oracle import henry as oh
    from oracle import kl as okl
    sl, modes = henry.kl_basis(0, kl_terms=terms, kl_corr_len=ell)
    b = okl.KLBasis(n_terms=terms, ell=ell)
    grid = oh.Grid.level(oh.Params(), 0)
    xc = (np.arange(grid.nx) + 0.5) * grid.h
    yc = (np.arange(grid.ny) + 0.5) * grid.h
    lmax = b.lam.max()
    assert np.abs(sl ** 2 - b.lam).max() <= 1e-13 * lmax
    f_lib = sl[:, None, None] * modes
    f_orc = np.sqrt(b.lam)[:, None, None] * b.modes(xc, yc)
    d = np.abs(f_lib - f_orc).reshape(terms, -1).max(axis=1)
    resolved = b.lam >= 1e-12 * lmax
    assert d[resolved].max() <= 1e-9 * np.sqrt(lmax)
    if (~resolved).any():
        assert d[~resolved].max() <= 1e-6 * np.sqrt(lmax)


ints = st.one_of(st.integers(min_value=-3, max_value=70), st.sampled_from([0, 1 << 20, 1 << 29, (1 << 31) - 1, -(1 << 31)]))
reals = st.one_of(st.floats(allow_nan=True, allow_infinity=True, width=64), st.sampled_from([0.0, -1.0, 1e-300]))


@settings(max_examples=300, deadline=None)
@given(ny0=st.one_of(st.sampled_from([4, 8, 16, 32, 64]), ints), max_level=ints, steps0=ints, precision=ints,
       coef_model=ints, qoi_set=ints, T=reals, lin_rtol=reals, Ly=st.sampled_from([1.0, 0.5, -1.0, 0.0]))
def test_create_accepts_only_valid_configurations(henry, ny0, max_level, steps0, precision, coef_model, qoi_set, T,
                                                   lin_rtol, Ly):
    """henry_create on random configurations (host only; no device memory is
    touched): it returns OK or EINVAL, never anything else, and a
    configuration it accepts satisfies the documented rules."""
    import ctypes
    cfg = henry.default_config()
    nx0 = 2 * ny0 if -(1 << 30) < ny0 < (1 << 30) else ny0
    for k, v in dict(ny0=ny0, nx0=nx0, max_level=max_level, steps0=steps0, precision=precision,
                     coef_model=coef_model, qoi_set=qoi_set, T=T, lin_rtol=lin_rtol, Ly=Ly, Lx=2 * Ly).items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = henry.lib().henry_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc in (henry.HENRY_OK, henry.HENRY_EINVAL)
    if rc == henry.HENRY_OK:
        henry.lib().henry_destroy(h)
        assert ny0 >= 4 and ny0 & (ny0 - 1) == 0 and 0 <= max_level <= 8
        assert ((2 * ny0) << max_level) * (ny0 << max_level) <= 1 << 30 and 0 < steps0 <= (1 << 30) >> max_level
        assert precision in (henry.HENRY_FP64, henry.HENRY_MIXED) and 0 <= coef_model <= 2 and 0 <= qoi_set <= 3
        assert math.isfinite(T) and T > 0 and math.isfinite(lin_rtol) and lin_rtol > 0 and Ly > 0
    else:
        assert henry.lib().henry_last_error()


def test_create_rejects_nan_and_non_positive_physics(henry):
    import ctypes
    fields = ("Lx", "Ly", "T", "rho0", "rho1", "mu", "g", "Dm", "phi_mean", "K_mean", "qin_mean", "phi_amp",
              "logK_amp", "qin_amp", "newton_atol", "newton_dxtol", "lin_rtol", "workspace_bytes",
              "newton_predictor", "newton_dc_limit", "kl_corr_len", "kl_sigma_logK", "kl_sigma_phi", "phi_lo",
              "phi_hi", "adj_rtol")
    for f in fields:
        for bad in (math.nan, math.inf):
            cfg = henry.default_config()
            setattr(cfg, f, bad)
            h = ctypes.c_void_p()
            assert henry.lib().henry_create(ctypes.byref(cfg), ctypes.byref(h)) == henry.HENRY_EINVAL, (f, bad)
    for f, bad in (("rho0", 0.0), ("mu", -1e-3), ("g", 0.0), ("Dm", 0.0), ("K_mean", 0.0), ("phi_mean", 1.0),
                   ("newton_atol", -1.0)):
        cfg = henry.default_config()
        setattr(cfg, f, bad)
        h = ctypes.c_void_p()
        assert henry.lib().henry_create(ctypes.byref(cfg), ctypes.byref(h)) == henry.HENRY_EINVAL, (f, bad)


anyf = st.floats(allow_nan=True, allow_infinity=True, width=64)


@settings(max_examples=300, deadline=None)
@given(st.lists(st.tuples(anyf, anyf, anyf), min_size=1, max_size=6), anyf, anyf, st.integers(-1, 6))
def test_host_mlmc_functions_on_arbitrary_doubles(henry, rows, budget, alpha, first):
    """mlmc_allocate, mlmc_rates and mlmc_bias_test on any doubles (NaN,
    infinities, negatives, denormals): OK or EINVAL, and an OK result is
    finite and in range."""
    import ctypes
    L = henry.lib()
    n = len(rows)
    mean = (ctypes.c_double * n)(*[r[0] for r in rows])
    V = (ctypes.c_double * n)(*[r[1] for r in rows])
    s = (ctypes.c_double * n)(*[r[2] for r in rows])
    m = (ctypes.c_int64 * n)()
    rc = L.mlmc_allocate(n, V, s, budget, m)
    assert rc in (henry.HENRY_OK, henry.HENRY_EINVAL)
    if rc == henry.HENRY_OK:
        assert all(0 <= v < 9.0e18 for v in m)
    a, b, g = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = L.mlmc_rates(n, first, mean, V, s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(g))
    assert rc in (henry.HENRY_OK, henry.HENRY_EINVAL)
    if rc == henry.HENRY_OK:
        assert all(math.isfinite(x.value) for x in (a, b, g))
    bias, ok = ctypes.c_double(), ctypes.c_int32()
    rc = L.mlmc_bias_test(n, mean, alpha, budget, ctypes.byref(bias), ctypes.byref(ok))
    assert rc in (henry.HENRY_OK, henry.HENRY_EINVAL)
    if rc == henry.HENRY_OK:
        assert math.isfinite(bias.value) and bias.value >= 0 and ok.value in (0, 1)
