"""Thin ctypes binding of libhenry (include/henry.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
turns torch tensors into device pointers and the current CUDA stream into a
``cudaStream_t``.  There is no CPU fallback: ``lib()`` raises if the library
is missing or cannot be loaded.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhenry.so")

HENRY_OK, HENRY_EINVAL, HENRY_ECUDA, HENRY_ENOMEM, HENRY_ENOCONV, HENRY_ELIMIT = range(6)
HENRY_SAMPLE_OK, HENRY_SAMPLE_NEWTON, HENRY_SAMPLE_LINEAR, HENRY_SAMPLE_NONFINITE = range(4)
HENRY_FP64, HENRY_MIXED = 0, 1
HENRY_COARSE_REDISCRETISE, HENRY_COARSE_GALERKIN = 0, 1
HENRY_SCHEME_CELL, HENRY_SCHEME_VERTEX = 0, 1
HENRY_MODEL_UNIFORM3, HENRY_MODEL_KL, HENRY_MODEL_TWO_LAYER = 0, 1, 2
HENRY_QOI_STANDARD, HENRY_QOI_PAPER, HENRY_QOI_PAPER_FIELD, HENRY_QOI_PAPER_SERIES = 0, 1, 2, 3
N_QOI = 2
N_XI = 3

EXPORTS = ("henry_default_config", "henry_create", "henry_destroy", "henry_last_error", "henry_sample_xi",
           "henry_level_batch_solve", "mlmc_accumulate", "mlmc_allocate", "henry_assemble",
           "henry_apply_jacobian", "henry_precondition", "henry_linear_solve", "henry_profile",
           "henry_profile_read", "henry_level_batch_solve_static", "henry_batch_solve_mixed", "mlmc_rates", "mlmc_bias_test", "henry_adjoint", "henry_n_qoi",
           "henry_paper_config", "henry_kl_basis", "henry_autotune", "henry_get_tuning",
           "henry_set_tuning", "henry_vc_assemble", "mlmc_bias_test_fit")
KERNEL_CLASSES = ("assemble", "coarse_ops", "state_restrict", "smooth", "residual_restrict", "coarse_solve",
                  "spmv", "krylov", "newton", "qoi", "fused", "smooth_coarse", "residual", "mg_tail")


class HenryConfig(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("Lx", "Ly", "T", "rho0", "rho1", "mu", "g", "Dm")] + \
               [(n, ctypes.c_double) for n in ("phi_mean", "K_mean", "qin_mean")] + \
               [(n, ctypes.c_double) for n in ("phi_amp", "logK_amp", "qin_amp")] + \
               [(n, ctypes.c_int32) for n in ("nx0", "ny0", "steps0", "max_level", "precision", "coarse_op")] + \
               [(n, ctypes.c_double) for n in ("newton_atol", "newton_dxtol", "lin_rtol")] + \
               [(n, ctypes.c_int32) for n in ("newton_maxit", "lin_maxit", "nu1", "nu2")] + \
               [("workspace_bytes", ctypes.c_double), ("newton_predictor", ctypes.c_double),
                ("newton_dc_limit", ctypes.c_double),
                ("fused_small_grids", ctypes.c_int32), ("coef_model", ctypes.c_int32), ("kl_terms", ctypes.c_int32)] + \
               [(n, ctypes.c_double) for n in ("kl_corr_len", "kl_sigma_logK", "kl_sigma_phi", "phi_lo", "phi_hi")] + \
               [("lin_retry", ctypes.c_int32), ("finalize_nct", ctypes.c_int32), ("adj_rtol", ctypes.c_double),
                ("adj_maxit", ctypes.c_int32), ("cuda_graphs", ctypes.c_int32), ("qoi_set", ctypes.c_int32),
                ("tile_assembly", ctypes.c_int32), ("newton_residual_first", ctypes.c_int32),
                ("mg_tail_cells", ctypes.c_int32), ("mg_tail_batch_cells", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("newton_jacobian_every", ctypes.c_int32),
                ("level_priority", ctypes.c_int32), ("assembly_tile_w", ctypes.c_int32),
                ("mg_threads", ctypes.c_int32), ("newton_predictor_order", ctypes.c_int32)]


class HenryStats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int64), ("linear_iters", ctypes.c_int64),
                ("newton_solves", ctypes.c_int64), ("failed_samples", ctypes.c_int64),
                ("cell_steps", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HenryError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libhenry error %d: %s" % (code, msg))
        self.code = code


_lib = None


class HenryTuning(ctypes.Structure):
    """henry_tuning: a level's solver settings chosen by henry_autotune."""
    _fields_ = [("lin_rtol", ctypes.c_double), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("fused_small_grids", ctypes.c_int32), ("cell_steps_per_s", ctypes.c_double),
                ("mg_tail_cells", ctypes.c_int32), ("newton_residual_first", ctypes.c_int32),
                ("newton_jacobian_every", ctypes.c_int32), ("assembly_tile_w", ctypes.c_int32),
                ("mg_threads", ctypes.c_int32), ("newton_predictor_order", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """Load libhenry.so (built by ``paper_2302_07804_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhenry.so is not built (%s); run paper_2302_07804_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        U64 = ctypes.c_uint64
        L.henry_default_config.argtypes = [ctypes.POINTER(HenryConfig)]
        L.henry_default_config.restype = None
        L.henry_paper_config.argtypes = [ctypes.POINTER(HenryConfig)]
        L.henry_paper_config.restype = None
        L.henry_n_qoi.argtypes = [ctypes.POINTER(HenryConfig)]
        L.henry_kl_basis.argtypes = [ctypes.POINTER(HenryConfig), I, P, P]
        L.henry_autotune.argtypes = [P, I, I, P, I, ctypes.POINTER(HenryTuning), P]
        L.henry_get_tuning.argtypes = [P, I, ctypes.POINTER(HenryTuning)]
        L.henry_set_tuning.argtypes = [P, I, ctypes.POINTER(HenryTuning)]
        L.henry_create.argtypes = [ctypes.POINTER(HenryConfig), ctypes.POINTER(P)]
        L.henry_destroy.argtypes = [P]
        L.henry_destroy.restype = None
        L.henry_last_error.restype = ctypes.c_char_p
        L.henry_sample_xi.argtypes = [U64, I, U64, I, P, P]
        L.henry_level_batch_solve.argtypes = [P, I, I, P, I, P, P, P, ctypes.POINTER(HenryStats), P]
        L.henry_adjoint.argtypes = [P, I, P, I, P, P, P, I, P, P]
        L.henry_batch_solve_mixed.argtypes = [P, P, I, I, P, P, P, P, ctypes.POINTER(HenryStats), P]
        L.mlmc_accumulate.argtypes = [I, I, I, P, P, P, P, P]
        L.mlmc_allocate.argtypes = [I, ctypes.POINTER(D), ctypes.POINTER(D), D, ctypes.POINTER(I64)]
        L.mlmc_rates.argtypes = [I, I, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D),
                                 ctypes.POINTER(D), ctypes.POINTER(D)]
        L.mlmc_bias_test.argtypes = [I, ctypes.POINTER(D), D, D, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_int32)]
        L.mlmc_bias_test_fit.argtypes = [I, I, ctypes.POINTER(D), D, D, ctypes.POINTER(D), ctypes.POINTER(D),
                                         ctypes.POINTER(ctypes.c_int32)]
        L.henry_assemble.argtypes = [P, I, P, I, P, P, P, P, P]
        L.henry_apply_jacobian.argtypes = [P, I, P, I, P, P, P, P, P]
        L.henry_precondition.argtypes = [P, I, P, I, P, P, P, P, P]
        L.henry_linear_solve.argtypes = [P, I, P, I, P, P, P, P, P, P]
        L.henry_vc_assemble.argtypes = [P, I, P, I, P, P, P, P, P]
        L.henry_level_batch_solve_static.argtypes = [ctypes.POINTER(HenryConfig), I, I, P, I, P, P, P, P]
        L.henry_profile.argtypes = [P, I]
        L.henry_profile_read.argtypes = [P, I, ctypes.POINTER(D), ctypes.POINTER(I64), ctypes.POINTER(D),
                                         ctypes.POINTER(D)]
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("henry_default_config", "henry_destroy", "henry_last_error"):
                f.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc, allow=()):
    if rc != HENRY_OK and rc not in allow:
        raise HenryError(rc, lib().henry_last_error().decode())
    return rc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _expect(t, dtype, shape=None, name="tensor"):
    """Check a tensor the library will read or write through a raw pointer:
    its shape, dtype, contiguity and that it lives on the current CUDA device
    (the device the library launches on).  Raises ValueError otherwise."""
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s: expected a torch.Tensor, got %s" % (name, type(t).__name__))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s: expected shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if t.dtype != dtype:
        raise ValueError("%s: expected %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s: expected a contiguous tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s: expected a CUDA tensor, got one on %s" % (name, t.device))
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s: on %s, not on the current device cuda:%d" % (name, t.device, torch.cuda.current_device()))
    return t


def _dev_f64(t, shape=None, name="tensor"):
    return _expect(t, torch.float64, shape, name)


def _dev_i32(t, shape=None, name="tensor"):
    return _expect(t, torch.int32, shape, name)


def _outputs(out, n, nq, with_coarse, device):
    """The (qoi_fine, qoi_coarse or None, status) buffers of a batch solve:
    new tensors, or the caller's ``out`` after checking their shapes."""
    if out is None:
        qf = torch.empty((n, nq), dtype=torch.float64, device=device)
        qc = torch.empty((n, nq), dtype=torch.float64, device=device) if with_coarse else None
        st = torch.empty((n,), dtype=torch.int32, device=device)
        return qf, qc, st
    qf, qc, st = out
    _dev_f64(qf, (n, nq), "out[0] (qoi_fine)")
    if with_coarse:
        _dev_f64(qc, (n, nq), "out[1] (qoi_coarse)")
    else:
        qc = None
    _dev_i32(st, (n,), "out[2] (status)")
    return qf, qc, st


def default_config(**overrides):
    cfg = HenryConfig()
    lib().henry_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def paper_config(**overrides):
    """henry_paper_config: the paper's variant (constants, T = 6016 s in 188
    level-0 steps, two-layer porosity, the paper's QoIs) as Solver keyword
    arguments, with ``overrides`` applied."""
    cfg = HenryConfig()
    lib().henry_paper_config(ctypes.byref(cfg))
    kw = {name: getattr(cfg, name) for name, _ in HenryConfig._fields_}
    kw.update(overrides)
    return kw


def kl_basis(level, **overrides):
    """henry_kl_basis (host): (sqrt_lam[kl_terms], modes[kl_terms][ny][nx]) as
    numpy arrays for the configuration with ``overrides``."""
    import numpy as np
    cfg = default_config(**overrides)
    ny, nx = cfg.ny0 << level, cfg.nx0 << level
    sl = np.empty(cfg.kl_terms)
    modes = np.empty((cfg.kl_terms, ny, nx))
    _check(lib().henry_kl_basis(ctypes.byref(cfg), level, sl.ctypes.data_as(ctypes.c_void_p),
                                modes.ctypes.data_as(ctypes.c_void_p)))
    return sl, modes


def sample_xi(seed, level, first_sample, n, device="cuda", stream=None):
    """xi[n][3] on the device from Philox4x32-10 (henry_sample_xi)."""
    xi = torch.empty((n, N_XI), dtype=torch.float64, device=device)
    _check(lib().henry_sample_xi(seed, level, first_sample, n, _ptr(xi), _stream(stream)))
    return xi


def mlmc_accumulate(level, qoi_fine, qoi_coarse, status, sums, stream=None):
    """Merge a batch into sums[2][n_qoi][3] (count, mean, M2) in place."""
    if not isinstance(qoi_fine, torch.Tensor) or qoi_fine.dim() != 2:
        raise ValueError("qoi_fine: expected a [n][n_qoi] tensor")
    n, nq = qoi_fine.shape
    _dev_f64(qoi_fine, None, "qoi_fine")
    _dev_f64(sums, (2, nq, 3), "sums")
    if qoi_coarse is not None:
        _dev_f64(qoi_coarse, (n, nq), "qoi_coarse")
    if status is not None:
        _dev_i32(status, (n,), "status")
    _check(lib().mlmc_accumulate(level, n, nq, _ptr(qoi_fine), _ptr(qoi_coarse), _ptr(status), _ptr(sums),
                                 _stream(stream)))
    return sums


def mlmc_allocate(V, s, var_budget):
    """Eq. (M_ell) sample numbers (host)."""
    L = len(V)
    Va = (ctypes.c_double * L)(*[float(v) for v in V])
    sa = (ctypes.c_double * L)(*[float(v) for v in s])
    out = (ctypes.c_int64 * L)()
    _check(lib().mlmc_allocate(L, Va, sa, float(var_budget), out))
    return [int(v) for v in out]


def mlmc_rates(mean_Y=None, V=None, s=None, first_level=1):
    """(alpha, beta, gamma_d) of Theorem (costMLMC) from per-level statistics
    (host; mlmc_rates).  A rate whose input is None is returned as None."""
    ins = [mean_Y, V, s]
    n = len(next(a for a in ins if a is not None))
    arrs = [None if a is None else (ctypes.c_double * n)(*[float(v) for v in a]) for a in ins]
    outs = [ctypes.c_double() for _ in ins]
    refs = [None if a is None else ctypes.byref(o) for a, o in zip(ins, outs)]
    _check(lib().mlmc_rates(n, first_level, *arrs, *refs))
    return tuple(None if a is None else o.value for a, o in zip(ins, outs))


def mlmc_bias_test(mean_Y, alpha, eps):
    """(bias estimate |mean_Y[L]| / (2^alpha - 1), bias <= eps / sqrt 2) (host; mlmc_bias_test)."""
    n = len(mean_Y)
    arr = (ctypes.c_double * n)(*[float(v) for v in mean_Y])
    b, ok = ctypes.c_double(), ctypes.c_int32()
    _check(lib().mlmc_bias_test(n, arr, float(alpha), float(eps), ctypes.byref(b), ctypes.byref(ok)))
    return b.value, bool(ok.value)


def mlmc_bias_test_fit(mean_Y, eps, first_level=1, alpha_min=0.5):
    """(bias estimate from the fitted weak error model, passed, alpha) (host; mlmc_bias_test_fit)."""
    n = len(mean_Y)
    arr = (ctypes.c_double * n)(*[float(v) for v in mean_Y])
    a, b, ok = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().mlmc_bias_test_fit(n, first_level, arr, float(alpha_min), float(eps), ctypes.byref(a),
                                    ctypes.byref(b), ctypes.byref(ok)))
    return b.value, bool(ok.value), a.value


def level_batch_solve_static(cfg, level, xi, with_coarse=False, stream=None, allow_failures=False):
    """henry_level_batch_solve_static: the batch solve with the library's
    compiled-in device workspace (no device allocation by the library); for
    callers that cannot allocate.  Returns (qoi_fine, qoi_coarse or None, status)."""
    n = xi.shape[0]
    _dev_f64(xi, (n, N_XI), "xi")
    qf, qc, st = _outputs(None, n, N_QOI, with_coarse, xi.device)
    rc = lib().henry_level_batch_solve_static(ctypes.byref(cfg), level, 1 if with_coarse else 0, _ptr(xi), n,
                                              _ptr(qf), _ptr(qc), _ptr(st), _stream(stream))
    _check(rc, allow=(HENRY_ENOCONV,) if allow_failures else ())
    return qf, qc, st


class Solver:
    """Owns a henry_handle; see include/henry.h for the semantics of each call."""

    def __init__(self, **overrides):
        self.cfg = default_config(**overrides)
        h = ctypes.c_void_p()
        _check(lib().henry_create(ctypes.byref(self.cfg), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().henry_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, enable=True):
        """Turn per-kernel-class event timing on (counters reset) or off."""
        _check(lib().henry_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{class: (ms, launches, algorithmic bytes, algorithmic flops)} since the last reset."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            ms, n, b, f = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
            _check(lib().henry_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                            ctypes.byref(f)))
            out[name] = (ms.value, n.value, b.value, f.value)
        return out

    @property
    def n_qoi(self):
        """QoIs per sample for this configuration's qoi_set (henry_n_qoi)."""
        rc = lib().henry_n_qoi(ctypes.byref(self.cfg))
        if rc < 0:
            raise HenryError(-rc, lib().henry_last_error().decode())
        return rc

    @property
    def n_xi(self):
        """Random inputs per sample for this configuration's coefficient model."""
        return 2 * self.cfg.kl_terms + 1 if self.cfg.coef_model == HENRY_MODEL_KL else N_XI

    def grid(self, level):
        return (self.cfg.ny0 << level, self.cfg.nx0 << level)

    def state_shape(self, level):
        """(rows, columns) of a per-step state: cells, or vertices for the
        vertex-centred scheme."""
        ny, nx = self.grid(level)
        return (ny + 1, nx + 1) if self.cfg.scheme == HENRY_SCHEME_VERTEX else (ny, nx)

    def level_batch_solve(self, level, xi, with_coarse=False, stream=None, allow_failures=False, out=None):
        """Returns (qoi_fine[n][2], qoi_coarse[n][2] or None, status[n] int32, stats dict)."""
        n = xi.shape[0]
        _dev_f64(xi, (n, self.n_xi), "xi")
        qf, qc, st = _outputs(out, n, self.n_qoi, with_coarse, xi.device)
        stats = HenryStats()
        rc = lib().henry_level_batch_solve(self._h, level, 1 if with_coarse else 0, _ptr(xi), n, _ptr(qf), _ptr(qc),
                                           _ptr(st), ctypes.byref(stats), _stream(stream))
        _check(rc, allow=(HENRY_ENOCONV,) if allow_failures else ())
        return qf, qc, st, stats.as_dict()

    def batch_solve_mixed(self, levels, xi, with_coarse=False, stream=None, allow_failures=False, out=None):
        """Uneven batch: sample i at level levels[i] (henry_batch_solve_mixed).
        Returns (qoi_fine[n][2], qoi_coarse[n][2] or None, status[n] int32, stats dict)."""
        import numpy as np
        lv = np.ascontiguousarray(np.asarray(levels, dtype=np.int32))
        n = xi.shape[0]
        if lv.shape != (n,):
            raise ValueError("levels must hold one level per row of xi")
        _dev_f64(xi, (n, self.n_xi), "xi")
        qf, qc, st = _outputs(out, n, self.n_qoi, with_coarse, xi.device)
        stats = HenryStats()
        rc = lib().henry_batch_solve_mixed(self._h, lv.ctypes.data_as(ctypes.c_void_p), n, 1 if with_coarse else 0,
                                           _ptr(xi), _ptr(qf), _ptr(qc), _ptr(st), ctypes.byref(stats),
                                           _stream(stream))
        _check(rc, allow=(HENRY_ENOCONV,) if allow_failures else ())
        return qf, qc, st, stats.as_dict()

    def adjoint(self, level, xi, weights, checkpoint_every=20, stream=None, allow_failures=False):
        """dQ/dxi for Q = weights[:, 0] mass + weights[:, 1] c_point (henry_adjoint).
        Returns (grad[n][n_xi], qoi[n][2], status[n] int32)."""
        n = xi.shape[0]
        _dev_f64(xi, (n, self.n_xi), "xi")
        _dev_f64(weights, (n, N_QOI), "weights")
        grad = torch.empty((n, self.n_xi), dtype=torch.float64, device=xi.device)
        qoi = torch.empty((n, self.n_qoi), dtype=torch.float64, device=xi.device)
        st = torch.empty((n,), dtype=torch.int32, device=xi.device)
        rc = lib().henry_adjoint(self._h, level, _ptr(xi), n, _ptr(weights), _ptr(grad), _ptr(qoi),
                                 int(checkpoint_every), _ptr(st), _stream(stream))
        _check(rc, allow=(HENRY_ENOCONV,) if allow_failures else ())
        return grad, qoi, st

    def autotune(self, level, xi, with_coarse=False, stream=None):
        """henry_autotune: time the candidate settings on the trial batch xi and
        keep the fastest for this level; returns it as a dict."""
        n = xi.shape[0]
        _dev_f64(xi, (n, self.n_xi), "xi")
        t = HenryTuning()
        _check(lib().henry_autotune(self._h, level, 1 if with_coarse else 0, _ptr(xi), n, ctypes.byref(t),
                                    _stream(stream)))
        return t.as_dict()

    def set_tuning(self, level, tuning):
        """henry_set_tuning: a dict as returned by tuning() / autotune(), or None."""
        if tuning is None:
            _check(lib().henry_set_tuning(self._h, level, None))
            return
        t = HenryTuning()
        for k, _ in HenryTuning._fields_:
            setattr(t, k, tuning.get(k, 0))
        _check(lib().henry_set_tuning(self._h, level, ctypes.byref(t)))

    def tuning(self, level):
        """The settings this level's solves use (henry_get_tuning)."""
        t = HenryTuning()
        _check(lib().henry_get_tuning(self._h, level, ctypes.byref(t)))
        return t.as_dict()

    def _states(self, level, xi, state, state_old):
        ny, nx = self.state_shape(level)
        n = state.shape[0]
        _dev_f64(xi, (n, self.n_xi), "xi")
        _dev_f64(state, (n, ny, nx, 2), "state")
        _dev_f64(state_old, (n, ny, nx, 2), "state_old")
        return n, ny, nx

    def assemble(self, level, xi, state, state_old, with_jacobian=True, stream=None):
        n, ny, nx = self._states(level, xi, state, state_old)
        nb = 9 if self.cfg.scheme == HENRY_SCHEME_VERTEX else 5
        F = torch.empty((n, ny, nx, 2), dtype=torch.float64, device=state.device)
        J = torch.empty((n, ny, nx, nb, 2, 2), dtype=torch.float64, device=state.device) if with_jacobian else None
        _check(lib().henry_assemble(self._h, level, _ptr(xi), n, _ptr(state), _ptr(state_old), _ptr(F), _ptr(J),
                                    _stream(stream)))
        return F, J

    def apply_jacobian(self, level, xi, state, state_old, x, stream=None):
        n, ny, nx = self._states(level, xi, state, state_old)
        _dev_f64(x, (n, ny, nx, 2), "x")
        y = torch.empty_like(x)
        _check(lib().henry_apply_jacobian(self._h, level, _ptr(xi), n, _ptr(state), _ptr(state_old), _ptr(x),
                                          _ptr(y), _stream(stream)))
        return y

    def precondition(self, level, xi, state, state_old, b, stream=None):
        n, ny, nx = self._states(level, xi, state, state_old)
        _dev_f64(b, (n, ny, nx, 2), "b")
        z = torch.empty_like(b)
        _check(lib().henry_precondition(self._h, level, _ptr(xi), n, _ptr(state), _ptr(state_old), _ptr(b),
                                        _ptr(z), _stream(stream)))
        return z

    def linear_solve(self, level, xi, state, state_old, b, stream=None):
        n, ny, nx = self._states(level, xi, state, state_old)
        _dev_f64(b, (n, ny, nx, 2), "b")
        x = torch.empty_like(b)
        its = torch.empty((n,), dtype=torch.int32, device=b.device)
        _check(lib().henry_linear_solve(self._h, level, _ptr(xi), n, _ptr(state), _ptr(state_old), _ptr(b),
                                        _ptr(x), _ptr(its), _stream(stream)))
        return x, its

    def vc_assemble(self, level, xi, state, state_old, with_jacobian=True, stream=None):
        """henry_vc_assemble: residual (n, ny+1, nx+1, 2) and Jacobian rows
        (n, ny+1, nx+1, 3, 3, 2, 2) of the vertex-centred scheme at the vertex
        states (n, ny+1, nx+1, 2)."""
        ny, nx = self.grid(level)
        n = state.shape[0]
        _dev_f64(xi, (n, self.n_xi), "xi")
        _dev_f64(state, (n, ny + 1, nx + 1, 2), "state")
        _dev_f64(state_old, (n, ny + 1, nx + 1, 2), "state_old")
        R = torch.empty_like(state)
        J = torch.empty((n, ny + 1, nx + 1, 3, 3, 2, 2), dtype=torch.float64, device=state.device) \
            if with_jacobian else None
        _check(lib().henry_vc_assemble(self._h, level, _ptr(xi), n, _ptr(state), _ptr(state_old), _ptr(R),
                                       _ptr(J), _stream(stream)))
        return R, J


class _ScenarioQoI(torch.autograd.Function):
    """qoi[n][2] = solve(xi) with the discrete adjoint as its backward: the
    forward is henry_level_batch_solve; backward calls henry_adjoint with the
    incoming gradient as the QoI weights (the adjoint recomputes the forward
    with checkpoints)."""

    @staticmethod
    def forward(ctx, xi, solver, level, checkpoint_every):
        qf, _, st, _ = solver.level_batch_solve(level, xi.detach().contiguous(), allow_failures=True)
        ctx.solver, ctx.level, ctx.ckpt = solver, level, checkpoint_every
        ctx.save_for_backward(xi)
        ctx.status = st
        return qf

    @staticmethod
    def backward(ctx, grad_out):
        (xi,) = ctx.saved_tensors
        grad, _, _ = ctx.solver.adjoint(ctx.level, xi.detach().contiguous(), grad_out.contiguous(),
                                        checkpoint_every=ctx.ckpt, allow_failures=True)
        return grad, None, None, None


def scenario_qoi(solver, level, xi, checkpoint_every=20):
    """Differentiable QoIs of a batch of scenarios (torch.autograd): qoi[n][2]
    at MLMC level ``level`` for inputs xi[n][n_xi]; backward through
    henry_adjoint."""
    return _ScenarioQoI.apply(xi, solver, level, checkpoint_every)
