"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws reproducible
random arrays (states, vectors, seeds) of given shapes and ranges with numpy's
PCG64 generator.  Random numbers the method itself draws (the xi of each
scenario) come from Philox, implemented separately on each side.
"""
import numpy as np

#: Seed used for every synthetic workload (the arXiv number of the paper).
SEED = 230207804


def rng(tag: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED, int(tag)]))


def smooth_field(gen, ny, nx, lo, hi, modes=3):
    """A smooth random field on an (ny, nx) cell grid with values in [lo, hi]:
    a few random low-order cosine modes, rescaled."""
    y = (np.arange(ny) + 0.5) / ny
    x = (np.arange(nx) + 0.5) / nx
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = gen.integers(0, 4, size=2)
        ph = gen.uniform(0, 2 * np.pi, size=2)
        f += gen.normal() * np.cos(np.pi * kx * x + ph[0])[None, :] * np.cos(np.pi * ky * y + ph[1])[:, None]
    f += 0.2 * gen.standard_normal((ny, nx))
    f = (f - f.min()) / max(f.max() - f.min(), 1e-300)
    return lo + (hi - lo) * f


def random_states(tag, n, ny, nx, p_top, p_bottom, dp):
    """n random (p, c) pairs shaped (n, ny, nx): p a linear-in-depth profile from
    p_top (top row) to p_bottom (bottom row) plus a smooth perturbation of
    amplitude dp; c a smooth field in [0, 1]."""
    gen = rng(tag)
    y = (np.arange(ny) + 0.5) / ny
    base = p_bottom + (p_top - p_bottom) * y
    p = np.empty((n, ny, nx))
    c = np.empty((n, ny, nx))
    for i in range(n):
        p[i] = base[:, None] + smooth_field(gen, ny, nx, -dp, dp)
        c[i] = smooth_field(gen, ny, nx, 0.0, 1.0)
    return p, c


def random_vectors(tag, n, ny, nx):
    """n standard-normal vectors shaped (n, ny, nx, 2)."""
    return rng(tag).standard_normal((n, ny, nx, 2))


def uniform_xi(tag, n, n_xi=3):
    """n points uniform on [-1, 1]^n_xi (for tests that pass xi in directly)."""
    return rng(tag).uniform(-1.0, 1.0, size=(n, n_xi))


def kl_inputs(tag, n, terms=32):
    """n inputs of the KL random-field model: 2 x terms standard normals
    (theta_K, theta_phi) and one uniform on [-1, 1] (xi3), shaped (n, 2 terms + 1)."""
    gen = rng(tag)
    return np.concatenate([gen.standard_normal((n, 2 * terms)), gen.uniform(-1.0, 1.0, (n, 1))], axis=1)
