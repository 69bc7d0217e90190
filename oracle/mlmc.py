"""Multilevel Monte Carlo estimator and sample allocation (oracle; test infrastructure only).

Follows Sec. 3 of arXiv 2302.07804:

* Eq. (EgL): E[g_L] = E[g_0] + sum_{l=1}^{L} E[g_l - g_{l-1}].
* Eq. (A) and Def. (Yell): Y_l = mean over m_l independent samples of
  g_l - g_{l-1} (with g_{-1} = 0), fine and coarse of one sample driven by the
  same xi, independent xi across levels; Y = sum_l Y_l; Var[Y] = sum_l V_l / m_l.
* Eq. (M_ell): m_l = eps^-2 sqrt(V_l / s_l) sum_i sqrt(V_i s_i), with the total
  cost S = eps^-2 (sum_l sqrt(V_l s_l))^2 (here eps^2 is the variance budget
  passed in; Eq. (MSE) splits a mean-squared-error target eps^2 into eps^2/2
  for the variance and eps^2/2 for the squared bias).

Moments use the two-pass formula (mean first, then the centred sum of squares),
deliberately a different method from the one-pass pairwise merge of the CUDA
path.
"""
import math

import numpy as np


def level_differences(q_fine, q_coarse):
    """Y samples of one level: g_l - g_{l-1} (q_coarse None at level 0)."""
    q_fine = np.asarray(q_fine, dtype=np.float64)
    if q_coarse is None:
        return q_fine.copy()
    return q_fine - np.asarray(q_coarse, dtype=np.float64)


def two_pass_moments(y):
    """(n, mean, M2) per column of y[n][q], M2 = sum (y - mean)^2."""
    y = np.asarray(y, dtype=np.float64)
    n = y.shape[0]
    if n == 0:
        return 0, np.zeros(y.shape[1:]), np.zeros(y.shape[1:])
    mean = y.sum(axis=0) / n
    m2 = ((y - mean) ** 2).sum(axis=0)
    return n, mean, m2


def estimator(per_level_y):
    """MLMC estimate sum_l mean(Y_l) and its variance sum_l Var(Y_l)/m_l
    (unbiased sample variances) from lists of Y samples per level."""
    est = 0.0
    var = 0.0
    for y in per_level_y:
        n, mean, m2 = two_pass_moments(y)
        est = est + mean
        var = var + (m2 / (n - 1)) / n
    return est, var


def allocate(V, s, var_budget):
    """Eq. (M_ell): m_l = ceil(var_budget^-1 sqrt(V_l/s_l) sum_i sqrt(V_i s_i))."""
    V = [float(v) for v in V]
    s = [float(x) for x in s]
    # plain FP64 accumulation, level by level: ceil() is an integer decision
    # taken on a floating-point value, and both sides take it on the same
    # value (Python's sum() of floats is compensated, so it is not used here)
    tot = 0.0
    for v, c in zip(V, s):
        tot += math.sqrt(v * c)
    return [int(math.ceil(math.sqrt(v / c) * tot / var_budget)) for v, c in zip(V, s)]


def total_cost(V, s, var_budget):
    """S = var_budget^-1 (sum_l sqrt(V_l s_l))^2."""
    return (sum(math.sqrt(float(v) * float(c)) for v, c in zip(V, s))) ** 2 / var_budget


def rates(mean_Y, V, s, first_level=1):
    """Rates of Theorem (costMLMC) from per-level statistics: the least-squares
    slopes (numpy polyfit, degree 1) of log2 |E[Y_l]| (alpha = -slope, the weak
    error model), log2 V_l (beta = -slope, the variance model) and log2 s_l
    (gamma_d = d gamma = +slope, the cost model) over l = first_level .. L."""
    lev = np.arange(first_level, len(V))

    def slope(y):
        return np.polyfit(lev, np.log2(np.asarray(y, dtype=np.float64)[first_level:]), 1)[0]

    return -slope(np.abs(mean_Y)), -slope(V), slope(s)


def bias_test(mean_Y, alpha, eps):
    """Remaining bias of a level-L estimator under the weak error model
    |E[g_l - g]| = c 2^(-alpha l): E[g - g_L] = sum_{l > L} E[Y_l] = E[Y_L] / (2^alpha - 1)
    (geometric series); Eq. (MSE) asks its square to stay below eps^2 / 2.
    Returns (estimate, passed)."""
    b = abs(float(mean_Y[-1])) / (2.0 ** alpha - 1.0)
    return b, b <= eps / math.sqrt(2.0)


def bias_test_fit(mean_Y, eps, first_level=1, alpha_min=0.5):
    """The same remaining-bias estimate with E[Y_L] taken from the fitted weak
    error model instead of the level-L sample mean alone: log2 |E[Y_l]| =
    a - alpha l fitted by least squares (numpy polyfit) over l = first_level
    .. L; alpha = max(fitted slope, alpha_min), a refitted for that alpha
    (mean of log2 |E[Y_l]| + alpha l); E[Y_L] ~ 2^(a - alpha L), bias =
    E[Y_L] / (2^alpha - 1).  Returns (bias, passed, alpha)."""
    lev = np.arange(first_level, len(mean_Y))
    y = np.log2(np.abs(np.asarray(mean_Y, dtype=np.float64)[first_level:]))
    alpha = max(-np.polyfit(lev, y, 1)[0], alpha_min)
    a = float(np.mean(y + alpha * lev))
    b = float(2.0 ** (a - alpha * lev[-1]) / (2.0 ** alpha - 1.0))
    return b, bool(b <= eps / math.sqrt(2.0)), float(alpha)
