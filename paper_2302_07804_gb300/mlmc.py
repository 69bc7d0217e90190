"""Host-side MLMC driver over libhenry (Sec. 3 of arXiv 2302.07804).

For each level l the driver draws fresh xi with Philox (counters continue
from the samples already used on that level, so batches are independent and
a run resumes exactly from its counters), solves the fine scenario and its
coarse partner with the same xi in one ``henry_level_batch_solve`` call, and
merges Y_l = g_l - g_{l-1} into per-level running (count, mean, M2) sums on
the device with ``mlmc_accumulate`` (Eqs. EgL, A and Def. Yell).  Sample
numbers follow Eq. (M_ell) through ``mlmc_allocate``, with the variance
budget eps^2 / 2 of Eq. (MSE) and the level cost s_l proportional to the
cell-steps of a sample and its coarse partner (Eq. CompComplexity:
s_l = O(n_l r_l)), or the measured GPU time per sample.
"""
import json
import math
import time

import torch

from . import henry


def level_cost_model(cfg, level):
    """Cell-steps of one level-l sample plus its coarse partner."""
    def cs(l):
        return (cfg.nx0 << l) * (cfg.ny0 << l) * (cfg.steps0 << l)
    return cs(level) + (cs(level - 1) if level > 0 else 0)


class LevelState:
    def __init__(self, level, device, n_qoi=henry.N_QOI):
        self.level = level
        self.n_used = 0          # Philox counter offset: samples drawn so far
        self.sums = torch.zeros((2, n_qoi, 3), dtype=torch.float64, device=device)
        self.gpu_seconds = 0.0
        self.cell_steps = 0.0
        self.failed = 0

    def moments(self):
        """(count, mean[q], var[q]) of Y_l from the device sums."""
        S = self.sums.cpu()
        n = float(S[0, 0, 0])
        mean = S[0, :, 1].tolist()
        var = [(float(S[0, q, 2]) / (n - 1)) if n > 1 else float("nan") for q in range(S.shape[1])]
        return n, mean, var

    def to_json(self):
        return {"level": self.level, "n_used": self.n_used, "sums": self.sums.cpu().tolist(),
                "gpu_seconds": self.gpu_seconds, "cell_steps": self.cell_steps, "failed": self.failed}

    @staticmethod
    def from_json(d, device):
        st = LevelState(d["level"], device, n_qoi=len(d["sums"][0]))
        st.n_used = d["n_used"]
        st.sums = torch.tensor(d["sums"], dtype=torch.float64, device=device)
        st.gpu_seconds = d["gpu_seconds"]
        st.cell_steps = d["cell_steps"]
        st.failed = d["failed"]
        return st


def run_level(solver, st, n, seed, stream=None, xi=None):
    """Solve n new samples of level st.level (with coarse partners) and merge
    them into st.sums; returns the henry_stats of the call."""
    lev = st.level
    if xi is not None and xi.shape[0] != n:
        raise ValueError("xi holds %d samples, n = %d" % (xi.shape[0], n))
    if xi is None:
        xi = henry.sample_xi(seed, lev, st.n_used, n, device=st.sums.device, stream=stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s = stream if stream is not None else torch.cuda.current_stream()
    e0.record(s)
    qf, qc, status, stats = solver.level_batch_solve(lev, xi, with_coarse=lev > 0, stream=stream,
                                                     allow_failures=True)
    henry.mlmc_accumulate(lev, qf, qc, status, st.sums, stream=stream)
    e1.record(s)
    e1.synchronize()
    st.gpu_seconds += e0.elapsed_time(e1) / 1e3
    st.n_used += n
    st.cell_steps += stats["cell_steps"]
    st.failed += int(stats["failed_samples"])
    return stats


def run_levels(solver, states, counts, seed):
    """Solve counts[i] new samples of every level states[i].level (with coarse
    partners) in ONE henry_batch_solve_mixed call, so that the levels run
    concurrently, and merge each level's Y into its sums.  The samples, their
    Philox counters and each level's accumulation batches are those of
    run_level called level by level, so the sums are the same."""
    import numpy as np
    dev = states[0].sums.device
    todo = [(st, n) for st, n in zip(states, counts) if n > 0]
    if not todo:
        return
    xs = [henry.sample_xi(seed, st.level, st.n_used, n, device=dev) for st, n in todo]
    levels = np.concatenate([np.full(n, st.level, dtype=np.int32) for st, n in todo])
    xi = torch.cat(xs).contiguous()
    qf, qc, status, _ = solver.batch_solve_mixed(levels, xi, with_coarse=True, allow_failures=True)
    a = 0
    for st, n in todo:
        b = a + n
        henry.mlmc_accumulate(st.level, qf[a:b], qc[a:b] if st.level > 0 else None, status[a:b], st.sums)
        st.n_used += n
        st.cell_steps += n * level_cost_model(solver.cfg, st.level)
        st.failed += int((status[a:b] != 0).sum())
        a = b


def merge_sums(parts):
    """Chan's pairwise merge of a list of (count, mean, M2) tables, on the host
    (used to combine replicas that ran disjoint counter ranges)."""
    out = None
    for p in parts:
        p = torch.as_tensor(p, dtype=torch.float64).cpu().clone()
        if out is None:
            out = p
            continue
        na, ma, m2a = out[..., 0], out[..., 1], out[..., 2]
        nb, mb, m2b = p[..., 0], p[..., 1], p[..., 2]
        n = na + nb
        d = mb - ma
        safe = torch.where(n > 0, n, torch.ones_like(n))
        mean = torch.where(n > 0, ma + d * nb / safe, ma)
        m2 = torch.where(n > 0, m2a + m2b + d * d * na * nb / safe, m2a)
        out = torch.stack([n, mean, m2], dim=-1)
    return out


def run_mlmc(solver, eps=1e-3, max_level=3, pilot=(1000, 200, 50, 20), seed=None, qoi=1, cost="model",
             var_fraction=0.5, max_rounds=4, state=None, log=None, concurrent=True):
    """MLMC estimate of E[g_L] for QoI ``qoi`` (0 salt mass, 1 c at the point)
    to a variance budget var_fraction * eps^2 (Eq. MSE); returns a dict.
    concurrent (with the model cost): each round's samples of all levels go
    to one henry_batch_solve_mixed call; otherwise level by level (needed for
    cost="measured", which times each level's solves)."""
    from . import inputs
    if not 0 <= max_level <= solver.cfg.max_level:
        raise ValueError("max_level %d outside [0, %d]" % (max_level, solver.cfg.max_level))
    if len(pilot) < max_level + 1:
        raise ValueError("pilot gives %d levels' sample numbers, max_level %d needs %d"
                         % (len(pilot), max_level, max_level + 1))
    if state and len(state) > max_level + 1:
        raise ValueError("state holds %d levels, more than max_level + 1 = %d" % (len(state), max_level + 1))
    seed = inputs.SEED if seed is None else seed
    dev = torch.device("cuda", torch.cuda.current_device())
    levels = list(state) if state else []
    levels += [LevelState(l, dev, n_qoi=solver.n_qoi) for l in range(len(levels), max_level + 1)]
    t0 = time.perf_counter()
    together = concurrent and cost == "model"

    def solve_round(counts):
        if together:
            run_levels(solver, levels, counts, seed)
        else:
            for st, n in zip(levels, counts):
                if n:
                    run_level(solver, st, n, seed)

    solve_round([max(0, pilot[l] - levels[l].n_used) for l in range(max_level + 1)])
    budget = var_fraction * eps * eps
    alloc = None
    for rnd in range(max_rounds):
        V = []
        s = []
        for st in levels:
            n, mean, var = st.moments()
            V.append(max(var[qoi], 1e-300))
            s.append(level_cost_model(solver.cfg, st.level) if cost == "model"
                     else st.gpu_seconds / max(st.n_used, 1))
        alloc = henry.mlmc_allocate(V, s, budget)
        extra = [max(0, m - st.n_used) for m, st in zip(alloc, levels)]
        if log:
            log("round %d: V=%s m=%s extra=%s" % (rnd, ["%.3g" % v for v in V], alloc, extra))
        if sum(extra) == 0:
            break
        solve_round(extra)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    est = 0.0
    var_est = 0.0
    per = []
    for st in levels:
        n, mean, var = st.moments()
        est += mean[qoi]
        var_est += var[qoi] / n
        per.append({"level": st.level, "n": int(n), "mean_Y": mean[qoi], "var_Y": var[qoi],
                    "gpu_seconds": st.gpu_seconds, "cell_steps": st.cell_steps, "failed": st.failed})
    return {"estimate": est, "variance": var_est, "rmse_stat": math.sqrt(var_est), "eps": eps,
            "var_budget": budget, "alloc": alloc, "wall_seconds": wall,
            "cell_steps": sum(p["cell_steps"] for p in per), "levels": per,
            "checkpoint": json.dumps([st.to_json() for st in levels]), "state": levels}


def run_mlmc_adaptive(solver, eps=1e-3, L_start=2, L_max=None, pilot=(1000, 200, 50, 20, 10, 10, 10, 10, 10),
                      seed=None, qoi=1, cost="model", alpha_min=0.5, log=None, bias="last"):
    """MLMC with the finest level chosen by the bias test (Sec. 3: Eq. (MSE)
    splits eps^2 into eps^2 / 2 for the variance and eps^2 / 2 for the
    squared bias).  Levels 0 .. L_start are allocated as in run_mlmc; the weak
    rate alpha is fitted over levels 1 .. L (mlmc_rates, at least alpha_min),
    and level L + 1 is added while the bias test fails and L < L_max.
    bias = "last": E[Y_L] is the level-L sample mean (mlmc_bias_test);
    "fit": E[Y_L] from the fitted weak error model (mlmc_bias_test_fit).  The
    result of the last run_mlmc pass carries L, the rates and the bias test
    (both estimates)."""
    if bias not in ("last", "fit"):
        raise ValueError("bias must be 'last' or 'fit'")
    rule = bias
    L_max = solver.cfg.max_level if L_max is None else L_max
    if L_start < 2 or L_start > L_max:
        raise ValueError("need 2 <= L_start <= L_max to fit the weak rate over levels 1 .. L")
    t0 = time.perf_counter()
    state = None
    L = L_start
    while True:
        res = run_mlmc(solver, eps, max_level=L, pilot=pilot, seed=seed, qoi=qoi, cost=cost, state=state, log=log)
        state = res["state"]
        means = [p["mean_Y"] for p in res["levels"]]
        var = [p["var_Y"] for p in res["levels"]]
        s = [level_cost_model(solver.cfg, l) for l in range(L + 1)]
        alpha, beta, gamma_d = henry.mlmc_rates(means, var, s, first_level=1)
        alpha_used = max(alpha, alpha_min)
        bias_last, ok_last = henry.mlmc_bias_test(means, alpha_used, eps)
        bias_fit, ok_fit, _ = henry.mlmc_bias_test_fit(means, eps, first_level=1, alpha_min=alpha_min)
        bias_est, ok = (bias_fit, ok_fit) if rule == "fit" else (bias_last, ok_last)
        if log:
            log("L=%d alpha=%.3f beta=%.3f gamma_d=%.3f bias=%.3g ok=%s" % (L, alpha, beta, gamma_d, bias_est, ok))
        res.update({"L": L, "alpha": alpha, "alpha_used": alpha_used, "beta": beta, "gamma_d": gamma_d,
                    "bias_est": bias_est, "bias_ok": ok, "bias_rule": rule, "bias_est_last": bias_last,
                    "bias_est_fit": bias_fit, "wall_seconds": time.perf_counter() - t0,
                    "cell_steps": sum(st.cell_steps for st in state)})
        if ok or L >= L_max:
            # Eq. (MSE) asks variance + bias^2 <= eps^2; the split into halves
            # is a choice.  When the bias test still fails at L_max, the
            # variance gets the rest of the budget, eps^2 - bias^2, if any.
            if not ok and bias_est < eps:
                frac = (eps * eps - bias_est * bias_est) / (eps * eps)
                if res["variance"] > frac * eps * eps:
                    res2 = run_mlmc(solver, eps, max_level=L, pilot=pilot, seed=seed, qoi=qoi, cost=cost,
                                    state=state, log=log, var_fraction=frac)
                    keep = {k: res[k] for k in res if k not in res2}
                    res = dict(res2, **keep)
            res["rmse_bound"] = math.sqrt(res["variance"] + res["bias_est"] ** 2)
            res["rmse_ok"] = res["rmse_bound"] <= eps
            res["wall_seconds"] = time.perf_counter() - t0
            res["cell_steps"] = sum(st.cell_steps for st in res["state"])
            return res
        L += 1
