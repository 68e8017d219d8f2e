"""Logical-error-rate and clearing-time studies on the CUDA library.

The paper's numerics (Sec. S4) estimate, per code size d and physical error
rate p, the logical error rate with adaptive Monte Carlo (500,000 shots or 100
logical failures, whichever comes first), the clearing time t_clr of the shots
whose syndrome clears (Fig. 2b, Fig. 3-4 insets, histograms of Fig. S2), and
fit E[t_clr] against the code size (Sec. "Local inference on the rep code":
O(log d); 2D/3D toric: a (log d)^2 + b; membrane and BB: a log d + b and
a (log sqrt(2 l m))^2 + b).  This module runs those studies for the named
workloads of ``inputs.WORKLOADS`` and writes one JSON record per point.

Usage::

    python -m paper_2609_38139_b300.study --workload toric2d_fine_dt \\
        --max-shots 20000 --max-failures 100 --out ler.jsonl
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from typing import Dict, List, Sequence

import numpy as np

from . import dist as D
from . import inputs as I
from . import lim


def workload_params(w: dict, precision: str = "f32", rule: str = "", feedback: str = "") -> lim.Params:
    rule = rule or w.get("rule", "minsum")
    qs = lim.default_quant_scale(precision, w["q"])
    return lim.params(rule=rule, feedback=feedback or w.get("feedback", "check_move"),
                      precision=precision,
                      quant_scale=qs, q=w["q"], clamp=w["clamp"], tau=w["tau"],
                      dt_tick=w["dt_tick"], sweeps_per_tick=w["K"], tick_budget=1,
                      tie_rel=lim.default_tie_rel(precision, rule))


def point_stats(t: np.void, dt_tick: float) -> Dict[str, float]:
    """Per-point estimates from an integer tally: LER with its binomial standard
    error, and the mean / standard deviation of t_clr (in decoder time units,
    ticks x dt) over the shots that cleared."""
    n = int(t["shots"])
    f = int(t["failures"])
    c = n - int(t["nonconverged"])
    ler = f / n if n else float("nan")
    se = math.sqrt(max(ler * (1 - ler), 1.0 / max(n, 1)) / n) if n else float("nan")
    mean = t["sum_t"] / c if c else float("nan")
    var = t["sum_t2"] / c - mean * mean if c else float("nan")
    return {"shots": n, "failures": f, "nonconverged": int(t["nonconverged"]), "cleared": c,
            "ler": ler, "ler_se": se, "t_clr_mean": mean * dt_tick,
            "t_clr_std": math.sqrt(max(var, 0.0)) * dt_tick, "ticks": int(t["ticks"]),
            "moves": int(t["moves"]), "hist_log2_ticks": [int(x) for x in t["hist"]]}


def run_study(ctx: lim.Context, name: str, precision: str = "f32", rule: str = "",
              max_shots: int = 20000, max_failures: int = 100, batch_shots: int = 1000,
              seed: int = 0, sizes: Sequence = (), ps: Sequence[float] = (),
              feedback: str = "") -> List[dict]:
    """Adaptive Monte Carlo over every (size, p) point of workload ``name``: all
    unfinished points run together, ``batch_shots`` fresh shot ids per point per
    launch, until each has ``max_shots`` shots or ``max_failures`` failures."""
    w = I.WORKLOADS[name]
    rule = rule or w.get("rule", "minsum")
    feedback = feedback or w.get("feedback", "check_move")
    prm = workload_params(w, precision, rule, feedback)
    codes, pts, meta = {}, [], []
    for fam, size, p, pid in I.workload_points(name):
        if sizes and size not in sizes:
            continue
        if ps and not any(abs(p - x) < 1e-9 for x in ps):
            continue
        if size not in codes:
            codes[size] = ctx.from_inputs(I.make_code(fam, size))
        T = I.tick_budget(w["budget"], size, w["dt_tick"])
        pts.append((codes[size], p, batch_shots, 0, pid, T))
        meta.append((fam, size, p, pid, T))
    t0 = time.perf_counter()
    tot = D.run_until(D.gpu_runner(ctx, prm, seed), pts, batch_shots, max_shots, max_failures)
    wall = time.perf_counter() - t0
    rows = []
    for (fam, size, p, pid, T), t in zip(meta, tot):
        c = codes[size]
        r = {"workload": name, "family": fam, "size": size, "n": c.n, "k": c.k, "p": p,
             "point_id": pid, "tick_budget": T, "precision": precision, "rule": rule,
             "feedback": feedback,
             "tau": w["tau"], "dt_tick": w["dt_tick"], "seed": seed}
        r.update(point_stats(t, w["dt_tick"]))
        rows.append(r)
    ticks = sum(r["ticks"] for r in rows)
    for r in rows:
        r["study_wall_s"] = wall
        r["study_shot_ticks_per_s"] = ticks / wall if wall > 0 else float("nan")
    return rows


def fit_clear_time(sizes: Sequence[float], means: Sequence[float], form: str = "log2"):
    """Least-squares fit of mean clearing times against code size ``d``:
    ``log``: a log d + b; ``log2``: a (log d)^2 + b.  Returns (a, b, rms residual)."""
    x = np.log(np.asarray(sizes, dtype=np.float64))
    if form == "log2":
        x = x * x
    elif form != "log":
        raise ValueError(form)
    y = np.asarray(means, dtype=np.float64)
    A = np.stack([x, np.ones_like(x)], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - (a * x + b)
    return float(a), float(b), float(np.sqrt(np.mean(res * res)))


def fit_slope(sizes: Sequence[float], lers: Sequence[float], p: float, p_th: float):
    """Fig. S1(b): the slope alpha(p) of p_L = A(p) (p / p_th)^(alpha(p) d) at one p,
    from a least-squares line through log p_L against the distance d.  Returns
    (alpha, log A, rms residual of log p_L); points with p_L = 0 are left out."""
    d = np.asarray([x for x, y in zip(sizes, lers) if y > 0], dtype=np.float64)
    y = np.log(np.asarray([y for y in lers if y > 0], dtype=np.float64))
    if len(d) < 2:
        raise ValueError("need two sizes with failures")
    A = np.stack([d, np.ones_like(d)], axis=1)
    (slope, logA), *_ = np.linalg.lstsq(A, y, rcond=None)
    res = y - (slope * d + logA)
    return float(slope / math.log(p / p_th)), float(logA), float(np.sqrt(np.mean(res * res)))


def crossings(rows: List[dict]) -> List[dict]:
    """Where the LER curves of consecutive sizes cross: for each pair of sizes,
    the p at which log LER(small) - log LER(large) changes sign (linear
    interpolation between grid points).  A threshold estimate."""
    by = {}
    for r in rows:
        by.setdefault(r["size"], []).append(r)
    keys = sorted(by, key=lambda s: by[s][0]["n"])
    out = []
    for a, b in zip(keys, keys[1:]):
        A = {round(r["p"], 9): r for r in by[a]}
        B = {round(r["p"], 9): r for r in by[b]}
        grid = sorted(set(A) & set(B))
        prev = None
        for p in grid:
            la, lb = A[p]["ler"], B[p]["ler"]
            if la <= 0 or lb <= 0:
                prev = None
                continue
            g = math.log(la) - math.log(lb)
            if prev is not None and (prev[1] > 0) != (g > 0):
                p0, g0 = prev
                out.append({"sizes": [a, b], "p_cross": p0 + (p - p0) * g0 / (g0 - g)})
            prev = (p, g)
    return out


def summarize(rows: List[dict], p_th: float = 0.0) -> dict:
    """Crossings of the LER curves and, below the threshold (p_th, else the mean
    crossing), the slope fits alpha(p) for codes with a scalar size."""
    summ = {"crossings": crossings(rows)}
    if not p_th and summ["crossings"]:
        p_th = float(np.mean([c["p_cross"] for c in summ["crossings"]]))
    if p_th > 0 and all(not isinstance(r["size"], (list, tuple)) for r in rows):
        summ["p_th_for_slopes"] = p_th
        summ["slopes"] = []
        for p in sorted({r["p"] for r in rows}):
            rr = [r for r in rows if r["p"] == p]
            # alpha divides by log(p / p_th): only points clearly below the threshold
            if p < 0.99 * p_th and sum(r["failures"] > 0 for r in rr) >= 2:
                al, logA, res = fit_slope([r["size"] for r in rr], [r["ler"] for r in rr], p, p_th)
                summ["slopes"].append({"p": p, "alpha": al, "log_A": logA, "rms": res})
    return summ


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", required=True, choices=sorted(I.WORKLOADS))
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--rule", default="", help="minsum | sumproduct (default: the workload's)")
    ap.add_argument("--feedback", default="",
                    help="check_move | check_move_multi | bit_discrete (default: the workload's)")
    ap.add_argument("--max-shots", type=int, default=20000)
    ap.add_argument("--max-failures", type=int, default=100)
    ap.add_argument("--batch-shots", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--sizes", default="", help="comma-separated subset of sizes")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--p-th", type=float, default=0.0,
                    help="threshold for the slope fits (default: mean of the crossings)")
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    ctx = lim.Context(a.device)
    sizes = []
    if a.sizes:
        allowed = {str(s): s for s in I.WORKLOADS[a.workload]["sizes"]}
        sizes = [allowed[s] for s in a.sizes.split(",")]
    rows = run_study(ctx, a.workload, a.precision, a.rule, a.max_shots, a.max_failures,
                     a.batch_shots, a.seed, sizes, feedback=a.feedback)
    out = open(a.out, "w") if a.out else sys.stdout
    for r in rows:
        out.write(json.dumps(r) + "\n")
    summ = dict(summarize(rows, a.p_th), workload=a.workload)
    out.write(json.dumps(summ) + "\n")
    if a.out:
        out.close()
    for r in rows:
        print(f"{r['family']:16s} {str(r['size']):8s} p={r['p']:.4f} shots={r['shots']:7d} "
              f"LER={r['ler']:.4g}+-{r['ler_se']:.2g} t_clr={r['t_clr_mean']:.4g}", file=sys.stderr)
    print(json.dumps(summ), file=sys.stderr)
    return 0


if __name__ == "__main__":
    sys.exit(main())
