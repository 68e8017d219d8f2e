"""Helpers shared by the GPU parity tests: run the same keyed shots through the
CUDA library and through the oracle, in the same precision."""
import os

import numpy as np

import oracle as O

THREADS = max(1, min(16, os.cpu_count() or 1))


def oracle_params(prm, precision=None):
    """Oracle parameters equal to a library ``Params``."""
    from paper_2609_38139_b300 import lim
    rule = {v: k for k, v in lim.RULE.items()}[prm.rule]
    fb = {v: k for k, v in lim.FEEDBACK.items()}[prm.feedback]
    prec = precision or lim.prec_name(prm)
    return O.params(rule=rule, feedback=fb, precision=prec, quant_scale=prm.quant_scale, q=prm.q,
                    clamp=prm.clamp, tau=prm.tau, dt_tick=prm.dt_tick,
                    sweeps_per_tick=prm.sweeps_per_tick, ring_prob=prm.ring_prob,
                    tick_budget=prm.tick_budget, gauge_on_move=prm.gauge_on_move,
                    tie_rel=prm.tie_rel)


def oracle_point(code, prm, p, seed, point_id, shot0, nshots, tick_budget=0, precision=None):
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm, precision)
    if tick_budget:
        op.tick_budget = tick_budget
    return O.run_shots(oc, op, p, seed, point_id, shot0, nshots, threads=THREADS)


def oracle_finals(code, prm, p, seed, point_id, shots, tick_budget=0):
    """Final residual bits of selected shots, packed like the library's e_final rows."""
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    if tick_budget:
        op.tick_budget = tick_budget
    rows = []
    for sh in shots:
        r = O.run_shot(oc, op, p, seed, point_id, int(sh), trace_ticks=0)
        e = r["trace"]["e_hist"][0]
        rows.append(e)
    return np.array(rows)


def final_state(code, prm, p, seed, point_id, shot, tick_budget=0):
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    if tick_budget:
        op.tick_budget = tick_budget
    T = op.tick_budget
    r = O.run_shot(oc, op, p, seed, point_id, int(shot), trace_ticks=T)
    return r["trace"]["e_hist"][T], r


def oracle_shots_with_finals(code, op, p, seed, point_id, shot0, nshots):
    """Records (RECORD_DTYPE) and final errors (bytes [nshots, n]) of the oracle
    for shots shot0 .. shot0+nshots-1, over a thread pool."""
    from concurrent.futures import ThreadPoolExecutor
    oc = O.OracleCode.from_code(code)
    recs = np.zeros(nshots, dtype=O.RECORD_DTYPE)
    fins = np.zeros((nshots, code.n), dtype=np.uint8)

    def one(i):
        r = O.run_shot(oc, op, p, seed, point_id, shot0 + i, trace_ticks=0)
        for f in O.RECORD_DTYPE.names:
            recs[i][f] = r[f]
        fins[i] = r["trace"]["e_final"]

    with ThreadPoolExecutor(max_workers=THREADS) as ex:
        list(ex.map(one, range(nshots)))
    return recs, fins


def compare_records(gpu, ora, what=""):
    for f in ("t_clr", "converged", "failed", "moves", "ticks", "sweeps"):
        bad = np.nonzero(gpu[f] != ora[f])[0]
        assert len(bad) == 0, f"{what}: field {f} differs at shots {bad[:10]}: gpu {gpu[f][bad[:5]]} oracle {ora[f][bad[:5]]}"


def paired_ok(fail_a, fail_b):
    """McNemar-style 3-sigma agreement of two failure vectors on the same shots."""
    b = int(np.sum((fail_a == 1) & (fail_b == 0)))
    c = int(np.sum((fail_a == 0) & (fail_b == 1)))
    return abs(b - c) <= 3.0 * np.sqrt(b + c) + 1.0, (b, c)
