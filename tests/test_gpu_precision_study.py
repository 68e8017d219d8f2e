"""Reduced-precision study on fixed states (GPU against the FP64 oracle).

States are snapshots of FP64 oracle trajectories: the messages read at a random
tick t and the syndrome before that tick's feedback.  For every reduced storage
precision the test reports
  * the message error of one BP sweep against FP64 (max and RMS of
    |m - m64| / max(1, |m64|)), and
  * the decision-flip rate: the fraction of active checks whose feedback
    decision (Evidence pass, and the set of argmax qubits when it passes)
    differs from the FP64 decision,
and checks them against bounds from the storage formats.  Set LIM_STUDY_OUT to
a file path to keep the numbers as JSON.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    ("toric2d_16", lambda: I.toric2d(16), 0.05, "f16", 0.0),
    ("toric2d_16", lambda: I.toric2d(16), 0.05, "bf16", 0.0),
    ("toric2d_16", lambda: I.toric2d(16), 0.05, "i16", 2 ** -6),
    ("toric3d_point_6", lambda: I.toric3d_point(6), 0.02, "f16", 0.0),
    ("toric3d_point_6", lambda: I.toric3d_point(6), 0.02, "bf16", 0.0),
    ("toric3d_membrane_4", lambda: I.toric3d_membrane(4), 0.05, "i16", 2 ** -6),
    ("bb_12_6", lambda: I.bb_code(12, 6), 0.04, "i8", 0.25),
]
# Bounds: one store rounding has relative error 2^-11 (f16), 2^-8 (bf16); the
# integer grids have absolute error Delta/2 per input (inputs are rounded too,
# and a qubit sum adds up to DV of them).
MSG_BOUND = {"f16": 4e-3, "bf16": 3e-2, "i16": 0.1, "i8": 2.0}
FLIP_BOUND = {"f16": 0.05, "bf16": 0.15, "i16": 0.05, "i8": 0.25}

_results = {}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_38139_b300 import build, lim
    build.build()
    return lim


def _snapshots(code, q, p, nstates, rng):
    oc = O.OracleCode.from_code(code)
    out = []
    shot = 0
    while len(out) < nstates and shot < 20 * nstates:
        t = int(rng.integers(3, 40))
        prm = O.params(precision="f64", q=q, tick_budget=t)
        r = O.run_shot(oc, prm, p, 123, 7, shot, trace_ticks=t)
        shot += 1
        if r["ticks"] < t:  # cleared earlier: no state at tick t
            continue
        s_before = r["trace"]["s_hist"][t - 1]
        if not s_before.any():
            continue
        out.append((r["trace"]["cv"].copy(), r["trace"]["vc"].copy(), s_before.copy()))
    return out


def _quantize(x, prec, delta, clamp_q):
    if prec == "f16":
        return torch.from_numpy(x).half()
    if prec == "bf16":
        return torch.from_numpy(x).bfloat16()
    q = np.where(x < 0, -np.floor(-x / delta + 0.5), np.floor(x / delta + 0.5))
    q = np.clip(q, -clamp_q, clamp_q)
    return torch.from_numpy(q.astype(np.int16 if prec == "i16" else np.int8))


def _decisions(code, L, s, theta_of_d):
    out = []
    for c in np.nonzero(s)[0]:
        nb = code.hx_col[code.hx_ptr[c]:code.hx_ptr[c + 1]]
        vals = L[nb]
        best = vals.max()
        ev = bool(best >= theta_of_d(len(nb)))
        out.append((ev, tuple(nb[vals == best]) if ev else ()))
    return out


@pytest.mark.parametrize("name,maker,p,prec,delta", CASES)
def test_precision_study(L, name, maker, p, prec, delta):
    code = maker()
    q = 0.125 if "membrane" in name else 0.05
    ctx = L.Context(0)
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, quant_scale=delta or 2 ** -6, q=q, tau=0, dt_tick=0)
    rng = np.random.default_rng(hash(name) % 2 ** 31)
    snaps = _snapshots(code, q, p, 24, rng)
    assert len(snaps) >= 8
    oc = O.OracleCode.from_code(code)
    op64 = O.params(precision="f64", q=q, tau=0, dt_tick=0)
    is_int = prec in ("i16", "i8")
    qmax = 32767 if prec == "i16" else 127
    clamp_q = min(qmax, round(1000.0 / delta)) if is_int else 0
    scale = delta if is_int else 1.0
    errs = []
    errs_in = []
    flips = 0
    checks = 0
    for cv, vc, s in snaps:
        rc, rv = O.bp_sweeps(oc, op64, s, cv, vc, 1)
        cvq = _quantize(cv, prec, delta, clamp_q).unsqueeze(0).cuda()
        vcq = _quantize(vc, prec, delta, clamp_q).unsqueeze(0).cuda()
        sd = torch.from_numpy(s.astype(np.uint8)).unsqueeze(0).cuda()
        gc, gv = L.bp_sweeps(lc, prm, sd, cvq, vcq, 1)
        gc = gc.double().cpu().numpy()[0] * scale
        gv = gv.double().cpu().numpy()[0] * scale
        # The integer grids saturate at Qmax * Delta (512 LLR for int16 at 2^-6,
        # 31.75 for int8 at 2^-2), below CLAMP = 1000.  The quantisation error
        # alone is measured against an FP64 sweep with that saturation level.
        if is_int:
            sat = clamp_q * delta
            opsat = O.params(precision="f64", q=q, tau=0, dt_tick=0, clamp=sat)
            rcs, rvs = O.bp_sweeps(oc, opsat, s, np.clip(cv, -sat, sat), np.clip(vc, -sat, sat), 1)
        else:
            rcs, rvs = rc, rv
        for got, ref, refs in ((gc, rc, rcs), (gv, rv, rvs)):
            errs.append(np.abs(got - ref) / np.maximum(1.0, np.abs(ref)))
            errs_in.append(np.abs(got - refs) / np.maximum(1.0, np.abs(refs)))
        L64 = O.readout(oc, op64, cv)
        Lp = L.readout(lc, prm, cvq).double().cpu().numpy()[0]
        if is_int:
            th = lambda d: math.ceil(-math.log(d - 1) / delta) if d > 1 else math.inf
        else:
            th = lambda d: float(np.float32(-math.log(d - 1))) if d > 1 else math.inf
        d64 = _decisions(code, L64, s, lambda d: -math.log(d - 1) if d > 1 else math.inf)
        dp = _decisions(code, Lp, s, th)
        flips += sum(a != b for a, b in zip(d64, dp))
        checks += len(d64)
    e = np.concatenate(errs)
    ei = np.concatenate(errs_in)
    res = {"code": name, "precision": prec, "delta": delta, "states": len(snaps),
           "msg_err_max": float(e.max()), "msg_err_rms": float(np.sqrt(np.mean(e ** 2))),
           "msg_err_in_range_max": float(ei.max()),
           "saturation_llr": float(clamp_q * delta) if is_int else None,
           "active_checks": checks, "decision_flip_rate": flips / max(1, checks)}
    _results[f"{name}/{prec}"] = res
    print(json.dumps(res))
    out = os.environ.get("LIM_STUDY_OUT")
    if out:
        json.dump(_results, open(out, "w"), indent=1)
    assert res["msg_err_in_range_max"] <= MSG_BOUND[prec], res
    assert res["decision_flip_rate"] <= FLIP_BOUND[prec], res
