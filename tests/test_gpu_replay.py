"""Trajectory replay through lim_trace: the CUDA path re-runs a trajectory of the
oracle under the oracle's own moves, so that its messages and beliefs can be
compared tick by tick under identical decisions (Algorithm 1; Eq. 1-3).

Bars:
  * replaying an FP64 oracle trajectory in binary32: every read-out L_v of every
    tick within |L32 - L64| <= 1e-5 max(1, |L64|) -- relative 1e-5 for
    |L64| >= 1 LLR unit and absolute 1e-5 below it (a pure relative bar is not
    defined where a belief crosses zero);
  * replaying in the kernel's own storage precision: every belief bit-exact
    against the oracle's emulation of that precision (integer steps exactly);
  * in both: e, s, ticks, moves and the termination exactly as the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import inputs as I

from parity import oracle_params

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_38139_b300 import build, lim
    build.build()
    return lim


@pytest.fixture(scope="module")
def ctx(L):
    return L.Context(0)


def _replay(L, ctx, code, prm, op, p, seed, point, shot, T):
    """Oracle trajectory (params op) and its replay on the GPU (params prm)."""
    oc = O.OracleCode.from_code(code)
    r = O.run_shot(oc, op, p, seed, point, shot, trace_ticks=T, move_cap=1 << 17, want_l=True)
    assert r["trace"]["n_moves"] <= 1 << 17
    moves = r["trace"]["moves"]
    lc = ctx.from_inputs(code)
    eh, sh, rec, lh = L.trace(ctx, lc, prm, p, seed, point, shot, T, forced_moves=moves, want_l=True)
    tend = int(r["ticks"])
    assert rec["ticks"] == tend and rec["t_clr"] == r["t_clr"] and rec["converged"] == r["converged"]
    assert rec["moves"] == r["moves"] and rec["failed"] == r["failed"]
    assert np.array_equal(L.bits_to_bytes(eh, code.n), r["trace"]["e_hist"])
    assert np.array_equal(L.bits_to_bytes(sh, code.m), r["trace"]["s_hist"])
    return tend, r["trace"]["l_hist"][1:tend + 1], lh[1:tend + 1].astype(np.float64)


@pytest.mark.parametrize("maker,p,T", [(lambda: I.toric2d(16), 0.08, 640),
                                       (lambda: I.toric3d_point(6), 0.03, 240)])
@pytest.mark.parametrize("rule", ["minsum", "sumproduct"])
def test_fp32_replay_of_fp64_trajectories(L, ctx, maker, p, T, rule):
    """FP32 messages against FP64 along whole trajectories (the FP32 bar of the
    precision policy), decisions forced to the FP64 oracle's."""
    code = maker()
    prm = L.params(precision="f32", rule=rule, tick_budget=T)
    op = oracle_params(prm, precision="f64")
    long_runs = 0
    worst = 0.0
    for shot in range(10):
        tend, L64, L32 = _replay(L, ctx, code, prm, op, p, 0, 4, shot, T)
        err = np.abs(L32 - L64) / np.maximum(1.0, np.abs(L64))
        worst = max(worst, float(err.max()) if err.size else 0.0)
        assert np.all(err <= 1e-5), (shot, float(err.max()))
        long_runs += tend >= 20
    assert long_runs >= 3, "too few trajectories of 20 ticks or more"
    print(f"{code.name} {rule}: worst |L32-L64|/max(1,|L64|) = {worst:.3g}")


@pytest.mark.parametrize("maker,prec,qs,q,fb,gauge,dt,variant", [
    (lambda: I.toric2d(8), "f16", 2 ** -6, 0.05, "check_move", 0, 0.1, "cta"),
    (lambda: I.toric2d(8), "bf16", 2 ** -6, 0.05, "check_move", 0, 0.1, "warp"),
    (lambda: I.toric3d_membrane(3), "i16", 2 ** -6, 0.125, "check_move", 0, 0.1, "warp"),
    (lambda: I.bb_code(6, 6), "i8", 0.25, 0.05, "check_move_multi", 0, 0.1, "cta"),
    (lambda: I.toric2d(6), "f32", 2 ** -6, 0.05, "check_move", 1, 0.1, "cta"),
    (lambda: I.toric2d(6), "f32", 2 ** -6, 0.05, "check_move", 0, 0.03, "cta"),
    (lambda: I.toric3d_point(3), "i16", 2 ** -6, 0.05, "check_move", 1, 0.05, "warp"),
])
def test_replay_in_own_precision_is_bit_exact(L, ctx, maker, prec, qs, q, fb, gauge, dt, variant):
    """Replay of the oracle's own trajectory in the same storage precision: every
    belief of every tick equals the oracle's (binary32 emulation or integer
    steps), including relaxed ticks (alpha < 1), the gauge switch on moves and
    the multi-qubit move."""
    code = maker()
    prm = L.params(precision=prec, quant_scale=qs, q=q, feedback=fb, gauge_on_move=gauge, tau=0.1,
                   dt_tick=dt, tick_budget=150, variant=variant)
    op = oracle_params(prm)
    for shot in range(6):
        tend, Lo, Lg = _replay(L, ctx, code, prm, op, 0.07, 3, 2, shot, 150)
        assert np.array_equal(Lg, Lo), (shot, np.argwhere(Lg != Lo)[:4])


def test_replay_without_moves_and_with_a_foreign_list(L, ctx):
    """An empty list freezes e (no move ever happens); a list from another shot's
    trajectory is applied as given (the flips are the list's, the syndrome
    follows H_X)."""
    code = I.toric2d(6)
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", tick_budget=30)
    eh, sh, rec = L.trace(ctx, lc, prm, 0.08, 1, 0, 3, 30, forced_moves=np.zeros((0, 3)))
    assert rec["moves"] == 0 and (rec["converged"] == 0 or rec["t_clr"] == 0)
    assert all(np.array_equal(eh[t], eh[0]) for t in range(31))
    oc = O.OracleCode.from_code(code)
    r = O.run_shot(oc, oracle_params(prm), 0.08, 1, 0, 9, trace_ticks=30, move_cap=4096)
    mv = r["trace"]["moves"]
    eh, sh, rec = L.trace(ctx, lc, prm, 0.08, 1, 0, 3, 30, forced_moves=mv)
    e0 = L.bits_to_bytes(eh[0], code.n).astype(np.int64)
    hx = code.hx_dense().astype(np.int64)
    for t in range(1, int(rec["ticks"]) + 1):
        want = e0.copy()
        for tk, _, v in mv:
            if tk <= t:
                want[v] ^= 1
        got = L.bits_to_bytes(eh[t], code.n).astype(np.int64)
        assert np.array_equal(got, want), t
        assert np.array_equal(L.bits_to_bytes(sh[t], code.m), hx @ got % 2), t
