"""The one-shot-per-lane kernel (LIM_VARIANT_LANE) against the oracle and against
the team kernels, shot by shot: records, tallies and final residuals bit-exact,
for every degree pair it is compiled for, every storage precision, both check
rules, several sweeps per tick, mixed codes in one launch, given initial errors,
and ticks with more ringing checks than its registers hold (the ordered slow
path)."""
import math

import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

from parity import compare_records, oracle_params, oracle_point, oracle_shots_with_finals, paired_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PRIOR_STEP = abs(math.log(0.05 / 0.95))


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


CASES = [
    # id, code, precision, Delta, q, rule, p, budget, ring_prob, K, tau, shots
    ("bb66-i8", lambda: I.bb_code(6, 6), "i8", PRIOR_STEP, 0.05, "minsum", 0.05, 300, -1.0, 1, 0.1, 300),
    ("bb126-i8-q4", lambda: I.bb_code(12, 6), "i8", 0.25, 0.05, "minsum", 0.08, 300, -1.0, 1, 0.1, 300),
    ("bb153-i16", lambda: I.bb_code(15, 3), "i16", 2 ** -6, 0.05, "minsum", 0.06, 300, -1.0, 1, 0.1, 300),
    ("toric2d8-f32", lambda: I.toric2d(8), "f32", 2 ** -6, 0.05, "minsum", 0.05, 32, -1.0, 1, 0.1, 1000),
    ("toric2d5-f16", lambda: I.toric2d(5), "f16", 2 ** -6, 0.05, "minsum", 0.08, 100, -1.0, 1, 0.1, 300),
    ("point3-bf16", lambda: I.toric3d_point(3), "bf16", 2 ** -6, 0.05, "minsum", 0.05, 100, -1.0, 1, 0.1, 300),
    ("membrane3-i16", lambda: I.toric3d_membrane(3), "i16", 2 ** -6, 0.125, "minsum", 0.1, 300, -1.0, 1, 0.1, 300),
    ("ring12-f32", lambda: I.rep_code(12, periodic=True), "f32", 2 ** -6, 0.05, "minsum", 0.2, 60, -1.0, 1, 0.1, 300),
    ("toric2d6-sp", lambda: I.toric2d(6), "f32", 2 ** -6, 0.05, "sumproduct", 0.07, 100, -1.0, 1, 0.1, 300),
    ("bb126-rings", lambda: I.bb_code(12, 6), "i8", PRIOR_STEP, 0.05, "minsum", 0.1, 200, 1.0, 1, 0.1, 200),
    ("toric2d8-rings", lambda: I.toric2d(8), "f32", 2 ** -6, 0.05, "minsum", 0.15, 64, 1.0, 1, 0.1, 200),
    ("toric2d6-K2", lambda: I.toric2d(6), "f16", 2 ** -6, 0.05, "minsum", 0.07, 80, -1.0, 2, 0.05, 200),
]


@pytest.mark.parametrize("cid,maker,prec,qs,q,rule,p,T,ring,K,tau,shots", CASES, ids=[c[0] for c in CASES])
def test_lane_kernel_against_oracle(L, ctx, cid, maker, prec, qs, q, rule, p, T, ring, K, tau, shots):
    code = maker()
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, quant_scale=qs, q=q, rule=rule, tick_budget=T, ring_prob=ring,
                   sweeps_per_tick=K, tau=tau, variant="lane")
    shape, _ = L.plan_describe(ctx, [(lc, p, shots, 0, 3)], prm)
    assert shape["variant"] == "lane"
    tal, rec, fin = L.run_batch(ctx, [(lc, p, shots, 0, 3)], prm, 21, e_final=True)
    if rule == "sumproduct":
        # the box-plus corrections use the hardware exp/log, so sum-product is
        # compared bit for bit with the team kernel (the same arithmetic) and
        # with the oracle through the logical error rate
        prm_c = L.params(precision=prec, quant_scale=qs, q=q, rule=rule, tick_budget=T, ring_prob=ring,
                         sweeps_per_tick=K, tau=tau, variant="cta")
        tal_c, rec_c, fin_c = L.run_batch(ctx, [(lc, p, shots, 0, 3)], prm_c, 21, e_final=True)
        assert np.array_equal(rec, rec_c) and np.array_equal(tal, tal_c) and np.array_equal(fin, fin_c)
        ora = oracle_point(code, prm, p, 21, 3, 0, shots, precision="f64")
        ok, bc = paired_ok(rec["failed"], ora["failed"])
        assert ok, bc
        return
    op = oracle_params(prm)
    ora, fins = oracle_shots_with_finals(code, op, p, 21, 3, 0, shots)
    compare_records(rec, ora, cid)
    assert np.array_equal(L.bits_to_bytes(fin, code.n), fins)
    assert tal[0]["shots"] == shots and tal[0]["errors"] == 0
    assert tal[0]["failures"] == int(ora["failed"].sum())
    assert tal[0]["sweeps"] == int(ora["sweeps"].sum())
    assert tal[0]["msg_updates"] == int(ora["sweeps"].sum()) * 2 * code.E
    conv = ora["converged"] == 1
    assert tal[0]["sum_t"] == int(ora["t_clr"][conv].sum())
    if ring == 1.0:
        # every active check rings: the first tick of a shot with more than eight
        # defects has more candidates than the registers hold and takes the
        # ordered passes over the ring set; the trajectories above went through it
        _, s0 = L.sample_noise(lc, p, 21, 3, 0, shots)
        defects = L.bits_to_bytes(s0.cpu().numpy(), code.m).sum(axis=1)
        assert int((defects > 8).sum()) > shots // 4
        assert int(ora["moves"].sum()) > 4 * shots


def test_lane_mixed_codes_equal_team_kernels(L, ctx):
    """The bivariate-bicycle mix of the benchmark (three codes, several rates and
    budgets, uneven termination) in one launch: the lane kernel's records,
    tallies and residuals equal those of the block- and warp-per-shot kernels."""
    codes = [I.bb_code(12, 6), I.bb_code(15, 3), I.bb_code(6, 6)]
    lcs = [ctx.from_inputs(c) for c in codes]
    pts = []
    for i, lc in enumerate(lcs):
        for j, p in enumerate((0.02, 0.05, 0.08)):
            pts.append((lc, p, 97 + 13 * j, 50 * i, 10 * i + j, 100 + 150 * j))
    prm = dict(precision="i8", quant_scale=PRIOR_STEP, tick_budget=1)
    out = {}
    for variant in ("lane", "warp", "cta"):
        out[variant] = L.run_batch(ctx, pts, L.params(variant=variant, **prm), 8, e_final=True)
    for variant in ("warp", "cta"):
        for a, b in zip(out["lane"], out[variant]):
            assert np.array_equal(a, b), variant
    row = 0
    for (lc, p, n, s0, pid, T), code in zip(pts, [c for c in codes for _ in range(3)]):
        ora = oracle_point(code, L.params(**prm), p, 8, pid, s0, n, tick_budget=T)
        compare_records(out["lane"][1][row:row + n], ora, f"{code.name} p={p}")
        row += n


def test_lane_given_errors_and_edge_cases(L, ctx):
    """lim_run_batch_from through the lane kernel (errors in, residuals out) equals
    the team kernel; an empty point, p = 0 (every shot clear at the start) and a
    zero budget (every shot with defects fails at once) are handled."""
    code = I.bb_code(6, 6)
    lc = ctx.from_inputs(code)
    pts = [(lc, 0.0, 64, 0, 0)]
    prm_l = L.params(precision="f32", tick_budget=200, variant="lane")
    prm_c = L.params(precision="f32", tick_budget=200, variant="cta")
    e, _ = L.sample_noise(lc, 0.06, 5, 9, 0, 64)
    b_l = L.Batch(ctx, pts, prm_l, records=True, e_final=True)
    b_c = L.Batch(ctx, pts, prm_c, records=True, e_final=True)
    b_l.run(3, e0=e.contiguous().view(-1))
    b_c.run(3, e0=e.contiguous().view(-1))
    torch.cuda.synchronize()
    assert np.array_equal(b_l.records(), b_c.records())
    assert np.array_equal(b_l.finals(), b_c.finals())
    assert b_l.records()["moves"].sum() > 0
    tal, rec = L.run_batch(ctx, [(lc, 0.0, 40, 0, 0), (lc, 0.05, 0, 0, 1), (lc, 0.1, 30, 0, 2)],
                           L.params(precision="f32", tick_budget=50, variant="lane"), 1)
    assert np.all(rec["t_clr"][:40] == 0) and np.all(rec["failed"][:40] == 0)
    assert tal[1]["shots"] == 0
    ora = oracle_point(code, L.params(precision="f32", tick_budget=50), 0.1, 1, 2, 0, 30)
    compare_records(rec[40:], ora, "budget 50")
    prm0 = L.params(precision="f32", tick_budget=0, variant="lane")
    tal, rec = L.run_batch(ctx, [(lc, 0.1, 30, 0, 2)], prm0, 1)
    ora = oracle_point(code, prm0, 0.1, 1, 2, 0, 30)
    compare_records(rec, ora, "zero budget")
    assert np.all(rec["ticks"] == 0)


def test_auto_picks_lane_for_small_codes_only(L, ctx):
    lc = ctx.from_inputs(I.bb_code(12, 6))
    bb = [(lc, 0.05, 200000, 0, 0)]
    # a batch with few shots per lane keeps one warp per shot
    assert L.plan_describe(ctx, [(lc, 0.05, 1000, 0, 0)],
                           L.params(precision="i8", quant_scale=PRIOR_STEP))[0]["variant"] == "warp"
    big = [(ctx.from_inputs(I.toric2d(64)), 0.05, 10, 0, 0)]
    assert L.plan_describe(ctx, bb, L.params(precision="i8", quant_scale=PRIOR_STEP))[0]["variant"] == "lane"
    assert L.plan_describe(ctx, big, L.params(precision="f32"))[0]["variant"] == "cta"
    # rules the lane kernel does not cover fall back to the team kernels
    for kw in (dict(feedback="check_move_multi"), dict(gauge_on_move=1), dict(dt_tick=0.05),
               dict(feedback="bit_discrete")):
        assert L.plan_describe(ctx, bb, L.params(precision="f32", **kw))[0]["variant"] != "lane"
    with pytest.raises(L.LimError, match="LIM_E_UNSUPPORTED"):
        L.plan_describe(ctx, bb, L.params(precision="f32", feedback="check_move_multi", variant="lane"))
