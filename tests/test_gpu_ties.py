"""Binary16 and bfloat16 storage with LocalMove's tie tolerance (lim_params.tie_rel).

LocalMove flips a qubit of the argmax of the beliefs around a ringing check,
ties broken uniformly at random (Algorithm 1).  With alpha = 1 the exact
min-sum beliefs are integer combinations of the prior, so exact ties are
frequent; 16-bit floating storage turns them into near-ties a few ulps apart.
The tie set {L_v >= best - tie_rel * max(1, |best|)} (binary32 arithmetic)
keeps them ties.

* Parity: every kernel that takes the argmax (block and warp teams, one shot
  per lane, the sequential gauge-switch path, the multi-qubit move) against the
  oracle in the same storage format and tolerance, shot by shot: records,
  tallies and final residuals bit-exact.
* Logical error rate against FP64 (the configuration target: within 3 binomial
  sigma), paired on the same shots: with the default tolerance of its format,
  binary16 and bfloat16 storage reproduce FP64's failures on the 2D and 3D
  point-like toric codes, where exact ties (tie_rel = 0) fall short by 4-14 %.
"""
import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

from parity import compare_records, oracle_params, oracle_point, oracle_shots_with_finals, paired_ok

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


PARITY = [
    # id, code, precision, variant, feedback, gauge_on_move, p, budget, shots
    ("toric2d8-f16-cta", lambda: I.toric2d(8), "f16", "cta", "check_move", 0, 0.08, 320, 300),
    ("toric2d8-bf16-warp", lambda: I.toric2d(8), "bf16", "warp", "check_move", 0, 0.08, 320, 300),
    ("toric2d8-f16-lane", lambda: I.toric2d(8), "f16", "lane", "check_move", 0, 0.08, 320, 512),
    ("point4-bf16-lane", lambda: I.toric3d_point(4), "bf16", "lane", "check_move", 0, 0.03, 160, 512),
    ("point6-f16-warp", lambda: I.toric3d_point(6), "f16", "warp", "check_move", 0, 0.025, 240, 300),
    ("point6-bf16-cta", lambda: I.toric3d_point(6), "bf16", "cta", "check_move", 0, 0.025, 240, 300),
    ("toric2d6-f16-gauge", lambda: I.toric2d(6), "f16", "cta", "check_move", 1, 0.07, 120, 200),
    ("toric2d6-bf16-multi", lambda: I.toric2d(6), "bf16", "cta", "check_move_multi", 0, 0.07, 120, 200),
]


@pytest.mark.parametrize("cid,maker,prec,variant,fb,gauge,p,T,shots", PARITY, ids=[c[0] for c in PARITY])
def test_tie_tolerance_bit_exact(L, ctx, cid, maker, prec, variant, fb, gauge, p, T, shots):
    code = maker()
    lc = ctx.from_inputs(code)
    tol = L.default_tie_rel(prec)
    assert tol > 0
    prm = L.params(precision=prec, feedback=fb, gauge_on_move=gauge, tick_budget=T, variant=variant,
                   tie_rel=tol)
    pts = [(lc, p, shots, 0, 5)]
    shape, _ = L.plan_describe(ctx, pts, prm)
    assert shape["variant"] == variant, shape
    tal, rec, fin = L.run_batch(ctx, pts, prm, 13, e_final=True)
    ora, fins = oracle_shots_with_finals(code, oracle_params(prm), p, 13, 5, 0, shots)
    compare_records(rec, ora, cid)
    assert int(tal[0]["failures"]) == int(ora["failed"].sum()) and int(tal[0]["errors"]) == 0
    assert np.array_equal(L.bits_to_bytes(fin, code.n), fins), cid
    # the tolerance is taken: the same shots with exact ties follow other trajectories
    _, rec0 = L.run_batch(ctx, pts, L.params(precision=prec, feedback=fb, gauge_on_move=gauge,
                                              tick_budget=T, variant=variant), 13)
    assert not np.array_equal(rec0["moves"], rec["moves"]), cid


LER = [
    # name, code, tick budget, error rates
    ("toric2d_16", lambda: I.toric2d(16), 640, (0.06, 0.10)),
    ("point_8", lambda: I.toric3d_point(8), 320, (0.01, 0.03)),
]


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("name,maker,T,ps", LER, ids=[c[0] for c in LER])
def test_ler_paired_against_fp64_with_tie_tolerance(L, ctx, name, maker, T, ps, prec):
    """300 shots at two error rates against the FP64 oracle, paired."""
    code = maker()
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, tick_budget=T, tie_rel=L.default_tie_rel(prec))
    shots = 300
    pts = [(lc, p, shots, 0, 20 + i) for i, p in enumerate(ps)]
    _, rec = L.run_batch(ctx, pts, prm, 1)
    for i, p in enumerate(ps):
        gpu = rec[i * shots:(i + 1) * shots]
        ora = oracle_point(code, prm, p, 1, 20 + i, 0, shots, precision="f64")
        ok, (b, c) = paired_ok(gpu["failed"], ora["failed"])
        print(f"{name} {prec} p={p}: failures gpu {int(gpu['failed'].sum())} fp64 "
              f"{int(ora['failed'].sum())}, discordant {b}/{c}")
        assert ok, (name, prec, p, b, c)


LARGE = [
    ("point_8", lambda: I.toric3d_point(8), 320, 0.015, "f16"),
    ("point_8", lambda: I.toric3d_point(8), 320, 0.015, "bf16"),
    ("toric2d_16", lambda: I.toric2d(16), 640, 0.06, "f16"),
    ("toric2d_16", lambda: I.toric2d(16), 640, 0.06, "bf16"),
]


@pytest.mark.parametrize("name,maker,T,p,prec", LARGE, ids=[f"{c[0]}-{c[4]}" for c in LARGE])
def test_ler_large_sample_with_tie_tolerance(L, ctx, name, maker, T, p, prec):
    """20,000 shots of one point against the same shots in FP32, whose failures
    stand for FP64's (checked on the first 400 against the oracle); paired
    3-sigma bar.  These are the points where exact ties miss FP64 by 4-9 %."""
    code = maker()
    lc = ctx.from_inputs(code)
    n = 20000
    pts = [(lc, p, n, 0, 77)]
    _, rec32 = L.run_batch(ctx, pts, L.params(precision="f32", tick_budget=T), 4)
    ora = oracle_point(code, L.params(precision="f32", tick_budget=T), p, 4, 77, 0, 400, precision="f64")
    ok, (b, c) = paired_ok(rec32["failed"][:400], ora["failed"])
    assert ok and b + c <= 8, ("FP32 does not stand for FP64 here", b, c)
    _, rec = L.run_batch(ctx, pts, L.params(precision=prec, tick_budget=T,
                                            tie_rel=L.default_tie_rel(prec)), 4)
    ok, (b, c) = paired_ok(rec["failed"], rec32["failed"])
    print(f"{name} {prec} p={p}: failures {int(rec['failed'].sum())} vs FP32/FP64 "
          f"{int(rec32['failed'].sum())} of {n}, discordant {b}/{c}")
    assert ok, (name, prec, p, b, c)
