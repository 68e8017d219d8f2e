"""Logical error rates of the CUDA path against the FP64 oracle, paired on the
same shots, for every configuration's storage precision.

The bar is a McNemar-style paired test: over the shots where exactly one of the
two fails (b GPU-only failures, c oracle-only failures), |b - c| <= 3 sqrt(b + c)
(+1 for the discreteness of small counts).  Points are the configurations' own
error rates plus, for the membrane sector (whose configuration grid 0.01-0.06 is
far below its threshold, so that no shot fails there), points near the
threshold of Table S1 where failures occur.

FP32 reproduces FP64's failures (no discordant shot on the samples here), and
so does integer storage (int16 with Delta = 2^-6, int8 with Delta = |pi|): with
alpha = 1 every min-sum message is a clamped integer combination of the prior,
and exact arithmetic keeps the exact ties among the beliefs of a check, which
LocalMove breaks uniformly at random ("breaking ties randomly", Algorithm 1).
Binary16 and bfloat16 storage round those values (by ~1e-3 at |L| ~ 3) and
turn exact ties into near-ties that the argmax then breaks by rounding noise
instead of by the random pick: on large samples their logical error rate is
lower than FP64's by 5-15 %, beyond 3 sigma.  So is int8's with Delta = 2^-2,
whose messages saturate at 127 steps = 31.75 LLR instead of CLAMP = 1000.
Those tests state the target and are marked as expected failures: they run
binary16 and bfloat16 with exact ties (tie_rel = 0).  With the library's
default tie tolerance of their format the same points meet the target
(tests/test_gpu_ties.py).
"""
import numpy as np
import pytest

from paper_2609_38139_b300 import inputs as I

from parity import oracle_point, paired_ok

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


# int8 step: one per prior unit |log(q/(1-q))| at q = 0.05 (the library's default)
PRIOR_STEP = abs(np.log(0.05 / 0.95))

CASES = [
    # name, code maker, precision, Delta, q, tick budget, error rates, shots per rate
    ("toric2d_16", lambda: I.toric2d(16), "f32", 2 ** -6, 0.05, 640, (0.06, 0.10), 300),
    ("toric2d_16", lambda: I.toric2d(16), "i16", 2 ** -6, 0.05, 640, (0.06, 0.10), 300),
    ("point_8", lambda: I.toric3d_point(8), "f32", 2 ** -6, 0.05, 320, (0.01, 0.03), 300),
    ("point_8", lambda: I.toric3d_point(8), "i16", 2 ** -6, 0.05, 320, (0.01, 0.03), 300),
    ("membrane_6", lambda: I.toric3d_membrane(6), "i16", 2 ** -6, 0.125, 10000, (0.06, 0.14), 300),
    ("bb_6_6", lambda: I.bb_code(6, 6), "i8", PRIOR_STEP, 0.05, 10000, (0.04, 0.08), 300),
    ("bb_12_6", lambda: I.bb_code(12, 6), "i8", PRIOR_STEP, 0.05, 10000, (0.01, 0.08), 300),
]


@pytest.mark.parametrize("name,maker,prec,qs,q,T,ps,shots", CASES, ids=[f"{c[0]}-{c[2]}" for c in CASES])
def test_ler_paired_against_fp64(L, ctx, name, maker, prec, qs, q, T, ps, shots):
    code = maker()
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, quant_scale=qs, q=q, tick_budget=T)
    pts = [(lc, p, shots, 0, 10 + i) for i, p in enumerate(ps)]
    _, rec = L.run_batch(ctx, pts, prm, 1)
    for i, p in enumerate(ps):
        gpu = rec[i * shots:(i + 1) * shots]
        ora = oracle_point(code, prm, p, 1, 10 + i, 0, shots, precision="f64")
        ok, (b, c) = paired_ok(gpu["failed"], ora["failed"])
        print(f"{name} {prec} p={p}: failures gpu {int(gpu['failed'].sum())} fp64 "
              f"{int(ora['failed'].sum())}, discordant {b}/{c}")
        assert ok, (name, prec, p, b, c)


LARGE = [
    # the GPU's FP32 failures stand for FP64's on large samples (checked here on a
    # prefix of the same shots against the oracle)
    ("point_8", lambda: I.toric3d_point(8), "i16", 2 ** -6, 0.05, 320, 0.015),
    ("toric2d_16", lambda: I.toric2d(16), "i16", 2 ** -6, 0.05, 640, 0.06),
    ("bb_12_6", lambda: I.bb_code(12, 6), "i8", PRIOR_STEP, 0.05, 10000, 0.04),
    pytest.param("bb_12_6", lambda: I.bb_code(12, 6), "i8", 0.25, 0.05, 10000, 0.04,
                 marks=pytest.mark.xfail(strict=True, reason="int8 with Delta = 2^-2 saturates at "
                                         "31.75 LLR; its LER is below FP64's beyond 3 sigma")),
    pytest.param("point_8", lambda: I.toric3d_point(8), "f16", 2 ** -6, 0.05, 320, 0.015,
                 marks=pytest.mark.xfail(strict=True, reason="binary16 storage with exact ties breaks the "
                                         "exact belief ties of min-sum; its LER is below FP64's beyond 3 sigma")),
    pytest.param("point_8", lambda: I.toric3d_point(8), "bf16", 2 ** -6, 0.05, 320, 0.015,
                 marks=pytest.mark.xfail(strict=True, reason="bfloat16 storage with exact ties breaks the "
                                         "exact belief ties of min-sum; its LER is below FP64's beyond 3 sigma")),
    pytest.param("toric2d_16", lambda: I.toric2d(16), "f16", 2 ** -6, 0.05, 640, 0.06,
                 marks=pytest.mark.xfail(strict=True, reason="binary16 storage with exact ties breaks the "
                                         "exact belief ties of min-sum; its LER is below FP64's beyond 3 sigma")),
]


@pytest.mark.parametrize("name,maker,prec,qs,q,T,p", LARGE, ids=["point_8-i16", "toric2d_16-i16",
                                                               "bb_12_6-i8", "bb_12_6-i8-step-0.25",
                                                               "point_8-f16", "point_8-bf16",
                                                               "toric2d_16-f16"])
def test_ler_large_sample_against_fp64(L, ctx, name, maker, prec, qs, q, T, p):
    """20,000 shots of one point in the storage precision against the same shots
    in FP32, whose failures equal FP64's (checked on the first 400 shots against
    the oracle); paired 3-sigma bar."""
    code = maker()
    lc = ctx.from_inputs(code)
    n = 20000
    pts = [(lc, p, n, 0, 77)]
    _, rec32 = L.run_batch(ctx, pts, L.params(precision="f32", q=q, tick_budget=T), 4)
    ora = oracle_point(code, L.params(precision="f32", q=q, tick_budget=T), p, 4, 77, 0, 400,
                       precision="f64")
    ok, (b, c) = paired_ok(rec32["failed"][:400], ora["failed"])
    assert ok and b + c <= 8, ("FP32 does not stand for FP64 here", b, c)
    _, rec = L.run_batch(ctx, pts, L.params(precision=prec, quant_scale=qs, q=q, tick_budget=T), 4)
    ok, (b, c) = paired_ok(rec["failed"], rec32["failed"])
    print(f"{name} {prec} p={p}: failures {int(rec['failed'].sum())} vs FP32/FP64 "
          f"{int(rec32['failed'].sum())} of {n}, discordant {b}/{c}")
    assert ok, (name, prec, p, b, c)
