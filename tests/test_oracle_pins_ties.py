"""Pin of the oracle's LocalMove tie set in binary16 and bfloat16 storage.

LocalMove flips a qubit of the argmax of the beliefs around a ringing check,
ties broken uniformly at random (Algorithm 1).  With alpha = 1 (one undamped
min-sum sweep per tick) the exact beliefs are integer combinations of the prior
(and of CLAMP), so the beliefs around a check are often exactly equal, and
beliefs that differ at all differ by about a prior unit.  FP64 and binary32
keep those ties exact.  Binary16 and bfloat16 storage rounds the messages and
turns the ties into near-ties a few storage ulps apart.  The oracle's tie set
under ``tie_rel`` (every belief >= best - tie_rel * max(1, |best|)) restores
them.

The pin is against the paper's own arithmetic: with the library's default
tolerance for the format, every shot of the reduced-precision oracle has the
record of the FP64 oracle (clearing tick, convergence, failure, number of
moves, ticks), on 2D and 3D point-like toric codes.  A tolerance that is not
applied, or one that is too small, fails the pin: with exact ties only about
a third to two thirds of the shots keep FP64's record.
"""
import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import inputs as I
from paper_2609_38139_b300 import lim

FIELDS = ("t_clr", "converged", "failed", "moves", "ticks")
THREADS = 8
SHOTS = 300

CASES = [
    # name, code maker, error rate, tick budget
    ("toric2d_8", lambda: I.toric2d(8), 0.08, 320),
    ("toric2d_12", lambda: I.toric2d(12), 0.08, 480),
    ("point_6", lambda: I.toric3d_point(6), 0.025, 240),
]


def _identical(a, b):
    return np.all(np.stack([a[f] == b[f] for f in FIELDS]), axis=0)


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("name,maker,p,T", CASES, ids=[c[0] for c in CASES])
def test_tie_tolerance_reproduces_fp64_records(name, maker, p, T, prec):
    oc = O.OracleCode.from_code(maker())
    ref = O.run_shots(oc, O.params(precision="f64", tick_budget=T), p, 3, 7, 0, SHOTS, threads=THREADS)
    tol = lim.default_tie_rel(prec)
    assert tol > 0
    r = O.run_shots(oc, O.params(precision=prec, tick_budget=T, tie_rel=tol), p, 3, 7, 0, SHOTS,
                    threads=THREADS)
    same = _identical(r, ref)
    assert same.all(), (name, prec, np.nonzero(~same)[0][:10])
    assert 0 < int(ref["failed"].sum()) < SHOTS  # the sample decides something
    # exact ties in the same storage leave many shots on other trajectories
    r0 = O.run_shots(oc, O.params(precision=prec, tick_budget=T, tie_rel=0.0), p, 3, 7, 0, SHOTS,
                     threads=THREADS)
    assert _identical(r0, ref).mean() < 0.9


def test_fp64_and_binary32_ties_are_exact():
    """FP64 and binary32 keep the exact ties: a tolerance changes no record."""
    oc = O.OracleCode.from_code(I.toric2d(8))
    base = O.run_shots(oc, O.params(precision="f64", tick_budget=320), 0.08, 3, 7, 0, SHOTS,
                       threads=THREADS)
    for prec in ("f64", "f32"):
        r = O.run_shots(oc, O.params(precision=prec, tick_budget=320, tie_rel=2.0 ** -5), 0.08, 3,
                        7, 0, SHOTS, threads=THREADS)
        assert _identical(r, base).all(), prec


def test_tie_rel_refused_outside_its_domain():
    oc = O.OracleCode.from_code(I.toric2d(4))
    for prec, tol in (("f16", -0.01), ("f16", 0.6), ("f32", float("nan")), ("i16", 2.0 ** -5)):
        with pytest.raises(RuntimeError):
            O.run_shots(oc, O.params(precision=prec, tie_rel=tol), 0.05, 0, 0, 0, 2)
