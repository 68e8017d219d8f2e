"""Pins of the oracle's randomness, clock process and quantised constants.

* Philox4x32-10 (Salmon et al., SC'11) is checked against two implementations
  that share nothing with the oracle: cuRAND's host-side Philox generator (run,
  on the CPU) and Triton's Philox (run in Triton's CPU interpreter).  A wrong
  round multiplier, Weyl constant or word permutation changes every block.
* The clock process of Algorithm 1 -- independent rate-1 Poisson clocks on the
  active checks, whose superposition rings after an Exp(|S(t)|) waiting time --
  discretised per tick (every active check rings with probability
  rho = 1 - exp(-dt), the rings of a tick act in the order of their ring times):
  its rate, its waiting time and its order are observed through trajectories
  of the oracle on codes built so that every ring becomes a move.
* The quantised prior and clamp of the integer path: pi_q is the integer step
  nearest to the prior log(q/(1-q)) (Sec. S1), CLAMP_q the step nearest to CLAMP
  (Sec. S4) unless the storage saturates first (|m| <= Qmax).
"""
import ctypes
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import inputs as I


# ---------------------------------------------------------------------------
# Philox4x32-10 against independent implementations
# ---------------------------------------------------------------------------
CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # curandRngType value in curand.h


def _curand():
    names = []
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH") or "/usr/local/cuda"
    names.append(os.path.join(home, "lib64", "libcurand.so"))
    names.append("libcurand.so")
    for nm in names:
        try:
            return ctypes.CDLL(nm)
        except OSError:
            continue
    return None


def test_philox4x32_matches_curand_host_generator():
    """cuRAND's host Philox4x32-10 generator with seed S emits, as its i-th
    block of four words, Philox4x32-10 of counter (0, 0, i, 0) under the key
    (S mod 2^32, S div 2^32) (the layout was found by running it: block i is
    subsequence i).  The generator runs on the CPU; no GPU is involved."""
    cr = _curand()
    assert cr is not None, "libcurand from the CUDA toolkit is required for this pin"
    nblocks = 96
    for seed in (0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF, 0x00000001FFFFFFFF, 2 ** 32):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
        try:
            assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
            out = np.zeros(4 * nblocks, dtype=np.uint32)
            assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.c_size_t(out.size)) == 0
        finally:
            cr.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in range(nblocks):
            got = O.philox4x32([0, 0, i, 0], key)
            assert [int(x) for x in got] == [int(x) for x in out[4 * i:4 * i + 4]], (hex(seed), i)


_TRITON_SCRIPT = r"""
import json, sys
import torch, triton, triton.language as tl

@triton.jit
def _philox(out_ptr, c_ptr, seed):
    c0 = tl.load(c_ptr + 0)
    c1 = tl.load(c_ptr + 1)
    c2 = tl.load(c_ptr + 2)
    c3 = tl.load(c_ptr + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 0, a)
    tl.store(out_ptr + 1, b)
    tl.store(out_ptr + 2, c)
    tl.store(out_ptr + 3, d)

res = []
for ctr, seed in json.load(sys.stdin):
    out = torch.zeros(4, dtype=torch.uint32)
    _philox[(1,)](out, torch.tensor(ctr, dtype=torch.uint32), seed)
    res.append([int(x) for x in out])
print(json.dumps(res))
"""


def test_philox4x32_matches_triton_interpreter():
    """Triton's tl.philox (seed split into the two key words, ten rounds),
    executed by Triton's CPU interpreter, on arbitrary counters and keys."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    cases = [([int(x) for x in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)],
              int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))) for _ in range(40)]
    cases += [([0, 0, 0, 0], 0), ([0xFFFFFFFF] * 4, 2 ** 64 - 1)]
    env = dict(os.environ, TRITON_INTERPRET="1")
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(cases),
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    ref = json.loads(r.stdout.strip().splitlines()[-1])
    for (ctr, seed), want in zip(cases, ref):
        got = O.philox4x32(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert [int(x) for x in got] == want, (ctr, hex(seed))


# ---------------------------------------------------------------------------
# The clock process (Algorithm 1's Poisson clocks, per tick)
# ---------------------------------------------------------------------------
def _pairs_code(K):
    """K disjoint checks {2i, 2i+1}.  With q = 1/2 the prior is 0, every message
    stays 0, so every belief is L = 0 >= theta_2 = -log(1) = 0: Evidence always
    holds and a ring of an active check is always a move, which clears it."""
    return I.code_from_rows(f"pairs{K}", 2 * K, [[2 * i, 2 * i + 1] for i in range(K)], [],
                            logicals=[])


def _clear_ticks(K, dt, seed, shot, T):
    """Tick at which each of the K initially active checks rang (0 = never)."""
    code = _pairs_code(K)
    oc = O.OracleCode.from_code(code)
    prm = O.params(q=0.5, dt_tick=dt, tau=dt, tick_budget=T)  # alpha = 1
    e0 = np.zeros(code.n, np.uint8)
    e0[0::2] = 1
    r = O.run_shot(oc, prm, 0.0, seed, 0, shot, e0=e0, trace_ticks=T)
    s = r["trace"]["s_hist"]
    assert s[0].all()
    out = np.zeros(K, np.int64)
    for t in range(1, T + 1):
        rang = (s[t - 1] == 1) & (s[t] == 0)
        out[rang] = t
    # each check clears exactly once and only by its own ring
    assert r["moves"] == int((out > 0).sum())
    return out


@pytest.mark.parametrize("dt", [0.1, 0.5])
def test_ring_rate_is_one_minus_exp_minus_dt(dt):
    """Each active check rings within a tick of length dt with probability
    1 - exp(-dt) (a rate-1 Poisson clock).  Counted over every (tick, active
    check): rings / trials within 3 binomial sigma; the alternatives dt and
    exp(-dt) lie far outside at dt = 0.5."""
    K, T = 3000, 200
    ct = _clear_ticks(K, dt, seed=5, shot=0, T=T)
    assert (ct > 0).all(), "budget too small for the test"
    trials = int(ct.sum())            # a check is active (a trial) up to and including its ring tick
    rings = K
    rho = 1.0 - math.exp(-dt)
    sig = math.sqrt(trials * rho * (1 - rho))
    assert abs(rings - rho * trials) <= 3 * sig, (rings, rho * trials, sig)
    for wrong in (dt, math.exp(-dt)):
        if abs(wrong - rho) > 0.05:
            assert abs(rings - wrong * trials) > 10 * sig


def test_waiting_time_of_the_first_ring_is_exponential_in_active_checks():
    """With |S| active checks the first ring comes after an Exp(|S|) waiting
    time (superposition of |S| rate-1 clocks; the simulation rule of the
    numerics paragraph).  Per tick: P(no ring in the first t ticks) =
    exp(-|S| dt t).  The empirical survival function of the first ring's tick
    over many shots matches it within 3 sigma at every t (dt = 0.05, |S| = 4)."""
    K, dt, shots = 4, 0.05, 1500
    code = _pairs_code(K)
    oc = O.OracleCode.from_code(code)
    prm = O.params(q=0.5, dt_tick=dt, tick_budget=400)
    e0 = np.zeros(code.n, np.uint8)
    e0[0::2] = 1
    first = []
    for sh in range(shots):
        r = O.run_shot(oc, prm, 0.0, 9, 3, sh, e0=e0, trace_ticks=0, move_cap=1)
        assert r["trace"]["n_moves"] >= 1
        first.append(int(r["trace"]["moves"][0][0]))
    first = np.array(first)
    for t in (1, 2, 3, 5, 8, 12, 20):
        surv = np.mean(first > t)
        p = math.exp(-K * dt * t)
        assert abs(surv - p) <= 3 * math.sqrt(p * (1 - p) / shots) + 1e-12, (t, surv, p)
    # mean waiting time in clock units: dt / (1 - e^{-|S| dt}) -> 1/|S| as dt -> 0
    mean_t = first.mean() * dt
    want = dt / (1 - math.exp(-K * dt))
    sd = want * math.exp(-K * dt / 2) / math.sqrt(shots)  # sd of a geometric mean, in time units
    assert abs(mean_t - want) <= 3 * sd + 1e-12, (mean_t, want)
    assert abs(want - 1.0 / K) < dt


def test_ring_order_is_ring_time_order():
    """Two active checks sharing a qubit: chain 0-1-2, checks c0 = {0,1},
    c1 = {1,2}, error on qubit 1, every clock rings (rho = 1), all beliefs tied
    (q = 1/2).  The rings act in the order of their ring times (word 1 of the
    check's Philox block (shot, tick, check, point<<4 | 1); ties by check
    index); each picks qubit N(c)[(u2 * 2) >> 32]; a check that an earlier move
    has cleared does nothing.  The state after tick 1 is predicted by hand from
    the Philox words for 400 shots and must cover both orders and all outcomes."""
    code = I.code_from_rows("chain3", 3, [[0, 1], [1, 2]], [], logicals=[])
    oc = O.OracleCode.from_code(code)
    prm = O.params(q=0.5, dt_tick=0.1, ring_prob=1.0, tick_budget=1)
    e0 = np.array([0, 1, 0], np.uint8)
    seed, point = 77, 6
    seen_orders, seen_outcomes = set(), set()
    rows = [[0, 1], [1, 2]]
    for shot in range(400):
        words = {c: O.philox4x32([shot, 1, c, (point << 4) | 1], [seed & 0xFFFFFFFF, seed >> 32])
                 for c in (0, 1)}
        order = sorted((0, 1), key=lambda c: (int(words[c][1]), c))
        e = e0.copy()
        for c in order:
            if (e[rows[c][0]] ^ e[rows[c][1]]) == 0:
                continue  # cleared by the earlier move
            v = rows[c][(int(words[c][2]) * 2) >> 32]
            e[v] ^= 1
        r = O.run_shot(oc, prm, 0.0, seed, point, shot, e0=e0, trace_ticks=1)
        assert np.array_equal(r["trace"]["e_hist"][1], e), (shot, order)
        seen_orders.add(tuple(order))
        seen_outcomes.add(tuple(e))
    assert len(seen_orders) == 2 and len(seen_outcomes) >= 3


# ---------------------------------------------------------------------------
# Quantised prior and clamp of the integer path
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,q,delta", [("i16", 0.05, 2 ** -6), ("i16", 0.125, 2 ** -6),
                                          ("i8", 0.05, 0.25), ("i8", 0.125, 0.25),
                                          ("i16", 0.3, 2 ** -3)])
def test_quantised_prior_is_the_nearest_step(prec, q, delta):
    """The prior LLR log(q/(1-q)) (Sec. S1) in integer steps of Delta is the
    nearest step: the read-out of tick 1 (m = 0, Eq. 3) is pi_q for every qubit,
    with |pi_q Delta - pi| <= Delta/2.  With no rings, tick 2 still reads pi_q
    (the first Jacobi sweep from m = 0 leaves every check message at 0) and at
    tick 3 every belief on the 2D toric code is pi_q plus, per check of the
    qubit, (-1)^{s_c + d_c} times the sign product of the others times |pi_q|
    (min-sum on equal magnitudes), computed here by hand.  The cases put
    pi/Delta on both sides of a half step, so floor and truncation both fail
    one of them."""
    pi = math.log(q / (1 - q))
    code = I.toric2d(4)
    oc = O.OracleCode.from_code(code)
    prm = O.params(precision=prec, quant_scale=delta, q=q, tick_budget=3, ring_prob=0.0)
    r = O.run_shot(oc, prm, 0.12, 3, 0, 1, trace_ticks=3, want_l=True)
    s0 = r["trace"]["s_hist"][0]
    assert s0.any(), "need a nonzero syndrome"
    L1 = r["trace"]["l_hist"][1]
    pq = L1[0]
    assert np.all(L1 == pq) and pq == int(pq)
    assert abs(pq * delta - pi) <= delta / 2 + 1e-15, (pq, pi / delta)
    # no ring (rho = 0): tick 2 reads the first sweep from m = 0, which (Jacobi:
    # both families from the previous iterate) leaves every check message at 0
    assert np.all(r["trace"]["l_hist"][2] == pq)
    # tick 3 reads the second sweep: every qubit->check message is pi_q, so each
    # check message is (-1)^{s_c + d_c} (sign of pi_q)^{d_c - 1} |pi_q|
    L3 = r["trace"]["l_hist"][3]
    hx = code.hx_dense()
    for v in range(code.n):
        want = pq
        for c in np.nonzero(hx[:, v])[0]:
            d = int(hx[c].sum())
            neg = (int(s0[c]) + d + (d - 1)) & 1  # every input is pi_q < 0
            want += -abs(pq) if neg else abs(pq)
        assert L3[v] == want, v


@pytest.mark.parametrize("prec,delta,clamp,want", [
    ("i16", 0.25, 10.4, 42),        # 41.6 steps: nearest 42 (floor and truncation give 41)
    ("i16", 0.25, 10.6, 42),        # 42.4 steps: nearest 42 (ceiling gives 43)
    ("i16", 2 ** -6, 1000.0, 32767),  # 64000 steps: saturates at Qmax
    ("i8", 0.25, 1000.0, 127),      # 4000 steps: saturates at Qmax, never -128
    ("i8", 0.25, 20.1, 80),         # 80.4 steps
])
def test_quantised_clamp_is_the_nearest_step_or_qmax(prec, delta, clamp, want):
    """CLAMP on every message (Sec. S4) in integer steps: the step nearest to
    CLAMP/Delta, or Qmax when the storage saturates first.  Observed as the
    magnitude a sweep gives to a message whose BP value is far beyond CLAMP,
    on both families (check->qubit from a large qubit->check input, qubit->check
    from large check->qubit inputs), with both signs."""
    assert want == min({"i16": 32767, "i8": 127}[prec], round(clamp / delta))
    # qubit 0 in checks 0, 1, 2; qubits 1, 2, 3 in one check each
    code = I.code_from_rows("star", 4, [[0, 1], [0, 2], [0, 3]], [], logicals=[])
    oc = O.OracleCode.from_code(code)
    prm = O.params(precision=prec, quant_scale=delta, clamp=clamp, q=0.05)
    big = 30000.0 if prec == "i16" else 120.0
    # edges: 0=(c0,q0) 1=(c0,q1) 2=(c1,q0) 3=(c1,q2) 4=(c2,q0) 5=(c2,q3)
    cv = np.array([0.0, 0.0, big, 0.0, big, 0.0])
    vc = np.array([big, -big, big, big, big, big])
    ncv, nvc = O.bp_sweeps(oc, prm, np.zeros(3, np.uint8), cv, vc, 1)
    # q0 -> c0 = pi + 2 big: clamped
    assert nvc[0] == want
    # c0 -> q0 = (-1)^{0+2} * (-big) and c0 -> q1 = +big (sign of q0's input): clamped both
    # ways (a min-sum output is one of its stored inputs, so it only meets a clamp below them)
    assert ncv[0] == -min(big, want) and ncv[1] == min(big, want)
    cv2 = -cv
    _, nvc2 = O.bp_sweeps(oc, prm, np.zeros(3, np.uint8), cv2, vc, 1)
    assert nvc2[0] == -want
