"""GPU parity: the CUDA path against the oracle, shot by shot, through the C ABI.

Bars (derived from the arithmetic; see the design notes):
  * integer, bit and index results (noise, syndromes, t_clr, flags, moves,
    final residuals, integer messages) are bit-exact;
  * floating min-sum messages are bit-exact against the oracle's emulation of
    the same precision (binary32 ops in the same order, same storage rounding),
    and within |m32 - m64| <= 1e-5 max(1, |m64|) of the FP64 oracle;
  * sum-product messages (transcendentals) are within that tolerance of FP64;
  * logical error rates agree with the FP64 oracle within 3 sigma (paired test).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import inputs as I

from parity import compare_records, oracle_params, oracle_point, paired_ok

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


def _unpack(words, nbits):
    from paper_2609_38139_b300.lim import bits_to_bytes
    return bits_to_bytes(np.asarray(words).view(np.uint32), nbits)


# ---------------------------------------------------------------------------
# noise
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("maker", [lambda: I.toric2d(8), lambda: I.toric2d(5), lambda: I.rep_code(2000),
                                   lambda: I.bb_code(12, 6), lambda: I.toric3d_membrane(3)])
@pytest.mark.parametrize("p", [0.0, 0.05, 0.45, 1.0])
def test_noise_bit_exact(L, ctx, maker, p):
    code = maker()
    lc = ctx.from_inputs(code)
    e, s = L.sample_noise(lc, p, 77, 3, 5, 40)
    torch.cuda.synchronize()
    e = _unpack(e.cpu().numpy(), code.n)
    s = _unpack(s.cpu().numpy(), code.m)
    oc = O.OracleCode.from_code(code)
    for i in range(40):
        eo, so = O.noise(oc, p, 77, 3, 5 + i)
        assert np.array_equal(e[i], eo), i
        assert np.array_equal(s[i], so), i


# ---------------------------------------------------------------------------
# fixed-state sweeps and read-out
# ---------------------------------------------------------------------------
def _random_state(rng, code, prec, B, scale):
    if prec in ("i16", "i8"):
        q = 3000 if prec == "i16" else 120
        cv = rng.integers(-q, q + 1, (B, code.E)).astype(np.float64)
        vc = rng.integers(-q, q + 1, (B, code.E)).astype(np.float64)
    else:
        cv = rng.normal(0, scale, (B, code.E))
        vc = rng.normal(0, scale, (B, code.E))
        cv[:, ::7] = 0.0
        cv, vc = np.float32(cv).astype(np.float64), np.float32(vc).astype(np.float64)
        if prec == "f16":
            cv, vc = np.float16(cv).astype(np.float64), np.float16(vc).astype(np.float64)
        if prec == "bf16":
            cv = torch.from_numpy(cv).to(torch.bfloat16).double().numpy()
            vc = torch.from_numpy(vc).to(torch.bfloat16).double().numpy()
    s = rng.integers(0, 2, (B, code.m)).astype(np.uint8)
    return s, cv, vc


def _to_dev(L, prm, a):
    return torch.from_numpy(a).to(L.torch_msg_dtype(prm)).cuda()


CODES = {"toric2d_6": lambda: I.toric2d(6), "bb_6_6": lambda: I.bb_code(6, 6),
         "membrane_3": lambda: I.toric3d_membrane(3), "repP_9": lambda: I.rep_code(9, True),
         "point_3": lambda: I.toric3d_point(3)}


@pytest.mark.parametrize("cname", list(CODES))
@pytest.mark.parametrize("prec", ["f32", "f16", "bf16", "i16", "i8"])
@pytest.mark.parametrize("relaxed", [False, True])
def test_minsum_sweeps_bit_exact(L, ctx, cname, prec, relaxed):
    code = CODES[cname]()
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, quant_scale=2 ** -6 if prec == "i16" else 0.25, clamp=40.0,
                   tau=0.1, dt_tick=0.03 if relaxed else 0.1)
    rng = np.random.default_rng(hash((cname, prec)) % 2 ** 32)
    B, K = 6, 3
    s, cv, vc = _random_state(rng, code, prec, B, 15.0)
    cvo, vco = L.bp_sweeps(lc, prm, torch.from_numpy(s).cuda(), _to_dev(L, prm, cv), _to_dev(L, prm, vc), K)
    cvo = cvo.double().cpu().numpy()
    vco = vco.double().cpu().numpy()
    Lg = L.readout(lc, prm, _to_dev(L, prm, cv)).double().cpu().numpy()
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    for b in range(B):
        rc, rv = O.bp_sweeps(oc, op, s[b], cv[b], vc[b], K)
        assert np.array_equal(cvo[b], rc), (b, np.max(np.abs(cvo[b] - rc)))
        assert np.array_equal(vco[b], rv), (b, np.max(np.abs(vco[b] - rv)))
        assert np.array_equal(Lg[b], O.readout(oc, op, cv[b])), b


@pytest.mark.parametrize("cname", ["toric2d_6", "bb_6_6", "membrane_3"])
@pytest.mark.parametrize("rule", ["minsum", "sumproduct"])
def test_f32_sweeps_match_fp64_oracle(L, ctx, cname, rule):
    """The 1e-5 relative bar against FP64 messages, on fixed states."""
    code = CODES[cname]()
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", rule=rule)
    rng = np.random.default_rng(5)
    B = 8
    s, cv, vc = _random_state(rng, code, "f32", B, 6.0)
    cvo, vco = L.bp_sweeps(lc, prm, torch.from_numpy(s).cuda(), _to_dev(L, prm, cv), _to_dev(L, prm, vc), 1)
    cvo = cvo.double().cpu().numpy()
    vco = vco.double().cpu().numpy()
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm, precision="f64")
    for b in range(B):
        rc, rv = O.bp_sweeps(oc, op, s[b], cv[b], vc[b], 1)
        assert np.all(np.abs(cvo[b] - rc) <= 1e-5 * np.maximum(1.0, np.abs(rc))), b
        assert np.all(np.abs(vco[b] - rv) <= 1e-5 * np.maximum(1.0, np.abs(rv))), b


# ---------------------------------------------------------------------------
# whole trajectories, shot by shot
# ---------------------------------------------------------------------------
def _batch_vs_oracle(L, ctx, code, prm, p, nshots, seed=11, point_id=2, shot0=0, finals=True):
    lc = ctx.from_inputs(code)
    tal, rec, fin = L.run_batch(ctx, [(lc, p, nshots, shot0, point_id)], prm, seed, e_final=True)
    ora = oracle_point(code, prm, p, seed, point_id, shot0, nshots)
    compare_records(rec, ora, f"{code.name} {L.prec_name(prm)}")
    assert tal[0]["shots"] == nshots and tal[0]["errors"] == 0
    assert tal[0]["failures"] == int(ora["failed"].sum())
    assert tal[0]["nonconverged"] == int((ora["converged"] == 0).sum())
    assert tal[0]["sweeps"] == int(ora["sweeps"].sum())
    if finals:
        # residual of each shot = e0 + correction; check it through the syndrome-free
        # failure test and, on a sample, against the oracle's final state
        oc = O.OracleCode.from_code(code)
        op = oracle_params(prm)
        e_gpu = _unpack(fin, code.n)
        for sh in range(0, nshots, max(1, nshots // 16)):
            r = O.run_shot(oc, op, p, seed, point_id, shot0 + sh, trace_ticks=0)
            assert r["ticks"] == rec[sh]["ticks"]
            e_or = _final_e(oc, op, p, seed, point_id, shot0 + sh)
            assert np.array_equal(e_gpu[sh], e_or), sh
    return tal, rec


def _final_e(oc, op, p, seed, pid, shot):
    T = op.tick_budget
    r = O.run_shot(oc, op, p, seed, pid, shot, trace_ticks=T)
    return r["trace"]["e_hist"][T]


@pytest.mark.parametrize("variant", ["cta", "warp"])
def test_toric2d_L8_config_f32(L, ctx, variant):
    """2D toric code L=8, p=0.05, FP32 min-sum, 1 sweep per tick, budget 4L, 1000 shots."""
    prm = L.params(precision="f32", tick_budget=32, variant=variant)
    _batch_vs_oracle(L, ctx, I.toric2d(8), prm, 0.05, 1000)


@pytest.mark.parametrize("prec", ["f32", "i16"])
def test_rep_chain_2000_discrete(L, ctx, prec):
    """Open repetition chain d=2000, p=0.45, bit-centric machine (BP exact on the chain)."""
    prm = L.params(feedback="bit_discrete", precision=prec, quant_scale=2 ** -6, tick_budget=8001,
                   variant="cta")
    tal, rec = _batch_vs_oracle(L, ctx, I.rep_code(2000), prm, 0.45, 96, finals=False)
    # Theorem (rep code): failure iff the initial error has a majority
    oc = O.OracleCode.from_code(I.rep_code(2000))
    for sh in range(96):
        e0, _ = O.noise(oc, 0.45, 11, 2, sh)
        w = int(e0.sum())
        if 2 * w != 2000:
            assert rec[sh]["failed"] == int(2 * w > 2000)


@pytest.mark.parametrize("maker,prec,qs,variant", [
    (lambda: I.toric3d_membrane(4), "i16", 2 ** -6, "cta"),
    (lambda: I.toric3d_membrane(3), "i16", 2 ** -6, "warp"),
    (lambda: I.bb_code(6, 6), "i8", 0.25, "warp"),
    (lambda: I.bb_code(12, 6), "i8", 0.25, "cta"),
    (lambda: I.toric3d_point(4), "f16", 0, "cta"),
    (lambda: I.toric3d_point(4), "bf16", 0, "warp"),
    (lambda: I.toric2d(5), "f32", 0, "warp"),
])
def test_precisions_bit_exact(L, ctx, maker, prec, qs, variant):
    code = maker()
    q = 0.125 if "membrane" in code.name else 0.05
    prm = L.params(precision=prec, quant_scale=qs or 2 ** -6, q=q, tick_budget=200, variant=variant)
    _batch_vs_oracle(L, ctx, code, prm, 0.06, 160)


def test_relaxed_multi_sweep_and_gauge(L, ctx):
    """K = 2 sweeps per tick with alpha = dt/(K tau) = 0.5, and the gauge-on-move flag."""
    code = I.toric2d(6)
    prm = L.params(precision="f32", dt_tick=0.1, tau=0.1, sweeps_per_tick=2, tick_budget=120)
    _batch_vs_oracle(L, ctx, code, prm, 0.06, 120)
    prm = L.params(precision="f32", tick_budget=120, gauge_on_move=1)
    _batch_vs_oracle(L, ctx, code, prm, 0.06, 120)
    prm = L.params(precision="i16", tick_budget=120, gauge_on_move=1, dt_tick=0.05, variant="warp")
    _batch_vs_oracle(L, ctx, I.toric3d_membrane(3), prm, 0.05, 80)


@pytest.mark.parametrize("maker,prec,q,dt,p,variant", [
    (lambda: I.toric2d(6), "f32", 0.05, 0.001, 0.06, "warp"),
    (lambda: I.toric2d(8), "f32", 0.05, 0.001, 0.08, "cta"),
    (lambda: I.toric3d_point(3), "f16", 0.05, 0.001, 0.03, "cta"),
    (lambda: I.toric3d_membrane(3), "i16", 0.125, 0.01, 0.12, "warp"),
    (lambda: I.bb_code(6, 6), "i8", 0.05, 0.01, 0.05, "warp"),
])
def test_fine_dt_trajectories(L, ctx, maker, prec, q, dt, p, variant):
    """Table S1 discretisations: relaxation alpha = dt/tau (0.01 or 0.1), ring
    probability 1 - exp(-dt) per tick, and a budget of 100 time units (1e4 or 1e5
    ticks); every shot's trajectory summary equals the oracle's."""
    prm = L.params(precision=prec, quant_scale=0.25 if prec == "i8" else 2 ** -6, q=q, tau=0.1,
                   dt_tick=dt, tick_budget=int(round(100 / dt)), variant=variant)
    _batch_vs_oracle(L, ctx, maker(), prm, p, 16, finals=False)


@pytest.mark.parametrize("prec", ["f32", "i16"])
def test_bp_decoder_row_matches_oracle_decoder(L, ctx, prec):
    """Ordinary BP decoding of the 2D toric code, the comparison decoder: the
    bit-centric machine on the GPU against the oracle's gauge-free BP decoder
    (fixed syndrome, hard decision after every iteration), shot by shot, final
    residual e0 + ehat included."""
    code = I.toric2d(8)
    prm = L.params(feedback="bit_discrete", precision=prec, tick_budget=100)
    lc = ctx.from_inputs(code)
    tal, rec, fin = L.run_batch(ctx, [(lc, 0.05, 64, 0, 4)], prm, 13, e_final=True)
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    ora = O.bp_decode_shots(oc, op, 0.05, 13, 4, 0, 64)
    compare_records(rec, ora, f"bp decoder {prec}")
    e_gpu = _unpack(fin, code.n)
    for sh in range(64):
        _, ehat = O.bp_decode(oc, op, 0.05, 13, 4, sh)
        e0, _ = O.noise(oc, 0.05, 13, 4, sh)
        assert np.array_equal(e_gpu[sh], e0 ^ ehat), sh


def test_study_runner_on_rep_fig2(L, ctx):
    """The adaptive Monte Carlo runner on the Fig. 2 workload (d = 20): per point,
    the failures are the shots whose initial error has a strict majority, up to
    exact ties and non-converged shots (Theorem on the rep code)."""
    from paper_2609_38139_b300 import study as S
    rows = S.run_study(ctx, "rep_fig2", max_shots=256, max_failures=10 ** 9, batch_shots=128,
                       sizes=[20])
    assert len(rows) == 9
    oc = O.OracleCode.from_code(I.rep_code(20))
    for r in rows:
        assert r["shots"] == 256
        maj = ties = 0
        for sh in range(256):
            w = int(O.noise(oc, r["p"], 0, r["point_id"], sh)[0].sum())
            maj += 2 * w > 20
            ties += 2 * w == 20
        assert maj <= r["failures"] <= maj + ties + r["nonconverged"], r


def _pack_rows(bits, words):
    """0/1 rows -> rows of 32-bit words (bit v % 32 of word v // 32)."""
    out = np.zeros((bits.shape[0], words), dtype=np.uint32)
    for v in range(bits.shape[1]):
        out[:, v // 32] |= bits[:, v].astype(np.uint32) << np.uint32(v % 32)
    return out


def test_run_from_given_errors(L, ctx):
    """lim_run_batch_from / lim_run_batch_host: (a) the device's own noise fed
    back gives exactly lim_run_batch's records, residuals and tallies; (b) hand-made
    initial errors (one qubit, a row of a logical, a dense random pattern) give the
    oracle's trajectories from the same errors; (c) the host-buffer call returns
    the same."""
    code = I.toric2d(8)
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", tick_budget=64)
    pts = [(lc, 0.06, 40, 0, 3), (lc, 0.1, 24, 100, 5)]
    ref = L.Batch(ctx, pts, prm, e_final=True)
    ref.run(9)
    torch.cuda.synchronize()
    words = ref.words
    e0 = torch.zeros((ref.nshots, words), dtype=torch.int32, device="cuda")
    row = 0
    for (c, p, n, s0, pid) in pts:
        e, _ = L.sample_noise(c, p, 9, pid, s0, n)
        e0[row:row + n, :e.shape[1]] = e
        row += n
    got = L.Batch(ctx, pts, prm, e_final=True)
    got.run(9, e0=e0.view(-1))
    torch.cuda.synchronize()
    assert np.array_equal(got.records(), ref.records())
    assert np.array_equal(got.finals(), ref.finals())
    assert np.array_equal(got.tallies().view(np.int64), ref.tallies().view(np.int64))
    # (c) the same through host buffers
    hb = L.HostBatch(ctx, pts, prm)
    hb.e0.copy_(e0.view(-1).cpu())
    hb.run(9)
    assert np.array_equal(hb.records(), ref.records())
    assert np.array_equal(hb.finals(), ref.finals())
    assert np.array_equal(hb.tallies().view(np.int64), ref.tallies().view(np.int64))
    hb.run(9, with_e0=False)  # noise sampled on the device
    assert np.array_equal(hb.records(), ref.records())
    # (b) hand-made errors against the oracle's run from the same errors
    rng = np.random.default_rng(4)
    n = code.n
    bits = np.zeros((6, n), dtype=np.uint8)
    bits[0, 17] = 1
    bits[1, np.nonzero(code.logicals[0])[0][:5]] = 1
    bits[2] = rng.integers(0, 2, n)
    bits[3] = (rng.random(n) < 0.15)
    bits[4, :] = 1
    pts1 = [(lc, 0.0, 6, 0, 7)]
    b1 = L.Batch(ctx, pts1, prm, e_final=True)
    b1.run(13, e0=torch.from_numpy(_pack_rows(bits, b1.words).view(np.int32).reshape(-1)).cuda())
    torch.cuda.synchronize()
    rec = b1.records()
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    for i in range(6):
        r = O.run_shot(oc, op, 0.0, 13, 7, i, e0=bits[i])
        for f in ("t_clr", "converged", "failed", "moves", "ticks", "sweeps"):
            assert rec[i][f] == r[f], (i, f, rec[i][f], r[f])


@pytest.mark.parametrize("maker,prec,q,qs,variant,gauge,dt", [
    (lambda: I.toric2d(6), "f32", 0.05, 0, "cta", 0, 0.1),
    (lambda: I.toric2d(6), "f32", 0.05, 0, "warp", 1, 0.1),
    (lambda: I.toric3d_membrane(4), "i16", 0.125, 2 ** -6, "cta", 0, 0.1),
    (lambda: I.toric3d_membrane(3), "i16", 0.125, 2 ** -6, "warp", 0, 0.01),
    (lambda: I.bb_code(6, 6), "i8", 0.05, 0.25, "warp", 0, 0.1),
    (lambda: I.bb_code(12, 6), "f16", 0.05, 0, "cta", 0, 0.1),
])
def test_multi_qubit_move_trajectories(L, ctx, maker, prec, q, qs, variant, gauge, dt):
    """The multi-qubit LocalMove (most probable odd-weight subset of N(c)),
    shot by shot against the oracle: fused and relaxed sweeps, both team
    variants, the one-thread path of the gauge switch."""
    budget = 200 if dt == 0.1 else 2000
    prm = L.params(feedback="check_move_multi", precision=prec, quant_scale=qs or 2 ** -6, q=q,
                   dt_tick=dt, tick_budget=budget, variant=variant, gauge_on_move=gauge)
    _batch_vs_oracle(L, ctx, maker(), prm, 0.08, 96, finals=(dt == 0.1))


def test_graph_replay_from_given_errors(L, ctx):
    """lim_graph_create_from: a graph captured over a device error buffer, replayed
    after refilling the buffer, equals lim_run_batch_from on the same errors."""
    code = I.toric2d(6)
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", tick_budget=64)
    pts = [(lc, 0.0, 48, 0, 2)]
    g = L.Batch(ctx, pts, prm, e_final=True)
    buf = torch.zeros(g.nshots * g.words, dtype=torch.int32, device="cuda")
    g.capture(e0=buf)
    rng = np.random.default_rng(8)
    for trial in range(2):
        bits = (rng.random((g.nshots, code.n)) < 0.08 + 0.04 * trial).astype(np.uint8)
        host = torch.from_numpy(_pack_rows(bits, g.words).view(np.int32).reshape(-1))
        buf.copy_(host.cuda())
        g.replay(5, 0)
        torch.cuda.synchronize()
        ref = L.Batch(ctx, pts, prm, e_final=True)
        ref.run(5, e0=host.cuda())
        torch.cuda.synchronize()
        assert np.array_equal(g.records(), ref.records()), trial
        assert np.array_equal(g.finals(), ref.finals()), trial


def test_discrete_machine_on_a_quantum_code(L, ctx):
    prm = L.params(feedback="bit_discrete", precision="f32", tick_budget=60, tau=0, dt_tick=0)
    _batch_vs_oracle(L, ctx, I.toric2d(6), prm, 0.04, 100)


def test_mixed_batch_and_launch_shape_invariance(L, ctx):
    """Mixed codes, sizes and p in one launch; results equal per-point runs and do
    not depend on block shape (randomness is keyed by (seed, point, shot))."""
    codes = [I.bb_code(6, 6), I.bb_code(15, 3), I.bb_code(12, 6)]
    lcs = [ctx.from_inputs(c) for c in codes]
    prm = L.params(precision="i8", quant_scale=0.25, tick_budget=300)
    pts = []
    pid = 0
    for lc in lcs:
        for p in (0.02, 0.05, 0.08):
            pts.append((lc, p, 40, 7, pid))
            pid += 1
    tal, rec = L.run_batch(ctx, pts, prm, 3)
    off = 0
    for (lc, p, n, s0, pid_), code in zip(pts, [c for c in codes for _ in range(3)]):
        ora = oracle_point(code, prm, p, 3, pid_, s0, n)
        compare_records(rec[off:off + n], ora, f"{code.name} p={p}")
        off += n
    for variant, bt in (("cta", 128), ("cta", 192), ("warp", 64), ("warp", 512)):
        prm2 = L.params(precision="i8", quant_scale=0.25, tick_budget=300, variant=variant,
                        block_threads=bt)
        _, rec2 = L.run_batch(ctx, pts, prm2, 3)
        assert np.array_equal(rec2, rec), (variant, bt)


def test_trace_matches_oracle_every_tick(L, ctx):
    code = I.toric2d(6)
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", tick_budget=80)
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm)
    for shot in range(6):
        eh, sh, rec = L.trace(ctx, lc, prm, 0.07, 4, 1, shot, 80)
        r = O.run_shot(oc, op, 0.07, 4, 1, shot, trace_ticks=80)
        assert np.array_equal(_unpack(eh, code.n), r["trace"]["e_hist"]), shot
        assert np.array_equal(_unpack(sh, code.m), r["trace"]["s_hist"]), shot
        assert rec["t_clr"] == r["t_clr"]


def test_edge_cases(L, ctx):
    code = I.toric2d(8)
    lc = ctx.from_inputs(code)
    prm = L.params(precision="f32", tick_budget=32)
    tal, rec = L.run_batch(ctx, [(lc, 0.0, 20, 0, 0), (lc, 1.0, 5, 0, 1), (lc, 0.05, 0, 0, 2)], prm, 1)
    assert np.all(rec["t_clr"] == 0) and np.all(rec["moves"] == 0)
    assert np.all(rec["failed"][:20] == 0)
    assert np.all(rec["failed"][20:] == 0)  # all-ones on even L: winds an even number of times
    assert tal[2]["shots"] == 0
    # zero budget: every shot with a nonzero syndrome is a non-convergent failure
    prm0 = L.params(precision="f32", tick_budget=0)
    tal, rec = L.run_batch(ctx, [(lc, 0.1, 50, 0, 0)], prm0, 1)
    ora = oracle_point(code, prm0, 0.1, 1, 0, 0, 50)
    compare_records(rec, ora, "T=0")
    # odd L: all-ones residual is a logical failure
    code5 = I.toric2d(5)
    tal, rec = L.run_batch(ctx, [(ctx.from_inputs(code5), 1.0, 3, 0, 0)], prm, 1)
    assert np.all(rec["failed"] == 1) and np.all(rec["t_clr"] == 0)


def _irregular_code(seed, n=40, m=30):
    """A random irregular check matrix with check degrees 1..8 and qubit degrees
    at most 8 (the library's limits), no Z checks: the X-logicals are a basis of
    the vectors modulo row(H_X)."""
    rng = np.random.default_rng(seed)
    deg = np.zeros(n, dtype=int)
    rows = []
    for c in range(m):
        w = int(rng.integers(1, 9))
        free = [v for v in rng.permutation(n) if deg[v] < 8][:w]
        for v in free:
            deg[v] += 1
        rows.append(sorted(int(v) for v in free))
    rows[0] = rows[0][:1]   # keep at least one degree-1 check
    return I.code_from_rows(f"irregular{seed}", n, rows, [])


def test_maximum_sizes_and_irregular_codes(L, ctx):
    """One launch at the library's limits -- LIM_MAX_CODES codes (families and
    irregular codes with check degrees 1..8, qubit degrees up to 8) and
    LIM_MAX_POINTS points -- equals the oracle shot by shot; one code or one
    point more is refused."""
    codes = [I.toric2d(5), I.toric2d(6), I.toric3d_point(3), I.toric3d_membrane(3), I.bb_code(6, 6),
             I.rep_code(17), I.rep_code(12, periodic=True)] + [_irregular_code(s) for s in range(9)]
    assert len(codes) == L.LIM_MAX_CODES
    dc = max(int(np.diff(c.hx_ptr).max()) for c in codes)
    dv = max(int(np.bincount(c.hx_col, minlength=c.n).max()) for c in codes)
    assert dc == 8 and dv == 8
    lcs = [ctx.from_inputs(c) for c in codes]
    prm = L.params(precision="f32", tick_budget=40)
    pts = [(lcs[i % 16], 0.02 + 0.01 * (i % 7), 2, 3 * i, i) for i in range(L.LIM_MAX_POINTS)]
    tal, rec = L.run_batch(ctx, pts, prm, 21)
    assert int(tal["errors"].sum()) == 0
    row = 0
    for (lc, p, n, s0, pid) in pts:
        ora = oracle_point(codes[pid % 16], prm, p, 21, pid, s0, n)
        compare_records(rec[row:row + n], ora, f"point {pid}")
        row += n
    with pytest.raises(L.LimError):
        L.run_batch(ctx, pts + [pts[0][:4] + (999,)], prm, 21)
    with pytest.raises(L.LimError):
        L.run_batch(ctx, [(c, 0.05, 1, 0, i) for i, c in enumerate(lcs + [ctx.from_inputs(I.toric2d(4))])],
                    prm, 21)


def test_ler_f32_agrees_with_fp64_oracle(L, ctx):
    code = I.toric2d(8)
    prm = L.params(precision="f32", tick_budget=32)
    _, rec = L.run_batch(ctx, [(ctx.from_inputs(code), 0.05, 1000, 0, 0)], prm, 0)
    ora = oracle_point(code, prm, 0.05, 0, 0, 0, 1000, precision="f64")
    ok, bc = paired_ok(rec["failed"], ora["failed"])
    assert ok, bc


@pytest.mark.parametrize("prec", ["f32", "f16", "bf16"])
def test_sumproduct_ler_agrees_with_fp64_oracle(L, ctx, prec):
    code = I.toric2d(8)
    prm = L.params(precision=prec, rule="sumproduct", tick_budget=64)
    _, rec = L.run_batch(ctx, [(ctx.from_inputs(code), 0.06, 600, 0, 0)], prm, 2)
    ora = oracle_point(code, prm, 0.06, 2, 0, 0, 600, precision="f64")
    ok, bc = paired_ok(rec["failed"], ora["failed"])
    assert ok, bc


# storage unit roundoff of each format (round to nearest: half an ulp, relative)
UNIT_ROUNDOFF = {"f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.mark.parametrize("cname", ["toric2d_6", "bb_6_6", "point_3"])
@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("relaxed", [False, True])
def test_sumproduct_sweeps_reduced_precision(L, ctx, cname, prec, relaxed):
    """Sum-product with 16-bit storage against FP64 on the same stored inputs: each
    output is the FP64 value up to one rounding to the storage format (relative u)
    plus the binary32 arithmetic before it (1e-5 max(1, |m|))."""
    code = CODES[cname]()
    lc = ctx.from_inputs(code)
    prm = L.params(precision=prec, rule="sumproduct", clamp=40.0, tau=0.1,
                   dt_tick=0.03 if relaxed else 0.1)
    rng = np.random.default_rng(17)
    B = 6
    s, cv, vc = _random_state(rng, code, prec, B, 4.0)
    cvo, vco = L.bp_sweeps(lc, prm, torch.from_numpy(s).cuda(), _to_dev(L, prm, cv), _to_dev(L, prm, vc), 1)
    cvo = cvo.double().cpu().numpy()
    vco = vco.double().cpu().numpy()
    oc = O.OracleCode.from_code(code)
    op = oracle_params(prm, precision="f64")
    u = UNIT_ROUNDOFF[prec]
    for b in range(B):
        rc, rv = O.bp_sweeps(oc, op, s[b], cv[b], vc[b], 1)
        for got, ref in ((cvo[b], rc), (vco[b], rv)):
            tol = u * np.abs(ref) + 1e-5 * np.maximum(1.0, np.abs(ref))
            assert np.all(np.abs(got - ref) <= tol), (b, np.max(np.abs(got - ref) - tol))
        # and the oracle's own 16-bit mode (FP64 value rounded once) agrees to one ulp
        rc16, _ = O.bp_sweeps(oc, oracle_params(prm), s[b], cv[b], vc[b], 1)
        assert np.all(np.abs(cvo[b] - rc16) <= 2 * u * np.abs(rc16) + 1e-6), b


@pytest.mark.parametrize("L_,p,shots", [(128, 0.02, 3), (128, 0.12, 1), (64, 0.08, 3)])
def test_full_size_toric2d_sampled(L, ctx, L_, p, shots):
    """Full-size 2D toric shots (global-memory arena) in the benchmark's launch
    configuration, against the oracle shot by shot."""
    code = I.toric2d(L_)
    prm = L.params(precision="f32", tick_budget=40 * L_, variant="cta")
    _batch_vs_oracle(L, ctx, code, prm, p, shots, seed=0, point_id=5, shot0=1000, finals=False)


@pytest.mark.parametrize("rule,fb", [("minsum", "check_move"), ("minsum", "bit_discrete"),
                                     ("sumproduct", "check_move"), ("minsum", "check_move_multi")])
def test_plain_path_equals_batched_kernel(L, ctx, rule, fb):
    """The plain baseline (one launch per tick, host-polled termination, HBM
    state) computes the same trajectories as the persistent kernel."""
    c6, c8 = ctx.from_inputs(I.toric2d(6)), ctx.from_inputs(I.toric2d(8))
    pts = [(c6, 0.05, 50, 0, 0, 60), (c8, 0.07, 30, 5, 1, 40)]
    kw = dict(precision="f32", rule=rule, feedback=fb, tick_budget=60)
    tal_b, rec_b = L.run_batch(ctx, pts, L.params(**kw), 9)
    tal_p, rec_p = L.run_batch(ctx, pts, L.params(variant="plain", **kw), 9)
    assert np.array_equal(rec_p, rec_b)
    assert np.array_equal(tal_p, tal_b)
    if rule == "minsum":
        ora = oracle_point(I.toric2d(6), L.params(**kw), 0.05, 9, 0, 0, 50)
        compare_records(rec_p[:50], ora, "plain")


@pytest.mark.parametrize("variant", ["auto", "cta", "warp", "lane"])
def test_graph_replay_equals_run_batch(L, ctx, variant):
    """A batch captured as a CUDA graph and replayed with new seeds and shot
    windows gives exactly the results of direct lim_run_batch calls, for every
    launch kind (the lane kernel's per-code queues included)."""
    c8 = ctx.from_inputs(I.toric2d(8))
    bb = ctx.from_inputs(I.bb_code(6, 6))
    prm = L.params(precision="f32", tick_budget=40, variant=variant)
    pts = [(c8, 0.05, 64, 10, 0), (bb, 0.04, 64, 10, 1)]
    b = L.Batch(ctx, pts, prm)
    b.capture()
    for seed, off in ((3, 0), (4, 500)):
        b.replay(seed, off)
        torch.cuda.synchronize()
        shifted = [(c, p, n, s0 + off, pid) for c, p, n, s0, pid in pts]
        tal, rec = L.run_batch(ctx, shifted, prm, seed)
        assert np.array_equal(b.records(), rec)
        assert np.array_equal(b.tallies(), tal)


def test_autotuner_picks_a_working_shape(L, ctx):
    c16 = ctx.from_inputs(I.toric2d(16))
    bb = ctx.from_inputs(I.bb_code(12, 6))
    prm = L.params(precision="f32", tick_budget=64)
    pts = [(c16, 0.06, 32, 0, 0), (bb, 0.04, 32, 0, 1)]
    best, rate = L.autotune(ctx, pts, prm, sample_shots=8, sample_ticks=32)
    assert rate > 0 and best.variant in (1, 2)
    _, rec_a = L.run_batch(ctx, pts, prm, 5)
    _, rec_b = L.run_batch(ctx, pts, best, 5)
    assert np.array_equal(rec_a, rec_b)  # the shape never changes results


def test_misaligned_workspace_is_refused(L, ctx):
    """A workspace that is not 256-byte aligned is refused (LIM_E_INVAL) before
    anything is launched; the same buffer at its aligned start runs."""
    import ctypes
    code = ctx.from_inputs(I.toric2d(8))
    prm = L.params(precision="f32", tick_budget=8)
    pts = [(code, 0.05, 4, 0, 0)]
    arr = L._points(pts)
    ws_bytes = L.workspace_size(ctx, pts, prm)
    buf = torch.empty(ws_bytes + 512, dtype=torch.uint8, device="cuda")
    assert buf.data_ptr() % 256 == 0
    tally = torch.zeros(L.TALLY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for off in (16, 128):
        st = L.lib().lim_run_batch(ctx.handle, arr, 1, ctypes.byref(prm), 1, buf.data_ptr() + off,
                                   ws_bytes, None, None, tally.data_ptr(), None)
        assert L.STATUS[st] == "LIM_E_INVAL", st
        assert "aligned" in L.lib().lim_last_error().decode()
    st = L.lib().lim_run_batch(ctx.handle, arr, 1, ctypes.byref(prm), 1, buf.data_ptr(), ws_bytes,
                               None, None, tally.data_ptr(), None)
    assert st == 0
    torch.cuda.synchronize()
    t = np.frombuffer(tally.cpu().numpy().tobytes(), dtype=L.TALLY_DTYPE)
    assert int(t["shots"][0]) == 4 and int(t["errors"][0]) == 0
