#!/usr/bin/env python3
"""Benchmark of the batched inference-machine simulation on B300.

Workload (default): the batched 2D toric sweep -- L in {16, 32, 64, 128}, 11
error rates p in 0.02..0.12, FP32 min-sum, check-centric feedback, one BP
sweep per tick (dt = tau = 0.1), tick budget 40L, all points mixed in one
persistent launch.  One step = one persistent launch over ``--shots`` fresh
shots of every point (a sample of the configuration's 10^5 per point), run to
completion: the batch is captured once as a CUDA graph (lim_graph_create) and
each step replays it on its own window of shot ids (lim_graph_launch).

Prints one JSON line.  ``value`` is shot-ticks per second of the main arm
(ticks executed, summed over shots, divided by the device time of the steps).
Alongside: msg-updates/s; the roofline of the batch kernel per memory class
(codes whose messages live in shared memory against the shared-memory copy
bandwidth measured in this run, codes whose messages live in global memory
against the measured HBM copy bandwidth) with the measured DRAM traffic;
``lowprec``: the same shots with 16-bit storage (f16, i16); ``vs_plain``: the
plain FP32 per-shot path (one launch per tick, host-polled termination) on the
shots of step 0, with every arm's failures on those shots paired against it;
the oracle's CPU rate; the end-to-end rate through the public API (host
buffers, copies inside the timed region); the SM clocks seen during the timed
regions and the number of our kernel launches.

``--impl reference`` times the CPU oracle (the plain reference implementation)
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2609_38139_b300 import inputs as I  # noqa: E402

METRIC = "shot-ticks/s & msg-updates/s vs HBM/SMEM roofline; batched+lowprec vs plain at equal P_L"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
# the launch shape is tuned on a whole step when a step has at most this many shots;
# a larger step is tuned on that many of its shots, each cut at TUNE_TICKS ticks (the
# rare shots that run a long budget would otherwise decide the sample's time)
TUNE_MAX_SHOTS = 40000
TUNE_TICKS = 256


def workload(name: str, shots: int, sizes=None, ps=None):
    """Points of a named workload; ``sizes``/``ps`` restrict it (profiling runs)."""
    w = I.WORKLOADS[name]
    pts = []
    for fam, size, p, pid in I.workload_points(name):
        if sizes and str(size) not in sizes:
            continue
        if ps and not any(abs(p - float(x)) < 1e-9 for x in ps):
            continue
        pts.append(dict(family=fam, size=size, p=p, point_id=pid, shots=shots,
                        T=I.tick_budget(w["budget"], size, w["dt_tick"])))
    # most expensive points first: the queue hands out work in this order
    pts.sort(key=lambda d: (-I.make_code(d["family"], d["size"]).E * d["T"], -d["p"]))
    return w, pts


def lib_params(L, w, name, prec, variant="auto"):
    qs = L.default_quant_scale(prec, w["q"])
    return L.params(rule=w.get("rule", "minsum"), feedback=w.get("feedback", "check_move"),
                    precision=prec, quant_scale=qs,
                    q=w["q"], clamp=w["clamp"], tau=w["tau"],
                    dt_tick=w["dt_tick"], sweeps_per_tick=w["K"], tick_budget=w.get("T", 0) or 1,
                    variant=variant, tie_rel=L.default_tie_rel(prec, w.get("rule", "minsum")))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip() == "Active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the CUDA sources: a traffic figure measured on other sources is stale."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_38139_b300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")) +
                    glob.glob(os.path.join(csrc, "*.h"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, prec: str, algorithmic_bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary of this workload, scaled
    to this run's launches by their algorithmic bytes; None if the summary was
    taken on other kernel sources or another workload."""
    f = os.path.join(ROOT, "profiles", f"batch_kernel__{workload}__{prec}__dram.json")
    try:
        d = json.load(open(f))
    except Exception:
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d["dram_bytes"] * algorithmic_bytes_per_launch / d["algorithmic_bytes"]


def peak_hbm():
    try:
        d = json.load(open(PEAKS_FILE))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _default_quant_scale(prec: str, q: float) -> float:
    from paper_2609_38139_b300 import lim
    return lim.default_quant_scale(prec, q)


def _default_tie_rel(prec: str, rule: str) -> float:
    from paper_2609_38139_b300 import lim
    return lim.default_tie_rel(prec, rule)


def cpu_baseline(name: str, prec: str, seconds: float = 15.0, threads: int = 0, rule: str = "",
                 sweeps: int = 0, feedback: str = ""):
    """The oracle timed on this host's cores on a bounded sample of the workload:
    shots of every point in turn (same keyed shot ids as the GPU's step 0) until
    about ``seconds`` of wall time have passed."""
    import oracle as O
    from concurrent.futures import ThreadPoolExecutor
    w, pts = workload(name, 1)
    if rule:
        w = dict(w, rule=rule)
    if sweeps > 0:
        w = dict(w, K=sweeps)
    if feedback:
        w = dict(w, feedback=feedback)
    threads = threads or (os.cpu_count() or 1)
    codes = {}
    t0 = time.perf_counter()
    ticks = 0
    shots = 0
    upd = 0
    jobs = []
    for d in sorted(pts, key=lambda d: d["point_id"]):
        key = (d["family"], d["size"])
        if key not in codes:
            c = I.make_code(*key)
            codes[key] = (c, O.OracleCode.from_code(c))
        jobs.append(d)
    # one shot per point per round, all points, over `threads` threads
    rnd = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < seconds:
            futs = []
            for d in jobs:
                c, oc = codes[(d["family"], d["size"])]
                op = O.params(precision=prec if prec in ("f32", "f16", "bf16", "i16", "i8") else "f64",
                              rule=w.get("rule", "minsum"), feedback=w.get("feedback", "check_move"),
                              quant_scale=_default_quant_scale(prec, w["q"]),
                              q=w["q"], clamp=w["clamp"], tau=w["tau"],
                              dt_tick=w["dt_tick"], sweeps_per_tick=w["K"], tick_budget=d["T"],
                              tie_rel=_default_tie_rel(prec, w.get("rule", "minsum")))
                futs.append((c, ex.submit(O.run_shots, oc, op, d["p"], 0, d["point_id"], rnd, 1)))
            for c, f in futs:
                r = f.result()
                ticks += int(r["ticks"].sum())
                upd += int(r["sweeps"].sum()) * 2 * c.E
                shots += len(r)
            rnd += 1
    dt = time.perf_counter() - t0
    return {"value": ticks / dt, "unit": "shot-ticks/s", "cores": threads, "kind": "oracle",
            "msg_updates_per_s": upd / dt,
            "sample": f"{shots} shots ({rnd} per point, every point of the workload, same shot ids "
                      f"as the GPU's first step), {prec} oracle, {dt:.1f} s wall"}


def arm_config(args, w, npoints: int) -> dict:
    """The workload as both arms describe it in their JSON lines (identical for
    both; what each arm actually timed is in its ``sample`` key)."""
    return {"workload": args.workload, "codes": f"{w['family']} sizes {w['sizes']}",
            "points": npoints,
            "shots_per_point": f"timed on samples of fresh shot ids; the configuration has "
                               f"{w['shots']} per point",
            "rule": w.get("rule", "minsum"), "feedback": w.get("feedback", "check_move"),
            "tau": w["tau"], "dt_tick": w["dt_tick"], "sweeps_per_tick": w.get("K", 1),
            "tick_budget": w["budget"], "variant": args.variant,
            "l2": "flushed between steps (256 MiB write, outside the timed window)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.shots <= 0:
        args.shots = I.WORKLOADS[args.workload].get("bench_shots", 32)
    w = dict(I.WORKLOADS[args.workload])
    for key, val in (("rule", args.rule), ("feedback", args.feedback)):
        if val:
            w[key] = val
    if args.sweeps_per_tick > 0:
        w["K"] = args.sweeps_per_tick
    npts = len(I.workload_points(args.workload))
    steps = []
    # each step a bounded sample: about --ref-seconds, less when many steps are asked
    # for, so that the whole run stays within a few minutes
    per_step = min(args.ref_seconds, max(2.0, 150.0 / max(1, args.steps)))
    for _ in range(args.warmup):
        cpu_baseline(args.workload, args.precision, seconds=max(1.0, per_step / 4),
                     rule=args.rule, sweeps=args.sweeps_per_tick, feedback=args.feedback)
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(args.workload, args.precision, seconds=per_step, rule=args.rule,
                            sweeps=args.sweeps_per_tick, feedback=args.feedback)
        steps.append(last)
    wall = time.perf_counter() - t0
    val = statistics.mean(s["value"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "shot-ticks/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": dict(arm_config(args, w, npts), parallelism="host threads",
                           launch_shape="oracle, shots of every point in turn"),
            "sample": f"each step: {last['sample']}",
            "cpu_baseline": {"value": val, "unit": "shot-ticks/s", "cores": last["cores"],
                             "kind": "oracle", "sample": last["sample"]},
            "e2e": {"value": val, "unit": "shot-ticks/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="toric2d_sweep")
    ap.add_argument("--precision", default="f32")
    ap.add_argument("--lowprec", default="auto",
                    help="comma list of further storage precisions timed on the same shots "
                         "(auto: f16,i16 when the main arm is f32; none: skip)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-tick FP32 path")
    ap.add_argument("--variant", default="auto")
    ap.add_argument("--shots", type=int, default=0,
                    help="shots per point per step (default: the workload's bench_shots, else 32)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--rule", default="", help="minsum | sumproduct (default: the workload's)")
    ap.add_argument("--feedback", default="",
                    help="check_move | check_move_multi | bit_discrete (default: the workload's)")
    ap.add_argument("--sweeps-per-tick", type=int, default=0,
                    help="K (default: the workload's); relaxation alpha = dt / (K tau)")
    ap.add_argument("--smem-cap", type=int, default=0, help="max shared memory per block in bytes (0 automatic, <0 all that fits)")
    ap.add_argument("--phases", action="store_true", help="report the kernel's per-phase cycle shares")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the library's default launch shape instead of the one lim_autotune picks")

    ap.add_argument("--print-source-hash", action="store_true")
    ap.add_argument("--sizes", default="", help="comma list restricting the code sizes")
    ap.add_argument("--ps", default="", help="comma list restricting the error rates")
    ap.add_argument("--tie-rel", type=float, default=-1.0,
                    help="LocalMove tie tolerance of the binary16/bfloat16 arms (default: the "
                         "library's default for the format; 0: exact ties)")
    args = ap.parse_args()
    if args.print_source_hash:
        print(kernel_source_hash())
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2609_38139_b300 import lim as L

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    ctx = L.Context(local)
    sizes = [x for x in args.sizes.split(",") if x]
    ps = [x for x in args.ps.split(",") if x]
    if args.shots <= 0:
        args.shots = I.WORKLOADS[args.workload].get("bench_shots", 32)
    w, pts = workload(args.workload, args.shots, sizes, ps)
    if args.rule:
        w = dict(w, rule=args.rule)
    if args.sweeps_per_tick > 0:
        w = dict(w, K=args.sweeps_per_tick)
    if args.feedback:
        w = dict(w, feedback=args.feedback)
    codes = {}
    for d in pts:
        key = (d["family"], d["size"])
        if key not in codes:
            codes[key] = ctx.from_inputs(I.make_code(*key))

    def make_params(prec, variant=None):
        prm = lib_params(L, w, args.workload, prec, variant or args.variant)
        prm.block_threads = args.block_threads
        prm.blocks_per_sm = args.blocks_per_sm
        prm.profile = 1 if args.phases else 0
        prm.smem_cap = args.smem_cap
        if args.tie_rel >= 0 and prec in ("f16", "bf16"):
            prm.tie_rel = args.tie_rel
        return prm

    def tuned_params(prec, variant=None):
        """The arm's parameters with the launch shape lim_autotune picks on a sample
        of this step's points (untimed); the shape never changes results."""
        prm = make_params(prec, variant)
        if args.block_threads or args.blocks_per_sm or args.smem_cap or (variant or args.variant) != "auto":
            return prm, "given"
        if args.no_autotune:
            return prm, "library default"
        if args.shots * len(pts) <= TUNE_MAX_SHOTS:
            # tuned on the step itself: every shape times the shots of step 0 to the end
            best, rate = L.autotune(ctx, step_points(0), prm, sample_shots=args.shots, sample_ticks=0)
            sample = "the shots of step 0, run to the end, once per shape (untimed)"
        else:
            # one shot per lane needs many shots per lane to pay off, which a sample
            # this size does not have: a step the library runs that way keeps it
            if L.plan_describe(ctx, step_points(0), prm)[0]["variant"] == "lane":
                return prm, "library default (one shot per lane)"
            n = max(1, TUNE_MAX_SHOTS // len(pts))
            best, rate = L.autotune(ctx, step_points(0, n), prm, sample_shots=n, sample_ticks=TUNE_TICKS)
            sample = (f"the first {n} shots of every point of step 0, each cut at {TUNE_TICKS} ticks, "
                      "once per shape (untimed)")
        best.profile = prm.profile
        return best, {"tuned_by": "lim_autotune", "variant": {v: k for k, v in L.VARIANT.items()}[int(best.variant)],
                      "block_threads": int(best.block_threads), "blocks_per_sm": int(best.blocks_per_sm),
                      "smem_cap": int(best.smem_cap), "tuning_rate_shot_ticks_per_s": rate,
                      "sample": sample}

    prm = make_params(args.precision)

    # weak scaling: every rank runs its own disjoint shot ids of every point;
    # every arm below runs the same shot ids (step i of an arm = step i of another)
    def step_points(step, shots=None):
        n = shots or args.shots
        base = (step * world + rank) * args.shots
        return [(codes[(d["family"], d["size"])], d["p"], n, base, d["point_id"], d["T"])
                for d in pts]

    prm, tuned = tuned_params(args.precision)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 126 MB L2

    def timed_arm(arm_prm):
        """W untimed and K timed steps of one storage precision: device times of the
        steps (CUDA events on the launching stream), their tallies, and the step-0
        records (for the paired comparisons).  The step's batch is captured once as
        a CUDA graph (queue reset, tally reset, the persistent kernel) and every
        step replays it on its own window of shot ids."""
        batch = L.Batch(ctx, step_points(0), arm_prm, records=True)
        batch.capture()

        def run_step(step, timed_events=None):
            flush.fill_(step & 0xFF)  # evict L2 between steps (outside the timed window)
            if timed_events:
                timed_events[0].record(stream)
            # step_points(step) = step_points(0) shifted by step * world * shots
            batch.replay(0, step * world * args.shots, stream)
            if timed_events:
                timed_events[1].record(stream)

        for i in range(args.warmup):
            run_step(args.steps + i)  # warm-up on shot ids the timed steps do not use
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        tallies, rec0 = [], None
        torch.cuda.synchronize()
        for i in range(args.steps):
            run_step(i, evs[i])
            tallies.append(batch.tally.clone())
            if i == 0:
                rec0 = batch.rec.clone()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        arrs = [np.frombuffer(t.cpu().numpy().tobytes(), dtype=L.TALLY_DTYPE) for t in tallies]
        for a in arrs:
            assert int(a["errors"].sum()) == 0, "device-side error counter set"
        recs = np.frombuffer(rec0.cpu().numpy().tobytes()[:batch.nshots * L.RECORD_DTYPE.itemsize],
                             dtype=L.RECORD_DTYPE).copy()
        return {"ms": sum(ms), "tallies": arrs, "rec0": recs, "ms_steps": ms}

    def reduce_arm(arm):
        """Whole-job totals of an arm: max of the ranks' device times, sums of work."""
        tot_ms = arm["ms"]
        ticks = sum(int(a["ticks"].sum()) for a in arm["tallies"])
        upd = sum(int(a["msg_updates"].sum()) for a in arm["tallies"])
        shots = sum(int(a["shots"].sum()) for a in arm["tallies"])
        fails = sum(int(a["failures"].sum()) for a in arm["tallies"])
        if dist:
            t = torch.tensor([tot_ms, ticks, upd, shots, fails], dtype=torch.float64, device="cuda")
            mx = t.clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            tot_ms = float(mx[0])
            ticks, upd, shots, fails = (int(x) for x in t[1:].tolist())
        return tot_ms, ticks, upd, shots, fails

    hbm, hbm_src = peak_hbm()
    smem_copy_gbs, smem_load_gbs = L.smem_bandwidth(ctx)

    def roofline(arm, prec, tot_ms, arm_prm):
        """Roofline of the batch kernel per memory class: codes whose messages live
        in shared memory against the measured shared-memory copy bandwidth, codes
        whose messages live in global memory against the measured HBM copy
        bandwidth; the class whose bytes take longer at its peak bounds the launch.
        Algorithmic bytes: 2 x b per message update (read the old message, write the
        new one)."""
        bpm = L.MSG_BYTES[prec]
        _, sm = L.plan_describe(ctx, step_points(0), arm_prm)
        # this rank's launches (the roofline is per GPU): its own tallies
        upd_pt = np.sum([a["msg_updates"] for a in arm["tallies"]], axis=0).astype(np.float64)
        b_smem = float(upd_pt[sm].sum()) * 2 * bpm
        b_glob = float(upd_pt[~sm].sum()) * 2 * bpm
        sec = tot_ms / 1000.0
        cls = {"smem": {"bytes_per_launch": b_smem / args.steps, "achieved_gbs": b_smem / sec / 1e9,
                        "peak_gbs": smem_copy_gbs, "frac": b_smem / sec / 1e9 / smem_copy_gbs,
                        "peak_source": "measured (lim_smem_bandwidth copy, this run)"},
               "global": {"bytes_per_launch": b_glob / args.steps, "achieved_gbs": b_glob / sec / 1e9,
                          "peak_gbs": hbm, "frac": b_glob / sec / 1e9 / hbm,
                          "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)"}}
        dom = "smem" if b_smem / smem_copy_gbs > b_glob / hbm else "global"
        c = cls[dom]
        # the records are of the workload's own rule, feedback and sweeps per tick
        own = not (args.rule or args.feedback or args.sweeps_per_tick > 0 or sizes or ps)
        traffic = measured_traffic(args.workload, prec, (b_smem + b_glob) / args.steps) if own else None
        out = {"bound": "smem" if dom == "smem" else "hbm", "achieved": c["achieved_gbs"],
               "peak": c["peak_gbs"], "unit": "GB/s", "frac": c["frac"], "traffic": traffic,
               "kernel": "batch_kernel (persistent)",
               "algorithmic_bytes": "2 x msg bytes per message update (read old, write new), "
                                    "of the codes in the bounding memory class",
               "peak_source": c["peak_source"], "classes": cls}
        if traffic is not None:
            out["dram_achieved_gbs"] = traffic * args.steps / sec / 1e9
            out["dram_frac"] = out["dram_achieved_gbs"] / hbm
        return out

    clocks = Clocks(local)
    main_arm = timed_arm(prm)
    tot_ms, ticks, upd, shots, fails = reduce_arm(main_arm)
    value = ticks / (tot_ms / 1000.0)
    line = {"metric": METRIC, "value": value, "unit": "shot-ticks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": dict(arm_config(args, w, len(pts)),
                           parallelism=f"replicas x{world}, disjoint shot ids",
                           launch_shape=tuned),
            "sample": f"{args.shots} fresh shot ids of every point per step "
                      f"({args.shots * len(pts)} shots per launch, one launch per step: a replay of "
                      "the batch captured once as a CUDA graph, lim_graph_launch)",
            "ms_steps": [round(x, 3) for x in main_arm["ms_steps"]],
            "msg_updates_per_s": upd / (tot_ms / 1000.0),
            "ler_sample": fails / max(1, shots),
            "roofline": roofline(main_arm, args.precision, tot_ms, prm),
            "smem_peak": {"copy_gbs": smem_copy_gbs, "load_gbs": smem_load_gbs,
                          "how": "lim_smem_bandwidth: two 1024-thread blocks per SM moving 16-byte "
                                 "words in shared memory, best of three launches"},
            "gpu_launches": args.steps}
    if args.phases:
        phase = np.sum([a["phase_cycles"].sum(axis=0) for a in main_arm["tallies"]], axis=0)
        if phase.sum() > 0:
            line["phase_share"] = {n: round(float(v / phase.sum()), 4) for n, v in zip(L.PHASES, phase)}
            line["phase_cycles_per_tick"] = float(phase.sum() / max(1, ticks))

    # the same shots in reduced-precision storage
    low = [x for x in args.lowprec.split(",") if x] if args.lowprec != "auto" else \
        (["f16", "i16"] if args.precision == "f32" else [])
    if args.lowprec == "none":
        low = []
    arms = {args.precision: main_arm}
    lowprec = {}
    for lp in low:
        lp_prm, lp_shape = tuned_params(lp)
        arm = timed_arm(lp_prm)
        arms[lp] = arm
        a_ms, a_ticks, a_upd, a_shots, a_fails = reduce_arm(arm)
        lowprec[lp] = {"value": a_ticks / (a_ms / 1000.0), "unit": "shot-ticks/s",
                       "ms_per_step": a_ms / args.steps,
                       "msg_updates_per_s": a_upd / (a_ms / 1000.0),
                       "ler_sample": a_fails / max(1, a_shots),
                       "launch_shape": lp_shape,
                       "tie_rel": float(lp_prm.tie_rel),
                       "roofline": roofline(arm, lp, a_ms, lp_prm)}
    if lowprec:
        line["lowprec"] = lowprec
    clk = clocks.stop()
    line["clocks"] = clk
    line["gpu_launches"] = args.steps * (1 + len(low))

    # the plain FP32 per-shot path (one launch per tick, host-polled termination)
    # on the shots of step 0, and every batched arm's failures on those shots
    if not args.no_plain and world == 1:
        # the plain path runs one point at a time with a host round trip per tick:
        # at most 4096 shots of every point (the first shot ids of step 0)
        pshots = min(args.shots, 4096)
        plain_prm = make_params("f32", variant="plain")
        pb = L.Batch(ctx, step_points(0, pshots), plain_prm, records=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pb.run(0, stream)
        torch.cuda.synchronize()
        p_dt = time.perf_counter() - t0
        p_tal = pb.tallies()
        p_rec = pb.records()
        sub = np.concatenate([np.arange(i * args.shots, i * args.shots + pshots) for i in range(len(pts))])
        vs = {"plain_f32": {"value": int(p_tal["ticks"].sum()) / p_dt, "unit": "shot-ticks/s",
                            "shots": int(p_tal["shots"].sum()),
                            "failures": int(p_tal["failures"].sum()),
                            "ler": float(p_tal["failures"].sum() / max(1, p_tal["shots"].sum())),
                            "timing": "wall clock of one lim_run_batch (the plain path polls the "
                                      "host every tick), on the first shot ids of every arm's step 0 "
                                      f"({pshots} per point)"}}
        for prec, arm in arms.items():
            r0 = arm["rec0"][sub]
            b = int(np.sum((r0["failed"] == 1) & (p_rec["failed"] == 0)))
            c = int(np.sum((r0["failed"] == 0) & (p_rec["failed"] == 1)))
            rate = value if prec == args.precision else lowprec[prec]["value"]
            vs[f"batched_{prec}"] = {
                "failures_same_shots": int(r0["failed"].sum()),
                "paired_vs_plain": {"gpu_only": b, "plain_only": c,
                                    "within_3_sigma": bool(abs(b - c) <= 3 * np.sqrt(b + c) + 1)},
                "identical_records": bool(np.array_equal(r0, p_rec)),
                "speedup_shot_ticks": rate / vs["plain_f32"]["value"]}
        line["vs_plain"] = vs

    # end to end through the public API: lim_run_batch_host, one blocking call per
    # step with host buffers -- the step's initial errors are copied in from
    # page-locked host memory, the records, final residuals and tallies are
    # copied back.  The errors are the library's own samples for those shot ids
    # (lim_sample_noise, drawn before the timed region), so the work per step is
    # the same as in the device-timed steps.
    if not args.no_e2e:
        hb = L.HostBatch(ctx, [pt[:3] + (0,) + tuple(pt[4:]) for pt in step_points(0)], prm)
        e2e_steps = []
        for i in range(args.steps):
            off = (i * world + rank) * args.shots
            buf = torch.zeros(hb.nshots * hb.words, dtype=torch.int32, pin_memory=True)
            view = buf.view(hb.nshots, hb.words)
            row = 0
            for pt in hb.points:
                c, p, n, s0, pid = pt[:5]
                e, _ = L.sample_noise(c, p, 0, pid, s0 + off, n)
                view[row:row + n, :e.shape[1]].copy_(e.cpu())
                row += n
            e2e_steps.append((off, buf))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e_ticks = 0
        for off, buf in e2e_steps:
            hb.set_shot_offset(off)
            hb.run(0, e0=buf, stream=stream)
            e_ticks += int(hb.tallies()["ticks"].sum())
        e_dt = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([e_dt], dtype=torch.float64, device=torch.device("cuda", local))
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e_dt = float(tt.item())
            tk = torch.tensor([e_ticks], dtype=torch.float64, device=torch.device("cuda", local))
            dist.all_reduce(tk, op=dist.ReduceOp.SUM)
            e_ticks = int(tk.item())
        line["e2e"] = {"value": e_ticks / e_dt, "unit": "shot-ticks/s",
                       "h2d_bytes_per_step": hb.h2d_bytes(),
                       "d2h_bytes_per_step": hb.d2h_bytes(),
                       "note": "lim_run_batch_host per step: initial errors of the step's shots "
                               "copied in from page-locked host memory, records, final residuals "
                               "and tallies copied back, inside the timed region"}
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.precision, args.cpu_seconds,
                                            rule=args.rule, sweeps=args.sweeps_per_tick, feedback=args.feedback)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
