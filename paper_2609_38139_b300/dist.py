"""Multi-process runs of the batched simulation: shot sharding, tally merge,
checkpoint and resume.

Shots are independent and their randomness is keyed by (seed, point, shot),
so ranks run disjoint shot ids of every point and the only exchange is a sum
of integer tallies at the end (no collective on the data path).  Integer sums
make a sharded or resumed run bit-identical to an uninterrupted single-GPU
run of the same shot ids.

A *runner* is any callable ``runner(points) -> tallies`` taking the point
tuples ``(code, p, shots, shot0, point_id[, tick_budget])`` used by
``lim.run_batch`` and returning one tally record per point (``lim.TALLY_DTYPE``);
``gpu_runner`` wraps the CUDA library.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, List, Sequence

import numpy as np

from . import lim

TALLY_DTYPE = lim.TALLY_DTYPE


def shard(points: Sequence, rank: int, world: int, mode: str = "weak") -> List[tuple]:
    """This rank's part of a point list.

    ``weak``: every rank runs ``shots`` shots of every point, rank r taking the
    window starting at ``shot0 + r * shots`` (total work grows with the world).
    ``strong``: every point's ``shots`` are split into contiguous ranges."""
    out = []
    for pt in points:
        code, p, shots, shot0, pid = pt[:5]
        rest = tuple(pt[5:])
        if mode == "weak":
            out.append((code, p, shots, shot0 + rank * shots, pid) + rest)
        elif mode == "strong":
            lo = shots * rank // world
            hi = shots * (rank + 1) // world
            out.append((code, p, hi - lo, shot0 + lo, pid) + rest)
        else:
            raise ValueError(mode)
    return out


def merge_tallies(tally: np.ndarray, group=None) -> np.ndarray:
    """Sum per-point tallies over all ranks of the default (or given) process
    group; every field is an int64 counter, so the sum is exact."""
    import torch
    import torch.distributed as dist
    flat = np.ascontiguousarray(tally).view(np.int64).copy()
    backend = dist.get_backend(group)
    t = torch.from_numpy(flat)
    if backend == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().view(TALLY_DTYPE).copy()


def config_hash(points: Sequence, prm_fields: dict, seed: int) -> str:
    """Identifies a run so that a checkpoint is only resumed by the same run."""
    desc = {"seed": int(seed), "params": {k: prm_fields[k] for k in sorted(prm_fields)},
            "points": [[str(getattr(pt[0], "name", pt[0])), float(pt[1]), int(pt[2]), int(pt[3]),
                        int(pt[4])] + [int(x) for x in pt[5:]] for pt in points]}
    return hashlib.sha256(json.dumps(desc, sort_keys=True).encode()).hexdigest()


def save_checkpoint(path: str, run_hash: str, next_batch: int, tally: np.ndarray) -> None:
    """Atomic JSON checkpoint: run identity, next batch index, integer tallies."""
    state = {"hash": run_hash, "next_batch": int(next_batch),
             "tally": np.ascontiguousarray(tally).view(np.int64).tolist()}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(state, f)
    os.replace(tmp, path)


def load_checkpoint(path: str, run_hash: str, npts: int):
    """(next_batch, tally) of a matching checkpoint, else (0, zeros)."""
    zero = np.zeros(npts, dtype=TALLY_DTYPE)
    if not os.path.exists(path):
        return 0, zero
    state = json.load(open(path))
    if state.get("hash") != run_hash:
        raise ValueError(f"checkpoint {path} belongs to another run")
    tally = np.array(state["tally"], dtype=np.int64).view(TALLY_DTYPE)
    return int(state["next_batch"]), tally.reshape(npts).copy()


def run_resumable(runner: Callable, points: Sequence, batch_shots: int, nbatches: int,
                  ckpt_path: str, run_hash: str, stop_after: int = -1) -> np.ndarray:
    """Run ``nbatches`` windows of ``batch_shots`` shots of every point, batch b
    covering shots ``shot0 + b*batch_shots ...``, saving a checkpoint after each
    batch; a rerun with the same arguments resumes after the last saved batch.
    ``stop_after`` >= 0 stops after that many batches of this call (for tests).
    Returns the accumulated tallies."""
    b0, total = load_checkpoint(ckpt_path, run_hash, len(points))
    done = 0
    for b in range(b0, nbatches):
        if 0 <= stop_after <= done:
            break
        window = [(pt[0], pt[1], batch_shots, pt[3] + b * batch_shots, pt[4]) + tuple(pt[5:])
                  for pt in points]
        t = runner(window)
        acc = total.view(np.int64) + np.ascontiguousarray(t).view(np.int64)
        total = acc.view(TALLY_DTYPE).copy()
        save_checkpoint(ckpt_path, run_hash, b + 1, total)
        done += 1
    return total


def gpu_runner(ctx, prm, seed: int) -> Callable:
    """A runner on the CUDA library (lim.run_batch, synchronous)."""
    def run(points):
        tal, _ = lim.run_batch(ctx, points, prm, seed)
        return tal
    return run


def run_until(runner: Callable, points: Sequence, batch_shots: int, max_shots: int,
              max_failures: int) -> np.ndarray:
    """Monte Carlo estimate per point with the stopping rule of the paper's
    numerics: keep adding batches of ``batch_shots`` fresh shots to a point until
    it has ``max_shots`` shots or ``max_failures`` logical failures, whichever
    comes first (Sec. S4: 500,000 shots or 100 logical errors).  Points still
    running are batched together.  Returns the per-point tallies."""
    total = np.zeros(len(points), dtype=TALLY_DTYPE)
    done = np.zeros(len(points), dtype=bool)
    b = 0
    while not done.all():
        idx = [i for i in range(len(points)) if not done[i]]
        window = []
        for i in idx:
            pt = points[i]
            n = min(batch_shots, max_shots - int(total[i]["shots"]))
            window.append((pt[0], pt[1], n, pt[3] + b * batch_shots, pt[4]) + tuple(pt[5:]))
        t = runner(window)
        for j, i in enumerate(idx):
            acc = total[i:i + 1].view(np.int64) + t[j:j + 1].view(np.int64)
            total[i] = acc.view(TALLY_DTYPE)[0]
            done[i] = total[i]["shots"] >= max_shots or total[i]["failures"] >= max_failures
        b += 1
    return total
