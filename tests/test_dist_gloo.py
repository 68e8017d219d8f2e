"""Multi-process host logic on CPU (gloo, world size 2): sharded runs merge to
the single-process result exactly, checkpoints resume exactly, and a rank
that dies before the merge is detected by the survivor (no GPU involved;
the shot runner here is the CPU oracle)."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_2609_38139_b300 import dist as D
from paper_2609_38139_b300 import inputs as I
from paper_2609_38139_b300.lim import TALLY_DTYPE

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _tally_from_records(recs, E):
    t = np.zeros(1, dtype=TALLY_DTYPE)[0]
    t["shots"] = len(recs)
    t["failures"] = int(recs["failed"].sum())
    t["nonconverged"] = int((recs["converged"] == 0).sum())
    conv = recs["converged"] == 1
    t["sum_t"] = int(recs["t_clr"][conv].sum())
    t["sum_t2"] = int((recs["t_clr"][conv].astype(np.int64) ** 2).sum())
    for x in recs["t_clr"][conv]:
        b = 0 if x <= 0 else min(int(x).bit_length(), 23)
        t["hist"][b] += 1
    t["moves"] = int(recs["moves"].sum())
    t["ticks"] = int(recs["ticks"].sum())
    t["sweeps"] = int(recs["sweeps"].sum())
    t["msg_updates"] = int(recs["sweeps"].sum()) * 2 * E
    return t


class _Code:
    def __init__(self, code):
        self.code, self.oc, self.name = code, O.OracleCode.from_code(code), code.name


def oracle_runner(seed):
    prm = O.params(precision="f32", tick_budget=24)

    def run(points):
        out = np.zeros(len(points), dtype=TALLY_DTYPE)
        for i, (c, p, n, s0, pid) in enumerate(points):
            recs = O.run_shots(c.oc, prm, p, seed, pid, s0, n)
            out[i] = _tally_from_records(recs, c.code.E)
        return out
    return run


def _points():
    return [(_Code(I.toric2d(4)), 0.06, 24, 0, 0), (_Code(I.bb_code(6, 6)), 0.04, 16, 100, 1)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, mode, outdir, fail_rank):
    import datetime

    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    pts = _points()
    mine = D.shard(pts, rank, world, mode)
    t = oracle_runner(7)(mine)
    if rank == fail_rank:
        os._exit(3)  # dies without joining the merge
    try:
        merged = D.merge_tallies(t)
        np.save(os.path.join(outdir, f"merged{rank}.npy"), merged.view(np.int64))
    except Exception as e:  # the survivor of a dead rank lands here
        open(os.path.join(outdir, f"error{rank}.txt"), "w").write(repr(e))
    dist.destroy_process_group() if fail_rank < 0 else None


def _spawn(mode, tmp_path, fail_rank=-1):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, str(tmp_path), fail_rank))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        if p.is_alive():
            p.kill()
    return procs


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_sharded_merge_equals_single_process(tmp_path, mode):
    _spawn(mode, tmp_path)
    pts = _points()
    if mode == "weak":  # rank r ran the window shot0 + r*shots
        ref = sum(oracle_runner(7)(D.shard(pts, r, 2, "weak")).view(np.int64) for r in range(2))
    else:               # the two ranges together are the original points
        ref = oracle_runner(7)(pts).view(np.int64)
    for r in range(2):
        got = np.load(os.path.join(tmp_path, f"merged{r}.npy"))
        assert np.array_equal(got, ref.reshape(got.shape))


def test_dead_rank_is_detected(tmp_path):
    _spawn("weak", tmp_path, fail_rank=1)
    assert os.path.exists(os.path.join(tmp_path, "error0.txt"))
    assert not os.path.exists(os.path.join(tmp_path, "merged0.npy"))


def test_checkpoint_resume_is_exact(tmp_path):
    pts = _points()
    run = oracle_runner(11)
    h = D.config_hash(pts, {"precision": "f32", "T": 24}, 11)
    full = D.run_resumable(run, pts, 6, 4, str(tmp_path / "full.json"), h)
    ck = str(tmp_path / "part.json")
    part = D.run_resumable(run, pts, 6, 4, ck, h, stop_after=2)   # "crash" after 2 batches
    assert part["shots"].tolist() == [12, 12]
    resumed = D.run_resumable(run, pts, 6, 4, ck, h)                # resume
    assert np.array_equal(resumed.view(np.int64), full.view(np.int64))
    with pytest.raises(ValueError):
        D.load_checkpoint(ck, "other-run", len(pts))


def test_adaptive_stopping_rule():
    """Sec. S4: a point stops at max_shots shots or max_failures failures."""
    pts = [(_Code(I.toric2d(4)), 0.2, 0, 0, 0), (_Code(I.toric2d(4)), 0.01, 0, 0, 1)]
    tot = D.run_until(oracle_runner(3), pts, batch_shots=16, max_shots=96, max_failures=10)
    hi, lo = tot[0], tot[1]
    assert hi["failures"] >= 10 and hi["shots"] < 96 and hi["shots"] % 16 == 0
    assert lo["shots"] == 96 and lo["failures"] < 10


def test_strong_shards_cover_every_shot_once():
    """Strong scaling splits each point's shots into contiguous, disjoint ranges
    that cover all shot ids, also when shots < ranks or do not divide evenly."""
    pts = [("c", 0.1, 7, 100, 0), ("c", 0.2, 2, 0, 1), ("c", 0.3, 0, 5, 2)]
    for world in (1, 2, 3, 4):
        for i, (_, _, shots, shot0, _) in enumerate(pts):
            ids = []
            for r in range(world):
                _, _, n, s0, _ = D.shard(pts, r, world, "strong")[i]
                ids.extend(range(s0, s0 + n))
            assert sorted(ids) == list(range(shot0, shot0 + shots)), (world, i)
    with pytest.raises(ValueError):
        D.shard(pts, 0, 2, "diagonal")


def test_config_hash_identifies_the_run():
    pts = _points()
    h = D.config_hash(pts, {"precision": "f32", "T": 24}, 11)
    assert h == D.config_hash(pts, {"T": 24, "precision": "f32"}, 11)    # key order irrelevant
    assert h != D.config_hash(pts, {"precision": "f16", "T": 24}, 11)
    assert h != D.config_hash(pts, {"precision": "f32", "T": 24}, 12)
    moved = [pts[0][:3] + (pts[0][3] + 1,) + pts[0][4:]] + pts[1:]
    assert h != D.config_hash(moved, {"precision": "f32", "T": 24}, 11)
