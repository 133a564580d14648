"""The benchmark's multi-rank path on CPU with world size 2 over gloo.

Each rank steps its own packing (seed offset by rank, same size: weak
scaling); the only cross-rank traffic is the max over ranks of the times and
the sum over ranks of the work, and rank 0 alone prints the JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_body(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    import torch.distributed as dist
    args = argparse.Namespace(impl="ours", workload="dense_biaxial_discs_2d", n=300, max_sweeps=50, alpha=1e-6)
    r, w, local = bench.dist_init(args, backend="gloo")
    assert (r, w, local) == (rank, ws, rank)
    wl = bench.workload(args, r)
    # per-rank times and work: rank r took (1 + r) ms and did 10 (r + 1) updates
    (t_max,), (work,) = bench.reduce_max_sum([1.0 + r], [10.0 * (r + 1)], w, "cpu")
    bench.barrier(w)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), x=wl.x, n=wl.n, seed=wl.seed, t_max=t_max, work=work)
    dist.destroy_process_group()


def test_ranks_own_packings_and_reduce_max_and_sum(tmp_path):
    ws = 2
    mp.start_processes(_rank_body, args=(ws, free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    # weak scaling: the same size of packing on every rank, a different seed
    assert int(r0["n"]) == int(r1["n"]) == 300
    assert int(r0["seed"]) != int(r1["seed"])
    assert not np.array_equal(r0["x"], r1["x"])
    for r in (r0, r1):
        assert float(r["t_max"]) == 2.0
        assert float(r["work"]) == 30.0


SHARD_BATCH = dict(seed=1108, n_packings=7, nmin=60, nmax=160)


def _oracle_updates(batch, steps=2):
    """Contact updates (sweeps x contacts) of `steps` oracle steps of every
    packing, each solved alone (the batched system gives each packing its
    stand-alone result)."""
    import oracle as O
    from oracle_adapter import system
    total = 0
    for wl in batch:
        s = system(wl, criterion=O.CRIT_GLOBAL_REL, alpha=1e-6, max_sweeps=200, order=O.ORDER_COLOUR)
        for _ in range(steps):
            st = s.step()
            total += st["sweeps"] * s.nc
    return total


def _shard_body(rank, ws, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import argparse
    import bench
    import torch.distributed as dist
    from paper_1104_3516_gb300 import workloads as W
    args = argparse.Namespace(impl="ours")
    r, w, _ = bench.dist_init(args, backend="gloo")
    shard = W.batched_settling(shard=(r, w), **SHARD_BATCH)
    lo, hi = W.shard_range(SHARD_BATCH["n_packings"], r, w)
    upd = _oracle_updates(shard)
    (t_max,), (work,) = bench.reduce_max_sum([float(r)], [float(upd)], w, "cpu")
    bench.barrier(w)
    np.savez(os.path.join(out_dir, f"shard{r}.npz"), lo=lo, hi=hi, n=[b.n for b in shard],
             x=np.concatenate([b.x.reshape(-1) for b in shard]), mu=[b.mu for b in shard], work=work)
    dist.destroy_process_group()


def test_batch_shards_are_a_disjoint_cover_and_the_work_sums(tmp_path):
    """Two ranks split a small seeded batch: rank r builds exactly the
    packings a single process builds at the indices of its range, the ranges
    are disjoint and cover the batch, and the contact updates summed over the
    ranks (the benchmark's only cross-rank reduction) equal the single
    process's count."""
    from paper_1104_3516_gb300 import workloads as W
    ws = 2
    mp.start_processes(_shard_body, args=(ws, free_port(), str(tmp_path)), nprocs=ws, join=True,
                       start_method="spawn")
    full = W.batched_settling(**SHARD_BATCH)
    got = [np.load(tmp_path / f"shard{r}.npz") for r in range(ws)]
    assert [(int(g["lo"]), int(g["hi"])) for g in got] == [(0, 3), (3, 7)]
    for g in got:
        lo, hi = int(g["lo"]), int(g["hi"])
        assert list(g["n"]) == [b.n for b in full[lo:hi]]
        assert list(g["mu"]) == [b.mu for b in full[lo:hi]]
        assert np.array_equal(g["x"], np.concatenate([b.x.reshape(-1) for b in full[lo:hi]]))
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    single = _oracle_updates(full)
    assert float(got[0]["work"]) == float(got[1]["work"]) == float(single)


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--n-discs", "400", "--cpu-sweeps", "5"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["n_gpus"] == 2
    assert d["scaling"] == "weak"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
