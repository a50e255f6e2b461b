"""The multi-rank logic of bench.py on CPU: two gloo ranks, each a replica
with its own step time and counts; times combine by max, counts by sum, and
the reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = bench.Ranks(dist, "cpu")
    r.barrier()
    q.put((rank, r.max(10.0 + rank), r.sum(1000.0 * (rank + 1))))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_by_max_and_counts_by_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 11.0, 3000.0), (1, 11.0, 3000.0)]


def test_single_process_ranks_are_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(None, "cpu")
    r.barrier()
    assert r.max(2.5) == 2.5 and r.sum(7) == 7.0


@pytest.mark.parametrize("rank", ["0", "1"])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=rank, WORLD_SIZE="2", LOCAL_RANK=rank)
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--ref-seconds", "0.5", "--workload", "uniform_small"],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    if rank == "1":
        assert lines == []
    else:
        line = json.loads(lines[-1])
        assert line["impl"] == "reference" and line["unit"] == "interactions/s" and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_result_lines_append_to_a_jsonl_log(tmp_path):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    path = tmp_path / "runs" / "bench.jsonl"
    for k in range(2):
        bench.emit({"metric": "m", "value": float(k)}, argparse.Namespace(jsonl=str(path)))
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    assert rows == [{"metric": "m", "value": 0.0}, {"metric": "m", "value": 1.0}]
    bench.emit({"metric": "m"}, argparse.Namespace(jsonl=""))   # no log: stdout only
