"""The N > 1 launch of bench.py on CPU: two ranks over gloo on 127.0.0.1 run the
host-side replica logic (rank discovery, barrier, max of the per-rank step times,
the whole-job value world x units / max time) and only rank 0 of the reference arm
does any work or prints.  Replicas share nothing else: the path does not shard."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_setup()
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slower replica
    bench.barrier(w)
    worst = bench.max_over_ranks(ms, w)
    units = 1_000_000                       # per-rank work of one step
    q.put((r, w, local, worst, w * units / (worst * 1e-3)))
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_replica():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 2, 0), (1, 2, 1)]
    assert all(o[3] == 15.0 for o in out)                 # max over ranks, seen by both
    assert out[0][4] == pytest.approx(2 * 1_000_000 / 15e-3)


@pytest.mark.parametrize("workload", ["torus1m", "density", "isosurface"])
def test_reference_arm_only_rank0_prints(workload):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--workload", workload], env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "sphere1500", "--steps", "1", "--warmup", "0", "--ref-rows", "200"], env=env,
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["unit"] == "pair-evals/s"
