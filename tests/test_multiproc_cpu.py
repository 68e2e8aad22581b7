"""The N > 1 path of bench.py on CPU: world size 2 over gloo.

Every rank assembles its own replica of the workload (no data-path
collective); the only cross-rank steps are the barrier around the timed
region and the max over ranks of the step time.  These run here with the
gloo backend; the GPU work of each rank is the single-GPU path tested
elsewhere.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, lr = bench.dist_setup()
    assert (w, r, lr) == (world, rank, rank)
    bench.barrier(w)
    m = bench.allreduce_max(float(rank + 1) * 1.5, w)
    bench.barrier(w)
    q.put((rank, m))
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    if torch.cuda.is_available():
        pytest.skip("exercises the gloo path of a CPU-only host")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 3.0), (1, 3.0)]


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` under torchrun: rank 0 prints one JSON line,
    the other rank exits 0 without work."""
    pytest.importorskip("torch")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "3",
           "--ref-sample", "20000", "--workload", "cube8"]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "elements/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_batch_meshes_sharded_over_ranks():
    """The batched workload splits its independent meshes over the ranks:
    each mesh on exactly one rank, element counts balanced within the largest
    mesh (longest-first greedy), one rank = the whole batch."""
    sys.path.insert(0, ROOT)
    import bench

    sizes = [6 * int(n) ** 3 for n in np.random.default_rng(3).integers(10, 61, size=64)]
    for world in (1, 2, 3, 4, 8):
        parts = bench.shard_meshes(sizes, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert bench.shard_meshes(sizes, 1) == [list(range(64))]
