"""Host logic of the N-rank bench on CPU: world_size-2 process groups over gloo.

The solver path does not shard (one GPU solves one problem; N GPUs run N
replicas), so the only cross-rank steps are the barriers around the timed
region and the maximum of the per-rank times.  Both are exercised here
without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_0810_0330_gb300 import inputs as I
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        got = bench.max_over_ranks(values[rank], dist, torch.device("cpu"))
        # every replica builds the same workload from the same seeds
        U = I.random_su3_links((2, 2, 2, 2), 0.3, seed=0)
        eta = I.point_sources((2, 2, 2, 2), 12)
        h = float(np.abs(U).sum() + np.abs(eta).sum() * 1e-3 + U[0, 0, 0, 0].real)
        hs = [None] * world
        dist.all_gather_object(hs, h)
        dist.barrier()
        out_q.put((rank, got, hs))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [3.25, 7.5]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, hs in res:
        assert got == max(values), (rank, got)
        assert hs[0] == hs[1]


def _replica_that_may_die(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import time
    import bench
    d = bench.init_replicas("gloo", timeout_s=10)
    if rank == 1:
        os._exit(3)   # a replica that is gone between steps, without a word
    t0 = time.time()
    try:
        bench.replicas_barrier(d, "test")
        out_q.put((rank, "passed", time.time() - t0))
    except RuntimeError as e:
        out_q.put((rank, str(e), time.time() - t0))
    out_q.close()
    out_q.join_thread()
    os._exit(0)


def test_dead_replica_ends_the_next_barrier_with_an_error():
    """Failure detection on the host: when one replica exits, the others'
    next barrier raises (peer gone, or the process group's timeout) instead
    of waiting forever."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_that_may_die, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, msg, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and msg != "passed", msg
    assert "rank 0" in msg and "another rank" in msg, msg
    assert waited < 60.0, waited
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0


def test_max_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.5, None, None) == 1.5


def test_reference_arm_nonzero_rank_exits_without_work():
    """Under torchrun only rank 0 runs the oracle and prints; other ranks exit 0 silently."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_bench_json_contract_keys():
    """The JSON line's reference-arm fields are complete (the line is built from a tiny fake timing)."""
    sys.path.insert(0, ROOT)
    import bench
    obj = bench.cpu_obj(1.234, dict(threads=4, seed_iters=10, cg_iters=[3, 4]))
    assert obj["kind"] == "oracle" and obj["unit"] == "ms" and obj["cores"] == 4
    assert "not a sample" in obj["sample"] and "4 threads" in obj["sample"]
    assert obj["host"]["logical_cores"] >= 1
    assert json.loads(json.dumps(obj))["value"] == 1234.0
