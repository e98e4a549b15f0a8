"""Multi-process plumbing of bench.py on CPU: gloo ranks, world size 2.

bench.py times each rank and reports the maximum over ranks; under torchrun the
reference arm runs on rank 0 only and the other ranks exit without work."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(world)
    m = bench.max_over_ranks(float(10 + rank), world)
    q.put((rank, m))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29000 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    port = str(30000 + os.getpid() % 1000)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", port, os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "cfg1", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "Gop/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_shard_rows_partition():
    """sr_shard_rows: disjoint, in rank order, covering [0, R), whole groups of `align`
    rows, sizes within one group of each other."""
    from paper_1705_08743_gb300 import _capi as sr
    for R in (0, 1, 127, 128, 129, 1000, 4096, 8193):
        for world in (1, 2, 3, 4, 8):
            for align in (1, 64, 128):
                rr = [sr.sr_shard_rows(R, world, r, align) for r in range(world)]
                assert rr[0][0] == 0 and rr[-1][1] == R
                for (a0, a1), (b0, b1) in zip(rr, rr[1:]):
                    assert a1 == b0 and a0 <= a1
                groups = [-(-(a1 - a0) // align) for a0, a1 in rr]
                assert max(groups) - min(groups) <= 1
                assert all(a0 % align == 0 or a0 == R for a0, _ in rr)      # empty ranges sit at R
    with pytest.raises(sr.SemiringError):
        sr.sr_shard_rows(10, 2, 2)


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_1705_08743_gb300 import shard
    S = 255
    R, K, N = 300, 77, 130
    A = torch.from_numpy(oracle.encode_antidist(synth.weighted_graph(R, K, 0.2, 1, 60, 7, 0), S).astype(np.uint8))
    Bfull = oracle.encode_antidist(synth.weighted_graph(K, N, 0.2, 1, 60, 7, 3), S).astype(np.uint8)
    B = torch.from_numpy(Bfull) if rank == 0 else torch.zeros((K, N), dtype=torch.uint8)   # B only on rank 0

    calls = []

    def local_mul(A_rows, B_, C_rows):          # stands in for the GPU call of this rank
        calls.append(A_rows.shape[0])
        C_rows.copy_(torch.from_numpy(oracle.mul(A_rows.numpy(), B_.numpy(), S)))

    C = shard.sharded_mul(local_mul, A, B, rank, world, align=64)
    q.put((rank, C.numpy().tobytes(), calls))
    dist.destroy_process_group()


def test_sharded_product_gloo_world2():
    """A product split by row blocks over two gloo ranks (B broadcast from rank 0, each
    rank's rows multiplied locally, the blocks gathered) equals the oracle's product."""
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31000 + os.getpid() % 1000
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {r: (c, calls) for r, c, calls in (q.get(timeout=180) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    S = 255
    A = oracle.encode_antidist(synth.weighted_graph(300, 77, 0.2, 1, 60, 7, 0), S).astype(np.uint8)
    B = oracle.encode_antidist(synth.weighted_graph(77, 130, 0.2, 1, 60, 7, 3), S).astype(np.uint8)
    want = oracle.mul(A, B, S).astype(np.uint8)
    for r in (0, 1):
        got = np.frombuffer(res[r][0], dtype=np.uint8).reshape(300, 130)
        assert np.array_equal(got, want)
    assert res[0][1] == [192] and res[1][1] == [108]       # rows 0..191 and 192..299 (64-row groups)
