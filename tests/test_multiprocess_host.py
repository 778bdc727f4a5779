"""The N > 1 host path of bench.py on CPU: two gloo ranks (one process per
GPU on a real node) rendezvous on 127.0.0.1, the timing reduction takes the
maximum over ranks, every rank registers its own seeded pair (replicas: no
data-path collective), and the reference arm leaves every rank but 0
without work."""
import argparse
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), BENCH_BACKEND="gloo")
    import bench
    from paper_2509_25044_gb300 import synth
    try:
        r, w, local = bench.setup_dist(world)
        assert (r, w, local) == (rank, world, rank)
        bench.barrier(w)
        # the step time reported by rank 0 is the slowest rank's
        assert bench.max_over_ranks(1.5 + rank, w, "cpu") == 1.5 + world - 1
        # replicas: each rank draws its own pair (seed + 1000 * rank) at the workload's recipe
        d = synth.make("c0", n=16, seed=synth.CONFIGS["c0"]["seed"] + 1000 * rank)
        sig = torch.tensor([float(d["F"].double().sum()), float(d["M"].double().sum())], dtype=torch.float64)
        sigs = [torch.zeros(2, dtype=torch.float64) for _ in range(w)]
        dist.all_gather(sigs, sig)
        distinct = len({tuple(t.tolist()) for t in sigs}) == w
        # the reference arm: only rank 0 runs the oracle and prints
        out = None
        if rank != 0:
            args = argparse.Namespace(gpus=w, steps=1, warmup=0, config="c0", n=None, impl="reference",
                                      no_cpu_baseline=False)
            out = bench.run_reference(args)
        bench.barrier(w)
        q.put((rank, distinct, out, None))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, False, None, repr(e)))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_gloo_ranks_bench_host_path():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    for rank, distinct, out, err in res:
        assert err is None, (rank, err)
        assert distinct, rank
        assert out is None
    assert all(p.exitcode == 0 for p in procs)


def test_reference_arm_json_contract():
    """bench.py --impl reference prints one JSON line with the contract's keys:
    the oracle timed on the host's cores, its cpu_baseline and an e2e object
    with zero transfer bytes."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("metric", "value", "unit", "impl", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["d2h_bytes_per_step"] == 0
    assert out["e2e"]["value"] == out["value"] and "workload" in out["config"]
