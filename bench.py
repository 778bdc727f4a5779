"""Benchmark: one fused registration iteration (warp + similarity fwd/bwd +
diffusion regulariser + Adam) on synthetic volumes, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c1] [--impl ours|reference]

Default workload (c1): 192^3 FP32 multimodal pair, 32-bin cubic B-spline
Parzen MI, diffusion lambda = 0.05, Adam.  A step is one iteration over the
whole volume.  Prints one JSON line (rank 0).  With N > 1 (torchrun), every
rank registers its own independent pair (replicas, weak scaling); only the
timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "warp+loss fwd+bwd Gvoxel-iter/s (full iteration incl. diffusion + Adam)"
UNIT = "Gvoxel-iter/s"
WORKLOADS = {
    "c0": "64^3 FP32 mono-modal pair, LNCC 7^3, diffusion lambda 0.1, Adam (FP32 moments)",
    "c1": "192^3 FP32 multimodal phantom pair, 32-bin cubic B-spline Parzen MI, diffusion lambda 0.05, Adam (FP32 moments)",
    "c2": "512^3 BF16-stored mono-modal pair, LNCC 9^3, diffusion lambda 0.1, Adam (BF16 moments)",
    "c4": "1280^3 BF16-stored multimodal phantom pair, 32-bin Parzen MI, diffusion lambda 0.05, Adam (BF16 moments)",
}
# algorithmic bytes per voxel of one iteration (each compulsory tensor moved once)
#   sweep 1: F, M (one gather counted once), u;  LNCC also writes 3 FP32 coefficient fields
#   sweep 2: F, M, u (12 B), m, v (3 components each) read; u' (12 B), m, v written;
#            LNCC also reads the coefficient fields
def bytes_per_voxel(kind, img_bytes, mom_bytes):
    s1 = 2 * img_bytes + 12 + (12 if kind == "lncc" else 0)
    s2 = 2 * img_bytes + 12 + 12 + 2 * (2 * 3 * mom_bytes) + (12 if kind == "lncc" else 0)
    return s1, s2


def csrc_sha() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2509_25044_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def read_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (null otherwise)."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(p):
        return None
    sha = bytes_ = None
    for line in open(p):
        if line.startswith("csrc_sha:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            bytes_ = float(line.split(":", 1)[1].strip())
    return bytes_ if sha == csrc_sha() else None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def setup_dist(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): the FP64 oracle as it stands
# ---------------------------------------------------------------------------
def oracle_sample(cfg_name: str, budget_s: float = 20.0):
    """A bounded sample of the workload for the oracle: z-slabs of the same
    volume, grown until one iteration takes a few seconds."""
    import numpy as np
    from paper_2509_25044_gb300 import synth
    d = synth.make(cfg_name) if cfg_name in ("c0", "c1") else synth.make(cfg_name, n=128)
    c = d["config"]
    F, M = d["F"].double().numpy(), d["M"].double().numpy()
    u = (-0.5 * d["u_true"]).double().numpy()
    return c, F, M, u, d


def time_oracle_iteration(cfg_name: str, nz: int | None = None):
    import numpy as np
    import oracle as O
    c, F, M, u, d = oracle_sample(cfg_name)
    if nz is not None:
        F, M, u = F[:nz].copy(), M[:nz].copy(), u[:, :nz].copy()
    if c["kind"] == "lncc":
        spec = O.LossSpec(kind=O.LOSS_LNCC, window=c["window"], eps=1e-9)
    else:
        spec = O.LossSpec(kind=O.LOSS_MI, bins=c["bins"], f_range=d["f_range"], m_range=d["m_range"])
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    t0 = time.perf_counter()
    O.iterate(F, M, u, m, v, 1, spec, c["lam"], c["lr"], bf16_moments=(c["dtype"] == "bf16"))
    dt = time.perf_counter() - t0
    return F.size, dt


def oracle_threads():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    except ValueError:
        return os.cpu_count()


def cpu_baseline(cfg_name: str):
    n_vox, dt = time_oracle_iteration(cfg_name)
    return {"value": n_vox / dt / 1e9, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
            "sample": f"one full FP64 oracle iteration of the {cfg_name} workload ({n_vox} voxels, {dt:.1f} s)"}


def run_reference(args):
    rank, world, local = setup_dist(args.gpus)
    if rank != 0:
        return
    # each step: one FP64 oracle iteration on a z-slab sample of the same workload
    cfg = args.config
    nz = 48 if cfg == "c1" else None
    for _ in range(args.warmup):
        time_oracle_iteration(cfg, nz)
    tot_vox, tot_t = 0, 0.0
    for _ in range(args.steps):
        n, dt = time_oracle_iteration(cfg, nz)
        tot_vox += n
        tot_t += dt
    value = tot_vox / tot_t / 1e9
    sample = f"z-slab of {nz} planes of the {cfg} volume per step" if nz else f"full {cfg} volume per step"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOADS[cfg], "name": cfg},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = setup_dist(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2509_25044_gb300 import build, capi, synth
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    capi.load()

    cfg = synth.CONFIGS[args.config]
    kind = cfg["kind"]
    bf16 = cfg["dtype"] == "bf16"
    d = synth.make(args.config, device=dev, seed=cfg["seed"] + 1000 * rank, n=args.n)
    F = d["F"].to(torch.bfloat16 if bf16 else torch.float32).contiguous()
    M = d["M"].to(torch.bfloat16 if bf16 else torch.float32).contiguous()
    shape = tuple(F.shape)
    N = F.numel()
    del d["u_true"]
    if kind == "lncc":
        loss = capi.lncc_desc(cfg["window"], 1e-9, ants=args.lncc_grad == "ants")
    else:
        loss = capi.mi_desc(d["f_range"], d["m_range"], cfg["bins"], hard=args.mi_estimator == "hard")
    mdt = capi.REG_BF16 if bf16 else capi.REG_F32
    mtype = torch.bfloat16 if bf16 else torch.float32
    u = [torch.zeros((3,) + shape, device=dev), torch.zeros((3,) + shape, device=dev)]
    m = torch.zeros((3,) + shape, dtype=mtype, device=dev)
    v = torch.zeros((3,) + shape, dtype=mtype, device=dev)
    ws = capi.workspace(loss, F)
    obj = torch.zeros(2, dtype=torch.float64, device=dev)
    adam = capi.adam_desc(cfg["lr"], moment_dtype=mdt, grad_scale=float(N))
    lam = cfg["lam"]
    stream = torch.cuda.current_stream(dev)

    step_no = [0]

    def step():
        step_no[0] += 1
        a, b = u[(step_no[0] - 1) % 2], u[step_no[0] % 2]
        capi.reg_iterate(loss, F, M, a, b, m, v, lam, adam, step_no[0], ws, obj=obj)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if capi.reg_get_device_error() != 0:
        raise RuntimeError("device error during warm-up")

    # ---- timed region: K iterations, per-sweep events on every iteration ----
    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for trip in evs:  # torch creates the CUDA event on its first record
        for e in trip:
            e.record(stream)
    start.record(stream)
    end.record(stream)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    start.record(stream)
    for k in range(K):
        capi.reg_set_timing_events(evs[k])
        step()
    end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    ms_max = max_over_ranks(ms, world, dev)
    s1 = [e[0].elapsed_time(e[1]) for e in evs]
    s2 = [e[1].elapsed_time(e[2]) for e in evs]
    err = capi.reg_get_device_error()
    objv = obj.cpu().tolist()

    # ---- end to end: host (pinned) images in, objective out, every step ----
    # Every step copies its own F and M from pinned host memory and reads its
    # objective back.  The copies run on their own stream into two device
    # buffers, so step k + 1's inputs arrive while step k computes; events
    # order each copy after the compute that last read its buffer, and each
    # compute after its inputs' copy.
    Fh = F.cpu().pin_memory()
    Mh = M.cpu().pin_memory()
    objh = torch.zeros(2, dtype=torch.float64).pin_memory()
    Fd2 = [torch.empty_like(F), torch.empty_like(F)]
    Md2 = [torch.empty_like(M), torch.empty_like(M)]
    cstream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ke = max(1, min(K, 200))
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    cstream.wait_event(e0)

    def h2d(k):
        i = k % 2
        with torch.cuda.stream(cstream):
            if k >= 2:
                cstream.wait_event(consumed[i])
            Fd2[i].copy_(Fh, non_blocking=True)
            Md2[i].copy_(Mh, non_blocking=True)
            copied[i].record(cstream)

    h2d(0)
    for k in range(Ke):
        if k + 1 < Ke:
            h2d(k + 1)
        i = k % 2
        stream.wait_event(copied[i])
        step_no[0] += 1
        a, b = u[(step_no[0] - 1) % 2], u[step_no[0] % 2]
        capi.reg_iterate(loss, Fd2[i], Md2[i], a, b, m, v, lam, adam, step_no[0], ws, obj=obj)
        consumed[i].record(stream)
        objh.copy_(obj, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)

    if rank != 0:
        return
    value = world * N * K / (ms_max * 1e-3) / 1e9
    e2e_value = world * N * Ke / (e2e_ms * 1e-3) / 1e9
    ib = 2 if bf16 else 4  # images and Adam moments share the storage type in every workload
    b1, b2 = bytes_per_voxel(kind, ib, ib)
    peak, peak_kind = read_peaks()
    t2 = statistics.median(s2)
    t1 = statistics.median(s1)
    ach2 = b2 * N / (sum(s2) / K * 1e-3) / 1e9
    ach1 = b1 * N / (sum(s1) / K * 1e-3) / 1e9
    dom = "sweep2" if t2 >= t1 else "sweep1"
    kname = {("mi", "sweep2"): "mi_sweep2", ("mi", "sweep1"): "mi_hist", ("lncc", "sweep2"): "lncc_sweep2",
             ("lncc", "sweep1"): "lncc_stats"}[(kind, dom)]
    if kind == "lncc" and args.lncc_grad == "ants" and dom == "sweep2":
        kname = "lncc_sweep2_ants"
    ach = ach2 if dom == "sweep2" else ach1
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32" if bf16 else "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + (", ANTs gradient approximation"
                                                         if kind == "lncc" and args.lncc_grad == "ants" else "")
                   + (", hard-binned histogram" if kind == "mi" and args.mi_estimator == "hard" else ""),
                   "name": args.config, "n": shape[0],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs larger than L2 (working set {(b1 + b2) * N / 1e9:.2f} GB/iteration > 129 MB)"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_voxel": b2 if dom == "sweep2" else b1,
                     "traffic": read_traffic(kname, args.config)},
        "sweeps_ms": {"sweep1_median": t1, "sweep2_median": t2,
                      "sweep1_GBps": ach1, "sweep2_GBps": ach2,
                      "iteration_GBps": (b1 + b2) * N / (ms_max / K * 1e-3) / 1e9},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * N * ib, "d2h_bytes_per_step": 16,
                "note": "per step: pinned host F, M -> device (a copy stream, two device buffers: "
                        "step k+1's copy overlaps step k's compute), one iteration, objective -> host"},
        "gpu_launches": 3 * K,  # MI: histogram, finalize, sweep 2; LNCC: warp, window statistics, sweep 2
        "clocks": clk,
        "objective_last": objv, "device_error": err, "wall_s": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.config)
    if not args.no_unet:
        out["tensor_core"] = unet_tensor_core(dev, read_bf16_peak())
    print(json.dumps(out), flush=True)


def read_bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    return 1900.0, "fallback 1.9 PFLOP/s"


def unet_tensor_core(dev, peak):
    """The learned initialiser's forward pass at a 128^3 input (the only
    tensor-core work): 13 tcgen05 convolutions plus pooling / upsampling.
    Timed with CUDA events after the registration run (outside its timed
    region); FLOPs are the convolutions' algorithmic 2 * 27 * Cin * Cout per
    output voxel with the real channel counts (2 input channels, 3 output)."""
    import torch
    from paper_2509_25044_gb300 import capi
    from paper_2509_25044_gb300.unet import LAYERS, UNet
    n = 128
    net = UNet(n_in=n, seed=0, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    F = torch.rand((n, n, n), generator=g, device=dev)
    M = torch.rand((n, n, n), generator=g, device=dev)
    net.pack(F, M, 1, (0.0, 1.0), (0.0, 1.0))
    real = {"c0a": (2, 16), "head": (32, 3)}
    flops = sum(2.0 * 27 * real.get(nm, (ci, co))[0] * real.get(nm, (ci, co))[1] * net.V[lv]
                for nm, ci, co, lv in LAYERS)
    for _ in range(3):
        net.forward()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        net.forward()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # the largest convolution alone (d1a: 96 -> 32 channels at 64^3)
    nm, ci, co, lv = [l for l in LAYERS if l[0] == "d1a"][0]
    src = torch.zeros((net.V[lv], ci), dtype=torch.bfloat16, device=dev)
    dst = torch.empty((net.V[lv], co), dtype=torch.bfloat16, device=dev)
    for _ in range(3):
        net._conv(nm, src, dst, lv)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        net._conv(nm, src, dst, lv)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_k = e0.elapsed_time(e1) / reps
    fl_k = 2.0 * 27 * ci * co * net.V[lv]
    tf_k = fl_k / (ms_k * 1e-3) / 1e12
    return {"workload": "U-Net initialiser forward, 128^3 x 2-channel input, BF16 x BF16 -> FP32 (tcgen05)",
            "ms_forward": ms, "tflops_forward": flops / (ms * 1e-3) / 1e12, "gflop_forward": flops / 1e9,
            "kernel": "conv_view_kernel (d1a, 96 -> 32 channels, 64^3)", "kernel_ms": ms_k,
            "roofline": {"bound": "tensor", "achieved": tf_k, "peak": peak[0], "unit": "TFLOP/s",
                         "frac": tf_k / peak[0], "peak_source": peak[1]},
            "device_error": capi.reg_get_device_error()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default="c1", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=None, help="override the grid size (profiling runs)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-unet", action="store_true", help="skip the tensor-core (U-Net) measurement")
    ap.add_argument("--lncc-grad", default="exact", choices=["exact", "ants"],
                    help="LNCC gradient: exact adjoint or the ANTs approximation (no second box sum)")
    ap.add_argument("--mi-estimator", default="parzen", choices=["parzen", "hard"],
                    help="MI histogram: cubic B-spline Parzen estimate or the hard-binned approximation")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
