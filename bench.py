"""Benchmark: one fused registration iteration (warp + similarity fwd/bwd +
diffusion regulariser + Adam) on synthetic volumes, through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c4] [--impl ours|reference]

Default workload (c4): 1280^3 (2.1 G voxels) BF16-stored multimodal pair,
32-bin cubic B-spline Parzen MI, diffusion lambda = 0.05, Adam with BF16
moments -- the largest workload that fits one GPU.  A step is one iteration
over the whole volume.  The 192^3 MI (c1) and 512^3 LNCC (c2) workloads are
timed after it as sub-records, each with its own roofline, and the BF16
storage form is compared with plain FP32 on time to solution (c2).  Prints
one JSON line (rank 0).  With N > 1 (torchrun), every rank registers its own
independent pair (replicas, weak scaling); only the timing is reduced across
ranks.
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
_SAMPLES = {}


def oracle_sample(cfg_name: str):
    """The oracle's bounded sample of a workload: the workload itself for the
    192^3 and 64^3 ones; for the 512^3 and 1280^3 ones the same recipe at
    128^3 (the FP64 oracle would need 15 GB / 235 GB for them).  Generated
    once per process."""
    if cfg_name not in _SAMPLES:
        from paper_2509_25044_gb300 import synth
        d = synth.make(cfg_name) if cfg_name in ("c0", "c1") else synth.make(cfg_name, n=128)
        F, M = d["F"].double().numpy(), d["M"].double().numpy()
        u = (-0.5 * d["u_true"]).double().numpy()
        _SAMPLES[cfg_name] = (d["config"], F, M, u, d)
    c, F, M, u, d = _SAMPLES[cfg_name]
    return c, F, M, u.copy(), d


def sample_name(cfg_name: str) -> str:
    return f"the {cfg_name} workload" if cfg_name in ("c0", "c1") else f"the {cfg_name} recipe at 128^3"


def time_oracle_iteration(cfg_name: str, nz: int | None = None, reps: int = 1):
    """(voxels per iteration, seconds per iteration) of the FP64 oracle."""
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
    for _ in range(reps):
        O.iterate(F, M, u, m, v, 1, spec, c["lam"], c["lr"], bf16_moments=(c["dtype"] == "bf16"))
    dt = (time.perf_counter() - t0) / reps
    return F.size, dt


def oracle_threads():
    try:
        return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    except ValueError:
        return os.cpu_count()


def cpu_baseline(cfg_name: str):
    """The FP64 oracle as it stands on the host cores: all of them (this
    process), and one (a child process started with OMP_NUM_THREADS=1, since
    OpenMP fixes its thread count when the library loads)."""
    n_vox, dt = time_oracle_iteration(cfg_name, reps=3)
    rec = {"value": n_vox / dt / 1e9, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
           "sample": f"three full FP64 oracle iterations of {sample_name(cfg_name)} ({n_vox} voxels, "
                     f"{dt:.2f} s each)"}
    env = dict(os.environ, OMP_NUM_THREADS="1")
    code = ("import json, bench; n, dt = bench.time_oracle_iteration(%r); print(json.dumps([n, dt]))" % cfg_name)
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        n1, dt1 = json.loads(r.stdout.strip().splitlines()[-1])
        rec["single_thread"] = {"value": n1 / dt1 / 1e9, "unit": UNIT, "cores": 1,
                                "sample": f"one FP64 oracle iteration of {sample_name(cfg_name)} "
                                          f"({n1} voxels, {dt1:.2f} s)"}
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        rec["single_thread"] = {"value": None, "error": str(e)[:200]}
    return rec


def run_reference(args):
    rank, world, local = setup_dist(args.gpus)
    if rank != 0:
        return
    # each step: one FP64 oracle iteration on the bounded sample of the workload
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
    sample = (f"z-slab of {nz} planes of the {cfg} volume per step" if nz else
              f"{sample_name(cfg)} per step")
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
def alg_bytes(kind: str, bf16: bool):
    """Algorithmic bytes per voxel, each compulsory tensor moved once (images
    and Adam moments share the storage type in every workload):
      MI, two sweeps (the joint histogram is global): sweep 1 reads F, M, u;
        sweep 2 reads F, M, u, m, v and writes u', m, v -> 20 + 80 (FP32),
        16 + 52 (BF16);
      LNCC, one iteration: F, M, u, m, v read, u', m, v written -> 80 (FP32),
        52 (BF16); intermediates the library keeps between its own kernels
        are not counted."""
    ib = 2 if bf16 else 4
    step = 2 * ib + 12 + 12 + 2 * (2 * 3 * ib)
    if kind == "mi":
        return 2 * ib + 12, step
    return None, step


def measure(name, K, W, dev, rank, world, n=None, e2e=False, lncc_grad="exact", mi_estimator="parzen"):
    """K timed iterations (after W untimed ones) of workload `name` in one
    reg_run call (the library's multi-iteration entry point), with CUDA events
    around each iteration's sweeps; with e2e, a second pass through
    reg_iterate with the inputs copied from pinned host memory every step and
    the result read back."""
    import torch
    from paper_2509_25044_gb300 import capi, synth
    cfg = synth.CONFIGS[name]
    kind = cfg["kind"]
    bf16 = cfg["dtype"] == "bf16"
    d = synth.make(name, device=dev, seed=cfg["seed"] + 1000 * rank, n=n)
    F = d["F"].to(torch.bfloat16 if bf16 else torch.float32).contiguous()
    M = d["M"].to(torch.bfloat16 if bf16 else torch.float32).contiguous()
    f_range, m_range = d.get("f_range"), d.get("m_range")
    del d
    shape = tuple(F.shape)
    N = F.numel()
    if kind == "lncc":
        loss = capi.lncc_desc(cfg["window"], 1e-9, ants=lncc_grad == "ants")
    else:
        loss = capi.mi_desc(f_range, m_range, cfg["bins"], hard=mi_estimator == "hard")
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
    cur, t = [0], [0]  # u[cur] holds the current iterate; t iterations done
    hist = torch.zeros((max(K, W, 1), 2), dtype=torch.float64, device=dev)

    def run(iters):
        capi.reg_run(loss, F, M, u[cur[0]], u[1 - cur[0]], m, v, lam, adam, t[0], iters, ws, obj_hist=hist[:iters])
        t[0] += iters
        cur[0] = (cur[0] + iters) % 2

    def step(Fd=F, Md=M):
        t[0] += 1
        a, b = u[cur[0]], u[1 - cur[0]]
        capi.reg_iterate(loss, Fd, Md, a, b, m, v, lam, adam, t[0], ws, obj=obj)
        cur[0] = 1 - cur[0]
        return b

    if W > 0:
        run(W)
    torch.cuda.synchronize()
    if capi.reg_get_device_error() != 0:
        raise RuntimeError(f"device error during the warm-up of {name}")

    # ---- timed region: one reg_run call of K iterations, events around each
    # iteration's sweeps ----
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3 * K)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for ev in evs:  # torch creates the CUDA event on its first record
        ev.record(stream)
    start.record(stream)
    end.record(stream)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    start.record(stream)
    capi.reg_set_timing_events(evs)
    run(K)
    end.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    ms = start.elapsed_time(end)
    ms_max = max_over_ranks(ms, world, dev)
    s1 = [evs[3 * k].elapsed_time(evs[3 * k + 1]) for k in range(K)]
    s2 = [evs[3 * k + 1].elapsed_time(evs[3 * k + 2]) for k in range(K)]
    err = capi.reg_get_device_error()
    objv = hist[K - 1].cpu().tolist()
    b1, b2 = alg_bytes(kind, bf16)
    peak, peak_kind = read_peaks()
    t1, t2 = statistics.median(s1), statistics.median(s2)
    mean1, mean2 = sum(s1) / K, sum(s2) / K
    it_ms = ms_max / K
    if kind == "mi":
        # the second sweep dominates; sweep 1 is the histogram
        kname = "mi_sweep2_tma" if (shape[2] % 8 == 0) else "mi_sweep2"
        ach = b2 * N / (mean2 * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": kname, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "algorithmic_bytes_per_voxel": b2, "traffic": read_traffic(kname, name)}
        sweeps = {"sweep1_median_ms": t1, "sweep2_median_ms": t2,
                  "sweep1_GBps": b1 * N / (mean1 * 1e-3) / 1e9, "sweep2_GBps": ach,
                  "sweep1_frac": b1 * N / (mean1 * 1e-3) / 1e9 / peak,
                  "iteration_GBps": (b1 + b2) * N / (it_ms * 1e-3) / 1e9,
                  "iteration_frac": (b1 + b2) * N / (it_ms * 1e-3) / 1e9 / peak}
    else:
        # one LNCC iteration is the unit: its kernels (warp, window statistics,
        # adjoint + step) together against the single-sweep bytes
        ach = b2 * N / (it_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": "lncc iteration (all kernels)", "achieved": ach, "peak": peak,
                "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes_per_voxel": b2,
                "traffic": None}
        sweeps = {"warp_and_statistics_median_ms": t1, "adjoint_and_step_median_ms": t2}
    roof["peak_source"] = (f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                           else "fallback 6.8 TB/s")
    out = {"name": name, "n": shape[0], "voxels": N, "steps": K, "warmup": W, "ms_per_step": it_ms,
           "value": world * N * K / (ms_max * 1e-3) / 1e9, "roofline": roof, "sweeps": sweeps, "clocks": clk,
           "objective_last": objv, "device_error": err, "wall_s": wall, "bf16": bf16, "kind": kind,
           "gpu_launches": 3 * K + (1 if kind == "lncc" else 0)}

    if e2e:
        # ---- end to end: pinned host images in, objective out every step; the
        # final field u' read back into pinned host memory at the end ----
        # The copies run on their own stream into two device buffers, so step
        # k + 1's inputs arrive while step k computes; events order each copy
        # after the compute that last read its buffer.
        Fh = F.cpu().pin_memory()
        Mh = M.cpu().pin_memory()
        objh = torch.zeros(2, dtype=torch.float64).pin_memory()
        uh = torch.empty((3,) + shape, dtype=torch.float32).pin_memory()
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
        last = None
        for k in range(Ke):
            if k + 1 < Ke:
                h2d(k + 1)
            i = k % 2
            stream.wait_event(copied[i])
            last = step(Fd2[i], Md2[i])
            consumed[i].record(stream)
            objh.copy_(obj, non_blocking=True)
        uh.copy_(last, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        ib = 2 if bf16 else 4
        out["e2e"] = {"value": world * N * Ke / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                      "h2d_bytes_per_step": 2 * N * ib, "d2h_bytes_per_step": 16 + 12 * N / Ke,
                      "steps": Ke,
                      "note": "per step: pinned host F, M -> device (a copy stream, two device buffers: step k+1's "
                              "copy overlaps step k's compute), one iteration, objective (16 B) -> pinned host; "
                              f"after the last step the field u' ({12 * N} B) -> pinned host, counted per step "
                              f"over the {Ke} steps"}
        del Fh, Mh, uh, Fd2, Md2
    return out


def time_to_solution_record(config: str, n=None, lam_scale: float = 20.0):
    """BF16 storage form vs plain FP32 on one workload: iterations and time to
    the FP32 run's progress target L <= L* + 0.01 (L0 - L*), final objective,
    fold check."""
    from paper_2509_25044_gb300 import experiments
    r = experiments.time_to_loss(config, iters=None, eval_every=10, n=n, lam_scale=lam_scale)
    keep = ("ms_per_iter", "iters_to_target", "iters_to_target_upper", "time_to_target_ms", "final",
            "final_on_fp32_images", "final_rel_to_fp32_final", "fold")
    return {"workload": f"{WORKLOADS[config]}, at {r['n']}^3, lambda {r['lam']:g}", "iters": r["iters"],
            "target": r["target"],
            "fp32": {k: r["fp32"][k] for k in keep if k in r["fp32"]},
            "bf16": {k: r["bf16"][k] for k in keep if k in r["bf16"]},
            "speedup_bf16_vs_fp32": r.get("speedup_bf16_vs_fp32")}


def run_ours(args):
    import torch
    rank, world, local = setup_dist(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2509_25044_gb300 import build, capi
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    capi.load()

    K, W = args.steps, args.warmup
    head = measure(args.config, K, W, dev, rank, world, n=args.n, e2e=True, lncc_grad=args.lncc_grad,
                   mi_estimator=args.mi_estimator)
    torch.cuda.empty_cache()
    subs = {}
    if not args.no_subs:
        for name in [c for c in args.subs.split(",") if c and c != args.config]:
            r = measure(name, min(K, 100) if name != "c2" else min(K, 30), max(3, min(W, 5)), dev, rank, world)
            subs[name] = {k: r[k] for k in ("n", "voxels", "steps", "ms_per_step", "value", "roofline", "sweeps",
                                            "clocks")}
            subs[name]["workload"] = WORKLOADS[name]
            torch.cuda.empty_cache()
    if rank != 0:
        return
    kind = head["kind"]
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32" if head["bf16"] else "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + (", ANTs gradient approximation"
                                                         if kind == "lncc" and args.lncc_grad == "ants" else "")
                   + (", hard-binned histogram" if kind == "mi" and args.mi_estimator == "hard" else ""),
                   "name": args.config, "n": head["n"], "voxels": head["voxels"],
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (the iteration streams "
                         f"{head['voxels'] * (68 if head['bf16'] else 100) / 1e9:.1f} GB > 129 MB)"},
        "roofline": head["roofline"], "sweeps": head["sweeps"], "e2e": head["e2e"],
        # MI: histogram, finalize, step; LNCC: warp, window statistics, step,
        # plus F's window statistics once per reg_run call
        "gpu_launches": head["gpu_launches"],
        "clocks": head["clocks"], "objective_last": head["objective_last"], "device_error": head["device_error"],
        "wall_s": head["wall_s"],
    }
    if subs:
        out["workloads"] = subs
    if world == 1 and not args.no_ttl:
        # the precision form's own workload (512^3 LNCC), and the 192^3 MI
        # recipe at 512^3, whose sweeps sit nearer the bandwidth roofline
        out["time_to_solution"] = {"lncc_c2": time_to_solution_record("c2", args.ttl_n),
                                   "mi_c1_recipe": time_to_solution_record("c1", args.ttl_n or 512,
                                                                           lam_scale=100.0)}
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default="c4", choices=sorted(WORKLOADS))
    ap.add_argument("--subs", default="c1,c2", help="further workloads timed as sub-records (comma-separated)")
    ap.add_argument("--no-subs", action="store_true")
    ap.add_argument("--no-ttl", action="store_true", help="skip the BF16 vs FP32 time-to-solution record")
    ap.add_argument("--ttl-n", type=int, default=None, help="grid size of the time-to-solution record (512)")
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
