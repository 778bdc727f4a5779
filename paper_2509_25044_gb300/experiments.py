"""Time-to-solution experiments on the synthetic workloads.

    python -m paper_2509_25044_gb300.experiments ttl --config c2 [--iters 300]

`ttl` (time to loss): runs the plain FP32 registration (FP32 images and Adam
moments) and the BF16 storage form (BF16 images and moments, FP32 arithmetic)
of the same pair for the same number of iterations.  The target comes from
the FP32 run's objective C + lambda R on the FP32 images: its final value L*
and its start value L0.  A run reaches the target when its iterate, evaluated
on the FP32 images, has made 99 % of the FP32 run's decrease, i.e.
L <= L* + 0.01 (L0 - L*) (the objective itself can barely move -- 1 - S near
1 on noisy windows -- so 1 % of L* would say nothing).  Each run's time to
solution is its number of iterations to the target times its measured
time per iteration (CUDA events).  The BF16 run is repeated
deterministically to evaluate its iterates on the FP32 images every few
iterations outside the timed pass.  Both final fields are checked for folding
(det(I + grad u) > 0 everywhere).  Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import capi, synth
from .register import RegConfig, Registration

# LNCC epsilon for the count-normalised moments A, B, C: below the variance
# product of the 0.02 acquisition noise (1.6e-7), so flat windows keep
# their texture signal
LNCC_EPS = 1e-9


def _cfg(c: dict, d: dict, moments: str, lam_scale: float = 1.0, adam_eps: float = 1e-8) -> RegConfig:
    lam = c["lam"] * lam_scale
    if c["kind"] == "lncc":
        return RegConfig(loss="lncc", window=c["window"], eps=LNCC_EPS, lam=lam, lr=c["lr"], moments=moments,
                         adam_eps=adam_eps)
    return RegConfig(loss="mi", bins=c["bins"], f_range=d["f_range"], m_range=d["m_range"], lam=lam, lr=c["lr"],
                     moments=moments, adam_eps=adam_eps)


def _warm(F, M, cfg, affine=None, iters: int = 2):
    """A couple of untimed iterations of the same configuration on a scratch
    state, so that the timed run does not pay the first launch of each kernel
    (module loading, attribute and occupancy queries)."""
    Registration(F, M, cfg, affine=affine).run(iters)
    torch.cuda.synchronize()


def _first_within(values, target, tol):
    idx = np.nonzero(np.asarray(values) <= target + tol)[0]
    return int(idx[0]) if idx.size else None


def time_to_loss(config: str, iters: int | None = None, eval_every: int = 1, n: int | None = None,
                 rel_tol: float = 0.01, lam_scale: float = 1.0, adam_eps: float = 1e-8) -> dict:
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    d = synth.make(config, device=dev, n=n)
    c = d["config"]
    iters = iters or c["iters"]
    F32, M32 = d["F"].contiguous(), d["M"].contiguous()
    del d["u_true"]

    # plain FP32 run: its own per-iteration objective is already on FP32 images
    r32 = Registration(F32, M32, _cfg(c, d, "f32", lam_scale, adam_eps))
    _warm(r32.F, r32.M, r32.cfg, affine=r32.affine)
    res32 = r32.run(iters)
    final32 = r32.objective()
    fold32 = r32.fold_check()
    L_star = final32["objective"]
    L0 = float(res32.objective[0])
    tol = rel_tol * max(L0 - L_star, 0.0)
    trace32 = np.append(res32.objective[1:], final32["objective"])  # objective after each step
    k32 = _first_within(trace32, L_star, tol)

    # BF16 storage form: timed pass, then a deterministic replay evaluated on FP32 images
    Fb, Mb = F32.to(torch.bfloat16).contiguous(), M32.to(torch.bfloat16).contiguous()
    cfg_b = _cfg(c, d, "bf16", lam_scale, adam_eps)
    if cfg_b.loss == "mi":  # ranges of the stored BF16 values
        cfg_b.f_range = (float(Fb.min()), float(Fb.max()))
        cfg_b.m_range = (float(Mb.min()), float(Mb.max()))
    rb = Registration(Fb, Mb, cfg_b)
    _warm(rb.F, rb.M, rb.cfg, affine=rb.affine)
    resb = rb.run(iters)
    foldb = rb.fold_check()
    rb2 = Registration(Fb, Mb, cfg_b)
    checkpoints, evals = [], []
    done = 0
    while done < iters:
        step = min(eval_every, iters - done)
        rb2.run(step)
        done += step
        checkpoints.append(done)
        evals.append(rb2.objective(F=F32, M=M32)["objective"])
    same = bool(torch.equal(rb2.current, rb.current))
    kb_idx = _first_within(evals, L_star, tol)
    kb = checkpoints[kb_idx] if kb_idx is not None else None

    out = {
        "experiment": "time_to_loss", "config": config, "n": F32.shape[0], "iters": iters,
        "lam": c["lam"] * lam_scale, "lr": c["lr"], "adam_eps": adam_eps,
        "target": {"objective_fp32_start": L0, "objective_fp32_final": L_star,
                   "rule": f"L <= L* + {rel_tol} (L0 - L*)"},
        "fp32": {"ms_per_iter": res32.ms_per_iter, "iters_to_target": (k32 + 1) if k32 is not None else None,
                 "time_to_target_ms": (k32 + 1) * res32.ms_per_iter if k32 is not None else None,
                 "final": final32, "fold": fold32},
        "bf16": {"ms_per_iter": resb.ms_per_iter, "iters_to_target_upper": kb,
                 "time_to_target_ms": kb * resb.ms_per_iter if kb is not None else None,
                 "final_on_fp32_images": evals[-1], "final_rel_to_fp32_final": (evals[-1] - L_star) / abs(L_star),
                 "final_progress_vs_fp32": (L0 - evals[-1]) / max(L0 - L_star, 1e-300),
                 "fold": foldb, "replay_bitwise_identical": same, "eval_every": eval_every},
    }
    if out["fp32"]["time_to_target_ms"] and out["bf16"]["time_to_target_ms"]:
        out["speedup_bf16_vs_fp32"] = out["fp32"]["time_to_target_ms"] / out["bf16"]["time_to_target_ms"]
    return out


def approx_vs_exact(config: str, variant: str = "ants", iters: int | None = None, n: int | None = None,
                    lam_scale: float = 20.0, rel_tol: float = 0.01) -> dict:
    """An approximate variant of the paper against the exact form (both FP32
    storage): "ants" (LNCC gradient without the second box sum) or "mi_hard"
    (hard-binned MI histogram).  Time for the approximate run to reach the
    exact run's target L <= L* + rel_tol (L0 - L*), with both runs' objectives
    evaluated by the exact form (for "ants" the objective is the same
    function; for "mi_hard" the approximate run is replayed and evaluated
    with the Parzen estimator).  Fold checks of both."""
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    d = synth.make(config, device=dev, n=n)
    c = d["config"]
    iters = iters or c["iters"]
    F, M = d["F"].contiguous(), d["M"].contiguous()
    out = {"experiment": "approx_vs_exact", "variant": variant, "config": config, "n": F.shape[0],
           "iters": iters, "lam": c["lam"] * lam_scale}
    cfg0 = _cfg(c, d, "f32", lam_scale)
    r0 = Registration(F, M, cfg0)
    _warm(r0.F, r0.M, r0.cfg, affine=r0.affine)
    res0 = r0.run(iters)
    fin0 = r0.objective()
    L0, Lstar = float(res0.objective[0]), fin0["objective"]
    tol = rel_tol * max(L0 - Lstar, 0.0)
    k0 = _first_within(np.append(res0.objective[1:], Lstar), Lstar, tol)
    out["exact"] = {"ms_per_iter": res0.ms_per_iter, "iters_to_target": None if k0 is None else k0 + 1,
                    "time_to_target_ms": None if k0 is None else (k0 + 1) * res0.ms_per_iter, "final": fin0,
                    "fold": r0.fold_check()}
    cfg1 = _cfg(c, d, "f32", lam_scale)
    setattr(cfg1, "ants" if variant == "ants" else "mi_hard", True)
    r1 = Registration(F, M, cfg1)
    _warm(r1.F, r1.M, r1.cfg, affine=r1.affine)
    res1 = r1.run(iters)
    # the exact form's objective along the approximate run (a replay: the
    # iteration is deterministic), so both runs are scored by one function
    exact = Registration(F, M, cfg0)
    rep = Registration(F, M, cfg1)
    trace = []
    for _ in range(iters):
        rep.run(1)
        trace.append(exact.objective(u=rep.current)["objective"])
    k1 = _first_within(trace, Lstar, tol)
    out["approx"] = {"ms_per_iter": res1.ms_per_iter, "iters_to_target": None if k1 is None else k1 + 1,
                     "time_to_target_ms": None if k1 is None else (k1 + 1) * res1.ms_per_iter,
                     "final_exact_objective": trace[-1], "fold": r1.fold_check(),
                     "replay_bitwise_identical": bool(torch.equal(rep.current, r1.current))}
    if out["exact"]["time_to_target_ms"] and out["approx"]["time_to_target_ms"]:
        out["speedup_approx_vs_exact"] = out["exact"]["time_to_target_ms"] / out["approx"]["time_to_target_ms"]
    return out


def regularisers(config: str = "c0", iters: int = 50, n: int | None = None) -> dict:
    """The diffusion penalty against the Gaussian smoothing regularisation
    (sigma_grad before each Adam step, sigma_warp after it) on one
    mono-modal workload: final objective, error to the inverse of the true
    field, folds and time per iteration."""
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    d = synth.make(config, device=dev, n=n)
    c = d["config"]
    rows = []
    for sg, sw, lam in ((0.0, 0.0, 0.0), (0.0, 0.0, 2.0), (1.0, 0.5, 0.0), (1.0, 1.0, 0.0), (2.0, 1.0, 0.0)):
        cfg = RegConfig(loss="lncc", window=c["window"], eps=LNCC_EPS, lam=lam, lr=c["lr"], sigma_grad=sg,
                        sigma_warp=sw)
        r = Registration(d["F"], d["M"], cfg)
        _warm(r.F, r.M, r.cfg, affine=r.affine)
        res = r.run(iters)
        err = float(((r.current + d["u_true"]).norm() / d["u_true"].norm()).item())
        rows.append({"sigma_grad": sg, "sigma_warp": sw, "lam": lam, "similarity_loss_final": float(1.0 - res.sim[-1]),
                     "rel_err_vs_inverse_true": err, "fold": r.fold_check()["n_fold"], "ms_per_iter": res.ms_per_iter})
    return {"experiment": "regularisers", "config": config, "iters": iters, "rows": rows}


def multiscale_vs_single(n_pairs: int = 8, n: int = 128, seed0: int = 90_000, window: int = 7, lam: float = 2.0,
                         lr: float = 0.1, iters: int = 200, scales=(4, 2, 1), ms_iters=(100, 100, 200),
                         rel_tol: float = 0.01) -> dict:
    """Held-out pairs of the training distribution (fields up to 10 voxels)
    registered single-scale from zero and coarse-to-fine: time for the
    multi-scale schedule (coarse levels included) to bring the full-resolution
    objective to the single-scale run's target, final objectives, folds and
    error to the known field."""
    from .register import register_multiscale
    from .unet import training_pair
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    cfg = RegConfig(loss="lncc", window=window, eps=LNCC_EPS, lam=lam, lr=lr)
    rows = []
    for i in range(n_pairs):
        p = training_pair(n, seed0 + i, dev)
        F, M, v = p["F"].contiguous(), p["M"].contiguous(), p["v"]
        r0 = Registration(F, M, cfg)
        _warm(r0.F, r0.M, r0.cfg, affine=r0.affine)
        res0 = r0.run(iters)
        fin0 = r0.objective()
        L0, Lstar = float(res0.objective[0]), fin0["objective"]
        tol = rel_tol * max(L0 - Lstar, 0.0)
        k0 = _first_within(np.append(res0.objective[1:], Lstar), Lstar, tol)
        register_multiscale(F, M, cfg, scales, tuple(1 for _ in scales))  # warm-up (untimed)
        out = register_multiscale(F, M, cfg, scales, ms_iters)
        last = out["levels"][-1]["result"]
        coarse_ms = out["ms"] - last.ms_per_iter * ms_iters[-1]
        rfin = Registration(F, M, cfg, u0=out["u"])
        fin1 = rfin.objective()
        k1 = _first_within(np.append(last.objective[1:], fin1["objective"]), Lstar, tol)
        err = lambda u: float(((u - v).norm() / v.norm()).item())
        row = {"seed": seed0 + i, "max_disp": float(v.norm(dim=0).max().item()),
               "single": {"iters_to_target": None if k0 is None else k0 + 1, "L_final": Lstar,
                          "ms_per_iter": res0.ms_per_iter, "fold": r0.fold_check()["n_fold"], "rel_err": err(r0.current)},
               "multi": {"coarse_ms": coarse_ms, "full_iters_to_target": None if k1 is None else k1 + 1,
                         "L_final": fin1["objective"], "ms_total": out["ms"], "fold": rfin.fold_check()["n_fold"],
                         "rel_err": err(out["u"])}}
        if k0 is not None and k1 is not None:
            t0 = (k0 + 1) * res0.ms_per_iter
            t1 = coarse_ms + (k1 + 1) * last.ms_per_iter
            row["time_to_target_ms"] = {"single": t0, "multi": t1}
            row["speedup"] = t0 / t1
        rows.append(row)
    sp = [r["speedup"] for r in rows if "speedup" in r]
    return {"experiment": "multiscale_vs_single", "n": n, "pairs": n_pairs, "scales": list(scales),
            "iters": list(ms_iters), "single_iters": iters, "lam": lam, "median_speedup": float(np.median(sp)) if sp else None,
            "reached": len(sp), "rows": rows}


def affine_pipeline(n: int = 192, seed: int = 7, iters: int = 200, lam: float = 1.0, lr: float = 0.1,
                    scales=(4, 2, 1), aff_iters=(100, 60, 40), rel_tol: float = 0.01) -> dict:
    """The paper's two-stage pipeline on a multi-modal pair whose moving image
    is also moved by a known affine map (rotation about two axes, anisotropic
    scale, shift): (a) deformable MI registration alone from the identity;
    (b) the multi-scale affine stage, then the deformable stage under the
    composite transform phi = A p + t + u.  Reports the recovered affine
    error, the final objectives and the time for (b), affine stage included,
    to reach (a)'s target."""
    from . import synth
    from .register import affine_about_centre, register_affine
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    pair = synth.multimodal_pair(n, seed, field_sigma=6.0, max_disp=3.0, device=dev)
    F, Md = pair["F"].contiguous(), pair["M"].contiguous()
    shape = tuple(F.shape)
    a, b = 0.08, 0.04
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    A_true, t_true = affine_about_centre(Rz @ Rx @ np.diag([1.05, 0.96, 1.02]), (0.03 * n, -0.02 * n, 0.015 * n),
                                         shape)
    Ai = np.linalg.inv(A_true)
    M = capi.reg_warp_composite(Md, capi.affine_desc(Ai, -Ai @ t_true))
    cfg = RegConfig(loss="mi", bins=32, f_range=pair["f_range"], m_range=(float(M.min()), float(M.max())),
                    lam=lam, lr=lr)
    # (a) deformable alone
    r0 = Registration(F, M, cfg)
    _warm(r0.F, r0.M, r0.cfg, affine=r0.affine)
    res0 = r0.run(iters)
    fin0 = r0.objective()
    L0 = float(res0.objective[0])
    # (b) affine stage, then deformable under the composite transform
    register_affine(F, M, cfg, scales=scales, iters=tuple(2 for _ in scales))  # warm-up (untimed)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    out = register_affine(F, M, cfg, scales=scales, iters=aff_iters)
    ev1.record()
    torch.cuda.synchronize()
    aff_ms = ev0.elapsed_time(ev1)
    T = capi.affine_desc(out["A"], out["t"])
    r1 = Registration(F, M, cfg, affine=T)
    _warm(r1.F, r1.M, r1.cfg, affine=r1.affine)
    res1 = r1.run(iters)
    fin1 = r1.objective()
    X = np.stack(np.meshgrid(np.arange(shape[2]), np.arange(shape[1]), np.arange(shape[0]),
                             indexing="ij")).reshape(3, -1).astype(np.float64)
    e = np.linalg.norm((out["A"] - A_true) @ X + (out["t"] - t_true)[:, None], axis=0)
    e0 = np.linalg.norm((np.eye(3) - A_true) @ X - t_true[:, None], axis=0)
    Lstar = fin0["objective"]
    tol = rel_tol * max(L0 - Lstar, 0.0)
    k1 = _first_within(np.append(res1.objective[1:], fin1["objective"]), Lstar, tol)
    row = {"experiment": "affine_pipeline", "n": n, "iters": iters, "lam": lam, "scales": list(scales),
           "aff_iters": list(aff_iters),
           "affine_error_vox": {"identity_mean": float(e0.mean()), "identity_max": float(e0.max()),
                                "recovered_mean": float(e.mean()), "recovered_max": float(e.max())},
           "affine_stage_ms": aff_ms,
           "deformable_only": {"L0": L0, "L_final": Lstar, "ms_per_iter": res0.ms_per_iter,
                               "fold": r0.fold_check()["n_fold"]},
           "composite": {"L_start": float(res1.objective[0]), "L_final": fin1["objective"],
                         "ms_per_iter": res1.ms_per_iter, "iters_to_target": None if k1 is None else k1 + 1}}
    if k1 is not None:
        t_a = iters * res0.ms_per_iter
        t_b = aff_ms + (k1 + 1) * res1.ms_per_iter
        row["time_to_target_ms"] = {"deformable_only": t_a, "affine_then_composite": t_b}
        row["speedup"] = t_a / t_b
    return row


def svf_vs_displacement(config: str = "c0", iters: int = 100, steps_list=(6, 8), lams=(0.0, 2.0)) -> dict:
    """Displacement-field registration (the fused iteration) against the
    stationary velocity field form (u = exp(v), scaling and squaring and its
    backward): final objective, error to the true field, folded voxels and
    time per iteration, at each regulariser weight."""
    from . import synth
    from .register import register_svf
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    c = synth.CONFIGS[config]
    d = synth.make(config, device=dev)
    F, M, ut = d["F"].contiguous(), d["M"].contiguous(), d["u_true"]
    rows = []
    err = lambda u: float(((u + ut).norm() / ut.norm()).item())  # M = F o (id + u_true): u* ~ -u_true
    for lam in lams:
        if c["kind"] == "lncc":
            cfg = RegConfig(loss="lncc", window=c["window"], eps=LNCC_EPS, lam=lam, lr=0.1)
        else:
            cfg = RegConfig(loss="mi", bins=c["bins"], f_range=d["f_range"], m_range=d["m_range"], lam=lam, lr=0.1)
        r = Registration(F, M, cfg)
        _warm(r.F, r.M, r.cfg, affine=r.affine)
        res = r.run(iters)
        fin = r.objective()
        row = {"lam": lam,
               "displacement": {"L_final": fin["objective"], "sim_final": fin["sim"],
                                "fold": r.fold_check()["n_fold"], "rel_err": err(r.current),
                                "ms_per_iter": res.ms_per_iter}, "svf": []}
        for steps in steps_list:
            register_svf(F, M, cfg, 2, steps=steps)  # warm-up (untimed)
            out = register_svf(F, M, cfg, iters, steps=steps)
            mn, nf = capi.reg_jacdet_min(out["u"])
            row["svf"].append({"steps": steps, "L_last": float(out["objective"][-1]),
                               "sim_last": float(out["sim"][-1]), "fold": int(nf.item()),
                               "min_det": float(mn.item()), "rel_err": err(out["u"]),
                               "ms_per_iter": out["ms_per_iter"]})
        rows.append(row)
    return {"experiment": "svf_vs_displacement", "config": config, "iters": iters, "rows": rows}


def eval_init_pairs(net, n_pairs: int = 8, n: int = 128, seed0: int = 90_000, iters: int = 200, window: int = 7,
                    lam: float = 1.0, lr: float = 0.1, rel_tol: float = 0.01) -> dict:
    """Held-out pairs of the training distribution (seeds never used in
    training), registered with LNCC from zero and from the network's field:
    iterations (and time, inference included) for the learned-init run to
    reach the zero-init run's target (reading: L <= L* + rel_tol (L0 - L*),
    L0 and L* the zero-init run's first and final objectives), final
    objectives, fold checks and the error to the known field."""
    from .unet import training_pair
    dev = torch.device("cuda", torch.cuda.current_device())
    rows = []
    for i in range(n_pairs):
        p = training_pair(n, seed0 + i, dev)
        F, M, v = p["F"].contiguous(), p["M"].contiguous(), p["v"]
        cfg = RegConfig(loss="lncc", window=window, eps=LNCC_EPS, lam=lam, lr=lr)
        r0 = Registration(F, M, cfg)
        _warm(r0.F, r0.M, r0.cfg, affine=r0.affine)
        res0 = r0.run(iters)
        fin0 = r0.objective()
        L0, Lstar = float(res0.objective[0]), fin0["objective"]
        tol = rel_tol * max(L0 - Lstar, 0.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        u0 = net.predict_init(F, M, (float(F.min()), float(F.max())), (float(M.min()), float(M.max())))
        ev1.record()
        torch.cuda.synchronize()
        init_ms = ev0.elapsed_time(ev1)
        r1 = Registration(F, M, cfg, u0=u0)
        _warm(r1.F, r1.M, r1.cfg, affine=r1.affine)
        res1 = r1.run(iters)
        fin1 = r1.objective()
        k0 = _first_within(np.append(res0.objective[1:], Lstar), Lstar, tol)
        k1 = _first_within(np.append(res1.objective[1:], fin1["objective"]), Lstar, tol)
        err = lambda u: float(((u - v).norm() / v.norm()).item())
        row = {"seed": seed0 + i, "max_disp": float(v.norm(dim=0).max().item()),
               "zero": {"L0": L0, "L_final": Lstar, "iters_to_target": None if k0 is None else k0 + 1,
                        "fold": r0.fold_check()["n_fold"], "rel_err": err(r0.current)},
               "learned": {"L0": float(res1.objective[0]), "L_final": fin1["objective"],
                           "iters_to_target": None if k1 is None else k1 + 1, "init_ms": init_ms,
                           "fold": r1.fold_check()["n_fold"], "rel_err": err(r1.current), "init_rel_err": err(u0)},
               "ms_per_iter": res0.ms_per_iter}
        if k0 is not None and k1 is not None:
            row["time_to_target_ms"] = {"zero": (k0 + 1) * res0.ms_per_iter,
                                        "learned": init_ms + (k1 + 1) * res1.ms_per_iter}
            row["speedup"] = row["time_to_target_ms"]["zero"] / row["time_to_target_ms"]["learned"]
        rows.append(row)
    sp = [r["speedup"] for r in rows if "speedup" in r]
    return {"experiment": "eval_init_pairs", "n": n, "pairs": n_pairs, "iters": iters, "window": window, "lam": lam,
            "lr": lr, "median_speedup": float(np.median(sp)) if sp else None, "reached": len(sp), "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("ttl")
    t.add_argument("--config", default="c2")
    t.add_argument("--iters", type=int, default=None)
    t.add_argument("--n", type=int, default=None)
    t.add_argument("--eval-every", type=int, default=1)
    t.add_argument("--lam-scale", type=float, default=1.0)
    t.add_argument("--adam-eps", type=float, default=1e-8)
    msp = sub.add_parser("multiscale")
    msp.add_argument("--pairs", type=int, default=8)
    msp.add_argument("--lam", type=float, default=2.0)
    msp.add_argument("--ms-iters", default="100,100,200", help="iterations per level, coarse to fine")
    afp = sub.add_parser("affine")
    afp.add_argument("--n", type=int, default=192)
    afp.add_argument("--lam", type=float, default=1.0)
    svp = sub.add_parser("svf")
    svp.add_argument("--config", default="c0")
    svp.add_argument("--iters", type=int, default=100)
    rg = sub.add_parser("regularisers")
    rg.add_argument("--config", default="c0")
    rg.add_argument("--iters", type=int, default=50)
    rg.add_argument("--n", type=int, default=None)
    an = sub.add_parser("approx")
    an.add_argument("--variant", default="ants", choices=["ants", "mi_hard"])
    an.add_argument("--config", default="c2")
    an.add_argument("--iters", type=int, default=None)
    an.add_argument("--n", type=int, default=None)
    an.add_argument("--lam-scale", type=float, default=20.0)
    li = sub.add_parser("learned-init")
    li.add_argument("--pairs", type=int, default=2000)
    li.add_argument("--epochs", type=int, default=4)
    li.add_argument("--lr", type=float, default=2e-4)
    li.add_argument("--eval-config", default="c2")
    li.add_argument("--eval-n", type=int, default=None)
    li.add_argument("--save", default=None)
    li.add_argument("--eval-pairs", type=int, default=8)
    li.add_argument("--eval-lam", type=float, default=2.0, help="regulariser weight of the evaluation runs")
    li.add_argument("--train-noise", type=float, default=0.02,
                    help="noise of the training pairs (0.0025: a 512^3 pair as the network sees it, pooled 4^3)")
    li.add_argument("--train-kind", default="mono", choices=["mono", "multi"],
                    help="mono-modal blob pairs (LNCC workloads) or two-modality phantoms (MI workloads)")
    li.add_argument("--train-smooth", type=float, default=1.0, help="smoothing of the two-modality phantoms")
    li.add_argument("--eval-moments", default="f32", choices=["f32", "bf16"], help="Adam moments of the evaluation")
    args = ap.parse_args()
    if args.cmd == "learned-init":
        tr, net = train_init(args.pairs, args.epochs, lr=args.lr, out_path=args.save, noise=args.train_noise,
                             kind=args.train_kind, smooth=args.train_smooth)
        print(json.dumps(tr), flush=True)
        if args.eval_pairs > 0:
            print(json.dumps(eval_init_pairs(net, n_pairs=args.eval_pairs, lam=args.eval_lam)), flush=True)
        if args.eval_config != "none":
            lam_scale = args.eval_lam / synth.CONFIGS[args.eval_config]["lam"]
            print(json.dumps(eval_init(net, args.eval_config, n=args.eval_n, lam_scale=lam_scale,
                                       moments=args.eval_moments)), flush=True)
        return
    if args.cmd == "multiscale":
        its = tuple(int(x) for x in args.ms_iters.split(","))
        print(json.dumps(multiscale_vs_single(args.pairs, lam=args.lam, ms_iters=its)))
        return
    if args.cmd == "affine":
        print(json.dumps(affine_pipeline(args.n, lam=args.lam)))
        return
    if args.cmd == "svf":
        print(json.dumps(svf_vs_displacement(args.config, args.iters)))
        return
    if args.cmd == "regularisers":
        print(json.dumps(regularisers(args.config, args.iters, args.n)))
        return
    if args.cmd == "approx":
        print(json.dumps(approx_vs_exact(args.config, args.variant, args.iters, args.n, args.lam_scale)))
        return
    if args.cmd == "ttl":
        print(json.dumps(time_to_loss(args.config, args.iters, args.eval_every, args.n, lam_scale=args.lam_scale,
                                      adam_eps=args.adam_eps)))


# ---------------------------------------------------------------------------
# learned initialiser: training and evaluation
# ---------------------------------------------------------------------------
def train_init(n_pairs: int = 2000, epochs: int = 4, n: int = 128, lr: float = 2e-4, seed0: int = 10_000,
               out_path: str | None = None, log_every: int = 200, noise: float = 0.02, kind: str = "mono",
               smooth: float = 1.0) -> dict:
    """Train the U-Net on n_pairs seeded pairs made with the library's warp
    (targets: the known fields pooled to n/2), with acquisition noise `noise`:
    mono-modal blob pairs (training_pair) or, kind="multi", the MI workloads'
    two-modality phantoms smoothed at `smooth` (multimodal_training_pair).
    Pairs are generated once and kept on the device (packed inputs +
    targets)."""
    import time
    from .unet import UNet, multimodal_training_pair, training_pair
    dev = torch.device("cuda", torch.cuda.current_device())
    capi.load()
    net = UNet(n_in=n, seed=0, device=dev)
    L = net.L
    t0 = time.perf_counter()
    xs, ts = [], []
    for i in range(n_pairs):
        p = (multimodal_training_pair(n, seed0 + i, dev, noise=noise, smooth=smooth) if kind == "multi"
             else training_pair(n, seed0 + i, dev, noise=noise))
        # images kept as BF16 (the network sees them in BF16 anyway); packed per step
        xs.append((p["F"].to(torch.bfloat16), p["M"].to(torch.bfloat16),
                   (float(p["F"].min()), float(p["F"].max())), (float(p["M"].min()), float(p["M"].max()))))
        t = torch.empty((3, (n // 2) ** 3), device=dev)
        capi.nn_check(L.reg_nn_field_down2(capi.ptr(p["v"]), capi.RegDims(n, n, n), capi.ptr(t), capi.stream_of(t)),
                      "field_down2")
        ts.append(t)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    hist = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    order_rng = np.random.default_rng(seed0)
    for ep in range(epochs):
        order = order_rng.permutation(n_pairs)
        tot = torch.zeros((), dtype=torch.float64, device=dev)
        for j, i in enumerate(order):
            Fb, Mb, fr, mr = xs[i]
            net.pack(Fb, Mb, 1, fr, mr)
            net.forward()
            tot += net.loss_and_backward(ts[i])[0]
            net.step(lr)
        hist.append(float(tot.item()) / n_pairs)
    ev1.record()
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    # baseline: predicting zero
    zero = float(np.mean([float((t ** 2).mean().item()) for t in ts[:200]]))
    out = {"experiment": "train_init", "kind": kind, "n_pairs": n_pairs, "epochs": epochs, "n": n, "lr": lr,
           "noise": noise,
           "pair_generation_s": gen_s, "train_ms": train_ms, "ms_per_pair_step": train_ms / (epochs * n_pairs),
           "loss_per_epoch": hist, "zero_prediction_loss": zero, "device_error": capi.reg_get_device_error()}
    if out_path:
        state = {k: (P.w.cpu(), P.b.cpu()) for k, P in net.p.items()}
        torch.save({"state": state, "meta": out}, out_path)
    return out, net


def eval_init(net, config: str = "c2", iters: int | None = None, lam_scale: float = 10.0, n: int | None = None,
              rel_tol: float = 0.01, moments: str = "f32") -> dict:
    """Registration of a held-out pair from zero and from the network's
    initial field: iterations (and time) for the learned-init run to reach
    the zero-init run's final objective within 1 % of the zero-init run's
    total decrease; fold checks of both.  The zero-init run is released
    before the learned-init one starts (gigavoxel pairs)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    d = synth.make(config, device=dev, n=n)
    c = d["config"]
    iters = iters or c["iters"]
    F, M = d["F"].contiguous(), d["M"].contiguous()
    cfg = _cfg(c, d, moments, lam_scale)
    err = lambda u: float(((u + d["u_true"]).norm() / d["u_true"].norm()).item())
    r0 = Registration(F, M, cfg)
    _warm(r0.F, r0.M, r0.cfg, affine=r0.affine)
    res0 = r0.run(iters)
    fin0 = r0.objective()
    fold0, err0 = r0.fold_check(), err(r0.current)
    del r0
    torch.cuda.empty_cache()
    L0, Lstar = float(res0.objective[0]), fin0["objective"]
    tol = rel_tol * max(L0 - Lstar, 0.0)
    ranges = (float(F.min()), float(F.max())), (float(M.min()), float(M.max()))
    net.predict_init(F, M, *ranges)  # untimed: first-call set-up, as the registrations are warmed
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    u0 = net.predict_init(F, M, *ranges)
    ev1.record()
    torch.cuda.synchronize()
    init_ms = ev0.elapsed_time(ev1)
    r1 = Registration(F, M, cfg, u0=u0)
    _warm(r1.F, r1.M, r1.cfg, affine=r1.affine)
    res1 = r1.run(iters)
    fin1 = r1.objective()
    tr0 = np.append(res0.objective[1:], Lstar)
    tr1 = np.append(res1.objective[1:], fin1["objective"])
    k0 = _first_within(tr0, Lstar, tol)
    k1 = _first_within(tr1, Lstar, tol)
    out = {"experiment": "eval_init", "config": config, "n": F.shape[0], "iters": iters, "lam": cfg.lam,
           "moments": moments,
           "zero_init": {"objective_start": L0, "objective_final": Lstar, "iters_to_target": None if k0 is None else k0 + 1,
                         "ms_per_iter": res0.ms_per_iter, "fold": fold0, "rel_err_vs_inverse_true": err0},
           "learned_init": {"objective_start": float(res1.objective[0]), "objective_final": fin1["objective"],
                            "iters_to_target": None if k1 is None else k1 + 1, "ms_per_iter": res1.ms_per_iter,
                            "init_ms": init_ms, "fold": r1.fold_check(), "rel_err_vs_inverse_true": err(r1.current),
                            "init_rel_err_vs_inverse_true": err(u0)}}
    if k0 is not None and k1 is not None:
        t0 = (k0 + 1) * res0.ms_per_iter
        t1 = init_ms + (k1 + 1) * res1.ms_per_iter
        out["time_to_target_ms"] = {"zero_init": t0, "learned_init": t1, "speedup": t0 / t1}
    return out


if __name__ == "__main__":
    main()
