#!/usr/bin/env python
"""Benchmark: staggered even-odd CG (Dslash inside CG) on one GB300, through the C-ABI.

Default workload (cg32_mixed): the 32^4 Haar lattice at m = 0.01. One step = one pass of the whole
hot path: pack the gauge field at FP64 and FP32 recon-12 (qcd_load_links), run the mixed-precision
even-odd CG (FP32 recon-12 recursion with the fused Dslash/CG kernels, FP64 reliable updates) to a
true relative residual of 1e-10, form y = D_oe x and recompute the FP64 true residual
(qcd_cg_solve). The same line carries the plain FP64, FP16 recon-12 and df64 solves of the same
problem (speedups), each solution's residual recomputed by the oracle at sampled sites, each
precision's operator alone, and the 24^4 x 16 RHS and 64-lattice batched solves with their
speedups over one-by-one plain FP64 CG. Other workloads: --workload.

value = Dslash GFLOP/s sustained inside the solve: 570 flop per output site of every
half-lattice operator application the solve performs (2 per CG iteration, 2 more for y and
the true residual, 2 per reliable update), divided by the step's device time.

Timing: W untimed warm-up steps, then exactly K timed steps, each bracketed by CUDA events on
the library's stream; the L2 cache is flushed (a 512 MB write) before every step, outside the
events. Under torchrun each rank runs an independent replica (the solve does not shard).
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & %HBM roofline; CG time-to-1e-10, mixed/batched vs FP64"
FLOP_PER_SITE = 570
# FP64 FMA peak of GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

WORKLOADS = {
    # the headline: 32^4 Haar, m = 0.01, mixed FP32 recon-12 CG with FP64 reliable updates, with the
    # plain FP64, FP16 and df64 solves, the operators alone and the batched solves on the same line
    "cg32_mixed": dict(kind_solve="mixed32", dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10,
                       inner="half12",
                       desc="staggered 32^4 Haar SU(3), m=0.01, mixed CG: 16-bit recon-12 inner (fixed-point links, "
                            "FP16 vectors with a per-site scale, FP32 arithmetic), FP64 reliable updates every 100 "
                            "iterations, to true rel. residual 1e-10 (vs plain FP64, FP32 recon-12 and df64 on the "
                            "same lattice; 24^4 x 16 RHS and 64-lattice batches beside)"),
    # the 16^4 FP64 workload: Haar links, m = 0.1, plain FP64 even-odd CG
    "cg16_fp64": dict(dims=(16, 16, 16, 16), kind="haar", mass=0.1, tol=1e-10, inner="double",
                      desc="staggered 16^4 Haar SU(3), m=0.1, plain FP64 even-odd CG to true rel. residual 1e-10"),
    "cg16_fp64_nearid_m0.02": dict(dims=(16, 16, 16, 16), kind="near_identity", mass=0.02, tol=1e-10, inner="double",
                                   desc="staggered 16^4 near-identity (eps=0.3), m=0.02, FP64 CG to 1e-10"),
    "cg32_fp64": dict(dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10, inner="double",
                      desc="staggered 32^4 Haar SU(3), m=0.01, plain FP64 even-odd CG to 1e-10"),
    "cg32_single12": dict(dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10, inner="single12",
                          desc="staggered 32^4 Haar, m=0.01, mixed CG: FP32 recon-12 inner, FP64 reliable updates"),
    "cg32_half12": dict(dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10, inner="half12",
                        desc="staggered 32^4 Haar, m=0.01, mixed CG: 16-bit recon-12 inner (fixed-point links, FP16 "
                             "vectors), FP64 reliable updates"),
    "cg16_df64": dict(dims=(16, 16, 16, 16), kind="haar", mass=0.1, tol=1e-10, inner="df64",
                      desc="staggered 16^4 Haar SU(3), m=0.1, even-odd CG in df64 (float-float on the FP32 pipes) "
                           "with FP64 reliable updates, to true rel. residual 1e-10"),
    "cg32_df64": dict(dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10, inner="df64",
                      desc="staggered 32^4 Haar, m=0.01, even-odd CG in df64 with FP64 reliable updates"),
    "mrhs24_single12": dict(kind_solve="mrhs", dims=(24, 24, 24, 24), kind="haar", mass=0.05, tol=1e-10,
                            inner="single12", nrhs=16,
                            desc="staggered 24^4 Haar, m=0.05, 16 RHS in one multi-RHS CG: FP32 recon-12 inner, "
                                 "FP64 reliable updates"),
    "mrhs24_half12": dict(kind_solve="mrhs", dims=(24, 24, 24, 24), kind="haar", mass=0.05, tol=1e-10,
                          inner="half12", nrhs=16,
                          desc="staggered 24^4 Haar, m=0.05, 16 RHS in one multi-RHS CG: 16-bit recon-12 inner "
                               "(fixed-point links, FP16 vectors), FP64 reliable updates"),
    "wilson32c64_8rhs": dict(kind_solve="wilson", dims=(32, 32, 32, 64), kind="haar", kappa=0.125, tol=1e-10,
                             inner="single18", nrhs=8,
                             desc="Wilson 32^3x64 Haar SU(3), kappa=0.125, 8 RHS in one multi-RHS CGNR on M^dagger M: "
                                  "FP32 recursion with FP64 reliable updates, to 1e-10"),
    "wilson24c48_single": dict(kind_solve="wilson", dims=(24, 24, 24, 48), kind="haar", kappa=0.125, tol=1e-10,
                               inner="single18", nrhs=1,
                               desc="Wilson 24^3x48 Haar SU(3), kappa=0.125, CGNR, FP32 recursion with FP64 reliable "
                                    "updates, to 1e-10 (the small case for counter captures)"),
    "wilson32c64_single": dict(kind_solve="wilson", dims=(32, 32, 32, 64), kind="haar", kappa=0.125, tol=1e-10,
                               inner="single18", nrhs=1,
                               desc="Wilson 32^3x64 Haar SU(3), kappa=0.125, CGNR on M^dagger M: FP32 recursion with "
                                    "FP64 reliable updates, to 1e-10"),
    "wilson32c64_single_df64": dict(kind_solve="wilson", dims=(32, 32, 32, 64), kind="haar", kappa=0.125, tol=1e-10,
                                    inner="single18", nrhs=1, outer="df64", reliable_delta=0.01,
                                    traffic_key="wilson32c64_single",
                                    desc="Wilson 32^3x64 Haar SU(3), kappa=0.125, CGNR on M^dagger M: FP32 recursion "
                                         "with df64 reliable updates (delta 0.01) and solution, to 1e-10"),
    "wilson32c64_8rhs_df64": dict(kind_solve="wilson", dims=(32, 32, 32, 64), kind="haar", kappa=0.125, tol=1e-10,
                                  inner="single18", nrhs=8, outer="df64", reliable_delta=0.01,
                                  traffic_key="wilson32c64_8rhs",
                                  desc="Wilson 32^3x64 Haar SU(3), kappa=0.125, 8 RHS in one multi-RHS CGNR on "
                                       "M^dagger M: FP32 recursion with df64 reliable updates (delta 0.01) and "
                                       "solution, to 1e-10"),
    "full32_single12": dict(kind_solve="full", dims=(32, 32, 32, 32), kind="haar", mass=0.01, tol=1e-10, inner="single12",
                            desc="full-system solve M x = b (both parities) on 32^4 Haar, m=0.01: even-odd reduction "
                                 "onto the mixed CG (FP32 recon-12 inner, FP64 reliable updates), full FP64 residual 1e-10"),
    "force32_fp64": dict(kind_solve="force", dims=(32, 32, 32, 32), mass=0.1, tol=1e-10,
                         desc="staggered fermion force on every link of a 32^4 Haar lattice from the CG's x and "
                              "y = D_oe x (m = 0.1), FP64"),
    "batch64_half12": dict(kind_solve="batched", n=64, tol=1e-10, inner="half12",
                           desc="64 independent staggered lattices {4^4,6^4,8^4,8^3x16}, m in [0.02,0.5], one "
                                "persistent clustered CG launch: 16-bit recon-12 inner (fixed-point links, FP16 "
                                "vectors), FP64 reliable updates"),
    "batch64_single12": dict(kind_solve="batched", n=64, tol=1e-10, inner="single12",
                             desc="64 independent staggered lattices {4^4,6^4,8^4,8^3x16}, m in [0.02,0.5], one "
                                  "persistent clustered CG launch: FP32 recon-12 inner, FP64 reliable updates"),
}
DEFAULT_WORKLOAD = "cg32_mixed"
PRECS = {"double": (0, 18), "single18": (1, 18), "single12": (1, 12), "half12": (2, 12), "df64": (3, 18)}
# the default line's config-4 legs (multi-RHS and many-lattice solves), at the headline's precision
BATCHED_LEGS = ("mrhs24_half12", "batch64_half12")
NAMES = {"double": "FP64", "single18": "FP32 recon-18", "single12": "FP32 recon-12",
         "half12": "16-bit recon-12 (fixed-point links, FP16 vectors)", "df64": "df64"}
DTYPE = {"double": "f64", "single18": "f32 (FP64 reliable updates)", "single12": "f32 (FP64 reliable updates)",
         "half12": "f32 (16-bit storage: fixed-point links, FP16 vectors; FP64 reliable updates)",
         "df64": "df64 (float-float, 48-bit significand; FP64 reliable updates)"}


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _clock_sampler(device_uuid):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"]
    if device_uuid:
        cmd += ["-i", device_uuid]
    try:
        p = subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL)
    except (OSError, ValueError):
        return None, f.name
    return p, f.name


def _device_uuid(local):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        return None


def _clock_summary(proc, path):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    sm, smax, power, reasons = [], [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as fh:
        for line in fh:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def sources_sha(files) -> str:
    """sha256 over the listed CUDA sources of the library (ncu traffic figures hold only for these)."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(f.encode())
        with open(os.path.join(ROOT, "paper_1311_2719_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(workload):
    """DRAM bytes per launch of the workload's dominant kernel (the mean of K1 and K2 for a CG) from
    profiles/ncu_traffic.json, or None when
    the file has no entry for the workload or the entry was taken on other kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
            w = json.load(fh).get("workloads", {}).get(workload)
        if not w or w.get("sources_sha256") != sources_sha(w["sources"]):
            return None
    except (OSError, ValueError, KeyError):
        return None
    return w["bytes"] if "bytes" in w else (w["K1_bytes"] + w["K2_bytes"]) / 2


def reduce_over_ranks(max_vals, sum_vals, device="cuda"):
    """Whole-job figures of N replicas: the elementwise max over ranks of `max_vals` (times) and the
    sum of `sum_vals` (work done). With one process (no process group) the inputs come back as they
    are. The caller's process group sets the backend (NCCL on GPUs; the tests use gloo on CPU)."""
    import torch
    import torch.distributed as dist
    mx = torch.tensor([float(v) for v in max_vals], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in sum_vals], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist(), sm.tolist()


def _half_dslash_count(info):
    return 2 * info["iterations"] + 2 + 2 * info["reliable_updates"]


def run_gpu(args, wl):
    import numpy as np
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims, mass, tol, inner = wl["dims"], wl["mass"], wl["tol"], wl["inner"]
    U = I.make_links(dims, kind=wl["kind"], seed=1)
    b = I.make_source(dims, seed=2)
    V = U.shape[0]
    Vh = V // 2

    stream = torch.cuda.Stream()
    lat = Q.Lattice(dims)
    U_host = torch.from_numpy(U).pin_memory()
    b_host = torch.from_numpy(b).pin_memory()
    U_dev = U_host.to("cuda", non_blocking=False)
    b_dev = b_host.to("cuda", non_blocking=False)
    x_dev = torch.zeros_like(b_dev)
    y_dev = torch.zeros_like(b_dev)
    x_host = torch.empty_like(b_host).pin_memory()
    y_host = torch.empty_like(b_host).pin_memory()
    packed = {}
    prec_in, recon_in = PRECS[inner]
    for p, r in {(0, 18), (prec_in, recon_in)}:
        packed[p] = (lat.empty_bytes(Q.qcd_links_bytes(lat.handle, p, r)), r)
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = prec_in, recon_in
    ws = lat.workspace(opts)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step(host_io=False, profile=False):
        launches = 0
        opts.profile = 1 if profile else 0
        with torch.cuda.stream(stream):
            if host_io:
                U_dev.copy_(U_host, non_blocking=True)
                b_dev.copy_(b_host, non_blocking=True)
            for p, (buf, r) in packed.items():
                Q.qcd_load_links(lat.handle, U_dev, buf, p, r, stream)
                launches += 1
            rc, info = Q.qcd_cg_solve(lat.handle, x_dev, b_dev, mass, tol, 100000, opts, ws, y_dev, stream=stream)
            if host_io:
                x_host.copy_(x_dev, non_blocking=True)
                y_host.copy_(y_dev, non_blocking=True)
        if rc != Q.QCD_OK:
            raise RuntimeError(f"solve failed: {Q.qcd_status_string(rc)} {info}")
        info["launches"] = launches + info["kernel_launches"]
        return info

    def timed(n, host_io=False, profile=False):
        ms, infos = [], []
        for _ in range(n):
            flush.fill_(1)  # evict L2 between steps (outside the timed events)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(host_io, profile))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    proc, cpath = _clock_sampler(uuid)
    time.sleep(0.3)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms, infos = timed(args.steps)  # production path: graph-replayed chunks, no per-launch events
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    # the same steps with CUDA events around every operator launch (direct launches): kernel time
    ms_prof, infos_prof = timed(args.steps, profile=True)
    clocks = _clock_summary(proc, cpath)
    if world > 1:
        dist.barrier()
    ms_e2e, infos_e2e = timed(args.steps, host_io=True)
    torch.cuda.synchronize()

    flops = [FLOP_PER_SITE * Vh * _half_dslash_count(i) for i in infos]
    total_ms = sum(ms)
    total_ms_e2e = sum(ms_e2e)
    flops_e2e = [FLOP_PER_SITE * Vh * _half_dslash_count(i) for i in infos_e2e]
    (total_ms, total_ms_e2e), (sum_flops, sum_flops_e2e) = reduce_over_ranks([total_ms, total_ms_e2e],
                                                                             [sum(flops), sum(flops_e2e)])
    value = sum_flops / (total_ms * 1e-3) / 1e9
    e2e_value = sum_flops_e2e / (total_ms_e2e * 1e-3) / 1e9

    # dominant kernel: the half-lattice operator launches inside the iterations (CUDA events)
    d_ms = sum(i["dslash_ms"] for i in infos_prof)
    d_n = sum(i["dslash_launches"] for i in infos_prof)
    per_launch_ms = d_ms / d_n
    achieved_tflops = FLOP_PER_SITE * Vh / (per_launch_ms * 1e-3) / 1e12
    # algorithmic bytes per site of the two operator launches of an iteration (links and every
    # vector read or written once): K1 = links + p (in) + ap (out); K2 = links + ap (in) + p, r, x
    # read + r, x written. The average of the two is the per-launch figure.
    link_b, fld_b, x_b = {"double": (1152, 48, 48), "single18": (576, 24, 24), "single12": (384, 24, 24),
                          "half12": (192, 16, 24), "df64": (1152, 48, 48)}[inner]
    k1_b = link_b + 2 * fld_b
    k2_b = link_b + fld_b + 2 * fld_b + x_b + fld_b + x_b
    alg_bytes = (k1_b + k2_b) / 2 * Vh
    achieved_gbs = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if inner == "double":
        roofline = {"bound": "alu", "kernel": "dslash_kernel (CG K1+K2 launches)", "achieved": round(achieved_tflops, 4),
                    "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(achieved_tflops / FP64_PEAK_TFLOPS, 4),
                    "peak_source": "derived FP64 FMA peak (152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz)",
                    "traffic": ncu_traffic(args.workload),
                    "hbm_model_gbs": round(achieved_gbs, 1), "hbm_model_frac": round(achieved_gbs / hbm_peak, 4),
                    "alg_bytes_per_launch": alg_bytes, "alg_bytes_per_site_k1_k2": [k1_b, k2_b],
                    "alg_flops_per_launch": FLOP_PER_SITE * Vh, "avg_launch_us": round(per_launch_ms * 1e3, 3)}
    else:
        roofline = {"bound": "hbm", "kernel": "dslash_kernel (CG K1+K2 launches)", "achieved": round(achieved_gbs, 1),
                    "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved_gbs / hbm_peak, 4),
                    "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)", "traffic": ncu_traffic(args.workload),
                    "alg_bytes_per_launch": alg_bytes, "alg_bytes_per_site_k1_k2": [k1_b, k2_b],
                    "alg_flops_per_launch": FLOP_PER_SITE * Vh,
                    "achieved_tflops": round(achieved_tflops, 4), "avg_launch_us": round(per_launch_ms * 1e3, 3)}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[inner], "data": "synthetic (seeded Haar/near-identity SU(3) links, Gaussian source)",
        "config": {"workload": wl["desc"], "dims": list(dims), "mass": mass, "tol": tol, "inner": inner,
                   "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "step": "qcd_load_links + qcd_cg_solve (CG, y = D_oe x, FP64 true residual)"},
        "cg": {"iterations": infos[-1]["iterations"], "true_rel_residual": infos[-1]["true_rel_residual"],
               "reliable_updates": infos[-1]["reliable_updates"], "time_to_solution_ms": round(total_ms / args.steps, 4),
               "half_dslash_per_solve": _half_dslash_count(infos[-1])},
        "roofline": roofline,
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(U_host.numel() * 16 + b_host.numel() * 16),
                "d2h_bytes_per_step": int(x_host.numel() * 16 + y_host.numel() * 16),
                "ms_per_step": round(total_ms_e2e / args.steps, 4)},
        "gpu_launches": int(sum(i["launches"] for i in infos)),
        "clocks": clocks,
        "wall_s_timed_region": round(t_wall, 4),
        "ms_per_step_profiled_direct_launches": round(sum(ms_prof) / args.steps, 4),
    }
    if inner == "double" and not args.no_variant:
        # the same workload with the recursion in df64 (FP32-pipe float-float arithmetic, FP64 reliable
        # updates and FP64 true residual): reported beside the FP64 headline, not instead of it
        packed[3] = (lat.empty_bytes(Q.qcd_links_bytes(lat.handle, 3, 18)), 18)
        opts.prec_inner, opts.recon_inner = 3, 18
        ws = lat.workspace(opts)
        for _ in range(args.warmup):
            step()
        ms_v, infos_v = timed(args.steps)
        _, infos_vp = timed(max(1, min(args.steps, 3)), profile=True)
        del packed[3]
        fl_v = sum(FLOP_PER_SITE * Vh * _half_dslash_count(i) for i in infos_v)
        pl_ms = sum(i["dslash_ms"] for i in infos_vp) / sum(i["dslash_launches"] for i in infos_vp)
        ach = (k1_b + k2_b) / 2 * Vh / (pl_ms * 1e-3) / 1e9
        out["df64_variant"] = {
            "value": round(fl_v / (sum(ms_v) * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
            "ms_per_step": round(sum(ms_v) / len(ms_v), 4), "dtype": DTYPE["df64"],
            "iterations": infos_v[-1]["iterations"], "true_rel_residual": infos_v[-1]["true_rel_residual"],
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(ach / hbm_peak, 4), "avg_launch_us": round(pl_ms * 1e3, 3),
                         "note": "L2-resident at 16^4: df64 is FP32-pipe/latency bound here, HBM-bound at 32^4"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_iters)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


# Algorithmic bytes per output site of one half-lattice operator launch (links once, every vector
# read or written once) for the two operator launches of a CG iteration: K1 = links + p + ap; K2 =
# links + ap + (p, r, x) read + (r, x) written (x at FP32 for the mixed precisions); and for the
# operator alone (qcd_dslash: links + in + out).
OP_BYTES = {  # name: (link bytes, field bytes, x bytes)
    "double": (1152, 48, 48), "single18": (576, 24, 24), "single12": (384, 24, 24), "half12": (192, 16, 24),
    "df64": (1152, 48, 48)}


def _k1_k2_bytes(inner, folded=False):
    """(K1, K2) algorithmic bytes per output site. `folded`: the FP32 recursion's K1 forms
    p = r + beta p_old itself, so it reads r and p_old and writes p and ap (no separate p kernel)."""
    link_b, fld_b, x_b = OP_BYTES[inner]
    k1 = link_b + 4 * fld_b if folded else link_b + 2 * fld_b
    return k1, link_b + fld_b + 2 * fld_b + x_b + fld_b + x_b


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def fp64_gemm_tflops(n=4096, reps=3):
    """FP64 throughput measured on this GPU by a cuBLAS DGEMM (torch.matmul in float64, n^3):
    the measured FP64 peak beside the derived one (2 FP64 FMA per SM per clock)."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty_like(a)
    torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def sampled_oracle_residual(U, x, b, dims, mass, n_sites=2000, seed=0):
    """|b - A x| / |b| over `n_sites` random even sites, A applied by the FP64 oracle's site-local form."""
    from oracle import staggered as S
    rng = np.random.default_rng(seed)
    V = U.shape[0]
    cand = rng.choice(V, 3 * n_sites, replace=False)
    sites = cand[S.parity_of_sites(dims, cand) == 0][:n_sites]
    r = b[sites] - S.mdagm_sites(U, x, dims, mass, sites)
    return float(np.linalg.norm(r) / np.linalg.norm(b[sites]))


def run_gpu_mixed32(args, wl):
    """32^4 Haar, m = 0.01: the mixed-precision even-odd CG (the workload's inner recursion: 16-bit
    recon-12 by default, FP64 reliable updates) as the headline, with on the same line and the same
    lattice and source:
      fp64      - the plain FP64 CG and the mixed solve's speedup over it;
      single12 / half12 / df64 - the other recursions (FP32 recon-12, 16-bit recon-12, df64);
      accuracy  - each solution's FP64 residual recomputed by the oracle at sampled sites, and its
                  distance to the plain FP64 GPU solution;
      operators - each precision's half-lattice operator alone (qcd_dslash, back-to-back launches);
      batched   - the 24^4 x 16 RHS and the 64-lattice solves and their speedups over one-by-one
                  plain FP64 CG.
    One timed step = qcd_load_links (FP64 and the inner links) + qcd_cg_solve (CG, y, true residual)."""
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims, mass, tol = wl["dims"], wl["mass"], wl["tol"]
    U = I.make_links(dims, kind=wl["kind"], seed=1)
    b = I.make_source(dims, seed=2)
    Vh = U.shape[0] // 2
    peaks = _measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    leg_steps = max(1, min(args.steps, args.leg_steps))

    stream = torch.cuda.Stream()
    lat = Q.Lattice(dims)
    U_host = torch.from_numpy(U).pin_memory()
    b_host = torch.from_numpy(b).pin_memory()
    U_dev = U_host.to("cuda")
    b_dev = b_host.to("cuda")
    x_dev = torch.zeros_like(b_dev)
    y_dev = torch.zeros_like(b_dev)
    x_host = torch.empty_like(b_host).pin_memory()
    y_host = torch.empty_like(b_host).pin_memory()
    pack_of = {"double": (0, 18), "single12": (1, 12), "half12": (2, 12), "df64": (3, 18)}
    bufs = {p: lat.empty_bytes(Q.qcd_links_bytes(lat.handle, p, r)) for p, r in pack_of.values()}
    opts = Q.qcd_solver_opts_default()
    ws = {}
    for name, (p, r) in pack_of.items():
        opts.prec_inner, opts.recon_inner = p, r
        ws[name] = lat.empty_bytes(Q.qcd_workspace_bytes(lat.handle, opts, 1))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step(inner, host_io=False, profile=False):
        p_in, r_in = pack_of[inner]
        opts.prec_inner, opts.recon_inner = p_in, r_in
        opts.profile = 1 if profile else 0
        launches = 0
        with torch.cuda.stream(stream):
            if host_io:
                U_dev.copy_(U_host, non_blocking=True)
                b_dev.copy_(b_host, non_blocking=True)
            for p, r in sorted({(0, 18), (p_in, r_in)}):
                Q.qcd_load_links(lat.handle, U_dev, bufs[p], p, r, stream)
                launches += 1
            rc, info = Q.qcd_cg_solve(lat.handle, x_dev, b_dev, mass, tol, 100000, opts, ws[inner], y_dev,
                                      stream=stream)
            if host_io:
                x_host.copy_(x_dev, non_blocking=True)
                y_host.copy_(y_dev, non_blocking=True)
        if rc != Q.QCD_OK:
            raise RuntimeError(f"{inner} solve failed: {Q.qcd_status_string(rc)} {info}")
        info["launches"] = launches + info["kernel_launches"]
        return info

    def timed(inner, n, host_io=False, profile=False):
        ms, infos = [], []
        for _ in range(n):
            flush.fill_(1)  # evict L2 between steps (outside the timed events)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(inner, host_io, profile))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, infos

    def flops_of(infos):
        return sum(FLOP_PER_SITE * Vh * _half_dslash_count(i) for i in infos)

    # ---- headline: the workload's mixed solve
    head = wl["inner"]
    folded = head == "single12"  # the FP32 recursion forms p = r + beta p inside K1
    for _ in range(args.warmup):
        step(head)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    proc, cpath = _clock_sampler(_device_uuid(local))
    time.sleep(0.3)
    t_wall = time.perf_counter()
    ms, infos = timed(head, args.steps)
    t_wall = time.perf_counter() - t_wall
    clocks = _clock_summary(proc, cpath)
    if world > 1:
        dist.barrier()
    x_mixed = x_dev.cpu().numpy()
    ms_e2e, infos_e2e = timed(head, leg_steps, host_io=True)
    ms_prof, infos_prof = timed(head, 1, profile=True)
    (total_ms, total_e2e), (fl, fl_e2e) = reduce_over_ranks([sum(ms), sum(ms_e2e)], [flops_of(infos), flops_of(infos_e2e)])
    value = fl / (total_ms * 1e-3) / 1e9
    e2e_value = fl_e2e / (total_e2e * 1e-3) / 1e9
    t_mixed = sum(ms) / len(ms)

    # ---- the other recursions on the same lattice and source
    legs, sols = {}, {head: x_mixed}
    for inner in (() if args.no_legs else tuple(n for n in ("double", "single12", "half12", "df64") if n != head)):
        if inner == "df64" and args.no_variant:
            continue
        step(inner)
        ms_l, inf_l = timed(inner, leg_steps)
        sols[inner] = x_dev.cpu().numpy()
        i = inf_l[-1]
        legs[inner] = {"dtype": DTYPE[inner], "ms_per_step": round(sum(ms_l) / len(ms_l), 4), "steps": len(ms_l),
                       "value": round(flops_of(inf_l) / (sum(ms_l) * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                       "iterations": i["iterations"], "reliable_updates": i["reliable_updates"],
                       "true_rel_residual": i["true_rel_residual"]}
    t_fp64 = legs["double"]["ms_per_step"] if legs else None

    # ---- accuracy of every solution: oracle residual at sampled sites, distance to the FP64 solution
    x64 = sols.get("double")
    accuracy = {}
    for inner, xs in sols.items():
        accuracy[inner] = {"oracle_rel_residual_2000_even_sites": sampled_oracle_residual(U, xs, b, dims, mass)}
        if x64 is not None:
            accuracy[inner]["rel_diff_vs_plain_fp64_gpu_solution"] = float(np.linalg.norm(xs - x64) / np.linalg.norm(x64))

    # ---- the half-lattice operator alone, per precision: back-to-back qcd_dslash launches that
    # alternate between two lattices with their own links (so that the links stream from DRAM even
    # where one precision's links would fit in L2), CUDA events around the whole loop
    lat2 = Q.Lattice(dims)
    bufs2 = {p: lat2.empty_bytes(Q.qcd_links_bytes(lat2.handle, p, r)) for p, r in pack_of.values()}
    operators = {}
    fp64_meas = None if args.no_legs else fp64_gemm_tflops()
    n_op = 40
    for name, (p, r) in (() if args.no_legs else pack_of.items()):
        with torch.cuda.stream(stream):
            for L_, B_ in ((lat, bufs), (lat2, bufs2)):
                Q.qcd_load_links(L_.handle, U_dev, B_[p], p, r, stream)
            fin = lat.field(p)
            Q.qcd_pack_field(lat.handle, fin, b_dev, Q.QCD_EVEN, p, stream)
            fouts = [lat.field(p), lat2.field(p)]
            for k in range(4):  # warm-up
                Q.qcd_dslash((lat, lat2)[k & 1].handle, fouts[k & 1], fin, Q.QCD_ODD, p, stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(n_op):
            Q.qcd_dslash((lat, lat2)[k & 1].handle, fouts[k & 1], fin, Q.QCD_ODD, p, stream)
        e1.record(stream)
        e1.synchronize()
        t_us = e0.elapsed_time(e1) * 1e3 / n_op
        link_b, fld_b, _ = OP_BYTES[name]
        bps = link_b + 2 * fld_b
        gbs = bps * Vh / (t_us * 1e-6) / 1e9
        tf = FLOP_PER_SITE * Vh / (t_us * 1e-6) / 1e12
        o = {"us_per_launch": round(t_us, 3), "gflops": round(tf * 1e3, 1), "alg_bytes_per_site": bps,
             "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / hbm_peak, 4)}
        if name == "double":
            o.update({"frac_fp64_peak_derived": round(tf / FP64_PEAK_TFLOPS, 4),
                      "frac_fp64_peak_measured_dgemm": round(tf / fp64_meas, 4),
                      "bound": "FP64 pipe (570 flop vs 1248 B per site; the FP64 pipe caps it near "
                               f"{FP64_PEAK_TFLOPS / FLOP_PER_SITE * 1e3 * bps:.0f} GB/s)"})
        elif name == "df64":
            o["note"] = ("df64 = float-float pairs (48-bit significand, FP32's 8-bit exponent): an inner-solver "
                         "precision narrower than FP64, run on the FP32 pipes")
        operators[name] = o
        del fin, fouts
    del lat2, bufs2

    # ---- roofline of the dominant kernel family: every kernel of the timed step's CG iterations (K1,
    # K2 and, unless K1 forms p itself, the p update) and the FP64 operator launches of the reliable
    # updates, y and the true residual, charged with ALL of the step's time: a lower bound on their
    # rate that agrees by construction with the step time.
    i = infos[-1]
    n32 = 2 * i["iterations"]
    n_all = _half_dslash_count(i)
    n64 = n_all - n32
    k1_in, k2_in = _k1_k2_bytes(head, folded=folded)
    k3_in = 0 if folded else 3 * OP_BYTES[head][1]  # p = r + beta p: r, p read, p written
    k1_64, k2_64 = _k1_k2_bytes("double")
    alg_step = Vh * (i["iterations"] * (k1_in + k2_in + k3_in) + n64 / 2 * (k1_64 + k2_64))
    per_launch_us = t_mixed * 1e3 / n_all
    achieved = alg_step / (t_mixed * 1e-3) / 1e9
    d_ms, d_n = infos_prof[-1]["dslash_ms"], infos_prof[-1]["dslash_launches"]
    roofline = {
        "bound": "hbm",
        "kernel": f"dslash_kernel (CG K1+K2 launches, {NAMES[head]}; FP64 in the reliable updates)"
                  + ("" if folded else " + cg_p_kernel"),
        "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
        "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
        "traffic": ncu_traffic(args.workload),
        "method": "all of the timed step's time charged to its CG kernels (a lower bound on their rate); bytes = "
                  "links and every vector read or written once per launch at the launch's precision"
                  + (" (the FP32 K1 also forms p = r + beta p: links + r + p_old + p + ap)" if folded else
                     " (K1 = links + p + ap, K2 = links + ap + p + r in/out + x in/out, p update = r + p in + p out)")
                  + "; traffic = ncu DRAM bytes per K1/K2 launch",
        "alg_bytes_per_site_k1_k2": [k1_in, k2_in], "alg_bytes_per_site_p_update": k3_in,
        "alg_bytes_per_site_k1_k2_fp64": [k1_64, k2_64],
        "alg_bytes_per_step": round(alg_step), "alg_bytes_per_launch_inner": (k1_in + k2_in) / 2 * Vh,
        "check": {"operator_launches": n_all, "inner_launches": n32, "fp64_launches": n64,
                  "per_launch_us": round(per_launch_us, 3),
                  "launches_x_per_launch_ms": round(n_all * per_launch_us / 1e3, 4),
                  "ms_per_step": round(t_mixed, 4),
                  "ok": bool(n_all * per_launch_us / 1e3 <= t_mixed * (1 + 1e-9))},
        "direct_launch_events": {"us_per_launch": round(d_ms / d_n * 1e3, 3), "launches": d_n,
                                 "note": "a separate pass of direct launches with CUDA events around each "
                                         "operator launch (includes event overhead)"}}

    # ---- config 4: the multi-RHS and many-lattice solves (their own lattices and sources)
    batched = {}
    if not args.no_batched and not args.no_legs:
        for key in BATCHED_LEGS:
            # launch shapes chosen by the library's autotuner first (outside the timed steps)
            bl = batched_leg(WORKLOADS[key], leg_steps if key.startswith("mrhs") else max(leg_steps, 5), 1, True,
                             key, world, local, fp64_steps=max(1, min(leg_steps, 2)), sample_clocks=False)
            batched[key] = {"workload": WORKLOADS[key]["desc"], "value": bl["value"], "unit": bl["unit"],
                            "ms_per_step": bl["ms_per_step"], "steps": bl["steps"], "cg": bl["cg"],
                            "roofline": bl["roofline"], "gpu_launches": bl["gpu_launches"], "tuned": bl["tuned"]}
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_mixed, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[head],
        "data": "synthetic (seeded Haar SU(3) links, Gaussian source)",
        "config": {"workload": wl["desc"], "dims": list(dims), "mass": mass, "tol": tol, "inner": head,
                   "reliable_update_interval": 100, "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "step": f"qcd_load_links (FP64 + {NAMES[head]}) + qcd_cg_solve (CG, y = D_oe x, FP64 true residual)",
                   "legs": f"the other solves, e2e and batched: {leg_steps} timed steps each after one untimed"},
        "cg": {"iterations": i["iterations"], "true_rel_residual": i["true_rel_residual"],
               "reliable_updates": i["reliable_updates"], "time_to_solution_ms": round(t_mixed, 4),
               "half_dslash_per_solve": n_all, "plain_fp64_ms": t_fp64,
               "speedup_vs_fp64": round(t_fp64 / t_mixed, 3) if t_fp64 else None,
               "speedup_vs_fp64_legs": {n: round(t_fp64 / l["ms_per_step"], 3) for n, l in legs.items()
                                        if n != "double"} if t_fp64 else None},
        "legs": legs,
        "accuracy": accuracy,
        "roofline": roofline,
        "operators": operators,
        "fp64_peak": {"derived_tflops": round(FP64_PEAK_TFLOPS, 4),
                      "measured_dgemm_tflops": round(fp64_meas, 4) if fp64_meas else None,
                      "note": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz; measured: cuBLAS DGEMM 4096^3 "
                              "(torch.matmul float64), best of 3"},
        "batched": batched,
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(U_host.numel() * 16 + b_host.numel() * 16),
                "d2h_bytes_per_step": int(x_host.numel() * 16 + y_host.numel() * 16),
                "ms_per_step": round(total_e2e / len(ms_e2e), 4), "steps": len(ms_e2e)},
        "gpu_launches": int(sum(i_["launches"] for i_ in infos)),
        "clocks": clocks,
        "wall_s_timed_region": round(t_wall, 4),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_all_cores(wl, U, b)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_gpu_batched(args, wl):
    """Multi-RHS (one lattice, nrhs sources) or multi-lattice (one persistent launch) workloads.

    One step = pack every lattice's links (FP64 + inner precision) and run the batched mixed
    solve. Reported beside: the same problems solved one by one with plain FP64 CG on the GPU
    (time and the speedup of the batched mixed solve over it).
    """
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    out = batched_leg(wl, args.steps, args.warmup, args.tune, args.workload, world, local,
                      fp64_steps=0 if args.no_legs else 3)
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def batched_leg(wl, steps, warmup, tune, workload_key, world=1, local=0, fp64_steps=3, sample_clocks=True):
    """The multi-RHS or many-lattice solve of `wl`: `warmup` untimed and `steps` timed steps (L2
    flushed before each), then the same problems one by one with plain FP64 CG (`fp64_steps` timed
    after one untimed). Returns the bench line's fields (whole-job value over ranks)."""
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    inner = wl["inner"]
    prec_in, recon_in = PRECS[inner]
    tol = wl["tol"]
    stream = torch.cuda.Stream()
    if wl["kind_solve"] == "mrhs":
        specs = [(wl["dims"], wl["mass"], 1, None)]
        nrhs = wl["nrhs"]
    else:
        specs = I.make_lattice_batch(wl["n"], seed=4)
        nrhs = 1
    lats, U_dev, b_dev, x_dev, packed = [], [], [], [], []
    for dims, m, ls, ss in specs:
        lat = Q.Lattice(dims)
        lats.append(lat)
        U_dev.append(torch.from_numpy(I.make_links(dims, kind="haar", seed=ls)).cuda())
        if nrhs > 1:
            b_dev.append(torch.from_numpy(I.make_sources(dims, nrhs, first_seed=2)).cuda())
        else:
            b_dev.append(torch.from_numpy(I.make_source(dims, seed=ss)).cuda())
        x_dev.append(torch.zeros_like(b_dev[-1]))
        packed.append([(p, r, lat.empty_bytes(Q.qcd_links_bytes(lat.handle, p, r))) for p, r in
                       sorted({(0, 18), (prec_in, recon_in)})])
    masses = [s[1] for s in specs]
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = prec_in, recon_in
    if wl["kind_solve"] == "mrhs":
        ws = lats[0].workspace(opts, nrhs)
    else:
        ws = torch.empty(Q.qcd_workspace_bytes_batched([l.handle for l in lats], opts), dtype=torch.uint8, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def load_links():
        n = 0
        for lat, Ud, pk in zip(lats, U_dev, packed):
            for p, r, buf in pk:
                Q.qcd_load_links(lat.handle, Ud, buf, p, r, stream)
                n += 1
        return n

    def step():
        with torch.cuda.stream(stream):
            n = load_links()
            if wl["kind_solve"] == "mrhs":
                rc, infos = Q.qcd_cg_solve_mrhs(lats[0].handle, nrhs, x_dev[0], b_dev[0], masses[0], tol, 100000, opts,
                                                ws, None, stream=stream)
                vh = [lats[0].Vh] * nrhs
            else:
                rc, infos = Q.qcd_cg_solve_batched([l.handle for l in lats], x_dev, b_dev, None, masses, tol, 100000,
                                                   opts, ws, stream=stream)
                vh = [l.Vh for l in lats]
        if rc != Q.QCD_OK:
            raise RuntimeError(f"batched solve failed: {Q.qcd_status_string(rc)}")
        flops = sum(FLOP_PER_SITE * v * _half_dslash_count(i) for v, i in zip(vh, infos))
        return flops, infos, n + sum(i["kernel_launches"] for i in infos)

    def timed(fn, n):
        ms, outs = [], []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            outs.append(fn())
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, outs

    tuned = None
    if tune:
        with torch.cuda.stream(stream):
            load_links()
            if wl["kind_solve"] == "mrhs":
                tuned = {"rhs_block": Q.qcd_tune_mrhs(lats[0].handle, nrhs, x_dev[0], b_dev[0], masses[0], opts, ws,
                                                      stream=stream)}
            else:
                c, blk = Q.qcd_tune_batched([l.handle for l in lats], x_dev, b_dev, masses, tol, 100000, opts, ws,
                                            stream=stream)
                tuned = {"cluster_size": c, "block_size": blk}
        torch.cuda.synchronize()
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = None
    if sample_clocks:
        proc, cpath = _clock_sampler(_device_uuid(local))
        time.sleep(0.3)
    ms, outs = timed(step, steps)
    if sample_clocks:
        clocks = _clock_summary(proc, cpath)

    # the same problems, one by one, with plain FP64 CG on the GPU
    o64 = Q.qcd_solver_opts_default()
    def fp64_step():
        with torch.cuda.stream(stream):
            for lat, Ud, pk in zip(lats, U_dev, packed):
                Q.qcd_load_links(lat.handle, Ud, pk[0][2], 0, 18, stream)
            for j, (lat, m) in enumerate(zip(lats, masses)):
                ws64 = lat.workspace(o64)
                for r in range(nrhs):
                    bj = b_dev[j][r] if nrhs > 1 else b_dev[j]
                    xj = x_dev[j][r] if nrhs > 1 else x_dev[j]
                    rc, _ = Q.qcd_cg_solve(lat.handle, xj, bj, m, tol, 100000, o64, ws64, None, stream=stream)
                    if rc != Q.QCD_OK:
                        raise RuntimeError("FP64 reference solve failed")
        return 0
    ms64 = []
    if fp64_steps > 0:
        fp64_step()
        ms64, _ = timed(fp64_step, fp64_steps)

    (t_all,), (fl_all,) = reduce_over_ranks([sum(ms)], [sum(o[0] for o in outs)])
    value = fl_all / (t_all * 1e-3) / 1e9
    infos = outs[-1][1]
    t_batched = sum(ms) / steps
    t_fp64 = sum(ms64) / len(ms64) if ms64 else None
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": round(t_batched, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[inner], "data": "synthetic (seeded Haar SU(3) links, Gaussian sources)",
        "config": {"workload": wl["desc"], "problems": len(specs) * nrhs, "tol": tol, "inner": inner,
                   "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "step": "qcd_load_links for every lattice + " +
                           ("qcd_cg_solve_mrhs" if nrhs > 1 else "qcd_cg_solve_batched (one persistent launch)")},
        "cg": {"time_to_solution_ms": round(t_batched, 4),
               "max_iterations": max(i["iterations"] for i in infos),
               "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
               "reliable_updates": sum(i["reliable_updates"] for i in infos),
               "plain_fp64_gpu_cg_ms": round(t_fp64, 4) if t_fp64 else None, "plain_fp64_steps": len(ms64),
               "speedup_vs_plain_fp64_gpu_cg": round(t_fp64 / t_batched, 3) if t_fp64 else None},
        "gpu_launches": int(sum(o[2] for o in outs)),
        "clocks": clocks,
        "tuned": tuned,
    }
    # roofline. Algorithmic bytes per output site of a half-lattice operator at the inner precision:
    # links once per launch (shared by every RHS), and per RHS K1 = p in + ap out, K2 = ap in, p in,
    # r and x read and written (x at FP32).
    link_b, fld_b, x_b = {"single18": (576, 24, 24), "single12": (384, 24, 24), "half12": (192, 16, 24)}[inner]
    k1_rhs = 2 * fld_b
    k2_rhs = fld_b + fld_b + 2 * fld_b + 2 * x_b
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if wl["kind_solve"] == "mrhs":
        opts.profile = 1
        _, outs_p = timed(step, 1)
        infos_p = outs_p[0][1]
        opts.profile = 0
        Vh = lats[0].Vh
        d_ms, d_n = infos_p[0]["dslash_ms"], infos_p[0]["dslash_launches"]
        pairs = max(i["iterations"] for i in infos_p)
        rhs_its = sum(i["iterations"] for i in infos_p)
        alg = Vh * (2 * link_b * pairs + (k1_rhs + k2_rhs) * rhs_its)
        ach = alg / (d_ms * 1e-3) / 1e9
        rb_used = (tuned or {}).get("rhs_block", -1 if nrhs >= 8 else 1)
        kname = "dslash_mrhs_shared_kernel" if rb_used == -1 else f"dslash_mrhs_cg_kernel (register block {rb_used})"
        out["roofline"] = {"bound": "hbm", "kernel": kname + " (K1+K2 launches)", "achieved": round(ach, 1),
                           "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                           "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)", "traffic": ncu_traffic(workload_key),
                           "alg_bytes_per_launch": round(alg / d_n), "avg_launch_us": round(d_ms / d_n * 1e3, 3),
                           "alg_bytes_per_site": {"links_per_launch": link_b, "k1_per_rhs": k1_rhs, "k2_per_rhs": k2_rhs},
                           "note": f"the links ({Q.qcd_links_bytes(lats[0].handle, prec_in, recon_in) / 1e6:.0f} MB) "
                                   "stay in L2 across the RHS blocks"}
    else:
        # one persistent launch does every solve: algorithmic bytes of all its operator applications
        # (2 per iteration per lattice) over the whole kernel time; the lattices (4^4..8^3x16) live in L2
        alg = sum(l.Vh * (2 * link_b + k1_rhs + k2_rhs) * i["iterations"] for l, i in zip(lats, infos))
        ach = alg / (t_batched * 1e-3) / 1e9
        out["roofline"] = {"bound": "latency", "kernel": "batched_cg_kernel (whole batch, one launch)",
                           "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                           "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)", "traffic": ncu_traffic(workload_key),
                           "alg_bytes_per_launch": round(alg),
                           "note": "L2-resident lattices; every CG step ends in a cluster barrier: latency-bound by design"}
    return out


WILSON_FLOP_PER_SITE = 1320


def _wilson_dw_count(info):
    """FP32/FP64 D_W applications of one RHS's CGNR: M and M^dagger per iteration, M^dagger b at
    start-up, M and M^dagger per reliable update (the convergence check included)."""
    return 2 * info["iterations"] + 1 + 2 * info["reliable_updates"]


def run_gpu_wilson(args, wl):
    """Wilson CGNR (M = 1 - kappa D_W on the full lattice) on nrhs right-hand sides in one multi-RHS
    solve. One step = pack the links at the outer precision (the workload's "outer": FP64 or df64)
    and at FP32, and run the mixed CGNR on every RHS; value = Wilson D_W GFLOP/s inside the solve
    (1320 flop per site per D_W application). The same RHS solved with the other outer precision and
    by plain FP64 CGNR on the GPU are timed beside."""
    import numpy as np
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims, kappa, tol, R = wl["dims"], wl["kappa"], wl["tol"], wl["nrhs"]
    stream = torch.cuda.Stream()
    lat = Q.Lattice(dims)
    V = lat.V
    U_np = I.make_links(dims, kind=wl["kind"], seed=1)
    U_host = torch.from_numpy(U_np).pin_memory()
    b_host = torch.from_numpy(np.stack([I.make_spinor(dims, seed=2 + k) for k in range(R)])).pin_memory()
    U_dev = U_host.to("cuda")
    b_dev = b_host.to("cuda")
    x_dev = torch.zeros_like(b_dev)
    x_host = torch.empty_like(b_host).pin_memory()
    outer = Q.PREC_NAMES[wl.get("outer", "double")]
    other = Q.QCD_PREC_DF64 if outer == Q.QCD_PREC_DOUBLE else Q.QCD_PREC_DOUBLE
    bufs = {p: lat.empty_bytes(Q.qcd_wilson_links_bytes(lat.handle, p)) for p in (0, 1, 3)}
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.prec_outer = 1, outer
    delta = args.reliable_delta if args.reliable_delta is not None else wl.get("reliable_delta")
    if delta is not None:
        opts.reliable_delta = delta
    ws = {1: lat.empty_bytes(Q.qcd_wilson_workspace_bytes(lat.handle, opts, R))}  # FP32 inner, either outer
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    launches_links = 2

    def solve(prec, host_io=False, profile=False, hi=None):
        # one step packs the links the solve reads: the inner precision and the outer one
        hi = (outer if hi is None else hi) if prec != 0 else 0
        opts.prec_inner, opts.prec_outer = prec, hi
        opts.profile = 1 if profile else 0
        with torch.cuda.stream(stream):
            if host_io:
                U_dev.copy_(U_host, non_blocking=True)
                b_dev.copy_(b_host, non_blocking=True)
            for p in sorted({prec, hi}):
                Q.qcd_wilson_load_links(lat.handle, U_dev, bufs[p], p, stream)
            rc, infos = Q.qcd_wilson_cgnr_mrhs(lat.handle, R, x_dev, b_dev, kappa, tol, 100000, opts, ws[prec],
                                               stream=stream)
            if host_io:
                x_host.copy_(x_dev, non_blocking=True)
        if rc != Q.QCD_OK:
            raise RuntimeError(f"Wilson CGNR failed: {Q.qcd_status_string(rc)} {infos}")
        return infos

    def timed(prec, n, host_io=False, profile=False, hi=None):
        ms, runs = [], []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            runs.append(solve(prec, host_io, profile, hi))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, runs

    def flops_of(runs):
        return sum(WILSON_FLOP_PER_SITE * V * _wilson_dw_count(i) for infos in runs for i in infos)

    for _ in range(args.warmup):
        solve(1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    proc, cpath = _clock_sampler(uuid)
    time.sleep(0.3)
    ms, runs = timed(1, args.steps)
    clocks = _clock_summary(proc, cpath)
    if world > 1:
        dist.barrier()
    ms_prof, runs_prof = timed(1, max(1, min(args.steps, 3)), profile=True)
    ms_e2e, runs_e2e = timed(1, args.steps, host_io=True)
    ms_oth, runs_oth = None, None
    if not args.no_variant and not args.no_legs:
        solve(1, hi=other)
        ms_oth, runs_oth = timed(1, max(1, min(args.steps, 2)), hi=other)
    ms64, runs64 = None, None
    if not args.no_legs:
        del ws[1]
        opts.prec_inner, opts.prec_outer = 0, 0
        ws[0] = lat.empty_bytes(Q.qcd_wilson_workspace_bytes(lat.handle, opts, R))
        solve(0)
        ms64, runs64 = timed(0, max(1, min(args.steps, 2)))

    # operator kernels alone (CUDA events on the launching stream, L2 flushed before each)
    with torch.cuda.stream(stream):
        for p in (0, 1, 3):
            Q.qcd_wilson_load_links(lat.handle, U_dev, bufs[p], p, stream)

    def op_time(prec, nrhs, reps=5):
        fb = Q.qcd_wilson_field_bytes(lat.handle, prec)
        fin, fout = lat.empty_bytes(nrhs * fb), lat.empty_bytes(nrhs * fb)
        with torch.cuda.stream(stream):
            for k in range(nrhs):
                Q.qcd_wilson_pack_field(lat.handle, fin[k * fb:(k + 1) * fb], b_dev[k], prec, stream)
        t = []
        for _ in range(reps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if nrhs == 1:
                Q.qcd_wilson_op(lat.handle, fout, fin, kappa, Q.QCD_WILSON_M, prec, stream)
            else:
                Q.qcd_wilson_op_mrhs(lat.handle, fout, fin, nrhs, kappa, Q.QCD_WILSON_M, prec, stream)
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.median(t)

    if args.no_legs:
        t_op64 = t_opdf = t_op32 = t_op32_r = float("nan")
    else:
        t_op64 = op_time(0, 1)
        t_opdf = op_time(3, 1)
        t_op32 = op_time(1, 1)
        t_op32_r = op_time(1, R) if R > 1 else t_op32

    (total_ms, total_ms_e2e), (fl0, fl1) = reduce_over_ranks([sum(ms), sum(ms_e2e)],
                                                              [flops_of(runs), flops_of(runs_e2e)])
    value = fl0 / (total_ms * 1e-3) / 1e9
    e2e_value = fl1 / (total_ms_e2e * 1e-3) / 1e9
    t_mixed = sum(ms) / len(ms)
    t_64 = sum(ms64) / len(ms64) if ms64 else float("nan")

    # roofline of the FP32 operator launches inside the solve (K1: t = M p, K2: M^dagger t + update).
    # Algorithmic bytes: the links once per launch (4 links x 72 B per site, FP32 recon-18) and, per
    # running RHS and site, K1 = p (in) + t (out) = 192 B, K2 = t (in) + p + r, x (read, written) = 576 B.
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    link_b, k1_b, k2_b = 288, 192, 576
    d_ms = sum(infos[0]["dslash_ms"] for infos in runs_prof)
    d_launches = sum(infos[0]["dslash_launches"] for infos in runs_prof)
    pairs = sum(max(i["iterations"] for i in infos) for infos in runs_prof)
    rhs_its = sum(i["iterations"] for infos in runs_prof for i in infos)
    alg = V * (2 * link_b * pairs + (k1_b + k2_b) * rhs_its)
    achieved = alg / (d_ms * 1e-3) / 1e9
    op_flops = WILSON_FLOP_PER_SITE * V
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_mixed, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 reliable updates)" if outer == 0 else "f32 (df64 reliable updates)",
        "data": "synthetic (seeded Haar SU(3) links, Gaussian spinors)",
        "config": {"workload": wl["desc"], "dims": list(dims), "kappa": kappa, "tol": tol, "nrhs": R,
                   "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "outer": wl.get("outer", "double"), "reliable_delta": opts.reliable_delta,
                   "step": "qcd_wilson_load_links (" + ("FP64" if outer == 0 else "df64") +
                           " + FP32) + qcd_wilson_cgnr_mrhs"},
        "cg": {"iterations": [i["iterations"] for i in runs[-1]],
               "reliable_updates": [i["reliable_updates"] for i in runs[-1]],
               "max_true_rel_residual": max(i["true_rel_residual"] for i in runs[-1]),
               "time_to_solution_ms": round(t_mixed, 4), "plain_fp64_cgnr_ms": round(t_64, 4) if ms64 else None,
               "plain_fp64_iterations": [i["iterations"] for i in runs64[-1]] if runs64 else None,
               "speedup_vs_plain_fp64_cgnr": round(t_64 / t_mixed, 3) if ms64 else None},
        "roofline": {"bound": "hbm", "kernel": "wilson_mrhs_kernel (CGNR K1+K2 launches, FP32)",
                     "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
                     "traffic": ncu_traffic(wl.get("traffic_key", args.workload)),
                     "alg_bytes_per_launch": round(alg / d_launches),
                     "alg_bytes_per_site": {"links_per_launch": link_b, "k1_per_rhs": k1_b, "k2_per_rhs": k2_b},
                     "avg_launch_us": round(d_ms / d_launches * 1e3, 3)},
        "operator_alone": {
            "fp32_M_1rhs": {"us": round(t_op32 * 1e3, 2), "gbs": round(480 * V / (t_op32 * 1e-3) / 1e9, 1),
                            "frac_hbm": round(480 * V / (t_op32 * 1e-3) / 1e9 / hbm_peak, 4),
                            "alg_bytes_per_site": 480},
            f"fp32_M_{R}rhs": {"us": round(t_op32_r * 1e3, 2),
                               "gbs": round((288 + 192 * R) * V / (t_op32_r * 1e-3) / 1e9, 1),
                               "frac_hbm": round((288 + 192 * R) * V / (t_op32_r * 1e-3) / 1e9 / hbm_peak, 4),
                               "alg_bytes_per_site": 288 + 192 * R},
            "fp64_M_1rhs": {"us": round(t_op64 * 1e3, 2), "tflops": round(op_flops / (t_op64 * 1e-3) / 1e12, 4),
                            "frac_fp64_peak": round(op_flops / (t_op64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                            "note": "FP64 D_W is FP64-pipe bound on GB300 (1320 flop vs 960 B per site)"},
            "df64_M_1rhs": {"us": round(t_opdf * 1e3, 2),
                            "gbs": round(960 * V / (t_opdf * 1e-3) / 1e9, 1),
                            "frac_hbm": round(960 * V / (t_opdf * 1e-3) / 1e9 / hbm_peak, 4),
                            "alg_bytes_per_site": 960,
                            "speedup_vs_fp64_M": round(t_op64 / t_opdf, 3),
                            "note": "df64 D_W: FP32 pairs on the FP32 pipes, 960 B per site like FP64"}},
        "other_outer_precision": None if ms_oth is None else {
            "outer": "df64" if other == Q.QCD_PREC_DF64 else "double",
            "ms_per_step": round(sum(ms_oth) / len(ms_oth), 4),
            "value": round(flops_of(runs_oth) / (sum(ms_oth) * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
            "iterations": [i["iterations"] for i in runs_oth[-1]],
            "reliable_updates": [i["reliable_updates"] for i in runs_oth[-1]],
            "max_true_rel_residual": max(i["true_rel_residual"] for i in runs_oth[-1]),
            "time_ratio_vs_headline": round((sum(ms_oth) / len(ms_oth)) / t_mixed, 3)},
        "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": int(U_host.numel() * 16 + b_host.numel() * 16),
                "d2h_bytes_per_step": int(x_host.numel() * 16), "ms_per_step": round(total_ms_e2e / args.steps, 4)},
        "gpu_launches": int(sum(launches_links + infos[0]["kernel_launches"] for infos in runs)),
        "clocks": clocks,
        "ms_per_step_profiled": round(sum(ms_prof) / len(ms_prof), 4),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = wilson_cpu_baseline(wl, U_np, b_host[0].numpy())
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def run_gpu_full(args, wl):
    """Full-system solve M x = b on both parities (qcd_solve_full: even-odd reduction onto the CG,
    odd half reconstructed, full FP64 residual |b - M x| / |b|). One step = qcd_load_links + the solve;
    value = Dslash GFLOP/s (570 flop per output site of every half-lattice operator application:
    those of the even CG plus the source b', and the two of the final full residual)."""
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims, mass, tol, inner = wl["dims"], wl["mass"], wl["tol"], wl["inner"]
    prec_in, recon_in = PRECS[inner]
    stream = torch.cuda.Stream()
    lat = Q.Lattice(dims)
    Vh = lat.Vh
    U_np = I.make_links(dims, kind="haar", seed=1)
    b_np = I.make_source(dims, seed=2)
    U_host, b_host = torch.from_numpy(U_np).pin_memory(), torch.from_numpy(b_np).pin_memory()
    U_dev, b_dev = U_host.to("cuda"), b_host.to("cuda")
    x_dev = torch.zeros_like(b_dev)
    x_host = torch.empty_like(b_host).pin_memory()
    packed = {p: (lat.empty_bytes(Q.qcd_links_bytes(lat.handle, p, r)), r) for p, r in {(0, 18), (prec_in, recon_in)}}
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = prec_in, recon_in
    ws = lat.empty_bytes(Q.qcd_workspace_bytes_full(lat.handle, opts))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step(host_io=False, profile=False):
        opts.profile = 1 if profile else 0
        with torch.cuda.stream(stream):
            if host_io:
                U_dev.copy_(U_host, non_blocking=True)
                b_dev.copy_(b_host, non_blocking=True)
            for p, (buf, r) in packed.items():
                Q.qcd_load_links(lat.handle, U_dev, buf, p, r, stream)
            rc, info = Q.qcd_solve_full(lat.handle, x_dev, b_dev, mass, tol, 100000, opts, ws, stream=stream)
            if host_io:
                x_host.copy_(x_dev, non_blocking=True)
        if rc != Q.QCD_OK:
            raise RuntimeError(f"full solve failed: {Q.qcd_status_string(rc)} {info}")
        return info

    def timed(n, host_io=False, profile=False):
        ms, infos = [], []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step(host_io, profile))
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, infos

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    proc, cpath = _clock_sampler(uuid)
    time.sleep(0.3)
    ms, infos = timed(args.steps)
    clocks = _clock_summary(proc, cpath)
    _, infos_p = timed(max(1, min(args.steps, 2)), profile=True)
    ms_e2e, infos_e2e = timed(args.steps, host_io=True)

    def flops(i):
        return FLOP_PER_SITE * Vh * (_half_dslash_count(i) + 3)

    (t_ms, t_e2e), (f_all, f_e2e) = reduce_over_ranks([sum(ms), sum(ms_e2e)],
                                                       [sum(flops(i) for i in infos), sum(flops(i) for i in infos_e2e)])
    link_b, fld_b, x_b = {"double": (1152, 48, 48), "single18": (576, 24, 24), "single12": (384, 24, 24),
                          "half12": (192, 16, 24), "df64": (1152, 48, 48)}[inner]
    k1_b, k2_b = link_b + 2 * fld_b, link_b + fld_b + 2 * fld_b + x_b + fld_b + x_b
    per_ms = sum(i["dslash_ms"] for i in infos_p) / sum(i["dslash_launches"] for i in infos_p)
    alg = (k1_b + k2_b) / 2 * Vh
    ach = alg / (per_ms * 1e-3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    out = {
        "metric": METRIC, "value": round(f_all / (t_ms * 1e-3) / 1e9, 2), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[inner], "data": "synthetic (seeded Haar SU(3) links, Gaussian source)",
        "config": {"workload": wl["desc"], "dims": list(dims), "mass": mass, "tol": tol, "inner": inner,
                   "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "step": "qcd_load_links + qcd_solve_full (both parities, full FP64 residual)"},
        "cg": {"iterations": infos[-1]["iterations"], "full_rel_residual": infos[-1]["true_rel_residual"],
               "reliable_updates": infos[-1]["reliable_updates"], "time_to_solution_ms": round(t_ms / args.steps, 4)},
        "roofline": {"bound": "hbm", "kernel": "dslash_kernel (K1+K2 launches of the even CG)", "achieved": round(ach, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                     "peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)", "traffic": ncu_traffic(args.workload),
                     "alg_bytes_per_launch": alg, "avg_launch_us": round(per_ms * 1e3, 3)},
        "e2e": {"value": round(f_e2e / (t_e2e * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int((U_host.numel() + b_host.numel()) * 16), "d2h_bytes_per_step": int(x_host.numel() * 16),
                "ms_per_step": round(t_e2e / args.steps, 4)},
        "gpu_launches": int(sum(len(packed) + i["kernel_launches"] for i in infos)),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import staggered as So
        t0 = time.perf_counter()
        res = So.solve_full(U_np, b_np, dims, mass, tol, 6)
        dt = time.perf_counter() - t0
        # the oracle's full-lattice CG: 2 full D (= 4 half-lattice operators) per iteration, 1 for M^dagger b,
        # 3 for the final residuals
        f_cpu = FLOP_PER_SITE * Vh * (4 * res["iterations"] + 2 + 6)
        out["cpu_baseline"] = {"value": round(f_cpu / dt / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": f"FP64 numpy oracle full-lattice CG on the same {tuple(dims)} workload, first "
                                         f"{res['iterations']} iterations + residuals ({dt:.1f} s)"}
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


FORCE_FLOP_PER_LINK = 162  # U b (66) + a b^dagger (54) + coefficient (6) + i (W - W^dagger) (18) + trace removal (18)


def run_gpu_force(args, wl):
    """The fermion force on every link of the lattice from the CG's x and y = D_oe x (a mixed CG
    solve produces them once, outside the timed region). One step = qcd_fermion_force on the whole
    lattice; value = GFLOP/s at 162 flop per link; the kernel is bound by the FP64 pipe on GB300."""
    import numpy as np
    import torch

    from paper_1311_2719_gb300 import inputs as I
    from paper_1311_2719_gb300 import qcd as Q

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dims, mass = wl["dims"], wl["mass"]
    stream = torch.cuda.Stream()
    lat = Q.Lattice(dims)
    V = lat.V
    U_np = I.make_links(dims, kind="haar", seed=1)
    U_host = torch.from_numpy(U_np).pin_memory()
    U_dev = U_host.to("cuda")
    b_dev = torch.from_numpy(I.make_source(dims, seed=2)).cuda()
    x_dev, y_dev = torch.zeros_like(b_dev), torch.zeros_like(b_dev)
    for p, r in ((0, 18), (1, 12)):
        lat.load_links(U_dev, p, r)
    opts = Q.qcd_solver_opts_default()
    opts.prec_inner, opts.recon_inner = 1, 12
    ws = lat.workspace(opts)
    with torch.cuda.stream(stream):
        rc, info = Q.qcd_cg_solve(lat.handle, x_dev, b_dev, mass, 1e-10, 100000, opts, ws, y_dev, stream=stream)
    if rc != Q.QCD_OK:
        raise RuntimeError(f"CG for the force inputs failed: {Q.qcd_status_string(rc)}")
    del ws
    x_host = x_dev.cpu().pin_memory()
    y_host = y_dev.cpu().pin_memory()
    f_dev = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
    f_host = torch.empty((V, 4, 3, 3), dtype=torch.complex128).pin_memory()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def step(host_io=False):
        with torch.cuda.stream(stream):
            if host_io:
                U_dev.copy_(U_host, non_blocking=True)
                x_dev.copy_(x_host, non_blocking=True)
                y_dev.copy_(y_host, non_blocking=True)
            Q.qcd_fermion_force(lat.handle, f_dev, U_dev, x_dev, y_dev, stream)
            if host_io:
                f_host.copy_(f_dev, non_blocking=True)

    def timed(n, host_io=False):
        ms = []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(host_io)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    proc, cpath = _clock_sampler(uuid)
    time.sleep(0.3)
    ms = timed(args.steps)
    clocks = _clock_summary(proc, cpath)
    ms_e2e = timed(args.steps, host_io=True)
    flops = FORCE_FLOP_PER_LINK * 4 * V
    (t_ms, t_e2e), (fl_all,) = reduce_over_ranks([sum(ms), sum(ms_e2e)], [args.steps * flops])
    value = fl_all / (t_ms * 1e-3) / 1e9
    per = t_ms / args.steps
    achieved = flops / (per * 1e-3) / 1e12
    alg_bytes = 1200 * V  # links 576 + force 576 + the site's own x or y 48 B per site
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(per, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Haar SU(3) links, Gaussian source; x, y from the CG)",
        "config": {"workload": wl["desc"], "dims": list(dims), "mass": mass, "parallelism": f"replicas x{world} (no sharding)",
                   "l2": "flushed before every step (512 MB write, outside the timed events)",
                   "step": "qcd_fermion_force (every link)"},
        "roofline": {"bound": "alu", "kernel": "force_kernel", "achieved": round(achieved, 4),
                     "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4),
                     "peak_source": "derived FP64 FMA peak (152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz)",
                     "traffic": ncu_traffic(args.workload), "alg_bytes_per_launch": alg_bytes,
                     "hbm_model_gbs": round(alg_bytes / (per * 1e-3) / 1e9, 1),
                     "hbm_model_frac": round(alg_bytes / (per * 1e-3) / 1e9 / hbm_peak, 4),
                     "alg_flops_per_launch": flops, "avg_launch_us": round(per * 1e3, 3)},
        "e2e": {"value": round(fl_all / (t_e2e * 1e-3) / 1e9, 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int((U_host.numel() + x_host.numel() + y_host.numel()) * 16),
                "d2h_bytes_per_step": int(f_host.numel() * 16), "ms_per_step": round(t_e2e / args.steps, 4)},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "cg_for_inputs": {"iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"]},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import force as Fo
        t0 = time.perf_counter()
        Fo.fermion_force(U_np, x_host.numpy(), y_host.numpy(), dims)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(flops / dt / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                               "sample": f"FP64 numpy oracle: the force on every link of the {dims} lattice ({dt:.1f} s), "
                                         f"{FORCE_FLOP_PER_LINK} flop/link"}
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def _wilson_oracle_sample(wl, U=None, b=None):
    """One application of M = 1 - kappa D_W by the FP64 oracle on the full lattice (flops, seconds)."""
    from oracle import wilson as Wo
    from paper_1311_2719_gb300 import inputs as I

    dims = wl["dims"]
    if U is None:
        U = I.make_links(dims, kind=wl["kind"], seed=1)
        b = I.make_spinor(dims, seed=2)
    t0 = time.perf_counter()
    Wo.apply_m(U, b, dims, wl["kappa"])
    dt = time.perf_counter() - t0
    return WILSON_FLOP_PER_SITE * U.shape[0], dt


def wilson_cpu_baseline(wl, U=None, b=None):
    f, dt = _wilson_oracle_sample(wl, U, b)
    return {"value": round(f / dt / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle: one M = 1 - kappa D_W application on the full {wl['dims']} lattice "
                      f"({dt:.1f} s), 1320 flop/site"}


def _oracle_sample(wl, iters, U=None, b=None):
    """Time the FP64 oracle CG, as it stands, for `iters` iterations of the workload."""
    from oracle import staggered as S
    from paper_1311_2719_gb300 import inputs as I

    dims = wl["dims"]
    if U is None:
        U = I.make_links(dims, kind=wl["kind"], seed=1)
        b = I.make_source(dims, seed=2)
    t0 = time.perf_counter()
    res = S.cg_solve(U, b, dims, wl["mass"], wl["tol"], iters)
    dt = time.perf_counter() - t0
    Vh = U.shape[0] // 2
    flops = FLOP_PER_SITE * Vh * (2 * res["iterations"] + 2)
    return flops, dt, res["iterations"]


def cpu_baseline(wl, iters):
    flops, dt, n = _oracle_sample(wl, iters)
    return {"value": round(flops / dt / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle CG on the same {wl['dims']} workload, first {n} iterations + y + true "
                      f"residual ({dt:.1f} s), algorithmic 570 flop/site per half-lattice operator"}


# ---- the FP64 oracle on all host cores: one process per core (spawned, never forked after the GPU
# is in use), each applying the oracle's normal operator A = m^2 - D_eo D_oe (its site-local form)
# to a slice of the even sites of the same lattice; the links and the source are shared read-only
# through a memory-mapped file.
_ORACLE_SHARED = {}


def _oracle_worker_init(path_u, path_b, dims, mass):
    _ORACLE_SHARED.update(U=np.load(path_u, mmap_mode="r"), b=np.load(path_b, mmap_mode="r"), dims=tuple(dims),
                          mass=mass)


def _oracle_worker_apply(sites):
    from oracle import staggered as S
    d = _ORACLE_SHARED
    S.mdagm_sites(d["U"], d["b"], d["dims"], d["mass"], sites)
    return len(sites)


class OraclePool:
    """`cores` oracle processes over the even sites of one lattice; pass() applies A everywhere once."""

    def __init__(self, U, b, dims, mass, cores=None):
        import multiprocessing as mp
        from oracle import staggered as S
        self.cores = cores or os.cpu_count() or 1
        self.dir = tempfile.mkdtemp(prefix="oracle_")
        pu, pb = os.path.join(self.dir, "U.npy"), os.path.join(self.dir, "b.npy")
        np.save(pu, U)
        np.save(pb, b)
        V = U.shape[0]
        even = np.nonzero(S.parity_of_sites(dims, np.arange(V)) == 0)[0]
        self.n_even = len(even)
        self.slices = np.array_split(even, self.cores)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"  # one thread per process: the process count is the core count
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_worker_init,
                                                     initargs=(pu, pb, tuple(dims), mass))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run_pass(self):
        t0 = time.perf_counter()
        done = sum(self.pool.map(_oracle_worker_apply, self.slices, chunksize=1))
        return 2 * FLOP_PER_SITE * done, time.perf_counter() - t0

    def close(self):
        import shutil
        self.pool.close()
        self.pool.join()
        shutil.rmtree(self.dir, ignore_errors=True)


def cpu_baseline_all_cores(wl, U, b, min_seconds=8.0):
    """The oracle as it stands on the host: all cores (one process each) applying A over the whole
    lattice, repeated for at least `min_seconds`; and, beside it, one thread running the oracle CG
    (first iteration + y + true residual) on the same lattice."""
    pool = OraclePool(U, b, wl["dims"], wl["mass"])
    try:
        pool.run_pass()  # warm-up: worker start-up, page-in of the mapped links
        fl, dt, passes = 0.0, 0.0, 0
        while dt < min_seconds:
            f, t = pool.run_pass()
            fl, dt, passes = fl + f, dt + t, passes + 1
    finally:
        pool.close()
    f1, dt1, n1 = _oracle_sample(wl, 1, U, b)
    return {"value": round(fl / dt / 1e9, 4), "unit": "GFLOP/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"FP64 numpy oracle normal operator A = m^2 - D_eo D_oe (site-local form) over all "
                      f"{pool.n_even} even sites of the {tuple(wl['dims'])} lattice, {passes} passes ({dt:.1f} s) on "
                      f"{pool.cores} processes of one thread; 1140 flop per even site",
            "single_thread": {"value": round(f1 / dt1 / 1e9, 4), "unit": "GFLOP/s", "cores": 1,
                              "sample": f"FP64 numpy oracle CG on the same lattice: {n1} iteration + y + true "
                                        f"residual ({dt1:.1f} s), 570 flop/site per half-lattice operator"}}


def run_reference(args, wl):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload per step (rank 0 only)."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return None
    from paper_1311_2719_gb300 import inputs as I

    kind = wl.get("kind_solve")
    if kind == "mixed32":
        dims = wl["dims"]
        U = I.make_links(dims, kind=wl["kind"], seed=1)
        b = I.make_source(dims, seed=2)
        pool = OraclePool(U, b, dims, wl["mass"])
        pool.run_pass()
        for _ in range(args.warmup):
            pool.run_pass()
        tot_f, tot_t = 0.0, 0.0
        for _ in range(args.steps):
            f, t = pool.run_pass()
            tot_f, tot_t = tot_f + f, tot_t + t
        pool.close()
        v = tot_f / tot_t / 1e9
        what = (f"each step: FP64 numpy oracle normal operator A = m^2 - D_eo D_oe (site-local form) over all "
                f"{pool.n_even} even sites of the {dims} lattice, on {pool.cores} processes of one thread; "
                f"1140 flop per even site")
        return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t / args.steps * 1e3, 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Haar SU(3) links, Gaussian source)",
                "config": {"workload": wl["desc"], "tol": wl["tol"], "dims": list(dims), "mass": wl["mass"],
                           "parallelism": "cpu oracle, rank 0 only"},
                "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": pool.cores, "kind": "oracle",
                                 "sample": what},
                "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if kind == "wilson":
        from oracle import wilson as Wo
        dims = wl["dims"]
        U = I.make_links(dims, kind=wl["kind"], seed=1)
        b = I.make_spinor(dims, seed=2)
        sites = np.arange(0, U.shape[0], 32)

        def sample():
            t0 = time.perf_counter()
            Wo.dslash_w_sites(U, b, dims, sites)
            return WILSON_FLOP_PER_SITE * len(sites), time.perf_counter() - t0

        what = (f"each step: FP64 numpy oracle Wilson D_W at every 32nd site ({len(sites)} sites) of the {dims} "
                f"lattice, 1320 flop/site, 1 thread")
        cfg = {"dims": list(dims), "kappa": wl["kappa"], "nrhs": wl["nrhs"]}
    elif kind == "force":
        from oracle import force as Fo
        dims = wl["dims"]
        U = I.make_links(dims, kind="haar", seed=1)
        x, y = I.make_source(dims, seed=2), I.make_source(dims, seed=3)
        V = U.shape[0]
        sites = np.arange(0, V, 64)
        sites4 = np.repeat(sites, 4)
        mus4 = np.tile(np.arange(4), len(sites))

        def sample():
            t0 = time.perf_counter()
            Fo.fermion_force_links(U, x, y, dims, sites4, mus4)
            return FORCE_FLOP_PER_LINK * len(sites4), time.perf_counter() - t0

        what = (f"each step: FP64 numpy oracle force on the links of every 64th site ({len(sites)} sites) of the "
                f"{dims} lattice, {FORCE_FLOP_PER_LINK} flop/link, 1 thread")
        cfg = {"dims": list(dims), "mass": wl["mass"]}
    else:
        if kind == "batched":  # the largest lattice of the batch stands in for the batch
            spec = max(I.make_lattice_batch(wl["n"], seed=4), key=lambda t: int(np.prod(t[0])))
            owl = dict(dims=spec[0], kind="haar", mass=spec[1], tol=wl["tol"])
            U = I.make_links(spec[0], kind="haar", seed=spec[2])
            b = I.make_source(spec[0], seed=spec[3])
        else:
            owl = wl
            U = I.make_links(wl["dims"], kind=wl["kind"], seed=1)
            b = I.make_source(wl["dims"], seed=2)
        n_it = [0]

        def sample():
            f, t, n_it[0] = _oracle_sample(owl, args.ref_iters, U, b)
            return f, t

        what = (f"each step: FP64 numpy oracle CG on the {tuple(owl['dims'])} lattice for {args.ref_iters} iterations "
                f"+ y + true residual (bounded sample), 1 thread")
        cfg = {"dims": list(owl["dims"]), "mass": owl["mass"]}
    for _ in range(args.warmup):
        sample()
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t = sample()
        tot_f += f
        tot_t += t
    v = tot_f / tot_t / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tot_t / args.steps * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Haar SU(3) links, Gaussian source)",
            "config": dict({"workload": wl["desc"], "tol": wl["tol"], "parallelism": "cpu oracle, rank 0 only"}, **cfg),
            "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": what},
            "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-iters", type=int, default=64, help="oracle CG iterations timed for cpu_baseline")
    ap.add_argument("--ref-iters", type=int, default=12, help="oracle CG iterations per --impl reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", action="store_true", help="run the autotuner before the batched workloads")
    ap.add_argument("--no-variant", action="store_true", help="skip the df64 run beside an FP64 workload")
    ap.add_argument("--leg-steps", type=int, default=3,
                    help="timed steps of each side measurement of the cg32_mixed workload (after one untimed)")
    ap.add_argument("--no-batched", action="store_true", help="cg32_mixed: skip the batched solves")
    ap.add_argument("--no-legs", action="store_true",
                    help="the headline solve only (cg32_mixed: no other precisions, operators or batched solves; "
                         "batched workloads: no one-by-one FP64 comparison), for counter captures")
    ap.add_argument("--reliable-delta", type=float, default=None,
                    help="mixed Wilson CGNR: reliable-update threshold (default: the workload's, else the library's)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        out = run_reference(args, wl)
    elif wl.get("kind_solve") == "mixed32":
        out = run_gpu_mixed32(args, wl)
    elif wl.get("kind_solve") in ("mrhs", "batched"):
        out = run_gpu_batched(args, wl)
    elif wl.get("kind_solve") == "wilson":
        out = run_gpu_wilson(args, wl)
    elif wl.get("kind_solve") == "force":
        out = run_gpu_force(args, wl)
    elif wl.get("kind_solve") == "full":
        out = run_gpu_full(args, wl)
    else:
        out = run_gpu(args, wl)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
