"""Benchmark of the EM-stack colour correction (smoothing + per-slice screened-Poisson solve).

One step = one emfuse_correct_stack call on a synthetic stack of 64 slices of 2048 x 2048
float32 (seeded generator shaped like the paper's EM data): anisotropic smoothing along z,
then every slice solved to relative residual 1e-6 with FP32 multigrid V-cycles inside FP64
defect correction.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--alpha A] [--impl reference]

`--impl reference` times the CPU FP64 oracle (NumPy/SciPy) on the host cores on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank corrects its own stack
(independent problems, no collective on the data path: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NZ, NY, NX = 64, 2048, 2048
SEED = 1  # seed of the 64 x 2048^2 workload
METRIC = "voxels/sec corrected at rel. residual 1e-6"
WORKLOAD = "64 slices x 2048 x 2048 fp32, sigma_xy=1, sigma_z=3, FP32 multigrid + FP64 defect correction to rel. residual 1e-6"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--alpha", type=float, default=1e-3)
    p.add_argument("--impl", default="emfuse", choices=["emfuse", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--tile-rows", type=int, default=0,
                   help="rows per work item of the finest level's wavefront kernels (0 = chosen; "
                        "for profiling smaller stacks with the 64-slice step's items)")
    p.add_argument("--no-graphs", action="store_true",
                   help="launch every solver kernel directly instead of replaying CUDA graphs (for "
                        "profilers that do not look inside graphs with conditional nodes)")
    p.add_argument("--nz", type=int, default=NZ, help="slices (smaller stacks for profiling only)")
    p.add_argument("--paper-scale", type=int, default=0, metavar="NZ",
                   help="instead: stream NZ paper-scale slices (21504 x 26624 uint8) from pinned host memory")
    p.add_argument("--host-pipeline", type=int, default=0, choices=[0, 1, 2],
                   help="host-buffer schedule of --paper-scale: 0 chosen by memory, 1 slabs, 2 whole input resident")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def cpu_oracle_sample(I0_cpu, alpha, planes=8):
    """Time the CPU FP64 oracle on a bounded sample of the workload: smoothing of a slab of
    `planes` consecutive planes from the middle of the stack (x, y and z passes) and the DCT
    solve of one slice.  A whole-stack run smooths every plane once and solves every slice
    once, so its rate is 1 / (smoothing seconds per voxel + solve seconds per voxel).  (Inside
    a thin slab the z pass has fewer in-stack taps than in the whole stack, so the sample, if
    anything, flatters the oracle.)  Returns (voxels/s, seconds, sample description)."""
    from oracle import emfuse_oracle as O
    nz, ny, nx = I0_cpu.shape
    z0 = max(0, nz // 2 - planes // 2)
    slab = I0_cpu[z0:z0 + planes].double().numpy()
    t0 = time.perf_counter()
    s = O.smooth_stack(slab, 1.0, 3.0)
    t1 = time.perf_counter()
    O.solve_dct(s[planes // 2], slab[planes // 2], alpha)
    t2 = time.perf_counter()
    plane = ny * nx
    per_voxel = (t1 - t0) / (planes * plane) + (t2 - t1) / plane
    return 1.0 / per_voxel, t2 - t0, (f"smoothing of a {planes}-plane {ny}x{nx} slab + 1 DCT solve; "
                                      f"voxels/s = 1 / (smoothing s/voxel + solve s/voxel)")


def oracle_slice_errors(out, I0, alpha, slices, s_oracle=None):
    """max |f - f_oracle| and relative L2 error on sampled slices of a corrected stack, against
    the CPU FP64 oracle (smoothing of the slice's floor(3 sigma_z) neighbourhood, then its DCT
    solve); the worst over the slices.  s_oracle caches the oracle's smoothed slices."""
    import numpy as np
    from oracle import emfuse_oracle as O
    nz = I0.shape[0]
    worst_abs, worst_l2 = 0.0, 0.0
    for j in slices:
        if s_oracle is not None and j in s_oracle:
            s, o = s_oracle[j]
        else:
            a, b = max(0, j - 9), min(nz, j + 10)
            slab = I0[a:b].double().cpu().numpy()
            s, o = O.smooth_stack(slab, 1.0, 3.0)[j - a], slab[j - a]
            if s_oracle is not None:
                s_oracle[j] = (s, o)
        ref = O.solve_dct(s, o, alpha)
        d = out[j].double().cpu().numpy() - ref
        worst_abs = max(worst_abs, float(np.max(np.abs(d))))
        worst_l2 = max(worst_l2, float(np.linalg.norm(d) / np.linalg.norm(ref)))
    return {"slices": list(slices), "max_abs_err": worst_abs, "rel_to_255": worst_abs / 255.0,
            "rel_l2_err": worst_l2}


def make_input(device, nz=NZ):
    import torch
    from paper_1506_02079_gb300.synthetic import make_stack
    return make_stack(nz, NY, NX, SEED, device=device, out_dtype=torch.float32)


def run_reference(args):
    import torch
    rank, _, world = dist_env()
    if world > 1 and rank != 0:
        return
    I0 = make_input("cpu")
    cores = os.cpu_count()
    for _ in range(args.warmup):
        cpu_oracle_sample(I0, args.alpha, planes=2)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        v, dt, sample = cpu_oracle_sample(I0, args.alpha, planes=6)
        vals.append(v)
        secs += dt
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "voxels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "alpha": args.alpha, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": sample + " per step; extrapolated to voxels/s"},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_extra(dev, alpha, steps=3):
    """The batched configuration: 512 independent slices, square, sides log-uniform in
    [256, 4096] (seed 2, about 1.54 Gpx), solved in one ragged batch per call.  The schedule
    is autotuned once (rows per work item x sweeps), then timed with the V-cycles replayed as
    CUDA graphs and, for comparison, launched directly."""
    import torch
    from paper_1506_02079_gb300 import api
    from paper_1506_02079_gb300.synthetic import make_ragged_batch

    s, o, ny, nx, offs = make_ragged_batch(512, seed=2, device=dev, dtype=torch.float32)
    px = int((ny * nx).sum())
    f = torch.empty_like(s)
    tuned = api.default_opts(tol=1e-6, autotune=1)
    api.emfuse_screened_poisson(s, o, alpha, tuned, nx=nx, ny=ny, offsets=offs, out=f)
    table = api.emfuse_autotune_result()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"slices": 512, "pixels": px, "alpha": alpha, "autotune": table}
    for label, opts in (("graphs", tuned), ("direct", api.default_opts(tol=1e-6, autotune=1, no_graphs=1))):
        api.emfuse_screened_poisson(s, o, alpha, opts, nx=nx, ny=ny, offsets=offs, out=f)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            _, st = api.emfuse_screened_poisson(s, o, alpha, opts, nx=nx, ny=ny, offsets=offs, out=f,
                                                return_stats=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[label] = {"value": px / (ms * 1e-3), "unit": "pixels/s", "ms": ms,
                      "vcycles": max(a["vcycles"] for a in st),
                      "max_rel_residual": max(a["rel_residual"] for a in st)}
    # errors against the oracle on the smallest, the median and the largest slice, and the
    # reported residual against its plain FP64 recomputation on every slice
    import numpy as np
    from oracle import emfuse_oracle as O
    vopts = api.default_opts(tol=1e-6, autotune=1, verify_residual=1)
    _, st = api.emfuse_screened_poisson(s, o, alpha, vopts, nx=nx, ny=ny, offsets=offs, out=f, return_stats=True)
    order = np.argsort(ny * nx, kind="stable")
    worst_abs, worst_l2 = 0.0, 0.0
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        a, h, w = int(offs[i]), int(ny[i]), int(nx[i])
        sl = lambda t: t[a:a + h * w].view(h, w).double().cpu().numpy()
        ref = O.solve_dct(sl(s), sl(o), alpha)
        d = sl(f) - ref
        worst_abs = max(worst_abs, float(np.abs(d).max()))
        worst_l2 = max(worst_l2, float(np.linalg.norm(d) / np.linalg.norm(ref)))
    res["oracle_error"] = {"slices": "smallest, median, largest", "max_abs_err": worst_abs,
                           "rel_to_255": worst_abs / 255.0, "rel_l2_err": worst_l2}
    res["residual_check"] = {"max_rel_residual_fp64_recomputed": max(a["rel_residual_check"] for a in st),
                             "max_rel_diff_reported_vs_recomputed":
                                 max(abs(a["rel_residual"] - a["rel_residual_check"]) / a["rel_residual_check"]
                                     for a in st if a["rel_residual_check"] > 0)}
    del s, o, f
    torch.cuda.empty_cache()
    return res


PAPER_NY, PAPER_NX = 21504, 26624
PAPER_SEED = 4


def paper_scale_stack(nz, dev):
    """Synthetic stand-in for the paper's largest stack, slice size 21504 x 26624, uint8, in
    pinned host memory: the first nz slices of the 64-slice stack generator (seed 4, per-slice
    gain and offset artefacts) evaluated at full size on the GPU, tile by tile."""
    import torch
    from paper_1506_02079_gb300.synthetic import evaluate_stack_tiled, stack_params

    p = stack_params(64, PAPER_NY, PAPER_NX, PAPER_SEED)
    host = torch.empty((nz, PAPER_NY, PAPER_NX), dtype=torch.uint8, pin_memory=True)
    evaluate_stack_tiled(p, 0, nz, device=dev, dtype=torch.float32, out_dtype=torch.uint8, out=host)
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return host


def run_paper_scale(args):
    """End-to-end streaming of a paper-scale stack through the public API (host in, host out):
    every step copies the uint8 stack to the device in z-chunks with their halo planes,
    smooths, solves and copies the FP32 result back, all inside the timed region."""
    import torch
    from paper_1506_02079_gb300 import api
    from paper_1506_02079_gb300.profiling import profile_steps

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nz = args.paper_scale
    t0 = time.perf_counter()
    I0 = paper_scale_stack(nz, dev)
    out = torch.empty((nz, PAPER_NY, PAPER_NX), dtype=torch.float32, pin_memory=True)
    t_gen = time.perf_counter() - t0
    opts = api.default_opts(tol=1e-6)
    opts.host_pipeline = args.host_pipeline
    step = lambda: api.emfuse_correct_stack(I0, 1.0, 3.0, args.alpha, opts, out=out, return_stats=True)
    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches0 = api.lib().emfuse_kernel_launches()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, stats = step()
        torch.cuda.synchronize()
        secs = (time.perf_counter() - t0) / args.steps
    launches = api.lib().emfuse_kernel_launches() - launches0
    prof = profile_steps(step, 1)
    # a property that holds at any size: the DCT mode 0 of Eq. (1) has gain 1, so every
    # corrected slice keeps the mean of its smoothed slice (checked on the middle slice)
    j = nz // 2
    a, b = max(0, j - 9), min(nz, j + 10)
    s_j = api.emfuse_smooth_z(I0[a:b].to(dev), 1.0, 3.0, z0=j - a, z1=j - a + 1)
    mean_s = float(s_j.double().mean())
    mean_f = float(out[j].to(dev).double().mean())
    del s_j
    # the host link on these buffers: one whole copy each way (after the check above: the
    # D2H copy overwrites the output)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dtmp = torch.empty((nz, PAPER_NY, PAPER_NX), dtype=torch.float32, device=dev)
    din = dtmp.view(torch.uint8).view(-1)[: I0.numel()].view(I0.shape)
    link_h2d, link_d2h = [], []
    for _ in range(3):
        e0.record(); din.copy_(I0, non_blocking=True); e1.record()
        torch.cuda.synchronize()
        link_h2d.append(round(I0.numel() / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1))
        e0.record(); out.copy_(dtmp, non_blocking=True); e1.record()
        torch.cuda.synchronize()
        link_d2h.append(round(out.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9, 1))
    del dtmp, din
    torch.cuda.empty_cache()
    vox = nz * PAPER_NY * PAPER_NX
    h2d, d2h = I0.numel(), out.numel() * 4
    kernel_ms = sum(p["ms_per_step"] for p in prof)
    line = {"metric": METRIC + " (streamed from host)", "value": vox / secs, "unit": "voxels/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": 1e3 * secs,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (stack generator evaluated at full size on the GPU)",
            "config": {"workload": f"{nz} slices x {PAPER_NY} x {PAPER_NX} uint8 from pinned host, sigma_xy=1, "
                                   "sigma_z=3, FP32 multigrid + FP64 defect correction to rel. residual 1e-6",
                       "host_pipeline": ["auto", "slabs", "resident"][args.host_pipeline],
                       "alpha": args.alpha, "nz": nz, "ny": PAPER_NY, "nx": PAPER_NX, "seed": PAPER_SEED},
            "e2e": {"value": vox / secs, "unit": "voxels/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "link_gbs": (h2d + d2h) / secs / 1e9, "link_h2d_gbs_whole_copy": link_h2d, "link_d2h_gbs_whole_copy": link_d2h,
            "kernel_ms_per_step": kernel_ms,
            "gpu_launches": int(launches // max(args.steps, 1)) * args.steps,
            "vcycles": max(s["vcycles"] for s in stats), "max_rel_residual": max(s["rel_residual"] for s in stats),
            "clocks": clk.summary(), "input_generation_s": t_gen,
            "mean_check": {"slice": j, "mean_s": mean_s, "mean_f": mean_f, "rel_diff": abs(mean_f - mean_s) / abs(mean_s)},
            "kernels": prof[:8]}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import numpy as np
    import torch
    from paper_1506_02079_gb300 import api
    from paper_1506_02079_gb300.profiling import profile_steps, kernel_roofline, relaxation_roofline, measured_hbm_peak

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L = api.lib()
    I0 = make_input(dev, args.nz)
    out = torch.empty_like(I0)
    opts = api.default_opts(tol=1e-6, precision=api.PREC_MIXED, no_graphs=int(args.no_graphs),
                            tile_rows=args.tile_rows)
    step = lambda: api.emfuse_correct_stack(I0, 1.0, 3.0, args.alpha, opts, out=out, return_stats=True)

    for _ in range(max(3, args.warmup)):
        _, stats = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = L.emfuse_kernel_launches()
    vcycles = []
    with ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            _, stats = step()
            vcycles.append(max(s["vcycles"] for s in stats))
        e1.record(stream)
        torch.cuda.synchronize()
    launches = L.emfuse_kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    voxels = args.nz * NY * NX
    value = voxels * world / (ms * 1e-3)
    worst_res = max(s["rel_residual"] for s in stats)

    extras = {}
    if rank == 0 and not args.no_extras:
        # per-kernel CUDA-event timing over the same steps (a separate pass so the timed
        # value above carries no instrumentation)
        prof = profile_steps(step, args.steps)
        extras["kernels"] = prof
        # the FP64 roofline denominator: FP64 FMA throughput measured on this GPU (CUDA events),
        # with the clocks seen meanwhile
        with ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0) as clk64:
            rates = [api.emfuse_probe_fp64_fma_rate(dev) for _ in range(5)]
        fp64_peak = statistics.median(rates)
        roof = kernel_roofline(prof, fp64_peak)
        roof["fp64_probe"] = {"tflops_median": fp64_peak, "tflops_all": rates, "clocks": clk64.summary()}
        top = next((p for p in prof if p["name"] == roof["kernel"]), None)
        if top and roof["bound"] == "alu":
            # the same kernel against HBM at a round 40 B per cell and FP64 pass (s, o, e, r, out in
            # FP32 and the FP64 iterate read and written: 36 B, plus slack for the halo)
            cells = voxels
            roof["hbm_frac_at_40B_per_cell"] = (cells * 40.0 / (top["ms_per_step"] / max(top["launches"], 1) * 1e-3)
                                                / 1e9 / measured_hbm_peak()[0])
        extras["roofline_relaxation"] = relaxation_roofline(prof)
        # whole-step effective HBM fraction: voxels/s times the bytes per voxel the method must
        # move (input 4 + output 4 + first residual 12 + 16 per V-cycle + 40 per FP64 correction
        # pass; counts from this step's launches) over the measured HBM peak
        per = {p["name"]: p["launches"] for p in prof}  # launches per step
        n_v, n_outer = per.get("wave_up_l0", 0.0), per.get("residual_update", 0.0)
        b_alg = 4.0 + 4.0 + 12.0 + 16.0 * n_v + 40.0 * n_outer
        eff_gbs = voxels * world / (ms * 1e-3) * b_alg / 1e9
        extras["effective_hbm"] = {"bytes_per_voxel": b_alg, "vcycles": n_v, "fp64_passes": n_outer,
                                   "gbs": eff_gbs, "frac": eff_gbs / measured_hbm_peak()[0]}
        # end to end through the public API with host buffers
        I0_h = I0.cpu().pin_memory()
        out_h = torch.empty_like(I0_h).pin_memory()
        api.emfuse_correct_stack(I0_h, 1.0, 3.0, args.alpha, opts, out=out_h)
        ne = max(5, args.steps)
        e2e_steps = []
        for _ in range(ne):
            t0 = time.perf_counter()
            api.emfuse_correct_stack(I0_h, 1.0, 3.0, args.alpha, opts, out=out_h)  # returns when out_h is filled
            e2e_steps.append(time.perf_counter() - t0)
        e2e_s = sum(e2e_steps) / ne
        # the host link as this run saw it: one whole-stack copy each way on these buffers
        dev_tmp = torch.empty_like(I0)
        torch.cuda.synchronize()
        e0.record(stream)
        dev_tmp.copy_(I0_h, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = I0_h.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9
        e0.record(stream)
        out_h.copy_(dev_tmp, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        d2h_gbs = out_h.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del dev_tmp
        e2e = {"value": voxels / e2e_s, "unit": "voxels/s", "h2d_bytes_per_step": I0_h.numel() * 4,
               "d2h_bytes_per_step": out_h.numel() * 4, "ms_per_step": 1e3 * e2e_s,
               "link_h2d_gbs": h2d_gbs, "link_d2h_gbs": d2h_gbs,
               "step_ms": [round(1e3 * s, 2) for s in e2e_steps],
               "median_ms": round(1e3 * sorted(e2e_steps)[len(e2e_steps) // 2], 2)}
        # plain FP64 GPU solve at the same tolerance
        o64 = api.default_opts(tol=1e-6, precision=api.PREC_FP64)
        api.emfuse_correct_stack(I0, 1.0, 3.0, args.alpha, o64, out=out)
        torch.cuda.synchronize()
        e0.record(stream)
        n64 = 2
        for _ in range(n64):
            _, st64 = api.emfuse_correct_stack(I0, 1.0, 3.0, args.alpha, o64, out=out, return_stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        s_cache = {}
        sample = (args.nz // 2, args.nz - 1)
        extras["fp64_plain_solve"] = {"value": voxels / (ms64 * 1e-3), "unit": "voxels/s", "ms_per_step": ms64,
                                      "vcycles": max(s["vcycles"] for s in st64),
                                      "max_rel_residual": max(s["rel_residual"] for s in st64),
                                      "oracle_error": oracle_slice_errors(out, I0, args.alpha, sample, s_cache)}
        extras["mixed_over_fp64"] = (voxels / (ms * 1e-3)) / extras["fp64_plain_solve"]["value"]
        # the other screening weights of the configuration
        per_alpha = {}
        for a in (1e-3, 1e-2, 1e-1):
            step_a = lambda: api.emfuse_correct_stack(I0, 1.0, 3.0, a, opts, out=out, return_stats=True)
            step_a()
            torch.cuda.synchronize()
            e0.record(stream)
            _, sa = step_a()
            e1.record(stream)
            torch.cuda.synchronize()
            per_alpha[str(a)] = {"ms": e0.elapsed_time(e1), "vcycles": max(s["vcycles"] for s in sa),
                                 "max_rel_residual": max(s["rel_residual"] for s in sa),
                                 "oracle_error": oracle_slice_errors(out, I0, a, sample, s_cache)}
        extras["per_alpha"] = per_alpha
        extras["batched_512"] = batched_extra(dev, args.alpha)
        # the first "next" row: smoothing with robust averaging across slices, against the
        # plain smoothing of the same stack (both read the stack once and write s once)
        sm = {}
        for label, fn in (("plain", lambda: api.emfuse_smooth_z(I0, 1.0, 3.0, out=out)),
                          ("robust_kappa2", lambda: api.emfuse_smooth_z_robust(I0, 1.0, 3.0, 2.0, out=out))):
            fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(5):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s = e0.elapsed_time(e1) / 5
            gbs = voxels * 8.0 / (ms_s * 1e-3) / 1e9
            sm[label] = {"ms": ms_s, "value": voxels / (ms_s * 1e-3), "unit": "voxels/s", "gbs": gbs,
                         "hbm_frac": gbs / measured_hbm_peak()[0]}
        extras["smoothing"] = sm
        # the second next row: the direct FFT solve of the same 64 solves (mirror extension,
        # cuFFT) against the multigrid solve alone, and their largest difference
        s_c2 = api.emfuse_smooth_z(I0, 1.0, 3.0)
        sol = {}
        for label, fn in (("multigrid_mixed", lambda: api.emfuse_screened_poisson(s_c2, I0, args.alpha, opts)),
                          ("fft_fp32", lambda: api.emfuse_screened_poisson_dct(s_c2, I0, args.alpha, api.PREC_FP32)),
                          ("fft_fp64", lambda: api.emfuse_screened_poisson_dct(s_c2, I0, args.alpha, api.PREC_FP64))):
            res = fn()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(2):
                res = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            sol[label] = {"ms": e0.elapsed_time(e1) / 2, "value": voxels / (e0.elapsed_time(e1) / 2 * 1e-3),
                          "unit": "voxels/s"}
            sol[label + "_out"] = res
        # the solves alone against the oracle's DCT solve of the same smoothed slices
        from oracle import emfuse_oracle as O
        for label in ("multigrid_mixed", "fft_fp32", "fft_fp64"):
            worst_abs, worst_l2 = 0.0, 0.0
            for j in sample:
                ref = O.solve_dct(s_c2[j].double().cpu().numpy(), I0[j].double().cpu().numpy(), args.alpha)
                dj = sol[label + "_out"][j].double().cpu().numpy() - ref
                worst_abs = max(worst_abs, float(np.max(np.abs(dj))))
                worst_l2 = max(worst_l2, float(np.linalg.norm(dj) / np.linalg.norm(ref)))
            sol[label]["oracle_error"] = {"slices": list(sample), "max_abs_err": worst_abs,
                                          "rel_to_255": worst_abs / 255.0, "rel_l2_err": worst_l2}
        sol["max_abs_diff_multigrid_vs_fft_fp64"] = float((sol.pop("multigrid_mixed_out") - sol["fft_fp64_out"]).abs().max())
        sol["max_abs_diff_fft_fp32_vs_fft_fp64"] = float((sol.pop("fft_fp32_out") - sol.pop("fft_fp64_out")).abs().max())
        extras["solve_multigrid_vs_fft"] = sol
        del s_c2
        api.emfuse_release_cache()
        torch.cuda.empty_cache()
        # colour / monochrome fusion (Sec. 3 colour example): 4 images of 4096 x 4096, RGB value
        # constraints (colour casts of the synthetic base), grey gradient constraints
        from paper_1506_02079_gb300.synthetic import make_stack as _mk
        base = _mk(4, 4096, 4096, 5, device=dev)
        casts = torch.tensor([[1.1, 5.0], [0.9, -3.0], [1.0, 12.0]], device=dev)
        s_rgb = (base[:, None] * casts[None, :, 0, None, None] + casts[None, :, 1, None, None]).clamp_(0, 255)
        s_rgb = s_rgb.contiguous()
        api.emfuse_fuse_color(s_rgb, base, args.alpha)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            f_rgb, stc = api.emfuse_fuse_color(s_rgb, base, args.alpha, return_stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_c = e0.elapsed_time(e1) / 3
        # the first image's three channels against the oracle
        ref_c = O.fuse_color(s_rgb[0].double().cpu().numpy(), base[0].double().cpu().numpy(), args.alpha)
        dc = f_rgb[0].double().cpu().numpy() - ref_c
        extras["color_fusion"] = {"images": 4, "ny": 4096, "nx": 4096, "channels": 3, "ms": ms_c,
                                  "value": s_rgb.numel() / (ms_c * 1e-3), "unit": "pixels/s",
                                  "vcycles": max(a["vcycles"] for a in stc),
                                  "max_rel_residual": max(a["rel_residual"] for a in stc),
                                  "oracle_error": {"image": 0, "max_abs_err": float(np.max(np.abs(dc))),
                                                   "rel_to_255": float(np.max(np.abs(dc))) / 255.0,
                                                   "rel_l2_err": float(np.linalg.norm(dc) / np.linalg.norm(ref_c))}}
        del f_rgb, ref_c, dc
        del base, s_rgb
        torch.cuda.empty_cache()
        # the fourth next row: phase 1 as the 3-D gradient-domain problem of the earlier method
        # (exact, one 3-D FFT of the mirror-extended stack) beside the Gaussian smoothing above;
        # alpha = 0.1 damps per-slice offsets over about 1 / sqrt(alpha) ~ 3 slices, like sigma_z = 3
        gd, outs = {}, {}
        for label, prec in (("fp32", api.PREC_FP32), ("fp64", api.PREC_FP64)):
            outs[label] = api.emfuse_smooth_gradient_domain(I0, 0.1, prec)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(2):
                outs[label] = api.emfuse_smooth_gradient_domain(I0, 0.1, prec, out=outs[label])
            e1.record(stream)
            torch.cuda.synchronize()
            ms_g = e0.elapsed_time(e1) / 2
            gd[label] = {"ms": ms_g, "value": voxels / (ms_g * 1e-3), "unit": "voxels/s"}
        # the same problem by the 3-D multigrid (FP32 V-cycles, FP64 defect correction, tol 1e-6)
        mg_out, mg_st = api.emfuse_smooth_gradient_domain_mg(I0, 0.1, api.default_opts(tol=1e-6),
                                                             return_stats=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(2):
            api.emfuse_smooth_gradient_domain_mg(I0, 0.1, api.default_opts(tol=1e-6), out=mg_out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_g = e0.elapsed_time(e1) / 2
        mg_prof = profile_steps(lambda: api.emfuse_smooth_gradient_domain_mg(
            I0, 0.1, api.default_opts(tol=1e-6), out=mg_out), 1)
        gd["multigrid"] = {"ms": ms_g, "value": voxels / (ms_g * 1e-3), "unit": "voxels/s",
                           "vcycles": mg_st["vcycles"], "rel_residual": mg_st["rel_residual"],
                           "max_abs_diff_vs_fft_fp64": float((mg_out - outs["fp64"]).abs().max()),
                           "kernels": [{"name": q["name"], "launches": q["launches"],
                                        "ms": round(q["ms_per_step"], 3), "gbs": round(q["gbs"] or 0.0, 1)}
                                       for q in mg_prof[:8]]}
        del mg_out
        tot_in = float(I0.double().sum())
        gd.update({"alpha": 0.1, "gaussian_smoothing_ms": sm["plain"]["ms"],
                   "max_abs_diff_fp32_vs_fp64": float((outs["fp32"] - outs["fp64"]).abs().max()),
                   "total_rel_diff_fp64": abs(float(outs["fp64"].double().sum()) - tot_in) / abs(tot_in),
                   "mean_abs_interslice_diff": {"input": float((I0[1:] - I0[:-1]).abs().mean()),
                                                "gradient_domain": float((outs["fp64"][1:] - outs["fp64"][:-1]).abs().mean())}})
        extras["gradient_domain_smoothing"] = gd
        del outs
        api.emfuse_release_cache()
        torch.cuda.empty_cache()
        # parity of the timed configuration vs the CPU FP64 oracle on sampled slices (the middle
        # of the stack and its last slice, whose z-window is cut by the stack end), and the
        # reported residual against its plain FP64 recomputation on every slice
        vopts = api.default_opts(tol=1e-6, precision=api.PREC_MIXED, verify_residual=1)
        _, stv = api.emfuse_correct_stack(I0, 1.0, 3.0, args.alpha, vopts, out=out, return_stats=True)
        extras["parity_sampled_slices"] = oracle_slice_errors(out, I0, args.alpha, sample, s_cache)
        extras["residual_check"] = {
            "max_rel_residual_reported": max(a["rel_residual"] for a in stv),
            "max_rel_residual_fp64_recomputed": max(a["rel_residual_check"] for a in stv),
            "max_rel_diff_reported_vs_recomputed": max(abs(a["rel_residual"] - a["rel_residual_check"])
                                                       / a["rel_residual_check"] for a in stv)}
        cpu = None
        if not args.no_cpu_baseline:
            v, dt, sample = cpu_oracle_sample(I0.cpu(), args.alpha, planes=12)
            cpu = {"value": v, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": sample + f"; {dt:.1f} s, extrapolated to voxels/s"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.nz == NZ else f"{args.nz} slices x 2048 x 2048 (profiling case)",
                           "alpha": args.alpha, "nz": args.nz, "ny": NY, "nx": NX,
                           "seed": SEED, "l2": "inputs (1.07 GB) larger than L2 (129 MB)",
                           "parallelism": f"replicas x{world}",
                           "launch": "direct kernel launches" if args.no_graphs else "CUDA graphs",
                           "tile_rows": args.tile_rows or "chosen"},
                "gpu_launches": int(launches), "vcycles": max(vcycles), "max_rel_residual": worst_res,
                "clocks": clk.summary()}
        if extras:
            line["e2e"] = e2e
            line["roofline"] = roof
            line["cpu_baseline"] = cpu
            line.update({k: v for k, v in extras.items() if k != "kernels"})
            line["kernels"] = extras["kernels"][:8]
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.paper_scale:
        run_paper_scale(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
