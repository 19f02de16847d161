"""Per-kernel timing and roofline numbers from the library's own CUDA-event instrumentation.

``profile_steps`` runs a callable with ``emfuse_profile_begin/end`` around it: every kernel
launch of the library is bracketed by CUDA events on its own stream and carries the
algorithmic bytes of the launch (each needed input element read once, each output written
once).  ``kernel_roofline`` turns the dominant kernel's totals into achieved GB/s against the
measured HBM copy bandwidth of the machine.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os

from . import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FALLBACK_HBM_GBS = 6800.0


class _Prof(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double), ("fp64_flops", ctypes.c_double)]


def profile_steps(step, n: int) -> list[dict]:
    L = api.lib()
    L.emfuse_profile_begin.argtypes = []
    L.emfuse_profile_begin.restype = None
    L.emfuse_profile_end.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.emfuse_profile_end.restype = ctypes.c_int
    L.emfuse_profile_begin()
    try:
        for _ in range(n):
            step()
    finally:
        buf = (_Prof * 64)()
        k = L.emfuse_profile_end(ctypes.addressof(buf), 64)
    if k < 0:
        raise api.EmfuseError(2, L.emfuse_last_error().decode())
    total = sum(buf[i].total_ms for i in range(min(k, 64))) or 1.0
    out = []
    for i in range(min(k, 64)):
        p = buf[i]
        out.append({"name": p.name.decode(), "launches": int(p.launches) // max(n, 1),
                    "ms_per_step": p.total_ms / n, "share": p.total_ms / total,
                    "gbs": (p.bytes / (p.total_ms * 1e-3) / 1e9) if p.total_ms > 0 else None,
                    "bytes_per_launch": p.bytes / max(p.launches, 1),
                    "fp64_tflops": (p.fp64_flops / (p.total_ms * 1e-3) / 1e12) if p.total_ms > 0 else None,
                    "fp64_flops_per_launch": p.fp64_flops / max(p.launches, 1)})
    return out


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# CUDA sources each instrumented kernel is built from (the others: every source)
_KERNEL_SOURCES = {
    "residual": ("multigrid.cu", "fpconv.cuh", "mg_fused.cuh", "emfuse_common.cuh"),
    "wave": ("fused_impl.cuh", "fused_launch.cuh", "fused_f32.cu", "fused_f64.cu", "fused_f32_s68.cu",
             "fused_f64_s68.cu", "mg_fused.cuh", "tma.cuh", "emfuse_common.cuh"),
    "coarse_tail": ("fused_impl.cuh", "fused_launch.cuh", "fused_f32.cu", "fused_f64.cu", "mg_fused.cuh",
                    "emfuse_common.cuh"),
    "smooth": ("smooth.cu", "tma.cuh", "emfuse_common.cuh"),
}


def kernel_source_hash(name: str) -> str:
    """Hash of the CUDA sources of kernel `name`, so stored ncu traffic is dropped once that
    kernel's code changes."""
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    files = None
    for prefix, fs in _KERNEL_SOURCES.items():
        if name.startswith(prefix):
            files = fs
    if files is None:
        files = tuple(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh")))
    h = hashlib.sha256()
    for f in sorted(files):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(name: str):
    """dram read+write bytes per launch of kernel `name` from the committed ncu summary
    (profiles/traffic.json), or None if absent or taken on different sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(name)
    if not e or e.get("source_hash") != kernel_source_hash(name):
        return None
    return e.get("dram_bytes_per_launch")


# FP64 peak of GB300 derived from its unit counts and clock: 152 SMs x 2 DFMA per clock per SM
# x 2 flops x 2.07 GHz (the nominal 1.25 TFLOP/s); no measured FP64 peak is provided.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _hbm_roofline(p: dict) -> dict:
    peak, kind = measured_hbm_peak()
    return {"kernel": p["name"], "bound": "hbm", "achieved": p["gbs"], "peak": peak, "unit": "GB/s",
            "frac": (p["gbs"] / peak) if p["gbs"] else None, "peak_source": f"hbm_gbs of {kind}",
            "share_of_step": p["share"], "bytes_per_launch": p["bytes_per_launch"],
            "traffic": stored_traffic(p["name"])}


def kernel_roofline(prof: list[dict], fp64_measured_tflops: float | None = None) -> dict:
    """Roofline of the dominant kernel (largest share of the step): FP64-pipe bound ("alu")
    when it does FP64 work, else HBM bound.  For the FP64 case the peak is the FP64 FMA rate
    measured on this GPU (emfuse_probe_fp64_fma_rate) when given, with the peak derived from
    the unit counts and clock beside it, and the kernel's HBM fraction at its algorithmic bytes."""
    top = max(prof, key=lambda p: p["share"])
    if top.get("fp64_flops_per_launch"):
        peak = fp64_measured_tflops or FP64_PEAK_TFLOPS
        hbm, kind = measured_hbm_peak()
        return {"kernel": top["name"], "bound": "alu", "achieved": top["fp64_tflops"],
                "peak": peak, "unit": "TFLOP/s", "frac": top["fp64_tflops"] / peak,
                "peak_source": ("FP64 FMA rate measured on this GPU by CUDA events (emfuse_probe_fp64_fma_rate)"
                                if fp64_measured_tflops else
                                "FP64 derived from unit counts and clock (152 SMs x 2 DFMA/clk x 2.07 GHz)"),
                "peak_derived": FP64_PEAK_TFLOPS, "frac_of_derived": top["fp64_tflops"] / FP64_PEAK_TFLOPS,
                "hbm_gbs": top["gbs"], "hbm_frac": top["gbs"] / hbm if top["gbs"] else None,
                "hbm_peak_source": f"hbm_gbs of {kind}",
                "share_of_step": top["share"], "flops_per_launch": top["fp64_flops_per_launch"],
                "bytes_per_launch": top["bytes_per_launch"], "traffic": stored_traffic(top["name"])}
    return _hbm_roofline(top)


def relaxation_roofline(prof: list[dict]) -> dict | None:
    """HBM roofline of the relaxation (wavefront V-cycle) kernel with the largest share."""
    waves = [p for p in prof if p["name"].startswith("wave_")]
    return _hbm_roofline(max(waves, key=lambda p: p["share"])) if waves else None
