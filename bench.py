"""Benchmark of the HBGK stream-collide hot path (one JSON line on rank 0).

Workload (default): D3Q19 HBGK on a 256^3 fully periodic lattice, porosity control
from a regular matrix of equal spheres (period 32 cells, radius 0.3 of the period,
smoothed over 2 cells), body force 1e-6 along x, tau = 0.6, FP32 deviation storage,
two-lattice pull streaming. One benchmark step = one check interval: 100 time steps
(fused stream-collide kernels, replayed from a CUDA graph) plus the FP64 diagnostics
reduction (mass, momentum, plane flux, apparent permeability, residual max|du|).

value : MLUPS = cells * time steps / device time (CUDA events, max over ranks).
e2e   : the same metric through the C ABI with host buffers: per step the porosity field
        is copied from pinned host memory (set_porosity), the lattice re-initialised,
        100 time steps run and the diagnostics read back to the host.
roofline : the stream-collide kernel's algorithmic bytes (q*2*sizeof(T) + 4 per cell
        update) over its average launch time, against the measured HBM copy bandwidth.
cpu_baseline : the FP64 CPU oracle timed on the host cores on a bounded sample (a few
        time steps of the same 256^3 workload).

Legs of the default line: "aa" (the workload in place), "reduced_precision" (FP16 / BF16 at
384^3 on the random sphere matrix, and their error against the FP64 oracle at 96^3),
"adjoint" (the 128^3 x 2000-step gradient), "serving" (16 requests of the serving trace,
batched server vs the plain FP32 loop, with the served results against FP64).
Other modes: --workload W (another lattice workload), --serving-only (a longer serving trace),
--serving-class (throughput of server slot sets), --adjoint-only.

--impl reference times that oracle alone (the deliberately slow reference program) on
the same workload and prints the same line with "impl": "reference".
Multi-GPU (torchrun): independent replicas, one lattice per GPU (weak scaling); the
single-lattice path has no exchange step here.
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

METRIC = "D3Q19 HBGK MLUPS & % HBM roofline; p50/p99 solve latency, batched vs plain"
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel, from the
# ncu capture summarised under profiles/. Each entry records the hash of the sources of that
# kernel (kernel_source_hash(kernel)) it was captured from; when those sources have changed
# since, the bench reports traffic as null instead of a stale figure.
KERNEL_TRAFFIC_BYTES = {
    # k_step<19, StoreF32, periodic, two-lattice, int, shift-fx>, 256^3: mean of two launches
    # (1342250752 + 1228698112 and 1342237696 + 1217931008 bytes)
    ("stream_collide_d3q19_f32_two", 256): {"bytes": 2565558784, "source_hash": "76d4a47919d1105a"},
    # k_step<19, StoreF32, periodic, AA even / AA odd, int, shift-fx>, 256^3: mean of the even
    # (1342202368 + 1217577984) and odd (1342190336 + 1217456640 bytes) launch of one capture
    ("stream_collide_d3q19_f32_aa", 256): {"bytes": 2559713664, "source_hash": "76d4a47919d1105a"},
    # k_step_pair<19, StoreF16, shift-fx, two-lattice>, 384^3 Boolean sphere matrix: mean of two launches
    # (2378278656 + 2107357184 and 2378211072 + 2106170112 bytes)
    ("stream_collide_d3q19_f16_two", 384): {"bytes": 4485008512, "source_hash": "59ee95aa12972e25"},
    # k_step_pair<19, StoreBF16, shift-fx, two-lattice> (56 registers), 384^3 Boolean sphere matrix: mean of
    # two launches (2378226176 + 2104031232 and 2378216704 + 2103352064 bytes)
    ("stream_collide_d3q19_bf16_two", 384): {"bytes": 4481913088, "source_hash": "e6debcdf9dc15415"},
    # k_step_pair<19, StoreF16, shift-fx, AA even / AA odd>, 384^3 Boolean sphere matrix: mean of an
    # even (2378207744 + 2097896192) and an odd (2378275584 + 2150258944 bytes) launch
    ("stream_collide_d3q19_f16_aa", 384): {"bytes": 4502319232, "source_hash": "59ee95aa12972e25"},
}

# the sources each step kernel is compiled from (csrc/)
_COMMON_SOURCES = ("lattice.cuh", "internal.h", "k_step.cuh", "k_step.cu")
KERNEL_SOURCES = {
    "f64": _COMMON_SOURCES + ("k_step_f64.cu",),
    "f32": _COMMON_SOURCES + ("k_step_f32.cu",),
    "f16": _COMMON_SOURCES + ("k_step_pair.cuh", "k_step_f16.cu"),
    "bf16": _COMMON_SOURCES + ("k_step_pair.cuh", "k_step_bf16.cu"),
}


def kernel_source_hash(kname):
    """sha256 (first 16 hex digits) over the sources of the step kernel `kname`
    (stream_collide_d3q19_<storage>_<pattern>)."""
    import hashlib
    storage = kname.split("_")[3]
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[storage]:
        with open(os.path.join(ROOT, "paper_2310_14746_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def kernel_traffic(kname, n):
    """(bytes per launch or None, note) for the kernel as it is now."""
    e = KERNEL_TRAFFIC_BYTES.get((kname, n))
    if e is None:
        return None, "not captured"
    if e["source_hash"] != kernel_source_hash(kname):
        return None, "stale: kernel sources changed since the capture"
    return e["bytes"], "ncu capture of these sources"


WORKLOADS = {
    "d3q19_256_f32": dict(q=19, n=256, storage="f32", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                          period=32, ratio=0.3,
                          desc="D3Q19 HBGK 256^3 periodic, regular sphere matrix (period 32, r = 0.3 P, "
                               "smoothed), F = 1e-6, tau = 0.6, FP32 deviation storage, two-lattice"),
    "d3q19_128_f32": dict(q=19, n=128, storage="f32", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                          period=32, ratio=0.3,
                          desc="D3Q19 HBGK 128^3 periodic, regular sphere matrix (period 32, r = 0.3 P), FP32 "
                               "deviation storage, two-lattice (profiling size)"),
    "d3q19_256_f32_aa": dict(q=19, n=256, storage="f32", pattern="aa", tau=0.6, F=(1e-6, 0.0, 0.0),
                             period=32, ratio=0.3,
                             desc="as d3q19_256_f32 with in-place AA streaming"),
    "d3q19_256_f64": dict(q=19, n=256, storage="f64", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                          period=32, ratio=0.3, desc="as d3q19_256_f32 with FP64 storage and arithmetic"),
    "d3q19_256_f16": dict(q=19, n=256, storage="f16", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                          period=32, ratio=0.3, desc="as d3q19_256_f32 with FP16 deviation storage"),
    "d3q19_256_bf16": dict(q=19, n=256, storage="bf16", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                           period=32, ratio=0.3, desc="as d3q19_256_f32 with BF16 deviation storage"),
    "d3q19_384_f16": dict(q=19, n=384, storage="f16", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                          field="boolean",
                          desc="D3Q19 HBGK 384^3 random periodic Boolean sphere matrix (seeded, radius "
                               "P*U[0.1,0.45], P = 32, phi* ~ U[0.4,0.9]), F = 1e-6, tau = 0.6, FP16 deviation "
                               "storage (s = 2^12), two-lattice"),
    "d3q19_384_bf16": dict(q=19, n=384, storage="bf16", pattern="two", tau=0.6, F=(1e-6, 0.0, 0.0),
                           field="boolean",
                           desc="D3Q19 HBGK 384^3 random periodic Boolean sphere matrix (as d3q19_384_f16), "
                                "BF16 deviation storage, two-lattice"),
    "d3q19_384_f16_aa": dict(q=19, n=384, storage="f16", pattern="aa", tau=0.6, F=(1e-6, 0.0, 0.0),
                             field="boolean", desc="as d3q19_384_f16 with in-place AA streaming"),
    "d3q19_384_bf16_aa": dict(q=19, n=384, storage="bf16", pattern="aa", tau=0.6, F=(1e-6, 0.0, 0.0),
                              field="boolean", desc="as d3q19_384_bf16 with in-place AA streaming"),
}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def shard(items, rank, world):
    """The units (requests, replicas) this rank owns: a strided split, no overlap."""
    return list(items)[rank::world]


def max_over_ranks(x, dist=None, device="cpu"):
    """Max of a scalar over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist=None, device="cpu"):
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


BOOLEAN_SEED = 2310147460 + 3  # seed of the random sphere-matrix workload


def make_field(w, render_n=None):
    """The porosity-control field of a workload: the regular sphere matrix, or the seeded random
    Boolean matrix (rendered at render_n to sample the same continuous geometry on a coarser grid)."""
    from paper_2310_14746_gb300 import inputs
    if w.get("field") == "boolean":
        return inputs.random_sphere_field(w["n"], BOOLEAN_SEED, render_n=render_n)[0]
    return inputs.regular_sphere_field(render_n or w["n"], period=w["period"], radius_ratio=w["ratio"])


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def oracle_mlups(w, varpi, steps=None, budget_s=15.0, threads=None):
    """FP64 oracle MLUPS on the full lattice of the workload; times `steps` time steps, or
    as many as fit in ~budget_s after a 1-step probe. threads: OpenMP threads (default: all
    host cores). Returns (mlups, steps, seconds, threads used)."""
    import oracle
    oracle.set_threads(threads or os.cpu_count() or 1)
    q, n = w["q"], w["n"]
    f = oracle.equilibrium_state(q, (n, n, n))
    vp = varpi.astype(np.float64)
    if steps is None:
        t0 = time.perf_counter()
        f = oracle.run(f, vp, w["tau"], w["F"], (0, 0, 0), 1)
        dt = time.perf_counter() - t0
        steps = int(max(1, min(50, budget_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    f = oracle.run(f, vp, w["tau"], w["F"], (0, 0, 0), steps)
    dt = time.perf_counter() - t0
    used = oracle.get_threads()
    oracle.set_threads(os.cpu_count() or 1)
    return n ** 3 * steps / dt / 1e6, steps, dt, used


def oracle_reference_96(w, field96, steps):
    """CPU-baseline run of the FP64 oracle at the error-check size of the random-sphere workload
    (96^3, the same continuous geometry, `steps` time steps from rest), on all host cores.
    Returns its timing and the reference velocity and apparent permeability the reduced-precision
    results are compared with."""
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    ref = oracle.run(oracle.equilibrium_state(19, field96.shape), field96.astype(np.float64), w["tau"], w["F"],
                     (0, 0, 0), steps)
    dt = time.perf_counter() - t0
    _, u = oracle.moments(ref, w["F"], (0, 0, 0))
    st = oracle.stats(ref, w["tau"], w["F"], (0, 0, 0))
    cells = int(np.prod(field96.shape))
    return {"mlups": cells * steps / dt / 1e6, "seconds": dt, "cores": oracle.get_threads(),
            "sample": "%d FP64 oracle time steps of the 96^3 resampled field" % steps}, u, st["k_app"]


def workload_config(w, check_every, world):
    """The `config` object of the bench line (the same for both arms)."""
    bpl = 2 * w["q"] * {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[w["storage"]] + 4
    cells = w["n"] ** 3
    return {"workload": w["desc"], "cells": cells, "time_steps_per_step": check_every, "check_every": check_every,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (%.2f GB streamed per time step)" % (bpl * cells / 1e9)}


def run_reference(args, w, rank):
    if rank != 0:
        return
    varpi = make_field(w)
    total_steps = 0
    total_t = 0.0
    # W warm-up + K timed oracle time steps, each a bounded sample of the workload
    oracle_mlups(w, varpi, steps=max(1, args.warmup))
    mlups, steps, dt, cores = oracle_mlups(w, varpi, steps=max(1, args.steps))
    total_steps += steps
    total_t += dt
    value = mlups
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / total_steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w, args.check_every, args.gpus),
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d FP64 oracle time steps of the full %d^3 lattice (each timed step of this "
                                   "arm is one oracle time step, a bounded sample of the workload)"
                                   % (steps, w["n"])},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_lattice(lat, inner, steps, warmup, stream):
    """Warm up, then time `steps` bench steps (inner time steps + one FP64 reduction) with CUDA
    events on the launching stream. Returns (ms per bench step, ms per time step of the step
    kernel alone, last diagnostics)."""
    import torch
    for _ in range(warmup):
        lat.step(inner)
        lat.reduce()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    st = None
    for a, b in evs:
        a.record(stream)
        lat.step(inner)
        b.record(stream)
        st = lat.reduce()
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps, sum(a.elapsed_time(b) for a, b in evs) / (steps * inner), st


def lattice_leg(w, field, storage, pattern, inner, steps, warmup, stream):
    """GLUPS, step-kernel time and roofline fraction of one workload through the product API."""
    import paper_2310_14746_gb300 as hb
    n, q = w["n"], w["q"]
    lat = hb.Lattice(q, n, n, n, storage, pattern)
    lat.set_relaxation(w["tau"])
    lat.set_force(*w["F"])
    lat.set_porosity(field)
    lat.init_equilibrium()
    ms_step, kern_ms, st = time_lattice(lat, inner, steps, warmup, stream)
    lat.close()
    cells = n ** 3
    bpl = 2 * q * hb.STORAGE_BYTES[storage] + 4
    peak, kind = measured_hbm_peak()
    achieved = bpl * cells / (kern_ms * 1e-3) / 1e9
    sname = {v: k for k, v in (("f64", hb.HLBM_F64), ("f32", hb.HLBM_F32), ("f16", hb.HLBM_F16DEV),
                               ("bf16", hb.HLBM_BF16DEV))}[storage]
    kname = "stream_collide_d%dq%d_%s_%s" % (3 if q == 19 else 2, q, sname,
                                             "aa" if pattern == hb.HLBM_AA else "two")
    traffic, note = kernel_traffic(kname, n)
    return {"glups": cells * inner / (ms_step * 1e-3) / 1e9, "ms_per_step": ms_step, "kernel_ms": kern_ms,
            "bytes_per_lup": bpl, "achieved_GBps": achieved, "frac": achieved / peak, "peak_kind": kind,
            "kernel": kname, "traffic": traffic, "traffic_note": note,
            "k_app": st["k_app"], "mass_rel_drift": st["mass"] / cells - 1.0}


def reduced_precision_leg(args, stream, with_oracle):
    """The random-sphere workload: FP16 and BF16 deviation storage at 384^3 (throughput and roofline
    at 80 B per lattice update), and at 96^3 on the same continuous geometry the velocity and
    apparent-permeability error of FP32, FP16 and BF16 after 2000 steps against the FP64 oracle
    (run on the host cores as the CPU baseline of this workload; skipped with_oracle=False)."""
    import paper_2310_14746_gb300 as hb
    w16 = WORKLOADS["d3q19_384_f16"]
    field = make_field(w16)
    out = {"workload": w16["desc"], "steps_per_bench_step": args.check_every}
    for name, storage in (("f16", hb.HLBM_F16DEV), ("bf16", hb.HLBM_BF16DEV)):
        out[name + "_384"] = lattice_leg(w16, field, storage, hb.HLBM_TWO_LATTICE, args.check_every,
                                         args.leg_steps, 3, stream)
    del field
    err_steps = 2000
    field96 = make_field(w16, render_n=96)
    gpu = {}
    for name, storage in (("f32", hb.HLBM_F32), ("f16", hb.HLBM_F16DEV), ("bf16", hb.HLBM_BF16DEV)):
        lat = hb.Lattice(19, 96, 96, 96, storage, hb.HLBM_TWO_LATTICE)
        lat.set_relaxation(w16["tau"])
        lat.set_force(*w16["F"])
        lat.set_porosity(field96)
        lat.init_equilibrium()
        lat.step(err_steps)
        st = lat.reduce()
        _, u = lat.moments()
        lat.close()
        gpu[name] = (u, st["k_app"])
    if with_oracle:
        timing, u_ref, k_ref = oracle_reference_96(w16, field96, err_steps)
        scale = float(np.abs(u_ref).max())
        out["error_96"] = {
            name: {"velocity_rel_err": float(np.abs(u.astype(np.float64) - u_ref).max() / scale),
                   "k_app_rel_err": abs(k - k_ref) / abs(k_ref)}
            for name, (u, k) in gpu.items()}
        out["error_96"]["reference"] = "FP64 oracle, 96^3, %d steps, k_app %.6g" % (err_steps, k_ref)
        out["oracle_96"] = timing
    return out


def aa_leg(args, w, field, stream):
    """The benchmark workload with in-place AA streaming, through the product API."""
    import paper_2310_14746_gb300 as hb
    return dict(lattice_leg(w, field, hb.HLBM_F32, hb.HLBM_AA, args.check_every, args.leg_steps, 3, stream),
                workload="as the benchmark workload, in-place AA streaming (one population copy)")


def adjoint_leg(n=128, nsteps=2000, every=45, period=32, ratio=0.3, tau=0.6, F=(1e-6, 0.0, 0.0)):
    """Gradient of the outflow flux w.r.t. varpi on the adjoint workload (128^3 regular spheres,
    2000 steps, state kept every 45 steps): wall time of the whole call and its algorithmic
    bytes (forward run + segment recomputation at 156 B/LUP, reverse steps at 240 B/LUP)."""
    import torch
    import paper_2310_14746_gb300 as hb
    from paper_2310_14746_gb300 import inputs
    vp = inputs.regular_sphere_field(n, period=period, radius_ratio=ratio)
    lat = hb.Lattice(19, n, n, n, hb.HLBM_F32, hb.HLBM_TWO_LATTICE)
    lat.set_relaxation(tau)
    lat.set_force(*F)
    lat.set_porosity(vp)
    grad = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    lat.init_equilibrium()
    lat.adjoint_flux_grad(2 * every, every, n - 1, grad)  # warm-up (allocator, modules)
    lat.init_equilibrium()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, _ = lat.adjoint_flux_grad(nsteps, every, n - 1, grad)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    lat.close()
    cells = n ** 3
    nsnap = (nsteps - 1) // every + 1
    algo = cells * ((2 * nsteps - nsnap) * 156 + nsteps * 240)
    peak, kind = measured_hbm_peak()
    return {"workload": "D3Q19 %d^3 regular spheres (period %d, r = %.1f P), %d steps, checkpoint every %d"
                        % (n, period, ratio, nsteps, every),
            "seconds": dt, "J": J, "adjoint_mlups": cells * nsteps / dt / 1e6,
            "achieved_GBps": algo / dt / 1e9, "frac_of_peak": algo / dt / 1e9 / peak, "peak_kind": kind,
            "grad_abs_max": float(grad.abs().max().item())}


def served_vs_fp64(trace, res_b, res_p, field_of, max_edge=64, lu_budget=1.2e10, tau=0.6, F=(1e-6, 0.0, 0.0),
                   steady_tol=1e-8, check=100):
    """Velocity error of served results against FP64. Each request of edge <= max_edge (smallest
    first, within lu_budget lattice updates) is re-run with FP64 storage and arithmetic on the
    same field from the same rest state (the FP64 policy equals the FP64 oracle to round-off in
    the parity tests):
      - "same_step": max|u - u64(n)| / max|u64(n)| at the step count n at which the batched server
        and the plain FP32 loop each returned it (how far the trajectory moved: FP16 rounding
        during the transient for the batched form, FP32 rounding for the plain loop);
      - "steady": max|u - u64_inf| / max|u64_inf| against the FP64 steady state, run on until
        max|du| over `check` steps falls below steady_tol (100x under the serving tolerance),
        which also counts the distance from steady state at which the serving tolerance stops
        either form."""
    import paper_2310_14746_gb300 as hb
    by_tag = {rq["id"]: rq for rq in trace}
    plain = {r["tag"]: r for r in res_p}
    cand = sorted((r for r in res_b if by_tag[r["tag"]]["edge"] <= max_edge and r["tag"] in plain
                   and r["u"] is not None and plain[r["tag"]]["u"] is not None),
                  key=lambda r: by_tag[r["tag"]]["edge"] ** 3 * max(r["steps"], plain[r["tag"]]["steps"]))
    rows, lu = [], 0.0
    for r in cand:
        rq, rp = by_tag[r["tag"]], plain[r["tag"]]
        n = rq["edge"]
        served = max(r["steps"], rp["steps"])
        cap = 4 * served + 20000  # steps of the steady-state run at most
        if lu + float(n) ** 3 * cap > lu_budget:
            break
        lat = hb.Lattice(19, n, n, n, hb.HLBM_F64, hb.HLBM_TWO_LATTICE)
        lat.set_relaxation(tau)
        lat.set_force(*F)
        lat.set_porosity(field_of(rq))
        lat.init_equilibrium()
        err, done = {}, 0
        served_u = {"batched": r["u"].astype(np.float64), "plain_f32": rp["u"].astype(np.float64)}
        for name, steps in sorted((("batched", r["steps"]), ("plain_f32", rp["steps"])), key=lambda t: t[1]):
            lat.step(steps - done)
            done = steps
            u64 = lat.moments(f64=True)[1]
            err[name] = float(np.abs(served_u[name] - u64).max() / np.abs(u64).max())
        lat.reduce()  # residual reference at the last served step
        converged = False
        while done < cap:
            lat.step(check)
            done += check
            if lat.reduce()["max_du"] < steady_tol:
                converged = True
                break
        u_inf = lat.moments(f64=True)[1]
        lat.close()
        lu += float(n) ** 3 * done
        scale = np.abs(u_inf).max()
        rows.append({"edge": n, "steps_batched": r["steps"], "steps_plain": rp["steps"],
                     "same_step": {"batched": err["batched"], "plain_f32": err["plain_f32"]},
                     "steady": {k: float(np.abs(v - u_inf).max() / scale) for k, v in served_u.items()},
                     "steady_steps": done, "steady_converged": converged})
    if not rows:
        return None
    return {"requests": len(rows),
            "max_same_step": {k: max(x["same_step"][k] for x in rows) for k in ("batched", "plain_f32")},
            "max_steady": {k: max(x["steady"][k] for x in rows) for k in ("batched", "plain_f32")},
            "per_request": rows,
            "reference": "FP64 storage and arithmetic on the GPU, same field: the state at the served step count, "
                         "and the steady state (max|du| < %g per %d steps)" % (steady_tol, check)}


def serving_leg(n_requests, seed, max_edge=192, tol=1e-6, budget_gb=64, rank=0, world=1, dist=None,
                capacity_requests=0, backfill=None):
    """Serving stream sample: the first n_requests of the seeded trace (edges up to max_edge).
    1) capacity: all requests (or the first capacity_requests of them) at t = 0 through the
       batched FP16 server -> solves/s;
    2) Poisson arrivals at 0.8x that capacity, replayed in real time through the batched server
       and through the plain FP32 loop (one solve at a time, one launch per step);
    returns p50/p99 time-to-steady-state of both, throughput, and the permeability difference
    between the FP16 batched and FP32 plain results."""
    from paper_2310_14746_gb300 import inputs
    from paper_2310_14746_gb300 import serving as sv
    import paper_2310_14746_gb300 as hb

    base = [r for r in inputs.serving_requests(4 * n_requests, seed, rate_per_s=1.0) if r["edge"] <= max_edge]
    base = shard(base[:n_requests], rank, world)  # requests are independent: split them over ranks
    cache = {}

    def field_of(rq):
        key = (rq["edge"], rq["period"], round(rq["radius_ratio"], 12))
        if key not in cache:
            cache[key] = inputs.regular_sphere_field(rq["edge"], period=rq["period"], radius_ratio=rq["radius_ratio"])
        return cache[key]

    for rq in base:
        field_of(rq)
    cap_set = base[:capacity_requests] if capacity_requests > 0 else base
    res0, info0 = sv.run_stream(cap_set, field_of, storage=hb.HLBM_F16DEV, mem_budget=budget_gb << 30, tol=tol,
                                realtime=False, backfill=backfill)
    cap = len(res0) / max(max(r["t_finish"] for r in res0), 1e-9)
    rate = 0.8 * cap
    trace = [dict(rq) for rq in base]
    t = 0.0
    rng = np.random.default_rng(seed + 1)
    for rq in trace:
        t += float(rng.exponential(1.0 / rate))
        rq["arrival_s"] = t
    want_u = len(trace) <= 64  # final velocities kept on the host for the comparison
    res_b, info_b = sv.run_stream(trace, field_of, storage=hb.HLBM_F16DEV, mem_budget=budget_gb << 30, tol=tol,
                                  want_u=want_u, backfill=backfill)
    res_p, info_p = sv.plain_loop(trace, field_of, tol=tol, want_u=want_u)
    kb = {r["tag"]: r["k_app"] for r in res_b}
    kp = {r["tag"]: r["k_app"] for r in res_p}
    kerr = max(abs(kb[k] - kp[k]) / abs(kp[k]) for k in kb if k in kp and kp[k] != 0)
    uerr = None
    fp64 = None
    if want_u:
        ub = {r["tag"]: r["u"] for r in res_b}
        uerr = max(float(np.abs(ub[r["tag"]] - r["u"]).max() / np.abs(r["u"]).max()) for r in res_p)
        fp64 = served_vs_fp64(trace, res_b, res_p, field_of)
    cells_of = {rq["id"]: rq["edge"] ** 3 for rq in trace}
    lu_all = sum(r["steps"] * cells_of[r["tag"]] for r in res_b)
    lu_low = sum(r["steps_low"] * cells_of[r["tag"]] for r in res_b)
    pb = sv.percentiles([r["latency_s"] for r in res_b])
    pp = sv.percentiles([r["latency_s"] for r in res_p])
    span_b = max(r["t_finish"] for r in res_b)
    per_request = None
    if len(trace) <= 32:
        lp = {r["tag"]: r["latency_s"] for r in res_p}
        per_request = [{"edge": cells_of[r["tag"]] ** (1 / 3), "steps": r["steps"], "steps_low": r["steps_low"],
                        "latency_batched_s": r["latency_s"], "latency_plain_s": lp.get(r["tag"])}
                       for r in sorted(res_b, key=lambda r: r["tag"])]
        for e in per_request:
            e["edge"] = int(round(e["edge"]))
    if dist is not None:  # whole-job throughput; tail latency as the worst rank's
        pb["p99_s"] = max_over_ranks(pb["p99_s"], dist, "cuda")
        pp["p99_s"] = max_over_ranks(pp["p99_s"], dist, "cuda")
        kerr = max_over_ranks(kerr, dist, "cuda")
    by_edge = {}
    lp_all = {r["tag"]: r["latency_s"] for r in res_p}
    for e in sorted({rq["edge"] for rq in trace}):
        tb = [r["latency_s"] for r in res_b if cells_of[r["tag"]] == e ** 3]
        tp = [lp_all[r["tag"]] for r in res_b if cells_of[r["tag"]] == e ** 3 and r["tag"] in lp_all]
        by_edge[str(e)] = {"n": len(tb), "batched": sv.percentiles(tb), "plain": sv.percentiles(tp)}
    return {
        "requests": len(trace), "edges": sorted({r["edge"] for r in trace}), "tol_max_du": tol,
        "backfill": backfill if backfill is not None else "library default",
        "capacity_solves_per_s": cap, "capacity_requests": len(cap_set), "arrival_rate_per_s": rate,
        "by_edge": by_edge if len(trace) > 32 else None,
        "lattice_updates": {"batched": int(lu_all), "low_precision": int(lu_low)},
        "batched_f16": {"p50_s": pb["p50_s"], "p99_s": pb["p99_s"],
                        "solves_per_s": sum_over_ranks(len(res_b) / span_b, dist, "cuda"),
                        "mlups": sum_over_ranks(info_b["lattice_updates"] / info_b["elapsed_s"] / 1e6, dist, "cuda"),
                        "converged": sum(r["status"] == 0 for r in res_b),
                        "refined_to_fp32": sum(r.get("final_storage") == hb.HLBM_F32 for r in res_b)},
        "plain_f32": {"p50_s": pp["p50_s"], "p99_s": pp["p99_s"],
                      "solves_per_s": sum_over_ranks(len(res_p) / info_p["elapsed_s"], dist, "cuda"),
                      "mlups": sum_over_ranks(info_p["lattice_updates"] / info_p["elapsed_s"] / 1e6, dist, "cuda"),
                      "converged": sum(r["status"] == 0 for r in res_p)},
        "k_app_rel_diff_f16_batched_vs_f32_plain": kerr,
        "velocity_rel_diff_batched_vs_f32_plain": uerr,
        "velocity_rel_err_vs_fp64": fp64,
        "lattice_update_share_16bit": lu_low / max(lu_all, 1),
        "per_request": per_request,
        "steps": {"min": int(min(r["steps"] for r in res_b)), "max": int(max(r["steps"] for r in res_b))},
    }


def serving_class_leg(groups, rounds=20, warm_rounds=3, check_every=100, period=32, ratio=0.3):
    """Throughput of kernel classes of the batched server: for each (edge, count, storage) of
    `groups`, `count` identical slots of edge `edge` (regular sphere matrix) in `storage`, all of
    them in one server and in every round (processor sharing), never retired or widened (a
    tolerance of 1e-300, no refinement). Each round is check_every batched time steps (one graph
    replay) plus the per-slot FP64 check, timed on the host around hlbm_server_pump (which
    synchronises). Returns GLUPS and the fraction of the measured copy bandwidth at the storages'
    algorithmic bytes per lattice update."""
    import paper_2310_14746_gb300 as hb
    from paper_2310_14746_gb300 import inputs
    from paper_2310_14746_gb300 import serving as sv
    kinds = {"f32": hb.HLBM_F32, "f16": hb.HLBM_F16DEV, "bf16": hb.HLBM_BF16DEV}
    srv = sv.Server(96 << 30, kinds[groups[0][2]], check_every, refine=False, backfill=1e6)
    total, lups, byts, tag = 0, 0.0, 0.0, 0
    for edge, count, storage_name in groups:
        storage = kinds[storage_name]
        # a request's storage is the server's (it starts every slot in that storage); a group in
        # another storage needs its own server, so mixed specs keep one storage
        if storage != kinds[groups[0][2]]:
            raise SystemExit("--serving-class: the groups of one spec share a storage")
        field = inputs.regular_sphere_field(edge, period=min(period, edge), radius_ratio=ratio)
        for _ in range(count):
            srv.submit(field, tol=1e-300, max_steps=10 ** 9, tag=tag)
            tag += 1
        total += count
        cells = float(count) * edge ** 3
        lups += cells * check_every * rounds
        byts += cells * check_every * rounds * (2 * 19 * hb.STORAGE_BYTES[storage] + 4)
    for _ in range(warm_rounds):
        srv.pump()
    t0 = time.perf_counter()
    for _ in range(rounds):
        a, _w = srv.pump()
    dt = time.perf_counter() - t0
    srv.close()
    if a != total:
        raise RuntimeError("serving class: %d of %d slots live" % (a, total))
    peak, kind = measured_hbm_peak()
    return {"groups": [{"edge": e, "slots": c, "storage": st} for e, c, st in groups], "rounds": rounds,
            "check_every": check_every, "seconds": dt, "glups": lups / dt / 1e9,
            "achieved_GBps": byts / dt / 1e9, "frac": byts / dt / 1e9 / peak, "peak_kind": kind}


def run_adjoint_only(args, local_rank):
    """--adjoint-only: the adjoint-gradient leg alone (config-5 workload by default), one JSON line."""
    import torch
    from paper_2310_14746_gb300 import build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local_rank)
    build.build()
    out = adjoint_leg(n=args.adjoint_n, nsteps=args.adjoint_steps)
    print(json.dumps({"metric": METRIC, "impl": "ours", "mode": "adjoint-only", "adjoint": out}), flush=True)


def run_serving_class(args, local_rank):
    """--serving-class EDGE:COUNT:STORAGE[,...]: one JSON line with each class's throughput."""
    import torch
    from paper_2310_14746_gb300 import build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local_rank)
    build.build()
    out = []
    for spec in args.serving_class.split(","):
        groups = [(int(e), int(c), st) for e, c, st in (g.split(":") for g in spec.split("+"))]
        out.append(serving_class_leg(groups, rounds=args.steps, warm_rounds=max(1, args.warmup)))
    print(json.dumps({"metric": METRIC, "impl": "ours", "mode": "serving-class", "classes": out}), flush=True)


def run_serving_only(args, rank, world, local_rank):
    """Only the serving leg (for long traces): one JSON line with the serving object."""
    import torch
    from paper_2310_14746_gb300 import build
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local_rank)
    build.build()
    t0 = time.perf_counter()
    serving = serving_leg(args.serving_requests, 2310147460 + 4, max_edge=args.serving_max_edge,
                          rank=rank, world=world, capacity_requests=args.serving_capacity_requests,
                          backfill=args.serving_backfill)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "impl": "ours", "mode": "serving-only", "n_gpus": world,
                          "wall_s": time.perf_counter() - t0, "serving": serving}), flush=True)


def run_gpu(args, w, rank, world, local_rank):
    import torch
    import paper_2310_14746_gb300 as hb
    from paper_2310_14746_gb300 import build

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local_rank)
    build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    storage = {"f64": hb.HLBM_F64, "f32": hb.HLBM_F32, "f16": hb.HLBM_F16DEV, "bf16": hb.HLBM_BF16DEV}[w["storage"]]
    pattern = hb.HLBM_AA if w["pattern"] == "aa" else hb.HLBM_TWO_LATTICE
    n, q = w["n"], w["q"]
    cells = n ** 3
    inner = args.check_every
    varpi = make_field(w)
    varpi_pinned = torch.from_numpy(varpi).pin_memory()
    stream = torch.cuda.current_stream()

    lat = hb.Lattice(q, n, n, n, storage, pattern)
    lat.set_relaxation(w["tau"])
    lat.set_force(*w["F"])
    lat.set_porosity(varpi_pinned.numpy())
    lat.init_equilibrium()

    launches_per_step = inner + 2  # stream-collide launches + 2 reduction kernels

    def one_step(ev_a=None, ev_b=None):
        if ev_a is not None:
            ev_a.record(stream)
        lat.step(inner)
        if ev_b is not None:
            ev_b.record(stream)
        return lat.reduce()

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            st = one_step(*evs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed_ms = t_start.elapsed_time(t_end)
    kern_ms = sum(a.elapsed_time(b) for a, b in evs) / (args.steps * inner)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, "cuda")
    value = world * cells * inner * args.steps / (elapsed_ms * 1e-3) / 1e6

    # ---- e2e through the C ABI with host buffers --------------------------------
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_porosity(varpi_pinned.numpy())  # host -> device, validated
        lat.init_equilibrium()
        lat.step(inner)
        st_e2e = lat.reduce()                   # device -> host diagnostics
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = world * cells * inner * e2e_steps / e2e_s / 1e6
    h2d = cells * 4 + q * 8
    d2h = 8 * 8

    bytes_per_lup = 2 * q * hb.STORAGE_BYTES[storage] + 4
    achieved = bytes_per_lup * cells / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = measured_hbm_peak()
    kname = "stream_collide_d%dq%d_%s_%s" % (3 if q == 19 else 2, q, w["storage"], w["pattern"])
    traffic, traffic_note = kernel_traffic(kname, n)

    aa = None
    if not args.no_legs and w["pattern"] == "two" and w["storage"] == "f32":
        aa = aa_leg(args, w, varpi, stream)

    reduced = None
    if not args.no_legs and rank == 0:
        reduced = reduced_precision_leg(args, stream, with_oracle=(world == 1 and not args.no_cpu_baseline))

    adjoint = None
    if not args.no_adjoint and not args.no_legs:
        adjoint = adjoint_leg()

    serving = None
    if args.serving_requests > 0:
        lat.close()
        lat = None
        serving = serving_leg(args.serving_requests, 2310147460 + 4, max_edge=args.serving_max_edge,
                              rank=rank, world=world, dist=dist)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, ksteps, dt, cores = oracle_mlups(w, varpi, budget_s=args.cpu_budget)
        m1, s1, d1, _ = oracle_mlups(w, varpi, steps=1, threads=1)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "%d FP64 oracle time steps of the full %d^3 lattice (%.1f s)" % (ksteps, n, dt),
               "cores_1": {"value": m1, "unit": "MLUPS", "cores": 1,
                           "sample": "%d FP64 oracle time step of the full %d^3 lattice on one core (%.1f s)"
                                     % (s1, n, d1)}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": w["storage"], "data": "synthetic",
            "config": workload_config(w, inner, world),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_note": traffic_note,
                         "kernel_source_hash": kernel_source_hash(kname), "peak_kind": peak_kind,
                         "kernel": kname, "kernel_ms": kern_ms, "bytes_per_lup": bytes_per_lup},
            "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "stats": {"k_app": st["k_app"], "mass_rel_drift": st["mass"] / cells - 1.0, "max_du": st["max_du"]},
            "aa": aa,
            "reduced_precision": reduced,
            "adjoint": adjoint,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if lat is not None:
        lat.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="d3q19_256_f32")
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=16,
                    help="replay this many requests of the seeded serving trace, batched vs plain (0: skip)")
    ap.add_argument("--serving-max-edge", type=int, default=128)
    ap.add_argument("--serving-capacity-requests", type=int, default=0,
                    help="measure the batched capacity on the first K requests only (0: all of them)")
    ap.add_argument("--serving-backfill", type=float, default=None,
                    help="age-priority window of the batched server in the serving leg (default: the library's)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving leg (long traces) and print its JSON object")
    ap.add_argument("--serving-class", default="",
                    help="EDGE:COUNT:STORAGE[+EDGE:COUNT:STORAGE...][,...] (storage f32|f16|bf16): time these "
                         "batched-server slot sets (COUNT identical slots per group, the groups of one spec in one "
                         "server, --steps rounds after --warmup) and print their throughput only")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the adjoint-gradient leg (--adjoint-n, --adjoint-steps) and print it")
    ap.add_argument("--adjoint-n", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-gradient leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the AA, reduced-precision and adjoint legs (the main line only)")
    ap.add_argument("--leg-steps", type=int, default=5, help="timed bench steps of each lattice leg")
    args = ap.parse_args()
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w, rank)
    elif args.serving_class:
        run_serving_class(args, local_rank)
    elif args.adjoint_only:
        run_adjoint_only(args, local_rank)
    elif args.serving_only:
        run_serving_only(args, rank, world, local_rank)
    else:
        run_gpu(args, w, rank, world, local_rank)


if __name__ == "__main__":
    main()
