"""Serving: a request loop over the library's continuous-batching server.

Server wraps the C ABI (hlbm_server_*). run_stream() replays a request trace with
arrival times in real time: requests are submitted when they arrive, every round
admits what fits, advances all live solves by one check interval in batched
persistent launches and retires converged ones. plain_loop() is the comparison: one
FP32 solve at a time through the single-lattice API, one kernel launch per time step.
Latency = finish - arrival (time to steady state, queueing included).
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import (HLBM_F16DEV, HLBM_F32, HLBM_D3Q19, HLBM_TWO_LATTICE, Lattice, hlbm_request,
               hlbm_server_cancel, hlbm_server_create, hlbm_server_destroy, hlbm_server_info,
               hlbm_server_inject_alloc_failures, hlbm_server_poll, hlbm_server_pump, hlbm_server_set_priority,
               hlbm_server_set_refinement, hlbm_server_submit)


class Server:
    def __init__(self, mem_budget=32 << 30, storage=HLBM_F16DEV, check_every=100, stream=None, refine=None,
                 floor_coef=None, backfill=None):
        self.s = hlbm_server_create(mem_budget, storage, check_every, stream)
        if backfill is not None:
            hlbm_server_set_priority(self.s, backfill)
        self._keep = {}  # id -> (field, u_out) kept alive until polled
        if refine is not None or floor_coef is not None:
            default = 1.6e-2 if storage == 3 else 2e-3
            hlbm_server_set_refinement(self.s, True if refine is None else refine,
                                       default if floor_coef is None else floor_coef)

    def close(self):
        if self.s:
            hlbm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, varpi, tau=0.6, F=(1e-6, 0.0, 0.0), tol=1e-6, max_steps=10 ** 6, want_u=False, tag=0):
        varpi = np.ascontiguousarray(varpi, dtype=np.float32)
        nz, ny, nx = varpi.shape
        u_out = np.empty((3, nz, ny, nx), dtype=np.float32) if want_u else None
        req = hlbm_request(nx=nx, ny=ny, nz=nz, tau=tau, F=(ctypes.c_double * 3)(*F),
                           varpi=varpi.ctypes.data, tol=tol, max_steps=max_steps,
                           u_out=None if u_out is None else u_out.ctypes.data, tag=tag)
        rid = hlbm_server_submit(self.s, req)
        self._keep[rid] = u_out
        return rid

    def pump(self):
        return hlbm_server_pump(self.s)

    def poll(self):
        out = []
        for r in hlbm_server_poll(self.s):
            r["u"] = self._keep.pop(r["id"], None)
            out.append(r)
        return out

    def cancel(self, rid):
        hlbm_server_cancel(self.s, rid)

    def info(self):
        return hlbm_server_info(self.s)

    def inject_alloc_failures(self, n):
        hlbm_server_inject_alloc_failures(self.s, n)

    def run_until_idle(self):
        results = []
        while True:
            a, w = self.pump()
            results += self.poll()
            if a == 0 and w == 0:
                return results


def run_stream(trace, field_of, storage=HLBM_F16DEV, mem_budget=64 << 30, check_every=100, tol=1e-6,
               max_steps=10 ** 6, tau=0.6, F=(1e-6, 0.0, 0.0), realtime=True, want_u=False, backfill=None):
    """Replay `trace` (dicts with id and arrival_s, sorted by arrival) through a server.
    Requests are submitted once their arrival time has passed (checked between rounds);
    latency = finish - arrival on the server's clock, which starts with the trace.
    With realtime=False every request arrives at t = 0. want_u: each result carries its final
    velocity as "u". backfill: the server's age-priority window (None: the library default).
    Returns (results, info)."""
    srv = Server(mem_budget, storage, check_every, backfill=backfill)
    t0 = time.perf_counter()  # the server clock started just before
    arrival = {}
    results = []
    k = 0
    while True:
        now = time.perf_counter() - t0
        while k < len(trace) and (not realtime or trace[k]["arrival_s"] <= now):
            rq = trace[k]
            rid = srv.submit(field_of(rq), tau=tau, F=F, tol=tol, max_steps=max_steps, tag=rq["id"],
                             want_u=want_u)
            arrival[rid] = rq["arrival_s"] if realtime else 0.0
            k += 1
        a, w = srv.pump()
        results += srv.poll()
        if a == 0 and w == 0:
            if k >= len(trace):
                break
            wait = trace[k]["arrival_s"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
    info = srv.info()
    srv.close()
    for r in results:
        r["latency_s"] = r["t_finish"] - arrival[r["id"]]
    return results, info


def plain_loop(trace, field_of, tol=1e-6, max_steps=10 ** 6, tau=0.6, F=(1e-6, 0.0, 0.0), check_every=100,
               realtime=True, want_u=False):
    """One FP32 solve at a time, one launch per time step (no graphs, no batching).
    Returns results with latency = finish - arrival (and the final velocity as "u" with want_u)."""
    t0 = time.perf_counter()
    results = []
    lups = 0
    for rq in trace:
        if realtime:
            wait = rq["arrival_s"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        f = field_of(rq)
        nz, ny, nx = f.shape
        lat = Lattice(HLBM_D3Q19, nx, ny, nz, HLBM_F32, HLBM_TWO_LATTICE)
        lat.set_relaxation(tau)
        lat.set_force(*F)
        lat.set_porosity(f)
        lat.init_equilibrium()
        steps = 0
        status = 0
        while True:
            for _ in range(check_every):
                lat.step(1)
            steps += check_every
            st = lat.reduce()
            if st["max_du"] < tol:
                break
            if steps >= max_steps:
                status = -4
                break
        lups += steps * nx * ny * nz
        t_fin = time.perf_counter() - t0
        u = lat.moments()[1] if want_u else None
        results.append({"tag": rq["id"], "status": status, "steps": steps, "k_app": st["k_app"],
                        "latency_s": t_fin - (rq["arrival_s"] if realtime else 0.0), "nx": nx, "u": u})
        lat.close()
    return results, {"lattice_updates": lups, "elapsed_s": time.perf_counter() - t0}


def percentiles(lat_s):
    a = np.sort(np.asarray(lat_s, dtype=np.float64))
    if a.size == 0:
        return {"p50_s": None, "p99_s": None}
    return {"p50_s": float(np.percentile(a, 50)), "p99_s": float(np.percentile(a, 99)),
            "mean_s": float(a.mean()), "max_s": float(a.max())}
