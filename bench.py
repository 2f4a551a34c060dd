"""Benchmark: fused Shan-Chen lattice-Boltzmann steps on GB300.

Workload (the headline configuration): D3Q19, E8 forcing stencil (92
vectors), 256^3 periodic box with one bubble of radius 40 (rho 0.15 inside,
1.9 outside, tanh width 2), shifted binary32 populations, G = -5 (force
without c_s^2), tau = 1.  One step = psi, stencil force, BGK + Guo
collision and streaming over all 16.8 M nodes.  Populations (2 x 1.27 GB)
are far larger than L2, so no flush is needed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  ``value`` is MLUPS over all ranks (one independent
replica per GPU: the workload has no exchange step on one device), timed
with CUDA events on the library's stream between barriers, max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline (D3Q19 E8, FP32 vs FP64); adjoint steps/s at 1e-3 sigma"
NX = NY = NZ = 256
RADIUS = 40.0
G = -5.0
# G = -5 read with the force of eq. sc_f as printed (G c_s^2): supercritical,
# the run stays physical for any number of steps.  Read without c_s^2 (the
# library's default convention) the same G is a deep quench whose spinodal
# exterior blows up near step 90 on this machine; the bench times that reading
# too, over the steps before the blow-up ("literal_g"), with the same kernels.
CONVENTION = "paper"
WORKLOAD = ("D3Q19 E8 (92-vector forcing stencil) 256^3 periodic, bubble R=40 "
            "(rho_in 0.15, rho_out 1.9, tanh width 2), shifted FP32, G=-5 (G c_s^2 in the "
            "force), tau=1")
# algorithmic bytes per node update and kernel (population read + write,
# plus the psi field where a kernel reads or writes it)
ALG_BYTES = {"fused": 2 * 19 * 4, "collide": 2 * 19 * 4 + 4, "psi": 19 * 4 + 4}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources that decide what the fused D3Q19 step kernel reads and writes:
# the kernel, its helpers and parameters, and the padded population layout
# (api.cu); the 2D, binary64 and adjoint units, and the binary64 exp/pow
# (expcr.cuh, which the binary32 kernel includes but never calls), do not
FUSED_SOURCES = ("api.cu", "fused3d.cu", "fused3d_tma.cu", "fusedcommon.cuh", "internal.h",
                 "kernels.cuh")


def _src_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_23647_gb300", "csrc")
    for f in FUSED_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        with open(p) as fh:
            d = json.loads("".join(l for l in fh if not l.startswith("#")))
    except Exception:
        return None
    e = d.get(kernel)
    if not e or e.get("src_sha") != _src_hash():
        return None
    return e.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws
    return None, 0, 1


def reduce_max(dist, value, device=None):
    """Max over ranks (identity without a process group)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(dist, ms, nodes, steps, ws, device=None):
    """Whole-job MLUPS of N replicas: every rank updated `nodes` nodes for
    `steps` steps; the job took the slowest rank's time (ms, max over ranks)."""
    ms_max = reduce_max(dist, ms, device)
    return ms_max, nodes * steps * ws / (ms_max * 1e3)


def _workload_rho():
    import lbinputs as L
    return L.tanh_sphere(NX, NY, NZ, RADIUS, 0.15, 1.9, 2.0)


# ---------------------------------------------------------------------------
def oracle_mlups(sub, steps):
    """The FP64 oracle as it stands, single thread, on a centred sub-box of
    the workload (same lattice, stencil and physics); returns MLUPS."""
    import lbinputs as L
    import oracle
    rho = _workload_rho()
    c = NX // 2
    h = sub // 2
    box = np.ascontiguousarray(rho[c - h:c - h + sub, c - h:c - h + sub, c - h:c - h + sub])
    o = oracle.Oracle("D3Q19", box.shape, L.E8_3D.groups, tau=1.0, G=G, convention=CONVENTION)
    o.init_equilibrium(box)
    o.step(1)  # warm
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return box.size * steps / dt / 1e6, dt


def _oracle_box_worker(args):
    """One process of the all-core baseline: the oracle on its own copy of
    the centred sub-box; returns (node updates, seconds)."""
    sub, steps = args
    v, dt = oracle_mlups(sub, steps)
    return v * 1e6 * dt, dt


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_mlups_allcore(sub, steps, procs):
    """The oracle on every host core at once: `procs` processes (started with
    spawn), each stepping its own copy of the sub-box; aggregate MLUPS =
    total node updates / the slowest process's time."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_box_worker, [(sub, steps)] * procs)
    return sum(r[0] for r in res) / max(r[1] for r in res) / 1e6, max(r[1] for r in res)


def run_reference(args, dist, rank, ws):
    if rank != 0:
        return
    # each step: one oracle step of a centred sub-box sized so the whole
    # --steps/--warmup run stays within about two minutes
    per_node = 2.8e-6
    budget = 100.0
    sub = int(max(8, min(64, (budget / (per_node * max(1, args.steps + args.warmup))) ** (1 / 3))))
    import lbinputs as L
    import oracle
    rho = _workload_rho()
    c, h = NX // 2, sub // 2
    box = np.ascontiguousarray(rho[c - h:c - h + sub, c - h:c - h + sub, c - h:c - h + sub])
    o = oracle.Oracle("D3Q19", box.shape, L.E8_3D.groups, tau=1.0, G=G, convention=CONVENTION)
    o.init_equilibrium(box)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = box.size * args.steps / dt / 1e6
    sample = f"FP64 C oracle, 1 thread, {sub}^3 centred sub-box of the workload per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# Configurations as written: C1 (the 256 x 4 binary64 slab) and C2 (the 20
# droplet / bubble runs), each with the coupling read literally (G' = G =
# -5, the library's default), read with c_s^2 (G' = -5/3, the printed eq.
# sc_f) and, as a stable two-phase companion, G' = -3 from its coexistence
# densities (eq. SCMaxwell).  Physics from the library's own binary64
# interface observables (lb_flat_interfaces, lb_curved_interface, fits).
COEX_GP3 = (0.4558015024901948, 2.249571904134268)   # eq. SCMaxwell at G' = -3


def _slab_rho(L, nx, ny, n_gas, n_liq):
    return L.tanh_slab(nx, ny, 1, 64 * nx // 256, 192 * nx // 256, n_gas, n_liq, 2.0)


def c1_leg(P, L, stream, steps=10000):
    """C1: D2Q9 E4 binary64, tau = 1, periodic 256 x 4, liquid slab x in
    [64, 192) with rho = 0.15 + 1.75 (tanh((x-64)/2) - tanh((x-192)/2))/2,
    10,000 steps: per reading, stability (or the first failing step), mass
    drift, and for a two-phase state the coexistence densities, sigma_0 and
    the Tolman length of both interfaces."""
    import torch
    out = {"lattice": "D2Q9 E4 256x4 binary64, tau 1", "steps": steps}
    readings = [("literal_G-5", -5.0, "literal", (0.15, 1.9)),
                ("cs2_G-5", -5.0, "paper", (0.15, 1.9)),
                ("companion_Gp-3", -3.0, "literal", COEX_GP3)]
    for name, G_, conv, (ng, nl) in readings:
        rho = _slab_rho(L, 256, 4, ng, nl)
        lat = P.Lattice("D2Q9", (256, 4), rho, L.E4_2D.bases, L.E4_2D.weights, precision="fp64",
                        tau=1.0, G=G_, convention=conv, stream=stream.cuda_stream)
        m0 = lat.observables()["mass"]
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ob = lat.observables()
        r = {"G": G_, "G_prime": G_ / 3.0 if conv == "paper" else G_, "initial": [ng, nl],
             "stable": ob["status"] == P.LB_OK, "first_failing_step": ob["error_step"],
             "steps_per_s": steps / (ms * 1e-3), "rho_min": ob["rho_min"], "rho_max": ob["rho_max"]}
        if r["stable"]:
            r["mass_drift_rel"] = (ob["mass"] - m0) / m0
            ifs = lat.flat_interfaces()
            r["interfaces"] = len(ifs)
            if ifs:
                r["n_l"] = [i["n_l"] for i in ifs]
                r["n_g"] = [i["n_g"] for i in ifs]
                r["sigma0"] = [i["sigma"] for i in ifs]
                r["delta"] = [i["delta"] for i in ifs]
                r["delta_ads"] = [i["delta_ads"] for i in ifs]
        lat.close()
        out[name] = r
    return out


def c2_leg(P, L, stream, steps=40000):
    """C2: D2Q9 E8 (24 vectors), 10 droplets and 10 bubbles, R = 8 .. 48 in
    periodic 256 x 256 boxes, tanh width 2, 40,000 steps, shifted binary32
    (one batch) and binary64 (each lattice on its own stream): per run
    stability, R_e, R_s, sigma_s, Delta P; the Laplace sigma and the curved
    Tolman length over the stable runs, and their binary32-vs-binary64
    relative differences.  sigma_0 for the Tolman fit: a 256 x 4 binary64
    slab of the same model."""
    import torch
    radii = (8, 12, 16, 20, 24, 28, 32, 36, 40, 48)
    c = (128.0, 128.0)
    out = {"lattice": "D2Q9 E8 256x256, tau 1", "steps": steps, "radii": list(radii)}
    readings = [("literal_G-5", -5.0, "literal", (0.15, 1.9)),
                ("companion_Gp-3", -3.0, "literal", COEX_GP3)]
    for name, G_, conv, (ng, nl) in readings:
        rhos = [L.tanh_sphere(256, 256, 1, R, nl, ng, 2.0, center=(c[0], c[1], 0.0)) for R in radii] + \
               [L.tanh_sphere(256, 256, 1, R, ng, nl, 2.0, center=(c[0], c[1], 0.0)) for R in radii]
        res = {}
        t0 = time.perf_counter()
        for prec in ("fp32", "fp64"):
            if prec == "fp32":
                lats = [P.Lattice("D2Q9", (256, 256), r, L.E8_2D.bases, L.E8_2D.weights,
                                  precision="fp32", tau=1.0, G=G_, convention=conv,
                                  stream=stream.cuda_stream) for r in rhos]
                b = P.Batch(lats, stream=stream.cuda_stream)
                b.step(steps)
                b.sync()
                b.close()
            else:
                lats = [P.Lattice("D2Q9", (256, 256), r, L.E8_2D.bases, L.E8_2D.weights,
                                  precision="fp64", tau=1.0, G=G_, convention=conv) for r in rhos]
                for _ in range(steps // 1000):
                    for lat in lats:
                        lat.step(1000)
            torch.cuda.synchronize()
            runs = []
            for lat in lats:
                ob = lat.observables()
                r = {"stable": ob["status"] == P.LB_OK, "first_failing_step": ob["error_step"],
                     "rho_min": ob["rho_min"], "rho_max": ob["rho_max"]}
                if r["stable"]:
                    try:
                        r.update(lat.curved_interface(c))
                    except P.LbError:
                        r["interface"] = False
                runs.append(r)
                lat.close()
            res[prec] = runs
        fin = lambda x: x["stable"] and all(k in x and np.isfinite(x[k]) and x[k] > 0
                                             for k in ("R_e", "R_s", "dP"))
        ok = [i for i in range(20) if all(fin(res[p][i]) for p in res)]
        # sigma_0 of the same model: a flat 256 x 4 binary64 slab
        sig0 = None
        try:
            sl = P.Lattice("D2Q9", (256, 4), _slab_rho(L, 256, 4, ng, nl), L.E8_2D.bases,
                           L.E8_2D.weights, precision="fp64", tau=1.0, G=G_, convention=conv,
                           stream=stream.cuda_stream)
            sl.step(10000)
            if sl.observables()["status"] == P.LB_OK:
                ifs = sl.flat_interfaces()
                if ifs:
                    sig0 = float(np.mean([i["sigma"] for i in ifs]))
            sl.close()
        except P.LbError:
            pass
        r = {"G": G_, "initial": [ng, nl], "stable_runs": {p: sum(x["stable"] for x in res[p]) for p in res},
             "first_failing_steps": {p: [x["first_failing_step"] for x in res[p]] for p in res},
             "seconds": time.perf_counter() - t0, "sigma0_flat": sig0}
        if len(ok) >= 2:
            fits = {}
            for p in res:
                sel = [res[p][i] for i in ok]
                try:
                    fits[p] = {"laplace_sigma": P.lb_fit_laplace(sel, 2)[0]}
                    if sig0:
                        fits[p]["tolman_delta"] = P.lb_fit_tolman(sel, 2, sig0)[0]
                except P.LbError:
                    fits[p] = {}
            r["fits"] = fits
            rel = lambda a, b: abs(a - b) / abs(b)
            r["fp32_vs_fp64_rel"] = {k: rel(fits["fp32"][k], fits["fp64"][k]) for k in fits["fp64"]
                                     if k in fits["fp32"]}
            r["fp32_vs_fp64_rel"]["R_s_max"] = max(rel(res["fp32"][i]["R_s"], res["fp64"][i]["R_s"]) for i in ok)
            r["fp32_vs_fp64_rel"]["sigma_s_max"] = max(rel(res["fp32"][i]["sigma_s"], res["fp64"][i]["sigma_s"]) for i in ok)
            r["runs_fp64"] = [{k: res["fp64"][i][k] for k in ("bubble", "R_e", "R_s", "sigma_s", "dP")}
                              for i in ok]
        r["runs_with_interface"] = len(ok)
        out[name] = r
    return out


def run_gb300(args, dist, rank, ws):
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    import lbinputs as L
    import paper_2505_23647_gb300 as P

    # a dedicated stream: the library orders all its work on it, and the
    # timing events are recorded on the same stream (the legacy default
    # stream has handle 0, which the C ABI reads as "create a stream")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    N = NX * NY * NZ
    rho = _workload_rho()
    # pinned host copy of the input (used by the end-to-end measurement)
    rho_pinned = torch.empty(rho.size, dtype=torch.float64, pin_memory=True)
    rho_pinned.numpy()[:] = rho.ravel()

    lat = P.Lattice("D3Q19", (NX, NY, NZ), rho_pinned.numpy(), L.E8_3D.bases,
                    L.E8_3D.weights, precision="fp32", tau=1.0, G=G, convention=CONVENTION,
                    stream=stream.cuda_stream)
    if args.zchunk:
        P.lb_set_option(lat.ctx, P.LB_OPT_ZCHUNK, args.zchunk)
    fused = P.lb_fused_active(lat.ctx)
    lat.step(args.warmup)
    lat.sync()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[local] if vis else str(local)
    sampler = ClockSampler(smi_index)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lat.launches()
    P.lb_timing(lat.ctx, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    kt = P.lb_timing_read(lat.ctx)
    P.lb_timing(lat.ctx, 0)
    launches = lat.launches() - launches0
    stable = lat.sync() == P.LB_OK
    ms_max, value = job_throughput(dist, ms, N, args.steps, ws, dev)

    # dominant kernel of the step and its roofline
    kind = max((k for k in kt if kt[k][1]), key=lambda k: kt[k][0])
    kms, kn = kt[kind]
    peak, peak_src = _peaks()
    achieved = ALG_BYTES[kind] * N / (kms / kn * 1e-3) / 1e9
    traffic = _traffic(kind)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": kind,
                "alg_bytes_per_node": ALG_BYTES[kind], "peak_source": f"{peak_src} hbm_gbs",
                "kernel_ms_avg": kms / kn,
                "step_kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in kt.items() if v[1]}}
    obs = lat.observables()
    # cost of one observables call (one fused pass, binary64 sums), host
    # wall time around the synchronous call, best of 5
    obs_ms = 1e9
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.observables()
        obs_ms = min(obs_ms, (time.perf_counter() - t0) * 1e3)
    lat.close()

    # end to end through the C ABI with host buffers, right after the main
    # workload (as a job of its own would run it): create from the pinned
    # host density (H2D), K steps, read back the density (D2H) and the
    # observables
    e2e = None
    if not args.no_e2e:
        rho_out = torch.empty(N, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = P.lb_create(P.make_params("D3Q19", (NX, NY, NZ), "fp32", 1.0, G, CONVENTION),
                          rho_pinned.numpy(), None, stream.cuda_stream)
        P.lb_set_stencil(ctx, 3, L.E8_3D.bases, L.E8_3D.weights)
        ta = time.perf_counter()       # lb_create synchronises: the upload is done
        P.lb_step(ctx, args.steps)
        P.lb_sync(ctx)
        tb = time.perf_counter()
        P._check(P._lib.lb_get_fields(P._vp(ctx), P._ptr(rho_out.numpy()), None), "lb_get_fields")
        o2 = P.lb_observables(ctx)
        t1 = time.perf_counter()
        P.lb_destroy(ctx)
        dt = reduce_max(dist, t1 - t0, dev)
        # where the time goes: the fixed costs (allocation, upload and
        # initialisation; read-back) against the steps, which they amortise
        e2e = {"value": N * args.steps * ws / dt / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": N * 8 / args.steps,
               "d2h_bytes_per_step": (N * 8 + 88) / args.steps,
               "seconds": dt, "mass": o2["mass"],
               "phases_s": {"create_upload": ta - t0, "steps": tb - ta, "readback": t1 - tb},
               "steps_only_mlups": N * args.steps / (tb - ta) / 1e6}

    # the literal reading of G (no c_s^2) over its stable window
    lit = None
    if not args.no_literal:
        latl = P.Lattice("D3Q19", (NX, NY, NZ), rho_pinned.numpy(), L.E8_3D.bases,
                         L.E8_3D.weights, precision="fp32", tau=1.0, G=G, convention="literal",
                         stream=stream.cuda_stream)
        latl.step(3)
        e0.record(stream)
        latl.step(60)
        e1.record(stream)
        torch.cuda.synchronize()
        msl = e0.elapsed_time(e1)
        okl = latl.sync() == P.LB_OK
        latl.close()
        lit = {"value": N * 60 / (msl * 1e3), "unit": "MLUPS", "steps": 60, "warmup": 3,
               "stable": okl}

    def time_variant(lat, steps):
        """Time `steps` steps of a 3D variant of the workload after the warm-up:
        throughput, the fused kernel's average time and its roofline fraction."""
        fused_k = P.lb_fused_active(lat.ctx)
        lat.step(args.warmup)
        P.lb_timing(lat.ctx, 1)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_v = e0.elapsed_time(e1)
        kt_v = P.lb_timing_read(lat.ctx)
        P.lb_timing(lat.ctx, 0)
        ok_v = lat.sync() == P.LB_OK
        ob_v = lat.observables()
        lat.close()
        kms_v, kn_v = kt_v.get("fused", (0.0, 0))
        return {"value": N * steps / (ms_v * 1e3), "unit": "MLUPS", "steps": steps,
                "ms_per_step": ms_v / steps, "fused_kernel": fused_k,
                "kernel_ms_avg": kms_v / kn_v if kn_v else None,
                "hbm_frac": ALG_BYTES["fused"] * N / (kms_v / kn_v * 1e-3) / 1e9 / peak
                if kn_v else None,
                "stable": ok_v, "rho_min": ob_v["rho_min"], "rho_max": ob_v["rho_max"]}

    # the same bubble with psi_eps (eq. psieps; eps = 10/31 of the E8 stencil's
    # e4 by eq. eps_moments) at 1.1 times its critical coupling, started from
    # its coexistence pair: the fused kernel's psi_eps instantiation
    peps = None
    if not args.no_psi_eps:
        pe = L.PSI_EPS_BUBBLE
        rho_e = L.tanh_sphere(NX, NY, NZ, RADIUS, pe["n_gas"], pe["n_liquid"], 2.0)
        peps = time_variant(P.Lattice("D3Q19", (NX, NY, NZ), rho_e, L.E8_3D.bases,
                                      L.E8_3D.weights, precision="fp32", tau=1.0, G=pe["Gp"],
                                      convention="literal", psi_eps=pe["eps"],
                                      stream=stream.cuda_stream), min(args.steps, 1000))
        peps.update({"eps": pe["eps"], "Gp": pe["Gp"], "densities": [pe["n_gas"], pe["n_liquid"]]})

    # the same bubble with the F^2 forcing variant (Sec. VI: T = 2 u F -
    # (A/tau) F F in eq. GuoForcing; the paper fixes no A, this uses 0.25):
    # the fused kernel's F^2 instantiation
    f2 = None
    if not args.no_f2:
        A_f2 = 0.25
        f2 = time_variant(P.Lattice("D3Q19", (NX, NY, NZ), rho_pinned.numpy(), L.E8_3D.bases,
                                    L.E8_3D.weights, precision="fp32", tau=1.0, G=G,
                                    convention=CONVENTION, forcing_A=A_f2,
                                    stream=stream.cuda_stream), min(args.steps, 1000))
        f2["A"] = A_f2

    # the paper's wide tuned stencils, which the fused kernels do not cover
    # (groups beyond radius 2): Table tab:e4e6_tuning_8 in 3D (N_e = 140, up
    # to (4,0,0), (3,3,0), (2,2,1)) on the same bubble, and in 2D (N_e = 32)
    # on a 2048^2 lattice; the generic binary32 two-kernel path (psi into a
    # halo'd field, then force from a shared-memory psi box + collision),
    # algorithmic bytes 80 + 156 per node
    wide = None
    if not args.no_wide:
        wide = {}
        st3 = L.stencil_e4e6_tuning_8(3, 0, 0)
        w3 = time_variant(P.Lattice("D3Q19", (NX, NY, NZ), rho_pinned.numpy(), st3.bases, st3.weights,
                                    precision="fp32", tau=1.0, G=G, convention=CONVENTION,
                                    stream=stream.cuda_stream), min(args.steps, 200))
        wide["d3q19_e4e6_tuning_8"] = w3
        n2 = 2048
        st2 = L.stencil_e4e6_tuning_8(2, 0, 0)
        rho2 = L.tanh_sphere(n2, n2, 1, 320.0, 0.15, 1.9, 2.0)
        lat2 = P.Lattice("D2Q9", (n2, n2), rho2, st2.bases, st2.weights, precision="fp32",
                         tau=1.0, G=G, convention=CONVENTION, stream=stream.cuda_stream)
        lat2.step(args.warmup)
        P.lb_timing(lat2.ctx, 1)
        k2 = min(args.steps, 200)
        e0.record(stream)
        lat2.step(k2)
        e1.record(stream)
        torch.cuda.synchronize()
        ms2 = e0.elapsed_time(e1)
        kt2 = P.lb_timing_read(lat2.ctx)
        P.lb_timing(lat2.ctx, 0)
        ok2 = lat2.sync() == P.LB_OK
        lat2.close()
        wide["d2q9_e4e6_tuning_8_2048"] = {
            "value": n2 * n2 * k2 / (ms2 * 1e3), "unit": "MLUPS", "ms_per_step": ms2 / k2,
            "stable": ok2, "step_kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in kt2.items() if v[1]}}
        for key, nodes, b in (("d3q19_e4e6_tuning_8", N, 2 * 19 * 4), ("d2q9_e4e6_tuning_8_2048", n2 * n2, 2 * 9 * 4)):
            v = wide[key]
            v["n_vectors"] = 140 if key.startswith("d3") else 32
            v["hbm_frac_two_kernel_bytes"] = (b + 8) * nodes / (v["ms_per_step"] * 1e-3) / 1e9 / peak
            v["hbm_frac_min_bytes"] = b * nodes / (v["ms_per_step"] * 1e-3) / 1e9 / peak

    # FP64 path on the same workload (fewer steps; binary64 arithmetic)
    fp64 = None
    if not args.no_fp64:
        lat64 = P.Lattice("D3Q19", (NX, NY, NZ), rho_pinned.numpy(), L.E8_3D.bases,
                          L.E8_3D.weights, precision="fp64", tau=1.0, G=G,
                          convention=CONVENTION, stream=stream.cuda_stream)
        lat64.step(2)
        lat64.sync()
        k64 = max(4, args.steps // 20)
        P.lb_timing(lat64.ctx, 1)
        e0.record(stream)
        lat64.step(k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        kt64 = P.lb_timing_read(lat64.ctx)
        lat64.close()
        v64 = N * k64 / (ms64 * 1e3)
        fp64 = {"value": v64, "unit": "MLUPS", "steps": k64, "ms_per_step": ms64 / k64,
                "hbm_frac": (2 * 19 * 8 + 16) * v64 * 1e6 / 1e9 / peak,
                "step_kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in kt64.items() if v[1]}}
        # the psi_eps bubble in binary64: the correctly rounded power per node
        if not args.no_psi_eps:
            pe = L.PSI_EPS_BUBBLE
            rho_e = L.tanh_sphere(NX, NY, NZ, RADIUS, pe["n_gas"], pe["n_liquid"], 2.0)
            late = P.Lattice("D3Q19", (NX, NY, NZ), rho_e, L.E8_3D.bases, L.E8_3D.weights,
                             precision="fp64", tau=1.0, G=pe["Gp"], convention="literal",
                             psi_eps=pe["eps"], stream=stream.cuda_stream)
            late.step(2)
            late.sync()
            P.lb_timing(late.ctx, 1)
            e0.record(stream)
            late.step(k64)
            e1.record(stream)
            torch.cuda.synchronize()
            mse = e0.elapsed_time(e1)
            kte = P.lb_timing_read(late.ctx)
            oke = late.sync() == P.LB_OK
            late.close()
            fp64["psi_eps"] = {"value": N * k64 / (mse * 1e3), "unit": "MLUPS", "steps": k64,
                               "ms_per_step": mse / k64, "stable": oke,
                               "step_kernels": {k: {"ms_total": v[0], "launches": v[1]}
                                                for k, v in kte.items() if v[1]}}

    # the small binary64 slab: D2Q9, E4, 256 x 4, liquid slab x in [64, 192)
    # (tanh width 2), 10,000 steps; launch-bound, stepped through the
    # context's CUDA graph.  G' = -3 from its coexistence pair (0.456, 2.25):
    # a 1.9 / 0.15 slab at G' = -5/3 drives the gas below zero
    slab = None
    if not args.no_small:
        rho_s = L.tanh_slab(256, 4, 1, 64, 192, 0.456, 2.25, 2.0)
        lats = P.Lattice("D2Q9", (256, 4), rho_s, L.E4_2D.bases, L.E4_2D.weights,
                         precision="fp64", tau=1.0, G=-3.0, convention="literal",
                         stream=stream.cuda_stream)
        lats.step(100)
        ks = 10000
        l0 = lats.launches()
        e0.record(stream)
        lats.step(ks)
        e1.record(stream)
        torch.cuda.synchronize()
        mss = e0.elapsed_time(e1)
        oks = lats.sync() == P.LB_OK
        slab = {"value": ks / (mss * 1e-3), "unit": "steps/s", "steps": ks,
                "mlups": 1024 * ks / (mss * 1e3), "ms_per_step": mss / ks,
                "launches_per_step": (lats.launches() - l0) / ks, "precision": "fp64",
                "stable": oks}
        lats.close()

    # 20 droplet / bubble runs (R = 8 .. 48 in 256 x 256 boxes, E8): binary32
    # as one batch, binary64 lattice by lattice.  G' = -3 from its coexistence
    # pair (0.456, 2.25): droplets of 1.9 in gas of 0.15 at G' = -5/3 drive the
    # gas below zero
    drops = None
    if not args.no_droplets:
        radii = (8, 12, 16, 20, 24, 28, 32, 36, 40, 48)
        rhos = [L.tanh_sphere(256, 256, 1, r, 2.25, 0.456, 2.0) for r in radii] + \
               [L.tanh_sphere(256, 256, 1, r, 0.456, 2.25, 2.0) for r in radii]
        nd = 20 * 256 * 256
        l32 = [P.Lattice("D2Q9", (256, 256), r, L.E8_2D.bases, L.E8_2D.weights, precision="fp32",
                         tau=1.0, G=-3.0, convention="literal", stream=stream.cuda_stream)
               for r in rhos]
        bd = P.Batch(l32, stream=stream.cuda_stream)
        bd.tune(20)
        bd.step(64)
        kd = 1024
        e0.record(stream)
        bd.step(kd)
        e1.record(stream)
        torch.cuda.synchronize()
        msd = e0.elapsed_time(e1)
        okd = bd.sync() == P.LB_OK
        bd.close()
        for l in l32:
            l.close()
        l64 = [P.Lattice("D2Q9", (256, 256), r, L.E8_2D.bases, L.E8_2D.weights, precision="fp64",
                         tau=1.0, G=-3.0, convention="literal", stream=stream.cuda_stream)
               for r in rhos]
        for l in l64:
            l.step(2)
        k64d = 40
        e0.record(stream)
        for l in l64:
            l.step(k64d)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64d = e0.elapsed_time(e1)
        ok64 = all(l.sync() == P.LB_OK for l in l64)
        for l in l64:
            l.close()
        drops = {"fp32_batch": {"value": nd * kd / (msd * 1e3), "unit": "MLUPS", "steps": kd,
                                "ms_per_step": msd / kd, "stable": okd},
                 "fp64": {"value": nd * k64d / (ms64d * 1e3), "unit": "MLUPS", "steps": k64d,
                          "ms_per_step": ms64d / k64d, "stable": ok64},
                 "lattices": 20, "nodes": nd}

    # the many-instance 2D workload: 64 seeded D2Q9 droplets/bubbles of
    # uneven size (sides 64..512, mixed E4/E6/E8 stencils), one launch per
    # step for all of them, replayed from a CUDA graph; tile shape tuned.
    # Coupling G' = -3 from its coexistence densities (0.456, 2.25): every
    # instance is a stable two-phase system (droplets of 1.9 in gas of 0.15
    # at G' = -5/3 rarefy the gas to n < 0 within 100 steps, in the oracle too)
    batched = None
    if not args.no_batch:
        inst = L.batched_instances(64)
        lats = []
        for d in inst:
            s = d["side"]
            rin, rout = (0.456, 2.25) if d["bubble"] else (2.25, 0.456)
            lats.append(P.Lattice("D2Q9", (s, s), L.tanh_sphere(s, s, 1, d["radius"], rin, rout, 2.0),
                                  d["stencil"].bases, d["stencil"].weights, precision="fp32",
                                  tau=1.0, G=-3.0, convention="literal", stream=stream.cuda_stream))
        nb = sum(d["side"] ** 2 for d in inst)
        bt = P.Batch(lats, stream=stream.cuda_stream)
        best, tms = bt.tune(20)
        bt.step(64)
        kb = 2048
        e0.record(stream)
        bt.step(kb)
        e1.record(stream)
        torch.cuda.synchronize()
        msb = e0.elapsed_time(e1)
        okb = bt.sync() == P.LB_OK
        vb = nb * kb / (msb * 1e3)
        shapes = P.lb_batch_tile_shapes()
        batched = {"value": vb, "unit": "MLUPS", "instances": len(inst), "nodes": nb,
                   "coupling": "G' = -3 (literal), coexistence densities 0.456 / 2.25",
                   "steps": kb, "ms_per_step": msb / kb, "launches_per_step": 1,
                   "graph_steps": 64, "tile": list(shapes[best]),
                   "tune_ms": {f"{a}x{c}": float(t) for (a, c), t in zip(shapes, tms)},
                   "alg_bytes_per_node": 2 * 9 * 4,
                   "hbm_frac": 2 * 9 * 4 * vb * 1e6 / 1e9 / peak, "stable": okb}
        bt.close()
        for l in lats:
            l.close()

    # adjoint tuning as configured: D2Q9 E8, a flat 512 x 4 slab (binary32
    # forward, 4,000 steps, checkpoint every 100, binary64 adjoint); Newton
    # steps on the five group weights and G take (sigma_0, delta) to 1.2 x and
    # 0.5 x their untuned values at fixed interface width and density ratio;
    # the companion 512^2 droplet (R = 64) before and after, measured after
    # 40,000 steps (at 4,000 its Laplace pressure is a third of equilibrium)
    adjoint = None
    if not args.no_adjoint:
        import paper_2505_23647_gb300.adjoint as PA
        ng3, nl3 = COEX_GP3
        na, ka, ca = 512, 4000, 100

        def c5_slab(W, G_):
            rho_s = L.tanh_slab(na, 4, 1, na // 4, 3 * na // 4, ng3, nl3, 2.0)
            return P.Lattice("D2Q9", (na, 4), rho_s, L.E8_2D.bases, W, precision="fp32",
                             tau=1.0, G=G_, convention="literal", stream=stream.cuda_stream)

        def c5_drop(W, G_):
            rho_d = L.tanh_sphere(na, na, 1, 64.0, nl3, ng3, 2.0, center=(na / 2.0, na / 2.0, 0.0))
            latd = P.Lattice("D2Q9", (na, na), rho_d, L.E8_2D.bases, W, precision="fp32",
                             tau=1.0, G=G_, convention="literal", stream=stream.cuda_stream)
            latd.step(40000)
            okd = latd.sync() == P.LB_OK
            r = latd.curved_interface((na / 2.0, na / 2.0)) if okd else {"stable": False}
            latd.close()
            return r

        w0 = np.array([float(w) for w in L.E8_2D.weights])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v0, _, _ = PA.slab_observables(lambda: c5_slab(list(w0), -3.0), ka, na // 2, 0, nl3, ng3, ca)
        targets = v0 * np.array([1.2, 0.5, 1.0, 1.0])
        wt, Gt, vals, hist = PA.tune_slab(c5_slab, lambda k: [float(v) for v in k], w0, -3.0, targets,
                                          ka, na // 2, 0, nl3, ng3, ca, rtol=1e-3, max_iter=12)
        torch.cuda.synchronize()
        dta = reduce_max(dist, time.perf_counter() - t0, dev)
        sweeps = 4 * (len(hist) + 1)      # adjoint sweeps of ka steps (4 quantities per Jacobian)
        d0, d1 = c5_drop(list(w0), -3.0), c5_drop(list(wt), float(Gt))
        adjoint = {"value": sweeps * ka / dta, "unit": "adjoint steps/s (whole solve)",
                   "lattice": f"D2Q9 E8 {na}x4 slab, binary32 forward, binary64 adjoint",
                   "steps": ka, "checkpoint_every": ca, "newton_iterations": len(hist),
                   "seconds": dta, "untuned": {"sigma0": v0[0], "delta": v0[1], "width": v0[2],
                                               "ratio": v0[3]},
                   "targets": list(targets), "achieved": list(vals),
                   "max_rel_error": float(np.max(np.abs(vals / targets - 1.0))),
                   "weights": {"untuned": list(w0), "tuned": [float(v) for v in wt], "G": float(Gt)},
                   "droplet_512_R64_40000_steps": {"untuned": d0, "tuned": d1},
                   "accuracy": "gradients vs central differences and the binary64 oracle adjoint: "
                               "tests/test_gpu_adjoint.py; this solve: tests/test_gpu_c5.py"}

    c1 = c2 = None
    if not args.no_configs:
        c1 = c1_leg(P, L, stream)
        c2 = c2_leg(P, L, stream)

    cpu = None
    if rank == 0 and not args.no_cpu:
        sub, csteps = 64, 12
        v1, dt1 = oracle_mlups(sub, csteps)
        procs = os.cpu_count() or 1
        vall, dtall = oracle_mlups_allcore(sub, csteps, procs)
        cpu = {"value": vall, "unit": "MLUPS", "cores": procs, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"{csteps} steps of the FP64 C oracle on the {sub}^3 centred sub-box "
                         f"of the workload, one copy per core in {procs} processes "
                         f"({dtall:.1f} s); MLUPS = all updates / the slowest process's time",
               "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1, "seconds": dt1}}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "D3Q19", "stencil": "E8 (92 vectors)",
                       "nodes": N, "precision": "fp32 shifted (g = f - w rho0)",
                       "parallelism": f"replicas x{ws}",
                       "l2": "inputs larger than L2 (2 x 1.27 GB populations)"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": launches, "fp64": fp64, "literal_g": lit, "psi_eps": peps,
            "f2_forcing": f2, "wide_stencils": wide,
            "fused_kernel": fused,
            "batched_2d": batched, "adjoint": adjoint, "slab_fp64": slab,
            "droplets_2d": drops, "c1": c1, "c2": c2,
            "observables": {"call_ms": obs_ms, "call_in_steps": obs_ms / (ms_max / args.steps),
                            "mass": obs["mass"], "umax": obs["umax"],
                            "rho_min": obs["rho_min"], "rho_max": obs["rho_max"],
                            "stable": stable, "first_unstable_step": obs["error_step"]},
        }
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-literal", action="store_true")
    ap.add_argument("--no-psi-eps", action="store_true")
    ap.add_argument("--no-f2", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-droplets", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-wide", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the C1 / C2 runs as written (physics, ~1 min)")
    ap.add_argument("--zchunk", type=int, default=0,
                    help="z planes per CTA of the fused kernel (default: the library's)")
    ap.add_argument("--size", type=int, default=256,
                    help="cube edge (default 256, the workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global NX, NY, NZ, RADIUS, WORKLOAD
    if args.size != 256:
        NX = NY = NZ = args.size
        RADIUS = 40.0 * args.size / 256.0
        WORKLOAD = WORKLOAD.replace("256^3", f"{NX}^3 (profiling size)").replace(
            "R=40", f"R={RADIUS:g}")
    dist, rank, ws = _dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist, rank, ws)
        else:
            run_gb300(args, dist, rank, ws)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
