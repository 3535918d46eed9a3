#!/usr/bin/env python3
"""Throughput of the particle time step on one GB300 (or N independent replicas).

Workload: the wall-refined channel with 50,000 triangles and 500 particles per element (25M
particles, three velocity components, frequency and one scalar released from a line source at
y = 0.67; Re_tau = 180, dt = 1e-3), initialised on the device by lpdf_particles_init, with
synthetic node fields of the channel's structure held fixed (the gridpoint solves are not part
of the timed step). One step = lpdf_pdf_step: Eq. 4/5/9/2 for every particle, wrap and wall
reflection, exact point location, scalar sources, the re-bucketing of the ensemble by element
(a stable counting sort) and the moment sums at gridpoints.

Prints one JSON line. `--impl reference` times the FP64 CPU oracle instead (a bounded sample of
the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s (SDE+locate+stats) at 25M particles; % HBM roofline"
UNIT = "particle-updates/s"
# algorithmic bytes of one particle update (ns = 1): read x, y, u, v, w, omega, psi, elem, pid
# (36 B) and write x, y, u, v, w, omega, psi, elem (32 B)
BYTES_PER_UPDATE = 68
# kernels of one lpdf_pdf_step: element-field table, advance, histogram, 3 scan kernels, record
# scatter, record offsets, particle scatter, moments
LAUNCHES_PER_STEP = 10


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources of the advance kernel: a traffic figure taken on other sources is stale
KERNEL_SOURCES = ("lpdf_pipeline.cu", "lpdf_device.cuh", "lpdf_internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "advance_kernel_channel25M_traffic.txt")


def kernel_source_hash():
    """Hash of the advance kernel's code: its sources without comments and blank lines, so that
    an edit of a comment keeps a traffic figure while any change of code drops it."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1006_0549_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("\n".join(ln.strip() for ln in text.splitlines() if ln.strip()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(n_particles: int, variant: int):
    """DRAM bytes (read + write) of one advance-kernel launch of the given launch variant, from the
    committed summary of one-pass ncu captures of this workload (bytes per particle times the
    particles of the launch); None when the summary was taken on other kernel sources or lacks
    the variant."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    d = {}
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if ":" in line:
                k, v = line.split(":", 1)
                d[k.strip()] = v.strip()
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    key = f"variant {variant} bytes per particle"
    if key not in d:
        return None
    return float(d[key]) * n_particles


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        try:
            import torch
            uuid = str(torch.cuda.get_device_properties(gpu_index).uuid)
            self.gpu = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            pass
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else 0.0,
                                 parts[5], parts[6], parts[7], parts[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in load:
            for nm, v in zip(names, r[3:]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in load),
                "reasons": sorted(reasons), "samples": len(load)}


def replica_seed(rank: int) -> int:
    """Each rank runs an independent replica of the ensemble (replicas only: the path has no
    exchange between ensembles), drawn from its own seed."""
    return 1006054902 + 7919 * rank


def combine_ranks(dist, maxed, summed, device):
    """The job-wide figures of a replicated run: the maximum over ranks of the times (`maxed`)
    and the sum of the work (`summed`); no collective on the data path, only this one at the end."""
    if dist is None:
        return list(maxed), list(summed)
    import torch
    t = torch.tensor(list(maxed), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor(list(summed), dtype=torch.float64, device=device)
    dist.all_reduce(n)
    return [float(v) for v in t], [float(v) for v in n]


def build_workload(rank: int, ppe: int):
    import torch
    from paper_1006_0549_gb300 import lpdf, workloads as wl
    wk = wl.channel_25m(seed=replica_seed(rank))
    wk.n_per_elem = ppe
    mesh = lpdf.Mesh(wk.mesh)
    params = lpdf.params_for(wk)
    ctx = lpdf.Context(mesh, params, wk.n_particles)
    init = torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda()
    ctx.particles_init(wk.n_per_elem, init, m_erlang=4)
    fields = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    ctx.status()
    return wk, mesh, ctx, fields


def run_gpu(args, rank, world, dist):
    import torch
    from paper_1006_0549_gb300 import lpdf
    wk, mesh, ctx, fields = build_workload(rank, args.ppe)
    P = ctx.n
    stream = torch.cuda.current_stream()
    # launch configuration of the step's kernels, chosen by the library's autotuner on this
    # ensemble (every configuration gives bit-identical results)
    if args.tune == "auto":
        tune, tune_ms, step = ctx.autotune(fields, 0, steps_per_trial=4, rounds=3)
    else:
        tune, tune_ms, step = tuple(int(v) for v in args.tune.split(",")), [], 0
        ctx.set_tune(*tune)
    for _ in range(args.warmup):
        ctx.pdf_step(fields, step)
        step += 1
    torch.cuda.synchronize()
    ctx.status()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.timings()
    with ClockSampler(torch.cuda.current_device()) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(K):
            ev[k][0].record(stream)
            ctx.pdf_step(fields, step)
            ev[k][1].record(stream)
            step += 1
        t1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    kms, ksteps = ctx.timings()
    ctx.set_timing(False)
    kernel_ms = {"advance": kms[0] / ksteps, "rebucket": kms[1] / ksteps, "moments": kms[2] / ksteps}
    per = [a.elapsed_time(b) for a, b in ev]
    print("per-step ms:", " ".join(f"{x:.3f}" for x in per), file=sys.stderr)
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"step status {rc}: {status}")
    hops = status[3] / (P * K)
    # e2e: the same step through the C-ABI with host buffers: every step's node fields go up from
    # pinned host memory and its statistics come back and are read by the host. The copies run on
    # two copy streams with double buffers, so they and the host's read of step k's statistics
    # overlap step k + 1; events order each buffer's reuse.
    nq = 11 + 2 * wk.ns
    h_fields = torch.empty_like(fields, device="cpu").pin_memory()
    h_fields.copy_(fields.cpu())
    d_fields = [torch.empty_like(fields) for _ in range(2)]
    d_stats = [torch.empty((mesh.n_nodes, nq), dtype=torch.float64, device="cuda") for _ in range(2)]
    h_stats = [torch.empty((mesh.n_nodes, nq), dtype=torch.float64).pin_memory() for _ in range(2)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    main = torch.cuda.current_stream()
    stepped, fetched = [None, None], [None, None]
    Ke = max(3, min(K, 10))
    seen = 0.0
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(Ke):
        b = k % 2
        with torch.cuda.stream(up):
            if stepped[b] is not None:
                up.wait_event(stepped[b])              # step k - 2 has read d_fields[b]
            d_fields[b].copy_(h_fields, non_blocking=True)
            uploaded = up.record_event()
        main.wait_event(uploaded)
        if fetched[b] is not None:
            main.wait_event(fetched[b])                # step k - 2's statistics have left d_stats[b]
        ctx.pdf_step(d_fields[b], step)
        ctx.grid_statistics(d_stats[b], raw=False)
        stepped[b] = main.record_event()
        with torch.cuda.stream(down):
            down.wait_event(stepped[b])
            h_stats[b].copy_(d_stats[b], non_blocking=True)
            fetched[b] = down.record_event()
        if k >= 1:                                     # the host reads step k - 1's statistics
            fetched[1 - b].synchronize()
            seen += float(h_stats[1 - b][0, 0])
        step += 1
    fetched[(Ke - 1) % 2].synchronize()
    seen += float(h_stats[(Ke - 1) % 2][0, 0])
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - te) / Ke
    d_stats = d_stats[(Ke - 1) % 2]
    # the same step with compensated moment sums (lpdf_params.moment_sums = 1: within 1e-9 of the
    # FP64 sums instead of 48 eps32), beside the metric
    ctx.set_params(lpdf.params_for(wk, moment_sums=1))
    for _ in range(2):
        ctx.pdf_step(fields, step)
        step += 1
    torch.cuda.synchronize()
    ctx.set_timing(True)
    ctx.timings()
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(K):
        ctx.pdf_step(fields, step)
        step += 1
    c1.record(stream)
    torch.cuda.synchronize()
    ckms, cks = ctx.timings()
    ctx.set_timing(False)
    ctx.set_params(lpdf.params_for(wk))
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"step status {rc}: {status} (compensated moment sums)")
    comp_ms = c0.elapsed_time(c1) / K
    compensated = {"ms_per_step": comp_ms, "value": P / (comp_ms * 1e-3), "unit": UNIT,
                   "kernels_ms_per_step": {"advance": ckms[0] / cks, "rebucket": ckms[1] / cks,
                                           "moments": ckms[2] / cks},
                   "note": "the same workload with lpdf_params.moment_sums = 1: gridpoint sums in compensated "
                           "FP32 (double-float), within 1e-9 of sum |lambda q| of the FP64 oracle instead of "
                           "48 eps32"}
    # the gridpoint side (not part of the metric): node fields from the last statistics, elliptic
    # relaxation and mean-pressure CGs to a relative residual of 1e-6 (far below the statistical noise
    # of the moments); cold (from zero), then warm
    # (from the previous solution, on the statistics one step later, as in a time loop)
    gp = lpdf.params_for(wk, gmodel=0, pressure_solve=1, dpdx0=-1.0)
    out_fields = torch.empty_like(fields)
    mesh.elliptic_relax_solve(gp, d_stats, out_fields, 1e-6, 20000)     # tables built, warm caches
    torch.cuda.synchronize()
    tg = time.perf_counter()
    its_cold = mesh.elliptic_relax_solve(gp, d_stats, out_fields, 1e-6, 20000)
    torch.cuda.synchronize()
    cold_ms = 1e3 * (time.perf_counter() - tg)
    ctx.pdf_step(fields, step)
    ctx.grid_statistics(d_stats, raw=False)
    gp.cg_warm_start = 1
    torch.cuda.synchronize()
    tg = time.perf_counter()
    its_warm = mesh.elliptic_relax_solve(gp, d_stats, out_fields, 1e-6, 20000)
    torch.cuda.synchronize()
    warm_ms = 1e3 * (time.perf_counter() - tg)
    solve = {"cold_ms": cold_ms, "cold_cg_iterations": list(its_cold), "warm_ms": warm_ms,
             "warm_cg_iterations": list(its_warm), "nodes": mesh.n_nodes,
             "note": "lpdf_elliptic_relax_solve: recovery, FP64 elliptic-relaxation and pressure CGs, "
                     "host-timed (it synchronises); not included in the step"}
    return dict(P=P, total_ms=total_ms, per=per, kernel_ms=kernel_ms, clocks=clk.summary(), hops=hops, e2e_s=e2e_s,
                compensated=compensated,
                h2d=int(h_fields.numel() * 4), d2h=int(h_stats[0].numel() * 8), wk=wk, solve=solve,
                tune={"advance_variant": tune[0], "moments_variant": tune[1],
                      "trial_ms_per_step": [round(float(x), 4) for x in tune_ms]})


def run_cavity(steps: int, warmup: int, peak: float):
    """The lid-driven cavity (199,712 triangles, 100 particles per element, four scalars from point
    sources, lid velocity 1, nu = 1e-4): the same step on the second configuration, autotuned,
    with fixed synthetic node fields of the cavity's structure."""
    import torch
    from paper_1006_0549_gb300 import lpdf, workloads as wl
    wk = wl.cavity_20m()
    gm = lpdf.Mesh(wk.mesh)
    params = lpdf.params_for(wk)
    ctx = lpdf.Context(gm, params, wk.n_particles)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda(), m_erlang=4)
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    ctx.status()
    tune, tune_ms, step = ctx.autotune(F, 0, steps_per_trial=4, rounds=3)
    for _ in range(warmup):
        ctx.pdf_step(F, step)
        step += 1
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx.set_timing(True)
    ctx.timings()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        ctx.pdf_step(F, step)
        step += 1
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    kms, ks = ctx.timings()
    ctx.set_timing(False)
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"cavity step status {rc}: {status}")
    P = ctx.n
    # algorithmic bytes: read x, y, u, v, w, omega, psi[ns], elem, pid; write all but pid (92 B at ns = 4)
    bytes_per_update = (8 + wk.ns) * 4 + (7 + wk.ns) * 4
    adv = kms[0] / ks
    achieved = bytes_per_update * P / (adv * 1e-3) / 1e9
    return {"workload": f"{wk.name}: lid-driven cavity, {wk.mesh.n_tri} triangles, {wk.n_per_elem} particles "
                        f"per element, {wk.ns} scalars", "particles": int(P), "steps": steps,
            "ms_per_step": ms / steps, "value": P * steps / (ms * 1e-3), "unit": "particle-updates/s",
            "kernels_ms_per_step": {"advance": adv, "rebucket": kms[1] / ks, "moments": kms[2] / ks},
            "advance_roofline": {"bytes_per_update": bytes_per_update, "achieved_gbs": achieved, "frac": achieved / peak},
            "mean_walk_hops": float(status[3]) / (P * steps),
            "tune": {"advance_variant": tune[0], "moments_variant": tune[1]}}


def run_batched(steps: int, warmup: int):
    """64 independent channel ensembles of uneven size (meshes of 2k-40k triangles, 50-400
    particles per element, own seeds and source heights) in one multi-component mesh: autotuned
    launch configuration, steps replayed from CUDA graphs, node fields fixed."""
    import torch
    from paper_1006_0549_gb300 import lpdf, workloads as wl
    t = time.perf_counter()
    wk = wl.batched_channels()
    gm = lpdf.Mesh(wk.mesh)
    params = lpdf.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seeds[0], ns=wk.ns)
    n = wk.n_particles
    ctx = lpdf.Context(gm, params, n)
    ctx.set_components(list(zip(wk.seeds, wk.sources)))
    parts = wk.mesh.parts
    init = torch.from_numpy(wl.stack_node_arrays([wl.node_init_fields(m) for m in parts])).cuda()
    ctx.particles_init_multi(wk.n_per_elem, init)
    F = torch.from_numpy(wl.stack_node_arrays([wl.synthetic_node_fields(m, wk.ns, seed=5 + k)
                                               for k, m in enumerate(parts)])).cuda()
    ctx.status()
    setup_s = time.perf_counter() - t
    tune, tune_ms, step = ctx.autotune(F, 0, steps_per_trial=3, rounds=3)
    ctx.pdf_steps(F, step, warmup)
    step += warmup
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    ctx.pdf_steps(F, step, steps)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"batched step status {rc}: {status}")
    return {"workload": f"{wk.name}: {len(parts)} channel ensembles in one multi-component mesh",
            "triangles": int(wk.mesh.n_tri), "particles": int(n),
            "triangles_per_component": [int(m.n_tri) for m in (min(parts, key=lambda m: m.n_tri),
                                                               max(parts, key=lambda m: m.n_tri))],
            "particles_per_element": [int(min(wk.n_per_elem)), int(max(wk.n_per_elem))],
            "steps": steps, "ms_per_step": ms / steps, "value": n * steps / (ms * 1e-3),
            "unit": "particle-updates/s", "graph": "pairs of steps replayed from one CUDA graph",
            "tune": {"advance_variant": tune[0], "moments_variant": tune[1],
                     "trial_ms_per_step": [round(float(x), 3) for x in tune_ms]},
            "setup_s": setup_s}


def aux_section(fn, *args, **kwargs):
    """fn(*args) for a report beside the metric; a library status error (LpdfError, or the
    RuntimeError of a bad step status) becomes {"error": message}. Anything else is raised."""
    from paper_1006_0549_gb300 import lpdf
    try:
        return fn(*args, **kwargs)
    except (lpdf.LpdfError, RuntimeError) as e:
        print(f"{getattr(fn, '__name__', 'section')}: {e}", file=sys.stderr)
        return {"error": str(e)}


def _timed(ctx, F, step: int, steps: int, warmup: int, per_step=None):
    """`warmup` then `steps` steps of ctx (with `per_step(step)` after each, inside the timed
    region); returns (ms, per-kernel ms per step, status, next step)."""
    import torch
    from paper_1006_0549_gb300 import lpdf
    for _ in range(warmup):
        ctx.pdf_step(F, step)
        if per_step:
            per_step(step)
        step += 1
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ctx.set_timing(True)
    ctx.timings()
    ctx.status()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        ctx.pdf_step(F, step)
        if per_step:
            per_step(step)
        step += 1
    t1.record(stream)
    torch.cuda.synchronize()
    kms, ks = ctx.timings()
    ctx.set_timing(False)
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"step status {rc}: {status}")
    return t0.elapsed_time(t1), {"advance": kms[0] / ks, "rebucket": kms[1] / ks, "moments": kms[2] / ks}, status, step


def _line(name, P, steps, ms, kms, status, ns, peak):
    bytes_per_update = (8 + ns) * 4 + (7 + ns) * 4
    achieved = bytes_per_update * P / (kms["advance"] * 1e-3) / 1e9
    return {"workload": name, "particles": int(P), "steps": steps, "ms_per_step": ms / steps,
            "value": P * steps / (ms * 1e-3), "unit": "particle-updates/s", "kernels_ms_per_step": kms,
            "advance_roofline": {"bytes_per_update": bytes_per_update, "achieved_gbs": achieved,
                                 "frac": achieved / peak},
            "mean_walk_hops": float(status[3]) / (P * steps)}


def run_mixing(steps: int, warmup: int, peak: float):
    """Eq. 9 with IECM and a reactive source on the 25M channel: three scalars (two released from
    line sources, psi_0 + psi_1 -> psi_2 at rate 4), and every step the loop of the method's
    mixing: the step (which also sums the scalar fluxes at the gridpoints), the statistics, the
    flux covariances and the conditional-mean slopes for the next step."""
    import torch
    from paper_1006_0549_gb300 import lpdf, workloads as wl
    wk = wl.channel_25m()
    wk.ns = 3
    wk.sources = [(0.25, 0.67, 0.02, 0), (0.25, 1.33, 0.02, 1)]
    gm = lpdf.Mesh(wk.mesh)
    params = lpdf.params_for(wk, mixing=1, react_k=4.0, react_a=0, react_b=1, react_p=2)
    ctx = lpdf.Context(gm, params, wk.n_particles)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda(), m_erlang=4)
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    N = wk.mesh.n_nodes
    S = torch.empty((N, 11 + 2 * wk.ns), dtype=torch.float64, device="cuda")
    Fx = torch.empty((N, 3 * wk.ns), dtype=torch.float64, device="cuda")
    beta = torch.zeros((N, 3 * wk.ns), dtype=torch.float32, device="cuda")
    ctx.set_iecm(beta)
    ctx.status()
    tune, _, step = ctx.autotune(F, 0, steps_per_trial=3, rounds=3)

    def slopes(_):
        ctx.grid_statistics(S, raw=False)
        ctx.grid_flux_statistics(Fx, raw=False)
        gm.iecm_coefficients(wk.ns, S, Fx, beta)

    ms, kms, status, _ = _timed(ctx, F, step, steps, warmup, slopes)
    out = _line(f"channel-50k-25M with IECM and a reaction: {wk.ns} scalars, conditional-mean slopes from "
                "the gridpoint fluxes every step", ctx.n, steps, ms, kms, status, wk.ns, peak)
    out["tune"] = {"advance_variant": tune[0], "moments_variant": tune[1]}
    return out


def run_walls(steps: int, warmup: int, peak: float):
    """Walls of any shape: the channel with a smooth bump on its bottom wall (250 x 100 cells,
    50,000 triangles, 500 particles per element, one scalar): particles that cross the curved
    wall are mirrored across the wall edge inside the walk."""
    import torch
    from paper_1006_0549_gb300 import lpdf, workloads as wl
    wk = wl.channel_25m()
    wk.mesh = wl.bump_channel_mesh(250, 100, 1006054905)
    gm = lpdf.Mesh(wk.mesh)
    ctx = lpdf.Context(gm, lpdf.params_for(wk), wk.n_particles)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda(), m_erlang=4)
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    ctx.status()
    tune, _, step = ctx.autotune(F, 0, steps_per_trial=3, rounds=3)
    ms, kms, status, _ = _timed(ctx, F, step, steps, warmup)
    out = _line("bump-channel-50k-25M: the channel with a curved bottom wall (edge walls mirrored in the walk)",
                ctx.n, steps, ms, kms, status, wk.ns, peak)
    out["tune"] = {"advance_variant": tune[0], "moments_variant": tune[1]}
    return out


def run_surrogate(wk, train_steps: int, run_steps: int, check_every: int, threshold: float, pressure_solve: int = 0,
                  dpdx0: float = -1.0, tol: float = 1e-8, maxit: int = 20000):
    """The learned surrogate of the gridpoint solve beside the plain solve, in the coupled time loop
    of the same workload: train on the fields of `train_steps` plain steps (on the GPU, with the
    library's forward and backward kernels), then continue from one state for `run_steps` steps with
    the plain solve, with the plain solve under another random seed (the ensemble's statistical
    spread) and with the surrogate; report the solve times and the differences in the Reynolds
    stresses and the scalar variance."""
    import torch
    from paper_1006_0549_gb300 import lpdf, timeloop as tl
    params = lpdf.params_for(wk, gmodel=0, pressure_solve=pressure_solve, dpdx0=dpdx0)
    loop = tl.TimeLoop(wk, params, tol=tol, maxit=maxit)
    t = time.perf_counter()
    feat, tgt = tl.collect_training_data(loop, train_steps)
    torch.cuda.synchronize()
    collect_s = time.perf_counter() - t
    t = time.perf_counter()
    net, losses = tl.train_surrogate(feat, tgt)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    net.set_policy(check_every, threshold)
    snap = loop.snapshot()

    def run_plain(p):
        loop.restore(snap, p)
        times = []
        for _ in range(run_steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            loop.solve_plain()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            loop.advance()
        loop.ctx.status()
        return loop.S.cpu().numpy(), float(np.median(times))

    def run_net(retrain_steps):
        loop.restore(snap, params)
        net.set_params(p0, n0)
        net.set_policy(check_every, threshold)
        r = tl.run_surrogate(loop, net, run_steps, feat, tgt, retrain_steps=retrain_steps)
        loop.ctx.status()
        t = [ms for ms, plain in r["times"] if not plain]
        return loop.S.cpu().numpy(), (float(np.median(t)) if t else None), r

    p0, n0 = net.get_params()
    plain, t_plain = run_plain(params)
    other = lpdf.params_for(wk, gmodel=0, pressure_solve=pressure_solve, dpdx0=dpdx0)
    other.seed = params.seed + 12345
    spread, _ = run_plain(other)
    surr, t_surr, r_fixed = run_net(0)
    surr_rt, t_surr_rt, r_rt = run_net(400)
    errs, used = r_fixed["check_errors"], r_fixed["network_used_on"]
    R, PHI = [4, 5, 6, 7, 8, 9], [11 + wk.ns + a for a in range(wk.ns)]
    solve = "elliptic relaxation and mean-pressure CGs" if pressure_solve else \
        "elliptic relaxation, fixed mean pressure gradient"
    return {"workload": f"{wk.name}, coupled loop ({solve})",
            "train_steps": train_steps, "train_rows": int(feat.shape[0]), "adam_steps": int(len(losses)),
            "final_loss": float(np.mean(losses[-200:])), "collect_s": collect_s, "train_s": train_s,
            "run_steps": run_steps, "check_every": check_every, "threshold": threshold,
            "check_errors": errs, "network_used_on": used,
            "plain_solve_ms": t_plain, "surrogate_solve_ms": t_surr,
            "speedup": (t_plain / t_surr) if t_surr else None,
            "reynolds_stress_rel_diff": {"surrogate_vs_plain": tl.relative_difference(surr, plain, R),
                                         "other_seed_vs_plain": tl.relative_difference(spread, plain, R)},
            "scalar_variance_rel_diff": {"surrogate_vs_plain": tl.relative_difference(surr, plain, PHI),
                                         "other_seed_vs_plain": tl.relative_difference(spread, plain, PHI)},
            "with_retraining": {"adam_steps_per_failed_check": 400, "retrains": r_rt["retrains"],
                                "check_errors": r_rt["check_errors"], "network_used_on": r_rt["network_used_on"],
                                "surrogate_solve_ms": t_surr_rt,
                                "reynolds_stress_rel_diff": tl.relative_difference(surr_rt, plain, R),
                                "scalar_variance_rel_diff": tl.relative_difference(surr_rt, plain, PHI)},
            "note": "errors: Frobenius norms over all nodes after run_steps; solve times: CUDA events, median "
                    "over the calls that ran the plain solve alone / the network alone"}


C1_RECORD = (1, 10, 50, 200)
C1_GROUPS = {"U_i": [1, 2, 3], "u_i u_j": [4, 5, 6, 7, 8, 9], "omega": [10], "phi": [11], "phi'^2": [12]}
C1_SOLVE = dict(gmodel=0, pressure_solve=1, dpdx0=-1.0)


def _dev_state(st):
    import torch
    d = {k: torch.from_numpy(np.ascontiguousarray(getattr(st, k))).cuda() for k in ("x", "y", "u", "v", "w", "omega")}
    d["psi"] = torch.from_numpy(np.ascontiguousarray(st.psi)).cuda()
    d["elem"] = torch.from_numpy(np.ascontiguousarray(st.elem, dtype=np.int32)).cuda()
    d["pid"] = torch.from_numpy(np.ascontiguousarray(st.pid).view(np.int32)).cuda()
    return d


def c1_inputs():
    """C1: the 1,000-triangle channel, 50 particles per element (50,000), one scalar, its seeded
    start state and first node fields, and the plain gridpoint solve (elliptic relaxation and
    mean-pressure projection)."""
    from paper_1006_0549_gb300 import workloads as wl
    wk = wl.channel_small()
    st0 = wl.synthetic_state(wk.mesh, wk.n_per_elem, wk.ns, seed=1006054901)
    F0 = wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)
    return wk, st0, F0


def run_c1(steps: int = 200):
    """C1 on the GPU: the coupled loop (step, statistics, gridpoint solve) for `steps` steps from
    the seeded state, and the same loop under another seed (the ensemble's statistical spread);
    device times of the step with its statistics and of the solve."""
    import torch
    from paper_1006_0549_gb300 import lpdf, timeloop as tl
    wk, st0, F0 = c1_inputs()
    params = lpdf.params_for(wk, **C1_SOLVE)
    g, timing, (rc, status) = tl.run_coupled(wk, params, _dev_state(st0), torch.from_numpy(F0).cuda(), steps,
                                             C1_RECORD, timing=True)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"C1 step status {rc}: {status}")
    other = lpdf.params_for(wk, **C1_SOLVE)
    other.seed = params.seed + 12345
    s, _, (rc, status) = tl.run_coupled(wk, other, _dev_state(st0), torch.from_numpy(F0).cuda(), steps, C1_RECORD)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"C1 step status {rc}: {status}")
    step_ms = float(np.median(timing["step_ms"]))
    return {"workload": f"{wk.name}: coupled loop, {steps} steps (step, statistics, elliptic relaxation and "
                        "mean-pressure solve)", "particles": int(st0.n), "steps": steps,
            "gpu_step_ms_median": step_ms, "gpu_step_value": st0.n / (step_ms * 1e-3),
            "gpu_solve_ms_median": float(np.median(timing["solve_ms"][:-1])), "unit": "particle-updates/s",
            "_stats": g, "_spread": s, "_params_seed": int(params.seed)}


def c1_against_oracle(c1):
    """The FP64 oracle's own coupled loop from the same state (CPU-baseline leg): its host time on
    one thread, and the relative error (Frobenius over all nodes) of every statistic of the GPU loop
    against it at the recorded steps, beside the GPU seed-to-seed spread."""
    import oracle
    from oracle import timeloop as otl
    from paper_1006_0549_gb300 import timeloop as tl
    wk, st0, F0 = c1_inputs()
    op = oracle.make_params(nu=wk.nu, dt=wk.dt, seed=c1["_params_seed"], ns=wk.ns, sources=wk.sources,
                            lid_u=wk.lid_u)
    times = {}
    o, _, lost = otl.run_coupled(wk.mesh, op, st0, F0, c1["steps"], C1_RECORD, solve=dict(nu=wk.nu, **C1_SOLVE),
                                 timings=times)
    g, s = c1.pop("_stats"), c1.pop("_spread")
    c1.pop("_params_seed")
    table = {str(n): {k: {"gpu_vs_oracle": tl.relative_difference(g[n], o[n], cols),
                          "seed_spread": tl.relative_difference(s[n], g[n], cols)}
                      for k, cols in C1_GROUPS.items()} for n in C1_RECORD}
    c1.update({"oracle_lost": int(lost), "oracle_step_s": times["step_s"], "oracle_solve_s": times["solve_s"],
               "oracle_step_value_1core": st0.n * c1["steps"] / times["step_s"], "relative_error": table,
               "note": "relative error = Frobenius norm over all nodes of (GPU - oracle) / oracle per statistic "
                       "group; seed spread = the GPU loop under another seed against the GPU loop"})
    return c1


def run_surrogate_cavity(train_steps: int = 100, train_every: int = 5, run_steps: int = 200, check_every: int = 50,
                         threshold: float = 0.02, tol: float = 1e-8, maxit: int = 20000):
    """The learned surrogate on the lid-driven cavity (199,712 triangles, ~20M particles, four
    scalars) with the node fields held fixed, as in the cavity's throughput configuration (the
    coupled loop does not run on this mesh). During the first `train_steps` steps, every
    `train_every`-th step's statistics go through the plain gridpoint solve and become training
    rows; the network is trained on the GPU; then every `check_every`-th step of the next
    `run_steps` the same statistics go to the plain solve and to the surrogate solve, whose
    checking call measures the error of G_ij and C_0 eps against the plain fields and falls back
    above `threshold`. Solve times: CUDA events; the network-only time is that of a
    non-checking call (it runs the plain solve instead when the last check failed)."""
    import torch
    from paper_1006_0549_gb300 import lpdf, timeloop as tl, workloads as wl
    wk = wl.cavity_20m()
    gm = lpdf.Mesh(wk.mesh)
    params = lpdf.params_for(wk, gmodel=0, pressure_solve=0)
    ctx = lpdf.Context(gm, params, wk.n_particles)
    ctx.particles_init(wk.n_per_elem, torch.from_numpy(wl.node_init_fields(wk.mesh)).cuda(), m_erlang=4)
    F = torch.from_numpy(wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)).cuda()
    ctx.set_tune(2, 1)
    N, nq, nfp = wk.mesh.n_nodes, 11 + 2 * wk.ns, wl.n_fields_padded(wk.ns)
    S = torch.empty((N, nq), dtype=torch.float64, device="cuda")
    out_p, out_s = (torch.empty((N, nfp), dtype=torch.float32, device="cuda") for _ in range(2))
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        a, b = ev(), ev()
        a.record()
        r = fn()
        b.record()
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    def rows():
        f = torch.empty((N, lpdf.MLP_IN), dtype=torch.float32, device="cuda")
        g = torch.empty((N, lpdf.MLP_OUT), dtype=torch.float32, device="cuda")
        gm.surrogate_features(params, S, f, out_p, g)
        # resolved nodes: the weight of at least 8 particles and a turbulent kinetic energy above
        # 1e-3 of the median (the central moments of a few particles are near zero)
        k = 0.5 * (S[:, 4] + S[:, 7] + S[:, 9])
        ok = S[:, 0] >= 8.0
        ok &= k >= 1e-3 * torch.median(k[ok])
        return f, g, ok

    t = time.perf_counter()
    feats, tgts, step, n_all = [], [], 0, 0
    for k in range(train_steps):
        ctx.pdf_step(F, step)
        step += 1
        if k % train_every == 0:
            ctx.grid_statistics(S, raw=False)
            gm.elliptic_relax_solve(params, S, out_p, tol, maxit)
            f, g, ok = rows()
            feats.append(f[ok])
            tgts.append(g[ok])
            n_all += N
    torch.cuda.synchronize()
    collect_s = time.perf_counter() - t
    t = time.perf_counter()
    net, losses = tl.train_surrogate(torch.cat(feats), torch.cat(tgts))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    y = torch.empty((N, lpdf.MLP_OUT), dtype=torch.float32, device="cuda")
    checks = []
    for k in range(run_steps):
        ctx.pdf_step(F, step)
        step += 1
        if (k + 1) % check_every:
            continue
        ctx.grid_statistics(S, raw=False)
        _, plain_ms = timed(lambda: gm.elliptic_relax_solve(params, S, out_p, tol, maxit))
        net.set_policy(1, threshold)
        (checked, err, used_plain, _), check_ms = timed(lambda: gm.surrogate_relax_solve(net, params, S, out_s, tol,
                                                                                         maxit))
        net.set_policy(0, threshold)
        (_, _, net_plain, _), net_ms = timed(lambda: gm.surrogate_relax_solve(net, params, S, out_s, tol, maxit))
        # the network's outputs against the plain solve's targets (G_ij / <omega>, C_0 eps / (k <omega>))
        # at the resolved nodes
        f, g, ok = rows()
        _, fwd_ms = timed(lambda: net.forward(f, y))
        d = (y - g)[ok][:, :6]
        res_err = float(torch.linalg.norm(d) / torch.linalg.norm(g[ok][:, :6]))
        checks.append({"step": step, "error": err, "fallback": bool(err > threshold), "plain_solve_ms": plain_ms,
                       "checking_call_ms": check_ms, "network_solve_ms": net_ms, "network_call_ran_plain": net_plain,
                       "resolved_nodes": int(ok.sum()), "resolved_target_error": res_err,
                       "network_forward_ms": fwd_ms})
    rc, status = ctx.status(raise_on_error=False)
    if rc != lpdf.LPDF_OK:
        raise RuntimeError(f"cavity surrogate step status {rc}: {status}")
    errs = [c["error"] for c in checks]
    return {"workload": f"{wk.name}: lid-driven cavity, {wk.mesh.n_tri} triangles, {ctx.n} particles, node fields "
                        "held fixed; the gridpoint solve fed the same statistics as the plain solve",
            "train_solves": len(feats), "train_rows": int(sum(f.shape[0] for f in feats)), "candidate_rows": n_all,
            "adam_steps": int(len(losses)), "final_loss": float(np.mean(losses[-200:])), "collect_s": collect_s,
            "train_s": train_s, "threshold": threshold, "check_every_steps": check_every, "checks": checks,
            "max_error": max(errs) if errs else None, "fallbacks": int(sum(c["fallback"] for c in checks)),
            "plain_solve_ms_median": float(np.median([c["plain_solve_ms"] for c in checks])),
            "network_solve_ms_median": float(np.median([c["network_solve_ms"] for c in checks])),
            "max_resolved_target_error": max(c["resolved_target_error"] for c in checks) if checks else None,
            "note": "error: |F_net - F_plain| / |F_plain| over the G_ij and C_0 eps columns of all nodes (the "
                    "surrogate's checking call); resolved_target_error: the network's outputs against the plain "
                    "solve's targets (G_ij / <omega>, C_0 eps / (k <omega>)) over the resolved nodes (the weight of at "
                    "least 8 particles, k above 1e-3 of the median), on which alone it is trained (at "
                    "under-resolved wall nodes k is near 0 "
                    "and the plain G_ij = (wp_ij - eps/2)/k reaches 1e10); solves: elliptic relaxation with a "
                    "fixed (zero) mean pressure gradient, CG tolerance 1e-8"}


def workload_config(wk, P: int, world: int, parallelism: str | None = None) -> dict:
    """The `config` of the JSON line: the workload by name and its sizes (both arms)."""
    name = "channel-50k-25M" if wk.n_per_elem == 500 else f"channel-50k-{P}"
    return {"workload": name, "particles_per_gpu": P, "triangles": wk.mesh.n_tri,
            "particles_per_element": wk.n_per_elem, "scalars": wk.ns,
            "l2": "inputs larger than L2 (state 0.9 GB per step)", "node_fields": "synthetic, held fixed",
            "parallelism": parallelism or (f"replicas x{world}" if world > 1 else "single GPU")}


def cpu_baseline_sample(wk, n_sample: int, first_elem: int = 0):
    """FP64 oracle (single-threaded C) on n_sample particles of the same workload (the particles of
    the elements from first_elem on, at the workload's particles per element): one step plus the
    gridpoint moments."""
    import oracle
    from paper_1006_0549_gb300 import workloads as wl
    om = oracle.OracleMesh(wk.mesh)
    p = oracle.make_params(nu=wk.nu, dt=wk.dt, seed=wk.seed, ns=wk.ns, sources=wk.sources, lid_u=wk.lid_u)
    n_el = max(1, n_sample // wk.n_per_elem)
    e0 = min(first_elem, wk.mesh.n_tri - n_el)
    sub = wl.Mesh(wk.mesh.node_xy, wk.mesh.tri[e0:e0 + n_el], wk.mesh.edge_tag[e0:e0 + n_el], wk.mesh.period_x,
                  wk.mesh.box, wk.mesh.kind, wk.mesh.nx, wk.mesh.ny)
    st = wl.synthetic_state(sub, wk.n_per_elem, wk.ns, seed=3)
    st.elem = (st.elem + e0).astype(np.int32)
    F = wl.synthetic_node_fields(wk.mesh, wk.ns, seed=5)
    t = time.perf_counter()
    res, elem, aux, lost = oracle.pdf_step(om, p, F, st, 0)
    S, _ = oracle.moments(om, wk.ns, res["x"], res["y"], res["u"], res["v"], res["w"], res["omega"], res["psi"],
                          elem, with_abs=False)
    dt = time.perf_counter() - t
    return st.n, dt


def _cpu_worker(args):
    """One host core's share of the parallel oracle baseline (a process of its own)."""
    sys.path.insert(0, ROOT)
    from paper_1006_0549_gb300 import workloads as wl
    n_sample, first_elem = args
    wk = wl.channel_25m()
    return cpu_baseline_sample(wk, n_sample, first_elem)


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
                if line.lower().startswith("cpu part"):
                    part = line.split(":", 1)[1].strip()
                    return {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1"}.get(part, "Arm part " + part)
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline_parallel(n_per_core: int, cores: int):
    """The oracle on every host core at once: `cores` processes (started with spawn), each on its
    own elements of the 25M channel; particles per second = all particles / the slowest process."""
    import multiprocessing as mpr
    per_elem = 500
    chunks = [(n_per_core, k * (n_per_core // per_elem)) for k in range(cores)]
    with mpr.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_cpu_worker, chunks)
    n = sum(r[0] for r in res)
    return n, max(r[1] for r in res)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=4_000_000)
    ap.add_argument("--surrogate-train-steps", type=int, default=100,
                    help="plain steps whose fields train the surrogate (0: no surrogate report)")
    ap.add_argument("--surrogate-run-steps", type=int, default=40)
    ap.add_argument("--batched", type=int, default=1, help="1: also report the 64-ensemble batched step")
    ap.add_argument("--c1", type=int, default=1,
                    help="1: also report the 200-step coupled loop on the small channel against the oracle's")
    ap.add_argument("--cavity", type=int, default=1, help="1: also report the 20M-particle cavity step")
    ap.add_argument("--mixing", type=int, default=1, help="1: also report the step with IECM and a reaction")
    ap.add_argument("--walls", type=int, default=1, help="1: also report the channel with a curved wall")
    ap.add_argument("--surrogate-cavity", type=int, default=200,
                    help="steps of the cavity surrogate report after its 100 training steps, checked every 50 "
                         "(0: none)")
    ap.add_argument("--tune", default="auto",
                    help="launch configuration of the step: 'auto' (the library's autotuner) or 'adv,mom'")
    ap.add_argument("--ppe", type=int, default=500,
                    help="particles per element (500 = the 25M-particle workload; smaller only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        if rank != 0:
            return
        from paper_1006_0549_gb300 import workloads as wl
        wk = wl.channel_25m()
        n_s = 200_000
        times = []
        for i in range(args.warmup + args.steps):
            n, dt = cpu_baseline_sample(wk, n_s)
            if i >= args.warmup:
                times.append(dt)
        v = n * len(times) / sum(times)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": workload_config(wk, wk.n_particles, 1, "FP64 oracle, one host thread, on a bounded sample"),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"{n} particles of the channel workload per step (one FP64 step + moments)"},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist = tdist
    from paper_1006_0549_gb300 import _build
    if rank == 0:
        _build.build()
    if dist is not None:
        dist.barrier()
    r = run_gpu(args, rank, world, dist)
    total_ms = r["total_ms"]
    P = r["P"]
    (total_ms, e2e_s), (P_all,) = combine_ranks(dist, [total_ms, r["e2e_s"]], [float(P)], "cuda")
    if rank != 0:
        dist.destroy_process_group()
        return
    K = args.steps
    ms_step = total_ms / K
    value = P_all * K / (total_ms * 1e-3)
    kms = r["kernel_ms"]
    peak, peak_kind = measured_peaks()
    # the advance kernel reads and writes the whole state: the step's algorithmic bytes
    achieved = BYTES_PER_UPDATE * P / (kms["advance"] * 1e-3) / 1e9
    step_gbs = BYTES_PER_UPDATE * P / (ms_step * 1e-3) / 1e9
    traffic = ncu_traffic(P, r["tune"]["advance_variant"])
    # the other configurations are reports beside the metric: an error in one of them (a status
    # the library returns, e.g. a lost particle) is recorded in its place, not raised
    c1 = aux_section(run_c1) if args.c1 else None
    # CPU-baseline leg (the FP64 oracle on the host cores): the channel sample on one core and on
    # all cores, the cavity sample on one core, and the oracle's own C1 loop with the error of the
    # GPU loop's statistics against it
    cpu_n, cpu_dt = cpu_baseline_sample(r["wk"], args.cpu_sample)
    ncores = os.cpu_count() or 1
    par_n, par_dt = cpu_baseline_parallel(max(500, args.cpu_sample // ncores), ncores)
    from paper_1006_0549_gb300 import workloads as wl_
    cav_n, cav_dt = cpu_baseline_sample(wl_.cavity_20m(), 200_000)
    if c1 is not None and "error" not in c1:
        c1 = c1_against_oracle(c1)
    batched = aux_section(run_batched, args.steps, args.warmup) if args.batched else None
    cavity = aux_section(run_cavity, args.steps, args.warmup, peak) if args.cavity else None
    mixing = aux_section(run_mixing, args.steps, args.warmup, peak) if args.mixing else None
    walls = aux_section(run_walls, args.steps, args.warmup, peak) if args.walls else None
    surrogate = surrogate_cavity = None
    if args.surrogate_train_steps > 0:
        surrogate = aux_section(run_surrogate, r["wk"], args.surrogate_train_steps, args.surrogate_run_steps, 10,
                                0.02)
    if args.surrogate_cavity:
        surrogate_cavity = aux_section(run_surrogate_cavity, run_steps=args.surrogate_cavity)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_step, "ms_per_step_median": statistics.median(r["per"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(workload_config(r["wk"], P, world), mean_walk_hops=r["hops"]),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
                     "kernel": "advance_kernel", "bytes_per_update": BYTES_PER_UPDATE,
                     "kernel_ms": kms["advance"], "kernels_ms_per_step": kms,
                     "step_achieved_gbs": step_gbs, "step_frac": step_gbs / peak},
        "cpu_baseline": {"value": par_n / par_dt, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"{par_n} particles of the same workload ({ncores} processes on the host cores, "
                                   f"{cpu_model()}, each on its own elements), one FP64 step + gridpoint moments; "
                                   f"single core: {cpu_n / cpu_dt:.4g} particle-updates/s on {cpu_n} particles",
                         "single_core": cpu_n / cpu_dt,
                         "cavity_single_core": {"value": cav_n / cav_dt, "sample": f"{cav_n} particles of the "
                                                "cavity-200k-20M workload, one FP64 step + gridpoint moments"}},
        "clocks": r["clocks"],
        "e2e": {"value": P_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "note": "per step: node fields host->device from pinned memory, pdf_step, grid_statistics, "
                        "statistics device->host and read by the host; the copies run on two copy streams "
                        "(double-buffered) and the host reads step k's statistics while step k + 1 runs; the "
                        "particle state stays resident in HBM"},
        "gpu_launches": K * LAUNCHES_PER_STEP,
        "moment_sums_compensated": r["compensated"],
        "gridpoint_solve": r["solve"],
        "c1": c1,
        "surrogate": surrogate,
        "surrogate_cavity": surrogate_cavity,
        "batched": batched,
        "mixing": mixing,
        "walls": walls,
        "cavity": cavity,
        "tune": r["tune"],
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
