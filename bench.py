#!/usr/bin/env python
"""Throughput of the volume-potential hot path on one GB300 (or N replicas).

Workload (the configuration the headline metric is quoted on): graded star
domain r(t) = 1 + 0.3 cos 5t, 16,384 triangles, 19-node degree-9 rule
(311,296 nodes), targets = all nodes + 10,000 random interior points,
density = sum of 4 seeded Gaussians.  All inputs are synthetic and seeded.

One step = one pass of the whole hot path over that input, device-resident:
mesh upload (nodes and weights), near-field build (point location, lists,
near and self correction weights) and one potential evaluation (far sum +
corrections) in the requested precision.  value = targets evaluated per
second (one target-eval = one (target, density) output).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--impl vp|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "star5_16384tri_19pt_targets_nodes_plus_10k_gauss4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=["mixed", "fp64", "fmm"], default="mixed",
                    help="mixed: direct float-float far sum (default); fp64; fmm: far sum by the fast multipole method")
    ap.add_argument("--impl", choices=["vp", "reference"], default="vp")
    ap.add_argument("--ntri", type=int, default=16384)
    ap.add_argument("--extra", type=int, default=10000)
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--fp64-weights", action="store_true",
                    help="correction-weight node quadratures in FP64 (VP_NF_FP64_WEIGHTS) instead of float-float")
    ap.add_argument("--config", type=int, default=2, choices=[2, 3, 4, 5, 6, 7, 8],
                    help="2: the 16,384-triangle star (default); 3: 64 densities; 4: 200 uneven meshes in one "
                         "batched launch; 5: serving loop with Poisson arrivals; 6: annulus with curved boundary "
                         "elements; 7: interpolation on a staggered mesh; 8: far/near balance over the far rules and tolerances")
    ap.add_argument("--nmesh", type=int, default=200)
    ap.add_argument("--requests", type=int, default=10000, help="requests of the --config 5 trace")
    ap.add_argument("--direct-requests", type=int, default=120,
                    help="--config 5: requests of the trace served with the direct far sum")
    ap.add_argument("--tmax", type=int, default=64000, help="largest pool mesh (triangles) for --config 5")
    ap.add_argument("--slots", type=int, default=8)
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples (every 200 ms) during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(prefix="vpclk", suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ inputs
def make_inputs(ntri, m_extra):
    from paper_2205_04401_gb300 import inputs
    mesh, f, extra = inputs.config2(n_tri=ntri, m_extra=m_extra)
    return mesh, f, extra


def oracle_baseline(mesh, fun, extra, budget_s=12.0, seed=1):
    """Time the FP64 CPU oracle (as it stands) on a bounded sample of targets."""
    from oracle.oracle import Oracle
    o = Oracle("far19")
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    f = fun(s["yxy"])[None, :]
    M = len(s["txy"])
    rng = np.random.default_rng(seed)
    n = 32
    t0 = time.perf_counter()
    o.potential(s, f, targets=rng.choice(M, n, replace=False))
    dt = time.perf_counter() - t0
    n2 = int(max(32, min(M, n * budget_s / max(dt, 1e-3))))
    sample = np.sort(rng.choice(M, n2, replace=False))
    t0 = time.perf_counter()
    u, _ = o.potential(s, f, targets=sample)
    dt = time.perf_counter() - t0
    return dict(value=n2 / dt, seconds=dt, targets=n2, s=s, f=f, sample=sample, u=u)


# ------------------------------------------------------------ launches
def count_launches(fn):
    """Kernel launches of this library (its kernels are named k_*) while fn
    runs, from the profiler's CUDA activity records; None if the profiler
    cannot record device activity here."""
    import re

    import torch
    try:
        from torch.profiler import ProfilerActivity, profile
        pat = re.compile(r"(^|[\s:])k_[A-Za-z0-9_]+")
        # the first profiling session of a process can come back without
        # device records (the activity tracer starts up): a short one first
        with profile(activities=[ProfilerActivity.CUDA]):
            torch.zeros(1, device="cuda").add_(1.0)
            torch.cuda.synchronize()
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        n = 0
        for e in prof.events():
            if str(getattr(e, "device_type", "")).endswith("CUDA") and pat.search(e.name or ""):
                n += 1
        return n if n > 0 else None
    except Exception:
        return None


# ------------------------------------------------------------ multi-rank
def whole_job(t_local_ms, units_per_rank, world, device=None):
    """The slowest rank's timed total (max over ranks) and the whole-job
    throughput: every rank processed units_per_rank units of its own replica
    in that time.  Needs torch.distributed initialised when world > 1."""
    import torch
    import torch.distributed as dist
    tt = torch.tensor([float(t_local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t = float(tt.item())
    return t, world * units_per_rank / (t / 1e3)


# --------------------------------------------------------------- reference
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mesh, fun, extra = make_inputs(args.ntri, args.extra)
    vals = []
    for _ in range(args.warmup):
        oracle_baseline(mesh, fun, extra, budget_s=2.0)
    t_all = 0.0
    info = None
    for k in range(args.steps):
        info = oracle_baseline(mesh, fun, extra, budget_s=8.0, seed=10 + k)
        vals.append(info["value"])
        t_all += info["seconds"]
    v = float(np.mean(vals))
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "target_evals_per_s", "value": v, "unit": "target-evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "targets": int(len(info["s"]["txy"])), "densities": 1},
        "cpu_baseline": {"value": v, "unit": "target-evals/s", "cores": cores, "kind": "oracle",
                         "sample": f"{info['targets']} random targets of the workload per step (far sum over all "
                                   f"311,296 nodes, lists, near/self weights), OpenMP over targets"},
        "e2e": {"value": v, "unit": "target-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------ many densities
def run_many(args):
    """The star workload with 64 densities at once: 56 seeded Gaussian
    mixtures and the manufactured f = -2 k^2 sin(kx) cos(ky), k = 1..8.
    A step is one resident evaluation (far sum + corrections) of all 64;
    the error is stated per density against the GPU FP64 path and, on
    sampled targets, against the oracle."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    mesh, _, extra = make_inputs(args.ntri, args.extra)
    fs = inputs.config3_densities(mesh)
    ctx = vp.Context(0)
    dev = torch.device("cuda", 0)
    mh = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, mh, node_targets=True, txy=torch.from_numpy(extra).to(dev))
    y, _ = vp.mesh_nodes(mh)
    yn = y.cpu().numpy()
    f_np = np.ascontiguousarray(np.stack([fn(yn) for fn in fs]))
    f = torch.from_numpy(f_np).to(dev)
    d = f.shape[0]
    M = nf.M
    stream = torch.cuda.current_stream()
    u = torch.empty((d, M), dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 1)):
        vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED, out=u)
    vp.profile_enable(ctx, True)
    vp.profile_reset(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED, out=u)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = vp.profile_read(ctx)
    vp.profile_enable(ctx, False)
    ms = e0.elapsed_time(e1) / args.steps
    per_density = None
    ms64 = None
    if not args.no_fp64:
        # the FP64 path on 5 of the densities (all 64 take minutes)
        sub = [0, 20, 40, 56, 63]
        fsub = f[sub].contiguous()
        e0.record(stream)
        u64 = vp.potential_eval(ctx, nf, fsub, precision=vp.VP_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) * d / len(sub)
        per_density = {str(k): float(v) for k, v in
                       zip(sub, ((u[sub] - u64).abs().amax(1) / u64.abs().amax(1)).cpu().numpy())}
    # the tensor-core correction apply (digit split of C and f), 5, 4 and 3 digits
    tc = {}
    for levels in (5, 4, 3):
        t0 = time.perf_counter()
        vp.nf_prepare_tc(nf, levels)
        prep_s = time.perf_counter() - t0
        ut = torch.empty_like(u)
        vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED_TC, out=ut)
        vp.profile_enable(ctx, True)
        vp.profile_reset(ctx)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED_TC, out=ut)
        e1.record(stream)
        torch.cuda.synchronize()
        status = vp.device_status(ctx)
        p2 = vp.profile_read(ctx)
        vp.profile_enable(ctx, False)
        rec = {"levels": levels, "ms_per_step": e0.elapsed_time(e1) / args.steps, "device_status": status,
               "apply_tc_ms": round(p2["apply_tc"][1] / args.steps, 3) if p2.get("apply_tc", (0,))[0] else None,
               "prepare_s": prep_s, "plan": vp.nf_tc_info(nf)}
        if per_density is not None:
            rec["rel_err_per_density_vs_gpu_fp64"] = {
                str(k): float(v) for k, v in
                zip(sub, ((ut[sub] - u64).abs().amax(1) / u64.abs().amax(1)).cpu().numpy())}
        rec["rel_err_vs_mixed_fp64_apply_max"] = float(((ut - u).abs().amax(1) / u.abs().amax(1)).max())
        tc[str(levels)] = rec
        if levels == 5:
            u_tc5 = ut
    rel_or = None
    rel_or_tc = None
    if not args.no_oracle_check:
        from oracle.oracle import Oracle
        o = Oracle("far19")
        s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
        fo = np.stack([fn(s["yxy"]) for fn in fs])
        smp = np.sort(np.random.default_rng(3).choice(M, 48, replace=False))
        uo, _ = o.potential(s, fo, targets=smp)
        ug = u.cpu().numpy()[:, smp]
        rel_or = (np.abs(ug - uo).max(1) / np.abs(uo).max(1)).tolist()
        ug = u_tc5.cpu().numpy()[:, smp]
        rel_or_tc = (np.abs(ug - uo).max(1) / np.abs(uo).max(1)).tolist()
    line = {
        "metric": "target_evals_per_s", "value": d * M / (ms / 1e3), "unit": "target-evals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": "star5_16384tri_19pt_64densities", "targets": M, "nodes": nf.mesh.N, "densities": d,
                   "step": "resident potential_eval of 64 densities"},
        "pair_densities_per_s": d * M * nf.mesh.N / (ms / 1e3), "clocks": clk,
        "fp64_ms_extrapolated_to_64": ms64, "mixed_over_fp64": (ms64 / ms) if ms64 else None,
        "rel_err_per_density_vs_gpu_fp64": per_density, "rel_err_per_density_vs_oracle_sampled": rel_or,
        "tensor_core_apply": tc, "tc5_rel_err_per_density_vs_oracle_sampled": rel_or_tc,
        "stage_ms": {k: round(v[1] / args.steps, 3) for k, v in prof.items() if v[0]},
    }
    print(json.dumps(line))


# ------------------------------------------------------- batched workload
def run_batch(args):
    """200 seeded meshes (disks, annuli, 3-7-lobed stars, L-shapes; 500-20,000
    triangles log-uniform; 19-node rule; 1-8 densities; targets = nodes),
    evaluated by one graph-captured batch.  A step is one batch launch."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    t0 = time.perf_counter()
    meshes = inputs.batch_meshes(n_mesh=args.nmesh, relax_iters=2)
    t_mesh = time.perf_counter() - t0
    ctx = vp.Context(0)
    items, nfs = [], []
    t0 = time.perf_counter()
    build_ms = 0.0
    for m, d, seed in meshes:
        mh = vp.mesh_upload(ctx, m.vxy, m.tri, vp.VP_RULE_19_D9)
        nf = vp.nearfield_build(ctx, mh, node_targets=True)
        build_ms += vp.nf_stats(nf)["build_ms"]
        y, _ = vp.mesh_nodes(mh)
        yn = y.cpu().numpy()
        f = np.stack([inputs.gaussian_mix(m, seed + 31 * k)(yn) for k in range(d)])
        fd = torch.from_numpy(f).cuda()
        u = torch.empty((d, nf.M), dtype=torch.float64, device="cuda")
        items.append((nf, fd, u))
        nfs.append((mh, nf, m, f, seed))
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch = vp.Batch(ctx, items, precision=vp.VP_MIXED)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    evals = sum(nf.M * f.shape[0] for nf, f, _ in items)
    pairs = sum(nf.M * nf.mesh.N for nf, _, _ in items)
    pair_dens = sum(nf.M * nf.mesh.N * f.shape[0] for nf, f, _ in items)
    for _ in range(max(args.warmup, 1)):
        batch.launch()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    e0.record(stream)
    for _ in range(args.steps):
        batch.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # accuracy: the smallest items against the GPU FP64 path and the oracle
    order = sorted(range(len(items)), key=lambda i: items[i][0].M)
    rel64, relor = [], []
    from oracle.oracle import Oracle
    o = Oracle("far19")
    for i in order[:3]:
        nf, fd, u = items[i]
        u64 = vp.potential_eval(ctx, nf, fd, precision=vp.VP_FP64)
        rel64.append(float(((u - u64).abs().amax(1) / u64.abs().amax(1)).max()))
        mh, _, m, f, _ = nfs[i]
        s = o.setup(m.vxy, m.tri)
        fo = np.stack([inputs.gaussian_mix(m, nfs[i][4] + 31 * k)(s["yxy"]) for k in range(f.shape[0])])
        smp = np.random.default_rng(i).choice(nf.M, 64, replace=False)
        uo, _ = o.potential(s, fo, targets=smp)
        ug = u.cpu().numpy()[:, smp]
        relor.append(float((np.abs(ug - uo).max(1) / np.abs(uo).max(1)).max()))
    # the same batch with the far sums by the fast multipole method (one graph of per-item evaluations)
    u_direct = [u.clone() for _, _, u in items]
    t0 = time.perf_counter()
    batch_f = vp.Batch(ctx, items, precision=vp.VP_MIXED_FMM)
    torch.cuda.synchronize()
    t_plan_fmm = time.perf_counter() - t0
    for _ in range(max(args.warmup, 1)):
        batch_f.launch()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        batch_f.launch()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_fmm = e0.elapsed_time(e1) / args.steps
    rel_fmm = max(float(((u - ud).abs().amax(1) / ud.abs().amax(1)).max()) for (_, _, u), ud in zip(items, u_direct))
    batch_f.release()
    for (_, _, u), ud in zip(items, u_direct):
        u.copy_(ud)
    line = {
        "metric": "target_evals_per_s", "value": evals / (ms / 1e3), "unit": "target-evals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "fmm_batch": {"ms_per_step": ms_fmm, "target_evals_per_s": evals / (ms_fmm / 1e3), "plan_s": t_plan_fmm,
                      "rel_err_vs_direct_batch_max": rel_fmm},
        "config": {"workload": f"batch_{len(items)}_meshes_500-20000tri_19pt_d1-8", "targets": int(sum(nf.M for nf, _, _ in items)),
                   "target_evals_per_step": int(evals), "pairs_per_step": pairs, "pair_densities_per_step": pair_dens,
                   "step": "one graph-captured batch launch (resident near fields)"},
        "pair_densities_per_s": pair_dens / (ms / 1e3),
        "clocks": clk,
        "setup_s": {"meshes": t_mesh, "upload_and_build": t_build, "device_build_ms": build_ms, "plan_and_autotune": t_plan},
        "accuracy": {"rel_err_vs_gpu_fp64_smallest3": rel64, "rel_err_vs_oracle_smallest3_sampled": relor},
    }
    print(json.dumps(line))
    batch.release()


# ------------------------------------------------------------ serving loop
def run_serving(args):
    """The serving workload: a pool of 50 resident meshes (disks, lobed stars,
    L-shapes; triangle counts log-uniform on [1,000, 64,000]) plus 3 cold
    meshes (5% of the requests) that are uploaded and built on first use;
    10,000 requests with 1-16 densities each arrive as a seeded Poisson
    process (mean 2 ms) and are served by the library's continuous-batching
    loop (slots = concurrent streams, admission by HBM footprint).

    Passes over the same seeded trace: the far sum by the fast multipole
    method, saturated (every request as specified) and at 70% of the
    capacity it measured; the direct float-float far sum, saturated and at
    70% of its capacity, on the first requests of the trace (the offered
    load is far above the direct sum's capacity, so the whole trace would
    take hours); the served FP64 path against the mixed ones on the trace's
    requests to the smallest meshes."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    rng = np.random.default_rng(2205044015)
    t0 = time.perf_counter()
    pool = []
    for i in range(53):
        t = int(round(math.exp(rng.uniform(math.log(1000), math.log(args.tmax)))))
        kind = i % 3
        sd = 2205044015000 + i
        m = (inputs.disk_uniform_mesh(t, sd, 2) if kind == 0 else
             inputs.lobed_mesh(t, sd, 3 + i % 5, 0.1 + 0.05 * (i % 5), 2) if kind == 1 else inputs.lshape_mesh(t, sd, 2))
        pool.append(m)
    t_mesh = time.perf_counter() - t0
    ctx = vp.Context(0)
    resident, nodes = [], []
    t0 = time.perf_counter()
    for m in pool[:50]:
        mh = vp.mesh_upload(ctx, m.vxy, m.tri, vp.VP_RULE_19_D9)
        nf = vp.nearfield_build(ctx, mh, node_targets=True)
        y, _ = vp.mesh_nodes(mh)
        resident.append((mh, nf))
        nodes.append(y.cpu().numpy())
    for m in pool[50:]:                    # node coordinates of the cold meshes (densities are evaluated there)
        mh = vp.mesh_upload(ctx, m.vxy, m.tri, vp.VP_RULE_19_D9)
        y, _ = vp.mesh_nodes(mh)
        nodes.append(y.cpu().numpy())
        mh.release()
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    resident_bytes = int(sum(vp.nf_stats(nf)["bytes_device"] for _, nf in resident))
    tri_counts = [len(m.tri) for m in pool]

    # Host buffers per mesh: 16 densities [16][N] and an output [16][M]; a
    # request with d densities reads the first d rows and writes the first d
    # rows of its mesh's output (a bounded footprint for 10,000 requests).
    # Requests on one mesh write the same values for the same density (the
    # evaluation is deterministic; only the far sum's kernel can differ with d,
    # within rounding), so overlapping writes leave a valid result.
    dens, outs = [], []
    for k in range(53):
        y = nodes[k]
        cs = np.random.default_rng(2205044015 + 17 * k).uniform(-0.6, 0.6, (16, 2))
        f = vp.pinned_empty((16, len(y)))
        for j, c in enumerate(cs):
            f[j] = np.exp(-((y - c) ** 2).sum(1) / 0.1)
        dens.append(f)
        outs.append(vp.pinned_empty((16, len(y))))

    def trace(n, mean_s, seed):
        r = np.random.default_rng(seed)
        arr = np.cumsum(r.exponential(mean_s, n))
        keys = np.where(r.random(n) < 0.05, 50 + r.integers(0, 3, n), r.integers(0, 50, n))
        ds = r.integers(1, 17, n)
        return arr, keys, ds

    def serve(n, mean_s, precision, seed, check=0, only=None, cold=True):
        """Serve the first n requests of the seeded trace (those on the meshes
        in `only`, if given) at the trace's arrival times scaled to mean_s."""
        srv = vp.Server(ctx, slots=args.slots, hbm_budget_bytes=24 << 30, precision=precision)
        for k, (_, nf) in enumerate(resident):
            srv.register(k, nf)
        if cold:
            for k in range(50, 53):
                srv.register_cold(k, pool[k].vxy, pool[k].tri, vp.VP_RULE_19_D9)
        arr, keys, ds = trace(10000 if only is None else 200000, 0.002, seed)
        sel = np.arange(len(keys)) if only is None else np.flatnonzero(np.isin(keys, only))
        sel = sel[:n]
        arr = (arr[sel] - arr[sel[0]]) * (mean_s / 0.002 if only is None else 1.0)
        if only is not None:
            arr = np.arange(len(sel)) * mean_s
        keys, ds = keys[sel], ds[sel]
        reqs = []
        clocks = Clocks(0)
        start = time.perf_counter()
        for i in range(len(sel)):
            k, d = int(keys[i]), int(ds[i])
            delay = start + arr[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            reqs.append((k, d, srv.submit(k, dens[k][:d], outs[k][:d])))
        lat = [srv.wait(t, 7200.0)[1] for _, _, t in reqs]
        wall = time.perf_counter() - start
        clk = clocks.stop()
        st = srv.stats()
        srv.close()
        errs = []
        seen = set()
        for k, d, t in reqs:
            if len(errs) >= check:
                break
            if k >= 50 or k in seen or tri_counts[k] > 4000:     # FP64 references on the smaller meshes
                continue
            seen.add(k)
            f = torch.from_numpy(np.ascontiguousarray(dens[k][:d])).cuda()
            u = np.array(outs[k][:d])
            if precision == vp.VP_FP64:
                ref = vp.potential_eval(ctx, resident[k][1], f, precision=vp.VP_MIXED_FMM).cpu().numpy()
            else:
                ref = vp.potential_eval(ctx, resident[k][1], f[:1].contiguous(), precision=vp.VP_FP64).cpu().numpy()
                u = u[:1]
            errs.append(float((np.abs(u - ref).max(1) / np.abs(ref).max(1)).max()))
        evals = sum(d * len(nodes[k]) for k, d, _ in reqs)
        return dict(requests=len(reqs), mean_interarrival_ms=1e3 * mean_s, wall_s=wall, evals=int(evals),
                    evals_per_s=evals / wall, req_per_s=len(reqs) / wall, p50_ms=float(np.percentile(lat, 50)),
                    p99_ms=float(np.percentile(lat, 99)), p50_wait_ms=st["p50_wait_ms"],
                    max_concurrent=st["max_concurrent"], cold_builds=st["cold_builds"], failed=st["failed"],
                    peak_bytes=st["peak_bytes"], clocks=clk, max_rel_err=max(errs) if errs else None,
                    err_checked_meshes=len(errs))

    n = args.requests
    fmm_sat = serve(n, 0.002, vp.VP_MIXED_FMM, 11, check=8)
    fmm_light = serve(n, 1.0 / (0.7 * fmm_sat["req_per_s"]), vp.VP_MIXED_FMM, 11, check=4)
    nd = args.direct_requests
    dir_sat = serve(nd, 0.002, vp.VP_MIXED, 11, check=4)
    dir_light = serve(max(10, nd // 4), 1.0 / (0.7 * dir_sat["req_per_s"]), vp.VP_MIXED, 11, check=2)
    # FP64 against the mixed paths on the trace's requests to the three smallest resident meshes
    small = list(np.argsort(tri_counts[:50])[:3])
    f64 = serve(12, 0.002, vp.VP_FP64, 11, check=3, only=small, cold=False)
    mix_small = serve(12, 0.002, vp.VP_MIXED, 11, only=small, cold=False)
    fmm_small = serve(12, 0.002, vp.VP_MIXED_FMM, 11, only=small, cold=False)
    line = {
        "metric": "target_evals_per_s", "value": fmm_sat["evals_per_s"], "unit": "target-evals/s", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * fmm_sat["wall_s"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": f"serving_pool50+3cold_1000-{args.tmax}tri_d1-16_poisson2ms_{n}req",
                   "slots": args.slots, "hbm_budget_bytes": 24 << 30, "requests": n,
                   "value_from": "saturated pass, far sum by the fast multipole method",
                   "pool_triangles": {"min": int(min(tri_counts[:50])), "max": int(max(tri_counts[:50])),
                                      "sum": int(sum(tri_counts[:50])), "cold": tri_counts[50:]},
                   "resident_bytes": resident_bytes},
        "saturated_fmm": fmm_sat, "seventy_percent_load_fmm": fmm_light,
        "saturated_direct": dir_sat, "seventy_percent_load_direct": dir_light,
        "direct_passes": f"first {nd} (saturated) and {max(10, nd // 4)} (70% load) requests of the trace",
        "fp64_vs_mixed_small_meshes": {"meshes": [int(k) for k in small],
                                       "triangles": [int(tri_counts[k]) for k in small],
                                       "fp64": f64, "direct_mixed": mix_small, "fmm": fmm_small,
                                       "direct_mixed_over_fp64": mix_small["evals_per_s"] / f64["evals_per_s"],
                                       "fmm_over_fp64": fmm_small["evals_per_s"] / f64["evals_per_s"]},
        "setup_s": {"meshes": t_mesh, "upload_and_build": t_build},
    }
    print(json.dumps(line))


# ------------------------------------------------------ curved elements
def run_curved(args):
    """Annulus 0.45 < |x| < 1 with both circles represented exactly by curved
    boundary elements (blending map), args.ntri triangles, 19-node rule,
    targets = nodes + args.extra uniform points, f = 1.  A step is the config-2
    step on this mesh: curved mesh upload + near-field build + mixed
    evaluation.  With f = 1 the exact potential is known,
    u = (|x|^2 - 1)/4 - (r0^2/2) log|x|, and the error is stated against it;
    the same mesh with straight (chord) boundary elements is timed beside."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    r0 = 0.45
    circles = [(0.0, 0.0, 1.0), (0.0, 0.0, r0)]
    mesh = inputs.snap_to_circles(inputs.annulus_mesh(args.ntri, 2205044016, r0), circles)
    tri, cur = inputs.curved_boundary(mesh, circles)
    rng = np.random.default_rng(2205044016)
    rr = np.sqrt(rng.uniform(r0 ** 2, 1.0, args.extra))
    th = rng.random(args.extra) * 2 * np.pi
    extra = np.ascontiguousarray(np.stack([rr * np.cos(th), rr * np.sin(th)], 1))
    ctx = vp.Context(0)
    dev = torch.device("cuda", 0)
    extra_d = torch.from_numpy(extra).to(dev)
    N = mesh.nt * 19
    M = N + len(extra)
    f_d = torch.ones((1, N), dtype=torch.float64, device=dev)
    u_d = torch.empty((1, M), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(curved):
        mh = (vp.mesh_upload_curved(ctx, mesh.vxy, tri, cur, vp.VP_RULE_19_D9) if curved
              else vp.mesh_upload(ctx, mesh.vxy, tri, vp.VP_RULE_19_D9))
        nf = vp.nearfield_build(ctx, mh, node_targets=True, txy=extra_d)
        vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED, out=u_d)
        return mh, nf

    res = {}
    for curved in (True, False):
        for _ in range(max(args.warmup, 1)):
            mh, nf = step(curved)
            torch.cuda.synchronize()
            nf.release()
            mh.release()
        vp.profile_enable(ctx, True)
        vp.profile_reset(ctx)
        clocks = Clocks(0)
        t_all = 0.0
        for k in range(args.steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mh, nf = step(curved)
            e1.record(stream)
            torch.cuda.synchronize()
            t_all += e0.elapsed_time(e1)
            st = vp.nf_stats(nf)
            y, _ = vp.mesh_nodes(mh)
            if k < args.steps - 1:
                nf.release()
                mh.release()
        clk = clocks.stop()
        prof = vp.profile_read(ctx)
        vp.profile_enable(ctx, False)
        u = u_d.cpu().numpy()[0]
        txy = np.vstack([y.cpu().numpy(), extra])
        r = np.hypot(txy[:, 0], txy[:, 1])
        ex = (r ** 2 - 1) / 4 - 0.5 * r0 ** 2 * np.log(r)
        res[curved] = dict(ms=t_all / args.steps, clocks=clk, stats=st,
                           stage_ms={k2: round(v[1] / args.steps, 3) for k2, v in prof.items() if v[0]},
                           err=float(np.abs(u - ex).max() / np.abs(ex).max()), mh=mh, nf=nf)
        if not curved:
            nf.release()
            mh.release()
    c, sline = res[True], res[False]
    n_curved_pairs = None
    cpu = None
    if not args.no_oracle_check:
        from oracle.oracle import Oracle
        o = Oracle("far19")
        s = o.setup(mesh.vxy, tri, node_targets=True, extra=extra, curves=cur)
        smp = np.sort(np.random.default_rng(5).choice(M, 64, replace=False))
        t0 = time.perf_counter()
        f = np.ones((1, s["N"]))
        uo, info = o.potential(s, f, targets=smp)
        dt = time.perf_counter() - t0
        n2 = int(max(64, min(M, 64 * 10.0 / max(dt, 1e-3))))
        smp2 = np.sort(np.random.default_rng(6).choice(M, n2, replace=False))
        t0 = time.perf_counter()
        uo2, info2 = o.potential(s, f, targets=smp2)
        dt = time.perf_counter() - t0
        ug = u_d  # the last curved evaluation is overwritten by the straight run: evaluate again
        vp.potential_eval(ctx, c["nf"], f_d, precision=vp.VP_MIXED, out=u_d)
        ug = u_d.cpu().numpy()[0]
        c["err_vs_oracle_sampled"] = float(np.abs(ug[smp2] - uo2[0]).max() / np.abs(uo2[0]).max())
        n_curved_pairs = int((cur["cidx"][info2["ptri"]] >= 0).sum())
        cpu = {"value": n2 / dt, "unit": "target-evals/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n2} random targets of the curved annulus (far sum over all nodes, lists, near/self "
                         f"weights with curved elements), OpenMP over targets, {dt:.1f} s"}
    c["nf"].release()
    c["mh"].release()
    line = {
        "metric": "target_evals_per_s", "value": M / (c["ms"] / 1e3), "unit": "target-evals/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": c["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": f"annulus_curved_{mesh.nt}tri_19pt_targets_nodes_plus_{len(extra)}_f1",
                   "targets": M, "nodes": N, "curved_triangles": int((cur["cidx"] >= 0).sum()),
                   "step": "mesh_upload_curved+nearfield_build+potential_eval", "l2": "256 MiB flush between steps"},
        "clocks": c["clocks"],
        "rel_err_vs_exact": c["err"], "rel_err_vs_oracle_sampled": c.get("err_vs_oracle_sampled"),
        "curved_pairs_in_oracle_sample": n_curved_pairs,
        "nf_stats": {k: c["stats"][k] for k in ("n_pairs", "n_self", "n_near", "near_leaves", "self_panels",
                                                 "depth_capped", "build_ms")},
        "stage_ms": c["stage_ms"],
        "straight_chords": {"ms_per_step": sline["ms"], "rel_err_vs_exact": sline["err"],
                            "stage_ms": sline["stage_ms"]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    ctx.close()


# ------------------------------------------------ staggered interpolation
def run_interp(args):
    """Interpolation of the potential over a staggered mesh (Sections 3.5 and
    4.3) on the unit disk at the paper's finest mesh size: quadrature mesh of
    2,766 curved triangles (h0 = 0.05), 19-node rule; interpolation meshes of
    order N_s = 20 (231 nodes per element, 638,946 targets): the quadrature
    mesh itself, and a staggered mesh of the same size.  f = 1, so the exact
    potential (|x|^2 - 1)/4 is known.  A step is: near-field build for the
    interpolation nodes + mixed evaluation + expansion coefficients +
    interpolation at 10^6 random points (staggered mesh); value = interpolated
    point values per second.  The near corrections (c), sub-triangles (s_n)
    and self panels (s_l) per target of both meshes are reported (Tables
    near_corr and self_stag)."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    circ = [(0.0, 0.0, 1.0)]
    q = inputs.disk_mesh(n_b=126, n_i=1321)
    tq, cq = inputs.curved_boundary(q, circ)
    st = inputs.disk_mesh(n_b=126, n_i=1321, stagger=True)
    ts, cs = inputs.curved_boundary(st, circ)
    Ns = 20
    ctx = vp.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    mesh = vp.mesh_upload_curved(ctx, q.vxy, tq, cq, vp.VP_RULE_19_D9)
    f = torch.ones((1, mesh.N), dtype=torch.float64, device=dev)
    rng = np.random.default_rng(2205044017)
    mq = 1_000_000
    r = np.sqrt(rng.random(mq)) * (1 - 1e-12)
    th = rng.random(mq) * 2 * np.pi
    pts_np = np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th)], 1))
    pts = torch.from_numpy(pts_np).to(dev)
    ex = (np.sum(pts_np ** 2, 1) - 1) / 4
    res = {}
    for name, (vxy, tri, cur) in (("same", (q.vxy, tq, cq)), ("staggered", (st.vxy, ts, cs))):
        it = vp.Interp(ctx, vxy, tri, Ns, curves=cur)
        nodes = it.nodes()

        def step():
            nf = vp.nearfield_build(ctx, mesh, node_targets=False, txy=nodes)
            u = vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED)
            coef = it.coeffs(u)
            val, elem = it.eval(coef, pts)
            return nf, val, elem

        for _ in range(max(args.warmup, 1)):
            nf, _, _ = step()
            torch.cuda.synchronize()
            nf.release()
        clocks = Clocks(0)
        vp.profile_enable(ctx, True)
        vp.profile_reset(ctx)
        t_all = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for k in range(args.steps):
            e0.record(stream)
            nf, val, elem = step()
            e1.record(stream)
            torch.cuda.synchronize()
            t_all += e0.elapsed_time(e1)
            stt = vp.nf_stats(nf)
            if k < args.steps - 1:
                nf.release()
        clk = clocks.stop()
        prof = vp.profile_read(ctx)
        vp.profile_enable(ctx, False)
        # the interpolation kernels alone
        u = vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED)
        torch.cuda.synchronize()
        e0.record(stream)
        coef = it.coeffs(u)
        e1.record(stream)
        torch.cuda.synchronize()
        coef_ms = e0.elapsed_time(e1)
        e0.record(stream)
        val, elem = it.eval(coef, pts)
        e1.record(stream)
        torch.cuda.synchronize()
        eval_ms = e0.elapsed_time(e1)
        v = val.cpu().numpy()[0]
        ok = elem.cpu().numpy() >= 0
        M = it.n_nodes
        res[name] = dict(
            ms_per_step=t_all / args.steps, targets=M, clocks=clk,
            c_per_target=stt["n_near"] / M, s_n_per_target=stt["near_leaves"] / M,
            s_l_per_target=stt["self_panels"] / M, outside=stt["outside"], build_ms=stt["build_ms"],
            stage_ms={k2: round(v2[1] / args.steps, 3) for k2, v2 in prof.items() if v2[0]},
            coeffs_ms=coef_ms, interp_eval_ms=eval_ms, interp_points_per_s=mq / (eval_ms / 1e3),
            points_located=int(ok.sum()),
            rel_err_interp_vs_exact=float(np.abs(v[ok] - ex[ok]).max() / np.abs(ex).max()),
            rel_err_nodes_vs_exact=float(np.abs(u.cpu().numpy()[0] - (np.sum(nodes.cpu().numpy() ** 2, 1) - 1) / 4).max()
                                         / 0.25))
        nf.release()
        it.release()
    cpu = None
    if not args.no_oracle_check:
        from oracle.oracle import Oracle
        o = Oracle("far19")
        it = vp.Interp(ctx, st.vxy, ts, Ns, curves=cs)
        nodes = it.nodes().cpu().numpy()
        it.release()
        s = o.setup(q.vxy, tq, node_targets=False, extra=nodes, curves=cq)
        n2 = 2000
        smp = np.sort(np.random.default_rng(9).choice(len(nodes), n2, replace=False))
        t0 = time.perf_counter()
        o.potential(s, np.ones((1, s["N"])), targets=smp)
        dt = time.perf_counter() - t0
        cpu = {"value": n2 / dt, "unit": "target-evals/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n2} random interpolation nodes of the staggered mesh (far sum, lists, near/self weights "
                         f"with curved elements), OpenMP over targets, {dt:.1f} s"}
    stg, same = res["staggered"], res["same"]
    line = {
        "metric": "interpolated_points_per_s", "value": 1e6 / (stg["ms_per_step"] / 1e3), "unit": "points/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": stg["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": "disk_curved_2766tri_19pt_interp_Ns20_staggered_f1", "quadrature_nodes": mesh.N,
                   "interp_nodes": stg["targets"], "query_points": mq,
                   "step": "nearfield_build(interp nodes)+potential_eval+interp_coeffs+interp_eval(1e6 points)"},
        "target_evals_per_s_at_nodes": stg["targets"] / (stg["ms_per_step"] / 1e3),
        "staggered": stg, "same_mesh": same,
        "ratios_staggered_over_same": {"c": stg["c_per_target"] / same["c_per_target"],
                                       "s_n": stg["s_n_per_target"] / same["s_n_per_target"],
                                       "s_l": stg["s_l_per_target"] / same["s_l_per_target"],
                                       "step_time": stg["ms_per_step"] / same["ms_per_step"]},
        "cpu_baseline": cpu,
    }
    mesh.release()
    print(json.dumps(line))
    ctx.close()


# ------------------------------------------------------ far / near balance
def run_offload(args):
    """The offloading of Section 4.2 (Fig. offload): raising the order N_f of
    the far rule shrinks the near field (Eq. rho0) and moves work from the
    near-field corrections to the far sum.  The paper's setting: the unit disk
    (curved, h0 = 0.1: 721 triangles), its two-Gaussian density, targets = the
    interpolation nodes of a staggered mesh of order N_s = 12 or 20, eps =
    1e-10 or 1e-14; far rules: the built-in degree-8 (16 nodes) and degree-9
    (19 nodes) ones (C_N = 1), and the S3-symmetric rules (33-453 nodes) and
    the conical-product rules (49-676 nodes) of degree 12, 20, 25, 30, 40, 50
    with C_N of Table "C_N values".  Per point: near
    corrections c, sub-triangles s_n and panels s_l per target, the near-field
    build (T_N with the apply), the far sum T_F by the FMM and directly, and
    the error of the FMM result for f = 1 against (|x|^2 - 1)/4."""
    import torch
    from paper_2205_04401_gb300 import inputs, vp
    circ = [(0.0, 0.0, 1.0)]
    q = inputs.disk_mesh(n_b=63, n_i=330)
    tq, cq = inputs.curved_boundary(q, circ)
    st = inputs.disk_mesh(n_b=63, n_i=330, stagger=True)
    ts, cs = inputs.curved_boundary(st, circ)
    ctx = vp.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    cn = {12: 12.0, 20: 6.8, 25: 3.0, 30: 2.5, 40: 2.0, 50: 1.0}
    rules = [(16, 8, 1.0, "builtin"), (19, 9, 1.0, "builtin")] + \
        [(vp.VP_RULE_SYM(n), n, cn[n], "symmetric") for n in vp.VP_RULE_SYM_DEGREES] + \
        [(vp.VP_RULE_CONICAL(n), n, cn[n], "conical") for n in (12, 20, 25, 30, 40, 50)]
    targets = {}
    for Ns in (12, 20):
        it = vp.Interp(ctx, st.vxy, ts, Ns, curves=cs)
        targets[Ns] = it.nodes().clone()
        it.release()

    def timed(fn, reps=3):
        fn()
        vp.profile_enable(ctx, True)
        vp.profile_reset(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        prof = vp.profile_read(ctx)
        vp.profile_enable(ctx, False)
        return e0.elapsed_time(e1) / reps, {k: v[1] / reps for k, v in prof.items() if v[0]}

    rows = []
    clocks = Clocks(0)
    for rule, deg, c_far, family in rules:
        mesh = vp.mesh_upload_curved(ctx, q.vxy, tq, cq, rule)
        y, _ = vp.mesh_nodes(mesh)
        yn = y.cpu().numpy()
        f2g = torch.from_numpy(inputs.two_gaussian_poly(yn)[None, :].copy()).to(dev)
        f1 = torch.ones((1, mesh.N), dtype=torch.float64, device=dev)
        for Ns in (12, 20):
            txy = targets[Ns]
            ex = (txy.cpu().numpy() ** 2).sum(1) / 4 - 0.25
            for eps in (1e-10, 1e-14):
                nf = vp.nearfield_build(ctx, mesh, node_targets=False, txy=txy, eps=eps, c_far=c_far)
                torch.cuda.synchronize()
                nf.release()
                nf = vp.nearfield_build(ctx, mesh, node_targets=False, txy=txy, eps=eps, c_far=c_far)
                sts = vp.nf_stats(nf)
                M = nf.M
                rec = {"degree": deg, "family": family, "nq": mesh.N // len(tq), "c_far": c_far, "eps": eps, "N_s": Ns, "targets": M,
                       "nodes": mesh.N, "c": sts["n_near"] / M, "s_n": sts["near_leaves"] / M,
                       "s_l": sts["self_panels"] / M, "build_ms": sts["build_ms"],
                       "weights_gb": sts["n_pairs"] * mesh.N // len(tq) * 16 / 1e9}
                u = vp.potential_eval(ctx, nf, f2g, precision=vp.VP_MIXED_FMM)
                for name, prec in (("fmm", vp.VP_MIXED_FMM), ("direct", vp.VP_MIXED)):
                    ms, prof = timed(lambda: vp.potential_eval(ctx, nf, f2g, precision=prec, out=u))
                    rec[name + "_eval_ms"] = ms
                    rec[name + "_far_ms"] = sum(v for k, v in prof.items() if k.startswith("far"))
                    rec[name + "_apply_ms"] = prof.get("apply", 0.0)
                u1 = vp.potential_eval(ctx, nf, f1, precision=vp.VP_MIXED_FMM)
                rec["T_N_ms"] = rec["build_ms"] + rec["fmm_apply_ms"]
                rec["T_F_ms"] = rec["fmm_far_ms"]
                rec["rel_err_f1_vs_exact"] = float(np.abs(u1.cpu().numpy()[0] - ex).max() / np.abs(ex).max())
                rows.append(rec)
                nf.release()
        mesh.release()
    ck = clocks.stop()
    sel = [r for r in rows if r["eps"] == 1e-14 and r["N_s"] == 20]
    best = min(sel, key=lambda r: r["T_N_ms"] + r["T_F_ms"])
    line = {
        "metric": "target_evals_per_s", "value": best["targets"] / ((best["T_N_ms"] + best["T_F_ms"]) / 1e3),
        "unit": "target-evals/s", "n_gpus": 1, "steps": 3, "warmup": 1,
        "ms_per_step": best["T_N_ms"] + best["T_F_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32x2+f64", "data": "synthetic",
        "config": {"workload": "disk_curved_h0.1_721tri_staggered_interp_targets_Ns12_20_two_gaussian_"
                               "far_orders_8_to_50_eps1e-10_1e-14",
                   "step": "near-field build + resident FMM evaluation at the best far order (eps 1e-14, N_s 20)"},
        "clocks": ck, "best": {k: best[k] for k in ("degree", "family", "nq", "T_N_ms", "T_F_ms")},
        "sweep": rows,
    }
    print(json.dumps(line))
    ctx.close()


# ----------------------------------------------------------------- main arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == 3:
        return run_many(args)
    if args.config == 4:
        return run_batch(args)
    if args.config == 5:
        return run_serving(args)
    if args.config == 6:
        return run_curved(args)
    if args.config == 7:
        return run_interp(args)
    if args.config == 8:
        return run_offload(args)
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2205_04401_gb300 import vp
    prec = {"mixed": vp.VP_MIXED, "fp64": vp.VP_FP64, "fmm": vp.VP_MIXED_FMM}[args.precision]

    mesh, fun, extra = make_inputs(args.ntri, args.extra)
    ctx = vp.Context(local)
    stream = torch.cuda.current_stream()
    vxy_d = torch.from_numpy(mesh.vxy).to(dev)
    tri_d = torch.from_numpy(mesh.tri).to(dev)
    extra_d = torch.from_numpy(extra).to(dev)
    # density at the nodes (an input: evaluated once from the node coordinates)
    m0 = vp.mesh_upload_dev(ctx, vxy_d, tri_d, vp.VP_RULE_19_D9)
    y0, _ = vp.mesh_nodes(m0)
    f_np = fun(y0.cpu().numpy())[None, :]
    m0.release()
    f_d = torch.from_numpy(f_np).to(dev)
    N = mesh.nt * 19
    M = N + len(extra)
    u_d = torch.empty((1, M), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        mh = vp.mesh_upload_dev(ctx, vxy_d, tri_d, vp.VP_RULE_19_D9)
        nf = vp.nearfield_build(ctx, mh, node_targets=True, txy=extra_d, fp64_weights=args.fp64_weights)
        vp.potential_eval(ctx, nf, f_d, precision=prec, out=u_d)
        return mh, nf

    for _ in range(max(args.warmup, 0)):
        mh, nf = step()
        torch.cuda.synchronize()
        nf.release()
        mh.release()

    vp.profile_enable(ctx, True)
    vp.profile_reset(ctx)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    stats = None
    for k in range(args.steps):
        flush.fill_(float(k))                      # evict L2 between steps (outside the timed events)
        ev0[k].record(stream)
        mh, nf = step()
        ev1[k].record(stream)
        torch.cuda.synchronize()
        stats = vp.nf_stats(nf)
        nf.release()
        mh.release()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = vp.profile_read(ctx)
    vp.profile_enable(ctx, False)
    t_steps = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_total, value = whole_job(sum(t_steps), args.steps * M, world, dev)
    # the library's kernel launches in one more step of the same kind, listed
    # by the profiler (CUPTI); times the timed steps
    per_step = count_launches(lambda: [h.release() for h in reversed(step())])
    launches = per_step * args.steps if per_step is not None else None

    # resident evaluation (weights cached, serving mode) and FP64 comparison
    mh = vp.mesh_upload_dev(ctx, vxy_d, tri_d, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, mh, node_targets=True, txy=extra_d)
    u_mixed = vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    reps = 3
    for _ in range(reps):
        vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED, out=u_mixed)
    e1.record(stream)
    torch.cuda.synchronize()
    resident_ms = e0.elapsed_time(e1) / reps
    # the same resident evaluation with the far sum by the fast multipole method
    t0 = time.perf_counter()
    u_fmm = vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED_FMM)
    torch.cuda.synchronize()
    fmm_first_s = time.perf_counter() - t0
    e0.record(stream)
    for _ in range(reps):
        vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED_FMM, out=u_fmm)
    e1.record(stream)
    torch.cuda.synchronize()
    fmm_ms = e0.elapsed_time(e1) / reps
    rel_fmm_vs_mixed = float((u_fmm - u_mixed).abs().max() / u_mixed.abs().max())
    fp64_ms = None
    rel_mixed_vs_fp64 = None
    u64 = None
    if not args.no_fp64:
        e0.record(stream)
        u64 = vp.potential_eval(ctx, nf, f_d, precision=vp.VP_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = e0.elapsed_time(e1)
        rel_mixed_vs_fp64 = float((u_mixed - u64).abs().max() / u64.abs().max())

    # end to end through the host-buffer API: host mesh/targets/density in, host u out
    f_pin = torch.from_numpy(f_np).pin_memory()
    x_pin = torch.from_numpy(extra).pin_memory()
    u_host = np.empty((1, M))
    e2e_t = []
    for k in range(args.steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mh2 = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, vp.VP_RULE_19_D9)
        nf2 = vp.nearfield_build_host(ctx, mh2, node_targets=True, txy=x_pin.numpy(), fp64_weights=args.fp64_weights)
        vp.potential_eval_host(ctx, nf2, f_pin.numpy(), precision=prec, out=u_host)
        t1 = time.perf_counter()
        nf2.release()
        mh2.release()
        if k > 0:
            e2e_t.append(t1 - t0)
    e2e_value = world * M / float(np.mean(e2e_t))
    h2d = mesh.vxy.nbytes + mesh.tri.nbytes + extra.nbytes + f_np.nbytes
    d2h = u_host.nbytes

    # accuracy against the oracle on sampled targets, and the CPU baseline
    cpu = None
    rel_oracle = None
    if rank == 0 and not args.no_oracle_check:
        ob = oracle_baseline(mesh, fun, extra, budget_s=10.0)
        um = u_mixed.cpu().numpy()[0, ob["sample"]]
        rel_oracle = float(np.abs(um - ob["u"][0]).max() / np.abs(ob["u"][0]).max())
        cpu = {"value": ob["value"], "unit": "target-evals/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{ob['targets']} random targets of the workload (far sum over all nodes, lists, "
                         f"near/self weights), OpenMP over targets, {ob['seconds']:.1f} s"}

    # roofline of the dominant stage (device time per launch from the library's CUDA events)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 pipe peak (bound "alu"): 152 SMs x 128 FP32 lanes x the maximum SM
    # clock, in thread-instructions per second (no FP32 peak is measured in the
    # peaks file; this is derived from the unit counts and the clock)
    fp32_peak = 152 * 128 * sm_mhz * 1e6
    nq = 19
    # Far sum, algorithmic work per ordered (target, source) pair of the 1e-10
    # float-float path: 45 FP32-pipe instructions, the estimate for one pair
    # evaluated on its own (float-float dx, dy and r^2 from split coordinates
    # ~15; a table logarithm of the float-float r^2 with a short log1p series
    # and its error terms ~22; the float-float charge product and compensated
    # accumulation ~8).  Pairs = N M ordered pairs, whatever the kernel's own
    # scheme (the symmetric kernel shares a pair's distance and logarithm
    # between its two directions and so can exceed this count's roofline).
    ALG_FAR_PER_PAIR = 45.0
    pairs = float(N) * float(M)
    work = {
        "far_ff": ("alu", pairs * ALG_FAR_PER_PAIR * args.steps, fp32_peak / 1e12, "Tinst/s",
                   "algorithmic: 45 FP32-pipe instructions per ordered pair x N M pairs"),
        "apply": ("hbm", float(stats["n_pairs"] * (8 * nq + 4) + N * 8 + M * 8 + M * 8 * 2) * args.steps,
                  hbm, "GB/s", "algorithmic: P (8 nq + 4) + 8 N + 24 M bytes"),
        # list filling copies the counting pass's entries: targets read (16 B), per pair triangle +
        # target + kind written (9 B), row pointers
        "list_fill": ("hbm", float(M * 16 + stats["n_pairs"] * 9 + (M + 1) * 8) * args.steps, hbm, "GB/s",
                      "algorithmic: 16 M + 9 P + 8 (M + 1) bytes"),
    }
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dname, (dn, dms) = dom
    roof = None
    if dname in work and dn > 0:
        bound, units, peak, unit, model = work[dname]
        scale = 1e9 if unit == "GB/s" else 1e12
        achieved = units / (dms / 1e3) / scale
        roof = {"kernel": dname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "launches": dn, "ms_per_launch": dms / dn,
                "model": model, "peak_source": "derived: 152 SMs x 128 FP32 lanes x max SM clock" if bound == "alu"
                else "MEASURED_PEAKS.json hbm_gbs"}
    stage_share = {k: round(v[1] / max(1e-9, sum(x[1] for x in prof.values())), 4) for k, v in prof.items() if v[0]}
    # every modelled stage against its own bound (the dominant one is "roofline")
    rooflines = {}
    for k, (bound, units, peak, unit, model) in work.items():
        n_l, ms_l = prof.get(k, (0, 0.0))
        if n_l and ms_l > 0:
            sc = 1e9 if unit == "GB/s" else 1e12
            a = units / (ms_l / 1e3) / sc
            rooflines[k] = {"bound": bound, "achieved": round(a, 3), "peak": peak, "unit": unit,
                            "frac": round(a / peak, 4), "ms_per_launch": round(ms_l / n_l, 4), "model": model}
    # correction weights: the paper's work counters per second (no roofline
    # fraction: their float-float instruction mix has no algorithmic count)
    n_near = len(vp.rule_table(33)[2])           # the near rule's length
    n_rad = 8 if args.fp64_weights else 5        # radial points: GGQ-8 (FP64 kernel), 5-point rule (float-float)
    for k, cnt, what in (("weights_near", stats["near_leaves"] * n_near,
                          f"near-rule node evaluations (leaves x {n_near})"),
                         ("weights_self", stats["self_panels"] * 16 * n_rad,
                          f"self panel points (panels x 16 arc-length x {n_rad} radial)")):
        n_l, ms_l = prof.get(k, (0, 0.0))
        if n_l and ms_l > 0:
            rooflines[k] = {"bound": "alu", "units_per_s": round(cnt * args.steps / (ms_l / 1e3), 1),
                            "unit": what, "frac": None, "ms_per_launch": round(ms_l / n_l, 4)}
    # list counting: FP64 ellipse predicates per (target, candidate) behind FP32 pre-tests; no algorithmic model
    n_l, ms_l = prof.get("list_count", (0, 0.0))
    if n_l and ms_l > 0:
        rooflines["list_count"] = {"bound": "fp64 predicates / latency", "frac": None,
                                   "ms_per_launch": round(ms_l / n_l, 4)}

    if rank == 0:
        line = {
            "metric": "target_evals_per_s", "value": value, "unit": "target-evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == vp.VP_FP64 else "f32x2+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "targets": M, "nodes": N, "densities": 1, "precision": args.precision,
                       "weights": ("FP64 node quadratures (VP_NF_FP64_WEIGHTS)" if args.fp64_weights else
                                   "float-float node quadratures; FP64 trees and predicates"),
                       "step": "mesh_upload+nearfield_build+potential_eval", "l2": "256 MiB flush between steps",
                       "parallelism": f"replicas{world}"},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "target-evals/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches,
            "roofline": roof,
            "rooflines_by_stage": rooflines,
            "cpu_baseline": cpu,
            "accuracy": {"rel_err_mixed_vs_oracle_sampled": rel_oracle, "rel_err_mixed_vs_fp64_gpu": rel_mixed_vs_fp64},
            "resident_eval": {"mixed_ms": resident_ms, "fp64_ms": fp64_ms, "fmm_ms": fmm_ms,
                              "fmm_first_call_s": fmm_first_s, "fmm_target_evals_per_s": M / (fmm_ms / 1e3),
                              "rel_err_fmm_vs_mixed": rel_fmm_vs_mixed,
                              "mixed_target_evals_per_s": M / (resident_ms / 1e3),
                              "fp64_target_evals_per_s": (M / (fp64_ms / 1e3)) if fp64_ms else None,
                              "mixed_pairs_per_s": M * N / (resident_ms / 1e3)},
            "nf_stats": {k: stats[k] for k in ("n_pairs", "n_self", "n_near", "near_leaves", "self_panels",
                                               "depth_capped", "build_ms")},
            "stage_ms": {k: round(v[1] / max(1, args.steps), 3) for k, v in prof.items() if v[0]},
            "stage_share": stage_share,
        }
        print(json.dumps(line))
    nf.release()
    mh.release()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
