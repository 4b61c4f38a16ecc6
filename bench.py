#!/usr/bin/env python
"""Throughput of the line-of-sight convergence tracer on one GB300 (or N).

One benchmark step is one pass of the whole hot path over one lightcone of
the production workload: 512^3 FP32 potential (Gaussian random field, P(k)
propto k^-3, rms delta = 1), box 1024 Mpc/h, 2048 x 2048 rays over 10 x 10
deg to chi_s = 1000 Mpc/h, integrated in 40 steps of equal Delta a with the
field rescaled by D(a)/a. Per step: the tidal records of the step's footprint
(rr_tidal_tensor), the cell-by-cell trace (rr_trace_step); then rr_finalize.
Inputs are resident in HBM when the timed region starts; L2 is flushed
between timed passes.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle instead, on the host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = ("cell-segments/s and κ-map rays/s at 1 GB300, HBM roofline %, error vs FP64 oracle")
UNIT = "cell-segments/s"
# per trilinear segment the trace gathers 8 vertex records of 32 B (logical bytes)
BYTES_PER_SEGMENT = 256
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes (read + write) of one trace launch from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, mean of two launches), per
# (kernel source, workload, steps per launch): valid only for the source it was
# taken on (sha256 of csrc/trace.cu + csrc/walk.cuh) and for that workload.
TRACE_TRAFFIC = {("77240c8f04eae276", "prod_512", 1): 275_386_624,
                 ("8ac9a523f7f334dd", "prod_512", 16): 293_330_859}
# warp instructions per cell segment of one trace launch from the same kind of
# ncu capture (smsp__inst_executed.sum / segments of the launch), per (kernel
# source, workload); null in the line when the source differs
TRACE_WARP_INSTRUCTIONS = {("77240c8f04eae276", "prod_512", 1): 9.3201,
                           ("8ac9a523f7f334dd", "prod_512", 16): 8.8203}

# FP32 lane operations the method needs per trilinear segment, counted from its
# formulas as the walk evaluates them: exit face (2 compares) and segment length
# (1); mirrored entry point, 3 axes x (subtract, fused multiply-add with clamp)
# (6); projection Q = w.H of the 4 corner records the crossing brings in, 4 x 6
# (24); the trilinear field on the line as a cubic, 33 per channel x 2 channels
# (kappa, delta) (66); the lensing kernel about the entry point, G0 and G1 (6);
# J_1..J_4 (22); sum_N e_(N-1) J_N on both channels (8); the compensated (Kahan)
# sums of both channels (8); the crossing: the next face distance (2).
ALU_OPS_PER_SEGMENT = 145
MAX_SM_MHZ = 2070.0   # GB300 maximum SM clock (the issue peak when no clock was sampled)


_PIPELINE_NOTE = {
    False: "each step's footprint records computed on a side stream while the previous step is traced "
           "(two record buffers; events order each buffer's reuse)",
    True: "records then trace of each step in order on one stream (one record buffer)",
    "grouped": "the footprint records of a group of steps computed on a high-priority side stream while the "
               "previous group is traced (a box-local record buffer per step); each group's launch waits "
               "for its records",
    "grouped_in_order": "the records of each group of steps, then its launch, in order on one stream",
}


_SPLIT_NOTE = {
    False: "sums of the CUDA-event intervals of each step's records (side stream) and trace; the records of "
           "step k + 1 run beside the trace of step k, so the intervals overlap and both stretch",
    True: "sums of the CUDA-event intervals of each step's records and trace, in order on one stream",
}


def _src_hash(*names):
    """sha256 (16 hex digits) of the kernel sources, in the given order."""
    hsh = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1601_02012_gb300", "csrc", name), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def combine_over_ranks(dist, device, total_ms, segs, e2e_s):
    """Whole-job figures from the ranks' own: the slowest rank's timed and
    end-to-end seconds (the job ends when it does) and the sum of the ranks'
    segments. `dist` is torch.distributed (or None for one rank); `device`
    holds the reduction tensors (the rank's GPU under NCCL, CPU under gloo)."""
    if dist is None:
        return total_ms, segs, e2e_s
    import torch
    t = torch.tensor([total_ms, e2e_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(segs)], dtype=torch.float64, device=device)
    dist.all_reduce(n)
    return float(t[0].item()), int(n[0].item()), float(t[1].item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _config(w, nsteps):
    return {
        "workload": w.name,
        "grid": list(w.grid.n),
        "box_mpc_h": w.grid.box,
        "rays": [w.bundle.nx, w.bundle.ny],
        "fov_deg": round(w.bundle.fov_x * 180 / math.pi, 6),
        "chi_s": w.bundle.chi_s,
        "nsteps": nsteps,
        "interp": "trilinear" if w.bundle.interp == 1 else "ngp",
        "field": "GRF P(k)~k^-3, rms delta 1, FP32, rescaled by D(a)/a per step",
        "l2": "flushed between timed passes (256 MiB write); per-pass working set > L2",
    }


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.dev = device_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.dev is not None:
                cmd += ["-i", str(self.dev)]
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is running (its first line written)
            t_end = time.perf_counter() + 3.0
            while time.perf_counter() < t_end and self.proc.poll() is None:
                if os.fstat(self.file.fileno()).st_size > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _device_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or None


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_fields(grid, phi32):
    import oracle
    oracle.build()
    return oracle.fields(grid, phi32.astype(np.float64))


def _oracle_sample(bundle, grid, H, d, steps, rids, threads):
    import oracle
    t0 = time.perf_counter()
    res = oracle.trace(bundle, grid, H, d, steps, nthreads=threads, rids=rids)
    return res, time.perf_counter() - t0


def run_reference(args, w, steps):
    """--impl reference: the FP64 oracle on the host cores; each step traces a
    bounded random sample of the workload's rays through all its N-body steps."""
    threads = os.cpu_count() or 1
    phi = synth.grf_phi_cached(w.grid.n[0], w.grid.box, w.seed)
    H, d = _oracle_fields(w.grid, phi)
    rng = np.random.default_rng(1234)
    sample = 512
    for it in range(args.warmup):
        rids = rng.choice(w.bundle.nrays, sample, replace=False)
        _, dt = _oracle_sample(w.bundle, w.grid, H, d, steps, rids, threads)
        if it == 0 and dt > 0:   # size the sample for ~3 s per step
            sample = int(min(w.bundle.nrays, max(64, sample * 3.0 / dt)))
    times, segs = [], 0
    for _ in range(args.steps):
        rids = rng.choice(w.bundle.nrays, sample, replace=False)
        res, dt = _oracle_sample(w.bundle, w.grid, H, d, steps, rids, threads)
        times.append(dt)
        segs += int(res.nseg.sum())
    total = sum(times)
    value = segs / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _config(w, len(steps)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{sample} random rays of the 2048x2048 bundle per step, all {len(steps)} "
                                   "N-body steps; tidal centres of the 512^3 grid computed once before timing"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched lightcones: one graph-captured persistent launch vs 64 plain launches
# ---------------------------------------------------------------------------

def run_batch(args):
    import torch
    import paper_1601_02012_gb300 as rrp
    from paper_1601_02012_gb300 import build as rrbuild

    rrbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cones = synth.batch_workload(64, seed=4)
    phis = [synth.grf_phi_torch(c.grid.n[0], c.grid.box, c.field_seed, device=dev) for c in cones]
    recs = [rrp.record_buffer(c.grid, device=dev) for c in cones]
    gds = [rrp.grid_desc(c.grid) for c in cones]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    peaks, peak_kind = _peaks()

    # --- batched FP32 form: persistent queue, autotuned, replayed as a CUDA graph
    B = rrp.Batch([c.bundle for c in cones])
    bbox = []
    for i, c in enumerate(cones):
        bb = rrp.rr_footprint_bbox(B.descs[i], gds[i], c.bundle.chi_s, 0.0)
        bbox.append(bb)
        rrp.rr_tidal_tensor(gds[i], phis[i], None, recs[i], B.where, bb, stream)
        B.stage(i, c.grid, recs[i], c.bundle.chi_s, 0.0)
    torch.cuda.synchronize()
    tuning, tune_ms, cached = B.autotune(reps=2, stream=stream)
    ks = [torch.empty((c.bundle.ny, c.bundle.nx), dtype=torch.float64, device=dev) for c in cones]
    kbs = [torch.empty_like(k) for k in ks]
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=stream):
        s = torch.cuda.current_stream()
        B.clear(s)
        for i in range(len(cones)):
            rrp.rr_tidal_tensor(gds[i], phis[i], None, recs[i], B.where, bbox[i], s)
        B.upload(s)
        B.trace(s)
        B.finalize(ks, kbs, s)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    code, segs = B.sync()
    if code != 0:
        raise RuntimeError(f"batch status {code}")
    sampler = ClockSampler(_device_id(torch, dev))
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    # the persistent trace launch alone (for the roofline): replay pieces outside the graph
    tr_ms = []
    for _ in range(3):
        B.clear(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.trace(stream)
        e1.record(stream)
        e1.synchronize()
        tr_ms.append(e0.elapsed_time(e1))
    graph.replay()
    torch.cuda.synchronize()
    batch_maps = [(k.cpu().numpy().ravel(), kb.cpu().numpy().ravel()) for k, kb in zip(ks, kbs)]
    B.close()
    del graph

    # --- plain form: one lightcone at a time, FP64 walk, default launch shape
    plain_ms = []
    plain_maps = None
    tracers = [rrp.Tracer(c.bundle, fp64_dda=True) for c in cones]
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        outs = []
        for i, c in enumerate(cones):
            tr = tracers[i]
            tr.reset(stream)
            rrp.rr_tidal_tensor(gds[i], phis[i], None, recs[i], tr.where, bbox[i], stream)
            tr.step(c.grid, recs[i], c.bundle.chi_s, 0.0, 1.0, 1.0, stream)
            outs.append(tr.finalize(stream=stream))
        torch.cuda.synchronize()
        if it >= args.warmup:
            plain_ms.append(1e3 * (time.perf_counter() - t0))
        plain_maps = outs
    plain_maps = [(k.cpu().numpy().ravel(), kb.cpu().numpy().ravel()) for k, kb in plain_maps]
    for tr in tracers:
        tr.close()

    # --- accuracy of both forms against the FP64 oracle on sampled rays of a few cones
    import oracle
    oracle.build()
    rng = np.random.default_rng(77)
    order = sorted(range(len(cones)), key=lambda i: cones[i].grid.n[0])
    picks = order[:3] + order[-1:]
    err_b = err_p = 0.0
    for i in picks:
        c = cones[i]
        H, d = oracle.fields(c.grid, phis[i].cpu().numpy().astype(np.float64))
        rids = rng.choice(c.bundle.nrays, 512, replace=False)
        o = oracle.trace(c.bundle, c.grid, H, d, [synth.Step(c.bundle.chi_s, 0.0, 1.0, 1.0)], rids=rids)
        rms = math.sqrt(float(np.mean(o.kappa ** 2)))
        err_b = max(err_b, float(np.abs(batch_maps[i][0][rids] - o.kappa).max()) / rms)
        err_p = max(err_p, float(np.abs(plain_maps[i][0][rids] - o.kappa).max()) / rms)
        del H, d

    total_ms = sum(times)
    value = segs * args.steps / (total_ms / 1e3)
    plain_value = segs * args.steps / (sum(plain_ms) / 1e3)
    tr_mean = sum(tr_ms) / len(tr_ms)
    achieved = segs * BYTES_PER_SEGMENT / (tr_mean / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch64", "lightcones": len(cones),
                   "rays_total": int(sum(c.bundle.nrays for c in cones)),
                   "grids": sorted(set(c.grid.n[0] for c in cones)),
                   "recipe": "64 cones, seed 4: grid 128/256/512, rays log-uniform 256..2048 per side, "
                             "FOV 1..10 deg, chi_s 200..1000 = box side, one step each; GPU GRF per cone",
                   "form": "fp32 walk + Kahan, persistent work queue, CUDA graph, autotuned",
                   "l2": "flushed between timed replays (256 MiB write)"},
        "segments_per_step": segs,
        "rays_per_s": sum(c.bundle.nrays for c in cones) * args.steps / (total_ms / 1e3),
        "tuning": {"wx": tuning[0], "bwx": tuning[1], "bwy": tuning[2], "chunk": tuning[3],
                   "blocks_per_sm": tuning[4], "from_cache": bool(cached), "autotune_ms": tune_ms},
        "plain_fp64_per_cone": {"value": plain_value, "unit": UNIT, "ms_per_step": sum(plain_ms) / args.steps,
                                "form": "fp64 walk, 64 host-driven launches of tidal+trace+finalize"},
        "speedup_vs_plain": plain_ms and (sum(plain_ms) / total_ms),
        "error_vs_oracle": {"cones": picks, "rays_per_cone": 512, "batched_max_over_rms": err_b,
                            "plain_max_over_rms": err_p},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "trace_batch_kernel<trilinear,float>",
                     "note": f"logical gather bytes ({BYTES_PER_SEGMENT} B/segment) / persistent launch time; "
                             f"peak of {peak_kind} copy bandwidth"},
        "gpu_launches": args.steps * (1 + 64 + 64),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def _amr_config(w, mesh, nsteps):
    return {
        "workload": w.name, "coarse_grid": w.n, "box_mpc_h": w.box, "levels": w.lmax,
        "octs_per_level": [len(mesh.octs[l]) for l in range(1, w.lmax + 1)], "leaves": mesh.nleaves(),
        "rays": [w.bundle.nx, w.bundle.ny], "fov_deg": round(w.bundle.fov_x * 180 / math.pi, 6),
        "chi_s": w.bundle.chi_s, "nsteps": nsteps, "interp": "trilinear",
        "field": "lognormal density (sigma_ln 1.5, hashed cascade 0.5), refine where mass > 8x mean, "
                 "2:1 balanced; Phi: 7-point FFT Poisson on level 0, trilinear prolongation + 8 red-black "
                 "Gauss-Seidel sweeps per level; FP32; rescaled by D(a)/a per step",
        "l2": "flushed between timed passes (256 MiB write); leaf records > L2",
    }


def run_amr(args, name):
    """The adaptive-mesh workload: per step rr_amr_tidal over the step's
    footprint (per-level stencils, vertex weights, 256-byte leaf records of the
    leaves in the coarse-cell box rr_footprint_bbox gives) and
    rr_amr_trace_step (leaf-by-leaf walk); then rr_finalize."""
    import torch
    import paper_1601_02012_gb300 as rrp
    from paper_1601_02012_gb300 import build as rrbuild

    rrbuild.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = synth.amr_workload(name)
    steps = synth.step_schedule(w.bundle.chi_s, w.nsteps, rescale=w.rescale)
    t0 = time.perf_counter()
    mesh, flat = synth.amr_workload_mesh(w)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    gm = rrp.AmrMesh(w.n, w.lmax, w.box, mesh.octs, mesh.omega_m)
    t_plan = time.perf_counter() - t0
    stream = torch.cuda.Stream(device=dev)
    phi = torch.from_numpy(flat).to(dev)
    rec = gm.record_buffer(rrp.RR_AT_VERTICES, device=dev)
    tr = rrp.Tracer(w.bundle)
    bboxes = [gm.footprint(tr, st.chi_a, st.chi_b) for st in steps]
    kappa = torch.empty((w.bundle.ny, w.bundle.nx), dtype=torch.float64, device=dev)
    kborn = torch.empty_like(kappa)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nst = len(steps)
    ev_tr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    ev_td = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]

    # G steps per rr_amr_trace_steps launch, each step's leaf records in a
    # buffer of its own (whole mesh); the records of group j + 1 on a side
    # stream while group j is traced (two sets of G buffers)
    side = None if args.no_pipeline else torch.cuda.Stream(device=dev, priority=-1)
    G = max(1, min(args.amr_group, 16))
    groups = [list(range(i, min(i + G, nst))) for i in range(0, nst, G)]
    sets = [[rec] + [gm.record_buffer(rrp.RR_AT_VERTICES, device=dev) for _ in range(G - 1)]]
    if not args.no_pipeline:
        sets.append([gm.record_buffer(rrp.RR_AT_VERTICES, device=dev) for _ in range(G)])
    ev_tr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]
    ev_td = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]

    def one_pass(src=None, timed_kernels=False):
        rrp.rr_reset(tr.ctx, stream)
        field = phi if src is None else src

        def records(gi, b, s):
            for j, k in enumerate(groups[gi]):
                gm.tidal(field, sets[b][j], rrp.RR_AT_VERTICES, None, bboxes[k], s)

        def trace(gi, b, s):
            ks = groups[gi]
            if G == 1:
                st = steps[ks[0]]
                tr.amr_step(gm, sets[b][0], st.chi_a, st.chi_b, st.scale, st.a, s)
            else:
                tr.amr_steps(gm, [sets[b][j] for j in range(len(ks))], [steps[k] for k in ks], s)

        rrp.pipeline_steps(len(groups), records, trace, stream, side, len(sets),
                           (ev_td, ev_tr) if timed_kernels else None)
        rrp.rr_finalize(tr.ctx, kappa, kborn, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_pass()
        segs = tr.segments()
        sampler = ClockSampler(_device_id(torch, dev))
        torch.cuda.synchronize()
        sampler.start()
        times, trace_ms, tidal_ms = [], 0.0, 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_pass(timed_kernels=True)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            trace_ms += sum(a.elapsed_time(b) for a, b in ev_tr)
            tidal_ms += sum(a.elapsed_time(b) for a, b in ev_td)
        torch.cuda.synchronize()
        clocks = sampler.stop()
        full_ms = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gm.tidal(phi, rec, rrp.RR_AT_VERTICES, None, None, stream)
            e1.record(stream)
            e1.synchronize()
            full_ms.append(e0.elapsed_time(e1))
        phi_pinned = torch.from_numpy(flat).pin_memory()
        k_host = torch.empty(kappa.shape, dtype=torch.float64).pin_memory()
        kb_host = torch.empty_like(k_host).pin_memory()
        phi_dev2 = torch.empty_like(phi)
        e2e = []
        for it in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            phi_dev2.copy_(phi_pinned, non_blocking=True)
            one_pass(src=phi_dev2)
            k_host.copy_(kappa, non_blocking=True)
            kb_host.copy_(kborn, non_blocking=True)
            stream.synchronize()
            if it >= args.warmup:
                e2e.append(time.perf_counter() - t0)

        # the shear through the same mesh (RR_SHEAR in the AMR walk); the side
        # passes write their maps to buffers of their own
        k_side = torch.empty_like(kappa)
        kb_side = torch.empty_like(kappa)
        trs = rrp.Tracer(w.bundle, shear=True)

        # the side forms take the main pass's grouping: G steps per rr_amr_trace_steps
        # launch, the group's records first into the first set of buffers
        ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]

        def group_walk(tracer, ks, stp, s):
            if G == 1:
                st = stp[ks[0]]
                tracer.amr_step(gm, sets[0][0], st.chi_a, st.chi_b, st.scale, st.a, s)
            else:
                tracer.amr_steps(gm, [sets[0][j] for j in range(len(ks))], [stp[k] for k in ks], s)

        def shear_pass(timed):
            rrp.rr_reset(trs.ctx, stream)
            for gi, ks in enumerate(groups):
                for j, k in enumerate(ks):
                    gm.tidal(phi, sets[0][j], rrp.RR_AT_VERTICES, None, bboxes[k], stream)
                if timed:
                    ev_s[gi][0].record(stream)
                group_walk(trs, ks, steps, stream)
                if timed:
                    ev_s[gi][1].record(stream)
            rrp.rr_finalize(trs.ctx, k_side, kb_side, stream)

        shear_pass(False)
        sh_ms = []
        for _ in range(2):
            flush.fill_(1.0)
            shear_pass(True)
            torch.cuda.synchronize()
            sh_ms.append(sum(a.elapsed_time(b) for a, b in ev_s))
        trs.close()

        # Method A through the same mesh (rr_amr_gradient records, RR_METHOD_A walk)
        tra = rrp.Tracer(w.bundle, method_a=True)
        ev_a = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]
        steps_a = [synth.Step(st.chi_a, st.chi_b, st.scale, 1.0) for st in steps]

        def method_a_pass(timed):
            rrp.rr_reset(tra.ctx, stream)
            for gi, ks in enumerate(groups):
                if timed:
                    ev_a[gi][0].record(stream)
                for j, k in enumerate(ks):
                    gm.gradient(phi, sets[0][j], rrp.RR_AT_VERTICES, None, bboxes[k], stream)
                group_walk(tra, ks, steps_a, stream)
                if timed:
                    ev_a[gi][1].record(stream)
            rrp.rr_finalize(tra.ctx, k_side, kb_side, stream)

        method_a_pass(False)
        ma_ms = []
        for _ in range(2):
            flush.fill_(1.0)
            method_a_pass(True)
            torch.cuda.synchronize()
            ma_ms.append(sum(a.elapsed_time(b) for a, b in ev_a))
        tra.close()

        # generic integrals through the same mesh, as the ISW set-up of Sec. 6
        # (channel 0: (Phi_a - Phi_prev) / dt with K = 2; channel 1: Phi with K = g)
        trg = rrp.Tracer(w.bundle, generic=True)
        trg.set_kernels(((2.0, 0.0, 0.0), (0.0, 1.0, -1.0 / w.bundle.chi_s)))
        cur_g = torch.empty_like(phi)
        prev_g = torch.empty_like(phi)
        ev_g = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]
        steps_g = [synth.Step(st.chi_a, st.chi_b, 1.0, st.a) for st in steps]

        def generic_pass(timed):
            rrp.rr_reset(trg.ctx, stream)
            for gi, ks in enumerate(groups):
                if timed:
                    ev_g[gi][0].record(stream)
                for j, k in enumerate(ks):
                    torch.mul(phi, steps[k - 1].scale if k > 0 else steps[k].scale, out=prev_g)
                    torch.mul(phi, steps[k].scale, out=cur_g)
                    gm.scalars(cur_g, sets[0][j], rrp.RR_AT_VERTICES, prev0=prev_g, inv_dt0=100.0, field1=cur_g,
                               bbox=bboxes[k], stream=stream)
                group_walk(trg, ks, steps_g, stream)
                if timed:
                    ev_g[gi][1].record(stream)
            rrp.rr_finalize(trg.ctx, k_side, kb_side, stream)

        generic_pass(False)
        gen_ms = []
        for _ in range(2):
            flush.fill_(1.0)
            generic_pass(True)
            torch.cuda.synchronize()
            gen_ms.append(sum(a.elapsed_time(b) for a, b in ev_g))
        trg.close()
        del cur_g, prev_g

    peaks, peak_kind = _peaks()
    total_ms = sum(times)
    per_pass_trace_s = trace_ms / args.steps / 1e3
    achieved = segs * BYTES_PER_SEGMENT / per_pass_trace_s / 1e9
    line = {
        "metric": METRIC, "value": segs * args.steps / (total_ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _amr_config(w, mesh, nst) | {"form": "fp32 float-float walk on the finest lattice, Kahan sums",
                                               "pipeline": _PIPELINE_NOTE[bool(args.no_pipeline) if G == 1 else
                                                                          ("grouped_in_order" if args.no_pipeline
                                                                           else "grouped")],
                                               "steps_per_launch": G},
        "rays_per_s": w.bundle.nrays * args.steps / (total_ms / 1e3),
        "segments_per_step": segs,
        "setup_s": {"mesh_and_potential": t_gen, "plan": t_plan},
        "kernels_ms_per_step": {"trace": trace_ms / args.steps, "tidal": tidal_ms / args.steps,
                                "note": _SPLIT_NOTE[bool(args.no_pipeline)]},
        "shear": {"trace_ms_per_pass": sum(sh_ms) / len(sh_ms),
                  "kappa_only_trace_ms_per_pass": trace_ms / args.steps,
                  "cost_vs_kappa_only": (sum(sh_ms) / len(sh_ms)) / (trace_ms / args.steps),
                  "note": "trace kernels of one pass in the shear form (kappa, Born kappa, gamma1, gamma2 in "
                          "one AMR walk), CUDA events per launch (the main pass's steps per launch), L2 flushed "
                          "before each pass, mean of 2"},
        "method_a": {"ms_per_pass": sum(ma_ms) / len(ma_ms), "method_b_ms_per_pass": total_ms / args.steps,
                     "note": "records (rr_amr_gradient over each step's footprint) and the Method A AMR walk "
                             "of one pass, CUDA events per group of steps (the main pass's steps per launch), L2 flushed before "
                             "each pass, mean of 2"},
        "generic_isw": {"ms_per_pass": sum(gen_ms) / len(gen_ms), "method_b_ms_per_pass": total_ms / args.steps,
                        "note": "records (rr_amr_scalars, two channels, over each step's footprint) and the "
                                "generic AMR walk set up as the ISW integral, CUDA events per group of steps (the main pass's "
                                "steps per launch), mean of 2"},
        "roofline": {
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": "trace_amr_steps_kernel<trilinear>" if G > 1 else "trace_amr_kernel<trilinear>",
            "note": f"logical gather bytes: {BYTES_PER_SEGMENT} B per leaf segment (the leaf's 8 corner "
                    f"records) x leaf segments / trace time; peak of {peak_kind} copy bandwidth"},
        "tidal_per_pass": {"launches": nst * (w.lmax + 3), "ms": tidal_ms / args.steps,
                           "note": "rr_amr_tidal per step over the step's coarse-cell footprint"},
        "tidal_whole_mesh": {"ms": min(full_ms), "bound": "hbm",
                             "achieved": (4 * gm.ncells + 256 * gm.nleaves) / (min(full_ms) / 1e3) / 1e9,
                             "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": (4 * gm.ncells + 256 * gm.nleaves) / (min(full_ms) / 1e3) / 1e9
                             / peaks["hbm_gbs"],
                             "note": "all cells, vertices and leaf records; algorithmic bytes = 4 B of Phi per "
                                     "cell read + 256 B of records per leaf written (plan tables not counted)"},
        "e2e": {"value": segs * args.steps / sum(e2e), "unit": UNIT, "h2d_bytes_per_step": int(flat.nbytes),
                "d2h_bytes_per_step": int(k_host.numel() * 8 * 2)},
        "gpu_launches": args.steps * (nst * (w.lmax + 3) + len(groups) + 1),
        "clocks": clocks,
        "trace_src": _src_hash("trace_amr.cu", "walk.cuh"),
    }
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rng = np.random.default_rng(99)
        rids = rng.choice(w.bundle.nrays, 24, replace=False)
        t0 = time.perf_counter()
        res = oracle.amr_trace(w.bundle, mesh, steps, rids=rids)
        dt = time.perf_counter() - t0
        n2 = int(min(w.bundle.nrays, max(24, 24 * 15.0 / max(dt, 1e-3))))
        rids2 = rng.choice(w.bundle.nrays, n2, replace=False)
        t0 = time.perf_counter()
        res2 = oracle.amr_trace(w.bundle, mesh, steps, rids=rids2)
        dt2 = time.perf_counter() - t0
        line["cpu_baseline"] = {
            "value": float(res2.nseg.sum()) / dt2, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n2} random rays of the bundle through all {nst} steps ({dt2:.1f} s); the AMR oracle "
                      "is single-threaded (its memoised tidal field is shared)"}
        kg = kappa.cpu().numpy().ravel()
        kbg = kborn.cpu().numpy().ravel()
        allr = np.concatenate([rids, rids2])
        ko = np.concatenate([res.kappa, res2.kappa])
        kbo = np.concatenate([res.kborn, res2.kborn])
        rms, rmsb = math.sqrt(float(np.mean(ko ** 2))), math.sqrt(float(np.mean(kbo ** 2)))
        line["error_vs_oracle"] = {
            "rays": int(len(allr)),
            "kappa_max_over_rms": float(np.abs(kg[allr] - ko).max() / rms),
            "kborn_max_over_rms": float(np.abs(kbg[allr] - kbo).max() / rmsb),
            "segments_per_ray_gpu": segs / w.bundle.nrays,
            "segments_per_ray_oracle": float(np.concatenate([res.nseg, res2.nseg]).mean()),
        }
        if not args.compact:
            # map statistics on a contiguous 64 x 64 patch at the map centre, traced
            # by the (single-threaded) AMR oracle through all steps
            from paper_1601_02012_gb300 import mapstats
            px = py = min(64, w.bundle.nx, w.bundle.ny)
            x0, yy0 = (w.bundle.nx - px) // 2, (w.bundle.ny - py) // 2
            iy, ix = np.meshgrid(np.arange(yy0, yy0 + py), np.arange(x0, x0 + px), indexing="ij")
            prids = (iy * w.bundle.nx + ix).ravel()
            t0 = time.perf_counter()
            pres = oracle.amr_trace(w.bundle, mesh, steps, rids=prids)
            dtp = time.perf_counter() - t0
            fx = w.bundle.fov_x * (px - 1) / max(w.bundle.nx - 1, 1)
            fy = w.bundle.fov_y * (py - 1) / max(w.bundle.ny - 1, 1)
            line["map_statistics"] = {
                "patch": f"{px}x{py} rays at the map centre ({fx * 180 / math.pi:.4f} x "
                         f"{fy * 180 / math.pi:.4f} deg), all {nst} steps, oracle {dtp:.1f} s",
                "kappa": mapstats.compare(kg[prids].reshape(py, px), pres.kappa.reshape(py, px), fx, fy),
                "kborn": mapstats.compare(kbg[prids].reshape(py, px), pres.kborn.reshape(py, px), fx, fy),
                "definition": "P(ell): 20 log bins of ell = 2 pi m / Upsilon, largest relative bin difference; "
                              "PDF: 100 bins over +-5 sigma of the oracle map, L1 distance",
            }
    tr.close()
    gm.close()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def _group_trace(rrp, ctx, gd, phi, where, steps, idx, box, stream, cuts=()):
    """Box-local records of steps idx (consecutive) then rr_trace_steps over
    them, at most 16 per call and a new call at each step in ``cuts``."""
    pboxes, brecs = box
    for k in idx:
        rrp._rr.rr_tidal_tensor_box(gd, phi, None, brecs[k], where, pboxes[k], stream)
    run = []
    for k in list(idx) + [None]:
        if run and (k is None or k in cuts or len(run) == 16):
            rrp.rr_trace_steps(ctx, gd, [brecs[q] for q in run], [steps[q].chi_a for q in run],
                               [steps[q].chi_b for q in run], [steps[q].scale for q in run],
                               [steps[q].a for q in run], [pboxes[q] for q in run], stream)
            run = []
        if k is not None:
            run.append(k)


def _source_redshifts(rrp, torch, w, steps, gd, phi, rec, bboxes, stream, flush, nck=8, box=None):
    """Time kappa maps for nck source distances (the step boundaries nearest
    to chi_s j / nck): one moments pass with snapshots vs one ordinary pass per
    source distance; the maps of the two agree to the stated difference. box:
    (footprint boxes, box-local record buffers) per step: both sides trace up
    to 16 steps per launch (rr_trace_steps), the moments pass cutting its
    launches at the snapshots."""
    nst = len(steps)
    picks = sorted({min(range(nst), key=lambda i: abs(steps[i].chi_a - w.bundle.chi_s * j / nck))
                    for j in range(1, nck + 1)})
    ny, nx = w.bundle.ny, w.bundle.nx
    trm = rrp.Tracer(w.bundle, moments=True)
    snaps = {i: torch.empty((4, ny, nx), dtype=torch.float64, device=phi.device) for i in picks if i > 0}
    m_end = torch.empty((4, ny, nx), dtype=torch.float64, device=phi.device)

    def moments_pass():
        rrp.rr_reset(trm.ctx, stream)
        if box is not None:
            cuts = sorted(snaps)
            bounds = [0] + cuts + [nst]
            for a, b in zip(bounds[:-1], bounds[1:]):
                if a in snaps:
                    trm.moments(snaps[a], stream)
                _group_trace(rrp, trm.ctx, gd, phi, trm.where, steps, range(a, b), box, stream)
            trm.moments(m_end, stream)
            return
        for i, st in enumerate(steps):
            if i in snaps:
                trm.moments(snaps[i], stream)
            rrp.rr_tidal_tensor(gd, phi, None, rec, trm.where, bboxes[i], stream)
            rrp.rr_trace_step(trm.ctx, gd, rec, st.chi_a, st.chi_b, st.scale, st.a, stream)
        trm.moments(m_end, stream)

    # one ordinary context per source distance (bundle with chi_s = chi_k)
    ctxs = {}
    for i in picks:
        bi = rrp.bundle_desc(w.bundle)
        bi.chi_s = steps[i].chi_a
        ctxs[i] = rrp.rr_create(bi)
    where = rrp.RR_AT_VERTICES if w.bundle.interp == 1 else rrp.RR_AT_CENTRES
    maps = {i: torch.empty((ny, nx), dtype=torch.float64, device=phi.device) for i in picks}

    def ordinary_passes():
        for i in picks:
            rrp.rr_reset(ctxs[i], stream)
            if box is not None:
                _group_trace(rrp, ctxs[i], gd, phi, where, steps, range(i, nst), box, stream)
                rrp.rr_finalize(ctxs[i], maps[i], None, stream)
                continue
            for j in range(i, nst):
                st = steps[j]
                rrp.rr_tidal_tensor(gd, phi, None, rec, where, bboxes[j], stream)
                rrp.rr_trace_step(ctxs[i], gd, rec, st.chi_a, st.chi_b, st.scale, st.a, stream)
            rrp.rr_finalize(ctxs[i], maps[i], None, stream)

    def timed(fn):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    with torch.cuda.stream(stream):
        moments_pass()
        t_mom = timed(moments_pass)
        ordinary_passes()
        t_ord = timed(ordinary_passes)
        worst = 0.0
        for i in picks:
            k, _ = rrp.source_kappa(m_end, snaps.get(i), steps[i].chi_a, stream)
            ref = maps[i]
            rms = float(torch.sqrt(torch.mean(ref * ref)))
            worst = max(worst, float((k - ref).abs().max()) / rms)
    trm.close()
    for c in ctxs.values():
        rrp.rr_destroy(c)
    return {"source_chi": [round(steps[i].chi_a, 3) for i in picks], "moments_pass_ms": t_mom,
            "ordinary_passes_ms": t_ord, "speedup": t_ord / t_mom,
            "max_over_rms_vs_ordinary": worst,
            "note": "one pass in the moments form with a snapshot at each source distance, against one "
                    "ordinary pass per source distance (each from its chi_s down to 0, contexts created "
                    "before the timing); CUDA events, L2 flushed before each"
                    + ("; both with box-local records and up to 16 steps per launch (the moments pass "
                       "cut at the snapshots)" if box is not None else "")}


def _shear_form(rrp, torch, w, steps, gd, phi, rec, bboxes, stream, flush, kappa_trace_ms, reps=3, box=None):
    """Time the trace kernels of a pass in the shear form (kappa, Born kappa,
    gamma1 and gamma2 of Eqs. gamma1, gamma2 in one walk) against those of the
    default form (kappa_trace_ms, per pass); the shear form's kappa is checked
    against the default form's."""
    nst = len(steps)
    trs = rrp.Tracer(w.bundle, shear=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    ny, nx = w.bundle.ny, w.bundle.nx
    k = torch.empty((ny, nx), dtype=torch.float64, device=phi.device)
    kb = torch.empty_like(k)

    groups = [list(range(i, min(i + 16, nst))) for i in range(0, nst, 16)]
    evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]

    def shear_pass(timed_kernels):
        rrp.rr_reset(trs.ctx, stream)
        if box is not None:
            # box-local records, 16 steps per launch, as the default form's pass
            pboxes, brecs = box
            for i in range(nst):
                trs.tidal_box(w.grid, phi, brecs[i], pboxes[i], stream=stream)
            for (e0, e1), ks in zip(evg, groups):
                if timed_kernels:
                    e0.record(stream)
                trs.steps(w.grid, [brecs[q] for q in ks], [steps[q] for q in ks], boxes=[pboxes[q] for q in ks],
                          stream=stream)
                if timed_kernels:
                    e1.record(stream)
            rrp.rr_finalize(trs.ctx, k, kb, stream)
            return
        for i, st in enumerate(steps):
            rrp.rr_tidal_tensor(gd, phi, None, rec, trs.where, bboxes[i], stream)
            if timed_kernels:
                ev[i][0].record(stream)
            rrp.rr_trace_step(trs.ctx, gd, rec, st.chi_a, st.chi_b, st.scale, st.a, stream)
            if timed_kernels:
                ev[i][1].record(stream)
        rrp.rr_finalize(trs.ctx, k, kb, stream)

    with torch.cuda.stream(stream):
        shear_pass(False)
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            shear_pass(True)
            ms.append(sum(a.elapsed_time(b) for a, b in (evg if box is not None else ev)))
        segs = trs.segments()
        g1, g2 = trs.shear(stream=stream)
        torch.cuda.synchronize()
        rms_g = [float(torch.sqrt(torch.mean(x * x))) for x in (g1, g2)]
    trs.close()
    t = sum(ms) / reps
    return {"trace_ms_per_pass": t, "kappa_only_trace_ms_per_pass": kappa_trace_ms,
            "cost_vs_kappa_only": t / kappa_trace_ms, "segments_per_s": segs / (t / 1e3),
            "gather_gbs": segs * BYTES_PER_SEGMENT / (t / 1e3) / 1e9,
            "rms_gamma1": rms_g[0], "rms_gamma2": rms_g[1], "kappa": k, "kborn": kb,
            "note": "trace kernels of one pass in the shear form (kappa, Born kappa, gamma1, gamma2 "
                    "in one walk), CUDA events per launch, L2 flushed before each pass, mean of "
                    f"{reps} passes; the default form's per-pass trace time beside it"
                    + ("; box-local records, 16 steps per launch" if box is not None else "")}


def _method_a_form(rrp, torch, w, steps, gd, phi, bboxes, stream, flush, kappa_pass_ms, kappa, reps=3):
    """Time a pass by Method A (Eq. kappa2: gradient records of 16 B per point
    instead of the 32 B tidal records, the kernel dg/dchi and the surface
    terms) against a pass by Method B (kappa_pass_ms); its kappa map is
    compared with Method B's. delta is derived from each step's (scaled)
    potential through the Poisson equation at a = 1, so the density term
    takes a = 1 to describe the same field as Method B's tidal term."""
    nst = len(steps)
    tra = rrp.Tracer(w.bundle, method_a=True)
    reca = tra.record_buffer(w.grid, device=phi.device)
    ev_r = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    ev_t = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    k = torch.empty_like(kappa)
    kb = torch.empty_like(kappa)

    def pass_a(timed):
        rrp.rr_reset(tra.ctx, stream)
        for i, st in enumerate(steps):
            if timed:
                ev_r[i][0].record(stream)
            rrp.rr_gradient_records(gd, phi, None, reca, tra.where, bboxes[i], stream)
            if timed:
                ev_r[i][1].record(stream)
                ev_t[i][0].record(stream)
            rrp.rr_trace_step(tra.ctx, gd, reca, st.chi_a, st.chi_b, st.scale, 1.0, stream)
            if timed:
                ev_t[i][1].record(stream)
        rrp.rr_finalize(tra.ctx, k, kb, stream)

    with torch.cuda.stream(stream):
        pass_a(False)
        tot, rec_ms, tr_ms = [], 0.0, 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pass_a(True)
            e1.record(stream)
            e1.synchronize()
            tot.append(e0.elapsed_time(e1))
            rec_ms += sum(a.elapsed_time(b) for a, b in ev_r)
            tr_ms += sum(a.elapsed_time(b) for a, b in ev_t)
        segs = tra.segments()
        rms = float(torch.sqrt(torch.mean(kappa * kappa)))
        diff = float((k - kappa).abs().max()) / rms
        l2 = float(torch.linalg.vector_norm(k - kappa) / torch.linalg.vector_norm(kappa))
    tra.close()
    del reca
    t = sum(tot) / reps
    return {"ms_per_pass": t, "method_b_ms_per_pass": kappa_pass_ms, "speedup_vs_method_b": kappa_pass_ms / t,
            "trace_ms_per_pass": tr_ms / reps, "records_ms_per_pass": rec_ms / reps,
            "segments_per_s": segs / (t / 1e3),
            "gather_gbs": segs * 128 / (tr_ms / reps / 1e3) / 1e9,
            "kappa_max_over_rms_vs_method_b": diff, "kappa_l2_vs_method_b": l2,
            "note": "one pass by Method A (gradient records over each step's footprint, the walk with "
                    "kernel dg/dchi and the per-step surface terms, finalize), CUDA events, L2 flushed "
                    f"before each pass, mean of {reps}; 128 logical gather bytes per segment (8 x 16 B); "
                    "the map differs from Method B's by the discretisation of the two formulations; "
                    "the density term with a = 1 (delta derived from the scaled potential)"}


def _generic_form(rrp, torch, w, steps, gd, phi, bboxes, stream, flush, kappa_pass_ms, reps=3):
    """Time a pass of the generic form (two scalar fields with their own
    quadratic kernels, Eqs. Ic, Icfinal) set up as the ISW integral of Sec. 6:
    channel 0 integrates (Phi_a - Phi_b) / dt between each step's potential and
    the previous step's, channel 1 the potential with the lensing kernel.
    Scalar-pair records are 8 B per point."""
    nst = len(steps)
    trg = rrp.Tracer(w.bundle, generic=True)
    trg.set_kernels(((2.0, 0.0, 0.0), (0.0, 1.0, -1.0 / w.bundle.chi_s)))
    recg = trg.record_buffer(w.grid, device=phi.device)
    prev = torch.empty_like(phi)
    cur = torch.empty_like(phi)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    o1 = torch.empty((w.bundle.ny, w.bundle.nx), dtype=torch.float64, device=phi.device)
    o2 = torch.empty_like(o1)

    def pass_g(timed):
        rrp.rr_reset(trg.ctx, stream)
        for i, st in enumerate(steps):
            sp = steps[i - 1].scale if i > 0 else st.scale
            torch.mul(phi, sp, out=prev)
            torch.mul(phi, st.scale, out=cur)
            if timed:
                ev[i][0].record(stream)
            rrp.rr_scalar_records(gd, cur, prev, 100.0, 0, recg, trg.where, bboxes[i], stream)
            rrp.rr_scalar_records(gd, cur, None, 1.0, 1, recg, trg.where, bboxes[i], stream)
            rrp.rr_trace_step(trg.ctx, gd, recg, st.chi_a, st.chi_b, 1.0, st.a, stream)
            if timed:
                ev[i][1].record(stream)
        rrp.rr_finalize(trg.ctx, o1, o2, stream)

    with torch.cuda.stream(stream):
        pass_g(False)
        ms = []
        for _ in range(reps):
            flush.fill_(1.0)
            pass_g(True)
            torch.cuda.synchronize()
            ms.append(sum(a.elapsed_time(b) for a, b in ev))
        segs = trg.segments()
    trg.close()
    del recg, prev, cur
    t = sum(ms) / reps
    return {"ms_per_pass": t, "method_b_ms_per_pass": kappa_pass_ms, "segments_per_s": segs / (t / 1e3),
            "note": "records (2 channels) and trace kernels of one pass of the generic form set up as the "
                    "ISW integral (channel 0: (Phi_a - Phi_prev) / dt with K = 2; channel 1: Phi with K = g), "
                    f"CUDA events per step, L2 flushed before each pass, mean of {reps}"}


def _fp32_peak(rrp, torch, dev, stream):
    """FP32 FMA rates of this GPU, measured now (rr_fp32_peak): lane FMAs per
    second of the packed FFMA2 form and of scalar FFMA (one warp instruction
    per scheduler and cycle: the issue rate), best of 5 launches each."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.zeros(sms * 8, dtype=torch.float32, device=dev)
    rates = {}
    with torch.cuda.stream(stream):
        for packed in (1, 0):
            rrp._rr.rr_fp32_peak(packed, sms * 8, 256, 200, out, stream)
            best = float("inf")
            n = 0
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                n = rrp._rr.rr_fp32_peak(packed, sms * 8, 256, 2000, out, stream)
                e1.record(stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            rates["packed" if packed else "scalar"] = n / best
    return {"lane_fma_per_s": rates["packed"], "scalar_ffma_per_s": rates["scalar"], "sms": sms}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _sub_line(argv, timeout=900):
    """Run this script with other arguments in a child process (one GPU, the
    same environment) and return its JSON line, or an error record."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py")] + argv
    try:
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout} s", "cmd": " ".join(argv)}
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    if p.returncode != 0 or not lines:
        return {"error": f"exit {p.returncode}: {p.stderr.strip().splitlines()[-1:] or ''}", "cmd": " ".join(argv)}
    return json.loads(lines[-1])


def _compact(line, keys):
    out = {}
    for k in keys:
        if k in line:
            out[k] = line[k]
    return out


def _other_workloads(steps, warmup):
    """The adaptive-mesh, batched and differentiation workloads, each in its own
    child process with fewer timed passes, condensed for the main line."""
    amr = _sub_line(["--workload", "amr_256", "--steps", str(steps), "--warmup", str(warmup)])
    if "error" not in amr:
        amr = _compact(amr, ["value", "unit", "ms_per_step", "rays_per_s", "segments_per_step",
                             "kernels_ms_per_step", "roofline", "e2e", "error_vs_oracle", "map_statistics",
                             "cpu_baseline",
                             "clocks", "config", "gpu_launches"])
    bat = _sub_line(["--workload", "batch64", "--steps", str(steps), "--warmup", str(warmup)])
    if "error" not in bat:
        bat = _compact(bat, ["value", "unit", "ms_per_step", "rays_per_s", "segments_per_step",
                             "plain_fp64_per_cone", "speedup_vs_plain", "error_vs_oracle", "tuning", "roofline",
                             "clocks", "config", "gpu_launches"])
    adj = _sub_line(["--workload", "adjoint_256", "--with-backward", "--compact", "--no-sub",
                     "--steps", str(steps), "--warmup", str(warmup)])
    if "error" not in adj:
        adj = _compact(adj, ["value", "unit", "ms_per_step", "segments_per_step", "backward",
                             "error_vs_oracle", "map_statistics", "gradient_vs_oracle", "clocks", "config"])
    return {"amr_256": amr, "batch64": bat, "adjoint_256": adj,
            "note": f"each workload run by this script in a child process (--workload NAME --steps {steps} "
                    f"--warmup {warmup}; the adjoint with --with-backward), condensed"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="prod_512")
    ap.add_argument("--fp64-dda", action="store_true", help="plain FP64 walk instead of the FP32 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--with-backward", action="store_true",
                    help="also time rr_trace_backward (dL/dPhi of a squared-distance loss) per pass")
    ap.add_argument("--compact", action="store_true",
                    help="skip the side measurements (other forms, map statistics) and use a small oracle sample")
    ap.add_argument("--no-sub", action="store_true",
                    help="do not run the adaptive-mesh, batched and differentiation workloads after the main one")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="compute each step's records and trace it in order on one stream (one record buffer)")
    ap.add_argument("--amr-group", type=int, default=4,
                    help="adaptive mesh: steps traced per launch (rr_amr_trace_steps; a whole-mesh leaf-record "
                         "buffer per step of a group, two sets); 1: one rr_amr_trace_step per step")
    ap.add_argument("--group", type=int, default=16,
                    help="uniform grid: steps traced per launch (rr_trace_steps on box-local records of each "
                         "step's footprint); 1: one rr_trace_step per step on whole-grid records")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload.startswith("amr_"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the production "
                              "uniform workload; the AMR line carries its own oracle sample"}))
            return
        if rank == 0:
            run_amr(args, args.workload)
        return
    if args.workload == "batch64":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the production "
                              "workload; the batch workload is compared against plain per-cone launches"}))
            return
        w, steps = None, None
    else:
        w = synth.workload(args.workload)
        steps = synth.step_schedule(w.bundle.chi_s, w.nsteps, rescale=w.rescale) if w.nsteps > 1 else \
            [synth.Step(w.bundle.chi_s, 0.0, 1.0, 1.0)]

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w, steps)
        return
    if w is None:
        if rank == 0:
            run_batch(args)
        return

    import torch
    import paper_1601_02012_gb300 as rrp
    from paper_1601_02012_gb300 import build as rrbuild
    from paper_1601_02012_gb300 import shard

    rrbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    # one bundle; with several ranks each traces a band of its rows (whole ray
    # tiles) and the maps are gathered at the end of every pass
    y0, y1 = shard.band_rows(w.bundle.ny, rank, world)
    if y1 <= y0:
        raise SystemExit(f"rank {rank}: no rows of the {w.bundle.ny}-row bundle left for this rank")
    rows = None if world == 1 else (y0, y1)
    phi_host = synth.grf_phi_cached(w.grid.n[0], w.grid.box, w.seed)
    stream = torch.cuda.Stream(device=dev)
    phi = torch.from_numpy(phi_host).to(dev)
    rec = rrp.record_buffer(w.grid, device=dev)
    tr = rrp.Tracer(w.bundle, fp64_dda=args.fp64_dda, rows=rows)
    gd = rrp.grid_desc(w.grid)
    bboxes = [tr.footprint(w.grid, st.chi_a, st.chi_b) for st in steps]
    kappa = torch.empty((y1 - y0, w.bundle.nx), dtype=torch.float64, device=dev)
    kborn = torch.empty_like(kappa)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nst = len(steps)
    ev_tr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    ev_td = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nst)]
    whole = {}

    def gather():
        # the whole maps on every rank (one all-gather per map; nothing for one rank)
        if world > 1:
            whole["k"] = shard.gather_rows(kappa, w.bundle.ny, rank, world)
            whole["kb"] = shard.gather_rows(kborn, w.bundle.ny, rank, world)
        else:
            whole["k"], whole["kb"] = kappa, kborn

    side = None if args.no_pipeline else torch.cuda.Stream(device=dev, priority=-1)
    G = 1 if args.fp64_dda else max(1, min(args.group, 16))
    if G > 1:
        # box-local records need every step's (widened) footprint to be smaller
        # than the grid on every axis; otherwise whole-grid records, step by step
        pboxes = [tr.footprint(w.grid, st.chi_a, st.chi_b, pad=1) for st in steps]
        if any(bb[2 * a + 1] - bb[2 * a] >= int(w.grid.n[a]) for bb in pboxes for a in range(3)):
            G = 1
    if G > 1:
        # every step's records over its footprint box (widened by a point) in
        # a box-local buffer of its own; G steps per rr_trace_steps launch; the
        # records of group j + 1 on the side stream while group j is traced
        brecs = [rrp.box_record_buffer(bb, device=dev) for bb in pboxes]
        groups = [list(range(i, min(i + G, nst))) for i in range(0, nst, G)]
        ev_tr = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]
        ev_td = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in groups]

        def group_records(gi, b, s, field):
            for k in groups[gi]:
                tr.tidal_box(w.grid, field, brecs[k], pboxes[k], stream=s)

        def group_trace(gi, b, s):
            ks = groups[gi]
            tr.steps(w.grid, [brecs[k] for k in ks], [steps[k] for k in ks], boxes=[pboxes[k] for k in ks],
                     stream=s)
    else:
        # the records of step k + 1 on a side stream while step k is traced (two record buffers)
        recs = [rec] if args.no_pipeline else [rec, rrp.record_buffer(w.grid, device=dev)]

    def one_pass(src=None, timed_kernels=False):
        rrp.rr_reset(tr.ctx, stream)
        field = phi if src is None else src
        if G > 1:
            rrp.pipeline_steps(len(groups), lambda gi, b, s: group_records(gi, b, s, field), group_trace,
                               stream, side, 1 if args.no_pipeline else 2,
                               (ev_td, ev_tr) if timed_kernels else None)
        else:
            rrp.pipeline_steps(
                nst, lambda i, b, s: rrp.rr_tidal_tensor(gd, field, None, recs[b], tr.where, bboxes[i], s),
                lambda i, b, s: rrp.rr_trace_step(tr.ctx, gd, recs[b], steps[i].chi_a, steps[i].chi_b,
                                                  steps[i].scale, steps[i].a, s),
                stream, side, len(recs), (ev_td, ev_tr) if timed_kernels else None)
        rrp.rr_finalize(tr.ctx, kappa, kborn, stream)   # synchronises the stream
        gather()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_pass()
        segs = tr.segments()

        sampler = ClockSampler(_device_id(torch, dev))
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        times, trace_ms, tidal_ms = [], 0.0, 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one_pass(timed_kernels=True)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            trace_ms += sum(a.elapsed_time(b) for a, b in ev_tr)
            tidal_ms += sum(a.elapsed_time(b) for a, b in ev_td)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        clocks = sampler.stop()
        total_ms = sum(times)

        # the tidal kernel on the whole grid (its HBM roofline; not part of a pass)
        full_ms = []
        for _ in range(3):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rrp.rr_tidal_tensor(gd, phi, None, rec, tr.where, None, stream)
            e1.record(stream)
            e1.synchronize()
            full_ms.append(e0.elapsed_time(e1))

        # adjoint: dL/dPhi for L = ||kappa - 0.9 kappa||^2-like target, after a pass
        bwd = None
        grad_check = None
        if args.with_backward:
            gradbuf = rrp.grad_buffer(w.grid, device=dev)
            dphi = torch.zeros_like(phi)
            one_pass()
            dk = (0.2 * kappa).contiguous()
            bw_ms = []
            for _ in range(args.warmup + args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rrp.rr_trace_backward(tr.ctx, dk, None, gradbuf, dphi, None, stream)
                e1.record(stream)
                e1.synchronize()
                bw_ms.append(e0.elapsed_time(e1))
            bw = sum(bw_ms[args.warmup:]) / args.steps
            fw = total_ms / args.steps
            bwd = {"ms_per_step": bw, "segments_per_s": segs / (bw / 1e3), "backward_over_forward": bw / fw,
                   "note": "rr_trace_backward over all steps: zero the gradient records, the adjoint of "
                           "every step (warp sums added with FP64 atomics), the transposed stencils into dL/dPhi; "
                           "backward_over_forward against the forward pass of this line"}
            if world == 1 and not args.no_cpu_baseline:
                # the gradient against the FP64 oracle's: dL/dkappa, dL/dkborn non-zero on sampled
                # rays (the oracle's adjoint skips the others), dL/dPhi over the whole grid
                import oracle
                oracle.build()
                rng = np.random.default_rng(11)
                rids = rng.choice(w.bundle.nrays, 2000, replace=False)
                yk = np.zeros(w.bundle.nrays)
                yb = np.zeros(w.bundle.nrays)
                yk[rids] = rng.standard_normal(len(rids))
                yb[rids] = rng.standard_normal(len(rids))
                dphi.zero_()
                rrp.rr_trace_backward(tr.ctx, torch.from_numpy(yk).to(dev), torch.from_numpy(yb).to(dev),
                                      gradbuf, dphi, None, stream)
                stream.synchronize()
                got = dphi.cpu().numpy().astype(np.float64).ravel()
                t0 = time.perf_counter()
                want, _ = oracle.trace_adjoint(w.bundle, w.grid, steps, yk, yb)
                dto = time.perf_counter() - t0
                want = want.ravel()
                sup = want != 0.0
                rmsg = math.sqrt(float(np.mean(want[sup] ** 2)))
                grad_check = {"rays": len(rids), "l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                              "max_over_rms_support": float(np.abs(got - want).max() / rmsg),
                              "support_fraction": float(sup.mean()), "oracle_s": dto,
                              "note": "dL/dkappa and dL/dkborn standard normal on the sampled rays, zero "
                                      "elsewhere; dL/dPhi on every cell, GPU (FP32 walk, FP64 atomic sums) "
                                      "against the FP64 oracle's adjoint; max difference over the rms of the "
                                      "gradient on the cells it reaches"}
            del gradbuf

        # end to end through the public API with host buffers: the potential
        # streamed from pinned host memory step by step (rr_upload_box of each
        # step's footprint on a copy stream, two device buffers, overlapped
        # with the previous step), the pass, the maps gathered, D2H of both
        k_dev = whole["k"].clone()
        kb_dev = whole["kb"].clone()
        phi_pinned = torch.from_numpy(phi_host).pin_memory()
        k_host = torch.empty(tuple(whole["k"].shape), dtype=torch.float64).pin_memory()
        kb_host = torch.empty_like(k_host).pin_memory()
        bufs = [torch.zeros_like(phi) for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=dev)
        e2e_times = []
        h2d_bytes = 0
        for it in range(args.warmup + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            rrp.rr_reset(tr.ctx, stream)
            if G > 1:
                h2d_bytes = tr.trace_streamed(w.grid, phi_pinned, steps, rec, bufs, stream, copy_stream, pboxes,
                                              group=G, box_recs=brecs, rec_stream=side)
            else:
                h2d_bytes = tr.trace_streamed(w.grid, phi_pinned, steps, rec, bufs, stream, copy_stream, bboxes)
            rrp.rr_finalize(tr.ctx, kappa, kborn, stream)
            gather()
            k_host.copy_(whole["k"], non_blocking=True)
            kb_host.copy_(whole["kb"], non_blocking=True)
            stream.synchronize()
            if it >= args.warmup:
                e2e_times.append(time.perf_counter() - t0)
        e2e_s = sum(e2e_times)
        e2e_diff = max(float((k_host.to(dev) - k_dev).abs().max()), float((kb_host.to(dev) - kb_dev).abs().max()))
        del bufs
        total_ms, segs_all, e2e_s = combine_over_ranks(dist, dev, total_ms, segs, e2e_s)

        # kappa for several source distances from one pass (Eqs. Isources,
        # Isources1): the moments form with snapshots at step boundaries, against
        # one ordinary pass per source distance
        sources = None
        shear = None
        method_a = None
        generic = None
        if world == 1 and not args.compact:
            box = (pboxes, brecs) if G > 1 else None
            sources = _source_redshifts(rrp, torch, w, steps, gd, phi, rec, bboxes, stream, flush, box=box)
            # the shear in the same walk (Eqs. gamma1, gamma2)
            shear = _shear_form(rrp, torch, w, steps, gd, phi, rec, bboxes, stream, flush,
                                trace_ms / args.steps, box=box)
            one_pass()
            ks, kbs = shear.pop("kappa"), shear.pop("kborn")
            rms = float(torch.sqrt(torch.mean(kappa * kappa)))
            shear["kappa_max_over_rms_vs_default_form"] = float((ks - kappa).abs().max()) / rms
            del ks, kbs
            # Method A (Eq. kappa2) in the same configuration
            method_a = _method_a_form(rrp, torch, w, steps, gd, phi, bboxes, stream, flush,
                                      total_ms / args.steps, kappa)
            # generic K.Q integrals (the ISW set-up of Sec. 6)
            generic = _generic_form(rrp, torch, w, steps, gd, phi, bboxes, stream, flush, total_ms / args.steps)
        peak = _fp32_peak(rrp, torch, dev, stream) if rank == 0 else None

    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return

    peaks, peak_kind = _peaks()
    nlaunch = len(groups) if G > 1 else nst      # trace launches per pass
    per_launch_s = trace_ms / args.steps / nlaunch / 1e3
    segs_per_launch = segs / nlaunch
    gather_gbs = segs_per_launch * BYTES_PER_SEGMENT / per_launch_s / 1e9
    alu_gops = segs_per_launch * ALU_OPS_PER_SEGMENT / per_launch_s / 1e9
    alu_peak = peak["lane_fma_per_s"] / 1e9
    tidal_points = sum((b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4]) for b in bboxes)
    h = _src_hash("trace.cu", "walk.cuh")
    traffic = TRACE_TRAFFIC.get((h, w.name, G))
    wi = TRACE_WARP_INSTRUCTIONS.get((h, w.name, G))
    sm_mhz = (clocks or {}).get("sm_mhz") or MAX_SM_MHZ
    issue_peak = 4.0 * peak["sms"] * sm_mhz * 1e6          # warp instructions per second
    issue = None
    if wi is not None:
        issue = {"warp_instructions_per_segment": wi, "achieved_per_s": wi * segs_per_launch / per_launch_s,
                 "peak_per_s": issue_peak, "frac": wi * segs_per_launch / per_launch_s / issue_peak}
    value = segs_all * args.steps / (total_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w, nst),
        # how this arm runs the workload (the config above is the workload alone, the
        # same in the reference arm's line)
        "execution": {"form": "fp64 walk" if args.fp64_dda else "fp32 walk, Kahan sums",
                      "pipeline": _PIPELINE_NOTE[bool(args.no_pipeline) if G == 1 else
                                                 ("grouped_in_order" if args.no_pipeline else "grouped")],
                      "steps_per_launch": G,
                      "records": ("each step's footprint box (widened by a point), box-local"
                                  if G > 1 else "whole grid, each step's footprint rewritten"),
                      "parallelism": f"one bundle, its rows split over {world} GPU(s) in "
                                     "whole ray tiles; maps all-gathered every pass"},
        "rays_per_s": w.bundle.nrays * args.steps / (total_ms / 1e3),
        "segments_per_step": segs_all,
        "roofline": {
            "bound": "alu", "achieved": alu_gops, "peak": alu_peak, "unit": "Gop/s", "frac": alu_gops / alu_peak,
            "traffic": traffic, "kernel": "trace_steps_kernel<trilinear, flat>" if G > 1 else "trace_kernel<trilinear,float>",
            "algorithmic_ops_per_segment": ALU_OPS_PER_SEGMENT,
            "algorithmic_ops_per_launch": segs_per_launch * ALU_OPS_PER_SEGMENT,
            "mean_launch_ms": per_launch_s * 1e3,
            "note": f"FP32 lane operations the method needs per trilinear segment ({ALU_OPS_PER_SEGMENT}: "
                    "exit face, entry point, the projection of the 4 new corner records, the line cubic and "
                    "the kernel integrals of both channels, the compensated sums, the crossing) x segments "
                    "per launch / mean launch time (CUDA events, all launches of the timed passes); peak: "
                    "the packed FFMA2 lane rate measured in this run (rr_fp32_peak); traffic: DRAM bytes "
                    "read + written per launch (ncu), null when the kernel source differs from the captured one",
            "fp32_peak": {"lane_fma_per_s": peak["lane_fma_per_s"], "scalar_ffma_per_s": peak["scalar_ffma_per_s"],
                          "nominal_lane_fma_per_s": peak["sms"] * 128 * MAX_SM_MHZ * 1e6,
                          "kind": "measured in this run"},
            "issue": issue,
            "gather": {"achieved": gather_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": gather_gbs / peaks["hbm_gbs"],
                       "note": f"logical gather bytes ({BYTES_PER_SEGMENT} B per segment: 8 vertex records) / "
                               f"launch time against the {peak_kind} HBM copy bandwidth; served by L1 and L2 "
                               "(10^2-10^4 rays cross each cell), not by DRAM: above 1 by cache reuse"},
        },
        "kernels_ms_per_step": {"trace": trace_ms / args.steps, "tidal": tidal_ms / args.steps,
                                "note": _SPLIT_NOTE[bool(args.no_pipeline)],
                                "tidal_points_per_step": tidal_points},
        "tidal_roofline": {"bound": "hbm",
                           "achieved": w.grid.ncells * 36 / (min(full_ms) / 1e3) / 1e9,
                           "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": w.grid.ncells * 36 / (min(full_ms) / 1e3) / 1e9 / peaks["hbm_gbs"],
                           "ms_full_grid": min(full_ms),
                           "per_step_footprint_gbs": tidal_points * 36 / (tidal_ms / args.steps / 1e3) / 1e9,
                           "note": "whole-grid launch, 36 B per point (4 B potential read, 32 B record written); "
                                   "the per-step footprint launches are small and latency-bound"},
        "backward": bwd,
        "gradient_vs_oracle": grad_check,
        "e2e": {"value": segs_all * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d_bytes),
                "d2h_bytes_per_step": int(k_host.numel() * 8 * 2),
                "max_abs_diff_vs_device_maps": e2e_diff,
                "note": "host potential (pinned, the whole field) streamed per step: rr_upload_box of the "
                        "step's footprint plus the stencil reach on a copy stream into one of two device "
                        "buffers, overlapped with the previous step; both whole maps read back (rank 0's "
                        "bytes; every rank streams its own footprints)"},
        "source_redshifts": sources,
        "shear": shear,
        "method_a": method_a,
        "generic_isw": generic,
        "gpu_launches": args.steps * (nst + nlaunch + 1),
        "clocks": clocks,
        "trace_src": h,
    }

    if world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle on the host cores, on a bounded sample of the same
        # workload; the sampled rays also give the error of the GPU map
        threads = os.cpu_count() or 1
        budget = 4.0 if args.compact else 12.0
        H, d = _oracle_fields(w.grid, phi_host)
        rng = np.random.default_rng(4321)
        rids = rng.choice(w.bundle.nrays, 256, replace=False)
        res, dt = _oracle_sample(w.bundle, w.grid, H, d, steps, rids, threads)
        n2 = int(min(w.bundle.nrays, max(256, 256 * budget / max(dt, 1e-3))))
        rids2 = rng.choice(w.bundle.nrays, n2, replace=False)
        res2, dt2 = _oracle_sample(w.bundle, w.grid, H, d, steps, rids2, threads)
        # one thread, on a sample sized for ~budget / 3 s
        n1 = int(min(w.bundle.nrays, max(16, 256 * (budget / 3.0) / max(dt * threads, 1e-3))))
        rids1 = rng.choice(w.bundle.nrays, n1, replace=False)
        res1, dt1 = _oracle_sample(w.bundle, w.grid, H, d, steps, rids1, 1)
        line["cpu_baseline"] = {
            "value": float(res2.nseg.sum()) / dt2, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n2} random rays of the bundle through all {nst} steps ({dt2:.1f} s); "
                      "tidal centres of the full grid computed once outside the timing",
            "single_thread": {"value": float(res1.nseg.sum()) / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} random rays through all {nst} steps ({dt1:.1f} s)"},
            "cpu_model": _cpu_model(), "host_threads": threads}
        kg = whole["k"].cpu().numpy().ravel()
        kbg = whole["kb"].cpu().numpy().ravel()
        allr = np.concatenate([rids, rids2, rids1])
        ko = np.concatenate([res.kappa, res2.kappa, res1.kappa])
        kbo = np.concatenate([res.kborn, res2.kborn, res1.kborn])
        rms, rmsb = math.sqrt(float(np.mean(ko ** 2))), math.sqrt(float(np.mean(kbo ** 2)))
        per_ray = torch.zeros(w.bundle.nrays, dtype=torch.int32, device=dev)
        tr.segments(per_ray=per_ray)
        torch.cuda.synchronize()
        nseg_gpu = per_ray.cpu().numpy().view(np.uint32).astype(np.int64)
        nseg_ora = np.concatenate([res.nseg, res2.nseg, res1.nseg])
        line["error_vs_oracle"] = {
            "rays": int(len(allr)),
            "kappa_max_over_rms": float(np.abs(kg[allr] - ko).max() / rms),
            "kborn_max_over_rms": float(np.abs(kbg[allr] - kbo).max() / rmsb),
            "segments_per_ray_gpu": segs / w.bundle.nrays,
            "segments_sampled_rays_gpu": int(nseg_gpu[allr].sum()),
            "segments_sampled_rays_oracle": int(nseg_ora.sum()),
            "segments_rel_diff": float(abs(int(nseg_gpu[allr].sum()) - int(nseg_ora.sum())) / nseg_ora.sum()),
        }
        if not args.compact or w.name == "adjoint_256":
            # map statistics: a contiguous patch of the map (its centre quarter per
            # side) traced by the oracle through all steps, P(ell) and PDF vs the GPU's
            # (the one-step differentiation workload's patch takes the oracle ~3 s)
            from paper_1601_02012_gb300 import mapstats
            px = min(512, w.bundle.nx)
            py = min(512, w.bundle.ny)
            x0, yy0 = (w.bundle.nx - px) // 2, (w.bundle.ny - py) // 2
            iy, ix = np.meshgrid(np.arange(yy0, yy0 + py), np.arange(x0, x0 + px), indexing="ij")
            prids = (iy * w.bundle.nx + ix).ravel()
            t0 = time.perf_counter()
            pres, _ = _oracle_sample(w.bundle, w.grid, H, d, steps, prids, threads)
            dtp = time.perf_counter() - t0
            fx = w.bundle.fov_x * (px - 1) / max(w.bundle.nx - 1, 1)
            fy = w.bundle.fov_y * (py - 1) / max(w.bundle.ny - 1, 1)
            line["map_statistics"] = {
                "patch": f"{px}x{py} rays at the map centre ({fx * 180 / math.pi:.3f} x "
                         f"{fy * 180 / math.pi:.3f} deg), all {nst} steps, oracle {dtp:.1f} s",
                "kappa": mapstats.compare(kg[prids].reshape(py, px), pres.kappa.reshape(py, px), fx, fy),
                "kborn": mapstats.compare(kbg[prids].reshape(py, px), pres.kborn.reshape(py, px), fx, fy),
                "definition": "P(ell): 20 log bins of ell = 2 pi m / Upsilon, largest relative bin difference; "
                              "PDF: 100 bins over +-5 sigma of the oracle map, L1 distance",
            }
            # the same statistics for the FP32 walk without compensated sums (one pass)
            trp = rrp.Tracer(w.bundle, plain_sums=True)
            with torch.cuda.stream(stream):
                for i, st in enumerate(steps):
                    rrp.rr_tidal_tensor(gd, phi, None, rec, trp.where, bboxes[i], stream)
                    rrp.rr_trace_step(trp.ctx, gd, rec, st.chi_a, st.chi_b, st.scale, st.a, stream)
                kp, kbp = trp.finalize(stream=stream)
            trp.close()
            kpg, kbpg = kp.cpu().numpy().ravel(), kbp.cpu().numpy().ravel()
            line["map_statistics"]["plain_fp32_sums"] = {
                "kappa": mapstats.compare(kpg[prids].reshape(py, px), pres.kappa.reshape(py, px), fx, fy),
                "kborn": mapstats.compare(kbpg[prids].reshape(py, px), pres.kborn.reshape(py, px), fx, fy),
                "note": "the same pass with uncompensated FP32 sums within and across steps (RR_PLAIN_SUMS)",
            }
    if world == 1 and not args.no_sub:
        # free this workload's device memory before the child processes run
        tr.close()
        del rec, phi, kappa, kborn, flush, whole, k_dev, kb_dev
        torch.cuda.empty_cache()
        line["other_workloads"] = _other_workloads(3, 3)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
