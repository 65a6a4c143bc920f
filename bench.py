#!/usr/bin/env python
"""Benchmark of the UniMGS hot path on one GB300: per-frame proxy deformation
+ single-pass mesh/3DGS rasterization at 1080p.

Workload (synthetic, seeded): 1,000,000 Gaussians with SH degree 3 on a noisy
unit-sphere shell, a 200,000-face torus (30% of faces with alpha U[0.2,0.8])
intersecting it, a 20,480-face proxy icosphere displaced every frame by a sum
of 8 sinusoids (amplitude 0.1); Gaussians bound to the proxy once (BBX mode,
100 cameras), then every step = one frame:
    umgs_deform (per-face gradients, per-vertex polar/log table, Eq. 12-13)
    umgs_render (projection, triangle setup, binning into tile lists, composite).

One JSON line on rank 0.  `--impl reference` times the CPU oracle instead
(a bounded sample of the same frame per step, extrapolated to frames/s).
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "single-pass mesh+3DGS frames/s at 1080p (fwd, fwd+bwd), % roofline vs plain form"
WORKLOAD = "1080p deform+render: 1M Gaussians SH3 + 200k-face torus, 20,480-face proxy, 1 view"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="umgs", choices=["umgs", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-spatial-order", action="store_true",
                   help="keep the Gaussians in the order generated instead of umgs_spatial_order's")
    p.add_argument("--n-gauss", type=int, default=1_000_000)
    p.add_argument("--no-forms", action="store_true", help="skip the multi-view / differentiable / mixed forms")
    p.add_argument("--forms", default="all",
                   help="comma list of the forms to run: multiview, closeup, differentiable (with soft edges), mixed, nested")
    p.add_argument("--forms-only", action="store_true",
                   help="run the selected forms only (no 1080p frame) and print their JSON")
    return p.parse_args()


def aggregate_ranks(ms_local, steps, world, device=None):
    """Whole-job timing over `world` replicas that each timed `steps` frames:
    the slowest rank's time (all_reduce MAX) and the throughput of all ranks
    together, steps * world frames in that time."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_local = float(t.item())
    return ms_local, steps * world / (ms_local / 1e3)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------------------
# clocks sampling during the timed region

class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # the timed region starts once the sampler has written its first row
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# workload

def build_workload(n_gauss, frames):
    from paper_2601_19233_gb300 import scenes
    sc = scenes.config1(n_gauss=n_gauss)
    disp = [scenes.displace(sc.proxy_verts, sc.extra["sinusoids"], f) for f in range(frames)]
    return sc, np.stack(disp, 0)


def stage_names():
    return ["project_gaussians", "setup_triangles", "scan", "scatter", "sort", "composite", "deform_faces",
            "deform_vertices", "deform_gaussians", "bind_grid", "bind_raycast", "bind_nearest",
            "backward_composite", "backward_project", "shade_gaussians", "s15"]


def run_umgs(args, rank, world, local_rank):
    # the oracle's process pool starts before the first CUDA call (spawned
    # workers, rank 0 of a single-GPU run only): the 4K crops of the
    # mixed-precision form render on the host cores while the GPU works
    pool = crops = None
    workers = max(1, host_cores() - 2)
    which = FORMS if args.forms == "all" else tuple(x.strip() for x in args.forms.split(","))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(workers)
        if not args.no_forms and "mixed" in which:
            crops = CropOracle(pool, bands=max(1, workers // 4))
    import torch
    from paper_2601_19233_gb300 import build, umgs
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    K, Wm = args.steps, args.warmup
    if args.forms_only:
        dev = torch.device("cuda", local_rank)
        ctx = umgs.Context(local_rank)
        res = {"forms": run_forms(ctx, dev, max(3, min(20, K)), crops, which)}
        if pool is not None:
            pool.close()
            pool.join()
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    nframes = 100
    sc, disp = build_workload(args.n_gauss, nframes)
    dev = torch.device("cuda", local_rank)
    ctx = umgs.Context(local_rank)
    g = umgs.gaussians_to_device(sc.gaussians, dev)
    # the model stored in spatial order once, when it is loaded (before the
    # binding): umgs_spatial_order's Morton order of the means, every
    # per-Gaussian array gathered by it
    order = "index order (as generated)"
    if not args.no_spatial_order:
        perm = umgs.spatial_order(ctx, g.means).long()
        g = umgs.DevGaussians(*(x.index_select(0, perm).contiguous() for x in (g.means, g.quats, g.scales,
                                                                               g.opacities, g.sh)), g.sh_degree)
        del perm
        order = "spatial: Morton order of the means (umgs_spatial_order), applied once at load"
    mesh = umgs.mesh_to_device(sc.meshes[0], dev)
    PV = torch.as_tensor(sc.proxy_verts).to(dev)
    PF = torch.as_tensor(sc.proxy_faces).to(dev)
    Vd_all = torch.as_tensor(disp).to(dev)  # [frames, nv, 3], resident before timing
    cam = sc.cameras[0]
    H, W = cam.height, cam.width

    # bind once (timed separately)
    torch.cuda.synchronize()
    t0 = time.time()
    face, bary, _, _, nfb = umgs.bind(ctx, g, PV, PF, sc.bind_cameras, mode=umgs.BIND_BBX)
    torch.cuda.synchronize()
    bind_s = time.time() - t0
    bind_info = "umgs_bind BBX k=3, %d cameras, %d fallback targets" % (len(sc.bind_cameras), nfb)
    # the binding regrouped per Gaussian into its distinct proxy vertices and
    # weights, packed (CSR; once, like the binding itself); every step deforms
    # through it
    t0 = time.time()
    boff, bent = umgs.binding_csr(ctx, face, bary, PF, PV.shape[0])
    torch.cuda.synchronize()
    compact_s = time.time() - t0

    n = g.n
    mu2 = torch.empty((n, 3), device=dev)
    cov2 = torch.empty((n, 6), device=dev)
    out = torch.empty((1, H, W, 4), device=dev)
    gdef = umgs.DevGaussians(mu2, g.quats, g.scales, g.opacities, g.sh, g.sh_degree, cov3d=cov2)
    frame = umgs.Frame(ctx)
    # one synchronous render sizes the frame; the timed steps render
    # asynchronously (no host read-back) into a pair capacity of 1.25x that
    # count, and umgs_frame_check after the region confirms no step overflowed
    umgs.deform_csr(ctx, g, boff, bent, PV, Vd_all[0], PF, out=(mu2, cov2, None))
    umgs.render(ctx, gdef, [mesh], [cam], umgs.render_opts(16), out=out, frame=frame)
    frame.reserve(int(frame.counts()[0] * 1.25) + 4096)
    opts = umgs.render_opts(16, asynchronous=True)

    def step(f, vd=None):
        umgs.deform_csr(ctx, g, boff, bent, PV, Vd_all[f % nframes] if vd is None else vd, PF,
                            out=(mu2, cov2, None))
        umgs.render(ctx, gdef, [mesh], [cam], opts, out=out, frame=frame)

    for f in range(Wm):
        step(f)
    torch.cuda.synchronize()
    frame.check()
    ctx.sync()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    # the timed region runs without per-stage events (they would sit between
    # the kernels and stop each kernel from being scheduled during its
    # predecessor); the stage breakdown comes from a separate profiled pass
    clocks = ClockSampler(local_rank)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = umgs.kernel_launches()
    e0.record()
    for f in range(K):
        step(Wm + f)
    e1.record()
    launches = umgs.kernel_launches() - launches0
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    frame.check()
    ms_total = e0.elapsed_time(e1)
    umgs.profile_enable(ctx, True)
    for f in range(min(K, 100)):
        step(Wm + f)
    torch.cuda.synchronize()
    stage_ms, stage_n = umgs.profile_read(ctx)
    umgs.profile_enable(ctx, False)
    ms_total, value = aggregate_ranks(ms_total, K, world, dev)
    ms_step = ms_total / K
    # counts of the last timed frame's input, from a synchronous render of it
    umgs.render(ctx, gdef, [mesh], [cam], umgs.render_opts(16), out=out, frame=frame)
    nkeys, ntiles = frame.counts()

    # forward + backward: the render keeps its backward state and the gradient
    # of a fixed synthetic upstream dL/d(rgb, T) is propagated to the deformed
    # Gaussians (means, cov3d, opacity, SH) and the mesh (vertices, colours, alpha)
    opts_s = umgs.render_opts(16, save=True, asynchronous=True)
    gen = torch.Generator(device=dev).manual_seed(1)
    dl = torch.randn((1, H, W, 4), generator=gen, device=dev) * 1e-3

    def step_fb(f):
        step_deform(f)
        umgs.render(ctx, gdef, [mesh], [cam], opts_s, out=out, frame=frame)
        return umgs.render_backward(ctx, frame, gdef, [mesh], dl)

    def step_deform(f):
        umgs.deform_csr(ctx, g, boff, bent, PV, Vd_all[f % nframes], PF, out=(mu2, cov2, None))

    for f in range(max(2, Wm)):
        step_fb(f)
    torch.cuda.synchronize()
    Kb = max(5, K // 2)
    b0 = torch.cuda.Event(enable_timing=True)
    b1 = torch.cuda.Event(enable_timing=True)
    b0.record()
    for f in range(Kb):
        step_fb(f)
    b1.record()
    torch.cuda.synchronize()
    frame.check()
    fb_ms = b0.elapsed_time(b1) / Kb
    umgs.profile_read(ctx)
    umgs.profile_enable(ctx, True)
    for f in range(min(Kb, 50)):
        step_fb(f)
    torch.cuda.synchronize()
    fb_stage_ms, fb_stage_n = umgs.profile_read(ctx)
    umgs.profile_enable(ctx, False)

    # end to end: every step uploads its proxy frame from pinned host memory
    # and reads its image back into pinned host memory.  The readback of
    # step f runs on a copy stream while step f + 1 computes (two image
    # buffers; a buffer is rendered again only after its copy has finished);
    # the region ends when the last copy has landed.
    host_vd = torch.as_tensor(disp).pin_memory()
    host_out = [torch.empty((1, H, W, 4), dtype=torch.float32).pin_memory() for _ in range(2)]
    outs = [out, torch.empty_like(out)]
    vd_dev = torch.empty_like(Vd_all[0])
    comp = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream()
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]

    def step_e2e(f):
        b = f % 2
        if f >= 2:
            comp.wait_event(copied[b])
        vd_dev.copy_(host_vd[f % nframes], non_blocking=True)
        umgs.deform_csr(ctx, g, boff, bent, PV, vd_dev, PF, out=(mu2, cov2, None))
        umgs.render(ctx, gdef, [mesh], [cam], opts, out=outs[b], frame=frame)
        rendered[b].record(comp)
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(rendered[b])
            host_out[b].copy_(outs[b], non_blocking=True)
            copied[b].record(copy_s)

    for f in range(2):
        step_e2e(f)
    torch.cuda.synchronize()
    Ke = max(5, K // 2)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record()
    for f in range(Ke):
        step_e2e(f)
    comp.wait_event(copied[(Ke - 1) % 2])
    a1.record()
    torch.cuda.synchronize()
    frame.check()
    e2e_ms = a0.elapsed_time(a1) / Ke
    h2d = int(host_vd[0].numel() * 4)
    d2h = int(host_out[0].numel() * 4)

    # fragment counts of the last frame: N_alg (evaluations: (pixel, record)
    # pairs whose footprint holds the pixel, up to termination, counted on the
    # device) and the tile-granularity pairs (list length x pixels of the tile)
    fstats = frame.stats()
    evals = fstats["gaussian_evals"] + fstats["triangle_evals"]
    tptr, _, _ = frame.lists()
    tl = (tptr[1:] - tptr[:-1]).double()
    ts = 16
    tx_n = (W + ts - 1) // ts
    tix = torch.arange(tl.numel(), device=dev)
    tw = torch.clamp(W - (tix % tx_n) * ts, max=ts).double()
    th = torch.clamp(H - (tix // tx_n) * ts, max=ts).double()
    tile_pairs = int((tl * tw * th).sum().item())

    # mesh-added vs Gaussians-only (and mesh-only) render time of the same frame
    def t_render(gg, mm, k=max(5, K // 4)):
        for _ in range(3):
            umgs.render(ctx, gg, mm, [cam], opts, out=out, frame=frame)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record()
        for _ in range(k):
            umgs.render(ctx, gg, mm, [cam], opts, out=out, frame=frame)
        r1.record()
        torch.cuda.synchronize()
        frame.check()
        return r0.elapsed_time(r1) / k
    render_ms = {"gaussians_and_mesh": round(t_render(gdef, [mesh]), 4),
                 "gaussians_only": round(t_render(gdef, []), 4),
                 "mesh_only": round(t_render(None, [mesh]), 4)}

    names = stage_names()
    stages = {names[k]: {"ms_per_launch": stage_ms[k] / stage_n[k], "launches": int(stage_n[k])}
              for k in range(16) if stage_n[k] > 0}
    # algorithmic binding bytes per Gaussian: its offset and its packed entries
    bind_bytes = 4.0 + 8.0 * float(bent.shape[0]) / n
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = roofline(stages, nkeys, n, sc, clk, fstats, ms_step, bind_bytes, num_sms)
    comp_ms = stages["composite"]["ms_per_launch"] if "composite" in stages else float("nan")
    frags = {"n_alg": int(evals), "gaussian_evals": fstats["gaussian_evals"],
             "triangle_evals": fstats["triangle_evals"], "mfragments_per_s": round(evals / comp_ms / 1e3, 1),
             "tile_pairs": tile_pairs, "tile_pairs_over_n_alg": round(tile_pairs / max(evals, 1), 3),
             "fp64_conics": fstats["fp64_conics"]}
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "frames/s",
        "fwd_bwd_frames_per_s": round(1e3 / fb_ms * world, 3), "n_gpus": world, "steps": K,
        "warmup": Wm, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "resolution": [W, H], "gaussians": n, "sh_degree": 3,
                   "triangles": int(sc.meshes[0].nf), "proxy_faces": int(sc.proxy_faces.shape[0]),
                   "binding": bind_info, "gaussian_order": order, "tile": 16, "keys_per_frame": int(nkeys),
                   "l2": "inputs larger than L2 (Gaussians 236 MB per frame)", "parallelism": "replicas"},
        "e2e": {"value": round(1e3 / e2e_ms * world, 3), "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "stages_ms": {k: round(v["ms_per_launch"], 4) for k, v in stages.items()},
        "fwd_bwd": {"value": round(1e3 / fb_ms * world, 3), "unit": "frames/s", "ms_per_step": round(fb_ms, 4),
                    "steps": Kb, "backward_stages_ms": {names[k]: round(fb_stage_ms[k] / fb_stage_n[k], 4)
                                                        for k in (12, 13) if fb_stage_n[k] > 0}},
        "bind_s": round(bind_s, 3),
        "binding_compact_s": round(compact_s, 4),
        "fragments": frags,
        "render_ms": render_ms,
        "roofline": roof,
        "clocks": clk,
    }
    if not args.no_forms:
        res["forms"] = run_forms(ctx, dev, min(20, max(3, K // 6)), crops, which)
    if pool is not None:
        res["cpu_baseline"] = cpu_baseline(pool, workers, sc)
        pool.close()
        pool.join()
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# Algorithmic work of one compositor evaluation (a (pixel, record) pair of
# N_alg), in lane operations: a Gaussian is 12 FP32 operations and one
# exponential on the special-function unit (Eq. 1-2); a triangle is 12
# sample/edge tests (an int64 add and compare each: 2 operations), about 25
# FP32 operations of attribute interpolation and entity blending (Eq. 7-9)
# and one reciprocal.
G_ALU, G_SFU = 12, 1
T_ALU, T_SFU = 12 * 2 + 25, 1
ALU_LANES, SFU_LANES = 128, 16   # per SM and clock (FP32/INT32 lanes; special-function lanes)


def roofline(stages, nkeys, n, sc, clk, fstats, ms_step, bind_bytes, num_sms):
    """Roofline of the dominant stage, plus HBM figures of the streaming stages.

    composite: bound by instruction issue on the ALU (FP32/INT32) lanes or by
    the special-function unit, whichever needs longer for the algorithmic work
    of its N_alg evaluations (counted on the device per record kind, see
    G_ALU..T_SFU), at the sampled SM clock and the device's SM count.
    Streaming stages: algorithmic bytes per Gaussian / triangle / key against
    the measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs).
    """
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    hsrc = "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    ng, nt = n, sc.meshes[0].nf
    npf, npv = int(sc.proxy_faces.shape[0]), int(sc.proxy_verts.shape[0])
    alg = {  # algorithmic bytes per launch
        "project_gaussians": ng * (12 + 28 + 4 + 36 + 16),
        "shade_gaussians": ng * (192 + 12 + 16 + 12),
        "setup_triangles": nt * (12 + 16 + 160 + 16) + sc.meshes[0].nv * 28,
        "deform_gaussians": ng * (bind_bytes + 40 + 36),
        "deform_faces": npf * (12 + 72) + npv * 40,
        "deform_vertices": npv * (40 + 24 + 48),
        # binning (stages scan + scatter + sort): per record its info read,
        # (depth, id) written, one read+write of it (a single sort pass), a
        # count and an offset written; per tile-list entry its id written
        "binning": (ng + nt) * (16 + 8 + 16 + 8) + nkeys * 4,
    }
    stages = dict(stages)
    if all(k in stages for k in ("scan", "scatter", "sort")):
        stages["binning"] = {"ms_per_launch": sum(stages[k]["ms_per_launch"] for k in ("scan", "scatter", "sort"))}
    hbm_stages = {}
    for k, b in alg.items():
        if k in stages:
            t = stages[k]["ms_per_launch"] * 1e-3
            hbm_stages[k] = {"achieved_gbs": round(b / t / 1e9, 1), "frac": round(b / t / 1e9 / hbm, 4)}
    for k in ("scan", "scatter", "sort"):
        stages.pop(k, None)
    dom = max(stages, key=lambda k: stages[k]["ms_per_launch"])
    t = stages[dom]["ms_per_launch"] * 1e-3
    mhz = clk.get("sm_mhz") or 2070.0
    alu_peak = ALU_LANES * num_sms * mhz * 1e6      # lane operations / s
    sfu_peak = SFU_LANES * num_sms * mhz * 1e6
    eg, et = fstats["gaussian_evals"], fstats["triangle_evals"]
    alu_ops = G_ALU * eg + T_ALU * et
    sfu_ops = G_SFU * eg + T_SFU * et
    t_comp = max(alu_ops / alu_peak, sfu_ops / sfu_peak)
    # whole frame: sum of the per-stage lower bounds against the step time
    t_bound = sum(b / (hbm * 1e9) for k, b in alg.items() if k in stages) + t_comp
    frame = {"bound_ms": round(t_bound * 1e3, 4), "ms_per_step": round(ms_step, 4),
             "frac": round(t_bound * 1e3 / ms_step, 4)}
    if dom == "composite":
        ach = alu_ops / t / 1e12
        return {"bound": "alu", "stage": dom, "achieved": round(ach, 3), "peak": round(alu_peak / 1e12, 2),
                "unit": "Tops/s", "frac": round(ach * 1e12 / alu_peak, 4),
                "traffic": kernel_traffic("composite_kernel<16, 0, 0>"),
                "sfu": {"achieved": round(sfu_ops / t / 1e12, 3), "peak": round(sfu_peak / 1e12, 3),
                        "unit": "Tops/s", "frac": round(sfu_ops / t / sfu_peak, 4)},
                "bound_us": round(t_comp * 1e6, 2), "measured_us": round(t * 1e6, 2),
                "evaluations": {"gaussian": int(eg), "triangle": int(et)},
                "work": "lane ops per evaluation: Gaussian %d ALU + %d SFU, triangle %d ALU + %d SFU"
                        % (G_ALU, G_SFU, T_ALU, T_SFU),
                "peak_source": "%d ALU / %d SFU lanes x %d SMs at %.0f MHz (sampled)"
                               % (ALU_LANES, SFU_LANES, num_sms, mhz),
                "hbm_stages": hbm_stages, "hbm_peak_gbs": hbm, "hbm_peak_source": hsrc, "frame": frame}
    b = alg.get(dom)
    ach = b / t / 1e9 if b else None
    return {"bound": "hbm", "stage": dom, "achieved": ach and round(ach, 1), "peak": hbm, "unit": "GB/s",
            "frac": ach and round(ach / hbm, 4), "traffic": None, "peak_source": hsrc, "hbm_stages": hbm_stages,
            "frame": frame}


def kernel_traffic(kernel):
    """DRAM bytes per launch of `kernel` at the bench workload, from the ncu
    figures kept in profiles/traffic.txt (one line per kernel: name, bytes per
    launch, SHA-256 of the kernel's sources at capture time); None when the
    sources have changed since, or no figure was kept."""
    import hashlib
    try:
        for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
            if line.startswith("#") or "\t" not in line:
                continue
            name, nbytes, files, sha = line.rstrip("\n").split("\t")
            if name != kernel:
                continue
            h = hashlib.sha256()
            for f in files.split(","):
                h.update(open(os.path.join(ROOT, "paper_2601_19233_gb300", "csrc", f), "rb").read())
            return int(nbytes) if h.hexdigest() == sha else None
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------
# the other forms, each next to the plain fp32 forward on the same GPU, and the
# separate-pass baseline on a nested-transparency scene

def _time(fn, steps, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


FORMS = ("multiview", "closeup", "differentiable", "mixed", "nested")


def run_forms(ctx, dev, steps, crops=None, which=FORMS):
    import torch
    from paper_2601_19233_gb300 import scenes, umgs
    forms = {}
    if "multiview" in which:
        # config 2: 64 orbit views of 800x800, clustered Gaussians (uneven tile load)
        sc = scenes.config2()
        g = umgs.gaussians_to_device(sc.gaussians, dev)
        ms = [umgs.mesh_to_device(m, dev) for m in sc.meshes]
        nv = len(sc.cameras)
        out = torch.empty((nv, 800, 800, 4), device=dev)
        plain = umgs.render_opts(16)
        fr = umgs.Frame(ctx)
        t_plain = _time(lambda: umgs.render(ctx, g, ms, sc.cameras, plain, out=out, frame=fr), steps)
        evals_plain = fr.evaluations()
        # per-stage split of the plain render (a separate profiled pass)
        umgs.profile_read(ctx)
        umgs.profile_enable(ctx, True)
        for _ in range(3):
            umgs.render(ctx, g, ms, sc.cameras, plain, out=out, frame=fr)
        torch.cuda.synchronize()
        st_ms, st_n = umgs.profile_read(ctx)
        umgs.profile_enable(ctx, False)
        names = stage_names()
        mv_stages = {names[k]: round(st_ms[k] / st_n[k], 3) for k in range(16) if st_n[k] > 0}
        # the per-tile work split alone, at each length the autotuner tries
        split_ms = {str(sp): round(_time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, split=sp),
                                                             out=out, frame=fr), steps), 3)
                    for sp in (512, 1024, 2048)}
        best, t_tune = umgs.autotune(ctx, g, ms, sc.cameras, plain, out)
        fr2 = umgs.Frame(ctx)
        # the scene and cameras are the same every replay: pair capacity = the
        # sizing render's count (+ 4096), no 25% headroom
        gr = umgs.Graph(ctx, fr2, g, ms, sc.cameras, best, out, key_headroom=1.0)
        t_graph = _time(lambda: gr.launch(), steps)
        gr.check()
        forms["multiview_64x800"] = {
            "workload": "64 orbit views 800x800, 500k Gaussians SH3 (70% in 3 blobs) + 100k-face torus",
            "plain_views_per_s": round(nv * 1e3 / t_plain, 1), "plain_ms": round(t_plain, 3),
            "graph_views_per_s": round(nv * 1e3 / t_graph, 1), "graph_ms": round(t_graph, 3),
            "split_ms": split_ms,
            "autotuned": {"tile_size": best.tile_size, "sched": best.sched, "split": best.split, "ms": round(t_tune, 3)},
            "keys": int(fr.counts()[0]), "evaluations": int(evals_plain), "plain_stages_ms": mv_stages}
        del gr, fr, fr2, out, g, ms
        torch.cuda.empty_cache()
    if "closeup" in which:
        # the per-tile work split where it pays: 16 tiles of ~40k records
        sc = scenes.closeup_scene()
        g = umgs.gaussians_to_device(sc.gaussians, dev)
        ms = [umgs.mesh_to_device(m, dev) for m in sc.meshes]
        out = torch.empty((1, 512, 512, 4), device=dev)
        fr = umgs.Frame(ctx)
        t_plain = _time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16), out=out, frame=fr), steps)
        nk = int(fr.counts()[0])
        split_ms = {str(sp): round(_time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, split=sp),
                                                             out=out, frame=fr), steps), 3)
                    for sp in (512, 1024, 2048)}
        best, t_tune = umgs.autotune(ctx, g, ms, sc.cameras, umgs.render_opts(16), out)
        fr2 = umgs.Frame(ctx)
        gr = umgs.Graph(ctx, fr2, g, ms, sc.cameras, best, out, key_headroom=1.0)
        t_graph = _time(lambda: gr.launch(), steps)
        gr.check()
        forms["split_closeup_512"] = {
            "workload": "512x512 close-up: 400k faint Gaussians in a 64x64 px square (16 tiles of ~40k records, "
                        "no early termination) + 320-face icosphere",
            "plain_ms": round(t_plain, 3), "split_ms": split_ms,
            "autotuned": {"tile_size": best.tile_size, "sched": best.sched, "split": best.split, "ms": round(t_tune, 3)},
            "graph_ms": round(t_graph, 3), "graph_vs_plain": round(t_plain / t_graph, 2), "keys": nk}
        del gr, fr, fr2, out, g, ms
        torch.cuda.empty_cache()
    if "differentiable" in which:
        # config 3: 8 views of 512x512, forward vs forward+backward (L2 loss to a
        # render of a perturbed copy of the scene)
        sc = scenes.config3()
        rng = np.random.default_rng(7)
        pert = scenes.config3()
        pert.gaussians.means = (pert.gaussians.means + rng.normal(0, 0.01, pert.gaussians.means.shape)).astype(np.float32)
        pert.gaussians.sh = (pert.gaussians.sh + rng.normal(0, 0.05, pert.gaussians.sh.shape)).astype(np.float32)
        o = np.clip(pert.gaussians.opacities.astype(np.float64), 1e-6, 1 - 1e-6)
        logit = np.log(o / (1 - o)) + rng.normal(0, 0.2, o.shape)
        pert.gaussians.opacities = (1 / (1 + np.exp(-logit))).astype(np.float32)
        for m in pert.meshes:
            m.verts = (m.verts + rng.normal(0, 0.005, m.verts.shape)).astype(np.float32)
            m.vcolor = np.clip(m.vcolor + rng.normal(0, 0.05, m.vcolor.shape), 0, 1).astype(np.float32)
        mp = [umgs.mesh_to_device(m, dev) for m in pert.meshes]
        g = umgs.gaussians_to_device(sc.gaussians, dev)
        ms = [umgs.mesh_to_device(m, dev) for m in sc.meshes]
        gp = umgs.gaussians_to_device(pert.gaussians, dev)
        nv = len(sc.cameras)
        target = umgs.render(ctx, gp, mp, sc.cameras, umgs.render_opts(16)).clone()
        out = torch.empty_like(target)
        fr = umgs.Frame(ctx)
        t_f = _time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16), out=out, frame=fr), steps)
        so = umgs.render_opts(16, save=True)

        def fb():
            umgs.render(ctx, g, ms, sc.cameras, so, out=out, frame=fr)
            dl = (2.0 / out.numel()) * (out - target)
            return umgs.render_backward(ctx, fr, g, ms, dl)
        t_fb = _time(fb, steps)
        keys_bin = int(fr.counts()[0])
        forms["differentiable_8x512"] = {
            "workload": "8 orbit views 512x512, 300k Gaussians SH3 + 50k-face torus, L2 loss to the render of a "
                        "perturbed copy (means, SH, opacity logits, vertices, colours)",
            "fwd_views_per_s": round(nv * 1e3 / t_f, 1), "fwd_ms": round(t_f, 3),
            "fwd_bwd_views_per_s": round(nv * 1e3 / t_fb, 1), "fwd_bwd_ms": round(t_fb, 3)}
        # the same step with soft-edge triangle coverage (sigma 0.5 px): the
        # backward also reaches the vertex positions through coverage
        sig = 0.5
        t_sf = _time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, edge_sigma=sig), out=out, frame=fr),
                     steps)
        keys_soft = int(fr.counts()[0])
        so_soft = umgs.render_opts(16, save=True, edge_sigma=sig)

        def fb_soft():
            umgs.render(ctx, g, ms, sc.cameras, so_soft, out=out, frame=fr)
            dl = (2.0 / out.numel()) * (out - target)
            return umgs.render_backward(ctx, fr, g, ms, dl)
        t_sfb = _time(fb_soft, steps)
        forms["soft_edge_8x512"] = {
            "workload": "differentiable_8x512 with soft-edge triangle coverage, edge_sigma 0.5 px (rects widened 4 px)",
            "fwd_views_per_s": round(nv * 1e3 / t_sf, 1), "fwd_ms": round(t_sf, 3),
            "fwd_bwd_views_per_s": round(nv * 1e3 / t_sfb, 1), "fwd_bwd_ms": round(t_sfb, 3),
            "keys": keys_soft, "keys_binary_coverage": keys_bin}
        del g, ms, gp, mp, target, out, fr
        torch.cuda.empty_cache()
    if "mixed" in which:
        # config 4: 4K, 6M Gaussians + 2M triangles, fp32 vs bf16 SH + fp16 records
        sc = scenes.config4()
        g32 = umgs.gaussians_to_device(sc.gaussians, dev)
        g16 = umgs.gaussians_to_device(sc.gaussians, dev, sh_dtype=torch.bfloat16)
        ms = [umgs.mesh_to_device(m, dev) for m in sc.meshes]
        out32 = torch.empty((1, 2160, 3840, 4), device=dev)
        out16 = torch.empty_like(out32)
        fr = umgs.Frame(ctx)
        t32 = _time(lambda: umgs.render(ctx, g32, ms, sc.cameras, umgs.render_opts(16), out=out32, frame=fr), steps)
        keys4 = fr.counts()[0]
        t16 = _time(lambda: umgs.render(ctx, g16, ms, sc.cameras, umgs.render_opts(16, mixed=True), out=out16, frame=fr),
                    steps)
        # per-stage split of both renders and the frame counters (a separate profiled pass)
        st4 = {}
        for name, gg, oo, mixed in (("fp32", g32, out32, False), ("mixed", g16, out16, True)):
            umgs.profile_read(ctx)
            umgs.profile_enable(ctx, True)
            umgs.render(ctx, gg, ms, sc.cameras, umgs.render_opts(16, mixed=mixed), out=oo, frame=fr)
            torch.cuda.synchronize()
            st_ms, st_n = umgs.profile_read(ctx)
            umgs.profile_enable(ctx, False)
            st4[name] = {stage_names()[k]: round(st_ms[k] / st_n[k], 3) for k in range(16) if st_n[k] > 0}
        stats4 = fr.stats()
        d = (out16[..., :3] - out32[..., :3]).abs().flatten()
        mse = float(((out16[..., :3] - out32[..., :3]) ** 2).mean())
        forms["mixed_4k"] = {
            "workload": "3840x2160, 6M Gaussians SH3 + 2M-face torus (30% transparent)",
            "fp32_frames_per_s": round(1e3 / t32, 2), "fp32_ms": round(t32, 3),
            "mixed_frames_per_s": round(1e3 / t16, 2), "mixed_ms": round(t16, 3), "keys": int(keys4),
            "mixed_vs_fp32": {"max_abs": float(d.max()), "p99_9": float(torch.quantile(d[::7].float(), 0.999)),
                              "psnr_db": round(10 * math.log10(1.0 / max(mse, 1e-20)), 2)},
            "stages_ms": st4, "fp64_conics": stats4["fp64_conics"],
            "evaluations": {"gaussian": stats4["gaussian_evals"], "triangle": stats4["triangle_evals"]}}
        if crops is not None:
            # fp64 oracle (fp32 SH, not rounded to bf16) on 4 crops: the error of
            # the mixed form against the exact composite, and of the fp32 form
            img16 = out16[0, ..., :3].cpu().numpy().astype(np.float64)
            img32 = out32[0, ..., :3].cpu().numpy().astype(np.float64)
            ref, wall = crops.result()
            forms["mixed_4k"]["vs_fp64_oracle"] = {
                "crops": "%d crops of %dx%d (centre + 3 seeded positions)" % (len(ref), CROP, CROP),
                "mixed": crop_errors(ref, img16), "fp32": crop_errors(ref, img32), "oracle_wall_s": round(wall, 1)}
        del g32, g16, ms, out32, out16, fr
        torch.cuda.empty_cache()
    if "nested" in which:
        # nested transparency (Fig. 5b): Gaussians and an opaque ball inside a
        # transparent sphere, single pass vs the separate-pass baseline (the two
        # representations rendered apart with their expected depths and
        # composited per pixel by depth); errors against the single pass, which
        # the tests hold to the oracle
        sc, ga, me = scenes.nested_scene(size=1024, n_gauss=400_000, bowl_subdiv=5)
        bg = (0.05, 0.05, 0.08)
        g = umgs.gaussians_to_device(sc.gaussians, dev)
        ms = [umgs.mesh_to_device(m, dev) for m in sc.meshes]
        one = torch.empty((1, 1024, 1024, 4), device=dev)
        la, lb = torch.empty_like(one), torch.empty_like(one)
        fa, fb_, fr = umgs.Frame(ctx), umgs.Frame(ctx), umgs.Frame(ctx)
        depth_opts = umgs.render_opts(16, depth=True)
        da = torch.empty((1, 1024, 1024), device=dev)
        db = torch.empty_like(da)
        sep = torch.empty_like(one)

        def separate():
            umgs.render(ctx, g, [], sc.cameras, depth_opts, out=la, frame=fa)
            umgs.render(ctx, None, ms, sc.cameras, depth_opts, out=lb, frame=fb_)
            lib = umgs.lib()
            ctx.check(lib.umgs_frame_depth(fa._h, umgs._ptr(da), umgs._stream()), "umgs_frame_depth")
            ctx.check(lib.umgs_frame_depth(fb_._h, umgs._ptr(db), umgs._stream()), "umgs_frame_depth")
            umgs.composite_layers(ctx, la, da, lb, db, bg=bg, out=sep)
        t_one = _time(lambda: umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, bg=bg), out=one, frame=fr), steps)
        t_sep = _time(separate, steps)
        d = (sep[..., :3] - one[..., :3]).abs()
        seen = (one[..., 3] < 0.999)  # pixels where something is blended
        mse = float(((sep[..., :3] - one[..., :3]) ** 2)[seen].mean())
        forms["nested_transparency_1024"] = {
            "workload": "1024x1024, 400k Gaussians (3 boxes) + opaque 320-face ball inside a transparent "
                        "20,480-face sphere (alpha 0.35)",
            "single_pass_ms": round(t_one, 3), "separate_pass_ms": round(t_sep, 3),
            "separate_vs_single": {"max_abs": round(float(d.max()), 4),
                                   "pixels_off_by_0.01": round(float((d.amax(-1) > 0.01).float()[seen].mean()), 4),
                                   "psnr_db_blended_pixels": round(10 * math.log10(1.0 / max(mse, 1e-20)), 2)}}
        del g, ms, one, la, lb, fa, fb_, fr, da, db, sep
        torch.cuda.empty_cache()
    return forms


# ----------------------------------------------------------------------------
# CPU oracle legs.  They run in a process pool started with `spawn` (the GPU
# process may already hold a CUDA context), over all host cores.

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def _subscene(sc, gi, ti, cam):
    """The primitives gi (Gaussians) and ti (faces of mesh 0) of `sc`, in
    their unified-id order, seen by `cam`.  Dropping primitives leaves every
    remaining fragment, its colour and its (depth bits, id) order unchanged,
    so pixels whose fragments are all kept composite exactly as in `sc`."""
    from paper_2601_19233_gb300 import scenes as S
    g = sc.gaussians
    G = S.Gaussians(g.means[gi], g.quats[gi], g.scales[gi], g.opacities[gi], g.sh[gi], g.sh_degree)
    meshes = []
    if sc.meshes:
        m = sc.meshes[0]
        meshes = [S.Mesh(m.verts, m.faces[ti], m.vcolor, m.valpha, None if m.falpha is None else m.falpha[ti])]
    return S.Scene(G, meshes, [cam], tile=sc.tile)


def _canonical_rects(sc, cam):
    """Pixel rects (x0, x1, y0, y1) and validity of every Gaussian and face (oracle, canonical fp32)."""
    from oracle import canonical as cn
    g = sc.gaussians
    pg = cn.project_gaussians(g.means, g.quats, g.scales, None, cam)
    if sc.meshes:
        m = sc.meshes[0]
        tr = cn.setup_triangles(m.verts, m.faces, cam)
        return pg["rect"], pg["valid"], tr["rect"], tr["valid"]
    return pg["rect"], pg["valid"], np.zeros((0, 4), np.int64), np.zeros(0, bool)


def _touching(rect, valid, win):
    x0, x1, y0, y1 = win
    return np.nonzero(valid & (rect[:, 0] <= x1) & (rect[:, 1] >= x0) & (rect[:, 2] <= y1) & (rect[:, 3] >= y0))[0]


def _oracle_share(task):
    """One worker's share of one sample step: Eq. 12-13 for a slice of the
    Gaussians (the proxy's per-vertex table given) and the composite of a band
    of pixels (primitive-major gather of the oracle's full-image path, cut to
    the band).  Returns the seconds of each part."""
    from oracle import deform as OD
    from oracle import render as OR
    (g_def, face, bary, PV, VD, PF, table), (band_scene, window) = task
    t0 = time.perf_counter()
    if len(face):
        OD.deform_gaussians(g_def[0], g_def[1], g_def[2], face, bary, PV, VD, PF, table=table)
    t1 = time.perf_counter()
    if band_scene is not None:
        OR.render_image(band_scene, window=window)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


class OracleSample:
    """A bounded, measured sample of the 1080p deform + render frame for the
    CPU oracle.  A step is 1/K of a frame (K = frame pixels / 1024): the
    deformation of N/K Gaussians (Eq. 12-13) and the composite of one 32 x 32
    pixel block, both split over `workers` processes, plus 1/K of the two
    per-frame parts, each measured once per run: the proxy's per-vertex table
    (Sec. 3.3) and the frame setup (projection, SH colour, triangle setup of
    every primitive).  The binding the deformation reads is a seeded random
    face / barycentric table (binding is a one-time step, timed on the GPU
    only)."""

    BLOCK = 32

    def __init__(self, sc, workers, seed=0):
        from oracle import render as OR
        self.sc = sc
        self.P = max(1, int(workers))
        cam = sc.cameras[0]
        self.cam = cam
        self.K = (cam.width * cam.height) // (self.BLOCK * self.BLOCK)
        rng = np.random.default_rng(seed)
        n = sc.gaussians.n
        self.face = rng.integers(0, len(sc.proxy_faces), size=(n, 8)).astype(np.int32)
        b = rng.uniform(0, 1, size=(n, 8, 2))
        self.bary = np.where(b.sum(-1, keepdims=True) > 1, 1 - b, b).astype(np.float32)
        self.rng = rng
        t0 = time.perf_counter()
        fr = OR.Frame(sc)
        self.setup_s = time.perf_counter() - t0
        P_ = fr.P
        ng = sc.gaussians.n
        self.rects = (P_.rect[:ng], P_.valid[:ng], P_.rect[ng:], P_.valid[ng:])
        del fr

    def tasks(self, step):
        from oracle import deform as OD
        from paper_2601_19233_gb300 import scenes
        sc, P, K, B = self.sc, self.P, self.K, self.BLOCK
        g = sc.gaussians
        n = g.n
        vd = scenes.displace(sc.proxy_verts, sc.extra["sinusoids"], step)
        t0 = time.perf_counter()
        table = OD.vertex_transforms(sc.proxy_verts, vd, sc.proxy_faces)
        table_s = time.perf_counter() - t0
        ng_share = max(1, n // (K * P))
        bx = int(self.rng.integers(0, self.cam.width // B)) * B
        by = int(self.rng.integers(0, self.cam.height // B)) * B
        rows = np.array_split(np.arange(by, by + B), P)
        out = []
        for p in range(P):
            a = int(self.rng.integers(0, n - ng_share))
            sl = slice(a, a + ng_share)
            dfm = ((g.means[sl], g.quats[sl], g.scales[sl]), self.face[sl], self.bary[sl], sc.proxy_verts, vd,
                   sc.proxy_faces, table)
            band = (None, None)
            if len(rows[p]):
                win = (bx, bx + B - 1, int(rows[p][0]), int(rows[p][-1]))
                gi = _touching(self.rects[0], self.rects[1], win)
                ti = _touching(self.rects[2], self.rects[3], win)
                band = (_subscene(sc, gi, ti, self.cam), win)
            out.append((dfm, band))
        return out, table_s

    def run(self, pool, steps, warmup=0):
        """Time `steps` sample steps (after `warmup` untimed ones).  Returns
        (seconds per step including the 1/K shares of the per-frame parts,
        dict of the parts)."""
        times, parts, tables = [], [], []
        for k in range(warmup + steps):
            tasks, table_s = self.tasks(k)
            t0 = time.perf_counter()
            res = pool.map(_oracle_share, tasks)
            dt = time.perf_counter() - t0
            if k >= warmup:
                times.append(dt)
                tables.append(table_s)
                parts.append(np.sum(np.asarray(res), 0))
        s_step = float(np.mean(times)) + (float(np.mean(tables)) + self.setup_s) / self.K
        cpu = np.mean(parts, 0)
        return s_step, {"parallel_s_per_step": round(float(np.mean(times)), 4),
                        "cpu_s_per_step_deform": round(float(cpu[0]), 4),
                        "cpu_s_per_step_composite": round(float(cpu[1]), 4),
                        "proxy_table_s_per_frame": round(float(np.mean(tables)), 4),
                        "setup_s_per_frame": round(self.setup_s, 3)}

    def describe(self):
        return ("per step 1/%d of the 1080p frame: oracle deform of %d Gaussians and composite (primitive-major "
                "gather) of one 32x32 pixel block over %d processes, plus 1/%d of the per-frame proxy table and "
                "frame setup (each measured once); value = frame fraction per step / step time"
                % (self.K, max(1, self.sc.gaussians.n // self.K), self.P, self.K))


def cpu_baseline(pool, workers, sc, steps=6):
    smp = OracleSample(sc, workers, seed=3)
    s_step, parts = smp.run(pool, steps, warmup=1)
    return {"value": (1.0 / smp.K) / s_step, "unit": "frames/s", "cores": smp.P, "host_cores": host_cores(),
            "kind": "oracle", "sample": smp.describe() + "; %d steps" % steps,
            "s_per_step": round(s_step, 4), "frame_s_extrapolated": round(s_step * smp.K, 1), "parts": parts}


# 4K crops of the mixed-precision form against the fp64 oracle on the
# un-rounded (fp32) SH: the centre and three seeded positions
CROP = 64


def crop_windows(W, H, size=CROP, seed=1104):
    """The centre crop and three seeded crops whose centres lie within 900 px
    of the image centre (the shell of Gaussians covers a disc of about 1,180 px
    radius at 4K)."""
    rng = np.random.default_rng(seed)
    wins = [(W // 2 - size // 2, H // 2 - size // 2)]
    for _ in range(3):
        r, th = 900.0 * math.sqrt(rng.uniform()), rng.uniform(0, 2 * math.pi)
        wins.append((int(W / 2 + r * math.cos(th)) - size // 2, int(H / 2 + r * math.sin(th)) - size // 2))
    return [(x, x + size - 1, y, y + size - 1) for x, y in wins]


def _crop_prep(bands):
    """Config-4 scene, cut per (crop, band) to the primitives whose rect meets it."""
    from paper_2601_19233_gb300 import scenes
    sc = scenes.config4()
    cam = sc.cameras[0]
    rects = _canonical_rects(sc, cam)
    out = []
    for ci, (x0, x1, y0, y1) in enumerate(crop_windows(cam.width, cam.height)):
        for rows in np.array_split(np.arange(y0, y1 + 1), bands):
            win = (x0, x1, int(rows[0]), int(rows[-1]))
            gi = _touching(rects[0], rects[1], win)
            ti = _touching(rects[2], rects[3], win)
            out.append((ci, win, _subscene(sc, gi, ti, cam)))
    return out


def _crop_band(task):
    from oracle import render as OR
    ci, win, sub = task
    r = OR.render_image(sub, window=win)
    x0, x1, y0, y1 = win
    return ci, win, r["rgb"][y0:y1 + 1, x0:x1 + 1], r["tie"][y0:y1 + 1, x0:x1 + 1]


class CropOracle:
    """fp64 oracle renders of the 4K crops, computed in the pool while the GPU works."""

    def __init__(self, pool, bands):
        self.pool = pool
        self.jobs = []
        self.t0 = time.perf_counter()
        self.prep = pool.apply_async(_crop_prep, (bands,), callback=self._submit)

    def _submit(self, tasks):
        self.jobs = [self.pool.apply_async(_crop_band, (t,)) for t in tasks]

    def result(self, timeout=1800):
        self.prep.wait(timeout)
        if not self.prep.successful():
            self.prep.get()
        while not self.jobs:
            time.sleep(0.05)
        out = {}
        for j in self.jobs:
            ci, win, rgb, tie = j.get(timeout)
            out.setdefault(ci, []).append((win, rgb, tie))
        return out, time.perf_counter() - self.t0


def crop_errors(crops, img):
    """max-abs, p99.9 and PSNR of img [H,W,3] (numpy) against the oracle crops, tie pixels excluded."""
    diffs, ties = [], 0
    for ci, bands in crops.items():
        for (x0, x1, y0, y1), rgb, tie in bands:
            d = np.abs(img[y0:y1 + 1, x0:x1 + 1] - rgb)
            diffs.append(d[~tie].ravel())
            ties += int(tie.sum())
    d = np.concatenate(diffs)
    mse = float((d ** 2).mean())
    return {"max_abs": float(d.max()), "p99_9": float(np.quantile(d, 0.999)),
            "psnr_db": round(10 * math.log10(1.0 / max(mse, 1e-30)), 2), "tie_pixels": ties}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2601_19233_gb300 import scenes
    sc = scenes.config1(n_gauss=args.n_gauss)
    workers = host_cores()
    pool = oracle_pool(workers)
    try:
        smp = OracleSample(sc, workers, seed=0)
        s_step, parts = smp.run(pool, args.steps, warmup=args.warmup)
    finally:
        pool.close()
        pool.join()
    value = (1.0 / smp.K) / s_step
    res = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(s_step * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "frame_fraction_per_step": 1.0 / smp.K},
           "frame_s_extrapolated": round(s_step * smp.K, 1),
           "cpu_baseline": {"value": value, "unit": "frames/s", "cores": smp.P, "host_cores": host_cores(),
                            "kind": "oracle", "sample": smp.describe(), "parts": parts},
           "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_umgs(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
