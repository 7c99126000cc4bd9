#!/usr/bin/env python
"""Benchmark of the Language Embedded 3D Gaussians hot path on GB300.

Workload (the training-loop configuration): 1M Gaussians (50-cluster mixture,
SH degree 3, 8-dim semantic feature + uncertainty), 16 camera poses on a
circle of radius 3, 1296x840, 128-entry codebook with per-view Voronoi index
maps.  One step = preprocess -> binning/sort -> render forward -> RGB L1 ->
decoder D_MLP + uncertainty-weighted CE (training) -> render backward (all
Gaussian parameters) -> Adam, on view (step mod 16), all through the C ABI.
Also measured: the query render (same 1M Gaussians and view size, decode to a
256-entry codebook of 896-dim entries, relevancy for 4 prompts / 4 negatives)
and the fused BF16 vs unfused FP32 decoder paths.

Prints one JSON line.  --impl reference times the FP64 CPU oracle instead (a
bounded sample of the same step, extrapolated; see `reference_step`).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per fwd+bwd step and per query render at 1M Gaussians; % HBM roofline; fused vs plain"
N_GAUSS, W, H, N_VIEWS = 1_000_000, 1296, 840, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--decoder", default="auto", choices=["auto", "fused", "unfused"])
    ap.add_argument("--n", type=int, default=N_GAUSS, help="Gaussian count (default: the workload's 1M)")
    ap.add_argument("--no-extras", action="store_true", help="skip the query / unfused comparison legs")
    ap.add_argument("--only", choices=["quantize", "smooth", "query", "decoder_wide", "configs"], default=None,
                    help="run one leg alone (quantize: the quantisation stage on --features rows; smooth: "
                         "the adaptive smoothing on --n Gaussians; query: the fused relevancy query and the "
                         "feature-map export on --features random rendered features, without rendering; "
                         "decoder_wide: one training call of the 8-128-256-128 decoder on --features pixels; configs: "
                         "the c1 / c3 autograd steps and the c2 training step at their stated sizes)")
    ap.add_argument("--features", type=int, default=W * H, help="feature rows / pixels for --only quantize|query")
    return ap.parse_args()


# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) > 8:
                for k, v in zip(names, r[5:9]):
                    if "Active" in v and "Not" not in v:
                        reasons.add(k)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, device, world: int) -> float:
    """Largest value over all ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_step(ms_max: float, steps: int, world: int) -> float:
    """Whole-job time per step: `world` replicas each ran `steps` steps within ms_max."""
    return ms_max / (steps * world)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# ---------------------------------------------------------------------------
STAGE_CALLS = {"preprocess": "le_preprocess (preprocess_kernel)",
               "bin_render": "le_bin_render_fwd (depth radix sort, chunk counts, scan, lazily placed copies "
                             "and compositing)",
               "decoder": "le_decode_l1 fused (dec_train_kernel with the RGB L1 term in the same pass)",
               "render_bwd": "le_render_bwd_screen (render_bwd_kernel)",
               "project_bwd_adam": "le_project_bwd_adam (preprocess_bwd_kernel with the Gaussians' Adam step "
                                   "fused in)",
               "adam": "le_adam (adam_kernel, decoder parameters)"}
STAGE_SOURCES = {"preprocess": ["preprocess.cu"], "bin_render": ["binning.cu", "render.cu"],
                 "decoder": ["decoder_tc.cu", "tc_common.cuh", "train.cu"],
                 "render_bwd": ["render.cu", "common.cuh"], "project_bwd_adam": ["preprocess.cu", "common.cuh"],
                 "adam": ["train.cu", "common.cuh"]}

# FP32 operations (an FMA counts 2) per (pixel, Gaussian) pair of the render
# backward, from the arithmetic of the compositing adjoint.  Every walked pair
# (each list position below the pixel's n_contrib): d = mu - pixel (2), the
# quadratic form q (8), alpha = min(0.99, o 2^-q) (2), the two skip tests (2),
# plus one exp.  Every contributing pair (q >= 0, alpha >= 1/255) adds: T
# recovery by division (2), w = alpha T (1), the 12 channel gradients and the
# dot product f.dL/dC (48), dL/dalpha (5), the colour-behind recurrence (3),
# opacity and power terms (3), conic (11) and mean (10) terms: 83.
BWD_FLOP_WALKED, BWD_FLOP_CONTRIB = 14, 83
# The same for the forward compositing: every walked pair the 14 of the skip
# tests above; every contributing pair T (1 - alpha) and the stop test (3),
# w = alpha T (1) and the 12 blended channels (24): 28.
FWD_FLOP_WALKED, FWD_FLOP_CONTRIB = 14, 28
DEC_FLOP_PER_PX = 3 * 2 * (8 * 64 + 64 * 128 + 128 * 128)    # forward + input and weight gradients


def stage_bytes(N, n_vis, K, P, T, nc, total_scalars, K_read):
    """Compulsory HBM bytes per call of each stage (each input read once, each output written once).
    project_bwd_adam applies the Gaussians' Adam step: read grad2d, the parameters, m and v,
    write parameters, m and v."""
    par = 4 * (3 + 3 + 4 + 1 + 3 * nc + 8 + 1)          # all per-Gaussian parameters
    return {
        "preprocess": N * par + N * (80 + 4 + 4 + 8 + 4 + 1 + 32),
        # binning inputs, the list entries the compositing reads (written once, read once), records, images
        "bin_render": N * (4 + 4) + n_vis * (8 + 32) + 8 * T + 8 * K_read + 80 * n_vis + 56 * P,
        "decoder": (36 + 4 + 36) * P + 36 * P,     # decoder + RGB L1
        # list entries, records, T_final + n_contrib + upstream gradients, grad2d (zeroed, accumulated)
        "render_bwd": 4 * K_read + 80 * n_vis + 56 * P + 80 * N,
        "project_bwd_adam": 80 * N + 5 * N + 6 * par * N,
        "adam": 28 * (total_scalars - par // 4 * N),
    }


def pair_counts(img, ids, ranges, splat, TX, sample_tiles=256, seed=0):
    """(walked, contributing) (pixel, Gaussian) pairs of the render backward.
    walked = sum of n_contrib (exact); the contributing fraction is measured on
    a seeded sample of tiles by evaluating the skip tests of the renderer
    (q >= 0, alpha >= 1/255 with the record's base-2 conic) in torch."""
    import torch
    nc = img.n_contrib
    walked = int(nc.sum().item())
    H, W = nc.shape
    ncb = torch.nn.functional.pad(nc.float(), (0, (-W) % 16, 0, (-H) % 16))
    tmax = torch.nn.functional.max_pool2d(ncb[None, None], 16)[0, 0].flatten().long()
    live = torch.nonzero(tmax > 0).flatten()
    if walked == 0 or live.numel() == 0:
        return walked, 0
    g = torch.Generator(device="cpu").manual_seed(seed)
    pick = live[torch.randperm(live.numel(), generator=g)[:sample_tiles].to(live.device)]
    rg = ranges.view(-1, 2).long()
    s_walk = s_con = 0
    for t in pick.tolist():
        m = int(tmax[t])
        ty, tx = divmod(t, TX)
        gid = ids[int(rg[t, 0]):int(rg[t, 0]) + m].long()
        r = splat[gid]                                                    # [m, 20]
        ys = torch.arange(ty * 16, ty * 16 + 16, device=r.device)
        xs = torch.arange(tx * 16, tx * 16 + 16, device=r.device)
        py, px = torch.meshgrid(ys, xs, indexing="ij")
        inside = (py < H) & (px < W)
        py, px = py[inside].float(), px[inside].float()
        ncp = nc[py.long(), px.long()]
        dx = r[None, :, 0] - px[:, None]
        dy = r[None, :, 1] - py[:, None]
        q = r[None, :, 2] * dx * dx + r[None, :, 3] * dx * dy + r[None, :, 4] * dy * dy
        alpha = torch.clamp(r[None, :, 5] * torch.exp2(-q), max=0.99)
        pos = torch.arange(m, device=r.device)[None, :]
        walk = pos < ncp[:, None].long()
        con = walk & (q >= 0) & (alpha >= 1.0 / 255.0)
        s_walk += int(walk.sum().item())
        s_con += int(con.sum().item())
    return walked, int(round(walked * s_con / max(s_walk, 1)))


def _sources_sha(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2311_18482_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def stage_traffic(stage):
    """DRAM bytes per call measured by ncu (profiles/traffic.json), or None when the
    kernel sources changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(stage)
    if not rec or rec.get("sources_sha") != _sources_sha(STAGE_SOURCES[stage]):
        return None
    return rec.get("dram_bytes_per_call")


def workload_config(n, world):
    """The `config` of both arms' JSON lines (the same dict)."""
    return {"workload": "c5 training step: 1M Gaussians, SH deg 3, 1296x840, 16 poses, 128-entry codebook",
            "gaussians": n, "width": W, "height": H,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "inputs larger than L2 (272 MB of parameters + 2.2 GB of state per step)"}


def setup_workload(n, pin=True):
    import numpy as np
    import torch
    from paper_2311_18482_gb300 import synth
    c = synth.config("c5", n=n)
    scene, dec = c["scene"], c["decoder"]
    cams, rgb_t, idx_t = [], [], []
    for k in range(N_VIEWS):
        cams.append(synth.circle_pose(k, N_VIEWS, W, H))
        rgb_t.append(synth.smooth_rgb_target(2000 + k, W, H))
        idx_t.append(synth.voronoi_index_map(1000 + k, W, H, 128))
    rgb_host = torch.from_numpy(np.stack(rgb_t))
    idx_host = torch.from_numpy(np.stack(idx_t))
    if pin:
        rgb_host, idx_host = rgb_host.pin_memory(), idx_host.pin_memory()
    return scene, dec, cams, rgb_host, idx_host


def run_ours(args, rank, world):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2311_18482_gb300 as leg
    from paper_2311_18482_gb300 import synth
    from paper_2311_18482_gb300.training import TrainState

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    dev = "cuda"
    leg.load()
    scene, dec, cams, rgb_host, idx_host = setup_workload(args.n)
    rgb_dev, idx_dev = rgb_host.to(dev), idx_host.to(dev)
    hbm_peak, bf16_peak, peak_kind = measured_peaks()

    def make_state(mode):
        return TrainState(scene, dec, W, H, dev, decoder_mode=mode)

    mode_name = args.decoder
    if mode_name == "auto":
        try:
            st = make_state(leg.FUSED_BF16)
            st.step(cams[0], rgb_dev[0], idx_dev[0])
            mode_name = "fused"
        except leg.LegError:
            mode_name = "unfused"
    mode = leg.FUSED_BF16 if mode_name == "fused" else leg.UNFUSED_FP32
    st = make_state(mode)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        st.step(cams[i % N_VIEWS], rgb_dev[i % N_VIEWS], idx_dev[i % N_VIEWS])
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    barrier()
    clocks.start()
    leg.reset_launch_count()
    st.events = []
    torch.cuda.reset_peak_memory_stats()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ks = []
    t0.record()
    for i in range(args.steps):
        k = (args.warmup + i) % N_VIEWS
        st.step(cams[k], rgb_dev[k], idx_dev[k])
        Ks.append(st.K)
    t1.record()
    barrier()
    launches = leg.launch_count()
    clk = clocks.stop()
    peak_alloc, peak_reserved = torch.cuda.max_memory_allocated(), torch.cuda.max_memory_reserved()
    ms = t0.elapsed_time(t1)
    stage_ms = {}
    evs = st.events
    st.events = None
    for (na, ea), (nb, eb) in zip(evs[:-1], evs[1:]):
        if nb == "start":
            continue
        stage_ms.setdefault(nb, []).append(ea.elapsed_time(eb))
    stage_ms = {k: sum(v) / len(v) for k, v in stage_ms.items()}
    ms = max_over_ranks(ms, dev, world)
    ms_step = job_ms_per_step(ms, args.steps, world)
    K_mean = float(np.mean(Ks))

    # --- end to end through the public API: per step H2D of the view's targets
    # from pinned host memory, the step, D2H of the loss vector.  The targets of
    # step i + 1 are copied on a second stream into the other of two staging
    # buffers while step i computes (events order each copy after the step that
    # last read its buffer, and the step after its copy); every copy and every
    # loss read-back lies inside the timed region.
    loss_host = torch.empty((args.steps, 3), dtype=torch.float32).pin_memory()
    rgb_stage = [torch.empty_like(rgb_dev[0]) for _ in range(2)]
    idx_stage = [torch.empty_like(idx_dev[0]) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    main_stream = torch.cuda.current_stream()

    def stage(i):
        b, k = i & 1, i % N_VIEWS
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(consumed[b])
            rgb_stage[b].copy_(rgb_host[k], non_blocking=True)
            idx_stage[b].copy_(idx_host[k], non_blocking=True)
            copied[b].record(copy_stream)

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0 = time.perf_counter()
    e0.record()
    copy_stream.wait_event(e0)
    stage(0)
    for i in range(args.steps):
        b, k = i & 1, i % N_VIEWS
        if i + 1 < args.steps:
            stage(i + 1)
        main_stream.wait_event(copied[b])
        loss = st.step(cams[k], rgb_stage[b], idx_stage[b])
        consumed[b].record(main_stream)
        loss_host[i].copy_(loss, non_blocking=True)
    e1.record()
    barrier()
    e2e_wall_ms = (time.perf_counter() - h0) * 1e3 / args.steps
    e2e_ms = e0.elapsed_time(e1) / args.steps
    h2d = rgb_stage[0].numel() * 4 + idx_stage[0].numel() * 4

    out = {"metric": METRIC, "value": round(ms_step, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if mode_name == "unfused" else "f32+bf16",
           "data": "synthetic (seeded 50-cluster scene, Voronoi index maps, smooth RGB targets)",
           "config": workload_config(args.n, world), "decoder_path": mode_name,
           "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 12,
                   "host_wall_ms": round(e2e_wall_ms, 4),
                   "note": "each step's targets are copied from pinned host memory on a second stream while "
                           "the previous step computes, and each step's loss is read back to pinned memory; "
                           "value = events around the whole loop on the compute stream, host_wall_ms = host "
                           "clock around the same loop (synchronised at both ends)"},
           "gpu_launches": launches, "clocks": clk, "stages_ms": {k: round(v, 4) for k, v in stage_ms.items()},
           "instances_K": K_mean,
           "peak_hbm": {"allocated_gb": round(peak_alloc / 1e9, 3), "reserved_gb": round(peak_reserved / 1e9, 3),
                        "note": "device memory in use over the timed steps (torch's caching allocator): the "
                                "Gaussians and their Adam moments, the 16 views' targets and every step buffer; "
                                "the library allocates none itself"}}
    # (instances_read is added with the roofline below)

    # --- roofline of the dominant kernel (render_bwd_kernel, FP32-ALU bound):
    # algorithmic FP32 flops of the compositing adjoint per launch / its
    # event-timed duration, against the FP32 peak of the device's SM count x
    # 128 lanes x 2 flops (FMA) x the maximum SM clock.  The other stages against HBM
    # (compulsory bytes) and the decoder against the bf16 tensor peak.
    P = W * H
    nc = (scene.sh_degree + 1) ** 2
    N = args.n
    TX, TY = (W + 15) // 16, (H + 15) // 16
    # per-view work counts (one more step on each view after the timing), each view weighted by
    # how often the timed loop rendered it: visible Gaussians, list entries any pixel reads (per
    # tile the largest n_contrib), and the (pixel, Gaussian) pairs of render_bwd_kernel (walked
    # pairs exact, contributing fraction sampled)
    per_view = {}
    for k in range(N_VIEWS):
        st.step(cams[k], rgb_dev[k], idx_dev[k])
        ncb = torch.nn.functional.pad(st.img.n_contrib.float(), (0, (-W) % 16, 0, (-H) % 16))
        per_view[k] = (int((st.proj.tiles_touched > 0).sum().item()),
                       int(torch.nn.functional.max_pool2d(ncb[None, None], 16).sum().item()),
                       *pair_counts(st.img, st.bins.ids, st.bins.ranges, st.proj.splat, TX, sample_tiles=96))
    timed_views = [(args.warmup + i) % N_VIEWS for i in range(args.steps)]
    n_vis, K_read, walked, contrib = (sum(per_view[k][c] for k in timed_views) / len(timed_views) for c in range(4))
    alg_bytes = stage_bytes(N, n_vis, K_mean, P, TX * TY, nc, st.layout.total, K_read)
    sm_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    bwd_flop = BWD_FLOP_WALKED * walked + BWD_FLOP_CONTRIB * contrib
    t_bwd = stage_ms["render_bwd"] * 1e-3
    ach = bwd_flop / t_bwd / 1e12
    out["roofline"] = {"kernel": STAGE_CALLS["render_bwd"], "bound": "alu", "achieved": round(ach, 2),
                       "peak": round(fp32_peak, 1), "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                       "traffic": stage_traffic("render_bwd"), "peak_kind": f"derived: {n_sm} SMs (read from the device) x 128 "
                       f"FP32 lanes x 2 x {sm_mhz:.0f} MHz", "algorithmic_flop": round(bwd_flop), "pairs_walked": round(walked),
                       "pairs_contributing": round(contrib),
                       "note": f"{BWD_FLOP_WALKED} flop per walked pair + {BWD_FLOP_CONTRIB} per contributing "
                               "pair (FMA = 2), pairs averaged over the timed steps' views; traffic is DRAM "
                               "bytes per launch from ncu"}
    # forward compositing: the blend loop of the render phases, timed alone as le_render_fwd
    # (render_fwd_kernel, the same per-pixel loop in one launch) over one view's full lists
    k0 = timed_views[0]
    leg.le_preprocess(st.g, cams[k0], st.proj)
    fb = leg.BinSortBuffers()
    ids_f, rng_f, _, _ = leg.le_bin_sort(cams[k0], st.proj, fb)
    img_f = leg.Image.empty(H, W, "cuda")
    for _ in range(3):
        leg.le_render_fwd(cams[k0], st.proj, ids_f, rng_f, out=img_f)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(20):
        leg.le_render_fwd(cams[k0], st.proj, ids_f, rng_f, out=img_f)
    f1.record()
    torch.cuda.synchronize()
    t_fwd = f0.elapsed_time(f1) / 20 * 1e-3
    walked_f, contrib_f = pair_counts(img_f, ids_f, rng_f, st.proj.splat, TX, sample_tiles=96)
    fwd_flop = FWD_FLOP_WALKED * walked_f + FWD_FLOP_CONTRIB * contrib_f
    ach_f = fwd_flop / t_fwd / 1e12
    out["roofline_fwd"] = {"kernel": "le_render_fwd (render_fwd_kernel: the compositing loop of the render "
                                     "phases, on one view's full lists)", "bound": "alu",
                           "achieved": round(ach_f, 2), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                           "frac": round(ach_f / fp32_peak, 4), "traffic": None, "ms": round(t_fwd * 1e3, 4),
                           "algorithmic_flop": round(fwd_flop), "pairs_walked": walked_f,
                           "pairs_contributing": contrib_f,
                           "note": f"{FWD_FLOP_WALKED} flop per walked pair + {FWD_FLOP_CONTRIB} per contributing "
                                   "pair (FMA = 2); walked = the sum of n_contrib, a lower bound (pixels that "
                                   "never stop also test the rest of their list)"}
    del fb, ids_f, rng_f, img_f
    t_pb = stage_ms["project_bwd_adam"] * 1e-3
    ach_h = alg_bytes["project_bwd_adam"] / t_pb / 1e9
    out["roofline_hbm"] = {"kernel": STAGE_CALLS["project_bwd_adam"], "bound": "hbm", "achieved": round(ach_h, 1),
                           "peak": hbm_peak, "unit": "GB/s", "frac": round(ach_h / hbm_peak, 4),
                           "traffic": stage_traffic("project_bwd_adam"), "peak_kind": peak_kind,
                           "algorithmic_bytes": round(alg_bytes["project_bwd_adam"])}
    if mode_name == "fused":
        t_dec = stage_ms["decoder"] * 1e-3
        ach_t = DEC_FLOP_PER_PX * P / t_dec / 1e12
        out["roofline_tensor"] = {"kernel": STAGE_CALLS["decoder"], "bound": "tensor", "achieved": round(ach_t, 1),
                                  "peak": bf16_peak, "unit": "TFLOP/s", "frac": round(ach_t / bf16_peak, 4),
                                  "traffic": stage_traffic("decoder"), "peak_kind": peak_kind + " bf16 burst",
                                  "algorithmic_flop": DEC_FLOP_PER_PX * P}
    out["stage_hbm_frac"] = {k: round(alg_bytes[k] / (stage_ms[k] * 1e-3) / 1e9 / hbm_peak, 4)
                             for k in stage_ms if k in alg_bytes}
    out["visible_gaussians"] = round(n_vis)
    out["instances_read"] = round(K_read)

    if not args.no_extras and rank == 0:
        out["fused_vs_plain"] = compare_decoders(leg, st, mode_name, make_state, cams, rgb_dev, idx_dev, args)
        out["query"] = query_leg(leg, synth, scene, cams, args)
        out["query_c4"] = query_c4_leg(leg, synth, args)
        out["decoder_paper_widths"] = decoder_wide_leg(leg, synth, args, bf16_peak)
        out["configs"] = configs_leg(leg, synth, args)
        out["quantize"] = quant_leg(leg, synth, args, hbm_peak, bf16_peak, peak_kind)
        out["smooth"] = smooth_leg(leg, synth, st, args, bf16_peak)
        out["rgb_dssim"] = rgb_dssim_leg(leg, st, rgb_dev, args, hbm_peak)
        out["densify"] = densify_leg(leg, st, args, hbm_peak)
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(scene, dec, cams[0], rgb_host[0].numpy(), idx_host[0].numpy(),
                                           budget_s=20.0)
        print(json.dumps(out), flush=True)


def compare_decoders(leg, st, mode_name, make_state, cams, rgb_dev, idx_dev, args):
    import torch
    res = {}
    for name, mode in (("fused", leg.FUSED_BF16), ("unfused", leg.UNFUSED_FP32)):
        try:
            before = torch.cuda.memory_allocated()
            s2 = st if name == mode_name else make_state(mode)
            s2.events = []
            for i in range(3):
                s2.step(cams[i], rgb_dev[i], idx_dev[i])
            torch.cuda.synchronize()
            torch.cuda.reset_peak_memory_stats()
            s2.events = []
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            n = max(5, args.steps // 2)
            for i in range(n):
                s2.step(cams[i % N_VIEWS], rgb_dev[i % N_VIEWS], idx_dev[i % N_VIEWS])
            t1.record()
            torch.cuda.synchronize()
            dec_ms = [ea.elapsed_time(eb) for (na, ea), (nb, eb) in zip(s2.events[:-1], s2.events[1:])
                      if nb == "decoder"]
            s2.events = None
            res[name] = {"step_ms": round(t0.elapsed_time(t1) / n, 4),
                         "decoder_ms": round(sum(dec_ms) / len(dec_ms), 4)}
            if s2 is not st:
                # device memory this path needs on top of what was already in use
                res[name]["extra_peak_hbm_gb"] = round((torch.cuda.max_memory_allocated() - before) / 1e9, 3)
        except leg.LegError as e:
            res[name] = {"unavailable": str(e)[:200]}
    return res


def query_leg(leg, synth, scene, cams, args, Wq=W, Hq=H, dec=None, qin=None):
    """Query render: preprocess, bin, render, decode to the 256-entry codebook of
    896-dim entries, relevancy for 4 prompts / 4 negatives (fused and unfused)."""
    import torch
    qin = qin or synth.query_inputs(303, 256)
    dec = dec or synth.decoder_init(103, 256)
    dev = "cuda"
    t = lambda a: torch.from_numpy(a).to(dev).contiguous()
    dec_t = tuple(t(getattr(dec, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    cb, text, negs = t(qin.codebook), t(qin.text), t(qin.negs)
    g = leg.Gaussians.from_scene(scene)
    proj = leg.Projected.empty(scene.N)
    bins = leg.BinSortBuffers()
    img = leg.Image.empty(Hq, Wq)
    P = Wq * Hq
    res = {}
    for name, mode in (("fused", leg.FUSED_BF16), ("unfused", leg.UNFUSED_FP32)):
        try:
            decs = leg.decoder_struct(*dec_t)
            ws_q = torch.empty(max(leg.le_query_workspace(mode, P, 256, qin.d_clip), 1), dtype=torch.uint8,
                               device=dev)
            ws_d = torch.empty(max(leg.le_decode_workspace(leg.UNFUSED_FP32, P, decs), 1), dtype=torch.uint8,
                               device=dev)
            prob = torch.empty((256, P), dtype=torch.float32, device=dev) if mode == leg.UNFUSED_FP32 else None
            rel = torch.empty((4, P), dtype=torch.float32, device=dev)

            def once(k):
                leg.le_preprocess(g, cams[k], proj)
                ids, ranges, K, _ = leg.le_bin_render_fwd(cams[k], proj, bins, img)
                if mode == leg.UNFUSED_FP32:
                    leg.le_decode_raw(mode, P, img.feat, None, decs, None, 1.0, 1.0, None, None, None, None, None,
                                      prob, None, ws_d)
                    leg.le_query(mode, P, cb, qin.d_clip, text, negs, dec_t=dec_t, prob=prob, workspace=ws_q,
                                 out=rel)
                else:
                    leg.le_query(mode, P, cb, qin.d_clip, text, negs, feat=img.feat, dec_t=dec_t, workspace=ws_q,
                                 out=rel)
            for i in range(3):
                once(i % len(cams))
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n = max(5, args.steps // 2)
            t0.record()
            for i in range(n):
                once(i % len(cams))
            t1.record()
            torch.cuda.synchronize()
            res[name] = {"ms_per_query_render": round(t0.elapsed_time(t1) / n, 4)}
            del prob, ws_q, ws_d
        except leg.LegError as e:
            res[name] = {"unavailable": str(e)[:200]}
    if Wq != W or Hq != H:
        return res
    # the materialised language feature map F = M_infer S (BF16, [P, 896]) of the last render
    try:
        Fm = torch.empty((P, qin.codebook.shape[1]), dtype=torch.bfloat16, device=dev)
        for _ in range(3):
            leg.le_feature_map(img.feat.view(8, P), dec_t, cb, out=Fm)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(5, args.steps // 4)
        t0.record()
        for _ in range(n):
            leg.le_feature_map(img.feat.view(8, P), dec_t, cb, out=Fm)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / n
        byts = P * qin.codebook.shape[1] * 2 + P * 8 * 4
        hbm, _, kind = measured_peaks()
        res["feature_map"] = {"ms": round(ms, 4), "bytes": byts, "hbm_frac": round(byts / ms / 1e6 / hbm, 4),
                              "peak_kind": kind, "note": "le_feature_map: decode + softmax + F = p S, BF16 out"}
    except leg.LegError as e:
        res["feature_map"] = {"unavailable": str(e)[:200]}
    return res


def decoder_wide_leg(leg, synth, args, bf16_peak, P=W * H):
    """The decoder at the widths of supp. Tab. dmlp (8 -> 128 -> 256 -> 128 codes): one training
    call (forward, uncertainty-weighted CE, every gradient) on a 1296x840 view's rendered features
    (N(0,1) stand-ins) on the tensor cores against the unfused FP32 path."""
    import torch
    dec = synth.decoder_init(105, 128, h1=128, h2=256)
    dec_t = tuple(torch.from_numpy(getattr(dec, k)).cuda() for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    g = torch.Generator(device="cuda").manual_seed(6)
    feat = torch.randn((8, P), generator=g, device="cuda")
    unc = torch.rand(P, generator=g, device="cuda")
    tgt = torch.randint(0, 128, (P,), generator=g, device="cuda", dtype=torch.int32)
    res = {"pixels": P, "widths": "8-128-256-128"}
    for name, mode in (("fused", leg.FUSED_BF16), ("unfused", leg.UNFUSED_FP32)):
        try:
            out = leg.le_decode(mode, feat, dec_t, unc=unc, target=tgt)
            ws = out["workspace"]
            for _ in range(2):
                leg.le_decode(mode, feat, dec_t, unc=unc, target=tgt, workspace=ws)
            torch.cuda.synchronize()
            n = max(5, args.steps // 4)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(n):
                leg.le_decode(mode, feat, dec_t, unc=unc, target=tgt, workspace=ws)
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / n
            res[name] = {"ms": round(ms, 4)}
            del ws, out
        except leg.LegError as e:
            res[name] = {"unavailable": str(e)[:200]}
    flop = 3 * 2 * (8 * 128 + 128 * 256 + 256 * 128) * P
    if "ms" in res.get("fused", {}):
        res["fused"]["tensor_frac"] = round(flop / res["fused"]["ms"] / 1e9 / bf16_peak, 4)
    res["algorithmic_flop"] = flop
    torch.cuda.empty_cache()
    return res


def configs_leg(leg, synth, args):
    """The smaller workloads at their stated sizes, each timed with CUDA events after warm-up:
    c1 (2,000 Gaussians, 128x128, SH degree 0) and c3 (1M Gaussians, 1296x840, SH degree 3) as
    the autograd step -- rasterize forward, a fixed random upstream gradient on RGB, feature and
    uncertainty, backward to every per-Gaussian parameter -- and c2 (100k Gaussians, 640x480, SH
    degree 3) as the training step with decoder training (fused BF16 and unfused FP32 decoder)."""
    import torch
    from paper_2311_18482_gb300.training import TrainState

    def timed(f, n, warm=3):
        for _ in range(warm):
            f()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(n):
            f()
        t1.record()
        torch.cuda.synchronize()
        return round(t0.elapsed_time(t1) / n, 4)

    def autograd_step(name, n_iter):
        c = synth.config(name)
        sc, cam = c["scene"], c["camera"]
        params = [torch.from_numpy(getattr(sc, k)).cuda().requires_grad_(True)
                  for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")]
        gen = torch.Generator(device="cuda").manual_seed(7)
        dr = torch.randn((3, cam.H, cam.W), generator=gen, device="cuda")
        df = torch.randn((8, cam.H, cam.W), generator=gen, device="cuda")
        du = torch.randn((cam.H, cam.W), generator=gen, device="cuda")

        def step():
            for p in params:
                p.grad = None
            rgb, feat, unc, _ = leg.rasterize(*params, cam, sc.sh_degree)
            ((rgb * dr).sum() + (feat * df).sum() + (unc * du).sum()).backward()
        ms = timed(step, n_iter)
        del params
        # the same forward and backward as direct C-ABI calls into preallocated buffers (the lazily
        # placed binning of the training step, no autograd or torch ops around them)
        g = leg.Gaussians.from_scene(sc)
        proj = leg.Projected.empty(sc.N, "cuda")
        bins, img = leg.BinSortBuffers(), leg.Image.empty(cam.H, cam.W, "cuda")
        grads = g.zeros_like()
        grad2d = torch.empty((sc.N, leg.SPLAT_STRIDE), device="cuda")

        def calls():
            leg.le_preprocess(g, cam, proj)
            ids, ranges, _, _ = leg.le_bin_render_fwd(cam, proj, bins, img)
            leg.le_render_bwd(cam, g, proj, ids, ranges, img, dr, df, du, grads=grads, grad2d=grad2d)
        ms_calls = timed(calls, n_iter)
        del g, proj, bins, img, grads, grad2d
        torch.cuda.empty_cache()
        return {"gaussians": sc.N, "width": cam.W, "height": cam.H, "sh_degree": sc.sh_degree,
                "ms_fwd_bwd": ms, "path": "torch.autograd.Function (le_preprocess, le_bin_render_fwd, le_render_bwd; "
                                          "fresh outputs per call); includes the host read of K",
                "ms_fwd_bwd_calls": ms_calls,
                "calls": "le_preprocess, le_bin_render_fwd, le_render_bwd into preallocated buffers"}

    res = {"c1": autograd_step("c1", 50)}
    c = synth.config("c2")
    cam = c["camera"]
    rgb = torch.from_numpy(c["rgb_target"]).cuda()
    idx = torch.from_numpy(c["target_idx"]).cuda()
    c2 = {"gaussians": c["scene"].N, "width": cam.W, "height": cam.H, "codebook": 128}
    for name, mode in (("fused", leg.FUSED_BF16), ("unfused", leg.UNFUSED_FP32)):
        st = TrainState(c["scene"], c["decoder"], cam.W, cam.H, "cuda", decoder_mode=mode)
        c2[name] = {"ms_per_step": timed(lambda: st.step(cam, rgb, idx), 30)}
        del st
        torch.cuda.empty_cache()
    res["c2"] = c2
    res["c3"] = autograd_step("c3", 10)
    return res


def query_c4_leg(leg, synth, args):
    """The query-render workload at its own size: 3M Gaussians (50 clusters) at
    1920x1080, pose 0, decode to 256 codes of 896 dims, relevancy for 4 prompts /
    4 negatives; the same view every iteration."""
    import torch
    c = synth.config("c4")
    res = query_leg(leg, synth, c["scene"], [c["camera"]], args, Wq=c["camera"].W, Hq=c["camera"].H,
                    dec=c["decoder"], qin=c["query"])
    res["workload"] = "c4: 3M Gaussians, 1920x1080, 256 codes x 896 dims, 4 prompts + 4 negatives"
    torch.cuda.empty_cache()
    return res


# forward (3-128-128-128-8), input gradients of layers 4, 3, 2, weight gradients of all four
SMOOTH_FLOP_PER_GAUSSIAN = 2 * (3 * 128 + 2 * 128 * 128 + 128 * 8) + 2 * (8 * 128 + 2 * 128 * 128) \
    + 2 * (3 * 128 + 2 * 128 * 128 + 8 * 128)


def smooth_leg(leg, synth, st, args, bf16_peak):
    """Adaptive spatial smoothing (Sec. 3.4) over the training state's Gaussians:
    MLP(p) forward, L_smo and its backward, d_feat accumulated into grad2d's
    feature slots as in a training step."""
    import torch
    mlp = synth.smooth_mlp_init(5)
    params = {k: torch.from_numpy(getattr(mlp, k)).cuda() for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")}
    g = st.g
    grads = [torch.empty_like(v) for v in params.values()]
    rec = st.grad2d[:, 10:]
    try:
        for _ in range(3):
            leg.le_smooth(g.means, g.feat, g.unc, params, d_feat=rec, d_feat_stride=20, grads=grads)
        torch.cuda.synchronize()
        n = max(5, args.steps // 4)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(n):
            loss, _, _, _ = leg.le_smooth(g.means, g.feat, g.unc, params, d_feat=rec, d_feat_stride=20, grads=grads)
        t1.record()
        torch.cuda.synchronize()
    except leg.LegError as e:
        return {"unavailable": str(e)[:200]}
    ms = t0.elapsed_time(t1) / n
    flop = SMOOTH_FLOP_PER_GAUSSIAN * g.n
    return {"ms": round(ms, 4), "gaussians": g.n, "loss": round(float(loss.item()), 6),
            "tensor": {"achieved_tflops": round(flop / ms / 1e9, 1), "peak": bf16_peak,
                       "frac": round(flop / ms / 1e9 / bf16_peak, 4), "algorithmic_flop": flop}}


def rgb_dssim_leg(leg, st, rgb_dev, args, hbm_peak):
    """3DGS's RGB loss (1 - 0.2) L1 + 0.2 D-SSIM (le_rgb_loss, forward and gradient) on the last
    rendered 1296x840 view, in place of the L1 term of the training-loop configuration."""
    import torch
    ws = torch.empty(leg.le_rgb_loss_workspace(W, H), dtype=torch.uint8, device="cuda")
    loss, grad = torch.empty(3, device="cuda"), torch.empty_like(st.img.rgb)
    for _ in range(3):
        leg.le_rgb_loss(st.img.rgb, rgb_dev[0], 0.2, loss=loss, grad=grad, workspace=ws)
    torch.cuda.synchronize()
    n = max(5, args.steps // 4)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(n):
        leg.le_rgb_loss(st.img.rgb, rgb_dev[0], 0.2, loss=loss, grad=grad, workspace=ws)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / n
    byts = W * H * (12 + 12 + 36 + 36 + 12 + 12 + 12)   # fwd: image, target, 3 maps x 3 ch; bwd: maps, image, target, grad
    return {"ms": round(ms, 4), "hbm_frac": round(byts / ms / 1e6 / hbm_peak, 4), "algorithmic_bytes": byts,
            "loss": [round(float(x), 6) for x in loss.cpu()]}


def densify_leg(leg, st, args, hbm_peak):
    """Adaptive density control over the training state's 1M Gaussians: statistics from the last
    step's screen-space gradients (a synthetic accumulated state: every visible Gaussian seen on
    10 steps), then one clone/split/prune call into new buffers with 3DGS's size pruning on
    (largest screen radius > 20 px, largest scale > 0.1 x extent), and one opacity reset."""
    import torch
    g = st.g
    n = g.n
    acc = torch.zeros(n, device="cuda")
    cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    mr = torch.zeros(n, dtype=torch.int32, device="cuda")
    for _ in range(10):
        leg.le_densify_stats(st.grad2d, st.proj.radius, acc, cnt, mr)
    noise = torch.randn((n, 2, 3), generator=torch.Generator(device="cuda").manual_seed(5), device="cuda")
    thresh = float(torch.quantile((acc / cnt.clamp_min(1))[cnt > 0][:1_000_000], 0.9))   # densify ~10 %
    kw = dict(grad_thresh=thresh, percent_dense=0.01, scene_extent=4.0, min_opacity=0.005, n_cap=2 * n,
              max_radius=mr, max_screen_size=20.0, world_frac=0.1)
    for _ in range(2):
        out = leg.le_densify(g, st.gm, st.gvv, acc, cnt, noise, **kw)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    t0.record()
    for _ in range(reps):
        out = leg.le_densify(g, st.gm, st.gvv, acc, cnt, noise, **kw)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / reps
    n2 = out[0].n
    op, om, ov = (x.opacity_raw.clone() for x in out)
    t0.record()
    for _ in range(reps):
        leg.le_opacity_reset(op, om, ov, 0.01)
    t1.record()
    torch.cuda.synchronize()
    ms_reset = t0.elapsed_time(t1) / reps
    par = 4 * (3 + 3 + 4 + 1 + 48 + 8 + 1)
    byts = 3 * par * n + 3 * par * n2 + 16 * n     # read params, m, v; write them for n2; statistics
    return {"ms": round(ms, 4), "gaussians_in": n, "gaussians_out": n2, "hbm_frac": round(byts / ms / 1e6 / hbm_peak, 4),
            "opacity_reset_ms": round(ms_reset, 4),
            "note": "one le_densify call (classify with size pruning, scan, host read of the totals, scatter)"}


def quant_leg(leg, synth, args, hbm_peak, bf16_peak, peak_kind):
    """Quantisation stage (Sec. 3.3) on one view's features: 1296x840 = 1,088,640
    hybrid features of 896 dims (BF16, 1.95 GB, far larger than L2), 128-entry
    codebook: argmax index map, L_cos, load balancing.  Features are drawn on the
    GPU (seeded) around 128 hidden codes laid out by a Voronoi map of the view."""
    import math
    import numpy as np
    import torch
    K, N, dc, dd = getattr(args, "features", W * H), 128, 512, 384
    d = dc + dd
    rng = np.random.default_rng(77)
    centres = np.concatenate([synth.unit_rows(rng, N, dc), synth.unit_rows(rng, N, dd)], axis=1)
    Hk = (K + W - 1) // W
    lab = torch.from_numpy(synth.voronoi_index_map(78, W, Hk, N, n_seeds=60).reshape(-1)[:K].astype(np.int64)).cuda()
    g = torch.Generator(device="cuda").manual_seed(79)
    F = torch.from_numpy(centres).cuda()[lab]
    F += torch.randn(F.shape, generator=g, device="cuda") * (0.6 / math.sqrt(d))
    Fb = F.to(torch.bfloat16)
    S = F[torch.randint(0, K, (N,), generator=g, device="cuda")].contiguous()
    del F, lab
    out = (torch.empty(K, dtype=torch.int32, device="cuda"), torch.empty(N, device="cuda"),
           torch.empty(N, device="cuda"), torch.empty(3, device="cuda"))
    ws = torch.empty(leg.le_quantize_workspace(N, d), dtype=torch.uint8, device="cuda")
    try:
        for _ in range(3):
            leg.le_quantize(Fb, S, out=out, workspace=ws)
        torch.cuda.synchronize()
        n = max(5, args.steps // 4)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(n):
            leg.le_quantize(Fb, S, out=out, workspace=ws)
        t1.record()
        torch.cuda.synchronize()
    except leg.LegError as e:
        return {"unavailable": str(e)[:200]}
    ms = t0.elapsed_time(t1) / n
    # the codebook gradient (le_quantize_grad: recompute D and write g / |F|, contraction over the features)
    gws = torch.empty(leg.le_quantize_grad_workspace(K, N, d), dtype=torch.uint8, device="cuda")
    grad = torch.empty((N, d), device="cuda")
    for _ in range(3):
        leg.le_quantize_grad(Fb, S, out[1], out=grad, workspace=gws)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(n):
        leg.le_quantize_grad(Fb, S, out[1], out=grad, workspace=gws)
    t1.record()
    torch.cuda.synchronize()
    ms_g = t0.elapsed_time(t1) / n
    bytes_g = 2 * K * d * 2 + 2 * 2 * K * N * 2       # features twice, g / |F| written and read (two parts)
    byts = K * d * 2 + K * 4 + N * d * 4
    flop = 2.0 * K * N * d
    return {"ms": round(ms, 4), "features": K, "dims": d, "codebook": N,
            "hbm": {"achieved_gbs": round(byts / ms / 1e6, 1), "peak": hbm_peak, "frac": round(byts / ms / 1e6 / hbm_peak, 4),
                    "peak_kind": peak_kind, "algorithmic_bytes": byts},
            "tensor": {"achieved_tflops": round(flop / ms / 1e9, 1), "peak": bf16_peak,
                       "frac": round(flop / ms / 1e9 / bf16_peak, 4)},
            "loss": [round(float(x), 6) for x in out[3].cpu()],
            "codebook_grad": {"ms": round(ms_g, 4), "hbm_frac": round(bytes_g / ms_g / 1e6 / hbm_peak, 4),
                              "algorithmic_bytes": bytes_g,
                              "note": "le_quantize_grad: 4 launches (prep, D recompute + g, split-K tcgen05 "
                                      "contraction, finalize); the codebook's Adam step is le_adam"}}


# ---------------------------------------------------------------------------
# Pixels of the oracle's decoder loss that one sampled oracle step times (the
# centre 128 x 128 window); every other stage runs on the full view.
ORACLE_DEC_PX = 16384
REF_BUDGET_S = 150.0      # host time of one --impl reference run (warm-up + timed oracle steps)


def reference_step(scene, dec, cam, rgb_target, idx_target, state, dec_px=ORACLE_DEC_PX):
    """The FP64 oracle doing one training step of the workload, sampled only where its
    cost does not depend on the scene: the key path, projection, binning (the oracle's
    stable sort of all tile copies), compositing, RGB L1, compositing adjoint,
    projection adjoint and Adam all run on the full view and all N Gaussians; the
    decoder loss (a dense per-pixel MLP, the same work for every pixel) runs on
    `dec_px` pixels of the centre and is scaled to the view.  The compositing adjoint
    gets the sampled pixels' decoder gradients and zeros elsewhere (its cost does not
    depend on the values).  Returns (measured seconds, estimated full-step seconds,
    per-stage seconds)."""
    import numpy as np
    import oracle
    P = cam.W * cam.H
    side = int(round(dec_px ** 0.5))
    x0, y0 = cam.W // 2 - side // 2, cam.H // 2 - side // 2
    sel = (slice(y0, y0 + side), slice(x0, x0 + side))
    npx = side * side
    tm = {}

    def timed(name, f):
        t = time.perf_counter()
        r = f()
        tm[name] = time.perf_counter() - t
        return r

    kp = timed("keypath", lambda: oracle.keypath(scene, cam))
    pr = timed("project", lambda: oracle.project(scene, cam, kp["tiles"]))
    _, vals, rr = timed("bin", lambda: oracle.bin(cam, kp))
    img = timed("render", lambda: oracle.render(cam, scene, pr, vals, rr))
    l1, d_rgb = timed("l1", lambda: oracle.l1(img["rgb"], rgb_target))
    dl = timed("decoder", lambda: oracle.decoder_loss(img["feat"][:, sel[0], sel[1]].reshape(8, -1),
                                                        img["unc"][sel].reshape(-1), idx_target[sel].reshape(-1),
                                                        dec))
    d_feat = np.zeros((8, cam.H, cam.W))
    d_unc = np.zeros((cam.H, cam.W))
    d_feat[:, sel[0], sel[1]] = dl["d_feat"].reshape(8, side, side)
    d_unc[sel] = dl["d_unc"].reshape(side, side)
    g2 = timed("render_bwd", lambda: oracle.render_bwd(cam, scene, pr, vals, rr, d_rgb, d_feat, d_unc))
    gp = timed("project_bwd", lambda: oracle.project_bwd(scene, cam, kp["tiles"], g2["mean2d"], g2["conic"],
                                                          g2["opacity"], g2["rgb"]))

    def adam():
        flat_g = np.concatenate([gp["means"].ravel(), gp["log_scales"].ravel(), gp["quats"].ravel(),
                                 gp["opacity_raw"].ravel(), gp["sh"].ravel(), g2["feat"].ravel(), g2["unc"].ravel()])
        if state.get("p") is None:
            state["p"] = np.concatenate([scene.means.ravel(), scene.log_scales.ravel(), scene.quats.ravel(),
                                         scene.opacity_raw.ravel(), scene.sh.ravel(), scene.feat.ravel(),
                                         scene.unc.ravel()]).astype(np.float64)
            state["m"] = np.zeros_like(state["p"])
            state["v"] = np.zeros_like(state["p"])
            state["step"] = 0
        state["step"] += 1
        oracle.adam(state["p"], flat_g, state["m"], state["v"], state["step"])
    timed("adam", adam)
    measured = sum(tm.values())
    est = measured + tm["decoder"] * (P / npx - 1.0)
    return measured, est, tm


def oracle_sample_text(npx, cores):
    return (f"FP64 oracle training step on {cores} host threads: key path, projection, full binning, "
            f"compositing, L1, compositing adjoint, projection adjoint and Adam on the full 1296x840 view and all "
            f"Gaussians; the decoder loss (dense per-pixel MLP) on the {npx} centre pixels, scaled "
            f"x{W * H / npx:.1f} to the view")


def cpu_baseline(scene, dec, cam, rgb_target, idx_target, budget_s=20.0):
    import oracle
    oracle.build()
    state = {}
    ests, meas, n = [], [], 0
    start = time.perf_counter()
    while n == 0 or (time.perf_counter() - start < budget_s and n < 3):
        m, e, tm = reference_step(scene, dec, cam, rgb_target, idx_target, state)
        meas.append(m)
        ests.append(e)
        n += 1
    est = min(ests)
    return {"value": round(est * 1e3, 1), "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
            "sample": oracle_sample_text(ORACLE_DEC_PX, os.cpu_count()) + f"; best of {n} steps, "
                      f"{min(meas):.1f} s of it measured",
            "stages_s": {k: round(v, 3) for k, v in tm.items()}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import numpy as np
    scene, dec, cams, rgb_host, idx_host = setup_workload(args.n, pin=False)
    import oracle
    oracle.build()
    state = {}
    rgb, idx = rgb_host.numpy(), idx_host.numpy()
    # the oracle has nothing to warm beyond its first call, and each of its steps takes seconds: one
    # warm-up step at most, then steps until K are done or REF_BUDGET_S of host time is spent (>= 1)
    t0 = time.perf_counter()
    for i in range(min(args.warmup, 1)):
        reference_step(scene, dec, cams[i % N_VIEWS], rgb[i % N_VIEWS], idx[i % N_VIEWS], state)
    est, meas = [], []
    for i in range(args.steps):
        if est and time.perf_counter() - t0 > REF_BUDGET_S:
            break
        k = (args.warmup + i) % N_VIEWS
        m, e, _ = reference_step(scene, dec, cams[k], rgb[k], idx[k], state)
        est.append(e)
        meas.append(m)
    ms = 1e3 * float(np.mean(est))
    cb = {"kind": "oracle", "cores": os.cpu_count(), "value": round(ms, 1), "unit": "ms",
          "sample": oracle_sample_text(ORACLE_DEC_PX, os.cpu_count()) + f"; measured {np.mean(meas):.2f} s per step; "
                    f"{len(est)} of {args.steps} requested steps timed within a {REF_BUDGET_S:.0f} s budget"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms", "n_gpus": world,
                      "steps": args.steps, "steps_timed": len(est), "warmup": args.warmup, "ms_per_step": round(ms, 1),
                      "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic (seeded 50-cluster scene, Voronoi index maps, smooth RGB targets)",
                      "config": workload_config(args.n, world), "cpu_baseline": cb,
                      "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def decode_query_leg(leg, synth, args, hbm, kind):
    """The query's decode + relevancy kernel and the feature-map export alone, on
    --features pixels of N(0, 1) rendered features (256 codes, 896 dims)."""
    import torch
    P = args.features
    dec = synth.decoder_init(103, 256)
    qin = synth.query_inputs(303, 256)
    t = lambda a: torch.from_numpy(a).cuda().contiguous()
    dec_t = tuple(t(getattr(dec, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    cb, text, negs = t(qin.codebook), t(qin.text), t(qin.negs)
    feat = torch.randn((8, P), generator=torch.Generator(device="cuda").manual_seed(1), device="cuda")
    ws = torch.empty(max(leg.le_query_workspace(leg.FUSED_BF16, P, 256, qin.d_clip), 1), dtype=torch.uint8,
                     device="cuda")
    rel = torch.empty((4, P), dtype=torch.float32, device="cuda")
    Fm = torch.empty((P, qin.codebook.shape[1]), dtype=torch.bfloat16, device="cuda")
    calls = {"query": lambda: leg.le_query(leg.FUSED_BF16, P, cb, qin.d_clip, text, negs, feat=feat, dec_t=dec_t,
                                           workspace=ws, out=rel),
             "feature_map": lambda: leg.le_feature_map(feat, dec_t, cb, out=Fm)}
    res = {"pixels": P}
    for name, f in calls.items():
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(5, args.steps)
        t0.record()
        for _ in range(n):
            f()
        t1.record()
        torch.cuda.synchronize()
        res[name + "_ms"] = round(t0.elapsed_time(t1) / n, 4)
    leg.le_device_status()
    byts = P * qin.codebook.shape[1] * 2 + P * 8 * 4
    res["feature_map_hbm_frac"] = round(byts / res["feature_map_ms"] / 1e6 / hbm, 4)
    res["peak_kind"] = kind
    return res


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.only is not None:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_2311_18482_gb300 as leg
        from paper_2311_18482_gb300 import synth
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        leg.load()
        hbm, bf16, kind = measured_peaks()
        if args.only == "quantize":
            res = quant_leg(leg, synth, args, hbm, bf16, kind)
        elif args.only == "query":
            res = decode_query_leg(leg, synth, args, hbm, kind)
        elif args.only == "decoder_wide":
            res = decoder_wide_leg(leg, synth, args, bf16, P=args.features)
        elif args.only == "configs":
            res = configs_leg(leg, synth, args)
        else:
            from paper_2311_18482_gb300.training import TrainState
            c = synth.config("c5", n=args.n)
            res = smooth_leg(leg, synth, TrainState(c["scene"], c["decoder"], W, H, "cuda"), args, bf16)
        print(json.dumps({"leg": args.only, **res}), flush=True)
        return
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
