#!/usr/bin/env python3
"""Benchmark: Cascade-of-Gaussians background subtraction on GB300.

One step = one 1920x1080 frame of a synthetic surveillance stream through
the whole cascade (one cog_apply call: two kernel launches), K = 5
Gaussians, FP16 model state
with FP32 arithmetic.  Frames are generated on the device before timing;
the L2 cache is flushed (a 512 MB write) between timed frames and each
frame is timed with CUDA events on the stream the kernel runs on.  The
plain full-GMM path runs over the same frames with the same protocol.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); each rank owns its own camera
stream (pixels and streams are independent), no data-path collective;
weak scaling.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload (one band of rows per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CoG Mpixel/s and % HBM peak vs plain full-GMM on same GB300; mask agreement vs FP64"
UNIT = "Mpixel/s"
W_, H_, K_ = 1920, 1080, 5
N_TRAIN = 500
N_TEST_MAX = 2000
FALLBACK_HBM = 6800.0


def stream_seed(base: int, rank: int) -> int:
    """Each rank owns its own camera stream (weak scaling, no exchange)."""
    return base + rank


def max_over_ranks(values, world: int, device=None):
    """Max of per-rank timings (the slowest rank defines the job's time).
    The only collective the benchmark uses; it carries no pixel data."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_mpixel_per_s(pixels_per_step: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank processed its own stream's pixels in
    at most ms_max milliseconds."""
    return world * pixels_per_step * steps / (ms_max / 1e3) / 1e6


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


# ---------------------------------------------------------------- byte model
def cog_bytes(stats: dict, P: int, elem: int, K: int, nv: int = 7):
    """Algorithmic bytes the cascade touches over a set of frames, from the
    per-stage occupancy counters and the per-stage byte table:
      every pixel (stage 0, first kernel): reads I, J, label, C and writes
        mask, label, C: 3+3+1+e + 1+1+e bytes;
      a pixel past stage 0 (first kernel): reads the residue weights and the
        running average and writes the running average: 2 + 12e;
      a pixel at the mixture stage (second kernel): reads and writes its K*7
        parameters, reads three prior bytes counted as 32-byte sectors, and
        reseeds the running average: 14Ke + 96 + 6e.
    Returns (first kernel, second kernel) bytes."""
    n = stats["n_stage"]
    frames = stats["frames"]
    past0 = n[1] + stats["n_gmm"]
    skipped = n[5] if len(n) > 5 else 0
    # a pixel skipped by the temporal sampling reads J, label and C and
    # writes its mask: 3 + 1 + e + 1
    k1 = (frames * P - skipped) * (9 + 2 * elem) + skipped * (5 + elem) + past0 * (2 + 12 * elem)
    k2 = stats["n_gmm"] * (2 * nv * K * elem + 96 + 6 * elem)   # nv = 7, or 9 per-channel
    return int(k1), int(k2)


def clip_bytes(stats: dict, P: int, elem: int, K: int, clips: int) -> int:
    """Algorithmic bytes of the clip path over `clips` launches:
      per pixel and launch, its stage-0/1 state (previous frame + label 4,
        C e, running average and residue weights 6e + 2) read once, written
        once and copied once to the undo log: 3 (6 + 7e);
      per pixel and frame, the frame's 3 bytes in and the mask byte out;
      per pixel at the mixture stage, its K*7 parameters read and written
        and three prior bytes counted as 32-byte sectors: 14Ke + 96.
    (The undo copies of touched mixture records are not counted.)"""
    per_pixel_frames = stats["frames"] * P
    return int(clips * P * 3 * (6 + 7 * elem) + per_pixel_frames * 4 + stats["n_gmm"] * (14 * K * elem + 96))


def plain_bytes(frames: int, P: int, elem: int, K: int) -> int:
    """The plain mixture reads I and the K*7 parameters and writes them
    back with the mask: 3 + 14Ke + 1 bytes per pixel."""
    return int(frames * P * (4 + 14 * K * elem))


# the files that define or instantiate the kernels (host-only files such as
# the ABI, the batch host code, the server and the self-test are left out)
KERNEL_SOURCES = ("cog_internal.h", "cog_device.cuh", "cog_apply.cuh", "cog_mixture.cuh", "cog_clip.cuh",
                  "cog_inst.cuh", "cog_f32.cu", "cog_f16.cu", "cog_bf16.cu", "cog_kde.cu")
# the sources each profiled kernel is compiled from: its counts stay valid
# while these are unchanged
APPLY_SOURCES = ("cog_internal.h", "cog_device.cuh", "cog_apply.cuh", "cog_inst.cuh", "cog_f32.cu", "cog_f16.cu",
                 "cog_bf16.cu")
SOURCES_OF = {"stage01_kernel": APPLY_SOURCES, "stage2_kernel": APPLY_SOURCES,
              "plain_gmm_kernel": APPLY_SOURCES + ("cog_mixture.cuh",),
              "clip_kernel": APPLY_SOURCES + ("cog_clip.cuh",),
              "group_features_kernel": ("cog_internal.h", "cog_device.cuh", "cog_group.cu")}


def source_hash(sources=KERNEL_SOURCES) -> str:
    """Hash of the kernel sources; ncu counts taken on other sources are not used."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1705_09339_gb300", "csrc")
    for f in sources:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_counts(kernel: str):
    """Per-launch ncu counts of the committed summary (DRAM bytes, warp
    instructions), if they were taken on the kernel's current sources."""
    sources = SOURCES_OF.get(kernel, KERNEL_SOURCES)
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(kernel)
        if e and e.get("source_hash") == source_hash(sources):
            return e
    except Exception:
        pass
    return None


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was
    taken on the current kernel sources; else None."""
    e = ncu_counts(kernel)
    return float(e["dram_bytes_per_launch"]) if e else None


# warp-instruction issue peak of the GPU: 152 SMs x 4 schedulers x one warp
# instruction per clock at the 2070 MHz maximum SM clock
ISSUE_PEAK = 152 * 4 * 2.070e9


def issue_rate(kernel: str, ms_per_launch: float):
    """Warp instructions per second the kernel issued (ncu count per launch
    over the live CUDA-event time) against the scheduler peak; None when the
    committed counts are not for the current sources."""
    e = ncu_counts(kernel)
    if not e or "warp_instructions_per_launch" not in e or ms_per_launch <= 0:
        return None
    a = float(e["warp_instructions_per_launch"]) / (ms_per_launch / 1e3)
    return {"achieved": round(a / 1e12, 4), "peak": round(ISSUE_PEAK / 1e12, 4), "unit": "Twarp-inst/s",
            "frac": round(a / ISSUE_PEAK, 4), "warp_instructions_per_launch": e["warp_instructions_per_launch"]}


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu,"
         "pstate,clocks.mem")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix=f"cog_clocks_{self.idx}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons, util, mem, pst = [], 0.0, set(), [], [], {}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        try:
            os.unlink(self.path)
        except OSError:
            pass
        for line in lines:
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                mx = max(mx, float(v[2]))
            except ValueError:
                continue
            for n, x in zip(names, v[5:9]):
                if x.lower().startswith("active"):
                    reasons.add(n)
            try:
                util.append(float(v[9]))
            except (IndexError, ValueError):
                pass
            if len(v) > 11:
                pst[v[10]] = pst.get(v[10], 0) + 1
                try:
                    mem.append(float(v[11]))
                except ValueError:
                    pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "gpu_util_pct_median": statistics.median(util) if util else None,
                "mem_mhz": statistics.median(mem) if mem else None, "pstates": pst}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, local_rank, world):
    import torch
    import torch.distributed as dist
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)          # create the context before setting its limit
    if args.l2_fetch >= 0:
        cog.cog_set_l2_fetch_bytes(args.l2_fetch)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    wl = workload("hd_dynamic", fg_frac=args.fg, seed=stream_seed(3, rank))
    sc = wl["scene"]
    P = sc.P
    n_test = args.warmup + 2 * args.steps
    if n_test > N_TEST_MAX:
        raise SystemExit(f"--warmup + 2 * --steps must be <= {N_TEST_MAX} test frames")
    stream = torch.cuda.current_stream(dev)
    gs = GpuScene(sc, dev)
    train = gs.render(0, N_TRAIN)
    test, gt = gs.render(N_TRAIN, n_test, gt=True)
    p_cog = cog.cog_default_params(W_, H_, K_, state_dtype="f16")
    if args.sample:
        p_cog.flags |= cog.COG_SAMPLE
    if args.mode1:
        p_cog.flags |= cog.COG_MODE1
    if args.perchan:
        p_cog.flags |= cog.COG_PERCHAN
    p_cog.kde_bits = args.kde_bits
    p_gmm = cog.cog_default_params(W_, H_, K_, state_dtype="f16")
    tuned = None
    if args.autotune:
        from paper_1705_09339_gb300 import autotune
        tuned = autotune.tune(p_cog, train, test[:15], n_frames=12, warmup=3)
    ctx = cog.cog_create(p_cog, stream.cuda_stream)
    ctx_g = cog.cog_create(p_gmm, stream.cuda_stream)
    shape = tuple(tuned["best"]) if tuned else (128, 64, 0)
    cog.cog_set_launch(ctx, *shape)
    cog.cog_train_prior(ctx_g, train, N_TRAIN)
    # training (scene prior, residue weights, mixture warm-up) on the same
    # 500 frames, timed once with CUDA events
    ev_t = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    ev_t[0].record(stream)
    cog.cog_train_prior(ctx, train, N_TRAIN)
    ev_t[1].record(stream)
    torch.cuda.synchronize()
    ms_train = ev_t[0].elapsed_time(ev_t[1])
    cog.cog_sync(ctx)
    del train
    torch.cuda.empty_cache()
    masks = torch.empty((n_test, H_, W_), dtype=torch.uint8, device=dev)
    masks_g = torch.empty((n_test, H_, W_), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, first, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            fn(first + i)
            ev[i][1].record(stream)
        return ev

    for i in range(args.warmup):
        cog.cog_apply(ctx, test[i], masks[i])
        cog.cog_apply_plain_gmm(ctx_g, test[i], masks_g[i])
    cog.cog_sync(ctx)
    _, tot0 = cog.cog_read_stats(ctx)
    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ev_c = timed(lambda i: cog.cog_apply(ctx, test[i], masks[i]), args.warmup, args.steps)
    torch.cuda.synchronize()
    ev_g = timed(lambda i: cog.cog_apply_plain_gmm(ctx_g, test[i], masks_g[i]), args.warmup, args.steps)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    cog.cog_sync(ctx)
    _, tot1 = cog.cog_read_stats(ctx)
    # per-kernel durations: a second timed pass over the next K frames with
    # CUDA events around each of the two kernels on their stream (events
    # between the kernels serialise them, so the main pass above runs
    # without them and lets the second kernel's launch overlap the first)
    cog.cog_profile_begin(ctx, args.steps)
    timed(lambda i: cog.cog_apply(ctx, test[i], masks[i]), args.warmup + args.steps, args.steps)
    ms_k1, ms_k2, nprof = cog.cog_profile_end(ctx)
    _, tot2 = cog.cog_read_stats(ctx)
    # the streaming floor at this size: the probe kernel moves stage 0's
    # planes (16 B per pixel, no arithmetic) under the same flush and events
    pr_jl = torch.randint(0, 2**31, (P,), dtype=torch.int32, device=dev)
    pr_c = torch.randint(0, 2**15, (P,), dtype=torch.int16, device=dev)
    pr_jo, pr_co = torch.empty_like(pr_jl), torch.empty_like(pr_c)
    pr_m = torch.empty((P,), dtype=torch.uint8, device=dev)
    probe = lambda i: cog.cog_probe_stream(pr_jl, pr_c, test[i], pr_jo, pr_co, pr_m, stream.cuda_stream)
    ms_p = None
    if P % 4 == 0 and (P * 3) % 16 == 0:   # the probe's frame words stay 16-byte aligned
        timed(probe, 0, 3)
        ev_p = timed(probe, args.warmup, args.steps)
        torch.cuda.synchronize()
        ms_p = sum(a.elapsed_time(b) for a, b in ev_p)
    del pr_jl, pr_c, pr_jo, pr_co, pr_m
    ms_c = sum(a.elapsed_time(b) for a, b in ev_c)
    ms_g = sum(a.elapsed_time(b) for a, b in ev_g)
    st = dict(n_stage=[b - a for a, b in zip(tot0["n_stage"], tot1["n_stage"])],
              n_gmm=tot1["n_gmm"] - tot0["n_gmm"], frames=args.steps)
    st_prof = dict(n_stage=[b - a for a, b in zip(tot1["n_stage"], tot2["n_stage"])],
                   n_gmm=tot2["n_gmm"] - tot1["n_gmm"], frames=args.steps)
    ms_c, ms_g = max_over_ranks([ms_c, ms_g], world, dev)

    # accuracy against the generator's ground truth on the timed frames:
    # misclassified pixels (mask != ground truth), and their split into
    # false positives and false negatives, for the cascade and the plain
    # mixture (the paper's comparison, Sec. 3.2)
    def misclass(mk):
        m = mk[args.warmup:args.warmup + args.steps] > 0
        g = gt[args.warmup:args.warmup + args.steps] > 0
        n = float(m.numel())
        return {"misclassified": round(float((m != g).sum()) / n, 6),
                "false_positive": round(float((m & ~g).sum()) / n, 6),
                "false_negative": round(float((~m & g).sum()) / n, 6)}
    acc = {"cog": misclass(masks), "plain_gmm": misclass(masks_g),
           "ground_truth_foreground": round(float((gt[args.warmup:args.warmup + args.steps] > 0).float().mean()), 6),
           "frames": args.steps}
    del gt

    # end to end through the C ABI with host buffers (pinned): a fresh
    # context trained on the same frames takes the stream's first warm-up
    # frames untimed, then three timed rounds of consecutive, never repeated
    # frames -- the frames the device-timed pass above ran -- so the model
    # advances through the stream as it would live
    n_e2e = max(1, args.steps // 3)
    host_frames = test[:args.warmup + 3 * n_e2e].cpu().pin_memory()
    host_masks = torch.empty((args.warmup + 3 * n_e2e, H_, W_), dtype=torch.uint8).pin_memory()
    hf, hm = host_frames.numpy(), host_masks.numpy()
    ctx_e = cog.cog_create(p_cog, stream.cuda_stream)
    tr2 = gs.render(0, N_TRAIN)
    cog.cog_train_prior(ctx_e, tr2, N_TRAIN)
    cog.cog_sync(ctx_e)
    del tr2
    cog.cog_apply_host_frames(ctx_e, hf[:args.warmup], hm[:args.warmup])   # creates the pipeline's slots
    if world > 1:
        dist.barrier()
    t_rounds = []
    for r in range(3):
        a = args.warmup + r * n_e2e
        t0 = time.perf_counter()
        cog.cog_apply_host_frames(ctx_e, hf[a:a + n_e2e], hm[a:a + n_e2e])
        t_rounds.append(time.perf_counter() - t0)
    t_e2e = sorted(t_rounds)[1]
    # and the synchronous per-frame call, for comparison (a second fresh
    # context over the same frames)
    ctx_s = cog.cog_create(p_cog, stream.cuda_stream)
    tr2 = gs.render(0, N_TRAIN)
    cog.cog_train_prior(ctx_s, tr2, N_TRAIN)
    cog.cog_sync(ctx_s)
    del tr2
    for i in range(args.warmup):
        cog.cog_apply_host(ctx_s, hf[i], hm[i])
    t_sync_rounds = []
    for r in range(3):
        a = args.warmup + r * n_e2e
        t0 = time.perf_counter()
        for i in range(a, a + n_e2e):
            cog.cog_apply_host(ctx_s, hf[i], hm[i])
        t_sync_rounds.append(time.perf_counter() - t0)
    t_e2e_sync = sorted(t_sync_rounds)[1]
    t_e2e, t_e2e_sync = max_over_ranks([t_e2e, t_e2e_sync], world, dev)
    cog.cog_destroy(ctx_e)
    cog.cog_destroy(ctx_s)
    del host_frames, host_masks, hf, hm

    result = None
    if rank == 0:
        hbm, hbm_src = peaks()
        value = job_mpixel_per_s(P, args.steps, ms_c, world)
        value_g = job_mpixel_per_s(P, args.steps, ms_g, world)
        nv = 9 if args.perchan else 7
        bytes_c = sum(cog_bytes(st, P, 2, K_, nv))
        b1, b2 = cog_bytes(st_prof, P, 2, K_, nv)
        bytes_g = plain_bytes(args.steps, P, 2, K_)
        ach_c = bytes_c / (ms_c / 1e3) / 1e9
        ach_g = bytes_g / (ms_g / 1e3) / 1e9
        ach_1 = b1 / (ms_k1 / 1e3) / 1e9
        ach_2 = b2 / (ms_k2 / 1e3) / 1e9 if ms_k2 > 0 else 0.0
        dom = "stage01_kernel" if ms_k1 >= ms_k2 else "stage2_kernel"
        ach_d, ms_d, b_d = (ach_1, ms_k1, b1) if dom == "stage01_kernel" else (ach_2, ms_k2, b2)
        tr_c = ncu_traffic(dom)
        tr_g = ncu_traffic("plain_gmm_kernel")
        occ = {k: v / (P * args.steps) for k, v in zip(("fd", "rga", "gmm_bg", "fg", "illum", "skipped"), st["n_stage"])}
        cpu = cpu_baseline(sc, masks[args.warmup:args.warmup + args.steps], args) if not args.no_cpu_baseline else None
        result = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_c / args.steps, 5), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{W_}x{H_} RGB u8 dynamic-background stream, K={K_}, FP16 state / FP32 math, "
                                   f"{N_TRAIN} train frames, fg {args.fg:.3f}, one frame per step"
                                   + (", temporal sampling on" if args.sample else "")
                                   + (", stage 1 = the mixture's rank-1 mode (Fig. 1 reading)" if args.mode1 else "")
                                   + (", per-channel independent mixtures" if args.perchan else ""),
                       "temporal_sampling": bool(args.sample), "mode1": bool(args.mode1), "kde_bits": args.kde_bits,
                       "perchan": bool(args.perchan),
                       "width": W_, "height": H_, "K": K_, "state_dtype": "f16", "n_train": N_TRAIN,
                       "fg_frac": args.fg, "l2": "flushed (512 MB write) between timed steps",
                       "l2_fetch_bytes": args.l2_fetch,
                       "launch_shape": {"k1_threads": shape[0], "k2_threads": shape[1], "k2_ctas_per_sm": shape[2],
                                        "chosen_by": "autotuner" if tuned else "default"},
                       "parallelism": f"stream-sharded x{world} (one camera per GPU, no collective)"},
            "roofline": {"bound": "hbm", "achieved": round(ach_d, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(ach_d / hbm, 4), "traffic": tr_c, "peak_source": hbm_src,
                         "kernel": dom, "ms_per_launch": round(ms_d / args.steps, 5),
                         "algorithmic_bytes_per_launch": b_d // args.steps,
                         "issue": issue_rate(dom, ms_d / args.steps),
                         "floor": None if ms_p is None else {"kernel": "probe_stream_kernel (cog_probe_stream)",
                                   "bytes_per_launch": 16 * P, "ms_per_launch": round(ms_p / args.steps, 5),
                                   "achieved": round(16 * P * args.steps / (ms_p / 1e3) / 1e9, 1),
                                   "frac_of_peak": round(16 * P * args.steps / (ms_p / 1e3) / 1e9 / hbm, 4),
                                   "kernel_frac_of_floor": round(ach_d / (16 * P * args.steps / (ms_p / 1e3) / 1e9), 4),
                                   "note": "stage 0's planes streamed with no arithmetic (9 B/px in, 7 out), "
                                           "one launch per frame under the same L2 flush and events: the "
                                           "bandwidth a pass of this size reaches at best"}},
            "kernels": {"stage01_kernel": {"ms_per_launch": round(ms_k1 / args.steps, 5),
                                           "achieved_gbs": round(ach_1, 1),
                                           "algorithmic_bytes_per_launch": b1 // args.steps},
                        "stage2_kernel": {"ms_per_launch": round(ms_k2 / args.steps, 5),
                                          "achieved_gbs": round(ach_2, 1),
                                          "algorithmic_bytes_per_launch": b2 // args.steps},
                        "profiled_frames": nprof,
                        "note": "second timed pass over the next K frames with CUDA events around each kernel"},
            "step_roofline": {"bound": "hbm", "achieved": round(ach_c, 1), "peak": hbm, "unit": "GB/s",
                              "frac": round(ach_c / hbm, 4), "algorithmic_bytes_per_step": bytes_c // args.steps},
            "plain_gmm": {"value": round(value_g, 1), "unit": UNIT, "ms_per_step": round(ms_g / args.steps, 5),
                          "roofline": {"bound": "hbm", "achieved": round(ach_g, 1), "peak": hbm, "unit": "GB/s",
                                       "frac": round(ach_g / hbm, 4), "traffic": tr_g,
                                       "algorithmic_bytes_per_step": bytes_g // args.steps}},
            "speedup_vs_plain_gmm": round(ms_g / ms_c, 3),
            "training": {"ms": round(ms_train, 3), "frames": N_TRAIN,
                         "bytes": 2 * N_TRAIN * P * 3 + P * 768 + P * (4 + 2 + 16 + 80),
                         "achieved_gbs": round((2 * N_TRAIN * P * 3 + P * 768 + P * (4 + 2 + 16 + 80))
                                               / (ms_train / 1e3) / 1e9, 1),
                         "note": "cog_train_prior: the prior kernel and the warm-up kernel each read the "
                                 "N frames; the prior (768 B/px) and the state are written"},
            "stage_occupancy": {k: round(v, 5) for k, v in occ.items()},
            "e2e": {"value": round(world * P * n_e2e / t_e2e / 1e6, 1), "unit": UNIT,
                    "h2d_bytes_per_step": P * 3, "d2h_bytes_per_step": P, "steps": n_e2e,
                    "rounds": [round(world * P * n_e2e / t / 1e6, 1) for t in t_rounds],
                    "api": "cog_apply_host_frames (pinned host frames in, masks out; uploads and downloads "
                           "overlap the kernels; returns when every mask is on the host)",
                    "protocol": f"three rounds of {n_e2e} consecutive frames each (the device-timed frames), "
                                f"never repeated, after {args.warmup} untimed frames through the same "
                                f"context; median round",
                    "per_frame_sync_value": round(world * P * n_e2e / t_e2e_sync / 1e6, 1),
                    "per_frame_sync_api": "cog_apply_host, one synchronous call per frame (median of three rounds "
                                          "over the same frames as the pipelined rounds)",
                    "per_frame_sync_rounds": [round(world * P * n_e2e / t / 1e6, 1) for t in t_sync_rounds]},
            "accuracy": acc,
            "gpu_launches": 2 * args.steps,
            "cpu_baseline": cpu,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 3),
        }
    for c in (ctx, ctx_g):
        cog.cog_destroy(c)
    if world > 1:
        dist.destroy_process_group()
    if result is not None and world == 1 and args.extras:
        # the other deployment forms of the same step, each in its own
        # timed region after this one: the 64-stream batch and the served
        # cameras
        del test, masks, masks_g, flush
        torch.cuda.empty_cache()
        result["batch64"] = sub_batch(args, rank, local_rank, world)
        torch.cuda.empty_cache()
        result["serve"] = sub_serve(args, rank, local_rank, world)
    return result


def sub_batch(args, rank, local_rank, world, steps=100, warmup=5) -> dict:
    """The 64-stream batch workload (run_batch) with a bounded number of
    steps, summarised for the default bench line."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = steps, warmup
    r = run_batch(a, rank, local_rank, world)
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "config", "roofline", "plain_gmm",
            "speedup_vs_plain_gmm", "stage_occupancy", "gpu_launches", "clocks")
    return {k: r[k] for k in keep if k in r}


def sub_serve(args, rank, local_rank, world, duration=60.0, cameras=256) -> dict:
    """The served-cameras workload (run_serve) for the specified 60 s of
    Poisson arrivals from 256 cameras, summarised for the default bench line."""
    import copy
    a = copy.copy(args)
    a.duration, a.cameras, a.timeline = duration, cameras, ""
    r = run_serve(a, rank, local_rank, world)
    keep = ("metric", "config", "latency_ms", "latency_split_ms", "frames", "steps", "aggregate_mpixel_per_s",
            "frame_period_ms", "p99_under_frame_period", "clocks", "h2d_probe")
    return {k: r[k] for k in keep if k in r}


# ------------------------------------------------------------ profile case
def run_profile_case(args, rank, local_rank, world):
    """The small case that detailed ncu captures run: the same 1080p stream
    and kernels as the default workload (K=5, FP16 state, default launch
    shape, 500 training frames, freed after training), but one context and
    only warmup + steps test frames on the device (about 2 GB held while
    the cascade runs), each frame after the same 512 MB L2 flush.  Prints
    the mean frame time and the stage occupancy; not a bench line."""
    import torch
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    if args.l2_fetch >= 0:
        cog.cog_set_l2_fetch_bytes(args.l2_fetch)
    sc = workload("hd_dynamic", fg_frac=args.fg, seed=3)["scene"]
    n_train, n_test = N_TRAIN, args.warmup + args.steps
    stream = torch.cuda.current_stream(dev)
    gs = GpuScene(sc, dev)
    train = gs.render(0, n_train)
    test = gs.render(n_train, n_test)
    p = cog.cog_default_params(W_, H_, K_, state_dtype="f16")
    if args.sample:
        p.flags |= cog.COG_SAMPLE
    ctx = cog.cog_create(p, stream.cuda_stream)
    if args.launch:
        cog.cog_set_launch(ctx, *[int(x) for x in args.launch.split(",")])
    cog.cog_train_prior(ctx, train, n_train)
    cog.cog_sync(ctx)
    del train
    torch.cuda.empty_cache()
    masks = torch.empty((n_test, H_, W_), dtype=torch.uint8, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_test)]
    for i in range(n_test):
        if i == args.warmup:
            cog.cog_sync(ctx)
            _, tot0 = cog.cog_read_stats(ctx)
        flush.zero_()
        ev[i][0].record(stream)
        cog.cog_apply(ctx, test[i], masks[i])
        ev[i][1].record(stream)
    cog.cog_sync(ctx)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev[args.warmup:]]
    _, tot1 = cog.cog_read_stats(ctx)
    cog.cog_destroy(ctx)
    occ = [(b - a) / (W_ * H_ * args.steps) for a, b in zip(tot0["n_stage"], tot1["n_stage"])]
    return {"profile_case": f"{W_}x{H_} dynamic stream, K={K_}, FP16, {n_train} training frames",
            "frames": args.steps, "ms_per_frame": round(sum(ms) / len(ms), 5),
            "stage_occupancy": [round(x, 4) for x in occ]}


# ---------------------------------------------------------------- clips
CLIP_T = 32


def run_clip(args, rank, local_rank, world):
    """Recorded video: one step = one launch of cog_apply_clip over the next
    32 frames of the 1920x1080 stream (results identical to 32 cog_apply
    calls).  Per-frame cascade and plain mixture run over the same frames,
    32 launches per step, with the same L2 flush between steps."""
    import torch
    import torch.distributed as dist
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    if args.l2_fetch >= 0:
        cog.cog_set_l2_fetch_bytes(args.l2_fetch)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    T = CLIP_T
    n_test = (args.warmup + args.steps) * T
    if n_test > N_TEST_MAX:
        raise SystemExit(f"clip workload: (--warmup + --steps) * {T} must be <= {N_TEST_MAX} test frames")
    sc = workload("hd_dynamic", fg_frac=args.fg, seed=stream_seed(3, rank))["scene"]
    P = sc.P
    stream = torch.cuda.current_stream(dev)
    gs = GpuScene(sc, dev)
    train = gs.render(0, N_TRAIN)
    test, gt = gs.render(N_TRAIN, n_test, gt=True)
    p_cog = cog.cog_default_params(W_, H_, K_, state_dtype="f16")
    ctxs = {k: cog.cog_create(p_cog, stream.cuda_stream) for k in ("clip", "frame", "plain")}
    for c in ctxs.values():
        cog.cog_train_prior(c, train, N_TRAIN)
    cog.cog_sync(ctxs["clip"])
    del train
    torch.cuda.empty_cache()
    masks = {k: torch.empty((n_test, H_, W_), dtype=torch.uint8, device=dev) for k in ctxs}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(kind, j):
        sl = slice(j * T, (j + 1) * T)
        if kind == "clip":
            cog.cog_apply_clip(ctxs["clip"], test[sl], T, masks["clip"][sl])
        else:
            f = cog.cog_apply if kind == "frame" else cog.cog_apply_plain_gmm
            for i in range(j * T, (j + 1) * T):
                f(ctxs[kind], test[i], masks[kind][i])

    def timed(kind):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step(kind, args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    for k in range(args.warmup):
        for kind in ctxs:
            step(kind, k)
    cog.cog_sync(ctxs["clip"])
    _, tot0 = cog.cog_read_stats(ctxs["clip"])
    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    ms = {kind: timed(kind) for kind in ("clip", "frame", "plain")}
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    _, tot1 = cog.cog_read_stats(ctxs["clip"])
    runs = cog.cog_clip_runs(ctxs["clip"])
    same = bool(torch.equal(masks["clip"][args.warmup * T:], masks["frame"][args.warmup * T:]))
    st = dict(n_stage=[b - a for a, b in zip(tot0["n_stage"], tot1["n_stage"])],
              n_gmm=tot1["n_gmm"] - tot0["n_gmm"], frames=args.steps * T)
    ms_c, ms_f, ms_g = max_over_ranks([ms["clip"], ms["frame"], ms["plain"]], world, dev)

    # end to end: each step copies its 32 frames from pinned host memory,
    # runs the clip and copies the 32 masks back
    n_e2e = min(args.steps, 8)
    hf = test[args.warmup * T:(args.warmup + n_e2e) * T].cpu().pin_memory()
    hm = torch.empty((n_e2e * T, H_, W_), dtype=torch.uint8).pin_memory()
    dfr = torch.empty((T, H_, W_, 3), dtype=torch.uint8, device=dev)
    dmk = torch.empty((T, H_, W_), dtype=torch.uint8, device=dev)
    ctx_e = cog.cog_create(p_cog, stream.cuda_stream)
    tr2 = gs.render(0, N_TRAIN)
    cog.cog_train_prior(ctx_e, tr2, N_TRAIN)
    del tr2
    cog.cog_sync(ctx_e)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(n_e2e):
        dfr.copy_(hf[k * T:(k + 1) * T], non_blocking=True)
        cog.cog_apply_clip(ctx_e, dfr, T, dmk)
        hm[k * T:(k + 1) * T].copy_(dmk, non_blocking=True)
        stream.synchronize()
    t_e2e = max_over_ranks([time.perf_counter() - t0], world, dev)[0]
    cog.cog_destroy(ctx_e)

    result = None
    if rank == 0:
        hbm, hbm_src = peaks()
        frames = args.steps * T
        b_clip = clip_bytes(st, P, 2, K_, args.steps)
        ach = b_clip / (ms_c / 1e3) / 1e9
        tr = ncu_traffic("clip_kernel")
        cpu = cpu_baseline(sc, masks["clip"][args.warmup * T:(args.warmup + args.steps) * T],
                           argparse.Namespace(steps=frames, warmup=args.warmup * T)) if not args.no_cpu_baseline else None
        occ = {k: v / (P * frames) for k, v in zip(("fd", "rga", "gmm_bg", "fg", "illum", "skipped"), st["n_stage"])}
        result = {
            "metric": METRIC, "value": round(job_mpixel_per_s(P, frames, ms_c, world), 1), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_c / args.steps, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{W_}x{H_} RGB u8 dynamic-background stream (recorded video), K={K_}, "
                                   f"FP16 state / FP32 math, {N_TRAIN} train frames, fg {args.fg:.3f}, "
                                   f"{T} frames per step (one cog_apply_clip launch)",
                       "width": W_, "height": H_, "K": K_, "state_dtype": "f16", "n_train": N_TRAIN,
                       "frames_per_step": T, "fg_frac": args.fg,
                       "l2": "flushed (512 MB write) between timed steps; a step's 32 frames (199 MB) exceed L2",
                       "l2_fetch_bytes": args.l2_fetch,
                       "parallelism": f"stream-sharded x{world} (one camera per GPU, no collective)"},
            "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(ach / hbm, 4), "traffic": tr, "peak_source": hbm_src,
                         "kernel": "clip_kernel", "ms_per_launch": round(ms_c / args.steps, 5),
                         "algorithmic_bytes_per_launch": b_clip // args.steps,
                         "issue": issue_rate("clip_kernel", ms_c / args.steps)},
            "per_frame_cog": {"value": round(job_mpixel_per_s(P, frames, ms_f, world), 1), "unit": UNIT,
                              "ms_per_frame": round(ms_f / frames, 5),
                              "masks_identical_to_clip": same},
            "plain_gmm": {"value": round(job_mpixel_per_s(P, frames, ms_g, world), 1), "unit": UNIT,
                          "ms_per_frame": round(ms_g / frames, 5)},
            "speedup_vs_plain_gmm": round(ms_g / ms_c, 3),
            "speedup_vs_per_frame_cog": round(ms_f / ms_c, 3),
            "clip_runs_last_launch": runs,
            "stage_occupancy": {k: round(v, 5) for k, v in occ.items()},
            "e2e": {"value": round(world * P * n_e2e * T / t_e2e / 1e6, 1), "unit": UNIT,
                    "h2d_bytes_per_step": T * P * 3, "d2h_bytes_per_step": T * P, "steps": n_e2e,
                    "api": "pinned host frames -> device, cog_apply_clip, masks -> pinned host, per step"},
            "gpu_launches": args.steps,
            "cpu_baseline": cpu,
            "clocks": clk,
            "wall_s_timed_region": round(t_wall, 3),
        }
    for c in ctxs.values():
        cog.cog_destroy(c)
    if world > 1:
        dist.destroy_process_group()
    return result


# ---------------------------------------------------------------- batched
SIZES = [(160, 120), (320, 240), (640, 480), (1280, 720), (1920, 1080)]


def run_batch(args, rank, local_rank, world):
    """64 camera streams of uneven resolution (drawn uniformly from five
    sizes), K = 3 or 5 per stream, FP16 state, 100 training frames each,
    1-5 % foreground; one step = one frame of every stream through
    cog_batch_apply (one captured CUDA graph).  The working set of a step is
    far larger than L2, so no flush is needed between steps."""
    import torch
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    if args.l2_fetch >= 0:
        cog.cog_set_l2_fetch_bytes(args.l2_fetch)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    rng = np.random.default_rng(4 + 1000 * rank)
    NS, NT = 64, 100
    nf = args.warmup + args.steps
    stream = torch.cuda.Stream(dev)
    specs, ctxs, ctxg, frames, masks = [], [], [], [], []
    with torch.cuda.stream(stream):
        for i in range(NS):
            w, h = SIZES[int(rng.integers(0, 5))]
            k = int(rng.choice([3, 5]))
            fg = float(rng.uniform(0.01, 0.05))
            sc = Scene(w, h, 5000 + 64 * rank + i, kind="dynamic", n_train=NT, fg_frac=fg, switch_at=10 ** 6)
            gs = GpuScene(sc, dev)
            tr = gs.render(0, NT)
            p = cog.cog_default_params(w, h, k, state_dtype="f16")
            c = cog.cog_create(p, stream.cuda_stream)
            g = cog.cog_create(p, stream.cuda_stream)
            cog.cog_train_prior(c, tr, NT)
            cog.cog_train_prior(g, tr, NT)
            cog.cog_sync(c)
            del tr
            frames.append(gs.render(NT, nf))
            masks.append(torch.empty((h, w), dtype=torch.uint8, device=dev))
            specs.append((w, h, k, fg))
            ctxs.append(c)
            ctxg.append(g)
    P_tot = sum(w * h for w, h, _, _ in specs)
    # launch shape of the batch kernels (each group takes its first stream's
    # cog_set_launch shape when the batch is created): the fastest of four
    # over three steps each, on the warm-up frames
    shape, chosen = (128, 64, 0), "default"
    if args.autotune:
        best = None
        for sh in ((128, 64, 0), (256, 64, 0), (128, 128, 0), (256, 128, 0)):
            for c in ctxs:
                cog.cog_set_launch(c, *sh)
            bt = cog.cog_batch_create(ctxs, stream.cuda_stream)
            with torch.cuda.stream(stream):
                cog.cog_batch_apply(bt, [f[0] for f in frames], masks)
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for t in range(1, 4):
                    cog.cog_batch_apply(bt, [f[t % max(1, args.warmup)] for f in frames], masks)
                e.record(stream)
            cog.cog_batch_sync(bt)
            cog.cog_batch_destroy(bt)
            ms_sh = a.elapsed_time(e)
            if best is None or ms_sh < best[0]:
                best = (ms_sh, sh)
        shape, chosen = best[1], "autotuner (4 shapes, 3 steps each on the warm-up frames)"
        for c in ctxs:
            cog.cog_set_launch(c, *shape)
    b = cog.cog_batch_create(ctxs, stream.cuda_stream)
    with torch.cuda.stream(stream):
        for t in range(args.warmup):
            cog.cog_batch_apply(b, [f[t] for f in frames], masks)
            for c, f, m in zip(ctxg, frames, masks):
                cog.cog_apply_plain_gmm(c, f[t], m)
        cog.cog_batch_sync(b)
        tot0 = [cog.cog_read_stats(c)[1] for c in ctxs]
        clocks = Clocks(local_rank)
        clocks.start()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = []
        for t in range(args.warmup, nf):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cog.cog_batch_apply(b, [f[t] for f in frames], masks)
            e.record(stream)
            ev.append((a, e))
        torch.cuda.synchronize()
        evg = []
        for t in range(args.warmup, nf):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for c, f, m in zip(ctxg, frames, masks):
                cog.cog_apply_plain_gmm(c, f[t], m)
            e.record(stream)
            evg.append((a, e))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clk = clocks.stop()
        cog.cog_batch_sync(b)
    ms = sum(a.elapsed_time(e) for a, e in ev)
    ms_g = sum(a.elapsed_time(e) for a, e in evg)
    ms, ms_g = max_over_ranks([ms, ms_g], world, dev)
    tot1 = [cog.cog_read_stats(c)[1] for c in ctxs]
    bytes_c = bytes_g = 0
    occ = np.zeros(6)
    for (w, h, k, _), a0, a1 in zip(specs, tot0, tot1):
        st = dict(n_stage=[y - x for x, y in zip(a0["n_stage"], a1["n_stage"])], n_gmm=a1["n_gmm"] - a0["n_gmm"],
                  frames=args.steps)
        bytes_c += sum(cog_bytes(st, w * h, 2, k))
        bytes_g += plain_bytes(args.steps, w * h, 2, k)
        occ += np.array(st["n_stage"])
    cog.cog_batch_destroy(b)
    for c in ctxs + ctxg:
        cog.cog_destroy(c)
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return None
    hbm, src = peaks()
    ach = bytes_c / (ms / 1e3) / 1e9
    ach_g = bytes_g / (ms_g / 1e3) / 1e9
    mix = {f"{w}x{h}": sum(1 for s in specs if s[:2] == (w, h)) for (w, h) in SIZES}
    return {
        "metric": METRIC, "value": round(world * P_tot * args.steps / (ms / 1e3) / 1e6, 1), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch of {NS} streams of uneven resolution per rank, K=3/5, FP16 state, "
                               f"{NT} train frames, one frame of every stream per step (cog_batch_apply, captured graph)",
                   "streams": NS, "pixels_per_step": P_tot, "size_mix": mix,
                   "K_mix": {"3": sum(1 for s in specs if s[2] == 3), "5": sum(1 for s in specs if s[2] == 5)},
                   "l2": "working set per step far larger than L2 (no flush)", "l2_fetch_bytes": args.l2_fetch,
                   "launch_shape": {"k1_threads": shape[0], "k2_threads": shape[1], "k2_ctas_per_sm": shape[2],
                                    "chosen_by": chosen},
                   "parallelism": f"stream-sharded x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(ach / hbm, 4),
                     "traffic": None, "kernel": "whole step (all streams' stage01 + stage2 launches)",
                     "algorithmic_bytes_per_step": bytes_c // args.steps, "peak_source": src},
        "plain_gmm": {"value": round(world * P_tot * args.steps / (ms_g / 1e3) / 1e6, 1), "unit": UNIT,
                      "ms_per_step": round(ms_g / args.steps, 4),
                      "roofline": {"bound": "hbm", "achieved": round(ach_g, 1), "peak": hbm, "unit": "GB/s",
                                   "frac": round(ach_g / hbm, 4)}},
        "speedup_vs_plain_gmm": round(ms_g / ms, 3),
        "stage_occupancy": {k: round(float(v) / (P_tot * args.steps), 5)
                            for k, v in zip(("fd", "rga", "gmm_bg", "fg", "illum", "skipped"), occ)},
        "gpu_launches": (2 * len({(s[2]) for s in specs}) + len({(s[2]) for s in specs})) * args.steps,
        "clocks": clk,
    }


# ---------------------------------------------------------------- serving
def run_serve(args, rank, local_rank, world):
    """Serving: `--cameras` cameras (40 % at 640x480, 15 % at each of the
    four other sizes), K=5, FP16 state resident on the device, 100 training
    frames each; each camera emits frames with exponential inter-arrival
    times of mean 1/30 s for `--duration` seconds.  Frames come from a pool
    of eight host frames per camera in one block of the server's arena
    (registered huge-page memory) taken after the cameras are admitted.  The server admits cameras by
    free HBM; the native server (cog_server_*) runs continuous batching
    (cog_batch_apply_active).  Reports p50/p99 latency from submission to
    mask in host memory, and aggregate Mpixel/s."""
    import heapq
    import threading

    import torch
    from cogsynth import Scene
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog
    from paper_1705_09339_gb300.serve import FrameServer

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    if args.l2_fetch >= 0:
        cog.cog_set_l2_fetch_bytes(args.l2_fetch)
    rng = np.random.default_rng(5 + 1000 * rank)
    nc = args.cameras
    sizes = [SIZES[2]] * int(round(0.4 * nc))
    while len(sizes) < nc:
        sizes.append(SIZES[[0, 1, 3, 4][len(sizes) % 4]])
    rng.shuffle(sizes)
    srv = FrameServer(dev, reserve_bytes=8 << 30, frame_memory=args.frame_mem, mask_memory=args.mask_mem)
    staged = {}
    for i, (w, h) in enumerate(sizes):
        sc = Scene(w, h, 7000 + 1000 * rank + i, kind="dynamic", n_train=100, fg_frac=float(rng.uniform(0.01, 0.05)))
        gs = GpuScene(sc, dev)
        cam = srv.admit(w, h, 5, "f16", gs.render(0, 100))
        if cam is None:
            continue
        staged[cam.id] = gs.render(100, 8).cpu()
    # every camera's frame pool in one block of page-locked memory taken
    # after the cameras' device memory: memory locked after the device
    # allocations kept 158-181 GB/s host-to-device in every process measured,
    # memory locked before them often far less
    srv.arena.reserve(sum(8 * ((t.shape[1] * t.shape[2] * 3 + 255) // 256 * 256) for t in staged.values()))
    pools = {}
    for cid, pool in staged.items():
        pools[cid] = [srv.arena.take(tuple(pool.shape[1:])) for _ in range(8)]
        for j in range(8):
            pools[cid][j].copy_(pool[j])
    del staged
    h2d = h2d_probe(torch, dev, [f for cid in pools for f in pools[cid]])
    h2d["arena_huge_kb"] = [_huge_kb(int(t.data_ptr()), t.numel()) for _, t in srv.arena.blocks]
    # everything allocated so far lives for the whole run: keep it out of
    # the garbage collector's passes so they stay short while serving
    import gc
    gc.collect()
    gc.freeze()
    # warm-up, left out of the statistics: every frame buffer of every
    # camera once (both device slots, the batch graph's first launch, and
    # each host buffer's first copy, which ran slower); the Poisson stream
    # then continues each camera's frames
    srv.start(warmup_frames={cid: pools[cid] for cid in pools})
    clocks = Clocks(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    heap = [(t0 + float(rng.exponential(1 / 30)), c.id) for c in srv.cameras]
    heapq.heapify(heap)
    sent = 0
    t_end = t0 + args.duration
    while heap:
        t, cid = heapq.heappop(heap)
        if t > t_end:
            break
        now = time.perf_counter()
        if t > now:
            time.sleep(t - now)
        cam = srv.cameras[cid]
        srv.submit(cam, pools[cid][cam.seq % 8], t)
        sent += 1
        heapq.heappush(heap, (t + float(rng.exponential(1 / 30)), cid))
    st = srv.stop()
    clk = clocks.stop()
    if args.timeline:
        np.savez_compressed(args.timeline, submit_ms=srv.timeline[0], wait_ms=srv.timeline[1],
                            latency_ms=srv.timeline[2], enqueue_ms=srv.steps[0], step_parts_ms=srv.steps[1])
    demand = sum(c.P for c in srv.cameras) * 30 / 1e6
    srv.close()
    if rank != 0:
        return None
    lat = st["latency_ms"]
    split = st.get("latency_split_ms")
    return {
        "metric": "serving: p50/p99 frame latency (submission to mask in host memory) and aggregate Mpixel/s",
        "value": lat["p99"], "unit": "ms (p99 latency)", "n_gpus": world, "steps": st["steps"], "warmup": 0,
        "ms_per_step": round(st["wall_s"] * 1e3 / max(1, st["steps"]), 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{nc} cameras, 40% 640x480 and 15% each of 160x120/320x240/1280x720/1920x1080, "
                               f"K=5 FP16, Poisson arrivals at 30 fps for {args.duration:.0f} s, continuous batching",
                   "cameras_admitted": st["cameras"], "cameras_refused": st["refused"],
                   "demand_mpixel_per_s": round(demand, 1), "frames_sent": sent},
        "latency_ms": lat, "latency_split_ms": split, "frames": st["frames"],
        "aggregate_mpixel_per_s": st["mpixel_per_s"],
        "frame_period_ms": 33.3, "p99_under_frame_period": lat["p99"] is not None and lat["p99"] < 33.3,
        "clocks": clk, "h2d_probe": h2d,
    }


def _registered_copy(torch, frames, huge: bool):
    """The pool's frames copied into one anonymous mapping (transparent huge
    pages asked for, or refused) that is then page-locked with
    cudaHostRegister; returns (tensors, release) or None."""
    import mmap
    total = sum((f.numel() + 255) // 256 * 256 for f in frames)
    align = 512 << 20
    try:
        mm = mmap.mmap(-1, total + align, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        mm.madvise(mmap.MADV_HUGEPAGE if huge else mmap.MADV_NOHUGEPAGE)
    except Exception:
        return None
    raw = np.frombuffer(mm, dtype=np.uint8)
    off = (-raw.ctypes.data) % align
    buf = torch.from_numpy(raw[off:off + total])
    views, o = [], 0
    for f in frames:
        n = f.numel()
        v = buf[o:o + n].view(f.shape)
        v.copy_(f)
        views.append(v)
        o += (n + 255) // 256 * 256
    cudart = torch.cuda.cudart()
    if int(cudart.cudaHostRegister(buf.data_ptr(), total, 0)) != 0:
        return None

    def release():
        cudart.cudaHostUnregister(buf.data_ptr())
    return views, release, mm


def _huge_kb(addr: int, nbytes: int) -> int:
    """AnonHugePages (kB) of the mappings overlapping [addr, addr + nbytes)."""
    tot, cur = 0, False
    try:
        with open("/proc/self/smaps") as f:
            for line in f:
                head = line.split()[0]
                if "-" in head and not head.endswith(":"):
                    a, b = (int(x, 16) for x in head.split("-"))
                    cur = a < addr + nbytes and b > addr
                elif cur and head == "AnonHugePages:":
                    tot += int(line.split()[1])
    except OSError:
        return -1
    return tot


def run_h2d(args, rank, local_rank, world):
    """Host-to-device copy probe alone: 2048 frames of the serving size mix
    (3.6 GB) in each kind of page-locked memory (the serving arena's
    cog_host_alloc blocks, cudaHostAlloc blocks, one cog_host_alloc block,
    one huge-page mapping locked after it is written), with the huge pages
    each received."""
    import torch
    from paper_1705_09339_gb300 import cog
    from paper_1705_09339_gb300.serve import PinnedArena
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    sizes = [SIZES[2]] * 102 + [SIZES[[0, 1, 3, 4][i % 4]] for i in range(154)]
    shapes = [(h, w, 3) for (w, h) in sizes for _ in range(8)]
    out = {"thp_pmd_bytes": None}
    try:
        out["thp_pmd_bytes"] = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
        out["thp_enabled"] = open("/sys/kernel/mm/transparent_hugepage/enabled").read().strip()
    except OSError:
        pass
    for kind in ("registered", "hostalloc"):
        ar = PinnedArena(kind=kind)
        fr = [ar.take(sh) for sh in shapes]
        for i, f in enumerate(fr):
            f.fill_(i & 255)
        r = h2d_probe(torch, dev, fr, variants=False)
        out[kind] = {k: v for k, v in r.items() if k.endswith("_gbs")}
        out[kind]["huge_kb"] = [_huge_kb(int(t.data_ptr()), t.numel()) for _, t in ar.blocks]
        del fr
        ar.release()
    # one cog_host_alloc block for the whole pool
    total = sum((int(np.prod(sh)) + 255) // 256 * 256 for sh in shapes)
    addr = cog.cog_host_alloc(total)
    import ctypes
    arr = np.ctypeslib.as_array(ctypes.cast(addr, ctypes.POINTER(ctypes.c_uint8)), shape=(total,))
    buf = torch.from_numpy(arr)
    fr, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        fr.append(buf[o:o + n].view(sh))
        o += (n + 255) // 256 * 256
    for i, f in enumerate(fr):
        f.fill_(i & 255)
    r = h2d_probe(torch, dev, fr, variants=False)
    out["one_block"] = {k: v for k, v in r.items() if k.endswith("_gbs")}
    out["one_block"]["huge_kb"] = _huge_kb(addr, total)
    del fr, buf, arr
    cog.cog_host_free(addr)
    return {"metric": "host-to-device copy probe", "h2d": out}


def h2d_probe(torch, dev, frames, variants: bool = True) -> dict:
    """Host-to-device copy bandwidth from the serving pool's frames (the
    server's arena: cog_host_alloc), timed with events on one stream: one
    large frame copied 20 times, then every frame of the pool once, twice
    over.  The same for copies of the pool in cudaHostAlloc memory (one
    pinned tensor per frame, `hostalloc_`) and in memory with transparent
    huge pages locked by cudaHostRegister (`reg_thp_`)."""
    st = torch.cuda.Stream(dev)
    big_n = max(f.numel() for f in frames)
    dst = torch.empty(big_n, dtype=torch.uint8, device=dev)
    out = {"pool_gb": round(sum(f.numel() for f in frames) / 1e9, 3), "frames": len(frames)}

    def run(tag, fr):
        big = max(fr, key=lambda f: f.numel())
        with torch.cuda.stream(st):
            for name, seq in (("hot", [big] * 20), ("pass1", fr), ("pass2", fr)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for f in seq:
                    dst[:f.numel()].copy_(f.view(-1), non_blocking=True)
                e1.record(st)
                st.synchronize()
                out[f"{tag}{name}_gbs"] = round(sum(f.numel() for f in seq) / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)

    run("", frames)
    if not variants:
        return out

    # device-to-host into mask-sized buffers (one byte per pixel) of each kind
    def run_d2h(tag, dsts):
        src = torch.zeros(big_n, dtype=torch.uint8, device=dev)
        with torch.cuda.stream(st):
            for name in ("pass1", "pass2"):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for d in dsts:
                    d.copy_(src[:d.numel()], non_blocking=True)
                e1.record(st)
                st.synchronize()
                out[f"d2h_{tag}{name}_gbs"] = round(sum(d.numel() for d in dsts) / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    from paper_1705_09339_gb300.serve import PinnedArena
    for kind in ("registered", "hostalloc"):
        ar = PinnedArena(kind=kind)
        run_d2h(kind + "_", [ar.take((f.numel() // 3,)) for f in frames])
        ar.release()
    # the same frames in cudaHostAlloc memory, one pinned tensor each
    pinned = [f.pin_memory() for f in frames]
    run("hostalloc_", pinned)
    del pinned
    for tag, huge in (("reg_thp_", True),):
        r = _registered_copy(torch, frames, huge)
        if r is None:
            out[tag + "error"] = "mapping or cudaHostRegister failed"
            continue
        views, release, mm = r
        run(tag, views)
        out[tag + "huge_kb"] = _huge_kb(int(views[0].data_ptr()), sum(v.numel() for v in views))
        release()          # the copies have finished (run synchronises)
        del views, mm      # the mapping goes with its last reference
    return out


def _oracle_sample(sc, rows, n_frames, t0):
    """Pixels of a band of rows and their frames t0..t0+n-1 (numpy renderer)."""
    y0 = sc.height // 2 - rows // 2
    pix = np.arange(y0 * sc.width, (y0 + rows) * sc.width)
    fr = np.stack([sc.render(t, pix)[0] for t in range(t0, t0 + n_frames)])
    return pix, fr


def cpu_baseline(sc, gpu_masks, args):
    """The FP64 oracle on a bounded sample: a band of 10 rows (19,200
    pixels) trained on the 500 training frames, then the timed frames.
    Also the FP16 GPU masks' agreement with it on that band."""
    import oracle
    rows = 10
    n = args.steps
    pix, tr = _oracle_sample(sc, rows, N_TRAIN, 0)
    _, te = _oracle_sample(sc, rows, args.warmup + n, N_TRAIN)
    d = oracle.default_params(sc.width, rows, K_)
    o = oracle.Oracle(d)
    o.train(tr)
    for i in range(args.warmup):
        o.apply(te[i], want_stage=False, want_near=False)
    gm = gpu_masks.reshape(n, -1)[:, pix].cpu().numpy()
    agree = 0
    t0 = time.perf_counter()
    for i in range(n):
        m, _, _, _ = o.apply(te[args.warmup + i], want_stage=False, want_near=False)
        agree += int((m == gm[i]).sum())
    dt = time.perf_counter() - t0
    # the same oracle on one core, over the next frames (at most 20)
    n1 = min(n, 20)
    cores = oracle.oracle_threads()
    oracle.set_threads(1)
    t0 = time.perf_counter()
    for i in range(n1):
        o.apply(te[args.warmup + i], want_stage=False, want_near=False)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": round(len(pix) * n / dt / 1e6, 3), "unit": UNIT, "cores": cores,
            "single_core_value": round(len(pix) * n1 / dt1 / 1e6, 3),
            "kind": "oracle",
            "sample": f"{rows} rows x {sc.width} px (band at mid-height) x {n} test frames of the same stream, "
                      f"after the same {N_TRAIN} training frames; apply phase timed",
            "mask_agreement_fp16_gpu_vs_fp64": round(agree / (len(pix) * n), 6)}


# ------------------------------------------------------------- grouping
def run_group(args, rank, local_rank, world):
    """Spatio-temporal grouping (Sec. 2, steps 1-6 and Eq. 3) of the
    1920x1080 dynamic stream's 500 training frames, K=5, FP16 state: one
    step is one cog_group call (the warm-up replay that yields the two
    feature codes, the K-means iterations and the Eq. 3 cores).  The
    training frames (3.1 GB) exceed L2, so no flush is needed between steps."""
    import torch
    import torch.distributed as dist
    from cogsynth import workload
    from cogsynth.gpu import GpuScene
    from paper_1705_09339_gb300 import cog

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    torch.zeros(1, device=dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    sc = workload("hd_dynamic", fg_frac=args.fg, seed=stream_seed(3, rank))["scene"]
    P = sc.P
    stream = torch.cuda.current_stream(dev)
    train = GpuScene(sc, dev).render(0, N_TRAIN)
    p = cog.cog_default_params(W_, H_, K_, state_dtype="f16")
    ctx = cog.cog_create(p, stream.cuda_stream)
    cog.cog_train_prior(ctx, train, N_TRAIN)
    codes = torch.empty((2, P), dtype=torch.int16, device=dev)
    labels = torch.empty(P, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        st = cog.cog_group(ctx, train, N_TRAIN, codes, labels)
    clocks = Clocks(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st = cog.cog_group(ctx, train, N_TRAIN, codes, labels)
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    (ms,) = max_over_ranks([ms], world, dev)
    result = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            import oracle
            idx = np.random.default_rng(0).choice(P, 2048, replace=False)
            sub = train.reshape(N_TRAIN, P, 3)[:, torch.from_numpy(idx).to(dev)].cpu().numpy()
            o = oracle.Oracle(dict(oracle.default_params(2048, 1, K_), flags=0))
            t0 = time.perf_counter()
            cv, cw = o.group_features(sub)
            oracle.group_cluster(cv, cw)
            t_cpu = time.perf_counter() - t0
            cpu = {"value": round(2048 / t_cpu / 1e6, 6), "unit": "Mpixel/s", "cores": oracle.oracle_threads(),
                   "kind": "oracle", "sample": "2048 random pixels' 500-frame training series: features "
                                               "(FP64 warm-up replay) and K-means on them"}
        e = ncu_counts("group_features_kernel")
        roof = {"bound": "alu", "kernel": "group_features_kernel", "unit": "Twarp-inst/s",
                "peak": round(ISSUE_PEAK / 1e12, 4), "achieved": None, "frac": None, "traffic": None,
                "note": "the warm-up replay issues instructions (FP32 mixture step per pixel and frame); "
                        "peak = 152 SMs x 4 schedulers x 1 warp instruction per clock x 2070 MHz; the "
                        "count is per launch from profiles/traffic.json over the whole cog_group time"}
        if e and "warp_instructions_per_launch" in e:
            a = float(e["warp_instructions_per_launch"]) / (ms / args.steps / 1e3)
            roof.update(achieved=round(a / 1e12, 4), frac=round(a / ISSUE_PEAK, 4),
                        traffic=e.get("dram_bytes_per_launch"))
        result = {
            "metric": "CoG spatio-temporal grouping Mpixel/s (500 training frames per pixel)",
            "value": round(world * P * args.steps / (ms / 1e3) / 1e6, 2), "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{W_}x{H_} RGB u8 dynamic-background stream, {N_TRAIN} training frames, "
                                   f"K={K_}, FP16 state: one cog_group per step",
                       "l2": "training frames (3.1 GB) exceed L2; no flush"},
            "groups": {k: st[k] for k in ("iterations", "converged", "n", "n_core", "centroid", "sd")},
            "roofline": roof, "gpu_launches": 67 * args.steps, "e2e": None, "cpu_baseline": cpu, "clocks": clk,
        }
    cog.cog_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return result


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The FP64 CPU oracle, as it stands, on the host cores: each step is
    one frame of a 20-row band (38,400 pixels) of the same stream."""
    if rank != 0:
        return None
    import oracle
    from cogsynth import workload
    sc = workload("hd_dynamic", fg_frac=args.fg, seed=3)["scene"]
    rows = 20
    pix, tr = _oracle_sample(sc, rows, N_TRAIN, 0)
    _, te = _oracle_sample(sc, rows, args.warmup + args.steps, N_TRAIN)
    o = oracle.Oracle(oracle.default_params(sc.width, rows, K_))
    o.train(tr)
    for i in range(args.warmup):
        o.apply(te[i], want_stage=False, want_near=False)
    t0 = time.perf_counter()
    for i in range(args.steps):
        o.apply(te[args.warmup + i], want_stage=False, want_near=False)
    dt = time.perf_counter() - t0
    v = round(len(pix) * args.steps / dt / 1e6, 3)
    cores = oracle.oracle_threads()
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{W_}x{H_} RGB u8 dynamic-background stream, K={K_}, FP64 oracle on the host",
                       "width": W_, "height": H_, "K": K_, "n_train": N_TRAIN, "fg_frac": args.fg},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{rows} rows x {sc.width} px band of the stream per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fg", type=float, default=0.02)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="hd", choices=["hd", "clip", "batch64", "serve", "group", "profile", "h2d"])
    ap.add_argument("--duration", type=float, default=20.0, help="serve: seconds of camera traffic")
    ap.add_argument("--cameras", type=int, default=256, help="serve: cameras")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--kde-bits", type=int, default=8, choices=[8, 4],
                    help="scene prior levels: 8-bit (768 B/px) or 4-bit (384 B/px)")
    ap.add_argument("--frame-mem", default="registered", choices=["registered", "hostalloc"],
                    help="serve: page-locked memory of the host frames")
    ap.add_argument("--mask-mem", default="hostalloc", choices=["registered", "hostalloc"],
                    help="serve: page-locked memory of the host masks")
    ap.add_argument("--launch", default="",
                    help="profile case: launch shape 'k1_threads,k2_threads,k2_ctas_per_sm' (cog_set_launch)")
    ap.add_argument("--sample", action="store_true",
                    help="hd: confidence-based temporal sampling on (saturated pixels every 4 frames)")
    ap.add_argument("--mode1", action="store_true",
                    help="hd: COG_MODE1, stage 1 as the mixture's rank-1 mode (the Fig. 1 reading)")
    ap.add_argument("--perchan", action="store_true",
                    help="hd: COG_PERCHAN, per-channel independent mixtures")
    ap.add_argument("--l2-fetch", type=int, default=32,
                    help="L2 fetch granularity in bytes for the process (-1 keeps the driver default)")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="hd: skip the batch64 and serve sub-results of the default line")
    ap.add_argument("--timeline", default="", help="serve: write the per-frame timeline (npz) to this path")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank, local_rank, world = rank_info()
    if args.impl == "reference":
        r = run_reference(args, rank, world)
    else:
        import __graft_entry__
        __graft_entry__.build()
        r = {"batch64": run_batch, "serve": run_serve, "clip": run_clip,
             "group": run_group, "profile": run_profile_case, "h2d": run_h2d}.get(args.workload, run_ours)(
            args, rank, local_rank, world)
    if r is not None and rank == 0:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
