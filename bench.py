#!/usr/bin/env python
"""Throughput of the CDVS front end (keypoints + 128-D descriptors) on GB300.

Workload: a batch of 256 synthetic 640x480 8-bit images (seeds 1..256 of the
blob generator; they stand in for the paper's 640x480 test images), default
parameters (4 octaves, 4 LoG scales fitted by the ALP cubic, N = 300 points,
128-D float descriptors, FP32 scale space).  One step = one cdvs_extract call
on the whole batch with inputs and outputs resident in device memory; `value`
is images/s.  `e2e` is the same call with pinned host inputs and host outputs
(copies inside the timed region).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank runs its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_IMAGES, WIDTH, HEIGHT, BASE_SEED = 256, 640, 480, 1
UNEVEN_SEED = 3
METRIC = "images/s CDVS keypoints+descriptors @640px (batched/learned vs plain), HBM GB/s"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (Blackwell SM: 4 partitions x 32)
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k1_detect_traffic.json")


def _gen(i):
    from paper_1705_09776_gb300 import synth
    return synth.blob_image(synth.image_seed(BASE_SEED, i), WIDTH, HEIGHT)


def make_batch(n, offset=0):
    """Seeded images offset .. offset+n-1 (generated in a spawn pool: no fork
    after CUDA is initialised)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 1)) as pool:
        imgs = pool.map(_gen, range(offset, offset + n))
    return np.stack(imgs)


def detect_counts(p, width=None, height=None):
    """Algorithmic FLOPs and bytes of the detection stage (K1) per image (640x480 by default)
    and per octave, FP32 levels: S1 filters (2 passes x 2 flops per tap,
    identity levels free), S2 Laplacian (7 flops per level), S3 cubic fit (32),
    S4 roots (25); bytes = octave base read + every level written once (level 0
    of octaves >= 1 is written by the previous octave as its decimated base)."""
    s = [float(p["sigma0"][0]) * 2 ** (k / 3) for k in range(4)]
    flops, byts = [], []
    w, h = width or WIDTH, height or HEIGHT
    for o in range(int(p["num_octaves"][0])):
        base = float(p["sigma_in"][0]) if o == 0 else float(p["sigma0"][0])
        per_px = 0.0
        for k in range(4):
            t2 = s[k] * s[k] - base * base
            if t2 > 0:
                r = math.ceil(4 * math.sqrt(t2))
                per_px += 4 * (2 * r + 1)
        per_px += 4 * 7 + 32 + 25
        flops.append(per_px * w * h)
        levels_written = 4 if o == 0 else 3
        decimated = 4 * ((w + 1) // 2) * ((h + 1) // 2) if o + 1 < int(p["num_octaves"][0]) else 0
        byts.append((w * h if o == 0 else 4 * w * h) + 4 * levels_written * w * h + decimated)
        w, h = (w + 1) // 2, (h + 1) // 2
    return flops, byts


def resize_target(w, h, max_side):
    """S0 output size: the larger side becomes max_side, the other is scaled and
    rounded to nearest, ties to even (the library's rule)."""
    if max_side <= 0 or max(w, h) <= max_side:
        return w, h

    def rhe(num, den):
        q, r = divmod(num, den)
        return q + (1 if 2 * r > den or (2 * r == den and q & 1) else 0)
    if w >= h:
        return max_side, max(1, rhe(h * max_side, w))
    return max(1, rhe(w * max_side, h)), max_side


def alu_peak_tflops(torch, local, sm_mhz):
    """FP32 peak derived from the device: SMs x 128 FMA lanes x 2 flop x the
    SM clock (the maximum clock nvidia-smi reports)."""
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12, sms


def measure_sgemm_tflops(torch, n=8192, reps=5):
    """A measured FP32 (non-tensor) throughput: cuBLAS SGEMM n^3 with TF32 off,
    best of `reps` after a warm-up, CUDA events."""
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        c = a @ b
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b, c
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = f"/tmp/cdvs_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.remove(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def kernel_sha():
    """sha256 of K1's sources (the kernel header and its variant launchers)."""
    h = hashlib.sha256()
    for f in ("detect_kernel.cuh", "detect.cu", "detect_vb.cu", "detect_vc.cu", "detect_vd.cu"):
        h.update(open(os.path.join(ROOT, "paper_1705_09776_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def load_traffic(variant=0):
    """DRAM bytes per image of the octave-0 detection launch of a K1 variant,
    from the committed ncu summary, when it was taken on the current sources."""
    try:
        t = json.load(open(TRAFFIC_FILE))
        if t.get("kernel_sha256") == kernel_sha():
            return t["variants"].get(str(variant))
    except Exception:
        pass
    return None


def cpu_baseline(imgs, n_sample=32):
    from oracle import oracle as O
    O.build()
    p = O.params()
    sample = list(imgs[:n_sample])
    t0 = time.perf_counter()
    O.extract_batch(sample, p, cap=2048)
    dt = time.perf_counter() - t0
    return {"value": n_sample / dt, "unit": "images/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"first {n_sample} images of the 256-image 640x480 batch, FP64 oracle, "
                      f"image-parallel over all host threads, {dt:.2f} s"}


def run_reference(args, rank):
    """The oracle as the reference arm: each step extracts a bounded sample of
    the workload on the host cores."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    p = O.params()
    threads = O.num_threads()
    n_sample = max(8, threads)
    imgs = make_batch(n_sample)
    for _ in range(args.warmup):
        O.extract_batch(list(imgs), p, cap=2048)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.extract_batch(list(imgs), p, cap=2048)
    dt = time.perf_counter() - t0
    value = n_sample * args.steps / dt
    sample = f"{n_sample} of the 640x480 workload images per step, FP64 oracle on {threads} threads"
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{N_IMAGES}x {WIDTH}x{HEIGHT} u8 blob images (oracle sample per step)",
                      "n_images_per_step": n_sample},
           "cpu_baseline": {"value": value, "unit": "images/s", "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_e2e(ctx, imgs, sizes, p, cap, stream, args, barrier, dist, cdvs, torch):
    """Same call with pinned host inputs and host outputs: the H2D copy of the
    batch and the D2H copy of every record and descriptor are timed.  The
    calls are asynchronous (CDVS_ASYNC): batch k's records go out while
    batch k+1 is processed, and the cdvs_wait that completes the last batch's
    copies is inside the timed region."""
    n, H, W = imgs.shape
    h_img = torch.from_numpy(imgs).pin_memory()
    h_kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    h_desc = torch.zeros(cap, 128, dtype=torch.float32).pin_memory()
    h_cnt = torch.zeros(n, dtype=torch.int32).pin_memory()
    hptrs = [h_img.data_ptr() + i * H * W for i in range(n)]

    def step_e2e():
        return ctx.extract_raw(n, hptrs, sizes, p, h_kp, h_desc, cap, h_cnt, cdvs.CDVS_ASYNC, stream)

    for _ in range(3):
        step_e2e()
    ctx.wait(stream)
    k_e2e = max(3, args.steps // 2)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        step_e2e()
    ctx.wait(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / k_e2e
    if dist is not None:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_records = int(h_cnt.sum().item())

    return e2e_ms, e2e_records


def run_per_image(ctx, cdvs, torch, dptrs, sizes, p, d_kp, d_desc, d_cnt, stream, passes=3):
    """The batched call against one image per call: the same images, device-
    resident, one cdvs_extract per image (enqueued asynchronously, so host
    work overlaps the GPU); images/s over `passes` passes over the batch."""
    n = len(dptrs)
    flags = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE | cdvs.CDVS_ASYNC
    cap1 = int(p["max_keypoints"][0]) * int(p["max_orientations"][0])

    def one_pass():
        for i in range(n):
            ctx.extract_raw(1, [dptrs[i]], sizes[i:i + 1], p, d_kp, d_desc, cap1, d_cnt[i:i + 1], flags, stream)

    one_pass()
    ctx.wait(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(passes):
        one_pass()
    e1.record(stream)
    ctx.wait(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / passes
    return {"value": n / (ms * 1e-3), "unit": "images/s", "ms_per_batch": ms, "calls_per_batch": n}


def record_keys(kp):
    k = np.stack([kp["image"], kp["octave"], kp["x"].view(np.int32), kp["y"].view(np.int32),
                  kp["sigma"].view(np.int32), kp["theta"].view(np.int32)], 1)
    return set(map(tuple, k.tolist()))


def tile_modes(logits, zt, H, W, reach):
    """Counts of first-octave tiles (128 x 32 px) per mode, by the library's
    rule: detect when a block with logit > zt lies within one block of the
    tile; store levels when a detecting tile lies within the descriptor reach."""
    tx_n, ty_n = -(-W // 128), -(-H // 32)
    ny, nx = int(np.ceil(reach / 32)), int(np.ceil(reach / 128))
    counts = np.zeros(3, np.int64)
    for z in logits:
        th, tw = z.shape
        det = np.zeros((ty_n, tx_n), bool)
        for ty in range(ty_n):
            for tx in range(tx_n):
                win = z[max(2 * ty - 1, 0):min(2 * ty + 3, th), max(8 * tx - 1, 0):min(8 * tx + 9, tw)]
                det[ty, tx] = (win > zt).any()
        for ty in range(ty_n):
            for tx in range(tx_n):
                if det[ty, tx]:
                    counts[2] += 1
                elif det[max(ty - ny, 0):ty + ny + 1, max(tx - nx, 0):tx + nx + 1].any():
                    counts[1] += 1
                else:
                    counts[0] += 1
    return counts


def break_even_share(network_ms, octave0_plain_ms, octave0_none_ms):
    """The share of first-octave tiles a mask must take out of detection (to
    their cheapest mode) for the saving to pay for the network and its
    tile-mode passes: network time / (plain octave 0 - octave 0 with no block
    proposed), assuming the saving grows in proportion to the tiles skipped.
    None when masking saves nothing."""
    saving = octave0_plain_ms - octave0_none_ms
    return network_ms / saving if saving > 0 else None


def run_learned(ctx, imgs, step_with, p_plain, args, cdvs, torch, plain_kp):
    """The same batch with the learned block proposal masking first-octave
    detection: throughput, keypoint recall against the plain detector (exact
    record identity), and how the first-octave tiles were treated.  Also the
    mechanism's floor on this batch: the same step with a network that
    proposes no block (every first-octave tile takes its cheapest mode, the
    network still runs at full cost)."""
    theta, thr = cdvs.load_proposal_weights()
    p = cdvs.params(storage=int(p_plain["storage"][0]), use_proposal=1, proposal_threshold=thr)
    stream = torch.cuda.current_stream()

    def timed(weights):
        ctx.set_proposal(weights)
        for _ in range(args.warmup):
            step_with(p)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            kp, _ = step_with(p)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        return e0.elapsed_time(e1) / args.steps, prof, kp

    none = np.zeros_like(theta)
    none[-1] = -20.0  # head bias only: every logit is -20
    ms_none, prof_none, _ = timed(none)
    ms, prof, kp = timed(theta)
    learned_kp = kp()
    plain = record_keys(plain_kp)
    recall = len(plain & record_keys(learned_kp)) / max(len(plain), 1)
    zt = float(np.log(thr / (1 - thr)))
    reach = max(float(p["desc_radius"][0]), float(p["ori_radius"][0])) * 2 * float(p["sigma0"][0]) * 1.001 + 2
    counts = tile_modes(ctx.proposal_logits(list(imgs)), zt, imgs.shape[1], imgs.shape[2], reach)
    n = len(imgs)
    return {"value": n / (ms * 1e-3), "unit": "images/s", "ms_per_step": ms, "threshold": thr,
            "recall_vs_plain": recall, "records_per_step": int(len(learned_kp)),
            "first_octave_tiles": {"detect": int(counts[2]), "levels_only": int(counts[1]),
                                   "level3_only": int(counts[0])},
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "no_block_proposed": {"ms_per_step": ms_none,
                                  "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof_none.items()}},
            "weights": "paper_1705_09776_gb300/proposal_weights.npz (train_proposal.py; images of seeds 1e6+i and, "
                       "with the high-resolution statistics, 5e6+i)"}


def _gen_uneven(args):
    from paper_1705_09776_gb300 import synth
    i, w, h = args
    return synth.blob_image(synth.image_seed(UNEVEN_SEED, i), width=w, height=h,
                            n_blobs=max(8, int(round(200 * w * h / (WIDTH * HEIGHT)))))


def gen_uneven(n, seed_offset=0):
    import multiprocessing as mp

    from paper_1705_09776_gb300 import synth
    sizes = synth.uneven_sizes(n, base_seed=UNEVEN_SEED + seed_offset)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        imgs = pool.map(_gen_uneven, [(i, w, h) for i, (w, h) in enumerate(sizes)], chunksize=8)
    return imgs, sizes


def k1_roofline(flops, launch_ms, alu_peak, what):
    return {"kernel": what, "bound": "alu", "achieved": flops / (launch_ms * 1e-3) / 1e12, "peak": alu_peak,
            "unit": "TFLOP/s", "frac": flops / (launch_ms * 1e-3) / 1e12 / alu_peak,
            "algorithmic_flops_per_launch": flops, "launch_ms": launch_ms}


def uneven_leg(ctx, cdvs, torch, imgs, sizes, args, alu_peak, steps=None):
    """Uneven batch (config 3): images with sides in 240..1280 and aspect
    0.5..2 (blob count scaled by area), resized on the GPU to larger side 640
    (S0) and extracted in one call per step; device-resident inputs and
    outputs, the call's work replayed as one CUDA graph, calls enqueued
    asynchronously (CDVS_ASYNC).  FP32 and FP16 level storage, and FP32
    without the graph."""
    steps = steps or args.steps
    n = len(imgs)
    flat = np.concatenate([im.ravel() for im in imgs])
    offs = np.cumsum([0] + [im.size for im in imgs])
    d_img = torch.from_numpy(flat).cuda()
    ptrs = [d_img.data_ptr() + int(o) for o in offs[:-1]]
    desc_sizes = np.array([(im.shape[1], im.shape[0], im.shape[1]) for im in imgs], cdvs.IMAGE_DESC_DTYPE)
    cap = n * 300 * 4
    stream = torch.cuda.current_stream()
    d_kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d_desc = torch.zeros(cap, 128, dtype=torch.float32, device="cuda")
    d_cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    flags = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE

    def timed(p, graph):
        ctx.set_graph(graph)
        for _ in range(args.warmup):
            ctx.extract_raw(n, ptrs, desc_sizes, p, d_kp, d_desc, cap, d_cnt, flags | cdvs.CDVS_ASYNC, stream)
        ctx.wait(stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.extract_raw(n, ptrs, desc_sizes, p, d_kp, d_desc, cap, d_cnt, flags | cdvs.CDVS_ASYNC, stream)
        e1.record(stream)
        ctx.wait(stream)
        torch.cuda.synchronize()
        ctx.set_graph(False)
        return e0.elapsed_time(e1) / steps, int(d_cnt.sum().item())

    p32 = cdvs.params(max_side=640)
    p16 = cdvs.params(max_side=640, storage=cdvs.CDVS_STORAGE_FP16)
    ms32, rec32 = timed(p32, True)
    ms16, rec16 = timed(p16, True)
    ms_direct, _ = timed(p32, False)
    tuning = ctx.detect_tuning()
    # the same FP32 graph leg with K1's work shape fixed to variant 0 (the
    # 128 x 32 tile, one 512-thread CTA per SM) instead of the tuned choice
    ctx.set_detect_variant(0)
    ms_fixed, _ = timed(p32, True)
    ctx.set_detect_variant(-1)
    # stage times from profiled (direct) calls
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(3):
        ctx.extract_raw(n, ptrs, desc_sizes, p32, d_kp, d_desc, cap, d_cnt, flags, stream)
    torch.cuda.synchronize()
    prof = {k: v[0] / 3 for k, v in ctx.profile_read(reset=True).items()}
    ctx.profile(False)
    flops0 = sum(detect_counts(p32, *resize_target(w, h, 640))[0][0] for w, h in sizes)
    area = float(sum(w * h for w, h in sizes))
    return {"value": n / (ms32 * 1e-3), "unit": "images/s", "ms_per_step": ms32, "steps": steps,
            "config": {"workload": f"{n}x uneven u8 seeded blob images (sides 240-1280, aspect 0.5-2, blobs by area), "
                                   "S0 area resize to larger side 640, 4 octaves x 4 LoG scales, N=300",
                       "mean_input_megapixels": area / n / 1e6, "storage": "fp32", "graph": True,
                       "records_per_step": rec32},
            "fp16": {"value": n / (ms16 * 1e-3), "ms_per_step": ms16, "records_per_step": rec16},
            "direct_launches": {"value": n / (ms_direct * 1e-3), "ms_per_step": ms_direct},
            "fixed_variant0": {"value": n / (ms_fixed * 1e-3), "ms_per_step": ms_fixed},
            "detect_tuning": tuning,
            "stage_ms_per_call": prof,
            "roofline": k1_roofline(flops0, prof["detect_octave0"], alu_peak,
                                    "detect_kernel, octave-0 launch on the resized images")}


def run_uneven(args, rank, world, local):
    """--workload uneven: the config-3 leg alone, as its own JSON line."""
    imgs, sizes = gen_uneven(args.images, rank)
    import torch
    torch.cuda.set_device(local)
    from paper_1705_09776_gb300 import cdvs
    ctx = cdvs.Context(local)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    alu_peak, _ = alu_peak_tflops(torch, local, device_max_mhz())
    leg = uneven_leg(ctx, cdvs, torch, imgs, sizes, args, alu_peak)
    clocks = sampler.stop()
    out = {"metric": METRIC, "value": leg.pop("value"), "unit": "images/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": leg.pop("ms_per_step"), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "clocks": clocks}
    leg["config"]["l2"] = "working set > L2"
    out.update(leg)
    print(json.dumps(out), flush=True)
    ctx.close()


HIGHRES_W, HIGHRES_H, HIGHRES_SEED = 2048, 1536, 5


def _gen_highres(i):
    from paper_1705_09776_gb300 import synth
    k = HIGHRES_W * HIGHRES_H / (WIDTH * HEIGHT)
    return synth.blob_image(synth.image_seed(HIGHRES_SEED, i), HIGHRES_W, HIGHRES_H, n_blobs=int(round(200 * k)),
                            sigma_range=(1.5 * 3.2, 20.0 * 3.2))


def gen_highres(n, offset=0):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return np.stack(pool.map(_gen_highres, range(offset, offset + n)))


def highres_leg(ctx, cdvs, torch, imgs, args, alu_peak, steps=None):
    """High-resolution stress (config 5): 2048 x 1536 images (blob count by
    area, blob sizes x3.2), 6 octaves, up to 2000 points each; plain FP32
    against FP16 level storage, and FP16 with the learned block proposal;
    device-resident."""
    steps = steps or args.steps
    n, H, W = imgs.shape
    d_img = torch.from_numpy(imgs).cuda()
    ptrs = [d_img.data_ptr() + i * H * W for i in range(n)]
    sizes = np.array([(W, H, W)] * n, cdvs.IMAGE_DESC_DTYPE)
    N = 2000
    cap = n * N * 4
    stream = torch.cuda.current_stream()
    d_kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d_desc = torch.zeros(cap, 128, dtype=torch.float32, device="cuda")
    d_cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    flags = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE

    def call(p):
        ctx.extract_raw(n, ptrs, sizes, p, d_kp, d_desc, cap, d_cnt, flags, stream)

    def timed(p):
        for _ in range(args.warmup):
            call(p)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            call(p)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        tot = int(d_cnt.sum().item())
        kp = d_kp[:tot * cdvs.KEYPOINT_DTYPE.itemsize].cpu().numpy().view(cdvs.KEYPOINT_DTYPE).copy()
        return e0.elapsed_time(e1) / steps, kp, {k: v[0] / steps for k, v in prof.items()}

    p32 = cdvs.params(num_octaves=6, max_keypoints=N)
    ms32, kp32, st32 = timed(p32)
    p16 = cdvs.params(num_octaves=6, max_keypoints=N, storage=cdvs.CDVS_STORAGE_FP16)
    ms16, kp16, st16 = timed(p16)
    tuning = ctx.detect_tuning()
    learned = None
    if os.path.exists(cdvs.PROPOSAL_WEIGHTS):
        theta, thr = cdvs.load_proposal_weights(highres=True)
        ctx.set_proposal(theta)
        pl = cdvs.params(num_octaves=6, max_keypoints=N, storage=cdvs.CDVS_STORAGE_FP16, use_proposal=1,
                         proposal_threshold=thr)
        msl, kpl, stl = timed(pl)
        base = record_keys(kp16)
        learned = {"value": n / (msl * 1e-3), "ms_per_step": msl, "threshold": thr,
                   "recall_vs_fp16_plain": len(base & record_keys(kpl)) / max(len(base), 1),
                   "stage_ms_per_step": stl}
    flops_o, bytes_o = detect_counts(p32, W, H)
    return {"value": n / (ms32 * 1e-3), "unit": "images/s", "ms_per_step": ms32, "steps": steps,
            "config": {"workload": f"{n}x {W}x{H} u8 seeded blob images (blobs x3.2, count by area), 6 octaves x 4 "
                                   "LoG scales, N=2000, 128-D float descriptors", "storage": "fp32",
                       "records_per_step": int(len(kp32))},
            "stage_ms_per_step": st32,
            "detect_tuning": tuning,
            "roofline": k1_roofline(flops_o[0] * n, st32["detect_octave0"], alu_peak,
                                    "detect_kernel, octave-0 launch (2048x1536)"),
            "fp16": {"value": n / (ms16 * 1e-3), "ms_per_step": ms16, "records_per_step": int(len(kp16)),
                     "stage_ms_per_step": st16},
            "fp16_learned": learned}


def run_highres(args, rank, world, local):
    """--workload highres: the config-5 leg alone, as its own JSON line."""
    imgs = gen_highres(args.images, rank * args.images)
    import torch
    torch.cuda.set_device(local)
    from paper_1705_09776_gb300 import cdvs
    ctx = cdvs.Context(local)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    alu_peak, _ = alu_peak_tflops(torch, local, device_max_mhz())
    leg = highres_leg(ctx, cdvs, torch, imgs, args, alu_peak)
    clocks = sampler.stop()
    out = {"metric": METRIC, "value": leg.pop("value"), "unit": "images/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": leg.pop("ms_per_step"), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "clocks": clocks}
    leg["config"]["l2"] = "working set > L2"
    out.update(leg)
    print(json.dumps(out), flush=True)
    ctx.close()


def device_max_mhz():
    """The maximum SM clock of GPU 0 as nvidia-smi reports it (the measured
    peaks file's figure when nvidia-smi is not there)."""
    try:
        r = subprocess.run(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"), "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
        return float(r.stdout.strip().splitlines()[0])
    except Exception:
        return float(load_peaks().get("sm_max_mhz", 2070.0))


def run_scfv(ctx, cdvs, torch, d_desc, counts, args):
    """SCFV aggregation (Sec. III-D) of the batch's descriptors, device-resident,
    with the oracle-derived stand-in PCA/GMM model; ms per batch."""
    path = os.path.join(ROOT, "tests", "golden", "scfv_model.npz")
    if not os.path.exists(path):
        return None
    ctx.set_scfv_model(dict(np.load(path)))
    n = len(counts)
    cnt = np.ascontiguousarray(counts, np.int32)
    outs = [torch.zeros(n, 512, 32, device="cuda"), torch.zeros(n, 512, 32, device="cuda"),
            torch.zeros(n, 512, device="cuda"), torch.zeros(n, 512, dtype=torch.int32, device="cuda"),
            torch.zeros(n, 64, dtype=torch.int32, device="cuda")]
    stream = torch.cuda.current_stream()
    flags = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE

    def call():
        st = ctx._L.cdvs_scfv(ctx.handle, n, d_desc.data_ptr(), cnt.ctypes.data, 64, *[o.data_ptr() for o in outs],
                              flags, stream.cuda_stream)
        ctx._check(st)
    for _ in range(args.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"ms_per_batch": ms, "images_per_s": n / (ms * 1e-3), "records": int(cnt.sum()), "components": 512,
            "n_select": 64, "model": "tests/golden/scfv_model.npz (stand-in PCA/GMM from oracle descriptors)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--images", type=int, default=N_IMAGES, help="images per rank (profiling runs)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal leg")
    ap.add_argument("--no-legs", action="store_true", help="skip the uneven (config 3) and high-resolution "
                                                            "(config 5) legs of the default line")
    ap.add_argument("--uneven-images", type=int, default=1024, help="images of the uneven leg")
    ap.add_argument("--detect-variant", type=int, default=-1, help="K1 work shape: -1 tuned (default), 0..3 fixed")
    ap.add_argument("--highres-images", type=int, default=64, help="images of the high-resolution leg")
    ap.add_argument("--workload", default="batch", choices=["batch", "uneven", "highres"],
                    help="batch: 256 x 640x480 (default); uneven: 1024 uneven images resized to 640; "
                         "highres: 512 x 2048x1536, 6 octaves, N=2000")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "uneven":
        if args.images == N_IMAGES:
            args.images = 1024
        return run_uneven(args, rank, world, local)
    if args.workload == "highres":
        if args.images == N_IMAGES:
            args.images = 512
        return run_highres(args, rank, world, local)

    imgs = make_batch(args.images, offset=rank * args.images)  # before any CUDA call
    legs = None
    if not args.no_legs:
        legs = (gen_uneven(args.uneven_images, rank), gen_highres(args.highres_images, rank * args.highres_images))
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_09776_gb300 import cdvs

    n, H, W = imgs.shape
    p = cdvs.params(storage=cdvs.CDVS_STORAGE_FP16 if args.storage == "fp16" else cdvs.CDVS_STORAGE_FP32)
    cap = n * int(p["max_keypoints"][0]) * int(p["max_orientations"][0])
    ctx = cdvs.Context(local)
    ctx.set_detect_variant(args.detect_variant)
    stream = torch.cuda.current_stream()
    d_img = torch.from_numpy(imgs).cuda()
    d_kp = torch.zeros(cap * cdvs.KEYPOINT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    d_desc = torch.zeros(cap, 128, dtype=torch.float32, device="cuda")
    d_cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
    sizes = np.array([(W, H, W)] * n, cdvs.IMAGE_DESC_DTYPE)
    dptrs = [d_img.data_ptr() + i * H * W for i in range(n)]
    dev_flags = cdvs.CDVS_INPUT_DEVICE | cdvs.CDVS_OUTPUT_DEVICE

    def step():
        # enqueued without host synchronisation: the host prepares the next
        # batch while the GPU runs this one (cdvs_wait after the loop)
        return ctx.extract_raw(n, dptrs, sizes, p, d_kp, d_desc, cap, d_cnt, dev_flags | cdvs.CDVS_ASYNC, stream)

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    ctx.wait(stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    ctx.wait(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)
    clocks = sampler.stop()
    tuning = ctx.detect_tuning()
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    records = int(d_cnt.sum().item())
    value = n * world / (ms * 1e-3)

    def read_kp():
        tot = int(d_cnt.sum().item())
        return d_kp[:tot * cdvs.KEYPOINT_DTYPE.itemsize].cpu().numpy().view(cdvs.KEYPOINT_DTYPE).copy()

    plain_kp = read_kp()
    scfv = run_scfv(ctx, cdvs, torch, d_desc, d_cnt.cpu().numpy(), args)
    learned = None
    if not args.no_learned and os.path.exists(cdvs.PROPOSAL_WEIGHTS):
        def step_with(pp):
            ctx.extract_raw(n, dptrs, sizes, pp, d_kp, d_desc, cap, d_cnt, dev_flags, stream)
            return read_kp, d_cnt
        learned = run_learned(ctx, imgs, step_with, p, args, cdvs, torch, plain_kp)

    # ---- end to end through the C ABI: pinned host inputs, host outputs
    if args.no_e2e:
        e2e_ms, e2e_records = float("nan"), 0
    else:
        e2e_ms, e2e_records = run_e2e(ctx, imgs, sizes, p, cap, stream, args, barrier, dist, cdvs, torch)
    h2d = n * H * W
    d2h = n * 4 + e2e_records * (cdvs.KEYPOINT_DTYPE.itemsize + 128 * 4) + 8
    try:
        per_image = run_per_image(ctx, cdvs, torch, dptrs, sizes, p, d_kp, d_desc, d_cnt, stream)
    except Exception as ex:  # reported, never fatal to the main line
        per_image = {"error": str(ex)}
    # ---- roofline of the dominant kernel: the octave-0 detection launch (K1)
    peaks = load_peaks()
    flops_o, bytes_o = detect_counts(p)
    o0_ms = prof["detect_octave0"][0] / args.steps
    tflops = flops_o[0] * n / (o0_ms * 1e-3) / 1e12
    sm_max = clocks.get("sm_max_mhz") or device_max_mhz()
    alu_peak, sms = alu_peak_tflops(torch, local, sm_max)
    try:
        sgemm = measure_sgemm_tflops(torch)
    except Exception:
        sgemm = None
    try:
        ffma2 = ctx.probe_fp32_rate()
    except Exception:
        ffma2 = None
    gbs = bytes_o[0] * n / (o0_ms * 1e-3) / 1e9
    v0 = int(tuning["last_call_variants"][0])
    traffic = load_traffic(v0)
    det_ms = prof["detect"][0] / args.steps
    roofline = {"kernel": "detect_kernel, octave-0 launch (K1: 4 Gaussian levels + LoG + ALP + extremum + refine), "
                          f"variant {v0}: {tuning['variants'][v0]}",
                "bound": "alu", "achieved": tflops, "peak": alu_peak, "unit": "TFLOP/s", "frac": tflops / alu_peak,
                "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz "
                               "(SM count and maximum clock queried from the device)",
                "measured_fp32": {"sgemm_tflops": sgemm, "frac": (tflops / sgemm) if sgemm else None,
                                  "source": "cuBLAS SGEMM 8192^3 with TF32 off, best of 5 (of measured)"},
                "measured_ffma2": {"tflops": ffma2, "frac": (tflops / ffma2) if ffma2 else None,
                                   "source": "cdvs_probe_fp32_rate: fma.rn.f32x2 register loop on every SM "
                                             "(of measured)"},
                "traffic": (traffic["dram_bytes_per_image_octave0"] * n if traffic else None),
                "algorithmic_flops_per_launch": flops_o[0] * n, "algorithmic_bytes_per_launch": bytes_o[0] * n,
                "launch_ms": o0_ms,
                "hbm": {"achieved": gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                        "frac": (gbs / peaks["hbm_gbs"]) if peaks.get("hbm_gbs") else None,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
                "all_octaves": {"ms": det_ms, "tflops": sum(flops_o) * n / (det_ms * 1e-3) / 1e12,
                                "gbs": sum(bytes_o) * n / (det_ms * 1e-3) / 1e9},
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    launches = sum(v[1] for k, v in prof.items() if k != "detect_octave0")

    out = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.storage == "fp32" else "f32 (fp16 level storage)",
           "data": "synthetic",
           "config": {"workload": f"{N_IMAGES}x {WIDTH}x{HEIGHT} u8 seeded blob images, 4 octaves x 4 LoG scales, "
                                  f"N=300, 128-D float descriptors", "n_images_per_rank": n,
                      "storage": args.storage, "parallelism": f"replicas x{world} (image-sharded)",
                      "l2": "working set > L2: each step writes 1.7 GB of levels", "records_per_step": records},
           "e2e": {"value": (n * world / (e2e_ms * 1e-3)) if e2e_ms == e2e_ms else None, "unit": "images/s",
                   "ms_per_step": e2e_ms if e2e_ms == e2e_ms else None,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": launches, "roofline": roofline, "clocks": clocks, "detect_tuning": tuning}
    out["one_image_per_call"] = per_image
    if legs is not None:
        (u_imgs, u_sizes), h_imgs = legs
        try:
            out["uneven"] = uneven_leg(ctx, cdvs, torch, u_imgs, u_sizes, args, alu_peak)
        except Exception as ex:  # reported, never fatal to the main line
            out["uneven"] = {"error": str(ex)}
        try:
            out["highres"] = highres_leg(ctx, cdvs, torch, h_imgs, args, alu_peak)
        except Exception as ex:
            out["highres"] = {"error": str(ex)}
    if learned is not None:
        st_none = learned["no_block_proposed"]["stage_ms_per_step"]
        learned["break_even_skipped_tile_share"] = break_even_share(
            st_none.get("proposal", float("nan")), o0_ms, st_none.get("detect_octave0", float("nan")))
        out["learned"] = learned
    if scfv is not None:
        out["scfv"] = scfv
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(imgs)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    ctx.close()


if __name__ == "__main__":
    main()
