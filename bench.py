#!/usr/bin/env python
"""Throughput of one mapping-loop step (fwd + bwd) on GB300.

Workload "indoor-640x480-300k": 300k Gaussians uniform in a 6x6x3 m room,
one 640x480 keyframe (fx=fy=525) on a 2 m arc around the room centre,
RGB + depth + a 16-d language feature.  A step is the whole hot path:
projection, tile binning, compositing, the L1 terms of Eq. 1, the frozen
decoder with the L1 distillation loss of Eq. 2 and its gradient, and the
render backward down to every Gaussian parameter.  The plain path renders
all 512 embedding channels instead of the decoder (reported beside it).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on bounded crops of the same workload instead.
"""
from __future__ import annotations

import argparse
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

METRIC = "fwd+bwd Mpix/s, 300k Gaussians 640x480, 16-d vs plain 512-d; % of roofline"
WORKLOAD = "indoor-640x480-300k"
L2_BYTES = 129 * 2 ** 20
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="lgs", choices=["lgs", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain 512-d path")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline")
    ap.add_argument("--ae-steps", type=int, default=200)
    ap.add_argument("--no-window", action="store_true",
                    help="skip the 8-keyframe window workload")
    ap.add_argument("--no-outdoor", action="store_true",
                    help="skip the outdoor-scale workload (2M Gaussians, 8 x 1200x680)")
    ap.add_argument("--profile", action="store_true",
                    help="run warmup + steps eager mapping steps and exit (for ncu)")
    ap.add_argument("--profile-ae", action="store_true",
                    help="run warmup + steps eager ae_train_step calls (RECON, 65,536 "
                         "unit-norm 512-d pixels) and exit (for ncu)")
    ap.add_argument("--profile-prune", action="store_true",
                    help="run warmup + steps eager gs_prune calls on the indoor map with its "
                         "encoder-prior features and exit (for ncu)")
    return ap.parse_args()


# --------------------------------------------------------------------------- workload

def build_workload(rank):
    """Host arrays of the workload: the indoor scene with spatially coherent
    512-d semantics (64 3D Voronoi cells of the room), its 8 arc keyframes,
    the keyframe this rank renders, and RGB / depth targets."""
    from paper_2511_16144_gb300 import synth
    scene, cams = synth.indoor(n_cams=8)
    g512 = synth.semantic_features(scene.means, synth.ROOM_LO, synth.ROOM_HI, seed=1005)
    cam = cams[keyframe_of_rank(rank)]
    (rgb_t, dep_t, _), = synth.targets([cam], feat_dim=16, seed=2001 + rank)
    return dict(scene=scene, cams=cams, cam=cam, g512=g512, rgb_t=rgb_t, dep_t=dep_t)


def keyframe_of_rank(rank, n_keyframes=8):
    """Replicas: rank r renders keyframe r mod 8 of the window against its
    own copy of the map (no exchange between ranks)."""
    return rank % n_keyframes


def max_over_ranks(x, world, device="cpu"):
    """The largest x over all ranks of the process group (x when alone): the
    job's time is its slowest rank's."""
    if world == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pixels_per_rank, steps, world, total_ms):
    """Whole-job Mpix/s: every rank's pixels of every timed step over the
    slowest rank's time."""
    return world * pixels_per_rank * steps / 1e6 / (total_ms / 1e3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(1.0)  # the sampler's own start-up, before the timed region
        except OSError:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *exc):
        self.t1 = time.time()
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(f[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + f[0].split(".")[1]) if "." in f[0] else 0.0
            except (ValueError, IndexError):
                ts = None
            rows.append((ts, f[1:]))
        # samples taken while the timed steps ran (all of them if none parse)
        inside = [f for ts, f in rows if ts is not None and self.t0 - 0.05 <= ts <= self.t1 + 0.05]
        for f in inside or [f for _, f in rows]:
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_window": bool(inside)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------- GPU arm

def run_gpu(args, rank, world):
    import torch
    from paper_2511_16144_gb300 import build, lgs, synth
    from paper_2511_16144_gb300.ae import AutoEncoder
    from paper_2511_16144_gb300.pipeline import MappingStep
    from paper_2511_16144_gb300.render import DeviceScene

    build.build()
    lgs.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.profile_ae:
        m = AutoEncoder(*synth.ae_init(seed=3001), device=dev)
        gen = torch.Generator(device="cpu").manual_seed(0)
        x = torch.nn.functional.normalize(torch.randn(65536, 512, generator=gen), dim=1)
        x = x.to(dev).bfloat16()
        loss = torch.zeros(1, device=dev)
        for _ in range(args.warmup + args.steps):
            m.train_step(x, lr=1e-4, loss=loss)
        torch.cuda.synchronize()
        print(f"profile-ae: {args.warmup + args.steps} eager training steps, loss {loss.item():.4f}")
        return
    W = build_workload(rank)
    scene, cam = W["scene"], W["cam"]
    from paper_2511_16144_gb300.render import Frame

    geom = DeviceScene.from_host(scene, device=dev)
    colors_bf = geom.colors.bfloat16()
    g512_bf = torch.from_numpy(W["g512"]).to(dev).bfloat16()
    g512_f32 = torch.from_numpy(W["g512"]).to(dev)
    s512 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                       colors_bf, g512_bf)
    s512_f32 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                           geom.colors, g512_f32)
    # the extractor's per-frame 512-d maps: the semantic field rendered by the
    # plain path for every keyframe of the window (BF16), F_gt = this rank's
    frames = [Frame(s512, [c]).out["feat"][0].reshape(-1, 512).bfloat16() for c in W["cams"]]
    f_gt = frames[keyframe_of_rank(rank)].contiguous()

    # scene-adaptive autoencoder pretrained online on those maps (Sec. IV-A.2);
    # the encoder prior gives the Gaussians' 16-d features (Sec. III-B.2)
    enc, dec = synth.ae_init(seed=3001)
    model = AutoEncoder(enc, dec, device=dev)
    train = torch.cat(frames)
    gen = torch.Generator(device=dev).manual_seed(rank)
    ae_losses = []
    t0 = time.time()
    for _ in range(args.ae_steps):
        idx = torch.randint(0, train.shape[0], (65536,), device=dev, generator=gen)
        ae_losses.append(model.train_step(train[idx].contiguous(), lr=5e-3))
    torch.cuda.synchronize()
    ae_train_s = time.time() - t0
    ae_losses = [float(l.item()) for l in ae_losses] or [float("nan")]
    del train
    f16 = model.encode(g512_bf)
    s16_bf = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                         colors_bf, f16.bfloat16().contiguous())
    s16_f32 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                          geom.colors, f16.contiguous())
    rgb_t = torch.from_numpy(W["rgb_t"][None]).to(dev).contiguous()
    dep_t = torch.from_numpy(W["dep_t"][None]).to(dev).contiguous()
    cams = [cam]
    W["f_gt"] = f_gt.float().cpu().numpy().reshape(cam.height, cam.width, 512)

    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(step, k, warm, clocks=None):
        return timed_graph_steps(step.run, k, warm, flush, world, clocks)

    if args.profile_prune:
        params = lgs.prune_params(synth.ROOM_LO, synth.ROOM_HI, **PRUNE_PARAMS)
        for _ in range(args.warmup + args.steps):
            mask, cnt = lgs.gs_prune(s16_bf.means, s16_bf.opacity_logits, s16_bf.log_scales,
                                     s16_bf.feats, params)
        torch.cuda.synchronize()
        print(f"profile-prune: {args.warmup + args.steps} eager calls, {int(cnt.item())} pruned")
        return
    step16 = MappingStep(s16_bf, cams, rgb_t, dep_t, f_gt, model=model)
    if args.profile:
        for _ in range(args.warmup + args.steps):
            step16.run()
        torch.cuda.synchronize()
        print(f"profile: {args.warmup + args.steps} eager steps, K = {int(step16.k_dev.item())}")
        return
    clocks = Clocks(torch.cuda.current_device())
    t16, g16, nodes16 = timed(step16, args.steps, args.warmup, clocks)
    step16.check()  # the bins held every instance of every timed step
    k_inst = int(step16.k_dev.item())
    ms16 = float(np.mean(t16))
    total_ms = max_over_ranks(float(sum(t16)), world, dev)
    pixels = step16.pixels
    value = job_throughput(pixels, args.steps, world, total_ms)

    # per-call durations of one eager step (events on the launching stream)
    calls = per_call_times(step16, flush, reps=5)
    kern, counts = rooflines(step16, calls)
    top = max(calls, key=calls.get)
    rf = dict(kern[top], kernel=top)

    # FP32-channel variant and the plain 512-channel path (same geometry)
    extra = {}
    step16f = MappingStep(s16_f32, cams, rgb_t, dep_t, f_gt, model=model,
                          capacity=step16.bufs.capacity)
    tf, _, _ = timed(step16f, max(5, args.steps // 2), 2)
    extra["fp32_channels"] = {"value": pixels / 1e6 / (np.mean(tf) / 1e3), "ms_per_step": float(np.mean(tf))}
    plain = None
    cos_err = None
    if not args.no_plain:
        step512 = MappingStep(s512, cams, rgb_t, dep_t, f_gt, model=None,
                              capacity=step16.bufs.capacity)
        tp, _, _ = timed(step512, max(5, args.steps // 2), 2)
        plain = {"value": pixels / 1e6 / (np.mean(tp) / 1e3), "ms_per_step": float(np.mean(tp)),
                 "channels": "bf16", "feat_dim": 512}
        plain["speedup_of_16d"] = value / world / plain["value"]
        del step512
    # feature-width sweep (the d ablation of Sec. IV): the same step rendering
    # d BF16 channels with an L1 against a d-channel target, no autoencoder
    sweep = []
    if not args.no_plain:
        gen_f = torch.Generator(device=dev).manual_seed(4000)
        for d in (8, 16, 32, 64, 128):
            fd = torch.randn((scene.n, d), device=dev, generator=gen_f)
            fd = (fd / fd.norm(dim=1, keepdim=True)).bfloat16().contiguous()
            tgt = torch.randn((pixels, d), device=dev, generator=gen_f).bfloat16()
            sd = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                             colors_bf, fd)
            st = MappingStep(sd, cams, rgb_t, dep_t, tgt, model=None,
                             capacity=step16.bufs.capacity)
            td, _, _ = timed(st, max(5, args.steps // 4), 3)
            sweep.append({"d": d, "ms_per_step": float(np.mean(td)),
                          "Mpix_per_s": pixels / 1e6 / (np.mean(td) / 1e3),
                          "map_bytes_per_gaussian": 44 + 6 + 2 * d})
            del st, sd, fd, tgt
    # decoded 16-d features against the plain 512-channel FP32 render, per pixel
    step16.run()
    torch.cuda.synchronize()
    y = model.decode(step16.out["feat"].reshape(-1, 16).contiguous())
    ref = Frame(s512_f32, cams).out["feat"][0].reshape(-1, 512)
    nr = ref.norm(dim=1)
    keep = nr > 1e-6
    cos = (y * ref).sum(1)[keep] / (y.norm(dim=1)[keep] * nr[keep]).clamp_min(1e-30)
    cos_err = {"mean": float((1 - cos).mean().item()), "excluded_pixels": int((~keep).sum().item()),
               "reference": "plain 512-channel FP32 render of the same Gaussians"}
    del y, ref

    window = None if args.no_window else measure_window(W, s16_bf, frames, model, flush, dev,
                                                        world)
    del frames

    # end to end through the C ABI with host buffers: per step the keyframe's
    # targets (RGB, depth, F_gt) go host -> device from pinned memory and the
    # loss comes back
    prune = measure_prune(s16_bf, flush)
    extras = measure_loss_pose(step16, flush)
    ae_rf = measure_autoencoder(enc, dec, g512_bf, flush, dev)
    extras.update(measure_loop_query(step16, f_gt, flush))

    rgb_b, dep_b, fgt_b = rgb_t.clone(), dep_t.clone(), f_gt.clone()
    step16b = MappingStep(s16_bf, cams, rgb_b, dep_b, fgt_b, model=model,
                          capacity=step16.bufs.capacity)
    _, g16b, _ = timed(step16b, 1, 1)
    e2e = measure_e2e([step16, step16b], [g16, g16b], args.steps, args.warmup)
    del step16b, g16b, step16f
    outdoor = None
    if not args.no_outdoor:
        del g16
        outdoor = measure_outdoor(args, flush, dev, world)

    if rank == 0:
        peaks, kind = measured_peaks()
        cpu = None if args.no_cpu else cpu_baseline(W, budget_s=15.0)
        line = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms16,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": scene.n, "cameras": 1, "width": 640,
                       "height": 480, "feat_dim": 16, "channels": "bf16",
                       "precision": "fp32 alpha/T/accumulation; bf16 channels and AE GEMMs",
                       "instances": k_inst, "l2": "flushed before every step (258 MB write)",
                       "graph": "one CUDA graph per step", "parallelism": "replicas" if world > 1 else "single"},
            "gpu_launches": nodes16 * args.steps if nodes16 > 0 else None,
            "kernels_per_step": nodes16,
            "roofline": rf, "rooflines": kern, "work_counts": counts,
            "e2e": e2e,
            "clocks": clocks.summary(),
            "speedup_16d_over_plain_512": plain["speedup_of_16d"] if plain else None,
            "decoded_cosine_error_mean": cos_err["mean"] if cos_err else None,
            "plain_512": plain, "decoded_cosine_error": cos_err, "variants": extra,
            "workloads": {"indoor-window-8x640x480-300k": window,
                          "outdoor-8x1200x680-2M": outdoor},
            "prune": prune, "feature_dim_sweep": sweep, "dssim_and_pose": extras,
            "per_call_ms": calls,
            "ae_pretrain": {"steps": args.ae_steps, "loss_first": ae_losses[0],
                            "loss_last": ae_losses[-1], "seconds": ae_train_s},
            "autoencoder": ae_rf,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def step_report(step, run, k, warm, flush, world, pixels):
    """Times one composed step (graph replays) and its call groups; returns
    the per-step figures, the per-call rooflines and the work counts."""
    t, _, nodes = timed_graph_steps(run, k, warm, flush, world)
    step.check()  # LGS_ERR_CAPACITY etc. would have emptied the bins
    ms = float(np.mean(t))
    calls = per_call_times(step, flush, reps=3)
    kern, counts = rooflines(step, calls)
    return {"ms_per_step": ms, "value": pixels / 1e6 / (ms / 1e3), "unit": "Mpix/s",
            "kernels_per_step": nodes, "per_call_ms": calls, "rooflines": kern,
            "work_counts": counts}


def measure_window(W, s16_bf, f_gt_frames, model, flush, dev, world, k=20, warm=3):
    """The differentiable mapping window: the 8 arc keyframes of the room
    (640x480, 300k Gaussians) in one launch, 2.46 Mpx per step.  Two
    variants: the window's own loss, L1 on RGB + 0.1 L1 on depth + L1 on the
    16-d feature against a 16-d target (no decoder), and the production path
    with the feature term through the frozen decoder against the 512-d F_gt
    of every keyframe (Eq. 2)."""
    import torch
    from paper_2511_16144_gb300 import synth
    from paper_2511_16144_gb300.pipeline import MappingStep
    cams = W["cams"]
    tg = synth.targets(cams, feat_dim=16, seed=2100)
    rgb8 = torch.from_numpy(np.stack([t[0] for t in tg])).to(dev)
    dep8 = torch.from_numpy(np.stack([t[1] for t in tg])).to(dev)
    f16 = torch.from_numpy(np.stack([t[2] for t in tg]).reshape(-1, 16)).to(dev).bfloat16()
    pixels = len(cams) * cams[0].width * cams[0].height
    out = {"workload": "indoor-window-8x640x480-300k", "cameras": len(cams), "pixels": pixels}
    st = MappingStep(s16_bf, cams, rgb8, dep8, f16, model=None)
    out["l1_16d"] = step_report(st, st.run, k, warm, flush, world, pixels)
    out["instances"] = int(st.k_dev.item())
    cap = st.bufs.capacity
    del st
    f_gt8 = torch.cat(f_gt_frames).contiguous()
    st = MappingStep(s16_bf, cams, rgb8, dep8, f_gt8, model=model, capacity=cap)
    out["decoded"] = step_report(st, st.run, k, warm, flush, world, pixels)
    del st, f_gt8
    return out


def measure_outdoor(args, flush, dev, world, k=8, warm=3):
    """The outdoor-scale window: 2M Gaussians in a 40x40x8 m volume, 8
    keyframes of 1200x680 (6.53 Mpx), BF16 channels, the 16-d render with the
    feature term through the decoder (Eq. 2), plus one online autoencoder
    step (RECON, 65,536 pixels of the window's maps) per window, after a
    pretraining of three times the room's steps; against the plain path that
    renders all 512 channels, with the decoded 16-d
    features' cosine error against the plain FP32 render of the first
    keyframe.  The 512-d semantic field is generated on the device (same
    recipe as the room's, 64 Voronoi cells of the volume)."""
    import torch
    from paper_2511_16144_gb300 import lgs, synth
    from paper_2511_16144_gb300.ae import AutoEncoder
    from paper_2511_16144_gb300.pipeline import MappingStep
    from paper_2511_16144_gb300.render import DeviceScene, Frame
    t0 = time.time()
    scene, cams = synth.outdoor()
    geom = DeviceScene.from_host(scene, device=dev)
    colors_bf = geom.colors.bfloat16()
    g512 = synth.semantic_features_device(geom.means, (0.0, 0.0, 0.0), (40.0, 40.0, 8.0),
                                          seed=1006, out_dtype=torch.bfloat16)
    s512 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits,
                       colors_bf, g512)
    frames = [Frame(s512, [c]).out["feat"][0].reshape(-1, 512).bfloat16() for c in cams]
    enc, dec = synth.ae_init(seed=3004)
    model = AutoEncoder(enc, dec, device=dev)
    train = torch.cat(frames)
    gen = torch.Generator(device=dev).manual_seed(11)
    # the outdoor window's maps hold 21x the room's pixels: three times the
    # steps (at twice, the seeded run stops at 0.020 mean cosine error; at
    # three times it reaches 0.007)
    for _ in range(3 * args.ae_steps):
        idx = torch.randint(0, train.shape[0], (65536,), device=dev, generator=gen)
        model.train_step(train[idx].contiguous(), lr=5e-3)
    batch = train[torch.randint(0, train.shape[0], (65536,), device=dev, generator=gen)].contiguous()
    del train
    f16 = model.encode(g512)
    s16 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits, colors_bf,
                      f16.bfloat16().contiguous())
    tg = synth.targets(cams, feat_dim=16, seed=2200)
    rgb8 = torch.from_numpy(np.stack([t[0] for t in tg])).to(dev)
    dep8 = torch.from_numpy(np.stack([t[1] for t in tg])).to(dev)
    f_gt8 = torch.cat(frames).contiguous()
    del frames
    pixels = len(cams) * cams[0].width * cams[0].height
    setup_s = time.time() - t0
    out = {"workload": "outdoor-8x1200x680-2M", "gaussians": scene.n, "cameras": len(cams),
           "pixels": pixels, "channels": "bf16", "setup_s": setup_s}
    # decoded features of the first keyframe against the plain FP32 render
    st = MappingStep(s16, cams[:1], rgb8[:1].contiguous(), dep8[:1].contiguous(),
                     f_gt8[:cams[0].width * cams[0].height], model=model)
    st.run()
    torch.cuda.synchronize()
    y = model.decode(st.out["feat"].reshape(-1, 16).contiguous())
    del st
    g32 = DeviceScene(geom.means, geom.quats, geom.log_scales, geom.opacity_logits, geom.colors,
                      g512.float())
    ref = Frame(g32, cams[:1]).out["feat"][0].reshape(-1, 512)
    del g32
    nr = ref.norm(dim=1)
    keep = nr > 1e-6
    cos = (y * ref).sum(1)[keep] / (y.norm(dim=1)[keep] * nr[keep]).clamp_min(1e-30)
    out["decoded_cosine_error"] = {"mean": float((1 - cos).mean().item()),
                                   "excluded_pixels": int((~keep).sum().item()),
                                   "keyframe": 0}
    del y, ref
    step = MappingStep(s16, cams, rgb8, dep8, f_gt8, model=model)
    ae_loss = torch.zeros(1, device=dev)

    def run16():
        step.run()
        model.train_step(batch, lr=1e-4, loss=ae_loss)  # one online AE step per window

    out["decoded"] = step_report(step, run16, k, warm, flush, world, pixels)
    out["instances"] = int(step.k_dev.item())
    cap = step.bufs.capacity
    t_ae, _, _ = timed_graph_steps(lambda: model.train_step(batch, lr=1e-4, loss=ae_loss), 5, 2,
                                   flush, world)
    out["decoded"]["ae_train_step_ms"] = float(np.mean(t_ae))
    del step
    if not args.no_plain:
        plain = MappingStep(s512, cams, rgb8, dep8, f_gt8, model=None, capacity=cap)
        t, _, _ = timed_graph_steps(plain.run, 3, 1, flush, world)
        plain.check()
        ms = float(np.mean(t))
        out["plain_512"] = {"ms_per_step": ms, "value": pixels / 1e6 / (ms / 1e3),
                            "channels": "bf16", "feat_dim": 512}
        out["speedup_16d_over_plain_512"] = out["decoded"]["value"] / out["plain_512"]["value"]
        del plain
    lgs.check_device("outdoor workload")
    return out



def timed_graph_steps(run, k, warm, flush, world, clocks=None):
    """Captures run() (one step's enqueues) in a CUDA graph and replays it:
    warm untimed replays, then k replays each between CUDA events on the
    launching stream, L2 flushed before every replay outside the events.
    Returns (per-replay ms, graph, kernel nodes of one step)."""
    import torch
    dev = torch.cuda.current_device()
    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run()  # eager once (also sets kernel attributes and workspaces)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    torch.cuda.synchronize()
    nodes = kernel_nodes(run)
    for _ in range(warm):
        flush.fill_(1.0)
        g.replay()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(k)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        for i in range(k):
            flush.fill_(1.0)
            ev[i][0].record()
            g.replay()
            ev[i][1].record()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    return [a.elapsed_time(b) for a, b in ev], g, nodes



class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def kernel_nodes(fn):
    """Kernel nodes in a CUDA graph captured from fn (every one is a liblgs
    kernel: the step's fills are memset nodes), or -1 if unavailable."""
    import ctypes

    import torch
    from paper_2511_16144_gb300 import lgs
    try:
        g = torch.cuda.CUDAGraph(keep_graph=True)
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        n = int(lgs.load().lgs_graph_kernel_nodes(ctypes.c_void_p(int(g.raw_cuda_graph()))))
        del g
        return n
    except (TypeError, RuntimeError, AttributeError):
        return -1


def per_call_times(step, flush, reps=5):
    """Average device time (ms) of each C-ABI call group of the step: each is
    captured in its own CUDA graph and replayed between CUDA events on the
    launching stream, with L2 flushed before every replay."""
    import torch
    step.run()
    torch.cuda.synchronize()
    out = {}
    for name, fn in step.calls():
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        flush.fill_(1.0)
        g.replay()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.mean(ts))
        del g
    return out


# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch
# of each call group at this workload, from the capture summarised under
# profiles/, with a digest of the sources of that call group's kernels at
# capture time: a figure whose sources have changed since is reported as
# None instead of a stale number.
TRAFFIC_SOURCES = {
    "gs_project": ("project.cu", "common.cuh", "kernels.cuh"),
    "gs_bin_sort": ("binning.cu", "common.cuh", "kernels.cuh"),
    "gs_render_fwd": ("render.cu", "common.cuh", "kernels.cuh"),
    "l1_losses": ("api.cu", "common.cuh"),
    "ae_decode": ("ae_fused.cu", "tc05.cuh", "common.cuh", "kernels.cuh"),
    "gs_render_bwd": ("render.cu", "project.cu", "common.cuh", "kernels.cuh"),
}
TRAFFIC = {  # call group -> (bytes per launch, source digest)
    "gs_project": (13217024, "11cb2be17fcb"),
    "gs_bin_sort": (37627648, "18d76b8a2256"),
    "gs_render_fwd": (5515264, "011d53f72718"),
    "l1_losses": (9845504, "792f0809c2a4"),
    "ae_decode": (349692160, "ec4aea27d248"),
    "gs_render_bwd": (41203456, "5fcc646473a8"),
}


def source_digest(group):
    """First 12 hex digits of the SHA-256 of the sources of a call group."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[group]:
        with open(os.path.join(ROOT, "paper_2511_16144_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def current_traffic(group):
    entry = TRAFFIC.get(group)
    if entry is None or entry[1] != source_digest(group):
        return None
    return entry[0]


def rooflines(step, calls):
    """Roofline position of every call group of the step.

    Algorithmic work per launch (the per-unit figures of the hot-path scope,
    times the units one launch processes):
      gs_project    HBM  44 B per Gaussian read + 40 B per (camera, Gaussian) written
      gs_bin_sort   HBM  36 B per instance (emit write + one read/write pass of
                         12-byte records) + 8 B per tile range + 40 B per
                         (camera, Gaussian) record read (rect and the tile
                         test's projected record)
      gs_render_fwd ALU  10 FLOP per evaluated (pixel, instance) pair E +
                         2 (4 + d) + 4 per blended pair B
      l1_losses     HBM  48 B per pixel (RGB and depth: prediction, target, gradient)
      ae_decode     BF16 tensor  2 x 346 112 FLOP per pixel (decoder forward and
                         gradient to the rendered map)
      gs_render_bwd ALU  10 FLOP per E + 4 (4 + d) + 25 per B
    E = sum over pixels of `last` (instances walked), B = instances blended,
    both read from the forward.  Peaks: measured HBM copy bandwidth and bf16
    GEMM rate (burst: each call is timed alone), FP32 lanes x clock for ALU."""
    peaks, kind = measured_peaks()
    E = float(step.out["last"].double().sum().item())
    B = float(step.count_blended().double().sum().item())
    K = float(step.k_dev.item())
    d, n, c, P = step.D, step.scene.n, len(step.cams), step.pixels
    tiles = step.bufs.tiles_x * step.bufs.tiles_y * c
    alu = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    hbm, tc = float(peaks["hbm_gbs"]), float(peaks["bf16_tflops"])
    work = {
        "gs_project": ("hbm", 44.0 * n + 40.0 * c * n),
        "gs_bin_sort": ("hbm", 36.0 * K + 8.0 * tiles + 40.0 * c * n),
        "gs_render_fwd": ("alu", 10.0 * E + (2.0 * (4 + d) + 4.0) * B),
        "l1_losses": ("hbm", 48.0 * P),
        "ae_decode": ("tensor", 2.0 * 346112.0 * P),
        "gs_render_bwd": ("alu", 10.0 * E + (4.0 * (4 + d) + 25.0) * B),
    }
    out = {}
    for name, ms in calls.items():
        bound, units = work[name]
        if bound == "hbm":
            achieved, peak, unit = units / (ms / 1e3) / 1e9, hbm, "GB/s"
        else:
            achieved = units / (ms / 1e3) / 1e12
            peak, unit = (tc, "TFLOP/s") if bound == "tensor" else (alu, "TFLOP/s")
        out[name] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                     "frac": achieved / peak, "traffic": current_traffic(name),
                     "work_per_launch": units, "ms_per_launch": ms,
                     "peak_source": ("fp32 lanes: " + FP32_PEAK_NOTE) if bound == "alu"
                     else kind + (" bf16 burst" if bound == "tensor" else " copy")}
    counts = {"E_pairs": E, "B_pairs": B, "instances": K}
    return out, counts


PRUNE_PARAMS = dict(k=8, tau_dist=0.05, tau_sim=0.9, min_opacity=0.005, max_scale=0.5)


def measure_prune(scene, flush, reps=20):
    """Language-guided pruning (Sec. III-C, Eq. 4 + geometric criteria) over
    the whole map with its 16-d BF16 features, and the compaction of every
    parameter array that follows; each captured in a CUDA graph and timed
    between CUDA events with L2 flushed before every replay.  Algorithmic
    bytes of the mask: one read of the parameters the rule looks at (means,
    logit, log-scales, 16 BF16 features = 60 B) + 1 mask byte per Gaussian."""
    import ctypes

    import torch
    from paper_2511_16144_gb300 import lgs, synth
    L = lgs.load()
    n = scene.n
    dev = scene.means.device
    params = lgs.prune_params(synth.ROOM_LO, synth.ROOM_HI, **PRUNE_PARAMS)
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    cnt = torch.empty(1, dtype=torch.int64, device=dev)
    ws = torch.empty(int(L.gs_prune_workspace(n)), dtype=torch.uint8, device=dev)
    arrays = [scene.means, scene.quats, scene.log_scales, scene.opacity_logits, scene.colors,
              scene.feats]
    dst = [torch.empty_like(a) for a in arrays]
    new_index = torch.empty(n, dtype=torch.int32, device=dev)
    kept = torch.empty(1, dtype=torch.int64, device=dev)
    cws = torch.empty(int(L.gs_compact_workspace(n)), dtype=torch.uint8, device=dev)
    p = lgs._p

    def run_prune():
        lgs.gs_prune(scene.means, scene.opacity_logits, scene.log_scales, scene.feats, params,
                     mask, cnt, ws)

    def run_compact():
        lgs._check(L.gs_compact_index(p(mask), n, p(new_index), p(kept), p(cws), cws.numel(),
                                      lgs._stream()), "gs_compact_index")
        for a, d in zip(arrays, dst):
            lgs._check(L.gs_gather_rows(p(a), n, a[0].numel() * a.element_size(), p(new_index),
                                        p(d), lgs._stream()), "gs_gather_rows")

    def time_graph(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    ms = time_graph(run_prune)
    m = mask.cpu().numpy()
    ms_c = time_graph(run_compact)
    peaks, kind = measured_peaks()
    achieved = 61.0 * n / (ms / 1e3) / 1e9
    return {"ms": ms, "gaussians_per_s": n / (ms / 1e3), "params": PRUNE_PARAMS,
            "pruned_fraction": float((m != 0).mean()),
            "redundant_fraction": float(((m & 2) != 0).mean()),
            "geometric_fraction": float(((m & 1) != 0).mean()),
            "compaction_ms": ms_c,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]),
                         "unit": "GB/s", "frac": achieved / float(peaks["hbm_gbs"]),
                         "traffic": None, "peak_source": kind + " copy",
                         "note": "61 B per Gaussian: the inputs the rule reads once, the mask byte"}}


def measure_loss_pose(step, flush, reps=20):
    """The D-SSIM term of L_rgb (Sec. III-B.3) on the step's 640x480 render
    and the camera pose gradient (Sec. III-B.2) from its backward's 2D
    records, each alone in a CUDA graph between CUDA events (L2 flushed)."""
    import torch
    from paper_2511_16144_gb300 import lgs
    step.run()
    torch.cuda.synchronize()
    rgb = step.out["rgb"]
    grad = torch.zeros_like(rgb)
    loss = torch.zeros(1, device=rgb.device)
    ws = torch.empty(int(lgs.load().lgs_dssim_workspace(*rgb.shape[:3])), dtype=torch.uint8,
                     device=rgb.device)
    sc = step.scene
    d_pose = torch.empty((len(step.cams), 6), device=rgb.device)

    def dssim():
        lgs.lgs_dssim_loss(rgb, step.rgb_t, 0.2, grad, loss, ws)

    def pose():
        lgs.gs_pose_grad(sc.means, sc.quats, sc.log_scales, sc.opacity_logits, step.cams,
                         step.grad2d, d_pose)

    out = {}
    for name, fn in (("dssim_ms", dssim), ("pose_grad_ms", pose)):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.median(ts))
    px = rgb.shape[0] * rgb.shape[1] * rgb.shape[2]
    # algorithmic bytes of D-SSIM: read pred and target, write and re-read the
    # three gradient maps, read-modify-write the gradient (12 B per value each)
    byts = px * 3 * 4 * (2 + 3 + 3 + 2)
    peaks, kind = measured_peaks()
    out["dssim_roofline"] = {"bound": "hbm", "achieved": byts / (out["dssim_ms"] / 1e3) / 1e9,
                             "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                             "frac": byts / (out["dssim_ms"] / 1e3) / 1e9 / float(peaks["hbm_gbs"]),
                             "peak_source": kind + " copy"}
    return out


def measure_loop_query(step, f_gt, flush, reps=20, K=256, Q=8):
    """The keyframe's loop signature (Sec. III-D: closest of K codewords for
    every 512-d F_gt pixel on the tensor cores, histogram) and the relevance
    of Q compact-space queries (Sec. I) over the rendered 16-d map, each
    alone in a CUDA graph between CUDA events (L2 flushed).  The codebook is
    synthetic (unit codewords): the paper's comes from external datasets."""
    import torch
    from paper_2511_16144_gb300 import lgs
    dev = f_gt.device
    gen = torch.Generator(device=dev).manual_seed(4100)
    cb = torch.randn((K, 512), device=dev, generator=gen)
    cb = (cb / cb.norm(dim=1, keepdim=True)).bfloat16().contiguous()
    hist = torch.zeros(K, dtype=torch.int32, device=dev)
    ws = torch.empty(int(lgs.load().lgs_codebook_workspace(K)), dtype=torch.uint8, device=dev)
    feat = step.out["feat"].reshape(-1, step.D)
    q = torch.randn((Q, step.D), device=dev, generator=gen)
    rel = torch.empty((feat.shape[0], Q), device=dev)

    def assign():
        lgs.lgs_codebook_assign(f_gt, cb, hist=hist, ws=ws)

    def query():
        lgs.gs_query_relevance(feat, q, rel)

    out = {}
    for name, fn in (("codebook_assign_ms", assign), ("query_relevance_ms", query)):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.median(ts))
    peaks, kind = measured_peaks()
    P = f_gt.shape[0]
    fl = 2.0 * P * 512 * K
    out["codebook_assign_roofline"] = {
        "bound": "tensor", "achieved": fl / (out["codebook_assign_ms"] / 1e3) / 1e12,
        "peak": float(peaks["bf16_tflops"]), "unit": "TFLOP/s",
        "frac": fl / (out["codebook_assign_ms"] / 1e3) / 1e12 / float(peaks["bf16_tflops"]),
        "peak_source": kind + " bf16 burst", "codebook": K}
    byts = float(feat.numel() * 4 + P * Q * 4)
    out["query_relevance_roofline"] = {
        "bound": "hbm", "achieved": byts / (out["query_relevance_ms"] / 1e3) / 1e9,
        "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
        "frac": byts / (out["query_relevance_ms"] / 1e3) / 1e9 / float(peaks["hbm_gbs"]),
        "peak_source": kind + " copy", "queries": Q}
    return out


def measure_autoencoder(enc, dec, g512_bf, flush, dev, reps=20):
    """Roofline of the autoencoder calls outside the step: one ae_train_step
    (RECON, 65,536 pixels: forward, gradient to the activations and to the
    weights, and Adam, for encoder and decoder) and one ae_encode of the
    Gaussians' 512-d features, each captured in a CUDA graph and replayed
    between CUDA events with L2 flushed before every replay.  A fresh model
    from the same initialisation is used, so the timed Adam steps leave the
    benchmarked one untouched."""
    import torch
    from paper_2511_16144_gb300 import lgs
    from paper_2511_16144_gb300.ae import AutoEncoder
    peaks, kind = measured_peaks()
    m = AutoEncoder(enc, dec, device=dev)
    gen = torch.Generator(device=dev).manual_seed(7)
    x = g512_bf[torch.randint(0, g512_bf.shape[0], (65536,), device=dev, generator=gen)].contiguous()
    loss = torch.zeros(1, device=dev)

    def timed_graph(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        ts = []
        for _ in range(reps + 2):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            g.replay()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        del g
        return float(np.mean(ts[2:]))

    out = {}
    ms = timed_graph(lambda: m.train_step(x, lr=1e-4, loss=loss))
    # MACs per pixel: forward and weight gradient of all eight layers
    # (2 x 346,112) and the input gradient of layers 1-7 (346,112 - 512 x 256:
    # the batch itself needs none), 2 FLOP each
    flop = 2 * (2 * 346112 + 346112 - 512 * 256) * x.shape[0]
    out["ae_train_step"] = {
        "pixels": int(x.shape[0]), "ms": ms,
        "roofline": {"bound": "tensor", "achieved": flop / (ms * 1e-3) / 1e12,
                     "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": flop / (ms * 1e-3) / 1e12 / peaks["bf16_tflops"], "traffic": None,
                     "peak_source": kind + " bf16 burst",
                     "note": "25 kernel launches (8 layers forward, 8 weight and bias gradient partials, 7 input gradients, Adam with the fixed-order sum of the partials, BF16 repack)"}}
    z = torch.empty((g512_bf.shape[0], 16), dtype=torch.float32, device=dev)
    ws = m._ws.get("enc")
    ms = timed_graph(lambda: lgs.ae_encode(m.weights, g512_bf, z, ws=ws))
    flop = 2 * 173056 * g512_bf.shape[0]
    out["ae_encode"] = {
        "pixels": int(g512_bf.shape[0]), "ms": ms,
        "roofline": {"bound": "tensor", "achieved": flop / (ms * 1e-3) / 1e12,
                     "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": flop / (ms * 1e-3) / 1e12 / peaks["bf16_tflops"], "traffic": None,
                     "peak_source": kind + " bf16 burst"}}
    del m
    return out


def measure_e2e(steps, graphs, k, warm):
    """End to end through the C ABI with host buffers: every step uploads its
    keyframe's targets (RGB, depth, F_gt) from pinned host memory and reads
    the loss back.  Uploads run on a copy stream into one of two target sets
    while the other set's step computes (keyframe k+1 arrives while the map
    is optimised on keyframe k); all copies stay inside the timed region."""
    import torch
    host = [(st.rgb_t.cpu().pin_memory(), st.depth_t.cpu().pin_memory(),
             st.feat_t.cpu().pin_memory()) for st in steps]
    loss_h = [torch.empty(1, dtype=torch.float32).pin_memory() for _ in steps]
    copy = torch.cuda.Stream()
    comp = torch.cuda.current_stream()
    copied = [torch.cuda.Event() for _ in steps]
    freed = [torch.cuda.Event() for _ in steps]
    for e in freed:
        e.record(comp)

    def run(n):
        for i in range(n):
            j = i % 2
            st = steps[j]
            with torch.cuda.stream(copy):
                copy.wait_event(freed[j])
                st.rgb_t.copy_(host[j][0], non_blocking=True)
                st.depth_t.copy_(host[j][1], non_blocking=True)
                st.feat_t.copy_(host[j][2], non_blocking=True)
                copied[j].record(copy)
            comp.wait_event(copied[j])
            graphs[j].replay()
            loss_h[j].copy_(st.loss, non_blocking=True)
            freed[j].record(comp)

    run(warm)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    copy.wait_event(a)
    run(k)
    copy_done = torch.cuda.Event()
    copy_done.record(copy)
    comp.wait_event(copy_done)
    b.record(comp)
    b.synchronize()
    ms = a.elapsed_time(b) / k
    h2d = sum(t.numel() * t.element_size() for t in host[0])
    return {"value": steps[0].pixels / 1e6 / (ms / 1e3), "unit": "Mpix/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 4,
            "overlap": "targets double-buffered on a copy stream"}


# --------------------------------------------------------------------------- oracle

def oracle_prepare(W):
    """Oracle-side inputs that are not part of a step: the FP64 autoencoder
    at its initial weights and the Gaussians' 16-d encoder prior."""
    from oracle import ae
    from paper_2511_16144_gb300 import synth
    enc, dec = [[[w.astype(np.float64), b.astype(np.float64)] for w, b in L]
                for L in synth.ae_init(seed=3001)]
    sc = W["scene"].with_feats(ae.encode(enc, W["g512"]).astype(np.float32))
    return sc, dec


def centre_crop(cam, px):
    """A centre crop of about px pixels with the frame's aspect ratio."""
    w = max(8, min(cam.width, int(math.sqrt(px * cam.width / cam.height))))
    h = max(8, min(cam.height, int(px // w)))
    return (cam.width // 2 - w // 2, cam.height // 2 - h // 2, w, h)


def crop_f_gt(W, crop):
    """F_gt of a crop: the GPU arm's target map when there is one, else the
    semantic field rendered by the oracle itself (512 channels)."""
    import oracle
    x0, y0, w, h = crop
    if W.get("f_gt") is not None:
        return W["f_gt"][y0:y0 + h, x0:x0 + w].reshape(-1, 512)
    cache = W.setdefault("f_gt_crops", {})
    if crop not in cache:
        o = oracle.render(W["scene"].with_feats(W["g512"]), W["cam"], crop=crop)
        cache[crop] = o["feat"].reshape(-1, 512)
    return cache[crop]


def oracle_step(W, crop, prep):
    """One bounded sample of the workload on the FP64 oracle: a crop rendered
    (RGB, depth, 16-d feature), decoded against F_gt with its gradient, and
    back-propagated to every Gaussian parameter.  Returns (pixels, seconds)."""
    import oracle
    from oracle import ae
    sc, dec = prep
    cam = W["cam"]
    x0, y0, w, h = crop
    f_gt = crop_f_gt(W, crop)
    t0 = time.time()
    o = oracle.render(sc, cam, crop=crop)
    _, g_rgb = oracle.l1_loss_grad(o["rgb"], W["rgb_t"][y0:y0 + h, x0:x0 + w])
    _, g_dep = oracle.l1_loss_grad(o["depth"], W["dep_t"][y0:y0 + h, x0:x0 + w], 0.1)
    _, dz = ae.distill(dec, o["feat"].reshape(-1, 16), f_gt)
    oracle.render_backward(sc, cam, g_rgb, g_dep, dz.reshape(h, w, 16), crop=crop)
    return w * h, time.time() - t0


def size_crop(W, prep, budget_s):
    """Grows a centre crop (x4 pixels a time) until one oracle step takes an
    eighth of budget_s, then scales it to about budget_s (at most the whole
    frame)."""
    cam = W["cam"]
    px = 256
    while True:
        n, dt = oracle_step(W, centre_crop(cam, px), prep)
        if dt >= budget_s / 8 or n >= cam.width * cam.height:
            break
        px *= 4
    return centre_crop(cam, min(cam.width * cam.height, n * budget_s / max(dt, 1e-3)))


def cpu_baseline(W, budget_s=15.0):
    """Times the oracle on one crop sized to about budget_s seconds."""
    import oracle
    oracle.build()
    prep = oracle_prepare(W)
    crop = size_crop(W, prep, budget_s)
    px, dt = oracle_step(W, crop, prep)
    return {"value": px / 1e6 / dt, "unit": "Mpix/s", "cores": oracle.num_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"{crop[2]}x{crop[3]} centre crop of the 640x480 frame, 300k Gaussians: "
                      "FP64 brute-force render + decoder L1 + analytic backward"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    W = build_workload(0)
    W["f_gt"] = None  # rendered by the oracle per crop, outside the timed steps
    prep = oracle_prepare(W)
    crop = size_crop(W, prep, 150.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        oracle_step(W, crop, prep)
    ts = []
    for _ in range(args.steps):
        px, dt = oracle_step(W, crop, prep)
        ts.append(dt)
    ms = 1e3 * float(np.mean(ts))
    value = px / 1e6 / (ms / 1e3)
    sample = f"{crop[2]}x{crop[3]} centre crop of the 640x480 frame per step, FP64 brute force"
    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "gaussians": W["scene"].n, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        # the oracle is plain CPU code; start its thread pool before any GPU work
        run_reference(args, rank, world)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    try:
        run_gpu(args, rank, world)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
