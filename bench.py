"""Benchmark of the ISAAC volume ray caster on one B300 (or N replicas).

Workload (default ``pic512``): E and B (3-component) and a density (scalar)
on 512^3 interior cells + 4 guard cells per side, float32, AoS, the
PIConGPU-shaped chains, LUTs, weights and clip plane of the multi-source
configuration, rendered at 1920x1080 with step 0.5 voxel from 32 cameras on a
Fibonacci sphere at twice the box diagonal.  One step = one frame (the whole
plain path: ray setup, sampling, chains, classification, blend, compositing,
quantisation) for the next camera.

Reports ray samples/s (device-timed, CUDA events on the render stream, L2
flushed between steps), frames/s, an end-to-end figure through the C ABI with
host-side inputs and the image read back, the roofline of the ray-cast kernel,
and the FP64 CPU oracle as the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray samples/s & fps at 1080p/512^3; learned+lowprec vs plain at ≤1 LSB; p99 ms"
L2_FLUSH_BYTES = 256 << 20


def reduce_over_ranks(values, op, device):
    """Max or sum of ``values`` over the ranks of the default process group
    (the values themselves without one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workload

def make_workload(name):
    from paper_1611_09048_b300 import synth
    if name == "pic512":
        n, W, H = 512, 1920, 1080
    elif name == "pic256":
        n, W, H = 256, 1920, 1080
    elif name == "blobs64":
        sc = synth.scene_blobs(64, 256, 256, seed=0)
        cams = [synth.random_orbit_camera((64,) * 3, 256, 256, seed=1000 + i) for i in range(32)]
        return sc, cams, {"workload": "blobs64_256x256", "n": 64, "guard": 0,
                          "sources": "blobs(1)", "width": 256, "height": 256}
    else:
        raise ValueError(name)
    sc = synth.scene_pic(n=n, guard=4, width=W, height=H, seed=0)
    cams = synth.fibonacci_cameras((n, n, n), W, H, count=32, seed=0)
    cfg = {"workload": f"pic{n}_fp32_{W}x{H}", "n": n, "guard": 4,
           "sources": "E(3) B(3) rho(1), float32 AoS, zero-copy", "width": W, "height": H,
           "step": sc.step, "interp": "trilinear", "term_alpha": sc.term, "clip_planes": 1,
           "cameras": len(cams), "camera_distance": "2x box diagonal, Fibonacci sphere"}
    return sc, cams, cfg


def bytes_per_cell(scene):
    return sum(4 * s.fdim for i, s in enumerate(scene.sources) if (scene.mask >> i) & 1)


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1611_09048_b300 import isaac

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sc, cams, cfg = make_workload(args.workload)
    ds = isaac.DeviceScene(sc, device=dev)
    stream = torch.cuda.Stream(device=dev)
    W, H = sc.width, sc.height
    fb = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)

    # untimed pre-pass per camera: composited samples and the cells read
    samples, touched_cells, ray_stats = [], [], []
    ns = torch.empty((H, W), dtype=torch.int32, device=dev)
    bits = torch.zeros(ds.footprint_words(), dtype=torch.int32, device=dev)
    with torch.cuda.stream(stream):
        for mv, proj in cams:
            bits.zero_()
            ds.render(mv, proj, out=fb, nsamples=ns, touched=bits, stream=stream)
            samples.append(int(ns.sum(dtype=torch.int64).item()))
            hit = ns[ns > 0].float()
            ray_stats.append((int(hit.numel()), float(hit.max().item()) if hit.numel() else 0.0))
            popc = torch.bitwise_and(bits.view(torch.int32).unsqueeze(-1),
                                     torch.tensor([1 << i for i in range(31)] + [-(1 << 31)],
                                                  dtype=torch.int32, device=dev)) != 0
            touched_cells.append(int(popc.sum().item()))
    del bits
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    prepared = [ds.prepare(mv, proj, out=fb) for mv, proj in cams]

    def frame(i):
        ds.launch(prepared[i % len(cams)], stream)

    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            frame(i)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # events the library records around the march kernel of each timed frame
    mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in mev:
        a.record(stream)
        b.record(stream)
    # The clock sampler (200 ms period) runs over a window that starts with
    # >= 1 s of further untimed frames (GPU under the same load) and ends
    # after the timed steps, so short timed regions still get clock samples.
    with ClockSampler(local_rank) as clocks:
        t_pre = time.perf_counter()
        i = 0
        while time.perf_counter() - t_pre < args.preroll:
            with torch.cuda.stream(stream):
                for _ in range(8):
                    frame(i)
                    i += 1
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t_wall0 = time.perf_counter()
        torch.cuda.nvtx.range_push("timed")
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()                      # evict L2 between timed frames
                isaac.time_march(*mev[i])
                ev[i][0].record(stream)
                frame(args.warmup + i)
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        isaac.time_march()
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall0
        if world > 1:
            torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    march_ms = [a.elapsed_time(b) for a, b in mev]
    dev_ms = sum(step_ms)
    timed_idx = [(args.warmup + i) % len(cams) for i in range(args.steps)]
    n_samp = sum(samples[j] for j in timed_idx)
    cells = [touched_cells[j] for j in timed_idx]

    # End to end through the C ABI: every step uploads the LUTs from pinned
    # host memory, renders, and reads the RGBA8 image back into pinned host
    # memory.  Two framebuffers, two LUT buffers and two render streams used
    # in turn: step i's read-back runs on a copy stream while step i+1
    # renders, step i's LUT upload runs on an upload stream while step i-1
    # renders (an upload on the render stream waited behind the copy engine's
    # read-back: 0.392 against 0.363 ms per step), and step i+1's frame, on the
    # other render stream (its own workspace), starts while step i's march
    # drains (0.363 -> 0.330 ms per step).  A framebuffer is rendered into
    # again only after its read-back has finished, a LUT buffer is overwritten
    # only after the frame that read it has finished.
    luts_host = torch.from_numpy(np.ascontiguousarray(sc.luts, np.float32)).pin_memory()
    fbs = [fb, torch.empty_like(fb)]
    lut_bufs = [torch.empty_like(ds.luts) for _ in range(2)]
    preps = [[ds.prepare(mv, proj, out=fbs[b], luts=lut_bufs[b]) for mv, proj in cams] for b in range(2)]
    imgs = [torch.empty((H, W, 4), dtype=torch.uint8).pin_memory() for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    upload_stream = torch.cuda.Stream(device=dev)
    render_streams = [stream, torch.cuda.Stream(device=dev)]
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    uploaded = [torch.cuda.Event() for _ in range(2)]
    def pipeline(steps, first):
        """`steps` frames through the pipeline, cameras from `first` on;
        returns the device time from its start to the last image read back."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        upload_stream.wait_event(e0)
        render_streams[1].wait_event(e0)
        for i in range(steps):
            b = i % 2
            rs = render_streams[b]
            if i >= 2:
                upload_stream.wait_event(rendered[b])
            with torch.cuda.stream(upload_stream):
                lut_bufs[b].copy_(luts_host, non_blocking=True)
            uploaded[b].record(upload_stream)
            rs.wait_event(uploaded[b])
            if i >= 2:
                rs.wait_event(copied[b])
            with torch.cuda.stream(rs):
                ds.launch(preps[b][(first + i) % len(cams)], rs)
            rendered[b].record(rs)
            copy_stream.wait_event(rendered[b])
            with torch.cuda.stream(copy_stream):
                imgs[b].copy_(fbs[b], non_blocking=True)
            copied[b].record(copy_stream)
        for b in range(min(2, steps)):
            stream.wait_event(copied[b])
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    pipeline(args.warmup, 0)                 # untimed: the streams' and buffers' first use
    e2e_ms = pipeline(args.steps, args.warmup)

    variants = {} if args.no_variants else \
        run_variants(args, ds, cams, prepared, samples, stream, flush, fb)
    iso = None if args.no_variants else run_iso(args, ds, cams, stream, flush)
    comp = None if args.no_variants else run_composite(args, dev, stream, flush)
    copy = None if args.no_variants else run_source_copy(args, ds, stream, flush)
    closeup = None if args.no_variants else run_closeup(args, ds, stream, flush)
    learned = None if args.no_learned or rank != 0 else run_learned(args, dev, stream, flush)
    serving = None if args.no_serving or rank != 0 else run_serving(args, ds, dev)

    # times: max over ranks; samples: sum over ranks (whole-job throughput)
    dev_ms, e2e_ms, t_wall = reduce_over_ranks([dev_ms, e2e_ms, t_wall], "max", dev)
    (all_samp,) = reduce_over_ranks([float(n_samp)], "sum", dev)
    if rank != 0:
        return None

    hbm_peak, peak_kind = _peaks()
    bpc = bytes_per_cell(sc)
    alg_bytes = [c * bpc + W * H * 4 for c in cells]
    mean_launch_ms = statistics.mean(march_ms)
    achieved = (sum(alg_bytes) / args.steps) / (mean_launch_ms * 1e-3) / 1e9
    prof, traffic_source = _ncu_traffic(cfg["workload"])
    prof = prof or {}
    traffic = prof.get("dram_bytes_per_launch")
    l2_peak = _l2_peak(dev)
    lts = prof.get("lts_bytes_per_launch")
    res = {
        "metric": METRIC,
        "value": all_samp / (dev_ms * 1e-3),
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dev_ms / args.steps,
        "ms_per_step_median": statistics.median(step_ms),
        "ms_per_step_min": min(step_ms),
        "fps": world * args.steps / (dev_ms * 1e-3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded plane-wave E/B fields + log-normal density, PIConGPU-shaped)",
        "config": dict(cfg, parallelism=f"replicas{world}",
                       l2="flushed between timed steps (256 MiB write, untimed)",
                       samples_per_frame_mean=n_samp / args.steps,
                       hit_rays_per_frame_mean=sum(ray_stats[j][0] for j in timed_idx) / args.steps,
                       samples_per_ray_max=max(ray_stats[j][1] for j in timed_idx),
                       cells_read_per_frame_mean=sum(cells) / len(cells)),
        "wall_s_timed_region": t_wall,
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                     "traffic": traffic,
                     "traffic_source": traffic_source,
                     "kernel": "k_raycast (march), CUDA events recorded by the library around "
                               "its launch on the render stream",
                     "launch_ms_mean": mean_launch_ms,
                     "frame_share": sum(march_ms) / dev_ms,
                     "algorithmic_bytes": "distinct cells read x 28 B (E,B,rho) + W*H*4 B image",
                     "binding_unit": prof.get("binding_unit"),
                     # the same launch against the L2 (the copy of roofline_l2 below, kept
                     # inside this object so that readers of the roofline see both)
                     "l2_achieved": (lts / (mean_launch_ms * 1e-3) / 1e9) if lts else None,
                     "l2_peak": l2_peak,
                     "l2_frac": (lts / (mean_launch_ms * 1e-3) / 1e9 / l2_peak) if lts else None,
                     "l2_bytes": "ncu lts__t_bytes per launch (" + traffic_source + ")",
                     "l2_peak_kind": "measured here: isaac_probe_read over half the L2, best of 10"},
        "roofline_l2": {"achieved": (lts / (mean_launch_ms * 1e-3) / 1e9) if lts else None,
                        "peak": l2_peak, "unit": "GB/s",
                        "frac": (lts / (mean_launch_ms * 1e-3) / 1e9 / l2_peak) if lts else None,
                        "bytes": "ncu lts__t_bytes per k_raycast launch (" + traffic_source + ")",
                        "time": "mean march launch of this run (CUDA events)",
                        "peak_kind": "measured here: isaac_probe_read over half the L2, best of 10"},
        "e2e": {"value": all_samp / (e2e_ms * 1e-3), "unit": "samples/s",
                "h2d_bytes_per_step": int(luts_host.numel() * 4),
                "d2h_bytes_per_step": int(W * H * 4),
                "overlap": "step i's image read-back (copy stream) overlaps step i+1's frame, "
                           "step i's LUT upload (upload stream) overlaps step i-1's frame, "
                           "consecutive frames on two render streams overlap where one's march "
                           "drains; two framebuffers and two LUT buffers, pinned host memory"},
        "clocks": clocks.summary(),
        "variants": variants,
        "iso": iso,
        "composite": comp,
        "source_copy": copy,
        "closeup": closeup,
        "learned": learned,
        "serving": serving,
    }
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(sc, cams, args.cpu_seconds)
    return res


def run_variants(args, ds, cams, prepared_f32, samples, stream, flush, fb_f32):
    """Packed copies (FP32, BF16, FP16, E4M3) of the same sources: pack time,
    samples/s over the same cameras, and the difference to the FP32 zero-copy
    frame over the image's hit pixels: 8-bit (mean and max LSB, share of
    pixels over 1 LSB) and before quantisation (max per channel, mean)."""
    import torch
    out = {}
    W, H = ds.scene.width, ds.scene.height
    n_cam = len(cams)
    steps = min(args.steps, 4 * n_cam)
    ref_imgs = []
    with torch.cuda.stream(stream):
        for j in range(n_cam):
            ds.launch(prepared_f32[j], stream)
            ref_imgs.append(fb_f32.clone())
    torch.cuda.synchronize()
    read_bytes = sum(t.numel() * t.element_size() for t in ds.data)   # the sources, read once
    for fmt in ("f32", "bf16", "f16", "e4m3"):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pv = ds.pack(fmt, stream=stream)      # allocates the copy (untimed)
        torch.cuda.synchronize()
        flush.zero_()
        e0.record(stream)
        pv.repack(stream=stream)              # the per-time-step conversion
        e1.record(stream)
        torch.cuda.synchronize()
        pack_ms = e0.elapsed_time(e1)
        fb = torch.empty_like(fb_f32)
        prep = [pv.prepare(mv, proj, out=fb) for mv, proj in cams]
        lsb_sum, lsb_max, npx, over1, nhit = 0.0, 0, 0, 0, 0
        abs_max = torch.zeros(4, dtype=torch.float32, device=fb.device)
        abs_sum = 0.0
        ref32 = torch.empty((H, W, 4), dtype=torch.float32, device=fb.device)
        var32 = torch.empty_like(ref32)
        tmp8 = torch.empty_like(fb_f32)
        with torch.cuda.stream(stream):
            for j in range(n_cam):
                pv.launch(prep[j], stream)
                d = (fb.to(torch.int16) - ref_imgs[j].to(torch.int16)).abs()
                hit = ref_imgs[j][..., 3] > 0
                lsb_sum += float(d[hit].float().sum().item())
                lsb_max = max(lsb_max, int(d.max().item()))
                npx += int(hit.sum().item()) * 4
                over1 += int((d.amax(-1)[hit] > 1).sum().item())
                nhit += int(hit.sum().item())
                # before quantisation: the packed frame against the FP32 zero-copy frame
                mv, proj = cams[j]
                ds.render(mv, proj, out=tmp8, rgba32=ref32, stream=stream)
                pv.render(mv, proj, out=tmp8, rgba32=var32, stream=stream)
                e = (var32 - ref32).abs()
                abs_max = torch.maximum(abs_max, e.reshape(-1, 4).amax(0))
                abs_sum += float(e[hit].sum().item())
            for i in range(args.warmup):
                pv.launch(prep[i % n_cam], stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.nvtx.range_push(f"timed_{fmt}")
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                pv.launch(prep[(args.warmup + i) % n_cam], stream)
                ev[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        ns = sum(samples[(args.warmup + i) % n_cam] for i in range(steps))
        out[fmt] = {"samples_per_s": ns / (ms * 1e-3), "ms_per_frame": ms / steps,
                    "pack_ms": pack_ms,
                    "pack_gb_per_s": (read_bytes + pv.data.numel()) / (pack_ms * 1e-3) / 1e9,
                    "bytes": int(pv.data.numel()) +
                    (int(pv.scales.numel()) * 4 if pv.scales is not None else 0),
                    "lsb_vs_f32_mean": lsb_sum / max(1, npx), "lsb_vs_f32_max": lsb_max,
                    "hit_px_over_1lsb_frac": over1 / max(1, nhit),
                    "abs_vs_f32_max_rgba": [float(v) for v in abs_max.tolist()],
                    "abs_vs_f32_mean": abs_sum / max(1, npx),
                    "steps": steps}
        del pv, prep
        torch.cuda.empty_cache()
    return out


def run_iso(args, ds, cams, stream, flush):
    """Iso-surface frames (isaac_render_iso) over the same cameras: E and B
    lengths and the density at seeded thresholds of their normalised chain
    outputs; time per frame, samples evaluated per second, pixels hit."""
    import torch
    iso = [0.6, 0.6, 0.55]
    W, H = ds.scene.width, ds.scene.height
    fb = torch.empty((H, W, 4), dtype=torch.uint8, device=ds.device)
    ns = torch.empty((H, W), dtype=torch.int32, device=ds.device)
    samples, hits = 0, 0
    with torch.cuda.stream(stream):
        for mv, proj in cams:
            ds.render_iso(iso, mv, proj, out=fb, stream=stream, want_nsamp=False)
    torch.cuda.synchronize()
    prep = [ds.prepare_iso(iso, mv, proj, out=fb, nsamples=ns) for mv, proj in cams]
    with torch.cuda.stream(stream):
        for j in range(len(cams)):
            ds.launch_iso(prep[j], stream)
            samples += int(ns.sum(dtype=torch.int64).item())
            hits += int((fb[..., 3] == 255).sum().item())
    prep = [ds.prepare_iso(iso, mv, proj, out=fb) for mv, proj in cams]
    steps = min(args.steps, 2 * len(cams))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        torch.cuda.nvtx.range_push("timed_iso")
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            ds.launch_iso(prep[i % len(cams)], stream)
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    per_frame = samples / len(cams)
    return {"iso": iso, "ms_per_frame": ms, "fps": 1e3 / ms,
            "samples_per_frame": per_frame, "samples_per_s": per_frame / (ms * 1e-3),
            "hit_pixels_per_frame": hits / len(cams), "steps": steps}


def run_composite(args, dev, stream, flush, n_layers=8, W=1920, H=1080):
    """Sort-last compositing (isaac_composite) of n_layers 1080p partial images
    (premultiplied RGBA32 + depth, seeded): time per composite and its bytes
    (n_layers * 20 B read + 20 B written per pixel) against the HBM peak."""
    import torch
    from paper_1611_09048_b300 import isaac
    g = torch.Generator(device=dev).manual_seed(11)
    layers = []
    for _ in range(n_layers):
        a = torch.rand((H, W, 1), device=dev, generator=g) * 0.5
        c = torch.cat([torch.rand((H, W, 3), device=dev, generator=g) * a, a], -1).contiguous()
        d = torch.rand((H, W), device=dev, generator=g) * 1000.0
        layers.append((c, d))
    out8 = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
    out32 = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    for _ in range(3):
        isaac.composite(layers, out=out8, rgba32=out32, stream=stream)
    steps = max(8, min(args.steps, 32))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            isaac.composite(layers, out=out8, rgba32=out32, stream=stream)
            b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    nbytes = W * H * (n_layers * 20 + 20)
    peak, kind = _peaks()
    return {"layers": n_layers, "width": W, "height": H, "ms": ms,
            "gb_per_s": nbytes / (ms * 1e-3) / 1e9, "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peak,
            "peak_kind": kind, "bytes_per_pixel": n_layers * 20 + 20}


def run_source_copy(args, ds, stream, flush):
    """Non-persistent sources (isaac_copy_source): copy every source of the
    workload through its accessor (interior + one guard layer) into a buffer
    of its own; time one copy of all sources and its bytes (4 B read + 4 B
    written per copied element) against the HBM peak."""
    import torch
    from paper_1611_09048_b300 import isaac
    n = ds.scene.n
    srcs = [isaac.Source.from_buffer_copy(ds.sources[s]) for s in range(len(ds.scene.sources))]
    bufs = [torch.empty(isaac.copy_bytes(n, d.f_dim, d.guard) // 4, dtype=torch.float32,
                        device=ds.device) for d in srcs]

    def copy_all():
        for d, b in zip(srcs, bufs):
            isaac.copy_source(d, n, b, stream)
    for _ in range(3):
        copy_all()
    steps = max(4, min(args.steps, 16))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            copy_all()
            b.record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    nbytes = 2 * sum(b.numel() * 4 for b in bufs)
    peak, kind = _peaks()
    del bufs
    return {"sources": len(srcs), "copied_bytes": nbytes // 2, "ms": ms,
            "gb_per_s": nbytes / (ms * 1e-3) / 1e9, "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / peak,
            "peak_kind": kind, "launches": len(srcs)}


def run_closeup(args, ds, stream, flush, count=4, dist=0.9):
    """Stress row: the same volume from cameras at 0.9x the box diagonal, so
    that the box fills the frame (every ray hits, long chords): per-frame
    time and composited samples/s, L2 flushed between frames."""
    import torch
    from paper_1611_09048_b300 import isaac, synth
    sc = ds.scene
    W, H = sc.width, sc.height
    cams = synth.fibonacci_cameras(tuple(sc.n), W, H, count=count, seed=7, dist_factor=dist)
    out = torch.empty((H, W, 4), dtype=torch.uint8, device=ds.device)
    out_staged = torch.empty((H, W, 4), dtype=torch.uint8, device=ds.device)
    ns = torch.empty((H, W), dtype=torch.int32, device=ds.device)
    samples, rays, same = 0, 0, True
    ms = {False: [], True: []}
    for mv, proj in cams:
        with torch.cuda.stream(stream):
            ds.render(mv, proj, out=out, nsamples=ns, stream=stream)
            ds.render(mv, proj, out=out_staged, stream=stream, staged=True)
        torch.cuda.synchronize()
        samples += int(ns.sum(dtype=torch.int64).item())
        rays += int((ns > 0).sum().item())
        same &= bool(torch.equal(out, out_staged))
        # the default gather march, then the staged march (ISAAC_MARCH_STAGED)
        for staged in (False, True):
            prep = ds.prepare(mv, proj, out, staged=staged)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            with torch.cuda.stream(stream):
                ds.launch(prep, stream)
                for a, b in ev:
                    flush.zero_()
                    a.record(stream)
                    ds.launch(prep, stream)
                    b.record(stream)
            torch.cuda.synchronize()
            ms[staged] += [a.elapsed_time(b) for a, b in ev]
    per_frame, staged_frame = statistics.mean(ms[False]), statistics.mean(ms[True])
    return {"cameras": count, "camera_distance": f"{dist}x box diagonal",
            "ms_per_frame": per_frame, "samples_per_frame": samples / count,
            "hit_rays_per_frame": rays / count,
            "samples_per_s": (samples / count) / (per_frame * 1e-3),
            "staged_ms_per_frame": staged_frame, "staged_speedup": per_frame / staged_frame,
            "staged_bitwise_equal": same,
            "staged_note": "ISAAC_MARCH_STAGED: one thread per ray, per-warp shared-memory boxes of the "
                           "field (opt-in; the default is the gather march)"}


def run_learned(args, dev, stream, flush):
    """Bubble workload (512^3 scalar: an ellipsoidal shell moving through
    mostly empty space, 1920x1080): train the interval proposal on traced
    frames (random cameras and transfer functions), then time plain and
    learned marching in float32 zero-copy and BF16 packed form on unseen
    frames; the learned forms include the per-frame max-opacity grid."""
    import torch
    from paper_1611_09048_b300 import isaac, synth
    n, W, H, cell = args.learned_n, 1920, 1080, 16
    t_begin = time.perf_counter()
    noise = synth.value_noise(n, 77, device=dev)
    Xs, Rs = [], []
    for fi, f in enumerate(range(0, 100, 10)):
        field = synth.bubble_field(n, f, 0, noise=noise, device=dev)
        for c in range(args.learned_views):
            sc = synth.scene_bubble(n, frame=f, seed=1000 * fi + c, width=480, height=270,
                                    field=field, lut_seed=500 + (7 * fi + c) % 16)
            ds = isaac.DeviceScene(sc, device=dev)
            rays, count, *_ = ds.trace()
            k = int(count.item())
            if k == 0:
                continue
            grid = ds.opacity_grid(cell)
            Xs.append(isaac.mlp_features(rays[:k], k, sc.n, sc.step, grid, cell))
            Rs.append(rays[:k].clone())
    X, R = torch.cat(Xs), torch.cat(Rs)
    t_data = time.perf_counter() - t_begin
    model = isaac.MLPModel(isaac.pack_mlp_params(synth.mlp_params(3)), device=dev)
    gen = torch.Generator(device="cpu").manual_seed(0)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    t1 = time.perf_counter()
    for it in range(args.learned_steps):
        idx = torch.randint(0, X.shape[0], (8192,), generator=gen).to(dev)
        if it == args.learned_steps - 1:
            loss.zero_()
        model.train_step(X[idx].contiguous(), R[idx].contiguous(), lr=1e-3, margin=2,
                         loss_sum=loss if it == args.learned_steps - 1 else None)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1

    kinds = ("plain_f32", "skip_f32", "learned_f32", "plain_bf16", "learned_bf16",
             "learned_bf16_nowiden", "gridhull_f32", "gridhull_bf16")
    acc = {k: {"ms": [], "march_ms": [], "samples": 0, "lsb_sum": 0.0, "lsb_max": 0, "px": 0,
               "px_over1": 0, "hit_px": 0} for k in kinds}
    grid_ms, grid16_ms, range_ms, conv_ms = [], [], [], []
    stats = torch.zeros(2, dtype=torch.int32, device=dev)
    stats_off = torch.zeros(2, dtype=torch.int32, device=dev)
    # the test protocol: consecutive frames of the moving bubble (100 by
    # default), one unseen camera and transfer function each
    for f in range(args.learned_frames):
        field = synth.bubble_field(n, f, 0, noise=noise, device=dev)
        sc = synth.scene_bubble(n, frame=f, seed=77000 + f, width=W, height=H,
                                field=field, lut_seed=500 + (3 * f) % 16)
        ds = isaac.DeviceScene(sc, device=dev)
        pv = ds.pack("bf16")
        grid = torch.empty(tuple((k + cell - 1) // cell for k in sc.n[::-1]),
                           dtype=torch.float32, device=dev)
        prop = model.proposal(grid, cell, threshold=args.learned_threshold,
                              margin=args.learned_margin, stats=stats)
        prop_off = model.proposal(grid, cell, threshold=args.learned_threshold,
                                  margin=args.learned_margin, stats=stats_off, widen=False)
        # the grid's part of the learned frame without the network: every ray
        # keeps the hull of its samples in nonzero macro cells
        prop_hull = isaac.grid_proposal(grid, cell)
        ranges = ds.range_grid(cell)
        outs = {k: torch.empty((H, W, 4), dtype=torch.uint8, device=dev) for k in kinds}
        nss = {}

        def run(kind, count=None):
            if kind.endswith("bf16") or kind.endswith("nowiden"):
                # every frame is a new simulation step: its BF16 copy is made per frame
                pv.repack(stream=stream)
            if kind in ("learned_f32", "gridhull_f32"):
                ds.opacity_grid(cell, out=grid, stream=stream)
            if kind.startswith("learned_bf16") or kind == "gridhull_bf16":   # the copy's grid
                pv.opacity_grid(cell, out=grid, stream=stream)
            if kind.startswith("skip"):
                ds.range_grid(cell, out=ranges, stream=stream)
            tgt = ds if kind.endswith("f32") else pv
            kw = dict(out=outs[kind], stream=stream)
            if kind.startswith("gridhull"):
                return tgt.render_learned(prop_hull, want_nsamp=count is not None, **kw)
            if kind.startswith("learned"):
                return tgt.render_learned(prop_off if kind.endswith("nowiden") else prop,
                                          want_nsamp=count is not None, **kw)
            if kind.startswith("skip"):
                return ds.render_skip(ranges, cell, want_nsamp=count is not None, **kw)
            return tgt.render(want_nsamp=count is not None, **kw)

        with torch.cuda.stream(stream):
            for kind in kinds:           # counting pass (untimed)
                nss[kind] = run(kind, count=True)[2]
        torch.cuda.synchronize()
        ref = outs["plain_f32"]
        hit = ref[..., 3] > 0
        for kind in kinds:
            d = (outs[kind].to(torch.int16) - ref.to(torch.int16)).abs()
            dm = d.amax(-1)
            a = acc[kind]
            a["lsb_sum"] += float(d.float().sum().item())
            a["px"] += d.numel()
            a["lsb_max"] = max(a["lsb_max"], int(dm.max().item()))
            a["px_over1"] += int((dm > 1).sum().item())
            a["hit_px"] += int(hit.sum().item())
            a["samples"] += int(nss[kind].sum(dtype=torch.int64).item())
        ev = {k: [torch.cuda.Event(enable_timing=True) for _ in range(4)] for k in kinds}
        with torch.cuda.stream(stream):
            for kind in kinds:           # the library records the march events on launch
                ev[kind][2].record(stream)
                ev[kind][3].record(stream)
            for kind in kinds:
                run(kind)                # warm
                a, b, ma, mb = ev[kind]
                flush.zero_()
                isaac.time_march(ma, mb)
                if f == 0:
                    torch.cuda.nvtx.range_push(f"timed_{kind}")
                a.record(stream)
                run(kind)
                b.record(stream)
                isaac.time_march()       # the next kind's warm frame is not timed
                if f == 0:
                    torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        isaac.time_march()
        for kind in kinds:
            a, b, ma, mb = ev[kind]
            acc[kind]["ms"].append(a.elapsed_time(b))
            acc[kind]["march_ms"].append(ma.elapsed_time(mb))
        if f % 10 == 0:   # the per-frame grids alone (part of the learned / skip frames above)
            for fn, sink in ((lambda: ds.opacity_grid(cell, out=grid, stream=stream), grid_ms),
                             (lambda: pv.opacity_grid(cell, out=grid, stream=stream), grid16_ms),
                             (lambda: ds.range_grid(cell, out=ranges, stream=stream), range_ms),
                             (lambda: pv.repack(stream=stream), conv_ms)):
                gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(3)]
                with torch.cuda.stream(stream):
                    fn()
                    for a, b in gev:
                        flush.zero_()
                        a.record(stream)
                        fn()
                        b.record(stream)
                torch.cuda.synchronize()
                sink += [a.elapsed_time(b) for a, b in gev]
        del ds, pv
    frames = len(acc["plain_f32"]["ms"])
    seen, restricted = stats.tolist()
    res = {"workload": f"bubble{n}_{W}x{H}", "train_rays": int(X.shape[0]),
           "train_steps": args.learned_steps, "train_s": t_train, "data_s": t_data,
           "final_loss": float(loss.item()), "threshold": args.learned_threshold,
           "margin": args.learned_margin, "restricted_frac": restricted / max(1, seen),
           "test_frames": frames,
           "test_protocol": "frames 0..N-1 of the moving bubble, one unseen camera and LUT each; "
                            "one timed frame per kind per frame, L2 flushed before it",
           "opacity_grid_ms": statistics.mean(grid_ms),
           "opacity_grid_bf16_ms": statistics.mean(grid16_ms),
           "range_grid_ms": statistics.mean(range_ms),
           "bf16_conversion_ms": statistics.mean(conv_ms),
           # the field read once, the copy's records over [-1, n]^3 written once
           "bf16_conversion_gb_per_s": (n ** 3 * 4 + (n + 2) ** 3 * 2)
           / (statistics.mean(conv_ms) * 1e-3) / 1e9}
    for kind in kinds:
        a = acc[kind]
        ms = statistics.mean(a["ms"])
        res[kind] = {"ms_per_frame": ms, "fps": 1e3 / ms,
                     "ms_per_frame_median": statistics.median(a["ms"]),
                     "march_ms": statistics.mean(a["march_ms"]),
                     "samples_per_frame": a["samples"] / frames,
                     "lsb_vs_plain_f32_mean": a["lsb_sum"] / max(1, a["px"]),
                     "lsb_vs_plain_f32_max": a["lsb_max"],
                     "hit_px_over_1lsb_frac": a["px_over1"] / max(1, a["hit_px"])}
    res["speedup_learned_bf16_vs_plain_f32"] = res["plain_f32"]["ms_per_frame"] / \
        res["learned_bf16"]["ms_per_frame"]
    res["speedup_skip_f32_vs_plain_f32"] = res["plain_f32"]["ms_per_frame"] / \
        res["skip_f32"]["ms_per_frame"]
    res["speedup_learned_bf16_vs_skip_f32"] = res["skip_f32"]["ms_per_frame"] / \
        res["learned_bf16"]["ms_per_frame"]
    res["speedup_gridhull_bf16_vs_plain_f32"] = res["plain_f32"]["ms_per_frame"] / \
        res["gridhull_bf16"]["ms_per_frame"]
    res["note"] = ("every frame is a new simulation step: the *_bf16 frames include the "
                   "per-frame BF16 conversion of the float32 field (isaac_pack, "
                   "bf16_conversion_ms alone); "
                   "learned_* include the per-frame max-opacity grid (learned_bf16* computes it "
                   "from its BF16 copy), skip_f32 the per-frame "
                   "value-range grid (the field changes every frame); skip_f32 is exact "
                   "(bit-identical to plain_f32), learned_* within the stated LSB; "
                   "learned_bf16_nowiden: the same proposal without widening by the grid; "
                   "gridhull_*: the widening alone, without a network (each ray keeps the "
                   "hull of its samples in macro cells with a nonzero max-opacity grid value)")
    return res


def run_serving(args, ds, dev):
    """Serving loop over the resident 512^3 E/B/rho volume in BF16: clients
    with Poisson arrivals (open loop), image sizes drawn from {256^2, 512^2,
    1280x720, 1920x1080}, cameras on seeded random walks, a share of requests
    steering (new LUTs or functor parameters that the client then keeps).
    Reports latency percentiles (submit -> image in pinned host memory),
    frames/s and the batch sizes the server formed; then a closed-loop burst
    for the saturated throughput."""
    import torch
    from paper_1611_09048_b300 import isaac, synth
    sc = ds.scene
    pv = ds.pack("bf16")
    torch.cuda.synchronize()
    rng = np.random.default_rng(2024)
    sizes = [(256, 256), (512, 512), (1280, 720), (1920, 1080)]
    n_cl = args.serve_clients
    state = [{"theta": rng.uniform(0, 2 * math.pi), "phi": rng.uniform(-0.5, 0.5),
              "luts": None, "chains": None} for _ in range(n_cl)]
    base_chains = [list(c) for c in sc.chains]
    # pinned output buffers, recycled (a request holds one until its result)
    n_buf = args.serve_buffers
    bufs = [torch.empty(1920 * 1080 * 4, dtype=torch.uint8).pin_memory() for _ in range(n_buf)]
    free = list(range(n_buf))

    def schedule(rate, dur):
        n = int(rate * dur)
        return {"rate": rate, "n": n, "t": np.cumsum(rng.exponential(1.0 / rate, n)),
                "who": rng.integers(0, n_cl, n), "size": rng.integers(0, len(sizes), n),
                "steer": rng.uniform(0, 1, n) < args.serve_steer}

    def make(sch, i):
        c = state[sch["who"][i]]
        c["theta"] += math.radians(rng.normal(0, 2.0))
        c["phi"] = float(np.clip(c["phi"] + math.radians(rng.normal(0, 2.0)), -1.2, 1.2))
        if sch["steer"][i]:
            if rng.uniform() < 0.5:
                c["luts"] = np.stack([synth.lut_from_points(int(rng.integers(1 << 30)))
                                      for _ in range(pv.luts.shape[0])])
            else:
                ch = [list(x) for x in base_chains]
                f = float(rng.uniform(0.7, 1.3))
                ch[0] = [(op[0], tuple(a * f for a in op[1])) if op[0] == "mul" else op
                         for op in ch[0]]
                c["chains"] = ch
        W, H = sizes[sch["size"][i]]
        mv, proj = synth.orbit_camera(sc.n, W, H, c["theta"], c["phi"], dist_factor=2.0)
        return mv, proj, W, H, c["luts"], c["chains"]

    def run_open(srv, sch):
        res, stalls, t0 = [], 0, time.perf_counter()
        held = {}
        i, n, t_arr = 0, sch["n"], sch["t"]
        while i < n or held:
            now = time.perf_counter() - t0
            if i < n and now >= t_arr[i]:
                if not free:
                    stalls += 1
                    for r in srv.poll(wait=0.001):
                        free.append(held.pop(r["tag"]))
                        res.append(r)
                    continue
                mv, proj, W, H, luts, chains = make(sch, i)
                b = free.pop()
                out = bufs[b][: W * H * 4]
                held[srv.submit(mv, proj, W, H, out, luts=luts, chains=chains)] = b
                i += 1
                continue
            wait = max(0.0, (t_arr[i] - now) if i < n else 0.002)
            for r in srv.poll(wait=min(wait, 0.002)):
                free.append(held.pop(r["tag"]))
                res.append(r)
        assert all(r["status"] == 0 for r in res)
        lat = np.array([r["t_done"] - r["t_submit"] for r in res]) * 1e3
        qwait = np.array([r["t_launch"] - r["t_submit"] for r in res]) * 1e3
        span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
        px = sum(sizes[k][0] * sizes[k][1] for k in sch["size"])
        bs = np.array([r["batch_size"] for r in res])
        sizes_seen, counts = np.unique(bs, return_counts=True)
        return {"offered_rate_per_s": sch["rate"], "requests": n,
                "requests_by_batch_size": {int(k): int(v) for k, v in zip(sizes_seen, counts)},
                "device_overlap": overlap_stats(res),
                "latency_ms": {"p50": float(np.percentile(lat, 50)),
                               "p90": float(np.percentile(lat, 90)),
                               "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                               "mean": float(lat.mean())},
                "queue_ms": {"p50": float(np.percentile(qwait, 50)),
                             "p99": float(np.percentile(qwait, 99))},
                "fps": n / span, "mpix_per_s": px / span / 1e6,
                "batch_size": {"mean": float(bs.mean()), "max": int(bs.max())},
                "generator_stalls": stalls}

    with isaac.Server(pv, budget=args.serve_budget << 20, n_streams=args.serve_streams,
                      max_batch=args.serve_max_batch) as srv:
        # warm-up: a few requests of every size
        for k in range(8):
            mv, proj = synth.orbit_camera(sc.n, *sizes[k % 4], 0.1 * k, 0.1)
            srv.submit(mv, proj, *sizes[k % 4], bufs[k][: sizes[k % 4][0] * sizes[k % 4][1] * 4])
        srv.drain()
        main = run_open(srv, schedule(args.serve_rate, args.serve_seconds))
        stress = run_open(srv, schedule(args.serve_stress_rate, args.serve_stress_seconds)) \
            if args.serve_stress_seconds > 0 else None
        # offered far beyond what the GPU serves: the queue stays long, batches fill up
        overload = run_open(srv, schedule(args.serve_overload_rate, args.serve_overload_seconds)) \
            if args.serve_overload_seconds > 0 else None
        # closed loop: keep every buffer in flight, 1080p only
        burst = []
        held = {}
        t0 = time.perf_counter()
        n_burst = args.serve_burst
        sent = 0
        while sent < n_burst or held:
            while free and sent < n_burst:
                mv, proj = synth.orbit_camera(sc.n, 1920, 1080, 0.37 * sent, 0.2 * math.sin(sent))
                b = free.pop()
                held[srv.submit(mv, proj, 1920, 1080, bufs[b])] = b
                sent += 1
            for r in srv.poll(wait=0.01):
                free.append(held.pop(r["tag"]))
                burst.append(r)
        t_burst = time.perf_counter() - t0
    assert all(r["status"] == 0 for r in burst)
    res = {
        "workload": "serve_pic512_bf16",
        "clients": n_cl, "sizes": [f"{w}x{h}" for w, h in sizes],
        "steering_share": args.serve_steer, "budget_mib": args.serve_budget,
        "streams": args.serve_streams, "max_batch": args.serve_max_batch,
        "saturated_1080p_fps": len(burst) / t_burst,
        "latency_note": "submit -> RGBA8 image in pinned host memory, measured by the server's own "
                        "clock; includes queueing, the batch's kernels and its device-to-host copy",
    }
    res.update(main)
    res["stress"] = stress
    res["overload"] = overload
    return res


def overlap_stats(results):
    """From the device-clock intervals of the requests' batches: the time the
    GPU held at least one request, the share of it with two or more requests
    in flight (in one batch or in batches overlapping on several streams),
    and the share with two or more batches overlapping."""
    batches = {}
    for r in results:
        if r.get("t_gpu_start", -1.0) < 0:
            continue
        key = (r["stream"], r["t_gpu_start"], r["t_gpu_end"])
        batches[key] = r["batch_size"]
    ev = []
    for (_, a, b), n in batches.items():
        ev += [(a, n, 1), (b, -n, -1)]
    ev.sort(key=lambda e: (e[0], e[1]))
    busy = ge2_req = ge2_batch = 0.0
    inflight = nb = 0
    for i, (t, dn, db) in enumerate(ev):
        if i:
            dt = t - ev[i - 1][0]
            if inflight >= 1:
                busy += dt
            if inflight >= 2:
                ge2_req += dt
            if nb >= 2:
                ge2_batch += dt
        inflight += dn
        nb += db
    return {"busy_s": busy, "share_two_or_more_requests": ge2_req / busy if busy else 0.0,
            "share_two_or_more_batches": ge2_batch / busy if busy else 0.0,
            "batches": len(batches)}


def _l2_peak(dev):
    """L2 read bandwidth: isaac_probe_read (16-byte loads cached in L2 only)
    over a buffer of half the L2, resident after the first pass; best of 10
    runs of 20 passes, CUDA events."""
    import torch
    from paper_1611_09048_b300 import isaac
    n = torch.cuda.get_device_properties(dev).L2_cache_size // 2
    buf = torch.ones(n // 4, dtype=torch.float32, device=dev)
    sink = torch.zeros(1024, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    isaac.probe_read(buf, 3, sink, stream)
    best = float("inf")
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        isaac.probe_read(buf, 20, sink, stream)
        b.record(stream)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return 20 * buf.numel() * 4 / (best * 1e-3) / 1e9


# Source files that define the plain march kernel: a traffic figure taken by
# ncu applies to the build it was captured from only.
MARCH_SOURCES = ("paper_1611_09048_b300/csrc/raycast.cuh", "paper_1611_09048_b300/csrc/raycast_kernels.cu",
                 "paper_1611_09048_b300/csrc/ff.cuh")


def march_source_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in MARCH_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _ncu_traffic(workload):
    """Per-launch ncu counters of the march kernel from the committed capture
    summary (profiles/traffic.json), when it was taken from the march sources
    of this build; else None with the reason."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None, "no ncu capture summary"
    with open(path) as f:
        d = json.load(f).get(workload)
    if d is None:
        return None, "no ncu capture of this workload"
    if d.get("kernel_source_sha256") != march_source_sha256():
        return None, "stale: the march kernel's sources changed since the ncu capture"
    return d, "ncu capture, profiles/traffic.json: " + d.get("command", "")


# ------------------------------------------------------------ CPU oracle arm

def cpu_baseline(sc, cams, budget_s):
    """The FP64 oracle, as it stands, on the host cores: whole frames of the
    same workload, camera after camera, until ``budget_s`` seconds of work."""
    import oracle
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    total, frames = 0, 0
    for mv, proj in cams:
        r = oracle.render(sc.with_camera(mv, proj), threads=threads)
        total += int(r["nsamp"].sum())
        frames += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    # one thread, on the centre rows of the first camera (a bounded sample)
    H, W = sc.height, sc.width
    rows = max(1, H // 16)
    pix = (np.arange(rows)[:, None] + (H - rows) // 2) * W + np.arange(W)[None, :]
    t1 = time.perf_counter()
    r1 = oracle.render(sc.with_camera(*cams[0]), pixels=pix.reshape(-1), threads=1)
    dt1 = time.perf_counter() - t1
    n1 = int(r1["nsamp"].sum())
    return {"value": total / dt, "unit": "samples/s", "cores": threads, "kind": "oracle",
            "sample": f"{frames} full {sc.width}x{sc.height} frame(s) of the same workload "
                      f"({total} samples, {dt:.1f} s)",
            "single_thread": {"value": n1 / dt1, "unit": "samples/s",
                              "sample": f"the centre {rows} rows of camera 0 ({n1} samples, "
                                        f"{dt1:.1f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    sc, cams, cfg = make_workload(args.workload)
    threads = oracle.max_threads()
    # each step: a bounded sample of one frame -- the centre rows of the image
    rows = max(1, int(sc.height * args.ref_rows))
    y0 = (sc.height - rows) // 2
    pix = np.arange(y0 * sc.width, (y0 + rows) * sc.width, dtype=np.int64)

    def step(i):
        mv, proj = cams[i % len(cams)]
        r = oracle.render(sc.with_camera(mv, proj), pixels=pix, threads=threads)
        return int(r["nsamp"].sum())

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    total = sum(step(args.warmup + i) for i in range(args.steps))
    dt = time.perf_counter() - t0
    v = total / dt
    sample = (f"{rows} centre rows x {sc.width} px of each frame ({len(pix)} rays), "
              f"one camera per step, {total} samples")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "samples/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, parallelism="cpu"),
            "cpu_baseline": {"value": v, "unit": "samples/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pic512", choices=["pic512", "pic256", "blobs64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-rows", type=float, default=0.25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the packed-copy variants (FP32/BF16/FP16/E4M3)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-proposal comparison on the bubble workload")
    ap.add_argument("--learned-n", type=int, default=512)
    ap.add_argument("--learned-views", type=int, default=14)
    ap.add_argument("--learned-frames", type=int, default=100,
                    help="test frames of the moving bubble (one camera each)")
    ap.add_argument("--learned-steps", type=int, default=1500)
    ap.add_argument("--learned-threshold", type=float, default=0.9)
    ap.add_argument("--learned-margin", type=int, default=4)
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-loop measurement")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rate", type=float, default=600.0)
    ap.add_argument("--serve-clients", type=int, default=48)
    ap.add_argument("--serve-steer", type=float, default=0.1)
    ap.add_argument("--serve-budget", type=int, default=256, help="MiB")
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-max-batch", type=int, default=16)
    ap.add_argument("--serve-buffers", type=int, default=64)
    ap.add_argument("--serve-stress-rate", type=float, default=3000.0,
                    help="second open-loop point, above what one request at a time sustains")
    ap.add_argument("--serve-stress-seconds", type=float, default=4.0)
    ap.add_argument("--serve-overload-rate", type=float, default=20000.0,
                    help="a third open-loop point far beyond capacity (full batches)")
    ap.add_argument("--serve-overload-seconds", type=float, default=1.0)
    ap.add_argument("--serve-burst", type=int, default=400)
    ap.add_argument("--preroll", type=float, default=1.0,
                    help="seconds of untimed frames inside the clock-sampling window")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
        res = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
