#!/usr/bin/env python
"""Benchmark of the data-parallel brick ray-march + sort-last compositing
path on B300 (one JSON line on stdout).

A step is one pass of the whole hot path over one batch: cull and work list,
brick ray-march, sort-last composite (the forward frame of every camera),
then the adjoint (compositor backward, ray-march replay with TF and volume
gradients) for a fixed upstream image gradient.  The scene (bricks, TF,
cameras, upstream gradient) is resident in HBM before timing; every
workload's volume is larger than L2, so no flush is needed between steps.

The default workload is the largest single-GPU one: a 2048^3 field stored
as bf16, 64 bricks, 8 cameras at 3840x2160.  `value` is the forward sample
rate (samples the ray-march evaluated per second of forward device time);
frames/s and the backward sample rate are reported beside it, and
`ms_per_step` covers the whole step.  `roofline` describes the kernel with
the larger share of the step (`roofline_forward` and `roofline_backward`
describe both).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config large_bf16]
  python bench.py --impl reference      # the FP64 CPU oracle, bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_00179_b300 import build as _build  # noqa: E402
from paper_2407_00179_b300 import inputs  # noqa: E402

METRIC = "Gsamples/s and composited frames/s at 1 B300 (% HBM roofline); backward Gsamples/s"
BYTES_PER_VOXEL = {"f32": 4, "f16": 2, "bf16": 2, "fp8": 1}
# DRAM bytes (read + write) per unit of work of the timed kernels, and their
# L1 / L2 sector hit rates, each from one ncu capture summarised under
# profiles/ (the file is named in "capture").  "source" is the digest of the
# kernel sources (csrc/kernels.cu, csrc/dpv_internal.cuh) the capture ran;
# once those sources change, the figures no longer describe the kernel and
# the line reports traffic null.  Where the bench's workload is too large to
# capture, the capture is of a smaller case of the same kernel (same storage
# and gather layout), and the bytes per evaluated sample scale to the full
# launch by its sample count.
TRAFFIC = {
    # one-pass captures (time, DRAM read, DRAM write) of the bench's own
    # timed steps at full size: 3 steps, 4.7465e10 samples each
    "large_bf16_fwd": {"bytes_per_sample": 14.248, "l1_hit": None, "l2_hit": None,
                       "capture": "profiles/bench_large_bf16_launch_list.md",
                       "case": "2048^3 bf16, 64 bricks, 8 x 3840x2160, quad layout with pair-wide loads, persistent, "
                               "8x32 tiles (the bench's timed steps)",
                       "source": "e4384e70632415e5"},
    "large_bf16_bwd": {"bytes_per_sample": 54.426, "l1_hit": None, "l2_hit": None,
                       "capture": "profiles/bench_large_bf16_launch_list.md",
                       "case": "2048^3 bf16, the same steps; two replay launches per step (face-buffer groups)",
                       "source": "e4384e70632415e5"},
    # mid: the bench's timed steps (3 steps, 3.7027e8 samples each)
    "mid_fwd": {"bytes_per_sample": 14.341, "l1_hit": None, "l2_hit": None,
                "capture": "profiles/bench_mid_launch_list.md",
                "case": "512^3 f32, 8 bricks, 1920x1080, cell layout, persistent, 16x16 tiles (the bench's timed steps)",
                "source": "e4384e70632415e5"},
    "mid_bwd": {"bytes_per_sample": 29.936, "l1_hit": None, "l2_hit": None,
                "capture": "profiles/bench_mid_launch_list.md",
                "case": "512^3 f32, the same steps", "source": "e4384e70632415e5"},
}

# the capture whose per-sample traffic stands for each (workload, kernel)
TRAFFIC_FOR = {
    ("large_bf16", "march"): "large_bf16_fwd",
    ("large_bf16", "march_bwd"): "large_bf16_bwd",
    ("mid", "march"): "mid_fwd",
    ("mid", "march_bwd"): "mid_bwd",
}

# FP32 arithmetic per sample counted in the source (an FMA counts once):
# forward: position 6, trilinear 14, TF lookup 15, opacity 11, emission-
# absorption and termination 8; the adjoint adds the recurrence adjoints,
# the TF-lerp and trilinear-weight gradients and their run sums (about 60).
FP32_OPS_PER_SAMPLE = {"march": 54, "march_bwd": 114}

CONFIGS = {
    # 512^3 f32, 64 blobs + 3-octave noise, 2x2x2 bricks, 1920x1080, ERT 0.99
    "mid": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=1, width=1920, height=1080, ert=0.99,
                storage="f32", cams="direction", compare_storage="f16"),
    # the mid field made opaque (sigma_max 64, termination at 0.99), marched in
    # visibility order with global early termination (forward only), beside
    # the sort-last form with per-fragment termination
    "mid_ordered": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=1, width=1920, height=1080,
                        ert=0.99, sigma_max=64.0, storage="f32", cams="direction", ordered=True),
    # iso-surface fragments of the mid field (forward only: no adjoint)
    "mid_iso": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=1, width=1920, height=1080, ert=0.0,
                    storage="f32", cams="direction", iso=0.5),
    # the mid field under a TF that hides the values below 0.4 (opacity 0),
    # marched with empty-space skipping (macro-cells of 8^3 cells whose value
    # range reaches only transparent TF entries are not sampled), beside the
    # same frame without skipping
    "mid_ess": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=1, width=1920, height=1080, ert=0.99,
                    storage="f32", cams="direction", skip=True, tf_cut=0.4),
    # volumetric shadows by ray forwarding: 256^3 f32, 16 blobs, 2x2x2 bricks,
    # 512^2, a directional light, one shadow ray per sample at 1 voxel
    # (forward only); TF transparent below 0.05
    "shadow": dict(dims=(256, 256, 256), field="diff", splits=(2, 2, 2), ncam=1, width=512, height=512, ert=0.0,
                   storage="f32", cams="direction", shadow=((-0.4, 0.8, 0.45), 1.0, 0.25), tf_cut=0.05),
    "mid_f16": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=1, width=1920, height=1080, ert=0.99,
                    storage="f16", cams="direction"),
    # the 2048^3 workload's kernels on a case small enough for a full ncu
    # capture: 512^3 bf16 (a 2 GB quad layout), 2x2x2 bricks, 2 orbit cameras
    # at 1920x1080, no early termination
    "mid_bf16": dict(dims=(512, 512, 512), field="mid", splits=(2, 2, 2), ncam=2, width=1920, height=1080, ert=0.0,
                     storage="bf16", cams="orbit", compare_f32=False),
    # 64^3 f32, 8 blobs, 2x1x1 bricks, 256x256, no ERT
    "small": dict(dims=(64, 64, 64), field="small", splits=(2, 1, 1), ncam=1, width=256, height=256, ert=0.0,
                  storage="f32", cams="direction"),
    # 1024x1024x512 f16 turbulence, k-d 37 bricks, 16 orbit cameras at 1024^2
    "batched": dict(dims=(1024, 1024, 512), field="turbulent", kd=37, ncam=16, width=1024, height=1024, ert=0.0,
                    storage="f16", cams="orbit", subsample=4),
    # 256^3 f32, 16 blobs, 2x2x2, 32 sphere cameras at 512^2
    "diff": dict(dims=(256, 256, 256), field="diff", splits=(2, 2, 2), ncam=32, width=512, height=512, ert=0.0,
                 storage="f32", cams="sphere"),
    # 2048^3, 4-octave noise + 256 blobs, 4x4x4 bricks, 8 orbit cameras at 3840x2160, bf16 / fp8 storage
    # (the default workload: the largest single-GPU one); the CPU baseline
    # and the parity report take the 1/16 pixel subsample of camera 0; after
    # the timed run, the same batch from fp8 storage and the cameras as
    # separate float32 frames
    "large_bf16": dict(dims=(2048, 2048, 2048), field="large", splits=(4, 4, 4), ncam=8, width=3840, height=2160,
                       ert=0.0, storage="bf16", cams="orbit", compare_f32=False, subsample=4,
                       after_release={"storage": "fp8", "separate_f32": True}),
    "large_fp8": dict(dims=(2048, 2048, 2048), field="large", splits=(4, 4, 4), ncam=8, width=3840, height=2160,
                      ert=0.0, storage="fp8", cams="orbit", compare_f32=False, subsample=4,
                      after_release={"storage": "bf16", "separate_f32": True}),
}


def _field(cfg, device):
    fn = {"mid": inputs.field_mid, "small": inputs.field_small, "turbulent": inputs.field_turbulent,
          "diff": inputs.field_diff, "large": inputs.field_large}[cfg["field"]]
    return fn(0, cfg["dims"], device=device)


def _partition(cfg):
    if cfg.get("kd"):
        return inputs.kd_partition(cfg["dims"], cfg["kd"], seed=0)
    return inputs.regular_partition(cfg["dims"], cfg["splits"])


def _cameras(cfg, rank=0):
    dims = cfg["dims"]
    if cfg["cams"] == "direction":
        return [inputs.camera_from_direction(dims, (1.0, 0.7, 0.5))] * cfg["ncam"]
    if cfg["cams"] == "orbit":
        return inputs.orbit_cameras(dims, cfg["ncam"], seed=rank)
    return inputs.sphere_cameras(dims, cfg["ncam"], seed=rank)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_source_digest() -> str:
    """Digest of the kernel sources a traffic capture describes."""
    import hashlib
    h = hashlib.sha256()
    for name in ("kernels.cu", "dpv_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2407_00179_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(cfg_name, kind, samples):
    """(DRAM bytes of one launch, L1 hit, L2 hit, capture record) of the
    workload's kernel `kind` ("march" or "march_bwd"), from its capture
    scaled by the launch's evaluated samples; Nones where no capture of the
    current kernel source exists."""
    key = TRAFFIC_FOR.get((cfg_name, kind))
    rec = TRAFFIC.get(key) if key else None
    if not rec or rec["source"] != kernel_source_digest():
        return None, None, None, ({"capture": rec["capture"], "stale": True} if rec else None)
    return (rec["bytes_per_sample"] * samples, rec.get("l1_hit"), rec.get("l2_hit"),
            {"capture": rec["capture"], "case": rec["case"], "bytes_per_sample": rec["bytes_per_sample"],
             "scaled_by": "evaluated samples of the launch"})


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(dist, device, times, counts):
    """Whole-job figures of a run on several ranks: the max over ranks of each
    timed interval and the sum over ranks of each work count (ranks render
    different cameras, so their sample counts differ).  With dist None (one
    process) the inputs come back unchanged."""
    if dist is None:
        return list(times), list(counts)
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_bricks(cfg, field_np, part):
    """The oracle's bricks of the workload: its own stored values (the
    oracle's encoders), built once per process."""
    import oracle
    oracle.build()
    return oracle.make_bricks(field_np, part, oracle.DTYPE_NAMES[cfg["storage"]])


def cpu_baseline(cfg_name, cfg, bricks, part, tf, cams, budget_s=12.0, one_core=True):
    """The FP64 oracle as it stands, on this host's cores, on a bounded pixel
    sample of the same workload: pixel rows spread over the image (with
    cfg["subsample"] = s, the rows y % s == 0 and in them the pixels
    x % s == 0: the 1/s^2 subsample of the frame)."""
    import oracle
    oracle.build()
    ncores = len(os.sched_getaffinity(0))
    oracle.set_threads(ncores)
    fr = oracle.Frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"])
    W, H = cfg["width"], cfg["height"]
    sub = int(cfg.get("subsample", 1))
    # the camera and spacing exactly as the C ABI receives them (float32),
    # so the oracle's frame is comparable with the GPU's
    f32 = lambda v: tuple(float(x) for x in np.asarray(v, np.float32))
    c0 = cams[0]
    cam = inputs.Camera(f32(c0.eye), f32(c0.center), f32(c0.up), float(np.float32(c0.fovy_deg)))
    sp = float(np.float32(1.0 / (max(cfg["dims"]) - 1)))

    iso = cfg.get("iso")
    sh = cfg.get("shadow")
    row_ids = np.arange(0, H, sub)                  # the rows the sample may take
    xs = np.arange(0, W, sub, dtype=np.int32)

    def run(rows):
        pix = np.concatenate([xs + W * int(r) for r in rows])
        t = time.perf_counter()
        if sh is not None:
            out = oracle.render_shadow(cfg["dims"], tf, cam, fr, oracle.Light(sh[0], step_voxels=sh[1], ambient=sh[2]),
                                       bricks=bricks, pix=pix, spacing=sp)
            return time.perf_counter() - t, int(out["nsamples"].sum() + out["nshadow"].sum()), len(pix), out, pix
        if iso is not None:
            out = oracle.render_iso(cfg["dims"], tf, cam, fr, iso, bricks=bricks, pix=pix, spacing=sp)
            return time.perf_counter() - t, 0, len(pix), out, pix
        if cfg.get("ordered"):
            out = oracle.render_ordered(cfg["dims"], tf, cam, fr, bricks=bricks, pix=pix, spacing=sp)
            return time.perf_counter() - t, int(out["nsamples"].sum()), len(pix), out, pix
        out = oracle.render_bricks(cfg["dims"], bricks, tf, cam, fr, pix=pix, spacing=sp)
        return time.perf_counter() - t, int(out["nsamples"].sum()), len(pix), out, pix

    def spread(n):
        return row_ids[np.linspace(0, len(row_ids) - 1, max(1, min(n, len(row_ids)))).astype(int)]

    # calibrate on 8 rows spread over the image, then size the sample so the
    # oracle works about budget_s seconds
    cal = spread(8)
    dt, ns, npx, _, _ = run(cal)
    per_row_s = max(dt, 1e-6) / len(cal)
    # a subsample whose every row takes less than half the budget is made
    # denser (half the stride in x and y) so that the sample still takes
    # about budget_s
    while sub > 1 and per_row_s * len(row_ids) < 0.5 * budget_s:
        sub //= 2
        per_row_s *= 2.0                            # twice the pixels per row
        row_ids = np.arange(0, H, sub)
        xs = np.arange(0, W, sub, dtype=np.int32)
    rows = spread(int(max(8, budget_s / per_row_s)))
    dt, ns, npx, ref_out, ref_pix = run(rows)
    ref = {"pix": ref_pix, "rgba": ref_out["rgba"], "flags": ref_out["flags"], "order": ref_out.get("order")}
    what = "pixels x %% %d == 0 of %d of the %d rows y %% %d == 0" % (sub, len(rows), len(row_ids), sub) if sub > 1 \
        else "%d of %d pixel rows" % (len(rows), H)
    one = None
    if one_core:
        # one core on a reduced image: rows spread over the frame, about 3 s
        oracle.set_threads(1)
        rows1 = spread(int(max(2, 3.0 / (per_row_s * ncores))))
        dt1, ns1, npx1, _, _ = run(rows1)
        oracle.set_threads(ncores)
        one = (dt1, ns1, npx1, len(rows1))
    if iso is not None:
        # the iso oracle evaluates every sample of the ray: its rate is in pixels
        return {"value": npx / dt / 1e6, "unit": "Mpixels/s", "cores": ncores, "kind": "oracle",
                "sample": "%s (%d pixels) of camera 0, iso-surface, FP64, %.1f s" % (what, npx, dt),
                "one_core": None if one is None else {
                    "value": one[2] / one[0] / 1e6, "unit": "Mpixels/s", "cores": 1,
                    "sample": "%d pixel rows (%d pixels) of camera 0, %.1f s" % (one[3], one[2], one[0])},
                "seconds": dt, "samples": npx, "rows": rows, "ref": ref}
    return {"value": ns / dt / 1e9, "unit": "Gsamples/s", "cores": ncores, "kind": "oracle",
            "sample": "%s (%d pixels, %d samples) of camera 0, FP64, %.1f s" % (what, npx, ns, dt),
            "one_core": None if one is None else {
                "value": one[1] / one[0] / 1e9, "unit": "Gsamples/s", "cores": 1,
                "sample": "%d pixel rows (%d pixels, %d samples) of camera 0, %.1f s" % (one[3], one[2], one[1],
                                                                                        one[0])},
            "seconds": dt, "samples": ns, "rows": rows, "ref": ref}


def run_reference(args, cfg_name, cfg):
    ws, rank, local = _dist()
    if rank != 0:
        return
    f = _field(cfg, "cuda" if torch.cuda.is_available() else "cpu").cpu().numpy()
    part = _partition(cfg)
    bricks = oracle_bricks(cfg, f, part)
    del f
    tf = inputs.make_tf(1234, transparent_below=cfg.get("tf_cut", 0.0))
    cams = _cameras(cfg)
    steps = []
    base = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(cfg_name, cfg, bricks, part, tf, cams, budget_s=args.ref_budget, one_core=False)
        if i >= args.warmup:
            steps.append(r)
        base = r
    tot_s = sum(r["seconds"] for r in steps)
    tot_n = sum(r["samples"] for r in steps)
    unit = base["unit"]
    val = tot_n / tot_s / (1e6 if unit == "Mpixels/s" else 1e9)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_s / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": cfg_name, "dims": list(cfg["dims"]), "bricks": part.num_ranks,
                       "cameras": cfg["ncam"], "image": [cfg["width"], cfg["height"]], "storage": cfg["storage"],
                       "ert": cfg["ert"]},
            "cpu_baseline": {"value": val, "unit": unit, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def after_release(args, cfg, field_host, part, tf, cams, tune, img0, batch_ms, batch_samples, device):
    """Comparisons for workloads whose main device leaves no room for a
    second one: run after it is released, from the host copy of the field.

    * "storage": the same batch of cameras from another storage format, in
      the main run's launch form: forward rate and image difference (camera
      0) from the main run's frame;
    * "separate_f32": every camera rendered as its own float32-storage frame
      (one device, one camera at a time, its default launch form): their
      summed forward time against the batched reduced-precision forward,
      and camera 0's image difference (the storage error of the batched
      form)."""
    from paper_2407_00179_b300 import dpv
    out = {}
    W, H = cfg["width"], cfg["height"]
    stream = torch.cuda.current_stream(device)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    what = cfg["after_release"]
    fl = tune["flags"] if tune else 0
    if "storage" in what:
        alt = dpv.Device(part.num_ranks, device.index or 0)
        alt.set_geometry(cfg["dims"])
        alt.commit_partition(field_host, part, what["storage"])
        alt.set_tf(tf)
        alt.set_cameras(cams)
        alt.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (0, 0), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT))
        for _ in range(2):
            alt.render()
        torch.cuda.synchronize()
        a0, a1 = ev(), ev()
        n = max(2, min(args.steps, 5))
        a0.record(stream)
        for _ in range(n):
            alt.render()
        a1.record(stream)
        torch.cuda.synchronize()
        ms = a0.elapsed_time(a1) / n
        d = (alt.map_frame(0)[0] - img0).abs()
        out["storage_comparison"] = {
            "storage": what["storage"], "forward_ms_per_step": ms,
            "value": alt.stats()["samples_forward"] / (ms * 1e-3) / 1e9, "unit": "Gsamples/s",
            "launch_form": "the main run's", "image_difference_vs_%s_camera0" % cfg["storage"]: {
                "max": float(d.max()), "mean": float(d.mean())}}
        alt.release()
        del d
        torch.cuda.empty_cache()
    if what.get("separate_f32"):
        sep = dpv.Device(part.num_ranks, device.index or 0)
        sep.set_geometry(cfg["dims"])
        sep.commit_partition(field_host, part, "f32")
        sep.set_tf(tf)
        total, samples, err = 0.0, 0, None
        for c, cam in enumerate(cams):
            sep.set_cameras([cam])
            sep.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"])
            sep.render()
            torch.cuda.synchronize()
            s0, s1 = ev(), ev()
            s0.record(stream)
            for _ in range(2):
                sep.render()
            s1.record(stream)
            torch.cuda.synchronize()
            total += s0.elapsed_time(s1) / 2
            samples += sep.stats()["samples_forward"]
            if c == 0:
                d = (sep.map_frame(0)[0] - img0).abs()
                err = {"max": float(d.max()), "mean": float(d.mean())}
                del d
        sep.release()
        torch.cuda.empty_cache()
        out["separate_f32"] = {
            "what": "each camera its own float32-storage frame, one after another (default launch form)",
            "forward_ms_total": total, "gsamples_per_s": samples / (total * 1e-3) / 1e9,
            "batched_%s_forward_ms" % cfg["storage"]: batch_ms,
            "speedup_of_batched_%s" % cfg["storage"]: total / batch_ms,
            "image_difference_camera0_batched_%s_vs_f32" % cfg["storage"]: err}
    return out


def run_ours(args, cfg_name, cfg):
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2407_00179_b300 import dpv
    _build.build()
    dpv.load()
    device = torch.device("cuda", local)
    field = _field(cfg, device)
    part = _partition(cfg)
    tf_np = inputs.make_tf(1234, transparent_below=cfg.get("tf_cut", 0.0))
    cams = _cameras(cfg, rank)
    W, H = cfg["width"], cfg["height"]
    ncam = len(cams)

    dev = dpv.Device(part.num_ranks, local)
    dev.set_geometry(cfg["dims"])
    dev.commit_partition(field, part, cfg["storage"])
    compare_f32 = cfg.get("compare_f32", True)
    # keep a host copy for the CPU baseline and free the device field
    field_host = field.cpu().numpy() if (rank == 0 and (not args.no_cpu_baseline or cfg.get("after_release"))) \
        else None
    field_dev = field if ((compare_f32 and ncam > 1) or cfg.get("compare_storage")) else None
    del field
    torch.cuda.empty_cache()
    tf = torch.from_numpy(tf_np).to(device)
    dev.set_tf(tf)
    dev.set_cameras(cams)
    iso = cfg.get("iso")
    ordered = bool(cfg.get("ordered"))
    skip = bool(cfg.get("skip"))
    shadow = cfg.get("shadow")
    if shadow is not None:
        dev.set_light(*shadow)
    dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                  tile=(args.tile_w, args.tile_h), iso=iso, ordered=ordered, skip=skip, shadow=shadow is not None)
    tune = None
    if args.gather:
        # a fixed launch form instead of the autotuner's choice, recorded as
        # the choice so that every later frame of the run keeps it
        tune = {"tile": [args.tile_w or 16, args.tile_h or 16],
                "flags": dpv.GATHER_FLAGS[args.gather] | (dpv.FRAME_PERSISTENT if args.persistent else 0),
                "ms": None, "candidates": 0, "cached": False, "fixed": True}
        fl = tune["flags"]
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"], tile=tuple(tune["tile"]),
                      gather=args.gather, persistent=args.persistent, iso=iso, ordered=ordered, skip=skip,
                      shadow=shadow is not None)
    elif not args.no_autotune:
        tune = dev.autotune(frames=3, cache=args.autotune_cache, key=cfg_name)
        fl = tune["flags"]
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"], tile=tuple(tune["tile"]),
                      gather=dpv.gather_of(fl), persistent=bool(fl & dpv.FRAME_PERSISTENT), iso=iso, ordered=ordered,
                      skip=skip, shadow=shadow is not None)
    grad = None
    if iso is None and not ordered and shadow is None:
        # fixed upstream gradient: d/dI of mean (I - I*)^2 with I* from a perturbed TF
        dev.set_tf(torch.from_numpy(inputs.perturb_tf(tf_np, 0)).to(device))
        dev.render()
        target = dev.frames()[0].clone()
        dev.set_tf(tf)
        dev.render()
        grad = (2.0 / target.numel()) * (dev.frames()[0] - target)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(device)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        dev.render()
        if ev:
            ev[1].record(stream)
        if grad is not None:          # iso-surface and ordered frames have no adjoint
            dev.backward(grad, volume_grad=True)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dev.set_profiling(True)
    dev.reset_stats()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")       # lets a profiler capture the timed steps alone
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    st = dev.stats()
    img0 = dev.map_frame(0)[0].clone()           # camera 0 of the timed frame, for the parity report
    dev.set_profiling(False)
    total_ms = t0.elapsed_time(t1)
    fwd_ms = sum(e[0].elapsed_time(e[1]) for e in evs)
    bwd_ms = sum(e[1].elapsed_time(e[2]) for e in evs)
    # samples per step (deterministic); shadowed frames count the shadow
    # samples the forwarding rounds evaluate too
    per_step = st["samples_forward"] + (st["samples_shadow"] if shadow is not None else 0)
    n_fwd = per_step * args.steps
    n_bwd = st["samples_backward"] * args.steps
    launches = st["kernel_launches"]
    frames = ncam * args.steps
    (total_ms, fwd_ms, bwd_ms), (n_fwd, n_bwd, frames) = reduce_over_ranks(
        pg, device, [total_ms, fwd_ms, bwd_ms], [n_fwd, n_bwd, frames])
    # rooflines of the two hot kernels on the stencil-byte model, each from
    # its own device time in the timed region (library CUDA events on the
    # device stream around its launches); `roofline` is the one that takes
    # the larger share of the step
    bpv = BYTES_PER_VOXEL[cfg["storage"]]
    steps = args.steps
    march_ms = st["stage_ms"]["march"] / steps                 # one launch per step
    march_bwd_ms = st["stage_ms"]["march_bwd"] / steps         # one launch per face-buffer group
    face_ms = st["stage_ms"]["face"] / steps
    fwd_bytes = per_step * 8 * bpv
    bwd_bytes = st["samples_backward"] * (8 * bpv + 8 * 4)
    peak, peak_kind = _peaks()

    # compulsory bytes (each stored brick read once + fragment writes), the
    # DRAM traffic ncu measured, hit rates, and an FP32 ALU ceiling from the
    # device's SM count and the sampled maximum SM clock
    brick_bytes = 0
    for k in range(part.num_ranks):
        n_nodes = 1
        for a in range(3):
            lo = max(int(part.lo[k][a]) - 1, 0)
            hi = min(int(part.hi[k][a]), cfg["dims"][a] - 1)
            n_nodes *= hi - lo + 1
        brick_bytes += n_nodes * bpv
    nsm = torch.cuda.get_device_properties(device).multi_processor_count
    tile_px = (tune["tile"][0] * tune["tile"][1]) if tune else (args.tile_w or 16) * (args.tile_h or 16)

    def roofline(kind, ms, samples, nbytes, kernel, model, sm_mhz):
        # fragments written (RGBA + key per slot) by the forward; the adjoint
        # writes the field gradient (4 B per global node)
        out = st["work_items"] * tile_px * 20 if kind == "march" else int(np.prod(cfg["dims"])) * 4
        comp = brick_bytes + out
        traffic, l1, l2, cap = traffic_for(cfg_name, kind, samples)
        alu = (128 * nsm * sm_mhz * 1e6 / FP32_OPS_PER_SAMPLE[kind] / 1e9) if sm_mhz else None
        rate = samples / (ms * 1e-3) / 1e9
        achieved = nbytes / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kernel, "model": model, "peak_kind": peak_kind,
                "ms_per_step": ms, "share_of_step": ms / (total_ms / steps),
                "detail": {"compulsory_bytes": comp, "compulsory_frac": comp / (ms * 1e-3) / 1e9 / peak,
                           "dram_traffic_bytes": traffic,
                           "dram_gbs": traffic / (ms * 1e-3) / 1e9 if traffic else None,
                           "traffic_capture": cap, "l1_hit": l1, "l2_hit": l2,
                           "fp32_ops_per_sample": FP32_OPS_PER_SAMPLE[kind],
                           "alu_ceiling_gsamples": alu, "alu_frac": rate / alu if alu else None,
                           "alu_basis": "128 FP32 lanes x %d SMs x max SM clock / FP32 ops per sample" % nsm}}

    roof_fwd = roofline("march", march_ms, per_step, fwd_bytes,
                        ("k_iso_fwd<%s>" if iso is not None else "k_march_ordered<%s>" if ordered
                         else "k_shadow_round<%s> + k_march_shadowed (march stage)" if shadow is not None
                         else "k_march_fwd<%s>") % cfg["storage"],
                        "stencil bytes: 8 corners x %d B per evaluated sample" % bpv, clk.get("sm_max_mhz"))
    roof_bwd = None
    if grad is not None:
        roof_bwd = roofline("march_bwd", march_bwd_ms, st["samples_backward"], bwd_bytes,
                            "k_march_bwd<%s>" % cfg["storage"],
                            "stencil bytes: 8 corners x %d B read + 8 x 4 B field-gradient adds per replayed "
                            "sample" % bpv, clk.get("sm_max_mhz"))
        roof_bwd["face_buffer_ms_per_step"] = face_ms

    # many cameras: the same forward replayed from a CUDA graph, and the
    # cameras rendered as separate float32 per-camera frames for comparison
    batch = None
    if ncam > 1 and compare_f32:
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"], tile=tuple(tune["tile"]) if tune else
                      (args.tile_w, args.tile_h), gather=dpv.gather_of(tune["flags"]) if tune else "auto", persistent=bool(tune and tune["flags"] & dpv.FRAME_PERSISTENT), graph=True)
        for _ in range(2):
            dev.render()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.steps):
            dev.render()
        g1.record(stream)
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        batched_img = dev.frames()[0].clone()
        graph_used = dev.stats()["graph_launches"]
        sep_ms = 0.0
        err = 0.0
        sep = dpv.Device(part.num_ranks, local)
        sep.set_geometry(cfg["dims"])
        sep.commit_partition(field_dev, part, "f32")
        sep.set_tf(tf)
        for c, cam in enumerate(cams):
            sep.set_cameras([cam])
            sep.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"])
            sep.render()
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(2):
                sep.render()
            s1.record(stream)
            torch.cuda.synchronize()
            sep_ms += s0.elapsed_time(s1) / 2
            err = max(err, float((sep.map_frame(0)[0] - batched_img[c]).abs().max()))
        sep.release()
        batch = {"graph_fwd_ms_per_step": graph_ms, "graph_launches": int(graph_used),
                 "separate_f32_ms": sep_ms, "separate_f32_gsamples_per_s": st["samples_forward"] / (sep_ms * 1e-3) / 1e9,
                 "speedup_vs_separate_f32": sep_ms / graph_ms,
                 "max_abs_diff_vs_separate_f32": err}

    # the same frame from reduced-precision storage at FP32 accumulation:
    # forward rate and image error against the float32-storage frame
    storage_cmp = None
    if cfg.get("compare_storage"):
        cs = cfg["compare_storage"]
        ref_img = dev.frames()[0].clone()
        alt = dpv.Device(part.num_ranks, local)
        alt.set_geometry(cfg["dims"])
        alt.commit_partition(field_dev, part, cs)
        alt.set_tf(tf)
        alt.set_cameras(cams)
        fl = tune["flags"] if tune else 0
        alt.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (args.tile_w, args.tile_h), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT))
        for _ in range(max(3, args.warmup)):
            alt.render()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            alt.render()
        a1.record(stream)
        torch.cuda.synchronize()
        alt_ms = a0.elapsed_time(a1) / args.steps
        diff = (alt.frames()[0] - ref_img).abs()
        storage_cmp = {"storage": cs, "forward_ms_per_step": alt_ms,
                       "value": alt.stats()["samples_forward"] / (alt_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                       "image_error_vs_f32_storage": {"max": float(diff.max()), "mean": float(diff.mean())}}
        alt.release()

    # the ordered march beside the sort-last form (per-fragment termination)
    # of the same frame on the same device: time, samples, image difference
    order_cmp = None
    if ordered:
        ord_img = dev.frames()[0].clone()
        ord_samples = dev.stats()["samples_forward"]
        # the sort-last form in its own best launch form
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=(args.tile_w, args.tile_h))
        sl_tune = None
        if not args.no_autotune:
            sl_tune = dev.autotune(frames=3)
            fl = sl_tune["flags"]
            dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                          tile=tuple(sl_tune["tile"]), gather=dpv.gather_of(fl),
                          persistent=bool(fl & dpv.FRAME_PERSISTENT))
        for _ in range(max(3, args.warmup)):
            dev.render()
        torch.cuda.synchronize()
        o0, o1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        o0.record(stream)
        for _ in range(args.steps):
            dev.render()
        o1.record(stream)
        torch.cuda.synchronize()
        sl_ms = o0.elapsed_time(o1) / args.steps
        sl_samples = dev.stats()["samples_forward"]
        d = (dev.frames()[0] - ord_img).abs()
        order_cmp = {"sort_last_forward_ms_per_step": sl_ms, "sort_last_samples_per_step": sl_samples,
                     "sort_last_autotune": sl_tune,
                     "ordered_samples_per_step": ord_samples, "speedup_vs_sort_last": sl_ms / (fwd_ms / args.steps),
                     "image_difference_vs_sort_last": {"max": float(d.max()), "mean": float(d.mean())}}
        # back to the ordered frame for the end-to-end loop
        fl = tune["flags"] if tune else 0
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (args.tile_w, args.tile_h), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT), ordered=True)

    # empty-space skipping beside the same frame without it, in its own best
    # launch form: time, samples evaluated, and the frames (bit-identical)
    skip_cmp = None
    if skip:
        skip_img = dev.frames()[0].clone()
        skip_samples = dev.stats()["samples_forward"]
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=(args.tile_w, args.tile_h))
        ns_tune = None
        if not args.no_autotune:
            ns_tune = dev.autotune(frames=3)
            nfl = ns_tune["flags"]
            dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                          tile=tuple(ns_tune["tile"]), gather=dpv.gather_of(nfl),
                          persistent=bool(nfl & dpv.FRAME_PERSISTENT))
        for _ in range(max(3, args.warmup)):
            dev.render()
        torch.cuda.synchronize()
        dev.reset_stats()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(args.steps):
            dev.render()
        k1.record(stream)
        torch.cuda.synchronize()
        full_ms = k0.elapsed_time(k1) / args.steps
        full_samples = dev.stats()["samples_forward"]
        skip_cmp = {"no_skip_forward_ms_per_step": full_ms, "no_skip_samples_per_step": full_samples,
                    "no_skip_autotune": ns_tune,
                    "skip_samples_per_step": skip_samples, "evaluated_fraction": skip_samples / max(1, full_samples),
                    "speedup_vs_no_skip": full_ms / (fwd_ms / args.steps),
                    "ray_samples_per_s": full_samples * args.steps / (fwd_ms * 1e-3) / 1e9,
                    "frames_bit_identical": bool(torch.equal(dev.frames()[0], skip_img))}
        # deep fragments: the same skipping, each brick's segment split at
        # its transparent macro-cells into up to DEEP_MAX fragments
        fl = tune["flags"] if tune else 0
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (args.tile_w, args.tile_h), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT), deep=True)
        for _ in range(max(3, args.warmup)):
            dev.render()
        torch.cuda.synchronize()
        k0.record(stream)
        for _ in range(args.steps):
            dev.render()
        k1.record(stream)
        torch.cuda.synchronize()
        d = (dev.frames()[0] - skip_img).abs()
        skip_cmp["deep_fragments"] = {"forward_ms_per_step": k0.elapsed_time(k1) / args.steps,
                                      "max_layers_per_brick": dpv.DEEP_MAX,
                                      "image_difference_vs_skip": {"max": float(d.max()), "mean": float(d.mean())}}
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (args.tile_w, args.tile_h), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT), skip=True)

    # end to end through the public API: TF from pinned host memory in, the
    # composited frames to pinned host memory out, every step
    tf_host = torch.from_numpy(tf_np).pin_memory()
    frame_host = torch.empty((ncam, H, W, 4), dtype=torch.float32).pin_memory()
    for _ in range(2):
        dev.set_tf(tf_host.numpy())
        dev.render()
        dev.copy_frame(0, frame_host[0])
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps)
    if pg:
        pg.barrier()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        dev.set_tf(tf_host.numpy())
        dev.render()
        # every camera's frame to pinned host memory on the copy stream,
        # beside the next step's render
        dev.copy_frame_async(-1, frame_host)
    dev.copy_wait()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    (e2e_s,), (e2e_n,) = reduce_over_ranks(pg, device, [e2e_s], [per_step * e2e_steps])
    e2e_val = e2e_n / e2e_s / 1e9
    value = n_fwd / (fwd_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "Gsamples/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if cfg["storage"] == "f32" else "f32 math, %s storage" % cfg["storage"],
        "data": "synthetic (seeded field, TF, cameras; no paper dataset)",
        "config": {"workload": cfg_name, "dims": list(cfg["dims"]), "bricks": part.num_ranks,
                   "cameras_per_gpu": ncam, "image": [W, H], "storage": cfg["storage"], "ert": cfg["ert"],
                   "step_voxels": 0.5, "sigma_max": cfg.get("sigma_max", 8.0), "mode": (
                       "iso-surface" if iso is not None else "ordered" if ordered else "sort-last") + (
                       ", empty-space skipping" if skip else "") + (
                       ", shadows by ray forwarding" if shadow is not None else ""),
                   "tile": list(tune["tile"]) if tune else [args.tile_w or 16, args.tile_h or 16],
                   "l2": "inputs larger than L2 (%d MiB volume), no flush" % (
                       np.prod(cfg["dims"]) * bpv // 2 ** 20),
                   "parallelism": "weak: each GPU renders its own cameras over its own copy of the bricks"},
        "frames_per_s": frames / (fwd_ms * 1e-3),
        "forward_ms_per_step": fwd_ms / args.steps,
        "backward": ({"value": n_bwd / (bwd_ms * 1e-3) / 1e9, "unit": "Gsamples/s",
                      "ms_per_step": bwd_ms / args.steps} if grad is not None else None),
        "mpixels_per_s": frames * W * H / (fwd_ms * 1e-3) / 1e6,
        "samples_per_step": {"forward": n_fwd / args.steps, "backward": n_bwd / args.steps},
        "stage_ms_per_step": {k: v / max(1, args.steps) for k, v in st["stage_ms"].items()},
        "value_basis": ("forward samples evaluated / forward time (cull + march + composite) of the timed steps; "
                        "each step also runs the backward, reported under 'backward' and in ms_per_step"
                        if grad is not None else
                        "samples evaluated up to each brick's first hit / forward time (cull + iso march + depth "
                        "composite); iso-surface frames have no adjoint, a step is the forward frame"
                        if iso is not None else
                        "primary + shadow samples evaluated / forward time (cull, shadow-ray spawn, %d forwarding "
                        "rounds, shading march, composite); shadowed frames have no adjoint, a step is the forward "
                        "frame" % part.num_ranks
                        if shadow is not None else
                        "samples evaluated up to the global termination / forward time (cull + ordered march); "
                        "ordered frames have no adjoint, a step is the forward frame"),
        "roofline": (roof_bwd if roof_bwd is not None and march_bwd_ms > march_ms else roof_fwd),
        "roofline_forward": roof_fwd,
        "roofline_backward": roof_bwd,
        "e2e": {"value": e2e_val, "unit": "Gsamples/s", "h2d_bytes_per_step": int(tf_np.nbytes),
                "d2h_bytes_per_step": int(ncam * H * W * 16), "what": "set TF from pinned host, render, copy frames"
                " to pinned host (asynchronous, overlapping the next render; all copies complete inside the "
                "timed region), per step (forward)"},
        "gpu_launches": int(launches),
        "clocks": clk,
        "error_flags": st["error_flags"],
        "autotune": tune,
    }
    if batch:
        line["batched"] = batch
    if storage_cmp:
        line["storage_comparison"] = storage_cmp
    if order_cmp:
        line["sort_last_comparison"] = order_cmp
    if shadow is not None:
        line["shadow"] = {"light_direction": list(shadow[0]), "shadow_step_voxels": shadow[1], "ambient": shadow[2],
                          "primary_samples_per_step": st["samples_forward"],
                          "shadow_samples_per_step": st["samples_shadow"],
                          "wave_front_rounds": part.num_ranks}
        line["config"]["tf_transparent_below"] = cfg["tf_cut"]
    if skip_cmp:
        line["skip_comparison"] = skip_cmp
        line["config"]["tf_transparent_below"] = cfg["tf_cut"]
    # the per-pixel order of camera 0 (sort-last modes), for the parity report
    order0 = None
    if rank == 0 and not args.no_cpu_baseline and iso is None and not ordered and shadow is None:
        fl = tune["flags"] if tune else 0
        dev.set_frame(W, H, step_voxels=0.5, sigma_max=cfg.get("sigma_max", 8.0), ert=cfg["ert"],
                      tile=tuple(tune["tile"]) if tune else (args.tile_w, args.tile_h), gather=dpv.gather_of(fl),
                      persistent=bool(fl & dpv.FRAME_PERSISTENT), skip=skip, order=True)
        dev.render()
        order0 = dev.order(0).reshape(-1, part.num_ranks).cpu().numpy()
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cb = cpu_baseline(cfg_name, cfg, oracle_bricks(cfg, field_host, part), part, tf_np, cams,
                              budget_s=args.ref_budget)
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "one_core")}
        except Exception as e:  # the oracle is a reported baseline, never the product
            cb = None
            line["cpu_baseline"] = {"value": None, "unit": "Gsamples/s", "cores": None, "kind": "oracle",
                                    "sample": "failed: %s" % e}
        if cb is not None:
            # the timed frame against the oracle's frame of the same rows
            ref = cb["ref"]
            img = img0.reshape(-1, 4).double().cpu().numpy()[ref["pix"]]
            ok = (ref["flags"].astype(np.int64) & ~1) == 0     # every ambiguity flag excluded
            err = np.abs(img - ref["rgba"])[ok]
            par = {"reference": "FP64 oracle, same stored values, camera 0, the cpu_baseline rows",
                   "pixels": int(ok.sum()), "flagged": int((~ok).sum()),
                   "max_abs": float(err.max()) if err.size else None,
                   "mean_abs": float(err.mean()) if err.size else None,
                   "max_abs_per_channel": err.max(axis=0).tolist() if err.size else None}
            if order0 is not None and ref["order"] is not None:
                o = order0[ref["pix"]]
                par["order_mismatches"] = int((o[ok] != ref["order"][ok]).any(axis=1).sum())
            line["parity"] = par
    dev.release()
    del grad
    torch.cuda.empty_cache()
    if rank == 0 and cfg.get("after_release") and field_host is not None:
        line.update(after_release(args, cfg, field_host, part, tf, cams, tune, img0, fwd_ms / steps, per_step,
                                  device))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large_bf16", choices=sorted(CONFIGS))
    ap.add_argument("--tile-w", type=int, default=0)
    ap.add_argument("--tile-h", type=int, default=0)
    ap.add_argument("--ref-budget", type=float, default=12.0, help="seconds of oracle work per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--gather", default=None, choices=["cell", "quad", "linear"],
                    help="fixed gather layout (with --tile-w/--tile-h, --persistent) instead of the autotuner's choice")
    ap.add_argument("--persistent", action="store_true", help="with --gather: the persistent launch form")
    ap.add_argument("--autotune-cache", default=None,
                    help="JSON file: reuse the stored launch choice for this workload and GPU, else tune and store it")
    args = ap.parse_args()
    cfg = CONFIGS[args.config]
    if args.impl == "reference":
        if args.steps * args.ref_budget > 240:
            args.ref_budget = max(2.0, 240.0 / max(1, args.steps + args.warmup))
        run_reference(args, args.config, cfg)
    else:
        run_ours(args, args.config, cfg)


if __name__ == "__main__":
    main()
