#!/usr/bin/env python
"""Throughput of the adaptive box-spline filter on GB300.

One step = one pass of the whole path over one image: the non-adaptive step
(abf_integrate: row scan + look-back line scans) and the adaptive step
(abf_filter: per-pixel mesh), exact form, inputs resident in HBM.

Workload (default): 2048x2048 float32 image on the 2^-16 grid (smooth field +
edges), order n = 2, per-pixel ellipse fields (sigma in [1, 24], elongation in
[1, 6], orientation uniform) mapped to the four steps by the moment rule,
Q = 8.  Synthetic, seeded.

Multi-GPU: images are independent, so N ranks run N replicas (each its own
image, no collective on the data path); value = pixels of all ranks / max time.

--impl reference: the exact CPU oracle as it stands, timed on this host on a
bounded sample of the same workload (per-pixel evaluation).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixel/s adaptive filter, chosen vs FP64 form at stated error; p50/p99 latency"
UNIT = "Mpixel/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while the
    timed region runs (entering waits for the first sample, so sampling is
    under way before the region starts)."""

    def __init__(self, index=0, interval_ms=50):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.first = threading.Event()

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=5.0)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _workload(name, rank, shape=None):
    import synthetic
    return synthetic.workload(name, shape=shape, seed_offset=rank)


WORKLOAD_TEXT = {
    "c1": "f64 integers 0..255, order n=1, paper scales a_k in [1,8], Q=8",
    "c2": "f32 (2^-16 grid), order n=2, per-pixel ellipse (sigma 1-24, elongation 1-6), Q=8",
    "c3": "u16, order n=3, paper scales a_k in [1,48], Q=8",
}


def _shape(args):
    if not args.shape:
        return None
    h, w = args.shape.lower().split("x")
    return int(h), int(w)


MESH_DRAM_BYTES = 158931200 + 27586816
# DRAM bytes (read + write) of the four integrate passes (row scan + v2, v3, v4
# line scans) on the same workload, from one ncu capture of the current kernels
INTEG_DRAM_BYTES = 630252544


def _algorithmic_macs(n):
    """Non-zero ZP^{*n} stencil MACs per pixel: (n+1)^4 taps x 7 n^2 (the area
    of the support octagon of ZP^{*n}, i.e. its average count of non-zero
    lattice weights)."""
    return (n + 1) ** 4 * 7 * n * n


def _host_tensor(img):
    """numpy image -> CPU tensor (uint16 through an int16 view: numpy has no torch bridge for it)."""
    import torch
    if img.dtype == np.uint16:
        return torch.from_numpy(img.view(np.int16).copy()).view(torch.uint16)
    return torch.from_numpy(np.ascontiguousarray(img))


def e2e_pipelined(filt, f_h, s_h, H, W, K, stream):
    """K steps through the public API with every step's H2D copy of its
    inputs and D2H copy of its result inside the timed region, the copies on
    their own streams so that they overlap the neighbouring steps' kernels.
    Returns the elapsed milliseconds (CUDA events, rank-local)."""
    import torch
    dev = stream.device
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    f_d = [torch.empty(f_h.shape, dtype=f_h.dtype, device=dev) for _ in range(2)]
    s_d = [torch.empty(s_h.shape, dtype=s_h.dtype, device=dev) for _ in range(2)]
    o_d = [torch.empty((H, W), dtype=torch.float64, device=dev) for _ in range(2)]
    o_h = [torch.empty((H, W), dtype=torch.float64).pin_memory() for _ in range(2)]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_free = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(k):
        b = k & 1
        with torch.cuda.stream(h2d):
            if k >= 2:
                h2d.wait_event(ev_free[b])   # step k-2 no longer reads these buffers
            f_d[b].copy_(f_h, non_blocking=True)
            s_d[b].copy_(s_h, non_blocking=True)
            ev_in[b].record(h2d)

    torch.cuda.synchronize()
    e0.record(stream)
    h2d.wait_stream(stream)
    upload(0)
    for k in range(K):
        b = k & 1
        stream.wait_event(ev_in[b])
        filt.integrate(f_d[b])
        if k >= 2:
            stream.wait_event(ev_down[b])    # step k-2's result has left o_d[b]
        filt.filter(s_d[b], o_d[b])
        ev_out[b].record(stream)
        ev_free[b].record(stream)
        if k + 1 < K:
            upload(k + 1)
        with torch.cuda.stream(d2h):
            d2h.wait_event(ev_out[b])
            o_h[b].copy_(o_d[b], non_blocking=True)
            ev_down[b].record(d2h)
    stream.wait_stream(d2h)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def max_over_ranks(ms, world, device):
    """The slowest rank's time (every rank gets it); the identity at world 1."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(pixels_per_rank, steps, world, total_ms):
    """Whole-job Mpixel/s of N replicas: all ranks' pixels over the slowest rank's time."""
    return pixels_per_rank * steps * world / (total_ms * 1e-3) / 1e6


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_0908_3861_gb300 import AdaptiveFilter, AbfError, ellipse_product_bound
    import __graft_entry__

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    w = _workload(args.workload, rank, _shape(args))
    img, sc = w["image"], w["scales"]
    H, W = img.shape
    n = w["n"]
    f_t = _host_tensor(img).to(dev)
    s_t = torch.from_numpy(sc.astype(np.float32)).to(dev)
    # the plan's scale-product bound comes from the workload's parameter range
    # (sigma <= 24, elongation <= 6), not from this image's field
    max_prod = (ellipse_product_bound(w["sigma_max"], w["e_max"], n, w["q_bits"], w["cmax"], device=dev)
                if w["scale_kind"] == "ellipse" else 0.0)
    tin = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64,
           np.dtype(np.uint8): torch.uint8, np.dtype(np.uint16): torch.uint16}[img.dtype]
    # binary64 output: the forms are compared at 1e-12 of the value range
    filt = AdaptiveFilter(W, H, n, tin, scale_kind=w["scale_kind"], q_bits=w["q_bits"], frac_bits=w["frac_bits"],
                          max_scale=w["cmax"], out="f64", value_bound=w["value_bound"],
                          max_scale_product=max_prod, device=dev)
    out = torch.empty((H, W), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        filt.integrate(f_t)
        filt.filter(s_t, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tuned_rows, tuned_ms = filt.autotune(s_t, out)
    torch.cuda.synchronize()
    assert filt.device_status() == 0

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(K):
            ev[i][0].record(stream)
            filt.integrate(f_t)
            ev[i][1].record(stream)
            filt.filter(s_t, out)
            ev[i][2].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    integ_ms = sum(a.elapsed_time(b) for a, b, c in ev) / K
    mesh_ms = sum(b.elapsed_time(c) for a, b, c in ev) / K
    assert filt.device_status() == 0

    # End to end through the public API with host buffers (pinned), H2D + D2H inside.
    f_h = _host_tensor(img).pin_memory()
    s_h = torch.from_numpy(sc.astype(np.float32)).pin_memory()
    o_h = torch.empty((H, W), dtype=torch.float64).pin_memory()
    f_d = torch.empty_like(f_t)
    s_d = torch.empty_like(s_t)
    for _ in range(max(1, args.warmup // 2)):
        f_d.copy_(f_h, non_blocking=True)
        s_d.copy_(s_h, non_blocking=True)
        filt.integrate(f_d)
        filt.filter(s_d, out)
        o_h.copy_(out, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        f_d.copy_(f_h, non_blocking=True)
        s_d.copy_(s_h, non_blocking=True)
        filt.integrate(f_d)
        filt.filter(s_d, out)
        o_h.copy_(out, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_serial_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    # The same, pipelined as a user would: step k+1's inputs go up on a copy
    # stream while step k computes, step k's result comes down on another
    # while step k+1 computes (two device buffers for inputs and outputs).
    e2e_ms = max_over_ranks(e2e_pipelined(filt, f_h, s_h, H, W, K, stream), world, dev)

    out_exact = out.clone()
    forms = {"exact": {"value": None, "ms_per_step": round(total_ms / K, 4), "numerator": "bit-exact vs the oracle"}}
    for form in args.compare:
        try:
            ff = AdaptiveFilter(W, H, n, tin, scale_kind=w["scale_kind"], q_bits=w["q_bits"],
                                frac_bits=w["frac_bits"], max_scale=w["cmax"], out="f64", form=form,
                                value_bound=w["value_bound"], device=dev)
        except AbfError as e:
            forms[form] = {"value": None, "unsupported": "plan refused (%s): the form's error bound cannot meet "
                                                         "its tolerance at order %d" % (e, n)}
            continue
        o2 = torch.empty_like(out)
        for _ in range(args.warmup):
            ff(f_t, s_t, o2)
        torch.cuda.synchronize()
        a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            ff(f_t, s_t, o2)
        c.record(stream)
        torch.cuda.synchronize()
        st2 = ff.device_status()
        ms2 = a.elapsed_time(c) / K
        o2h = o2.cpu().numpy()
        forms[form] = {"value": round(H * W / (ms2 * 1e-3) / 1e6, 3), "ms_per_step": round(ms2, 4),
                       "device_status": st2, "flagged_pixels": int((~np.isfinite(o2h)).sum()),
                       "tolerance": "1e-12" if form == "plain_f64" else "1e-5", "out": o2h}
        ff.close()

    pix = float(H * W)
    value = replica_throughput(pix, K, world, total_ms)
    forms["exact"]["value"] = round(value, 3)
    forms["exact"]["out"] = out_exact.cpu().numpy()
    e2e_value = replica_throughput(pix, K, world, e2e_ms)
    peaks = _peaks()
    L = filt.limbs
    macs = _algorithmic_macs(n) * pix
    # peak (derived): 152 SMs x 64 INT32 multiply-add lanes / clock x SM clock,
    # divided by the 32-bit multiply-adds one MAC needs (the partial products of
    # a 2L-word g and a k-word weight that land below bit 64 L, low and high
    # halves counted separately).
    wwords = {1: 1, 2: 2, 3: 4}[n]
    imad_per_mac = (sum(1 for i in range(2 * L) for j in range(wwords) if i + j <= 2 * L - 1)
                    + sum(1 for i in range(2 * L) for j in range(wwords) if i + j <= 2 * L - 2))
    clk = clk.summary()
    sm_mhz = clk["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    peak_macs = 152 * 64 * sm_mhz * 1e6 / imad_per_mac
    # the probes behind the derived peak, measured now (ops/s -> per clock per SM at the sampled clock)
    probe = {}
    try:
        from paper_0908_3861_gb300 import _abf as _A
        with ClockSampler(local) as pclk:
            imad_s = _A.abf_probe_alu(0)
            mac_s = _A.abf_probe_alu(1)
        pmhz = pclk.summary()["sm_mhz"] or sm_mhz
        probe = {"imad_per_clk_per_sm": round(imad_s / (152 * pmhz * 1e6), 2),
                 "mac2x64_per_clk_per_sm": round(mac_s / (152 * pmhz * 1e6), 3),
                 "sm_mhz": pmhz, "source": "abf_probe_alu (independent chains, every SM)"}
    except Exception as e:  # the probe is context for the peak, not part of the step
        probe = {"error": str(e)[:120]}
    achieved = macs / (mesh_ms * 1e-3)
    hl = filt.info["halo_lrbt"]
    gw, gh = W + hl[0] + hl[1], H + hl[3]
    integ_bytes = float(img.nbytes) + 7.0 * gw * gh * 8 * L
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(total_ms / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64x%d" % L, "data": "synthetic",
        "config": {"workload": "%dx%d %s, exact form (%d-limb wrap-around integers)" % (
                       H, W, WORKLOAD_TEXT[args.workload], L),
                   "image": [H, W], "order_n": n, "form": "exact", "limbs": L,
                   "l2": "inputs larger than L2 (integrated image %.0f MB + scales %.0f MB)" % (
                       filt.info["integrated_bytes"] / 1e6, H * W * 16 / 1e6),
                   "parallelism": "replicas x%d" % world},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT,
                "h2d_bytes_per_step": int(f_h.numel() * f_h.element_size() + s_h.numel() * 4),
                "d2h_bytes_per_step": int(o_h.numel() * 8),
                "copies": "pinned host buffers; H2D and D2H on their own streams, overlapped with the previous / "
                          "next step's kernels (two device buffers each)",
                "serial_value": round(replica_throughput(pix, K, world, e2e_serial_ms), 3)},
        # per step: one row scan, one fused n-fold line scan per direction
        # (v2, v3, v4), one mesh launch
        "gpu_launches": int(K * (1 + 3 + 1)),
        "kernels_ms": {"integrate": round(integ_ms, 4), "mesh": round(mesh_ms, 4)},
        "autotune": {"rows_per_cta": tuned_rows, "candidates": [4, 8, 16], "ms": [round(t, 3) for t in tuned_ms]},
        "roofline": {"bound": "alu", "achieved": round(achieved / 1e9, 2), "peak": round(peak_macs / 1e9, 2),
                     "unit": "G MAC/s (%d-limb integer x %d-bit weight)" % (L, 32 * wwords),
                     "frac": round(achieved / peak_macs, 4),
                     # DRAM bytes (read + write) of one launch of this kernel on this workload,
                     # from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum)
                     "traffic": MESH_DRAM_BYTES if (n == 2 and L == 2 and (H, W) == (2048, 2048)) else None,
                     "kernel": "mesh_exact_kernel",
                     "peak_note": "derived: 152 SM x 64 INT32 multiply-add lanes x median SM clock / %d "
                                  "32-bit multiply-adds per MAC; achieved = (n+1)^4 x 7n^2 stencil MACs per pixel"
                                  % imad_per_mac,
                     "probe": probe},
        "roofline_integrate": {"bound": "hbm", "achieved": round(integ_bytes / (integ_ms * 1e-3) / 1e9, 1),
                               "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                               "frac": (round(integ_bytes / (integ_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)
                                        if peaks.get("hbm_gbs") else None),
                               "traffic": INTEG_DRAM_BYTES if (n == 2 and L == 2 and (H, W) == (2048, 2048)) else None,
                               "kernel": "row_scan_warp_kernel + 3 x line_scan_kernel",
                               "bytes_note": "f read once, g written by the row scan, then read and written "
                                             "once per line direction: |f| + 7 |g| per integrate"},
        "clocks": clk,
    }
    hbm = peaks.get("hbm_gbs")
    if hbm:
        # whole step against its bounds, the kernels in sequence: the integrate at
        # the copy peak for its algorithmic bytes, then the mesh at the larger of
        # its ALU time (derived peak) and its HBM time (scales, g once, output)
        t_integ = integ_bytes / (hbm * 1e9) * 1e3
        t_alu = macs / peak_macs * 1e3
        t_mesh_hbm = pix * (16.0 + 8.0 * L + out_exact.element_size()) / (hbm * 1e9) * 1e3
        lower = t_integ + max(t_alu, t_mesh_hbm)
        line["roofline_path"] = {
            "lower_bound_ms": round(lower, 4), "achieved_ms": round(total_ms / K, 4),
            "frac": round(lower / (total_ms / K), 4),
            "parts_ms": {"integrate_hbm": round(t_integ, 4), "mesh_alu": round(t_alu, 4),
                         "mesh_hbm": round(t_mesh_hbm, 4)},
            "note": "integrate bytes / measured copy peak + max(mesh MACs / derived ALU peak, "
                    "mesh bytes / measured copy peak)"}
    if rank == 0 and args.cpu_baseline:
        cb, pts, vals = cpu_baseline(w, seconds=args.cpu_seconds, keep=True)
        try:
            done, el, procs = cpu_baseline_all_cores(args.workload, _shape(args), args.cpu_seconds)
            cb = {"value": done / el / 1e6, "unit": UNIT, "cores": procs, "kind": "oracle",
                  "sample": "%d random pixels of the same workload, exact per-pixel evaluation, one process per "
                            "host core for %.1f s; single core: %s" % (done, el, cb["sample"]),
                  "single_core_value": cb["value"]}
        except Exception as e:  # keep the single-core figure if a pool cannot start here
            cb["all_cores_error"] = str(e)[:200]
        line["cpu_baseline"] = cb
        for k, v in forms.items():
            if "out" not in v:
                continue
            v["err_range_vs_oracle"] = err_range(v["out"], pts, vals, img)
            v["err_sample"] = "%d sampled pixels" % len(pts)
    for v in forms.values():
        v.pop("out", None)
    line["forms"] = forms
    if rank == 0 and args.serving and world == 1:
        line["serving"] = serving_leg(dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    filt.close()
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """64 images of uneven size (sides 128..2048), orders mixed over {1, 2, 3},
    float32 on the 2^-16 grid, paper scales in [1, 32]: every image's
    non-adaptive step, then one persistent launch of the adaptive step over
    all images, captured once in a CUDA graph and replayed; compared with the
    same images filtered one at a time."""
    import torch
    import synthetic
    from paper_0908_3861_gb300 import AdaptiveFilter, Batch
    import __graft_entry__
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    small = args.workload == "c4s"
    jobs = (synthetic.batch_workload(count=512, lo=32, hi=256, seed_offset=rank) if small
            else synthetic.batch_workload(seed_offset=rank))
    fl, imgs, scs, outs = [], [], [], []
    for w in jobs:
        H, W = w["image"].shape
        fl.append(AdaptiveFilter(W, H, w["n"], torch.float32, scale_kind="a4", q_bits=w["q_bits"], frac_bits=16,
                                 max_scale=w["cmax"], out="f32", value_bound=255.0, device=dev))
        imgs.append(torch.from_numpy(w["image"]).to(dev))
        scs.append(torch.from_numpy(w["scales"]).to(dev))
        outs.append(torch.empty((H, W), dtype=torch.float32, device=dev))
    pix = float(sum(w["image"].size for w in jobs))
    batch = Batch(fl, dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            batch(imgs, scs, outs)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    tuned_rows, tuned_ms = batch.autotune(imgs, scs, outs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch(imgs, scs, outs)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    K = args.steps
    with ClockSampler(local) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(K):
            graph.replay()
        t1.record(stream)
        torch.cuda.synchronize()
    batch_ms = t0.elapsed_time(t1) / K
    assert all(f.device_status() == 0 for f in fl)
    # the same images one at a time
    ref = [o.clone() for o in outs]
    t0.record(stream)
    for f, i, s, o in zip(fl, imgs, scs, outs):
        f(i, s, o)
    t1.record(stream)
    torch.cuda.synchronize()
    single_ms = t0.elapsed_time(t1)
    same = all(torch.equal(a, b) for a, b in zip(ref, outs))
    # one clear, then per (limbs, order, input type) group a row pass and three
    # line passes, then one batch launch per (order, limbs, path) group present
    groups = set((w["n"], f.limbs) for w, f in zip(jobs, fl))
    n_launch = 1 + 4 * len(groups) + len(groups)
    line = {"metric": METRIC, "value": round(pix / (batch_ms * 1e-3) / 1e6, 3), "unit": UNIT, "n_gpus": 1,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(batch_ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64 limbs (2 or 4 per image)", "data": "synthetic",
            "config": {"workload": ("512 images, sides U{32..256}" if small else "64 images, sides U{128..2048}")
                                   + ", n U{1,2,3}, f32 2^-16 grid, a_k in [1,32], Q=8, exact form; one launch per "
                                   "pass and group for the non-adaptive step, one persistent launch per group for "
                                   "the adaptive step, CUDA graph replay",
                       "pixels_per_step": int(pix), "l2": "inputs larger than L2"},
            "gpu_launches": int(K * n_launch),
            "batched_vs_single": {"batched_ms": round(batch_ms, 3), "single_ms": round(single_ms, 3),
                                  "speedup": round(single_ms / batch_ms, 3), "bit_identical": bool(same)},
            "autotune": {"rows_per_cta": tuned_rows, "candidates": [4, 8, 16],
                         "ms": [round(t, 3) for t in tuned_ms]},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    for f in fl:
        f.close()


def run_line1d(args):
    """The 1-D scale-adaptive B-spline filter of Sec. 3 on 2048 signals of
    65536 samples (float32 on the 2^-16 grid, n1 = 1, n2 = 3, a in [1, 64]):
    Msample/s of integrate + filter, exact form."""
    import torch
    import torch.distributed as dist
    import synthetic
    from paper_0908_3861_gb300 import AdaptiveFilter1D
    import __graft_entry__
    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    shp = _shape(args) or (2048, 65536)
    w = synthetic.workload_1d(count=shp[0], length=shp[1], seed_offset=rank)
    if args.n1 is not None:
        w["n1"] = args.n1
    if args.n2 is not None:
        w["n2"] = args.n2
    f, a = w["signals"], w["scales"]
    count, length = f.shape
    flt = AdaptiveFilter1D(length, count, w["n1"], w["n2"], torch.float32, q_bits=w["q_bits"],
                           frac_bits=w["frac_bits"], max_scale=w["max_scale"], value_bound=w["value_bound"],
                           out="f32", device=dev)
    f_t = torch.from_numpy(f).to(dev)
    a_t = torch.from_numpy(a).to(dev)
    out = torch.empty((count, length), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        flt.integrate(f_t)
        flt.filter(a_t, out)
    torch.cuda.synchronize()
    assert flt.device_status() == 0
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(K):
            ev[i][0].record(stream)
            flt.integrate(f_t)
            ev[i][1].record(stream)
            flt.filter(a_t, out)
            ev[i][2].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world, dev)
    integ_ms = sum(x.elapsed_time(y) for x, y, z in ev) / K
    mesh_ms = sum(y.elapsed_time(z) for x, y, z in ev) / K
    assert flt.device_status() == 0
    # end to end: pinned host buffers, copies inside the timed region
    f_h, a_h = torch.from_numpy(f).pin_memory(), torch.from_numpy(a).pin_memory()
    o_h = torch.empty((count, length), dtype=torch.float32).pin_memory()
    f_d, a_d = torch.empty_like(f_t), torch.empty_like(a_t)

    def e2e_step():
        f_d.copy_(f_h, non_blocking=True)
        a_d.copy_(a_h, non_blocking=True)
        flt.integrate(f_d)
        flt.filter(a_d, out)
        o_h.copy_(out, non_blocking=True)
    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    samples = float(count * length)
    value = replica_throughput(samples, K, world, total_ms)
    L = flt.limbs
    N = w["n1"] + w["n2"] + 1
    K_nb = N + 1 if N % 2 else N + 2
    macs = (w["n2"] + 2) * K_nb
    imad = {1: 4, 2: 12, 3: 20, 4: 28}[L]
    clk = clk.summary()
    sm_mhz = clk["sm_mhz"] or _peaks().get("sm_max_mhz", 2070.0)
    peak = 152 * 64 * sm_mhz * 1e6 / imad
    achieved = macs * samples / (mesh_ms * 1e-3)
    line = {
        "metric": "Msample/s 1-D scale-adaptive B-spline filter (Sec. 3), exact form", "value": round(value, 3),
        "unit": "Msample/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(total_ms / K, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64x%d" % L, "data": "synthetic",
        "config": {"workload": "%d signals x %d samples f32 (2^-16 grid), n1=%d, n2=%d, a in [1,64], Q=8, exact form%s"
                               % (count, length, w["n1"], w["n2"],
                                  " (c = f * (b^n1)^-1 on the 2^-16 grid)" if w["n1"] >= 2 else ""),
                   "l2": "inputs larger than L2 (signals %.0f MB, scales %.0f MB)"
                               % (f.nbytes / 1e6, a.nbytes / 1e6), "parallelism": "replicas x%d" % world},
        "e2e": {"value": round(replica_throughput(samples, K, world, e2e_ms), 3), "unit": "Msample/s",
                "h2d_bytes_per_step": int(f.nbytes + a.nbytes), "d2h_bytes_per_step": int(o_h.numel() * 4)},
        "gpu_launches": int(K * (3 if w["n1"] >= 2 else 2)),
        "kernels_ms": {"integrate": round(integ_ms, 4), "mesh": round(mesh_ms, 4)},
        "roofline": {"bound": "alu", "achieved": round(achieved / 1e9, 2), "peak": round(peak / 1e9, 2),
                     "unit": "G MAC/s (%d-limb integer x 64-bit weight)" % L, "frac": round(achieved / peak, 4),
                     "traffic": None, "kernel": "mesh1d_kernel",
                     "peak_note": "derived: 152 SM x 64 INT32 multiply-add lanes x median SM clock / %d 32-bit "
                                  "multiply-adds per MAC; achieved = (n2+2) x %d stencil MACs per sample"
                                  % (imad, K_nb)},
        "roofline_integrate": {"bound": "hbm", "achieved": round((f.nbytes + samples * 8 * L) / (integ_ms * 1e-3)
                                                                 / 1e9, 1),
                               "peak": _peaks().get("hbm_gbs"), "unit": "GB/s",
                               "bytes_note": "f read once, g written once" +
                                             ("; prefilter + row pass" if w["n1"] >= 2 else "")},
        "clocks": clk,
    }
    if rank == 0 and args.cpu_baseline:
        from oracle import line1d as o
        t_start = time.perf_counter()
        done = 0
        rng = np.random.default_rng(7)
        fi = (f.astype(np.float64) * 65536.0).astype(np.int64)
        while time.perf_counter() - t_start < args.cpu_seconds:
            r = int(rng.integers(0, count))
            ms = sorted(rng.integers(0, length, 64).tolist())
            A = o.quantise(a[r], w["q_bits"])
            if w["n1"] >= 2:
                kq, cq = o.prefilter_quantised([int(v) for v in fi[r]], w["n1"])
            else:
                kq, cq = 0, list(fi[r])
            o.filter_paper_at(cq, A, w["n1"], w["n2"], w["q_bits"], w["frac_bits"], ms, k_first=kq)
            done += len(ms)
        el = time.perf_counter() - t_start
        line["cpu_baseline"] = {"value": done / el / 1e6, "unit": "Msample/s", "cores": 1, "kind": "oracle",
                                "sample": "%d samples (64 per signal, each signal's running sums in full), "
                                          "exact, %.1f s" % (done, el)}
    flt.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_scale_map(args):
    """Scale-map estimation (structure tensor -> ellipse per pixel) on the
    2048x2048 order-2 image, then the exact filter driven by that field:
    Mpixel/s of estimate + integrate + filter, and of the estimator alone."""
    import torch
    import synthetic
    from paper_0908_3861_gb300 import AdaptiveFilter, estimate_ellipses
    import __graft_entry__
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    shp = _shape(args) or (2048, 2048)
    w = synthetic.workload("c2", shape=shp, seed_offset=rank)
    img = w["image"]
    H, W = img.shape
    f_t = torch.from_numpy(img).to(dev)
    filt = AdaptiveFilter(W, H, 2, torch.float32, scale_kind="ellipse", q_bits=8, frac_bits=16, max_scale=64.0,
                          out="f32", value_bound=255.0, device=dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)

    def step():
        field = estimate_ellipses(f_t, rho=2.0, sigma0=6.0, e_max=4.0)
        filt.integrate(f_t)
        filt.filter(field, out)
        return field
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert filt.device_status() == 0
    stream = torch.cuda.current_stream(dev)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(K):
            ev[i][0].record(stream)
            field = estimate_ellipses(f_t, rho=2.0, sigma0=6.0, e_max=4.0)
            ev[i][1].record(stream)
            filt.integrate(f_t)
            filt.filter(field, out)
        t1.record(stream)
        torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1) / K
    est_ms = sum(a.elapsed_time(b) for a, b in ev) / K
    assert filt.device_status() == 0
    pix = float(H * W)
    line = {"metric": "Mpixel/s scale-map estimation + exact adaptive filter (ellipse per pixel from the structure "
                      "tensor)", "value": round(pix / (total_ms * 1e-3) / 1e6, 3), "unit": "Mpixel/s", "n_gpus": 1,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(total_ms, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 tensor, f64 eigen, int64x%d filter" % filt.limbs,
            "data": "synthetic",
            "config": {"workload": "%dx%d f32 (2^-16 grid) image of the order-2 recipe; rho 2, sigma0 6, e_max 4; "
                                   "exact order-2 filter, Q=8" % (H, W)},
            "estimator": {"ms": round(est_ms, 4), "mpix_s": round(pix / (est_ms * 1e-3) / 1e6, 1),
                          "hbm_bytes_note": "f read, 3 planes written, read and written (row pass), read (column "
                                            "pass), float4 written: %.0f MB" % ((4 + 12 + 24 + 12 + 16) * pix / 1e6)},
            "gpu_launches": int(K * (3 + 5)),
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    filt.close()


def run_constant_cost(args):
    """Sec. 7 states that the cost per output pixel does not depend on the
    scale vector.  Mesh time per Mpixel for spatially constant steps
    c1 = c2 = c3 = c4 = c in {1, 4, 16, 64} on the 2048^2 image of the order-2
    recipe, orders 1 and 2, one plan per order (max_scale 64, so the limb
    count is the same for every c), CUDA events on the launching stream."""
    import torch
    import synthetic
    from paper_0908_3861_gb300 import AdaptiveFilter
    import __graft_entry__
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    shp = _shape(args) or (2048, 2048)
    w = synthetic.workload("c2", shape=shp)
    img = w["image"]
    H, W = img.shape
    f_t = torch.from_numpy(img).to(dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = {}
    launches = 0
    with ClockSampler(local) as clk:
        for n in (1, 2):
            filt = AdaptiveFilter(W, H, n, torch.float32, scale_kind="c4", q_bits=8, frac_bits=16, max_scale=64.0,
                                  out="f32", value_bound=255.0, device=dev)
            filt.integrate(f_t)
            per = {}
            for c in (1.0, 4.0, 16.0, 64.0):
                sc = torch.full((H, W, 4), c, dtype=torch.float32, device=dev)
                for _ in range(args.warmup):
                    filt.filter(sc, out)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(args.steps):
                    filt.filter(sc, out)
                b.record(stream)
                torch.cuda.synchronize()
                launches += args.steps
                ms = a.elapsed_time(b) / args.steps
                per[str(int(c))] = {"mesh_ms": round(ms, 4), "ms_per_mpixel": round(ms / (H * W / 1e6), 5)}
            assert filt.device_status() == 0
            vals = [v["ms_per_mpixel"] for v in per.values()]
            rows["n%d" % n] = {"limbs": filt.limbs, "by_step": per,
                               "max_over_min": round(max(vals) / min(vals), 3)}
            filt.close()
    base = rows["n2"]["by_step"]["1"]["mesh_ms"]
    line = {"metric": "mesh ms per Mpixel vs constant step c (Sec. 7: cost independent of the scales)",
            "value": rows["n2"]["max_over_min"], "unit": "max/min ms per Mpixel over c in {1,4,16,64}, order 2",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": base,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64 limbs",
            "data": "synthetic",
            "config": {"workload": "%dx%d f32 image of the order-2 recipe, constant steps c1=c2=c3=c4=c, exact form, "
                                   "Q=8, max_scale 64" % (H, W), "l2": "inputs larger than L2"},
            "gpu_launches": launches, "orders": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


GENERAL = {
    # N = 2 (theta = 0, pi/2), order 2, steps c1, c3 in [1, 24], phi = delta
    "n2": dict(directions=2, n=2, model_boxes=0, lo=1.0, hi=24.0, q_bits=6,
               text="N = 2 (tensor box splines), order n=2, steps c1, c3 in [1,24] from S(64) fields, phi = delta"),
    # N = 4, order 1 (Sec. 7), cubic B-spline model phi with its 2-D prefilter
    "m3": dict(directions=4, n=1, model_boxes=4, lo=1.0, hi=8.0, q_bits=6,
               text="N = 4, order n=1, cubic B-spline model phi (prefilter in the step), paper scales a_k in [1,8]"),
}


def _stencil_macs(directions, n, E):
    """Algorithmic MACs per pixel of a generalised plan: taps prod (r_k + 1)
    times the area of the interpolation kernel's support (the zonotope of its
    directions: sum over pairs m_i m_j |det(v_i, v_j)|, its average count of
    non-zero lattice weights)."""
    V = ((1, 0), (1, 1), (0, 1), (-1, 1))
    r = (n, n if directions == 4 else 0, n, n if directions == 4 else 0)
    m = (r[0] + E, r[1], r[2] + E, r[3])
    area = sum(m[i] * m[j] * abs(V[i][0] * V[j][1] - V[i][1] * V[j][0]) for i in range(4) for j in range(i + 1, 4))
    taps = 1
    for rk in r:
        taps *= rk + 1
    return taps * area


def run_general(args):
    """Generalised plans on the 2048^2 image of the order-2 recipe: N = 2
    ('n2') or the cubic B-spline model ('m3'): Mpixel/s of integrate (with the
    model's prefilter) + filter, exact form, and the mesh against the derived
    integer peak."""
    import torch
    import synthetic
    from paper_0908_3861_gb300 import AdaptiveFilter
    import __graft_entry__
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    cfg = GENERAL[args.workload]
    shp = _shape(args) or (2048, 2048)
    w = synthetic.workload("c2", shape=shp, seed_offset=rank)
    img = w["image"]
    H, W = img.shape
    rng = np.random.default_rng(synthetic.SEED_BASE + 5)
    sc = synthetic.scales_a4(rng, (H, W), cfg["lo"], cfg["hi"], 64.0).astype(np.float32)
    kind = "a4"
    if cfg["directions"] == 2:
        sc[..., 1] = 1.0
        sc[..., 3] = 1.0
        kind = "c4"
    filt = AdaptiveFilter(W, H, cfg["n"], torch.float32, scale_kind=kind, q_bits=cfg["q_bits"], frac_bits=16,
                          max_scale=cfg["hi"], out="f32", value_bound=255.0, device=dev,
                          directions=cfg["directions"], model_boxes=cfg["model_boxes"])
    f_t = torch.from_numpy(img).to(dev)
    s_t = torch.from_numpy(sc).to(dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        filt.integrate(f_t)
        filt.filter(s_t, out)
    torch.cuda.synchronize()
    assert filt.device_status() == 0
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(K):
            ev[i][0].record(stream)
            filt.integrate(f_t)
            ev[i][1].record(stream)
            filt.filter(s_t, out)
            ev[i][2].record(stream)
        t1.record(stream)
        torch.cuda.synchronize()
    total_ms = t0.elapsed_time(t1) / K
    integ_ms = sum(a.elapsed_time(b) for a, b, c in ev) / K
    mesh_ms = sum(b.elapsed_time(c) for a, b, c in ev) / K
    assert filt.device_status() == 0
    pix = float(H * W)
    L = filt.limbs
    clk = clk.summary()
    sm_mhz = clk["sm_mhz"] or _peaks().get("sm_max_mhz", 2070.0)
    D = filt.denominator()
    Dv = sum(int(v) << (32 * i) for i, v in enumerate(D)) if not isinstance(D, int) else D
    wwords = 2 if Dv < (1 << 64) else 4   # 64-bit or 128-bit table weights
    imad = (sum(1 for i in range(2 * L) for j in range(wwords) if i + j <= 2 * L - 1)
            + sum(1 for i in range(2 * L) for j in range(wwords) if i + j <= 2 * L - 2))
    macs = _stencil_macs(cfg["directions"], cfg["n"], cfg["model_boxes"]) * pix
    peak = 152 * 64 * sm_mhz * 1e6 / imad
    achieved = macs / (mesh_ms * 1e-3)
    line = {"metric": "Mpixel/s adaptive filter, generalised plan (%s)" % args.workload,
            "value": round(pix / (total_ms * 1e-3) / 1e6, 3), "unit": "Mpixel/s", "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": round(total_ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64x%d" % L, "data": "synthetic",
            "config": {"workload": "%dx%d f32 (2^-16 grid) image of the order-2 recipe; %s; Q=%d; exact form"
                                   % (H, W, cfg["text"], cfg["q_bits"]), "l2": "inputs larger than L2"},
            "gpu_launches": int(K * (5 if cfg["model_boxes"] >= 3 else 3) + K * (1 if cfg["directions"] == 2 else 3)),
            "kernels_ms": {"integrate": round(integ_ms, 4), "mesh": round(mesh_ms, 4)},
            "roofline": {"bound": "alu", "achieved": round(achieved / 1e9, 2), "peak": round(peak / 1e9, 2),
                         "unit": "G MAC/s (%d-limb integer x %d-bit weight)" % (L, 32 * wwords),
                         "frac": round(achieved / peak, 4), "traffic": None, "kernel": "mesh_gen_kernel",
                         "peak_note": "derived as for the main line; achieved = taps x support area of the "
                                      "interpolation kernel (%d MACs per pixel)"
                                      % _stencil_macs(cfg["directions"], cfg["n"], cfg["model_boxes"])},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    filt.close()


def _serve_pool(npool, inflight, dev, rank=0):
    """Distinct jobs of the serving recipe: sides U{256..4096}, float32 images
    on the 2^-16 grid (smooth field + edges), ellipse fields as the 2048^2
    order-2 workload; one descriptor per order n in {1, 2}, whose scale-product
    bound comes from the recipe's parameter range (sigma <= 24, elongation <= 6)."""
    import torch
    import synthetic
    from paper_0908_3861_gb300 import make_desc, ellipse_product_bound
    rng = np.random.default_rng(synthetic.SEED_BASE + 4 + 97 * rank)
    prods = {n: ellipse_product_bound(24.0, 6.0, n, 8, 150.0, device=dev) for n in (1, 2)}
    pool = []
    for i in range(npool):
        h, w = int(rng.integers(256, 4097)), int(rng.integers(256, 4097))
        r = np.random.default_rng(synthetic.SEED_BASE + 4 + 1000 * (i + 1))
        img = synthetic.image_f32_grid(r, (h, w), 24.0, 12, 16)
        sc = synthetic.ellipse_field(r, (h, w))
        pool.append(dict(img=torch.from_numpy(img).pin_memory(), sc=torch.from_numpy(sc).pin_memory(),
                         outs=[torch.empty((h, w), dtype=torch.float32).pin_memory() for _ in range(inflight + 2)],
                         desc={n: make_desc(w, h, n, torch.float32, scale_kind="ellipse", q_bits=8, frac_bits=16,
                                            max_scale=150.0, out="f32", value_bound=255.0,
                                            max_scale_product=prods[n]) for n in (1, 2)},
                         px=h * w, next=0))
    return pool


def _serve_stream(pool, budget, inflight, lam, njobs, warm, seed, dev, group=True):
    """One request stream through the library's server: njobs jobs drawn from
    the pool (order n U{1,2}) with exponential gaps of mean 1/lam seconds (lam
    = 0: all at once); latency = done - submit of the jobs after the first
    `warm`.  Every job's status must be ok."""
    from paper_0908_3861_gb300 import Server
    srv = Server(budget, max_inflight=inflight, device=dev, group_mesh=group)
    rg = np.random.default_rng(seed)

    def submit(e, n):
        o = e["outs"][e["next"] % len(e["outs"])]
        e["next"] += 1
        return srv.submit(e["desc"][n], e["img"], e["sc"], o), e["px"]

    for e in pool:                       # plans and tables, outside the measurement
        for n in (1, 2):
            srv.wait(submit(e, n)[0])
    gaps = rg.exponential(1.0 / lam, njobs) if lam else np.zeros(njobs)
    t0 = time.perf_counter()
    due = t0
    tickets = []
    for k in range(njobs):
        due += gaps[k]
        dt = due - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        e = pool[int(rg.integers(0, len(pool)))]
        tickets.append(submit(e, int(rg.integers(1, 3))))
    stats = [(srv.wait(t), px) for t, px in tickets]
    peak = srv.stats()["peak"]
    srv.close()
    assert all(s["status"] == 0 and s["device_status"] == 0 for s, _ in stats)
    meas = stats[warm:]
    lat = np.array([(s["t_done_us"] - s["t_submit_us"]) * 1e-3 for s, _ in meas])
    span = (max(s["t_done_us"] for s, _ in meas) - min(s["t_submit_us"] for s, _ in meas)) * 1e-6
    # device overlap: pairs of consecutive jobs whose device-clock intervals intersect
    iv = sorted((s["t_gpu_start_us"], s["t_gpu_end_us"]) for s, _ in meas)
    overl = sum(1 for a, b in zip(iv, iv[1:]) if b[0] < a[1])
    return dict(p50_ms=round(float(np.percentile(lat, 50)), 2), p99_ms=round(float(np.percentile(lat, 99)), 2),
                mpix_s=round(sum(px for _, px in meas) / span / 1e6, 2), jobs=len(meas), warmup_jobs=warm,
                jobs_per_s=round(len(meas) / span, 2), overlapping_neighbours=overl, peak_bytes=int(peak),
                budget_bytes=int(budget))


def serving_leg(dev, npool=4, inflight=4, sat_jobs=32, jobs=300, warm=30):
    """A short serving measurement for the default line: saturation rate from
    a burst, then p50/p99 latency of a Poisson stream at 0.8 of it."""
    import torch
    pool = _serve_pool(npool, inflight, dev)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(free * 0.5)
    sat = _serve_stream(pool, budget, inflight, 0.0, sat_jobs, 0, 11, dev)
    load = _serve_stream(pool, budget, inflight, 0.8 * sat["jobs_per_s"], jobs + warm, warm, 80, dev)
    return {"workload": "Poisson stream at 0.8 x the saturation rate, %d distinct jobs, sides U{256..4096}, "
                        "n U{1,2}, f32 + ellipse fields; exact form; %d slots, jobs admitted together share "
                        "one batched adaptive-step launch; HBM budget half the free memory" % (npool, inflight),
            "saturation_mpix_s": sat["mpix_s"], "saturation_jobs_per_s": sat["jobs_per_s"],
            "p50_ms": load["p50_ms"], "p99_ms": load["p99_ms"], "mpix_s": load["mpix_s"], "jobs": load["jobs"],
            "warmup_jobs": warm, "overlapping_neighbours": load["overlapping_neighbours"]}


def run_serve(args):
    """Poisson-arrival stream of filter jobs (sides U{256..4096}, n U{1,2},
    float32 images on the 2^-16 grid with ellipse fields as the 2048^2 case)
    through the library's request loop, admitted by device-memory footprint
    (budget: half the free HBM).  Measures the saturation rate, then p50/p99
    latency (done - arrival) at 0.5, 0.8 and 0.95 of it (--jobs measured jobs
    after a warm-up of a tenth as many); and the same stream at 0.8 of it
    through a one-job-at-a-time server."""
    import torch
    import __graft_entry__
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    pool = _serve_pool(args.pool, args.inflight, dev, rank)
    free, _ = torch.cuda.mem_get_info(dev)
    budget = int(free * 0.5)
    warm = max(args.jobs // 10, 1)
    with ClockSampler(local) as clk:
        sat = _serve_stream(pool, budget, args.inflight, 0.0, args.sat_jobs, 0, 11, dev)
        mu = sat["jobs_per_s"]
        loads = {}
        for frac in (0.5, 0.8, 0.95):
            loads[str(frac)] = _serve_stream(pool, budget, args.inflight, frac * mu, args.jobs + warm, warm,
                                             int(frac * 100), dev)
        fifo = _serve_stream(pool, budget, 1, 0.8 * mu, args.jobs + warm, warm, 80, dev)
        ungrouped = _serve_stream(pool, budget, args.inflight, 0.8 * mu, args.jobs + warm, warm, 80, dev,
                                  group=False)
    line = {"metric": METRIC, "value": sat["mpix_s"], "unit": UNIT, "n_gpus": 1, "steps": args.sat_jobs,
            "warmup": 2 * len(pool), "ms_per_step": round(1e3 / mu, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64 limbs", "data": "synthetic",
            "config": {"workload": "Poisson stream of filter jobs, sides U{256..4096}, n U{1,2}, f32 2^-16 grid, "
                                   "ellipse fields; exact form; HBM budget = half the free memory",
                       "pool_images": len(pool), "slots": args.inflight, "budget_bytes": budget},
            "saturation": sat, "latency": loads, "fifo_at_0.8": fifo, "ungrouped_at_0.8": ungrouped,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, seconds=15.0, sample=None, keep=False):
    """The oracle (exact, per-pixel windows) on a bounded sample of the workload."""
    from oracle import paper, scales as osc
    img, sc = w["image"], w["scales"]
    H, W = img.shape
    fi = (img.astype(np.float64) * float(1 << w["frac_bits"])).astype(np.int64)
    rng = np.random.default_rng(7)
    C = osc.scales_to_C(w["scale_kind"], sc, w["n"], w["q_bits"], w["cmax"])
    done, t0 = 0, time.perf_counter()
    pts, vals = [], []
    while time.perf_counter() - t0 < seconds and (sample is None or done < sample):
        p = (int(rng.integers(0, W)), int(rng.integers(0, H)))
        _, sv = paper.filter_pixels(fi, C, w["n"], w["q_bits"], w["frac_bits"], [p])
        pts.append(p)
        vals.append(float(sv[0]))
        done += 1
    el = time.perf_counter() - t0
    out = {"value": done / el / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d random pixels of the same workload, exact per-pixel evaluation, %.1f s" % (done, el)}
    if keep:
        return out, pts, vals
    return out


_WORKER_CACHE = {}


def _oracle_sample_worker(job):
    """One host core: the oracle as it stands on random pixels of the workload
    (regenerated from its seed once per process), for `seconds`."""
    name, shape, seed, seconds = job
    from oracle import paper, scales as osc
    key = (name, shape)
    if key not in _WORKER_CACHE:
        w = _workload(name, 0, shape)
        fi = (w["image"].astype(np.float64) * float(1 << w["frac_bits"])).astype(np.int64)
        C = osc.scales_to_C(w["scale_kind"], w["scales"], w["n"], w["q_bits"], w["cmax"])
        _WORKER_CACHE[key] = (w, fi, C)
    w, fi, C = _WORKER_CACHE[key]
    H, W = fi.shape
    rng = np.random.default_rng(seed)
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        p = (int(rng.integers(0, W)), int(rng.integers(0, H)))
        paper.filter_pixels(fi, C, w["n"], w["q_bits"], w["frac_bits"], [p])
        done += 1
    return done, time.perf_counter() - t0


def _oracle_pool(procs):
    """One process per host core, started with spawn (the parent may hold a CUDA
    context).  An executor, not a Pool: a worker that cannot start raises
    instead of being restarted forever."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn"))


def _oracle_round(ex, procs, name, shape, seconds, seed0):
    jobs = [(name, shape, seed0 + i, seconds) for i in range(procs)]
    res = list(ex.map(_oracle_sample_worker, jobs, timeout=seconds + 300.0))
    return sum(d for d, _ in res), max(t for _, t in res)


def cpu_baseline_all_cores(name, shape, seconds, procs=None):
    """The same oracle sample on every host core at once.  Returns (pixels,
    seconds of the slowest worker's timed loop, processes)."""
    procs = procs or os.cpu_count() or 1
    with _oracle_pool(procs) as ex:
        done, el = _oracle_round(ex, procs, name, shape, seconds, 1000)
    return done, el, procs


def err_range(out, pts, vals, img):
    """max |s - s_oracle| / (max f - min f) over the sampled pixels that the
    form did not flag (NaN: its error bound exceeded its tolerance)."""
    d = [abs(float(out[y, x]) - v) for (x, y), v in zip(pts, vals) if np.isfinite(out[y, x])]
    if not d:
        return None
    rng = float(img.max()) - float(img.min())
    return max(d) / rng


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    w = _workload(args.workload, 0, _shape(args))
    K = args.steps
    per = max(1.0, min(20.0, 150.0 / max(K, 1)))
    procs = os.cpu_count() or 1
    with _oracle_pool(procs) as ex:
        # warm-up rounds also build each worker's copy of the workload
        for i in range(max(args.warmup, 1)):
            _oracle_round(ex, procs, args.workload, _shape(args), 0.2, 500 + i * procs)
        t0 = time.perf_counter()
        tot_pix = 0
        for k in range(K):
            done, _ = _oracle_round(ex, procs, args.workload, _shape(args), per, 1000 + k * procs)
            tot_pix += done
        el = time.perf_counter() - t0
    value = tot_pix / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": el * 1e3 / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "exact (python int)", "data": "synthetic",
            "config": {"workload": "%dx%d %s" % (w["image"].shape[0], w["image"].shape[1],
                                                   WORKLOAD_TEXT[args.workload])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": "%d random pixels per step (%.1f s of the oracle on each of %d host "
                                       "cores), exact per-pixel evaluation" % (tot_pix // K, per, procs)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--shape", default="", help="HxW: the same recipe at another size (profiling, sweeps)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--n1", type=int, default=None, help="d1: model degree (2..5 interpolate the samples)")
    ap.add_argument("--n2", type=int, default=None, help="d1: analysis degree")
    ap.add_argument("--pool", type=int, default=8, help="c5: distinct images in the request pool")
    ap.add_argument("--inflight", type=int, default=4, help="c5: concurrent jobs (slots)")
    ap.add_argument("--jobs", type=int, default=2000, help="c5: measured jobs per load (after a tenth as many)")
    ap.add_argument("--sat-jobs", dest="sat_jobs", type=int, default=200, help="c5: jobs of the saturation burst (long enough for a sustained rate)")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="default workload: skip the short serving leg")
    ap.add_argument("--compare", default="plain_f64,tile_f32",
                    help="comma-separated forms timed beside the exact form ('' for none)")
    args = ap.parse_args()
    args.compare = [c for c in args.compare.split(",") if c]
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("c4", "c4s"):
        run_batch(args)
    elif args.workload == "c5":
        run_serve(args)
    elif args.workload == "d1":
        run_line1d(args)
    elif args.workload == "s2":
        run_scale_map(args)
    elif args.workload == "cc":
        run_constant_cost(args)
    elif args.workload in GENERAL:
        run_general(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
