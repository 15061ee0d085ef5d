"""Benchmark of the specular ray-tracing hot path on GB300.

One step = one pass of the whole path over the seeded synthetic city
(4802 triangles, 1 transmitter with a TR 38.901 dual-polarized sector
pattern, 1000 receivers, 3.5 GHz):
  LBVH build -> compute_paths (1e6 Fibonacci rays, max_depth 3: shooting and
  bouncing, duplicate removal, image method, LOS) -> CIR -> H(f) at 1024
  subcarriers of 30 kHz -> coverage map (500 x 500 cells of 1 m at 1.5 m,
  1e6 rays, max_depth 3) -> VJP of H(f) and of the CIR w.r.t. materials and
  transmitter pose.
metric = rays*bounces/s: ray segments tested against the scene in the whole
job / time: closest-hit queries (shooting and bouncing, and every coverage
segment that can reflect again) plus the coverage rays' last segments, each
tested up to the map plane by an any-hit query. Last segments that cannot
reach the map inside the grid are not traced and not counted.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: replicas only (each rank traces its own copy of the workload,
no collective on the data path), launched with torch.distributed.run.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_RAYS = 1_000_000
MAX_DEPTH = 3
N_RX = 1000
N_SC = 1024
SC_SPACING = 30e3
FC = 3.5e9
GRID = dict(x0=-250.0, y0=-250.0, cell=1.0, nx=500, ny=500, h=1.5)
WORKLOAD = "city-4802tri-1tx-1000rx-1e6rays-d3-1024sc-cm500x500"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class _Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml ships with the driver)."""

    SM = 1
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, device_index: int):
        import ctypes
        import torch
        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(device_index)
        ok = False
        uuid = getattr(props, "uuid", None)
        if uuid is not None:
            ok = self.lib.nvmlDeviceGetHandleByUUID(f"GPU-{uuid}".encode(), ctypes.byref(self.h)) == 0
        if not ok:
            bus = f"{props.pci_domain_id:08x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0".encode()
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(self.h)) == 0
        if not ok:
            raise OSError("no NVML handle for the CUDA device")
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn if fn is not None else self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        v = self.c.c_uint()
        m = self.c.c_uint()
        r = self.c.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.c.byref(v)) or
                self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, self.c.byref(m)) or
                self.reasons_fn(self.h, self.c.byref(r))):
            return None
        return float(v.value), float(m.value), sorted(n for b, n in self.REASONS.items() if r.value & b)


class Clocks:
    """Samples SM clocks and throttle reasons during the timed region: NVML
    every 2 ms from a thread (nvidia-smi at 10 ms if NVML cannot be loaded)."""

    def __init__(self, index: int, period_s: float = 0.002):
        self.index = index
        self.period = period_s
        self.samples = []      # (sm_mhz, max_mhz, [reasons])
        self.proc = None
        self.stop = threading.Event()
        self.thread = None
        self.source = None

    def __enter__(self):
        try:
            nv = _Nvml(self.index)
            self.source = "nvml, 2 ms"

            def run():
                while not self.stop.is_set():
                    s = nv.sample()
                    if s is not None:
                        self.samples.append(s)
                    time.sleep(self.period)
            s0 = nv.sample()
            if s0 is not None:
                self.samples.append(s0)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return self
        except (OSError, AttributeError):
            pass
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi, 10 ms"
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6 and parts[0].replace(".", "").isdigit() and parts[1].replace(".", "").isdigit():
                self.samples.append((float(parts[0]), float(parts[1]),
                                     [names[k] for k in range(4) if parts[2 + k] == "Active"]))

    def __exit__(self, *a):
        self.stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "source": self.source}
        sm = [x[0] for x in self.samples]
        mx = [x[1] for x in self.samples]
        reasons = sorted({r for x in self.samples for r in x[2]})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "sm_min_mhz": min(sm),
                "reasons": reasons, "samples": len(self.samples), "source": self.source}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import scenes as S
    from paper_2303_11103_gb300.shard import max_over_ranks, sum_over_ranks

    world, rank, local = dist_init()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    # the step runs on a high-priority stream: the coverage map on the
    # context's second stream (lowest priority, short-lived blocks) then
    # yields its SM slots to the candidate refinement, CIR and H(f) kernels
    torch.cuda.set_stream(torch.cuda.Stream(device=dev, priority=-1))

    scene = S.city_scene(20)
    # replicas: every rank traces its own transmitter (independent problems, no collective)
    tx, rx = S.city_devices(scene, n_rx=N_RX, seed=2 + rank)
    freqs_h =(np.arange(N_SC, dtype=np.float64) - N_SC // 2) * SC_SPACING
    # pinned host inputs (end-to-end leg) and device-resident copies (kernel leg)
    host = {"verts": torch.from_numpy(scene.verts).pin_memory(),
            "mat": torch.from_numpy(scene.mat_id).pin_memory(),
            "mats": torch.from_numpy(scene.materials).pin_memory(),
            "txp": torch.from_numpy(tx.pos).pin_memory(), "txy": torch.from_numpy(tx.ypr).pin_memory(),
            "rxp": torch.from_numpy(rx.pos).pin_memory(), "rxy": torch.from_numpy(rx.ypr).pin_memory(),
            "freqs": torch.from_numpy(freqs_h).pin_memory()}
    devin = {k: v.to(dev) for k, v in host.items()}
    tr = rt.Tracer(local, FC)
    ctx = tr.ctx
    grid = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    n_pairs = N_RX
    nrp, ntp = rx.antenna.n_ports, tx.antenna.n_ports
    H = torch.empty((n_pairs, nrp, ntp, N_SC, 2), dtype=torch.float32, device=dev)
    gain = torch.empty((1, GRID["ny"], GRID["nx"]), dtype=torch.float32, device=dev)
    hits = torch.empty((1, GRID["ny"], GRID["nx"]), dtype=torch.int32, device=dev)
    g_eps = torch.zeros(3, device=dev)
    g_sig = torch.zeros(3, device=dev)
    g_pos = torch.zeros((1, 3), device=dev)
    g_ypr = torch.zeros((1, 3), device=dev)
    state = {}

    def step(inp, concurrent=True, after_freq=None):
        """One pass of the hot path. concurrent: the coverage map is traced on
        the context's second stream (rt_coverage_map_async), from the end of
        the path trace, beside the candidate refinement, CIR, H(f), the
        read-back of H and the VJPs (--schedule after_trace, the default), or
        from the time compute_paths returns (after_paths);
        otherwise every call runs in order on one stream. after_freq: called
        once H is final (the end-to-end leg starts its read-back there)."""
        rt.rt_set_stream(ctx)
        # the devices do not depend on the scene: set them first, so their host
        # work is not a gap after the scene load's readback
        rt.rt_set_tx(ctx, inp["txp"], inp["txy"], tx.antenna)
        rt.rt_set_rx(ctx, inp["rxp"], inp["rxy"], rx.antenna)
        rt.rt_load_scene(ctx, inp["verts"], inp["mat"], inp["mats"])
        if concurrent and args.schedule == "after_trace":
            rt.rt_coverage_map_async(ctx, grid, MAX_DEPTH, N_RAYS, 0, gain, hits, rt.ASYNC_AFTER_TRACE,
                                     args.side_blocks)
        if concurrent and args.schedule == "with_trace":
            rt.rt_coverage_map_async(ctx, grid, MAX_DEPTH, N_RAYS, 0, gain, hits, 0, args.side_blocks)
        P = rt.rt_compute_paths(ctx, MAX_DEPTH, N_RAYS, rt.RT_LOS | rt.RT_REFLECTION)
        if concurrent and args.schedule == "after_paths":
            rt.rt_coverage_map_async(ctx, grid, MAX_DEPTH, N_RAYS, 0, gain, hits, 0, args.side_blocks)
        a = torch.empty((max(P, 1), nrp, ntp, 2), dtype=torch.float32, device=dev)
        tau = torch.empty(max(P, 1), dtype=torch.float32, device=dev)
        rt.rt_cir(ctx, rt.RT_LOS | rt.RT_REFLECTION, a, tau)
        rt.rt_freq_response(ctx, a, tau, inp["freqs"], H)
        if after_freq is not None:
            after_freq()
        if not concurrent:
            rt.rt_coverage_map(ctx, grid, MAX_DEPTH, N_RAYS, 0, gain, hits)
        # VJP of L = 0.5 ||H||^2: grad_H = H
        ga = torch.empty_like(a)
        gt = torch.empty_like(tau)
        rt.rt_freq_response_backward(ctx, a, tau, inp["freqs"], H, ga, gt)
        rt.rt_cir_backward(ctx, rt.RT_LOS | rt.RT_REFLECTION, ga, gt, g_eps, g_sig, g_pos, g_ypr)
        if concurrent:
            rt.rt_join(ctx)
        state["P"] = P
        state["a"], state["tau"] = a, tau

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    # untimed: per-kernel work counts of one step (counting kernel variants)
    for _ in range(max(args.warmup, 3)):
        step(devin)
    torch.cuda.synchronize()
    rt.rt_profile(ctx, rt.PROFILE_COUNT)
    rt.rt_profile_report(ctx, reset=True)
    rt.rt_load_scene(ctx, devin["verts"], devin["mat"], devin["mats"])
    rt.rt_set_tx(ctx, devin["txp"], devin["txy"], tx.antenna)
    rt.rt_set_rx(ctx, devin["rxp"], devin["rxy"], rx.antenna)
    rt.rt_compute_paths(ctx, MAX_DEPTH, N_RAYS, rt.RT_LOS | rt.RT_REFLECTION)
    sbr_counts = rt.rt_profile_report(ctx, reset=True)
    path_stats = {k: sbr_counts[k] for k in ("sbr_keys", "candidates", "paths")}
    rt.rt_coverage_map(ctx, grid, MAX_DEPTH, N_RAYS, 0, gain, hits)
    cov_counts = rt.rt_profile_report(ctx, reset=True)
    step(devin, concurrent=False)   # the second stream's map has its own work counter
    one = rt.rt_profile_report(ctx, reset=True)
    bounces_per_step = one["closest_hit"] + one.get("plane_segments", 0)
    rt.rt_profile(ctx, False)

    # per-kernel breakdown: every launch bracketed by CUDA events, outside the timed region
    stream = torch.cuda.current_stream()
    n_prof = max(3, min(args.steps, 20))
    # the same step on one stream, timed as a whole (the overlap's gain)
    seq_ms = []
    for _ in range(n_prof):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(devin, concurrent=False)
        e1.record(stream)
        e1.synchronize()
        seq_ms.append(e0.elapsed_time(e1))
    rt.rt_profile(ctx, True)
    rt.rt_profile_report(ctx, reset=True)
    for _ in range(n_prof):
        flush.zero_()
        step(devin, concurrent=False)   # one stream: durations without overlap
    torch.cuda.synchronize()
    breakdown = rt.rt_profile_report(ctx, reset=True)["kernels"]

    dom = max(breakdown, key=lambda k: breakdown[k][1])

    # timed kernel leg: inputs resident in HBM; only the dominant kernel is
    # bracketed by events (its launch durations feed the roofline)
    times = []
    rt.rt_profile_select(ctx, [dom])
    rt.rt_profile_report(ctx, reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(devin)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    prof = rt.rt_profile_report(ctx, reset=True)
    rt.rt_profile_select(ctx, None)
    rt.rt_profile(ctx, False)
    total_ms = max_over_ranks(sum(times), dev)
    job_bounces = sum_over_ranks(bounces_per_step * args.steps, dev)
    value = job_bounces / (total_ms / 1e3)

    # end-to-end leg: pinned host inputs copied in, results read back, every step
    e2e_times = []
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    out_h = {"H": torch.empty(H.shape, dtype=H.dtype).pin_memory(),
             "gain": torch.empty(gain.shape, dtype=gain.dtype).pin_memory()}
    copy_stream = torch.cuda.Stream(device=dev)
    pin = {"a": torch.empty(1 << 16, dtype=torch.float32).pin_memory(),
           "tau": torch.empty(1 << 14, dtype=torch.float32).pin_memory()}

    def read_H():
        # the 16 MB H(f) goes back on a copy stream while the VJPs and the
        # coverage map still run
        ev = torch.cuda.Event()
        ev.record(stream)
        copy_stream.wait_event(ev)
        with torch.cuda.stream(copy_stream):
            out_h["H"].copy_(H, non_blocking=True)

    # the step's inputs packed into one pinned host buffer (16-byte aligned
    # slots), copied to the device in one transfer per step
    slots, off = {}, 0
    for k, v in host.items():
        nb = v.numel() * v.element_size()
        slots[k] = (off, nb)
        off += (nb + 15) // 16 * 16
    host_blob = torch.empty(off, dtype=torch.uint8).pin_memory()
    for k, v in host.items():
        o, nb = slots[k]
        host_blob[o:o + nb].copy_(v.reshape(-1).view(torch.uint8))
    dev_blob = torch.empty(off, dtype=torch.uint8, device=dev)
    h2d = off   # bytes copied per step (the inputs and their alignment padding)

    def inputs_from(blob):
        return {k: blob[o:o + nb].view(host[k].dtype).view(host[k].shape) for k, (o, nb) in slots.items()}

    # views into the device buffer, made once: every step's copy overwrites
    # the memory they alias
    inp = inputs_from(dev_blob)
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dev_blob.copy_(host_blob, non_blocking=True)
        step(inp, after_freq=read_H)
        out_h["gain"].copy_(gain, non_blocking=True)
        # a and tau into pinned host buffers (grown when a step has more paths)
        na, nt = state["a"].numel(), state["tau"].numel()
        if pin["a"].numel() < na:
            pin["a"] = torch.empty(2 * na, dtype=torch.float32).pin_memory()
        if pin["tau"].numel() < nt:
            pin["tau"] = torch.empty(2 * nt, dtype=torch.float32).pin_memory()
        pin["a"][:na].copy_(state["a"].reshape(-1), non_blocking=True)
        pin["tau"][:nt].copy_(state["tau"].reshape(-1), non_blocking=True)
        stream.wait_stream(copy_stream)
        e1.record(stream)
        e1.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    d2h = (H.numel() * 4 + gain.numel() * 4 + state["a"].numel() * 4 + state["tau"].numel() * 4)
    e2e_ms = max_over_ranks(sum(e2e_times), dev)
    e2e_value = job_bounces / (e2e_ms / 1e3)

    # dominant kernel and its roofline (durations measured in the timed region)
    kern = prof["kernels"]
    hbm, src = peaks()
    probe = traversal_probe(ctx, cov_counts)
    roof = roofline(dom, kern[dom], sbr_counts, cov_counts, hbm, src, probe)
    if roof.get("frac") is not None and dom in breakdown:
        # the same kernel launched alone (the one-stream steps, outside the
        # timed region): in the timed step it shares the SMs with the other
        # stream's kernels, so its launch time there includes theirs
        alone = breakdown[dom][1] / breakdown[dom][0]
        roof["ms_per_launch_alone"] = alone
        roof["frac_alone"] = roof["frac"] * roof["ms_per_launch"] / alone
        roof["alone_note"] = ("launch duration on one stream, outside the timed region; achieved/frac above: "
                              "inside the timed step, beside the other stream's kernels")
    extras = {}
    if rank == 0 and not args.no_extras:
        extras = extra_measurements(tr, scene, dev, args)
        if not args.no_surrogate:
            sweep = [parse_sigma(item) for item in args.sur_sweep.split(",")] if args.sur_sweep else None
            sig, _ = parse_sigma(args.sur_sigma + ":0")
            extras.update(surrogate_measurement(tr, scene, n_tx=args.sur_tx, n_rx=args.sur_rx,
                                                epochs=args.sur_epochs, sigma=sig, sweep=sweep))

    if world > 1:
        dist.barrier()
    if rank != 0:
        return
    cpu = cpu_baseline(scene, tx, rx) if (world == 1 and not args.no_cpu) else None
    line = {
        "metric": "rays*bounces/s",
        "value": value,
        "unit": "rays*bounces/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded city; no dataset)",
        "config": {"workload": WORKLOAD, "tris": int(scene.n_tris), "n_tx": 1, "n_rx": N_RX,
                   "num_rays": N_RAYS, "max_depth": MAX_DEPTH, "subcarriers": N_SC,
                   "coverage_cells": GRID["nx"] * GRID["ny"], "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas{world}"},
        "paths_per_step": state["P"],
        "paths_per_s": state["P"] * args.steps / (total_ms / 1e3),
        "paths_per_s_note": "valid paths of compute_paths per second of the whole timed step",
        "compute_paths_counts": path_stats,
        "ray_bounces_per_step": bounces_per_step,
        "ray_bounces_basis": {"closest_hit": one["closest_hit"], "plane_segments": one.get("plane_segments", 0),
                              "note": "closest-hit queries plus the coverage rays' last segments tested up to "
                                      "the map plane (any hit); untraced last segments are not counted"},
        "gpu_launches": prof["launches"],
        "kernel_ms_per_step": {k: v[1] / n_prof for k, v in sorted(breakdown.items(), key=lambda x: -x[1][1])},
        "kernel_ms_note": f"{n_prof} steps outside the timed region on one stream, every launch bracketed by "
                          "CUDA events",
        "ms_per_step_one_stream": statistics.median(seq_ms),
        "step_note": f"timed step on a high-priority stream; coverage map on the context's second stream "
                     f"(rt_coverage_map_async, short-lived blocks), schedule {args.schedule}: started after the path "
                     f"trace, beside the refinement, CIR, H(f) and the VJPs (after_trace) or when compute_paths "
                     f"returns (after_paths); "
                     "ms_per_step_one_stream: the same calls in order on one stream (median, outside the timed region)",
        "e2e": {"value": e2e_value, "unit": "rays*bounces/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps},
        "roofline": roof,
        "clocks": clk.summary(),
    }
    line.update(extras)
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))


# Algorithmic FP32/ALU operations of the traversal: one octant-selected box
# test per child (6 FMA + 4 min/max + 1 compare = 11), i.e. 22 per node
# record of the default binary layout (its ray-octant copies), 88 per node
# record of the 8-wide layout; one Moller-Trumbore test per triangle record
# (35).
BVH_WIDTH = 2
OPS_PER_NODE = {8: 88, 2: 22}[BVH_WIDTH]
BYTES_PER_NODE = {8: 240, 2: 64}[BVH_WIDTH]
OPS_PER_TRI = 35
# Lane-operation count of the SMs: 152 SMs x 128 lanes x 2070 MHz (one op per
# lane per clock, an FMA counted as one operation); reported beside the
# measured peak, which is what the fraction uses.
ALU_PEAK_GOPS = 152 * 128 * 2.070
# DRAM bytes (read + write) of one k_coverage launch of this workload, from
# the ncu capture summarised in profiles/k_coverage_city_1e6rays.md; set to
# None whenever the kernel changes until it is captured again.
K_COVERAGE_TRAFFIC = 20.60e6
# L1/TEX throughput of the same launch (% of its peak, elapsed) and the
# sector hit rate: the traversal's record reads are served by L1.
K_COVERAGE_L1 = {"l1tex_throughput_pct": 61.3, "l1tex_sector_hit_pct": 85.9, "lts_throughput_pct": 2.8,
                 "source": "profiles/k_coverage_city_1e6rays.md (ncu --set full, one launch)"}


def traversal_probe(ctx, counts, n_tri=4):
    """Measured issue peak of the traversal arithmetic (rt_probe_peak): the
    tracer's own box and triangle tests on register data, in the mix of box
    tests (8 per wide node record, 2 per binary one) to triangle tests the
    counting pass of the coverage kernel measured. Returns (Gop/s, mix)."""
    from paper_2303_11103_gb300 import rt
    per_node = 8 if BVH_WIDTH == 8 else 2
    boxes_per_tri = per_node * counts["nodes"] / max(counts["tris"], 1)
    n_box = max(8, int(round(boxes_per_tri * n_tri / 8.0)) * 8)
    gops = rt.rt_probe_peak(ctx, rt.PROBE_TRAVERSAL, n_box, n_tri) / 1e9
    return gops, {"box_tests": n_box, "triangle_tests": n_tri}


def roofline(name, rec, sbr_counts, cov_counts, hbm, src, probe):
    """Roofline of the dominant kernel: algorithmic work per launch / mean duration.

    The traversal kernels keep the BVH and triangles in L1/L2 (ncu: 94 % L1
    hits, 4.3 MB of DRAM traffic per coverage launch), so their bound is
    instruction issue, not HBM. The peak is measured: rt_probe_peak runs the
    traversal's own slab and triangle tests on register data in the
    kernel's measured mix. The node/triangle record bytes requested are
    reported beside it (`requested_gbs`) for comparison with the HBM peak.
    """
    launches, ms = rec
    per_launch_s = ms / launches / 1e3
    counts = {"k_coverage": cov_counts, "k_sbr": sbr_counts, "k_validate": sbr_counts}.get(name)
    peak, mix = probe
    if counts is None:
        return {"kernel": name, "bound": "alu", "achieved": None, "peak": peak, "unit": "Gop/s",
                "frac": None, "traffic": None, "note": "no algorithmic model for this kernel"}
    ops = counts["nodes"] * OPS_PER_NODE + counts["tris"] * OPS_PER_TRI
    req_bytes = counts["nodes"] * BYTES_PER_NODE + counts["tris"] * 48
    ach = ops / per_launch_s / 1e9
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "Gop/s",
            "frac": ach / peak,
            "traffic": K_COVERAGE_TRAFFIC if name == "k_coverage" else None,
            "l1": K_COVERAGE_L1 if name == "k_coverage" else None,
            "peak_source": "measured: rt_probe_peak(RT_PROBE_TRAVERSAL), "
                           "the traversal's box and Moller-Trumbore tests on register data, "
                           f"{mix['box_tests']} box tests per {mix['triangle_tests']} triangle tests "
                           "(the kernel's counted mix), best of 5",
            "bvh_width": BVH_WIDTH,
            "lane_count_gops": ALU_PEAK_GOPS, "frac_of_lane_count": ach / ALU_PEAK_GOPS,
            "ops_per_launch": ops, "ops_basis": f"{OPS_PER_NODE} per BVH node record ({BVH_WIDTH}-wide), "
                                                f"{OPS_PER_TRI} per triangle record",
            "requested_gbs": req_bytes / per_launch_s / 1e9, "hbm_peak_gbs": hbm, "hbm_peak_source": src,
            "ms_per_launch": per_launch_s * 1e3,
            "nodes_per_query": counts["nodes"] / max(queries(counts), 1),
            "tris_per_query": counts["tris"] / max(queries(counts), 1)}


def queries(counts):
    """Every traversal query of a counting pass: closest hit, any hit and the
    coverage rays' last-segment plane tests."""
    return counts["closest_hit"] + counts["any_hit"] + counts.get("plane_segments", 0)


def extra_measurements(tr, scene, dev, args):
    """Batched coverage maps: 64 Tx x 1e7 rays, max_depth 5, 500 x 500 cells, one launch."""
    import torch
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import scenes as S
    txs = S.rooftop_transmitters(scene, 64)
    rxd = S.Devices(np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), S.V_ISO)
    tr.load_scene(scene)
    tr.set_devices(txs, rxd)
    grid = rt.rt_grid(GRID["x0"], GRID["y0"], GRID["cell"], GRID["h"], GRID["nx"], GRID["ny"])
    gain = torch.empty((64, GRID["ny"], GRID["nx"]), dtype=torch.float32, device=dev)
    hits = torch.empty((64, GRID["ny"], GRID["nx"]), dtype=torch.int32, device=dev)
    n = 10_000_000
    ctx = tr.ctx
    # launch configuration picked by the autotuner (timed on 2e6 rays per Tx)
    tuning_default = rt.rt_get_tuning(ctx)
    rt.rt_autotune(ctx, grid, 5, 2_000_000, gain, hits)
    tuning = rt.rt_get_tuning(ctx)
    # ray segments of one map (counting variant, untimed)
    rt.rt_profile(ctx, rt.PROFILE_COUNT)
    rt.rt_profile_report(ctx, reset=True)
    rt.rt_coverage_map(ctx, grid, 5, n, 0, gain, hits)
    cnt = rt.rt_profile_report(ctx, reset=True)
    rt.rt_profile(ctx, False)
    # the whole map (zeroing + one persistent launch over all 64 Tx) as a CUDA graph, replayed
    stream = torch.cuda.current_stream()
    rt.rt_set_stream(ctx)
    rt.rt_graph_begin(ctx)
    rt.rt_coverage_map(ctx, grid, 5, n, 0, gain, hits)
    rt.rt_graph_end(ctx)
    rt.rt_graph_launch(ctx)
    torch.cuda.synchronize()
    ts = []
    for _ in range(10):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rt.rt_graph_launch(ctx)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    rt.rt_set_tuning(ctx, *tuning_default)
    ext = cir_extensions_measurement(tr, scene, dev)
    ext["freq_response_dense"] = freq_dense_measurement(tr)
    ext["differentiation"] = differentiation_measurement()
    return {**ext, "coverage_map_ms": ms,
            "coverage_map_config": "64 tx x 1e7 rays, max_depth 5, 500x500 cells of 1 m, one persistent launch "
                                   "in a captured CUDA graph, median of 10 replays",
            "coverage_map_tuning": {"block": tuning[0], "chunk": tuning[1], "smem_nodes": tuning[2]},
            "coverage_map_rays_bounces_per_s": (cnt["closest_hit"] + cnt.get("plane_segments", 0)) / (ms / 1e3)}


def cir_extensions_measurement(tr, scene, dev, T=14, fs=1e6):
    """On the city workload's paths: the CIR's time evolution (Sec. II-A
    Listing 3 settings: 1 MHz sampling, 14 steps, Tx at [3, 0, 0] m/s;
    receivers at 1.5 m/s in seeded directions; rt_apply_doppler) and the
    synthetic transmit array of Listing 2 (rt_apply_array); medians of 20
    CUDA-event timings."""
    import torch
    from paper_2303_11103_gb300 import scenes as S
    tx, rx = S.city_devices(scene, n_rx=N_RX)
    tr.load_scene(scene)
    tr.set_devices(tx, rx)
    tr.compute_paths(MAX_DEPTH, N_RAYS)
    a, _ = tr.cir()
    rng = np.random.default_rng(5)
    vr = rng.normal(size=(N_RX, 3))
    vr[:, 2] = 0.0
    vr = torch.as_tensor((1.5 * vr / np.linalg.norm(vr, axis=1, keepdims=True)).astype(np.float32), device=dev)
    vt = torch.tensor([[3.0, 0.0, 0.0]], dtype=torch.float32, device=dev)
    for _ in range(3):
        at = tr.apply_doppler(a, fs, T, vt, vr)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(20):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        at = tr.apply_doppler(a, fs, T, vt, vr)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    # synthetic arrays: the paper's transmit array (8 x 2, spacings 0.7 / 0.5 wavelengths) on the same paths
    from paper_2303_11103_gb300 import rt
    tx_el = torch.as_tensor(rt.planar_array(8, 2, 0.7, 0.5, 299792458.0 / FC), device=dev)
    for _ in range(3):
        ael = tr.apply_array(a, tx_el)
    ts = []
    for _ in range(20):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ael = tr.apply_array(a, tx_el)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return {"doppler": {"paths": int(a.shape[0]), "time_steps": T, "outputs": int(at.numel()), "ms": ms,
                        "config": "city workload paths (1 Tx, 1000 Rx, 1e6 rays, depth 3), fs 1 MHz, Tx [3,0,0] m/s, "
                                  "Rx 1.5 m/s horizontal in seeded directions; velocities resident on the GPU"},
            "diffraction": diffraction_measurement(tr),
            "scattering": scattering_measurement(tr, scene),
            "synthetic_array": {"paths": int(a.shape[0]), "outputs": int(ael.numel()), "ms": statistics.median(ts),
                                "config": "the same paths, Tx planar array 8 x 2 (0.7 / 0.5 wavelengths), "
                                          "dual-polarized TR 38.901 elements, single-element Rx"}}


def _event_ms(fn, reps=20, warm=3):
    """Median CUDA-event time (ms) of fn() on torch's current stream."""
    import torch
    for _ in range(warm):
        fn()
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def freq_dense_measurement(tr, n_pairs=1000, mean_paths=64, K=N_SC):
    """H(f) where it is compute-bound: a seeded dense path list (Poisson(64)
    paths per pair, 1000 pairs, 2 x 2 port pairs, 1024 subcarriers of
    30 kHz) through rt_freq_response_paths; FP32 work = 8 flops per complex
    MAC per (path, subcarrier, port pair) + 6 per twiddle step per (path,
    subcarrier), against the measured FP32 FMA peak (rt_probe_peak)."""
    import torch
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import scenes as S
    dev = tr.device
    off, a, tau = S.dense_path_list(n_pairs, mean_paths, 4, seed=10)
    off_d = torch.as_tensor(off, device=dev)
    a_d = torch.view_as_real(torch.as_tensor(a, device=dev)).contiguous()
    tau_d = torch.as_tensor(tau, device=dev)
    f_d = torch.as_tensor((np.arange(K, dtype=np.float64) - K // 2) * SC_SPACING, device=dev)
    H = torch.empty((n_pairs, 4, K, 2), dtype=torch.float32, device=dev)
    rt.rt_set_stream(tr.ctx)
    ms = _event_ms(lambda: rt.rt_freq_response_paths(tr.ctx, off_d, 4, a_d, tau_d, f_d, H))
    P = int(off[-1])
    flops = P * K * (8 * 4 + 6)
    peak = rt.rt_probe_peak(tr.ctx, rt.PROBE_FFMA) / 1e12
    tf = flops / (ms / 1e3) / 1e12
    return {"pairs": n_pairs, "paths": P, "subcarriers": K, "port_pairs": 4, "ms": ms,
            "path_subcarrier_terms_per_s": P * K * 4 / (ms / 1e3), "tflops": tf,
            "fp32_peak_tflops": peak, "fp32_frac": tf / peak,
            "peak_source": "measured: rt_probe_peak(RT_PROBE_FFMA), 8 chains of FP32 FMA per thread, best of 5",
            "output_bytes": n_pairs * 4 * K * 8,
            "config": "seeded dense path list (scenes.dense_path_list, seed 10): Poisson(64) paths per pair, "
                      "tau U(0.2, 3.3) us, 2x2 port pairs; median of 20 CUDA-event timings"}


def differentiation_measurement(n_rx=256, n_mat=8):
    """The differentiation workload: the seeded city with 8 materials, 1 TR
    38.901 dual-polarized transmitter, 256 receivers, 1e6 rays, max_depth 3.
    Times the path search once, then (median of 20) the forward CIR and the
    backward pass of L = sum_rx 10 log10(sum |a|^2) through rt.CIR (the
    replayed-path VJP kernels), and of the NMSE of H(f) at 128 subcarriers
    through rt.CIR and rt.FreqResponse (Sec. III-A)."""
    import torch
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import scenes as S
    scene = S.city_scene(20, n_materials=n_mat)
    tx, rx = S.city_devices(scene, n_rx=n_rx, tx_antenna=S.TR38901_VH)
    tr = rt.Tracer(0, FC)
    dev = tr.device
    tr.load_scene(scene)
    tr.set_devices(tx, rx)
    t_paths = _event_ms(lambda: tr.compute_paths(MAX_DEPTH, N_RAYS), reps=5, warm=1)
    P = tr.compute_paths(MAX_DEPTH, N_RAYS)
    freqs = torch.as_tensor((np.arange(128, dtype=np.float64) - 64) * SC_SPACING, device=dev)
    rx_of = torch.repeat_interleave(torch.arange(n_rx, device=dev),
                                    torch.diff(tr.paths()["offsets"]).to(dev))
    eps = torch.tensor(scene.materials[:, 0], device=dev, requires_grad=True)
    sig = torch.tensor(scene.materials[:, 1], device=dev, requires_grad=True)
    pos = torch.tensor(tx.pos, device=dev, requires_grad=True)
    ypr = torch.tensor(tx.ypr, device=dev, requires_grad=True)
    with torch.no_grad():
        a0, t0 = rt.CIR.apply(tr, eps, sig, pos, ypr)
        H_ref = rt.FreqResponse.apply(tr, a0, t0, freqs)

    def power_step():
        for p in (eps, sig, pos, ypr):
            p.grad = None
        a, _ = rt.CIR.apply(tr, eps, sig, pos, ypr)
        pw = torch.zeros(n_rx, device=dev).index_add(0, rx_of, (a.abs() ** 2).sum(dim=(1, 2)))
        (10 * torch.log10(pw[pw > 0])).sum().backward()

    def nmse_step():
        for p in (eps, sig, pos, ypr):
            p.grad = None
        a, tau = rt.CIR.apply(tr, eps, sig, pos, ypr)
        H = rt.FreqResponse.apply(tr, a, tau, freqs)
        (((H - H_ref).abs() ** 2).sum() / (H_ref.abs() ** 2).sum()).backward()

    t_pw = _event_ms(power_step)
    t_nm = _event_ms(nmse_step)
    ga = torch.randn((max(P, 1), tr.nrp, tr.ntp), dtype=torch.complex64, device=dev)
    t_vjp = _event_ms(lambda: tr.cir_backward(ga))
    tr.close()
    return {"paths": P, "receivers": n_rx, "materials": n_mat, "parameters": 2 * n_mat + 6,
            "compute_paths_ms": t_paths, "power_db_grad_step_ms": t_pw, "nmse_grad_step_ms": t_nm,
            "cir_vjp_ms": t_vjp,
            "config": "city 4802 tris, 8 materials (eps_r U(2,8), sigma logU(1e-3,1)), 1 TR 38.901 dual-pol Tx, "
                      "256 Rx, 1e6 rays, max_depth 3; grad steps = forward CIR (+ H(f) at 128 subcarriers) + "
                      "loss + backward through the replayed paths; medians of 20 CUDA-event timings"}


def diffraction_measurement(tr):
    """First-order diffraction on the city workload as loaded (1 Tx, 1000 Rx):
    rt_compute_diffraction (all pairs x all wedges) and rt_diffraction_cir,
    medians of 10 host-timed calls (the search reads its path count back)."""
    import torch
    tr.compute_diffraction()
    tr.diffraction_cir()
    torch.cuda.synchronize()
    t_find, t_cir = [], []
    for _ in range(10):
        t0 = time.perf_counter()
        P = tr.compute_diffraction()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        a, _ = tr.diffraction_cir()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_find.append((t1 - t0) * 1e3)
        t_cir.append((t2 - t1) * 1e3)
    faces, _ = tr.wedges()
    # the diffracted part of the step's 500 x 500 coverage map (every cell centre against every wedge)
    tr.coverage_map_diffraction(GRID, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gd = tr.coverage_map_diffraction(GRID, 0)
    torch.cuda.synchronize()
    t_map = (time.perf_counter() - t0) * 1e3
    cells = GRID["nx"] * GRID["ny"]
    return {"wedges": int(faces.shape[0]), "pairs": int(tr.n_pairs), "diffracted_paths": int(P),
            "find_ms": statistics.median(t_find), "cir_ms": statistics.median(t_cir),
            "candidates_per_s": int(faces.shape[0]) * int(tr.n_pairs) / (statistics.median(t_find) / 1e3),
            "map_ms": t_map, "map_cells": cells, "map_cells_with_diffraction": int((gd > 0).sum().item()),
            "map_candidates_per_s": int(faces.shape[0]) * cells / (t_map / 1e3)}


def scattering_measurement(tr, scene, n_rays=100_000, S_m=0.3):
    """First-order diffuse scattering on the city workload as loaded (1 Tx,
    1000 Rx, every material S = 0.3): rt_scattering_gain over n_rays lattice
    rays, every ray's hit against every receiver; median of 5 CUDA-event
    timings."""
    import torch
    tr.set_scattering(np.full(len(scene.materials), S_m, np.float32))
    g = tr.scattering_gain(n_rays)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = tr.scattering_gain(n_rays)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    return {"rays": n_rays, "receivers": int(tr.n_pairs), "ms": ms,
            "ray_receiver_pairs_per_s": n_rays * int(tr.n_pairs) / (ms / 1e3),
            "links_with_scattering": int((g.sum(dim=(1, 2)) > 0).sum().item())}


def surrogate_measurement(tr, scene, n_tx=40_000, n_rx=250, num_rays=200_000, max_depth=3, epochs=40,
                          n_query=100_000_000, n_heldout=100_000, batch=16384, lr=1.5e-3, oversample=4,
                          sigma=(0.25, 4.0, 0.0, 0.0), sweep=None):
    """Learned surrogate on the city (config S): tracer labels for 1e7 (tx, rx)
    pairs over n_tx transmitters on rooftops (continuous positions along roof
    edges, scenes.surrogate_sites, seed 4), training, and the error against
    the tracer on 1e5 pairs of transmitters the network never saw (seed 14),
    beside new receivers of the training sites; q/s against the tracer.
    sweep: list of (sigma, epochs) settings to train and evaluate as well."""
    import torch
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import surrogate as SG
    from paper_2303_11103_gb300 import scenes as S
    t0 = time.perf_counter()
    tr.load_scene(scene)
    tx, rx = S.surrogate_sites(scene, n_tx, n_rx, seed=4)
    x, t = SG.tracer_labels(tr, tx, rx, num_rays, max_depth)
    n_new = max(1, n_heldout // n_rx)
    txn, rxn = S.surrogate_sites(scene, n_new, n_rx, seed=14)
    xn, tn = SG.tracer_labels(tr, txn, rxn, num_rays, max_depth)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    n = x.shape[0]
    g = torch.Generator(device=x.device).manual_seed(11)
    perm = torch.randperm(n, generator=g, device=x.device)
    held, train_idx = perm[:n_heldout], perm[n_heldout:]
    lo = np.array([-250, -250, 0, -250, -250, 0], np.float32)
    hi = np.array([250, 250, 70, 250, 250, 3], np.float32)

    def fit(sig, ep):
        """sig: isotropic Fourier scale, or (sigma_tx, sigma_rx, rel_frac, sigma_rel)."""
        iso = not isinstance(sig, (tuple, list))
        sur = rt.Surrogate(lo, hi, n_freq=32, width=256, n_hidden=8, sigma=sig if iso else 1.0, seed=1)
        if not iso:
            SG.set_fourier(sur, *sig, seed=1)
        t1 = time.perf_counter()
        losses = SG.train(sur, x[train_idx], t[train_idx], epochs=ep, batch=batch, lr=lr, oversample=oversample)
        torch.cuda.synchronize()
        return sur, losses, time.perf_counter() - t1

    sweep_out = []
    for sig, ep in (sweep or []):
        s2, l2, ts2 = fit(sig, ep)
        sweep_out.append({"fourier_scales": sig, "epochs": ep, "train_s": ts2, "final_loss": l2[-1],
                          "new_sites": SG.evaluate(s2, xn, tn), "seen_sites": SG.evaluate(s2, x[held], t[held])})
        s2.close()
    sur, losses, t_train = fit(sigma, epochs)
    ev_new = SG.evaluate(sur, xn, tn)
    ev_seen = SG.evaluate(sur, x[held], t[held])
    q_sur, ms_sur = SG.time_inference(sur, n_query, lo, hi, reps=2)
    # tracer queries: one site with 1000 receivers per call (the city step's
    # receiver count), and with all of the site's receivers in one call (the
    # ray trace shared by the most receivers: the tracer's best case)
    # one site with 1000 receivers of its own (the training sites have n_rx each)
    txq, rxq = S.surrogate_sites(scene, 1, 1000, seed=24)
    q_tr, s_tr = SG.time_tracer_queries(tr, txq, rxq, num_rays, max_depth, n_rx=1000)
    q_tr_all, s_tr_all = SG.time_tracer_queries(tr, tx, rx, num_rays, max_depth)
    sur.close()
    out = {"surrogate": {
        "train_pairs": int(len(train_idx)), "epochs": epochs, "batch": batch, "lr": lr,
        "fourier_scales": sigma if not isinstance(sigma, tuple) else
        {"sigma_tx": sigma[0], "sigma_rx": sigma[1], "rel_frac": sigma[2], "sigma_rel": sigma[3]},
        "path_pair_oversample": oversample, "final_loss": losses[-1],
        "label_s": t_label, "train_s": t_train,
        "heldout": ev_new,
        "heldout_note": "headline: 1e5 pairs of 25 transmitter sites not in training (independent draw of "
                        "rooftop-edge positions); rms_db_all_path_pairs is over every held-out pair with a path, "
                        "rms_db_answered over those the network answers (|logit| >= margin)",
        "heldout_sites": n_new,
        "heldout_seen_sites": ev_seen,
        "queries": n_query, "infer_ms": ms_sur, "queries_per_s": q_sur,
        "tracer_queries_per_s": q_tr, "speedup_vs_tracer": q_sur / q_tr,
        "tracer_note": "compute_paths + cir + pair gain at the label settings, one site with 1000 receivers per call",
        "tracer_queries_per_s_site_rx": q_tr_all, "speedup_vs_tracer_site_rx": q_sur / q_tr_all,
        "tracer_site_rx_note": f"the same with one training site's {n_rx} receivers per call",
        "config": f"city 4802 tris; {n_tx} rooftop Tx (1 m outside a roof-edge point, mast 1-5 m) x {n_rx} street "
                  f"Rx within 100 m; labels: {num_rays} rays, max_depth {max_depth}; MLP 64 Fourier features, "
                  f"8 x 256 ReLU, BF16 tcgen05"}}
    if sweep_out:
        out["surrogate"]["sweep"] = sweep_out
    return out


def parse_sigma(item: str):
    """'sigma:epochs' (isotropic Fourier scale) or 'sigma_tx:sigma_rx:rel_frac:sigma_rel:epochs'."""
    v = [float(x) for x in item.split(":")]
    return (v[0] if len(v) == 2 else tuple(v[:4])), int(v[-1])


def cpu_baseline(scene, tx, rx, seconds=15.0):
    """The FP64 oracle on the host cores: shooting and bouncing of a ray sample."""
    from oracle import oracle as O
    osc = O.make_scene(scene)
    cores = O.nthreads()
    n = 2000
    t0 = time.perf_counter()
    ids = np.arange(n, dtype=np.int64) * (N_RAYS // n)
    hits, _ = O.trace_sbr(osc, tx.pos[0], N_RAYS, MAX_DEPTH, ids)
    dt = time.perf_counter() - t0
    if dt < seconds / 4:
        n = int(n * seconds / max(dt, 1e-3) / 1.2)
        ids = (np.arange(n, dtype=np.int64) * (N_RAYS / n)).astype(np.int64)
        t0 = time.perf_counter()
        hits, _ = O.trace_sbr(osc, tx.pos[0], N_RAYS, MAX_DEPTH, ids)
        dt = time.perf_counter() - t0
    queries = int(n + (hits[:, :-1] >= 0).sum())
    return {"value": queries / dt, "unit": "rays*bounces/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} of the {N_RAYS} lattice rays of the city workload, max_depth {MAX_DEPTH}, "
                      f"brute-force FP64 closest hit ({queries} queries in {dt:.1f} s)"}


# ------------------------------------------------------------ reference arm
def run_reference(args):
    world, rank, local = dist_init()
    if rank != 0:
        return
    from paper_2303_11103_gb300 import scenes as S
    scene = S.city_scene(20)
    tx, rx = S.city_devices(scene, n_rx=N_RX)
    # each step a bounded sample, sized so that the whole run stays within a few minutes
    per_step = max(0.5, min(6.0, 150.0 / max(args.steps, 1)))
    for _ in range(args.warmup):
        cpu_baseline(scene, tx, rx, seconds=min(2.0, per_step))
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(scene, tx, rx, seconds=per_step))
    total = time.perf_counter() - t_all
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": "rays*bounces/s", "value": v, "unit": "rays*bounces/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded city; no dataset)",
            "config": {"workload": WORKLOAD, "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": "rays*bounces/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "rays*bounces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_kernel_case(args):
    """One kernel of the step on its own (for ncu captures):
    `--only coverage|paths|freq|freq_dense|tail|scatter|mlp_infer|mlp_train`;
    freq_dense = H(f) on the seeded dense path list; tail =
    compute_paths, cir, H(f) and both VJPs (the calls after the ray trace);
    scatter = first-order diffuse scattering (every material S = 0.3) over
    --rays lattice rays to the 1000 receivers."""
    import torch
    from paper_2303_11103_gb300 import rt
    from paper_2303_11103_gb300 import scenes as S
    if args.only.startswith("mlp"):
        # surrogate at its configured size (64 features, 8 x 256), random init
        lo, hi = (-250.0, -250.0, 0.0, -250.0, -250.0, 0.0), (250.0, 250.0, 70.0, 250.0, 250.0, 70.0)
        sur = rt.Surrogate(lo, hi, n_freq=32, width=256, n_hidden=8, sigma=1.0, seed=0)
        g = torch.Generator(device="cuda").manual_seed(1)
        lo_t, hi_t = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
        x = lo_t + (hi_t - lo_t) * torch.rand((args.queries, 6), generator=g, device="cuda")
        t = torch.stack([torch.ones(args.queries, device="cuda"), torch.full((args.queries,), -90.0, device="cuda")], 1)
        acc = torch.zeros(1, device="cuda")
        for _ in range(args.warmup + args.steps):
            if args.only == "mlp_infer":
                sur.infer(x)
            else:   # one optimisation step on a training batch of 8192 pairs
                sur.train_step(x[:8192], t[:8192], 1e-4, acc)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.only, "queries": args.queries, "launches": args.warmup + args.steps}))
        return
    if args.only == "freq_dense":
        # H(f) on the seeded dense path list (64 paths per pair, 1000 pairs, 2 x 2 ports, 1024 subcarriers)
        tr = rt.Tracer(0, FC)
        off, a, tau = S.dense_path_list(1000, 64, 4, seed=10)
        off_d = torch.as_tensor(off, device="cuda")
        a_d = torch.view_as_real(torch.as_tensor(a, device="cuda")).contiguous()
        tau_d = torch.as_tensor(tau, device="cuda")
        f_d = torch.as_tensor((np.arange(N_SC, dtype=np.float64) - N_SC // 2) * SC_SPACING, device="cuda")
        H = torch.empty((1000, 4, N_SC, 2), dtype=torch.float32, device="cuda")
        rt.rt_set_stream(tr.ctx)
        for _ in range(args.warmup + args.steps):
            rt.rt_freq_response_paths(tr.ctx, off_d, 4, a_d, tau_d, f_d, H)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.only, "paths": int(off[-1]), "launches": args.warmup + args.steps}))
        return
    scene = S.city_scene(20)
    tx, rx = S.city_devices(scene, n_rx=N_RX)
    tr = rt.Tracer(0, FC)
    tr.load_scene(scene)
    tr.set_devices(tx, rx)
    if args.only in ("freq", "tail"):
        tr.compute_paths(MAX_DEPTH, args.rays)
        a, tau = tr.cir_raw()
        freqs = (np.arange(N_SC, dtype=np.float64) - N_SC // 2) * SC_SPACING
    if args.only == "scatter":
        tr.set_scattering(np.full(len(scene.materials), 0.3, np.float32))
    for _ in range(args.warmup + args.steps):
        if args.only == "coverage":
            g, h = tr.coverage_map(GRID, MAX_DEPTH, args.rays, 0)
        elif args.only == "freq":
            tr.freq_response_raw(a, tau, freqs)
        elif args.only == "tail":
            tr.compute_paths(MAX_DEPTH, args.rays)
            ac, tauc = tr.cir()
            Hc = tr.freq_response(ac, tauc, freqs)
            ga, gt = tr.freq_response_backward(ac, tauc, freqs, Hc)
            tr.cir_backward(ga, gt)
        elif args.only == "scatter":
            tr.scattering_gain(args.rays)
        else:
            tr.compute_paths(MAX_DEPTH, args.rays)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.only, "rays": args.rays, "launches": args.warmup + args.steps}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", choices=["coverage", "paths", "freq", "freq_dense", "tail", "scatter", "mlp_infer",
                                       "mlp_train"], default=None,
                    help="run one kernel case of the step (profiling)")
    ap.add_argument("--rays", type=int, default=N_RAYS)
    ap.add_argument("--queries", type=int, default=1 << 20, help="surrogate queries (--only mlp_*)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--schedule", default="after_trace", choices=["after_trace", "after_paths", "with_trace"],
                    help="when the coverage map starts on the second stream: after the path trace (beside the "
                         "candidate refinement), after compute_paths returns (beside CIR, H(f) and the VJPs), "
                         "or before compute_paths (beside the path trace too)")
    ap.add_argument("--side-blocks", type=int, default=0,
                    help="coverage map on the second stream: 0 = short-lived blocks that free SM slots for the "
                         "context's (higher-priority) stream; N > 0 = one persistent launch with N blocks per SM")
    ap.add_argument("--sur-tx", type=int, default=40_000, help="surrogate training transmitter sites")
    ap.add_argument("--sur-rx", type=int, default=250, help="surrogate receivers per transmitter site")
    ap.add_argument("--sur-epochs", type=int, default=40)
    ap.add_argument("--sur-sigma", default="0.25:4:0:0",
                    help="Fourier scales of the surrogate: 'sigma' (all coordinates) or "
                         "'sigma_tx:sigma_rx:rel_frac:sigma_rel'")
    ap.add_argument("--sur-sweep", default="",
                    help="extra surrogate settings to train and evaluate, comma-separated 'sigma:epochs' or "
                         "'sigma_tx:sigma_rx:rel_frac:sigma_rel:epochs' (e.g. 4:40,1:8:0.5:8:40)")
    args = ap.parse_args()
    if args.only:
        run_kernel_case(args)
        return
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
