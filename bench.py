"""Benchmark: MLUPS and HBM-roofline fraction of the fused FP32 step on the
4000 x 4000 cavity with 4800 hot disks of radius 10 (the paper's
sedimentation benchmark shape, Sec. 2.6.3 / Sec. 3).

One bench step = one full time step of the method: link gather + curved
bounce-back + momentum exchange, particle update, owner map and flags, and the
fused stream-collide-refill over all 16 M nodes.  MLUPS counts every node,
solid ones included (the paper's definition, Sec. 3).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank runs an independent replica (the method is
not sharded here) and rank 0 prints the whole-job MLUPS over the slowest
rank's time.  ``--impl reference`` times the FP64 CPU oracle on the host cores
on a bounded 1000 x 1000 crop of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2308_16597_gb300 import metrics, workloads as W  # noqa: E402

METRIC = "MLUPS"
# plane storage: lbm_params.storage code and bytes per stored population
STORAGE_CODES = {"fp32": 0, "bf16": 1, "fp16": 2}
STORAGE_BYTES = {"fp32": 4, "bf16": 2, "fp16": 2}
UNIT = "MLUPS"
CROP = 1000


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job MLUPS: lattice updates of all ranks over the slowest rank's time."""
    return metrics.mlups(nodes_per_rank * world, 1, steps, max_seconds)


def crop(wl: W.Workload, size: int) -> W.Workload:
    """A size x size cavity holding the disks of the workload's lower-left
    window that lies in the seeded band (same density, radius, parameters)."""
    y0 = wl.ny - size - 1
    p = wl.particles
    r = p["r"]
    keep = (p["x"] - r > 4) & (p["x"] + r < size - 5) & (p["y"] - r > y0 + 4) & \
           (p["y"] + r < y0 + size - 5)
    parts = p[keep].copy()
    parts["y"] -= y0
    return W.Workload("%s_crop%d" % (wl.name, size), W.cavity(size, size), parts, dict(wl.params))


# ------------------------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (ctypes, read-only
    queries) every `period` seconds by a background thread, so that samples
    fall inside timed regions of a few milliseconds; `window()` marks the
    host-side span of each timed region and `summary()` keeps only the
    samples inside them.  The device is found by its PCI address."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, dev, period: float = 5e-4):
        import ctypes
        import threading
        self.period, self.samples, self.windows = period, [], []
        self.ok, self.max_mhz, self.err = False, None, None
        self._stop = threading.Event()
        self._thread = None
        try:
            import torch
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            pr = torch.cuda.get_device_properties(dev)
            bus = getattr(pr, "pci_bus_id", None)
            rc = -1
            if bus is not None:
                bid = "%08x:%02x:%02x.0" % (getattr(pr, "pci_domain_id", 0), bus, getattr(pr, "pci_device_id", 0))
                rc = lib.nvmlDeviceGetHandleByPciBusId_v2(bid.encode(), ctypes.byref(h))
            if rc != 0:
                cnt = ctypes.c_uint(0)
                lib.nvmlDeviceGetCount_v2(ctypes.byref(cnt))
                if cnt.value != 1 or lib.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    raise OSError("no NVML handle for the device")
            mx = ctypes.c_uint(0)
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            self.lib, self.h, self.ok = lib, h, True
        except Exception as e:  # noqa: BLE001 - the line then says why there are no samples
            self.err = str(e)

    def _run(self):
        import ctypes
        mhz, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while not self._stop.is_set():
            t = time.perf_counter()
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) == 0 and \
                    self._reasons(self.h, ctypes.byref(rs)) == 0:
                self.samples.append((t, float(mhz.value), int(rs.value)))
            time.sleep(self.period)

    def start(self):
        if self.ok:
            import threading
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()

    def window(self, t0: float, t1: float):
        self.windows.append((t0, t1))

    def summary(self) -> dict:
        if not self.ok:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["NVML unavailable: %s" % self.err],
                    "samples": 0}
        inside = [x for x in self.samples if any(a <= x[0] <= b for a, b in self.windows)]
        reasons = sorted({name for _, _, r in inside for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median([m for _, m, _ in inside]) if inside else None,
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples": len(inside),
                "source": "NVML every %.1f ms inside the timed windows" % (self.period * 1e3)}


def timed_windows(step, record, dev, steps: int, windows: int, sampler, world: int = 1):
    """`windows` back-to-back timed regions of exactly `steps` steps each,
    every one bracketed by a barrier (N > 1) and a device synchronisation on
    both sides and timed with CUDA events on the launching stream (`record`
    records an event there); returns the milliseconds of each region."""
    import torch
    out = []
    for _ in range(windows):
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        record(e0)
        step(steps)
        record(e1)
        torch.cuda.synchronize(dev)
        sampler.window(t0, time.perf_counter())
        if world > 1:
            dist.barrier()
        out.append(e0.elapsed_time(e1))
    return out


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.txt)
    for this kernel and workload, if it was taken on the current source of the
    kernel's file; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#") or len(f) < 5 or f[0] != kernel or f[1] != workload:
            continue
        src = os.path.join(ROOT, "paper_2308_16597_gb300", "csrc", f[2])
        digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return int(f[4]) if digest == f[3] else None
    return None


# ------------------------------------------------------------------------------------ oracle
def cpu_baseline(wl: W.Workload, seconds: float = 12.0, max_steps: int = 400):
    """FP64 oracle on the host cores, on the CROP x CROP sample of the workload:
    oracle steps until about `seconds` of CPU work (at most max_steps)."""
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import oracle.oracle as orc
    sample = crop(wl, CROP)
    ref = orc.Oracle(sample.domain, sample.particles, sample.params)
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps and (time.perf_counter() - t0) < seconds:
        ref.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": metrics.mlups(sample.nx, sample.ny, steps, dt), "unit": UNIT,
            "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
            "sample": "%dx%d crop of the %s workload with %d particles, %d FP64 oracle steps"
                      % (sample.nx, sample.ny, wl.name, len(sample.particles), steps),
            "seconds": dt}


def reference_sample(wl, steps: int, budget_s: float = 90.0) -> W.Workload:
    """Crop of the workload sized so that `steps` oracle steps take about
    budget_s on this host (probed with one step of a 256 x 256 crop)."""
    import oracle.oracle as orc
    probe = crop(wl, 256)
    ref = orc.Oracle(probe.domain, probe.particles, probe.params)
    t0 = time.perf_counter()
    ref.step(1)
    per_node = (time.perf_counter() - t0) / (256 * 256)
    side = int((budget_s / max(steps, 1) / per_node) ** 0.5) // 8 * 8
    return crop(wl, max(128, min(CROP, side)))


def run_reference(args, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(threads))
    import oracle.oracle as orc
    sample = reference_sample(wl, args.steps + args.warmup)
    ref = orc.Oracle(sample.domain, sample.particles, sample.params)
    ref.step(args.warmup)
    t0 = time.perf_counter()
    ref.step(args.steps)
    dt = time.perf_counter() - t0
    v = metrics.mlups(sample.nx, sample.ny, args.steps, dt)
    sample_desc = "%dx%d crop of %s (%d particles), one FP64 oracle step per bench step" % (
        sample.nx, sample.ny, wl.name, len(sample.particles))
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": sample_desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_of(wl, args):
    p = wl.particles
    es = 4 if getattr(args, "storage", "fp32") == "fp32" else 2
    state_gb = 2 * 14 * ((wl.nx + 31) // 32 * 32) * wl.ny * es / 1e9  # both distribution buffers
    return {"workload": wl.name, "nx": wl.nx, "ny": wl.ny, "particles": int(len(p)),
            "radius": float(p["r"][0]) if len(p) else None,
            "minor_axis": float(p["b"][0]) if len(p) and p["b"][0] > 0 else None,
            "storage": getattr(args, "storage", "fp32"), "links": getattr(args, "links", "index"),
            # the kernel that ran: FP32 storage always takes one block per row tile
            "stream_collide": ("one_block_per_tile" if getattr(args, "storage", "fp32") == "fp32"
                               or getattr(args, "stream_collide", "staged") == "unstaged" else "staged"),
            "density_ratio": float(p["rho"][0]) if len(p) else None,
            "parallelism": "replicas%d" % args.gpus,
            "l2": "no flush: each step reads one distribution buffer and writes the other, %.2f GB "
                  "together, %.1fx the 129 MB L2" % (state_gb, state_gb / 0.129)}


# ------------------------------------------------------------------------------------ ours
def kernel_pass(sim, steps: int) -> dict:
    """Per-kernel times: `steps` steps launched directly, one kernel at a
    time, each bracketed by CUDA events on the launching stream."""
    sim.kernel_timing(True)
    sim.step(3)
    sim.sync()
    sim.kernel_times()  # reset
    sim.step(steps)
    kt = sim.kernel_times()
    sim.kernel_timing(False)
    sim.sync()
    return kt


def storage_leg(wl, storage: str, args, dev, stream, sampler) -> dict:
    """The same workload with the 14 planes stored as `storage`: MLUPS of the
    graph-replayed step (median of the timed windows) and the stream-collide
    kernel against the copy bandwidth on its algorithmic bytes per update."""
    from paper_2308_16597_gb300 import lbm
    sim = lbm.Simulation(wl.domain, wl.particles, wl.params, stream=stream, storage=STORAGE_CODES[storage])
    sim.step(args.warmup)
    sim.sync()
    ms = timed_windows(sim.step, lambda e: e.record(stream), dev, args.steps, args.windows, sampler)
    kt = kernel_pass(sim, args.steps)
    sim.close()
    med = statistics.median(ms) / args.steps
    nodes = wl.nx * wl.ny
    B_LU = metrics.bytes_per_update(STORAGE_BYTES[storage])
    peak = measured_peaks()["hbm_gbs"]
    sc_ms = kt["stream_collide"][0] / max(kt["stream_collide"][1], 1)
    return {"value": nodes / (med / 1e3) / 1e6, "unit": UNIT, "ms_per_step": med,
            "bytes_per_update": B_LU,
            "whole_step_hbm_frac": B_LU * nodes / (med / 1e3) / 1e9 / peak,
            "stream_collide": {"avg_launch_ms": sc_ms, "achieved_gbs": B_LU * nodes / (sc_ms / 1e3) / 1e9,
                               "frac": B_LU * nodes / (sc_ms / 1e3) / 1e9 / peak}}


def run_ours(args, wl):
    import torch
    from paper_2308_16597_gb300 import build as B, lbm

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)
    nodes = wl.nx * wl.ny
    storage = STORAGE_CODES[args.storage]
    flags = lbm.LBM_FLAG_DIRECT_LINKS if args.links == "direct" else 0
    if args.stream_collide == "unstaged":
        flags |= lbm.LBM_FLAG_SC_UNSTAGED
    if getattr(args, "overlap", False):
        flags |= lbm.LBM_FLAG_OVERLAP
    sampler = NvmlSampler(dev)
    with torch.cuda.stream(stream):
        sim = lbm.Simulation(wl.domain, wl.particles, wl.params, stream=stream, storage=storage, flags=flags)
        sim.step(args.warmup)
        sim.sync()
        clocks = ClockSampler(local)
        clocks.start()
        sampler.start()
        time.sleep(0.4)
        # headline: `windows` regions of exactly K steps each, replayed from
        # the captured CUDA graphs; the value is the median region
        launches0 = sim.launch_count()
        win_ms = timed_windows(sim.step, lambda e: e.record(stream), dev, args.steps, args.windows, sampler, world)
        launches = (sim.launch_count() - launches0) // args.windows
        ktimes = kernel_pass(sim, args.steps)
        smi = clocks.stop()
    ms = statistics.median(win_ms)
    max_ms = max_over_ranks(ms, world, dev)
    value = aggregate_mlups(nodes, args.steps, world, max_ms / 1e3)

    # end to end through the C ABI with host buffers: init from host particles,
    # every step the particle state read back to pinned host memory, the
    # fields read back at the end
    e2e = None
    if not args.no_e2e:
        del sim
        torch.cuda.empty_cache()
        pinned_p = torch.empty(len(wl.particles) * lbm.PARTICLE_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        pview = pinned_p.numpy().view(lbm.PARTICLE_DTYPE)
        fields = [torch.empty((wl.ny, wl.nx), dtype=torch.float32, pin_memory=True)
                  for _ in range(4)]
        params = lbm.make_params(**dict(wl.params, storage=storage, flags=flags))
        dom = lbm.make_domain(**wl.domain)
        parts = lbm.pack_particles(wl.particles)
        ws_bytes = lbm.lbm_query_footprint(dom, parts, params)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        e2e_steps = max(1, args.steps)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h = lbm.lbm_init(dom, parts, params, ws.data_ptr(), ws_bytes, stream.cuda_stream)
        lbm.lbm_sync(h)
        t_init = time.perf_counter()
        for _ in range(e2e_steps):
            lbm.lbm_step(h, 1)
            # each step's particle states to page-locked host memory, the
            # copy overlapping the next step's kernels
            lbm.lbm_get_particles_async(h, pview)
        lbm.lbm_sync(h)
        t_steps = time.perf_counter()
        lbm.lbm_get_fields(h, *[f.data_ptr() for f in fields], 0)
        t1 = time.perf_counter()
        lbm.lbm_destroy(h)
        e2e_s = max_over_ranks(t1 - t0, world, dev)
        pbytes = len(wl.particles) * lbm.PARTICLE_DTYPE.itemsize
        e2e = {"value": aggregate_mlups(nodes, e2e_steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": pbytes / e2e_steps,
               "d2h_bytes_per_step": pbytes + 4 * 4 * nodes / e2e_steps,
               "steps": e2e_steps,
               "seconds": {"init": t_init - t0, "steps": t_steps - t_init, "fields_readback": t1 - t_steps},
               "includes": "lbm_init from host particles (raster, initial collision, graph capture), per "
                           "step lbm_step(1) + lbm_get_particles_async to pinned host (the copy overlaps the "
                           "next step), final lbm_sync and lbm_get_fields of rho-1, ux, uy, T (%d MB) to "
                           "host; at %d steps the init and the field read-back are a large share of the "
                           "time (see seconds)" % (16 * nodes // 1000000, e2e_steps)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # one lattice update per step, in one pass or in a far-tile pass beside
    # the particle kernels plus a near-tile pass after them
    k_ms, k_n = ktimes["stream_collide"]
    k_ms += ktimes.get("stream_collide_near", (0.0, 0))[0]
    avg_s = k_ms / 1e3 / max(k_n, 1)
    B_LU = metrics.bytes_per_update(STORAGE_BYTES[args.storage])
    peaks = measured_peaks()
    achieved = B_LU * nodes / avg_s / 1e9
    traffic = profiled_traffic("stream_collide" if args.storage == "fp32" else "stream_collide_" + args.storage,
                               wl.name)
    step_ms = max_ms / args.steps
    direct_ms = sum(v[0] for v in ktimes.values()) / args.steps
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": "k_stream_collide" + (" (far-tile + near-tile passes of one step)"
                                                if ktimes.get("stream_collide_near", (0.0, 0))[1] else ""),
                "algorithmic_bytes_per_launch": B_LU * nodes,
                "avg_launch_ms": avg_s * 1e3, "peak_source": peaks["source"] + " (hbm_gbs)",
                "kernel_times_from": "a second pass of the same number of steps, launched directly with "
                                     "CUDA events around every kernel: its kernels sum to %.4f ms per step "
                                     "against %.4f ms per graph-replayed step (the boundary kernel runs "
                                     "beside stream-collide in the graph, after it here)" % (direct_ms, step_ms)}
    per_kernel = {k: {"ms_per_step": v[0] / max(v[1], 1), "launches": v[1],
                      "share": v[0] / max(sum(x[0] for x in ktimes.values()), 1e-12)}
                  for k, v in ktimes.items() if v[1]}
    clk = sampler.summary()
    clk["nvidia_smi"] = smi
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_of(wl, args), timed_windows=args.windows),
            "windows_ms_per_step": [w / args.steps for w in win_ms],
            "roofline": roofline, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk, "kernels": per_kernel,
            "particle_part_ms_per_step": sum(v["ms_per_step"] for k, v in per_kernel.items()
                                             if k in ("link_gather_bb_force", "particle_update", "node_flags")),
            "whole_step_hbm_frac": B_LU * nodes / (step_ms / 1e3) / 1e9 / peaks["hbm_gbs"]}
    if world == 1 and not args.no_extra and args.workload == "cavity4000" and args.storage == "fp32":
        with torch.cuda.stream(stream):
            sampler.windows.clear()
            line["reduced"] = {st: storage_leg(wl, st, args, dev, stream, sampler) for st in ("bf16", "fp16")}
            line["reduced"]["clocks"] = sampler.summary()
            sampler.stop()
        line["ensemble"] = run_ensemble(args, summary=True)
        line["served"] = run_served(args, summary=True)
        bf16 = argparse.Namespace(**dict(vars(args), storage="bf16"))
        line["ensemble_bf16"] = run_ensemble(bf16, summary=True)
        line["served_bf16"] = run_served(bf16, summary=True)
    else:
        sampler.stop()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------ batched ensemble
# lbm_batch_autotune's choices: three block shapes of the one-block-per-tile
# kernel, and (BF16 / FP16 storage) the staged kernel over the batch
TILE_NAMES = ["128x1", "64x2", "32x4", "staged"]
TILE_KERNELS = ["k_stream_collide_batch"] * 3 + ["k_stream_collide_staged_batch"]


def run_ensemble(args, summary: bool = False):
    """64 uneven cavities stepped as one batch (one graph per step, tile shape
    from the autotuner): aggregate MLUPS over all instances.  summary: called
    from the headline run on one GPU (FP32 and BF16, K steps in the
    headline's number of windows); returns the key's dict instead of
    printing a line."""
    import torch
    from paper_2308_16597_gb300 import build as B, lbm

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if summary:
        world, rank = 1, 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wls = W.ensemble(64, seed=4)
    storage = STORAGE_CODES[args.storage]
    nodes = sum(w.nx * w.ny for w in wls)
    stream = torch.cuda.Stream(device=dev)
    sampler = NvmlSampler(dev)
    with torch.cuda.stream(stream):
        t_init0 = time.perf_counter()
        sims = [lbm.Simulation(w.domain, w.particles, w.params, stream=stream, storage=storage) for w in wls]
        batch = lbm.Batch(sims, stream=stream)
        torch.cuda.synchronize(dev)
        t_init = time.perf_counter() - t_init0
        tile = batch.autotune(3)
        batch.step(args.warmup)
        batch.sync()
        clocks = ClockSampler(local)
        clocks.start()
        sampler.start()
        time.sleep(0.4)
        l0 = batch.launch_count()
        win_ms = timed_windows(batch.step, lambda e: e.record(stream), dev, args.steps, args.windows, sampler, world)
        ms = statistics.median(win_ms)
        launches = (batch.launch_count() - l0) // args.windows
        # end to end: every instance's particles and fields read back to the host
        t0 = time.perf_counter()
        d2h = 0
        for s in sims:
            s.particles()
            f = s.fields()
            d2h += len(s._parts) * lbm.PARTICLE_DTYPE.itemsize + sum(a.nbytes for a in f)
        t_read = time.perf_counter() - t0
        smi = clocks.stop()
        sampler.stop()
        clk = dict(sampler.summary(), nvidia_smi=smi)
        batch.sync()
        sc_ms = batch.tuned_ms
        batch.close()
        for s in sims:
            s.close()
    max_ms = max_over_ranks(ms, world, dev)
    value = aggregate_mlups(nodes, args.steps, world, max_ms / 1e3)
    B_LU = metrics.bytes_per_update(STORAGE_BYTES[args.storage])
    peaks = measured_peaks()
    achieved = B_LU * nodes / (sc_ms / 1e3) / 1e9
    if summary:
        return {"workload": "ensemble64_seed4", "instances": len(wls), "nodes": nodes,
                "particles": int(sum(len(w.particles) for w in wls)), "storage": args.storage,
                "value": value, "unit": UNIT, "ms_per_step": max_ms / args.steps,
                "windows_ms_per_step": [w / args.steps for w in win_ms],
                "tile": TILE_NAMES[tile], "gpu_launches_per_window": int(launches),
                "whole_step_hbm_frac": B_LU * nodes / (max_ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"],
                "stream_collide": {"kernel": TILE_KERNELS[tile], "avg_launch_ms": sc_ms,
                                   "achieved_gbs": achieved, "frac": achieved / peaks["hbm_gbs"],
                                   "time_from": "the autotuner's timing of the chosen tile shape"},
                "clocks": clk}
    if rank == 0:
        e2e_s = (max_ms / 1e3) + t_init + t_read
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "ensemble64_seed4", "instances": len(wls), "nodes": nodes,
                           "particles": int(sum(len(w.particles) for w in wls)),
                           "storage": args.storage, "tile": TILE_NAMES[tile],
                           "parallelism": "replicas%d" % world,
                           "l2": "no flush: %.2f GB of distributions, %.0fx the 129 MB L2"
                                 % (nodes * B_LU / 1e9, nodes * B_LU / 129e6)},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                             "kernel": TILE_KERNELS[tile],
                             "algorithmic_bytes_per_launch": B_LU * nodes, "avg_launch_ms": sc_ms,
                             "peak_source": peaks["source"] + " (hbm_gbs)",
                             "kernel_times_from": "the autotuner's timing of the chosen tile shape"},
                "e2e": {"value": aggregate_mlups(nodes, args.steps, world, e2e_s), "unit": UNIT,
                        "h2d_bytes_per_step": sum(len(w.particles) * lbm.PARTICLE_DTYPE.itemsize for w in wls) / args.steps,
                        "d2h_bytes_per_step": d2h / args.steps,
                        "includes": "lbm_init of all instances from host particles, batch creation, "
                                    "the timed steps, and every instance's particles and fields read back"},
                "gpu_launches": int(launches), "clocks": clk,
                "whole_step_hbm_frac": B_LU * nodes / (max_ms / args.steps / 1e3) / 1e9 / peaks["hbm_gbs"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def weighted_percentile(values, weights, q: float) -> float:
    """Smallest value whose cumulative weight (values ascending) reaches q of
    the total: the q-quantile of per-step latency when each round's latency
    per step is weighted by the steps the round took."""
    o = np.argsort(values)
    cw = np.cumsum(np.asarray(weights, float)[o])
    return float(np.asarray(values)[o][min(np.searchsorted(cw, q * cw[-1]), len(cw) - 1)])


# ------------------------------------------------------------------------------ served stream
def run_served(args, summary: bool = False):
    """Poisson stream of 40 sedimentation requests (512^2-2048^2, 2000-20000
    steps) through the request loop: aggregate MLUPS over the wall time from
    the first arrival to the last result, p50/p99 per-step and per-request
    latency.  summary: called from the headline run on one GPU, the first 10
    requests of the same stream (FP32 and BF16); returns the key's dict
    instead of printing a line."""
    import torch
    from paper_2308_16597_gb300 import build as B, lbm

    rank, world, local = dist_env()
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if summary:
        world, rank = 1, 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    reqs = W.served_stream(40, seed=5)
    if summary:
        reqs = reqs[:10]
    storage = STORAGE_CODES[args.storage]
    free, _ = torch.cuda.mem_get_info(dev)
    pool = int(min(0.6 * free, 64 << 30))
    stream = torch.cuda.Stream(device=dev)
    step_ms, step_w, lat, updates, dev_ms = [], [], [], 0, 0.0
    max_active = 0
    with torch.cuda.stream(stream):
        srv = lbm.Server(pool, max_active=32, stream=stream)
        clocks = ClockSampler(local)
        clocks.start()
        pending = list(reqs)
        outstanding = {}
        t0 = time.perf_counter()
        while pending or outstanding:
            now = time.perf_counter() - t0
            while pending and pending[0][0] <= now:
                t_arr, wl, steps = pending.pop(0)
                rid = srv.submit(wl.domain, wl.particles, wl.params, steps, storage=storage)
                outstanding[rid] = t_arr
            st = srv.tick(args.tick_steps)
            if st["steps"] == 0 and st["queued"] == 0 and not outstanding and pending:
                time.sleep(max(0.0, pending[0][0] - (time.perf_counter() - t0)))
                continue
            if st["steps"]:
                step_ms.append(st["ms"] / st["steps"])
                step_w.append(st["steps"])
                updates += st["updates"]
                dev_ms += st["ms"]
            max_active = max(max_active, st["active"] + st["retired"])
            now = time.perf_counter() - t0
            for rid in list(outstanding):
                state, err = srv.status(rid)
                if state == lbm.SERVER_FAILED:
                    raise RuntimeError("request %d failed: %s" % (rid, lbm.lbm_strerror(err)))
                if state == lbm.SERVER_DONE:
                    srv.result(rid)
                    lat.append(now - outstanding.pop(rid))
        wall = time.perf_counter() - t0 - reqs[0][0]
        clk = clocks.stop()
        srv.close()
    latency = {"step_ms_p50": weighted_percentile(step_ms, step_w, 0.5),
               "step_ms_p99": weighted_percentile(step_ms, step_w, 0.99),
               "request_s_p50": float(np.percentile(lat, 50)),
               "request_s_p99": float(np.percentile(lat, 99))}
    if summary:
        return {"workload": "served_poisson20_%dreq_seed5" % len(reqs), "requests": len(reqs),
                "storage": args.storage, "value": updates / wall / 1e6, "unit": UNIT,
                "device_mlups": updates / (dev_ms / 1e3) / 1e6, "latency": latency,
                "steps": int(sum(step_w)), "tick_steps": args.tick_steps, "peak_concurrent": max_active,
                "wall_s": wall, "includes": "submission of host inputs, admission, all steps, results read back"}
    if rank == 0:
        line = {"metric": METRIC, "value": updates / wall / 1e6, "unit": UNIT, "n_gpus": world,
                "steps": int(sum(step_w)), "warmup": 0, "ms_per_step": float(np.average(step_ms, weights=step_w)),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "served_poisson20_40req_seed5", "requests": len(reqs),
                           "storage": args.storage, "pool_gb": pool / 1e9, "max_active": 32,
                           "tick_steps": args.tick_steps, "peak_concurrent": max_active,
                           "parallelism": "replicas%d" % world},
                "latency": latency,
                "device_mlups": updates / (dev_ms / 1e3) / 1e6,
                "e2e": {"value": updates / wall / 1e6, "unit": UNIT,
                        "includes": "submission of host inputs, admission, all steps, results read back"},
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["cavity4000", "cavity2000", "cavity256", "cavity1024", "ellipses129",
                                           "paper4800", "ensemble64", "served"],
                    default="cavity4000")
    ap.add_argument("--tick-steps", type=int, default=100, help="served: steps per scheduling round")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline only: no reduced-storage, ensemble and served keys")
    ap.add_argument("--windows", type=int, default=5,
                    help="timed regions of exactly --steps steps each; the value is their median")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--links", choices=["index", "direct"], default="index",
                    help="links from the fixed index array (default) or by direct addressing (the paper's "
                         "comparison, Table 1)")
    ap.add_argument("--stream-collide", choices=["staged", "unstaged"], default="staged",
                    help="whole-lattice stream-collide kernel with BF16 / FP16 storage: persistent blocks "
                         "staging row tiles in shared memory (default), or one block per tile reading global "
                         "memory (comparison; FP32 storage always runs the latter)")
    ap.add_argument("--overlap", action="store_true",
                    help="stream-collide of the tiles away from every particle beside the particle kernels "
                         "(LBM_FLAG_OVERLAP), the rest after them")
    ap.add_argument("--storage", choices=sorted(STORAGE_CODES), default="fp32",
                    help="plane storage: FP32 (the headline), or BF16 / scaled FP16 deviations")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.windows < 1:
        ap.error("--windows must be at least 1")
    if args.workload in ("ensemble64", "served"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the 4000^2 workload only"}))
            return 0
        return run_ensemble(args) if args.workload == "ensemble64" else run_served(args)
    wl = {"cavity4000": W.sedimentation_4000, "cavity2000": W.sedimentation_2000,
          "cavity256": W.parity_256,
          "cavity1024": W.crop_1024, "ellipses129": W.ellipse_cluster_129,
          "paper4800": W.paper_4800}[args.workload]()
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
