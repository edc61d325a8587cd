#!/usr/bin/env python3
"""Benchmark: SurfaceNets extract + constrained smoothing throughput on one GB300.

One step = sn_extract of one label map resident in HBM (including the count
read-back that sizes the outputs) + sn_smooth + sn_free.  Default workload: the
largest single-GPU configuration, the 1024x1024x512 uint32 connectomics-like map
(50,000 Voronoi cells, spacing (1,1,4), 5% background gaps; stand-in for the
paper's EM connectome), 8 iterations, relaxation 0.5, constraint 1 voxel.  The
map (2.1 GB) is larger than L2, so no flush is needed between steps.

The same line carries, as secondary objects measured after the headline: the
512^3 uint16 atlas-like map (93 labels, 16 iterations), the learned-proposal
comparison on that map, the 256 batched maps of uneven sizes, and the
label-count sweep (--no-secondary skips them).

Prints ONE JSON line (rank 0).  Under torchrun each rank processes its own copy
of the map (independent units, weak scaling, no collective on the data path);
value = voxels of all ranks / max time over ranks.

--impl reference times the FP64 sequential oracle on the host cores on a
bounded slab of the same map (the CPU baseline arm).
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = "extract+smooth Gvoxels/s & HBM roofline frac; learned vs plain at ≤1e-3 vox"
UNIT = "Gvoxels/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c3slab", "c5", "synthetic"])
    p.add_argument("--slabs", action="store_true",
                   help="split the map into z-slabs over the ranks (extract + smooth + count exchange + stitch "
                        "on each rank's GPU; strong scaling) instead of running replicas")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the secondary objects (atlas map, batched maps, label sweep)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-learned", action="store_true",
                   help="skip the learned-proposal comparison (plain smoothing vs proposal + corrections)")
    p.add_argument("--cpu-slab", type=int, default=0, help="z-slices of the map the oracle baseline runs on")
    p.add_argument("--label-sweep", action="store_true",
                   help="time extract + smooth with the first k of 128 sphere labels selected, k = 1..128")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def make_workload(name):
    import sn_synth
    if name == "c1":
        return sn_synth.config1()
    if name == "c2":
        return sn_synth.config2()
    if name == "c3":
        return sn_synth.config3()
    if name == "c3slab":
        return sn_synth.config3_slab()
    return sn_synth.paper_synthetic()


def count_labels(labels, background):
    """Distinct non-background values (by slabs, so that a 2 GB map needs no 4 GB temporary)."""
    top = int(labels.max()) if labels.size else 0
    if top >= 1 << 27:
        return int(len(np.unique(labels)) - (1 if (labels == background).any() else 0))
    seen = np.zeros(top + 1, dtype=bool)
    for z in range(0, labels.shape[0], 32):
        seen |= np.bincount(labels[z:z + 32].ravel(), minlength=top + 1) > 0
    if background <= top:
        seen[background] = False
    return int(seen.sum())


def workload_config(w, extra=None):
    cfg = {"workload": w.name, "dims": list(w.dims), "label_dtype": str(w.labels.dtype),
           "labels": count_labels(w.labels, w.background),
           "iterations": w.iterations, "relaxation": w.relaxation, "constraint_voxels": w.constraint,
           "spacing": list(w.spacing),
           "l2": "inputs larger than L2 (%.0f MB label map), no flush" % (w.labels.nbytes / 1e6),
           "map_sha256": hashlib.sha256(w.labels.tobytes()).hexdigest()[:16]}
    if extra:
        cfg.update(extra)
    return cfg


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # let nvidia-smi finish starting up (its first query) before the timed region: its start can
            # hold the driver for tens of milliseconds
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.05)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------- roofline inputs
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(V, b, P, Q, S, n):
    """Bytes the method must move: read labels once, write the mesh once, and
    read + write every offset float3 once per Jacobi sweep."""
    return {"labels": V * b, "mesh": 12 * P + (16 + 2 * b) * Q + 8 * (P + 1) + 4 * S, "smooth": 24 * n * P}


def kernel_units(name, V, b, P, Q, S, n):
    """(algorithmic bytes per launch, unit description) for each kernel."""
    if name == "k_smooth":
        return 24 * P, "24 B per point (read+write one float3 offset)"
    if name == "k_smooth_first2":
        return 48 * P, "48 B per point (sweeps 1 and 2: read+write one float3 offset each)"
    if name in ("k_count", "k_planes"):
        return V * b, "%d B per voxel (labels read once)" % b
    if name in ("k_emit_tile", "k_emit"):
        return 12 * P + (16 + 2 * b) * Q + 8 * (P + 1) + 4 * S, "mesh bytes written once"
    return None, None


KERNEL_SOURCES = {
    "k_smooth": ["paper_2401_14906_gb300/csrc/sn_smooth.cu", "paper_2401_14906_gb300/csrc/sn_sweep.cuh"],
    "k_count": ["paper_2401_14906_gb300/csrc/sn_extract.cu", "paper_2401_14906_gb300/csrc/sn_count.cuh"],
    "k_emit_tile": ["paper_2401_14906_gb300/csrc/sn_emit.cu", "paper_2401_14906_gb300/csrc/sn_emit_tile.cuh"],
    "k_scan": ["paper_2401_14906_gb300/csrc/sn_extract.cu", "paper_2401_14906_gb300/csrc/sn_scan.cuh"],
}


def sources_sha(kernel):
    """sha256 (16 hex digits) of the sources a kernel is built from, concatenated."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(kernel, []):
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel, workload):
    """Per-launch DRAM bytes of `kernel` on `workload` from the committed ncu summary, if it was taken
    with the current sources (a summary may be scaled from a smaller case of the same shape, as it says)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        ent = json.load(open(path)).get(kernel, {}).get(workload)
        if not ent or ent.get("sources_sha256") != sources_sha(kernel):
            return None
        return ent["dram_bytes_per_launch_full"]
    except Exception:
        return None


def host_link_floor(h2d_bytes, d2h_bytes, reps=5):
    """The step's copies alone, pinned host <-> device (torch copies on two streams): H2D only, D2H only, and
    both at once -- the floor under the end-to-end step.  Never raises: a failure is reported in the result."""
    import torch
    try:
        h_in = torch.empty(h2d_bytes, dtype=torch.uint8, pin_memory=True)
        d_in = torch.empty(h2d_bytes, dtype=torch.uint8, device="cuda")
        d_out = torch.empty(d2h_bytes, dtype=torch.uint8, device="cuda")
        h_out = torch.empty(d2h_bytes, dtype=torch.uint8, pin_memory=True)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

        def h2d():
            with torch.cuda.stream(s_in):
                d_in.copy_(h_in, non_blocking=True)

        def d2h():
            with torch.cuda.stream(s_out):
                h_out.copy_(d_out, non_blocking=True)

        def both():
            h2d()
            d2h()

        def timed(fn):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / reps * 1e3
        a, b, c = timed(h2d), timed(d2h), timed(both)
        return {"h2d_ms": a, "h2d_gbs": h2d_bytes / a / 1e6, "d2h_ms": b, "d2h_gbs": d2h_bytes / b / 1e6,
                "both_ms": c, "timing": "host clock, pinned buffers, the two directions on two streams"}
    except Exception as e:  # the measurement is context for e2e; it must not cost the bench line
        return {"error": str(e)}


# ---------------------------------------------------------------- reference
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    w = make_workload(args.workload)
    nz = w.labels.shape[0]
    slab = args.cpu_slab or max(2, min(nz, 16))
    z0 = max(0, nz // 2 - slab // 2)
    lab = np.ascontiguousarray(w.labels[z0:z0 + slab])
    V = lab.size

    def once():
        t = time.perf_counter()
        m = oracle.extract(lab, w.spacing, w.origin, background=w.background)
        oracle.smooth(m, w.spacing, w.origin, w.iterations, w.relaxation, w.constraint)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        once()
    ts = [once() for _ in range(args.steps)]
    tot = sum(ts)
    value = V * args.steps / tot / 1e9
    sample = "slices z=[%d,%d) of the map (%dx%dx%d voxels) per step, extract + %d sweeps" % (
        z0, z0 + slab, lab.shape[2], lab.shape[1], lab.shape[0], w.iterations)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, {"sample": sample}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(w, seconds_per_run=4.0):
    """The oracle's extract + smooth on a bounded slab of the map, on 1 host core: the slab is sized to
    about seconds_per_run, then 1 warm-up run and the median of 3 runs."""
    import oracle
    nz = w.labels.shape[0]

    def run(slab):
        z0 = max(0, nz // 2 - slab // 2)
        lab = np.ascontiguousarray(w.labels[z0:z0 + slab])
        t = time.perf_counter()
        m = oracle.extract(lab, w.spacing, w.origin, background=w.background)
        oracle.smooth(m, w.spacing, w.origin, w.iterations, w.relaxation, w.constraint)
        return time.perf_counter() - t, z0, lab.size

    slab = max(2, min(nz, 4))
    dt, _, _ = run(slab)  # sizing run (also warms the oracle's library)
    if dt < seconds_per_run / 2 and slab < nz:
        slab = int(min(nz, max(slab + 1, slab * seconds_per_run / max(dt, 1e-3))))
    run(slab)  # warm-up at the chosen size
    runs = [run(slab) for _ in range(3)]
    dts = sorted(r[0] for r in runs)
    med = dts[1]
    z0, vox = runs[0][1], runs[0][2]
    sample = "slices z=[%d,%d) of the map (%d voxels), extract + %d sweeps; 1 warm-up, median of 3 runs" % (
        z0, z0 + slab, vox, w.iterations)
    return {"value": vox / med / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "seconds_per_run": dts, "host": host_cpu(),
            "paper_cpu_context": "the paper's TBB implementation on a 10-core i9 laptop, extract + 25 sweeps + "
                                 "triangulation: Synthetic 512^3 u16 0.405 s at 16 threads (0.33 Gvoxels/s), "
                                 "Connectome 2048^3 (240 labels) 9.98 s (0.86 Gvoxels/s); other hardware, "
                                 "context only"}


def host_cpu():
    """The host's logical CPU count and model name (from /proc/cpuinfo or lscpu)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "processor name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "model": model}


# --------------------------------------------------------------------- ours
def to_device(labels):
    import torch
    isz = labels.dtype.itemsize
    t = torch.from_numpy(np.ascontiguousarray(labels).view({1: np.uint8, 2: np.int16, 4: np.int32}[isz]))
    return t.cuda().view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[isz])


def measure_device(w, args, stream, clocks=False):
    """Device-resident steps of one workload: CUDA-event time of K steps after W warm-up steps, the
    per-step median, per-kernel durations (a second pass with events around every launch), and the
    roofline objects.  The map is larger than L2 (no flush between steps)."""
    import torch
    from paper_2401_14906_gb300 import sn
    rank, world, _ = dist_env()
    V, b = w.voxels, w.labels.dtype.itemsize
    lab_dev = to_device(w.labels)

    def step():
        m = sn.sn_extract(lab_dev, w.spacing, w.origin, background=w.background, stream=stream)
        sn.sn_smooth(m, w.iterations, w.relaxation, w.constraint)
        cnt = m.counts
        rec = sn.sn_mesh_record_bytes(m)
        m.free()
        return cnt, rec

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            counts, rec = step()
        torch.cuda.synchronize()
        P, Q, S = counts
        sampler = None
        if clocks:
            sampler = ClockSampler(torch.cuda.current_device())
            sampler.start()
            time.sleep(0.3)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        clk = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())

        # per-step times (events between steps): the median beside the mean above
        per_step = []
        for _ in range(args.steps):
            a_, z_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            step()
            z_.record(stream)
            per_step.append((a_, z_))
        torch.cuda.synchronize()
        ms_median = statistics.median(a_.elapsed_time(z_) for a_, z_ in per_step)

        # per-kernel durations: the same steps again with events around every launch
        sn.sn_profile_read(reset=True)
        sn.sn_profile_enable(True)
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        prof = sn.sn_profile_read(reset=True)
        sn.sn_profile_enable(False)
    del lab_dev

    ms_step = ms / args.steps
    value = world * V * args.steps / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    alg = algorithmic_bytes(V, b, P, Q, S, w.iterations)
    alg_total = sum(alg.values())
    kernels = {}
    launches_per_step = 0
    for name, (n, tot) in prof.items():
        per = n / args.steps
        launches_per_step += per
        kernels[name] = {"launches_per_step": per, "ms_per_step": tot / args.steps, "ms_per_launch": tot / max(n, 1)}
        by, _ = kernel_units(name, V, b, P, Q, S, w.iterations)
        if by is not None:
            kernels[name]["achieved_gbs"] = by / (kernels[name]["ms_per_launch"] / 1e3) / 1e9
            kernels[name]["frac"] = kernels[name]["achieved_gbs"] / peak
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"]) if kernels else None
    roof = None
    if dom:
        by, unit_desc = kernel_units(dom, V, b, P, Q, S, w.iterations)
        if by is not None:
            ach = by / (kernels[dom]["ms_per_launch"] / 1e3) / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_kind": peak_kind + " (burst copy)",
                    "frac_of_nominal_7900": ach / 7900.0, "traffic": traffic_for(dom, w.name),
                    "algorithmic_bytes_per_launch": by, "unit_bytes": unit_desc}
    path_time = ms_step / 1e3
    return {"value": value, "ms_per_step": ms_step, "ms_per_step_median": ms_median,
            "counts": (P, Q, S), "record_bytes_per_point": rec,
            "roofline": roof,
            "path_roofline": {"algorithmic_bytes_per_step": alg_total, "bytes_breakdown": alg,
                              "achieved_gbs": alg_total / path_time / 1e9, "peak": peak,
                              "frac": alg_total / path_time / 1e9 / peak,
                              "frac_of_nominal_7900": alg_total / path_time / 1e9 / 7900.0},
            "kernels": kernels, "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clk}


def measure_e2e(w, args, stream, counts):
    """End to end through the C ABI with host buffers: pinned labels in, the full mesh out, every
    step, inside the timed region (host clock)."""
    import ctypes

    import torch
    from paper_2401_14906_gb300 import sn
    rank, world, _ = dist_env()
    V, b = w.voxels, w.labels.dtype.itemsize
    P, Q, S = counts
    host_lab = torch.empty(w.labels.size * b, dtype=torch.uint8, pin_memory=True)
    host_lab.numpy()[:] = np.ascontiguousarray(w.labels).view(np.uint8).ravel()
    out_bufs = {k: torch.empty(n, dtype=torch.uint8, pin_memory=True) for k, n in
                [("points", 12 * P), ("quads", 16 * Q), ("quad_labels", 2 * b * Q),
                 ("stencil_offsets", 8 * (P + 1)), ("stencil_ids", 4 * S)]}
    d2h = sum(t.numel() for t in out_bufs.values())
    lib = sn.load()

    def c_args():
        return ((ctypes.c_int64 * 3)(*w.dims), (ctypes.c_double * 3)(*w.spacing),
                (ctypes.c_double * 3)(*w.origin))

    def upload():
        """start copying the step's labels to the device (returns at once)"""
        d, _, _ = c_args()
        up = ctypes.c_void_p()
        rc = lib.sn_labels_upload(ctypes.c_void_p(host_lab.data_ptr()), b, d, ctypes.byref(up))
        assert rc == 0, sn.sn_last_error()
        return up

    def start(bufs, up=None):
        """extract + smooth of one map, from its upload or (up None) from host labels copied during the
        call, then the asynchronous copy-out into `bufs`"""
        d, sp, org = c_args()
        out = ctypes.c_void_p()
        st = ctypes.c_void_p(stream.cuda_stream)
        if up is None:
            rc = lib.sn_extract(ctypes.c_void_p(host_lab.data_ptr()), b, d, sp, org, None, 0,
                                w.background, st, ctypes.byref(out))
        else:
            rc = lib.sn_extract_labels(up, sp, org, None, 0, w.background, st, ctypes.byref(out))
            lib.sn_labels_free(up, st)
        assert rc == 0, sn.sn_last_error()
        rc = lib.sn_smooth(out, w.iterations, w.relaxation, w.constraint)
        assert rc == 0
        rc = lib.sn_mesh_copy_to_host_async(out, *[ctypes.c_void_p(bufs[k].data_ptr()) for k in
                                                   ("points", "quads", "quad_labels", "stencil_offsets",
                                                    "stencil_ids")], None)
        assert rc == 0, sn.sn_last_error()
        return out

    def finish(out):
        rc = lib.sn_mesh_wait(out)
        assert rc == 0, sn.sn_last_error()
        lib.sn_free(out)

    def e2e_run(steps, pipelined):
        """one step at a time (host labels copied inside sn_extract), or pipelined: each step's labels
        are uploaded while the previous step is extracted and smoothed, and its copy-out overlaps
        the next step (two output buffers)"""
        prev = None
        up = upload() if pipelined and steps else None
        for k in range(steps):
            if not pipelined:
                finish(start(out_sets[k % 2]))
                continue
            nxt = upload() if k + 1 < steps else None
            cur = start(out_sets[k % 2], up)
            up = nxt
            if prev is not None:
                finish(prev)
            prev = cur
        if prev is not None:
            finish(prev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    out_sets = [out_bufs, {k: torch.empty_like(v).pin_memory() for k, v in out_bufs.items()}]
    e2e_ms = {}
    with torch.cuda.stream(stream):
        for pipelined in (False, True):
            e2e_run(2, pipelined)
            torch.cuda.synchronize()
            barrier()
            t0 = time.perf_counter()
            e2e_run(args.steps, pipelined)
            torch.cuda.synchronize()
            barrier()
            ems = (time.perf_counter() - t0) * 1e3
            if world > 1:
                import torch.distributed as dist
                t = torch.tensor([ems], device="cuda")
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
                ems = float(t.item())
            e2e_ms[pipelined] = ems
    ems = e2e_ms[True]
    res = {"value": world * V * args.steps / (ems / 1e3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": V * b, "d2h_bytes_per_step": int(d2h),
           "ms_per_step": ems / args.steps,
           "timing": "host clock around K steps; each step uploads its labels from pinned memory "
                     "(sn_labels_upload, issued one step ahead so that it overlaps the previous step), "
                     "extracts (sn_extract_labels), smooths and copies its mesh back to pinned memory "
                     "(sn_mesh_copy_to_host_async, overlapping the next step)",
           "one_step_at_a_time_ms_per_step": e2e_ms[False] / args.steps}
    del out_sets, out_bufs, host_lab
    res["host_link"] = host_link_floor(V * b, int(d2h))
    return res


def secondary_atlas(args, stream):
    """The 512^3 uint16 atlas-like map (93 labels, 16 iterations): device-resident rate and rooflines,
    then the learned-proposal comparison on the same map."""
    w = make_workload("c2")
    r = measure_device(w, args, stream)
    P, Q, S = r.pop("counts")
    out = {"config": workload_config(w, {"points": P, "quads": Q, "stencil_entries": S}), "unit": UNIT}
    out.update(r)
    if not args.no_learned:
        out["learned"] = learned_comparison(w, args.steps)
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2401_14906_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2401_14906_gb300 import sn
    sn.load()

    w = make_workload(args.workload)
    V, b = w.voxels, w.labels.dtype.itemsize
    stream = torch.cuda.Stream()
    r = measure_device(w, args, stream, clocks=True)
    P, Q, S = r["counts"]
    e2e = None if args.no_e2e else measure_e2e(w, args, stream, r["counts"])

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"],
            "ms_per_step_median": r["ms_per_step_median"],
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u%d+f32" % (8 * b), "data": "synthetic",
            "config": workload_config(w, {"parallelism": "replicas" if world > 1 else "single",
                                          "points": P, "quads": Q, "stencil_entries": S,
                                          "sweep_record_bytes_per_point": r["record_bytes_per_point"]}),
            "roofline": r["roofline"], "path_roofline": r["path_roofline"], "kernels": r["kernels"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "e2e": e2e}
    if world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(w)
        line["cpu_baseline"] = cb
    if world == 1 and not args.no_secondary and args.workload == "c3":
        del w
        torch.cuda.empty_cache()
        line["c2_atlas"] = secondary_atlas(args, stream)
        line["c5_batch"] = batch_object(args)
        line["label_sweep"] = label_sweep_object(args)
    elif world == 1 and not args.no_learned and args.workload == "c2":
        line["learned"] = learned_comparison(w, args.steps)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def learned_comparison(w, repeats):
    """Plain smoothing (the step's iteration count) vs the learned proposal + k correction sweeps on the
    bench map, with the committed trained parameters: device times and the largest offset difference."""
    from paper_2401_14906_gb300 import proposal
    if not os.path.exists(proposal.PROPOSAL_PARAMS):
        return {"unavailable": "no trained parameters (python -m paper_2401_14906_gb300.proposal)"}
    L = proposal.load_learner()
    r = proposal.evaluate(L, w.labels, w.spacing, w.iterations, w.relaxation, w.constraint,
                          corrections=(0, 1, 2, 4, 8), repeats=max(3, repeats), engines=("mma_sync", "tcgen05"))
    L.free()
    target = {"max_err_vox": 1e-3, "speedup_vs_plain": 2.0}
    met = [c for c in r["learned"]
           if c["max_err_vox"] <= target["max_err_vox"] and (c["speedup"] or 0) >= target["speedup_vs_plain"]]
    return {"plain_ms": r["ms_plain"], "iterations": r["iterations"], "proposals": r["learned"],
            "target": target, "met": bool(met),
            "model": "MLP 32-64-64-3 BF16 (tensor cores: mma.sync and tcgen05 engines), trained on 200 seeded "
                     "256^3 maps"}


def label_sweep_object(args, steps=None, ks=(1, 2, 4, 8, 16, 32, 64, 128)):
    """Slowdown as the number of extracted labels grows: the 512^3 uint16 map of 128 overlapping
    spheres (the paper's Synthetic dataset shape), labels 1..k selected, the rest background."""
    import torch

    from paper_2401_14906_gb300 import sn
    steps = steps or args.steps
    w = make_workload("synthetic")
    lab = to_device(w.labels)
    stream = torch.cuda.Stream()
    rows = []
    with torch.cuda.stream(stream):
        for k in ks:
            sel = list(range(1, k + 1))

            def step():
                m = sn.sn_extract(lab, w.spacing, w.origin, selected=sel, background=0, stream=stream)
                sn.sn_smooth(m, w.iterations, w.relaxation, w.constraint)
                cnt = m.counts
                m.free()
                return cnt

            for _ in range(max(2, min(args.warmup, 3))):
                cnt = step()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(steps):
                step()
            z.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(z) / steps
            rows.append({"labels": k, "ms_per_step": ms, "points": cnt[0], "quads": cnt[1]})
    base = rows[0]["ms_per_step"]
    for r in rows:
        r["slowdown"] = r["ms_per_step"] / base
    return {"metric": "extract+smooth time vs number of selected labels", "unit": "ms",
            "config": workload_config(w, {"sweep": "selected = labels 1..k"}), "steps": steps,
            "timing": "CUDA events around the steps of each k, device-resident map", "results": rows}


def run_label_sweep(args):
    from paper_2401_14906_gb300 import build, sn
    build.build()
    sn.load()
    print(json.dumps(label_sweep_object(args)))
    return 0


def batch_object(args, steps=None, loop=True):
    """The 256 seeded maps of uneven sizes (edges 32-256, uint8/uint16): a step is extract + 16 sweeps of every
    map.  Timed with the host clock around the whole step (host work included) after a device sync, for the
    batched call (one launch per phase, tuned tile shapes), the same with the graph (one executable graph per
    layout, updated in place), and a loop of single-map calls."""
    import torch
    import sn_synth
    from paper_2401_14906_gb300 import sn
    steps = steps or args.steps
    ws = sn_synth.config5_maps()
    V = sum(w.voxels for w in ws)
    labs = [to_device(w.labels) for w in ws]
    it, lam, d = ws[0].iterations, ws[0].relaxation, ws[0].constraint

    def batched(graph=False):
        ms = sn.sn_extract_smooth_batch(labs, iterations=it, relaxation=lam, constraint_distance=d, graph=graph)
        torch.cuda.synchronize()
        return ms

    def looped():
        ms = []
        for t in labs:
            m = sn.sn_extract(t)
            sn.sn_smooth(m, it, lam, d)
            ms.append(m)
        torch.cuda.synchronize()
        return ms

    per_step = {}

    def timed(fn, name):
        for _ in range(max(3, min(args.warmup, 5))):
            for m in fn():
                m.free()
        torch.cuda.synchronize()
        marks = []
        t0 = time.perf_counter()
        for _ in range(steps):
            for m in fn():  # (each call ends with a device sync: the step's own end)
                m.free()
            marks.append(time.perf_counter())
        torch.cuda.synchronize()
        total = (time.perf_counter() - t0) * 1e3 / steps
        d = np.diff(np.array([t0] + marks)) * 1e3
        per_step[name] = {"median": float(np.median(d)), "max": float(d.max())}
        return total

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms_batch = timed(batched, "batched")
    clocks = sampler.stop()
    ms_graph = timed(lambda: batched(True), "graph")
    ms_loop = timed(looped, "loop") if loop else None
    counts = [m.counts for m in batched()]
    P = sum(c[0] for c in counts)
    return {"metric": METRIC, "value": V / (ms_batch / 1e3) / 1e9, "unit": UNIT, "steps": steps,
            "ms_per_step": ms_batch, "dtype": "u8/u16+f32",
            "config": {"workload": "c5_256maps_edges32-256_u8u16", "maps": len(ws), "voxels": V, "points": P,
                       "iterations": it, "timing": "host clock around each step (allocation, launches, waits)",
                       "batched": "sn_extract_smooth_batch: one counting launch per label type over all maps, one "
                                  "scan launch, one totals wait, one emission launch per label type, one sweep "
                                  "launch per iteration over all maps, tuned counting and emission tiles"},
            "ms_per_step_median": per_step["batched"]["median"], "ms_per_step_max": per_step["batched"]["max"],
            "graph_mode_ms_per_step": ms_graph, "graph_mode_gvoxels_s": V / (ms_graph / 1e3) / 1e9,
            "graph_mode_ms_per_step_median": per_step["graph"]["median"],
            "single_map_loop_ms_per_step": ms_loop,
            "single_map_loop_gvoxels_s": V / (ms_loop / 1e3) / 1e9 if ms_loop else None,
            "clocks": clocks}


def run_batch(args):
    from paper_2401_14906_gb300 import build
    build.build()
    from paper_2401_14906_gb300 import sn
    sn.load()
    r = batch_object(args)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic",
            "config": r["config"], "clocks": r["clocks"],
            "graph_mode_ms_per_step": r["graph_mode_ms_per_step"],
            "single_map_loop_ms_per_step": r["single_map_loop_ms_per_step"]}
    print(json.dumps(line))
    return 0


def run_slabs(args):
    """z-slab decomposition of one map over the ranks (strong scaling): every rank extracts and smooths its
    slab with ghost slices, the owned counts are exchanged (an allgather of three integers, NCCL under
    torchrun), and each rank stitches its owned part with global ids on its GPU.  value = voxels of the map
    / max over ranks of the time per step."""
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2401_14906_gb300 import build, slabs
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2401_14906_gb300 import sn
    sn.load()
    w = make_workload(args.workload)
    nz = w.labels.shape[0]
    p = slabs.slab_plan(nz, world, w.iterations)[rank]
    lab = to_device(np.ascontiguousarray(w.labels[p["s0"]:p["s1"]]))
    stream = torch.cuda.Stream()

    def gather(vec):
        if world == 1:
            return np.asarray(vec, dtype=np.int64).reshape(1, 3)
        return slabs.torch_allgather(vec)

    def step():
        part, _ = slabs.run_rank_device(lab, w.spacing, w.origin, w.iterations, w.relaxation, w.constraint, rank,
                                        world, nz, gather, stream)
        return part

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            part = step()
        e1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    if rank == 0:
        V = w.voxels
        print(json.dumps({"metric": METRIC, "value": V * args.steps / (ms / 1e3) / 1e9, "unit": UNIT,
                          "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
                          "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
                          "vs_baseline": None, "dtype": "u%d+f32" % (8 * w.labels.dtype.itemsize),
                          "data": "synthetic",
                          "config": workload_config(w, {"parallelism": "z-slabs over %d ranks" % world,
                                                        "slab_rank0": [p["s0"], p["s1"]],
                                                        "owned_points_rank0": int(part["stencil_offsets"].numel()),
                                                        "timing": "CUDA events on rank 0's stream around K steps "
                                                                  "(extract, smooth, count allgather, stitch), "
                                                                  "max over ranks"})}))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.slabs and args.impl != "reference":
        return run_slabs(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.label_sweep:
        return run_label_sweep(args)
    if args.workload == "c5":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
