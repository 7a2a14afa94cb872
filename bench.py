"""Benchmark: wire-scan depth reconstruction on GB300.

Default workload (one "step" = one full reconstruction of one scan):
2048x2048-pixel detector, 401 wire steps, 1001 depth bins of 1 um over
[-500, 500] um; uint16 images [401][2048][2048] (3.36 GB) resident in HBM,
FP32 output [1001][2048][2048] (16.8 GB).  Both exceed the 129 MB L2, so no
flush is needed between steps.  Synthetic forward-model scan (200 Gaussian
spots at seeded depths, Poisson background 20), standing in for the paper's
HDF5 beamline scans.

Prints ONE JSON line (rank 0).  `value` is pixel*steps/s over all ranks (each
rank reconstructs its own scan: replicas, weak scaling); `e2e` is the same
metric through dr_reconstruct_host with pinned host buffers (host->device
upload and device->host download of the whole result inside the timed
region); `roofline` compares the kernel's algorithmic bytes per launch with
the measured HBM copy bandwidth; `cpu_baseline` times the FP64 CPU oracle on
a bounded sample of rows of the same scan.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel·steps/s and % of HBM peak; served scans/s with p50/p99 latency"
UNIT = "pixel·steps/s"
WORKLOAD = ("plain method, full detector: 2048x2048 uint16 pixels, 401 wire steps of 1 um, "
            "1001 bins of 1 um over [-500,500] um, FP32 output [1001][2048][2048], "
            "device-resident input")
FALLBACK_HBM_GBS = 6800.0
PROFILE_TRAFFIC = {
    "rows": os.path.join(ROOT, "profiles", "rows_kernel_full_detector_traffic.txt"),
    "pixels": os.path.join(ROOT, "profiles", "pixels_kernel_rotated_detector_traffic.txt"),
}
# the rows kernel's code ends where the per-pixel kernel's section begins,
# which ends where the persistent batch kernel begins
ROWS_KERNEL_END = "// ------------------------------------------------------- pixels kernel ---"
PIXELS_KERNEL_BEGIN = ROWS_KERNEL_END
PIXELS_KERNEL_END = "// ------------------------------------------------- persistent batch kernel ---"


def kernel_source_hash(kernel="rows", device_src=None, tables_src=None):
    """Hash of the code a kernel is built from: the device header up to the
    per-pixel kernel's section (helpers, depth model, row tables, rows_tile,
    rows_kernel), for the per-pixel kernel also its own section, and the
    table layouts."""
    csrc = os.path.join(ROOT, "paper_2201_13309_gb300", "csrc")
    if device_src is None:
        device_src = open(os.path.join(csrc, "dr_device.cuh"), "rb").read()
    if tables_src is None:
        tables_src = open(os.path.join(csrc, "dr_tables.h"), "rb").read()
    h = hashlib.sha256()
    cut = device_src.find(ROWS_KERNEL_END.encode())
    h.update(device_src[:cut] if cut >= 0 else device_src)
    if kernel == "pixels":
        b = device_src.find(PIXELS_KERNEL_BEGIN.encode())
        e = device_src.find(PIXELS_KERNEL_END.encode())
        h.update(device_src[b:e] if 0 <= b < e else device_src)
    h.update(tables_src)
    return h.hexdigest()[:16]


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel="rows"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    try:
        kv = {}
        for line in open(PROFILE_TRAFFIC[kernel]):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_source_sha") != kernel_source_hash(kernel):
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML while running."""

    REASONS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}

    def __init__(self, index, uuid=None, period=0.005):
        self.samples = []
        self.period = period
        self.ok = False
        self.max_mhz = None
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            found = False
            if uuid:
                u = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
                found = self.nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(self.h)) == 0
            if not found and self.nv.nvmlDeviceGetHandleByIndex_v2(
                    index, ctypes.byref(self.h)) != 0:
                return
            m = ctypes.c_uint()
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = int(m.value)
            self.ok = True
        except OSError:
            pass

    def _read(self):
        c = ctypes.c_uint()
        r = ctypes.c_ulonglong()
        self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c))
        fn = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.h, ctypes.byref(r))
        return int(c.value), int(r.value)

    def _loop(self):
        while not self._stop.is_set():
            self.samples.append(self._read())
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self._stop = threading.Event()
            self._t = threading.Thread(target=self._loop, daemon=True)
            self._t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self._t.join()
            self.samples.append(self._read())

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"],
                    "samples": 0}
        mhz = [c for c, _ in self.samples]
        mask = 0
        for _, r in self.samples:
            mask |= r
        reasons = [n for b, n in self.REASONS.items() if mask & b and n != "gpu_idle"]
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples)}


def gpu_local_cpus(dev):
    """CPUs local to the GPU (sysfs: the PCI device's local_cpulist, else its
    NUMA node's cpulist), intersected with the CPUs this process may use."""
    import torch

    def parse(text):
        cpus = set()
        for part in text.strip().split(","):
            if not part:
                continue
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus

    try:
        props = torch.cuda.get_device_properties(dev)
        bus = f"{props.pci_domain_id:04x}:{props.pci_bus_id:02x}:{props.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bus}"
        cpus = set()
        if os.path.exists(f"{base}/local_cpulist"):
            cpus = parse(open(f"{base}/local_cpulist").read())
        if not cpus and os.path.exists(f"{base}/numa_node"):
            node = int(open(f"{base}/numa_node").read())
            if node >= 0:
                cpus = parse(open(f"/sys/devices/system/node/node{node}/cpulist").read())
        return sorted(cpus & os.sched_getaffinity(0))
    except Exception:
        return []


def page_nodes(ptr, nbytes, samples=256):
    """Memory node of `samples` evenly spaced pages of a host buffer (the
    move_pages system call without a target node reports where each page
    is), as {node: pages}; None where the call is not available."""
    import ctypes
    import platform

    nr = {"aarch64": 239, "x86_64": 279}.get(platform.machine())
    if nr is None or nbytes <= 0:
        return None
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        page = os.sysconf("SC_PAGE_SIZE")
        addrs = sorted({(ptr + i * nbytes // samples) // page * page for i in range(samples)})
        arr = (ctypes.c_void_p * len(addrs))(*addrs)
        status = (ctypes.c_int * len(addrs))()
        rc = libc.syscall(ctypes.c_long(nr), ctypes.c_int(0), ctypes.c_ulong(len(addrs)), arr,
                          None, status, ctypes.c_int(0))
        if rc != 0:
            return None
        hist = {}
        for v in status:
            hist[str(v)] = hist.get(str(v), 0) + 1
        return hist
    except Exception:
        return None


class near_gpu:
    """Run the enclosed host allocations on CPUs local to the GPU, so that
    pinned pages are placed in the memory node next to it."""

    def __init__(self, dev):
        self.cpus = gpu_local_cpus(dev)

    def __enter__(self):
        self.saved = os.sched_getaffinity(0)
        if self.cpus:
            os.sched_setaffinity(0, self.cpus)
        return self

    def __exit__(self, *a):
        os.sched_setaffinity(0, self.saved)


def reduce_max(x, device):
    """Max of a float over all ranks (the slowest rank's time); identity on
    one process."""
    import torch
    import torch.distributed as tdist

    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, max_ms):
    """Units all ranks processed per second, timed by the slowest rank."""
    return world * units_per_rank_step * steps / (max_ms * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    machine type)."""
    import platform
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine() or "unknown"


def cpu_oracle_sample(spec, host_rows, rows_idx, threads, budget_s=None):
    """Time the FP64 oracle on the given rows (one-row geometries)."""
    from oracle import oracle as O

    t0 = time.perf_counter()
    for r, img in zip(rows_idx, host_rows):
        g = dict(spec.geom)
        g["det_origin"] = (np.asarray(spec.geom["det_origin"])
                           + r * np.asarray(spec.geom["row_step"])).tolist()
        g["rows"] = 1
        O.reconstruct(g, spec.wires, img, spec.edges, threads=threads)
        if budget_s and time.perf_counter() - t0 > budget_s:
            break
    return time.perf_counter() - t0


def synth_rows_host(spec, rows_idx, seed=0):
    """uint16 [K, 1, W] stacks of the chosen rows, generated on the host with
    the same forward model as the device scan (spots + Poisson background)."""
    from tests.gen import synth

    rng = np.random.Generator(np.random.PCG64(seed + 12345))
    idx, val = synth.spot_contributions(spec.geom, spec.wires, spec.scat)
    H, W, K = spec.geom["rows"], spec.geom["cols"], spec.K
    out = []
    kk = idx // (H * W)
    rr = (idx // W) % H
    cc = idx % W
    for r in rows_idx:
        rate = np.full((K, 1, W), 20.0)
        sel = rr == r
        np.add.at(rate, (kk[sel], 0, cc[sel]), val[sel])
        out.append(synth.poisson_u16(rng, rate))
    return out


def run_reference(args, world, rank):
    """The reference arm: the FP64 CPU oracle as it stands, on host cores."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    from tests.gen import synth

    O.build()
    spec = synth.full_scan_spec(0)
    threads = os.cpu_count() or 1
    rows_per_step = max(1, threads // 4)
    pool_idx = [int(r) for r in np.linspace(0, 2047, 32)]
    pool = synth_rows_host(spec, pool_idx)
    times = []
    for s in range(args.warmup + args.steps):
        pick = [(s * rows_per_step + i) % len(pool_idx) for i in range(rows_per_step)]
        dt = cpu_oracle_sample(spec, [pool[i] for i in pick], [pool_idx[i] for i in pick],
                               threads)
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    units = rows_per_step * spec.geom["cols"] * spec.K * args.steps
    value = units / tot
    sample = (f"{rows_per_step} detector rows per step ({rows_per_step * 2048} pixels x 401 "
              f"steps x 1001 bins), FP64, {threads} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_precision(args, spec, images, dev):
    """Error of each arithmetic variant against the FP64 oracle on sampled
    rows of the scan, the conservation error on every pixel whose depth range
    lies inside the bins, and the exactness of the integer differences."""
    import torch

    from oracle import oracle as O
    from paper_2201_13309_gb300 import dr

    O.build()
    H, W = spec.geom["rows"], spec.geom["cols"]
    rows = [int(r) for r in np.linspace(0, H - 1, args.precision_rows)]
    threads = os.cpu_count() or 1
    host_rows, refs = {}, {}
    for r in rows:
        host_rows[r] = images[:, r:r + 1, :].cpu().numpy().view(np.uint16)
        g = dict(spec.geom)
        g["det_origin"] = (np.asarray(spec.geom["det_origin"])
                           + r * np.asarray(spec.geom["row_step"])).tolist()
        g["rows"] = 1
        refs[r] = O.reconstruct(g, spec.wires, host_rows[r], spec.edges, threads=threads)
    # integer differences, bit-exact check on the sampled rows
    mism, checked = 0, 0
    for r in rows:
        d = dr.image_differences(images[:, r:r + 1, :].contiguous()).cpu().numpy()
        mism += int(np.count_nonzero(d.astype(np.int64) != O.differences(host_rows[r])))
        checked += d.size
    # pixels whose whole depth range lies inside the bins (conservation holds)
    g1 = dict(spec.geom, cols=1)
    dd = O.depths(g1, spec.wires)[:, 0, [0, -1]]
    inside = torch.from_numpy((dd[:, 0] > spec.edges[0]) & (dd[:, 1] < spec.edges[-1])).to(dev)
    first = images[0].to(torch.int32) & 0xFFFF
    last = images[-1].to(torch.int32) & 0xFFFF
    sabs = torch.zeros((H, W), dtype=torch.float64, device=dev)
    for k0 in range(0, spec.K - 1, 32):
        k1 = min(spec.K - 1, k0 + 32)
        a = images[k0:k1 + 1].to(torch.int32) & 0xFFFF
        sabs += (a[:-1] - a[1:]).abs().sum(0).double()
    variants = []
    for geom_p in ("fp32", "fp64"):
        for out_t in ("f32", "bf16"):
            plan = dr.Plan(spec.geom, spec.wires, spec.edges, out_dtype=out_t,
                           geom_precision=geom_p)
            out = plan.empty_output(dev)
            for _ in range(2):
                plan.reconstruct(images, out)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.precision_reps):
                plan.reconstruct(images, out)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / args.precision_reps
            worst = 0.0
            for r in rows:
                got = out[:, r:r + 1, :].float().cpu().numpy().astype(np.float64)
                s = np.abs(np.diff(host_rows[r].astype(np.int64), axis=0)).sum(0)[None]
                worst = max(worst, float((np.abs(got - refs[r]) / np.maximum(s, 1)).max()))
            tot = out.sum(0, dtype=torch.float64)
            cons = ((tot - (first - last).double()).abs() / sabs.clamp(min=1))[inside, :]
            variants.append({
                "geometry": geom_p, "output": out_t, "ms": ms,
                "GBps": plan.info()["bytes_per_call"] / ms / 1e6,
                "max_bin_err_over_sum_abs_dI": worst,
                "max_conservation_err_over_sum_abs_dI": float(cons.max()),
                "meets_1e-4": worst <= 1e-4})
            plan.close()
            del out
    return {"mode": "precision", "metric": "max |bin - oracle| / sum_k |dI_k| per pixel",
            "workload": WORKLOAD, "oracle_rows": len(rows),
            "conservation_pixels": int(inside.sum()) * W,
            "differences": {"checked": checked, "mismatches": mism}, "variants": variants}


def batch_waves(specs, budget_bytes):
    """Greedy packing of scans (in order) into waves whose inputs + outputs
    fit the HBM budget."""
    waves, cur, used = [], [], 0
    for sp in specs:
        need = sp.P * (2 * sp.K + 4 * sp.B)
        if cur and used + need > budget_bytes:
            waves.append(cur)
            cur, used = [], 0
        cur.append(sp)
        used += need
    if cur:
        waves.append(cur)
    return waves


def small_roi_spec(seed, rotate_deg=0.0):
    """A scan of the uneven-batch distribution restricted to small ROIs
    (256^2 or 512^2), where launch tails dominate a per-scan loop."""
    from tests.gen import synth

    for s in range(seed * 1000, seed * 1000 + 1000):
        sp = synth.batch_scan_spec(s, rotate_deg)
        if sp.geom["rows"] <= 512:
            return sp
    raise RuntimeError("no small ROI found")


def run_batched(args, dev, specs=None):
    """Uneven scans: per-scan launch loop vs one persistent launch per wave
    (replayed from a captured CUDA graph), same plans, same buffers."""
    import torch

    from paper_2201_13309_gb300 import autotune, dr
    from tests.gen import synth

    if specs is None:
        specs = [synth.batch_scan_spec(s, args.rotate) for s in range(args.batch_scans)]
    waves = batch_waves(specs, args.budget_gb * 1e9)
    tot_loop = tot_batch = 0.0
    units = bytes_alg = 0.0
    per_wave = []
    ok = True
    for wave in waves:
        jobs = []
        for sp in wave:
            img = synth.device_spot_images(sp.geom, sp.wires, sp.scat, seed=1000 + len(jobs),
                                           background=20.0, device=dev)
            out = torch.empty((sp.B, sp.geom["rows"], sp.geom["cols"]), device=dev)
            plan, _ = autotune.tuned_plan(sp.geom, sp.wires, sp.edges, img, out=out, reps=3)
            jobs.append((plan, img, out))
            units += sp.P * sp.K
            bytes_alg += plan.info()["bytes_per_call"]
        batch, btune = autotune.tuned_batch(jobs)
        # per-scan launch loop
        for plan, img, out in jobs:
            plan.reconstruct(img, out)
        torch.cuda.synchronize()
        ref = None
        if args.check:  # sampled bin planes (bitwise) and the exact FP64 sum of each output
            ref = []
            for _, _, out in jobs:
                sel = torch.linspace(0, out.shape[0] - 1, 8, device=dev).long()
                ref.append((sel, out[sel].clone(), out.sum(dtype=torch.float64)))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.batch_reps):
            for plan, img, out in jobs:
                plan.reconstruct(img, out)
        e1.record()
        e1.synchronize()
        t_loop = e0.elapsed_time(e1) / args.batch_reps
        for _, _, out in jobs:
            out.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        batch.check_device()
        if ref is not None:
            for (_, _, out), (sel, planes, total) in zip(jobs, ref):
                ok &= bool(torch.equal(out[sel].view(torch.int32), planes.view(torch.int32)))
                ok &= bool(torch.equal(out.sum(dtype=torch.float64), total))
            del ref
        e0.record()
        for _ in range(args.batch_reps):
            batch.launch()
        e1.record()
        e1.synchronize()
        t_batch = e0.elapsed_time(e1) / args.batch_reps
        tot_loop += t_loop
        tot_batch += t_batch
        per_wave.append({"scans": len(wave), "loop_ms": t_loop, "batch_ms": t_batch,
                         "items": batch.info()["items"], "ctas_per_sm": btune["ctas_per_sm"],
                         "max_tile_cols": btune["max_tile_cols"], "threads": btune["threads"]})
        batch.close()
        for plan, img, out in jobs:
            plan.close()
        del jobs, img, out
        torch.cuda.empty_cache()
    n = len(specs)
    peak, kind = measured_hbm_peak()
    return {
        "mode": "batched", "metric": "scans/s", "scans": n, "waves": len(waves),
        "budget_GB": args.budget_gb,
        "loop": {"scans_per_s": n / (tot_loop * 1e-3), "ms": tot_loop,
                 "pixel_steps_per_s": units / (tot_loop * 1e-3),
                 "GBps": bytes_alg / (tot_loop * 1e-3) / 1e9},
        "batch": {"scans_per_s": n / (tot_batch * 1e-3), "ms": tot_batch,
                  "pixel_steps_per_s": units / (tot_batch * 1e-3),
                  "GBps": bytes_alg / (tot_batch * 1e-3) / 1e9,
                  "hbm_frac": bytes_alg / (tot_batch * 1e-3) / 1e9 / peak},
        "speedup": tot_loop / tot_batch, "bitwise_equal": ok if args.check else None,
        "peak_GBps": peak, "peak_kind": kind, "per_wave": per_wave,
        "workload": ("64 uneven scans (seeds 0-63): ROI in {256^2, 512^2, 1024^2, 2048x1024, "
                     "2048^2}, 51-801 steps, bins of 0.5/1/2 um over +-400 um, FP32"),
    }


def hugepage_pinned(shape, keep):
    """An int16 host tensor in anonymous memory advised for transparent huge
    pages and page-locked with cudaHostRegister (instead of cudaHostAlloc);
    the mapping is appended to keep, which must outlive the tensor."""
    import ctypes
    import mmap

    import torch

    n = int(np.prod(shape)) * 2
    m = mmap.mmap(-1, n, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    if hasattr(mmap, "MADV_HUGEPAGE"):
        m.madvise(mmap.MADV_HUGEPAGE)
    buf = (ctypes.c_uint8 * n).from_buffer(m)
    ctypes.memset(buf, 0, n)  # touch every page before registering
    err = torch.cuda.cudart().cudaHostRegister(ctypes.addressof(buf), n, 0)
    if int(err) != 0:
        raise RuntimeError(f"cudaHostRegister failed ({err})")
    keep.append((m, buf))
    return torch.frombuffer(buf, dtype=torch.int16).view(shape)


def run_served(args, dev):
    """Poisson arrival streams of scans from the uneven-batch distribution into
    the server (admission against an HBM budget, pinned uploads overlapped on
    slot streams, results left on the device until the client releases them);
    plus a saturation run against a serial plan-upload-reconstruct loop.

    Every request is a scan of its own (batch_scan_spec of a seed of its own:
    its ROI origin and size, step count and bin width), so every request
    builds its plan.  Its images are the first K planes of one pinned
    forward-model scan per ROI size with the largest step count of the
    distribution (1000 distinct multi-GB scans do not fit in host memory;
    the kernels' time does not depend on the counts)."""
    import threading as th

    import torch

    from paper_2201_13309_gb300 import dr
    from tests.gen import synth

    placement = near_gpu(dev)
    keep = []  # the mappings behind hugepage-pinned buffers
    kmax = 801
    buffers, up_gbs, pool_nodes = {}, {}, {}
    for i, (rows, cols) in enumerate(synth.ROI_CHOICES):
        rng = np.random.Generator(np.random.PCG64(3000 + i))
        geom = synth.detector_geometry(rows, cols, (0, 0), synth.FULL_DET, synth.FULL_DET)
        wires = synth.wire_path(kmax)
        scat = synth.spot_scatterers(rng, max(5, int(round(200 * rows * cols / 2048 ** 2))),
                                     rows, cols)
        img = synth.device_spot_images(geom, wires, scat, seed=2000 + i, background=20.0,
                                       device=dev)
        with placement:
            h = (hugepage_pinned(img.shape, keep) if args.served_pin == "hugepage"
                 else torch.empty(img.shape, dtype=torch.int16, pin_memory=True))
            h.copy_(img)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        img.copy_(h, non_blocking=True)
        torch.cuda.synchronize()
        up_gbs[f"{rows}x{cols}"] = h.numel() * 2 / (time.perf_counter() - t0) / 1e9
        pool_nodes[f"{rows}x{cols}"] = page_nodes(h.data_ptr(), h.numel() * 2)
        buffers[(rows, cols)] = h
        del img
    torch.cuda.empty_cache()

    def images_of(sp):
        return buffers[(sp.geom["rows"], sp.geom["cols"])][:sp.K]

    budget = int(args.budget_gb * 1e9)
    results = []
    rates = [float(r) for r in args.rates.split(",") if r]
    srv = dr.Server(budget, slots=args.slots)
    # per-request timestamps (seconds since the server's creation), one JSON
    # object per line, when asked for
    trace = open(args.served_trace, "w") if args.served_trace else None
    for ri, rate in enumerate(rates):
        specs = [synth.batch_scan_spec(100000 * (ri + 1) + i) for i in range(args.served_scans)]
        rng = np.random.Generator(np.random.PCG64(1000 + int(rate)))
        gaps = rng.exponential(1.0 / rate, args.served_scans)
        ids, lat, parts = [], [], []
        lock = th.Lock()
        have = th.Semaphore(0)
        built0 = srv.stats()["plans_built"]

        def consumer():
            for i in range(args.served_scans):
                have.acquire()
                with lock:
                    rid = ids[i]
                srv.wait(rid)
                _, t = srv.fetch(rid)
                lat.append(t["done"] - t["submitted"])
                sp = specs[i]
                parts.append((sp.P * sp.K * 2, t["planned"] - t["submitted"],
                              t["admitted"] - t["submitted"], t["uploaded"] - t["admitted"],
                              t["done"] - t["uploaded"], t["issued"] - t["admitted"],
                              t["copy"]))
                if trace is not None:
                    trace.write(json.dumps(dict(t, rate=rate, i=i, rows=sp.geom["rows"],
                                                cols=sp.geom["cols"], K=sp.K, B=sp.B)) + "\n")
                srv.release(rid)

        ct = th.Thread(target=consumer)
        ct.start()
        t0 = time.perf_counter()
        nxt = t0
        for i in range(args.served_scans):
            nxt += gaps[i]
            d = nxt - time.perf_counter()
            if d > 0:
                time.sleep(d)
            sp = specs[i]
            rid = srv.submit(sp.geom, sp.wires, sp.edges, images_of(sp))
            with lock:
                ids.append(rid)
            have.release()
        ct.join()
        wall = time.perf_counter() - t0
        lat_ms = np.array(lat) * 1e3
        pa = np.array([p[1:] for p in parts]) * 1e3
        in_gb = np.array([p[0] for p in parts]) / 1e9
        big = in_gb >= np.percentile(in_gb, 90)
        # phases from arrival: plan ready, admitted (plan ready, slot and
        # memory free), upload done (after earlier uploads), kernel done
        names = ("plan_wait", "queue", "upload", "kernel", "issue", "copy")
        results.append({"offered_scans_per_s": rate, "scans": args.served_scans,
                        "achieved_scans_per_s": args.served_scans / wall,
                        "plans_built": srv.stats()["plans_built"] - built0,
                        "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)),
                        "mean_ms": float(lat_ms.mean()), "max_ms": float(lat_ms.max()),
                        "phase_p50_ms": {n: float(np.percentile(pa[:, c], 50))
                                         for c, n in enumerate(names)},
                        "phase_p99_ms": {n: float(np.percentile(pa[:, c], 99))
                                         for c, n in enumerate(names)},
                        "largest_tenth_inputs": {
                            "input_GB_min": float(in_gb[big].min()),
                            "p50_ms": float(np.percentile(lat_ms[big], 50)),
                            "upload_p50_ms": float(np.percentile(pa[big, 2], 50)),
                            "upload_GBps_p50": float(np.percentile(
                                in_gb[big] / np.maximum(pa[big, 2] * 1e-3, 1e-9), 50))}})
        print(json.dumps({"served_rate": results[-1]}), file=sys.stderr, flush=True)
    if trace is not None:
        trace.close()
    st = srv.stats()
    srv.close()
    # saturation: everything submitted at once, against the serial loop over
    # the same scans (plan, upload, reconstruct, one after the other)
    n_sat = args.saturation_scans
    sat_specs = [synth.batch_scan_spec(900000 + i) for i in range(n_sat)]
    srv = dr.Server(budget, slots=args.slots)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ids = [srv.submit(sp.geom, sp.wires, sp.edges, images_of(sp)) for sp in sat_specs]
    for rid in ids:
        srv.wait(rid)
        srv.release(rid)
    t_srv = time.perf_counter() - t0
    srv.close()
    d_img = torch.empty(max(h.numel() for h in buffers.values()), dtype=torch.int16, device=dev)
    d_out = torch.empty(max(sp.P * sp.B for sp in sat_specs), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sp in sat_specs:
        h = images_of(sp)
        p = dr.Plan(sp.geom, sp.wires, sp.edges)
        di = d_img[:h.numel()].view(h.shape)
        do = d_out[:sp.P * sp.B].view(sp.B, sp.geom["rows"], sp.geom["cols"])
        with torch.cuda.stream(stream):
            di.copy_(h, non_blocking=True)
            p.reconstruct(di, do, stream=stream)
        stream.synchronize()
        p.close()
    t_loop = time.perf_counter() - t0
    mean_in = float(np.mean([sp.P * sp.K * 2 for sp in sat_specs])) / 1e9
    return {"mode": "served", "metric": "scans/s and p50/p99 latency (arrival -> result on device)",
            "budget_GB": args.budget_gb, "slots": args.slots,
            "pin": args.served_pin, "pinned_upload_GBps": up_gbs, "alloc_cpus": placement.cpus,
            "pool_page_nodes": pool_nodes,
            "mean_input_GB": mean_in, "rates": results,
            "plan_cache": {"plans_built": st["plans_built"], "failed": st["failed"]},
            "saturation": {"scans": n_sat, "server_scans_per_s": n_sat / t_srv,
                           "serial_loop_scans_per_s": n_sat / t_loop,
                           "speedup": t_loop / t_srv},
            "workload": ("every request a scan of its own from the uneven-batch distribution "
                         "(ROI 256^2..2048^2 at its own origin, 51-801 steps, 0.5/1/2 um bins "
                         "over +-400 um), so every request builds its plan; images are the "
                         "first K planes of one pinned forward-model scan per ROI size")}


def run_link(args, dev):
    """Host-to-device link under intermittent use: a 2.5 GiB pinned upload
    every 200 ms (the gaps of a lightly loaded server), first as single
    copies, then alternating a single copy with the same bytes as 128 MiB
    pieces, then back-to-back single copies.  Each copy is timed with CUDA
    events on its stream; nothing else runs in the process meanwhile."""
    import torch

    n = int(2.5 * (1 << 30))
    piece = 128 << 20
    with near_gpu(dev) as place:
        h = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        h.fill_(1)
    nodes_before = page_nodes(h.data_ptr(), n)
    d = torch.empty(n, dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream(device=dev)

    def timed(pieces):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for off in range(0, n, n if not pieces else piece):
                m = min(n - off, piece) if pieces else n
                d[off:off + m].copy_(h[off:off + m], non_blocking=True)
            e1.record(st)
        e1.synchronize()
        return n / (e0.elapsed_time(e1) * 1e-3) / 1e9

    def paced(seconds, kinds):
        got = {k: [] for k in kinds}
        t_end, i = time.perf_counter() + seconds, 0
        while time.perf_counter() < t_end:
            t = time.perf_counter()
            k = kinds[i % len(kinds)]
            i += 1
            got[k].append(timed(k == "pieces"))
            time.sleep(max(0.0, 0.2 - (time.perf_counter() - t)))
        return got

    def summary(v):
        v = sorted(v)
        return {"copies": len(v), "GBps_p50": round(v[len(v) // 2], 1),
                "GBps_p10": round(v[len(v) // 10], 1), "GBps_min": round(v[0], 1)}

    first = paced(args.link_seconds, ["single"])["single"]
    tenth = max(1, len(first) // 10)
    mixed = paced(args.link_seconds, ["single", "pieces"])
    busy = []
    t_end = time.perf_counter() + 5.0
    while time.perf_counter() < t_end:
        busy.append(timed(False))
    try:
        online = open("/sys/devices/system/node/online").read().strip()
    except OSError:
        online = None
    return {"mode": "link", "metric": "pinned host-to-device GB/s, 2.5 GiB uploads",
            "upload_GiB": 2.5, "piece_MiB": 128, "interval_ms": 200,
            "numa_nodes_online": online, "alloc_cpus": place.cpus,
            "page_nodes_before": nodes_before,
            "page_nodes_after": page_nodes(h.data_ptr(), n),
            "single_first_tenth": summary(first[:tenth]),
            "single_last_tenth": summary(first[-tenth:]),
            "mixed_single": summary(mixed["single"]), "mixed_pieces": summary(mixed["pieces"]),
            "back_to_back_single": summary(busy)}


def run_pixels(args, spec, images, dev):
    """The paper's pixel-percentage sweep on the full-detector scan: the
    pixels carrying the most signal (activity = sum |dI|) are selected and
    only they are reconstructed (compacted output), against the full scan."""
    import torch

    from paper_2201_13309_gb300 import dr

    plan = dr.Plan(spec.geom, spec.wires, spec.edges)
    out_full = plan.empty_output(dev)

    def t(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    full_ms = t(lambda: plan.reconstruct(images, out_full))
    act = dr.pixel_activity(images)
    act_ms = t(lambda: dr.pixel_activity(images))
    flat = act.reshape(-1)
    vals = flat.cpu().numpy()
    rows = []
    for pct in (25, 50, 75, 100):
        thr = float(np.percentile(vals, 100 - pct)) if pct < 100 else -1.0
        sel_ms = t(lambda: dr.select_pixels(flat, thr))
        idx, n = dr.select_pixels(flat, thr)
        out = torch.empty((spec.B, n), dtype=torch.float32, device=dev)
        rec_ms = t(lambda: plan.reconstruct_selected(images, idx, n, out), reps=3)
        ok = bool(torch.equal(out[:, ::max(1, n // 4096)].view(torch.int32),
                              out_full.reshape(spec.B, -1)[:, idx.long()][:, ::max(1, n // 4096)]
                              .view(torch.int32)))
        rows.append({"percent": pct, "pixels": n, "activity_ms": act_ms, "select_ms": sel_ms,
                     "reconstruct_ms": rec_ms, "total_ms": act_ms + sel_ms + rec_ms,
                     "equal_to_full": ok})
        del out
    return {"mode": "pixels", "workload": WORKLOAD, "full_scan_ms": full_ms, "sweep": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--slab-rows", type=int, default=256)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--mode", default="plain",
                    choices=["plain", "precision", "batched", "served", "pixels", "link"])
    ap.add_argument("--link-seconds", type=float, default=60.0,
                    help="link: seconds of paced uploads in each of its two phases")
    ap.add_argument("--rates", default="5,20,50")
    ap.add_argument("--served-scans", type=int, default=1000)
    ap.add_argument("--saturation-scans", type=int, default=96)
    ap.add_argument("--served-pin", default="torch", choices=["torch", "hugepage"],
                    help="served: pinned image pool from cudaHostAlloc (torch) or from "
                         "huge-page memory registered with cudaHostRegister")
    ap.add_argument("--served-trace", default="",
                    help="served: write every request's timestamps to this file")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--batch-scans", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=3)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--check", action="store_true", help="batched: compare outputs bitwise")
    ap.add_argument("--precision-rows", type=int, default=24)
    ap.add_argument("--precision-reps", type=int, default=20)
    ap.add_argument("--tile-cols", type=int, default=0, help="fixed tile width (0: autotune)")
    ap.add_argument("--bin-groups", type=int, default=0)
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--rotate", type=float, default=0.0,
                    help="rotate the detector in its plane (degrees): per-pixel depths")
    ap.add_argument("--tilt", type=float, default=0.0, help="tilt the detector about x (degrees)")
    ap.add_argument("--wire-climb", type=float, default=0.0,
                    help="wire also moves across the beam (um per step along y): depths "
                         "of some pixels then run in both directions (interval kernel)")
    ap.add_argument("--wire-jitter", type=float, default=0.0,
                    help="seeded normal jitter of the wire centre across the beam (um)")
    ap.add_argument("--intervals", action="store_true",
                    help="use the interval kernel (depths in any order) on the same scan")
    ap.add_argument("--rows", type=int, default=2048,
                    help="reconstruct only the first ROWS detector rows (small profiling case)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch

    import __graft_entry__
    from paper_2201_13309_gb300 import dr
    from tests.gen import synth

    if world > 1:
        import torch.distributed as tdist

        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        tdist.barrier()
        __graft_entry__.build()

    if args.mode == "batched":
        if rank == 0:
            res = run_batched(args, dev)
            small = run_batched(args, dev, [small_roi_spec(s, args.rotate)
                                            for s in range(args.batch_scans)])
            res["small_roi_mix"] = {k: small[k] for k in ("scans", "waves", "loop", "batch",
                                                          "speedup", "bitwise_equal")}
            res["small_roi_mix"]["workload"] = ("64 scans of the same distribution restricted "
                                                "to 256^2 and 512^2 ROIs")
            if args.rotate:
                rot = f"; detector rotated {args.rotate} deg (per-pixel kernel)"
                res["workload"] += rot
                res["small_roi_mix"]["workload"] += rot
            print(json.dumps(res), flush=True)
        return 0
    if args.mode == "served":
        if rank == 0:
            print(json.dumps(run_served(args, dev)), flush=True)
        return 0
    if args.mode == "link":
        if rank == 0:
            print(json.dumps(run_link(args, dev)), flush=True)
        return 0

    spec = synth.full_scan_spec(0)
    if args.rotate or args.tilt:
        spec.geom = synth.detector_geometry(2048, 2048, rotate_deg=args.rotate,
                                            tilt_deg=args.tilt)
    if args.wire_climb or args.wire_jitter:
        rng = np.random.Generator(np.random.PCG64(7))
        spec.wires = spec.wires.copy()
        spec.wires[:, 1] += (args.wire_climb * 1e-3 * np.arange(spec.K)
                             + rng.normal(0.0, args.wire_jitter * 1e-3, spec.K))
    if args.rows != spec.geom["rows"]:
        spec.geom = dict(spec.geom, rows=args.rows)
        keep = spec.scat.spot_row < args.rows - 2
        spec.scat = synth.Scatterers(spec.scat.depth[keep], spec.scat.peak[keep],
                                     spec.scat.spot_row[keep], spec.scat.spot_col[keep])
    images = synth.device_spot_images(spec.geom, spec.wires, spec.scat, seed=rank, background=20.0,
                                      device=dev)
    if args.mode == "precision":
        if rank == 0:
            print(json.dumps(run_precision(args, spec, images, dev)), flush=True)
        return 0
    if args.mode == "pixels":
        if rank == 0:
            print(json.dumps(run_pixels(args, spec, images, dev)), flush=True)
        return 0

    from paper_2201_13309_gb300 import autotune

    out = torch.empty((spec.B, spec.geom["rows"], spec.geom["cols"]), dtype=torch.float32,
                      device=dev)
    # plan-build time of this workload (host sample, device constants and the
    # check of every (group, step)), outside the timed region
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    dr.Plan(spec.geom, spec.wires, spec.edges, force_intervals=args.intervals).close()
    plan_ms = (time.perf_counter() - t_plan) * 1e3
    tuned = None
    if args.intervals:
        plan = dr.Plan(spec.geom, spec.wires, spec.edges, force_intervals=True)
    elif args.tile_cols:
        plan = dr.Plan(spec.geom, spec.wires, spec.edges, tile_cols=args.tile_cols,
                       bin_groups=args.bin_groups)
    else:
        plan = dr.Plan(spec.geom, spec.wires, spec.edges)
        if plan.info()["kernel"] != "intervals":  # (depths in both directions: no shape to tune)
            plan.close()
            plan, tuned = autotune.tuned_plan(spec.geom, spec.wires, spec.edges, images, out=out,
                                              use_cache=not args.retune)
    info = plan.info()
    stream = torch.cuda.Stream(dev)
    P = spec.P
    units_per_step = P * spec.K

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            tdist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.reconstruct(images, out, stream=stream)
    barrier()
    plan.check_device()
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(dev.index, uuid)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    barrier()
    with sampler:
        start.record(stream)
        for _ in range(args.steps):
            plan.reconstruct(images, out, stream=stream)
        stop.record(stream)
        stop.synchronize()
    barrier()
    plan.check_device()
    elapsed_ms = reduce_max(start.elapsed_time(stop), dev)
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(units_per_step, args.steps, world, elapsed_ms)

    # kernel roofline: one launch per step, so the event time per step is
    # the kernel's average launch duration
    peak, peak_kind = measured_hbm_peak()
    alg_bytes = info["bytes_per_call"]
    achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    traffic = profiled_traffic(info["kernel"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_kind": peak_kind,
                "kernel": {"rows": "rows_kernel<GeoFx,float,tma,4>",
                           "pixels": ("pixels_poly_kernel<float,tma,"
                                      f"one_step={info['one_step_per_bin']}>"
                                      if info["depth_form"] == 2 else
                                      f"pixels_kernel<GeoFx,float,tma,"
                                      f"one_step={info['one_step_per_bin']}>"),
                           "intervals": "intervals_kernel<GeoFx,float,tma>"}[info["kernel"]],
                "algorithmic_bytes_per_launch": alg_bytes}

    # end to end through the public API with host buffers: the streamed form
    # (row slabs, uploads / kernels / downloads overlapped on three streams);
    # the unpipelined form (whole upload, kernel, whole download) beside it
    e2e = None
    if not args.no_e2e:
        with near_gpu(dev):
            h_img = torch.empty(images.shape, dtype=torch.int16, pin_memory=True)
            h_img.copy_(images)
            h_out = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
            h_out.zero_()
        slab = args.slab_rows
        per = (-(-slab * spec.geom["cols"] * spec.K * 2 // 256) * 256
               + -(-slab * spec.geom["cols"] * spec.B * 4 // 256) * 256)
        ws = torch.empty(3 * per, dtype=torch.uint8, device=dev)

        def timed(fn, n):
            fn()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(n):
                fn()
            e1.record(stream)
            e1.synchronize()
            barrier()
            return reduce_max(e0.elapsed_time(e1), dev)

        e2e_ms = timed(lambda: plan.reconstruct_streamed(h_img, h_out, ws, slab_rows=slab,
                                                         stream=stream), args.e2e_steps)
        serial_ms = timed(lambda: plan.reconstruct_host(h_img, h_out, images, out, stream=stream),
                          args.e2e_steps)
        e2e = {"value": whole_job_rate(units_per_step, args.e2e_steps, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(images.numel() * 2),
               "d2h_bytes_per_step": int(out.numel() * out.element_size()),
               "steps": args.e2e_steps, "ms_per_step": e2e_ms / args.e2e_steps,
               "api": f"dr_reconstruct_streamed ({slab}-row slabs, 3 slab buffers in a "
                      f"{3 * per / 1e9:.2f} GB workspace, pinned host buffers: uploads "
                      "overlapped with the kernels, which store the bins straight into "
                      "the pinned host output)",
               "unpipelined_ms_per_step": serial_ms / args.e2e_steps}
        del h_img, h_out, ws

    cpu = None
    if rank == 0 and not args.no_cpu:
        from oracle import oracle as O

        O.build()
        threads = os.cpu_count() or 1
        probe = [1023]
        host = synth_rows_host(spec, probe)
        t1 = cpu_oracle_sample(spec, host, probe, threads)
        n = max(1, min(512, int(args.cpu_seconds / max(t1, 1e-3))))
        rows_idx = [int(r) for r in np.linspace(0, 2047, n)]
        host = synth_rows_host(spec, rows_idx)
        dt = cpu_oracle_sample(spec, host, rows_idx, threads)
        cpu = {"value": len(rows_idx) * spec.geom["cols"] * spec.K / dt, "unit": UNIT,
               "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": (f"{len(rows_idx)} of 2048 detector rows ({len(rows_idx) * 2048} pixels "
                          f"x 401 steps x 1001 bins), FP64, {threads} threads, {dt:.1f} s")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.rows == 2048 else
                                    WORKLOAD + f" (first {args.rows} rows only)")
                       + (f"; detector rotated {args.rotate} deg, tilted {args.tilt} deg"
                          if args.rotate or args.tilt else "")
                       + ("; interval kernel (depths in any order) forced"
                          if args.intervals else "")
                       + (f"; wire also moving across the beam ({args.wire_climb} um per step, "
                          f"{args.wire_jitter} um jitter, seed 7)"
                          if args.wire_climb or args.wire_jitter else ""),
                       "pixels": P, "wire_steps": spec.K,
                       "bins": spec.B, "parallelism": f"replicas x{world}",
                       "l2": f"input ({2 * units_per_step / 1e9:.2f} GB) and output "
                             f"({4 * P * spec.B / 1e9:.1f} GB) larger than L2; no flush",
                       "kernel": info["kernel"], "depth_form": info["depth_form"],
                       "geometry": "fp64" if info["geom_precision"] else "fp32",
                       "plan_ms": round(plan_ms, 1),
                       "one_step_per_bin": info["one_step_per_bin"],
                       "tile_cols": info["tile_cols"],
                       "pixels_per_thread": info["pixels_per_thread"],
                       "bin_groups": info["bin_groups"], "threads": info["threads"],
                       "smem_bytes": info["smem_bytes"],
                       "autotuned": None if tuned is None else {
                           "cached": tuned["cached"],
                           "candidates_ms": {f"{c['tile_cols']}x{c['bin_groups']}": round(c["ms"], 4)
                                             for c in tuned.get("candidates", [])}}},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": sampler.summary(),
            "hbm_frac": roofline["frac"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
