"""Benchmark of the equilibrium projection on GB300 (one JSON line on stdout, rank 0).

Workload: one 512^3 periodic field, FP32, 5000 Voronoi grains with per-grain stress ~ N(0, 200 MPa)
per Voigt component plus voxel noise ~ N(0, 20 MPa), DDO (modified wavevector).  A step is one
eq_project of the field (every pass of the hot path including the FP64 mean and norm
finalisation).  The field (3.2 GB in, 3.2 GB out) is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank projects its own field (replicas, no collective on the data path);
value = voxels of all ranks / max elapsed over ranks.  ``--impl reference`` times the CPU FP64
oracle (the only other place this file runs it) on the host cores instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "equilibrated voxels/s at 512³ (FP32 vs FP64), % HBM roofline; served p50/p99"
UNIT = "voxels/s"
N = 512
GRAINS = 5000
SEED = 210501612 + 2            # workload seed of the 512^3 Voronoi field (rank added)
BYTES_PER_VOXEL_PASS = 48        # FP32: read 6 x 4 B + write 6 x 4 B per voxel


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=N)
    ap.add_argument("--grid", type=int, nargs=3, metavar=("NX", "NY", "NZ"), default=None,
                    help="profiling cases: a non-cubic grid instead of size^3")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64, cuFFT, e2e and CPU comparison legs")
    ap.add_argument("--fp64-only", action="store_true",
                    help="profiling case: only the FP64 projection of the --grid / --size field "
                         "(synthetic Voronoi input), its time and per-pass times")
    ap.add_argument("--batch-fields", type=int, default=0, metavar="K",
                    help="profiling case: only the uneven-batch leg, on the first K of its 64 "
                         "fields, with the plan's default pass shapes (no autotuning)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------ CPU oracle leg

def cpu_oracle_sample(n_cpu: int = N):
    """Time the FP64 oracle on one n_cpu^3 field of the same recipe (grains scaled with volume):
    the whole headline field at the default size (project_large / norms_large, the oracle's
    component-at-a-time forms, so that host memory stays bounded)."""
    import oracle
    from fieldgen import voronoi_stress_field
    grains = max(8, int(round(GRAINS * (n_cpu / N) ** 3)))
    s = voronoi_stress_field((n_cpu,) * 3, grains, 200.0, 20.0, SEED, dtype=torch_f32()).numpy()
    t0 = time.perf_counter()
    out = oracle.project_large(s, "ddo")
    oracle.norms_large(s, out, "ddo")
    dt = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    return {"value": n_cpu ** 3 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one {n_cpu}^3 field ({grains} grains, same recipe, FP32 values), FP64 "
                      f"numpy/scipy oracle: projection + norms (with both divergences), "
                      f"{dt:.2f} s wall on {cores} host threads"}


def torch_f32():
    import torch
    return torch.float32


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_cpu = 128
    for _ in range(args.warmup):
        cpu_oracle_sample(64)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_oracle_sample(n_cpu))
    el = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[0])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{N}^3 Voronoi {GRAINS} grains DDO; each reference step is a "
                                   f"bounded sample: one {n_cpu}^3 field of the same recipe",
                       "grid": [N, N, N], "op": "ddo"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join("/tmp", f"eq_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9 or (self.uuid and self.uuid not in parts[0]):
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------ GPU legs

# algorithmic flops per voxel of the projection: 3-D complex FFTs of the three complex fields
# (pairs of Voigt planes) counted as 5 M log2 M per complex transform of M = nx ny nz points,
# forward and inverse (2 x 3 x 5 x log2 M per voxel; 810 at 512^3), plus about 70 for the per-mode
# projector and its norm terms
def flops_per_voxel(vox: int) -> float:
    return 2 * 3 * 5 * math.log2(vox) + 70.0


def fma_peak(dev, dtype_code: int, iters: int, reps: int = 3):
    """Measured FMA throughput (TFLOP/s) of this GPU: every thread of 8 blocks of 256 threads per
    SM runs 8 independent FMA chains (eqm_fma_probe); best of `reps` CUDA-event-timed launches."""
    import torch
    from paper_2105_01612_gb300 import _measure
    props = torch.cuda.get_device_properties(dev)
    blocks, threads = props.multi_processor_count * 8, 256
    buf = torch.empty(blocks * threads, dtype=torch.float64 if dtype_code else torch.float32,
                      device=dev)
    st = torch.cuda.current_stream(dev)
    _measure.fma_probe(dtype_code, buf.data_ptr(), blocks, threads, max(1, iters // 10),
                       st.cuda_stream)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _measure.fma_probe(dtype_code, buf.data_ptr(), blocks, threads, iters, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    flops = 16.0 * iters * blocks * threads
    return flops / (best / 1e3) / 1e12, best


def gpu_numa_node(dev):
    """NUMA node of the GPU's PCI function as the kernel reports it (None if unknown)."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    bdf = "%04x:%02x:%02x.0" % (getattr(p, "pci_domain_id", 0), getattr(p, "pci_bus_id", 0),
                                getattr(p, "pci_device_id", 0))
    try:
        with open(f"/sys/bus/pci/devices/{bdf}/numa_node") as f:
            return bdf, int(f.read().strip())
    except (OSError, ValueError):
        return bdf, None


def link_leg(hin, hout, dev, reps: int = 3):
    """Host link bandwidth measured in the same run with the e2e leg's own pinned buffers: one
    field's bytes host-to-device, device-to-host, and both directions at once (two streams);
    best of `reps`, CUDA events.  both_ms_per_field is the copy floor of an end-to-end step."""
    import torch
    nbytes = hin.numel() * hin.element_size()
    da, db = torch.empty(hin.shape, dtype=hin.dtype, device=dev), torch.empty(hin.shape, dtype=hin.dtype, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def timed_all(fn):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s1)
            fn()
            e1.record(s1)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts

    def timed(fn):
        return min(timed_all(fn))

    def h2d():
        with torch.cuda.stream(s1):
            da.copy_(hin, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s1):
            hout.copy_(db, non_blocking=True)

    def both():
        ev = torch.cuda.Event()
        ev.record(s1)
        s2.wait_event(ev)
        with torch.cuda.stream(s1):
            da.copy_(hin, non_blocking=True)
        with torch.cuda.stream(s2):
            hout.copy_(db, non_blocking=True)
        ev2 = torch.cuda.Event()
        ev2.record(s2)
        s1.wait_event(ev2)

    t_in, t_out, t_both = timed(h2d), timed(d2h), timed(both)
    t_both_med = statistics.median(timed_all(both))
    bdf, node = gpu_numa_node(dev)
    del da, db
    return {"bytes_per_direction": nbytes, "h2d_gbs": nbytes / (t_in / 1e3) / 1e9,
            "d2h_gbs": nbytes / (t_out / 1e3) / 1e9,
            "both_gbs_total": 2 * nbytes / (t_both / 1e3) / 1e9,
            "both_ms_per_field": t_both, "both_ms_per_field_median": t_both_med,
            "gpu_pci": bdf, "gpu_numa_node": node,
            "method": "torch copies between the e2e leg's pinned host buffers and device "
                      "tensors, best (and median) of 3, CUDA events"}


def fp64_native_ms(x64, o64, n, dev, stream, k: int = 2) -> float:
    """The same FP64 projection with FP64 instructions for the transforms (EQ_F64_ARITH=native,
    read at plan creation), for comparison."""
    import torch
    import paper_2105_01612_gb300 as eq
    old = os.environ.get("EQ_F64_ARITH")
    os.environ["EQ_F64_ARITH"] = "native"
    try:
        p = eq.Plan(n, n, n, torch.float64, 1, "ddo", device=dev)
    finally:
        if old is None:
            del os.environ["EQ_F64_ARITH"]
        else:
            os.environ["EQ_F64_ARITH"] = old
    y = torch.empty_like(o64)
    p.project(x64, y)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(k):
        p.project(x64, y)
    f1.record(stream)
    torch.cuda.synchronize()
    p.close()
    del y
    return f0.elapsed_time(f1) / k


def fp64_case(args):
    """The FP64 plain projection alone on the --grid (or --size^3) field: the profiling case of
    the double-float passes."""
    import torch
    from fieldgen import voronoi_stress_field
    import paper_2105_01612_gb300 as eq
    nx, ny, nz = args.grid if args.grid else (args.size,) * 3
    dev = torch.device("cuda", 0)
    grains = max(8, int(round(GRAINS * nx * ny * nz / N ** 3)))
    x = voronoi_stress_field((nz, ny, nx), grains, 200.0, 20.0, SEED, dtype=torch.float64,
                             device=dev).unsqueeze(0)
    y = torch.empty_like(x)
    p = eq.Plan(nx, ny, nz, torch.float64, 1, "ddo", device=dev)
    for _ in range(max(1, args.warmup)):
        p.project(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        p.project(x, y)
    e1.record()
    torch.cuda.synchronize()
    p.set_timing(1)
    p.project(x, y)
    per_pass, _ = p.pass_ms()
    p.close()
    return {"case": f"FP64 {nx}x{ny}x{nz} Voronoi, DDO", "ms_per_step": e0.elapsed_time(e1) / args.steps,
            "pass_ms": per_pass}


def fp64_leg(x, out, n, dev, stream):
    """The FP64 path on the same field: time per projection (double-float arithmetic between FP64
    reads and writes), the same with FP64 instructions, the FP32-vs-FP64 difference, and the
    algorithmic FP64 flop rate against the DFMA rate measured here (GB300's FP64 units, not HBM,
    bound an FP64-instruction path)."""
    import torch
    import paper_2105_01612_gb300 as eq
    x64 = x.double()
    o64 = torch.empty_like(x64)
    p64 = eq.Plan(n, n, n, torch.float64, 1, "ddo", device=dev)
    p64.project(x64, o64)
    torch.cuda.synchronize()
    k64 = 3
    clk = ClockSampler(str(getattr(torch.cuda.get_device_properties(dev), "uuid", "")))
    clk.start()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(k64):
        p64.project(x64, o64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = f0.elapsed_time(f1) / k64
    p64.set_timing(1)
    p64.project(x64, o64)
    per_pass, _ = p64.pass_ms()
    peak, probe_ms = fma_peak(dev, 1, 100000)
    clocks = clk.stop()
    p64.close()
    vox = x.numel() // 6
    w = torch.tensor([1.0, 1, 1, 2, 2, 2], device=dev, dtype=torch.float64).view(1, 6, 1, 1, 1)
    d = out.double() - o64
    fp32_err = math.sqrt(float((w * d * d).sum() / (w * o64 * o64).sum()))
    del d
    # the plain FP64 projection runs in double-float arithmetic (pairs of FP32 values, about
    # 48-bit significands) on the FP32 units; its algorithmic FP64 flops against the FP64 FMA rate
    # say how it compares with the best FP64 instructions could do
    achieved = flops_per_voxel(vox) * vox / (ms64 / 1e3) / 1e12
    native_ms = fp64_native_ms(x64, o64, n, dev, stream)
    del x64
    return {"value": vox / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
            "arithmetic": "double-float (FP32 pairs) between FP64 reads and writes",
            "fp64_instructions_ms": native_ms,
            "fp32_vs_fp64_rel_l2": fp32_err, "pass_ms": per_pass,
            "roofline": {"bound": "fp64_alu_equivalent", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "flops_per_voxel": flops_per_voxel(vox),
                         "flops_counted": "algorithmic FP64 flops (transforms 5 M log2 M, projector "
                                          "70) against the FP64 FMA rate; the work runs as "
                                          "double-float on the FP32 units",
                         "peak_kind": f"measured here: FP64 FMA probe (8 chains per thread, "
                                      f"{probe_ms:.1f} ms launch)"},
            "clocks": clocks}, o64


def cufft_leg(x, out, o64, dev, stream, steps: int):
    """Comparison baseline on the same GPU: torch.fft (cuFFT) r2c / c2r around one hand-written
    projector kernel over the half spectrum (eqm_project_half, the same per-mode Q S Q), FP32
    and FP64; and the two transforms alone, the floor of any cuFFT-based projection."""
    import torch
    from paper_2105_01612_gb300 import _measure
    nz, ny, nx = x.shape[-3:]
    res = {"method": "torch.fft.rfftn over (z, y, x) of the six planes, eqm_project_half in "
                     "place on the half spectrum, torch.fft.irfftn; norms not computed"}
    w = torch.tensor([1.0, 1, 1, 2, 2, 2], device=dev, dtype=torch.float64).view(6, 1, 1, 1)
    for name, dt, code, ref in (("f32", torch.float32, 0, out[0]), ("f64", torch.float64, 1, o64[0])):
        xs = x[0].to(dt)

        def xi(m):
            k = torch.arange(m, dtype=torch.float64)
            sgn = torch.where(k < m / 2, k, k - m)
            v = torch.sin(2 * math.pi * sgn / m)
            if m % 2 == 0:
                v[m // 2] = 0.0
            return v.to(dt).to(dev)
        xx, xy, xz = xi(nx)[: nx // 2 + 1].contiguous(), xi(ny), xi(nz)

        def both():
            sh = torch.fft.rfftn(xs, dim=(-3, -2, -1))
            _measure.project_half(code, sh.data_ptr(), nz, ny, nx // 2 + 1, xx.data_ptr(),
                                  xy.data_ptr(), xz.data_ptr(), stream.cuda_stream)
            return torch.fft.irfftn(sh, s=(nz, ny, nx), dim=(-3, -2, -1))

        def transforms():
            return torch.fft.irfftn(torch.fft.rfftn(xs, dim=(-3, -2, -1)), s=(nz, ny, nx),
                                    dim=(-3, -2, -1))

        times = {}
        for key, fn in (("cufft_plus_kernel_ms", both), ("cufft_only_ms", transforms)):
            for _ in range(2):
                y = fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                y = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            times[key] = e0.elapsed_time(e1) / steps
            if key == "cufft_plus_kernel_ms":
                dd = y.double() - ref.double()
                times["rel_l2_vs_ours"] = math.sqrt(float((w * dd * dd).sum() /
                                                          (w * ref.double() ** 2).sum()))
                del dd
            del y
        torch.cuda.empty_cache()
        res[name] = times
    vox = nx * ny * nz
    res["value"] = vox / (res["f32"]["cufft_plus_kernel_ms"] / 1e3)
    res["unit"] = UNIT
    res["ms_per_step"] = res["f32"]["cufft_plus_kernel_ms"]
    return res


def kernel_traffic(dominant: str):
    """DRAM traffic per launch of `dominant` from the committed ncu summary, if the kernel
    sources are unchanged since it was taken (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic_512cubed_fp32.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != source_hash():
        return None
    return d.get("traffic_bytes_per_launch", {}).get(dominant)


# the sources that define and instantiate the five pass kernels of the fixed-size path
PASS_KERNEL_SOURCES = ("eq_dispatch.cuh", "eq_f32.cu", "eq_f64.cu", "eq_fft.cuh", "eq_fft_pair.cuh",
                       "eq_internal.h", "eq_kernels.cuh", "eq_tma.cuh", "eq_xrow.cuh")


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2105_01612_gb300", "csrc")
    for f in PASS_KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def job_timing(ms_local: float, voxels_per_rank: int, steps: int, world: int, device=None):
    """The whole job's timed region and throughput.  Every rank projects its own field (replicas,
    no data exchanged), so the job takes the slowest rank's time (a MAX all-reduce over the
    default process group) and processes world x voxels x steps voxels in it."""
    ms_total = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    return ms_total, world * voxels_per_rank * steps / (ms_total / 1e3)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from fieldgen import voronoi_stress_field
    import paper_2105_01612_gb300 as eq
    from paper_2105_01612_gb300 import _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_base = None
    if rank == 0 and not args.no_extras:
        cpu_base = cpu_oracle_sample(N)            # before any CUDA work on this process
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    _build.build()
    n = args.size
    gx, gy, gz = args.grid if args.grid else (n, n, n)
    vox = gx * gy * gz
    x = voronoi_stress_field((gz, gy, gx), max(8, GRAINS * vox // N ** 3), 200.0, 20.0, SEED + rank,
                             dtype=torch.float32, device=dev).unsqueeze(0).contiguous()
    out = torch.empty_like(x)
    plan = eq.Plan(gx, gy, gz, torch.float32, 1, "ddo", device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        plan.project(x, out)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(dev)
    clk = ClockSampler(str(getattr(props, "uuid", "")))
    clk.start()
    time.sleep(0.1)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.project(x, out)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # per-pass device times: the same projections again, launched pass by pass with events
    # between the passes (the timed region above replays the plan's CUDA graph, the default path)
    kp = max(3, min(args.steps, 20))
    plan.set_timing(kp)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(kp):
        plan.project(x, out)
    p1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms_passes_step = p0.elapsed_time(p1) / kp
    ms_total, value = job_timing(e0.elapsed_time(e1), vox, args.steps, world, dev)
    per_pass, ncalls = plan.pass_ms()
    nrm = plan.norms()[0]
    ms_step = ms_total / args.steps

    # roofline of the dominant kernel: algorithmic bytes per launch / mean launch time
    peak, peak_kind = measured_peaks()
    big = {k: v for k, v in per_pass.items() if "finalise" not in k}
    dominant = max(big, key=big.get)
    dom_ms = per_pass[dominant] / max(1, ncalls)
    dom_bytes = BYTES_PER_VOXEL_PASS * vox + (24 * vox if dominant == "z_inverse" else 0)
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = kernel_traffic(dominant)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{gx}x{gy}x{gz} periodic field, {GRAINS * vox // N ** 3} Voronoi "
                               f"grains N(0,200 MPa) + noise N(0,20 MPa), FP32, DDO, one field per GPU",
                   "grid": [gx, gy, gz], "op": "ddo", "nyq": "keep", "batch_per_gpu": 1,
                   "l2": "inputs larger than L2 (3.2 GB per field); no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic,
                     "algorithmic_bytes_per_launch": dom_bytes},
        "pipeline": {"pass_ms": {k: v / max(1, ncalls) for k, v in per_pass.items()},
                     "pass_timing": f"{ncalls} further projections launched pass by pass with "
                                    f"events between passes, right after the timed region "
                                    f"(graph replay there): {ms_passes_step:.3f} ms per step",
                     "algorithmic_frac": BYTES_PER_VOXEL_PASS * vox / (ms_step / 1e3) / 1e9 / peak,
                     "five_pass_frac": 5 * BYTES_PER_VOXEL_PASS * vox / (ms_step / 1e3) / 1e9 / peak},
        "timing": "CUDA events on the launch stream around K replays of the plan's captured "
                  "CUDA graph (the default eq_project path)",
        "gpu_launches": 8 * args.steps,
        "clocks": clocks,
        "norms": {k: nrm[k] for k in ("norm_in", "norm_out", "resid_rel", "div_in_l2", "div_out_l2")},
    }
    if rank == 0 and not args.no_extras:
        # end to end through the C ABI with pinned host buffers (copies inside the timed region).
        # Headline: eq_project_host_async on three plans and three streams, three fields in flight
        # (the host link runs both directions at once, so one field's copy in overlaps another's
        # copy out and a third's projection); each step copies its field in, projects it, copies
        # it back and reads its norms.  Also the one-at-a-time blocking call.
        depth = 3
        hin = x.cpu().pin_memory()
        houts = [torch.empty_like(hin).pin_memory() for _ in range(depth)]
        # fresh plans: none of the headline plan's timing state carries over
        plans = tuple(eq.Plan(n, n, n, torch.float32, 1, "ddo", device=dev) for _ in range(depth))
        streams = tuple(torch.cuda.Stream(dev) for _ in range(depth))
        for k in range(2 * depth):
            j = k % depth
            if k >= depth:
                plans[j].norms()
            plans[j].project_host(hin, houts[j], stream=streams[j], wait=False)
        for j in range(depth):
            plans[j].norms()
        # the host link is shared with the machine's other GPUs, so one window can catch
        # another tenant's traffic: time three windows and report the median (all are listed)
        ke = max(2 * depth, min(args.steps, 10))
        windows = []
        for _ in range(3):
            t0 = time.perf_counter()
            for k in range(ke):
                j = k % depth
                if k >= depth:
                    plans[j].norms()              # step k - depth done: output and norms read
                plans[j].project_host(hin, houts[j], stream=streams[j], wait=False)
            for j in range(depth):
                plans[j].norms()
            windows.append((time.perf_counter() - t0) / ke)
        te = statistics.median(windows)
        plans[0].project_host(hin, houts[0])
        t0 = time.perf_counter()
        ks = max(1, min(args.steps, 5))
        for _ in range(ks):
            plans[0].project_host(hin, houts[0])
            plans[0].norms()
        ts = (time.perf_counter() - t0) / ks
        line["e2e"] = {"value": vox / te, "unit": UNIT, "h2d_bytes_per_step": hin.numel() * 4,
                       "d2h_bytes_per_step": hin.numel() * 4 + 112,
                       "ms_per_step": te * 1e3, "steps": 3 * ke,
                       "windows_ms": [w * 1e3 for w in windows],
                       "method": "eq_project_host_async, three plans on three streams (three "
                                 "fields in flight), pinned host buffers, norms read every step; "
                                 f"median of three windows of {ke} steps",
                       "blocking_call": {"value": vox / ts, "ms_per_step": ts * 1e3,
                                         "method": "eq_project_host (waits for each field)"}}
        for q in plans:
            q.close()
        link = link_leg(hin, houts[0], dev)
        link["e2e_frac_of_link_bound"] = link["both_ms_per_field"] / (te * 1e3)
        line["e2e"]["host_link"] = link
        del hin, houts
        # the FP64 path on the same field, against the FP64 FMA rate measured here
        fp64, o64 = fp64_leg(x, out, n, dev, stream)
        line["fp64"] = fp64
        # cuFFT (r2c / c2r) with and without one hand-written projector kernel, FP32 and FP64
        line["cufft_baseline"] = cufft_leg(x, out, o64, dev, stream, max(1, min(args.steps, 5)))
        del o64
        torch.cuda.empty_cache()
        if not args.grid:
            line["grain_average"] = grain_leg(x, out, plan, n, dev, stream, peak)
        line["cpu_baseline"] = cpu_base
        del x, out
        plan.close()
        torch.cuda.empty_cache()
        line["batch"] = batch_leg(dev, max(3, min(args.steps, 10)))
        torch.cuda.empty_cache()
        line["serving"] = serving_leg(dev)
        line["serving"]["fresh_shapes"] = serving_leg(dev, fresh=True)
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def grain_leg(x, out, plan, n, dev, stream, peak):
    """Sec. 5.1 / Table 1 workload on the headline field: average it over its 5000 grains (the
    map the field was generated from), then project the grain average.  Times the averaging
    (per-grain FP64 means + the averaged field) and the average-then-project step."""
    import torch
    from fieldgen import periodic_voronoi_map
    import paper_2105_01612_gb300 as eq
    t0 = time.perf_counter()
    gmap = periodic_voronoi_map((n, n, n), GRAINS, SEED)
    gr = eq.Grains(gmap, GRAINS, device=dev)
    setup_s = time.perf_counter() - t0
    del gmap
    avg = torch.empty_like(x)
    means, _ = gr.average(x, out=avg)
    torch.cuda.synchronize()
    k = 5
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(k):
        gr.average(x, means=means, out=avg)
    e1.record(stream)
    for _ in range(k):
        gr.average(x, means=means, out=avg)
        plan.project(avg, out)
    e2.record(stream)
    torch.cuda.synchronize()
    ms_avg = e0.elapsed_time(e1) / k
    ms_both = e1.elapsed_time(e2) / k
    vox = n ** 3
    alg = 56 * vox          # field read 24 B, voxel list 4 B, grain map 4 B, averaged field 24 B
    gr.close()
    del avg, means
    return {"workload": f"{n}^3 headline field averaged over its {GRAINS} Voronoi grains, then "
                        "projected (Sec. 5.1 recovery from grain-averaged data)",
            "ms_average": ms_avg, "average_gbs": alg / (ms_avg / 1e3) / 1e9,
            "average_frac_of_peak": alg / (ms_avg / 1e3) / 1e9 / peak,
            "ms_average_then_project": ms_both,
            "value": vox / (ms_both / 1e3), "unit": UNIT, "grain_map_setup_s": setup_s}


def batch_leg(dev, steps: int, nfields: int = 64, tune: bool = True):
    """64 fields, each axis uniform in 64..256, Voronoi 50..2000 grains ~ N(0,150 MPa), FP32, DDO:
    one launch per pass over all fields, replayed from a captured CUDA graph.  nfields < 64 keeps
    the first fields of the same draw (profiling cases); tune=False keeps the default shapes."""
    import numpy as np
    import torch
    from fieldgen import voronoi_stress_field
    import paper_2105_01612_gb300 as eq
    rng = np.random.Generator(np.random.PCG64(210501612 + 3))
    dims = [tuple(int(v) for v in rng.integers(64, 257, size=3)) for _ in range(64)][:nfields]
    grains = [int(g) for g in rng.integers(50, 2001, size=64)][:nfields]
    plan = eq.VarlenPlan(dims, torch.float32, "ddo", device=dev)
    flat = torch.empty(plan.numel, dtype=torch.float32, device=dev)
    off = 0
    for i, (nx, ny, nz) in enumerate(dims):
        n = 6 * nx * ny * nz
        flat[off:off + n] = voronoi_stress_field((nz, ny, nx), grains[i], 150.0, 0.0,
                                                 210501612 + 3 + i, dtype=torch.float32,
                                                 device=dev).reshape(-1)
        off += n
    out = torch.empty_like(flat)
    # radix / tile choices per pass: the plan's autotuner (cached in $EQ_TUNE_CACHE, a file of
    # the run's temporary directory unless the caller names one)
    os.environ.setdefault("EQ_TUNE_CACHE", os.path.join("/tmp", f"eq_tune_{os.getpid()}.txt"))
    t0 = time.perf_counter()
    if tune:
        plan.autotune(flat, out)
    tune_s = time.perf_counter() - t0
    for _ in range(3):
        plan.project(flat, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.current_stream(dev)
    e0.record(st)
    for _ in range(steps):
        plan.project(flat, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    vox = plan.numel // 6
    plan.set_timing(1)
    plan.project(flat, out)
    per_pass, _ = plan.pass_ms()
    plan.close()
    peak, _ = measured_peaks()
    return {"workload": f"{nfields} fields, axes uniform 64..256, 50..2000 Voronoi grains, FP32, "
                        "DDO; one launch per pass over all fields, CUDA graph replay",
            "voxels": vox, "value": vox / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "pass_ms": per_pass, "autotune_s": tune_s,
            "pass_frac": {k: BYTES_PER_VOXEL_PASS * vox / (v / 1e3) / 1e9 / peak
                          for k, v in per_pass.items() if "finalise" not in k and v > 0},
            "algorithmic_frac": BYTES_PER_VOXEL_PASS * vox / (ms / 1e3) / 1e9 / peak}


def serving_leg(dev, rate: float = 200.0, warm: int = 200, measured: int = 2000,
                pool_size: int = 48, fresh: bool = False):
    """Poisson arrivals at `rate` req/s of single fields, each axis log-uniform in [32, 256],
    FP32 Voronoi fields, admitted by HBM footprint; p50/p99 latency from submit to completion
    and completed voxels/s.  fresh=False: a pool of `pool_size` pre-generated fields, cycled
    (after warm-up every plan is cached); fresh=True: every request draws its own grid (about
    10^7 possible shapes, so nearly every request needs a new plan), its values the leading
    part of one pre-generated 256^3 Voronoi field."""
    import numpy as np
    import torch
    from fieldgen import voronoi_stress_field, log_uniform_int
    import paper_2105_01612_gb300 as eq
    rng = np.random.Generator(np.random.PCG64(210501612 + 4 + (1000 if fresh else 0)))
    nreq = warm + measured
    if fresh:
        big = voronoi_stress_field((256, 256, 256), 2000, 150.0, 0.0, 210501612 + 4,
                                   dtype=torch.float32, device=dev).cpu().reshape(-1).pin_memory()
        shapes = [tuple(log_uniform_int(rng, 32, 256) for _ in range(3)) for _ in range(nreq)]
        nbuf = 16
        outs = [torch.empty(big.numel(), dtype=torch.float32).pin_memory() for _ in range(nbuf)]

        def field(i):
            nx, ny, nz = shapes[i]
            n = 6 * nx * ny * nz
            return big[:n].view(6, nz, ny, nx), outs[i % nbuf][:n].view(6, nz, ny, nx), i % nbuf
    else:
        pool = []
        for i in range(pool_size):
            nx, ny, nz = (log_uniform_int(rng, 32, 256) for _ in range(3))
            g = int(rng.integers(50, 2001))
            f = voronoi_stress_field((nz, ny, nx), g, 150.0, 0.0, 210501612 + 4 + i,
                                     dtype=torch.float32, device=dev).cpu().pin_memory()
            pool.append((f, torch.empty_like(f).pin_memory()))

        def field(i):
            f, o = pool[i % pool_size]
            return f, o, i % pool_size
    srv = eq.Server(64 << 30, max_inflight=8, device=dev)
    gaps = rng.exponential(1.0 / rate, size=nreq)
    pending = {}
    busy_out = {}
    lat, vox_done, offered = [], 0, []
    t_next = time.perf_counter()
    t_meas0 = None
    t_last = None
    st0 = None

    def drain(block: bool):
        nonlocal vox_done, t_last
        for tk in list(pending):
            r = srv.poll(tk, 0) if not block else srv.wait(tk)
            if r is None:
                continue
            i, nv, k = pending.pop(tk)
            busy_out.pop(k, None)
            if i >= warm:
                lat.append(r[1])
                vox_done += nv
                t_last = time.perf_counter()

    for i in range(nreq):
        t_next += gaps[i]
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            drain(False)
            time.sleep(min(2e-4, max(0.0, t_next - now)))
        if i == warm:
            t_meas0 = time.perf_counter()
            st0 = srv.stats()
        f, o, k = field(i)
        if k in busy_out:                      # output buffer still in use: wait for it
            tk_prev = busy_out[k]
            r = srv.wait(tk_prev)
            j, nv, _ = pending.pop(tk_prev)
            busy_out.pop(k, None)
            if j >= warm:
                lat.append(r[1])
                vox_done += nv
                t_last = time.perf_counter()
        tk = srv.submit(f, o)
        pending[tk] = (i, f.numel() // 6, k)
        busy_out[k] = tk
        offered.append(f.numel() // 6)
    drain(True)
    st1 = srv.stats()
    srv.close()
    wall = (t_last or time.perf_counter()) - t_meas0
    lat_ms = sorted(1e3 * v for v in lat)
    q = lambda p: lat_ms[min(len(lat_ms) - 1, int(round(p * (len(lat_ms) - 1))))]
    created = st1["plans_created"] - st0["plans_created"]
    plan_s = st1["plan_create_seconds"] - st0["plan_create_seconds"]
    what = ("every request a fresh grid (one 256^3 Voronoi field's leading values)" if fresh
            else f"{pool_size} pre-generated Voronoi fields cycled")
    return {"workload": f"Poisson {rate:g} req/s, single FP32 fields, axes log-uniform 32..256, "
                        f"{what}, 8 slots, 64 GiB budget",
            "requests": len(lat_ms), "warmup_requests": warm, "p50_ms": q(0.5), "p99_ms": q(0.99),
            "max_ms": lat_ms[-1], "value": vox_done / wall, "unit": UNIT,
            "offered_voxels_per_s": rate * float(np.mean(offered)),
            "plans_created": created, "plans_reused": st1["plans_reused"] - st0["plans_reused"],
            "plans_evicted": st1["plans_evicted"] - st0["plans_evicted"],
            "plan_create_ms_mean": 1e3 * plan_s / max(1, created),
            "plan_thread_busy_frac": plan_s / wall, "inflight_peak": st1["inflight_peak"],
            "hbm_in_use_peak_gib": st1["hbm_in_use_peak"] / 2 ** 30}


def main():
    args = parse()
    if args.fp64_only:
        print(json.dumps(fp64_case(args)), flush=True)
        return
    if args.batch_fields:
        import torch
        print(json.dumps(batch_leg(torch.device("cuda", 0), args.steps, args.batch_fields,
                                   tune=False)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
