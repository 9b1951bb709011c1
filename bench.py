"""Benchmark of the fused compressible-Euler step on GB300.

Default workload: 3D single-fluid Rayleigh-Taylor, 256^3 cells on
[0,1]x[0,1]x[0,2], FP64, periodic x/y, reflecting z, g = -1, seeded
multimode perturbation; a bench step is one full time step (one fused
kernel launch) of the whole grid.  Metric: zone-updates/s (cells x steps /
s), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

One JSON line is printed by rank 0.  Under torchrun (N > 1) each rank runs
an independent replica on its own GPU (the update does not shard across
GPUs here), timing is max over ranks, and value = all ranks' zone-updates /
that time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1510_05061_gb300 import inputs  # noqa: E402

METRIC = "zone-updates/s"
UNIT = "zone-updates/s"

# Algorithmic work per zone-update of the fused step: bytes = read U^n once +
# write U^{n+1} once = 2 * nvar * sizeof(T); floating-point operations of the
# scheme counted once per cell and once per face (ndim faces per cell),
# divisions, square roots and min/max counted as one operation each:
# 3D = primitives 13 + MC slopes 75 + half step 83 + face states 60 +
#      3 HLLC x 72 + update 70 + CFL speed 25 = 542;
# 2D = 10 + 40 + 50 + 32 + 2 x 64 + 42 + 19 = 321.
FLOPS_PER_ZONE_3D = 542
FLOPS_PER_ZONE_2D = 321
# SSP-RK2 method of lines, per step: two stages without the half step
# (3D 13 + 75 + 60 + 216 + 70 = 434, 2D 10 + 40 + 32 + 128 + 42 = 252), the
# stage average (2 per variable) and one CFL speed.  Bytes per zone-update:
# stage 1 reads U and writes U1, stage 2 reads U1 and U and writes U^{n+1}.
FLOPS_PER_ZONE_3D_RK2 = 2 * 434 + 10 + 25
FLOPS_PER_ZONE_2D_RK2 = 2 * 252 + 8 + 19
# PPM face states instead of W -/+ dW/2, per variable and axis: the interface
# value (5) and the monotone-parabola limiter (14) on top of the MC slope:
# 3D stage 13 + 75 + 15 x 19 + 216 + 70 = 659, 2D 10 + 40 + 8 x 19 + 128 + 42 = 372.
FLOPS_PER_ZONE_3D_PPM = 2 * 659 + 10 + 25
FLOPS_PER_ZONE_2D_PPM = 2 * 372 + 8 + 19
# Corner transport upwind, per step: primitives, slopes, three (two) one-axis
# predictors of 35 each, face states, first-pass HLLC, the corrections of
# both face states per axis (to conserved, two transverse differences, back:
# 42 per state; 2D 26), final HLLC, update and CFL speed.
FLOPS_PER_ZONE_3D_CTU = 13 + 75 + 3 * 35 + 60 + 216 + 3 * 2 * 42 + 216 + 70 + 25
FLOPS_PER_ZONE_2D_CTU = 10 + 40 + 2 * 25 + 32 + 128 + 2 * 2 * 26 + 128 + 42 + 19

# tile shape of each 3D variant; variants 4..7 stage the next plane asynchronously
TILE_NAMES = {0: "32, 8", 1: "32, 4", 2: "16, 16", 3: "32, 16", 4: "32, 8", 5: "32, 4", 6: "16, 16", 7: "32, 16"}
# paired-cell FP32 variants: threads (x, y) per tile (two x-adjacent cells per thread)
PAIR_THREADS = {8: (16, 16), 9: (16, 8), 10: (8, 16)}

CONFIGS = {
    # name: (builder, description, precision, hse)
    "rt256-fp64": dict(n=256, precision=inputs.FP64, hse=0,
                       desc="3D single-fluid Rayleigh-Taylor 256^3 FP64 (g=-1, modes 4-16, amp 0.01), 200-step run"),
    "rt256-fp64-hse": dict(n=256, precision=inputs.FP64, hse=1,
                           desc="3D Rayleigh-Taylor 256^3 FP64 with hydrostatic-background subtraction"),
    "rt512-fp32": dict(n=512, precision=inputs.FP32, hse=1,
                       desc="3D Rayleigh-Taylor 512^3 FP32 bulk, FP64 dt/totals/background subtraction"),
    "rt256-fp32": dict(n=256, precision=inputs.FP32, hse=1,
                       desc="3D Rayleigh-Taylor 256^3 FP32 bulk with hydrostatic-background subtraction"),
    "sod128": dict(kind="sod", n=128, precision=inputs.FP64, hse=0,
                   desc="2D Sod shock tube 128^2 FP64 (latency-bound: 0.5 MB state fits in L2)"),
    "kh2d-2048-fp32": dict(kind="kh2d", n=2048, precision=inputs.FP32, hse=0,
                           desc="2D Kelvin-Helmholtz 2048^2 FP32 (largest 2D served size)"),
    "served": dict(served=True, rate=50.0,
                   desc="served workload: Poisson arrivals (50/s, seed 151005063), 50/50 2D KH n in [64, 2048] "
                        "and 3D RT n in [32, 256] (log-uniform), 100-1000 steps each, FP32 with FP64 "
                        "reductions, 150 GB HBM budget, continuous batching"),
    "served-saturation": dict(served=True, rate=500.0,
                              desc="served workload as above with arrivals 10x faster (saturation run)"),
    "served-light": dict(served=True, rate=10.0,
                         desc="served workload as above with arrivals at 10/s (a load the GPU carries: "
                              "latency without queueing)"),
    "rt256-fp64-rk2": dict(n=256, precision=inputs.FP64, hse=0, scheme=inputs.SSPRK2,
                           desc="3D Rayleigh-Taylor 256^3 FP64 with the SSP-RK2 method-of-lines integrator "
                                "(two stage kernels per step)"),
    "rt512-fp32-rk2": dict(n=512, precision=inputs.FP32, hse=1, scheme=inputs.SSPRK2,
                           desc="3D Rayleigh-Taylor 512^3 FP32 bulk with background subtraction, SSP-RK2 "
                                "method of lines"),
    "rt256-fp64-ppm": dict(n=256, precision=inputs.FP64, hse=0, scheme=inputs.SSPRK2, recon=inputs.PPM,
                           desc="3D Rayleigh-Taylor 256^3 FP64, SSP-RK2 method of lines with PPM face states"),
    "rt512-fp32-ppm": dict(n=512, precision=inputs.FP32, hse=0, scheme=inputs.SSPRK2, recon=inputs.PPM,
                           desc="3D Rayleigh-Taylor 512^3 FP32 (FP64 dt and reductions), SSP-RK2 with PPM"),
    "rt256-fp64-ctu": dict(n=256, precision=inputs.FP64, hse=0, scheme=inputs.CTU,
                           desc="3D Rayleigh-Taylor 256^3 FP64, corner transport upwind (one fused kernel per step)"),
    "rt512-fp32-ctu": dict(n=512, precision=inputs.FP32, hse=1, scheme=inputs.CTU,
                           desc="3D Rayleigh-Taylor 512^3 FP32 bulk with background subtraction, corner "
                                "transport upwind"),
    "rt256-fp64-slabs4": dict(n=256, precision=inputs.FP64, hse=0, slabs=4,
                              desc="3D Rayleigh-Taylor 256^3 FP64 cut into 4 z slabs run as virtual ranks "
                                   "(depth-2 halo exchange + dt max-reduction every step)"),
    "kh-batch": dict(batch=True, count=64, precision=inputs.FP32,
                     desc="64 independent 3D periodic Kelvin-Helmholtz boxes, n log-uniform in [32, 192] "
                          "(seed 151005062), FP32; one persistent launch per step, autotuned tiles"),
}


def step_kernel_names(prob, variant: int):
    """The kernels of one step of `prob` with 3D tile variant `variant`, as
    the profiler prints their names (the keys of profiles/traffic.json)."""
    itemsize = 4 if prob.precision == inputs.FP32 else 8
    rk2 = prob.scheme == inputs.SSPRK2
    tile = TILE_NAMES.get(variant, "32, 8") if prob.ndim == 3 else "32, 8"
    tname = "double" if itemsize == 8 else "float"
    stages = (1, 2) if rk2 else (0,)
    # template arguments: stage, reconstruction, staging depth (the tuned one
    # for the MUSCL-Hancock step, the precision's default for the stages),
    # and whether the FP64 MUSCL-Hancock step takes the kernel for gravity
    # along z only (without the x and y gravity terms)
    async_flag = int(variant >= 4) if not rk2 else int(itemsize == 8)
    gz = int(itemsize == 8 and not rk2 and bool(prob.hse_subtract or (prob.grav[0] == 0 and prob.grav[1] == 0)))
    if prob.scheme == inputs.CTU:
        return [f"ctu3d_kernel<{tname}, {prob.hse_subtract}, 16, {16 if itemsize == 4 else 8}>" if prob.ndim == 3
                else f"ctu2d_kernel<{tname}, 32, 8>"]
    if prob.ndim == 3 and variant in PAIR_THREADS and not rk2 and itemsize == 4:
        # paired-cell FP32 MUSCL-Hancock step: threads (x, y) of the tile
        pgz = int(bool(prob.hse_subtract or (prob.grav[0] == 0 and prob.grav[1] == 0)))
        txp, typ = PAIR_THREADS[variant]
        minb = 2 if variant == 8 else 3
        return [f"step3d_pair_kernel<{prob.hse_subtract}, {txp}, {typ}, {pgz}, {minb}>"]
    return [(f"step3d_kernel<{tname}, {prob.hse_subtract}, {tile}, {st}, {prob.recon}, {async_flag}, {gz}>"
             if prob.ndim == 3 else f"step2d_kernel<{tname}, 32, 8, {st}, {prob.recon}>") for st in stages]


# translation units that compile (and launch) each kernel family; a kernel's
# source hash covers them and every csrc header they include
KERNEL_UNITS = {
    "step3d_kernel": ("step3d_f64.cu", "step3d_f32.cu", "stage3d_f64.cu", "stage3d_f32.cu"),
    "step3d_pair_kernel": ("pair3d_f32.cu",),
    "step3d_batch_kernel": ("batch3d_f64.cu", "batch3d_f32.cu"),
    "step2d_kernel": ("step2d.cu",),
    "step2d_batch_kernel": ("batch2d.cu",),
    "ctu3d_kernel": ("ctu3d.cu",),
    "ctu2d_kernel": ("ctu2d.cu",),
}


def _csrc_closure(units):
    """The units and every csrc file they include, transitively."""
    import re

    csrc = os.path.join(ROOT, "paper_1510_05061_gb300", "csrc")
    seen, todo = set(), list(units)
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(csrc, f)):
            continue
        seen.add(f)
        with open(os.path.join(csrc, f)) as fh:
            todo += [m for m in re.findall(r'#include\s+"([^"/]+)"', fh.read())]
    return sorted(seen)


def kernel_source_sha(kernel: str = "") -> str:
    """Hash of the CUDA sources a kernel is built from (its family's
    translation units and the csrc headers they include; every source when
    the kernel is not known): measured traffic is valid only for the
    sources it was taken from."""
    import glob
    import hashlib

    csrc = os.path.join(ROOT, "paper_1510_05061_gb300", "csrc")
    family = kernel.split("<")[0].strip()
    if family in KERNEL_UNITS:
        files = [os.path.join(csrc, f) for f in _csrc_closure(KERNEL_UNITS[family])]
    else:
        files = [f for f in sorted(glob.glob(os.path.join(csrc, "*"))) if f.endswith((".cu", ".cuh", ".h"))]
    h = hashlib.sha1()
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(config: str, kernel: str):
    """DRAM bytes per launch of `kernel` on `config` from the committed ncu
    table (profiles/traffic.json), or None when absent or stale."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        return None
    e = table.get(config, {}).get(kernel)
    if not e or e.get("source_sha") != kernel_source_sha(kernel):
        return None
    return float(e["bytes_per_launch"])


def record_traffic(config: str, csv_path: str, scale: float = 1.0, note: str = "") -> int:
    """Read an ncu CSV (--csv --log-file) of this benchmark taken with
    --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum,
    store each kernel's mean DRAM bytes per launch for `config` in
    profiles/traffic.json (with the current source hash) and print the launch
    list (launches, device time, share, traffic) as a markdown table.  With
    scale != 1 the capture was taken on a smaller grid of the workload and
    its bytes are scaled to the workload's cells (traffic proportional to
    the cells processed); `note` says so in the table."""
    import csv
    import re

    per = {}
    with open(csv_path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    for row in csv.DictReader(lines):
        name = re.sub(r"^void\s+", "", row["Kernel Name"])
        name = re.sub(r"\(.*\)$", "", name).strip()
        name = re.sub(r"^(\w+::|\(anonymous namespace\)::|<?unnamed>::)+", "", name)
        d = per.setdefault(name, {})
        d.setdefault(row["ID"], {})[row["Metric Name"]] = float(row["Metric Value"].replace(",", ""))
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        table = {}
    # entries of this workload taken from other sources are stale: drop them
    table[config] = {k: v for k, v in table.get(config, {}).items()
                     if v.get("source_sha") == kernel_source_sha(k)}
    rows = []
    total_ns = 0.0
    for name, launches in per.items():
        ns = sum(m.get("gpu__time_duration.sum", 0.0) for m in launches.values())
        byts = [m.get("dram__bytes_read.sum", 0.0) + m.get("dram__bytes_write.sum", 0.0) for m in launches.values()]
        rows.append((name, len(launches), ns, sum(byts) / len(byts)))
        total_ns += ns
        entry = {"bytes_per_launch": scale * sum(byts) / len(byts), "launches": len(launches),
                 "source_sha": kernel_source_sha(name)}
        if scale != 1.0:
            entry["scaled"] = note or f"captured on a smaller grid, bytes x {scale:g}"
        table.setdefault(config, {})[name] = entry
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    print("| kernel | launches | device time (ms) | share | DRAM bytes per launch |")
    print("|---|---:|---:|---:|---:|")
    for name, n, ns, b in sorted(rows, key=lambda r: -r[2]):
        print(f"| `{name}` | {n} | {ns / 1e6:.3f} | {ns / total_ns:.1%} | {b / 1e9:.3f} GB |")
    return 0


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def fp64_peak_tflops(sm_mhz: float) -> float:
    """Dense FP64 peak from unit counts and clock: 152 SMs x 2 FP64 FMA/clk
    x 2 flop x clock (1.26 TFLOP/s at 2070 MHz, the part's nominal figure)."""
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def measure_fma_peak(precision: int, target_ms: float = 40.0) -> dict:
    """Measured FMA-pipe throughput of one precision on the current device:
    the library's probe kernel (8 CTAs of 256 threads per SM, 8 independent
    FMA chains per thread) timed with CUDA events on its stream, best of
    three launches of about target_ms each, with the SM clock sampled."""
    import torch

    from paper_1510_05061_gb300 import hydro

    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ctas, threads = 8 * sms, 256
    dt = torch.float64 if precision == inputs.FP64 else torch.float32
    out = torch.empty(ctas * threads, dtype=dt, device="cuda")
    s = torch.cuda.current_stream()

    def timed(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        hydro.hydro_fma_probe(precision, iters, ctas, threads, out.data_ptr(), s.cuda_stream)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1)

    iters = 2000 if precision == inputs.FP64 else 100000
    timed(iters)
    ms = timed(iters)
    iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
    with ClockSampler(dev) as clk:
        best = min(timed(iters) for _ in range(3))
    flops = hydro.hydro_fma_probe_flops(iters, ctas, threads)
    return {"tflops": flops / (best * 1e-3) / 1e12, "ms": best, "iters": iters, "ctas": ctas,
            "threads": threads, "clocks": clk.summary(),
            "how": "FMA probe kernel: 8 CTAs x 256 threads per SM, 8 independent chains x <- x*a + b "
                   "per thread, CUDA events, best of 3"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


GRID_OVERRIDE = None   # --n: profiling runs of an RT workload on a smaller grid


def build_workload(cfg):
    c = dict(CONFIGS[cfg])
    if GRID_OVERRIDE is not None and c.get("kind", "rt") == "rt" and "n" in c:
        c["n"] = GRID_OVERRIDE
    if c.get("batch") or c.get("served"):
        raise ValueError("batch and served configs have no single workload")
    kind = c.get("kind", "rt")
    if kind == "sod":
        prob, W = inputs.sod(c["n"], precision=c["precision"])
    elif kind == "kh2d":
        prob, W = inputs.kelvin_helmholtz(c["n"], ndim=2, U=1.0, ratio=2.0, precision=c["precision"])
    else:
        prob, W = inputs.rayleigh_taylor(c["n"], precision=c["precision"], hse_subtract=c["hse"])
    prob = prob.replace(scheme=c.get("scheme", inputs.HANCOCK), recon=c.get("recon", inputs.PLM))
    return prob, W, c


# --------------------------------------------------------------- oracle
def host_cpu_model() -> str:
    """The host CPU's model name as lscpu prints it ("" when unavailable)."""
    import subprocess

    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return ""
    for line in out.splitlines():
        if line.strip().startswith("Model name:"):
            return line.split(":", 1)[1].strip()
    return ""


def oracle_sample(seconds: float = 10.0, max_steps: int = 1000, cfg="rt256-fp64", nz_slab=None,
                  threads: int = 0):
    """Time the FP64 CPU oracle, as it stands, on a bounded sample of the
    workload, on all host cores (threads = 0) or on the given number of
    threads.  Returns (zone-updates/s, cores, sample description)."""
    import oracle

    oracle.build()
    prob, W, c = build_workload(cfg)
    desc = f"full {'x'.join(str(v) for v in prob.n[:prob.ndim])} grid"
    if nz_slab is not None and prob.ndim == 3 and prob.n[2] > nz_slab:
        # a slab of nz_slab planes around the interface, same x-y extent
        k0 = prob.n[2] // 2 - nz_slab // 2
        z_lo = prob.lo[2] + k0 * prob.dx()[2]
        z_hi = z_lo + nz_slab * prob.dx()[2]
        kw = dict(n=(prob.n[0], prob.n[1], nz_slab), lo=(0.0, 0.0, z_lo), hi=(1.0, 1.0, z_hi))
        if prob.hse_subtract:
            kw.update(bg_rho_c=prob.bg_rho_c[k0:k0 + nz_slab + 4], bg_p_c=prob.bg_p_c[k0:k0 + nz_slab + 4],
                      bg_rho_f=prob.bg_rho_f[k0:k0 + nz_slab + 5], bg_p_f=prob.bg_p_f[k0:k0 + nz_slab + 5])
        prob = prob.replace(**kw)
        W = np.ascontiguousarray(W[:, k0:k0 + nz_slab])
        desc = f"{prob.n[0]}x{prob.n[1]}x{nz_slab} slab of the {c['n']}^3 initial state around the interface"
    o = oracle.Oracle(prob, threads=threads)
    U = o.state_from_prim(W)
    cores = o.L.orc_max_threads()
    done, t0 = 0, time.perf_counter()
    while done < max_steps:
        U, _, s, _ = o.run(U, max_steps=1)
        done += s
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return prob.ncell * done / el, cores, f"{desc}, {done} oracle step(s), {el:.1f} s"


def fp32_accuracy(cfg: str, t_end: float = 0.5) -> dict:
    """FP32 error against the FP64 oracle: the FP32 GPU path and the oracle
    run the workload's problem at a reduced grid (RT 64^3, 2D KH 256^2) to
    t_end from the same seeded initial state; density L1-relative
    difference at t_end (about 1-5 s of oracle time on 16 cores)."""
    import oracle

    from paper_1510_05061_gb300 import hydro

    c = CONFIGS[cfg]
    kind = c.get("kind", "rt")
    if kind == "kh2d":
        prob, W = inputs.kelvin_helmholtz(256, ndim=2, U=1.0, ratio=2.0, precision=inputs.FP32)
    else:
        prob, W = inputs.rayleigh_taylor(64, precision=inputs.FP32, hse_subtract=c["hse"])
    prob = prob.replace(scheme=c.get("scheme", inputs.HANCOCK), recon=c.get("recon", inputs.PLM))
    sim = hydro.Simulation(prob, W)
    steps, t = sim.advance_to(t_end)
    rho_gpu = sim.primitive()[0]
    sim.close()
    oracle.build()
    o = oracle.Oracle(prob.replace(precision=inputs.FP64))
    V, to, so, _ = o.run(o.state_from_prim(W), t_end=t_end)
    rho = o.prim(V)[0]
    return {"vs": "FP64 CPU oracle", "grid": list(prob.n[:prob.ndim]), "t": t_end,
            "steps_fp32": steps, "steps_oracle": so,
            "density_l1_rel": float(np.abs(rho_gpu - rho).sum() / np.abs(rho).sum())}


def batch_accuracy(b, items, count: int = 4) -> dict:
    """FP32 batch instances against the FP64 oracle: the `count` smallest
    boxes after the steps they have taken (the oracle takes as many steps from
    the same initial state); the largest density L1-relative difference."""
    import oracle

    oracle.build()
    order = sorted(range(len(items)), key=lambda i: items[i][0].ncell)[:count]
    worst, steps = 0.0, []
    for i in order:
        p, W = items[i]
        n = b.nstep(i)
        rho_gpu = b.conserved(i)[0]
        o = oracle.Oracle(p.replace(precision=inputs.FP64))
        V, _, s, _ = o.run(o.state_from_prim(W), max_steps=n)
        rho = o.total(V)[0]
        worst = max(worst, float(np.abs(rho_gpu - rho).sum() / np.abs(rho).sum()))
        steps.append(n)
    return {"vs": "FP64 CPU oracle, same number of steps", "instances": [items[i][0].n[0] for i in order],
            "steps": steps, "density_l1_rel_max": worst}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    cfg = args.config
    if CONFIGS[cfg].get("batch") or CONFIGS[cfg].get("served"):
        cfg = "rt256-fp64"      # the oracle times a single solve; batches are sums of such solves
    prob, W, c = build_workload(cfg)
    import oracle

    oracle.build()
    nz_slab = 16
    if prob.ndim == 3 and prob.n[2] > nz_slab:
        k0 = prob.n[2] // 2 - nz_slab // 2
        sprob = prob.replace(n=(prob.n[0], prob.n[1], nz_slab),
                             lo=(0.0, 0.0, prob.lo[2] + k0 * prob.dx()[2]),
                             hi=(1.0, 1.0, prob.lo[2] + (k0 + nz_slab) * prob.dx()[2]))
        if prob.hse_subtract:
            sprob = sprob.replace(bg_rho_c=prob.bg_rho_c[k0:k0 + nz_slab + 4], bg_p_c=prob.bg_p_c[k0:k0 + nz_slab + 4],
                                  bg_rho_f=prob.bg_rho_f[k0:k0 + nz_slab + 5], bg_p_f=prob.bg_p_f[k0:k0 + nz_slab + 5])
        Ws = np.ascontiguousarray(W[:, k0:k0 + nz_slab])
        sample_desc = (f"{sprob.n[0]}x{sprob.n[1]}x{nz_slab} slab of the {c['n']}^3 initial state "
                       f"around the interface; one FP64 oracle step per bench step")
    else:
        sprob, Ws = prob, W
        sample_desc = f"the full {'x'.join(str(v) for v in prob.n[:prob.ndim])} grid; one oracle step per bench step"
    o = oracle.Oracle(sprob)
    U = o.state_from_prim(Ws)
    for _ in range(args.warmup):
        U, _, _, _ = o.run(U, max_steps=1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, _, _, _ = o.run(U, max_steps=1)
    el = time.perf_counter() - t0
    value = sprob.ncell * args.steps / el
    cores = o.L.orc_max_threads()
    sample = sample_desc
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": c["desc"], "grid": list(prob.n), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- batch arm
def kh_batch_items(count=64, seed=151005062):
    return [inputs.kelvin_helmholtz(s["n"], ndim=3, U=s["U"], ratio=s["ratio"], seed=seed,
                                    instance=s["instance"], precision=inputs.FP32)
            for s in inputs.kh_batch_sizes(count=count, seed=seed)]


def run_gpu_batch(args):
    import torch

    from paper_1510_05061_gb300 import autotune
    from paper_1510_05061_gb300 import build as hbuild
    from paper_1510_05061_gb300 import hydro

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    hbuild.build()
    hydro.load()
    c = CONFIGS[args.config]
    items = kh_batch_items(c["count"])
    b = hydro.Batch(items)
    if args.no_tune:
        tune = {"variant": 7, "tile": [32, 16], "async_staging": True, "zchunk": 0, "cached": False,
                "note": "library defaults (no autotuning)"}
    else:
        tune = autotune.tune_batch(b, use_cache=not args.retune)
    b.step(args.warmup)
    torch.cuda.synchronize()
    n0 = b.launches()
    s = b.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(s)
        b.step(args.steps)
        ev1.record(s)
        torch.cuda.synchronize()
    barrier(world)
    launches = b.launches() - n0
    el_ms = max_over_ranks(world, ev0.elapsed_time(ev1))
    cells = b.cells()
    value = world * cells * args.steps / (el_ms * 1e-3)
    per_launch_ms = el_ms / args.steps
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = 2 * 5 * 4 * cells / (per_launch_ms * 1e-3) / 1e9
    items3, items2, grid3, grid2 = b.items()
    accuracy = batch_accuracy(b, items) if rank == 0 and not args.no_accuracy else None
    b.close()
    kname = f"step3d_batch_kernel<float, 0, {TILE_NAMES[tune['variant']]}, {int(tune['variant'] >= 4)}>"
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": c["desc"], "instances": len(items), "cells": cells,
                       "tile": tune["tile"], "zchunk": tune["zchunk"], "work_items": items3,
                       "persistent_grid": grid3,
                       "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (cells * 20 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_kind": peak_kind, "kernel": kname,
                         "traffic": args.traffic if args.traffic is not None else measured_traffic(args.config, kname),
                         "algorithmic_bytes": 2 * 5 * 4 * cells},
            "autotune": {k: v for k, v in tune.items() if k != "table"},
            "accuracy": accuracy,
            "cpu_baseline": None, "e2e": None,
            "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- served arm
def run_served(args):
    import torch

    from paper_1510_05061_gb300 import build as hbuild
    from paper_1510_05061_gb300 import hydro, serve

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    hbuild.build()
    hydro.load()
    c = CONFIGS[args.config]
    t0 = time.perf_counter()
    # payloads are built ahead of admission on a background thread
    reqs = serve.requests_from_inputs(count=args.requests, rate=c["rate"], lazy=True)
    prep_s = time.perf_counter() - t0
    # the three cheapest requests' results are kept for the FP32 error against the oracle
    check_ids = {r.id for r in sorted(reqs, key=lambda r: r.n ** (2 if r.family == "kh2d" else 3) * r.steps)[:3]}
    srv = serve.Server(budget_bytes=args.budget_gb * 1e9, max_active=args.max_active)
    barrier(world)
    with ClockSampler(local) as clk:
        stats = srv.run(reqs, keep_results=lambda r: r.id in check_ids)
    srv.close()
    accuracy = None
    if rank == 0 and not args.no_accuracy:
        import oracle

        oracle.build()
        worst, checked = 0.0, []
        for r in reqs:
            if r.id not in check_ids or r.result is None:
                continue
            p = serve.make_payload(serve.Request(id=r.id, arrival=0.0, family=r.family, n=r.n, steps=r.steps,
                                                 seed=r.seed))
            o = oracle.Oracle(p.prob.replace(precision=inputs.FP64))
            V, _, _, _ = o.run(o.state_from_prim(p.W), max_steps=r.steps)
            rho = o.total(V)[0]
            rho_gpu = o.total(r.result.astype(np.float64))[0]
            worst = max(worst, float(np.abs(rho_gpu - rho).sum() / np.abs(rho).sum()))
            checked.append(f"{r.family} n={r.n} steps={r.steps}")
        accuracy = {"vs": "FP64 CPU oracle, same steps from the same seeded state", "requests": checked,
                    "density_l1_rel_max": worst}
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    busy_gbs = stats["busy_hbm_gbs"] or 0.0
    value = stats["zone_updates_per_s"] * world
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": stats["ticks"], "warmup": 0, "ms_per_step": 1e3 * stats["busy_s"] / max(stats["ticks"], 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": c["desc"], "requests": stats["requests"], "rate_per_s": c["rate"],
                       "budget_gb": args.budget_gb, "max_active": args.max_active,
                       "request_stream_prep_s": prep_s,
                       "payloads": "initial fields built on a background thread ahead of admission (seeded)",
                       "step": "one tick = one batched step of every active solve; steps, admissions and "
                               "retirements enqueued without stream synchronisation, up to 8 steps in flight",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "latency": {"p50_s": stats["p50_latency_s"], "p99_s": stats["p99_latency_s"],
                        "makespan_s": stats["makespan_s"]},
            "roofline": {"bound": "hbm", "achieved": busy_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": busy_gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "step3d_batch_kernel<float> + step2d_batch_kernel<float>",
                         "note": "algorithmic bytes over busy (tick) time"},
            "busy_zone_updates_per_s": stats["busy_zone_updates_per_s"],
            "accuracy": accuracy,
            "cpu_baseline": None, "e2e": None, "gpu_launches": stats["launches"], "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------ z-slab decomposition
def run_gpu_slabs(args):
    """The decomposed step (R slabs on one GPU) timed beside the undivided
    step on the same grid; both start from the same state."""
    import torch

    from paper_1510_05061_gb300 import autotune
    from paper_1510_05061_gb300 import build as hbuild
    from paper_1510_05061_gb300 import hydro

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    hbuild.build()
    hydro.load()
    prob, W, c = build_workload(args.config)
    R = c["slabs"]
    stream = torch.cuda.current_stream()
    sim = hydro.Simulation(prob, W, stream=stream)
    tune = None
    if not args.no_tune:
        tune = autotune.tune_simulation(sim, use_cache=not args.retune)
        tune = {k: v for k, v in tune.items() if k != "table"}
        sim.close()
        sim = hydro.Simulation(prob, W, stream=stream)
        sim.configure(tune["variant"], tune["zchunk"])
    slabs = hydro.Slabs(prob, W, R, stream=stream)
    if tune is not None:
        slabs.configure(tune["variant"], tune["zchunk"])

    def timed(step):
        for _ in range(args.warmup):
            step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(world, e0.elapsed_time(e1))

    whole_ms = timed(lambda: sim.step())
    n0 = slabs.launches()
    with ClockSampler(local) as clk:
        el_ms = timed(lambda: slabs.step(1))
    launches = slabs.launches() - n0 - args.warmup * (R + 1)
    same = bool(np.array_equal(sim.get_state(), slabs.get_state()))
    sim.close()
    slabs.close()
    N = prob.ncell
    value = world * N * args.steps / (el_ms * 1e-3)
    peaks, peak_kind = measured_peaks()
    fma = measure_fma_peak(inputs.FP64)
    peak_tf = fma["tflops"]
    ach_tf = FLOPS_PER_ZONE_3D * N / (el_ms / args.steps * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": c["desc"], "grid": list(prob.n), "slabs": R,
                       "l2": "inputs larger than L2 (state %.0f MB > 129 MB)" % (N * 40 / 1e6),
                       "parallelism": "virtual ranks on one GPU"},
            "undivided_ms_per_step": whole_ms / args.steps,
            "decomposition_overhead": el_ms / whole_ms - 1.0,
            "bitwise_equal_to_undivided": same,
            "autotune": tune,
            "roofline": {"bound": "alu", "achieved": ach_tf, "peak": peak_tf, "unit": "TFLOP/s",
                         "frac": ach_tf / peak_tf, "traffic": None,
                         "peak_kind": "measured: FP64 FMA probe (" + fma["how"] + ")",
                         "peak_derived": fp64_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0))),
                         "kernel": "step3d_kernel<double, 0, ...> over all slabs (whole step time)"},
            "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- GPU arm
def run_gpu(args):
    if CONFIGS[args.config].get("slabs"):
        return run_gpu_slabs(args)
    if CONFIGS[args.config].get("batch"):
        return run_gpu_batch(args)
    if CONFIGS[args.config].get("served"):
        return run_served(args)
    import torch

    from paper_1510_05061_gb300 import build as hbuild
    from paper_1510_05061_gb300 import hydro

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    hbuild.build()
    hydro.load()
    prob, W, c = build_workload(args.config)
    N = prob.ncell
    itemsize = 4 if prob.precision == inputs.FP32 else 8
    stream = torch.cuda.current_stream()

    # ---- device-resident run: inputs in HBM before the timed region
    sim = hydro.Simulation(prob, W, stream=stream)
    tune = None
    if args.variant is not None and prob.ndim == 3:
        # a fixed tile variant and z-chunk (profiling runs)
        tune = {"variant": args.variant, "zchunk": args.zchunk, "cached": False, "note": "fixed by --variant"}
        sim.close()
        sim = hydro.Simulation(prob, W, stream=stream)
        sim.configure(tune["variant"], tune["zchunk"])
    elif not args.no_tune and prob.ndim == 3:
        from paper_1510_05061_gb300 import autotune

        tune = autotune.tune_simulation(sim, use_cache=not args.retune)
        if args.show_tuning:
            print(json.dumps({"autotune_table": tune.get("table")}), file=sys.stderr, flush=True)
        tune = {k: v for k, v in tune.items() if k != "table"}
        # tuning advanced the solve: start the measured run from the initial state
        sim.close()
        sim = hydro.Simulation(prob, W, stream=stream)
        sim.configure(tune["variant"], tune["zchunk"])
    for _ in range(args.warmup):
        sim.step()
    torch.cuda.synchronize()
    nlaunch0 = sim.launches()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_all0.record(stream)
        for i in range(args.steps):
            starts[i].record(stream)
            sim.step()
            ends[i].record(stream)
        t_all1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = sim.launches() - nlaunch0
    el_ms = t_all0.elapsed_time(t_all1)
    el_ms = max_over_ranks(world, el_ms)
    kern_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_avg_ms = sum(kern_ms) / len(kern_ms)
    t_sim = sim.t
    ok = np.isfinite(t_sim)
    sim.close()
    del sim

    value = world * N * args.steps / (el_ms * 1e-3)

    # ---- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        W_pin = torch.empty(W.shape, dtype=torch.float64, pin_memory=True)
        W_pin.numpy()[...] = W
        out_pin = torch.empty(prob.shape, dtype=torch.float32 if itemsize == 4 else torch.float64,
                              pin_memory=True)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2 = hydro.Simulation(prob, W_pin.numpy(), stream=stream)
        if tune is not None:
            sim2.configure(tune["variant"], tune["zchunk"])
        for _ in range(args.steps):
            sim2.step()
        hydro.hydro_get_state(sim2.h, out_pin.numpy())
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(world, time.perf_counter() - t0)
        sim2.close()
        e2e = {"value": world * N * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(W.nbytes / args.steps),
               "d2h_bytes_per_step": int(N * prob.nvar * itemsize / args.steps),
               "note": "hydro_init from pinned host primitives + K steps + hydro_get_state to pinned host"}

    # ---- roofline of the step kernel
    peaks, peak_kind = measured_peaks()
    rk2 = prob.scheme == inputs.SSPRK2
    # per step: one kernel (MUSCL-Hancock) or the two stage kernels (SSP-RK2)
    bytes_per_zone = (5 if rk2 else 2) * prob.nvar * itemsize
    zones_per_launch = N
    if prob.scheme == inputs.CTU:
        flops_per_zone = FLOPS_PER_ZONE_3D_CTU if prob.ndim == 3 else FLOPS_PER_ZONE_2D_CTU
    elif rk2 and prob.recon == inputs.PPM:
        flops_per_zone = FLOPS_PER_ZONE_3D_PPM if prob.ndim == 3 else FLOPS_PER_ZONE_2D_PPM
    elif rk2:
        flops_per_zone = FLOPS_PER_ZONE_3D_RK2 if prob.ndim == 3 else FLOPS_PER_ZONE_2D_RK2
    else:
        flops_per_zone = FLOPS_PER_ZONE_3D if prob.ndim == 3 else FLOPS_PER_ZONE_2D
    achieved_gbs = bytes_per_zone * zones_per_launch / (kern_avg_ms * 1e-3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    clocks = clk.summary()
    variant = tune["variant"] if tune else (0 if itemsize == 4 else 4)
    knames = step_kernel_names(prob, variant)
    kname = " + ".join(knames)
    # DRAM bytes of one step: the sum over its kernels (null if any is missing or stale)
    traffic = args.traffic
    if traffic is None:
        per = [measured_traffic(args.config, k) for k in knames]
        traffic = sum(per) if all(v is not None for v in per) else None
    ach_tf = flops_per_zone * zones_per_launch / (kern_avg_ms * 1e-3) / 1e12
    fma = measure_fma_peak(prob.precision)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    if prob.precision == inputs.FP64:
        peak_tf = fma["tflops"]
        roofline = {"bound": "alu", "achieved": ach_tf, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": ach_tf / peak_tf, "traffic": traffic,
                    "peak_kind": "measured: FP64 FMA probe (" + fma["how"] + ")",
                    "peak_derived": fp64_peak_tflops(sm_mhz),
                    "peak_probe_clocks": fma["clocks"],
                    "kernel": kname, "algorithmic_bytes": bytes_per_zone * zones_per_launch,
                    "algorithmic_flops": flops_per_zone * zones_per_launch,
                    "hbm": {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                            "frac": achieved_gbs / hbm_peak, "peak_kind": peak_kind}}
    else:
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved_gbs / hbm_peak, "traffic": traffic,
                    "peak_kind": peak_kind, "kernel": kname,
                    "algorithmic_bytes": bytes_per_zone * zones_per_launch,
                    "alu": {"achieved": ach_tf, "peak": fma["tflops"], "unit": "TFLOP/s",
                            "frac": ach_tf / fma["tflops"],
                            "peak_kind": "measured: FP32 FMA probe (" + fma["how"] + ")"}}
    accuracy = None
    if prob.precision == inputs.FP32 and rank == 0 and not args.no_accuracy:
        accuracy = fp32_accuracy(args.config)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(cfg=args.config, nz_slab=32)
        v1, _, sample1 = oracle_sample(seconds=5.0, cfg=args.config, nz_slab=8, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "cpu_model": host_cpu_model(),
               "one_core": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if itemsize == 4 else "f64", "data": "synthetic",
            "config": {"workload": c["desc"], "grid": list(prob.n), "precision": "fp32" if itemsize == 4 else "fp64",
                       "hse_subtract": prob.hse_subtract, "state_bytes": N * prob.nvar * itemsize,
                       "l2": ("inputs larger than L2 (state %.0f MB > 129 MB)" if N * prob.nvar * itemsize > 129e6 else
               "state %.1f MB fits in L2 (latency-bound configuration)") % (N * prob.nvar * itemsize / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "kernel_ms_avg": kern_avg_ms,
            "autotune": tune,
            "roofline": roofline,
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "t_sim": t_sim if ok else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_precision_report(args):
    """RT n^3 to t = 0.5 in FP32 (bulk) and FP64, both with hydrostatic-
    background subtraction: density L1-relative difference and throughput."""
    import torch

    from paper_1510_05061_gb300 import build as hbuild
    from paper_1510_05061_gb300 import hydro

    hbuild.build()
    n = args.precision_n
    out = {"workload": f"Rayleigh-Taylor {n}^3, hse subtraction, t_end = {args.t_end}"}
    rho = {}
    for prec, name in ((inputs.FP32, "fp32"), (inputs.FP64, "fp64")):
        prob, W = inputs.rayleigh_taylor(n, precision=prec, hse_subtract=1)
        sim = hydro.Simulation(prob, W)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, t = sim.advance_to(args.t_end)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        P = sim.primitive()
        rho[name] = P[0]
        out[name] = {"steps": steps, "t": t, "seconds": el,
                     "zone_updates_per_s": prob.ncell * steps / el}
        sim.close()
        del P
    diff = float(np.abs(rho["fp32"] - rho["fp64"]).sum() / np.abs(rho["fp64"]).sum())
    out["density_l1_rel_fp32_vs_fp64"] = diff
    out["fp32_over_fp64_throughput"] = out["fp32"]["zone_updates_per_s"] / out["fp64"]["zone_updates_per_s"]
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="rt256-fp64", choices=sorted(CONFIGS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="FP32 workloads: skip the error against the FP64 oracle")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch of the step kernel from an ncu capture")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuner cache")
    ap.add_argument("--no-tune", action="store_true", help="default tile shape and z-chunk")
    ap.add_argument("--variant", type=int, default=None, help="single 3D solves: fixed tile variant (no tuning)")
    ap.add_argument("--zchunk", type=int, default=0,
                    help="with --variant: z-chunk (0 = default; negative: the balanced grid, -1 over whole columns)")
    ap.add_argument("--show-tuning", action="store_true", help="print the autotuner's timing table to stderr")
    ap.add_argument("--requests", type=int, default=200, help="served configs: number of requests")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="served configs: HBM budget")
    ap.add_argument("--max-active", type=int, default=64, help="served configs: concurrent solves")
    ap.add_argument("--precision-report", action="store_true",
                    help="FP32 vs FP64 Rayleigh-Taylor density error at t_end (no JSON bench line)")
    ap.add_argument("--precision-n", type=int, default=512)
    ap.add_argument("--t-end", type=float, default=0.5)
    ap.add_argument("--traffic-scale", type=float, default=1.0,
                    help="with --record-traffic: scale the captured bytes to the workload's cells")
    ap.add_argument("--traffic-note", default="", help="with --record-traffic: how the capture was scaled")
    ap.add_argument("--n", type=int, default=None,
                    help="Rayleigh-Taylor configs: grid n^3 instead of the workload's (profiling a smaller case)")
    ap.add_argument("--record-traffic", metavar="NCU_CSV", default=None,
                    help="store DRAM bytes per launch from an ncu CSV of --config into profiles/traffic.json")
    args = ap.parse_args()
    global GRID_OVERRIDE
    GRID_OVERRIDE = args.n
    if args.record_traffic:
        return record_traffic(args.config, args.record_traffic, args.traffic_scale, args.traffic_note)
    if args.precision_report:
        return run_precision_report(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
