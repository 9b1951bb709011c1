"""Host-side checks of bench.py's profiler kernel names: the keys under which
profiles/traffic.json stores each workload's measured DRAM traffic must be
the names bench.py derives for the kernels it times."""

import json
import os

import pytest

import bench
from paper_1510_05061_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def small(cfg):
    """The workload's problem at a small size (names do not depend on n)."""
    c = bench.CONFIGS[cfg]
    prob, _ = inputs.rayleigh_taylor(8, precision=c["precision"], hse_subtract=c["hse"])
    return prob.replace(scheme=c.get("scheme", inputs.HANCOCK), recon=c.get("recon", inputs.PLM))


def test_fp64_step_with_gravity_along_z_takes_the_specialised_kernel():
    prob = small("rt256-fp64")
    assert bench.step_kernel_names(prob, 6) == ["step3d_kernel<double, 0, 16, 16, 0, 0, 1, 1>"]
    # gravity with an x component: the general kernel
    assert bench.step_kernel_names(prob.replace(grav=(0.1, 0.0, -1.0)), 6) == \
        ["step3d_kernel<double, 0, 16, 16, 0, 0, 1, 0>"]
    # the background mode always has gravity along z only
    assert bench.step_kernel_names(small("rt256-fp64-hse"), 2) == ["step3d_kernel<double, 1, 16, 16, 0, 0, 0, 1>"]


def test_fp32_stage_and_ctu_names():
    assert bench.step_kernel_names(small("rt512-fp32"), 7) == ["step3d_kernel<float, 1, 32, 16, 0, 0, 1, 0>"]
    assert bench.step_kernel_names(small("rt512-fp32-rk2"), 0) == [
        "step3d_kernel<float, 1, 32, 8, 1, 0, 0, 0>", "step3d_kernel<float, 1, 32, 8, 2, 0, 0, 0>"]
    assert bench.step_kernel_names(small("rt256-fp64-ppm"), 6) == [
        "step3d_kernel<double, 0, 16, 16, 1, 1, 1, 0>", "step3d_kernel<double, 0, 16, 16, 2, 1, 1, 0>"]
    assert bench.step_kernel_names(small("rt256-fp64-ctu"), 0) == ["ctu3d_kernel<double, 0, 16, 8>"]
    assert bench.step_kernel_names(small("rt512-fp32-ctu"), 0) == ["ctu3d_kernel<float, 1, 16, 16>"]


def test_recorded_traffic_keys_are_names_bench_derives():
    """Every recorded step-kernel entry of the latest capture is a name the
    bench derives, so that bench.py finds it and reports it as
    roofline.traffic while the kernel sources still hash to the captured ones
    (entries of other sources are reported as null traffic)."""
    import collections

    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        table = json.load(fh)
    entries = []
    for cfg, kernels in table.items():
        c = bench.CONFIGS.get(cfg)
        if c is None or c.get("batch") or c.get("served") or c.get("slabs"):
            continue
        for k, e in kernels.items():
            if k.startswith(("step3d_kernel", "ctu3d_kernel")):
                entries.append((cfg, k, e.get("source_sha")))
    current = [(cfg, k, sha) for cfg, k, sha in entries if sha == bench.kernel_source_sha(k)]
    if len(current) >= 8:
        entries = current
    else:    # the sources moved on since the capture: check the latest capture's names
        latest = collections.Counter(sha for _, _, sha in entries).most_common(1)[0][0]
        entries = [e for e in entries if e[2] == latest]
    checked = 0
    for cfg, k, sha in entries:
        derived = {n for v in range(8) for n in bench.step_kernel_names(small(cfg), v)}
        assert k in derived, (cfg, k)
        checked += 1
    assert checked >= 8


def test_profile_commands_name_existing_workloads():
    """The commands quoted in profiles/*.md run committed files only: every
    --config they name is a bench.py workload."""
    import glob
    import re

    names = set()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as fh:
            names |= set(re.findall(r"--config\s+([A-Za-z0-9_.-]+)", fh.read()))
    names -= {"<cfg>", "$c"}
    names = {n for n in names if not n.startswith(("<", "$"))}
    assert names, "no workload named in the profiles"
    missing = sorted(n for n in names if n not in bench.CONFIGS)
    assert not missing, missing


def test_source_hash_follows_a_kernels_own_sources():
    """A kernel's traffic stays valid when only other kernels' sources change:
    its hash covers its translation units and the headers they include."""
    files = bench._csrc_closure(bench.KERNEL_UNITS["step3d_kernel"])
    assert "step3d.cuh" in files and "hydro_device.cuh" in files and "hydro_internal.h" in files
    assert "pair3d.cuh" not in files and "ctu3d.cuh" not in files
    pair = bench._csrc_closure(bench.KERNEL_UNITS["step3d_pair_kernel"])
    assert "pair_math.cuh" in pair and "step3d.cuh" in pair
    assert bench.kernel_source_sha("step3d_kernel<double, 0, 16, 16, 0, 0, 1, 1>") != \
        bench.kernel_source_sha("ctu3d_kernel<double, 0, 16, 8>")
