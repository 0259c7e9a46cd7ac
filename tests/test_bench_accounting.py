"""The benchmark's roofline accounting, checked on the CPU: the algorithmic
bytes and flops it divides by, against values written out by hand from the
definitions (compulsory bytes: every sphere entry, stick row and cube point
read or written once; flops: 5 L log2 L per length-L line over the pruned
line counts), and the workload definitions against the oracle's spheres."""
import math

import numpy as np
import pytest

import bench
from oracle import sphere_gvectors


def test_workloads_match_their_definitions():
    w = bench.Workload("sphere64_rt")
    assert (w.n, w.radius, w.bands, w.direction) == ((64, 64, 64), 16.0, [64], "roundtrip")
    assert len(sphere_gvectors(w.n, w.radius)) == 17077
    w = bench.Workload("sphere128_apply")
    assert (w.n, w.radius, w.bands, w.direction) == ((128, 128, 128), 32.0, [256], "apply")
    w = bench.Workload("sphere256_e2")
    assert (w.n, w.radius, w.bands) == ((256, 256, 256), 64.0, [256])
    w = bench.Workload("sphere96_multik")
    assert w.nk == 8 and all(16 <= b <= 128 for b in w.bands) and w.total_bands == sum(w.bands)
    assert bench.Workload("sphere64_rt_batchfast").plan_kw()["layout"] == 1
    with pytest.raises(SystemExit):
        bench.Workload("no_such_workload")


def test_stage_bytes_64_round_trip():
    w = bench.Workload("sphere64_rt")
    info = {"complex_bytes": 8}
    ngw, sticks = 17077, 797
    cube = 64 * 64 ** 3
    stk = 64 * sticks * 64
    sph = 64 * ngw
    # compulsory: the cube for the plane stages, the sphere for the z stages;
    # the stick rows between them are this design's intermediate
    assert bench.stage_bytes("plane_r2g", w, info, [ngw], [sticks]) == (8 * cube, 8 * stk)
    assert bench.stage_bytes("plane_g2r", w, info, [ngw], [sticks]) == (8 * cube, 8 * stk)
    assert bench.stage_bytes("stick_g2r", w, info, [ngw], [sticks]) == (8 * sph, 8 * stk)
    assert bench.stage_bytes("stick_r2g", w, info, [ngw], [sticks]) == (8 * sph, 8 * stk)
    # 134.2 MB of cube per r -> G launch, 26.1 MB of stick rows beside it
    comp, inter = bench.stage_bytes("plane_r2g", w, info, [ngw], [sticks])
    assert abs(comp / 1e6 - 134.2) < 0.05 and abs(inter / 1e6 - 26.1) < 0.05


def test_default_workload_is_the_largest_single_gpu_configuration():
    """160^3, |G| <= 40 (267 761 G), 512 bands, round trip streamed in band chunks."""
    w = bench.Workload(bench.DEFAULT_WORKLOAD)
    assert (w.n, w.radius, w.bands, w.direction) == ((160, 160, 160), 40.0, [512], "roundtrip")
    assert len(sphere_gvectors(w.n, w.radius)) == 267761
    # compulsory bytes of the round trip per band: 2 (ngw + N^3) complex64 = 69.8 MB
    assert abs(2 * (267761 + 160 ** 3) * 8 / 1e6 - 69.8) < 0.05


def test_apply_flops_and_fp32_peak():
    w = bench.Workload("sphere128_apply")
    x_slabs = 65  # occupied x values of |G| <= 32
    per_dir = x_slabs * 128 * 5 * 128 * math.log2(128) + 128 * 128 * 5 * 128 * math.log2(128)
    assert bench.stage_flops("plane_apply", w, [x_slabs]) == pytest.approx(256 * 2 * per_dir)
    assert bench.stage_flops("plane_apply", w, [x_slabs]) / 1e9 == pytest.approx(56.665, rel=1e-4)
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(152 * 128 * 2 * 2.07e-3)


def test_kernel_source_hash_covers_the_profiled_kernels():
    import json
    import os
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")))
    assert set(d["kernels"]) == {"stick_g2r", "plane_g2r", "plane_r2g", "stick_r2g"}
    for k, v in d["kernels"].items():
        assert v["dram_bytes_per_band"] == round((v["read_bytes"] + v["write_bytes"]) / v["bands_per_launch"])
    assert len(bench.kernel_source_hash()) == 16


def test_kernel_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The traffic record stays valid across comment edits of the kernel
    sources and goes stale on any code edit."""
    import os
    import shutil
    src = os.path.join(bench.ROOT, "paper_2406_05577_gb300", "csrc")
    dst = tmp_path / "paper_2406_05577_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    f = dst / "line_fft.cuh"
    text = f.read_text()
    f.write_text("// a new comment line\n\n" + text.replace("#pragma once", "#pragma once  // trailing note", 1))
    assert bench.kernel_source_hash() == h0
    f.write_text(text.replace("#pragma once", "#pragma once\nconstexpr int fftb_unused_probe = 1;", 1))
    assert bench.kernel_source_hash() != h0
