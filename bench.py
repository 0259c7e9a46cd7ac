"""Benchmark: batched pruned sphere <-> cube FFT, bands/s.

Default workload (the headline, the largest single-GPU configuration):
160^3 grid, cutoff |G| <= 40 (267 761 G vectors), 512 bands, FP32
coefficients complex Gaussian, round trip G -> r -> G with the 16.8 GB
real-space cube set written to HBM and read back, processed in band chunks.
A step is one fftb_execute of the whole batch. The plain FP64 GPU path and
the split-precision tensor-core path (MIXED_TC) run the same workload beside
it, each compared with the FP64 path's output; the 64^3 workload (|G| <= 16,
64 bands) is timed as a second figure. Other workloads (``--workload``):
64^3 alone, 96^3 with 8 k-points and uneven band counts in one graph-
replayed, autotuned launch sequence; 128^3 local-potential apply V(r) psi(r)
with 256 bands; 256^3 (sphere diameter 128) with 256 bands, the paper's own
single-GPU shape; the 64^3 workload in the batch-fastest layout.

Under torchrun the job is one global batch of world x B bands per k-point;
each rank transforms its contiguous shard of B bands (band_shard) on its own
GPU (bands are independent: weak scaling, no collective on the data path;
the only collectives are the timing barrier and the max of the step time
over ranks).
Timing follows the paper's protocol (Sec. 4.2: warm-up iterations, then
timed iterations, mean) with CUDA events on the launching stream; L2 is
flushed between timed steps. ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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

import fftb_inputs as fi  # noqa: E402

# the largest single-GPU configuration: 160^3, |G| <= 40, 512 bands
DEFAULT_WORKLOAD = "sphere160_large"
METRIC = "sphere-FFT bands/sec (G->r->G) and % HBM roofline, mixed vs FP64 at L2<=1e-5"
L2_FLUSH_BYTES = 256 << 20


class Workload:
    """One benchmark configuration: grid, spheres, bands, direction."""

    def __init__(self, name):
        self.name = name
        self.layout = 0
        if name == "sphere64_rt":
            self.n, self.radius, self.kshift, self.bands = (64, 64, 64), 16.0, None, [64]
            self.direction, self.desc = "roundtrip", \
                "64^3 grid, |G|<=16 (17077 G), 64 bands, G->r->G round trip, cube kept in HBM"
            self.envelope, self.seed, self.graph, self.tune = 8.0, 2, True, True
        elif name == "sphere64_rt_batchfast":
            self.n, self.radius, self.kshift, self.bands = (64, 64, 64), 16.0, None, [64]
            self.direction, self.desc = "roundtrip", \
                ("64^3 grid, |G|<=16 (17077 G), 64 bands, G->r->G round trip, cube kept in HBM, batch-fastest "
                 "layout (sphere [ngw][B], cube [N2][N1][N0][B])")
            self.envelope, self.seed, self.graph, self.tune = 8.0, 2, False, True
            self.layout = 1
        elif name == "sphere96_multik":
            self.n, self.radius = (96, 96, 96), 24.0
            self.kshift = fi.kshifts(8, 3)
            self.bands = [int(b) for b in fi.band_counts(8, 16, 128, 3)]
            self.direction = "roundtrip"
            self.desc = ("96^3 grid, 8 k-points k~U[-0.5,0.5)^3, |G+k|<=24, bands per k-point U{16..128} "
                         f"({sum(self.bands)} total), G->r->G, one graph-replayed autotuned launch sequence")
            self.envelope, self.seed, self.graph, self.tune = None, 3, True, True
        elif name == "sphere128_apply":
            self.n, self.radius, self.kshift, self.bands = (128, 128, 128), 32.0, None, [256]
            self.direction = "apply"
            self.desc = ("128^3 grid, |G|<=32 (137065 G), 256 bands, psi_G -> V(r) psi(r) -> G sphere, "
                         "V = 32 Gaussians of width 4, cube never stored")
            self.envelope, self.seed, self.graph, self.tune = None, 4, False, True
        elif name == "sphere160_large":
            self.n, self.radius, self.kshift, self.bands = (160, 160, 160), 40.0, None, [512]
            self.direction = "roundtrip"
            self.desc = ("160^3 grid, |G|<=40 (267761 G), 512 bands, G->r->G with the 16.8 GB cube set "
                         "kept in HBM, processed in band chunks")
            self.envelope, self.seed, self.graph, self.tune = None, 5, False, True
        elif name == "sphere256_e2":
            self.n, self.radius, self.kshift, self.bands = (256, 256, 256), 64.0, None, [256]
            self.direction = "roundtrip"
            self.desc = ("256^3 grid, |G|<=64 (sphere diameter 128, 1097917 G), 256 bands, G->r->G with the "
                         "34 GB cube set kept in HBM, processed in band chunks (the paper's E2 shape on one GPU)")
            self.envelope, self.seed, self.graph, self.tune = None, 6, False, True
        else:
            raise SystemExit(f"unknown workload {name}")
        self.total_bands = sum(self.bands)
        self.nk = len(self.bands)

    def plan_kw(self):
        kw = dict(radius=self.radius, bands=self.bands)
        if self.layout:
            kw["layout"] = self.layout
        if self.kshift is not None:
            kw["kshift"] = self.kshift
        return kw

    def coefficients(self, spheres, rank=0, world=1):
        """This rank's bands of the job's global batch: per k-point the job
        holds world * B_k bands (weak scaling: B_k per rank), split by
        band_shard into contiguous shards; band i of a k-point's global batch
        is drawn from its own stream, so the shards are slices of one batch
        whatever the world size."""
        from paper_2406_05577_gb300.shard import band_shard
        parts = []
        for k, (g, b) in enumerate(zip(spheres, self.bands)):
            start, count = band_shard(world * b, world, rank)
            c = fi.complex_gaussian_bands(start, count, len(g), self.seed + 100 * k)
            if self.envelope:
                c = c * fi.gaussian_envelope(g, self.envelope)[None, :]
            parts.append(c)
        return parts

    def potential(self):
        return fi.gaussian_potential(self.n, 32, 4.0, seed=self.seed)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the kernel sources the ncu traffic record was taken with, over
    their code only: line comments and blank lines do not count."""
    h = hashlib.sha256()
    for f in ("fft_core.cuh", "line_fft.cuh", "kernels.cuh", "async_copy.cuh", "check.cuh", "k_f32_pf.cu",
              "k_f32_alt.cu", "k_f32_zq.cu"):
        for line in open(os.path.join(ROOT, "paper_2406_05577_gb300", "csrc", f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_traffic(workload, kernel):
    """DRAM bytes per band of one kernel from the committed ncu summary, or
    None when the kernel sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_source_hash") != kernel_source_hash() or d.get("workload") != workload:
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_band")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis and vis.split(",")[0].strip().isdigit():
            cmd += ["-i", vis.split(",")[0].strip()]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_step(w, spheres, parts, v, bands_idx):
    """The FP64 oracle on the listed (k, band) pairs of the workload."""
    import oracle
    for k, b in bands_idx:
        if w.direction == "apply":
            oracle.apply_potential(spheres[k], parts[k][b], v, w.n)
        else:
            oracle.roundtrip(spheres[k], parts[k][b], w.n)


def band_list(w):
    return [(k, b) for k in range(w.nk) for b in range(w.bands[k])]


def time_oracle(w, spheres, parts, v, budget_s):
    allb = band_list(w)
    done, t0 = 0, time.perf_counter()
    while True:
        oracle_step(w, spheres, parts, v, [allb[done % len(allb)]])
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done / el, done, el


def _oracle_worker(job):
    """One host process of the all-cores oracle timing: rebuilds the
    workload's inputs from their seeds and runs the oracle on its share of the
    bands until the budget is spent."""
    name, share, budget_s = job
    import oracle
    w = Workload(name)
    ks = w.kshift if w.kshift is not None else [(0.0, 0.0, 0.0)]
    sph = [oracle.sphere_gvectors(w.n, w.radius, k) for k in ks]
    parts = w.coefficients(sph)
    v = w.potential().astype(np.float32).astype(np.float64) if w.direction == "apply" else None
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        oracle_step(w, sph, parts, v, [share[done % len(share)]])
        done += 1
    return done, time.perf_counter() - t0


def time_oracle_all_cores(w, budget_s):
    """The oracle over bands in one spawned process per host core (spawn: this
    process already holds a CUDA context)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    allb = band_list(w)
    jobs = [(w.name, [allb[i % len(allb)] for i in range(c, c + len(allb), cores)] or [allb[0]], budget_s)
            for c in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    done = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return done / busy, done, busy, wall, cores


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts name the core in lscpu only
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    w = Workload(args.workload)
    ks = w.kshift if w.kshift is not None else [(0.0, 0.0, 0.0)]
    spheres = [oracle.sphere_gvectors(w.n, w.radius, k) for k in ks]
    parts = w.coefficients(spheres)
    v = w.potential().astype(np.float32).astype(np.float64) if w.direction == "apply" else None
    allb = band_list(w)
    sample = {"sphere64_rt": 16, "sphere64_rt_batchfast": 16, "sphere96_multik": 4, "sphere128_apply": 2,
              "sphere160_large": 1, "sphere256_e2": 1}[w.name]
    times = []
    for step in range(args.warmup + args.steps):
        idx = [allb[(step * sample + i) % len(allb)] for i in range(sample)]
        t0 = time.perf_counter()
        oracle_step(w, spheres, parts, v, idx)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.desc, "grid": list(w.n), "radius": w.radius, "bands": w.total_bands,
                       "precision": "fp64 (CPU oracle)", "step_sample_bands": sample},
            "cpu_baseline": {"value": value, "unit": "bands/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample} bands of the workload per step, numpy pocketfft FP64"},
            "e2e": {"value": value, "unit": "bands/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def stage_bytes(kind, w, info, ngws, sticks):
    """Bytes of one stage kind over the whole batch, as (compulsory,
    intermediate). Compulsory bytes are the transform's own input and output
    read or written once (the cube for the y/x stages, the sphere for the z
    stages); intermediate bytes are the stick rows T that this design passes
    between its z stage and its plane stage (written once, read once)."""
    c = info["complex_bytes"]
    vol = w.n[0] * w.n[1] * w.n[2]
    n2 = w.n[2]
    sph = sum(b * g for b, g in zip(w.bands, ngws))
    stk = sum(b * s * n2 for b, s in zip(w.bands, sticks))
    cube = w.total_bands * vol
    return {"stick_g2r": (sph * c, stk * c), "plane_g2r": (cube * c, stk * c), "plane_r2g": (cube * c, stk * c),
            "stick_r2g": (sph * c, stk * c), "plane_apply": (vol * c // 2, 2 * stk * c)}[kind]


# FP32 arithmetic peak of the GPU from its unit counts and clock: 152 SMs x 128
# FP32 lanes x 2 flops per fused multiply-add x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def stage_flops(kind, w, slabs):
    """Algorithmic flops of one plane stage over the whole batch: 5 L log2 L
    per length-L line, pruned line counts (y lines of the occupied x-slabs,
    every x line); the fused apply runs both directions."""
    n0, n1, n2 = w.n
    per_band = sum(b * (x * n2 * 5 * n1 * np.log2(n1) + n1 * n2 * 5 * n0 * np.log2(n0))
                   for b, x in zip(w.bands, slabs))
    return per_band * (2 if kind == "plane_apply" else 1)


def make_plan(fftb, w, prec, dev):
    import torch
    plan = fftb.Plan(w.n, w.direction, prec, **w.plan_kw())
    v_dev = None
    if w.direction == "apply":
        v_dev = torch.from_numpy(w.potential().astype(np.float64 if prec == "fp64" else np.float32)).to(dev)
        plan.set_potential(v_dev)
    if w.tune:
        plan.autotune(3)
    if w.graph:
        plan.set_graph(True)
    return plan, v_dev


def time_workload(fftb, name, dev, flush, stream, args):
    """A second workload timed like the headline (FP32, autotuned, L2 flushed
    between steps, CUDA events on the launching stream)."""
    import torch
    w = Workload(name)
    plan, _ = make_plan(fftb, w, "fp32", dev)
    spheres = [plan.sphere(k) for k in range(w.nk)]
    ngws = [len(g) for g in spheres]
    c = np.concatenate([(p.T if w.layout else p).reshape(-1) for p in w.coefficients(spheres)]).astype(np.complex64)
    x = torch.from_numpy(c).to(dev)
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device=dev) \
        if w.direction == "roundtrip" else None
    for _ in range(args.warmup):
        plan.execute(x, out, cube)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        plan.execute(x, out, cube)
        b.record(stream)
    torch.cuda.synchronize(dev)
    plan.check()
    ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    vol = w.n[0] * w.n[1] * w.n[2]
    step_bytes = 2 * (sum(b * g for b, g in zip(w.bands, ngws)) + w.total_bands * vol) * 8
    hbm, _ = peaks()
    res = {"workload": w.desc, "value": w.total_bands / (ms / 1e3), "unit": "bands/s", "ms_per_step": ms,
           "step_compulsory_frac": step_bytes / (ms / 1e3) / 1e9 / hbm}
    if w.direction == "roundtrip":
        res["rel_l2_roundtrip"] = (torch.linalg.vector_norm(out - vol * x) /
                                   torch.linalg.vector_norm(vol * x)).item()
    del x, out, cube, plan
    return res


def gpu_local_cpus(dev_index):
    """Host CPUs on the GPU's NUMA node (its PCI device's local_cpulist in sysfs)
    that this process may use, or None when that cannot be read."""
    import torch
    bdf = None
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        bdf = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
    except Exception:
        try:
            out = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", str(dev_index)],
                                 capture_output=True, text=True, timeout=20).stdout.strip().lower()
            dom, rest = out.split(":", 1)
            bdf = f"{int(dom, 16):04x}:{rest}"
        except Exception:
            return None
    try:
        txt = open(f"/sys/bus/pci/devices/{bdf}/local_cpulist").read().strip()
    except OSError:
        return None
    cpus = set()
    for part in txt.split(","):
        if "-" in part:
            lo, hi = part.split("-")
            cpus.update(range(int(lo), int(hi) + 1))
        elif part:
            cpus.add(int(part))
    local = cpus & os.sched_getaffinity(0)
    return local or None


def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb

    w = Workload(args.workload)
    plan, v_dev = make_plan(fftb, w, "fp32", dev)
    info = plan.info
    spheres = [plan.sphere(k) for k in range(w.nk)]
    ngws = [len(g) for g in spheres]
    sticks = [fftb.fftb_sphere_sticks(w.n, g)[0] for g in spheres]
    slabs = [fftb.fftb_sphere_sticks(w.n, g)[1] for g in spheres]
    parts = w.coefficients(spheres, rank, world)
    # batch-fastest: each k-point's block is [ngw][B]
    c = np.concatenate([(p.T if w.layout else p).reshape(-1) for p in parts]).astype(np.complex64)
    x = torch.from_numpy(c).to(dev)
    out = torch.empty_like(x)

    def band_major(t):  # a sphere batch in band-major order (a view when it already is)
        if not w.layout:
            return t
        blocks, o = [], 0
        for b, ng in zip(w.bands, ngws):
            blocks.append(t[o:o + b * ng].view(ng, b).t().reshape(-1))
            o += b * ng
        return torch.cat(blocks)
    cube = None
    if w.direction == "roundtrip":
        cube = torch.empty(info["cube_elems"], dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan.execute(x, out, cube)
    torch.cuda.synchronize(dev)
    # correctness of this very run: a round trip returns N0 N1 N2 times its
    # input exactly (the oracle's result); every precision is also compared
    # with the FP64 GPU path below (rank 0)
    err = None
    if w.direction == "roundtrip":
        vol = float(np.prod(w.n))
        err = (torch.linalg.vector_norm(out - vol * x) / torch.linalg.vector_norm(vol * x)).item()

    # timed region 1: steps bracketed by events, L2 flushed in between
    sampler = ClockSampler()
    launches0 = plan.launches()
    graphs0 = fftb.fftb_plan_get_info(plan.handle)["graph_launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        plan.execute(x, out, cube)
        evs[i][1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = plan.launches() - launches0
    graph_steps = fftb.fftb_plan_get_info(plan.handle)["graph_launches"] - graphs0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    from paper_2406_05577_gb300.shard import max_over_ranks
    ms = max_over_ranks(ms, device=dev)
    value = world * w.total_bands / (ms / 1e3)

    # short steps: also the median of 50 more steps (same flushing)
    median50 = None
    if ms < 2.0:
        ev50 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(50)]
        for a, b in ev50:
            flush.zero_()
            a.record(stream)
            plan.execute(x, out, cube)
            b.record(stream)
        torch.cuda.synchronize(dev)
        median50 = statistics.median(a.elapsed_time(b) for a, b in ev50)

    # per-kernel event times over the same steps (graphs off while timing)
    fftb.fftb_plan_set_timing(plan.handle, True)
    fftb.fftb_plan_stage_times(plan.handle)
    for i in range(args.steps):
        flush.zero_()
        plan.execute(x, out, cube)
    stage = fftb.fftb_plan_stage_times(plan.handle)
    fftb.fftb_plan_set_timing(plan.handle, False)

    hbm, peak_kind = peaks()
    dom = max((k for k in stage if stage[k][1] > 0), key=lambda k: stage[k][0])
    dom_ms, dom_n = stage[dom]
    comp, inter = stage_bytes(dom, w, info, ngws, sticks)
    launches_per_step = dom_n / args.steps
    alg = comp / launches_per_step  # compulsory bytes per launch
    launch_s = dom_ms / dom_n / 1e3
    achieved = alg / launch_s / 1e9
    traffic_band = ncu_traffic(w.name, dom)
    launch_bands = w.total_bands / launches_per_step
    vol = w.n[0] * w.n[1] * w.n[2]
    sph_elems = sum(b * g for b, g in zip(w.bands, ngws))
    if w.direction == "apply":
        step_bytes = 2 * sph_elems * 8 + vol * 4
    else:
        step_bytes = 2 * (sph_elems + w.total_bands * vol) * 8
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg,
                "what": "compulsory bytes of the kernel (cube points for the y/x stages, sphere entries for the z "
                        "stages, each once) per launch over the CUDA-event launch time",
                "intermediate_bytes_per_launch": inter / launches_per_step,
                "with_intermediate_gbs": (alg + inter / launches_per_step) / launch_s / 1e9,
                "traffic": None if traffic_band is None else traffic_band * launch_bands,
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in stage.items() if v[1]},
                "step_compulsory_gbs": step_bytes / (ms / 1e3) / 1e9,
                "step_compulsory_frac": step_bytes / (ms / 1e3) / 1e9 / hbm}
    if roofline["traffic"] is not None:
        # the ncu DRAM bytes of one launch over the event-timed launch
        roofline["traffic_gbs"] = roofline["traffic"] / launch_s / 1e9
        roofline["traffic_frac"] = roofline["traffic_gbs"] / hbm
    if dom == "plane_apply":
        # the fused apply keeps the cube on chip: its kernel is bound by FP32
        # arithmetic, so it is measured in algorithmic flops against the FP32
        # peak; the byte figures stay beside it
        tflops = stage_flops(dom, w, slabs) / launches_per_step / launch_s / 1e12
        roofline.update({"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tflops / FP32_PEAK_TFLOPS, "peak_source": "derived (FP32 units x clock)",
                         "traffic": None, "algorithmic_gbs": achieved, "algorithmic_gbs_frac": achieved / hbm})

    if rank == 0:
        # FP64 GPU path and the split-precision tensor-core path on the same workload
        def time_plan(prec, reps=3, ref=None):
            """Times one precision's plan on the same inputs; returns its
            figures and its output (for the comparisons between precisions)."""
            p2, vd2 = make_plan(fftb, w, prec, dev)
            cdt = torch.complex128 if prec == "fp64" else torch.complex64
            x2 = torch.from_numpy(np.concatenate([(p.T if w.layout else p).reshape(-1) for p in parts])) \
                .to(torch.complex64).to(cdt).to(dev)
            o2 = torch.empty_like(x2)
            cube2 = None
            if w.direction == "roundtrip":
                cube2 = torch.empty(p2.info["cube_elems"], dtype=cdt, device=dev)
            def run_timed():
                for _ in range(2):
                    p2.execute(x2, o2, cube2)
                evs2 = []
                for _ in range(reps):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    p2.execute(x2, o2, cube2)
                    b.record(stream)
                    evs2.append((a, b))
                torch.cuda.synchronize(dev)
                p2.check()
                return sum(a.elapsed_time(b) for a, b in evs2) / len(evs2)

            def tc_stages():
                return {"tcgen05_plane_stages": p2.info["tensor_core_planes"],
                        "mma_sync_passes_mask_z1_plane2": p2.info["tensor_core_passes"]}

            def errors(d):
                if w.direction == "roundtrip":
                    vol = float(np.prod(w.n))
                    d["rel_l2_roundtrip"] = (torch.linalg.vector_norm(o2 - vol * x2) /
                                             torch.linalg.vector_norm(vol * x2)).item()
                if ref is not None:
                    d["rel_l2_vs_fp64_gpu"] = rel_l2(o2, ref)

            ms2 = run_timed()
            res = {"value": w.total_bands / (ms2 / 1e3), "ms_per_step": ms2, "ratio_vs_fp32": ms2 / ms}
            errors(res)
            if prec == "mixed":
                # which stages ran on the tensor cores (none where no length has a tensor-core pass,
                # or where the autotuner measured the FP32 kernels faster)
                res["tensor_core_stages"] = tc_stages()
                res["tensor_cores_available"] = bool(p2.info["tensor_cores_available"])
                if p2.info["tensor_cores_available"]:
                    # the setting the autotuner did not keep (default schedules), same inputs
                    in_use = (p2.info["tensor_core_planes"] | p2.info["tensor_core_passes"]) != 0
                    p2.set_tensor_cores(not in_use)
                    ms_o = run_timed()
                    other = {"tensor_cores": not in_use, "value": w.total_bands / (ms_o / 1e3),
                             "ms_per_step": ms_o, "tensor_core_stages": tc_stages()}
                    errors(other)
                    res["other_setting"] = other
            del x2, cube2, p2, vd2
            return res, o2

        def rel_l2(a, ref):
            d = a.to(torch.complex128) - ref
            return (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(ref)).item()

        o64 = None
        try:
            fp64, o64 = time_plan("fp64")
        except fftb.FFTBError as e:
            fp64 = {"unavailable": str(e)}
        try:
            mixed_tc, o_tc = time_plan("mixed", reps=5, ref=o64)
            del o_tc
        except fftb.FFTBError as e:
            mixed_tc = {"unavailable": str(e)}
        err_vs_fp64 = None if o64 is None else rel_l2(out, o64)
        if err is None:
            err = err_vs_fp64
        del o64
        fastest = max([("fp32", value)] + ([("mixed_tc", mixed_tc["value"])] if "value" in mixed_tc else []),
                      key=lambda t: t[1])
        mixed_vs_fp64 = {"mixed": fastest[0], "mixed_bands_per_s": fastest[1],
                         "fp64_bands_per_s": fp64.get("value"),
                         "ratio": None if "value" not in fp64 else fastest[1] / fp64["value"],
                         "mixed_rel_l2_vs_fp64_gpu": err_vs_fp64 if fastest[0] == "fp32"
                         else mixed_tc.get("rel_l2_vs_fp64_gpu"),
                         "what": "the fastest path whose bulk butterflies run in FP32 (FP32 on CUDA cores, or "
                                 "MIXED_TC with split-FP16 tensor-core DFT stages) against the plain FP64 GPU "
                                 "path, same workload"}

        # context: the same transform without pruning, as the padded full-cube
        # 3D FFT a plane-wave code would otherwise run (scatter into the cube,
        # cuFFT through torch.fft, gather), in FP32
        def time_full_cube(reps=3):
            xm, om = band_major(x), band_major(out)
            n0, n1, n2 = w.n
            vol = n0 * n1 * n2
            idx = []
            for g in spheres:
                g = np.asarray(g)
                flat = ((g[:, 2] % n2) * n1 + (g[:, 1] % n1)) * n0 + (g[:, 0] % n0)
                idx.append(torch.from_numpy(flat.astype(np.int64)).to(dev))
            vd = torch.from_numpy(w.potential().astype(np.float32)).to(dev) if w.direction == "apply" else None
            chunk = max(1, min(64, (2 << 30) // (vol * 8)))
            pad = torch.empty(chunk * vol, dtype=torch.complex64, device=dev)
            res = torch.empty_like(xm)

            def run():
                off = 0
                for k, (ik, b) in enumerate(zip(idx, w.bands)):
                    ng = ik.numel()
                    for b0 in range(0, b, chunk):
                        nb = min(chunk, b - b0)
                        src = xm[off + b0 * ng: off + (b0 + nb) * ng].view(nb, ng)
                        cube_c = pad[: nb * vol].view(nb, vol)
                        cube_c.zero_()
                        cube_c.index_copy_(1, ik, src)
                        r = torch.fft.ifftn(cube_c.view(nb, n2, n1, n0), dim=(1, 2, 3), norm="forward")
                        if vd is not None:
                            r = r * vd
                        f = torch.fft.fftn(r, dim=(1, 2, 3), norm="backward").view(nb, vol)
                        res[off + b0 * ng: off + (b0 + nb) * ng].view(nb, ng).copy_(f.index_select(1, ik))
                    off += b * ng

            run()
            evs3 = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run()
                b.record(stream)
                evs3.append((a, b))
            torch.cuda.synchronize(dev)
            ms3 = sum(a.elapsed_time(b) for a, b in evs3) / len(evs3)
            agree = (torch.linalg.vector_norm(res - om) / torch.linalg.vector_norm(om)).item()
            del pad, res
            return {"value": w.total_bands / (ms3 / 1e3), "ms_per_step": ms3, "ratio_vs_fp32": ms3 / ms,
                    "rel_l2_vs_ours": agree,
                    "what": "zero-padded full-cube 3D FFT per band (scatter, torch.fft/cuFFT inverse and forward, "
                            "gather), FP32; no pruning"}
        try:
            full_cube = time_full_cube()
        except Exception as e:  # a context figure: report, never fail the bench
            full_cube = {"unavailable": f"{type(e).__name__}: {e}"}

        # context: this engine without pruning, a plan over the whole
        # frequency box (every stick and slab occupied), FP32 and autotuned,
        # on a band prefix of the first k-point; checked against the pruned
        # result on those bands
        def time_full_box(reps=3):
            xm, om = band_major(x), band_major(out)
            n0, n1, n2 = w.n
            vol = n0 * n1 * n2
            nb = int(max(1, min(w.bands[0], (6 << 30) // (3 * vol * 8))))
            gbox = fftb.fftb_box_enumerate(w.n)
            pb = fftb.Plan(w.n, w.direction, "fp32", g_lists=[gbox], bands=[nb])
            if w.direction == "apply":
                vbox = torch.from_numpy(w.potential().astype(np.float32)).to(dev)
                pb.set_potential(vbox)
            pb.autotune(2)
            g0 = np.asarray(spheres[0]).astype(np.int64)
            pos = torch.from_numpy(((g0[:, 1] + n1 // 2) * n0 + (g0[:, 0] + n0 // 2)) * n2 +
                                   (g0[:, 2] + n2 // 2)).to(dev)
            ng = len(g0)
            if w.direction == "r2g":
                xb = x[: nb * vol].clone()
            else:
                xb = torch.zeros(nb, vol, dtype=torch.complex64, device=dev)
                xb.index_copy_(1, pos, xm[: nb * ng].view(nb, ng))
                xb = xb.view(-1)
            ob = torch.empty(nb * vol, dtype=torch.complex64, device=dev)
            cb = torch.empty(nb * vol, dtype=torch.complex64, device=dev) if w.direction == "roundtrip" else None
            for _ in range(2):
                pb.execute(xb, ob, cb)
            evb = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                pb.execute(xb, ob, cb)
                b.record(stream)
                evb.append((a, b))
            torch.cuda.synchronize(dev)
            msb = sum(a.elapsed_time(b) for a, b in evb) / len(evb)
            if w.direction == "g2r":
                got, ref = ob, out[: nb * vol]
            else:
                got, ref = ob.view(nb, vol).index_select(1, pos), om[: nb * ng].view(nb, ng)
            agree = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
            per_band_pruned = ms / w.total_bands
            del xb, ob, cb, pb
            return {"value": nb / (msb / 1e3), "bands": nb, "ms": msb, "rel_l2_vs_ours": agree,
                    "ratio_per_band_vs_fp32": (msb / nb) / per_band_pruned,
                    "what": "this engine over the whole frequency box (no pruning: every stick and slab), FP32, "
                            "autotuned, first k-point's bands"}
        try:
            full_box = time_full_box()
        except Exception as e:  # a context figure: report, never fail the bench
            full_box = {"unavailable": f"{type(e).__name__}: {e}"}

        # end to end through the C ABI with host buffers (copies in the timed region);
        # the pinned buffers are allocated from the CPUs local to the GPU, so their
        # pages sit on the GPU's NUMA node
        affinity = os.sched_getaffinity(0)
        local_cpus = gpu_local_cpus(local)
        if local_cpus:
            os.sched_setaffinity(0, local_cpus)
        try:
            pin_in = torch.from_numpy(c).pin_memory()
            pin_out = torch.empty_like(pin_in).pin_memory()
        finally:
            os.sched_setaffinity(0, affinity)
        pin_node = "gpu-local NUMA node" if local_cpus else "default placement"
        cptr = None if cube is None else cube.data_ptr()
        for _ in range(2):
            fftb.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cptr, stream.cuda_stream)
        t_e2e = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fftb.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cptr, stream.cuda_stream)
            t_e2e.append(time.perf_counter() - t0)
        e2e_s = sum(t_e2e) / len(t_e2e)
        e2e_ms = sorted(1e3 * t for t in t_e2e)
        nbytes = pin_in.numel() * 8

        cpu = None
        if world == 1:
            import oracle
            ks = w.kshift if w.kshift is not None else [(0.0, 0.0, 0.0)]
            osph = [oracle.sphere_gvectors(w.n, w.radius, k) for k in ks]
            v64 = w.potential().astype(np.float32).astype(np.float64) if w.direction == "apply" else None
            rate, done, el = time_oracle(w, osph, w.coefficients(osph), v64, budget_s=10.0)
            cpu = {"value": rate, "unit": "bands/s", "cores": 1, "kind": "oracle",
                   "sample": f"{done} band transforms of the workload ({el:.1f} s), numpy pocketfft FP64",
                   "cpu_model": cpu_model(), "host_cores": os.cpu_count()}
            try:
                r_all, d_all, busy, wall, cores = time_oracle_all_cores(w, budget_s=8.0)
                cpu["all_cores"] = {"value": r_all, "unit": "bands/s", "cores": cores, "kind": "oracle",
                                    "sample": f"{d_all} band transforms over {cores} spawned processes, "
                                              f"{busy:.1f} s each ({wall:.1f} s with start-up)"}
            except Exception as e:  # context only: never fail the bench
                cpu["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}

        # the 64^3 workload (64 bands, cube kept in HBM) timed the same way,
        # as a figure beside the headline
        extra = {}
        if w.name != "sphere64_rt" and not args.no_extra:
            try:
                extra["sphere64_rt"] = time_workload(fftb, "sphere64_rt", dev, flush, stream, args)
            except Exception as e:  # context only: never fail the bench
                extra["sphere64_rt"] = {"unavailable": f"{type(e).__name__}: {e}"}

        line = {"metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_median_of_50": median50,
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": w.desc, "name": w.name, "grid": list(w.n), "radius": w.radius,
                           "ngw": ngws, "bands_per_gpu": w.total_bands, "precision": "fp32",
                           "parallelism": f"bands x{world}", "global_bands": world * w.total_bands,
                           "shard": "contiguous band shards of one global batch (band_shard), no collective "
                                    "on the data path",
                           "chunk_bands": plan.info["chunk_bands"],
                           "graph": w.graph, "graph_launches_in_timed_steps": graph_steps, "autotuned": w.tune,
                           "l2": "flushed between timed steps (256 MiB write)"},
                "rel_l2": err,
                "rel_l2_vs_fp64_gpu": err_vs_fp64,
                "mixed_vs_fp64": mixed_vs_fp64,
                "fp64_gpu": fp64,
                "mixed_tc_gpu": mixed_tc,
                "full_cube_cufft_gpu": full_cube,
                "full_box_ours_gpu": full_box,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": {"value": w.total_bands / e2e_s, "unit": "bands/s", "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes, "ms_per_step_min_median_max":
                        [round(e2e_ms[0], 3), round(statistics.median(e2e_ms), 3), round(e2e_ms[-1], 3)],
                        "host_buffers": f"pinned, {pin_node}"},
                "gpu_launches": launches,
                "clocks": clocks,
                "other_workloads": extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["sphere64_rt", "sphere96_multik", "sphere128_apply", "sphere160_large", "sphere256_e2",
                             "sphere64_rt_batchfast"])
    ap.add_argument("--no-extra", action="store_true", help="skip the 64^3 figure beside the headline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
