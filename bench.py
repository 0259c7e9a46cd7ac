"""Benchmark: batched pruned sphere <-> cube FFT, G -> r -> G, bands/s.

Workload (one GPU): 64^3 grid, cutoff |G| <= 16 (17077 G vectors), 64 bands,
FP32, coefficients complex Gaussian x exp(-|G|^2/(2*64)), round trip
G -> r -> G with the real-space cube written to HBM and read back. A step is
one fftb_execute of the whole batch. Under torchrun each rank runs its own 64
bands on its own GPU (bands are independent: weak scaling, no collective on
the data path).

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

METRIC = "sphere-FFT bands/sec (G->r->G) and % HBM roofline, mixed vs FP64 at L2<=1e-5"
N, RADIUS, BANDS, SEED = (64, 64, 64), 16.0, 64, 2
WORKLOAD = "64^3 grid, |G|<=16 (17077 G), 64 bands, G->r->G round trip, cube kept in HBM"
L2_FLUSH_BYTES = 256 << 20


def workload_inputs(g):
    c = fi.complex_gaussian((BANDS, len(g)), SEED) * fi.gaussian_envelope(g, 8.0)[None, :]
    return c


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fft_core.cuh", "kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2406_05577_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per band of one kernel from the committed ncu summary, or
    None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_band")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if bus_id:
            cmd += ["-i", bus_id]
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


def time_oracle(g, c, budget_s):
    """Bands/s of the FP64 oracle round trip over a bounded sample."""
    import oracle
    done, t0 = 0, time.perf_counter()
    while True:
        b = done % BANDS
        oracle.roundtrip(g, c[b], N)
        done += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            return done / el, done, el


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    g = oracle.sphere_gvectors(N, RADIUS)
    c = workload_inputs(g)
    sample = 16
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for b in range(sample):
            oracle.roundtrip(g, c[(step * sample + b) % BANDS], N)
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = sample / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(N), "radius": RADIUS, "bands": BANDS,
                       "precision": "fp64 (CPU oracle)", "step_sample_bands": sample},
            "cpu_baseline": {"value": value, "unit": "bands/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample} bands of the workload per step, numpy pocketfft FP64"},
            "e2e": {"value": value, "unit": "bands/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def stage_bytes(kind, plan_info, ngw, S):
    """Algorithmic (compulsory) bytes per band of one kernel kind."""
    c = plan_info["complex_bytes"]
    vol = N[0] * N[1] * N[2]
    return {"stick_g2r": (ngw + S * N[2]) * c, "plane_g2r": (S * N[2] + vol) * c,
            "plane_r2g": (vol + S * N[2]) * c, "stick_r2g": (S * N[2] + ngw) * c,
            "plane_apply": 2 * S * N[2] * c}[kind]


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

    plan = fftb.Plan(N, "roundtrip", "fp32", radius=RADIUS, bands=[BANDS])
    info = plan.info
    g = plan.sphere(0)
    S = info["max_sticks"]
    c = workload_inputs(g).astype(np.complex64)
    x = torch.from_numpy(c.reshape(-1)).to(dev)
    out = torch.empty_like(x)
    cube = torch.empty(info["cube_elems"], dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        plan.execute(x, out, cube)
    torch.cuda.synchronize(dev)
    # correctness of this very run: round trip returns N0 N1 N2 * c
    err = (torch.linalg.vector_norm(out - float(np.prod(N)) * x) /
           torch.linalg.vector_norm(float(np.prod(N)) * x)).item()

    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id  # may not exist on older torch
    except Exception:
        bus = None
    sampler = ClockSampler(None)
    fftb.fftb_plan_set_timing(plan.handle, True)
    fftb.fftb_plan_stage_times(plan.handle)  # reset
    launches0 = plan.launches()
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
    stage = fftb.fftb_plan_stage_times(plan.handle)
    fftb.fftb_plan_set_timing(plan.handle, False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    value = world * BANDS / (ms / 1e3)

    # dominant kernel roofline (algorithmic bytes / live event duration)
    hbm, peak_kind = peaks()
    dom = max((k for k in stage if stage[k][1] > 0), key=lambda k: stage[k][0])
    dom_ms, dom_n = stage[dom]
    per_launch_bands = BANDS / (dom_n / args.steps)
    alg = stage_bytes(dom, info, len(g), S) * per_launch_bands
    achieved = alg / (dom_ms / dom_n / 1e3) / 1e9
    traffic_band = ncu_traffic(dom)
    vol = N[0] * N[1] * N[2]
    step_bytes = 2 * (len(g) + vol) * 8 * BANDS
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": peak_kind,
                "traffic": None if traffic_band is None else traffic_band * per_launch_bands,
                "stage_ms_per_step": {k: v[0] / args.steps for k, v in stage.items() if v[1]},
                "step_compulsory_gbs": step_bytes / (ms / 1e3) / 1e9,
                "step_compulsory_frac": step_bytes / (ms / 1e3) / 1e9 / hbm}

    line = None
    if rank == 0:
        # FP64 GPU path on the same workload (the comparison the metric names)
        p64 = fftb.Plan(N, "roundtrip", "fp64", radius=RADIUS, bands=[BANDS])
        x64 = torch.from_numpy(workload_inputs(g).reshape(-1)).to(dev)
        o64 = torch.empty_like(x64)
        cube64 = torch.empty(p64.info["cube_elems"], dtype=torch.complex128, device=dev)
        for _ in range(3):
            p64.execute(x64, o64, cube64)
        e64 = []
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            p64.execute(x64, o64, cube64)
            b.record(stream)
            e64.append((a, b))
        torch.cuda.synchronize(dev)
        ms64 = sum(a.elapsed_time(b) for a, b in e64) / len(e64)
        del cube64, o64, x64, p64

        # end to end through the C ABI with host buffers (copies in the timed region)
        pin_in = torch.from_numpy(c.reshape(-1)).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        for _ in range(2):
            fftb.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cube.data_ptr(),
                                   stream.cuda_stream)
        t_e2e = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            fftb.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cube.data_ptr(),
                                   stream.cuda_stream)
            t_e2e.append(time.perf_counter() - t0)
        e2e_s = sum(t_e2e) / len(t_e2e)
        nbytes = pin_in.numel() * 8

        cpu = None
        if world == 1:
            import oracle  # noqa: F401
            rate, done, el = time_oracle(g, workload_inputs(g), budget_s=10.0)
            cpu = {"value": rate, "unit": "bands/s", "cores": 1, "kind": "oracle",
                   "sample": f"{done} band round trips of the workload ({el:.1f} s), numpy pocketfft FP64"}

        line = {"metric": METRIC, "value": value, "unit": "bands/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "grid": list(N), "radius": RADIUS, "ngw": int(len(g)),
                           "bands_per_gpu": BANDS, "precision": "fp32", "parallelism": f"bands x{world}",
                           "l2": "flushed between timed steps (256 MiB write)"},
                "rel_l2_roundtrip": err,
                "fp64_gpu": {"value": BANDS / (ms64 / 1e3), "ms_per_step": ms64,
                             "ratio_fp32_over_fp64": ms64 / ms},
                "roofline": roofline,
                "cpu_baseline": cpu,
                "e2e": {"value": BANDS / e2e_s, "unit": "bands/s", "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes},
                "gpu_launches": launches,
                "clocks": clocks}
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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
