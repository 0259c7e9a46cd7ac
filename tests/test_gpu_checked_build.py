"""The checked build (libfftb_check.so, kernels compiled with FFTB_CHECK:
every global and slab-plane index of the stick and plane kernels is tested
against its buffer before the access, a failure reported as
FFTB_ERR_DEVICE_BOUNDS). Valid plans of every kernel family the checks cover
run through it in a child process (FFTB_LIBRARY selects the library) and
must report nothing and match the FP64 oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import fftb_inputs as fi, oracle
from paper_2406_05577_gb300 import fftb
assert fftb.LIB_PATH.endswith("libfftb_check.so"), fftb.LIB_PATH

def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

def roundtrip(n, r, prec, bands, **kw):
    sched = kw.pop("sched", None)
    pf = kw.pop("prefetch", None)
    clusters = kw.pop("clusters", False)
    plan = fftb.Plan(n, "roundtrip", prec, radius=r, bands=bands, **kw)
    if clusters:
        plan.set_plane_clusters(True)
    if sched is not None:
        plan.set_radix_schedule(*sched)
    if pf is not None:
        plan.set_prefetch(pf)
    gs = [plan.sphere(k) for k in range(len(bands))]
    cd = np.complex128 if prec == "fp64" else np.complex64
    parts = [fi.complex_gaussian((b, len(g)), 7 + k).astype(cd) for k, (g, b) in enumerate(zip(gs, bands))]
    lay = kw.get("layout", 0)
    x = torch.from_numpy(np.concatenate([(p.T if lay else p).reshape(-1) for p in parts])).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=x.dtype, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    plan.check()  # raises on FFTB_ERR_DEVICE_BOUNDS
    tol = 1e-12 if prec == "fp64" else 2e-6
    vol = n[0] * n[1] * n[2]
    assert rel(out.cpu().numpy(), vol * x.cpu().numpy()) <= tol, (n, prec)
    if not lay:
        R0 = cube[:vol].cpu().numpy()
        assert rel(R0, oracle.g2r(gs[0], parts[0][0].astype(np.complex128), n).reshape(-1)) <= tol, (n, prec)

roundtrip((24, 24, 24), 6.0, "fp64", [3])
roundtrip((64, 64, 64), 16.0, "fp32", [4], prefetch=2)
roundtrip((64, 64, 64), 16.0, "fp32", [4], prefetch=0)
roundtrip((160, 160, 160), 40.0, "fp32", [2], sched=(1, 1))
roundtrip((160, 160, 160), 40.0, "fp32", [2], prefetch=2)
roundtrip((32, 32, 48), 10.0, "fp32", [2, 3], kshift=[(0.1, 0.2, -0.3), (-0.4, 0.0, 0.25)], layout=1)
roundtrip((256, 256, 256), 64.0, "fp32", [1])
roundtrip((256, 256, 256), 64.0, "fp32", [2], clusters=True)   # slab planes split over two-CTA clusters
roundtrip((128, 128, 128), 32.0, "fp64", [1])
roundtrip((72, 80, 90), 17.5, "fp32", [3], max_chunk_bands=2)   # generic-extent path
roundtrip((15, 27, 25), 5.0, "fp64", [2], layout=1)

# the apply on two-CTA clusters
n = (256, 256, 256)
plan = fftb.Plan(n, "apply", "fp32", radius=64.0, bands=[1])
plan.set_plane_clusters(True)
v = fi.gaussian_potential(n, 8, 6.0, seed=6).astype(np.float32)
plan.set_potential(torch.from_numpy(v).cuda())
g = plan.sphere(0)
c = fi.complex_gaussian((1, len(g)), 10).astype(np.complex64)
x = torch.from_numpy(c.reshape(-1)).cuda()
out = torch.empty_like(x)
plan.execute(x, out)
torch.cuda.synchronize()
plan.check()
assert rel(out.cpu().numpy(), oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), n)) <= 2e-6
del plan, out, x
torch.cuda.empty_cache()

# apply and an explicit (non-canonical) sphere order
n, r = (32, 32, 32), 8.0
g = oracle.sphere_gvectors(n, r)
gu = g[np.random.default_rng(3).permutation(len(g))]
v = fi.gaussian_potential(n, 8, 3.0, seed=5).astype(np.float32)
plan = fftb.Plan(n, "apply", "fp32", g_lists=[gu], bands=[2])
plan.set_potential(torch.from_numpy(v).cuda())
c = fi.complex_gaussian((2, len(gu)), 9).astype(np.complex64)
x = torch.from_numpy(c.reshape(-1)).cuda()
out = torch.empty_like(x)
plan.execute(x, out)
torch.cuda.synchronize()
plan.check()
want = oracle.apply_potential(gu, c.astype(np.complex128), v.astype(np.float64), n)
assert rel(out.cpu().numpy(), want) <= 2e-6

# the allocation-free entry point
n, r = (64, 64, 64), 16.0
g = fftb.fftb_sphere_enumerate(n, r)
c = fi.complex_gaussian((3, len(g)), 11).astype(np.complex64)
x = torch.from_numpy(c.reshape(-1)).cuda()
o = torch.empty(3 * 64 ** 3, dtype=torch.complex64, device="cuda")
fftb.fftb_g2r_noalloc(n, r, None, 3, x.data_ptr(), o.data_ptr(), None)
torch.cuda.synchronize()
assert rel(o[:64 ** 3].cpu().numpy(), oracle.g2r(g, c[0].astype(np.complex128), n).reshape(-1)) <= 2e-6
print("checked build: every plan clean")
'''


def test_checked_build_runs_clean_and_matches_the_oracle():
    from paper_2406_05577_gb300 import build
    lib = build.build(check=True)
    assert lib.endswith("libfftb_check.so") and os.path.exists(lib)
    env = dict(os.environ, FFTB_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "every plan clean" in r.stdout
