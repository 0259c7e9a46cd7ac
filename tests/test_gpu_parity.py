"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 over the whole output batch): FP64 <= 1e-12,
FP32 <= 2e-6. Inputs are rounded to the plan's precision first and the
oracle sees the rounded values widened to float64, so input rounding is not
charged to the transform.
"""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-6, "mixed": 1e-5}


@pytest.fixture(scope="module")
def F():
    import torch
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb
    assert torch.cuda.is_available()
    return fftb


def relerr(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x, prec):
    import torch
    dt = torch.complex128 if prec == "fp64" else torch.complex64  # fp32 and mixed store complex64
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


def rounded(x, prec):
    return x.astype(np.complex128 if prec == "fp64" else np.complex64).astype(np.complex128)


def sphere_batch(ngws, bands, seed, prec):
    parts = [rounded(fi.complex_gaussian((b, n), seed + 17 * k), prec)
             for k, (n, b) in enumerate(zip(ngws, bands))]
    return parts


def run_plan(F, n, direction, prec, x_host, **kw):
    import torch
    plan = F.Plan(n, direction, prec, **kw)
    info = plan.info
    cd = plan.complex_dtype
    x = to_dev(x_host, prec)
    if direction == "g2r":
        out = torch.empty(info["cube_elems"], dtype=cd, device="cuda")
    else:
        out = torch.empty(info["sphere_elems"], dtype=cd, device="cuda")
    cube = None
    if direction == "roundtrip":
        cube = torch.empty(info["cube_elems"], dtype=cd, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.complex128)
    cube_np = cube.cpu().numpy().astype(np.complex128) if cube is not None else None
    return plan, res, cube_np


CASES = [
    # (grid, radius, kshift)
    ((24, 24, 24), 6.0, None),
    ((32, 32, 48), 10.0, (0.25, -0.4, 0.1)),
    ((20, 20, 40), 6.5, (-0.5, 0.3, 0.45)),
    ((12, 12, 16), 3.0, (0.1, 0.2, -0.3)),
    ((48, 48, 24), 9.0, None),
    ((16, 16, 96), 4.5, (0.0, 0.5, -0.25)),
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,r,k", CASES)
def test_g2r_r2g_roundtrip_vs_oracle(F, n, r, k, prec):
    bands = 5
    g = oracle.sphere_gvectors(n, r, k if k else (0, 0, 0))
    c = sphere_batch([len(g)], [bands], seed=31, prec=prec)[0]
    kw = dict(radius=r, bands=[bands])
    if k:
        kw["kshift"] = [k]
    # G -> r
    plan, cube, _ = run_plan(F, n, "g2r", prec, c, **kw)
    assert np.array_equal(plan.sphere(0), g)
    want = oracle.g2r(g, c, n).reshape(-1)
    assert relerr(cube, want) <= TOL[prec]
    # r -> G on an independent random cube
    R = rounded(fi.complex_gaussian((bands, n[2], n[1], n[0]), 32), prec)
    _, sph, _ = run_plan(F, n, "r2g", prec, R, **kw)
    assert relerr(sph, oracle.r2g(g, R, n).reshape(-1)) <= TOL[prec]
    # round trip keeps the cube and returns N0 N1 N2 * c
    _, back, cub = run_plan(F, n, "roundtrip", prec, c, **kw)
    assert relerr(cub, want) <= TOL[prec]
    assert relerr(back, np.prod(n) * c.reshape(-1)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uneven_kpoints_and_chunks(F, prec):
    n, r = (24, 24, 24), 6.0
    ks = fi.kshifts(4, seed=7)
    bands = [3, 0, 5, 2]  # a k-point without bands
    gs = [oracle.sphere_gvectors(n, r, k) for k in ks]
    cs = sphere_batch([len(g) for g in gs], bands, seed=41, prec=prec)
    x = np.concatenate([c.reshape(-1) for c in cs])
    # chunk of 3 bands: chunks straddle k-points and end ragged (10 bands)
    plan, cube, _ = run_plan(F, n, "g2r", prec, x, radius=r, kshift=ks, bands=bands, max_chunk_bands=3)
    assert plan.info["chunk_bands"] == 3 and plan.info["total_bands"] == 10
    want = np.concatenate([oracle.g2r(g, c, n).reshape(-1) for g, c in zip(gs, cs) if len(c)])
    assert relerr(cube, want) <= TOL[prec]
    _, back, _ = run_plan(F, n, "roundtrip", prec, x, radius=r, kshift=ks, bands=bands, max_chunk_bands=3)
    assert relerr(back, np.prod(n) * x) <= TOL[prec]


def test_explicit_user_order_and_empty_sphere(F):
    n = (32, 32, 48)
    g = oracle.sphere_gvectors(n, 9.0)
    perm = np.random.default_rng(5).permutation(len(g))
    gu = g[perm]
    c = fi.complex_gaussian((2, len(gu)), 51)
    empty = np.zeros((0, 3), np.int32)
    x = c.reshape(-1)
    plan, cube, _ = run_plan(F, n, "g2r", "fp64", x, g_lists=[gu, empty], bands=[2, 1])
    assert np.array_equal(plan.sphere(0), gu) and plan.ngw(1) == 0
    want = oracle.g2r(gu, c, n).reshape(-1)
    vol = np.prod(n)
    assert relerr(cube[: 2 * vol], want) <= 1e-12
    assert np.abs(cube[2 * vol:]).max() == 0.0  # empty sphere -> zero cube
    R = fi.complex_gaussian((3, n[2], n[1], n[0]), 52)
    _, sph, _ = run_plan(F, n, "r2g", "fp64", R, g_lists=[gu, empty], bands=[2, 1])
    assert relerr(sph, oracle.r2g(gu, R[:2], n).reshape(-1)) <= 1e-12


def test_single_g_vector_sphere(F):
    # r = 0: only G = 0; the cube is the constant c(0)
    n = (16, 16, 16)
    c = np.array([[1.5 - 0.5j], [2.0 + 1.0j]])
    _, cube, _ = run_plan(F, n, "g2r", "fp64", c, radius=0.0, bands=[2])
    cube = cube.reshape(2, -1)
    assert np.abs(cube - c).max() < 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,r", [((24, 24, 24), 6.0), ((32, 32, 48), 10.0)])
def test_apply_potential_vs_oracle(F, n, r, prec):
    import torch
    bands = 3
    g = oracle.sphere_gvectors(n, r)
    c = sphere_batch([len(g)], [bands], seed=61, prec=prec)[0]
    v = fi.gaussian_potential(n, 8, 2.0, seed=62)
    vr = v.astype(np.float64 if prec == "fp64" else np.float32)
    plan = F.Plan(n, "apply", prec, radius=r, bands=[bands])
    vd = torch.from_numpy(np.ascontiguousarray(vr)).cuda()
    plan.set_potential(vd)
    x = to_dev(c, prec)
    out = torch.empty_like(x)
    plan.execute(x, out)
    torch.cuda.synchronize()
    want = oracle.apply_potential(g, c, vr.astype(np.float64), n)
    assert relerr(out.cpu().numpy(), want) <= TOL[prec]


def test_execute_argument_errors(F):
    import torch
    plan = F.Plan((24, 24, 24), "roundtrip", "fp32", radius=6.0, bands=[2])
    x = torch.zeros(plan.info["sphere_elems"], dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(F.FFTBError):  # ROUNDTRIP needs a cube
        F.fftb_execute(plan.handle, x.data_ptr(), y.data_ptr(), None, None)
    with pytest.raises(F.FFTBError):  # in == out
        F.fftb_execute(plan.handle, x.data_ptr(), x.data_ptr(), y.data_ptr(), None)
    with pytest.raises(F.FFTBError):  # misaligned
        F.fftb_execute(plan.handle, x.data_ptr() + 4, y.data_ptr(), y.data_ptr(), None)
    ap = F.Plan((24, 24, 24), "apply", "fp32", radius=6.0, bands=[2])
    with pytest.raises(F.FFTBError):  # apply without a potential
        F.fftb_execute(ap.handle, x.data_ptr(), y.data_ptr(), None, None)


def test_host_buffer_entry_point(F):
    n, r = (24, 24, 24), 6.0
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((3, len(g)), 71)
    plan = F.Plan(n, "roundtrip", "fp64", radius=r, bands=[3])
    xin = np.ascontiguousarray(c.reshape(-1))
    xout = np.zeros_like(xin)
    F.fftb_execute_host(plan.handle, xin.ctypes.data, xout.ctypes.data, None, None)
    assert relerr(xout, np.prod(n) * xin) <= 1e-12
    # two pieces (one and two bands), four kernels each
    assert plan.launches() == 2 * plan.info["kernels_per_execute"]


@pytest.mark.parametrize("direction", ["g2r", "r2g", "roundtrip", "apply"])
def test_host_pipeline_matches_device_execute(F, direction):
    """The host-buffer entry point splits the bands into pieces (here across a
    k-point boundary and band chunks) and overlaps copies with transforms: its
    results are those of the device entry point, bit for bit."""
    import torch
    n, r = (32, 32, 32), 7.5
    ks = np.array([(0.1, 0.2, -0.3), (-0.4, 0.0, 0.25), (0.3, -0.45, 0.0)])
    bands = [3, 1, 6]
    plan = F.Plan(n, direction, "fp32", radius=r, kshift=ks, bands=bands, max_chunk_bands=2)
    info = plan.info
    if direction == "apply":
        v = fi.gaussian_potential(n, 8, 3.0, seed=81).astype(np.float32)
        plan.set_potential(torch.from_numpy(v).cuda())
    nin = info["cube_elems"] if direction == "r2g" else info["sphere_elems"]
    nout = info["cube_elems"] if direction == "g2r" else info["sphere_elems"]
    xin = fi.complex_gaussian((nin,), 82).astype(np.complex64)
    xd = torch.from_numpy(xin).cuda()
    od = torch.empty(nout, dtype=torch.complex64, device="cuda")
    cd = torch.empty(info["cube_elems"], dtype=torch.complex64, device="cuda") if direction == "roundtrip" else None
    plan.execute(xd, od, cd)
    torch.cuda.synchronize()
    want = od.cpu().numpy()
    pin_in = torch.from_numpy(xin).pin_memory()
    pin_out = torch.empty(nout, dtype=torch.complex64).pin_memory()
    cube_ptr = None
    if direction == "roundtrip":
        cube2 = torch.empty(info["cube_elems"], dtype=torch.complex64, device="cuda")
        cube_ptr = cube2.data_ptr()
    s = torch.cuda.Stream()
    F.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cube_ptr, s.cuda_stream)
    assert np.array_equal(pin_out.numpy(), want)
    if direction == "roundtrip":
        assert torch.equal(cube2, cd)


def test_plan_execute_host_method_and_context(F):
    """The Plan class's host-buffer call (pinned CPU tensors) equals the
    device call; a plan used as a context manager is released on exit."""
    import torch
    n, r, bands = (32, 32, 32), 8.0, 3
    with F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands]) as plan:
        g = plan.sphere(0)
        c = fi.complex_gaussian((bands, len(g)), 84).astype(np.complex64).reshape(-1)
        x = torch.from_numpy(c).cuda()
        out = torch.empty_like(x)
        cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
        plan.execute(x, out, cube)
        torch.cuda.synchronize()
        hin = torch.from_numpy(c).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        plan.execute_host(hin, hout)
        assert np.array_equal(hout.numpy(), out.cpu().numpy())
        with pytest.raises(ValueError):
            plan.execute_host(x, hout)  # a device tensor where host memory is expected
    assert plan.handle is None


def test_graph_replay_and_update(F):
    import torch
    n, r, bands = (32, 32, 48), 10.0, 6
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((bands, len(g)), 81).astype(np.complex64)
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands], max_chunk_bands=4)
    plan.set_graph(True)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    outs = [torch.empty_like(x) for _ in range(2)]
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.execute(x, outs[0], cube)   # records and instantiates
        plan.execute(x, outs[0], cube)   # replays
        plan.execute(x, outs[1], cube)   # new buffers: graph update
    torch.cuda.synchronize()
    want = np.prod(n) * c.reshape(-1).astype(np.complex128)
    for o in outs:
        assert relerr(o.cpu().numpy(), want) <= TOL["fp32"]
    assert relerr(cube.cpu().numpy(), oracle.g2r(g, c.astype(np.complex128), n).reshape(-1)) <= TOL["fp32"]
    assert plan.launches() == 3 * plan.info["kernels_per_execute"]
    assert F.fftb_plan_get_info(plan.handle)["graph_launches"] == 3


def test_graph_on_the_default_stream(F):
    """The legacy default stream cannot be captured: the plan records on its
    own stream and replays the graph on the default stream."""
    import torch
    n, r, bands = (32, 32, 32), 8.0, 5
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((bands, len(g)), 83).astype(np.complex64)
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands], max_chunk_bands=2)
    plan.set_graph(True)
    x = torch.from_numpy(c.reshape(-1)).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    assert torch.cuda.current_stream().cuda_stream == 0
    for _ in range(3):
        out.zero_()
        plan.execute(x, out, cube)
    torch.cuda.synchronize()
    assert F.fftb_plan_get_info(plan.handle)["graph_launches"] == 3
    assert relerr(out.cpu().numpy(), np.prod(n) * c.reshape(-1).astype(np.complex128)) <= TOL["fp32"]
    assert relerr(cube.cpu().numpy(), oracle.g2r(g, c.astype(np.complex128), n).reshape(-1)) <= TOL["fp32"]


def test_autotune_keeps_results(F, tmp_path, monkeypatch):
    import torch
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    n, r = (24, 24, 24), 6.0
    ks = fi.kshifts(3, seed=9)
    bands = [5, 2, 7]
    gs = [oracle.sphere_gvectors(n, r, k) for k in ks]
    cs = [fi.complex_gaussian((b, len(gk)), 90 + i) for i, (gk, b) in enumerate(zip(gs, bands))]
    x = np.concatenate([c.reshape(-1) for c in cs])
    for attempt in range(2):  # second plan reads the cache
        plan = F.Plan(n, "g2r", "fp64", radius=r, kshift=ks, bands=bands)
        plan.autotune(2)
        assert 1 <= plan.info["chunk_bands"] <= 14
        xd = torch.from_numpy(x).cuda()
        out = torch.empty(plan.info["cube_elems"], dtype=torch.complex128, device="cuda")
        plan.execute(xd, out)
        torch.cuda.synchronize()
        want = np.concatenate([oracle.g2r(gk, c, n).reshape(-1) for gk, c in zip(gs, cs)])
        assert relerr(out.cpu().numpy(), want) <= TOL["fp64"]
    lines = (tmp_path / "tune.txt").read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("24x24x24|")


@pytest.mark.parametrize("n,r,k,bands", [((64, 64, 64), 16.0, (0.3, -0.2, 0.1), 6),
                                         ((128, 128, 128), 32.0, None, 2),
                                         ((64, 64, 32), 12.0, None, 4),
                                         ((24, 24, 24), 6.0, None, 3)])
def test_mixed_tc_vs_oracle(F, n, r, k, bands):
    """Split-precision tensor-core radix-8 passes: relative L2 <= 1e-5."""
    tol = 1e-5
    g = oracle.sphere_gvectors(n, r, k if k else (0, 0, 0))
    c = fi.complex_gaussian((bands, len(g)), 111).astype(np.complex64).astype(np.complex128)
    kw = dict(radius=r, bands=[bands])
    if k:
        kw["kshift"] = [k]
    _, cube, _ = run_plan(F, n, "g2r", "mixed", c, **kw)
    want = oracle.g2r(g, c, n).reshape(-1)
    e1 = relerr(cube, want)
    R = rounded(fi.complex_gaussian((bands, n[2], n[1], n[0]), 112), "fp32")
    _, sph, _ = run_plan(F, n, "r2g", "mixed", R, **kw)
    e2 = relerr(sph, oracle.r2g(g, R, n).reshape(-1))
    _, back, _ = run_plan(F, n, "roundtrip", "mixed", c, **kw)
    e3 = relerr(back, np.prod(n) * c.reshape(-1))
    assert max(e1, e2, e3) <= tol, (e1, e2, e3)


def test_mixed_tc_apply_vs_oracle(F):
    import torch
    n, r, bands = (64, 64, 64), 16.0, 4
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((bands, len(g)), 121).astype(np.complex64).astype(np.complex128)
    v = fi.gaussian_potential(n, 32, 4.0, seed=122).astype(np.float32)
    plan = F.Plan(n, "apply", "mixed", radius=r, bands=[bands])
    vd = torch.from_numpy(v).cuda()
    plan.set_potential(vd)
    x = torch.from_numpy(c.astype(np.complex64).reshape(-1)).cuda()
    out = torch.empty_like(x)
    plan.execute(x, out)
    torch.cuda.synchronize()
    want = oracle.apply_potential(g, c, v.astype(np.float64), n)
    assert relerr(out.cpu().numpy(), want) <= 1e-5


def test_host_pipeline_many_pieces(F):
    """A band-major batch of 25 600 (band, z) planes goes through the
    host-buffer pipeline in three pieces (about 8192 planes each): bit for bit
    the device entry point's results."""
    import torch
    n, r, bands = (64, 64, 64), 16.0, 400
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, bands=[bands])
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 85).astype(np.complex64).reshape(-1)
    x = torch.from_numpy(c).cuda()
    out = torch.empty_like(x)
    cube = torch.empty(plan.info["cube_elems"], dtype=torch.complex64, device="cuda")
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    l0 = plan.launches()
    hin = torch.from_numpy(c).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    cube2 = torch.empty_like(cube)
    F.fftb_execute_host(plan.handle, hin.data_ptr(), hout.data_ptr(), cube2.data_ptr(), None)
    assert np.array_equal(hout.numpy(), out.cpu().numpy())
    assert torch.equal(cube2, cube)
    # three pieces, each its own launch sequence (at least one chunk each)
    assert plan.launches() - l0 >= 3 * 4
