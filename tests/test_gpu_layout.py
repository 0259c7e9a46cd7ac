"""Batch-fastest layout (Sec. 3.3: the batch dimension declared first is the
fastest in memory): per k-point the sphere batch is [ngw_k][B_k] and the cube
batch [N2][N1][N0][B_k]. The arithmetic is the band-major plan's, so FP32 and
FP64 results equal its results, permuted, bit for bit; every direction is also
checked against the FP64 oracle."""
import numpy as np
import pytest

import fftb_inputs as fi
import oracle

pytestmark = pytest.mark.gpu


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


def sph_bf(flat, ngws, bands):
    """band-major sphere batch -> batch-fastest (per k-point [ngw][B])"""
    out, o = [], 0
    for ng, b in zip(ngws, bands):
        out.append(flat[o:o + ng * b].reshape(b, ng).T.reshape(-1))
        o += ng * b
    return np.concatenate(out)


def cube_bf(flat, n, bands):
    """band-major cube batch -> batch-fastest (per k-point [N2][N1][N0][B])"""
    vol = n[0] * n[1] * n[2]
    out, o = [], 0
    for b in bands:
        out.append(flat[o:o + vol * b].reshape(b, vol).T.reshape(-1))
        o += vol * b
    return np.concatenate(out)


def execute(F, plan, x, direction, dtype):
    import torch
    info = plan.info
    nout = info["cube_elems"] if direction == "g2r" else info["sphere_elems"]
    out = torch.full((nout,), float("nan"), dtype=dtype, device="cuda")
    cube = torch.empty(info["cube_elems"], dtype=dtype, device="cuda") if direction == "roundtrip" else None
    plan.execute(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out, cube)
    torch.cuda.synchronize()
    plan.check()
    return out.cpu().numpy(), (cube.cpu().numpy() if cube is not None else None)


CASES = [
    # grid, radius, k-shifts, bands per k, precision
    ((32, 32, 32), 8.0, [(0.3, -0.2, 0.1), (-0.45, 0.4, -0.3)], [3, 5], "fp32"),
    ((64, 64, 64), 16.0, None, [6], "fp32"),
    ((96, 96, 96), 24.0, [(0.25, 0.0, -0.5)], [4], "fp32"),
    ((128, 128, 128), 32.0, None, [3], "fp32"),
    ((24, 24, 24), 6.0, [(0.1, 0.2, 0.3), (0.0, 0.0, 0.0), (-0.3, 0.45, -0.1)], [2, 1, 4], "fp64"),
    ((48, 48, 48), 12.0, None, [5], "fp64"),
]


@pytest.mark.parametrize("n,r,ks,bands,prec", CASES)
def test_batch_fastest_roundtrip_equals_band_major(F, n, r, ks, bands, prec):
    import torch
    kw = dict(radius=r, bands=bands)
    if ks is not None:
        kw["kshift"] = np.array(ks)
    p0 = F.Plan(n, "roundtrip", prec, **kw)
    p1 = F.Plan(n, "roundtrip", prec, layout=1, **kw)
    assert p1.info["sphere_elems"] == p0.info["sphere_elems"] and p1.info["cube_elems"] == p0.info["cube_elems"]
    gs = [p0.sphere(k) for k in range(len(bands))]
    ngws = [len(g) for g in gs]
    cd, td = (np.complex128, torch.complex128) if prec == "fp64" else (np.complex64, torch.complex64)
    parts = [fi.complex_gaussian((b, ng), 300 + k).astype(cd) for k, (ng, b) in enumerate(zip(ngws, bands))]
    x0 = np.concatenate([p.reshape(-1) for p in parts])
    out0, cube0 = execute(F, p0, x0, "roundtrip", td)
    out1, cube1 = execute(F, p1, sph_bf(x0, ngws, bands), "roundtrip", td)
    assert np.array_equal(out1, sph_bf(out0, ngws, bands))
    assert np.array_equal(cube1, cube_bf(cube0, n, bands))
    # and against the oracle: the last band of every k-point, read in place
    vol = n[0] * n[1] * n[2]
    tol = 1e-12 if prec == "fp64" else 2e-6
    b0 = 0
    for k, (g, b) in enumerate(zip(gs, bands)):
        blk = cube1[b0 * vol:(b0 + b) * vol].reshape(n[2], n[1], n[0], b)
        want = oracle.g2r(g, parts[k][b - 1].astype(np.complex128), n)
        assert relerr(blk[..., b - 1], want) <= tol
        b0 += b
    assert relerr(out1, vol * sph_bf(x0, ngws, bands).astype(np.complex128)) <= tol


def test_batch_fastest_one_way_directions_vs_oracle(F):
    """G -> r and r -> G (of a cube that is not band-limited) on a user list in
    its own order (the gather/scatter path of the z stage), and the fused apply."""
    import torch
    n = (32, 32, 48)
    g = oracle.sphere_gvectors(n, 9.0)
    perm = np.random.default_rng(5).permutation(len(g))
    gl = g[perm]
    bands = 5
    c = fi.complex_gaussian((bands, len(gl)), 311).astype(np.complex64)
    p = F.Plan(n, "g2r", "fp32", g_lists=[gl], bands=[bands], layout=1)
    out, _ = execute(F, p, c.T.reshape(-1), "g2r", torch.complex64)
    R = out.reshape(n[2], n[1], n[0], bands)
    want = oracle.g2r(gl, c.astype(np.complex128), n)
    for b in range(bands):
        assert relerr(R[..., b], want[b]) <= 2e-6
    Rin = fi.complex_gaussian((bands, n[2], n[1], n[0]), 312).astype(np.complex64)
    p2 = F.Plan(n, "r2g", "fp32", g_lists=[gl], bands=[bands], layout=1)
    o2, _ = execute(F, p2, np.moveaxis(Rin, 0, -1).reshape(-1), "r2g", torch.complex64)
    want2 = oracle.r2g(gl, Rin.astype(np.complex128), n)
    assert relerr(o2.reshape(len(gl), bands).T, want2) <= 2e-6
    v = fi.gaussian_potential(n, 8, 3.0, seed=313).astype(np.float32)
    pa = F.Plan(n, "apply", "fp32", g_lists=[gl], bands=[bands], layout=1)
    pa.set_potential(torch.from_numpy(v).cuda())
    oa, _ = execute(F, pa, c.T.reshape(-1), "apply", torch.complex64)
    wanta = oracle.apply_potential(gl, c.astype(np.complex128), v.astype(np.float64), n)
    assert relerr(oa.reshape(len(gl), bands).T, wanta) <= 2e-6


def test_batch_fastest_mixed_precision_and_chunks(F):
    """MIXED_TC in the batch-fastest layout runs its plane stages on the
    mma.sync path (the tcgen05 kernels take band-major planes); band chunks
    that split k-points keep every band in place."""
    import torch
    n, r = (64, 64, 64), 16.0
    ks = np.array([(0.1, -0.25, 0.4), (-0.3, 0.2, 0.0)])
    bands = [3, 4]
    p = F.Plan(n, "roundtrip", "mixed", radius=r, kshift=ks, bands=bands, layout=1, max_chunk_bands=2)
    assert p.info["tensor_core_planes"] == 0 and p.info["chunk_bands"] == 2
    gs = [p.sphere(k) for k in range(2)]
    ngws = [len(g) for g in gs]
    parts = [fi.complex_gaussian((b, ng), 320 + k).astype(np.complex64) for k, (ng, b) in enumerate(zip(ngws, bands))]
    x0 = np.concatenate([q.reshape(-1) for q in parts])
    out, cube = execute(F, p, sph_bf(x0, ngws, bands), "roundtrip", torch.complex64)
    vol = 64 ** 3
    assert relerr(out, vol * sph_bf(x0, ngws, bands).astype(np.complex128)) <= 1e-5
    b0 = 0
    for k, (g, b) in enumerate(zip(gs, bands)):
        blk = cube[b0 * vol:(b0 + b) * vol].reshape(64, 64, 64, b)
        want = oracle.g2r(g, parts[k].astype(np.complex128), n)
        for j in range(b):
            assert relerr(blk[..., j], want[j]) <= 1e-5
        b0 += b
    # FP32 with the same chunks equals the unchunked plan bit for bit
    pa = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands, layout=1, max_chunk_bands=2)
    pb = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands, layout=1)
    oa, ca = execute(F, pa, sph_bf(x0, ngws, bands), "roundtrip", torch.complex64)
    ob, cb = execute(F, pb, sph_bf(x0, ngws, bands), "roundtrip", torch.complex64)
    assert np.array_equal(oa, ob) and np.array_equal(ca, cb)


@pytest.mark.parametrize("bands", [[7], [3, 1, 6]])
def test_batch_fastest_host_pipeline(F, bands):
    """The host-buffer entry point splits batch-fastest batches only at a
    k-point boundary (one k-point: one piece); results equal the device call."""
    import torch
    n, r = (32, 32, 32), 7.5
    ks = np.array([(0.1, 0.2, -0.3), (-0.4, 0.0, 0.25), (0.3, -0.45, 0.0)])[:len(bands)]
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands, layout=1)
    info = plan.info
    xin = fi.complex_gaussian((info["sphere_elems"],), 330).astype(np.complex64)
    want, wcube = execute(F, plan, xin, "roundtrip", torch.complex64)
    pin_in = torch.from_numpy(xin).pin_memory()
    pin_out = torch.empty(info["sphere_elems"], dtype=torch.complex64).pin_memory()
    cube2 = torch.empty(info["cube_elems"], dtype=torch.complex64, device="cuda")
    before = plan.launches()
    s = torch.cuda.Stream()
    F.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cube2.data_ptr(), s.cuda_stream)
    pieces = 1 if len(bands) == 1 else 2
    chunks = int(np.ceil(sum(bands) / info["chunk_bands"]))
    assert plan.launches() - before >= pieces * 4 and plan.launches() - before <= (chunks + pieces) * 4
    assert np.array_equal(pin_out.numpy(), want)
    assert np.array_equal(cube2.cpu().numpy(), wcube)


@pytest.mark.parametrize("n,r,ks,bands,group", [((64, 64, 64), 16.0, None, [7], 4),
                                                ((32, 32, 32), 8.0, [(0.3, -0.2, 0.1), (-0.45, 0.4, -0.3)], [3, 5], 4),
                                                ((48, 48, 48), 12.0, None, [6], 4),
                                                ((96, 96, 96), 24.0, None, [5], 4),
                                                ((128, 128, 128), 32.0, None, [3], 2),
                                                ((160, 160, 160), 40.0, None, [2], 0)])
def test_band_groups_same_results(F, n, r, ks, bands, group):
    """The grouped plane kernels (several bands of one k-point per CTA, cube
    rows band-contiguous) give the per-band kernels' results bit for bit,
    including partial groups at k-point ends and a chunk smaller than a group."""
    import torch
    kw = dict(radius=r, bands=bands)
    if ks is not None:
        kw["kshift"] = np.array(ks)
    p = F.Plan(n, "roundtrip", "fp32", layout=1, **kw)
    assert p.info["plane_band_group"] == group
    gs = [p.sphere(k) for k in range(len(bands))]
    ngws = [len(g) for g in gs]
    x = sph_bf(np.concatenate([fi.complex_gaussian((b, ng), 340 + k).astype(np.complex64).reshape(-1)
                               for k, (ng, b) in enumerate(zip(ngws, bands))]), ngws, bands)
    o1, c1 = execute(F, p, x, "roundtrip", torch.complex64)
    if group == 0:
        with pytest.raises(F.FFTBError) as ei:
            p.set_band_groups(True)
        assert ei.value.status == F.FFTB_ERR_UNSUPPORTED
        return
    p.set_band_groups(False)
    assert p.info["plane_band_group"] == 0
    o0, c0 = execute(F, p, x, "roundtrip", torch.complex64)
    assert np.array_equal(o0, o1) and np.array_equal(c0, c1)
    small = F.Plan(n, "roundtrip", "fp32", layout=1, max_chunk_bands=1, **kw)
    assert small.info["plane_band_group"] == group
    o2, c2 = execute(F, small, x, "roundtrip", torch.complex64)
    assert np.array_equal(o2, o1) and np.array_equal(c2, c1)
    vol = n[0] * n[1] * n[2]
    assert relerr(o1, vol * x.astype(np.complex128)) <= 2e-6


def test_batch_fastest_autotune(F, tmp_path, monkeypatch):
    """The autotuner may choose grouped or per-band plane stages (and every
    other schedule) for a batch-fastest plan; results stay at the FP32 bound,
    and a band prefix of a large batch stays inside its k-point's cube block."""
    import torch
    monkeypatch.setenv("FFTB_TUNE_CACHE", str(tmp_path / "tune.txt"))
    n, r = (64, 64, 64), 16.0
    bands = [9, 4]
    ks = np.array([(0.2, 0.1, -0.3), (-0.1, 0.4, 0.25)])
    p = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands, layout=1)
    p.autotune(2)
    line = (tmp_path / "tune.txt").read_text().strip().split()
    assert len(line) == 14  # key, chunk, 3 plane CTAs, z CTAs, level, buffers, 2 schedules, pdl, group, tc, cl
    assert int(line[-3]) == p.info["plane_band_group"] and line[-3] in ("0", "4") and line[-2:] == ["0", "0"]
    gs = [p.sphere(k) for k in range(2)]
    ngws = [len(g) for g in gs]
    parts = [fi.complex_gaussian((b, ng), 350 + k).astype(np.complex64) for k, (ng, b) in enumerate(zip(ngws, bands))]
    x = sph_bf(np.concatenate([q.reshape(-1) for q in parts]), ngws, bands)
    out, cube = execute(F, p, x, "roundtrip", torch.complex64)
    vol = 64 ** 3
    assert relerr(out, vol * x.astype(np.complex128)) <= 2e-6
    blk = cube[9 * vol:13 * vol].reshape(64, 64, 64, 4)
    assert relerr(blk[..., 3], oracle.g2r(gs[1], parts[1][3].astype(np.complex128), n)) <= 2e-6
