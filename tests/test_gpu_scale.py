"""Optional output normalisation (the transforms themselves are unscaled,
Sec. 2.1-2.2): the cube of G->r outputs times g2r, r->G outputs times r2g,
the sphere output of a round trip or an apply times both."""
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


def run(plan, x, direction, dtype):
    import torch
    info = plan.info
    nout = info["cube_elems"] if direction == "g2r" else info["sphere_elems"]
    out = torch.empty(nout, dtype=dtype, device="cuda")
    cube = torch.empty(info["cube_elems"], dtype=dtype, device="cuda") if direction == "roundtrip" else None
    plan.execute(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out, cube)
    torch.cuda.synchronize()
    return out.cpu().numpy(), (cube.cpu().numpy() if cube is not None else None)


@pytest.mark.parametrize("prec,layout", [("fp32", 0), ("fp64", 0), ("fp32", 1)])
def test_round_trip_normalised_to_identity(F, prec, layout):
    import torch
    n, r, bands = (32, 32, 32), 8.0, 5
    vol = 32 ** 3
    plan = F.Plan(n, "roundtrip", prec, radius=r, bands=[bands], layout=layout)
    cd, td = (np.complex128, torch.complex128) if prec == "fp64" else (np.complex64, torch.complex64)
    g = plan.sphere(0)
    c = fi.complex_gaussian((bands, len(g)), 501).astype(cd)
    x = (c.T if layout else c).reshape(-1)
    out0, cube0 = run(plan, x, "roundtrip", td)
    plan.set_scale(1.0, 1.0 / vol)
    assert plan.info["scale_r2g"] == 1.0 / vol and plan.info["kernels_per_execute"] == 5
    out1, cube1 = run(plan, x, "roundtrip", td)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert relerr(out1, x.astype(np.complex128)) <= tol
    assert np.array_equal(cube1, cube0)  # the cube is a G->r output: g2r = 1 leaves it as it was
    plan.set_scale(0.25, 2.0)            # powers of two: exact
    out2, cube2 = run(plan, x, "roundtrip", td)
    assert np.array_equal(cube2, 0.25 * cube0)
    assert np.array_equal(out2, 0.5 * out0)


def test_one_way_and_apply_scaled(F):
    import torch
    n, r, bands = (24, 24, 24), 6.0, 3
    g = oracle.sphere_gvectors(n, r)
    c = fi.complex_gaussian((bands, len(g)), 502).astype(np.complex64)
    p = F.Plan(n, "g2r", "fp32", radius=r, bands=[bands])
    p.set_scale(3.0, 5.0)                # r2g does not apply to G -> r
    assert p.info["kernels_per_execute"] == 3
    out, _ = run(p, c.reshape(-1), "g2r", torch.complex64)
    assert relerr(out, 3.0 * oracle.g2r(g, c.astype(np.complex128), n)) <= 2e-6
    R = fi.complex_gaussian((bands, 24, 24, 24), 503).astype(np.complex64)
    p2 = F.Plan(n, "r2g", "fp32", radius=r, bands=[bands])
    p2.set_scale(7.0, 1.0 / 24 ** 3)     # g2r does not apply to r -> G
    o2, _ = run(p2, R.reshape(-1), "r2g", torch.complex64)
    assert relerr(o2, oracle.r2g(g, R.astype(np.complex128), n).reshape(-1) / 24 ** 3) <= 2e-6
    v = fi.gaussian_potential(n, 8, 3.0, seed=504).astype(np.float32)
    pa = F.Plan(n, "apply", "fp32", radius=r, bands=[bands])
    pa.set_potential(torch.from_numpy(v).cuda())
    pa.set_scale(3.0, 0.5)
    oa, _ = run(pa, c.reshape(-1), "apply", torch.complex64)
    want = oracle.apply_potential(g, c.astype(np.complex128), v.astype(np.float64), n)
    assert relerr(oa, 1.5 * want.reshape(-1)) <= 2e-6
    with pytest.raises(F.FFTBError) as ei:
        pa.set_scale(float("nan"), 1.0)
    assert ei.value.status == F.FFTB_ERR_INVALID_ARG


def test_scaled_host_pipeline_and_graph(F):
    """The scaling is part of every path: the host-buffer pipeline (per piece)
    and graph replay give the device call's result."""
    import torch
    n, r = (32, 32, 32), 7.5
    ks = np.array([(0.1, 0.2, -0.3), (-0.4, 0.0, 0.25), (0.3, -0.45, 0.0)])
    bands = [3, 1, 6]
    plan = F.Plan(n, "roundtrip", "fp32", radius=r, kshift=ks, bands=bands, max_chunk_bands=2)
    plan.set_scale(0.5, 1.0 / 32 ** 3)
    info = plan.info
    xin = fi.complex_gaussian((info["sphere_elems"],), 505).astype(np.complex64)
    want, wcube = run(plan, xin, "roundtrip", torch.complex64)
    assert relerr(want, 0.5 * xin.astype(np.complex128)) <= 2e-6
    pin_in = torch.from_numpy(xin).pin_memory()
    pin_out = torch.empty(info["sphere_elems"], dtype=torch.complex64).pin_memory()
    cube2 = torch.empty(info["cube_elems"], dtype=torch.complex64, device="cuda")
    s = torch.cuda.Stream()
    F.fftb_execute_host(plan.handle, pin_in.data_ptr(), pin_out.data_ptr(), cube2.data_ptr(), s.cuda_stream)
    assert np.array_equal(pin_out.numpy(), want)
    assert np.array_equal(cube2.cpu().numpy(), wcube)
    plan.set_graph(True)
    for _ in range(2):
        got, gcube = run(plan, xin, "roundtrip", torch.complex64)
        assert np.array_equal(got, want) and np.array_equal(gcube, wcube)
