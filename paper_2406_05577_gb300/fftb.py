"""ctypes binding of libfftb.so (the C ABI in include/fftb.h).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels. The functions keep the C names; ``Plan`` wraps a plan handle
and accepts torch tensors (device memory and streams come from PyTorch).
The library must be built (``paper_2406_05577_gb300.build.build()``); if it
is missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FFTB_LIBRARY selects another in-tree build of the library, e.g. the checked
# one (build.build(check=True) -> libfftb_check.so)
LIB_PATH = os.environ.get("FFTB_LIBRARY") or os.path.join(HERE, "libfftb.so")

FFTB_OK, FFTB_ERR_INVALID_ARG, FFTB_ERR_UNSUPPORTED, FFTB_ERR_ALLOC, FFTB_ERR_CUDA, \
    FFTB_ERR_DEVICE_TIMEOUT, FFTB_ERR_DEVICE_BOUNDS = range(7)
FFTB_G_TO_R, FFTB_R_TO_G, FFTB_ROUNDTRIP, FFTB_APPLY_LOCAL = 1, -1, 0, 2
FFTB_FP64, FFTB_FP32, FFTB_MIXED_TC = 0, 1, 2
FFTB_INJECT_SKIP_FIRST_PREFETCH = 1

DIRECTIONS = {"g2r": FFTB_G_TO_R, "r2g": FFTB_R_TO_G, "roundtrip": FFTB_ROUNDTRIP,
              "apply": FFTB_APPLY_LOCAL}
PRECISIONS = {"fp64": FFTB_FP64, "fp32": FFTB_FP32, "mixed": FFTB_MIXED_TC}


class fftb_desc(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("n_kpoints", ctypes.c_int32),
        ("bands", ctypes.POINTER(ctypes.c_int32)),
        ("radius", ctypes.c_double),
        ("kshift", ctypes.POINTER(ctypes.c_double)),
        ("g_list", ctypes.POINTER(ctypes.c_int32)),
        ("g_count", ctypes.POINTER(ctypes.c_int64)),
        ("layout", ctypes.c_int32),
        ("max_chunk_bands", ctypes.c_int32),
    ]


class fftb_plan_info_t(ctypes.Structure):
    _fields_ = [
        ("sphere_elems", ctypes.c_int64),
        ("cube_elems", ctypes.c_int64),
        ("scratch_bytes", ctypes.c_int64),
        ("total_bands", ctypes.c_int32),
        ("max_sticks", ctypes.c_int32),
        ("max_slabs", ctypes.c_int32),
        ("chunk_bands", ctypes.c_int32),
        ("kernels_per_execute", ctypes.c_int32),
        ("complex_bytes", ctypes.c_int32),
        ("stick_ctas", ctypes.c_int32),
        ("plane_ctas", ctypes.c_int32),
        ("prefetch", ctypes.c_int32),
        ("slab_buffers", ctypes.c_int32),
        ("tensor_core_planes", ctypes.c_int32),
        ("slab_planes_global", ctypes.c_int32),
        ("radix_schedule_plane", ctypes.c_int32),
        ("radix_schedule_stick", ctypes.c_int32),
        ("dependent_launch", ctypes.c_int32),
        ("plane_band_group", ctypes.c_int32),
        ("graph_launches", ctypes.c_int64),
        ("scale_g2r", ctypes.c_double),
        ("scale_r2g", ctypes.c_double),
        ("generic_path", ctypes.c_int32),
        ("tensor_core_passes", ctypes.c_int32),
        ("tensor_cores_available", ctypes.c_int32),
        ("plane_clusters", ctypes.c_int32),
        ("pruned_lines", ctypes.c_int32),
    ]


EXPORTS = {
    "fftb_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(fftb_desc),
                                        ctypes.c_int, ctypes.c_int]),
    "fftb_plan_ngw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "fftb_plan_sphere": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "fftb_plan_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fftb_plan_info_t)]),
    "fftb_set_potential": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fftb_execute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "fftb_execute_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "fftb_plan_launches": (ctypes.c_int64, [ctypes.c_void_p]),
    "fftb_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "fftb_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "fftb_last_error": (ctypes.c_char_p, []),
    "fftb_version": (ctypes.c_char_p, []),
    "fftb_plan_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fftb_g2r_noalloc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fftb_plan_set_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_prefetch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_check": (ctypes.c_int, [ctypes.c_void_p]),
    "fftb_plan_set_slab_buffers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_radix_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "fftb_plan_set_pdl": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_band_groups": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_tensor_cores": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_plane_clusters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_plan_set_scale": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    "fftb_plan_inject": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fftb_sphere_enumerate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_int64)]),
    "fftb_sphere_sticks": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "fftb_box_enumerate": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_int64]),
    "fftb_glist_from_offsets": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int64, ctypes.c_void_p]),
}

_lib = None


def lib():
    """Loads libfftb.so once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2406_05577_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class FFTBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(status):
    if status != FFTB_OK:
        L = lib()
        detail = L.fftb_last_error().decode()
        raise FFTBError(status, f"{L.fftb_error_string(status).decode()}: {detail}")


# ------------------------------------------------------------ C-named calls

def fftb_plan_create(n, direction, precision, radius=0.0, kshift=None, bands=None,
                     g_lists=None, max_chunk_bands=0, layout=0):
    """Returns a plan handle (int). n = (N0, N1, N2); kshift (nk, 3);
    bands (nk,); g_lists: list of (ngw_k, 3) int arrays (explicit spheres)."""
    L = lib()
    if isinstance(direction, str):
        direction = DIRECTIONS[direction]
    if isinstance(precision, str):
        precision = PRECISIONS[precision]
    nk = 1
    if g_lists is not None:
        nk = len(g_lists)
    elif kshift is not None:
        nk = int(np.asarray(kshift).reshape(-1, 3).shape[0])
    elif bands is not None:
        nk = len(bands)
    d = fftb_desc()
    d.n[0], d.n[1], d.n[2] = (int(v) for v in n)
    d.n_kpoints = nk
    d.radius = float(radius)
    d.layout = int(layout)
    d.max_chunk_bands = int(max_chunk_bands)
    keep = []
    if bands is not None:
        b = np.ascontiguousarray(np.asarray(bands, dtype=np.int32).reshape(-1))
        keep.append(b)
        d.bands = b.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if kshift is not None:
        k = np.ascontiguousarray(np.asarray(kshift, dtype=np.float64).reshape(-1))
        keep.append(k)
        d.kshift = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if g_lists is not None:
        parts = [np.asarray(g, dtype=np.int32).reshape(-1, 3) for g in g_lists]
        gl = np.ascontiguousarray(np.concatenate(parts, axis=0) if parts else np.zeros((0, 3), np.int32))
        gc = np.ascontiguousarray(np.array([len(p) for p in parts], dtype=np.int64))
        if gl.size == 0:
            gl = np.zeros(3, np.int32)  # non-NULL pointer for empty spheres
        keep += [gl, gc]
        d.g_list = gl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.g_count = gc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    h = ctypes.c_void_p()
    _check(L.fftb_plan_create(ctypes.byref(h), ctypes.byref(d), int(direction), int(precision)))
    return h.value


def fftb_plan_ngw(plan, kpoint):
    v = ctypes.c_int64()
    _check(lib().fftb_plan_ngw(plan, int(kpoint), ctypes.byref(v)))
    return v.value


def fftb_plan_sphere(plan, kpoint):
    ngw = fftb_plan_ngw(plan, kpoint)
    out = np.zeros((max(ngw, 1), 3), dtype=np.int32)
    _check(lib().fftb_plan_sphere(plan, int(kpoint), out.ctypes.data))
    return out[:ngw]


def fftb_plan_get_info(plan):
    info = fftb_plan_info_t()
    _check(lib().fftb_plan_get_info(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in fftb_plan_info_t._fields_}


def fftb_set_potential(plan, v_ptr):
    _check(lib().fftb_set_potential(plan, v_ptr))


def fftb_execute(plan, in_ptr, out_ptr, cube_ptr=None, stream=None):
    _check(lib().fftb_execute(plan, in_ptr, out_ptr, cube_ptr, stream))


def fftb_execute_host(plan, in_host_ptr, out_host_ptr, cube_ptr=None, stream=None):
    _check(lib().fftb_execute_host(plan, in_host_ptr, out_host_ptr, cube_ptr, stream))


STAGE_KINDS = ("stick_g2r", "plane_g2r", "plane_r2g", "stick_r2g", "plane_apply")


def fftb_plan_set_timing(plan, enable):
    _check(lib().fftb_plan_set_timing(plan, 1 if enable else 0))


def fftb_plan_stage_times(plan):
    """{kind: (ms, launches)} since the previous query (waits for the events)."""
    ms = np.zeros(len(STAGE_KINDS), np.float64)
    cnt = np.zeros(len(STAGE_KINDS), np.int64)
    _check(lib().fftb_plan_stage_times(plan, ms.ctypes.data, cnt.ctypes.data))
    return {k: (float(m), int(c)) for k, m, c in zip(STAGE_KINDS, ms, cnt)}


def fftb_plan_set_graph(plan, enable):
    _check(lib().fftb_plan_set_graph(plan, 1 if enable else 0))


def fftb_plan_autotune(plan, trials=3):
    _check(lib().fftb_plan_autotune(plan, int(trials)))


def fftb_plan_set_prefetch(plan, level):
    """level 0 off, 1 where no resident CTA is lost (default), 2 wherever it fits."""
    _check(lib().fftb_plan_set_prefetch(plan, int(level)))


def fftb_plan_set_slab_buffers(plan, nbuf):
    _check(lib().fftb_plan_set_slab_buffers(plan, int(nbuf)))


def fftb_plan_set_radix_schedule(plan, plane, stick):
    _check(lib().fftb_plan_set_radix_schedule(plan, int(plane), int(stick)))


def fftb_plan_set_pdl(plan, enable):
    _check(lib().fftb_plan_set_pdl(plan, 1 if enable else 0))


def fftb_plan_set_scale(plan, g2r=1.0, r2g=1.0):
    _check(lib().fftb_plan_set_scale(plan, float(g2r), float(r2g)))


def fftb_plan_set_band_groups(plan, enable):
    _check(lib().fftb_plan_set_band_groups(plan, 1 if enable else 0))


def fftb_plan_set_tensor_cores(plan, enable):
    _check(lib().fftb_plan_set_tensor_cores(plan, 1 if enable else 0))


def fftb_plan_set_plane_clusters(plan, enable):
    _check(lib().fftb_plan_set_plane_clusters(plan, 1 if enable else 0))


def fftb_plan_check(plan):
    """Raises FFTBError (status FFTB_ERR_DEVICE_TIMEOUT) if a device wait ran out."""
    _check(lib().fftb_plan_check(plan))


def fftb_plan_inject(plan, flags):
    _check(lib().fftb_plan_inject(plan, int(flags)))


def fftb_plan_launches(plan):
    return int(lib().fftb_plan_launches(plan))


def fftb_destroy(plan):
    if plan:
        _check(lib().fftb_destroy(plan))


def fftb_sphere_enumerate(n, radius, kshift=None):
    """Cutoff sphere in canonical order, (ngw, 3) int32 (host only)."""
    L = lib()
    nn = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    k = None if kshift is None else np.ascontiguousarray(np.asarray(kshift, np.float64).reshape(3))
    kp = None if k is None else k.ctypes.data
    cnt = ctypes.c_int64()
    _check(L.fftb_sphere_enumerate(nn, float(radius), kp, None, 0, ctypes.byref(cnt)))
    out = np.zeros((max(cnt.value, 1), 3), np.int32)
    _check(L.fftb_sphere_enumerate(nn, float(radius), kp, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
    return out[:cnt.value]


def fftb_sphere_sticks(n, g):
    """(n_sticks, n_slabs) of an explicit sphere (host only)."""
    L = lib()
    nn = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    gg = np.ascontiguousarray(np.asarray(g, np.int32).reshape(-1, 3))
    s, x = ctypes.c_int32(), ctypes.c_int32()
    _check(L.fftb_sphere_sticks(nn, gg.ctypes.data if gg.size else None, len(gg),
                                ctypes.byref(s), ctypes.byref(x)))
    return s.value, x.value


def fftb_box_enumerate(n):
    """Every G of the grid's frequency box in canonical order, (N0 N1 N2, 3)
    int32 (host only): the g_list of the unpruned full-cube transform."""
    nn = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    vol = int(n[0]) * int(n[1]) * int(n[2])
    out = np.zeros((vol, 3), np.int32)
    _check(lib().fftb_box_enumerate(nn, out.ctypes.data, vol))
    return out


def fftb_glist_from_offsets(n, lo, hi, offsets, z_index):
    """(nnz, 3) int32 G list of an offset array over the bounding domain
    [lo, hi] (inclusive corners; x-fastest columns, per-entry z), host only."""
    nn = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    l3 = (ctypes.c_int32 * 3)(*[int(v) for v in lo])
    h3 = (ctypes.c_int32 * 3)(*[int(v) for v in hi])
    off = np.ascontiguousarray(np.asarray(offsets, np.int64).reshape(-1))
    zi = np.ascontiguousarray(np.asarray(z_index, np.int32).reshape(-1))
    out = np.zeros((max(len(zi), 1), 3), np.int32)
    _check(lib().fftb_glist_from_offsets(nn, l3, h3, off.ctypes.data, zi.ctypes.data if zi.size else None,
                                         len(zi), out.ctypes.data))
    return out[:len(zi)]


def fftb_g2r_noalloc(n, radius, kshift, bands, in_ptr, out_ptr, stream=None):
    """Allocation-free G -> r (FP32, one cutoff sphere); see include/fftb.h."""
    nn = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    k = None if kshift is None else np.ascontiguousarray(np.asarray(kshift, np.float64).reshape(3))
    _check(lib().fftb_g2r_noalloc(nn, float(radius), None if k is None else k.ctypes.data, int(bands),
                                  in_ptr, out_ptr, stream))


def fftb_version():
    return lib().fftb_version().decode()


# -------------------------------------------------------- torch convenience

class Plan:
    """Owns one plan handle; execute() takes torch tensors on the plan's GPU."""

    def __init__(self, n, direction, precision, **kw):
        self.n = tuple(int(v) for v in n)
        self.direction = DIRECTIONS[direction] if isinstance(direction, str) else direction
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        self.handle = fftb_plan_create(self.n, self.direction, self.precision, **kw)
        self.info = fftb_plan_get_info(self.handle)
        self.nk = kw.get("g_lists") and len(kw["g_lists"]) or (
            np.asarray(kw["kshift"]).reshape(-1, 3).shape[0] if kw.get("kshift") is not None
            else (len(kw["bands"]) if kw.get("bands") is not None else 1))
        self._v = None

    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == FFTB_FP64 else torch.complex64

    @property
    def real_dtype(self):
        import torch
        return torch.float64 if self.precision == FFTB_FP64 else torch.float32

    def ngw(self, k=0):
        return fftb_plan_ngw(self.handle, k)

    def sphere(self, k=0):
        return fftb_plan_sphere(self.handle, k)

    def _ptr(self, t, dtype, numel, what):
        if t is None:
            return None
        if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{what}: need a contiguous CUDA tensor of {dtype}")
        if t.numel() < numel:
            raise ValueError(f"{what}: need at least {numel} elements, got {t.numel()}")
        return t.data_ptr()

    def set_potential(self, v):
        n0, n1, n2 = self.n
        fftb_set_potential(self.handle, self._ptr(v, self.real_dtype, n0 * n1 * n2, "potential"))
        self._v = v  # keep it alive while the plan may use it

    def execute(self, x, out, cube=None, stream=None):
        import torch
        sph, cub = self.info["sphere_elems"], self.info["cube_elems"]
        nin, nout = sph, sph
        if self.direction == FFTB_G_TO_R:
            nout = cub
        elif self.direction == FFTB_R_TO_G:
            nin = cub
        cd = self.complex_dtype
        s = stream if stream is not None else torch.cuda.current_stream()
        fftb_execute(self.handle, self._ptr(x, cd, nin, "in"), self._ptr(out, cd, nout, "out"),
                     self._ptr(cube, cd, cub, "cube"), s.cuda_stream)

    def execute_host(self, x, out, cube=None, stream=None):
        """fftb_execute_host: x and out are contiguous CPU tensors of the
        plan's complex type (page-locked for full-speed, overlapped copies);
        cube (ROUNDTRIP only, optional) is a CUDA tensor. Returns when done."""
        import torch
        sph, cub = self.info["sphere_elems"], self.info["cube_elems"]
        nin = cub if self.direction == FFTB_R_TO_G else sph
        nout = cub if self.direction == FFTB_G_TO_R else sph
        cd = self.complex_dtype
        for t, n, what in ((x, nin, "in"), (out, nout, "out")):
            if t.is_cuda or t.dtype != cd or not t.is_contiguous():
                raise ValueError(f"{what}: need a contiguous CPU tensor of {cd}")
            if t.numel() < n:
                raise ValueError(f"{what}: need at least {n} elements, got {t.numel()}")
        s = stream if stream is not None else torch.cuda.current_stream()
        fftb_execute_host(self.handle, x.data_ptr(), out.data_ptr(), self._ptr(cube, cd, cub, "cube"),
                          s.cuda_stream)

    def launches(self):
        return fftb_plan_launches(self.handle)

    def set_graph(self, enable=True):
        fftb_plan_set_graph(self.handle, enable)

    def autotune(self, trials=3):
        fftb_plan_autotune(self.handle, trials)
        self.info = fftb_plan_get_info(self.handle)

    def set_prefetch(self, level=1):
        fftb_plan_set_prefetch(self.handle, int(level))
        self.info = fftb_plan_get_info(self.handle)

    def set_slab_buffers(self, nbuf):
        fftb_plan_set_slab_buffers(self.handle, nbuf)
        self.info = fftb_plan_get_info(self.handle)

    def set_radix_schedule(self, plane=0, stick=0):
        fftb_plan_set_radix_schedule(self.handle, plane, stick)
        self.info = fftb_plan_get_info(self.handle)

    def set_pdl(self, enable=True):
        fftb_plan_set_pdl(self.handle, enable)
        self.info = fftb_plan_get_info(self.handle)

    def set_scale(self, g2r=1.0, r2g=1.0):
        fftb_plan_set_scale(self.handle, g2r, r2g)
        self.info = fftb_plan_get_info(self.handle)

    def set_band_groups(self, enable=True):
        fftb_plan_set_band_groups(self.handle, enable)
        self.info = fftb_plan_get_info(self.handle)

    def set_tensor_cores(self, enable=True):
        fftb_plan_set_tensor_cores(self.handle, enable)
        self.info = fftb_plan_get_info(self.handle)

    def set_plane_clusters(self, enable=True):
        fftb_plan_set_plane_clusters(self.handle, enable)
        self.info = fftb_plan_get_info(self.handle)

    def check(self):
        fftb_plan_check(self.handle)

    def inject(self, flags):
        fftb_plan_inject(self.handle, flags)

    def close(self):
        if self.handle:
            fftb_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
