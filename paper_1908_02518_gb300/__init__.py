"""GB300-native Vietoris–Rips persistence barcodes (Ripser's method, arXiv 1908.02518).

Thin Python binding over the C ABI of ``librips.so`` (include/rips.h).  Every
step of the computation runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory and streams.

    res = barcodes(dist, dim_max=2, threshold=1.0, p=2)   # dist: torch.cuda or numpy
    res.bars            # structured numpy array (dim, birth, death, cloud, birth_simplex, death_simplex)
    res.dim(1)          # bars of H1
    res.stats           # per-dimension counters (Table 2 categories)
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field

import numpy as np

from . import _lib
from ._lib import RipsError

__all__ = ["barcodes", "barcodes_packed", "barcodes_sparse", "barcodes_sparse_points", "barcodes_batched", "barcodes_batched_dists", "distance_matrix", "backward",
           "backward_dist", "Result", "RipsError",
           "RipsBarcodes", "launch_count", "set_kernel_timing", "BAR_DTYPE"]

BAR_DTYPE = np.dtype({
    "names": ["dim", "birth", "death", "cloud", "birth_simplex", "death_simplex"],
    "formats": [np.int32, np.float32, np.float32, np.int32, np.uint64, np.uint64],
    "offsets": [0, 4, 8, 12, 16, 24], "itemsize": 32})


@dataclass
class Result:
    """Bars and statistics of one call (copied out of the library's result)."""
    bars: np.ndarray
    thresholds: list
    stats: list                 # stats[cloud][dim] -> dict
    phase_ms: list
    kernel_ms: dict             # kernel class -> (ms, timed regions), when timing is on
    dim_max: int
    clouds: int
    _handle: object = field(default=None, repr=False)

    def dim(self, d: int, cloud: int | None = None) -> np.ndarray:
        m = self.bars["dim"] == d
        if cloud is not None:
            m &= self.bars["cloud"] == cloud
        return self.bars[m]

    @property
    def threshold(self) -> float:
        return self.thresholds[0]

    def free(self):
        if self._handle is not None and self._handle.value:
            _lib.load().rips_result_free(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _collect(lib, handle, keep_handle: bool) -> Result:
    nb = lib.rips_result_num_bars(handle, -1, -1)
    arr = np.zeros(max(nb, 0), dtype=BAR_DTYPE)
    if nb > 0:
        ptr = lib.rips_result_bars(handle, -1, -1)
        C.memmove(arr.ctypes.data, ptr, nb * 32)
    clouds = lib.rips_result_num_clouds(handle)
    dim_max = lib.rips_result_dim_max(handle)
    stats = []
    for c in range(clouds):
        row = []
        for d in range(dim_max + 1):
            s = _lib.Stats()
            lib.rips_result_stats(handle, c, d, C.byref(s))
            row.append({f: int(getattr(s, f)) for f, _ in _lib.Stats._fields_})
        stats.append(row)
    ph = (C.c_float * 16)()
    k = lib.rips_result_phase_ms(handle, ph, 16)
    kms = {}
    for q, name in enumerate(_lib.KERNEL_CLASSES):
        ms = C.c_float()
        reg = C.c_int64()
        lib.rips_result_kernel_ms(handle, q, C.byref(ms), C.byref(reg))
        kms[name] = (float(ms.value), int(reg.value))
    res = Result(arr, [float(lib.rips_result_threshold(handle, c)) for c in range(clouds)], stats,
                 [float(ph[i]) for i in range(max(k, 0))], kms, dim_max, clouds)
    if keep_handle:
        res._handle = handle
    else:
        lib.rips_result_free(handle)
    return res


def barcodes(dist, dim_max: int = 1, threshold: float = math.inf, p: int = 2, stream=None,
             keep_handle: bool = False) -> Result:
    """Barcodes H0..H_dim_max of the Rips filtration of a distance matrix.

    ``dist``: n x n FP32, either a CUDA tensor (device path,
    ``rips_barcodes_device``) or a host array (``rips_barcodes``: the copy to the
    device is part of the call).  Only the strict lower triangle is read.
    """
    lib = _lib.load()
    out = C.c_void_p()
    if hasattr(dist, "is_cuda") and dist.is_cuda:
        import torch
        d = dist.contiguous()
        if d.dtype != torch.float32 or d.dim() != 2 or d.shape[0] != d.shape[1]:
            raise ValueError("dist must be an n x n float32 tensor")
        st = lib.rips_barcodes_device(C.c_void_p(d.data_ptr()), d.shape[0], dim_max, C.c_float(threshold), p,
                                      _stream_ptr(stream), C.byref(out))
    else:
        d = np.ascontiguousarray(np.asarray(dist, dtype=np.float32))
        if d.ndim != 2 or d.shape[0] != d.shape[1]:
            raise ValueError("dist must be n x n")
        st = lib.rips_barcodes(d.ctypes.data_as(C.POINTER(C.c_float)), d.shape[0], dim_max, C.c_float(threshold),
                               p, C.byref(out))
    _lib.check(st, "rips_barcodes")
    return _collect(lib, out, keep_handle)


def barcodes_packed(packed, n: int, layout: str = "lower", dim_max: int = 1, threshold: float = math.inf,
                    p: int = 2, stream=None, keep_handle: bool = False) -> Result:
    """Barcodes of a distance matrix given as its strict lower or upper
    triangle packed row by row (n(n-1)/2 FP32 entries, a CUDA tensor or a host
    array, which is copied to the device)."""
    import torch
    lib = _lib.load()
    t = packed if hasattr(packed, "is_cuda") else torch.from_numpy(np.ascontiguousarray(packed, dtype=np.float32))
    t = t.contiguous().float().cuda()
    if t.numel() != n * (n - 1) // 2:
        raise ValueError("packed triangle must hold n(n-1)/2 entries")
    code = {"lower": 0, "upper": 1}[layout]
    out = C.c_void_p()
    st = lib.rips_barcodes_packed(C.c_void_p(t.data_ptr() if t.numel() else 0), n, code, dim_max,
                                  C.c_float(threshold), p, _stream_ptr(stream), C.byref(out))
    _lib.check(st, "rips_barcodes_packed")
    return _collect(lib, out, keep_handle)


def barcodes_sparse(i, j, length, n: int, dim_max: int = 1, threshold: float = math.inf, p: int = 2, stream=None,
                    keep_handle: bool = False) -> Result:
    """Barcodes of a sparse distance matrix given as (i, j, length) entries
    (each unordered pair once; missing pairs are infinitely far), with no n x n
    array anywhere.  Host arrays are copied to the device."""
    import torch
    lib = _lib.load()
    ti = torch.as_tensor(np.asarray(i, dtype=np.int32) if not hasattr(i, "is_cuda") else i).to(torch.int32).cuda()
    tj = torch.as_tensor(np.asarray(j, dtype=np.int32) if not hasattr(j, "is_cuda") else j).to(torch.int32).cuda()
    tl = torch.as_tensor(np.asarray(length, dtype=np.float32) if not hasattr(length, "is_cuda") else length)
    tl = tl.to(torch.float32).cuda()
    m = ti.numel()
    if tj.numel() != m or tl.numel() != m:
        raise ValueError("i, j and length must have the same length")
    out = C.c_void_p()
    st = lib.rips_barcodes_sparse(C.c_void_p(ti.data_ptr() if m else 0), C.c_void_p(tj.data_ptr() if m else 0),
                                  C.c_void_p(tl.data_ptr() if m else 0), m, n, dim_max, C.c_float(threshold), p,
                                  _stream_ptr(stream), C.byref(out))
    _lib.check(st, "rips_barcodes_sparse")
    return _collect(lib, out, keep_handle)


def barcodes_sparse_points(points, threshold: float, dim_max: int = 1, p: int = 2, stream=None,
                           keep_handle: bool = False) -> Result:
    """Barcodes of a point cloud ((n, k) FP32 CUDA tensor) at a finite
    threshold, keeping only the pairs within it (no n x n array)."""
    import torch
    lib = _lib.load()
    x = points.contiguous()
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise ValueError("points must be an (n, k) float32 CUDA tensor")
    out = C.c_void_p()
    st = lib.rips_barcodes_sparse_points(C.c_void_p(x.data_ptr()), x.shape[0], x.shape[1], dim_max,
                                         C.c_float(threshold), p, _stream_ptr(stream), C.byref(out))
    _lib.check(st, "rips_barcodes_sparse_points")
    return _collect(lib, out, keep_handle)


def distance_matrix(points, stream=None):
    """n x n FP32 distances of an (n, k) FP32 CUDA tensor of points."""
    import torch
    lib = _lib.load()
    x = points.contiguous()
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise ValueError("points must be an (n, k) float32 CUDA tensor")
    n, k = x.shape
    d = torch.empty((n, n), dtype=torch.float32, device=x.device)
    _lib.check(lib.rips_distance_matrix_device(C.c_void_p(x.data_ptr()), n, k, C.c_void_p(d.data_ptr()),
                                               _stream_ptr(stream)), "rips_distance_matrix_device")
    return d


def barcodes_batched(points, offsets, dim_max: int = 1, threshold: float = math.inf, p: int = 2, stream=None,
                     keep_handle: bool = False) -> Result:
    """Barcodes of many clouds: ``points`` (N, k) FP32 CUDA tensor of all clouds
    back to back, ``offsets`` (batch + 1) point offsets."""
    import torch
    lib = _lib.load()
    x = points.contiguous()
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2:
        raise ValueError("points must be an (N, k) float32 CUDA tensor")
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    out = C.c_void_p()
    st = lib.rips_barcodes_batched(C.c_void_p(x.data_ptr()), off.ctypes.data_as(C.POINTER(C.c_int64)),
                                   len(off) - 1, x.shape[1], dim_max, C.c_float(threshold), p, _stream_ptr(stream),
                                   C.byref(out))
    _lib.check(st, "rips_barcodes_batched")
    return _collect(lib, out, keep_handle)


def barcodes_batched_dists(dists, dim_max: int = 1, threshold: float = math.inf, p: int = 2, stream=None,
                           keep_handle: bool = False) -> Result:
    """Barcodes of many finite metric spaces: ``dists`` is a list of n_c x n_c
    FP32 CUDA tensors (``rips_barcodes_batched_dists``)."""
    import torch
    lib = _lib.load()
    mats = [d.contiguous() for d in dists]
    for d in mats:
        if not d.is_cuda or d.dtype != torch.float32 or d.dim() != 2 or d.shape[0] != d.shape[1]:
            raise ValueError("every matrix must be an n x n float32 CUDA tensor")
    ptrs = (C.c_void_p * len(mats))(*[d.data_ptr() for d in mats])
    ns = np.array([d.shape[0] for d in mats], dtype=np.int64)
    out = C.c_void_p()
    st = lib.rips_barcodes_batched_dists(ptrs, ns.ctypes.data_as(C.POINTER(C.c_int64)), len(mats), dim_max,
                                         C.c_float(threshold), p, _stream_ptr(stream), C.byref(out))
    _lib.check(st, "rips_barcodes_batched_dists")
    return _collect(lib, out, keep_handle)


def backward_dist(result: Result, dists, grad_birth, grad_death, stream=None):
    """dL/dD for each cloud of ``result`` (made with keep_handle=True) from the
    distance matrices it was computed from (list of CUDA tensors): returns one
    n_c x n_c tensor per cloud, the gradient on its strict lower triangle."""
    import torch
    lib = _lib.load()
    if result._handle is None:
        raise ValueError("result was freed; call the forward with keep_handle=True")
    mats = [d.contiguous() for d in dists]
    grads = [torch.zeros_like(d) for d in mats]
    dp = (C.c_void_p * len(mats))(*[d.data_ptr() for d in mats])
    gp = (C.c_void_p * len(grads))(*[g.data_ptr() for g in grads])
    gb = grad_birth.contiguous().float()
    gd = grad_death.contiguous().float()
    st = lib.rips_barcodes_backward_dist(result._handle, dp, C.c_void_p(gb.data_ptr()), C.c_void_p(gd.data_ptr()),
                                         gp, _stream_ptr(stream))
    _lib.check(st, "rips_barcodes_backward_dist")
    return grads


def backward(result: Result, points, grad_birth, grad_death, grad_dist=None, stream=None):
    """dL/dpoints from dL/dbirth and dL/ddeath (CUDA tensors, one entry per bar
    of ``result`` in its order).  ``result`` must have been made with
    keep_handle=True."""
    import torch
    lib = _lib.load()
    if result._handle is None:
        raise ValueError("result was freed; call the forward with keep_handle=True")
    x = points.contiguous()
    g = torch.zeros_like(x)
    gb = grad_birth.contiguous().float()
    gd = grad_death.contiguous().float()
    st = lib.rips_barcodes_backward(result._handle, C.c_void_p(x.data_ptr()), x.shape[1], C.c_void_p(gb.data_ptr()),
                                    C.c_void_p(gd.data_ptr()), C.c_void_p(g.data_ptr()),
                                    C.c_void_p(grad_dist.data_ptr()) if grad_dist is not None else None,
                                    _stream_ptr(stream))
    _lib.check(st, "rips_barcodes_backward")
    return g


def set_limits(barrier_wait_ns: int = 0, chain_ns: int = 0, arena_entries: int = 0, table_slots: int = 0) -> None:
    """Bounds of the device waits and first buffer sizes (0 = default); small
    values inject the failures the library reports as status codes."""
    lim = _lib.Limits(barrier_wait_ns, chain_ns, arena_entries, table_slots)
    _lib.check(_lib.load().rips_set_limits(C.byref(lim)), "rips_set_limits")


def set_options(apparent: bool = True, emergent: bool = True) -> None:
    """Ablation switches (Table 3 of the paper): turn the apparent-pair skip or
    the emergent first-pivot shortcut off for later calls; bars never change."""
    flags = (0 if apparent else 1) | (0 if emergent else 2)
    _lib.check(_lib.load().rips_set_options(flags), "rips_set_options")


def get_options() -> dict:
    f = int(_lib.load().rips_get_options())
    return {"apparent": not (f & 1), "emergent": not (f & 2)}


def get_limits() -> dict:
    lim = _lib.Limits()
    _lib.check(_lib.load().rips_get_limits(C.byref(lim)), "rips_get_limits")
    return {f: int(getattr(lim, f)) for f, _ in _lib.Limits._fields_}


class BatchPlan:
    """Barcodes H0 and H1 of batches of clouds with fixed sizes, every launch
    fixed in advance (``rips_batch_plan_*``): ``run`` enqueues the whole forward
    for new coordinates without host synchronisation or allocation, so it can
    be captured into a CUDA graph (``capture``) and replayed; ``result`` waits
    for the stream and returns the last run's bars."""

    def __init__(self, offsets, k: int, threshold: float = math.inf, p: int = 2, arena_entries: int = 0):
        self._lib = _lib.load()
        self._off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.k = k
        h = C.c_void_p()
        _lib.check(self._lib.rips_batch_plan_create(self._off.ctypes.data_as(C.POINTER(C.c_int64)), len(self._off) - 1,
                                                    k, C.c_float(threshold), p, arena_entries, C.byref(h)),
                   "rips_batch_plan_create")
        self._h = h

    def run(self, points, stream=None) -> None:
        import torch
        if not points.is_cuda or points.dtype != torch.float32 or not points.is_contiguous():
            raise ValueError("points must be a contiguous float32 CUDA tensor")
        _lib.check(self._lib.rips_batch_plan_run(self._h, C.c_void_p(points.data_ptr()), _stream_ptr(stream)),
                   "rips_batch_plan_run")

    def result(self, stream=None, keep_handle: bool = False) -> Result:
        out = C.c_void_p()
        _lib.check(self._lib.rips_batch_plan_result(self._h, _stream_ptr(stream), C.byref(out)),
                   "rips_batch_plan_result")
        return _collect(self._lib, out, keep_handle)

    def capture(self, points):
        """A CUDA graph of ``run(points)``; replay it after writing new
        coordinates into ``points`` (same tensor), then call ``result``."""
        import torch
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):  # a first run outside the capture (kernel attributes set, memory touched)
            self.run(points, side)
            self.result(side)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            self.run(points, torch.cuda.current_stream())
        return g

    def free(self) -> None:
        if getattr(self, "_h", None):
            self._lib.rips_batch_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def launch_count(reset: bool = False) -> int:
    return int(_lib.load().rips_kernel_launch_count(1 if reset else 0))


def set_kernel_timing(enable: bool) -> bool:
    """Record CUDA events around each kernel class in later calls (profiling)."""
    return bool(_lib.load().rips_set_kernel_timing(1 if enable else 0))


def _torch_autograd():
    import torch

    class RipsBarcodes(torch.autograd.Function):
        """Bars of point clouds as differentiable tensors.

        forward(points (N, k) CUDA FP32, offsets, dim_max, threshold, p) returns
        (birth, death, dim, cloud) tensors with one entry per bar; backward maps
        dL/dbirth and dL/ddeath to dL/dpoints through the critical edges.
        """

        @staticmethod
        def forward(ctx, points, offsets, dim_max=1, threshold=math.inf, p=2):
            res = barcodes_batched(points.detach(), offsets, dim_max, threshold, p, keep_handle=True)
            dev = points.device
            ctx.res = res
            ctx.save_for_backward(points)
            birth = torch.from_numpy(res.bars["birth"].copy()).to(dev)
            death = torch.from_numpy(res.bars["death"].copy()).to(dev)
            dim = torch.from_numpy(res.bars["dim"].astype(np.int64)).to(dev)
            cloud = torch.from_numpy(res.bars["cloud"].astype(np.int64)).to(dev)
            ctx.mark_non_differentiable(dim, cloud)
            return birth, death, dim, cloud

        @staticmethod
        def backward(ctx, g_birth, g_death, _gdim, _gcloud):
            (points,) = ctx.saved_tensors
            if g_birth is None:
                g_birth = torch.zeros(len(ctx.res.bars), device=points.device)
            if g_death is None:
                g_death = torch.zeros(len(ctx.res.bars), device=points.device)
            g_death = torch.where(torch.isfinite(g_death), g_death, torch.zeros_like(g_death))
            gx = backward(ctx.res, points.detach(), g_birth, g_death)
            return gx, None, None, None, None

    return RipsBarcodes


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _torch_autograd()
        return getattr(_Lazy._cls, name)


RipsBarcodes = _Lazy()
