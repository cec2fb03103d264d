"""CPU oracle for Vietoris–Rips persistence barcodes -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does.  It is a ctypes wrapper around ``rips_oracle.c``,
which is built with plain gcc by :func:`build`.

Methods (see ``rips_oracle.h``):
  ``"def"`` -- explicit filtration boundary matrix + standard reduction
              (Algorithm 1), homology, all dimensions at once;
  ``"coh"`` -- cohomology with clearing (Algorithm 2 on coboundary matrices,
              Sections 3.3-3.4), implicit coboundary columns, Kruskal for H0,
              without the apparent/emergent shortcuts.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rips_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "librips_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/ (host architecture)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rips_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Bar(C.Structure):
    _fields_ = [("dim", C.c_int32), ("birth", C.c_float), ("death", C.c_float),
                ("birth_simplex", C.c_int64), ("death_simplex", C.c_int64)]


class _Stats(C.Structure):
    _fields_ = [("simplices", C.c_int64), ("columns", C.c_int64), ("pairs", C.c_int64),
                ("zero_pairs", C.c_int64), ("essential", C.c_int64), ("apparent_zero", C.c_int64),
                ("additions", C.c_int64)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    fp = C.POINTER(C.c_float)
    i64p = C.POINTER(C.c_int64)
    lib.oracle_barcodes.argtypes = [fp, C.c_int64, C.c_int32, C.c_float, C.c_uint32, C.c_int32,
                                    C.POINTER(C.c_void_p)]
    lib.oracle_barcodes.restype = C.c_int
    lib.oracle_result_num_bars.argtypes = [C.c_void_p]
    lib.oracle_result_num_bars.restype = C.c_int64
    lib.oracle_result_bars.argtypes = [C.c_void_p]
    lib.oracle_result_bars.restype = C.POINTER(_Bar)
    lib.oracle_result_threshold.argtypes = [C.c_void_p]
    lib.oracle_result_threshold.restype = C.c_float
    lib.oracle_result_stats.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_Stats)]
    lib.oracle_result_stats.restype = C.c_int
    lib.oracle_result_free.argtypes = [C.c_void_p]
    lib.oracle_result_free.restype = None
    lib.oracle_result_cocycle.argtypes = [C.c_void_p, C.c_int64, i64p, C.POINTER(C.c_uint32), C.c_int64]
    lib.oracle_result_cocycle.restype = C.c_int64
    lib.oracle_simplex_index.argtypes = [i64p, C.c_int32]
    lib.oracle_simplex_index.restype = C.c_int64
    lib.oracle_simplex_vertices.argtypes = [C.c_int64, C.c_int32, C.c_int64, i64p]
    lib.oracle_simplex_vertices.restype = C.c_int
    lib.oracle_filtration.argtypes = [fp, C.c_int64, C.c_int32, C.c_float, C.POINTER(C.c_int32),
                                      i64p, fp, C.c_int64]
    lib.oracle_filtration.restype = C.c_int64
    lib.oracle_apparent_pairs.argtypes = [fp, C.c_int64, C.c_int32, C.c_float, i64p, i64p, C.c_int64]
    lib.oracle_apparent_pairs.restype = C.c_int64
    lib.oracle_boundary_matrix.argtypes = [fp, C.c_int64, C.c_int32, C.c_float, C.c_uint32, i64p,
                                           i64p, C.POINTER(C.c_uint32), C.c_int64]
    lib.oracle_boundary_matrix.restype = C.c_int64
    lib.oracle_count_simplices.argtypes = [fp, C.c_int64, C.c_int32, C.c_float]
    lib.oracle_count_simplices.restype = C.c_int64
    lib.oracle_enclosing_radius.argtypes = [fp, C.c_int64]
    lib.oracle_enclosing_radius.restype = C.c_float
    _lib = lib
    return lib


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _i64(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _as_matrix(dist) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(dist, dtype=np.float32))
    if d.ndim != 2 or d.shape[0] != d.shape[1]:
        raise ValueError("distance matrix must be n x n")
    return d


class OracleError(RuntimeError):
    pass


@dataclass
class OracleResult:
    """Bars (structured numpy array) plus per-dimension statistics."""
    bars: np.ndarray          # fields dim, birth, death, birth_simplex, death_simplex
    threshold: float          # effective threshold used
    stats: list               # list of dicts per dimension 0..dim_max
    # with cocycles=True: per bar (same order), its representative cocycle as
    # (d-simplex indices, Z/p coefficients), empty for H0 bars
    cocycles: list | None = None

    def dim(self, d: int) -> np.ndarray:
        return self.bars[self.bars["dim"] == d]


BAR_DTYPE = np.dtype([("dim", np.int32), ("birth", np.float32), ("death", np.float32),
                      ("birth_simplex", np.int64), ("death_simplex", np.int64)])


def barcodes(dist, dim_max: int, threshold: float = math.inf, p: int = 2,
             method: str = "coh", keep_zero: bool = False, cocycles: bool = False) -> OracleResult:
    """Persistence barcodes H0..H_dim_max of the Rips filtration of ``dist``.

    With ``keep_zero`` the zero-persistence pairs are listed as bars too (birth
    equal to death), which exposes every persistence pair of the refined
    filtration.  With ``cocycles`` (method "coh") every bar of dimension d >= 1
    also gets its representative cocycle: the column V_j of the coboundary
    reduction of its birth simplex (Sections 3.1 and 3.4), R_j = delta V_j.
    """
    lib = _load()
    d = _as_matrix(dist)
    n = d.shape[0]
    out = C.c_void_p()
    m = {"def": 0, "coh": 1}[method] | (0x10 if keep_zero else 0)
    rc = lib.oracle_barcodes(_fptr(d), n, dim_max, C.c_float(threshold), p, m, C.byref(out))
    if rc != 0:
        raise OracleError(f"oracle_barcodes failed with status {rc}")
    try:
        nb = lib.oracle_result_num_bars(out)
        ptr = lib.oracle_result_bars(out)
        arr = np.zeros(nb, dtype=BAR_DTYPE)
        if nb:
            raw = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_uint8)), shape=(nb * C.sizeof(_Bar),))
            src = np.frombuffer(raw.tobytes(), dtype=np.dtype({
                "names": ["dim", "birth", "death", "birth_simplex", "death_simplex"],
                "formats": [np.int32, np.float32, np.float32, np.int64, np.int64],
                "offsets": [_Bar.dim.offset, _Bar.birth.offset, _Bar.death.offset,
                            _Bar.birth_simplex.offset, _Bar.death_simplex.offset],
                "itemsize": C.sizeof(_Bar)}))
            for f in BAR_DTYPE.names:
                arr[f] = src[f]
        stats = []
        for k in range(dim_max + 1):
            s = _Stats()
            lib.oracle_result_stats(out, k, C.byref(s))
            stats.append({f: int(getattr(s, f)) for f, _ in _Stats._fields_})
        t = float(lib.oracle_result_threshold(out))
        cocs = None
        if cocycles:
            cocs = []
            for q in range(nb):
                ln = int(lib.oracle_result_cocycle(out, q, None, None, 0))
                idx = np.zeros(max(ln, 1), dtype=np.int64)
                cf = np.zeros(max(ln, 1), dtype=np.uint32)
                if ln > 0:
                    lib.oracle_result_cocycle(out, q, _i64(idx), cf.ctypes.data_as(C.POINTER(C.c_uint32)), ln)
                cocs.append((idx[:ln], cf[:ln]))
    finally:
        lib.oracle_result_free(out)
    order = np.lexsort((arr["birth_simplex"], arr["death"], arr["birth"], arr["dim"]))
    return OracleResult(arr[order], t, stats, [cocs[i] for i in order] if cocs is not None else None)


def simplex_index(vertices) -> int:
    lib = _load()
    v = np.ascontiguousarray(np.asarray(vertices, dtype=np.int64))
    return int(lib.oracle_simplex_index(_i64(v), len(v) - 1))


def simplex_vertices(index: int, d: int, n: int) -> list[int]:
    lib = _load()
    out = np.zeros(d + 1, dtype=np.int64)
    if lib.oracle_simplex_vertices(index, d, n, _i64(out)) != 0:
        raise OracleError("bad simplex index")
    return [int(x) for x in out]


def filtration(dist, maxdim: int, threshold: float = math.inf):
    """(dims, indices, diameters) of the maxdim-skeleton in filtration order."""
    lib = _load()
    d = _as_matrix(dist)
    n = d.shape[0]
    cnt = lib.oracle_filtration(_fptr(d), n, maxdim, C.c_float(threshold), None, None, None, 0)
    if cnt < 0:
        raise OracleError(f"oracle_filtration failed with status {cnt}")
    dims = np.zeros(cnt, dtype=np.int32)
    idx = np.zeros(cnt, dtype=np.int64)
    diam = np.zeros(cnt, dtype=np.float32)
    lib.oracle_filtration(_fptr(d), n, maxdim, C.c_float(threshold),
                          dims.ctypes.data_as(C.POINTER(C.c_int32)), _i64(idx), _fptr(diam), cnt)
    return dims, idx, diam


def apparent_pairs(dist, maxdim: int, threshold: float = math.inf):
    """Apparent pairs (sigma position, tau position) of the refined filtration."""
    lib = _load()
    d = _as_matrix(dist)
    n = d.shape[0]
    cnt = lib.oracle_apparent_pairs(_fptr(d), n, maxdim, C.c_float(threshold), None, None, 0)
    if cnt < 0:
        raise OracleError(f"oracle_apparent_pairs failed with status {cnt}")
    s = np.zeros(cnt, dtype=np.int64)
    t = np.zeros(cnt, dtype=np.int64)
    lib.oracle_apparent_pairs(_fptr(d), n, maxdim, C.c_float(threshold), _i64(s), _i64(t), cnt)
    return list(zip(s.tolist(), t.tolist()))


def boundary_matrix(dist, maxdim: int, threshold: float = math.inf, p: int = 2) -> np.ndarray:
    """Dense filtration boundary matrix (rows and columns in filtration order)."""
    lib = _load()
    d = _as_matrix(dist)
    n = d.shape[0]
    cnt = lib.oracle_boundary_matrix(_fptr(d), n, maxdim, C.c_float(threshold), p, None, None, None, 0)
    if cnt < 0:
        raise OracleError(f"oracle_boundary_matrix failed with status {cnt}")
    rows = np.zeros(cnt, dtype=np.int64)
    cols = np.zeros(cnt, dtype=np.int64)
    coef = np.zeros(cnt, dtype=np.uint32)
    lib.oracle_boundary_matrix(_fptr(d), n, maxdim, C.c_float(threshold), p, _i64(rows), _i64(cols),
                               coef.ctypes.data_as(C.POINTER(C.c_uint32)), cnt)
    dims, _, _ = filtration(d, maxdim, threshold)
    m = np.zeros((len(dims), len(dims)), dtype=np.int64)
    m[rows, cols] = coef
    return m


def count_simplices(dist, d: int, threshold: float = math.inf) -> int:
    lib = _load()
    m = _as_matrix(dist)
    r = lib.oracle_count_simplices(_fptr(m), m.shape[0], d, C.c_float(threshold))
    if r < 0:
        raise OracleError(f"oracle_count_simplices failed with status {r}")
    return int(r)


def enclosing_radius(dist) -> float:
    lib = _load()
    m = _as_matrix(dist)
    return float(lib.oracle_enclosing_radius(_fptr(m), m.shape[0]))
