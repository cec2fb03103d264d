"""Seeded synthetic inputs for Vietoris–Rips barcode workloads.

This module only draws point clouds and turns them into FP32 distance matrices.
It holds none of the persistence arithmetic, so both the CUDA path and the CPU
oracle can read its output without sharing any method code.

Bit reproducibility across hosts (x86 and Arm) matters, because the same seed
must give the same FP32 matrix everywhere.  Every value is therefore produced by
IEEE-754 basic operations only (+, -, *, /, sqrt, which are correctly rounded on
every platform), starting from ``Generator.random`` on a PCG64 stream (53 random
bits scaled by 2**-53, exact).  Transcendental library calls (cos, sin, log),
whose last bit can differ between libm implementations, are avoided:

* a uniform direction in R^k comes from rejection sampling in the unit ball
  followed by normalisation;
* a uniform angle on the circle is represented by its (cos, sin) pair, drawn as a
  uniform direction in R^2;
* Gaussian noise uses Marsaglia's polar method, with the natural logarithm
  evaluated by ``_ln`` below (frexp plus a fixed-length atanh series).

Distances follow one rule for every workload: coordinates are rounded to FP32;
each squared difference is formed in float64 and summed over coordinates in
index order with separate rounding per operation (no fused multiply-add); the
float64 square root is rounded to FP32.  The device computes distances from FP32
coordinates with the same rule.

Workloads (seeds are PCG64 seeds):

* ``cube``   -- n points i.i.d. uniform in [0,1]^3 (seed 1001 for 100 points).
* ``torus``  -- n points on the torus in R^3 with major radius 2, minor radius 1,
  both angles i.i.d. uniform, plus isotropic N(0, 0.02^2) noise (seed 1002).
* ``so3``    -- n Haar-random rotation matrices flattened row-major to R^9, from
  unit quaternions uniform on S^3 (seed 1003).
* ``batch``  -- 256 clouds with sizes uniform in {64..512}; each cloud is a noisy
  circle (radius 1 in the xy-plane, sigma 0.05), a noisy torus (R=2, r=1,
  sigma 0.02) or a uniform cube sample, chosen uniformly (meta seed 4000, cloud c
  seed 40000 + c).
* ``sphere3``-- n points uniform on the unit sphere S^3 in R^4 (seed 1005).
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

_LN2 = 0.6931471805599453  # nearest double to ln 2


def _ln(x: np.ndarray) -> np.ndarray:
    """Natural log of positive float64 values with basic IEEE operations only.

    x = m * 2**e with m in [0.5, 1) (frexp is exact); ln m = 2 atanh(y) with
    y = (m - 1)/(m + 1), |y| <= 1/3, summed as a fixed 24-term odd series by
    Horner's rule.  Accurate to a few ulp and identical on every IEEE host.
    """
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    y = (m - 1.0) / (m + 1.0)
    y2 = y * y
    acc = np.zeros_like(y)
    for k in range(23, -1, -1):
        acc = acc * y2 + 1.0 / (2 * k + 1)
    return e.astype(np.float64) * _LN2 + 2.0 * y * acc


def _unit_vectors(rng: np.random.Generator, count: int, k: int) -> np.ndarray:
    """``count`` directions uniform on S^(k-1), by rejection from the unit ball."""
    out = np.empty((0, k), dtype=np.float64)
    while out.shape[0] < count:
        need = count - out.shape[0]
        batch = 2.0 * rng.random((max(64, 4 * need), k)) - 1.0
        r2 = np.zeros(batch.shape[0])
        for c in range(k):
            r2 = r2 + batch[:, c] * batch[:, c]
        keep = (r2 > 1e-12) & (r2 <= 1.0)
        b = batch[keep]
        r = np.sqrt(r2[keep])
        out = np.concatenate([out, b / r[:, None]], axis=0)
    return out[:count]


def _gaussian(rng: np.random.Generator, count: int) -> np.ndarray:
    """``count`` standard normal samples by Marsaglia's polar method."""
    out = np.empty(0, dtype=np.float64)
    while out.shape[0] < count:
        need = count - out.shape[0]
        u = 2.0 * rng.random(max(64, need)) - 1.0
        v = 2.0 * rng.random(max(64, need)) - 1.0
        s = u * u + v * v
        ok = (s > 0.0) & (s < 1.0)
        u, v, s = u[ok], v[ok], s[ok]
        f = np.sqrt((-2.0 * _ln(s)) / s)
        out = np.concatenate([out, u * f, v * f])
    return out[:count]


def cube_points(n: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, 3)).astype(np.float32)


def _torus(rng: np.random.Generator, n: int, R: float, r: float, sigma: float) -> np.ndarray:
    a = _unit_vectors(rng, n, 2)  # (cos theta, sin theta)
    b = _unit_vectors(rng, n, 2)  # (cos phi, sin phi)
    ring = R + r * b[:, 0]
    pts = np.stack([ring * a[:, 0], ring * a[:, 1], r * b[:, 1]], axis=1)
    noise = _gaussian(rng, 3 * n).reshape(n, 3)
    return pts + sigma * noise


def torus_points(n: int, seed: int, R: float = 2.0, r: float = 1.0, sigma: float = 0.02) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return _torus(rng, n, R, r, sigma).astype(np.float32)


def so3_points(n: int, seed: int) -> np.ndarray:
    """Haar-random rotations (unit quaternions uniform on S^3) flattened to R^9."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = _unit_vectors(rng, n, 4)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    m = np.stack([
        1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
        2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
        2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y),
    ], axis=1)
    return m.astype(np.float32)


def sphere_points(n: int, seed: int, k: int = 4) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return _unit_vectors(rng, n, k).astype(np.float32)


def clifford_points(n: int, seed: int) -> np.ndarray:
    """Points uniform on the Clifford torus S^1(1/sqrt 2) x S^1(1/sqrt 2) in R^4
    (the torus4 data set of the paper's experiments is such a sample): two
    independent uniform unit vectors of R^2, scaled by 1/sqrt 2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = _unit_vectors(rng, n, 2)
    v = _unit_vectors(rng, n, 2)
    s = 1.0 / np.sqrt(2.0)
    return (np.concatenate([u, v], axis=1) * s).astype(np.float32)


def circle_points(rng: np.random.Generator, n: int, sigma: float = 0.05) -> np.ndarray:
    a = _unit_vectors(rng, n, 2)
    pts = np.stack([a[:, 0], a[:, 1], np.zeros(n)], axis=1)
    return pts + sigma * _gaussian(rng, 3 * n).reshape(n, 3)


def distance_matrix(points: np.ndarray) -> np.ndarray:
    """FP32 Euclidean distance matrix of FP32 points (rule in the module docstring)."""
    x = np.asarray(points, dtype=np.float32).astype(np.float64)
    n, k = x.shape
    acc = np.zeros((n, n), dtype=np.float64)
    for c in range(k):
        diff = x[:, None, c] - x[None, :, c]
        acc = acc + diff * diff
    return np.sqrt(acc).astype(np.float32)


def matrix_digest(d: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(d, dtype=np.float32).tobytes()).hexdigest()


@dataclass
class Workload:
    """One barcode problem: points, FP32 distances and the call parameters."""
    name: str
    points: np.ndarray
    dim_max: int
    threshold: float  # +inf means: no threshold (enclosing radius is used)
    p: int
    description: str = ""
    _dist: np.ndarray | None = field(default=None, repr=False)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])

    @property
    def dist(self) -> np.ndarray:
        if self._dist is None:
            self._dist = distance_matrix(self.points)
        return self._dist


def cube_100() -> Workload:
    return Workload("cube100", cube_points(100, 1001), 1, float("inf"), 2,
                    "100 points uniform in [0,1]^3, full Rips, H0-H1, Z/2")


def torus_1000() -> Workload:
    return Workload("torus1000", torus_points(1000, 1002), 2, 1.0, 2,
                    "1000 points on a noisy 2-torus in R^3, threshold 1.0, H0-H2, Z/2")


def so3_4096() -> Workload:
    return Workload("so3_4096", so3_points(4096, 1003), 2, 1.4, 2,
                    "4096 Haar-random rotations in R^9, threshold 1.4, H0-H2, Z/2")


def sphere3_192() -> Workload:
    return Workload("s3_192", sphere_points(192, 1005, 4), 3, float("inf"), 3,
                    "192 points uniform on S^3 in R^4, full Rips, H0-H3, Z/3")


def clifford_1500() -> Workload:
    return Workload("clifford1500", clifford_points(1500, 1006), 2, 0.4, 2,
                    "1500 points on the Clifford torus in R^4, threshold 0.4, H0-H2, Z/2 (sparse path)")


def clifford(n: int, threshold: float, dim_max: int, seed: int = 1007) -> Workload:
    """The torus4 configuration of the paper (n = 50,000, t = 0.15) or a smaller
    one at the same average degree: t = 0.15 sqrt(50000 / n)."""
    return Workload(f"clifford{n}", clifford_points(n, seed), dim_max, threshold, 2,
                    f"{n} points on the Clifford torus in R^4, threshold {threshold}, H0-H{dim_max}, Z/2 (sparse path)")


def batch_clouds(count: int = 256, lo: int = 64, hi: int = 512, meta_seed: int = 4000,
                 cloud_seed: int = 40000) -> list[np.ndarray]:
    """Ragged list of FP32 point clouds (circle / torus / cube mix)."""
    meta = np.random.Generator(np.random.PCG64(meta_seed))
    sizes = meta.integers(lo, hi + 1, size=count)
    kinds = meta.integers(0, 3, size=count)
    clouds = []
    for c in range(count):
        rng = np.random.Generator(np.random.PCG64(cloud_seed + c))
        n = int(sizes[c])
        if kinds[c] == 0:
            pts = circle_points(rng, n, 0.05)
        elif kinds[c] == 1:
            pts = _torus(rng, n, 2.0, 1.0, 0.02)
        else:
            pts = rng.random((n, 3))
        clouds.append(pts.astype(np.float32))
    return clouds


WORKLOADS = {
    "cube100": cube_100,
    "torus1000": torus_1000,
    "so3_4096": so3_4096,
    "s3_192": sphere3_192,
    "clifford1500": clifford_1500,
}


def rectangle() -> np.ndarray:
    """Vertices of the 3x4 rectangle, the worked example of Section 2."""
    return np.array([[0, 0], [3, 0], [0, 4], [3, 4]], dtype=np.float32)


def regular_polygon_matrix(n: int) -> np.ndarray:
    """Distances of a regular n-gon indexed by cyclic step (exact ties).

    d(i, j) = 2 sin(pi * s / n), s = min(|i - j|, n - |i - j|), computed once per
    step s so that equal steps give bit-identical FP32 values.
    """
    steps = np.array([2.0 * np.sin(np.pi * s / n) for s in range(n // 2 + 1)], dtype=np.float64)
    vals = steps.astype(np.float32)
    i = np.arange(n)
    diff = np.abs(i[:, None] - i[None, :])
    s = np.minimum(diff, n - diff)
    return vals[s]


def octahedron_matrix() -> np.ndarray:
    pts = np.concatenate([np.eye(3), -np.eye(3)]).astype(np.float32)
    return distance_matrix(pts)


def regular_simplex_matrix(n: int) -> np.ndarray:
    d = np.ones((n, n), dtype=np.float32)
    np.fill_diagonal(d, 0.0)
    return d


def random_integer_matrix(n: int, seed: int, levels: int = 5) -> np.ndarray:
    """Symmetric matrix with small integer distances in [1, levels]: many ties."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.integers(1, levels + 1, size=(n, n)).astype(np.float32)
    d = np.tril(a, -1)
    d = d + d.T
    return d
