"""Seeded synthetic inputs for HODLRdD: point clouds and right-hand sides.

This module is the one piece shared by the CPU oracle's tests and the GPU
path's tests and benchmark. It draws random numbers only; it holds none of the
method's arithmetic (no kernel evaluation, no tree, no compression).

The paper uses no public dataset. Its matvec experiment places points uniformly
in a hyper-cube (Section "HODLRdD fast matrix-vector product"); its SVM
experiment uses non-uniform random data (Section "HODLRdD accelerated classical
kernel SVM"). The workloads below reproduce those shapes:

* ``uniform``   i.i.d. uniform points in ``[lo, hi]^d``;
* ``clustered`` Gaussian clusters with resampling until every point lies in
  ``[-1, 1]^d`` (the non-uniform case);
* ``grid``      a cell-centred tensor grid ``(k - 1/2) r / n`` (the placement the
  rank study assumes: ``N = n^d`` sources uniformly spread inside a cube).

Every generator takes a seed and draws from one ``numpy.random.default_rng``
stream: points first, then the right-hand sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kernel ids of the C ABI (include/hodlrdd.h). Repeated here as plain integers so
# that tests and the benchmark can name workloads without importing either side.
K_LOG, K_INV_R, K_MATERN32, K_GAUSS, K_EXP, K_INV_R2_4D, K_R, K_SIN, K_INV_SQRT1P = range(9)
KERNEL_NAMES = {
    K_LOG: "log r", K_INV_R: "1/r", K_MATERN32: "matern-3/2", K_GAUSS: "gaussian",
    K_EXP: "exp(-r/l)", K_INV_R2_4D: "-1/(4 pi^2 r^2)", K_R: "r", K_SIN: "sin r",
    K_INV_SQRT1P: "1/sqrt(1+r)",
}


@dataclass
class Workload:
    """One HODLRdD problem: points, kernel, build knobs and right-hand sides."""

    name: str
    d: int
    N: int
    kernel: int
    params: tuple  # (scale, diag, p0, p1): K_ij = scale * F(x_i, x_j; p0, p1) + diag * [i == j]
    leaf: int
    tol: float
    nrhs: int
    seed: int
    dist: str = "uniform"
    box: tuple = (-1.0, 1.0)
    points: np.ndarray = field(default=None, repr=False)
    x: np.ndarray = field(default=None, repr=False)


def uniform_points(rng: np.random.Generator, N: int, d: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.ascontiguousarray(rng.uniform(lo, hi, size=(N, d)), dtype=np.float64)


def clustered_points(rng: np.random.Generator, N: int, d: int, n_clusters: int = 8, sigma: float = 0.1) -> np.ndarray:
    """Gaussian clusters inside [-1,1]^d; points falling outside are redrawn."""
    centres = rng.uniform(-1.0, 1.0, size=(n_clusters, d))
    labels = rng.integers(0, n_clusters, size=N)
    pts = centres[labels] + sigma * rng.standard_normal((N, d))
    bad = np.any(np.abs(pts) > 1.0, axis=1)
    while bad.any():
        k = int(bad.sum())
        pts[bad] = centres[labels[bad]] + sigma * rng.standard_normal((k, d))
        bad = np.any(np.abs(pts) > 1.0, axis=1)
    return np.ascontiguousarray(pts, dtype=np.float64)


def grid_points(n: int, d: int, r: float = 1.0, offset=None) -> np.ndarray:
    """Cell-centred n^d grid in [0, r]^d, shifted by ``offset`` (length-d)."""
    axis = (np.arange(1, n + 1) - 0.5) * (r / n)
    mesh = np.meshgrid(*([axis] * d), indexing="ij")
    pts = np.stack([m.reshape(-1) for m in mesh], axis=1)
    if offset is not None:
        pts = pts + np.asarray(offset, dtype=np.float64)[None, :]
    return np.ascontiguousarray(pts, dtype=np.float64)


def make(name: str, d: int, N: int, kernel: int, params=(1.0, 0.0, 0.0, 0.0), leaf: int = 64,
         tol: float = 1e-8, nrhs: int = 1, seed: int = 0, dist: str = "uniform",
         box=(-1.0, 1.0)) -> Workload:
    """Draw points then right-hand sides (standard normal, N x nrhs row-major)."""
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        pts = uniform_points(rng, N, d, box[0], box[1])
    elif dist == "clustered":
        pts = clustered_points(rng, N, d)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    x = np.ascontiguousarray(rng.standard_normal((N, nrhs)), dtype=np.float64)
    p = tuple(float(v) for v in (list(params) + [0.0] * 4)[:4])
    return Workload(name, d, N, kernel, p, leaf, tol, nrhs, seed, dist, tuple(box), pts, x)


# --- The five workload shapes ------------------------------------------------------------
def plain_fp64_2d(N: int = 4096, seed: int = 0) -> Workload:
    """d=2, uniform in [-1,1]^2, F = log r with F(x,x)=0, leaf 64, tol 1e-8, nrhs 1."""
    return make("plain-fp64 d=2 log r", 2, N, K_LOG, (1.0, 0.0, 0.0, 0.0), 64, 1e-8, 1, seed)


def precision_3d(N: int = 262144, seed: int = 0, system: bool = False) -> Workload:
    """d=3, uniform in [-1,1]^3, F = 1/r with zero diagonal, leaf 64, tol 1e-7.

    ``system=True`` gives the second-kind operator I + K/N (scale 1/N, diag 1).
    """
    params = (1.0 / N, 1.0, 0.0, 0.0) if system else (1.0, 0.0, 0.0, 0.0)
    return make("precision d=3 1/r", 3, N, K_INV_R, params, 64, 1e-7, 1, seed)


def many_rhs_4d(N: int = 65536, nrhs: int = 64, seed: int = 0) -> Workload:
    """d=4, uniform in [0,1]^4, Matern-3/2 with l = 0.2, leaf 128, tol 1e-8."""
    return make("many-rhs d=4 matern-3/2", 4, N, K_MATERN32, (1.0, 0.0, 0.2, 0.0), 128, 1e-8, nrhs, seed,
                box=(0.0, 1.0))


def uneven_instances(n_sets: int = 48, base_seed: int = 1000):
    """48 clustered d=3 sets, N log-uniform in [2048, 131072], Gaussian h=0.5 + 1e-3 I."""
    out = []
    for s in range(n_sets):
        rng = np.random.default_rng(base_seed + s)
        N = int(round(math.exp(rng.uniform(math.log(2048), math.log(131072)))))
        nrhs = int(rng.integers(1, 17))
        pts = clustered_points(rng, N, 3)
        x = np.ascontiguousarray(rng.standard_normal((N, nrhs)), dtype=np.float64)
        out.append(Workload(f"uneven set {s}", 3, N, K_GAUSS, (1.0, 1e-3, 0.5, 0.0), 64, 1e-6, nrhs,
                            base_seed + s, "clustered", (-1.0, 1.0), pts, x))
    return out


def subsample(w: Workload, N: int, seed: int = 12345) -> Workload:
    """A smaller draw from the same distribution (for bounded CPU samples)."""
    return make(w.name + f" (N={N})", w.d, N, w.kernel, w.params, w.leaf, w.tol, w.nrhs, seed, w.dist, w.box)
