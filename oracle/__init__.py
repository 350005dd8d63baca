"""CPU oracle for HODLRdD -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C++ restatement of the method (``hodlrdd_oracle.cpp``) with a
ctypes wrapper. Only the tests, the smoke check and the benchmark's CPU-baseline
leg may import this package. It shares no code with the CUDA library.

* ``direct``          the exact O(N^2) product y = K x (kernel-matrix definition);
* ``Tree``            the balanced 2^d tree, interaction lists (clan / IL
                      definitions and the HODLRdD admissibility condition), ACA of
                      every IL block (Eq. keq1/keq2, Algorithm 1) and the matvec of
                      Algorithm 2, in stored-factor and memory-efficient forms;
* ``aca_dense``       ACA of an explicit matrix, for pinning the ACA itself;
* ``kernel_block``    a dense block F(X_i, Y_j), for pinning the kernels.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hodlrdd_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_DENSE_IF_CHEAPER = 1
FLAG_DENSE_LEAF_ONLY = 2

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (FP contraction off, OpenMP on)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        lib.or_set_threads.argtypes = [C.c_int]
        lib.or_set_threads.restype = C.c_int
        lib.or_direct_rows.argtypes = [_f64p, C.c_int, C.c_int64, C.c_int, _f64p, _f64p, C.c_int, C.c_int64,
                                       C.c_int64, _f64p]
        lib.or_kernel_block.argtypes = [_f64p, C.c_int64, _f64p, C.c_int64, C.c_int, C.c_int, _f64p, _f64p]
        lib.or_aca_dense.argtypes = [_f64p, C.c_int64, C.c_int64, C.c_double, C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), _i64p, _i64p, _f64p, _f64p]
        lib.or_build.argtypes = [_f64p, C.c_int, C.c_int64, C.c_int, _f64p, C.c_int, C.c_double, C.c_int,
                                 C.POINTER(C.c_void_p)]
        lib.or_build_ex.argtypes = [_f64p, C.c_int, C.c_int64, C.c_int, _f64p, C.c_int, C.c_double, C.c_int,
                                    C.c_int, C.POINTER(C.c_void_p)]
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_destroy.restype = None
        lib.or_info.argtypes = [C.c_void_p, _i64p]
        lib.or_cube.argtypes = [C.c_void_p, _f64p, _f64p]
        lib.or_perm.argtypes = [C.c_void_p, _i64p, _u64p]
        lib.or_level_nboxes.argtypes = [C.c_void_p, C.c_int]
        lib.or_level_nboxes.restype = C.c_int64
        lib.or_level.argtypes = [C.c_void_p, C.c_int, _i64p, _u64p]
        lib.or_il_size.argtypes = [C.c_void_p, C.c_int]
        lib.or_il_size.restype = C.c_int64
        lib.or_il.argtypes = [C.c_void_p, C.c_int, _i64p, _i64p]
        lib.or_near.argtypes = [C.c_void_p, _i64p, _i64p]
        lib.or_blocks.argtypes = [C.c_void_p, _i64p]
        lib.or_block_factors.argtypes = [C.c_void_p, C.c_int64, _i64p, _i64p, C.c_void_p, C.c_void_p]
        lib.or_matvec.argtypes = [C.c_void_p, _f64p, _f64p, C.c_int]
        lib.or_matvec_skeleton.argtypes = [C.c_void_p, _f64p, _f64p, C.c_int]
        _lib = lib
        return lib


def set_threads(n: int) -> int:
    return _load().or_set_threads(int(n))


def _params(params) -> np.ndarray:
    p = np.zeros(4, np.float64)
    p[0] = 1.0
    if params is not None:
        v = np.asarray(params, np.float64).reshape(-1)
        p[: min(4, v.size)] = v[:4]
    return p


def _as2d(x, N):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x.reshape(N, 1)
    return x


def direct(points, kernel, params, x, rows=None) -> np.ndarray:
    """y = K x by direct summation (rows: optional (r0, r1) range)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    N, d = pts.shape
    xx = _as2d(x, N)
    nrhs = xx.shape[1]
    r0, r1 = (0, N) if rows is None else rows
    y = np.zeros((r1 - r0, nrhs), np.float64)
    rc = _load().or_direct_rows(pts, d, N, int(kernel), _params(params), xx, nrhs, r0, r1, y)
    if rc:
        raise ValueError("or_direct_rows: invalid arguments")
    return y


def kernel_block(X, Y, kernel, params=None) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros((X.shape[0], Y.shape[0]), np.float64)
    if _load().or_kernel_block(X, X.shape[0], Y, Y.shape[0], X.shape[1], int(kernel), _params(params), out):
        raise ValueError("or_kernel_block: invalid kernel")
    return out


def aca_dense(A, tol, flags=0):
    """ACA of a dense matrix: returns (rank, dense, sigma, tau, U (m x p), V (n x p))."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    k = min(m, n)
    sig = np.zeros(k, np.int64)
    tau = np.zeros(k, np.int64)
    U = np.zeros(m * k, np.float64)
    V = np.zeros(n * k, np.float64)
    rank = C.c_int(0)
    dense = C.c_int(0)
    if _load().or_aca_dense(A, m, n, float(tol), int(flags), C.byref(rank), C.byref(dense), sig, tau, U, V):
        raise ValueError("or_aca_dense: invalid arguments")
    p = rank.value
    return (p, dense.value, sig[:p].copy(), tau[:p].copy(), U[: m * p].reshape(p, m).T.copy(),
            V[: n * p].reshape(p, n).T.copy())


class Tree:
    """The oracle's HODLRdD representation of K for one point set."""

    def __init__(self, points, kernel, params=None, leaf=64, tol=1e-8, dense_if_cheaper=False, admissible_face_dim=0):
        lib = _load()
        pts = np.ascontiguousarray(points, dtype=np.float64)
        self.N, self.d = pts.shape
        self.kernel = int(kernel)
        self.params = _params(params)
        h = C.c_void_p()
        # dense_if_cheaper: False / True, or "leaf" (the rule at the leaf level only)
        flags = (FLAG_DENSE_IF_CHEAPER | FLAG_DENSE_LEAF_ONLY if dense_if_cheaper == "leaf"
                 else FLAG_DENSE_IF_CHEAPER if dense_if_cheaper else 0)
        rc = lib.or_build_ex(pts, self.d, self.N, self.kernel, self.params, int(leaf), float(tol), flags,
                             int(admissible_face_dim), C.byref(h))
        if rc:
            raise ValueError(f"or_build failed ({rc})")
        self._h = h
        self._lib = lib
        info = np.zeros(8, np.int64)
        lib.or_info(h, info)
        (self.kappa, self.B, self.nblocks, self.nnear, self.factor_elems, self.n_dense, self.n_capped,
         self.max_rank) = (int(v) for v in info)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_destroy(h)
            self._h = None

    def cube(self):
        lo = np.zeros(self.d, np.float64)
        si = np.zeros(2, np.float64)
        self._lib.or_cube(self._h, lo, si)
        return lo, float(si[0]), float(si[1])

    def perm(self):
        p = np.zeros(self.N, np.int64)
        k = np.zeros(self.N, np.uint64)
        self._lib.or_perm(self._h, p, k)
        return p, k

    def level(self, l):
        nb = self._lib.or_level_nboxes(self._h, int(l))
        st = np.zeros(nb + 1, np.int64)
        bk = np.zeros(nb, np.uint64)
        self._lib.or_level(self._h, int(l), st, bk)
        return st, bk

    def il(self, l):
        nb = self._lib.or_level_nboxes(self._h, int(l))
        ne = self._lib.or_il_size(self._h, int(l))
        off = np.zeros(nb + 1, np.int64)
        idx = np.zeros(max(ne, 0), np.int64)
        self._lib.or_il(self._h, int(l), off, idx)
        return off, idx

    def near(self):
        nb = self._lib.or_level_nboxes(self._h, self.kappa)
        off = np.zeros(nb + 1, np.int64)
        idx = np.zeros(self.nnear, np.int64)
        self._lib.or_near(self._h, off, idx)
        return off, idx

    def blocks(self):
        """(nblocks, 10) int64: level, ti, sj, I0, m, J0, n, rank, dense, capped."""
        if getattr(self, "_blocks", None) is None:
            rec = np.zeros(max(self.nblocks, 1) * 10, np.int64)
            self._lib.or_blocks(self._h, rec)
            self._blocks = rec[: self.nblocks * 10].reshape(self.nblocks, 10)
            self._blocks.setflags(write=False)
        return self._blocks

    def factors(self, b):
        rec = self.blocks()[b]
        m, n, p = int(rec[4]), int(rec[6]), int(rec[7])
        sig = np.zeros(max(p, 1), np.int64)
        tau = np.zeros(max(p, 1), np.int64)
        U = np.zeros(max(m * p, 1), np.float64)
        V = np.zeros(max(n * p, 1), np.float64)
        self._lib.or_block_factors(self._h, int(b), sig, tau, U.ctypes.data_as(C.c_void_p),
                                   V.ctypes.data_as(C.c_void_p))
        return sig[:p], tau[:p], U[: m * p].reshape(p, m).T, V[: n * p].reshape(p, n).T

    def matvec(self, x, skeleton=False):
        xx = _as2d(x, self.N)
        y = np.zeros_like(xx)
        f = self._lib.or_matvec_skeleton if skeleton else self._lib.or_matvec
        if f(self._h, xx, y, xx.shape[1]):
            raise ValueError("oracle matvec failed")
        return y
