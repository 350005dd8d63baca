"""ctypes binding of libhodlrdd (include/hodlrdd.h): argument marshalling only.

Every computation happens in the CUDA library. Arrays may be numpy arrays (host
memory) or torch tensors (host or CUDA); torch is used for device memory and
streams only. If the compiled library is missing this module raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libhodlrdd.so")
HEADER = os.path.join(ROOT, "include", "hodlrdd.h")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_NUMERIC = range(7)
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "fp32+fp16": 4, "fp16x2": 5}
MAX_LEVELS = 64


class HodlrddError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("dense_if_cheaper", C.c_int), ("max_nrhs", C.c_int),
                ("aca_max_rank", C.c_int), ("near_mode", C.c_int), ("admissible_face_dim", C.c_int),
                ("lowrank_form", C.c_int), ("near_coords", C.c_int), ("fp64_near", C.c_int),
                ("near_sms", C.c_int), ("reserved", C.c_int * 2)]


class SolveOptions(C.Structure):
    _fields_ = [("tol", C.c_double), ("inner_tol", C.c_double), ("restart", C.c_int), ("max_inner_iters", C.c_int),
                ("max_refine", C.c_int), ("reserved", C.c_int * 5)]


class SolveStats(C.Structure):
    _fields_ = [("refinements", C.c_int), ("inner_iterations", C.c_int), ("residual", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("d", C.c_int), ("kappa", C.c_int), ("precision", C.c_int), ("max_rank", C.c_int),
        ("N", C.c_int64), ("n_blocks", C.c_int64), ("n_lowrank", C.c_int64), ("n_dense", C.c_int64),
        ("n_rank_capped", C.c_int64), ("n_near", C.c_int64), ("factor_elems", C.c_int64),
        ("factor_bytes", C.c_int64), ("dense_pairs", C.c_int64),
        ("boxes_per_level", C.c_int64 * MAX_LEVELS), ("blocks_per_level", C.c_int64 * MAX_LEVELS),
        ("max_rank_per_level", C.c_int * MAX_LEVELS), ("mean_rank_per_level", C.c_double * MAX_LEVELS),
        ("t_tree_ms", C.c_double), ("t_classify_ms", C.c_double), ("t_aca_ms", C.c_double),
        ("t_pack_ms", C.c_double), ("t_build_ms", C.c_double), ("device_bytes", C.c_int64),
        ("factor_bytes_u", C.c_int64), ("factor_bytes_v", C.c_int64), ("total_rank", C.c_int64),
        ("lowrank_form", C.c_int), ("skeleton_bytes", C.c_int64), ("skeleton_pairs", C.c_int64),
        ("tail_cols", C.c_int64), ("skeleton_terms", C.c_int64), ("near_sms", C.c_int),
    ]


_lib = None


def load():
    """Load the compiled library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libhodlrdd.so not found at {LIB_PATH}: run "
                          "`python -c 'import __graft_entry__ as g; g.build()'` first (no CPU fallback exists)")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "hodlrdd_options_default": (i32, [C.POINTER(Options)]),
        "hodlrdd_build": (i32, [vp, i32, i64, i32, vp, i32, dbl, C.POINTER(vp)]),
        "hodlrdd_build_ex": (i32, [vp, i32, i64, i32, vp, i32, dbl, C.POINTER(Options), C.POINTER(vp)]),
        "hodlrdd_matvec": (i32, [vp, vp, vp, i32, vp]),
        "hodlrdd_matvec_noalloc": (i32, [vp, vp, vp, i32, vp]),
        "hodlrdd_direct": (i32, [vp, vp, vp, vp]),
        "hodlrdd_batch_create": (i32, [C.POINTER(vp), C.POINTER(C.c_int), i32, C.POINTER(vp)]),
        "hodlrdd_batch_run": (i32, [vp, C.POINTER(vp), C.POINTER(vp), vp]),
        "hodlrdd_batch_destroy": (i32, [vp]),
        "hodlrdd_forest_create": (i32, [C.POINTER(vp), C.POINTER(C.c_int), i32, C.POINTER(vp)]),
        "hodlrdd_forest_run": (i32, [vp, C.POINTER(vp), C.POINTER(vp), vp]),
        "hodlrdd_forest_stats": (i32, [vp, C.POINTER(i64)]),
        "hodlrdd_forest_profile": (i32, [vp, vp]),
        "hodlrdd_forest_destroy": (i32, [vp]),
        "hodlrdd_debug_ff_eval": (i32, [i32, vp, dbl, vp, vp, i64]),
        "hodlrdd_debug_aca_pool_bytes": (i32, [i64]),
        "hodlrdd_solve_options_default": (i32, [C.POINTER(SolveOptions)]),
        "hodlrdd_solve": (i32, [vp, vp, vp, vp, C.POINTER(SolveOptions), C.POINTER(SolveStats), vp]),
        "hodlrdd_destroy": (i32, [vp]),
        "hodlrdd_get_stats": (i32, [vp, C.POINTER(Stats)]),
        "hodlrdd_error_string": (C.c_char_p, [i32]),
        "hodlrdd_last_error": (C.c_char_p, []),
        "hodlrdd_get_tree": (i32, [vp, vp, vp]),
        "hodlrdd_get_cube": (i32, [vp, vp, vp]),
        "hodlrdd_get_level": (i32, [vp, i32, C.POINTER(i64), vp, vp]),
        "hodlrdd_get_il": (i32, [vp, i32, C.POINTER(i64), vp, vp]),
        "hodlrdd_get_near": (i32, [vp, C.POINTER(i64), vp, vp]),
        "hodlrdd_get_blocks": (i32, [vp, vp]),
        "hodlrdd_get_pivots": (i32, [vp, i64, vp, vp]),
        "hodlrdd_get_factors": (i32, [vp, i64, vp, vp]),
        "hodlrdd_import_factors": (i32, [vp, vp, vp, vp, vp]),
        "hodlrdd_debug_fail_alloc_after": (i32, [i64]),
        "hodlrdd_set_profiling": (i32, [vp, i32]),
        "hodlrdd_sync": (i32, [vp]),
        "hodlrdd_get_profile": (i32, [vp, vp, C.POINTER(i64), C.POINTER(i64)]),
        "hodlrdd_debug_expire_wait": (i32, [vp, C.c_longlong]),
        "hodlrdd_probe_peaks": (i32, [vp, i32, vp]),
        "hodlrdd_server_create": (i32, [i64, i32, C.POINTER(vp)]),
        "hodlrdd_server_add": (i32, [vp, vp, i32, i64, i32, vp, i32, dbl, C.POINTER(Options), C.POINTER(i64)]),
        "hodlrdd_server_submit": (i32, [vp, i64, i32, vp, vp, i32, C.POINTER(i64)]),
        "hodlrdd_server_wait": (i32, [vp, i64, vp]),
        "hodlrdd_server_stats": (i32, [vp, vp]),
        "hodlrdd_server_set_batching": (i32, [vp, i32]),
        "hodlrdd_server_batch_stats": (i32, [vp, C.POINTER(i64)]),
        "hodlrdd_server_destroy": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of every function include/hodlrdd.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(hodlrdd_\w+)\s*\(", text, re.M)))


def _check(status: int, where: str):
    if status != OK:
        lib = load()
        detail = lib.hodlrdd_last_error().decode(errors="replace")
        raise HodlrddError(status, where, detail or lib.hodlrdd_error_string(status).decode())


def _ptr(a):
    """(address, keepalive) of a numpy array or torch tensor (any device)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)!r}")


def _check_io(a, name, N, io_dtype, device, like=None):
    """Reject an x or y the C library would read or write out of bounds: the
    leading dimension must be N, the element type the handle's (float64 for
    FP64 handles, float32 otherwise), a CUDA tensor must sit on the handle's
    device, and y must have x's shape. Raises ValueError before any C call."""
    shape = tuple(int(v) for v in a.shape)
    if len(shape) not in (1, 2) or shape[0] != N or (len(shape) == 2 and shape[1] < 1):
        raise ValueError(f"{name}: shape {shape}, expected ({N},) or ({N}, nrhs)")
    if like is not None and shape != tuple(int(v) for v in like.shape):
        raise ValueError(f"{name}: shape {shape} differs from x's {tuple(int(v) for v in like.shape)}")
    want = np.dtype(io_dtype)
    if isinstance(a, np.ndarray):
        got = a.dtype
    else:
        try:
            got = np.dtype(str(a.dtype).replace("torch.", ""))
        except TypeError:  # a type numpy does not know (bfloat16, ...)
            got = str(a.dtype)
        if getattr(a, "is_cuda", False) and device is not None and a.device.index != device:
            raise ValueError(f"{name}: on cuda:{a.device.index}, the handle lives on cuda:{device}")
    if got != want:
        raise ValueError(f"{name}: element type {got}, the handle computes in {want}")


def _current_device():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_device()
    except ImportError:
        pass
    return None


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


# What a low-rank block keeps: its factors U_b, V_b, or the skeleton (pivots and
# the LU factors of K(sigma, tau)) with kernel entries evaluated on the fly.
NEAR_COORDS = {"hilo": 0, "hi": 1}
FP64_NEAR = {"fp64": 0, "ff": 1}
LOWRANK_FORM = {"factors": 0, "skeleton": 1}


class Handle:
    """A HODLRdD representation of K on the current CUDA device."""

    def __init__(self, points, kernel: int, params=None, leaf: int = 64, tol: float = 1e-8,
                 precision: str = "fp64", dense_if_cheaper: bool = True, max_nrhs: int = 8,
                 aca_max_rank: int = 1024, near_mode: int = 0, admissible_face_dim: int = 0,
                 lowrank_form: str = "factors", near_coords: str = "hilo", fp64_near: str = "fp64",
                 near_sms: int = 0):
        lib = load()
        if isinstance(points, np.ndarray):
            points = np.ascontiguousarray(points, dtype=np.float64)
        if points.ndim != 2:
            raise ValueError("points must be N x d")
        self.N, self.d = int(points.shape[0]), int(points.shape[1])
        self.device = _current_device()  # the library builds on the current device
        self.precision = precision
        self.io_dtype = np.float64 if precision == "fp64" else np.float32
        opt = Options()
        lib.hodlrdd_options_default(C.byref(opt))
        opt.precision = PREC[precision]
        # True / False, or "leaf": the rule at the leaf level only (coarser blocks keep their factors)
        opt.dense_if_cheaper = 2 if dense_if_cheaper == "leaf" else 1 if dense_if_cheaper else 0
        opt.max_nrhs = int(max_nrhs)
        opt.aca_max_rank = int(aca_max_rank)
        opt.near_mode = int(near_mode)
        opt.admissible_face_dim = int(admissible_face_dim)
        opt.lowrank_form = LOWRANK_FORM[lowrank_form]
        # "hilo": FP32 hi + lo coordinate pairs (exact distances); "hi": hi only
        opt.near_coords = NEAR_COORDS[near_coords]
        # FP64 handles: near field in FP64 ("fp64") or float-float on the FP32 pipes ("ff")
        opt.fp64_near = FP64_NEAR[fp64_near]
        # SMs given to the single-RHS FP32 near field (0: it shares every SM with the
        # applies; "auto" or -1: chosen by the build from timed products)
        opt.near_sms = -1 if near_sms == "auto" else int(near_sms)
        p = np.zeros(4, np.float64)
        p[0] = 1.0
        if params is not None:
            v = np.asarray(params, np.float64).reshape(-1)
            p[: min(4, v.size)] = v[:4]
        self.params = p
        addr, keep = _ptr(points)
        h = C.c_void_p()
        st = lib.hodlrdd_build_ex(addr, self.d, self.N, int(kernel), p.ctypes.data, int(leaf), float(tol),
                                  C.byref(opt), C.byref(h))
        _check(st, "hodlrdd_build")
        self._h = h
        self._lib = lib
        self.kernel = int(kernel)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.hodlrdd_destroy(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the product ---------------------------------------------------------------
    def _io(self, x, y):
        _check_io(x, "x", self.N, self.io_dtype, self.device)
        if y is not None:
            _check_io(y, "y", self.N, self.io_dtype, self.device, like=x)

    def matvec(self, x, y=None, stream=None):
        """y = K x. x: (N,) or (N, nrhs), numpy (host) or torch (host / CUDA)."""
        self._io(x, y)
        nrhs = 1 if x.ndim == 1 else int(x.shape[1])
        if y is None:
            if isinstance(x, np.ndarray):
                y = np.empty(x.shape, dtype=self.io_dtype)
            else:
                y = x.new_empty(x.shape)
        xa, kx = _ptr(x)
        ya, ky = _ptr(y)
        st = self._lib.hodlrdd_matvec(self._h, xa, ya, nrhs, _stream_ptr(stream))
        _check(st, "hodlrdd_matvec")
        return y

    def direct(self, x, y=None, stream=None):
        """y = K x by direct O(N^2) summation on the GPU (FP32; x a CUDA tensor, one column)."""
        _check_io(x, "x", self.N, np.float32, self.device)
        if x.ndim != 1 and int(x.shape[1]) != 1:
            raise ValueError("x: the direct sum takes one right-hand side")
        if y is not None:
            _check_io(y, "y", self.N, np.float32, self.device, like=x)
        if y is None:
            y = x.new_empty(x.shape)
        xa, kx = _ptr(x)
        ya, ky = _ptr(y)
        _check(self._lib.hodlrdd_direct(self._h, xa, ya, _stream_ptr(stream)), "hodlrdd_direct")
        return y

    def matvec_noalloc(self, x, y=None, stream=None):
        """y = K x through hodlrdd_matvec_noalloc: host buffers are staged in the
        library's fixed static device scratch, never in newly allocated memory."""
        self._io(x, y)
        nrhs = 1 if x.ndim == 1 else int(x.shape[1])
        if y is None:
            if isinstance(x, np.ndarray):
                y = np.empty(x.shape, dtype=self.io_dtype)
            else:
                y = x.new_empty(x.shape)
        xa, kx = _ptr(x)
        ya, ky = _ptr(y)
        st = self._lib.hodlrdd_matvec_noalloc(self._h, xa, ya, nrhs, _stream_ptr(stream))
        _check(st, "hodlrdd_matvec_noalloc")
        return y

    # -- statistics and introspection ----------------------------------------------
    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.hodlrdd_get_stats(self._h, C.byref(s)), "hodlrdd_get_stats")
        k = s.kappa
        out = {name: getattr(s, name) for name, _ in Stats._fields_ if not name.endswith("_level")}
        out["boxes_per_level"] = list(s.boxes_per_level[: k + 1])
        out["blocks_per_level"] = list(s.blocks_per_level[: k + 1])
        out["max_rank_per_level"] = list(s.max_rank_per_level[: k + 1])
        out["mean_rank_per_level"] = list(s.mean_rank_per_level[: k + 1])
        return out

    def sync(self):
        """Wait for the device; raise if a matvec kernel recorded a failed bounded wait."""
        _check(self._lib.hodlrdd_sync(self._h), "hodlrdd_sync")

    def set_profiling(self, on: bool):
        _check(self._lib.hodlrdd_set_profiling(self._h, 1 if on else 0), "hodlrdd_set_profiling")

    def profile(self) -> dict:
        """Accumulated stage times (ms) since profiling was enabled, and launch count."""
        ms = np.zeros(4, np.float64)
        chunks = C.c_int64()
        launches = C.c_int64()
        _check(self._lib.hodlrdd_get_profile(self._h, ms.ctypes.data, C.byref(chunks), C.byref(launches)),
               "hodlrdd_get_profile")
        return {"gather_ms": ms[0], "vapply_ms": ms[1], "uapply_ms": ms[2], "near_ms": ms[3],
                "chunks": chunks.value, "launches": launches.value}

    def tree(self):
        perm = np.zeros(self.N, np.int64)
        keys = np.zeros(self.N, np.uint64)
        _check(self._lib.hodlrdd_get_tree(self._h, perm.ctypes.data, keys.ctypes.data), "hodlrdd_get_tree")
        return perm, keys

    def cube(self):
        lo = np.zeros(self.d, np.float64)
        si = np.zeros(2, np.float64)
        _check(self._lib.hodlrdd_get_cube(self._h, lo.ctypes.data, si.ctypes.data), "hodlrdd_get_cube")
        return lo, float(si[0]), float(si[1])

    def level(self, l):
        nb = C.c_int64()
        _check(self._lib.hodlrdd_get_level(self._h, int(l), C.byref(nb), None, None), "hodlrdd_get_level")
        st = np.zeros(nb.value + 1, np.int64)
        bk = np.zeros(nb.value, np.uint64)
        _check(self._lib.hodlrdd_get_level(self._h, int(l), C.byref(nb), st.ctypes.data, bk.ctypes.data),
               "hodlrdd_get_level")
        return st, bk

    def il(self, l):
        nb = C.c_int64()
        self._lib.hodlrdd_get_level(self._h, int(l), C.byref(nb), None, None)
        nnz = C.c_int64()
        _check(self._lib.hodlrdd_get_il(self._h, int(l), C.byref(nnz), None, None), "hodlrdd_get_il")
        off = np.zeros(nb.value + 1, np.int64)
        idx = np.zeros(nnz.value, np.int64)
        _check(self._lib.hodlrdd_get_il(self._h, int(l), C.byref(nnz), off.ctypes.data, idx.ctypes.data),
               "hodlrdd_get_il")
        return off, idx

    def near(self):
        s = self.stats()
        nb = s["boxes_per_level"][s["kappa"]]
        nnz = C.c_int64()
        off = np.zeros(nb + 1, np.int64)
        idx = np.zeros(s["n_near"], np.int64)
        _check(self._lib.hodlrdd_get_near(self._h, C.byref(nnz), off.ctypes.data, idx.ctypes.data),
               "hodlrdd_get_near")
        return off, idx

    def blocks(self):
        """(n_blocks, 9) int64: level, target, source, I0, m, J0, n, rank, dense."""
        nb = self.stats()["n_blocks"]
        rec = np.zeros(max(nb, 1) * 9, np.int64)
        _check(self._lib.hodlrdd_get_blocks(self._h, rec.ctypes.data), "hodlrdd_get_blocks")
        return rec[: nb * 9].reshape(nb, 9)

    def pivots(self, b, rank):
        sig = np.zeros(max(rank, 1), np.int64)
        tau = np.zeros(max(rank, 1), np.int64)
        _check(self._lib.hodlrdd_get_pivots(self._h, int(b), sig.ctypes.data, tau.ctypes.data),
               "hodlrdd_get_pivots")
        return sig[:rank], tau[:rank]

    def factors(self, b, m, n, rank):
        U = np.zeros(max(m * rank, 1), np.float64)
        V = np.zeros(max(n * rank, 1), np.float64)
        _check(self._lib.hodlrdd_get_factors(self._h, int(b), U.ctypes.data, V.ctypes.data), "hodlrdd_get_factors")
        return U[: m * rank].reshape(rank, m).T, V[: n * rank].reshape(rank, n).T

    def debug_expire_wait(self, cycles: int = 2_000_000_000):
        """Run one bounded device wait that nothing completes (test of the timeout path)."""
        _check(self._lib.hodlrdd_debug_expire_wait(self._h, int(cycles)), "hodlrdd_debug_expire_wait")

    def import_factors(self, ranks, dense, U_all, V_all):
        r = np.ascontiguousarray(ranks, np.int32)
        dn = np.ascontiguousarray(dense, np.int32)
        U = np.ascontiguousarray(U_all, np.float64)
        V = np.ascontiguousarray(V_all, np.float64)
        _check(self._lib.hodlrdd_import_factors(self._h, r.ctypes.data, dn.ctypes.data, U.ctypes.data,
                                                V.ctypes.data), "hodlrdd_import_factors")


def solve(inner: "Handle", outer: "Handle", b, x=None, tol: float = 1e-10, inner_tol: float = 1e-5,
          restart: int = 50, max_inner_iters: int = 500, max_refine: int = 20, stream=None):
    """x with K x = b: GMRES on `inner` inside FP64 refinement with `outer`
    (b, x: CUDA float64 tensors, original order). Returns (x, stats)."""
    lib = load()
    o = SolveOptions()
    lib.hodlrdd_solve_options_default(C.byref(o))
    o.tol, o.inner_tol, o.restart = float(tol), float(inner_tol), int(restart)
    o.max_inner_iters, o.max_refine = int(max_inner_iters), int(max_refine)
    for name, a in (("b", b), ("x", x)):
        if a is None:
            continue
        if isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False):
            raise ValueError(f"{name}: the solve takes CUDA tensors")
        _check_io(a, name, inner.N, np.float64, inner.device, like=b if name == "x" else None)
        if a.ndim != 1 and int(a.shape[1]) != 1:
            raise ValueError(f"{name}: one right-hand side per solve")
    if x is None:
        x = b.new_empty(b.shape)
    st = SolveStats()
    ba, kb = _ptr(b)
    xa, kx = _ptr(x)
    _check(lib.hodlrdd_solve(inner._h, outer._h, ba, xa, C.byref(o), C.byref(st), _stream_ptr(stream)),
           "hodlrdd_solve")
    return x, {"refinements": st.refinements, "inner_iterations": st.inner_iterations, "residual": st.residual}


class Batch:
    """One request per handle, captured into a CUDA graph and replayed."""

    def __init__(self, handles, nrhs):
        lib = load()
        self._handles = list(handles)
        n = len(self._handles)
        hs = (C.c_void_p * n)(*[h._h for h in self._handles])
        nr = (C.c_int * n)(*[int(k) for k in nrhs])
        self.nrhs = [int(k) for k in nrhs]
        b = C.c_void_p()
        _check(lib.hodlrdd_batch_create(hs, nr, n, C.byref(b)), "hodlrdd_batch_create")
        self._b = b
        self._lib = lib

    def run(self, xs, ys=None, stream=None):
        """y_i = K_i x_i for every request; xs / ys: numpy or torch arrays."""
        n = len(self._handles)
        if len(xs) != n or (ys is not None and len(ys) != n):
            raise ValueError(f"one x (and y) per request: {n}")
        for i, (x, h) in enumerate(zip(xs, self._handles)):
            _check_io(x, f"xs[{i}]", h.N, h.io_dtype, h.device)
            if x.ndim == 2 and int(x.shape[1]) != self.nrhs[i] or x.ndim == 1 and self.nrhs[i] != 1:
                raise ValueError(f"xs[{i}]: {self.nrhs[i]} right-hand sides expected")
            if ys is not None:
                _check_io(ys[i], f"ys[{i}]", h.N, h.io_dtype, h.device, like=x)
        if ys is None:
            ys = [np.empty(x.shape, dtype=h.io_dtype) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
                  for x, h in zip(xs, self._handles)]
        keep = [_ptr(a) for a in list(xs) + list(ys)]
        xp = (C.c_void_p * n)(*[keep[i][0] for i in range(n)])
        yp = (C.c_void_p * n)(*[keep[n + i][0] for i in range(n)])
        _check(self._lib.hodlrdd_batch_run(self._b, xp, yp, _stream_ptr(stream)), "hodlrdd_batch_run")
        return ys

    def close(self):
        if getattr(self, "_b", None):
            self._lib.hodlrdd_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Forest:
    """Products over many FP16X2 trees merged into one launch per stage."""

    def __init__(self, handles, nrhs):
        lib = load()
        self._handles = list(handles)
        n = len(self._handles)
        hs = (C.c_void_p * n)(*[h._h for h in self._handles])
        nr = (C.c_int * n)(*[int(k) for k in nrhs])
        self.nrhs = [int(k) for k in nrhs]
        f = C.c_void_p()
        _check(lib.hodlrdd_forest_create(hs, nr, n, C.byref(f)), "hodlrdd_forest_create")
        self._f = f
        self._lib = lib

    def run(self, xs, ys=None, stream=None):
        """y_i = K_i x_i for every tree; xs / ys: FP32 numpy or torch arrays."""
        n = len(self._handles)
        if len(xs) != n or (ys is not None and len(ys) != n):
            raise ValueError(f"one x (and y) per tree: {n}")
        for i, (x, h) in enumerate(zip(xs, self._handles)):
            _check_io(x, f"xs[{i}]", h.N, h.io_dtype, h.device)
            if x.ndim == 2 and int(x.shape[1]) != self.nrhs[i] or x.ndim == 1 and self.nrhs[i] != 1:
                raise ValueError(f"xs[{i}]: {self.nrhs[i]} right-hand sides expected")
            if ys is not None:
                _check_io(ys[i], f"ys[{i}]", h.N, h.io_dtype, h.device, like=x)
        if ys is None:
            ys = [np.empty(x.shape, dtype=h.io_dtype) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
                  for x, h in zip(xs, self._handles)]
        keep = [_ptr(a) for a in list(xs) + list(ys)]
        xp = (C.c_void_p * n)(*[keep[i][0] for i in range(n)])
        yp = (C.c_void_p * n)(*[keep[n + i][0] for i in range(n)])
        _check(self._lib.hodlrdd_forest_run(self._f, xp, yp, _stream_ptr(stream)), "hodlrdd_forest_run")
        return ys

    def stats(self):
        out = (C.c_int64 * 7)()
        _check(self._lib.hodlrdd_forest_stats(self._f, out), "hodlrdd_forest_stats")
        keys = ("points", "plane_bytes", "panels", "near_passes", "launches_per_run", "tuned_fixed_v",
                "tuned_fixed_u")
        return {k: int(v) for k, v in zip(keys, out)}

    def profile(self):
        """Stage times (ms) of one extra run on the last run's inputs."""
        ms = np.zeros(5, np.float64)
        _check(self._lib.hodlrdd_forest_profile(self._f, ms.ctypes.data), "hodlrdd_forest_profile")
        return dict(zip(("gather_ms", "vapply_ms", "uapply_ms", "near_ms", "run_ms"), (float(v) for v in ms)))

    def close(self):
        if getattr(self, "_f", None):
            self._lib.hodlrdd_forest_destroy(self._f)
            self._f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


REQ_MATVEC, REQ_SOLVE = 0, 1


class Server:
    """Request loop over models kept resident under a device-memory budget."""

    def __init__(self, budget_bytes: int, workers: int = 4):
        lib = load()
        s = C.c_void_p()
        _check(lib.hodlrdd_server_create(int(budget_bytes), int(workers), C.byref(s)), "hodlrdd_server_create")
        self._s = s
        self._lib = lib
        self._keep = {}
        self._models = []

    def add(self, points, kernel: int, params=None, leaf: int = 64, tol: float = 1e-8, precision: str = "fp32",
            **options) -> int:
        """Register a model (host points, N x d); returns its id."""
        pts = np.ascontiguousarray(points, dtype=np.float64)
        opt = Options()
        self._lib.hodlrdd_options_default(C.byref(opt))
        opt.precision = PREC[precision]
        for k, v in options.items():
            setattr(opt, k, LOWRANK_FORM[v] if k == "lowrank_form" else int(v))
        p = np.zeros(4, np.float64)
        p[0] = 1.0
        if params is not None:
            v = np.asarray(params, np.float64).reshape(-1)
            p[: min(4, v.size)] = v[:4]
        mid = C.c_int64()
        _check(self._lib.hodlrdd_server_add(self._s, pts.ctypes.data, pts.shape[1], pts.shape[0], int(kernel),
                                            p.ctypes.data, int(leaf), float(tol), C.byref(opt), C.byref(mid)),
               "hodlrdd_server_add")
        self._models.append((pts.shape[0], np.float64 if precision == "fp64" else np.float32))
        return mid.value

    def submit(self, model: int, x, kind: int = REQ_MATVEC, y=None) -> int:
        """Queue y = K x (kind REQ_MATVEC) or K u = b (REQ_SOLVE, FP64 host arrays)."""
        if not 0 <= model < len(self._models):
            raise HodlrddError(ERR_INVALID, "hodlrdd_server_submit", "unknown model")
        N, io = self._models[model]
        if kind == REQ_SOLVE:
            if not isinstance(x, np.ndarray) or (y is not None and not isinstance(y, np.ndarray)):
                raise ValueError("a solve request takes host (numpy) arrays")
            x = np.ascontiguousarray(x, dtype=np.float64)
            io = np.float64
        _check_io(x, "x", N, io, _current_device())
        if y is not None:
            _check_io(y, "y", N, io, _current_device(), like=x)
        if y is None:
            y = np.empty(x.shape, dtype=io) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        nrhs = 1 if x.ndim == 1 else int(x.shape[1])
        xa, kx = _ptr(x)
        ya, ky = _ptr(y)
        rid = C.c_int64()
        _check(self._lib.hodlrdd_server_submit(self._s, int(model), int(kind), xa, ya, nrhs, C.byref(rid)),
               "hodlrdd_server_submit")
        self._keep[rid.value] = (kx, ky)
        return rid.value

    def wait(self, request: int, service: bool = False):
        """(result, latency in ms) of a request; with service=True also the
        start-to-done time: (result, latency, service)."""
        lat = (C.c_double * 2)()
        st = self._lib.hodlrdd_server_wait(self._s, int(request), lat)
        kx, ky = self._keep.pop(request, (None, None))
        _check(st, "hodlrdd_server_wait")
        return (ky, lat[0], lat[1]) if service else (ky, lat[0])

    def stats(self) -> dict:
        out = np.zeros(5, np.int64)
        _check(self._lib.hodlrdd_server_stats(self._s, out.ctypes.data), "hodlrdd_server_stats")
        b = (C.c_int64 * 2)()
        _check(self._lib.hodlrdd_server_batch_stats(self._s, b), "hodlrdd_server_batch_stats")
        return {"resident_bytes": int(out[0]), "resident_models": int(out[1]), "builds": int(out[2]),
                "evictions": int(out[3]), "queued": int(out[4]), "batches": int(b[0]), "batched_requests": int(b[1])}

    def set_batching(self, max_cols: int):
        """Columns of one batched product (0 or 1: products of a model run alone)."""
        _check(self._lib.hodlrdd_server_set_batching(self._s, int(max_cols)), "hodlrdd_server_set_batching")

    def close(self):
        if getattr(self, "_s", None):
            self._lib.hodlrdd_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_peaks(stream=None) -> dict:
    """Measured arithmetic throughput of the current device (hodlrdd_probe_peaks)."""
    out = np.zeros(4, np.float64)
    _check(load().hodlrdd_probe_peaks(out.ctypes.data, 4, _stream_ptr(stream)), "hodlrdd_probe_peaks")
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "mufu_rsqrt_gops": float(out[2]),
            "mufu_ex2_gops": float(out[3])}


def debug_fail_alloc_after(k: int):
    load().hodlrdd_debug_fail_alloc_after(int(k))


def debug_ff_eval(kernel: int, params, h: float, s) -> np.ndarray:
    """Kernel values F(s) in the float-float arithmetic of the FP64 near field
    with fp64_near "ff", at box size h (hodlrdd_debug_ff_eval)."""
    p = np.zeros(4, np.float64)
    v = np.asarray(params, np.float64).reshape(-1)
    p[: min(4, v.size)] = v[:4]
    sa = np.ascontiguousarray(s, np.float64).reshape(-1)
    out = np.empty_like(sa)
    _check(load().hodlrdd_debug_ff_eval(int(kernel), p.ctypes.data, float(h), sa.ctypes.data, out.ctypes.data,
                                        int(sa.size)), "hodlrdd_debug_ff_eval")
    return out


def debug_aca_pool_bytes(nbytes: int):
    """Cap the ACA's one-pass factor pool (bytes; -1: default, 0: two passes)."""
    load().hodlrdd_debug_aca_pool_bytes(int(nbytes))
