"""GB300-native HODLRdD: hierarchical kernel-matrix products on one GPU.

Public API (a thin ctypes layer over include/hodlrdd.h; every step runs in the
CUDA library, there is no CPU fallback):

    Handle(points, kernel, params, leaf, tol, precision=...)   build (Algorithm 1)
    Handle.matvec(x)                                            y = K x (Algorithm 2)
    Handle.stats()                                              ranks, sizes, phase times
    solve(inner, outer, b)                                      GMRES with FP64 refinement
    Batch(handles, nrhs).run(xs)                                graph-replayed batch of products
    Forest(handles, nrhs).run(xs)                               FP16X2 trees merged, one launch per stage
    Server(budget).add / submit / wait                          request loop under an HBM budget
    probe_peaks()                                               measured FP32 / FP64 / MUFU throughput
"""
from ._binding import (  # noqa: F401
    Batch,
    ERR_CUDA,
    ERR_INVALID,
    ERR_NUMERIC,
    ERR_OOM,
    ERR_TIMEOUT,
    ERR_UNSUPPORTED,
    Forest,
    OK,
    PREC,
    REQ_MATVEC,
    REQ_SOLVE,
    Handle,
    Server,
    HodlrddError,
    header_functions,
    load,
    probe_peaks,
    solve,
)

K_LOG, K_INV_R, K_MATERN32, K_GAUSS, K_EXP, K_INV_R2_4D, K_R, K_SIN, K_INV_SQRT1P = range(9)
