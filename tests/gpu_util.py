"""Helpers shared by the GPU tests: device fixtures and oracle comparisons."""
import numpy as np
import pytest


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_05819_gb300 import build

    build.build()
    return torch


def relerr(a, b):
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def gpu_handle(hd, w, **kw):
    import torch

    return hd.Handle(torch.from_numpy(w.points).cuda(), w.kernel, w.params, w.leaf, w.tol, **kw)


def gpu_matvec(h, x, dtype=None):
    import torch

    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=dtype or h.io_dtype)).cuda()
    y = h.matvec(xt)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def oracle_factors(T):
    """Per-block ranks, dense flags and concatenated U, V of an oracle tree."""
    rec = T.blocks()
    ranks = rec[:, 7].astype(np.int32)
    dense = rec[:, 8].astype(np.int32)
    Us, Vs = [], []
    for b in range(len(rec)):
        if ranks[b] > 0:
            _, _, U, V = T.factors(b)
            Us.append(U.T.reshape(-1))  # column-major m x p
            Vs.append(V.T.reshape(-1))
    U_all = np.concatenate(Us) if Us else np.zeros(1)
    V_all = np.concatenate(Vs) if Vs else np.zeros(1)
    return ranks, dense, U_all, V_all
