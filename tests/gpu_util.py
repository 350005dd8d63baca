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


# kernels whose FP64 entries use only correctly rounded operations (sqrt,
# division), so the GPU ACA reproduces the oracle's pivots on every block;
# log, exp and sin come from different libraries on the two sides and can
# flip a near-tie pivot in about one block in a hundred
EXACT_KERNELS = (1, 5, 6, 8)  # 1/r, -1/(4 pi^2 r^2), r, 1/sqrt(1 + r)


def pivot_mismatches(T, h):
    """Blocks whose rank, dense flag or ACA pivots differ between the oracle
    tree T and the GPU handle h (same block structure asserted)."""
    bo, bg = T.blocks(), h.blocks()
    assert np.array_equal(bo[:, :7], bg[:, :7])
    out = []
    for b in range(len(bo)):
        ro, rg = int(bo[b, 7]), int(bg[b, 7])
        if ro != rg or bo[b, 8] != bg[b, 8]:
            out.append(b)
            continue
        if ro == 0:
            continue
        so, to, _, _ = T.factors(b)
        sg, tg = h.pivots(b, rg)
        if not (np.array_equal(so, sg) and np.array_equal(to, tg)):
            out.append(b)
    return out


def min_pivot_agreement(kernel, d, tol):
    """Fraction of blocks whose ACA pivots must agree with the oracle's: every
    block for the correctly rounded kernels; 99% where log / exp / sin differ by
    an ulp between the libraries; 95% for the 1-D exp(-r) kernel at tol <= 1e-10,
    which is separable between separated intervals, so that its trailing ACA
    pivots are rounding-level residuals and ulp differences reorder near-ties."""
    if kernel in EXACT_KERNELS:
        return 1.0
    if kernel == 4 and d == 1 and tol <= 1e-10:
        return 0.95
    return 0.99


def assert_matches_oracle_hodlrdd(oracle, T, h, w, yg, tol, kernel, skeleton=False, base=1e-10, aca_factor=10.0):
    """The GPU FP64 product yg against the oracle's HODLRdD product, with no
    branch that skips the comparison.

    Blocks where the GPU's ACA took the oracle's pivots give the same factors
    (to rounding), so with every pivot agreeing the products agree to `base`.
    Where a pivot differs (ulp-level differences between CUDA's and the host's
    log / exp / sin flipping a near-tie), both factorisations still approximate
    the exact block A_b = K(I, J), so the products may differ by at most
        sum_b ||(A_b - O_b) x(J)|| + aca_factor tol ||A_b||_F ||x(J)||,
    the oracle's own error on that block (computed) plus the GPU's, whose size
    is asserted per block against the exact entries. Asserted: the fraction of
    agreeing blocks (min_pivot_agreement),
    the GPU's per-block error on the others, and the product bound per column."""
    mism = pivot_mismatches(T, h)
    nb = max(len(T.blocks()), 1)
    frac = 1.0 - len(mism) / nb
    assert frac >= min_pivot_agreement(kernel, w.d, tol), (frac, mism[:10])
    bo = T.blocks()
    perm = T.perm()[0]
    P = w.points[perm]
    xt = np.asarray(w.x, np.float64).reshape(w.N, -1)[perm]
    yo = T.matvec(w.x)
    slack = np.zeros(xt.shape[1])
    for b in mism:
        I0, m, J0, n = (int(v) for v in bo[b, 3:7])
        A = oracle.kernel_block(P[I0:I0 + m], P[J0:J0 + n], w.kernel, w.params)
        xs = xt[J0:J0 + n]
        An = np.linalg.norm(A)
        ro = int(bo[b, 7])
        if bo[b, 8] or ro == 0:
            eo = np.zeros(xs.shape[1])
        else:
            _, _, Uo, Vo = T.factors(b)
            eo = np.linalg.norm(A @ xs - Uo @ (Vo.T @ xs), axis=0)
        rg = int(h.blocks()[b, 7])
        if not h.blocks()[b, 8] and rg > 0:
            if skeleton:
                sg, tg = h.pivots(b, rg)
                G = A[:, tg] @ np.linalg.solve(A[np.ix_(sg, tg)], A[sg, :])
            else:
                Ug, Vg = h.factors(b, m, n, rg)
                G = Ug @ Vg.T
            assert np.linalg.norm(A - G) <= aca_factor * tol * An, b
        slack += eo + aca_factor * tol * An * np.linalg.norm(xs, axis=0)
    diff = np.linalg.norm(np.asarray(yg, np.float64).reshape(w.N, -1) - yo, axis=0)
    bound = base * np.linalg.norm(yo, axis=0) + slack
    assert np.all(diff <= bound), (diff / np.linalg.norm(yo, axis=0), len(mism))
    return frac, float(np.max(diff / np.linalg.norm(yo, axis=0)))
