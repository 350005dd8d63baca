"""CPU models of two storage rules of the GPU path, on the oracle's own ACA
factors, checked against the oracle's FP64 product. They pin the arithmetic the
rules rely on, independently of the GPU kernels:

* mixed FP32 / FP16 storage: each block's terms after the last one with
  ||u_k|| ||v_k|| > 2^-13 ||A_b||_F are rounded to FP16 (with a power-of-two
  scale per column), the others to FP32; the product stays within the FP32
  bound of the FP64 product, while rounding every term to FP16 does not;
* FP32 skeleton form: with FP32-sized errors in the entries of K(sigma, J) and
  K(I, tau), the skeleton product K(I, tau) U^-1 L^-1 K(sigma, J) x blows up
  for blocks with tiny trailing pivots, and keeping only the terms whose pivot
  is at least 2^-23 of the largest before it brings it back to FP32 size.
"""
import numpy as np

import workloads as W

ETA = 2.0 ** -13
THETA = 2.0 ** -23


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def round_cols(M, dtype):
    """Each column scaled by a power of two >= its largest entry, rounded to dtype, scaled back."""
    out = np.empty_like(M)
    for k in range(M.shape[1]):
        mx = np.abs(M[:, k]).max()
        s = 2.0 ** np.ceil(np.log2(mx)) if mx > 0 else 1.0
        out[:, k] = (M[:, k] / s).astype(dtype).astype(np.float64) * s
    return out


def blocks_with_factors(T):
    rec = T.blocks()
    for b in range(len(rec)):
        l, ti, sj, I0, m, J0, n, p, dn = [int(v) for v in rec[b][:9]]
        if p > 0 and not dn:
            sig, tau, U, V = T.factors(b)
            yield I0, m, J0, n, p, sig, tau, U, V


def test_mixed_fp32_fp16_storage_rule(oracle_mod):
    w = W.make("t", 3, 6000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=31)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 32, 1e-8, dense_if_cheaper=True)
    perm = T.perm()[0]
    x = w.x[perm, 0]
    y64 = np.zeros(w.N)
    ymix = np.zeros(w.N)
    y16 = np.zeros(w.N)
    tail = total = 0
    for I0, m, J0, n, p, sig, tau, U, V in blocks_with_factors(T):
        tn = np.linalg.norm(U, axis=0) * np.linalg.norm(V, axis=0)
        S = np.sqrt((tn ** 2).sum())
        kb = p
        while kb > 0 and tn[kb - 1] <= ETA * S:
            kb -= 1
        tail += (p - kb) * (m + n)
        total += p * (m + n)
        xs = x[J0:J0 + n]
        y64[I0:I0 + m] += U @ (V.T @ xs)
        Um = np.hstack([round_cols(U[:, :kb], np.float32), round_cols(U[:, kb:], np.float16)])
        Vm = np.hstack([round_cols(V[:, :kb], np.float32), round_cols(V[:, kb:], np.float16)])
        ymix[I0:I0 + m] += Um @ (Vm.T @ xs)
        y16[I0:I0 + m] += round_cols(U, np.float16) @ (round_cols(V, np.float16).T @ xs)
    assert 0.2 < tail / total < 0.95  # a large share of the entries goes to two bytes
    assert relerr(ymix, y64) <= 2e-7  # the low-rank part keeps FP32-sized rounding
    assert relerr(y16, y64) > 10 * relerr(ymix, y64)  # all-FP16 storage does not


def test_fp32_skeleton_truncation_rule(oracle_mod):
    # 1-D exp(-r): separable between separated intervals, so ACA's trailing
    # pivots are at rounding level
    w = W.make("t", 1, 3001, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-10, nrhs=1, seed=3012)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 16, 1e-10, dense_if_cheaper=True)
    perm = T.perm()[0]
    P = w.points[perm]
    x = w.x[perm, 0]
    rng = np.random.default_rng(1)
    eps = 2.0 ** -23
    y64 = np.zeros(w.N)
    yfull = np.zeros(w.N)
    ytrunc = np.zeros(w.N)
    for I0, m, J0, n, p, sig, tau, U, V in blocks_with_factors(T):
        Ks = oracle_mod.kernel_block(P[I0 + sig], P[J0:J0 + n], w.kernel, w.params)
        Kt = oracle_mod.kernel_block(P[I0:I0 + m], P[J0 + tau], w.kernel, w.params)
        Ks = Ks * (1 + eps * rng.uniform(-1, 1, Ks.shape))  # FP32-sized entry errors
        Kt = Kt * (1 + eps * rng.uniform(-1, 1, Kt.shape))
        xs = x[J0:J0 + n]
        y64[I0:I0 + m] += U @ (V.T @ xs)
        piv = np.abs(U[sig, np.arange(p)])
        keep = p
        for q in range(p):
            if not piv[q] >= THETA * piv[: q + 1].max():
                keep = q
                break

        def skeleton(k):
            L = U[sig[:k], :k]             # L(l, q) = u_q(sigma_l)
            Uu = V[tau[:k], :k].T          # U(q, l) = v_q(tau_l)
            w_ = np.linalg.solve(Uu, np.linalg.solve(L, Ks[:k] @ xs))
            return Kt[:, :k] @ w_

        yfull[I0:I0 + m] += skeleton(p)
        if keep > 0:
            ytrunc[I0:I0 + m] += skeleton(keep)
    assert relerr(yfull, y64) > 1e-3     # tiny trailing pivots amplify the entry errors
    assert relerr(ytrunc, y64) <= 2e-6   # the truncated skeleton stays FP32-sized
