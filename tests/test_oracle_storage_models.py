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
import pytest

import storage_model as SM
import workloads as W

ETA = SM.ETA
THETA = 2.0 ** -23


def relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def round_cols(M, kind):
    """Each column rounded as the GPU stores it (storage_model.round_col)."""
    out = np.empty_like(M)
    for k in range(M.shape[1]):
        out[:, k] = SM.round_col(M[:, k], kind)
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
        Um = np.hstack([round_cols(U[:, :kb], "fp32"), round_cols(U[:, kb:], "fp16")])
        Vm = np.hstack([round_cols(V[:, :kb], "fp32"), round_cols(V[:, kb:], "fp16")])
        assert kb == SM.head_terms(U, V)
        ymix[I0:I0 + m] += Um @ (Vm.T @ xs)
        y16[I0:I0 + m] += round_cols(U, "fp16") @ (round_cols(V, "fp16").T @ xs)
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


def test_rounding_rules_pinned():
    """The model's rounding against values fixed by the formats: a power-of-two
    scale puts the column's largest entry in [1/2, 1); FP16 keeps 11 significant
    bits, BF16 8 (ties to even), FP32 24."""
    col = np.array([3.0, -0.75, 1.0 + 2.0 ** -12, 1.0 + 3 * 2.0 ** -9, 2.0 ** -30])
    assert SM.pow2_scale(col) == 4.0
    assert SM.pow2_scale(np.array([1.0])) == 2.0
    assert SM.pow2_scale(np.zeros(3)) == 1.0
    f16 = SM.round_col(col, "fp16")
    assert f16[0] == 3.0 and f16[1] == -0.75
    assert f16[2] == 1.0  # 1 + 2^-12 is below half an FP16 ulp of 1 (2^-10 at scale 4: 2^-11 relative)
    bf = SM.round_col(col, "bf16")
    # at scale 4, 1 + 3 * 2^-9 becomes 0.25 + 3 * 2^-11; BF16 spacing in [1/4, 1/2) is
    # 2^-9, so 0.75 of a spacing rounds up to 0.25 + 2^-9 (times 4: 1 + 2^-7)
    assert bf[3] == 1.0 + 2.0 ** -7
    assert bf[0] == 3.0 and f16[4] == 0.0  # 2^-32 at scale 4 is below FP16's smallest subnormal
    assert SM.round_col(np.array([1.0 + 2.0 ** -30]), "fp32")[0] == 1.0
    assert SM.to_bf16(np.array([1.0 + 2.0 ** -8], np.float32))[0] == 1.0  # tie to even
    assert SM.to_bf16(np.array([1.0 + 3 * 2.0 ** -8], np.float32))[0] == 1.0 + 2.0 ** -6


@pytest.mark.parametrize("precision,lo,hi", [("fp64", 0.0, 1e-15), ("fp32", 1e-10, 1e-7), ("fp32+fp16", 1e-10, 2e-7),
                                             ("fp16", 1e-6, 2e-3), ("bf16", 1e-5, 1.5e-2)])
def test_storage_product_error_sizes(oracle_mod, precision, lo, hi):
    """storage_product: the oracle's product with the factors rounded as the GPU
    stores them; its error against the FP64 product sits in the band the
    format's unit roundoff sets (FP64 reproduces it)."""
    w = W.make("t", 3, 5000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=2, seed=33)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 32, 1e-8, dense_if_cheaper=True)
    y = T.matvec(w.x)
    e = relerr(SM.storage_product(T, w.x, precision), y)
    assert lo <= e <= hi, e
