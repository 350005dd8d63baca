"""CPU model of the GPU path's factor storage, applied to the oracle's own ACA
factors (test infrastructure, numpy only, no CUDA).

The GPU stores each low-rank block's factors U_b (m x p) and V_b (n x p) in
the handle's precision: FP64 and FP32 by plain rounding; FP16 and BF16 per
column, divided by a power of two 2^e with 2^(e-1) <= max |entry| < 2^e, rounded
through FP32 to the 16-bit type; the mixed FP32 / FP16 storage keeps a block's
leading terms in FP32 and its terms after the last one with
||u_k|| ||v_k|| > 2^-13 (sum_k ||u_k||^2 ||v_k||^2)^(1/2) in scaled FP16. The
model rounds the oracle's factors by the same rules, so the GPU product on
imported oracle factors differs from the model's FP64 product of the rounded
factors only by the GPU's own FP32 arithmetic.
"""
import numpy as np

ETA = 2.0 ** -13


def pow2_scale(col):
    mx = float(np.abs(col).max()) if col.size else 0.0
    if mx == 0.0:
        return 1.0
    _, e = np.frexp(mx)
    return float(2.0 ** int(e))


def to_bf16(a32):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP64."""
    b = np.ascontiguousarray(a32, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def round_col(col, kind):
    if kind == "fp64":
        return col.copy()
    if kind == "fp32":
        return col.astype(np.float32).astype(np.float64)
    s = pow2_scale(col)
    v32 = (col / s).astype(np.float32)
    if kind == "fp16":
        return v32.astype(np.float16).astype(np.float64) * s
    if kind == "bf16":
        return to_bf16(v32) * s
    raise ValueError(kind)


def head_terms(U, V):
    """Number of leading terms the mixed storage keeps in FP32."""
    tn = np.linalg.norm(U, axis=0) * np.linalg.norm(V, axis=0)
    S = np.sqrt((tn ** 2).sum())
    kb = U.shape[1]
    while kb > 0 and tn[kb - 1] <= ETA * S:
        kb -= 1
    return kb


def stored(U, V, precision):
    """(U, V) as the GPU stores them in `precision` ("fp64", "fp32", "fp16",
    "bf16", "fp32+fp16"), values in FP64."""
    p = U.shape[1]
    if precision == "fp32+fp16":
        kb = head_terms(U, V)
        kinds = ["fp32"] * kb + ["fp16"] * (p - kb)
    else:
        kinds = [precision] * p
    Us = np.empty_like(U)
    Vs = np.empty_like(V)
    for k in range(p):
        Us[:, k] = round_col(U[:, k], kinds[k])
        Vs[:, k] = round_col(V[:, k], kinds[k])
    return Us, Vs


def storage_product(T, x, precision):
    """The oracle's HODLRdD product with every low-rank block's factors as the
    GPU stores them in `precision`: T.matvec(x) + sum_b (Us Vs^T - U V^T) x(J_b).
    x: (N, nrhs) in original order; returns (N, nrhs) in original order."""
    x = np.asarray(x, np.float64).reshape(T.N, -1)
    perm = T.perm()[0]
    xt = x[perm]
    dy = np.zeros_like(xt)
    rec = T.blocks()
    for b in range(len(rec)):
        I0, m, J0, n, p, dn = (int(v) for v in (rec[b, 3], rec[b, 4], rec[b, 5], rec[b, 6], rec[b, 7], rec[b, 8]))
        if dn or p == 0:
            continue
        _, _, U, V = T.factors(b)
        Us, Vs = stored(U, V, precision)
        xs = xt[J0:J0 + n]
        dy[I0:I0 + m] += Us @ (Vs.T @ xs) - U @ (V.T @ xs)
    y = T.matvec(x)
    y[perm] += dy
    return y
