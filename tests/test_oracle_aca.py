"""Pins for the oracle's partial-pivoted ACA (no GPU).

The ACA compresses each IL block as K(I,J) ~ K(I,tau) K(sigma,tau)^-1 K(sigma,J)
(Eq. keq1), with the LU factors of K(sigma,tau) a by-product (Eq. keq2). Pinned by
exact low rank, the skeleton identity, the SVD, and the structure pivoting
implies.
"""
import numpy as np
import pytest

import workloads as W


def test_exact_low_rank(oracle_mod):
    rng = np.random.default_rng(0)
    for r in (1, 3, 7):
        A = rng.standard_normal((60, r)) @ rng.standard_normal((r, 45))
        p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, 1e-10)
        assert r <= p <= r + 1  # the term that meets the tolerance is kept
        assert np.linalg.norm(A - U @ V.T) <= 1e-13 * np.linalg.norm(A)


def test_separable_kernel(oracle_mod):
    # (1 + x.y)^2 in d dims has rank (d+1)(d+2)/2; built from the kernel-free points.
    rng = np.random.default_rng(1)
    d = 3
    X = rng.uniform(-1, 1, (50, d))
    Y = rng.uniform(-1, 1, (40, d))
    A = (1.0 + X @ Y.T) ** 2
    p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, 1e-12)
    assert p in ((d + 1) * (d + 2) // 2, (d + 1) * (d + 2) // 2 + 1)
    assert np.linalg.norm(A - U @ V.T) <= 1e-12 * np.linalg.norm(A)


def test_1d_closed_form_ranks(oracle_mod):
    # Far-field intervals: exp(-r) has rank 1, r and sin r rank 2 (exact closed forms).
    Y = W.grid_points(200, 1)
    X = W.grid_points(200, 1, 1.0, [-2.0])
    for kern, params, r in ((W.K_EXP, (1, 0, 1.0, 0), 1), (W.K_R, None, 2), (W.K_SIN, None, 2)):
        A = oracle_mod.kernel_block(X, Y, kern, params)
        p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, 1e-12)
        assert r <= p <= r + 1
        assert np.linalg.norm(A - U @ V.T) <= 1e-14 * np.linalg.norm(A)


def test_pivot_structure_and_skeleton(oracle_mod):
    Y = W.grid_points(12, 2)
    X = W.grid_points(12, 2, 1.0, [-1.0, -1.0])  # vertex-sharing squares
    A = oracle_mod.kernel_block(X, Y, W.K_LOG)
    p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, 1e-9)
    assert p >= 3
    # first pivot: row 0, column of the largest |A(0, j)| (lowest index on ties)
    assert sig[0] == 0
    assert tau[0] == int(np.flatnonzero(np.abs(A[0]) == np.abs(A[0]).max())[0])
    assert len(set(sig)) == p and len(set(tau)) == p
    # v_q(tau_q) = 1 and |v_q| <= 1 (row normalised by its largest entry)
    assert np.allclose(V[tau, np.arange(p)], 1.0)
    assert np.abs(V).max() <= 1.0 + 1e-15
    # L(l, q) = u_q(sigma_l) is lower triangular, U(q, l) = v_q(tau_l) unit upper triangular
    L = U[sig, :]
    Ut = V[tau, :].T
    assert np.allclose(np.triu(L, 1), 0.0, atol=1e-14 * np.abs(A).max())
    # below the diagonal v_q(tau_l) is a rounding-level residual divided by the pivot u_q(sigma_q)
    assert np.abs(np.tril(Ut, -1) * np.diag(L)[:, None]).max() <= 1e-14 * np.abs(A).max()
    # K(sigma, tau) = L U, and U V^T = K(:, tau) K(sigma, tau)^-1 K(sigma, :) (Eq. keq1/keq2)
    M = A[np.ix_(sig, tau)]
    assert np.allclose(L @ Ut, M, rtol=0, atol=1e-13 * np.abs(A).max())
    skel = A[:, tau] @ np.linalg.solve(M, A[sig, :])
    assert np.linalg.norm(skel - U @ V.T) <= 1e-11 * np.linalg.norm(A)
    # second pivot row: largest |u_0| among rows not used yet
    u0 = np.abs(U[:, 0]).copy()
    u0[sig[0]] = -1
    assert sig[1] == int(np.argmax(u0))


def test_error_against_svd(oracle_mod):
    Y = W.grid_points(20, 2)
    X = W.grid_points(20, 2, 1.0, [-2.0, 0.0])  # far-field squares
    A = oracle_mod.kernel_block(X, Y, W.K_INV_R)
    s = np.linalg.svd(A, compute_uv=False)
    for tol in (1e-4, 1e-8, 1e-12):
        p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, tol)
        err = np.linalg.norm(A - U @ V.T) / np.linalg.norm(A)
        assert err <= 10 * tol
        # no rank-p matrix beats the truncated SVD: ACA's error >= the SVD tail
        assert err >= np.sqrt((s[p:] ** 2).sum()) / np.linalg.norm(s) * (1 - 1e-6)


def test_zero_rows_skipped(oracle_mod):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((10, 3)) @ rng.standard_normal((3, 8))
    A[0] = 0.0
    A[4] = 0.0
    p, dense, sig, tau, U, V = oracle_mod.aca_dense(A, 1e-12)
    assert sig[0] == 1
    assert 0 not in sig and 4 not in sig
    assert np.linalg.norm(A - U @ V.T) <= 1e-13 * np.linalg.norm(A)
    Z = np.zeros((5, 4))
    p, dense, sig, tau, U, V = oracle_mod.aca_dense(Z, 1e-8)
    assert p == 0


def test_dense_if_cheaper(oracle_mod):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((8, 8))
    p, dense, *_ = oracle_mod.aca_dense(A, 1e-12, flags=oracle_mod.FLAG_DENSE_IF_CHEAPER)
    assert dense == 1 and p == 0
    p, dense, *_ = oracle_mod.aca_dense(A, 1e-12)
    assert dense == 0 and p == 8
    B = rng.standard_normal((40, 2)) @ rng.standard_normal((2, 40))
    p, dense, *_ = oracle_mod.aca_dense(B, 1e-12, flags=oracle_mod.FLAG_DENSE_IF_CHEAPER)
    assert dense == 0 and p in (2, 3)
