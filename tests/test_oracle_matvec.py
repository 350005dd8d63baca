"""Pins for the oracle's HODLRdD matvec (Algorithm 2) against the exact product.

The direct O(N^2) sum is the definition of y = K x. HODLRdD approximates it with
ACA tolerance tol: the relative 2-norm error (the paper's error measure) must be
at most 10 tol, and tol = 1e-14 must reproduce the direct sum to 1e-12.
"""
import numpy as np
import pytest

import workloads as W

CASES = [
    (1, 2000, W.K_LOG, None, 16),
    (2, 2000, W.K_LOG, None, 32),
    (3, 2000, W.K_INV_R, None, 32),
    (4, 2000, W.K_LOG, None, 40),
    (2, 1500, W.K_MATERN32, (1, 0, 0.2, 0), 32),
    (3, 1500, W.K_GAUSS, (1, 1e-3, 0.5, 0), 24),
    (3, 1500, W.K_EXP, (1, 0, 1.0, 0), 24),
    (4, 1500, W.K_INV_R2_4D, None, 24),
    (2, 1500, W.K_R, None, 32),
    (2, 1500, W.K_SIN, None, 32),
    (3, 1500, W.K_INV_SQRT1P, None, 32),
]


def relerr(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("d,N,kern,params,leaf", CASES)
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_matvec_error_bound(oracle_mod, d, N, kern, params, leaf, tol):
    w = W.make("t", d, N, kern, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=d + N)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, leaf, tol)
    assert T.kappa >= 1
    y = T.matvec(w.x)
    yd = oracle_mod.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(y, yd) <= 10 * tol


@pytest.mark.parametrize("d", [2, 3])
def test_tight_tolerance_reproduces_direct(oracle_mod, d):
    w = W.make("t", d, 1800, W.K_LOG if d == 2 else W.K_INV_R, leaf=24, tol=1e-14, seed=4)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 24, 1e-14)
    assert relerr(T.matvec(w.x), oracle_mod.direct(w.points, w.kernel, w.params, w.x)) <= 1e-12


def test_skeleton_form_matches_stored_factors(oracle_mod):
    w = W.make("t", 3, 1500, W.K_INV_R, leaf=24, tol=1e-8, nrhs=2, seed=9)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 24, 1e-8)
    assert relerr(T.matvec(w.x, skeleton=True), T.matvec(w.x)) <= 1e-12


def test_dense_if_cheaper_only_helps(oracle_mod):
    w = W.make("t", 3, 2000, W.K_INV_R, leaf=16, tol=1e-6, seed=12)
    yd = oracle_mod.direct(w.points, w.kernel, w.params, w.x)
    T0 = oracle_mod.Tree(w.points, w.kernel, w.params, 16, 1e-6)
    T1 = oracle_mod.Tree(w.points, w.kernel, w.params, 16, 1e-6, dense_if_cheaper=True)
    assert T1.n_dense > 0
    assert T1.factor_elems < T0.factor_elems
    assert relerr(T1.matvec(w.x), yd) <= 10 * 1e-6


def test_single_leaf_is_exact(oracle_mod):
    w = W.make("t", 3, 50, W.K_INV_R, leaf=64, seed=1)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 64, 1e-8)
    assert T.kappa == 0 and T.nblocks == 0
    assert relerr(T.matvec(w.x), oracle_mod.direct(w.points, w.kernel, w.params, w.x)) <= 1e-15


def test_identity_shift_and_columns(oracle_mod):
    # (I + K/N) x: diag = 1 adds x exactly once; columns are independent.
    N = 1200
    w = W.make("t", 3, N, W.K_INV_R, (1.0 / N, 1.0, 0, 0), 32, 1e-9, nrhs=3, seed=2)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, 32, 1e-9)
    y = T.matvec(w.x)
    T0 = oracle_mod.Tree(w.points, w.kernel, (1.0 / N, 0.0, 0, 0), 32, 1e-9)
    assert np.allclose(y - T0.matvec(w.x), w.x, rtol=0, atol=1e-13)
    for c in range(3):
        assert np.array_equal(T.matvec(w.x[:, c])[:, 0], y[:, c])


def test_dense_rule_at_the_leaf_level_only(oracle_mod):
    """dense_if_cheaper="leaf": the storage rule marks blocks dense at the leaf
    level only; every coarser IL block keeps its ACA factors (rank up to
    min(m, n)), and the product still meets the tolerance against the direct sum."""
    import workloads as W

    w = W.make("t", 3, 8000, W.K_MATERN32, (1, 0, 0.3, 0), 32, 1e-8, nrhs=2, seed=21)
    T = oracle_mod.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, dense_if_cheaper="leaf")
    rec = T.blocks()
    coarse = rec[:, 0] < T.kappa
    assert coarse.any() and not rec[coarse, 8].any()
    Tall = oracle_mod.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, dense_if_cheaper=True)
    assert np.array_equal(rec[~coarse, 7:9], Tall.blocks()[~coarse, 7:9])  # the leaf level is unchanged
    assert Tall.blocks()[coarse, 8].any()  # the plain rule would have made some coarse block dense
    yd = oracle_mod.direct(w.points, w.kernel, w.params, w.x)
    err = np.max(np.linalg.norm(T.matvec(w.x) - yd, axis=0) / np.linalg.norm(yd, axis=0))
    assert err <= 10 * w.tol
