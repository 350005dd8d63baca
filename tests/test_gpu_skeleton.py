"""The memory-efficient skeleton form of the low-rank blocks (Eq. keq2 and the
remark after it): the GPU keeps the ACA pivots and the LU factors of
K(sigma, tau), evaluates K(sigma, J) and K(I, tau) on the fly and solves with L
and U. Checked against

* the oracle's own skeleton form (same pivots, FP64) and the direct sum;
* the GPU's stored-factor form on the same handle structure (the two forms are
  algebraically equal, Eq. keq2);
* the FP64 HODLRdD result, for the FP32 form, within its stated bound;

plus the memory it saves, determinism and the rejected configurations.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import assert_matches_oracle_hodlrdd, gpu_handle, gpu_matvec, relerr, require_cuda

pytestmark = pytest.mark.gpu

# FP32 skeleton form against the FP64 HODLRdD product. Kernel entries in FP32
# on hi + lo coordinates carry a few 2^-24 relative error each (squared
# distance and function rounding). A term with pivot L(q, q) turns the rounding
# of s_q into eps |s| / |L(q, q)| in w_q, which FP32 entries of K(I, tau) cannot
# cancel (cross term eps^2 |s| / |L(q, q)|); the FP32 form keeps the terms whose
# pivot is at least 2^-23 of the largest before it, so that term is about eps.
# What remains is first order: the rounding of s = K(sigma, J) x (compensated
# sums, entries to about one ulp) times the interpolation operator
# K(I, tau) K(sigma, tau)^-1, whose entries for partial-pivoted ACA reach 5-10
# typically and 50-200 in the worst blocks of the tight-tolerance cases here
# (log r and sin r at tol 1e-9). 2e-7 x 25 = 5e-6. log r and sin r pass through
# zero (r = 1, r = pi), where their FP32 values keep an absolute error of about
# 1e-7 instead of a relative one, and their interpolation operators are the
# largest here: 4x that.
SKELETON_FP32_BOUND = 5e-6
SKELETON_FP32_BOUND_ZERO_CROSSING = 2e-5


def fp32_bound(kernel):
    return SKELETON_FP32_BOUND_ZERO_CROSSING if kernel in (W.K_LOG, W.K_SIN) else SKELETON_FP32_BOUND


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


# (d, N, kernel, params, leaf, tol): ragged boxes; the 2-D and 3-D cases have
# level-1 source boxes larger than one staged chunk (partial sums)
CASES = [
    (1, 3001, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-10),
    (2, 4096, W.K_LOG, None, 64, 1e-8),
    (2, 9000, W.K_LOG, None, 40, 1e-9),
    (3, 9000, W.K_INV_R, None, 32, 1e-8),
    (3, 5000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 32, 1e-6),
    (4, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7),
    (4, 3000, W.K_INV_R2_4D, None, 30, 1e-8),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
    (3, 3000, W.K_INV_SQRT1P, None, 25, 1e-9),
]


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", CASES)
def test_fp64_skeleton_matches_oracle(env, d, N, kernel, params, leaf, tol):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 5 * d)
    h = gpu_handle(hd, w, lowrank_form="skeleton")
    yg = gpu_matvec(h, w.x)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(yg, yd) <= 10 * tol
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=True)
    # same pivots: same skeletons (the stored and skeleton forms of the oracle
    # agree to 1e-12); blocks with a flipped pivot within the ACA bound
    assert_matches_oracle_hodlrdd(oracle, T, h, w, yg, tol, kernel, skeleton=True)
    assert relerr(T.matvec(w.x, skeleton=True), T.matvec(w.x)) <= 1e-12


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", CASES[:6])
def test_skeleton_equals_stored_form(env, d, N, kernel, params, leaf, tol):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=1, seed=N + 7 * d)
    hs = gpu_handle(hd, w, lowrank_form="skeleton")
    hf = gpu_handle(hd, w)
    assert np.array_equal(hs.blocks(), hf.blocks())
    assert relerr(gpu_matvec(hs, w.x), gpu_matvec(hf, w.x)) <= 1e-10
    ss, sf = hs.stats(), hf.stats()
    assert ss["lowrank_form"] == 1 and sf["lowrank_form"] == 0
    assert ss["skeleton_terms"] == ss["total_rank"]  # FP64 keeps every ACA term
    # one kernel evaluation per factor entry the stored form keeps
    assert ss["skeleton_pairs"] == sf["factor_elems"] == ss["factor_elems"]
    # p^2 FP64 LU entries plus two pivot indices per rank, against p (m + n) factor entries
    ranks = hs.blocks()[:, 7]
    assert ss["factor_bytes"] == 8 * int((ranks.astype(np.int64) ** 2).sum()) + 8 * int(ranks.sum())


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", [c for c in CASES if c[0] <= 4])
def test_fp32_skeleton_bound(env, d, N, kernel, params, leaf, tol):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 11 * d)
    h64 = gpu_handle(hd, w)
    h32 = gpu_handle(hd, w, precision="fp32", lowrank_form="skeleton")
    assert np.array_equal(h64.blocks(), h32.blocks())
    err = relerr(gpu_matvec(h32, w.x), gpu_matvec(h64, w.x))
    assert err <= fp32_bound(kernel), err
    s = h32.stats()
    assert s["skeleton_terms"] <= s["total_rank"]
    assert (s["skeleton_terms"] > 0) == (s["total_rank"] > 0)


@pytest.mark.parametrize("amax", [-1, 0, 2])
def test_admissibility_variants(env, amax):
    torch, oracle, hd = env
    w = W.make("t", 3, 6000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=40 + amax)
    h = gpu_handle(hd, w, lowrank_form="skeleton", admissible_face_dim=amax)
    T = oracle.Tree(w.points, w.kernel, w.params, 32, 1e-8, dense_if_cheaper=True, admissible_face_dim=amax)
    yg = gpu_matvec(h, w.x)
    bound = 100 * 1e-8 if amax == 2 else 10 * 1e-8
    assert relerr(yg, oracle.direct(w.points, w.kernel, w.params, w.x)) <= bound
    assert_matches_oracle_hodlrdd(oracle, T, h, w, yg, 1e-8, w.kernel, skeleton=True)
    h32 = gpu_handle(hd, w, precision="fp32", lowrank_form="skeleton", admissible_face_dim=amax)
    h64 = gpu_handle(hd, w, admissible_face_dim=amax)
    assert relerr(gpu_matvec(h32, w.x), gpu_matvec(h64, w.x)) <= SKELETON_FP32_BOUND


def test_memory_saving_and_determinism(env):
    torch, oracle, hd = env
    w = W.make("t", 3, 40000, W.K_INV_R, (1, 0, 0, 0), 64, 1e-7, nrhs=1, seed=5)
    hs = gpu_handle(hd, w, precision="fp32", lowrank_form="skeleton")
    hf = gpu_handle(hd, w, precision="fp32")
    ss, sf = hs.stats(), hf.stats()
    # the skeleton keeps a few times less than the stored FP32 factors here
    assert ss["skeleton_bytes"] * 2 < sf["factor_bytes_u"] + sf["factor_bytes_v"]
    assert ss["device_bytes"] < sf["device_bytes"]
    x = torch.from_numpy(np.ascontiguousarray(w.x, dtype=np.float32)).cuda()
    y1 = hs.matvec(x)
    y2 = hs.matvec(x)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    yf = hf.matvec(x)
    torch.cuda.synchronize()
    assert relerr(y1.cpu().numpy(), yf.cpu().numpy()) <= 2 * SKELETON_FP32_BOUND


def test_many_right_hand_sides_and_host_buffers(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 5000, W.K_LOG, (1, 0, 0, 0), 32, 1e-9, nrhs=5, seed=8)
    h = gpu_handle(hd, w, lowrank_form="skeleton")
    Y = gpu_matvec(h, w.x)
    for c in (0, 3, 4):
        assert relerr(Y[:, c : c + 1], gpu_matvec(h, w.x[:, c : c + 1])) <= 1e-14
    yh = h.matvec(np.ascontiguousarray(w.x))  # host arrays in and out
    assert relerr(np.asarray(yh), Y) <= 1e-14


def test_rejected_configurations(env):
    torch, oracle, hd = env
    w = W.make("t", 3, 2000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=2)
    for prec in ("fp16", "bf16"):
        with pytest.raises(hd.HodlrddError) as e:
            gpu_handle(hd, w, precision=prec, lowrank_form="skeleton")
        assert e.value.status == hd.ERR_UNSUPPORTED
    w5 = W.make("t", 5, 1500, W.K_GAUSS, (1, 0, 0.5, 0), 32, 1e-6, nrhs=1, seed=2)
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w5, lowrank_form="skeleton")
    assert e.value.status == hd.ERR_UNSUPPORTED
    with pytest.raises(hd.HodlrddError) as e:
        gpu_handle(hd, w, lowrank_form="skeleton", aca_max_rank=2000)
    assert e.value.status == hd.ERR_UNSUPPORTED
    h = gpu_handle(hd, w, lowrank_form="skeleton")
    rec = h.blocks()
    b = int(np.flatnonzero(rec[:, 7] > 0)[0])
    with pytest.raises(hd.HodlrddError) as e:
        h.factors(b, int(rec[b, 4]), int(rec[b, 6]), int(rec[b, 7]))
    assert e.value.status == hd.ERR_UNSUPPORTED
    with pytest.raises(hd.HodlrddError) as e:
        h.import_factors(rec[:, 7], rec[:, 8], np.zeros(1), np.zeros(1))
    assert e.value.status == hd.ERR_UNSUPPORTED
    # the pivots stay readable: they are the skeleton
    sig, tau = h.pivots(b, int(rec[b, 7]))
    assert len(set(sig.tolist())) == rec[b, 7] and len(set(tau.tolist())) == rec[b, 7]
