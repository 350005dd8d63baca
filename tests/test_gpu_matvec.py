"""GPU matvec (a7-a10) against the oracle.

* apply parity: with the oracle's own factors imported, the GPU FP64 matvec
  equals the oracle's Algorithm 2 to 1e-12 (relative 2-norm per column);
* end to end FP64: GPU build + matvec within 1e-10 of the oracle's HODLRdD and
  within 10 tol of the direct sum;
* mixed precision: FP32 / FP16 / BF16 factors, FP32 arithmetic, each with its
  stated bound against the FP64 oracle;
* right-hand sides, host and device buffers, determinism, edge cases.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import assert_matches_oracle_hodlrdd, gpu_handle, gpu_matvec, oracle_factors, relerr, require_cuda

pytestmark = pytest.mark.gpu

# stated error bounds of the mixed-precision forms against the FP64 result
MIXED_BOUND = {"fp32": 2e-6, "fp16": 2e-3, "bf16": 1.5e-2}
# FP32 with chunks of 4 or 8 right-hand sides: the low-rank applies accumulate
# without compensation (register budget), a few thousand FP32 products per
# output, so the bound is looser than the compensated one- and two-RHS form
FP32_WIDE_BOUND = 5e-6


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


APPLY_CASES = [
    (2, 4096, W.K_LOG, None, 64, 1e-8),
    (3, 9000, W.K_INV_R, None, 32, 1e-8),
    (4, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7),
    (3, 5000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 32, 1e-6),
    (1, 3001, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-10),
    (4, 3000, W.K_INV_R2_4D, None, 30, 1e-8),
    (2, 3000, W.K_R, None, 25, 1e-9),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
    (3, 3000, W.K_INV_SQRT1P, None, 25, 1e-9),
]


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", APPLY_CASES)
@pytest.mark.parametrize("dense_if_cheaper", [False, True])
def test_apply_parity_with_oracle_factors(env, d, N, kernel, params, leaf, tol, dense_if_cheaper):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=3, seed=N + d)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=dense_if_cheaper)
    h = gpu_handle(hd, w, dense_if_cheaper=dense_if_cheaper)
    h.import_factors(*oracle_factors(T))
    yg = gpu_matvec(h, w.x)
    yo = T.matvec(w.x)
    assert relerr(yg, yo) <= 1e-12


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", APPLY_CASES[:5])
def test_end_to_end_fp64(env, d, N, kernel, params, leaf, tol):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 2 * d)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=True)
    h = gpu_handle(hd, w)
    yg = gpu_matvec(h, w.x)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(yg, yd) <= 10 * tol
    # 1e-10 against the oracle's HODLRdD where every pivot agrees, the ACA
    # bound on the few blocks where a library ulp flipped one
    assert_matches_oracle_hodlrdd(oracle, T, h, w, yg, tol, kernel)


def test_config1_plain_fp64(env):
    """d=2, N=4096 uniform [-1,1]^2 (seed 0), log r with F(x,x)=0, leaf 64, tol 1e-8."""
    torch, oracle, hd = env
    w = W.plain_fp64_2d()
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, dense_if_cheaper=True)
    h = gpu_handle(hd, w)
    yg = gpu_matvec(h, w.x)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    yo = T.matvec(w.x)
    assert relerr(yg, yd) <= 10 * w.tol
    assert relerr(yg, yo) <= 1e-10


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", [APPLY_CASES[1], APPLY_CASES[2], APPLY_CASES[0]])
def test_mixed_precision_bounds(env, precision, d, N, kernel, params, leaf, tol):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 3 * d)
    h64 = gpu_handle(hd, w)
    hm = gpu_handle(hd, w, precision=precision)
    y64 = gpu_matvec(h64, w.x)
    ym = gpu_matvec(hm, w.x)
    err = relerr(ym, y64)
    assert err <= MIXED_BOUND[precision], err
    # same structure and ranks: only the storage precision differs
    assert np.array_equal(h64.blocks(), hm.blocks())


@pytest.mark.parametrize("precision", ["fp64", "fp16"])
def test_many_right_hand_sides(env, precision):
    torch, oracle, hd = env
    w = W.make("t", 3, 7000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=13, seed=3)
    h = gpu_handle(hd, w, precision=precision)
    Y = gpu_matvec(h, w.x)
    for c in (0, 5, 8, 12):
        yc = gpu_matvec(h, w.x[:, c : c + 1])
        assert relerr(Y[:, c : c + 1], yc) <= (1e-14 if precision == "fp64" else 1e-6)
    for k in (2, 3, 4, 8):
        Yk = gpu_matvec(h, w.x[:, :k])
        assert relerr(Y[:, :k], Yk) <= (1e-14 if precision == "fp64" else 1e-6)


def test_host_buffers_and_determinism(env):
    torch, oracle, hd = env
    w = W.make("t", 3, 8000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, nrhs=2, seed=4)
    h = gpu_handle(hd, w)
    yh = h.matvec(np.ascontiguousarray(w.x))  # host in, host out
    yd1 = gpu_matvec(h, w.x)
    yd2 = gpu_matvec(h, w.x)
    assert np.array_equal(yd1, yd2)
    assert np.array_equal(yh, yd1)
    h2 = gpu_handle(hd, w)
    assert np.array_equal(gpu_matvec(h2, w.x), yd1)


def test_identity_shift_operator(env):
    torch, oracle, hd = env
    N = 6000
    w = W.make("t", 3, N, W.K_INV_R, (1.0 / N, 1.0, 0, 0), 32, 1e-9, nrhs=1, seed=5)
    h = gpu_handle(hd, w)
    yg = gpu_matvec(h, w.x)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(yg, yd) <= 10 * w.tol


@pytest.mark.parametrize("N,leaf", [(1, 4), (37, 64), (65, 64), (130, 7)])
def test_small_and_ragged(env, N, leaf):
    torch, oracle, hd = env
    w = W.make("t", 2, N, W.K_LOG, (1, 0, 0, 0), leaf, 1e-12, nrhs=3, seed=N)
    h = gpu_handle(hd, w)
    yg = gpu_matvec(h, w.x)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    if N == 1:
        assert np.all(yg == 0.0)
    else:
        assert relerr(yg, yd) <= 1e-10


def test_rejects_overlap_and_bad_nrhs(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 500, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, seed=1)
    h = gpu_handle(hd, w)
    x = torch.zeros(500, dtype=torch.float64, device="cuda")
    with pytest.raises(hd.HodlrddError):
        h.matvec(x, x)
    st = h._lib.hodlrdd_matvec(h._h, x.data_ptr(), x.data_ptr() + 8 * 500, 0, None)
    assert st == hd.ERR_INVALID


def test_injected_allocation_failure_is_clean(env):
    torch, oracle, hd = env
    from paper_2209_05819_gb300 import _binding as B

    w = W.make("t", 3, 5000, W.K_INV_R, (1, 0, 0, 0), 32, 1e-8, seed=2)
    pts = torch.from_numpy(w.points).cuda()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (0, 3, 10, 25):
        B.debug_fail_alloc_after(k)
        with pytest.raises(hd.HodlrddError) as e:
            hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol)
        assert e.value.status == hd.ERR_OOM
    B.debug_fail_alloc_after(-1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < (64 << 20)
    h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol)  # still usable
    assert h.stats()["n_blocks"] > 0


PACKED_CASES = [
    (1, 3000, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-9),
    (2, 4096, W.K_LOG, None, 64, 1e-8),
    (2, 3000, W.K_R, None, 25, 1e-9),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
    (3, 9000, W.K_INV_R, None, 32, 1e-8),
    (3, 5000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 32, 1e-6),
    (3, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7),
    (3, 4000, W.K_INV_R2_4D, None, 30, 1e-8),
    (3, 3000, W.K_INV_SQRT1P, None, 25, 1e-9),
]


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", PACKED_CASES)
def test_fp32_single_rhs_packed_near_field(env, d, N, kernel, params, leaf, tol):
    """One right-hand side in FP32 uses packed box-relative points and a
    kernel-specialised pair loop; it must agree with the FP64 form and with the
    general (two right-hand sides) FP32 path."""
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 5 * d)
    h64 = gpu_handle(hd, w)
    h32 = gpu_handle(hd, w, precision="fp32")
    y64 = gpu_matvec(h64, w.x[:, :1])
    y1 = gpu_matvec(h32, w.x[:, :1])
    y2 = gpu_matvec(h32, w.x)
    h32.sync()
    assert relerr(y1, y64) <= MIXED_BOUND["fp32"]
    # both FP32 forms carry the FP32 bound against FP64, so they differ by at most twice it
    assert relerr(y1, y2[:, :1]) <= 2 * MIXED_BOUND["fp32"]


TILE_CASES = [
    (2, 4096, W.K_LOG, None, 64, 1e-8),          # leaf IL blocks partly low-rank: tiles subtract them
    (3, 9000, W.K_INV_R, None, 32, 1e-8),
    (3, 20000, W.K_INV_R, None, 64, 1e-7),       # small leaves: leaf IL blocks dense
    (1, 3000, W.K_EXP, (1, 0, 1.0, 0), 16, 1e-9),
    (3, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7),
    (2, 3000, W.K_SIN, None, 25, 1e-9),
]


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", TILE_CASES)
def test_near_field_tiles_and_lists_agree(env, d, N, kernel, params, leaf, tol):
    """The packed near field as parent tiles (near_mode 1, low-rank leaf IL
    blocks subtracted) and as per-leaf-box lists (near_mode 2) must both agree
    with the FP64 form and with each other."""
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=1, seed=N + 7 * d)
    h64 = gpu_handle(hd, w)
    y64 = gpu_matvec(h64, w.x)
    ys = []
    for mode in (1, 2):
        h = gpu_handle(hd, w, precision="fp32", near_mode=mode)
        ys.append(gpu_matvec(h, w.x))
        h.sync()
        assert relerr(ys[-1], y64) <= MIXED_BOUND["fp32"], mode
    assert relerr(ys[0], ys[1]) <= 2 * MIXED_BOUND["fp32"]


DIRECT_CASES = [
    (1, 3000, W.K_EXP, (1, 0, 1.0, 0)),
    (2, 4000, W.K_LOG, None),
    (3, 6000, W.K_INV_R, None),
    (3, 5000, W.K_MATERN32, (1, 0, 0.2, 0)),
    (3, 3000, W.K_INV_R2_4D, None),
    (2, 3000, W.K_SIN, None),
    (3, 4000, W.K_INV_R, (1.0 / 4000, 1.0, 0, 0)),  # I + K/N
]


@pytest.mark.parametrize("d,N,kernel,params", DIRECT_CASES)
def test_direct_sum_matches_oracle(env, d, N, kernel, params):
    """The on-the-fly O(N^2) GPU product equals the oracle's FP64 direct sum
    within the FP32 bound."""
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=N + 11 * d)
    h = gpu_handle(hd, w, precision="fp32")
    x = torch.from_numpy(np.ascontiguousarray(w.x[:, 0], dtype=np.float32)).cuda()
    y = h.direct(x)
    torch.cuda.synchronize()
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(y.cpu().numpy()[:, None], yd) <= MIXED_BOUND["fp32"]


def test_direct_rejects_fp64_and_host_buffers(env):
    torch, oracle, hd = env
    w = W.make("t", 2, 500, W.K_LOG, (1, 0, 0, 0), 32, 1e-8, seed=2)
    h64 = gpu_handle(hd, w)
    x = torch.zeros(500, dtype=torch.float32, device="cuda")
    with pytest.raises(hd.HodlrddError) as e:
        h64.direct(x)
    assert e.value.status == hd.ERR_UNSUPPORTED
    h32 = gpu_handle(hd, w, precision="fp32")
    with pytest.raises(hd.HodlrddError) as e:
        h32.direct(np.zeros(500, np.float32), np.zeros(500, np.float32))
    assert e.value.status == hd.ERR_INVALID


@pytest.mark.parametrize("nrhs", [1, 3, 8])
@pytest.mark.parametrize("kernel,params", [(W.K_MATERN32, (1, 0, 0.2, 0)), (W.K_INV_R2_4D, None)])
def test_fp32_four_dims_multi_rhs(env, nrhs, kernel, params):
    """d = 4 and several right-hand sides use the multi-RHS near-field tiles:
    each column agrees with the FP64 form within the FP32 bound."""
    torch, oracle, hd = env
    w = W.make("t", 4, 6000, kernel, params or (1, 0, 0, 0), 40, 1e-7, nrhs=nrhs, seed=6000 + nrhs)
    h64 = gpu_handle(hd, w)
    h32 = gpu_handle(hd, w, precision="fp32")
    y64 = gpu_matvec(h64, w.x)
    y32 = gpu_matvec(h32, w.x)
    h32.sync()
    assert relerr(y32, y64) <= (MIXED_BOUND["fp32"] if nrhs < 4 else FP32_WIDE_BOUND)


@pytest.mark.parametrize("d,nrhs", [(3, 16), (4, 20), (2, 35)])
def test_fp32_wide_chunks(env, d, nrhs):
    """With max_nrhs >= 16 an FP32 handle applies chunks of 16 right-hand sides
    (panels and near-field tiles 16 wide); every column agrees with the FP64 form
    and with the same columns applied alone."""
    torch, oracle, hd = env
    w = W.make("t", d, 7000, W.K_MATERN32 if d == 4 else W.K_INV_R, (1, 0, 0.3, 0) if d == 4 else (1, 0, 0, 0),
               40, 1e-7, nrhs=nrhs, seed=7000 + nrhs)
    h64 = gpu_handle(hd, w)
    hw = gpu_handle(hd, w, precision="fp32", max_nrhs=64)
    y64 = gpu_matvec(h64, w.x)
    yw = gpu_matvec(hw, w.x)
    hw.sync()
    assert relerr(yw, y64) <= FP32_WIDE_BOUND
    y1 = gpu_matvec(hw, w.x[:, 3:4])
    assert relerr(yw[:, 3:4], y1) <= 2 * FP32_WIDE_BOUND


@pytest.mark.parametrize("d,amax", [(2, -1), (2, 1), (3, -1), (3, 2)])
def test_matvec_any_admissibility(env, d, amax):
    """Strong and weak admissibility end to end: the FP64 product equals the
    oracle's under the same structure (pivots agreeing) and the FP32 packed
    form (leaf tiles and lists) stays within the FP32 bound of it."""
    torch, oracle, hd = env
    w = W.make("t", d, 5000, W.K_INV_R if d == 3 else W.K_LOG, (1, 0, 0, 0), 32, 1e-8, nrhs=1, seed=50 + d)
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, dense_if_cheaper=True, admissible_face_dim=amax)
    h64 = gpu_handle(hd, w, admissible_face_dim=amax)
    y64 = gpu_matvec(h64, w.x)
    assert_matches_oracle_hodlrdd(oracle, T, h64, w, y64, w.tol, w.kernel)
    yd = oracle.direct(w.points, w.kernel, w.params, w.x)
    assert relerr(y64, yd) <= (10 if amax < d - 1 else 100) * w.tol
    for mode in (1, 2):
        h32 = gpu_handle(hd, w, precision="fp32", admissible_face_dim=amax, near_mode=mode)
        y32 = gpu_matvec(h32, w.x)
        h32.sync()
        assert relerr(y32, y64) <= MIXED_BOUND["fp32"], mode


@pytest.mark.parametrize("d,N,kernel,params,leaf,tol", [(3, 8000, W.K_MATERN32, (1, 0, 0.3, 0), 32, 1e-8),
                                                         (2, 6000, W.K_LOG, None, 32, 1e-10)])
def test_dense_rule_leaf_only_fp64(env, d, N, kernel, params, leaf, tol):
    """dense_if_cheaper="leaf" (coarse blocks keep their factors): the GPU FP64
    product against the oracle's HODLRdD product built with the same rule."""
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, nrhs=2, seed=N + 9)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper="leaf")
    h = gpu_handle(hd, w, dense_if_cheaper="leaf")
    rec = h.blocks()
    assert not rec[rec[:, 0] < h.stats()["kappa"], 8].any()
    yg = gpu_matvec(h, w.x)
    assert relerr(yg, oracle.direct(w.points, w.kernel, w.params, w.x)) <= 10 * tol
    assert_matches_oracle_hodlrdd(oracle, T, h, w, yg, tol, kernel)
