"""GPU batched ACA (a5) against the oracle's ACA.

Same algorithm, FP64, same tie-breaks: ranks and pivots agree on at least 99%
of blocks (kernel values from CUDA's log/exp may differ from the host's in the
last bit, which can flip a near-tie; 1/r uses only correctly rounded operations
and must agree on every block). Where pivots agree the factors agree to
rounding.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


def compare(T, h, exact, max_factor_checks=400):
    """Fraction of blocks with identical rank, dense flag and pivots.

    For those blocks the factors are compared: bit-identical when every kernel
    value is correctly rounded on both sides (exact), else through the product
    U V^T (late ACA terms divide rounding-level residuals by small pivots, so
    ulp differences between CUDA's and the host's log / exp show up in v_k
    entries of negligible weight)."""
    bo = T.blocks()
    bg = h.blocks()
    checked = 0
    assert np.array_equal(bo[:, :7], bg[:, :7])
    same = 0
    for b in range(len(bo)):
        ro, rg = int(bo[b, 7]), int(bg[b, 7])
        if ro != rg or bo[b, 8] != bg[b, 8]:
            continue
        if ro == 0:
            same += 1
            continue
        so, to, Uo, Vo = T.factors(b)
        sg, tg = h.pivots(b, rg)
        if np.array_equal(so, sg) and np.array_equal(to, tg):
            same += 1
            if checked < max_factor_checks:
                checked += 1
                Ug, Vg = h.factors(b, int(bo[b, 4]), int(bo[b, 6]), rg)
                if exact:
                    assert np.array_equal(Ug, Uo) and np.array_equal(Vg, Vo)
                else:
                    Ao = Uo @ Vo.T
                    assert np.linalg.norm(Ug @ Vg.T - Ao) <= 1e-12 * np.linalg.norm(Ao)
    return same / max(len(bo), 1)


@pytest.mark.parametrize("dense_if_cheaper", [False, True])
@pytest.mark.parametrize(
    "d,N,kernel,params,leaf,tol,exact",
    [
        (3, 12000, W.K_INV_R, None, 32, 1e-8, True),
        (2, 4096, W.K_LOG, None, 64, 1e-8, False),
        (4, 5000, W.K_MATERN32, (1, 0, 0.2, 0), 40, 1e-7, False),
        (3, 6000, W.K_GAUSS, (1, 1e-3, 0.5, 0), 32, 1e-6, False),
        (1, 5000, W.K_LOG, None, 16, 1e-10, False),
    ],
)
def test_ranks_and_pivots_match_oracle(env, d, N, kernel, params, leaf, tol, exact, dense_if_cheaper):
    torch, oracle, hd = env
    w = W.make("t", d, N, kernel, params or (1, 0, 0, 0), leaf, tol, 1, seed=d * 7 + 1)
    T = oracle.Tree(w.points, w.kernel, w.params, leaf, tol, dense_if_cheaper=dense_if_cheaper)
    h = gpu_handle(hd, w, dense_if_cheaper=dense_if_cheaper)
    frac = compare(T, h, exact)
    assert frac == 1.0 if exact else frac >= 0.99
    s = h.stats()
    assert s["n_rank_capped"] == 0


def test_large_blocks_use_cta_teams(env):
    # d=2 with few levels: level-1 blocks are > 2048 x 2048 (CTA teams); their
    # sums reduce in a different order, so compare ranks loosely, errors tightly.
    torch, oracle, hd = env
    w = W.make("t", 2, 20000, W.K_LOG, (1, 0, 0, 0), 1500, 1e-9, 1, seed=2)
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol)
    h = gpu_handle(hd, w, dense_if_cheaper=False)
    bo, bg = T.blocks(), h.blocks()
    assert bo[:, 4].max() > 2048
    assert np.array_equal(bo[:, :7], bg[:, :7])
    assert np.all(np.abs(bo[:, 7] - bg[:, 7]) <= 1)


def test_repeated_builds_are_bitwise_identical():
    """Clustered points with a smooth kernel give large blocks handled by CTA
    teams; every build must produce the same ranks, pivots and factors (a race
    between reading the pivot and rescaling its row once broke this)."""
    torch = require_cuda()
    import paper_2209_05819_gb300 as hd

    w = W.make("t", 3, 60000, W.K_GAUSS, (1.0, 1e-3, 0.5, 0), 64, 1e-6, nrhs=1, seed=1017, dist="clustered")
    pts = torch.from_numpy(w.points).cuda()
    ref = None
    for _ in range(3):
        h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol)
        rec = h.blocks()
        big = [b for b in np.argsort(-(rec[:, 4] * rec[:, 6]))[:20] if rec[b, 7] > 0]
        got = (rec.copy(), [h.factors(b, int(rec[b, 4]), int(rec[b, 6]), int(rec[b, 7])) for b in big])
        h.close()
        if ref is None:
            ref = got
            continue
        assert np.array_equal(ref[0], got[0])
        for (U0, V0), (U1, V1) in zip(ref[1], got[1]):
            assert np.array_equal(U0, U1) and np.array_equal(V0, V1)


@pytest.mark.parametrize("pool_bytes", [0, 1 << 16, 1 << 22])
def test_one_pass_pool_does_not_change_the_factors(pool_bytes):
    """The ACA keeps each block's factors in a device pool during its one pass;
    blocks that find the pool full are recomputed by a second pass. A pool of
    0 (two passes for every block), 64 KB (a few blocks fit) or 4 MB gives the
    same ranks, pivots, factors and product, bitwise, as the default pool."""
    torch = require_cuda()
    import paper_2209_05819_gb300 as hd
    from paper_2209_05819_gb300 import _binding as B

    w = W.make("t", 3, 12000, W.K_INV_R, (1.0, 0.0, 0, 0), 32, 1e-8, nrhs=1, seed=77)
    pts = torch.from_numpy(w.points).cuda()
    x = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()

    def build():
        h = hd.Handle(pts, w.kernel, w.params, w.leaf, w.tol)
        rec = h.blocks()
        low = np.flatnonzero(rec[:, 7] > 0)
        pick = low[:: max(1, len(low) // 40)]
        fac = [h.factors(b, int(rec[b, 4]), int(rec[b, 6]), int(rec[b, 7])) for b in pick]
        piv = [h.pivots(b, int(rec[b, 7])) for b in pick]
        y = h.matvec(x).cpu().numpy()
        h.close()
        return rec, fac, piv, y

    ref = build()
    try:
        B.debug_aca_pool_bytes(pool_bytes)
        got = build()
    finally:
        B.debug_aca_pool_bytes(-1)
    assert np.array_equal(ref[0], got[0])
    for (U0, V0), (U1, V1) in zip(ref[1], got[1]):
        assert np.array_equal(U0, U1) and np.array_equal(V0, V1)
    for (s0, t0), (s1, t1) in zip(ref[2], got[2]):
        assert np.array_equal(s0, s1) and np.array_equal(t0, t1)
    assert np.array_equal(ref[3], got[3])
