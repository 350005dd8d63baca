"""GPU tree and interaction lists are bit-exact against the oracle.

Integer work (a1-a4): bounding cube, Morton keys, stable tree order, level
tables, IL and near lists, block table. Compared element by element.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import require_cuda, gpu_handle

pytestmark = pytest.mark.gpu

CASES = [
    ("c1 d=2 log", dict(d=2, N=4096, kernel=W.K_LOG, leaf=64, seed=0)),
    ("d=1 ragged", dict(d=1, N=3001, kernel=W.K_LOG, leaf=16, seed=3)),
    ("d=3 uniform", dict(d=3, N=20000, kernel=W.K_INV_R, leaf=32, seed=5)),
    ("d=4 uniform", dict(d=4, N=6000, kernel=W.K_LOG, leaf=20, seed=6)),
    ("d=3 clustered", dict(d=3, N=9000, kernel=W.K_INV_R, leaf=24, seed=7, dist="clustered")),
    ("d=5 small", dict(d=5, N=3000, kernel=W.K_INV_R, leaf=40, seed=8)),
    ("d=8 small", dict(d=8, N=1500, kernel=W.K_GAUSS, leaf=100, seed=9)),
    ("single leaf", dict(d=3, N=50, kernel=W.K_INV_R, leaf=64, seed=1)),
    ("one point", dict(d=2, N=1, kernel=W.K_LOG, leaf=4, seed=1)),
]


def _workload(kw):
    params = (1, 0, 0.5, 0) if kw["kernel"] in (W.K_GAUSS, W.K_MATERN32, W.K_EXP) else (1, 0, 0, 0)
    return W.make("t", kw["d"], kw["N"], kw["kernel"], params, kw["leaf"], 1e-6, 1, kw["seed"],
                  kw.get("dist", "uniform"))


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_tree_and_lists_bit_exact(env, name, kw):
    torch, oracle, hd = env
    w = _workload(kw)
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol)
    h = gpu_handle(hd, w)
    s = h.stats()
    assert s["kappa"] == T.kappa
    lo_o, side_o, inv_o = T.cube()
    lo_g, side_g, inv_g = h.cube()
    assert np.array_equal(lo_o, lo_g) and side_o == side_g and inv_o == inv_g
    po, ko = T.perm()
    pg, kg = h.tree()
    assert np.array_equal(po, pg)
    assert np.array_equal(ko, kg)
    for l in range(T.kappa + 1):
        so, bo = T.level(l)
        sg, bg = h.level(l)
        assert np.array_equal(so, sg), l
        assert np.array_equal(bo, bg), l
    for l in range(1, T.kappa + 1):
        oo, io = T.il(l)
        og, ig = h.il(l)
        assert np.array_equal(oo, og), l
        assert np.array_equal(io, ig), l
    no, nio = T.near()
    ng, nig = h.near()
    assert np.array_equal(no, ng) and np.array_equal(nio, nig)
    bo = T.blocks()
    bg = h.blocks()
    assert np.array_equal(bo[:, :7], bg[:, :7])
    h.close()


def test_duplicate_points_reach_the_finest_level(env):
    torch, oracle, hd = env
    rng = np.random.default_rng(0)
    pts = np.concatenate([rng.uniform(-1, 1, (300, 1)), np.full((40, 1), 0.125)])
    T = oracle.Tree(pts, W.K_LOG, None, 8, 1e-6)
    h = hd.Handle(torch.from_numpy(pts).cuda(), W.K_LOG, None, 8, 1e-6)
    assert T.kappa == T.B == h.stats()["kappa"] == 32
    assert np.array_equal(T.perm()[0], h.tree()[0])
    for l in range(1, T.kappa + 1):
        assert np.array_equal(T.il(l)[1], h.il(l)[1])


def test_host_and_device_points_agree(env):
    torch, oracle, hd = env
    w = _workload(CASES[2][1])
    h1 = hd.Handle(w.points, w.kernel, w.params, w.leaf, w.tol)
    h2 = gpu_handle(hd, w)
    assert np.array_equal(h1.tree()[0], h2.tree()[0])
    assert np.array_equal(h1.blocks(), h2.blocks())


def test_nonfinite_points_rejected_on_device(env):
    torch, oracle, hd = env
    pts = torch.zeros((100, 3), dtype=torch.float64, device="cuda")
    pts[17, 1] = float("nan")
    with pytest.raises(hd.HodlrddError) as e:
        hd.Handle(pts, W.K_INV_R, None, 8, 1e-6)
    assert e.value.status == hd.ERR_INVALID


ADM_CASES = [
    (dict(d=2, N=4096, kernel=W.K_LOG, leaf=40, seed=10), -1),
    (dict(d=2, N=4096, kernel=W.K_LOG, leaf=40, seed=10), 1),
    (dict(d=3, N=12000, kernel=W.K_INV_R, leaf=32, seed=11), -1),
    (dict(d=3, N=12000, kernel=W.K_INV_R, leaf=32, seed=11), 1),
    (dict(d=3, N=12000, kernel=W.K_INV_R, leaf=32, seed=11), 2),
    (dict(d=4, N=5000, kernel=W.K_LOG, leaf=20, seed=12, dist="clustered"), 2),
]


@pytest.mark.parametrize("kw,amax", ADM_CASES)
def test_lists_bit_exact_any_admissibility(env, kw, amax):
    """Strong (-1), intermediate and weak (d - 1) admissibility: IL and near
    lists and the block table equal the oracle's."""
    torch, oracle, hd = env
    w = _workload(kw)
    T = oracle.Tree(w.points, w.kernel, w.params, w.leaf, w.tol, admissible_face_dim=amax)
    h = gpu_handle(hd, w, admissible_face_dim=amax)
    for l in range(1, T.kappa + 1):
        oo, io = T.il(l)
        og, ig = h.il(l)
        assert np.array_equal(oo, og) and np.array_equal(io, ig), l
    no, nio = T.near()
    ng, nig = h.near()
    assert np.array_equal(no, ng) and np.array_equal(nio, nig)
    assert np.array_equal(T.blocks()[:, :7], h.blocks()[:, :7])
    h.close()


def test_admissibility_out_of_range_rejected(env):
    torch, oracle, hd = env
    w = _workload(dict(d=2, N=500, kernel=W.K_LOG, leaf=20, seed=1))
    for amax in (-2, 2):
        with pytest.raises(hd.HodlrddError) as e:
            gpu_handle(hd, w, admissible_face_dim=amax)
        assert e.value.status == hd.ERR_INVALID
