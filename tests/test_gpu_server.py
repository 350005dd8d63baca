"""hodlrdd_server: requests over models kept resident under a device-memory
budget. A product that runs alone equals the model's handle alone bitwise; a
batched product (continuous batching of one model's queued products) equals it
within the chunked FP32 bound; a budget below the models' total size evicts and
rebuilds without changing a result; solves reach the FP64 system's tolerance."""
import numpy as np
import pytest

import workloads as W
from gpu_util import gpu_handle, relerr, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = require_cuda()
    import oracle
    import paper_2209_05819_gb300 as hd

    oracle.build()
    return torch, oracle, hd


def models():
    """Five uneven second-kind systems (I + K/N): d = 2..4, four kernels."""
    specs = [(2, 3000, W.K_LOG, 32, 1e-8), (3, 9000, W.K_INV_R, 32, 1e-8), (4, 5000, W.K_MATERN32, 40, 1e-7),
             (3, 6000, W.K_GAUSS, 32, 1e-6), (2, 12000, W.K_INV_R, 64, 1e-8)]
    out = []
    for i, (d, N, k, leaf, tol) in enumerate(specs):
        p0 = {W.K_MATERN32: 0.2, W.K_GAUSS: 0.5}.get(k, 0.0)
        out.append(W.make(f"m{i}", d, N, k, (1.0 / N, 1.0, p0, 0), leaf, tol, nrhs=2, seed=500 + i))
    return out


def alone(hd, ws, prec):
    ys, sizes = [], []
    for w in ws:
        h = gpu_handle(hd, w, precision=prec)
        ys.append(np.asarray(h.matvec(np.ascontiguousarray(w.x, dtype=h.io_dtype))))
        sizes.append(h.stats()["device_bytes"])
        h.close()
    return ys, sizes


@pytest.mark.parametrize("tight", [False, True])
def test_products_equal_alone_and_in_the_mix(env, tight):
    torch, oracle, hd = env
    ws = models()
    prec = "fp32+fp16"
    ref, sizes = alone(hd, ws, prec)
    # tight: room for the largest model and a bit more, far below all of them together
    budget = int(1.5 * max(sizes)) if tight else int(64e9)
    srv = hd.Server(budget, workers=3)
    srv.set_batching(0)  # every product alone: bitwise equal to the handle's
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision=prec) for w in ws]
    rng = np.random.default_rng(0)
    order = rng.integers(0, len(ws), 40)
    reqs = [(m, srv.submit(ids[m], np.ascontiguousarray(ws[m].x, dtype=np.float32))) for m in order]
    for m, r in reqs:
        y, lat = srv.wait(r)
        assert np.array_equal(y, ref[m])
        assert lat > 0.0
    st = srv.stats()
    assert st["resident_bytes"] <= budget
    if tight:  # smaller than the models together: evictions and rebuilds
        assert st["evictions"] > 0 and st["builds"] > len(ws)
        assert st["resident_models"] >= 1
    else:
        assert st["evictions"] == 0 and st["builds"] == len(ws)
    srv.close()


FP32_WIDE_BOUND = 5e-6  # FP32 forms, chunks of 4-16 right-hand sides (uncompensated applies)
TC_BOUND = 5e-6         # the tensor-core form


@pytest.mark.parametrize("prec", ["fp32+fp16", "fp16x2"])
def test_continuous_batching(env, prec):
    """Many products of two models submitted at once: a worker that starts one
    takes the model's other queued products along and runs them as one product
    over their columns. Every result stays within the form's bound of the
    handle alone, and the server reports the batches."""
    torch, oracle, hd = env
    ws = [models()[1], models()[3]]
    bound = TC_BOUND if prec == "fp16x2" else FP32_WIDE_BOUND
    hs = [gpu_handle(hd, w, precision=prec) for w in ws]
    rng = np.random.default_rng(3)
    xs = [[np.ascontiguousarray(rng.standard_normal((w.N, k)), dtype=np.float32) for k in (1, 2, 3, 1, 5, 1, 2, 1)]
          for w in ws]
    ref = [[np.asarray(h.matvec(x)) for x in xl] for h, xl in zip(hs, xs)]
    for h in hs:
        h.close()
    srv = hd.Server(int(64e9), workers=1)
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision=prec) for w in ws]
    # build both models first, then queue everything while the worker is busy
    for m in range(2):
        srv.wait(srv.submit(ids[m], xs[m][0]))
    reqs = []
    for k in range(len(xs[0])):
        for m in range(2):
            reqs.append((m, k, srv.submit(ids[m], xs[m][k])))
    for m, k, r in reqs:
        y, _ = srv.wait(r)
        assert relerr(y, ref[m][k]) <= bound, (m, k)
    st = srv.stats()
    assert st["batches"] >= 1 and st["batched_requests"] >= 2
    srv.close()


def test_solves_and_mixed_kinds(env):
    torch, oracle, hd = env
    ws = models()[:3]
    srv = hd.Server(int(64e9), workers=2)
    ids = [srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision="fp32") for w in ws]
    reqs = []
    for m, w in enumerate(ws):
        reqs.append(("solve", m, srv.submit(ids[m], w.x, kind=hd.REQ_SOLVE)))
        reqs.append(("matvec", m, srv.submit(ids[m], np.ascontiguousarray(w.x, dtype=np.float32))))
    for kind, m, r in reqs:
        y, _ = srv.wait(r)
        w = ws[m]
        if kind == "solve":
            # the FP64 HODLRdD operator applied to u reproduces b
            h64 = gpu_handle(hd, w)
            b = np.asarray(h64.matvec(np.ascontiguousarray(y)))
            assert relerr(b, w.x) <= 1.1e-10
            h64.close()
    assert srv.stats()["builds"] == 2 * len(ws)  # each model and its FP64 twin
    srv.close()


def test_rejections(env):
    torch, oracle, hd = env
    with pytest.raises(hd.HodlrddError):
        hd.Server(0)
    srv = hd.Server(int(1e9), workers=1)
    w = models()[0]
    mid = srv.add(w.points, w.kernel, w.params, w.leaf, w.tol)
    with pytest.raises(hd.HodlrddError):
        srv.submit(mid + 5, np.zeros((w.N, 1), np.float32))
    # a model larger than the budget fails its request, the server keeps going
    tiny = hd.Server(1000, workers=1)
    t = tiny.add(w.points, w.kernel, w.params, w.leaf, w.tol)
    r = tiny.submit(t, np.ascontiguousarray(w.x, dtype=np.float32))
    with pytest.raises(hd.HodlrddError) as e:
        tiny.wait(r)
    assert e.value.status == hd.ERR_OOM
    tiny.close()
    srv.close()


def test_bounded_wait_expiry_is_reported_and_recoverable(env):
    """A bounded device wait that nothing completes (about a second) records its
    error code; hodlrdd_sync reports ERR_TIMEOUT, clears it, and the handle's
    next product is correct."""
    torch, oracle, hd = env
    w = models()[1]
    h = gpu_handle(hd, w, precision="fp32")
    x = np.ascontiguousarray(w.x, dtype=np.float32)
    y0 = np.asarray(h.matvec(x))
    h.debug_expire_wait(2_000_000_000)
    with pytest.raises(hd.HodlrddError) as e:
        h.sync()
    assert e.value.status == hd.ERR_TIMEOUT
    h.sync()  # cleared
    assert np.array_equal(np.asarray(h.matvec(x)), y0)
    h.close()


def test_solve_whose_twin_does_not_fit_beside_running_products(env):
    """Budget room for the FP32 model but not its FP64 twin: a solve on it fails
    with ERR_OOM while products on the same model run on other workers. The
    server must not free the model's handle under their kernels (it waits for
    them), and every product stays bitwise equal to the model alone."""
    torch, oracle, hd = env
    w = models()[1]
    ref, sizes = alone(hd, [w], "fp32")
    h64 = gpu_handle(hd, w)
    twin = h64.stats()["device_bytes"]
    h64.close()
    budget = sizes[0] + twin // 2
    srv = hd.Server(budget, workers=3)
    srv.set_batching(0)  # products alone: bitwise equal to the model's handle
    mid = srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision="fp32")
    x = np.ascontiguousarray(w.x, dtype=np.float32)
    y0, _ = srv.wait(srv.submit(mid, x))  # resident before the mix
    assert np.array_equal(y0, ref[0])
    prods = [srv.submit(mid, x) for _ in range(6)]
    sol = srv.submit(mid, w.x, kind=hd.REQ_SOLVE)
    prods += [srv.submit(mid, x) for _ in range(6)]
    for r in prods:
        y, _ = srv.wait(r)
        assert np.array_equal(y, ref[0])
    with pytest.raises(hd.HodlrddError) as e:
        srv.wait(sol)
    assert e.value.status == hd.ERR_OOM
    y1, _ = srv.wait(srv.submit(mid, x))  # rebuilt if it was dropped
    assert np.array_equal(y1, ref[0])
    assert srv.stats()["resident_bytes"] <= budget
    srv.close()


def test_failed_twin_build_keeps_accounting_exact(env):
    """A solve's first request builds the model and then its FP64 twin; an
    allocation failure injected into the twin's build leaves the model resident
    and its bytes counted (resident_bytes is the model's size, not 0)."""
    torch, oracle, hd = env
    from paper_2209_05819_gb300 import _binding as B

    w = models()[0]
    ref, _ = alone(hd, [w], "fp32")
    h = gpu_handle(hd, w, precision="fp32")
    size = h.stats()["device_bytes"]  # as built, before any host-buffer staging
    h.close()
    srv = hd.Server(int(64e9), workers=1)
    mid = srv.add(w.points, w.kernel, w.params, w.leaf, w.tol, precision="fp32")
    hit_twin = False
    try:
        for k in range(0, 2000, 3):
            B.debug_fail_alloc_after(k)
            r = srv.submit(mid, w.x, kind=hd.REQ_SOLVE)
            try:
                srv.wait(r)
                break  # both builds and the solve got through
            except hd.HodlrddError as e:
                assert e.status == hd.ERR_OOM
            B.debug_fail_alloc_after(-1)
            st = srv.stats()
            assert st["resident_models"] in (0, 1)
            if st["resident_models"] == 1:
                # the model alone (its twin's build failed), or model and twin
                # (a later allocation of the solve failed)
                hit_twin |= st["resident_bytes"] == size
                assert st["resident_bytes"] >= size
            else:
                assert st["resident_bytes"] == 0
    finally:
        B.debug_fail_alloc_after(-1)
    assert hit_twin
    y, _ = srv.wait(srv.submit(mid, np.ascontiguousarray(w.x, dtype=np.float32)))
    assert np.array_equal(y, ref[0])
    srv.close()


def test_solve_reports_an_expired_wait(env):
    """A bounded wait that expired on the inner handle before or during a solve
    makes the solve return ERR_TIMEOUT (it reads and clears both handles' error
    words); the next solve is clean."""
    torch, oracle, hd = env
    w = models()[1]
    hi = gpu_handle(hd, w, precision="fp32")
    ho = gpu_handle(hd, w)
    b = torch.from_numpy(np.ascontiguousarray(w.x[:, 0])).cuda()
    hi.debug_expire_wait(200_000_000)
    with pytest.raises(hd.HodlrddError) as e:
        hd.solve(hi, ho, b)
    assert e.value.status == hd.ERR_TIMEOUT
    x, st = hd.solve(hi, ho, b)
    assert st["residual"] <= 1e-10
    hi.sync()
    ho.sync()
