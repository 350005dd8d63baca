"""The C-ABI library loads and exports what include/hodlrdd.h declares (no GPU).

Only host-side behaviour is exercised: symbol presence, defaults, and argument
checks that the library performs before any CUDA call.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2209_05819_gb300 as hd
from paper_2209_05819_gb300 import _binding as B


@pytest.fixture(scope="module")
def lib():
    from paper_2209_05819_gb300 import build

    build.build()
    return hd.load()


def test_every_declared_symbol_is_exported(lib):
    names = hd.header_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing


def test_option_defaults(lib):
    o = B.Options()
    assert lib.hodlrdd_options_default(C.byref(o)) == hd.OK
    assert (o.precision, o.dense_if_cheaper, o.max_nrhs, o.aca_max_rank) == (0, 1, 8, 1024)
    assert (o.near_mode, o.admissible_face_dim, o.lowrank_form, o.near_coords) == (0, 0, 0, 0)
    assert (o.fp64_near, o.near_sms) == (0, 0)
    assert C.sizeof(B.Options) == 12 * 4
    assert lib.hodlrdd_options_default(None) == hd.ERR_INVALID


def test_error_strings(lib):
    for s in range(7):
        assert lib.hodlrdd_error_string(s)
    assert lib.hodlrdd_error_string(99) == b"unknown status"


@pytest.mark.parametrize(
    "kw,msg",
    [
        (dict(d=0), b"d must be"),
        (dict(d=9), b"d must be"),
        (dict(N=0), b"N must be"),
        (dict(leaf=0), b"leaf_size"),
        (dict(tol=0.0), b"tol"),
        (dict(tol=float("nan")), b"tol"),
        (dict(kernel=9), b"kernel"),
        (dict(kernel=-1), b"kernel"),
        (dict(kernel=2, params=(1, 0, 0.0, 0)), b"kernel"),  # Matern needs l > 0
        (dict(kernel=3, params=(1, 0, -1.0, 0)), b"kernel"),  # Gaussian needs h > 0
        (dict(params=(float("inf"), 0, 0, 0)), b"kernel"),
        (dict(points=None), b"points is NULL"),
        (dict(out=None), b"out is NULL"),
    ],
)
def test_build_rejects_invalid_arguments(lib, kw, msg):
    pts = np.zeros((10, 2))
    a = dict(points=pts.ctypes.data, d=2, N=10, kernel=0, params=None, leaf=8, tol=1e-8)
    a.update({k: v for k, v in kw.items() if k not in ("out", "points", "params")})
    if "points" in kw:
        a["points"] = kw["points"]
    prm = np.asarray(kw["params"], np.float64) if "params" in kw else None
    h = C.c_void_p()
    out = C.byref(h) if "out" not in kw else None
    rc = lib.hodlrdd_build(a["points"], a["d"], a["N"], a["kernel"], prm.ctypes.data if prm is not None else None,
                           a["leaf"], a["tol"], out)
    assert rc == hd.ERR_INVALID
    assert msg in lib.hodlrdd_last_error()


def test_build_ex_rejects_bad_options(lib):
    pts = np.zeros((10, 2))
    o = B.Options()
    lib.hodlrdd_options_default(C.byref(o))
    o.precision = 7
    h = C.c_void_p()
    assert lib.hodlrdd_build_ex(pts.ctypes.data, 2, 10, 0, None, 8, 1e-8, C.byref(o), C.byref(h)) == hd.ERR_INVALID
    lib.hodlrdd_options_default(C.byref(o))
    o.max_nrhs = 0
    assert lib.hodlrdd_build_ex(pts.ctypes.data, 2, 10, 0, None, 8, 1e-8, C.byref(o), C.byref(h)) == hd.ERR_INVALID
    lib.hodlrdd_options_default(C.byref(o))
    o.near_coords = 2
    assert lib.hodlrdd_build_ex(pts.ctypes.data, 2, 10, 0, None, 8, 1e-8, C.byref(o), C.byref(h)) == hd.ERR_INVALID
    lib.hodlrdd_options_default(C.byref(o))
    o.near_sms = -2
    assert lib.hodlrdd_build_ex(pts.ctypes.data, 2, 10, 0, None, 8, 1e-8, C.byref(o), C.byref(h)) == hd.ERR_INVALID
    assert b"near_sms" in lib.hodlrdd_last_error()


def test_null_handle_calls(lib):
    assert lib.hodlrdd_matvec(None, None, None, 1, None) == hd.ERR_INVALID
    assert lib.hodlrdd_get_stats(None, None) == hd.ERR_INVALID
    assert lib.hodlrdd_destroy(None) == hd.OK
    n = C.c_int64()
    assert lib.hodlrdd_get_level(None, 0, C.byref(n), None, None) == hd.ERR_INVALID
    assert lib.hodlrdd_get_il(None, 1, C.byref(n), None, None) == hd.ERR_INVALID
    assert lib.hodlrdd_import_factors(None, None, None, None, None) == hd.ERR_INVALID


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        B.load()


def _fake_handle(N=100, io=np.float32, device=0):
    """A Handle whose C handle was never built: every check that runs before the
    C call can be exercised without a GPU."""
    h = B.Handle.__new__(B.Handle)
    h.N, h.d, h.io_dtype, h.device, h._h, h._lib = N, 2, io, device, None, None
    return h


class _FakeCuda:
    """Duck-typed CUDA tensor on another device (shape, dtype, device only)."""

    def __init__(self, shape, dtype, index):
        import torch

        self.shape, self.ndim, self.dtype, self.is_cuda = shape, len(shape), dtype, True
        self.device = torch.device("cuda", index)


@pytest.mark.parametrize(
    "x,y,match",
    [
        (np.zeros(99, np.float32), None, "shape"),                     # short x
        (np.zeros((100, 2), np.float64), None, "element type"),         # FP64 x for an FP32 handle
        (np.zeros((100, 2), np.float32), np.zeros((100, 3), np.float32), "differs"),
        (np.zeros((100, 2), np.float32), np.zeros((50, 2), np.float32), "shape"),
        (np.zeros((100, 2), np.float32), np.zeros((100, 2), np.float64), "element type"),
        (np.zeros((100, 0), np.float32), None, "shape"),
        (np.zeros((100, 2, 2), np.float32), None, "shape"),
    ],
)
def test_binding_rejects_mismatched_buffers(x, y, match):
    h = _fake_handle()
    for f in (h.matvec, h.matvec_noalloc):
        with pytest.raises(ValueError, match=match):
            f(x, y)


def test_binding_rejects_other_device_and_torch_types():
    torch = pytest.importorskip("torch")
    h = _fake_handle(io=np.float64, device=0)
    with pytest.raises(ValueError, match="cuda:1"):
        h.matvec(_FakeCuda((100, 1), torch.float64, 1))
    with pytest.raises(ValueError, match="element type"):
        h.matvec(torch.zeros(100, dtype=torch.float32))
    with pytest.raises(ValueError, match="element type"):
        h.matvec(torch.zeros(100, dtype=torch.bfloat16))
    with pytest.raises(ValueError, match="shape"):
        h.matvec(torch.zeros(100, dtype=torch.float64), torch.zeros(101, dtype=torch.float64))
    h32 = _fake_handle()
    with pytest.raises(ValueError, match="one right-hand side"):
        h32.direct(torch.zeros((100, 2), dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA tensors"):
        B.solve(h32, h, np.zeros(100), None)
