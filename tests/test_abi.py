"""The C-ABI library builds, loads and exports every entry point that
include/gpe.h declares; host-side argument validation rejects bad input
before anything touches a GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_1709_04423_gb300 import build, gpe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gpe.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared("gpe.h")
    assert "gp_init" in names and "gp_step_real" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(gpe.ABI_SYMBOLS)


def _init(lib, dim=3, n=(8, 8, 8), dx=(0.1, 0.1, 0.1), dt=1e-3, nkl=(1, 1, 1), g=1.0, prec=0):
    h = ctypes.c_void_p()
    rc = lib.gp_init(ctypes.byref(h), dim, (ctypes.c_int * 3)(*n), (ctypes.c_double * 3)(*dx), dt,
                     (ctypes.c_double * 3)(*nkl), g, prec, None)
    return rc, h


@pytest.mark.parametrize("kw", [
    dict(dim=0), dict(dim=4), dict(n=(2, 8, 8)), dict(n=(8, 8, 1)), dict(dx=(0.1, 0.0, 0.1)),
    dict(dx=(0.1, -1.0, 0.1)), dict(dt=0.0), dict(dt=float("nan")), dict(g=float("nan")),
    dict(g=float("inf")), dict(prec=7), dict(nkl=(1, float("nan"), 1)),
    dict(n=(2048, 2048, 1024)),
])
def test_init_rejects_bad_arguments(lib, kw):
    rc, h = _init(lib, **kw)
    assert rc == gpe.GP_ERR_INVALID
    assert not h.value
    assert lib.gp_last_error().decode()


def test_null_handles_are_rejected(lib):
    assert lib.gp_step_real(None, 1) == gpe.GP_ERR_INVALID
    assert lib.gp_step_imag(None, 1) == gpe.GP_ERR_INVALID
    assert lib.gp_set_g(None, 1.0) == gpe.GP_ERR_INVALID
    assert lib.gp_set_dt(None, 1.0) == gpe.GP_ERR_INVALID
    assert lib.gp_destroy(None) == gpe.GP_OK
    assert lib.gp_npoints(None) == 0


def test_init_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _init(lib)
    assert rc == gpe.GP_ERR_CUDA
    assert "cuda" in lib.gp_last_error().decode().lower()


def test_batch_init_rejects_bad_arguments(lib):
    def init(n, dx=(0.1, 0.1), nk=(1.0, 1.0), g=1.0, nruns=1, dt=1e-3):
        b = ctypes.c_void_p()
        na = (ctypes.c_int * 2)(*n)
        return lib.gp_batch_init(ctypes.byref(b), nruns, na, (ctypes.c_double * 2)(*dx), dt,
                                 (ctypes.c_double * 2)(*nk), (ctypes.c_double * 1)(g), 1, None), b
    for kw in (dict(n=(2, 8)), dict(n=(8, 515)), dict(n=(8, 8), dx=(0.0, 0.1)), dict(n=(8, 8), g=float("nan")),
               dict(n=(8, 8), nruns=0), dict(n=(8, 8), dt=0.0)):
        rc, b = init(**kw)
        assert rc == gpe.GP_ERR_INVALID, kw
        assert not b.value


def test_missing_library_fails_loudly(lib, monkeypatch, tmp_path):
    """No CPU fallback: without libgpe.so the binding raises instead of
    running anything else."""
    monkeypatch.setattr(gpe, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gpe.load(str(tmp_path / "libgpe.so"))
