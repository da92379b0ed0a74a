"""The checking build (libgpe_check.so: GPE_BOUNDS_CHECK) on edge grids.

compute-sanitizer is not available on this machine, so the library is built a
second time with an index test before every state and shared-memory access of
the sweep and observables kernels (a failed test records a code and skips the
access) and with 64 KB guard bands of 0xFF bytes around every device buffer.
Here it runs the grids where an index is most likely to slip -- one interior
point per axis, even and odd sizes from 3 to 17, lines of 514 and 515 points
(the longest segmented line and the first thread-per-line one) -- in every
precision and in both time directions, with enough steps for the graph
replays, in the default kernel shapes and in the fused-plane, pipelined and
TMA shapes, and a batch of edge sizes in both launch forms.  The two libraries are loaded into the
same process, which the test suite thereby also checks.  After every case gp_check_status must
report no failed check and intact guard bands; the FP64 runs must also match
the oracle (1e-12), so that a skipped access would show.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I

pytestmark = pytest.mark.gpu

C3I, C3D = ctypes.c_int * 3, ctypes.c_double * 3
PREC = {"f64": 0, "f32": 1, "df64": 2}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1709_04423_gb300 import gpe
    assert torch.cuda.is_available()
    L = gpe.load_check()
    code = ctypes.c_int()
    assert L.gp_check_status(ctypes.byref(code)) == 0 and code.value == 0   # a checking build, clean at start
    return L


def status(lib):
    code = ctypes.c_int()
    rc = lib.gp_check_status(ctypes.byref(code))
    return rc, code.value, lib.gp_last_error().decode()


def run(lib, dim, n, dx, prec, imag, steps, shapes=None, g=8.0):
    nkl = [1.0, 1.3, 1.6][:dim]
    dt = 1e-3 if imag else 2e-4
    h = ctypes.c_void_p()
    pad = lambda v, f: (list(v) + [f] * 3)[:3]
    rc = lib.gp_init(ctypes.byref(h), dim, C3I(*pad(n, 1)), C3D(*pad(dx, 1.0)), dt, C3D(*pad(nkl, 1.0)), g,
                     PREC[prec], None)
    assert rc == 0, lib.gp_last_error()
    try:
        if shapes is not None:
            assert lib.gp_set_shapes(h, *shapes) == 0, lib.gp_last_error()
        phi0 = I.gaussian_state(dim, n, dx, nkl, seed=sum(n) + dim, noise=1e-3)
        a = np.ascontiguousarray(phi0, dtype=np.complex64 if prec == "f32" else np.complex128)
        assert lib.gp_set_state(h, a.ctypes.data_as(ctypes.c_void_p), 0) == 0
        assert (lib.gp_step_imag if imag else lib.gp_step_real)(h, ctypes.c_long(steps)) == 0, lib.gp_last_error()
        from paper_1709_04423_gb300.gpe import GpObs
        ob = GpObs()
        assert lib.gp_observables(h, ctypes.byref(ob), None, 0) == 0, lib.gp_last_error()
        out = np.empty_like(a)
        assert lib.gp_get_state(h, out.ctypes.data_as(ctypes.c_void_p), 0) == 0
    finally:
        lib.gp_destroy(h)
    assert np.all(np.isfinite(out)) and np.isfinite(ob.mu)
    if prec == "f64":
        ref = O.run(O.Grid(dim, n, dx, dt, nkl, g), phi0, imag, steps)
        assert np.linalg.norm(out - ref) <= 1e-12 * max(np.linalg.norm(ref), 1e-300)
    return out


EDGE = [
    (1, [3], [0.5]), (1, [4], [0.5]), (1, [17], [0.3]), (1, [514], [0.02]), (1, [515], [0.02]),
    (2, [3, 3], [0.5, 0.5]), (2, [5, 17], [0.4, 0.3]), (2, [16, 4], [0.3, 0.5]),
    (2, [514, 4], [0.02, 0.5]), (2, [6, 515], [0.4, 0.02]),
    (3, [3, 4, 5], [0.5, 0.5, 0.5]), (3, [17, 16, 3], [0.3, 0.3, 0.5]), (3, [32, 9, 7], [0.25, 0.4, 0.4]),
    (3, [16, 6, 515], [0.3, 0.4, 0.02]), (3, [514, 4, 3], [0.02, 0.5, 0.5]),
]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("dim,n,dx", EDGE)
def test_edge_grids_pass_the_checks(lib, dim, n, dx, prec, imag):
    if prec == "df64" and max(n) > 514:
        pytest.skip("the double-float form takes at most 514 points per axis (refused at gp_init)")
    run(lib, dim, n, dx, prec, imag, 40)
    rc, code, msg = status(lib)
    assert rc == 0 and code == 0, (code, msg)


# (tile_x, seg_x, seg_c, flags) on the 32 x 9 x 7 grid (FP32): the fused x + y
# plane kernel, the pipelined sweeps, the TMA sweeps
SHAPES = [(1, 8, 4, 8), (1, 16, 4, 8), (1, 8, 4, 2 | 4), (1, 8, 8, 32), (1, 8, 8, 16), (1, 16, 8, 48)]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("shapes", SHAPES)
def test_kernel_shapes_pass_the_checks(lib, shapes, imag):
    got = run(lib, 3, [32, 9, 7], [0.25, 0.4, 0.4], "f32", imag, 40, shapes=shapes)
    ref = run(lib, 3, [32, 9, 7], [0.25, 0.4, 0.4], "f64", imag, 40)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    rc, code, msg = status(lib)
    assert rc == 0 and code == 0, (code, msg)


@pytest.mark.parametrize("prec,mode", [("f64", 0), ("f32", 0), ("f32", 1), ("df64", 0)])
def test_batch_of_edge_sizes_passes_the_checks(lib, prec, mode):
    sizes = [(3, 3), (17, 5), (514, 4), (4, 514), (64, 48)]   # a batch takes at most 514 points per axis
    nr = len(sizes)
    n = (ctypes.c_int * (2 * nr))(*[v for s in sizes for v in s])
    dxs = (ctypes.c_double * (2 * nr))(*([0.3, 0.3] * nr))
    nkl = (ctypes.c_double * (2 * nr))(*([1.0, 1.4] * nr))
    g = (ctypes.c_double * nr)(*([5.0] * nr))
    b = ctypes.c_void_p()
    assert lib.gp_batch_init(ctypes.byref(b), nr, n, dxs, 5e-4, nkl, g, PREC[prec], None) == 0, lib.gp_last_error()
    try:
        assert lib.gp_batch_set_mode(b, mode) == 0, lib.gp_last_error()   # 1: the one-launch form
        for r, (nx, ny) in enumerate(sizes):
            a = np.ascontiguousarray(I.gaussian_state(2, [nx, ny], [0.3, 0.3], [1.0, 1.4]),
                                     dtype=np.complex64 if prec == "f32" else np.complex128)
            assert lib.gp_batch_set_state(b, r, a.ctypes.data_as(ctypes.c_void_p), 0) == 0
        assert lib.gp_batch_step_real(b, ctypes.c_long(40)) == 0, lib.gp_last_error()
        from paper_1709_04423_gb300.gpe import GpObs
        obs = (GpObs * nr)()
        assert lib.gp_batch_observables(b, obs) == 0, lib.gp_last_error()
        assert all(np.isfinite(o.mu) for o in obs)
    finally:
        lib.gp_batch_destroy(b)
    rc, code, msg = status(lib)
    assert rc == 0 and code == 0, (code, msg)


def test_normal_library_reports_no_checks():
    from paper_1709_04423_gb300 import gpe
    code = ctypes.c_int()
    assert gpe.load().gp_check_status(ctypes.byref(code)) == 0
    assert code.value == -1
