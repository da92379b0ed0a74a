"""The segment carries cut to the precision's reach.

The host reads off each segmentation's tables how many segments a carry
crosses and how many points at a segment's start and end take one (rounded up
to 4, 8, 12 or every point; the sweeps are unrolled for each class), so that
every term left out is at most 2^-48 (FP32 state) or 2^-64 (otherwise).  Here
the time step and spacing are chosen so that the recurrence coefficient
|alpha| ~ dt/(4 dx^2) puts the sweeps in every class -- 4, 8, 12, every point
and carries that cross several segments -- on ragged lines (a partial last
segment), in the tile, column, fused-plane and TMA shapes, and the results
are held to the oracle: FP64 and double-float at rel-L2 1e-12 after 60 steps,
FP32 at the FP32 bounds of the other parity tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1709_04423_gb300 import gpe
    gpe.load()
    assert torch.cuda.is_available()
    return gpe


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# (dt, dx): |alpha| ~ 1e-5 (4 points), ~6e-4 (8), ~1e-2 (8 in FP32, 12 otherwise),
# ~0.2 (every point, carries across segments)
STEPS = [(1e-5, 0.5), (2e-4, 0.3), (1e-3, 0.15), (1e-3, 0.03)]
SHAPES2 = [(1, 4, 4, 0), (1, 8, 8, 0), (1, 16, 16, 0)]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("dt,h", STEPS)
def test_carry_classes_2d_ragged(G, dt, h, prec, imag):
    n, nkl = [37, 45], [1.0, 1.3]
    dx = [h, h * 1.1]
    gr = O.Grid(2, n, dx, dt, nkl, 15.0)
    phi0 = I.gaussian_state(2, n, dx, nkl, seed=61, noise=1e-3)
    ref = O.run(gr, phi0, imag, 60)
    tol = 1e-12 if prec != "f32" else (2e-5 if imag else 1e-4)
    for shapes in SHAPES2:
        p = G.Propagator(2, n, dx, dt, nkl, 15.0, precision=prec)
        G.gp_set_shapes(p.h, *shapes)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(60)
        got = p.get_state(device=False).astype(np.complex128)
        p.close()
        assert rel_l2(got, ref) <= tol, (shapes, rel_l2(got, ref))


# 3d FP32: the fused x + y plane kernel (flag 8), the TMA y/z sweeps (16) and
# the TMA x sweep (32) beside the register sweeps
SHAPES3 = [(1, 8, 8, 0), (1, 8, 8, 8), (1, 16, 8, 16), (1, 16, 16, 48)]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dt,h", STEPS)
def test_carry_classes_3d_fp32_shapes(G, dt, h, imag):
    n, nkl = [48, 37, 30], [1.0, 1.3, 1.6]
    dx = [h, h * 1.1, h * 1.2]
    gr = O.Grid(3, n, dx, dt, nkl, 15.0)
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=62, noise=1e-3)
    ref = O.run(gr, phi0, imag, 60)
    for shapes in SHAPES3:
        p = G.Propagator(3, n, dx, dt, nkl, 15.0, precision="f32")
        G.gp_set_shapes(p.h, *shapes)
        assert p.shapes()["flags"] & shapes[3] == shapes[3], (shapes, p.shapes())
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(60)
        got = p.get_state(device=False).astype(np.complex128)
        p.close()
        assert rel_l2(got, ref) <= (2e-5 if imag else 1e-4), (shapes, rel_l2(got, ref))
