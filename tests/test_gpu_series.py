"""Observables recorded during a run (gp_step_series) against the oracle and
against stepping + gp_observables."""
import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I

pytestmark = pytest.mark.gpu

KEYS = ("norm", "energy", "mu", "rms_x", "rms_y", "rms_z", "rms_r")


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1709_04423_gb300 import gpe
    gpe.load()
    assert torch.cuda.is_available()
    return gpe


def test_real_time_series_matches_oracle(G):
    """Breathing after a quench: records every 10 steps of a 3d real-time run
    against the oracle's observables of its own run at the same steps."""
    dim, n, dx, nkl = 3, [24, 22, 20], [0.35, 0.35, 0.35], [1.0, 1.2, 1.4]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=61)
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 20.0, precision="f64")
    p.set_state(phi0)
    rec = p.step_series(False, 105, 10, device=False)
    assert rec.shape == (10, 7)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 20.0)
    ref = phi0.copy()
    for r in range(10):
        ref = O.run(gr, ref, False, 10)
        ob = O.observables(gr, ref)
        for q, k in enumerate(KEYS):
            assert rec[r, q] == pytest.approx(ob[k], rel=1e-11, abs=1e-12), (r, k)
    ref = O.run(gr, ref, False, 5)                      # the 5 leftover steps
    assert np.linalg.norm(p.get_state(device=False) - ref) <= 1e-12 * np.linalg.norm(ref)
    p.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("imag", [True, False])
def test_series_equals_stepping_and_observables(G, prec, imag):
    dim, n, dx, nkl = 2, [40, 36], [0.25, 0.25], [1.0, 1.3]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=62, noise=1e-2)
    a = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision=prec)
    b = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision=prec)
    a.set_state(phi0)
    b.set_state(phi0)
    rec_d = a.step_series(imag, 70, 7, device=True).cpu().numpy()
    for r in range(10):
        (b.step_imag if imag else b.step_real)(7)
        ob = b.observables()
        for q, k in enumerate(KEYS):
            assert rec_d[r, q] == pytest.approx(ob[k], rel=1e-14, abs=1e-15), (r, k)
    if imag:
        assert np.allclose(rec_d[:, 0], 1.0, rtol=0, atol=(1e-6 if prec == "f32" else 1e-12))
    a.set_state(phi0)
    rec_h = a.step_series(imag, 70, 7, device=False)
    assert np.array_equal(rec_h, rec_d)
    a.close()
    b.close()


def test_series_edge_cases(G):
    dim, n, dx, nkl = 1, [64], [0.2], [1.0]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=63)
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 5.0, precision="f64")
    q = G.Propagator(dim, n, dx, 1e-3, nkl, 5.0, precision="f64")
    p.set_state(phi0)
    q.set_state(phi0)
    assert p.step_series(True, 5, 10, device=False).shape == (0, 7)   # no record, steps still run
    q.step_imag(5)
    assert np.array_equal(p.get_state(device=False), q.get_state(device=False))
    out = np.zeros(7)
    for args in ((True, -1, 1), (True, 10, 0), (False, 10, -3)):
        with pytest.raises(G.GPError):
            G.gp_step_series(p.h, args[0], args[1], args[2], out.ctypes.data, 0)
    p.close()
    q.close()
