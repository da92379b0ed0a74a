"""A real imaginary-time state (gp_set_real_state) against the FP64 oracle and
against the complex state.

With real coefficients and a real sub-step N the real state computes the
complex path's real parts with the same operations; only the order in which
the last sweep adds up the norm differs (two x weights per packed complex
point), which moves the FP32 renormalisation factor by an FP32 rounding.
Tolerances: FP64 relative L2 <= 1e-12 against the oracle after 1000 steps,
|d mu| <= 1e-10; FP32 as for the complex FP32 form (2e-5, |d mu| within the
FP32 bound of tests/tolerances.py).
"""
import numpy as np
import pytest

import oracle as O
from tolerances import mu_tol_f32
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


CASES = [
    (2, [34, 21], [0.25, 0.3]),            # odd line count: a lone real line in the last tile column
    (2, [64, 48], [0.2, 0.2]),
    (3, [40, 33, 25], [0.25, 0.3, 0.35]),  # 825 x lines; y/z views with 20 points per row
    (3, [18, 12, 9], [0.4, 0.45, 0.5]),
]


@pytest.mark.parametrize("dim,n,dx", CASES)
def test_real_state_1000_steps_f64(G, dim, n, dx):
    nkl = [1.0, 1.4, 1.8][:dim]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=31 + dim, noise=1e-3)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 20.0)
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 20.0, precision="f64")
    p.set_state(phi0)
    p.set_real_state(True)
    p.step_imag(1000)
    got = p.get_state(device=False)
    ref = O.run(gr, phi0, True, 1000)
    assert np.all(got.imag == 0)
    assert rel_l2(got, ref) <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    for k in ("norm", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(ob[k] - obr[k]) <= 1e-11 * max(1.0, abs(obr[k]))
    p.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 2e-5)])
@pytest.mark.parametrize("dim,n,dx", [CASES[0], CASES[2]])
def test_real_state_matches_complex_state(G, dim, n, dx, prec, tol):
    """One step element by element, then 300 steps, against the complex path
    on the same real input (and the oracle)."""
    nkl = [1.0, 1.4, 1.8][:dim]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=41, noise=1e-3)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 25.0)
    a = G.Propagator(dim, n, dx, 1e-3, nkl, 25.0, precision=prec)
    b = G.Propagator(dim, n, dx, 1e-3, nkl, 25.0, precision=prec)
    a.set_state(phi0)
    b.set_state(phi0)
    a.set_real_state(True)
    a.step_imag(1)
    b.step_imag(1)
    sa, sb = a.get_state(device=False), b.get_state(device=False)
    assert np.max(np.abs(sa - sb)) <= (1e-15 if prec == "f64" else 2e-7) * np.max(np.abs(sb))
    a.step_imag(299)
    b.step_imag(299)
    sa = a.get_state(device=False).astype(np.complex128)
    sb = b.get_state(device=False).astype(np.complex128)
    assert rel_l2(sa, sb) <= tol
    ref = O.run(gr, phi0, True, 300)
    assert rel_l2(sa, ref) <= (1e-12 if prec == "f64" else 2e-5)
    mu_a, mu_r = a.observables()["mu"], O.observables(gr, ref)["mu"]
    assert abs(mu_a - mu_r) <= (1e-10 if prec == "f64" else mu_tol_f32(mu_r))
    a.close()
    b.close()


def test_real_state_user_potential_and_kernel_shapes(G, monkeypatch):
    """A Gaussian-bump potential, and the y/z input kept in registers or
    streamed, against the oracle."""
    dim, n, dx, nkl = 3, [40, 33, 25], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8]
    gr0 = O.Grid(dim, n, dx, 1e-3, nkl, 20.0)
    dV, _ = I.gaussian_bumps(dim, n, dx, seed=43)
    V = O.potential(gr0) + dV
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=44, noise=1e-3)
    ref = O.run(gr0.with_(V=V), phi0, True, 60)
    for env in ({}, {"GPE_SEG_YZ": "8", "GPE_KEEP": "0"}, {"GPE_SEG_X": "32", "GPE_SEG_YZ": "32"},
                {"GPE_PIPE": "1"}):
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        for prec, tol in (("f64", 1e-13), ("f32", 3e-6)):
            p = G.Propagator(dim, n, dx, 1e-3, nkl, 20.0, precision=prec)
            p.set_potential(V)
            p.set_state(phi0)
            p.set_real_state(True)
            p.step_imag(60)
            assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= tol, (env, prec)
            p.close()
        for k in env:
            monkeypatch.delenv(k)


def test_real_state_full_size_128cube(G):
    """The benchmark's grid (128^3, dx = 0.1, g = 50, dt = 1e-3): two FP32
    and two FP64 steps against the oracle."""
    n, dx, nkl = [128] * 3, [0.1] * 3, [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1710, noise=1e-3)
    ref = O.run(O.Grid(3, n, dx, 1e-3, nkl, 50.0), phi0, True, 2)
    for prec, tol in (("f64", 1e-13), ("f32", 2e-6)):
        p = G.Propagator(3, n, dx, 1e-3, nkl, 50.0, precision=prec)
        p.set_state(phi0)
        p.set_real_state(True)
        p.step_imag(2)
        assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= tol, prec
        p.close()


def test_real_state_series_reduced_density_and_switching(G):
    dim, n, dx, nkl = 2, [36, 30], [0.25, 0.25], [1.0, 1.3]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=45, noise=1e-2)
    a = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision="f64")
    b = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision="f64")
    a.set_state(phi0)
    b.set_state(phi0)
    a.set_real_state(True)
    rec_a = a.step_series(True, 70, 7, device=False)
    rec_b = b.step_series(True, 70, 7, device=False)
    assert np.allclose(rec_a, rec_b, rtol=1e-13, atol=1e-14)
    ra, rb = a.reduced_density((0,), device=False), b.reduced_density((0,), device=False)
    assert np.allclose(ra, rb, rtol=1e-13, atol=1e-15)
    a.set_real_state(False)                     # back to complex: real-time steps allowed again
    a.step_real(20)
    b.step_real(20)
    assert rel_l2(a.get_state(device=False), b.get_state(device=False)) <= 1e-13
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision="f64")
    p.set_state(phi0 * np.exp(0.3j))            # not real: refused, complex state kept
    with pytest.raises(G.GPError):
        p.set_real_state(True)
    p.set_state(phi0)
    p.set_real_state(True)
    for call in (lambda: p.step_real(1), lambda: p.set_splitting("strang"), lambda: G.gp_adjoint_forward(p.h, 4, 2),
                 lambda: G.gp_set_real_state(p.h, 2), lambda: G.gp_autotune(p.h, 0, 4)):
        with pytest.raises(G.GPError):
            call()
    before = p.get_state(device=False)
    p.autotune(True, nsteps=2, cache=False)     # real-state shapes; the state is put back
    assert np.array_equal(p.get_state(device=False), before)
    assert p.shapes()["tile_x"] == 1 and p.shapes()["flags"] & (G.GP_SHAPE_PIPE_X | G.GP_SHAPE_PIPE_YZ) == 0
    with pytest.raises(G.GPError):              # complex input while real: refused, real mode left
        p.set_state(phi0 * 1j)
    p.step_real(1)                              # complex again
    p.close()
    for args in ((1, [64], [0.2]), (2, [33, 20], [0.3, 0.3])):   # 1d; odd nx
        q = G.Propagator(args[0], args[1], args[2], 1e-3, [1.0, 1.0][:args[0]], 1.0, precision="f64")
        with pytest.raises(G.GPError):
            q.set_real_state(True)
        q.close()
    q = G.Propagator(2, [32, 20], [0.3, 0.3], 1e-3, [1.0, 1.0], 1.0, precision="df64")
    with pytest.raises(G.GPError):
        q.set_real_state(True)
    q.close()
    a.close()
    b.close()
