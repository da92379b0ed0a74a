"""Spherically symmetric trap (the radial problem for u = sqrt(4 pi) r phi)
against the FP64 oracle, and its closed-form g = 0 ground state."""
import numpy as np
import pytest

import oracle as O
from tolerances import mu_tol_f32

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


def u_start(n, dr, seed_shift=0.0):
    r = np.arange(n) * dr
    return (np.sqrt(4 * np.pi) * r * np.exp(-0.6 * (r - seed_shift) ** 2)).astype(complex)


@pytest.mark.parametrize("n,dr", [(257, 0.04), (600, 0.02)])   # segmented sweep; long-line kernel
@pytest.mark.parametrize("imag", [True, False])
def test_spherical_1000_steps_f64(G, n, dr, imag):
    dt, nu, g = (1e-3 if imag else 2e-4), 1.2, 40.0
    p = G.Propagator(1, [n], [dr], dt, [nu], g, precision="f64", spherical=True)
    gr = O.Grid(1, [n], [dr], dt, [nu], g, geom=1)
    u0 = u_start(n, dr)
    p.set_state(u0)
    (p.step_imag if imag else p.step_real)(1000)
    ref = O.run(gr, u0, imag, 1000)
    assert rel_l2(p.get_state(device=False), ref) <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    assert ob["rms_x"] == pytest.approx(obr["rms_x"], rel=1e-11)
    p.close()


@pytest.mark.parametrize("prec,tol", [("f32", 2e-5), ("df64", 1e-12)])
def test_spherical_other_precisions(G, prec, tol):
    n, dr, dt, nu, g = 257, 0.04, 1e-3, 1.0, 40.0
    p = G.Propagator(1, [n], [dr], dt, [nu], g, precision=prec, spherical=True)
    gr = O.Grid(1, [n], [dr], dt, [nu], g, geom=1)
    u0 = u_start(n, dr)
    p.set_state(u0)
    p.step_imag(1000)
    ref = O.run(gr, u0, True, 1000)
    assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= tol
    mur = O.observables(gr, ref)["mu"]
    assert abs(p.observables()["mu"] - mur) <= (mu_tol_f32(mur) if prec == "f32" else 1e-10)
    p.close()


def test_spherical_harmonic_ground_state(G):
    """g = 0: mu = E = 3 nu/2, rms radius sqrt(3/(2 nu)) (discretisation error
    below 1e-4 in mu at dr = 0.025)."""
    nu, n, dr = 1.3, 321, 0.025
    p = G.Propagator(1, [n], [dr], 1e-3, [nu], 0.0, precision="f64", spherical=True)
    p.set_state(u_start(n, dr))
    p.step_imag(12000)
    ob = p.observables()
    assert ob["mu"] == pytest.approx(1.5 * nu, abs=1e-4)
    assert ob["energy"] == pytest.approx(ob["mu"], abs=1e-13)
    assert ob["rms_x"] == pytest.approx(np.sqrt(1.5 / nu), abs=1e-3)
    assert ob["rms_y"] == 0.0 and ob["rms_z"] == 0.0
    p.close()


def test_spherical_observables_of_a_state(G):
    n, dr = 200, 0.05
    p = G.Propagator(1, [n], [dr], 1e-3, [1.0], 25.0, precision="f64", spherical=True)
    gr = O.Grid(1, [n], [dr], 1e-3, [1.0], 25.0, geom=1)
    r = np.arange(n) * dr
    u = (r * np.exp(-0.5 * r ** 2) * (1 + 0.3j * np.sin(r))).astype(complex)
    p.set_state(u)
    ob, obr = p.observables(), O.observables(gr, u)
    for k in O.OBS_KEYS:
        assert ob[k] == pytest.approx(obr[k], rel=1e-12, abs=1e-14), k
    with pytest.raises(G.GPError):
        G.gp_adjoint_forward(p.h, 4, 2)
    p.close()
