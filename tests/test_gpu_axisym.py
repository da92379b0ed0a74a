"""Circularly symmetric 2d and axially symmetric 3d traps (rho on the
staggered grid rho_i = (i - 1/2) drho, non-symmetric Crank-Nicolson rows along
rho) against the FP64 oracle.

Tolerances as for the Cartesian grids: FP64 relative L2 <= 1e-12 after 1000
steps and |d mu| <= 1e-10; FP32 relative L2 2e-5 (imaginary) / 1e-4 (real)
and |d mu| within the FP32 bound of tests/tolerances.py; double-float 1e-12.
"""
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


def start(dim, n, dx, nkl, seed=0.0):
    rho = O.axisym_coords(n[0], dx[0])
    if dim == 1:
        return (np.exp(-0.5 * nkl[0] * rho ** 2) * (1 + 0.05 * np.cos(3 * rho + seed))).astype(complex)
    z = O.coords(n[1], dx[1])
    return (np.exp(-0.5 * (nkl[0] * rho[None, :] ** 2 + nkl[1] * (z[:, None] - 0.2) ** 2))
            * (1 + 0.05 * np.cos(3 * rho[None, :] + seed))).astype(complex)


CASES = [
    (1, [257], [0.03], [1.2]),          # circular, segmented one-warp sweep
    (1, [160], [0.05], [1.0]),          # even n
    (2, [96, 130], [0.08, 0.07], [1.0, 1.7]),    # axial, rho through the x tile
    (2, [33, 40], [0.25, 0.2], [1.3, 0.9]),
]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx,nkl", CASES)
def test_axisym_1000_steps_f64(G, dim, n, dx, nkl, imag):
    dt = 1e-3 if imag else 2e-4
    p = G.Propagator(dim, n, dx, dt, nkl, 30.0, precision="f64", axisym=True)
    gr = O.Grid(dim, n, dx, dt, nkl, 30.0, geom=2)
    phi0 = start(dim, n, dx, nkl)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    ref = O.run(gr, phi0, imag, 1000)
    assert rel_l2(p.get_state(device=False), ref) <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    for k in ("norm", "rms_x", "rms_y", "rms_r"):
        assert abs(ob[k] - obr[k]) <= 1e-11 * max(1.0, abs(obr[k])), k
    p.close()


def test_axial_without_the_x_tile(G, monkeypatch):
    """The rho axis through the one-warp-per-line sweep (tile off)."""
    monkeypatch.setenv("GPE_TILE_X", "0")
    dim, n, dx, nkl = CASES[2]
    for imag in (True, False):
        p = G.Propagator(dim, n, dx, 5e-4, nkl, 30.0, precision="f64", axisym=True)
        assert p.shapes()["tile_x"] == 0
        gr = O.Grid(dim, n, dx, 5e-4, nkl, 30.0, geom=2)
        phi0 = start(dim, n, dx, nkl, 1.0)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(300)
        assert rel_l2(p.get_state(device=False), O.run(gr, phi0, imag, 300)) <= 1e-12
        p.close()


@pytest.mark.parametrize("prec", ["f32", "df64"])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("case", [0, 2])
def test_axisym_other_precisions(G, case, prec, imag):
    dim, n, dx, nkl = CASES[case]
    dt = 1e-3 if imag else 2e-4
    p = G.Propagator(dim, n, dx, dt, nkl, 30.0, precision=prec, axisym=True)
    gr = O.Grid(dim, n, dx, dt, nkl, 30.0, geom=2)
    phi0 = start(dim, n, dx, nkl)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    ref = O.run(gr, phi0, imag, 1000)
    got = p.get_state(device=False).astype(np.complex128)
    if prec == "f32":
        assert rel_l2(got, ref) <= (2e-5 if imag else 1e-4)
    else:
        assert rel_l2(got, ref) <= 1e-12
    mu, mur = p.observables()["mu"], O.observables(gr, ref)["mu"]
    assert abs(mu - mur) <= (mu_tol_f32(mur) if prec == "f32" else 1e-10)
    p.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6), ("df64", 1e-12)])
@pytest.mark.parametrize("case", [1, 3])
def test_axisym_observables_of_a_state(G, case, prec, tol):
    dim, n, dx, nkl = CASES[case]
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 25.0, precision=prec, axisym=True)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 25.0, geom=2)
    phi = start(dim, n, dx, nkl, 0.5) * np.exp(0.3j * np.arange(int(np.prod(n))).reshape(gr.shape) / 50)
    p.set_state(phi)
    state = p.get_state(device=False).astype(np.complex128)
    ob, obr = p.observables(), O.observables(gr, state)
    for k in O.OBS_KEYS:
        assert ob[k] == pytest.approx(obr[k], rel=tol, abs=tol * 1e-2), k
    p.close()


def test_axisym_closed_forms_and_features(G):
    """g = 0: mu = nu (circular) and nu + lambda/2 (axial) to the grid's
    accuracy; Strang steps and reduced densities against the oracle."""
    p = G.Propagator(1, [161], [0.05], 1e-3, [1.3], 0.0, precision="f64", axisym=True)
    p.set_state(start(1, [161], [0.05], [1.3]))
    p.step_imag(12000)
    assert p.observables()["mu"] == pytest.approx(1.3, abs=5e-4)
    p.close()
    dim, n, dx, nkl = CASES[3]
    q = G.Propagator(dim, n, dx, 2e-3, nkl, 0.0, precision="f64", axisym=True)
    q.set_state(start(dim, n, dx, nkl))
    q.step_imag(6000)
    assert q.observables()["mu"] == pytest.approx(nkl[0] + nkl[1] / 2, abs=2e-2)
    q.close()
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 20.0, geom=2, split=1)
    phi0 = start(dim, n, dx, nkl)
    for imag in (True, False):
        s = G.Propagator(dim, n, dx, 1e-3, nkl, 20.0, precision="f64", axisym=True)
        s.set_splitting("strang")
        s.set_state(phi0)
        (s.step_imag if imag else s.step_real)(200)
        ref = O.run(gr, phi0, imag, 200)
        assert rel_l2(s.get_state(device=False), ref) <= 1e-12, imag
        state = s.get_state(device=False)
        for keep in ((0,), (1,)):
            red = s.reduced_density(keep, device=False)
            want = O.reduced_density(gr, state, keep)
            assert np.max(np.abs(red - want)) <= 1e-13 * np.max(want), keep
        s.close()


def test_axisym_rejections(G):
    with pytest.raises(G.GPError):
        G.Propagator(1, [600], [0.01], 1e-3, [1.0], 1.0, precision="f64", axisym=True)   # > 514 points
    p = G.Propagator(2, [40, 40], [0.2, 0.2], 1e-3, [1.0, 1.0], 1.0, precision="f64", axisym=True)
    for call in (lambda: G.gp_adjoint_forward(p.h, 4, 2), lambda: p.set_real_state(True),
                 lambda: G.gp_set_shapes(p.h, 1, 4, 4, G.GP_SHAPE_PIPE_X), lambda: G.gp_set_shapes(p.h, 0, 0, 4, 0)):
        with pytest.raises(G.GPError):
            call()
    p.close()
