"""Parity of the double-float form (GP_DF64) with the FP64 CPU oracle.

The double-float state carries about 48 significant bits (two floats), so
one step rounds at a few 2^-48 ~ 1e-14 relative, against 2^-53 for FP64; the
potential factors are exact triple-float images of the FP64 factors, so
nothing is rounded identically step after step beyond what FP64 itself
rounds.  The form is held to the FP64 bar: relative L2 <= 1e-12 on phi after
1000 steps and 1e-10 on mu; single steps element by element to 1e-13 of the
largest value.
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


def make(G, dim, n, dx, dt, nkl, g):
    p = G.Propagator(dim, n, dx, dt, nkl, g, precision="df64")
    gr = O.Grid(dim, n, dx, dt, nkl, g)
    return p, gr


CASES = [
    (1, [17], [0.3]),
    (1, [256], [0.05]),
    (2, [33, 20], [0.25, 0.3]),
    (2, [64, 48], [0.2, 0.2]),
    (3, [17, 12, 9], [0.4, 0.45, 0.5]),
    (3, [40, 33, 24], [0.25, 0.3, 0.35]),
]


def test_state_round_trip(G):
    """complex128 -> double-float -> complex128 keeps 48 bits."""
    dim, n, dx = 3, [20, 18, 16], [0.3, 0.3, 0.3]
    p, gr = make(G, dim, n, dx, 1e-3, [1.0, 1.0, 1.0], 0.0)
    u = I.uniform(5, 2 * gr.npoints).reshape((2,) + gr.shape)
    phi = (u[0] - 0.5) + 1j * (u[1] - 0.5)
    p.set_state(phi)
    back = p.get_state(device=False)
    assert back.dtype == np.complex128
    d = np.abs(back - phi)
    assert np.all(d <= 2.0 ** -47 * np.abs(phi) + 1e-300)
    p.close()


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", CASES)
def test_one_step_elementwise_df64(G, dim, n, dx, imag):
    nkl = [1.0, 1.4, 1.8][:dim]
    p, gr = make(G, dim, n, dx, 2e-3, nkl, 12.0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=1709 + dim, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1)
    got = p.get_state(device=False)
    ref = O.step(gr, phi0, imag)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    p.close()


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", [CASES[2], CASES[5]])
def test_1000_steps_df64(G, dim, n, dx, imag):
    nkl = [1.0, 1.4, 1.8][:dim]
    dt = 1e-3 if imag else 2e-4
    p, gr = make(G, dim, n, dx, dt, nkl, 20.0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=7, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    got = p.get_state(device=False)
    ref = O.run(gr, phi0, imag, 1000)
    err = rel_l2(got, ref)
    print(f"df64 {dim}d {n} imag={imag}: rel-L2 after 1000 steps {err:.3e}")
    assert err <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    p.close()


def test_large_nonlinear_phase_df64(G):
    """dt g |phi|^2 above 1/8 takes the FP64 branch of the sub-step N."""
    dim, n, dx = 2, [40, 36], [0.25, 0.25]
    p, gr = make(G, dim, n, dx, 2e-2, [1.0, 1.2], 60.0)
    phi0 = I.gaussian_state(dim, n, dx, [1.0, 1.2], seed=11) * 3.0
    assert 2e-2 * 60.0 * np.max(np.abs(phi0)) ** 2 > 0.125
    for imag in (True, False):
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(5)
        got = p.get_state(device=False)
        ref = O.run(gr, phi0, imag, 5)
        assert rel_l2(got, ref) <= 1e-13
    p.close()


def test_user_potential_and_quench_df64(G):
    dim, n, dx = 2, [48, 40], [0.25, 0.25]
    nkl = [1.0, 1.3]
    p, gr = make(G, dim, n, dx, 5e-4, nkl, 10.0)
    dV, _ = I.gaussian_bumps(dim, n, dx, seed=1713)
    V = O.potential(gr) + dV
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=3)
    p.set_state(phi0)
    p.set_potential(V)
    p.step_real(300)
    p.set_g(25.0)
    p.step_real(300)
    got = p.get_state(device=False)
    g1 = gr.with_(V=V)
    ref = O.run(g1, phi0, False, 300)
    ref = O.run(g1.with_(g=25.0), ref, False, 300)
    assert rel_l2(got, ref) <= 1e-12
    p.close()


def test_observables_df64(G):
    dim, n, dx = 3, [21, 18, 16], [0.3, 0.3, 0.3]
    p, gr = make(G, dim, n, dx, 1e-3, [1.0, 1.2, 1.5], 9.0)
    phi = I.gaussian_state(dim, n, dx, [1.0, 1.2, 1.5], seed=4, noise=1e-2)
    p.set_state(phi)
    ob = p.observables(density=True)
    obr = O.observables(gr, phi, density=True)
    for k in O.OBS_KEYS:
        assert ob[k] == pytest.approx(obr[k], rel=1e-13, abs=1e-15)
    p.close()


def test_df64_shapes_and_autotune(G):
    """Every x tile / y-z segment shape gives the same result; the tuner
    never offers the pipelined (FP32/FP64-only) shapes."""
    dim, n, dx = 3, [40, 33, 24], [0.25, 0.3, 0.35]
    nkl = [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=9, noise=1e-3)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 20.0)
    ref = O.run(gr, phi0, True, 40)
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 20.0, precision="df64")
    for tile, sx, sc, flags in [(1, 4, 4, 1), (1, 8, 8, 0), (1, 16, 16, 0), (0, 2, 4, 0)]:
        G.gp_set_shapes(p.h, tile, sx, sc, flags)
        p.set_state(phi0)
        p.step_imag(40)
        assert rel_l2(p.get_state(device=False), ref) <= 1e-13
    with pytest.raises(G.GPError):
        G.gp_set_shapes(p.h, 1, 8, 8, G.GP_SHAPE_PIPE_X)
    p.autotune(imag=True, nsteps=4, cache=False)
    assert not (p.shapes()["flags"] & (G.GP_SHAPE_PIPE_X | G.GP_SHAPE_PIPE_YZ))
    p.close()


def test_df64_limits(G):
    with pytest.raises(G.GPError):
        G.Propagator(1, [600], [0.01], 1e-4, [1.0], 1.0, precision="df64")
    p = G.Propagator(2, [24, 20], [0.3, 0.3], 1e-3, [1.0, 1.0], 1.0, precision="df64")
    with pytest.raises(G.GPError):
        G.gp_adjoint_forward(p.h, 4, 2)
    p.close()
    b = G.Batch([(16, 16)], [(0.1, 0.1)], 1e-3, [(1.0, 1.0)], [1.0], precision="df64")   # the batch takes it
    with pytest.raises(G.GPError):
        b.set_mode(1)                                     # but not its one-launch form (FP32 only)
    b.close()
