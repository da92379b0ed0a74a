"""The symmetric (Strang) splitting of the CUDA path -- N(dt/2), the sweeps,
N(dt/2) -- against the FP64 oracle run with the same splitting.

Tolerances as for the Lie splitting: FP64 relative L2 <= 1e-12 after 1000
steps and |d mu| <= 1e-10; the FP32 form relative L2 2e-5 (imaginary time) /
1e-4 (real time) and |d mu| within the FP32 bound of tests/tolerances.py; the
double-float form 1e-12.
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


def make(G, dim, n, dx, dt, nkl, g, prec="f64", V=None):
    p = G.Propagator(dim, n, dx, dt, nkl, g, precision=prec)
    p.set_splitting("strang")
    gr = O.Grid(dim, n, dx, dt, nkl, g, V=V, split=1)
    if V is not None:
        p.set_potential(V)
    return p, gr


CASES = [
    (1, [17], [0.3]),
    (1, [256], [0.05]),
    (2, [33, 20], [0.25, 0.3]),
    (3, [17, 12, 9], [0.4, 0.45, 0.5]),
    (3, [40, 33, 24], [0.25, 0.3, 0.35]),
]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", CASES)
def test_one_step_elementwise_f64(G, dim, n, dx, imag):
    nkl = [1.0, 1.4, 1.8][:dim]
    p, gr = make(G, dim, n, dx, 2e-3, nkl, 12.0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=1714 + dim, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1)
    ref = O.step(gr, phi0, imag)
    assert np.max(np.abs(p.get_state(device=False) - ref)) <= 1e-13 * np.max(np.abs(ref))
    p.close()


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", [CASES[2], CASES[4]])
def test_1000_steps_f64(G, dim, n, dx, imag):
    nkl = [1.0, 1.4, 1.8][:dim]
    dt = 1e-3 if imag else 2e-4
    p, gr = make(G, dim, n, dx, dt, nkl, 20.0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=8, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    ref = O.run(gr, phi0, imag, 1000)
    assert rel_l2(p.get_state(device=False), ref) <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    for k in ("norm", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(ob[k] - obr[k]) <= 1e-11 * max(1.0, abs(obr[k]))
    p.close()


@pytest.mark.parametrize("prec", ["f32", "df64"])
@pytest.mark.parametrize("imag", [True, False])
def test_1000_steps_other_precisions(G, prec, imag):
    dim, n, dx, nkl = 3, [40, 33, 24], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8]
    dt = 1e-3 if imag else 2e-4
    p, gr = make(G, dim, n, dx, dt, nkl, 20.0, prec=prec)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=8, noise=1e-3)
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


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_user_potential(G, prec):
    """A Gaussian-bump potential: the per-point dt/2 factors, set before and
    after switching to the Strang splitting."""
    dim, n, dx, nkl = 2, [33, 20], [0.25, 0.3], [1.0, 1.4]
    gr0 = O.Grid(dim, n, dx, 1e-3, nkl, 15.0)
    dV, _ = I.gaussian_bumps(dim, n, dx, seed=5)
    V = O.potential(gr0) + dV
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=9, noise=1e-3)
    tol = 2e-5 if prec == "f32" else 1e-12
    for order in ("potential_first", "splitting_first"):
        p = G.Propagator(dim, n, dx, 1e-3, nkl, 15.0, precision=prec)
        if order == "potential_first":
            p.set_potential(V)
            p.set_splitting("strang")
        else:
            p.set_splitting("strang")
            p.set_potential(V)
        gr = O.Grid(dim, n, dx, 1e-3, nkl, 15.0, V=V, split=1)
        for imag in (True, False):
            p.set_state(phi0)
            (p.step_imag if imag else p.step_real)(200)
            got = p.get_state(device=False).astype(np.complex128)
            assert rel_l2(got, O.run(gr, phi0, imag, 200)) <= tol, (order, imag)
        p.close()


def test_long_lines_and_spherical(G):
    """Lines longer than the segmented kernels (thread-per-line sweeps) and
    the spherical trap's radial problem (weighted nonlinear term)."""
    dim, n, dx = 2, [600, 40], [0.05, 0.2]
    p, gr = make(G, dim, n, dx, 5e-4, [1.0, 1.2], 5.0)
    phi0 = I.gaussian_state(dim, n, dx, [1.0, 1.2], seed=24)
    p.set_state(phi0)
    p.step_imag(30)
    assert rel_l2(p.get_state(device=False), O.run(gr, phi0, True, 30)) <= 1e-13
    p.close()
    nr, dr = 257, 0.04
    r = np.arange(nr) * dr
    u0 = (np.sqrt(4 * np.pi) * r * np.exp(-0.6 * r ** 2)).astype(complex)
    for prec, tol in (("f64", 1e-12), ("f32", 2e-5), ("df64", 1e-12)):
        q = G.Propagator(1, [nr], [dr], 1e-3, [1.2], 40.0, precision=prec, spherical=True)
        q.set_splitting("strang")
        grs = O.Grid(1, [nr], [dr], 1e-3, [1.2], 40.0, geom=1, split=1)
        q.set_state(u0)
        q.step_imag(500)
        ref = O.run(grs, u0, True, 500)
        assert rel_l2(q.get_state(device=False).astype(np.complex128), ref) <= tol, prec
        q.close()


def test_second_order_in_dt(G):
    """Real time over t = 0.2 in 2d: against a dt/8 Strang run, halving dt
    cuts the Strang error by ~4 and the Lie error by ~2."""
    dim, n, dx, nkl = 2, [48, 40], [0.25, 0.25], [1.0, 1.3]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=10, noise=0.0)
    T, dts = 0.2, [4e-3, 2e-3, 1e-3]

    def run(dt, split):
        p = G.Propagator(dim, n, dx, dt, nkl, 30.0, precision="f64")
        p.set_splitting(split)
        p.set_state(phi0)
        p.step_real(int(round(T / dt)))
        out = p.get_state(device=False)
        p.close()
        return out

    fine = run(dts[-1] / 8, "strang")
    for split, order in (("strang", 2.0), ("lie", 1.0)):
        err = [np.linalg.norm(run(dt, split) - fine) for dt in dts]
        for i in range(len(dts) - 1):
            assert np.log2(err[i] / err[i + 1]) == pytest.approx(order, abs=0.15), (split, err)


def test_switching_back_and_rejections(G):
    dim, n, dx, nkl = 3, [17, 12, 9], [0.4, 0.45, 0.5], [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=11, noise=1e-3)
    a = G.Propagator(dim, n, dx, 1e-3, nkl, 10.0, precision="f64")
    b = G.Propagator(dim, n, dx, 1e-3, nkl, 10.0, precision="f64")
    a.set_splitting("strang")
    a.set_state(phi0)
    a.step_imag(40)                                  # graph captured with the Strang step
    a.set_splitting("lie")
    a.set_state(phi0)
    b.set_state(phi0)
    a.step_imag(40)
    b.step_imag(40)
    assert np.array_equal(a.get_state(device=False), b.get_state(device=False))
    a.set_splitting("strang")
    a.set_dt(5e-4)                                   # the dt/2 factors follow dt
    a.set_state(phi0)
    a.step_real(50)
    ref = O.run(O.Grid(dim, n, dx, 5e-4, nkl, 10.0, split=1), phi0, False, 50)
    assert rel_l2(a.get_state(device=False), ref) <= 1e-13
    with pytest.raises(G.GPError):
        G.gp_set_splitting(a.h, 2)
    with pytest.raises(G.GPError):
        G.gp_adjoint_forward(a.h, 4, 2)
    with pytest.raises(ValueError):
        a.set_splitting("yoshida")
    a.close()
    b.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 2e-6), ("df64", 1e-13)])
def test_real_time_halves_merged(G, prec, tol):
    """A run of real-time Strang steps merges the closing half of each step
    with the opening half of the next (one N(dt) between sweeps, N(dt/2) at
    both ends): the same result as lone steps, up to rounding, with one launch
    per sweep and a single closing launch."""
    dim, n, dx, nkl = 3, [24, 20, 18], [0.35, 0.35, 0.35], [1.0, 1.2, 1.4]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=12, noise=1e-3)
    a = G.Propagator(dim, n, dx, 5e-4, nkl, 30.0, precision=prec)
    b = G.Propagator(dim, n, dx, 5e-4, nkl, 30.0, precision=prec)
    for p in (a, b):
        p.set_splitting("strang")
        p.set_state(phi0)
    for _ in range(40):
        a.step_real(1)
    l0 = G.gp_kernel_launches()
    b.step_real(40)
    assert G.gp_kernel_launches() - l0 == 40 * dim + 1
    sa = a.get_state(device=False).astype(np.complex128)
    sb = b.get_state(device=False).astype(np.complex128)
    assert rel_l2(sb, sa) <= tol
    ref = O.run(O.Grid(dim, n, dx, 5e-4, nkl, 30.0, split=1), phi0, False, 40)
    assert rel_l2(sb, ref) <= (1e-12 if prec != "f32" else 1e-5)
    a.close()
    b.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5), ("df64", 1e-12)])
@pytest.mark.parametrize("env,fused", [({}, True), ({"GPE_KEEP": "0"}, True), ({"GPE_PIPE": "1"}, False)],
                         ids=["keep", "streamed", "pipelined"])
def test_imaginary_time_closing_half_fused_into_the_last_sweep(G, monkeypatch, env, fused, prec, tol):
    """2d/3d imaginary time: the closing N(dt/2) runs inside the last y/z sweep
    (one launch per sweep) or, for the pipelined y/z sweeps, in its own pass;
    both against the oracle."""
    if prec == "df64" and "GPE_PIPE" in env:
        pytest.skip("no pipelined double-float sweeps")
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    dim, n, dx, nkl = 3, [40, 33, 24], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8]
    p, gr = make(G, dim, n, dx, 1e-3, nkl, 20.0, prec=prec)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=13, noise=1e-3)
    p.set_state(phi0)
    l0 = G.gp_kernel_launches()
    p.step_imag(40)
    launches = G.gp_kernel_launches() - l0
    assert launches == 40 * (dim + (0 if fused else 1)) + 1
    ref = O.run(gr, phi0, True, 40)
    assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= tol
    p.close()
