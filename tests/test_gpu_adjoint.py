"""Differentiation form: the hand-written adjoint of real-time propagation.

Checked three ways: against the CPU FP64 adjoint of the oracle (which keeps
the whole trajectory; different code, same mathematics), against central
finite differences through torch.autograd, and for independence from the
checkpoint interval.  The full-size case is the 3d real-time workload of the
differentiation form: 128^3, dx = 0.1, dt = 5e-4, 1000 steps, isotropic trap
plus a smooth random potential (8 Gaussian bumps, amplitude <= 0.5), g = 30,
checkpoints every 50 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1709_04423_gb300 import gpe
    gpe.load()
    return gpe


def problem(dim, n, dx, nkl, g, dt, seed):
    gr = O.Grid(dim, n, dx, dt, nkl, g)
    dV, bp = I.gaussian_bumps(dim, n, dx, seed=seed, count=4, amp=0.5, center=2.0)
    V = O.potential(gr) + dV
    phi0 = O.run(gr.with_(dt=5e-3), I.gaussian_state(dim, n, dx, nkl), True, 100)  # near a ground state
    target = I.gaussian_state(dim, n, dx, nkl, shift=(0.4, 0.0, 0.0))
    return gr.with_(V=V), V, phi0, target, bp


def gpu_adjoint(G, prec, gr, V, phi0, target, nsteps, K):
    import torch
    p = G.Propagator(gr.dim, gr.n[:gr.dim], gr.dx[:gr.dim], gr.dt, gr.nkl[:gr.dim], gr.g, precision=prec)
    p.set_potential(V)
    p.set_state(phi0)
    G.gp_adjoint_forward(p.h, nsteps, K)
    phiT = p.get_state(device=False).astype(np.complex128)
    dvol = float(np.prod(gr.dx[:gr.dim]))
    c = np.sum(np.conj(target) * phiT) * dvol
    J = abs(c) ** 2
    lam = torch.tensor((2 * c * target * dvol).astype(p.get_state(device=False).dtype), device="cuda")
    dJdV = torch.empty(gr.shape, dtype=torch.float64, device="cuda")
    lam0 = torch.empty_like(lam)
    dJdg = G.gp_adjoint_backward(p.h, lam.data_ptr(), 1, dJdV.data_ptr(), 1, lam0.data_ptr())
    p.close()
    return J, phiT, dJdV.cpu().numpy(), dJdg, lam0.cpu().numpy()


@pytest.mark.parametrize("dim,n,dx,nsteps,K", [
    (2, [24, 22], [0.4, 0.4], 40, 7),
    (3, [14, 12, 11], [0.5, 0.55, 0.6], 24, 5),
    (1, [64], [0.2], 50, 50),
])
def test_adjoint_matches_cpu_adjoint_f64(G, dim, n, dx, nsteps, K):
    nkl = [1.0, 1.2, 1.4][:dim]
    gr, V, phi0, target, _ = problem(dim, n, dx, nkl, 6.0, 5e-3, seed=1713)
    J, phiT, dJdV, dJdg, lam0 = gpu_adjoint(G, "f64", gr, V, phi0, target, nsteps, K)
    Jr, phiTr, dJdVr, dJdgr = O.adjoint_real(gr, phi0, target, nsteps)
    assert J == pytest.approx(Jr, rel=1e-12)
    assert np.max(np.abs(dJdV - dJdVr)) <= 1e-10 * np.max(np.abs(dJdVr))
    assert dJdg == pytest.approx(dJdgr, rel=1e-10)


def test_checkpoint_interval_does_not_change_the_gradient(G):
    gr, V, phi0, target, _ = problem(2, [30, 26], [0.35, 0.4], [1.0, 1.3], 9.0, 4e-3, seed=1714)
    res = [gpu_adjoint(G, "f64", gr, V, phi0, target, 33, K) for K in (1, 4, 33, 100)]
    for J, _, dJdV, dJdg, lam0 in res[1:]:
        assert J == res[0][0]
        assert np.max(np.abs(dJdV - res[0][2])) <= 1e-14 * np.max(np.abs(res[0][2]))
        assert dJdg == pytest.approx(res[0][3], rel=1e-13)
        assert np.max(np.abs(lam0 - res[0][4])) <= 1e-13 * np.max(np.abs(res[0][4]))


def test_adjoint_state_errors(G):
    p = G.Propagator(2, [16, 16], [0.3, 0.3], 1e-3, [1, 1], 1.0)
    import torch
    lam = torch.zeros((16, 16), dtype=torch.complex128, device="cuda")
    with pytest.raises(G.GPError) as e:
        G.gp_adjoint_backward(p.h, lam.data_ptr(), 1)
    assert e.value.code == G.GP_ERR_STATE
    p.set_state(I.gaussian_state(2, [16, 16], [0.3, 0.3], [1, 1]))
    G.gp_adjoint_forward(p.h, 10, 3)
    p.set_dt(2e-3)
    with pytest.raises(G.GPError) as e:
        G.gp_adjoint_backward(p.h, lam.data_ptr(), 1)
    assert e.value.code == G.GP_ERR_STATE
    p.close()


def torch_objective(G, prop, phi0, Vtrap, bumps, A, g, target, nsteps, K, dvol):
    import torch
    V = Vtrap + torch.einsum("k,k...->...", A, bumps)
    phiT = G.real_time_evolution(prop, phi0, V, g, nsteps, K)
    c = torch.sum(torch.conj(target) * phiT) * dvol
    return (c.real ** 2 + c.imag ** 2)


def test_autograd_function_matches_finite_differences(G):
    import torch
    dim, n, dx, nkl, dt, nsteps, K = 2, [28, 24], [0.4, 0.4], [1.0, 1.2], 4e-3, 30, 8
    gr0 = O.Grid(dim, n, dx, dt, nkl, 7.0)
    dV, bp = I.gaussian_bumps(dim, n, dx, seed=1715, count=4, amp=0.5, center=2.0)
    Vtrap = torch.tensor(O.potential(gr0), device="cuda")
    bumps = torch.tensor(np.stack(bp["bumps"]), device="cuda")
    A = torch.tensor(bp["A"], device="cuda", requires_grad=True)
    g = torch.tensor(7.0, dtype=torch.float64, device="cuda", requires_grad=True)
    phi0 = torch.tensor(O.run(gr0.with_(dt=5e-3), I.gaussian_state(dim, n, dx, nkl), True, 100), device="cuda",
                        requires_grad=True)
    target = torch.tensor(I.gaussian_state(dim, n, dx, nkl, shift=(0.4, 0.0, 0.0)), device="cuda")
    dvol = float(np.prod(dx))
    prop = G.Propagator(dim, n, dx, dt, nkl, 7.0, precision="f64")
    L = torch_objective(G, prop, phi0, Vtrap, bumps, A, g, target, nsteps, K, dvol)
    L.backward()
    gA, gg, gphi = A.grad.cpu().numpy(), float(g.grad), phi0.grad.cpu().numpy()
    h = 1e-5
    with torch.no_grad():
        def Lat(Ax=None, gx=None, ph=None):
            return float(torch_objective(G, prop, phi0 if ph is None else ph, Vtrap, bumps, A if Ax is None else Ax,
                                         g if gx is None else gx, target, nsteps, K, dvol))
        for k in range(4):
            e = torch.zeros(4, dtype=torch.float64, device="cuda")
            e[k] = h
            fd = (Lat(Ax=A + e) - Lat(Ax=A - e)) / (2 * h)
            assert gA[k] == pytest.approx(fd, rel=1e-6, abs=1e-10), k
        fd = (Lat(gx=g + h) - Lat(gx=g - h)) / (2 * h)
        assert gg == pytest.approx(fd, rel=1e-6)
        # directional derivative along a random complex perturbation of phi(0)
        u = I.uniform(77, 2 * int(np.prod(n))).reshape((2,) + tuple(reversed(n))) - 0.5
        d = torch.tensor(u[0] + 1j * u[1], device="cuda")
        fd = (Lat(ph=phi0 + h * d) - Lat(ph=phi0 - h * d)) / (2 * h)
        assert float(np.real(np.vdot(gphi, d.cpu().numpy()))) == pytest.approx(fd, rel=1e-6)
    prop.close()


def test_full_size_adjoint_finite_differences(G):
    """128^3, dx = 0.1, dt = 5e-4, 1000 steps, isotropic trap + 8 Gaussian
    bumps (amplitude <= 0.5), g = 30, checkpoints every 50 steps; FP64 adjoint
    against central finite differences in g and in two bump amplitudes, and
    the FP32 forward's gradient against the FP64 one."""
    import torch
    dim, n, dx, nkl, dt, nsteps, K, g = 3, [128] * 3, [0.1] * 3, [1.0] * 3, 5e-4, 1000, 50, 30.0
    gr0 = O.Grid(dim, n, dx, dt, nkl, g)
    dV, bp = I.gaussian_bumps(dim, n, dx, seed=1713, count=8, amp=0.5, center=3.0)
    Vtrap = O.potential(gr0)
    V = torch.tensor(Vtrap + dV, device="cuda")
    # phi(0): imaginary-time ground state at g = 30 in the trap without the bumps
    p = G.Propagator(dim, n, dx, 1e-3, nkl, g, precision="f64")
    p.set_state(I.gaussian_state(dim, n, dx, nkl, seed=1714, noise=1e-3))
    p.step_imag(2000)
    phi0 = p.get_state(device=True)
    p.close()
    target = torch.tensor(I.gaussian_state(dim, n, dx, nkl, shift=(0.5, 0.0, 0.0)), device="cuda")
    dvol = 0.1 ** 3

    def run(prec, Vv, gv, adjoint):
        q = G.Propagator(dim, n, dx, dt, nkl, gv, precision=prec)
        q.set_potential(Vv)
        q.set_state(phi0)
        G.gp_adjoint_forward(q.h, nsteps, K)
        phiT = q.get_state(device=True).to(torch.complex128)
        c = torch.sum(torch.conj(target) * phiT) * dvol
        J = float(c.real ** 2 + c.imag ** 2)
        out = None
        if adjoint:
            lam = (2 * c * target * dvol).to(q.ctype).contiguous()
            dJdV = torch.empty(tuple(n), dtype=torch.float64, device="cuda")
            dJdg = G.gp_adjoint_backward(q.h, lam.data_ptr(), 1, dJdV.data_ptr(), 1)
            out = (dJdV, dJdg)
        q.close()
        return J, out

    J, (dJdV, dJdg) = run("f64", V, g, True)
    h = 1e-4
    fd = (run("f64", V, g + h, False)[0] - run("f64", V, g - h, False)[0]) / (2 * h)
    assert dJdg == pytest.approx(fd, rel=1e-6)
    for k in (0, 5):
        Gk = torch.tensor(bp["bumps"][k], device="cuda")
        fd = (run("f64", V + h * Gk, g, False)[0] - run("f64", V - h * Gk, g, False)[0]) / (2 * h)
        assert float(torch.sum(dJdV * Gk)) == pytest.approx(fd, rel=1e-6), k
    J32, (dJdV32, dJdg32) = run("f32", V, g, True)
    assert J32 == pytest.approx(J, rel=1e-4)
    assert dJdg32 == pytest.approx(dJdg, rel=1e-3)
    assert float(torch.linalg.norm(dJdV32 - dJdV) / torch.linalg.norm(dJdV)) < 1e-3
