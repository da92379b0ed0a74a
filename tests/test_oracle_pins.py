"""Pins of the FP64 CPU oracle against what the mathematics fixes.

The paper names the method (split-step Crank-Nicolson, imaginary and real
time; "Solution method") and the quantities it reports (energy, chemical
potential, rms sizes, densities; abstract) but prints no formula and no worked
example, so every pin here is a closed form, an invariant, a brute-force dense
solve or a finite-difference check, chosen so that a dropped term, a wrong
sign, a wrong index or a transposed operand fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def rdot(a, b):
    """Real inner product <a, b> = Re sum conj(a) b."""
    return float(np.real(np.vdot(a.ravel(), b.ravel())))


def rand_complex(shape, seed):
    u = I.uniform(seed, 2 * int(np.prod(shape))).reshape((2,) + tuple(shape))
    return (u[0] - 0.5) + 1j * (u[1] - 0.5)


# ---------------------------------------------------------------- inputs / grid

def test_splitmix64_published_vector():
    lines = [l.strip() for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt"))
             if l.strip() and not l.startswith("#")]
    expect = [int(h, 16) for h in lines]
    got = [int(v) for v in I.splitmix64(0, len(expect))]
    assert got == expect


def test_grid_matches_stated_interval():
    # 1d workload: N = 256 points, dx = 0.05 on [-6.4, 6.4)
    x = O.coords(256, 0.05)
    assert x[0] == pytest.approx(-6.4, abs=1e-15)
    assert x[-1] == pytest.approx(6.4 - 0.05, abs=1e-14)
    assert np.allclose(np.diff(x), 0.05, atol=1e-15)


# ---------------------------------------------------------------- Simpson (R7)

@pytest.mark.parametrize("n", [5, 6, 17, 18, 101])
def test_simpson_exact_on_cubics(n):
    dx = 0.37
    w = O.simpson_weights(n, dx)
    x = O.coords(n, dx)
    m = n if n % 2 else n - 1
    a, b = x[0], x[m - 1]
    f = lambda t: 1.5 - 2.0 * t + 0.7 * t ** 2 + 0.3 * t ** 3
    F = lambda t: 1.5 * t - t ** 2 + 0.7 * t ** 3 / 3 + 0.3 * t ** 4 / 4
    assert np.dot(w, f(x)) == pytest.approx(F(b) - F(a), rel=1e-13, abs=1e-13)
    if n % 2 == 0:
        assert w[-1] == 0.0


def test_simpson_gaussian_normalised():
    for dx in (0.1, 0.05):
        n = int(round(20 / dx)) + 1
        x = O.coords(n, dx)
        w = O.simpson_weights(n, dx)
        assert np.dot(w, np.exp(-x ** 2) / np.sqrt(np.pi)) == pytest.approx(1.0, abs=1e-12)


# ---------------------------------------------------------------- sweeps (R5)

@pytest.mark.parametrize("imag", [False, True])
@pytest.mark.parametrize("dim,axis", [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_sweep_sine_mode_eigenfactor(imag, dim, axis):
    """A sine mode vanishing at both ends is an eigenvector of the held-zero
    discrete Laplacian; one CN sweep multiplies it by (1-z/2)/(1+z/2), with
    z = i dt E_k (real) or dt E_k (imag), E_k = 2 sin^2(k pi/(2(n-1)))/dx^2."""
    n = [9, 12, 7][:dim]
    dx = [0.3, 0.25, 0.4][:dim]
    dt = 0.02
    gr = O.Grid(dim, n, dx, dt)
    nd = n[axis]
    k = 3
    i = np.arange(nd)
    mode = np.sin(k * np.pi * i / (nd - 1))
    oshape = list(gr.shape)
    oshape[dim - 1 - axis] = 1             # arbitrary across the other axes
    other = rand_complex(oshape, 11)
    shape = [1] * dim
    shape[dim - 1 - axis] = nd
    phi = other * mode.reshape(shape)
    Ek = 2.0 * np.sin(k * np.pi / (2 * (nd - 1))) ** 2 / dx[axis] ** 2
    z = dt * Ek * (1.0 if imag else 1j)
    factor = (1 - z / 2) / (1 + z / 2)
    out = O.sweep(gr, phi, imag, axis)
    assert np.max(np.abs(out - factor * phi)) < 1e-14


def _cn_matrix(n, dx, dt, imag):
    """Full-line CN map (ends held at zero) built densely from H = -D^2/2."""
    M = n - 2
    T = (np.diag(2.0 * np.ones(M)) - np.diag(np.ones(M - 1), 1) - np.diag(np.ones(M - 1), -1)) / dx ** 2
    H = 0.5 * T
    z = dt * (1.0 if imag else 1j)
    A = np.eye(M) + 0.5 * z * H
    B = np.eye(M) - 0.5 * z * H
    C = np.linalg.solve(A, B)
    full = np.zeros((n, n), dtype=complex)
    full[1:-1, 1:-1] = C
    return full


@pytest.mark.parametrize("imag", [False, True])
@pytest.mark.parametrize("n", [3, 4, 9, 17])
def test_sweep_dense_solve_1d(imag, n):
    dx, dt = 0.2, 0.05
    gr = O.Grid(1, [n], [dx], dt)
    phi = rand_complex((n,), 5 + n)   # nonzero ends too: they are ignored
    out = O.sweep(gr, phi, imag, 0)
    ref = _cn_matrix(n, dx, dt, imag) @ phi
    assert np.max(np.abs(out - ref)) < 1e-13


def _phase_np(phi, V, g, dt, imag):
    th = dt * (V + g * np.abs(phi) ** 2)
    return np.exp(-th) * phi if imag else np.exp(-1j * th) * phi


@pytest.mark.parametrize("imag", [False, True])
def test_full_step_dense_2d(imag):
    n, dx, dt, g = [7, 9], [0.35, 0.3], 0.03, 2.5
    nkl = [1.0, 1.7]
    gr = O.Grid(2, n, dx, dt, nkl, g)
    phi = rand_complex(gr.shape, 3)
    V = O.potential(gr)
    Cx = _cn_matrix(n[0], dx[0], dt, imag)
    Cy = _cn_matrix(n[1], dx[1], dt, imag)
    u = _phase_np(phi, V, g, dt, imag)
    u = u @ Cx.T           # along x (last array axis)
    u = Cy @ u             # along y
    if imag:
        w = np.multiply.outer(O.simpson_weights(n[1], dx[1]), O.simpson_weights(n[0], dx[0]))
        u = u / np.sqrt(np.sum(w * np.abs(u) ** 2))
    out = O.step(gr, phi, imag)
    assert np.max(np.abs(out - u)) < 1e-13


@pytest.mark.parametrize("imag", [False, True])
def test_full_step_dense_3d(imag):
    n, dx, dt, g = [5, 6, 7], [0.4, 0.35, 0.3], 0.02, 1.5
    nkl = [1.0, 1.4, 1.8]
    gr = O.Grid(3, n, dx, dt, nkl, g)
    phi = rand_complex(gr.shape, 4)
    V = O.potential(gr)
    C = [_cn_matrix(n[d], dx[d], dt, imag) for d in range(3)]
    u = _phase_np(phi, V, g, dt, imag)
    u = np.einsum("ai,zyi->zya", C[0], u)
    u = np.einsum("bj,zjx->zbx", C[1], u)
    u = np.einsum("ck,kyx->cyx", C[2], u)
    if imag:
        w = np.einsum("k,j,i->kji", *[O.simpson_weights(n[d], dx[d]) for d in (2, 1, 0)])
        u = u / np.sqrt(np.sum(w * np.abs(u) ** 2))
    out = O.step(gr, phi, imag)
    assert np.max(np.abs(out - u)) < 1e-13


def test_potential_harmonic_values():
    gr = O.Grid(3, [4, 5, 6], [0.5, 0.4, 0.3], 0.1, [1.0, 1.4, 1.8])
    V = O.potential(gr)
    # corner (i, j, k) = (0, 0, 0): x = -1, y = -1, z = -0.9
    assert V[0, 0, 0] == pytest.approx(0.5 * (1.0 + 1.96 + 3.24 * 0.81), rel=1e-15)
    # i = n/2 sits at the origin for even n (x = z = 0); n = 5 has y[2] = -0.2
    assert V[3, 2, 2] == pytest.approx(0.5 * 1.96 * 0.2 ** 2, rel=1e-14)
    x = O.coords(4, 0.5); y = O.coords(5, 0.4); z = O.coords(6, 0.3)
    k, j, i = 5, 3, 1
    assert V[k, j, i] == pytest.approx(0.5 * (x[i] ** 2 + 1.96 * y[j] ** 2 + 3.24 * z[k] ** 2), rel=1e-15)


# ---------------------------------------------------------------- phase (R4)

def test_phase_real_time_keeps_modulus_and_composes():
    gr = O.Grid(2, [11, 13], [0.3, 0.25], 0.07, [1.0, 1.3], 4.0)
    phi = rand_complex(gr.shape, 8)
    one = O.phase(gr, phi, False)
    assert np.max(np.abs(np.abs(one) - np.abs(phi))) < 1e-15
    # |phi| is unchanged, so two half steps equal one full step
    half = gr.with_(dt=gr.dt / 2)
    two = O.phase(half, O.phase(half, phi, False), False)
    assert np.max(np.abs(two - one)) < 1e-14
    # and the step is undone by the step with -dt
    back = O.phase(gr.with_(dt=-gr.dt), one, False)
    assert np.max(np.abs(back - phi)) < 1e-14


def test_phase_imag_time_is_real_positive_decay():
    gr = O.Grid(1, [8], [0.5], 0.1, [1.0], 0.0)    # even n: x = 0 is a grid point
    phi = rand_complex(gr.shape, 9)
    out = O.phase(gr, phi, True)
    ratio = out / phi
    assert np.max(np.abs(ratio.imag)) < 1e-15
    V = O.potential(gr)
    # V = x^2/2 >= 0: the factor is at most 1 and equals 1 where V = 0
    assert np.all(ratio.real <= 1.0 + 1e-15)
    assert ratio.real[np.argmin(V)] == pytest.approx(1.0, abs=1e-15)
    order = np.argsort(V)
    assert np.all(np.diff(ratio.real[order]) <= 1e-15)   # larger V decays more


# ---------------------------------------------------------------- real time

def test_real_time_conserves_discrete_norm():
    gr = O.Grid(1, [64], [0.25], 0.01, [1.0], 5.0)
    phi = I.gaussian_state(1, [64], [0.25], [1.0], seed=21, noise=1e-2)
    phi[0] = phi[-1] = 0.0
    n0 = np.sum(np.abs(phi) ** 2)
    out = O.run(gr, phi, False, 10000)
    # unitary up to rounding: about one ulp of drift per step
    assert abs(np.sum(np.abs(out) ** 2) / n0 - 1.0) < 1e-11


def test_real_time_step_is_reversible():
    gr = O.Grid(3, [9, 10, 11], [0.4, 0.35, 0.3], 0.01, [1.0, 1.4, 1.8], 3.0)
    phi = rand_complex(gr.shape, 2)
    phi[0, :, :] = phi[-1, :, :] = 0
    phi[:, 0, :] = phi[:, -1, :] = 0
    phi[:, :, 0] = phi[:, :, -1] = 0
    fwd = O.step(gr, phi, False)
    back = fwd
    for d in (2, 1, 0):
        back = O.sweep(gr, back, False, d, sign=-1.0)
    back = O.phase(gr.with_(dt=-gr.dt), back, False)
    assert np.max(np.abs(back - phi)) < 1e-13


def test_real_time_energy_bounded():
    gr = O.Grid(2, [40, 40], [0.3, 0.3], 5e-3, [1.0, 1.0], 8.0)
    phi = I.gaussian_state(2, [40, 40], [0.3, 0.3], [1.0, 1.0])
    phi = O.run(gr, phi, True, 400)                     # near the ground state
    E0 = O.observables(gr, phi)["energy"]
    q = gr.with_(g=16.0)                                # quench: g -> 2g
    Eq0 = O.observables(q, phi)["energy"]
    Es = []
    for _ in range(10):
        phi = O.run(q, phi, False, 100)
        Es.append(O.observables(q, phi)["energy"])
    drift = np.abs(np.array(Es) - Eq0) / Eq0
    assert np.max(drift) < 5e-3          # O(dt) oscillation, no secular growth
    assert abs(Es[-1] - Eq0) / Eq0 < 5e-3
    assert Eq0 > E0


def test_ground_state_rotates_at_mu():
    """A stationary state evolves in real time as exp(-i mu t) phi; pins the sign
    of both sub-steps and the consistency of the mu functional."""
    g, n, dx = 10.0, 256, 0.05
    gr = O.Grid(1, [n], [dx], 1e-3, [1.0], g)
    phi = O.run(gr, I.gaussian_state(1, [n], [dx], [1.0]), True, 15000)
    mu = O.observables(gr, phi)["mu"]
    T = 0.5                                   # mu T near pi/2: signs well apart
    out = O.run(gr.with_(dt=1e-4), phi, False, 5000)
    rel = np.linalg.norm(out - np.exp(-1j * mu * T) * phi) / np.linalg.norm(phi)
    assert rel < 5e-4
    wrong = np.linalg.norm(out - np.exp(+1j * mu * T) * phi) / np.linalg.norm(phi)
    assert wrong > 1.0


def test_trap_quench_breathing_closed_form():
    """g = 0, Gaussian ground state of nu evolved in nu': <x^2>(t) =
    cos^2(nu' t)/(2 nu) + nu sin^2(nu' t)/(2 nu'^2)."""
    nu, nup = 1.0, 1.5
    n, dx, dt = 400, 0.04, 5e-4
    gr = O.Grid(1, [n], [dx], dt, [nup], 0.0)
    phi = I.gaussian_state(1, [n], [dx], [nu])
    for k in range(1, 7):
        phi = O.run(gr, phi, False, 500)
        t = k * 500 * dt
        ex = np.cos(nup * t) ** 2 / (2 * nu) + nu * np.sin(nup * t) ** 2 / (2 * nup ** 2)
        assert abs(O.observables(gr, phi)["rms_x"] ** 2 - ex) < 5e-4


# ---------------------------------------------------------------- observables (R8)

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_observables_on_analytic_gaussian(dim):
    """For psi = prod (nu_d/pi)^(1/4) exp(-nu_d x_d^2/2):
    kinetic = potential = sum nu_d/4, int |psi|^4 = prod sqrt(nu_d/(2 pi)),
    rms_d = 1/sqrt(2 nu_d)."""
    nkl = [1.0, 1.4, 1.8][:dim]
    dx = [0.08, 0.1, 0.1][:dim]
    n = [161, 121, 121][:dim]
    g = 7.0
    gr = O.Grid(dim, n, dx, 1e-3, nkl, g)
    phi = 2.0 * I.gaussian_state(dim, n, dx, nkl) * np.exp(0.3j)
    ob = O.observables(gr, phi)
    quart = np.prod([np.sqrt(v / (2 * np.pi)) for v in nkl])
    assert ob["norm"] == pytest.approx(4.0, rel=1e-9)
    # the derivative's truncation error is O(dx^4): ~1e-5 relative here
    assert ob["energy"] == pytest.approx(sum(nkl) / 2 + 0.5 * g * quart, rel=1e-4)
    assert ob["mu"] == pytest.approx(sum(nkl) / 2 + g * quart, rel=1e-4)
    for d in range(dim):
        assert ob["rms_" + "xyz"[d]] == pytest.approx(1 / np.sqrt(2 * nkl[d]), rel=1e-8)
    assert ob["rms_r"] == pytest.approx(np.sqrt(sum(1 / (2 * v) for v in nkl)), rel=1e-8)


def _poly_line(n, dx, coef):
    """A polynomial f (degree <= 4, complex coefficients) sampled on the R1
    grid, and the derivative the R8 stencils give for it, in closed form from
    the analytic derivatives (no finite differences): the 4th-order central
    difference is exact on quartics; the 2nd-order one at i = 1 and n - 2 is
    f' + h^2 f'''/6 exactly (its error series stops there on quartics); the
    end points carry 0."""
    P = np.polynomial.polynomial
    x = O.coords(n, dx)
    f = P.polyval(x, coef)
    d = P.polyval(x, P.polyder(coef))
    d3 = P.polyval(x, P.polyder(coef, 3))
    d[[1, n - 2]] += dx * dx / 6.0 * d3[[1, n - 2]]
    d[[0, n - 1]] = 0.0
    return f, d


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_kinetic_term_boundary_stencils_on_polynomials(dim):
    """R8's derivative branches pinned where they matter: a product of
    quartics with nonzero values at every index (including i = 0, 1, n-2,
    n-1).  With V = 0 and g = 0, E = mu = sum_q w_q |grad phi|_q^2 / 2 over
    sum_q w_q |phi_q|^2, the gradient from the closed form of _poly_line.  A
    wrong stencil, order or index at i = 1 / n - 2, or a nonzero end value,
    changes the sum."""
    n = [9, 12, 7][:dim]          # odd and even n (even: Simpson on n - 1 points)
    dx = [0.3, 0.25, 0.4][:dim]
    coefs = [np.array([0.7 + 0.2j, -0.4 + 0.9j, 0.35 - 0.1j, 0.08 + 0.05j, -0.03 + 0.02j]),
             np.array([1.1 - 0.3j, 0.5 + 0.2j, -0.6 + 0.4j, 0.1 - 0.07j, 0.04]),
             np.array([0.9, -0.2 - 0.5j, 0.3 + 0.3j, -0.05j, 0.02 - 0.01j])]
    lines = [_poly_line(n[d], dx[d], coefs[d]) for d in range(dim)]
    w = [O.simpson_weights(n[d], dx[d]) for d in range(dim)]
    # arrays in (z, y, x) order: axis d of the grid is array axis dim-1-d
    def outer(vs):
        out = np.ones((), dtype=np.complex128)
        for v in reversed(vs):
            out = np.multiply.outer(out, v)
        return out
    phi = outer([l[0] for l in lines])
    W = np.real(outer([wd.astype(np.complex128) for wd in w]))
    grad2 = np.zeros(phi.shape)
    for d in range(dim):
        comp = outer([lines[e][1] if e == d else lines[e][0] for e in range(dim)])
        grad2 += np.abs(comp) ** 2
    kin = 0.5 * np.sum(W * grad2)
    nrm = np.sum(W * np.abs(phi) ** 2)
    gr = O.Grid(dim, n, dx, 1e-3, [0.0] * dim, 0.0)
    ob = O.observables(gr, phi)
    assert ob["norm"] == pytest.approx(nrm, rel=1e-13)
    assert ob["energy"] == pytest.approx(kin / nrm, rel=1e-12)
    assert ob["mu"] == pytest.approx(kin / nrm, rel=1e-12)
    # the same state read with the 2nd-order stencil everywhere, or with the
    # boundary branch dropped (0 at i = 1, n - 2), gives a different kinetic
    # term: the pin separates the readings
    x0 = O.coords(n[0], dx[0])
    f0 = lines[0][0]
    alt = np.zeros(n[0], dtype=np.complex128)
    alt[1:-1] = (f0[2:] - f0[:-2]) / (2 * dx[0])
    assert not np.allclose(alt, lines[0][1], rtol=1e-6, atol=0)
    assert abs(lines[0][1][1]) > 1e-3 and abs(lines[0][1][n[0] - 2]) > 1e-3 and abs(x0[0]) > 0


def test_kinetic_term_is_fourth_order():
    """Halving dx divides the kinetic-energy error of a Gaussian by ~16."""
    errs = []
    for dx in (0.32, 0.16, 0.08):
        n = int(round(24 / dx)) + 1
        gr = O.Grid(1, [n], [dx], 1e-3, [1.0], 0.0)
        ob = O.observables(gr, I.gaussian_state(1, [n], [dx], [1.0]))
        errs.append(abs(ob["energy"] - 0.5))
    orders = [np.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(3.6 < o < 4.4 for o in orders), orders


def test_density_output():
    gr = O.Grid(2, [10, 12], [0.3, 0.3], 1e-3, [1, 1], 0.0)
    phi = rand_complex(gr.shape, 31)
    ob = O.observables(gr, phi, density=True)
    assert np.allclose(ob["density"], np.abs(phi) ** 2, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- imaginary time

def _ground(dim, n, dx, dt, nkl, g, steps):
    gr = O.Grid(dim, n, dx, dt, nkl, g)
    phi = O.run(gr, I.gaussian_state(dim, n, dx, nkl, seed=7, noise=1e-3), True, steps)
    return gr, phi, O.observables(gr, phi)


def test_harmonic_ground_state_1d_and_orders():
    """g = 0: mu = E = nu/2, rms = 1/sqrt(2 nu); rms converges at first order in
    dt and second order in dx."""
    res = {}
    for dx, dt in [(0.1, 1e-3), (0.1, 5e-4), (0.1, 2.5e-4), (0.2, 2.5e-4), (0.05, 2.5e-4)]:
        n = int(round(16 / dx))
        res[(dx, dt)] = _ground(1, [n], [dx], dt, [1.0], 0.0, int(12 / dt))[2]
    for ob in res.values():
        assert abs(ob["mu"] - 0.5) < 1.5e-4
        assert abs(ob["energy"] - ob["mu"]) < 1e-13
        assert abs(ob["rms_x"] - 1 / np.sqrt(2)) < 4e-3
    r = lambda dx, dt: res[(dx, dt)]["rms_x"]
    order_t = np.log2((r(0.1, 1e-3) - r(0.1, 5e-4)) / (r(0.1, 5e-4) - r(0.1, 2.5e-4)))
    order_x = np.log2((r(0.2, 2.5e-4) - r(0.1, 2.5e-4)) / (r(0.1, 2.5e-4) - r(0.05, 2.5e-4)))
    assert 0.8 < order_t < 1.2
    assert 1.7 < order_x < 2.3


def test_harmonic_ground_state_3d_anisotropic():
    nkl = [1.0, 1.4, 1.8]
    _, _, ob = _ground(3, [32, 28, 26], [0.25, 0.25, 0.25], 5e-3, nkl, 0.0, 2000)
    assert ob["mu"] == pytest.approx(sum(nkl) / 2, abs=3e-3)
    assert ob["energy"] == pytest.approx(ob["mu"], abs=1e-12)
    for d in range(3):
        assert ob["rms_" + "xyz"[d]] == pytest.approx(1 / np.sqrt(2 * nkl[d]), rel=2e-2)


def test_thomas_fermi_limit_1d():
    """mu_TF = (3 g nu / (4 sqrt 2))^(2/3) for norm 1; the relative error must
    shrink as g grows."""
    errs = []
    for g in (50.0, 200.0, 800.0, 3200.0):
        dx = 0.05 * (g / 50) ** (1 / 3)
        _, _, ob = _ground(1, [800], [dx], 2e-3, [1.0], g, 8000)
        errs.append(ob["mu"] / (3 * g / (4 * np.sqrt(2))) ** (2 / 3) - 1)
    assert all(e > 0 for e in errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4


def test_thomas_fermi_limit_2d_3d():
    _, _, ob = _ground(2, [96, 96], [0.25, 0.25], 2e-3, [1.0, 1.0], 600.0, 2500)
    mu2 = np.sqrt(600.0 / np.pi)
    assert abs(ob["mu"] / mu2 - 1) < 0.05
    _, _, ob3 = _ground(3, [40, 40, 40], [0.4, 0.4, 0.4], 4e-3, [1, 1, 1], 2000.0, 800)
    mu3 = 0.5 * (15 * 2000.0 / (4 * np.pi)) ** 0.4
    assert abs(ob3["mu"] / mu3 - 1) < 0.05


def test_imag_time_mu_from_norm_decay():
    """Near convergence one unnormalised step shrinks the norm by exp(-2 mu dt)."""
    dt = 1e-3
    gr, phi, ob = _ground(1, [256], [0.05], dt, [1.0], 10.0, 15000)
    u = O.phase(gr, phi, True)
    u = O.sweep(gr, u, True, 0)
    mu_decay = -np.log(O.norm(gr, u) / O.norm(gr, phi)) / (2 * dt)
    assert abs(mu_decay - ob["mu"]) < 20 * dt


# ---------------------------------------------------------------- adjoint

def test_adjoint_sweep_transpose():
    gr = O.Grid(3, [7, 8, 9], [0.3, 0.35, 0.4], 0.05)
    lam = rand_complex(gr.shape, 41)
    dl = rand_complex(gr.shape, 42)
    for axis in range(3):
        lhs = rdot(lam, O.sweep(gr, dl, False, axis))
        rhs = rdot(O.sweep(gr, lam, False, axis, sign=-1.0), dl)
        assert abs(lhs - rhs) < 1e-13 * max(1.0, abs(lhs))


def test_adjoint_phase_transpose_fd():
    gr = O.Grid(2, [9, 10], [0.3, 0.3], 0.05, [1.0, 1.5], 3.0)
    phi = rand_complex(gr.shape, 51)
    lam = rand_complex(gr.shape, 52)
    dphi = rand_complex(gr.shape, 53)
    dV = I.uniform(54, gr.npoints).reshape(gr.shape) - 0.5
    lam_in, dJdV, dJdg = O.adjoint_phase(gr, phi, lam)
    eps = 1e-6
    fd = (O.phase(gr, phi + eps * dphi, False) - O.phase(gr, phi - eps * dphi, False)) / (2 * eps)
    assert rdot(lam, fd) == pytest.approx(rdot(lam_in, dphi), rel=1e-7)
    V0 = O.potential(gr)
    fdV = (O.phase(gr.with_(V=V0 + eps * dV), phi, False) - O.phase(gr.with_(V=V0 - eps * dV), phi, False)) / (2 * eps)
    assert rdot(lam, fdV) == pytest.approx(float(np.sum(dJdV * dV)), rel=1e-7)
    fdg = (O.phase(gr.with_(g=gr.g + eps), phi, False) - O.phase(gr.with_(g=gr.g - eps), phi, False)) / (2 * eps)
    assert rdot(lam, fdg) == pytest.approx(dJdg, rel=1e-7)


def test_adjoint_gradient_matches_finite_differences():
    n, dx, dt, steps, g = [24, 22], [0.4, 0.4], 5e-3, 40, 6.0
    nkl = [1.0, 1.2]
    base = O.Grid(2, n, dx, dt, nkl, g)
    Vtrap = O.potential(base)
    dV, bp = I.gaussian_bumps(2, n, dx, seed=1713, count=4, amp=0.5, center=2.0)
    V = Vtrap + dV
    gr = base.with_(V=V)
    phi0 = O.run(base, I.gaussian_state(2, n, dx, nkl), True, 200)
    target = I.gaussian_state(2, n, dx, nkl, shift=(0.4, 0.0, 0.0))
    J, phiT, dJdV, dJdg = O.adjoint_real(gr, phi0, target, steps)
    assert J > 1e-3
    h = 1e-5
    Jp = O.adjoint_real(gr.with_(g=g + h), phi0, target, steps)[0]
    Jm = O.adjoint_real(gr.with_(g=g - h), phi0, target, steps)[0]
    assert dJdg == pytest.approx((Jp - Jm) / (2 * h), rel=1e-6)
    for k in range(4):
        Gk = bp["bumps"][k]
        Jp = O.adjoint_real(gr.with_(V=V + h * Gk), phi0, target, steps)[0]
        Jm = O.adjoint_real(gr.with_(V=V - h * Gk), phi0, target, steps)[0]
        assert float(np.sum(dJdV * Gk)) == pytest.approx((Jp - Jm) / (2 * h), rel=1e-6, abs=1e-12)


# ---------------------------------------------------------------- reduced densities (R12)

def _keeps(dim):
    import itertools
    return [k for r in range(1, dim + 1) for k in itertools.combinations(range(dim), r)]


def test_reduced_density_of_trap_ground_state_is_gaussian():
    """The g = 0 trap ground state prod_d (nu_d/pi)^(1/4) exp(-nu_d x^2/2)
    integrates over the dropped axes to prod_kept (nu/pi)^(1/2) exp(-nu x^2)
    (each dropped factor's Simpson integral is 1 to ~1e-12 at dx = 0.1)."""
    n, dx, nkl = [129, 121, 113], [0.1, 0.1, 0.1], [1.0, 1.4, 1.8]
    gr = O.Grid(3, n, dx, 1e-3, nkl, 0.0)
    xs = [O.coords(n[d], dx[d]) for d in range(3)]
    f = [(nkl[d] / np.pi) ** 0.25 * np.exp(-nkl[d] * xs[d] ** 2 / 2) for d in range(3)]
    phi = f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    for keep in _keeps(3):
        got = O.reduced_density(gr, phi, keep)
        want = np.ones(())
        for d in reversed(range(3)):
            if d in keep:
                want = np.multiply.outer(want, f[d] ** 2)
        assert np.max(np.abs(got - want)) <= 1e-9 * np.max(want), keep


@pytest.mark.parametrize("dim", [2, 3])
def test_reduced_density_factorises_on_product_states(dim):
    """For phi = prod_d f_d(x_d) with random complex factors the reduced
    density is prod_kept |f_d|^2 times prod_dropped (Simpson norm of f_d):
    pins which axis is summed, the weights used and the output layout."""
    n, dx = [9, 8, 7][:dim], [0.3, 0.25, 0.2][:dim]
    gr = O.Grid(dim, n, dx, 1e-3, [1.0] * dim, 0.0)
    f = [rand_complex((n[d],), 300 + d) for d in range(dim)]
    phi = np.ones(())
    for d in reversed(range(dim)):
        phi = np.multiply.outer(phi, f[d])
    norms = [float(np.dot(O.simpson_weights(n[d], dx[d]), np.abs(f[d]) ** 2)) for d in range(dim)]
    for keep in _keeps(dim):
        want = np.ones(())
        scale = 1.0
        for d in reversed(range(dim)):
            if d in keep:
                want = np.multiply.outer(want, np.abs(f[d]) ** 2)
            else:
                scale *= norms[d]
        got = O.reduced_density(gr, phi, keep)
        assert got.shape == want.shape
        assert np.allclose(got, want * scale, rtol=1e-13, atol=0), keep


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_reduced_density_integrates_to_the_norm(dim):
    """Integrating a reduced density over its kept axes gives the full Simpson
    norm (tensor-product weights), for every choice of kept axes."""
    n, dx = [11, 10, 9][:dim], [0.3, 0.25, 0.2][:dim]
    gr = O.Grid(dim, n, dx, 1e-3, [1.0] * dim, 0.0)
    phi = rand_complex(gr.shape, 310 + dim)
    N = O.norm(gr, phi)
    for keep in _keeps(dim):
        r = O.reduced_density(gr, phi, keep)
        kept = sorted(keep, reverse=True)        # array axes: outermost kept axis first
        while np.ndim(r) > 0:                    # contract the last array axis (smallest kept d)
            d = kept[np.ndim(r) - 1]
            r = r @ O.simpson_weights(n[d], dx[d])
        assert float(r) == pytest.approx(N, rel=1e-13), keep


# ---------------------------------------------------------------- spherical trap (R13)

def _sph_ground(n, dr, dt, nu, g, t_end):
    gr = O.Grid(1, [n], [dr], dt, [nu], g, geom=1)
    r = np.arange(n) * dr
    u0 = (np.sqrt(4 * np.pi) * r * np.exp(-0.6 * r ** 2)).astype(complex)   # not the ground state
    return gr, O.run(gr, u0, True, int(round(t_end / dt)))


def test_spherical_harmonic_ground_state():
    """g = 0, isotropic 3d trap: mu = E = 3 nu/2 and the rms radius is
    sqrt(3/(2 nu)); the kinetic integral of the exact state converges at
    second order or better in dr (the derivative at r = 0 from the odd
    extension of u)."""
    nu = 1.3
    gr, u = _sph_ground(321, 0.025, 1e-3, nu, 0.0, 12.0)
    ob = O.observables(gr, u)
    assert ob["mu"] == pytest.approx(1.5 * nu, abs=1e-4)
    assert ob["energy"] == pytest.approx(ob["mu"], abs=1e-14)
    assert ob["rms_x"] == pytest.approx(np.sqrt(1.5 / nu), abs=1e-3)
    errs = []
    for n, dr in ((321, 0.025), (641, 0.0125)):
        g2 = O.Grid(1, [n], [dr], 1e-3, [1.0], 0.0, geom=1)
        r = np.arange(n) * dr
        ue = (np.sqrt(4 * np.pi) * r * np.pi ** -0.75 * np.exp(-r ** 2 / 2)).astype(complex)
        ob = O.observables(g2, ue)
        assert ob["norm"] == pytest.approx(1.0, abs=1e-12)
        assert ob["rms_x"] == pytest.approx(np.sqrt(1.5), abs=1e-12)
        errs.append(abs(ob["energy"] - 1.5))
    assert errs[1] <= errs[0] / 4


def test_spherical_thomas_fermi_limit():
    """Large g: mu -> (1/2)(15 g nu^3/(4 pi))^(2/5), the error shrinking as g
    grows (pins the 1/(4 pi r^2) weight of the nonlinear term)."""
    rel = []
    for g in (200.0, 800.0, 3200.0):
        gr, u = _sph_ground(401, 0.03, 5e-4, 1.0, g, 8.0)
        mu_tf = 0.5 * (15 * g / (4 * np.pi)) ** 0.4
        rel.append(O.observables(gr, u)["mu"] / mu_tf - 1)
    assert all(r > 0 for r in rel) and rel[0] > rel[1] > rel[2] and rel[2] < 0.01


def test_spherical_real_time_conserves_norm():
    gr, u = _sph_ground(201, 0.04, 1e-3, 1.0, 50.0, 2.0)
    gr2 = gr.with_(g=100.0)
    n0 = O.norm(gr2, u)
    u1 = O.run(gr2, u, False, 2000)
    assert O.norm(gr2, u1) == pytest.approx(n0, rel=1e-12)


# ---------------------------------------------------------------- Strang splitting (R14)

def _quenched_ground(n, dx):
    phi0 = I.gaussian_state(1, [n], [dx], [1.3], seed=3, noise=1e-2)
    return O.run(O.Grid(1, [n], [dx], 1e-3, [1.0], 5.0), phi0, True, 10000)


def test_strang_real_time_is_second_order():
    """Real time after a quench (|phi| is invariant under N, so the half steps
    are exact): successive differences of phi(T = 1) shrink 4x per halving of
    dt for Strang (order 2) and 2x for Lie (order 1)."""
    n, dx = 201, 0.08
    gs = _quenched_ground(n, dx)
    for split, order in ((1, 2.0), (0, 1.0)):
        st = [O.run(O.Grid(1, [n], [dx], dt, [1.0], 10.0, split=split), gs, False, int(round(1.0 / dt)))
              for dt in (0.02, 0.01, 0.005, 0.0025)]
        d = [np.linalg.norm(st[i] - st[i + 1]) for i in range(3)]
        for i in range(2):
            assert np.log2(d[i] / d[i + 1]) == pytest.approx(order, abs=0.05), (split, i)


def test_strang_real_time_is_reversible():
    """The symmetric step undoes itself: S(-dt)^m S(dt)^m phi = phi (to
    rounding), which the Lie step does not (error ~5e-3 here)."""
    n, dx = 201, 0.08
    gs = _quenched_ground(n, dx)
    for split, tol in ((1, 1e-12), (0, None)):
        gr = O.Grid(1, [n], [dx], 0.01, [1.0], 10.0, split=split)
        back = O.run(gr.with_(dt=-0.01), O.run(gr, gs, False, 50), False, 50)
        err = np.linalg.norm(back - gs) / np.linalg.norm(gs)
        if tol:
            assert err <= tol
        else:
            assert err > 1e-4


def test_strang_step_is_half_phases_around_the_sweeps():
    """One Strang step = N(dt/2), the Lie sweeps, N(dt/2), then (imaginary
    time) renormalisation, composed from the oracle's own sub-steps."""
    dim, n, dx = 2, [12, 10], [0.3, 0.35]
    phi = rand_complex((10, 12), 77) * 0.5
    for imag in (True, False):
        gr = O.Grid(dim, n, dx, 4e-3, [1.0, 1.2], 7.0, split=1)
        half = gr.with_(dt=2e-3, split=0)
        want = O.phase(half, phi, imag)
        for d in range(dim):
            want = O.sweep(gr.with_(split=0), want, imag, d)
        want = O.phase(half, want, imag)
        if imag:
            want = want / np.sqrt(O.norm(gr, want))
        assert np.allclose(O.step(gr, phi, imag), want, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- circular and axial traps (R15)

def _gauss_rho(rho, nu):
    return np.sqrt(nu / np.pi) * np.exp(-nu * rho ** 2 / 2)


def test_axisym_grid_and_weights():
    """rho_i = (i - 1/2) drho with the phantom i = 0 at the mirror image of
    rho_1; the midpoint weights integrate 2 pi rho over [0, (n - 2) drho]
    exactly and 2 pi rho^3 to second order."""
    n, dr = 41, 0.1
    rho, w = O.axisym_coords(n, dr), O.axisym_weights(n, dr)
    assert rho[0] == pytest.approx(-rho[1]) and rho[1] == pytest.approx(0.05)
    assert w[0] == 0.0 and w[-1] == 0.0
    R = (n - 2) * dr
    assert np.sum(w) == pytest.approx(np.pi * R ** 2, rel=1e-13)
    e = [abs(np.sum(O.axisym_weights(m, R / (m - 2)) * O.axisym_coords(m, R / (m - 2)) ** 2) - np.pi * R ** 4 / 2)
         for m in (22, 42)]
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.01)


@pytest.mark.parametrize("imag", [True, False])
def test_rho_sweep_is_the_dense_cn_solve(imag):
    """One CN sweep along rho against a dense solve of (1 + A) u = (1 - A) p
    with A = r T, T's row k = (-(1 - h_k), 2, -(1 + h_k)), h_k = drho/(2 rho_k),
    on a small axial grid (every z line), ends held at zero."""
    nr, nz, dr, dz, dt = 7, 5, 0.3, 0.4, 0.05
    gr = O.Grid(2, [nr, nz], [dr, dz], dt, [1.0, 1.3], 2.0, geom=2)
    phi = rand_complex((nz, nr), 91)
    got = O.sweep(gr, phi, imag, 0)
    r = dt / (4 * dr * dr) * (1 if imag else 1j)
    rho = O.axisym_coords(nr, dr)
    M = nr - 2
    T = np.zeros((M, M))
    for a in range(M):
        k = a + 1
        h = dr / (2 * rho[k])
        T[a, a] = 2
        if a > 0:
            T[a, a - 1] = -(1 - h)
        if a < M - 1:
            T[a, a + 1] = -(1 + h)
    A = r * T
    for j in range(nz):
        p = phi[j, 1:-1]
        u = np.linalg.solve(np.eye(M) + A, (np.eye(M) - A) @ p)
        assert np.allclose(got[j, 1:-1], u, rtol=0, atol=1e-13)
        assert got[j, 0] == 0 and got[j, -1] == 0


def test_circular_harmonic_ground_state():
    """g = 0 circular trap: mu = E = nu, and the exact state
    sqrt(nu/pi) exp(-nu rho^2/2) has norm 1, energy nu and rms radius
    1/sqrt(nu) up to errors that shrink 4x per halving of drho (the even
    extension across the axis in the derivative)."""
    nu = 1.3
    n, dr = 161, 0.05
    gr = O.Grid(1, [n], [dr], 1e-3, [nu], 0.0, geom=2)
    rho = O.axisym_coords(n, dr)
    u = O.run(gr, np.exp(-0.5 * rho ** 2).astype(complex), True, 12000)
    ob = O.observables(gr, u)
    assert ob["mu"] == pytest.approx(nu, abs=5e-4)
    assert ob["energy"] == pytest.approx(ob["mu"], abs=1e-14)
    errs = []
    for m, h in ((161, 0.05), (321, 0.025)):
        g2 = O.Grid(1, [m], [h], 1e-3, [nu], 0.0, geom=2)
        ob = O.observables(g2, _gauss_rho(O.axisym_coords(m, h), nu).astype(complex))
        errs.append([abs(ob["norm"] - 1), abs(ob["energy"] - nu), abs(ob["rms_x"] - 1 / np.sqrt(nu))])
    for a, b in zip(*errs):
        assert a / b == pytest.approx(4.0, rel=0.05)


def test_axial_harmonic_ground_state():
    """g = 0 axial trap: the exact state has energy nu + lambda/2, rms_rho =
    1/sqrt(nu), rms_z = 1/sqrt(2 lambda) (errors second order or better); the
    imaginary-time ground state reaches mu = nu + lambda/2."""
    nu, lam = 1.2, 1.6
    errs = []
    for nr, nz, dr, dz in ((81, 64, 0.1, 0.15), (161, 128, 0.05, 0.075)):
        gr = O.Grid(2, [nr, nz], [dr, dz], 1e-3, [nu, lam], 0.0, geom=2)
        rho, z = O.axisym_coords(nr, dr), O.coords(nz, dz)
        ex = (_gauss_rho(rho, nu)[None, :] * (lam / np.pi) ** 0.25 * np.exp(-lam * z[:, None] ** 2 / 2)).astype(complex)
        ob = O.observables(gr, ex)
        assert ob["rms_y"] == pytest.approx(1 / np.sqrt(2 * lam), abs=1e-12)
        errs.append([abs(ob["norm"] - 1), abs(ob["energy"] - (nu + lam / 2)), abs(ob["rms_x"] - 1 / np.sqrt(nu))])
    for a, b in zip(*errs):   # second order or better (the z part converges faster)
        assert 3.5 <= a / b <= 5.0
    gr = O.Grid(2, [81, 64], [0.1, 0.15], 2e-3, [nu, lam], 0.0, geom=2)
    rho, z = O.axisym_coords(81, 0.1), O.coords(64, 0.15)
    u = O.run(gr, np.exp(-0.4 * (rho[None, :] ** 2 + z[:, None] ** 2)).astype(complex), True, 5000)
    assert O.observables(gr, u)["mu"] == pytest.approx(nu + lam / 2, abs=2e-3)


def test_circular_thomas_fermi_limit():
    """Large g: mu -> nu sqrt(g/pi) (2d Thomas-Fermi), the relative error
    shrinking as g grows (pins the 2 pi rho weight of the norm)."""
    rel = []
    for g in (100.0, 400.0, 1600.0):
        gr = O.Grid(1, [201], [0.05], 5e-4, [1.0], g, geom=2)
        rho = O.axisym_coords(201, 0.05)
        u = O.run(gr, np.exp(-0.1 * rho ** 2).astype(complex), True, 16000)
        rel.append(O.observables(gr, u)["mu"] / np.sqrt(g / np.pi) - 1)
    assert all(r > 0 for r in rel) and rel[0] > rel[1] > rel[2] and rel[2] < 0.005


def test_circular_real_time_conserves_the_rho_weighted_norm():
    """(1 + h_k) rho_k = (1 - h_{k+1}) rho_{k+1}: the rho operator is symmetric
    in the rho-weighted inner product, so CN keeps the midpoint norm (to
    rounding) through a quench; a transposed coefficient pair would not."""
    gr = O.Grid(1, [201], [0.04], 1e-3, [1.0], 20.0, geom=2)
    rho = O.axisym_coords(201, 0.04)
    u = O.run(gr, np.exp(-0.5 * rho ** 2).astype(complex), True, 3000)
    g2 = gr.with_(g=40.0)
    u1 = O.run(g2, u, False, 2000)
    assert O.norm(g2, u1) == pytest.approx(O.norm(g2, u), rel=1e-12)
    assert abs(O.observables(g2, u1)["rms_x"] - O.observables(g2, u)["rms_x"]) > 0.1   # it does breathe


def test_axial_ground_state_approaches_the_3d_cartesian_one():
    """An axial trap (nu, lambda) is the 3d trap (nu, nu, lambda): at g = 10
    the axial mu approaches the 3d Cartesian mu as drho shrinks, and the
    rms radius matches sqrt(rms_x^2 + rms_y^2)."""
    nu, lam, g = 1.0, 1.5, 10.0
    gr3 = O.Grid(3, [40] * 3, [0.3] * 3, 2e-3, [nu, nu, lam], g)
    u3 = O.run(gr3, I.gaussian_state(3, [40] * 3, [0.3] * 3, [nu, nu, lam]), True, 2500)
    ob3 = O.observables(gr3, u3)
    diffs = []
    for nr, nz, dr, dz in ((21, 40, 0.3, 0.3), (41, 80, 0.15, 0.15)):
        gra = O.Grid(2, [nr, nz], [dr, dz], 2e-3, [nu, lam], g, geom=2)
        rho, z = O.axisym_coords(nr, dr), O.coords(nz, dz)
        ua = O.run(gra, np.exp(-0.5 * (nu * rho[None, :] ** 2 + lam * z[:, None] ** 2)).astype(complex), True, 2500)
        oba = O.observables(gra, ua)
        diffs.append(abs(oba["mu"] - ob3["mu"]))
    assert diffs[1] < diffs[0] and diffs[1] < 3e-3 * ob3["mu"]
    assert oba["rms_x"] == pytest.approx(np.hypot(ob3["rms_x"], ob3["rms_y"]), rel=2e-3)
