"""The TMA-pipelined sweeps (GP_SHAPE_TMA_YZ, GP_SHAPE_TMA_X; FP32 states)
against the other sweeps and the FP64 oracle, and their bounded waits.

The per-line arithmetic is that of the register y/z sweeps (the same
increment-form recurrences and segment carries), so real-time runs -- which
carry no norm -- must be bit for bit those of the register kernel at the same
segment length.  In imaginary time the norm sums are accumulated per CTA in a
different order, so the renormalisation factor may differ in its last bit:
the runs are compared with the oracle instead (relative L2 as for the other
FP32 tests, |d mu| within the FP32 bound of tests/tolerances.py).  Grids
cover ragged x tiles (nx not a multiple of 32), 2d and 3d, lines of up to 256
points, and graph replays.
The x sweep's segments are aligned to even points (a different reassociation
from the register sweeps'), so it is held to the oracle only, including one
step element by element.  A wait made to run out (the test hook) must come
back as GP_ERR_TIMEOUT with the context still usable.
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


GRIDS = [
    (2, [64, 48], [0.2, 0.25]),
    (2, [34, 256], [0.3, 0.05]),
    (3, [40, 33, 24], [0.25, 0.3, 0.35]),
    (3, [96, 40, 130], [0.12, 0.3, 0.1]),
]


def shapes_for(G, p, tma, seg):
    s = p.shapes()
    flags = G.GP_SHAPE_TMA_YZ if tma else 0
    G.gp_set_shapes(p.h, s["tile_x"], s["seg_x"], seg, flags)
    got = p.shapes()
    assert bool(got["flags"] & G.GP_SHAPE_TMA_YZ) == tma
    return got


@pytest.mark.parametrize("seg", [8, 16])
@pytest.mark.parametrize("dim,n,dx", GRIDS)
def test_tma_yz_real_time_bitwise_equals_register_sweeps(G, dim, n, dx, seg):
    if max(n[1:]) - 2 > 16 * seg:
        pytest.skip("more than 16 segments per line")
    nkl = [1.0, 1.4, 1.8][:dim]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=41, noise=1e-3)
    out = []
    for tma in (False, True):
        p = G.Propagator(dim, n, dx, 2e-4, nkl, 20.0, precision="f32")
        shapes_for(G, p, tma, seg)
        p.set_state(phi0)
        p.step_real(40)                      # eager steps and one 16-step graph replay block
        out.append(p.get_state(device=False))
        p.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("dim,n,dx", GRIDS)
def test_tma_yz_imag_time_matches_oracle(G, dim, n, dx):
    nkl = [1.0, 1.4, 1.8][:dim]
    dt = 1e-3
    p = G.Propagator(dim, n, dx, dt, nkl, 20.0, precision="f32")
    seg = 16 if max(n[1:]) > 130 else 8
    shapes_for(G, p, True, seg)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=42, noise=1e-3)
    p.set_state(phi0)
    p.step_imag(200)
    got = p.get_state(device=False).astype(np.complex128)
    ob = p.observables()
    p.close()
    gr = O.Grid(dim, n, dx, dt, nkl, 20.0)
    ref = O.run(gr, phi0, True, 200)
    obr = O.observables(gr, ref)
    assert rel_l2(got, ref) <= 2e-5
    assert abs(ob["mu"] - obr["mu"]) <= mu_tol_f32(obr["mu"])
    assert abs(ob["norm"] - 1.0) <= 1e-6


def test_tma_yz_strang_closing_half_matches_oracle(G):
    dim, n, dx, nkl, dt = 3, [40, 33, 24], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8], 1e-3
    p = G.Propagator(dim, n, dx, dt, nkl, 20.0, precision="f32")
    p.set_splitting("strang")
    shapes_for(G, p, True, 8)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=43, noise=1e-3)
    p.set_state(phi0)
    p.step_imag(100)
    got = p.get_state(device=False).astype(np.complex128)
    p.close()
    gr = O.Grid(dim, n, dx, dt, nkl, 20.0, split=1)
    ref = O.run(gr, phi0, True, 100)
    assert rel_l2(got, ref) <= 2e-5


def test_tma_yz_full_size_quench_grid(G):
    """256^3 (dx = 0.08, dt = 2e-4, g = 40): the grid the TMA sweeps are for;
    two real-time steps bit for bit against the register sweeps."""
    import torch
    n, dx, nkl = [256] * 3, [0.08] * 3, [1.0] * 3
    phi0 = torch.tensor(I.gaussian_state(3, n, dx, nkl, seed=1711, noise=1e-3).astype(np.complex64), device="cuda")
    out = []
    for tma in (False, True):
        p = G.Propagator(3, n, dx, 2e-4, nkl, 40.0, precision="f32")
        shapes_for(G, p, tma, 16)
        p.set_state(phi0)
        p.step_real(2)
        out.append(p.get_state(device=True).clone())
        p.close()
    assert torch.equal(out[0], out[1])


def test_tma_shape_refused_where_it_does_not_fit(G):
    p = G.Propagator(3, [33, 20, 18], [0.3] * 3, 1e-3, [1.0] * 3, 5.0, precision="f32")   # nx odd
    with pytest.raises(G.GPError):
        G.gp_set_shapes(p.h, 1, 4, 8, G.GP_SHAPE_TMA_YZ)
    p.close()
    p = G.Propagator(3, [32, 20, 18], [0.3] * 3, 1e-3, [1.0] * 3, 5.0, precision="f64")   # FP64 state
    with pytest.raises(G.GPError):
        G.gp_set_shapes(p.h, 1, 4, 8, G.GP_SHAPE_TMA_YZ)
    p.close()


XGRIDS = [
    (2, [64, 48], [0.2, 0.25]),
    (2, [256, 34], [0.05, 0.3]),
    (2, [256, 40], [0.02, 0.3]),   # |alpha| ~ 0.4 along x: carries cross several segments (depth > 1)
    (3, [48, 33, 24], [0.25, 0.3, 0.35]),
    (3, [128, 40, 30], [0.1, 0.3, 0.35]),
]


def x_shapes(G, p, seg, yz_tma):
    s = p.shapes()
    flags = G.GP_SHAPE_TMA_X | (G.GP_SHAPE_TMA_YZ if yz_tma else 0)
    # the TMA y/z sweeps take 8- to 32-point segments, at most 16 per line
    seg_c = max(8, s["seg_c"]) if yz_tma else s["seg_c"]
    G.gp_set_shapes(p.h, 1, seg, seg_c, flags)
    assert p.shapes()["flags"] & G.GP_SHAPE_TMA_X


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", XGRIDS)
def test_tma_x_matches_oracle(G, dim, n, dx, imag):
    """The TMA x sweep (N and the pending renormalisation fused, segments
    aligned to even points) with the TMA y/z sweeps where they fit, against
    the oracle: FP32 tolerances of the other FP32 parity tests."""
    nkl = [1.0, 1.4, 1.8][:dim]
    dt = 1e-3 if imag else 2e-4
    p = G.Propagator(dim, n, dx, dt, nkl, 20.0, precision="f32")
    x_shapes(G, p, 16 if n[0] > 128 else 8, yz_tma=max(n[1:]) <= 256 and n[0] % 2 == 0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=44, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(200)
    got = p.get_state(device=False).astype(np.complex128)
    ob = p.observables()
    p.close()
    gr = O.Grid(dim, n, dx, dt, nkl, 20.0)
    ref = O.run(gr, phi0, imag, 200)
    obr = O.observables(gr, ref)
    assert rel_l2(got, ref) <= (2e-5 if imag else 1e-4)
    assert abs(ob["mu"] - obr["mu"]) <= mu_tol_f32(obr["mu"])


@pytest.mark.parametrize("imag", [True, False])
def test_tma_x_one_step_elementwise(G, imag):
    """One step element by element against the oracle (the x sweep's first
    and last points, the even-aligned segment joints and the ragged last tile
    of lines all included): FP32 rounding of one step."""
    dim, n, dx, nkl = 3, [48, 33, 20], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8]
    p = G.Propagator(dim, n, dx, 2e-3, nkl, 12.0, precision="f32")
    x_shapes(G, p, 8, yz_tma=False)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=45, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1)
    got = p.get_state(device=False).astype(np.complex128)
    p.close()
    ref = O.step(O.Grid(dim, n, dx, 2e-3, nkl, 12.0), phi0, imag)
    assert np.max(np.abs(got - ref)) <= 1e-6 * np.max(np.abs(ref))


def test_tma_x_user_potential_and_strang(G):
    dim, n, dx, nkl, dt = 3, [64, 40, 24], [0.2, 0.3, 0.35], [1.0, 1.3, 1.6], 5e-4
    gr = O.Grid(dim, n, dx, dt, nkl, 15.0, split=1)
    dV, _ = I.gaussian_bumps(dim, n, dx, seed=46)
    V = O.potential(gr) + dV
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=46, noise=1e-3)
    for imag in (True, False):
        p = G.Propagator(dim, n, dx, dt, nkl, 15.0, precision="f32")
        p.set_potential(V)
        p.set_splitting("strang")
        x_shapes(G, p, 8, yz_tma=True)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(100)
        got = p.get_state(device=False).astype(np.complex128)
        p.close()
        ref = O.run(O.Grid(dim, n, dx, dt, nkl, 15.0, V=V, split=1), phi0, imag, 100)
        assert rel_l2(got, ref) <= (2e-5 if imag else 1e-4)


def test_tma_x_full_size_quench_grid(G):
    """256^3 (dx = 0.08, dt = 2e-4, g = 40) with both TMA sweeps, two
    real-time steps against the register sweeps (different segment alignment
    along x, so FP32 rounding apart)."""
    import torch
    n, dx, nkl = [256] * 3, [0.08] * 3, [1.0] * 3
    phi0 = torch.tensor(I.gaussian_state(3, n, dx, nkl, seed=1711, noise=1e-3).astype(np.complex64), device="cuda")
    out = []
    for tma in (False, True):
        p = G.Propagator(3, n, dx, 2e-4, nkl, 40.0, precision="f32")
        if tma:
            x_shapes(G, p, 16, yz_tma=True)
        p.set_state(phi0)
        p.step_real(2)
        out.append(p.get_state(device=True).clone())
        p.close()
    d = torch.linalg.norm(out[1] - out[0]) / torch.linalg.norm(out[0])
    assert float(d) <= 1e-6


def test_tma_wait_that_runs_out_returns_gp_err_timeout(G, monkeypatch):
    """A TMA tile load that announces more bytes than it moves (the test hook)
    can never complete its wait: the sweep gives up after the wait limit
    (50 ms here), the next gp_observables returns GP_ERR_TIMEOUT, and the
    context stays usable -- a fresh handle on the same device steps and
    matches the oracle."""
    monkeypatch.setenv("GPE_WAIT_LIMIT_MS", "50")
    dim, n, dx, nkl = 3, [32, 20, 18], [0.3, 0.3, 0.3], [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=47, noise=1e-3)
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 10.0, precision="f32")
    x_shapes(G, p, 8, yz_tma=True)
    p.set_state(phi0)
    G.gp_test_stall_transfers(p.h, 16)
    p.step_imag(2)
    with pytest.raises(G.GPError) as e:
        p.observables()
    assert e.value.code == G.GP_ERR_TIMEOUT
    G.gp_test_stall_transfers(p.h, 0)
    p.set_state(phi0)
    p.step_imag(5)
    ob = p.observables()                      # the flag was cleared: no timeout now
    p.close()
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 10.0)
    assert abs(ob["mu"] - O.observables(gr, O.run(gr, phi0, True, 5))["mu"]) <= mu_tol_f32(ob["mu"])
