"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Inputs are seeded and synthetic (trapped Gaussian condensate plus noise,
harmonic traps, Gaussian-bump potentials).  Tolerances: the FP64 path must
match the oracle to a relative L2 error <= 1e-12 on phi after 1000 steps and
to 1e-10 on mu; single steps are compared element by element.  The FP32 form
is held to |d mu| <= 1e-6 at the end of the 128^3 job and, part way through a
run, to the FP32 bound of tests/tolerances.py, with a relative L2 error that
FP32 rounding allows.
"""
import numpy as np
import pytest

import oracle as O
from paper_1709_04423_gb300 import inputs as I
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


def make(G, dim, n, dx, dt, nkl, g, prec="f64"):
    p = G.Propagator(dim, n, dx, dt, nkl, g, precision=prec)
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


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dim,n,dx", CASES)
def test_one_step_elementwise_f64(G, dim, n, dx, imag):
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
def test_1000_steps_f64(G, dim, n, dx, imag):
    nkl = [1.0, 1.4, 1.8][:dim]
    dt = 1e-3 if imag else 2e-4
    p, gr = make(G, dim, n, dx, dt, nkl, 20.0)
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=7, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    got = p.get_state(device=False)
    ref = O.run(gr, phi0, imag, 1000)
    assert rel_l2(got, ref) <= 1e-12
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert abs(ob["energy"] - obr["energy"]) <= 1e-10
    for k in ("norm", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(ob[k] - obr[k]) <= 1e-11 * max(1.0, abs(obr[k]))
    p.close()


def test_1d_ground_state_workload_f64(G):
    """1d imaginary time: N = 256, dx = 0.05 on [-6.4, 6.4), dt = 1e-4,
    V = x^2/2, g = 10, 20000 steps, Gaussian plus 1e-3 seeded noise."""
    n, dx, dt, g = [256], [0.05], 1e-4, 10.0
    p, gr = make(G, 1, n, dx, dt, [1.0], g)
    phi0 = I.gaussian_state(1, n, dx, [1.0], seed=1709, noise=1e-3)
    p.set_state(phi0)
    p.step_imag(20000)
    got = p.get_state(device=False)
    ref = O.run(gr, phi0, True, 20000)
    assert rel_l2(got, ref) <= 1e-12
    ob = p.observables(density=True)
    obr = O.observables(gr, ref, density=True)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    assert np.max(np.abs(ob["density"].cpu().numpy() - obr["density"])) <= 1e-12 * obr["density"].max()
    p.close()


@pytest.mark.parametrize("imag", [True, False])
def test_fp32_form_mu_error(G, imag):
    dim, n, dx = 3, [40, 33, 24], [0.25, 0.3, 0.35]
    nkl = [1.0, 1.4, 1.8]
    dt = 1e-3 if imag else 2e-4
    p, gr = make(G, dim, n, dx, dt, nkl, 20.0, prec="f32")
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=7, noise=1e-3)
    p.set_state(phi0)
    (p.step_imag if imag else p.step_real)(1000)
    got = p.get_state(device=False).astype(np.complex128)
    ref = O.run(gr, phi0, imag, 1000)
    assert rel_l2(got, ref) <= (2e-5 if imag else 1e-4)
    ob, obr = p.observables(), O.observables(gr, ref)
    assert abs(ob["mu"] - obr["mu"]) <= mu_tol_f32(obr["mu"])
    p.close()


def test_observables_random_state_f64(G):
    dim, n, dx = 3, [21, 18, 16], [0.3, 0.3, 0.3]
    p, gr = make(G, dim, n, dx, 1e-3, [1.0, 1.2, 1.5], 9.0)
    u = I.uniform(99, 2 * gr.npoints).reshape((2,) + gr.shape)
    phi = (u[0] - 0.5) + 1j * (u[1] - 0.5)
    p.set_state(phi)
    ob = p.observables()
    obr = O.observables(gr, phi)
    for k in O.OBS_KEYS:
        assert ob[k] == pytest.approx(obr[k], rel=1e-12, abs=1e-14)
    p.close()


def test_user_potential_and_quench(G):
    dim, n, dx = 2, [48, 40], [0.25, 0.25]
    nkl = [1.0, 1.3]
    p, gr = make(G, dim, n, dx, 5e-4, nkl, 10.0)
    dV, _ = I.gaussian_bumps(dim, n, dx, seed=1713)
    V = O.potential(gr) + dV
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=3)
    p.set_state(phi0)
    p.set_potential(V)
    p.step_real(50)
    p.set_g(25.0)
    p.step_real(50)
    p.set_dt(2.5e-4)
    p.step_imag(40)
    grV = gr.with_(V=V)
    ref = O.run(grV, phi0, False, 50)
    ref = O.run(grV.with_(g=25.0), ref, False, 50)
    ref = O.run(grV.with_(g=25.0, dt=2.5e-4), ref, True, 40)
    got = p.get_state(device=False)
    assert rel_l2(got, ref) <= 1e-12
    ob, obr = p.observables(), O.observables(grV.with_(g=25.0), ref)
    assert abs(ob["mu"] - obr["mu"]) <= 1e-10
    p.set_potential(None)   # back to the harmonic trap
    p.step_real(5)
    ref = O.run(gr.with_(g=25.0, dt=2.5e-4), ref, False, 5)
    assert rel_l2(p.get_state(device=False), ref) <= 1e-12
    p.close()


def test_device_state_roundtrip_and_stream(G):
    import torch
    dim, n, dx = 3, [20, 16, 12], [0.3, 0.3, 0.3]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p = G.Propagator(dim, n, dx, 1e-3, [1, 1, 1], 5.0, precision="f64", stream=s)
        phi0 = torch.tensor(I.gaussian_state(dim, n, dx, [1, 1, 1], seed=5), device="cuda")
        p.set_state(phi0)
        p.step_imag(37)
        out = p.get_state(device=True)
    s.synchronize()
    gr = O.Grid(dim, n, dx, 1e-3, [1, 1, 1], 5.0)
    ref = O.run(gr, phi0.cpu().numpy(), True, 37)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-13
    p.close()


def test_nonfinite_state_is_reported(G):
    p, gr = make(G, 2, [16, 16], [0.3, 0.3], 1e-3, [1, 1], 1.0)
    phi = I.gaussian_state(2, [16, 16], [0.3, 0.3], [1, 1])
    phi[5, 7] = np.nan
    p.set_state(phi)
    with pytest.raises(G.GPError) as e:
        p.observables()
    assert e.value.code == G.GP_ERR_NONFINITE
    p.close()


def test_zero_steps_and_graph_boundaries(G):
    """Step counts around the graph block size give the same result as one-by-one."""
    dim, n, dx = 2, [24, 20], [0.3, 0.3]
    phi0 = I.gaussian_state(dim, n, dx, [1, 1], seed=11)
    res = []
    for chunks in ([0, 33], [1] * 33, [31, 2], [32, 1]):
        p, gr = make(G, dim, n, dx, 1e-3, [1, 1], 4.0)
        p.set_state(phi0)
        for c in chunks:
            p.step_imag(c)
        res.append(p.get_state(device=False))
        p.close()
    for r in res[1:]:
        assert rel_l2(r, res[0]) <= 1e-14


@pytest.mark.parametrize("imag", [True, False])
def test_full_size_128cube_two_steps(G, imag):
    """3d 128^3 anisotropic trap (dx = 0.1, nu, kappa, lambda = 1, 1.4, 1.8,
    g = 50), the size the benchmark runs: two steps against the oracle."""
    n, dx, nkl = [128] * 3, [0.1] * 3, [1.0, 1.4, 1.8]
    for prec in ("f64", "f32"):
        p, gr = make(G, 3, n, dx, 1e-3, nkl, 50.0, prec=prec)
        phi0 = I.gaussian_state(3, n, dx, nkl, seed=1710, noise=1e-3)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(2)
        got = p.get_state(device=False).astype(np.complex128)
        ref = O.run(gr, phi0, imag, 2)
        assert rel_l2(got, ref) <= (1e-14 if prec == "f64" else 2e-6)
        p.close()


def test_full_size_256cube_quench_two_steps(G):
    """The 256^3 real-time quench grid (dx = 0.08, isotropic trap, g = 40, dt =
    2e-4) in the shapes the benchmark's autotuner picks for it (the pipelined
    y/z sweeps among the candidates): two real-time steps of every precision
    form against the oracle."""
    n, dx, nkl = [256] * 3, [0.08] * 3, [1.0] * 3
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1711, noise=1e-3)
    ref = O.run(O.Grid(3, n, dx, 2e-4, nkl, 40.0), phi0, False, 2)
    for prec, tol in (("f64", 1e-13), ("f32", 2e-6), ("df64", 1e-13)):
        p = G.Propagator(3, n, dx, 2e-4, nkl, 40.0, precision=prec)
        p.autotune(imag=False, cache=False)
        p.set_state(phi0)
        p.step_real(2)
        assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= tol, (prec, p.shapes())
        p.close()


SHAPES = [
    {"GPE_SEG_X": "0", "GPE_SEG_YZ": "0"},                     # thread-per-line kernels
    {"GPE_TILE_X": "0"},                                       # warp-per-line x sweep
    {"GPE_TILE_X": "0", "GPE_SEG_X": "2", "GPE_SEG_YZ": "16"},
    {},                                                        # default shapes
    {"GPE_SEG_X": "4", "GPE_SEG_YZ": "4"},
    {"GPE_SEG_X": "16", "GPE_SEG_YZ": "8"},
    {"GPE_SEG_X": "32", "GPE_SEG_YZ": "32"},
    {"GPE_SEG_YZ": "8", "GPE_KEEP": "0"},                      # y/z input streamed and re-read
    {"GPE_PIPE": "1"},                                         # persistent double-buffered sweeps
    {"GPE_PIPE": "1", "GPE_SEG_X": "4", "GPE_SEG_YZ": "16"},
]


@pytest.mark.parametrize("env", SHAPES, ids=lambda e: "-".join(f"{k[4:]}{v}" for k, v in e.items()) or "default")
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_every_kernel_shape_matches_oracle(G, monkeypatch, env, prec):
    """All line-segment shapes the autotuner may pick (and the thread-per-line
    kernels kept for long lines) give the oracle's result."""
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    dim, n, dx = 3, [40, 33, 24], [0.25, 0.3, 0.35]
    nkl = [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=17, noise=1e-3)
    for imag in (True, False):
        dt = 1e-3 if imag else 2e-4
        p, gr = make(G, dim, n, dx, dt, nkl, 20.0, prec=prec)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(40)
        got = p.get_state(device=False).astype(np.complex128)
        ref = O.run(gr, phi0, imag, 40)
        assert rel_l2(got, ref) <= (1e-13 if prec == "f64" else 3e-6), (imag, rel_l2(got, ref))
        p.close()


def test_long_lines_use_fallback_kernels(G):
    """Lines longer than the segmented kernels take (n = 600 along x and y)."""
    dim, n, dx = 2, [600, 530], [0.05, 0.05]
    p, gr = make(G, dim, n, dx, 5e-4, [1.0, 1.2], 5.0)
    phi0 = I.gaussian_state(dim, n, dx, [1.0, 1.2], seed=23)
    p.set_state(phi0)
    p.step_real(3)
    ref = O.run(gr, phi0, False, 3)
    assert rel_l2(p.get_state(device=False), ref) <= 1e-13
    p.close()


def test_autotune_picks_valid_shapes_and_keeps_parity(G, tmp_path, monkeypatch):
    import json
    monkeypatch.setenv("GPE_TUNE_CACHE", str(tmp_path / "shapes.json"))
    dim, n, dx = 3, [40, 33, 24], [0.25, 0.3, 0.35]
    nkl = [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=19, noise=1e-3)
    for prec, tol in (("f64", 1e-13), ("f32", 3e-6)):
        p, gr = make(G, dim, n, dx, 1e-3, nkl, 20.0, prec=prec)
        s = p.autotune(imag=True, nsteps=2)
        assert s == p.shapes()
        table = json.load(open(tmp_path / "shapes.json"))
        assert any(k.endswith(f"{prec}|imag") for k in table)
        p.set_state(phi0)
        p.step_imag(40)
        assert rel_l2(p.get_state(device=False).astype(np.complex128), O.run(gr, phi0, True, 40)) <= tol
        q, _ = make(G, dim, n, dx, 1e-3, nkl, 20.0, prec=prec)
        assert q.autotune(imag=True) == s          # from the cache file, no timing
        with pytest.raises(G.GPError):
            G.gp_set_shapes(q.h, 1, 3, 8, 1)      # 3 is not a segment length
        p.close()
        q.close()


EDGE_GRIDS = [
    (1, [3], [0.4]), (1, [4], [0.4]), (1, [5], [0.4]),      # one, two, three interior points
    (2, [3, 3], [0.4, 0.4]), (2, [3, 40], [0.4, 0.2]), (2, [40, 3], [0.2, 0.4]),
    (3, [3, 4, 5], [0.4, 0.4, 0.4]), (3, [5, 3, 17], [0.4, 0.4, 0.3]),
    (1, [514], [0.02]),                                     # longest segmented line (16 x 32)
    (2, [514, 6], [0.02, 0.3]), (2, [6, 514], [0.3, 0.02]),
    (1, [515], [0.02]),                                     # one point more: thread-per-line kernels
]


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("dim,n,dx", EDGE_GRIDS, ids=lambda v: str(v) if not isinstance(v, list) else "x".join(map(str, v)))
def test_degenerate_and_boundary_sizes(G, dim, n, dx, prec):
    """Grids with one interior point per axis up to the longest lines each
    kernel family takes, imaginary and real time, against the oracle (the
    double-float form refuses lines over 514 points)."""
    nkl = [1.0, 1.3, 1.6][:dim]
    if prec == "df64" and max(n) > 514:
        with pytest.raises(G.GPError):
            G.Propagator(dim, n, dx, 1e-3, nkl, 5.0, precision=prec)
        return
    phi0 = I.gaussian_state(dim, n, dx, nkl, seed=77, noise=1e-2)
    tol = 2e-5 if prec == "f32" else 1e-12
    for imag in (True, False):
        p, gr = make(G, dim, n, dx, 1e-3, nkl, 5.0, prec=prec)
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(20)
        got = p.get_state(device=False).astype(np.complex128)
        ref = O.run(gr, phi0, imag, 20)
        if np.linalg.norm(ref) == 0:
            assert np.linalg.norm(got) == 0
        else:
            assert rel_l2(got, ref) <= tol, (imag, rel_l2(got, ref))
        p.close()


@pytest.mark.parametrize("imag", [True, False])
def test_fused_xy_sweeps(G, imag):
    """GP_SHAPE_FUSE_XY (x and y sweeps in one kernel per xy plane): bit for
    bit the tile and column sweeps with the same 16-point segments at 128^3,
    and the oracle on a ragged grid, with the Lie and the Strang splitting."""
    n, dx, nkl = [128] * 3, [0.1] * 3, [1.0, 1.4, 1.8]
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1710, noise=1e-3)
    dt = 1e-3 if imag else 2e-4
    states = []
    for flags in (G.GP_SHAPE_KEEP_YZ, G.GP_SHAPE_KEEP_YZ | G.GP_SHAPE_FUSE_XY):
        p = G.Propagator(3, n, dx, dt, nkl, 50.0, precision="f32")
        G.gp_set_shapes(p.h, 1, 16, 16, flags)
        assert p.shapes()["flags"] == flags
        p.set_state(phi0)
        l0 = G.gp_kernel_launches()
        (p.step_imag if imag else p.step_real)(40)
        launches = G.gp_kernel_launches() - l0
        assert launches == 40 * (2 if flags & G.GP_SHAPE_FUSE_XY else 3) + (1 if imag else 0)
        states.append(p.get_state(device=False))
        p.close()
    assert np.array_equal(states[0], states[1])
    n, dx, nkl = [100, 90, 50], [0.12, 0.13, 0.2], [1.0, 1.3, 1.7]
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1711, noise=1e-3)
    for split in (0, 1):
        p = G.Propagator(3, n, dx, dt, nkl, 50.0, precision="f32")
        G.gp_set_shapes(p.h, 1, 16, 16, G.GP_SHAPE_KEEP_YZ | G.GP_SHAPE_FUSE_XY)
        if split:
            p.set_splitting("strang")
        p.set_state(phi0)
        (p.step_imag if imag else p.step_real)(60)
        ref = O.run(O.Grid(3, n, dx, dt, nkl, 50.0, split=split), phi0, imag, 60)
        assert rel_l2(p.get_state(device=False).astype(np.complex128), ref) <= 3e-6, split
        p.close()


def test_fused_xy_rejections(G):
    for prec, dim, n in (("f64", 3, [64, 64, 64]), ("f32", 2, [64, 64]), ("f32", 3, [160, 64, 32])):
        p = G.Propagator(dim, n, [0.2] * dim, 1e-3, [1.0] * dim, 1.0, precision=prec)
        with pytest.raises(G.GPError):
            G.gp_set_shapes(p.h, 1, 16, 16, G.GP_SHAPE_FUSE_XY)
        p.close()


def test_fused_xy_sweeps_with_a_user_potential(G):
    """The fused x + y kernel's per-point potential path: bit for bit the
    separate sweeps, imaginary then real time, and the oracle."""
    n, dx, nkl = [96, 80, 40], [0.15, 0.15, 0.2], [1.0, 1.3, 1.6]
    gr = O.Grid(3, n, dx, 1e-3, nkl, 30.0)
    dV, _ = I.gaussian_bumps(3, n, dx, seed=1714)
    V = O.potential(gr) + dV
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1715, noise=1e-3)
    states = []
    for flags in (G.GP_SHAPE_KEEP_YZ, G.GP_SHAPE_KEEP_YZ | G.GP_SHAPE_FUSE_XY):
        p = G.Propagator(3, n, dx, 1e-3, nkl, 30.0, precision="f32")
        G.gp_set_shapes(p.h, 1, 16, 16, flags)
        p.set_potential(V)
        p.set_state(phi0)
        p.step_imag(30)
        p.set_dt(2e-4)
        p.step_real(30)
        states.append(p.get_state(device=False))
        p.close()
    assert np.array_equal(states[0], states[1])
    ref = O.run(gr.with_(V=V), phi0, True, 30)
    ref = O.run(gr.with_(V=V, dt=2e-4), ref, False, 30)
    assert rel_l2(states[1].astype(np.complex128), ref) <= 3e-6


def test_headline_job_as_tuned(G):
    """The 128^3 imaginary-time job (dx = 0.1, dt = 1e-3, trap 1, 1.4, 1.8, g = 50,
    5000 steps) exactly as the benchmark runs it: FP32 form, kernel shapes from
    the autotuner, programmatic dependent launch on, calls of 100 steps -- an
    eager first step, 16-step graph replays, an eager tail and the final
    scaling -- then the observables.  After the first call the state is
    compared with the oracle element by element (relative L2); at the job's end
    every observable is compared, mu within 1e-6 absolute (the FP32 form's
    gate, where it applies: at the end of the configuration's run)."""
    n, dx, nkl, dt, g = [128] * 3, [0.1] * 3, [1.0, 1.4, 1.8], 1e-3, 50.0
    p, gr = make(G, 3, n, dx, dt, nkl, g, prec="f32")
    p.autotune(imag=True, cache=False)
    phi0 = I.gaussian_state(3, n, dx, nkl, seed=1710, noise=1e-3)
    p.set_state(phi0)
    p.step_imag(100)
    ref = O.run(gr, phi0, True, 100)
    err100 = rel_l2(p.get_state(device=False).astype(np.complex128), ref)
    assert err100 <= 2e-6
    for _ in range(49):
        p.step_imag(100)
    got = p.get_state(device=False).astype(np.complex128)
    ob = p.observables()
    ref = O.run(gr, ref, True, 4900)
    obr = O.observables(gr, ref)
    err = rel_l2(got, ref)
    print("headline job as tuned: shapes", p.shapes(), "rel-L2 after 100 steps", err100, "at the end", err,
          {k: abs(ob[k] - obr[k]) for k in O.OBS_KEYS})
    assert err <= 5e-6
    assert abs(ob["mu"] - obr["mu"]) <= mu_tol_f32(obr["mu"], transient=False)
    assert abs(ob["energy"] - obr["energy"]) <= 1e-6
    assert abs(ob["norm"] - obr["norm"]) <= 1e-6
    for k in ("rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(ob[k] - obr[k]) <= 1e-5 * obr[k]
    p.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_observables_on_polynomial_state(G, dim, prec):
    """The observables of a product of quartics with nonzero values at every
    index (the state that pins the derivative's boundary branches in the
    oracle tests) against the oracle: FP64 to 1e-12, FP32 to its rounding."""
    n = [9, 12, 7][:dim]
    dx = [0.3, 0.25, 0.4][:dim]
    nkl = [1.0, 1.4, 1.8][:dim]
    coefs = [[0.7 + 0.2j, -0.4 + 0.9j, 0.35 - 0.1j, 0.08 + 0.05j, -0.03 + 0.02j],
             [1.1 - 0.3j, 0.5 + 0.2j, -0.6 + 0.4j, 0.1 - 0.07j, 0.04],
             [0.9, -0.2 - 0.5j, 0.3 + 0.3j, -0.05j, 0.02 - 0.01j]]
    phi = np.ones((), dtype=np.complex128)
    for d in reversed(range(dim)):
        phi = np.multiply.outer(phi, np.polynomial.polynomial.polyval(O.coords(n[d], dx[d]), coefs[d]))
    p, gr = make(G, dim, n, dx, 1e-3, nkl, 3.0, prec=prec)
    p.set_state(phi)
    ob, obr = p.observables(), O.observables(gr, phi)
    tol = 1e-12 if prec == "f64" else 1e-6
    for k in O.OBS_KEYS:
        assert ob[k] == pytest.approx(obr[k], rel=tol, abs=1e-14), k
    p.close()
