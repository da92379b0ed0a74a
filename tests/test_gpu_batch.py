"""Batched form: independent 2d real-time runs of uneven size stepped together.

A run in a batch must give exactly what the same run gives in its own handle
(same kernels, same coefficient tables), and the FP64 batch must match the
oracle run by run.  The full-size case is the 64-run workload (sizes drawn
from {128, 192, 256, 384, 512}^2, dx = 0.1, dt = 5e-4, g ~ U[0, 50], nu = 1,
kappa ~ U[1, 2]) in the launch configuration the benchmark times, checked on
sampled runs against the oracle.
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


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


RUNS = [  # (nx, ny), (dx, dy), (nu, kappa), g -- one per segment class and ragged sizes
    ((17, 20), (0.4, 0.35), (1.0, 1.3), 5.0),
    ((130, 96), (0.12, 0.15), (1.0, 1.7), 12.0),
    ((131, 160), (0.1, 0.1), (1.0, 1.1), 30.0),
    ((64, 259), (0.2, 0.07), (1.4, 1.0), 0.0),
    ((300, 41), (0.06, 0.3), (1.0, 2.0), 44.0),
    ((400, 24), (0.05, 0.3), (1.0, 1.5), 8.0),     # FP64: x lines run one warp per line
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_equals_each_run_alone(G, prec):
    sizes = [r[0] for r in RUNS]
    b = G.Batch(sizes, [r[1] for r in RUNS], 5e-4, [r[2] for r in RUNS], [r[3] for r in RUNS], precision=prec)
    states = []
    for i, (n, dx, nk, g) in enumerate(RUNS):
        phi = I.gaussian_state(2, list(n), list(dx), list(nk), seed=40 + i, noise=1e-2)
        states.append(phi)
        b.set_state(i, phi)
    b.step_real(37)          # a graph block plus eager steps
    for i, (n, dx, nk, g) in enumerate(RUNS):
        p = G.Propagator(2, list(n), list(dx), 5e-4, list(nk), g, precision=prec)
        p.set_state(states[i])
        p.step_real(37)
        alone = p.get_state(device=False)
        p.close()
        assert np.array_equal(b.get_state(i), alone), i
    b.close()


def test_batch_f64_matches_oracle(G):
    sizes = [r[0] for r in RUNS]
    b = G.Batch(sizes, [r[1] for r in RUNS], 5e-4, [r[2] for r in RUNS], [r[3] for r in RUNS], precision="f64")
    refs = []
    for i, (n, dx, nk, g) in enumerate(RUNS):
        phi = I.gaussian_state(2, list(n), list(dx), list(nk), seed=50 + i, noise=1e-2)
        b.set_state(i, phi)
        refs.append(O.run(O.Grid(2, list(n), list(dx), 5e-4, list(nk), g), phi, False, 60))
    b.step_real(60)
    obs = b.observables()
    for i, (n, dx, nk, g) in enumerate(RUNS):
        assert rel_l2(b.get_state(i), refs[i]) <= 1e-12, i
        ob = O.observables(O.Grid(2, list(n), list(dx), 5e-4, list(nk), g), refs[i])
        for k in ("norm", "energy", "mu", "rms_x", "rms_y", "rms_r"):
            assert obs[i][k] == pytest.approx(ob[k], rel=1e-11, abs=1e-13), (i, k)
    b.close()


def test_batch_64_runs_full_size_sampled(G):
    """The 64-run workload as the benchmark runs it (FP32, graph-captured step
    blocks); runs 0..63 all advance, two sampled runs are checked against the
    FP64 oracle after 40 steps and every run's norm is conserved."""
    P = I.batch_runs(seed=1712, nruns=64)
    sizes = [(int(n), int(n)) for n in P["n"]]
    dx = [(0.1, 0.1)] * 64
    nk = [(1.0, float(k)) for k in P["kappa"]]
    g = [float(v) for v in P["g"]]
    b = G.Batch(sizes, dx, 5e-4, nk, g, precision="f32")
    phis = [I.gaussian_state(2, list(s), [0.1, 0.1], list(k)) for s, k in zip(sizes, nk)]
    for i, phi in enumerate(phis):
        b.set_state(i, phi)
    ob0 = b.observables()
    b.step_real(40)
    ob1 = b.observables()
    for i in range(64):
        assert abs(ob1[i]["norm"] / ob0[i]["norm"] - 1) < 2e-5, i
    smallest = int(np.argmin(P["n"]))
    largest = int(np.argmax(P["n"]))
    for i in (smallest, largest):
        gr = O.Grid(2, list(sizes[i]), [0.1, 0.1], 5e-4, list(nk[i]), g[i])
        ref = O.run(gr, phis[i], False, 40)
        assert rel_l2(b.get_state(i).astype(np.complex128), ref) <= 2e-5, i
        assert ob1[i]["mu"] == pytest.approx(O.observables(gr, ref)["mu"], rel=1e-5)
    b.close()
