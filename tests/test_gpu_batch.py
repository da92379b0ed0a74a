"""Batched form: independent 2d real-time runs of uneven size stepped together.

A run in a batch must give exactly what the same run gives in its own handle
(same kernels, same coefficient tables), and the FP64 batch must match the
oracle run by run.  The full-size case is the 64-run workload (sizes drawn
from {128, 192, 256, 384, 512}^2, dx = 0.1, dt = 5e-4, g ~ U[0, 50], nu = 1,
kappa ~ U[1, 2]) in the launch configuration the benchmark times, checked on
sampled runs against the oracle; so must the double-float batch (FP64-class
results on the FP32 pipes), which must also equal each run alone.  The one-launch form (FP32; per-run step
waits inside one persistent launch) must give the per-class launches' states
bit for bit, its bounded waits must come back as GP_ERR_TIMEOUT when made to
run out, and the autotuner must keep the faster form and leave the states as
they were.
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


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
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


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_batch_f64_matches_oracle(G, prec):
    """The FP64 and double-float batches against the oracle run by run (the
    double-float states rounded to complex128)."""
    sizes = [r[0] for r in RUNS]
    b = G.Batch(sizes, [r[1] for r in RUNS], 5e-4, [r[2] for r in RUNS], [r[3] for r in RUNS], precision=prec)
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


# ---------------------------------------------------------------- one persistent launch

def fp32_batch(G, runs, seed, mode):
    b = G.Batch([r[0] for r in runs], [r[1] for r in runs], 5e-4, [r[2] for r in runs], [r[3] for r in runs],
                precision="f32")
    b.set_mode(mode)
    assert b.mode() == mode
    for i, (n, dx, nk, g) in enumerate(runs):
        b.set_state(i, I.gaussian_state(2, list(n), list(dx), list(nk), seed=seed + i, noise=1e-2))
    return b


@pytest.mark.parametrize("nsteps", [1, 5, 37])
def test_persistent_batch_bitwise_equals_class_launches(G, nsteps):
    """Mode 1 (one launch per block of steps, per-run step waits) against mode
    0 (one launch per sweep and class): the same per-line arithmetic, so the
    same states bit for bit -- one step, a few, and graph blocks plus a tail."""
    out = []
    for mode in (0, 1):
        b = fp32_batch(G, RUNS, 60, mode)
        b.step_real(nsteps)
        out.append([b.get_state(i) for i in range(len(RUNS))])
        b.close()
    for i in range(len(RUNS)):
        assert np.array_equal(out[0][i], out[1][i]), i


def test_persistent_batch_64_runs_full_size(G):
    """The 64-run workload in mode 1 as the benchmark times it (graph blocks of
    16 steps): bit for bit the per-class launches after 40 steps; one sampled
    run against the FP64 oracle."""
    P = I.batch_runs(seed=1712, nruns=64)
    runs = [((int(n), int(n)), (0.1, 0.1), (1.0, float(k)), float(g)) for n, k, g in zip(P["n"], P["kappa"], P["g"])]
    out, obs = [], []
    for mode in (0, 1):
        b = fp32_batch(G, runs, 70, mode)
        b.step_real(40)
        obs.append(b.observables())
        out.append([b.get_state(i) for i in range(64)])
        b.close()
    for i in range(64):
        assert np.array_equal(out[0][i], out[1][i]), i
        assert obs[0][i]["mu"] == obs[1][i]["mu"], i
    i = int(np.argmax(P["n"]))
    (n, dx, nk, g) = runs[i]
    gr = O.Grid(2, list(n), list(dx), 5e-4, list(nk), g)
    ref = O.run(gr, I.gaussian_state(2, list(n), list(dx), list(nk), seed=70 + i, noise=1e-2), False, 40)
    assert rel_l2(out[1][i].astype(np.complex128), ref) <= 2e-5


def test_persistent_batch_refused_for_fp64(G):
    b = G.Batch([r[0] for r in RUNS[:2]], [r[1] for r in RUNS[:2]], 5e-4, [r[2] for r in RUNS[:2]],
                [r[3] for r in RUNS[:2]], precision="f64")
    with pytest.raises(G.GPError):
        b.set_mode(1)
    assert b.mode() == 0
    assert b.autotune(4) == [-1.0, -1.0] and b.mode() == 0
    b.close()


def test_batch_autotune_keeps_the_faster_form_and_the_states(G):
    b = fp32_batch(G, RUNS, 80, 0)
    before = [b.get_state(i) for i in range(len(RUNS))]
    ms = b.autotune(8)
    assert ms[0] > 0 and ms[1] > 0
    assert b.mode() == (1 if ms[1] < ms[0] else 0)
    for i in range(len(RUNS)):
        assert np.array_equal(b.get_state(i), before[i]), i
    b.step_real(3)
    assert all(np.isfinite(o["mu"]) for o in b.observables())
    b.close()


def test_persistent_batch_wait_that_runs_out_returns_gp_err_timeout(G, monkeypatch):
    """With the test hook every step wait of mode 1 asks for more finished
    items than the launch counts: the first y sweep's waits give up after the
    wait limit (50 ms here), the next gp_batch_observables returns
    GP_ERR_TIMEOUT, and the context stays usable -- the same batch, hook off
    and states set again, steps bit for bit as the per-class launches."""
    monkeypatch.setenv("GPE_WAIT_LIMIT_MS", "50")
    b = fp32_batch(G, RUNS, 90, 1)
    G.gp_test_batch_stall(b.b, 1000)
    b.step_real(3)
    with pytest.raises(G.GPError) as e:
        b.observables()
    assert e.value.code == G.GP_ERR_TIMEOUT
    G.gp_test_batch_stall(b.b, 0)
    for i, (n, dx, nk, g) in enumerate(RUNS):
        b.set_state(i, I.gaussian_state(2, list(n), list(dx), list(nk), seed=90 + i, noise=1e-2))
    b.step_real(3)
    b.observables()                            # the flag was cleared: no timeout now
    got = [b.get_state(i) for i in range(len(RUNS))]
    b.close()
    c = fp32_batch(G, RUNS, 90, 0)
    c.step_real(3)
    for i in range(len(RUNS)):
        assert np.array_equal(c.get_state(i), got[i]), i
    c.close()
