"""Reduced (integrated) densities of the CUDA path against the FP64 oracle.

Every choice of kept axes in 1d, 2d and 3d, every state precision, host and
device outputs.  FP64 and double-float: the same FP64 sums in another order
(relative 1e-13 of the largest value).  FP32: |phi|^2 is formed in FP32 from
the FP32 state, so each term carries a relative rounding of ~1e-7; compared
with the oracle on the same FP32 state (upcast), relative 1e-6.
"""
import itertools

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


def keeps(dim):
    return [k for r in range(1, dim + 1) for k in itertools.combinations(range(dim), r)]


CASES = [
    (1, [37], [0.2]),
    (2, [33, 20], [0.25, 0.3]),
    (3, [40, 33, 24], [0.25, 0.3, 0.35]),
    (3, [17, 12, 9], [0.4, 0.45, 0.5]),
]


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("dim,n,dx", CASES)
def test_reduced_density_matches_oracle(G, dim, n, dx, prec):
    nkl = [1.0, 1.4, 1.8][:dim]
    p = G.Propagator(dim, n, dx, 1e-3, nkl, 5.0, precision=prec)
    gr = O.Grid(dim, n, dx, 1e-3, nkl, 5.0)
    phi = I.gaussian_state(dim, n, dx, nkl, seed=41 + dim, noise=1e-2)
    p.set_state(phi)
    p.step_imag(3)                       # a state the kernels produced
    state = p.get_state(device=False).astype(np.complex128)
    tol = 1e-6 if prec == "f32" else 1e-13
    for keep in keeps(dim):
        ref = O.reduced_density(gr, state, keep)
        got_d = p.reduced_density(keep, device=True).cpu().numpy()
        got_h = p.reduced_density(keep, device=False)
        assert got_d.shape == ref.shape, keep
        assert np.array_equal(got_d, got_h), keep
        assert np.max(np.abs(got_d - ref)) <= tol * np.max(ref), (keep, np.max(np.abs(got_d - ref)) / np.max(ref))
    p.close()


def test_reduced_density_full_size_128cube(G):
    """128^3, the benchmark's grid: 1d and 2d reductions against the oracle."""
    n, dx, nkl = [128] * 3, [0.1] * 3, [1.0, 1.4, 1.8]
    p = G.Propagator(3, n, dx, 1e-3, nkl, 50.0, precision="f64")
    gr = O.Grid(3, n, dx, 1e-3, nkl, 50.0)
    phi = I.gaussian_state(3, n, dx, nkl, seed=1710, noise=1e-3)
    p.set_state(phi)
    for keep in [(0,), (1,), (2,), (0, 1), (1, 2)]:
        ref = O.reduced_density(gr, phi, keep)
        got = p.reduced_density(keep, device=True).cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(ref), keep
    p.close()


def test_reduced_density_rejects_bad_masks(G):
    p = G.Propagator(2, [16, 12], [0.3, 0.3], 1e-3, [1.0, 1.0], 1.0, precision="f64")
    out = np.zeros(16 * 12)
    for mask in (0, 4, 8, -1):
        with pytest.raises(G.GPError):
            G.gp_reduced_density(p.h, mask, out.ctypes.data, 0)
    p.close()
