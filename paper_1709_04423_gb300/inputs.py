"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no step of the propagator's arithmetic: it only draws the
random numbers and builds the initial states and potentials that both sides
take as inputs, so that the CUDA path and the oracle start from identical bits.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += golden gamma, then two
xor-shift-multiply mixing rounds; a double in [0, 1) takes the top 53 bits.

The paper's own sample inputs are not available, so these synthetic states and
potentials stand in for them: a trapped Gaussian condensate plus a small
uniform noise, harmonic traps with the stated frequencies, and a smooth random
potential made of Gaussian bumps.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """``count`` successive SplitMix64 outputs (uint64) from ``seed``."""
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from SplitMix64(seed)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def axis_coords(n: int, dx: float) -> np.ndarray:
    """Cell-start grid positions -n*dx/2 + i*dx used to place initial states."""
    return -0.5 * n * dx + np.arange(n, dtype=np.float64) * dx


def gaussian_state(dim, n, dx, nkl, seed=None, noise=1e-3, shift=(0.0, 0.0, 0.0)):
    """Product of trap ground-state Gaussians (nu_d/pi)^(1/4) exp(-nu_d x^2/2),
    plus ``noise`` * U[0,1) real noise from SplitMix64(seed) in storage order.

    Returned as complex128 of shape (nz, ny, nx) truncated to ``dim``; not
    renormalised.
    """
    axes = []
    for d in range(dim):
        x = axis_coords(n[d], dx[d]) - shift[d]
        nu = nkl[d]
        axes.append((nu / np.pi) ** 0.25 * np.exp(-0.5 * nu * x * x))
    psi = axes[0]
    for d in range(1, dim):
        psi = np.multiply.outer(axes[d], psi)
    psi = np.asarray(psi, dtype=np.float64)
    if seed is not None and noise != 0.0:
        psi = psi + noise * uniform(seed, psi.size).reshape(psi.shape)
    return psi.astype(np.complex128)


def gaussian_bumps(dim, n, dx, seed, count=8, amp=0.5, center=3.0, width=(0.5, 1.5)):
    """Smooth random potential: sum of ``count`` Gaussians
    A_k exp(-|r - c_k|^2 / (2 s_k^2)), A_k ~ U[-amp, amp], c_k ~ U[-center,
    center]^dim, s_k ~ U[width].  Returns (dV array, params dict)."""
    u = uniform(seed, count * (2 + dim))
    A = (2.0 * u[:count] - 1.0) * amp
    s = width[0] + (width[1] - width[0]) * u[count:2 * count]
    c = (2.0 * u[2 * count:].reshape(count, dim) - 1.0) * center
    coords = [axis_coords(n[d], dx[d]) for d in range(dim)]
    mesh = np.meshgrid(*reversed(coords), indexing="ij")  # (z, y, x) order
    mesh = list(reversed(mesh))                            # mesh[d] is axis d
    dV = np.zeros(tuple(reversed(n[:dim])), dtype=np.float64)
    bumps = []
    for k in range(count):
        r2 = sum((mesh[d] - c[k, d]) ** 2 for d in range(dim))
        G = np.exp(-r2 / (2.0 * s[k] ** 2))
        bumps.append(G)
        dV += A[k] * G
    return dV, {"A": A, "s": s, "c": c, "bumps": bumps}


def batch_runs(seed, nruns=64, sizes=(128, 192, 256, 384, 512), g_max=50.0, kappa=(1.0, 2.0)):
    """Parameters of a batch of independent 2d runs: square grids drawn from
    ``sizes``, g ~ U[0, g_max], kappa ~ U[kappa]."""
    u = uniform(seed, 3 * nruns)
    idx = np.minimum((u[:nruns] * len(sizes)).astype(np.int64), len(sizes) - 1)
    n = np.array([sizes[i] for i in idx], dtype=np.int64)
    g = u[nruns:2 * nruns] * g_max
    ka = kappa[0] + (kappa[1] - kappa[0]) * u[2 * nruns:]
    return {"n": n, "g": g, "kappa": ka}
