"""FP64 CPU oracle for the split-step Crank-Nicolson Gross-Pitaevskii propagator.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA library is checked against; only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  The product path never
calls it, and it shares no code with the CUDA library.

The arithmetic lives in ``gpo.c`` (plain C, FP64, one OpenMP pragma over
independent lines); this module only marshals numpy arrays through ctypes.
The readings of the paper that the C code follows (grid, splitting order,
boundary, Simpson rule, observables, adjoint) are listed at the top of
``gpo.c``.  Every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants and dense solves; the one unpinned aspect is
the last-ulp agreement of host ``sin/cos/exp`` with CUDA's, which only the
parity tolerances cover ("parity unpinned" for that rounding).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gpo.c`` into ``liboracle.so`` (plain gcc, no arch flags)."""
    src = os.path.join(_HERE, "gpo.c")
    hdr = os.path.join(_HERE, "gpo.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("nkl", ctypes.c_double * 3),
        ("g", ctypes.c_double),
        ("V", ctypes.POINTER(ctypes.c_double)),
        ("geom", ctypes.c_int),
        ("split", ctypes.c_int),
    ]


_P = ctypes.POINTER(Problem)
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.gpo_npoints.argtypes = [_P]
        lib.gpo_npoints.restype = ctypes.c_long
        lib.gpo_coords.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        lib.gpo_potential.argtypes = [_P, _D]
        lib.gpo_simpson_weights.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        lib.gpo_axisym_coords.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        lib.gpo_axisym_weights.argtypes = [ctypes.c_int, ctypes.c_double, _D]
        lib.gpo_phase.argtypes = [_P, ctypes.c_int, _D]
        lib.gpo_sweep.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _D]
        lib.gpo_step.argtypes = [_P, ctypes.c_int, _D]
        lib.gpo_run.argtypes = [_P, ctypes.c_int, ctypes.c_long, _D]
        lib.gpo_norm.argtypes = [_P, _D]
        lib.gpo_norm.restype = ctypes.c_double
        lib.gpo_observables.argtypes = [_P, _D, _D, _D]
        lib.gpo_reduced_density.argtypes = [_P, _D, ctypes.c_int, _D]
        lib.gpo_adjoint_real.argtypes = [_P, ctypes.c_long, _D, _D, _D, _D, _D]
        lib.gpo_adjoint_real.restype = ctypes.c_double
        lib.gpo_adjoint_phase.argtypes = [_P, _D, _D, _D, _D]
        lib.gpo_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D)


class Grid:
    """Problem description: dim, points per axis, spacing, dt, trap, g, potential.

    ``V`` is ``None`` for the harmonic trap ``(nu^2 x^2 + kappa^2 y^2 +
    lambda^2 z^2)/2`` or an FP64 array of the grid's shape (z, y, x order).
    """

    def __init__(self, dim, n, dx, dt, nkl=(1.0, 1.0, 1.0), g=0.0, V=None, geom=0, split=0):
        self.split = int(split)       # 0 Lie (N, L_x, L_y, L_z), 1 Strang (N/2, L, N/2)
        # 0 Cartesian, 1 spherically symmetric 3d trap (dim 1, u = sqrt(4 pi) r phi), 2 circularly (dim 1)
        # or axially (dim 2) symmetric trap with axis 0 = rho on rho_i = (i - 1/2) drho
        self.geom = int(geom)
        if self.geom == 1 and int(dim) != 1:
            raise ValueError("the spherical trap is a 1d radial problem")
        if self.geom == 2 and int(dim) not in (1, 2):
            raise ValueError("the circular (dim 1) and axial (dim 2) traps have one or two axes")
        self.dim = int(dim)
        n = list(n) + [1] * (3 - len(n))
        dx = list(dx) + [1.0] * (3 - len(dx))
        nkl = list(nkl) + [1.0] * (3 - len(nkl))
        self.n = [int(v) for v in n[:3]]
        self.dx = [float(v) for v in dx[:3]]
        self.dt = float(dt)
        self.nkl = [float(v) for v in nkl[:3]]
        self.g = float(g)
        self.V = None if V is None else np.ascontiguousarray(V, dtype=np.float64).reshape(self.shape)

    @property
    def shape(self):
        """Array shape, slowest axis first: (nz, ny, nx) truncated to dim."""
        return tuple(reversed(self.n[: self.dim]))

    @property
    def npoints(self):
        return int(np.prod(self.n[: self.dim]))

    def _struct(self):
        p = Problem()
        p.dim = self.dim
        for d in range(3):
            p.n[d] = self.n[d]
            p.dx[d] = self.dx[d]
            p.nkl[d] = self.nkl[d]
        p.dt = self.dt
        p.g = self.g
        p.V = _ptr(self.V) if self.V is not None else ctypes.cast(None, _D)
        p.geom = self.geom
        p.split = self.split
        return p

    def with_(self, **kw):
        args = dict(dim=self.dim, n=self.n, dx=self.dx, dt=self.dt, nkl=self.nkl, g=self.g, V=self.V, geom=self.geom,
                    split=self.split)
        args.update(kw)
        return Grid(**args)


def _state(grid, phi):
    a = np.ascontiguousarray(phi, dtype=np.complex128).reshape(grid.shape).copy()
    return a


def coords(n, dx):
    out = np.empty(int(n), dtype=np.float64)
    _load().gpo_coords(int(n), float(dx), _ptr(out))
    return out


def potential(grid):
    out = np.empty(grid.shape, dtype=np.float64)
    p = grid._struct()
    _load().gpo_potential(ctypes.byref(p), _ptr(out))
    return out


def simpson_weights(n, dx):
    out = np.empty(int(n), dtype=np.float64)
    _load().gpo_simpson_weights(int(n), float(dx), _ptr(out))
    return out


def axisym_coords(n, drho):
    """R15: rho_i = (i - 1/2) drho (i = 0 is the phantom point)."""
    out = np.empty(int(n), dtype=np.float64)
    _load().gpo_axisym_coords(int(n), float(drho), _ptr(out))
    return out


def axisym_weights(n, drho):
    """R15: midpoint weights 2 pi rho_i drho on i = 1..n-2, 0 at the ends."""
    out = np.empty(int(n), dtype=np.float64)
    _load().gpo_axisym_weights(int(n), float(drho), _ptr(out))
    return out


def phase(grid, phi, imag):
    a = _state(grid, phi)
    p = grid._struct()
    _load().gpo_phase(ctypes.byref(p), int(bool(imag)), _ptr(a))
    return a


def sweep(grid, phi, imag, axis, sign=1.0):
    a = _state(grid, phi)
    p = grid._struct()
    _load().gpo_sweep(ctypes.byref(p), int(bool(imag)), int(axis), float(sign), _ptr(a))
    return a


def step(grid, phi, imag):
    a = _state(grid, phi)
    p = grid._struct()
    _load().gpo_step(ctypes.byref(p), int(bool(imag)), _ptr(a))
    return a


def run(grid, phi, imag, nsteps):
    a = _state(grid, phi)
    p = grid._struct()
    _load().gpo_run(ctypes.byref(p), int(bool(imag)), int(nsteps), _ptr(a))
    return a


def norm(grid, phi):
    a = _state(grid, phi)
    p = grid._struct()
    return float(_load().gpo_norm(ctypes.byref(p), _ptr(a)))


OBS_KEYS = ("norm", "energy", "mu", "rms_x", "rms_y", "rms_z", "rms_r")


def observables(grid, phi, density=False):
    """Returns a dict of norm, energy, mu, rms_x/y/z, rms_r (and density)."""
    a = _state(grid, phi)
    p = grid._struct()
    out = np.zeros(7, dtype=np.float64)
    den = np.empty(grid.shape, dtype=np.float64) if density else None
    _load().gpo_observables(ctypes.byref(p), _ptr(a), _ptr(out),
                            _ptr(den) if den is not None else ctypes.cast(None, _D))
    res = dict(zip(OBS_KEYS, out.tolist()))
    if density:
        res["density"] = den
    return res


def reduced_density(grid, phi, keep):
    """Reduced density on the axes in ``keep`` (a tuple of axis numbers, 0 = x):
    Simpson sum of |phi|^2 over the other axes (reading R12).  Returns an array
    of shape (n_z, n_y, n_x) restricted to the kept axes."""
    a = _state(grid, phi)
    p = grid._struct()
    mask = sum(1 << d for d in keep)
    shape = tuple(grid.n[d] for d in reversed(range(grid.dim)) if d in keep)
    out = np.empty(shape, dtype=np.float64)
    _load().gpo_reduced_density(ctypes.byref(p), _ptr(a), int(mask), _ptr(out))
    return out


def adjoint_real(grid, phi0, target, nsteps):
    """Real-time run of ``nsteps`` from phi0 and the gradient of
    J = |sum conj(target) phi(T) dV|^2.  Returns (J, phiT, dJdV, dJdg)."""
    if grid.geom != 0:
        raise ValueError("the oracle adjoint is written for Cartesian grids")
    a0 = _state(grid, phi0)
    tg = _state(grid, target)
    phiT = np.empty(grid.shape, dtype=np.complex128)
    dJdV = np.empty(grid.shape, dtype=np.float64)
    dJdg = np.zeros(1, dtype=np.float64)
    p = grid._struct()
    J = _load().gpo_adjoint_real(ctypes.byref(p), int(nsteps), _ptr(a0), _ptr(tg), _ptr(phiT),
                                 _ptr(dJdV), _ptr(dJdg))
    return float(J), phiT, dJdV, float(dJdg[0])


def adjoint_phase(grid, phi_in, lam):
    """Adjoint of the real-time N sub-step at state phi_in applied to lam.
    Returns (lam_in, dJdV contribution, dJdg contribution)."""
    if grid.geom != 0:
        raise ValueError("the oracle adjoint is written for Cartesian grids")
    a = _state(grid, phi_in)
    lm = _state(grid, lam)
    dJdV = np.zeros(grid.shape, dtype=np.float64)
    dJdg = np.zeros(1, dtype=np.float64)
    p = grid._struct()
    _load().gpo_adjoint_phase(ctypes.byref(p), _ptr(a), _ptr(lm), _ptr(dJdV), _ptr(dJdg))
    return lm, dJdV, float(dJdg[0])


def num_threads():
    return int(_load().gpo_num_threads())
