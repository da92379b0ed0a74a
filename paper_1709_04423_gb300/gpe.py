"""Python binding of the GB300 split-step Crank-Nicolson GP library.

Argument marshalling only: every step of the propagator runs in the CUDA
kernels of ``libgpe.so`` behind the C ABI of ``include/gpe.h``.  The
functions ``gp_*`` mirror the C entry points one to one (same names, same
argument order); :class:`Propagator` is a small convenience wrapper that owns a
handle and exchanges states as torch tensors (device memory and streams come
from PyTorch).  There is no CPU fallback: if the library is missing or cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgpe.so")

GP_OK = 0
GP_ERR_INVALID = -1
GP_ERR_CUDA = -2
GP_ERR_NONFINITE = -3
GP_ERR_TIMEOUT = -4
GP_ERR_STATE = -5
GP_F64 = 0
GP_F32 = 1
GP_DF64 = 2
PRECISIONS = {"f64": GP_F64, "f32": GP_F32, "df64": GP_DF64}
GP_SHAPE_KEEP_YZ = 1
GP_SHAPE_PIPE_X = 2
GP_SHAPE_PIPE_YZ = 4
GP_SHAPE_TMA_YZ = 16
GP_SHAPE_TMA_X = 32
GP_SHAPE_FUSE_XY = 8

# every entry point declared in include/gpe.h
ABI_SYMBOLS = (
    "gp_init", "gp_set_state", "gp_get_state", "gp_set_potential", "gp_set_g", "gp_set_dt",
    "gp_step_imag", "gp_step_real", "gp_observables", "gp_npoints", "gp_precision_of",
    "gp_destroy", "gp_last_error", "gp_kernel_launches", "gp_time_sweeps", "gp_observables_noalloc",
    "gp_batch_init", "gp_batch_set_state", "gp_batch_get_state", "gp_batch_step_real", "gp_batch_observables",
    "gp_batch_offset", "gp_batch_destroy", "gp_adjoint_forward", "gp_adjoint_backward",
    "gp_autotune", "gp_set_shapes", "gp_get_shapes", "gp_reduced_density", "gp_step_series",
    "gp_init_spherical", "gp_set_splitting", "gp_set_real_state", "gp_init_circular", "gp_init_axial",
    "gp_test_stall_transfers", "gp_time_sweeps_graph", "gp_fp_fma_rates", "gp_check_status",
    "gp_batch_set_mode", "gp_batch_get_mode", "gp_batch_autotune", "gp_test_batch_stall",
)


class GPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class GpObs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("energy", ctypes.c_double), ("mu", ctypes.c_double),
                ("rms", ctypes.c_double * 3), ("rms_r", ctypes.c_double)]


_lib = None
_lib_check = None
_vp = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Loads libgpe.so (raises if it is absent: build it with build())."""
    global _lib
    if _lib is not None:
        return _lib
    _lib = _open(path)
    return _lib


def load_check():
    """The checking build, libgpe_check.so (index checks in the kernels, guard
    bands around every device buffer; see gp_check_status), as a separate
    ctypes library with the same entry points and argument types."""
    global _lib_check
    if _lib_check is None:
        _lib_check = _open(os.path.join(os.path.dirname(LIB_PATH), "libgpe_check.so"))
    return _lib_check


def _open(path):
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} is not built ({path}); run paper_1709_04423_gb300.build.build()")
    lib = ctypes.CDLL(path)
    I, D, L = ctypes.c_int, ctypes.c_double, ctypes.c_long
    lib.gp_init.argtypes = [ctypes.POINTER(_vp), I, ctypes.POINTER(I), ctypes.POINTER(D), D,
                            ctypes.POINTER(D), D, I, _vp]
    lib.gp_set_state.argtypes = [_vp, _vp, I]
    lib.gp_get_state.argtypes = [_vp, _vp, I]
    lib.gp_set_potential.argtypes = [_vp, _vp, I]
    lib.gp_set_g.argtypes = [_vp, D]
    lib.gp_set_dt.argtypes = [_vp, D]
    lib.gp_set_splitting.argtypes = [_vp, I]
    lib.gp_set_real_state.argtypes = [_vp, I]
    lib.gp_step_imag.argtypes = [_vp, L]
    lib.gp_step_real.argtypes = [_vp, L]
    lib.gp_observables.argtypes = [_vp, ctypes.POINTER(GpObs), _vp, I]
    lib.gp_time_sweeps.argtypes = [_vp, I, L, ctypes.POINTER(D)]
    lib.gp_time_sweeps_graph.argtypes = [_vp, I, I, ctypes.POINTER(D)]
    lib.gp_fp_fma_rates.argtypes = [ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.gp_test_stall_transfers.argtypes = [_vp, I]
    lib.gp_check_status.argtypes = [ctypes.POINTER(I)]
    lib.gp_observables_noalloc.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(D), D, I,
                                           _vp, _vp, _vp, _vp]
    lib.gp_autotune.argtypes = [_vp, I, I, ctypes.POINTER(D)]
    lib.gp_set_shapes.argtypes = [_vp, I, I, I, I]
    lib.gp_get_shapes.argtypes = [_vp, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.gp_reduced_density.argtypes = [_vp, I, _vp, I]
    lib.gp_init_spherical.argtypes = [ctypes.POINTER(_vp), I, D, D, D, D, I, _vp]
    lib.gp_init_circular.argtypes = [ctypes.POINTER(_vp), I, D, D, D, D, I, _vp]
    lib.gp_init_axial.argtypes = [ctypes.POINTER(_vp), I, I, D, D, D, D, D, D, I, _vp]
    lib.gp_step_series.argtypes = [_vp, I, L, I, _vp, I]
    lib.gp_adjoint_forward.argtypes = [_vp, L, I]
    lib.gp_adjoint_backward.argtypes = [_vp, _vp, I, _vp, I, ctypes.POINTER(D), _vp]
    lib.gp_batch_init.argtypes = [ctypes.POINTER(_vp), I, ctypes.POINTER(I), ctypes.POINTER(D), D,
                                  ctypes.POINTER(D), ctypes.POINTER(D), I, _vp]
    lib.gp_batch_set_state.argtypes = [_vp, I, _vp, I]
    lib.gp_batch_get_state.argtypes = [_vp, I, _vp, I]
    lib.gp_batch_step_real.argtypes = [_vp, L]
    lib.gp_batch_observables.argtypes = [_vp, ctypes.POINTER(GpObs)]
    lib.gp_batch_offset.argtypes = [_vp, I]
    lib.gp_batch_offset.restype = L
    lib.gp_batch_destroy.argtypes = [_vp]
    lib.gp_batch_set_mode.argtypes = [_vp, I]
    lib.gp_batch_get_mode.argtypes = [_vp]
    lib.gp_batch_autotune.argtypes = [_vp, L, ctypes.POINTER(D)]
    lib.gp_test_batch_stall.argtypes = [_vp, I]
    lib.gp_npoints.argtypes = [_vp]
    lib.gp_npoints.restype = L
    lib.gp_precision_of.argtypes = [_vp]
    lib.gp_destroy.argtypes = [_vp]
    lib.gp_last_error.restype = ctypes.c_char_p
    lib.gp_kernel_launches.restype = ctypes.c_ulonglong
    return lib


def _check(rc):
    if rc != GP_OK:
        raise GPError(rc, load().gp_last_error().decode())
    return rc


def _ptr(x):
    """Device or host address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# ----------------------------------------------------------------- raw ABI

def gp_init(dim, n, dx, dt, nkl, g, prec=GP_F64, stream=None):
    h = _vp()
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n)))[:3])
    dx3 = (ctypes.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx)))[:3])
    nkl3 = (ctypes.c_double * 3)(*(list(nkl) + [1.0] * (3 - len(nkl)))[:3])
    _check(load().gp_init(ctypes.byref(h), int(dim), n3, dx3, float(dt), nkl3, float(g), int(prec),
                          stream))
    return h


def gp_init_spherical(n, dr, dt, nu, g, prec=GP_F64, stream=None):
    h = _vp()
    _check(load().gp_init_spherical(ctypes.byref(h), int(n), float(dr), float(dt), float(nu), float(g), int(prec),
                                    stream))
    return h


def gp_init_circular(n, drho, dt, nu, g, prec=GP_F64, stream=None):
    h = _vp()
    _check(load().gp_init_circular(ctypes.byref(h), int(n), float(drho), float(dt), float(nu), float(g), int(prec),
                                   stream))
    return h


def gp_init_axial(n_rho, n_z, drho, dz, dt, nu, lam, g, prec=GP_F64, stream=None):
    h = _vp()
    _check(load().gp_init_axial(ctypes.byref(h), int(n_rho), int(n_z), float(drho), float(dz), float(dt), float(nu),
                                float(lam), float(g), int(prec), stream))
    return h


def gp_set_state(h, psi_ptr, on_device):
    return _check(load().gp_set_state(h, psi_ptr, int(on_device)))


def gp_get_state(h, psi_ptr, on_device):
    return _check(load().gp_get_state(h, psi_ptr, int(on_device)))


def gp_set_potential(h, V_ptr, on_device):
    return _check(load().gp_set_potential(h, V_ptr, int(on_device)))


def gp_set_g(h, g):
    return _check(load().gp_set_g(h, float(g)))


def gp_set_dt(h, dt):
    return _check(load().gp_set_dt(h, float(dt)))


def gp_set_splitting(h, strang):
    return _check(load().gp_set_splitting(h, int(strang)))


def gp_set_real_state(h, real):
    return _check(load().gp_set_real_state(h, int(real)))


def gp_step_imag(h, nsteps):
    return _check(load().gp_step_imag(h, int(nsteps)))


def gp_step_real(h, nsteps):
    return _check(load().gp_step_real(h, int(nsteps)))


def gp_observables(h, density_ptr=None, density_on_device=0):
    out = GpObs()
    _check(load().gp_observables(h, ctypes.byref(out), density_ptr, int(density_on_device)))
    return out


def gp_reduced_density(h, keep_mask, out_ptr, out_on_device):
    return _check(load().gp_reduced_density(h, int(keep_mask), out_ptr, int(out_on_device)))


def gp_step_series(h, imag, nsteps, every, out_ptr, out_on_device):
    return _check(load().gp_step_series(h, int(imag), int(nsteps), int(every), out_ptr, int(out_on_device)))


def gp_time_sweeps(h, imag, nsteps):
    """Mean per-launch duration (ms) of each axis' sweep kernel over nsteps steps."""
    ms = (ctypes.c_double * 3)()
    _check(load().gp_time_sweeps(h, int(bool(imag)), int(nsteps), ms))
    return list(ms)


def gp_time_sweeps_graph(h, imag, reps):
    """Mean per-launch duration (ms) of each axis' sweep kernel launched reps
    times back to back inside a CUDA graph (as in a step's graph)."""
    ms = (ctypes.c_double * 3)()
    _check(load().gp_time_sweeps_graph(h, int(bool(imag)), int(reps), ms))
    return list(ms)


def gp_fp_fma_rates():
    """Measured FP64 and FP32 FMA thread-instruction rates (per second) of the device."""
    d, f = ctypes.c_double(), ctypes.c_double()
    _check(load().gp_fp_fma_rates(ctypes.byref(d), ctypes.byref(f)))
    return d.value, f.value


def gp_observables_noalloc(dim, n, dx, nkl, g, prec, psi_ptr, V_ptr, out_ptr, stream=None):
    """Observables of a device state into a device buffer of 7 doubles, with
    no handle and no allocation (see include/gpe.h); asynchronous on stream."""
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n)))[:3])
    dx3 = (ctypes.c_double * 3)(*(list(dx) + [1.0] * (3 - len(dx)))[:3])
    nkl3 = (ctypes.c_double * 3)(*(list(nkl) + [1.0] * (3 - len(nkl)))[:3])
    return _check(load().gp_observables_noalloc(int(dim), n3, dx3, nkl3, float(g), int(prec), psi_ptr, V_ptr,
                                                out_ptr, stream))


def gp_autotune(h, imag, nsteps=8, timings=False):
    """Times the valid kernel shapes and keeps the fastest; with timings=True
    returns (best x-sweep ms, best y+z-sweep ms)."""
    if timings:
        ms = (ctypes.c_double * 2)()
        _check(load().gp_autotune(h, int(bool(imag)), int(nsteps), ms))
        return float(ms[0]), float(ms[1])
    _check(load().gp_autotune(h, int(bool(imag)), int(nsteps), None))
    return None


def gp_set_shapes(h, tile_x, seg_x, seg_c, flags=GP_SHAPE_KEEP_YZ):
    return _check(load().gp_set_shapes(h, int(tile_x), int(seg_x), int(seg_c), int(flags)))


def gp_get_shapes(h):
    t, x, c, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().gp_get_shapes(h, ctypes.byref(t), ctypes.byref(x), ctypes.byref(c), ctypes.byref(k)))
    return {"tile_x": t.value, "seg_x": x.value, "seg_c": c.value, "flags": k.value}


def gp_adjoint_forward(h, nsteps, ckpt_every):
    return _check(load().gp_adjoint_forward(h, int(nsteps), int(ckpt_every)))


def gp_adjoint_backward(h, lam_ptr, lam_on_device, dJdV_ptr=None, dJdV_on_device=1, lam0_ptr=None):
    """Returns dJ/dg; writes dJ/dV and lambda(0) where pointers are given."""
    dJdg = ctypes.c_double(0.0)
    _check(load().gp_adjoint_backward(h, lam_ptr, int(lam_on_device), dJdV_ptr, int(dJdV_on_device),
                                      ctypes.byref(dJdg), lam0_ptr))
    return float(dJdg.value)


def gp_batch_init(nruns, n, dx, dt, nkl, g, prec=GP_F32, stream=None):
    """n, dx, nkl: sequences of (x, y) pairs per run; g: one value per run."""
    b = _vp()
    na = (ctypes.c_int * (2 * nruns))(*[int(v) for pair in n for v in pair])
    dxa = (ctypes.c_double * (2 * nruns))(*[float(v) for pair in dx for v in pair])
    nka = (ctypes.c_double * (2 * nruns))(*[float(v) for pair in nkl for v in pair])
    ga = (ctypes.c_double * nruns)(*[float(v) for v in g])
    _check(load().gp_batch_init(ctypes.byref(b), int(nruns), na, dxa, float(dt), nka, ga, int(prec), stream))
    return b


def gp_batch_set_state(b, run, psi_ptr, on_device):
    return _check(load().gp_batch_set_state(b, int(run), psi_ptr, int(on_device)))


def gp_batch_get_state(b, run, psi_ptr, on_device):
    return _check(load().gp_batch_get_state(b, int(run), psi_ptr, int(on_device)))


def gp_batch_step_real(b, nsteps):
    return _check(load().gp_batch_step_real(b, int(nsteps)))


def gp_batch_observables(b, nruns):
    out = (GpObs * nruns)()
    _check(load().gp_batch_observables(b, out))
    return [obs_dict(o) for o in out]


def gp_batch_offset(b, run):
    return int(load().gp_batch_offset(b, int(run)))


def gp_batch_destroy(b):
    return _check(load().gp_batch_destroy(b))


def gp_batch_set_mode(b, persistent):
    return _check(load().gp_batch_set_mode(b, int(persistent)))


def gp_batch_get_mode(b):
    return int(load().gp_batch_get_mode(b))


def gp_batch_autotune(b, nsteps):
    ms = (ctypes.c_double * 2)()
    _check(load().gp_batch_autotune(b, int(nsteps), ms))
    return [float(ms[0]), float(ms[1])]


def gp_test_batch_stall(b, extra):
    """Test hook: the one-launch batch form's step waits ask for more items
    than will finish, so they run out (see include/gpe.h)."""
    return _check(load().gp_test_batch_stall(b, int(extra)))


def gp_npoints(h):
    return int(load().gp_npoints(h))


def gp_precision_of(h):
    return int(load().gp_precision_of(h))


def gp_destroy(h):
    return _check(load().gp_destroy(h))


def gp_last_error():
    return load().gp_last_error().decode()


def gp_kernel_launches():
    return int(load().gp_kernel_launches())


def gp_test_stall_transfers(h, extra_bytes):
    """Test hook: TMA tile loads announce extra bytes, so their bounded waits
    run out (see include/gpe.h)."""
    return _check(load().gp_test_stall_transfers(h, int(extra_bytes)))


# ----------------------------------------------------------------- wrapper

def obs_dict(o: GpObs):
    return {"norm": o.norm, "energy": o.energy, "mu": o.mu, "rms_x": o.rms[0], "rms_y": o.rms[1],
            "rms_z": o.rms[2], "rms_r": o.rms_r}


class Propagator:
    """One GP problem on the current CUDA device.

    ``precision``: ``"f64"`` (plain FP64), ``"f32"`` (FP32 state and sweeps,
    FP64 reductions and renormalisation) or ``"df64"`` (double-float state and
    sweeps on the FP32 pipes, exchanged as complex128).  States are complex
    tensors of shape (nz, ny, nx) truncated to ``dim`` (x fastest).
    """

    def __init__(self, dim, n, dx, dt, nkl=(1.0, 1.0, 1.0), g=0.0, precision="f64", stream=None,
                 spherical=False, axisym=False):
        """``spherical=True``: a spherically symmetric 3d trap (dim 1, n radial
        points, dx = (dr,), nkl = (nu,)); the state is u = sqrt(4 pi) r phi on
        r_i = i dr (see gp_init_spherical).  ``axisym=True``: a circularly
        symmetric 2d trap (dim 1: n = (n_rho,)) or an axially symmetric 3d
        trap (dim 2: n = (n_rho, n_z), dx = (drho, dz), nkl = (nu, lambda)) on
        rho_i = (i - 1/2) drho (see gp_init_circular / gp_init_axial)."""
        import torch
        self.torch = torch
        self.dim = int(dim)
        self.n = list(n)[: self.dim]
        self.shape = tuple(reversed(self.n))
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.real_state = False
        self.precision = precision
        self.ctype = torch.complex64 if precision == "f32" else torch.complex128
        self.npdtype = np.complex64 if precision == "f32" else np.complex128
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if spherical:
            if self.dim != 1:
                raise ValueError("the spherical trap is a 1d radial problem")
            self.h = gp_init_spherical(n[0], dx[0], dt, nkl[0], g, PRECISIONS[precision], stream.cuda_stream)
        elif axisym:
            if self.dim == 1:
                self.h = gp_init_circular(n[0], dx[0], dt, nkl[0], g, PRECISIONS[precision], stream.cuda_stream)
            elif self.dim == 2:
                self.h = gp_init_axial(n[0], n[1], dx[0], dx[1], dt, nkl[0], nkl[1], g, PRECISIONS[precision],
                                       stream.cuda_stream)
            else:
                raise ValueError("the circular (dim 1) and axial (dim 2) traps have one or two axes")
        else:
            self.h = gp_init(dim, n, dx, dt, nkl, g, PRECISIONS[precision], stream.cuda_stream)

    def close(self):
        if self.h is not None:
            gp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, psi):
        torch = self.torch
        if isinstance(psi, np.ndarray):
            a = np.ascontiguousarray(psi.reshape(self.shape), dtype=self.npdtype)
            gp_set_state(self.h, a.ctypes.data, 0)
            return
        t = psi.reshape(self.shape).to(dtype=self.ctype).contiguous()
        on_dev = t.is_cuda
        gp_set_state(self.h, t.data_ptr(), 1 if on_dev else 0)

    def get_state(self, device=True):
        torch = self.torch
        if device:
            out = torch.empty(self.shape, dtype=self.ctype, device="cuda")
            gp_get_state(self.h, out.data_ptr(), 1)
            return out
        out = np.empty(self.shape, dtype=self.npdtype)
        gp_get_state(self.h, out.ctypes.data, 0)
        return out

    def set_potential(self, V):
        if V is None:
            gp_set_potential(self.h, None, 0)
            return
        if isinstance(V, np.ndarray):
            a = np.ascontiguousarray(V.reshape(self.shape), dtype=np.float64)
            gp_set_potential(self.h, a.ctypes.data, 0)
            return
        t = V.reshape(self.shape).to(dtype=self.torch.float64).contiguous()
        gp_set_potential(self.h, t.data_ptr(), 1 if t.is_cuda else 0)

    def set_g(self, g):
        gp_set_g(self.h, g)

    def set_dt(self, dt):
        gp_set_dt(self.h, dt)

    def set_real_state(self, real=True):
        """Hold the state as real numbers (imaginary time only; see
        gp_set_real_state).  States in and out stay complex."""
        gp_set_real_state(self.h, 1 if real else 0)
        self.real_state = bool(real)

    def set_splitting(self, splitting):
        """``"lie"`` (N, then the sweeps; the default) or ``"strang"``
        (N(dt/2), the sweeps, N(dt/2)); see gp_set_splitting."""
        if splitting not in ("lie", "strang"):
            raise ValueError("splitting must be 'lie' or 'strang'")
        gp_set_splitting(self.h, 1 if splitting == "strang" else 0)

    def step_imag(self, nsteps):
        gp_step_imag(self.h, nsteps)

    def step_real(self, nsteps):
        gp_step_real(self.h, nsteps)

    def time_sweeps(self, imag, nsteps):
        return gp_time_sweeps(self.h, imag, nsteps)

    def time_sweeps_graph(self, imag, reps=32):
        return gp_time_sweeps_graph(self.h, imag, reps)

    def shapes(self):
        return gp_get_shapes(self.h)

    def autotune(self, imag, nsteps=8, cache=True):
        """Picks the fastest kernel shapes for this grid (see gp_autotune).
        With ``cache`` the result is kept in a JSON file keyed by GPU name,
        grid, precision and mode ($GPE_TUNE_CACHE, default
        ~/.cache/gpe_gb300/shapes.json), so later processes skip the timing."""
        import json
        import torch
        path = os.environ.get("GPE_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gpe_gb300",
                                                             "shapes.json"))
        key = "|".join([torch.cuda.get_device_name(), "x".join(map(str, self.n)), self.precision,
                        "imag" if imag else "real"] + (["real_state"] if self.real_state else []))
        table = {}
        if cache and os.path.exists(path):
            try:
                with open(path) as f:
                    table = json.load(f)
            except Exception:
                table = {}
        if cache and key in table:
            s = table[key]
            gp_set_shapes(self.h, s["tile_x"], s["seg_x"], s["seg_c"], s.get("flags", GP_SHAPE_KEEP_YZ))
            return s
        gp_autotune(self.h, imag, nsteps)
        s = gp_get_shapes(self.h)
        if cache:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                table[key] = s
                tmp = path + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(table, f, indent=1, sort_keys=True)
                os.replace(tmp, path)
            except OSError:
                pass
        return s

    def observables(self, density=False):
        den = None
        if density:
            den = self.torch.empty(self.shape, dtype=self.torch.float64, device="cuda")
        o = gp_observables(self.h, den.data_ptr() if den is not None else None, 1 if den is not None else 0)
        d = obs_dict(o)
        if density:
            d["density"] = den
        return d

    def step_series(self, imag, nsteps, every, device=True):
        """Runs nsteps steps and returns the observables recorded every
        ``every`` steps: an array (nsteps // every, 7) with columns norm,
        energy, mu, rms_x, rms_y, rms_z, rms_r (device tensor or numpy)."""
        nrec = int(nsteps) // int(every)
        if device:
            out = self.torch.empty((max(nrec, 1), 7), dtype=self.torch.float64, device="cuda")
            gp_step_series(self.h, imag, nsteps, every, out.data_ptr(), 1)
            return out[:nrec]
        out = np.empty((max(nrec, 1), 7), dtype=np.float64)
        gp_step_series(self.h, imag, nsteps, every, out.ctypes.data, 0)
        return out[:nrec]

    def reduced_density(self, keep, device=True):
        """Reduced (integrated) density on the axes in ``keep`` (tuple of axis
        numbers, 0 = x): |phi|^2 Simpson-summed over the other axes.  Shape:
        the kept axes' lengths, outermost first (x last)."""
        mask = sum(1 << int(d) for d in keep)
        shape = tuple(self.n[d] for d in reversed(range(self.dim)) if d in keep)
        if device:
            out = self.torch.empty(shape, dtype=self.torch.float64, device="cuda")
            gp_reduced_density(self.h, mask, out.data_ptr(), 1)
            return out
        out = np.empty(shape, dtype=np.float64)
        gp_reduced_density(self.h, mask, out.ctypes.data, 0)
        return out


class Batch:
    """Independent 2d real-time runs stepped together (see gp_batch_init).

    ``sizes``: list of (nx, ny); ``dx``, ``nkl``: lists of (x, y) pairs; ``g``:
    list of floats.  States are exchanged per run as (ny, nx) complex tensors.
    """

    def __init__(self, sizes, dx, dt, nkl, g, precision="f32", stream=None):
        import torch
        self.torch = torch
        self.sizes = [tuple(int(v) for v in s) for s in sizes]
        self.nruns = len(self.sizes)
        if precision not in ("f64", "f32", "df64"):
            raise ValueError("batched runs take precision 'f64', 'f32' or 'df64'")
        self.precision = precision
        wide = precision != "f32"   # double-float states are exchanged as complex128
        self.ctype = torch.complex128 if wide else torch.complex64
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.b = gp_batch_init(self.nruns, self.sizes, dx, dt, nkl, g,
                               {"f64": GP_F64, "f32": GP_F32, "df64": GP_DF64}[precision], stream.cuda_stream)

    def close(self):
        if self.b is not None:
            gp_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, run, psi):
        nx, ny = self.sizes[run]
        if isinstance(psi, np.ndarray):
            a = np.ascontiguousarray(psi.reshape(ny, nx),
                                     dtype=np.complex64 if self.precision == "f32" else np.complex128)
            gp_batch_set_state(self.b, run, a.ctypes.data, 0)
            return
        t = psi.reshape(ny, nx).to(dtype=self.ctype).contiguous()
        gp_batch_set_state(self.b, run, t.data_ptr(), 1 if t.is_cuda else 0)

    def set_all(self, flat):
        """All runs at once from a flat (back-to-back) device tensor or host array."""
        if isinstance(flat, np.ndarray):
            gp_batch_set_state(self.b, -1, flat.ctypes.data, 0)
        else:
            gp_batch_set_state(self.b, -1, flat.data_ptr(), 1 if flat.is_cuda else 0)

    def get_state(self, run, device=False):
        nx, ny = self.sizes[run]
        if device:
            out = self.torch.empty((ny, nx), dtype=self.ctype, device="cuda")
            gp_batch_get_state(self.b, run, out.data_ptr(), 1)
            return out
        out = np.empty((ny, nx), dtype=np.complex64 if self.precision == "f32" else np.complex128)
        gp_batch_get_state(self.b, run, out.ctypes.data, 0)
        return out

    def step_real(self, nsteps):
        gp_batch_step_real(self.b, nsteps)

    def observables(self):
        return gp_batch_observables(self.b, self.nruns)

    def set_mode(self, persistent):
        """0: per-class launches; 1: one persistent launch (FP32)."""
        gp_batch_set_mode(self.b, persistent)

    def mode(self):
        return gp_batch_get_mode(self.b)

    def autotune(self, nsteps=32):
        """Times both launch forms over nsteps steps and keeps the faster;
        returns their times in ms (-1 where not timed)."""
        return gp_batch_autotune(self.b, nsteps)


def real_time_evolution(prop, phi0, V, g, nsteps, ckpt_every):
    """Differentiable real-time propagation: phi(T) from phi(0), with gradients
    flowing to phi0 (complex tensor), V (real FP64 tensor: the full potential on
    the grid) and g (0-dim real tensor).  ``prop`` is a Propagator that this
    call owns until the backward pass has run; the forward pass keeps a
    checkpoint every ``ckpt_every`` steps and the backward pass recomputes
    between checkpoints (gp_adjoint_forward / gp_adjoint_backward)."""
    return _RealTimeEvolution.apply(phi0, V, g, prop, int(nsteps), int(ckpt_every))


def _make_function():
    import torch

    class RealTimeEvolution(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi0, V, g, prop, nsteps, ckpt_every):
            prop.set_potential(V.detach().to(torch.float64).contiguous())
            prop.set_g(float(g))
            prop.set_state(phi0.detach())
            gp_adjoint_forward(prop.h, nsteps, ckpt_every)
            ctx.prop = prop
            ctx.V_dtype, ctx.g_dtype = V.dtype, g.dtype
            return prop.get_state(device=True)

        @staticmethod
        def backward(ctx, grad_out):
            prop = ctx.prop
            lam = grad_out.to(prop.ctype).contiguous()
            dJdV = torch.empty(prop.shape, dtype=torch.float64, device="cuda")
            lam0 = torch.empty_like(lam)
            dJdg = gp_adjoint_backward(prop.h, lam.data_ptr(), 1, dJdV.data_ptr(), 1, lam0.data_ptr())
            return (lam0, dJdV.to(ctx.V_dtype), torch.tensor(dJdg, dtype=ctx.g_dtype, device="cuda"),
                    None, None, None)

    return RealTimeEvolution


class _Lazy:
    def __init__(self):
        self.fn = None

    def apply(self, *args):
        if self.fn is None:
            self.fn = _make_function()
        return self.fn.apply(*args)


_RealTimeEvolution = _Lazy()
