"""gp_observables_noalloc -- the allocation-free observables entry point.

Callers that cannot allocate device memory when they need the observables
(an application that owns the whole device-memory budget, a loop that must
not synchronise the device) use this entry point; it must give what
gp_observables gives for the same state.  This file is
collected last so that a stop-at-first-failure run has already run every
other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("norm", "energy", "mu", "rms_x", "rms_y", "rms_z", "rms_r")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_handle_observables_on_two_calls(prec):
    import torch

    from paper_1709_04423_gb300 import gpe, inputs
    gpe.load()
    code = gpe.GP_F64 if prec == "f64" else gpe.GP_F32
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    cases = [
        (3, [40, 33, 24], [0.25, 0.3, 0.35], [1.0, 1.4, 1.8], 20.0, 31, False),
        (2, [64, 48], [0.2, 0.25], [1.0, 1.3], 7.5, 32, True),
        (1, [257], [0.05], [1.0], 10.0, 33, False),   # both absent axes on one-point tables
    ]
    for dim, n, dx, nkl, g, seed, with_v in cases:   # two calls in a row
        p = gpe.Propagator(dim, n, dx, 1e-3, nkl, g, precision=prec)
        p.set_state(inputs.gaussian_state(dim, n, dx, nkl, seed=seed, noise=0.05))
        V = None
        if with_v:
            dV, _ = inputs.gaussian_bumps(dim, n, dx, seed=seed)
            x = [inputs.axis_coords(n[d], dx[d]) for d in range(dim)]
            assert dim == 2
            harm = 0.5 * (nkl[1] ** 2 * x[1][:, None] ** 2 + nkl[0] ** 2 * x[0][None, :] ** 2)
            V = torch.tensor(harm + dV, dtype=torch.float64, device="cuda")
            p.set_potential(V)
        p.step_imag(3)
        ref = p.observables()                       # the existing entry point
        psi = p.get_state(device=True)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        gpe.gp_observables_noalloc(dim, n, dx, nkl, g, code, psi.data_ptr(),
                                   V.data_ptr() if V is not None else None, out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i, k in enumerate(KEYS):
            assert got[i] == pytest.approx(ref[k], rel=1e-12, abs=1e-14), (dim, k, got[i], ref[k])
        p.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1709_04423_gb300 import gpe
    with pytest.raises(gpe.GPError) as e:
        gpe.gp_observables_noalloc(1, [5000], [0.1], [1.0], 1.0, gpe.GP_F64, 1, None, 1, None)
    assert e.value.code == gpe.GP_ERR_INVALID
    assert "4096" in str(e.value)
    with pytest.raises(gpe.GPError) as e:
        gpe.gp_observables_noalloc(1, [64], [0.1], [1.0], 1.0, gpe.GP_DF64, 1, None, 1, None)
    assert e.value.code == gpe.GP_ERR_INVALID
    assert "GP_DF64" in str(e.value)
