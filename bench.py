"""Benchmark of the split-step Crank-Nicolson GP propagator on GB300.

Workload (default): the 3d imaginary-time anisotropic trap -- 128^3 grid,
dx = 0.1, dt = 1e-3, V = (nu^2 x^2 + kappa^2 y^2 + lambda^2 z^2)/2 with
nu, kappa, lambda = 1, 1.4, 1.8, g = 50, seeded-noise Gaussian initial state.
One bench step = ``--inner`` imaginary-time steps (renormalised every step)
followed by one evaluation of the observables (norm, energy, mu, rms), i.e.
one pass of the whole hot path.  The metric is grid-point-steps per second.

Two forms are timed: the plain FP64 path and the chosen FP32 form (FP32 state
and sweeps, FP64 norm/energy/mu reductions and renormalisation).  ``value`` is
the FP32 form's throughput; its mu error is measured against the FP64 path
over the full 5000-step job (the FP64 path itself is held to the CPU oracle
by the parity tests).

The state (16.8 MB FP32, 33.5 MB FP64) fits in the 129 MB L2, so L2 is
flushed (a 256 MB write) before every timed bench step; within a bench step
the state stays resident across time steps, as it does in a real run.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "name": "imag3d_128: 3d imaginary-time anisotropic trap, 128^3, dx=0.1, dt=1e-3, "
            "nu,kappa,lambda=1,1.4,1.8, g=50, 5000-step job",
    "dim": 3, "n": [128, 128, 128], "dx": [0.1, 0.1, 0.1], "dt": 1e-3,
    "nkl": [1.0, 1.4, 1.8], "g": 50.0, "seed": 1710, "job_steps": 5000,
}
METRIC = "3d split-step CN grid-point-steps/s: FP32/batched vs FP64 at fixed mu error"
UNIT = "grid-point-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", type=int, default=100, help="time steps per bench step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mu-check", action="store_true")
    ap.add_argument("--no-quench", action="store_true", help="skip the 256^3 real-time form")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint form")
    ap.add_argument("--quench-imag-steps", type=int, default=1500)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched form")
    ap.add_argument("--no-spherical", action="store_true", help="skip the spherical-trap form")
    ap.add_argument("--no-strang", action="store_true", help="skip the Strang-splitting form")
    ap.add_argument("--no-real", action="store_true", help="skip the real-state form")
    ap.add_argument("--forms", default="f64,f32,df64",
                    help="precision forms of the headline workload to time (the line needs f32; f64 for ratios)")
    ap.add_argument("--only", choices=["headline", "quench256", "batched", "adjoint", "spherical", "strang", "real"],
                    help="time one form only (for profiling); the other forms are reported as null")
    args = ap.parse_args()
    if "f32" not in args.forms.split(","):
        ap.error("--forms must include f32 (the headline form)")
    return args


def replica_throughput(points_per_rank, seconds, device="cpu"):
    """Whole-job throughput of independent replicas: the points all ranks
    processed divided by the slowest rank's time (one process per GPU; no
    collective on the data path, only this reduction of the timings)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return points_per_rank / seconds, seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    n = torch.tensor([float(points_per_rank)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(n.item()) / float(t.item()), float(t.item())


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


SWEEP_SOURCES = ("gpe_common.cuh", "gpe_df.cuh", "gpe_sweep2.cuh", "gpe_step.cuh")


def src_hash():
    """Hash of the sources that define and launch the sweep kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1709_04423_gb300", "csrc")
    for name in SWEEP_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel_key):
    """DRAM bytes per launch from a committed ncu capture, if the kernels have
    not changed since it was taken (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    r = rec.get(kernel_key)
    if not r or r.get("src_hash") != src_hash():
        return None
    return r.get("bytes_per_launch")


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not getattr(self, "rows", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = sorted(sm)[len(sm) // 4:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------- CPU oracle

def oracle_rate(target_s=12.0, max_steps=2000):
    """Oracle (FP64, C, OpenMP over lines) on the host cores: imaginary-time
    steps of the same workload, as many as fit in about target_s seconds."""
    import numpy as np

    import oracle as O
    from paper_1709_04423_gb300 import inputs
    w = WORKLOAD
    gr = O.Grid(w["dim"], w["n"], w["dx"], w["dt"], w["nkl"], w["g"])
    phi = inputs.gaussian_state(w["dim"], w["n"], w["dx"], w["nkl"], seed=w["seed"], noise=1e-3)
    t0 = time.perf_counter()
    phi = O.run(gr, phi, True, 1)
    t1 = time.perf_counter() - t0
    k = max(1, min(max_steps, int(target_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    phi = O.run(gr, phi, True, k)
    dt = time.perf_counter() - t0
    np_ = int(np.prod(w["n"]))
    return {"value": k * np_ / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{k} imaginary-time steps of the 128^3 workload (FP64, OpenMP over lines)",
            "seconds": dt}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    import numpy as np

    from paper_1709_04423_gb300 import inputs
    w = WORKLOAD
    gr = O.Grid(w["dim"], w["n"], w["dx"], w["dt"], w["nkl"], w["g"])
    phi = inputs.gaussian_state(w["dim"], w["n"], w["dx"], w["nkl"], seed=w["seed"], noise=1e-3)
    np_ = int(np.prod(w["n"]))
    per = 40  # imaginary-time steps of the oracle per bench step (~0.6 s on 16 Grace cores)
    for _ in range(args.warmup):
        phi = O.run(gr, phi, True, per)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        phi = O.run(gr, phi, True, per)
        O.observables(gr, phi)
    dt = time.perf_counter() - t0
    value = args.steps * per * np_ / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w["name"], "inner_steps_per_step": per, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{per} imaginary-time steps + observables of the 128^3 workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch

    from paper_1709_04423_gb300 import build as B
    B.build()
    from paper_1709_04423_gb300 import gpe, inputs

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = WORKLOAD
    np_ = int(np.prod(w["n"]))
    phi0 = inputs.gaussian_state(w["dim"], w["n"], w["dx"], w["nkl"], seed=w["seed"], noise=1e-3)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def make(prec):
        with torch.cuda.stream(stream):
            p = gpe.Propagator(w["dim"], w["n"], w["dx"], w["dt"], w["nkl"], w["g"], precision=prec,
                               stream=stream)
            p.autotune(imag=True, cache=False)   # kernel shapes for this grid (untimed)
            p.set_state(torch.tensor(phi0, device="cuda"))
        return p

    results = {}
    # ---- mu accuracy of the FP32 form over the full job (untimed)
    mu = {}
    forms_sel = [f for f in ("f64", "f32", "df64") if f in args.forms.split(",")]
    mu_conv = {}
    if not args.no_mu_check:
        for prec in forms_sel:
            p = make(prec)
            with torch.cuda.stream(stream):
                p.step_imag(w["job_steps"])
                mu[prec] = p.observables()
                # continued to 20000 steps: the state no longer changes (FP32: an
                # exact fixed point of the rounded step), mu is the converged one
                p.step_imag(20000 - w["job_steps"])
                mu_conv[prec] = p.observables()
            p.close()
    # ---- timed forms
    for prec in (forms_sel if not args.no_headline else ()):
        p = make(prec)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                p.step_imag(args.inner)
                p.observables()
            barrier()
            l0 = gpe.gp_kernel_launches()
            torch.cuda.nvtx.range_push(f"timed_{prec}")   # profilers can select the timed launches
            with ClockSampler(local) as clk:
                for s in range(args.steps):
                    flush.fill_(float(s))                 # evict the state from L2
                    ev[s][0].record(stream)
                    p.step_imag(args.inner)
                    p.observables()
                    ev[s][1].record(stream)
                barrier()
            torch.cuda.nvtx.range_pop()
            launches = gpe.gp_kernel_launches() - l0
            ms = [a.elapsed_time(b) for a, b in ev]
            # whole-job throughput over replicas: all ranks' points / slowest rank's time
            value, total_s = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
            # per-kernel durations, same state and sizes, right after the timed region
            kms = p.time_sweeps(True, 64)
            ob = p.observables()
            shp = p.shapes()
            # reduced densities of the final state (1d along x, 2d in x-y), device outputs
            red = {}
            for keep in ((0,), (0, 1)):
                for _ in range(3):
                    p.reduced_density(keep)
                r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                r0.record(stream)
                for _ in range(20):
                    p.reduced_density(keep)
                r1.record(stream)
                r1.synchronize()
                us = r0.elapsed_time(r1) / 20 * 1e3
                red["keep_" + "".join("xyz"[d] for d in keep)] = {
                    "us": us, "state_read_gbs": np_ * (8 if prec == "f32" else 16) / (us * 1e-6) / 1e9}
        p.close()
        results[prec] = {"total_s": total_s, "value": value, "ms": ms, "launches": launches,
                         "clocks": clk.summary(), "kernel_ms": kms, "obs": ob, "shapes": shp,
                         "reduced_density": red}
    # ---- batched form: 64 independent 2d real-time runs (sizes from
    # {128..512}^2, dx = 0.1, dt = 5e-4, g ~ U[0, 50], nu = 1, kappa ~ U[1, 2]),
    # each from its g = 0 trap ground state (an interaction quench)
    P = inputs.batch_runs(seed=1712, nruns=64)
    bsizes = [(int(v), int(v)) for v in P["n"]]
    bnk = [(1.0, float(k)) for k in P["kappa"]]
    bg = [float(v) for v in P["g"]]
    bpts = sum(a * b for a, b in bsizes)
    bphi = [torch.tensor(inputs.gaussian_state(2, list(sz), [0.1, 0.1], list(k)), device="cuda")
            for sz, k in zip(bsizes, bnk)]

    def make_batch(prec):
        with torch.cuda.stream(stream):
            bb = gpe.Batch(bsizes, [(0.1, 0.1)] * 64, 5e-4, bnk, bg, precision=prec, stream=stream)
            for i, ph in enumerate(bphi):
                bb.set_state(i, ph)
        return bb

    bres = {}
    bmu = {}
    for prec in (("f64", "f32") if not args.no_batched else ()):
        bb = make_batch(prec)
        with torch.cuda.stream(stream):
            if not args.no_mu_check:
                bb.step_real(400)
                bmu[prec] = [o["mu"] for o in bb.observables()]
                for i, ph in enumerate(bphi):
                    bb.set_state(i, ph)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for _ in range(args.warmup):
                bb.step_real(args.inner)
                bb.observables()
            barrier()
            l0 = gpe.gp_kernel_launches()
            torch.cuda.nvtx.range_push(f"timed_batched_{prec}")
            for s in range(args.steps):
                flush.fill_(float(s))
                ev[s][0].record(stream)
                bb.step_real(args.inner)
                bb.observables()
                ev[s][1].record(stream)
            barrier()
            torch.cuda.nvtx.range_pop()
            blaunch = gpe.gp_kernel_launches() - l0
            bt = max_over_ranks(sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3)
        bb.close()
        bres[prec] = {"value": world * args.steps * args.inner * bpts / bt, "ms_per_step": 1e3 * bt / args.steps,
                      "gpu_launches": blaunch}
    bmu_err = bmu_rel = bmu_worst = None
    if bmu:
        diffs = [(abs(a - b_), abs(a - b_) / abs(b_), b_, i) for i, (a, b_) in enumerate(zip(bmu["f32"], bmu["f64"]))]
        bmu_err = max(d[0] for d in diffs)
        bmu_rel = max(d[1] for d in diffs)
        w_ = max(diffs)
        # an FP32 state's own rounding (~6e-8 relative) bounds |dmu| at ~6e-8 mu
        bmu_worst = {"run": w_[3], "mu_f64": w_[2], "abs_diff": w_[0], "rel_diff": w_[1],
                     "mu_range_f64": [min(bmu["f64"]), max(bmu["f64"])]}

    # ---- 3d real-time quench at 256^3 (dx = 0.08, dt = 2e-4, isotropic trap):
    # imaginary-time ground state at g = 20, then real time at g = 40.  The
    # state (134 MB FP32, 268 MB FP64) is larger than L2, so these sweeps run
    # from HBM; timed per kernel like the headline form.
    qres = {}
    if not args.no_quench:
        qn, qdx = [256] * 3, [0.08] * 3
        qnp = 256 ** 3
        qphi = torch.tensor(inputs.gaussian_state(3, qn, qdx, [1.0] * 3, seed=1711, noise=1e-3), device="cuda")
        for prec in forms_sel:
            with torch.cuda.stream(stream):
                q = gpe.Propagator(3, qn, qdx, 1e-3, [1.0] * 3, 20.0, precision=prec, stream=stream)
                q.set_state(qphi)
                q.step_imag(args.quench_imag_steps)
                q.set_dt(2e-4)
                q.set_g(40.0)
                q.autotune(imag=False, cache=False)
                ob0 = q.observables()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for _ in range(args.warmup):
                    q.step_real(args.inner)
                barrier()
                torch.cuda.nvtx.range_push(f"timed_quench_{prec}")
                recs = []
                for s_ in range(args.steps):
                    ev[s_][0].record(stream)
                    # inner steps + the observables at their end, recorded on the device
                    recs.append(q.step_series(False, args.inner, args.inner, device=True))
                    ev[s_][1].record(stream)
                barrier()
                torch.cuda.nvtx.range_pop()
                rms_t = [[args.warmup * args.inner + (i + 1) * args.inner, float(r_[0, 6])]
                         for i, r_ in enumerate(recs)]
                qt = max_over_ranks(sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3)
                kms = q.time_sweeps(False, 16)
                ob1 = q.observables()
                q.close()
            esize = 8 if prec == "f32" else 16
            axis = max(range(3), key=lambda d: kms[d])
            ach = 2 * esize * qnp / (kms[axis] * 1e-3) / 1e9
            qres[prec] = {"value": world * args.steps * args.inner * qnp / qt, "ms_per_step": 1e3 * qt / args.steps,
                          "kernel_ms": kms, "dominant_sweep_axis": axis, "achieved_gbs": ach,
                          "frac_of_measured_hbm": ach / float(measured_peaks()[0]["hbm_gbs"]),
                          "energy_drift_rel": abs(ob1["energy"] / ob0["energy"] - 1),
                          "norm_drift_rel": abs(ob1["norm"] / ob0["norm"] - 1),
                          "rms_r_t": rms_t}

    # ---- spherically symmetric trap (radial problem for u = sqrt(4 pi) r phi):
    # n = 513 points on [0, 10.24], dt = 1e-4, nu = 1, g = 100, imaginary time
    # (a 1d line: launch-latency bound, one sweep kernel per step)
    sres = {}
    if not args.no_spherical:
        sn, sdr = 513, 0.02
        sr = np.arange(sn) * sdr
        su = torch.tensor((np.sqrt(4 * np.pi) * sr * np.exp(-0.6 * sr ** 2)).astype(np.complex128), device="cuda")
        smu = {}
        for prec in forms_sel:
            with torch.cuda.stream(stream):
                q = gpe.Propagator(1, [sn], [sdr], 1e-4, [1.0], 100.0, precision=prec, stream=stream, spherical=True)
                q.set_state(su)
                q.step_imag(20000)
                smu[prec] = q.observables()
                q.set_state(su)
                for _ in range(args.warmup):
                    q.step_imag(2000)
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    q.step_imag(2000)
                e1.record(stream)
                barrier()
                st = max_over_ranks(e0.elapsed_time(e1) / 1e3)
                q.close()
            sres[prec] = {"value": world * args.steps * 2000 * sn / st, "us_per_step": 1e6 * st / (args.steps * 2000),
                          "mu_after_20000_steps": smu[prec]["mu"], "rms_radius": smu[prec]["rms_x"]}
        if "f64" in smu:
            for prec in sres:
                sres[prec]["mu_diff_vs_f64"] = abs(smu[prec]["mu"] - smu["f64"]["mu"])

    # ---- circularly symmetric 2d trap (513 rho points, drho = 0.02, g = 100,
    # dt = 1e-4) and axially symmetric 3d trap (rho x z = 256 x 512, drho = dz
    # = 0.04, nu = 1, lambda = 2, g = 100, dt = 5e-4), imaginary time, every
    # form; mu after 20000 / 4000 steps against the FP64 form's
    ares_sym = {}
    if not args.no_spherical:
        cases = {"circular": (1, [513], [0.02], [1.0], 1e-4, 20000, 2000),
                 "axial": (2, [256, 512], [0.04, 0.04], [1.0, 2.0], 5e-4, 4000, 200)}
        for name, (cd, cn, cdx, cnkl, cdt, cmu_steps, cblock) in cases.items():
            rho = np.arange(cn[0]) * cdx[0] - 0.5 * cdx[0]
            if cd == 1:
                cphi = np.exp(-0.3 * rho ** 2)
            else:
                zz = inputs.axis_coords(cn[1], cdx[1])
                cphi = np.exp(-0.3 * (rho[None, :] ** 2 + 2.0 * zz[:, None] ** 2))
            cphi = torch.tensor(cphi.astype(np.complex128), device="cuda")
            cmu, cres = {}, {}
            for prec in forms_sel:
                with torch.cuda.stream(stream):
                    q = gpe.Propagator(cd, cn, cdx, cdt, cnkl, 100.0, precision=prec, stream=stream, axisym=True)
                    q.set_state(cphi)
                    q.step_imag(cmu_steps)
                    cmu[prec] = q.observables()
                    q.set_state(cphi)
                    for _ in range(args.warmup):
                        q.step_imag(cblock)
                    barrier()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(args.steps):
                        q.step_imag(cblock)
                    e1.record(stream)
                    barrier()
                    st = max_over_ranks(e0.elapsed_time(e1) / 1e3)
                    q.close()
                npts = int(np.prod(cn))
                cres[prec] = {"value": world * args.steps * cblock * npts / st,
                              "us_per_step": 1e6 * st / (args.steps * cblock),
                              "mu": cmu[prec]["mu"], "rms_rho": cmu[prec]["rms_x"]}
            if "f64" in cmu:
                for prec in cres:
                    cres[prec]["mu_diff_vs_f64"] = abs(cmu[prec]["mu"] - cmu["f64"]["mu"])
            ares_sym[name] = cres

    # ---- real state (imaginary-time maps keep the real input real): the
    # headline workload and loop with the state held as np real values;
    # mu after the full job against the complex FP64 form's
    rres = {}
    if not args.no_real:
        for prec in [f for f in forms_sel if f != "df64"]:
            p = make(prec)
            p.set_real_state(True)
            p.autotune(imag=True, cache=False)   # shapes for the real state (untimed)
            with torch.cuda.stream(stream):
                p.step_imag(w["job_steps"])
                rmu = p.observables()["mu"]
                p.set_state(torch.tensor(phi0, device="cuda"))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            with torch.cuda.stream(stream):
                for _ in range(args.warmup):
                    p.step_imag(args.inner)
                    p.observables()
                barrier()
                l0 = gpe.gp_kernel_launches()
                torch.cuda.nvtx.range_push(f"timed_real_{prec}")
                with ClockSampler(local) as rclk:
                    for s in range(args.steps):
                        flush.fill_(float(s))
                        ev[s][0].record(stream)
                        p.step_imag(args.inner)
                        p.observables()
                        ev[s][1].record(stream)
                    barrier()
                torch.cuda.nvtx.range_pop()
                launches = gpe.gp_kernel_launches() - l0
            ms = [a.elapsed_time(b) for a, b in ev]
            value, total_s = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
            kms = p.time_sweeps(True, 64)
            p.close()
            esz = 4 if prec == "f32" else 8
            rres[prec] = {"value": value, "ms_per_step": 1e3 * total_s / args.steps, "gpu_launches": launches,
                          "clocks": rclk.summary(), "kernel_ms": kms,
                          "sweep_state_gbs": [2 * esz * np_ / (t * 1e-3) / 1e9 for t in kms],
                          "mu_after_job": rmu,
                          "mu_err_vs_complex_f64": abs(rmu - mu["f64"]["mu"]) if "f64" in mu else None,
                          "speedup_vs_complex": (value / results[prec]["value"]) if prec in results else None}

    # ---- Strang splitting (N(dt/2), the sweeps, N(dt/2)) on the headline
    # workload, timed like the Lie step; and its accuracy: real-time runs of a
    # 64^3 grid (dx = 0.2, trap (1, 1.4, 1.8), g = 50) to t = 0.1 with dt =
    # 2e-3, 1e-3, 5e-4 against a Strang run with dt = 6.25e-5, FP64, for both
    # splittings (relative L2 error of phi(t), observed order)
    stres = {}
    if not args.no_strang:
        for prec in forms_sel:
            p = make(prec)
            stres[prec] = {}
            for mode in ("imag", "real"):
                for split in ("lie", "strang"):
                    p.set_splitting(split)
                    run = p.step_imag if mode == "imag" else p.step_real
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(args.steps)]
                    with torch.cuda.stream(stream):
                        p.set_state(torch.tensor(phi0, device="cuda"))
                        for _ in range(args.warmup):
                            run(args.inner)
                        barrier()
                        l0 = gpe.gp_kernel_launches()
                        torch.cuda.nvtx.range_push(f"timed_{split}_{mode}_{prec}")
                        for s in range(args.steps):
                            flush.fill_(float(s))
                            ev[s][0].record(stream)
                            run(args.inner)
                            ev[s][1].record(stream)
                        barrier()
                        torch.cuda.nvtx.range_pop()
                        launches = gpe.gp_kernel_launches() - l0
                    ms = [a.elapsed_time(b) for a, b in ev]
                    value, total_s = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
                    stres[prec][f"{split}_{mode}"] = {"value": value, "us_per_time_step": 1e6 * total_s / (
                        args.steps * args.inner), "gpu_launches": launches}
            for mode in ("imag", "real"):
                stres[prec][f"strang_time_over_lie_{mode}"] = (stres[prec][f"lie_{mode}"]["value"] /
                                                                stres[prec][f"strang_{mode}"]["value"])
            p.close()
        sn_, sdx, snkl, sT = [64] * 3, [0.2] * 3, [1.0, 1.4, 1.8], 0.1
        sphi = torch.tensor(inputs.gaussian_state(3, sn_, sdx, snkl, seed=1715, noise=0.0), device="cuda")

        def run_rt(dt, split):
            with torch.cuda.stream(stream):
                q = gpe.Propagator(3, sn_, sdx, dt, snkl, 50.0, precision="f64", stream=stream)
                q.set_splitting(split)
                q.set_state(sphi)
                q.step_real(int(round(sT / dt)))
                out = q.get_state(device=True).clone()
                q.close()
            stream.synchronize()
            return out
        sdts = [2e-3, 1e-3, 5e-4]
        fine = run_rt(sdts[-1] / 8, "strang")
        acc = {}
        for split in ("lie", "strang"):
            errs = [float(torch.linalg.norm(run_rt(dt, split) - fine) / torch.linalg.norm(fine)) for dt in sdts]
            acc[split] = {"rel_l2_err": errs,
                          "observed_order": [float(np.log2(errs[i] / errs[i + 1])) for i in range(len(sdts) - 1)]}
        stres["accuracy"] = {"dt": sdts, **acc}

    # ---- differentiation form: gradient of |<phi_target|phi(T)>|^2 w.r.t. V
    # and g at 128^3 (dx = 0.1, dt = 5e-4, 1000 steps, g = 30, isotropic trap +
    # 8 Gaussian bumps, checkpoints every 50 steps); FP32 forward, FP64
    # accumulation of the gradients.  One timed unit = forward + backward.
    ares = {}
    if not args.no_adjoint:
        an, adx = [128] * 3, [0.1] * 3
        anp = 128 ** 3
        dV, _bp = inputs.gaussian_bumps(3, an, adx, seed=1713, count=8, amp=0.5, center=3.0)
        xs = inputs.axis_coords(128, 0.1)
        harm = 0.5 * (xs[:, None, None] ** 2 + xs[None, :, None] ** 2 + xs[None, None, :] ** 2)
        AV = torch.tensor(harm + dV, device="cuda")
        aphi = torch.tensor(inputs.gaussian_state(3, an, adx, [1.0] * 3), device="cuda")
        atgt = torch.tensor(inputs.gaussian_state(3, an, adx, [1.0] * 3, shift=(0.5, 0.0, 0.0)), device="cuda")
        for prec in ("f32",):
            with torch.cuda.stream(stream):
                q = gpe.Propagator(3, an, adx, 5e-4, [1.0] * 3, 30.0, precision=prec, stream=stream)
                q.set_potential(AV)
                times = []
                for rep in range(1 + 2):
                    q.set_state(aphi)
                    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                    barrier()
                    e0.record(stream)
                    gpe.gp_adjoint_forward(q.h, 1000, 50)
                    e1.record(stream)
                    phiT = q.get_state(device=True).to(torch.complex128)
                    c = torch.sum(torch.conj(atgt) * phiT) * 1e-3
                    lam = (2 * c * atgt * 1e-3).to(q.ctype).contiguous()
                    dJdV = torch.empty(tuple(an), dtype=torch.float64, device="cuda")
                    e_b = torch.cuda.Event(enable_timing=True)
                    e_b.record(stream)
                    torch.cuda.nvtx.range_push(f"adjoint_backward_{prec}")
                    dJdg = gpe.gp_adjoint_backward(q.h, lam.data_ptr(), 1, dJdV.data_ptr(), 1)
                    torch.cuda.nvtx.range_pop()
                    e2.record(stream)
                    barrier()
                    if rep:
                        times.append((e0.elapsed_time(e1), e_b.elapsed_time(e2)))
                q.close()
            tf = sum(t[0] for t in times) / len(times)
            tb = sum(t[1] for t in times) / len(times)
            ares[prec] = {"forward_ms": tf, "backward_ms": tb,
                          "value": world * 1000 * anp / ((tf + tb) * 1e-3),
                          "backward_over_forward": tb / tf, "dJdg": dJdg}

    if args.only and args.only != "headline":
        # profiling run of a single form: report it and stop
        if rank == 0:
            print(json.dumps({"only": args.only, "quench256": qres or None, "adjoint": ares or None,
                              "batched": bres or None, "spherical": sres or None,
                              "axisym": ares_sym or None, "strang": stres or None, "real": rres or None}),
                  flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- end to end through the public API with host buffers (FP32 form)
    e2e = None
    p = make("f32")
    host = torch.tensor(phi0.astype(np.complex64)).pin_memory()
    hnp = host.numpy()
    with torch.cuda.stream(stream):
        for _ in range(2):
            p.set_state(hnp)
            p.step_imag(args.inner)
            p.observables()
        barrier()
        t0 = time.perf_counter()
        for s in range(args.steps):
            p.set_state(hnp)                       # H2D of the state from pinned host memory
            p.step_imag(args.inner)
            ob = p.observables()                   # D2H of the observables
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
    p.close()
    e2e = {"value": world * args.steps * args.inner * np_ / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hnp.nbytes), "d2h_bytes_per_step": 7 * 8}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])

    def roofline(prec):
        r = results[prec]
        kms = r["kernel_ms"]
        axis = max(range(3), key=lambda d: kms[d])
        esize = 8 if prec == "f32" else 16
        # algorithmic bytes: one read + one write of the state per sweep; the
        # fused x + y kernel (shape flag 8) does the x and the y sweep in one
        # launch, so it carries two sweeps' bytes (its DRAM traffic is one
        # read + one write: the intermediate round trip is what fusion saves)
        fused = axis == 0 and bool(r["shapes"]["flags"] & gpe.GP_SHAPE_FUSE_XY)
        algo = (2 if fused else 1) * 2 * esize * np_
        achieved = algo / (kms[axis] * 1e-3) / 1e9
        key = f"sweep_xy_{prec}_imag_128cube" if fused else f"sweep_axis{axis}_{prec}_imag_128cube"
        tr = traffic_record(key)
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": tr, "kernel": key, "sweeps_per_launch": 2 if fused else 1,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s",
                "kernel_ms": kms}

    forms = {}
    for prec in forms_sel:
        r = results[prec]
        v = r["value"]
        forms[prec] = {"value": v, "ms_per_step": 1e3 * r["total_s"] / args.steps,
                       "mu": r["obs"]["mu"], "roofline": roofline(prec)}
    mu_err = abs(mu["f32"]["mu"] - mu["f64"]["mu"]) if "f32" in mu and "f64" in mu else None
    mu_err_df = abs(mu["df64"]["mu"] - mu["f64"]["mu"]) if "df64" in mu and "f64" in mu else None

    def conv_err(prec):
        return abs(mu_conv[prec]["mu"] - mu_conv["f64"]["mu"]) if prec in mu_conv and "f64" in mu_conv else None

    def ratio(a, b):
        return forms[a]["value"] / forms[b]["value"] if a in forms and b in forms else None
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_rate()
    head = forms["f32"]
    r32 = results["f32"]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state+sweeps, f64 reductions",
        "data": "synthetic (seeded Gaussian + 1e-3 SplitMix64 noise)",
        "config": {"workload": w["name"], "global_batch": 1, "inner_steps_per_step": args.inner,
                   "points": np_, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": head["roofline"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
        "forms": {
            "f64": ({"value": forms["f64"]["value"], "ms_per_step": forms["f64"]["ms_per_step"],
                     "roofline": forms["f64"]["roofline"], "gpu_launches": results["f64"]["launches"],
                     "clocks": results["f64"]["clocks"]} if "f64" in forms else None),
            "f32": {"value": forms["f32"]["value"], "speedup_vs_f64": ratio("f32", "f64"),
                    "reduced_density": results["f32"]["reduced_density"],
                    "mu_err_vs_f64_full_job": mu_err, "mu_err_vs_f64_converged_20000_steps": conv_err("f32"),
                    "mu_f32": mu["f32"]["mu"] if "f32" in mu else None,
                    "mu_f64": mu["f64"]["mu"] if "f64" in mu else None},
            "df64": ({"value": forms["df64"]["value"], "ms_per_step": forms["df64"]["ms_per_step"],
                      "speedup_vs_f64": ratio("df64", "f64"),
                      "mu_err_vs_f64_full_job": mu_err_df,
                      "mu_err_vs_f64_converged_20000_steps": conv_err("df64"), "roofline": forms["df64"]["roofline"],
                      "note": "double-float state and sweeps on the FP32 pipes (~48-bit), exact triple-float "
                              "potential factors, FP64 reductions; FP32-ALU bound"} if "df64" in forms else None),
            "quench256": ({"workload": "3d real-time quench, 256^3, dx=0.08, dt=2e-4, isotropic trap, imaginary-time "
                                       f"ground state at g=20 ({args.quench_imag_steps} steps) then g=40; L2 not flushed "
                                       "(state larger than L2)",
                           "f64": qres.get("f64"), "f32": qres.get("f32"), "df64": qres.get("df64"),
                           "speedup_f32_vs_f64": (qres["f32"]["value"] / qres["f64"]["value"]
                                                  if "f64" in qres else None),
                           "speedup_df64_vs_f64": (qres["df64"]["value"] / qres["f64"]["value"]
                                                   if "df64" in qres and "f64" in qres else None)} if qres else None),
            "adjoint": ({"workload": "gradient of |<phi_target|phi(T)>|^2 w.r.t. V (per grid value) and g: 128^3, "
                                     "dx=0.1, dt=5e-4, 1000 real-time steps, g=30, isotropic trap + 8 Gaussian bumps "
                                     "(amplitude <= 0.5), checkpoints every 50 steps; value = forward+backward "
                                     "point-steps/s; FP32 forward, FP64 gradient accumulation",
                         "f32": ares.get("f32")} if ares else None),
            "spherical": ({"workload": "spherically symmetric 3d trap as the radial problem for u = sqrt(4 pi) r phi: "
                                       "513 points on [0, 10.24], dt=1e-4, nu=1, g=100, imaginary time; one 1d line, "
                                       "launch-latency bound", **sres} if sres else None),
            "axisym": ({"workload": "circularly symmetric 2d trap (513 rho points, drho=0.02, nu=1, g=100, "
                                    "dt=1e-4) and axially symmetric 3d trap (rho x z = 256 x 512, drho=dz=0.04, nu=1, "
                                    "lambda=2, g=100, dt=5e-4), imaginary time; rho_i = (i - 1/2) drho",
                        **ares_sym} if ares_sym else None),
            "real_state": ({"workload": "the headline workload (its input is real) with the state held as np real "
                                        "values: imaginary-time maps keep it real; same loop, observables per step, "
                                        "L2 flushed", **rres} if rres else None),
            "strang": ({"workload": "the headline grid (128^3, dt=1e-3, g=50) stepped with the Lie and the Strang "
                                    "splitting N(dt/2), sweeps, N(dt/2), imaginary time (renormalised after the "
                                    "closing half) and real time (halves between steps merged), no observables, L2 "
                                    "flushed before every timed step; accuracy: 64^3 real time to t=0.1 against a "
                                    "dt=6.25e-5 Strang run, FP64",
                        **stres} if stres else None),
            "batched": ({"workload": "64 independent 2d real-time runs, sizes from {128,192,256,384,512}^2 "
                                    "(SplitMix64 seed 1712), dx=0.1, dt=5e-4, g~U[0,50], nu=1, kappa~U[1,2], "
                                    "g=0 trap ground state quenched; one launch per sweep and segment class, "
                                    "graph-captured; L2 flushed before every timed step",
                        "points": bpts,
                        "value_f32": bres["f32"]["value"], "value_f64": bres["f64"]["value"],
                        "speedup_f32_vs_f64": bres["f32"]["value"] / bres["f64"]["value"],
                        "ms_per_step_f32": bres["f32"]["ms_per_step"], "gpu_launches_f32": bres["f32"]["gpu_launches"],
                        "max_abs_mu_diff_f32_vs_f64_after_400_steps": bmu_err,
                        "max_rel_mu_diff_f32_vs_f64_after_400_steps": bmu_rel,
                        "largest_abs_mu_diff_run": bmu_worst} if bres else None),
        },
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.only:
        args.no_quench = args.only != "quench256"
        args.no_adjoint = args.only != "adjoint"
        args.no_batched = args.only != "batched"
        args.no_spherical = args.only != "spherical"
        args.no_strang = args.only != "strang"
        args.no_real = args.only != "real"
        args.no_headline = args.only != "headline"
        if args.only != "headline":
            args.no_cpu_baseline = True
            args.no_mu_check = True
    else:
        args.no_headline = False
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
