"""Benchmark of the split-step Crank-Nicolson GP propagator on GB300.

Headline workload: the 3d imaginary-time anisotropic trap -- 128^3 grid,
dx = 0.1, dt = 1e-3, V = (nu^2 x^2 + kappa^2 y^2 + lambda^2 z^2)/2 with
nu, kappa, lambda = 1, 1.4, 1.8, g = 50, seeded-noise Gaussian initial state
(the 5000-step job).  One bench step = ``--inner`` imaginary-time steps
(renormalised every step) followed by one evaluation of the observables, i.e.
one pass of the whole hot path; the metric is grid-point-steps per second.

Forms: the plain FP64 path, the chosen FP32 form (FP32 state and sweeps, FP64
norm/energy/mu reductions and renormalisation; ``value``) and the
double-float form (FP64-class accuracy on the FP32 pipes).  Each form's
observables are compared with the FP64 path's after the full job and when
converged (the FP64 path itself is held to the CPU oracle by the parity
tests).  The 128^3 FP32 state fits in the 129 MB L2, so L2 is flushed (a
256 MB write) before every timed bench step.

Also measured, in the same run: the 256^3 real-time quench (the state is
larger than L2, so its sweeps stream from HBM: the HBM roofline is measured
there), the 64-run batched form, the 128^3 adjoint, and the symmetric-trap,
Strang and real-state forms.  Kernel durations for the rooflines are those of
the kernels launched back to back inside a CUDA graph (as in the step graph).
The FP64 sweeps are bound by the FP64 pipe, so they are also held to the
measured FP64 FMA rate.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step), on the same config.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "name": "imag3d_128: 3d imaginary-time anisotropic trap, 128^3, dx=0.1, dt=1e-3, "
            "nu,kappa,lambda=1,1.4,1.8, g=50, 5000-step job",
    "dim": 3, "n": [128, 128, 128], "dx": [0.1, 0.1, 0.1], "dt": 1e-3,
    "nkl": [1.0, 1.4, 1.8], "g": 50.0, "seed": 1710, "job_steps": 5000,
}
QUENCH = "3d real-time quench, 256^3, dx=0.08, dt=2e-4, isotropic trap, g=20 ground state -> g=40, 10000 steps"
QUENCH_STEPS = 10000
BATCH_STEPS = 4000
METRIC = "3d split-step CN grid-point-steps/s: FP32/batched vs FP64 at fixed mu error"
UNIT = "grid-point-steps/s"
OBS = ("norm", "energy", "mu", "rms_x", "rms_y", "rms_z", "rms_r")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", type=int, default=100, help="time steps per bench step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mu-check", action="store_true",
                    help="skip the untimed accuracy runs (the job's mu, the batch's 400 steps, the Strang study)")
    ap.add_argument("--quench-imag-steps", type=int, default=1500)
    ap.add_argument("--forms", default="f64,f32,df64",
                    help="precision forms to time (the line needs f32; f64 for ratios and errors)")
    ap.add_argument("--only", choices=["headline", "quench256", "batched", "adjoint", "spherical", "strang", "real",
                                       "dp-peak"],
                    help="time one part only (for profiling); the others are skipped")
    ap.add_argument("--details", default=None, help="also write every measured number to this JSON file")
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


SWEEP_SOURCES = ("gpe_common.cuh", "gpe_df.cuh", "gpe_sweep2.cuh", "gpe_step.cuh", "gpe_tma.cuh")


def src_hash():
    """Hash of the sources that define and launch the sweep kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1709_04423_gb300", "csrc")
    for name in SWEEP_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_record(name, key):
    """A per-launch counter (DRAM bytes, FP64 instructions) from a committed ncu
    summary under profiles/, if the sweep sources have not changed since it was
    taken (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
    except Exception:
        return None
    r = rec.get(key)
    if not r or r.get("src_hash") != src_hash():
        return None
    return r


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """SM clock and throttle reasons of the GPU, sampled every 2 ms by a
    thread through NVML (ctypes; nvidia-smi as a fallback); summary() keeps
    the samples between mark_start() and mark_end()."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.samples = []
        self.t0 = self.t1 = None
        self.stop = threading.Event()
        self.nvml = None
        self.smi = None
        self.max_mhz = None

    def __enter__(self):
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            idx = int(vis.split(",")[self.idx]) if vis and vis.split(",")[0].isdigit() else self.idx
            if nv.nvmlDeviceGetHandleByIndex_v2(idx, ctypes.byref(h)) != 0:
                raise OSError("handle")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = float(mx.value)
            self.nvml, self.h = nv, h
            self.thr = threading.Thread(target=self._poll, daemon=True)
            self.thr.start()
        except Exception:
            self.nvml = None
            try:
                self.smi = subprocess.Popen(
                    ["nvidia-smi", "-i", str(self.idx), "--query-gpu=timestamp,clocks.sm,clocks.max.sm,"
                     "clocks_event_reasons.active", "--format=csv,noheader,nounits", "-lms", "50"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self.smi = None
        return self

    def _poll(self):
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop.is_set():
            t = time.perf_counter()
            a = self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk))
            b = self.nvml.nvmlDeviceGetCurrentClocksEventReasons(self.h, ctypes.byref(rs))
            if a == 0 and b == 0:
                self.samples.append((t, float(clk.value), int(rs.value)))
            time.sleep(0.002)

    def mark_start(self):
        self.t0 = time.perf_counter()

    def mark_end(self):
        self.t1 = time.perf_counter()

    def __exit__(self, *a):
        self.stop.set()
        if self.nvml is not None:
            self.thr.join(timeout=2)
        if self.smi is not None:
            self.smi.terminate()
            try:
                out, _ = self.smi.communicate(timeout=5)
            except Exception:
                self.smi.kill()
                out = ""
            # no usable timestamps against perf_counter: keep every sample
            for line in out.strip().splitlines():
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 4 and p[1].replace(".", "").isdigit():
                    self.max_mhz = float(p[2]) if p[2].replace(".", "").isdigit() else self.max_mhz
                    self.samples.append((None, float(p[1]), int(p[3], 16) if p[3].startswith("0x") else 0))

    def summary(self):
        s = [x for x in self.samples if x[0] is None or (self.t0 is not None and self.t0 <= x[0] <= (self.t1 or 1e30))]
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0}
        reasons = sorted({name for _, _, r in s for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(x[1] for x in s), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(s), "source": "nvml" if self.nvml is not None else "nvidia-smi"}


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
            "seconds": round(dt, 2)}


def line_config(world):
    """The config both arms print (the workload, not how a bench step samples it)."""
    w = WORKLOAD
    return {"workload": w["name"], "global_batch": 1, "points": w["n"][0] * w["n"][1] * w["n"][2],
            "parallelism": "replicas" if world > 1 else "single GPU"}


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
        "data": "synthetic, seeded",
        "config": line_config(1),
        "timing": {"inner_steps_per_step": per, "l2": "n/a (CPU)"},
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
    peaks, peak_src = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    peak_note = "measured hbm_gbs" if peak_src == "measured" else "fallback 6.8 TB/s"
    w = WORKLOAD
    np_ = int(np.prod(w["n"]))
    phi0 = inputs.gaussian_state(w["dim"], w["n"], w["dx"], w["nkl"], seed=w["seed"], noise=1e-3)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    only = args.only
    run = (lambda part: only is None or only == part)
    forms_sel = [f for f in ("f64", "f32", "df64") if f in args.forms.split(",")]
    R = {}  # everything measured (written with --details)

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

    def errs(a, b, keys=OBS):
        return {k: abs(a[k] - b[k]) for k in keys}

    # ---- FP64 / FP32 FMA rates of this GPU (the FP64 sweeps' ALU roof)
    dfma, ffma = gpe.gp_fp_fma_rates()
    R["fp_rates"] = {"dfma_per_s": dfma, "ffma_per_s": ffma}
    if only == "dp-peak":
        if rank == 0:
            print(json.dumps({"only": "dp-peak", **R["fp_rates"]}), flush=True)
        return

    def make(prec, n=w["n"], dx=w["dx"], dt=w["dt"], nkl=w["nkl"], g=w["g"], phi=phi0, imag=True):
        with torch.cuda.stream(stream):
            p = gpe.Propagator(w["dim"], n, dx, dt, nkl, g, precision=prec, stream=stream)
            p.autotune(imag=imag, cache=False)   # kernel shapes for this grid (untimed)
            p.set_state(torch.tensor(phi, device="cuda") if isinstance(phi, np.ndarray) else phi)
        return p

    def fp64_alu(kms, key_fmt, npts):
        """FP64 sweeps against the measured DFMA rate: DP thread instructions
        per point from a committed ncu capture of the same kernels."""
        out = []
        for d, t in enumerate(kms):
            rec = profile_record("fp64_dp_ops.json", key_fmt.format(d))
            if not t or not rec:
                out.append(None)
                continue
            rate = rec["dp_inst_per_point"] * npts / (t * 1e-3)
            out.append({"dp_inst_per_point": rec["dp_inst_per_point"], "achieved": rate, "frac": rate / dfma})
        return out

    # ---- headline: 128^3 imaginary time, every form
    head = {}
    if run("headline"):
        mu_job, mu_conv = {}, {}
        if not args.no_mu_check:
            for prec in forms_sel:
                p = make(prec)
                with torch.cuda.stream(stream):
                    p.step_imag(w["job_steps"])
                    mu_job[prec] = p.observables()
                    # continued to 20000 steps: converged (FP32: an exact fixed point of the rounded step)
                    p.step_imag(20000 - w["job_steps"])
                    mu_conv[prec] = p.observables()
                p.close()
        for prec in forms_sel:
            p = make(prec)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            with torch.cuda.stream(stream), ClockSampler(local) as clk:
                for _ in range(args.warmup):
                    p.step_imag(args.inner)
                    p.observables()
                barrier()
                l0 = gpe.gp_kernel_launches()
                torch.cuda.nvtx.range_push(f"timed_{prec}")   # profilers can select the timed launches
                clk.mark_start()
                for s in range(args.steps):
                    flush.fill_(float(s))                 # evict the state from L2
                    ev[s][0].record(stream)
                    p.step_imag(args.inner)
                    p.observables()
                    ev[s][1].record(stream)
                barrier()
                clk.mark_end()
                torch.cuda.nvtx.range_pop()
            launches = gpe.gp_kernel_launches() - l0
            ms = [a.elapsed_time(b) for a, b in ev]
            value, total_s = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
            kms = p.time_sweeps_graph(True, 32)       # in-graph per-launch durations, same state and sizes
            shp = p.shapes()
            p.close()
            head[prec] = {"value": value, "ms_per_step": 1e3 * total_s / args.steps, "launches": launches,
                          "clocks": clk.summary(), "kernel_ms": kms, "shapes": shp}
        R["headline"] = head
        R["headline_mu"] = {"job_end": mu_job, "converged_20000": mu_conv}

    # ---- 256^3 real-time quench: HBM-resident sweeps
    quench = {}
    if run("quench256"):
        qn, qdx, qnp = [256] * 3, [0.08] * 3, 256 ** 3
        qphi = torch.tensor(inputs.gaussian_state(3, qn, qdx, [1.0] * 3, seed=1711, noise=1e-3), device="cuda")
        qsteps, qwarm = min(args.steps, 5), min(args.warmup, 3)
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
                      for _ in range(qsteps)]
                for _ in range(qwarm):
                    q.step_real(args.inner)
                barrier()
                torch.cuda.nvtx.range_push(f"timed_quench_{prec}")
                recs = []
                for s_ in range(qsteps):
                    ev[s_][0].record(stream)
                    # inner steps + the observables at their end, recorded on the device
                    recs.append(q.step_series(False, args.inner, args.inner, device=True))
                    ev[s_][1].record(stream)
                barrier()
                torch.cuda.nvtx.range_pop()
                qt = max_over_ranks(sum(a.elapsed_time(b_) for a, b_ in ev) / 1e3)
                kms = q.time_sweeps_graph(False, 16)
                done = (qwarm + qsteps) * args.inner
                if not args.no_mu_check and done < QUENCH_STEPS:   # the rest of the 10000-step run, untimed
                    q.step_real(QUENCH_STEPS - done)
                    done = QUENCH_STEPS
                ob1 = q.observables()
                shp = q.shapes()
                q.close()
            esize = 8 if prec == "f32" else 16
            step_us = 1e6 * qt / (qsteps * args.inner)
            quench[prec] = {"value": world * qsteps * args.inner * qnp / qt, "us_per_time_step": step_us,
                            "sweep_us": [1e3 * t for t in kms],
                            "sweep_frac_hbm": [(2 * esize * qnp / (t * 1e-3) / 1e9 / hbm) if t else None for t in kms],
                            "step_frac_hbm": 6 * esize * qnp / (step_us * 1e-6) / 1e9 / hbm,
                            "energy_drift_rel": abs(ob1["energy"] / ob0["energy"] - 1),
                            "norm_drift_rel": abs(ob1["norm"] / ob0["norm"] - 1), "obs_start": ob0, "obs_end": ob1,
                            "steps_at_end": done,
                            "rms_r_t": [float(r_[0, 6]) for r_ in recs], "shapes": shp}
            if prec == "f64":
                quench[prec]["alu"] = fp64_alu(kms, "sweep{}_f64_real_256", qnp)
        R["quench256"] = quench

    # ---- batched form: 64 independent 2d real-time runs
    bres, bmu = {}, {}
    if run("batched"):
        P = inputs.batch_runs(seed=1712, nruns=64)
        bsizes = [(int(v), int(v)) for v in P["n"]]
        bnk = [(1.0, float(k)) for k in P["kappa"]]
        bg = [float(v) for v in P["g"]]
        bpts = sum(a * b for a, b in bsizes)
        bphi = [torch.tensor(inputs.gaussian_state(2, list(sz), [0.1, 0.1], list(k)), device="cuda")
                for sz, k in zip(bsizes, bnk)]
        for key, prec, mode in (("f64", "f64", 0), ("f32_class", "f32", 0), ("f32_one_launch", "f32", 1),
                                ("df64", "df64", 0)):
            with torch.cuda.stream(stream):
                bb = gpe.Batch(bsizes, [(0.1, 0.1)] * 64, 5e-4, bnk, bg, precision=prec, stream=stream)
                for i, ph in enumerate(bphi):
                    bb.set_state(i, ph)
                if mode == 0 and prec == "f32":
                    bres["autotune_ms_class_vs_one_launch"] = bb.autotune(32)   # keeps the faster form
                    bres["autotune_choice"] = "one_launch" if bb.mode() == 1 else "class"
                bb.set_mode(mode)
                if not args.no_mu_check and mode == 0:
                    bb.step_real(BATCH_STEPS)
                    bmu[prec] = bb.observables()
                    for i, ph in enumerate(bphi):
                        bb.set_state(i, ph)
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for _ in range(args.warmup):
                    bb.step_real(args.inner)
                    bb.observables()
                barrier()
                l0 = gpe.gp_kernel_launches()
                torch.cuda.nvtx.range_push(f"timed_batched_{key}")
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
            bres[key] = {"value": world * args.steps * args.inner * bpts / bt, "ms_per_step": 1e3 * bt / args.steps,
                         "gpu_launches": blaunch}
        # the FP32 batch as the library runs it after gp_batch_autotune: the faster form
        fast = max(("f32_class", "f32_one_launch"), key=lambda k: bres[k]["value"])
        bres["f32"] = {**bres[fast], "form": fast}
        R["batched"] = {"points": bpts, **bres}
        if bmu:
            worst = {k: max(abs(a[k] - b[k]) for a, b in zip(bmu["f32"], bmu["f64"])) for k in OBS}
            run_w = max(range(64), key=lambda i: abs(bmu["f32"][i]["mu"] - bmu["f64"][i]["mu"]))
            R["batched"]["f32_err_vs_f64_4000_steps"] = {"worst_per_observable": worst, "worst_mu_run": run_w,
                                                         "mu_f64_of_that_run": bmu["f64"][run_w]["mu"]}
            if "df64" in bmu:
                R["batched"]["df64_err_vs_f64_4000_steps"] = {
                    "worst_per_observable": {k: max(abs(a[k] - b[k]) for a, b in zip(bmu["df64"], bmu["f64"]))
                                             for k in OBS}}

    # ---- differentiation form: gradient of |<phi_target|phi(T)>|^2 w.r.t. V and g
    ares = {}
    if run("adjoint"):
        an, adx = [128] * 3, [0.1] * 3
        anp = 128 ** 3
        dV, _bp = inputs.gaussian_bumps(3, an, adx, seed=1713, count=8, amp=0.5, center=3.0)
        xs = inputs.axis_coords(128, 0.1)
        harm = 0.5 * (xs[:, None, None] ** 2 + xs[None, :, None] ** 2 + xs[None, None, :] ** 2)
        AV = torch.tensor(harm + dV, device="cuda")
        aphi = torch.tensor(inputs.gaussian_state(3, an, adx, [1.0] * 3), device="cuda")
        atgt = torch.tensor(inputs.gaussian_state(3, an, adx, [1.0] * 3, shift=(0.5, 0.0, 0.0)), device="cuda")
        with torch.cuda.stream(stream):
            q = gpe.Propagator(3, an, adx, 5e-4, [1.0] * 3, 30.0, precision="f32", stream=stream)
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
                torch.cuda.nvtx.range_push("timed_adjoint_backward_f32")
                e_b.record(stream)
                dJdg = gpe.gp_adjoint_backward(q.h, lam.data_ptr(), 1, dJdV.data_ptr(), 1)
                e2.record(stream)
                barrier()
                torch.cuda.nvtx.range_pop()
                if rep:
                    times.append((e0.elapsed_time(e1), e_b.elapsed_time(e2)))
            q.close()
        tf = sum(t[0] for t in times) / len(times)
        tb = sum(t[1] for t in times) / len(times)
        ares = {"forward_ms": tf, "backward_ms": tb, "value": world * 1000 * anp / ((tf + tb) * 1e-3),
                "backward_over_forward": tb / tf, "dJdg": dJdg}
        R["adjoint_f32"] = ares

    # ---- symmetric traps: spherical (513 radial points), circular (513 rho
    # points), axial (rho x z = 256 x 512); imaginary time, every form
    sym = {}
    if run("spherical"):
        sr = np.arange(513) * 0.02
        cases = {"spherical": (1, [513], [0.02], [1.0], 1e-4, 20000, 2000, dict(spherical=True),
                               (np.sqrt(4 * np.pi) * sr * np.exp(-0.6 * sr ** 2)).astype(np.complex128)),
                 "circular": (1, [513], [0.02], [1.0], 1e-4, 20000, 2000, dict(axisym=True), None),
                 "axial": (2, [256, 512], [0.04, 0.04], [1.0, 2.0], 5e-4, 4000, 200, dict(axisym=True), None)}
        for name, (cd, cn, cdx, cnkl, cdt, cmu_steps, cblock, kw, cphi) in cases.items():
            if cphi is None:
                rho = np.arange(cn[0]) * cdx[0] - 0.5 * cdx[0]
                if cd == 1:
                    cphi = np.exp(-0.3 * rho ** 2)
                else:
                    zz = inputs.axis_coords(cn[1], cdx[1])
                    cphi = np.exp(-0.3 * (rho[None, :] ** 2 + 2.0 * zz[:, None] ** 2))
                cphi = cphi.astype(np.complex128)
            cphi = torch.tensor(cphi, device="cuda")
            cres, cmu = {}, {}
            for prec in forms_sel:
                with torch.cuda.stream(stream):
                    q = gpe.Propagator(cd, cn, cdx, cdt, cnkl, 100.0, precision=prec, stream=stream, **kw)
                    if not args.no_mu_check:   # mu after cmu_steps (untimed)
                        q.set_state(cphi)
                        q.step_imag(cmu_steps)
                        cmu[prec] = q.observables()
                    q.set_state(cphi)
                    for _ in range(args.warmup):
                        q.step_imag(cblock)
                    barrier()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.nvtx.range_push(f"timed_{name}_{prec}")
                    e0.record(stream)
                    for _ in range(args.steps):
                        q.step_imag(cblock)
                    e1.record(stream)
                    barrier()
                    torch.cuda.nvtx.range_pop()
                    st = max_over_ranks(e0.elapsed_time(e1) / 1e3)
                    q.close()
                npts = int(np.prod(cn))
                cres[prec] = {"value": world * args.steps * cblock * npts / st,
                              "us_per_step": 1e6 * st / (args.steps * cblock),
                              "mu": cmu[prec]["mu"] if prec in cmu else None}
            if "f64" in cmu:
                for prec in cres:
                    cres[prec]["mu_diff_vs_f64"] = abs(cmu[prec]["mu"] - cmu["f64"]["mu"])
            sym[name] = cres
        R["symmetric_traps"] = sym

    # ---- real state: the headline workload held as np real values
    rres = {}
    if run("real"):
        for prec in [f for f in forms_sel if f != "df64"]:
            p = make(prec)
            p.set_real_state(True)
            p.autotune(imag=True, cache=False)
            with torch.cuda.stream(stream):
                rmu = None
                if not args.no_mu_check:   # mu after the job (untimed)
                    p.step_imag(w["job_steps"])
                    rmu = p.observables()["mu"]
                    p.set_state(torch.tensor(phi0, device="cuda"))
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(args.steps)]
                for _ in range(args.warmup):
                    p.step_imag(args.inner)
                    p.observables()
                barrier()
                torch.cuda.nvtx.range_push(f"timed_real_{prec}")
                for s in range(args.steps):
                    flush.fill_(float(s))
                    ev[s][0].record(stream)
                    p.step_imag(args.inner)
                    p.observables()
                    ev[s][1].record(stream)
                barrier()
                torch.cuda.nvtx.range_pop()
            ms = [a.elapsed_time(b) for a, b in ev]
            value, total_s = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
            p.close()
            rres[prec] = {"value": value, "ms_per_step": 1e3 * total_s / args.steps, "mu_after_job": rmu}
        R["real_state"] = rres

    # ---- Strang splitting on the headline grid; accuracy study at 64^3
    stres = {}
    if run("strang"):
        for prec in forms_sel:
            p = make(prec)
            stres[prec] = {}
            for mode in ("imag", "real"):
                for split in ("lie", "strang"):
                    p.set_splitting(split)
                    stepper = p.step_imag if mode == "imag" else p.step_real
                    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                          for _ in range(args.steps)]
                    with torch.cuda.stream(stream):
                        p.set_state(torch.tensor(phi0, device="cuda"))
                        for _ in range(args.warmup):
                            stepper(args.inner)
                        barrier()
                        torch.cuda.nvtx.range_push(f"timed_{split}_{mode}_{prec}")
                        for s in range(args.steps):
                            flush.fill_(float(s))
                            ev[s][0].record(stream)
                            stepper(args.inner)
                            ev[s][1].record(stream)
                        barrier()
                        torch.cuda.nvtx.range_pop()
                    ms = [a.elapsed_time(b) for a, b in ev]
                    value, _ = replica_throughput(args.steps * args.inner * np_, sum(ms) / 1e3, device="cuda")
                    stres[prec][f"{split}_{mode}"] = value
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
        if not args.no_mu_check:   # the accuracy study (untimed)
            fine = run_rt(sdts[-1] / 8, "strang")
            for split in ("lie", "strang"):
                e_ = [float(torch.linalg.norm(run_rt(dt, split) - fine) / torch.linalg.norm(fine)) for dt in sdts]
                stres[f"{split}_order"] = [float(np.log2(e_[i] / e_[i + 1])) for i in range(len(sdts) - 1)]
        R["strang"] = stres

    if only is not None:
        if rank == 0:
            print(json.dumps({"only": only, **{k: v for k, v in R.items() if k != "headline_mu"}}, default=str),
                  flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- end to end through the public API with host buffers (FP32 form)
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
            p.observables()                        # D2H of the observables
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0)
    p.close()
    e2e = {"value": world * args.steps * args.inner * np_ / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(hnp.nbytes), "d2h_bytes_per_step": 7 * 8}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline else oracle_rate()

    # ---- the headline's roofline: its dominant kernel as it runs in the step graph
    h32 = head["f32"]
    kms = h32["kernel_ms"]
    axis = max(range(3), key=lambda d: kms[d])
    fused = axis == 0 and bool(h32["shapes"]["flags"] & gpe.GP_SHAPE_FUSE_XY)
    algo = (2 if fused else 1) * 2 * 8 * np_   # one read + one write of the state per sweep
    achieved = algo / (kms[axis] * 1e-3) / 1e9
    key = f"sweep_xy_f32_imag_128cube" if fused else f"sweep_axis{axis}_f32_imag_128cube"
    tr = profile_record("traffic.json", key)
    step_ms = h32["ms_per_step"] / args.inner
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": tr["bytes_per_launch"] if tr else None, "algorithmic_bytes": algo,
            "kernel": key, "peak_source": peak_note,
            "regime": "L2-resident 16.8 MB state, latency-bound; HBM roofline: hbm256",
            "kernel_ms_in_graph": kms, "kernel_sum_over_time_step": sum(kms) / step_ms}
    mu = R["headline_mu"]

    LINE_OBS = ("norm", "energy", "mu", "rms_r")

    def form_err(prec, which):
        d = mu[which]
        return errs(d[prec], d["f64"], LINE_OBS) if prec in d and "f64" in d else None

    q = R.get("quench256", {})

    def qform(prec):
        r = q.get(prec)
        if not r:
            return None
        out = {"value": r["value"], "step_frac_hbm": r["step_frac_hbm"], "sweep_frac_hbm": r["sweep_frac_hbm"]}
        if prec == "f32":
            out.update({"us_step": r["us_per_time_step"], "sweep_us": r["sweep_us"],
                        "dE_rel": r["energy_drift_rel"], "dnorm_rel": r["norm_drift_rel"]})
            # DRAM bytes per sweep launch (committed ncu capture) over one read + one write of the state
            trs = [profile_record("traffic.json", f"sweep_axis{d}_f32_real_256cube") for d in range(3)]
            out["sweep_dram_over_algo"] = [t_["bytes_per_launch"] / (2 * 8 * 256 ** 3) if t_ else None for t_ in trs]
        if r.get("alu"):
            out["sweep_frac_fp64_fma"] = [a["frac"] if a else None for a in r["alu"]]
        return out

    def ratio(a, b):
        return a / b if a and b else None
    hv = {p_: head[p_]["value"] for p_ in head}
    qv = {p_: q[p_]["value"] for p_ in q}
    bat = R.get("batched", {})
    line = {
        "metric": METRIC, "value": h32["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h32["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 state+sweeps, f64 reductions",
        "data": "synthetic, seeded",
        "config": line_config(world),
        "timing": {"inner_steps_per_step": args.inner, "l2": "flushed before every timed step"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": h32["launches"],
        "clocks": h32["clocks"],
        "f32_err_vs_f64": {"job_end_5000": form_err("f32", "job_end"), "converged_20000": form_err("f32", "converged_20000"),
                           "quench256_end": errs(q["f32"]["obs_end"], q["f64"]["obs_end"], LINE_OBS)
                           if "f32" in q and "f64" in q else None,
                           "batched_worst_run_4000": {k: v for k, v in bat.get("f32_err_vs_f64_4000_steps", {})
                                                     .get("worst_per_observable", {}).items() if k in LINE_OBS}},
        "df64_mu_err_vs_f64": {"job_end_5000": (form_err("df64", "job_end") or {}).get("mu"),
                               "converged_20000": (form_err("df64", "converged_20000") or {}).get("mu"),
                               "batched_worst_run_4000": bat.get("df64_err_vs_f64_4000_steps", {})
                               .get("worst_per_observable", {}).get("mu")},
        "hbm256": {"workload": QUENCH, "f32": qform("f32"), "f64": qform("f64"), "df64": qform("df64")},
        "speedups": {"f32_vs_f64_128": ratio(hv.get("f32"), hv.get("f64")),
                     "df64_vs_f64_128": ratio(hv.get("df64"), hv.get("f64")),
                     "f32_vs_f64_256": ratio(qv.get("f32"), qv.get("f64")),
                     "df64_vs_f64_256": ratio(qv.get("df64"), qv.get("f64")),
                     "batched_f32_vs_f64": ratio(bat.get("f32", {}).get("value"), bat.get("f64", {}).get("value")),
                     "batched_df64_vs_f64": ratio(bat.get("df64", {}).get("value"), bat.get("f64", {}).get("value"))},
        "values": {"f64_128": hv.get("f64"), "df64_128": hv.get("df64"),
                   "batched_f32": bat.get("f32", {}).get("value"), "batched_f64": bat.get("f64", {}).get("value"),
                   "batched_df64": bat.get("df64", {}).get("value"),
                   "batched_f32_class_vs_one_launch": [bat.get("f32_class", {}).get("value"),
                                                       bat.get("f32_one_launch", {}).get("value")],
                   "adjoint_f32_fwd_bwd": R.get("adjoint_f32", {}).get("value")},
        "fp_rates": R["fp_rates"],
    }
    for k in ("f32_err_vs_f64", "df64_mu_err_vs_f64", "hbm256", "speedups", "values", "fp_rates"):
        line[k] = compact(line[k], 3)
    line = compact(line)
    print(json.dumps(line, separators=(",", ":")), flush=True)
    if args.details:
        with open(args.details, "w") as f:
            json.dump({"line": line, "all": R}, f, indent=1, default=str)
    if world > 1:
        torch.distributed.destroy_process_group()


def compact(obj, sig=4):
    """Floats to `sig` significant digits (the line stays within the few KB
    of output a driver keeps)."""
    if isinstance(obj, float):
        return float(f"{obj:.{sig}g}")
    if isinstance(obj, dict):
        return {k: compact(v, sig) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [compact(v, sig) for v in obj]
    return obj


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
