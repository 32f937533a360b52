#!/usr/bin/env python3
"""Throughput benchmark of the FDLB solver: cell-velocity updates per second.

Workload: Sod shock tube, Nx = 2^22 cells, Q = 32 velocities, E_l = 0.1 and
Kn = 0.05 on the left state, rho_R = rho_L / 8, fixed ghosts, dense Pr.  One
benchmark step is one full time step of Eq. (rk3) (three fused stage kernels)
over the whole grid; one update advances phi_k and theta_k of one cell by one
step.  With --gpus N every rank advances its own copy (replicas; the value sums
the ranks' updates over the slowest rank's time).

--impl reference times the FP64 CPU oracle on the host cores instead, on a
bounded window of the same workload (see the "sample" field).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ORACLE_SAMPLE_NX = 8192   # cells of the Sod tube (around the membrane) per oracle step


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def _tensor_roofline(achieved_tflops):
    """The closure's training step (BF16 mma.sync with FP32 accumulation; convolution FLOPs of the forward and
    both backward passes) against the measured dense BF16 rate; sustained figure, the step runs for seconds."""
    peaks = _peaks()
    if peaks and "bf16_tflops_sustained" in peaks:
        peak, src = float(peaks["bf16_tflops_sustained"]), "measured (sustained)"
    else:
        peak, src = 1700.0, "fallback (sustained)"
    return {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved_tflops / peak, "traffic": None, "peak_source": src,
            "kernel": "closure training step: conv_kernel, wgrad_kernel, transposed conv_kernel"}


# Sources the stage kernels of each precision are compiled from (the unit and what it includes).
_STAGE_SOURCES = {
    "fp32": ("paper_2211_16933_gb300/csrc/fdlb_f32.cu", "paper_2211_16933_gb300/csrc/fdlb_impl.cuh",
             "paper_2211_16933_gb300/csrc/fdlb_kernels.cuh", "paper_2211_16933_gb300/csrc/qlbm_internal.h",
             "include/qlbm.h"),
    # the generic large-Q kernels (fdlb_lq.cuh) share the FP64 translation unit but not the tiled kernel's code
    "fp64": ("paper_2211_16933_gb300/csrc/fdlb_f64.cu", "paper_2211_16933_gb300/csrc/fdlb_impl.cuh",
             "paper_2211_16933_gb300/csrc/fdlb_kernels.cuh", "paper_2211_16933_gb300/csrc/qlbm_internal.h",
             "include/qlbm.h"),
}


def _code_only(text):
    """C/CUDA source without comments, trailing blanks and empty lines (the sources hold no comment markers
    inside string literals), so that a comment edit leaves the fingerprint unchanged."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def _kernel_hash(precision_name="fp32"):
    """Fingerprint of the code the stage kernel of this precision is compiled from."""
    h = hashlib.sha256()
    for f in _STAGE_SOURCES[precision_name]:
        h.update(_code_only(open(os.path.join(ROOT, f), encoding="utf-8").read()).encode())
    return h.hexdigest()[:16]


def _flops_per_update(precision_name, Q=32):
    """Floating-point operations per cell-velocity update (all three stages) from the committed ncu counts,
    if they were taken on this kernel source and velocity set (the Hermite sum makes them grow with Q)."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_flops.json")))
        e = t.get(precision_name)
        if e and e.get("kernel_hash") == _kernel_hash(precision_name) and e.get("Q") == Q:
            return float(e["flop_per_update"])
    except Exception:
        pass
    return None


# ALU peaks from unit counts and the maximum SM clock (152 SMs, 2.07 GHz): FP32 128 FMA lanes per SM,
# FP64 2 FMA per clock per SM (GB300's 1.25 TFLOP/s FP64 figure); an FMA counts as 2 operations.
ALU_PEAK_TFLOPS = {"fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 152 * 2 * 2 * 2.07e9 / 1e12}


def _alu_roofline(precision_name, updates_per_s, Q=32, kernel="fdlb_stage_kernel"):
    f = _flops_per_update(precision_name, Q)
    if f is None:
        return None
    achieved = f * updates_per_s / 1e12
    peak = ALU_PEAK_TFLOPS[precision_name]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "peak_source": "derived from unit counts and the maximum SM clock",
            "flop_per_update": f, "kernel": kernel}


def _traffic_per_step(precision_name, Q=32, nx=1 << 22):
    """DRAM bytes per step from the committed ncu summary, if it was taken on this kernel source and scaled
    to this workload's size."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")))
        e = t.get(precision_name)
        if (e and e.get("kernel_hash") == _kernel_hash(precision_name) and e.get("Q") == Q
                and e.get("scaled_to_nx") == nx):
            return e["dram_bytes_per_step"]
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int) -> float:
    """Largest value of x over the ranks of the default process group (x itself for one rank); the
    reduction runs on the current GPU for NCCL and on the host for gloo."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, max_seconds: float) -> float:
    """Units processed by all ranks (weak scaling: the same work per rank) over the slowest rank's time."""
    return units_per_rank * ws / max_seconds


def _oracle_sample(w, steps, warmup):
    """Times the FP64 oracle on a window of the workload; returns (updates/s, seconds, sample text)."""
    import oracle as O
    Q, nx = w["Q"], w["nx"]
    p, _ = O.quadrature(Q)
    dx = w["length"] / nx
    from paper_2211_16933_gb300 import inputs
    dt = inputs.cfl_dt(dx, abs(p).max())
    ns = ORACLE_SAMPLE_NX
    a = nx // 2 - ns // 2
    gm = O.make_model(Q, nx, w["length"], dt, w["denseness"], w["kn"], pr_mode=1, bc=O.BC_FIXED)
    r, u, T = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], a, ns)
    gl = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], a - 3, 3)
    gr = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], a + ns, 3)
    m = O.make_model(Q, ns, ns * dx, dt, w["denseness"], w["kn"] * w["length"] / (ns * dx), pr_mode=1,
                     bc=O.BC_FIXED)
    O.set_ghosts(m, np.stack(gl, 1), np.stack(gr, 1))
    ph, th = O.equilibrium_state(m, r, u, T)
    for _ in range(warmup):
        ph, th = O.run(m, ph, th, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        ph, th = O.run(m, ph, th, 1)
    el = time.perf_counter() - t0
    ups = ns * Q * steps / el
    sample = (f"{steps} oracle RK3 steps (FP64, 1 thread) on {ns} cells around the membrane of the "
              f"Nx={nx}, Q={Q} Sod tube, same dx and dt")
    # the window problem and its oracle result, for the error statement of the GPU run
    window = dict(Q=Q, nx=ns, length=ns * dx, dt=dt, denseness=w["denseness"], kn=w["kn"] * w["length"] / (ns * dx),
                  fields=(r, u, T), ghost=[tuple(c) for c in np.stack(gl, 1)] + [tuple(c) for c in np.stack(gr, 1)],
                  steps=warmup + steps, model=m, phi=ph, theta=th)
    return ups, el, sample, window


def _errors_vs_oracle(window, precision, sums=0):
    """L-inf and L2 errors of rho, u, T, P, q of the library's run of the oracle's window problem (same cells,
    ghosts, dx, dt and steps), each normalised by its reference scale: rho_ref, sqrt(T_ref), T_ref,
    rho_ref T_ref (1 + Y0), rho_ref T_ref^(3/2) with rho_ref = T_ref = 1."""
    import oracle as O
    from paper_2211_16933_gb300 import qlbm as q
    r, u, T = window["fields"]
    s = q.Solver(window["Q"], window["nx"], window["length"], window["dt"], window["denseness"], window["kn"],
                 bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_FIELDS, rho=r, u=u, T=T,
                 ghost=np.asarray(window["ghost"], dtype=float).ravel(), precision=precision, pr_mode=q.QL_PR_DENSE,
                 sums=sums)
    s.step(window["steps"])
    f_gpu = s.moments()
    s.close()
    m = window["model"]
    f_or = O.fields(m, window["phi"], window["theta"])
    Y0 = 4.0 * m.eta0 * O.chi_set(m.eta0)
    scale = dict(rho=1.0, u=1.0, T=1.0, P=1.0 + Y0, q=1.0)
    out = {"steps": window["steps"], "cells": window["nx"], "reference": "FP64 oracle, same window",
           "normalisation": "rho_ref, sqrt(T_ref), T_ref, rho_ref T_ref (1 + Y0), rho_ref T_ref^1.5"}
    for k, sc in scale.items():
        d = (f_gpu[k] - f_or[k]) / sc
        out[k] = {"linf": float(np.abs(d).max()), "l2": float(np.sqrt(np.mean(d * d)))}
    return out


def run_reference(args, w):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    steps = max(1, args.steps)
    ups, el, sample, _ = _oracle_sample(w, steps, min(args.warmup, 1))
    line = {"impl": "reference", "metric": "cell-velocity updates/s", "value": ups, "unit": "updates/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "nx": w["nx"], "Q": w["Q"]},
            "cpu_baseline": {"value": ups, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": ups, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e datasheet bandwidth (context beside the measured copy)


def _hbm_roofline(elem, nx, Q, step_s, precision_name, steps_per_launch, kernel):
    """The stepping kernel against the measured copy bandwidth: 16 words of phi and theta per update per step
    (stage 1 reads 2 / writes 2, stages 2-3 read 4 / write 2).  fdlb_run_kernel: one launch runs
    steps_per_launch steps; fdlb_stage_kernel: one launch is one stage, a third of a step."""
    bytes_per_step = 16 * elem * nx * Q
    launches_per_step = 1.0 / steps_per_launch if kernel == "fdlb_run_kernel" else 3.0
    achieved = bytes_per_step / step_s / 1e9
    peaks = _peaks()
    if peaks and "hbm_gbs" in peaks:
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    tr = _traffic_per_step(precision_name, Q, nx)
    # the DRAM view: ncu's DRAM bytes (scaled to this size) over the same time, and both against the nominal
    # HBM3e bandwidth beside the measured copy
    dram = None if tr is None else tr / step_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None if tr is None else tr / launches_per_step, "peak_source": peak_src,
            "algorithmic_bytes_per_launch": bytes_per_step / launches_per_step,
            "launches_per_step": launches_per_step, "kernel": kernel,
            "dram_achieved": dram, "dram_frac": None if dram is None else dram / peak,
            "peak_nominal": HBM_NOMINAL_GBS, "frac_of_nominal": achieved / HBM_NOMINAL_GBS}


def _stepping(q, s, steps):
    """The kernel a solver's step calls launch, and how many launches `steps` steps in one call take."""
    per = s.steps_per_launch()
    if per > 0:
        return "fdlb_run_kernel", -(-steps // per)
    return "fdlb_stage_kernel", 3 * steps


_LAUNCH = {"auto": lambda q: q.QL_LAUNCH_AUTO, "run": lambda q: q.QL_LAUNCH_RUN,
           "stages": lambda q: q.QL_LAUNCH_STAGES}


def _timed_run(s, steps, warmup, stream):
    """Time (ms) of `steps` steps in one call after `warmup` steps, CUDA events on the solver's stream."""
    import torch
    s.step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _forms(args, w, window, q, inputs, dev, stream):
    """The other forms of the precision study and the batched form, each timed on the same GPU (sub-records
    of the bench line): FP32 with FP64 per-cell conserved sums, FP64, and the 4096-instance batch."""
    import torch
    Q, nx = w["Q"], w["nx"]
    pmax = float(np.abs(q.ql_velocity_set(Q)[0]).max())
    dt = inputs.cfl_dt(w["length"] / nx, pmax)
    out = {}
    for name, prec, sums, steps in (("fp32_sums_fp64", q.QL_FP32, q.QL_SUMS_FP64, args.steps),
                                    ("fp64", q.QL_FP64, q.QL_SUMS_DFP32, min(args.steps, args.fp64_steps))):
        s = q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_FIXED,
                     init_kind=q.QL_INIT_RIEMANN, prm=w["prm"], precision=prec, pr_mode=q.QL_PR_DENSE, device=dev,
                     sums=sums, launch=_LAUNCH[args.launch](q))
        ms = _timed_run(s, steps, max(3, min(args.warmup, 3)), stream)
        kern, launches = _stepping(q, s, steps)
        s.close()
        del s
        torch.cuda.empty_cache()
        step_s = ms * 1e-3 / steps
        elem = 4 if prec == q.QL_FP32 else 8
        pname = "fp32" if prec == q.QL_FP32 else "fp64"
        rec = {"value": nx * Q / step_s, "unit": "updates/s", "steps": steps, "ms_per_step": step_s * 1e3,
               "dtype": "f32" if prec == q.QL_FP32 else "f64",
               "sums": "f64 per-cell conserved sums" if sums == q.QL_SUMS_FP64 or prec == q.QL_FP64 else "double-f32",
               "roofline_hbm": _hbm_roofline(elem, nx, Q, step_s, pname, steps / launches, kern),
               "roofline_alu": _alu_roofline(pname, nx * Q / step_s, Q, kern), "kernel": kern,
               "gpu_launches": launches}
        if window is not None:
            rec["errors_vs_oracle"] = _errors_vs_oracle(window, prec, sums)
        out[name] = rec
    if args.batch_n > 0:
        insts, keep, spec = _batch_instances(q, inputs, args.batch_n, 20221130)
        for name, sums in (("batch_fp32", q.QL_SUMS_DFP32), ("batch_fp32_sums_fp64", q.QL_SUMS_FP64)):
            b = q.Batch(insts, precision=q.QL_FP32, sums=sums)
            warps, ctas = b.tune(3)
            upd = b.info()[1]
            b.run(min(args.warmup, 3))
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ks = min(args.steps, 20)
            e0.record(b._stream)
            b.run(ks)
            e1.record(b._stream)
            e1.synchronize()
            flags = b.sync()
            bms = e0.elapsed_time(e1)
            b.close()
            out[name] = {"value": upd * ks / (bms * 1e-3), "unit": "updates/s", "steps": ks, "ms_per_step": bms / ks,
                         "instances": args.batch_n, "updates_per_step": upd, "tuned_warps_per_cta": warps,
                         "tuned_ctas_per_sm": ctas, "nonphysical_instances": int((flags & 1).sum()),
                         "sums": "f64 per-cell conserved sums" if sums == q.QL_SUMS_FP64 else "double-f32",
                         "graph": "one CUDA graph launch of 3 x steps persistent stage kernels per velocity set"}
        del keep
        torch.cuda.empty_cache()
    return out


def run_ours(args, w):
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import inputs
    from paper_2211_16933_gb300 import qlbm as q

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.build()
    Q, nx = w["Q"], w["nx"]
    prec = q.QL_FP32 if args.precision == "fp32" else q.QL_FP64
    elem = 4 if prec == q.QL_FP32 else 8
    pmax = float(np.abs(q.ql_velocity_set(Q)[0]).max())
    dt = inputs.cfl_dt(w["length"] / nx, pmax)
    s = q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                 prm=w["prm"], precision=prec, pr_mode=q.QL_PR_DENSE, device=dev, launch=_LAUNCH[args.launch](q))
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # --- device-resident throughput: K timed steps in one call (one launch of the whole-run kernel, or three
    # stage launches per step)
    s.step(args.warmup)
    barrier()
    clk = ClockSampler(dev)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    total_ms = e0.elapsed_time(e1)
    s.sync()
    max_ms = max_over_ranks(total_ms, ws)
    value = whole_job_rate(nx * Q * args.steps, ws, max_ms * 1e-3)
    kern, launches = _stepping(q, s, args.steps)

    # roofline of the stepping kernel: algorithmic bytes = 16 words per update per step
    hbm_roofline = _hbm_roofline(elem, nx, Q, total_ms * 1e-3 / args.steps, args.precision,
                                 args.steps / launches, kern)
    alu_roofline = _alu_roofline(args.precision, nx * Q * args.steps / (total_ms * 1e-3), Q, kern)
    # FP32: the metric's HBM roofline, the FP32-pipe view beside it; FP64: bound by GB300's FP64 rate
    if args.precision == "fp64" and alu_roofline is not None:
        roofline, other_roofline = alu_roofline, hbm_roofline
    else:
        roofline, other_roofline = hbm_roofline, alu_roofline

    # --- end to end through the C ABI with pinned host buffers: upload initial
    # fields, K x (step + read back domain totals), read back all fields
    e2e = None
    if not args.no_e2e:
        gm_r, gm_u, gm_T = [torch.empty(nx, dtype=torch.float64, pin_memory=True) for _ in range(3)]
        x = (np.arange(nx) + 0.5) / nx
        left = x < 0.5
        gm_r.numpy()[:] = np.where(left, w["prm"][0], w["prm"][3])
        gm_u.numpy()[:] = np.where(left, w["prm"][1], w["prm"][4])
        gm_T.numpy()[:] = np.where(left, w["prm"][2], w["prm"][5])
        outs = [torch.empty(nx, dtype=torch.float64, pin_memory=True) for _ in range(6)]
        tot = torch.empty(3, dtype=torch.float64, pin_memory=True)
        ke = max(1, args.steps)
        barrier()
        t0 = time.perf_counter()
        q.ql_load_fields(s.ctx, gm_r.numpy(), gm_u.numpy(), gm_T.numpy())
        for _ in range(ke):
            q.ql_step(s.ctx, 1)
            q.ql_totals(s.ctx, tot.numpy())
        q.ql_moments(s.ctx, *[o.numpy() for o in outs], tot.numpy())
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, ws)
        e2e = {"value": whole_job_rate(nx * Q * ke, ws, el), "unit": "updates/s",
               "h2d_bytes_per_step": 3 * 8 * nx / ke, "d2h_bytes_per_step": 3 * 8 + 6 * 8 * nx / ke,
               "steps": ke, "pattern": "load fields (pinned) + K x (step, totals) + all fields"}

    cpu = None
    errors = None
    window = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        ups, el, sample, window = _oracle_sample(w, args.cpu_steps, 0)
        cpu = {"value": ups, "unit": "updates/s", "cores": 1, "kind": "oracle", "sample": sample}
        errors = _errors_vs_oracle(window, prec)
    forms = None
    if rank == 0 and ws == 1 and not args.no_forms and prec == q.QL_FP32:
        s.close()
        torch.cuda.empty_cache()
        forms = _forms(args, w, window, q, inputs, dev, stream)

    s.close()
    if rank == 0:
        line = {"metric": "cell-velocity updates/s", "value": value, "unit": "updates/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == q.QL_FP32 else "f64", "data": "synthetic",
                "config": {"workload": w["name"], "nx": nx, "Q": Q, "precision": args.precision,
                           "sums": "per-cell conserved sums: f32 groups of 8 pairs combined in double-f32, u and T in double-f32"
                           if prec == q.QL_FP32 else "f64",
                           "parallelism": f"replicas{ws}" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (3 state buffers of %.2f GiB)" % (
                               2 * Q * nx * elem / 2 ** 30)},
                "roofline": roofline, "roofline_other": other_roofline, "cpu_baseline": cpu,
                "errors_vs_oracle": errors, "e2e": e2e, "forms": forms,
                "gpu_launches": launches, "kernel": kern, "launch": args.launch, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _batch_instances(q, inputs, n, seed, nx_div=1):
    keep, insts, spec = [], [], inputs.batch_instances(n=n, seed=seed)
    for d in spec:
        nx = d["nx"] // nx_div
        p, _ = q.ql_velocity_set(d["Q"])
        dt = inputs.cfl_dt(d["length"] / nx, abs(p).max())
        sound = d["kind"] == "sound"
        insts.append(q.make_instance(d["Q"], nx, d["length"], dt, d["denseness"], d["kn"],
                                     bc=q.QL_BC_PERIODIC if sound else q.QL_BC_FIXED,
                                     init_kind=q.QL_INIT_SOUND if sound else q.QL_INIT_SHOCK, prm=d["prm"],
                                     keep=keep))
    return insts, keep, spec


def run_batch(args):
    """Batched form: 4096 uneven instances (seed 20221130), FP32 state with double-FP32 conserved sums,
    one CUDA-graph launch of K steps; plus time to solution against plain FP64 solves."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import inputs
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    insts, keep, spec = _batch_instances(q, inputs, args.batch_n, 20221130)
    t0 = time.perf_counter()
    b = q.Batch(insts, precision=q.QL_FP32)
    setup_s = time.perf_counter() - t0
    warps, ctas = b.tune(3)
    info = b.info()
    upd_per_step = info[1]
    stream = b._stream
    b.run(args.warmup)
    b.sync()
    clk = ClockSampler(0)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.run(args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks = clk.stop()
    flags = b.sync()
    ms = e0.elapsed_time(e1)
    value = upd_per_step * args.steps / (ms * 1e-3)
    b.close()

    # time to solution on a subset: batched FP32 vs plain FP64 solves one after another
    sub_n, sub_steps = args.tts_instances, args.tts_steps
    sub, keep2, sspec = _batch_instances(q, inputs, sub_n, 20221130)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bs = q.Batch(sub, precision=q.QL_FP32)
    bs.run(sub_steps)
    bs.sync()
    t_batch = time.perf_counter() - t0
    fields32 = [bs.moments(i) for i in range(sub_n)]
    bs.close()
    t_plain, err = 0.0, {k: 0.0 for k in ("rho", "u", "T", "P", "q")}
    for i, I in enumerate(sub):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = q.Solver(I.vs.Q, I.grid.nx, I.grid.length, I.grid.dt, I.denseness, I.kn, bc=I.bc.kind,
                     init_kind=I.init.kind, prm=list(I.init.prm)[:4], precision=q.QL_FP64, pr_mode=q.QL_PR_DENSE)
        s.step(sub_steps)
        f64 = s.moments()
        t_plain += time.perf_counter() - t0
        s.close()
        for k in err:
            err[k] = max(err[k], float(np.abs(f64[k] - fields32[i][k]).max()))
    line = {"metric": "cell-velocity updates/s", "value": value, "unit": "updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch_{args.batch_n}_uneven_sound_and_shock", "instances": args.batch_n,
                       "updates_per_step": upd_per_step, "tuned_warps_per_cta": warps, "tuned_ctas_per_sm": ctas,
                       "graph": "one CUDA graph launch of 3 x steps persistent stage kernels",
                       "sums": "per-cell conserved sums combined in double-f32", "setup_s": setup_s},
            # one persistent launch per stage and velocity set present
            "gpu_launches": 3 * len(set(b.Qs)) * args.steps, "clocks": clocks,
            "nonphysical_instances": int((flags & 1).sum()),
            "time_to_solution": {"instances": sub_n, "steps": sub_steps, "batched_fp32_s": t_batch,
                                 "plain_fp64_sequential_s": t_plain, "speedup": t_plain / t_batch,
                                 "max_field_error_fp32_vs_fp64": err}}
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Learned coarse closure: training pairs from the solver (fine 4096 / coarse 512 cells), training on the
    GPU with the library's BF16 kernels, held-out errors against the fine solve, and time to solution of
    coarse + network against the fine solve (batched FP32, and plain FP64 single-domain solves)."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import learned as L
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    S = args.fine_steps

    def gen(specs, chunk=4096):
        parts = [L.generate(specs[c:c + chunk], fine_steps=S) for c in range(0, len(specs), chunk)]
        return [torch.cat([p[k] for p in parts]) for k in range(4)]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, y, per, _ = gen(L.pair_specs(args.pairs, 0))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    # warm-up (untimed): a short training run on the first batches loads the kernels and builds the
    # step graph once, so that the timed run measures training itself
    wb = min(x.shape[0], 4 * args.train_batch)
    L.train(x[:wb], y[:wb], per[:wb], epochs=2, batch=args.train_batch, lr=args.lr, seed=0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net, losses = L.train(x, y, per, epochs=args.epochs, batch=args.train_batch, lr=args.lr, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    nsamp = (x.shape[0] // args.train_batch) * args.train_batch * args.epochs
    # conv FLOPs of one sample over real channels: forward 2 X 5 sum(cin cout); training about 3x forward
    X = x.shape[1]
    fwd = sum(2 * X * 5 * ci * co for ci, co in [(7, 64), (64, 64), (64, 64), (64, 64), (64, 5)])
    train_tflops = 3 * fwd * nsamp / t_train / 1e12
    del x, y, per

    # held-out pairs, 8 snapshots each: coarse and coarse + network against the fine solve
    xt, yt, pt, _ = gen(L.pair_specs(args.eval_pairs, 10 ** 6))
    pred = L.predict(net, xt, pt, args.train_batch)
    held = {"pairs": args.eval_pairs, "snapshots": 8, "reference": "fine FP32 batched solve",
            "err_coarse": L.field_errors(yt * 0, yt), "err_coarse_plus_net": L.field_errors(pred, yt)}
    del xt, yt, pt, pred

    # time to solution on a subset, final snapshot: coarse FP32 batch + network, fine FP32 batch, and plain
    # FP64 fine solves one after another (the paper's method at full resolution)
    specs = L.pair_specs(args.tts_pairs, 2 * 10 ** 6)
    n = len(specs)
    consts, periodic = L.const_channels(specs, torch.device("cuda", 0))
    cf = torch.empty(n * 5 * L.NC, dtype=torch.float64, device="cuda")
    ff = torch.empty(n * 5 * L.NC, dtype=torch.float64, device="cuda")
    cur = torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ci, keep_c = L._instances(specs, L.NC, lambda s_: 8.0 * L._fine_dt(s_))
    cb = q.Batch(ci, precision=q.QL_FP32)
    cb._stream.wait_stream(cur)
    cb.run(S // 8)
    cb.fields(L.NC, cf)
    cur.wait_stream(cb._stream)
    Cc = cf.view(n, 5, L.NC).permute(0, 2, 1).float().contiguous()
    corr = L.predict(net, torch.cat([Cc, consts[:, None, :].expand(n, L.NC, 2)], dim=2).contiguous(), periodic,
                     args.train_batch)
    learned = (Cc + corr).double().cpu()
    t_learned = time.perf_counter() - t0
    cb.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fi, keep_f = L._instances(specs, L.NF, L._fine_dt)
    fb = q.Batch(fi, precision=q.QL_FP32)
    fb._stream.wait_stream(cur)
    fb.run(S)
    fb.fields(L.NC, ff)
    cur.wait_stream(fb._stream)
    fine32 = ff.view(n, 5, L.NC).permute(0, 2, 1).cpu()
    t_fine32 = time.perf_counter() - t0
    fb.close()
    t0 = time.perf_counter()
    fine64 = []
    for s_ in specs:
        sound = s_["kind"] == "sound"
        sv = q.Solver(s_["Q"], L.NF, s_["length"], L._fine_dt(s_), s_["denseness"], s_["kn"],
                      bc=q.QL_BC_PERIODIC if sound else q.QL_BC_FIXED,
                      init_kind=q.QL_INIT_SOUND if sound else q.QL_INIT_SHOCK, prm=s_["prm"], precision=q.QL_FP64,
                      pr_mode=q.QL_PR_DENSE)
        sv.step(S)
        f = sv.moments()
        sv.close()
        fine64.append(np.stack([f[k].reshape(L.NC, 8).mean(1) for k in L.FIELDS], axis=1))
    t_fine64 = time.perf_counter() - t0
    ref = torch.tensor(np.stack(fine64))
    line = {"metric": "training samples/s", "value": nsamp / t_train, "unit": "samples/s", "n_gpus": 1,
            "steps": args.epochs, "warmup": 2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "learned_closure_conv1d_5x64_k5", "pairs": args.pairs, "snapshots": 8,
                       "fine_cells": L.NF, "coarse_cells": L.NC, "fine_steps": S, "epochs": args.epochs,
                       "batch": args.train_batch, "lr": args.lr, "lr_schedule": "cosine to lr/20"},
            # per training step (graph nodes): gather + pack, 5 convs, mse, 5 wgrads + 5 partial sums,
            # 4 edge terms + 4 transposed convs, loss sum, adam (with the weight casts), step counter
            "gpu_launches": 28 * (nsamp // args.train_batch), "train_conv_tflops": train_tflops,
            "roofline": _tensor_roofline(train_tflops), "data_generation_s": t_gen,
            "train_s": t_train, "loss_per_epoch": losses, "held_out": held,
            "time_to_solution": {"pairs": n, "coarse_fp32_batch_plus_net_s": t_learned,
                                 "fine_fp32_batch_s": t_fine32, "plain_fp64_fine_sequential_s": t_fine64,
                                 "speedup_vs_fp64_fine": t_fine64 / t_learned,
                                 "speedup_vs_fp32_fine_batch": t_fine32 / t_learned,
                                 "err_vs_fp64_fine": {"coarse_plus_net": L.field_errors(learned, ref),
                                                      "fine_fp32_batch": L.field_errors(fine32, ref)}}}
    print(json.dumps(line), flush=True)


def run_launch_sizes(args):
    """Step time of the whole-run launch against per-stage launches across domain sizes (FP32 Sod tube): per row,
    5 warm-up steps, then K steps in one ql_step(K) call between two CUDA events, best of 3, each launch mode on
    a solver of its own.  One JSON line per row, then a summary line."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import inputs
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    rows = []
    for Q, nx in ((8, 1600), (32, 1600), (32, 8192), (32, 32768), (32, 131072), (32, 524288), (32, 2097152),
                  (32, 4194304)):
        K = min(5000, max(20, int(3e8 / (nx * Q))))
        p, _ = q.ql_velocity_set(Q)
        dt = inputs.cfl_dt(1.0 / nx, float(np.abs(p).max()))
        w = inputs.sod_tube(nx=nx, Q=Q)
        row = {"Q": Q, "nx": nx, "K": K}
        for name, lm in (("stages", q.QL_LAUNCH_STAGES), ("run", q.QL_LAUNCH_RUN), ("auto", q.QL_LAUNCH_AUTO)):
            s = q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_FIXED,
                         init_kind=q.QL_INIT_RIEMANN, prm=w["prm"], precision=q.QL_FP32, pr_mode=q.QL_PR_DENSE,
                         launch=lm)
            best = float("inf")
            for _ in range(3):
                best = min(best, _timed_run(s, K, 5, stream) / K)
            if name == "auto":
                row["auto_picks"] = "run" if s.steps_per_launch() > 0 else "stages"
            s.sync()
            s.close()
            row[name + "_ms_per_step"] = best
        row["run_over_stages"] = row["run_ms_per_step"] / row["stages_ms_per_step"]
        print(json.dumps(row), flush=True)
        rows.append(row)
    print(json.dumps({"metric": "ms per step by launch mode", "workload": "launch_sizes", "rows": len(rows),
                      "data": "synthetic"}), flush=True)


def run_dispersion(args):
    """Sound-wave dispersion study (Sec. IV.A): a batch of sound waves over a sweep of E_l, the density-mode
    amplitude sampled in time, a Levenberg-Marquardt fit of c_s, alpha_a, alpha_t against linear theory."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import dispersion as D
    torch.cuda.set_device(0)
    B.build()
    El = np.geomspace(0.01, 6.3, args.sweep)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rows, updates = D.study(El, t_end=5.0, samples=500)
    el = time.perf_counter() - t0
    line = {"metric": "cell-velocity updates/s", "value": updates / el, "unit": "updates/s", "n_gpus": 1,
            "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sound_wave_dispersion_sweep_{args.sweep}", "nx": 128, "Q": 16, "kn": 0.005,
                       "amplitude": 1e-3, "t_end": 5.0, "samples": 500,
                       "timing": "whole study incl. 500 projections and host fits"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def _shock_to_steady(q, inputs, mach, El, precision, max_steps, tol, chunk=8192):
    """Runs the standing shock (128 upstream mean free paths, N_x = 4096, Q = 32) in chunks until the residual
    max |d rho| / (dt rho) over a chunk falls below tol, or max_steps; returns the record of the run."""
    import torch
    w = inputs.normal_shock(mach, El)
    p, _ = q.ql_velocity_set(w["Q"])
    dt = inputs.cfl_dt(w["length"] / w["nx"], float(np.abs(p).max()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = q.Solver(w["Q"], w["nx"], w["length"], dt, El, w["kn"], bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_SHOCK,
                 prm=w["prm"], precision=precision, pr_mode=q.QL_PR_DENSE)
    u1, r2, u2, T2 = q.ql_rankine_hugoniot(s.eta0, 1.0, 1.0, 1.0, mach)
    x = (np.arange(w["nx"]) + 0.5) * w["length"] / w["nx"]
    rho_old, n, hist = s.moments()["rho"], 0, []
    while n < max_steps:
        s.step(chunk)
        n += chunk
        m = s.moments()
        rho = m["rho"]
        res = float(np.max(np.abs(rho - rho_old) / rho) / (chunk * dt))
        rho_old = rho
        mid = 0.5 * (1.0 + r2)
        j = int(np.argmax(rho > mid))
        hist.append((n, res, float(x[j - 1] + (mid - rho[j - 1]) / (rho[j] - rho[j - 1]) * (x[j] - x[j - 1]))))
        if res < tol:
            break
    wall = time.perf_counter() - t0
    far = {"rho1": abs(rho[:8].mean() - 1.0), "u1": abs(m["u"][:8].mean() / u1 - 1.0), "T1": abs(m["T"][:8].mean() - 1.0),
           "rho2": abs(rho[-8:].mean() / r2 - 1.0), "u2": abs(m["u"][-8:].mean() / u2 - 1.0),
           "T2": abs(m["T"][-8:].mean() / T2 - 1.0)}
    s.close()
    last = hist[-1]
    back = hist[max(0, len(hist) - 5)]
    return {"denseness": El, "mach": mach, "precision": "fp64" if precision == q.QL_FP64 else "fp32", "steps": n,
            "t": n * dt, "wall_s": wall, "residual": last[1], "converged": last[1] < tol, "tol": tol,
            "far_field_rel_err": far, "mass_flux_spread": float(np.max(np.abs(rho * m["u"] / u1 - 1.0))),
            "shock_position_l0": last[2], "start_position_l0": 0.5 * w["length"],
            "drift_last_chunks_l0": last[2] - back[2], "drift_steps": last[0] - back[0]}


def run_standing_shock(args):
    """C2: the Mach 1.4 standing shock at E_l = 0.05, 0.1, 0.2 (N_x = 4096, Q = 32, 128 upstream mean free
    paths, Rankine-Hugoniot ghosts) run to a steady profile: FP64 to a residual below 1e-9 (or --shock-steps),
    FP32 to the floor where its update falls below the rounding of the stored state."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import inputs
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    rows = []
    for El in (0.05, 0.1, 0.2):
        rows.append(_shock_to_steady(q, inputs, 1.4, El, q.QL_FP64, args.shock_steps, 1e-9))
        rows.append(_shock_to_steady(q, inputs, 1.4, El, q.QL_FP32, args.shock_steps, 1e-8))
    steps = sum(r["steps"] for r in rows)
    line = {"metric": "time to steady profile", "value": sum(r["wall_s"] for r in rows if r["precision"] == "fp64"),
            "unit": "s", "n_gpus": 1, "steps": steps, "warmup": 0, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "gpu_launches": 3 * steps,
            "config": {"workload": "standing_shock_M1.4_nx4096_Q32", "length_l0": 128, "tol_fp64": 1e-9,
                       "tol_fp32": 1e-8, "max_steps": args.shock_steps,
                       "value": "sum of the FP64 runs' times, solver creation to the last residual check"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_inviscid(args):
    """The paper's near-inviscid shock tube (Sec. IV.B, "Inviscid regime"): L = 80, sigma = 1e-6 (tau~ = 1e-6) with
    eta_i = 0.05 (E_l = 0.4825), chi_SET, N_x = 8e4 (dx = 1e-3), dt = 1e-6, Q = 8, Sod state with the membrane at
    L / 2, fixed ends, dense Pr; FP64 and FP32 to t = --inviscid-t.  Per precision: wall time of the step loop
    (CUDA events), updates/s, and the profile errors against the exact inviscid solution (ql_riemann_exact)
    inside the fan and the two plateaus, eight cells away from their edges, plus the shock position."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    L, nx, El, sigma, dt, Q = 80.0, 80000, 0.4825, 1e-6, 1e-6, 8
    steps = int(round(args.inviscid_t / dt))
    t = steps * dt
    eta0 = q.ql_eta_of_denseness(El)
    x = (np.arange(nx) + 0.5) * L / nx
    xi = (x - 0.5 * L) / t
    waves, r_ex, u_ex, T_ex = q.ql_riemann_exact(eta0, 1.0, (1.0, 1.0), (0.125, 1.0), xi)
    pad = 8 * L / nx / t
    regions = {"fan": (waves["xi_head"] + pad, waves["xi_tail"] - pad),
               "plateau_left": (waves["xi_tail"] + pad, waves["u_c"] - pad),
               "plateau_right": (waves["u_c"] + pad, waves["xi_shock"] - pad)}
    stream = torch.cuda.current_stream()
    rows, fields = [], {}
    for prec, name in ((q.QL_FP64, "fp64"), (q.QL_FP32, "fp32")):
        s = q.Solver(Q, nx, L, dt, El, sigma / (El * L), bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                     prm=(1.0, 0.0, 1.0, 0.125, 0.0, 1.0), precision=prec, pr_mode=q.QL_PR_DENSE)
        s.step(3)  # warm-up: loads the kernels and records the step graph
        s.sync()
        s.close()
        s = q.Solver(Q, nx, L, dt, El, sigma / (El * L), bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                     prm=(1.0, 0.0, 1.0, 0.125, 0.0, 1.0), precision=prec, pr_mode=q.QL_PR_DENSE)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        f = s.moments()
        s.close()
        sec = e0.elapsed_time(e1) * 1e-3
        err = {}
        for reg, (a, b) in regions.items():
            sel = (xi > a) & (xi < b)
            err[reg] = {k: float(np.abs(f[k][sel] - ref[sel]).max() / max(1.0, np.abs(ref[sel]).max()))
                        for k, ref in (("rho", r_ex), ("u", u_ex), ("T", T_ex))}
            err[reg]["cells"] = int(sel.sum())
        mid = 0.5 * (waves["rho2"] + 0.125)
        i = np.flatnonzero((f["rho"][:-1] >= mid) & (f["rho"][1:] < mid) & (x[:-1] > 0.5 * L + waves["u_c"] * t))[0]
        x_s = x[i] + (f["rho"][i] - mid) / (f["rho"][i] - f["rho"][i + 1]) * (x[i + 1] - x[i])
        fields[name] = f
        rows.append({"precision": name, "steps": steps, "t": t, "step_loop_s": sec,
                     "updates_per_s": nx * Q * steps / sec, "errors_vs_inviscid": err,
                     "shock_offset_cells": float((x_s - (0.5 * L + waves["xi_shock"] * t)) / (L / nx))})
    rows[1]["fp32_vs_fp64"] = {k: float(np.abs(fields["fp32"][k] - fields["fp64"][k]).max() /
                                        np.abs(fields["fp64"][k]).max()) for k in ("rho", "u", "T", "P")}
    line = {"metric": "time to solution", "value": rows[0]["step_loop_s"], "unit": "s", "n_gpus": 1, "steps": steps,
            "warmup": 3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "gpu_launches": 3 * steps,
            "config": {"workload": "near_inviscid_shock_tube", "length": L, "nx": nx, "Q": Q, "sigma": sigma, "dt": dt,
                       "denseness": El, "chi": "SET", "t_end": t,
                       "value": "FP64 step loop on CUDA events; FP32 in rows"},
            "waves": waves, "rows": rows}
    print(json.dumps(line), flush=True)


# The paper's timed shock-tube runs (Table comp_time): sigma, Q, N_x, and the LB wall time on one core of an
# Intel Xeon Gold 6330.
PAPER_SHOCK_TABLE = [(0.001, 8, 1600, 62.0), (0.01, 8, 800, 32.0), (0.1, 20, 640, 71.0), (1.0, 200, 160, 176.0)]


def run_paper_table(args):
    """The shock tubes the paper times on one CPU core (Sec. IV, Table comp_time), on the GPU: Sod initial
    state with eta_i = 0.05 (E_l = 0.4825) on the left and eta_i / 8 on the right, T = 1, u = 0, L = 80,
    dt = 1e-3, chi_RET-FM, FP64, dense Pr, fixed ends, to t = 9 (9000 steps: the paper states no final time;
    t = 9 is the reading of its section label, and it gives every row about the same time per update on the
    paper's core).  Per row: time to solution from solver creation to the fields on the host, and the step
    loop alone on CUDA events."""
    import torch
    from paper_2211_16933_gb300 import build as B
    from paper_2211_16933_gb300 import qlbm as q
    torch.cuda.set_device(0)
    B.build()
    El, L, dt, nsteps = 0.4825, 80.0, 1e-3, args.table_steps
    prm = (1.0, 0.0, 1.0, 0.125, 0.0, 1.0)

    def make(sig, Q, nx, prec):
        return q.Solver(Q, nx, L, dt, El, sig / (El * L), bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN, prm=prm,
                        precision=prec, pr_mode=q.QL_PR_DENSE, chi_mode=q.QL_CHI_RET_FM, device=0)

    stream = torch.cuda.current_stream()

    def timed(sig, Q, nx, prec):
        w = make(sig, Q, nx, prec)  # warm-up: loads this row's kernels
        w.step(3)
        w.sync()
        del w
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = make(sig, Q, nx, prec)
        m0 = s.totals()[0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(nsteps)
        e1.record(stream)
        f = s.moments()  # raises QLError on a non-physical state
        return f, time.perf_counter() - t0, e0.elapsed_time(e1) * 1e-3, abs(f["totals"][0] - m0) / m0

    rows = []
    for sig, Q, nx, t_paper in PAPER_SHOCK_TABLE:
        try:
            f, tts, steps_s, dm = timed(sig, Q, nx, q.QL_FP64)
        except q.QLError as e:  # a non-physical state is reported, not timed
            rows.append({"sigma": sig, "Q": Q, "nx": nx, "error": str(e)})
            continue
        tiled = Q in q.SUPPORTED_Q
        row = {"sigma": sig, "Q": Q, "nx": nx, "steps": nsteps, "time_to_solution_s": tts,
               "step_loop_s": steps_s, "updates_per_s": nx * Q * nsteps / steps_s,
               "paper_single_core_s": t_paper, "paper_over_ours": t_paper / tts, "mass_rel_change": dm,
               "path": "tiled" if tiled else "generic large-Q"}
        if tiled:  # the FP32 form on the same run, its fields against the FP64 ones (max-normalised L-inf)
            try:
                f32, tts32, steps32, dm32 = timed(sig, Q, nx, q.QL_FP32)
                err = {k: float(np.abs(f32[k] - f[k]).max() / np.abs(f[k]).max()) for k in ("rho", "u", "T", "P", "q")}
                row["fp32"] = {"time_to_solution_s": tts32, "step_loop_s": steps32,
                               "paper_over_ours": t_paper / tts32, "mass_rel_change": dm32, "linf_vs_fp64": err}
            except q.QLError as e:
                row["fp32"] = {"error": str(e)}
        rows.append(row)
    # stepping kernels per step (graph nodes): tiled, 3 stages + 3 ball averages; generic path, 4 per stage
    launches = sum(r["steps"] * (6 if r["path"] == "tiled" else 12) * (2 if "fp32" in r else 1)
                   for r in rows if "steps" in r)
    line = {"metric": "time to solution", "value": sum(r.get("time_to_solution_s", float("nan")) for r in rows),
            "unit": "s", "gpu_launches": launches,
            "n_gpus": 1, "steps": nsteps, "warmup": 3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "paper_shock_table_chi_ret_fm", "length": L, "dt": dt, "denseness": El,
                       "t_end": nsteps * dt, "reading": "t_end = 9 (not stated in the paper)",
                       "paper_hardware": "1 core of an Intel Xeon Gold 6330"},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--launch", choices=["auto", "run", "stages"], default="auto",
                    help="ql_opts.launch: auto (the library picks by domain size), run (one launch per step call), "
                         "stages (one launch per Runge-Kutta stage)")
    ap.add_argument("--nx", type=int, default=1 << 22)
    ap.add_argument("--q", type=int, default=32)
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32-with-FP64-sums, FP64 and batch sub-records")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--workload", choices=["sod", "batch", "learned", "dispersion", "paper_table", "standing_shock",
                                           "inviscid", "launch_sizes"], default="sod")
    ap.add_argument("--inviscid-t", type=float, default=0.05)
    ap.add_argument("--shock-steps", type=int, default=1_200_000)
    ap.add_argument("--table-steps", type=int, default=9000)
    ap.add_argument("--sweep", type=int, default=16)
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--eval-pairs", type=int, default=1000)
    ap.add_argument("--tts-pairs", type=int, default=16)
    ap.add_argument("--fine-steps", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--train-batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch-n", type=int, default=4096)
    ap.add_argument("--tts-instances", type=int, default=64)
    ap.add_argument("--tts-steps", type=int, default=100)
    args = ap.parse_args()
    from paper_2211_16933_gb300 import inputs
    w = inputs.sod_tube(nx=args.nx, Q=args.q)
    if args.workload == "batch" and args.impl == "ours":
        run_batch(args)
        return
    if args.workload == "learned" and args.impl == "ours":
        run_learned(args)
        return
    if args.workload == "dispersion" and args.impl == "ours":
        run_dispersion(args)
        return
    if args.workload == "paper_table" and args.impl == "ours":
        run_paper_table(args)
        return
    if args.workload == "standing_shock" and args.impl == "ours":
        run_standing_shock(args)
        return
    if args.workload == "inviscid" and args.impl == "ours":
        run_inviscid(args)
        return
    if args.workload == "launch_sizes" and args.impl == "ours":
        run_launch_sizes(args)
        return
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
