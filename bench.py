"""Benchmark: 4D grid-point updates/s of the two-electron Strang propagation.

Workload (default): the full-scale configuration, 256x64 grid per electron
(268,435,456 points, complex64 state of 2 GiB, larger than the 129 MB L2),
dt = 0.002, Coulomb strength 1 (softening 0.25), QPC height 1 / width 2,
packets of energy 3 started at x = -24 / +24.  One bench "step" is one pass
of the hot path at the workload's observation cadence: 100 Strang steps
(two HBM round trips each: the autotuner's launch sequence of kinetic passes
and transposes, potential phase fused) followed by one evaluation
of the observables (norm, energy terms, bunching probability).

  value  = whole-job grid-point updates per second (points x Strang steps /
           time), inputs resident in HBM, max time over ranks;
  e2e    = the same metric through the C ABI with the state copied from
           pinned host memory every step and the observables read back
           (two contexts alternate, so each copy overlaps the other
           context's steps; the one-context serial figure is reported beside);
  roofline = the dominant kernel's algorithmic bytes (16 B per point per
           launch in complex64: one read, one write) over its average
           CUDA-event duration, against the measured HBM copy bandwidth; beside
           it (roofline.alu) its FP32 flops against this GPU's FMA rate
           measured by the library's own throughput kernel.  The per-launch
           durations come from a profiled run of the same bench steps after
           the timed region (the timed region replays CUDA graphs).  traffic
           (DRAM bytes) and ncu_pipes (FMA pipe, issue, L1 data pipe and DRAM
           utilisation) come from the committed ncu summary of the same kernel
           sources, and are null for any other sources;
  cpu_baseline = the FP64 oracle on the host cores on a bounded sample.

Multi-GPU: one process per GPU (torchrun); each rank propagates its own
simulation (weak scaling), no collective on the data path.
``--impl reference`` times the oracle (the only reference this method has).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

INNER = 100          # Strang steps per bench step (the observation cadence)
SAMPLE_NY = 32       # oracle sample: the full-scale workload at 256 x 32 per electron


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--inner", type=int, default=INNER)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-tc-trial", action="store_true")
    ap.add_argument("--workload", default="fullscale", choices=["fullscale", "batched"],
                    help="fullscale: one 256x64 simulation (the headline); batched: 32 simulations of 128x32")
    ap.add_argument("--pin", default=None,
                    help="fix the kernel choice instead of autotuning: 'transposing variant,in-place variant,strategy'")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dft_flops(n: int, tw_general: int = 14, split44: bool = False) -> int:
    """FP32 flops of the in-register DFT of length n (add, sub, mul = 1, FMA =
    2): radix 2 up to 8 points, 4 x 4 for 16; butterflies cost 4, a trivial
    twiddle (1, -i) 0, a (1 -+ i)/sqrt2 twiddle 8 (two sums, two compensated
    scalings) and any other compensated twiddle 14 (two products and two FMAs
    per component)."""
    if n == 1:
        return 0
    if n == 2:
        return 4
    if n == 16 and split44:
        # 4 x 4 split (the x axis of the 256 x 64 grid): eight 4-point DFTs
        # (8 complex additions each), four general and four eighth-root twiddles
        return 8 * 16 + 4 * tw_general + 4 * 8
    tw = 0
    for k in range(1, n // 2):
        if 4 * k == n:
            continue
        tw += 8 if 8 * k in (n, 3 * n) else tw_general
    return 2 * _dft_flops(n // 2, tw_general) + 4 * (n // 2) + tw


def _split(n: int):
    n1 = n if n <= 16 else (16 if n >= 128 else 8)
    return n1, n // n1


def sandwich_flops(nx: int, ny: int, fp64: bool = False) -> float:
    """Algorithmic FP32 flops per point of one kinetic sandwich as the kernels
    compute it: the x and y DFT stages, the compensated inter-stage twiddles
    (14), the T_x/2 and T_y phases applied as v + v*d (8 each) and the 1/(nx ny)
    scale (2).  In FP64 a general twiddle is a plain complex product (6): the
    low parts of the compensated pairs are FP32-only."""
    tw, ph = (6.0 if fp64 else 14.0), 8.0
    dft = (lambda n, s44=False: _dft_flops(n, 6, s44)) if fp64 else (lambda n, s44=False: _dft_flops(n, 14, s44))
    x44 = nx == 256                  # the kernels split the x axis' 16-point DFTs 4 x 4 there
    f = 0.0
    n1, n2 = _split(nx)
    if n2 == 1:
        f += dft(nx, x44) / nx + ph + dft(nx, x44) / nx
    else:
        f += dft(n1, x44) / n1 + tw * (n1 - 1) / n1 + dft(n2, x44) / n2 + ph       # forward x, T_x/2
        f += dft(n2, x44) / n2 + tw * (n2 - 1) / n2 + dft(n1, x44) / n1            # inverse x
    m1, m2 = _split(ny)
    if m2 == 1:
        f += 2 * dft(ny) / ny + ph + 2 + ph
    else:
        f += dft(m1) / m1 + tw * (m1 - 1) / m1
        f += 2 * dft(m2) / m2 + ph + tw * (m2 - 1) / m2
        f += dft(m1) / m1 + 2 + ph
    return f


VPHASE_FLOPS = 22.0   # three deltas combined (two complex products, four adds) and applied


KINETIC_SOURCES = ["hom_fft.cuh", "hom_pass.cuh", "hom_kern.inc", "hom_kern_c64.cu", "hom_kern_c64_rows.cu"]


def code_tokens(text: str) -> str:
    """C/C++/CUDA source with its comments removed and its whitespace
    collapsed, so that editing a comment or the layout leaves it unchanged."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash() -> str:
    """Hash of the code (comments and whitespace ignored) of the sources that
    define the kinetic passes."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1903_02581_gb300", "csrc")
    for f in KINETIC_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update((f + "\n" + code_tokens(fh.read())).encode())
    return h.hexdigest()[:16]


def _ncu_summary() -> dict:
    """Key/value lines of the committed ncu summary, or {} when it is absent
    or was taken on different kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return {}
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256_16") != kernel_hash():
        return {}
    return vals


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary, or
    None when the summary was taken on different kernel sources."""
    v = _ncu_summary().get(f"{kernel}_dram_bytes_per_launch_full_scale")
    return float(v) if v else None


def ncu_pipes(kernel: str):
    """Pipe utilisation of ``kernel`` (fractions of ncu's peaks) from the same
    summary: FMA pipe, instruction issue, L1 data pipe, DRAM; None when absent."""
    vals = _ncu_summary()
    keys = {"fma_pipe": "fma_pipe_active", "issue": "issue_active",
            "l1_data_pipe": "l1_data_pipe_wavefronts", "dram": "dram_throughput"}
    out = {k: float(vals[f"{kernel}_{v}"]) for k, v in keys.items() if f"{kernel}_{v}" in vals}
    return out or None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for i, nm in enumerate(names):
                    if r[5 + i].strip().lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_rate(steps: int = 1, workload: str = "fullscale"):
    """FP64 oracle on the bounded sample; returns (updates/s, seconds, description)."""
    import numpy as np

    from oracle import adapter as A
    from oracle import hom_oracle as O
    from paper_1903_02581_gb300 import workloads as W

    if workload == "batched":
        w = W.batched()
        sim = w["sims"][0]
        w["sims"] = [sim]
        m = A.model_for(w, sim)
        psi = A.initial_state(w, sim)
        V = O.v_total(m)
        t0 = time.perf_counter()
        for _ in range(steps):
            psi = O.strang_step(psi, m, vtot=V)
        sec = time.perf_counter() - t0
        pts = (w["nx"] * w["ny"]) ** 2
        assert np.isfinite(psi).all()
        return pts * steps / sec, sec, (f"oracle Strang step(s) on simulation 0 of the batched workload "
                                        f"(128x32 per electron, {pts:,} points, FP64, numpy), {steps} step(s)")
    w = W.fullscale(sigma=2.0)
    w = W.shrink(w, ny=SAMPLE_NY)
    w["dy"] = 0.25
    sim = w["sims"][0]
    m = A.model_for(w, sim)
    psi = A.initial_state(w, sim)
    V = O.v_total(m)
    t0 = time.perf_counter()
    for _ in range(steps):
        psi = O.strang_step(psi, m, vtot=V)
    sec = time.perf_counter() - t0
    pts = (w["nx"] * w["ny"]) ** 2
    desc = (f"oracle Strang step(s) on the full-scale workload at 256x{SAMPLE_NY} per electron "
            f"({pts:,} points, FP64, numpy), {steps} step(s); per-point work of the x transforms as at "
            f"256x64, y transforms half as long")
    assert np.isfinite(psi).all()
    return pts * steps / sec, sec, desc


def _timed_run(w: dict, device: str, nsteps: int):
    """Observables after nsteps of workload w and the seconds the steps and the
    observables took (graph replay; module load and capture in a warm-up run)."""
    import torch

    from paper_1903_02581_gb300 import binding as H

    pr = H.Propagator(w, device=device)
    pr.step(nsteps)
    pr.observables()
    pr.close()
    pr = H.Propagator(w, device=device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pr.step(nsteps)
    obs = pr.observables()
    sec = time.perf_counter() - t0
    pr.close()
    return obs, sec


def precision_study(device: str):
    """FP32 against FP64 at equal bunching-probability accuracy on the sweep32
    workload (6 simulations, 32x32 per electron, t = 5), plus both precisions
    at an HBM-resident size.

    Accuracy of a run = |P_b - P_b(dt -> 0)| with P_b(dt -> 0) the Richardson
    extrapolation (4 P(dt/2) - P(dt)) / 3 of complex128 runs at dt = 0.005 and
    0.0025 (the Strang product is second order).  complex64 runs at the
    workload's dt = 0.005; complex128 at dt = 0.02, 0.01, 0.005 and 0.0025.
    The FP64 run matched to FP32 is the largest dt whose worst error over the
    6 simulations is no larger than complex64's; time to solution is the
    device time of all steps plus the observables.  Errors against the FP64
    oracle's stored observables at dt = 0.005 (tests/golden/sweep32_oracle.json,
    written by tests/golden/make_golden.py from the oracle only) are reported
    beside them."""
    from paper_1903_02581_gb300 import workloads as W

    path = os.path.join(ROOT, "tests", "golden", "sweep32_oracle.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)
    T = 5.0
    out = {"workload": "sweep32: 6 simulations x 32x32 per electron (1,048,576 points each), t = 5",
           "reference": "FP64 oracle (numpy) observables at dt = 0.005 after 1000 steps",
           "accuracy": "|P_b - P_b(dt->0)|, P_b(dt->0) Richardson-extrapolated from complex128 at dt 0.005/0.0025"}
    runs = {}
    for prec, dt in (("c64", 0.005), ("c128", 0.02), ("c128", 0.01), ("c128", 0.005), ("c128", 0.0025)):
        w = W.sweep32(prec=prec)
        w["dt"] = dt
        n = int(round(T / dt))
        obs, sec = _timed_run(w, device, n)
        runs[(prec, dt)] = (obs, sec, n)
    pts = (32 * 32) ** 2 * 6
    limit = [(4 * b["p_bunch"] - a["p_bunch"]) / 3.0
             for a, b in zip(runs[("c128", 0.005)][0], runs[("c128", 0.0025)][0])]
    table = []
    for (prec, dt), (obs, sec, n) in runs.items():
        g = [s_["obs"]["1000"] for s_ in gold["sims"]]
        table.append({"prec": prec, "dt": dt, "steps": n, "seconds": sec, "updates_per_s": pts * n / sec,
                      "max_abs_p_bunch_err": max(abs(o["p_bunch"] - l) for o, l in zip(obs, limit)),
                      "max_abs_p_bunch_err_vs_oracle_dt0.005": max(abs(o["p_bunch"] - a["p_bunch"])
                                                                   for o, a in zip(obs, g)),
                      "max_norm_drift": max(abs(o["norm"] - 1.0) for o in obs)})
    out["runs"] = table
    f32 = next(r for r in table if r["prec"] == "c64")
    ok = [r for r in table if r["prec"] == "c128" and r["max_abs_p_bunch_err"] <= f32["max_abs_p_bunch_err"]]
    if ok:
        m64 = max(ok, key=lambda r: r["dt"])
        out["equal_accuracy"] = {"c64_dt": f32["dt"], "c64_err": f32["max_abs_p_bunch_err"],
                                 "c64_seconds": f32["seconds"], "c128_dt": m64["dt"],
                                 "c128_err": m64["max_abs_p_bunch_err"], "c128_seconds": m64["seconds"],
                                 "fp32_speedup_at_equal_accuracy": m64["seconds"] / f32["seconds"]}
    # both precisions on one HBM-resident grid: the full-scale workload at
    # 128x64 per electron (complex128: 1 GiB, the largest plane it supports)
    hbm = {}
    for prec in ("c64", "c128"):
        w = W.shrink(W.fullscale(), nx=128)
        w["prec"] = prec
        obs, sec = _timed_run(w, device, 24)
        hbm[prec] = {"seconds_24_steps": sec, "updates_per_s": (128 * 64) ** 2 * 24 / sec,
                     "state_gib": (128 * 64) ** 2 * (8 if prec == "c64" else 16) / 2 ** 30}
    hbm["fp32_speedup"] = hbm["c64"]["updates_per_s"] / hbm["c128"]["updates_per_s"]
    out["hbm_resident_128x64"] = hbm
    return out


def tc_trial(device: str, sm_mhz: float, sms: int):
    """The tensor-core y sandwich (hom_ysandwich_tc, a design trial) on the
    full-scale plane count's worth of 64-point lines: device time per launch,
    cycles per 256-line plane (the unit the FFT form's 12.3 k cycles per plane
    were measured in), and on the first 8192 lines its error and mean norm
    change per line against numpy's FFT in FP64."""
    import numpy as np
    import torch

    from paper_1903_02581_gb300 import binding as H

    nplanes, dt, dy = 4096, 0.002, 0.25
    nlines = nplanes * 256
    rng = np.random.default_rng(11)
    x = (rng.standard_normal((nlines, 64)) + 1j * rng.standard_normal((nlines, 64))).astype(np.complex64)
    d_in = torch.from_numpy(x).to(device)
    d_out = torch.empty_like(d_in)
    wb = H.lib().hom_ysandwich_tc_work_bytes()
    work = torch.empty(wb, dtype=torch.uint8, device=device)
    ms = H.hom_ysandwich_tc(d_in.data_ptr(), d_out.data_ptr(), nlines, dt, dy, work.data_ptr(), wb, 5)
    k = 2 * np.pi * np.fft.fftfreq(64, d=dy)
    x64 = x[:8192].astype(np.complex128)
    ref = np.fft.ifft(np.exp(-0.5j * dt * k * k)[None, :] * np.fft.fft(x64, axis=1), axis=1)
    got = d_out[:8192].cpu().numpy().astype(np.complex128)
    n0 = np.sum(np.abs(x64) ** 2, axis=1)
    ch = (np.sum(np.abs(got) ** 2, axis=1) - n0) / n0
    return {"lines": nlines, "ms_per_launch": ms,
            "cycles_per_256_line_plane": ms * 1e-3 * sm_mhz * 1e6 * sms / nplanes,
            "fft_form_cycles_per_plane": 12.3e3,
            "tensor_tflops_bf16": 6 * 2 * 128 * 128 * nlines / (ms * 1e-3) / 1e12,
            "max_err_rel": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
            "mean_norm_change_per_line": float(np.mean(ch)), "rms_norm_change_per_line": float(np.sqrt(np.mean(ch ** 2)))}


def run_config(w: dict, wname: str, inner: int, world: int) -> dict:
    """The ``config`` object of the JSON line, shared by both arms."""
    pts = (w["nx"] * w["ny"]) ** 2
    batch = len(w["sims"])
    return {"workload": wname, "nx": w["nx"], "ny": w["ny"], "points_per_sim": pts,
            "sims_per_gpu": batch, "state": "complex64", "strang_steps_per_step": inner,
            "observables_per_step": 1, "parallelism": f"replicas{world}",
            "l2": f"inputs larger than L2 ({batch * pts * 8 / 2**30:.0f} GiB state), no flush"}


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1903_02581_gb300 import replicas as RP

    w, wname = RP.rank_workload(args.workload, 0)
    for _ in range(args.warmup):
        oracle_sample_rate(1, args.workload)
    rates, secs = [], 0.0
    desc = ""
    for _ in range(args.steps):
        r, s, desc = oracle_sample_rate(1, args.workload)
        rates.append(r)
        secs += s
    value = len(rates) / sum(1.0 / r for r in rates)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": "4D grid-point updates/s (Strang split-step, two electrons)",
        "value": value, "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * secs / len(rates), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        # the workload the metric is quoted on; what was timed of it is the sample
        "config": run_config(w, wname, args.inner, 1),
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def gb300_arm(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1903_02581_gb300 import binding as H
    from paper_1903_02581_gb300 import build as Bd
    from paper_1903_02581_gb300 import replicas as RP

    if rank == 0:
        Bd.build()
    if world > 1:
        dist.barrier()
    H.lib()

    w, wname = RP.rank_workload(args.workload, rank)
    pts = (w["nx"] * w["ny"]) ** 2
    batch = len(w["sims"])
    pr = H.Propagator(w, device=f"cuda:{local}")
    if args.pin:
        H.hom_autotune_set(pr.ctx, *[int(v) for v in args.pin.split(",")])
    stream = pr.stream

    def bench_step():
        pr.step(args.inner)
        return pr.observables()

    # measured arithmetic peaks of this GPU (the kinetic passes' ALU roofline)
    sink = torch.zeros(4, dtype=torch.float64, device=f"cuda:{local}")
    fp32_peak = H.hom_alu_peak(0, sink.data_ptr(), stream.cuda_stream) / 1e12
    fp64_peak = H.hom_alu_peak(1, sink.data_ptr(), stream.cuda_stream) / 1e12

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: the production path (each hom_step replays its CUDA graph)
    sampler = ClockSampler(local)
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    obs = None
    for _ in range(args.steps):
        obs = bench_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms_max = RP.slowest(ev0.elapsed_time(ev1), device=f"cuda:{local}")
    value = RP.job_rate(world, batch, pts, args.inner * args.steps, ms_max / 1000.0)

    # per-kernel split: the same bench steps again, launched pass by pass with
    # a CUDA-event pair around every kernel on the context's stream (hom_profile)
    H.hom_profile(pr.ctx, True)
    evp0 = torch.cuda.Event(enable_timing=True)
    evp1 = torch.cuda.Event(enable_timing=True)
    evp0.record(stream)
    for _ in range(args.steps):
        bench_step()
    evp1.record(stream)
    torch.cuda.synchronize()
    prof = H.hom_profile_read(pr.ctx)
    tuning = H.hom_autotune_info(pr.ctx)
    H.hom_profile(pr.ctx, False)
    ms_profiled = evp0.elapsed_time(evp1)

    # dominant kernel and its roofline.  Algorithmic bytes: one read and one
    # write of the state per launch (16 B per point in complex64).  Algorithmic
    # FP32 flops per point: the textbook count for one Strang step,
    # 10 log2(points) + 50 (5 N log2 N per complex FFT, ~50 for the phases),
    # which is what the double pass computes (two sandwiches of one particle
    # and the potential); and the kernels' own count of their FP32 operations.
    algo_bytes = batch * pts * 8 * 2
    sw = sandwich_flops(w["nx"], w["ny"])
    nlogn_step = 10.0 * math.log2(pts) + 50.0
    kinds = [("kinetic_pass_t", prof["ms_transposing"], prof["n_transposing"], sw, nlogn_step / 2),
             ("kinetic_pass", prof["ms_in_place"], prof["n_in_place"], sw, nlogn_step / 2),
             ("transpose_state", prof["ms_transpose"], prof["n_transpose"], 0.0, 0.0),
             ("kinetic_pass_double", prof["ms_double"], prof["n_double"], 2 * sw + VPHASE_FLOPS, nlogn_step)]
    peak, peak_kind = load_peaks()
    per_kernel = {}
    for k, t, c_, fl, fs in kinds:
        if not c_:
            continue
        avg = t / c_ / 1000.0
        per_kernel[k] = {"launches": c_, "avg_ms": avg * 1000.0, "share": t / max(sum(q[1] for q in kinds), 1e-12),
                         "hbm_gbs": algo_bytes / avg / 1e9, "hbm_frac": algo_bytes / avg / 1e9 / peak,
                         "fp32_tflops_kernel_count": fl * batch * pts / avg / 1e12,
                         "fp32_frac_kernel_count": fl * batch * pts / avg / 1e12 / fp32_peak,
                         "fp32_tflops_nlogn_count": fs * batch * pts / avg / 1e12,
                         "fp32_frac_nlogn_count": fs * batch * pts / avg / 1e12 / fp32_peak,
                         "flops_per_point_kernel_count": fl, "flops_per_point_nlogn_count": fs}
    name, tot_ms, cnt, _, _ = max(kinds, key=lambda k: k[1])
    dom = per_kernel[name]
    traffic = ncu_traffic(name) if args.workload == "fullscale" else None
    roofline = {"bound": "hbm", "achieved": dom["hbm_gbs"], "peak": peak, "unit": "GB/s", "frac": dom["hbm_frac"],
                "traffic": traffic, "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy)",
                # what actually limits the kinetic passes: FP32 arithmetic and
                # instruction issue, against this GPU's measured FMA rate
                "alu": {"achieved_tflops_nlogn_count": dom["fp32_tflops_nlogn_count"],
                        "achieved_tflops_kernel_count": dom["fp32_tflops_kernel_count"],
                        "peak_tflops": fp32_peak, "frac_nlogn_count": dom["fp32_frac_nlogn_count"],
                        "frac_kernel_count": dom["fp32_frac_kernel_count"],
                        "peak_source": "measured: hom_alu_peak FP32 FMA throughput kernel, best of 3"},
                "fp64_peak_tflops_measured": fp64_peak,
                "sms": torch.cuda.get_device_properties(local).multi_processor_count}
    step_ms = sum(k[1] for k in kinds) / max(args.steps * args.inner, 1)
    roofline.update({
        # one ncu --set full capture of the same kernel sources (null otherwise):
        # how busy the pipes that bound it were
        "ncu_pipes": ncu_pipes(name) if args.workload == "fullscale" else None,
        "hbm_frac_ncu_bytes": (traffic / (dom["avg_ms"] / 1000.0) / 1e9 / peak) if traffic else None,
        "kernel": name, "kernels": per_kernel, "hbm_peak_gbs": peak,
        # the two-round-trip floor: 32 B per point per Strang step (complex64),
        # over the step time of the graph-replayed timed region
        "step_algorithmic_hbm_frac": 2 * algo_bytes / (ms_max / 1000.0 / (args.steps * args.inner)) / 1e9 / peak,
        "step_ms_graph": ms_max / (args.steps * args.inner),
        "step_ms_profiled_kernels": step_ms,
        "ms_per_bench_step_profiled": ms_profiled / args.steps,
        "autotune": tuning})

    # end to end through the C ABI: the state copied in from pinned host memory
    # for every bench step and the observables read back, all inside the timed
    # region.  Two contexts alternate (double buffering): while one steps, the
    # host copies the next step's input into the other, so the copy engine
    # overlaps the kernels as a pipeline over a stream of inputs would.  The
    # same loop with one context (copy, then steps) is reported beside it.
    e2e = None
    if not args.no_e2e:
        host = torch.empty((batch, pts), dtype=torch.complex64, pin_memory=True)
        hview = host.numpy()
        for b in range(batch):
            H.hom_copy_state(pr.ctx, b, hview[b], to_device=False)
        nrep = max(2, args.steps)
        pr2 = H.Propagator(w, device=f"cuda:{local}", init=False)
        if args.pin:
            H.hom_autotune_set(pr2.ctx, *[int(v) for v in args.pin.split(",")])
        for b in range(batch):
            H.hom_copy_state(pr2.ctx, b, hview[b], to_device=True)
        pr2.step(args.inner)                        # autotune and graph capture, untimed
        pr2.observables()
        ctxs = [pr, pr2]

        def copy_in(q):
            for b in range(batch):
                H.hom_copy_state(q.ctx, b, hview[b], to_device=True)     # waits for this copy only

        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        pending = None
        for r in range(nrep):
            q = ctxs[r % 2]
            copy_in(q)                              # overlaps the other context's steps
            if pending is not None:
                # read back the previous step's result before launching this
                # one: the binding orders each call after the caller's stream,
                # so reading it later would also wait for this step
                pending.observables()
            q.step(args.inner)
            pending = q
        pending.observables()
        torch.cuda.synchronize()
        sec = RP.slowest(time.perf_counter() - t0, device=f"cuda:{local}")
        # serial: copy, steps, read back, one context
        torch.cuda.synchronize()
        ts = time.perf_counter()
        reps = []
        for _ in range(nrep):
            ta = time.perf_counter()
            copy_in(pr)
            tb = time.perf_counter()
            pr.step(args.inner)
            pr.observables()
            reps.append([round((tb - ta) * 1e3, 2), round((time.perf_counter() - tb) * 1e3, 2)])
        torch.cuda.synchronize()
        sec_serial = RP.slowest(time.perf_counter() - ts, device=f"cuda:{local}")
        pr2.close()
        e2e = {"value": RP.job_rate(world, batch, pts, args.inner * nrep, sec), "unit": "updates/s",
               "h2d_bytes_per_step": int(hview.nbytes), "d2h_bytes_per_step": 48 * batch, "steps": nrep,
               "pipeline": "two contexts, each step's host-to-device copy overlapping the other context's steps",
               "serial_value": RP.job_rate(world, batch, pts, args.inner * nrep, sec_serial),
               "serial_ms_copy_and_steps_per_rep": reps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sec, desc = oracle_sample_rate(1, args.workload)
        cpu = {"value": rate, "unit": "updates/s", "cores": os.cpu_count(), "kind": "oracle", "sample": desc,
               "seconds": sec}

    precision = None
    if rank == 0 and world == 1 and not args.no_precision:
        precision = precision_study(f"cuda:{local}")

    trial = None
    if rank == 0 and world == 1 and not args.no_tc_trial:
        trial = tc_trial(f"cuda:{local}", (clocks or {}).get("sm_mhz", 2070.0), roofline["sms"])

    launches = args.steps * 4 + sum(k[2] for k in kinds)
    if rank == 0:
        line = {
            "metric": "4D grid-point updates/s (Strang split-step, two electrons)",
            "value": value, "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": run_config(w, wname, args.inner, world),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "precision": precision, "tc_trial": trial, "p_bunch_last": obs[0]["p_bunch"] if obs else None,
            "norm_last": obs[0]["norm"] if obs else None,
        }
        print(json.dumps(line), flush=True)
    pr.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return gb300_arm(args)


if __name__ == "__main__":
    sys.exit(main())
