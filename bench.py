"""Benchmark: FP64 grid-point updates/s of the time-domain Teukolsky step on GB300.

Workload: Kerr a = 0.9M, s = -2, m = 2, grid 8192 r* x 128 theta,
r* in [-100M, 1000M], circular equatorial orbit r0 = 10M with a Gaussian source
of width 0.05M, waveform sampled at r* = 500M every 10 steps, FP64, time step
c_theta = 0.8 with the angular Kreiss-Oliger dissipation at eps = 1.  One
benchmark step = `--chunk` time steps of Eqs. (3)-(4) (graph replays of the
split kernels), on inputs resident in HBM.  The per-step working set (state
2 x 33.5 MB + coefficient planes 193 MB) is larger than the 129 MB L2.  The
default run also reports the batched workloads (waveforms/s batched against
one job at a time) and the serving stream (p50/p99 latency), each on a stated
fraction of its step counts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--chunk C] [--impl reference]

Under torchrun (N > 1) every rank evolves its own copy of the workload
(independent problems, no collective on the data path); `value` is the sum
over ranks divided by the slowest rank's time.

--impl reference times the FP64 CPU oracle (the reference arm) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kerr_a0.9_s-2_m2_8192x128_r0_10"
HBM_PROBE = "kerr_a0.9_s-2_m2_32768x512_r0_10"   # state far beyond L2: where "% of HBM roof" is quoted
METRIC = "FP64 grid-pt updates/s"
UNIT = "grid-pt updates/s"
# FP64 work of one interior point update in the folded formulation of
# Eqs. (3)-(4): 8 adds + 4 multiplies + 44 FMAs = 100 flops (algorithmic);
# per kernel: predictor (one mid-point) 4 adds + 4 multiplies + 20 FMAs = 48 flops,
# corrector (one node) 4 adds + 24 FMAs = 52 flops.  The angular dissipation
# adds to the corrector, per real component of Phi and Pi, 3 pair sums and the
# weighted sum k1 s1 + k2 s2 + k3 s3 (1 multiply + 2 FMAs), and applies it with
# the central weight (1 FMA for Phi, 1 multiply for Pi): 10 + 9 flops per
# complex component pair, 38 per node (algorithmic: the fixed-point kernels
# form these sums as exact integer sums instead).
FLOPS_PER_UPDATE = 100
FLOPS_PREDICTOR_POINT = 48
FLOPS_CORRECTOR_POINT = 52
FLOPS_DISSIPATION_POINT = 38
# Algorithmic HBM bytes of one point update: read u^n, write u^{n+1} (4 doubles each).
BYTES_PER_UPDATE_ALG = 64
# Nominal FP64 rate of GB300 (152 SMs x 2 FP64 FMA/clk/SM x 2 flops x 2.07 GHz).
FP64_PEAK_FLOPS = 1.25e12
# Instruction issue: 4 warp schedulers per SM, one warp instruction each per clock.
ISSUE_PER_CLK_SM = 4
# How the kernels execute that work: the Phi rows and the sums tau, sigma on
# the FP64 pipe (20 instructions per update, adds and multiplies issued as
# FMAs), the Pi rows as fixed-point sums of 38 exact integer products per
# update on the integer pipes.  The dissipation adds 2 FP64 instructions (its
# term in the Phi row) and four exact integer sixth differences per node; with
# eps/64 a power of two (eps = 1 here) its term in the Pi rows enters their
# fixed-point sums as an integer addend, not a product.  Measured FP64 issue
# rate on GB300 (FMA-chain probe): 1.906 per clock per SM.
FP64_INSTR_PER_UPDATE = 20
FIXED_POINT_PRODUCTS_PER_UPDATE = 38
FP64_INSTR_DISSIPATION = 2
FIXED_POINT_PRODUCTS_DISSIPATION = 0
FP64_FMA_PER_CLK_SM = 1.906
NUM_SMS = 152
# --batch-mode letters -> index into the binding's BATCH_FORMS (the index
# teuk_batch_autotune reports): per-job, multi-job one CTA per tile, persistent
BATCH_FORM_INDEX = {"1": 0, "0": 1, "p": 3}
# DRAM bytes (read + write) per launch of each step kernel from one ncu capture
# of the split kernels on the 8192 x 128 workload at step 40192 (a developed
# field), valid for the kernel and launch sources whose SHA-256 is recorded
# here; reported as null otherwise.
NCU_TRAFFIC = dict(predictor=125.86e6 + 15.95e6, corrector=151.04e6 + 19.77e6,
                   # warp instructions per launch (smsp__inst_executed.sum), same capture
                   predictor_inst=27.866492e6, corrector_inst=46.855361e6,
                   sources_sha256="ced5fa33b2030b52cb83bb77c9acfd39a9f6eeb00ed3b37a44dcfc8939d1c634")
TRAFFIC_SOURCES = ["paper_1206_0270_gb300/csrc/teuk_kernels.cu",   # kernels and their launchers
                   "paper_1206_0270_gb300/csrc/teuk_fixed.h",      # their arithmetic
                   "paper_1206_0270_gb300/csrc/teuk_internal.h",   # parameter layout, thread limits
                   "paper_1206_0270_gb300/csrc/teuk_handle.h"]     # launch defaults (PDL, graph chunk)


def sources_sha256():
    """SHA-256 of the code of TRAFFIC_SOURCES with comments and blank space
    removed, so that editing a comment does not invalidate the capture."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                 # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json),
    else the stated fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback: 6.8 TB/s, one earlier GB300 measurement"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, device) -> float:
    """Max of x over the ranks of the default process group (x itself when
    there is no group).  NCCL needs device="cuda"; gloo works with "cpu"."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, slowest_seconds: float) -> float:
    """Replicas: every rank processes units_per_rank; the job takes as long as
    the slowest rank."""
    return world * units_per_rank / slowest_seconds


def workload():
    from paper_1206_0270_gb300 import inputs
    return dict(inputs.WORKLOADS[WORKLOAD])


# ---------------------------------------------------------------------------
# Reference arm / CPU baseline: the oracle on host cores
# ---------------------------------------------------------------------------

def oracle_rate(steps_per_sample: int, samples: int, warmup: int = 0):
    """Time the oracle on the full 8192 x 128 grid of the workload."""
    from oracle import oracle as O
    w = workload()
    dt = O.stable_dt(w["nr"], w["nth"], w["rstar_min"], w["rstar_max"], w["a"], w["s"], w["m"],
                     w["c_r"], w["c_theta"])
    S = O.Solver(w["nr"], w["nth"], w["rstar_min"], w["rstar_max"], dt, w["a"], w["s"], w["m"])
    S.set_dissipation(w["eps"])
    S.set_initial(np.zeros((w["nr"], w["nth"]), complex))
    S.set_source(**w["source"])
    S.set_extraction(w["extraction"]["rstar"], w["extraction"]["every"])
    for _ in range(warmup):
        S.step(steps_per_sample)
    times = []
    for _ in range(samples):
        t0 = time.perf_counter()
        S.step(steps_per_sample)
        times.append(time.perf_counter() - t0)
    upd = (w["nr"] - 2) * w["nth"] * steps_per_sample
    return upd, times


def cores_used():
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    per = args.ref_steps
    upd, times = oracle_rate(per, args.steps, warmup=args.warmup)
    total = sum(times)
    value = upd * args.steps / total
    sample = ("FP64 C oracle (OpenMP over r* rows), 8192x128 Kerr a=0.9 grid with source and angular "
              "dissipation (eps = 1), %d time steps per benchmark step" % per)
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * total / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, nr=8192, nth=128, time_steps_per_step=per),
                cpu_baseline=dict(value=value, unit=UNIT, cores=cores_used(), kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return dict(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1206_0270_gb300 import build
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_1206_0270_gb300 import teuk as T

    w = workload()
    nr, nth = w["nr"], w["nth"]
    dt = T.stable_dt(nr, nth, w["rstar_min"], w["rstar_max"], w["a"], w["s"], w["m"], w["c_r"], w["c_theta"])
    stream = torch.cuda.Stream()
    S = T.Solver(nr, nth, w["rstar_min"], w["rstar_max"], dt, w["a"], w["s"], w["m"], stream=stream)
    S.set_dissipation(w["eps"])
    S.set_initial(np.zeros((nr, nth), complex), np.zeros((nr, nth), complex))
    S.set_source(**w["source"])
    if args.pre_steps:  # untimed evolution first (profiles of a developed field)
        S.step(args.pre_steps)
        torch.cuda.synchronize()
    ex = w["extraction"]
    samples_per_step = args.chunk // ex["every"]
    S.set_extraction(ex["rstar"], ex["every"], capacity=max(16, 2 * samples_per_step * (args.steps + args.warmup + 2)))
    upd_per_step = (nr - 2) * nth * args.chunk

    # ---- device-resident throughput -------------------------------------------------
    for _ in range(args.warmup):
        S.step(args.chunk)
    torch.cuda.synchronize()
    # the state where the timed region starts: the end-to-end leg below times
    # the same time steps, resumed from it through the C ABI
    pin = lambda: torch.zeros((nr, nth), dtype=torch.complex128, pin_memory=True).numpy()
    phi_h, pi_h = pin(), pin()
    T._check(T.teuk_get_state(S.h, phi_h.ctypes.data_as(T._dp), pi_h.ctypes.data_as(T._dp)), S.h, "teuk_get_state")
    n_start = S.step_count
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            S.step(args.chunk)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = reduce_max(total_ms, "cuda")
    if ws > 1:
        torch.distributed.barrier()
    assert S.check_finite(), "state became non-finite"
    S.state_at_end = S.state()
    launches = args.steps * S.launches_for(args.chunk)
    value = whole_job_rate(ws, upd_per_step * args.steps, total_ms / 1e3)

    # ---- per-kernel roofline ------------------------------------------------------------
    # The time step is two kernels of nearly equal cost; each is timed live with
    # CUDA events on the solver's stream (teuk_time_kernels, plain launches) and
    # the longer one is reported as the dominant kernel.
    per_launch_s = (total_ms / 1e3) / (args.steps * args.chunk)     # one step, inside the graph replay
    upd_per_launch = (nr - 2) * nth
    ms_pred, ms_corr = S.time_kernels(args.kernel_timing_steps)
    ko = w["eps"] > 0
    flops_corr = FLOPS_CORRECTOR_POINT + (FLOPS_DISSIPATION_POINT if ko else 0)
    flops_update = FLOPS_PER_UPDATE + (FLOPS_DISSIPATION_POINT if ko else 0)
    kern = dict(lw_predict_split=(FLOPS_PREDICTOR_POINT * (nr - 1) * nth, ms_pred, "predictor"),
                lw_correct_split=(flops_corr * (nr - 2) * nth, ms_corr, "corrector"))
    dom = max(kern, key=lambda k: kern[k][1])
    flops, ms, key = kern[dom]
    achieved = flops / (ms / 1e3)
    same_src = NCU_TRAFFIC["sources_sha256"] == sources_sha256()
    measured_fp64 = NUM_SMS * FP64_FMA_PER_CLK_SM * 2 * 2.07e9     # the DFMA probe's rate at 2070 MHz
    roofline = dict(bound="alu", achieved=achieved / 1e12, peak=FP64_PEAK_FLOPS / 1e12, unit="TFLOP/s",
                    frac=achieved / FP64_PEAK_FLOPS, traffic=NCU_TRAFFIC[key] if same_src else None,
                    kernel=dom, launch_ms=ms,
                    peak_source="nominal FP64 (152 SMs x 2 FMA/clk x 2 flops x 2.07 GHz); achieved counts the "
                                "algorithmic FP64 flops, of which the Pi-row products run on the integer pipes",
                    frac_of_measured_dfma=achieved / measured_fp64,
                    measured_dfma_tflops=measured_fp64 / 1e12,
                    flops_per_launch=flops, flops_per_node=flops_corr if key == "corrector" else FLOPS_PREDICTOR_POINT,
                    kernels={k: dict(ms=v[1], tflops=v[0] / (v[1] / 1e3) / 1e12) for k, v in kern.items()},
                    step_in_graph=dict(ms=per_launch_s * 1e3,
                                       tflops=flops_update * upd_per_launch / per_launch_s / 1e12),
                    hbm_alg_gbs=BYTES_PER_UPDATE_ALG * upd_per_launch / per_launch_s / 1e9)
    # the binding resource of this integer-heavy path: instruction issue, from
    # the warp instructions per launch of the ncu capture (valid while the
    # kernel sources hash to the captured version) over the CUDA-event times
    if same_src:
        inst = {"lw_predict_split": NCU_TRAFFIC["predictor_inst"], "lw_correct_split": NCU_TRAFFIC["corrector_inst"]}
        issue_peak = NUM_SMS * ISSUE_PER_CLK_SM * 2.07e9
        roofline["issue"] = dict(
            unit="warp instructions/s", peak=issue_peak,
            peak_source="152 SMs x 4 schedulers x 1 warp instruction/clk x 2.07 GHz",
            kernels={k: dict(warp_instructions=inst[k], achieved=inst[k] / (kern[k][1] / 1e3),
                             frac=inst[k] / (kern[k][1] / 1e3) / issue_peak) for k in inst},
            thread_instructions_per_update=32 * (inst["lw_predict_split"] / ((nr - 1) * nth) +
                                                 inst["lw_correct_split"] / ((nr - 2) * nth)))
    # secondary roof: HBM (not binding here), against the measured copy bandwidth
    hbm_peak, hbm_src = measured_hbm_gbs()
    dram_step = (NCU_TRAFFIC["predictor"] + NCU_TRAFFIC["corrector"]) if same_src else None
    roofline["hbm"] = dict(
        peak_gbs=hbm_peak, peak_source=hbm_src,
        algorithmic_gbs=roofline["hbm_alg_gbs"], frac_algorithmic=roofline["hbm_alg_gbs"] / hbm_peak,
        dram_gbs=None if dram_step is None else dram_step / per_launch_s / 1e9,
        frac_dram=None if dram_step is None else dram_step / per_launch_s / 1e9 / hbm_peak)

    # ---- end to end through the C ABI with host buffers ------------------------------
    # Every step uploads the state from pinned host memory (teuk_set_state at
    # the current step count, so the evolution resumes where it stood), runs
    # the chunk, reads the waveform samples back and downloads the new state:
    # the same time steps as the device-resident region, plus the copies.
    t_buf = np.zeros(samples_per_step + 1)
    w_buf = torch.zeros((samples_per_step + 1, nth), dtype=torch.complex128, pin_memory=True).numpy()
    E = T.Solver(nr, nth, w["rstar_min"], w["rstar_max"], dt, w["a"], w["s"], w["m"], stream=stream)
    E.set_dissipation(w["eps"])
    E.set_source(**w["source"])
    E.set_extraction(ex["rstar"], ex["every"], capacity=samples_per_step + 1)
    import ctypes as C
    dp = lambda a: a.ctypes.data_as(T._dp)
    e2e_at = [n_start]

    def e2e_step():
        T._check(T.teuk_set_state(E.h, dp(phi_h), dp(pi_h), e2e_at[0]), E.h, "teuk_set_state")   # H2D
        E.step(args.chunk)
        n = C.c_long()
        rc = T.teuk_extract(E.h, dp(t_buf), dp(w_buf), len(t_buf), C.byref(n))    # D2H waveform (synchronises)
        T._check(rc, E.h, "teuk_extract")
        T._check(T.teuk_get_state(E.h, dp(phi_h), dp(pi_h)), E.h, "teuk_get_state")  # D2H state
        e2e_at[0] += args.chunk
        return n.value
    # one untimed step (graph capture, first-touch of the pinned buffers), then
    # back to the snapshot where the device-resident timed region started
    snap = (phi_h.copy(), pi_h.copy())
    for _ in range(max(1, args.warmup)):
        e2e_step()
    np.copyto(phi_h, snap[0])
    np.copyto(pi_h, snap[1])
    e2e_at[0] = n_start
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nsamp = 0
    for _ in range(args.steps):
        nsamp = e2e_step()
    e2e_s = reduce_max(time.perf_counter() - t0, "cuda")
    # the resumed run reproduces the device-resident one: same steps, same bits
    e2e_same = bool(np.array_equal(phi_h, S.state_at_end[0])) if hasattr(S, "state_at_end") else None
    e2e = dict(value=whole_job_rate(ws, upd_per_step * args.steps, e2e_s), unit=UNIT,
               h2d_bytes_per_step=2 * nr * nth * 16,
               d2h_bytes_per_step=2 * nr * nth * 16 + nsamp * (nth * 16 + 8),
               time_steps=[n_start, e2e_at[0]], same_steps_as_value=True, bitwise_equal_to_value=e2e_same)
    E.close()

    # ---- the same workload with every Pi-row product as an FP64 FMA ------------------
    F = T.Solver(nr, nth, w["rstar_min"], w["rstar_max"], dt, w["a"], w["s"], w["m"], stream=stream)
    F.set_dissipation(w["eps"])
    F.set_option(T.TEUK_OPT_FIXED_POINT, 0)
    F.set_initial(np.zeros((nr, nth), complex), np.zeros((nr, nth), complex))
    F.set_source(**w["source"])
    F.set_extraction(ex["rstar"], ex["every"], capacity=max(16, 2 * samples_per_step * 16))
    n_fp64 = min(args.steps, 5)
    for _ in range(max(1, args.warmup)):
        F.step(args.chunk)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_fp64):
        F.step(args.chunk)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = reduce_max(e0.elapsed_time(e1), "cuda")
    all_fp64 = dict(value=whole_job_rate(ws, upd_per_step * n_fp64, fp64_ms / 1e3), unit=UNIT, steps=n_fp64,
                    arithmetic="every Pi-row product as an FP64 FMA (TEUK_OPT_FIXED_POINT 0)")
    F.close()
    hbm_probe = run_hbm_probe(T, stream, ws, hbm_peak, hbm_src, same_src) if args.hbm_probe else None

    if rank != 0:
        S.close()
        return 0

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                evolved_M_per_s=value / ((nr - 2) * nth) * dt,
                config=dict(workload=WORKLOAD, nr=nr, nth=nth, a=w["a"], s=w["s"], m=w["m"],
                            rstar=[w["rstar_min"], w["rstar_max"]], dt=dt, c_r=w["c_r"], c_theta=w["c_theta"],
                            eps=w["eps"], time_steps_per_step=args.chunk,
                            evolved_M_per_step=args.chunk * dt,
                            timed_time_steps=[n_start, n_start + args.steps * args.chunk],
                            workload_time_steps=w["steps"],
                            kernel="split predictor/corrector tiles, CUDA-graph replay",
                            arithmetic="FP64; Pi-row sums as exact integer products in 64-bit fixed point, "
                                       "rounded once to FP64 (error <= n 2^-57 max|c x| + 2^-53 |sum|)",
                            l2="inputs larger than L2 (state 2x33.5 MB + coefficients 193 MB per time step)",
                            parallelism="replicas" if ws > 1 else "single GPU"),
                roofline=roofline, e2e=e2e, gpu_launches=int(launches), all_fp64=all_fp64, hbm_probe=hbm_probe,
                step_ms_min=min(step_ms), step_ms_median=statistics.median(step_ms))
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
        # FP64 pipe occupancy at the clock seen during the timed region
        pipe = NUM_SMS * FP64_FMA_PER_CLK_SM * clocks["sm_mhz"] * 1e6
        fp64_instr = FP64_INSTR_PER_UPDATE + (FP64_INSTR_DISSIPATION if ko else 0)
        roofline["fp64_instr_per_update"] = fp64_instr
        roofline["fixed_point_products_per_update"] = (FIXED_POINT_PRODUCTS_PER_UPDATE +
                                                       (FIXED_POINT_PRODUCTS_DISSIPATION if ko else 0))
        roofline["fp64_pipe_frac"] = fp64_instr * upd_per_launch / per_launch_s / pipe
    if ws == 1 and args.batched:
        # the other parts of the workload metric, on stated fractions of their
        # step counts: batched waveforms/s against one job at a time, and the
        # serving stream's latency
        from paper_1206_0270_gb300 import inputs, serve as SV
        line["batched"] = optional_block(lambda: [
            batch_result(T, "batch_modes", 0.2, "all"), batch_result(T, "template_bank", 0.01, "all"),
            batch_result(T, "small_bank", 0.2, "all")])
        line["serving"] = optional_block(lambda: dict(
            serving_result(T, SV, inputs.serving_requests(64, 4.0), slice_steps=640, fill_points=2_000_000,
                           memory_gb=200.0, policies=("async", "async-remaining")),
            rate_per_s=4.0, step_fraction=1.0, steps="logU[1e3, 1e4]"))
        # a long request on the GPU while short ones arrive: 32 requests at
        # 4/s, the first an 8192 x 128 job of 1e5 steps
        line["serving_long_tail"] = optional_block(lambda: dict(
            serving_result(T, SV, inputs.serving_requests(32, 4.0, long_tail=1, long_steps=(1e5, 1e5),
                                                          long_grids=((8192, 128),), long_weights=None),
                           slice_steps=640, fill_points=2_000_000, memory_gb=200.0,
                           policies=("async-remaining", "async")),
            rate_per_s=4.0, steps="logU[1e3, 1e4]; first request 8192x128, 1e5 steps"))
        # many small requests at once (overload): 128 requests at 200/s on
        # 256..512 x 16..32 grids, 2e3..8e3 steps each
        small = dict(grids=((256, 16), (256, 32), (512, 16), (512, 32)), grid_weights=(1, 1, 1, 1),
                     step_range=(2e3, 8e3))
        line["serving_small"] = optional_block(lambda: dict(
            serving_result(T, SV, inputs.serving_requests(128, 200.0, **small), slice_steps=640,
                           fill_points=2_000_000, memory_gb=200.0, policies=("fill+multi", "share+multi", "async")),
            rate_per_s=200.0, grids="256..512 x 16..32", steps="logU[2e3, 8e3]"))
    if ws == 1 and not args.no_cpu_baseline:
        def cpu_baseline():
            per = args.cpu_sample_steps
            upd, times = oracle_rate(per, 1)
            return dict(value=upd / times[0], unit=UNIT, cores=cores_used(), kind="oracle",
                        sample="%d time steps of the 8192x128 workload grid, FP64 C oracle "
                               "(OpenMP over r* rows), source and angular dissipation (eps = 1)" % per)
        line["cpu_baseline"] = optional_block(cpu_baseline)
    print(json.dumps(line), flush=True)
    S.close()
    return 0


def optional_block(fn):
    """Run one part of the bench line that follows the measured headline
    (batched and serving blocks, the CPU baseline).  An exception there is
    recorded in the line as {"error": ...} instead of losing the line."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 -- any failure of an optional part
        return {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}


def run_hbm_probe(T, stream, ws, hbm_peak, hbm_src, same_src, chunk=64, reps=6):
    """The same physics on 32768 x 512 (state 2 x 537 MB, planes 2.8 GB per
    time step: far beyond L2): point updates/s and the HBM figures on a grid
    where every time step must stream its whole working set from DRAM."""
    import torch
    from paper_1206_0270_gb300 import inputs
    w = dict(inputs.WORKLOADS[HBM_PROBE])
    nr, nth = w["nr"], w["nth"]
    dt = T.stable_dt(nr, nth, w["rstar_min"], w["rstar_max"], w["a"], w["s"], w["m"], w["c_r"], w["c_theta"])
    P = T.Solver(nr, nth, w["rstar_min"], w["rstar_max"], dt, w["a"], w["s"], w["m"], stream=stream)
    try:
        # smooth random data: every point carries a normal-sized value from the
        # start, as a developed field does (zero data would leave most of this
        # grid at exactly zero for the probe's few hundred steps)
        P.set_initial(*inputs.random_fields(nr, nth, seed=11))
        P.set_source(**w["source"])
        P.set_dissipation(w["eps"])
        ex = w["extraction"]
        P.set_extraction(ex["rstar"], ex["every"], capacity=chunk * (reps + 3) // ex["every"] + 16)
        for _ in range(2):
            P.step(chunk)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            P.step(chunk)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = reduce_max(e0.elapsed_time(e1), "cuda")
        assert P.check_finite(), "state became non-finite"
    finally:
        P.close()
    upd = (nr - 2) * nth * chunk * reps
    rate = upd / (ms / 1e3)
    alg = BYTES_PER_UPDATE_ALG * rate / 1e9
    # DRAM bytes per point update from the 8192 x 128 capture, scaled by the
    # points processed (traffic is proportional to the grid: planes, state and
    # half step are each read or written once per step)
    dram_per_upd = (NCU_TRAFFIC["predictor"] + NCU_TRAFFIC["corrector"]) / (8190 * 128) if same_src else None
    return dict(workload=HBM_PROBE, nr=nr, nth=nth, time_steps=chunk * reps, initial_data="smooth random fields",
                value=whole_job_rate(ws, upd, ms / 1e3), unit=UNIT, peak_gbs=hbm_peak, peak_source=hbm_src,
                algorithmic_gbs=alg, frac_algorithmic=alg / hbm_peak,
                dram_gbs=None if dram_per_upd is None else dram_per_upd * rate / 1e9,
                frac_dram=None if dram_per_upd is None else dram_per_upd * rate / 1e9 / hbm_peak,
                dram_source="ncu bytes per point update on 8192 x 128, scaled to this grid")


# ---------------------------------------------------------------------------
# Batched workloads: waveforms/s batched vs one job at a time
# ---------------------------------------------------------------------------

def batch_jobs(kind, scale):
    """Job list (dicts) of a batched workload, step counts scaled by `scale`."""
    from paper_1206_0270_gb300 import inputs
    jobs = []
    if kind == "batch_modes":
        w = inputs.MODE_BATCH
        for m, nth in w["modes"]:
            jobs.append(dict(a=w["a"], s=w["s"], m=m, nr=w["nr"], nth=nth, r0=w["r0"], sigma=w["sigma"],
                             steps=max(2, int(round(w["steps"] * scale)))))
    elif kind == "small_bank":
        for j in inputs.small_bank(128):
            j = dict(j)
            j["sigma"] = max(0.05, 2.0 * 700.0 / (j["nr"] - 1))
            j["steps"] = max(2, int(round(j["steps"] * scale)))
            jobs.append(j)
    else:
        for j in inputs.template_bank(256):
            j = dict(j)
            # the bank fixes no source width: two radial cells, at least 0.05M
            j["sigma"] = max(0.05, 2.0 * 700.0 / (j["nr"] - 1))
            j["steps"] = max(2, int(round(j["steps"] * scale)))
            jobs.append(j)
    return jobs


def batch_result(T, kind, scale, batch_mode="auto"):
    """Waveforms/s of a batched workload against the same jobs one at a time
    (each job's own graph-replayed steps, jobs in sequence)."""
    import torch
    from paper_1206_0270_gb300 import inputs
    rule = inputs.STEP_RULE
    rmin, rmax, ext = -100.0, 600.0, dict(rstar=500.0, every=10)
    jobs = batch_jobs(kind, scale)
    stream = torch.cuda.Stream()
    dts = {}
    for j in jobs:
        key = (j["nr"], j["nth"], j["a"], j["s"], j["m"])
        if key not in dts:
            dts[key] = T.stable_dt(j["nr"], j["nth"], rmin, rmax, j["a"], j["s"], j["m"], rule["c_r"],
                                   rule["c_theta"])
        j["dt"] = dts[key]

    def make_all(own_streams=False):
        out = []
        for j in jobs:
            g = T.Solver(j["nr"], j["nth"], rmin, rmax, j["dt"], j["a"], j["s"], j["m"],
                         stream=None if own_streams else stream)
            g.set_dissipation(rule["eps"])
            g.set_source(r0=j["r0"], sigma=j["sigma"])
            g.set_extraction(ext["rstar"], ext["every"], capacity=j["steps"] // ext["every"] + 1)
            out.append(g)
        torch.cuda.synchronize()
        return out

    upd = sum((j["nr"] - 2) * j["nth"] * j["steps"] for j in jobs)
    solvers = make_all()
    t0 = time.perf_counter()
    for g, j in zip(solvers, jobs):
        g.step(j["steps"])
        g.extract()
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    launches_single = sum(g.launches_for(j["steps"]) for g, j in zip(solvers, jobs))
    finite = all(g.check_finite() for g in solvers)
    for g in solvers:
        g.close()
    # batched: every job in one batch (each job on its own stream, so that
    # per-job launches can overlap), in each launch form: per-job launches
    # ("1"), multi-job launches with one CTA per tile ("0"), persistent
    # multi-job launches ("p"); or the form the autotuner picks on the jobs
    # themselves ("auto", its timed steps counting as progress)
    forms = {}
    for form in (("1", "0", "p") if batch_mode == "all" else (batch_mode,)):
        solvers = make_all(own_streams=True)
        B = T.Batch(stream=stream)
        for g, j in zip(solvers, jobs):
            B.add(g, j["steps"])
        t0 = time.perf_counter()
        if form == "auto":
            best = B.autotune()
        else:
            best = BATCH_FORM_INDEX[form]
            B.set_option(T.TEUK_OPT_BATCH_CTAS, 8 if form == "p" else 0)
            B.set_option(T.TEUK_OPT_BATCH_MODE, 1 if form == "1" else 0)
        launches = B.launches_for(1)
        B.step(10 ** 9)
        B.sync()
        for g in solvers:
            g.extract()
        t_batch = time.perf_counter() - t0
        B.close()
        finite = finite and all(g.check_finite() for g in solvers)
        for g in solvers:
            g.close()
        forms[T.BATCH_FORMS[best]] = dict(value=len(jobs) / t_batch, unit="waveforms/s", seconds=t_batch,
                                          grid_pt_updates_per_s=upd / t_batch, launches_per_time_step=launches,
                                          speedup=t_single / t_batch)
    name, top = max(forms.items(), key=lambda kv: kv[1]["value"])
    n = len(jobs)
    return dict(workload=kind, jobs=n, step_fraction=scale, point_updates=upd,
                value=top["value"], unit="waveforms/s", seconds=top["seconds"],
                grid_pt_updates_per_s=top["grid_pt_updates_per_s"], batch_mode=name, forms=forms,
                one_by_one=dict(value=n / t_single, unit="waveforms/s", seconds=t_single,
                                gpu_launches=int(launches_single), grid_pt_updates_per_s=upd / t_single),
                speedup=t_single / top["seconds"], finite=finite)


def run_batch_workload(args):
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import teuk as T
    r = batch_result(T, args.workload, args.steps_scale, args.batch_mode)
    line = dict(metric="batched waveforms/s", value=r["value"], unit="waveforms/s", n_gpus=1,
                steps=1, warmup=0, ms_per_step=1e3 * r["seconds"], higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, jobs=r["jobs"], steps_scale=args.steps_scale,
                            point_updates=r["point_updates"], batch_mode=r["batch_mode"]),
                forms=r["forms"],
                one_by_one=r["one_by_one"], batched=dict(seconds=r["seconds"],
                                                         grid_pt_updates_per_s=r["grid_pt_updates_per_s"]),
                speedup=r["speedup"])
    print(json.dumps(line), flush=True)
    return 0


def serving_result(T, S, raw, *, slice_steps, fill_points, memory_gb, policies=("async",), sweep=(), n_requests=None,
                   rate=None):
    """A Poisson stream of requests through the continuous-batching service:
    p50/p99 latency and waveforms/s for each policy, beside the same stream
    served one job at a time in arrival order (same kernels, no batching)."""
    import torch
    from paper_1206_0270_gb300 import inputs

    def request(d):
        sigma = max(0.05, 2.0 * 700.0 / (d["nr"] - 1))
        return S.Request(a=d["a"], s=d["s"], m=d["m"], nr=d["nr"], nth=d["nth"], steps=d["steps"], r0=d["r0"],
                         sigma=sigma, arrival=d["arrival"], **inputs.STEP_RULE)
    reqs = [request(d) for d in raw]
    upd = sum((r.nr - 2) * r.nth * r.steps for r in reqs)
    budget = int(memory_gb * 2 ** 30)

    def served(reqs, policy):
        # "async-remaining": the async policy ranking jobs by remaining work;
        # "share+multi": the share policy with multi-job launches (batch mode 0)
        base, _, multi = policy.partition("+")
        name, _, order = base.partition("-")
        svc = S.WaveformService(memory_budget=budget, slice_steps=slice_steps, policy=name,
                                fill_points=fill_points, order=order or "age",
                                batch_mode=0 if multi == "multi" else None)
        for r in reqs:
            svc.submit(r)
        torch.cuda.synchronize()
        t0 = svc.now()
        res = svc.run()
        out = (svc.now() - t0, S.latency_stats(res), res)
        svc.close()
        return out

    def one_at_a_time(reqs):
        t_start = time.perf_counter()
        lat = []
        for r in reqs:
            now = time.perf_counter() - t_start
            if now < r.arrival:
                time.sleep(r.arrival - now)
            dt = T.stable_dt(r.nr, r.nth, r.rstar_min, r.rstar_max, r.a, r.s, r.m, r.c_r, r.c_theta)
            g = T.Solver(r.nr, r.nth, r.rstar_min, r.rstar_max, dt, r.a, r.s, r.m)
            g.set_dissipation(r.eps)
            g.set_source(r0=r.r0, sigma=r.sigma)
            g.set_extraction(r.rstar_ext, r.every, capacity=r.steps // r.every + 1)
            g.step(r.steps)
            g.extract()
            g.close()
            lat.append(time.perf_counter() - t_start - r.arrival)
        return time.perf_counter() - t_start, np.array(lat)

    def stats(st):
        return dict(p50=st["p50"], p99=st["p99"], mean=st["mean"])

    n = len(reqs)
    per_policy = {policy: served(reqs, policy) for policy in policies}
    wall1, lat1 = one_at_a_time(reqs)
    lat_1 = dict(p50=float(np.percentile(lat1, 50)), p99=float(np.percentile(lat1, 99)), mean=float(lat1.mean()))
    out = dict(requests=n, point_updates=upd, slice_steps=slice_steps, fill_points=fill_points,
               memory_budget_gb=memory_gb,
               policies={p: dict(value=n / w, unit="waveforms/s", latency_s=stats(st), grid_pt_updates_per_s=upd / w)
                         for p, (w, st, _) in per_policy.items()},
               one_by_one=dict(value=n / wall1, unit="waveforms/s", latency_s=lat_1))
    # latency by request size: the short jobs' tail beside the long ones
    first = per_policy[policies[0]][2]
    short = [x for x in first.values() if x.request.steps * x.request.nr * x.request.nth < np.median(
        [r.steps * r.nr * r.nth for r in reqs])]
    if short:
        ls = np.array([x.latency for x in short])
        ids = [x.rid for x in short]
        l1s = lat1[ids]
        out["short_half"] = dict(policy=policies[0], p50=float(np.percentile(ls, 50)), p99=float(np.percentile(ls, 99)),
                                 one_by_one_p50=float(np.percentile(l1s, 50)),
                                 one_by_one_p99=float(np.percentile(l1s, 99)))
    if sweep:
        rows = []
        for mult in sweep:
            r8 = mult * n / wall1
            rq = [request(d) for d in inputs.serving_requests(n_requests, r8)]
            w_f, st_f, _ = served(rq, "fill")
            w_a, st_a, _ = served(rq, "async")
            w_1, l_1 = one_at_a_time(rq)
            rows.append(dict(rate_per_s=r8, load=mult,
                             fill=dict(value=n / w_f, **stats(st_f)), async_policy=dict(value=n / w_a, **stats(st_a)),
                             one_by_one=dict(value=n / w_1, p50=float(np.percentile(l_1, 50)),
                                             p99=float(np.percentile(l_1, 99)), mean=float(l_1.mean()))))
        out["rate_sweep"] = rows
    return out


def run_serving(args):
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import inputs, serve as S
    from paper_1206_0270_gb300 import teuk as T
    long_steps = tuple(float(x) for x in args.long_steps.split(","))
    long_grids = tuple(tuple(int(v) for v in g.split("x")) for g in args.long_grids.split(","))
    raw = inputs.serving_requests(args.requests, args.rate, long_tail=args.long_tail, long_steps=long_steps,
                                  long_grids=long_grids, long_weights=None)
    sweep = [float(x) for x in args.rate_sweep.split(",") if x.strip()]
    policies = tuple(x for x in args.policies.split(",") if x)
    r = serving_result(T, S, raw, slice_steps=args.slice, fill_points=args.fill_points, memory_gb=args.memory_gb,
                       policies=policies, sweep=sweep, n_requests=args.requests, rate=args.rate)
    pol = policies[0]
    a = r["policies"][pol]
    line = dict(metric="served waveforms/s", value=a["value"], unit="waveforms/s", n_gpus=1, steps=1, warmup=0,
                ms_per_step=1e3 * r["requests"] / a["value"], higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload="serving", requests=r["requests"], rate_per_s=args.rate,
                            slice_steps=args.slice, fill_points=args.fill_points, memory_budget_gb=args.memory_gb,
                            point_updates=r["point_updates"], grids="2048x64..32768x512",
                            steps="logU[1e3, 1e4]", long_tail=args.long_tail,
                            long_steps=args.long_steps if args.long_tail else None,
                            long_grids=args.long_grids if args.long_tail else None),
                policy=pol, latency_s=a["latency_s"], grid_pt_updates_per_s=a["grid_pt_updates_per_s"],
                policies=r["policies"], one_by_one=r["one_by_one"], short_half=r.get("short_half"),
                rate_sweep=r.get("rate_sweep"))
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 157 benchmark steps of 640 time steps after 3 warm-up ones: the timed
    # region covers the Kerr workload's whole run (steps 1920..102400 of its
    # 1e5), from the first outgoing burst to a field that fills the grid
    ap.add_argument("--steps", type=int, default=157)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=640, help="time steps per benchmark step")
    ap.add_argument("--pre-steps", type=int, default=0,
                    help="untimed time steps before the warm-up (to profile a developed field)")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--ref-steps", type=int, default=100,
                    help="oracle time steps per reference step (~0.2 s of host work each)")
    ap.add_argument("--cpu-sample-steps", type=int, default=4000,
                    help="oracle time steps of the cpu_baseline sample (~10 s of host work)")
    ap.add_argument("--kernel-timing-steps", type=int, default=64,
                    help="steps timed kernel by kernel (after the timed region) for the roofline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-hbm-probe", dest="hbm_probe", action="store_false",
                    help="skip the 32768 x 512 HBM-roof probe")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch_modes", "template_bank", "small_bank", "serving"],
                    help="single: the Kerr 8192x128 step (default); batch_modes / template_bank: batched "
                         "waveforms/s against one job at a time")
    ap.add_argument("--steps-scale", type=float, default=0.2,
                    help="batched workloads: fraction of each job's step count that is run")
    ap.add_argument("--batch-mode", default="all", choices=["all", "auto", "0", "1", "p"],
                    help="batch workloads: launch form (1 per-job launches, 0 multi-job launches with one CTA "
                         "per tile, p persistent multi-job launches, auto the autotuner's pick; all: each of "
                         "1, 0, p, the best reported)")
    ap.add_argument("--requests", type=int, default=64, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=4.0, help="serving: Poisson arrival rate (1/s)")
    ap.add_argument("--slice", type=int, default=640, help="serving: time steps per batch slice")
    ap.add_argument("--fill-points", type=int, default=2_000_000,
                    help="serving: grid points the fill/priority/async policies keep running")
    ap.add_argument("--rate-sweep", default="0.5,1,2",
                    help="serving: arrival rates to sweep, as multiples of the measured one-at-a-time capacity "
                         "('' to skip)")
    ap.add_argument("--memory-gb", type=float, default=200.0, help="serving: device memory budget (GiB)")
    ap.add_argument("--long-tail", type=int, default=0,
                    help="serving: number of long requests in the stream (the earliest arrivals)")
    ap.add_argument("--long-steps", default="1e5,1e6", help="serving: step range of the long requests (logU)")
    ap.add_argument("--long-grids", default="32768x512,8192x128,16384x256",
                    help="serving: grids of the long requests, taken in turn")
    ap.add_argument("--policies", default="async,async-remaining,fill,share,priority",
                    help="serving: scheduling policies to run (the first is the line's value)")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the batched and serving blocks of the default run")
    args = ap.parse_args()
    if args.workload == "serving":
        return run_serving(args)
    if args.workload != "single":
        return run_batch_workload(args)
    if args.warmup < 3 and args.impl == "gpu":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
