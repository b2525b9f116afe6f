"""Benchmark: seeded random circuits on B300, gates/s and achieved HBM GB/s.

Default workload (one "step"): a 30-qubit complex128 state vector (16 GiB),
|0...0> initialisation, the 1259-gate depth-40 random circuit (H, CZ,
sqrt(X), sqrt(Y), T, Haar compactUnitary, 3-control phase flip per layer),
then calcTotalProb and calcProbOfOutcome(qubit 0) returned to the host.
value = gates/s of the whole job (sum over ranks).  The state (16 GiB) is
far larger than L2 (126 MB), so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec 128|64] [--arith fp64|df] [--qubits n] [--no-variants]

Multi-GPU: replicas only (every rank simulates its own register; no data
exchange), launched by torchrun; the time is the max over ranks.
--impl reference times the CPU oracle on the host cores instead (bounded
sample of the same workload).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1802_08032_b300 import circuits as C  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6400.0
FP64_NOMINAL_TFLOPS = 1.25   # B300 dense FP64 (non-tensor), nominal
FP32_NOMINAL_TFLOPS = 75.0   # B300 FP32: 148 SMs x 128 lanes x 2 x ~2.0 GHz
FP32_ISSUE_TINSTR = 148 * 128 * 2.032e9 / 1e12   # FP32 instructions/s at the 2032 MHz max clock
# DRAM bytes (read + write) per amplitude per launch, from one ncu capture of
# the kernel as built (profiles/<kernel>_*_ncu_full.md); scaled by the
# amplitudes a launch processes.  Entries are removed when a kernel changes.
MEASURED_TRAFFIC_PER_AMP = {
    "fused_c128": 2.089e9 / (1 << 26),      # profiles/fused_c128_fp64_sv26_ncu_full.md
    # generated complex64 pass kernel, async-copy pipeline
    "fused_c64": 1.014e9 / (1 << 26),       # profiles/qs_pass_c64_async_sv26_ncu_full.md
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", type=int, default=128, choices=[64, 128])
    ap.add_argument("--arith", default="fp64", choices=["fp64", "df"],
                    help="complex128 arithmetic of fused passes")
    ap.add_argument("--qubits", type=int, default=30)
    ap.add_argument("--serve-requests", type=int, default=60,
                    help="serving variant: requests per arrival rate (at most)")
    ap.add_argument("--serve-seconds", type=float, default=0.0,
                    help="serving variant: also cap each rate's trace at this many seconds of arrivals "
                         "(0 = no cap); 2000 and 60 give the full-length sweep")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg (profiling runs)")
    ap.add_argument("--jit-copy", type=int, default=None, choices=[0, 1, 2],
                    help="generated pass kernels move tiles by coalesced loads (0), bulk (TMA) copies "
                         "double-buffered (1) or async copies double-buffered (2)")
    ap.add_argument("--jit-ctas", type=int, default=None, help="resident CTAs per SM of generated kernels")
    ap.add_argument("--jit-direct", type=int, default=None, choices=[0, 1],
                    help="the last stage of a generated pass stores straight to HBM")
    ap.add_argument("--jit-swizzle", type=int, default=None, choices=[0, 1],
                    help="generated kernels swizzle the tile in shared memory")
    ap.add_argument("--tile-qubits", type=int, default=None, help="fused tile size k (0 = automatic)")
    ap.add_argument("--tile-low", type=int, default=None,
                    help="lowest qubits every fused tile holds (0 = automatic: 4 complex64, 3 complex128)")
    ap.add_argument("--jit", type=int, default=1, choices=[0, 1, 2],
                    help="fused passes: 0 interpreting kernel, 1 runtime-compiled kernels "
                         "(compiled in the warm-up), 2 compiled in the background")
    ap.add_argument("--variants", default="",
                    help="comma-separated variant names to run (default: all)")
    ap.add_argument("--cpu-gates", type=int, default=40,
                    help="gates in the bounded CPU-oracle sample")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def cpu_model():
    """The host CPU's model name and logical CPU count."""
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"model": model, "nproc": os.cpu_count()}


def cpu_oracle_sample(n, ops, ngates, one_core_gates=0):
    """Times the CPU oracle on a bounded sample: `ngates` gates spread evenly
    over the circuit, applied to an n-qubit state (allocation and |0>
    excluded from the timing, as in the paper's methodology); with
    one_core_gates > 0 also the first that many of the sample on one host
    thread."""
    from oracle import oracle as O
    stride = max(1, len(ops) // ngates)
    sample = ops[::stride][:ngates]
    st, secs = O.timed_run(n, sample)
    del st
    out = {"value": len(sample) / secs, "unit": "gates/s", "cores": O.num_threads(),
           "kind": "oracle", "cpu": cpu_model(),
           "sample": f"{len(sample)} gates (every {stride}th of the {len(ops)}-gate circuit) on a "
                     f"{n}-qubit complex128 state vector, FP64 C oracle, OpenMP over "
                     f"{O.num_threads()} host threads, {secs:.1f} s"}
    if one_core_gates > 0:
        full = O.num_threads()
        O.set_num_threads(1)
        try:
            st, secs1 = O.timed_run(n, sample[:one_core_gates])
            del st
        finally:
            O.set_num_threads(full)
        out["one_core"] = {"value": one_core_gates / secs1, "unit": "gates/s", "cores": 1,
                           "sample": f"the first {one_core_gates} gates of the same sample, {secs1:.1f} s"}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = args.qubits
    ops = C.workload_30q(n)
    vals = []
    for _ in range(args.warmup + args.steps):
        r = cpu_oracle_sample(n, ops, args.cpu_gates)
        vals.append(r["value"])
    timed = vals[args.warmup:]
    v = len(timed) / sum(1.0 / x for x in timed)
    line = {"metric": "gates/s (30q random circuit)", "value": v, "unit": "gates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * args.cpu_gates / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{n}-qubit complex128 state vector, seeded depth-40 random "
                                   "circuit (bounded CPU sample)", "qubits": n},
            "cpu_baseline": {"value": v, "unit": "gates/s", "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"], "cpu": r["cpu"]},
            "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "thread_scaling": oracle_thread_scaling(n - 4, C.workload_30q(n - 4), args.cpu_gates)}
    print(json.dumps(line), flush=True)


def oracle_thread_scaling(n, ops, ngates):
    """CPU-side context in the manner of the paper's thread-scaling figure
    (Sec. III): the same bounded gate sample on an n-qubit state with 1, 2,
    4, ... host threads up to all of them; gates/s and speed-up over one
    thread."""
    from oracle import oracle as O
    full = O.num_threads()
    counts = sorted({t for t in (1, 2, 4, 8, 16, 32, 64, 128) if t < full} | {full})
    rows = []
    try:
        for t in counts:
            O.set_num_threads(t)
            rows.append({"threads": t, "gates_per_s": cpu_oracle_sample(n, ops, ngates)["value"]})
    finally:
        O.set_num_threads(full)
    for r in rows:
        r["speedup"] = r["gates_per_s"] / rows[0]["gates_per_s"]
    return {"qubits": n, "gates": ngates, "rows": rows}


def job_max(x, world, device):
    """Largest value of x over the ranks of the job (the job's time is its
    slowest rank's)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def job_throughput(units_per_rank, world, seconds_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (replicas: every rank runs the same workload)."""
    return units_per_rank * world / seconds_max


def roofline(stats, amps_per_launch=None):
    """Roofline of the kernel class with the most time: HBM bytes per second
    against the measured copy bandwidth, and arithmetic instructions per
    second against the issue peak of its precision; the larger fraction
    names the bound."""
    hbm_peak, peak_src = peaks()
    dom = max(stats, key=lambda s: s["total_ms"]) if stats else None
    if not dom or dom["total_ms"] <= 0:
        return None
    per_launch_ms = dom["total_ms"] / dom["launches"]
    secs = per_launch_ms / 1e3
    gbs = dom["bytes"] / dom["launches"] / secs / 1e9
    fp64 = dom["name"].endswith("c128")
    if dom.get("alu_ops"):
        alu = dom["alu_ops"] / dom["launches"] / secs / 1e12
        alu_peak = FP64_NOMINAL_TFLOPS / 2 if fp64 else FP32_ISSUE_TINSTR
        alu_unit = "T FP64 instr/s" if fp64 else "T FP32 instr/s"
        alu_src = ("nominal B300 FP64 1.25 TFLOP/s = 0.625 T instructions/s (FMA = 1)" if fp64 else
                   "148 SMs x 128 FP32 lanes x 2.032 GHz = 38.5 T instructions/s")
    else:
        alu = dom["flops"] / dom["launches"] / secs / 1e12
        alu_peak = FP64_NOMINAL_TFLOPS if fp64 else FP32_NOMINAL_TFLOPS
        alu_unit = "TFLOP/s"
        alu_src = "nominal B300 FP64 1.25 TFLOP/s" if fp64 else "nominal B300 FP32 75 TFLOP/s"
    if gbs / hbm_peak >= alu / alu_peak:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak, "traffic": None,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                "alu_achieved": alu, "alu_unit": alu_unit, "alu_frac": alu / alu_peak}
    else:
        roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": alu_unit,
                "frac": alu / alu_peak, "traffic": None, "peak_source": alu_src,
                "hbm_gbs": gbs, "hbm_frac": gbs / hbm_peak}
    per_amp = MEASURED_TRAFFIC_PER_AMP.get(dom["name"])
    if per_amp is not None and amps_per_launch:
        roof["traffic"] = per_amp * amps_per_launch
        roof["traffic_source"] = "ncu dram bytes of a 26-qubit capture, scaled by amplitudes"
    roof.update({"kernel": dom["name"], "launch_ms": per_launch_ms,
                 "bytes_per_launch": dom["bytes"] / dom["launches"],
                 "flops_per_launch": dom["flops"] / dom["launches"],
                 "alu_ops_per_launch": dom.get("alu_ops", 0) / dom["launches"]})
    return roof


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_1802_08032_b300 import qsim as Q

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return job_max(x, world, "cuda")

    n, prec = args.qubits, args.prec
    ops = C.workload_30q(n)
    ngates = len(ops)
    env = Q.createQuESTEnv()
    Q.setEnvOption(env, "arith", 1 if args.arith == "df" else 0)
    # fused passes as runtime-compiled kernels, compiled during the warm-up
    # (the first step waits for them; timed steps reuse the cached kernels)
    Q.setEnvOption(env, "jit", args.jit)
    for opt, val in (("jit_copy", args.jit_copy), ("jit_ctas", args.jit_ctas), ("tile_qubits", args.tile_qubits),
                     ("tile_low_qubits", args.tile_low),
                     ("jit_direct", args.jit_direct), ("jit_swizzle", args.jit_swizzle)):
        if val is not None:
            Q.setEnvOption(env, opt, val)
    stream = torch.cuda.Stream()
    Q.setStream(env, stream)
    q = Q.createQureg(n, prec, env)
    # the gate list lives in pinned host memory (the step's host input)
    arr, nops = Q.to_qsops(ops)
    raw = bytes(arr)
    pinned = torch.empty(len(raw), dtype=torch.uint8, pin_memory=True)
    ctypes.memmove(pinned.data_ptr(), raw, len(raw))
    qsops = (ctypes.cast(pinned.data_ptr(), ctypes.POINTER(Q.QSOp)), nops)
    h2d, d2h = len(raw), 2 * 8

    def step():
        Q.initZeroState(q)
        Q.applyCircuit(q, qsops)
        return Q.calcTotalProb(q), Q.calcProbOfOutcome(q, 0, 0)

    for _ in range(args.warmup):
        step()
    Q.resetKernelStats(env)
    Q.setEnvOption(env, "profile", 1)
    l0 = Q.getEnvOption(env, "launches")
    p0 = Q.getEnvOption(env, "fused_passes")
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    dev_ms = max_over_ranks(e0.elapsed_time(e1))
    launches = Q.getEnvOption(env, "launches") - l0
    passes = (Q.getEnvOption(env, "fused_passes") - p0) / args.steps
    stats = Q.getKernelStats(env)
    Q.setEnvOption(env, "profile", 0)

    # e2e: host wall clock around the same public-API step (gate list in from
    # pinned host memory, probabilities out), no profiling events
    step()
    barrier()
    te = time.perf_counter()
    for _ in range(args.steps):
        step()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - te)

    total_gates = ngates * args.steps * world  # = job_throughput(...) x time
    # double-float is an out-of-spec precision form (48-bit significands),
    # never reported as complex128 arithmetic
    dtype = "f32" if prec == 64 else ("df64 (f32 pairs, out of spec)" if args.arith == "df" else "f64")
    line = {
        "metric": "gates/s (30q random circuit)", "value": total_gates / (dev_ms / 1e3),
        "unit": "gates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": f"{n}-qubit complex{prec} state vector, seeded depth-40 random "
                               f"circuit ({ngates} gates) + calcTotalProb + calcProbOfOutcome",
                   "qubits": n, "precision": f"complex{prec}", "arith": args.arith,
                   "gates_per_step": ngates, "parallelism": f"replicas x{world}",
                   "l2": "state 2^n amplitudes >> 126 MB L2, no flush",
                   "fused_passes_per_step": passes,
                   "tile_qubits": Q.getEnvOption(env, "tile_qubits"),
                   "jit": {"mode": args.jit, "kernels": Q.getEnvOption(env, "jit_ready"),
                           "tile_copy": ["coalesced loads", "bulk (TMA) copies, double-buffered",
                                         "async copies, double-buffered"][Q.getEnvOption(env, "jit_copy")],
                           "ctas_per_sm": Q.getEnvOption(env, "jit_ctas"),
                           "compile_ms_total": Q.getEnvOption(env, "jit_compile_ms"),
                           "launches": Q.getEnvOption(env, "jit_launches")}},
        "roofline": roofline(stats, 1 << n),
        "e2e": {"value": total_gates / e2e_s, "unit": "gates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "result": {"total_prob": res[0], "prob_q0_0": res[1]},
        "kernels": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in s.items()}
                    for s in sorted(stats, key=lambda s: -s["total_ms"])[:6]],
    }
    Q.destroyQureg(q)
    if rank == 0 and world == 1 and not args.no_variants:
        line["variants"] = variants(Q, env, torch, stream,
                                    [v for v in args.variants.split(",") if v], n,
                                    (args.serve_requests, args.serve_seconds))
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            line["cpu_baseline"] = cpu_oracle_sample(n, ops, args.cpu_gates, one_core_gates=6)
        except Exception as e:  # host without room for the sample
            line["cpu_baseline"] = {"value": None, "unavailable": str(e)}
    Q.destroyQuESTEnv(env)
    if "variants" in line:
        # last key of the line: the figures stay in view when only the end
        # of the output is kept
        line["summary"] = compact_summary(line["variants"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


class _DeviceAmps:
    """__cuda_array_interface__ over a register's device amplitudes (as
    interleaved reals), so that torch can read them for error reports."""

    def __init__(self, ptr, count, prec):
        self.__cuda_array_interface__ = {
            "shape": (2 * count,), "typestr": "<f8" if prec == 128 else "<f4",
            "data": (ptr, False), "version": 3, "strides": None}


def reg_view(Q, torch, q):
    info = Q.getQuregInfo(q)
    prec = info["precision"]
    count = 1 << (info["numQubits"] * (2 if info["isDensity"] else 1))
    t = torch.as_tensor(_DeviceAmps(info["devicePtr"], count, prec), device="cuda")
    return torch.view_as_complex(t.view(-1, 2))


def c64_error(Q, torch, q64, q128, chunk=1 << 27):
    """Error of a complex64 register against the complex128 register of the
    same circuit run with IEEE FP64 arithmetic (which the parity tests hold
    to the FP64 oracle at 1e-12): max |a64 - a128| over every amplitude,
    raw overlap |<a128|a64>|^2, fidelity of the normalised states
    |<a128|a64>|^2 / (<a128|a128> <a64|a64>) and the complex64 norm drift,
    all reduced in FP64."""
    ip = Q.calcInnerProduct(q128, q64)
    n128, n64 = Q.calcTotalProb(q128), Q.calcTotalProb(q64)
    a, b = reg_view(Q, torch, q128), reg_view(Q, torch, q64)
    worst = 0.0
    for i in range(0, a.numel(), chunk):
        d = (a[i:i + chunk] - b[i:i + chunk].to(torch.complex128)).abs().max().item()
        worst = max(worst, d)
    raw = abs(ip) ** 2
    fid = raw / (n128 * n64)
    return {"max_abs_err": worst, "fidelity": fid, "one_minus_fidelity": 1.0 - fid,
            "raw_overlap": raw, "one_minus_raw_overlap": 1.0 - raw, "norm_dev": abs(n64 - 1.0)}


def golden_sample_error(Q, q, name="sv30_depth40.json"):
    """max |a - a_oracle| over the sampled amplitudes the FP64 oracle wrote
    for this workload (tests/golden), and the largest outcome-probability
    difference; None when the file is absent."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        g = json.load(f)
    worst = 0.0
    for i, (re, im) in zip(g["indices"], g["amps"]):
        worst = max(worst, abs(Q.copyStateToHost(q, int(i), 1)[0] - complex(re, im)))
    pw = max(abs(Q.calcProbOfOutcome(q, k, 1) - p) for k, p in enumerate(g["prob_outcome_1"]))
    return {"max_abs_err_vs_fp64_oracle": worst, "amplitudes": len(g["indices"]),
            "max_prob_err_vs_fp64_oracle": pw, "total_prob_err": abs(Q.calcTotalProb(q) - g["total_prob"])}


def timed(torch, stream, fn, reps):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def pass_kernel_roofline(Q, env, run):
    """One more run with per-kernel CUDA events: the fused pass kernels'
    algorithmic bytes (one read and one write of the register per pass) over
    their summed kernel time, against the measured HBM copy bandwidth."""
    Q.resetKernelStats(env)
    Q.setEnvOption(env, "profile", 1)
    try:
        run()
    finally:
        Q.setEnvOption(env, "profile", 0)
    ks = [k for k in Q.getKernelStats(env) if k["name"].startswith(("fused", "jit", "qs_pass", "sv_fused"))]
    ms = sum(k["total_ms"] for k in ks)
    if ms <= 0:
        return {}
    gbs = sum(k["bytes"] for k in ks) / ms / 1e6
    return {"pass_kernel_ms": ms, "pass_kernel_launches": sum(k["launches"] for k in ks),
            "pass_kernel_GBps": gbs, "pass_kernel_hbm_frac_of_measured": gbs / peaks()[0]}


def compact_summary(v):
    """The variants' headline figures in a few hundred characters (the
    full detail is under "variants"), rounded, in the units of their
    sources: gates/s, circuits/s, GB/s, ms, us."""
    import statistics
    out = {}

    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r(x, nd=3):
        return None if x is None else float(f"{x:.{nd}g}")

    if "sv12_c128" in v:
        out["sv12_us"] = r(g(v, "sv12_c128", "us_per_circuit"))
    for name in ("sv30_c64", "sv33_c128", "sv33_c64", "sv30_df64_out_of_spec"):
        if name in v:
            out[name] = [r(g(v, name, "gates_per_s")), r(g(v, name, "pass_kernel_hbm_frac_of_measured"), 2),
                         r(g(v, name, "error_vs_fp64", "max_abs_err"), 2),
                         r(g(v, name, "error_vs_fp64", "one_minus_fidelity"), 2)]
    if "dm14_c128" in v:
        out["dm14_ops_s"] = r(g(v, "dm14_c128", "ops_per_s"))
    for name, key in (("single_gate_sweep", "sweep30"), ("single_gate_sweep_33q", "sweep33")):
        sw = v.get(name)
        if isinstance(sw, dict) and "targets" in sw:
            row = {}
            for kind in ("H", "U", "T", "CZ", "MCPF"):
                for prec in (64, 128):
                    vals = sw.get(f"{kind}_c{prec}_GBps_by_target")
                    if vals:
                        hi = vals[5:-3] or vals   # bits the sector rule does not touch
                        row[f"{kind}{prec}"] = [round(min(hi)), round(statistics.median(hi))]
            out[key + "_bits5up_min_med_GBps"] = row
    b = v.get("batch4096_c64")
    if isinstance(b, dict) and "circuits_per_s" in b:
        out["batch"] = {"c_s": r(b["circuits_per_s"]), "plain_c128_c_s": r(b.get("plain_c128_circuits_per_s")),
                        "k": b.get("tile_qubits"), "sched": "persist" if "persist" in str(b.get("schedule")) else "waves",
                        "err": r(g(b, "error_vs_fp64_all_registers", "max_abs_err"), 2),
                        "1-F": r(g(b, "error_vs_fp64_all_registers", "max_one_minus_fidelity"), 2)}
    m = v.get("multi_target_passes")
    if isinstance(m, dict):
        out["multi_GBps"] = {k: round(x["GBps"]) for k, x in m.items()
                             if isinstance(x, dict) and "GBps" in x and k in (
                                 "c64_m4", "c64_m5", "c64_m5_low_targets_tensor_cores",
                                 "c64_m4_low_targets", "c128_m2")}
    sv = v.get("serving")
    if isinstance(sv, dict):
        rows = {}
        for rate, d in sv.items():
            if isinstance(d, dict) and "served" in d:
                rows[rate.split("_")[0]] = [r(g(d, "served", "circuits_per_s")), r(g(d, "served", "p50_ms")),
                                            r(g(d, "served", "p99_ms")),
                                            r(g(d, "served_shed_after_1s", "p99_ms")),
                                            r(g(d, "plain_c128_one_at_a_time", "circuits_per_s"))]
        out["serve_c_s_p50ms_p99ms_p99shedms_plainc128"] = rows
    p = v.get("partitioned_28q_4parts")
    if isinstance(p, dict) and "gates_per_s" in p:
        out["part28_4_gates_s"] = r(p["gates_per_s"])
    return out


def variants(Q, env, torch, stream, only=(), qubits=30, serve=(60, 0.0)):
    """Other configurations of the same metric, measured outside the timed
    region: the 12-qubit circuit (latency), complex64 and double-float
    complex128 at 30 qubits, the 33-qubit
    (128 GiB complex128, 64 GiB complex64) depth-40 circuits, the 14-qubit
    noisy density matrix, single-gate pass bandwidth by target bit, batches,
    serving and multi-target passes (on a register of `qubits` qubits, the
    headline's size)."""
    out = {}
    ops = C.workload_30q(30)

    def sv(prec, arith, n=30, reps=2, ref=None):
        """One circuit variant; with ref (a complex128 register holding the
        same circuit's IEEE-FP64 result) a complex64 run also states its
        error and fidelity against it."""
        def run_variant():
            circ = ops if n == 30 else C.workload_30q(n)
            Q.setEnvOption(env, "arith", arith)
            q = Q.createQureg(n, prec, env)

            def run():
                Q.initZeroState(q)
                Q.applyCircuit(q, circ)
                Q.calcTotalProb(q)

            try:
                ms = timed(torch, stream, run, reps)
                res = {"qubits": n, "gates": len(circ), "gates_per_s": len(circ) / ms * 1e3,
                       "ms_per_circuit": ms}
                res.update(pass_kernel_roofline(Q, env, run))
                if prec == 64 and ref is not None and ref.get("q") is not None:
                    res["error_vs_fp64"] = c64_error(Q, torch, q, ref["q"])
                if n == 30:
                    g = golden_sample_error(Q, q)
                    if g is not None:
                        res["error_vs_fp64_oracle_sample"] = g
            finally:
                Q.destroyQureg(q)
                Q.setEnvOption(env, "arith", 0)
            if arith == 1:
                res["precision"] = ("double-float (float pairs, 48-bit significands): an out-of-spec "
                                    "form, not complex128 arithmetic; complex128 storage")
            return res
        return run_variant

    def fp64_reference(n, keep):
        """Runs the n-qubit workload in complex128 (IEEE FP64) and keeps the
        register in keep["q"] as the reference of the complex64 variant; with
        n = 33 the run is timed as the sv33_c128 variant."""
        def run_variant():
            circ = ops if n == 30 else C.workload_30q(n)
            q = Q.createQureg(n, 128, env)
            keep["q"] = q

            def run():
                Q.initZeroState(q)
                Q.applyCircuit(q, circ)
                Q.calcTotalProb(q)

            ms = timed(torch, stream, run, 1)
            return {"qubits": n, "gates": len(circ), "gates_per_s": len(circ) / ms * 1e3,
                    "ms_per_circuit": ms}
        return run_variant

    def release(keep):
        def run_variant():
            if keep.get("q") is not None:
                Q.destroyQureg(keep.pop("q"))
            return None
        return run_variant

    ref30, ref33 = {}, {}

    def sweep(n, targets):
        # single-gate passes (fusion off) on an n-qubit register, GB/s by
        # target bit.  "GBps" counts the algorithmic bytes (touched amplitudes
        # read + written); "sector" counts the least DRAM traffic at 32-byte
        # sector granularity (a sector is moved when any of its amplitudes is
        # touched), which is the whole vector for diagonal ops on the lowest
        # bits.  U is compactUnitary with fixed Haar-random (alpha, beta);
        # MCPF flips the sign where qubits t, t+1, t+2 are all 1.
        Q.setEnvOption(env, "fusion", 0)
        ab = C.haar_alpha_beta(C.SplitMix64(33))
        res = {}
        try:
            for prec in (64, 128):
                reg = Q.createQureg(n, prec, env)
                S = 16 if prec == 128 else 8
                lg = (32 // S).bit_length() - 1   # amplitude-index bits inside a sector
                kinds = (
                    ("H", lambda t: Q.hadamard(reg, t), lambda t: 0),
                    ("U", lambda t: Q.compactUnitary(reg, t, complex(ab[0], ab[1]),
                                                     complex(ab[2], ab[3])), lambda t: 0),
                    ("T", lambda t: Q.tGate(reg, t), lambda t: 1 << t),
                    ("CZ", lambda t: Q.controlledPhaseFlip(reg, t, (t + 1) % n),
                     lambda t: (1 << t) | (1 << ((t + 1) % n))),
                    ("MCPF", lambda t: Q.multiControlledPhaseFlip(reg, [t, (t + 1) % n, (t + 2) % n]),
                     lambda t: (1 << t) | (1 << ((t + 1) % n)) | (1 << ((t + 2) % n))))
                try:
                    for name, fn, cond in kinds:
                        row, srow = [], []
                        for t in targets:
                            ms = timed(torch, stream, lambda: fn(t), 2)
                            c = cond(t)
                            frac = 2.0 ** -bin(c).count("1")
                            sfrac = 2.0 ** -bin(c >> lg).count("1")
                            row.append(round(2 * frac * (1 << n) * S / ms / 1e6, 1))
                            srow.append(round(2 * sfrac * (1 << n) * S / ms / 1e6, 1))
                        res[f"{name}_c{prec}_GBps_by_target"] = row
                        if cond(1) != 0:
                            res[f"{name}_c{prec}_sector_GBps_by_target"] = srow
                finally:
                    Q.destroyQureg(reg)
        finally:
            Q.setEnvOption(env, "fusion", 1)
        res["targets"] = list(targets)
        return res

    def dm14():
        dops = C.workload_dm14()
        d = Q.createDensityQureg(14, 128, env)

        def run():
            Q.initZeroState(d)
            Q.applyCircuit(d, dops)
            Q.calcTotalProb(d)
            Q.calcPurity(d)

        try:
            ms = timed(torch, stream, run, 2)
        finally:
            Q.destroyQureg(d)
        return {"ops_per_s": len(dops) / ms * 1e3, "ms_per_circuit": ms, "ops": len(dops)}

    def sv12(reps=300, tiles=(0, 9, 10)):
        # the 12-qubit complex128 depth-20 circuit (64 KiB: one fused tile,
        # spread over a cluster of 8 CTAs): latency-bound, so whole circuits
        # are timed on the host clock, each reset, planned, run and reduced
        # (calcTotalProb reads its result)
        import time
        ops12 = Q.to_qsops(C.workload_12q())
        q = Q.createQureg(12, 128, env)
        try:
            def run():
                Q.initZeroState(q)
                Q.applyCircuit(q, ops12)
                return Q.calcTotalProb(q)
            by_tile = {}
            for k in tiles:   # tile size: 0 = the planner's choice
                Q.setEnvOption(env, "tile_qubits", k)
                for _ in range(10):
                    run()
                t0 = time.perf_counter()
                for _ in range(reps):
                    run()
                by_tile[k] = (time.perf_counter() - t0) / reps * 1e6
            Q.setEnvOption(env, "tile_qubits", 0)
            us = by_tile[0]
            # without thread-block clusters (two tiles of 2^11 on two CTAs)
            Q.setEnvOption(env, "fused_cluster", 0)
            try:
                for _ in range(10):
                    run()
                t0 = time.perf_counter()
                for _ in range(reps):
                    run()
                us_one_cta = (time.perf_counter() - t0) / reps * 1e6
            finally:
                Q.setEnvOption(env, "fused_cluster", 8)
            # the same with generated pass kernels (compiled in the first
            # run; the 12-qubit passes run on 2 SMs, latency- not FP64-bound)
            saved = {o: Q.getEnvOption(env, o) for o in ("jit", "jit_fp64", "jit_min_qubits", "fused_cluster")}
            for opt, val in (("jit", 1), ("jit_fp64", 1), ("jit_min_qubits", 1), ("fused_cluster", 0)):
                Q.setEnvOption(env, opt, val)
            try:
                for _ in range(10):
                    run()
                t0 = time.perf_counter()
                for _ in range(reps):
                    run()
                us_jit = (time.perf_counter() - t0) / reps * 1e6
            finally:
                for opt, val in saved.items():
                    Q.setEnvOption(env, opt, val)
            # where the time goes: kernel time per circuit (CUDA events)
            Q.resetKernelStats(env)
            Q.setEnvOption(env, "profile", 1)
            for _ in range(20):
                run()
            Q.setEnvOption(env, "profile", 0)
            kstats = Q.getKernelStats(env)
        finally:
            Q.destroyQureg(q)
        gpu_us = sum(k["total_ms"] for k in kstats) * 1e3 / 20
        return {"qubits": 12, "gates": ops12[1], "us_per_circuit": us,
                "gates_per_s": ops12[1] / us * 1e6, "circuits_per_s": 1e6 / us,
                "kernel_us_per_circuit": gpu_us,
                "us_per_circuit_by_tile_qubits": {str(k): round(v, 1) for k, v in by_tile.items()},
                "us_per_circuit_one_cta": us_one_cta,
                "us_per_circuit_generated_kernels": us_jit,
                "kernels": {k["name"]: round(k["total_ms"] * 1e3 / 20, 2) for k in kstats}}

    for name, fn in (("sv12_c128", sv12), ("_ref30", fp64_reference(30, ref30)),
                     ("sv30_c64", sv(64, 0, ref=ref30)), ("_rel30", release(ref30)),
                     ("sv30_df64_out_of_spec", sv(128, 1)),
                     ("sv33_c128", fp64_reference(33, ref33)), ("sv33_c64", sv(64, 0, 33, ref=ref33)),
                     ("_rel33", release(ref33)),
                     ("single_gate_sweep", lambda: sweep(30, range(30))),
                     ("single_gate_sweep_33q", lambda: sweep(33, range(33))),
                     ("dm14_c128", dm14),
                     ("batch4096_c64", lambda: batch_variant(Q, env, torch, stream)),
                     ("partitioned_28q_4parts", lambda: partition_variant(Q, env, torch, stream)),
                     ("multi_target_passes", lambda: multi_sweep(Q, env, torch, stream, qubits)),
                     # last: after a serving sweep's many large allocations the process's later
                     # registers measured up to 15 % slower in latency-bound passes
                     ("serving", lambda: serve_sweep(Q, env, [10, 30, 100, 300, 1000, 2000], serve[0],
                                                     seconds=serve[1]))):
        # the "_" entries keep / release the FP64 reference registers of
        # the sv<n> variants: they run when any sv<n>_ variant is wanted
        if only and name not in only and not (
                name.startswith("_") and any(o.startswith("sv" + name[4:] + "_") for o in only)):
            continue
        try:
            r = fn()
            if not name.startswith("_"):
                out[name] = r
        except Exception as e:
            out[name] = {"error": str(e)}
    for keep in (ref30, ref33):
        if keep.get("q") is not None:
            Q.destroyQureg(keep.pop("q"))
    return out


def batch_variant(Q, env, torch, stream, count=4096, depth=30):
    """4096 independent complex64 state vectors, qubit counts uniform in
    8..20 (seed 4096), register i running its own depth-30 random circuit
    (seed 4096 + i), advanced together by one graph replay of the batched
    engine with an autotuned tile size.  Compared with running the same
    circuits one at a time through the unfused complex128 path (timed on a
    subset).  Every register's error and fidelity is stated against the same
    circuit run with IEEE FP64 arithmetic (a complex128 batch, which the
    parity tests hold to the FP64 oracle at 1e-12)."""
    import numpy as np
    rng = C.SplitMix64(4096)
    sizes = [8 + rng.below(13) for _ in range(count)]
    circs = [C.random_circuit(n, depth, 4096 + i) for i, n in enumerate(sizes)]
    regs, regs128 = [], []
    try:
        for n, ops in zip(sizes, circs):
            q = Q.createQureg(n, 64, env)
            Q.applyCircuit(q, ops)
            regs.append(q)
        b = Q.createBatch(env, regs)
        # tile size and fusion depth tuned together (tiles below 10 act as 10
        # on registers of 10 or more qubits: a complex64 tile holds at least
        # 2^(R + 5) amplitudes, R = 5)
        k, depth = Q.tuneBatchJoint(b, [8, 10, 11, 12, 13], [0, 32, 64, 128], replays=1)
        # both schedules at the tuned plan: one launch per wave (graph of
        # waves) and one persistent launch over every wave; the batch keeps
        # the faster one
        form_ms = {}
        for persistent in (0, 1):
            Q.setEnvOption(env, "batch_persistent", persistent)
            Q.tuneBatchJoint(b, [k], [depth], replays=1)    # re-plans in this form
            form_ms[persistent] = timed(torch, stream, lambda: Q.runBatch(b), 3)
        best_form = min(form_ms, key=form_ms.get)
        Q.setEnvOption(env, "batch_persistent", best_form)
        Q.tuneBatchJoint(b, [k], [depth], replays=1)
        Q.setEnvOption(env, "batch_persistent", 1)
        ms = timed(torch, stream, lambda: Q.runBatch(b), 3)
        info = Q.getBatchInfo(b)
        norms = Q.getBatchNorms(b)
        for n, ops in zip(sizes, circs):
            q = Q.createQureg(n, 128, env)
            Q.applyCircuit(q, ops)
            regs128.append(q)
        b128 = Q.createBatch(env, regs128)
        Q.runBatch(b128)
        Q.syncQuESTEnv(env)
        errs = [c64_error(Q, torch, regs[i], regs128[i]) for i in range(count)]
        Q.destroyBatch(b128)
        Q.destroyBatch(b)
    finally:
        for q in regs + regs128:
            Q.destroyQureg(q)
    maxerr = np.array([e["max_abs_err"] for e in errs])
    infid = np.array([e["one_minus_fidelity"] for e in errs])
    raw = np.array([e["one_minus_raw_overlap"] for e in errs])
    # plain per-register complex128 path (one kernel per gate), subset
    Q.setEnvOption(env, "fusion", 0)
    sub = list(range(0, count, count // 64))
    try:
        reg128 = {}

        def plain():
            for i in sub:
                q = reg128.get(i)
                if q is None:
                    q = reg128[i] = Q.createQureg(sizes[i], 128, env)
                Q.initZeroState(q)
                Q.applyCircuit(q, circs[i])
            Q.syncQuESTEnv(env)

        ms_plain = timed(torch, stream, plain, 1)
        for q in reg128.values():
            Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "fusion", 1)
    return {"circuits_per_s": count / ms * 1e3, "ms_per_batch": ms, "tile_qubits": k,
            "fusion_depth": depth or "planner default (256 ops per pass)",
            "tuned_over": {"tile_qubits": [8, 10, 11, 12, 13], "fusion_depth": [0, 32, 64, 128]},
            "schedule": "persistent launch" if best_form else "one launch per wave (graph)",
            "ms_per_batch_by_schedule": {"graph_of_waves": form_ms[0], "persistent": form_ms[1]},
            "registers": count, "amplitudes": int(sum(1 << n for n in sizes)),
            "gates": int(sum(len(c) for c in circs)), "passes": info["passes"],
            "waves": info["waves"], "alg_GBps": info["bytes"] / ms / 1e6,
            "error_vs_fp64_all_registers": {
                "registers": count,
                "reference": "same circuits, complex128 batch, IEEE FP64 arithmetic",
                "max_abs_err": float(maxerr.max()), "median_max_abs_err": float(np.median(maxerr)),
                "fidelity_definition": "|<a128|a64>|^2 / (<a128|a128> <a64|a64>) (normalised states)",
                "min_fidelity": float(1.0 - infid.max()), "max_one_minus_fidelity": float(infid.max()),
                "max_one_minus_raw_overlap": float(raw.max()),
                "max_norm_dev": float(max(e["norm_dev"] for e in errs))},
            "norm_max_dev": float(np.max(np.abs(norms - 1))),
            "plain_c128_circuits_per_s": len(sub) / ms_plain * 1e3,
            "plain_c128_subset": f"{len(sub)} of the same registers, one at a time, one kernel per gate"}


def partition_variant(Q, env, torch, stream, n=28, k=2, prec=64):
    """The paper's distribution scheme with every part on this GPU: the
    28-qubit depth-40 workload over 4 parts of 26 qubits, qubit swaps as
    device-to-device exchanges between send and receive buffers.  Each run
    starts from a fresh register (the same swap schedule, so the warm-up run
    compiled every pass kernel the timed one needs).  Stated beside the same
    circuit on one 28-qubit register; a deployment with one part per GPU is
    not built (one GPU per run), so this is no multi-GPU figure."""
    import time
    ops = Q.to_qsops(C.workload_30q(n))

    def one_run():
        r = Q.createPartitionedQureg(n, k, prec, env)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Q.partApplyCircuit(r, ops)
            Q.partCalcTotalProb(r)            # waits for the parts
            return (time.perf_counter() - t0) * 1e3, Q.partGetInfo(r)
        finally:
            Q.destroyPartitionedQureg(r)

    one_run()                                 # warm-up (compiles the pass kernels)
    ms, info = one_run()
    q = Q.createQureg(n, prec, env)
    try:
        ms1 = timed(torch, stream, lambda: (Q.initZeroState(q), Q.applyCircuit(q, ops), Q.calcTotalProb(q)), 1)
    finally:
        Q.destroyQureg(q)
    return {"qubits": n, "parts": 1 << k, "precision": f"complex{prec}", "gates": ops[1],
            "ms_per_circuit": ms, "gates_per_s": ops[1] / ms * 1e3, "swaps_per_circuit": info["swaps"],
            "exchanged_GB_per_circuit": info["exchangedBytes"] / 1e9,
            "one_register_ms_per_circuit": ms1,
            "note": "all parts on one GPU: the exchange is a device-to-device copy (host clock, "
                    "fresh register per run)"}


def multi_sweep(Q, env, torch, stream, n=30):
    """One dense 2^m x 2^m gate (targets 7..7+m-1) as a single pass over an
    n-qubit register: algorithmic GB/s (read + write of every amplitude).
    Complex64 with m = 4, 5 picks the tensor cores or the CUDA cores by the
    targets' positions; both are also timed forced, with these targets and
    with the targets on the lowest bits."""
    import numpy as np
    out = {}
    Q.setEnvOption(env, "fusion", 0)
    try:
        for prec in (64, 128):
            q = Q.createQureg(n, prec, env)
            S = 16 if prec == 128 else 8
            try:
                for m in range(1, 6):
                    g = np.random.default_rng(m)
                    U = np.linalg.qr(g.normal(size=(1 << m, 1 << m)) + 1j * g.normal(size=(1 << m, 1 << m)))[0]
                    tg = tuple(range(7, 7 + m))
                    ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, tg, U), 2)
                    out[f"c{prec}_m{m}"] = {"ms": ms, "GBps": 2 * (1 << n) * S / ms / 1e6}
                    if m in (2, 3) or (prec == 128 and m >= 4):
                        # the same gate on the lowest qubits (contiguous runs
                        # in every block); complex64 m = 4, 5 below
                        low = tuple(range(m))
                        ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, low, U), 2)
                        out[f"c{prec}_m{m}_low_targets"] = {"ms": ms, "GBps": 2 * (1 << n) * S / ms / 1e6}
                    if prec == 128 and m >= 2:
                        # complex128 in double-float arithmetic (FP32 pipes)
                        Q.setEnvOption(env, "arith", 1)
                        try:
                            ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, tg, U), 2)
                        finally:
                            Q.setEnvOption(env, "arith", 0)
                        out[f"c128_df_m{m}"] = {"ms": ms, "GBps": 2 * (1 << n) * S / ms / 1e6}
                    if prec == 64 and m >= 4:
                        # the same pass on the CUDA cores, and with the targets on the lowest bits
                        low = tuple(range(m))
                        try:
                            for mode, stage, name in ((0, 1, "cuda_cores"), (2, 1, "tensor_cores"),
                                                      (2, 0, "tensor_cores_gather")):
                                Q.setEnvOption(env, "multi_tc", mode)
                                Q.setEnvOption(env, "multi_tc_stage", stage)
                                ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, tg, U), 2)
                                out[f"c64_m{m}_{name}"] = {"ms": ms, "GBps": 2 * (1 << n) * S / ms / 1e6}
                                ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, low, U), 2)
                                out[f"c64_m{m}_low_targets_{name}"] = {"ms": ms,
                                                                       "GBps": 2 * (1 << n) * S / ms / 1e6}
                        finally:
                            Q.setEnvOption(env, "multi_tc", 1)
                            Q.setEnvOption(env, "multi_tc_stage", 1)
                        ms = timed(torch, stream, lambda: Q.multiQubitUnitary(q, low, U), 2)
                        out[f"c64_m{m}_low_targets"] = {"ms": ms, "GBps": 2 * (1 << n) * S / ms / 1e6}
            finally:
                Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "fusion", 1)
    return out


def serve_trace(rate, count, seed0=5000, arrival_seed=55, max_sv=28, max_dm=13):
    """Serving workload: Poisson arrivals at `rate` req/s (exponential gaps
    from their own SplitMix64 stream), request i seeded 5000 + i: type
    uniform over {state vector c64, state vector c128, density matrix};
    state vectors n ~ U{10..28}, density matrices N ~ U{6..13} with
    dephasing 0.01 after every gate; depth ~ U{10..50}.  A density matrix's
    precision (complex64 or complex128, uniform) is the request's last draw."""
    import math
    arr = C.SplitMix64(arrival_seed)
    t, trace = 0.0, []
    for i in range(count):
        t += -math.log(1.0 - arr.uniform()) / rate
        rng = C.SplitMix64(seed0 + i)
        kind = rng.below(3)
        depth = 10 + rng.below(41)
        if kind == 2:
            N = 6 + rng.below(max_dm - 5)
            ops = C.with_noise(C.random_circuit(N, depth, seed0 + i), 0.01, 0.0)
            trace.append((t, True, N, 64 if rng.below(2) == 0 else 128, ops))
        else:
            n = 10 + rng.below(max_sv - 9)
            trace.append((t, False, n, 64 if kind == 0 else 128,
                          C.random_circuit(n, depth, seed0 + i)))
    return trace


def run_trace(Q, env, trace, slots, fusion, force_c128=False, capture=None, max_queue_us=0):
    """Submits each request at its arrival time, collects every result;
    returns latency percentiles and throughput.  capture: optional dict
    {request index: None}; those requests return their full final state
    (filled in place)."""
    import numpy as np
    srv = Q.serveCreate(env, slots=slots, budgetBytes=150 * 10 ** 9, fusion=fusion)
    if max_queue_us:
        Q.serveSetOption(srv, "max_queue_us", max_queue_us)
    prepared = [(t, dens, n, 128 if force_c128 else prec, Q.to_qsops(ops))
                for (t, dens, n, prec, ops) in trace]
    tickets = []
    try:
        t0 = time.perf_counter()
        for i, (t, dens, n, prec, qs) in enumerate(prepared):
            wait = t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            out = None
            if capture is not None and i in capture:
                out = capture[i] = np.zeros(1 << (2 * n if dens else n), dtype=np.complex128)
            tickets.append(Q.serveSubmit(srv, qs, n, prec, dens, outAmps=out))
        res = [Q.servePoll(srv, tk, timeoutUs=600_000_000) for tk in tickets]
        wall = time.perf_counter() - t0
    finally:
        Q.serveDestroy(srv)
    ok = [r for r in res if r["status"] == 0]
    shed = sum(Q.ERRORS.get(r["status"]) == "QS_E_BUSY" for r in res)
    lat = np.array([r["latencyUs"] for r in ok] or [0.0]) / 1e3
    return {"requests": len(res), "completed": len(ok), "shed": int(shed),
            "failed": int(len(res) - len(ok) - shed), "circuits_per_s": len(ok) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_queued_ms": float(np.mean([r["queuedUs"] for r in ok] or [0.0]) / 1e3),
            "slots_used": len({r["slot"] for r in ok})}


def served_c64_error(Q, env, trace, captured):
    """Per captured complex64 request: max |a64 - a128|, the normalised
    fidelity and the raw overlap against the same circuit run with IEEE FP64
    arithmetic in a complex128 register (held to the FP64 oracle at 1e-12 by
    the parity tests).  Returns the worst over the sample."""
    import numpy as np
    rows = []
    for i, got in captured.items():
        if got is None:
            continue
        _, _, n, _, ops = trace[i]
        q = Q.createQureg(n, 128, env)
        try:
            Q.applyCircuit(q, ops)
            ref = Q.copyStateToHost(q)
        finally:
            Q.destroyQureg(q)
        ip = np.vdot(ref, got)
        n_ref, n_got = np.vdot(ref, ref).real, np.vdot(got, got).real
        rows.append((float(np.max(np.abs(got - ref))), 1.0 - abs(ip) ** 2 / (n_ref * n_got),
                     1.0 - abs(ip) ** 2))
    if not rows:
        return None
    return {"requests": len(rows), "max_abs_err": max(r[0] for r in rows),
            "max_one_minus_fidelity": max(r[1] for r in rows),
            "max_one_minus_raw_overlap": max(r[2] for r in rows)}


def serve_sweep(Q, env, rates, per_rate, slots=16, baseline_rates=None, seconds=0.0):
    """Per arrival rate: `per_rate` requests, or fewer if `seconds` > 0 caps
    the trace at that many seconds of arrivals (rate x seconds requests)."""
    out = {}
    for rate in rates:
        count = per_rate if seconds <= 0 else max(1, min(per_rate, int(rate * seconds)))
        trace = serve_trace(rate, count)
        # complex64 state-vector requests of up to 22 qubits return their
        # states: error and fidelity against the same circuit in IEEE FP64
        cap = {i: None for i, (_, dens, n, prec, _) in enumerate(trace) if not dens and prec == 64 and n <= 22}
        cap = dict(list(cap.items())[:12])
        row = {"served": run_trace(Q, env, trace, slots, 1, capture=cap)}
        row["served"]["c64_error_vs_fp64"] = served_c64_error(Q, env, trace, cap)
        # admission policy past saturation: requests that cannot start within
        # 1 s are shed, which bounds the latency of the ones served
        row["served_shed_after_1s"] = run_trace(Q, env, trace, slots, 1, max_queue_us=1_000_000)
        if baseline_rates is None or rate in baseline_rates:
            row["plain_c128_one_at_a_time"] = run_trace(Q, env, trace, 1, 0, force_c128=True)
        out[f"{rate}_req_per_s"] = row
    return out


if __name__ == "__main__":
    main()
