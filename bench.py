#!/usr/bin/env python3
"""Benchmark: optimisation sweeps of the scale-invariant binary MERA
(critical transverse-field Ising chain, spins blocked in pairs, tau* = 3,
20 power steps for rho* per sweep) on one GB300 per rank.

A step is one full sweep (ascend h through the transitional layers, rho*
power iteration, u/w environments and polar updates of every layer, rho
descent, energy) at the precision configuration's bond dimension chi = 32 in
split-BF16 (BF16X3) by default.  Inputs are synthetic (seeded QR isometries)
and resident in HBM when the timed region starts; `e2e` repeats the
measurement through the C ABI with host buffers (inputs copied in, energy
copied out per step).  The same line carries the accuracy of that sweep
against the fixed-point split mode OZ4 (whose own error against FP64 is
measured at chi = 16 in the same run), and a chi = 16 block with the plain
FP64 GPU sweep and the energy gap of every mode after one sweep.

`--impl reference` times the FP64 CPU oracle on the host cores instead, on a
bounded sample of the same workload per step (a whole oracle sweep where
that takes seconds, else one scale-invariant descending diagram at
min(chi, 16) scaled to the sweep by flops, marked "extrapolated"); it loads
no part of the CUDA library.

Multi-GPU: independent replicas (one MERA per rank, no data-path
collective); the value is the sum of sweeps over ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MERA sweep iters/s & contraction TFLOP/s vs chi; mixed vs FP64 at dE<=1e-6/site"
N_POW = 20
HZ = 1.0
SEED = 0
DEFAULT_CHI = 32
# nominal dense tensor/FP64 rates (PFLOP/s) used only to carry the measured
# BF16 peak over to the other modes, in algorithmic flops (a split mode
# issues 3, 6 or 10 BF16 products per algorithmic one)
NOMINAL = {"bf16": 2.25, "tf32": 1.1, "f64": 0.00125, "bf16x3": 2.25 / 3.0, "bf16x6": 2.25 / 6.0,
           "oz3": 2.25 / 6.0, "oz4": 2.25 / 10.0}

# Flops of one diagram of the contraction programs per layer shape
# (chi_bottom, chi_top): the min-flop pairwise orders of the library's
# planner (mera_flops / number of diagrams; tests/test_bench_cpu.py checks
# this table against the library).  Kept here so that the reference arm
# needs no part of the library.  An operation has 2 (ascend, descend),
# 4 (env_u) or 6 (env_w) diagrams of equal cost.
DIAGRAM_FLOPS = {
    (4, 4): 1593344.0, (4, 8): 13402112.0, (4, 12): 110817280.0, (4, 16): 577077248.0,
    (8, 8): 672268288.0, (12, 12): 24091914240.0, (16, 16): 309308948480.0, (16, 20): 427987042304.0,
    (16, 24): 590215118848.0, (16, 32): 1288574074880.0, (16, 40): 3190868148224.0,
    (20, 20): 2253068800000.0, (24, 24): 11448628936704.0, (32, 32): 149538010562560.0,
    (40, 40): 1101021593600000.0,
}
N_DIAGRAMS = {"ascend": 2, "descend": 2, "env_u": 4, "env_w": 6}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--chi", type=int, default=DEFAULT_CHI)
    ap.add_argument("--prec", default="bf16x3", choices=["f64", "tf32", "bf16", "bf16x3", "bf16x6", "oz3", "oz4"])
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="FP64 sweeps timed at chi = 16 (0: skip the chi = 16 block)")
    ap.add_argument("--eval-pow", type=int, default=20,
                    help="power steps for rho* when the final state is evaluated in two modes")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy block at the headline chi")
    ap.add_argument("--slice-gib", type=float, default=None,
                    help="slice rank-7 intermediates larger than this (GiB; default 16)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time direct mera_sweep calls instead of graph replays")
    ap.add_argument("--tune", action="store_true", help="--case ascend|descend|env_u|env_w: autotune the map first")
    ap.add_argument("--widths", default=None,
                    help="JSON list of recorded tile widths (from --save-widths) to set instead of autotuning")
    ap.add_argument("--save-widths", default=None, help="write the autotuned tile widths to this JSON file")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the planner's tile widths (no mera_autotune before timing)")
    ap.add_argument("--sweeps", type=int, default=300, help="--case precision: optimisation sweeps per run")
    ap.add_argument("--polish", type=int, default=20, help="--case precision: FP64 sweeps after the mixed ones")
    ap.add_argument("--z2", action="store_true",
                    help="--case precision: parity-symmetric (Z2 block-diagonal) starting tensors")
    ap.add_argument("--riemannian-eta", type=float, default=0.0,
                    help="--case precision: also run Riemannian-gradient sweeps with this step size")
    ap.add_argument("--grow-from", type=int, default=0,
                    help="--case precision: also optimise at this chi first and grow to --chi")
    ap.add_argument("--grow-sweeps", type=int, default=2000, help="--case precision: sweeps before growing")
    ap.add_argument("--batch-chis", default="8,12,16",
                    help="--case batch: comma-separated bond dimensions the 32 MERAs draw from")
    ap.add_argument("--scaling-k", type=int, default=0,
                    help="--case precision: scaling dimensions (FP64 and mixed Arnoldi) of the final state")
    ap.add_argument("--ref-prec", default="f64", choices=["f64", "oz4", "oz3"],
                    help="--case precision: the mode of the reference run")
    ap.add_argument("--spectrum-chis", default="4,6,8,10,12,14,16",
                    help="--case spectrum: bond dimensions of the growth ladder (parity-symmetric MERA)")
    ap.add_argument("--spectrum-sweeps", default="4000,4000,4000,4000,4000,4000,6000",
                    help="--case spectrum: sweeps at each of them")
    ap.add_argument("--case", default="sweep",
                    choices=["sweep", "ascend", "descend", "env_u", "env_w", "batch", "precision", "spectrum"])
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)  # internal: oracle timing child
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the default process group (x itself
    without one).  `device`: where the reduction tensor lives (the rank's GPU
    for NCCL, the CPU for gloo)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return x
    if torch.distributed.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_throughput(world: int, steps: int, max_ms: float) -> float:
    """Whole-job sweeps per second: every rank runs `steps` sweeps of its own
    replica, and the job takes as long as its slowest rank (max_ms)."""
    return world * steps / (max_ms / 1e3)


def _heuristic_bn(prec: str, n: int) -> int:
    """The planner's tile width when nothing is tuned (for reporting): for
    N > 128 the width of 256, 192, 160 with the least ceil(N / w) (128 + w)."""
    if n > 128:
        if prec in ("bf16x6", "oz3", "oz4"):
            return 128
        return min((256, 192, 160), key=lambda w: (-(-n // w) * (128 + w), -w))
    return 128 if n > 64 else 64 if n > 16 else 16


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _peak_tflops(prec: str, sustained: bool = True):
    """Peak of a mode in algorithmic flops: the measured BF16 peak (burst for
    a kernel timed alone, sustained for one timed inside long steps) times
    the nominal ratio of the mode."""
    d, src = _peaks()
    base = d.get("bf16_tflops_sustained" if sustained else "bf16_tflops", d.get("bf16_tflops"))
    return base * NOMINAL[prec] / NOMINAL["bf16"], f"{src} {'sustained' if sustained else 'burst'}"


# DRAM bytes per launch of the chi^9-class GEMMs, from the ncu capture named
# here (profiles/).  Reported only for the workload it was taken on; it must
# be retaken (or set to None) whenever the kernel changes.
ROOFLINE_TRAFFIC = {("bf16x3", 32): (17.46e9, "profiles/tc_gemm_bf16x3_chi32_descend_dram.md (48 chi^9-class "
                                              "launches of the descending map, the sweep's most frequent, per launch)")}


def _layer_dims(chi: int):
    """(chi_bottom, chi_top) per layer, tau* = 3, blocked sites of dimension 4
    (the same rule as mera_inputs.layer_dims; no import of the package)."""
    dims, bottom = [], 4
    for _ in range(3):
        top = min(bottom * bottom, chi)
        dims.append((bottom, top))
        bottom = top
    return dims


def _map_flops(op: str, cb: int, ct: int) -> float:
    if (cb, ct) not in DIAGRAM_FLOPS:
        raise KeyError(f"no flop count recorded for the layer shape ({cb}, {ct})")
    return N_DIAGRAMS[op] * DIAGRAM_FLOPS[(cb, ct)]


def _sweep_flops(chi: int) -> float:
    """Algorithmic flops of one sweep: ascend h up the transitional layers,
    N_POW descending steps for rho*, both environments of every layer, rho
    down the middle transitional layer, and the energy (an ascend of h1)."""
    dims = _layer_dims(chi)
    total = 0.0
    for k, (cb, ct) in enumerate(dims):
        if k < len(dims) - 1:
            total += _map_flops("ascend", cb, ct)
        else:
            total += N_POW * _map_flops("descend", cb, ct)
        total += _map_flops("env_u", cb, ct) + _map_flops("env_w", cb, ct)
        if 0 < k < len(dims) - 1:
            total += _map_flops("descend", cb, ct)
        elif k == 0:
            total += _map_flops("ascend", cb, ct)
    return total


def _config(chi: int):
    """The workload, identical for the native and the reference arm."""
    return {"workload": f"critical-Ising scale-invariant binary MERA sweep, chi={chi}, tau*=3, "
                        f"{N_POW} rho* power steps, blocked d=4", "chi": chi, "n_pow": N_POW, "hz": HZ,
            "seed": SEED, "layer_dims": [list(x) for x in _layer_dims(chi)], "sweep_flops": _sweep_flops(chi),
            "parallelism": "replicas",
            "l2": "256 MB buffer written between timed steps (untimed); working set > L2"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mera_bench_clocks_{os.getpid()}_{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def _oracle_sample(kind: str, chi: int, repeats: int):
    """Times the FP64 oracle as it stands: `kind` "sweep" (a whole
    optimisation sweep from the seeded start, continuing the state between
    repeats) or "diag" (one scale-invariant descending diagram, even
    position).  Returns (seconds per repeat, flops per repeat)."""
    import numpy as np

    import mera_inputs as I
    from oracle import mera_oracle as O

    times = []
    if kind == "sweep":
        layers = [(u.copy(), w.copy()) for u, w in I.init_mera(SEED, chi)]
        h1, shift = O.ising_h1(HZ)
        rho = O.identity_density(chi)
        for _ in range(repeats):
            t = time.perf_counter()
            layers, rho, _ = O.sweep(layers, h1, shift, rho, N_POW)
            times.append(time.perf_counter() - t)
        return times, _sweep_flops(chi)
    rng = np.random.default_rng(SEED)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    rho = I.random_density(rng, chi)
    for _ in range(repeats):
        t = time.perf_counter()
        O.descend_case(rho, u, w, "even")
        times.append(time.perf_counter() - t)
    return times, DIAGRAM_FLOPS[(chi, chi)]


def _oracle_child(spec: str, threads: int):
    """Runs _oracle_sample in a fresh interpreter (no CUDA context, BLAS
    threads fixed before numpy loads); spec is kind:chi:repeats."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", spec], env=env, cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(f"oracle timing child failed: {out.stderr[-2000:]}")
    return json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])


def _run_cpu_sample(spec: str):
    kind, chi, reps = spec.split(":")
    times, flops = _oracle_sample(kind, int(chi), int(reps))
    print(json.dumps({"kind": kind, "chi": int(chi), "times_s": times, "flops": flops,
                      "threads": os.environ.get("OPENBLAS_NUM_THREADS")}), flush=True)


def _cpu_baseline(chi: int):
    """The oracle on the host cores: all cores and one thread, each sample
    repeated three times (medians).  Whole sweeps at chi = 8 are measured
    as they are; the figure at the benchmarked chi scales the all-core rate
    of one chi = 16 diagram (the largest that takes seconds) to that sweep's
    flops, and says so."""
    cores = os.cpu_count() or 1
    res = {}
    for label, threads, specs in (("all_cores", cores, ("sweep:8:3", f"diag:{min(chi, 16)}:3")),
                                  ("one_thread", 1, ("sweep:8:3", f"diag:{min(chi, 12)}:3"))):
        block = {"threads": threads}
        for spec in specs:
            r = _oracle_child(spec, threads)
            med = statistics.median(r["times_s"])
            key = f"{r['kind']}_chi{r['chi']}"
            block[key] = {"seconds": med, "repeats": len(r["times_s"]), "gflops": r["flops"] / med / 1e9}
            if r["kind"] == "sweep":
                block[key]["sweeps_per_s"] = 1.0 / med
        res[label] = block
    dkey = f"diag_chi{min(chi, 16)}"
    rate = res["all_cores"][dkey]["gflops"] * 1e9
    exact = chi == 8
    value = res["all_cores"]["sweep_chi8"]["sweeps_per_s"] if exact else rate / _sweep_flops(chi)
    sample = ("whole chi=8 oracle sweeps (median of 3)" if exact else
              f"one chi={min(chi, 16)} scale-invariant descending diagram with numpy float64 (median of 3), "
              f"its flop rate scaled to the chi={chi} sweep ({_sweep_flops(chi):.3e} flop)")
    return {"value": value, "unit": "sweep/s", "cores": cores, "kind": "oracle", "extrapolated": not exact,
            "sample": sample, "measured": res}


def run_reference(args):
    """The FP64 oracle on the host cores, one bounded sample of the sweep
    per step; no part of the CUDA library is loaded."""
    _, rank, _ = _dist()
    if rank != 0:
        return
    chi = args.chi
    sweep_flops = _sweep_flops(chi)
    whole = chi <= 8
    kind, cs = ("sweep", chi) if whole else ("diag", min(chi, 16))
    _oracle_sample(kind, cs, args.warmup)
    times, flops = _oracle_sample(kind, cs, args.steps)
    dt = sum(times) / len(times)
    value = 1.0 / dt if whole else (flops / dt) / sweep_flops
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    sample = (f"per step one whole chi={chi} oracle sweep" if whole else
              f"per step one chi={cs} scale-invariant descending diagram ({flops:.3e} flop) with numpy float64, "
              f"its flop rate scaled to the chi={chi} sweep ({sweep_flops:.3e} flop)")
    one = None
    try:  # one BLAS thread, as in the paper's 1-core comparison (Sec. III B)
        r = _oracle_child(f"{kind}:{min(cs, 12) if not whole else cs}:1", 1)
        t1 = r["times_s"][0]
        one = {"threads": 1, "seconds": t1, "gflops": r["flops"] / t1 / 1e9,
               "value": (1.0 / t1) if whole else (r["flops"] / t1) / sweep_flops,
               "sample": f"{r['kind']} at chi={r['chi']}"}
    except Exception as exc:  # the line is still valid without it
        one = {"error": str(exc)[:200]}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sweep/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "extrapolated": not whole,
        "tflops": sweep_flops * value / 1e12,
        "config": _config(chi),
        "cpu_baseline": {"value": value, "unit": "sweep/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "extrapolated": not whole, "one_thread": one},
        "e2e": {"value": value, "unit": "sweep/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "note": "ms_per_step is the timed sample; value scales its flop rate to a whole sweep" if not whole
        else "ms_per_step is one whole oracle sweep",
    }
    print(json.dumps(line), flush=True)


def run_native(args):
    import numpy as np
    import torch

    import mera_inputs as I

    world, rank, local = _dist()
    chi = args.chi
    # the oracle's timings first, in child processes, before this process
    # holds a CUDA context (and so that they do not overlap the GPU timing)
    cpu = _cpu_baseline(chi) if (not args.no_cpu_baseline and world == 1) else None

    import paper_1906_12030_gb300 as m

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    prec = m.PRECS[args.prec]
    h1_host, shift = m.mera_ising_h1(HZ)
    h1 = torch.from_numpy(h1_host.reshape(-1)).to(dev)
    # a stream of our own (sweep graphs cannot be recorded on the legacy
    # default stream); torch's own work (the L2 flush) is ordered on it too
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    class Run:
        """A seeded MERA at bond dimension c, its sweep workspace in mode p,
        and one sweep (direct call) or a recorded sweep graph."""

        def __init__(self, p, c):
            layers = I.init_mera(SEED, c)
            self.c, self.p = c, p
            self.us = [torch.from_numpy(u).to(dev).reshape(-1).contiguous() for u, _ in layers]
            self.ws = [torch.from_numpy(w).to(dev).contiguous() for _, w in layers]
            n3 = c ** 3
            self.rho = (torch.eye(n3, dtype=torch.float64, device=dev) / n3).reshape(-1).contiguous()
            self.st = m.MeraState(self.us, self.ws, self.rho)
            self.wsb = m.workspace(m.mera_sweep_workspace_size(self.st.chi_b, self.st.chi_t, p), dev)
            self.e = torch.empty(1, dtype=torch.float64, device=dev)
            self.graph = None

        def sweep(self):
            try:
                m.mera_sweep(self.st, h1, shift, N_POW, self.e, prec=self.p, ws=self.wsb, stream=stream)
            except m.MeraNotConverged:
                pass  # a polar update hit its cap; the sweep is complete

        def record(self):
            self.graph = m.mera_sweep_graph(self.st, h1, shift, N_POW, self.e, prec=self.p, ws=self.wsb,
                                            stream=stream)

        def step(self):
            if self.graph is not None:
                self.graph.launch(stream)
            else:
                self.sweep()

        def close(self):
            if self.graph is not None:
                self.graph.close()
                self.graph = None

    def timed(fn, n, sample_clocks=False):
        """n calls of fn, each bracketed by CUDA events on the stream, the L2
        flushed (untimed) before each; returns (total ms, clock summary)."""
        a = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        for k in range(n):
            flush.fill_(k & 0xFF)
            a[k].record(stream)
            fn()
            b[k].record(stream)
        torch.cuda.synchronize(dev)
        if clk:
            clk.__exit__(None, None, None)
        if world > 1:
            torch.distributed.barrier()
        return sum(x.elapsed_time(y) for x, y in zip(a, b)), (clk.summary() if clk else None)

    def evaluate(run, p, n_pow):
        """Energy per spin of run's state with every map in mode p: rho* by
        n_pow power steps from the state's warm start, rho down the
        transitional layers, tr(h1 rho1) + shift over two spins."""
        dims = I.layer_dims(run.c)
        rho = run.rho.clone()
        ws_fp = m.workspace(m.mera_workspace_size(m.OP_FIXED_POINT, run.c, run.c, p), dev)
        m.mera_fixed_point_rho(run.us[-1], run.ws[-1], run.c, rho, n_pow, prec=p, ws=ws_fp, stream=stream)
        del ws_fp
        for t in range(len(dims) - 2, 0, -1):
            cb, ct = dims[t]
            out = torch.empty(cb ** 6, dtype=torch.float64, device=dev)
            m.mera_descend(rho, run.us[t], run.ws[t], cb, ct, out, prec=p, stream=stream)
            rho = out
        cb, ct = dims[0]
        e = torch.empty(1, dtype=torch.float64, device=dev)
        m.mera_energy(h1, rho, run.us[0], run.ws[0], cb, ct, e, prec=p, stream=stream)
        return 0.5 * (float(e.item()) + shift)

    # ---- tile widths: the library's autotuner (or widths recorded earlier) ----
    tuned = None
    if not args.no_autotune and prec != m.PREC_F64:
        n_shapes, moved = 0, set()
        if args.widths:  # recorded widths of an earlier run, set without timing
            with open(args.widths) as f:
                for pr, M, N, K, cf, bn in json.load(f):
                    m.mera_set_tile_width(pr, M, N, K, cf, bn)
                    n_shapes += 1
        else:
            for cb, ct in I.layer_dims(chi):
                for op in (m.OP_ASCEND, m.OP_DESCEND, m.OP_ENV_U, m.OP_ENV_W):
                    n_shapes += m.mera_autotune(op, cb, ct, prec, device=dev)
        if args.save_widths and local == 0:
            with open(args.save_widths, "w") as f:
                json.dump([list(x) for x in m.mera_tile_widths()], f)
        for cb, ct in I.layer_dims(chi):
            for op in (m.OP_ASCEND, m.OP_DESCEND, m.OP_ENV_U, m.OP_ENV_W):
                for dg in m.mera_plan_json(op, cb, ct, prec)["diagrams"]:
                    for st in dg["steps"]:
                        if st["kind"] == "gemm" and st["bn"] != _heuristic_bn(args.prec, st["N"]):
                            moved.add((st["M"], st["N"], st["K"], st["bn"], bool(st["dominant"])))
        tuned = {"shapes_timed" if not args.widths else "shapes_loaded": n_shapes, "moved": sorted(moved)}

    sweep_flops = _sweep_flops(chi)
    run = Run(prec, chi)
    if not args.no_graph:
        run.record()
    # ---- headline: W untimed steps, then exactly K timed ones -----------------
    for _ in range(args.warmup):
        run.step()
    torch.cuda.synchronize(dev)
    launches0 = m.mera_launch_count()
    total_ms, clk = timed(run.step, args.steps, sample_clocks=True)
    launches = m.mera_launch_count() - launches0
    total_ms = _max_over_ranks(total_ms, dev)
    energy = run.e.item()

    # ---- direct calls with per-kernel events: roofline and stage split --------
    n_direct = max(1, min(args.steps, 2))
    m.mera_profile_enable(True)
    l0 = m.mera_launch_count()
    direct_ms, clk_direct = timed(run.sweep, n_direct, sample_clocks=True)
    launches_direct = m.mera_launch_count() - l0
    dom = m.mera_profile_read(m.PROF_GEMM_DOMINANT)
    allg = m.mera_profile_read(m.PROF_GEMM)
    perm = m.mera_profile_read(m.PROF_PERMUTE)
    m.mera_profile_enable(False)
    direct_ms = _max_over_ranks(direct_ms, dev)
    direct = {"value": _job_throughput(world, n_direct, direct_ms), "unit": "sweep/s",
              "ms_per_step": direct_ms / n_direct, "steps": n_direct, "gpu_launches": launches_direct,
              "clocks": clk_direct, "note": "one mera_sweep call per step; per-kernel CUDA events on the launching "
                                            "stream give the roofline and the stage split"}

    # ---- end to end through the C ABI with host buffers ---------------------
    # (mera_sweep_host: the state and h1 copied in from pinned host memory,
    # the sweep -- a replay of the recorded graph --, the energy copied out)
    e2e = None
    if not args.no_e2e:
        host_us = [t.detach().reshape(-1).cpu().pin_memory() for t in run.us]
        host_ws = [t.detach().reshape(-1).cpu().pin_memory() for t in run.ws]
        host_rho = run.rho.detach().cpu().pin_memory()
        host_h1 = h1.detach().cpu().pin_memory()
        e_host = torch.empty(1, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host_us + host_ws + [host_rho, host_h1])
        n_e2e = max(1, min(args.steps, 3))

        def e2e_step():
            m.mera_sweep_host(run.st, host_us, host_ws, host_rho, host_h1, h1, shift, N_POW, run.e, e_host,
                              prec=prec, ws=run.wsb, graph=run.graph, stream=stream)

        e2e_ms, _ = timed(e2e_step, n_e2e)
        e2e_ms = _max_over_ranks(e2e_ms, dev)
        e2e = {"value": _job_throughput(world, n_e2e, e2e_ms), "unit": "sweep/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8, "steps": n_e2e,
               "path": "mera_sweep_host (graph replay)" if run.graph is not None else "mera_sweep_host",
               "note": "per step, one C-ABI call: the state (u, w of every layer, rho*, h1) copied in from pinned "
                       "host memory, one sweep, the energy copied out"}
    run.close()
    run.wsb = None  # the sweep scratch is not needed for the evaluations below
    torch.cuda.empty_cache()

    # ---- accuracy of the headline mode at the headline chi --------------------
    accuracy = None
    if not args.no_accuracy and rank == 0 and prec not in (m.PREC_F64, m.PREC_OZ4):
        t0 = time.perf_counter()
        e_mode = evaluate(run, prec, args.eval_pow)
        t1 = time.perf_counter()
        e_oz4 = evaluate(run, m.PREC_OZ4, args.eval_pow)
        t2 = time.perf_counter()
        # one descending map of the same rho* in both modes
        n6 = chi ** 6
        d_mode = torch.empty(n6, dtype=torch.float64, device=dev)
        d_oz4 = torch.empty(n6, dtype=torch.float64, device=dev)
        m.mera_descend(run.rho, run.us[-1], run.ws[-1], chi, chi, d_mode, prec=prec, stream=stream)
        m.mera_descend(run.rho, run.us[-1], run.ws[-1], chi, chi, d_oz4, prec=m.PREC_OZ4, stream=stream)
        rel = float((d_mode - d_oz4).abs().max() / d_oz4.abs().max())
        del d_mode, d_oz4
        torch.cuda.empty_cache()
        accuracy = {"reference_mode": "oz4",
                    "energy_per_spin": {args.prec: e_mode, "oz4": e_oz4},
                    "dE_per_site_eval": abs(e_mode - e_oz4),
                    "descend_rel_err_vs_oz4": rel,
                    "eval": f"state after the timed sweeps; rho* by {args.eval_pow} power steps from its warm start, "
                            f"descended, energy per spin, every map in the named mode",
                    "seconds": {args.prec: t1 - t0, "oz4": t2 - t1}}

    # ---- the fixed-point split mode OZ4 at the headline chi ------------------
    # (its sweep energies track FP64 to ~1e-9 per site; here its throughput
    # and tensor-pipe rate at this size, against the FP64 sweep's estimate)
    oz4 = None
    if not args.no_accuracy and rank == 0 and prec != m.PREC_OZ4 and chi >= 24:
        r = Run(m.PREC_OZ4, chi)
        r.sweep()  # plans, recordings of the polar loops
        m.mera_profile_enable(True)
        ms, clk_oz = timed(r.sweep, 1, sample_clocks=True)
        d4 = m.mera_profile_read(m.PROF_GEMM_DOMINANT)
        c4 = m.mera_profile_read(m.PROF_PERMUTE)
        m.mera_profile_enable(False)
        tf4 = d4[2] / (d4[1] / 1e3) / 1e12 if d4[1] > 0 else None
        pk4, pk4_src = _peak_tflops("oz4", sustained=True)
        oz4 = {"sweeps_per_s": 1e3 / ms, "ms_per_step": ms, "steps": 1, "tflops": sweep_flops / ms / 1e9,
               "energy_per_spin_after_2_sweeps": r.e.item(),
               "dominant_tflops": tf4, "frac_of_mode_peak": (tf4 / pk4) if tf4 else None,
               "peak": pk4, "peak_source": f"{pk4_src} bf16 / 10 products, of measured",
               "copy_cast_split_ms": c4[1], "clocks": clk_oz,
               "note": "one direct sweep after one warm sweep from the seeded start, per-kernel events"}
        r.wsb = None
        del r
        torch.cuda.empty_cache()

    # ---- chi = 16: the plain FP64 GPU sweep and every mode's energy gap -------
    chi16 = None
    if args.fp64_steps > 0 and rank == 0:
        c16 = 16
        modes = ["f64", "bf16x3", "oz3", "oz4"]
        energies, rates = {}, {}
        for name in modes:
            r = Run(m.PRECS[name], c16)
            ms, _ = timed(r.sweep, 1)  # one sweep from the seeded start
            energies[name] = r.e.item()
            if name == "f64":
                reps = max(0, args.fp64_steps - 1)
                if reps:
                    ms2, _ = timed(r.sweep, reps)
                    ms = (ms + ms2) / (1 + reps)
                rates[name] = {"sweeps_per_s": 1e3 / ms, "ms_per_step": ms, "steps": 1 + reps,
                               "tflops": _sweep_flops(c16) / ms / 1e9}
            else:
                r.record()
                r.step()
                ms, _ = timed(r.step, 3)
                rates[name] = {"sweeps_per_s": 3e3 / ms, "ms_per_step": ms / 3, "steps": 3,
                               "tflops": _sweep_flops(c16) / (ms / 3) / 1e9, "path": "graph replay"}
                r.close()
            del r
            torch.cuda.empty_cache()
        # the split mode used as the chi = 32 reference, against FP64 on one map
        rng = np.random.default_rng(SEED)
        u, w = I.random_u(rng, c16), I.random_w(rng, c16, c16)
        hh = torch.from_numpy(I.random_operator(rng, c16)).to(dev).reshape(-1)
        ud, wd = torch.from_numpy(u).to(dev).reshape(-1), torch.from_numpy(w).to(dev).reshape(-1)
        outs = {}
        for name in ("f64", "oz4", "oz3", "bf16x3"):
            o = torch.empty(c16 ** 6, dtype=torch.float64, device=dev)
            m.mera_ascend(hh, ud, wd, c16, c16, o, prec=m.PRECS[name], stream=stream)
            outs[name] = o
        scale = float(outs["f64"].abs().max())
        chi16 = {"chi": c16,
                 "energy_per_spin_after_1_sweep": energies,
                 "dE_per_site_after_1_sweep": {k: abs(v - energies["f64"]) for k, v in energies.items() if k != "f64"},
                 "ascend_rel_err_vs_f64": {k: float((v - outs["f64"]).abs().max()) / scale
                                           for k, v in outs.items() if k != "f64"},
                 "throughput": rates,
                 "fp64_sweeps_per_s_at_headline_chi_estimate": rates["f64"]["tflops"] * 1e12 / sweep_flops,
                 "fp64_estimate_note": "the chi = 16 FP64 sweep's flop rate (the FP64 pipe limit) over the "
                                       "headline chi's sweep flops",
                 "note": "one sweep from the seeded QR start in every mode; FP64 timed directly (its polar "
                         "updates and maps dominate), the others as replayed sweep graphs"}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    value = _job_throughput(world, args.steps, total_ms)
    peak, peak_src = _peak_tflops(args.prec, sustained=True)
    dom_tflops = dom[2] / (dom[1] / 1e3) / 1e12 if dom[1] > 0 else None
    cfg = _config(chi)
    cfg["parallelism"] = f"replicas{world}"
    line = {
        "metric": METRIC, "value": value, "unit": "sweep/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "tflops": sweep_flops * value / world / 1e12,
        "config": cfg,
        "timing": "one mera_sweep call per step" if args.no_graph
        else "mera_sweep recorded once as a CUDA graph, replayed each step",
        "energy_per_spin": energy,
        "accuracy": accuracy,
        "oz4": oz4,
        "chi16": chi16,
        "roofline": {"bound": "tensor" if args.prec != "f64" else "fp64", "achieved": dom_tflops, "peak": peak,
                     "unit": "TFLOP/s", "frac": (dom_tflops / peak) if dom_tflops else None,
                     "traffic": ROOFLINE_TRAFFIC.get((args.prec, chi), (None, None))[0],
                     "traffic_source": ROOFLINE_TRAFFIC.get((args.prec, chi), (None, None))[1],
                     "kernel": "gemm_f64_kernel" if args.prec == "f64" else "tcgen05 GEMM (chi^9-class steps)",
                     "launches": dom[0], "kernel_ms": dom[1],
                     "peak_source": f"{peak_src} bf16 x nominal ratio of the mode (algorithmic flops), of measured",
                     "timed_in": f"{n_direct} direct sweeps, CUDA events on the launching stream"},
        "stage_ms_per_step": {"gemm": allg[1] / n_direct, "gemm_dominant": dom[1] / n_direct,
                              "copy_cast_split": perm[1] / n_direct, "sweep": direct_ms / n_direct},
        "gpu_launches": launches,
        "gpu_launches_counting": ("kernel nodes of the recorded sweep per replay; the body of each polar update's "
                                  "while loop counts once although it runs several times") if not args.no_graph
        else "kernel launches issued by the library",
        "autotune": tuned,
        "direct": direct,
        "clocks": clk,
        "e2e": e2e,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_case(args):
    """One warm call and one timed call of a single map (profiling target)."""
    import numpy as np
    import torch

    import mera_inputs as I
    import paper_1906_12030_gb300 as m

    chi, prec = args.chi, m.PRECS[args.prec]
    rng = np.random.default_rng(SEED)
    u, w = I.random_u(rng, chi), I.random_w(rng, chi, chi)
    d = lambda x: torch.from_numpy(x).cuda().reshape(-1)  # noqa: E731
    ud, wd = d(u), d(w)
    need_h = args.case != "descend"
    need_rho = args.case != "ascend"
    if chi < 24:
        hd = d(I.random_operator(rng, chi)) if need_h else None
        rd = d(I.random_density(rng, chi)) if need_rho else None
    else:
        # chi^3 x chi^3 operators (33 GB each at chi = 40): seeded symmetric
        # Gaussians drawn on the device, rho scaled to unit trace.  The maps
        # are linear, so the timing does not depend on positivity.
        g = torch.Generator(device="cuda")
        g.manual_seed(SEED)

        def sym(trace_one):
            n3 = chi ** 3
            x = torch.randn(n3, n3, dtype=torch.float64, device="cuda", generator=g)
            x.add_(x.t().contiguous()).mul_(0.5)
            if trace_one:
                x.diagonal().add_(1.0 / n3 - float(x.diagonal().sum()) / n3)
            return x.reshape(-1)

        hd = sym(False) if need_h else None
        rd = sym(True) if need_rho else None
        torch.cuda.empty_cache()
    op = {"ascend": m.OP_ASCEND, "descend": m.OP_DESCEND, "env_u": m.OP_ENV_U, "env_w": m.OP_ENV_W}[args.case]
    ws = m.workspace(m.mera_workspace_size(op, chi, chi, prec))
    out = torch.empty(chi ** 6, dtype=torch.float64, device="cuda")

    def call():
        if args.case == "ascend":
            m.mera_ascend(hd, ud, wd, chi, chi, out, prec=prec, ws=ws)
        elif args.case == "descend":
            m.mera_descend(rd, ud, wd, chi, chi, out, prec=prec, ws=ws)
        elif args.case == "env_u":
            m.mera_env_u(hd, rd, ud, wd, chi, chi, out[: chi ** 4], prec=prec, ws=ws)
        else:
            m.mera_env_w(hd, rd, ud, wd, chi, chi, out[: chi ** 3], prec=prec, ws=ws)

    if args.tune:
        m.mera_autotune(op, chi, chi, prec)
        ws = m.workspace(m.mera_workspace_size(op, chi, chi, prec))
    call()
    torch.cuda.synchronize()
    m.mera_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # ncu --nvtx --nvtx-include "timed/" selects this call
    e0.record()
    call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    dom, allg, perm = (m.mera_profile_read(k) for k in (m.PROF_GEMM_DOMINANT, m.PROF_GEMM, m.PROF_PERMUTE))
    m.mera_profile_enable(False)
    fl = m.mera_flops(op, chi, chi)
    dom_tf = dom[2] / dom[1] / 1e9 if dom[1] else None
    print(json.dumps({"case": args.case, "chi": chi, "prec": args.prec, "ms": ms, "tflops": fl / ms / 1e9,
                      "dominant": {"launches": dom[0], "ms": dom[1], "tflops": dom_tf},
                      "gemm_ms": allg[1], "permute_ms": perm[1], "device_status": m.mera_device_status()}), flush=True)


def run_batch(args):
    """Batching: 32 independent MERAs, h ~ U[0.9, 1.1], chi drawn (seeded) from
    --batch-chis, one sweep each per step.  Modes: one at a time (one shared
    scratch), mera_sweep_batch over lanes (mera_batch_lanes: one scratch and
    one stream per lane, under a budget of the device memory left after the
    states), and one recorded sweep graph per MERA replayed on its lane's
    stream."""
    import numpy as np
    import torch

    import mera_inputs as I
    import paper_1906_12030_gb300 as m

    prec = m.PRECS[args.prec]
    pool = [int(c) for c in args.batch_chis.split(",")]
    rng = np.random.default_rng(SEED)
    specs = [(s, int(rng.choice(pool)), float(rng.uniform(0.9, 1.1))) for s in range(32)]

    def make():
        out = []
        for seed, chi, hz in specs:
            layers = I.init_mera(seed, chi)
            us = [torch.from_numpy(u).cuda().reshape(-1).contiguous() for u, _ in layers]
            ws_ = [torch.from_numpy(w).cuda().contiguous() for _, w in layers]
            rho = (torch.eye(chi ** 3, dtype=torch.float64, device="cuda") / chi ** 3).reshape(-1).contiguous()
            h1, shift = m.mera_ising_h1(hz)
            out.append((m.MeraState(us, ws_, rho), torch.from_numpy(h1.reshape(-1)).cuda(), shift))
        return out

    flops = sum(_sweep_flops(chi) for _, chi, _ in specs)
    res = {}
    n_lanes = 0
    for mode in ("one_at_a_time", "batched", "graphs"):
        ms = make()
        states = [x[0] for x in ms]
        e = torch.empty(len(ms), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if mode == "one_at_a_time":
            shared = m.workspace(max(m.mera_sweep_workspace_size(st.chi_b, st.chi_t, prec) for st in states))
        else:
            free, _ = torch.cuda.mem_get_info()
            wss, streams = m.batch_resources(states, prec, budget_bytes=int(0.9 * free), n_pow=N_POW)
            n_lanes = len({id(x) for x in streams})
        graphs = []
        if mode == "graphs":  # one recorded sweep per MERA, replayed on its lane's stream
            for i, (st, h1, shift) in enumerate(ms):
                graphs.append(m.mera_sweep_graph(st, h1, shift, N_POW, e[i:i + 1], prec=prec, ws=wss[i],
                                                 stream=streams[i]))

        def step():
            if mode == "graphs":
                cur = torch.cuda.current_stream()
                for sm in streams:
                    sm.wait_stream(cur)
                for g, sm in zip(graphs, streams):
                    g.launch(sm)
                for sm in streams:
                    cur.wait_stream(sm)
            elif mode == "batched":
                try:
                    m.mera_sweep_batch(states, [x[1] for x in ms], [x[2] for x in ms], N_POW, e, prec=prec,
                                       wss=wss, streams=streams, n_threads=16)
                except m.MeraNotConverged:
                    pass
            else:
                for i, (st, h1, shift) in enumerate(ms):
                    try:
                        m.mera_sweep(st, h1, shift, N_POW, e[i:i + 1], prec=prec, ws=shared)
                    except m.MeraNotConverged:
                        pass

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        res[mode] = {"mera_sweeps_per_s": len(ms) / dt, "ms_per_step": dt * 1e3, "tflops": flops / dt / 1e12,
                     "energies": e.cpu().tolist()}
        for g in graphs:
            g.close()
        del ms, states, e
        shared = wss = streams = None
        torch.cuda.empty_cache()
    same = (res["batched"]["energies"] == res["one_at_a_time"]["energies"]
            and res["graphs"]["energies"] == res["one_at_a_time"]["energies"])
    for r in res.values():
        r.pop("energies")
    base = res["one_at_a_time"]["mera_sweeps_per_s"]
    print(json.dumps({"case": "batch", "prec": args.prec, "n_meras": len(specs),
                      "chis": [c for _, c, _ in specs], "n_lanes": n_lanes, "steps": args.steps,
                      "warmup": args.warmup, "results": res,
                      "speedup": res["batched"]["mera_sweeps_per_s"] / base,
                      "speedup_graphs": res["graphs"]["mera_sweeps_per_s"] / base,
                      "identical_energies": same}), flush=True)


def run_precision(args):
    """Mixed precision against a reference mode (--ref-prec: FP64, or the
    fixed-point split mode OZ4 where FP64 sweeps take hours) on the same MERA
    (same seed, same sweep count):
    - ref:    S sweeps in the reference mode;
    - mixed:  S sweeps in the mixed mode;
    - polish: S - P mixed sweeps, then P sweeps in the reference mode.
    Each final state is evaluated in the reference mode (rho* by 60 power
    steps from its warm start, descent to the bottom layer, energy per spin);
    the mixed state is also evaluated in the mixed mode.  All contractions
    run in the library."""
    import numpy as np
    import torch

    import mera_inputs as I
    import paper_1906_12030_gb300 as m
    from paper_1906_12030_gb300 import scaling

    dev = torch.device("cuda", 0)
    chi, prec = args.chi, m.PRECS[args.prec]
    ref = m.PRECS[args.ref_prec]
    h1_host, shift = m.mera_ising_h1(HZ)
    h1 = torch.from_numpy(h1_host.reshape(-1)).to(dev)
    S, P = args.sweeps, min(args.polish, args.sweeps)

    def fresh():
        layers = I.init_mera(SEED, chi, z2=args.z2)
        us = [torch.from_numpy(u).to(dev).reshape(-1).contiguous() for u, _ in layers]
        ws_ = [torch.from_numpy(w).to(dev).contiguous() for _, w in layers]
        n3 = chi ** 3
        rho = (torch.eye(n3, dtype=torch.float64, device=dev) / n3).reshape(-1).contiguous()
        return m.MeraState(us, ws_, rho), us, ws_, rho

    def run(state, schedule):
        """Sweeps in the given precisions, each one a replay of a recorded
        sweep graph of that precision (same state tensors)."""
        stream = torch.cuda.Stream(dev)
        graphs, es = {}, {}
        for p in sorted(set(schedule)):
            es[p] = torch.empty(1, dtype=torch.float64, device=dev)
            wsp = m.workspace(m.mera_sweep_workspace_size(state.chi_b, state.chi_t, p), dev)
            graphs[p] = m.mera_sweep_graph(state, h1, shift, N_POW, es[p], prec=p, ws=wsp, stream=stream)
        hist = torch.empty(len(schedule), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i, p in enumerate(schedule):
                graphs[p].launch(stream)
                hist[i:i + 1].copy_(es[p])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if m.mera_device_status(clear=True) != 0:
            print("note: a recorded polar update reported non-convergence", flush=True)
        for g in graphs.values():
            g.close()
        return hist.cpu().tolist(), dt

    def evaluate(us, ws_, rho_star, p):
        """Energy per spin of a state, every map in mode p."""
        dims = I.layer_dims(chi)
        n = len(dims)
        rho = rho_star.clone()
        ws_fp = m.workspace(m.mera_workspace_size(m.OP_FIXED_POINT, chi, chi, p), dev)
        m.mera_fixed_point_rho(us[-1], ws_[-1], chi, rho, 60, prec=p, ws=ws_fp)
        for t in range(n - 2, 0, -1):  # rho* sits on top of layer n-2; descend to the top of layer 0
            cb, ct = dims[t]
            out = torch.empty(cb ** 6, dtype=torch.float64, device=dev)
            m.mera_descend(rho, us[t], ws_[t], cb, ct, out, prec=p)
            rho = out
        cb, ct = dims[0]
        e = torch.empty(1, dtype=torch.float64, device=dev)
        m.mera_energy(h1, rho, us[0], ws_[0], cb, ct, e, prec=p)
        return 0.5 * (float(e.item()) + shift)

    out = {"case": "precision", "chi": chi, "prec": args.prec, "sweeps": S, "polish_ref_sweeps": P, "z2": args.z2,
           "exact_infinite_chain": -4.0 / np.pi,
           "ref_mode": args.ref_prec}
    st, us, ws_, rho = fresh()
    hist_m, t_m = run(st, [prec] * S)
    out["mixed"] = {"sweep_energy_last": hist_m[-1], "sweep_energy_change_last10": hist_m[-1] - hist_m[-11]
                    if S > 10 else None, "seconds": t_m,
                    "energy_ref_eval": evaluate(us, ws_, rho, ref),
                    "energy_mixed_eval": evaluate(us, ws_, rho, prec)}
    out["mixed"]["dE_eval_mixed_vs_ref"] = abs(out["mixed"]["energy_mixed_eval"] - out["mixed"]["energy_ref_eval"])
    if args.scaling_k > 0:
        d64 = scaling.scaling_dimensions(us[-1], ws_[-1], chi, k=args.scaling_k, prec=ref, tol=1e-10)
        dmx = scaling.scaling_dimensions(us[-1], ws_[-1], chi, k=args.scaling_k, prec=prec, tol=1e-10)
        out["mixed"]["scaling_dims_ref"] = [float(x) for x in d64]
        out["mixed"]["scaling_dims_max_abs_err"] = float(np.max(np.abs(d64 - dmx)))
    if args.riemannian_eta > 0:
        st, us, ws_, rho = fresh()
        er = torch.empty(S, dtype=torch.float64, device=dev)
        wsr = m.workspace(m.mera_sweep_workspace_size(st.chi_b, st.chi_t, prec), dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(S):
            try:
                m.mera_sweep_riemannian(st, h1, shift, N_POW, args.riemannian_eta, er[i:i + 1], prec=prec, ws=wsr)
            except m.MeraNotConverged:
                pass
        torch.cuda.synchronize()
        hr = er.cpu().tolist()
        out["riemannian"] = {"eta": args.riemannian_eta, "sweep_energy_last": hr[-1],
                             "sweep_energy_at_quarter": hr[max(0, S // 4 - 1)],
                             "seconds": time.perf_counter() - t0,
                             "energy_ref_eval": evaluate(us, ws_, rho, ref)}
        out["mixed"]["sweep_energy_at_quarter"] = hist_m[max(0, S // 4 - 1)]
    if args.grow_from > 0:
        from paper_1906_12030_gb300 import grow

        layers0 = I.init_mera(SEED, args.grow_from, z2=args.z2)
        st0 = m.MeraState([torch.from_numpy(u).to(dev).reshape(-1).contiguous() for u, _ in layers0],
                          [torch.from_numpy(w).to(dev).contiguous() for _, w in layers0],
                          (torch.eye(args.grow_from ** 3, dtype=torch.float64, device=dev)
                           / args.grow_from ** 3).reshape(-1).contiguous())
        h0, t0 = run(st0, [prec] * args.grow_sweeps)
        stg = grow.grow_state(st0, I.layer_dims(chi), seed=SEED, eps=1e-4)
        hist_g, t_g = run(stg, [prec] * S)
        out["grown"] = {"from_chi": args.grow_from, "sweeps_before": args.grow_sweeps,
                        "energy_before_growth": h0[-1], "sweep_energy_last": hist_g[-1],
                        "seconds": t0 + t_g,
                        "energy_ref_eval": evaluate(stg.us, stg.ws, stg.rho_star, ref)}
    if P > 0:
        st, us, ws_, rho = fresh()
        hist_p, t_p = run(st, [prec] * (S - P) + [ref] * P)
        out["polish"] = {"sweep_energy_last": hist_p[-1], "seconds": t_p,
                         "energy_ref_eval": evaluate(us, ws_, rho, ref)}
    if args.fp64_steps > 0:
        st, us, ws_, rho = fresh()
        hist_r, t_r = run(st, [ref] * S)
        e_ref = evaluate(us, ws_, rho, ref)
        out["ref_run"] = {"sweep_energy_last": hist_r[-1], "sweep_energy_change_last10": hist_r[-1] - hist_r[-11]
                           if S > 10 else None, "seconds": t_r, "energy_ref_eval": e_ref}
        out["mixed"]["dE_vs_ref_run"] = abs(out["mixed"]["energy_ref_eval"] - e_ref)
        if P > 0:
            out["polish"]["dE_vs_ref_run"] = abs(out["polish"]["energy_ref_eval"] - e_ref)
    print(json.dumps(out), flush=True)


def run_spectrum(args):
    """Scaling dimensions of the Ising CFT (Sec. III A, Fig. 7) from a
    parity-symmetric MERA optimised up a ladder of bond dimensions: Z2 start
    at the first, sweeps in the chosen mode (recorded sweep graphs replayed),
    growth to the next with the parity kept (grow.grow_state(z2=True)), and
    so on.  The final state's energy per spin (rho* by 60 power steps from
    its warm start, descent, energy) and the 12 lowest scaling dimensions of
    its scale-invariant ascending map are evaluated with the fixed-point split
    mode OZ4."""
    import numpy as np
    import torch

    import mera_inputs as I
    import paper_1906_12030_gb300 as m
    from paper_1906_12030_gb300 import grow, scaling

    dev = torch.device("cuda", 0)
    prec = m.PRECS[args.prec]
    chis = [int(x) for x in args.spectrum_chis.split(",")]
    counts = [int(x) for x in args.spectrum_sweeps.split(",")]
    h1n, shift = m.mera_ising_h1(HZ)
    h1 = torch.from_numpy(h1n.reshape(-1)).to(dev)
    layers = I.init_mera(SEED, chis[0], z2=True)
    st = m.MeraState([torch.from_numpy(u).to(dev).reshape(-1).contiguous() for u, _ in layers],
                     [torch.from_numpy(w).to(dev).contiguous() for _, w in layers],
                     (torch.eye(chis[0] ** 3, dtype=torch.float64, device=dev) / chis[0] ** 3).reshape(-1))
    stages = []
    for i, (chi, n) in enumerate(zip(chis, counts)):
        if i > 0:
            st = grow.grow_state(st, I.layer_dims(chi), seed=SEED + i, eps=1e-4, z2=True,
                                 bottom_parity=I.parity_labels(4, physical=True))
        stream = torch.cuda.Stream(dev)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        wsb = m.workspace(m.mera_sweep_workspace_size(st.chi_b, st.chi_t, prec), dev)
        g = m.mera_sweep_graph(st, h1, shift, N_POW, e, prec=prec, ws=wsb, stream=stream)
        hist = torch.empty(max(1, n // 100), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(n):
                g.launch(stream)
                if (k + 1) % 100 == 0:
                    hist[(k + 1) // 100 - 1:(k + 1) // 100].copy_(e)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        g.close()
        del wsb
        torch.cuda.empty_cache()
        h = hist.cpu().tolist()
        stages.append({"chi": chi, "sweeps": n, "seconds": dt, "sweep_energy_last": h[-1],
                       "energy_every_100": h[:: max(1, len(h) // 20)]})
    status = m.mera_device_status(clear=True)
    chi = chis[-1]
    dims = I.layer_dims(chi)
    oz4 = m.PREC_OZ4
    rho = st.rho_star.clone()
    ws_fp = m.workspace(m.mera_workspace_size(m.OP_FIXED_POINT, chi, chi, oz4), dev)
    m.mera_fixed_point_rho(st.us[-1], st.ws[-1], chi, rho, 60, prec=oz4, ws=ws_fp)
    for t in range(len(dims) - 2, 0, -1):
        cb, ct = dims[t]
        out = torch.empty(cb ** 6, dtype=torch.float64, device=dev)
        m.mera_descend(rho, st.us[t], st.ws[t], cb, ct, out, prec=oz4)
        rho = out
    ee = torch.empty(1, dtype=torch.float64, device=dev)
    m.mera_energy(h1, rho, st.us[0], st.ws[0], dims[0][0], dims[0][1], ee, prec=oz4)
    energy = 0.5 * (float(ee.item()) + shift)
    exact = -4.0 / np.pi
    deltas = scaling.scaling_dimensions(st.us[-1], st.ws[-1], chi, k=12, prec=oz4, tol=1e-10)
    cft = [0.0, 0.125, 1.0, 1.125, 1.125]
    print(json.dumps({"case": "spectrum", "prec": args.prec, "stages": stages, "chi": chi,
                      "energy_per_spin_oz4": energy, "exact_infinite_chain": exact,
                      "relative_energy_error": (energy - exact) / abs(exact),
                      "scaling_dims_oz4": [float(x) for x in deltas],
                      "ising_cft_lowest": cft,
                      "abs_dev_lowest5": [float(abs(a - b)) for a, b in zip(deltas[:5], cft)],
                      "device_status": status}), flush=True)


def main():
    args = _args()
    if args.cpu_sample:
        _run_cpu_sample(args.cpu_sample)
        return
    if args.slice_gib is not None and args.impl == "native":
        import paper_1906_12030_gb300 as m
        m.mera_set_slice_bytes(int(args.slice_gib * 2**30))
    if args.case == "batch":
        run_batch(args)
        return
    if args.case == "precision":
        run_precision(args)
        return
    if args.case == "spectrum":
        run_spectrum(args)
        return
    if args.case != "sweep":
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
