#!/usr/bin/env python
"""Benchmark of the compressed simulator's hot path on GB300.

Workload (one step): the 28-qubit QFT (420 gates: H, controlled phases,
final swaps) on a seeded basis state, state stored as compressed tiles of
2^8 amplitudes (items of 16 tiles: up to four paired high qubits) in blocks of 2^20, point-wise relative bound 1e-4,
normalize on (Algorithm 2), sweeps of up to 512 fused gates.  A step is
reset to |x>, all 420 gates, flush (every sweep of decompress -> normalize
-> gates -> compress), i.e. one full circuit.

Prints one JSON line: gates/s (whole job), the sweep kernel's roofline
(FP64 pipe), the HBM fraction, fidelity against the uncompressed FP64 GPU
run and the closed form, compression ratios per bound, an end-to-end
number through the public API, clock samples, and the CPU oracle timed on
a bounded sample of the same workload.

Multi-GPU (torchrun): every rank runs an independent replica (its own
seeded basis state); there is no exchange step, so the scaling is weak.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates/s and HBM fraction at fixed fidelity; compression ratio; circuits/s + p99 latency"
N_QUBITS, BLOCK_LOG2, EPS = 28, 20, 1e-4
FP64_PEAK_TFLOPS = 1.25        # nominal dense FP64 of GB300 (no measured FP64 peak on this machine)
PROFILE_FILE = os.path.join(ROOT, "profiles", "sweep_kernel_qft28.md")
KERNEL_SRC = os.path.join(ROOT, "paper_1811_05140_gb300", "csrc", "kernels.cu")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 5; 1 for --workload grover, minutes per circuit)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--eps", type=float, default=EPS)
    ap.add_argument("--depth", type=int, default=512)
    ap.add_argument("--tile-log2", type=int, default=8, help="tile size (log2 amplitudes)")
    ap.add_argument("--pairs", type=int, default=4, help="paired high qubits per sweep")
    ap.add_argument("--sweep-threads", type=int, default=256, help="sweep kernel CTA size (128, 256, 512)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip bound sweep / AALC / e2e")
    ap.add_argument("--workload", choices=["qft28", "serving", "grover", "aalc"], default="qft28")
    ap.add_argument("--grover-n", type=int, default=36, help="grover: qubits")
    ap.add_argument("--iterations", type=int, default=8, help="grover: Grover iterations")
    ap.add_argument("--requests", type=int, default=2000, help="serving: circuits")
    ap.add_argument("--nmin", type=int, default=10, help="serving: smallest qubit count")
    ap.add_argument("--nmax", type=int, default=30, help="serving: largest qubit count")
    ap.add_argument("--rate-factor", type=float, default=1.5, help="serving: arrival rate / one-at-a-time capacity")
    ap.add_argument("--tune", action="store_true", help="serving: autotuned schedule per (n, class)")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 1 if args.workload == "grover" else 5
    return args


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def profile_figures():
    """Per-launch DRAM bytes and warp instructions of the sweep kernel from
    the committed ncu summary, when it was taken on the current kernel
    source: ({"traffic": bytes, "warp_inst": count}, note)."""
    try:
        text = open(PROFILE_FILE).read()
    except OSError:
        return {}, "no ncu summary"
    m = re.search(r"kernels\.cu sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"dram bytes per full-size launch:\s*([0-9.eE+]+)", text)
    w = re.search(r"warp instructions per full-size launch:\s*([0-9.eE+]+)", text)
    if not m or not t:
        return {}, "no per-launch figures in the ncu summary"
    cur = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    if cur != m.group(1):
        return {}, "kernel changed since the ncu capture"
    out = {"traffic": float(t.group(1))}
    if w:
        out["warp_inst"] = float(w.group(1))
    return out, None


ISSUE_PER_CLK = 4 * 152                     # warp instructions per clock: 4 schedulers x 152 SMs


def roofline_line(figs, per_launch_s, fp64_tflops, fp64_meas, traffic, hbm_gbs, hbm_peak, hbm_measured,
                  clocks):
    """Roofline of the sweep kernel.  The kernel is bound by instruction
    issue and latency (integer codec and gate loops, FP64 mostly idle), so
    the top-level figure is the issue rate: warp instructions per launch
    (the committed ncu count, while it matches the kernel source) over the
    live launch time, against one warp instruction per scheduler and clock
    at the maximum SM clock.  The executed FP64 work and the DRAM bytes
    give the two other rooflines beside it."""
    fp64 = {"achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": fp64_tflops / FP64_PEAK_TFLOPS, "counts": "FP64 instructions executed (FMA-slot flops)",
            "measured_peak": fp64_meas, "frac_of_measured": fp64_tflops / fp64_meas}
    hbm = {"achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak,
           "peak_source": "measured" if hbm_measured else "fallback"}
    line = {"kernel": "sweep_kernel", "per_launch_ms": per_launch_s * 1e3, "traffic": traffic,
            "fp64": fp64, "hbm": hbm}
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    if "warp_inst" in figs and per_launch_s > 0:
        peak = ISSUE_PER_CLK * mhz * 1e6 / 1e12
        ach = figs["warp_inst"] / per_launch_s / 1e12
        line.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": "Twarp-inst/s", "frac": ach / peak,
                     "counts": "warp instructions issued per launch (ncu summary) over the live launch time",
                     "peak_source": "4 schedulers x 152 SMs x max SM clock"})
    else:
        line.update({"bound": "alu", "achieved": fp64_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": fp64_tflops / FP64_PEAK_TFLOPS, "counts": "FP64 instructions executed",
                     "peak_source": "nominal FP64; FMA-slot flops"})
    return line


# ------------------------------------------------------------------ CPU oracle
def host_cores() -> int:
    """Cores this process may run on (the machine's host cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _expand_item(item, H, c):
    T = item
    for q in sorted(H):
        b = q - c
        T = ((T >> b) << (b + 1)) | (T & ((1 << b) - 1))
    return T


def _members(T, H, c):
    out = []
    for j in range(1 << len(H)):
        t = T
        for i, q in enumerate(sorted(H)):
            if (j >> i) & 1:
                t |= 1 << (q - c)
        out.append(t)
    return out


def oracle_sample(n, eps, depth, xval, items_per_sweep, seed=0, threads=1):
    """Time the oracle (Algorithm 2 over tiles, plain C) on a run of
    `items_per_sweep` consecutive tile groups, at a seeded offset, of every
    sweep of the QFT and extrapolate to the whole circuit by group count.
    threads == 1: the oracle's own sweep over those groups; threads > 1:
    the same groups' item sweeps (identical arithmetic) spread over
    `threads` host threads, inputs taken from the oracle's own state.
    Returns (gates/s, seconds timed, description, extrapolation factor)."""
    import oracle
    from paper_1811_05140_gb300 import inputs as I

    c = min(BLOCK_LOG2, n, 8)
    gates = I.qft(n)
    shifts = [oracle.shift_for_eps(eps)]
    cs = oracle.CSim(n, c, shifts, None, True)
    cs.reset_basis(xval)
    sweeps = oracle.partition(gates, n, c, 4, depth)
    rng = I.Rng(I.BASE_SEED + 3 + seed)
    est_total, spent, done, total_items = 0.0, 0.0, 0, 0
    for lo, hi, H in sweeps:
        nitems = 1 << (n - c - len(H))
        k = min(items_per_sweep, nitems)
        first = rng.below(nitems - k + 1)
        if threads == 1:
            t0 = time.perf_counter()
            cs.sweep_sample(gates[lo:hi], H, first, first + k)
            dt = time.perf_counter() - t0
        else:
            bases = [_expand_item(i, H, c) for i in range(first, first + k)]
            tiles = [t for T in bases for t in _members(T, H, c)]
            streams = [cs.stream(t) for t in tiles]
            raw = b"".join(streams)
            sizes = [len(x) for x in streams]
            alpha = cs.alpha
            t0 = time.perf_counter()
            res = oracle.item_sweep_batch(n, c, H, bases, raw, sizes, alpha, gates[lo:hi], shifts,
                                          None, threads)
            dt = time.perf_counter() - t0
            for t, x in zip(tiles, (x for item in res for x in item)):
                cs.set_stream(t, x)
        spent += dt
        done += k
        total_items += nitems
        est_total += dt * nitems / k
    how = "1 thread" if threads == 1 else f"{threads} threads over the groups"
    desc = (f"oracle (plain C, {how}) on {done} tile groups ({items_per_sweep} consecutive ones, or all, at a "
            f"seeded offset in each of the {len(sweeps)} sweeps) of the {n}-qubit QFT's {total_items}, "
            f"extrapolated by group count")
    return len(gates) / est_total, spent, desc, total_items / done


def oracle_items_for(n, eps, depth, xval, target_s, threads=1):
    """Tile groups per sweep for about target_s seconds of oracle work."""
    probe = 4 * threads
    _, probe_s, _, _ = oracle_sample(n, eps, depth, xval, probe, threads=threads)
    return max(probe, min(1 << 14, int(probe * target_s / max(probe_s, 1e-3))))


def cpu_baselines(n, eps, depth, xval, target_s):
    """The oracle on one thread and on every host core, each a bounded sample."""
    cores = host_cores()
    out = {}
    for threads in sorted({1, cores}):
        items = oracle_items_for(n, eps, depth, xval, target_s, threads)
        v, spent, desc, factor = oracle_sample(n, eps, depth, xval, items, threads=threads)
        out[threads] = {"value": v, "unit": "gates/s", "cores": threads, "kind": "oracle", "sample": desc,
                        "seconds": round(spent, 2), "extrapolation_factor": round(factor, 1)}
    best = out[cores]
    line = dict(best)
    line["host_cores"] = cores
    line["one_thread"] = {k: out[1][k] for k in ("value", "seconds", "sample", "extrapolation_factor")}
    return line


# ------------------------------------------------------------------ ranks
def replica_seed(rank: int) -> int:
    """Seed of rank's replica: every rank simulates its own basis state."""
    from paper_1811_05140_gb300 import inputs as I
    return I.BASE_SEED + rank


def max_over_ranks(ms: float, world: int, device: str) -> float:
    """The slowest rank's time (the timed region ends when every rank has)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, gates: int, steps: int, ms_max: float) -> float:
    """Whole-job gates/s: every rank's gates over the slowest rank's time."""
    return world * gates * steps / (ms_max / 1000.0)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1811_05140_gb300 import build as B
    from paper_1811_05140_gb300 import inputs as I
    from paper_1811_05140_gb300 import qsim

    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.set_device(local_rank)
    n, eps = args.n, args.eps
    c = min(BLOCK_LOG2, n, 8)
    xval = I.seeded_basis(n, replica_seed(rank))
    gates = I.qft(n)
    stream = torch.cuda.Stream()
    st = qsim.State(n, BLOCK_LOG2, "rel", eps, stream=stream)
    c = min(args.tile_log2, n)
    if args.depth != 512 or c != 8 or args.pairs != 4:
        st.set_schedule(c, args.pairs, args.depth)
    if args.sweep_threads != 256:
        st.set_sweep_threads(args.sweep_threads)

    def step():
        st.reset_basis(xval)
        st.apply_all(gates)
        st.flush()

    for _ in range(max(3, args.warmup)):
        step()
    st.set_profiling(True)
    launches0 = st.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    ms = ev0.elapsed_time(ev1)
    prof = st.profile()
    launches = st.stats()["kernel_launches"] - launches0
    stats = st.stats()
    ms_max = max_over_ranks(ms, world, "cuda")
    result = {
        "ms": ms_max, "prof": prof, "launches": launches, "stats": stats,
        "clocks": clk.summary(), "xval": xval,
        "fp64_tflops": 2.0 * qsim.fp64_rate(local_rank) / 1e12,     # FMA-slot TFLOP/s, measured
    }
    if rank != 0:
        return None
    # quality and ratios (untimed)
    raw = 16.0 * (1 << n)
    sb, fp = st.compressed_bytes()
    ref = qsim.State(n, BLOCK_LOG2, "none", 0.0, stream=stream)
    if c != 8 or args.pairs != 4:
        ref.set_schedule(c, args.pairs, 512)               # same tiles: fidelity is taken tile by tile
    ref.reset_basis(xval)
    ref.apply_all(gates)
    ref.flush()
    F_ref = st.fidelity_state(ref)
    F_cf = st.fidelity_qft(xval)
    result.update(F_ref=F_ref, F_cf=F_cf, ratio_final=raw / sb,
                  ratio_min=raw / max(1, stats["max_stream_bytes_seen"]), footprint=fp)
    if not args.no_extras:
        per_bound = []
        for e in (1e-2, 1e-3, 1e-4, 1e-5):
            s2 = qsim.State(n, BLOCK_LOG2, "rel", e, stream=stream)
            s2.reset_basis(xval)
            t0 = time.perf_counter()
            s2.apply_all(gates)
            s2.flush()
            dt = time.perf_counter() - t0
            b2, _ = s2.compressed_bytes()
            st2 = s2.stats()
            per_bound.append({"eps": e, "fidelity_vs_fp64": round(s2.fidelity_state(ref), 9),
                              "ratio_final": round(raw / b2, 3),
                              "ratio_min": round(raw / max(1, st2["max_stream_bytes_seen"]), 3),
                              "gates_per_s": round(len(gates) / dt, 1)})
            s2.close()
        result["per_bound"] = per_bound
        per_bound_polar = []
        for e in (1e-2, 1e-3, 1e-4, 1e-5):                # the POLAR variant (magnitude + phase)
            s2 = qsim.State(n, BLOCK_LOG2, "rel", e, stream=stream)
            s2.set_polar(True)
            s2.reset_basis(xval)
            t0 = time.perf_counter()
            s2.apply_all(gates)
            s2.flush()
            dt = time.perf_counter() - t0
            b2, _ = s2.compressed_bytes()
            st2 = s2.stats()
            per_bound_polar.append({"eps": e, "fidelity_vs_fp64": round(s2.fidelity_state(ref), 9),
                                    "ratio_final": round(raw / b2, 3),
                                    "ratio_min": round(raw / max(1, st2["max_stream_bytes_seen"]), 3),
                                    "gates_per_s": round(len(gates) / dt, 1)})
            s2.close()
        result["per_bound_polar"] = per_bound_polar
        s3 = qsim.State(n, BLOCK_LOG2, "aalc", 1e-2, stream=stream)
        s3.set_aalc(16.0, [1e-5, 1e-4, 1e-3, 1e-2])
        s3.reset_basis(xval)
        s3.apply_all(gates)
        s3.flush()
        b3, _ = s3.compressed_bytes()
        st3 = s3.stats()
        result["aalc_theta16"] = {"fidelity_vs_fp64": round(s3.fidelity_state(ref), 9),
                                  "ratio_final": round(raw / b3, 3),
                                  "ratio_min": round(raw / max(1, st3["max_stream_bytes_seen"]), 3),
                                  "level_hist": st3["level_hist"][:5]}
        s3.close()
        s4 = qsim.State(n, BLOCK_LOG2, "aalc", 1e-2, stream=stream)
        s4.set_aalc(16.0, [1e-5, 1e-4, 1e-3, 1e-2])
        s4.set_polar(True)
        s4.reset_basis(xval)
        s4.apply_all(gates)
        s4.flush()
        b4, _ = s4.compressed_bytes()
        st4 = s4.stats()
        result["aalc_theta16_polar"] = {"fidelity_vs_fp64": round(s4.fidelity_state(ref), 9),
                                        "ratio_final": round(raw / b4, 3),
                                        "ratio_min": round(raw / max(1, st4["max_stream_bytes_seen"]), 3),
                                        "tiles_over_limit": st4["tiles_over_limit"],
                                        "level_hist": st4["level_hist"][:5]}
        s4.close()
        # end to end through the public API: host gate list in, host result out
        qs = [0, n // 2, n - 1]
        st.reset_basis(xval)
        torch.cuda.synchronize()
        s0 = st.stats()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st.reset_basis(xval)
            st.apply_all(gates)
            st.probabilities(qs)
        t1 = time.perf_counter()
        s1 = st.stats()
        result["e2e_s"] = (t1 - t0) / args.steps
        # bytes the library copied between host and device (its own counters)
        result["e2e_h2d"] = (s1["h2d_bytes"] - s0["h2d_bytes"]) // args.steps
        result["e2e_d2h"] = (s1["d2h_bytes"] - s0["d2h_bytes"]) // args.steps
    ref.close()
    return result


# ------------------------------------------------------------------ Grover search
def run_grover(args):
    """Grover search on n qubits (default 36: 1 TiB as complex128), one
    seeded marked item, oracle = multi-controlled Z on its pattern,
    diffusion = H^n X^n MCZ X^n H^n, 8 iterations, blocks of 2^22,
    relative bound 1e-4.  A step is reset to |0...0>, every gate, flush.
    Warm-up runs one iteration per step (the arenas reach their size);
    the state never exists uncompressed anywhere."""
    import math

    import numpy as np
    import torch

    from paper_1811_05140_gb300 import build as B
    from paper_1811_05140_gb300 import inputs as I
    from paper_1811_05140_gb300 import qsim

    B.build()
    torch.cuda.set_device(0)
    n, iters, eps = args.grover_n, args.iterations, 1e-4
    marked = I.seeded_basis(n, I.BASE_SEED)
    gates = I.grover(n, marked, iters)
    warm = I.grover(n, marked, 1)
    stream = torch.cuda.Stream()
    st = qsim.State(n, 22, "rel", eps, stream=stream)
    for _ in range(max(3, args.warmup)):
        st.reset_basis(0)
        st.apply_all(warm)
        st.flush()
    torch.cuda.synchronize()
    st.set_profiling(True)
    launches0 = st.stats()["kernel_launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            st.reset_basis(0)
            st.apply_all(gates)
            st.flush()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof = st.profile()
    stats = st.stats()
    launches = stats["kernel_launches"] - launches0
    sb, fp = st.compressed_bytes()
    free, total = torch.cuda.mem_get_info()
    F = st.fidelity_grover(marked, iters)
    th = math.asin(1.0 / math.sqrt(2.0 ** n))
    sgn = -1.0 if iters % 2 else 1.0
    want_m = sgn * math.sin((2 * iters + 1) * th)
    want_o = sgn * math.cos((2 * iters + 1) * th) / math.sqrt(2.0 ** n - 1.0)
    rng = I.Rng(I.BASE_SEED + 77)
    others = [o for o in (rng.below(1 << n) for _ in range(64)) if o != marked]
    got_m = st.amplitudes(marked, 1)[0]
    got_o = np.array([st.amplitudes(o, 1)[0] for o in others])
    err_m = abs(got_m - want_m) / abs(want_m)
    err_o = float(np.max(np.abs(got_o - want_o)) / abs(want_o))
    sweep_s = prof["sweep_ms"] / 1000.0
    tflops = 2.0 * prof["dp_ops"] / sweep_s / 1e12 if sweep_s > 0 else 0.0
    hbm_gbs = prof["bytes"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    raw = 16.0 * 2.0 ** n
    value = len(gates) * args.steps / (ms / 1000.0)
    fp64_meas = 2.0 * qsim.fp64_rate(0) / 1e12
    line = {
        "metric": "gates/s (Grover search, state held compressed)", "value": value, "unit": "gates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"grover{n}_it{iters}_rel{eps:g}", "n_qubits": n, "iterations": iters,
                   "marked": marked, "block_log2": 22, "tile_log2": stats["tile_log2"], "pair_slots": stats["hmax"],
                   "gates": len(gates), "rel_err_bound": eps, "normalize": True,
                   "warmup_steps": "one Grover iteration each",
                   "l2": "inputs larger than L2 (compressed state > 129 MB), no flush"},
        "fidelity_vs_closed_form": F,
        "amplitude_rel_err": {"marked": err_m, "max_of_sampled_others": err_o, "sampled": len(others)},
        "stream_bytes_final": sb, "footprint_bytes": fp, "uncompressed_bytes": raw,
        "compression_ratio_final": raw / sb,
        "compression_ratio_min": raw / max(1, stats["max_stream_bytes_seen"]),
        "footprint_ratio": raw / fp,
        "device_bytes_in_use": total - free,
        "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "sweep_kernel",
                     "fp64_measured_tflops": fp64_meas, "frac_of_measured_fp64": tflops / fp64_meas,
                     "sweep_launches": prof["sweep_launches"],
                     "peak_source": "nominal FP64 (no measured FP64 peak); FMA-slot flops",
                     "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    st.close()
    print(json.dumps(line))


# ------------------------------------------------------------------ AALC threshold sweep
def run_aalc(args):
    """The 26-qubit QFT (the paper's size) under the error-bound ladder
    {lossless, 1e-5, 1e-4, 1e-3, 1e-2} with thresholds 4, 8, 16, 32 and 64
    decided per tile, with thresholds 4, 8, 16 and 32 decided per stride of
    2^20 amplitudes (Algorithm 2), with the POLAR variant on every lossy
    level, and under fixed bounds: fidelity against the uncompressed FP64
    run, minimum and final compression ratio, level histogram, tiles that
    met no level's size limit (over every sweep), gates/s."""
    import torch

    from paper_1811_05140_gb300 import build as B
    from paper_1811_05140_gb300 import inputs as I
    from paper_1811_05140_gb300 import qsim

    B.build()
    torch.cuda.set_device(0)
    n = 26
    x = I.seeded_basis(n, I.BASE_SEED)
    gates = I.qft(n)
    raw = 16.0 * 2.0 ** n
    ref = qsim.State(n, 20, "none", 0.0)
    ref.reset_basis(x)
    ref.apply_all(gates)
    ref.flush()
    ladder = [1e-5, 1e-4, 1e-3, 1e-2]
    rows = []

    def one(label, make):
        st = make()
        st.reset_basis(x)
        st.apply_all(gates)
        st.flush()                                    # warm
        st.reset_basis(x)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.apply_all(gates)
        st.flush()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        stats = st.stats()
        rows.append({"setting": label, "fidelity_vs_fp64": st.fidelity_state(ref),
                     "ratio_final": raw / st.compressed_bytes()[0],
                     "ratio_min": raw / max(1, stats["max_stream_bytes_seen"]),
                     "level_hist": stats["level_hist"][:len(ladder) + 1],
                     "tiles_over_limit": stats["tiles_over_limit"],
                     "tiles_written": sum(stats["level_hist"]), "gates_per_s": len(gates) / dt})
        st.close()

    for theta in (4.0, 8.0, 16.0, 32.0, 64.0):
        def make(theta=theta):
            st = qsim.State(n, 20, "aalc", ladder[-1])
            st.set_aalc(theta, ladder)
            return st
        one(f"aalc theta={theta:g}", make)
    for theta in (4.0, 8.0, 16.0, 32.0):
        def make(theta=theta):                        # Algorithm 2's decision per stride of 2^20
            st = qsim.State(n, 20, "aalc", ladder[-1])
            st.set_aalc(theta, ladder)
            st.set_aalc_unit(20)
            return st
        one(f"aalc per stride theta={theta:g}", make)
    for theta in (4.0, 8.0, 16.0, 32.0, 64.0):
        def make(theta=theta):                        # the POLAR variant on every lossy level
            st = qsim.State(n, 20, "aalc", ladder[-1])
            st.set_aalc(theta, ladder)
            st.set_polar(True)
            return st
        one(f"aalc polar theta={theta:g}", make)
    for eps in (1e-2, 1e-3, 1e-4):
        one(f"fixed rel {eps:g}", lambda eps=eps: qsim.State(n, 20, "rel", eps))
    for eps in (1e-3, 1e-4):
        def make(eps=eps):
            st = qsim.State(n, 20, "rel", eps)
            st.set_polar(True)
            return st
        one(f"fixed rel {eps:g} polar", make)
    ref.close()
    print(json.dumps({"metric": "fidelity and compression ratio per threshold (QFT-26)", "unit": "table",
                      "config": {"workload": "qft26_aalc_thresholds", "ladder": [0.0] + ladder,
                                 "tile_log2": 8, "block_log2": 20},
                      "rows": rows}))


# ------------------------------------------------------------------ serving mix
def serving_requests(count, nmin, nmax, seed):
    """The serving mix: 40% QFT on a random basis state, 30% Grover (2-6
    iterations), 30% random grid (depth 8-20); n uniform in [nmin, nmax];
    relative bound 1e-3 or 1e-4; three read-out qubits."""
    from paper_1811_05140_gb300 import inputs as I
    rng = I.Rng(seed)
    reqs = []
    cache = {}
    for _ in range(count):
        n = nmin + rng.below(nmax - nmin + 1)
        u = rng.below(10)
        eps = (1e-3, 1e-4)[rng.below(2)]
        if u < 4:
            cls = "qft"
            if ("qft", n) not in cache:
                cache[("qft", n)] = I.qft(n)
            gates, x = cache[("qft", n)], rng.below(1 << n)
        elif u < 7:
            cls = "grover"
            gates, x = I.grover(n, rng.below(1 << n), 2 + rng.below(5)), 0
        else:
            cls = "grid"
            r, c = I.grid_shape(n)
            gates, x = I.random_grid(r, c, 8 + rng.below(13), rng.next()), 0
        readout = list(dict.fromkeys(rng.below(n) for _ in range(3)))
        reqs.append({"n": n, "cls": cls, "gates": gates, "x": x, "eps": eps, "readout": readout})
    return reqs


def run_serving(args):
    """The serving mix, every request run one at a time and through the
    serving loop on the same circuits and bounds (saturated: everything
    queued at once), with the library's default schedules and, with --tune,
    with autotuned ones; then Poisson arrivals at rate_factor times the
    one-at-a-time capacity."""
    import numpy as np
    import torch

    from paper_1811_05140_gb300 import build as B
    from paper_1811_05140_gb300 import inputs as I
    from paper_1811_05140_gb300 import qsim

    B.build()
    torch.cuda.set_device(0)
    reqs = serving_requests(args.requests, args.nmin, args.nmax, I.BASE_SEED + 5)
    tuned = None
    tune_s = 0.0
    if args.tune:
        # one tuned schedule per (qubit count, circuit class), timed on the
        # first request of that key at bound 1e-4; large circuits try the
        # shapes that differ in CTA size, tile size and pair slots only
        from paper_1811_05140_gb300 import autotune
        big = [(8, 4, 512, 256), (8, 4, 512, 128), (7, 4, 512, 256), (9, 3, 512, 256)]
        small = autotune.Tuner(reps=1)
        large = autotune.Tuner(candidates=big, reps=1)
        tuned = {}
        t0 = time.perf_counter()
        for q in reqs:
            key = (q["n"], q["cls"])
            if key not in tuned:
                tu = large if q["n"] >= 25 else small
                tuned[key] = tu.schedule(q["n"], q["cls"], q["gates"], "rel", 1e-4, q["x"])
        tune_s = time.perf_counter() - t0

    def sched_of(q, schedules):
        return schedules.get((q["n"], q["cls"])) if schedules else None

    def one_at_a_time(schedules):
        probs = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for q in reqs:
            st = qsim.State(q["n"], 8, "rel", q["eps"])
            sc = sched_of(q, schedules)
            if sc:
                st.set_schedule(*sc[:3])
                if len(sc) > 3:
                    st.set_sweep_threads(sc[3])
            st.reset_basis(q["x"])
            st.apply_all(q["gates"])
            probs.append(st.probabilities(q["readout"]))
            st.close()
        secs = time.perf_counter() - t0
        return {"cps": len(reqs) / secs, "seconds": secs}, probs

    free, total = torch.cuda.mem_get_info()
    budget = int(free * 0.8)

    def serve(arrival_rate, schedules, want):
        srv = qsim.Server(budget, max_resident=64, sweeps_per_tick=2)
        rng = I.Rng(I.BASE_SEED + 9)
        tickets = []
        t_start = time.perf_counter()
        next_t = 0.0
        for q in reqs:
            if arrival_rate:
                next_t += -np.log(1.0 - rng.uniform()) / arrival_rate
                dt = next_t - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
            tickets.append(srv.submit(q["n"], q["gates"], eps=q["eps"], basis=q["x"], readout=q["readout"],
                                      schedule=sched_of(q, schedules)))
        srv.drain(36000)
        st = srv.stats()
        same = all(np.array_equal(srv.result(t)[1], p) for t, p in zip(tickets, want))
        srv.close()
        out = {"cps": st["throughput_cps"], "p50_s": st["p50_latency_s"], "p99_s": st["p99_latency_s"],
               "mean_s": st["mean_latency_s"], "peak_footprint": st["peak_footprint"],
               "max_resident": st["max_resident_seen"], "ticks": st["ticks"], "completed": st["completed"],
               "failed": st["failed"], "same_as_alone": same}
        if arrival_rate:
            out["rate_cps"] = arrival_rate
        return out

    alone_def, probs_def = one_at_a_time(None)
    sat_def = serve(0.0, None, probs_def)
    result = {"default": {"one_at_a_time": alone_def, "batched": sat_def,
                          "speedup": sat_def["cps"] / alone_def["cps"]}}
    best = sat_def
    if tuned is not None:
        alone_tun, probs_tun = one_at_a_time(tuned)
        sat_tun = serve(0.0, tuned, probs_tun)
        result["tuned"] = {"one_at_a_time": alone_tun, "batched": sat_tun,
                           "speedup": sat_tun["cps"] / alone_tun["cps"],
                           "tuning_seconds": tune_s,
                           "schedules_not_default": sum(1 for v in tuned.values()
                                                        if tuple(v) != (8, 4, 512, 256)),
                           "keys": len(tuned)}
        if sat_tun["cps"] > best["cps"]:
            best = sat_tun
        lam = args.rate_factor * alone_tun["cps"]
        poi = serve(lam, tuned, probs_tun)
    else:
        lam = args.rate_factor * alone_def["cps"]
        poi = serve(lam, None, probs_def)
    raw = sum(16 << q["n"] for q in reqs)
    line = {
        "metric": "circuits/s + p99 latency (serving mix)", "value": best["cps"],
        "unit": "circuits/s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serving_mix", "requests": len(reqs), "n_range": [args.nmin, args.nmax],
                   "mix": "40% QFT / 30% Grover 2-6 it / 30% random grid depth 8-20",
                   "bounds": [1e-3, 1e-4], "tuned_schedules": tuned is not None,
                   "budget_bytes": budget, "admission": "reservation = max(measured footprint, growth bound)"},
        "modes": result,
        "poisson": poi,
        "uncompressed_bytes_all_circuits": raw,
    }
    print(json.dumps(line))


def run_reference(args):
    """The oracle as the reference arm, on every host core: each step runs a
    bounded sample of the workload (consecutive tile groups of every sweep)
    and is timed as it runs; value extrapolates the sample to the whole
    circuit by group count (the factor is printed)."""
    from paper_1811_05140_gb300 import inputs as I
    import oracle
    oracle.build()
    cores = host_cores()
    xval = I.seeded_basis(args.n, I.BASE_SEED)
    items = oracle_items_for(args.n, args.eps, args.depth, xval, 4.0, cores)     # about 4 s per step
    vals, secs = [], []
    desc, factor = "", 1.0
    for i in range(args.warmup + args.steps):
        v, spent, desc, factor = oracle_sample(args.n, args.eps, args.depth, xval, items, seed=i,
                                               threads=cores)
        if i >= args.warmup:
            vals.append(v)
            secs.append(spent)
    v = statistics.median(vals)
    ms = 1000.0 * statistics.median(secs)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "gates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"qft{args.n}_rel{args.eps:g}", "n_qubits": args.n,
                   "block_log2": BLOCK_LOG2, "rel_err_bound": args.eps, "gates": 420},
        "step": ("one step = the sampled tile groups of every sweep, timed on the host; value = "
                 "gates of the whole circuit / (step time x extrapolation_factor)"),
        "extrapolation_factor": round(factor, 1),
        "cpu_baseline": {"value": v, "unit": "gates/s", "cores": cores, "kind": "oracle",
                         "sample": desc, "host_cores": cores},
        "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.workload == "serving":
        if rank == 0:
            run_serving(args)
        return
    if args.workload == "grover":
        if rank == 0:
            run_grover(args)
        return
    if args.workload == "aalc":
        if rank == 0:
            run_aalc(args)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        n = args.n
        ng = 420 if n == 28 else len(__import__("paper_1811_05140_gb300.inputs", fromlist=["qft"]).qft(n))
        ms_step = res["ms"] / args.steps
        value = job_rate(world, ng, args.steps, res["ms"])
        prof = res["prof"]
        sweep_s = prof["sweep_ms"] / 1000.0
        launches = max(1, prof["sweep_launches"])
        per_launch_s = sweep_s / launches
        achieved_tflops = 2.0 * prof["dp_ops"] / sweep_s / 1e12 if sweep_s > 0 else 0.0
        hbm_gbs = prof["bytes"] / sweep_s / 1e9 if sweep_s > 0 else 0.0
        peaks = measured_peaks()
        hbm_peak = peaks.get("hbm_gbs", 6800.0)
        figs, why = profile_figures()
        traffic = figs.get("traffic")
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            # each sample sized for about 8 s of CPU work (1 thread, all cores)
            cpu = cpu_baselines(n, args.eps, args.depth, res["xval"], 8.0)
        line = {
            "metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"qft{n}_rel{args.eps:g}", "n_qubits": n,
                       "block_log2": BLOCK_LOG2, "tile_log2": min(args.tile_log2, n), "pair_slots": args.pairs,
                       "sweep_threads": args.sweep_threads, "rel_err_bound": args.eps,
                       "gates": ng, "sweep_depth": args.depth, "normalize": True,
                       "l2": "inputs larger than L2 (compressed state > 129 MB), no flush",
                       "parallelism": f"replicas x{world}"},
            "fidelity_vs_fp64_gpu": res["F_ref"], "fidelity_vs_closed_form": res["F_cf"],
            "compression_ratio_final": res["ratio_final"], "compression_ratio_min": res["ratio_min"],
            # device bytes the state holds (both arenas, tables, norm partials) against 16 B per amplitude
            "footprint_bytes": res["footprint"], "footprint_ratio": 16.0 * 2.0 ** n / res["footprint"],
            "hbm_frac": hbm_gbs / hbm_peak,
            # every sweep reads and writes the whole logical state (16 B per amplitude each way)
            "logical_gbs": 32.0 * 2.0 ** n * launches / sweep_s / 1e9 if sweep_s > 0 else None,
            "roofline": roofline_line(figs, per_launch_s, achieved_tflops, res["fp64_tflops"], traffic,
                                      hbm_gbs, hbm_peak, "hbm_gbs" in peaks, res["clocks"]),
            "gpu_launches": res["launches"],
            "clocks": res["clocks"],
        }
        if why:
            line["roofline"]["traffic_note"] = why
        if cpu:
            line["cpu_baseline"] = cpu
        if "e2e_s" in res:
            line["e2e"] = {"value": ng / res["e2e_s"], "unit": "gates/s",
                           "h2d_bytes_per_step": res["e2e_h2d"], "d2h_bytes_per_step": res["e2e_d2h"]}
            line["per_bound"] = res["per_bound"]
            line["per_bound_polar"] = res["per_bound_polar"]
            line["aalc_theta16"] = res["aalc_theta16"]
            line["aalc_theta16_polar"] = res["aalc_theta16_polar"]
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
