"""Schedule autotuner: tile size, pair slots, sweep depth and the sweep
kernel's CTA size by timed trials.

The sweep schedule (tile_log2 c, paired high qubits hmax, gates per sweep)
decides how much codec work a circuit costs (sweeps per circuit, tiles per
item) while the FP64 gate arithmetic stays the same; the CTA size (128,
256 or 512 threads, each compiled for its own register budget) decides how
the work of an item spreads over warps and how many CTAs share an SM.  The
best choice depends on the qubit count and on the circuit's structure, so
it is picked by running a representative circuit under each candidate on
the GPU and timing it with the CUDA events the library records around its
sweep launches (wall time breaks ties and covers the rest of the flush).
Results are cached per (qubit count, circuit class, codec, bound).

A schedule changes where the state is compressed, hence the stored values
of lossy codecs; results under one schedule are still exact against the
oracle run with the same partition.
"""
from __future__ import annotations

import time

from . import qsim

# (tile_log2, hmax, depth, sweep threads): items of 2^(c + hmax) <= 4096 amplitudes
CANDIDATES = [(8, 4, 512, 256), (8, 4, 512, 128), (8, 4, 512, 512), (8, 4, 48, 256), (9, 3, 512, 256),
              (10, 2, 512, 256), (7, 4, 512, 256), (6, 4, 512, 256), (8, 4, 12, 256)]
THREADS = (128, 256, 512)


def full(schedule) -> tuple:
    """A schedule as (c, hmax, depth, threads); threads default to 256."""
    return tuple(schedule) if len(schedule) > 3 else tuple(schedule) + (256,)


def valid(n: int, c: int, hmax: int) -> bool:
    return 1 <= c <= min(10, n) and 1 <= hmax <= 4 and c + hmax <= 12


def time_schedule(n, gates, schedule, codec="rel", eps=1e-4, basis=0, reps=2, block_log2=20,
                  stream=None) -> float:
    """Seconds per circuit under one schedule: the median over reps (after
    one warm-up) of the sweeps' device time from CUDA events, plus a small
    share of the wall time of the flush (host planning and read-back)."""
    c, hmax, depth, threads = full(schedule)
    st = qsim.State(n, max(block_log2, c), codec, eps, stream=stream)
    st.set_schedule(c, min(hmax, max(1, n - c)) if n > c else 1, depth)
    st.set_sweep_threads(threads)
    times = []
    for rep in range(reps + 1):
        st.reset_basis(basis)
        st.set_profiling(True)
        t0 = time.perf_counter()
        st.apply_all(gates)
        st.flush()
        wall = time.perf_counter() - t0
        dev = st.profile()["sweep_ms"] / 1000.0
        if rep:
            times.append(dev + 0.1 * wall)
    st.close()
    times.sort()
    return times[len(times) // 2]


def tune(n, gates, codec="rel", eps=1e-4, basis=0, candidates=None, reps=2) -> dict:
    """Time every valid candidate; returns {"best": schedule, "table": [...]}."""
    table = []
    for sch in candidates or CANDIDATES:
        c, hmax, _, threads = full(sch)
        if not valid(n, c, min(hmax, max(1, n - c))) or threads not in THREADS:
            continue
        table.append((time_schedule(n, gates, sch, codec, eps, basis, reps), sch))
    table.sort()
    return {"best": table[0][1], "table": [{"schedule": s, "seconds": t} for t, s in table]}


class Tuner:
    """Cache of tuned schedules keyed by (n, circuit class, codec, bound)."""

    def __init__(self, candidates=None, reps=2):
        self.candidates = candidates
        self.reps = reps
        self.cache: dict = {}

    def schedule(self, n, cls, gates, codec="rel", eps=1e-4, basis=0):
        key = (n, cls, codec, eps)
        if key not in self.cache:
            self.cache[key] = tune(n, gates, codec, eps, basis, self.candidates, self.reps)["best"]
        return self.cache[key]
