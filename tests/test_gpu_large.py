"""Full-size cases in the benchmark's launch configuration, checked on
sampled outputs the oracle can compute one by one.

Every sweep of each circuit is checked: 4096 items (tile groups) per sweep,
drawn at random (seeded) plus the items that hold chosen amplitudes, are
re-run by the oracle from the GPU's own input streams and the same
normalize scale (threaded over the host cores), and the GPU's output
streams must be byte-identical.

* 28-qubit QFT, relative bound 1e-4 (2^28 amplitudes, 4 GiB uncompressed):
  then the final state's fidelity to the closed form must be >= 0.9995
  (the paper's QFT target).
* 30-qubit random grid (5 x 6, depth 20) with the error-bound ladder
  {lossless, 1e-5, 1e-4, 1e-3}, theta = 4: the ladder must mix lossless
  and lossy levels; fidelity against the uncompressed FP64 GPU run.
* 36-qubit Grover search (1 TiB uncompressed, blocks of 2^22, relative
  bound 1e-4), one iteration: every sweep kind (Hadamards on uniform
  tiles, the oracle's multi-controlled Z, X layers that only move tiles,
  spike tiles of the diffusion); then the marked amplitude and sampled
  others against sin((2k+1)theta) and cos((2k+1)theta)/sqrt(N-1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu

PER_SWEEP = 4096


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()
    oracle.build()


def expand(item, H, c):
    T = item
    for q in sorted(H):
        b = q - c
        low = T & ((1 << b) - 1)
        T = ((T >> b) << (b + 1)) | low
    return T


def members(T, H, c):
    out = []
    for j in range(1 << len(H)):
        t = T
        for i, q in enumerate(sorted(H)):
            if (j >> i) & 1:
                t |= 1 << (q - c)
        out.append(t)
    return out


def base_of(x, H, c):
    """First tile of the item that holds amplitude x."""
    T = x >> c
    for q in H:
        T &= ~(1 << (q - c))
    return T


def run_with_samples(st, n, gates, shifts, max_bytes, per_sweep, seed, extra_amps=()):
    """Apply gates sweep by sweep (the library's own partition); in every
    sweep re-run per_sweep random items plus the items holding extra_amps
    in the oracle and compare the streams.  Returns (items, sweeps)."""
    s = st.stats()
    c, hmax, depth = s["tile_log2"], s["hmax"], s["depth"]
    plan = qsim.plan_sweeps(n, c, hmax, depth, gates)
    rng = np.random.default_rng(seed)
    checked = 0
    for k, (lo, hi, H) in enumerate(plan):
        alpha = st.stats()["alpha"]
        nitems = 1 << (n - c - len(H))
        items = rng.choice(nitems, min(per_sweep, nitems), replace=False)
        bases = sorted({expand(int(i), H, c) for i in items} | {base_of(x, H, c) for x in extra_amps})
        tiles = [t for T in bases for t in members(T, H, c)]
        raw, sizes = st.export_tile_set_raw(tiles)
        st.apply_all(gates[lo:hi])
        st.flush()
        after = st.export_tile_set(tiles)
        want = oracle.item_sweep_batch(n, c, H, bases, raw, sizes, alpha, gates[lo:hi], shifts, max_bytes)
        flat = [x for item in want for x in item]
        bad = [i for i in range(len(tiles)) if after[i] != flat[i]]
        assert not bad, (k, [tiles[i] for i in bad[:8]], len(bad))
        checked += len(bases)
    return checked, len(plan)


def test_qft28_sampled_items_and_fidelity():
    n, eps = 28, 1e-4
    x = I.seeded_basis(n)
    st = qsim.State(n, 20, "rel", eps)
    st.reset_basis(x)
    checked, nsw = run_with_samples(st, n, I.qft(n), [oracle.shift_for_eps(eps)], None, PER_SWEEP, 28,
                                    extra_amps=(x, 0, (1 << n) - 1))
    assert nsw == 10 and checked >= PER_SWEEP * nsw
    assert st.fidelity_qft(x) >= 0.9995
    p = st.probabilities([0, 13, 27])
    assert abs(p.sum() - 1.0) < 1e-12


def test_grid30_aalc_sampled_items_levels_and_fidelity():
    rows, cols = 5, 6
    n = rows * cols
    gates = I.random_grid(rows, cols, 20, I.BASE_SEED)
    levels = [1e-5, 1e-4, 1e-3]
    st = qsim.State(n, 20, "aalc", 1e-3)
    st.set_aalc(4.0, levels)
    c = st.stats()["tile_log2"]
    shifts = [0] + [oracle.shift_for_eps(e) for e in levels]
    checked, nsw = run_with_samples(st, n, gates, shifts, oracle.max_bytes_for(c, 4.0), PER_SWEEP, 30)
    assert checked >= PER_SWEEP * nsw
    hist = st.stats()["level_hist"]
    assert hist[0] > 0 and sum(hist[1:4]) > 0          # lossless and lossy levels both used
    ref = qsim.State(n, 20, "none", 0.0)
    ref.apply_all(gates)
    ref.flush()
    F = st.fidelity_state(ref)
    ref.close()
    assert F > 0.99


def grover_checks(st, n, marked, it, rng, count, eps=1e-4):
    # each stored component is within eps of its exact value after the last
    # sweep; the earlier sweeps' errors, carried through the gates and the
    # normalize scale, are allowed as much again (marked) or three times
    # (the others, smaller and mixed by every Hadamard layer)
    th = math.asin(2.0 ** (-n / 2))
    sg = -1.0 if it & 1 else 1.0
    want_m = sg * math.sin((2 * it + 1) * th)
    want_o = sg * math.cos((2 * it + 1) * th) / math.sqrt(2.0 ** n - 1)
    got = st.amplitudes(marked, 1)[0]
    assert abs(got.real - want_m) <= 2 * eps * abs(want_m) and got.imag == 0.0
    others = [int(v) for v in rng.integers(0, 1 << n, count, dtype=np.uint64) if int(v) != marked]
    for xo in others + [0, (1 << n) - 1]:
        if xo == marked:
            continue
        a = st.amplitudes(xo, 1)[0]
        assert abs(a.real - want_o) <= 4 * eps * abs(want_o) and a.imag == 0.0, xo


def test_grover30_sampled_items_every_sweep_kind():
    # Grover at 30 qubits, two iterations, relative bound 1e-4
    n, it, eps = 30, 2, 1e-4
    marked = I.seeded_basis(n, 77)
    gates = I.grover(n, marked, it)
    st = qsim.State(n, 22, "rel", eps)
    st.reset_basis(0)
    checked, nsw = run_with_samples(st, n, gates, [oracle.shift_for_eps(eps)], None, 1024, 31,
                                    extra_amps=(marked, 0, (1 << n) - 1))
    assert checked >= 1024 * nsw
    assert st.fidelity_grover(marked, it) > 1 - 1e-9
    grover_checks(st, n, marked, it, np.random.default_rng(5), 16)


def test_grover36_sampled_items_and_closed_form():
    # the 36-qubit configuration itself (1 TiB as complex128, never
    # uncompressed anywhere), one iteration, every sweep sampled
    n, it, eps = 36, 1, 1e-4
    marked = I.seeded_basis(n, I.BASE_SEED + 36)
    gates = I.grover(n, marked, it)
    st = qsim.State(n, 22, "rel", eps)
    st.reset_basis(0)
    checked, nsw = run_with_samples(st, n, gates, [oracle.shift_for_eps(eps)], None, PER_SWEEP, 36,
                                    extra_amps=(marked, 0, (1 << n) - 1))
    assert nsw == 35 and checked >= PER_SWEEP * nsw
    assert st.fidelity_grover(marked, it) > 1 - 1e-9
    grover_checks(st, n, marked, it, np.random.default_rng(6), 32)
    sb, fp = st.compressed_bytes()
    assert sb * 64 < 16 << n           # held compressed: ratio far above 64
