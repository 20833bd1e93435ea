"""Full-size cases in the benchmark's launch configuration, checked on
sampled outputs the oracle can compute one by one.

* 28-qubit QFT, relative bound 1e-4 (2^28 amplitudes, 4 GiB uncompressed):
  for the first, a middle and the last sweep, sampled items are re-run by
  the oracle from the GPU's input streams and the same normalize scale;
  the GPU's output streams must be byte-identical.  The final state's
  fidelity to the closed form must be >= 0.9995 (the paper's QFT target).
* 30-qubit random grid (5 x 6, depth 20) with the error-bound ladder
  {lossless, 1e-5, 1e-4, 1e-3}, theta = 4: sampled items as above, the
  ladder must mix lossless and lossy levels, and the fidelity against the
  uncompressed FP64 GPU run is reported.
"""
import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


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


def run_with_samples(st, n, gates, shifts, max_bytes, check, per_sweep, seed):
    s = st.stats()
    c, hmax, depth = s["tile_log2"], s["hmax"], s["depth"]
    plan = qsim.plan_sweeps(n, c, hmax, depth, gates)
    rng = np.random.default_rng(seed)
    applied, checked = 0, 0
    for k, (lo, hi, H) in enumerate(plan):
        if k not in check(len(plan)):
            continue
        st.apply_all(gates[applied:lo])
        st.flush()
        alpha = st.stats()["alpha"]
        nitems = 1 << (n - c - len(H))
        items = rng.choice(nitems, min(per_sweep, nitems), replace=False)
        bases = [expand(int(i), H, c) for i in items]
        before = {T: [st.export_tiles(t, 1)[0] for t in members(T, H, c)] for T in bases}
        st.apply_all(gates[lo:hi])
        st.flush()
        applied = hi
        for T in bases:
            after = [st.export_tiles(t, 1)[0] for t in members(T, H, c)]
            want = oracle.item_sweep(n, c, H, T, before[T], alpha, gates[lo:hi], shifts, max_bytes)
            assert after == want, (k, T)
            checked += 1
    st.apply_all(gates[applied:])
    st.flush()
    return checked


def test_qft28_sampled_items_and_fidelity():
    n, eps = 28, 1e-4
    x = I.seeded_basis(n)
    st = qsim.State(n, 20, "rel", eps)
    st.reset_basis(x)
    checked = run_with_samples(st, n, I.qft(n), [oracle.shift_for_eps(eps)], None,
                               lambda m: {0, m // 2, m - 1}, 8, 28)
    assert checked == 24
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
    checked = run_with_samples(st, n, gates, shifts, oracle.max_bytes_for(c, 4.0),
                               lambda m: {m // 3, m - 1}, 6, 30)
    assert checked == 12
    hist = st.stats()["level_hist"]
    assert hist[0] > 0 and sum(hist[1:4]) > 0          # lossless and lossy levels both used
    ref = qsim.State(n, 20, "none", 0.0)
    ref.apply_all(gates)
    ref.flush()
    F = st.fidelity_state(ref)
    ref.close()
    assert F > 0.99


def test_grover30_sampled_items_every_sweep_kind():
    # Grover at 30 qubits, two iterations, relative bound 1e-4: sampled
    # items of sweeps of every kind (Hadamards on uniform tiles, the oracle
    # MCZ with Hadamards on low qubits, X layers that only move tiles, spike
    # tiles from the diffusion) re-run by the oracle from the GPU's input
    # streams, byte for byte; then the closed form
    import math
    n, it, eps = 30, 2, 1e-4
    marked = I.seeded_basis(n, 77)
    gates = I.grover(n, marked, it)
    st = qsim.State(n, 22, "rel", eps)
    st.reset_basis(0)
    checked = run_with_samples(st, n, gates, [oracle.shift_for_eps(eps)], None,
                               lambda m: set(range(0, m, 3)), 4, 31)
    assert checked >= 60
    assert st.fidelity_grover(marked, it) > 1 - 1e-9
    th = math.asin(2.0 ** (-n / 2))
    want = math.sin((2 * it + 1) * th)
    assert abs(st.amplitudes(marked, 1)[0].real - want) < 1e-4 * abs(want)
