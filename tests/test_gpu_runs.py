"""GPU parity of diagonal runs (two or more consecutive diagonal gates of a
sweep applied as one diagonal operator) against the oracle, through the C
ABI, byte for byte: tables of the local product (class bits on high
qubits), the per-tile product, unit factors, the per-amplitude path of runs
whose local gates use more high qubits than the tables cover, runs longer
than a staging chunk, runs in uniform items, and the FP64 count the
profile reports for runs.
"""
import cmath
import math

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
    oracle.build()


def diag(*entries):
    return np.diag(np.asarray(entries, dtype=np.complex128))


def random_diag_run(n, rng, count, qubits=None):
    qs = list(range(n)) if qubits is None else list(qubits)
    gates = []
    for _ in range(count):
        kind = int(rng.integers(0, 8))
        q = [int(v) for v in rng.permutation(qs)[:4]]
        phi = float(rng.uniform(-math.pi, math.pi))
        if kind == 0:
            gates.append(I.cphase(phi, q[0], q[1]))
        elif kind == 1:
            gates.append(I.cz(q[0], q[1]))
        elif kind == 2:
            gates.append(I.Gate(diag(1, 1j), (q[0],), (q[1],), (int(rng.integers(0, 2)),)))
        elif kind == 3:
            gates.append(I.Gate(diag(1, -1j), (q[0],)))
        elif kind == 4:
            gates.append(I.Gate(diag(1, cmath.exp(1j * math.pi / 4)), (q[0],)))
        elif kind == 5:
            gates.append(I.Gate(diag(cmath.exp(-1j * phi), cmath.exp(1j * phi)), (q[0],), (q[2], q[3])))
        elif kind == 6:
            gates.append(I.Gate(diag(cmath.exp(1j * phi), 1, -1, cmath.exp(-2j * phi)), (q[0], q[1])))
        else:
            gates.append(I.Gate(diag(1, cmath.exp(1j * phi)), (q[0],), (q[1], q[2]), (1, 0)))
    return gates


def run_both(n, c, gates, eps=1e-4, hmax=4, depth=512, x=0, normalize=True):
    st = qsim.State(n, c, "rel", eps)
    st.set_schedule(c, hmax, depth)
    st.set_normalize(normalize)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(eps)], None, normalize)
    cs.reset_basis(x)
    cs.run(gates, hmax, depth)
    return st, cs


def same(st, cs, n, c):
    got = st.export_tiles()
    for t, s in enumerate(got):
        assert s == cs.stream(t), t
    assert st.stats()["alpha"] == cs.alpha


@pytest.mark.parametrize("n,c,hmax", [(12, 8, 4), (12, 5, 4), (11, 6, 2), (10, 3, 2), (13, 8, 4)])
def test_qft_runs_match_oracle(n, c, hmax):
    x = I.seeded_basis(n)
    st, cs = run_both(n, c, I.qft(n), x=x, hmax=hmax)
    same(st, cs, n, c)
    assert st.fidelity_qft(x) > 0.9999


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_random_diagonal_runs_match_oracle(seed):
    n, c = 11, 5
    rng = np.random.default_rng(seed)
    gates = [I.h(q) for q in range(n)]
    for _ in range(4):
        gates += random_diag_run(n, rng, int(rng.integers(2, 30)))
        gates += [I.h(q) for q in rng.permutation(n)[:3]]
    st, cs = run_both(n, c, gates)
    same(st, cs, n, c)


def test_runs_beyond_the_tables_and_the_staging_chunk():
    # local gates tied to six high qubits (more class bits than the tables
    # hold: the per-amplitude path) and a run of 120 gates (three chunks)
    n, c = 12, 4
    rng = np.random.default_rng(9)
    gates = [I.h(q) for q in range(n)]
    for hq in range(c, n):
        gates.append(I.cphase(float(rng.uniform(0.1, 3.0)), hq, int(rng.integers(0, c))))
    gates += [I.h(q) for q in range(n)]
    gates += random_diag_run(n, rng, 120)
    gates += [I.h(0)]
    st, cs = run_both(n, c, gates)
    same(st, cs, n, c)


def test_runs_on_uniform_items_and_unit_runs():
    # runs on high qubits only over tiles that stay uniform (one amplitude
    # per tile), and runs of CZ / S / S^dagger whose factors are units
    n, c = 12, 5
    rng = np.random.default_rng(21)
    gates = [I.h(q) for q in range(c, n)]
    gates += random_diag_run(n, rng, 10, qubits=range(c, n))
    gates += [I.h(q) for q in range(c, n)]
    for _ in range(6):
        a, b = (int(v) for v in rng.permutation(n)[:2])
        gates.append(I.cz(a, b))
        gates.append(I.Gate(diag(1, 1j), (b,), (a,)))
        gates.append(I.Gate(diag(1, -1j), (a,)))
    gates += [I.h(q) for q in range(n)]
    st, cs = run_both(n, c, gates, hmax=2)
    same(st, cs, n, c)


def test_gate_by_gate_mode_matches_unfused_oracle():
    n, c = 11, 6
    x = I.seeded_basis(n)
    gates = I.qft(n)
    st = qsim.State(n, c, "rel", 1e-4)
    st.set_fusion(False)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(1e-4)], None, True, fuse=False)
    cs.reset_basis(x)
    cs.run(gates, 4, 512)
    same(st, cs, n, c)


def test_profile_counts_run_arithmetic():
    # QFT-12 on 2^8 tiles: the FP64 count the profile reports is the
    # canonical count of the gates outside runs and scaled gates, plus what
    # the runs and scaled gates execute on the device (per visited nonzero
    # amplitude 4 for G a, 4 more for T*L, the table and tile products; per
    # formed Hadamard pair 4): below three quarters of the gate-by-gate count
    n, c = 12, 8
    x = I.seeded_basis(n)
    gates = I.qft(n)
    counts = {}
    for fuse in (True, False):
        st = qsim.State(n, c, "rel", 1e-4)
        st.set_fusion(fuse)
        st.reset_basis(x)
        st.set_profiling(True)
        st.apply_all(gates)
        st.flush()
        counts[fuse] = st.profile()["dp_ops"] / (1 << n)
    assert counts[True] < 0.75 * counts[False]
    assert counts[True] > 0
