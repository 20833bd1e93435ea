"""GPU parity of point items against the oracle, byte for byte.

A point item is a tile group in which every tile is exactly +0 but for at
most one amplitude, at a tile index common to the group (a basis state
after gates on high qubits: the QFT's first sweeps).  In a sweep whose
gates are diagonal-run members, scaled gates or permutations, the mixing
ones on qubits at or above the tile size, the kernel applies the gates to
that one amplitude per tile; the streams must equal the oracle's full
computation.  Items that are not point items (two amplitudes in a tile,
tiles that disagree on the index, zeros of negative sign kept by the
lossless level) take the full path, with the same result.
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


def point_sweep_gates(n, c, rng):
    """Hadamards on high qubits, runs of phases with controls below and
    above c, a SWAP and an X of high qubits, a CNOT among high qubits."""
    hi = list(range(c, n))
    gates = [I.h(q) for q in rng.permutation(hi)[:3]]
    for _ in range(6):
        t = int(rng.choice(hi))
        k = int(rng.integers(0, n))
        if k == t:
            k = (t + 1) % n
        gates.append(I.cphase(float(rng.uniform(-math.pi, math.pi)), t, k))
    gates.append(I.Gate(diag(1, cmath.exp(1j * 0.7)), (int(rng.choice(hi)),), (1,)))
    gates.append(I.Gate(diag(1, 1j), (int(rng.choice(hi)),)))
    a, b = (int(v) for v in rng.permutation(hi)[:2])
    gates.append(I.swap(a, b))
    gates.append(I.Gate(I.MAT_X, (int(rng.choice(hi)),), name="X"))
    gates.append(I.Gate(I.MAT_X, (a,), (b,), name="CX"))
    gates += [I.h(q) for q in rng.permutation(hi)[:2]]
    return gates


def run_pair(n, c, gates, codec, eps, psi=None, x=0, hmax=4):
    st = qsim.State(n, c, codec, eps)
    st.set_schedule(c, hmax, 512)
    if psi is None:
        st.reset_basis(x)
    else:
        st.set_amplitudes(psi)
    st.apply_all(gates)
    st.flush()
    shifts = [0] if codec == "lossless" else [oracle.shift_for_eps(eps)]
    cs = oracle.CSim(n, c, shifts, None, codec != "lossless")
    if psi is None:
        cs.reset_basis(x)
    else:
        cs.set_dense(psi)
    cs.run(gates, hmax, 512)
    got = st.export_tiles()
    for t, s in enumerate(got):
        assert s == cs.stream(t), t
    assert st.stats()["alpha"] == cs.alpha
    st.close()


@pytest.mark.parametrize("n,c", [(13, 8), (12, 6), (11, 5)])
def test_point_items_from_a_basis_state(n, c):
    rng = np.random.default_rng(n * 10 + c)
    x = I.seeded_basis(n, 100 + c)
    gates = point_sweep_gates(n, c, rng)
    # the QFT's own first sweeps too
    run_pair(n, c, gates, "rel", 1e-4, x=x)
    run_pair(n, c, I.qft(n), "rel", 1e-4, x=x)
    run_pair(n, c, gates, "lossless", 0.0, x=x)


def test_items_that_are_not_point_items():
    n, c = 12, 8
    rng = np.random.default_rng(4)
    gates = point_sweep_gates(n, c, rng)
    N = 1 << n
    # two amplitudes in some tiles
    psi = np.zeros(N, dtype=np.complex128)
    psi[rng.choice(N, 40, replace=False)] = rng.normal(size=40) + 1j * rng.normal(size=40)
    psi /= np.linalg.norm(psi)
    run_pair(n, c, gates, "rel", 1e-4, psi=psi)
    # one amplitude per tile, at tile indices that differ between tiles
    psi = np.zeros(N, dtype=np.complex128)
    for t in range(N >> c):
        psi[(t << c) | int(rng.integers(0, 1 << c))] = 1.0
    psi /= np.linalg.norm(psi)
    run_pair(n, c, gates, "rel", 1e-4, psi=psi)
    # a common index, but zeros of negative sign that the lossless level keeps
    psi = np.zeros(N, dtype=np.complex128)
    p = 37
    for t in range(N >> c):
        psi[(t << c) | p] = complex(rng.normal(), rng.normal())
    psi /= np.linalg.norm(psi)
    for l in rng.choice(N, 30, replace=False):
        if l & ((1 << c) - 1) != p:
            psi[l] = complex(-0.0, -0.0)
    run_pair(n, c, gates, "lossless", 0.0, psi=psi)
    run_pair(n, c, gates, "rel", 1e-4, psi=psi)


def test_point_items_under_a_negative_scale():
    """A scaled gate whose common factor is negative (-H) makes the decode
    scale negative, so exact zeros decode to -0: such items are not point
    items, and the streams still equal the oracle's; later sweeps of the
    same circuit (positive scale again) take the point path."""
    n, c = 12, 8
    rng = np.random.default_rng(7)
    hi = list(range(c, n))
    x = I.seeded_basis(n, 5)
    gates = [I.h(hi[0]), I.cphase(0.3, hi[0], 2), I.Gate(-I.MAT_H, (hi[1],), name="mH"),
             I.cphase(-1.1, hi[1], hi[0]), I.cphase(0.9, 3, hi[1])]
    gates += point_sweep_gates(n, c, rng)
    for hmax in (4, 2):
        run_pair(n, c, gates, "rel", 1e-4, x=x, hmax=hmax)
        run_pair(n, c, gates, "lossless", 0.0, x=x, hmax=hmax)
