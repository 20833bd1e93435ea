"""Pins of the oracle's gate fusion (O3).

Diagonal runs: two or more consecutive diagonal gates of a sweep applied
as one diagonal operator whose entry is the product of the gates' entries
(the product of diagonal matrices, Sec. II), with unit factors (-1, i, -i)
taken exactly and the other factors multiplied in gate order, split into
the part on qubits >= c and the rest.  Scaled gates: an uncontrolled gate
that is d times a matrix of units with one real d (a Hadamard) forms only
its unit sums; the sweep multiplies the product of those d into the
normalize scale at decompression (a scalar commutes with linear maps).

* Within rounding of the gates applied one by one (the dense simulator O1),
  on QFTs, grid circuits and random runs of controlled phases, CZ, S, T,
  Rz and two-target diagonal gates with controls on low and high qubits.
* Exact where the arithmetic is exact: runs of unit factors only give O1's
  amplitudes bit for bit, and so do runs in which every amplitude meets at
  most one other factor (G = that entry: the gate's own product); Hadamards
  on a basis state (one nonzero term per row) give O1's amplitudes bit for
  bit, d^n either way.
* Gates that are not scaled (controlled Hadamards, sqrt(X), X, a lone
  diagonal gate) keep the gate-by-gate arithmetic: bit-identical to O1.
* The fused QFT against its closed form e^{2 pi i x k / N} / sqrt(N).
* Runs are really fused: the QFT's amplitudes differ in rounding from the
  gate-by-gate sweep somewhere.
* Exact zeros: an amplitude whose components are both zero (either sign)
  keeps its bits under a run, and so does a pair of them under a scaled
  gate; an amplitude with one zero component is multiplied like any other.
"""
import cmath
import math

import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I


def lossless(n, c, gates, hmax, depth, fuse=True):
    cs = oracle.CSim(n, c, [0], normalize=False, fuse=fuse)
    cs.reset_basis(0)
    cs.run(gates, hmax, depth)
    return cs.dense()


def diag(*entries):
    return np.diag(np.asarray(entries, dtype=np.complex128))


def random_diag_run(n, rng, count):
    """Diagonal gates of every kind on random qubits (low and high)."""
    gates = []
    for _ in range(count):
        kind = rng.integers(0, 7)
        q = [int(v) for v in rng.permutation(n)[:4]]
        phi = float(rng.uniform(-math.pi, math.pi))
        if kind == 0:
            gates.append(I.cphase(phi, q[0], q[1]))
        elif kind == 1:
            gates.append(I.cz(q[0], q[1]))
        elif kind == 2:
            gates.append(I.Gate(diag(1, 1j), (q[0],), (q[1],), (int(rng.integers(0, 2)),)))   # controlled S
        elif kind == 3:
            gates.append(I.Gate(diag(1, -1j), (q[0],)))                                        # S^dagger
        elif kind == 4:
            gates.append(I.Gate(diag(1, cmath.exp(1j * math.pi / 4)), (q[0],)))                # T
        elif kind == 5:
            gates.append(I.Gate(diag(cmath.exp(-1j * phi), cmath.exp(1j * phi)), (q[0],), (q[2], q[3])))  # CC-Rz
        else:
            gates.append(I.Gate(diag(cmath.exp(1j * phi), 1, -1, cmath.exp(-2j * phi)), (q[0], q[1])))
    return gates


def mixed_circuit(n, seed, layers=3):
    rng = np.random.default_rng(seed)
    gates = I.basis_gates(n, int(rng.integers(0, 1 << n)))
    for _ in range(layers):
        gates += [I.h(q) for q in range(n)]
        gates += random_diag_run(n, rng, int(rng.integers(2, 12)))
    return gates


@pytest.mark.parametrize("n,c,hmax,depth", [(10, 4, 2, 512), (10, 4, 2, 6), (9, 9, 2, 40), (8, 2, 2, 7),
                                            (11, 5, 4, 512)])
def test_fused_runs_within_rounding_of_dense(n, c, hmax, depth):
    for gates in (I.basis_gates(n, I.seeded_basis(n)) + I.qft(n),
                  I.random_grid(*I.grid_shape(n), 4, 9),
                  mixed_circuit(n, n * 100 + c)):
        psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
        got = lossless(n, c, gates, hmax, depth)
        # a run multiplies each amplitude at most twice instead of once per
        # gate: a few ulps of the unit-norm state per amplitude
        assert np.max(np.abs(got - psi)) <= 1e-14


def sx(q):
    # a mixing gate that is not scaled (its rows' first entries differ)
    return I.Gate(I.MAT_SQRT_X, (q,), name="SX")


def test_unit_runs_are_exact():
    # CZ, Z, S, S^dagger, multi-controlled Z: factors -1, i, -i only
    n, c = 9, 4
    rng = np.random.default_rng(11)
    gates = I.basis_gates(n, 0x155)
    for _ in range(4):
        gates += [sx(q) for q in range(n)]
        for _ in range(8):
            a, b, d = (int(v) for v in rng.permutation(n)[:3])
            pick = int(rng.integers(0, 4))
            if pick == 0:
                gates.append(I.cz(a, b))
            elif pick == 1:
                gates.append(I.Gate(diag(1, 1j), (a,), (b,)))
            elif pick == 2:
                gates.append(I.Gate(diag(1, -1j), (a,), (b, d), (0, 1)))
            else:
                gates.append(I.mcz(n, int(rng.integers(0, 1 << n))))
    psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
    for hmax, depth in ((2, 512), (4, 9)):
        got = lossless(n, c, gates, hmax, depth)
        assert np.array_equal(got.view(np.uint64), psi.view(np.uint64))


def test_runs_with_one_general_factor_per_amplitude_are_exact():
    # phases on one target whose controls exclude one another (values 0 and
    # 1 of the same qubit, or of two qubits): each amplitude meets at most
    # one general factor, so G is that entry and the product is the gate's own
    n, c = 9, 4
    rng = np.random.default_rng(5)
    gates = I.basis_gates(n, 0x0F3) + [sx(q) for q in range(n)]
    for t, a in ((1, 6), (7, 2), (5, 8), (0, 3)):
        p = [cmath.exp(1j * float(v)) for v in rng.uniform(0.1, 3.0, 3)]
        gates.append(I.Gate(diag(1, p[0]), (t,), (a,), (0,)))
        gates.append(I.Gate(diag(1, p[1]), (t,), (a,), (1,)))
        gates.append(I.Gate(diag(p[2], 1), (t,)))                 # the other target value
        gates += [sx(q) for q in range(n)]
    psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
    got = lossless(n, c, gates, 2, 512)
    assert np.array_equal(got.view(np.uint64), psi.view(np.uint64))


@pytest.mark.parametrize("c", [3, 5, 8])
def test_fused_qft_closed_form(c):
    n = 12
    x = I.seeded_basis(n)
    got = lossless(n, c, I.basis_gates(n, x) + I.qft(n), 4, 512)
    k = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * k) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(got - ref)) <= 1e-12


def test_runs_are_fused():
    n, c = 10, 4
    gates = I.basis_gates(n, I.seeded_basis(n)) + I.qft(n)
    a = lossless(n, c, gates, 4, 512, fuse=True)
    b = lossless(n, c, gates, 4, 512, fuse=False)
    assert not np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_hadamards_on_a_basis_state_are_exact():
    # every row meets one nonzero amplitude: each Hadamard multiplies by d
    # once, gate by gate or folded into the sweep's scale (d^n, multiplied
    # in the same order, when the Hadamards share one sweep)
    for n, c, hmax in ((9, 5, 4), (10, 6, 4), (7, 7, 1)):
        gates = I.basis_gates(n, 0x1A5 & ((1 << n) - 1)) + [I.h(q) for q in range(n)]
        psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
        got = lossless(n, c, gates, hmax, 512)
        assert np.array_equal(got.view(np.uint64), psi.view(np.uint64))
        assert len(set(np.abs(got.real).view(np.uint64).tolist())) == 1


def test_gates_that_are_not_scaled_keep_their_arithmetic():
    n, c = 9, 4
    rng = np.random.default_rng(17)
    gates = I.basis_gates(n, 0x0B6)
    for _ in range(3):
        gates += [sx(q) for q in range(n)]
        gates.append(I.Gate(I.MAT_H, (2,), (7,)))                      # controlled Hadamard
        gates.append(I.x(int(rng.integers(0, n))))
        gates.append(I.cphase(0.3, 1, 5))                               # a lone diagonal gate
        gates += [sx(q) for q in rng.permutation(n)[:4]]
    psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
    got = lossless(n, c, gates, 4, 512)
    assert np.array_equal(got.view(np.uint64), psi.view(np.uint64))


def zero_mixed_state(n, seed):
    """A random state with exact zeros of both signs (both components),
    amplitudes with one zero component, and pairs (l, l ^ 8) of zeros."""
    rng = np.random.default_rng(seed)
    psi = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi /= np.linalg.norm(psi)
    nz, pz = -0.0, 0.0
    zs = [complex(pz, pz), complex(nz, nz), complex(pz, nz), complex(nz, pz)]
    idx = rng.permutation(1 << n)
    for j, l in enumerate(idx[:40]):
        psi[l] = zs[j % 4]
    for l in idx[40:50]:
        psi[l] = complex(0.0, psi[l].imag)            # zero real part
    for l in idx[50:60]:
        psi[l] = complex(psi[l].real, -0.0)           # zero imaginary part
    for j, l in enumerate(range(0, 1 << n, 37)):
        if not (l >> 3) & 1:                          # both members of the pair (l, l ^ 8)
            psi[l] = zs[j % 4]
            psi[l ^ 8] = zs[(j + 1) % 4]
    return psi


def test_zero_amplitudes_are_left_as_they_are():
    n, c = 8, 4
    psi0 = zero_mixed_state(n, 3)
    zero0 = (psi0.real == 0) & (psi0.imag == 0)
    # a run in which every amplitude meets one general factor (exact
    # against the gates one by one), then a Hadamard in a sweep of its own
    rng = np.random.default_rng(9)
    p = [cmath.exp(1j * float(v)) for v in rng.uniform(0.3, 2.8, 3)]
    run = [I.Gate(diag(1, p[0]), (1,), (6,), (0,)), I.Gate(diag(1, p[1]), (1,), (6,), (1,)),
           I.Gate(diag(p[2], 1), (1,))]
    cs = oracle.CSim(n, c, [0], normalize=False, fuse=True)
    cs.set_dense(psi0)
    cs.sweep(run, [])
    got = cs.dense()
    want = oracle.dense_run(psi0.copy(), n, run)
    assert np.array_equal(got[zero0].view(np.uint64), psi0[zero0].view(np.uint64))
    assert np.array_equal(got[~zero0].view(np.uint64), want[~zero0].view(np.uint64))
    # multiplying a zero would have changed some of their signs
    assert not np.array_equal(want[zero0].view(np.uint64), psi0[zero0].view(np.uint64))

    cs.sweep([I.h(3)], [])
    got2 = cs.dense()
    want2 = oracle.dense_run(got.copy(), n, [I.h(3)])
    lo = np.array([l for l in range(1 << n) if not (l >> 3) & 1])
    z = zero0.copy()
    pair_zero = z[lo] & z[lo ^ 8]
    one_nz = z[lo] ^ z[lo ^ 8]
    for sel in (lo[pair_zero], lo[pair_zero] ^ 8):
        assert np.array_equal(got2[sel].view(np.uint64), got[sel].view(np.uint64))
    assert pair_zero.sum() >= 5 and one_nz.sum() >= 5
    # a pair with one nonzero member: d x, exact either way
    for sel in (lo[one_nz], lo[one_nz] ^ 8):
        assert np.array_equal(got2[sel].view(np.uint64), want2[sel].view(np.uint64))
    assert np.max(np.abs(got2 - want2)) <= 1e-15
