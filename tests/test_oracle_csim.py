"""Pins of the oracle's compressed simulator (O3), norm and sweep partition.

* Lossless level without normalisation, every gate on its own: Algorithm 1
  over compressed tiles must reproduce the dense simulator bit for bit.
* Relative bound (Sec. III): after each sweep every stored component is
  within 2^(s-53)|x| of (normalize, then apply the sweep's gates) to the
  stored state before the sweep (Algorithm 2's per-stride steps).
* Normalisation: the scale used is 1/sqrt(sum |a^|^2) of the stored state,
  the sum taken exactly (checked with Python integers and fractions).
* Fidelity of the compressed QFT against the dense one.
* Partition: every sweep's mixing high qubits fit its pair set, sweeps are
  maximal, gates stay in order.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.partition import is_diagonal, partition
from paper_1811_05140_gb300 import inputs as I


def exact_units(values: np.ndarray) -> int:
    total = 0
    for x in np.asarray(values).view(np.float64).tolist():
        total += math.floor(Fraction(x) ** 2 * (1 << 112))
    return total


def test_norm_units_exact():
    rng = np.random.default_rng(3)
    v = (rng.normal(size=300) + 1j * rng.normal(size=300)) * np.ldexp(1.0, rng.integers(-70, 3, 300))
    v[:5] = [0, -0.0, 1e-300, 2.0**-56, 15.9]
    assert oracle.sum_sq_units(v) == exact_units(v)
    S = exact_units(v)
    assert oracle.units_to_double(S) == S / (1 << 112)          # correctly rounded
    for S in (1, (1 << 112), (1 << 112) + 1, (1 << 127) - 1, 3 << 70, (1 << 65) + (1 << 11) + 1):
        assert oracle.units_to_double(S) == S / (1 << 112)


@pytest.mark.parametrize("n,c,hmax,depth", [(10, 4, 2, 1), (10, 4, 2, 6), (9, 9, 2, 8), (8, 2, 2, 3), (7, 5, 1, 4)])
def test_lossless_compressed_equals_dense(n, c, hmax, depth):
    xval = I.seeded_basis(n)
    gates = I.basis_gates(n, xval) + I.qft(n) + I.random_grid(*I.grid_shape(n), 3, 9)
    cs = oracle.CSim(n, c, [0], normalize=False, fuse=False)
    cs.reset_basis(0)
    cs.run(gates, hmax, depth)
    psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
    got = cs.dense()
    assert np.array_equal(got.view(np.uint64), psi.view(np.uint64))


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_each_sweep_within_relative_bound(eps):
    n, c, hmax, depth = 9, 5, 2, 5
    s = oracle.shift_for_eps(eps)
    gates = I.basis_gates(n, 0b101100111) + I.qft(n)
    cs = oracle.CSim(n, c, [s], normalize=True)
    cs.reset_basis(0)
    for lo, hi, H in partition(gates, n, c, hmax, depth):
        before = cs.dense()
        alpha = cs.alpha
        exp_units = exact_units(before)
        assert cs.norm_units() == exp_units
        nrm = exp_units / (1 << 112)
        assert alpha == 1.0 / math.sqrt(nrm)
        ref = before.copy()
        if alpha != 1.0:
            ref = (ref.view(np.float64) * alpha).view(np.complex128)
        oracle.dense_run(ref, n, gates[lo:hi])
        cs.sweep(gates[lo:hi], H)
        got = cs.dense()
        r, g = ref.view(np.float64), got.view(np.float64)
        nz = r != 0
        assert np.all(np.abs(g - r)[nz] < np.ldexp(np.abs(r[nz]), s - 53))
        assert np.all(g[~nz] == 0)
        assert np.all(np.abs(g - r) <= eps * np.abs(r))


def test_compressed_qft_fidelity():
    n, c = 12, 8
    xval = I.seeded_basis(n)
    for eps, floor in ((1e-4, 0.99999), (1e-2, 0.99)):
        cs = oracle.CSim(n, c, [oracle.shift_for_eps(eps)], normalize=True)
        cs.reset_basis(xval)
        cs.run(I.qft(n), 2, 8)
        psi = cs.dense()
        k = np.arange(1 << n)
        ref = np.exp(2j * np.pi * ((xval * k) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
        F = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
        assert F >= floor


def test_aalc_ladder_meets_threshold_or_uses_last_level():
    n, c = 10, 6
    shifts = [0, 36, 39, 43]
    for theta in (2.0, 4.0, 8.0):
        mb = oracle.max_bytes_for(c, theta)
        cs = oracle.CSim(n, c, shifts, mb, normalize=True)
        cs.reset_basis(I.seeded_basis(n))
        cs.run(I.qft(n), 2, 4)
        for t in range(1 << (n - c)):
            st = cs.stream(t)
            assert len(st) <= mb or st[2] == len(shifts) - 1
        assert sum(cs.hist()) > 0


def test_items_without_touching_gates_are_skipped():
    n, c = 10, 4
    cs = oracle.CSim(n, c, [0], normalize=False)
    cs.reset_basis(0)
    # controlled on two high qubits: only items with both bits set change
    g = I.Gate(I.MAT_H, (0,), (8, 9), (1, 1))
    cs.sweep([g], [])
    done, skipped = cs.items()
    assert done == (1 << (n - c)) // 4 and skipped == 3 * (1 << (n - c)) // 4
    # a diagonal gate whose entry on the item's fixed target value is 1
    cs2 = oracle.CSim(n, c, [0], normalize=False)
    cs2.reset_basis(0)
    cs2.sweep([I.Gate(I.phase(0.3), (7,))], [])
    done, skipped = cs2.items()
    assert done == skipped == (1 << (n - c)) // 2


def test_partition_properties():
    n, c = 14, 6
    gates = I.qft(n) + I.grover(n, 1234, 1) + I.random_grid(2, 7, 6, 5)
    one_target = [g for g in gates if len(g.targets) == 1]
    with pytest.raises(ValueError):
        partition(I.qft(n), n, c, 1, 8)        # SWAP of two high qubits
    for hmax, depth, gl in ((2, 1, gates), (2, 4, gates), (2, 64, gates), (1, 8, one_target)):
        gates = gl
        sw = partition(gates, n, c, hmax, depth)
        assert sw[0][0] == 0 and sw[-1][1] == len(gates)
        for (lo, hi, H), nxt in zip(sw, sw[1:] + [None]):
            assert 0 < hi - lo <= depth
            assert len(H) == min(hmax, n - c) and all(q >= c for q in H)
            mix = set()
            for g in gates[lo:hi]:
                if not is_diagonal(g.matrix):
                    mix |= {t for t in g.targets if t >= c}
            assert mix <= set(H)
            pad = sorted(set(H) - mix)
            free = [q for q in range(c, n) if q not in mix]
            assert pad == free[:len(pad)]               # padding: smallest free high qubits
            if nxt is not None:
                g = gates[hi]
                gm = set() if is_diagonal(g.matrix) else {t for t in g.targets if t >= c}
                assert hi - lo == depth or len(mix | gm) > hmax
    # QFT: every H on a high qubit needs a pair slot; CP gates are diagonal
    assert len(partition(I.qft(n), n, c, 2, 10**6)) >= math.ceil((n - c) / 2)


def test_normalisation_reduces_norm_drift():
    n, c = 10, 5
    s = oracle.shift_for_eps(1e-2)
    gates = I.random_grid(2, 5, 12, 21)
    a = oracle.CSim(n, c, [s], normalize=True)
    b = oracle.CSim(n, c, [s], normalize=False)
    a.reset_basis(0)
    b.reset_basis(0)
    a.run(gates, 2, 1)
    b.run(gates, 2, 1)
    assert abs(a.norm() - 1) < abs(b.norm() - 1) or abs(a.norm() - 1) < 1e-3


def test_sweeps_that_only_move_tiles():
    """A sweep of permutation gates on qubits >= c moves whole tiles: the
    stored state afterwards is the exact permutation of the stored state
    before (no normalize, no re-quantisation), each stream moves unchanged
    to its image tile, and the scale stays the same.  With a low qubit
    involved the sweep decompresses as usual (normalize, then gates)."""
    n, c = 10, 4
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(1e-3)], normalize=True)
    cs.reset_basis(0)
    cs.run(I.random_grid(2, 5, 6, 4), 2, 8)
    alpha = cs.alpha
    assert alpha != 1.0
    moves = [I.x(9), I.swap(5, 8), I.Gate(I.MAT_X, (6,), (7,), (1,)), I.x(7)]
    before = cs.dense()
    streams = [cs.stream(t) for t in range(1 << (n - c))]
    for lo, hi, Hs in partition(moves, n, c, 4, 8):
        cs.sweep(moves[lo:hi], Hs)
    want = oracle.dense_run(before.copy(), n, moves)
    assert np.array_equal(cs.dense().view(np.uint64), want.view(np.uint64))
    assert cs.alpha == alpha
    # every stream is one of the old streams, moved whole
    assert sorted(cs.stream(t) for t in range(1 << (n - c))) == sorted(streams)
    # a permutation on a low qubit decompresses: the values are rescaled
    cs.sweep([I.x(0)], [])
    ref = (want.copy().view(np.float64) * alpha).view(np.complex128)
    oracle.dense_run(ref, n, [I.x(0)])
    got = cs.dense()
    r, g = ref.view(np.float64), got.view(np.float64)
    nz = r != 0
    assert np.all(np.abs(g - r)[nz] <= 1e-3 * np.abs(r[nz]))
