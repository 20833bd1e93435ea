"""Pins of the oracle's per-stride AALC decision (Algorithm 2 decides once
per stride: compress the stride at the ladder's first bound, test the
stride's ratio against theta, retry at the next bound, keep the last).

* Special cases that reduce to the fixed-bound codec: theta so small that
  the lossless level always passes (every stream equals the per-tile
  lossless one), theta so large that no level passes (every stream is the
  fixed-bound stream of the last level, only the level byte differs).
* All-zero strides: 32-byte CONST streams at level 0, written out by hand.
* A mixed state: the stride levels equal the rule evaluated with O2's
  single-level encoder, and differ from the per-tile decisions where a
  compressible tile shares a stride with an incompressible one.
* Sweeps: with the lossless level passing and no normalize, stride sweeps
  give the same streams as tile sweeps; after a lossy QFT every stride holds one level
  and meets its limit unless it is at the last level.
"""

import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I

LADDER = [1e-5, 1e-4, 1e-3, 1e-2]


def shifts():
    return [0] + [oracle.shift_for_eps(e) for e in LADDER]


def unit_csim(n, c, u, theta, normalize=True):
    cs = oracle.CSim(n, c, shifts(), oracle.max_bytes_for(c, theta), normalize)
    ut = cs.set_unit(u, theta)
    return cs, ut


def level_of(stream):
    return stream[2]


def mixed_state(n, c, u, seed):
    return I.strided_mix_state(n, c, u, seed)


def test_decision_unit_is_capped():
    cs, ut = unit_csim(10, 4, 4, 4.0)
    assert ut == 0                                   # stride of one tile: per tile
    cs, ut = unit_csim(10, 4, 7, 4.0)
    assert ut == 3
    cs, ut = unit_csim(10, 4, 30, 4.0)
    assert ut == 6                                   # whole state
    cs = oracle.CSim(10, 4, [oracle.shift_for_eps(1e-3)], None)
    assert cs.set_unit(8, 4.0) == 0                  # one level: nothing to decide


def test_zero_strides_are_const_lossless_by_hand():
    n, c, u = 8, 4, 6
    cs, _ = unit_csim(n, c, u, 4.0)
    psi = mixed_state(n, c, u, I.BASE_SEED + 40)
    cs.set_dense(psi)
    const0 = bytes(24) + bytes([c]) + bytes(7)       # CONST, s = 0, level 0, zero anchors
    for t in range(0, 4):                            # stride 0 is all zero
        assert cs.stream(t) == const0


def test_tiny_theta_keeps_everything_lossless():
    n, c, u = 9, 4, 7
    psi = mixed_state(n, c, u, I.BASE_SEED + 41)
    cs, _ = unit_csim(n, c, u, 1e-9)
    cs.set_dense(psi)
    for t in range(1 << (n - c)):
        want, _, _ = oracle.encode_tile(psi[t << c:(t + 1) << c], c, [0])
        assert cs.stream(t) == want
    assert np.array_equal(cs.dense().view(np.uint64), psi.view(np.uint64))


def test_huge_theta_gives_the_last_fixed_bound():
    n, c, u = 9, 4, 7
    psi = mixed_state(n, c, u, I.BASE_SEED + 42)
    cs, _ = unit_csim(n, c, u, 1e9)
    cs.set_dense(psi)
    last = len(shifts()) - 1
    s_last = shifts()[-1]
    for t in range(1 << (n - c)):
        want, _, _ = oracle.encode_tile(psi[t << c:(t + 1) << c], c, [s_last])
        got = cs.stream(t)
        assert level_of(got) == last
        assert got[:2] + got[3:] == want[:2] + want[3:]      # same stream but the level byte
    assert cs.hist()[last] == 0                       # hist is reset after a dense set


@pytest.mark.parametrize("theta", [2.0, 3.0, 5.0, 8.0])
def test_stride_levels_follow_the_ratio_test(theta):
    n, c, u = 10, 5, 7
    nt, N = 1 << (u - c), 1 << c
    psi = mixed_state(n, c, u, I.BASE_SEED + 43)
    cs, _ = unit_csim(n, c, u, theta)
    cs.set_dense(psi)
    sh = shifts()
    limit = oracle.max_bytes_for(u, theta)
    levels, tile_levels = set(), []
    for s0 in range(0, 1 << (n - c), nt):
        tiles = [psi[(s0 + j) * N:(s0 + j + 1) * N] for j in range(nt)]
        want_k = len(sh) - 1
        for k in range(len(sh)):
            if sum(len(oracle.encode_tile_level(a, c, sh, k)[0]) for a in tiles) <= limit:
                want_k = k
                break
        levels.add(want_k)
        for j, a in enumerate(tiles):
            got = cs.stream(s0 + j)
            assert got == oracle.encode_tile_level(a, c, sh, want_k)[0]
            tile_levels.append((want_k, oracle.encode_tile(a, c, sh, oracle.max_bytes_for(c, theta))[1]))
    assert len(levels) >= 2
    # a stride's level is not a per-tile level: some tile is coded at
    # another level than it would pick alone
    assert any(ks != kt for ks, kt in tile_levels)


def test_stride_sweeps_equal_tile_sweeps_when_lossless_passes():
    # without normalize: tile sweeps keep untouched items and move the
    # streams of SWAP sweeps, stride sweeps decode and re-encode them
    # losslessly, which gives the same bytes
    n, c, u = 10, 4, 7
    gates = I.basis_gates(n, I.seeded_basis(n)) + I.qft(n)
    a, _ = unit_csim(n, c, u, 1e-9, normalize=False)
    a.reset_basis(0)
    a.run(gates, 2, 7)
    b = oracle.CSim(n, c, shifts(), oracle.max_bytes_for(c, 1e-9), False)
    b.reset_basis(0)
    b.run(gates, 2, 7)
    for t in range(1 << (n - c)):
        assert a.stream(t) == b.stream(t)
    assert a.alpha == b.alpha


@pytest.mark.parametrize("theta", [4.0, 6.0])
def test_stride_sweeps_one_level_per_stride(theta):
    n, c, u = 12, 5, 8
    x = I.seeded_basis(n)
    gates = I.basis_gates(n, x) + I.qft(n)
    cs, ut = unit_csim(n, c, u, theta)
    cs.reset_basis(0)
    cs.run(gates, 4, 20)
    limit = oracle.max_bytes_for(u, theta)
    last = len(shifts()) - 1
    for s0 in range(0, 1 << (n - c), 1 << ut):
        st = [cs.stream(s0 + j) for j in range(1 << ut)]
        ks = {level_of(s) for s in st}
        assert len(ks) == 1
        assert sum(len(s) for s in st) <= limit or ks == {last}
    psi = cs.dense()
    k = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * k) % (1 << n)) / (1 << n))
    F = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(ref, ref).real * np.vdot(psi, psi).real)
    assert F > 0.999


def test_stride_sweeps_cannot_be_sampled():
    cs, _ = unit_csim(8, 4, 6, 4.0)
    cs.reset_basis(0)
    with pytest.raises(RuntimeError):
        cs.sweep_sample([I.h(0)], [], 0, 1)


def test_level_encoder_special_values():
    # the level encoder keeps the per-tile rules: a non-finite value gives a
    # RAW stream (mode 2) at level 0 and the non-finite flag; a subnormal
    # forces shift 0 but keeps the requested level byte
    c, sh = 4, shifts()
    a = I.random_state(c, I.BASE_SEED + 44)
    st, fl = oracle.encode_tile_level(a, c, sh, 3)
    want, _, _ = oracle.encode_tile(a, c, [sh[3]])
    assert fl == 0 and st[2] == 3 and st[1] == sh[3]
    assert st[:2] + st[3:] == want[:2] + want[3:]
    b = a.copy()
    b[5] = complex(float("nan"), 0.0)
    st, fl = oracle.encode_tile_level(b, c, sh, 3)
    assert fl & 1 and st[0] == 2 and st[2] == 0 and len(st) == 32 + 16 * (1 << c)
    b = a.copy()
    b[7] = complex(5e-324, 0.0)
    st, fl = oracle.encode_tile_level(b, c, sh, 4)
    assert fl & 2 and st[1] == 0 and st[2] == 4
    assert np.array_equal(oracle.decode_tile(st, c).view(np.uint64), b.view(np.uint64))


def test_stride_sweep_on_its_own_matches_the_full_sweep():
    # every stride of every sweep recomputed from the sweep's input streams
    # of the items that hold its tiles, against the full per-stride sweep
    from oracle.partition import partition
    n, c, u, theta = 11, 4, 7, 4.0
    gates = I.basis_gates(n, 0x2A5) + I.qft(n) + I.random_grid(*I.grid_shape(n), 3, 4)
    cs, ut = unit_csim(n, c, u, theta)
    cs.reset_basis(0)
    for lo, hi, H in partition(gates, n, c, 4, 9):
        before = [cs.stream(t) for t in range(1 << (n - c))]
        alpha = cs.alpha
        cs.sweep(gates[lo:hi], H)
        for t0 in range(0, 1 << (n - c), 1 << ut):
            need = oracle.stride_items_tiles(c, H, u, t0)
            got = oracle.stride_sweep(n, c, H, u, theta, t0, {t: before[t] for t in need}, alpha,
                                      gates[lo:hi], shifts())
            assert got == [cs.stream(t0 + j) for j in range(1 << ut)]
    need = oracle.stride_items_tiles(c, [c + 3], u, 0)
    with pytest.raises(RuntimeError):
        oracle.stride_sweep(n, c, [c + 3], u, theta, 0, {t: before[t] for t in need[:-1]}, 1.0,
                            [I.h(c + 3)], shifts())
