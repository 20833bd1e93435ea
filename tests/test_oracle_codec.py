"""Pins of the oracle's tile codec (O2).

* Hand-derived streams (tests/golden/codec_examples.txt) fix the byte
  layout, the quantiser, the residual/zigzag/width stage, the packing and
  the mode rule.
* The point-wise relative bound (Sec. III with the relative error bound of
  ref. [xin2018]): every reconstructed component satisfies
  |x^ - x| < 2^(s-53) |x| <= eps |x|, checked exactly (rational arithmetic)
  around every binade boundary and every rounding boundary, and on random
  values.
* Lossless level: bit-exact round trip of arbitrary finite bit patterns.
* Algorithm 2's ladder: the level picked is the first whose stream is
  within max_bytes, else the last (sizes measured level by level).
"""
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "codec_examples.txt")


def d(bits: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def load_examples():
    ex, cur = [], None
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        if not line.startswith(" "):
            name, c, s, *spec = line.split()
            cur = {"name": name, "c": int(c), "s": int(s), "spec": spec, "hex": ""}
            ex.append(cur)
        else:
            cur["hex"] += "".join(line.split())
    return ex


def amplitudes(e):
    N = 1 << e["c"]
    spec = e["spec"]
    if spec == ["ramp"]:
        re = [d(0x3FE0000000000000 + (i << 39)) for i in range(N)]
        return np.array(re, dtype=np.complex128)
    if spec == ["sparse"]:
        re = [d(0x3FE0000000000000 + ((i // 2) << 39)) if i % 2 == 0 else 0.0 for i in range(N)]
        return np.array(re, dtype=np.complex128)
    if spec == ["signs"]:
        out = np.zeros(N, dtype=np.complex128)
        for i in range(N):
            g, l = divmod(i, 32)
            if N == 64:
                word = 0x0F0F0F0F if g == 0 else 0xF0F0F0F0
            else:
                word = 0x0F0F0F0F if g == 2 else 0xFFFFFFFF
            out[i] = -1.0 if (word >> l) & 1 else 1.0
        return out
    vals = []
    for item in spec:
        pair, _, cnt = item.partition("*")
        r, i = pair.split(":")
        vals += [complex(d(int(r, 16)), d(int(i, 16)))] * (int(cnt) if cnt else 1)
    return np.array(vals, dtype=np.complex128)


@pytest.mark.parametrize("e", load_examples(), ids=lambda e: e["name"])
def test_golden_stream(e):
    a = amplitudes(e)
    stream, level, flags = oracle.encode_tile(a, e["c"], [e["s"]])
    assert stream.hex() == e["hex"]
    assert level == 0 and flags == 0
    back = oracle.decode_tile(stream, e["c"])
    if e["s"] == 0 or e["name"] in ("const_c5", "ramp_c5", "signs_c6", "signs_c7", "delta_c6",
                                         "sparse_c5"):
        # these inputs are exactly representable at their shift
        assert back.view(np.uint64).tolist() == a.view(np.uint64).tolist()


def test_shift_for_eps():
    # largest s with 2^(s-53) <= eps, checked with exact rationals
    for eps in (1e-2, 1e-3, 1e-4, 1e-5, 1e-8, 0.3, 2.0**-53, 2.0**-54, 0.0):
        s = oracle.shift_for_eps(eps)
        if s == 0:
            assert Fraction(eps) < Fraction(2) ** (1 - 53)
        else:
            assert Fraction(2) ** (s - 53) <= Fraction(eps)
            assert s == 52 or Fraction(2) ** (s + 1 - 53) > Fraction(eps)
    assert [oracle.shift_for_eps(e) for e in (1e-2, 1e-3, 1e-4, 1e-5)] == [46, 43, 39, 36]


def roundtrip_components(vals: np.ndarray, s: int, c: int = 10) -> np.ndarray:
    """Encode/decode the components, 2^c amplitudes per tile."""
    comps = np.ascontiguousarray(vals, dtype=np.float64)
    per = 2 << c
    pad = (-comps.size) % per
    comps = np.concatenate([comps, np.full(pad, 0.5)])
    out = np.empty_like(comps)
    for t in range(comps.size // per):
        a = comps[t * per:(t + 1) * per].view(np.complex128)
        stream, _, flags = oracle.encode_tile(a, c, [s])
        assert flags & 1 == 0          # 2 = lossless forced (fine at s = 0)
        out[t * per:(t + 1) * per] = oracle.decode_tile(stream, c).view(np.float64)
    return out[:vals.size]


def boundary_values(s: int) -> np.ndarray:
    """Magnitude bit patterns around every binade start and around the
    rounding points k*2^s + 2^(s-1) nearest to it, both signs."""
    pats = []
    for E in range(1, 2046):
        base = E << 52
        for k in (-2, -1, 0, 1):
            mid = base + k * (1 << s) + (1 << (s - 1))
            for dd in (-2, -1, 0, 1, 2):
                pats.append(mid + dd)
        for dd in (-1, 0, 1, 2):
            pats.append(base + dd)
    pats = [p for p in pats if 0x0010000000000000 <= p < 0x7FE0000000000000]
    arr = np.array(pats, dtype=np.uint64)
    arr = np.concatenate([arr, arr | np.uint64(1 << 63)])
    return arr.view(np.float64)


@pytest.mark.parametrize("s", [36, 39, 43, 46, 52])
def test_relative_bound_exact_at_boundaries(s):
    x = boundary_values(s)
    xr = roundtrip_components(x, s)
    bound = Fraction(2) ** (s - 53)
    for a, b in zip(x.tolist(), xr.tolist()):
        fa, fb = Fraction(a), Fraction(b)
        assert abs(fb - fa) < bound * abs(fa), (s, a, b)
        assert (a < 0) == (b < 0)


@pytest.mark.parametrize("s", [36, 39, 43, 46])
def test_relative_bound_random(s):
    rng = np.random.default_rng(s)
    # magnitudes over a wide exponent range, both signs
    e = rng.integers(-300, 300, size=400_000)
    m = rng.random(400_000) + 1.0
    x = np.ldexp(m, e) * np.where(rng.random(400_000) < 0.5, -1.0, 1.0)
    xr = roundtrip_components(x, s)
    diff = np.abs(xr - x)                # exact (Sterbenz: xr/x in [1/2, 2])
    assert np.all(diff < np.ldexp(np.abs(x), s - 53))
    eps = {36: 1e-5, 39: 1e-4, 43: 1e-3, 46: 1e-2}[s]
    assert np.all(diff <= eps * np.abs(x))
    assert np.all(np.signbit(xr) == np.signbit(x))


def test_lossless_roundtrip_bit_exact():
    rng = np.random.default_rng(5)
    pats = rng.integers(0, 2**63, size=60_000, dtype=np.uint64)
    pats ^= rng.integers(0, 2, size=pats.size, dtype=np.uint64) << np.uint64(63)
    pats = pats[(pats & np.uint64(0x7FF0000000000000)) != np.uint64(0x7FF0000000000000)]
    edge = [0x0, 1 << 63, 1, 0x000FFFFFFFFFFFFF, 0x0010000000000000, 0x3FF0000000000000,
            0x3FEFFFFFFFFFFFFF, 0x7FEFFFFFFFFFFFFF, 0x7FE0000000000000, 0x3CA0000000000000,
            0x8000000000000001]
    pats = np.concatenate([np.array(edge, dtype=np.uint64), pats])
    x = pats.view(np.float64)
    for c in (1, 4, 5, 6, 10):
        xr = roundtrip_components(x, 0, c)
        assert np.array_equal(xr.view(np.uint64), x.view(np.uint64))


def test_out_of_lossy_range_forces_lossless():
    a = np.full(64, 0.3 + 0.1j)
    a[7] = complex(d(0x0000000000000123), 0.2)      # subnormal component
    stream, _, flags = oracle.encode_tile(a, 6, [39])
    back = oracle.decode_tile(stream, 6)
    assert flags == 2
    assert np.array_equal(back.view(np.uint64), a.view(np.uint64))
    a[7] = complex(d(0x7FE0000000000001), 0.2)      # |x| >= 2^1023
    stream, _, flags = oracle.encode_tile(a, 6, [39])
    assert flags == 2
    assert np.array_equal(oracle.decode_tile(stream, 6).view(np.uint64), a.view(np.uint64))


def test_nonfinite_is_flagged_and_kept_raw():
    a = np.full(32, 0.5 + 0.5j)
    a[3] = complex(float("nan"), 0.0)
    stream, _, flags = oracle.encode_tile(a, 5, [39])
    assert flags == 1 and stream[0] == 2
    back = oracle.decode_tile(stream, 5)
    assert np.array_equal(back.view(np.uint64), a.view(np.uint64))


def test_zero_tile_and_signed_zeros():
    a = np.zeros(256, dtype=np.complex128)
    stream, _, _ = oracle.encode_tile(a, 8, [39])
    assert len(stream) == 32 and stream[0] == 0          # header only
    a = np.zeros(256, dtype=np.complex128)
    a.real[5] = -0.0
    # lossy level: a zero's sign is not kept, the tile is still CONST
    stream, _, _ = oracle.encode_tile(a, 8, [39])
    assert len(stream) == 32 and stream[0] == 0
    assert np.array_equal(oracle.decode_tile(stream, 8).view(np.uint64), np.zeros(512, np.uint64))
    # lossless level: bit-exact, -0 included
    stream, _, _ = oracle.encode_tile(a, 8, [0])
    back = oracle.decode_tile(stream, 8)
    assert np.array_equal(back.view(np.uint64), a.view(np.uint64))


def test_ladder_picks_first_level_within_limit():
    rng = np.random.default_rng(11)
    shifts = [0, 36, 39, 43, 46]
    c = 8
    for trial in range(40):
        ph = rng.random(1 << c) * 2 * np.pi * (trial % 7 + 1)
        a = np.exp(1j * np.cumsum(ph) / 50) / 16.0
        if trial % 3 == 0:
            a = a * (1 + 0.5 * rng.random(1 << c))
        sizes = [len(oracle.encode_tile(a, c, [s])[0]) for s in shifts]
        for theta in (1.0, 1.5, 2, 3, 4, 6, 8, 16, 1e9):
            mb = oracle.max_bytes_for(c, theta)
            stream, level, _ = oracle.encode_tile(a, c, shifts, mb)
            want = next((k for k, sz in enumerate(sizes) if sz <= mb), len(shifts) - 1)
            assert level == want
            assert len(stream) == sizes[want]
            assert stream[2] == want
            single = oracle.encode_tile(a, c, [shifts[want]])[0]
            assert stream[:2] + stream[3:] == single[:2] + single[3:]


def test_malformed_streams_are_rejected():
    a = np.exp(1j * (np.arange(64) * 0.37 + 0.1)) / 8
    stream, _, _ = oracle.encode_tile(a, 6, [39])
    with pytest.raises(ValueError):
        oracle.decode_tile(stream[:20], 6)                # short header
    with pytest.raises(ValueError):
        oracle.decode_tile(stream[:-16], 6)               # short body
    bad = bytearray(stream)
    bad[24] = 7                                           # wrong tile size
    with pytest.raises(ValueError):
        oracle.decode_tile(bytes(bad), 6)
    assert stream[0] == 1
    # a phase ramp: nonzero, mixed signs; no zero sections, sign words in
    # mode 4 (two groups of mixed words)
    assert stream[3] == 4 | 4 << 3 and stream[25] == 0
    woff = 32 + 8 + 8
    bad = bytearray(stream)
    bad[woff] = 65                                        # width > 64
    with pytest.raises(ValueError):
        oracle.decode_tile(bytes(bad), 6)
    bad = bytearray(stream)
    bad[woff] = 64                                        # data past the body
    with pytest.raises(ValueError):
        oracle.decode_tile(bytes(bad), 6)


@pytest.mark.parametrize("s", [0, 39])
def test_sparse_tiles_keep_zeros_and_bound(s):
    """Zero words: zero components (either sign) come back bit-exact, the
    others within the bound, for tiles from fully dense to a single spike."""
    rng = np.random.default_rng(17 + s)
    c = 8
    N = 1 << c
    for frac in (0.0, 0.3, 0.7, 0.97, 1.0):
        comps = rng.standard_normal(2 * N) / 16
        comps[rng.random(2 * N) < frac] = 0.0
        neg0 = (comps == 0) & (rng.random(2 * N) < 0.5)
        comps[neg0] = -0.0
        a = comps.view(np.complex128)
        stream, _, flags = oracle.encode_tile(a, c, [s])
        assert flags & 1 == 0
        back = oracle.decode_tile(stream, c).view(np.float64)
        z = comps == 0
        # zeros come back exactly; their sign only at the lossless level
        want = comps[z] if s == 0 else np.zeros(int(z.sum()))
        assert np.array_equal(back[z].view(np.uint64), want.view(np.uint64))
        if s == 0:
            assert np.array_equal(back.view(np.uint64), comps.view(np.uint64))
        else:
            diff = np.abs(back[~z] - comps[~z])
            assert np.all(diff < np.ldexp(np.abs(comps[~z]), s - 53))


def test_single_spike_tile_is_small():
    """A tile holding one nonzero amplitude costs a header, the zero words
    and the width bytes, not a word per value."""
    c = 8
    for pos in (0, 77, 255):
        a = np.zeros(1 << c, dtype=np.complex128)
        a[pos] = 0.3 - 0.7j
        stream, _, _ = oracle.encode_tile(a, c, [39])
        # header 32 + re zero exceptions 8 + im sign exceptions 8 + im
        # zero exceptions 8 + 16 width bytes = 72 -> body padded: 80
        assert stream[0] == 1 and len(stream) == 80
        back = oracle.decode_tile(stream, c)
        assert np.count_nonzero(back) == 1 and abs(back[pos] - a[pos]) < 1e-4


def test_relative_bound_hundred_million_values():
    # 1.04*10^8 seeded magnitudes through the oracle's quantiser: 2*10^6 at
    # each shift 1..52 (the binades below 2^-962 are covered exactly above);
    # a truncating quantiser would exceed the bound by up to a factor 2
    bad = sum(oracle.check_bound(s, 2_000_000, 0x5EED + s) for s in range(1, 53))
    assert bad == 0


def _sections_end(stream: bytes, G: int) -> int:
    """Body offset after the four word sections (signs re/im, zeros re/im)."""
    w0, = struct.unpack_from("<I", stream, 0)
    w6, = struct.unpack_from("<I", stream, 24)
    modes = [(w0 >> 24) & 7, (w0 >> 27) & 7, (w6 >> 8) & 7, (w6 >> 11) & 7]
    off = 0
    for m in modes:
        if m in (2, 3):          # exceptions: a bitmap word, then one word per set bit
            bm, = struct.unpack_from("<I", stream, 32 + off)
            off += 4 + 4 * bin(bm & ((1 << G) - 1)).count("1")
        elif m == 4:             # every word
            off += 4 * G
    return off


@pytest.mark.parametrize("s", [0, 21, 39, 52])
def test_one_amplitude_stream_is_its_anchors(s):
    """A tile that is +0 but for one amplitude: the first nonzero value of a
    component is coded against itself, so every residual and every width
    byte is zero and the header's anchors hold the amplitude's codes (the
    property a decoder may use to read such a tile from its header and
    sections alone)."""
    c = 8
    G = (1 << c) >> 5
    rng = np.random.default_rng(s)
    for pos in (0, 31, 32, 200, 255):
        for v in (complex(rng.normal(), rng.normal()), complex(-abs(rng.normal()), 0.0),
                  complex(0.0, rng.normal())):
            a = np.zeros(1 << c, dtype=np.complex128)
            a[pos] = v
            stream, _, _ = oracle.encode_tile(a, c, [s])
            assert stream[0] == 1                                   # PACKED
            body, = struct.unpack_from("<I", stream, 4)
            assert len(stream) == 32 + body
            a0, a1 = struct.unpack_from("<QQ", stream, 8)
            for comp, anc in ((v.real, a0), (v.imag, a1)):
                B = bits(comp) & ((1 << 63) - 1)
                q = B if s == 0 else (B + (1 << (s - 1))) >> s
                assert anc == q
            off = _sections_end(stream, G)
            widths = stream[32 + off: 32 + off + 2 * G]
            assert widths == bytes(2 * G)
            assert stream[32 + off:] == bytes(len(stream) - 32 - off)   # no data words
            back = oracle.decode_tile(stream, c)
            assert np.count_nonzero(back) == 1
            others = np.delete(back, pos)
            assert not np.any(others.view(np.uint64))                # every other entry +0
