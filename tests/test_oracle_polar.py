"""Pins of the oracle's POLAR tile mode (a codec variant: magnitude and
phase instead of the two components).

* The angle table equals round(2^64 atan(2^-k) / (2 pi)), computed here
  independently with Python's decimal arithmetic (Machin's formula for pi,
  the arctangent series for atan(2^-k)).
* The integer CORDIC angle of (x, y) matches atan2(y, x) / (2 pi) within
  its 30-step residual (below 3e-10 turn) in every quadrant and for
  components of very different size.
* Every amplitude a POLAR stream decodes to satisfies the level's bound on
  the complex amplitude, |a^ - a| <= 2^(s-53) |a|, checked in exact
  rational arithmetic, over tiles of wide dynamic range with zeros and
  amplitudes with one zero component, at shifts 8 .. 52.
* Tiles of equal magnitudes and phases linear in the index (the QFT's
  tiles) code to at least 30 times smaller streams; the mode is kept only
  when shorter than the componentwise stream; tiles it cannot serve (a
  component below 2^-400, shifts below 8, the lossless level) never use it.
* The bitwise-linear angle predictor (mode 4: a dense tile's angles from
  the angle at index 0 and one difference per index bit) gives a product
  state over the index bits zero residuals up to rounding: such a tile
  codes about as small as a linear one, and far smaller than with the
  order-2 predictor alone.
* The compressed QFT with the variant on keeps the paper's fidelity.
"""
import decimal
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I


def atan_decimal(x: decimal.Decimal, prec: int) -> decimal.Decimal:
    total, term, k = decimal.Decimal(0), x, 0
    x2 = x * x
    eps = decimal.Decimal(10) ** (-prec)
    while abs(term) > eps:
        total += term / (2 * k + 1) * (1 if k % 2 == 0 else -1)
        term *= x2
        k += 1
    return total


def test_angle_table_is_correctly_rounded():
    decimal.getcontext().prec = 80
    D = decimal.Decimal
    pi = 16 * atan_decimal(D(1) / 5, 78) - 4 * atan_decimal(D(1) / 239, 78)       # Machin
    table = oracle.polar_table(30)
    for k, got in enumerate(table):
        a = pi / 4 if k == 0 else atan_decimal(D(2) ** -k, 78)
        want = int((a / (2 * pi) * (D(2) ** 64)).to_integral_value(rounding=decimal.ROUND_HALF_EVEN))
        assert got == want, k


def test_cordic_angle_matches_atan2():
    rng = np.random.default_rng(3)
    pts = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0), (1.0, 1.0), (-1.0, -1.0), (3e-300, 1.0),
           (1.0, -5e-200), (-2.5, 1e-17)]
    for _ in range(400):
        x, y = rng.normal(size=2) * np.ldexp(1.0, rng.integers(-300, 3, 2))
        pts.append((float(x), float(y)))
    for x, y in pts:
        got = oracle.polar_angle(x, y) / 2.0 ** 64
        want = (math.atan2(y, x) / (2 * math.pi)) % 1.0
        d = abs((got - want + 0.5) % 1.0 - 0.5)
        assert d < 3e-10, (x, y, got, want)


def random_tile(rng, c):
    N = 1 << c
    mag = np.ldexp(rng.uniform(0.5, 1.0, N), rng.integers(-60, 4, N))
    ph = rng.uniform(0, 2 * np.pi, N)
    a = mag * np.exp(1j * ph)
    a[rng.random(N) < 0.1] = 0.0
    pick = rng.random(N)
    a[pick < 0.05] = a[pick < 0.05].real + 0j                  # one zero component
    a[(pick >= 0.05) & (pick < 0.1)] = 1j * a[(pick >= 0.05) & (pick < 0.1)].imag
    return a


def exact_within(dec, a, s):
    bound = Fraction(2) ** (2 * (s - 53))
    for d, x in zip(dec.tolist(), a.tolist()):
        dr = Fraction(d.real) - Fraction(x.real)
        di = Fraction(d.imag) - Fraction(x.imag)
        mag2 = Fraction(x.real) ** 2 + Fraction(x.imag) ** 2
        if not dr * dr + di * di <= bound * mag2:
            return False
        if mag2 == 0 and (d.real != 0 or d.imag != 0):
            return False
    return True


@pytest.mark.parametrize("s", [8, 20, 30, 36, 39, 43, 46, 52])
def test_polar_streams_meet_the_bound(s):
    rng = np.random.default_rng(100 + s)
    used = 0
    for t in range(6):
        c = 5 if t % 2 else 8
        a = random_tile(rng, c)
        if t >= 3:                                             # smoother: polar pays off
            k = np.arange(1 << c)
            a = np.abs(a).max() * np.exp(2j * np.pi * (0.01 * k + 0.3)) * (np.abs(a) > 0)
        st, _, _ = oracle.encode_tile(a, c, [s], polar=True)
        dec = oracle.decode_tile(st, c)
        if st[0] in (3, 4):
            used += 1
            assert exact_within(dec, a, s)
        st0, _, _ = oracle.encode_tile(a, c, [s])
        assert len(st) <= len(st0)                             # only when shorter
    if s >= 36:
        assert used >= 3


def test_linear_phase_tiles_code_small_and_ineligible_tiles_do_not_use_polar():
    c = 8
    k = np.arange(1 << c)
    for x in (1, 77, 12345, 2 ** 27 - 3):
        a = np.exp(2j * np.pi * x * k / 2 ** 28) / 2 ** 14
        for eps in (1e-3, 1e-4, 1e-5):
            s = oracle.shift_for_eps(eps)
            st, _, _ = oracle.encode_tile(a, c, [s], polar=True)
            assert st[0] in (3, 4) and 16 * (1 << c) / len(st) >= 30
            assert exact_within(oracle.decode_tile(st, c), a, s)
    a = np.exp(2j * np.pi * 5 * k / 2 ** 20) / 16
    a[4] = 2.0 ** -420 + 0j                                    # below 2^-400: the mode cannot serve it
    st, _, _ = oracle.encode_tile(a, c, [39], polar=True)
    assert st[0] not in (3, 4)
    b = np.exp(2j * np.pi * 5 * k / 2 ** 20) / 16
    for s in (0, 4, 7):
        st, _, _ = oracle.encode_tile(b, c, [s], polar=True)
        assert st[0] not in (3, 4)


def test_compressed_qft_with_polar_keeps_fidelity_and_shrinks():
    n, c = 12, 8
    x = I.seeded_basis(n)
    k = np.arange(1 << n)
    ref = np.exp(2j * np.pi * ((x * k) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    sizes = {}
    for polar in (False, True):
        cs = oracle.CSim(n, c, [oracle.shift_for_eps(1e-4)], None, True, polar=polar)
        cs.reset_basis(x)
        cs.run(I.qft(n), 4, 512)
        psi = cs.dense()
        F = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
        assert F >= 0.9999
        sizes[polar] = cs.nbytes()
    assert sizes[True] * 4 < sizes[False]


def test_bitwise_linear_phases_use_the_bitwise_predictor():
    # phases sum_b phi_b k_b with unrelated phi_b (a product state over the
    # index bits, the QFT before its swaps): mode 4, small, within the bound
    c = 8
    rng = np.random.default_rng(41)
    phi = rng.uniform(0, 2 * np.pi, c)
    k = np.arange(1 << c)
    bits = (k[:, None] >> np.arange(c)) & 1
    a = np.exp(1j * (bits @ phi)) / 2 ** 10
    for eps in (1e-2, 1e-4, 1e-5):
        s = oracle.shift_for_eps(eps)
        st, _, _ = oracle.encode_tile(a, c, [s], polar=True)
        assert st[0] == 4 and 16 * (1 << c) / len(st) >= 25, (eps, len(st))
        assert exact_within(oracle.decode_tile(st, c), a, s)
    a[17] = 0.0                                                # a zero amplitude: order 2 only
    st, _, _ = oracle.encode_tile(a, c, [oracle.shift_for_eps(1e-4)], polar=True)
    assert st[0] == 3
