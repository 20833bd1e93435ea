"""Seeded synthetic inputs: gate descriptions and circuit generators.

This module is shared by the tests, the benchmark, the CPU oracle drivers
and the GPU binding.  It builds circuits (lists of gates with their 2x2 /
4x4 matrices); it holds none of the simulator's or the codec's arithmetic.

Circuits
  * QFT on a basis state (Sec. IV, the paper's worst case for compression).
  * Grover search (Sec. IV, the paper's best case).
  * Random 2D-grid circuits with sqrt(X), sqrt(Y), sqrt(W) layers and CZ
    on alternating nearest-neighbour patterns (a low-compressibility stress
    input; not in the paper).

Qubit j is bit j of the amplitude index (little-endian).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(state: int) -> tuple[int, int]:
    """One step of SplitMix64 (Steele, Lea, Flood 2014): (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class Rng:
    """Stream of SplitMix64 outputs from a seed."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state, out = splitmix64(self.state)
        return out

    def below(self, m: int) -> int:
        return self.next() % m

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))


BASE_SEED = 20181113


@dataclass(frozen=True)
class Gate:
    """A k-target gate (k = 1 or 2) with optional controls.

    matrix: (2^k, 2^k) complex128; sub-index bit i selects qubit targets[i].
    control_values: required value of each control (default: all 1).
    """

    matrix: np.ndarray
    targets: tuple
    controls: tuple = ()
    control_values: tuple | None = None
    name: str = field(default="", compare=False)

    def cvals(self) -> tuple:
        if self.control_values is None:
            return tuple(1 for _ in self.controls)
        return tuple(self.control_values)

    def masks(self) -> tuple[int, int]:
        """(control mask, required values) over global index bits."""
        cm = cv = 0
        for q, v in zip(self.controls, self.cvals()):
            cm |= 1 << q
            if v:
                cv |= 1 << q
        return cm, cv


S2 = 1.0 / math.sqrt(2.0)
MAT_H = np.array([[S2, S2], [S2, -S2]], dtype=np.complex128)
MAT_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
MAT_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
MAT_SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
MAT_CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
_A = (1 + 1j) / 2
_B = (1 - 1j) / 2
MAT_SQRT_X = np.array([[_A, _B], [_B, _A]], dtype=np.complex128)
MAT_SQRT_Y = np.array([[_A, -_A], [_A, _A]], dtype=np.complex128)
MAT_SQRT_W = np.array([[_A, -1j * S2], [S2, _A]], dtype=np.complex128)


def phase(phi: float) -> np.ndarray:
    return np.array([[1, 0], [0, complex(math.cos(phi), math.sin(phi))]], dtype=np.complex128)


def h(q):
    return Gate(MAT_H, (q,), name="H")


def x(q):
    return Gate(MAT_X, (q,), name="X")


def cphase(phi, control, target):
    return Gate(phase(phi), (target,), (control,), name="CP")


def swap(a, b):
    return Gate(MAT_SWAP, (a, b), name="SWAP")


def cz(a, b):
    return Gate(MAT_CZ, (a, b), name="CZ")


def mcz(n: int, pattern: int) -> Gate:
    """Flip the sign of basis state |pattern> only: a phase gate on qubit 0
    controlled by every other qubit at its value in the pattern."""
    if n == 1:
        mat = MAT_Z if pattern & 1 else np.diag([-1, 1]).astype(np.complex128)
        return Gate(mat, (0,), name="MCZ")
    mat = MAT_Z if pattern & 1 else np.diag([-1, 1]).astype(np.complex128)
    ctrls = tuple(range(1, n))
    vals = tuple((pattern >> q) & 1 for q in ctrls)
    return Gate(mat, (0,), ctrls, vals, name="MCZ")


def qft(n: int) -> list[Gate]:
    """QFT, little-endian: for j = n-1..0: H(j), then for m = j-1..0 the
    controlled phase 2*pi/2^(j-m+1) (control m, target j); then SWAP(j,
    n-1-j) for j < n/2.  Maps |x> to sum_k e^{2 pi i x k / 2^n} |k> / sqrt(2^n)."""
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(h(j))
        for m in range(j - 1, -1, -1):
            gates.append(cphase(2 * math.pi / (1 << (j - m + 1)), m, j))
    for j in range(n // 2):
        gates.append(swap(j, n - 1 - j))
    return gates


def basis_gates(n: int, xval: int) -> list[Gate]:
    """X gates that prepare |xval> from |0...0>."""
    return [x(q) for q in range(n) if (xval >> q) & 1]


def grover(n: int, marked: int, iterations: int) -> list[Gate]:
    """Grover search from |0...0>: H^n, then per iteration the oracle (MCZ
    on the marked pattern) and the diffusion H^n X^n MCZ X^n H^n."""
    ones = (1 << n) - 1
    gates = [h(q) for q in range(n)]
    for _ in range(iterations):
        gates.append(mcz(n, marked))
        gates += [h(q) for q in range(n)]
        gates += [x(q) for q in range(n)]
        gates.append(mcz(n, ones))
        gates += [x(q) for q in range(n)]
        gates += [h(q) for q in range(n)]
    return gates


def grid_shape(n: int) -> tuple[int, int]:
    """rows x cols = n with the factor pair closest to square (rows <= cols)."""
    best = (1, n)
    for r in range(1, int(math.isqrt(n)) + 1):
        if n % r == 0:
            best = (r, n // r)
    return best


def grid_cz_pattern(rows: int, cols: int, which: int) -> list[tuple[int, int]]:
    """CZ pairs of pattern A/B/C/D (which = 0..3), qubit = cols*r + c:
    A horizontal pairs starting at even c, B at odd c, C vertical pairs
    starting at even r, D at odd r."""
    pairs = []
    if which in (0, 1):
        for r in range(rows):
            for c in range(which, cols - 1, 2):
                pairs.append((cols * r + c, cols * r + c + 1))
    else:
        for r in range(which - 2, rows - 1, 2):
            for c in range(cols):
                pairs.append((cols * r + c, cols * (r + 1) + c))
    return pairs


def random_grid(rows: int, cols: int, depth: int, seed: int) -> list[Gate]:
    """Depth layers; each: one gate from {sqrt X, sqrt Y, sqrt W} on every
    qubit (uniform, never the previous choice on that qubit), then the CZ
    pattern A, B, C, D in turn."""
    rng = Rng(seed)
    n = rows * cols
    mats = (MAT_SQRT_X, MAT_SQRT_Y, MAT_SQRT_W)
    names = ("SX", "SY", "SW")
    prev = [-1] * n
    gates = []
    for layer in range(depth):
        for q in range(n):
            if prev[q] < 0:
                choice = rng.below(3)
            else:
                choice = (prev[q] + 1 + rng.below(2)) % 3
            prev[q] = choice
            gates.append(Gate(mats[choice], (q,), name=names[choice]))
        for a, b in grid_cz_pattern(rows, cols, layer % 4):
            gates.append(cz(a, b))
    return gates


def seeded_basis(n: int, seed: int = BASE_SEED) -> int:
    return Rng(seed).next() % (1 << n)


def random_state(n: int, seed: int) -> np.ndarray:
    """A seeded normalised random state (Gaussian components via Box-Muller)."""
    rng = Rng(seed)
    N = 1 << n
    u1 = np.array([rng.uniform() for _ in range(2 * N)])
    u2 = np.array([rng.uniform() for _ in range(2 * N)])
    g = np.sqrt(-2.0 * np.log(1.0 - u1)) * np.cos(2 * math.pi * u2)
    psi = g[0::2] + 1j * g[1::2]
    return psi / np.linalg.norm(psi)


def strided_mix_state(n: int, tile_log2: int, stride_log2: int, seed: int) -> np.ndarray:
    """A seeded state whose strides of 2^stride_log2 amplitudes come in
    four kinds in turn: all zero; Gaussian with the first tile zero; a
    smooth phase ramp; Gaussian (strides that compress very differently)."""
    N, span = 1 << tile_log2, 1 << stride_log2
    psi = random_state(n, seed)
    ramp = np.exp(2j * np.pi * np.arange(1 << n) / (1 << n)) / math.sqrt(1 << n)
    for s0 in range(0, 1 << n, span):
        kind = (s0 // span) % 4
        if kind == 0:
            psi[s0:s0 + span] = 0
        elif kind == 1:
            psi[s0:s0 + N] = 0
        elif kind == 2:
            psi[s0:s0 + span] = ramp[s0:s0 + span]
    return psi
