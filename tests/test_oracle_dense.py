"""Pins of the oracle's dense simulator (O1) against mathematics.

* Sec. II: a single-qubit gate on qubit k is A = I x ... x U x ... x I;
  checked against numpy Kronecker products.
* Controlled and two-target gates: checked against the operator built
  column by column from its definition on basis states.
* QFT on a basis state: e^{2 pi i x k / N} / sqrt(N) (closed form).
* Grover: (-1)^k [sin((2k+1)t)|m> + cos((2k+1)t)/sqrt(N-1) sum_{i!=m} |i>],
  sin t = 1/sqrt(N).
* Random grid circuits preserve the norm.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I


def kron_single(n, k, U):
    """I x ... x U x ... x I with qubit n-1 leftmost (index bit j = qubit j)."""
    A = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        A = np.kron(A, U if q == k else np.eye(2))
    return A


def operator_from_definition(n, gate):
    """Column b of the operator: if the controls hold on b, row r of U
    sends b to b with its target bits replaced by r, weight U[r, s]."""
    N = 1 << n
    A = np.zeros((N, N), dtype=np.complex128)
    k = len(gate.targets)
    for b in range(N):
        ok = all(((b >> q) & 1) == v for q, v in zip(gate.controls, gate.cvals()))
        if not ok:
            A[b, b] = 1
            continue
        s = sum(((b >> t) & 1) << i for i, t in enumerate(gate.targets))
        for r in range(1 << k):
            out = b
            for i, t in enumerate(gate.targets):
                out = (out & ~(1 << t)) | (((r >> i) & 1) << t)
            A[out, b] += gate.matrix[r, s]
    return A


def random_matrix(rng, dim):
    """Random complex matrix whose entries cover every class the oracle
    distinguishes: general, real, imaginary and zero."""
    M = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    for r in range(dim):
        for c in range(dim):
            kind = rng.integers(0, 4)
            if kind == 1:
                M[r, c] = M[r, c].real
            elif kind == 2:
                M[r, c] = 1j * M[r, c].imag
            elif kind == 3 and r != c:
                M[r, c] = 0
    return M


def random_state(rng, n):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_single_qubit_is_kronecker_product(n):
    rng = np.random.default_rng(100 + n)
    for k in range(n):
        U = random_matrix(rng, 2)
        psi = random_state(rng, n)
        ref = kron_single(n, k, U) @ psi
        out = psi.copy()
        oracle.dense_apply(out, n, I.Gate(U, (k,)))
        assert np.max(np.abs(out - ref)) < 1e-14


@pytest.mark.parametrize("n", [3, 5, 8])
def test_controlled_and_two_target_gates_match_definition(n):
    rng = np.random.default_rng(200 + n)
    for trial in range(12):
        k = 1 + trial % 2
        qs = rng.permutation(n)
        targets = tuple(int(q) for q in qs[:k])
        nc = int(rng.integers(0, min(3, n - k) + 1))
        controls = tuple(int(q) for q in qs[k:k + nc])
        vals = tuple(int(v) for v in rng.integers(0, 2, size=nc))
        g = I.Gate(random_matrix(rng, 1 << k), targets, controls, vals)
        psi = random_state(rng, n)
        ref = operator_from_definition(n, g) @ psi
        out = psi.copy()
        oracle.dense_apply(out, n, g)
        assert np.max(np.abs(out - ref)) < 1e-14, (targets, controls, vals)


def test_diagonal_gate_on_any_qubit_and_swap_is_permutation():
    n = 6
    rng = np.random.default_rng(7)
    psi = random_state(rng, n)
    out = psi.copy()
    oracle.dense_apply(out, n, I.swap(1, 4))
    idx = np.arange(1 << n)
    swapped = (idx & ~0b10010) | (((idx >> 1) & 1) << 4) | (((idx >> 4) & 1) << 1)
    assert np.array_equal(out[swapped], psi)   # exact: entries equal to 1 copy
    out = psi.copy()
    oracle.dense_apply(out, n, I.cz(0, 5))
    sign = np.where(((idx & 1) == 1) & (((idx >> 5) & 1) == 1), -1.0, 1.0)
    assert np.array_equal(out, psi * sign)


@pytest.mark.parametrize("n", [3, 7, 12])
def test_qft_of_basis_state_closed_form(n):
    N = 1 << n
    for xval in (0, 1, I.seeded_basis(n), N - 1):
        psi = oracle.dense_basis(n, xval)
        oracle.dense_run(psi, n, I.qft(n))
        k = np.arange(N)
        ref = np.exp(2j * np.pi * ((xval * k) % N) / N) / math.sqrt(N)
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_qft3_golden_values():
    """QFT_8 |5>: amplitude k = e^{2 pi i 5k/8}/sqrt(8), written out from
    the closed form (tests/golden/qft3_x5.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "qft3_x5.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    ref = np.array([float(r[1]) + 1j * float(r[2]) for r in rows])
    psi = oracle.dense_basis(3, 5)
    oracle.dense_run(psi, 3, I.qft(3))
    assert np.max(np.abs(psi - ref)) < 1e-15


@pytest.mark.parametrize("n,marked", [(5, 19), (6, 0), (8, 173)])
def test_grover_closed_form(n, marked):
    N = 1 << n
    t = math.asin(1 / math.sqrt(N))
    for it in range(1, 5):
        psi = oracle.dense_zero(n)
        oracle.dense_run(psi, n, I.grover(n, marked, it))
        a_m = (-1) ** it * math.sin((2 * it + 1) * t)
        a_o = (-1) ** it * math.cos((2 * it + 1) * t) / math.sqrt(N - 1)
        ref = np.full(N, a_o, dtype=np.complex128)
        ref[marked] = a_m
        assert np.max(np.abs(psi - ref)) < 1e-12


def test_random_grid_preserves_norm():
    rows, cols = I.grid_shape(12)
    n = rows * cols
    psi = oracle.dense_zero(n)
    oracle.dense_run(psi, n, I.random_grid(rows, cols, 20, I.BASE_SEED))
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    # the circuit actually spreads the state
    assert np.count_nonzero(np.abs(psi) > 1e-6) > (1 << n) // 2


def test_non_diagonal_gate_needs_its_target():
    # the dense apply rejects nothing for full states; a 2-target gate with
    # an out-of-range target is a caller error caught on the Python side
    psi = oracle.dense_zero(3)
    oracle.dense_apply(psi, 3, I.h(2))
    assert abs(psi[0] - I.S2) < 1e-16 and abs(psi[4] - I.S2) < 1e-16


def unit_factor_matrix(rng, dim):
    """Rows whose nonzero entries are f * d, f in {1, -1, i, -i}, d the
    row's first nonzero entry of a random class: the factored rows."""
    M = np.zeros((dim, dim), dtype=np.complex128)
    for r in range(dim):
        d = complex(rng.normal(), rng.normal())
        kind = rng.integers(0, 3)
        if kind == 1:
            d = complex(d.real, 0.0)
        elif kind == 2:
            d = complex(0.0, d.imag)
        cols = [c for c in range(dim) if c == 0 or rng.random() < 0.8]
        for j, c in enumerate(cols):
            M[r, c] = d if j == 0 else d * [1, -1, 1j, -1j][rng.integers(0, 4)]
    return M


@pytest.mark.parametrize("n", [2, 4, 6])
def test_factored_rows_match_definition(n):
    rng = np.random.default_rng(300 + n)
    for trial in range(16):
        k = 1 + trial % 2
        targets = tuple(int(q) for q in rng.permutation(n)[:k])
        g = I.Gate(unit_factor_matrix(rng, 1 << k), targets)
        psi = random_state(rng, n)
        ref = operator_from_definition(n, g) @ psi
        out = psi.copy()
        oracle.dense_apply(out, n, g)
        assert np.max(np.abs(out - ref)) < 1e-14, (targets, g.matrix)


def test_hadamards_cancel_equal_amplitudes_exactly():
    """A Hadamard row is factored: on a uniform state H on every qubit
    leaves exact zeros everywhere but index 0, and H on one qubit of a
    pairwise-equal state leaves exact zeros in the odd half."""
    n = 8
    psi = np.full(1 << n, complex(0.37, -0.21))
    for q in range(n):
        oracle.dense_apply(psi, n, I.h(q))
    assert np.count_nonzero(psi) == 1 and abs(psi[0] - 16 * complex(0.37, -0.21)) < 1e-13
    rng = np.random.default_rng(9)
    half = rng.normal(size=1 << (n - 1)) + 1j * rng.normal(size=1 << (n - 1))
    psi = np.repeat(half, 2)                     # equal in qubit 0
    oracle.dense_apply(psi, n, I.h(0))
    assert np.all(psi[1::2] == 0)
