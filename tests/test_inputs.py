"""Seeded input generators: published SplitMix64 outputs, circuit shapes."""
import numpy as np

from paper_1811_05140_gb300 import inputs as I


def test_splitmix64_published_vector():
    # SplitMix64 from state 0: the first three outputs of the reference
    # algorithm (Steele, Lea, Flood 2014; the 0x9E3779B97F4A7C15 increment)
    r = I.Rng(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                            0x06C45D188009454F]


def test_gate_counts():
    n = 28
    assert len(I.qft(n)) == n + n * (n - 1) // 2 + n // 2 == 420
    assert len(I.grover(36, 5, 8)) == 36 + 8 * (2 + 4 * 36) == 1204
    g = I.random_grid(5, 6, 20, I.BASE_SEED)
    assert sum(len(x.targets) == 1 for x in g) == 600
    assert sum(len(x.targets) == 2 for x in g) == 245


def test_grid_patterns_cover_nearest_neighbours():
    rows, cols = 5, 6
    pats = [I.grid_cz_pattern(rows, cols, w) for w in range(4)]
    assert [len(p) for p in pats] == [15, 10, 12, 12]
    allpairs = {tuple(sorted(p)) for pat in pats for p in pat}
    assert len(allpairs) == 49          # every grid edge exactly once
    for a, b in allpairs:
        ra, ca = divmod(a, cols)
        rb, cb = divmod(b, cols)
        assert abs(ra - rb) + abs(ca - cb) == 1


def test_random_grid_never_repeats_a_qubits_gate():
    g = I.random_grid(3, 4, 12, 77)
    last = {}
    for x in g:
        if len(x.targets) == 1:
            q = x.targets[0]
            assert last.get(q) != x.name
            last[q] = x.name


def test_gate_matrices_are_unitary():
    for M in (I.MAT_H, I.MAT_X, I.MAT_SQRT_X, I.MAT_SQRT_Y, I.MAT_SQRT_W, I.MAT_SWAP,
              I.MAT_CZ, I.phase(0.7)):
        assert np.allclose(M.conj().T @ M, np.eye(M.shape[0]), atol=1e-15)
    assert np.allclose(I.MAT_SQRT_X @ I.MAT_SQRT_X, I.MAT_X)
    Y = np.array([[0, -1j], [1j, 0]])
    assert np.allclose(I.MAT_SQRT_Y @ I.MAT_SQRT_Y, Y)
    W = (I.MAT_X + Y) / np.sqrt(2)
    assert np.allclose(I.MAT_SQRT_W @ I.MAT_SQRT_W, W)
