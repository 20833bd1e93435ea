"""GPU parity: the CUDA path against the CPU oracle, through the C ABI.

Bar (integer and byte work is exact; floating point follows one canonical
operation order on both sides):
  * every tile stream the GPU writes is byte-identical to the oracle's for
    the same input, sweep partition and ladder (codec codes, lossless
    stages, modes, widths, signs and packing included);
  * GPU streams decode in the oracle, oracle streams decode on the GPU;
  * read-outs: amplitudes bit-exact, probabilities equal to the exactly
    summed oracle values, fidelity within 1e-12 of numpy.
"""
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


def oracle_cfg(codec, eps, c, aalc=None):
    if codec == "lossless":
        return [0], None, False
    if codec == "rel":
        return [oracle.shift_for_eps(eps)], None, True
    if codec == "aalc":
        theta, levels = aalc
        return [0] + [oracle.shift_for_eps(e) for e in levels], oracle.max_bytes_for(c, theta), True
    raise ValueError(codec)


def run_both(n, b, codec, eps, gates, x=0, hmax=4, depth=None, aalc=None):
    c = min(b, n, 8)
    st = qsim.State(n, b, codec, eps)
    if hmax != 4 or depth is not None:
        st.set_schedule(c, hmax, depth or 512)
    depth = st.stats()["depth"]
    if aalc:
        st.set_aalc(*aalc)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    shifts, mb, norm = oracle_cfg(codec, eps, c, aalc)
    cs = oracle.CSim(n, c, shifts, mb, norm)
    cs.reset_basis(x)
    cs.run(gates, hmax, depth)
    return st, cs, c


def assert_same_streams(st, cs, n, c):
    got = st.export_tiles()
    assert len(got) == 1 << (n - c)
    for t, s in enumerate(got):
        want = cs.stream(t)
        assert s == want, f"tile {t}: gpu {s[:40].hex()} oracle {want[:40].hex()}"


def qft_ref(n, x):
    k = np.arange(1 << n)
    return np.exp(2j * np.pi * ((x * k) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)


def fid(a, b):
    return abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real)


def test_qft12_rel_1e4_blocks_of_256():
    """12-qubit QFT on a seeded basis state, tiles of 2^8, relative bound 1e-4."""
    n, b = 12, 8
    x = I.seeded_basis(n)
    st, cs, c = run_both(n, b, "rel", 1e-4, I.qft(n), x=x)
    assert_same_streams(st, cs, n, c)
    psi = cs.dense()
    assert np.array_equal(st.amplitudes().view(np.uint64), psi.view(np.uint64))
    F = st.fidelity_qft(x)
    assert abs(F - fid(qft_ref(n, x), psi)) < 1e-12
    assert F >= 0.9999
    assert st.stats()["alpha"] == cs.alpha


@pytest.mark.parametrize("codec,eps", [("rel", 1e-2), ("rel", 1e-3), ("rel", 1e-5), ("lossless", 0.0)])
def test_random_grid_streams(codec, eps):
    rows, cols = 3, 4
    gates = I.random_grid(rows, cols, 10, I.BASE_SEED + 1)
    st, cs, c = run_both(rows * cols, 6, codec, eps, gates)
    assert_same_streams(st, cs, rows * cols, c)
    assert st.stats()["alpha"] == cs.alpha


def test_grover_streams_and_closed_form():
    n, m = 10, 613
    st, cs, c = run_both(n, 6, "rel", 1e-4, I.grover(n, m, 3))
    assert_same_streams(st, cs, n, c)
    assert st.fidelity_grover(m, 3) > 0.9999


@pytest.mark.parametrize("depth", [1, 3, 48, 49, 97, 512])
def test_fusion_depths(depth):
    n = 10
    gates = I.basis_gates(n, 0x2D3) + I.qft(n)
    st, cs, c = run_both(n, 5, "rel", 1e-3, gates, depth=depth)
    assert_same_streams(st, cs, n, c)


def test_long_sweep_many_gate_chunks():
    # about 500 gates in one sweep: the compact gates pass through shared
    # memory in chunks of 48, skipped chunks included
    n = 10
    gates = I.random_grid(2, 5, 40, 12) + I.qft(n)
    st, cs, c = run_both(n, 10, "rel", 1e-4, gates)
    assert st.stats()["sweeps"] <= 2
    assert_same_streams(st, cs, n, c)


def test_pair_limit_one():
    n = 9
    gates = [g for g in I.random_grid(3, 3, 6, 8) if len(g.targets) == 1] + [I.h(q) for q in range(n)]
    st, cs, c = run_both(n, 4, "rel", 1e-4, gates, hmax=1, depth=8)
    assert_same_streams(st, cs, n, c)


def random_unitary(rng, dim):
    z = rng.normal(size=(dim, dim)) + 1j * rng.normal(size=(dim, dim))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_general_two_target_gates_with_controls():
    rng = np.random.default_rng(9)
    n = 11
    gates = [I.h(q) for q in range(n)]
    for i in range(40):
        k = 1 + i % 2
        qs = rng.permutation(n)
        t = tuple(int(q) for q in qs[:k])
        nc = int(rng.integers(0, 3))
        ctl = tuple(int(q) for q in qs[k:k + nc])
        vals = tuple(int(v) for v in rng.integers(0, 2, nc))
        gates.append(I.Gate(random_unitary(rng, 1 << k), t, ctl, vals))
    for codec, eps in (("rel", 1e-4), ("lossless", 0.0)):
        st, cs, c = run_both(n, 7, codec, eps, gates)
        assert_same_streams(st, cs, n, c)


@pytest.mark.parametrize("n,b", [(1, 1), (2, 1), (3, 2), (4, 4), (5, 5), (6, 3), (7, 3)])
def test_small_states_and_partial_groups(n, b):
    rng = np.random.default_rng(n)
    gates = []
    for i in range(25):
        q = int(rng.integers(0, n))
        gates.append(I.Gate(random_unitary(rng, 2), (q,)))
        if n > 1 and i % 3 == 0:
            a, bb = rng.choice(n, 2, replace=False)
            gates.append(I.cz(int(a), int(bb)))
    for codec, eps in (("rel", 1e-4), ("lossless", 0.0)):
        st, cs, c = run_both(n, b, codec, eps, gates)
        assert_same_streams(st, cs, n, c)


def test_aalc_ladder_streams():
    rows, cols = 3, 4
    gates = I.random_grid(rows, cols, 12, 4242)
    for theta in (2.0, 4.0, 8.0):
        st, cs, c = run_both(rows * cols, 6, "aalc", 1e-3, gates, aalc=(theta, [1e-5, 1e-4, 1e-3]))
        assert_same_streams(st, cs, rows * cols, c)
        levels = {s[2] for s in st.export_tiles()}
        assert levels <= {0, 1, 2, 3}


def test_none_and_lossless_equal_dense_oracle():
    # gate by gate (no diagonal runs), the uncompressed and lossless paths
    # are the dense FP64 simulation bit for bit
    n = 10
    gates = I.basis_gates(n, 0x155) + I.qft(n) + I.random_grid(2, 5, 5, 11)
    psi = oracle.dense_run(oracle.dense_zero(n), n, gates)
    for codec in ("none", "lossless"):
        st = qsim.State(n, 6, codec, 0.0)
        st.set_fusion(False)
        st.apply_all(gates)
        st.flush()
        got = st.amplitudes()
        assert np.array_equal(got.view(np.uint64), psi.view(np.uint64)), codec


def test_arena_regrows_and_stays_exact():
    rows, cols = 3, 6
    n = rows * cols
    gates = I.random_grid(rows, cols, 4, 5)
    st, cs, c = run_both(n, 10, "lossless", 0.0, gates)
    assert st.stats()["arena_regrows"] >= 1
    assert_same_streams(st, cs, n, c)


def test_encode_of_given_amplitudes_matches_oracle():
    rng = np.random.default_rng(1)
    n, b = 11, 7
    c = b
    psi = I.random_state(n, 77)
    psi[5] = 0.0
    psi[6] = complex(-0.0, 0.0)
    psi[1 << c: 2 << c] = psi[1 << c]            # one constant tile
    psi[2 << c: 3 << c] = 0.0                      # one zero tile
    psi[3 << c: 4 << c] = np.where(rng.random(1 << c) < 0.5, -1, 1) * 0.01  # sign-pattern-ish
    for codec, eps in (("rel", 1e-4), ("rel", 1e-2), ("lossless", 0.0)):
        st = qsim.State(n, b, codec, eps)
        st.set_amplitudes(psi)
        shifts, mb, _ = oracle_cfg(codec, eps, c)
        got = st.export_tiles()
        for t, s in enumerate(got):
            want, _, _ = oracle.encode_tile(psi[t << c:(t + 1) << c], c, shifts, mb)
            assert s == want, t


def test_oracle_streams_decode_on_gpu_and_back():
    n, c = 10, 6
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(1e-3)], None, True)
    cs.reset_basis(0)
    cs.run(I.random_grid(2, 5, 8, 3), 4, 48)
    st = qsim.State(n, c, "rel", 1e-3)
    streams = [cs.stream(t) for t in range(1 << (n - c))]
    st.import_tiles(0, streams)
    assert np.array_equal(st.amplitudes().view(np.uint64), cs.dense().view(np.uint64))
    assert st.stats()["alpha"] == cs.alpha
    # and GPU-written streams decode in the oracle
    st.apply_all([I.h(q) for q in range(n)])
    st.flush()
    for t, s in enumerate(st.export_tiles()):
        dec = oracle.decode_tile(s, c)
        assert np.array_equal(dec.view(np.uint64), st.amplitudes(t << c, 1 << c).view(np.uint64))


def test_malformed_import_is_rejected_and_state_kept():
    n, c = 8, 5
    st = qsim.State(n, c, "rel", 1e-4)
    st.apply_all(I.qft(n))
    st.flush()
    before = st.amplitudes()
    good = st.export_tiles(0, 1)[0]
    bad = bytearray(good)
    bad[24] = 9                                   # wrong tile size field
    with pytest.raises(qsim.QsimError) as e:
        st.import_tiles(0, [bytes(bad)])
    assert e.value.status == 7
    assert np.array_equal(st.amplitudes().view(np.uint64), before.view(np.uint64))


def test_probabilities_exact_and_amplitude_ranges():
    n = 12
    x = I.seeded_basis(n, 5)
    st, cs, c = run_both(n, 8, "rel", 1e-3, I.qft(n)[:60], x=x)
    psi = cs.dense()
    for qs in ([0], [3, 1], [11, 0, 5], list(range(n))):
        got = st.probabilities(qs)
        idx = np.arange(1 << n)
        key = np.zeros(1 << n, dtype=np.int64)
        for i, q in enumerate(qs):
            key |= ((idx >> q) & 1) << i
        S = [oracle.sum_sq_units(psi[key == j]) for j in range(1 << len(qs))]
        tot = oracle.units_to_double(sum(S))
        want = np.array([oracle.units_to_double(s) / tot for s in S])
        assert np.array_equal(got, want)
    for start, count in ((0, 1), (255, 3), (1000, 3000), ((1 << n) - 1, 1)):
        a = st.amplitudes(start, count)
        assert np.array_equal(a.view(np.uint64), psi[start:start + count].view(np.uint64))


def test_fidelity_references():
    n = 10
    x = 0x155
    gates = I.qft(n)
    ref = qsim.State(n, 6, "none", 0.0)
    ref.reset_basis(x)
    ref.apply_all(gates)
    st = qsim.State(n, 6, "rel", 1e-2)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    a, r = st.amplitudes(), ref.amplitudes()
    want = fid(r, a)
    assert abs(st.fidelity_state(ref) - want) < 1e-12
    assert abs(st.fidelity_dense(r) - want) < 1e-12
    assert abs(st.fidelity_qft(x) - fid(qft_ref(n, x), a)) < 1e-12
    assert abs(ref.fidelity_qft(x) - 1.0) < 1e-12


def test_gate_validation():
    st = qsim.State(6, 4, "rel", 1e-4)
    with pytest.raises(qsim.QsimError):
        st.apply(I.Gate(np.array([[1, 1], [0, 1]], dtype=complex), (0,)))      # not unitary
    with pytest.raises(qsim.QsimError):
        st.apply(I.Gate(I.MAT_H, (6,)))                                          # out of range
    with pytest.raises(qsim.QsimError):
        st.apply(I.Gate(I.MAT_H, (2,), (2,)))                                    # repeated
    with pytest.raises(qsim.QsimError):
        st.apply(I.Gate(np.array([[np.nan, 0], [0, 1]]), (0,)))                  # not finite
    st.apply(I.h(0))
    st.flush()


def test_nonfinite_input_is_reported():
    st = qsim.State(6, 5, "rel", 1e-4)
    psi = np.zeros(64, dtype=complex)
    psi[0] = 1
    psi[3] = complex(np.inf, 0)
    with pytest.raises(qsim.QsimError) as e:
        st.set_amplitudes(psi)
    assert e.value.status == 4
    with pytest.raises(qsim.QsimError) as e:
        st.flush()
    assert e.value.status == 6


def test_compressed_bytes_counts_streams():
    n, c = 12, 8
    st = qsim.State(n, c, "rel", 1e-4)
    sb, fp = st.compressed_bytes()
    assert sb == 32 * (1 << (n - c)) + len(st.export_tiles(0, 1)[0]) - 32
    st.apply_all(I.qft(n))
    sb, fp = st.compressed_bytes()
    assert sb == sum(len(s) for s in st.export_tiles())
    assert fp >= sb


def test_decoders_agree_on_corrupted_streams():
    """Byte-level fuzz of the stream format: for streams with zero words,
    exception sections and packed data, flip bytes of the body and the
    mode bytes; the GPU decoder (through qsim_import_tiles) accepts
    exactly the streams the oracle's decoder accepts and yields the same
    bits, apart from streams whose values leave the state's range (|x|
    >= 16 or non-finite), which the import rejects by design."""
    rng = np.random.default_rng(2024)
    c = 6
    N = 1 << c
    comps = rng.standard_normal(2 * N) / 8
    comps[rng.random(2 * N) < 0.6] = 0.0
    a = comps.view(np.complex128)
    base, _, _ = oracle.encode_tile(a, c, [39])
    assert base[0] == 1 and (base[3] or base[25])
    st = qsim.State(c, c, "rel", 1e-4)
    agree = 0
    for trial in range(300):
        bad = bytearray(base)
        for _ in range(1 + trial % 3):
            pos = int(rng.choice([3, 25])) if trial % 5 == 0 else int(rng.integers(32, len(bad)))
            bad[pos] ^= int(rng.integers(1, 256))
        try:
            want = oracle.decode_tile(bytes(bad), c)
        except ValueError:
            want = None
        try:
            st.import_tiles(0, [bytes(bad)])
            got = st.amplitudes()
        except qsim.QsimError as e:
            assert e.status == 7
            got = None
        if want is None:
            assert got is None, trial
        elif got is None:
            w = want.view(np.float64)
            assert not np.all(np.isfinite(w)) or np.max(np.abs(w)) >= 16, trial
        else:
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), trial
            agree += 1
    assert agree >= 30
    st.close()


def test_tile_moving_sweeps_match_oracle():
    # permutations on qubits >= c only (X, SWAP, CNOT and Toffoli-type
    # controls on high qubits): the streams move whole, without normalize;
    # then ordinary sweeps, all byte-identical to the oracle
    n = 13
    moves = [I.x(12), I.swap(8, 11), I.Gate(I.MAT_X, (9,), (10,), (1,)),
             I.Gate(I.MAT_X, (12,), (8, 9), (1, 0)), I.x(10)]
    gates = I.random_grid(*I.grid_shape(n), 5, 21) + moves + I.qft(n)[:30] + moves[::-1]
    for codec, eps in (("rel", 1e-4), ("lossless", 0.0)):
        st, cs, c = run_both(n, 8, codec, eps, gates)
        assert_same_streams(st, cs, n, c)
