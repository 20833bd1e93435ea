"""GPU parity of per-stride AALC decisions (Algorithm 2 tests the ratio of
a whole stride): every tile stream byte-identical to the oracle's with the
same stride, ladder and theta, through fresh encodes (basis and dense),
sweeps of every kind (general, uniform items, tile-moving SWAPs, deep and
shallow fusion) and checkpoints; at larger sizes every stride holds one
level and meets its limit unless at the last level."""
import os

import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu

LADDER = [1e-5, 1e-4, 1e-3, 1e-2]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def gpu_state(n, b, c, theta, hmax=4, depth=512):
    st = qsim.State(n, b, "aalc", LADDER[-1])
    st.set_schedule(c, hmax, depth)
    st.set_aalc(theta, LADDER)
    st.set_aalc_unit()
    return st


def oracle_state(n, b, c, theta):
    shifts = [0] + [oracle.shift_for_eps(e) for e in LADDER]
    cs = oracle.CSim(n, c, shifts, oracle.max_bytes_for(c, theta), True)
    assert cs.set_unit(b, theta) == min(b, n) - c
    return cs


def same_streams(st, cs, n, c):
    got = st.export_tiles()
    assert len(got) == 1 << (n - c)
    for t, s in enumerate(got):
        want = cs.stream(t)
        assert s == want, f"tile {t}: gpu {s[:40].hex()} oracle {want[:40].hex()}"


@pytest.mark.parametrize("n,b,c,theta,depth", [(12, 8, 5, 3.0, 512), (12, 8, 5, 5.0, 7),
                                               (12, 9, 6, 8.0, 512), (11, 7, 4, 4.0, 1)])
def test_qft_streams(n, b, c, theta, depth):
    x = I.seeded_basis(n, 31)
    gates = I.qft(n)
    st = gpu_state(n, b, c, theta, depth=depth)
    st.reset_basis(x)
    cs = oracle_state(n, b, c, theta)
    cs.reset_basis(x)
    same_streams(st, cs, n, c)
    st.apply_all(gates)
    st.flush()
    cs.run(gates, 4, depth)
    same_streams(st, cs, n, c)
    assert st.stats()["alpha"] == cs.alpha


@pytest.mark.parametrize("theta", [2.0, 4.0, 6.0])
def test_dense_start_and_random_grid(theta):
    n, b, c = 12, 8, 5
    psi = I.strided_mix_state(n, c, b, I.BASE_SEED + 60)
    gates = I.random_grid(3, 4, 8, I.BASE_SEED + 61)
    st = gpu_state(n, b, c, theta, depth=40)
    st.set_amplitudes(psi)
    cs = oracle_state(n, b, c, theta)
    cs.set_dense(psi)
    assert len({cs.stream(t)[2] for t in range(1 << (n - c))}) >= 2     # strides at several levels
    same_streams(st, cs, n, c)
    st.apply_all(gates)
    st.flush()
    cs.run(gates, 4, 40)
    same_streams(st, cs, n, c)


def test_high_qubit_sweeps_uniform_items_and_swaps():
    # gates on qubits >= c only: uniform items, and SWAP sweeps that a
    # per-tile state would move as streams
    n, b, c = 12, 8, 4
    gates = [I.h(q) for q in range(c, n)] + [I.cphase(0.3 * q, q, n - 1) for q in range(c, n - 1)]
    gates += [I.swap(c, n - 1), I.swap(c + 1, n - 2)]
    st = gpu_state(n, b, c, 6.0, depth=9)
    st.reset_basis(0)
    st.apply_all(gates)
    st.flush()
    cs = oracle_state(n, b, c, 6.0)
    cs.reset_basis(0)
    cs.run(gates, 4, 9)
    same_streams(st, cs, n, c)


def test_unit_zero_and_small_units_decide_per_tile():
    n, b, c, theta = 11, 8, 5, 5.0
    gates = I.qft(n)
    a = gpu_state(n, b, c, theta)
    a.set_aalc_unit(0)
    b2 = gpu_state(n, b, c, theta)
    b2.set_aalc_unit(c)                      # a stride of one tile
    ref = qsim.State(n, b, "aalc", LADDER[-1])
    ref.set_schedule(c, 4, 512)
    ref.set_aalc(theta, LADDER)
    for st in (a, b2, ref):
        st.reset_basis(5)
        st.apply_all(gates)
        st.flush()
    assert a.export_tiles() == ref.export_tiles() == b2.export_tiles()


def test_batch_refuses_per_stride_handles():
    st = gpu_state(10, 8, 5, 4.0)
    other = qsim.State(10, 8, "rel", 1e-4)
    st.apply_all(I.qft(10))
    other.apply_all(I.qft(10))
    with pytest.raises(qsim.QsimError) as e:
        qsim.flush_batch([other, st])
    assert e.value.status == qsim.QSIM_ERR_ARG


def test_checkpoint_keeps_the_stride(tmp_path):
    n, b, c, theta = 12, 9, 5, 5.0
    gates = I.qft(n) + I.random_grid(3, 4, 4, 23)
    half = len(gates) // 2
    ref = gpu_state(n, b, c, theta)
    ref.reset_basis(77)
    ref.apply_all(gates[:half])
    ref.flush()
    path = os.path.join(tmp_path, "u.ckpt")
    ref.save(path)
    ref.apply_all(gates[half:])
    ref.flush()
    st = qsim.State.load(path)
    st.apply_all(gates[half:])
    st.flush()
    assert st.export_tiles() == ref.export_tiles()


def test_qft22_one_level_per_stride():
    n, b, theta = 22, 16, 6.0
    x = I.seeded_basis(n, 32)
    st = qsim.State(n, b, "aalc", LADDER[-1])
    st.set_aalc(theta, LADDER)
    st.set_aalc_unit()
    c = st.stats()["tile_log2"]
    st.reset_basis(x)
    st.apply_all(I.qft(n))
    st.flush()
    tiles = st.export_tiles()
    per = 1 << (b - c)
    limit = oracle.max_bytes_for(b, theta)
    last = len(LADDER)
    for s0 in range(0, len(tiles), per):
        ks = {t[2] for t in tiles[s0:s0 + per]}
        assert len(ks) == 1
        assert sum(len(t) for t in tiles[s0:s0 + per]) <= limit or ks == {last}
    assert st.fidelity_qft(x) > 0.999
