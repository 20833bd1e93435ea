"""GPU parity of the POLAR tile mode (magnitude and phase) against the
oracle, through the C ABI: streams byte for byte with the variant on (the
GPU's CORDIC table, angles, reconstruction, order-2 residuals, bound checks
and the choice against the componentwise stream all match), oracle streams
decoding on the GPU, AALC decisions per tile and per stride, small tiles,
and checkpoints keeping the setting.
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
    oracle.build()


def run_pair(n, c, gates, codec, eps, x=0, aalc=None, unit=None, hmax=4):
    st = qsim.State(n, c, codec, eps)
    st.set_schedule(c, hmax, 512)
    if aalc:
        st.set_aalc(*aalc)
    st.set_polar(True)
    if unit:
        st.set_aalc_unit(unit)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    if codec == "rel":
        shifts, mb = [oracle.shift_for_eps(eps)], None
    else:
        theta, levels = aalc
        shifts, mb = [0] + [oracle.shift_for_eps(e) for e in levels], oracle.max_bytes_for(c, theta)
    cs = oracle.CSim(n, c, shifts, mb, True, polar=True)
    if unit:
        cs.set_unit(unit, aalc[0])
    cs.reset_basis(x)
    cs.run(gates, hmax, 512)
    return st, cs


def same(st, cs):
    got = st.export_tiles()
    for t, s in enumerate(got):
        assert s == cs.stream(t), (t, s[:48].hex(), cs.stream(t)[:48].hex())
    assert st.stats()["alpha"] == cs.alpha
    return got


@pytest.mark.parametrize("c", [8, 5, 3])
def test_qft_polar_streams_match_oracle(c):
    n = 12
    x = I.seeded_basis(n)
    st, cs = run_pair(n, c, I.qft(n), "rel", 1e-4, x=x, hmax=min(4, 12 - c))
    got = same(st, cs)
    assert sum(s[0] in (3, 4) for s in got) > len(got) // 2     # the QFT's tiles go polar
    psi = cs.dense()
    assert np.array_equal(st.amplitudes().view(np.uint64), psi.view(np.uint64))
    assert st.fidelity_qft(x) > 0.9999


def test_aalc_with_polar_meets_theta_on_every_tile():
    n, c = 12, 8
    x = I.seeded_basis(n)
    for theta in (8.0, 16.0, 32.0):
        st, cs = run_pair(n, c, I.qft(n), "aalc", 1e-2, x=x, aalc=(theta, [1e-5, 1e-4, 1e-3, 1e-2]))
        got = same(st, cs)
        assert all(16 * (1 << c) / len(s) >= theta for s in got)
        assert st.stats()["tiles_over_limit"] == 0           # every tile of every sweep met theta
        assert st.fidelity_qft(x) > 0.9999


def test_random_grid_mixes_modes_and_matches_oracle():
    rows, cols = 3, 4
    gates = I.random_grid(rows, cols, 8, I.BASE_SEED + 5)
    for eps in (1e-2, 1e-4):
        st, cs = run_pair(rows * cols, 6, gates, "rel", eps)
        same(st, cs)
    st, cs = run_pair(rows * cols, 6, gates, "aalc", 1e-3, aalc=(4.0, [1e-5, 1e-4, 1e-3]))
    same(st, cs)


def test_per_stride_decisions_with_polar_match_oracle():
    n, c = 12, 6
    x = I.seeded_basis(n, 9)
    gates = I.qft(n)
    st, cs = run_pair(n, c, gates, "aalc", 1e-3, x=x, aalc=(16.0, [1e-5, 1e-4, 1e-3]), unit=9)
    same(st, cs)


def test_oracle_polar_streams_decode_on_the_gpu_and_checkpoint_keeps_polar(tmp_path):
    n, c = 10, 8
    k = np.arange(1 << n)
    psi = np.exp(2j * np.pi * 345 * k / (1 << n)) / math.sqrt(1 << n)
    psi[7] = 0.0
    phi = np.random.default_rng(8).uniform(0, 2 * np.pi, c)     # tiles 2, 3: one phase per index bit
    bits = (np.arange(1 << c)[:, None] >> np.arange(c)) & 1
    psi[2 << c:] = np.tile(np.exp(1j * (bits @ phi)), 2) / math.sqrt(1 << n)
    s = oracle.shift_for_eps(1e-4)
    streams = [oracle.encode_tile(psi[t << c:(t + 1) << c], c, [s], polar=True)[0] for t in range(1 << (n - c))]
    assert all(st[0] in (3, 4) for st in streams) and {st[0] for st in streams} == {3, 4}
    h = qsim.State(n, c, "rel", 1e-4)
    h.set_polar(True)
    h.import_tiles(0, streams)
    want = np.concatenate([oracle.decode_tile(st, c) for st in streams])
    assert np.array_equal(h.amplitudes().view(np.uint64), want.view(np.uint64))
    path = str(tmp_path / "polar.ckpt")
    h.apply_all(I.qft(n)[:5])
    h.save(path)
    h.apply_all(I.qft(n)[5:])
    h.flush()
    g = qsim.State.load(path)
    g.apply_all(I.qft(n)[5:])
    g.flush()
    assert g.export_tiles() == h.export_tiles()


def test_bitwise_predictor_streams_match_oracle():
    # a product state over the index bits (the QFT before its swaps) and
    # the full QFT on 14 qubits: dense tiles take the bitwise predictor,
    # byte for byte with the oracle, and AALC theta = 32 holds on every tile
    n, c = 14, 8
    x = I.seeded_basis(n, 3)
    gates = I.qft(n)[:-(n // 2)]                                 # without the final swaps
    st, cs = run_pair(n, c, gates, "rel", 1e-4, x=x)
    got = same(st, cs)
    assert sum(s[0] == 4 for s in got) > len(got) // 2
    st, cs = run_pair(n, c, I.qft(n), "aalc", 1e-2, x=x, aalc=(32.0, [1e-5, 1e-4, 1e-3, 1e-2]))
    same(st, cs)
    assert st.stats()["tiles_over_limit"] == 0
