"""Checkpoint / resume (qsim_save, qsim_load): a circuit saved halfway,
loaded into a new handle and continued gives the same streams as the run
that was never interrupted (REL with normalize, AALC, lossless), the file
decodes tile by tile in the oracle, and broken files are rejected."""
import os
import struct

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


def make(codec, eps, n):
    st = qsim.State(n, 8, codec, eps)
    if codec == "aalc":
        st.set_aalc(4.0, [1e-5, 1e-4, 1e-3])
    return st


@pytest.mark.parametrize("codec,eps", [("rel", 1e-4), ("aalc", 1e-3), ("lossless", 0.0)])
def test_resume_gives_the_same_streams(tmp_path, codec, eps):
    n = 14
    gates = I.qft(n) + I.random_grid(2, 7, 6, 17)
    half = len(gates) // 2
    x = I.seeded_basis(n, 5)
    ref = make(codec, eps, n)
    ref.reset_basis(x)
    ref.apply_all(gates[:half])
    ref.flush()
    path = os.path.join(tmp_path, "state.ckpt")
    ref.save(path)
    ref.apply_all(gates[half:])
    ref.flush()
    want = ref.export_tiles()
    st = qsim.State.load(path)
    assert st.stats()["n_qubits"] == n and st.stats()["tile_log2"] == 8
    st.apply_all(gates[half:])
    st.flush()
    assert st.export_tiles() == want
    st.close()
    ref.close()


def test_checkpoint_file_decodes_in_the_oracle(tmp_path):
    n, c = 11, 8
    st = qsim.State(n, c, "rel", 1e-4)
    st.reset_basis(I.seeded_basis(n, 9))
    st.apply_all(I.qft(n))
    st.flush()
    path = os.path.join(tmp_path, "s.ckpt")
    st.save(path)
    data = open(path, "rb").read()
    assert data[:8] == b"QSIMCKP1"
    hdr = struct.unpack_from("<8I8i2d3Q2i", data, 8)
    assert hdr[0] == 2 and hdr[1] == n and hdr[2] == c
    assert hdr[-2:] == (0, 0)                 # decisions per tile, reserved
    ntiles = hdr[-4]
    sizes = struct.unpack_from(f"<{ntiles}Q", data, 120)
    off = 120 + 8 * ntiles
    amps = []
    for t in range(ntiles):
        amps.append(oracle.decode_tile(data[off:off + sizes[t]], c))
        off += sizes[t]
    assert off == len(data)
    got = np.concatenate(amps)
    assert np.array_equal(got.view(np.uint64), st.amplitudes().view(np.uint64))
    st.close()


def test_broken_checkpoints_are_rejected(tmp_path):
    n = 10
    st = qsim.State(n, 8, "rel", 1e-3)
    st.apply_all(I.qft(n))
    path = os.path.join(tmp_path, "s.ckpt")
    st.save(path)
    data = bytearray(open(path, "rb").read())
    bad = os.path.join(tmp_path, "bad.ckpt")
    for mutate in (lambda d: d.__setitem__(0, ord("X")),            # magic
                   lambda d: d.__setitem__(12, 99),                 # n
                   lambda d: d.__delitem__(slice(len(d) - 40, None)),  # truncated
                   lambda d: d.__setitem__(112, 99),                # decision unit
                   lambda d: d.__setitem__(120 + 8 * 4 + 24, 7)):   # a stream's tile size field
        d = bytearray(data)
        mutate(d)
        open(bad, "wb").write(bytes(d))
        with pytest.raises(qsim.QsimError) as e:
            qsim.State.load(bad)
        assert e.value.status == qsim.QSIM_ERR_FORMAT
    with pytest.raises(qsim.QsimError):
        qsim.State.load(os.path.join(tmp_path, "missing.ckpt"))
    st.close()
