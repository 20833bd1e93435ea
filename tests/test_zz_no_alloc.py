"""qsim_encode_noalloc: the encode path for callers that may not allocate
device memory (for example code running under an application allocator
that owns all of the GPU's memory).  Its scratch is a fixed static device
array; the caller provides the input state and the output buffers.

Checked through the C ABI against the regular path (qsim_set_amplitudes
on a QSIM_CODEC_REL handle, then qsim_export_tiles): every tile stream must
be byte-identical, on two calls in a row with different states, so that a
stale scratch array from the previous call would show.  This file is
collected last so that a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def streams_from(out: np.ndarray, table: np.ndarray) -> list[bytes]:
    res = []
    for off in table.tolist():
        body = int(out[off + 4:off + 8].view(np.uint32)[0])
        res.append(out[off:off + 32 + body].tobytes())
    return res


def regular_streams(psi, n, c, eps) -> list[bytes]:
    st = qsim.State(n, c, "rel", eps)
    st.set_amplitudes(psi)
    s = st.export_tiles()
    st.close()
    return s


def test_noalloc_encode_matches_regular_path_twice():
    import torch
    n, c, eps = 14, 8, 1e-4
    ntiles = 1 << (n - c)
    cap = ntiles * (32 + (16 << c))
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    table = torch.zeros(ntiles, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    states = []
    a = I.random_state(n, 1234)
    b = np.zeros(1 << n, dtype=np.complex128)
    b[:] = I.random_state(n, 99)
    b[3 << c:5 << c] = 0.0                     # zero tiles
    b[7 << c:8 << c] = b[7 << c]               # a constant tile
    states = [a, b]
    for psi in states:
        dev = torch.from_numpy(psi.view(np.float64).copy()).to("cuda")
        used = qsim.encode_noalloc(dev.data_ptr(), n, c, eps, out.data_ptr(), cap,
                                   table.data_ptr(), stream)
        torch.cuda.synchronize()
        got = streams_from(out.cpu().numpy(), table.cpu().numpy())
        want = regular_streams(psi, n, c, eps)
        assert used == sum(len(s) for s in want)
        assert got == want


def test_noalloc_rejects_states_beyond_its_scratch():
    with pytest.raises(qsim.QsimError) as e:
        qsim.encode_noalloc(16, 24, 10, 1e-4, 16, 1 << 20, 16)     # 2^14 tiles > 4096
    assert e.value.status == 1
    assert "static scratch" in e.value.message
