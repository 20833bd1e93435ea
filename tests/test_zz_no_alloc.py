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


def encode_twice_compare(n, c, eps, psis):
    import torch
    ntiles = 1 << (n - c)
    cap = ntiles * (32 + (16 << c))
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    table = torch.zeros(ntiles, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    free = []
    for psi in psis:
        dev = torch.from_numpy(psi.view(np.float64).copy()).to("cuda")
        torch.cuda.synchronize()
        used = qsim.encode_noalloc(dev.data_ptr(), n, c, eps, out.data_ptr(), cap, table.data_ptr(), stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = streams_from(out.cpu().numpy(), table.cpu().numpy())
        want = regular_streams(psi, n, c, eps)
        assert used == sum(len(s) for s in want)
        assert got == want
        del dev
    return free


def test_noalloc_at_its_tile_limit_allocates_nothing():
    # exactly 4096 tiles (n - tile_log2 = 12), the largest state the static
    # scratch serves; the device's free memory is the same after a second
    # call as after the first (the call itself allocates nothing: any
    # difference would be memory the library took)
    import torch
    n, c, eps = 20, 8, 1e-4
    a = I.random_state(n, 7)
    b = np.exp(2j * np.pi * np.arange(1 << n) / (1 << n)) / np.sqrt(1 << n)
    ntiles = 1 << (n - c)
    cap = ntiles * (32 + (16 << c))
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    table = torch.zeros(ntiles, dtype=torch.int64, device="cuda")
    da = torch.from_numpy(a.view(np.float64).copy()).to("cuda")
    db = torch.from_numpy(b.view(np.float64).copy()).to("cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    qsim.encode_noalloc(da.data_ptr(), n, c, eps, out.data_ptr(), cap, table.data_ptr(), stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    used = qsim.encode_noalloc(db.data_ptr(), n, c, eps, out.data_ptr(), cap, table.data_ptr(), stream)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 == free1
    got = streams_from(out.cpu().numpy(), table.cpu().numpy())
    want = regular_streams(b, n, c, eps)
    assert used == sum(len(s) for s in want) and got == want
    # and twice in a row at the limit against the regular path
    encode_twice_compare(n, c, eps, [b, a])


def test_noalloc_reports_the_size_it_needs_then_fits():
    # out_cap too small: ERR_ARG with the bytes needed in *stream_bytes;
    # a second call with exactly that capacity gives the regular streams
    import torch
    n, c, eps = 14, 8, 1e-4
    psi = I.random_state(n, 4321)
    want = regular_streams(psi, n, c, eps)
    need = sum(len(s) for s in want)
    ntiles = 1 << (n - c)
    dev = torch.from_numpy(psi.view(np.float64).copy()).to("cuda")
    table = torch.zeros(ntiles, dtype=torch.int64, device="cuda")
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st, used = qsim.encode_noalloc(dev.data_ptr(), n, c, eps, small.data_ptr(), 64, table.data_ptr(),
                                   torch.cuda.current_stream(), check=False)
    assert st == 1 and used == need
    out = torch.zeros(used, dtype=torch.uint8, device="cuda")
    got_used = qsim.encode_noalloc(dev.data_ptr(), n, c, eps, out.data_ptr(), used, table.data_ptr(),
                                   torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert got_used == need
    assert streams_from(out.cpu().numpy(), table.cpu().numpy()) == want


def test_noalloc_rejects_a_non_finite_amplitude():
    import torch
    n, c = 12, 8
    psi = I.random_state(n, 11)
    psi[100] = complex(float("nan"), 0.0)
    ntiles = 1 << (n - c)
    cap = ntiles * (32 + (16 << c))
    dev = torch.from_numpy(psi.view(np.float64).copy()).to("cuda")
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    table = torch.zeros(ntiles, dtype=torch.int64, device="cuda")
    st, _ = qsim.encode_noalloc(dev.data_ptr(), n, c, 1e-4, out.data_ptr(), cap, table.data_ptr(),
                                torch.cuda.current_stream(), check=False)
    assert st == 4
