"""Arenas in a caller-owned buffer (qsim_set_pool): a torch tensor holds
the compressed state.  Streams stay byte-identical to a library-owned run
(and to the oracle), the tensor's bytes are the ones written, a pool that
is too small fails with OOM and invalidates the handle, and the state
moves back to library arenas intact."""
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def run(n, gates, x, pool=None, back=False):
    st = qsim.State(n, 8, "rel", 1e-4)
    st.reset_basis(x)
    if pool is not None:
        st.set_pool(pool)
    st.apply_all(gates[: len(gates) // 2])
    st.flush()
    if back:
        st.set_pool(None)
    st.apply_all(gates[len(gates) // 2:])
    st.flush()
    out = st.export_tiles()
    return st, out


def test_pool_streams_identical_and_in_tensor():
    import torch
    n = 12
    gates = I.qft(n)
    x = I.seeded_basis(n, 41)
    ref, want = run(n, gates, x)
    ref.close()
    pool = torch.zeros(1 << 22, dtype=torch.uint8, device="cuda")
    st, got = run(n, gates, x, pool)
    assert got == want
    # the tensor holds the streams: every exported stream occurs in it
    raw = pool.cpu().numpy().tobytes()
    for t in (0, 5, len(got) - 1):
        assert raw.find(got[t]) >= 0
    cs = oracle.CSim(n, 8, [oracle.shift_for_eps(1e-4)], None, True)
    cs.reset_basis(x)
    d = st.stats()["depth"]
    cs.run(gates[: len(gates) // 2], 4, d)          # the same two flushes
    cs.run(gates[len(gates) // 2:], 4, d)
    assert all(s == cs.stream(t) for t, s in enumerate(got))
    st.close()


def test_pool_back_to_library_arenas():
    import torch
    n = 12
    gates = I.random_grid(3, 4, 8, 7)
    _, want = run(n, gates, 0)
    pool = torch.zeros(1 << 22, dtype=torch.uint8, device="cuda")
    st, got = run(n, gates, 0, pool, back=True)
    assert got == want
    del pool
    st.apply_all([I.h(0)])
    st.flush()                            # runs on library arenas again
    st.close()


def test_pool_too_small_and_bad_arguments():
    import torch
    n = 14
    st = qsim.State(n, 8, "lossless", 0.0)
    st.reset_basis(3)
    with pytest.raises(qsim.QsimError):
        st.set_pool(torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")[1:])   # misaligned
    with pytest.raises(qsim.QsimError):
        st.set_pool(torch.zeros(1 << 20, dtype=torch.uint8))                     # host memory
    small = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")              # holds |x> only
    st.set_pool(small)
    st.apply_all(I.random_grid(2, 7, 6, 3))
    with pytest.raises(qsim.QsimError) as e:
        st.flush()
    assert e.value.status == qsim.QSIM_ERR_OOM
    with pytest.raises(qsim.QsimError) as e:
        st.probabilities([0])
    assert e.value.status == qsim.QSIM_ERR_STATE_INVALID
    st.close()
