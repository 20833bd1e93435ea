"""Batched flushes (qsim_flush_batch): many circuits' sweeps in one launch per
round.  Each circuit's stored streams must be byte-identical to the same
circuit flushed alone, with and without CUDA-graph capture, including a
circuit whose arena has to grow during the batch; one of them is also
checked against the oracle.
"""
import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def make_jobs():
    jobs = []
    for i, (n, b, codec, eps) in enumerate([(5, 3, "rel", 1e-4), (8, 6, "lossless", 0.0), (10, 8, "rel", 1e-3),
                                            (12, 8, "rel", 1e-4), (14, 8, "aalc", 1e-3), (9, 4, "none", 0.0),
                                            (16, 8, "lossless", 0.0), (11, 7, "rel", 1e-2)]):
        kind = i % 3
        if kind == 0:
            gates = I.qft(n)
            x = I.seeded_basis(n, 100 + i)
        elif kind == 1:
            gates = I.grover(n, (37 * i + 5) % (1 << n), 2)
            x = 0
        else:
            gates = I.random_grid(*I.grid_shape(n), 6 + i, 500 + i)
            x = 0
        jobs.append((n, b, codec, eps, gates, x))
    return jobs


def start(job):
    n, b, codec, eps, gates, x = job
    st = qsim.State(n, b, codec, eps)
    if codec == "aalc":
        st.set_aalc(4.0, [1e-5, 1e-4, 1e-3])
    st.reset_basis(x)
    st.apply_all(gates)
    return st


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_alone(use_graph):
    jobs = make_jobs()
    alone = []
    for job in jobs:
        st = start(job)
        st.flush()
        alone.append(st.export_tiles())
        st.close()
    batch = [start(job) for job in jobs]
    qsim.flush_batch(batch, use_graph=use_graph)
    for job, st, want in zip(jobs, batch, alone):
        assert st.export_tiles() == want, job[:4]
    # the 12-qubit QFT against the oracle as well
    n, b, codec, eps, gates, x = jobs[3]
    cs = oracle.CSim(n, min(b, n, 8), [oracle.shift_for_eps(eps)], None, True)
    cs.reset_basis(x)
    cs.run(gates, 4, batch[3].stats()["depth"])
    got = batch[3].export_tiles()
    assert all(s == cs.stream(t) for t, s in enumerate(got))


def test_batch_with_arena_growth_and_uneven_lengths():
    rows, cols = 3, 6
    big = (rows * cols, 8, "lossless", 0.0, I.random_grid(rows, cols, 5, 9), 0)   # grows its arena
    small = (7, 3, "rel", 1e-4, I.qft(7)[:10], 3)
    jobs = [small, big, small]
    alone = []
    for job in jobs:
        st = start(job)
        st.flush()
        alone.append(st.export_tiles())
    batch = [start(job) for job in jobs]
    qsim.flush_batch(batch)
    assert batch[1].stats()["arena_regrows"] >= 1
    for st, want in zip(batch, alone):
        assert st.export_tiles() == want


def test_batch_rejects_repeated_handles():
    st = qsim.State(6, 4, "rel", 1e-4)
    with pytest.raises(qsim.QsimError):
        qsim.flush_batch([st, st])
