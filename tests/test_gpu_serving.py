"""Serving loop (qsim_server_*): continuous batching of circuits of uneven
sizes.  Every circuit's read-out must equal the same circuit run alone
(bit for bit) and the oracle's exact probabilities of the same compressed
run, admission must respect the memory budget, and circuits that arrive
while others run must be admitted and finished.
"""
import time

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


def mix(count, seed, nmin=6, nmax=14):
    rng = I.Rng(seed)
    jobs = []
    for i in range(count):
        n = nmin + rng.below(nmax - nmin + 1)
        kind = rng.below(10)
        eps = (1e-3, 1e-4)[rng.below(2)]
        if kind < 4:
            gates, x = I.qft(n), rng.below(1 << n)
        elif kind < 7:
            gates, x = I.grover(n, rng.below(1 << n), 2 + rng.below(5)), 0
        else:
            gates, x = I.random_grid(*I.grid_shape(n), 8 + rng.below(13), rng.next()), 0
        readout = [rng.below(n) for _ in range(3)]
        readout = list(dict.fromkeys(readout))
        jobs.append((n, gates, x, eps, readout))
    return jobs


def alone(job):
    n, gates, x, eps, readout = job
    st = qsim.State(n, 8, "rel", eps)
    st.reset_basis(x)
    st.apply_all(gates)
    p = st.probabilities(readout)
    st.close()
    return p


def test_results_equal_alone_and_in_the_mix():
    jobs = mix(24, 7)
    srv = qsim.Server(8 << 30, max_resident=16, sweeps_per_tick=2)
    tickets = []
    for k, (n, gates, x, eps, readout) in enumerate(jobs):
        tickets.append(srv.submit(n, gates, eps=eps, basis=x, readout=readout))
        if k % 6 == 5:
            time.sleep(0.01)               # later arrivals join running ticks
    srv.drain(600)
    st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_resident_seen"] > 1
    for job, t in zip(jobs, tickets):
        info, probs = srv.result(t)
        assert info["done"] == 1 and info["status"] == 0
        assert np.array_equal(probs, alone(job))
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    srv.close()


def test_admission_respects_the_budget():
    budget = 96 << 20
    srv = qsim.Server(budget, max_resident=64, sweeps_per_tick=1)
    jobs = [(16, I.qft(16)[:60], 5, 1e-3, [0, 15])] * 12
    tickets = [srv.submit(n, g, eps=e, basis=x, readout=r) for n, g, x, e, r in jobs]
    srv.drain(600)
    st = srv.stats()
    assert st["completed"] == 12
    assert st["peak_footprint"] <= budget
    assert 1 <= st["max_resident_seen"] < 12       # not everything at once
    want = alone(jobs[0])
    for t in tickets:
        assert np.array_equal(srv.result(t)[1], want)
    srv.close()


def test_graph_captured_ticks_give_the_same_results():
    jobs = mix(8, 99, 5, 11)
    srv = qsim.Server(4 << 30, max_resident=8, sweeps_per_tick=3, use_graph=True)
    tickets = [srv.submit(n, g, eps=e, basis=x, readout=r) for n, g, x, e, r in jobs]
    srv.drain(600)
    for job, t in zip(jobs, tickets):
        assert np.array_equal(srv.result(t)[1], alone(job))
    srv.close()


def oracle_probs(job):
    """The oracle's read-out of a job: the compressed run with the library's
    default schedule for the job's size (tile 2^min(8, n), its pair slots and
    depth), then the exact sums of |a|^2 per read-out pattern, divided by
    the exact total (the library's definition)."""
    n, gates, x, eps, readout = job
    c = min(8, n)
    probe = qsim.State(n, 8, "rel", eps)
    s = probe.stats()
    probe.close()
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(eps)], None, True)
    cs.reset_basis(x)
    cs.run(gates, s["hmax"], s["depth"])
    psi = cs.dense()
    idx = np.arange(1 << n)
    key = np.zeros(1 << n, dtype=np.int64)
    for i, q in enumerate(readout):
        key |= ((idx >> q) & 1) << i
    S = [oracle.sum_sq_units(psi[key == j]) for j in range(1 << len(readout))]
    tot = oracle.units_to_double(sum(S))
    return np.array([oracle.units_to_double(v) / tot for v in S])


def test_mix_results_equal_the_oracle():
    # a mix of QFT, Grover and grid circuits of 5..12 qubits at both
    # bounds, served together (arrivals spread over the first ticks): every
    # read-out is bit-identical to the oracle's exact probabilities
    jobs = mix(18, 2024, 5, 12)
    srv = qsim.Server(2 << 30, max_resident=8, sweeps_per_tick=1)
    tickets = []
    for k, (n, gates, x, eps, readout) in enumerate(jobs):
        tickets.append(srv.submit(n, gates, eps=eps, basis=x, readout=readout))
        if k % 4 == 3:
            time.sleep(0.005)
    srv.drain(600)
    assert srv.stats()["completed"] == len(jobs)
    for job, t in zip(jobs, tickets):
        info, probs = srv.result(t)
        assert info["status"] == 0
        assert np.array_equal(probs, oracle_probs(job)), job[0]
    srv.close()
