"""Autotuner: picks a valid schedule by timing, and a circuit run under the
chosen schedule still matches the oracle run with that partition."""
import pytest

import oracle
from paper_1811_05140_gb300 import autotune
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1811_05140_gb300 import build
    build.build()


def test_tuned_schedule_is_valid_and_exact():
    n = 12
    gates = I.qft(n)
    x = I.seeded_basis(n)
    res = autotune.tune(n, gates, "rel", 1e-4, x, reps=1)
    c, hmax, depth, threads = res["best"]
    assert autotune.valid(n, c, hmax) and len(res["table"]) >= 3
    assert all(r["seconds"] > 0 for r in res["table"])
    assert {autotune.full(r["schedule"])[3] for r in res["table"]} == {128, 256, 512}
    st = qsim.State(n, 20, "rel", 1e-4)
    st.set_schedule(c, hmax, depth)
    st.set_sweep_threads(threads)
    st.reset_basis(x)
    st.apply_all(gates)
    st.flush()
    cs = oracle.CSim(n, c, [oracle.shift_for_eps(1e-4)], None, True)
    cs.reset_basis(x)
    cs.run(gates, hmax, depth)
    assert all(s == cs.stream(t) for t, s in enumerate(st.export_tiles()))
    tuner = autotune.Tuner(reps=1)
    assert tuner.schedule(n, "qft", gates, "rel", 1e-4, x) == tuner.schedule(n, "qft", gates, "rel", 1e-4, x)


@pytest.mark.parametrize("threads", [128, 512])
def test_every_sweep_shape_matches_oracle(threads):
    # the CTA size changes nothing in the result: QFT and a random grid
    # under each launch shape, byte for byte against the oracle
    for n, gates, x in ((12, I.qft(12), I.seeded_basis(12)), (12, I.random_grid(3, 4, 6, 77), 0)):
        st = qsim.State(n, 8, "rel", 1e-4)
        st.set_sweep_threads(threads)
        st.reset_basis(x)
        st.apply_all(gates)
        st.flush()
        cs = oracle.CSim(n, 8, [oracle.shift_for_eps(1e-4)], None, True)
        cs.reset_basis(x)
        cs.run(gates, 4, 512)
        assert all(s == cs.stream(t) for t, s in enumerate(st.export_tiles()))


def test_retiling_a_basis_state_encodes_it_afresh():
    # a 33-qubit basis state (2^37 bytes dense, beyond the dense re-tiling
    # path) re-tiles from 2^8 to 2^7 amplitudes per tile: its streams equal
    # those of a state created with 2^7-amplitude tiles; once a gate has run
    # the state is no longer a basis state and re-tiling needs n <= 32
    n, eps = 33, 1e-4
    x = I.seeded_basis(n, 3)
    st = qsim.State(n, 8, "rel", eps)
    st.reset_basis(x)
    st.set_schedule(7, 4, 512)
    ref = qsim.State(n, 7, "rel", eps)
    ref.reset_basis(x)
    tiles = [0, 1, x >> 7, (x >> 7) ^ 1, (1 << (n - 7)) - 1]
    assert st.export_tile_set(tiles) == ref.export_tile_set(tiles)
    assert st.stats()["tile_log2"] == 7
    ref.close()
    st.apply(I.h(0))
    st.flush()
    with pytest.raises(qsim.QsimError) as e:
        st.set_schedule(8, 4, 512)
    assert e.value.status == 1
    st.close()
