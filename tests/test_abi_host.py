"""Host-only checks of the C ABI library (no GPU needed).

* libqsim.so loads and exports every function include/qsim.h declares.
* The library's sweep planner gives the same partition as the oracle's
  independently written rule (oracle/partition.py).
* Calls that need a device fail with an error status, not a crash, when
  there is none.
"""
import os
import re

import pytest

import oracle
from paper_1811_05140_gb300 import inputs as I
from paper_1811_05140_gb300 import qsim

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1811_05140_gb300 import build
    build.build()
    return qsim.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "qsim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(qsim.EXPORTS)
    assert lib.qsim_version().decode().startswith("qsim-aalc")


@pytest.mark.parametrize("n,c,hmax,depth", [(14, 6, 2, 1), (14, 6, 2, 7), (14, 10, 2, 64), (20, 10, 2, 4096),
                                            (12, 8, 1, 16), (5, 3, 2, 3)])
def test_plan_matches_oracle_partition(lib, n, c, hmax, depth):
    gates = I.qft(n) + I.grover(n, 77 % (1 << n), 1) + I.random_grid(*I.grid_shape(n), 4, 3)
    if hmax == 1:
        gates = [g for g in gates if len(g.targets) == 1]
    got = qsim.plan_sweeps(n, c, hmax, depth, gates)
    want = oracle.partition(gates, n, c, hmax, depth)
    assert got == [(lo, hi, tuple(H)) for lo, hi, H in want]


def test_plan_rejects_gates_needing_more_pairs(lib):
    with pytest.raises(ValueError):
        qsim.plan_sweeps(12, 6, 1, 8, [I.swap(8, 10)])


def test_create_without_device_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(qsim.QsimError) as e:
        qsim.State(10, 8, "rel", 1e-4)
    assert e.value.status == 3            # QSIM_ERR_CUDA


def test_header_compiles_as_c_and_links(lib, tmp_path):
    """A plain C99 program (tests/abi_example.c) builds against
    include/qsim.h with warnings as errors, links libqsim.so and runs: the
    host-only planner works, and creating a state either succeeds (GPU
    present) or returns QSIM_ERR_CUDA with a message."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_1811_05140_gb300")
    exe = os.path.join(str(tmp_path), "abi_example")
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_example.c"),
                           "-o", exe, "-L", libdir, "-lqsim", "-Wl,-rpath," + libdir, "-lm"])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.split("\n")
    assert lines[0].startswith("sweeps ") and int(lines[0].split()[1]) >= 1
    assert lines[1].startswith("create 3 ") or lines[1].startswith("fidelity ")
