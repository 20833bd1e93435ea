"""GB300-native compressed full-amplitude quantum circuit simulator.

The state vector lives in HBM as independently compressed tiles; each sweep
decompresses a tile group on chip, applies a run of gates in FP64 complex,
and recompresses it with the amplitude-aware (point-wise relative) codec and
the error-bound ladder of "Amplitude-Aware Lossy Compression for Quantum
Circuit Simulation" (Algorithm 2).  All compute runs in the CUDA library
``libqsim.so`` behind the C ABI declared in ``include/qsim.h``; the Python
modules only marshal arguments.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "State", "load"]


def __getattr__(name):
    if name in ("State", "load", "QsimError"):
        from . import qsim
        return getattr(qsim, name)
    raise AttributeError(name)
