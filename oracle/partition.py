"""Sweep partition rule, restated for the oracle (test infrastructure).

Algorithm 1 visits every stride once per gate.  A sweep generalises one
visit to a run of consecutive gates: every tile group (item) is
decompressed once, the whole run is applied, and the item is compressed
once.  A run may only contain gates whose mixing qubits are inside the
item: the low qubits (index < c, inside one tile) plus at most hmax high
qubits H, whose partner tiles are loaded together (a target qubit at or
above the stride size needs the partner stride, which Algorithm 1 leaves
unsaid).

Rule: walk the gates in order.  A gate's mixing set is its targets when its
matrix has a nonzero off-diagonal entry, otherwise empty (a diagonal gate
only scales amplitudes and can use any qubit).  Add the gate to the open
sweep while the union of H with the gate's high mixing qubits has at most
hmax members and the sweep has fewer than `depth` gates; otherwise close
the sweep and open a new one with this gate.  A closed sweep's H is then
filled up to min(hmax, n - c) qubits with the smallest high qubits not
already in it, so that every item holds the same number of tiles.
"""
from __future__ import annotations

import numpy as np


def is_diagonal(matrix) -> bool:
    m = np.asarray(matrix)
    off = m - np.diag(np.diag(m))
    return not np.any(off != 0)


def partition(gates, n: int, c: int, hmax: int, depth: int):
    """Return [(lo, hi, H)] with gates[lo:hi] forming one sweep."""
    hcap = min(hmax, n - c)
    sweeps = []

    def padded(H):
        H = set(H)
        q = c
        while len(H) < hcap and q < n:
            H.add(q)
            q += 1
        return tuple(sorted(H))

    lo = 0
    H: set = set()
    for i, g in enumerate(gates):
        mix = set() if is_diagonal(g.matrix) else {t for t in g.targets if t >= c}
        if len(mix) > hcap:
            raise ValueError("gate needs more paired high qubits than allowed")
        if i > lo and (len(H | mix) > hcap or i - lo >= depth):
            sweeps.append((lo, i, padded(H)))
            lo = i
            H = set()
        H |= mix
    if lo < len(gates):
        sweeps.append((lo, len(gates), padded(H)))
    return sweeps
