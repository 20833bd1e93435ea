"""The oracle's single-item sweep equals its whole-state sweep on every item
(so sampled checks of large states use the same arithmetic)."""
import oracle
from oracle.partition import partition
from paper_1811_05140_gb300 import inputs as I


def test_item_sweep_matches_full_sweep():
    n, c, hmax, depth = 11, 5, 4, 12
    gates = I.basis_gates(n, 0x2A5) + I.qft(n) + I.random_grid(*I.grid_shape(n), 3, 4)
    for shifts, norm in (([39], True), ([0], False)):
        cs = oracle.CSim(n, c, shifts, None, norm)
        cs.reset_basis(0)
        for lo, hi, H in partition(gates, n, c, hmax, depth):
            before = [cs.stream(t) for t in range(1 << (n - c))]
            alpha = cs.alpha
            cs.sweep(gates[lo:hi], H)
            hb = [q - c for q in H]
            for T in range(1 << (n - c)):
                if any((T >> b) & 1 for b in hb):
                    continue
                members = []
                for j in range(1 << len(H)):
                    t = T
                    for i, b in enumerate(hb):
                        if (j >> i) & 1:
                            t |= 1 << b
                    members.append(t)
                got = oracle.item_sweep(n, c, H, T, [before[t] for t in members], alpha,
                                        gates[lo:hi], shifts)
                assert got == [cs.stream(t) for t in members]


def test_item_sweep_batch_matches_full_sweep_on_threads():
    # the threaded batch (sampled checks of large states, all-cores timing)
    # gives every item exactly what the whole-state sweep stores
    n, c, hmax, depth = 11, 5, 4, 12
    gates = I.basis_gates(n, 0x1C3) + I.qft(n) + I.random_grid(*I.grid_shape(n), 2, 9)
    shifts = [39]
    cs = oracle.CSim(n, c, shifts, None, True)
    cs.reset_basis(0)
    for lo, hi, H in partition(gates, n, c, hmax, depth):
        before = [cs.stream(t) for t in range(1 << (n - c))]
        alpha = cs.alpha
        cs.sweep(gates[lo:hi], H)
        hb = [q - c for q in sorted(H)]
        bases = [T for T in range(1 << (n - c)) if not any((T >> b) & 1 for b in hb)]
        members = []
        for T in bases:
            for j in range(1 << len(H)):
                t = T
                for i, b in enumerate(hb):
                    if (j >> i) & 1:
                        t |= 1 << b
                members.append(t)
        raw = b"".join(before[t] for t in members)
        sizes = [len(before[t]) for t in members]
        for threads in (1, 3):
            got = oracle.item_sweep_batch(n, c, H, bases, raw, sizes, alpha, gates[lo:hi], shifts,
                                          threads=threads)
            flat = [s for item in got for s in item]
            assert flat == [cs.stream(t) for t in members]
