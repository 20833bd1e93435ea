"""CPU oracle (test infrastructure only).

Python access to the plain C oracle in oracle.c:
  O1  dense FP64 simulator (the pair update of Sec. II),
  O2  tile codec (Sec. III relative error-bounded codec, lossless level,
      Algorithm 2's error-bound ladder) in the library's stream format,
  O3  compressed simulator (Algorithm 2 over tiles, sweep by sweep),
  N   exact state norm in fixed point.
plus the sweep partition rule (partition.py).

Only the tests, ``__graft_entry__.smoke`` and the CPU-baseline leg of
``bench.py`` use this package.  It never imports the GPU package, and the
GPU package never imports it.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

from .partition import partition  # noqa: F401

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread"]


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, SRC, "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


class OrGate(C.Structure):
    _fields_ = [
        ("k", C.c_int32),
        ("t", C.c_int32 * 2),
        ("pad", C.c_int32),
        ("cmask", C.c_uint64),
        ("cval", C.c_uint64),
        ("m", C.c_double * 32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        u8p = C.POINTER(C.c_uint8)
        ip = C.POINTER(C.c_int)
        u64p = C.POINTER(C.c_uint64)
        L.or_dense_apply.argtypes = [dp, C.c_int, C.POINTER(OrGate)]
        L.or_dense_apply.restype = C.c_int
        L.or_sum_sq.argtypes = [dp, C.c_uint64, u64p, u64p, ip]
        L.or_units_to_double.argtypes = [C.c_uint64, C.c_uint64]
        L.or_units_to_double.restype = C.c_double
        L.or_shift_for_eps.argtypes = [C.c_double]
        L.or_shift_for_eps.restype = C.c_int
        L.or_stream_cap.argtypes = [C.c_int]
        L.or_stream_cap.restype = C.c_size_t
        L.or_encode_tile.argtypes = [dp, C.c_int, ip, C.c_int, C.c_uint64, u8p, ip, ip]
        L.or_encode_tile.restype = C.c_size_t
        L.or_check_bound.argtypes = [C.c_int, C.c_uint64, C.c_uint64]
        L.or_check_bound.restype = C.c_uint64
        L.or_encode_tile_level.argtypes = [dp, C.c_int, ip, C.c_int, u8p, ip]
        L.or_encode_tile_level.restype = C.c_size_t
        L.or_decode_tile.argtypes = [u8p, C.c_size_t, C.c_int, dp]
        L.or_decode_tile.restype = C.c_int
        L.or_csim_new.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.c_uint64, C.c_int]
        L.or_csim_new.restype = C.c_void_p
        L.or_csim_free.argtypes = [C.c_void_p]
        L.or_csim_reset_basis.argtypes = [C.c_void_p, C.c_uint64]
        L.or_csim_set_unit.argtypes = [C.c_void_p, C.c_int, C.c_uint64]
        L.or_csim_set_unit.restype = C.c_int
        L.or_csim_set_fuse.argtypes = [C.c_void_p, C.c_int]
        L.or_csim_set_polar.argtypes = [C.c_void_p, C.c_int]
        L.or_polar_table.argtypes = [u64p, C.c_int]
        L.or_polar_angle.argtypes = [C.c_double, C.c_double]
        L.or_polar_angle.restype = C.c_uint64
        L.or_polar_recon.argtypes = [C.c_uint64, C.c_uint64, C.c_int, dp, dp]
        L.or_encode_tile_opt.argtypes = [dp, C.c_int, ip, C.c_int, C.c_uint64, C.c_int, u8p, ip, ip]
        L.or_encode_tile_opt.restype = C.c_size_t
        L.or_csim_set_dense.argtypes = [C.c_void_p, dp]
        L.or_csim_sweep.argtypes = [C.c_void_p, C.POINTER(OrGate), C.c_int, ip, C.c_int]
        L.or_csim_sweep.restype = C.c_int
        L.or_csim_sweep_sample.argtypes = [C.c_void_p, C.POINTER(OrGate), C.c_int, ip, C.c_int,
                                           C.c_uint64, C.c_uint64]
        L.or_csim_sweep_sample.restype = C.c_int
        L.or_item_sweep.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.c_uint64,
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_uint32), C.c_double,
                                    C.POINTER(OrGate), C.c_int, ip, C.c_int, C.c_uint64, C.c_int, u8p,
                                    C.c_size_t, C.POINTER(C.c_uint32)]
        L.or_item_sweep.restype = C.c_int
        L.or_item_sweep_batch.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.c_uint64, u64p, u8p, u64p,
                                          C.POINTER(C.c_uint32), C.c_double, C.POINTER(OrGate), C.c_int,
                                          ip, C.c_int, C.c_uint64, C.c_int, u8p, C.c_size_t,
                                          C.POINTER(C.c_uint32), ip, C.c_int]
        L.or_item_sweep_batch.restype = C.c_int
        L.or_stride_sweep.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.c_int, C.c_uint64, C.c_uint64,
                                      u64p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32), C.c_uint64,
                                      C.c_double, C.POINTER(OrGate), C.c_int, ip, C.c_int, C.c_int, u8p,
                                      C.c_size_t, C.POINTER(C.c_uint32)]
        L.or_stride_sweep.restype = C.c_int
        L.or_csim_dense.argtypes = [C.c_void_p, dp]
        L.or_csim_dense.restype = C.c_int
        L.or_csim_stream.argtypes = [C.c_void_p, C.c_uint64, u8p, C.c_uint32]
        L.or_csim_stream.restype = C.c_uint32
        L.or_csim_set_stream.argtypes = [C.c_void_p, C.c_uint64, u8p, C.c_uint32]
        L.or_csim_set_stream.restype = C.c_int
        L.or_csim_refresh_alpha.argtypes = [C.c_void_p]
        L.or_csim_alpha.argtypes = [C.c_void_p]
        L.or_csim_alpha.restype = C.c_double
        L.or_csim_err.argtypes = [C.c_void_p]
        L.or_csim_err.restype = C.c_int
        L.or_csim_norm_units.argtypes = [C.c_void_p, u64p, u64p]
        L.or_csim_bytes.argtypes = [C.c_void_p]
        L.or_csim_bytes.restype = C.c_uint64
        L.or_csim_hist.argtypes = [C.c_void_p, u64p]
        L.or_csim_items.argtypes = [C.c_void_p, u64p, u64p]
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def to_or_gate(g) -> OrGate:
    """Marshal an inputs.Gate into the oracle's struct."""
    og = OrGate()
    k = len(g.targets)
    og.k = k
    for i, t in enumerate(g.targets):
        og.t[i] = t
    cm, cv = g.masks()
    og.cmask = cm
    og.cval = cv
    m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
    for i, v in enumerate(m):
        og.m[2 * i] = v.real
        og.m[2 * i + 1] = v.imag
    return og


def gate_array(gates) -> C.Array:
    arr = (OrGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        arr[i] = to_or_gate(g)
    return arr


# ---------------------------------------------------------------- O1
def dense_zero(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def dense_basis(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def dense_apply(psi: np.ndarray, n: int, gate) -> None:
    """Apply one gate in place to a dense complex128 vector (Sec. II)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous and psi.size == 1 << n
    og = to_or_gate(gate)
    rc = lib().or_dense_apply(_dptr(psi.view(np.float64)), n, C.byref(og))
    if rc != 0:
        raise ValueError("gate target outside the state")


def dense_run(psi: np.ndarray, n: int, gates) -> np.ndarray:
    for g in gates:
        dense_apply(psi, n, g)
    return psi


# ---------------------------------------------------------------- norm
def sum_sq_units(values: np.ndarray) -> int:
    """Exact sum of floor(x^2 * 2^112) over all components."""
    v = np.ascontiguousarray(values).view(np.float64).reshape(-1)
    lo, hi, rng = C.c_uint64(), C.c_uint64(), C.c_int()
    lib().or_sum_sq(_dptr(v), v.size, C.byref(lo), C.byref(hi), C.byref(rng))
    if rng.value:
        raise ValueError("value outside the norm's range (|x| >= 16)")
    return (hi.value << 64) | lo.value


def units_to_double(S: int) -> float:
    return lib().or_units_to_double(S & ((1 << 64) - 1), S >> 64)


# ---------------------------------------------------------------- O2
def shift_for_eps(eps: float) -> int:
    return lib().or_shift_for_eps(eps)


def max_bytes_for(c: int, theta: float | None) -> int:
    """Largest stream size whose ratio 16*2^c/size is >= theta."""
    if theta is None or theta <= 0:
        return (1 << 64) - 1
    return int(math.floor((16.0 * (1 << c)) / theta))


def encode_tile(amps: np.ndarray, c: int, shifts, max_bytes: int | None = None, polar: bool = False):
    """Encode 2^c amplitudes; returns (stream bytes, level, flags).  polar:
    every lossy level also tries the POLAR mode and keeps the shorter."""
    a = np.ascontiguousarray(amps, dtype=np.complex128)
    assert a.size == 1 << c
    sh = (C.c_int * len(shifts))(*shifts)
    cap = lib().or_stream_cap(c)
    out = (C.c_uint8 * cap)()
    level, flags = C.c_int(), C.c_int()
    mb = (1 << 64) - 1 if max_bytes is None else max_bytes
    n = lib().or_encode_tile_opt(_dptr(a.view(np.float64)), c, sh, len(shifts), mb, int(bool(polar)), out,
                                 C.byref(level), C.byref(flags))
    return bytes(out[:n]), level.value, flags.value


def polar_table(count: int = 30) -> list[int]:
    """The POLAR mode's angle table: round(2^64 atan(2^-k) / (2 pi))."""
    out = (C.c_uint64 * count)()
    lib().or_polar_table(out, count)
    return list(out)


def polar_angle(x: float, y: float) -> int:
    """Angle of (x, y) in units of 2^-64 turn (the POLAR mode's CORDIC)."""
    return lib().or_polar_angle(x, y)


def polar_recon(qm: int, qa: int, s: int) -> complex:
    """The POLAR reconstruction of magnitude code qm and angle code qa at shift s."""
    re, im = C.c_double(), C.c_double()
    lib().or_polar_recon(qm, qa, s, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def check_bound(s: int, count: int, seed: int) -> int:
    """Violations of |x^ - x| < 2^(s-53)|x| over count seeded random
    magnitudes through the quantiser (0 expected)."""
    return lib().or_check_bound(s, count, seed)


def encode_tile_level(amps: np.ndarray, c: int, shifts, k: int):
    """Encode 2^c amplitudes at ladder level k, no size test; (bytes, flags)."""
    a = np.ascontiguousarray(amps, dtype=np.complex128)
    assert a.size == 1 << c and 0 <= k < len(shifts)
    sh = (C.c_int * len(shifts))(*shifts)
    out = (C.c_uint8 * lib().or_stream_cap(c))()
    flags = C.c_int()
    n = lib().or_encode_tile_level(_dptr(a.view(np.float64)), c, sh, k, out, C.byref(flags))
    return bytes(out[:n]), flags.value


def decode_tile(stream: bytes, c: int) -> np.ndarray:
    a = np.zeros(1 << c, dtype=np.complex128)
    buf = (C.c_uint8 * len(stream)).from_buffer_copy(stream)
    rc = lib().or_decode_tile(buf, len(stream), c, _dptr(a.view(np.float64)))
    if rc != 0:
        raise ValueError(f"malformed stream ({rc})")
    return a


def _opts(fuse: bool, polar: bool) -> int:
    return int(bool(fuse)) | (int(bool(polar)) << 1)


def item_sweep(n: int, c: int, H, base_tile: int, streams, alpha: float, gates, shifts,
               max_bytes: int | None = None, fuse: bool = True, polar: bool = False):
    """One item of a sweep on its own (sampled checks of large states):
    member j is tile base_tile | bits of j at H; returns the new streams."""
    H = sorted(H)
    h = len(H)
    assert len(streams) == 1 << h
    bufs = [(C.c_uint8 * len(st)).from_buffer_copy(st) for st in streams]
    ptrs = (C.c_void_p * len(bufs))(*[C.addressof(b) for b in bufs])
    lens = (C.c_uint32 * len(bufs))(*[len(st) for st in streams])
    hh = (C.c_int * max(1, h))(*H)
    sh = (C.c_int * len(shifts))(*shifts)
    cap = len(streams) * lib().or_stream_cap(c)
    out = (C.c_uint8 * cap)()
    out_len = (C.c_uint32 * len(streams))()
    arr = gate_array(gates)
    mb = (1 << 64) - 1 if max_bytes is None else max_bytes
    rc = lib().or_item_sweep(n, c, hh, h, base_tile, ptrs, lens, alpha, arr, len(gates), sh,
                             len(shifts), mb, _opts(fuse, polar), out, cap, out_len)
    if rc != 0:
        raise RuntimeError(f"oracle item sweep failed ({rc})")
    res, off = [], 0
    raw = bytes(out)
    for j in range(len(streams)):
        res.append(raw[off:off + out_len[j]])
        off += out_len[j]
    return res


def item_sweep_batch(n: int, c: int, H, bases, raw: bytes, sizes, alpha: float, gates, shifts,
                     max_bytes: int | None = None, threads: int | None = None, fuse: bool = True,
                     polar: bool = False):
    """Many items of one sweep, each as item_sweep computes it, on `threads`
    host threads (default: every core).  raw holds the members' streams
    concatenated item by item (member order as in item_sweep), sizes their
    lengths.  Returns a list, per item, of the members' new streams."""
    H = sorted(H)
    h = len(H)
    nm = 1 << h
    nitems = len(bases)
    assert len(sizes) == nitems * nm
    if nitems == 0:
        return []
    threads = threads or os.cpu_count() or 1
    offs = np.zeros(len(sizes), dtype=np.uint64)
    np.cumsum(np.asarray(sizes[:-1], dtype=np.uint64), out=offs[1:])
    inb = np.frombuffer(raw, dtype=np.uint8) if raw else np.zeros(1, np.uint8)
    inb = np.ascontiguousarray(inb)
    lens = np.asarray(sizes, dtype=np.uint32)
    bs = np.asarray(bases, dtype=np.uint64)
    stride = nm * lib().or_stream_cap(c)
    out = np.zeros(nitems * stride, dtype=np.uint8)
    out_len = np.zeros(nitems * nm, dtype=np.uint32)
    rc = np.zeros(nitems, dtype=np.int32)
    hh = (C.c_int * max(1, h))(*H)
    sh = (C.c_int * len(shifts))(*shifts)
    arr = gate_array(gates)
    mb = (1 << 64) - 1 if max_bytes is None else max_bytes
    u64p = C.POINTER(C.c_uint64)
    u8p = C.POINTER(C.c_uint8)
    bad = lib().or_item_sweep_batch(
        n, c, hh, h, nitems, bs.ctypes.data_as(u64p), inb.ctypes.data_as(u8p), offs.ctypes.data_as(u64p),
        lens.ctypes.data_as(C.POINTER(C.c_uint32)), alpha, arr, len(gates), sh, len(shifts), mb,
        _opts(fuse, polar), out.ctypes.data_as(u8p), stride, out_len.ctypes.data_as(C.POINTER(C.c_uint32)),
        rc.ctypes.data_as(C.POINTER(C.c_int)), threads)
    if bad:
        raise RuntimeError(f"oracle item sweep failed for {bad} item(s), codes {sorted(set(rc.tolist()))}")
    res = []
    for i in range(nitems):
        off = i * stride
        mem = []
        for j in range(nm):
            ln = int(out_len[i * nm + j])
            mem.append(out[off:off + ln].tobytes())
            off += ln
        res.append(mem)
    return res


def stride_items_tiles(c: int, H, stride_log2: int, t0: int) -> list[int]:
    """Every member tile of every item that holds a tile of the stride of
    2^(stride_log2 - c) tiles starting at tile t0 (ascending)."""
    hb = [q - c for q in sorted(H)]
    hmask = sum(1 << b for b in hb)
    nt = 1 << (stride_log2 - c)
    out = set()
    for t in range(t0, t0 + nt):
        T = t & ~hmask
        for j in range(1 << len(hb)):
            out.add(T | sum(1 << b for i, b in enumerate(hb) if (j >> i) & 1))
    return sorted(out)


def stride_sweep(n: int, c: int, H, stride_log2: int, theta: float, t0: int, streams: dict,
                 alpha: float, gates, shifts, fuse: bool = True, polar: bool = False):
    """One stride of a sweep that decides per stride (sampled checks of large
    states): streams maps every tile of stride_items_tiles(...) to its input
    stream; returns the stride's new streams in tile order."""
    H = sorted(H)
    ut = stride_log2 - c
    tiles = sorted(streams)
    bufs = [(C.c_uint8 * len(streams[t])).from_buffer_copy(streams[t]) for t in tiles]
    ptrs = (C.c_void_p * len(bufs))(*[C.addressof(b) for b in bufs])
    lens = (C.c_uint32 * len(bufs))(*[len(streams[t]) for t in tiles])
    tarr = (C.c_uint64 * len(tiles))(*tiles)
    hh = (C.c_int * max(1, len(H)))(*H)
    sh = (C.c_int * len(shifts))(*shifts)
    cap = (1 << ut) * lib().or_stream_cap(c)
    out = (C.c_uint8 * cap)()
    out_len = (C.c_uint32 * (1 << ut))()
    arr = gate_array(gates)
    rc = lib().or_stride_sweep(n, c, hh, len(H), ut, max_bytes_for(stride_log2, theta), t0, tarr, ptrs,
                               lens, len(tiles), alpha, arr, len(gates), sh, len(shifts),
                               _opts(fuse, polar), out, cap, out_len)
    if rc != 0:
        raise RuntimeError(f"oracle stride sweep failed ({rc})")
    res, off = [], 0
    raw = bytes(out)
    for j in range(1 << ut):
        res.append(raw[off:off + out_len[j]])
        off += out_len[j]
    return res


# ---------------------------------------------------------------- O3
class CSim:
    """Algorithm 2 over tiles of 2^c amplitudes (the compressed simulator).

    shifts: ladder of quantisation shifts (one entry for a fixed bound);
    max_bytes: the ratio threshold as a size limit (None = no threshold);
    normalize: apply 'normalize' before each sweep's gate computation;
    fuse: runs of two or more consecutive diagonal gates of a sweep are one
    diagonal operator (False: every gate on its own, so that lossless
    sweeps reproduce the dense simulator bit for bit); polar: every lossy
    level also tries the POLAR mode (magnitude + phase) and keeps the
    shorter stream.
    """

    def __init__(self, n: int, c: int, shifts, max_bytes: int | None = None,
                 normalize: bool = True, fuse: bool = True, polar: bool = False):
        self.n, self.c = n, c
        self.shifts = list(shifts)
        sh = (C.c_int * len(self.shifts))(*self.shifts)
        mb = (1 << 64) - 1 if max_bytes is None else max_bytes
        self.h = lib().or_csim_new(n, c, sh, len(self.shifts), mb, int(normalize))
        if not self.h:
            raise ValueError("bad oracle state parameters")
        lib().or_csim_set_fuse(self.h, int(bool(fuse)))
        lib().or_csim_set_polar(self.h, int(bool(polar)))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_csim_free(self.h)
            self.h = None

    def reset_basis(self, x: int = 0):
        lib().or_csim_reset_basis(self.h, x)

    def set_unit(self, unit_log2: int, theta: float) -> int:
        """One ladder decision per stride of 2^unit_log2 amplitudes (the
        stride Algorithm 2 decides on), ratio threshold theta; 0 = per tile.
        Returns log2 of the tiles per decision."""
        u = min(max(unit_log2, self.c), self.n)
        return lib().or_csim_set_unit(self.h, unit_log2, max_bytes_for(u, theta))

    def set_dense(self, amps: np.ndarray):
        a = np.ascontiguousarray(amps, dtype=np.complex128)
        assert a.size == 1 << self.n
        lib().or_csim_set_dense(self.h, _dptr(a.view(np.float64)))

    def sweep(self, gates, H):
        H = sorted(H)
        arr = gate_array(gates)
        hh = (C.c_int * max(1, len(H)))(*H)
        rc = lib().or_csim_sweep(self.h, arr, len(gates), hh, len(H))
        if rc != 0:
            raise RuntimeError(f"oracle sweep failed ({rc})")

    def sweep_sample(self, gates, H, item_lo: int, item_hi: int):
        """The sweep on items item_lo..item_hi-1 only (timing samples)."""
        H = sorted(H)
        arr = gate_array(gates)
        hh = (C.c_int * max(1, len(H)))(*H)
        rc = lib().or_csim_sweep_sample(self.h, arr, len(gates), hh, len(H), item_lo, item_hi)
        if rc != 0:
            raise RuntimeError(f"oracle sweep failed ({rc})")

    def run(self, gates, hmax: int, depth: int):
        """Apply gates with the sweep partition rule; returns the sweeps."""
        sweeps = partition(gates, self.n, self.c, hmax, depth)
        for lo, hi, H in sweeps:
            self.sweep(gates[lo:hi], H)
        return sweeps

    def dense(self) -> np.ndarray:
        out = np.zeros(1 << self.n, dtype=np.complex128)
        if lib().or_csim_dense(self.h, _dptr(out.view(np.float64))) != 0:
            raise RuntimeError("malformed stream in oracle state")
        return out

    def stream(self, t: int) -> bytes:
        L = lib()
        n = L.or_csim_stream(self.h, t, None, 0)
        buf = (C.c_uint8 * n)()
        L.or_csim_stream(self.h, t, buf, n)
        return bytes(buf)

    def set_stream(self, t: int, data: bytes) -> int:
        buf = (C.c_uint8 * len(data)).from_buffer_copy(data)
        return lib().or_csim_set_stream(self.h, t, buf, len(data))

    def refresh_alpha(self):
        lib().or_csim_refresh_alpha(self.h)

    @property
    def alpha(self) -> float:
        return lib().or_csim_alpha(self.h)

    @property
    def err(self) -> int:
        return lib().or_csim_err(self.h)

    def norm_units(self) -> int:
        lo, hi = C.c_uint64(), C.c_uint64()
        lib().or_csim_norm_units(self.h, C.byref(lo), C.byref(hi))
        return (hi.value << 64) | lo.value

    def norm(self) -> float:
        return units_to_double(self.norm_units())

    def nbytes(self) -> int:
        return lib().or_csim_bytes(self.h)

    def hist(self) -> list[int]:
        out = (C.c_uint64 * 8)()
        lib().or_csim_hist(self.h, out)
        return list(out)

    def items(self) -> tuple[int, int]:
        d, s = C.c_uint64(), C.c_uint64()
        lib().or_csim_items(self.h, C.byref(d), C.byref(s))
        return d.value, s.value
