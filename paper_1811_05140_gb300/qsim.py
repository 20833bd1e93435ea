"""Python binding of the C ABI in include/qsim.h (argument marshalling only).

Every step of the simulation runs in libqsim.so.  Importing this module
loads that library and fails loudly if it has not been built; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import inputs

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqsim.so")

CODECS = {"none": 0, "lossless": 1, "rel": 2, "aalc": 3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NONFINITE",
          5: "ERR_TIMEOUT", 6: "ERR_STATE_INVALID", 7: "ERR_FORMAT"}
QSIM_OK, QSIM_ERR_ARG, QSIM_ERR_OOM, QSIM_ERR_CUDA = 0, 1, 2, 3
QSIM_ERR_NONFINITE, QSIM_ERR_TIMEOUT, QSIM_ERR_STATE_INVALID, QSIM_ERR_FORMAT = 4, 5, 6, 7
REF_HANDLE, REF_QFT, REF_GROVER, REF_DENSE_HOST, REF_DENSE_DEVICE = range(5)

EXPORTS = ["qsim_create", "qsim_destroy", "qsim_set_stream", "qsim_set_aalc", "qsim_set_normalize",
           "qsim_set_schedule", "qsim_reset_basis", "qsim_set_amplitudes", "qsim_apply_gate",
           "qsim_flush", "qsim_probabilities", "qsim_amplitudes", "qsim_fidelity",
           "qsim_compressed_bytes", "qsim_stats", "qsim_last_error", "qsim_export_tiles",
           "qsim_import_tiles", "qsim_plan_sweeps", "qsim_version", "qsim_set_profiling",
           "qsim_profile", "qsim_encode_noalloc", "qsim_flush_batch", "qsim_server_create",
           "qsim_server_submit", "qsim_server_result", "qsim_server_wait", "qsim_server_drain",
           "qsim_server_stats", "qsim_server_destroy", "qsim_set_pool", "qsim_fp64_rate",
           "qsim_save", "qsim_load", "qsim_set_aalc_unit", "qsim_export_tile_set",
           "qsim_set_fusion", "qsim_set_sweep_threads", "qsim_set_polar"]


class QsimError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Ref(C.Structure):
    _fields_ = [("kind", C.c_int), ("other", C.c_void_p), ("x", C.c_ulonglong),
                ("iterations", C.c_int), ("dense", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("gates", C.c_ulonglong), ("sweeps", C.c_ulonglong),
                ("items_done", C.c_ulonglong), ("items_skipped", C.c_ulonglong),
                ("level_hist", C.c_ulonglong * 8), ("stream_bytes", C.c_ulonglong),
                ("min_stream_bytes_seen", C.c_ulonglong), ("max_stream_bytes_seen", C.c_ulonglong),
                ("arena_regrows", C.c_ulonglong), ("kernel_launches", C.c_ulonglong),
                ("alpha", C.c_double),
                ("tile_log2", C.c_int), ("hmax", C.c_int), ("depth", C.c_int),
                ("n_qubits", C.c_int), ("h2d_bytes", C.c_ulonglong), ("d2h_bytes", C.c_ulonglong),
                ("tiles_over_limit", C.c_ulonglong)]


class Profile(C.Structure):
    _fields_ = [("sweep_launches", C.c_ulonglong), ("sweep_ms", C.c_double),
                ("dp_ops", C.c_double), ("bytes", C.c_double),
                ("kernel_launches", C.c_ulonglong)]


class GateRec(C.Structure):
    _fields_ = [("n_targets", C.c_int), ("targets", C.c_int * 2), ("pad", C.c_int),
                ("control_mask", C.c_ulonglong), ("control_values", C.c_ulonglong),
                ("matrix", C.c_double * 32)]


class Request(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("block_log2", C.c_int), ("codec", C.c_int),
                ("n_readout", C.c_int), ("rel_err_bound", C.c_double), ("theta", C.c_double),
                ("basis", C.c_ulonglong), ("gates", C.POINTER(GateRec)), ("n_gates", C.c_int),
                ("readout", C.c_int * 16), ("tile_log2", C.c_int), ("hmax", C.c_int),
                ("depth", C.c_int), ("sweep_threads", C.c_int)]


class TicketInfo(C.Structure):
    _fields_ = [("done", C.c_int), ("status", C.c_int), ("submit_s", C.c_double),
                ("admit_s", C.c_double), ("finish_s", C.c_double),
                ("stream_bytes", C.c_ulonglong), ("peak_footprint", C.c_ulonglong)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_ulonglong), ("completed", C.c_ulonglong),
                ("failed", C.c_ulonglong), ("ticks", C.c_ulonglong),
                ("peak_footprint", C.c_ulonglong), ("budget", C.c_ulonglong),
                ("busy_s", C.c_double), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double),
                ("throughput_cps", C.c_double), ("max_resident_seen", C.c_int)]


_lib = None


def load() -> C.CDLL:
    """Load libqsim.so (built by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, u64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_ulonglong
    u64p = C.POINTER(C.c_ulonglong)
    sig = {
        "qsim_create": ([C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_double], C.c_int),
        "qsim_destroy": ([vp], C.c_int),
        "qsim_set_stream": ([vp, vp], C.c_int),
        "qsim_set_aalc": ([vp, C.c_double, dp, C.c_int], C.c_int),
        "qsim_set_aalc_unit": ([vp, C.c_int], C.c_int),
        "qsim_set_normalize": ([vp, C.c_int], C.c_int),
        "qsim_set_fusion": ([vp, C.c_int], C.c_int),
        "qsim_set_sweep_threads": ([vp, C.c_int], C.c_int),
        "qsim_set_polar": ([vp, C.c_int], C.c_int),
        "qsim_set_schedule": ([vp, C.c_int, C.c_int, C.c_int], C.c_int),
        "qsim_set_pool": ([vp, vp, C.c_size_t], C.c_int),
        "qsim_fp64_rate": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
        "qsim_save": ([vp, C.c_char_p], C.c_int),
        "qsim_load": ([C.POINTER(vp), C.c_char_p], C.c_int),
        "qsim_reset_basis": ([vp, u64], C.c_int),
        "qsim_set_amplitudes": ([vp, dp], C.c_int),
        "qsim_apply_gate": ([vp, dp, ip, C.c_int, ip, C.c_int, u64], C.c_int),
        "qsim_flush": ([vp], C.c_int),
        "qsim_flush_batch": ([C.POINTER(vp), C.c_int, C.c_int], C.c_int),
        "qsim_server_create": ([C.POINTER(vp), u64, C.c_int, C.c_int, C.c_int], C.c_int),
        "qsim_server_submit": ([vp, C.POINTER(Request), u64p], C.c_int),
        "qsim_server_result": ([vp, u64, C.POINTER(TicketInfo), dp], C.c_int),
        "qsim_server_wait": ([vp, u64, C.c_double], C.c_int),
        "qsim_server_drain": ([vp, C.c_double], C.c_int),
        "qsim_server_stats": ([vp, C.POINTER(ServerStats)], C.c_int),
        "qsim_server_destroy": ([vp], C.c_int),
        "qsim_probabilities": ([vp, ip, C.c_int, dp], C.c_int),
        "qsim_amplitudes": ([vp, u64, u64, dp], C.c_int),
        "qsim_fidelity": ([vp, C.POINTER(Ref), dp, dp], C.c_int),
        "qsim_compressed_bytes": ([vp, u64p, u64p], C.c_int),
        "qsim_stats": ([vp, C.POINTER(Stats)], C.c_int),
        "qsim_last_error": ([vp], C.c_char_p),
        "qsim_export_tiles": ([vp, u64, u64, vp, u64, u64p], C.c_int),
        "qsim_export_tile_set": ([vp, u64p, u64, vp, u64, u64p], C.c_int),
        "qsim_import_tiles": ([vp, u64, u64, vp, u64p], C.c_int),
        "qsim_plan_sweeps": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, dp, ip, ip,
                              ip, C.c_int], C.c_int),
        "qsim_version": ([], C.c_char_p),
        "qsim_set_profiling": ([vp, C.c_int], C.c_int),
        "qsim_profile": ([vp, C.POINTER(Profile)], C.c_int),
        "qsim_encode_noalloc": ([vp, C.c_int, C.c_int, C.c_double, vp, u64, vp, u64p, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def gate_args(g: inputs.Gate):
    """(matrix, targets, n_targets, controls, n_controls, control_values) for qsim_apply_gate."""
    m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128)).view(np.float64)
    t = (C.c_int * 2)(*g.targets, *([0] * (2 - len(g.targets))))
    nc = len(g.controls)
    ctl = (C.c_int * max(1, nc))(*g.controls)
    vals = 0
    for i, v in enumerate(g.cvals()):
        if v:
            vals |= 1 << i
    return m, t, len(g.targets), ctl, nc, vals


def plan_sweeps(n: int, c: int, hmax: int, depth: int, gates) -> list[tuple[int, int, tuple]]:
    """The library's sweep partition of a gate list (host only, no GPU)."""
    L = load()
    ng = len(gates)
    nt = (C.c_int * max(1, ng))(*[len(g.targets) for g in gates])
    tg = (C.c_int * max(2, 2 * ng))()
    mats = np.zeros((max(1, ng), 32))
    for i, g in enumerate(gates):
        for j, q in enumerate(g.targets):
            tg[2 * i + j] = q
        m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
        mats[i, :2 * m.size] = m.view(np.float64)
    cap = max(1, ng)
    lo, hh, HH = (C.c_int * cap)(), (C.c_int * cap)(), (C.c_int * (4 * cap))()
    r = L.qsim_plan_sweeps(n, c, hmax, depth, ng, nt, tg, _dp(mats), lo, hh, HH, cap)
    if r < 0:
        raise ValueError(f"qsim_plan_sweeps failed ({r})")
    out = []
    for s in range(r):
        hi = lo[s + 1] if s + 1 < r else ng
        out.append((lo[s], hi, tuple(HH[4 * s + i] for i in range(hh[s]))))
    return out


def fp64_rate(device: int = 0) -> float:
    """Measured FP64 FMA rate of the GPU (FMA per second)."""
    L = load()
    out = C.c_double()
    st = L.qsim_fp64_rate(device, C.byref(out))
    if st != 0:
        raise QsimError(st, L.qsim_last_error(None).decode())
    return out.value


def encode_noalloc(dev_amps: int, n: int, tile_log2: int, eps: float, dev_out: int,
                   out_cap: int, dev_table: int, stream=None, check: bool = True):
    """qsim_encode_noalloc on device pointers; returns the stream bytes used
    (check=False: returns (status, bytes used or needed) without raising)."""
    L = load()
    used = C.c_ulonglong()
    ptr = getattr(stream, "cuda_stream", stream)
    st = L.qsim_encode_noalloc(C.c_void_p(dev_amps), n, tile_log2, eps, C.c_void_p(dev_out),
                               out_cap, C.c_void_p(dev_table), C.byref(used), C.c_void_p(ptr or 0))
    if not check:
        return st, used.value
    if st != 0:
        raise QsimError(st, L.qsim_last_error(None).decode())
    return used.value


def flush_batch(states, use_graph: bool = False):
    """Flush several states together (qsim_flush_batch)."""
    L = load()
    arr = (C.c_void_p * len(states))(*[s.h for s in states])
    st = L.qsim_flush_batch(arr, len(states), int(bool(use_graph)))
    if st != 0:
        msgs = [s._L.qsim_last_error(s.h).decode() for s in states]
        raise QsimError(st, "; ".join(m for m in msgs if m) or L.qsim_last_error(None).decode())


class State:
    """An n-qubit state held compressed on the GPU (one qsim_t handle)."""

    def __init__(self, n: int, block_log2: int, codec: str = "rel", eps: float = 1e-4,
                 stream=None):
        self._L = load()
        h = C.c_void_p()
        self._check(self._L.qsim_create(C.byref(h), n, block_log2, CODECS[codec], eps), None)
        self.h = h
        self.n = n
        self.block_log2 = block_log2
        self.codec = codec
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def load(cls, path: str, stream=None) -> "State":
        """A state restored from a checkpoint written by save()."""
        L = load()
        h = C.c_void_p()
        st = L.qsim_load(C.byref(h), os.fsencode(path))
        if st != 0:
            raise QsimError(st, L.qsim_last_error(None).decode())
        self = cls.__new__(cls)
        self._L = L
        self.h = h
        self.n = self.stats()["n_qubits"]
        self.block_log2 = None              # the stride decision unit is restored from the file
        self.codec = None
        if stream is not None:
            self.set_stream(stream)
        return self

    def save(self, path: str):
        """Write a checkpoint (header and every tile stream) to path."""
        self._check(self._L.qsim_save(self.h, os.fsencode(path)))

    # -- plumbing
    def _check(self, status: int, h=-1):
        if status != 0:
            hh = self.h if h == -1 else h
            msg = self._L.qsim_last_error(hh).decode()
            raise QsimError(status, msg)

    def close(self):
        if getattr(self, "h", None):
            self._L.qsim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        self._check(self._L.qsim_set_stream(self.h, C.c_void_p(ptr or 0)))

    # -- configuration
    def set_aalc(self, theta: float, levels):
        arr = (C.c_double * max(1, len(levels)))(*levels)
        self._check(self._L.qsim_set_aalc(self.h, theta, arr, len(levels)))

    def set_aalc_unit(self, unit_log2: int | None = None):
        """One ladder decision per stride of 2^unit_log2 amplitudes
        (default: the block_log2 of the constructor, Algorithm 2's stride);
        0 decides per tile."""
        u = self.block_log2 if unit_log2 is None else unit_log2
        if u is None:
            raise ValueError("give unit_log2 for a state loaded from a checkpoint")
        self._check(self._L.qsim_set_aalc_unit(self.h, int(u)))

    def set_normalize(self, on: bool):
        self._check(self._L.qsim_set_normalize(self.h, int(bool(on))))

    def set_polar(self, on: bool = True):
        """Lossy levels also try the POLAR mode (magnitude + phase)."""
        self._check(self._L.qsim_set_polar(self.h, int(bool(on))))

    def set_sweep_threads(self, threads: int):
        """CTA size of the sweep kernel (128, 256 or 512)."""
        self._check(self._L.qsim_set_sweep_threads(self.h, int(threads)))

    def set_fusion(self, diag_runs: bool):
        """Runs of consecutive diagonal gates as one operator (default) or
        every gate on its own."""
        self._check(self._L.qsim_set_fusion(self.h, int(bool(diag_runs))))

    def set_schedule(self, tile_log2: int, hmax: int = 4, depth: int = 512):
        self._check(self._L.qsim_set_schedule(self.h, tile_log2, hmax, depth))

    def set_pool(self, buf=None, nbytes: int | None = None):
        """Put the stream arenas in a caller-owned device buffer: a CUDA
        torch tensor (its storage is used; keep the tensor alive) or a raw
        device pointer with nbytes.  None moves them back to the library."""
        if buf is None:
            self._check(self._L.qsim_set_pool(self.h, None, 0))
            self._pool = None
            return
        if hasattr(buf, "data_ptr"):
            ptr = buf.data_ptr()
            size = buf.numel() * buf.element_size() if nbytes is None else nbytes
        else:
            ptr, size = int(buf), int(nbytes)
        self._check(self._L.qsim_set_pool(self.h, C.c_void_p(ptr), size))
        self._pool = buf                  # keeps a tensor alive with the handle

    # -- state
    def reset_basis(self, x: int = 0):
        self._check(self._L.qsim_reset_basis(self.h, x))

    def set_amplitudes(self, psi: np.ndarray):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        assert a.size == 1 << self.n
        self._check(self._L.qsim_set_amplitudes(self.h, _dp(a.view(np.float64))))

    def apply(self, g: inputs.Gate):
        m, t, nt, ctl, nc, vals = gate_args(g)
        self._check(self._L.qsim_apply_gate(self.h, _dp(m), t, nt, ctl, nc, vals))

    def apply_all(self, gates):
        for g in gates:
            self.apply(g)

    def flush(self):
        self._check(self._L.qsim_flush(self.h))

    # -- read-outs
    def amplitudes(self, start: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = (1 << self.n) - start
        out = np.zeros(count, dtype=np.complex128)
        self._check(self._L.qsim_amplitudes(self.h, start, count, _dp(out.view(np.float64))))
        return out

    def probabilities(self, qubits) -> np.ndarray:
        qs = (C.c_int * max(1, len(qubits)))(*qubits)
        out = np.zeros(1 << len(qubits))
        self._check(self._L.qsim_probabilities(self.h, qs, len(qubits), _dp(out)))
        return out

    def _fid(self, ref: Ref) -> tuple[float, float]:
        F, ov = C.c_double(), C.c_double()
        self._check(self._L.qsim_fidelity(self.h, C.byref(ref), C.byref(F), C.byref(ov)))
        return F.value, ov.value

    def fidelity_qft(self, x: int) -> float:
        return self._fid(Ref(REF_QFT, None, x, 0, None))[0]

    def fidelity_grover(self, marked: int, iterations: int) -> float:
        return self._fid(Ref(REF_GROVER, None, marked, iterations, None))[0]

    def fidelity_dense(self, psi: np.ndarray) -> float:
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        return self._fid(Ref(REF_DENSE_HOST, None, 0, 0, a.ctypes.data))[0]

    def fidelity_device(self, ptr: int) -> float:
        return self._fid(Ref(REF_DENSE_DEVICE, None, 0, 0, ptr))[0]

    def fidelity_state(self, other: "State") -> float:
        return self._fid(Ref(REF_HANDLE, other.h, 0, 0, None))[0]

    def compressed_bytes(self) -> tuple[int, int]:
        a, b = C.c_ulonglong(), C.c_ulonglong()
        self._check(self._L.qsim_compressed_bytes(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.qsim_stats(self.h, C.byref(s)))
        d = {f: getattr(s, f) for f, _ in Stats._fields_}
        d["level_hist"] = list(s.level_hist)
        return d

    def set_profiling(self, on: bool = True):
        self._check(self._L.qsim_set_profiling(self.h, int(bool(on))))

    def profile(self) -> dict:
        p = Profile()
        self._check(self._L.qsim_profile(self.h, C.byref(p)))
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    # -- tile streams
    def export_tiles(self, first: int = 0, count: int | None = None) -> list[bytes]:
        st = self.stats()
        ntiles = 1 << (self.n - st["tile_log2"])
        if count is None:
            count = ntiles - first
        sizes = (C.c_ulonglong * max(1, count))()
        self._check(self._L.qsim_export_tiles(self.h, first, count, None, 0, sizes))
        total = sum(sizes[:count])
        buf = (C.c_uint8 * max(1, total))()
        self._check(self._L.qsim_export_tiles(self.h, first, count, buf, total, sizes))
        raw = bytes(buf)[:total]
        out, off = [], 0
        for i in range(count):
            out.append(raw[off:off + sizes[i]])
            off += sizes[i]
        return out

    def export_tile_set_raw(self, tiles) -> tuple[bytes, list[int]]:
        """Streams of the listed tiles (any order, repeats allowed),
        concatenated in list order, and their sizes."""
        count = len(tiles)
        if count == 0:
            return b"", []
        lst = np.ascontiguousarray(np.asarray(tiles, dtype=np.uint64))
        u64p = C.POINTER(C.c_ulonglong)
        sizes = np.zeros(count, dtype=np.uint64)
        self._check(self._L.qsim_export_tile_set(self.h, lst.ctypes.data_as(u64p), count, None, 0,
                                                 sizes.ctypes.data_as(u64p)))
        total = int(sizes.sum())
        buf = np.zeros(max(1, total), dtype=np.uint8)
        self._check(self._L.qsim_export_tile_set(self.h, lst.ctypes.data_as(u64p), count,
                                                 buf.ctypes.data_as(C.c_void_p), total,
                                                 sizes.ctypes.data_as(u64p)))
        return buf[:total].tobytes(), [int(v) for v in sizes]

    def export_tile_set(self, tiles) -> list[bytes]:
        """Streams of the listed tiles (any order, repeats allowed)."""
        raw, sizes = self.export_tile_set_raw(tiles)
        out, off = [], 0
        for sz in sizes:
            out.append(raw[off:off + sz])
            off += sz
        return out

    def import_tiles(self, first: int, streams):
        data = b"".join(streams)
        sizes = (C.c_ulonglong * max(1, len(streams)))(*[len(s) for s in streams])
        buf = (C.c_uint8 * max(1, len(data))).from_buffer_copy(data) if data else (C.c_uint8 * 1)()
        self._check(self._L.qsim_import_tiles(self.h, first, len(streams), buf, sizes))


def gate_rec(g: inputs.Gate) -> GateRec:
    r = GateRec()
    r.n_targets = len(g.targets)
    for i, t in enumerate(g.targets):
        r.targets[i] = t
    r.control_mask, r.control_values = g.masks()
    m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
    for i, v in enumerate(m):
        r.matrix[2 * i] = v.real
        r.matrix[2 * i + 1] = v.imag
    return r


class Server:
    """Continuous-batching serving loop (qsim_server_*)."""

    def __init__(self, mem_budget_bytes: int, max_resident: int = 64, sweeps_per_tick: int = 4,
                 use_graph: bool = False):
        self._L = load()
        h = C.c_void_p()
        st = self._L.qsim_server_create(C.byref(h), mem_budget_bytes, max_resident, sweeps_per_tick,
                                        int(bool(use_graph)))
        if st != 0:
            raise QsimError(st, "qsim_server_create failed")
        self.h = h
        self.readout = {}

    def submit(self, n: int, gates, block_log2: int = 8, codec: str = "rel", eps: float = 1e-4,
               basis: int = 0, readout=(), theta: float = 0.0, schedule=None) -> int:
        arr = (GateRec * max(1, len(gates)))(*[gate_rec(g) for g in gates])
        req = Request()
        req.n_qubits, req.block_log2, req.codec = n, block_log2, CODECS[codec]
        req.n_readout = len(readout)
        req.rel_err_bound, req.theta, req.basis = eps, theta, basis
        req.gates, req.n_gates = arr, len(gates)
        for i, q in enumerate(readout):
            req.readout[i] = q
        if schedule:
            req.tile_log2, req.hmax, req.depth = schedule[:3]
            if len(schedule) > 3:
                req.sweep_threads = schedule[3]
        t = C.c_ulonglong()
        st = self._L.qsim_server_submit(self.h, C.byref(req), C.byref(t))
        if st != 0:
            raise QsimError(st, "qsim_server_submit failed")
        self.readout[t.value] = len(readout)
        return t.value

    def result(self, ticket: int):
        info = TicketInfo()
        probs = np.zeros(1 << self.readout[ticket])
        st = self._L.qsim_server_result(self.h, ticket, C.byref(info), probs.ctypes.data_as(C.POINTER(C.c_double)))
        if st != 0:
            raise QsimError(st, "qsim_server_result failed")
        d = {f: getattr(info, f) for f, _ in TicketInfo._fields_}
        return d, probs

    def wait(self, ticket: int, timeout: float = 600.0):
        st = self._L.qsim_server_wait(self.h, ticket, timeout)
        if st != 0:
            raise QsimError(st, "qsim_server_wait timed out")

    def drain(self, timeout: float = 3600.0):
        st = self._L.qsim_server_drain(self.h, timeout)
        if st != 0:
            raise QsimError(st, "qsim_server_drain timed out")

    def stats(self) -> dict:
        s = ServerStats()
        self._L.qsim_server_stats(self.h, C.byref(s))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            self._L.qsim_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
