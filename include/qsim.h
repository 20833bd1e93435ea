/*
 * qsim.h -- C ABI of the GB300 compressed full-amplitude simulator.
 *
 * The library simulates an n-qubit state vector of FP64 complex amplitudes
 * (Sec. II of "Amplitude-Aware Lossy Compression for Quantum Circuit
 * Simulation": 2^n amplitudes, 16 bytes each) stored in GPU memory as
 * independently compressed tiles (the paper's strides, Sec. III).  Gates are
 * queued on the host and applied by sweeps: each sweep decompresses a tile
 * group on chip, normalises it, applies a run of gates and compresses it
 * again (Algorithm 2), all in one CUDA kernel.
 *
 * Conventions
 *   - Qubit j is bit j of the amplitude index (little-endian).
 *   - Matrices are row-major 2^k x 2^k complex, (re, im) interleaved;
 *     row/column sub-index bit i selects the value of targets[i].
 *   - Every pointer argument is caller-owned; the library copies what it
 *     keeps.  Host pointers are plain host memory unless noted.
 *   - Calls are host-synchronous: a call that returns QSIM_OK has finished
 *     its GPU work, except qsim_apply_gate, which only queues.
 *   - Errors: every call returns a qsim_status; qsim_last_error gives the
 *     message of the handle's last failing call.  After a device-side
 *     error other than arena growth the handle is marked invalid and only
 *     qsim_destroy, qsim_last_error and qsim_stats remain usable.
 *   - Not thread-safe per handle; distinct handles may be used from
 *     distinct threads (batched flushes of distinct handle sets are
 *     serialised internally).
 *
 * Tile stream format (identical in the CPU oracle, written independently):
 *   A tile holds 2^c amplitudes; its re and im components each form a
 *   stream of N = 2^c doubles cut into G = max(1, N/32) groups of
 *   L = min(N, 32) values.  Header (32 bytes, little-endian):
 *     [0] mode 0 CONST / 1 PACKED / 2 RAW   [1] shift s (0..52, 0 for RAW)
 *     [2] ladder level                       [3] sign modes (re bits 0-2,
 *                                                im 3-5; 0 for RAW)
 *     [4..7] body bytes (multiple of 16)     [8..15] anchor of re
 *     [16..23] anchor of im                  [24] c
 *     [25] zero modes (re bits 0-2, im 3-5; PACKED only, else 0)
 *     [26..31] zero
 *   Codes: B = magnitude bits of x, q = (B + 2^(s-1)) >> s (q = B at s = 0);
 *   reconstruction (q << s) with the sign bit.  q = 0 only for x = +-0
 *   (other values below the lossy range force s = 0); at s > 0 a zero's
 *   sign is stored as 0.  Anchor = first nonzero code (0 if none).
 *   Residuals run along the nonzero codes: r = q - previous nonzero code
 *   (the anchor for the first) mod 2^64, zigzag z, group width = bit
 *   length of the OR of the z of its nonzero values.
 *   Word sections (sign words; zero words, bit l set when value l is a
 *   zero), modes: 0 all words 0, 1 all words all-set, 2 / 3 exceptions to
 *   0 / to all-set (ceil(G/32) u32 bitmap words, bit g set when word g
 *   differs, then the differing words in group order), 4 one u32 word per
 *   group.  The encoder takes 0 or 1 when it applies, else the shortest of
 *   2, 3, 4, the lower on a tie.
 *   PACKED body: re signs, im signs, re zeros, im zeros, G width bytes
 *   (re), G (im), zero pad to 4, then per component and group
 *   ceil(nz*w/32) u32 words (nz nonzero values) with the k-th nonzero value
 *   at bits [k*w, (k+1)*w); zero pad to 16.  RAW body: 2N doubles.
 *   CONST when every z is 0 and every sign and zero mode is 0 or 1; else
 *   PACKED when shorter than RAW; else RAW.  The relative error of a
 *   component is below 2^(s-53) (Sec. III error bound, made point-wise
 *   relative as in the paper's ref. [xin2018]).
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsim_state *qsim_t;

typedef enum {
    QSIM_OK = 0,
    QSIM_ERR_ARG = 1,            /* invalid argument (nothing done) */
    QSIM_ERR_OOM = 2,            /* device or host allocation failed */
    QSIM_ERR_CUDA = 3,           /* CUDA runtime error (no GPU, launch failure) */
    QSIM_ERR_NONFINITE = 4,      /* a gate produced NaN/Inf; state invalid */
    QSIM_ERR_TIMEOUT = 5,        /* a host-side wait of the serving loop ran out (no call waits on the device) */
    QSIM_ERR_STATE_INVALID = 6,  /* handle unusable after an earlier error */
    QSIM_ERR_FORMAT = 7          /* malformed tile stream (import) */
} qsim_status;

typedef enum {
    QSIM_CODEC_NONE = 0,      /* uncompressed FP64 vector (Algorithm 1 without codec) */
    QSIM_CODEC_LOSSLESS = 1,  /* lossless level only (shift 0) */
    QSIM_CODEC_REL = 2,       /* fixed point-wise relative bound (Sec. III) */
    QSIM_CODEC_AALC = 3       /* error-bound ladder with ratio threshold (Algorithm 2) */
} qsim_codec;

/*
 * qsim_create -- new state |0...0> of n_qubits (1..40), stored in tiles of
 * 2^min(block_log2, n_qubits, 8) amplitudes (Sec. III strides; block_log2
 * >= 1; qsim_set_schedule changes the tile size, up to 2^10).  codec as
 * above; rel_err_bound is the point-wise relative bound eps of REL, and
 * the largest ladder bound of AALC (default ladder
 * {lossless, 1e-5, 1e-4, 1e-3, 1e-2} cut at eps, theta = 16; see
 * qsim_set_aalc).  REL and AALC normalise before every sweep (Algorithm 2);
 * NONE and LOSSLESS do not (Algorithm 1).  *out receives the handle.
 * Errors: ARG (ranges), CUDA (no device), OOM.
 */
qsim_status qsim_create(qsim_t *out, int n_qubits, int block_log2, qsim_codec codec,
                        double rel_err_bound);

/* qsim_destroy -- release the handle and its device memory (NULL is OK). */
qsim_status qsim_destroy(qsim_t h);

/*
 * qsim_set_stream -- run the handle's work on cuda_stream (a cudaStream_t,
 * e.g. a PyTorch stream); NULL selects the handle's own stream.  The stream
 * must outlive its use by the handle.
 */
qsim_status qsim_set_stream(qsim_t h, void *cuda_stream);

/*
 * qsim_set_aalc -- AALC ladder (Algorithm 2): levels delta_0 = lossless,
 * then eps_levels[0..n_levels-1] ascending (each > 0, n_levels <= 7), and
 * the ratio threshold theta (> 0).  A tile is stored at the first level
 * whose ratio 16*2^c / stream bytes is >= theta, else at the last level.
 * Only for QSIM_CODEC_AALC handles; flushes queued gates first.
 */
qsim_status qsim_set_aalc(qsim_t h, double theta, const double *eps_levels, int n_levels);

/*
 * qsim_set_aalc_unit -- how many amplitudes one ladder decision covers:
 * unit_log2 = 0 (the default) decides per tile as above; unit_log2 = the
 * handle's block_log2 decides once per stride as Algorithm 2 does: every
 * tile of a stride of 2^u amplitudes, u = min(max(unit_log2, tile_log2),
 * n), is stored at the stride's first level whose ratio
 * 16*2^u / (the stride's stream bytes) is >= theta, else at the last.
 * A sweep then computes and re-encodes every item (no tile is kept or
 * moved as a stream) in two passes: one that sizes every tile at every
 * level, one that encodes.  Has an effect only with a ladder of two or
 * more levels and strides larger than a tile; the current state keeps its
 * streams until the next encode (reset, set_amplitudes or sweep).  Such
 * handles are flushed by qsim_flush only (qsim_flush_batch returns
 * QSIM_ERR_ARG).  Flushes queued gates first.  Errors: QSIM_ERR_ARG
 * (unit_log2 outside 0..40).
 */
qsim_status qsim_set_aalc_unit(qsim_t h, int unit_log2);

/*
 * qsim_set_fusion -- diag_runs = 1 (the default): within a sweep, every run
 * of two or more consecutive diagonal gates is applied as one diagonal
 * operator (the product of diagonal matrices is diagonal, Sec. II): at
 * index x the gates whose controls hold contribute their entry at x's
 * target sub-index; entries exactly 1 contribute nothing; entries -1, i
 * and -i are collected exactly as i^k; the other entries are multiplied in
 * gate order, u applied to the running product p as u*p (general complex
 * product), into T (gates whose targets and controls are all qubits
 * >= tile_log2) and L (the others); the amplitude a becomes
 * i^k * ((T*L) a), with T*L replaced by whichever exists when only one
 * does.  Each amplitude is multiplied at most twice per run however long
 * the run is.  diag_runs = 0 applies every gate on its own (Algorithm 1
 * and 2 gate by gate; lossless sweeps then equal the dense FP64 simulation
 * bit for bit).  Flushes queued gates first.
 */
qsim_status qsim_set_fusion(qsim_t h, int diag_runs);

/*
 * qsim_set_normalize -- switch Algorithm 2's normalize step (on = 1) for
 * REL/AALC handles.  Flushes first.
 */
qsim_status qsim_set_normalize(qsim_t h, int on);

/*
 * qsim_set_schedule -- tile_log2 c (1..10, <= n), pair slots hmax (1..4,
 * c + hmax <= 12; default 4) and sweep depth (max gates per sweep, 1..512;
 * default 512).  Re-tiles the current state: a basis state set by
 * qsim_create or qsim_reset_basis (no gates applied since) is encoded
 * afresh in the new tiles, any n; any other state is decoded into a dense
 * device buffer of 2^(n+4) bytes and re-encoded (exact only for
 * RAW/lossless tiles; n <= 32), so call it before the first gate.  Used
 * by the autotuner.  Errors: ARG (ranges), OOM, CUDA.
 */
qsim_status qsim_set_schedule(qsim_t h, int tile_log2, int hmax, int depth);

/*
 * qsim_set_polar -- on = 1: every lossy level of a REL or AALC handle also
 * codes each tile in the POLAR mode and keeps the shorter stream (a codec
 * variant; the level decision of AALC then uses that size).  POLAR stream
 * (mode byte 3 or 4): each nonzero amplitude a = x + iy as its magnitude
 * m = sqrt(fma(x, x, y*y)) quantised like a component with shift s - 1,
 * and its angle from an integer CORDIC (30 steps of
 * round(2^64 atan(2^-k) / (2 pi)), units of 2^-64 turn) quantised with
 * shift P = s + 8 to B = 56 - s bits; reconstruction: the CORDIC rotation
 * (X, Y) of (2^59, 0) by the angle code, a^ = (m^ Xd r, m^ Yd r) with
 * r = 1 / sqrt(Xd^2 + Yd^2).  Magnitude codes: order-1 residuals from the
 * anchor (header 8..15).  Angle codes, mode 3: order-2 residuals modulo
 * 2^B from u0 (header 16..23) and the first difference d1 (header 26..31,
 * 48 bits), the first two nonzero amplitudes taking residual 0.  Mode 4
 * (tiles without zero amplitudes): the angle hp(i) of amplitude i rounded
 * to B + 8 bits is predicted as hp(0) (header 16..23) plus the basis
 * differences D_b = hp(2^b) - hp(0) mod 2^(B+8) of the set bits b of i,
 * rounded to B bits; residual = code - prediction mod 2^B; the c values
 * D_b follow the width bytes, packed at B + 8 bits each in u32 words
 * (header 26..31 zero).  The encoder takes the shorter of modes 3 and 4
 * (3 on a tie).  Body as PACKED with clear sign sections and equal zero
 * sections.  A tile takes the mode only for 8 <= s <= 52, every component
 * 0 or in [2^-400, 16), and every amplitude within
 * |a^ - a|^2 <= 2^(2(s-53)) (1 - 2^-10) |a|^2: the level's bound on the
 * complex amplitude, not on each component.  Phases linear in the index,
 * or sums of one phase per index bit (the QFT's tiles), cost almost
 * nothing.  Saved in checkpoints.  Flushes queued gates first.  Errors:
 * ARG (codec NONE or LOSSLESS).
 */
qsim_status qsim_set_polar(qsim_t h, int on);

/*
 * qsim_set_sweep_threads -- CTA size of the sweep kernel: 128, 256 (the
 * default) or 512 threads, compiled for 3, 3 and 1 resident CTAs per SM
 * (the register budget of each launch shape).  Results do not depend on it;
 * the autotuner times the shapes.  qsim_flush_batch launches with the
 * first handle's shape.  Flushes queued gates first.  Errors: ARG (other
 * sizes).
 */
qsim_status qsim_set_sweep_threads(qsim_t h, int threads);

/* Place the state's two stream arenas in a caller-owned device buffer (for
 * example the storage of a torch tensor) instead of library allocations
 * (Sec. III: the strides are stored compressed; this chooses where).
 *   dev_ptr: device memory of the handle's GPU, 256-byte aligned; bytes:
 *   its size.  The buffer is split into two arenas of floor(bytes/2)
 *   rounded down to 256 bytes; queued gates are flushed first and the
 *   current stream is copied in.  The caller keeps ownership: the buffer
 *   must stay allocated until qsim_destroy or the next qsim_set_pool, and
 *   the library never frees it.  Arenas in a pool do not grow: a flush
 *   whose output does not fit returns QSIM_ERR_OOM and leaves the handle
 *   STATE_INVALID.  dev_ptr = NULL with bytes = 0 moves the state back to
 *   library-owned arenas.  Tile tables, norm partials and counters stay
 *   library-allocated (24 bytes per tile plus a few KiB).
 *   Errors: QSIM_ERR_ARG (misaligned, not device memory of this GPU, a
 *   half smaller than the current stream or than 4 KiB, NULL with
 *   bytes != 0), QSIM_ERR_CUDA. */
qsim_status qsim_set_pool(qsim_t h, void *dev_ptr, size_t bytes);

/* qsim_reset_basis -- state |x> (x < 2^n); drops queued gates. */
qsim_status qsim_reset_basis(qsim_t h, unsigned long long x);

/*
 * qsim_set_amplitudes -- replace the state by amps (host, 2^n complex128,
 * interleaved), encoded with the handle's codec.  Drops queued gates.
 */
qsim_status qsim_set_amplitudes(qsim_t h, const double *amps);

/*
 * qsim_apply_gate -- queue U (Sec. II: single-qubit gate, controlled gate;
 * generalised to 1-2 targets and any number of controls).  matrix is
 * 2^n_targets x 2^n_targets complex (copied).  controls[i] must hold value
 * bit i of control_values (pass ~0ULL for "all ones").  Validated on the
 * host: qubits in range and distinct, entries finite, unitary within 1e-12.
 * Errors: ARG.
 */
qsim_status qsim_apply_gate(qsim_t h, const double *matrix, const int *targets, int n_targets,
                            const int *controls, int n_controls,
                            unsigned long long control_values);

/* qsim_flush -- run every queued gate (sweeps) and wait for the device. */
qsim_status qsim_flush(qsim_t h);

/*
 * qsim_flush_batch -- flush several handles together: round r runs the r-th
 * pending sweep of every handle that has one, all rounds as one persistent
 * launch each (plus one small finalize launch) on the first handle's stream,
 * optionally captured into a CUDA graph (use_graph = 1).  Each handle's
 * result is byte-identical to its own qsim_flush.  Handles that decide
 * per stride (qsim_set_aalc_unit) are refused with QSIM_ERR_ARG.  A handle
 * whose output arena overflows is grown and finished alone afterwards.
 * The handles must be distinct and on one device.  Returns the first
 * handle error (each handle keeps its own qsim_last_error).
 */
qsim_status qsim_flush_batch(qsim_t *handles, int count, int use_graph);

/*
 * qsim_probabilities -- flush, then out[j] (host, 2^nq doubles) = total
 * probability of the outcomes whose bits on qubits[0..nq-1] spell j (bit i
 * of j <-> qubits[i]), computed as RN(S_j) / RN(S) where S_j and S are the
 * exact sums of |a|^2 over the stored amplitudes (units of 2^-112, each
 * rounded once to double).  nq in 0..24, qubits distinct.
 */
qsim_status qsim_probabilities(qsim_t h, const int *qubits, int nq, double *out);

/*
 * qsim_amplitudes -- flush, then out (host, 2*count doubles, interleaved)
 * = stored amplitudes start .. start+count-1 (the decompressed state; the
 * pending normalisation scale is not applied).
 */
qsim_status qsim_amplitudes(qsim_t h, unsigned long long start, unsigned long long count,
                            double *out);

/* Reference state for qsim_fidelity. */
typedef enum {
    QSIM_REF_HANDLE = 0,       /* another handle with the same n and tile size */
    QSIM_REF_QFT_BASIS = 1,    /* QFT|x>: e^{2 pi i x k / 2^n} / sqrt(2^n) */
    QSIM_REF_GROVER = 2,       /* Grover after `iterations` from |0..0>, marked item */
    QSIM_REF_DENSE_HOST = 3,   /* host array of 2^n complex128 */
    QSIM_REF_DENSE_DEVICE = 4  /* device array of 2^n complex128 */
} qsim_ref_kind;

typedef struct {
    int kind;                  /* qsim_ref_kind */
    qsim_t other;              /* QSIM_REF_HANDLE */
    unsigned long long x;      /* QFT basis index, or Grover marked item */
    int iterations;            /* Grover iterations */
    const double *dense;       /* QSIM_REF_DENSE_* */
} qsim_ref;

/*
 * qsim_fidelity -- flush, then the pure-state fidelity of Sec. II between
 * the stored state psi and ref, both normalised:
 * *F = |<ref|psi>|^2 / (<ref|ref><psi|psi>) and *overlap_abs = sqrt(*F)
 * (the paper writes F = <psi_rho|psi_sigma>; the modulus squared is the
 * reading used here).  Either output may be NULL.
 */
qsim_status qsim_fidelity(qsim_t h, const qsim_ref *ref, double *F, double *overlap_abs);

/*
 * qsim_compressed_bytes -- flush, then *stream_bytes = sum of tile stream
 * sizes (headers included) and *footprint_bytes = device bytes held by the
 * state (both arenas, tile table, norm partials).  Either may be NULL.
 */
qsim_status qsim_compressed_bytes(qsim_t h, unsigned long long *stream_bytes,
                                  unsigned long long *footprint_bytes);

/* Counters since creation (or the last reset). */
typedef struct {
    unsigned long long gates;          /* gates applied */
    unsigned long long sweeps;         /* sweeps run */
    unsigned long long items_done;     /* tile groups decoded and re-encoded */
    unsigned long long items_skipped;  /* tile groups carried over unchanged */
    unsigned long long level_hist[8];  /* tiles written per ladder level */
    unsigned long long stream_bytes;   /* current sum of stream sizes */
    unsigned long long min_stream_bytes_seen; /* smallest total after a sweep */
    unsigned long long max_stream_bytes_seen; /* largest total after a sweep */
    unsigned long long arena_regrows;  /* sweeps re-run after growing the arena */
    unsigned long long kernel_launches; /* kernels launched by the handle */
    double alpha;                      /* scale of the next normalize step */
    int tile_log2, hmax, depth, n_qubits;
    unsigned long long h2d_bytes;      /* bytes the handle's calls copied host -> device since creation */
    unsigned long long d2h_bytes;      /* bytes the handle's calls copied device -> host since creation */
    unsigned long long tiles_over_limit; /* tiles written larger than the AALC size limit (no level met theta) */
} qsim_stats_t;

qsim_status qsim_stats(qsim_t h, qsim_stats_t *out);

/*
 * Profile of the sweep kernels (Algorithm 2 passes) since profiling was
 * switched on.  Device times come from CUDA events recorded on the
 * handle's stream around each sweep's launches (with per-stride ladder
 * decisions: the sizing pass, the level pass and the encoding pass).
 * Every flush and sweep is also an NVTX range ("qsim_flush", "qsim sweep
 * <id> (<gates> gates)", "qsim_flush_batch") for profilers.  dp_ops counts
 * the FP64 instructions of the canonical gate arithmetic (per matrix entry: first
 * term real/imaginary 1 per component, general 2; later terms 1 or 2;
 * entries 0 and leading +-1 free) plus 2 per amplitude for normalize;
 * bytes counts compressed stream bytes read and written plus 32 bytes per
 * tile of table and norm traffic.
 */
typedef struct {
    unsigned long long sweep_launches;
    double sweep_ms;
    double dp_ops;
    double bytes;
    unsigned long long kernel_launches;   /* every kernel the handle launched */
} qsim_profile_t;

/* qsim_set_profiling -- on = 1 starts recording (and zeroes the counters),
 * 0 stops.  Recording adds two event records per sweep. */
qsim_status qsim_set_profiling(qsim_t h, int on);

/* qsim_profile -- copy the counters (flushes first). */
qsim_status qsim_profile(qsim_t h, qsim_profile_t *out);

/* Message of the handle's last failing call ("" if none); h NULL: the
 * calling thread's last failing call that had no usable handle. */
const char *qsim_last_error(qsim_t h);

/*
 * qsim_export_tiles -- flush, then copy the streams of tiles
 * first .. first+count-1, concatenated in tile order, into out (host, cap
 * bytes) and their sizes into sizes (host, count entries).  With out NULL
 * only the sizes are written.  Errors: ARG when cap is too small.
 */
qsim_status qsim_export_tiles(qsim_t h, unsigned long long first, unsigned long long count,
                              void *out, unsigned long long cap, unsigned long long *sizes);

/*
 * qsim_export_tile_set -- as qsim_export_tiles for an arbitrary set of
 * tiles: tiles (host, count entries, each < 2^(n - tile_log2), repeats
 * allowed) lists them; their streams are concatenated in list order into
 * out (host, cap bytes) and their sizes written to sizes (host, count
 * entries).  With out NULL only the sizes are written.  Used to read the
 * tile groups of sampled items of large states.  Errors: ARG (null
 * arguments, a tile out of range, cap too small).
 */
qsim_status qsim_export_tile_set(qsim_t h, const unsigned long long *tiles, unsigned long long count,
                                 void *out, unsigned long long cap, unsigned long long *sizes);

/*
 * qsim_import_tiles -- flush, then replace tiles first .. first+count-1 by
 * the concatenated streams in data (host) with the given sizes.  Every
 * stream is first decoded on the device; if any fails, FORMAT is returned
 * and the state is unchanged.  The normalisation scale is recomputed.
 */
qsim_status qsim_import_tiles(qsim_t h, unsigned long long first, unsigned long long count,
                              const void *data, const unsigned long long *sizes);

/*
 * qsim_plan_sweeps -- host-only: the sweep partition the library uses for
 * a gate list (no GPU needed).  Gate g has ntargets[g] targets in
 * targets[2g..], matrix in matrices[32g..] (row-major complex, zero-padded).
 * Writes per sweep its first gate to out_lo, its pair count to out_h and
 * its pair qubits to out_H[4s..] (ascending; unused slots 0).  Returns the
 * number of sweeps, or -1 on bad arguments, or -2 when cap is too small.
 */
int qsim_plan_sweeps(int n, int tile_log2, int hmax, int depth, int ngates,
                     const int *ntargets, const int *targets, const double *matrices,
                     int *out_lo, int *out_h, int *out_H, int cap);

/*
 * qsim_encode_noalloc -- encode a dense state that already sits in device
 * memory into tile streams, allocating nothing.  The paper has no
 * counterpart: this entry point exists for callers that are not allowed to
 * allocate device memory, such as code that runs under an application
 * allocator owning all of the GPU's memory, a callback invoked from inside
 * such an allocator, or a latency-critical path that must not pay for the
 * device-wide synchronisation an allocation implies.
 *
 * dev_amps: device, 2^n_qubits complex128 (interleaved), 16-byte aligned.
 * Tiles of 2^tile_log2 amplitudes (1..min(10, n_qubits)), coded with the
 * fixed point-wise relative bound rel_err_bound (0 = lossless) in the
 * stream format above, exactly as qsim_set_amplitudes stores them for a
 * QSIM_CODEC_REL handle.  Outputs, all caller-owned: dev_out (device,
 * out_cap bytes, 16-byte aligned) receives the streams in no particular
 * order, dev_table (device, one entry per tile) the byte offset of each
 * tile's stream in dev_out, *stream_bytes (host) the bytes used.  The
 * call runs on cuda_stream (NULL = legacy default stream) and returns
 * after the work has finished.
 *
 * Scratch: one static device array, at most 4096 tiles
 * (n_qubits - tile_log2 <= 12), held by every GPU that loads the library
 * until the process exits.  Larger states are rejected with ERR_ARG.
 * The first call on a device looks up the array's device address (and sets
 * kernel attributes), once per device even when several host threads make
 * their first call at the same time; make that first call before any
 * stream capture.  cuda_stream must belong to the current device (ERR_ARG
 * otherwise), since the scratch address is the current device's.  All
 * calls share the array and it keeps the last call's contents; each call
 * clears what must start at zero.  Calls that overlap on the GPU (several
 * streams or threads at once) race on the array and must be serialised by
 * the caller.  Errors: ARG (ranges, alignment, out_cap too small: then
 * *stream_bytes holds the size needed), NONFINITE, CUDA; the message is in
 * qsim_last_error(NULL).
 */
qsim_status qsim_encode_noalloc(const double *dev_amps, int n_qubits, int tile_log2,
                                double rel_err_bound, void *dev_out, unsigned long long out_cap,
                                unsigned long long *dev_table, unsigned long long *stream_bytes,
                                void *cuda_stream);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of many circuits on one GPU            */
/* ------------------------------------------------------------------ */

/* One gate of a request, fixed size; controls as masks over qubit bits. */
typedef struct {
    int n_targets;                      /* 1 or 2 */
    int targets[2];
    int pad;
    unsigned long long control_mask;    /* bit q set: qubit q is a control */
    unsigned long long control_values;  /* bit q: required value of control q */
    double matrix[32];                  /* 2^k x 2^k complex, row-major, (re, im) */
} qsim_gate_rec;

/* One circuit to run: state |basis> of n_qubits, the gates in order, and
 * the qubits whose outcome probabilities are read out at the end. */
typedef struct {
    int n_qubits;
    int block_log2;
    int codec;                          /* qsim_codec */
    int n_readout;                      /* 0..16 */
    double rel_err_bound;
    double theta;                       /* AALC threshold; 0 keeps the default ladder */
    unsigned long long basis;
    const qsim_gate_rec *gates;         /* copied by qsim_server_submit */
    int n_gates;
    int readout[16];
    int tile_log2, hmax, depth;         /* schedule (qsim_set_schedule); 0 = default */
    int sweep_threads;                  /* qsim_set_sweep_threads; 0 = default (a batch launches
                                           with its first circuit's shape) */
} qsim_request;

typedef struct {
    int done;                           /* 1 once finished (or failed) */
    int status;                         /* QSIM_OK or the failing code */
    double submit_s, admit_s, finish_s; /* seconds since the server started */
    unsigned long long stream_bytes;    /* final compressed size */
    unsigned long long peak_footprint;  /* device bytes the circuit held at its peak */
} qsim_ticket_info;

typedef struct {
    unsigned long long submitted, completed, failed, ticks;
    unsigned long long peak_footprint;  /* device bytes of resident circuits, peak */
    unsigned long long budget;
    double busy_s;                      /* time spent in ticks */
    double p50_latency_s, p99_latency_s, mean_latency_s;
    double throughput_cps;              /* completed circuits / (last finish - first submit) */
    int max_resident_seen;
} qsim_server_stats_t;

typedef struct qsim_server *qsim_server_t;

/*
 * qsim_server_create -- start a serving loop on the current device (one
 * host thread and one CUDA stream of its own).  A waiting circuit is
 * admitted while the reservations of the resident circuits plus the
 * newcomer's stay within mem_budget_bytes and fewer than max_resident
 * circuits run; a circuit alone is always admitted.  A circuit's
 * reservation is the larger of its measured device footprint (before
 * admission: its initial footprint) and its growth bound: 32 bytes per
 * tile plus two arenas of the codec's stream bound, which is, per tile,
 * floor(16 * 2^c / theta) for AALC with theta > 0 (the ratio threshold),
 * the largest PACKED stream at the codec's shift s for REL (widths of at
 * most 65 - s bits), and the RAW size otherwise (tiles that the ladder
 * cannot bring under theta, or that hold values outside the lossy range,
 * may exceed it; the measured footprint then counts).  Each tick applies
 * the next sweeps_per_tick
 * sweeps of every resident circuit (cut at the circuit's own sweep
 * boundaries, qsim_plan_sweeps) as one batched flush
 * (qsim_flush_batch, CUDA-graph captured when use_graph), so newcomers join
 * at the next tick.  Results are identical to running each circuit alone.
 */
qsim_status qsim_server_create(qsim_server_t *out, unsigned long long mem_budget_bytes, int max_resident,
                               int sweeps_per_tick, int use_graph);

/* qsim_server_submit -- queue a circuit (copied); *ticket identifies it. */
qsim_status qsim_server_submit(qsim_server_t s, const qsim_request *req, unsigned long long *ticket);

/* qsim_server_result -- status of a ticket; once done, probs (host,
 * 2^n_readout doubles, may be NULL) receives the read-out probabilities. */
qsim_status qsim_server_result(qsim_server_t s, unsigned long long ticket, qsim_ticket_info *info,
                               double *probs);

/* qsim_server_wait / qsim_server_drain -- block until the ticket / every
 * submitted circuit is done, or timeout_s passes (QSIM_ERR_TIMEOUT). */
qsim_status qsim_server_wait(qsim_server_t s, unsigned long long ticket, double timeout_s);
qsim_status qsim_server_drain(qsim_server_t s, double timeout_s);

/* qsim_server_stats -- counters, p50/p99 latency, throughput. */
qsim_status qsim_server_stats(qsim_server_t s, qsim_server_stats_t *out);

/* qsim_server_destroy -- finish the queued circuits, stop, release all. */
qsim_status qsim_server_destroy(qsim_server_t s);

/* Checkpoint / resume (the state saved before a job's wall time runs out
 * and reloaded later).  qsim_save flushes the queued gates and writes
 *   a 120-byte little-endian header: "QSIMCKP1", u32 version (2), n, c,
 *   hmax, depth, codec, normalize, nlev, i32 shifts[8], f64 eps, theta,
 *   u64 max_bytes, ntiles, stream bytes, i32 unit_log2, i32 flags (bit 0 the
 *   POLAR mode, bit 1 gate by gate, see qsim_set_fusion; other bits 0);
 *   then, per chunk of up to 2^20 tiles in tile order, the u64 stream
 *   sizes of the chunk followed by its streams (the tile stream format
 *   above, so a host program can decode the file tile by tile).
 * qsim_load creates a handle from such a file on the current device: the
 * streams are validated and placed as by qsim_import_tiles, and the norm
 * and normalize scale are recomputed from them, so continuing a circuit
 * after save and load gives the same streams as continuing it without.
 * Counters start from zero.  The caller owns the returned handle.
 * Errors: QSIM_ERR_ARG (null argument, file not openable or not
 * writable), QSIM_ERR_FORMAT (not a checkpoint, inconsistent header,
 * truncated, a stream that does not decode), QSIM_ERR_OOM, QSIM_ERR_CUDA. */
qsim_status qsim_save(qsim_t h, const char *path);
qsim_status qsim_load(qsim_t *out, const char *path);

/* qsim_version -- library version string. */
const char *qsim_version(void);

/* qsim_fp64_rate -- measured FP64 fused multiply-add rate of GPU `device`
 * (FMA per second): independent DFMA chains over every SM, timed with CUDA
 * events after a warm-up launch (about 20 ms).  The denominator the
 * benchmark reports beside the nominal FP64 peak for the gate arithmetic,
 * which is FP64-bound on this part.  Errors: QSIM_ERR_ARG (null out),
 * QSIM_ERR_CUDA. */
qsim_status qsim_fp64_rate(int device, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
