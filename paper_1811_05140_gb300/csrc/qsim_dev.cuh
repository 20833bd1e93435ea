// Internal types shared by the device kernels and the host API of the
// compressed simulator (not part of the public C ABI).
#pragma once
#include <cstdint>
#include <vector_types.h>

namespace qs {

constexpr int THREADS = 256;            // CTA size of the helper kernels
constexpr int SWEEP_THREADS = 256;      // default CTA size of the sweep kernel (128, 256 or 512)
constexpr int MAX_C = 10;               // tile_log2 limit: G = 2^c/32 <= 32 groups
constexpr int MAX_ITEM_LOG2 = 12;       // c + pair count: 4096 amplitudes on chip
constexpr int MAX_PAIRS = 4;            // paired high qubits per sweep
constexpr int HDR = 32;                 // tile header bytes
constexpr int MAX_LEVELS = 8;

// sticky device error bits
enum : unsigned int {
    ERR_OVERFLOW = 1u,    // output arena too small: the host grows it and re-runs
    ERR_FORMAT = 2u,      // malformed tile stream
    ERR_NONFINITE = 4u,   // NaN/Inf amplitude
    ERR_RANGE = 8u        // |amplitude| >= 16: outside the norm's fixed point
};

// Device-resident counters and the normalisation scale of a state.
struct DevScalars {
    unsigned long long bump;        // bytes allocated in the output arena
    unsigned int err;               // sticky error bits
    unsigned int err_sweep;         // sweep id of the first error (+1; 0 = none)
    double alpha;                   // scale applied by the next sweep's normalize
    unsigned long long acc_lo, acc_hi;    // running sum of |a|^2 (units 2^-112)
    unsigned long long norm_lo, norm_hi;  // sum of the last finished pass
    unsigned long long used;        // stream bytes of the last finished pass
    unsigned long long hist[MAX_LEVELS];
    unsigned long long items_done, items_skipped;
    unsigned long long work;        // item counter of the sweep launch in flight
    unsigned long long run_dp;      // FP64 instructions executed by diagonal runs and scaled gates (running total)
    unsigned long long over_limit;  // tiles written above the ratio threshold's size (no level met it)
};

// A gate prepared for one sweep (positions are item-buffer bits).
struct DGate {
    double m[32];                   // 2^k x 2^k complex, row-major, re/im
    unsigned long long lcm, lcv;    // controls on buffer bits
    unsigned long long fcm, fcv;    // controls on fixed qubits (global bits)
    int k;                          // targets: 1 or 2
    int diag;                       // no nonzero off-diagonal entry
    int pos[2];                     // buffer bit of target i, -1 when fixed
    int t[2];                       // global qubit of target i
};

// A gate as staged in shared memory for one sweep (compact form).
struct SGate {
    double d[8];                    // diagonal gates: entry r (re, im), r < 2^k
    unsigned long long cls;         // entry classes, 3 bits each (see entry classes below)
    unsigned long long fac;         // factored rows: bit r row r; bits 8+2e factor of entry e
    unsigned long long fcm, fcv;    // controls on fixed qubits (global bits)
    uint32_t lcm, lcv;              // controls on buffer bits
    uint8_t kind;                   // 0 diagonal, 1 one-target, 2 two-target (non-diagonal)
    uint8_t k;                      // number of targets
    int8_t p0, p1;                  // buffer bit of each target, -1 when fixed
    uint8_t t0, t1;                 // global qubit of each target
    uint8_t one_mask;               // diagonal: bit r set when entry r is exactly 1
    uint8_t nins;                   // buffer bits pinned by targets and local controls
    uint8_t ins[12];                // those bits, ascending
    int16_t run;                    // >= 0: first gate of diagonal run `run`; -2 inside a run; -1 none
    uint8_t unscaled;               // scaled gate (nonzero): factored rows give their sums, d is in the
                                    // sweep's scale; the value is the FP64 instructions of one group
};

// Entry classes of a matrix entry u, decided on the host so that device
// code never compares doubles (FP64 compares occupy the FP64 pipe):
// diagonal gates use bits 3r of SGate::cls for entry (r, r); other gates
// bits 3(r*dim + c) for entry (r, c).
enum : unsigned {
    EC_ZERO = 0,       // u == 0
    EC_ONE = 1,        // u == 1 exactly
    EC_MINUS_ONE = 2,  // u == -1 exactly
    EC_REAL = 3,       // imaginary part 0
    EC_IMAG = 4,       // real part 0
    EC_GENERAL = 5
};

constexpr int MAX_SWEEP_GATES = 512;    // gates per sweep (depth limit)

// Diagonal runs: two or more consecutive diagonal gates of a sweep applied
// as one diagonal operator.  At index x the gates whose controls hold
// contribute their entry at x's target sub-index; entries exactly 1
// contribute nothing, entries -1, i, -i are collected as i^k, the other
// entries are multiplied in gate order into T (gates on qubits >= c only,
// constant over a tile) and L (the rest); a <- i^k * ((T*L) a).  An
// amplitude that is exactly zero is left as it is.

// A diagonal gate of a run, with its entries classified on the host.
struct RGate {
    double e[8];                    // entry r (re, im), r < 2^k
    unsigned long long cm, cv;      // controls over global index bits, required values
    uint8_t k, t0, t1;              // targets (global qubits)
    uint8_t code[4];                // entry r: 0 exactly 1, 1 unit, 2 general
    uint8_t uexp[4];                // unit entry r = i^uexp[r]
    uint8_t pad;
};
static_assert(sizeof(RGate) % 16 == 0, "RGate is copied to shared memory in 16-byte pieces");

constexpr int RUN_QMAX = 4;             // class bits of a tabled run (2^4 tables)

// One diagonal run of a flush.  The local product L depends on the tile
// bits (x < 2^c) and on the class bits q[] (the qubits >= c that local
// gates use); when tabled, L is read from 2^nq tables of 2^c entries.
struct DRun {
    unsigned long long table;       // first table entry of the run (tabled runs)
    int cls;                        // first class summary of the run (tabled runs)
    int tg, nt;                     // tile gates: rgates[tg .. tg+nt-1]
    int lg, nl;                     // local gates: rgates[lg .. lg+nl-1]
    int first, len;                 // the run's gates in its sweep (gate index, count)
    int nq;                         // class bits
    int tabled;
    int q[RUN_QMAX];                // class bit i = index bit q[i]
};

// Per class of a tabled run: where L or a unit factor exists.
struct RunClass {
    uint32_t active;                // entries with L or a unit power != 1
    uint32_t have;                  // entries with L (a general product)
    uint32_t pin_mask, pin_val;     // tile bits common to every active entry
};

// Table entry meta byte: bit 0 L exists, bits 1-2 unit exponent.

constexpr int GATE_CHUNK = 48;          // gates staged in shared memory at a time

// Codec configuration of a state.
struct CodecCfg {
    int c;                          // tile_log2
    int nlev;                       // ladder levels
    int shifts[MAX_LEVELS];         // quantisation shift per level
    unsigned long long max_bytes;   // ratio threshold as a stream size limit
    int force_raw;                  // uncompressed storage (QSIM_CODEC_NONE)
    int polar;                      // lossy levels also try the POLAR mode (magnitude + phase)
};

constexpr int POLAR_ITERS = 30;         // CORDIC steps of the POLAR mode

struct SweepParams {
    const uint8_t *in_arena;
    const unsigned long long *in_table;
    uint8_t *out_arena;
    unsigned long long *out_table;
    unsigned long long out_cap;
    unsigned long long *part;       // per tile: sum of |a^|^2, 2 words
    DevScalars *scal;
    const DGate *gates;             // full matrices (non-diagonal gates)
    const SGate *sgates;            // compact gates, staged in shared memory
    int ngates;
    int n, h;
    int H[MAX_PAIRS];               // paired high qubits, ascending
    CodecCfg cc;
    unsigned long long nitems;
    unsigned int sweep_id;
    int use_alpha;
    int low_free;                   // no gate of the sweep targets or controls a qubit < c
    int moves_tiles;                // low_free and every gate a permutation: tiles move whole
    int every_item;                 // compute and re-encode every item (per-stride decisions)
    int unit_shift;                 // log2 of the tiles one ladder decision covers
    unsigned long long *unit_bytes; // sizing pass: stream bytes per (stride, level); else null
    const uint8_t *unit_level;      // encode pass: ladder level of every stride; else null
    const DRun *runs;               // diagonal runs of the flush (SGate::run indexes them)
    const RGate *rgates;
    const double2 *rtab;            // run tables (value of L)
    const uint8_t *rmeta;           // run tables (meta bytes)
    const RunClass *rcls;
    int run_first, nruns;           // this sweep's runs: runs[run_first .. run_first+nruns-1]
    const double *dscale;           // product of the sweep's scaled gates' d (null: 1)
    int point_ok;                   // every gate a run member, or a scaled gate or permutation on
                                    // qubits >= c: items of point tiles take one amplitude per tile
    const int *glist;               // the gates that can apply (no later gate of a run), in order
    int nglist;
};

// End-of-pass bookkeeping of one state (norm, scale, used bytes).
struct FinalizeEntry {
    DevScalars *scal;
    unsigned long long *used_hist;   // per-sweep used bytes (may be null)
    unsigned slot;
    int use_alpha;
    int record_used;
};

// Four FP64 sums of a fidelity pass: Re<ref|psi>, Im<ref|psi>, <psi|psi>, <ref|ref>.
struct __align__(16) Acc4 {
    double x, y, z, w;
};

// Reference state of a fidelity computation.
struct RefSpec {
    int kind;                 // 0 handle, 1 QFT basis, 2 Grover, 3 dense device
    unsigned long long x;     // QFT basis index / Grover marked item
    double qft_mag;           // 1/sqrt(2^n)
    double grov_m, grov_o;    // Grover amplitudes: marked item, the others
    int n;
    const double2 *dense;
    const uint8_t *o_arena;
    const unsigned long long *o_table;
};

}  // namespace qs
