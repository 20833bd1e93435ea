// Internal types shared by the device kernels and the host API of the
// compressed simulator (not part of the public C ABI).
#pragma once
#include <cstdint>
#include <vector_types.h>

namespace qs {

constexpr int THREADS = 256;            // CTA size of every tile kernel
constexpr int NWARPS = THREADS / 32;
constexpr int MAX_C = 10;               // tile_log2 limit: G = 2^c/32 <= 32 groups
constexpr int MAX_ITEM_LOG2 = 12;       // c + pair count: 4096 amplitudes on chip
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
    unsigned long long pad[3];
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

// Codec configuration of a state.
struct CodecCfg {
    int c;                          // tile_log2
    int nlev;                       // ladder levels
    int shifts[MAX_LEVELS];         // quantisation shift per level
    unsigned long long max_bytes;   // ratio threshold as a stream size limit
    int force_raw;                  // uncompressed storage (QSIM_CODEC_NONE)
};

struct SweepParams {
    const uint8_t *in_arena;
    const unsigned long long *in_table;
    uint8_t *out_arena;
    unsigned long long *out_table;
    unsigned long long out_cap;
    unsigned long long *part;       // per tile: sum of |a^|^2, 2 words
    DevScalars *scal;
    const DGate *gates;
    int ngates;
    int n, h;
    int H[2];                       // paired high qubits, ascending
    CodecCfg cc;
    unsigned long long nitems;
    unsigned int sweep_id;
    int use_alpha;
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
