// Device code of the compressed simulator: the tile codec (decode/encode),
// the fused decompress -> normalize -> gate run -> compress sweep
// (Algorithm 2 of the paper, over tile groups), and the read-out kernels.
//
// Arithmetic contract (kept bit-identical with the CPU oracle, which is
// written separately):
//   * gate rows skip exactly-zero entries; first term a product, later
//     terms fused multiply-adds; real / imaginary / general entries as in
//     term_first / term_acc; explicit __dmul_rn/__fma_rn (no contraction);
//   * normalize multiplies each component by alpha (skipped when alpha==1);
//   * the codec is integer-only; the norm is an exact fixed-point sum.
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>

#include "qsim_dev.cuh"

namespace qs {

constexpr unsigned long long MAG = 0x7FFFFFFFFFFFFFFFull;
constexpr unsigned long long MIN_NORMAL = 0x0010000000000000ull;
constexpr unsigned long long LOSSY_LIMIT = 0x7FE0000000000000ull;
constexpr unsigned long long INF_BITS = 0x7FF0000000000000ull;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr unsigned long long SIGN_BIT = 0x8000000000000000ull;

enum { M_CONST = 0, M_PACKED = 1, M_RAW = 2, M_POLAR = 3, M_POLAR_B = 4 };
constexpr int POLAR_EXTRA = 8;          // extra angle bits of the bitwise-linear predictor
enum { S_CLEAR = 0, S_SET = 1, S_EXC_CLEAR = 2, S_EXC_SET = 3, S_WORDS = 4 };

__device__ __forceinline__ Acc4 make_acc4(double x, double y, double z, double w) {
    Acc4 a;
    a.x = x; a.y = y; a.z = z; a.w = w;
    return a;
}
__device__ __forceinline__ unsigned long long dbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double bitsd(unsigned long long u) {
    return __longlong_as_double((long long)u);
}
__device__ __forceinline__ unsigned long long quant(unsigned long long B, int s) {
    return s == 0 ? B : (B + (1ull << (s - 1))) >> s;
}
__device__ __forceinline__ unsigned long long zigzag(unsigned long long r) {
    return (r << 1) ^ (unsigned long long)((long long)r >> 63);
}
__device__ __forceinline__ unsigned long long unzigzag(unsigned long long z) {
    return (z >> 1) ^ (0ull - (z & 1ull));
}
__device__ __forceinline__ int bitlen64(unsigned long long v) { return 64 - __clzll(v); }

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    unsigned lo = __shfl_sync(FULL, (unsigned)v, src);
    unsigned hi = __shfl_sync(FULL, (unsigned)(v >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long shfl_up64(unsigned long long v, int d) {
    unsigned lo = __shfl_up_sync(FULL, (unsigned)v, d);
    unsigned hi = __shfl_up_sync(FULL, (unsigned)(v >> 32), d);
    return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long warp_or64(unsigned long long v) {
    unsigned lo = __reduce_or_sync(FULL, (unsigned)v);
    unsigned hi = __reduce_or_sync(FULL, (unsigned)(v >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// ---------------------------------------------------------------- norm
// floor(x^2 * 2^112) as (hi, lo); *range set when |x| >= 16.
__device__ __forceinline__ void sq_units(unsigned long long u, unsigned long long &lo,
                                         unsigned long long &hi, unsigned &range) {
    u &= MAG;
    unsigned long long E = u >> 52, F = u & 0xFFFFFFFFFFFFFull;
    lo = hi = 0;
    if (E >= 1027) { range = 1; return; }
    unsigned long long mant = E ? (F | (1ull << 52)) : F;
    long long Ee = E ? (long long)E : 1;
    unsigned long long pl = mant * mant, ph = __umul64hi(mant, mant);   // < 2^106
    long long sh = 2 * Ee - 2150 + 112;
    if (sh >= 0) {                       // sh <= 14
        if (sh == 0) { lo = pl; hi = ph; }
        else { hi = (ph << sh) | (pl >> (64 - sh)); lo = pl << sh; }
    } else {
        long long r = -sh;
        if (r >= 106) return;
        if (r >= 64) { lo = ph >> (r - 64); hi = 0; }
        else { lo = (pl >> r) | (r ? (ph << (64 - r)) : 0ull); hi = ph >> r; }
    }
}

// sq_units for a reconstructed value at shift s >= 21 (u = q << s): the
// significand's low s bits are zero, so (significand >> s)^2 fits one
// 32 x 32 -> 64-bit multiply and the result is placed by a shift.  Same
// value as sq_units(u); nonzero lossy values are normal.
__device__ __forceinline__ void sq_units_q(unsigned long long u, int s, unsigned long long &lo,
                                           unsigned long long &hi, unsigned &range) {
    u &= MAG;
    const unsigned long long E = u >> 52;
    lo = hi = 0;
    if (E >= 1027) { range = 1; return; }
    if (u == 0) return;
    const uint32_t m = (uint32_t)(((u & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> s);
    const unsigned long long sq = (unsigned long long)m * m;            // < 2^(106 - 2s)
    const int sh = 2 * (int)E - 2038 + 2 * s;                            // x^2 2^112 = sq 2^sh
    if (sh >= 64) { hi = sq << (sh - 64); }
    else if (sh > 0) { lo = sq << sh; hi = sq >> (64 - sh); }
    else if (sh == 0) { lo = sq; }
    else if (sh > -64) { lo = sq >> (-sh); }
}

// Code q = (B + 2^(s-1)) >> s of the magnitude bits B = mh:lo (high and
// low words) for 32 <= s <= 52, in 32-bit arithmetic: for s >= 33 the low
// word cannot carry into the result, for s = 32 it adds its top bit.
__device__ __forceinline__ uint32_t quant_hi(uint32_t mh, uint32_t lo, int s) {
    return s == 32 ? mh + (lo >> 31) : (mh + (1u << (s - 33))) >> (s - 32);
}

// sq_units of the reconstructed value q << s (32 <= s <= 52): the same value,
// from the code in 32-bit arithmetic (exponent q >> (52 - s), significand
// bits above the s zero bits).
__device__ __forceinline__ void sq_units_code(uint32_t q, int s, unsigned long long &lo,
                                              unsigned long long &hi, unsigned &range) {
    lo = hi = 0;
    if (q == 0) return;
    const int fb = 52 - s;                                   // fraction bits kept
    const uint32_t E = q >> fb;
    if (E >= 1027u) { range = 1; return; }
    const uint32_t m = (q & ((1u << fb) - 1u)) | (1u << fb);
    const unsigned long long sq = (unsigned long long)m * m;
    const int sh = 2 * (int)E - 2038 + 2 * s;
    if (sh >= 64) { hi = sq << (sh - 64); }
    else if (sh > 0) { lo = sq << sh; hi = sq >> (64 - sh); }
    else if (sh == 0) { lo = sq; }
    else if (sh > -64) { lo = sq >> (-sh); }
}

__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi,
                                       unsigned long long alo, unsigned long long ahi) {
    unsigned long long nlo = lo + alo;
    hi += ahi + (nlo < lo ? 1ull : 0ull);
    lo = nlo;
}

__device__ __forceinline__ void warp_sum128(unsigned long long &lo, unsigned long long &hi) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long olo = shfl64(lo, (threadIdx.x & 31) ^ o);
        unsigned long long ohi = shfl64(hi, (threadIdx.x & 31) ^ o);
        add128(lo, hi, olo, ohi);
    }
}

// add (lo, hi) to a global 128-bit accumulator; exact under concurrency
__device__ __forceinline__ void atomic_add128(unsigned long long *alo, unsigned long long *ahi,
                                              unsigned long long lo, unsigned long long hi) {
    unsigned long long old = atomicAdd(alo, lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(ahi, hi + carry);
}

// Per-CTA sums of one state's pass (norm units, tiles per ladder level,
// tiles over the size limit), kept in shared memory and added to the
// state's counters once per CTA and state: the tiles of a sweep then make
// no global atomics on these shared words, only the CTAs do.
struct PassAcc {
    unsigned long long lo, hi, over;
    unsigned long long hist[MAX_LEVELS];
};

// The bookkeeping of one written tile (one thread): its norm partial, its
// level and whether it is over the size limit; into acc, or into the
// state's counters when acc is null.
__device__ __forceinline__ void tally_tile(PassAcc *acc, DevScalars *scal, unsigned long long nlo,
                                           unsigned long long nhi, int level, bool over) {
    if (acc) {
        atomic_add128(&acc->lo, &acc->hi, nlo, nhi);
        atomicAdd(&acc->hist[level], 1ull);
        if (over) atomicAdd(&acc->over, 1ull);
    } else {
        atomic_add128(&scal->acc_lo, &scal->acc_hi, nlo, nhi);
        atomicAdd(&scal->hist[level], 1ull);
        if (over) atomicAdd(&scal->over_limit, 1ull);
    }
}

// A stream carried or moved unchanged: its norm partial only.
__device__ __forceinline__ void tally_norm(PassAcc *acc, DevScalars *scal, unsigned long long nlo,
                                           unsigned long long nhi) {
    if (acc) atomic_add128(&acc->lo, &acc->hi, nlo, nhi);
    else atomic_add128(&scal->acc_lo, &scal->acc_hi, nlo, nhi);
}

// Adds a CTA's sums to the state's counters and clears them (one thread).
__device__ void flush_acc(PassAcc *acc, DevScalars *scal) {
    if (acc->lo | acc->hi) atomic_add128(&scal->acc_lo, &scal->acc_hi, acc->lo, acc->hi);
    for (int lv = 0; lv < MAX_LEVELS; ++lv)
        if (acc->hist[lv]) atomicAdd(&scal->hist[lv], acc->hist[lv]);
    if (acc->over) atomicAdd(&scal->over_limit, acc->over);
    acc->lo = acc->hi = acc->over = 0;
    for (int lv = 0; lv < MAX_LEVELS; ++lv) acc->hist[lv] = 0;
}

// correctly rounded double of (hi, lo) * 2^-112
__device__ double units_to_double(unsigned long long lo, unsigned long long hi) {
    if (hi == 0 && lo == 0) return 0.0;
    if (hi == 0) {
        int p = bitlen64(lo);
        if (p <= 64) return ldexp(__ull2double_rn(lo), -112);
    }
    int p = 64 + bitlen64(hi);           // hi != 0
    int drop = p - 64;                   // 1..64
    unsigned long long top, rest;
    if (drop == 64) { top = hi; rest = lo; }
    else {
        top = (hi << (64 - drop)) | (lo >> drop);
        rest = lo & ((1ull << drop) - 1);
    }
    top |= (rest != 0) ? 1ull : 0ull;    // sticky bit keeps round-to-nearest exact
    return ldexp(__ull2double_rn(top), drop - 112);
}

// ---------------------------------------------------------------- gates
// y = u * x for one matrix entry of class `code` (first term of a row).
// The class only selects which operations run; the arithmetic is the
// canonical one (a leading +-1 is an exact copy / sign flip).
__device__ __forceinline__ void term_first(unsigned code, double ur, double ui, double xr,
                                           double xi, double &yr, double &yi) {
    switch (code) {
        case EC_ONE: yr = xr; yi = xi; break;
        case EC_MINUS_ONE: yr = -xr; yi = -xi; break;
        case EC_REAL: yr = __dmul_rn(ur, xr); yi = __dmul_rn(ur, xi); break;
        case EC_IMAG: yr = -__dmul_rn(ui, xi); yi = __dmul_rn(ui, xr); break;
        default:
            yr = __fma_rn(ur, xr, -__dmul_rn(ui, xi));
            yi = __fma_rn(ur, xi, __dmul_rn(ui, xr));
            break;
    }
}

// acc += u * x
__device__ __forceinline__ void term_acc(unsigned code, double ur, double ui, double xr,
                                         double xi, double &ar, double &ai) {
    if (code <= EC_REAL) {
        ar = __fma_rn(ur, xr, ar);
        ai = __fma_rn(ur, xi, ai);
    } else if (code == EC_IMAG) {
        ar = __fma_rn(-ui, xi, ar);
        ai = __fma_rn(ui, xr, ai);
    } else {
        ar = __fma_rn(ur, xr, __fma_rn(-ui, xi, ar));
        ai = __fma_rn(ur, xi, __fma_rn(ui, xr, ai));
    }
}

// t = f x for a factor code f (0: 1, 1: -1, 2: i, 3: -i): a selection and
// sign-bit flips, exact and off the FP64 pipe
__device__ __forceinline__ void unit_times(unsigned f, double xr, double xi, double &tr, double &ti) {
    const unsigned long long nr = (f == 1u || f == 2u) ? SIGN_BIT : 0ull;
    const unsigned long long ni = (f == 1u || f == 3u) ? SIGN_BIT : 0ull;
    const bool sw = f >= 2u;
    tr = bitsd(dbits(sw ? xi : xr) ^ nr);
    ti = bitsd(dbits(sw ? xr : xi) ^ ni);
}

// Row r of y = U x over the nonzero entries, in column order.  A factored
// row (bit r of fac: every nonzero entry is f d, f in {1, -1, i, -i}, d
// the first nonzero entry; f of entry e in bits 8 + 2e, codes 0..3 for
// 1, -1, i, -i) is summed first, S = sum f x with one rounded addition per
// later term, and multiplied by d once; equal inputs then cancel exactly.
template <int DIM>
__device__ __forceinline__ void row_eval(const double *m, unsigned long long cls, unsigned long long fac,
                                         int r, const double *xr, const double *xi, double &yr,
                                         double &yi, bool unscaled = false) {
    bool first = true;
    double ar = 0.0, ai = 0.0;
    if ((fac >> r) & 1ull) {
        unsigned dcode = 0;
        double dr = 0.0, di = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
            const int e = r * DIM + c;
            const unsigned code = (unsigned)(cls >> (3 * e)) & 7u;
            if (code == EC_ZERO) continue;
            if (first) {                      // the first entry is d itself: factor 1
                ar = xr[c]; ai = xi[c];
                dcode = code; dr = m[2 * e]; di = m[2 * e + 1];
                first = false;
                continue;
            }
            double tr, ti;
            unit_times((unsigned)(fac >> (8 + 2 * e)) & 3u, xr[c], xi[c], tr, ti);
            ar = __dadd_rn(ar, tr);
            ai = __dadd_rn(ai, ti);
        }
        if (unscaled) { yr = ar; yi = ai; return; }      // d is in the sweep's scale
        term_first(dcode, dr, di, ar, ai, yr, yi);
        return;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        unsigned code = (unsigned)(cls >> (3 * (r * DIM + c))) & 7u;
        if (code == EC_ZERO) continue;
        double ur = m[2 * (r * DIM + c)], ui = m[2 * (r * DIM + c) + 1];
        if (first) { term_first(code, ur, ui, xr[c], xi[c], ar, ai); first = false; }
        else term_acc(code, ur, ui, xr[c], xi[c], ar, ai);
    }
    yr = ar;
    yi = ai;
}

// both components exactly zero (either sign), by their bits (no FP64 compare)
__device__ __forceinline__ bool zero_amp(double xr, double xi) {
    return ((unsigned long long)(__double_as_longlong(xr) | __double_as_longlong(xi)) << 1) == 0ull;
}

// Point items: every member tile exactly +0 (all bits clear) but for at
// most one amplitude, at a tile index p common to the tiles.  Scans a
// decoded tile (warp-wide; the warp wrote it) and merges into the item's
// state: *pos the common index (-1: none seen yet), *bad set when a tile
// holds two such amplitudes or the tiles disagree.
__device__ __forceinline__ void point_scan(const double *re, const double *im, int N, int *pos, int *bad) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned cnt = 0;
    int at = -1;
    for (int b = 0; b < N; b += 32) {
        const int i = b + lane;
        const bool v = i < N && (unsigned long long)(__double_as_longlong(re[i]) | __double_as_longlong(im[i])) != 0ull;
        const unsigned bal = __ballot_sync(FULL, v);
        cnt += (unsigned)__popc(bal);
        if (bal) at = b + 31 - __clz(bal);
    }
    if (lane == 0 && cnt) {
        if (cnt > 1) {
            atomicOr(bad, 1);
        } else {
            const int old = atomicCAS(pos, -1, at);
            if (old != -1 && old != at) atomicOr(bad, 1);
        }
    }
}

// log2 of the warps of the CTA (a power of two: 4, 8 or 16 in the sweep)
__device__ __forceinline__ int log_nwarps() { return __ffs((int)(blockDim.x >> 5)) - 1; }

__device__ __forceinline__ unsigned insert_zero(unsigned v, int p) {
    unsigned lowm = (1u << p) - 1u;
    return ((v & ~lowm) << 1) | (v & lowm);
}

// buffer index of the f-th amplitude whose pinned bits (ascending ins[]) are 0
__device__ __forceinline__ unsigned deposit(unsigned f, const SGate &s) {
    for (int i = 0; i < s.nins; ++i) f = insert_zero(f, s.ins[i]);
    return f;
}

// Which gates of the sweep change something in the item with fixed bits
// `fixed`: fixed controls met, and for a diagonal gate whose targets are all
// fixed, its entry there is not exactly 1.  Bit g of the result.
__device__ __forceinline__ bool gate_active(const SGate &s, unsigned long long fixed) {
    if (((fixed ^ s.fcv) & s.fcm) != 0ull) return false;
    if (s.kind == 0 && s.p0 < 0 && (s.k < 2 || s.p1 < 0)) {
        int r = (int)((fixed >> s.t0) & 1ull);
        if (s.k > 1) r |= (int)((fixed >> s.t1) & 1ull) << 1;
        if ((s.one_mask >> r) & 1) return false;
    }
    return true;
}

// The barrier of a gate pass: the CTA's, or the warp's when one warp
// applies the gates alone (nth == 32: items of one amplitude per tile).
__device__ __forceinline__ void gsync(unsigned nth) {
    if (nth == 32u) __syncwarp();
    else __syncthreads();
}

// One diagonal gate, applied only where it changes something: the
// amplitudes whose local controls hold and whose target sub-index r has an
// entry other than exactly 1.  Enumerating just those keeps every lane of
// every FP64 instruction busy (masked lanes cost the same on this part).
__device__ void diag_gate(double *re, double *im, int mb, const SGate &s,
                          unsigned long long fixed, int red, unsigned roff,
                          unsigned tid, unsigned nth) {
    // sub-indices r to visit: entry != 1 and consistent with fixed targets
    unsigned rpack = 0;          // sub-indices, 2 bits each
    int nr = 0;
    const int dim = 1 << s.k;
    int fmask = 0, fval = 0;
    if (s.p0 < 0) { fmask |= 1; fval |= (int)((fixed >> s.t0) & 1ull); }
    if (s.k > 1 && s.p1 < 0) { fmask |= 2; fval |= (int)((fixed >> s.t1) & 1ull) << 1; }
    for (int r = 0; r < dim; ++r)
        if ((r & fmask) == fval && !((s.one_mask >> r) & 1)) rpack |= (unsigned)r << (2 * nr++);
    if (nr == 0) return;
    const int fb = mb - s.nins - red;           // free bits (the low `red` bits stay 0)
    const unsigned cnt = (unsigned)nr << fb;
    for (unsigned f = tid; f < cnt; f += nth) {
        int r = (int)((rpack >> (2 * (f >> fb))) & 3u);
        unsigned l = deposit((f & ((1u << fb) - 1u)) << red, s) | s.lcv | roff;
        if (s.p0 >= 0) l |= (unsigned)(r & 1) << s.p0;
        if (s.k > 1 && s.p1 >= 0) l |= (unsigned)((r >> 1) & 1) << s.p1;
        unsigned code = (unsigned)(s.cls >> (3 * r)) & 7u;
        double yr = 0.0, yi = 0.0;
        if (code != EC_ZERO) term_first(code, s.d[2 * r], s.d[2 * r + 1], re[l], im[l], yr, yi);
        re[l] = yr;
        im[l] = yi;
    }
}

// Warp-local form of diag_gate for an item of 2^mb amplitudes: warp w
// handles the amplitudes whose top log2(warps) index bits equal w, so
// consecutive diagonal gates need only __syncwarp between them (each
// amplitude still sees the gates in order, with the same arithmetic).
// Needs mb - log2(warps) >= 5.
__device__ void diag_gate_warp(double *re, double *im, int mb, const SGate &s, unsigned long long fixed) {
    const int lane = threadIdx.x & 31;
    const int cb = mb - log_nwarps();               // index bits that vary inside a warp's part
    const unsigned inmask = (1u << cb) - 1u;
    const unsigned W = (unsigned)(threadIdx.x >> 5) << cb;
    if (((W ^ s.lcv) & s.lcm & ~inmask) != 0u) return;      // a control outside the part fails
    int fmask = 0, fval = 0;                         // target bits fixed for this warp
    if (s.p0 < 0) { fmask |= 1; fval |= (int)((fixed >> s.t0) & 1ull); }
    else if (s.p0 >= cb) { fmask |= 1; fval |= (int)((W >> s.p0) & 1u); }
    if (s.k > 1) {
        if (s.p1 < 0) { fmask |= 2; fval |= (int)((fixed >> s.t1) & 1ull) << 1; }
        else if (s.p1 >= cb) { fmask |= 2; fval |= (int)((W >> s.p1) & 1u) << 1; }
    }
    unsigned rpack = 0;
    int nr = 0;
    for (int r = 0; r < (1 << s.k); ++r)
        if ((r & fmask) == fval && !((s.one_mask >> r) & 1)) rpack |= (unsigned)r << (2 * nr++);
    if (nr == 0) return;
    int nin = 0;                                     // pinned bits inside the part (ins is ascending)
    while (nin < s.nins && s.ins[nin] < cb) ++nin;
    const int fb = cb - nin;
    const unsigned cnt = (unsigned)nr << fb;
    const unsigned base = (s.lcv & inmask) | W;
    if (nr == 1) {
        // one entry (controlled phases, CZ, MCZ, Z, S, T): entry, class and
        // target bits held in registers across the loop
        const int r = (int)(rpack & 3u);
        const unsigned code = (unsigned)(s.cls >> (3 * r)) & 7u;
        const double ur = s.d[2 * r], ui = s.d[2 * r + 1];
        unsigned add = base;
        if (s.p0 >= 0 && s.p0 < cb) add |= (unsigned)(r & 1) << s.p0;
        if (s.k > 1 && s.p1 >= 0 && s.p1 < cb) add |= (unsigned)((r >> 1) & 1) << s.p1;
        uint8_t pos[12];
        for (int i = 0; i < nin; ++i) pos[i] = s.ins[i];
        for (unsigned f = lane; f < cnt; f += 32) {
            unsigned l = f;
            for (int i = 0; i < nin; ++i) l = insert_zero(l, pos[i]);
            l |= add;
            double yr = 0.0, yi = 0.0;
            if (code != EC_ZERO) term_first(code, ur, ui, re[l], im[l], yr, yi);
            re[l] = yr;
            im[l] = yi;
        }
        return;
    }
    for (unsigned f = lane; f < cnt; f += 32) {
        const int r = (int)((rpack >> (2 * (f >> fb))) & 3u);
        unsigned l = f & ((1u << fb) - 1u);
        for (int i = 0; i < nin; ++i) l = insert_zero(l, s.ins[i]);
        l |= base;
        if (s.p0 >= 0 && s.p0 < cb) l |= (unsigned)(r & 1) << s.p0;
        if (s.k > 1 && s.p1 >= 0 && s.p1 < cb) l |= (unsigned)((r >> 1) & 1) << s.p1;
        const unsigned code = (unsigned)(s.cls >> (3 * r)) & 7u;
        double yr = 0.0, yi = 0.0;
        if (code != EC_ZERO) term_first(code, s.d[2 * r], s.d[2 * r + 1], re[l], im[l], yr, yi);
        re[l] = yr;
        im[l] = yi;
    }
}

// A scaled gate (s.unscaled != 0) leaves a pair of exactly-zero amplitudes
// as it is and returns the FP64 instructions of the pairs it formed; other
// gates return 0 (their canonical count is the host's).
__device__ unsigned one_target(double *re, double *im, int mb, const SGate &s, const DGate &dg, int red,
                               unsigned roff, unsigned tid, unsigned nth) {
    double m[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) m[i] = dg.m[i];
    const unsigned bit = 1u << s.p0;
    const unsigned cnt = 1u << (mb - s.nins - red);
    if ((s.cls & 0xFFFull) == ((unsigned long long)EC_ONE << 3 | (unsigned long long)EC_ONE << 6)) {
        // X (entries 0 1 / 1 0, exactly): the pair is exchanged, the copies
        // the rows would make
        for (unsigned f = tid; f < cnt; f += nth) {
            const unsigned l0 = deposit(f << red, s) | s.lcv | roff, l1 = l0 | bit;
            const double ar = re[l0], ai = im[l0], br = re[l1], bi = im[l1];
            re[l0] = br; im[l0] = bi;
            re[l1] = ar; im[l1] = ai;
        }
        return 0;
    }
    if ((s.fac & 3ull) == 3ull && (s.cls & 7ull) == EC_REAL && ((s.cls >> 6) & 7ull) == EC_REAL) {
        // both rows factored with a real first entry (Hadamard-like):
        // y_r = d_r (x_0 + f_r x_1), the same arithmetic as row_eval
        const double d0 = m[0], d1 = m[4];
        const unsigned f0 = (unsigned)(s.fac >> 10) & 3u, f1 = (unsigned)(s.fac >> 14) & 3u;
        const int nins = s.nins;
        uint8_t pos[12];
        for (int i = 0; i < nins; ++i) pos[i] = s.ins[i];
        const unsigned lcv = s.lcv | roff;
        if (s.unscaled) {
            // a scaled gate: d is in the sweep's scale, the rows are their sums
            unsigned pairs = 0;
            for (unsigned f = tid; f < cnt; f += nth) {
                unsigned l = f << red;
                for (int i = 0; i < nins; ++i) l = insert_zero(l, pos[i]);
                const unsigned l0 = l | lcv;
                const unsigned l1 = l0 | bit;
                const double x0r = re[l0], x0i = im[l0], x1r = re[l1], x1i = im[l1];
                if (zero_amp(x0r, x0i) && zero_amp(x1r, x1i)) continue;
                double t0r, t0i, t1r, t1i;
                unit_times(f0, x1r, x1i, t0r, t0i);
                unit_times(f1, x1r, x1i, t1r, t1i);
                re[l0] = __dadd_rn(x0r, t0r);
                im[l0] = __dadd_rn(x0i, t0i);
                re[l1] = __dadd_rn(x0r, t1r);
                im[l1] = __dadd_rn(x0i, t1i);
                ++pairs;
            }
            return pairs * s.unscaled;
        }
        for (unsigned f = tid; f < cnt; f += nth) {
            unsigned l = f << red;
            for (int i = 0; i < nins; ++i) l = insert_zero(l, pos[i]);
            const unsigned l0 = l | lcv;
            const unsigned l1 = l0 | bit;
            const double x0r = re[l0], x0i = im[l0], x1r = re[l1], x1i = im[l1];
            double t0r, t0i, t1r, t1i;
            unit_times(f0, x1r, x1i, t0r, t0i);
            unit_times(f1, x1r, x1i, t1r, t1i);
            re[l0] = __dmul_rn(d0, __dadd_rn(x0r, t0r));
            im[l0] = __dmul_rn(d0, __dadd_rn(x0i, t0i));
            re[l1] = __dmul_rn(d1, __dadd_rn(x0r, t1r));
            im[l1] = __dmul_rn(d1, __dadd_rn(x0i, t1i));
        }
        return 0;
    }
    unsigned groups = 0;
    for (unsigned f = tid; f < cnt; f += nth) {
        unsigned l0 = deposit(f << red, s) | s.lcv | roff;
        unsigned l1 = l0 | bit;
        double xr[2] = {re[l0], re[l1]}, xi[2] = {im[l0], im[l1]};
        if (s.unscaled) {
            if (zero_amp(xr[0], xi[0]) && zero_amp(xr[1], xi[1])) continue;
            ++groups;
        }
        double y0r, y0i, y1r, y1i;
        row_eval<2>(m, s.cls, s.fac, 0, xr, xi, y0r, y0i, s.unscaled);
        row_eval<2>(m, s.cls, s.fac, 1, xr, xi, y1r, y1i, s.unscaled);
        re[l0] = y0r; im[l0] = y0i;
        re[l1] = y1r; im[l1] = y1i;
    }
    return groups * s.unscaled;
}

// As one_target, for gates on two targets.
__device__ unsigned two_target(double *re, double *im, int mb, const SGate &s, const DGate &dg, int red,
                               unsigned roff, unsigned tid, unsigned nth) {
    const unsigned cnt = 1u << (mb - s.nins - red);
    // a permutation (SWAP; X on one target controlled by the other): every
    // row one entry exactly 1 and the others exactly 0; row r copies x[src r]
    unsigned src = 0, moved = 0;
    bool perm = true;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        int ones = 0, zeros = 0, at = 0;
#pragma unroll
        for (int c2 = 0; c2 < 4; ++c2) {
            const unsigned code = (unsigned)(s.cls >> (3 * (r * 4 + c2))) & 7u;
            if (code == EC_ONE) { ++ones; at = c2; }
            else if (code == EC_ZERO) ++zeros;
        }
        perm &= ones == 1 && zeros == 3;
        src |= (unsigned)at << (2 * r);
        if (at != r) moved |= 1u << r;
    }
    if (perm) {
        for (unsigned f = tid; f < cnt && moved; f += nth) {
            const unsigned l = deposit(f << red, s) | s.lcv | roff;
            unsigned idx[4];
            double xr[4], xi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                idx[q] = l | ((unsigned)(q & 1) << s.p0) | ((unsigned)(q >> 1) << s.p1);
                xr[q] = re[idx[q]];
                xi[q] = im[idx[q]];
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (!((moved >> r) & 1u)) continue;
                const unsigned q = (src >> (2 * r)) & 3u;
                re[idx[r]] = q == 0 ? xr[0] : q == 1 ? xr[1] : q == 2 ? xr[2] : xr[3];
                im[idx[r]] = q == 0 ? xi[0] : q == 1 ? xi[1] : q == 2 ? xi[2] : xi[3];
            }
        }
        return 0;
    }
    unsigned groups = 0;
    for (unsigned f = tid; f < cnt; f += nth) {
        unsigned l = deposit(f << red, s) | s.lcv | roff;
        unsigned idx[4];
        double xr[4], xi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            idx[q] = l | ((unsigned)(q & 1) << s.p0) | ((unsigned)(q >> 1) << s.p1);
            xr[q] = re[idx[q]];
            xi[q] = im[idx[q]];
        }
        if (s.unscaled) {
            if (zero_amp(xr[0], xi[0]) && zero_amp(xr[1], xi[1]) && zero_amp(xr[2], xi[2]) &&
                zero_amp(xr[3], xi[3]))
                continue;
            ++groups;
        }
        double yr[4], yi[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) row_eval<4>(dg.m, s.cls, s.fac, r, xr, xi, yr[r], yi[r], s.unscaled);
#pragma unroll
        for (int q = 0; q < 4; ++q) { re[idx[q]] = yr[q]; im[idx[q]] = yi[q]; }
    }
    return groups * s.unscaled;
}

// tile index of an item: zero bits inserted at the tile-index positions
// hb[0] < hb[1] < ... of the h paired qubits
__device__ __forceinline__ unsigned long long expand_item(unsigned long long item, int h,
                                                           const int *hb) {
    unsigned long long v = item;
#pragma unroll
    for (int i = 0; i < MAX_PAIRS; ++i) {
        if (i >= h) break;
        const unsigned long long m = (1ull << hb[i]) - 1ull;
        v = ((v & ~m) << 1) | (v & m);
    }
    return v;
}

// tile of member j of the item whose first tile is T
__device__ __forceinline__ unsigned long long member_tile(unsigned long long T, int j, int h,
                                                          const int *hb) {
#pragma unroll
    for (int i = 0; i < MAX_PAIRS; ++i) {
        if (i >= h) break;
        T |= (unsigned long long)((j >> i) & 1) << hb[i];
    }
    return T;
}

// ---------------------------------------------------------------- diagonal runs
// general complex term y = u x (term_first's general arithmetic)
__device__ __forceinline__ void cmul(double ur, double ui, double xr, double xi, double &yr, double &yi) {
    const double r = __fma_rn(ur, xr, -__dmul_rn(ui, xi));
    const double i = __fma_rn(ur, xi, __dmul_rn(ui, xr));
    yr = r;
    yi = i;
}

// x <- i^k x (exact: a swap and sign-bit flips)
__device__ __forceinline__ void unit_pow(unsigned k, double &xr, double &xi) {
    k &= 3u;
    if (k == 0u) return;
    const unsigned f = k == 1u ? 2u : (k == 2u ? 1u : 3u);      // unit_times codes: 1 -> -1, 2 -> i, 3 -> -i
    double tr, ti;
    unit_times(f, xr, xi, tr, ti);
    xr = tr;
    xi = ti;
}

// Ordered product of the factors of gates g[0..n-1] at global index x:
// general factors into (pr, pi) (have set when one exists), unit
// exponents added to k.  Returns the FP64 instructions executed.
__device__ __forceinline__ unsigned run_factor(const RGate *g, int n, unsigned long long x, bool &have,
                                               double &pr, double &pi, unsigned &k) {
    unsigned ops = 0;
    for (int i = 0; i < n; ++i) {
        const RGate &G = g[i];
        if ((x & G.cm) != G.cv) continue;
        int r = (int)((x >> G.t0) & 1ull);
        if (G.k > 1) r |= (int)((x >> G.t1) & 1ull) << 1;
        const unsigned code = G.code[r];
        if (code == 0u) continue;
        if (code == 1u) { k += G.uexp[r]; continue; }
        if (have) { cmul(G.e[2 * r], G.e[2 * r + 1], pr, pi, pr, pi); ops += 4; }
        else { pr = G.e[2 * r]; pi = G.e[2 * r + 1]; have = true; }
    }
    return ops;
}

// Tables of the local product L of every tabled run: one CTA per (run,
// class), entry x_lo at runs[r].table + class * 2^c + x_lo; then the
// class's summary (active / general entry counts, tile bits common to the
// active entries).  The class index's bit i is index bit q[i].
__global__ void __launch_bounds__(256) run_tables_kernel(const DRun *runs, const int2 *classes, int nclasses,
                                                         const RGate *rgates, int c, double2 *tab,
                                                         uint8_t *meta, RunClass *rcls, DevScalars *scal) {
    __shared__ unsigned s_active, s_have, s_and, s_or;
    __shared__ unsigned long long s_ops;
    const int N = 1 << c;
    for (int ci = blockIdx.x; ci < nclasses; ci += gridDim.x) {
        const int r = classes[ci].x, kap = classes[ci].y;
        const DRun &R = runs[r];
        if (threadIdx.x == 0) { s_active = 0; s_have = 0; s_and = ~0u; s_or = 0; s_ops = 0; }
        __syncthreads();
        unsigned long long xh = 0;
        for (int i = 0; i < R.nq; ++i) xh |= (unsigned long long)((kap >> i) & 1) << R.q[i];
        unsigned act = 0, hv = 0, am = ~0u, om = 0, ops = 0;
        for (int xl = threadIdx.x; xl < N; xl += blockDim.x) {
            bool have = false;
            double pr = 0.0, pi = 0.0;
            unsigned k = 0;
            ops += run_factor(rgates + R.lg, R.nl, xh | (unsigned long long)xl, have, pr, pi, k);
            const unsigned long long e = R.table + (unsigned long long)kap * N + xl;
            tab[e] = make_double2(pr, pi);
            meta[e] = (uint8_t)((have ? 1u : 0u) | ((k & 3u) << 1));
            if (have || (k & 3u)) { ++act; am &= (unsigned)xl; om |= (unsigned)xl; }
            if (have) ++hv;
        }
        atomicAdd(&s_active, act);
        atomicAdd(&s_have, hv);
        atomicAnd(&s_and, am);
        atomicOr(&s_or, om);
        atomicAdd(&s_ops, (unsigned long long)ops);
        __syncthreads();
        if (threadIdx.x == 0) {
            RunClass rc;
            rc.active = s_active;
            rc.have = s_have;
            const unsigned lowm = (unsigned)N - 1u;
            rc.pin_mask = s_active ? ((s_and | ~s_or) & lowm) : 0u;
            rc.pin_val = s_active ? (s_and & lowm) : 0u;
            rcls[R.cls + kap] = rc;
            if (s_ops) atomicAdd(&scal->run_dp, s_ops);
        }
        __syncthreads();
    }
}

// D of every sweep of a flush: the product, in gate order starting from 1,
// of the first nonzero entry d of row 0 of each scaled gate (a gate that is
// d times a matrix of units), sweep j holding gates bounds[j].x .. .y - 1.
__global__ void sweep_scale_kernel(const SGate *sg, const DGate *dg, const int2 *bounds, int ns, double *D) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ns) return;
    double p = 1.0;
    for (int g = bounds[j].x; g < bounds[j].y; ++g) {
        if (!sg[g].unscaled) continue;
        const int dim = 1 << sg[g].k;
        int e = 0;
        while (e < dim && ((sg[g].cls >> (3 * e)) & 7ull) == EC_ZERO) ++e;
        p = __dmul_rn(p, dg[g].m[2 * e]);
    }
    D[j] = p;
}

// Per member tile of an item, for the run being applied.
struct RunMember {
    double tr, ti;                  // tile product T
    uint32_t count;                 // amplitudes to visit
    uint32_t pin_mask, pin_val;     // visited tile bits: all (mask 0) or the class's pinned subset
    uint16_t kap;                   // class
    uint8_t have_t, k_t;
};

// One diagonal run applied to an item buffer (every thread calls it).
// red > 0: one amplitude per tile (uniform items; such sweeps have no local
// gates).  An amplitude that is exactly zero is left as it is.  Returns the
// FP64 instructions this thread executed.
__device__ unsigned apply_run(double *re, double *im, int c, int h, int red, const DRun &Rg,
                              const SweepParams &P, unsigned long long T, const int *hb, RunMember *mem,
                              uint32_t *stage, int stage_words, unsigned roff,
                              unsigned tid, unsigned nth) {
    const DRun R = Rg;                             // in registers: one load of the descriptor
    const int ntl = 1 << h, N = 1 << c;
    unsigned ops = 0;
    // the run's tile gates copied to shared memory by the whole CTA (stage:
    // the encoder's packing area, idle while gates run), so that the member
    // products below walk them without a global load per gate
    const int nt = R.nt, tg = R.tg;
    const int nst = min(nt, stage_words / (int)(sizeof(RGate) / 4));
    {
        // 16-byte copies, several in flight per thread (one warp copies alone
        // in items of one amplitude per tile)
        const uint4 *src = reinterpret_cast<const uint4 *>(P.rgates + tg);
        uint4 *dst = reinterpret_cast<uint4 *>(stage);
        const int n4 = nst * (int)(sizeof(RGate) / 16);
#pragma unroll 4
        for (int i = (int)tid; i < n4; i += (int)nth) dst[i] = src[i];
    }
    // the run at amplitude xl of member j (whose setup is m)
    auto visit = [&](int j, unsigned xl, const RunMember &m) {
        const unsigned l = ((unsigned)j << c) | xl;
        double xr = re[l], xi = im[l];
        if (zero_amp(xr, xi)) return;             // a zero stays as it is
        bool have_l = false;
        double lr = 0.0, li = 0.0;
        unsigned k = m.k_t;
        if (R.nl) {
            if (R.tabled) {
                const unsigned long long e = R.table + (unsigned long long)m.kap * N + xl;
                const unsigned mt = P.rmeta[e];
                have_l = mt & 1u;
                k += mt >> 1;
                if (have_l) {
                    const double2 v = P.rtab[e];
                    lr = v.x;
                    li = v.y;
                }
            } else {
                const unsigned long long x = (member_tile(T, j, h, hb) << c) | xl;
                ops += run_factor(P.rgates + R.lg, R.nl, x, have_l, lr, li, k);
            }
        }
        const bool have_t = m.have_t;
        if (!have_t && !have_l && (k & 3u) == 0u) return;
        if (have_t || have_l) {
            double gr = have_t ? m.tr : lr, gi = have_t ? m.ti : li;
            if (have_t && have_l) { cmul(m.tr, m.ti, lr, li, gr, gi); ops += 4; }
            cmul(gr, gi, xr, xi, xr, xi);
            ops += 4;
        }
        unit_pow(k, xr, xi);
        re[l] = xr;
        im[l] = xi;
    };
    gsync(nth);
    if ((int)tid < ntl) {
        const int j = tid;
        const unsigned long long xb = member_tile(T, j, h, hb) << c;
        bool have = false;
        double tr = 0.0, ti = 0.0;
        unsigned k = 0;
        ops += run_factor(reinterpret_cast<const RGate *>(stage), nst, xb, have, tr, ti, k);
        ops += run_factor(P.rgates + tg + nst, nt - nst, xb, have, tr, ti, k);
        unsigned kap = 0;
        for (int i = 0; i < R.nq; ++i) kap |= (unsigned)((xb >> R.q[i]) & 1ull) << i;
        RunMember m;
        m.tr = tr;
        m.ti = ti;
        m.have_t = have ? 1 : 0;
        m.k_t = (uint8_t)(k & 3u);
        m.kap = (uint16_t)kap;
        m.pin_mask = 0;
        m.pin_val = 0;
        const bool tile_part = have || (k & 3u);
        if (red) m.count = (tile_part || R.nl) ? 1u : 0u;
        else if (tile_part) m.count = (uint32_t)N;
        else if (R.nl == 0) m.count = 0;
        else if (!R.tabled) m.count = (uint32_t)N;
        else {
            const RunClass rc = P.rcls[R.cls + kap];
            m.pin_mask = rc.pin_mask;
            m.pin_val = rc.pin_val;
            m.count = rc.active ? (uint32_t)N >> __popc(rc.pin_mask) : 0u;
        }
        // one amplitude per tile: member j's own thread visits it, no barrier
        if (red) {
            if (m.count) visit(j, roff, m);
        } else {
            mem[j] = m;
        }
    }
    if (red) return ops;
    gsync(nth);
    int j = 0;
    unsigned base = 0;
    for (unsigned w = tid;; w += nth) {
        while (j < ntl && w >= base + mem[j].count) { base += mem[j].count; ++j; }
        if (j >= ntl) break;
        const RunMember &m = mem[j];
        unsigned f = w - base;
        // deposit f into the tile bits outside pin_mask, pinned bits from pin_val
        unsigned pm = m.pin_mask, xl = f;
        while (pm) {
            const int b = __ffs(pm) - 1;
            xl = insert_zero(xl, b);
            pm &= pm - 1;
        }
        xl |= m.pin_val;
        visit(j, xl, m);
    }
    return ops;
}

// Apply the sweep's gates (in order) to an item buffer of 2^mb amplitudes.
// act: bit g set when gate g changes something in this item.  The compact
// gates are staged in shared memory GATE_CHUNK at a time (*chunk = first
// gate staged, -1 none); chunks without an active gate are not staged.
// red > 0: one amplitude per tile, at tile index roff (uniform items: 0,
// gates that touch no low qubit; point items: the common index of the
// tiles' one nonzero amplitude); warp 0 applies them alone and the other
// warps return at once.  Every thread must call it.
// A gate that starts a diagonal run (SGate::run >= 0) applies the whole run
// (apply_run); the run's other gates carry no activity bit (the sweep
// kernel moves the run's activity onto its first gate).  Returns the FP64
// instructions this thread executed in diagonal runs and scaled gates.
__device__ __noinline__ unsigned apply_gates(double *re, double *im, int mb, int red, const SGate *gsrc, SGate *sg,
                            int *chunk, const DGate *dg, int ngates, const unsigned *act,
                            unsigned long long fixed, const SweepParams &P, const int *hb, RunMember *mem,
                            uint32_t *stage, int stage_words, unsigned roff) {
    const bool warp_parts = red == 0 && mb - log_nwarps() >= 5;
    // one amplitude per tile (red > 0): warp 0 applies the gates alone,
    // with warp barriers; the caller joins the CTA afterwards
    const bool wo = red > 0;
    if (wo && threadIdx.x >= 32u) return 0;
    const unsigned tid = wo ? (threadIdx.x & 31u) : threadIdx.x, nth = wo ? 32u : blockDim.x;
    unsigned run_ops = 0;
    bool dirty = false;                              // warp-local gates since the last CTA barrier
    // the gates that can apply (a diagonal run's later gates apply with its
    // first): staged GATE_CHUNK list positions at a time
    const int *gl = P.glist;
    const int nl = P.nglist;
    constexpr int SW = (int)(sizeof(SGate) / 4);
    for (int base = 0; base < nl; base += GATE_CHUNK) {
        const int cn = min(GATE_CHUNK, nl - base);
        bool any = false;
        for (int i = 0; i < cn && !any; ++i) {
            const int g = gl[base + i];
            any = (act[g >> 5] >> (g & 31)) & 1u;
        }
        if (!any) continue;
        if (*chunk != base) {
            gsync(nth);
            uint32_t *dst = reinterpret_cast<uint32_t *>(sg);
            for (int idx = (int)tid; idx < cn * SW; idx += (int)nth) {
                const int i = idx / SW;
                dst[idx] = reinterpret_cast<const uint32_t *>(gsrc + gl[base + i])[idx - i * SW];
            }
            if (tid == 0) *chunk = base;
            gsync(nth);
        }
        for (int i = 0; i < cn; ++i) {
            const int g = gl[base + i];
            if (!((act[g >> 5] >> (g & 31)) & 1u)) continue;
            const SGate &s = sg[i];
            if (s.run != -1) {
                if (s.run < 0) continue;            // inside a run: applied with its first gate
                if (dirty) { __syncthreads(); dirty = false; }
                run_ops += apply_run(re, im, P.cc.c, mb - P.cc.c, red, P.runs[s.run], P, fixed >> P.cc.c, hb, mem,
                                     stage, stage_words, roff, tid, nth);
                gsync(nth);
                continue;
            }
            if (s.kind == 0 && warp_parts) {
                // runs of diagonal gates: warp-local, no CTA barrier between them
                diag_gate_warp(re, im, mb, s, fixed);
                __syncwarp();
                dirty = true;
                continue;
            }
            if (dirty) { __syncthreads(); dirty = false; }
            if (s.kind == 0) diag_gate(re, im, mb, s, fixed, red, roff, tid, nth);
            else if (s.kind == 1) run_ops += one_target(re, im, mb, s, dg[g], red, roff, tid, nth);
            else run_ops += two_target(re, im, mb, s, dg[g], red, roff, tid, nth);
            gsync(nth);
        }
    }
    if (dirty) __syncthreads();
    return run_ops;
}

// ---------------------------------------------------------------- warp codec
// One warp codes one whole tile: lane g holds the metadata of group g, the
// groups are walked in order with the running prefix (decode) or the last
// code of the previous group (encode) carried in registers.  No CTA
// barriers are involved, so the warps of a CTA code different tiles
// independently.

// exclusive prefix of v over the lanes; *total = sum over the warp
__device__ __forceinline__ uint32_t warp_exscan(uint32_t v, uint32_t &total) {
    const int lane = threadIdx.x & 31;
    uint32_t inc = v;
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(FULL, inc, d);
        if (lane >= d) inc += o;
    }
    total = __shfl_sync(FULL, inc, 31);
    return inc - v;
}

// bit mask of the lanes below this one
__device__ __forceinline__ uint32_t lanes_below() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

// Word section of per-group bit words (lane g holds the word of group g):
// mode 0 every word 0, 1 every word == lanes, else the shortest of 2
// (exceptions to 0), 3 (exceptions to `lanes`) and 4 (every word), the
// lower mode on a tie.  Exception modes store a bitmap word (bit g: word g
// differs from the base) and then the differing words in group order.
// Warp-uniform result; *bytes = the section's size.
__device__ __forceinline__ int section_mode(uint32_t v, int G, uint32_t lanes, uint32_t &bytes) {
    const int lane = threadIdx.x & 31;
    const uint32_t n0 = __popc(__ballot_sync(FULL, lane < G && v != 0u));
    const uint32_t n1 = __popc(__ballot_sync(FULL, lane < G && v != lanes));
    if (n0 == 0) { bytes = 0; return S_CLEAR; }
    if (n1 == 0) { bytes = 0; return S_SET; }
    const uint32_t nb = 4u * (uint32_t)((G + 31) >> 5);
    const uint32_t b2 = nb + 4u * n0, b3 = nb + 4u * n1, b4 = 4u * (uint32_t)G;
    int m = S_EXC_CLEAR;
    bytes = b2;
    if (b3 < bytes) { m = S_EXC_SET; bytes = b3; }
    if (b4 < bytes) { m = S_WORDS; bytes = b4; }
    return m;
}

// write a word section in mode md at sec (4-byte aligned)
__device__ __forceinline__ void write_section(uint32_t *sec, int md, uint32_t v, int G, uint32_t lanes) {
    const int lane = threadIdx.x & 31;
    if (md == S_WORDS) {
        if (lane < G) sec[lane] = v;
    } else if (md == S_EXC_CLEAR || md == S_EXC_SET) {
        const uint32_t base = md == S_EXC_SET ? lanes : 0u;
        const uint32_t bm = __ballot_sync(FULL, lane < G && v != base);
        if (lane == 0) sec[0] = bm;
        if ((bm >> lane) & 1u) sec[1 + __popc(bm & lanes_below())] = v;
    }
}

// Word i of a stream body: from mw (lane l holds body word l, l < 32,
// loaded once) when i < 32, else from memory.  Every lane must call it
// (the shuffle is warp-wide); `want` says whether this lane needs a value.
__device__ __forceinline__ uint32_t body_word(const uint32_t *b32, uint32_t mw, uint32_t i, bool want) {
    const uint32_t sv = __shfl_sync(FULL, mw, (int)(i & 31u));
    if (!want) return 0u;
    return i < 32u ? sv : __ldg(b32 + i);
}

// read a word section in mode md at body byte off (body bytes in total):
// lane g gets the word of group g; returns the section's size, or sets bad
__device__ __forceinline__ uint32_t read_section(const uint32_t *b32, uint32_t mw, uint32_t off, uint32_t body,
                                                 int md, int G, uint32_t lanes, uint32_t &v, bool &bad) {
    const int lane = threadIdx.x & 31;
    v = 0u;
    if (md == S_CLEAR) return 0u;
    if (md == S_SET) { v = lane < G ? lanes : 0u; return 0u; }
    if (md == S_WORDS) {
        if (off + 4u * (uint32_t)G > body) { bad = true; return 0u; }
        v = body_word(b32, mw, (off >> 2) + (uint32_t)lane, lane < G);
        return 4u * (uint32_t)G;
    }
    if (md > S_WORDS || off + 4u > body) { bad = true; return 0u; }
    const uint32_t gm = G == 32 ? FULL : ((1u << G) - 1u);
    const uint32_t bm = body_word(b32, mw, off >> 2, true) & gm;
    const uint32_t size = 4u + 4u * __popc(bm);
    if (off + size > body) { bad = true; return 0u; }
    const bool exc = lane < G && ((bm >> lane) & 1u);
    const uint32_t w = body_word(b32, mw, (off >> 2) + 1u + __popc(bm & lanes_below()), exc);
    if (lane < G) v = exc ? w : (md == S_EXC_SET ? lanes : 0u);
    return size;
}

// ---------------------------------------------------------------- polar mode
// POLAR tiles: every nonzero amplitude a = x + iy coded as its magnitude
// m = sqrt(fma(x, x, y*y)), quantised like a component with shift s - 2,
// and its angle in units of 2^-64 turn from a 30-step integer CORDIC,
// quantised with shift P = s + 8 to B = 56 - s bits.  Reconstruction:
// the CORDIC rotation (X, Y) of (2^59, 0) by the angle code, then
// a^ = (m^ (Xd r), m^ (Yd r)) with r = 1 / sqrt(fma(Xd, Xd, Yd*Yd)).  Used
// at a lossy level (8 <= s <= 52) only when every component is 0 or in
// [2^-400, 16), every reconstruction satisfies |a^ - a|^2 <= 2^(2(s-53))
// (1 - 2^-10) |a|^2, and the stream is shorter than the componentwise one.
// Codes run along the nonzero amplitudes: magnitudes by order-1 Lorenzo,
// angles by order-2 Lorenzo modulo 2^B from the anchor u0 and the first
// difference d1 (header bytes 26..31); the PACKED body layout with clear
// sign sections.

// round(2^64 atan(2^-k) / (2 pi)), written by configure_kernels
__constant__ unsigned long long c_polar_atan[POLAR_ITERS];

// fixed point of x with the larger component's biased exponent emax at 2^59
__device__ __forceinline__ long long polar_fix(double x, int emax) {
    const unsigned long long u = dbits(x);
    const int e = (int)((u >> 52) & 0x7FFull);
    const unsigned long long f = u & 0xFFFFFFFFFFFFFull;
    if (e == 0 && f == 0) return 0;
    const unsigned long long m = f | (1ull << 52);
    const int sh = 7 + e - emax;
    const unsigned long long v = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    return (u >> 63) ? -(long long)v : (long long)v;
}

// angle of (x, y) in units of 2^-64 turn (CORDIC vectoring)
__device__ __noinline__ unsigned long long polar_angle(double x, double y) {
    const int ex = (int)((dbits(x) >> 52) & 0x7FFull), ey = (int)((dbits(y) >> 52) & 0x7FFull);
    const int emax = ex > ey ? ex : ey;
    long long X = polar_fix(x, emax), Y = polar_fix(y, emax);
    unsigned long long th = 0;
    if (X < 0) { X = -X; Y = -Y; th = 1ull << 63; }
    for (int k = 0; k < POLAR_ITERS; ++k) {
        const long long dx = Y >> k, dy = X >> k;
        if (Y >= 0) { X += dx; Y -= dy; th += c_polar_atan[k]; }
        else { X -= dx; Y += dy; th -= c_polar_atan[k]; }
    }
    return th;
}

// a^ of magnitude code qm and angle code qa at shift s (CORDIC rotation)
__device__ __noinline__ void polar_recon(unsigned long long qm, unsigned long long qa, int s, double &re,
                                         double &im) {
    const unsigned long long th = qa << (s + 8);
    long long X = 1ll << 59, Y = 0;
    unsigned long long z = th;
    if (((th >> 62) + 1ull) & 2ull) { X = -X; z = th - (1ull << 63); }
    long long zz = (long long)z;
    for (int k = 0; k < POLAR_ITERS; ++k) {
        const long long dx = Y >> k, dy = X >> k;
        if (zz >= 0) { X -= dx; Y += dy; zz -= (long long)c_polar_atan[k]; }
        else { X += dx; Y -= dy; zz += (long long)c_polar_atan[k]; }
    }
    const double m = bitsd(qm << (s - 1));
    const double xd = __ll2double_rn(X), yd = __ll2double_rn(Y);
    const double r = __ddiv_rn(1.0, __dsqrt_rn(__fma_rn(xd, xd, __dmul_rn(yd, yd))));
    re = __dmul_rn(m, __dmul_rn(xd, r));
    im = __dmul_rn(m, __dmul_rn(yd, r));
}

__device__ __forceinline__ bool polar_comp_ok(double x) {
    const unsigned long long u = dbits(x);
    const unsigned e = (unsigned)((u >> 52) & 0x7FFull);
    return (u & MAG) == 0ull || (e >= 623u && e < 1027u);
}

// Codes of one amplitude at shift s; false when the amplitude rules the
// mode out.  nz: the amplitude is not zero.
__device__ __forceinline__ bool polar_codes(double x, double y, int s, bool &nz, unsigned long long &qm,
                                            unsigned long long &qa, unsigned long long &th, double &xr,
                                            double &xi) {
    nz = false;
    qm = qa = th = 0ull;
    xr = xi = 0.0;
    if (!polar_comp_ok(x) || !polar_comp_ok(y)) return false;
    if ((dbits(x) & MAG) == 0ull && (dbits(y) & MAG) == 0ull) return true;
    nz = true;
    const int P = s + 8, B = 64 - P;
    const double mm = __fma_rn(x, x, __dmul_rn(y, y));
    qm = quant(dbits(__dsqrt_rn(mm)), s - 1);
    th = polar_angle(x, y);
    qa = ((th + (1ull << (P - 1))) >> P) & ((1ull << B) - 1ull);
    polar_recon(qm, qa, s, xr, xi);
    const double dr = __dsub_rn(xr, x), di = __dsub_rn(xi, y);
    const double lim = ldexp(1.0 - 0x1p-10, 2 * (s - 53));
    return __fma_rn(dr, dr, __dmul_rn(di, di)) <= __dmul_rn(lim, mm);
}

// Sizing (WRITE false) or packing (WRITE true) pass of the POLAR mode over
// a tile at shift s.  Sizing: ok (every amplitude codable), dense (no zero
// amplitude), the anchors am / au, the first angle difference d1, hp0 and
// the basis differences D_b of the bitwise-linear predictor (lane b holds
// D_b for b < 5 in dl, lane b - 5 holds D_b for b >= 5 in dh), and in lane
// g the zero word and the residual widths of group g (w0 magnitudes, w1
// angles by order 2, w1b angles bitwise).  Packing: writes the residuals
// of group g at data + o0 (magnitudes) and data + o1 (angles of the
// predictor `bitwise`), the word offsets held in lane g, and adds the
// reconstructed values' norm.
struct PolarInfo {
    unsigned long long am, au, d1, hp0, dl, dh;
    uint32_t zw, w0, w1, w1b;
    bool ok, dense;
};

template <bool WRITE>
__device__ __noinline__ void polar_pass(const double *re, const double *im, int s, int c, int G, int L,
                                        PolarInfo &pi, bool bitwise, uint32_t *data, uint32_t o0, uint32_t o1,
                                        uint32_t *wstage, unsigned long long &nlo, unsigned long long &nhi,
                                        unsigned &rng) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = lanes_below();
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);
    const int B = 56 - s, P = s + 8, BE = B + POLAR_EXTRA;
    const unsigned long long bmask = (1ull << B) - 1ull, half = 1ull << (B - 1), emask = (1ull << BE) - 1ull;
    unsigned long long lastm = 0, last1 = 0, last2 = 0;
    uint32_t seen = 0;
    unsigned long long lowsum = 0;                   // this lane's sum of D_b over its lane bits
    if (!WRITE) {
        pi.am = pi.au = pi.d1 = pi.hp0 = pi.dl = pi.dh = 0;
        pi.zw = pi.w0 = pi.w1 = pi.w1b = 0;
        pi.ok = true;
        pi.dense = true;
    }
    for (int g = 0; g < G; ++g) {
        const int i = g * 32 + lane;
        const double x = lane < L ? re[i] : 0.0, y = lane < L ? im[i] : 0.0;
        bool nz;
        unsigned long long qm, qa, th = 0;
        double xr, xi;
        const bool okv = lane < L ? polar_codes(x, y, s, nz, qm, qa, th, xr, xi)
                                  : (nz = false, qm = qa = 0, xr = xi = 0.0, true);
        if (!WRITE && !__all_sync(FULL, okv)) { pi.ok = false; return; }
        const uint32_t nzm = __ballot_sync(FULL, nz);
        if (!WRITE) {
            if (lane == g) pi.zw = ~nzm & lanes;
            if (nzm != lanes) pi.dense = false;
        }
        // the bitwise-linear predictor's angle at B + 8 bits and its basis
        const unsigned long long hp = ((th + (1ull << (P - POLAR_EXTRA - 1))) >> (P - POLAR_EXTRA)) & emask;
        if (!WRITE) {
            if (g == 0) {
                pi.hp0 = shfl64(hp, 0);
                const unsigned long long hb = shfl64(hp, (1 << (lane & 7)) & 31);    // lane b < 5: hp(2^b)
                if (lane < 5 && lane < c) pi.dl = (hb - pi.hp0) & emask;
            }
            if (g > 0 && (g & (g - 1)) == 0) {       // group 2^(b-5): lane 0 is index 2^b
                const int b = 5 + (31 - __clz(g));
                const unsigned long long v = (shfl64(hp, 0) - pi.hp0) & emask;
                if (lane == b - 5) pi.dh = v;
            }
        }
        if (g == 0) {
            lowsum = 0;
            for (int b = 0; b < 5 && b < c; ++b) {
                const unsigned long long db = shfl64(pi.dl, b);
                if ((lane >> b) & 1) lowsum += db;
            }
        }
        unsigned long long gsum = 0;                 // sum of D_b over the set bits of g
        for (int b = 5; b < c; ++b) {
            const unsigned long long db = shfl64(pi.dh, b - 5);
            if ((g >> (b - 5)) & 1) gsum += db;
        }
        const unsigned long long pp = (pi.hp0 + lowsum + gsum + (1ull << (POLAR_EXTRA - 1))) & emask;
        const unsigned long long rb = (qa - (pp >> POLAR_EXTRA)) & bmask;
        const long long rbs = (long long)((rb ^ half) - half);
        const unsigned long long zb = nz ? (((unsigned long long)rbs << 1) ^ (unsigned long long)(rbs >> 63)) : 0ull;
        if (nzm == 0u) continue;
        const uint32_t pm = nzm & below;
        const int p1 = pm ? 31 - __clz(pm) : lane;
        const uint32_t pm2 = pm & ~(1u << (p1 & 31));
        const int p2 = pm2 ? 31 - __clz(pm2) : lane;
        const unsigned long long m1 = shfl64(qm, p1), a1 = shfl64(qa, p1), a2 = shfl64(qa, p2);
        const uint32_t rank = (uint32_t)__popc(pm), cnt = (uint32_t)__popc(nzm);
        const unsigned long long prevm = pm ? m1 : (seen ? lastm : qm);
        const unsigned long long prev1 = pm ? a1 : last1;
        const unsigned long long prev2 = pm2 ? a2 : (pm ? last1 : last2);
        const unsigned long long ra = (seen + rank >= 2u) ? ((qa - 2ull * prev1 + prev2) & bmask) : 0ull;
        const long long rs = (long long)((ra ^ half) - half);
        const bool nzl = nz;
        const unsigned long long zm = nzl ? zigzag(qm - prevm) : 0ull;
        const unsigned long long za = nzl ? (((unsigned long long)rs << 1) ^ (unsigned long long)(rs >> 63)) : 0ull;
        const int f0 = __ffs(nzm) - 1;
        if (!WRITE) {
            if (seen == 0u) { pi.am = shfl64(qm, f0); pi.au = shfl64(qa, f0); }
            if (seen < 2u && seen + cnt >= 2u) {
                // the second nonzero amplitude of the tile and its predecessor
                const int l1 = seen == 1u ? f0 : __ffs(nzm & ~(1u << f0)) - 1;
                const unsigned long long u1 = shfl64(qa, l1);
                pi.d1 = (u1 - (seen == 1u ? last1 : shfl64(qa, f0))) & bmask;
            }
            const uint32_t w0 = (uint32_t)bitlen64(warp_or64(zm)), w1 = (uint32_t)bitlen64(warp_or64(za));
            const uint32_t w1b = (uint32_t)bitlen64(warp_or64(zb));
            if (lane == g) { pi.w0 = w0; pi.w1 = w1; pi.w1b = w1b; }
        } else {
            if (nzl) {
                unsigned long long l0, h0, l1v, h1v;
                sq_units(dbits(xr) & MAG, l0, h0, rng);
                sq_units(dbits(xi) & MAG, l1v, h1v, rng);
                add128(l0, h0, l1v, h1v);
                add128(nlo, nhi, l0, h0);
            }
            for (int k = 0; k < 2; ++k) {
                const uint32_t w = __shfl_sync(FULL, k ? (bitwise ? pi.w1b : pi.w1) : pi.w0, g);
                if (w == 0) continue;
                const uint32_t wo = __shfl_sync(FULL, k ? o1 : o0, g);
                const uint32_t nwd = (cnt * w + 31u) >> 5;
                const unsigned long long z = k ? (bitwise ? zb : za) : zm;
                wstage[lane] = 0u;
                wstage[lane + 32] = 0u;
                __syncwarp();
                if (nzl) {
                    const uint32_t bo = rank * w, j0 = bo >> 5, sh = bo & 31u;
                    atomicOr(&wstage[j0], (uint32_t)(z << sh));
                    if (sh + w > 32) atomicOr(&wstage[j0 + 1], (uint32_t)(z >> (32 - sh)));
                    if (sh + w > 64) atomicOr(&wstage[j0 + 2], (uint32_t)(z >> (64 - sh)));
                }
                __syncwarp();
                if ((uint32_t)lane < nwd) data[wo + lane] = wstage[lane];
                if ((uint32_t)lane + 32 < nwd) data[wo + lane + 32] = wstage[lane + 32];
                __syncwarp();
            }
        }
        const int lastl = 31 - __clz(nzm);
        const unsigned long long ql = shfl64(qm, lastl), al = shfl64(qa, lastl);
        const uint32_t pml = nzm & ~(1u << lastl);
        const unsigned long long al2 = shfl64(qa, pml ? 31 - __clz(pml) : lastl);
        last2 = cnt >= 2u ? al2 : last1;
        last1 = al;
        lastm = ql;
        seen += cnt;
    }
}

// Words of the bitwise predictor's basis section: c differences of B + 8 bits.
__device__ __forceinline__ uint32_t polar_basis_words(int c, int s) {
    return ((uint32_t)c * (uint32_t)(56 - s + POLAR_EXTRA) + 31u) >> 5;
}

// Write the basis section (D_b at bits [b (B+8), (b+1) (B+8))) at sec.
__device__ void polar_write_basis(const PolarInfo &pi, int c, int s, uint32_t *sec, uint32_t *wstage) {
    const int lane = threadIdx.x & 31;
    const int BE = 56 - s + POLAR_EXTRA;
    const uint32_t nb = polar_basis_words(c, s);
    const unsigned long long dhs = shfl64(pi.dh, (lane - 5) & 31);
    const unsigned long long d = lane < 5 ? pi.dl : dhs;
    wstage[lane] = 0u;
    __syncwarp();
    if (lane < c) {
        const uint32_t bo = (uint32_t)lane * (uint32_t)BE, j0 = bo >> 5, sh = bo & 31u;
        atomicOr(&wstage[j0], (uint32_t)(d << sh));
        if (sh + BE > 32) atomicOr(&wstage[j0 + 1], (uint32_t)(d >> (32 - sh)));
        if (sh + BE > 64) atomicOr(&wstage[j0 + 2], (uint32_t)(d >> (64 - sh)));
    }
    __syncwarp();
    if ((uint32_t)lane < nb) sec[lane] = wstage[lane];
    __syncwarp();
}

// Body bytes of a POLAR stream from its sizing pass (warp-uniform): the
// order-2 stream, and when the tile is dense the bitwise stream if shorter
// (*bitwise set).
__device__ __forceinline__ uint32_t polar_body(const PolarInfo &pi, int c, int s, int G, uint32_t lanes, int &zmode,
                                               bool &bitwise) {
    const int lane = threadIdx.x & 31;
    uint32_t zb;
    zmode = section_mode(pi.zw, G, lanes, zb);
    const uint32_t nn = lane < G ? (uint32_t)__popc(~pi.zw & lanes) : 0u;
    const uint32_t wm = __reduce_add_sync(FULL, (nn * pi.w0 + 31u) >> 5);
    const uint32_t w2 = __reduce_add_sync(FULL, (nn * pi.w1 + 31u) >> 5);
    const uint32_t wbw = __reduce_add_sync(FULL, (nn * pi.w1b + 31u) >> 5);
    const uint32_t head = 2u * zb + ((2u * (uint32_t)G + 3u) & ~3u);
    const uint32_t b2 = (head + 4u * (wm + w2) + 15u) & ~15u;
    bitwise = false;
    if (!pi.dense) return b2;
    const uint32_t bb = (head + 4u * (polar_basis_words(c, s) + wm + wbw) + 15u) & ~15u;
    if (bb < b2) { bitwise = true; return bb; }
    return b2;
}

// Decode one stream into planar re/im (2^c values each), multiplied by
// alpha when `scale` (Algorithm 2's normalize, fused).  Warp-wide; returns
// nonzero (and zero-fills) on a malformed stream.  The first 128 body bytes
// (sections and widths, usually) come in with one load, and the packed
// words of the next group are loaded while the current one is scanned.
// sp != nullptr: a stream of one amplitude (at most one nonzero code per
// component, at a common index, every residual zero, and every zero
// decoding to +0) is decoded into that amplitude alone: its value is
// written at its index p, the other entries are left unwritten, *sp = p
// and the result is 2.
template <bool POLAR>
__device__ __forceinline__ int wdecode_impl(const uint8_t *src, int c, double *re, double *im, double alpha,
                                            bool scale, int *sp) {
    const int N = 1 << c;
    const int G = N >= 32 ? N >> 5 : 1;
    const int L = N >= 32 ? 32 : N;
    const int lane = threadIdx.x & 31;
    const uint32_t hw = lane < 8 ? __ldg(reinterpret_cast<const uint32_t *>(src) + lane) : 0u;
    const uint32_t h0 = __shfl_sync(FULL, hw, 0), body = __shfl_sync(FULL, hw, 1);
    const unsigned long long a0 = ((unsigned long long)__shfl_sync(FULL, hw, 3) << 32) | __shfl_sync(FULL, hw, 2);
    const unsigned long long a1 = ((unsigned long long)__shfl_sync(FULL, hw, 5) << 32) | __shfl_sync(FULL, hw, 4);
    const uint32_t h6 = __shfl_sync(FULL, hw, 6), h7 = __shfl_sync(FULL, hw, 7);
    const int hc = h6 & 0xFF;
    const int mode = h0 & 0xFF, s = (h0 >> 8) & 0xFF;
    const int sm0 = (h0 >> 24) & 7, sm1 = (h0 >> 27) & 7;
    const int zm0 = (h6 >> 8) & 7, zm1 = (h6 >> 11) & 7;
    const uint8_t *b = src + HDR;
    const uint32_t *b32 = reinterpret_cast<const uint32_t *>(b);
    const bool polar = POLAR && (mode == M_POLAR || mode == M_POLAR_B), pbit = POLAR && mode == M_POLAR_B;
    bool bad = hc != c || mode > (POLAR ? 4 : 2) || (mode != M_RAW && s > 52) || (body & 15u);
    if (!bad && polar) bad = s < 8 || sm0 != S_CLEAR || sm1 != S_CLEAR;
    if (!bad && pbit) bad = zm0 != S_CLEAR || zm1 != S_CLEAR;             // no zero amplitude
    if (!bad && mode == M_RAW) bad = body != 16u * (uint32_t)N;
    if (!bad && mode == M_CONST) bad = body != 0 || sm0 > 1 || sm1 > 1 || ((h6 >> 8) & 0xFFu);
    if (!bad && mode == M_CONST) {
        double v0 = bitsd((a0 << s) | ((unsigned long long)sm0 << 63));
        double v1 = bitsd((a1 << s) | ((unsigned long long)sm1 << 63));
        if (scale) { v0 = __dmul_rn(v0, alpha); v1 = __dmul_rn(v1, alpha); }
        for (int i = lane; i < N; i += 32) { re[i] = v0; im[i] = v1; }
        return 0;
    }
    if (!bad && mode == M_RAW) {
        const double2 *v = reinterpret_cast<const double2 *>(b);
        for (int i = lane; i < N; i += 32) {
            double2 x = __ldg(v + i);
            if (scale) { x.x = __dmul_rn(x.x, alpha); x.y = __dmul_rn(x.y, alpha); }
            re[i] = x.x;
            im[i] = x.y;
        }
        return 0;
    }
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);
    uint32_t sw0 = 0, sw1 = 0, zw0 = 0, zw1 = 0, w0 = 0, w1 = 0, doff = 0, off0 = 0, off1 = 0, boff = 0, wmax = 0;
    if (!bad) {
        const uint32_t mw = 4u * (uint32_t)lane < body ? __ldg(b32 + lane) : 0u;
        uint32_t off = 0;
        off += read_section(b32, mw, off, body, sm0, G, lanes, sw0, bad);
        if (!bad) off += read_section(b32, mw, off, body, sm1, G, lanes, sw1, bad);
        if (!bad) off += read_section(b32, mw, off, body, zm0, G, lanes, zw0, bad);
        if (!bad) off += read_section(b32, mw, off, body, zm1, G, lanes, zw1, bad);
        if (!bad && off + 2u * G > body) bad = true;
        if (!bad) {
            // width bytes off + g (re) and off + G + g (im)
            const uint32_t i0 = off + (uint32_t)lane, i1 = off + (uint32_t)G + (uint32_t)lane;
            const uint32_t x0 = body_word(b32, mw, i0 >> 2, lane < G);
            const uint32_t x1 = body_word(b32, mw, i1 >> 2, lane < G);
            if (lane < G) {
                w0 = (x0 >> (8u * (i0 & 3u))) & 0xFFu;
                w1 = (x1 >> (8u * (i1 & 3u))) & 0xFFu;
            }
            uint32_t tot0, tot1;
            off0 = warp_exscan(((uint32_t)__popc(~zw0 & lanes) * w0 + 31u) >> 5, tot0);
            off1 = warp_exscan(((uint32_t)__popc(~zw1 & lanes) * w1 + 31u) >> 5, tot1) + tot0;
            doff = (off + 2u * G + 3u) & ~3u;
            if (pbit) {
                // the basis section precedes the residual words
                boff = doff;
                doff += 4u * polar_basis_words(c, s);
            }
            wmax = __reduce_max_sync(FULL, max(w0, w1));
            bad = wmax > 64 || (unsigned long long)doff + 4ull * (tot0 + tot1) > body;
            // POLAR: a zero amplitude is zero in both code streams
            if (!bad && polar) bad = __any_sync(FULL, lane < G && zw0 != zw1);
        }
    }
    if (bad) {
        for (int i = lane; i < N; i += 32) { re[i] = 0.0; im[i] = 0.0; }
        return 1;
    }
    if (!POLAR && sp != nullptr && mode == M_PACKED && wmax == 0u && L == 32) {
        // every residual zero: a nonzero code of component k is its anchor
        const uint32_t nz0 = lane < G ? ~zw0 : 0u, nz1 = lane < G ? ~zw1 : 0u;
        const uint32_t n0 = __reduce_add_sync(FULL, (uint32_t)__popc(nz0));
        const uint32_t n1 = __reduce_add_sync(FULL, (uint32_t)__popc(nz1));
        const uint32_t zsg = __reduce_or_sync(FULL, lane < G ? ((sw0 & zw0) | (sw1 & zw1)) : 0u);
        const double zs = scale ? __dmul_rn(0.0, alpha) : 0.0;
        if (n0 <= 1u && n1 <= 1u && n0 + n1 >= 1u && zsg == 0u && dbits(zs) == 0ull) {
            const uint32_t gb0 = __ballot_sync(FULL, nz0 != 0u), gb1 = __ballot_sync(FULL, nz1 != 0u);
            const int g0 = gb0 ? __ffs(gb0) - 1 : 0, g1 = gb1 ? __ffs(gb1) - 1 : 0;
            const uint32_t m0 = __shfl_sync(FULL, nz0, g0), m1 = __shfl_sync(FULL, nz1, g1);
            const int p0 = n0 ? g0 * 32 + __ffs(m0) - 1 : -1, p1 = n1 ? g1 * 32 + __ffs(m1) - 1 : -1;
            const int p = n0 ? p0 : p1;
            const uint32_t sg0 = (__shfl_sync(FULL, sw0, p >> 5) >> (p & 31)) & 1u;
            const uint32_t sg1 = (__shfl_sync(FULL, sw1, p >> 5) >> (p & 31)) & 1u;
            // the full decode's value at p (a zero component: +0, its sign clear)
            auto value = [&](uint32_t n, unsigned long long q, uint32_t sg) {
                double x;
                if (!n) x = 0.0;
                else if (s >= 32) x = __hiloint2double((int)(((uint32_t)q << (s - 32)) | (sg << 31)), 0);
                else x = bitsd((q << s) | ((unsigned long long)sg << 63));
                return scale ? __dmul_rn(x, alpha) : x;
            };
            const double x0 = value(n0, a0, sg0), x1 = value(n1, a1, sg1);
            if (!(n0 && n1 && p0 != p1) && (dbits(x0) | dbits(x1)) != 0ull) {
                if (lane == 0) { re[p] = x0; im[p] = x1; }
                *sp = p;
                return 2;
            }
        }
    }
    const uint32_t *data = reinterpret_cast<const uint32_t *>(b + doff);
    const uint32_t below = lanes_below();
    // group t = k * G + g (component k, group g): uniform metadata, then
    // this lane's packed words
    auto meta = [&](int t, uint32_t &w, uint32_t &wo, uint32_t &sgw, uint32_t &nzw) {
        const bool k = t >= G;
        const int g = k ? t - G : t;
        w = __shfl_sync(FULL, k ? w1 : w0, g);
        wo = __shfl_sync(FULL, k ? off1 : off0, g);
        sgw = __shfl_sync(FULL, k ? sw1 : sw0, g);
        nzw = ~__shfl_sync(FULL, k ? zw1 : zw0, g) & lanes;
    };
    auto fetch = [&](uint32_t w, uint32_t wo, uint32_t nzw, uint32_t &x0, uint32_t &x1, uint32_t &x2,
                     uint32_t &sh) {
        x0 = x1 = x2 = sh = 0u;
        if (((nzw >> lane) & 1u) && w) {
            const bool dense = nzw == lanes;
            const uint32_t nwd = ((dense ? (uint32_t)L : (uint32_t)__popc(nzw)) * w + 31u) >> 5;
            const uint32_t rank = dense ? (uint32_t)lane : (uint32_t)__popc(nzw & below);
            const uint32_t bo = rank * w, j0 = bo >> 5;
            const uint32_t *base = data + wo;
            sh = bo & 31u;
            x0 = __ldg(base + j0);
            x1 = j0 + 1 < nwd && sh + w > 32u ? __ldg(base + j0 + 1) : 0u;
            x2 = j0 + 2 < nwd && sh + w > 64u ? __ldg(base + j0 + 2) : 0u;
        }
    };
    const int T = 2 * G;
    uint32_t w, wo, sgw, nzw, x0, x1, x2, sh;
    meta(0, w, wo, sgw, nzw);
    fetch(w, wo, nzw, x0, x1, x2, sh);
    unsigned long long carry = a0;
    // POLAR: magnitudes (component 0) are the codes with shift s - 1, kept
    // unscaled in re until the angles (component 1) reconstruct the values
    const int sv = polar ? s - 1 : s;
    const unsigned long long bmask = polar ? (1ull << (56 - s)) - 1ull : 0ull;
    const unsigned long long d1 = ((unsigned long long)h7 << 16) | (h6 >> 16);
    unsigned long long cu = 0, cd = 0;                       // angle carries: last code, last difference
    uint32_t seen = 0;                                       // nonzero amplitudes before this group
    // bitwise-linear predictor: lane b < c holds D_b; lowsum = sum of D_b
    // over this lane's set bits (b < 5)
    unsigned long long dbase = 0, lowsum = 0;
    const int BE = 56 - s + POLAR_EXTRA;
    const unsigned long long emask = pbit ? (1ull << BE) - 1ull : 0ull;
    if (pbit) {
        const uint32_t bo = (uint32_t)lane * (uint32_t)BE, j0 = bo >> 5, shb = bo & 31u;
        const uint32_t *bw = reinterpret_cast<const uint32_t *>(b + boff);
        const uint32_t nb = polar_basis_words(c, s);
        if (lane < c) {
            const unsigned long long lo = (unsigned long long)__ldg(bw + j0) |
                                          (j0 + 1 < nb ? (unsigned long long)__ldg(bw + j0 + 1) << 32 : 0ull);
            const unsigned long long hi = j0 + 2 < nb ? (unsigned long long)__ldg(bw + j0 + 2) : 0ull;
            dbase = ((lo >> shb) | (shb ? hi << (64 - shb) : 0ull)) & emask;
        }
        for (int bb = 0; bb < 5 && bb < c; ++bb) {
            const unsigned long long db = shfl64(dbase, bb);
            if ((lane >> bb) & 1) lowsum += db;
        }
    }
    for (int t = 0; t < T; ++t) {
        uint32_t wn = 0, won = 0, sgwn = 0, nzwn = 0, y0 = 0, y1 = 0, y2 = 0, shn = 0;
        if (t + 1 < T) {                                     // next group's words, in flight meanwhile
            meta(t + 1, wn, won, sgwn, nzwn);
            fetch(wn, won, nzwn, y0, y1, y2, shn);
        }
        const bool k = t >= G;
        const int g = k ? t - G : t;
        if (t == G) {
            carry = a1;
            cu = (a1 - d1) & bmask;
            cd = d1 & bmask;
        }
        double *v = k ? im : re;
        if (nzw == 0u) {                                     // all zeros: signs only
            if (lane < L) {
                double x = bitsd((unsigned long long)((sgw >> lane) & 1u) << 63);
                if (scale && !polar) x = __dmul_rn(x, alpha);
                v[g * 32 + lane] = x;
            }
        } else if (pbit && k) {
            // angles: the bitwise-linear prediction plus the residual
            unsigned long long z = 0;
            if (w) {
                if (w <= 32) {
                    const uint32_t z32 = __funnelshift_r(x0, x1, sh);
                    z = w == 32 ? z32 : (z32 & ((1u << w) - 1u));
                } else {
                    const unsigned long long lo = (unsigned long long)x0 | ((unsigned long long)x1 << 32);
                    const unsigned long long vv = sh ? ((lo >> sh) | ((unsigned long long)x2 << (64 - sh))) : lo;
                    z = w == 64 ? vv : (vv & ((1ull << w) - 1ull));
                }
            }
            unsigned long long gsum = 0;
            for (int bb = 5; bb < c; ++bb) {
                const unsigned long long db = shfl64(dbase, bb);
                if ((g >> (bb - 5)) & 1) gsum += db;
            }
            if (lane < L) {
                const unsigned long long pp = (a1 + lowsum + gsum + (1ull << (POLAR_EXTRA - 1))) & emask;
                const unsigned long long u = ((pp >> POLAR_EXTRA) + unzigzag(z)) & bmask;
                const unsigned long long qm = dbits(re[g * 32 + lane]) >> sv;
                double ar, ai;
                polar_recon(qm, u, s, ar, ai);
                if (scale) { ar = __dmul_rn(ar, alpha); ai = __dmul_rn(ai, alpha); }
                re[g * 32 + lane] = ar;
                im[g * 32 + lane] = ai;
            }
        } else if (polar && k) {
            // angles: second-order running sums modulo 2^B, the first two
            // nonzero amplitudes of the tile taking no residual
            const bool nzl = (nzw >> lane) & 1u;
            unsigned long long z = 0;
            if (nzl && w) {
                if (w <= 32) {
                    const uint32_t z32 = __funnelshift_r(x0, x1, sh);
                    z = w == 32 ? z32 : (z32 & ((1u << w) - 1u));
                } else {
                    const unsigned long long lo = (unsigned long long)x0 | ((unsigned long long)x1 << 32);
                    const unsigned long long vv = sh ? ((lo >> sh) | ((unsigned long long)x2 << (64 - sh))) : lo;
                    z = w == 64 ? vv : (vv & ((1ull << w) - 1ull));
                }
            }
            const uint32_t rank = (uint32_t)__popc(nzw & below);
            const unsigned long long rr = (nzl && seen + rank >= 2u) ? (unzigzag(z) & bmask) : 0ull;
            unsigned long long s1 = rr;
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long o = shfl_up64(s1, d);
                if (lane >= d) s1 += o;
            }
            unsigned long long s2 = nzl ? cd + s1 : 0ull;
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long o = shfl_up64(s2, d);
                if (lane >= d) s2 += o;
            }
            if (lane < L) {
                double ar = 0.0, ai = 0.0;
                if (nzl) {
                    const unsigned long long qm = dbits(re[g * 32 + lane]) >> sv;
                    polar_recon(qm, (cu + s2) & bmask, s, ar, ai);
                    if (scale) { ar = __dmul_rn(ar, alpha); ai = __dmul_rn(ai, alpha); }
                }
                re[g * 32 + lane] = ar;
                im[g * 32 + lane] = ai;
            }
            cd = (cd + shfl64(s1, 31)) & bmask;
            cu = (cu + shfl64(s2, 31)) & bmask;
            seen += (uint32_t)__popc(nzw);
        } else {
            const bool nzl = (nzw >> lane) & 1u;
            unsigned long long z = 0;
            if (nzl && w) {
                if (w <= 32) {                               // at most two words
                    const uint32_t z32 = __funnelshift_r(x0, x1, sh);
                    z = w == 32 ? z32 : (z32 & ((1u << w) - 1u));
                } else {
                    const unsigned long long lo = (unsigned long long)x0 | ((unsigned long long)x1 << 32);
                    const unsigned long long vv = sh ? ((lo >> sh) | ((unsigned long long)x2 << (64 - sh))) : lo;
                    z = w == 64 ? vv : (vv & ((1ull << w) - 1ull));
                }
            }
            const unsigned long long r = unzigzag(z);        // 0 for zeros and lanes >= L
            unsigned long long inc;
            if (w == 0) {                                    // every residual 0
                inc = 0;
            } else if (w <= 27) {                            // 32 partial sums of |r| < 2^26 fit in int32
                const uint32_t z32 = (uint32_t)z;
                int v32 = (int)((z32 >> 1) ^ (0u - (z32 & 1u)));
                for (int d = 1; d < 32; d <<= 1) {
                    int o = __shfl_up_sync(FULL, v32, d);
                    if (lane >= d) v32 += o;
                }
                inc = (unsigned long long)(long long)v32;
            } else {
                inc = r;
                for (int d = 1; d < 32; d <<= 1) {
                    unsigned long long o = shfl_up64(inc, d);
                    if (lane >= d) inc += o;
                }
            }
            const unsigned long long q = carry + inc;
            if (lane < L) {
                double x;
                if (sv >= 32) {                              // (q << sv) has a zero low word
                    const uint32_t hw = (nzl ? (uint32_t)q << (sv - 32) : 0u) | (((sgw >> lane) & 1u) << 31);
                    x = __hiloint2double((int)hw, 0);
                } else {
                    const unsigned long long sg = (unsigned long long)((sgw >> lane) & 1u) << 63;
                    x = bitsd(nzl ? ((q << sv) | sg) : sg);
                }
                if (scale && !polar) x = __dmul_rn(x, alpha);
                v[g * 32 + lane] = x;
            }
            carry = shfl64(q, L - 1);
        }
        w = wn; wo = won; sgw = sgwn; nzw = nzwn;
        x0 = y0; x1 = y1; x2 = y2; sh = shn;
    }
    return 0;
}

// Decode one stream (warp-wide): POLAR streams through their own function,
// so that the componentwise decoder keeps its registers.
__device__ __noinline__ int wdecode_polar(const uint8_t *src, int c, double *re, double *im, double alpha,
                                          bool scale) {
    return wdecode_impl<true>(src, c, re, im, alpha, scale, nullptr);
}

__device__ __forceinline__ int wdecode(const uint8_t *src, int c, double *re, double *im, double alpha,
                                       bool scale) {
    const uint32_t h0 = __ldg(reinterpret_cast<const uint32_t *>(src));
    if ((h0 & 0xFFu) >= (uint32_t)M_POLAR) return wdecode_polar(src, c, re, im, alpha, scale);
    return wdecode_impl<false>(src, c, re, im, alpha, scale, nullptr);
}

// wdecode, with a stream of one amplitude decoded as that amplitude alone
// (see wdecode_impl): 2 + its index p, the tile's other entries
// unwritten; else wdecode's result.  Its own function, so that the
// decoder of the other sweeps keeps its registers.  Warp-wide.
__device__ __noinline__ int wdecode_one(const uint8_t *src, int c, double *re, double *im, double alpha,
                                        bool scale) {
    const uint32_t h0 = __ldg(reinterpret_cast<const uint32_t *>(src));
    if ((h0 & 0xFFu) >= (uint32_t)M_POLAR) return wdecode_polar(src, c, re, im, alpha, scale);
    int p = 0;
    const int r = wdecode_impl<false>(src, c, re, im, alpha, scale, &p);
    return r == 2 ? 2 + p : r;
}

struct EncodeOut {
    unsigned long long off;
    bool ok;
};

// One pass over a tile: zero and sign words, the first nonzero magnitude,
// and group widths at every ladder level.
struct LevelSizes {
    unsigned long long wl0, wl1;      // lane g: width of group g per level (byte lv)
    uint32_t nz;                      // bit lv: some residual nonzero at level lv
    uint32_t sw0, sw1;                // lane g: sign words (every value)
    uint32_t zw0, zw1;                // lane g: zero words (bit l: magnitude 0)
    unsigned long long f0, f1;        // first nonzero magnitude bits (0 if none), warp-uniform
};

// Pass 1 of the encoder.  Residuals run along the nonzero values of a
// component: each against the previous nonzero code, the first against
// itself (the anchor).  A zero code only arises from a zero magnitude: any
// other value below the lossy range forces shift 0.  The predecessor's
// magnitude bits are found once per group; each level quantises both.
// force0: code every level with shift 0 (values outside the lossy range).
__device__ __forceinline__ void size_levels(const double *re, const double *im, const CodecCfg &cc,
                                            int G, int L, bool force0, LevelSizes &ls, int &nonfin,
                                            int &inel) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = lanes_below();
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);
    ls.wl0 = ls.wl1 = 0;
    ls.nz = 0;
    ls.sw0 = ls.sw1 = ls.zw0 = ls.zw1 = 0;
    ls.f0 = ls.f1 = 0;
    if (cc.nlev == 1 && !force0 && cc.shifts[0] >= 32) {
        // one lossy level at shift >= 32 (the common case): the same
        // quantities in 32-bit arithmetic on the high and low words
        const int s = cc.shifts[0];
        for (int k = 0; k < 2; ++k) {
            const double *v = k ? im : re;
            bool seen = false;
            uint32_t lastq = 0;
            unsigned long long first = 0, wl = 0;
            for (int g = 0; g < G; ++g) {
                const double x = lane < L ? v[g * 32 + lane] : 0.0;
                const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
                const uint32_t mh = hi & 0x7FFFFFFFu;
                const bool nzv = (mh | lo) != 0u;
                nonfin |= mh >= 0x7FF00000u;
                inel |= nzv && (mh < 0x00100000u || mh >= 0x7FE00000u);
                const uint32_t sw = __ballot_sync(FULL, hi >> 31);
                const uint32_t nzm = __ballot_sync(FULL, nzv);
                if (lane == g) {
                    if (k) { ls.sw1 = sw; ls.zw1 = ~nzm & lanes; }
                    else { ls.sw0 = sw; ls.zw0 = ~nzm & lanes; }
                }
                if (nzm == 0u) continue;
                const uint32_t q = quant_hi(mh, lo, s);
                uint32_t qp;
                if (nzm == lanes) {
                    const uint32_t up = __shfl_up_sync(FULL, q, 1);
                    qp = lane ? up : (seen ? lastq : q);
                } else {
                    const uint32_t pm = nzm & below;
                    const uint32_t qs = __shfl_sync(FULL, q, pm ? 31 - __clz(pm) : lane);
                    qp = pm ? qs : (seen ? lastq : q);
                }
                if (!seen) {
                    const int f = __ffs(nzm) - 1;
                    first = ((unsigned long long)__shfl_sync(FULL, mh, f) << 32) | __shfl_sync(FULL, lo, f);
                }
                const uint32_t r = q - qp;
                const uint32_t z = ((nzm >> lane) & 1u) ? (r << 1) ^ (uint32_t)((int)r >> 31) : 0u;
                const uint32_t oz = __reduce_or_sync(FULL, z);
                const uint32_t w = oz ? 32u - (uint32_t)__clz(oz) : 0u;
                if (w) ls.nz |= 1u;
                if (lane == g) wl = w;
                lastq = __shfl_sync(FULL, q, 31 - __clz(nzm));
                seen = true;
            }
            if (k) { ls.f1 = first; ls.wl1 = wl; } else { ls.f0 = first; ls.wl0 = wl; }
        }
        return;
    }
    for (int k = 0; k < 2; ++k) {
        const double *v = k ? im : re;
        bool seen = false;
        unsigned long long first = 0, lastB = 0, wl = 0;
        for (int g = 0; g < G; ++g) {
            const unsigned long long u = lane < L ? dbits(v[g * 32 + lane]) : 0ull;
            const unsigned long long B = u & MAG;
            nonfin |= lane < L && B >= INF_BITS;
            inel |= lane < L && B != 0 && (B < MIN_NORMAL || B >= LOSSY_LIMIT);
            const uint32_t sw = __ballot_sync(FULL, lane < L && (u >> 63));
            const uint32_t nzm = __ballot_sync(FULL, lane < L && B != 0);
            if (lane == g) {
                if (k) { ls.sw1 = sw; ls.zw1 = ~nzm & lanes; }
                else { ls.sw0 = sw; ls.zw0 = ~nzm & lanes; }
            }
            if (nzm == 0u) continue;                         // all zeros: width 0 at every level
            // magnitude bits of the previous nonzero value (uniform branch:
            // a group without zeros, the common case, takes the lane below)
            unsigned long long Bp;
            if (nzm == lanes) {
                const unsigned long long up = shfl_up64(B, 1);
                Bp = lane ? up : (seen ? lastB : B);
            } else {
                const uint32_t pm = nzm & below;             // nonzero lanes before this one
                const unsigned long long Bs = shfl64(B, pm ? 31 - __clz(pm) : lane);
                Bp = pm ? Bs : (seen ? lastB : B);
            }
            if (!seen && nzm) first = shfl64(B, __ffs(nzm) - 1);
            const bool nzl = (nzm >> lane) & 1u;
            unsigned long long wg = 0;
#pragma unroll
            for (int lv = 0; lv < MAX_LEVELS; ++lv) {
                if (lv >= cc.nlev) continue;
                const int s = force0 ? 0 : cc.shifts[lv];
                uint32_t w;
                if (s >= 32) {                               // codes < 2^31: 32-bit residuals
                    const uint32_t r = (uint32_t)quant(B, s) - (uint32_t)quant(Bp, s);
                    const uint32_t z = nzl ? (r << 1) ^ (uint32_t)((int)r >> 31) : 0u;
                    const uint32_t oz = __reduce_or_sync(FULL, z);
                    w = oz ? 32u - (uint32_t)__clz(oz) : 0u;
                } else {
                    const unsigned long long z = nzl ? zigzag(quant(B, s) - quant(Bp, s)) : 0ull;
                    const unsigned long long oz = warp_or64(z);
                    w = oz ? (uint32_t)bitlen64(oz) : 0u;
                }
                wg |= (unsigned long long)w << (8 * lv);
                if (w) ls.nz |= 1u << lv;
            }
            if (lane == g) wl = wg;
            if (nzm) lastB = shfl64(B, 31 - __clz(nzm));
            seen |= nzm != 0;
        }
        if (k) { ls.f1 = first; ls.wl1 = wl; } else { ls.f0 = first; ls.wl0 = wl; }
    }
}

// One pass over a tile for a single lossy level at shift s >= 32 (c >= 5,
// no value outside the lossy range): the sizes, sign and zero words and
// anchors of size_levels, the norm partial, and the packed words of every
// group, which are written over the group's own values in shared memory
// once all lanes have read them (at most 32 words, the first half of the
// group's 256 bytes).  Same quantities and words as size_levels followed
// by the packing pass.
__device__ void pack_onepass(double *re, double *im, int s, int G, LevelSizes &ls, unsigned long long &nlo,
                             unsigned long long &nhi, unsigned &rng, uint32_t *wstage) {
    const int lane = threadIdx.x & 31;
    const uint32_t below = lanes_below();
    ls.wl0 = ls.wl1 = 0;
    ls.nz = 0;
    ls.sw0 = ls.sw1 = ls.zw0 = ls.zw1 = 0;
    ls.f0 = ls.f1 = 0;
    for (int k = 0; k < 2; ++k) {
        double *v = k ? im : re;
        bool seen = false;
        uint32_t lastq = 0;
        unsigned long long first = 0, wl = 0;
        for (int g = 0; g < G; ++g) {
            const double x = v[g * 32 + lane];
            const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
            const uint32_t mh = hi & 0x7FFFFFFFu;
            const bool nzv = (mh | lo) != 0u;
            const uint32_t sw = __ballot_sync(FULL, hi >> 31);
            const uint32_t nzm = __ballot_sync(FULL, nzv);
            if (lane == g) {
                if (k) { ls.sw1 = sw; ls.zw1 = ~nzm; }
                else { ls.sw0 = sw; ls.zw0 = ~nzm; }
            }
            if (nzm == 0u) continue;
            const uint32_t q = nzv ? quant_hi(mh, lo, s) : 0u;
            const bool dense = nzm == FULL;
            uint32_t qp;
            if (dense) {
                const uint32_t up = __shfl_up_sync(FULL, q, 1);
                qp = lane ? up : (seen ? lastq : q);
            } else {
                const uint32_t pm = nzm & below;
                const uint32_t qs = __shfl_sync(FULL, q, pm ? 31 - __clz(pm) : lane);
                qp = pm ? qs : (seen ? lastq : q);
            }
            if (!seen) {
                const int f = __ffs(nzm) - 1;
                first = ((unsigned long long)__shfl_sync(FULL, mh, f) << 32) | __shfl_sync(FULL, lo, f);
            }
            const bool nzl = (nzm >> lane) & 1u;
            const uint32_t r = q - qp;
            const uint32_t z = nzl ? (r << 1) ^ (uint32_t)((int)r >> 31) : 0u;
            const uint32_t oz = __reduce_or_sync(FULL, z);
            const uint32_t w = oz ? 32u - (uint32_t)__clz(oz) : 0u;
            if (lane == g) wl = w;
            if (q) {
                unsigned long long l0, h0;
                sq_units_code(q, s, l0, h0, rng);
                add128(nlo, nhi, l0, h0);
            }
            if (w) {
                ls.nz = 1u;
                const uint32_t nwd = ((uint32_t)__popc(nzm) * w + 31u) >> 5;
                wstage[lane] = 0u;
                __syncwarp();
                if (nzl) {
                    const uint32_t rank = dense ? (uint32_t)lane : (uint32_t)__popc(nzm & below);
                    const uint32_t bo = rank * w, j0 = bo >> 5, sh = bo & 31u;
                    atomicOr(&wstage[j0], z << sh);
                    if (sh + w > 32) atomicOr(&wstage[j0 + 1], z >> (32 - sh));
                }
                __syncwarp();
                if ((uint32_t)lane < nwd) reinterpret_cast<uint32_t *>(v + g * 32)[lane] = wstage[lane];
                __syncwarp();
            }
            lastq = __shfl_sync(FULL, q, dense ? 31 : 31 - __clz(nzm));
            seen = true;
        }
        if (k) { ls.f1 = first; ls.wl1 = wl; } else { ls.f0 = first; ls.wl0 = wl; }
    }
}

// Section sizes and modes of a tile sized by size_levels (warp-uniform):
// zero words, sign words of every value (lossless) and of the nonzero
// values (lossy), width bytes, nonzero counts per group (lane g).
struct Sections {
    uint32_t zb0, zb1, sbl0, sbl1, sby0, sby1, wb, nn0, nn1;
    int zm0, zm1, sml0, sml1, smy0, smy1;
};

__device__ __forceinline__ void sections_of(const LevelSizes &ls, int G, uint32_t lanes, Sections &q) {
    const int lane = threadIdx.x & 31;
    q.zm0 = section_mode(ls.zw0, G, lanes, q.zb0);
    q.zm1 = section_mode(ls.zw1, G, lanes, q.zb1);
    q.sml0 = section_mode(ls.sw0, G, lanes, q.sbl0);
    q.sml1 = section_mode(ls.sw1, G, lanes, q.sbl1);
    q.smy0 = section_mode(ls.sw0 & ~ls.zw0, G, lanes, q.sby0);
    q.smy1 = section_mode(ls.sw1 & ~ls.zw1, G, lanes, q.sby1);
    q.wb = (2u * G + 3u) & ~3u;
    q.nn0 = lane < G ? (uint32_t)__popc(~ls.zw0 & lanes) : 0u;
    q.nn1 = lane < G ? (uint32_t)__popc(~ls.zw1 & lanes) : 0u;
}

// Mode and body bytes of the tile's stream at ladder level lv coded with
// shift slv (0 when the tile holds values outside the lossy range); s0, s1
// its sign modes.  Warp-wide: lv and slv are warp-uniform.
__device__ __forceinline__ uint32_t level_body(const LevelSizes &ls, const Sections &q, int lv, int slv,
                                               uint32_t raw_body, int &mode, int &s0, int &s1) {
    s0 = slv ? q.smy0 : q.sml0;
    s1 = slv ? q.smy1 : q.sml1;
    const uint32_t meta = (slv ? q.sby0 + q.sby1 : q.sbl0 + q.sbl1) + q.zb0 + q.zb1;
    if (!((ls.nz >> lv) & 1u) && s0 <= S_SET && s1 <= S_SET && q.zm0 <= S_SET && q.zm1 <= S_SET) {
        mode = M_CONST;
        return 0u;
    }
    const uint32_t w0 = (uint32_t)(ls.wl0 >> (8 * lv)) & 0xFFu, w1 = (uint32_t)(ls.wl1 >> (8 * lv)) & 0xFFu;
    const uint32_t words = __reduce_add_sync(FULL, ((q.nn0 * w0 + 31u) >> 5) + ((q.nn1 * w1 + 31u) >> 5));
    const uint32_t pb = (meta + q.wb + 4u * words + 15u) & ~15u;
    if (pb < raw_body) {
        mode = M_PACKED;
        return pb;
    }
    mode = M_RAW;
    return raw_body;
}

// Sizing pass of a per-stride ladder decision: the tile's stream size at
// every level, added to its stride's counts bytes[0 .. nlev-1].  Writes
// nothing else.  Warp-wide.
__device__ __noinline__ void wsize(const double *re, const double *im, const CodecCfg &cc,
                                   unsigned long long *bytes) {
    const int c = cc.c, N = 1 << c;
    const int G = N >= 32 ? N >> 5 : 1;
    const int L = N >= 32 ? 32 : N;
    const int lane = threadIdx.x & 31;
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);
    const uint32_t raw_body = 16u * (uint32_t)N;
    LevelSizes ls;
    int nonfin = 0, inel = 0;
    if (!cc.force_raw) {
        size_levels(re, im, cc, G, L, false, ls, nonfin, inel);
        nonfin = __any_sync(FULL, nonfin);
        inel = __any_sync(FULL, inel);
        if (inel && !nonfin) {
            int d0 = 0, d1 = 0;
            size_levels(re, im, cc, G, L, true, ls, d0, d1);
        }
    }
    const bool raw_only = cc.force_raw || nonfin;
    Sections q;
    if (!raw_only) sections_of(ls, G, lanes, q);
    for (int lv = 0; lv < cc.nlev; ++lv) {
        uint32_t body = raw_body;
        if (!raw_only) {
            int mode, s0, s1;
            const int slv = inel ? 0 : cc.shifts[lv];
            body = level_body(ls, q, lv, slv, raw_body, mode, s0, s1);
            if (cc.polar && !inel && slv >= 8 && slv <= 52) {
                unsigned long long d0 = 0, d1 = 0;
                unsigned dr = 0;
                PolarInfo pi;
                polar_pass<false>(re, im, slv, c, G, L, pi, false, nullptr, 0u, 0u, nullptr, d0, d1, dr);
                if (pi.ok) {
                    int pz;
                    bool bw;
                    const uint32_t pb = polar_body(pi, c, slv, G, lanes, pz, bw);
                    if (pb < body) body = pb;
                }
            }
        }
        if (lane == 0) atomicAdd(bytes + lv, (unsigned long long)(HDR + body));
    }
}

// The ladder of a tile with the POLAR variant on (a separate function so
// that the componentwise encoder keeps its registers): every level sized
// componentwise and in the POLAR mode, the shorter kept, the first level
// within the size limit (else the last, or force_lv) chosen.  When the
// chosen stream is a POLAR one it is written here (stream, table entry,
// norm, counters; *off = its offset, ~0 on overflow) and true returned;
// otherwise mode, level, bodyb and sm describe the componentwise stream
// for the caller to write.  Warp-wide.
__device__ __noinline__ bool polar_ladder(const double *re, const double *im, const CodecCfg &cc,
                                          const LevelSizes &ls, const Sections &q, uint32_t raw_body, int force_lv,
                                          unsigned long long tile, uint8_t *out_arena, unsigned long long out_cap,
                                          unsigned long long *out_table, unsigned long long *part,
                                          DevScalars *scal, unsigned sweep_id, uint32_t *wstage, int &mode,
                                          int &level, uint32_t &bodyb, int *sm, unsigned long long &off,
                                          PassAcc *acc) {
    const int c = cc.c, N = 1 << c;
    const int G = N >= 32 ? N >> 5 : 1;
    const int L = N >= 32 ? 32 : N;
    const int lane = threadIdx.x & 31;
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);
    PolarInfo pinfo{};
    int pz = 0;
    bool found = false;
    for (int lv = 0; lv < cc.nlev && !found; ++lv) {
        if (force_lv >= 0 && lv != force_lv) continue;
        const int slv = cc.shifts[lv];
        bodyb = level_body(ls, q, lv, slv, raw_body, mode, sm[0], sm[1]);
        if (slv >= 8 && slv <= 52) {
            unsigned long long d0 = 0, d1 = 0;
            unsigned dr = 0;
            PolarInfo pi;
            polar_pass<false>(re, im, slv, c, G, L, pi, false, nullptr, 0u, 0u, wstage, d0, d1, dr);
            if (pi.ok) {
                int z;
                bool bw;
                const uint32_t pb = polar_body(pi, c, slv, G, lanes, z, bw);
                if (pb < bodyb) {
                    mode = bw ? M_POLAR_B : M_POLAR;
                    bodyb = pb;
                    sm[0] = sm[1] = S_CLEAR;
                    pz = z;
                    pinfo = pi;
                }
            }
        }
        level = lv;
        found = force_lv >= 0 || (unsigned long long)(HDR + bodyb) <= cc.max_bytes;
    }
    if (mode != M_POLAR && mode != M_POLAR_B) return false;
    const int s = cc.shifts[level];
    const bool bw = mode == M_POLAR_B;
    const uint32_t size = HDR + bodyb;
    int ok = 0;
    off = 0;
    if (lane == 0) {
        off = atomicAdd(&scal->bump, (unsigned long long)size);
        ok = off + size <= out_cap;
        if (!ok) {
            atomicOr(&scal->err, ERR_OVERFLOW);
            atomicCAS(&scal->err_sweep, 0u, sweep_id + 1u);
        }
    }
    off = shfl64(off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    if (!ok) { off = ~0ull; return true; }
    uint8_t *dst = out_arena + off;
    const unsigned long long anc0 = pinfo.am, anc1 = bw ? pinfo.hp0 : pinfo.au;
    if (lane < 8) {
        uint32_t v = 0;
        switch (lane) {
            case 0: v = (uint32_t)mode | ((uint32_t)s << 8) | ((uint32_t)level << 16); break;
            case 1: v = bodyb; break;
            case 2: v = (uint32_t)anc0; break;
            case 3: v = (uint32_t)(anc0 >> 32); break;
            case 4: v = (uint32_t)anc1; break;
            case 5: v = (uint32_t)(anc1 >> 32); break;
            case 6:
                v = (uint32_t)c | ((uint32_t)(pz | (pz << 3)) << 8);
                if (!bw) v |= (uint32_t)(pinfo.d1 & 0xFFFFull) << 16;
                break;
            default: v = bw ? 0u : (uint32_t)(pinfo.d1 >> 16); break;
        }
        reinterpret_cast<uint32_t *>(dst)[lane] = v;
    }
    uint8_t *b = dst + HDR;
    // zero sections (sign sections clear), widths, [basis,] residual words
    const uint32_t wa = bw ? pinfo.w1b : pinfo.w1;
    uint32_t moff = 0, sz;
    write_section(reinterpret_cast<uint32_t *>(b), pz, pinfo.zw, G, lanes);
    moff += (section_mode(pinfo.zw, G, lanes, sz), sz);
    write_section(reinterpret_cast<uint32_t *>(b + moff), pz, pinfo.zw, G, lanes);
    moff += sz;
    const uint32_t nn = lane < G ? (uint32_t)__popc(~pinfo.zw & lanes) : 0u;
    uint32_t tot0, tot1;
    const uint32_t o0 = warp_exscan(lane < G ? (nn * pinfo.w0 + 31u) >> 5 : 0u, tot0);
    const uint32_t o1 = warp_exscan(lane < G ? (nn * wa + 31u) >> 5 : 0u, tot1) + tot0;
    const uint32_t wb = (2u * G + 3u) & ~3u;
    for (uint32_t base = 0; base < wb; base += 32) {          // uniform trip count
        const int t = (int)base + lane;
        const int src = t < G ? t : (t < 2 * G ? t - G : 0);
        const uint32_t a = __shfl_sync(FULL, pinfo.w0, src & 31);
        const uint32_t bb = __shfl_sync(FULL, wa, src & 31);
        if ((uint32_t)t < wb) b[moff + t] = (uint8_t)(t < G ? a : (t < 2 * G ? bb : 0u));
    }
    uint32_t doff = moff + wb;
    if (bw) {
        polar_write_basis(pinfo, c, s, reinterpret_cast<uint32_t *>(b + doff), wstage);
        doff += 4u * polar_basis_words(c, s);
    }
    unsigned long long nlo = 0, nhi = 0;
    unsigned rng = 0;
    polar_pass<true>(re, im, s, c, G, L, pinfo, bw, reinterpret_cast<uint32_t *>(b + doff), o0, o1, wstage,
                     nlo, nhi, rng);
    for (uint32_t p = doff + 4u * (tot0 + tot1) + lane; p < bodyb; p += 32) b[p] = 0;
    warp_sum128(nlo, nhi);
    rng = __any_sync(FULL, rng);
    if (lane == 0) {
        part[2 * tile] = nlo;
        part[2 * tile + 1] = nhi;
        tally_tile(acc, scal, nlo, nhi, level, (unsigned long long)size > cc.max_bytes);
        out_table[tile] = off;
        if (rng) atomicOr(&scal->err, ERR_RANGE);
    }
    __syncwarp();
    return true;
}

// Encode planar re/im (2^c values each) of tile `tile` into the output
// arena with Algorithm 2's ladder (every level sized in one pass), or at
// ladder level force_lv when it is >= 0 (the level of the tile's stride).
// Warp-wide.  Writes the stream, its table entry and norm partial, and adds
// to the running norm.  wstage: 64 words of shared memory of this warp.
// With one lossy level at shift >= 32 the tile is coded in one pass and
// its values in shared memory are overwritten.
// PT: the tile is +0 but for the amplitude (pvr, pvi) at index pp, which
// holds values that are zero or inside the lossy range (no uncompressed
// storage forced, c >= 5, componentwise codec); re and im are not read.
// The sizes, the stream and the norm are those of the full tile.
template <bool POLAR, bool PT = false>
__device__ __forceinline__ EncodeOut wencode_impl(double *re, double *im, const CodecCfg &cc,
                             unsigned long long tile, uint8_t *out_arena, unsigned long long out_cap,
                             unsigned long long *out_table, unsigned long long *part,
                             DevScalars *scal, unsigned sweep_id, uint32_t *wstage, int force_lv,
                             PassAcc *acc, double pvr = 0.0, double pvi = 0.0, int pp = 0) {
    const int c = cc.c, N = 1 << c;
    const int G = N >= 32 ? N >> 5 : 1;
    const int L = N >= 32 ? 32 : N;
    const int lane = threadIdx.x & 31;
    const uint32_t lanes = L == 32 ? FULL : ((1u << L) - 1u);

    LevelSizes ls;
    int nonfin = 0, inel = 0;
    unsigned long long nlo = 0, nhi = 0;
    unsigned rng = 0;
    bool onepass = !PT && !cc.force_raw && !cc.polar && cc.nlev == 1 && cc.shifts[0] >= 32 && c >= 5;
    if (PT) {
        // the words of size_levels for one amplitude: group pp >> 5 holds
        // it (lane g: group g's words), no residual is nonzero, the anchors
        // are its magnitudes
        const unsigned long long B0 = dbits(pvr) & MAG, B1 = dbits(pvi) & MAG;
        const uint32_t bit = 1u << (pp & 31);
        const bool at = lane == (pp >> 5);
        ls.wl0 = ls.wl1 = 0;
        ls.nz = 0;
        ls.sw0 = at && (dbits(pvr) >> 63) ? bit : 0u;
        ls.sw1 = at && (dbits(pvi) >> 63) ? bit : 0u;
        ls.zw0 = lane < G ? (at && B0 ? ~bit : FULL) : 0u;
        ls.zw1 = lane < G ? (at && B1 ? ~bit : FULL) : 0u;
        ls.f0 = B0;
        ls.f1 = B1;
    } else if (onepass) {                    // every value zero or inside the lossy range?
        bool odd = false;
        for (int i = lane; i < N; i += 32) {
            const uint32_t a = (uint32_t)__double2hiint(re[i]) & 0x7FFFFFFFu, al = (uint32_t)__double2loint(re[i]);
            const uint32_t b = (uint32_t)__double2hiint(im[i]) & 0x7FFFFFFFu, bl = (uint32_t)__double2loint(im[i]);
            odd |= a >= 0x7FE00000u || (a < 0x00100000u && (a | al) != 0u);
            odd |= b >= 0x7FE00000u || (b < 0x00100000u && (b | bl) != 0u);
        }
        onepass = !__any_sync(FULL, odd);
    }
    if (onepass) {
        pack_onepass(re, im, cc.shifts[0], G, ls, nlo, nhi, rng, wstage);
    } else if (!PT && !cc.force_raw) {
        size_levels(re, im, cc, G, L, false, ls, nonfin, inel);
        nonfin = __any_sync(FULL, nonfin);
        inel = __any_sync(FULL, inel);
        if (inel && !nonfin) {
            int d0 = 0, d1 = 0;
            size_levels(re, im, cc, G, L, true, ls, d0, d1);
        }
    }
    const bool raw_only = cc.force_raw || nonfin;

    // decision (warp-uniform).  A zero's sign is kept at shift 0 only, so
    // the sign sections come in two variants: every sign (lossless) and
    // the signs of the nonzero values (lossy).
    int mode, level = 0, s = 0, sm[2] = {0, 0}, zm[2] = {0, 0};
    uint32_t bodyb;
    const uint32_t raw_body = 16u * (uint32_t)N;
    unsigned long long res_off = 0;
    if (raw_only) {
        mode = M_RAW;
        bodyb = raw_body;
    } else {
        Sections q;
        sections_of(ls, G, lanes, q);
        zm[0] = q.zm0;
        zm[1] = q.zm1;
        mode = M_RAW;
        bodyb = raw_body;
        bool polar_done = false;
        if constexpr (POLAR) {
            // the ladder with the POLAR variant of every lossy level; a
            // POLAR stream is written there and the tile is done
            if (!inel && polar_ladder(re, im, cc, ls, q, raw_body, force_lv, tile, out_arena, out_cap, out_table,
                                      part, scal, sweep_id, wstage, mode, level, bodyb, sm, res_off, acc))
                return EncodeOut{res_off, res_off != ~0ull};
            polar_done = !inel;
        }
        if (!polar_done) {
            bool found = false;              // first level within the size limit, else the last
#pragma unroll
            for (int lv = 0; lv < MAX_LEVELS; ++lv) {
                if (lv >= cc.nlev || found || (force_lv >= 0 && lv != force_lv)) continue;
                bodyb = level_body(ls, q, lv, inel ? 0 : cc.shifts[lv], raw_body, mode, sm[0], sm[1]);
                level = lv;
                found = force_lv >= 0 || (unsigned long long)(HDR + bodyb) <= cc.max_bytes;
            }
        }
        s = mode == M_RAW ? 0 : (inel ? 0 : cc.shifts[level]);
    }
    const bool over = (unsigned long long)(HDR + bodyb) > cc.max_bytes;
    const uint32_t size = HDR + bodyb;
    unsigned long long off = 0;
    int ok = 0;
    if (lane == 0) {
        off = atomicAdd(&scal->bump, (unsigned long long)size);
        ok = off + size <= out_cap;
        if (!ok) {
            atomicOr(&scal->err, ERR_OVERFLOW);
            atomicCAS(&scal->err_sweep, 0u, sweep_id + 1u);
        }
        if (nonfin) atomicOr(&scal->err, ERR_NONFINITE);
    }
    off = shfl64(off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    EncodeOut res{off, ok != 0};
    if (!ok) return res;
    uint8_t *dst = out_arena + off;

    // header
    unsigned long long anc0 = 0, anc1 = 0;
    if (mode != M_RAW) {
        anc0 = quant(ls.f0, s);
        anc1 = quant(ls.f1, s);
    }
    if (lane < 8) {
        uint32_t v = 0;
        switch (lane) {
            case 0: {
                const uint32_t smb = mode == M_RAW ? 0u : (uint32_t)(sm[0] | (sm[1] << 3));
                v = (uint32_t)mode | ((uint32_t)s << 8) | ((uint32_t)level << 16) | (smb << 24);
                break;
            }
            case 1: v = bodyb; break;
            case 2: v = (uint32_t)anc0; break;
            case 3: v = (uint32_t)(anc0 >> 32); break;
            case 4: v = (uint32_t)anc1; break;
            case 5: v = (uint32_t)(anc1 >> 32); break;
            case 6: {
                const uint32_t zmb = mode == M_PACKED ? (uint32_t)(zm[0] | (zm[1] << 3)) : 0u;
                v = (uint32_t)c | (zmb << 8);
                break;
            }
            default: v = 0; break;
        }
        reinterpret_cast<uint32_t *>(dst)[lane] = v;
    }
    uint8_t *b = dst + HDR;
    if (mode == M_PACKED) {
        // sign sections, then zero sections
        const uint32_t sv0 = s ? ls.sw0 & ~ls.zw0 : ls.sw0, sv1 = s ? ls.sw1 & ~ls.zw1 : ls.sw1;
        uint32_t moff = 0, sz;
        write_section(reinterpret_cast<uint32_t *>(b + moff), sm[0], sv0, G, lanes);
        moff += (section_mode(sv0, G, lanes, sz), sz);
        write_section(reinterpret_cast<uint32_t *>(b + moff), sm[1], sv1, G, lanes);
        moff += (section_mode(sv1, G, lanes, sz), sz);
        write_section(reinterpret_cast<uint32_t *>(b + moff), zm[0], ls.zw0, G, lanes);
        moff += (section_mode(ls.zw0, G, lanes, sz), sz);
        write_section(reinterpret_cast<uint32_t *>(b + moff), zm[1], ls.zw1, G, lanes);
        moff += (section_mode(ls.zw1, G, lanes, sz), sz);
        // widths at the chosen level, word offsets
        const uint32_t ws0 = (uint32_t)(ls.wl0 >> (8 * level)) & 0xFFu;
        const uint32_t ws1 = (uint32_t)(ls.wl1 >> (8 * level)) & 0xFFu;
        uint32_t tot0, tot1;
        const uint32_t nn0 = __popc(~ls.zw0 & lanes), nn1 = __popc(~ls.zw1 & lanes);
        const uint32_t off0 = warp_exscan(lane < G ? (nn0 * ws0 + 31u) >> 5 : 0u, tot0);
        const uint32_t off1 = warp_exscan(lane < G ? (nn1 * ws1 + 31u) >> 5 : 0u, tot1) + tot0;
        const uint32_t wb = (2u * G + 3u) & ~3u;
        for (uint32_t base = 0; base < wb; base += 32) {          // uniform trip count
            const int t = (int)base + lane;
            const int src = t < G ? t : (t < 2 * G ? t - G : 0);
            const uint32_t a = __shfl_sync(FULL, ws0, src & 31);
            const uint32_t bb = __shfl_sync(FULL, ws1, src & 31);
            if ((uint32_t)t < wb) b[moff + t] = (uint8_t)(t < G ? a : (t < 2 * G ? bb : 0u));
        }
        const uint32_t doff = moff + wb;
        uint32_t *data = reinterpret_cast<uint32_t *>(b + doff);
        const uint32_t below = lanes_below();
        for (int k = 0; k < 2 && onepass; ++k) {      // packed words staged in shared memory
            const double *v = k ? im : re;
            const uint32_t wk = k ? ws1 : ws0, offk = k ? off1 : off0, nnk = k ? ~ls.zw1 : ~ls.zw0;
            for (int g = 0; g < G; ++g) {
                const uint32_t w = __shfl_sync(FULL, wk, g);
                if (w == 0) continue;
                const uint32_t wo = __shfl_sync(FULL, offk, g);
                const uint32_t nwd = ((uint32_t)__popc(__shfl_sync(FULL, nnk, g)) * w + 31u) >> 5;
                if ((uint32_t)lane < nwd) (data + wo)[lane] = reinterpret_cast<const uint32_t *>(v + g * 32)[lane];
            }
        }
        for (int k = 0; k < 2 && s >= 32 && !onepass && !PT; ++k) {
            // codes < 2^31 at shift >= 32: 32-bit codes, residuals and shuffles,
            // values spanning at most two words (the same bits as below)
            const double *v = k ? im : re;
            const uint32_t wk = k ? ws1 : ws0, offk = k ? off1 : off0;
            uint32_t carry = (uint32_t)quant(k ? ls.f1 : ls.f0, s);     // the anchor
            for (int g = 0; g < G; ++g) {
                const double x = lane < L ? v[g * 32 + lane] : 0.0;
                const uint32_t mh = (uint32_t)__double2hiint(x) & 0x7FFFFFFFu, lo = (uint32_t)__double2loint(x);
                const uint32_t nzm = __ballot_sync(FULL, (mh | lo) != 0u);
                if (nzm == 0u) continue;                     // all zeros: no norm, no data
                const uint32_t q = (mh | lo) ? quant_hi(mh, lo, s) : 0u;
                const bool dense = nzm == lanes;
                uint32_t qp;
                if (dense) {
                    const uint32_t up = __shfl_up_sync(FULL, q, 1);
                    qp = lane ? up : carry;
                } else {
                    const uint32_t pm = nzm & below;
                    const uint32_t qs = __shfl_sync(FULL, q, pm ? 31 - __clz(pm) : lane);
                    qp = pm ? qs : carry;
                }
                carry = __shfl_sync(FULL, q, dense ? L - 1 : 31 - __clz(nzm));
                if (q) {
                    unsigned long long l0, h0;
                    sq_units_code(q, s, l0, h0, rng);
                    add128(nlo, nhi, l0, h0);
                }
                const uint32_t w = __shfl_sync(FULL, wk, g);
                if (w == 0) continue;
                const uint32_t wo = __shfl_sync(FULL, offk, g);
                const uint32_t nwd = ((uint32_t)__popc(nzm) * w + 31u) >> 5;
                const bool nzl = (nzm >> lane) & 1u;
                const uint32_t r = q - qp;
                const uint32_t z = nzl ? (r << 1) ^ (uint32_t)((int)r >> 31) : 0u;
                wstage[lane] = 0u;
                __syncwarp();
                if (nzl) {
                    const uint32_t rank = dense ? (uint32_t)lane : (uint32_t)__popc(nzm & below);
                    const uint32_t bo = rank * w, j0 = bo >> 5, sh = bo & 31u;
                    atomicOr(&wstage[j0], z << sh);
                    if (sh + w > 32) atomicOr(&wstage[j0 + 1], z >> (32 - sh));
                }
                __syncwarp();
                if ((uint32_t)lane < nwd) (data + wo)[lane] = wstage[lane];
                __syncwarp();
            }
        }
        for (int k = 0; k < 2 && s < 32 && !PT; ++k) {
            const double *v = k ? im : re;
            const uint32_t wk = k ? ws1 : ws0, offk = k ? off1 : off0;
            unsigned long long carry = quant(k ? ls.f1 : ls.f0, s);     // the anchor
            for (int g = 0; g < G; ++g) {
                const unsigned long long B = lane < L ? (dbits(v[g * 32 + lane]) & MAG) : 0ull;
                const unsigned long long q = quant(B, s);
                const uint32_t nzm = __ballot_sync(FULL, lane < L && B != 0);
                if (nzm == 0u) continue;                     // all zeros: no norm, no data
                const bool dense = nzm == lanes;             // uniform: no zero in the group
                unsigned long long qp;
                if (dense) {
                    const unsigned long long up = shfl_up64(q, 1);
                    qp = lane ? up : carry;
                } else {
                    const uint32_t pm = nzm & below;
                    const unsigned long long qs = shfl64(q, pm ? 31 - __clz(pm) : lane);
                    qp = pm ? qs : carry;
                }
                const unsigned long long ql = shfl64(q, dense ? L - 1 : (nzm ? 31 - __clz(nzm) : 0));
                if (nzm) carry = ql;
                if (lane < L) {
                    unsigned long long l0, h0;
                    sq_units(q << s, l0, h0, rng);
                    add128(nlo, nhi, l0, h0);
                }
                const uint32_t w = __shfl_sync(FULL, wk, g);
                if (w == 0) continue;
                const uint32_t wo = __shfl_sync(FULL, offk, g);
                const uint32_t nwd = ((uint32_t)__popc(nzm) * w + 31u) >> 5;
                const bool nzl = (nzm >> lane) & 1u;
                const unsigned long long z = nzl ? zigzag(q - qp) : 0ull;
                wstage[lane] = 0u;
                wstage[lane + 32] = 0u;
                __syncwarp();
                if (nzl) {
                    const uint32_t rank = dense ? (uint32_t)lane : (uint32_t)__popc(nzm & below);
                    const uint32_t bo = rank * w, j0 = bo >> 5, sh = bo & 31u;
                    atomicOr(&wstage[j0], (uint32_t)(z << sh));
                    if (sh + w > 32) atomicOr(&wstage[j0 + 1], (uint32_t)(z >> (32 - sh)));
                    if (sh + w > 64) atomicOr(&wstage[j0 + 2], (uint32_t)(z >> (64 - sh)));
                }
                __syncwarp();
                uint32_t *gd = data + wo;
                if ((uint32_t)lane < nwd) gd[lane] = wstage[lane];
                if ((uint32_t)lane + 32 < nwd) gd[lane + 32] = wstage[lane + 32];
                __syncwarp();
            }
        }
        for (uint32_t p = doff + 4u * (tot0 + tot1) + lane; p < bodyb; p += 32) b[p] = 0;
    } else {
        if (mode == M_RAW) {
            double2 *o = reinterpret_cast<double2 *>(b);
            for (int i = lane; i < N; i += 32)
                o[i] = PT ? make_double2(i == pp ? pvr : 0.0, i == pp ? pvi : 0.0) : make_double2(re[i], im[i]);
        }
        for (int i = lane; i < N && !onepass && !PT; i += 32) {       // (one pass: norm already taken)
            unsigned long long u0 = dbits(re[i]) & MAG, u1 = dbits(im[i]) & MAG;
            if (mode == M_CONST) { u0 = quant(u0, s) << s; u1 = quant(u1, s) << s; }
            unsigned long long l0, h0, l1, h1;
            if (mode == M_CONST && s >= 21) {
                sq_units_q(u0, s, l0, h0, rng);
                sq_units_q(u1, s, l1, h1, rng);
            } else {
                sq_units(u0, l0, h0, rng);
                sq_units(u1, l1, h1, rng);
            }
            add128(nlo, nhi, l0, h0);
            add128(nlo, nhi, l1, h1);
        }
    }
    if (PT && lane == 0) {
        // the norm partial of the full tile: the amplitude's reconstruction
        unsigned long long l0, h0, l1, h1;
        const unsigned long long B0 = dbits(pvr) & MAG, B1 = dbits(pvi) & MAG;
        sq_units(mode == M_RAW ? B0 : quant(B0, s) << s, l0, h0, rng);
        sq_units(mode == M_RAW ? B1 : quant(B1, s) << s, l1, h1, rng);
        add128(l0, h0, l1, h1);
        nlo = l0;
        nhi = h0;
    }
    warp_sum128(nlo, nhi);
    rng = __any_sync(FULL, rng);
    if (lane == 0) {
        part[2 * tile] = nlo;
        part[2 * tile + 1] = nhi;
        tally_tile(acc, scal, nlo, nhi, level, over);
        out_table[tile] = off;
        if (rng) atomicOr(&scal->err, ERR_RANGE);
    }
    __syncwarp();
    return res;
}

// Encode with the POLAR variant (its own function, so that the
// componentwise encoder below keeps its registers).
__device__ __noinline__ EncodeOut wencode_polar(double *re, double *im, const CodecCfg &cc, unsigned long long tile,
                                                uint8_t *out_arena, unsigned long long out_cap,
                                                unsigned long long *out_table, unsigned long long *part,
                                                DevScalars *scal, unsigned sweep_id, uint32_t *wstage, int force_lv,
                                                PassAcc *acc) {
    return wencode_impl<true>(re, im, cc, tile, out_arena, out_cap, out_table, part, scal, sweep_id, wstage,
                              force_lv, acc);
}

// Encode a tile that is +0 but for the amplitude (vr, vi) at index p,
// exactly as wencode would, without reading the tile.  Tiles it does not
// take (uncompressed storage forced, the POLAR variant, c < 5, a nonzero
// component outside the lossy range) are left to wencode: false, nothing
// written.  Warp-wide.
__device__ __noinline__ bool wencode_point(double vr, double vi, int p, const CodecCfg &cc, unsigned long long tile,
                                           uint8_t *out_arena, unsigned long long out_cap,
                                           unsigned long long *out_table, unsigned long long *part,
                                           DevScalars *scal, unsigned sweep_id, int force_lv, PassAcc *acc) {
    const unsigned long long B0 = dbits(vr) & MAG, B1 = dbits(vi) & MAG;
    const bool odd = (B0 != 0ull && (B0 < MIN_NORMAL || B0 >= LOSSY_LIMIT)) ||
                     (B1 != 0ull && (B1 < MIN_NORMAL || B1 >= LOSSY_LIMIT));
    if (cc.force_raw || cc.polar || cc.c < 5 || odd) return false;
    wencode_impl<false, true>(nullptr, nullptr, cc, tile, out_arena, out_cap, out_table, part, scal, sweep_id,
                              nullptr, force_lv, acc, vr, vi, p);
    return true;
}

__device__ __forceinline__ EncodeOut wencode(double *re, double *im, const CodecCfg &cc, unsigned long long tile,
                                             uint8_t *out_arena, unsigned long long out_cap,
                                             unsigned long long *out_table, unsigned long long *part,
                                             DevScalars *scal, unsigned sweep_id, uint32_t *wstage, int force_lv,
                                             PassAcc *acc) {
    if (cc.polar)
        return wencode_polar(re, im, cc, tile, out_arena, out_cap, out_table, part, scal, sweep_id, wstage, force_lv,
                             acc);
    return wencode_impl<false>(re, im, cc, tile, out_arena, out_cap, out_table, part, scal, sweep_id, wstage,
                               force_lv, acc);
}

// Value of a well-formed CONST stream (the checks of wdecode), scaled like
// wdecode; false for any other stream.  One thread.
__device__ __forceinline__ bool const_value(const uint8_t *src, int c, double alpha, bool scale,
                                            double &vr, double &vi) {
    const uint4 w0 = __ldg(reinterpret_cast<const uint4 *>(src));
    const uint4 w1 = __ldg(reinterpret_cast<const uint4 *>(src) + 1);
    const int mode = w0.x & 0xFF, sh = (w0.x >> 8) & 0xFF;
    const int sm0 = (w0.x >> 24) & 7, sm1 = (w0.x >> 27) & 7;
    if (mode != M_CONST || sh > 52 || w0.y != 0u || sm0 > 1 || sm1 > 1 || (w1.z & 0xFFu) != (unsigned)c ||
        ((w1.z >> 8) & 0xFFu))
        return false;
    const unsigned long long a0 = ((unsigned long long)w0.w << 32) | w0.z;
    const unsigned long long a1 = ((unsigned long long)w1.y << 32) | w1.x;
    vr = bitsd((a0 << sh) | ((unsigned long long)sm0 << 63));
    vi = bitsd((a1 << sh) | ((unsigned long long)sm1 << 63));
    if (scale) { vr = __dmul_rn(vr, alpha); vi = __dmul_rn(vi, alpha); }
    return true;
}

// Fill a tile with its first amplitude (a uniform tile held as one value).
// Warp-wide.
__device__ __forceinline__ void fill_uniform(double *re, double *im, int N) {
    const int lane = threadIdx.x & 31;
    const double vr = re[0], vi = im[0];
    __syncwarp();
    for (int i = lane; i < N; i += 32) { re[i] = vr; im[i] = vi; }
    __syncwarp();
}

// Encode a uniform tile (every amplitude equal to re[0], im[0]) exactly as
// wencode would: a CONST stream at the first level whose 32 bytes fit the
// size limit, else at the last level, or at level force_lv when >= 0.
// Components that are non-finite or outside the lossy range, and
// uncompressed storage, are left to wencode: the tile is filled and false
// returned.  Warp-wide.
__device__ bool wencode_uniform(double *re, double *im, const CodecCfg &cc, unsigned long long tile,
                                uint8_t *out_arena, unsigned long long out_cap,
                                unsigned long long *out_table, unsigned long long *part,
                                DevScalars *scal, unsigned sweep_id, int force_lv, PassAcc *acc) {
    const int c = cc.c, N = 1 << c;
    const int lane = threadIdx.x & 31;
    const double vr = re[0], vi = im[0];
    const unsigned long long u0 = dbits(vr), u1 = dbits(vi), B0 = u0 & MAG, B1 = u1 & MAG;
    const bool odd0 = B0 >= INF_BITS || (B0 != 0 && (B0 < MIN_NORMAL || B0 >= LOSSY_LIMIT));
    const bool odd1 = B1 >= INF_BITS || (B1 != 0 && (B1 < MIN_NORMAL || B1 >= LOSSY_LIMIT));
    if (cc.force_raw || odd0 || odd1) {
        __syncwarp();
        for (int i = lane; i < N; i += 32) { re[i] = vr; im[i] = vi; }
        __syncwarp();
        return false;
    }
    const int level = force_lv >= 0 ? force_lv : (cc.max_bytes >= (unsigned long long)HDR ? 0 : cc.nlev - 1);
    const int s = cc.shifts[level];
    // stored signs: a zero keeps its sign only at shift 0
    const uint32_t sm0 = ((u0 >> 63) && (s == 0 || B0 != 0)) ? S_SET : S_CLEAR;
    const uint32_t sm1 = ((u1 >> 63) && (s == 0 || B1 != 0)) ? S_SET : S_CLEAR;
    const unsigned long long q0 = quant(B0, s), q1 = quant(B1, s);
    unsigned long long off = 0;
    int ok = 0;
    if (lane == 0) {
        off = atomicAdd(&scal->bump, (unsigned long long)HDR);
        ok = off + HDR <= out_cap;
        if (!ok) {
            atomicOr(&scal->err, ERR_OVERFLOW);
            atomicCAS(&scal->err_sweep, 0u, sweep_id + 1u);
        }
    }
    off = shfl64(off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    if (!ok) return true;
    if (lane < 8) {
        uint32_t v = 0;
        switch (lane) {
            case 0: v = ((uint32_t)s << 8) | ((uint32_t)level << 16) | ((sm0 | (sm1 << 3)) << 24); break;
            case 2: v = (uint32_t)q0; break;
            case 3: v = (uint32_t)(q0 >> 32); break;
            case 4: v = (uint32_t)q1; break;
            case 5: v = (uint32_t)(q1 >> 32); break;
            case 6: v = (uint32_t)c; break;
            default: v = 0; break;
        }
        reinterpret_cast<uint32_t *>(out_arena + off)[lane] = v;
    }
    if (lane == 0) {
        // norm partial: N times the exact square of each reconstructed component
        unsigned long long l0, h0, l1, h1;
        unsigned rng = 0;
        sq_units(q0 << s, l0, h0, rng);
        sq_units(q1 << s, l1, h1, rng);
        add128(l0, h0, l1, h1);
        const unsigned long long nlo = l0 << c, nhi = (h0 << c) | (c ? l0 >> (64 - c) : 0ull);
        part[2 * tile] = nlo;
        part[2 * tile + 1] = nhi;
        tally_tile(acc, scal, nlo, nhi, level, (unsigned long long)HDR > cc.max_bytes);
        out_table[tile] = off;
        if (rng) atomicOr(&scal->err, ERR_RANGE);
    }
    __syncwarp();
    return true;
}

// Copy one stream unchanged into the output arena (a tile no gate touches).
// Warp-wide.
__device__ void wcarry(const uint8_t *in_arena, const unsigned long long *in_table,
                       unsigned long long tile, uint8_t *out_arena, unsigned long long out_cap,
                       unsigned long long *out_table, const unsigned long long *part,
                       DevScalars *scal, unsigned sweep_id, PassAcc *acc) {
    const int lane = threadIdx.x & 31;
    const uint8_t *src = in_arena + in_table[tile];
    const uint32_t size = HDR + reinterpret_cast<const uint32_t *>(src)[1];
    unsigned long long off = 0;
    int ok = 0;
    if (lane == 0) {
        off = atomicAdd(&scal->bump, (unsigned long long)size);
        ok = off + size <= out_cap;
        if (!ok) {
            atomicOr(&scal->err, ERR_OVERFLOW);
            atomicCAS(&scal->err_sweep, 0u, sweep_id + 1u);
        }
        tally_norm(acc, scal, part[2 * tile], part[2 * tile + 1]);
        if (ok) out_table[tile] = off;
    }
    off = shfl64(off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    if (ok) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(out_arena + off);
        for (uint32_t i = lane; i < size / 16u; i += 32) d4[i] = s4[i];
    }
    __syncwarp();
}

// Move one stream unchanged from tile `src` of the input arena to tile
// `dst` of the output arena, with its norm partial (plo, phi).  Warp-wide.
__device__ void wmove(const uint8_t *in_arena, const unsigned long long *in_table, unsigned long long src,
                      unsigned long long dst, uint8_t *out_arena, unsigned long long out_cap,
                      unsigned long long *out_table, unsigned long long *part, unsigned long long plo,
                      unsigned long long phi, DevScalars *scal, unsigned sweep_id, PassAcc *acc) {
    const int lane = threadIdx.x & 31;
    const uint8_t *sp = in_arena + in_table[src];
    const uint32_t size = HDR + reinterpret_cast<const uint32_t *>(sp)[1];
    unsigned long long off = 0;
    int ok = 0;
    if (lane == 0) {
        off = atomicAdd(&scal->bump, (unsigned long long)size);
        ok = off + size <= out_cap;
        if (!ok) {
            atomicOr(&scal->err, ERR_OVERFLOW);
            atomicCAS(&scal->err_sweep, 0u, sweep_id + 1u);
        }
        tally_norm(acc, scal, plo, phi);
        part[2 * dst] = plo;
        part[2 * dst + 1] = phi;
        if (ok) out_table[dst] = off;
    }
    off = shfl64(off, 0);
    ok = __shfl_sync(FULL, ok, 0);
    if (ok) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(sp);
        uint4 *d4 = reinterpret_cast<uint4 *>(out_arena + off);
        for (uint32_t i = lane; i < size / 16u; i += 32) d4[i] = s4[i];
    }
    __syncwarp();
}

// exact norm of a decoded tile (warp-wide), for validation of imports
__device__ void wnorm(const double *re, const double *im, int N, unsigned long long &lo,
                      unsigned long long &hi, unsigned &rng) {
    lo = hi = 0;
    for (int i = threadIdx.x & 31; i < N; i += 32) {
        unsigned long long l0, h0, l1, h1;
        sq_units(dbits(re[i]), l0, h0, rng);
        sq_units(dbits(im[i]), l1, h1, rng);
        add128(lo, hi, l0, h0);
        add128(lo, hi, l1, h1);
    }
    warp_sum128(lo, hi);
}

// ---------------------------------------------------------------- point items, one per warp
// A point item (every member tile +0 but for at most one amplitude, at a
// tile index p common to the members) held as its 2^h amplitudes: entry j
// of cre/cim is member j's amplitude at p.  The gates run on those entries
// with the arithmetic of the item buffer's red = c pass, so the result is
// the same.

// apply_run (red = c) on the compact entries: lane j < 2^h takes member j.
__device__ unsigned apply_run_point(double *cre, double *cim, int c, int h, const DRun &Rg, const SweepParams &P,
                                    unsigned long long T, const int *hb, unsigned p) {
    const DRun R = Rg;
    const int j = threadIdx.x & 31, N = 1 << c;
    unsigned ops = 0;
    if (j >= (1 << h)) return 0;
    const unsigned long long xb = member_tile(T, j, h, hb) << c;
    bool have_t = false;
    double tr = 0.0, ti = 0.0;
    unsigned k = 0;
    ops += run_factor(P.rgates + R.tg, R.nt, xb, have_t, tr, ti, k);
    if (!(have_t || (k & 3u)) && R.nl == 0) return ops;          // nothing to visit
    double xr = cre[j], xi = cim[j];
    if (zero_amp(xr, xi)) return ops;                              // a zero stays as it is
    k &= 3u;
    bool have_l = false;
    double lr = 0.0, li = 0.0;
    if (R.nl) {
        if (R.tabled) {
            unsigned kap = 0;
            for (int i = 0; i < R.nq; ++i) kap |= (unsigned)((xb >> R.q[i]) & 1ull) << i;
            const unsigned long long e = R.table + (unsigned long long)kap * N + p;
            const unsigned mt = P.rmeta[e];
            have_l = mt & 1u;
            k += mt >> 1;
            if (have_l) {
                const double2 v = P.rtab[e];
                lr = v.x;
                li = v.y;
            }
        } else {
            ops += run_factor(P.rgates + R.lg, R.nl, xb | p, have_l, lr, li, k);
        }
    }
    if (!have_t && !have_l && (k & 3u) == 0u) return ops;
    if (have_t || have_l) {
        double gr = have_t ? tr : lr, gi = have_t ? ti : li;
        if (have_t && have_l) { cmul(tr, ti, lr, li, gr, gi); ops += 4; }
        cmul(gr, gi, xr, xi, xr, xi);
        ops += 4;
    }
    unit_pow(k, xr, xi);
    cre[j] = xr;
    cim[j] = xi;
    return ops;
}

// One item of a sweep whose gates keep zeros as they are (runs, scaled
// gates, permutations; the mixing ones on qubits >= c), on one warp with
// no CTA barrier.  wre/wim: the warp's tile scratch (2^c each); cre/cim:
// its 2^h entries; act: its activity words; wst: its packing stage.
// Returns false, having written nothing, when the item is not a point item
// (or holds a malformed stream): the CTA path takes it then.
__device__ __noinline__ bool point_item_warp(const SweepParams &P, unsigned long long item, double alpha, bool scale,
                                             double *wre, double *wim, double *cre, double *cim, unsigned *act,
                                             uint32_t *wst, PassAcc *acc, unsigned &run_ops) {
    const int lane = threadIdx.x & 31;
    const int c = P.cc.c, N = 1 << c, h = P.h, ntl = 1 << h;
    int hb[MAX_PAIRS];
#pragma unroll
    for (int i = 0; i < MAX_PAIRS; ++i) hb[i] = i < h ? P.H[i] - c : 0;
    const unsigned long long T = expand_item(item, h, hb);
    const unsigned long long fixed = T << c;
    // which gates change something here; a run's activity on its first gate
    bool any = false;
    for (int w = 0; w < (P.ngates + 31) >> 5; ++w) {
        const int g = (w << 5) + lane;
        const bool a = g < P.ngates && gate_active(P.sgates[g], fixed);
        const unsigned bal = __ballot_sync(FULL, a);
        if (lane == 0) act[w] = bal;
        any |= bal != 0u;
    }
    __syncwarp();
    for (int r = 0; r < P.nruns && any; ++r) {
        const DRun R = P.runs[P.run_first + r];
        bool ra = false;
        for (int g = R.first + lane; g < R.first + R.len; g += 32) ra |= (act[g >> 5] >> (g & 31)) & 1u;
        ra = __any_sync(FULL, ra);
        __syncwarp();
        for (int g = R.first + lane; g < R.first + R.len; g += 32) {
            const unsigned bit = 1u << (g & 31);
            if (g == R.first && ra) atomicOr(&act[g >> 5], bit);
            else atomicAnd(&act[g >> 5], ~bit);
        }
        __syncwarp();
    }
    if (!any && !scale) {
        for (int j = 0; j < ntl; ++j)
            wcarry(P.in_arena, P.in_table, member_tile(T, j, h, hb), P.out_arena, P.out_cap, P.out_table, P.part,
                   P.scal, P.sweep_id, acc);
        if (lane == 0) atomicAdd(&P.scal->items_skipped, 1ull);
        return true;
    }
    // members' amplitudes; every other entry must be +0
    int pos = -1;
    for (int j = 0; j < ntl; ++j) {
        const int r = wdecode_one(P.in_arena + P.in_table[member_tile(T, j, h, hb)], c, wre, wim, alpha, scale);
        if (r == 1) return false;
        int at = -1;
        if (r >= 2) {
            at = r - 2;
        } else {
            __syncwarp();
            unsigned cnt = 0;
            for (int b = 0; b < N; b += 32) {
                const int i = b + lane;
                const bool v = (unsigned long long)(__double_as_longlong(wre[i]) | __double_as_longlong(wim[i])) != 0ull;
                const unsigned bal = __ballot_sync(FULL, v);
                cnt += (unsigned)__popc(bal);
                if (bal) at = b + 31 - __clz(bal);
            }
            if (cnt > 1u) return false;
        }
        __syncwarp();
        double vr = 0.0, vi = 0.0;
        if (at >= 0) {
            if (pos >= 0 && pos != at) return false;
            pos = at;
            vr = wre[at];
            vi = wim[at];
        }
        __syncwarp();
        if (lane == 0) { cre[j] = vr; cim[j] = vi; }
    }
    __syncwarp();
    const unsigned roff = pos > 0 ? (unsigned)pos : 0u;
    if (any) {
        for (int i = 0; i < P.nglist; ++i) {
            const int g = P.glist[i];
            if (!((act[g >> 5] >> (g & 31)) & 1u)) continue;
            SGate s = P.sgates[g];
            if (s.run != -1) {
                if (s.run >= 0) run_ops += apply_run_point(cre, cim, c, h, P.runs[s.run], P, T, hb, roff);
                __syncwarp();
                continue;
            }
            // the gate on the 2^h entries: its buffer bits (all >= c in
            // such a sweep) lowered by c
            if (s.p0 >= 0) s.p0 = (int8_t)(s.p0 - c);
            if (s.p1 >= 0) s.p1 = (int8_t)(s.p1 - c);
            for (int q = 0; q < s.nins; ++q) s.ins[q] = (uint8_t)(s.ins[q] - c);
            s.lcm >>= c;
            s.lcv >>= c;
            if (s.kind == 0) diag_gate(cre, cim, h, s, fixed, 0, 0u, (unsigned)lane, 32u);
            else if (s.kind == 1) run_ops += one_target(cre, cim, h, s, P.gates[g], 0, 0u, (unsigned)lane, 32u);
            else run_ops += two_target(cre, cim, h, s, P.gates[g], 0, 0u, (unsigned)lane, 32u);
            __syncwarp();
        }
    }
    for (int j = 0; j < ntl; ++j) {
        const unsigned long long Tj = member_tile(T, j, h, hb);
        const int flv = P.unit_level ? (int)P.unit_level[Tj >> P.unit_shift] : -1;
        const double vr = cre[j], vi = cim[j];
        if (wencode_point(vr, vi, (int)roff, P.cc, Tj, P.out_arena, P.out_cap, P.out_table, P.part, P.scal,
                          P.sweep_id, flv, acc))
            continue;
        for (int i = lane; i < N; i += 32) {
            wre[i] = i == (int)roff ? vr : 0.0;
            wim[i] = i == (int)roff ? vi : 0.0;
        }
        __syncwarp();
        wencode(wre, wim, P.cc, Tj, P.out_arena, P.out_cap, P.out_table, P.part, P.scal, P.sweep_id, wst, flv, acc);
    }
    if (lane == 0) atomicAdd(&P.scal->items_done, 1ull);
    return true;
}

// ---------------------------------------------------------------- kernels
// Sweeps of Algorithm 2 over all items of a work list: entry e of plist is
// one sweep of one state, owning the global item indices istart[e] ..
// istart[e+1]-1.  A single-state flush passes a one-entry list; a batch
// passes one entry per state.  Per item: decompress (with normalize), apply
// the gate run, compress with the ladder.  Persistent CTAs loop over items;
// within an item every warp codes its own tiles.  A CTA reloads the
// parameters and gates whenever it crosses into another entry's items.
// SIZING: the sizing pass of per-stride ladder decisions (the same sweep,
// stream sizes counted per stride and level, nothing written); a separate
// instance so that the encoding sweep carries no extra call site.
// Items are handed out by an atomic counter (work, zero at launch), so a
// CTA that runs faster than its neighbours takes more items.
template <bool SIZING, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) sweep_kernel(const SweepParams *__restrict__ plist,
                                                          const unsigned long long *__restrict__ istart,
                                                          int nlist, unsigned long long *work) {
    extern __shared__ double smem[];
    __shared__ SGate sg[GATE_CHUNK];
    __shared__ SweepParams P;
    __shared__ unsigned s_act[MAX_SWEEP_GATES / 32];
    __shared__ int s_entry, s_skip, s_chunk, s_any, s_ppos, s_pbad;
    __shared__ unsigned long long s_gi;
    __shared__ int s_dest[1 << MAX_PAIRS];
    __shared__ unsigned long long s_plo[1 << MAX_PAIRS], s_phi[1 << MAX_PAIRS];
    __shared__ double s_alpha;
    __shared__ RunMember s_mem[1 << MAX_PAIRS];
    __shared__ unsigned long long s_rundp;
    __shared__ PassAcc s_acc;
    constexpr int NWARPS = NT / 32;
    __shared__ unsigned long long s_defer[NWARPS];    // items handed back by the warps (~0: none)
    __shared__ int s_dn, s_wm;
    const unsigned long long total = istart[nlist];
    if (threadIdx.x == 0) {
        s_rundp = 0;
        s_acc.lo = s_acc.hi = s_acc.over = 0;
        for (int lv = 0; lv < MAX_LEVELS; ++lv) s_acc.hist[lv] = 0;
        s_dn = NWARPS;
    }
    unsigned run_ops = 0;                 // FP64 instructions of diagonal runs (this thread)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cur = -1;
    uint32_t *wst = nullptr;              // the warp's packing stage, after the item buffer
    if (!SIZING && nlist == 1) {
        // A single state's sweep whose gates keep zeros as they are: its
        // point items run one per warp, with no CTA barrier, until the
        // items run out or the warp meets an item that is not a point item
        // (handed back to the CTA loop below, which takes it first).
        {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(plist);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
            for (int i = threadIdx.x; i < (int)(sizeof(SweepParams) / 4); i += NT) dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_chunk = -1;
            s_skip = *((volatile unsigned *)&P.scal->err) != 0u;
            s_alpha = P.use_alpha ? P.scal->alpha : 1.0;
            if (P.dscale) s_alpha = __dmul_rn(s_alpha, *P.dscale);
            const int c = P.cc.c, mb = c + P.h;
            // per warp: a tile (2^(c+1) doubles), 2^h entries of each
            // component (32 doubles at most) and the activity words (8)
            const bool fits = (long long)NWARPS * ((2ll << c) + 40) <= (2ll << mb);
            s_wm = P.point_ok && !P.moves_tiles && !P.every_item && !s_skip && c >= 5 && fits;
            if (s_wm) s_dn = 0;
        }
        __syncthreads();
        cur = 0;
        if (s_wm) {
            const int N = 1 << P.cc.c;
            double *wre = smem + warp * (2 * N + 40), *wim = wre + N, *cre = wim + N, *cim = cre + 16;
            unsigned *wact = reinterpret_cast<unsigned *>(cim + 16);
            wst = reinterpret_cast<uint32_t *>(smem + (2 << (P.cc.c + P.h))) + 64 * warp;
            const double alpha = s_alpha;
            unsigned long long mine = ~0ull;
            for (;;) {
                unsigned long long g = 0;
                if (lane == 0) g = atomicAdd(work, 1ull);
                g = shfl64(g, 0);
                if (g >= total) break;
                if (!point_item_warp(P, g - istart[0], alpha, alpha != 1.0, wre, wim, cre, cim, wact, wst, &s_acc,
                                     run_ops)) {
                    mine = g;
                    break;
                }
            }
            if (lane == 0) s_defer[warp] = mine;
        }
    }
    for (;;) {
        __syncthreads();                  // previous item finished by every warp
        if (threadIdx.x == 0) {           // next item; entry owning it: last e with istart[e] <= gi
            // items handed back by the warps first, then the counter
            while (s_dn < NWARPS && s_defer[s_dn] == ~0ull) ++s_dn;
            const unsigned long long g = s_dn < NWARPS ? s_defer[s_dn++] : atomicAdd(work, 1ull);
            int lo = 0, hi = nlist - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (istart[mid] <= g) lo = mid; else hi = mid - 1;
            }
            s_gi = g;
            s_entry = lo;
        }
        __syncthreads();
        const unsigned long long gi = s_gi;
        const int e = gi >= total ? -1 : s_entry;
        if (e != cur && cur >= 0) {
            // the CTA's diagonal-run FP64 count for the state it leaves: one
            // global atomic per CTA and state
            const unsigned wsum = __reduce_add_sync(FULL, run_ops);
            run_ops = 0;
            if (lane == 0 && wsum) atomicAdd(&s_rundp, (unsigned long long)wsum);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (s_rundp) atomicAdd(&P.scal->run_dp, s_rundp);
                s_rundp = 0;
                flush_acc(&s_acc, P.scal);      // the norm and level sums of the state it leaves
            }
            __syncthreads();
        }
        if (gi >= total) break;
        if (e != cur) {
            {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(plist + e);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&P);
                for (int i = threadIdx.x; i < (int)(sizeof(SweepParams) / 4); i += NT) dst[i] = src[i];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_chunk = -1;                 // gates are staged on first use
                // an earlier pass of this state failed: leave its state alone
                s_skip = *((volatile unsigned *)&P.scal->err) != 0u;
                s_alpha = P.use_alpha ? P.scal->alpha : 1.0;
                // the scaled gates' product joins the normalize scale
                if (P.dscale) s_alpha = __dmul_rn(s_alpha, *P.dscale);
            }
            __syncthreads();
            cur = e;
        }
        if (s_skip) continue;
        const int c = P.cc.c, N = 1 << c, h = P.h, mb = c + h, ntl = 1 << h;
        double *re = smem, *im = smem + (1 << mb);
        wst = reinterpret_cast<uint32_t *>(smem + (2 << mb)) + 64 * warp;
        const double alpha = s_alpha;
        const bool scale = alpha != 1.0;
        int hb[MAX_PAIRS];
#pragma unroll
        for (int i = 0; i < MAX_PAIRS; ++i) hb[i] = i < h ? P.H[i] - c : 0;
        const unsigned long long T = expand_item(gi - istart[e], h, hb);
        const unsigned long long fixed = T << c;
        // which gates change something in this item (from the compact
        // gates in global memory; one word of 32 gates per warp)
        if (threadIdx.x == 0) { s_any = 0; s_ppos = -1; s_pbad = 0; }
        __syncthreads();
        for (int w = warp; w < (P.ngates + 31) >> 5; w += NWARPS) {
            const int g = (w << 5) + lane;
            const bool a = g < P.ngates && gate_active(P.sgates[g], fixed);
            const unsigned bal = __ballot_sync(FULL, a);
            if (lane == 0) {
                s_act[w] = bal;
                if (bal) s_any = 1;
            }
        }
        __syncthreads();
        if (P.nruns && warp == 0) {
            // a diagonal run is active when any of its gates is; its activity
            // goes to its first gate, which applies the whole run
            for (int r = 0; r < P.nruns; ++r) {
                const DRun R = P.runs[P.run_first + r];
                bool any = false;
                for (int g = R.first + lane; g < R.first + R.len; g += 32)
                    any |= (s_act[g >> 5] >> (g & 31)) & 1u;
                any = __any_sync(FULL, any);
                __syncwarp();
                for (int g = R.first + lane; g < R.first + R.len; g += 32) {
                    const unsigned bit = 1u << (g & 31);
                    const bool on = g == R.first && any;
                    // lanes of one word change disjoint bits
                    if (on) atomicOr(&s_act[g >> 5], bit);
                    else atomicAnd(&s_act[g >> 5], ~bit);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const bool active = s_any != 0;
        if (!active && (!scale || P.moves_tiles) && !P.every_item) {
            for (int j = warp; j < ntl; j += NWARPS)
                wcarry(P.in_arena, P.in_table, member_tile(T, j, h, hb), P.out_arena, P.out_cap,
                       P.out_table, P.part, P.scal, P.sweep_id, &s_acc);
            if (threadIdx.x == 0) atomicAdd(&P.scal->items_skipped, 1ull);
            continue;
        }
        // Sweeps of permutations on qubits >= c move whole tiles: member j's
        // stream goes unchanged to the member the gates map it to (no
        // decompression, so no normalize; the norm is unchanged).
        if (P.moves_tiles) {
            if ((int)threadIdx.x < ntl) {
                unsigned L = (unsigned)threadIdx.x << c;     // buffer index of the member's first amplitude
                for (int g = 0; g < P.ngates; ++g) {
                    if (!((s_act[g >> 5] >> (g & 31)) & 1u)) continue;
                    const SGate &sgl = P.sgates[g];
                    if (sgl.kind == 0 || (L & sgl.lcm) != sgl.lcv) continue;    // identity / controls fail
                    const int dim = 1 << sgl.k;
                    int r = (int)((L >> sgl.p0) & 1u);
                    if (sgl.k > 1) r |= (int)((L >> sgl.p1) & 1u) << 1;
                    int r2 = r;
                    for (int row = 0; row < dim; ++row)
                        if (((sgl.cls >> (3 * (row * dim + r))) & 7ull) == EC_ONE) r2 = row;
                    L = (L & ~(1u << sgl.p0)) | ((unsigned)(r2 & 1) << sgl.p0);
                    if (sgl.k > 1) L = (L & ~(1u << sgl.p1)) | ((unsigned)((r2 >> 1) & 1) << sgl.p1);
                }
                const unsigned long long Tj = member_tile(T, threadIdx.x, h, hb);
                s_dest[threadIdx.x] = (int)(L >> c);
                s_plo[threadIdx.x] = P.part[2 * Tj];
                s_phi[threadIdx.x] = P.part[2 * Tj + 1];
            }
            __syncthreads();
            for (int j = warp; j < ntl; j += NWARPS)
                wmove(P.in_arena, P.in_table, member_tile(T, j, h, hb), member_tile(T, s_dest[j], h, hb),
                      P.out_arena, P.out_cap, P.out_table, P.part, s_plo[j], s_phi[j], P.scal, P.sweep_id, &s_acc);
            if (threadIdx.x == 0) atomicAdd(&P.scal->items_done, 1ull);
            continue;
        }
        // Uniform items: when every member tile is CONST and no gate of the
        // sweep touches a low qubit, every tile stays uniform; the gates run
        // on one amplitude per tile, each with the operands every amplitude
        // of the tile would see, and the tiles are written back as CONST.
        bool uni = false;
        if (P.low_free || !active) {
            bool ok = true;
            if ((int)threadIdx.x < ntl) {
                double vr, vi;
                ok = const_value(P.in_arena + P.in_table[member_tile(T, threadIdx.x, h, hb)], c, alpha,
                                 scale, vr, vi);
                re[threadIdx.x * N] = vr;
                im[threadIdx.x * N] = vi;
            }
            uni = __syncthreads_and(ok);
        }
        // point items: the gates run on one amplitude per tile (red = c) at
        // the tiles' common nonzero index; the other amplitudes are +0 and
        // every gate of such a sweep leaves them so
        const bool pscan = active && !uni && P.point_ok;
        if (!uni) {
            int bad = 0;
            for (int j = warp; j < ntl; j += NWARPS) {
                const unsigned long long Tj = member_tile(T, j, h, hb);
                bad |= wdecode(P.in_arena + P.in_table[Tj], c, re + j * N, im + j * N, alpha, scale);
                if (pscan) point_scan(re + j * N, im + j * N, N, &s_ppos, &s_pbad);
            }
            if (bad && lane == 0) atomicOr(&P.scal->err, ERR_FORMAT);
        }
        if (active) {
            __syncthreads();
            const bool point = pscan && !s_pbad;
            const unsigned roff = point && s_ppos > 0 ? (unsigned)s_ppos : 0u;
            // the packing stage after the item buffer (64 words per warp) is
            // free until the encoder runs
            run_ops += apply_gates(re, im, mb, (uni || point) ? c : 0, P.sgates, sg, &s_chunk, P.gates, P.ngates,
                                   s_act, fixed, P, hb, s_mem, reinterpret_cast<uint32_t *>(smem + (2 << mb)),
                                   64 * NWARPS, roff);
            if (uni || point) __syncthreads();       // warp 0 applied them alone
        }
        for (int j = warp; j < ntl; j += NWARPS) {
            const unsigned long long Tj = member_tile(T, j, h, hb);
            if (SIZING) {
                if (uni) fill_uniform(re + j * N, im + j * N, N);
                wsize(re + j * N, im + j * N, P.cc, P.unit_bytes + (Tj >> P.unit_shift) * MAX_LEVELS);
                continue;
            }
            const int flv = P.unit_level ? (int)P.unit_level[Tj >> P.unit_shift] : -1;
            if (uni && wencode_uniform(re + j * N, im + j * N, P.cc, Tj, P.out_arena, P.out_cap, P.out_table,
                                       P.part, P.scal, P.sweep_id, flv, &s_acc))
                continue;
            wencode(re + j * N, im + j * N, P.cc, Tj, P.out_arena, P.out_cap, P.out_table, P.part, P.scal,
                    P.sweep_id, wst, flv, &s_acc);
        }
        if (threadIdx.x == 0 && !SIZING) atomicAdd(&P.scal->items_done, 1ull);
    }
}

// Finish a pass of one state: publish the norm, the next normalize scale
// and the used bytes; reset the accumulators.  Leaves everything alone after
// an error so that the host can re-run the failed pass.
__device__ void finalize_state(const FinalizeEntry &f) {
    DevScalars *scal = f.scal;
    if (scal->err) return;
    scal->norm_lo = scal->acc_lo;
    scal->norm_hi = scal->acc_hi;
    scal->acc_lo = scal->acc_hi = 0;
    if (f.record_used) {
        scal->used = scal->bump;
        if (f.used_hist) f.used_hist[f.slot] = scal->bump;
        scal->bump = 0;
    }
    const double nrm = units_to_double(scal->norm_lo, scal->norm_hi);
    scal->alpha = (f.use_alpha && nrm > 0.0) ? __ddiv_rn(1.0, __dsqrt_rn(nrm)) : 1.0;
}

__global__ void finalize_kernel(FinalizeEntry f) {
    if (threadIdx.x == 0 && blockIdx.x == 0) finalize_state(f);
}

__global__ void finalize_list_kernel(const FinalizeEntry *list, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        finalize_state(list[i]);
}

// Per-warp tile kernels: TILE_WARPS warps per CTA, each owning a tile buffer
// of 2^c amplitudes (planar) in dynamic shared memory.
constexpr int TILE_WARPS = 4;

// Encode a state given densely (device, interleaved) or the basis state
// |x> (dense == nullptr) into every tile.
// FP64 issue-rate probe: eight independent DFMA chains per thread, so the
// pipe, not the chain latency, bounds it.  out[blockIdx.x*blockDim.x +
// threadIdx.x] keeps the results live.
__global__ void __launch_bounds__(256) fp64_rate_kernel(double *out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (double)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = __fma_rn(x[i], a, b);
    }
    double sum = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) sum += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// Encode a fresh state (dense amplitudes, or the basis state |x> when
// dense is null), one warp per tile.  With unit_bytes set this is the
// sizing pass of per-stride decisions (nothing written but the counts);
// with unit_level set every tile is coded at its stride's level.
__global__ void __launch_bounds__(32 * TILE_WARPS) init_kernel(
    const double2 *dense, unsigned long long x, CodecCfg cc, unsigned long long ntiles,
    uint8_t *out_arena, unsigned long long out_cap, unsigned long long *out_table,
    unsigned long long *part, DevScalars *scal, unsigned long long *unit_bytes,
    const uint8_t *unit_level, int unit_shift) {
    extern __shared__ double smem[];
    __shared__ uint32_t stage[64 * TILE_WARPS];
    __shared__ unsigned long long s_hist[MAX_LEVELS];
    const int c = cc.c, N = 1 << c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *re = smem + (size_t)warp * 2 * N, *im = re + N;
    uint32_t *wst = stage + 64 * warp;
    // A basis state's zero tiles are 32-byte CONST streams at fixed places
    // (tile t at 32 t, less one slot past the nonzero tile); the warp of the
    // nonzero tile reserves their range on the bump counter before its own
    // stream, which then follows them, so the zero tiles take no atomic each.
    // Their level counts are summed per CTA.
    const unsigned long long tx = x >> c;
    const bool zfixed = dense == nullptr && !cc.force_raw && unit_bytes == nullptr;
    if (threadIdx.x < MAX_LEVELS) s_hist[threadIdx.x] = 0;
    __syncthreads();
    for (unsigned long long t = (unsigned long long)blockIdx.x * TILE_WARPS + warp; t < ntiles;
         t += (unsigned long long)gridDim.x * TILE_WARPS) {
        if (dense == nullptr && (x >> c) != t) {
            // all-zero tile: CONST at every level (32 bytes), or RAW zeros
            const uint32_t size = cc.force_raw ? HDR + 16u * N : HDR;
            if (unit_bytes) {
                if (lane < cc.nlev) atomicAdd(unit_bytes + (t >> unit_shift) * MAX_LEVELS + lane, (unsigned long long)size);
                continue;
            }
            unsigned long long off = 0;
            int ok = 0;
            if (lane == 0) {
                off = zfixed ? (unsigned long long)HDR * (t - (t > tx ? 1ull : 0ull))
                             : atomicAdd(&scal->bump, (unsigned long long)size);
                ok = off + size <= out_cap;
                if (!ok) atomicOr(&scal->err, ERR_OVERFLOW);
            }
            off = shfl64(off, 0);
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) continue;
            const int lv = unit_level ? (int)unit_level[t >> unit_shift]
                                      : (cc.max_bytes >= (unsigned long long)HDR ? 0 : cc.nlev - 1);
            const int s = cc.force_raw ? 0 : cc.shifts[lv];
            uint32_t *d = reinterpret_cast<uint32_t *>(out_arena + off);
            if (lane < 8) {
                uint32_t v = 0;
                if (lane == 0) v = cc.force_raw ? (uint32_t)M_RAW : (((uint32_t)s << 8) | ((uint32_t)lv << 16));
                else if (lane == 1) v = cc.force_raw ? 16u * N : 0u;
                else if (lane == 6) v = (uint32_t)c;
                d[lane] = v;
            }
            if (cc.force_raw) {
                uint4 *d4 = reinterpret_cast<uint4 *>(out_arena + off + HDR);
                for (int i = lane; i < N; i += 32) d4[i] = make_uint4(0, 0, 0, 0);
            }
            if (lane == 0) {
                out_table[t] = off;
                part[2 * t] = part[2 * t + 1] = 0;
                atomicAdd(&s_hist[cc.force_raw ? 0 : lv], 1ull);
            }
            continue;
        }
        for (int i = lane; i < N; i += 32) {
            if (dense) {
                const double2 v = dense[t * (unsigned long long)N + i];
                re[i] = v.x;
                im[i] = v.y;
            } else {
                re[i] = (((t << c) | (unsigned long long)i) == x) ? 1.0 : 0.0;
                im[i] = 0.0;
            }
        }
        __syncwarp();
        if (unit_bytes) {
            wsize(re, im, cc, unit_bytes + (t >> unit_shift) * MAX_LEVELS);
            continue;
        }
        if (zfixed && lane == 0) atomicAdd(&scal->bump, (unsigned long long)HDR * (ntiles - 1));
        __syncwarp();
        wencode(re, im, cc, t, out_arena, out_cap, out_table, part, scal, 0u, wst,
                unit_level ? (int)unit_level[t >> unit_shift] : -1, nullptr);
    }
    __syncthreads();
    if (threadIdx.x < MAX_LEVELS && s_hist[threadIdx.x]) atomicAdd(&scal->hist[threadIdx.x], s_hist[threadIdx.x]);
}

// Ladder level of every stride from its streams' bytes at each level:
// the first level within the stride's size limit, else the last
// (Algorithm 2's ratio test, made once per stride).
__global__ void unit_level_kernel(const unsigned long long *bytes, uint8_t *level, unsigned long long nunits,
                                  int nlev, unsigned long long limit) {
    for (unsigned long long u = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; u < nunits;
         u += (unsigned long long)gridDim.x * blockDim.x) {
        int k = nlev - 1;
        for (int lv = nlev - 1; lv >= 0; --lv)
            if (bytes[u * MAX_LEVELS + lv] <= limit) k = lv;
        level[u] = (uint8_t)k;
    }
}

// Recompute the running norm from the per-tile partials (after an import).
__global__ void norm_from_parts_kernel(const unsigned long long *part, unsigned long long ntiles,
                                       DevScalars *scal) {
    unsigned long long lo = 0, hi = 0;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntiles;
         t += (unsigned long long)gridDim.x * blockDim.x)
        add128(lo, hi, part[2 * t], part[2 * t + 1]);
    warp_sum128(lo, hi);
    if ((threadIdx.x & 31) == 0 && (lo | hi)) atomic_add128(&scal->acc_lo, &scal->acc_hi, lo, hi);
}

// Stream sizes of tiles first..first+count-1, or of tiles list[0..count-1]
// when list is not null
__global__ void sizes_kernel(const uint8_t *arena, const unsigned long long *table,
                             unsigned long long first, unsigned long long count,
                             const unsigned long long *list, unsigned long long *sizes) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long t = list ? list[i] : first + i;
        const uint32_t *h = reinterpret_cast<const uint32_t *>(arena + table[t]);
        sizes[i] = HDR + (unsigned long long)h[1];
    }
}

// Sum of the stream sizes of all tiles
__global__ void sum_sizes_kernel(const uint8_t *arena, const unsigned long long *table,
                                 unsigned long long ntiles, unsigned long long *total) {
    unsigned long long s = 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < ntiles;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t *h = reinterpret_cast<const uint32_t *>(arena + table[i]);
        s += HDR + (unsigned long long)h[1];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(total, s);
}

// Gather streams (tiles first.., or list[i] when list is not null) into a
// contiguous buffer at the given offsets
__global__ void gather_kernel(const uint8_t *arena, const unsigned long long *table,
                              unsigned long long first, unsigned long long count,
                              const unsigned long long *list, const unsigned long long *offs,
                              const unsigned long long *sizes, uint8_t *out) {
    for (unsigned long long i = blockIdx.x; i < count; i += gridDim.x) {
        const unsigned long long t = list ? list[i] : first + i;
        const uint4 *s = reinterpret_cast<const uint4 *>(arena + table[t]);
        uint4 *d = reinterpret_cast<uint4 *>(out + offs[i]);
        for (unsigned long long j = threadIdx.x; j < sizes[i] / 16; j += blockDim.x) d[j] = s[j];
    }
}

// Validate imported streams (each at offs[i] in buf, sizes[i] bytes) by
// decoding them; record their norm partials.  bad[0] counts failures.
__global__ void __launch_bounds__(32 * TILE_WARPS) validate_kernel(
    const uint8_t *buf, const unsigned long long *offs, const unsigned long long *sizes,
    unsigned long long count, int c, unsigned long long *parts, unsigned int *bad) {
    extern __shared__ double smem[];
    const int N = 1 << c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *re = smem + (size_t)warp * 2 * N, *im = re + N;
    for (unsigned long long i = (unsigned long long)blockIdx.x * TILE_WARPS + warp; i < count;
         i += (unsigned long long)gridDim.x * TILE_WARPS) {
        const uint8_t *src = buf + offs[i];
        const uint32_t body = reinterpret_cast<const uint32_t *>(src)[1];
        int fail = sizes[i] < HDR || (sizes[i] & 15ull) || HDR + (unsigned long long)body != sizes[i];
        if (!fail) fail = wdecode(src, c, re, im, 1.0, false);
        unsigned long long lo = 0, hi = 0;
        unsigned rng = 0;
        if (!fail) wnorm(re, im, N, lo, hi, rng);
        rng = __any_sync(FULL, rng);
        if (lane == 0) {
            parts[2 * i] = lo;
            parts[2 * i + 1] = hi;
            if (fail || rng) atomicAdd(bad, 1u);
        }
        __syncwarp();
    }
}

// Copy validated streams into the arena and point the table at them.
__global__ void place_kernel(const uint8_t *buf, const unsigned long long *offs,
                             const unsigned long long *sizes, unsigned long long count,
                             unsigned long long first, unsigned long long base, uint8_t *arena,
                             unsigned long long *table, const unsigned long long *parts,
                             unsigned long long *part) {
    for (unsigned long long i = blockIdx.x; i < count; i += gridDim.x) {
        const uint4 *s = reinterpret_cast<const uint4 *>(buf + offs[i]);
        uint4 *d = reinterpret_cast<uint4 *>(arena + base + offs[i]);
        for (unsigned long long j = threadIdx.x; j < sizes[i] / 16; j += blockDim.x) d[j] = s[j];
        if (threadIdx.x == 0) {
            table[first + i] = base + offs[i];
            part[2 * (first + i)] = parts[2 * i];
            part[2 * (first + i) + 1] = parts[2 * i + 1];
        }
    }
}

// Decode tiles covering [start, start+count) into out (interleaved).
__global__ void __launch_bounds__(32 * TILE_WARPS) amplitudes_kernel(
    const uint8_t *arena, const unsigned long long *table, int c, unsigned long long start,
    unsigned long long count, double2 *out, DevScalars *scal) {
    extern __shared__ double smem[];
    const int N = 1 << c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *re = smem + (size_t)warp * 2 * N, *im = re + N;
    const unsigned long long t0 = start >> c, t1 = (start + count - 1) >> c;
    for (unsigned long long t = t0 + (unsigned long long)blockIdx.x * TILE_WARPS + warp; t <= t1;
         t += (unsigned long long)gridDim.x * TILE_WARPS) {
        if (wdecode(arena + table[t], c, re, im, 1.0, false) && lane == 0) atomicOr(&scal->err, ERR_FORMAT);
        __syncwarp();
        for (int i = lane; i < N; i += 32) {
            const unsigned long long gidx = (t << c) | (unsigned long long)i;
            if (gidx >= start && gidx < start + count) out[gidx - start] = make_double2(re[i], im[i]);
        }
        __syncwarp();
    }
}

// Exact per-outcome sums of |a|^2: bucket j gathers bit i of j from qubit qs[i].
// With at most PROBS_SMEM_BUCKETS buckets each CTA sums into shared-memory
// 128-bit buckets (integer adds, so the order does not matter) and adds
// them to the global buckets once at the end; larger bucket counts add
// straight into global memory.
constexpr int PROBS_SMEM_BUCKETS = 1024;
__global__ void __launch_bounds__(32 * TILE_WARPS) probs_kernel(
    const uint8_t *arena, const unsigned long long *table, int c, unsigned long long ntiles,
    const int *qs, int nq, unsigned long long *buckets, DevScalars *scal) {
    extern __shared__ double smem[];
    __shared__ int sq[32];
    __shared__ unsigned long long sb[2 * PROBS_SMEM_BUCKETS];
    const int N = 1 << c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *re = smem + (size_t)warp * 2 * N, *im = re + N;
    const int nb = 1 << nq;
    const bool local = nb <= PROBS_SMEM_BUCKETS;
    if (threadIdx.x < nq) sq[threadIdx.x] = qs[threadIdx.x];
    if (local)
        for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x) sb[i] = 0ull;
    __syncthreads();
    unsigned long long *dst = local ? sb : buckets;
    for (unsigned long long t = (unsigned long long)blockIdx.x * TILE_WARPS + warp; t < ntiles;
         t += (unsigned long long)gridDim.x * TILE_WARPS) {
        if (wdecode(arena + table[t], c, re, im, 1.0, false) && lane == 0) atomicOr(&scal->err, ERR_FORMAT);
        __syncwarp();
        for (int i = lane; i < N; i += 32) {
            const unsigned long long gidx = (t << c) | (unsigned long long)i;
            unsigned j = 0;
            for (int b = 0; b < nq; ++b) j |= (unsigned)((gidx >> sq[b]) & 1ull) << b;
            unsigned long long l0, h0, l1, h1;
            unsigned rng = 0;
            sq_units(dbits(re[i]), l0, h0, rng);
            sq_units(dbits(im[i]), l1, h1, rng);
            add128(l0, h0, l1, h1);
            if (l0 | h0) atomic_add128(&dst[2 * j], &dst[2 * j + 1], l0, h0);
        }
        __syncwarp();
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x)
            if (sb[2 * i] | sb[2 * i + 1]) atomic_add128(&buckets[2 * i], &buckets[2 * i + 1], sb[2 * i], sb[2 * i + 1]);
    }
}

// Fidelity partials: <ref|psi> (re, im), <psi|psi>, <ref|ref>, each summed
// over a tile in a fixed order (lane chunks, then a pairwise shuffle tree),
// then over chunks of `chunk` consecutive tiles (a power of two, at most
// FID_CHUNK) by the same pairwise tree in shared memory: chunk_sums[q] is
// the subtree of tiles q*chunk .. q*chunk+chunk-1, so finishing the tree
// over the chunk sums gives the perfect binary tree over all tiles.
constexpr int FID_CHUNK = 1024;
__global__ void __launch_bounds__(32 * TILE_WARPS) fidelity_kernel(
    const uint8_t *arena, const unsigned long long *table, int c, unsigned long long ntiles,
    int chunk, RefSpec rs, Acc4 *chunk_sums, DevScalars *scal) {
    extern __shared__ double smem[];
    __shared__ Acc4 ssum[FID_CHUNK];
    const int N = 1 << c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *re = smem + (size_t)warp * 4 * N, *im = re + N, *rre = re + 2 * N, *rim = re + 3 * N;
    const unsigned long long nchunks = ntiles / (unsigned long long)chunk;
    for (unsigned long long ck = blockIdx.x; ck < nchunks; ck += gridDim.x) {
    for (unsigned long long t = ck * chunk + warp; t < (ck + 1) * chunk; t += TILE_WARPS) {
        int bad = wdecode(arena + table[t], c, re, im, 1.0, false);
        if (rs.kind == 0) bad |= wdecode(rs.o_arena + rs.o_table[t], c, rre, rim, 1.0, false);
        if (bad && lane == 0) atomicOr(&scal->err, ERR_FORMAT);
        __syncwarp();
        Acc4 acc = make_acc4(0, 0, 0, 0);
        const int per = (N + 31) / 32;
        for (int q = 0; q < per; ++q) {
            const int i = lane * per + q;
            if (i >= N) break;
            const unsigned long long gidx = (t << c) | (unsigned long long)i;
            double ar, ai;
            if (rs.kind == 0) { ar = rre[i]; ai = rim[i]; }
            else if (rs.kind == 1) {
                const unsigned long long Nn = 1ull << rs.n;
                const unsigned long long ph = (rs.x * gidx) & (Nn - 1ull);
                double sn, cs;
                sincospi(ldexp((double)ph, 1 - rs.n), &sn, &cs);
                ar = cs * rs.qft_mag;
                ai = sn * rs.qft_mag;
            } else if (rs.kind == 2) {
                ar = gidx == rs.x ? rs.grov_m : rs.grov_o;
                ai = 0.0;
            } else {
                const double2 v = rs.dense[gidx];
                ar = v.x;
                ai = v.y;
            }
            const double pr = re[i], pi = im[i];
            acc.x = __fma_rn(ar, pr, __fma_rn(ai, pi, acc.x));     // Re <ref|psi>
            acc.y = __fma_rn(ar, pi, __fma_rn(-ai, pr, acc.y));    // Im <ref|psi>
            acc.z = __fma_rn(pr, pr, __fma_rn(pi, pi, acc.z));
            acc.w = __fma_rn(ar, ar, __fma_rn(ai, ai, acc.w));
        }
        for (int o = 1; o < 32; o <<= 1) {
            const double bx = __shfl_down_sync(FULL, acc.x, o), by = __shfl_down_sync(FULL, acc.y, o);
            const double bz = __shfl_down_sync(FULL, acc.z, o), bw = __shfl_down_sync(FULL, acc.w, o);
            if ((lane & (2 * o - 1)) == 0) { acc.x += bx; acc.y += by; acc.z += bz; acc.w += bw; }
        }
        if (lane == 0) ssum[t - ck * chunk] = acc;
        __syncwarp();
    }
    __syncthreads();
    for (int w = 1; w < chunk; w <<= 1) {
        for (int i = threadIdx.x * 2 * w; i < chunk; i += blockDim.x * 2 * w) {
            const Acc4 x = ssum[i], y = ssum[i + w];
            ssum[i] = make_acc4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_sums[ck] = ssum[0];
    __syncthreads();
    }
}

// One level of a pairwise tree: out[i] = in[2i] + in[2i+1]
__global__ void pair_sum_kernel(const Acc4 *in, Acc4 *out, unsigned long long nout) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nout;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const Acc4 a = in[2 * i], b = in[2 * i + 1];
        out[i] = make_acc4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
}

}  // namespace qs

// ---------------------------------------------------------------- launchers
namespace qs {

// dynamic shared memory of a sweep CTA: the item buffer (planar re / im)
// and a 256-byte packing stage per warp
size_t sweep_smem_bytes(int mb, int threads) { return ((size_t)16 << mb) + 256u * (size_t)(threads / 32); }

// the sweep kernel's launch shapes: threads per CTA and the CTAs per SM its
// register budget is compiled for (80 registers at 256 x 3)
bool sweep_threads_ok(int threads) { return threads == 128 || threads == 256 || threads == 512; }
static size_t tile_smem_bytes(int c, int bufs) { return (size_t)TILE_WARPS * bufs * (16u << c); }

template <bool SIZING>
static cudaError_t launch_sweep_shape(const SweepParams *plist, const unsigned long long *istart, int nlist,
                                      int mb, int grid, int threads, unsigned long long *work, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const size_t sm = sweep_smem_bytes(mb, threads);
    switch (threads) {
        case 128: sweep_kernel<SIZING, 128, 3><<<grid, 128, sm, st>>>(plist, istart, nlist, work); break;
        case 512: sweep_kernel<SIZING, 512, 1><<<grid, 512, sm, st>>>(plist, istart, nlist, work); break;
        default: sweep_kernel<SIZING, 256, 3><<<grid, 256, sm, st>>>(plist, istart, nlist, work); break;
    }
    return cudaGetLastError();
}

// work: the launch's item counter, zeroed on st before the launch.
cudaError_t launch_sweep(const SweepParams *plist, const unsigned long long *istart, int nlist,
                         int mb, int grid, int threads, unsigned long long *work, cudaStream_t st) {
    return launch_sweep_shape<false>(plist, istart, nlist, mb, grid, threads, work, st);
}

cudaError_t launch_sweep_sizing(const SweepParams *plist, const unsigned long long *istart, int nlist,
                                int mb, int grid, int threads, unsigned long long *work, cudaStream_t st) {
    return launch_sweep_shape<true>(plist, istart, nlist, mb, grid, threads, work, st);
}

cudaError_t launch_finalize(DevScalars *scal, int use_alpha, unsigned long long *used_hist,
                            unsigned slot, int record_used, cudaStream_t st) {
    FinalizeEntry f{scal, used_hist, slot, use_alpha, record_used};
    finalize_kernel<<<1, 32, 0, st>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_finalize_list(const FinalizeEntry *list, int n, cudaStream_t st) {
    finalize_list_kernel<<<(n + 127) / 128, 128, 0, st>>>(list, n);
    return cudaGetLastError();
}

static int tile_grid(int grid, unsigned long long ntiles) {
    unsigned long long need = (ntiles + TILE_WARPS - 1) / TILE_WARPS;
    unsigned long long g = (unsigned long long)grid;
    if (need < g) g = need;
    return g ? (int)g : 1;
}

cudaError_t launch_init(const double2 *dense, unsigned long long x, const CodecCfg &cc,
                        unsigned long long ntiles, uint8_t *arena, unsigned long long cap,
                        unsigned long long *table, unsigned long long *part, DevScalars *scal,
                        unsigned long long *unit_bytes, const uint8_t *unit_level, int unit_shift,
                        int grid, cudaStream_t st) {
    init_kernel<<<tile_grid(grid, ntiles), 32 * TILE_WARPS, tile_smem_bytes(cc.c, 1), st>>>(
        dense, x, cc, ntiles, arena, cap, table, part, scal, unit_bytes, unit_level, unit_shift);
    return cudaGetLastError();
}

cudaError_t launch_unit_level(const unsigned long long *bytes, uint8_t *level, unsigned long long nunits,
                              int nlev, unsigned long long limit, cudaStream_t st) {
    const unsigned long long g = (nunits + THREADS - 1) / THREADS;
    unit_level_kernel<<<g < 4096ull ? (int)g : 4096, THREADS, 0, st>>>(bytes, level, nunits, nlev, limit);
    return cudaGetLastError();
}

cudaError_t launch_norm_from_parts(const unsigned long long *part, unsigned long long ntiles,
                                   DevScalars *scal, int grid, cudaStream_t st) {
    norm_from_parts_kernel<<<grid, THREADS, 0, st>>>(part, ntiles, scal);
    return cudaGetLastError();
}

cudaError_t launch_sizes(const uint8_t *arena, const unsigned long long *table,
                         unsigned long long first, unsigned long long count, const unsigned long long *list,
                         unsigned long long *sizes, int grid, cudaStream_t st) {
    sizes_kernel<<<grid, THREADS, 0, st>>>(arena, table, first, count, list, sizes);
    return cudaGetLastError();
}

cudaError_t launch_sum_sizes(const uint8_t *arena, const unsigned long long *table,
                             unsigned long long ntiles, unsigned long long *total, int grid,
                             cudaStream_t st) {
    sum_sizes_kernel<<<grid, THREADS, 0, st>>>(arena, table, ntiles, total);
    return cudaGetLastError();
}

cudaError_t launch_gather(const uint8_t *arena, const unsigned long long *table,
                          unsigned long long first, unsigned long long count, const unsigned long long *list,
                          const unsigned long long *offs, const unsigned long long *sizes,
                          uint8_t *out, int grid, cudaStream_t st) {
    gather_kernel<<<grid, THREADS, 0, st>>>(arena, table, first, count, list, offs, sizes, out);
    return cudaGetLastError();
}

cudaError_t launch_validate(const uint8_t *buf, const unsigned long long *offs,
                            const unsigned long long *sizes, unsigned long long count, int c,
                            unsigned long long *parts, unsigned int *bad, int grid, cudaStream_t st) {
    validate_kernel<<<tile_grid(grid, count), 32 * TILE_WARPS, tile_smem_bytes(c, 1), st>>>(
        buf, offs, sizes, count, c, parts, bad);
    return cudaGetLastError();
}

cudaError_t launch_place(const uint8_t *buf, const unsigned long long *offs,
                         const unsigned long long *sizes, unsigned long long count,
                         unsigned long long first, unsigned long long base, uint8_t *arena,
                         unsigned long long *table, const unsigned long long *parts,
                         unsigned long long *part, int grid, cudaStream_t st) {
    place_kernel<<<grid, THREADS, 0, st>>>(buf, offs, sizes, count, first, base, arena, table, parts,
                                           part);
    return cudaGetLastError();
}

cudaError_t launch_amplitudes(const uint8_t *arena, const unsigned long long *table, int c,
                              unsigned long long start, unsigned long long count, double2 *out,
                              DevScalars *scal, int grid, cudaStream_t st) {
    const unsigned long long tiles = ((start + count - 1) >> c) - (start >> c) + 1;
    amplitudes_kernel<<<tile_grid(grid, tiles), 32 * TILE_WARPS, tile_smem_bytes(c, 1), st>>>(
        arena, table, c, start, count, out, scal);
    return cudaGetLastError();
}

cudaError_t launch_probs(const uint8_t *arena, const unsigned long long *table, int c,
                         unsigned long long ntiles, const int *qsel, int nq,
                         unsigned long long *buckets, DevScalars *scal, int grid, cudaStream_t st) {
    probs_kernel<<<tile_grid(grid, ntiles), 32 * TILE_WARPS, tile_smem_bytes(c, 1), st>>>(
        arena, table, c, ntiles, qsel, nq, buckets, scal);
    return cudaGetLastError();
}

// chunk sums land in chunk_sums[0 .. ntiles/fidelity_chunk(ntiles) - 1]
unsigned long long fidelity_chunk(unsigned long long ntiles) {
    return ntiles < (unsigned long long)FID_CHUNK ? ntiles : (unsigned long long)FID_CHUNK;
}

cudaError_t launch_fidelity(const uint8_t *arena, const unsigned long long *table, int c,
                            unsigned long long ntiles, const RefSpec &rs, Acc4 *chunk_sums,
                            DevScalars *scal, int grid, cudaStream_t st) {
    const unsigned long long ch = fidelity_chunk(ntiles);
    const unsigned long long nchunks = ntiles / ch;
    const int g = (unsigned long long)grid < nchunks ? grid : (int)nchunks;
    fidelity_kernel<<<g, 32 * TILE_WARPS, tile_smem_bytes(c, 2), st>>>(
        arena, table, c, ntiles, (int)ch, rs, chunk_sums, scal);
    return cudaGetLastError();
}

cudaError_t launch_run_tables(const DRun *runs, const int2 *classes, int nclasses, const RGate *rgates, int c,
                              double2 *tab, uint8_t *meta, RunClass *rcls, DevScalars *scal, int grid,
                              cudaStream_t st) {
    run_tables_kernel<<<grid < nclasses ? grid : nclasses, 256, 0, st>>>(runs, classes, nclasses, rgates, c, tab,
                                                                       meta, rcls, scal);
    return cudaGetLastError();
}

cudaError_t launch_sweep_scales(const SGate *sg, const DGate *dg, const int2 *bounds, int ns, double *D,
                                cudaStream_t st) {
    sweep_scale_kernel<<<(ns + 127) / 128, 128, 0, st>>>(sg, dg, bounds, ns, D);
    return cudaGetLastError();
}

cudaError_t launch_pair_sum(const Acc4 *in, Acc4 *out, unsigned long long nout, int grid,
                            cudaStream_t st) {
    pair_sum_kernel<<<grid, THREADS, 0, st>>>(in, out, nout);
    return cudaGetLastError();
}

// Fixed point with 124 fractional bits: arctan(1/n) = sum over j of
// (-1)^j / ((2j+1) n^(2j+1)), the positive and the negative terms summed
// apart (each truncated; the total error stays far below 2^-100).
static unsigned __int128 host_atan_recip(unsigned long long n) {
    const unsigned __int128 one = (unsigned __int128)1 << 124;
    unsigned __int128 pos = 0, neg = 0, pw = one / n;
    const unsigned __int128 n2 = (unsigned __int128)n * n;
    for (unsigned long long j = 0; pw != 0; ++j, pw /= n2) {
        if (j & 1) neg += pw / (2 * j + 1);
        else pos += pw / (2 * j + 1);
    }
    return pos - neg;
}

// The POLAR mode's CORDIC table: atan(2^-k) / (2 pi) in units of 2^-64
// turn, rounded to nearest; k = 0 is exactly 1/8 turn, pi comes from
// Machin's formula pi/4 = 4 atan(1/5) - atan(1/239).
static void host_polar_table(unsigned long long *t) {
    const unsigned __int128 quarter_pi = 4 * host_atan_recip(5) - host_atan_recip(239);
    const unsigned __int128 two_pi = 8 * quarter_pi;
    t[0] = 1ull << 61;
    for (int k = 1; k < POLAR_ITERS; ++k) {
        unsigned __int128 rem = host_atan_recip(1ull << k);          // < two_pi
        unsigned long long q = 0;
        for (int i = 0; i < 64; ++i) {                                // floor(rem * 2^64 / two_pi)
            rem <<= 1;
            q <<= 1;
            if (rem >= two_pi) { rem -= two_pi; q |= 1ull; }
        }
        t[k] = q + (2 * rem >= two_pi ? 1ull : 0ull);                 // round to nearest
    }
}

// Kernel attributes of the current device (dynamic shared memory above
// 48 KiB) and the POLAR table in its constant memory, set once per device:
// attributes apply to the device that is current when they are set.
static cudaError_t configure_current_device() {
    cudaError_t e;
    unsigned long long tab[POLAR_ITERS];
    host_polar_table(tab);
    if ((e = cudaMemcpyToSymbol(c_polar_atan, tab, sizeof tab))) return e;
    const int sm128 = (int)sweep_smem_bytes(MAX_ITEM_LOG2, 128), sm256 = (int)sweep_smem_bytes(MAX_ITEM_LOG2, 256),
              sm512 = (int)sweep_smem_bytes(MAX_ITEM_LOG2, 512);
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(sweep_kernel<false, 128, 3>, A, sm128))) return e;
    if ((e = cudaFuncSetAttribute(sweep_kernel<true, 128, 3>, A, sm128))) return e;
    if ((e = cudaFuncSetAttribute(sweep_kernel<false, 256, 3>, A, sm256))) return e;
    if ((e = cudaFuncSetAttribute(sweep_kernel<true, 256, 3>, A, sm256))) return e;
    if ((e = cudaFuncSetAttribute(sweep_kernel<false, 512, 1>, A, sm512))) return e;
    if ((e = cudaFuncSetAttribute(sweep_kernel<true, 512, 1>, A, sm512))) return e;
    const int t1 = (int)tile_smem_bytes(MAX_C, 1), t2 = (int)tile_smem_bytes(MAX_C, 2);
    if ((e = cudaFuncSetAttribute(init_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t1))) return e;
    if ((e = cudaFuncSetAttribute(validate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t1))) return e;
    if ((e = cudaFuncSetAttribute(amplitudes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t1))) return e;
    if ((e = cudaFuncSetAttribute(probs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t1))) return e;
    if ((e = cudaFuncSetAttribute(fidelity_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t2))) return e;
    return cudaSuccess;
}

constexpr int MAX_CONFIG_DEVICES = 64;
static std::once_flag g_config_once[MAX_CONFIG_DEVICES];
static cudaError_t g_config_err[MAX_CONFIG_DEVICES];

cudaError_t configure_kernels() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_CONFIG_DEVICES) return cudaErrorInvalidDevice;
    std::call_once(g_config_once[dev], [dev] { g_config_err[dev] = configure_current_device(); });
    return g_config_err[dev];
}

cudaError_t fp64_rate(int device, double *fma_per_s) {
    cudaError_t e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device))) return e;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(double) * blocks * threads))) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fp64_rate_kernel<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);    // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) fp64_rate_kernel<<<blocks, threads>>>(out, iters, 0.999999, 1e-9);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e == cudaSuccess) *fma_per_s = 5.0 * blocks * threads * iters * 8.0 / (ms * 1e-3);
    return e;
}

int sweep_blocks_per_sm(int mb, int threads) {
    int nb = 0;
    const size_t sm = sweep_smem_bytes(mb, threads);
    if (threads == 128) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<false, 128, 3>, 128, sm);
    else if (threads == 512) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<false, 512, 1>, 512, sm);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<false, 256, 3>, 256, sm);
    return nb > 0 ? nb : 1;
}

}  // namespace qs
