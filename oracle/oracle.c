/*
 * CPU oracle for the compressed full-amplitude simulator (test infrastructure).
 *
 * This file is the slow, plain, obviously-correct CPU statement of what the
 * GPU library computes.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Contents
 *   O1  dense simulator: the pair / quad update of Sec. II (single-qubit
 *       gate on qubit k, controlled gate), applied to a full 2^n vector.
 *   O2  tile codec: the amplitude-aware, point-wise relative error-bounded
 *       codec (Sec. III, SZ with a relative bound as in ref. [xin2018]) in
 *       the stream format below, plus the lossless level and the AALC
 *       error-bound ladder of Algorithm 2.
 *   O3  compressed simulator: Algorithm 2 (decompress, normalize, gate
 *       computation, compress with the error-bound ladder) over tiles, one
 *       sweep (a run of gates) at a time; a sweep whose gates only permute
 *       whole tiles moves their streams instead (sweep_moves_tiles).  The
 *       ladder's ratio test is made per tile, or once per stride of
 *       several tiles as Algorithm 2 prints it (or_csim_set_unit); single
 *       items (or_item_sweep) and single strides (or_stride_sweep) can be
 *       recomputed on their own for sampled checks of large states.
 *   N   the state norm used by "normalize": the exact sum of |a|^2 in
 *       fixed point (units of 2^-112), rounded once to double.
 *
 * Arithmetic conventions (both the oracle and the GPU follow them, each in
 * its own code):
 *   - a matrix row is evaluated over its exactly-nonzero entries in column
 *     order; the first term is a product, later terms are fused
 *     multiply-adds; an entry with zero imaginary part is "real", one with
 *     zero real part "imaginary", any other "general"; a row whose nonzero
 *     entries are all d, -d, i d or -i d for its first entry d is summed
 *     first and multiplied by d once (see row_eval);
 *   - compiled with -ffp-contract=off so that only the fma() calls fuse.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* gates                                                               */
/* ------------------------------------------------------------------ */

/* One gate: k targets (1 or 2), controls as a mask over global index
 * bits with the required values, and the 2^k x 2^k complex matrix in
 * row-major order with (re, im) interleaved.  Sub-index bit i of a row or
 * column selects the value of qubit t[i]. */
typedef struct {
    int32_t k;
    int32_t t[2];
    int32_t pad;
    uint64_t cmask;
    uint64_t cval;
    double m[32];
} or_gate;

/* y = u * x for one matrix entry u (Sec. II pair update, one term). */
static void term_first(double ur, double ui, double xr, double xi,
                       double *yr, double *yi)
{
    if (ui == 0.0) {            /* real entry */
        *yr = ur * xr;
        *yi = ur * xi;
    } else if (ur == 0.0) {     /* imaginary entry: (i ui)(xr + i xi) */
        *yr = -(ui * xi);
        *yi = ui * xr;
    } else {                    /* general entry */
        *yr = fma(ur, xr, -(ui * xi));
        *yi = fma(ur, xi, ui * xr);
    }
}

/* acc += u * x for one matrix entry u. */
static void term_acc(double ur, double ui, double xr, double xi,
                     double *ar, double *ai)
{
    if (ui == 0.0) {
        *ar = fma(ur, xr, *ar);
        *ai = fma(ur, xi, *ai);
    } else if (ur == 0.0) {
        *ar = fma(-ui, xi, *ar);
        *ai = fma(ui, xr, *ai);
    } else {
        *ar = fma(ur, xr, fma(-ui, xi, *ar));
        *ai = fma(ur, xi, fma(ui, xr, *ai));
    }
}

/* Factor of entry (ur, ui) relative to d = (dr, di), exact comparisons:
 * 0 when u == d, 1 when u == -d, 2 when u == i d, 3 when u == -i d, -1
 * otherwise (the first match counts). */
static int unit_factor(double ur, double ui, double dr, double di)
{
    if (ur == dr && ui == di) return 0;
    if (ur == -dr && ui == -di) return 1;
    if (ur == -di && ui == dr) return 2;
    if (ur == di && ui == -dr) return 3;
    return -1;
}

/* Row r of y = U x over the present sub-indices, skipping exactly-zero
 * entries.  A row with no nonzero present entry gives +0.
 *
 * Factored rows: when a row has two or more nonzero entries and each one
 * is f_j d with f_j in {1, -1, i, -i} and d the row's first nonzero entry,
 * the row is evaluated as y = d * S with S = sum_j f_j x_j: S starts as the
 * first term (an exact copy) and each later term is one rounded addition
 * per component; then y is one term_first of d and S.  Mathematically this
 * is the same row; in rounding it makes equal inputs cancel exactly (a
 * Hadamard row on two equal amplitudes gives an exact zero).  Every other
 * row: the first term is a product, later terms fused multiply-adds. */
static void row_eval(const double *m, int dim, int r, const double *x,
                     const int *present, int unscaled, double *yr, double *yi)
{
    int first = -1, count = 0, factored = 1;
    for (int c = 0; c < dim; ++c) {
        double ur = m[2 * (r * dim + c)], ui = m[2 * (r * dim + c) + 1];
        if (ur == 0.0 && ui == 0.0) continue;
        ++count;
        if (first < 0) first = c;
        else if (unit_factor(ur, ui, m[2 * (r * dim + first)], m[2 * (r * dim + first) + 1]) < 0)
            factored = 0;
    }
    if (count >= 2 && factored) {
        double dr = m[2 * (r * dim + first)], di = m[2 * (r * dim + first) + 1];
        double sr = 0.0, si = 0.0;
        int started = 0;
        for (int c = 0; c < dim; ++c) {
            double ur = m[2 * (r * dim + c)], ui = m[2 * (r * dim + c) + 1];
            if (!present[c] || (ur == 0.0 && ui == 0.0)) continue;
            double xr = x[2 * c], xi = x[2 * c + 1];
            int f = unit_factor(ur, ui, dr, di);
            /* f x: 1 -> x, -1 -> -x, i -> (-xi, xr), -i -> (xi, -xr) */
            double tr = f == 0 ? xr : (f == 1 ? -xr : (f == 2 ? -xi : xi));
            double ti = f == 0 ? xi : (f == 1 ? -xi : (f == 2 ? xr : -xr));
            if (!started) { sr = tr; si = ti; started = 1; }
            else { sr = sr + tr; si = si + ti; }
        }
        if (!started) { *yr = 0.0; *yi = 0.0; return; }
        if (unscaled) { *yr = sr; *yi = si; return; }     /* d taken out of the sweep (scaled gates) */
        term_first(dr, di, sr, si, yr, yi);
        return;
    }
    int firstt = 1;
    double ar = 0.0, ai = 0.0;
    for (int c = 0; c < dim; ++c) {
        if (!present[c]) continue;
        double ur = m[2 * (r * dim + c)], ui = m[2 * (r * dim + c) + 1];
        if (ur == 0.0 && ui == 0.0) continue;
        if (firstt) {
            term_first(ur, ui, x[2 * c], x[2 * c + 1], &ar, &ai);
            firstt = 0;
        } else {
            term_acc(ur, ui, x[2 * c], x[2 * c + 1], &ar, &ai);
        }
    }
    *yr = ar;
    *yi = ai;
}

static int gate_is_diagonal(const or_gate *g)
{
    int dim = 1 << g->k;
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c)
            if (r != c && (g->m[2 * (r * dim + c)] != 0.0 ||
                           g->m[2 * (r * dim + c) + 1] != 0.0))
                return 0;
    return 1;
}

/*
 * Apply one gate to a buffer of 2^mb amplitudes (re, im interleaved).
 * Buffer index bit p holds global qubit qb[p]; every other qubit has the
 * value it has in 'fixed' (bits at global positions).  A target that is
 * not in the buffer is allowed only for a diagonal gate.
 * Returns 0, or -1 when a non-diagonal gate has a target outside the buffer.
 */
static int apply_gate_rows(double *a, int mb, const int *qb, uint64_t fixed,
                           const or_gate *g, int unscaled);

static int apply_gate_buf(double *a, int mb, const int *qb, uint64_t fixed,
                          const or_gate *g)
{
    return apply_gate_rows(a, mb, qb, fixed, g, 0);
}

/* apply_gate_buf, with unscaled set: every factored row yields its sum S
 * without the final multiplication by its first entry d (the scaled gates
 * of a sweep, see gate_scale), and a group of 2^k amplitudes that are all
 * exactly zero (either sign) is left as it is: its sums are zeros, and only
 * the IEEE sign of a zero could differ from forming them. */
static int apply_gate_rows(double *a, int mb, const int *qb, uint64_t fixed,
                           const or_gate *g, int unscaled)
{
    int k = g->k, dim = 1 << k;
    int pos[2] = {-1, -1};
    for (int i = 0; i < k; ++i)
        for (int p = 0; p < mb; ++p)
            if (qb[p] == g->t[i]) pos[i] = p;
    int diag = gate_is_diagonal(g);
    for (int i = 0; i < k; ++i)
        if (pos[i] < 0 && !diag) return -1;

    uint64_t nb = 1ull << mb;
    double x[8], y[8];
    int present[4];
    uint64_t idx[4];
    for (uint64_t l = 0; l < nb; ++l) {
        int skip = 0;
        for (int i = 0; i < k; ++i)
            if (pos[i] >= 0 && ((l >> pos[i]) & 1)) skip = 1;
        if (skip) continue;
        uint64_t gl = fixed;
        for (int p = 0; p < mb; ++p)
            if ((l >> p) & 1) gl |= 1ull << qb[p];
        if ((gl & g->cmask) != g->cval) continue;
        /* gather the sub-vector; sub-indices whose fixed target bits do
         * not match this buffer are absent */
        for (int s = 0; s < dim; ++s) {
            present[s] = 1;
            idx[s] = l;
            for (int i = 0; i < k; ++i) {
                int bit = (s >> i) & 1;
                if (pos[i] >= 0) {
                    if (bit) idx[s] |= 1ull << pos[i];
                } else if ((int)((fixed >> g->t[i]) & 1) != bit) {
                    present[s] = 0;
                }
            }
            if (present[s]) {
                x[2 * s] = a[2 * idx[s]];
                x[2 * s + 1] = a[2 * idx[s] + 1];
            } else {
                x[2 * s] = 0.0;
                x[2 * s + 1] = 0.0;
            }
        }
        if (unscaled) {
            /* a scaled gate leaves a group of exactly-zero amplitudes as it is */
            int nz = 0;
            for (int j = 0; j < 2 * dim; ++j) nz |= x[j] != 0.0;
            if (!nz) continue;
        }
        for (int r = 0; r < dim; ++r)
            if (present[r]) row_eval(g->m, dim, r, x, present, unscaled, &y[2 * r], &y[2 * r + 1]);
        for (int r = 0; r < dim; ++r)
            if (present[r]) {
                a[2 * idx[r]] = y[2 * r];
                a[2 * idx[r] + 1] = y[2 * r + 1];
            }
    }
    return 0;
}

/*
 * Diagonal runs (the O3 gate computation; reading of the sweep's fused
 * gate run).  Two or more consecutive diagonal gates of a sweep form one
 * diagonal operator: its entry at index x is the product of the gates'
 * entries there, and the amplitude is multiplied by it once.  This is the
 * product of the run's matrices, written out with one fixed rounding order:
 *   - a gate contributes at x when its controls hold there; its factor is
 *     its diagonal entry at x's target sub-index, and a factor exactly 1
 *     contributes nothing;
 *   - factors exactly -1, i or -i ("units") are collected as a power i^k
 *     (exact: sign flips and swaps of the components);
 *   - the other factors are multiplied left to right in gate order, each new
 *     factor u applied to the running product p as the general complex
 *     term u*p; gates whose targets and controls are all qubits >= c
 *     (constant over a tile) form one product T, every other gate another
 *     product L;
 *   - the amplitude a becomes i^k * (G a) with G = T*L (T applied to L) when
 *     both exist, else the one that exists, and i^k * a when neither does;
 *   - an amplitude that is exactly zero (both components +0 or -0) is left
 *     as it is (every factor keeps it zero; only the IEEE sign of a zero
 *     could differ from multiplying it).
 * Mathematically the same operator as the gates one after the other
 * (Sec. II pair update for diagonal matrices); in rounding it multiplies
 * every amplitude twice at most, whatever the run's length.
 */

/* general complex term y = u * x (the rounding of term_first's general case) */
static void cmul(double ur, double ui, double xr, double xi, double *yr, double *yi)
{
    double r = fma(ur, xr, -(ui * xi));
    double i = fma(ur, xi, ui * xr);
    *yr = r;
    *yi = i;
}

/* exponent k with u == i^k for u in {-1, i, -i} (exact comparisons), else -1 */
static int unit_exponent(double ur, double ui)
{
    if (ur == -1.0 && ui == 0.0) return 2;
    if (ur == 0.0 && ui == 1.0) return 1;
    if (ur == 0.0 && ui == -1.0) return 3;
    return -1;
}

/* x <- i^k x, exact */
static void unit_apply(int k, double *xr, double *xi)
{
    double r = *xr, i = *xi;
    switch (k & 3) {
        case 1: *xr = -i; *xi = r; break;
        case 2: *xr = -r; *xi = -i; break;
        case 3: *xr = i; *xi = -r; break;
        default: break;
    }
}

/* every target and control of g is a qubit >= c */
static int gate_on_high_qubits(const or_gate *g, int c)
{
    if (g->cmask & ((1ull << c) - 1)) return 0;
    for (int i = 0; i < g->k; ++i)
        if (g->t[i] < c) return 0;
    return 1;
}

/* One diagonal run (gates g[0..ng-1], all diagonal) applied to a buffer as
 * apply_gate_buf addresses it. */
static void apply_diag_run(double *a, int mb, const int *qb, uint64_t fixed, const or_gate *g, int ng,
                           int c)
{
    uint64_t nb = 1ull << mb;
    for (uint64_t l = 0; l < nb; ++l) {
        if (a[2 * l] == 0.0 && a[2 * l + 1] == 0.0) continue;     /* a zero stays as it is */
        uint64_t gl = fixed;
        for (int p = 0; p < mb; ++p)
            if ((l >> p) & 1) gl |= 1ull << qb[p];
        int k = 0, have_t = 0, have_l = 0;
        double tr = 0.0, ti = 0.0, lr = 0.0, li = 0.0;
        for (int i = 0; i < ng; ++i) {
            if ((gl & g[i].cmask) != g[i].cval) continue;
            int dim = 1 << g[i].k, r = 0;
            for (int j = 0; j < g[i].k; ++j) r |= (int)((gl >> g[i].t[j]) & 1) << j;
            double ur = g[i].m[2 * (r * dim + r)], ui = g[i].m[2 * (r * dim + r) + 1];
            if (ur == 1.0 && ui == 0.0) continue;
            int e = unit_exponent(ur, ui);
            if (e >= 0) { k += e; continue; }
            if (gate_on_high_qubits(&g[i], c)) {
                if (have_t) cmul(ur, ui, tr, ti, &tr, &ti);
                else { tr = ur; ti = ui; have_t = 1; }
            } else {
                if (have_l) cmul(ur, ui, lr, li, &lr, &li);
                else { lr = ur; li = ui; have_l = 1; }
            }
        }
        double xr = a[2 * l], xi = a[2 * l + 1];
        if (have_t || have_l) {
            double gr = have_t ? tr : lr, gi = have_t ? ti : li;
            if (have_t && have_l) cmul(tr, ti, lr, li, &gr, &gi);
            cmul(gr, gi, xr, xi, &xr, &xi);
        }
        unit_apply(k, &xr, &xi);
        a[2 * l] = xr;
        a[2 * l + 1] = xi;
    }
}

/*
 * Scaled gates (the O3 gate computation, with fuse set): a gate without
 * controls whose every row has two or more nonzero entries, each its
 * first nonzero entry d times 1, -1, i or -i, with the same real d in every
 * row (a Hadamard; H (x) H), is d times a matrix of units.  A scalar commutes
 * with every linear map, so a sweep applies the product D of its scaled
 * gates' d (multiplied in gate order, starting from 1) together with the
 * normalize scale at decompression, a * (alpha * D), and each scaled gate
 * only forms its rows' unit sums.  Returns d for a scaled gate, else 0.
 */
static double gate_scale(const or_gate *g)
{
    if (g->cmask || gate_is_diagonal(g)) return 0.0;
    int dim = 1 << g->k;
    double d = 0.0;
    for (int r = 0; r < dim; ++r) {
        int first = -1, count = 0;
        for (int c = 0; c < dim; ++c) {
            double ur = g->m[2 * (r * dim + c)], ui = g->m[2 * (r * dim + c) + 1];
            if (ur == 0.0 && ui == 0.0) continue;
            ++count;
            if (first < 0) first = c;
            else if (unit_factor(ur, ui, g->m[2 * (r * dim + first)], g->m[2 * (r * dim + first) + 1]) < 0)
                return 0.0;
        }
        if (count < 2) return 0.0;
        double dr = g->m[2 * (r * dim + first)], di = g->m[2 * (r * dim + first) + 1];
        if (di != 0.0) return 0.0;
        if (r == 0) d = dr;
        else if (memcmp(&dr, &d, sizeof d) != 0) return 0.0;
    }
    return d;
}

/* D of a sweep: the product of its scaled gates' d in gate order (1 when
 * fuse is off or there are none). */
static double sweep_scale(const or_gate *g, int ng, int fuse)
{
    double D = 1.0;
    if (!fuse) return D;
    for (int i = 0; i < ng; ++i) {
        double d = gate_scale(&g[i]);
        if (d != 0.0) D = D * d;
    }
    return D;
}

/* A sweep's gates applied to an item buffer in order: with fuse set, each
 * run of two or more consecutive diagonal gates as one diagonal operator
 * (apply_diag_run) and each scaled gate without its d (the sweep applies D
 * at decompression), every other gate on its own.  Returns 0, or -1 when a
 * non-diagonal gate has a target outside the buffer. */
static int apply_gates_buf(double *a, int mb, const int *qb, uint64_t fixed, const or_gate *g, int ng,
                           int c, int fuse)
{
    int i = 0;
    while (i < ng) {
        int j = i;
        if (fuse)
            while (j < ng && gate_is_diagonal(&g[j])) ++j;
        if (j - i >= 2) {
            apply_diag_run(a, mb, qb, fixed, g + i, j - i, c);
            i = j;
            continue;
        }
        if (apply_gate_rows(a, mb, qb, fixed, &g[i], fuse && gate_scale(&g[i]) != 0.0) != 0) return -1;
        ++i;
    }
    return 0;
}

/* O1: apply a gate to a dense 2^n state (qubit j <-> index bit j). */
int or_dense_apply(double *psi, int n, const or_gate *g)
{
    int qb[64];
    for (int p = 0; p < n; ++p) qb[p] = p;
    return apply_gate_buf(psi, n, qb, 0, g);
}

/* ------------------------------------------------------------------ */
/* norm: exact sum of squares in units of 2^-112                        */
/* ------------------------------------------------------------------ */

#define NORM_FRAC 112

static uint64_t dbits(double x) { uint64_t u; memcpy(&u, &x, 8); return u; }
static double bitsd(uint64_t u) { double x; memcpy(&x, &u, 8); return x; }

/* floor(x^2 * 2^112).  Sets *range when |x| >= 16 (outside the format). */
static u128 sq_units(double x, int *range)
{
    uint64_t u = dbits(x) & 0x7FFFFFFFFFFFFFFFull;
    uint64_t E = u >> 52, F = u & 0xFFFFFFFFFFFFFull;
    if (E >= 2047) { *range = 1; return 0; }
    uint64_t mant = E ? (F | (1ull << 52)) : F;
    int64_t Ee = E ? (int64_t)E : 1;
    if (Ee > 1026) { *range = 1; return 0; }
    u128 m2 = (u128)mant * (u128)mant;              /* < 2^106 */
    int64_t sh = 2 * Ee - 2150 + NORM_FRAC;           /* x^2 = m2 * 2^(2Ee-2150) */
    if (sh >= 0) return m2 << sh;
    if (-sh >= 106) return 0;
    return m2 >> (-sh);
}

/* Correctly rounded double of S * 2^-112. */
static double units_to_double(u128 S)
{
    if (S == 0) return 0.0;
    int p = 0;
    for (u128 t = S; t; t >>= 1) ++p;                 /* bit length */
    uint64_t top;
    int e;
    if (p <= 64) {
        top = (uint64_t)S;
        e = 0;
    } else {
        int drop = p - 64;
        u128 rest = S & (((u128)1 << drop) - 1);
        top = (uint64_t)(S >> drop) | (rest != 0);    /* sticky bit */
        e = drop;
    }
    /* top has at most 64 bits; conversion to double rounds to nearest even */
    return ldexp((double)top, e - NORM_FRAC);
}

/* exact sum of squares of 2*count components (interleaved or not) */
static u128 sum_sq(const double *a, uint64_t ncomp, int *range)
{
    u128 S = 0;
    for (uint64_t i = 0; i < ncomp; ++i) S += sq_units(a[i], range);
    return S;
}

void or_sum_sq(const double *a, uint64_t ncomp, uint64_t *lo, uint64_t *hi,
               int *range)
{
    int r = 0;
    u128 S = sum_sq(a, ncomp, &r);
    *lo = (uint64_t)S;
    *hi = (uint64_t)(S >> 64);
    *range = r;
}

double or_units_to_double(uint64_t lo, uint64_t hi)
{
    return units_to_double(((u128)hi << 64) | lo);
}

/* ------------------------------------------------------------------ */
/* O2: tile codec                                                      */
/* ------------------------------------------------------------------ */


/*
 * Tile stream format (little-endian).  A tile is 2^c amplitudes; its two
 * component streams (re, im) each hold N = 2^c doubles, cut into
 * G = max(1, N/32) groups of L = min(N, 32) consecutive values.
 *
 * Header, 32 bytes:
 *   [0] mode: 0 CONST, 1 PACKED, 2 RAW      [1] shift s (0..52; 0 in RAW)
 *   [2] ladder level                          [3] sign mode of re (bits 0-2)
 *       and of im (bits 3-5); 0 in RAW
 *   [4..7]  body length in bytes (multiple of 16)
 *   [8..15] anchor of re                      [16..23] anchor of im
 *   [24] c                                    [25] zero mode of re (bits
 *       0-2) and of im (bits 3-5); 0 unless PACKED      [26..31] zero
 * Codes: B = magnitude bits of x (bits 0-62), q = (B + 2^(s-1)) >> s
 * (q = B when s = 0); reconstruction x^ = (q << s) | sign << 63.  A value
 * with q = 0 is a zero (q = 0 only for x = +-0: smaller nonzero values
 * force the lossless level); at s > 0 a zero's sign is stored as 0.  The
 * anchor is the first nonzero code (0 if none).  Residuals run along the
 * nonzero codes only: r = q - (previous nonzero code, the anchor for the
 * first), z = zigzag(r).  Group width w = bit length of the OR of the z of
 * its nonzero values.
 * Word sections (sign words: bit l = stored sign of value l; zero words:
 * bit l set when value l is a zero), mode: 0 every word 0, 1 every word
 * all L bits set, 2 / 3 exceptions to 0 / to all-set: ceil(G/32) u32
 * bitmap words (bit g set when word g differs from the base), then the
 * differing words in group order, 4 G u32 words.  The encoder picks 0 or
 * 1 when it applies, else the shortest of 2, 3, 4 (lowest on a tie).
 * CONST: body empty; every value of a component is (anchor << s) with the
 *   uniform sign of its sign mode (0 or 1).
 * PACKED body: sign sections of re and im, zero sections of re and im, G
 *   width bytes of re, G of im, zero pad to 4, then for re then im, group
 *   by group, ceil(nz*w/32) u32 words (nz = nonzero values of the group)
 *   holding the k-th nonzero value's z at bits [k*w, (k+1)*w), LSB first;
 *   zero pad to 16.
 * RAW body: the 2N doubles in memory order (re, im interleaved).
 * Mode rule at one level: CONST when every z is 0, both sign modes are 0
 * or 1 and both zero modes are 0 or 1; else PACKED when its body is
 * shorter than 16N; else RAW.
 */
#define HDR 32
enum { M_CONST = 0, M_PACKED = 1, M_RAW = 2, M_POLAR = 3, M_POLAR_B = 4 };
/* modes of a section of per-group bit words (sign words, zero words) */
enum { S_CLEAR = 0, S_SET = 1, S_EXC_CLEAR = 2, S_EXC_SET = 3, S_WORDS = 4 };
#define MAG 0x7FFFFFFFFFFFFFFFull
#define MIN_NORMAL 0x0010000000000000ull
#define LOSSY_LIMIT 0x7FE0000000000000ull   /* |x| < 2^1023 */
#define INF_BITS 0x7FF0000000000000ull

/* flags reported by the encoder */
#define OR_F_NONFINITE 1
#define OR_F_FORCED_LOSSLESS 2

/* Largest shift s in [0, 52] whose bound 2^(s-53) is <= eps; 0 when
 * eps < 2^-53.  Quantising the magnitude bits with shift s moves them by
 * at most 2^(s-1) units, which changes |x| by less than 2^(s-53)|x| (one
 * unit weighs at most 2^-52 |x| inside a binade, and a rounding that
 * crosses a binade boundary keeps the same bound). */
int or_shift_for_eps(double eps)
{
    for (int s = 52; s >= 1; --s)
        if (ldexp(1.0, s - 53) <= eps) return s;
    return 0;
}

static uint64_t quant(uint64_t B, int s)
{
    return s == 0 ? B : (B + (1ull << (s - 1))) >> s;
}

static int bitlen64(uint64_t v)
{
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

static void put32(uint8_t *p, uint32_t v) { for (int i = 0; i < 4; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static void put64(uint8_t *p, uint64_t v) { for (int i = 0; i < 8; ++i) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get32(const uint8_t *p) { uint32_t v = 0; for (int i = 3; i >= 0; --i) v = (v << 8) | p[i]; return v; }
static uint64_t get64(const uint8_t *p) { uint64_t v = 0; for (int i = 7; i >= 0; --i) v = (v << 8) | p[i]; return v; }

static size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

/* base word of an exception mode */
static uint32_t section_base(int mode, uint32_t lanes)
{
    return mode == S_EXC_SET ? lanes : 0;
}

/* bytes of a word section in the given mode */
static size_t section_bytes(int mode, const uint32_t *wd, int G, uint32_t lanes)
{
    if (mode == S_CLEAR || mode == S_SET) return 0;
    if (mode == S_WORDS) return 4 * (size_t)G;
    uint32_t base = section_base(mode, lanes);
    size_t n = 4 * (size_t)((G + 31) / 32);
    for (int g = 0; g < G; ++g)
        if (wd[g] != base) n += 4;
    return n;
}

/* mode of a word section: 0 when every word is 0, 1 when every word has
 * all L bits set, else the smallest of 2 (exceptions to 0), 3 (exceptions
 * to all-set) and 4 (every word), the lower mode on a tie */
static int word_mode(const uint32_t *wd, int G, uint32_t lanes)
{
    int any1 = 0, any0 = 0;
    for (int g = 0; g < G; ++g) {
        if (wd[g]) any1 = 1;
        if (wd[g] != lanes) any0 = 1;
    }
    if (!any1) return S_CLEAR;
    if (!any0) return S_SET;
    int best = S_EXC_CLEAR;
    for (int m = S_EXC_SET; m <= S_WORDS; ++m)
        if (section_bytes(m, wd, G, lanes) < section_bytes(best, wd, G, lanes)) best = m;
    return best;
}

static size_t write_section(uint8_t *b, size_t off, int mode, const uint32_t *wd, int G, uint32_t lanes)
{
    if (mode == S_WORDS) {
        for (int g = 0; g < G; ++g) put32(b + off + 4 * (size_t)g, wd[g]);
        return off + 4 * (size_t)G;
    }
    if (mode == S_EXC_CLEAR || mode == S_EXC_SET) {
        uint32_t base = section_base(mode, lanes);
        size_t nb = (size_t)((G + 31) / 32), e = off + 4 * nb;
        for (int g = 0; g < G; ++g)
            if (wd[g] != base) {
                size_t bo = off + 4 * (size_t)(g / 32);
                put32(b + bo, get32(b + bo) | (1u << (g % 32)));
                put32(b + e, wd[g]);
                e += 4;
            }
        return e;
    }
    return off;
}

static int popcount32(uint32_t v)
{
    int n = 0;
    while (v) { n += v & 1; v >>= 1; }
    return n;
}

/* bound on any stream for a tile of 2^c amplitudes */
size_t or_stream_cap(int c)
{
    return HDR + 16 * ((size_t)1 << c) + 64;
}

/*
 * Write a tile stream from its per-component word sections, zigzag
 * residuals and group widths (shared by the componentwise and the polar
 * modes).  polar = 0: CONST when every residual is 0 and every section
 * mode is 0 or 1, else PACKED when shorter than RAW, else RAW.  polar = 1:
 * the POLAR mode with the PACKED body layout (its sign sections clear),
 * d1 in header bytes 26..31; returns 0 when that body is not shorter than
 * RAW.  Returns the stream length.
 */
static size_t write_stream(const double *a, int c, int s, int level, const uint64_t *anchor, int allzero,
                           uint32_t **sw, uint32_t **zw, uint64_t **z, int **w, int **nnz,
                           const int *smode, const int *zmode, int polar, uint64_t d1,
                           const uint32_t *basis, size_t nbasis, uint8_t *out)
{
    uint64_t N = 1ull << c;
    int G = N >= 32 ? (int)(N / 32) : 1;
    int L = N >= 32 ? 32 : (int)N;
    uint32_t lanes = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1);
    size_t raw_body = 16 * N;
    int mode;
    size_t body;
    size_t data_words = 0;
    for (int k = 0; k < 2; ++k)
        for (int g = 0; g < G; ++g)
            data_words += ((size_t)nnz[k][g] * w[k][g] + 31) / 32;
    size_t meta = 0;
    for (int k = 0; k < 2; ++k)
        meta += section_bytes(smode[k], sw[k], G, lanes) + section_bytes(zmode[k], zw[k], G, lanes);
    size_t wbytes = round_up(meta + 2 * (size_t)G, 4) - meta;
    size_t packed_body = round_up(meta + wbytes + 4 * (nbasis + data_words), 16);

    if (polar) {
        if (packed_body >= raw_body) return 0;
        mode = polar == 2 ? M_POLAR_B : M_POLAR;
        body = packed_body;
    } else if (allzero && smode[0] <= S_SET && smode[1] <= S_SET && zmode[0] <= S_SET && zmode[1] <= S_SET) {
        mode = M_CONST;
        body = 0;
    } else if (packed_body < raw_body) {
        mode = M_PACKED;
        body = packed_body;
    } else {
        mode = M_RAW;
        body = raw_body;
    }

    memset(out, 0, HDR + body);
    out[0] = (uint8_t)mode;
    out[1] = (uint8_t)(mode == M_RAW ? 0 : s);
    out[2] = (uint8_t)level;
    if (mode != M_RAW) out[3] = (uint8_t)(smode[0] | (smode[1] << 3));
    if (mode == M_PACKED || mode == M_POLAR || mode == M_POLAR_B) out[25] = (uint8_t)(zmode[0] | (zmode[1] << 3));
    put32(out + 4, (uint32_t)body);
    if (mode != M_RAW) {
        put64(out + 8, anchor[0]);
        put64(out + 16, anchor[1]);
    }
    out[24] = (uint8_t)c;
    if (mode == M_POLAR)
        for (int i = 0; i < 6; ++i) out[26 + i] = (uint8_t)(d1 >> (8 * i));

    uint8_t *b = out + HDR;
    if (mode == M_RAW) {
        for (uint64_t i = 0; i < 2 * N; ++i) put64(b + 8 * i, dbits(a[i]));
    } else if (mode == M_PACKED || mode == M_POLAR || mode == M_POLAR_B) {
        size_t off = 0;
        for (int k = 0; k < 2; ++k) off = write_section(b, off, smode[k], sw[k], G, lanes);
        for (int k = 0; k < 2; ++k) off = write_section(b, off, zmode[k], zw[k], G, lanes);
        for (int k = 0; k < 2; ++k)
            for (int g = 0; g < G; ++g) b[off++] = (uint8_t)w[k][g];
        off = round_up(off, 4);
        for (size_t i = 0; i < nbasis; ++i, off += 4) put32(b + off, basis[i]);
        /* lane-major bit packing of the nonzero values: the k-th nonzero
         * value of a group occupies bits [k*w, (k+1)*w) of the group's
         * little-endian bit string */
        for (int k = 0; k < 2; ++k)
            for (int g = 0; g < G; ++g) {
                int wg = w[k][g];
                size_t nwords = ((size_t)nnz[k][g] * wg + 31) / 32;
                size_t rank = 0;
                for (int l = 0; l < L; ++l) {
                    uint64_t i = (uint64_t)g * 32 + l;
                    if ((zw[k][g] >> l) & 1) continue;
                    uint64_t v = z[k][i];
                    for (int bit = 0; bit < wg; ++bit)
                        if ((v >> bit) & 1) {
                            size_t pos = rank * wg + bit;
                            b[off + pos / 8] |= (uint8_t)(1u << (pos % 8));
                        }
                    ++rank;
                }
                off += 4 * nwords;
            }
    }
    return HDR + body;
}

/*
 * Encode one tile of 2^c amplitudes (re, im interleaved) at quantisation
 * shift s, as ladder level 'level'.  Writes the stream to out and returns
 * its length in bytes.
 */
static size_t encode_at(const double *a, int c, int s, int level, uint8_t *out)
{
    uint64_t N = 1ull << c;
    int G = N >= 32 ? (int)(N / 32) : 1;
    int L = N >= 32 ? 32 : (int)N;
    uint32_t lanes = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1);

    uint64_t *q[2], *z[2], anchor[2];
    uint32_t *sw[2], *zw[2];
    int *w[2], *nnz[2];
    int smode[2], zmode[2];
    for (int k = 0; k < 2; ++k) {
        q[k] = malloc(N * 8);
        z[k] = calloc(N, 8);
        sw[k] = calloc((size_t)G, 4);
        zw[k] = calloc((size_t)G, 4);
        w[k] = calloc((size_t)G, sizeof(int));
        nnz[k] = calloc((size_t)G, sizeof(int));
    }
    int allzero = 1;
    for (int k = 0; k < 2; ++k) {
        for (uint64_t i = 0; i < N; ++i) {
            uint64_t u = dbits(a[2 * i + k]);
            q[k][i] = quant(u & MAG, s);
            /* a zero keeps its sign only at the lossless level */
            if ((u >> 63) && (q[k][i] || s == 0)) sw[k][i / 32] |= 1u << (i % 32);
            if (q[k][i] == 0) zw[k][i / 32] |= 1u << (i % 32);
        }
        /* order-1 Lorenzo residuals along the nonzero codes, from the
         * anchor (the first nonzero code), then zigzag */
        anchor[k] = 0;
        for (uint64_t i = 0; i < N; ++i)
            if (q[k][i]) { anchor[k] = q[k][i]; break; }
        uint64_t prev = anchor[k];
        for (uint64_t i = 0; i < N; ++i) {
            if (!q[k][i]) continue;
            uint64_t r = q[k][i] - prev;
            prev = q[k][i];
            z[k][i] = (r << 1) ^ (uint64_t)((int64_t)r >> 63);
            if (z[k][i]) allzero = 0;
        }
        for (int g = 0; g < G; ++g) {
            uint64_t o = 0;
            for (int l = 0; l < L; ++l) o |= z[k][(uint64_t)g * 32 + l];
            w[k][g] = bitlen64(o);
            nnz[k][g] = popcount32(~zw[k][g] & lanes);
        }
        smode[k] = word_mode(sw[k], G, lanes);
        zmode[k] = word_mode(zw[k], G, lanes);
    }

    size_t len = write_stream(a, c, s, level, anchor, allzero, sw, zw, z, w, nnz, smode, zmode, 0, 0, NULL, 0, out);
    for (int k = 0; k < 2; ++k) {
        free(q[k]); free(z[k]); free(sw[k]); free(zw[k]); free(w[k]); free(nnz[k]);
    }
    return len;
}

/* ------------------------------------------------------------------ */
/* O2': polar tile mode (log-magnitude + phase)                        */
/* ------------------------------------------------------------------ */

/*
 * POLAR mode (a codec variant: amplitude-aware coding of magnitude and
 * phase instead of the two components).  At a lossy level of shift s
 * (8 <= s <= 52) every nonzero amplitude a = x + iy is coded as
 *   magnitude: m = sqrt(fma(x, x, y*y)) (IEEE, correctly rounded), code
 *     qm = quant(bits(m), s - 1), reconstructed m^ = bits(qm << (s - 1));
 *   phase: the angle of (x, y) in units of 2^-64 turn from the integer
 *     CORDIC below, code qa = round(angle / 2^P) mod 2^B with P = s + 8,
 *     B = 64 - P bits, reconstructed direction (X, Y) = CORDIC rotation of
 *     (2^59, 0) by qa << P;
 *   a^ = (m^ (Xd r), m^ (Yd r)) with Xd, Yd the doubles nearest X, Y
 *     and r = 1 / sqrt(fma(Xd, Xd, Yd*Yd)) (IEEE division and square root).
 * The mode is used only when every amplitude then satisfies
 * |a^ - a|^2 <= 2^(2(s-53)) (1 - 2^-10) |a|^2 (checked in IEEE arithmetic;
 * the margin covers the check's own rounding), i.e. the level's bound on
 * the complex amplitude (the componentwise mode bounds each component,
 * which implies it), and every component is 0 or has 2^-400 <= |x| < 16.
 * Codes run along the nonzero amplitudes: magnitudes by order-1 Lorenzo
 * from their anchor (header 8..15); phases by order-2 Lorenzo modulo 2^B
 * from u0 (header 16..23) and the first difference d1 (header 26..31):
 * residual r_j = u_j - 2 u_(j-1) + u_(j-2) for j >= 2 (0 for j < 2), as a
 * signed B-bit value, zigzagged (mode 3).  A tile without zero amplitudes
 * may instead take the bitwise-linear angle predictor (mode 4): with
 * hp(i) the angle of amplitude i rounded to B + 8 bits (8 more than the
 * code), hp(0) in header 16..23 and D_b = hp(2^b) - hp(0) mod 2^(B+8)
 * for b < c (a basis section of ceil(c (B+8) / 32) words after the widths,
 * D_b at bits [b (B+8), (b+1) (B+8))), the prediction of u_i is
 * (hp(0) + sum of D_b over the set bits b of i) mod 2^(B+8), rounded to B
 * bits, and the residual u_i - prediction is coded as above (header
 * 26..31 zero).  A product state over the index bits (the QFT before its
 * swaps, whose phases are sums of one phase per set bit) then costs
 * residuals near 0, like a phase linear in the index.  The encoder codes a
 * dense tile both ways and keeps the shorter (mode 3 on a tie).  Body: the
 * PACKED layout with clear sign sections and the zero words of both
 * components equal (a zero amplitude; mode 4 has none).
 */
#define POLAR_ITERS 30
#define POLAR_EXTRA 8                    /* extra angle bits of the bitwise-linear predictor */
#define POLAR_MIN_EXP 623                /* |x| >= 2^-400: biased exponent >= 1023 - 400 */
#define POLAR_MAX_EXP 1027               /* |x| < 16 */

static uint64_t polar_atan_turns[POLAR_ITERS];
static pthread_once_t polar_once = PTHREAD_ONCE_INIT;

/* arctan(1/n) in fixed point with 124 fractional bits, by its alternating
 * series sum (-1)^j / ((2j+1) n^(2j+1)); every term truncated (the error
 * stays below 2^-117, far under the 2^-64 of the table) */
static u128 atan_inv_fix(uint64_t n)
{
    u128 p = ((u128)1 << 124) / n, sum = 0;
    int neg = 0;
    for (uint64_t j = 0; p; ++j) {
        u128 t = p / (2 * j + 1);
        if (neg) sum -= t; else sum += t;
        neg = !neg;
        p /= (u128)n * n;
    }
    return sum;
}

/* Table of atan(2^-k) / (2 pi) in units of 2^-64 turn, rounded to nearest:
 * atan(1) = atan(1/2) + atan(1/3) (Euler), 2 pi = 8 atan(1). */
static void polar_init(void)
{
    u128 one = atan_inv_fix(2) + atan_inv_fix(3);           /* pi/4 */
    u128 twopi = one * 8;
    for (int k = 0; k < POLAR_ITERS; ++k) {
        u128 v = k == 0 ? one : atan_inv_fix(1ull << k);
        /* round(v * 2^64 / twopi) by binary long division (v < twopi) */
        u128 rem = v;
        uint64_t q = 0;
        for (int i = 0; i < 64; ++i) {
            rem <<= 1;
            q <<= 1;
            if (rem >= twopi) { rem -= twopi; q |= 1; }
        }
        if (rem >= twopi - rem) ++q;
        polar_atan_turns[k] = q;
    }
}

void or_polar_table(uint64_t *out, int n)
{
    pthread_once(&polar_once, polar_init);
    for (int k = 0; k < n && k < POLAR_ITERS; ++k) out[k] = polar_atan_turns[k];
}

/* signed fixed-point value of x with the exponent of the larger component
 * (biased exponent emax) mapped to 2^59: mantissa << (7 + e - emax),
 * truncated toward zero when the shift is negative */
static int64_t polar_fix(double x, int emax)
{
    uint64_t u = dbits(x);
    uint64_t e = (u >> 52) & 0x7FF, f = u & 0xFFFFFFFFFFFFFull;
    if (e == 0 && f == 0) return 0;
    uint64_t m = f | (1ull << 52);
    int sh = 7 + (int)e - emax;
    uint64_t v = sh >= 0 ? m << sh : (sh > -64 ? m >> (-sh) : 0);
    return (u >> 63) ? -(int64_t)v : (int64_t)v;
}

/* angle of (x, y) in units of 2^-64 turn: CORDIC vectoring on the fixed
 * point values (right half-plane first), POLAR_ITERS steps */
uint64_t or_polar_angle(double x, double y)
{
    pthread_once(&polar_once, polar_init);
    int ex = (int)((dbits(x) >> 52) & 0x7FF), ey = (int)((dbits(y) >> 52) & 0x7FF);
    int emax = ex > ey ? ex : ey;
    int64_t X = polar_fix(x, emax), Y = polar_fix(y, emax);
    uint64_t th = 0;
    if (X < 0) { X = -X; Y = -Y; th = 1ull << 63; }
    for (int k = 0; k < POLAR_ITERS; ++k) {
        int64_t dx = Y >> k, dy = X >> k;
        if (Y >= 0) { X += dx; Y -= dy; th += polar_atan_turns[k]; }
        else { X -= dx; Y += dy; th -= polar_atan_turns[k]; }
    }
    return th;
}

/* direction of angle th (units of 2^-64 turn): CORDIC rotation of
 * (2^59, 0), a half turn first when th is in the left half-plane */
static void polar_dir(uint64_t th, int64_t *px, int64_t *py)
{
    int64_t X = (int64_t)1 << 59, Y = 0;
    uint64_t z = th;
    if (((th >> 62) + 1) & 2) { X = -X; z = th - (1ull << 63); }    /* th in [1/4, 3/4) turn */
    int64_t zz = (int64_t)z;
    for (int k = 0; k < POLAR_ITERS; ++k) {
        int64_t dx = Y >> k, dy = X >> k;
        if (zz >= 0) { X -= dx; Y += dy; zz -= (int64_t)polar_atan_turns[k]; }
        else { X += dx; Y -= dy; zz += (int64_t)polar_atan_turns[k]; }
    }
    *px = X;
    *py = Y;
}

/* the reconstruction of (qm, qa) at shift s */
static void polar_recon(uint64_t qm, uint64_t qa, int s, double *re, double *im)
{
    int P = s + 8;
    double m = bitsd(qm << (s - 1));
    int64_t X, Y;
    polar_dir(qa << P, &X, &Y);
    double xd = (double)X, yd = (double)Y;
    double r = 1.0 / sqrt(fma(xd, xd, yd * yd));
    *re = m * (xd * r);
    *im = m * (yd * r);
}

void or_polar_recon(uint64_t qm, uint64_t qa, int s, double *re, double *im)
{
    pthread_once(&polar_once, polar_init);
    polar_recon(qm, qa, s, re, im);
}

static int polar_comp_ok(double x)
{
    uint64_t e = (dbits(x) >> 52) & 0x7FF;
    return (dbits(x) & MAG) == 0 || (e >= POLAR_MIN_EXP && e < POLAR_MAX_EXP);
}

/* Residual words of a code stream: zigzag z per value, group widths and
 * nonzero counts for the PACKED layout. */
static void code_widths(uint64_t *const *z, uint32_t *const *zw, int G, int L, uint32_t lanes, int **w, int **nnz)
{
    for (int k = 0; k < 2; ++k)
        for (int g = 0; g < G; ++g) {
            uint64_t o = 0;
            for (int l = 0; l < L; ++l) o |= z[k][(uint64_t)g * 32 + l];
            w[k][g] = bitlen64(o);
            nnz[k][g] = popcount32(~zw[k][g] & lanes);
        }
}

/* POLAR stream of a tile at shift s as ladder level `level`, or 0 when the
 * tile cannot use the mode (a value out of range or over the bound, or a
 * body not shorter than RAW).  A tile without zero amplitudes is coded
 * with both angle predictors, order 2 (mode 3) and bitwise linear (mode
 * 4), and keeps the shorter (mode 3 on a tie). */
static size_t encode_polar_at(const double *a, int c, int s, int level, uint8_t *out)
{
    if (s < 8 || s > 52) return 0;
    pthread_once(&polar_once, polar_init);
    uint64_t N = 1ull << c;
    int G = N >= 32 ? (int)(N / 32) : 1;
    int L = N >= 32 ? 32 : (int)N;
    uint32_t lanes = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1);
    int P = s + 8, B = 64 - P, BE = B + POLAR_EXTRA;
    uint64_t bmask = (1ull << B) - 1, half = 1ull << (B - 1), emask = (1ull << BE) - 1;
    double lim = ldexp(1.0 - ldexp(1.0, -10), 2 * (s - 53));
    uint64_t *qm = calloc(N, 8), *qa = calloc(N, 8), *hp = calloc(N, 8);
    uint64_t *z[2] = {calloc(N, 8), calloc(N, 8)}, *zb = calloc(N, 8);
    uint32_t *sw[2] = {calloc((size_t)G, 4), calloc((size_t)G, 4)};
    uint32_t *zw[2] = {calloc((size_t)G, 4), calloc((size_t)G, 4)};
    int *w[2] = {calloc((size_t)G, sizeof(int)), calloc((size_t)G, sizeof(int))};
    int *nnz[2] = {calloc((size_t)G, sizeof(int)), calloc((size_t)G, sizeof(int))};
    int ok = 1, dense = 1;
    for (uint64_t i = 0; i < N && ok; ++i) {
        double x = a[2 * i], y = a[2 * i + 1];
        if (!polar_comp_ok(x) || !polar_comp_ok(y)) { ok = 0; break; }
        if ((dbits(x) & MAG) == 0 && (dbits(y) & MAG) == 0) {
            zw[0][i / 32] |= 1u << (i % 32);
            zw[1][i / 32] |= 1u << (i % 32);
            dense = 0;
            continue;
        }
        double m = sqrt(fma(x, x, y * y));
        qm[i] = quant(dbits(m), s - 1);
        uint64_t th = or_polar_angle(x, y);
        qa[i] = ((th + (1ull << (P - 1))) >> P) & bmask;
        hp[i] = ((th + (1ull << (P - POLAR_EXTRA - 1))) >> (P - POLAR_EXTRA)) & emask;
        double xr, xi;
        polar_recon(qm[i], qa[i], s, &xr, &xi);
        double dr = xr - x, di = xi - y;
        if (!(fma(dr, dr, di * di) <= lim * fma(x, x, y * y))) ok = 0;
    }
    size_t len = 0;
    if (ok) {
        uint64_t anchor[2] = {0, 0}, d1 = 0;
        int j = 0;
        uint64_t prevm = 0, u1 = 0, u2 = 0;            /* previous two angle codes */
        for (uint64_t i = 0; i < N; ++i) {
            if ((zw[0][i / 32] >> (i % 32)) & 1) continue;
            if (j == 0) { anchor[0] = qm[i]; anchor[1] = qa[i]; prevm = qm[i]; }
            uint64_t rm = qm[i] - prevm;
            prevm = qm[i];
            z[0][i] = (rm << 1) ^ (uint64_t)((int64_t)rm >> 63);
            uint64_t ra = 0;
            if (j == 1) d1 = (qa[i] - u1) & bmask;
            if (j >= 2) ra = (qa[i] - 2 * u1 + u2) & bmask;
            int64_t rs = (int64_t)((ra ^ half) - half);     /* signed B-bit residual */
            z[1][i] = ((uint64_t)rs << 1) ^ (uint64_t)(rs >> 63);
            u2 = u1;
            u1 = qa[i];
            ++j;
        }
        int smode[2] = {S_CLEAR, S_CLEAR}, zmode[2];
        code_widths(z, zw, G, L, lanes, w, nnz);
        for (int k = 0; k < 2; ++k) zmode[k] = word_mode(zw[k], G, lanes);
        len = write_stream(a, c, s, level, anchor, 0, sw, zw, z, w, nnz, smode, zmode, 1, d1, NULL, 0, out);
        if (dense) {
            /* bitwise linear: the angle of index i predicted from hp(0) and
             * the differences D_b = hp(2^b) - hp(0) of its set bits, at
             * POLAR_EXTRA more bits, then rounded to the code */
            uint64_t D[16];
            size_t nb = ((size_t)c * BE + 31) / 32;
            uint32_t basis[32];
            memset(basis, 0, sizeof basis);
            for (int b = 0; b < c; ++b) {
                D[b] = (hp[1ull << b] - hp[0]) & emask;
                for (int bit = 0; bit < BE; ++bit)
                    if ((D[b] >> bit) & 1) {
                        size_t pos = (size_t)b * BE + bit;
                        basis[pos / 32] |= 1u << (pos % 32);
                    }
            }
            for (uint64_t i = 0; i < N; ++i) {
                uint64_t p = hp[0];
                for (int b = 0; b < c; ++b)
                    if ((i >> b) & 1) p += D[b];
                uint64_t pred = (((p + (1ull << (POLAR_EXTRA - 1))) & emask) >> POLAR_EXTRA) & bmask;
                uint64_t ra = (qa[i] - pred) & bmask;
                int64_t rs = (int64_t)((ra ^ half) - half);
                zb[i] = ((uint64_t)rs << 1) ^ (uint64_t)(rs >> 63);
            }
            uint64_t *zz[2] = {z[0], zb};
            code_widths(zz, zw, G, L, lanes, w, nnz);
            uint64_t anb[2] = {anchor[0], hp[0]};
            uint8_t *tmp = malloc(or_stream_cap(c) + 256);
            size_t lb = write_stream(a, c, s, level, anb, 0, sw, zw, zz, w, nnz, smode, zmode, 2, 0, basis, nb, tmp);
            if (lb && (!len || lb < len)) {
                memcpy(out, tmp, lb);
                len = lb;
            }
            free(tmp);
        }
    }
    free(qm); free(qa); free(hp); free(zb);
    for (int k = 0; k < 2; ++k) { free(z[k]); free(sw[k]); free(zw[k]); free(w[k]); free(nnz[k]); }
    return len;
}

/* A lossy level with the polar variant on: the POLAR stream when the tile
 * can use it and it is shorter than the componentwise stream, else the
 * componentwise stream (encode_at). */
static size_t encode_level(const double *a, int c, int s, int level, int polar, uint8_t *out)
{
    size_t len = encode_at(a, c, s, level, out);
    if (!polar || s < 8) return len;
    uint8_t *tmp = malloc(or_stream_cap(c));
    size_t lp = encode_polar_at(a, c, s, level, tmp);
    if (lp && lp < len) {
        memcpy(out, tmp, lp);
        len = lp;
    }
    free(tmp);
    return len;
}

/*
 * The quantiser's point-wise relative bound (Sec. III, made relative as in
 * ref. [xin2018]) on count magnitude bit patterns drawn with SplitMix64
 * (Steele, Lea and Flood, 2014) from seed, uniform over the normal range
 * from 2^-962 up to the lossy limit: every reconstruction
 * x^ = bits(quant(B, s) << s) must satisfy |x^ - x| < 2^(s-53) x.  The
 * difference is exact (x^ / x lies in [1/2, 2]) and the bound is a power
 * of two times x, still normal, so the comparison is exact.  Returns the
 * number of violations.  Test infrastructure.
 */
uint64_t or_check_bound(int s, uint64_t count, uint64_t seed)
{
    const uint64_t lo = MIN_NORMAL + (60ull << 52);
    uint64_t bad = 0, st = seed;
    for (uint64_t i = 0; i < count; ++i) {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        uint64_t B = lo + z % (LOSSY_LIMIT - lo);
        double x = bitsd(B), xr = bitsd(quant(B, s) << s);
        if (!(fabs(xr - x) < ldexp(x, s - 53))) ++bad;
    }
    return bad;
}

/* Scan a tile: any non-finite component, and whether every component is
 * zero or inside the lossy range (normal and below 2^1023). */
static void scan_tile(const double *a, int c, int *nonfinite, int *eligible)
{
    uint64_t N = 1ull << c;
    *nonfinite = 0;
    *eligible = 1;
    for (uint64_t i = 0; i < 2 * N; ++i) {
        uint64_t B = dbits(a[i]) & MAG;
        if (B >= INF_BITS) *nonfinite = 1;
        else if (B != 0 && (B < MIN_NORMAL || B >= LOSSY_LIMIT)) *eligible = 0;
    }
}

/* RAW stream of a tile holding a non-finite value (level 0; the caller
 * reports the error). */
static size_t encode_nonfinite(const double *a, int c, uint8_t *out)
{
    uint64_t N = 1ull << c;
    size_t len = HDR + 16 * N;
    memset(out, 0, len);
    out[0] = M_RAW;
    out[2] = 0;
    put32(out + 4, (uint32_t)(16 * N));
    out[24] = (uint8_t)c;
    for (uint64_t i = 0; i < 2 * N; ++i) put64(out + HDR + 8 * i, dbits(a[i]));
    return len;
}

/*
 * Encode one tile with the error-bound ladder of Algorithm 2: try the
 * levels in order (shifts[0..nlev-1], shifts[0] usually 0 = lossless) and
 * keep the first stream whose size is <= max_bytes (ratio >= theta, with
 * max_bytes = floor(16*2^c / theta)); if none qualifies, keep the last.
 * A tile holding a value outside the lossy range (subnormal, |x| >= 2^1023)
 * is coded with shift 0 at every level; a non-finite value forces RAW and
 * sets OR_F_NONFINITE.  out must hold or_stream_cap(c) bytes.
 */
size_t or_encode_tile_opt(const double *a, int c, const int *shifts, int nlev, uint64_t max_bytes,
                          int polar, uint8_t *out, int *level, int *flags);

size_t or_encode_tile(const double *a, int c, const int *shifts, int nlev,
                      uint64_t max_bytes, uint8_t *out, int *level, int *flags)
{
    return or_encode_tile_opt(a, c, shifts, nlev, max_bytes, 0, out, level, flags);
}

/* or_encode_tile with the polar variant on every lossy level (polar = 1):
 * each level keeps the shorter of its POLAR and componentwise streams. */
size_t or_encode_tile_opt(const double *a, int c, const int *shifts, int nlev, uint64_t max_bytes,
                          int polar, uint8_t *out, int *level, int *flags)
{
    int nonfinite, eligible;
    scan_tile(a, c, &nonfinite, &eligible);
    *flags = 0;
    if (nonfinite) {
        *level = 0;
        *flags = OR_F_NONFINITE;
        return encode_nonfinite(a, c, out);
    }
    if (!eligible) *flags |= OR_F_FORCED_LOSSLESS;
    size_t len = 0;
    for (int k = 0; k < nlev; ++k) {
        int s = eligible ? shifts[k] : 0;
        len = encode_level(a, c, s, k, polar, out);
        *level = k;
        if ((uint64_t)len <= max_bytes) break;
    }
    return len;
}

/*
 * Encode one tile at ladder level k (shift shifts[k]) with no size test:
 * the step Algorithm 2 takes for every tile of a stride once the stride's
 * level is known.  Same forced-lossless and non-finite rules as
 * or_encode_tile.
 */
size_t or_encode_tile_level_opt(const double *a, int c, const int *shifts, int k, int polar,
                                uint8_t *out, int *flags);

size_t or_encode_tile_level(const double *a, int c, const int *shifts, int k,
                            uint8_t *out, int *flags)
{
    return or_encode_tile_level_opt(a, c, shifts, k, 0, out, flags);
}

size_t or_encode_tile_level_opt(const double *a, int c, const int *shifts, int k, int polar,
                                uint8_t *out, int *flags)
{
    int nonfinite, eligible;
    scan_tile(a, c, &nonfinite, &eligible);
    *flags = 0;
    if (nonfinite) {
        *flags = OR_F_NONFINITE;
        return encode_nonfinite(a, c, out);
    }
    if (!eligible) *flags |= OR_F_FORCED_LOSSLESS;
    return encode_level(a, c, eligible ? shifts[k] : 0, k, polar, out);
}

/*
 * Decode one stream into 2^c amplitudes.  Returns 0, or a negative code
 * when the stream is malformed (nothing is read past len).
 */
int or_decode_tile(const uint8_t *in, size_t len, int c, double *a)
{
    if (len < HDR) return -1;
    uint64_t N = 1ull << c;
    int G = N >= 32 ? (int)(N / 32) : 1;
    int L = N >= 32 ? 32 : (int)N;
    uint32_t lanes = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1);
    int mode = in[0], s = in[1];
    int sm[2] = {in[3] & 7, (in[3] >> 3) & 7};
    int zm[2] = {in[25] & 7, (in[25] >> 3) & 7};
    size_t body = get32(in + 4);
    if (in[24] != (uint8_t)c) return -2;
    if (HDR + body > len) return -3;
    uint64_t anchor[2] = {get64(in + 8), get64(in + 16)};
    const uint8_t *b = in + HDR;
    if (mode == M_RAW) {
        if (body != 16 * N) return -4;
        for (uint64_t i = 0; i < 2 * N; ++i) a[i] = bitsd(get64(b + 8 * i));
        return 0;
    }
    if (s > 52) return -5;
    if (mode == M_CONST) {
        if (body != 0 || sm[0] > S_SET || sm[1] > S_SET || in[25]) return -6;
        for (int k = 0; k < 2; ++k) {
            uint64_t v = (anchor[k] << s) | ((uint64_t)sm[k] << 63);
            for (uint64_t i = 0; i < N; ++i) a[2 * i + k] = bitsd(v);
        }
        return 0;
    }
    if (mode != M_PACKED && mode != M_POLAR && mode != M_POLAR_B) return -7;
    if ((mode == M_POLAR || mode == M_POLAR_B) && (s < 8 || sm[0] != S_CLEAR || sm[1] != S_CLEAR)) return -7;
    if (mode == M_POLAR_B && (zm[0] != S_CLEAR || zm[1] != S_CLEAR)) return -7;    /* no zero amplitude */
    size_t off = 0;
    uint32_t *sw[2], *zw[2];
    for (int k = 0; k < 2; ++k) { sw[k] = calloc((size_t)G, 4); zw[k] = calloc((size_t)G, 4); }
    int rc = 0;
    /* sign sections, then zero sections */
    for (int pass = 0; pass < 4 && rc == 0; ++pass) {
        int k = pass & 1, md = pass < 2 ? sm[k] : zm[k];
        uint32_t *dst = pass < 2 ? sw[k] : zw[k];
        if (md > S_WORDS) { rc = -8; break; }
        if (md == S_CLEAR || md == S_SET) {
            for (int g = 0; g < G; ++g) dst[g] = md == S_SET ? lanes : 0;
        } else if (md == S_WORDS) {
            if (off + 4 * (size_t)G > body) { rc = -8; break; }
            for (int g = 0; g < G; ++g) dst[g] = get32(b + off + 4 * (size_t)g);
            off += 4 * (size_t)G;
        } else {
            /* exception bitmap, then the words that differ from the base */
            size_t nb = (size_t)((G + 31) / 32);
            if (off + 4 * nb > body) { rc = -8; break; }
            size_t e = off + 4 * nb;
            for (int g = 0; g < G && rc == 0; ++g) {
                dst[g] = section_base(md, lanes);
                if ((get32(b + off + 4 * (size_t)(g / 32)) >> (g % 32)) & 1) {
                    if (e + 4 > body) { rc = -8; break; }
                    dst[g] = get32(b + e);
                    e += 4;
                }
            }
            off = e;
        }
    }
    int *w[2] = {NULL, NULL};
    if (rc == 0 && off + 2 * (size_t)G > body) rc = -9;
    if (rc == 0) {
        for (int k = 0; k < 2; ++k) {
            w[k] = calloc((size_t)G, sizeof(int));
            for (int g = 0; g < G; ++g) {
                w[k][g] = b[off + (size_t)k * G + g];
                if (w[k][g] > 64) rc = -10;
            }
        }
        off = round_up(off + 2 * (size_t)G, 4);
    }
    if (rc == 0 && mode == M_POLAR) {
        for (int g = 0; g < G; ++g)
            if (zw[0][g] != zw[1][g]) rc = -12;     /* a zero amplitude is zero in both codes */
    }
    /* POLAR_B: the basis differences D_b (BE bits each) after the widths */
    uint64_t D[16];
    if (rc == 0 && mode == M_POLAR_B) {
        int BE = 56 - s + POLAR_EXTRA;
        size_t nb = ((size_t)c * BE + 31) / 32;
        if (off + 4 * nb > body) rc = -13;
        for (int bb = 0; bb < c && rc == 0; ++bb) {
            D[bb] = 0;
            for (int bit = 0; bit < BE; ++bit) {
                size_t pos = (size_t)bb * BE + bit;
                D[bb] |= (uint64_t)((get32(b + off + 4 * (pos / 32)) >> (pos % 32)) & 1) << bit;
            }
        }
        off += 4 * nb;
    }
    /* POLAR: the residuals of the two code streams, kept for the
     * reconstruction below */
    uint64_t *pz = (mode == M_POLAR || mode == M_POLAR_B) ? calloc(2 * N, 8) : NULL;
    for (int k = 0; k < 2 && rc == 0; ++k) {
        uint64_t q = anchor[k];
        for (int g = 0; g < G && rc == 0; ++g) {
            int wg = w[k][g];
            size_t nnz = (size_t)popcount32(~zw[k][g] & lanes);
            size_t nwords = (nnz * wg + 31) / 32;
            if (off + 4 * nwords > body) { rc = -11; break; }
            size_t rank = 0;
            for (int l = 0; l < L; ++l) {
                uint64_t i = (uint64_t)g * 32 + l;
                uint64_t sg = (sw[k][g] >> l) & 1;
                if ((zw[k][g] >> l) & 1) {           /* a zero value */
                    a[2 * i + k] = bitsd(sg << 63);
                    continue;
                }
                uint64_t v = 0;
                for (int bit = 0; bit < wg; ++bit) {
                    size_t pos = rank * wg + bit;
                    v |= (uint64_t)((b[off + pos / 8] >> (pos % 8)) & 1) << bit;
                }
                ++rank;
                if (pz) { pz[2 * i + k] = v; continue; }
                q += (v >> 1) ^ (0 - (v & 1));       /* un-zigzag, running sum */
                a[2 * i + k] = bitsd((q << s) | (sg << 63));
            }
            off += 4 * nwords;
        }
    }
    if (pz && rc == 0) {
        /* magnitudes: running sum from the anchor; phases: second-order
         * running sums modulo 2^B from u0 and d1 */
        pthread_once(&polar_once, polar_init);
        int B = 56 - s, BE = B + POLAR_EXTRA;
        uint64_t bmask = (1ull << B) - 1, emask = (1ull << BE) - 1, d1 = 0;
        for (int i = 0; i < 6; ++i) d1 |= (uint64_t)in[26 + i] << (8 * i);
        uint64_t qm = anchor[0], u = anchor[1] & bmask, d = d1 & bmask;
        uint64_t j = 0;
        for (uint64_t i = 0; i < N; ++i) {
            if ((zw[0][i / 32] >> (i % 32)) & 1) { a[2 * i] = 0.0; a[2 * i + 1] = 0.0; continue; }
            uint64_t vm = pz[2 * i], va = pz[2 * i + 1];
            qm += (vm >> 1) ^ (0 - (vm & 1));
            uint64_t ra = ((va >> 1) ^ (0 - (va & 1))) & bmask;
            if (mode == M_POLAR_B) {
                uint64_t p = anchor[1];
                for (int bb = 0; bb < c; ++bb)
                    if ((i >> bb) & 1) p += D[bb];
                u = ((((p + (1ull << (POLAR_EXTRA - 1))) & emask) >> POLAR_EXTRA) + ra) & bmask;
            } else if (j == 1) u = (u + d) & bmask;
            else if (j >= 2) { d = (d + ra) & bmask; u = (u + d) & bmask; }
            ++j;
            polar_recon(qm, u, s, &a[2 * i], &a[2 * i + 1]);
        }
    }
    free(pz);
    for (int k = 0; k < 2; ++k) { free(sw[k]); free(zw[k]); free(w[k]); }
    return rc;
}

/* ------------------------------------------------------------------ */
/* O3: compressed simulator (Algorithm 2 over tiles)                    */
/* ------------------------------------------------------------------ */

typedef struct {
    int n, c, nlev, normalize, err;
    int shifts[8];
    uint64_t max_bytes;
    int ut;              /* log2 of the tiles one AALC decision covers (0: one tile) */
    uint64_t umax;       /* the ratio threshold as a size limit of one such stride */
    uint64_t ntiles;
    uint8_t **st;
    uint32_t *len;
    u128 *part;          /* per-tile sum of squares of the stored values */
    double alpha;        /* scale applied at the next decode ("normalize") */
    uint64_t hist[8];    /* ladder level of every tile written */
    uint64_t items_done, items_skipped;
    int fuse;            /* diagonal runs as one operator (apply_gates_buf) */
    int polar;           /* lossy levels also try the POLAR mode */
} or_csim;

/* Keep buf (len bytes, malloc'ed) as tile t's stream: count its ladder
 * level and take the norm partial of what the next decode returns. */
static void csim_put(or_csim *cs, uint64_t t, uint8_t *buf, size_t len)
{
    uint64_t N = 1ull << cs->c;
    free(cs->st[t]);
    cs->st[t] = realloc(buf, len);
    cs->len[t] = (uint32_t)len;
    cs->hist[cs->st[t][2] & 7] += 1;
    double *rec = malloc(N * 16);
    or_decode_tile(cs->st[t], len, cs->c, rec);
    int range = 0;
    cs->part[t] = sum_sq(rec, 2 * N, &range);
    if (range) cs->err |= 2;
    free(rec);
}

static void csim_store(or_csim *cs, uint64_t t, const double *amps)
{
    int c = cs->c, level = 0, flags = 0;
    uint8_t *buf = malloc(or_stream_cap(c));
    size_t len = or_encode_tile_opt(amps, c, cs->shifts, cs->nlev, cs->max_bytes, cs->polar,
                                    buf, &level, &flags);
    if (flags & OR_F_NONFINITE) cs->err |= 1;
    csim_put(cs, t, buf, len);
}

/*
 * Algorithm 2's ratio test made once for a whole stride: the 2^ut tiles
 * t0 .. t0 + 2^ut - 1 with amplitudes amps (2^(ut+c) complex values).
 * Compress every tile of the stride at level k = 0, 1, ...; keep the first
 * level at which the stride's streams together take at most umax bytes
 * (stride ratio >= theta), else the last level.
 */
/* The ratio test of one stride: the nt tiles of amps (nt * 2^c complex
 * values) coded at level k = 0, 1, ... until their streams together take at
 * most umax bytes, else at the last level; buf[j] (or_stream_cap(c) bytes
 * each) and len[j] receive tile j's stream.  Returns 1 when a value is not
 * finite. */
static int encode_stride(const double *amps, uint64_t nt, int c, const int *shifts, int nlev,
                         uint64_t umax, int polar, uint8_t **buf, size_t *len)
{
    uint64_t N = 1ull << c;
    int nonfinite = 0;
    for (int k = 0; k < nlev; ++k) {
        uint64_t total = 0;
        nonfinite = 0;
        for (uint64_t j = 0; j < nt; ++j) {
            int flags = 0;
            len[j] = or_encode_tile_level_opt(amps + 2 * j * N, c, shifts, k, polar, buf[j], &flags);
            if (flags & OR_F_NONFINITE) nonfinite = 1;
            total += len[j];
        }
        if (total <= umax) break;
    }
    return nonfinite;
}

static void csim_store_unit(or_csim *cs, uint64_t t0, const double *amps)
{
    int c = cs->c;
    uint64_t nt = 1ull << cs->ut;
    uint8_t **buf = malloc(nt * sizeof *buf);
    size_t *len = malloc(nt * sizeof *len);
    for (uint64_t j = 0; j < nt; ++j) buf[j] = malloc(or_stream_cap(c));
    if (encode_stride(amps, nt, c, cs->shifts, cs->nlev, cs->umax, cs->polar, buf, len)) cs->err |= 1;
    for (uint64_t j = 0; j < nt; ++j) csim_put(cs, t0 + j, buf[j], len[j]);
    free(buf);
    free(len);
}

static void csim_update_alpha(or_csim *cs)
{
    if (!cs->normalize) { cs->alpha = 1.0; return; }
    u128 S = 0;
    for (uint64_t t = 0; t < cs->ntiles; ++t) S += cs->part[t];
    double nrm = units_to_double(S);
    cs->alpha = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
}

or_csim *or_csim_new(int n, int c, const int *shifts, int nlev,
                     uint64_t max_bytes, int normalize)
{
    if (c > n || nlev < 1 || nlev > 8) return NULL;
    or_csim *cs = calloc(1, sizeof(or_csim));
    cs->n = n;
    cs->c = c;
    cs->nlev = nlev;
    for (int i = 0; i < nlev; ++i) cs->shifts[i] = shifts[i];
    cs->max_bytes = max_bytes;
    cs->ut = 0;
    cs->umax = max_bytes;
    cs->normalize = normalize;
    cs->fuse = 1;
    cs->ntiles = 1ull << (n - c);
    cs->st = calloc(cs->ntiles, sizeof(uint8_t *));
    cs->len = calloc(cs->ntiles, sizeof(uint32_t));
    cs->part = calloc(cs->ntiles, sizeof(u128));
    cs->alpha = 1.0;
    return cs;
}

void or_csim_free(or_csim *cs)
{
    if (!cs) return;
    for (uint64_t t = 0; t < cs->ntiles; ++t) free(cs->st[t]);
    free(cs->st);
    free(cs->len);
    free(cs->part);
    free(cs);
}

/*
 * Make one AALC decision per stride of 2^unit_log2 amplitudes (Algorithm 2
 * decides per stride) instead of per tile, with umax the stride's size
 * limit (floor(16 * 2^u / theta) for the stride of 2^u amplitudes).  A
 * stride no larger than a tile, or a ladder of one level, means one
 * decision per tile.  Strides are capped at the whole state.  Returns the
 * log2 of the tiles per decision.
 */
int or_csim_set_unit(or_csim *cs, int unit_log2, uint64_t umax)
{
    int u = unit_log2 < cs->n ? unit_log2 : cs->n;
    cs->ut = (u > cs->c && cs->nlev > 1) ? u - cs->c : 0;
    cs->umax = cs->ut ? umax : cs->max_bytes;
    return cs->ut;
}

/* Diagonal runs on (1, the default) or gate by gate (0); the latter makes
 * lossless sweeps reproduce the dense simulator O1 bit for bit. */
void or_csim_set_fuse(or_csim *cs, int on) { cs->fuse = on ? 1 : 0; }

/* Lossy levels also try the POLAR mode (1) or only the componentwise one
 * (0, the default). */
void or_csim_set_polar(or_csim *cs, int on) { cs->polar = on ? 1 : 0; }

/* state |x>: every tile (or stride) encoded from its dense values */
void or_csim_reset_basis(or_csim *cs, uint64_t x)
{
    uint64_t N = 1ull << cs->c, nt = 1ull << cs->ut;
    double *amps = calloc(nt * N, 16);
    for (uint64_t t = 0; t < cs->ntiles; t += nt) {
        memset(amps, 0, nt * N * 16);
        if ((x >> cs->c) >= t && (x >> cs->c) < t + nt) amps[2 * (x - (t << cs->c))] = 1.0;
        if (cs->ut) csim_store_unit(cs, t, amps);
        else csim_store(cs, t, amps);
    }
    free(amps);
    memset(cs->hist, 0, sizeof cs->hist);
    cs->err = 0;
    csim_update_alpha(cs);
}

/* state given densely (2^n complex values, (re, im) interleaved), encoded
 * tile by tile (or stride by stride) */
void or_csim_set_dense(or_csim *cs, const double *amps)
{
    uint64_t N = 1ull << cs->c, nt = 1ull << cs->ut;
    cs->err = 0;
    for (uint64_t t = 0; t < cs->ntiles; t += nt) {
        if (cs->ut) csim_store_unit(cs, t, amps + 2 * t * N);
        else csim_store(cs, t, amps + 2 * t * N);
    }
    memset(cs->hist, 0, sizeof cs->hist);
    csim_update_alpha(cs);
}

/* Does gate g change any amplitude of the item whose non-buffer qubits
 * (mask fmask) have the values in 'fixed'? */
static int gate_touches(const or_gate *g, uint64_t fixed, uint64_t fmask)
{
    if (((fixed ^ g->cval) & g->cmask & fmask) != 0) return 0;
    int allfixed = 1;
    for (int i = 0; i < g->k; ++i)
        if (!((fmask >> g->t[i]) & 1)) allfixed = 0;
    if (allfixed) {
        int dim = 1 << g->k, r = 0;
        for (int i = 0; i < g->k; ++i) r |= (int)((fixed >> g->t[i]) & 1) << i;
        if (g->m[2 * (r * dim + r)] == 1.0 && g->m[2 * (r * dim + r) + 1] == 0.0) return 0;
    }
    return 1;
}

/* A gate whose matrix has only entries 0 and 1, with one 1 in every row
 * and column, maps basis states to basis states. */
static int gate_is_permutation(const or_gate *g)
{
    int dim = 1 << g->k;
    for (int r = 0; r < dim; ++r) {
        int ones_row = 0, ones_col = 0;
        for (int c = 0; c < dim; ++c) {
            double a = g->m[2 * (r * dim + c)], b = g->m[2 * (r * dim + c) + 1];
            double ac = g->m[2 * (c * dim + r)], bc = g->m[2 * (c * dim + r) + 1];
            if (b != 0.0 || !(a == 0.0 || a == 1.0)) return 0;
            ones_row += a == 1.0;
            ones_col += ac == 1.0 && bc == 0.0;
        }
        if (ones_row != 1 || ones_col != 1) return 0;
    }
    return 1;
}

/* A sweep moves whole tiles when every gate is a permutation whose
 * targets and controls are all qubits >= c: each tile's amplitudes go,
 * unchanged and in the same order, to one tile.  Such a sweep moves the
 * tile streams without decompressing them, so it applies no normalize
 * (the norm of the stored state is unchanged, and the next decompressing
 * sweep applies the scale). */
static int sweep_moves_tiles(const or_gate *g, int ng, int c)
{
    uint64_t low = (1ull << c) - 1;
    for (int i = 0; i < ng; ++i) {
        if (!gate_is_permutation(&g[i]) || (g[i].cmask & low)) return 0;
        for (int j = 0; j < g[i].k; ++j)
            if (g[i].t[j] < c) return 0;
    }
    return 1;
}

/* The member each member j of an item moves to: the gates applied to a
 * buffer of one marker value per member (member bit i <-> qubit H[i]). */
static int item_moves(const or_gate *g, int ng, const int *H, int h, uint64_t fixed, int *dest)
{
    int nm = 1 << h;
    double *mark = calloc((size_t)2 * nm, sizeof(double));
    for (int j = 0; j < nm; ++j) mark[2 * j] = j + 1;
    int rc = 0;
    for (int i = 0; i < ng && rc == 0; ++i)
        if (apply_gate_buf(mark, h, H, fixed, &g[i]) != 0) rc = -2;
    for (int j = 0; j < nm && rc == 0; ++j)
        dest[(int)mark[2 * j] - 1] = j;
    free(mark);
    return rc;
}

/*
 * One sweep: the gates g[0..ng-1] applied to every item.  An item is the
 * group of 2^h tiles whose tile indices differ only in the bits of the
 * high qubits H[0..h-1] (ascending, each >= c); its buffer index is
 * (member j) * 2^c + (low index), member bit i <-> qubit H[i].
 * Per item (Algorithm 2): decompress its tiles, normalize (multiply by the
 * scale of the previous sweep when that scale is not 1), apply the gates in
 * order, compress every tile with the ladder.  An item that no gate
 * touches is kept as it is when the scale is 1.  With one decision per
 * stride every item is computed and every stride compressed again
 * (csim_sweep_units).
 * Returns 0, or -1 on a malformed stream, -2 on a gate that needs a
 * target outside the item, -4 for a sample of a sweep that decides per
 * stride.
 */
static int csim_sweep_items(or_csim *cs, const or_gate *g, int ng, const int *H, int h,
                            uint64_t item_lo, uint64_t item_hi, int update_alpha);

int or_csim_sweep(or_csim *cs, const or_gate *g, int ng, const int *H, int h)
{
    return csim_sweep_items(cs, g, ng, H, h, 0, UINT64_MAX, 1);
}

/* The same sweep restricted to items item_lo .. item_hi-1 (item k is the
 * k-th tile group in increasing tile order) and without the norm update:
 * used to time a bounded sample of a large workload. */
int or_csim_sweep_sample(or_csim *cs, const or_gate *g, int ng, const int *H, int h,
                         uint64_t item_lo, uint64_t item_hi)
{
    return csim_sweep_items(cs, g, ng, H, h, item_lo, item_hi, 0);
}

/*
 * A sweep with one AALC decision per stride: every item is decompressed,
 * normalized and computed, none kept and no stream moved, since Algorithm 2
 * compresses every stride again; then each stride is compressed with its
 * own decision (csim_store_unit).
 */
static int csim_sweep_units(or_csim *cs, const or_gate *g, int ng, const int *H, int h,
                            int update_alpha)
{
    int c = cs->c, n = cs->n, mb = c + h;
    uint64_t N = 1ull << c, nt = 1ull << cs->ut;
    int qb[64];
    for (int p = 0; p < c; ++p) qb[p] = p;
    uint64_t hmask_tile = 0;
    for (int i = 0; i < h; ++i) {
        qb[c + i] = H[i];
        hmask_tile |= 1ull << (H[i] - c);
    }
    double alpha = cs->alpha * sweep_scale(g, ng, cs->fuse);   /* normalize and scaled gates */
    double *buf = malloc(((size_t)1 << mb) * 16);
    double *state = malloc(((size_t)1 << n) * 16);
    int rc = 0;
    for (uint64_t T = 0; T < cs->ntiles && rc == 0; ++T) {
        if (T & hmask_tile) continue;
        cs->items_done++;
        uint64_t fixed = T << c;
        for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            if (or_decode_tile(cs->st[Tj], cs->len[Tj], c, buf + 2 * j * N) != 0) rc = -1;
        }
        if (rc) break;
        if (alpha != 1.0)
            for (uint64_t i = 0; i < 2 * ((uint64_t)1 << mb); ++i) buf[i] = buf[i] * alpha;
        if (apply_gates_buf(buf, mb, qb, fixed, g, ng, c, cs->fuse) != 0) rc = -2;
        for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            memcpy(state + 2 * Tj * N, buf + 2 * j * N, N * 16);
        }
    }
    if (rc == 0)
        for (uint64_t t = 0; t < cs->ntiles; t += nt) csim_store_unit(cs, t, state + 2 * t * N);
    free(buf);
    free(state);
    if (rc == 0 && update_alpha) csim_update_alpha(cs);
    return rc;
}

static int csim_sweep_items(or_csim *cs, const or_gate *g, int ng, const int *H, int h,
                            uint64_t item_lo, uint64_t item_hi, int update_alpha)
{
    if (cs->ut) {                        /* strides decide as a whole: no samples */
        if (item_lo != 0 || item_hi != UINT64_MAX) return -4;
        return csim_sweep_units(cs, g, ng, H, h, update_alpha);
    }
    int c = cs->c, n = cs->n, mb = c + h;
    uint64_t N = 1ull << c;
    int qb[64];
    for (int p = 0; p < c; ++p) qb[p] = p;
    uint64_t hmask_tile = 0;
    for (int i = 0; i < h; ++i) {
        qb[c + i] = H[i];
        hmask_tile |= 1ull << (H[i] - c);
    }
    uint64_t fmask = 0;                          /* fixed qubits of an item */
    for (int q = c; q < n; ++q) fmask |= 1ull << q;
    for (int i = 0; i < h; ++i) fmask &= ~(1ull << H[i]);

    double alpha = cs->alpha * sweep_scale(g, ng, cs->fuse);   /* normalize and scaled gates */
    double *buf = malloc(((size_t)1 << mb) * 16);
    int rc = 0;
    uint64_t item = 0;
    const int moves = sweep_moves_tiles(g, ng, c);
    for (uint64_t T = 0; T < cs->ntiles && rc == 0; ++T) {
        if (T & hmask_tile) continue;
        if (item < item_lo || item >= item_hi) { ++item; continue; }
        ++item;
        uint64_t fixed = T << c;
        if (moves) {
            int touched = 0;
            for (int i = 0; i < ng && !touched; ++i)
                if (gate_touches(&g[i], fixed, fmask)) touched = 1;
            if (!touched) { cs->items_skipped++; continue; }
            cs->items_done++;
            int dest[16];
            uint64_t tj[16];
            uint8_t *st[16];
            uint32_t len[16];
            u128 part[16];
            if ((rc = item_moves(g, ng, H, h, fixed, dest)) != 0) break;
            for (int j = 0; j < (1 << h); ++j) {
                tj[j] = T;
                for (int i = 0; i < h; ++i)
                    if ((j >> i) & 1) tj[j] |= 1ull << (H[i] - c);
                st[j] = cs->st[tj[j]];
                len[j] = cs->len[tj[j]];
                part[j] = cs->part[tj[j]];
            }
            for (int j = 0; j < (1 << h); ++j) {
                cs->st[tj[dest[j]]] = st[j];
                cs->len[tj[dest[j]]] = len[j];
                cs->part[tj[dest[j]]] = part[j];
            }
            continue;
        }
        int touched = alpha != 1.0;
        for (int i = 0; i < ng && !touched; ++i)
            if (gate_touches(&g[i], fixed, fmask)) touched = 1;
        if (!touched) { cs->items_skipped++; continue; }
        cs->items_done++;
        for (uint64_t j = 0; j < (1ull << h); ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            if (or_decode_tile(cs->st[Tj], cs->len[Tj], c, buf + 2 * j * N) != 0) rc = -1;
        }
        if (rc) break;
        if (alpha != 1.0)
            for (uint64_t i = 0; i < 2 * ((uint64_t)1 << mb); ++i) buf[i] = buf[i] * alpha;
        if (apply_gates_buf(buf, mb, qb, fixed, g, ng, c, cs->fuse) != 0) rc = -2;
        if (rc) break;
        for (uint64_t j = 0; j < (1ull << h); ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            csim_store(cs, Tj, buf + 2 * j * N);
        }
    }
    free(buf);
    if (update_alpha) csim_update_alpha(cs);
    return rc;
}

/*
 * One item of a sweep on its own, for sampled checks of states too large
 * for the oracle: in[j] (in_len[j] bytes) is the stream of member j, the
 * tile base_tile | (bits of j at the positions H[i]-c); alpha is the
 * normalize scale of the pass.  Applies the same steps as or_csim_sweep to
 * this item (kept as it is when alpha is 1 and no gate touches it; streams
 * moved between members when the sweep only moves tiles) and writes the
 * members' new streams, concatenated, to out (out_len[j] each).
 * opts: bit 0 the fusion rules (diagonal runs, scaled gates; CSim fuse),
 * bit 1 the POLAR variant on lossy levels (CSim polar).
 * Returns 0, -1 on a malformed stream, -2 on a gate outside the item, -3
 * when out is too small.
 */
int or_item_sweep(int n, int c, const int *H, int h, uint64_t base_tile,
                  const uint8_t *const *in, const uint32_t *in_len, double alpha,
                  const or_gate *g, int ng, const int *shifts, int nlev, uint64_t max_bytes,
                  int opts, uint8_t *out, size_t out_cap, uint32_t *out_len)
{
    uint64_t N = 1ull << c;
    int mb = c + h;
    int qb[64];
    for (int p = 0; p < c; ++p) qb[p] = p;
    for (int i = 0; i < h; ++i) qb[c + i] = H[i];
    uint64_t fmask = 0;
    for (int q = c; q < n; ++q) fmask |= 1ull << q;
    for (int i = 0; i < h; ++i) fmask &= ~(1ull << H[i]);
    uint64_t fixed = base_tile << c;
    const int moves = sweep_moves_tiles(g, ng, c);
    alpha = alpha * sweep_scale(g, ng, opts & 1);              /* normalize and scaled gates */
    int touched = alpha != 1.0 && !moves;
    for (int i = 0; i < ng && !touched; ++i)
        if (gate_touches(&g[i], fixed, fmask)) touched = 1;
    size_t used = 0;
    if (touched && moves) {                      /* streams move to their members */
        int dest[16], src[16];
        if (item_moves(g, ng, H, h, fixed, dest) != 0) return -2;
        for (int j = 0; j < (1 << h); ++j) src[dest[j]] = j;
        for (int j = 0; j < (1 << h); ++j) {
            if (used + in_len[src[j]] > out_cap) return -3;
            memcpy(out + used, in[src[j]], in_len[src[j]]);
            out_len[j] = in_len[src[j]];
            used += in_len[src[j]];
        }
        return 0;
    }
    if (!touched) {
        for (uint64_t j = 0; j < (1ull << h); ++j) {
            if (used + in_len[j] > out_cap) return -3;
            memcpy(out + used, in[j], in_len[j]);
            out_len[j] = in_len[j];
            used += in_len[j];
        }
        return 0;
    }
    double *buf = malloc(((size_t)1 << mb) * 16);
    uint8_t *tmp = malloc(or_stream_cap(c));
    int rc = 0;
    for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j)
        if (or_decode_tile(in[j], in_len[j], c, buf + 2 * j * N) != 0) rc = -1;
    if (rc == 0 && alpha != 1.0)
        for (uint64_t i = 0; i < 2 * ((uint64_t)1 << mb); ++i) buf[i] = buf[i] * alpha;
    if (rc == 0 && apply_gates_buf(buf, mb, qb, fixed, g, ng, c, opts & 1) != 0) rc = -2;
    for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j) {
        int level = 0, flags = 0;
        size_t len = or_encode_tile_opt(buf + 2 * j * N, c, shifts, nlev, max_bytes, (opts >> 1) & 1, tmp,
                                        &level, &flags);
        if (used + len > out_cap) { rc = -3; break; }
        memcpy(out + used, tmp, len);
        out_len[j] = (uint32_t)len;
        used += len;
    }
    free(buf);
    free(tmp);
    return rc;
}

/*
 * Many items of one sweep, each exactly as or_item_sweep computes it, run
 * on `threads` host threads (the items are independent: each thread takes
 * items i = k, k + threads, ...).  Item i has base tile bases[i]; the
 * stream of its member j is in_buf + in_off[i*2^h + j], in_len[...] bytes.
 * Its output streams are written concatenated at out + i*out_stride
 * (out_len[i*2^h + j] bytes each) and its return code (as or_item_sweep)
 * to rc[i].  Used for sampled checks of large states and for the
 * all-cores timing of the oracle.  Returns the number of items whose code
 * is not 0.
 */
typedef struct {
    int n, c, h, ng, nlev, threads, k, opts;
    const int *H;
    uint64_t nitems, max_bytes;
    const uint64_t *bases, *in_off;
    const uint8_t *in_buf;
    const uint32_t *in_len;
    double alpha;
    const or_gate *g;
    const int *shifts;
    uint8_t *out;
    size_t out_stride;
    uint32_t *out_len;
    int *rc;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *b = arg;
    uint64_t nm = 1ull << b->h;
    const uint8_t *ptrs[16];
    for (uint64_t i = (uint64_t)b->k; i < b->nitems; i += (uint64_t)b->threads) {
        for (uint64_t j = 0; j < nm; ++j) ptrs[j] = b->in_buf + b->in_off[i * nm + j];
        b->rc[i] = or_item_sweep(b->n, b->c, b->H, b->h, b->bases[i], ptrs, b->in_len + i * nm,
                                 b->alpha, b->g, b->ng, b->shifts, b->nlev, b->max_bytes, b->opts,
                                 b->out + i * b->out_stride, b->out_stride, b->out_len + i * nm);
    }
    return NULL;
}

int or_item_sweep_batch(int n, int c, const int *H, int h, uint64_t nitems, const uint64_t *bases,
                        const uint8_t *in_buf, const uint64_t *in_off, const uint32_t *in_len,
                        double alpha, const or_gate *g, int ng, const int *shifts, int nlev,
                        uint64_t max_bytes, int opts, uint8_t *out, size_t out_stride, uint32_t *out_len,
                        int *rc, int threads)
{
    if (h < 0 || h > 4) return -1;
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    batch_job jobs[256];
    pthread_t tid[256];
    int started[256];
    for (int k = 0; k < threads; ++k) {
        batch_job b = {n, c, h, ng, nlev, threads, k, opts, H, nitems, max_bytes, bases, in_off, in_buf,
                       in_len, alpha, g, shifts, out, out_stride, out_len, rc};
        jobs[k] = b;
        started[k] = k > 0 && pthread_create(&tid[k], NULL, batch_worker, &jobs[k]) == 0;
    }
    batch_worker(&jobs[0]);
    for (int k = 1; k < threads; ++k) {
        if (started[k]) pthread_join(tid[k], NULL);
        else batch_worker(&jobs[k]);          /* no thread could start: run its share here */
    }
    int bad = 0;
    for (uint64_t i = 0; i < nitems; ++i) bad += rc[i] != 0;
    return bad;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/*
 * One stride of a sweep that decides per stride, on its own (sampled checks
 * of states too large for the oracle): the stride of 2^ut tiles starting at
 * tile t0, ladder decision against umax bytes.  The caller passes the input
 * streams of every member of every item that holds a tile of the stride:
 * ntl tiles, indices ascending in tiles[], stream k in in[k] (in_len[k]
 * bytes).  alpha is the pass's normalize scale.  The items are decoded,
 * normalized and computed as or_csim_sweep computes every item, then the
 * stride's tiles are compressed with one ladder decision (the rule of
 * csim_store_unit) and their streams written in tile order to out
 * (out_len[j] each).
 * Returns 0, -1 on a malformed stream, -2 on a gate outside an item, -3
 * when out is too small, -5 when a needed tile is missing from tiles[].
 */
int or_stride_sweep(int n, int c, const int *H, int h, int ut, uint64_t umax, uint64_t t0,
                    const uint64_t *tiles, const uint8_t *const *in, const uint32_t *in_len,
                    uint64_t ntl, double alpha, const or_gate *g, int ng, const int *shifts,
                    int nlev, int opts, uint8_t *out, size_t out_cap, uint32_t *out_len)
{
    uint64_t N = 1ull << c, nt = 1ull << ut;
    int mb = c + h, rc = 0;
    alpha = alpha * sweep_scale(g, ng, opts & 1);              /* normalize and scaled gates */
    int qb[64];
    for (int p = 0; p < c; ++p) qb[p] = p;
    uint64_t hmask_tile = 0;
    for (int i = 0; i < h; ++i) {
        qb[c + i] = H[i];
        hmask_tile |= 1ull << (H[i] - c);
    }
    (void)n;
    /* the items holding the stride's tiles, each once */
    uint64_t *items = malloc(nt * sizeof *items);
    for (uint64_t j = 0; j < nt; ++j) items[j] = (t0 + j) & ~hmask_tile;
    qsort(items, nt, sizeof *items, cmp_u64);
    double *buf = malloc(((size_t)1 << mb) * 16);
    double *sbuf = malloc(nt * N * 16);
    for (uint64_t ii = 0; ii < nt && rc == 0; ++ii) {
        if (ii && items[ii] == items[ii - 1]) continue;
        uint64_t T = items[ii];
        for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            const uint64_t *hit = bsearch(&Tj, tiles, ntl, sizeof *tiles, cmp_u64);
            if (!hit) { rc = -5; break; }
            uint64_t k = (uint64_t)(hit - tiles);
            if (or_decode_tile(in[k], in_len[k], c, buf + 2 * j * N) != 0) rc = -1;
        }
        if (rc) break;
        if (alpha != 1.0)
            for (uint64_t i = 0; i < 2 * ((uint64_t)1 << mb); ++i) buf[i] = buf[i] * alpha;
        if (apply_gates_buf(buf, mb, qb, T << c, g, ng, c, opts & 1) != 0) rc = -2;
        for (uint64_t j = 0; j < (1ull << h) && rc == 0; ++j) {
            uint64_t Tj = T;
            for (int i = 0; i < h; ++i)
                if ((j >> i) & 1) Tj |= 1ull << (H[i] - c);
            if (Tj >= t0 && Tj < t0 + nt) memcpy(sbuf + 2 * (Tj - t0) * N, buf + 2 * j * N, N * 16);
        }
    }
    if (rc == 0) {
        uint8_t **sb = malloc(nt * sizeof *sb);
        size_t *len = malloc(nt * sizeof *len);
        for (uint64_t j = 0; j < nt; ++j) sb[j] = malloc(or_stream_cap(c));
        encode_stride(sbuf, nt, c, shifts, nlev, umax, (opts >> 1) & 1, sb, len);
        size_t used = 0;
        for (uint64_t j = 0; j < nt; ++j) {
            if (rc == 0 && used + len[j] > out_cap) rc = -3;
            if (rc == 0) {
                memcpy(out + used, sb[j], len[j]);
                out_len[j] = (uint32_t)len[j];
                used += len[j];
            }
            free(sb[j]);
        }
        free(sb);
        free(len);
    }
    free(items);
    free(buf);
    free(sbuf);
    return rc;
}

/* decode every tile into a dense vector (the stored state, unscaled) */
int or_csim_dense(const or_csim *cs, double *out)
{
    uint64_t N = 1ull << cs->c;
    for (uint64_t t = 0; t < cs->ntiles; ++t)
        if (or_decode_tile(cs->st[t], cs->len[t], cs->c, out + 2 * t * N) != 0) return -1;
    return 0;
}

uint32_t or_csim_stream(const or_csim *cs, uint64_t t, uint8_t *out, uint32_t cap)
{
    if (t >= cs->ntiles) return 0;
    if (out && cap >= cs->len[t]) memcpy(out, cs->st[t], cs->len[t]);
    return cs->len[t];
}

/* replace a tile's stream (for decoding streams written elsewhere) and
 * recompute the norm bookkeeping; returns the decoder's status */
int or_csim_set_stream(or_csim *cs, uint64_t t, const uint8_t *in, uint32_t len)
{
    uint64_t N = 1ull << cs->c;
    double *rec = malloc(N * 16);
    int rc = or_decode_tile(in, len, cs->c, rec);
    if (rc == 0) {
        free(cs->st[t]);
        cs->st[t] = malloc(len);
        memcpy(cs->st[t], in, len);
        cs->len[t] = len;
        int range = 0;
        cs->part[t] = sum_sq(rec, 2 * N, &range);
    }
    free(rec);
    return rc;
}

void or_csim_refresh_alpha(or_csim *cs) { csim_update_alpha(cs); }

double or_csim_alpha(const or_csim *cs) { return cs->alpha; }
int or_csim_err(const or_csim *cs) { return cs->err; }

void or_csim_norm_units(const or_csim *cs, uint64_t *lo, uint64_t *hi)
{
    u128 S = 0;
    for (uint64_t t = 0; t < cs->ntiles; ++t) S += cs->part[t];
    *lo = (uint64_t)S;
    *hi = (uint64_t)(S >> 64);
}

uint64_t or_csim_bytes(const or_csim *cs)
{
    uint64_t s = 0;
    for (uint64_t t = 0; t < cs->ntiles; ++t) s += cs->len[t];
    return s;
}

void or_csim_hist(const or_csim *cs, uint64_t *out8)
{
    for (int i = 0; i < 8; ++i) out8[i] = cs->hist[i];
}

void or_csim_items(const or_csim *cs, uint64_t *done, uint64_t *skipped)
{
    *done = cs->items_done;
    *skipped = cs->items_skipped;
}
