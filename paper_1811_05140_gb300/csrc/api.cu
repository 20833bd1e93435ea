// Host side of the compressed simulator: the C ABI of include/qsim.h, the
// sweep planner (gate run partition, partner-tile pairing) and the pass
// control (launch, arena regrowth, re-run after an overflow).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "qsim.h"
#include "qsim_dev.cuh"

namespace qs {
void set_global_error(const char *msg);
size_t sweep_smem_bytes(int mb, int threads);
bool sweep_threads_ok(int threads);
cudaError_t launch_sweep(const SweepParams *plist, const unsigned long long *istart, int nlist,
                         int mb, int grid, int threads, unsigned long long *work, cudaStream_t st);
cudaError_t launch_sweep_sizing(const SweepParams *plist, const unsigned long long *istart, int nlist,
                                int mb, int grid, int threads, unsigned long long *work, cudaStream_t st);
cudaError_t launch_finalize_list(const FinalizeEntry *list, int n, cudaStream_t st);
cudaError_t launch_finalize(DevScalars *scal, int use_alpha, unsigned long long *used_hist,
                            unsigned slot, int record_used, cudaStream_t st);
cudaError_t launch_init(const double2 *dense, unsigned long long x, const CodecCfg &cc,
                        unsigned long long ntiles, uint8_t *arena, unsigned long long cap,
                        unsigned long long *table, unsigned long long *part, DevScalars *scal,
                        unsigned long long *unit_bytes, const uint8_t *unit_level, int unit_shift,
                        int grid, cudaStream_t st);
cudaError_t launch_unit_level(const unsigned long long *bytes, uint8_t *level, unsigned long long nunits,
                              int nlev, unsigned long long limit, cudaStream_t st);
cudaError_t launch_norm_from_parts(const unsigned long long *part, unsigned long long ntiles,
                                   DevScalars *scal, int grid, cudaStream_t st);
cudaError_t launch_sizes(const uint8_t *arena, const unsigned long long *table,
                         unsigned long long first, unsigned long long count, const unsigned long long *list,
                         unsigned long long *sizes, int grid, cudaStream_t st);
cudaError_t launch_sum_sizes(const uint8_t *arena, const unsigned long long *table,
                             unsigned long long ntiles, unsigned long long *total, int grid,
                             cudaStream_t st);
cudaError_t launch_gather(const uint8_t *arena, const unsigned long long *table,
                          unsigned long long first, unsigned long long count, const unsigned long long *list,
                          const unsigned long long *offs, const unsigned long long *sizes,
                          uint8_t *out, int grid, cudaStream_t st);
cudaError_t launch_validate(const uint8_t *buf, const unsigned long long *offs,
                            const unsigned long long *sizes, unsigned long long count, int c,
                            unsigned long long *parts, unsigned int *bad, int grid, cudaStream_t st);
cudaError_t launch_place(const uint8_t *buf, const unsigned long long *offs,
                         const unsigned long long *sizes, unsigned long long count,
                         unsigned long long first, unsigned long long base, uint8_t *arena,
                         unsigned long long *table, const unsigned long long *parts,
                         unsigned long long *part, int grid, cudaStream_t st);
cudaError_t launch_amplitudes(const uint8_t *arena, const unsigned long long *table, int c,
                              unsigned long long start, unsigned long long count, double2 *out,
                              DevScalars *scal, int grid, cudaStream_t st);
cudaError_t launch_probs(const uint8_t *arena, const unsigned long long *table, int c,
                         unsigned long long ntiles, const int *qsel, int nq,
                         unsigned long long *buckets, DevScalars *scal, int grid, cudaStream_t st);
unsigned long long fidelity_chunk(unsigned long long ntiles);
cudaError_t launch_sweep_scales(const SGate *sg, const DGate *dg, const int2 *bounds, int ns, double *D,
                                cudaStream_t st);
cudaError_t launch_run_tables(const DRun *runs, const int2 *classes, int nclasses, const RGate *rgates, int c,
                              double2 *tab, uint8_t *meta, RunClass *rcls, DevScalars *scal, int grid,
                              cudaStream_t st);
cudaError_t launch_fidelity(const uint8_t *arena, const unsigned long long *table, int c,
                            unsigned long long ntiles, const RefSpec &rs, Acc4 *tile_sums,
                            DevScalars *scal, int grid, cudaStream_t st);
cudaError_t launch_pair_sum(const Acc4 *in, Acc4 *out, unsigned long long nout, int grid,
                            cudaStream_t st);
cudaError_t configure_kernels();
int sweep_blocks_per_sm(int mb, int threads);
cudaError_t fp64_rate(int device, double *fma_per_s);
}  // namespace qs

namespace {

constexpr int MAX_QUBITS = 40;
constexpr int DEFAULT_TILE_LOG2 = 8;    // 2^8-amplitude tiles, up to 4 paired high qubits
constexpr double UNITARY_TOL = 1e-12;

struct HostGate {
    int k;
    int t[2];
    unsigned long long cm, cv;
    double m[32];
    bool diag;
};

struct Sweep {
    int lo, hi, h;
    int H[4];
};

// Message of the calling thread's last failing call without a handle.
thread_local std::string g_last_error;

bool matrix_is_diagonal(int k, const double *m) {
    int dim = 1 << k;
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c < dim; ++c)
            if (r != c && (m[2 * (r * dim + c)] != 0.0 || m[2 * (r * dim + c) + 1] != 0.0))
                return false;
    return true;
}

int popcount64(unsigned long long v) { return __builtin_popcountll(v); }

// Gate run partition: extend the open sweep while the union of its paired
// high qubits and the gate's mixing high qubits fits hmax and the sweep
// holds fewer than `depth` gates; diagonal gates mix nothing.  Each sweep's
// pair set is then filled up to min(hmax, n - c) with the smallest high
// qubits not in it, so that every item holds the same number of tiles.
int plan_sweeps(int n, int c, int hmax, int depth, const std::vector<HostGate> &g,
                std::vector<Sweep> &out) {
    out.clear();
    int hcap = std::min(hmax, n - c);
    if (hcap < 0) hcap = 0;
    int lo = 0;
    unsigned long long H = 0;
    auto emit = [&](int a, int b, unsigned long long Hm) {
        for (int q = c; q < n && popcount64(Hm) < hcap; ++q) Hm |= 1ull << q;
        Sweep s{a, b, 0, {0, 0, 0, 0}};
        for (int q = 0; q < 64; ++q)
            if ((Hm >> q) & 1ull) s.H[s.h++] = q;
        out.push_back(s);
    };
    for (int i = 0; i < (int)g.size(); ++i) {
        unsigned long long mix = 0;
        if (!g[i].diag)
            for (int j = 0; j < g[i].k; ++j)
                if (g[i].t[j] >= c) mix |= 1ull << g[i].t[j];
        if (popcount64(mix) > hcap) return -1;
        if (i > lo && (popcount64(H | mix) > hcap || i - lo >= depth)) {
            emit(lo, i, H);
            lo = i;
            H = 0;
        }
        H |= mix;
    }
    if (lo < (int)g.size()) emit(lo, (int)g.size(), H);
    return (int)out.size();
}

int shift_for_eps(double eps) {
    for (int s = 52; s >= 1; --s)
        if (std::ldexp(1.0, s - 53) <= eps) return s;
    return 0;
}

// correctly rounded double of a 128-bit count of 2^-112 units
double units_to_double_host(unsigned long long lo, unsigned long long hi) {
    if (hi == 0) {
        if (lo == 0) return 0.0;
        return std::ldexp((double)lo, -112);
    }
    int p = 128 - __builtin_clzll(hi);
    int drop = p - 64;
    unsigned long long top, rest;
    if (drop == 64) { top = hi; rest = lo; }
    else { top = (hi << (64 - drop)) | (lo >> drop); rest = lo & ((1ull << drop) - 1); }
    top |= rest ? 1ull : 0ull;
    return std::ldexp((double)top, drop - 112);
}

// class of a matrix entry (see the EC_* codes)
unsigned entry_class(double ur, double ui) {
    if (ur == 0.0 && ui == 0.0) return qs::EC_ZERO;
    if (ui == 0.0) return ur == 1.0 ? qs::EC_ONE : (ur == -1.0 ? qs::EC_MINUS_ONE : qs::EC_REAL);
    if (ur == 0.0) return qs::EC_IMAG;
    return qs::EC_GENERAL;
}

// Factor of entry u relative to d (exact comparisons): 0 u == d, 1 u == -d,
// 2 u == i d, 3 u == -i d, -1 none; the first match counts.
int unit_factor(double ur, double ui, double dr, double di) {
    if (ur == dr && ui == di) return 0;
    if (ur == -dr && ui == -di) return 1;
    if (ur == -di && ui == dr) return 2;
    if (ur == di && ui == -dr) return 3;
    return -1;
}

// Row factoring of a non-diagonal gate: bit r set when row r has two or
// more nonzero entries, each f d for its first nonzero entry d and f in
// {1, -1, i, -i}; the code of f for entry e in bits 8 + 2e.
unsigned long long row_factoring(const HostGate &g) {
    const int dim = 1 << g.k;
    unsigned long long fac = 0;
    for (int r = 0; r < dim; ++r) {
        int first = -1, count = 0;
        bool ok = true;
        unsigned long long codes = 0;
        for (int c = 0; c < dim; ++c) {
            const int e = r * dim + c;
            const double ur = g.m[2 * e], ui = g.m[2 * e + 1];
            if (ur == 0.0 && ui == 0.0) continue;
            ++count;
            if (first < 0) { first = e; continue; }
            const int f = unit_factor(ur, ui, g.m[2 * first], g.m[2 * first + 1]);
            if (f < 0) ok = false;
            else codes |= (unsigned long long)f << (8 + 2 * e);
        }
        if (ok && count >= 2) fac |= (1ull << r) | codes;
    }
    return fac;
}

// A scaled gate: no controls, not diagonal, every row factored (two or
// more nonzero entries, each a unit multiple of the row's first nonzero
// entry d) with the same real d in every row (a Hadamard, H (x) H).  Such
// a gate is d times a matrix of units; with fusion on, the sweep applies d
// in its decompression scale and the gate only forms its rows' sums.
bool is_scaled_gate(const HostGate &g) {
    if (g.cm || g.diag) return false;
    const int dim = 1 << g.k;
    const unsigned long long fac = row_factoring(g);
    double d = 0.0;
    for (int r = 0; r < dim; ++r) {
        if (!((fac >> r) & 1ull)) return false;
        int c = 0;
        while (g.m[2 * (r * dim + c)] == 0.0 && g.m[2 * (r * dim + c) + 1] == 0.0) ++c;
        const double dr = g.m[2 * (r * dim + c)], di = g.m[2 * (r * dim + c) + 1];
        if (di != 0.0) return false;
        if (r == 0) d = dr;
        else if (std::memcmp(&dr, &d, sizeof d) != 0) return false;
    }
    return true;
}

// Entries all exactly 0 or 1, one 1 in every row and every column: the
// gate maps basis states to basis states.
bool is_permutation(const HostGate &g) {
    const int dim = 1 << g.k;
    for (int r = 0; r < dim; ++r) {
        int row = 0, col = 0;
        for (int c = 0; c < dim; ++c) {
            const double a = g.m[2 * (r * dim + c)], b = g.m[2 * (r * dim + c) + 1];
            if (b != 0.0 || !(a == 0.0 || a == 1.0)) return false;
            row += a == 1.0;
            col += g.m[2 * (c * dim + r)] == 1.0 && g.m[2 * (c * dim + r) + 1] == 0.0;
        }
        if (row != 1 || col != 1) return false;
    }
    return true;
}

// FP64 instructions of one matrix entry's term, per component: zero and a
// leading +-1 are free, real and imaginary entries take one, general two.
double entry_cost(double ur, double ui, bool first) {
    if (ur == 0.0 && ui == 0.0) return 0.0;
    if (ui == 0.0) return (first && (ur == 1.0 || ur == -1.0)) ? 0.0 : 1.0;
    if (ur == 0.0) return 1.0;
    return 2.0;
}

// FP64 instructions a gate needs on an n-qubit state (controls restrict
// it); a scaled gate applied without its d (fusion) costs only its sums
double gate_dp_ops(const HostGate &g, int n, bool unscaled = false) {
    int dim = 1 << g.k;
    double groups = std::ldexp(1.0, n - g.k - popcount64(g.cm));
    const unsigned long long fac = g.diag ? 0ull : row_factoring(g);
    double per = 0.0;
    for (int r = 0; r < dim; ++r) {
        if (g.diag) {
            double ur = g.m[2 * (r * dim + r)], ui = g.m[2 * (r * dim + r) + 1];
            if (!(ur == 1.0 && ui == 0.0)) per += 2.0 * entry_cost(ur, ui, true);
            continue;
        }
        bool first = true;
        const bool factored = (fac >> r) & 1ull;
        for (int c = 0; c < dim; ++c) {
            double ur = g.m[2 * (r * dim + c)], ui = g.m[2 * (r * dim + c) + 1];
            if (ur == 0.0 && ui == 0.0) continue;
            // factored: one addition per later term, the first entry's product once
            per += 2.0 * (factored ? (first ? (unscaled ? 0.0 : entry_cost(ur, ui, true)) : 1.0)
                                   : entry_cost(ur, ui, first));
            first = false;
        }
    }
    return groups * per;
}

}  // namespace

void qs::set_global_error(const char *msg) { g_last_error = msg; }

unsigned long long qs_handle_footprint(qsim_t h);

struct qsim_state {
    int n = 0, c = 0, hmax = 2, depth = qs::MAX_SWEEP_GATES;
    qsim_codec codec = QSIM_CODEC_REL;
    double eps = 0.0;
    int normalize = 0;
    double theta = 16.0;
    qs::CodecCfg cc{};
    int device = 0, sms = 1;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    unsigned long long ntiles = 0;
    uint8_t *arena[2] = {nullptr, nullptr};
    unsigned long long cap[2] = {0, 0};
    int cur = 0;
    unsigned long long used = 0;          // bytes in arena[cur]
    unsigned long long *table[2] = {nullptr, nullptr};
    unsigned long long *part = nullptr;
    qs::DevScalars *scal = nullptr;
    qs::DevScalars *hscal = nullptr;      // pinned mirror
    qs::DGate *dgates = nullptr;
    size_t dgates_cap = 0;
    qs::DGate *hgates = nullptr;          // pinned staging
    size_t hgates_cap = 0;
    qs::SGate *dsg = nullptr, *hsg = nullptr;
    int *dglist = nullptr;                // per flush: the gates that can apply, sweep by sweep
    std::vector<int> hglist;
    qs::SweepParams *dparams = nullptr, *hparams = nullptr;   // one entry per sweep
    unsigned long long *distart = nullptr, *histart = nullptr; // (0, nitems) per sweep
    size_t params_cap = 0;
    unsigned long long *used_hist = nullptr;
    size_t used_hist_cap = 0;
    unsigned long long *hused = nullptr;  // pinned
    size_t hused_cap = 0;
    unsigned sweep_counter = 0;
    std::vector<HostGate> queue;
    qsim_stats_t st{};
    unsigned long long launches = 0;
    int profiling = 0;
    qsim_profile_t prof{};
    std::vector<cudaEvent_t> events;
    std::string err;
    bool invalid = false;
    bool basis = false;                   // the state is the basis state basis_x as encoded afresh
    unsigned long long basis_x = 0;
    bool pool = false;                    // arenas live in a caller-owned buffer
    int unit_log2 = 0;                    // amplitudes per ladder decision (log2); 0 = one tile
    unsigned long long *unit_bytes = nullptr;   // per stride and level: stream bytes
    uint8_t *unit_level = nullptr;        // per stride: chosen level
    unsigned long long units_cap = 0;
    void *rd = nullptr;                   // read-out scratch (probabilities, fidelity, sizes)
    size_t rd_cap = 0;
    unsigned long long h2d_bytes = 0, d2h_bytes = 0;   // since creation (never reset)
    int fuse = 1;                         // diagonal runs as one operator
    int polar = 0;                        // lossy levels also try the POLAR mode
    int threads = qs::SWEEP_THREADS;      // sweep kernel CTA size
    // diagonal runs of the flush in progress (host staging, device copies)
    std::vector<qs::DRun> hruns;
    std::vector<qs::RGate> hrg;
    std::vector<int2> hclasses;
    qs::DRun *druns = nullptr;
    qs::RGate *drg = nullptr;
    int2 *dclasses = nullptr;
    size_t druns_cap = 0, drg_cap = 0, dclasses_cap = 0;
    double2 *rtab = nullptr;
    uint8_t *rmeta = nullptr;
    size_t rtab_cap = 0, rmeta_cap = 0;
    qs::RunClass *rcls = nullptr;
    size_t rcls_cap = 0;
    // per sweep of the flush: gate bounds and the product of its scaled gates' d
    std::vector<int2> hbounds;
    int2 *dbounds = nullptr;
    double *dscale = nullptr;
    size_t scale_cap = 0;
};

namespace {

qsim_status fail(qsim_t h, qsim_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_last_error = buf;
    return code;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(h, e_ == cudaErrorMemoryAllocation ? QSIM_ERR_OOM : QSIM_ERR_CUDA, \
                        "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

unsigned long long tile_bytes_worst(const qsim_state *h) {
    return (unsigned long long)qs::HDR + (16ull << h->c);
}

unsigned long long round_up(unsigned long long v, unsigned long long a) { return (v + a - 1) / a * a; }

int grid_for(const qsim_state *h, unsigned long long work, int per_sm) {
    unsigned long long g = (unsigned long long)h->sms * (unsigned long long)per_sm;
    if (work < g) g = work;
    return g ? (int)g : 1;
}

qsim_status ensure_arena(qsim_t h, int which, unsigned long long need) {
    if (h->cap[which] >= need) return QSIM_OK;
    if (h->pool)
        return fail(h, QSIM_ERR_OOM, "pool arena of %llu bytes cannot hold %llu bytes", h->cap[which], need);
    unsigned long long worst = h->ntiles * tile_bytes_worst(h);
    unsigned long long nc = std::max(need, h->cap[which] + h->cap[which] / 2);
    nc = std::min(round_up(nc, 1ull << 21), round_up(worst, 256));
    if (nc < need) nc = need;
    CK(cudaStreamSynchronize(h->stream));
    if (h->arena[which]) CK(cudaFree(h->arena[which]));
    h->arena[which] = nullptr;
    h->cap[which] = 0;
    CK(cudaMalloc(&h->arena[which], nc));
    h->cap[which] = nc;
    return QSIM_OK;
}

// An NVTX range for the lifetime of the object: profilers attribute the
// launches enqueued inside it to the range (e.g. ncu --nvtx-include).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// log2 of the tiles one ladder decision covers: 0 (per tile) unless a
// stride of more than one tile was set and the ladder has several levels.
int unit_tiles_log2(const qsim_state *h) {
    if (h->unit_log2 <= 0 || h->cc.nlev < 2 || h->cc.force_raw) return 0;
    const int u = std::min(h->unit_log2, h->n);
    return u > h->c ? u - h->c : 0;
}

// A stride's stream size limit: ratio 16 * 2^u / size >= theta.
unsigned long long unit_limit(const qsim_state *h) {
    const int u = h->c + unit_tiles_log2(h);
    return (unsigned long long)std::floor(16.0 * std::ldexp(1.0, u) / h->theta);
}

// Per-stride counters for the current tiling, grown on demand.
qsim_status ensure_units(qsim_t h, unsigned long long nunits) {
    if (h->units_cap >= nunits) return QSIM_OK;
    CK(cudaStreamSynchronize(h->stream));
    if (h->unit_bytes) cudaFree(h->unit_bytes);
    if (h->unit_level) cudaFree(h->unit_level);
    h->unit_bytes = nullptr;
    h->unit_level = nullptr;
    h->units_cap = 0;
    CK(cudaMalloc(&h->unit_bytes, nunits * qs::MAX_LEVELS * sizeof(unsigned long long)));
    CK(cudaMalloc(&h->unit_level, nunits));
    h->units_cap = nunits;
    return QSIM_OK;
}

// cudaMemcpyAsync that counts the bytes a handle moves between host and
// device (qsim_stats_t h2d_bytes / d2h_bytes).
cudaError_t hcopy(qsim_t h, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
    if (kind == cudaMemcpyHostToDevice) h->h2d_bytes += bytes;
    else if (kind == cudaMemcpyDeviceToHost) h->d2h_bytes += bytes;
    return cudaMemcpyAsync(dst, src, bytes, kind, st);
}

// Device scratch of the read-outs, kept by the handle and grown on demand,
// so that repeated read-outs allocate nothing.
qsim_status ensure_readout(qsim_t h, size_t bytes) {
    if (h->rd_cap >= bytes) return QSIM_OK;
    CK(cudaStreamSynchronize(h->stream));
    if (h->rd) cudaFree(h->rd);
    h->rd = nullptr;
    h->rd_cap = 0;
    const size_t cap = std::max<size_t>(round_up(bytes, 4096), 65536);
    CK(cudaMalloc(&h->rd, cap));
    h->rd_cap = cap;
    return QSIM_OK;
}

qsim_status read_scalars(qsim_t h) {
    CK(hcopy(h, h->hscal, h->scal, sizeof(qs::DevScalars), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return QSIM_OK;
}

qsim_status clear_pass_state(qsim_t h) {
    // err, err_sweep, bump and the running norm restart from zero
    qs::DevScalars z{};
    CK(hcopy(h, &h->scal->bump, &z.bump, sizeof z.bump, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(&h->scal->err, 0, 2 * sizeof(unsigned), h->stream));
    CK(cudaMemsetAsync(&h->scal->acc_lo, 0, 2 * sizeof(unsigned long long), h->stream));
    return QSIM_OK;
}

qsim_status device_error(qsim_t h, unsigned err) {
    h->invalid = true;
    if (err & qs::ERR_NONFINITE) return fail(h, QSIM_ERR_NONFINITE, "a gate produced a non-finite amplitude");
    if (err & qs::ERR_FORMAT) return fail(h, QSIM_ERR_FORMAT, "malformed tile stream on the device");
    if (err & qs::ERR_RANGE) return fail(h, QSIM_ERR_NONFINITE, "amplitude magnitude >= 16 (state not normalised)");
    return fail(h, QSIM_ERR_CUDA, "device error 0x%x", err);
}

// Encode a dense state (device) or |x> into arena[cur], retrying with a
// larger arena after an overflow.
qsim_status encode_fresh(qsim_t h, const double2 *dense, unsigned long long x) {
    unsigned long long need = dense ? h->ntiles * tile_bytes_worst(h)
                                    : (h->cc.force_raw ? h->ntiles * tile_bytes_worst(h)
                                                       : h->ntiles * qs::HDR + tile_bytes_worst(h));
    if (dense) need = std::min(need, std::max<unsigned long long>(h->cap[h->cur], 1ull << 22));
    if (h->pool) need = std::min(need, h->cap[h->cur]);
    for (int attempt = 0; attempt < 64; ++attempt) {
        qsim_status s = ensure_arena(h, h->cur, need);
        if (s != QSIM_OK) {
            h->invalid = attempt > 0;     // an attempt wrote into the arena
            return s;
        }
        CK(cudaMemsetAsync(h->scal, 0, sizeof(qs::DevScalars), h->stream));
        const int ut = unit_tiles_log2(h);
        if (ut) {                         // one ladder decision per stride: size, decide, encode
            const unsigned long long nunits = h->ntiles >> ut;
            if ((s = ensure_units(h, nunits)) != QSIM_OK) return s;
            CK(cudaMemsetAsync(h->unit_bytes, 0, nunits * qs::MAX_LEVELS * sizeof(unsigned long long), h->stream));
            ++h->launches; CK(qs::launch_init(dense, x, h->cc, h->ntiles, nullptr, 0, nullptr, nullptr, h->scal,
                               h->unit_bytes, nullptr, ut, grid_for(h, h->ntiles, 4), h->stream));
            ++h->launches; CK(qs::launch_unit_level(h->unit_bytes, h->unit_level, nunits, h->cc.nlev,
                                                    unit_limit(h), h->stream));
        }
        ++h->launches; CK(qs::launch_init(dense, x, h->cc, h->ntiles, h->arena[h->cur], h->cap[h->cur],
                           h->table[h->cur], h->part, h->scal, nullptr, ut ? h->unit_level : nullptr, ut,
                           grid_for(h, h->ntiles, 4), h->stream));
        ++h->launches; CK(qs::launch_finalize(h->scal, h->normalize, nullptr, 0, 1, h->stream));
        if ((s = read_scalars(h)) != QSIM_OK) return s;
        if (h->hscal->err & qs::ERR_OVERFLOW) {
            need = std::max(need + need / 2, h->hscal->bump + h->hscal->bump / 8);
            continue;
        }
        if (h->hscal->err) return device_error(h, h->hscal->err);
        h->used = h->hscal->used;
        h->st.stream_bytes = h->used;
        h->basis = dense == nullptr;
        h->basis_x = x;
        return QSIM_OK;
    }
    return fail(h, QSIM_ERR_OOM, "arena could not hold the state");
}

qsim_status alloc_tiles(qsim_t h) {
    h->ntiles = 1ull << (h->n - h->c);
    for (int i = 0; i < 2; ++i) {
        CK(cudaMalloc(&h->table[i], h->ntiles * sizeof(unsigned long long)));
    }
    CK(cudaMalloc(&h->part, h->ntiles * 2 * sizeof(unsigned long long)));
    return QSIM_OK;
}

void free_tiles(qsim_t h) {
    for (int i = 0; i < 2; ++i) {
        if (h->table[i]) cudaFree(h->table[i]);
        h->table[i] = nullptr;
        if (h->pool) continue;            // the caller's buffer stays in place
        if (h->arena[i]) cudaFree(h->arena[i]);
        h->arena[i] = nullptr;
        h->cap[i] = 0;
    }
    if (h->part) cudaFree(h->part);
    h->part = nullptr;
}

void set_codec(qsim_t h) {
    qs::CodecCfg &cc = h->cc;
    cc = qs::CodecCfg{};
    cc.c = h->c;
    cc.max_bytes = ~0ull;
    cc.polar = h->polar;
    switch (h->codec) {
        case QSIM_CODEC_NONE:
            cc.force_raw = 1; cc.nlev = 1; cc.shifts[0] = 0; h->normalize = 0; break;
        case QSIM_CODEC_LOSSLESS:
            cc.nlev = 1; cc.shifts[0] = 0; h->normalize = 0; break;
        case QSIM_CODEC_REL:
            cc.nlev = 1; cc.shifts[0] = shift_for_eps(h->eps); h->normalize = 1; break;
        case QSIM_CODEC_AALC: {
            const double lad[4] = {1e-5, 1e-4, 1e-3, 1e-2};
            cc.nlev = 1;
            cc.shifts[0] = 0;
            for (double e : lad)
                if (e <= h->eps * (1 + 1e-12)) cc.shifts[cc.nlev++] = shift_for_eps(e);
            cc.max_bytes = (unsigned long long)std::floor(16.0 * (double)(1ull << h->c) / h->theta);
            h->normalize = 1;
            break;
        }
    }
}

qsim_status check_usable(qsim_t h) {
    if (!h) return fail(nullptr, QSIM_ERR_ARG, "null handle");
    if (h->invalid) return fail(h, QSIM_ERR_STATE_INVALID, "state invalid after an earlier error: %s", h->err.c_str());
    return QSIM_OK;
}

void prepare_gate(const HostGate &g, int c, const Sweep &sw, qs::DGate &d, qs::SGate &sgt) {
    d = qs::DGate{};
    sgt = qs::SGate{};
    std::memcpy(d.m, g.m, sizeof d.m);
    d.k = g.k;
    d.diag = g.diag ? 1 : 0;
    auto pos = [&](int q) -> int {
        if (q < c) return q;
        for (int i = 0; i < sw.h; ++i)
            if (sw.H[i] == q) return c + i;
        return -1;
    };
    for (int i = 0; i < 2; ++i) {
        d.t[i] = i < g.k ? g.t[i] : 0;
        d.pos[i] = i < g.k ? pos(g.t[i]) : -1;
    }
    for (int q = 0; q < 64; ++q) {
        if (!((g.cm >> q) & 1ull)) continue;
        int p = pos(q);
        unsigned long long v = (g.cv >> q) & 1ull;
        if (p >= 0) { d.lcm |= 1ull << p; d.lcv |= v << p; }
        else { d.fcm |= 1ull << q; d.fcv |= v << q; }
    }
    // compact form
    const int dim = 1 << g.k;
    sgt.kind = g.diag ? 0 : (uint8_t)g.k;
    sgt.k = (uint8_t)g.k;
    sgt.p0 = (int8_t)d.pos[0];
    sgt.p1 = (int8_t)(g.k > 1 ? d.pos[1] : -1);
    sgt.t0 = (uint8_t)d.t[0];
    sgt.t1 = (uint8_t)d.t[1];
    sgt.fcm = d.fcm;
    sgt.fcv = d.fcv;
    sgt.lcm = (uint32_t)d.lcm;
    sgt.lcv = (uint32_t)d.lcv;
    sgt.run = -1;
    if (g.diag) {
        for (int r = 0; r < dim; ++r) {
            sgt.d[2 * r] = g.m[2 * (r * dim + r)];
            sgt.d[2 * r + 1] = g.m[2 * (r * dim + r) + 1];
            unsigned code = entry_class(sgt.d[2 * r], sgt.d[2 * r + 1]);
            sgt.cls |= (unsigned long long)code << (3 * r);
            if (code == qs::EC_ONE) sgt.one_mask |= (uint8_t)(1u << r);
        }
    } else {
        for (int e = 0; e < dim * dim; ++e)
            sgt.cls |= (unsigned long long)entry_class(g.m[2 * e], g.m[2 * e + 1]) << (3 * e);
        sgt.fac = row_factoring(g);
    }
    // buffer bits pinned by local controls and buffer targets, ascending
    unsigned pinned = (unsigned)d.lcm;
    for (int i = 0; i < g.k; ++i)
        if (d.pos[i] >= 0) pinned |= 1u << d.pos[i];
    for (int b = 0; b < 32; ++b)
        if ((pinned >> b) & 1u) sgt.ins[sgt.nins++] = (uint8_t)b;
}

}  // namespace

// device bytes held by a state: both arenas, tile tables, norm partials
unsigned long long qs_handle_footprint(qsim_t h) {
    return h ? h->cap[0] + h->cap[1] + h->ntiles * 32ull : 0ull;
}

// Bound on the stream bytes of an n-qubit state in tiles of 2^c amplitudes
// under a codec.  AALC with theta > 0: the ratio threshold's size per tile,
// floor(16 * 2^c / theta) (the paper's ratio guarantee; a tile that no
// level brings under it shows in the measured footprint).  REL: the largest
// PACKED stream the format allows at the codec's shift s (two 4G-byte sign
// and zero sections per component, 2G width bytes, 65 - s bits per value
// and component, padding), at most the RAW size; a tile with a value
// outside the lossy range is stored losslessly and may reach RAW.  NONE and
// LOSSLESS: RAW.
unsigned long long qs_stream_bound(int n, int c, int codec, double eps, double theta) {
    const unsigned long long N = 1ull << c, G = N >= 32 ? N / 32 : 1;
    const unsigned long long ntiles = 1ull << (n - c);
    const unsigned long long raw = qs::HDR + 16ull * N;
    unsigned long long per = raw;
    if (codec == QSIM_CODEC_AALC && theta > 0.0) {
        per = std::min(raw, std::max<unsigned long long>(qs::HDR, round_up((unsigned long long)(16.0 * (double)N / theta), 16)));
    } else if (codec == QSIM_CODEC_REL || codec == QSIM_CODEC_AALC) {
        const int s = shift_for_eps(eps);
        const unsigned long long body = 16ull * G + round_up(2ull * G, 4) + N * (unsigned long long)(65 - s) / 4ull + 4ull;
        per = std::min(raw, round_up(qs::HDR + body, 16));
    }
    return ntiles * per;
}

extern "C" {

const char *qsim_version(void) { return "qsim-aalc 0.1 (sm_103a)"; }

qsim_status qsim_fp64_rate(int device, double *fma_per_s) {
    if (!fma_per_s) return fail(nullptr, QSIM_ERR_ARG, "null output");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_ERR_CUDA, "no CUDA device");
    }
    if (device < 0 || device >= count) return fail(nullptr, QSIM_ERR_ARG, "no device %d", device);
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess && cur != device) e = cudaSetDevice(device);
    if (e == cudaSuccess) e = qs::fp64_rate(device, fma_per_s);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, QSIM_ERR_CUDA, "fp64 probe: %s", cudaGetErrorString(e));
    }
    return QSIM_OK;
}

const char *qsim_last_error(qsim_t h) { return h ? h->err.c_str() : g_last_error.c_str(); }

qsim_status qsim_create(qsim_t *out, int n_qubits, int block_log2, qsim_codec codec, double rel_err_bound) {
    qsim_t h = nullptr;
    if (!out) return fail(nullptr, QSIM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > MAX_QUBITS) return fail(nullptr, QSIM_ERR_ARG, "n_qubits must be 1..%d", MAX_QUBITS);
    if (block_log2 < 1) return fail(nullptr, QSIM_ERR_ARG, "block_log2 must be >= 1");
    if (codec < QSIM_CODEC_NONE || codec > QSIM_CODEC_AALC) return fail(nullptr, QSIM_ERR_ARG, "unknown codec");
    if ((codec == QSIM_CODEC_REL || codec == QSIM_CODEC_AALC) && !(rel_err_bound >= 0.0 && rel_err_bound < 1.0))
        return fail(nullptr, QSIM_ERR_ARG, "rel_err_bound must be in [0, 1)");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(nullptr, QSIM_ERR_CUDA, "no CUDA device");
    h = new qsim_state();
    h->n = n_qubits;
    h->c = std::min(std::min(block_log2, n_qubits), DEFAULT_TILE_LOG2);
    h->hmax = qs::MAX_PAIRS;
    h->depth = qs::MAX_SWEEP_GATES;
    h->codec = codec;
    h->eps = rel_err_bound;
    qsim_status s = QSIM_OK;
    auto bail = [&](qsim_status code) { qsim_destroy(h); return code; };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(nullptr, QSIM_ERR_CUDA, "cudaGetDevice failed"));
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    const cudaError_t config_err = qs::configure_kernels();     // once per device
    if (config_err != cudaSuccess)
        return bail(fail(nullptr, QSIM_ERR_CUDA, "kernel setup: %s", cudaGetErrorString(config_err)));
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(nullptr, QSIM_ERR_CUDA, "stream creation failed"));
    h->stream = h->own_stream;
    if (cudaMalloc(&h->scal, sizeof(qs::DevScalars)) != cudaSuccess ||
        cudaMallocHost(&h->hscal, sizeof(qs::DevScalars)) != cudaSuccess)
        return bail(fail(nullptr, QSIM_ERR_OOM, "scalar allocation failed"));
    cudaMemset(h->scal, 0, sizeof(qs::DevScalars));
    set_codec(h);
    if ((s = alloc_tiles(h)) != QSIM_OK) { g_last_error = h->err; return bail(s); }
    if ((s = qsim_reset_basis(h, 0)) != QSIM_OK) { g_last_error = h->err; return bail(s); }
    *out = h;
    return QSIM_OK;
}

qsim_status qsim_destroy(qsim_t h) {
    if (!h) return QSIM_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_tiles(h);
    if (h->scal) cudaFree(h->scal);
    if (h->hscal) cudaFreeHost(h->hscal);
    if (h->dgates) cudaFree(h->dgates);
    if (h->hgates) cudaFreeHost(h->hgates);
    if (h->dsg) cudaFree(h->dsg);
    if (h->hsg) cudaFreeHost(h->hsg);
    if (h->dglist) cudaFree(h->dglist);
    if (h->dparams) cudaFree(h->dparams);
    if (h->hparams) cudaFreeHost(h->hparams);
    if (h->distart) cudaFree(h->distart);
    if (h->histart) cudaFreeHost(h->histart);
    if (h->used_hist) cudaFree(h->used_hist);
    if (h->hused) cudaFreeHost(h->hused);
    if (h->unit_bytes) cudaFree(h->unit_bytes);
    if (h->unit_level) cudaFree(h->unit_level);
    if (h->rd) cudaFree(h->rd);
    if (h->druns) cudaFree(h->druns);
    if (h->drg) cudaFree(h->drg);
    if (h->dclasses) cudaFree(h->dclasses);
    if (h->rtab) cudaFree(h->rtab);
    if (h->rmeta) cudaFree(h->rmeta);
    if (h->rcls) cudaFree(h->rcls);
    if (h->dbounds) cudaFree(h->dbounds);
    if (h->dscale) cudaFree(h->dscale);
    for (cudaEvent_t ev : h->events) cudaEventDestroy(ev);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return QSIM_OK;
}

qsim_status qsim_set_stream(qsim_t h, void *cuda_stream) {
    if (!h) return fail(nullptr, QSIM_ERR_ARG, "null handle");
    CK(cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    return QSIM_OK;
}

qsim_status qsim_set_pool(qsim_t h, void *dev_ptr, size_t bytes) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    CK(cudaStreamSynchronize(h->stream));
    if (!dev_ptr) {
        if (bytes) return fail(h, QSIM_ERR_ARG, "null pool with nonzero size");
        if (!h->pool) return QSIM_OK;
        // back to library-owned arenas: copy the current stream out
        const unsigned long long cap = std::max<unsigned long long>(round_up(h->used, 1ull << 21), 1ull << 22);
        uint8_t *own = nullptr;
        CK(cudaMalloc(&own, cap));
        cudaError_t e = hcopy(h, own, h->arena[h->cur], h->used, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { cudaFree(own); return fail(h, QSIM_ERR_CUDA, "set_pool: %s", cudaGetErrorString(e)); }
        h->arena[h->cur] = own;
        h->cap[h->cur] = cap;
        h->arena[h->cur ^ 1] = nullptr;
        h->cap[h->cur ^ 1] = 0;
        h->pool = false;
        return QSIM_OK;
    }
    if (reinterpret_cast<uintptr_t>(dev_ptr) & 255u) return fail(h, QSIM_ERR_ARG, "pool must be 256-byte aligned");
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, dev_ptr) != cudaSuccess || attr.type != cudaMemoryTypeDevice ||
        attr.device != h->device) {
        cudaGetLastError();
        return fail(h, QSIM_ERR_ARG, "pool is not device memory of the handle's GPU");
    }
    const unsigned long long half = ((unsigned long long)bytes / 2) & ~255ull;
    if (half < h->used || half < 4096) return fail(h, QSIM_ERR_ARG, "pool of %zu bytes cannot hold the state (%llu bytes per arena)", bytes, h->used);
    uint8_t *base = static_cast<uint8_t *>(dev_ptr);
    uint8_t *dst = base + (h->cur ? half : 0);
    CK(hcopy(h, dst, h->arena[h->cur], h->used, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (!h->pool)
        for (int i = 0; i < 2; ++i)
            if (h->arena[i]) cudaFree(h->arena[i]);
    h->arena[0] = base;
    h->arena[1] = base + half;
    h->cap[0] = h->cap[1] = half;
    h->pool = true;
    return QSIM_OK;
}

qsim_status qsim_reset_basis(qsim_t h, unsigned long long x) {
    if (!h) return fail(nullptr, QSIM_ERR_ARG, "null handle");
    if (h->invalid) return check_usable(h);
    if (x >> h->n) return fail(h, QSIM_ERR_ARG, "basis index out of range");
    h->queue.clear();
    qsim_status s = encode_fresh(h, nullptr, x);
    if (s == QSIM_OK) {
        h->st = qsim_stats_t{};
        h->st.stream_bytes = h->used;
        h->st.min_stream_bytes_seen = h->st.max_stream_bytes_seen = h->used;
    }
    return s;
}

qsim_status qsim_set_amplitudes(qsim_t h, const double *amps) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!amps) return fail(h, QSIM_ERR_ARG, "amps is NULL");
    h->queue.clear();
    size_t bytes = (size_t)16 << h->n;
    double2 *d = nullptr;
    CK(cudaMalloc(&d, bytes));
    cudaError_t e = hcopy(h, d, amps, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) s = encode_fresh(h, d, 0);
    cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "copy: %s", cudaGetErrorString(e));
    if (s == QSIM_OK) {
        h->st.stream_bytes = h->used;
        h->st.min_stream_bytes_seen = h->st.max_stream_bytes_seen = h->used;
    }
    return s;
}

qsim_status qsim_apply_gate(qsim_t h, const double *matrix, const int *targets, int n_targets,
                            const int *controls, int n_controls, unsigned long long control_values) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!matrix || !targets) return fail(h, QSIM_ERR_ARG, "matrix/targets NULL");
    if (n_targets < 1 || n_targets > 2) return fail(h, QSIM_ERR_ARG, "1 or 2 targets supported");
    if (n_controls < 0 || (n_controls > 0 && !controls)) return fail(h, QSIM_ERR_ARG, "bad controls");
    HostGate g{};
    g.k = n_targets;
    unsigned long long used = 0;
    for (int i = 0; i < n_targets; ++i) {
        int q = targets[i];
        if (q < 0 || q >= h->n) return fail(h, QSIM_ERR_ARG, "target %d out of range", q);
        if ((used >> q) & 1ull) return fail(h, QSIM_ERR_ARG, "repeated qubit %d", q);
        used |= 1ull << q;
        g.t[i] = q;
    }
    for (int i = 0; i < n_controls; ++i) {
        int q = controls[i];
        if (q < 0 || q >= h->n) return fail(h, QSIM_ERR_ARG, "control %d out of range", q);
        if ((used >> q) & 1ull) return fail(h, QSIM_ERR_ARG, "repeated qubit %d", q);
        used |= 1ull << q;
        g.cm |= 1ull << q;
        if (i >= 64 || ((control_values >> i) & 1ull)) g.cv |= 1ull << q;
    }
    int dim = 1 << n_targets;
    for (int i = 0; i < 2 * dim * dim; ++i) {
        if (!std::isfinite(matrix[i])) return fail(h, QSIM_ERR_ARG, "matrix entry not finite");
        g.m[i] = matrix[i];
    }
    // unitarity: max |(U^dagger U - I)_{ij}| <= 1e-12
    for (int i = 0; i < dim; ++i)
        for (int j = 0; j < dim; ++j) {
            double sr = 0, si = 0;
            for (int r = 0; r < dim; ++r) {
                double ar = g.m[2 * (r * dim + i)], ai = -g.m[2 * (r * dim + i) + 1];
                double br = g.m[2 * (r * dim + j)], bi = g.m[2 * (r * dim + j) + 1];
                sr += ar * br - ai * bi;
                si += ar * bi + ai * br;
            }
            if (std::fabs(sr - (i == j ? 1.0 : 0.0)) > UNITARY_TOL || std::fabs(si) > UNITARY_TOL)
                return fail(h, QSIM_ERR_ARG, "matrix is not unitary within 1e-12");
        }
    g.diag = matrix_is_diagonal(n_targets, g.m);
    if (!g.diag && h->hmax < 2 && n_targets == 2 && g.t[0] >= h->c && g.t[1] >= h->c && h->n - h->c >= 2)
        return fail(h, QSIM_ERR_ARG, "two high targets need hmax >= 2");
    h->queue.push_back(g);
    return QSIM_OK;
}

}  // extern "C"

namespace {

// One flush in progress: its sweeps and where its passes stand.
struct FlushCtx {
    std::vector<Sweep> sweeps;
    size_t ng = 0, ns = 0;
    int cur0 = 0;
    unsigned id0 = 0;
    unsigned long long used_before = 0;
    int regrows = 0;
    std::vector<int> run_first, nruns;    // per sweep: its diagonal runs
    std::vector<int> list_first, list_n;  // per sweep: its gates that can apply (hglist)
    std::vector<char> in_run;             // per gate: part of a diagonal run
    std::vector<char> scaled;             // per gate: a scaled gate applied without its d
    std::vector<char> sweep_scaled;       // per sweep: holds a scaled gate (its scale D is not 1)
    unsigned long long run_dp0 = 0;       // device FP64 count of runs when the flush began
};

constexpr int MAX_FLUSH_RUNS = 32767;     // SGate::run is 16-bit
constexpr unsigned long long MAX_RUN_TABLE = 1ull << 22;   // table entries per flush (17 bytes each)

// A diagonal gate in the form a run evaluates: entries classified exactly
// (1 contributes nothing; -1, i, -i are unit factors; the rest general).
qs::RGate run_gate(const HostGate &g) {
    qs::RGate r{};
    const int dim = 1 << g.k;
    r.k = (uint8_t)g.k;
    r.t0 = (uint8_t)g.t[0];
    r.t1 = (uint8_t)(g.k > 1 ? g.t[1] : 0);
    r.cm = g.cm;
    r.cv = g.cv;
    for (int i = 0; i < dim; ++i) {
        const double ur = g.m[2 * (i * dim + i)], ui = g.m[2 * (i * dim + i) + 1];
        r.e[2 * i] = ur;
        r.e[2 * i + 1] = ui;
        if (ur == 1.0 && ui == 0.0) r.code[i] = 0;
        else if (ur == -1.0 && ui == 0.0) { r.code[i] = 1; r.uexp[i] = 2; }
        else if (ur == 0.0 && ui == 1.0) { r.code[i] = 1; r.uexp[i] = 1; }
        else if (ur == 0.0 && ui == -1.0) { r.code[i] = 1; r.uexp[i] = 3; }
        else r.code[i] = 2;
    }
    return r;
}

// every target and control of g is a qubit >= c (its factor is constant over a tile)
bool on_high_qubits(const HostGate &g, int c) {
    if (g.cm & ((1ull << c) - 1ull)) return false;
    for (int i = 0; i < g.k; ++i)
        if (g.t[i] < c) return false;
    return true;
}

// Find the diagonal runs of every sweep of a flush (two or more consecutive
// diagonal gates), mark their gates in the staged compact gates, and build
// the run descriptors, run gates and table classes.
void plan_runs(qsim_t h, FlushCtx &fc) {
    h->hruns.clear();
    h->hrg.clear();
    h->hclasses.clear();
    fc.run_first.assign(fc.ns, 0);
    fc.nruns.assign(fc.ns, 0);
    fc.in_run.assign(fc.ng, 0);
    unsigned long long tab = 0;
    int cls = 0;
    for (size_t si = 0; si < fc.ns; ++si) {
        const Sweep &sw = fc.sweeps[si];
        fc.run_first[si] = (int)h->hruns.size();
        int i = sw.lo;
        while (i < sw.hi) {
            int j = i;
            if (h->fuse)
                while (j < sw.hi && h->queue[j].diag) ++j;
            if (j - i < 2 || (int)h->hruns.size() >= MAX_FLUSH_RUNS) { i = std::max(i + 1, j); continue; }
            qs::DRun R{};
            R.first = i - sw.lo;
            R.len = j - i;
            unsigned long long qmask = 0;
            std::vector<qs::RGate> tile, local;
            for (int g = i; g < j; ++g) {
                const HostGate &hg = h->queue[g];
                if (on_high_qubits(hg, h->c)) { tile.push_back(run_gate(hg)); continue; }
                local.push_back(run_gate(hg));
                qmask |= hg.cm & ~((1ull << h->c) - 1ull);
                for (int t = 0; t < hg.k; ++t)
                    if (hg.t[t] >= h->c) qmask |= 1ull << hg.t[t];
            }
            R.tg = (int)h->hrg.size();
            R.nt = (int)tile.size();
            h->hrg.insert(h->hrg.end(), tile.begin(), tile.end());
            R.lg = (int)h->hrg.size();
            R.nl = (int)local.size();
            h->hrg.insert(h->hrg.end(), local.begin(), local.end());
            R.nq = popcount64(qmask);
            const unsigned long long entries = (1ull << R.nq) << h->c;
            R.tabled = R.nl > 0 && R.nq <= qs::RUN_QMAX && tab + entries <= MAX_RUN_TABLE;
            if (R.tabled) {
                int b = 0;
                for (int q = 0; q < 64; ++q)
                    if ((qmask >> q) & 1ull) R.q[b++] = q;
                R.table = tab;
                R.cls = cls;
                const int rid = (int)h->hruns.size();
                for (int kap = 0; kap < (1 << R.nq); ++kap) h->hclasses.push_back(make_int2(rid, kap));
                tab += entries;
                cls += 1 << R.nq;
            } else {
                R.nq = 0;
            }
            h->hsg[i].run = (int16_t)h->hruns.size();
            for (int g = i; g < j; ++g) fc.in_run[g] = 1;
            for (int g = i + 1; g < j; ++g) h->hsg[g].run = -2;
            h->hruns.push_back(R);
            i = j;
        }
        fc.nruns[si] = (int)h->hruns.size() - fc.run_first[si];
    }
}

// Upload the flush's runs and build their tables on the device (stream st).
qsim_status stage_runs(qsim_t h, FlushCtx &fc, cudaStream_t st) {
    fc.run_dp0 = h->hscal->run_dp;
    if (h->hruns.empty()) return QSIM_OK;
    auto grow = [&](void **p, size_t &cap, size_t need, size_t unit) -> cudaError_t {
        if (cap >= need) return cudaSuccess;
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        if (*p) cudaFree(*p);
        *p = nullptr;
        cap = 0;
        const size_t n = std::max<size_t>(need, 16);
        e = cudaMalloc(p, n * unit);
        if (e == cudaSuccess) cap = n;
        return e;
    };
    unsigned long long entries = 0;
    int ncls = 0;
    for (const qs::DRun &R : h->hruns)
        if (R.tabled) { entries += (1ull << R.nq) << h->c; ncls += 1 << R.nq; }
    CK(grow((void **)&h->druns, h->druns_cap, h->hruns.size(), sizeof(qs::DRun)));
    CK(grow((void **)&h->drg, h->drg_cap, std::max<size_t>(1, h->hrg.size()), sizeof(qs::RGate)));
    CK(hcopy(h, h->druns, h->hruns.data(), h->hruns.size() * sizeof(qs::DRun), cudaMemcpyHostToDevice, st));
    if (!h->hrg.empty())
        CK(hcopy(h, h->drg, h->hrg.data(), h->hrg.size() * sizeof(qs::RGate), cudaMemcpyHostToDevice, st));
    if (ncls == 0) return QSIM_OK;
    CK(grow((void **)&h->dclasses, h->dclasses_cap, (size_t)ncls, sizeof(int2)));
    CK(grow((void **)&h->rcls, h->rcls_cap, (size_t)ncls, sizeof(qs::RunClass)));
    CK(grow((void **)&h->rtab, h->rtab_cap, (size_t)entries, sizeof(double2)));
    CK(grow((void **)&h->rmeta, h->rmeta_cap, (size_t)entries, 1));
    CK(hcopy(h, h->dclasses, h->hclasses.data(), (size_t)ncls * sizeof(int2), cudaMemcpyHostToDevice, st));
    ++h->launches;
    CK(qs::launch_run_tables(h->druns, h->dclasses, ncls, h->drg, h->c, h->rtab, h->rmeta, h->rcls, h->scal,
                             grid_for(h, (unsigned long long)ncls, 4), st));
    return QSIM_OK;
}

// Plan the queued gates into sweeps and upload them (prepared for their
// sweep) on stream st; size the per-sweep buffers.
qsim_status stage_flush(qsim_t h, FlushCtx &fc, cudaStream_t st) {
    if (plan_sweeps(h->n, h->c, h->hmax, h->depth, h->queue, fc.sweeps) < 0)
        return fail(h, QSIM_ERR_ARG, "a gate needs more paired qubits than hmax");
    const size_t ng = h->queue.size(), ns = fc.sweeps.size();
    fc.ng = ng;
    fc.ns = ns;
    if (h->hgates_cap < ng) {
        if (h->hgates) cudaFreeHost(h->hgates);
        if (h->hsg) cudaFreeHost(h->hsg);
        h->hgates = nullptr;
        h->hsg = nullptr;
        h->hgates_cap = 0;
        CK(cudaMallocHost(&h->hgates, ng * sizeof(qs::DGate)));
        CK(cudaMallocHost(&h->hsg, ng * sizeof(qs::SGate)));
        h->hgates_cap = ng;
    }
    if (h->dgates_cap < ng) {
        CK(cudaStreamSynchronize(st));
        if (h->dgates) cudaFree(h->dgates);
        if (h->dsg) cudaFree(h->dsg);
        if (h->dglist) cudaFree(h->dglist);
        h->dgates = nullptr;
        h->dsg = nullptr;
        h->dglist = nullptr;
        h->dgates_cap = 0;
        CK(cudaMalloc(&h->dgates, ng * sizeof(qs::DGate)));
        CK(cudaMalloc(&h->dsg, ng * sizeof(qs::SGate)));
        CK(cudaMalloc(&h->dglist, ng * sizeof(int)));
        h->dgates_cap = ng;
    }
    if (h->used_hist_cap < ns) {
        CK(cudaStreamSynchronize(st));
        if (h->used_hist) cudaFree(h->used_hist);
        if (h->hused) cudaFreeHost(h->hused);
        h->used_hist = nullptr;
        h->hused = nullptr;
        h->used_hist_cap = 0;
        CK(cudaMalloc(&h->used_hist, ns * sizeof(unsigned long long)));
        CK(cudaMallocHost(&h->hused, ns * sizeof(unsigned long long)));
        h->used_hist_cap = ns;
    }
    if (h->params_cap < ns) {
        CK(cudaStreamSynchronize(st));
        if (h->dparams) cudaFree(h->dparams);
        if (h->hparams) cudaFreeHost(h->hparams);
        if (h->distart) cudaFree(h->distart);
        if (h->histart) cudaFreeHost(h->histart);
        h->dparams = h->hparams = nullptr;
        h->distart = h->histart = nullptr;
        h->params_cap = 0;
        CK(cudaMalloc(&h->dparams, 2 * ns * sizeof(qs::SweepParams)));    // encode, sizing
        CK(cudaMallocHost(&h->hparams, 2 * ns * sizeof(qs::SweepParams)));
        CK(cudaMalloc(&h->distart, 2 * ns * sizeof(unsigned long long)));
        CK(cudaMallocHost(&h->histart, 2 * ns * sizeof(unsigned long long)));
        h->params_cap = ns;
    }
    for (size_t si = 0; si < ns; ++si)
        for (int gi = fc.sweeps[si].lo; gi < fc.sweeps[si].hi; ++gi)
            prepare_gate(h->queue[gi], h->c, fc.sweeps[si], h->hgates[gi], h->hsg[gi]);
    fc.scaled.assign(ng, 0);
    fc.sweep_scaled.assign(ns, 0);
    if (h->fuse)
        for (size_t si = 0; si < ns; ++si)
            for (int gi = fc.sweeps[si].lo; gi < fc.sweeps[si].hi; ++gi)
                if (is_scaled_gate(h->queue[gi])) {
                    // FP64 instructions of one group of 2^k amplitudes (4 for a
                    // Hadamard, at most 24): the device counts the groups it forms
                    const HostGate &g = h->queue[gi];
                    h->hsg[gi].unscaled = (uint8_t)std::max(1.0, gate_dp_ops(g, g.k, true));
                    fc.scaled[gi] = 1;
                    fc.sweep_scaled[si] = 1;
                }
    plan_runs(h, fc);
    // per sweep, the gates that can apply: all but the later gates of runs
    h->hglist.clear();
    fc.list_first.assign(ns, 0);
    fc.list_n.assign(ns, 0);
    for (size_t si = 0; si < ns; ++si) {
        fc.list_first[si] = (int)h->hglist.size();
        for (int gi = fc.sweeps[si].lo; gi < fc.sweeps[si].hi; ++gi)
            if (h->hsg[gi].run != -2) h->hglist.push_back(gi - fc.sweeps[si].lo);
        fc.list_n[si] = (int)h->hglist.size() - fc.list_first[si];
    }
    if (!h->hglist.empty())
        CK(hcopy(h, h->dglist, h->hglist.data(), h->hglist.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(hcopy(h, h->dgates, h->hgates, ng * sizeof(qs::DGate), cudaMemcpyHostToDevice, st));
    CK(hcopy(h, h->dsg, h->hsg, ng * sizeof(qs::SGate), cudaMemcpyHostToDevice, st));
    {
        qsim_status rs = stage_runs(h, fc, st);
        if (rs != QSIM_OK) return rs;
    }
    // the scale D of every sweep (product of its scaled gates' d), on the device
    if (h->scale_cap < ns) {
        CK(cudaStreamSynchronize(st));
        if (h->dbounds) cudaFree(h->dbounds);
        if (h->dscale) cudaFree(h->dscale);
        h->dbounds = nullptr;
        h->dscale = nullptr;
        h->scale_cap = 0;
        const size_t cap = std::max<size_t>(ns, 64);
        CK(cudaMalloc(&h->dbounds, cap * sizeof(int2)));
        CK(cudaMalloc(&h->dscale, cap * sizeof(double)));
        h->scale_cap = cap;
    }
    h->hbounds.resize(ns);
    for (size_t si = 0; si < ns; ++si) h->hbounds[si] = make_int2(fc.sweeps[si].lo, fc.sweeps[si].hi);
    CK(hcopy(h, h->dbounds, h->hbounds.data(), ns * sizeof(int2), cudaMemcpyHostToDevice, st));
    ++h->launches;
    CK(qs::launch_sweep_scales(h->dsg, h->dgates, h->dbounds, (int)ns, h->dscale, st));
    if (h->profiling) {
        while (h->events.size() < 2 * ns) {
            cudaEvent_t ev;
            CK(cudaEventCreate(&ev));
            h->events.push_back(ev);
        }
    }
    fc.used_before = h->used;
    fc.cur0 = h->cur;
    fc.id0 = h->sweep_counter;
    fc.regrows = 0;
    // the output of a pass rarely needs more than its input plus this slack;
    // an overflow is re-run with the exact size
    const unsigned long long first_need =
        std::max<unsigned long long>(h->used + h->used / 4 + (1ull << 20), 1ull << 22);
    if (h->pool) return QSIM_OK;          // fixed arenas: a pass that overflows fails
    return ensure_arena(h, h->cur ^ 1, first_need);
}

// Parameters of sweep j of a flush (arena parity alternates per sweep).
qs::SweepParams sweep_params(qsim_t h, const FlushCtx &fc, size_t j) {
    const Sweep &sw = fc.sweeps[j];
    const int in = fc.cur0 ^ (int)(j & 1), outa = in ^ 1;
    qs::SweepParams p{};
    p.in_arena = h->arena[in];
    p.in_table = h->table[in];
    p.out_arena = h->arena[outa];
    p.out_table = h->table[outa];
    p.out_cap = h->cap[outa];
    p.part = h->part;
    p.scal = h->scal;
    p.gates = h->dgates + sw.lo;
    p.sgates = h->dsg + sw.lo;
    p.ngates = sw.hi - sw.lo;
    p.n = h->n;
    p.h = sw.h;
    for (int i = 0; i < 4; ++i) p.H[i] = sw.H[i];
    p.cc = h->cc;
    p.nitems = h->ntiles >> sw.h;
    p.sweep_id = fc.id0 + (unsigned)j;
    p.runs = h->druns;
    p.rgates = h->drg;
    p.rtab = h->rtab;
    p.rmeta = h->rmeta;
    p.rcls = h->rcls;
    p.run_first = fc.run_first.empty() ? 0 : fc.run_first[j];
    p.nruns = fc.nruns.empty() ? 0 : fc.nruns[j];
    p.dscale = (!fc.sweep_scaled.empty() && fc.sweep_scaled[j]) ? h->dscale + j : nullptr;
    p.use_alpha = h->normalize;
    p.low_free = 1;
    p.moves_tiles = 1;
    const unsigned long long lowm = (1ull << h->c) - 1ull;
    for (int gi = sw.lo; gi < sw.hi && p.low_free; ++gi) {
        const HostGate &g = h->queue[gi];
        if (g.cm & lowm) p.low_free = 0;
        for (int i = 0; i < g.k; ++i)
            if (g.t[i] < h->c) p.low_free = 0;
        if (!is_permutation(g)) p.moves_tiles = 0;
    }
    p.moves_tiles &= p.low_free;
    // point items (every tile zero but for one amplitude at a common index,
    // the zeros +0): the sweep's gates leave the zeros as they are when each
    // is a member of a diagonal run, a scaled gate or a permutation, and the
    // mixing ones act on qubits >= c only
    p.glist = h->dglist + fc.list_first[j];
    p.nglist = fc.list_n[j];
    p.point_ok = h->fuse && !fc.in_run.empty();
    for (int gi = sw.lo; gi < sw.hi && p.point_ok; ++gi) {
        if (fc.in_run[gi]) continue;
        const HostGate &g = h->queue[gi];
        bool high = !(g.cm & lowm);
        for (int i = 0; i < g.k; ++i)
            if (g.t[i] < h->c) high = false;
        if (!high || !(fc.scaled[gi] || is_permutation(g))) p.point_ok = 0;
    }
    if (const int ut = unit_tiles_log2(h)) {
        // every stride is decided and re-encoded as a whole
        p.every_item = 1;
        p.moves_tiles = 0;
        p.unit_shift = ut;
        p.unit_level = h->unit_level;
    }
    return p;
}

// Run sweeps k .. ns-1 of a flush on the handle's stream, growing the
// output arena and re-running a pass whenever it overflows.
qsim_status run_from(qsim_t h, FlushCtx &fc, size_t k) {
    qsim_status s;
    const size_t ns = fc.ns;
    const int ut = unit_tiles_log2(h);
    const unsigned long long nunits = h->ntiles >> ut;
    if (ut && (s = ensure_units(h, nunits)) != QSIM_OK) return s;
    while (k < ns) {
        for (size_t j = k; j < ns; ++j) {
            h->hparams[j] = sweep_params(h, fc, j);
            h->histart[2 * j] = 0;
            h->histart[2 * j + 1] = h->hparams[j].nitems;
            if (ut) {                     // the sizing pass: same sweep, counts only
                h->hparams[ns + j] = h->hparams[j];
                h->hparams[ns + j].unit_level = nullptr;
                h->hparams[ns + j].unit_bytes = h->unit_bytes;
            }
        }
        CK(hcopy(h, h->dparams + k, h->hparams + k, (ns - k) * sizeof(qs::SweepParams),
                           cudaMemcpyHostToDevice, h->stream));
        if (ut)
            CK(hcopy(h, h->dparams + ns + k, h->hparams + ns + k, (ns - k) * sizeof(qs::SweepParams),
                               cudaMemcpyHostToDevice, h->stream));
        CK(hcopy(h, h->distart + 2 * k, h->histart + 2 * k, 2 * (ns - k) * sizeof(unsigned long long),
                           cudaMemcpyHostToDevice, h->stream));
        for (size_t j = k; j < ns; ++j) {
            const int mb = h->c + fc.sweeps[j].h;
            const int per_sm = qs::sweep_blocks_per_sm(mb, h->threads);
            char label[64];
            std::snprintf(label, sizeof label, "qsim sweep %u (%d gates)", fc.id0 + (unsigned)j,
                          fc.sweeps[j].hi - fc.sweeps[j].lo);
            NvtxRange range(label);
            if (h->profiling) CK(cudaEventRecord(h->events[2 * j], h->stream));
            if (ut) {                     // Algorithm 2's ratio test once per stride
                CK(cudaMemsetAsync(h->unit_bytes, 0, nunits * qs::MAX_LEVELS * sizeof(unsigned long long),
                                   h->stream));
                ++h->launches;
                CK(qs::launch_sweep_sizing(h->dparams + ns + j, h->distart + 2 * j, 1, mb,
                                           grid_for(h, h->hparams[j].nitems, per_sm), h->threads,
                                           &h->scal->work, h->stream));
                ++h->launches;
                CK(qs::launch_unit_level(h->unit_bytes, h->unit_level, nunits, h->cc.nlev, unit_limit(h),
                                         h->stream));
            }
            ++h->launches;
            CK(qs::launch_sweep(h->dparams + j, h->distart + 2 * j, 1, mb,
                                grid_for(h, h->hparams[j].nitems, per_sm), h->threads, &h->scal->work,
                                h->stream));
            if (h->profiling) CK(cudaEventRecord(h->events[2 * j + 1], h->stream));
            ++h->launches;
            CK(qs::launch_finalize(h->scal, h->normalize, h->used_hist, (unsigned)j, 1, h->stream));
        }
        if ((s = read_scalars(h)) != QSIM_OK) return s;
        const unsigned err = h->hscal->err;
        if (err & qs::ERR_OVERFLOW) {
            const unsigned failed = h->hscal->err_sweep - 1u - fc.id0;
            if (failed >= ns) return device_error(h, err);
            const int outa = (fc.cur0 ^ (int)(failed & 1)) ^ 1;
            const unsigned long long need = h->hscal->bump + h->hscal->bump / 8 + (1ull << 20);
            if ((s = ensure_arena(h, outa, need)) != QSIM_OK) return s;
            if ((s = clear_pass_state(h)) != QSIM_OK) return s;
            k = failed;
            ++fc.regrows;
            continue;
        }
        if (err) return device_error(h, err);
        break;
    }
    return QSIM_OK;
}

// Bookkeeping after every pass of a flush has succeeded.
qsim_status finish_flush(qsim_t h, FlushCtx &fc, bool timed) {
    const size_t ns = fc.ns;
    if (ns) h->basis = false;
    CK(hcopy(h, h->hused, h->used_hist, ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->cur = fc.cur0 ^ (int)(ns & 1);
    h->used = h->hscal->used;
    h->sweep_counter += (unsigned)ns;
    h->st.gates += fc.ng;
    h->st.sweeps += ns;
    h->st.arena_regrows += (unsigned long long)fc.regrows;
    for (size_t j = 0; j < ns; ++j) {
        h->st.min_stream_bytes_seen = std::min(h->st.min_stream_bytes_seen, h->hused[j]);
        h->st.max_stream_bytes_seen = std::max(h->st.max_stream_bytes_seen, h->hused[j]);
    }
    h->st.stream_bytes = h->used;
    if (h->profiling && timed) {
        for (size_t j = 0; j < ns; ++j) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, h->events[2 * j], h->events[2 * j + 1]));
            h->prof.sweep_ms += ms;
            h->prof.sweep_launches += 1;
            // the decompression scale: normalize and / or the scaled gates' D
            // (none in sweeps that move whole tiles: nothing is decompressed)
            const bool moved = sweep_params(h, fc, j).moves_tiles != 0;
            double dp = (!moved && (h->normalize || fc.sweep_scaled[j])) ? 2.0 * std::ldexp(1.0, h->n) : 0.0;
            for (int gi = fc.sweeps[j].lo; gi < fc.sweeps[j].hi; ++gi)
                if (!fc.in_run[gi] && !fc.scaled[gi]) dp += gate_dp_ops(h->queue[gi], h->n);
            h->prof.dp_ops += dp;
            const unsigned long long in = j == 0 ? fc.used_before : h->hused[j - 1];
            h->prof.bytes += (double)in + (double)h->hused[j] + 32.0 * (double)h->ntiles;
        }
    }
    if (h->profiling && timed)             // diagonal runs and scaled gates: counted on the device as executed
        h->prof.dp_ops += (double)(h->hscal->run_dp - fc.run_dp0);
    h->queue.clear();
    return QSIM_OK;
}

// Per-process workspace of batched flushes (grown, never shrunk).
struct BatchSpace {
    qs::SweepParams *dP = nullptr, *hP = nullptr;
    unsigned long long *dI = nullptr, *hI = nullptr;
    qs::FinalizeEntry *dF = nullptr, *hF = nullptr;
    unsigned long long *dW = nullptr;     // item counter of the round in flight
    size_t capP = 0, capI = 0;
} g_batch;
std::mutex g_batch_mutex;                 // one batched flush at a time uses g_batch

}  // namespace

extern "C" {

qsim_status qsim_flush(qsim_t h) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (h->queue.empty()) return QSIM_OK;
    NvtxRange range("qsim_flush");
    FlushCtx fc;
    if ((s = stage_flush(h, fc, h->stream)) != QSIM_OK) return s;
    if ((s = run_from(h, fc, 0)) != QSIM_OK) {
        // passes may have overwritten the input arena: the state is lost
        h->invalid = true;
        return s;
    }
    return finish_flush(h, fc, true);
}

qsim_status qsim_flush_batch(qsim_t *handles, int count, int use_graph) {
    if (!handles || count < 1) return fail(nullptr, QSIM_ERR_ARG, "qsim_flush_batch: no handles");
    std::lock_guard<std::mutex> batch_lock(g_batch_mutex);
    for (int i = 0; i < count; ++i) {
        if (!handles[i]) return fail(nullptr, QSIM_ERR_ARG, "qsim_flush_batch: NULL handle");
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return fail(nullptr, QSIM_ERR_ARG, "qsim_flush_batch: repeated handle");
        qsim_status s = check_usable(handles[i]);
        if (s != QSIM_OK) return s;
        if (unit_tiles_log2(handles[i]))
            return fail(handles[i], QSIM_ERR_ARG, "qsim_flush_batch: per-stride ladder decisions run through qsim_flush");
        if (handles[i]->device != handles[0]->device)
            return fail(nullptr, QSIM_ERR_ARG, "qsim_flush_batch: handles on different devices");
    }
    qsim_t h0 = handles[0];
    cudaStream_t st = h0->stream;
    for (int i = 1; i < count; ++i)
        if (handles[i]->stream != st && cudaStreamSynchronize(handles[i]->stream) != cudaSuccess)
            return fail(handles[i], QSIM_ERR_CUDA, "stream synchronisation failed");
    std::vector<FlushCtx> fcs(count);
    size_t rounds = 0, entries = 0;
    for (int i = 0; i < count; ++i) {
        qsim_t h = handles[i];
        if (h->queue.empty()) continue;
        qsim_status s = stage_flush(h, fcs[i], st);
        if (s != QSIM_OK) return s;
        rounds = std::max(rounds, fcs[i].ns);
        entries += fcs[i].ns;
    }
    if (rounds == 0) return QSIM_OK;
    qsim_t h = h0;   // for CK messages
    // work lists: round r holds sweep r of every handle that has one
    if (g_batch.capP < entries || g_batch.capI < entries + rounds) {
        CK(cudaStreamSynchronize(st));
        if (g_batch.dP) cudaFree(g_batch.dP);
        if (g_batch.hP) cudaFreeHost(g_batch.hP);
        if (g_batch.dI) cudaFree(g_batch.dI);
        if (g_batch.hI) cudaFreeHost(g_batch.hI);
        if (g_batch.dF) cudaFree(g_batch.dF);
        if (g_batch.hF) cudaFreeHost(g_batch.hF);
        if (g_batch.dW) cudaFree(g_batch.dW);
        g_batch = BatchSpace{};
        const size_t cp = std::max<size_t>(entries, 64), ci = cp + std::max<size_t>(rounds, 64);
        CK(cudaMalloc(&g_batch.dP, cp * sizeof(qs::SweepParams)));
        CK(cudaMallocHost(&g_batch.hP, cp * sizeof(qs::SweepParams)));
        CK(cudaMalloc(&g_batch.dF, cp * sizeof(qs::FinalizeEntry)));
        CK(cudaMallocHost(&g_batch.hF, cp * sizeof(qs::FinalizeEntry)));
        CK(cudaMalloc(&g_batch.dI, ci * sizeof(unsigned long long)));
        CK(cudaMallocHost(&g_batch.hI, ci * sizeof(unsigned long long)));
        CK(cudaMalloc(&g_batch.dW, sizeof(unsigned long long)));
        g_batch.capP = cp;
        g_batch.capI = ci;
    }
    std::vector<size_t> rstart(rounds + 1), rmb(rounds), ritems(rounds);
    size_t e = 0, ii = 0;
    std::vector<size_t> istart_at(rounds);
    for (size_t r = 0; r < rounds; ++r) {
        rstart[r] = e;
        istart_at[r] = ii;
        unsigned long long acc = 0;
        int mb = 0;
        for (int i = 0; i < count; ++i) {
            if (fcs[i].ns <= r) continue;
            qsim_t hh = handles[i];
            g_batch.hP[e] = sweep_params(hh, fcs[i], r);
            g_batch.hF[e] = qs::FinalizeEntry{hh->scal, hh->used_hist, (unsigned)r, hh->normalize, 1};
            g_batch.hI[ii++] = acc;
            acc += g_batch.hP[e].nitems;
            mb = std::max(mb, hh->c + fcs[i].sweeps[r].h);
            ++e;
        }
        g_batch.hI[ii++] = acc;
        rmb[r] = (size_t)mb;
        ritems[r] = acc;
    }
    rstart[rounds] = e;
    CK(cudaMemcpyAsync(g_batch.dP, g_batch.hP, e * sizeof(qs::SweepParams), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g_batch.dF, g_batch.hF, e * sizeof(qs::FinalizeEntry), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g_batch.dI, g_batch.hI, ii * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    NvtxRange range("qsim_flush_batch");
    if (use_graph) CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    for (size_t r = 0; r < rounds; ++r) {
        const int n_r = (int)(rstart[r + 1] - rstart[r]);
        const int mb = (int)rmb[r];
        const int per_sm = qs::sweep_blocks_per_sm(mb, h0->threads);
        cudaError_t le = qs::launch_sweep(g_batch.dP + rstart[r], g_batch.dI + istart_at[r], n_r, mb,
                                          grid_for(h0, ritems[r], per_sm), h0->threads, g_batch.dW, st);
        if (le == cudaSuccess) le = qs::launch_finalize_list(g_batch.dF + rstart[r], n_r, st);
        if (le != cudaSuccess) {
            if (use_graph) { cudaStreamEndCapture(st, &graph); if (graph) cudaGraphDestroy(graph); }
            return fail(h0, QSIM_ERR_CUDA, "batched launch: %s", cudaGetErrorString(le));
        }
        h0->launches += 2;
    }
    if (use_graph) {
        CK(cudaStreamEndCapture(st, &graph));
        cudaError_t ge = cudaGraphInstantiate(&exec, graph, 0);
        if (ge == cudaSuccess) ge = cudaGraphLaunch(exec, st);
        if (ge == cudaSuccess) ge = cudaStreamSynchronize(st);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ge != cudaSuccess) return fail(h0, QSIM_ERR_CUDA, "batch graph: %s", cudaGetErrorString(ge));
    }
    CK(cudaStreamSynchronize(st));
    // per handle: finish, or grow and re-run from its failed pass
    qsim_status first_err = QSIM_OK;
    for (int i = 0; i < count; ++i) {
        qsim_t hh = handles[i];
        FlushCtx &fc = fcs[i];
        if (fc.ns == 0) continue;
        qsim_status s = read_scalars(hh);
        if (s == QSIM_OK) {
            const unsigned err = hh->hscal->err;
            if (err & qs::ERR_OVERFLOW) {
                const unsigned failed = hh->hscal->err_sweep - 1u - fc.id0;
                if (failed >= fc.ns) s = device_error(hh, err);
                else {
                    const int outa = (fc.cur0 ^ (int)(failed & 1)) ^ 1;
                    const unsigned long long need = hh->hscal->bump + hh->hscal->bump / 8 + (1ull << 20);
                    s = ensure_arena(hh, outa, need);
                    if (s == QSIM_OK) s = clear_pass_state(hh);
                    ++fc.regrows;
                    if (s == QSIM_OK) s = run_from(hh, fc, failed);
                }
            } else if (err) {
                s = device_error(hh, err);
            }
        }
        if (s == QSIM_OK) s = finish_flush(hh, fc, false);
        else hh->invalid = true;          // passes may have overwritten its input arena
        if (s != QSIM_OK && first_err == QSIM_OK) first_err = s;
    }
    if (first_err != QSIM_OK) g_last_error = "qsim_flush_batch: a handle failed (see its qsim_last_error)";
    return first_err;
}

qsim_status qsim_set_profiling(qsim_t h, int on) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->profiling = on ? 1 : 0;
    h->prof = qsim_profile_t{};
    return QSIM_OK;
}

qsim_status qsim_profile(qsim_t h, qsim_profile_t *out) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!out) return fail(h, QSIM_ERR_ARG, "out is NULL");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    *out = h->prof;
    out->kernel_launches = h->launches;
    return QSIM_OK;
}

qsim_status qsim_set_aalc(qsim_t h, double theta, const double *eps_levels, int n_levels) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (h->codec != QSIM_CODEC_AALC) return fail(h, QSIM_ERR_ARG, "handle does not use the AALC codec");
    if (!(theta > 0.0) || !std::isfinite(theta)) return fail(h, QSIM_ERR_ARG, "theta must be > 0");
    if (n_levels < 0 || n_levels > qs::MAX_LEVELS - 1 || (n_levels > 0 && !eps_levels))
        return fail(h, QSIM_ERR_ARG, "0..%d levels", qs::MAX_LEVELS - 1);
    for (int i = 0; i < n_levels; ++i)
        if (!(eps_levels[i] > 0.0 && eps_levels[i] < 1.0) || (i && eps_levels[i] <= eps_levels[i - 1]))
            return fail(h, QSIM_ERR_ARG, "levels must ascend in (0, 1)");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->theta = theta;
    h->cc.nlev = 1 + n_levels;
    h->cc.shifts[0] = 0;
    for (int i = 0; i < n_levels; ++i) h->cc.shifts[1 + i] = shift_for_eps(eps_levels[i]);
    h->cc.max_bytes = (unsigned long long)std::floor(16.0 * (double)(1ull << h->c) / theta);
    return QSIM_OK;
}

qsim_status qsim_set_aalc_unit(qsim_t h, int unit_log2) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (unit_log2 < 0 || unit_log2 > MAX_QUBITS) return fail(h, QSIM_ERR_ARG, "unit_log2 must be 0..%d", MAX_QUBITS);
    if ((s = qsim_flush(h)) != QSIM_OK) return s;     // queued gates run under the old rule
    h->unit_log2 = unit_log2;
    return QSIM_OK;
}

qsim_status qsim_set_polar(qsim_t h, int on) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (h->codec != QSIM_CODEC_REL && h->codec != QSIM_CODEC_AALC)
        return fail(h, QSIM_ERR_ARG, "the POLAR mode needs a lossy codec (REL or AALC)");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->polar = on ? 1 : 0;
    h->cc.polar = h->polar;
    return QSIM_OK;
}

qsim_status qsim_set_sweep_threads(qsim_t h, int threads) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!qs::sweep_threads_ok(threads)) return fail(h, QSIM_ERR_ARG, "sweep threads must be 128, 256 or 512");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->threads = threads;
    return QSIM_OK;
}

qsim_status qsim_set_fusion(qsim_t h, int diag_runs) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->fuse = diag_runs ? 1 : 0;
    return QSIM_OK;
}

qsim_status qsim_set_normalize(qsim_t h, int on) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (h->codec != QSIM_CODEC_REL && h->codec != QSIM_CODEC_AALC)
        return fail(h, QSIM_ERR_ARG, "normalize applies to REL and AALC handles");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->normalize = on ? 1 : 0;
    // the scale of the next pass follows the switch
    CK(cudaMemsetAsync(&h->scal->acc_lo, 0, 2 * sizeof(unsigned long long), h->stream));
    ++h->launches; CK(qs::launch_norm_from_parts(h->part, h->ntiles, h->scal, grid_for(h, h->ntiles / qs::THREADS + 1, 4), h->stream));
    ++h->launches; CK(qs::launch_finalize(h->scal, h->normalize, nullptr, 0, 0, h->stream));
    return read_scalars(h);
}

qsim_status qsim_set_schedule(qsim_t h, int tile_log2, int hmax, int depth) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (tile_log2 < 1 || tile_log2 > qs::MAX_C || tile_log2 > h->n) return fail(h, QSIM_ERR_ARG, "tile_log2 must be 1..min(10, n)");
    if (hmax < 1 || hmax > qs::MAX_PAIRS || tile_log2 + hmax > qs::MAX_ITEM_LOG2)
        return fail(h, QSIM_ERR_ARG, "hmax must be 1..4 with tile_log2 + hmax <= 12");
    if (depth < 1 || depth > qs::MAX_SWEEP_GATES) return fail(h, QSIM_ERR_ARG, "depth must be 1..%d", qs::MAX_SWEEP_GATES);
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->hmax = hmax;
    h->depth = depth;
    if (tile_log2 == h->c) return QSIM_OK;
    // a basis state is encoded afresh in the new tiles; any other state is
    // decoded into a dense buffer first
    const bool basis = h->basis;
    const unsigned long long bx = h->basis_x;
    double2 *d = nullptr;
    if (!basis) {
        if (h->n > 32) return fail(h, QSIM_ERR_ARG, "re-tiling needs n <= 32");
        size_t bytes = (size_t)16 << h->n;
        CK(cudaMalloc(&d, bytes));
        ++h->launches;
        cudaError_t e = qs::launch_amplitudes(h->arena[h->cur], h->table[h->cur], h->c, 0, 1ull << h->n, d,
                                              h->scal, grid_for(h, h->ntiles, 4), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { cudaFree(d); return fail(h, QSIM_ERR_CUDA, "re-tile: %s", cudaGetErrorString(e)); }
    }
    free_tiles(h);
    h->c = tile_log2;
    double theta = h->theta;
    int nlev = h->cc.nlev;
    int shifts[qs::MAX_LEVELS];
    std::memcpy(shifts, h->cc.shifts, sizeof shifts);
    int force = h->cc.force_raw;
    h->cc.c = h->c;
    h->cc.nlev = nlev;
    std::memcpy(h->cc.shifts, shifts, sizeof shifts);
    h->cc.force_raw = force;
    if (h->codec == QSIM_CODEC_AALC)
        h->cc.max_bytes = (unsigned long long)std::floor(16.0 * (double)(1ull << h->c) / theta);
    h->used = 0;
    if ((s = alloc_tiles(h)) != QSIM_OK) { if (d) cudaFree(d); return s; }
    s = basis ? encode_fresh(h, nullptr, bx) : encode_fresh(h, d, 0);
    if (d) cudaFree(d);
    return s;
}

qsim_status qsim_amplitudes(qsim_t h, unsigned long long start, unsigned long long count, double *out) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!out && count) return fail(h, QSIM_ERR_ARG, "out is NULL");
    if (start > (1ull << h->n) || count > (1ull << h->n) - start) return fail(h, QSIM_ERR_ARG, "range outside the state");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    const unsigned long long chunk = 1ull << 26;
    double2 *d = nullptr;
    unsigned long long first = std::min(count, chunk);
    if (count == 0) return QSIM_OK;
    CK(cudaMalloc(&d, first * 16));
    for (unsigned long long done = 0; done < count;) {
        unsigned long long cnt = std::min(chunk, count - done);
        unsigned long long tiles = ((start + done + cnt - 1) >> h->c) - ((start + done) >> h->c) + 1;
        ++h->launches;
        cudaError_t e = qs::launch_amplitudes(h->arena[h->cur], h->table[h->cur], h->c, start + done, cnt, d,
                                              h->scal, grid_for(h, tiles, 4), h->stream);
        if (e == cudaSuccess) e = hcopy(h, out + 2 * done, d, cnt * 16, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { cudaFree(d); return fail(h, QSIM_ERR_CUDA, "amplitudes: %s", cudaGetErrorString(e)); }
        done += cnt;
    }
    cudaFree(d);
    if ((s = read_scalars(h)) != QSIM_OK) return s;
    if (h->hscal->err) return device_error(h, h->hscal->err);
    return QSIM_OK;
}

qsim_status qsim_probabilities(qsim_t h, const int *qubits, int nq, double *out) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (nq < 0 || nq > 24 || nq > h->n || !out || (nq && !qubits)) return fail(h, QSIM_ERR_ARG, "nq must be 0..24 with valid buffers");
    unsigned long long used = 0;
    for (int i = 0; i < nq; ++i) {
        if (qubits[i] < 0 || qubits[i] >= h->n || ((used >> qubits[i]) & 1ull)) return fail(h, QSIM_ERR_ARG, "bad qubit list");
        used |= 1ull << qubits[i];
    }
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    const size_t nb = (size_t)1 << nq;
    if ((s = ensure_readout(h, nb * 16 + 32 * sizeof(int))) != QSIM_OK) return s;
    unsigned long long *dbk = static_cast<unsigned long long *>(h->rd);
    int *dq = reinterpret_cast<int *>(dbk + 2 * nb);
    std::vector<unsigned long long> hb(2 * nb);
    cudaError_t e = cudaMemsetAsync(dbk, 0, nb * 16, h->stream);
    if (e == cudaSuccess && nq) e = hcopy(h, dq, qubits, nq * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) ++h->launches, e = qs::launch_probs(h->arena[h->cur], h->table[h->cur], h->c, h->ntiles, dq, nq, dbk,
                                               h->scal, grid_for(h, h->ntiles, 4), h->stream);
    if (e == cudaSuccess) e = hcopy(h, hb.data(), dbk, nb * 16, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "probabilities: %s", cudaGetErrorString(e));
    unsigned __int128 tot = 0;
    for (size_t j = 0; j < nb; ++j) tot += ((unsigned __int128)hb[2 * j + 1] << 64) | hb[2 * j];
    double dt = units_to_double_host((unsigned long long)tot, (unsigned long long)(tot >> 64));
    for (size_t j = 0; j < nb; ++j) {
        double v = units_to_double_host(hb[2 * j], hb[2 * j + 1]);
        out[j] = dt > 0.0 ? v / dt : 0.0;
    }
    if ((s = read_scalars(h)) != QSIM_OK) return s;
    if (h->hscal->err) return device_error(h, h->hscal->err);
    return QSIM_OK;
}

qsim_status qsim_fidelity(qsim_t h, const qsim_ref *ref, double *F, double *overlap_abs) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!ref) return fail(h, QSIM_ERR_ARG, "ref is NULL");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    qs::RefSpec rs{};
    rs.kind = ref->kind;
    rs.n = h->n;
    double2 *tmp = nullptr;
    const unsigned long long N = 1ull << h->n;
    switch (ref->kind) {
        case QSIM_REF_HANDLE: {
            qsim_t o = ref->other;
            if (!o || o->n != h->n || o->c != h->c) return fail(h, QSIM_ERR_ARG, "reference handle needs the same n and tile size");
            if (o != h && (s = qsim_flush(o)) != QSIM_OK) return fail(h, s, "reference flush failed: %s", o->err.c_str());
            CK(cudaStreamSynchronize(o->stream));
            rs.kind = 0;
            rs.o_arena = o->arena[o->cur];
            rs.o_table = o->table[o->cur];
            break;
        }
        case QSIM_REF_QFT_BASIS:
            if (ref->x >= N) return fail(h, QSIM_ERR_ARG, "x out of range");
            rs.kind = 1;
            rs.x = ref->x;
            rs.qft_mag = 1.0 / std::sqrt((double)N);
            break;
        case QSIM_REF_GROVER: {
            if (ref->x >= N || ref->iterations < 0) return fail(h, QSIM_ERR_ARG, "bad Grover reference");
            rs.kind = 2;
            rs.x = ref->x;
            double th = std::asin(1.0 / std::sqrt((double)N));
            int k = ref->iterations;
            double sg = (k & 1) ? -1.0 : 1.0;
            rs.grov_m = sg * std::sin((2 * k + 1) * th);
            rs.grov_o = N > 1 ? sg * std::cos((2 * k + 1) * th) / std::sqrt((double)(N - 1)) : 0.0;
            break;
        }
        case QSIM_REF_DENSE_HOST:
            if (!ref->dense) return fail(h, QSIM_ERR_ARG, "dense is NULL");
            CK(cudaMalloc(&tmp, N * 16));
            CK(hcopy(h, tmp, ref->dense, N * 16, cudaMemcpyHostToDevice, h->stream));
            rs.kind = 3;
            rs.dense = tmp;
            break;
        case QSIM_REF_DENSE_DEVICE:
            if (!ref->dense) return fail(h, QSIM_ERR_ARG, "dense is NULL");
            rs.kind = 3;
            rs.dense = reinterpret_cast<const double2 *>(ref->dense);
            break;
        default:
            return fail(h, QSIM_ERR_ARG, "unknown reference kind");
    }
    const unsigned long long nchunks = h->ntiles / qs::fidelity_chunk(h->ntiles);
    if ((s = ensure_readout(h, (nchunks + nchunks / 2 + 1) * sizeof(qs::Acc4))) != QSIM_OK) {
        if (tmp) cudaFree(tmp);
        return s;
    }
    qs::Acc4 *a = static_cast<qs::Acc4 *>(h->rd), *b = a + nchunks;
    ++h->launches;
    cudaError_t e = qs::launch_fidelity(h->arena[h->cur], h->table[h->cur], h->c, h->ntiles, rs, a, h->scal,
                                        grid_for(h, nchunks, 4), h->stream);
    unsigned long long cnt = nchunks;
    while (e == cudaSuccess && cnt > 1) {
        ++h->launches, e = qs::launch_pair_sum(a, b, cnt / 2, grid_for(h, cnt / 2 / qs::THREADS + 1, 8), h->stream);
        std::swap(a, b);
        cnt /= 2;
    }
    qs::Acc4 r{};
    if (e == cudaSuccess) e = hcopy(h, &r, a, sizeof r, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "fidelity: %s", cudaGetErrorString(e));
    double f = (r.z > 0 && r.w > 0) ? (r.x * r.x + r.y * r.y) / (r.z * r.w) : 0.0;
    if (F) *F = f;
    if (overlap_abs) *overlap_abs = std::sqrt(f);
    if ((s = read_scalars(h)) != QSIM_OK) return s;
    if (h->hscal->err) return device_error(h, h->hscal->err);
    return QSIM_OK;
}

qsim_status qsim_compressed_bytes(qsim_t h, unsigned long long *stream_bytes, unsigned long long *footprint_bytes) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    unsigned long long tot = 0;
    if ((s = ensure_readout(h, sizeof(unsigned long long))) != QSIM_OK) return s;
    unsigned long long *d = static_cast<unsigned long long *>(h->rd);
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof *d, h->stream);
    if (e == cudaSuccess)
        ++h->launches, e = qs::launch_sum_sizes(h->arena[h->cur], h->table[h->cur], h->ntiles, d,
                                 grid_for(h, h->ntiles / qs::THREADS + 1, 8), h->stream);
    if (e == cudaSuccess) e = hcopy(h, &tot, d, sizeof tot, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "sizes: %s", cudaGetErrorString(e));
    if (stream_bytes) *stream_bytes = tot;
    if (footprint_bytes)
        *footprint_bytes = h->cap[0] + h->cap[1] + h->ntiles * 32ull + sizeof(qs::DevScalars);
    return QSIM_OK;
}

qsim_status qsim_stats(qsim_t h, qsim_stats_t *out) {
    if (!h || !out) return fail(h, QSIM_ERR_ARG, "null argument");
    if (!h->invalid) {
        qsim_status s = read_scalars(h);
        if (s != QSIM_OK) return s;
    }
    *out = h->st;
    for (int i = 0; i < 8; ++i) out->level_hist[i] = h->hscal->hist[i];
    out->kernel_launches = h->launches;
    out->items_done = h->hscal->items_done;
    out->items_skipped = h->hscal->items_skipped;
    out->alpha = h->hscal->alpha;
    out->tile_log2 = h->c;
    out->hmax = h->hmax;
    out->depth = h->depth;
    out->n_qubits = h->n;
    out->h2d_bytes = h->h2d_bytes;
    out->d2h_bytes = h->d2h_bytes;
    out->tiles_over_limit = h->hscal->over_limit;
    return QSIM_OK;
}

}  // extern "C"

namespace {

// Export of tiles first..first+count-1 (list null) or of the tiles in the
// host array list[0..count-1]: sizes, then (out not null) the streams.
qsim_status export_impl(qsim_t h, unsigned long long first, unsigned long long count,
                        const unsigned long long *list, void *out, unsigned long long cap,
                        unsigned long long *sizes) {
    unsigned long long *dsz = nullptr, *doff = nullptr, *dlist = nullptr;
    uint8_t *dbuf = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        if (dsz) cudaFree(dsz);
        if (doff) cudaFree(doff);
        if (dlist) cudaFree(dlist);
        if (dbuf) cudaFree(dbuf);
    };
    cudaError_t e = cudaMalloc(&dsz, count * 8);
    if (e == cudaSuccess && list) e = cudaMalloc(&dlist, count * 8);
    if (e == cudaSuccess && list)
        e = hcopy(h, dlist, list, count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        ++h->launches, e = qs::launch_sizes(h->arena[h->cur], h->table[h->cur], first, count, dlist, dsz,
                                            grid_for(h, count / qs::THREADS + 1, 8), h->stream);
    if (e == cudaSuccess) e = hcopy(h, sizes, dsz, count * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { cleanup(); return fail(h, QSIM_ERR_CUDA, "export sizes: %s", cudaGetErrorString(e)); }
    if (!out) { cleanup(); return QSIM_OK; }
    std::vector<unsigned long long> offs(count);
    unsigned long long tot = 0;
    for (unsigned long long i = 0; i < count; ++i) { offs[i] = tot; tot += sizes[i]; }
    if (tot > cap) { cleanup(); return fail(h, QSIM_ERR_ARG, "export needs %llu bytes", tot); }
    e = cudaMalloc(&doff, count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dbuf, tot);
    if (e == cudaSuccess) e = hcopy(h, doff, offs.data(), count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        ++h->launches, e = qs::launch_gather(h->arena[h->cur], h->table[h->cur], first, count, dlist, doff, dsz,
                                             dbuf, grid_for(h, count, 8), h->stream);
    if (e == cudaSuccess) e = hcopy(h, out, dbuf, tot, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cleanup();
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "export: %s", cudaGetErrorString(e));
    return QSIM_OK;
}

}  // namespace

extern "C" {

qsim_status qsim_export_tiles(qsim_t h, unsigned long long first, unsigned long long count, void *out,
                              unsigned long long cap, unsigned long long *sizes) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!sizes || first > h->ntiles || count > h->ntiles - first) return fail(h, QSIM_ERR_ARG, "bad tile range");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    if (count == 0) return QSIM_OK;
    return export_impl(h, first, count, nullptr, out, cap, sizes);
}

qsim_status qsim_export_tile_set(qsim_t h, const unsigned long long *tiles, unsigned long long count,
                                 void *out, unsigned long long cap, unsigned long long *sizes) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!sizes || (count && !tiles)) return fail(h, QSIM_ERR_ARG, "null argument");
    for (unsigned long long i = 0; i < count; ++i)
        if (tiles[i] >= h->ntiles) return fail(h, QSIM_ERR_ARG, "tile %llu out of range", tiles[i]);
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    if (count == 0) return QSIM_OK;
    return export_impl(h, 0, count, tiles, out, cap, sizes);
}

qsim_status qsim_import_tiles(qsim_t h, unsigned long long first, unsigned long long count, const void *data,
                              const unsigned long long *sizes) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!data || !sizes || first > h->ntiles || count > h->ntiles - first) return fail(h, QSIM_ERR_ARG, "bad tile range");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    h->basis = false;
    if (count == 0) return QSIM_OK;
    std::vector<unsigned long long> offs(count);
    unsigned long long tot = 0;
    for (unsigned long long i = 0; i < count; ++i) {
        if (sizes[i] < (unsigned long long)qs::HDR || (sizes[i] & 15ull) || sizes[i] > tile_bytes_worst(h))
            return fail(h, QSIM_ERR_FORMAT, "tile %llu: bad stream size %llu", first + i, sizes[i]);
        offs[i] = tot;
        tot += sizes[i];
    }
    uint8_t *dbuf = nullptr;
    unsigned long long *doff = nullptr, *dsz = nullptr, *dparts = nullptr;
    unsigned int *dbad = nullptr, hbad = 0;
    CK(cudaMalloc(&dbuf, tot));
    cudaError_t e = cudaMalloc(&doff, count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dsz, count * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dparts, count * 16);
    if (e == cudaSuccess) e = cudaMalloc(&dbad, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(dbad, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = hcopy(h, dbuf, data, tot, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = hcopy(h, doff, offs.data(), count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = hcopy(h, dsz, sizes, count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) ++h->launches, e = qs::launch_validate(dbuf, doff, dsz, count, h->c, dparts, dbad, grid_for(h, count, 4), h->stream);
    if (e == cudaSuccess) e = hcopy(h, &hbad, dbad, sizeof hbad, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        if (dbuf) cudaFree(dbuf);
        if (doff) cudaFree(doff);
        if (dsz) cudaFree(dsz);
        if (dparts) cudaFree(dparts);
        if (dbad) cudaFree(dbad);
    };
    if (e != cudaSuccess) { cleanup(); return fail(h, QSIM_ERR_CUDA, "import: %s", cudaGetErrorString(e)); }
    if (hbad) { cleanup(); return fail(h, QSIM_ERR_FORMAT, "%u imported stream(s) failed to decode", hbad); }
    // append after the live bytes of the current arena (grow by copying)
    unsigned long long need = h->used + tot;
    if (h->cap[h->cur] < need) {
        uint8_t *na = nullptr;
        unsigned long long nc = round_up(need + need / 4, 1ull << 21);
        e = cudaMalloc(&na, nc);
        if (e == cudaSuccess && h->used) e = hcopy(h, na, h->arena[h->cur], h->used, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { if (na) cudaFree(na); cleanup(); return fail(h, QSIM_ERR_OOM, "import: %s", cudaGetErrorString(e)); }
        cudaFree(h->arena[h->cur]);
        h->arena[h->cur] = na;
        h->cap[h->cur] = nc;
    }
    ++h->launches, e = qs::launch_place(dbuf, doff, dsz, count, first, h->used, h->arena[h->cur], h->table[h->cur], dparts, h->part,
                         grid_for(h, count, 8), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&h->scal->acc_lo, 0, 2 * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) ++h->launches, e = qs::launch_norm_from_parts(h->part, h->ntiles, h->scal, grid_for(h, h->ntiles / qs::THREADS + 1, 4), h->stream);
    if (e == cudaSuccess) ++h->launches, e = qs::launch_finalize(h->scal, h->normalize, nullptr, 0, 0, h->stream);
    cleanup();
    if (e != cudaSuccess) return fail(h, QSIM_ERR_CUDA, "import: %s", cudaGetErrorString(e));
    h->used += tot;
    return read_scalars(h);
}

// ------------------------------------------------------------ checkpoints
namespace {
const char CKPT_MAGIC[8] = {'Q', 'S', 'I', 'M', 'C', 'K', 'P', '1'};
constexpr unsigned long long CKPT_CHUNK = 1ull << 20;      // tiles per chunk

struct CkptHeader {
    char magic[8];
    uint32_t version, n, c, hmax, depth, codec, normalize, nlev;
    int32_t shifts[8];
    double eps, theta;
    unsigned long long max_bytes, ntiles, stream_bytes;
    int32_t unit_log2, reserved;
};
static_assert(sizeof(CkptHeader) == 120, "checkpoint header layout");

struct FileCloser {
    FILE *f;
    ~FileCloser() { if (f) fclose(f); }
};
}  // namespace

qsim_status qsim_save(qsim_t h, const char *path) {
    qsim_status s = check_usable(h);
    if (s != QSIM_OK) return s;
    if (!path) return fail(h, QSIM_ERR_ARG, "null path");
    if ((s = qsim_flush(h)) != QSIM_OK) return s;
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) return fail(h, QSIM_ERR_ARG, "cannot open %s for writing", path);
    CkptHeader hd{};
    std::memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.version = 2;
    hd.n = (uint32_t)h->n;
    hd.c = (uint32_t)h->c;
    hd.hmax = (uint32_t)h->hmax;
    hd.depth = (uint32_t)h->depth;
    hd.codec = (uint32_t)h->codec;
    hd.normalize = (uint32_t)h->normalize;
    hd.nlev = (uint32_t)h->cc.nlev;
    for (int i = 0; i < 8; ++i) hd.shifts[i] = h->cc.shifts[i];
    hd.eps = h->eps;
    hd.theta = h->theta;
    hd.max_bytes = h->cc.max_bytes;
    hd.ntiles = h->ntiles;
    hd.stream_bytes = h->used;
    hd.unit_log2 = h->unit_log2;
    hd.reserved = (h->polar ? 1 : 0) | (h->fuse ? 0 : 2);      // flags: POLAR mode, gate by gate
    if (fwrite(&hd, sizeof hd, 1, fc.f) != 1) return fail(h, QSIM_ERR_ARG, "write failed: %s", path);
    std::vector<unsigned long long> sizes;
    std::vector<uint8_t> buf;
    for (unsigned long long first = 0; first < h->ntiles; first += CKPT_CHUNK) {
        const unsigned long long cnt = std::min(CKPT_CHUNK, h->ntiles - first);
        sizes.resize(cnt);
        if ((s = qsim_export_tiles(h, first, cnt, nullptr, 0, sizes.data())) != QSIM_OK) return s;
        unsigned long long tot = 0;
        for (unsigned long long v : sizes) tot += v;
        buf.resize(tot);
        if ((s = qsim_export_tiles(h, first, cnt, buf.data(), tot, sizes.data())) != QSIM_OK) return s;
        if (fwrite(sizes.data(), 8, cnt, fc.f) != cnt || fwrite(buf.data(), 1, tot, fc.f) != tot)
            return fail(h, QSIM_ERR_ARG, "write failed: %s", path);
    }
    return QSIM_OK;
}

qsim_status qsim_load(qsim_t *out, const char *path) {
    if (!out || !path) return fail(nullptr, QSIM_ERR_ARG, "null argument");
    *out = nullptr;
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) return fail(nullptr, QSIM_ERR_ARG, "cannot open %s", path);
    CkptHeader hd{};
    if (fread(&hd, sizeof hd, 1, fc.f) != 1 || std::memcmp(hd.magic, CKPT_MAGIC, 8) != 0 || hd.version != 2)
        return fail(nullptr, QSIM_ERR_FORMAT, "%s is not a checkpoint of this library", path);
    if (hd.n < 1 || hd.n > (uint32_t)MAX_QUBITS || hd.c < 1 || hd.c > (uint32_t)qs::MAX_C || hd.c > hd.n ||
        hd.codec > QSIM_CODEC_AALC || hd.nlev < 1 || hd.nlev > (uint32_t)qs::MAX_LEVELS ||
        hd.ntiles != (1ull << (hd.n - hd.c)) || hd.unit_log2 < 0 || hd.unit_log2 > MAX_QUBITS)
        return fail(nullptr, QSIM_ERR_FORMAT, "%s: inconsistent checkpoint header", path);
    for (uint32_t i = 0; i < hd.nlev; ++i)
        if (hd.shifts[i] < 0 || hd.shifts[i] > 52) return fail(nullptr, QSIM_ERR_FORMAT, "%s: bad shift", path);
    qsim_t h = nullptr;
    qsim_status s = qsim_create(&h, (int)hd.n, (int)hd.c, (qsim_codec)hd.codec, hd.eps);
    if (s != QSIM_OK) return s;
    auto bail = [&](qsim_status code) { qsim_destroy(h); return code; };
    if (hd.hmax < 1 || hd.hmax > (uint32_t)qs::MAX_PAIRS || hd.c + hd.hmax > (uint32_t)qs::MAX_ITEM_LOG2 ||
        hd.depth < 1 || hd.depth > (uint32_t)qs::MAX_SWEEP_GATES) {
        g_last_error = "checkpoint schedule out of range";
        return bail(QSIM_ERR_FORMAT);
    }
    if (h->c != (int)hd.c) {                 // tiles of the saved size (the new state is still |0>)
        free_tiles(h);
        h->c = (int)hd.c;
        h->cc.c = h->c;
        h->used = 0;
        if ((s = alloc_tiles(h)) != QSIM_OK || (s = encode_fresh(h, nullptr, 0)) != QSIM_OK) {
            g_last_error = h->err;
            return bail(s);
        }
    }
    h->hmax = (int)hd.hmax;
    h->depth = (int)hd.depth;
    h->theta = hd.theta;
    h->normalize = (int)hd.normalize;
    h->cc.nlev = (int)hd.nlev;
    for (int i = 0; i < qs::MAX_LEVELS; ++i) h->cc.shifts[i] = i < (int)hd.nlev ? hd.shifts[i] : 0;
    h->cc.max_bytes = hd.max_bytes;
    h->unit_log2 = hd.unit_log2;
    if (hd.reserved & ~3) { g_last_error = "unknown checkpoint flags"; return bail(QSIM_ERR_FORMAT); }
    h->polar = hd.reserved & 1;
    h->cc.polar = h->polar;
    h->fuse = (hd.reserved & 2) ? 0 : 1;
    std::vector<unsigned long long> sizes;
    std::vector<uint8_t> buf;
    for (unsigned long long first = 0; first < h->ntiles; first += CKPT_CHUNK) {
        const unsigned long long cnt = std::min(CKPT_CHUNK, h->ntiles - first);
        sizes.resize(cnt);
        if (fread(sizes.data(), 8, cnt, fc.f) != cnt) {
            g_last_error = "truncated checkpoint";
            return bail(QSIM_ERR_FORMAT);
        }
        unsigned long long tot = 0;
        for (unsigned long long v : sizes) {
            if (v > tile_bytes_worst(h)) { g_last_error = "bad stream size in checkpoint"; return bail(QSIM_ERR_FORMAT); }
            tot += v;
        }
        buf.resize(tot);
        if (fread(buf.data(), 1, tot, fc.f) != tot) {
            g_last_error = "truncated checkpoint";
            return bail(QSIM_ERR_FORMAT);
        }
        if ((s = qsim_import_tiles(h, first, cnt, buf.data(), sizes.data())) != QSIM_OK) {
            g_last_error = h->err;
            return bail(s);
        }
    }
    h->st = qsim_stats_t{};
    h->st.stream_bytes = h->used;
    h->st.min_stream_bytes_seen = h->st.max_stream_bytes_seen = h->used;
    *out = h;
    return QSIM_OK;
}

int qsim_plan_sweeps(int n, int tile_log2, int hmax, int depth, int ngates, const int *ntargets,
                     const int *targets, const double *matrices, int *out_lo, int *out_h, int *out_H,
                     int cap) {
    if (n < 1 || n > MAX_QUBITS || tile_log2 < 1 || tile_log2 > n || hmax < 1 || hmax > qs::MAX_PAIRS || depth < 1 ||
        ngates < 0 || (ngates && (!ntargets || !targets || !matrices)))
        return -1;
    std::vector<HostGate> g(ngates);
    for (int i = 0; i < ngates; ++i) {
        if (ntargets[i] < 1 || ntargets[i] > 2) return -1;
        g[i].k = ntargets[i];
        for (int j = 0; j < g[i].k; ++j) {
            g[i].t[j] = targets[2 * i + j];
            if (g[i].t[j] < 0 || g[i].t[j] >= n) return -1;
        }
        std::memcpy(g[i].m, matrices + 32 * i, sizeof g[i].m);
        g[i].diag = matrix_is_diagonal(g[i].k, g[i].m);
    }
    std::vector<Sweep> sw;
    if (plan_sweeps(n, tile_log2, hmax, depth, g, sw) < 0) return -1;
    if ((int)sw.size() > cap) return -2;
    for (size_t i = 0; i < sw.size(); ++i) {
        if (out_lo) out_lo[i] = sw[i].lo;
        if (out_h) out_h[i] = sw[i].h;
        if (out_H)
            for (int j = 0; j < 4; ++j) out_H[4 * i + j] = sw[i].H[j];
    }
    return (int)sw.size();
}

}  // extern "C"
