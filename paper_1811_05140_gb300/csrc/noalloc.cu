// qsim_encode_noalloc: tile encoding for callers that cannot allocate
// device memory.  The encode kernel's scratch (pass counters, error word,
// per-tile norm partials) lives in one file-scope static device array
// instead of memory obtained from cudaMalloc; the caller passes the input
// state and the output buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "qsim.h"
#include "qsim_dev.cuh"

namespace qs {
cudaError_t launch_init(const double2 *dense, unsigned long long x, const CodecCfg &cc,
                        unsigned long long ntiles, uint8_t *arena, unsigned long long cap,
                        unsigned long long *table, unsigned long long *part, DevScalars *scal,
                        unsigned long long *unit_bytes, const uint8_t *unit_level, int unit_shift,
                        int grid, cudaStream_t st);
cudaError_t configure_kernels();
void set_global_error(const char *msg);
}  // namespace qs

namespace {

// Largest state the static scratch serves: 4096 tiles.
constexpr unsigned long long NOALLOC_MAX_TILES = 4096;

struct NoallocScratch {
    qs::DevScalars scal;
    unsigned long long part[2 * NOALLOC_MAX_TILES];
};

constexpr int MAX_DEVICES = 64;
// Device address of the array and the set-up result, per device; each
// device's set-up runs exactly once even when host threads race on the
// first call (std::call_once).
NoallocScratch *g_scratch_addr[MAX_DEVICES];
cudaError_t g_setup_err[MAX_DEVICES];
std::once_flag g_setup_once[MAX_DEVICES];

qsim_status noalloc_fail(qsim_status code, const char *fmt, unsigned long long a = 0,
                         unsigned long long b = 0) {
    char buf[256];
    snprintf(buf, sizeof buf, fmt, a, b);
    qs::set_global_error(buf);
    return code;
}

int shift_for_bound(double eps) {
    for (int s = 52; s >= 1; --s)
        if (std::ldexp(1.0, s - 53) <= eps) return s;
    return 0;
}

}  // namespace

// Every GPU that loads the library holds this array (about 64 KiB) until
// the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

extern "C" qsim_status qsim_encode_noalloc(const double *dev_amps, int n_qubits, int tile_log2,
                                           double rel_err_bound, void *dev_out,
                                           unsigned long long out_cap,
                                           unsigned long long *dev_table,
                                           unsigned long long *stream_bytes, void *cuda_stream) {
    if (n_qubits < 1 || n_qubits > 40 || tile_log2 < 1 || tile_log2 > qs::MAX_C || tile_log2 > n_qubits)
        return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: need 1 <= tile_log2 <= min(10, n_qubits) <= 40");
    const unsigned long long ntiles = 1ull << (n_qubits - tile_log2);
    if (ntiles > NOALLOC_MAX_TILES)
        return noalloc_fail(QSIM_ERR_ARG,
                            "qsim_encode_noalloc: %llu tiles exceed the static scratch limit of %llu "
                            "tiles (need n_qubits - tile_log2 <= 12)",
                            ntiles, NOALLOC_MAX_TILES);
    if (!(rel_err_bound >= 0.0 && rel_err_bound < 1.0))
        return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: rel_err_bound must be in [0, 1)");
    if (!dev_amps || !dev_out || !dev_table || !stream_bytes)
        return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: NULL pointer argument");
    if (((unsigned long long)dev_out & 15ull) || ((unsigned long long)dev_amps & 15ull))
        return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: dev_out and dev_amps must be 16-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return noalloc_fail(QSIM_ERR_CUDA, "qsim_encode_noalloc: no usable CUDA device");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (st) {
        // the scratch address and the SM count below are the current device's
        int sdev = -1;
        if (cudaStreamGetDevice(st, &sdev) != cudaSuccess || sdev != dev)
            return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: cuda_stream must belong to the current device");
    }
    // first call on this device: kernel attributes and the array's device address
    std::call_once(g_setup_once[dev], [dev] {
        cudaError_t e = qs::configure_kernels();
        void *ptr = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e == cudaSuccess && !ptr) e = cudaErrorInvalidSymbol;
        if (e == cudaSuccess) g_scratch_addr[dev] = static_cast<NoallocScratch *>(ptr);
        g_setup_err[dev] = e;
    });
    if (g_setup_err[dev] != cudaSuccess)
        return noalloc_fail(QSIM_ERR_CUDA, "qsim_encode_noalloc: set-up (kernel attributes, scratch address) failed");
    NoallocScratch *scr = g_scratch_addr[dev];
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    qs::CodecCfg cc{};
    cc.c = tile_log2;
    cc.nlev = 1;
    cc.shifts[0] = shift_for_bound(rel_err_bound);
    cc.max_bytes = ~0ull;
    cc.force_raw = 0;

    // counters, error word and running norm start at zero on every call;
    // the per-tile partials are written for every tile by the kernel
    cudaError_t e = cudaMemsetAsync(&scr->scal, 0, sizeof(qs::DevScalars), st);
    unsigned long long grid = (unsigned long long)sms * 4ull;
    if (grid > ntiles) grid = ntiles;
    if (e == cudaSuccess)
        e = qs::launch_init(reinterpret_cast<const double2 *>(dev_amps), 0ull, cc, ntiles,
                            static_cast<uint8_t *>(dev_out), out_cap, dev_table, scr->part,
                            &scr->scal, nullptr, nullptr, 0, (int)grid, st);
    unsigned long long bump = 0;
    unsigned int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bump, &scr->scal.bump, sizeof bump, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &scr->scal.err, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(QSIM_ERR_CUDA, "qsim_encode_noalloc: CUDA error during the encode");
    *stream_bytes = bump;
    if (err & qs::ERR_OVERFLOW)
        return noalloc_fail(QSIM_ERR_ARG, "qsim_encode_noalloc: out_cap %llu is too small, %llu bytes needed",
                            out_cap, bump);
    if (err & (qs::ERR_NONFINITE | qs::ERR_RANGE))
        return noalloc_fail(QSIM_ERR_NONFINITE, "qsim_encode_noalloc: non-finite or out-of-range amplitude");
    return QSIM_OK;
}
