// homg_residual_norm_noalloc: the relative residual ||f - A u|| / ||f|| of device arrays without a
// handle and without allocating anything.
//
// Some callers cannot call cudaMalloc: cudaMalloc synchronises the whole device, which a caller in
// a latency-critical loop cannot afford, and it fails outright when another allocator (for example
// a framework's caching allocator) already holds the device memory. Creating a handle allocates the
// full multigrid level buffer, so such callers use this entry point to check a solution instead.
// It runs the same residual and reduction kernels as homg_residual_norm, but their scratch (one
// partial sum per thread block, and the small state block the kernels read their arguments from)
// lives in the file-scope array below, which every GPU that loads this library holds until the
// process exits.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/homg.h"
#include "homg_internal.h"

using namespace homg;

namespace {

// State block at the head of the array, rounded up to 32 doubles; then the r^2 and f^2 partials.
constexpr int kStateDoubles = 32;
static_assert(sizeof(State) <= kStateDoubles * sizeof(double), "State must fit its slot");
constexpr int kScratchDoubles = kStateDoubles + 2 * HOMG_NOALLOC_MAX_BLOCKS;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_scratch last looked up, per device ordinal

int fail(int code, const char* msg) {
    set_null_handle_error(msg);
    return code;
}

// Device address of g_scratch on the current device. A call made outside stream capture looks it
// up again every time: after cudaDeviceReset (or any other end of the device's context) the
// library's module is loaded anew and the array may sit at another address. A call made while `s`
// is capturing, or whose capture status cannot be read, reuses the address that the last call
// outside capture found on this device, and looks it up only if there is none yet.
cudaError_t scratch_address(int dev, cudaStream_t s, double** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool known = cudaStreamIsCapturing(s, &cs) == cudaSuccess;
    if (!known) cudaGetLastError();
    if (!g_scratch_addr[dev] || (known && cs == cudaStreamCaptureStatusNone)) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (double*)p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int homg_residual_norm_noalloc(int ndim, const int64_t* dims, const double* f, const double* u,
                                          double* relres_out, void* stream) {
    char msg[256];
    if (!dims || !f || !u || !relres_out) return fail(HOMG_EINVAL, "homg_residual_norm_noalloc: null argument");
    if (ndim != 2 && ndim != 3) return fail(HOMG_EINVAL, "homg_residual_norm_noalloc: ndim must be 2 or 3");
    for (int d = 1; d < ndim; ++d)
        if (dims[d] != dims[0]) return fail(HOMG_ESHAPE, "homg_residual_norm_noalloc: grid sides must be equal");
    const int64_t n = dims[0] - 1;
    int K = 0;
    while (K < 62 && ((int64_t)1 << K) < n) ++K;
    if (n < 2 || ((int64_t)1 << K) != n)
        return fail(HOMG_ESHAPE, "homg_residual_norm_noalloc: grid side must be 2^K + 1 with K >= 1");
    if (K > (ndim == 2 ? HOMG_MAX_K_2D : HOMG_MAX_K_3D))
        return fail(HOMG_ESHAPE, "homg_residual_norm_noalloc: grid side above the supported maximum");
    const int nblocks = residual_blocks(ndim, false, (int)n);
    if (nblocks > HOMG_NOALLOC_MAX_BLOCKS) {
        snprintf(msg, sizeof(msg),
                 "homg_residual_norm_noalloc: this grid needs %d partial sums, the static scratch holds %d "
                 "(2-D grids up to 8193^2, 3-D grids up to 513^3)",
                 nblocks, HOMG_NOALLOC_MAX_BLOCKS);
        return fail(HOMG_ESHAPE, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(HOMG_ECUDA, "homg_residual_norm_noalloc: no usable current device");
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = nullptr;
    e = scratch_address(dev, s, &scratch);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "homg_residual_norm_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return fail(HOMG_ECUDA, msg);
    }
    State* st = (State*)scratch;
    // The arguments block is rewritten on every call; each partial slot the reduction reads is
    // written by its block first, so nothing left by an earlier call is read.
    State hs;
    memset(&hs, 0, sizeof(hs));
    hs.f = f;
    hs.u = (double*)u;
    e = cudaMemcpyAsync(st, &hs, sizeof(State), cudaMemcpyHostToDevice, s);
    ResidArgs a{};
    a.st = st;
    a.inv_h2 = (double)n * (double)n;
    a.part_r = scratch + kStateDoubles;
    a.part_f = scratch + kStateDoubles + HOMG_NOALLOC_MAX_BLOCKS;
    if (e == cudaSuccess) e = launch_residual(ndim, PREC_FP64, false, a, (int)n, s);
    FinalizeArgs fa{};
    fa.st = st;
    fa.part_r = a.part_r;
    fa.part_f = a.part_f;
    fa.nparts = nblocks;
    fa.mode = FIN_NORM;
    if (e == cudaSuccess) e = launch_finalize(fa, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(State), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof(msg), "homg_residual_norm_noalloc: CUDA error: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return fail(HOMG_ECUDA, msg);
    }
    *relres_out = hs.relres;
    return HOMG_OK;
}
