// homg_fp64_issue_probe: the FP64 instruction rate of the GPU, measured by a kernel that does
// nothing but independent chains of FP64 fused multiply-adds (or additions).
//
// On GB300 the FP64 pipe, not DRAM, bounds every FP64 stencil kernel of this library: a level-0
// damped-Jacobi sweep issues five FP64 instructions (three additions, two fused multiply-adds) per
// 24 bytes of traffic. The roofline of those kernels therefore needs the pipe's own ceiling, taken
// on the same GPU, with the same clocks, as the kernels it judges.
#include "../../include/homg.h"
#include "homg_internal.h"

namespace {

constexpr int kChains = 8;     // independent dependency chains per thread (hides the pipe latency)
constexpr int kThreads = HOMG_PROBE_THREADS;

// Every thread runs kChains chains of `iters` steps; a step is x <- x * a + b (op 0) or x <- x + b
// (op 1), one FP64 instruction. a and b are kernel arguments, so nothing folds at compile time, and
// each thread stores the sum of its chains so that no chain is dead code.
template <int OP>
__global__ void __launch_bounds__(kThreads) k_fp64_issue(double a, double b, int iters, double* sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1.0e-3 * (double)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = OP == 0 ? fma(x[c], a, b) : x[c] + b;
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[(int64_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int homg_fp64_issue_probe(int op, int blocks, int iters, double* sink, void* stream,
                                     double* instructions_out) {
    if ((op != 0 && op != 1) || blocks < 1 || iters < 1 || !sink || !instructions_out) {
        homg::set_null_handle_error("homg_fp64_issue_probe: op must be 0 or 1, blocks and iters >= 1, pointers non-null");
        return HOMG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // a slightly below 1 keeps the multiply-add chains bounded; b is small and positive
    if (op == 0) k_fp64_issue<0><<<blocks, kThreads, 0, s>>>(0.9999999, 1.0e-7, iters, sink);
    else k_fp64_issue<1><<<blocks, kThreads, 0, s>>>(0.0, 1.0e-7, iters, sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        homg::set_null_handle_error(cudaGetErrorString(e));
        return HOMG_ECUDA;
    }
    *instructions_out = (double)blocks * kThreads * (double)iters * kChains;
    return HOMG_OK;
}
