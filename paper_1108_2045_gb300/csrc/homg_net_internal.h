// Private interface between the learned corrector (homg_net.cu) and the solver's host code
// (homg_api.cu): network inference on device buffers and the kernels that turn a solver residual
// into network features and a network output into a proposed correction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct homg_net;

namespace homg {

// y = network(x) for B images of H x W (layouts of include/homg_net.h); enqueues on s, no sync.
// Returns a HOMG_* code (device timeouts are reported by net_check_error after a sync).
int net_forward_dev(homg_net* net, const void* x, int B, int H, int W, float* y, cudaStream_t s);
// HOMG_OK, or HOMG_ECUDA when a network kernel gave up waiting on its tensor-core barrier.
int net_check_error(homg_net* net);

// Blocks of partial sums written by launch_feat_stats for an n-interval grid.
int feat_parts(int n);
// Partial sums of (g0 / D)^2 over the interior nodes; g0 = h^2 r in the cycle's storage type
// `prec` (rows of pitch_g), D from the FP64 level-0 face coefficients kx0, ky0 (rows of kpitch).
cudaError_t launch_feat_stats(int prec, const void* g0, int64_t pitch_g, const double* kx0, const double* ky0,
                              int64_t kpitch, int n, double* part, cudaStream_t s);
// *out = sqrt(sum(part[0..nparts)) / count) (fixed summation order), or the plain sum when count == 0.
cudaError_t launch_reduce(const double* part, int nparts, double count, double* out, cudaStream_t s);
// x (one image of (n+1)^2 pixels, 16 channels): channel 0 = bf16(g0 / D / rho) at interior nodes,
// channel 1 = logk, the rest 0.
cudaError_t launch_feat_write(int prec, const void* g0, int64_t pitch_g, const double* kx0, const double* ky0,
                              int64_t kpitch, int n, const double* rho, const uint16_t* logk, void* x, cudaStream_t s);
// t = (uref - u) / rho at interior nodes, 0 on the boundary (unpadded (n+1)^2 arrays).
cudaError_t launch_target(const double* uref, const double* u, int n, const double* rho, float* t, cudaStream_t s);
// e = rho * y at interior nodes, 0 on the boundary, in the cycle's storage type (rows of pitch).
cudaError_t launch_correct(int prec, const float* y, int n, const double* rho, void* e, int64_t pitch, cudaStream_t s);
// out = bf16(log k) for the (n+1)^2 node coefficients.
cudaError_t launch_logk(const double* k, int n, uint16_t* out, cudaStream_t s);

}  // namespace homg
