/*
 * Learned corrector for the HOMG restart loop -- C ABI.
 *
 * The paper has no learned component: this is an extension. A small convolutional network maps
 * the residual of the current iterate (and log k) to a proposed correction; the plain solver
 * judges every proposal with its FP64 residual and keeps it only when the residual norm drops,
 * then runs the ordinary HOMG cycle (Sec. 2 and the restart of Sec. 4) on the result. The
 * network runs on the tcgen05 tensor cores in bfloat16 with binary32 accumulation; it is trained
 * by this library's own kernels on error/residual pairs that the solver itself produces.
 *
 * Network (fixed): four 3x3 convolutions, zero padding, 2 -> 32 -> 32 -> 32 -> 1 channels, ReLU
 * after the first three. Parameters are binary32 ("master"), flat, per layer l = 0..3 the weights
 * W_l[out][in][3][3] (row-major) followed by the biases b_l[out]; homg_net_param_count() values.
 * Weights are rounded to bfloat16 for every use; hidden activations are stored in bfloat16.
 *
 * Image layout (device, bfloat16 bit patterns as uint16): B images of H x W pixels with 16
 * channels in two groups of 8, element (b, c, y, x) at ((b*H + y)*2 + c/8)*W*8 + x*8 + c%8.
 * Channel 0 = x_0, channel 1 = x_1, channels 2..15 must be 0. Outputs and targets: binary32,
 * [B][H][W].
 *
 * Features of a solver grid (homg_features): x_0(p) = h^2 r(p) / (D(p) rho) at interior nodes
 * (0 on the boundary), x_1(p) = log k(p), with r = f - A u (FP64), D(p) the sum of the node's four
 * face coefficients and rho the root mean square of h^2 r / D over the interior. The network's
 * output y is a correction in units of rho: u <- u + rho y.
 *
 * Return codes are those of homg.h. Every call synchronises the handle's stream unless stated.
 */
#ifndef HOMG_NET_H
#define HOMG_NET_H

#include <stdint.h>

#include "homg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct homg_net* homg_net_handle;

#define HOMG_NET_LAYERS 4
#define HOMG_NET_WIDTH 32
#define HOMG_NET_IN 2

/* Number of binary32 parameters of the network (weights and biases of the four layers). */
int64_t homg_net_param_count(void);

/* Create a network on the current device with all parameters 0 and fresh Adam state. Device
 * scratch for activations is allocated by later calls as image sizes require. */
int homg_net_create(homg_net_handle* out);

/* Use `stream` (a cudaStream_t, NULL = legacy default stream) for every later call on net. */
int homg_net_set_stream(homg_net_handle net, void* stream);

/* Copy `count` (= homg_net_param_count()) host binary32 parameters in / out. Setting parameters
 * resets the Adam state and the step counter. HOMG_EINVAL for a wrong count or null pointer. */
int homg_net_set_params(homg_net_handle net, const float* params, int64_t count);
int homg_net_get_params(homg_net_handle net, float* params, int64_t count);

/* Copy the parameter gradients of the last homg_net_train_step (same order and count as the
 * parameters; binary32) to the host. */
int homg_net_get_grads(homg_net_handle net, float* grads, int64_t count);

/* Inference: y[b][y][x] = network(x) for B device images (layout above) of H x W pixels.
 * B, H, W >= 1 and B*H*W < 2^31. */
int homg_net_forward(homg_net_handle net, const void* x, int B, int H, int W, float* y);

/* Training loss of homg_net_train_step.
 * HOMG_NET_LOSS_ERROR (default): mean squared error (1/N) sum (y - t)^2 over the N = B*H*W pixels,
 *   t the scaled true error of the iterate (homg_features).
 * HOMG_NET_LOSS_RESIDUAL: the residual the proposal leaves, (1/N) sum res^2 over the
 *   N = B*(H-2)*(W-2) inner pixels of the patches, res(p) = x_0(p) - (y(p) - sum_q w_q(p) y(q)),
 *   w_q(p) = k_pq / D(p) for the four neighbours q (column -1, +1, row -1, +1) with k = exp(x_1)
 *   taken from the patch's own log k channel, k_pq the harmonic mean at p and q, D(p) the sum of
 *   the four: the scaled residual of u + rho y, computed on the patch. t is not used (may be NULL).
 * The learned-corrector extension has no counterpart in the paper; the residual loss trains the
 * network toward corrections the solver's judge measures. HOMG_EINVAL for another kind. */
#define HOMG_NET_LOSS_ERROR 0
#define HOMG_NET_LOSS_RESIDUAL 1
int homg_net_set_loss(homg_net_handle net, int kind);

/* One training step on a batch: forward, the loss selected by homg_net_set_loss (mean squared error
 * against t ([B][H][W] device) by default), the gradient of every parameter (binary32
 * accumulation), one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr > 0.
 * *loss_out (optional) receives the batch loss before the step. The residual loss needs H, W >= 3. */
int homg_net_train_step(homg_net_handle net, const void* x, const float* t, int B, int H, int W, float lr,
                        float* loss_out);

/* Gather B square P x P patches from one device image x (H x W, layout above) and its target t
 * ([H][W]); corners (device int32, 2 per patch: row, column of the patch's first pixel) must
 * keep every patch inside the image (HOMG_EINVAL is not detected on the device: the caller owns
 * this). Writes xp ([B] images of P x P) and tp ([B][P][P]). Does not synchronise. */
int homg_net_gather_patches(homg_net_handle net, const void* x, const float* t, int H, int W, const int32_t* corners,
                            int B, int P, void* xp, float* tp);

/* Output rows per convolution tile (4 or 8, default 4; HOMG_EINVAL otherwise). A tile's
 * accumulators take rows x 32 TMEM columns and its staged input rows + 2 band rows of shared
 * memory; taller tiles make wider tensor-core instructions (a slice of up to three vertical taps
 * per instruction, see homg_net.cu) and fewer of them per output row. Results do not depend on it.
 * A tuning option of this library's network; the paper has no counterpart. */
int homg_net_set_tile_rows(homg_net_handle net, int rows);

/* Self-test of the failure path: launches one convolution whose tensor-core completion barrier
 * is never signalled (no MMA is issued). Every wait on such a barrier gives up after 0.5 s, records
 * the failure and frees the block's tensor memory, so the call returns HOMG_ECUDA with a timeout
 * message, *waited_ms holding the kernel's duration, and the context stays usable (the next call
 * on net works). HOMG_OK here would mean the wait is not bounded as documented. */
int homg_net_check_barrier_timeout(homg_net_handle net, double* waited_ms);

/* Message of the last hard error on net (or of the last failed homg_net_create when net is NULL). */
const char* homg_net_last_error(homg_net_handle net);

void homg_net_destroy(homg_net_handle net);

/* Network features of the grid iterate u for right-hand side f on a handle with variable
 * coefficients (homg_set_coefficient): x_out (one image of (n+1) x (n+1) pixels, layout above)
 * and *rho_out; when u_ref is given, t_out[(n+1)^2] receives the scaled error (u_ref - u) / rho
 * at interior nodes (0 on the boundary). f, u, u_ref: FP64 device arrays, unpadded (n+1)^2.
 * HOMG_EINVAL when the handle has no coefficient or rho = 0. */
int homg_features(homg_handle h, const double* f, const double* u, const double* u_ref, void* x_out, float* t_out,
                  double* rho_out);

/* How homg_solve_learned judges a proposal u' = u + rho y (the plain solver always decides, in FP64
 * residual norms computed by the same reduction):
 * HOMG_JUDGE_PROPOSAL (default): keep u' when ||f - A u'|| < ||f - A u||, then one HOMG cycle on the
 *   kept iterate's residual.
 * HOMG_JUDGE_AFTER_CYCLE: run one HOMG cycle from u and one from u' and keep the result whose
 *   residual is smaller (a proposal whose rough part the cycle removes can win here although its own
 *   residual is larger); two cycles per proposal.
 * The setting belongs to the handle h and applies to its later learned solves. HOMG_EINVAL for
 * another value. (Extension; the paper has no learned component.) */
#define HOMG_JUDGE_PROPOSAL 0
#define HOMG_JUDGE_AFTER_CYCLE 1
int homg_set_learned_judge(homg_handle h, int judge);

/* Restarted solve with the learned corrector ahead of every HOMG cycle (variable-coefficient
 * handles, HOMG_LAUNCH_GRAPH or STREAM alike: this loop is host-driven, one synchronisation per
 * proposal and per cycle): r = f - A u; stop as homg_solve does; features -> network -> proposal
 * u' = u + rho y, judged as homg_set_learned_judge selects; the cycle(s) of the Sec. 2 restart
 * follow. Once two proposals in a row have been rejected the network proposes nothing more in this
 * solve (plain HOMG cycles only). accepted_out (optional, max_cycles ints) receives the judge's
 * decisions (0 for cycles without a proposal). Returns like homg_solve. */
int homg_solve_learned(homg_handle h, homg_net_handle net, const double* f, double* u, double tol, int max_cycles,
                       int* cycles_out, double* relres_out, int* accepted_out);

#ifdef __cplusplus
}
#endif

#endif /* HOMG_NET_H */
