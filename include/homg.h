/*
 * homg.h -- C ABI of the GB300 (sm_103a) high-occupancy multigrid (HOMG) solver.
 *
 * Method: Becerra-Sagredo, Malaga and Mandujano, "A novel and scalable Multigrid algorithm for
 * many-core architectures" (arXiv:1108.2045). The library solves A u = f (Sec. 2, Eq. 1) for the
 * Poisson problem on the unit square or cube with zero Dirichlet boundary (Sec. 4, Eq. "poisson"),
 * A = -Laplacian discretised by the 5-point (2-D) or 7-point (3-D) stencil on a node grid of
 * (2^K + 1)^d nodes, h = 2^-K. The sign convention makes A positive definite (the paper writes
 * Laplacian(u) = f; pass -f to solve the paper's form).
 *
 * One solve = restarted HOMG cycles on the residual equation (Sec. 2, last paragraph) until
 *   ||f - A u||_2 / ||f||_2 <= tol      (2-norms over interior nodes)
 * Each cycle: residual and full-weighting restriction to every level (Sec. 2, restriction
 * paragraph), then the MFMG sequence of HOMG iterations from the coarsest level to the finest
 * (Sec. 2, steps (a)-(c), MFMG paragraph), each iteration relaxing the level-m lattice with damped
 * Jacobi (Sec. 2, relaxation formula) fused with the interpolation of the previous iteration's
 * variations on the rest of the grid, then u += e. Everything runs on the GPU: the cycle loop and
 * its convergence test are captured in one CUDA graph with device-side conditional nodes, and the
 * host synchronises once per solve.
 *
 * Conventions shared by every entry point:
 * - Return codes: 0 = HOMG_OK. Positive = soft outcome with valid outputs (HOMG_NOT_CONVERGED,
 *   HOMG_DIVERGED). Negative = hard error, outputs untouched (HOMG_EINVAL, HOMG_ESHAPE, HOMG_ECUDA,
 *   HOMG_ENOMEM); homg_last_error() then describes it. No C++ exception crosses this ABI and no
 *   kernel traps.
 * - Grid arrays are FP64, contiguous, row-major with x fastest: node (i, j[, k]) at
 *   j*(n+1) + i (2-D) or (k*(n+1) + j)*(n+1) + i (3-D), n = 2^K, covering the whole node grid
 *   including the boundary. Only interior nodes are read or written; the operator takes the
 *   boundary value 0.
 * - Device pointers are caller-owned CUDA device (or managed) memory on the handle's device.
 *   They must stay valid until the call returns; the library keeps no reference to them.
 * - A handle is not thread-safe: use one handle per host thread (or serialise calls).
 */
#ifndef HOMG_H
#define HOMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------------------------- */
#define HOMG_OK 0
#define HOMG_NOT_CONVERGED 1 /* max_cycles cycles done, relative residual still above tol       */
#define HOMG_DIVERGED 2      /* relative residual not finite, or above diverge_factor * initial   */
#define HOMG_TIMEOUT 3       /* a bounded device-side wait (persistent batch grid barrier) gave up */
#define HOMG_EINVAL (-1)     /* invalid argument (null pointer, level count, stencil, options ...)  */
#define HOMG_ESHAPE (-2)     /* grid sides not 2^K + 1, not all equal, or too large                 */
#define HOMG_ECUDA (-3)      /* a CUDA runtime call failed                                          */
#define HOMG_ENOMEM (-4)     /* device or pinned host allocation failed                             */

/* ---- execution forms of the same iterates -------------------------------------------------- */
/* HOMG_EXEC_WHOLEGRID: the paper's form (Sec. 2: "operations over the entire grid"): every HOMG
 *   iteration is one launch over every fine-grid node, relaxing the level-m lattice and adding the
 *   interpolated previous variation everywhere else (one working unit per iteration, Sec. 4).
 * HOMG_EXEC_LATTICE: the same iterates up to rounding order, computed level by level on each
 *   level's own lattice. The HOMG iterate restricted to the level-m lattice depends only on values
 *   on that lattice, so the iterations of level m run on its compact (n/2^m + 1)^d copy; at each
 *   level change one fused kernel interpolates the coarser lattice's iterate onto the finer one
 *   with the one-iteration delay of Sec. 4 (Fig. 3 discussion). Requires a schedule whose levels
 *   never increase (MFMG is such a schedule).
 * HOMG_EXEC_AUTO: LATTICE when the schedule allows it, else WHOLEGRID. */
#define HOMG_EXEC_AUTO 0
#define HOMG_EXEC_WHOLEGRID 1
#define HOMG_EXEC_LATTICE 2

/* Largest max_cycles accepted by homg_solve (the cycle loop is unrolled into the solve graph). */
#define HOMG_MAX_CYCLES 200
/* Largest grid side exponent K accepted: 2-D n <= 2^15, 3-D n <= 2^10. */
#define HOMG_MAX_K_2D 15
#define HOMG_MAX_K_3D 10

typedef struct homg_options {
    /* Damped-Jacobi weight omega_J; each relaxation uses omega = omega_J / (2d) (Sec. 2,
     * relaxation formula with the Jacobi diagonal 2d). 0 selects 4/5 (2-D) or 6/7 (3-D). */
    double omega_j;
    /* MaxI of the MFMG cycle (Sec. 2, MFMG paragraph): 2 iterations on the coarsest level,
     * doubling per finer level, capped at max_i. 0 selects 32, the paper's timing setting (Sec. 4). */
    int max_i;
    /* Optional explicit schedule (Sec. 2 step (c): "a chosen pattern"): n_schedule level indexes in
     * [0, levels), one per HOMG iteration, ending with 0. Copied by homg_create. 0/NULL = MFMG. */
    int n_schedule;
    const int* schedule;
    /* HOMG_EXEC_* (see above). */
    int exec_mode;
    /* 1: evaluate every formula in the CPU oracle's canonical operation order with no fused
     * multiply-add contraction (whole-grid form then reproduces the oracle's iterates bit for bit).
     * 0: reassociated forms with fewer FP64 instructions (results equal up to rounding). */
    int strict_fp;
    /* Divergence threshold on the relative residual, as a multiple of the initial one. 0 = 1e3. */
    double diverge_factor;
    /* HOMG_LAUNCH_GRAPH (default): the whole solve is one CUDA graph launch with device-side
     * conditional nodes. HOMG_LAUNCH_STREAM: the same kernels enqueued directly on the stream, the
     * host reading the cycle state once per cycle; meant for profilers and debuggers that cannot
     * look inside graphs with conditional nodes. Results are identical. */
    int launch_mode;
    /* Precision of each cycle's values (restricted sources, iterates, variations):
     * HOMG_PREC_FP64 (default), HOMG_PREC_FP32 (binary32), HOMG_PREC_BF16 (bfloat16 storage,
     * binary32 arithmetic). The residual, the update u += e and the norms are always FP64, so the
     * restart loop is iterative refinement and reaches the same tolerance (Sec. 4 ran the method in
     * single precision). */
    int precision;
    /* HOMG_CYCLE_HOMG (default): the paper's MFMG cycle of fused HOMG iterations.
     * HOMG_CYCLE_V: the classic V(v_pre, v_post) cycle of Sec. 2 (steps (a)-(e): damped-Jacobi
     * smoothing, full-weighting restriction of the residual, bilinear correction, rediscretised
     * coarse operators; coarsest level by max(1, n_c^2) undamped Jacobi sweeps), run through the
     * same restart loop: the comparator the paper's method is measured against. */
    int cycle;
    int v_pre;   /* V-cycle pre-smoothing sweeps  (0 = 2) */
    int v_post;  /* V-cycle post-smoothing sweeps (0 = 2) */
    /* HOMG_GEOM_NESTED (default): nested grids of 2^K + 1 nodes per side.
     * HOMG_GEOM_POW2: the power-of-two grids of Sec. 3 (2-D, 2^K nodes per side, boundary nodes
     * included, h = 1/(2^K - 1)): the grid is split into four quadrants; at every level m >= 1
     * each quadrant's lattice is marked from its external corner (spacing 2^m) and reaches one
     * row/column past the centre lines, so the coarsest level holds the four central points;
     * relaxations run on all marked nodes, interpolations on the rest from the node's own
     * quadrant only; level sources are the m-fold nested full weighting of the fine residual
     * (one hat stencil per node). HOMG cycles in the whole-grid form only (the default exec mode
     * selects it), levels <= K, not with strict_fp, the V-cycle, batches or coefficients. */
    int geometry;
    /* Lattice form of binary32 / bfloat16 HOMG cycles in 2-D (not strict_fp, not with
     * coefficients): every level run on a lattice of at most run_max_n intervals per side after
     * the coarsest ones -- the level change from the coarser lattice and all of the level's
     * sweeps (Sec. 2, MFMG: n_m iterations per level) -- is one launch of one block per problem
     * that keeps the lattice and its source in shared memory between sweeps, instead of a launch
     * per sweep or pair. 0 selects 128 (the largest, limited by shared memory), a negative value
     * turns it off; at most 128. The iterates are bit-identical either way. Persistent batches
     * never use it. */
    int run_max_n;
    /* Lattice form of binary32 / bfloat16 HOMG cycles (not strict_fp, one problem per handle;
     * batches never use it): pairs of plain sweeps on lattices of at least tma_min_n intervals per
     * side run as one launch whose blocks stage their tile of the iterate and the source (with a
     * two-node halo) in shared memory by TMA tensor copies, then run both sweeps from there (3-D:
     * rings of planes, each block marching down z). 0 selects the default threshold
     * (HOMG_TMA_MIN_N_DEFAULT), a negative value turns it off; values below 256 are raised to 256.
     * The iterates are bit-identical either way. */
    int tma_min_n;
} homg_options;

#define HOMG_TMA_MIN_N_DEFAULT 256

#define HOMG_GEOM_NESTED 0
#define HOMG_GEOM_POW2 1

#define HOMG_CYCLE_HOMG 0
#define HOMG_CYCLE_V 1

#define HOMG_PREC_FP64 0
#define HOMG_PREC_FP32 1
#define HOMG_PREC_BF16 2

#define HOMG_LAUNCH_GRAPH 0
#define HOMG_LAUNCH_STREAM 1
/* Batches only (homg_batch_create; homg_create rejects it): the whole batch solve is ONE
 * cooperative launch of a persistent kernel. Phase j of a cycle holds op j of every size group's
 * cycle (the same ops, with the same arithmetic, that the group's graph launches). A phase's work is
 * a queue of (op, problem, tile) items that the resident blocks draw from a counter, and a grid
 * barrier separates phases. Every barrier wait is bounded: a block that waits longer than a few
 * seconds records the failure, every block leaves the launch, and the solve returns HOMG_TIMEOUT. */
#define HOMG_LAUNCH_PERSISTENT 2

/* Statistics of the last homg_solve on a handle (times from CUDA events recorded on the handle's
 * stream inside the solve graph; zero when the last call failed). */
typedef struct homg_stats {
    int cycles;                  /* cycles performed                                            */
    int status;                  /* return code of the last solve                               */
    int exec_mode;               /* form actually used (HOMG_EXEC_WHOLEGRID / _LATTICE)          */
    int precision;               /* HOMG_PREC_* of the cycle arrays                              */
    int iterations_per_cycle;    /* HOMG iterations (working units) per cycle                    */
    int fine_iterations_per_cycle;   /* iterations on the finest level (level 0) per cycle      */
    int kernels_per_cycle;       /* kernel launches per cycle                                    */
    int kernels_fixed;           /* kernel launches per solve outside the cycles                 */
    long long kernel_launches;   /* total kernel launches of the last solve                      */
    double solve_ms;             /* whole solve graph, first node to last                        */
    double coarse_ms;            /* sum over cycles: iterations on levels >= 1                   */
    double fine_ms;              /* sum over cycles: iterations on level 0                       */
    double residual_ms;          /* sum over cycles: update + residual + restriction + test     */
    double setup_ms;             /* initial residual + final copy-out                            */
    double fine_bytes_per_iteration;   /* algorithmic DRAM bytes of one level-0 iteration       */
    double fine_flops_per_iteration;   /* algorithmic floating-point instructions (FP64 or FP32,
                                        * by precision) of one level-0 iteration                  */
    double coarse_bytes_per_cycle;     /* algorithmic DRAM bytes of the levels >= 1 per cycle   */
    double coarse_fp64_ops_per_cycle;  /* algorithmic FP64 instructions of levels >= 1 per cycle */
    int fine_launches_per_cycle;       /* level-0 sweep launches per cycle (binary32 cycles fuse
                                        * consecutive plain sweeps, so this can be fewer than
                                        * fine_iterations_per_cycle; each launch moves about
                                        * fine_bytes_per_iteration)                              */
} homg_stats;

typedef struct homg_ctx* homg_handle;

/* Fill *opt with the defaults described above. */
void homg_default_options(homg_options* opt);

/* Create a solver for a (2^K+1)^ndim node grid (Sec. 2: nested grids doubling the spacing), or a
 * (2^K)^2 grid with geometry HOMG_GEOM_POW2 (Sec. 3).
 *   ndim     2 or 3.
 *   dims     ndim node counts, all equal to 2^K + 1 with K >= 1 (power-of-two geometry: 2^K with
 *            2 <= K <= HOMG_MAX_K_2D) (ESHAPE otherwise).
 *   levels   number of levels L, 1 <= L <= K; level m has spacing 2^m h, the coarsest is L-1.
 *   stencil  5 (ndim 2) or 7 (ndim 3).
 *   opt      NULL for defaults.
 *   out      receives the handle (NULL on failure).
 * Allocates one device buffer holding every level (all compact level arrays, the fine iterates,
 * the per-level restricted sources, norm partials and the cycle state) on the current device,
 * and creates the handle's events and pinned host state. A 2-D handle in the fast lattice form
 * then times its marching sweeps once per lattice size on the legacy default stream (a few ms;
 * the choice changes launch shapes only, never results). Returns 0 or a negative code. */
int homg_create(int ndim, const int64_t* dims, int levels, int stencil, const homg_options* opt, homg_handle* out);

/* Use `stream` (a cudaStream_t, NULL = legacy default stream) for every later call on h. */
int homg_set_stream(homg_handle h, void* stream);

/* Restarted HOMG solve (Sec. 2 last paragraph; Sec. 4: "the residual equation is used to restart
 * the cycles as many times as needed").
 *   f           device pointer, right-hand side (interior nodes used).
 *   u           device pointer, in: initial guess, out: solution (interior nodes only).
 *   tol         stop when ||r||/||f|| <= tol (>= 0, finite).
 *   max_cycles  0 .. HOMG_MAX_CYCLES; 0 only evaluates the initial residual.
 *   cycles_out, relres_out  optional; receive the cycle count and the final relative residual.
 * Returns HOMG_OK, HOMG_NOT_CONVERGED or HOMG_DIVERGED (u holds the last iterate), or a negative
 * code. ||f|| = 0 gives u = 0 and relres 0 after 0 cycles. The call enqueues one graph launch on
 * the handle's stream and synchronises that stream once, at the end. */
int homg_solve(homg_handle h, const double* f, double* u, double tol, int max_cycles, int* cycles_out,
               double* relres_out);

/* Same as homg_solve with HOST arrays (pinned memory recommended): copies f and u to device
 * buffers owned by the handle (allocated on first use), solves, copies u back. */
int homg_solve_host(homg_handle h, const double* f_host, double* u_host, double tol, int max_cycles,
                    int* cycles_out, double* relres_out);

/* Switch h to the variable-coefficient operator A u = -div(k grad u) (an extension: the paper
 * solves the Poisson equation only). Five-point flux form: each face carries the harmonic mean
 * 2 k(p) k(q) / (k(p) + k(q)) of its two end nodes' coefficients; level m uses the same form
 * between lattice neighbours at spacing 2^m h with k taken at the lattice nodes (injection); the
 * HOMG relaxation (Sec. 2) becomes damped Jacobi with each node's own diagonal D (sum of its four
 * face coefficients) and weight omega_J / D, omega_J as in the options (4/5 by default).
 *   k  device pointer, FP64 node coefficients on the whole (n+1)^2 grid, boundary included (the
 *      boundary faces use them), row-major with x fastest, unpadded; only read during this call
 *      (the handle keeps its own derived coefficients). NULL switches back to the Poisson operator.
 * Needs a 2-D handle with HOMG cycles in the fast lattice form (not strict_fp, not the whole-grid
 * form, not the V-cycle): HOMG_EINVAL otherwise. k must be positive and finite at every node:
 * HOMG_EINVAL otherwise (the handle then stays on the Poisson operator). Later homg_solve and
 * homg_residual_norm calls use the operator. Allocates the coefficient arrays on first use
 * (~1/3 more than three fine-grid arrays) and synchronises the handle's stream. */
int homg_set_coefficient(homg_handle h, const double* k);

/* ||f - A u||_2 / ||f||_2 over interior nodes for device arrays f, u (relres_out required);
 * 0 when ||f|| = 0 and u's interior is 0, +inf when ||f|| = 0 otherwise. Synchronises the stream. */
int homg_residual_norm(homg_handle h, const double* f, const double* u, double* relres_out);

/* Self-test of the library's own binary64 <-> binary32 conversions. The fast residual kernels form
 * them with integer operations, from the IEEE 754 formats, to keep them off GB300's narrow FP64
 * pipe. For k < n: f_out[k] = d_in[k] rounded to binary32 (round to nearest, ties to even), d_out[k] =
 * f_in[k] widened to binary64. All four are device pointers; runs on the current device on the legacy
 * default stream and synchronises. Both results must equal the hardware conversions bit for bit.
 * HOMG_EINVAL for n < 0 or a null pointer with n > 0 (message in homg_last_error(NULL)). */
int homg_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n);

/* Self-test of the two-sweep kernels of binary32 cycles: consecutive plain damped-Jacobi sweeps
 * (Sec. 2, the relaxation formula) that the fast lattice form fuses two per launch. On a lattice of n
 * intervals per side (n+1 rows of `pitch` elements; pitch >= n + 2 and even) of `precision`
 * HOMG_PREC_FP32 (float) or HOMG_PREC_BF16 (bfloat16), two sweeps v' = c1 v + omega (sum of the four
 * neighbours) + g of the input e_old (binary32 arithmetic, each sweep's values rounded to the storage
 * type) are written to the interior of e_packed by the kernel with two columns per lane (packed
 * binary32 pairs) and to the interior of e_column by the kernel with one column per lane; boundary
 * nodes and padding of both outputs are left untouched, and e_old's boundary nodes are read as
 * stored. rows: lattice rows per block (0: 8). Device pointers aligned to two elements; runs on the
 * current device on the legacy default stream and synchronises. The two results must be equal bit
 * for bit. HOMG_EINVAL for another precision, n < 2, a null pointer, an odd or short pitch or an
 * unaligned pointer (message in homg_last_error(NULL)). */
int homg_check_sweep_pair(int precision, int n, int64_t pitch, const void* e_old, const void* g, void* e_packed,
                          void* e_column, double omega, double c1, int rows);

/* Relative residual before every cycle of the last solve: hist[0] = initial, hist[k] after k
 * cycles. Copies min(cap, cycles + 1) values; returns that count or a negative code. */
int homg_get_history(homg_handle h, double* hist, int cap);

/* Statistics of the last solve (see homg_stats). */
int homg_get_stats(homg_handle h, homg_stats* out);

/* Message for the last hard error on h (or of the last failed homg_create when h is NULL). */
const char* homg_last_error(homg_handle h);

/* Release every resource of h (no-op for NULL). */
void homg_destroy(homg_handle h);

/* ---- batched solves (many independent 2-D problems of uneven sizes) --------------------------
 * Problems of equal size form a group whose every kernel launch advances all of the group's
 * problems at once (problem index = third launch dimension); each problem keeps its own cycle
 * state and stops on its own test, its blocks exiting at once after it converged. Each group's
 * solve graph runs on its own stream, forked from the caller's stream. At creation an autotuner
 * times the level-0 sweep of every group with each candidate tile height (nodes per thread along
 * the march) and keeps the fastest. Fast arithmetic, lattice form and the HOMG cycle only. */
typedef struct homg_batch_ctx* homg_batch_handle;

#define HOMG_BATCH_MAX_GROUPS 16

typedef struct homg_batch_stats {
    int groups;                              /* distinct grid sizes                              */
    double solve_ms;                         /* last solve: caller-stream events around the batch */
    int64_t sides[HOMG_BATCH_MAX_GROUPS];    /* per group: nodes per side                        */
    int counts[HOMG_BATCH_MAX_GROUPS];       /* per group: problems                              */
    int rows[HOMG_BATCH_MAX_GROUPS];         /* per group: tuned nodes per thread, level-0 sweep */
    double tuned_us[HOMG_BATCH_MAX_GROUPS];  /* per group: time of one batched level-0 sweep      */
} homg_batch_stats;

/* Create a batch of nprob 2-D problems; sides[p] = 2^K_p + 1 nodes per side (levels = K_p each).
 * opt as for homg_create (NULL = defaults); strict_fp, the whole-grid form, explicit schedules, the
 * V-cycle and the stream launch mode are rejected (HOMG_EINVAL). At most HOMG_BATCH_MAX_GROUPS
 * distinct sizes. Allocates one level buffer per group and runs the autotuner (on the device). */
int homg_batch_create(int nprob, const int64_t* sides, const homg_options* opt, homg_batch_handle* out);

/* Stream of the caller (NULL = legacy default stream): the groups fork from it and join it. */
int homg_batch_set_stream(homg_batch_handle b, void* stream);

/* Solve every problem (Sec. 2 restart loop, per problem): f[p], u[p] are device pointers to the
 * (sides[p])^2 arrays of problem p (host array of nprob pointers). Optional outputs, nprob entries
 * each: status (HOMG_OK / HOMG_NOT_CONVERGED / HOMG_DIVERGED), cycles, final relres, and solve_ms,
 * the device time from the problem's initial residual test to its convergence (device clock).
 * Returns 0 when every problem converged, HOMG_NOT_CONVERGED / HOMG_DIVERGED when one did not
 * (worst status), or a negative code. Synchronises the caller's stream. */
int homg_batch_solve(homg_batch_handle b, const double* const* f, double* const* u, double tol, int max_cycles,
                     int* status, int* cycles, double* relres, double* solve_ms);

int homg_batch_get_stats(homg_batch_handle b, homg_batch_stats* out);

/* Release every resource of b (no-op for NULL). */
void homg_batch_destroy(homg_batch_handle b);

/* Self-test of the persistent batch kernel's failure path (b created with HOMG_LAUNCH_PERSISTENT):
 * launches the kernel so that its first grid barrier waits for one block more than the launch has,
 * with a 0.25 s limit. Nothing reads or writes problem data. Every block gives up, records the
 * failure and leaves, so the call returns HOMG_TIMEOUT with a message in homg_last_error(NULL),
 * *waited_ms (optional) the launch's duration, and the context stays usable (the next
 * homg_batch_solve works). HOMG_OK here would mean the wait is not bounded as documented;
 * HOMG_EINVAL for a batch without the persistent mode. Synchronises the batch's stream. */
int homg_batch_check_barrier_timeout(homg_batch_handle b, double* waited_ms);

/* Threads per block of homg_fp64_issue_probe. */
#define HOMG_PROBE_THREADS 256

/* Measurement service (the paper has no counterpart): the GPU's FP64 instruction issue rate, the
 * ceiling of this library's FP64 stencil kernels on GB300, whose FP64 pipe is far narrower than its
 * DRAM (a level-0 sweep issues 5 FP64 instructions per 24 bytes). Enqueues one kernel of `blocks`
 * blocks of HOMG_PROBE_THREADS threads on `stream` (a cudaStream_t, NULL = legacy default stream);
 * every thread runs 8 independent chains of `iters` dependent FP64 instructions, x <- x * a + b
 * (op 0, fused multiply-add) or x <- x + b (op 1, addition), and stores the sum of its chains at
 * sink[block * HOMG_PROBE_THREADS + thread] (caller-owned device array of at least
 * blocks * HOMG_PROBE_THREADS doubles). *instructions_out (host) receives the FP64 instructions the
 * launch executes, blocks * HOMG_PROBE_THREADS * iters * 8 (plus 8 per thread for the sums). The
 * caller times the launch (CUDA events on `stream`); the call does not synchronise. HOMG_EINVAL
 * for op outside {0, 1}, blocks or iters < 1, or a null pointer; HOMG_ECUDA if the launch fails
 * (message in homg_last_error(NULL)). */
int homg_fp64_issue_probe(int op, int blocks, int iters, double* sink, void* stream, double* instructions_out);

/* Capacity of the static scratch used by homg_residual_norm_noalloc: one partial sum per thread
 * block of the residual kernel, at most this many (2-D grids up to 8193^2, 3-D up to 513^3). */
#define HOMG_NOALLOC_MAX_BLOCKS 65536

/* Allocation-free relative residual ||f - A u||_2 / ||f||_2 (interior nodes) of device arrays f
 * and u on a (dims[0])^ndim node grid, for callers that cannot call cudaMalloc (it synchronises the
 * device, and fails when another allocator already holds the memory) and so cannot create a handle.
 * The paper has no counterpart: this is a service entry point of the library, the same computation
 * as homg_residual_norm without a handle.
 *   dims       ndim equal node counts 2^K + 1; grids needing more than HOMG_NOALLOC_MAX_BLOCKS
 *              partial sums are rejected with HOMG_ESHAPE and a message in homg_last_error(NULL).
 *   stream     cudaStream_t to run on (NULL = legacy default stream); synchronised before return.
 *   relres_out host pointer receiving the result (0 when f = 0 and u's interior is 0, +inf when
 *              f = 0 otherwise).
 * Scratch: a fixed file-scope device array of (32 + 2 * HOMG_NOALLOC_MAX_BLOCKS) doubles
 * (1,048,832 bytes, just over 1 MiB), held by every GPU that loads the library until the process
 * exits, shared by all calls and keeping the last call's contents (every value a call reads is
 * written by that call first). Calls whose work overlaps on one GPU (other host threads, other
 * streams) race on it: serialise them. The current device must be the one holding f and u. Each
 * call made outside stream capture looks up the array's device address on the current device
 * (cudaGetSymbolAddress), so a device reset leaves the entry point usable; a call made while
 * `stream` is capturing reuses the address found by the last call outside capture on that device,
 * so make the first call on each device before any stream capture. Allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine. */
int homg_residual_norm_noalloc(int ndim, const int64_t* dims, const double* f, const double* u, double* relres_out,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HOMG_H */
