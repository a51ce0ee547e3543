// Private declarations shared by the HOMG kernels and the host-side C ABI implementation.
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder comes from the runtime's entry-point query)
#include <cuda_runtime.h>
#include <stdint.h>

namespace homg {

// Storage precision of a cycle's arrays (restricted sources, iterates, variations). The residual,
// the update u += e and the norms are always FP64.
enum Prec { PREC_FP64 = 0, PREC_FP32 = 1, PREC_BF16 = 2 };

inline int prec_bytes(int prec) { return prec == PREC_FP64 ? 8 : (prec == PREC_FP32 ? 4 : 2); }

// Cycle state kept on the device for one solve (written by the host before the graph launch,
// updated by the convergence-test kernel, read back once at the end).
struct State {
    const double* f;   // caller right-hand side, unpadded (n+1)^d
    double* u;         // caller solution, unpadded (n+1)^d
    double tol;
    double div_factor;
    int max_cycles;
    int stages;        // cycle stages unrolled in the solve graph
    int stage_base;    // cycles completed before the current graph launch
    int cycle;         // cycles completed
    int status;        // -1 running, else HOMG_OK / HOMG_NOT_CONVERGED / HOMG_DIVERGED
    int done;
    int zero_u;        // ||f|| == 0: the solution is u = 0
    long long t_start; // batch solves: device clock (ns) at the initial test and at convergence
    long long t_done;
    double fnorm;
    double rr0;
    double relres;
    int fault;         // set by a kernel whose bounded wait gave up (a TMA copy that never arrived)
};

// A grid array of the cycle's storage type: `n` intervals per side, rows of `pitch` elements,
// (n+1) rows per plane.
struct Grid {
    void* p;
    int64_t pitch;
    int n;
    int64_t bstride = 0;  // elements between consecutive problems of a batch (0: one problem)
};

struct CGrid {
    const void* p;
    int64_t pitch;
    int n;
    int64_t bstride = 0;  // elements between consecutive problems of a batch (0: one problem)
};

// An FP64 grid (solution iterates).
struct DGrid {
    double* p;
    int64_t pitch;
    int n;
    int64_t bstride = 0;  // elements between consecutive problems of a batch (0: one problem)
};

struct CDGrid {
    const double* p;
    int64_t pitch;
    int n;
    int64_t bstride = 0;  // elements between consecutive problems of a batch (0: one problem)
};

// One HOMG iteration on a grid of n intervals per side (the fine grid in the whole-grid form, a
// level's compact lattice in the lattice form):
//   relax the stride-2^m lattice (source g, compact, one value per lattice node),
//   add the interpolation of the pending variation dprev (compact at stride 2^mp) off its lattice.
struct IterArgs {
    int nb = 1;                  // problems in the batch (launch z extent, 2-D only)
    const State* bst = nullptr;  // batch: per-problem states (problem z = blockIdx.z); nullptr: one problem
    CGrid e_old;    // p == nullptr: e_old = 0
    Grid e_new;
    CGrid g;        // compact level-m source, pre-scaled: h_m^2 F_m (strict) or omega h_m^2 F_m
    int m;          // relaxation stride exponent
    int mp;         // pending stride exponent, -1: none
    CGrid dprev;    // compact pending variation (level mp)
    Grid dnew;      // compact variation output (p == nullptr: not stored)
    double omega;   // damped-Jacobi weight omega_J / (2d)
    double c1;      // 1 - 2d omega (fast forms)
    int rows = 0;   // fast 2-D/3-D kernels: nodes per thread along the march (0: size heuristic)
    float omega_f;  // the same, rounded to binary32, for the binary32-arithmetic kernels
    float c1_f;
    // 1, as a run-time value: an addition written as fma(one, x, y) stays a fused multiply-add
    // (GB300's FP64 pipe issues those faster than additions), where a literal 1 would be folded.
    double one = 1.0;
    // Variable coefficients (2-D lattice form; nullptr: Poisson): per lattice node the east-face
    // and north-face coefficients and the Jacobi weight omega_J / D, in double for FP64 cycles and
    // float otherwise, rows of `kpitch` elements. The source g is then h_m^2 F_m (not omega-scaled).
    const void* kx = nullptr;
    const void* ky = nullptr;
    const void* wd = nullptr;
    int64_t kpitch = 0;
};

// Lattice form, level change: fine lattice G (stride 1) from the coarser lattice's final iterate
// Gc and last variation dl (both compact at stride 2^s on G): lattice nodes copy Gc, the others
// get the interpolant of (Gc - dl), the value the whole-grid iterate holds there before the
// delayed interpolation of dl is applied.
struct ProlongArgs {
    int nb = 1;                  // problems in the batch (launch z extent, 2-D only)
    const State* bst = nullptr;  // batch: per-problem states (problem z = blockIdx.z); nullptr: one problem
    Grid G;
    CGrid Gc;
    CGrid dl;
    int s;
};

// Update + residual: u_out = u_in (+ e); r = f - A_h u_out; g0 = scale * r; partial sums of r^2
// (and f^2) per block.
struct ResidArgs {
    State* st;
    CDGrid u_in;    // p == nullptr: read the caller's u (st->u, unpadded)
    CGrid e;        // p == nullptr: no update
    DGrid u_out;    // p == nullptr: not written
    Grid g0;        // p == nullptr: not written
    double scale;   // h^2 (strict) or omega h^2
    float scale_f;  // the same, rounded to binary32 (binary32 and bfloat16 sources of the fast forms)
    double inv_h2;
    double* part_r;
    double* part_f; // nullptr: not accumulated
    int64_t part_bstride = 0;  // batch: partials between consecutive problems
    int batch = 0;             // batch: st points at per-problem states, problem z = blockIdx.z
    int nb = 1;
    const double* kx = nullptr;  // variable coefficients (2-D): east / north face coefficients of
    const double* ky = nullptr;  // the fine grid, rows of kpitch; nullptr: Poisson
    int64_t kpitch = 0;
    double one = 1.0;            // run-time 1 (see IterArgs::one)
};

// Full weighting g_c = 4 * FW(g_f) (the factor 4 = 2^2 keeps the source pre-scaled by h_m^2),
// times `scale` in the fast forms (the V-cycle's coarsest level uses another Jacobi weight).
struct RestrictArgs {
    int nb = 1;                  // problems in the batch (launch z extent, 2-D only)
    const State* bst = nullptr;  // batch: per-problem states (problem z = blockIdx.z); nullptr: one problem
    CGrid gf;
    Grid gc;
    double scale;   // 1 in strict mode
};

// V-cycle comparator: level residual rho = g - omega lap(e) (pre-scaled like g; e_old == nullptr:
// e = 0), and prolongation-add e += P ec (bilinear from the coarser compact grid, in place).
struct VResidArgs {
    CGrid e;
    CGrid g;
    Grid rho;
    double omega;
};

struct ProlongAddArgs {
    Grid e;
    CGrid ec;
};

// Convergence test (one block): sums the residual partials in a fixed order and decides.
enum FinalizeMode { FIN_INIT = 0, FIN_CYCLE = 1, FIN_NORM = 2 };

struct FinalizeArgs {
    State* st;
    double* hist;
    const double* part_r;
    const double* part_f;
    int nparts;
    int mode;
    const cudaGraphConditionalHandle* handles;  // 3 per stage, stage k at [3k, 3k+3)
    int nstages;
    // batch (one block per problem): hist, partials and states advance by these strides;
    // `ticket` counts finished blocks so the last one decides whether the next stage runs.
    int batch = 0;
    int64_t hist_bstride = 0;
    int64_t part_bstride = 0;
    unsigned int* ticket = nullptr;
};

struct CopyOutArgs {
    State* st;
    int batch = 0;  // st points at per-problem states, problem z = blockIdx.z
    int nb = 1;
    CDGrid u0;   // internal iterate after an even number of cycles
    CDGrid u1;   // ... after an odd number
};

// Power-of-two grids (Sec. 3): N = 2^K nodes per side, four quadrant lattices per level m >= 1,
// each marked from its external corner (local nodes (a, b), 0 <= a, b <= n_m = (N/2) >> m), one
// row/column past the centre lines; quadrant q's level arrays sit at q * bstride elements.
struct Pow2IterArgs {
    int N;          // nodes per side; fine arrays hold N rows of `pitch` elements
    int m;          // relaxation level (0: every interior node)
    int mp;         // pending level >= 1, or -1
    CGrid e_old;    // fine iterate (p == nullptr: 0)
    Grid e_new;
    CGrid g;        // m = 0: fine source; m >= 1: the four quadrant arrays (pre-scaled: omega h_m^2 F)
    CGrid dprev;    // level mp: four quadrant arrays
    Grid dnew;      // level m >= 1: four quadrant arrays (p == nullptr: not stored)
    double omega, c1;
    float omega_f, c1_f;
};

// Level-m sources from the fine source g0 by the separable hat stencil (the m-fold nested full
// weighting), times 4^m to keep the h_m^2 scaling: a row pass into tmp, then a column pass.
struct Pow2RestrictArgs {
    int N, m;
    CGrid g0;       // fine source
    double* tmp;    // N rows x 2 x (n_m + 1)
    Grid gm;        // the four quadrant arrays of level m
};

// One op of the coarse-lattice block kernel (fast forms, lattice form only).
enum BlockKind { BLOCK_RESTRICT = 0, BLOCK_PROLONG = 1, BLOCK_ITER = 2 };

struct BlockOp {
    int kind;
    IterArgs it;
    ProlongArgs pr;
    RestrictArgs rs;
};

// ---- persistent batch kernel ------------------------------------------------------------------
// One cooperative launch runs a whole batch: every size group's cycle is a list of ops (the same
// ops its graph launches), and phase j of the launch holds op j of every group. A phase's work is a
// queue of (op, problem, tile) items, the op's blocks over all of its group's problems, which the
// resident blocks draw from a counter; a grid barrier separates phases.
enum PersistKind {
    PK_ITER = 0,      // marching damped-Jacobi sweep (sub = 2 * pending mode + variation stored)
    PK_ITER2 = 1,     // two fused plain sweeps
    PK_ITER4 = 2,     // four fused plain sweeps
    PK_ITERG = 3,     // generic HOMG iteration (tiles of BX x BY nodes)
    PK_PROLONG2 = 4,  // stride-2 level change (marching)
    PK_PROLONG = 5,   // generic level change (tiles)
    PK_RESTRICT = 6,  // full weighting (tiles)
    PK_BLOCK = 7,     // coarse-lattice op list, one block per problem
    PK_RESID = 8,     // update + residual + source + norm partials
    PK_FINAL = 9,     // convergence test, one block per problem
    PK_COPY = 10      // copy-out (tiles)
};

struct PersistItem {
    int kind = 0;
    int sub = 0;
    int rows = 0;               // nodes per thread along the march
    int n = 0;                  // PK_RESID, PK_COPY: intervals per side
    int gx = 1, gy = 1, gz = 1; // the op's blocks (gz: problems of the group)
    int nops = 0;               // PK_BLOCK
    const BlockOp* ops = nullptr;
    IterArgs it;
    ProlongArgs pr;
    RestrictArgs rs;
    ResidArgs ra;
    FinalizeArgs fa;
    CopyOutArgs co;
};

struct PersistPhase {
    int first, count;  // items
    int blocks;        // their blocks in total
};

struct PersistArgs {
    const PersistItem* items = nullptr;
    const PersistPhase* phases = nullptr;
    int init_first = 0, init_count = 0;  // initial residual and test
    int cyc_first[2] = {0, 0};           // a cycle of even / odd stage
    int cyc_count = 0;
    int copy_first = 0, copy_count = 0;
    int max_cycles = 0;
    unsigned int* sync = nullptr;        // [0] arrivals, [1] generation, [2..4] running problems (rotating)
    unsigned int* queue = nullptr;       // one work counter per phase executed, zero at launch
    int* err = nullptr;                  // 1 when a grid barrier gave up
    long long timeout_ns = 0;            // longest wait at one grid barrier
    int stall = 0;                       // self-test: the first barrier waits for one block more than exist
};

// Item builders (the same kernels and launch shapes as the graph launches of launch_iterate & co.)
void persist_iter(const IterArgs& a, PersistItem& it);
void persist_iter2(int sweeps, const IterArgs& a, PersistItem& it);
void persist_prolong(const ProlongArgs& a, PersistItem& it);
void persist_restrict(const RestrictArgs& a, PersistItem& it);
void persist_block(const BlockOp* ops, int nops, int nb, PersistItem& it);
void persist_resid(const ResidArgs& a, int n, PersistItem& it);
void persist_final(const FinalizeArgs& a, PersistItem& it);
void persist_copy(const CopyOutArgs& a, int n, PersistItem& it);
// Cooperative launch of the persistent kernel for storage precision prec: as many blocks as can be
// resident on the device at once (*blocks receives the count).
cudaError_t launch_persistent(int prec, const PersistArgs& a, int* blocks, cudaStream_t s);

// Launchers (enqueue on `s`; return the launch error). `prec` is the storage precision of the
// cycle arrays (Prec); `strict` selects the oracle's canonical operation order.
cudaError_t launch_iterate(int ndim, int prec, bool strict, const IterArgs& a, cudaStream_t s);
// f_out = binary64 -> binary32 (round to nearest even) of d_in, d_out = binary32 -> binary64 of f_in,
// with the integer conversions of the fast residual kernels (n elements, device pointers).
bool pairs_ok(int prec, const IterArgs& a);
cudaError_t launch_check_sweep_pair(int prec, const IterArgs& a, void* out_packed, cudaStream_t s);
cudaError_t launch_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n,
                                     cudaStream_t s);
// `sweeps` (2 or 4) plain lattice-form sweeps in one launch (2-D, FP32 / bfloat16 storage, no
// pending interpolation, no variation output): e_new = sweep(...sweep(e_old)).
cudaError_t launch_iterate2(int prec, int sweeps, const IterArgs& a, cudaStream_t s);
// Two fused plain sweeps with the tile staged by TMA (binary32 / bfloat16, 2-D, one problem):
// me = tensor map of e_old, mg = of g (tma_sweep_maps); fault = where a copy that never arrives is
// reported (State::fault).
struct TmaSweepMaps {
    CUtensorMap me;
    CUtensorMap mg;
};
constexpr int XT_MIN_N = 256;  // smallest lattice the TMA two-sweep kernel is planned for
cudaError_t tma_sweep_maps(int prec, const IterArgs& a, TmaSweepMaps* maps);
cudaError_t launch_iterate2_tma(int prec, const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s);
// The same for 3-D lattices (planes staged by TMA, the block marching down z).
cudaError_t tma_sweep_maps3(int prec, const IterArgs& a, TmaSweepMaps* maps);
cudaError_t launch_iterate3_2_tma(int prec, const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s);
// Two plain 3-D lattice-form sweeps in one launch (FP32 / bfloat16 storage).
cudaError_t launch_iterate3_2(int prec, const IterArgs& a, cudaStream_t s);
cudaError_t launch_prolong(int ndim, int prec, bool strict, const ProlongArgs& a, cudaStream_t s);
cudaError_t launch_residual(int ndim, int prec, bool strict, const ResidArgs& a, int n, cudaStream_t s);
int residual_blocks(int ndim, bool strict, int n);  // partial sums written by launch_residual
cudaError_t launch_restrict(int ndim, int prec, bool strict, const RestrictArgs& a, cudaStream_t s);
cudaError_t launch_coarse_block(int ndim, int prec, const BlockOp* ops, int nops, int nb, cudaStream_t s);
// Lattice form, binary32 cycles (2-D): a level change and the whole run of `sweeps` sweeps on a
// lattice of at most RUN_MAX_N intervals per side, in one block per problem (shared memory).
constexpr int RUN_MAX_N = 128;
cudaError_t launch_level_run(int prec, const ProlongArgs& pr, const IterArgs& it, int sweeps, int nb, cudaStream_t s);
// Raises the level-run kernel's shared-memory limit on the current device (before any capture).
cudaError_t prepare_level_run(int prec);
cudaError_t launch_vresid(int ndim, int prec, bool strict, const VResidArgs& a, cudaStream_t s);
cudaError_t launch_prolong_add(int ndim, int prec, bool strict, const ProlongAddArgs& a, cudaStream_t s);
cudaError_t launch_pow2_iterate(int prec, const Pow2IterArgs& a, cudaStream_t s);
cudaError_t launch_pow2_restrict(int prec, const Pow2RestrictArgs& a, cudaStream_t s);
cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s);
// Variable coefficients of level m from the node coefficient k ((n+1)^2, unpadded, FP64): for each
// lattice node the east- and north-face harmonic means and (wd != nullptr) the weight omega_J / D,
// stored as double (dbl) or float. Sets *bad when a node value is not positive and finite.
cudaError_t launch_vc_setup(const double* k, int n, int m, bool dbl, void* kx, void* ky, void* wd, int64_t pitch,
                            double omega_j, int* bad, cudaStream_t s);
cudaError_t launch_copy_out(int ndim, const CopyOutArgs& a, int n, cudaStream_t s);

// Message reported by homg_last_error(NULL) (errors of calls made without a handle).
void set_null_handle_error(const char* msg);

}  // namespace homg
