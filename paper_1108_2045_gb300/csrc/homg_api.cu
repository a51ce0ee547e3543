// Host side of the HOMG C ABI (include/homg.h): validation, the single level buffer, the cycle
// schedule and the solve graph.
//
// Solve graph (built once per handle and grown when a larger max_cycles is requested):
//   [initial residual + test] E0
//   for stage k = 1..S:  IF_A{restrict to every level; iterations on levels >= 1} E
//                        IF_B{iterations on level 0}                          E
//                        IF_C{u += e; residual; convergence test}            E
//   [copy the final iterate out] E_end
// The test kernel enables stage k+1's three conditional nodes only while the solve continues, so
// the cycle loop never returns to the host. Event nodes between the stages time each part.
#include <stdio.h>
#include <string.h>

#include <cmath>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/homg.h"
#include "../../include/homg_net.h"
#include "homg_internal.h"
#include "homg_net_internal.h"

using namespace homg;

namespace {

thread_local char g_create_error[512] = "";

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int64_t grid_elems(int ndim, int n, int64_t pitch) {
    return (ndim == 2) ? (int64_t)(n + 1) * pitch : (int64_t)(n + 1) * (n + 1) * pitch;
}

struct Level {
    int n;                 // intervals per side of the compact lattice
    int64_t pitch;         // elements per row
    void* g = nullptr;     // pre-scaled restricted source
    void* G[2] = {nullptr, nullptr};  // lattice iterates (lattice form; level 0 aliases e)
    void* d[2] = {nullptr, nullptr};  // compact variations
};

// One instantiated solve graph: `stages` unrolled cycle stages (three conditional IF nodes each)
// with event nodes between them; the handles of stage k sit at dhandles[3k .. 3k+2].
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    int stages = 0;
    bool with_init = false;
    std::vector<cudaEvent_t> ev;  // 3*stages + 3 events
    cudaGraphConditionalHandle* dhandles = nullptr;
};

// Cycle stages unrolled in one graph. Stages a solve does not reach cost a few microseconds each
// (their conditional nodes evaluate false), so the graph stays short and a solve that needs more
// cycles relaunches the continuation graph (one host synchronisation per kStagesPerGraph cycles).
constexpr int kStagesPerGraph = 12;  // even: keeps the ping-pong parity of the solution buffers

// NVTX range over a host scope (a solve, a graph launch, a cycle in stream mode): profilers that
// record NVTX (ncu --nvtx) can select a solve's kernels by it; without a tool attached it costs a
// function call.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Op {  // one kernel launch of a cycle part
    enum Kind { ITER, ITER2, PROLONG, RESTRICT, BLOCK, VRESID, PROLONG_ADD, POW2_ITER, POW2_RESTRICT, RUN } kind;
    int sweeps = 1;  // ITER2: plain sweeps fused into the launch (2 or 4); RUN: sweeps of the level run
    IterArgs it;
    Pow2IterArgs p2;
    Pow2RestrictArgs p2r;
    ProlongArgs pr;
    RestrictArgs rs;
    VResidArgs vr;
    ProlongAddArgs pa;
    int block_first = 0, block_count = 0;  // BLOCK: range of the device op list
    bool tma = false;                       // ITER2: the TMA-staged two-sweep kernel, with these maps
    TmaSweepMaps maps;
};

// Capacity of the coarse-lattice block's op list in the level buffer.
constexpr int kMaxBlockOps = 1024;

}  // namespace

struct homg_ctx {
    int ndim = 2, n = 0, K = 0, levels = 1, stencil = 5;
    homg_options opt{};
    std::vector<int> sched;
    int exec = HOMG_EXEC_WHOLEGRID;
    bool strict = false;
    double omega = 0.2;
    int device = 0;
    cudaStream_t stream = nullptr;

    char* arena = nullptr;
    size_t arena_bytes = 0;
    int64_t pitch0 = 0;
    std::vector<Level> L;
    int geometry = HOMG_GEOM_NESTED;
    double* p2tmp = nullptr;  // power-of-two geometry: the restriction's row-pass buffer
    int prec = PREC_FP64;     // storage precision of the cycle arrays
    int nbatch = 1;           // problems laid out at pstride bytes from each other (batch groups)
    size_t pstride = 0;
    unsigned int* dticket = nullptr;  // batch finalize: arrivals, cycles run, stage base
    double* uint_[2] = {nullptr, nullptr};
    void* e[2] = {nullptr, nullptr};
    double* part_r = nullptr;
    double* part_f = nullptr;
    int nparts = 0;
    State* dstate = nullptr;
    double* dhist = nullptr;
    cudaGraphConditionalHandle* dhandles = nullptr;

    State* hstate = nullptr;  // pinned
    double* hhist = nullptr;  // pinned

    std::vector<Op> partA, partB;  // cycle parts (A: restriction + levels >= 1, B: level 0)
    std::vector<BlockOp> block_ops; // coarse-lattice ops run by one block (fast lattice form)
    BlockOp* dblock_ops = nullptr;
    int e_final = 0;               // index of e[] holding the cycle's result (whole-grid form)
    int fine_iters = 0, coarse_iters = 0;

    SolveGraph gfirst;            // initial residual + up to kStagesPerGraph cycle stages
    SolveGraph gcont;             // continuation: further stages, launched while cycles remain
    std::vector<cudaEvent_t> sev; // events of the stream launch mode

    double* stage_f = nullptr;  // homg_solve_host staging
    double* stage_u = nullptr;

    // Variable coefficients (homg_set_coefficient): per level the east/north face coefficients and
    // Jacobi weights in the cycle's coefficient type, and the FP64 level-0 faces of the residual.
    bool vc = false;
    char* vc_arena = nullptr;
    std::vector<void*> vkx, vky, vwd;
    double* kx0 = nullptr;
    double* ky0 = nullptr;
    int* dbad = nullptr;
    uint16_t* logk = nullptr;  // bfloat16(log k) per node, the learned corrector's second input

    // Learned solve (homg_solve_learned / homg_features): network input image and output, the
    // proposal's correction and residual source, partial sums and device scalars.
    char* learn_arena = nullptr;
    void* lx = nullptr;
    float* ly = nullptr;
    void* lcorr = nullptr;
    void* lg0 = nullptr;
    double* lpart = nullptr;
    double* lpart2 = nullptr;
    double* lscal = nullptr;  // [0] rho, [1] ||r||^2, [2] ||r'||^2
    int learn_judge = HOMG_JUDGE_PROPOSAL;
    double* lu2 = nullptr;    // judged after the cycle: third FP64 iterate, saved source, partials
    void* lgs = nullptr;
    double* lpart3 = nullptr;

    homg_stats stats{};
    char err[512] = "";
};

namespace {

int fail(homg_ctx* h, int code, const char* fmt, const char* what = "", const char* extra = "") {
    char* dst = h ? h->err : g_create_error;
    snprintf(dst, 512, fmt, what, extra);
    return code;
}

int cuda_fail(homg_ctx* h, cudaError_t e, const char* where) {
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? HOMG_ENOMEM : HOMG_ECUDA, "CUDA error in %s: %s", where,
                cudaGetErrorString(e));
}

#define CK(h, call, where)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

// Default MFMG schedule (Sec. 2, MFMG paragraph): coarsest first, 2 iterations, doubling, MaxI cap.
std::vector<int> mfmg(int levels, int max_i) {
    std::vector<int> s;
    for (int m = levels - 1; m >= 0; --m) {
        long long nm = 2;
        for (int t = 0; t < levels - 1 - m && nm < max_i; ++t) nm *= 2;
        nm = std::min<long long>(nm, max_i);
        for (long long t = 0; t < nm; ++t) s.push_back(m);
    }
    return s;
}

CGrid cgrid(const void* p, int64_t pitch, int n) { return CGrid{p, pitch, n}; }
Grid grid(void* p, int64_t pitch, int n) { return Grid{p, pitch, n}; }
CDGrid cdgrid(const double* p, int64_t pitch, int n) { return CDGrid{p, pitch, n}; }
DGrid dgrid(double* p, int64_t pitch, int n) { return DGrid{p, pitch, n}; }

// Lay out every array in one buffer: returns bytes needed; assigns pointers when base != nullptr.
// The per-problem arrays form one block, repeated nbatch times pstride bytes apart (pointers refer to
// problem 0); the cycle states, histories, coarse-lattice op list and batch counters follow.
size_t layout(homg_ctx* h, char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        off = (size_t)round_up((int64_t)off, 256);
        void* p = base ? (void*)(base + off) : nullptr;
        off += bytes;
        return p;
    };
    const int nd = h->ndim;
    const size_t es = (size_t)prec_bytes(h->prec);
    const bool lattice = (h->exec == HOMG_EXEC_LATTICE);
    const bool vcyc = (h->opt.cycle == HOMG_CYCLE_V);
    const bool pow2 = (h->geometry == HOMG_GEOM_POW2);
    for (int m = 0; m < h->levels; ++m) {
        if (pow2) {  // four quadrant arrays per level m >= 1; level 0 only holds the fine source
            Level& lv = h->L[m];
            const int qn = (m == 0) ? 1 : 4;
            const size_t bytes = (size_t)qn * (size_t)grid_elems(nd, lv.n, lv.pitch) * es;
            lv.g = take(bytes);
            if (m >= 1) {
                lv.d[0] = take(bytes);
                lv.d[1] = take(bytes);
            }
            continue;
        }
        Level& lv = h->L[m];
        const size_t bytes = (size_t)grid_elems(nd, lv.n, lv.pitch) * es;
        lv.g = take(bytes);
        if (vcyc) {
            if (m >= 1) {
                lv.G[0] = take(bytes);
                lv.G[1] = take(bytes);
            }
            lv.d[0] = take(bytes);
        } else if (m >= 1) {
            if (lattice) {
                lv.G[0] = take(bytes);
                lv.G[1] = take(bytes);
                lv.d[0] = take(bytes);
            } else {
                lv.d[0] = take(bytes);
                lv.d[1] = take(bytes);
            }
        }
    }
    const size_t fine_lp = (size_t)grid_elems(nd, h->n, h->pitch0) * es;
    const size_t fine64 = (size_t)grid_elems(nd, h->n, h->pitch0) * sizeof(double);
    h->e[0] = take(fine_lp);
    h->e[1] = take(fine_lp);
    h->uint_[0] = (double*)take(fine64);
    h->uint_[1] = (double*)take(fine64);
    h->L[0].G[0] = h->e[0];
    h->L[0].G[1] = h->e[1];
    h->part_r = (double*)take((size_t)h->nparts * sizeof(double));
    h->part_f = (double*)take((size_t)h->nparts * sizeof(double));
    if (pow2 && h->levels > 1) h->p2tmp = (double*)take((size_t)(h->n + 1) * 2 * (size_t)(h->L[1].n + 1) * sizeof(double));
    h->pstride = (size_t)round_up((int64_t)off, 256);
    off = h->pstride * (size_t)h->nbatch;
    h->dstate = (State*)take((size_t)h->nbatch * sizeof(State));
    h->dhist = (double*)take((size_t)h->nbatch * (HOMG_MAX_CYCLES + 1) * sizeof(double));
    h->dblock_ops = (BlockOp*)take(kMaxBlockOps * sizeof(BlockOp));
    h->dticket = (unsigned int*)take(4 * sizeof(unsigned int));
    return (size_t)round_up((int64_t)off, 256);
}

// Batch groups: give every planned array its per-problem stride and every op the problem count
// and the per-problem states (problem z of a launch = blockIdx.z).
void apply_batch(homg_ctx* h) {
    if (h->nbatch <= 1) return;
    const int64_t sl = (int64_t)(h->pstride / (size_t)prec_bytes(h->prec));
    auto g = [&](auto& grid_) { grid_.bstride = sl; };
    auto fix_it = [&](IterArgs& a) { g(a.e_old); g(a.e_new); g(a.g); g(a.dprev); g(a.dnew); a.nb = h->nbatch; a.bst = h->dstate; };
    auto fix_pr = [&](ProlongArgs& a) { g(a.G); g(a.Gc); g(a.dl); a.nb = h->nbatch; a.bst = h->dstate; };
    auto fix_rs = [&](RestrictArgs& a) { g(a.gf); g(a.gc); a.nb = h->nbatch; a.bst = h->dstate; };
    for (auto* part : {&h->partA, &h->partB})
        for (Op& op : *part) {
            if (op.kind == Op::ITER || op.kind == Op::ITER2) fix_it(op.it);
            else if (op.kind == Op::PROLONG) fix_pr(op.pr);
            else if (op.kind == Op::RUN) { fix_it(op.it); fix_pr(op.pr); }
            else if (op.kind == Op::RESTRICT) fix_rs(op.rs);
        }
    for (BlockOp& b : h->block_ops) {
        if (b.kind == BLOCK_ITER) fix_it(b.it);
        else if (b.kind == BLOCK_PROLONG) fix_pr(b.pr);
        else fix_rs(b.rs);
    }
}

// Damped-Jacobi scalars of an iteration, computed once on the host (binary32 copies for the
// binary32-arithmetic kernels).
void set_weights(const homg_ctx* h, IterArgs& a) {
    a.omega = h->omega;
    a.c1 = 1.0 - 2.0 * h->ndim * h->omega;
    a.omega_f = (float)a.omega;
    a.c1_f = (float)a.c1;
}

// V(v_pre, v_post) cycle on A e = F0 from e = 0 (Sec. 2 steps (a)-(e), recursively). Part A holds
// everything up to the level-0 post-smoothing, part B the level-0 post-smoothing sweeps.
void plan_vcycle(homg_ctx* h) {
    h->partA.clear();
    h->partB.clear();
    const int M = h->levels - 1;
    const int nu1 = h->opt.v_pre, nu2 = h->opt.v_post;
    std::vector<int> cur(h->levels, 0);
    int iters = 0;
    auto sweep = [&](int m, bool from_zero, double omega, std::vector<Op>& out) {
        Level& lv = h->L[m];
        Op op{};
        op.kind = Op::ITER;
        IterArgs& a = op.it;
        a.e_old = from_zero ? cgrid(nullptr, lv.pitch, lv.n) : cgrid(lv.G[cur[m]], lv.pitch, lv.n);
        a.e_new = grid(lv.G[cur[m] ^ 1], lv.pitch, lv.n);
        a.g = cgrid(lv.g, lv.pitch, lv.n);
        a.m = 0;
        a.mp = -1;
        a.omega = omega;
        a.c1 = 1.0 - 2.0 * h->ndim * omega;
        a.omega_f = (float)a.omega;
        a.c1_f = (float)a.c1;
        a.dnew = grid(nullptr, 0, 0);
        out.push_back(op);
        cur[m] ^= 1;
        ++iters;
    };
    const double omega_c = 1.0 / (2.0 * h->ndim);
    for (int m = 0; m < M; ++m) {
        Level& lv = h->L[m];
        for (int s = 0; s < nu1; ++s) sweep(m, s == 0, h->omega, h->partA);
        Op r{};
        r.kind = Op::VRESID;
        r.vr.e = cgrid(lv.G[cur[m]], lv.pitch, lv.n);
        r.vr.g = cgrid(lv.g, lv.pitch, lv.n);
        r.vr.rho = grid(lv.d[0], lv.pitch, lv.n);
        r.vr.omega = h->omega;
        h->partA.push_back(r);
        Op rs{};
        rs.kind = Op::RESTRICT;
        rs.rs.gf = cgrid(lv.d[0], lv.pitch, lv.n);
        rs.rs.gc = grid(h->L[m + 1].g, h->L[m + 1].pitch, h->L[m + 1].n);
        // fast forms keep sources as omega h^2 F; the coarsest level relaxes with omega_c
        rs.rs.scale = (m + 1 == M) ? omega_c / h->omega : 1.0;
        h->partA.push_back(rs);
    }
    {
        const int nm = h->L[M].n;
        const long long sweeps = std::max<long long>(1, (long long)nm * nm);
        for (long long s = 0; s < sweeps; ++s) sweep(M, s == 0, omega_c, h->partA);
    }
    for (int m = M - 1; m >= 0; --m) {
        Level& lv = h->L[m];
        Op pa{};
        pa.kind = Op::PROLONG_ADD;
        pa.pa.e = grid(lv.G[cur[m]], lv.pitch, lv.n);  // written by this cycle's pre-smoothing (v_pre >= 1)
        pa.pa.ec = cgrid(h->L[m + 1].G[cur[m + 1]], h->L[m + 1].pitch, h->L[m + 1].n);
        h->partA.push_back(pa);
        for (int s = 0; s < nu2; ++s) sweep(m, false, h->omega, m == 0 ? h->partB : h->partA);
    }
    h->e_final = cur[0];
    h->fine_iters = (M >= 1) ? nu2 : 0;
    h->coarse_iters = iters - h->fine_iters;
    h->sched.assign(iters, 0);
}

// Power-of-two geometry (whole-grid form): part A = restriction of every level m >= 1 from the
// fine source (hat stencil, two passes) and the iterations on levels >= 1; part B = the level-0
// iterations (the first one also interpolates the pending level; the others are plain sweeps run by
// the marching Jacobi kernel).
void plan_pow2(homg_ctx* h) {
    h->partA.clear();
    h->partB.clear();
    const int N = h->n + 1;
    auto qs = [&](int m) { return (int64_t)grid_elems(2, h->L[m].n, h->L[m].pitch); };
    for (int m = 1; m < h->levels; ++m) {
        Op op{};
        op.kind = Op::POW2_RESTRICT;
        op.p2r.N = N;
        op.p2r.m = m;
        op.p2r.g0 = cgrid(h->L[0].g, h->pitch0, h->n);
        op.p2r.tmp = h->p2tmp;
        op.p2r.gm = grid(h->L[m].g, h->L[m].pitch, h->L[m].n);
        op.p2r.gm.bstride = qs(m);
        h->partA.push_back(op);
    }
    const std::vector<int>& s = h->sched;
    const int T = (int)s.size();
    int tail = T;
    while (tail > 0 && s[tail - 1] == 0) --tail;
    h->fine_iters = T - tail;
    h->coarse_iters = tail;
    int cur = 0, mprev = -1;
    int dpar[32] = {0};
    for (int t = 0; t < T; ++t) {
        const int m = s[t];
        Op op{};
        const bool plain = (m == 0 && mprev <= 0 && t > 0);
        if (plain) {
            op.kind = Op::ITER;
            IterArgs& a = op.it;
            a.e_old = cgrid(h->e[cur], h->pitch0, h->n);
            a.e_new = grid(h->e[cur ^ 1], h->pitch0, h->n);
            a.g = cgrid(h->L[0].g, h->pitch0, h->n);
            a.m = 0;
            a.mp = -1;
            a.dnew = grid(nullptr, 0, 0);
            set_weights(h, a);
        } else {
            op.kind = Op::POW2_ITER;
            Pow2IterArgs& a = op.p2;
            a.N = N;
            a.m = m;
            a.mp = (mprev >= 1) ? mprev : -1;
            a.e_old = (t == 0) ? cgrid(nullptr, h->pitch0, h->n) : cgrid(h->e[cur], h->pitch0, h->n);
            a.e_new = grid(h->e[cur ^ 1], h->pitch0, h->n);
            if (m == 0) {
                a.g = cgrid(h->L[0].g, h->pitch0, h->n);
                a.dnew = grid(nullptr, 0, 0);
            } else {
                a.g = cgrid(h->L[m].g, h->L[m].pitch, h->L[m].n);
                a.g.bstride = qs(m);
                a.dnew = grid(h->L[m].d[dpar[m]], h->L[m].pitch, h->L[m].n);
                a.dnew.bstride = qs(m);
            }
            if (a.mp >= 1) {
                const Level& lp = h->L[mprev];
                a.dprev = cgrid(lp.d[dpar[mprev] ^ 1], lp.pitch, lp.n);
                a.dprev.bstride = qs(mprev);
            }
            a.omega = h->omega;
            a.c1 = 1.0 - 4.0 * h->omega;
            a.omega_f = (float)a.omega;
            a.c1_f = (float)a.c1;
        }
        if (m >= 1) dpar[m] ^= 1;
        (t < tail ? h->partA : h->partB).push_back(op);
        cur ^= 1;
        mprev = m;
    }
    h->e_final = cur;
}

// Kernel sequence of one cycle's parts A (restriction + levels >= 1) and B (level 0).
void plan_cycle(homg_ctx* h) {
    if (h->opt.cycle == HOMG_CYCLE_V) {
        plan_vcycle(h);
        return;
    }
    if (h->geometry == HOMG_GEOM_POW2) {
        plan_pow2(h);
        return;
    }
    h->partA.clear();
    h->partB.clear();
    const int nd = h->ndim;
    (void)nd;
    for (int m = 1; m < h->levels; ++m) {
        Op op{};
        op.kind = Op::RESTRICT;
        op.rs.gf = cgrid(h->L[m - 1].g, h->L[m - 1].pitch, h->L[m - 1].n);
        op.rs.gc = grid(h->L[m].g, h->L[m].pitch, h->L[m].n);
        op.rs.scale = 1.0;
        h->partA.push_back(op);
    }
    const std::vector<int>& s = h->sched;
    const int T = (int)s.size();
    int tail = T;  // first index of the trailing run of level-0 iterations
    while (tail > 0 && s[tail - 1] == 0) --tail;
    h->fine_iters = T - tail;
    h->coarse_iters = tail;
    if (h->exec == HOMG_EXEC_WHOLEGRID) {
        int cur = 0;  // e[cur] holds the current iterate
        int mprev = -1;
        int dpar[32] = {0};
        for (int t = 0; t < T; ++t) {
            const int m = s[t];
            Op op{};
            op.kind = Op::ITER;
            IterArgs& a = op.it;
            a.e_old = (t == 0) ? cgrid(nullptr, h->pitch0, h->n) : cgrid(h->e[cur], h->pitch0, h->n);
            a.e_new = grid(h->e[cur ^ 1], h->pitch0, h->n);
            a.g = cgrid(h->L[m].g, h->L[m].pitch, h->L[m].n);
            a.m = m;
            set_weights(h, a);
            a.mp = -1;
            if (mprev >= 1) {
                a.mp = mprev;
                const Level& lp = h->L[mprev];
                a.dprev = cgrid(lp.d[dpar[mprev] ^ 1], lp.pitch, lp.n);
            }
            a.dnew = grid(nullptr, 0, 0);
            if (m >= 1) {
                a.dnew = grid(h->L[m].d[dpar[m]], h->L[m].pitch, h->L[m].n);
                dpar[m] ^= 1;
            }
            (t < tail ? h->partA : h->partB).push_back(op);
            cur ^= 1;
            mprev = m;
        }
        h->e_final = cur;
    } else {
        // Lattice form: runs of equal levels, never increasing.
        int t = 0, mprev = -1;
        int e_cur = 0;
        while (t < T) {
            const int m = s[t];
            int c = 0;
            while (t + c < T && s[t + c] == m) ++c;
            Level& lv = h->L[m];
            int cur = 0;
            const bool first_run = (mprev < 0);
            if (!first_run) {
                const Level& lc = h->L[mprev];
                Op op{};
                op.kind = Op::PROLONG;
                op.pr.G = grid(lv.G[0], lv.pitch, lv.n);
                op.pr.Gc = cgrid(lc.G[e_cur], lc.pitch, lc.n);
                op.pr.dl = cgrid(lc.d[0], lc.pitch, lc.n);
                op.pr.s = mprev - m;
                h->partA.push_back(op);
            }
            // binary32-arithmetic cycles pair consecutive plain sweeps (no pending interpolation, no
            // variation output) into one two-sweep launch: half the DRAM traffic, same results
            const bool pairable = !h->strict && h->prec != PREC_FP64 && !h->vc &&
                                  ((h->ndim == 2 && lv.n > 16) || (h->ndim == 3 && lv.n > 8));
            auto plain = [&](int q) { return q >= 1 && !(q == c - 1 && m >= 1); };
            for (int q = 0; q < c; ++q) {
                if (pairable && plain(q) && q + 1 < c && plain(q + 1)) {
                    // batches: four sweeps where the run allows (their launches cover every problem of
                    // the group, where the halved traffic outweighs the longer march); otherwise two
                    const int k = (h->nbatch > 1 && q + 3 < c && plain(q + 3)) ? 4 : 2;
                    Op op{};
                    op.kind = Op::ITER2;
                    op.sweeps = k;
                    IterArgs& a = op.it;
                    a.e_old = cgrid(lv.G[cur], lv.pitch, lv.n);
                    a.e_new = grid(lv.G[cur ^ 1], lv.pitch, lv.n);
                    a.g = cgrid(lv.g, lv.pitch, lv.n);
                    a.m = 0;
                    set_weights(h, a);
                    a.mp = -1;
                    a.dnew = grid(nullptr, 0, 0);
                    // large single-problem lattices: the two sweeps with the tile staged by TMA
                    if (k == 2 && h->nbatch == 1 && h->opt.tma_min_n > 0 && lv.n >= h->opt.tma_min_n &&
                        (h->ndim == 2 ? tma_sweep_maps(h->prec, a, &op.maps) : tma_sweep_maps3(h->prec, a, &op.maps)) ==
                            cudaSuccess)
                        op.tma = true;
                    (m == 0 ? h->partB : h->partA).push_back(op);
                    cur ^= 1;
                    q += k - 1;
                    continue;
                }
                Op op{};
                op.kind = Op::ITER;
                IterArgs& a = op.it;
                a.e_old = (first_run && q == 0) ? cgrid(nullptr, lv.pitch, lv.n) : cgrid(lv.G[cur], lv.pitch, lv.n);
                a.e_new = grid(lv.G[cur ^ 1], lv.pitch, lv.n);
                a.g = cgrid(lv.g, lv.pitch, lv.n);
                a.m = 0;
                set_weights(h, a);
                a.mp = -1;
                if (q == 0 && !first_run) {
                    const Level& lc = h->L[mprev];
                    a.mp = mprev - m;
                    a.dprev = cgrid(lc.d[0], lc.pitch, lc.n);
                }
                a.dnew = grid(nullptr, 0, 0);
                if (q == c - 1 && m >= 1) a.dnew = grid(lv.d[0], lv.pitch, lv.n);
                if (h->vc) {
                    a.kx = h->vkx[m];
                    a.ky = h->vky[m];
                    a.wd = h->vwd[m];
                    a.kpitch = lv.pitch;
                }
                (m == 0 ? h->partB : h->partA).push_back(op);
                cur ^= 1;
            }
            e_cur = cur;
            mprev = m;
            t += c;
        }
        h->e_final = e_cur;
    }
}

// Lattice form, binary32 cycles (2-D): each level run after the coarsest ones -- a stride-1 level
// change, then the level's sweeps, the first with the pending stride-2 interpolation -- on a lattice
// of at most opt.run_max_n intervals per side becomes one RUN op (k_level_run2: one block per
// problem, the lattice in shared memory). Level 0's sweeps (part B) stay separate launches.
void group_level_runs(homg_ctx* h) {
    if (h->opt.run_max_n <= 0 || h->strict || h->exec != HOMG_EXEC_LATTICE ||
        h->opt.cycle == HOMG_CYCLE_V || h->vc || h->ndim != 2 || h->geometry != HOMG_GEOM_NESTED ||
        h->prec == PREC_FP64)
        return;
    std::vector<Op> out;
    const std::vector<Op>& A = h->partA;
    for (size_t q = 0; q < A.size();) {
        const Op& op = A[q];
        const int n = (op.kind == Op::PROLONG) ? op.pr.G.n : 0;
        size_t r = q + 1;
        int sweeps = 0;
        if (op.kind == Op::PROLONG && op.pr.s == 1 && n >= 2 && n <= h->opt.run_max_n) {
            while (r < A.size() && (A[r].kind == Op::ITER || A[r].kind == Op::ITER2) && A[r].it.e_new.n == n) {
                sweeps += A[r].kind == Op::ITER2 ? A[r].sweeps : 1;
                ++r;
            }
        }
        const bool fuse = sweeps >= 1 && A[q + 1].kind == Op::ITER && A[q + 1].it.mp == 1 &&
                          A[q + 1].it.dprev.p == op.pr.dl.p;
        if (!fuse) {
            out.push_back(op);
            ++q;
            continue;
        }
        Op run{};
        run.kind = Op::RUN;
        run.sweeps = sweeps;
        run.pr = op.pr;
        run.it = A[r - 1].it;              // the last sweep's output: the run's final buffer and variation
        run.it.e_old = A[q + 1].it.e_old;  // not read (the level change fills shared memory)
        run.it.g = A[q + 1].it.g;
        run.it.mp = 1;
        run.it.dprev = A[q + 1].it.dprev;
        out.push_back(run);
        q = r;
    }
    h->partA = out;
}

// Fast lattice form: the restrictions to, and the leading runs on, the coarsest lattices (at most
// 16 intervals per side in 2-D, 8 in 3-D: a few hundred nodes, less than one per thread of the
// block) become one single-block launch. Larger lattices run faster as separate launches (or, in
// binary32 cycles, as one shared-memory launch per level run: group_level_runs).
void group_block_ops(homg_ctx* h) {
    h->block_ops.clear();
    if (h->strict || h->exec != HOMG_EXEC_LATTICE || h->opt.cycle == HOMG_CYCLE_V || h->vc) return;
    const int nb = (h->ndim == 2) ? 16 : 8;
    std::vector<Op> kept;
    std::vector<BlockOp> blk;
    size_t q = 0;
    // restrictions: the ones producing small lattices (they come last, coarsest)
    for (; q < h->partA.size() && h->partA[q].kind == Op::RESTRICT; ++q) {
        const Op& op = h->partA[q];
        if (op.rs.gc.n <= nb) {
            BlockOp b{};
            b.kind = BLOCK_RESTRICT;
            b.rs = op.rs;
            blk.push_back(b);
        } else {
            kept.push_back(op);
        }
    }
    // leading iterations / level changes on small lattices
    for (; q < h->partA.size(); ++q) {
        const Op& op = h->partA[q];
        if (op.kind != Op::ITER && op.kind != Op::PROLONG) break;
        const int n = (op.kind == Op::ITER) ? op.it.e_new.n : op.pr.G.n;
        if (n > nb) break;
        BlockOp b{};
        if (op.kind == Op::ITER) { b.kind = BLOCK_ITER; b.it = op.it; }
        else { b.kind = BLOCK_PROLONG; b.pr = op.pr; }
        blk.push_back(b);
    }
    if (blk.empty() || (int)blk.size() > kMaxBlockOps) return;
    Op bop{};
    bop.kind = Op::BLOCK;
    bop.block_first = 0;
    bop.block_count = (int)blk.size();
    kept.push_back(bop);
    for (; q < h->partA.size(); ++q) kept.push_back(h->partA[q]);
    h->partA = kept;
    h->block_ops = blk;
}

void group_coarse_block(homg_ctx* h) {
    group_block_ops(h);
    group_level_runs(h);
}

cudaError_t enqueue_ops(homg_ctx* h, const std::vector<Op>& ops, cudaStream_t s) {
    for (const Op& op : ops) {
        cudaError_t e = cudaSuccess;
        switch (op.kind) {
            case Op::ITER: e = launch_iterate(h->ndim, h->prec, h->strict, op.it, s); break;
            case Op::ITER2:
                e = op.tma ? (h->ndim == 3 ? launch_iterate3_2_tma(h->prec, op.it, op.maps, &h->dstate->fault, s)
                                           : launch_iterate2_tma(h->prec, op.it, op.maps, &h->dstate->fault, s))
                    : (h->ndim == 3) ? launch_iterate3_2(h->prec, op.it, s)
                                     : launch_iterate2(h->prec, op.sweeps, op.it, s);
                break;
            case Op::PROLONG: e = launch_prolong(h->ndim, h->prec, h->strict, op.pr, s); break;
            case Op::RESTRICT: e = launch_restrict(h->ndim, h->prec, h->strict, op.rs, s); break;
            case Op::VRESID: e = launch_vresid(h->ndim, h->prec, h->strict, op.vr, s); break;
            case Op::PROLONG_ADD: e = launch_prolong_add(h->ndim, h->prec, h->strict, op.pa, s); break;
            case Op::POW2_ITER: e = launch_pow2_iterate(h->prec, op.p2, s); break;
            case Op::POW2_RESTRICT: e = launch_pow2_restrict(h->prec, op.p2r, s); break;
            case Op::BLOCK:
                e = launch_coarse_block(h->ndim, h->prec, h->dblock_ops + op.block_first, op.block_count, h->nbatch, s);
                break;
            case Op::RUN: e = launch_level_run(h->prec, op.pr, op.it, op.sweeps, h->nbatch, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

ResidArgs resid_args(homg_ctx* h, int stage) {
    ResidArgs a{};
    a.st = h->dstate;
    const double hh = 1.0 / (double)h->n;
    a.inv_h2 = (double)h->n * (double)h->n;
    a.scale = h->strict ? hh * hh : h->omega * hh * hh;  // fast mode stores omega h^2 F
    if (h->vc) {  // variable coefficients: h^2 F (each node applies its own weight)
        a.scale = hh * hh;
        a.kx = h->kx0;
        a.ky = h->ky0;
        a.kpitch = h->pitch0;
    }
    a.scale_f = (float)a.scale;
    a.part_r = h->part_r;
    a.part_f = nullptr;
    a.g0 = grid(h->L[0].g, h->L[0].pitch, h->n);
    if (stage == 0) {
        a.u_in = cdgrid(nullptr, 0, h->n);
        a.e = cgrid(nullptr, 0, h->n);
        a.u_out = dgrid(h->uint_[0], h->pitch0, h->n);
        a.part_f = h->part_f;
    } else {
        a.u_in = cdgrid(h->uint_[(stage - 1) & 1], h->pitch0, h->n);
        a.e = cgrid(h->e[h->e_final], h->pitch0, h->n);
        a.u_out = dgrid(h->uint_[stage & 1], h->pitch0, h->n);
    }
    if (h->nbatch > 1) {
        const int64_t s64 = (int64_t)(h->pstride / sizeof(double)), slp = (int64_t)(h->pstride / prec_bytes(h->prec));
        a.batch = 1;
        a.nb = h->nbatch;
        a.u_in.bstride = s64;
        a.u_out.bstride = s64;
        a.e.bstride = slp;
        a.g0.bstride = slp;
        a.part_bstride = s64;
    }
    return a;
}

CopyOutArgs copy_args(homg_ctx* h) {
    CopyOutArgs c{};
    c.st = h->dstate;
    c.u0 = cdgrid(h->uint_[0], h->pitch0, h->n);
    c.u1 = cdgrid(h->uint_[1], h->pitch0, h->n);
    if (h->nbatch > 1) {
        c.batch = 1;
        c.nb = h->nbatch;
        c.u0.bstride = c.u1.bstride = (int64_t)(h->pstride / sizeof(double));
    }
    return c;
}

FinalizeArgs fin_args(homg_ctx* h, int mode, const SolveGraph* g) {
    FinalizeArgs f{};
    f.st = h->dstate;
    f.hist = h->dhist;
    f.part_r = h->part_r;
    f.part_f = (mode == FIN_CYCLE) ? nullptr : h->part_f;
    f.nparts = h->nparts;
    f.mode = mode;
    f.handles = g ? g->dhandles : nullptr;
    f.nstages = g ? g->stages : 0;
    if (h->nbatch > 1) {
        f.batch = h->nbatch;
        f.hist_bstride = HOMG_MAX_CYCLES + 1;
        f.part_bstride = (int64_t)(h->pstride / sizeof(double));
        f.ticket = h->dticket;
    }
    return f;
}

void destroy_graph(SolveGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (cudaEvent_t e : g.ev) cudaEventDestroy(e);
    g.ev.clear();
    if (g.dhandles) cudaFree(g.dhandles);
    g.dhandles = nullptr;
    g.stages = 0;
}

// Capture `fn(stream)` into the body graph `body` (or a fresh graph when body == nullptr).
template <typename Fn>
cudaError_t capture_into(cudaGraph_t body, cudaStream_t cap, Fn fn, cudaGraph_t* out) {
    cudaError_t e = body ? cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)
                         : cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t le = fn(cap);
    cudaGraph_t g = body;
    e = cudaStreamEndCapture(cap, &g);
    if (le != cudaSuccess) return le;
    if (out) *out = g;
    return e;
}

// Event layout: ev[0] at the start, ev[1] after the initial residual (first graph only; the
// continuation graph records ev[0], ev[1] back to back); stage k records ev[3k-1] after part A,
// ev[3k] after part B, ev[3k+1] after part C; ev[3S+2] after the copy-out.
int build_graph(homg_ctx* h, SolveGraph& G, int stages, bool with_init) {
    destroy_graph(G);
    std::vector<cudaGraphConditionalHandle> handles(3 * (stages + 1), 0);
    G.stages = stages;
    G.with_init = with_init;
    G.ev.assign(3 * stages + 3, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& ev : G.ev)
        if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaMalloc(&G.dhandles, handles.size() * sizeof(cudaGraphConditionalHandle));
    cudaStream_t cap = nullptr;
    cudaGraph_t top = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&top, 0);
    cudaGraphNode_t last = nullptr, node = nullptr;
    auto add_event = [&](int idx) -> cudaError_t {
        cudaError_t r = cudaGraphAddEventRecordNode(&node, top, last ? &last : nullptr, last ? 1 : 0, G.ev[idx]);
        if (r == cudaSuccess) last = node;
        return r;
    };
    // Append the kernels enqueued by fn directly to the top graph, after `last`.
    auto add_seq = [&](auto fn) -> cudaError_t {
        cudaError_t r = cudaStreamBeginCaptureToGraph(cap, top, last ? &last : nullptr, nullptr, last ? 1 : 0,
                                                      cudaStreamCaptureModeThreadLocal);
        if (r != cudaSuccess) return r;
        cudaError_t le = fn(cap);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaError_t qe = cudaStreamGetCaptureInfo(cap, &cs, nullptr, nullptr, &deps, nullptr, &nd);
        cudaGraphNode_t tail = (qe == cudaSuccess && nd == 1) ? deps[0] : nullptr;
        cudaGraph_t g = top;
        r = cudaStreamEndCapture(cap, &g);
        if (le != cudaSuccess) return le;
        if (qe != cudaSuccess) return qe;
        if (r != cudaSuccess) return r;
        if (!tail) return cudaErrorInvalidValue;
        last = tail;
        return cudaSuccess;
    };
    auto add_if = [&](int k, int part, auto fn) -> cudaError_t {
        cudaGraphConditionalHandle hd;
        // The first stage of the continuation graph runs whenever that graph is launched.
        const unsigned def = (!with_init && k == 1) ? 1u : 0u;
        cudaError_t r = cudaGraphConditionalHandleCreate(&hd, top, def, cudaGraphCondAssignDefault);
        if (r != cudaSuccess) return r;
        handles[3 * k + part] = hd;
        cudaGraphNodeParams p{};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = hd;
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        r = cudaGraphAddNode(&node, top, &last, nullptr, 1, &p);
        if (r != cudaSuccess) return r;
        last = node;
        return capture_into(p.conditional.phGraph_out[0], cap, fn, nullptr);
    };
    if (e == cudaSuccess) e = add_event(0);
    if (e == cudaSuccess && with_init)
        e = add_seq([&](cudaStream_t s) -> cudaError_t {
            cudaError_t r = launch_residual(h->ndim, h->prec, h->strict, resid_args(h, 0), h->n, s);
            if (r == cudaSuccess) r = launch_finalize(fin_args(h, FIN_INIT, &G), s);
            return r;
        });
    if (e == cudaSuccess) e = add_event(1);
    for (int k = 1; k <= stages && e == cudaSuccess; ++k) {
        e = add_if(k, 0, [&](cudaStream_t s) { return enqueue_ops(h, h->partA, s); });
        if (e == cudaSuccess) e = add_event(3 * k - 1);
        if (e == cudaSuccess) e = add_if(k, 1, [&](cudaStream_t s) { return enqueue_ops(h, h->partB, s); });
        if (e == cudaSuccess) e = add_event(3 * k);
        if (e == cudaSuccess)
            e = add_if(k, 2, [&](cudaStream_t s) -> cudaError_t {
                cudaError_t r = launch_residual(h->ndim, h->prec, h->strict, resid_args(h, k), h->n, s);
                if (r == cudaSuccess) r = launch_finalize(fin_args(h, FIN_CYCLE, &G), s);
                return r;
            });
        if (e == cudaSuccess) e = add_event(3 * k + 1);
    }
    if (e == cudaSuccess)
        e = add_seq([&](cudaStream_t s) -> cudaError_t { return launch_copy_out(h->ndim, copy_args(h), h->n, s); });
    if (e == cudaSuccess) e = add_event(3 * stages + 2);
    if (e == cudaSuccess)
        e = cudaMemcpy(G.dhandles, handles.data(), handles.size() * sizeof(handles[0]), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, top, 0);
    int rc = (e == cudaSuccess) ? HOMG_OK : cuda_fail(h, e, "building the solve graph");
    if (top) cudaGraphDestroy(top);
    if (cap) cudaStreamDestroy(cap);
    if (rc != HOMG_OK) destroy_graph(G);
    return rc;
}

double elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

// Per-part times of one graph launch, from its events (cycles [k0+1, k1] of the solve ran in it).
void add_graph_times(homg_stats& st, const std::vector<cudaEvent_t>& E, int local_cycles, int end_ev) {
    st.solve_ms += elapsed(E[0], E[end_ev]);
    for (int k = 1; k <= local_cycles; ++k) {
        st.coarse_ms += elapsed(E[3 * k - 2], E[3 * k - 1]);
        st.fine_ms += elapsed(E[3 * k - 1], E[3 * k]);
        st.residual_ms += elapsed(E[3 * k], E[3 * k + 1]);
    }
}

bool schedule_monotone(const std::vector<int>& s) {
    for (size_t t = 1; t < s.size(); ++t)
        if (s[t] > s[t - 1]) return false;
    return true;
}


}  // namespace

namespace homg {
void set_null_handle_error(const char* msg) { snprintf(g_create_error, sizeof(g_create_error), "%s", msg); }
}  // namespace homg

extern "C" {

void homg_default_options(homg_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->omega_j = 0.0;
    opt->max_i = 32;
    opt->exec_mode = HOMG_EXEC_AUTO;
    opt->diverge_factor = 1e3;
}

}  // extern "C"

namespace {

// Grid side n + 1 = 2^K + 1 with K >= 1 and within the maximum; returns K or a negative code.
int grid_exponent(int ndim, int64_t side, const char* who) {
    const int64_t n = side - 1;
    int K = 0;
    while (K < 62 && ((int64_t)1 << K) < n) ++K;
    if (n < 2 || ((int64_t)1 << K) != n) {
        char msg[160];
        snprintf(msg, sizeof(msg), "%s: grid side must be 2^K + 1 with K >= 1", who);
        return fail(nullptr, HOMG_ESHAPE, "%s%s", msg);
    }
    if (K > (ndim == 2 ? HOMG_MAX_K_2D : HOMG_MAX_K_3D)) {
        char msg[160];
        snprintf(msg, sizeof(msg), "%s: grid side above the supported maximum", who);
        return fail(nullptr, HOMG_ESHAPE, "%s%s", msg);
    }
    return K;
}

// Defaults and validation of the options (shared by the single and batch entry points).
int check_options(int ndim, homg_options& o) {
    if (o.omega_j == 0.0) o.omega_j = (ndim == 2) ? 4.0 / 5.0 : 6.0 / 7.0;
    if (o.max_i == 0) o.max_i = 32;
    if (o.run_max_n == 0) o.run_max_n = RUN_MAX_N;
    if (o.tma_min_n == 0) o.tma_min_n = HOMG_TMA_MIN_N_DEFAULT;
    if (o.tma_min_n > 0 && o.tma_min_n < XT_MIN_N) o.tma_min_n = XT_MIN_N;
    if (o.diverge_factor == 0.0) o.diverge_factor = 1e3;
    if (o.v_pre == 0) o.v_pre = 2;
    if (o.v_post == 0) o.v_post = 2;
    if (!(o.omega_j > 0.0 && o.omega_j <= 2.0) || o.max_i < 1 || !(o.diverge_factor > 1.0) || o.n_schedule < 0 ||
        (o.n_schedule > 0 && !o.schedule) || o.exec_mode < 0 || o.exec_mode > 2 || (o.strict_fp != 0 && o.strict_fp != 1) ||
        (o.launch_mode != HOMG_LAUNCH_GRAPH && o.launch_mode != HOMG_LAUNCH_STREAM &&
         o.launch_mode != HOMG_LAUNCH_PERSISTENT) ||
        (o.precision != HOMG_PREC_FP64 && o.precision != HOMG_PREC_FP32 && o.precision != HOMG_PREC_BF16) ||
        (o.cycle != HOMG_CYCLE_HOMG && o.cycle != HOMG_CYCLE_V) || o.v_pre < 0 || o.v_post < 0 || o.v_pre > 64 ||
        o.v_post > 64 || (o.cycle == HOMG_CYCLE_V && (o.n_schedule > 0 || o.exec_mode == HOMG_EXEC_WHOLEGRID)) ||
        (o.geometry != HOMG_GEOM_NESTED && o.geometry != HOMG_GEOM_POW2) || o.run_max_n > RUN_MAX_N)
        return fail(nullptr, HOMG_EINVAL, "homg_create: invalid options%s%s");
    if (o.geometry == HOMG_GEOM_POW2 &&
        (ndim != 2 || o.cycle != HOMG_CYCLE_HOMG || o.strict_fp || o.exec_mode == HOMG_EXEC_LATTICE))
        return fail(nullptr, HOMG_EINVAL,
                    "homg_create: power-of-two grids are 2-D HOMG cycles in the whole-grid fast form%s%s");
    return HOMG_OK;
}

// Build a solver context for nbatch equal-size problems (nbatch = 1: the single-problem handle).
int create_ctx(int ndim, int64_t n, int K, int levels, int stencil, const homg_options& o, int nbatch, homg_ctx** out) {
    *out = nullptr;
    homg_ctx* h = new (std::nothrow) homg_ctx();
    if (!h) return fail(nullptr, HOMG_ENOMEM, "homg_create: out of host memory%s%s");
    h->ndim = ndim;
    h->n = (int)n;
    h->K = K;
    h->levels = levels;
    h->stencil = stencil;
    h->opt = o;
    h->strict = (o.strict_fp == 1);
    h->prec = o.precision;
    h->geometry = o.geometry;
    h->nbatch = nbatch;
    h->omega = o.omega_j / (2.0 * ndim);
    if (o.n_schedule > 0) {
        h->sched.assign(o.schedule, o.schedule + o.n_schedule);
        for (int m : h->sched)
            if (m < 0 || m >= levels) {
                delete h;
                return fail(nullptr, HOMG_EINVAL, "homg_create: schedule level out of range%s%s");
            }
        if (h->sched.back() != 0) {
            delete h;
            return fail(nullptr, HOMG_EINVAL, "homg_create: schedule must end on level 0%s%s");
        }
        h->opt.schedule = nullptr;
    } else {
        h->sched = mfmg(levels, o.max_i);
    }
    if (o.cycle == HOMG_CYCLE_V && (n >> (levels - 1)) > 64) {
        delete h;
        return fail(nullptr, HOMG_EINVAL,
                    "homg_create: the V-cycle's coarsest level must have at most 64 intervals per side%s%s");
    }
    const bool mono = schedule_monotone(h->sched);
    if (o.exec_mode == HOMG_EXEC_LATTICE && !mono) {
        delete h;
        return fail(nullptr, HOMG_EINVAL, "homg_create: the lattice form needs a schedule whose levels never increase%s%s");
    }
    h->exec = (o.exec_mode == HOMG_EXEC_WHOLEGRID || !mono) ? HOMG_EXEC_WHOLEGRID : HOMG_EXEC_LATTICE;
    if (o.cycle == HOMG_CYCLE_V) h->exec = HOMG_EXEC_LATTICE;  // level arrays are compact by nature
    if (o.geometry == HOMG_GEOM_POW2) h->exec = HOMG_EXEC_WHOLEGRID;

    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) {
        int rc = cuda_fail(nullptr, ce, "cudaGetDevice");
        delete h;
        return rc;
    }
    h->pitch0 = round_up(n + 1, 16);
    h->L.resize(levels);
    for (int m = 0; m < levels; ++m) {
        // power-of-two grids: n + 1 = 2^K nodes; level m >= 1 holds quadrant lattices of n_m = 2^(K-1-m)
        h->L[m].n = (m == 0) ? (int)n : (o.geometry == HOMG_GEOM_POW2 ? (int)(((n + 1) / 2) >> m) : (int)(n >> m));
        h->L[m].pitch = (m == 0) ? h->pitch0 : round_up(h->L[m].n + 1, 16);
    }
    h->nparts = residual_blocks(ndim, h->strict, (int)n);
    h->arena_bytes = layout(h, nullptr);
    ce = cudaMalloc(&h->arena, h->arena_bytes);
    if (ce == cudaSuccess) ce = cudaMemset(h->arena, 0, h->arena_bytes);
    if (ce == cudaSuccess) ce = cudaMallocHost(&h->hstate, (size_t)nbatch * sizeof(State));
    if (ce == cudaSuccess) ce = cudaMallocHost(&h->hhist, (HOMG_MAX_CYCLES + 1) * sizeof(double));
    if (ce != cudaSuccess) {
        int rc = cuda_fail(nullptr, ce, "allocating the level buffer");
        homg_destroy(h);
        return rc;
    }
    layout(h, h->arena);
    plan_cycle(h);
    group_coarse_block(h);
    apply_batch(h);
    ce = prepare_level_run(h->prec);
    if (ce != cudaSuccess) {
        int rc = cuda_fail(nullptr, ce, "setting the level-run kernel's shared memory");
        homg_destroy(h);
        return rc;
    }
    if (!h->block_ops.empty()) {
        ce = cudaMemcpy(h->dblock_ops, h->block_ops.data(), h->block_ops.size() * sizeof(BlockOp), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            int rc = cuda_fail(nullptr, ce, "copying the coarse-lattice op list");
            homg_destroy(h);
            return rc;
        }
    }
    *out = h;
    return HOMG_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {
int autotune_rows(homg_ctx* h, cudaStream_t st, int* best_rows, double* best_us, double min_nodes = 0.0);
}

extern "C" {

int homg_create(int ndim, const int64_t* dims, int levels, int stencil, const homg_options* opt, homg_handle* out) {
    if (out) *out = nullptr;
    g_create_error[0] = 0;
    if (!out || !dims) return fail(nullptr, HOMG_EINVAL, "homg_create: null %s%s", !out ? "out" : "dims");
    if (ndim != 2 && ndim != 3) return fail(nullptr, HOMG_EINVAL, "homg_create: ndim must be 2 or 3%s%s");
    if ((ndim == 2 && stencil != 5) || (ndim == 3 && stencil != 7))
        return fail(nullptr, HOMG_EINVAL, "homg_create: stencil must be 5 (2-D) or 7 (3-D)%s%s");
    for (int d = 1; d < ndim; ++d)
        if (dims[d] != dims[0]) return fail(nullptr, HOMG_ESHAPE, "homg_create: grid sides must be equal%s%s");
    homg_options o;
    homg_default_options(&o);
    if (opt) o = *opt;
    int K;
    if (o.geometry == HOMG_GEOM_POW2) {
        K = 0;
        while (K < 62 && ((int64_t)1 << K) < dims[0]) ++K;
        if (dims[0] < 4 || ((int64_t)1 << K) != dims[0] || K > HOMG_MAX_K_2D)
            return fail(nullptr, HOMG_ESHAPE, "homg_create: power-of-two grid side must be 2^K with 2 <= K <= HOMG_MAX_K_2D%s%s");
    } else {
        K = grid_exponent(ndim, dims[0], "homg_create");
        if (K < 0) return K;
    }
    if (levels < 1 || levels > K) return fail(nullptr, HOMG_EINVAL, "homg_create: levels must be in [1, K]%s%s");
    int rc = check_options(ndim, o);
    if (rc != HOMG_OK) return rc;
    if (o.launch_mode == HOMG_LAUNCH_PERSISTENT)
        return fail(nullptr, HOMG_EINVAL, "homg_create: the persistent launch mode is for batches (homg_batch_create)%s%s");
    homg_ctx* h = nullptr;
    rc = create_ctx(ndim, dims[0] - 1, K, levels, stencil, o, 1, &h);
    if (rc != HOMG_OK) return rc;
    // fast 2-D lattice form: time the marching sweeps of the lattices of a million nodes or more
    // once, as the batches do (smaller sweeps are launch-latency bound, and timing them alone is
    // too noisy to beat the size heuristic)
    if (ndim == 2 && !h->strict && h->exec == HOMG_EXEC_LATTICE && h->geometry == HOMG_GEOM_NESTED) {
        int rows = 0;
        double us = 0.0;
        rc = autotune_rows(h, h->stream, &rows, &us, 1.0e6);
        if (rc != HOMG_OK) {
            set_null_handle_error(h->err);
            homg_destroy(h);
            return rc;
        }
    }
    *out = h;
    return HOMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched solves
// ---------------------------------------------------------------------------------------------
struct homg_batch_ctx {
    int nprob = 0;
    std::vector<int> group_of, index_in_group;
    std::vector<homg_ctx*> groups;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaStream_t stream = nullptr;
    homg_batch_stats stats{};
    unsigned int* hticket = nullptr;  // pinned, 4 per group: ticket counters read back after each launch
    // HOMG_LAUNCH_PERSISTENT: the program of the persistent kernel (items, phases, the groups' coarse
    // op lists) and its counters, in one device allocation
    bool persistent = false;
    int prec = PREC_FP64;
    char* parena = nullptr;
    PersistArgs pargs{};
    size_t nqueue = 0;
    int pblocks = 0;
    int* herr = nullptr;  // pinned: the kernel's barrier failure flag, read back after a launch
};

namespace {

// Autotuner: for every lattice size the group sweeps with the marching Jacobi kernels (single and
// fused sweeps separately; sizes of at least min_nodes nodes over all problems), time the plain
// sweep (all problems at once, 5 launches after 2 warm-ups) for each candidate number of nodes per
// thread along the march, keep the fastest, and use it for every sweep of that kind and size.
// Reports the level-0 choice of the single sweep (of the fused one when the level has no single
// plain sweep).
int autotune_rows(homg_ctx* h, cudaStream_t st, int* best_rows, double* best_us, double min_nodes) {
    *best_rows = 0;
    *best_us = 0.0;
    std::vector<const Op*> tmpl;
    for (auto* part : {&h->partA, &h->partB})
        for (const Op& op : *part) {
            const bool single = op.kind == Op::ITER && op.it.e_old.p;
            if ((!single && op.kind != Op::ITER2) || op.it.m != 0 || op.tma) continue;
            const double nodes = (double)h->nbatch * (double)(op.it.e_new.n - 1) * (double)(op.it.e_new.n - 1);
            if (nodes < min_nodes) continue;
            bool seen = false;
            for (const Op* t : tmpl) seen |= t->kind == op.kind && t->sweeps == op.sweeps && t->it.e_new.n == op.it.e_new.n;
            if (!seen) tmpl.push_back(&op);
        }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(h, cudaEventCreate(&e0), "cudaEventCreate");
    if (cudaError_t ce = cudaEventCreate(&e1); ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(h, ce, "cudaEventCreate");
    }
    bool level0_single = false;
    for (const Op* t : tmpl) {
        const Op::Kind kind = t->kind;
        const int sweeps = t->sweeps;
        IterArgs a = t->it;
        a.mp = -1;
        a.dnew = Grid{nullptr, 0, 0};
        const int n = a.e_new.n;
        auto launch = [&]() {
            return kind == Op::ITER2 ? launch_iterate2(h->prec, sweeps, a, st) : launch_iterate(h->ndim, h->prec, false, a, st);
        };
        double best = 1e30;
        int pick = 0;
        static const int kSingle[] = {1, 2, 4, 8, 16, 32}, kPaired[] = {4, 8, 16, 32, 64};
        const int* cand = kind == Op::ITER2 ? kPaired : kSingle;
        for (int c = 0; c < (kind == Op::ITER2 ? 5 : 6); ++c) {
            const int rows = cand[c];
            if (rows > n - 1) break;
            a.rows = rows;
            cudaError_t e = launch();  // warm-up
            if (e == cudaSuccess) e = launch();
            for (int r = 0; r < 5 && e == cudaSuccess; ++r) {
                if (r == 0) e = cudaEventRecord(e0, st);
                if (e == cudaSuccess) e = launch();
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(h, e, "autotuning the sweep");
            }
            const double us = 1e3 * ms / 5.0;
            if (us < best) { best = us; pick = rows; }
        }
        for (auto* part : {&h->partA, &h->partB})
            for (Op& op : *part)
                if (op.kind == kind && op.sweeps == sweeps && op.it.m == 0 && op.it.e_new.n == n) op.it.rows = pick;
        if (n == h->n && (kind == Op::ITER || !level0_single)) {
            *best_rows = pick;
            *best_us = best;
            level0_single |= kind == Op::ITER;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return HOMG_OK;
}

// A group of one problem was planned without batch views (nothing to index). Inside the persistent
// kernel every op must still skip a problem that has converged, so its ops get the views too.
void force_views(homg_ctx* h, PersistItem& it) {
    if (h->nbatch > 1) return;
    it.it.bst = h->dstate;
    it.it.nb = 1;
    it.pr.bst = h->dstate;
    it.pr.nb = 1;
    it.rs.bst = h->dstate;
    it.rs.nb = 1;
    if (it.kind == PK_RESID) {
        it.ra.batch = 1;
        it.ra.nb = 1;
    }
}

// The persistent kernel's program: per group the item lists of the initial residual and test, of a
// cycle with odd and with even stage (the solution buffers alternate), and of the copy-out; phase j
// of a segment holds item j of every group's list. One device allocation holds the items, the
// phases, copies of the groups' coarse-lattice op lists (with batch views), the barrier and running
// counters, the per-phase work counters and the failure flag.
int build_persistent(homg_batch_ctx* b) {
    const int G = (int)b->groups.size();
    std::vector<std::vector<BlockOp>> bops(G);
    std::vector<size_t> bop_off(G, 0);
    size_t nbops = 0;
    for (int g = 0; g < G; ++g) {
        homg_ctx* h = b->groups[g];
        bops[g] = h->block_ops;
        if (h->nbatch <= 1)
            for (BlockOp& o : bops[g]) {
                o.it.bst = o.pr.bst = o.rs.bst = h->dstate;
                o.it.nb = o.pr.nb = o.rs.nb = 1;
            }
        bop_off[g] = nbops;
        nbops += bops[g].size();
    }
    // item lists per group; BLOCK items get their op pointer once the allocation exists
    enum { SEG_INIT = 0, SEG_ODD = 1, SEG_EVEN = 2, SEG_COPY = 3 };
    std::vector<std::vector<PersistItem>> lists[4];
    std::vector<std::vector<int>> block_first[4];
    for (int seg = 0; seg < 4; ++seg) {
        lists[seg].resize(G);
        block_first[seg].resize(G);
    }
    for (int g = 0; g < G; ++g) {
        homg_ctx* h = b->groups[g];
        auto push = [&](int seg, PersistItem it, int bfirst) {
            force_views(h, it);
            lists[seg][g].push_back(it);
            block_first[seg][g].push_back(bfirst);
        };
        {
            PersistItem r, f;
            persist_resid(resid_args(h, 0), h->n, r);
            persist_final(fin_args(h, FIN_INIT, nullptr), f);
            push(SEG_INIT, r, -1);
            push(SEG_INIT, f, -1);
        }
        for (int seg : {SEG_ODD, SEG_EVEN}) {
            for (auto* part : {&h->partA, &h->partB})
                for (const Op& op : *part) {
                    PersistItem it;
                    int bf = -1;
                    switch (op.kind) {
                        case Op::ITER: persist_iter(op.it, it); break;
                        case Op::ITER2: persist_iter2(op.sweeps, op.it, it); break;
                        case Op::PROLONG: persist_prolong(op.pr, it); break;
                        case Op::RESTRICT: persist_restrict(op.rs, it); break;
                        case Op::BLOCK:
                            persist_block(nullptr, op.block_count, h->nbatch, it);
                            bf = (int)(bop_off[g] + (size_t)op.block_first);
                            break;
                        default: return fail(nullptr, HOMG_EINVAL, "homg_batch_create: op without a persistent form%s%s");
                    }
                    push(seg, it, bf);
                }
            PersistItem r, f;
            persist_resid(resid_args(h, seg == SEG_ODD ? 1 : 2), h->n, r);
            persist_final(fin_args(h, FIN_CYCLE, nullptr), f);
            push(seg, r, -1);
            push(seg, f, -1);
        }
        PersistItem c;
        persist_copy(copy_args(h), h->n, c);
        push(SEG_COPY, c, -1);
    }
    // merge: phase j of a segment = item j of every group that has one
    std::vector<PersistItem> items;
    std::vector<int> item_bfirst;
    std::vector<PersistPhase> phases;
    int seg_first[4], seg_count[4];
    for (int seg = 0; seg < 4; ++seg) {
        size_t len = 0;
        for (int g = 0; g < G; ++g) len = std::max(len, lists[seg][g].size());
        seg_first[seg] = (int)phases.size();
        seg_count[seg] = (int)len;
        for (size_t j = 0; j < len; ++j) {
            PersistPhase ph{(int)items.size(), 0, 0};
            for (int g = 0; g < G; ++g) {
                if (j >= lists[seg][g].size()) continue;
                const PersistItem& it = lists[seg][g][j];
                items.push_back(it);
                item_bfirst.push_back(block_first[seg][g][j]);
                ph.count += 1;
                ph.blocks += it.gx * it.gy * it.gz;
            }
            phases.push_back(ph);
        }
    }
    if (seg_count[SEG_ODD] != seg_count[SEG_EVEN])
        return fail(nullptr, HOMG_EINVAL, "homg_batch_create: cycle programs of unequal length%s%s");
    b->nqueue = (size_t)seg_count[SEG_INIT] + (size_t)HOMG_MAX_CYCLES * seg_count[SEG_ODD] + (size_t)seg_count[SEG_COPY];
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (size_t)round_up((int64_t)off, 256); size_t o = off; off += bytes; return o; };
    const size_t o_items = take(items.size() * sizeof(PersistItem));
    const size_t o_phases = take(phases.size() * sizeof(PersistPhase));
    const size_t o_bops = take(std::max<size_t>(nbops, 1) * sizeof(BlockOp));
    const size_t o_sync = take(8 * sizeof(unsigned int));
    const size_t o_err = take(sizeof(int));
    const size_t o_queue = take(b->nqueue * sizeof(unsigned int));
    CK(nullptr, cudaMalloc(&b->parena, (size_t)round_up((int64_t)off, 256)), "allocating the persistent program");
    CK(nullptr, cudaMallocHost(&b->herr, sizeof(int)), "cudaMallocHost");
    BlockOp* dbops = (BlockOp*)(b->parena + o_bops);
    for (size_t q = 0; q < items.size(); ++q)
        if (item_bfirst[q] >= 0) items[q].ops = dbops + item_bfirst[q];
    for (int g = 0; g < G; ++g)
        if (!bops[g].empty())
            CK(nullptr, cudaMemcpy(dbops + bop_off[g], bops[g].data(), bops[g].size() * sizeof(BlockOp), cudaMemcpyHostToDevice),
               "uploading the persistent program");
    CK(nullptr, cudaMemcpy(b->parena + o_items, items.data(), items.size() * sizeof(PersistItem), cudaMemcpyHostToDevice),
       "uploading the persistent program");
    CK(nullptr, cudaMemcpy(b->parena + o_phases, phases.data(), phases.size() * sizeof(PersistPhase), cudaMemcpyHostToDevice),
       "uploading the persistent program");
    PersistArgs& a = b->pargs;
    a.items = (const PersistItem*)(b->parena + o_items);
    a.phases = (const PersistPhase*)(b->parena + o_phases);
    a.init_first = seg_first[SEG_INIT];
    a.init_count = seg_count[SEG_INIT];
    a.cyc_first[1] = seg_first[SEG_ODD];   // cycle k odd
    a.cyc_first[0] = seg_first[SEG_EVEN];  // cycle k even
    a.cyc_count = seg_count[SEG_ODD];
    a.copy_first = seg_first[SEG_COPY];
    a.copy_count = seg_count[SEG_COPY];
    a.sync = (unsigned int*)(b->parena + o_sync);
    a.err = (int*)(b->parena + o_err);
    a.queue = (unsigned int*)(b->parena + o_queue);
    a.timeout_ns = 5000000000LL;
    b->persistent = true;
    return HOMG_OK;
}

// Clear the persistent kernel's counters and failure flag on `s` (before every launch).
cudaError_t persistent_reset(homg_batch_ctx* b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->pargs.sync, 0, 8 * sizeof(unsigned int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->pargs.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->pargs.queue, 0, b->nqueue * sizeof(unsigned int), s);
    return e;
}

void batch_destroy(homg_batch_ctx* b) {
    for (homg_ctx* h : b->groups) homg_destroy(h);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->t0) cudaEventDestroy(b->t0);
    if (b->t1) cudaEventDestroy(b->t1);
    if (b->hticket) cudaFreeHost(b->hticket);
    if (b->herr) cudaFreeHost(b->herr);
    if (b->parena) cudaFree(b->parena);
    delete b;
}

}  // namespace

extern "C" {

int homg_batch_create(int nprob, const int64_t* sides, const homg_options* opt, homg_batch_handle* out) {
    if (out) *out = nullptr;
    g_create_error[0] = 0;
    if (!out || !sides || nprob < 1) return fail(nullptr, HOMG_EINVAL, "homg_batch_create: null argument or no problems%s%s");
    homg_options o;
    homg_default_options(&o);
    if (opt) o = *opt;
    int rc = check_options(2, o);
    if (rc != HOMG_OK) return rc;
    if (o.strict_fp || o.exec_mode == HOMG_EXEC_WHOLEGRID || o.n_schedule > 0 || o.cycle != HOMG_CYCLE_HOMG ||
        o.launch_mode == HOMG_LAUNCH_STREAM || o.geometry != HOMG_GEOM_NESTED)
        return fail(nullptr, HOMG_EINVAL,
                    "homg_batch_create: batches use fast arithmetic, the lattice form, MFMG and graph or persistent launches%s%s");
    const bool persistent = o.launch_mode == HOMG_LAUNCH_PERSISTENT;
    o.launch_mode = HOMG_LAUNCH_GRAPH;  // the groups themselves are planned as for graph launches
    if (persistent) o.run_max_n = -1;   // its kernel runs every op as work items: no level runs
    o.tma_min_n = -1;                   // batch groups keep the per-problem views of the marching kernels
    std::vector<int64_t> distinct;
    std::vector<int> group_of(nprob), index_in_group(nprob);
    std::vector<int> counts;
    for (int p = 0; p < nprob; ++p) {
        if (grid_exponent(2, sides[p], "homg_batch_create") < 0) return HOMG_ESHAPE;
        size_t g = 0;
        while (g < distinct.size() && distinct[g] != sides[p]) ++g;
        if (g == distinct.size()) {
            if ((int)distinct.size() == HOMG_BATCH_MAX_GROUPS)
                return fail(nullptr, HOMG_EINVAL, "homg_batch_create: more than HOMG_BATCH_MAX_GROUPS sizes%s%s");
            distinct.push_back(sides[p]);
            counts.push_back(0);
        }
        group_of[p] = (int)g;
        index_in_group[p] = counts[g]++;
    }
    homg_batch_ctx* b = new (std::nothrow) homg_batch_ctx();
    if (!b) return fail(nullptr, HOMG_ENOMEM, "homg_batch_create: out of host memory%s%s");
    b->nprob = nprob;
    b->group_of = group_of;
    b->index_in_group = index_in_group;
    cudaError_t ce = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (ce == cudaSuccess) ce = cudaEventCreate(&b->t0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&b->t1);
    if (ce == cudaSuccess) ce = cudaMallocHost(&b->hticket, 4 * HOMG_BATCH_MAX_GROUPS * sizeof(unsigned int));
    if (ce != cudaSuccess) {
        rc = cuda_fail(nullptr, ce, "homg_batch_create");
        batch_destroy(b);
        return rc;
    }
    b->stats.groups = (int)distinct.size();
    for (size_t g = 0; g < distinct.size(); ++g) {
        const int K = grid_exponent(2, distinct[g], "homg_batch_create");
        homg_ctx* h = nullptr;
        rc = create_ctx(2, distinct[g] - 1, K, K, 5, o, counts[g], &h);
        if (rc != HOMG_OK) {
            batch_destroy(b);
            return rc;
        }
        b->groups.push_back(h);
        cudaStream_t s = nullptr;
        cudaEvent_t j = nullptr;
        ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
        if (ce != cudaSuccess) {
            rc = cuda_fail(nullptr, ce, "homg_batch_create: streams");
            batch_destroy(b);
            return rc;
        }
        b->streams.push_back(s);
        b->joins.push_back(j);
        h->stream = s;
        int rows = 0;
        double us = 0.0;
        rc = autotune_rows(h, s, &rows, &us);
        if (rc != HOMG_OK) {
            set_null_handle_error(h->err);
            batch_destroy(b);
            return rc;
        }
        b->stats.sides[g] = distinct[g];
        b->stats.counts[g] = counts[g];
        b->stats.rows[g] = rows;
        b->stats.tuned_us[g] = us;
    }
    b->prec = o.precision;
    if (persistent) {
        rc = build_persistent(b);
        if (rc != HOMG_OK) {
            batch_destroy(b);
            return rc;
        }
    }
    *out = b;
    return HOMG_OK;
}

int homg_batch_set_stream(homg_batch_handle b, void* stream) {
    if (!b) return HOMG_EINVAL;
    b->stream = (cudaStream_t)stream;
    return HOMG_OK;
}

int homg_batch_solve(homg_batch_handle b, const double* const* f, double* const* u, double tol, int max_cycles,
                     int* status, int* cycles, double* relres, double* solve_ms) {
    if (!b) return HOMG_EINVAL;
    if (!f || !u) return fail(nullptr, HOMG_EINVAL, "homg_batch_solve: null %s%s", !f ? "f" : "u");
    if (!(tol >= 0.0) || !std::isfinite(tol) || max_cycles < 0 || max_cycles > HOMG_MAX_CYCLES)
        return fail(nullptr, HOMG_EINVAL, "homg_batch_solve: invalid tol or max_cycles%s%s");
    for (int p = 0; p < b->nprob; ++p)
        if (!f[p] || !u[p]) return fail(nullptr, HOMG_EINVAL, "homg_batch_solve: null problem array%s%s");
    const int G = (int)b->groups.size();
    NvtxRange batch_range("homg_batch_solve");
    auto cfail = [&](cudaError_t e, const char* where) { return cuda_fail(nullptr, e, where); };
    cudaError_t e = cudaEventRecord(b->t0, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    if (e != cudaSuccess) return cfail(e, "homg_batch_solve");
    if (b->persistent) {
        // one cooperative launch on the caller's stream: states in, the kernel, states out
        for (int g = 0; g < G; ++g) {
            homg_ctx* h = b->groups[g];
            for (int q = 0; q < h->nbatch; ++q) memset(&h->hstate[q], 0, sizeof(State));
        }
        for (int p = 0; p < b->nprob; ++p) {
            homg_ctx* h = b->groups[b->group_of[p]];
            State& st = h->hstate[b->index_in_group[p]];
            st.f = f[p];
            st.u = u[p];
            st.tol = tol;
            st.div_factor = h->opt.diverge_factor;
            st.max_cycles = max_cycles;
            st.status = -1;
        }
        for (int g = 0; g < G && e == cudaSuccess; ++g) {
            homg_ctx* h = b->groups[g];
            e = cudaMemcpyAsync(h->dstate, h->hstate, (size_t)h->nbatch * sizeof(State), cudaMemcpyHostToDevice, b->stream);
        }
        if (e == cudaSuccess) e = persistent_reset(b, b->stream);
        PersistArgs pa = b->pargs;
        pa.max_cycles = max_cycles;
        pa.stall = 0;
        if (e == cudaSuccess) e = launch_persistent(b->prec, pa, &b->pblocks, b->stream);
        for (int g = 0; g < G && e == cudaSuccess; ++g) {
            homg_ctx* h = b->groups[g];
            e = cudaMemcpyAsync(h->hstate, h->dstate, (size_t)h->nbatch * sizeof(State), cudaMemcpyDeviceToHost, b->stream);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->herr, b->pargs.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->t1);
        if (e != cudaSuccess) return cfail(e, "homg_batch_solve: the persistent kernel");
        b->stats.solve_ms = elapsed(b->t0, b->t1);
        if (*b->herr)
            return fail(nullptr, HOMG_TIMEOUT, "homg_batch_solve: a grid barrier of the persistent kernel gave up%s%s");
    } else {
    const int want = std::min(std::max(max_cycles, 1), kStagesPerGraph);
    for (int g = 0; g < G; ++g) {
        homg_ctx* h = b->groups[g];
        for (int q = 0; q < h->nbatch; ++q) memset(&h->hstate[q], 0, sizeof(State));
        for (int p = 0; p < b->nprob; ++p) {
            if (b->group_of[p] != g) continue;
            State& st = h->hstate[b->index_in_group[p]];
            st.f = f[p];
            st.u = u[p];
            st.tol = tol;
            st.div_factor = h->opt.diverge_factor;
            st.max_cycles = max_cycles;
            st.status = -1;
        }
        if (!h->gfirst.exec || h->gfirst.stages < want) {
            int rc = build_graph(h, h->gfirst, want, true);
            if (rc != HOMG_OK) {
                set_null_handle_error(h->err);
                return rc;
            }
        }
        cudaStream_t s = b->streams[g];
        e = cudaStreamWaitEvent(s, b->fork, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->dstate, h->hstate, (size_t)h->nbatch * sizeof(State), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dticket, 0, 4 * sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaGraphLaunch(h->gfirst.exec, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->hstate, h->dstate, (size_t)h->nbatch * sizeof(State), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->hticket + 4 * g, h->dticket, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cfail(e, "homg_batch_solve: launching a group");
    }
    // Continuation launches while problems of a group still run and cycles remain. Each pass
    // waits for one group at a time but re-launches it before moving on, so groups never wait
    // for one another.
    std::vector<int> pending;
    for (int g = 0; g < G; ++g) pending.push_back(g);
    while (!pending.empty()) {
        std::vector<int> still;
        for (int g : pending) {
            homg_ctx* h = b->groups[g];
            cudaStream_t s = b->streams[g];
            unsigned int* tk = b->hticket + 4 * g;
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cfail(e, "homg_batch_solve");
            int running = 0;
            for (int q = 0; q < h->nbatch; ++q) running |= !h->hstate[q].done;
            const int done_cycles = (int)tk[1];
            if (!running || done_cycles >= max_cycles) {
                e = cudaEventRecord(b->joins[g], s);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->joins[g], 0);
                if (e != cudaSuccess) return cfail(e, "homg_batch_solve");
                continue;
            }
            if (!h->gcont.exec) {
                int rc = build_graph(h, h->gcont, kStagesPerGraph, false);
                if (rc != HOMG_OK) {
                    set_null_handle_error(h->err);
                    return rc;
                }
            }
            tk[2] = (unsigned int)done_cycles;
            e = cudaMemcpyAsync(h->dticket + 2, tk + 2, sizeof(unsigned int), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaGraphLaunch(h->gcont.exec, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->hstate, h->dstate, (size_t)h->nbatch * sizeof(State), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tk, h->dticket, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return cfail(e, "homg_batch_solve: continuation");
            still.push_back(g);
        }
        pending.swap(still);
    }
    e = cudaEventRecord(b->t1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b->t1);
    if (e != cudaSuccess) return cfail(e, "homg_batch_solve");
    b->stats.solve_ms = elapsed(b->t0, b->t1);
    }
    int worst = HOMG_OK;
    for (int p = 0; p < b->nprob; ++p) {
        const State& st = b->groups[b->group_of[p]]->hstate[b->index_in_group[p]];
        if (status) status[p] = st.status;
        if (cycles) cycles[p] = st.cycle;
        if (relres) relres[p] = st.relres;
        if (solve_ms) solve_ms[p] = 1e-6 * (double)(st.t_done - st.t_start);
        if (st.status > worst) worst = st.status;
    }
    return worst;
}

int homg_batch_check_barrier_timeout(homg_batch_handle b, double* waited_ms) {
    if (!b) return HOMG_EINVAL;
    if (!b->persistent)
        return fail(nullptr, HOMG_EINVAL, "homg_batch_check_barrier_timeout: the batch has no persistent kernel%s%s");
    PersistArgs pa = b->pargs;
    pa.stall = 1;  // the first barrier waits for one block more than the launch has
    pa.timeout_ns = 250000000LL;
    pa.max_cycles = 0;
    cudaError_t e = persistent_reset(b, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->t0, b->stream);
    int blocks = 0;
    if (e == cudaSuccess) e = launch_persistent(b->prec, pa, &blocks, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->t1, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->herr, b->pargs.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "homg_batch_check_barrier_timeout");
    if (waited_ms) *waited_ms = elapsed(b->t0, b->t1);
    if (*b->herr)
        return fail(nullptr, HOMG_TIMEOUT, "homg_batch_check_barrier_timeout: the grid barrier gave up after its time limit%s%s");
    return HOMG_OK;
}

int homg_batch_get_stats(homg_batch_handle b, homg_batch_stats* out) {
    if (!b || !out) return HOMG_EINVAL;
    *out = b->stats;
    return HOMG_OK;
}

void homg_batch_destroy(homg_batch_handle b) {
    if (!b) return;
    batch_destroy(b);
}

int homg_set_stream(homg_handle h, void* stream) {
    if (!h) return HOMG_EINVAL;
    h->stream = (cudaStream_t)stream;
    return HOMG_OK;
}

int homg_solve(homg_handle h, const double* f, double* u, double tol, int max_cycles, int* cycles_out, double* relres_out) {
    if (!h) return HOMG_EINVAL;
    memset(&h->stats, 0, sizeof(h->stats));
    if (!f || !u) return fail(h, HOMG_EINVAL, "homg_solve: null %s%s", !f ? "f" : "u");
    if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(h, HOMG_EINVAL, "homg_solve: tol must be finite and >= 0%s%s");
    if (max_cycles < 0 || max_cycles > HOMG_MAX_CYCLES)
        return fail(h, HOMG_EINVAL, "homg_solve: max_cycles must be in [0, HOMG_MAX_CYCLES]%s%s");
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    NvtxRange solve_range("homg_solve");
    State* s = h->hstate;
    memset(s, 0, sizeof(*s));
    s->f = f;
    s->u = u;
    s->tol = tol;
    s->div_factor = h->opt.diverge_factor;
    s->max_cycles = max_cycles;
    s->status = -1;
    homg_stats& st = h->stats;
    if (h->opt.launch_mode == HOMG_LAUNCH_GRAPH) {
        // First graph: initial residual and up to kStagesPerGraph cycles. Grown (rebuilt) when a
        // later solve allows more cycles, up to kStagesPerGraph.
        const int want = std::min(std::max(max_cycles, 1), kStagesPerGraph);
        if (!h->gfirst.exec || h->gfirst.stages < want) {
            int rc = build_graph(h, h->gfirst, want, true);
            if (rc != HOMG_OK) return rc;
        }
        s->stages = h->gfirst.stages;
        s->stage_base = 0;
        NvtxRange graph_range("homg_solve: graph launches");
        CK(h, cudaMemcpyAsync(h->dstate, s, sizeof(State), cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(state)");
        CK(h, cudaGraphLaunch(h->gfirst.exec, h->stream), "cudaGraphLaunch");
        CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(state)");
        CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        add_graph_times(st, h->gfirst.ev, s->cycle, 3 * h->gfirst.stages + 2);
        // Continuation launches while the solve runs and cycles remain (one host sync per launch).
        while (!s->done && s->cycle < max_cycles) {
            if (!h->gcont.exec) {
                int rc = build_graph(h, h->gcont, kStagesPerGraph, false);
                if (rc != HOMG_OK) return rc;
            }
            const int base = s->cycle;
            NvtxRange cont_range("homg_solve: continuation cycles (graph)");
            State* d = h->dstate;
            s->stage_base = base;
            s->stages = h->gcont.stages;
            CK(h, cudaMemcpyAsync(&d->stage_base, &s->stage_base, sizeof(int), cudaMemcpyHostToDevice, h->stream),
               "cudaMemcpyAsync(state)");
            CK(h, cudaGraphLaunch(h->gcont.exec, h->stream), "cudaGraphLaunch");
            CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(state)");
            CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            add_graph_times(st, h->gcont.ev, s->cycle - base, 3 * h->gcont.stages + 2);
        }
    } else {
        // Stream launch mode: same kernels and event layout, the host reads the state once per cycle.
        const size_t need = 3 * (size_t)max_cycles + 3;
        while (h->sev.size() < need) {
            cudaEvent_t e;
            CK(h, cudaEventCreate(&e), "cudaEventCreate");
            h->sev.push_back(e);
        }
        cudaStream_t sm = h->stream;
        CK(h, cudaMemcpyAsync(h->dstate, s, sizeof(State), cudaMemcpyHostToDevice, sm), "cudaMemcpyAsync(state)");
        CK(h, cudaEventRecord(h->sev[0], sm), "cudaEventRecord");
        CK(h, launch_residual(h->ndim, h->prec, h->strict, resid_args(h, 0), h->n, sm), "residual kernel");
        CK(h, launch_finalize(fin_args(h, FIN_INIT, nullptr), sm), "finalize kernel");
        CK(h, cudaEventRecord(h->sev[1], sm), "cudaEventRecord");
        CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync(state)");
        CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
        for (int k = 1; !s->done && k <= max_cycles; ++k) {
            NvtxRange cycle_range("homg cycle");
            CK(h, enqueue_ops(h, h->partA, sm), "cycle kernels");
            CK(h, cudaEventRecord(h->sev[3 * k - 1], sm), "cudaEventRecord");
            CK(h, enqueue_ops(h, h->partB, sm), "cycle kernels");
            CK(h, cudaEventRecord(h->sev[3 * k], sm), "cudaEventRecord");
            CK(h, launch_residual(h->ndim, h->prec, h->strict, resid_args(h, k), h->n, sm), "residual kernel");
            CK(h, launch_finalize(fin_args(h, FIN_CYCLE, nullptr), sm), "finalize kernel");
            CK(h, cudaEventRecord(h->sev[3 * k + 1], sm), "cudaEventRecord");
            CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync(state)");
            CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
        }
        CK(h, launch_copy_out(h->ndim, copy_args(h), h->n, sm), "copy-out kernel");
        const int end_ev = 3 * s->cycle + 2;
        CK(h, cudaEventRecord(h->sev[end_ev], sm), "cudaEventRecord");
        CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
        add_graph_times(st, h->sev, s->cycle, end_ev);
    }
    CK(h, cudaMemcpyAsync(h->hhist, h->dhist, (max_cycles + 1) * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
       "cudaMemcpyAsync(hist)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (s->fault)
        return fail(h, HOMG_ECUDA, "homg_solve: a two-sweep launch's TMA copy did not complete within its bound%s%s");
    const int cycles = s->cycle;
    if (cycles_out) *cycles_out = cycles;
    if (relres_out) *relres_out = s->relres;
    st.cycles = cycles;
    st.status = s->status;
    st.exec_mode = h->exec;
    st.iterations_per_cycle = (int)h->sched.size();
    st.fine_iterations_per_cycle = h->fine_iters;
    st.fine_launches_per_cycle = 0;
    for (const Op& op : h->partB) st.fine_launches_per_cycle += (op.kind == Op::ITER || op.kind == Op::ITER2) ? 1 : 0;
    st.kernels_per_cycle = (int)(h->partA.size() + h->partB.size()) + 2;
    st.kernels_fixed = 3;
    st.kernel_launches = st.kernels_fixed + (long long)cycles * st.kernels_per_cycle;
    st.setup_ms = st.solve_ms - st.coarse_ms - st.fine_ms - st.residual_ms;
    const double pts = (h->ndim == 2) ? (double)(h->n - 1) * (h->n - 1) : (double)(h->n - 1) * (h->n - 1) * (h->n - 1);
    st.precision = h->prec;
    st.fine_bytes_per_iteration = 3.0 * prec_bytes(h->prec) * pts;
    st.fine_flops_per_iteration = (h->ndim == 2 ? 5.0 : 7.0) * pts;
    return s->status;
}

int homg_solve_host(homg_handle h, const double* f_host, double* u_host, double tol, int max_cycles, int* cycles_out,
                    double* relres_out) {
    if (!h) return HOMG_EINVAL;
    if (!f_host || !u_host) return fail(h, HOMG_EINVAL, "homg_solve_host: null %s%s", !f_host ? "f" : "u");
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    const size_t bytes = (size_t)grid_elems(h->ndim, h->n, h->n + 1) * sizeof(double);
    if (!h->stage_f) {
        CK(h, cudaMalloc(&h->stage_f, bytes), "cudaMalloc(staging f)");
        CK(h, cudaMalloc(&h->stage_u, bytes), "cudaMalloc(staging u)");
    }
    CK(h, cudaMemcpyAsync(h->stage_f, f_host, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(f)");
    CK(h, cudaMemcpyAsync(h->stage_u, u_host, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(u)");
    int rc = homg_solve(h, h->stage_f, h->stage_u, tol, max_cycles, cycles_out, relres_out);
    if (rc < 0) return rc;
    CK(h, cudaMemcpyAsync(u_host, h->stage_u, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(u)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return rc;
}

int homg_set_coefficient(homg_handle h, const double* k) {
    if (!h) return HOMG_EINVAL;
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    if (k && (h->ndim != 2 || h->exec != HOMG_EXEC_LATTICE || h->strict || h->opt.cycle != HOMG_CYCLE_HOMG ||
              h->nbatch != 1))
        return fail(h, HOMG_EINVAL,
                    "homg_set_coefficient: variable coefficients need a 2-D handle with HOMG cycles in the fast "
                    "lattice form%s%s");
    if (k) {
        const bool dbl = (h->prec == PREC_FP64);
        const size_t ks = dbl ? sizeof(double) : sizeof(float);
        if (!h->vc_arena) {
            size_t off = 0;
            auto take = [&](size_t bytes) { off = (size_t)round_up((int64_t)off, 256); size_t o = off; off += bytes; return o; };
            std::vector<size_t> ox, oy, ow;
            for (int m = 0; m < h->levels; ++m) {
                const size_t bytes = (size_t)grid_elems(2, h->L[m].n, h->L[m].pitch) * ks;
                ox.push_back(take(bytes));
                oy.push_back(take(bytes));
                ow.push_back(take(bytes));
            }
            const size_t b0 = (size_t)grid_elems(2, h->n, h->pitch0) * sizeof(double);
            const size_t o0x = dbl ? 0 : take(b0), o0y = dbl ? 0 : take(b0);
            const size_t obad = take(sizeof(int));
            const size_t olog = take((size_t)(h->n + 1) * (h->n + 1) * sizeof(uint16_t));
            CK(h, cudaMalloc(&h->vc_arena, (size_t)round_up((int64_t)off, 256)), "allocating the coefficient arrays");
            for (int m = 0; m < h->levels; ++m) {
                h->vkx.push_back(h->vc_arena + ox[m]);
                h->vky.push_back(h->vc_arena + oy[m]);
                h->vwd.push_back(h->vc_arena + ow[m]);
            }
            h->kx0 = dbl ? (double*)h->vkx[0] : (double*)(h->vc_arena + o0x);
            h->ky0 = dbl ? (double*)h->vky[0] : (double*)(h->vc_arena + o0y);
            h->dbad = (int*)(h->vc_arena + obad);
            h->logk = (uint16_t*)(h->vc_arena + olog);
        }
        CK(h, cudaMemsetAsync(h->dbad, 0, sizeof(int), h->stream), "cudaMemsetAsync");
        for (int m = 0; m < h->levels; ++m)
            CK(h, launch_vc_setup(k, h->n, m, dbl, h->vkx[m], h->vky[m], h->vwd[m], h->L[m].pitch, h->opt.omega_j,
                                  h->dbad, h->stream),
               "coefficient set-up kernel");
        if (!dbl)
            CK(h, launch_vc_setup(k, h->n, 0, true, h->kx0, h->ky0, nullptr, h->pitch0, h->opt.omega_j, h->dbad,
                                  h->stream),
               "coefficient set-up kernel");
        CK(h, launch_logk(k, h->n, h->logk, h->stream), "log-coefficient kernel");
        int bad = 0;
        CK(h, cudaMemcpyAsync(&bad, h->dbad, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
        CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        if (bad) {
            h->vc = false;
            plan_cycle(h);
            group_coarse_block(h);
            destroy_graph(h->gfirst);
            destroy_graph(h->gcont);
            return fail(h, HOMG_EINVAL, "homg_set_coefficient: k must be positive and finite at every node%s%s");
        }
    }
    h->vc = (k != nullptr);
    plan_cycle(h);
    group_coarse_block(h);
    if (!h->block_ops.empty())
        CK(h, cudaMemcpy(h->dblock_ops, h->block_ops.data(), h->block_ops.size() * sizeof(BlockOp), cudaMemcpyHostToDevice),
           "copying the coarse-lattice op list");
    destroy_graph(h->gfirst);
    destroy_graph(h->gcont);
    return HOMG_OK;
}

}  // extern "C"

namespace {

// Buffers of the learned solve, allocated once per handle.
int ensure_learned(homg_ctx* h) {
    if (h->learn_arena) return HOMG_OK;
    const int64_t side = h->n + 1;
    const size_t es = (size_t)prec_bytes(h->prec);
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (size_t)round_up((int64_t)off, 256); size_t o = off; off += bytes; return o; };
    const size_t ox = take((size_t)side * side * 16 * 2);
    const size_t oy = take((size_t)side * side * sizeof(float));
    const size_t oc = take((size_t)grid_elems(2, h->n, h->pitch0) * es);
    const size_t og = take((size_t)grid_elems(2, h->n, h->pitch0) * es);
    const size_t op = take((size_t)std::max(feat_parts(h->n), h->nparts) * sizeof(double));
    const size_t op2 = take((size_t)h->nparts * sizeof(double));
    const size_t os = take(4 * sizeof(double));
    const size_t ou2 = take((size_t)grid_elems(2, h->n, h->pitch0) * sizeof(double));
    const size_t ogs = take((size_t)grid_elems(2, h->n, h->pitch0) * es);
    const size_t op3 = take((size_t)h->nparts * sizeof(double));
    CK(h, cudaMalloc(&h->learn_arena, (size_t)round_up((int64_t)off, 256)), "allocating the learned-solve buffers");
    CK(h, cudaMemset(h->learn_arena, 0, (size_t)round_up((int64_t)off, 256)), "cudaMemset");
    h->lx = h->learn_arena + ox;
    h->ly = (float*)(h->learn_arena + oy);
    h->lcorr = h->learn_arena + oc;
    h->lg0 = h->learn_arena + og;
    h->lpart = (double*)(h->learn_arena + op);
    h->lpart2 = (double*)(h->learn_arena + op2);
    h->lscal = (double*)(h->learn_arena + os);
    h->lu2 = (double*)(h->learn_arena + ou2);
    h->lgs = h->learn_arena + ogs;
    h->lpart3 = (double*)(h->learn_arena + op3);
    return HOMG_OK;
}

// Features of the residual currently held in g0 (h^2 r): rho into lscal[0], the image into x.
cudaError_t enqueue_features(homg_ctx* h, const void* g0, void* x, cudaStream_t s) {
    const double cnt = (double)(h->n - 1) * (double)(h->n - 1);
    cudaError_t e = launch_feat_stats(h->prec, g0, h->pitch0, h->kx0, h->ky0, h->pitch0, h->n, h->lpart, s);
    if (e == cudaSuccess) e = launch_reduce(h->lpart, feat_parts(h->n), cnt, h->lscal, s);
    if (e == cudaSuccess)
        e = launch_feat_write(h->prec, g0, h->pitch0, h->kx0, h->ky0, h->pitch0, h->n, h->lscal, h->logk, x, s);
    return e;
}

}  // namespace

extern "C" {

int homg_features(homg_handle h, const double* f, const double* u, const double* u_ref, void* x_out, float* t_out,
                  double* rho_out) {
    if (!h) return HOMG_EINVAL;
    if (!f || !u || !x_out || !rho_out || (t_out && !u_ref))
        return fail(h, HOMG_EINVAL, "homg_features: null argument%s%s");
    if (!h->vc) return fail(h, HOMG_EINVAL, "homg_features: the handle has no coefficient (homg_set_coefficient)%s%s");
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    int rc = ensure_learned(h);
    if (rc != HOMG_OK) return rc;
    cudaStream_t sm = h->stream;
    State* s = h->hstate;
    memset(s, 0, sizeof(*s));
    s->f = f;
    s->u = (double*)u;
    CK(h, cudaMemcpyAsync(h->dstate, s, sizeof(State), cudaMemcpyHostToDevice, sm), "cudaMemcpyAsync(state)");
    ResidArgs a = resid_args(h, 0);
    a.u_out = dgrid(nullptr, 0, h->n);
    a.part_f = nullptr;
    CK(h, launch_residual(2, h->prec, false, a, h->n, sm), "residual kernel");
    CK(h, enqueue_features(h, h->L[0].g, x_out, sm), "feature kernels");
    if (t_out) CK(h, launch_target(u_ref, u, h->n, h->lscal, t_out, sm), "target kernel");
    double rho = 0.0;
    CK(h, cudaMemcpyAsync(&rho, h->lscal, sizeof(double), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync");
    CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
    *rho_out = rho;
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail(h, HOMG_EINVAL, "homg_features: zero or non-finite residual scale%s%s");
    return HOMG_OK;
}

int homg_set_learned_judge(homg_handle h, int judge) {
    if (!h) return HOMG_EINVAL;
    if (judge != HOMG_JUDGE_PROPOSAL && judge != HOMG_JUDGE_AFTER_CYCLE)
        return fail(h, HOMG_EINVAL, "homg_set_learned_judge: judge must be HOMG_JUDGE_PROPOSAL or HOMG_JUDGE_AFTER_CYCLE%s%s");
    h->learn_judge = judge;
    return HOMG_OK;
}

int homg_solve_learned(homg_handle h, homg_net_handle net, const double* f, double* u, double tol, int max_cycles,
                       int* cycles_out, double* relres_out, int* accepted_out) {
    if (!h) return HOMG_EINVAL;
    memset(&h->stats, 0, sizeof(h->stats));
    if (!net || !f || !u) return fail(h, HOMG_EINVAL, "homg_solve_learned: null argument%s%s");
    if (!h->vc) return fail(h, HOMG_EINVAL, "homg_solve_learned: the handle has no coefficient (homg_set_coefficient)%s%s");
    NvtxRange learned_range("homg_solve_learned");
    if (!(tol >= 0.0) || !std::isfinite(tol) || max_cycles < 0 || max_cycles > HOMG_MAX_CYCLES)
        return fail(h, HOMG_EINVAL, "homg_solve_learned: invalid tol or max_cycles%s%s");
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    int rc = ensure_learned(h);
    if (rc != HOMG_OK) return rc;
    cudaStream_t sm = h->stream;
    const int side = h->n + 1;
    const size_t gbytes = (size_t)grid_elems(2, h->n, h->pitch0) * (size_t)prec_bytes(h->prec);
    State* s = h->hstate;
    memset(s, 0, sizeof(*s));
    s->f = f;
    s->u = u;
    s->tol = tol;
    s->div_factor = h->opt.diverge_factor;
    s->max_cycles = max_cycles;
    s->status = -1;
    while (h->sev.size() < 2) {
        cudaEvent_t e;
        CK(h, cudaEventCreate(&e), "cudaEventCreate");
        h->sev.push_back(e);
    }
    CK(h, cudaEventRecord(h->sev[0], sm), "cudaEventRecord");
    CK(h, cudaMemcpyAsync(h->dstate, s, sizeof(State), cudaMemcpyHostToDevice, sm), "cudaMemcpyAsync(state)");
    CK(h, launch_residual(2, h->prec, false, resid_args(h, 0), h->n, sm), "residual kernel");
    CK(h, launch_reduce(h->part_r, h->nparts, 0.0, h->lscal + 1, sm), "norm kernel");
    CK(h, launch_finalize(fin_args(h, FIN_INIT, nullptr), sm), "finalize kernel");
    CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync(state)");
    CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
    // Three FP64 iterates: U[cur] holds the current one; the others receive a proposal or a branch.
    double* U[3] = {h->uint_[0], h->uint_[1], h->lu2};
    int cur = 0;
    int kept = 0, rejected_in_a_row = 0;
    const bool after_cycle = h->learn_judge == HOMG_JUDGE_AFTER_CYCLE;
    ResidArgs base = resid_args(h, 1);
    // u_out = u_in + e, its residual source into g0 and the partial sums of ||r||^2 into part
    auto update = [&](const double* u_in, const void* e, double* u_out, void* g0, double* part) {
        ResidArgs c = base;
        c.u_in = cdgrid(u_in, h->pitch0, h->n);
        c.e = cgrid(e, h->pitch0, h->n);
        c.u_out = dgrid(u_out, h->pitch0, h->n);
        c.g0 = grid(g0, h->pitch0, h->n);
        c.part_r = part;
        c.part_f = nullptr;
        return launch_residual(2, h->prec, false, c, h->n, sm);
    };
    auto cycle = [&]() -> cudaError_t {  // one HOMG cycle on the source in g0: the correction in e[e_final]
        cudaError_t e = enqueue_ops(h, h->partA, sm);
        if (e == cudaSuccess) e = enqueue_ops(h, h->partB, sm);
        return e;
    };
    for (int k = 1; !s->done && k <= max_cycles; ++k) {
        if (accepted_out) accepted_out[k - 1] = 0;
        bool keep = false;
        int next = cur;  // iterate after this cycle
        // after two rejections in a row the network stops proposing: plain HOMG cycles only
        if (rejected_in_a_row < 2) {
            const int a = (cur + 1) % 3, b = (cur + 2) % 3;
            // proposal u' = u + rho y into U[a], its residual source into lg0
            CK(h, enqueue_features(h, h->L[0].g, h->lx, sm), "feature kernels");
            rc = net_forward_dev(net, h->lx, 1, side, side, h->ly, sm);
            if (rc != HOMG_OK) return fail(h, rc, "homg_solve_learned: network inference failed: %s%s", homg_net_last_error(net));
            CK(h, launch_correct(h->prec, h->ly, h->n, h->lscal, h->lcorr, h->pitch0, sm), "correction kernel");
            CK(h, update(U[cur], h->lcorr, U[a], h->lg0, h->lpart2), "residual kernel");
            CK(h, launch_reduce(h->lpart2, h->nparts, 0.0, h->lscal + 2, sm), "norm kernel");
            if (!after_cycle) {
                // judge the proposal's own residual against the current one
                double nrm[2] = {0.0, 0.0};
                CK(h, cudaMemcpyAsync(nrm, h->lscal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync");
                CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
                rc = net_check_error(net);
                if (rc != HOMG_OK) return fail(h, rc, "homg_solve_learned: %s%s", homg_net_last_error(net));
                keep = nrm[1] < nrm[0];  // the plain solver's FP64 residual judges the proposal
                int from = cur;
                if (keep) {
                    from = a;
                    CK(h, cudaMemcpyAsync(h->L[0].g, h->lg0, gbytes, cudaMemcpyDeviceToDevice, sm), "cudaMemcpyAsync");
                }
                // one HOMG cycle on the kept iterate's residual
                CK(h, cycle(), "cycle kernels");
                next = (from == cur) ? a : b;
                CK(h, update(U[from], h->e[h->e_final], U[next], h->L[0].g, h->part_r), "residual kernel");
            } else {
                // judge after the cycle: one HOMG cycle from u (into U[b]) and one from u' (into U[cur]),
                // keep the result with the smaller FP64 residual
                CK(h, cudaMemcpyAsync(h->lgs, h->L[0].g, gbytes, cudaMemcpyDeviceToDevice, sm), "cudaMemcpyAsync");
                CK(h, cycle(), "cycle kernels");
                CK(h, update(U[cur], h->e[h->e_final], U[b], h->lgs, h->part_r), "residual kernel");
                CK(h, launch_reduce(h->part_r, h->nparts, 0.0, h->lscal + 1, sm), "norm kernel");
                CK(h, cudaMemcpyAsync(h->L[0].g, h->lg0, gbytes, cudaMemcpyDeviceToDevice, sm), "cudaMemcpyAsync");
                CK(h, cycle(), "cycle kernels");
                CK(h, update(U[a], h->e[h->e_final], U[cur], h->L[0].g, h->lpart3), "residual kernel");
                CK(h, launch_reduce(h->lpart3, h->nparts, 0.0, h->lscal + 2, sm), "norm kernel");
                double nrm[2] = {0.0, 0.0};
                CK(h, cudaMemcpyAsync(nrm, h->lscal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync");
                CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
                rc = net_check_error(net);
                if (rc != HOMG_OK) return fail(h, rc, "homg_solve_learned: %s%s", homg_net_last_error(net));
                keep = nrm[1] < nrm[0];
                if (keep) {
                    next = cur;  // the proposal's branch; its source is in g0 already
                    CK(h, cudaMemcpyAsync(h->part_r, h->lpart3, (size_t)h->nparts * sizeof(double), cudaMemcpyDeviceToDevice,
                                          sm), "cudaMemcpyAsync");
                } else {
                    next = b;  // the plain branch
                    CK(h, cudaMemcpyAsync(h->L[0].g, h->lgs, gbytes, cudaMemcpyDeviceToDevice, sm), "cudaMemcpyAsync");
                }
            }
            if (accepted_out) accepted_out[k - 1] = keep ? 1 : 0;
            if (keep) {
                ++kept;
                rejected_in_a_row = 0;
            } else {
                ++rejected_in_a_row;
            }
        } else {
            CK(h, cycle(), "cycle kernels");
            next = (cur + 1) % 3;
            CK(h, update(U[cur], h->e[h->e_final], U[next], h->L[0].g, h->part_r), "residual kernel");
        }
        // the test on the kept iterate's residual
        CK(h, launch_reduce(h->part_r, h->nparts, 0.0, h->lscal + 1, sm), "norm kernel");
        CK(h, launch_finalize(fin_args(h, FIN_CYCLE, nullptr), sm), "finalize kernel");
        cur = next;
        CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, sm), "cudaMemcpyAsync(state)");
        CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
    }
    CopyOutArgs co = copy_args(h);
    co.u0 = co.u1 = cdgrid(U[cur], h->pitch0, h->n);
    CK(h, launch_copy_out(2, co, h->n, sm), "copy-out kernel");
    CK(h, cudaEventRecord(h->sev[1], sm), "cudaEventRecord");
    CK(h, cudaMemcpyAsync(h->hhist, h->dhist, (max_cycles + 1) * sizeof(double), cudaMemcpyDeviceToHost, sm),
       "cudaMemcpyAsync(hist)");
    CK(h, cudaStreamSynchronize(sm), "cudaStreamSynchronize");
    homg_stats& st = h->stats;
    st.cycles = s->cycle;
    st.status = s->status;
    st.exec_mode = h->exec;
    st.precision = h->prec;
    st.iterations_per_cycle = (int)h->sched.size();
    st.solve_ms = elapsed(h->sev[0], h->sev[1]);
    st.kernels_fixed = kept;  // proposals the judge kept
    if (cycles_out) *cycles_out = s->cycle;
    if (relres_out) *relres_out = s->relres;
    return s->status;
}

int homg_residual_norm(homg_handle h, const double* f, const double* u, double* relres_out) {
    if (!h) return HOMG_EINVAL;
    if (!f || !u || !relres_out) return fail(h, HOMG_EINVAL, "homg_residual_norm: null argument%s%s");
    CK(h, cudaSetDevice(h->device), "cudaSetDevice");
    State* s = h->hstate;
    memset(s, 0, sizeof(*s));
    s->f = f;
    s->u = (double*)u;
    CK(h, cudaMemcpyAsync(h->dstate, s, sizeof(State), cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(state)");
    ResidArgs a{};
    a.st = h->dstate;
    a.inv_h2 = (double)h->n * (double)h->n;
    a.part_r = h->part_r;
    a.part_f = h->part_f;
    if (h->vc) {
        a.kx = h->kx0;
        a.ky = h->ky0;
        a.kpitch = h->pitch0;
    }
    CK(h, launch_residual(h->ndim, h->prec, h->strict, a, h->n, h->stream), "residual kernel");
    FinalizeArgs fa = fin_args(h, FIN_NORM, nullptr);
    fa.part_f = h->part_f;
    CK(h, launch_finalize(fa, h->stream), "finalize kernel");
    CK(h, cudaMemcpyAsync(s, h->dstate, sizeof(State), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(state)");
    CK(h, cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    *relres_out = s->relres;
    return HOMG_OK;
}

int homg_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n) {
    if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out)))
        return fail(nullptr, HOMG_EINVAL, "homg_check_conversions: n < 0 or a null pointer%s%s");
    cudaError_t e = launch_check_conversions(d_in, f_out, f_in, d_out, n, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "homg_check_conversions");
    return HOMG_OK;
}

int homg_check_sweep_pair(int precision, int n, int64_t pitch, const void* e_old, const void* g, void* e_packed,
                          void* e_column, double omega, double c1, int rows) {
    if ((precision != HOMG_PREC_FP32 && precision != HOMG_PREC_BF16) || n < 2 || n > (1 << 20) || rows < 0 ||
        !e_old || !g || !e_packed || !e_column || !(omega == omega) || !(c1 == c1))
        return fail(nullptr, HOMG_EINVAL, "homg_check_sweep_pair: bad precision, size, rows or pointer%s%s");
    IterArgs a;
    a.e_old = CGrid{e_old, pitch, n};
    a.g = CGrid{g, pitch, n};
    a.e_new = Grid{e_column, pitch, n};
    a.m = 0;
    a.mp = -1;
    a.dprev = CGrid{nullptr, pitch, n};
    a.dnew = Grid{nullptr, pitch, n};
    a.omega = omega;
    a.c1 = c1;
    a.omega_f = (float)omega;
    a.c1_f = (float)c1;
    a.rows = rows;
    cudaError_t e = launch_check_sweep_pair(precision, a, e_packed, nullptr);
    if (e == cudaErrorInvalidValue)
        return fail(nullptr, HOMG_EINVAL, "homg_check_sweep_pair: pitch < n + 2, odd, or an unaligned pointer%s%s");
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "homg_check_sweep_pair");
    return HOMG_OK;
}

int homg_get_history(homg_handle h, double* hist, int cap) {
    if (!h || !hist || cap < 0) return HOMG_EINVAL;
    const int cnt = std::min(cap, h->stats.cycles + 1);
    memcpy(hist, h->hhist, (size_t)cnt * sizeof(double));
    return cnt;
}

int homg_get_stats(homg_handle h, homg_stats* out) {
    if (!h || !out) return HOMG_EINVAL;
    *out = h->stats;
    return HOMG_OK;
}

const char* homg_last_error(homg_handle h) { return h ? h->err : g_create_error; }

void homg_destroy(homg_handle h) {
    if (!h) return;
    cudaSetDevice(h->device);
    destroy_graph(h->gfirst);
    destroy_graph(h->gcont);
    for (cudaEvent_t e : h->sev) cudaEventDestroy(e);
    if (h->arena) cudaFree(h->arena);
    if (h->vc_arena) cudaFree(h->vc_arena);
    if (h->learn_arena) cudaFree(h->learn_arena);
    if (h->stage_f) cudaFree(h->stage_f);
    if (h->stage_u) cudaFree(h->stage_u);
    if (h->hstate) cudaFreeHost(h->hstate);
    if (h->hhist) cudaFreeHost(h->hhist);
    delete h;
}

}  // extern "C"
