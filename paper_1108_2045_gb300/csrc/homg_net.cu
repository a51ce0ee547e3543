// Learned corrector of the HOMG restart loop (an extension: the paper has no learned part).
//
// A 4-layer 3x3 convolutional network (2 -> 32 -> 32 -> 32 -> 1 channels) in bfloat16 with binary32
// accumulation. Every convolution is an implicit GEMM on the tcgen05 tensor cores: a CTA stages a
// band of input rows (with a one-pixel halo) in shared memory, and the A operand of each product
// is one band row read through a shifted shared-memory descriptor -- no im2col copy. Rows of A are
// 128 consecutive pixels of one band row (M = 128), columns are input channels (K = 16 per
// instruction). The accumulators of a CTA's R output rows (R x COUT TMEM columns, row r at columns
// r COUT ..) live in tensor memory (TMEM) until an epilogue reads them back with tcgen05.ld.
// Band row rho at column shift dx feeds output rows rho - dy for the three vertical taps dy, so
// one instruction covers all of them: B stacks the weights of taps (2, dx), (1, dx), (0, dx) (3
// COUT rows) and the instruction takes the contiguous slice of that stack whose output rows exist,
// N = COUT, 2 COUT or 3 COUT wide, writing the adjacent accumulators of those rows. That makes
// about a third as many instructions as one per tap and output row, each up to three times wider.
// One thread issues the MMAs; completion is signalled through an mbarrier whose wait is bounded
// (the kernel records an error and frees its TMEM rather than spin forever).
//
// Activations use a row-chunked layout: element (b, c, y, x) of a [B, C, H, W] tensor at
// ((b*H + y)*(C/8) + c/8)*W*8 + x*8 + c%8, so that, for a fixed row and group of 8 channels, the
// pixels' 16-byte chunks are contiguous -- exactly the core-matrix rows of the no-swizzle
// K-major operand layout. Input rows arrive by TMA tensor copies: the layout is a 5-D tensor
// (8 channels, W pixels, C/8 groups, H rows, B images) whose box (8 x 130 x C/8 x 1 x 1) -- one
// input row with a one-pixel halo, zero-filled outside the image -- lands in a slot of a ring of
// staged rows in exactly the operand's order. A CTA walks down a column of tiles, so each tile
// loads only its R new rows, ahead of time (see k_conv3x3).
//
// Training kernels: weight packing (forward and transposed/flipped for the data gradient), the
// MSE loss and its gradient, the weight gradient (CUDA cores, binary32), Adam. Solver-side
// kernels turn an FP64 residual into features and a network output into a correction.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder comes from the runtime's entry-point query)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "../../include/homg.h"
#include "../../include/homg_net.h"
#include "homg_internal.h"
#include "homg_net_internal.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TW = 128;           // output pixels per accumulator row (MMA M)
constexpr int BANDW = TW + 2;     // staged pixels per band row (one-pixel halo each side)
constexpr int NT = 128;           // threads per conv CTA: one per TMEM lane
constexpr long long kWaitNs = 500000000ll;  // a barrier wait gives up after 0.5 s

// ---- PTX wrappers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// make this thread's shared-memory writes visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false once kWaitNs have passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 5-D tiled TMA load of the tensor map's box at the given coordinates (innermost first) into shared
// memory; completion counts the box's bytes on the mbarrier.
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, bf16 x bf16 -> f32, shape from idesc.
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 (or 16) consecutive 32-bit TMEM columns: thread t of the warp receives lane
// (lane base + t), columns [col, col + N). The wait is part of the same statement, so the
// registers are never read before the load completes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle, K-major: 8-row x 16-byte core matrices, `lbo`
// bytes between core matrices along K, `sbo` bytes between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major, M x N.
constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&t);
}
// ---- the convolution ------------------------------------------------------------------------
enum ConvMode { CONV_RELU = 0, CONV_LAST = 1, CONV_MASK = 2 };

struct ConvArgs {
    const bf16* in;     // [B, CIN, H, W] row-chunked
    const bf16* w;      // packed [9][CIN/8][COUT][8]
    const float* bias;  // [nbias] (CONV_RELU, CONV_LAST); padded channels get 0
    int nbias;
    bf16* out;          // CONV_RELU, CONV_MASK: [B, COUT, H, W] row-chunked
    float* outf;        // CONV_LAST: channel 0, [B][H][W]
    const bf16* mask;   // CONV_MASK: out = acc where mask > 0, else 0 ([B, COUT, H, W])
    int B, H, W;
    int* err;
    int unsignalled;    // self-test of the bounded wait: issue no MMA, so the barrier never completes
    int rows;           // output rows per CTA tile: 4 or 8
};

// R output rows per CTA tile (R + 2 staged band rows, one accumulator per output row).
template <int CIN, int COUT, int R>
struct ConvShape {
    static constexpr int GI = CIN / 8, GO = COUT / 8, KS = CIN / 16;
    static constexpr int BOXB = GI * BANDW * 16;  // one staged input row (all channel groups)
    // ring slot of a row, padded so every slot starts on the 128-byte boundary that a TMA tensor
    // copy's shared-memory destination needs
    static constexpr int ROWB = (BOXB + 127) / 128 * 128;
    static constexpr int NRING = 2 * R + 2;         // staged rows: this tile's R + 2 and the next tile's R
    static constexpr int RING = NRING * ROWB;
    static constexpr int WB = 9 * GI * COUT * 16;
    static constexpr uint32_t NCOLS = R * COUT;
    // Shared memory requested per CTA: at least enough that no more CTAs fit on one SM (228 KB)
    // than its 512 TMEM columns can hold at once, so no CTA ever waits in tcgen05.alloc.
    static constexpr int SMEM_USED = RING + WB + 32;
    static constexpr int SMEM_FLOOR = 233472 / (int)(512 / NCOLS + 1) + 1024;
    static constexpr int SMEM = SMEM_USED > SMEM_FLOOR ? SMEM_USED : SMEM_FLOOR;
    // instruction shapes of a slice of one, two or three stacked taps
    static constexpr uint32_t IDESC1 = idesc_bf16(TW, COUT), IDESC2 = idesc_bf16(TW, 2 * COUT),
                              IDESC3 = idesc_bf16(TW, 3 * COUT);
    static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "shape");
    static_assert(R == 4 || R == 8, "rows per tile");
    static_assert(ROWB % 128 == 0 && RING % 128 == 0 && WB % 16 == 0, "TMA and descriptor alignment");
    static_assert(NCOLS >= 32 && (NCOLS & (NCOLS - 1)) == 0, "TMEM allocation must be a power of two >= 32");
};

template <int CIN, int COUT, int MODE, int R>
__global__ void __launch_bounds__(NT) k_conv3x3(ConvArgs a, const __grid_constant__ CUtensorMap tmap) {
    using S = ConvShape<CIN, COUT, R>;
    constexpr int GI = S::GI, GO = S::GO, NRING = S::NRING, ROWB = S::ROWB;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* ring = smem;
    unsigned char* wsm = smem + S::RING;
    uint64_t* bar = reinterpret_cast<uint64_t*>(wsm + S::WB);  // MMA completion
    uint64_t* tbar = bar + 1;                                     // row arrival (TMA), two alternating
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    __shared__ float sbias[COUT];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int H = a.H, W = a.W;

    for (int i = tid; i < S::WB / 16; i += NT) cp_async16(wsm + i * 16, a.w + (int64_t)i * 8, 16);
    cp_async_commit();
    if (tid < COUT) sbias[tid] = (MODE == CONV_MASK || tid >= a.nbias) ? 0.f : a.bias[tid];
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(tbar, 1);
        mbar_init(tbar + 1, 1);
    }
    if (warp == 0) tmem_alloc(tslot, S::NCOLS);
    cp_async_wait_all();
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    // Tiles in column-major order (image, tile column, tile row); each CTA walks one contiguous
    // chunk, so consecutive tiles of a column share two input rows. Input row y (-1 .. H) lives in
    // ring slot (y + 1) mod NRING: a tile needs R + 2 consecutive slots, and the next tile of the
    // same column adds R rows in slots only the previous tile used. Thread 0 loads those rows (one
    // TMA copy per row, zero-filled outside the image) at the start of a tile, so they arrive while
    // the tile's products and epilogue run; at a column change the ring is reloaded once the
    // current tile's products have completed.
    const int tx = (W + TW - 1) / TW, ty = (H + R - 1) / R;
    const long long tiles = (long long)a.B * ty * tx;
    const long long chunk = (tiles + gridDim.x - 1) / gridDim.x;
    const long long u0 = (long long)blockIdx.x * chunk;
    const long long u1 = u0 + chunk < tiles ? u0 + chunk : tiles;
    auto coords = [&](long long u, int& b, int& xt, int& yt) {
        yt = (int)(u % ty);
        const long long c = u / ty;
        xt = (int)(c % tx);
        b = (int)(c / tx);
    };
    // rows [ya, yb] of tile u's column, arriving on tbar[k & 1]
    auto load_rows = [&](long long u, int ya, int yb, int k) {
        int b, xt, yt;
        coords(u, b, xt, yt);
        mbar_expect_tx(tbar + (k & 1), (uint32_t)((yb - ya + 1) * S::BOXB));
        for (int y = ya; y <= yb; ++y)
            tma_load_5d(ring + ((y + 1) % NRING) * ROWB, &tmap, 0, xt * TW - 1, 0, y, b, tbar + (k & 1));
    };
    auto same_column = [&](long long u, long long v) { return u / ty == v / ty; };
    uint32_t parity = 0, tph = 0;  // tph bit j: phase of tbar[j]
    bool ok = true, mma_pending = false;
    int pending = 0;               // bit j: a copy on tbar[j] was issued and not yet waited for
    if (tid == 0 && u0 < u1) {
        const int yt = (int)(u0 % ty);
        load_rows(u0, yt * R - 1, yt * R + R, 0);
    }
    pending = u0 < u1 ? 1 : 0;
    int k = 0;
    for (long long u = u0; u < u1; ++u, ++k) {
        int b, xt, yt;
        coords(u, b, xt, yt);
        const int y0 = yt * R, x0 = xt * TW;
        const bool next = u + 1 < u1, cont = next && same_column(u, u + 1);
        if (cont) {  // the next tile's R new rows go to slots only the previous tile read
            if (tid == 0) load_rows(u + 1, y0 + R + 1, y0 + 2 * R, k + 1);
            pending |= 1 << ((k + 1) & 1);
        }
        const int j = k & 1;
        const bool arrived = mbar_wait(tbar + j, (tph >> j) & 1u);
        tph ^= 1u << j;
        pending &= ~(1 << j);
        if (!__syncthreads_and(arrived)) {
            ok = false;
            pending |= 1 << j;  // still to be waited for (its phase bit is flipped back below)
            tph ^= 1u << j;
            break;
        }
        if (tid == 0 && !a.unsignalled) {
            tc_fence_after();
            // Descriptors advance in 16-byte units, so every operand address below is a base
            // descriptor plus a compile-time offset (the loops are unrolled): a few instructions
            // per MMA, where one thread has to keep the tensor pipe fed.
            constexpr uint32_t LBO_B = 3 * COUT * 16;  // between the 8-channel groups of a tap stack
            const uint64_t bdesc = sdesc(smem_u32(wsm), LBO_B, 128);
            const uint32_t rb = smem_u32(ring);
            int slot = y0 % NRING;  // ring slot of band row 0 (input row y0 - 1)
            // Band row rho (input row y0 - 1 + rho) feeds output rows rf..rl (dy = rho - r in 0..2);
            // the stack slice starts at the tap of the largest dy, rho - rf. Output row rho (dy = 0)
            // gets its first product at dx = 0, s = 0: that instruction is split so the row starts
            // from zero while the rows above it keep accumulating.
#pragma unroll
            for (int rho = 0; rho < R + 2; ++rho) {
                const int rf = rho > 2 ? rho - 2 : 0, rl = rho < R - 1 ? rho : R - 1;
                const int nr = rl - rf + 1;
                const uint32_t dcol = tbase + (uint32_t)(rf * COUT);
                const uint64_t arow = sdesc(rb + (uint32_t)(slot * ROWB), BANDW * 16, 128);
                slot = slot + 1 == NRING ? 0 : slot + 1;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                    for (int s = 0; s < S::KS; ++s) {
                        const uint64_t ad = arow + (uint64_t)((2 * s) * BANDW + dx);
                        const uint64_t bs = bdesc + (uint64_t)((dx * GI + 2 * s) * 3 * COUT);
                        const uint64_t bd = bs + (uint64_t)((2 - (rho - rf)) * COUT);
                        if (rho < R && dx == 0 && s == 0) {
                            if (nr > 1) tc_mma(dcol, ad, bd, nr == 3 ? S::IDESC2 : S::IDESC1, 1u);
                            tc_mma(tbase + (uint32_t)(rho * COUT), ad, bs + (uint64_t)(2 * COUT), S::IDESC1, 0u);
                        } else {
                            tc_mma(dcol, ad, bd, nr == 3 ? S::IDESC3 : (nr == 2 ? S::IDESC2 : S::IDESC1), 1u);
                        }
                    }
                }
            }
            tc_commit(bar);
        }
        const bool done = mbar_wait(bar, parity);
        parity ^= 1u;
        ok = __syncthreads_and(done);
        tc_fence_after();
        if (!ok) {
            mma_pending = !a.unsignalled;
            break;
        }
        if (next && !cont) {  // a new column: every slot is free once the products have completed
            int b1, xt1, yt1;
            coords(u + 1, b1, xt1, yt1);
            if (tid == 0) load_rows(u + 1, yt1 * R - 1, yt1 * R + R, k + 1);
            pending |= 1 << ((k + 1) & 1);
        }
        // epilogue: thread tid holds pixel x0 + tid of each accumulator row
#pragma unroll 1
        for (int r = 0; r < R; ++r) {
            float v[COUT];
            const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * COUT);
            if (COUT == 32) tmem_ld32(ta, v);
            else tmem_ld16(ta, v);
            const int y = y0 + r, x = x0 + tid;
            if (y >= H || x >= W) continue;
            const int64_t pix = ((int64_t)b * H + y);
            if constexpr (MODE == CONV_LAST) {
                a.outf[pix * W + x] = v[0] + sbias[0];
            } else {
#pragma unroll
            for (int g = 0; g < GO; ++g) {
                const int64_t off = ((pix * GO + g) * W + x) * 8;
                float m[8];
                if (MODE == CONV_MASK) {
                    const uint4 mv = *reinterpret_cast<const uint4*>(a.mask + off);
                    const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        m[2 * e] = __uint_as_float(mw[e] << 16);
                        m[2 * e + 1] = __uint_as_float(mw[e] & 0xFFFF0000u);
                    }
                }
                float o[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float z = v[8 * g + e] + sbias[8 * g + e];
                    o[e] = (MODE == CONV_RELU) ? fmaxf(z, 0.f) : (m[e] > 0.f ? z : 0.f);
                }
                uint4 st;
                st.x = pack_bf16x2(o[0], o[1]);
                st.y = pack_bf16x2(o[2], o[3]);
                st.z = pack_bf16x2(o[4], o[5]);
                st.w = pack_bf16x2(o[6], o[7]);
                *reinterpret_cast<uint4*>(a.out + off) = st;
            }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        // a row copy or an MMA batch did not report completion in time: record it, give every copy
        // still in flight and the MMA batch one more bounded wait (on the phase each was issued in)
        // before shared and tensor memory are released, and leave (the self-test issues no MMA, so
        // there is no batch to wait for)
        if (tid == 0) atomicExch(a.err, 1);
        for (int j = 0; j < 2; ++j)
            if (pending & (1 << j)) mbar_wait(tbar + j, (tph >> j) & 1u);
        if (mma_pending) mbar_wait(bar, parity ^ 1u);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tbase, S::NCOLS);
}

// ---- weight packing -------------------------------------------------------------------------
// Taps (p, q) = (row, column) offsets, stacked per column offset q in the order p = 2, 1, 0:
// Forward: packed[((q*GI + ci/8)*3*COUTP + (2-p)*COUTP + co)*8 + ci%8] = bf16(W[co][ci][p][q]).
// Transposed (the data gradient of the layer is a convolution from its O outputs back to its C
// inputs with the kernel flipped in space): the same layout with O and C exchanged holding
// bf16(W[o][c][2-p][2-q]). Zero for padded channels.
__global__ void k_pack(const float* W, int O, int C, int cinp, int coutp, int transposed, bf16* out) {
    const int total = 9 * cinp * coutp;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int e = idx % 8, row = (idx / 8) % (3 * coutp), g = (idx / (8 * 3 * coutp)) % (cinp / 8),
              q = idx / (8 * 3 * coutp * (cinp / 8));
    const int n = row % coutp, p = 2 - row / coutp;
    const int k = 8 * g + e;
    float v = 0.f;
    if (!transposed) {
        if (n < O && k < C) v = W[((n * C + k) * 3 + p) * 3 + q];
    } else {
        if (k < O && n < C) v = W[((k * C + n) * 3 + (2 - p)) * 3 + (2 - q)];
    }
    out[idx] = __float2bfloat16_rn(v);
}

// ---- loss -----------------------------------------------------------------------------------
// part[block] = sum (y - t)^2; g (16-channel image) channel 0 = scale (y - t), other channels 0.
__global__ void k_loss(const float* y, const float* t, int B, int H, int W, float scale, bf16* g, double* part) {
    __shared__ double sh[8];
    const int64_t n = (int64_t)B * H * W;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        acc += (double)d * d;
        const int64_t x = i % W, row = i / W;
        uint4 c0 = make_uint4(pack_bf16x2(scale * d, 0.f), 0u, 0u, 0u), z = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(g + ((row * 2 + 0) * W + x) * 8) = c0;
        *reinterpret_cast<uint4*>(g + ((row * 2 + 1) * W + x) * 8) = z;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

// ---- residual loss ----------------------------------------------------------------------------
// The proposal y leaves the residual res(p) = x_0(p) - (y(p) - sum_q w_q(p) y(q)) at an inner pixel
// p of a patch (not on its border), in the network's units: x_0 = h^2 r / (D rho) is the scaled
// residual, and w_q(p) = k_pq / D(p) the Jacobi-scaled operator rebuilt from the patch's own log k
// channel (k = exp(x_1), faces k_pq the harmonic means, D(p) their sum; W, E, S, N = column - 1,
// column + 1, row - 1, row + 1). Loss: (1/N) sum res^2 over the N inner pixels of the batch.
// Pass 1 writes per pixel [res, w_W, w_E, w_S, w_N] (zeros on the border) and the partial sums of
// res^2; pass 2 forms dL/dy(q) = (2/N) (-res(q) + sum over the inner neighbours p of q of w(p) res(p),
// w(p) the weight p gives q) and writes it as channel 0 of the gradient image.
__device__ __forceinline__ float img_ch(const bf16* x, int b, int H, int W, int yy, int xx, int c) {
    return __bfloat162float(x[(((int64_t)b * H + yy) * 2 + c / 8) * W * 8 + (int64_t)xx * 8 + c % 8]);
}

__global__ void k_loss_resid_a(const float* y, const bf16* x, int B, int H, int W, float* R, double* part) {
    __shared__ double sh[8];
    const int64_t n = (int64_t)B * H * W;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / ((int64_t)H * W));
        const int rem = (int)(i % ((int64_t)H * W));
        const int r = rem / W, c = rem % W;
        float* o = R + 5 * i;
        if (r == 0 || c == 0 || r == H - 1 || c == W - 1) {
            o[0] = o[1] = o[2] = o[3] = o[4] = 0.f;
            continue;
        }
        const float kp = expf(img_ch(x, b, H, W, r, c, 1));
        const float kq[4] = {expf(img_ch(x, b, H, W, r, c - 1, 1)), expf(img_ch(x, b, H, W, r, c + 1, 1)),
                             expf(img_ch(x, b, H, W, r - 1, c, 1)), expf(img_ch(x, b, H, W, r + 1, c, 1))};
        float f[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) f[q] = ((2.f * kp) * kq[q]) / (kp + kq[q]);
        const float D = ((f[0] + f[1]) + f[2]) + f[3];
        const float w[4] = {f[0] / D, f[1] / D, f[2] / D, f[3] / D};
        const float* yb = y + (int64_t)b * H * W;
        const float ay = yb[r * W + c] - (((w[0] * yb[r * W + c - 1] + w[1] * yb[r * W + c + 1]) + w[2] * yb[(r - 1) * W + c]) +
                                          w[3] * yb[(r + 1) * W + c]);
        const float res = img_ch(x, b, H, W, r, c, 0) - ay;
        o[0] = res;
        o[1] = w[0];
        o[2] = w[1];
        o[3] = w[2];
        o[4] = w[3];
        acc += (double)res * res;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_loss_resid_b(const float* R, int B, int H, int W, float scale, bf16* g) {
    const int64_t n = (int64_t)B * H * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int rem = (int)(i % ((int64_t)H * W));
        const int r = rem / W, c = rem % W;
        float d = -R[5 * i];
        if (c + 1 < W) d += R[5 * (i + 1) + 1] * R[5 * (i + 1)];       // q is the west neighbour of (r, c+1)
        if (c - 1 >= 0) d += R[5 * (i - 1) + 2] * R[5 * (i - 1)];      // ... the east neighbour of (r, c-1)
        if (r + 1 < H) d += R[5 * (i + W) + 3] * R[5 * (i + W)];       // ... the south neighbour of (r+1, c)
        if (r - 1 >= 0) d += R[5 * (i - W) + 4] * R[5 * (i - W)];      // ... the north neighbour of (r-1, c)
        const int64_t x = i % W, row = i / W;
        uint4 c0 = make_uint4(pack_bf16x2(scale * d, 0.f), 0u, 0u, 0u), z = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(g + ((row * 2 + 0) * W + x) * 8) = c0;
        *reinterpret_cast<uint4*>(g + ((row * 2 + 1) * W + x) * 8) = z;
    }
}

// ---- weight gradient (CUDA cores) -------------------------------------------------------------
// dW[o][c][p][q] += sum over pixels g[o](y, x) a[c](y + p - 1, x + q - 1); db[o] += sum g[o].
// A block takes 32-pixel row segments; each thread owns a fixed set of (o, c, p, q) outputs and
// accumulates them in registers over its segments, then adds them to the global sums.
constexpr int WG_THREADS = 256;
constexpr int WG_PX = 32;

template <int CI, int CIP, int CO, int COP>
__global__ void __launch_bounds__(WG_THREADS) k_wgrad(const bf16* act, const bf16* g, int B, int H, int W, float* dW,
                                                     float* db) {
    constexpr int NW = CO * CI * 9, NOUT = NW + CO;
    constexpr int PER = (NOUT + WG_THREADS - 1) / WG_THREADS;
    __shared__ float sg[CO][WG_PX];
    __shared__ float sa[CI][3][WG_PX + 2];
    float acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.f;
    const int tid = threadIdx.x;
    const int segs = (W + WG_PX - 1) / WG_PX;
    const long long tiles = (long long)B * H * segs;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int s = (int)(t % segs);
        const long long row = t / segs;
        const int b = (int)(row / H), y = (int)(row % H), x0 = s * WG_PX;
        for (int i = tid; i < CO * WG_PX; i += WG_THREADS) {
            const int o = i / WG_PX, px = i % WG_PX, x = x0 + px;
            float v = 0.f;
            if (x < W) v = __bfloat162float(g[((((int64_t)b * H + y) * (COP / 8) + o / 8) * W + x) * 8 + o % 8]);
            sg[o][px] = v;
        }
        for (int i = tid; i < CI * 3 * (WG_PX + 2); i += WG_THREADS) {
            const int c = i / (3 * (WG_PX + 2)), p = (i / (WG_PX + 2)) % 3, px = i % (WG_PX + 2);
            const int yy = y + p - 1, xx = x0 + px - 1;
            float v = 0.f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                v = __bfloat162float(act[((((int64_t)b * H + yy) * (CIP / 8) + c / 8) * W + xx) * 8 + c % 8]);
            sa[c][p][px] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int idx = tid + k * WG_THREADS;
            if (idx < NW) {
                const int q = idx % 3, p = (idx / 3) % 3, c = (idx / 9) % CI, o = idx / (9 * CI);
                float s2 = 0.f;
#pragma unroll 8
                for (int px = 0; px < WG_PX; ++px) s2 = fmaf(sg[o][px], sa[c][p][px + q], s2);
                acc[k] += s2;
            } else if (idx < NOUT) {
                const int o = idx - NW;
                float s2 = 0.f;
                for (int px = 0; px < WG_PX; ++px) s2 += sg[o][px];
                acc[k] += s2;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int idx = tid + k * WG_THREADS;
        if (idx < NW) atomicAdd(dW + idx, acc[k]);
        else if (idx < NOUT) atomicAdd(db + (idx - NW), acc[k]);
    }
}

// ---- Adam -----------------------------------------------------------------------------------
__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ---- patches --------------------------------------------------------------------------------
__global__ void k_gather(const bf16* x, const float* t, int H, int W, const int32_t* corners, int B, int P, bf16* xp,
                         float* tp) {
    const int64_t n = (int64_t)B * P * P;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int px = (int)(i % P), py = (int)((i / P) % P), b = (int)(i / ((int64_t)P * P));
    const int y = corners[2 * b] + py, xx = corners[2 * b + 1] + px;
    for (int g = 0; g < 2; ++g) {
        const uint4 v = *reinterpret_cast<const uint4*>(x + (((int64_t)y * 2 + g) * W + xx) * 8);
        *reinterpret_cast<uint4*>(xp + ((((int64_t)b * P + py) * 2 + g) * P + px) * 8) = v;
    }
    tp[i] = t[(int64_t)y * W + xx];
}

// ---- solver-side features -------------------------------------------------------------------
template <typename T> __device__ __forceinline__ double ldd(const T* p) { return (double)*p; }
template <> __device__ __forceinline__ double ldd<bf16>(const bf16* p) { return (double)__bfloat162float(*p); }

__device__ __forceinline__ double diag_at(const double* kx, const double* ky, int64_t kp, int i, int j) {
    return ((kx[(int64_t)j * kp + i - 1] + kx[(int64_t)j * kp + i]) + ky[(int64_t)(j - 1) * kp + i]) + ky[(int64_t)j * kp + i];
}

constexpr int FB = 256;

template <typename T>
__global__ void __launch_bounds__(FB) k_feat_stats(const T* g0, int64_t pg, const double* kx, const double* ky, int64_t kp,
                                                   int n, double* part) {
    __shared__ double sh[FB / 32];
    double acc = 0.0;
    const int64_t m = (int64_t)(n - 1) * (n - 1);
    for (int64_t q = blockIdx.x * (int64_t)FB + threadIdx.x; q < m; q += (int64_t)gridDim.x * FB) {
        const int i = (int)(q % (n - 1)) + 1, j = (int)(q / (n - 1)) + 1;
        const double z = ldd(g0 + (int64_t)j * pg + i) / diag_at(kx, ky, kp, i, j);
        acc = fma(z, z, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < FB / 32; ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_reduce(const double* part, int nparts, double count, double* out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = (count > 0.0) ? sqrt(t / count) : t;
    }
}

template <typename T>
__global__ void k_feat_write(const T* g0, int64_t pg, const double* kx, const double* ky, int64_t kp, int n,
                             const double* rho, const uint16_t* logk, bf16* x) {
    const int64_t side = n + 1, m = side * side;
    const double r = *rho;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % side), j = (int)(q / side);
        float x0 = 0.f;
        if (i > 0 && j > 0 && i < n && j < n) x0 = (float)((ldd(g0 + (int64_t)j * pg + i) / diag_at(kx, ky, kp, i, j)) / r);
        // x0 is rounded twice (binary64 -> binary32 -> bfloat16); see the feature test's tolerance
        uint4 c;
        c.x = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x0)) | ((uint32_t)logk[q] << 16);
        c.y = c.z = c.w = 0u;
        *reinterpret_cast<uint4*>(x + (((int64_t)j * 2) * side + i) * 8) = c;
        *reinterpret_cast<uint4*>(x + (((int64_t)j * 2 + 1) * side + i) * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void k_target(const double* uref, const double* u, int n, const double* rho, float* t) {
    const int64_t side = n + 1, m = side * side;
    const double r = *rho;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % side), j = (int)(q / side);
        t[q] = (i > 0 && j > 0 && i < n && j < n) ? (float)((uref[q] - u[q]) / r) : 0.f;
    }
}

template <typename T> __device__ __forceinline__ T from_double(double v) { return (T)v; }
template <> __device__ __forceinline__ bf16 from_double<bf16>(double v) { return __float2bfloat16_rn((float)v); }

template <typename T>
__global__ void k_correct(const float* y, int n, const double* rho, T* e, int64_t pitch) {
    const int64_t side = n + 1, m = side * side;
    const double r = *rho;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % side), j = (int)(q / side);
        const bool in = (i > 0 && j > 0 && i < n && j < n);
        e[(int64_t)j * pitch + i] = from_double<T>(in ? r * (double)y[q] : 0.0);
    }
}

__global__ void k_logk(const double* k, int64_t m, uint16_t* out) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = __bfloat16_as_ushort(__float2bfloat16_rn((float)log(k[q])));
}

// ---- host helpers ---------------------------------------------------------------------------
int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// cuTensorMapEncodeTiled, obtained once through the runtime's driver entry-point query.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// The row tensor map of a row-chunked [B, 8 G, H, W] bf16 tensor: dims (8, W, G, H, B), box
// (8, 130, G, 1, 1) -- one staged input row --, zero fill outside.
cudaError_t band_tensor_map(CUtensorMap* map, const bf16* base, int B, int H, int W, int G) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)G, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[4] = {16, (cuuint64_t)W * 16, (cuuint64_t)G * W * 16, (cuuint64_t)H * G * W * 16};
    const cuuint32_t box[5] = {8, BANDW, (cuuint32_t)G, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CIN, int COUT, int MODE, int R>
cudaError_t launch_conv_r(const ConvArgs& a, cudaStream_t s) {
    using S = ConvShape<CIN, COUT, R>;
    static int per_sm = 0;
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3<CIN, COUT, MODE, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_conv3x3<CIN, COUT, MODE, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        // CTAs per SM: as many as the 228 KB of shared memory hold (1 KB reserved per CTA), never
        // more than the SM's 512 TMEM columns hold together
        per_sm = 233472 / (S::SMEM + 1024);
        per_sm = per_sm < (int)(512 / S::NCOLS) ? per_sm : (int)(512 / S::NCOLS);
        if (per_sm < 1) per_sm = 1;
    }
    const long long tiles = (long long)a.B * ((a.H + R - 1) / R) * ((a.W + TW - 1) / TW);
    const long long cap = (long long)num_sms() * per_sm;
    const int grid = (int)(tiles < cap ? tiles : cap);
    CUtensorMap map;
    cudaError_t e = band_tensor_map(&map, a.in, a.B, a.H, a.W, CIN / 8);
    if (e != cudaSuccess) return e;
    k_conv3x3<CIN, COUT, MODE, R><<<grid, NT, S::SMEM, s>>>(a, map);
    return cudaGetLastError();
}

template <int CIN, int COUT, int MODE>
cudaError_t launch_conv(const ConvArgs& a, cudaStream_t s) {
    return a.rows == 8 ? launch_conv_r<CIN, COUT, MODE, 8>(a, s) : launch_conv_r<CIN, COUT, MODE, 4>(a, s);
}

}  // namespace

// ---- network handle ---------------------------------------------------------------------------
namespace {
constexpr int kIn = HOMG_NET_IN, kWidth = HOMG_NET_WIDTH;
// per layer: (out, in) real channels, padded input / output channels
constexpr int kO[4] = {kWidth, kWidth, kWidth, 1};
constexpr int kC[4] = {kIn, kWidth, kWidth, kWidth};
constexpr int kCinP[4] = {16, 32, 32, 32};
constexpr int kCoutP[4] = {32, 32, 32, 16};

int64_t param_offset(int l) {
    int64_t off = 0;
    for (int k = 0; k < l; ++k) off += (int64_t)kO[k] * kC[k] * 9 + kO[k];
    return off;
}
thread_local char g_net_error[512] = "";
}  // namespace

struct homg_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    int64_t np = 0;
    float* params = nullptr;  // device binary32 master parameters
    float* grads = nullptr;
    float* am = nullptr;
    float* av = nullptr;
    bf16* wf[4] = {};  // packed forward weights
    bf16* wt[4] = {};  // packed transposed weights (layers 1..3)
    int step = 0;
    int64_t cap_px = 0;  // pixels the activation scratch holds
    bf16* act[3] = {};   // hidden activations a1..a3 ([*, 32, H, W])
    bf16* gA = nullptr;  // gradients ([*, 32, H, W])
    bf16* gB = nullptr;
    bf16* g4 = nullptr;  // last-layer gradient ([*, 16, H, W])
    float* y = nullptr;  // training output
    float* lres = nullptr;  // residual loss: [res, w_W, w_E, w_S, w_N] per pixel
    int loss_kind = HOMG_NET_LOSS_ERROR;
    int tile_rows = 4;  // output rows per convolution tile (4 or 8)
    double* part = nullptr;
    double* dloss = nullptr;
    int* derr = nullptr;
    char err[512] = "";
};

namespace {

constexpr int kLossBlocks = 1024;

int net_fail(homg_net* net, int code, const char* msg, const char* extra = "") {
    snprintf(net ? net->err : g_net_error, 512, "%s%s", msg, extra);
    return code;
}
int net_cuda(homg_net* net, cudaError_t e, const char* where) {
    cudaGetLastError();
    char buf[400];
    snprintf(buf, sizeof(buf), "CUDA error in %s: ", where);
    return net_fail(net, e == cudaErrorMemoryAllocation ? HOMG_ENOMEM : HOMG_ECUDA, buf, cudaGetErrorString(e));
}
#define NCK(net, call, where)                                    \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return net_cuda(net, e_, where);  \
    } while (0)

cudaError_t repack(homg_net* n, cudaStream_t s) {
    for (int l = 0; l < 4; ++l) {
        const float* W = n->params + param_offset(l);
        const int total = 9 * kCinP[l] * kCoutP[l];
        k_pack<<<(total + 255) / 256, 256, 0, s>>>(W, kO[l], kC[l], kCinP[l], kCoutP[l], 0, n->wf[l]);
        if (l >= 1) {
            // data gradient of layer l: from its padded outputs (as inputs) back to its inputs
            const int cinp = (kO[l] + 15) / 16 * 16, coutp = kC[l];
            const int tt = 9 * cinp * coutp;
            k_pack<<<(tt + 255) / 256, 256, 0, s>>>(W, kO[l], kC[l], cinp, coutp, 1, n->wt[l]);
        }
    }
    return cudaGetLastError();
}

int ensure_scratch(homg_net* n, int64_t px) {
    if (px <= n->cap_px) return HOMG_OK;
    for (auto*& p : n->act) { if (p) cudaFree(p); p = nullptr; }
    if (n->gA) cudaFree(n->gA);
    if (n->gB) cudaFree(n->gB);
    if (n->g4) cudaFree(n->g4);
    if (n->y) cudaFree(n->y);
    if (n->lres) cudaFree(n->lres);
    n->gA = n->gB = n->g4 = nullptr;
    n->y = nullptr;
    n->lres = nullptr;
    n->cap_px = 0;
    for (auto*& p : n->act) NCK(n, cudaMalloc(&p, (size_t)px * 32 * sizeof(bf16)), "allocating activations");
    NCK(n, cudaMalloc(&n->gA, (size_t)px * 32 * sizeof(bf16)), "allocating gradients");
    NCK(n, cudaMalloc(&n->gB, (size_t)px * 32 * sizeof(bf16)), "allocating gradients");
    NCK(n, cudaMalloc(&n->g4, (size_t)px * 16 * sizeof(bf16)), "allocating gradients");
    NCK(n, cudaMalloc(&n->y, (size_t)px * sizeof(float)), "allocating outputs");
    NCK(n, cudaMalloc(&n->lres, (size_t)px * 5 * sizeof(float)), "allocating the residual-loss scratch");
    n->cap_px = px;
    return HOMG_OK;
}

ConvArgs conv_args(homg_net* n, const bf16* in, int l, bf16* out, float* outf, int B, int H, int W) {
    ConvArgs a{};
    a.in = in;
    a.w = n->wf[l];
    a.bias = n->params + param_offset(l) + (int64_t)kO[l] * kC[l] * 9;
    a.nbias = kO[l];
    a.out = out;
    a.outf = outf;
    a.B = B;
    a.H = H;
    a.W = W;
    a.err = n->derr;
    a.rows = n->tile_rows;
    return a;
}

// forward into act[0..2] (training keeps all three) or ping-pong (inference)
int forward(homg_net* n, const bf16* x, int B, int H, int W, float* y, bool keep, cudaStream_t s) {
    bf16* a1 = n->act[0];
    bf16* a2 = n->act[1];
    bf16* a3 = keep ? n->act[2] : n->act[0];
    NCK(n, (launch_conv<16, 32, CONV_RELU>(conv_args(n, x, 0, a1, nullptr, B, H, W), s)), "conv layer 1");
    NCK(n, (launch_conv<32, 32, CONV_RELU>(conv_args(n, a1, 1, a2, nullptr, B, H, W), s)), "conv layer 2");
    NCK(n, (launch_conv<32, 32, CONV_RELU>(conv_args(n, a2, 2, a3, nullptr, B, H, W), s)), "conv layer 3");
    NCK(n, (launch_conv<32, 16, CONV_LAST>(conv_args(n, a3, 3, nullptr, y, B, H, W), s)), "conv layer 4");
    return HOMG_OK;
}

bool dims_ok(int B, int H, int W) { return B >= 1 && H >= 1 && W >= 1 && (long long)B * H * W < (1ll << 31); }

}  // namespace

namespace homg {

int net_forward_dev(homg_net* net, const void* x, int B, int H, int W, float* y, cudaStream_t s) {
    if (!net || !x || !y || !dims_ok(B, H, W)) return HOMG_EINVAL;
    int rc = ensure_scratch(net, (int64_t)B * H * W);
    if (rc != HOMG_OK) return rc;
    return forward(net, static_cast<const bf16*>(x), B, H, W, y, false, s);
}

int net_check_error(homg_net* net) {
    int e = 0;
    if (cudaMemcpy(&e, net->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HOMG_ECUDA;
    if (e) {
        cudaMemset(net->derr, 0, sizeof(int));
        return net_fail(net, HOMG_ECUDA, "a network kernel timed out waiting for its tensor-core barrier");
    }
    return HOMG_OK;
}

int feat_parts(int n) {
    const int64_t m = (int64_t)(n - 1) * (n - 1);
    const int64_t b = (m + FB - 1) / FB;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

#define NET_DISPATCH(prec, CALL)                                 \
    switch (prec) {                                              \
        case PREC_FP64: { using T = double; CALL; break; }       \
        case PREC_FP32: { using T = float; CALL; break; }        \
        case PREC_BF16: { using T = bf16; CALL; break; }         \
        default: return cudaErrorInvalidValue;                   \
    }

cudaError_t launch_feat_stats(int prec, const void* g0, int64_t pitch_g, const double* kx0, const double* ky0,
                              int64_t kpitch, int n, double* part, cudaStream_t s) {
    const int blocks = feat_parts(n);
    NET_DISPATCH(prec, (k_feat_stats<T><<<blocks, FB, 0, s>>>(static_cast<const T*>(g0), pitch_g, kx0, ky0, kpitch, n, part)));
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double* part, int nparts, double count, double* out, cudaStream_t s) {
    k_reduce<<<1, 1024, 0, s>>>(part, nparts, count, out);
    return cudaGetLastError();
}

cudaError_t launch_feat_write(int prec, const void* g0, int64_t pitch_g, const double* kx0, const double* ky0,
                              int64_t kpitch, int n, const double* rho, const uint16_t* logk, void* x, cudaStream_t s) {
    const int blocks = num_sms() * 8;
    NET_DISPATCH(prec, (k_feat_write<T><<<blocks, 256, 0, s>>>(static_cast<const T*>(g0), pitch_g, kx0, ky0, kpitch, n,
                                                                 rho, logk, static_cast<bf16*>(x))));
    return cudaGetLastError();
}

cudaError_t launch_target(const double* uref, const double* u, int n, const double* rho, float* t, cudaStream_t s) {
    k_target<<<num_sms() * 8, 256, 0, s>>>(uref, u, n, rho, t);
    return cudaGetLastError();
}

cudaError_t launch_correct(int prec, const float* y, int n, const double* rho, void* e, int64_t pitch, cudaStream_t s) {
    NET_DISPATCH(prec, (k_correct<T><<<num_sms() * 8, 256, 0, s>>>(y, n, rho, static_cast<T*>(e), pitch)));
    return cudaGetLastError();
}

cudaError_t launch_logk(const double* k, int n, uint16_t* out, cudaStream_t s) {
    k_logk<<<num_sms() * 8, 256, 0, s>>>(k, (int64_t)(n + 1) * (n + 1), out);
    return cudaGetLastError();
}

}  // namespace homg

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" {

int64_t homg_net_param_count(void) { return param_offset(4); }

int homg_net_create(homg_net_handle* out) {
    if (out) *out = nullptr;
    g_net_error[0] = 0;
    if (!out) return net_fail(nullptr, HOMG_EINVAL, "homg_net_create: null out");
    homg_net* n = new (std::nothrow) homg_net();
    if (!n) return net_fail(nullptr, HOMG_ENOMEM, "homg_net_create: out of host memory");
    cudaGetDevice(&n->device);
    n->np = param_offset(4);
    cudaError_t e = cudaSuccess;
    for (float** p : {&n->params, &n->grads, &n->am, &n->av})
        if (e == cudaSuccess) e = cudaMalloc(p, (size_t)n->np * sizeof(float));
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        e = cudaMalloc(&n->wf[l], (size_t)9 * kCinP[l] * kCoutP[l] * sizeof(bf16));
        if (e == cudaSuccess && l >= 1) e = cudaMalloc(&n->wt[l], (size_t)9 * 16 * 32 * 2 * sizeof(bf16));
    }
    if (e == cudaSuccess) e = cudaMalloc(&n->part, kLossBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&n->dloss, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&n->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(n->derr, 0, sizeof(int));
    for (float* p : {n->params, n->grads, n->am, n->av})
        if (e == cudaSuccess) e = cudaMemset(p, 0, (size_t)n->np * sizeof(float));
    if (e == cudaSuccess) e = repack(n, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        net_cuda(nullptr, e, "homg_net_create");
        homg_net_destroy(n);
        return e == cudaErrorMemoryAllocation ? HOMG_ENOMEM : HOMG_ECUDA;
    }
    *out = n;
    return HOMG_OK;
}

int homg_net_set_stream(homg_net_handle net, void* stream) {
    if (!net) return HOMG_EINVAL;
    net->stream = (cudaStream_t)stream;
    return HOMG_OK;
}

int homg_net_set_params(homg_net_handle net, const float* params, int64_t count) {
    if (!net) return HOMG_EINVAL;
    if (!params || count != net->np) return net_fail(net, HOMG_EINVAL, "homg_net_set_params: need homg_net_param_count() values");
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    NCK(net, cudaMemcpyAsync(net->params, params, (size_t)count * sizeof(float), cudaMemcpyHostToDevice, net->stream),
        "cudaMemcpyAsync");
    NCK(net, cudaMemsetAsync(net->am, 0, (size_t)count * sizeof(float), net->stream), "cudaMemsetAsync");
    NCK(net, cudaMemsetAsync(net->av, 0, (size_t)count * sizeof(float), net->stream), "cudaMemsetAsync");
    NCK(net, repack(net, net->stream), "packing weights");
    NCK(net, cudaStreamSynchronize(net->stream), "cudaStreamSynchronize");
    net->step = 0;
    return HOMG_OK;
}

int homg_net_get_params(homg_net_handle net, float* params, int64_t count) {
    if (!net) return HOMG_EINVAL;
    if (!params || count != net->np) return net_fail(net, HOMG_EINVAL, "homg_net_get_params: need homg_net_param_count() values");
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    NCK(net, cudaMemcpyAsync(params, net->params, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost, net->stream),
        "cudaMemcpyAsync");
    NCK(net, cudaStreamSynchronize(net->stream), "cudaStreamSynchronize");
    return HOMG_OK;
}

int homg_net_get_grads(homg_net_handle net, float* grads, int64_t count) {
    if (!net) return HOMG_EINVAL;
    if (!grads || count != net->np) return net_fail(net, HOMG_EINVAL, "homg_net_get_grads: need homg_net_param_count() values");
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    NCK(net, cudaMemcpyAsync(grads, net->grads, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost, net->stream),
        "cudaMemcpyAsync");
    NCK(net, cudaStreamSynchronize(net->stream), "cudaStreamSynchronize");
    return HOMG_OK;
}

int homg_net_forward(homg_net_handle net, const void* x, int B, int H, int W, float* y) {
    if (!net) return HOMG_EINVAL;
    if (!x || !y || !dims_ok(B, H, W)) return net_fail(net, HOMG_EINVAL, "homg_net_forward: null pointer or bad sizes");
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    int rc = homg::net_forward_dev(net, x, B, H, W, y, net->stream);
    if (rc != HOMG_OK) return rc;
    NCK(net, cudaStreamSynchronize(net->stream), "cudaStreamSynchronize");
    return homg::net_check_error(net);
}

int homg_net_train_step(homg_net_handle net, const void* xv, const float* t, int B, int H, int W, float lr,
                        float* loss_out) {
    if (!net) return HOMG_EINVAL;
    const bool resid = net->loss_kind == HOMG_NET_LOSS_RESIDUAL;
    if (!xv || (!t && !resid) || !dims_ok(B, H, W) || !(lr > 0.f) || (resid && (H < 3 || W < 3)))
        return net_fail(net, HOMG_EINVAL, "homg_net_train_step: null pointer, bad sizes or lr <= 0");
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    const int64_t px = (int64_t)B * H * W;
    int rc = ensure_scratch(net, px);
    if (rc != HOMG_OK) return rc;
    cudaStream_t s = net->stream;
    const bf16* x = static_cast<const bf16*>(xv);
    rc = forward(net, x, B, H, W, net->y, true, s);
    if (rc != HOMG_OK) return rc;
    const int lb = (int)((px + 255) / 256 < kLossBlocks ? (px + 255) / 256 : kLossBlocks);
    // loss terms: every pixel (error loss) or the inner pixels of every patch (residual loss)
    const int64_t nl = resid ? (int64_t)B * (H - 2) * (W - 2) : px;
    if (resid) {
        k_loss_resid_a<<<lb, 256, 0, s>>>(net->y, x, B, H, W, net->lres, net->part);
        k_loss_resid_b<<<lb, 256, 0, s>>>(net->lres, B, H, W, (float)(2.0 / (double)nl), net->g4);
    } else {
        k_loss<<<lb, 256, 0, s>>>(net->y, t, B, H, W, (float)(2.0 / (double)px), net->g4, net->part);
    }
    NCK(net, cudaGetLastError(), "loss kernel");
    NCK(net, homg::launch_reduce(net->part, lb, 0.0, net->dloss, s), "loss reduction");
    NCK(net, cudaMemsetAsync(net->grads, 0, (size_t)net->np * sizeof(float), s), "cudaMemsetAsync");
    auto dW = [&](int l) { return net->grads + param_offset(l); };
    auto db = [&](int l) { return net->grads + param_offset(l) + (int64_t)kO[l] * kC[l] * 9; };
    const long long segs = (long long)B * H * ((W + WG_PX - 1) / WG_PX);
    const int wgrid = (int)(segs < (long long)num_sms() * 4 ? segs : (long long)num_sms() * 4);
    // layer 4: inputs a3 (32 channels), gradient g4 (1 real of 16)
    k_wgrad<32, 32, 1, 16><<<wgrid, WG_THREADS, 0, s>>>(net->act[2], net->g4, B, H, W, dW(3), db(3));
    ConvArgs c{};
    c.B = B;
    c.H = H;
    c.W = W;
    c.err = net->derr;
    c.rows = net->tile_rows;
    c.in = net->g4;
    c.w = net->wt[3];
    c.out = net->gA;
    c.mask = net->act[2];
    NCK(net, (launch_conv<16, 32, CONV_MASK>(c, s)), "data gradient layer 4");
    k_wgrad<32, 32, 32, 32><<<wgrid, WG_THREADS, 0, s>>>(net->act[1], net->gA, B, H, W, dW(2), db(2));
    c.in = net->gA;
    c.w = net->wt[2];
    c.out = net->gB;
    c.mask = net->act[1];
    NCK(net, (launch_conv<32, 32, CONV_MASK>(c, s)), "data gradient layer 3");
    k_wgrad<32, 32, 32, 32><<<wgrid, WG_THREADS, 0, s>>>(net->act[0], net->gB, B, H, W, dW(1), db(1));
    c.in = net->gB;
    c.w = net->wt[1];
    c.out = net->gA;
    c.mask = net->act[0];
    NCK(net, (launch_conv<32, 32, CONV_MASK>(c, s)), "data gradient layer 2");
    k_wgrad<2, 16, 32, 32><<<wgrid, WG_THREADS, 0, s>>>(x, net->gA, B, H, W, dW(0), db(0));
    NCK(net, cudaGetLastError(), "weight gradient kernels");
    net->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float bc1 = (float)(1.0 - pow(b1, net->step)), bc2 = (float)(1.0 - pow(b2, net->step));
    const int np = (int)net->np;
    k_adam<<<(np + 255) / 256, 256, 0, s>>>(net->params, net->grads, net->am, net->av, np, lr, (float)b1, (float)b2, 1e-8f,
                                            bc1, bc2);
    NCK(net, cudaGetLastError(), "Adam kernel");
    NCK(net, repack(net, s), "packing weights");
    double loss = 0.0;
    NCK(net, cudaMemcpyAsync(&loss, net->dloss, sizeof(double), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    NCK(net, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (loss_out) *loss_out = (float)(loss / (double)nl);
    return homg::net_check_error(net);
}

int homg_net_set_loss(homg_net_handle net, int kind) {
    if (!net) return HOMG_EINVAL;
    if (kind != HOMG_NET_LOSS_ERROR && kind != HOMG_NET_LOSS_RESIDUAL)
        return net_fail(net, HOMG_EINVAL, "homg_net_set_loss: kind must be HOMG_NET_LOSS_ERROR or HOMG_NET_LOSS_RESIDUAL");
    net->loss_kind = kind;
    return HOMG_OK;
}

int homg_net_set_tile_rows(homg_net_handle net, int rows) {
    if (!net) return HOMG_EINVAL;
    if (rows != 4 && rows != 8) return net_fail(net, HOMG_EINVAL, "homg_net_set_tile_rows: rows must be 4 or 8");
    net->tile_rows = rows;
    return HOMG_OK;
}

int homg_net_check_barrier_timeout(homg_net_handle net, double* waited_ms) {
    if (!net || !waited_ms) return HOMG_EINVAL;
    NCK(net, cudaSetDevice(net->device), "cudaSetDevice");
    int rc = ensure_scratch(net, 16 * 16);
    if (rc != HOMG_OK) return rc;
    cudaEvent_t e0, e1;
    NCK(net, cudaEventCreate(&e0), "cudaEventCreate");
    NCK(net, cudaEventCreate(&e1), "cudaEventCreate");
    ConvArgs c = conv_args(net, net->act[0], 1, net->act[1], nullptr, 1, 16, 16);
    c.unsignalled = 1;
    cudaError_t e = cudaEventRecord(e0, net->stream);
    if (e == cudaSuccess) e = launch_conv<32, 32, CONV_RELU>(c, net->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, net->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return net_cuda(net, e, "homg_net_check_barrier_timeout");
    *waited_ms = ms;
    return homg::net_check_error(net);
}

int homg_net_gather_patches(homg_net_handle net, const void* x, const float* t, int H, int W, const int32_t* corners,
                            int B, int P, void* xp, float* tp) {
    if (!net) return HOMG_EINVAL;
    if (!x || !t || !corners || !xp || !tp || B < 1 || P < 1 || P > H || P > W)
        return net_fail(net, HOMG_EINVAL, "homg_net_gather_patches: null pointer or bad sizes");
    const int64_t n = (int64_t)B * P * P;
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, net->stream>>>(static_cast<const bf16*>(x), t, H, W, corners, B, P,
                                                                  static_cast<bf16*>(xp), tp);
    NCK(net, cudaGetLastError(), "patch gather");
    return HOMG_OK;
}

const char* homg_net_last_error(homg_net_handle net) { return net ? net->err : g_net_error; }

void homg_net_destroy(homg_net_handle n) {
    if (!n) return;
    for (float* p : {n->params, n->grads, n->am, n->av}) if (p) cudaFree(p);
    for (int l = 0; l < 4; ++l) {
        if (n->wf[l]) cudaFree(n->wf[l]);
        if (n->wt[l]) cudaFree(n->wt[l]);
    }
    for (bf16* p : n->act) if (p) cudaFree(p);
    for (void* p : {(void*)n->gA, (void*)n->gB, (void*)n->g4, (void*)n->y, (void*)n->part, (void*)n->dloss, (void*)n->derr})
        if (p) cudaFree(p);
    delete n;
}

}  // extern "C"
