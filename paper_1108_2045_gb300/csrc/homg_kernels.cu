// HOMG kernels for sm_103a: the fused relaxation+interpolation iteration, the lattice level change,
// update+residual, full-weighting restriction, the convergence test and the copy-out.
//
// Storage type T of a cycle's arrays: double (FP64 path), float (FP32 relaxation and transfers) or
// __nv_bfloat16 (bfloat16 storage, FP32 arithmetic). Arithmetic type C is double for T = double,
// float otherwise. The residual, the update and the norms always run in FP64.
//
// STRICT (S) kernels evaluate every formula in the CPU oracle's canonical operation order with
// round-to-nearest intrinsics (no FMA contraction), storing through the same rounding as the
// oracle. The fast kernels reassociate to issue fewer floating-point instructions.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <type_traits>

#include "../../include/homg.h"
#include "homg_internal.h"

namespace homg {
namespace {

constexpr int BX = 32;
constexpr int BY = 8;
constexpr int P2X = 128;  // power-of-two iteration: columns per block (dealt by residue class)
constexpr int P2Y = 2;

// ---- storage traits -------------------------------------------------------------------------
template <typename T> struct St;
template <> struct St<double> {
    using C = double;
    static __device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
    static __device__ __forceinline__ double rd(const double* p) { return *p; }
    static __device__ __forceinline__ double put(double x) { return x; }
    static __device__ __forceinline__ double from_d(double x) { return x; }
};
template <> struct St<float> {
    using C = float;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float rd(const float* p) { return *p; }
    static __device__ __forceinline__ float put(float x) { return x; }
    static __device__ __forceinline__ float from_d(double x) { return __double2float_rn(x); }
};
template <> struct St<__nv_bfloat16> {
    using C = float;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(p))));
    }
    static __device__ __forceinline__ float rd(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ __nv_bfloat16 put(float x) { return __float2bfloat16_rn(x); }
    // double -> binary32 -> bfloat16, each round-to-nearest (the oracle's storage rounding)
    static __device__ __forceinline__ float from_d(double x) { return __double2float_rn(x); }
};

// Loads of the marching kernels. In their own launches they read through the read-only path
// (__ldg). Inside the persistent batch kernel (P = true), a phase reads values that other blocks of
// the same launch wrote in an earlier phase, which the read-only path does not promise to see:
// those loads go to L2 (__ldcg), the point of coherence, after the grid barrier's fences.
template <typename T> __device__ __forceinline__ typename St<T>::C ld_cg(const T* p);
template <> __device__ __forceinline__ double ld_cg<double>(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<float>(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ float ld_cg<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short*>(p))));
}
template <typename T, bool P> __device__ __forceinline__ typename St<T>::C ldv(const T* p) {
    if constexpr (P) return ld_cg<T>(p);
    else return St<T>::ld(p);
}
template <bool P> __device__ __forceinline__ double ld64(const double* p) {
    if constexpr (P) return __ldcg(p);
    else return __ldg(p);
}

// ---- binary32 <-> binary64 conversions with integer operations ----------------------------------
// GB300 issues FP64 instructions, conversions to and from binary64 among them, at a small fraction
// of its integer rate, and the fast residual kernels are bound by that pipe. These two conversions
// are written out from the IEEE 754 formats (binary32: 1 sign, 8 exponent bits biased by 127, 23
// fraction bits; binary64: 1, 11 biased by 1023, 52): normal numbers and zeros take integer
// operations only; subnormals, infinities and NaNs, which these kernels practically never meet,
// use the hardware conversion. Both are exact copies of it (homg_check_conversions tests that).

// The rare classes go through out-of-line hardware conversions, so that the compiler cannot
// if-convert them into conversions issued for every element.
__device__ __noinline__ double widen_hw(float x) { return (double)x; }
__device__ __noinline__ float narrow_hw(double d) { return __double2float_rn(d); }

// binary32 -> binary64 (exact): re-bias the exponent, move the fraction to the top of the 52 bits.
__device__ __forceinline__ double widen_f32(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned ex = (b >> 23) & 0xffu;
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (__builtin_expect(ex == 0u || ex == 0xffu, 0)) return widen_hw(x);
    const unsigned hi = (b & 0x80000000u) | ((ex + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}

// binary64 -> binary32, round to nearest, ties to even: keep the top 23 of the 52 fraction bits and
// round on the 29 dropped ones; a carry out of the fraction steps the exponent (to infinity above
// the largest binary32, as rounding to nearest requires).
__device__ __forceinline__ float narrow_rn(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sg = hi & 0x80000000u;
    if (((hi & 0x7fffffffu) | lo) == 0u) return __uint_as_float(sg);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // binary32 biased exponent
    if (__builtin_expect(e <= 0 || e >= 255, 0)) return narrow_hw(d);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float((sg | ((unsigned)e << 23) | m) + up);
}

// Stored value -> binary64, with the conversions above.
template <typename T> __device__ __forceinline__ double to_d(T x);
template <> __device__ __forceinline__ double to_d<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_d<float>(float x) { return widen_f32(x); }

// The cycle's source scale * r stored from the FP64 residual r (fast forms). FP64 cycles form the
// product in binary64; binary32 and bfloat16 cycles narrow r first and multiply in binary32 (one
// rounding more than the binary64 product, within the cycle's own precision), which keeps the
// multiply off the FP64 pipe that bounds the residual kernels.
template <typename T> __device__ __forceinline__ T source_store(double r, double scale, float scale_f);
template <> __device__ __forceinline__ double source_store<double>(double r, double scale, float) { return scale * r; }
template <> __device__ __forceinline__ float source_store<float>(double r, double, float scale_f) {
    return narrow_rn(r) * scale_f;
}
template <> __device__ __forceinline__ __nv_bfloat16 source_store<__nv_bfloat16>(double r, double, float scale_f) {
    return __float2bfloat16_rn(narrow_rn(r) * scale_f);
}

// ---- arithmetic in the canonical order (S) or freely contracted ------------------------------
template <bool S> __device__ __forceinline__ double add(double a, double b) { return S ? __dadd_rn(a, b) : a + b; }
template <bool S> __device__ __forceinline__ double sub(double a, double b) { return S ? __dsub_rn(a, b) : a - b; }
template <bool S> __device__ __forceinline__ double mul(double a, double b) { return S ? __dmul_rn(a, b) : a * b; }
template <bool S> __device__ __forceinline__ float add(float a, float b) { return S ? __fadd_rn(a, b) : a + b; }
template <bool S> __device__ __forceinline__ float sub(float a, float b) { return S ? __fsub_rn(a, b) : a - b; }
template <bool S> __device__ __forceinline__ float mul(float a, float b) { return S ? __fmul_rn(a, b) : a * b; }

// Element (i, j, k) of a grid with `pitch` elements per row and (n+1) rows per plane.
__device__ __forceinline__ int64_t at(int64_t pitch, int n, int i, int j, int k) {
    return ((int64_t)k * (n + 1) + j) * pitch + i;
}

// 2^e in the arithmetic type (exact), and the per-type copy of a scalar argument.
template <typename C> __device__ __forceinline__ C pow2(int e);
template <> __device__ __forceinline__ double pow2<double>(int e) { return ldexp(1.0, e); }
template <> __device__ __forceinline__ float pow2<float>(int e) { return ldexpf(1.0f, e); }
template <typename C> __device__ __forceinline__ C pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// f * 2^-e for 0 <= f < 2^e (e <= 30), exactly, assembled from the IEEE-754 fields with integer
// operations only: exponent floor(log2 f) - e, fraction the bits of f below its leading one.
template <typename C> __device__ __forceinline__ C dyadic(int f, int e);
template <> __device__ __forceinline__ double dyadic<double>(int f, int e) {
    if (f == 0) return 0.0;
    const int p = 31 - __clz(f);
    const unsigned long long frac = ((unsigned long long)f << (52 - p)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)(((unsigned long long)(p - e + 1023) << 52) | frac));
}
template <> __device__ __forceinline__ float dyadic<float>(int f, int e) {
    if (f == 0) return 0.f;
    const int p = 31 - __clz(f);
    const unsigned frac = ((unsigned)f << (23 - p)) & ((1u << 23) - 1);
    return __uint_as_float(((unsigned)(p - e + 127) << 23) | frac);
}

// One damped-Jacobi update v' = c1 v + om (sum of the 2d neighbours) + g (g pre-scaled by om).
// FP64 (the FP64 pipe bounds these kernels on GB300, and it issues fused multiply-adds at 0.627
// against 0.528 T instr/s for additions, measured). 2-D: the neighbour pairs e + n and s + w, then
// three FMAs, in the order of the shared-pair sweeps (k_jacobi2d, k_jacobi2d2), which form each
// pair once for two nodes; the additions are FMAs by the run-time 1. 3-D: a chain of 7 FMAs, every
// neighbour scaled by om on its own. Binary32 (DRAM bound): the neighbour sum, then two FMAs.
__device__ __forceinline__ double jacobi_pairs(double c1, double om, double one, double vc, double g, double w,
                                               double e, double s, double n) {
    return fma(om, fma(one, e, n), fma(om, fma(one, s, w), fma(c1, vc, g)));
}
__device__ __forceinline__ float jacobi_update(float c1, float om, float vc, float g, float n0, float n1, float n2,
                                               float n3) {
    return fma(c1, vc, fma(om, (n0 + n1) + (n2 + n3), g));
}
__device__ __forceinline__ double jacobi_update(double c1, double om, double vc, double g, double n0, double n1,
                                                double n2, double n3, double n4, double n5) {
    double t = fma(om, n0, g);
    t = fma(om, n1, t);
    t = fma(om, n2, t);
    t = fma(om, n3, t);
    t = fma(om, n4, t);
    t = fma(om, n5, t);
    return fma(c1, vc, t);
}
__device__ __forceinline__ float jacobi_update(float c1, float om, float vc, float g, float n0, float n1, float n2,
                                               float n3, float n4, float n5) {
    return fma(c1, vc, fma(om, ((n0 + n1) + (n2 + n3)) + (n4 + n5), g));
}

// Programmatic dependent launch: every kernel is launched so that it may start while its
// predecessor in the stream finishes. Each kernel first waits until the predecessor grid has
// completed and its writes are visible (griddepcontrol.wait), then lets its own successor launch.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

template <typename T> __device__ __forceinline__ const T* cp(const CGrid& g) { return static_cast<const T*>(g.p); }
template <typename T> __device__ __forceinline__ T* wp(const Grid& g) { return static_cast<T*>(g.p); }

// ---- batches of equal-size 2-D problems: problem z = blockIdx.z, arrays z * bstride apart ------
template <typename T> __device__ __forceinline__ void shift(CGrid& g, int z) {
    if (g.p) g.p = static_cast<const T*>(g.p) + (int64_t)z * g.bstride;
}
template <typename T> __device__ __forceinline__ void shift(Grid& g, int z) {
    if (g.p) g.p = static_cast<T*>(g.p) + (int64_t)z * g.bstride;
}
__device__ __forceinline__ void shift(CDGrid& g, int z) { if (g.p) g.p += (int64_t)z * g.bstride; }
__device__ __forceinline__ void shift(DGrid& g, int z) { if (g.p) g.p += (int64_t)z * g.bstride; }

// Move the arguments to this block's problem; false when that problem has already finished.
template <typename T> __device__ __forceinline__ bool batch_view(IterArgs& a, int z) {
    if (!a.bst) return true;
    if (a.bst[z].done) return false;
    shift<T>(a.e_old, z); shift<T>(a.e_new, z); shift<T>(a.g, z); shift<T>(a.dprev, z); shift<T>(a.dnew, z);
    return true;
}
template <typename T> __device__ __forceinline__ bool batch_view(ProlongArgs& a, int z) {
    if (!a.bst) return true;
    if (a.bst[z].done) return false;
    shift<T>(a.G, z); shift<T>(a.Gc, z); shift<T>(a.dl, z);
    return true;
}
template <typename T> __device__ __forceinline__ bool batch_view(RestrictArgs& a, int z) {
    if (!a.bst) return true;
    if (a.bst[z].done) return false;
    shift<T>(a.gf, z); shift<T>(a.gc, z);
    return true;
}
template <typename T> __device__ __forceinline__ bool batch_view(ResidArgs& a, int z) {
    if (!a.batch) return true;
    a.st += z;
    if (a.st->done) return false;
    shift(a.u_in, z); shift<T>(a.e, z); shift(a.u_out, z); shift<T>(a.g0, z);
    a.part_r += (int64_t)z * a.part_bstride;
    if (a.part_f) a.part_f += (int64_t)z * a.part_bstride;
    return true;
}

__device__ __forceinline__ long long device_clock_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Value at (i, j[, k]) of the (bi/tri)linear interpolant of compact array d at stride 2^mp
// (Sec. 2: linear interpolation S; exact dyadic weights). Summation order as in the oracle:
// 2-D (w00 d00 + w10 d10) + (w01 d01 + w11 d11); 3-D x-pairs, then y, then z.
// With DIFF, the interpolated field is d - d2 (the level-change kernel's stale values).
template <int ND, bool S, bool DIFF, typename T>
__device__ __forceinline__ typename St<T>::C interp(CGrid d, CGrid d2, int mp, int i, int j, int k) {
    using C = typename St<T>::C;
    const int lp = 1 << mp;
    const C inv = pow2<C>(-mp);
    const int I0 = i >> mp, a = i & (lp - 1), I1 = a ? I0 + 1 : I0;
    const int J0 = j >> mp, b = j & (lp - 1), J1 = b ? J0 + 1 : J0;
    const C wx0 = (C)(lp - a) * inv, wx1 = (C)a * inv;
    const C wy0 = (C)(lp - b) * inv, wy1 = (C)b * inv;
    auto val = [&](int I, int J, int K) -> C {
        C v = St<T>::rd(cp<T>(d) + at(d.pitch, d.n, I, J, K));
        if (DIFF) v = sub<S>(v, St<T>::rd(cp<T>(d2) + at(d2.pitch, d2.n, I, J, K)));
        return v;
    };
    if (ND == 2) {
        C t00 = mul<S>(mul<S>(wx0, wy0), val(I0, J0, 0));
        C t10 = mul<S>(mul<S>(wx1, wy0), val(I1, J0, 0));
        C t01 = mul<S>(mul<S>(wx0, wy1), val(I0, J1, 0));
        C t11 = mul<S>(mul<S>(wx1, wy1), val(I1, J1, 0));
        return add<S>(add<S>(t00, t10), add<S>(t01, t11));
    } else {
        const int K0 = k >> mp, c = k & (lp - 1), K1 = c ? K0 + 1 : K0;
        const C wz0 = (C)(lp - c) * inv, wz1 = (C)c * inv;
        const C wx[2] = {wx0, wx1}, wy[2] = {wy0, wy1}, wz[2] = {wz0, wz1};
        const int Ix[2] = {I0, I1}, Jy[2] = {J0, J1}, Kz[2] = {K0, K1};
        C t[2][2][2];
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int y = 0; y < 2; ++y)
#pragma unroll
                for (int x = 0; x < 2; ++x)
                    t[z][y][x] = mul<S>(mul<S>(mul<S>(wx[x], wy[y]), wz[z]), val(Ix[x], Jy[y], Kz[z]));
        return add<S>(add<S>(add<S>(t[0][0][0], t[0][0][1]), add<S>(t[0][1][0], t[0][1][1])),
                      add<S>(add<S>(t[1][0][0], t[1][0][1]), add<S>(t[1][1][0], t[1][1][1])));
    }
}

// ---------------------------------------------------------------------------------------------
// K1: one HOMG iteration (Sec. 2: relaxations on the level-m lattice fused with interpolations of
// the previous iteration's variations on the complementary nodes; Sec. 4: the interpolation is
// delayed one iteration). e_old.p == nullptr means e_old = 0 (first iteration of a cycle).
// ---------------------------------------------------------------------------------------------
template <int ND, bool S, typename T>
__device__ __forceinline__ void iterate_point(const IterArgs& a, int i, int j, int k) {
    using C = typename St<T>::C;
    const int n = a.e_new.n;
    const bool zero = (a.e_old.p == nullptr);
    auto E = [&](int ii, int jj, int kk) -> C {
        return zero ? (C)0 : St<T>::rd(cp<T>(a.e_old) + at(a.e_old.pitch, n, ii, jj, kk));
    };
    const C omega = pick<C>(a.omega, a.omega_f);
    C v = E(i, j, k);
    const int l = 1 << a.m;
    if (((i | j | (ND == 3 ? k : 0)) & (l - 1)) == 0) {
        C lap;
        if (ND == 2) {
            lap = mul<S>((C)4, v);
            lap = sub<S>(lap, E(i - l, j, 0));
            lap = sub<S>(lap, E(i + l, j, 0));
            lap = sub<S>(lap, E(i, j - l, 0));
            lap = sub<S>(lap, E(i, j + l, 0));
        } else {
            lap = mul<S>((C)6, v);
            lap = sub<S>(lap, E(i - l, j, k));
            lap = sub<S>(lap, E(i + l, j, k));
            lap = sub<S>(lap, E(i, j - l, k));
            lap = sub<S>(lap, E(i, j + l, k));
            lap = sub<S>(lap, E(i, j, k - l));
            lap = sub<S>(lap, E(i, j, k + l));
        }
        const int I = i >> a.m, J = j >> a.m, K = (ND == 3) ? (k >> a.m) : 0;
        const C g = St<T>::rd(cp<T>(a.g) + at(a.g.pitch, a.g.n, I, J, K));
        // strict: g = h_m^2 F_m, delta = omega (g - lap); fast: g = omega h_m^2 F_m, delta = g - omega lap
        const C delta = S ? mul<S>(omega, sub<S>(g, lap)) : fma(-omega, lap, g);
        if (a.dnew.p) wp<T>(a.dnew)[at(a.dnew.pitch, a.dnew.n, I, J, K)] = St<T>::put(delta);
        v = add<S>(v, delta);
    }
    if (a.mp >= 0) {
        const int lpm = (1 << a.mp) - 1;
        if (((i | j | (ND == 3 ? k : 0)) & lpm) != 0) v = add<S>(v, interp<ND, S, false, T>(a.dprev, a.dprev, a.mp, i, j, k));
    }
    wp<T>(a.e_new)[at(a.e_new.pitch, n, i, j, k)] = St<T>::put(v);
}

template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_iterate(IterArgs a) {
    pdl_begin();
    if (ND == 2 && !batch_view<T>(a, blockIdx.z)) return;
    const int n = a.e_new.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    iterate_point<ND, S, T>(a, i, j, k);
}

// ---------------------------------------------------------------------------------------------
// Lattice form, level change (see ProlongArgs): stale values of the finer lattice.
// ---------------------------------------------------------------------------------------------
template <int ND, bool S, typename T>
__device__ __forceinline__ void prolong_point(const ProlongArgs& a, int i, int j, int k) {
    using C = typename St<T>::C;
    const int n = a.G.n;
    const int sm = (1 << a.s) - 1;
    C v;
    if (((i | j | (ND == 3 ? k : 0)) & sm) == 0)
        v = St<T>::rd(cp<T>(a.Gc) + at(a.Gc.pitch, a.Gc.n, i >> a.s, j >> a.s, (ND == 3) ? (k >> a.s) : 0));
    else
        v = interp<ND, S, true, T>(a.Gc, a.dl, a.s, i, j, k);
    wp<T>(a.G)[at(a.G.pitch, n, i, j, k)] = St<T>::put(v);
}

template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong(ProlongArgs a) {
    pdl_begin();
    if (ND == 2 && !batch_view<T>(a, blockIdx.z)) return;
    const int n = a.G.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    prolong_point<ND, S, T>(a, i, j, k);
}

// Fixed-order block sum of one value per thread (warp butterflies, then warps in order).
__device__ __forceinline__ double block_sum(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) / 32;
    __syncthreads();
    if ((tid & 31) == 0) sh[tid >> 5] = x;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < nw; ++w) s += sh[w];
    return s;
}

// ---------------------------------------------------------------------------------------------
// K2: update + residual (Sec. 2: residual r = f - A_h v of the two-grid scheme, restarted on the
// residual equation after each cycle) and the level-0 source of the next cycle. FP64 throughout;
// e is widened from the cycle's storage type and g0 rounded to it.
// ---------------------------------------------------------------------------------------------
template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_residual(ResidArgs a, int n) {
    pdl_begin();
    __shared__ double sh[BX * BY / 32];
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    const bool active = (i < n && j < n);
    const double* uc = a.u_in.p ? a.u_in.p : a.st->u;
    const int64_t upitch = a.u_in.p ? a.u_in.pitch : (int64_t)(n + 1);
    const double* f = a.st->f;
    auto U = [&](int ii, int jj, int kk) -> double {
        if (ii <= 0 || jj <= 0 || ii >= n || jj >= n) return 0.0;
        if (ND == 3 && (kk <= 0 || kk >= n)) return 0.0;
        double v = uc[at(upitch, n, ii, jj, kk)];
        if (a.e.p) v = add<S>(v, (double)St<T>::rd(cp<T>(a.e) + at(a.e.pitch, n, ii, jj, kk)));
        return v;
    };
    double rr = 0.0, ff = 0.0;
    if (active) {
        const double c = U(i, j, k);
        double lap;
        if (ND == 2) {
            lap = mul<S>(4.0, c);
            lap = sub<S>(lap, U(i - 1, j, 0));
            lap = sub<S>(lap, U(i + 1, j, 0));
            lap = sub<S>(lap, U(i, j - 1, 0));
            lap = sub<S>(lap, U(i, j + 1, 0));
        } else {
            lap = mul<S>(6.0, c);
            lap = sub<S>(lap, U(i - 1, j, k));
            lap = sub<S>(lap, U(i + 1, j, k));
            lap = sub<S>(lap, U(i, j - 1, k));
            lap = sub<S>(lap, U(i, j + 1, k));
            lap = sub<S>(lap, U(i, j, k - 1));
            lap = sub<S>(lap, U(i, j, k + 1));
        }
        const double fv = f[at(n + 1, n, i, j, k)];
        const double r = sub<S>(fv, mul<S>(lap, a.inv_h2));
        if (a.u_out.p) a.u_out.p[at(a.u_out.pitch, n, i, j, k)] = c;
        if (a.g0.p) wp<T>(a.g0)[at(a.g0.pitch, n, i, j, k)] = St<T>::put(St<T>::from_d(mul<S>(a.scale, r)));
        rr = r * r;
        ff = fv * fv;
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    double s = block_sum(rr, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part_r[bid] = s;
    if (a.part_f) {
        s = block_sum(ff, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) a.part_f[bid] = s;
    }
}

// ---------------------------------------------------------------------------------------------
// Restriction (Sec. 2: linearly weighted averages as nested reductions; full weighting).
// g_c = 4 FW(g_f): sources stay pre-scaled by h_m^2, so this equals h_{m+1}^2 FW(F_m) exactly.
// ---------------------------------------------------------------------------------------------
template <int ND, bool S, typename T>
__device__ __forceinline__ void restrict_point(const RestrictArgs& a, int I, int J, int K) {
    using C = typename St<T>::C;
    const int nc = a.gc.n;
    const int i = 2 * I, j = 2 * J, k = 2 * K;
    auto F = [&](int ii, int jj, int kk) -> C { return St<T>::rd(cp<T>(a.gf) + at(a.gf.pitch, a.gf.n, ii, jj, kk)); };
    C v;
    if (ND == 2) {
        const C c = F(i, j, 0);
        const C edges = add<S>(add<S>(add<S>(F(i - 1, j, 0), F(i + 1, j, 0)), F(i, j - 1, 0)), F(i, j + 1, 0));
        const C corners =
            add<S>(add<S>(add<S>(F(i - 1, j - 1, 0), F(i + 1, j - 1, 0)), F(i - 1, j + 1, 0)), F(i + 1, j + 1, 0));
        v = mul<S>(add<S>(add<S>(mul<S>((C)4, c), mul<S>((C)2, edges)), corners), (C)0.25);
        if (!S) v *= (C)a.scale;
    } else {
        const C c = F(i, j, k);
        C faces = 0, edges = 0, corners = 0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nz = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nz == 0) continue;
                    const C x = F(i + dx, j + dy, k + dz);
                    if (nz == 1) faces = add<S>(faces, x);
                    else if (nz == 2) edges = add<S>(edges, x);
                    else corners = add<S>(corners, x);
                }
        v = mul<S>(add<S>(add<S>(add<S>(mul<S>((C)8, c), mul<S>((C)4, faces)), mul<S>((C)2, edges)), corners), (C)0.0625);
        if (!S) v *= (C)a.scale;
    }
    wp<T>(a.gc)[at(a.gc.pitch, nc, I, J, K)] = St<T>::put(v);
}

template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_restrict(RestrictArgs a) {
    pdl_begin();
    if (ND == 2 && !batch_view<T>(a, blockIdx.z)) return;
    const int nc = a.gc.n;
    const int I = blockIdx.x * BX + threadIdx.x + 1;
    const int J = blockIdx.y * BY + threadIdx.y + 1;
    const int K = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (I >= nc || J >= nc) return;
    restrict_point<ND, S, T>(a, I, J, K);
}

// ---------------------------------------------------------------------------------------------
// K3: convergence test (Sec. 2, restart on the residual equation until the desired accuracy).
// One block; partial sums are added in a fixed order so the decision is reproducible. Enables the
// next cycle's conditional graph nodes while the solve continues.
// ---------------------------------------------------------------------------------------------
// Convergence decision for one problem (thread 0): relres, history, status, done; in single-problem
// graphs also enables the next stage's conditional nodes.
__device__ void finalize_decide(const FinalizeArgs& a, State* st, double* hist, double sr, double sf) {
    const double rn = sqrt(sr);
    if (a.mode == FIN_NORM) {
        const double fn = sqrt(sf);
        st->fnorm = fn;
        st->relres = (fn > 0.0) ? rn / fn : (rn == 0.0 ? 0.0 : INFINITY);
        return;
    }
    int k;
    double rel;
    if (a.mode == FIN_INIT) {
        const double fn = sqrt(sf);
        st->fnorm = fn;
        st->cycle = 0;
        st->t_start = device_clock_ns();
        if (fn == 0.0) {
            st->zero_u = 1;
            st->relres = 0.0;
            st->status = HOMG_OK;
            st->done = 1;
            st->t_done = st->t_start;
            hist[0] = 0.0;
            return;
        }
        st->zero_u = 0;
        rel = rn / fn;
        st->rr0 = rel;
        k = 0;
    } else {
        k = ++st->cycle;
        rel = rn / st->fnorm;
    }
    hist[k] = rel;
    st->relres = rel;
    int status = -1;
    if (rel <= st->tol) status = HOMG_OK;
    else if (!isfinite(rel) || rel > st->div_factor * st->rr0) status = HOMG_DIVERGED;
    else if (k >= st->max_cycles) status = HOMG_NOT_CONVERGED;
    st->status = status;
    st->done = (status >= 0);
    if (st->done) st->t_done = device_clock_ns();
    if (a.batch) return;
    const int local = k - st->stage_base;  // stage index within this graph launch
    if (status < 0 && local + 1 <= a.nstages) {
        for (int p = 0; p < 3; ++p) cudaGraphSetConditional(a.handles[3 * (local + 1) + p], 1u);
    }
}

__global__ void __launch_bounds__(1024) k_finalize(FinalizeArgs a) {
    pdl_begin();
    __shared__ double sh[32];
    const int z = a.batch ? blockIdx.x : 0;  // batch: one block per problem
    State* st = a.st + z;
    double* hist = a.hist + (int64_t)z * a.hist_bstride;
    const double* pr = a.part_r + (int64_t)z * a.part_bstride;
    const double* pf = a.part_f ? a.part_f + (int64_t)z * a.part_bstride : nullptr;
    const bool skip = a.batch && a.mode == FIN_CYCLE && st->done;  // finished earlier
    if (!skip) {
        double sr = 0.0, sf = 0.0;
        for (int t = threadIdx.x; t < a.nparts; t += blockDim.x) {
            sr += pr[t];
            if (pf) sf += pf[t];
        }
        sr = block_sum(sr, sh);
        if (pf) sf = block_sum(sf, sh);
        if (threadIdx.x == 0) finalize_decide(a, st, hist, sr, sf);
    }
    if (!a.batch) return;
    // batch: the last block to arrive enables the next stage while any problem is still running
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&a.ticket[0], 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int running = 0;
    for (int p = threadIdx.x; p < (int)gridDim.x; p += blockDim.x) running |= !((volatile State*)a.st)[p].done;
    running = __syncthreads_or(running);
    if (threadIdx.x == 0) {
        a.ticket[0] = 0;
        const int k = (a.mode == FIN_INIT) ? 0 : (int)++a.ticket[1];  // cycles run by the batch
        const int local = k - (int)a.ticket[2];                       // stage within this graph launch
        if (running && local + 1 <= a.nstages)
            for (int q = 0; q < 3; ++q) cudaGraphSetConditional(a.handles[3 * (local + 1) + q], 1u);
    }
}

// Copy the final iterate into the caller's u (interior nodes); u = 0 when ||f|| = 0.
template <int ND>
__global__ void __launch_bounds__(BX * BY) k_copy_out(CopyOutArgs a, int n) {
    pdl_begin();
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    const State* st = a.st;
    CDGrid u0 = a.u0, u1 = a.u1;
    if (ND == 2 && a.batch) {
        st += blockIdx.z;
        shift(u0, blockIdx.z);
        shift(u1, blockIdx.z);
    }
    double v = 0.0;
    if (!st->zero_u) {
        const CDGrid src = (st->cycle & 1) ? u1 : u0;
        v = src.p[at(src.pitch, n, i, j, k)];
    }
    st->u[at(n + 1, n, i, j, k)] = v;
}



// ---------------------------------------------------------------------------------------------
// V-cycle comparator (Sec. 2, the classic two-grid correction scheme). Level residual, pre-scaled
// like the source: strict rho = g - lap(e) = h_m^2 (F_m - A_m e); fast rho = g - omega lap(e).
// ---------------------------------------------------------------------------------------------
template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_vresid(VResidArgs a) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.rho.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    const bool zero = (a.e.p == nullptr);
    auto E = [&](int ii, int jj, int kk) -> C {
        return zero ? (C)0 : St<T>::rd(cp<T>(a.e) + at(a.e.pitch, n, ii, jj, kk));
    };
    C lap;
    if (ND == 2) {
        lap = mul<S>((C)4, E(i, j, 0));
        lap = sub<S>(lap, E(i - 1, j, 0));
        lap = sub<S>(lap, E(i + 1, j, 0));
        lap = sub<S>(lap, E(i, j - 1, 0));
        lap = sub<S>(lap, E(i, j + 1, 0));
    } else {
        lap = mul<S>((C)6, E(i, j, k));
        lap = sub<S>(lap, E(i - 1, j, k));
        lap = sub<S>(lap, E(i + 1, j, k));
        lap = sub<S>(lap, E(i, j - 1, k));
        lap = sub<S>(lap, E(i, j + 1, k));
        lap = sub<S>(lap, E(i, j, k - 1));
        lap = sub<S>(lap, E(i, j, k + 1));
    }
    const C g = St<T>::rd(cp<T>(a.g) + at(a.g.pitch, n, i, j, k));
    const C rho = S ? sub<S>(g, lap) : fma(-pick<C>(a.omega, (float)a.omega), lap, g);
    wp<T>(a.rho)[at(a.rho.pitch, n, i, j, k)] = St<T>::put(rho);
}

// Prolongation-add e += P ec in place: lattice nodes add the coarse value, the others its
// (bi/tri)linear interpolant (Sec. 2 step (d): interpolation of the coarse correction).
template <int ND, bool S, typename T>
__global__ void __launch_bounds__(BX * BY) k_prolong_add(ProlongAddArgs a) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.e.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    T* p = wp<T>(a.e) + at(a.e.pitch, n, i, j, k);
    const C v = St<T>::rd(p);
    *p = St<T>::put(add<S>(v, interp<ND, S, false, T>(a.ec, a.ec, 1, i, j, k)));
}

// ---------------------------------------------------------------------------------------------
// Coarsest lattices in one block: the restrictions, iterations and level changes of every level
// whose lattice is small run as one launch of a single 512-thread block, which steps through the
// op list with a block barrier between ops (a barrier also makes each op's global writes visible to
// the whole block). Replaces dozens of launches whose cost is pure launch latency.
// ---------------------------------------------------------------------------------------------
template <int ND, typename T>
__device__ __forceinline__ void coarse_block_body(const BlockOp* __restrict__ ops, int nops, int z) {
    const int tid = threadIdx.x;
    for (int o = 0; o < nops; ++o) {
        const int kind = ops[o].kind;
        RestrictArgs rs = ops[o].rs;
        ProlongArgs pr = ops[o].pr;
        IterArgs it = ops[o].it;
        bool live;
        int side;
        if (kind == BLOCK_RESTRICT) { live = batch_view<T>(rs, z); side = rs.gc.n - 1; }
        else if (kind == BLOCK_PROLONG) { live = batch_view<T>(pr, z); side = pr.G.n - 1; }
        else { live = batch_view<T>(it, z); side = it.e_new.n - 1; }
        if (!live) return;  // this problem has converged (uniform over the block)
        const int total = (ND == 2) ? side * side : side * side * side;
        for (int q = tid; q < total; q += blockDim.x) {
            const int i = q % side + 1, j = (q / side) % side + 1, k = (ND == 3) ? q / (side * side) + 1 : 0;
            if (kind == BLOCK_RESTRICT) restrict_point<ND, false, T>(rs, i, j, k);
            else if (kind == BLOCK_PROLONG) prolong_point<ND, false, T>(pr, i, j, k);
            else iterate_point<ND, false, T>(it, i, j, k);
        }
        __syncthreads();
    }
}

template <int ND, typename T>
__global__ void __launch_bounds__(512) k_coarse_block(const BlockOp* __restrict__ ops, int nops) {
    pdl_begin();
    coarse_block_body<ND, T>(ops, nops, (ND == 2) ? (int)blockIdx.z : 0);  // batch: one block per problem
}

// =============================================================================================
// Fast kernels (strict_fp = 0).
// =============================================================================================
constexpr int JX = 128;  // threads per block along x (2-D)
constexpr int JR = 16;   // nodes per thread along the march on large grids

// Stride-2 interpolation along a marching column: X(J) is the x-interpolant of compact row J at
// this thread's column (the lattice value itself on even columns); a fine row j takes X(j/2) when
// j is even and the mean of X(j/2) and X(j/2 + 1) when j is odd. X is formed once per coarse row
// and shared by the two fine rows it touches, and the form is branch-free across a warp.
template <typename T, bool P = false>
struct ColumnInterp2 {
    using C = typename St<T>::C;
    const T* d;    // compact array, offset to this column's left lattice neighbour
    const T* d2;   // second compact array subtracted from d (nullptr: none)
    int64_t pitch, pitch2;
    C hx;          // 0.5 on odd columns, 0 on even ones
    int cj = -1;
    C x0 = 0, x1 = 0;  // X(cj), X(cj + 1)

    __device__ __forceinline__ C X(int J) const {
        C a = ldv<T, P>(d + (int64_t)J * pitch), b = ldv<T, P>(d + (int64_t)J * pitch + 1);
        if (d2) {
            a -= ldv<T, P>(d2 + (int64_t)J * pitch2);
            b -= ldv<T, P>(d2 + (int64_t)J * pitch2 + 1);
        }
        return fma(hx, b - a, a);
    }
    __device__ __forceinline__ C at(int j) {
        const int J0 = j >> 1;
        if (J0 != cj) {
            x0 = (J0 == cj + 1) ? x1 : X(J0);
            x1 = X(J0 + 1);
            cj = J0;
        }
        return (j & 1) ? (C)0.5 * (x0 + x1) : x0;
    }
};

// Fast level-0 iteration (every iteration of the lattice form, the level-0 iterations of the
// whole-grid form): damped Jacobi on every interior node with the source pre-scaled by omega,
//   v' = (1 - c omega) v + omega * (sum of the 2d neighbours) + omega h^2 F
// = 5 FP instructions per node in 2-D (7 in 3-D), plus the pending interpolation on the first
// iteration of a level (PEND: 0 none, 1 stride 2, 2 any stride). Each thread marches one column
// (2-D: along y; 3-D: along z) keeping the centre and its two neighbours along the march in
// registers; the other neighbours come through L1. In FP64 the FP64 pipe bounds this kernel on
// GB300; in FP32/bfloat16, DRAM does.
template <int PEND, bool WD, typename T, bool BATCH, bool P>
__device__ __forceinline__ void jacobi2_body(IterArgs a, int rows, int bx, int by, int bz) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // compiled into batch launches only
    using C = typename St<T>::C;
    const int n = a.e_new.n;
    const int i = bx * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = by * rows + 1;
    const int j1 = min(j0 + rows, n);
    const T* __restrict__ E = cp<T>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    T* __restrict__ O = wp<T>(a.e_new);
    const int64_t po = a.e_new.pitch;
    const T* __restrict__ G = cp<T>(a.g);
    const int64_t pg = a.g.pitch;
    const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    ColumnInterp2<T, P> ci;
    if (PEND == 1) {
        ci.d = cp<T>(a.dprev) + (i >> 1);
        ci.d2 = nullptr;
        ci.pitch = a.dprev.pitch;
        ci.pitch2 = 0;
        ci.hx = (i & 1) ? (C)0.5 : (C)0;
    }
    C vs = ldv<T, P>(E + (int64_t)(j0 - 1) * pe + i);
    C vc = ldv<T, P>(E + (int64_t)j0 * pe + i);
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const T* row = E + (int64_t)j * pe + i;
        const C vn = ldv<T, P>(row + pe);
        const C w = ldv<T, P>(row - 1), e = ldv<T, P>(row + 1);
        const C g = ldv<T, P>(G + (int64_t)j * pg + i);
        C v;
        if constexpr (std::is_same<C, double>::value) v = jacobi_pairs(c1, om, a.one, vc, g, w, e, vs, vn);
        else v = jacobi_update(c1, om, vc, g, w, e, vs, vn);
        if (WD) wp<T>(a.dnew)[(int64_t)j * a.dnew.pitch + i] = St<T>::put(v - vc);
        if (PEND == 1) {
            const C sv = ci.at(j);
            v += ((i | j) & 1) ? sv : (C)0;
        }
        if (PEND == 2 && ((i | j) & lpm)) v += interp<2, false, false, T>(a.dprev, a.dprev, a.mp, i, j, 0);
        O[(int64_t)j * po + i] = St<T>::put(v);
        vs = vc;
        vc = vn;
    }
}

template <int PEND, bool WD, typename T, bool BATCH>
__global__ void __launch_bounds__(JX) k_jacobi2(IterArgs a, int rows) {
    pdl_begin();
    jacobi2_body<PEND, WD, T, BATCH, false>(a, rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// FP64 level iteration of a single problem with shared neighbour pairs. The pair
// D(i, j) = v(i+1, j) + v(i, j+1) is the east + north sum of node (i, j) and the west + south sum
// of node (i+1, j+1), so with one pair formed per node the update
//   v' = c1 v + om (D(i, j) + D(i-1, j-1)) + g
// costs one FP64 addition (written as an FMA by a run-time 1) and three FMAs: 4 FP64 instructions
// per node instead of the 5 of jacobi_update. A warp's lanes march 32 adjacent columns down the
// rows; D(i-1, j-1) is the left lane's pair from the row before (a shuffle). Lane 0 holds the
// column left of the warp's 31 output columns and only forms its pair, so the warp issues 4 x 32 / 31
// = 4.13 FP64 instructions per output node. Same values as jacobi2_body up to the order of the
// additions.
constexpr int JD_COLS = 31;  // output columns per warp
template <int PEND, bool WD>
__global__ void __launch_bounds__(JX) k_jacobi2d(IterArgs a, int rows) {
    pdl_begin();
    const int n = a.e_new.n;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.x * (JX / 32) + (threadIdx.x >> 5)) * JD_COLS;  // the warp's left column
    if (i0 + 1 > n - 1) return;                                              // warp-uniform: no output
    const int iu = i0 + lane;
    const int i = min(iu, n - 1);  // lanes past the last interior column load inside the lattice
    const bool out = lane > 0 && iu <= n - 1;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const double* __restrict__ E = cp<double>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    double* __restrict__ O = wp<double>(a.e_new);
    const int64_t po = a.e_new.pitch;
    const double* __restrict__ G = cp<double>(a.g);
    const int64_t pg = a.g.pitch;
    const double om = a.omega, c1 = a.c1, one = a.one;
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    ColumnInterp2<double, false> ci;
    if (PEND == 1) {
        ci.d = cp<double>(a.dprev) + (i >> 1);
        ci.d2 = nullptr;
        ci.pitch = a.dprev.pitch;
        ci.pitch2 = 0;
        ci.hx = (i & 1) ? 0.5 : 0.0;
    }
    double vc = __ldg(E + (int64_t)j0 * pe + i);
    double dp = fma(one, __ldg(E + (int64_t)(j0 - 1) * pe + i + 1), vc);  // D(i, j0 - 1)
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const double* row = E + (int64_t)j * pe + i;
        const double vn = __ldg(row + pe), e = __ldg(row + 1);
        const double g = __ldg(G + (int64_t)j * pg + i);
        const double dw = __shfl_up_sync(0xffffffffu, dp, 1);  // D(i-1, j-1): west + south
        const double dh = fma(one, e, vn);                       // D(i, j): east + north
        double v = fma(om, dh, fma(om, dw, fma(c1, vc, g)));
        if (WD && out) wp<double>(a.dnew)[(int64_t)j * a.dnew.pitch + i] = v - vc;
        if (PEND == 1) {
            const double sv = ci.at(j);
            v += ((i | j) & 1) ? sv : 0.0;
        }
        if (PEND == 2 && out && ((i | j) & lpm)) v += interp<2, false, false, double>(a.dprev, a.dprev, a.mp, i, j, 0);
        if (out) O[(int64_t)j * po + i] = v;
        dp = dh;
        vc = vn;
    }
}

// The same with two adjacent columns per lane (cA = i0 + 2 lane, cB = cA + 1; lane 0's cA is the
// helper column): 63 output columns per warp, 4 x 64 / 63 = 4.06 FP64 instructions per output node,
// one shuffle per two nodes. East of cA is cB's centre; west + south of cB is cA's pair from the row
// before. Lanes past the lattice clamp their columns to n (the boundary column); PEND reads clamp
// to n - 1.
constexpr int JD2_COLS = 63;
// Two columns per lane from this lattice size on. Measured in the 4097² FP64 solve: level-0 sweep
// 148.1 -> 145.9 us, but the smaller lattices slower (levels >= 1: 17.2 -> 18.0 ms per solve).
constexpr int JD2_MIN_N = 4096;
template <int PEND, bool WD>
__global__ void __launch_bounds__(JX) k_jacobi2d2(IterArgs a, int rows) {
    pdl_begin();
    const int n = a.e_new.n;
    const int lane = threadIdx.x & 31;
    const int i0 = (blockIdx.x * (JX / 32) + (threadIdx.x >> 5)) * JD2_COLS;
    if (i0 + 1 > n - 1) return;  // warp-uniform
    const int cA = i0 + 2 * lane, cB = cA + 1;
    const int iA = min(cA, n), iB = min(cB, n), iE = min(cB + 1, n);
    const bool outA = lane > 0 && cA <= n - 1, outB = cB <= n - 1;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const double* __restrict__ E = cp<double>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    double* __restrict__ O = wp<double>(a.e_new);
    const int64_t po = a.e_new.pitch;
    const double* __restrict__ G = cp<double>(a.g);
    const int64_t pg = a.g.pitch;
    const double om = a.omega, c1 = a.c1, one = a.one;
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    const int pA = min(cA, n - 1), pB = min(cB, n - 1);
    ColumnInterp2<double, false> ciA, ciB;
    if (PEND == 1) {
        ciA.d = cp<double>(a.dprev) + (pA >> 1);
        ciB.d = cp<double>(a.dprev) + (pB >> 1);
        ciA.d2 = ciB.d2 = nullptr;
        ciA.pitch = ciB.pitch = a.dprev.pitch;
        ciA.pitch2 = ciB.pitch2 = 0;
        ciA.hx = (pA & 1) ? 0.5 : 0.0;
        ciB.hx = (pB & 1) ? 0.5 : 0.0;
    }
    double vcA = __ldg(E + (int64_t)j0 * pe + iA), vcB = __ldg(E + (int64_t)j0 * pe + iB);
    double dpA = fma(one, __ldg(E + (int64_t)(j0 - 1) * pe + iB), vcA);  // D(cA, j0 - 1)
    double dpB = fma(one, __ldg(E + (int64_t)(j0 - 1) * pe + iE), vcB);  // D(cB, j0 - 1)
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        const double* row = E + (int64_t)j * pe;
        const double vnA = __ldg(row + pe + iA), vnB = __ldg(row + pe + iB), eB = __ldg(row + iE);
        const double* grow = G + (int64_t)j * pg;
        const double gA = __ldg(grow + iA), gB = __ldg(grow + iB);
        const double dwA = __shfl_up_sync(0xffffffffu, dpB, 1);  // D(cA-1, j-1)
        const double dhA = fma(one, vcB, vnA), dhB = fma(one, eB, vnB);
        double vA = fma(om, dhA, fma(om, dwA, fma(c1, vcA, gA)));
        double vB = fma(om, dhB, fma(om, dpA, fma(c1, vcB, gB)));
        if (WD) {
            double* D = wp<double>(a.dnew) + (int64_t)j * a.dnew.pitch;
            if (outA) D[cA] = vA - vcA;
            if (outB) D[cB] = vB - vcB;
        }
        if (PEND == 1) {
            const double sA = ciA.at(j), sB = ciB.at(j);
            vA += ((pA | j) & 1) ? sA : 0.0;
            vB += ((pB | j) & 1) ? sB : 0.0;
        }
        if (PEND == 2) {
            if (outA && ((cA | j) & lpm)) vA += interp<2, false, false, double>(a.dprev, a.dprev, a.mp, cA, j, 0);
            if (outB && ((cB | j) & lpm)) vB += interp<2, false, false, double>(a.dprev, a.dprev, a.mp, cB, j, 0);
        }
        double* orow = O + (int64_t)j * po;
        if (outA) orow[cA] = vA;
        if (outB) orow[cB] = vB;
        dpA = dhA;
        dpB = dhB;
        vcA = vnA;
        vcB = vnB;
    }
}

// Coefficient storage of the variable-coefficient kernels: double for FP64 cycles, float otherwise.
template <typename T> struct KT { using type = float; };
template <> struct KT<double> { using type = double; };

// Fast variable-coefficient iteration (2-D lattice form): damped Jacobi with each node's own weight
// wd = omega_J / D on -div(k grad .) with harmonic-mean faces,
//   v' = (1 - omega_J) v + wd (h_m^2 F + k_W w + k_E e + k_S s + k_N n)
// = 6 FP instructions per node. kx holds each node's east-face coefficient (the west face is the
// left neighbour's), ky its north face; the south face rides down the march in a register. The
// first iteration of a cycle (e_old = 0) reduces to v' = wd h_m^2 F.
template <int PEND, bool WD, typename T>
__global__ void __launch_bounds__(JX) k_jacobi2_vc(IterArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    using K = typename KT<T>::type;
    const int n = a.e_new.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const T* __restrict__ E = cp<T>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    T* __restrict__ O = wp<T>(a.e_new);
    const int64_t po = a.e_new.pitch;
    const T* __restrict__ G = cp<T>(a.g);
    const int64_t pg = a.g.pitch;
    const K* __restrict__ KX = static_cast<const K*>(a.kx);
    const K* __restrict__ KY = static_cast<const K*>(a.ky);
    const K* __restrict__ W = static_cast<const K*>(a.wd);
    const int64_t pk = a.kpitch;
    const C c1 = pick<C>(a.c1, a.c1_f);
    if (E == nullptr) {
        for (int j = j0; j < j1; ++j) {
            const C v = (C)__ldg(W + (int64_t)j * pk + i) * St<T>::ld(G + (int64_t)j * pg + i);
            if (WD) wp<T>(a.dnew)[(int64_t)j * a.dnew.pitch + i] = St<T>::put(v);
            O[(int64_t)j * po + i] = St<T>::put(v);
        }
        return;
    }
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    ColumnInterp2<T> ci;
    if (PEND == 1) {
        ci.d = cp<T>(a.dprev) + (i >> 1);
        ci.d2 = nullptr;
        ci.pitch = a.dprev.pitch;
        ci.pitch2 = 0;
        ci.hx = (i & 1) ? (C)0.5 : (C)0;
    }
    C vs = St<T>::ld(E + (int64_t)(j0 - 1) * pe + i);
    C vc = St<T>::ld(E + (int64_t)j0 * pe + i);
    C ks = (C)__ldg(KY + (int64_t)(j0 - 1) * pk + i);
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const T* row = E + (int64_t)j * pe + i;
        const C vn = St<T>::ld(row + pe);
        const C w = St<T>::ld(row - 1), e = St<T>::ld(row + 1);
        const C g = St<T>::ld(G + (int64_t)j * pg + i);
        const K* kr = KX + (int64_t)j * pk + i;
        const C kw = (C)__ldg(kr - 1), ke = (C)__ldg(kr);
        const C kn = (C)__ldg(KY + (int64_t)j * pk + i);
        const C wd = (C)__ldg(W + (int64_t)j * pk + i);
        C t = fma(kw, w, g);
        t = fma(ke, e, t);
        t = fma(ks, vs, t);
        t = fma(kn, vn, t);
        C v = fma(c1, vc, wd * t);
        if (WD) wp<T>(a.dnew)[(int64_t)j * a.dnew.pitch + i] = St<T>::put(v - vc);
        if (PEND == 1) {
            const C sv = ci.at(j);
            v += ((i | j) & 1) ? sv : (C)0;
        }
        if (PEND == 2 && ((i | j) & lpm)) v += interp<2, false, false, T>(a.dprev, a.dprev, a.mp, i, j, 0);
        O[(int64_t)j * po + i] = St<T>::put(v);
        ks = kn;
        vs = vc;
        vc = vn;
    }
}

// Harmonic mean ((2 a) b) / (a + b) of two node coefficients in round-to-nearest steps (the same
// value, bit for bit, whichever end comes first).
__device__ __forceinline__ double face_coef(double a, double b) {
    return __ddiv_rn(__dmul_rn(__dmul_rn(2.0, a), b), __dadd_rn(a, b));
}

// Coefficients of level m, one thread per lattice node (I, J) of the (n_m+1)^2 compact lattice:
// east face (I < n_m), north face (J < n_m), and at interior nodes the weight
// omega_J / (((k_W + k_E) + k_S) + k_N).
template <typename K>
__global__ void k_vc_setup(const double* __restrict__ k, int n, int m, K* kx, K* ky, K* wd, int64_t pitch,
                           double omega_j, int* bad) {
    const int nm = n >> m, l = 1 << m;
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I > nm || J > nm) return;
    const int64_t side = n + 1;
    const int64_t i = (int64_t)I << m, j = (int64_t)J << m;
    const double kp = k[j * side + i];
    if (!(kp > 0.0) || !isfinite(kp)) atomicOr(bad, 1);
    const int64_t q = (int64_t)J * pitch + I;
    const double ke = (I < nm) ? face_coef(kp, k[j * side + i + l]) : 0.0;
    const double kn = (J < nm) ? face_coef(kp, k[(j + l) * side + i]) : 0.0;
    kx[q] = (K)ke;
    ky[q] = (K)kn;
    if (wd) {
        double w = 0.0;
        if (I > 0 && J > 0 && I < nm && J < nm) {
            const double kw = face_coef(kp, k[j * side + i - l]);
            const double ks = face_coef(kp, k[(j - l) * side + i]);
            w = __ddiv_rn(omega_j, __dadd_rn(__dadd_rn(__dadd_rn(kw, ke), ks), kn));
        }
        wd[q] = (K)w;
    }
}

// Value of a stored element in the arithmetic type (undoes St<T>::put's rounding step only).
template <typename T> __device__ __forceinline__ typename St<T>::C as_c(T x) { return x; }
template <> __device__ __forceinline__ float as_c<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// Two plain damped-Jacobi sweeps in one pass (binary32 arithmetic: FP32 and bfloat16 cycles, where
// a sweep is DRAM-bound). Each warp owns a strip of 32 columns and marches down it: step r computes
// the first sweep's value at row r on all 32 columns (exactly a single sweep's operation order,
// rounded to the storage type; the column window of the input iterate rides in registers, the
// side neighbours come through L1) and the second sweep's value at row r - 1 on the 30 inner
// columns, the warp's output, taking the side neighbours' first-sweep values by shuffle. Strips
// overlap by one column on each side; a warp's rows overlap its neighbours' by one row above and
// below. No barrier: warps march independently and the unrolled march keeps several rows of loads
// in flight. Per node and pair of sweeps this reads e and g once and writes e once (12 B instead
// of 24 in FP32), and the result is bit-identical to two single sweeps.
constexpr int X2_OUT = 30;  // output columns per warp
template <typename T, bool BATCH, bool P>
__device__ __forceinline__ void jacobi2_x2_body(IterArgs a, int rows, int bx, int by, int bz) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // uniform over the block
    using C = typename St<T>::C;
    const int n = a.e_new.n;
    const int lane = threadIdx.x & 31;
    const int strip = bx * (JX / 32) + (threadIdx.x >> 5);
    if (strip * X2_OUT + 1 > n - 1) return;  // strip past the last column: the whole warp leaves
    const int i = strip * X2_OUT + lane;     // first-sweep column
    const bool col_in = i >= 1 && i <= n - 1;
    const bool out = col_in && lane >= 1 && lane <= X2_OUT;
    const int il = min(max(i, 1), n - 1);    // lanes outside the interior load from inside, keep 0
    const int j0 = by * rows + 1;    // second sweep: rows j0 .. j1 - 1
    const int j1 = min(j0 + rows, n);
    const int r0 = j0 - 1;                   // first sweep: rows r0 .. j1 (0 on rows 0 and n)
    const int64_t pe = a.e_old.pitch, pg = a.g.pitch, po = a.e_new.pitch;
    const int ra = max(r0, 1);
    const T* __restrict__ pE = cp<T>(a.e_old) + (int64_t)ra * pe + il;  // row r of the march
    const T* __restrict__ pG = cp<T>(a.g) + (int64_t)ra * pg + il;
    T* __restrict__ pO = wp<T>(a.e_new) + (int64_t)j0 * po + i;         // next output row
    const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
    C em = ldv<T, P>(pE - pe), ec = ldv<T, P>(pE);  // input iterate at rows r - 1, r
    // first sweep at row r (1 <= r <= n - 1), then advance the march one row
    auto first = [&](C& g) -> C {
        const C ep = ldv<T, P>(pE + pe), w = ldv<T, P>(pE - 1), e = ldv<T, P>(pE + 1);
        g = ldv<T, P>(pG);
        const C sum = (w + e) + (em + ep);
        const C v = as_c<T>(St<T>::put(fma(c1, ec, fma(om, sum, g))));
        em = ec;
        ec = ep;
        pE += pe;
        pG += pg;
        return col_in ? v : (C)0;
    };
    C s_prev = 0, s_cur = 0, g_cur = 0;  // first-sweep values at rows r - 2, r - 1; g at row r - 1
    // second sweep at row r - 1 given the first-sweep value v at row r
    auto second = [&](C v) {
        const C sw = __shfl_up_sync(0xffffffffu, s_cur, 1), se = __shfl_down_sync(0xffffffffu, s_cur, 1);
        if (out) *pO = St<T>::put(fma(c1, s_cur, fma(om, (sw + se) + (s_prev + v), g_cur)));
        pO += po;
    };
    if (r0 >= 1) s_cur = first(g_cur);  // row r0 (its g is never used)
    {
        C g;
        const C v = first(g);  // row j0
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    const int rb = min(j1, n - 1);
#pragma unroll 4
    for (int r = j0 + 1; r <= rb; ++r) {
        C g;
        const C v = first(g);
        second(v);
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    if (j1 == n) second((C)0);  // the first-sweep value on the boundary row n is 0
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(JX) k_jacobi2_x2(IterArgs a, int rows) {
    pdl_begin();
    jacobi2_x2_body<T, BATCH, false>(a, rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Packed binary32 pairs: add.f32x2 and fma.f32x2 (sm_100 and later) compute two binary32 results
// per instruction, each rounded exactly as the scalar instruction rounds it. (Written as PTX: the
// kernel below measured faster with these than with the runtime's intrinsics for the same
// instructions, 26.9 against 29.4 us per level-0 launch, at the same 32 registers.)
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
// Two adjacent stored values (4-byte aligned bfloat16 pair, 8-byte aligned binary32 pair) as
// binary32, the store of such a pair, and the storage rounding of a pair (bfloat16: to nearest).
template <typename T> __device__ __forceinline__ float2 ld2(const T* p);
template <> __device__ __forceinline__ float2 ld2<float>(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float2 unpack_bf16x2(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> __device__ __forceinline__ float2 ld2<__nv_bfloat16>(const __nv_bfloat16* p) {
    return unpack_bf16x2(__ldg(reinterpret_cast<const unsigned*>(p)));
}
__device__ __forceinline__ unsigned pack_bf16x2_rn(float2 v) {
    const __nv_bfloat162 t = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const unsigned*>(&t);
}
template <typename T> __device__ __forceinline__ void st2(T* p, float2 v);
template <> __device__ __forceinline__ void st2<float>(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
template <> __device__ __forceinline__ void st2<__nv_bfloat16>(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<unsigned*>(p) = pack_bf16x2_rn(v);
}
// Binary32 pairs in shared memory (the staged tiles of k_jacobi2_x2t): an aligned pair load and store.
__device__ __forceinline__ float2 ld2s(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2s(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
// Four adjacent bfloat16 values in shared memory (8-byte aligned) as two binary32 pairs, and back.
__device__ __forceinline__ void ld4s(const __nv_bfloat16* p, float2& lo, float2& hi) {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
    lo = unpack_bf16x2(w.x);
    hi = unpack_bf16x2(w.y);
}
__device__ __forceinline__ uint2 pack4(float2 lo, float2 hi) { return make_uint2(pack_bf16x2_rn(lo), pack_bf16x2_rn(hi)); }
template <typename T> __device__ __forceinline__ float2 round2(float2 v) { return v; }
template <> __device__ __forceinline__ float2 round2<__nv_bfloat16>(float2 v) { return unpack_bf16x2(pack_bf16x2_rn(v)); }

// Two plain damped-Jacobi sweeps in one pass, two adjacent columns per lane (binary32 arithmetic):
// the march of k_jacobi2_x2 with half the instructions per node. Lane L of a strip holds columns
// c0 and c0 + 1, c0 = 60 s - 2 + 2 L (even), and reads each row of e and g with one aligned pair
// load; the side neighbours of its two columns are its own pair and, for the outer ones, the
// adjacent lanes' (shuffle). Both sweeps run as packed binary32 pairs in the per-column kernel's
// operation order, so the result is bit-identical to two single sweeps. The first sweep runs on
// all 64 columns; lanes 1..30 store the second (60 output columns per strip). Pairs are loaded
// from column min(max(c0, 0), n rounded down to even), which may be the row's padding column
// n + 1 (the caller guarantees pitch >= n + 2); values of columns outside 1..n-1 are replaced by 0
// before any unmasked use.
// The solver uses this kernel for bfloat16 storage on lattices of at least X2P_MIN_N intervals:
// there the per-column kernel issues about 50 warp instructions per 32 nodes and pair of sweeps and
// is issue bound (70 % issue active), this one about 29. With binary32 storage (DRAM bound) and on
// smaller lattices (half as many warps) the per-column kernel measured faster.
constexpr int X2P_OUT = 60;     // output columns per warp
constexpr int X2P_MIN_N = 2048;
template <typename T, bool BATCH>
__device__ __forceinline__ void jacobi2_x2p_body(IterArgs a, int rows, int bx, int by, int bz) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // uniform over the block
    const int n = a.e_new.n;
    const int lane = threadIdx.x & 31;
    const int strip = bx * (JX / 32) + (threadIdx.x >> 5);
    if (strip * X2P_OUT > n - 1) return;  // strip past the last column: the whole warp leaves
    const int c0 = strip * X2P_OUT - 2 + 2 * lane;
    const int cl = min(max(c0, 0), n & ~1);
    const bool m0 = c0 >= 1 && c0 <= n - 1, m1 = c0 + 1 >= 1 && c0 + 1 <= n - 1;  // interior columns
    const bool mid = lane >= 1 && lane <= 30;
    const bool o0 = mid && m0, o1 = mid && m1;  // stored columns
    const int j0 = by * rows + 1;  // second sweep: rows j0 .. j1 - 1
    const int j1 = min(j0 + rows, n);
    const int r0 = j0 - 1;         // first sweep: rows r0 .. j1 (0 on rows 0 and n)
    const int64_t pe = a.e_old.pitch, pg = a.g.pitch, po = a.e_new.pitch;
    const int ra = max(r0, 1);
    const T* __restrict__ pE = cp<T>(a.e_old) + (int64_t)ra * pe + cl;  // row r of the march
    const T* __restrict__ pG = cp<T>(a.g) + (int64_t)ra * pg + cl;
    T* __restrict__ pO = wp<T>(a.e_new) + (int64_t)j0 * po + c0;        // next output row (stored when o0 or o1)
    const float2 om = make_float2(a.omega_f, a.omega_f), c1 = make_float2(a.c1_f, a.c1_f);
    float2 em = ld2<T>(pE - pe), ec = ld2<T>(pE);  // input iterate at rows r - 1, r
    // first sweep at row r (1 <= r <= n - 1) on the lane's two columns, then advance one row
    auto first = [&](float2& g) -> float2 {
        const float2 ep = ld2<T>(pE + pe);
        g = ld2<T>(pG);
        const float left = __shfl_up_sync(0xffffffffu, ec.y, 1), right = __shfl_down_sync(0xffffffffu, ec.x, 1);
        const float2 sum = add2(make_float2(left + ec.y, ec.x + right), add2(em, ep));  // (w + e) + (n + s)
        float2 v = round2<T>(fma2(c1, ec, fma2(om, sum, g)));
        v.x = m0 ? v.x : 0.f;
        v.y = m1 ? v.y : 0.f;
        em = ec;
        ec = ep;
        pE += pe;
        pG += pg;
        return v;
    };
    float2 s_prev = make_float2(0.f, 0.f), s_cur = s_prev, g_cur = s_prev;  // rows r - 2, r - 1; g at r - 1
    // second sweep at row r - 1 given the first-sweep values v at row r
    auto second = [&](float2 v) {
        const float sw = __shfl_up_sync(0xffffffffu, s_cur.y, 1), se = __shfl_down_sync(0xffffffffu, s_cur.x, 1);
        const float2 sum = add2(make_float2(sw + s_cur.y, s_cur.x + se), add2(s_prev, v));
        const float2 o = fma2(c1, s_cur, fma2(om, sum, g_cur));
        if (o0 && o1) st2<T>(pO, o);
        else {
            if (o0) pO[0] = St<T>::put(o.x);
            if (o1) pO[1] = St<T>::put(o.y);
        }
        pO += po;
    };
    if (r0 >= 1) s_cur = first(g_cur);  // row r0 (its g is never used)
    {
        float2 g;
        const float2 v = first(g);  // row j0
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    const int rb = min(j1, n - 1);
#pragma unroll 4
    for (int r = j0 + 1; r <= rb; ++r) {
        float2 g;
        const float2 v = first(g);
        second(v);
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    if (j1 == n) second(make_float2(0.f, 0.f));  // the first-sweep value on the boundary row n is 0
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(JX, 16) k_jacobi2_x2p(IterArgs a, int rows) {  // 32 registers: full occupancy
    pdl_begin();
    jacobi2_x2p_body<T, BATCH>(a, rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// K plain damped-Jacobi sweeps in one pass (K >= 3; binary32 arithmetic), the K-level form of
// k_jacobi2_x2: each warp marches a strip of 32 columns; step r computes sweep 1 at row r, sweep 2
// at row r - 1, ..., sweep K at row r - K + 1 (the output), each from the previous sweep's values
// at three rows (registers) and its side neighbours (shuffle), every intermediate rounded to the
// storage type as a stored sweep would be. A strip outputs its 34 - 2K inner columns; a block's
// march starts K - 1 rows above its output rows and ends K - 1 below. Sweep values on the boundary
// rows and columns are 0. Per node and K sweeps this reads e and g once and writes e once.
template <typename T, bool BATCH, int K, bool P>
__device__ __forceinline__ void jacobi2_xk_body(IterArgs a, int rows, int bx, int by, int bz) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // uniform over the block
    using C = typename St<T>::C;
    constexpr int OUTK = 34 - 2 * K;
    const int n = a.e_new.n;
    const int lane = threadIdx.x & 31;
    const int strip = bx * (JX / 32) + (threadIdx.x >> 5);
    if (strip * OUTK + 1 > n - 1) return;        // strip past the last column: the whole warp leaves
    const int i = strip * OUTK + lane - (K - 2);  // this lane's column
    const bool col_in = i >= 1 && i <= n - 1;
    const bool out = col_in && lane >= K - 1 && lane <= 32 - K;
    const int il = min(max(i, 1), n - 1);  // lanes outside the interior load from inside, keep 0
    const int j0 = by * rows + 1;  // output rows j0 .. j1 - 1
    const int j1 = min(j0 + rows, n);
    const int64_t pe = a.e_old.pitch, pg = a.g.pitch, po = a.e_new.pitch;
    const T* __restrict__ E0 = cp<T>(a.e_old) + il;
    const T* __restrict__ G0 = cp<T>(a.g) + il;
    T* __restrict__ O = wp<T>(a.e_new);
    const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
    // Loads use rows clamped into 0..n, so that the march has no branch and the unrolled loop can
    // issue several rows of loads ahead; values on rows outside 1..n-1 are then replaced by 0.
    auto rowE = [&](int row) { return E0 + (int64_t)min(max(row, 0), n) * pe; };
    const int rf = j0 - (K - 1), rl = j1 + K - 2;  // sweep-1 rows of the march
    C em = ldv<T, P>(rowE(rf - 1)), ec = ldv<T, P>(rowE(rf));  // input iterate at rows r - 1, r (exact where used)
    C sp[K], sc[K], gq[K];  // sweep l (1..K-1) at rows x - 1, x of sweep l + 1's row x; g at rows r .. r - K + 1
#pragma unroll
    for (int l = 0; l < K; ++l) sp[l] = sc[l] = gq[l] = 0;
#pragma unroll 4
    for (int r = rf; r <= rl; ++r) {
        C v[K + 1];
        const T* p = rowE(r);
        const C ep = ldv<T, P>(rowE(r + 1)), w = ldv<T, P>(p - 1), e = ldv<T, P>(p + 1);
        const C g = ldv<T, P>(G0 + (int64_t)min(max(r, 0), n) * pg);
        {
            const C y = as_c<T>(St<T>::put(fma(c1, ec, fma(om, (w + e) + (em + ep), g))));
            v[1] = (col_in && r >= 1 && r <= n - 1) ? y : (C)0;
        }
        em = ec;
        ec = ep;
#pragma unroll
        for (int l = K - 1; l >= 1; --l) gq[l] = gq[l - 1];
        gq[0] = g;
#pragma unroll
        for (int l = 2; l <= K; ++l) {
            const int x = r - l + 1;  // sweep l's row: sweep l - 1 is known at x - 1, x, x + 1
            const C sw = __shfl_up_sync(0xffffffffu, sc[l - 1], 1), se = __shfl_down_sync(0xffffffffu, sc[l - 1], 1);
            const C y = fma(c1, sc[l - 1], fma(om, (sw + se) + (sp[l - 1] + v[l - 1]), gq[l - 1]));
            if (l < K) {
                v[l] = (col_in && x >= 1 && x <= n - 1) ? as_c<T>(St<T>::put(y)) : (C)0;
            } else if (out && x >= j0 && x < j1) {
                O[(int64_t)x * po + i] = St<T>::put(y);
            }
            sp[l - 1] = sc[l - 1];
            sc[l - 1] = v[l - 1];
        }
    }
}

template <typename T, bool BATCH, int K>
__global__ void __launch_bounds__(JX) k_jacobi2_xk(IterArgs a, int rows) {
    pdl_begin();
    jacobi2_xk_body<T, BATCH, K, false>(a, rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Two plain damped-Jacobi sweeps of a large single-problem lattice with the tile staged by TMA
// (binary32 and bfloat16 storage, 2-D lattice form). A block owns XT_OUT output columns c0 ..
// c0 + XT_OUT - 1 (c0 = XT_OUT * blockIdx.x) and RT output rows r0 .. r0 + RT - 1. One thread
// issues two TMA tensor copies: the input iterate's rows r0 - 2 .. r0 + RT + 1 and the source's
// rows r0 - 1 .. r0 + RT, XT_W columns from c0 - 8 each (a multiple of 8: the copy's innermost
// coordinate must sit on a 16-byte boundary; zero outside the lattice), into shared memory. Thread t
// owns Q adjacent staged columns from Q t (Q = 2 for binary32, 4 for bfloat16; XT_W / Q threads):
// it computes the first sweep on rows r0 - 1 .. r0 + RT into a
// shared buffer (rounded to the storage type as a stored sweep is, 0 outside the interior), then,
// after a block barrier, the second sweep on the output rows, stored to global memory. Both
// sweeps run as packed binary32 pairs in the per-column kernel's operation order, so the result is
// bit-identical to two single sweeps. The copy's completion barrier is waited on with a bound: on
// expiry the block records State::fault, waits once more (bounded) so no copy lands after it
// leaves, and returns without storing.
constexpr int XT_W = 256;    // staged columns (the TMA box width)
constexpr int XT_OUT = 240;  // output columns per block (staged columns 8 .. 247)
constexpr long long kXtWaitNs = 1000000000ll;

__device__ __forceinline__ bool xt_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"((uint32_t)__cvta_generic_to_shared(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool xt_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = device_clock_ns();
    for (;;) {
        if (xt_try_wait(bar, parity)) return true;
        if (device_clock_ns() - t0 > kXtWaitNs) return false;
    }
}
__device__ __forceinline__ void xt_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"((uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
}

// The two sweeps of k_jacobi2_x2t from its staged tiles, two columns per thread (binary32 storage):
// first-sweep values outside the interior are replaced by 0 and stores are masked.
template <int RT>
__device__ __forceinline__ void x2t_sweeps(const IterArgs& a, const float* SE, const float* SG, float* S1, int x, int r0) {
    using T = float;
    constexpr bool MASK = true;
    constexpr int GR = RT + 2;
    const int t = threadIdx.x;
    const int n = a.e_new.n;
    const float2 om = make_float2(a.omega_f, a.omega_f), c1 = make_float2(a.c1_f, a.c1_f);
    const bool m0 = !MASK || (x >= 1 && x <= n - 1), m1 = !MASK || (x + 1 >= 1 && x + 1 <= n - 1);  // interior columns
    // first sweep, rows r0 - 1 .. r0 + RT (shared rows 0 .. GR - 1), staged columns 2 .. 253
    if (t >= 1 && t < XT_W / 2 - 1) {
        const T* col = SE + 2 * t;
        float2 em = ld2s(col), ec = ld2s(col + XT_W);
#pragma unroll 4
        for (int p = 0; p < GR; ++p) {
            const T* row = col + (p + 1) * XT_W;  // iterate row r0 - 1 + p
            const float2 ep = ld2s(row + XT_W);
            const float left = as_c<T>(row[-1]), right = as_c<T>(row[2]);
            const float2 g = ld2s(SG + p * XT_W + 2 * t);
            const float2 sum = add2(make_float2(left + ec.y, ec.x + right), add2(em, ep));  // (w + e) + (s + n)
            float2 v = fma2(c1, ec, fma2(om, sum, g));
            if (MASK) {
                const int r = r0 - 1 + p;
                const bool rin = r >= 1 && r <= n - 1;
                v.x = (rin && m0) ? v.x : 0.f;
                v.y = (rin && m1) ? v.y : 0.f;
            }
            st2s(S1 + p * XT_W + 2 * t, v);
            em = ec;
            ec = ep;
        }
    }
    __syncthreads();
    // second sweep, output rows r0 .. r0 + RT - 1 (shared rows 1 .. RT), staged columns 8 .. 247
    if (t >= 4 && t < 4 + XT_OUT / 2) {
        T* __restrict__ O = wp<T>(a.e_new);
        const int64_t po = a.e_new.pitch;
        const T* col = S1 + 2 * t;
        float2 sp = ld2s(col), sc = ld2s(col + XT_W);
        const int pe = MASK ? min(RT, n - r0) : RT;  // output rows inside the lattice
#pragma unroll 4
        for (int p = 1; p <= pe; ++p) {
            const T* row = col + p * XT_W;
            const float2 sn = ld2s(row + XT_W);
            const float left = as_c<T>(row[-1]), right = as_c<T>(row[2]);
            const float2 g = ld2s(SG + p * XT_W + 2 * t);
            const float2 sum = add2(make_float2(left + sc.y, sc.x + right), add2(sp, sn));
            const float2 o = fma2(c1, sc, fma2(om, sum, g));
            T* dst = O + (int64_t)(r0 - 1 + p) * po + x;
            if (m0 && m1) st2<T>(dst, o);
            else {
                if (m0) dst[0] = St<T>::put(o.x);
                if (m1) dst[1] = St<T>::put(o.y);
            }
            sp = sc;
            sc = sn;
        }
    }
}

// The two sweeps of k_jacobi2_x2t with four adjacent columns per thread (bfloat16 storage, whose
// kernel is bound by instruction issue): one 8-byte shared load per row for four columns, and the
// side neighbours of the outer two; the same per-column operations as two pairs.
template <int RT, bool MASK>
__device__ __forceinline__ void x2t_sweeps4(const IterArgs& a, const __nv_bfloat16* SE, const __nv_bfloat16* SG,
                                            __nv_bfloat16* S1, int x, int r0) {
    using T = __nv_bfloat16;
    constexpr int GR = RT + 2;
    const int t = threadIdx.x;
    const int n = a.e_new.n;
    const float2 om = make_float2(a.omega_f, a.omega_f), c1 = make_float2(a.c1_f, a.c1_f);
    bool m[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) m[k] = !MASK || (x + k >= 1 && x + k <= n - 1);  // interior columns
    // first sweep, rows r0 - 1 .. r0 + RT (shared rows 0 .. GR - 1), staged columns 4 .. 251
    if (t >= 1 && t < XT_W / 4 - 1) {
        const T* col = SE + 4 * t;
        float2 emL, emH, ecL, ecH;
        ld4s(col, emL, emH);
        ld4s(col + XT_W, ecL, ecH);
#pragma unroll 4
        for (int p = 0; p < GR; ++p) {
            const T* row = col + (p + 1) * XT_W;  // iterate row r0 - 1 + p
            float2 epL, epH, gL, gH;
            ld4s(row + XT_W, epL, epH);
            ld4s(SG + p * XT_W + 4 * t, gL, gH);
            const float left = as_c<T>(row[-1]), right = as_c<T>(row[4]);
            // (w + e) + (s + n) per column
            const float2 sL = add2(make_float2(left + ecL.y, ecL.x + ecH.x), add2(emL, epL));
            const float2 sH = add2(make_float2(ecL.y + ecH.y, ecH.x + right), add2(emH, epH));
            float2 vL = fma2(c1, ecL, fma2(om, sL, gL)), vH = fma2(c1, ecH, fma2(om, sH, gH));
            if (MASK) {
                const int r = r0 - 1 + p;
                const bool rin = r >= 1 && r <= n - 1;
                vL.x = (rin && m[0]) ? vL.x : 0.f;
                vL.y = (rin && m[1]) ? vL.y : 0.f;
                vH.x = (rin && m[2]) ? vH.x : 0.f;
                vH.y = (rin && m[3]) ? vH.y : 0.f;
            }
            *reinterpret_cast<uint2*>(S1 + p * XT_W + 4 * t) = pack4(vL, vH);  // rounded to bfloat16 (0 stays 0)
            emL = ecL;
            emH = ecH;
            ecL = epL;
            ecH = epH;
        }
    }
    __syncthreads();
    // second sweep, output rows r0 .. r0 + RT - 1 (shared rows 1 .. RT), staged columns 8 .. 247
    if (t >= 2 && t < 2 + XT_OUT / 4) {
        T* __restrict__ O = wp<T>(a.e_new);
        const int64_t po = a.e_new.pitch;
        const T* col = S1 + 4 * t;
        float2 spL, spH, scL, scH;
        ld4s(col, spL, spH);
        ld4s(col + XT_W, scL, scH);
        const int pe = MASK ? min(RT, n - r0) : RT;  // output rows inside the lattice
        const bool all = m[0] && m[1] && m[2] && m[3];
#pragma unroll 4
        for (int p = 1; p <= pe; ++p) {
            const T* row = col + p * XT_W;
            float2 snL, snH, gL, gH;
            ld4s(row + XT_W, snL, snH);
            ld4s(SG + p * XT_W + 4 * t, gL, gH);
            const float left = as_c<T>(row[-1]), right = as_c<T>(row[4]);
            const float2 sL = add2(make_float2(left + scL.y, scL.x + scH.x), add2(spL, snL));
            const float2 sH = add2(make_float2(scL.y + scH.y, scH.x + right), add2(spH, snH));
            const float2 oL = fma2(c1, scL, fma2(om, sL, gL)), oH = fma2(c1, scH, fma2(om, sH, gH));
            T* dst = O + (int64_t)(r0 - 1 + p) * po + x;
            if (all) *reinterpret_cast<uint2*>(dst) = pack4(oL, oH);
            else {
                const float o[4] = {oL.x, oL.y, oH.x, oH.y};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (m[k]) dst[k] = St<T>::put(o[k]);
            }
            spL = scL;
            spH = scH;
            scL = snL;
            scH = snH;
        }
    }
}

template <typename T, int RT, int Q>
__global__ void __launch_bounds__(XT_W / Q) k_jacobi2_x2t(IterArgs a, const __grid_constant__ CUtensorMap me,
                                                          const __grid_constant__ CUtensorMap mg, int* fault) {
    pdl_begin();
    constexpr int ER = RT + 4, GR = RT + 2;  // staged rows of the iterate and of the source
    extern __shared__ __align__(128) unsigned char xt_smem[];
    T* SE = reinterpret_cast<T*>(xt_smem);  // [ER][XT_W]: iterate rows r0 - 2 ..
    T* SG = SE + ER * XT_W;                  // [GR][XT_W]: source rows r0 - 1 ..
    T* S1 = SG + GR * XT_W;                  // [GR][XT_W]: first sweep, rows r0 - 1 ..
    uint64_t* bar = reinterpret_cast<uint64_t*>(S1 + GR * XT_W);
    const int t = threadIdx.x;
    const int n = a.e_new.n;
    const int c0 = blockIdx.x * XT_OUT, r0 = blockIdx.y * RT + 1;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (t == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
                     "r"((uint32_t)((ER + GR) * XT_W * sizeof(T)))
                     : "memory");
        xt_load_2d(SE, &me, c0 - 8, r0 - 2, bar);
        xt_load_2d(SG, &mg, c0 - 8, r0 - 1, bar);
    }
    if (!__syncthreads_and(xt_wait(bar, 0))) {
        if (t == 0) atomicExch(fault, 1);
        xt_wait(bar, 0);  // one more bounded wait before the block's shared memory is released
        return;
    }
    const int x = c0 - 8 + Q * t;  // this thread's first column
    // A tile whose first-sweep area (at most staged columns 2 .. 253, rows r0 - 1 .. r0 + RT) lies
    // inside the lattice's interior needs no masking. Measured at 4097² (same box, A/B, two columns
    // per thread): the bfloat16 kernel, bound by instruction issue, ran a level-0 pair in 23.4 us with
    // the unmasked interior path against 26.0 us without (20.9 us with four columns per thread); the
    // binary32 one, bound by memory latency, in 39.4 against 38.3 us, so it keeps the masked path.
    const bool inner = c0 - 6 >= 1 && c0 + 245 <= n - 1 && r0 - 1 >= 1 && r0 + RT <= n - 1;
    if constexpr (Q == 4) {
        if (inner) x2t_sweeps4<RT, false>(a, SE, SG, S1, x, r0);
        else x2t_sweeps4<RT, true>(a, SE, SG, S1, x, r0);
    } else {
        x2t_sweeps<RT>(a, SE, SG, S1, x, r0);
    }
}

// Fast lattice-form level change at stride 2 (2-D): lattice nodes copy Gc; the others take the
// stride-2 interpolant of Gc - dl, formed along each marching column (see ColumnInterp2).
template <typename T, bool BATCH, bool P>
__device__ __forceinline__ void prolong2_s1_body(ProlongArgs a, int rows, int bx, int by, int bz) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // compiled into batch launches only
    using C = typename St<T>::C;
    const int n = a.G.n;
    const int i = bx * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = by * rows + 1;
    const int j1 = min(j0 + rows, n);
    const bool iodd = i & 1;
    ColumnInterp2<T, P> ci;
    ci.d = cp<T>(a.Gc) + (i >> 1);
    ci.d2 = cp<T>(a.dl) + (i >> 1);
    ci.pitch = a.Gc.pitch;
    ci.pitch2 = a.dl.pitch;
    ci.hx = iodd ? (C)0.5 : (C)0;
    for (int j = j0; j < j1; ++j) {
        C v = ci.at(j);
        if (!(j & 1) && !iodd) v = ldv<T, P>(cp<T>(a.Gc) + (int64_t)(j >> 1) * a.Gc.pitch + (i >> 1));
        wp<T>(a.G)[(int64_t)j * a.G.pitch + i] = St<T>::put(v);
    }
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(JX) k_prolong2_s1(ProlongArgs a, int rows) {
    pdl_begin();
    prolong2_s1_body<T, BATCH, false>(a, rows, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Lattice form, binary32 cycles (2-D): one level's whole run on a small lattice (at most
// RUN_MAX_N intervals per side) in one block of n x RUN_Y threads, the level's iterate, source
// and pending variation held in shared memory between sweeps instead of one launch per sweep (or
// pair). Steps, in the arithmetic of the separate kernels: the level change from the coarser
// lattice's final iterate Gc and variation dl (k_prolong2_s1), then `sweeps` damped-Jacobi sweeps
// (k_jacobi2), the first adding the pending stride-2 interpolation of dl off the lattice, every
// sweep's values rounded to the storage type as a stored sweep is; the last sweep also writes the
// iterate (e_new) and, when requested, its variation (dnew). The results are bit-identical to the
// separate launches. Batches: one block per problem (blockIdx.z).
constexpr int RUN_Y = 8;  // thread rows of a level-run block (its columns: one per lattice column)

// One sweep of a level run: each thread marches down its column through its band of rows.
template <typename T, bool FIRST, bool LAST>
__device__ __forceinline__ void run_sweep(const T* __restrict__ src, T* __restrict__ dst, const T* __restrict__ SG,
                                          const T* __restrict__ SD, int n, int j0, int j1, typename St<T>::C c1,
                                          typename St<T>::C om, const IterArgs& it) {
    using C = typename St<T>::C;
    const int np = n + 1, nc = (n >> 1) + 1;  // row lengths of the lattice and of the coarse variation
    const int i = 1 + threadIdx.x;
    if (i >= n || j0 >= j1) return;
    const C hx = (i & 1) ? (C)0.5 : (C)0;
    auto X = [&](int JJ) -> C {  // x-interpolant of compact row JJ of dl at this column
        const C a = as_c<T>(SD[JJ * nc + (i >> 1)]), b = as_c<T>(SD[JJ * nc + (i >> 1) + 1]);
        return fma(hx, b - a, a);
    };
    C vs = as_c<T>(src[(j0 - 1) * np + i]), vc = as_c<T>(src[j0 * np + i]);
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const C vn = as_c<T>(src[(j + 1) * np + i]);
        const C w = as_c<T>(src[j * np + i - 1]), e = as_c<T>(src[j * np + i + 1]);
        C v = jacobi_update(c1, om, vc, as_c<T>(SG[j * np + i]), w, e, vs, vn);
        if (LAST && it.dnew.p) wp<T>(it.dnew)[(int64_t)j * it.dnew.pitch + i] = St<T>::put(v - vc);
        if (FIRST) {
            const C sv = (j & 1) ? (C)0.5 * (X(j >> 1) + X((j >> 1) + 1)) : X(j >> 1);
            v += ((i | j) & 1) ? sv : (C)0;
        }
        const T out = St<T>::put(v);
        dst[j * np + i] = out;
        if (LAST) wp<T>(it.e_new)[(int64_t)j * it.e_new.pitch + i] = out;
        vs = vc;
        vc = vn;
    }
}

template <typename T, bool BATCH>
__global__ void __launch_bounds__(RUN_MAX_N * RUN_Y) k_level_run2(ProlongArgs pr, IterArgs it, int sweeps) {
    pdl_begin();
    if (BATCH) {
        if (!batch_view<T>(pr, blockIdx.z)) return;  // this problem has converged (uniform over the block)
        batch_view<T>(it, blockIdx.z);
    }
    using C = typename St<T>::C;
    const int n = it.e_new.n, np = n + 1, nc = (n >> 1) + 1;
    extern __shared__ __align__(16) unsigned char run_smem[];
    T* S0 = reinterpret_cast<T*>(run_smem);  // iterate, ping
    T* S1 = S0 + np * np;                     // iterate, pong (holds Gc until the first sweep)
    T* SG = S1 + np * np;                     // source
    T* SD = SG + np * np;                     // the coarser lattice's variation dl (compact)
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * RUN_Y;
    // stage the source, Gc (into S1) and dl; zero the boundary of S0
    for (int q = tid; q < np * np; q += nt) {
        const int i = q % np, j = q / np;
        SG[q] = cp<T>(it.g)[(int64_t)j * it.g.pitch + i];
        if (i == 0 || j == 0 || i == n || j == n) S0[q] = St<T>::put((C)0);
    }
    for (int q = tid; q < nc * nc; q += nt) {
        const int I = q % nc, J = q / nc;
        S1[q] = cp<T>(pr.Gc)[(int64_t)J * pr.Gc.pitch + I];
        SD[q] = cp<T>(pr.dl)[(int64_t)J * pr.dl.pitch + I];
    }
    __syncthreads();
    // level change: lattice nodes copy Gc, the others take the stride-2 interpolant of Gc - dl
    for (int j = 1 + threadIdx.y; j < n; j += RUN_Y)
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
            const int I = i >> 1, J = j >> 1;
            const C hx = (i & 1) ? (C)0.5 : (C)0;
            auto X = [&](int JJ) -> C {
                C a = as_c<T>(S1[JJ * nc + I]), b = as_c<T>(S1[JJ * nc + I + 1]);
                a -= as_c<T>(SD[JJ * nc + I]);
                b -= as_c<T>(SD[JJ * nc + I + 1]);
                return fma(hx, b - a, a);
            };
            C v = (j & 1) ? (C)0.5 * (X(J) + X(J + 1)) : X(J);
            if (!(j & 1) && !(i & 1)) v = as_c<T>(S1[J * nc + I]);
            S0[j * np + i] = St<T>::put(v);
        }
    __syncthreads();
    // the boundary of S1 (the first sweep writes its interior)
    for (int q = tid; q < np * np; q += nt) {
        const int i = q % np, j = q / np;
        if (i == 0 || j == 0 || i == n || j == n) S1[q] = St<T>::put((C)0);
    }
    const C om = pick<C>(it.omega, it.omega_f), c1 = pick<C>(it.c1, it.c1_f);
    const int band = (n - 1 + RUN_Y - 1) / RUN_Y;
    const int j0 = 1 + threadIdx.y * band, j1 = min(j0 + band, n);
    if (sweeps == 1) {
        run_sweep<T, true, true>(S0, S1, SG, SD, n, j0, j1, c1, om, it);
        return;
    }
    run_sweep<T, true, false>(S0, S1, SG, SD, n, j0, j1, c1, om, it);
    __syncthreads();
    T* src = S1;
    T* dst = S0;
    for (int s = 1; s + 1 < sweeps; ++s) {
        run_sweep<T, false, false>(src, dst, SG, SD, n, j0, j1, c1, om, it);
        __syncthreads();
        T* t = src;
        src = dst;
        dst = t;
    }
    run_sweep<T, false, true>(src, dst, SG, SD, n, j0, j1, c1, om, it);
}

// Fast V-cycle kernels (2-D, column marching): level residual rho = g + omega (sum - 4 v) in 5
// instructions per node, and the stride-2 prolongation-add e += P ec with the x-interpolant shared
// down each column (lattice nodes take the coarse value itself, which ColumnInterp2 returns there).
template <typename T>
__global__ void __launch_bounds__(JX) k_vresid2_fast(VResidArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.rho.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const T* __restrict__ E = cp<T>(a.e);
    const int64_t pe = a.e.pitch;
    const T* __restrict__ G = cp<T>(a.g);
    const C om = pick<C>(a.omega, (float)a.omega);
    C vs = St<T>::ld(E + (int64_t)(j0 - 1) * pe + i);
    C vc = St<T>::ld(E + (int64_t)j0 * pe + i);
    for (int j = j0; j < j1; ++j) {
        const T* row = E + (int64_t)j * pe + i;
        const C vn = St<T>::ld(row + pe);
        const C sum = (St<T>::ld(row - 1) + St<T>::ld(row + 1)) + (vs + vn);
        const C g = St<T>::ld(G + (int64_t)j * a.g.pitch + i);
        wp<T>(a.rho)[(int64_t)j * a.rho.pitch + i] = St<T>::put(fma(om, fma((C)-4, vc, sum), g));
        vs = vc;
        vc = vn;
    }
}

template <typename T>
__global__ void __launch_bounds__(JX) k_prolong_add2_s1(ProlongAddArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.e.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    ColumnInterp2<T> ci;
    ci.d = cp<T>(a.ec) + (i >> 1);
    ci.d2 = nullptr;
    ci.pitch = a.ec.pitch;
    ci.pitch2 = 0;
    ci.hx = (i & 1) ? (C)0.5 : (C)0;
    T* __restrict__ E = wp<T>(a.e);
    for (int j = j0; j < j1; ++j) {
        T* p = E + (int64_t)j * a.e.pitch + i;
        *p = St<T>::put(St<T>::rd(p) + ci.at(j));
    }
}

constexpr int J3X = 32, J3Y = 4;

template <bool PEND, bool WD, typename T>
__global__ void __launch_bounds__(J3X * J3Y) k_jacobi3(IterArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.e_new.n;
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (i >= n || j >= n) return;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    const T* __restrict__ E = cp<T>(a.e_old);
    const int64_t pe = a.e_old.pitch, ple = (int64_t)(n + 1) * pe;
    T* __restrict__ O = wp<T>(a.e_new);
    const int64_t po = a.e_new.pitch, plo = (int64_t)(n + 1) * po;
    const T* __restrict__ G = cp<T>(a.g);
    const int64_t pg = a.g.pitch, plg = (int64_t)(n + 1) * pg;
    const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    const T* col = E + (int64_t)j * pe + i;
    C vb = St<T>::ld(col + (int64_t)(k0 - 1) * ple);
    C vc = St<T>::ld(col + (int64_t)k0 * ple);
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
        const T* p = col + (int64_t)k * ple;
        const C vt = St<T>::ld(p + ple);
        const C w = St<T>::ld(p - 1), e = St<T>::ld(p + 1), sn = St<T>::ld(p - pe), nn = St<T>::ld(p + pe);
        const C g = St<T>::ld(G + (int64_t)k * plg + (int64_t)j * pg + i);
        C v = jacobi_update(c1, om, vc, g, w, e, sn, nn, vb, vt);
        if (WD) wp<T>(a.dnew)[(int64_t)k * (n + 1) * a.dnew.pitch + (int64_t)j * a.dnew.pitch + i] = St<T>::put(v - vc);
        if (PEND && ((i | j | k) & lpm)) v += interp<3, false, false, T>(a.dprev, a.dprev, a.mp, i, j, k);
        O[(int64_t)k * plo + (int64_t)j * po + i] = St<T>::put(v);
        vb = vc;
        vc = vt;
    }
}

// FP64 3-D iteration with a shared neighbour pair: D(i, j, k) = v(i+1, j, k) + v(i, j, k+1) is the
// east + top sum of node (i, j, k) and the west + bottom sum of node (i+1, j, k+1), the left lane's
// pair from the step before. With the south + north sum that leaves 6 FP64 instructions per node
// instead of the 7 of the FMA chain; lane 0 of each warp holds the column left of the warp's 31
// output columns and only forms its pair (6 x 32 / 31 = 6.19 per output node).
template <bool PEND, bool WD>
__global__ void __launch_bounds__(J3X * J3Y) k_jacobi3d(IterArgs a, int rows) {
    pdl_begin();
    const int n = a.e_new.n;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (j >= n) return;  // uniform over the warp (one thread row)
    const int iu = blockIdx.x * JD_COLS + threadIdx.x;
    if (blockIdx.x * JD_COLS + 1 > n - 1) return;
    const int i = min(iu, n - 1);
    const bool out = threadIdx.x > 0 && iu <= n - 1;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    const double* __restrict__ E = cp<double>(a.e_old);
    const int64_t pe = a.e_old.pitch, ple = (int64_t)(n + 1) * pe;
    double* __restrict__ O = wp<double>(a.e_new);
    const int64_t po = a.e_new.pitch, plo = (int64_t)(n + 1) * po;
    const double* __restrict__ G = cp<double>(a.g);
    const int64_t pg = a.g.pitch, plg = (int64_t)(n + 1) * pg;
    const double om = a.omega, c1 = a.c1, one = a.one;
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    const double* col = E + (int64_t)j * pe + i;
    double vc = __ldg(col + (int64_t)k0 * ple);
    double dp = fma(one, __ldg(col + (int64_t)(k0 - 1) * ple + 1), vc);  // D(i, j, k0 - 1)
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
        const double* p = col + (int64_t)k * ple;
        const double vt = __ldg(p + ple);
        const double e = __ldg(p + 1), sn = __ldg(p - pe), nn = __ldg(p + pe);
        const double g = __ldg(G + (int64_t)k * plg + (int64_t)j * pg + i);
        const double dw = __shfl_up_sync(0xffffffffu, dp, 1);  // D(i-1, j, k-1): west + bottom
        const double dh = fma(one, e, vt);                       // D(i, j, k): east + top
        double v = fma(om, dh, fma(om, dw, fma(om, fma(one, sn, nn), fma(c1, vc, g))));
        if (WD && out) wp<double>(a.dnew)[(int64_t)k * (n + 1) * a.dnew.pitch + (int64_t)j * a.dnew.pitch + i] = v - vc;
        if (PEND && out && ((i | j | k) & lpm)) v += interp<3, false, false, double>(a.dprev, a.dprev, a.mp, i, j, k);
        if (out) O[(int64_t)k * plo + (int64_t)j * po + i] = v;
        dp = dh;
        vc = vt;
    }
}


// Two plain sweeps of the 3-D lattice form in one pass (binary32 arithmetic: FP32 and bfloat16
// cycles, where a sweep is DRAM bound). A block of 32 x J3Y2 threads owns a tile of columns
// (x, y) and marches down z: step r computes the first sweep at plane r on every thread of the
// tile (exactly a single sweep's operation order, rounded to the storage type; side neighbours
// through L1, the neighbours along z in registers) and the second sweep at plane r - 1 on the inner
// (32 - 2) x (J3Y2 - 2) threads, taking the first-sweep values of the x neighbours by shuffle and of
// the y neighbours from the previous step's plane in shared memory. Planes are triple-buffered, so
// one block barrier per step separates every write from the reads of it and from its next
// overwrite. Tiles overlap by one column and row on each side; a block's march starts one plane
// above its output planes and ends one below. Threads outside the interior load from inside (clamped
// indexes) and keep 0. Per node and pair of sweeps this reads e and g once and writes e once, and
// the result is bit-identical to two single sweeps.
constexpr int J3Y2 = 16;  // thread rows of the 3-D pair kernel
template <typename T>
__global__ void __launch_bounds__(J3X * J3Y2) k_jacobi3_x2(IterArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    __shared__ C pl[3][J3Y2][J3X];  // first-sweep planes, plane r in pl[r % 3]
    const int n = a.e_new.n;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.x * (J3X - 2) + tx;   // outputs on tx 1 .. J3X - 2
    const int j = blockIdx.y * (J3Y2 - 2) + ty;  // outputs on ty 1 .. J3Y2 - 2
    const bool col_in = i >= 1 && i <= n - 1 && j >= 1 && j <= n - 1;
    const bool out = col_in && tx >= 1 && tx <= J3X - 2 && ty >= 1 && ty <= J3Y2 - 2;
    const int il = min(max(i, 1), n - 1), jl = min(max(j, 1), n - 1);
    const int k0 = blockIdx.z * rows + 1;  // second sweep: planes k0 .. k1 - 1
    const int k1 = min(k0 + rows, n);
    const int r0 = k0 - 1;                 // first sweep: planes r0 .. k1 (0 on planes 0 and n)
    const int64_t pe = a.e_old.pitch, ple = (int64_t)(n + 1) * pe;
    const int64_t pg = a.g.pitch, plg = (int64_t)(n + 1) * pg;
    const int64_t po = a.e_new.pitch, plo = (int64_t)(n + 1) * po;
    const T* __restrict__ colE = cp<T>(a.e_old) + (int64_t)jl * pe + il;
    const T* __restrict__ colG = cp<T>(a.g) + (int64_t)jl * pg + il;
    T* __restrict__ colO = wp<T>(a.e_new) + (int64_t)j * po + i;
    const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
    const int ra = max(r0, 1);
    C em = St<T>::ld(colE + (int64_t)(ra - 1) * ple), ec = St<T>::ld(colE + (int64_t)ra * ple);
    // first sweep at plane r (1 <= r <= n - 1); returns the value (0 off the interior) and its g
    auto first = [&](int r, C& g) -> C {
        const T* p = colE + (int64_t)r * ple;
        const C ep = St<T>::ld(p + ple);
        const C w = St<T>::ld(p - 1), e = St<T>::ld(p + 1), sn = St<T>::ld(p - pe), nn = St<T>::ld(p + pe);
        g = St<T>::ld(colG + (int64_t)r * plg);
        const C y = as_c<T>(St<T>::put(fma(c1, ec, fma(om, ((w + e) + (sn + nn)) + (em + ep), g))));
        em = ec;
        ec = ep;
        return col_in ? y : (C)0;
    };
    C s_prev = 0, s_cur = 0, g_cur = 0;  // first-sweep values at planes x - 1, x; g at plane x
    // second sweep at plane x given the first-sweep value v at plane x + 1 (pl[x % 3] complete)
    auto second = [&](int x, C v) {
        const C sw = __shfl_up_sync(0xffffffffu, s_cur, 1), se = __shfl_down_sync(0xffffffffu, s_cur, 1);
        if (out) {
            const C ss = pl[x % 3][ty - 1][tx], sn = pl[x % 3][ty + 1][tx];
            colO[(int64_t)x * plo] = St<T>::put(fma(c1, s_cur, fma(om, ((sw + se) + (ss + sn)) + (s_prev + v), g_cur)));
        }
    };
    if (r0 >= 1) {
        C g;
        s_cur = first(r0, g);  // plane r0: only its own value is used (the z neighbour of plane k0)
    }
    {
        C g;
        const C v = first(k0, g);
        pl[k0 % 3][ty][tx] = v;
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    const int rb = min(k1, n - 1);
    for (int r = k0 + 1; r <= rb; ++r) {
        C g;
        const C v = first(r, g);
        pl[r % 3][ty][tx] = v;
        __syncthreads();  // plane r - 1 is complete (written last step); plane r's buffer is free
        second(r - 1, v);
        s_prev = s_cur;
        s_cur = v;
        g_cur = g;
    }
    if (k1 == n) {
        __syncthreads();
        second(n - 1, (C)0);  // the first-sweep value on the boundary plane n is 0
    }
}

// Two plain 3-D damped-Jacobi sweeps with the planes staged by TMA (binary32 and bfloat16 storage,
// lattice form, one problem). A block owns XT_OUT output columns c0 .., RY output rows y0 .. and RZ
// output planes z0 .. and marches down z. Its shared memory holds three rings of planes, each 256
// columns from c0 - 8 wide: the input iterate (4 slots, rows y0 - 2 .. y0 + RY + 1), the source (3
// slots, rows y0 - 1 .. y0 + RY) and the first sweep (3 slots, rows y0 - 1 .. y0 + RY). Step zf
// (first-sweep plane, z0 - 1 .. z0 + RZ): thread 0 copies iterate plane zf + 2 and source plane
// zf + 1 by TMA (zero outside the lattice) for the next step; all threads wait (bounded) for this
// step's planes, run the first sweep at plane zf over RY + 2 rows into the first-sweep ring, pass a
// block barrier, run the second sweep at plane zf - 1 over the output rows to global memory, and
// pass another. Thread t owns Q adjacent columns from Q t and marches down its rows, keeping the
// y neighbours in registers. Per node: the sums (w + e), (s + n) along y, (b + t) along z, added in
// the single-sweep kernel's order, as packed binary32 pairs; bit-identical to two single sweeps.
// tests/test_tma3_ring_model.py replays the ring schedule on the CPU.
template <typename T> __device__ __forceinline__ void ldq(const T* p, float2* v, int np);
template <> __device__ __forceinline__ void ldq<float>(const float* p, float2* v, int np) {
    if (np == 1) v[0] = *reinterpret_cast<const float2*>(p);
    else {
        const float4 w = *reinterpret_cast<const float4*>(p);
        v[0] = make_float2(w.x, w.y);
        v[1] = make_float2(w.z, w.w);
    }
}
template <> __device__ __forceinline__ void ldq<__nv_bfloat16>(const __nv_bfloat16* p, float2* v, int np) {
    if (np == 1) v[0] = unpack_bf16x2(*reinterpret_cast<const unsigned*>(p));
    else ld4s(p, v[0], v[1]);
}
template <typename T> __device__ __forceinline__ void stq(T* p, const float2* v, int np);
template <> __device__ __forceinline__ void stq<float>(float* p, const float2* v, int np) {
    if (np == 1) *reinterpret_cast<float2*>(p) = v[0];
    else *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
}
template <> __device__ __forceinline__ void stq<__nv_bfloat16>(__nv_bfloat16* p, const float2* v, int np) {
    if (np == 1) *reinterpret_cast<unsigned*>(p) = pack_bf16x2_rn(v[0]);
    else *reinterpret_cast<uint2*>(p) = pack4(v[0], v[1]);
}
__device__ __forceinline__ void xt_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            (uint32_t)__cvta_generic_to_shared(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"((uint32_t)__cvta_generic_to_shared(bar))
        : "memory");
}
__device__ __forceinline__ void xt_arm(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar)),
                 "r"(bytes)
                 : "memory");
}

// One row of a thread's Q = 2 NP columns of a 3-D sweep from staged planes: c the row in its plane,
// y neighbours in vm / vp (registers), z neighbours at b / t, source at g.
template <typename T, int NP>
__device__ __forceinline__ void sweep3_row(const T* c, const float2* vm, const float2* vc, const float2* vp, const T* b,
                                           const T* t, const T* g, float2 om, float2 c1, float2* o) {
    constexpr int Q = 2 * NP;
    float2 vb[NP], vt[NP], gv[NP];
    ldq<T>(b, vb, NP);
    ldq<T>(t, vt, NP);
    ldq<T>(g, gv, NP);
    const float left = as_c<T>(c[-1]), right = as_c<T>(c[Q]);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float w0 = k == 0 ? left : vc[k - 1].y, e1 = k == NP - 1 ? right : vc[k + 1].x;
        const float2 we = make_float2(w0 + vc[k].y, vc[k].x + e1);                  // (w + e)
        const float2 sum = add2(add2(we, add2(vm[k], vp[k])), add2(vb[k], vt[k]));  // + (s + n), + (b + t)
        o[k] = fma2(c1, vc[k], fma2(om, sum, gv[k]));
    }
}

template <typename T, int RY, int RZ, int NP, int D>
__global__ void __launch_bounds__(XT_W / (2 * NP)) k_jacobi3_x2t(IterArgs a, const __grid_constant__ CUtensorMap me,
                                                                 const __grid_constant__ CUtensorMap mg, int* fault) {
    pdl_begin();
    constexpr int Q = 2 * NP, ER = RY + 4, GR = RY + 2;
    constexpr int EP = ER * XT_W, GP = GR * XT_W;  // elements of one staged plane
    constexpr int NE = D + 3, NG = D + 2, NB = D + 1;  // ring slots; per-step barriers (bar[NB]: set-up)
    extern __shared__ __align__(128) unsigned char x3_smem[];
    T* E = reinterpret_cast<T*>(x3_smem);  // iterate plane p in slot (p + 2) mod NE, rows y0 - 2 ..
    T* G = E + NE * EP;                    // source plane p in slot (p + 1) mod NG, rows y0 - 1 ..
    T* S = G + NG * GP;                    // first sweep at plane p in slot (p + 1) mod 3, rows y0 - 1 ..
    uint64_t* bar = reinterpret_cast<uint64_t*>(S + 3 * GP);
    const int t = threadIdx.x;
    const int n = a.e_new.n;
    const int c0 = blockIdx.x * XT_OUT, y0 = blockIdx.y * RY + 1, z0 = blockIdx.z * RZ + 1;
    const int zlast = min(z0 + RZ, n);  // last first-sweep plane (the plane past the block's last output)
    const int zout = min(z0 + RZ - 1, n - 1);
    auto eslot = [&](int p) { return E + ((p + 2) % NE) * EP; };
    auto gslot = [&](int p) { return G + ((p + 1) % NG) * GP; };
    auto sslot = [&](int p) { return S + ((p + 1) % 3) * GP; };
    // step s's planes (iterate s + 1, source s) on bar[s mod NB]; step z0 - 1's on bar[NB]
    auto load_step = [&](int st) {
        uint64_t* b = bar + st % NB;
        xt_arm(b, (uint32_t)((EP + GP) * sizeof(T)));
        xt_load_3d(eslot(st + 1), &me, c0 - 8, y0 - 2, st + 1, b);
        xt_load_3d(gslot(st), &mg, c0 - 8, y0 - 1, st, b);
    };
    if (t == 0) {
        for (int k = 0; k <= NB; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(bar + k)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t pend = 0;  // bit k: bar[k] has a phase armed and not yet waited for (same on every thread)
    if (t == 0) {
        xt_arm(bar + NB, (uint32_t)((3 * EP + GP) * sizeof(T)));
        for (int p = z0 - 2; p <= z0; ++p) xt_load_3d(eslot(p), &me, c0 - 8, y0 - 2, p, bar + NB);
        xt_load_3d(gslot(z0 - 1), &mg, c0 - 8, y0 - 1, z0 - 1, bar + NB);
    }
    pend |= 1u << NB;
    for (int st = z0; st <= min(z0 + D - 2, zlast); ++st) {
        if (t == 0) load_step(st);
        pend |= 1u << (st % NB);
    }
    const float2 om = make_float2(a.omega_f, a.omega_f), c1 = make_float2(a.c1_f, a.c1_f);
    const int x = c0 - 8 + Q * t;  // this thread's first column
    bool mcol[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) mcol[k] = x + k >= 1 && x + k <= n - 1;
    const bool first_cols = t >= 1 && t < XT_W / Q - 1;      // staged columns Q .. 255 - Q (7 .. 248 needed)
    const bool out_cols = t >= 8 / Q && t < (8 + XT_OUT) / Q;  // staged columns 8 .. 247
    uint32_t phases = 0;  // bit k: phase of bar[k] to wait for next
    for (int zf = z0 - 1; zf <= zlast; ++zf) {
        // (a) the planes of step zf + D, into slots the previous steps' barriers freed
        if (zf + D <= zlast) {
            if (t == 0) load_step(zf + D);
            pend |= 1u << ((zf + D) % NB);
        }
        // (b) this step's planes
        const int wb = zf == z0 - 1 ? NB : zf % NB;
        const bool arrived = xt_wait(bar + wb, (phases >> wb) & 1u);
        phases ^= 1u << wb;
        pend &= ~(1u << wb);
        if (!__syncthreads_and(arrived)) {
            // record the failure, give every copy still in flight one more bounded wait, and leave
            if (t == 0) atomicExch(fault, 1);
            phases ^= 1u << wb;
            pend |= 1u << wb;
            for (int k = 0; k <= NB; ++k)
                if (pend & (1u << k)) xt_wait(bar + k, (phases >> k) & 1u);
            return;
        }
        // (c) first sweep at plane zf, rows y0 - 1 .. y0 + RY (0 off the interior)
        if (first_cols) {
            const T* ec = eslot(zf) + Q * t;
            const T* eb = eslot(zf - 1) + Q * t;
            const T* et = eslot(zf + 1) + Q * t;
            const T* gp = gslot(zf) + Q * t;
            T* sp = sslot(zf) + Q * t;
            const bool pin = zf >= 1 && zf <= n - 1;
            float2 vm[NP], vc[NP], vp[NP];
            ldq<T>(ec, vm, NP);            // iterate row y0 - 2
            ldq<T>(ec + XT_W, vc, NP);     // iterate row y0 - 1
#pragma unroll 2
            for (int r = 0; r < GR; ++r) {  // first-sweep row y0 - 1 + r = staged iterate row r + 1
                const int q = r + 1;
                ldq<T>(ec + (q + 1) * XT_W, vp, NP);
                float2 o[NP];
                sweep3_row<T, NP>(ec + q * XT_W, vm, vc, vp, eb + q * XT_W, et + q * XT_W, gp + r * XT_W, om, c1, o);
                const int ra = y0 - 1 + r;
                const bool in = pin && ra >= 1 && ra <= n - 1;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    o[k].x = (in && mcol[2 * k]) ? o[k].x : 0.f;
                    o[k].y = (in && mcol[2 * k + 1]) ? o[k].y : 0.f;
                }
                stq<T>(sp + r * XT_W, o, NP);
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    vm[k] = vc[k];
                    vc[k] = vp[k];
                }
            }
        }
        __syncthreads();
        // (e) second sweep at plane zs = zf - 1, rows y0 .. y0 + RY - 1, to global memory
        const int zs = zf - 1;
        if (zs >= z0 && zs <= zout && out_cols) {
            const T* sc = sslot(zs) + Q * t;
            const T* sb = sslot(zs - 1) + Q * t;
            const T* st = sslot(zs + 1) + Q * t;
            const T* gp = gslot(zs) + Q * t;
            T* O = wp<T>(a.e_new) + ((int64_t)zs * (n + 1) + y0) * a.e_new.pitch + x;
            const int pe = min(RY, n - y0);
            const bool all = mcol[0] && mcol[Q - 1];
            float2 vm[NP], vc[NP], vp[NP];
            ldq<T>(sc, vm, NP);          // first-sweep row y0 - 1
            ldq<T>(sc + XT_W, vc, NP);   // first-sweep row y0
#pragma unroll 2
            for (int r = 1; r <= pe; ++r) {
                ldq<T>(sc + (r + 1) * XT_W, vp, NP);
                float2 o[NP];
                sweep3_row<T, NP>(sc + r * XT_W, vm, vc, vp, sb + r * XT_W, st + r * XT_W, gp + r * XT_W, om, c1, o);
                T* d = O + (int64_t)(r - 1) * a.e_new.pitch;
                if (all) stq<T>(d, o, NP);
                else {
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        if (mcol[2 * k]) d[2 * k] = St<T>::put(o[k].x);
                        if (mcol[2 * k + 1]) d[2 * k + 1] = St<T>::put(o[k].y);
                    }
                }
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    vm[k] = vc[k];
                    vc[k] = vp[k];
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Fast 3-D update + residual in two passes: k_update3 forms u_out = u_in + e (one FP64 add per
// node), then k_residual3_fast marches each (i, j) column along z over the updated iterate with the
// vertical neighbours in registers: 9 FP64 instructions per node, instead of re-forming u + e for
// every neighbour.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(J3X * J3Y) k_copy_in3(ResidArgs a, int n, int rows) {
    pdl_begin();
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (i >= n || j >= n) return;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    for (int k = k0; k < k1; ++k)
        a.u_out.p[at(a.u_out.pitch, n, i, j, k)] = a.st->u[at(n + 1, n, i, j, k)];
}

template <typename T>
__global__ void __launch_bounds__(J3X * J3Y) k_update3(ResidArgs a, int n, int rows) {
    pdl_begin();
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (i >= n || j >= n) return;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    for (int k = k0; k < k1; ++k) {
        const double v = __ldg(a.u_in.p + at(a.u_in.pitch, n, i, j, k)) +
                         to_d(St<T>::ld(cp<T>(a.e) + at(a.e.pitch, n, i, j, k)));
        a.u_out.p[at(a.u_out.pitch, n, i, j, k)] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(J3X * J3Y) k_residual3_fast(ResidArgs a, int n, int rows) {
    pdl_begin();
    __shared__ double sh[J3X * J3Y / 32];
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    const bool active = (i < n && j < n);
    const double* __restrict__ U = a.u_in.p ? a.u_in.p : a.st->u;
    const int64_t pu = a.u_in.p ? a.u_in.pitch : (int64_t)(n + 1);
    const int64_t plu = (int64_t)(n + 1) * pu;
    const double* __restrict__ F = a.st->f;
    const int64_t pf = n + 1, plf = (int64_t)(n + 1) * pf;
    double rr = 0.0, ff = 0.0;
    if (active) {
        // boundary nodes of the caller's u are not read: the operator takes 0 there
        auto uval = [&](int ii, int jj, int kk) -> double {
            if (ii <= 0 || jj <= 0 || kk <= 0 || ii >= n || jj >= n || kk >= n) return 0.0;
            return __ldg(U + (int64_t)kk * plu + (int64_t)jj * pu + ii);
        };
        double vb = uval(i, j, k0 - 1), vc = uval(i, j, k0);
        for (int k = k0; k < k1; ++k) {
            const double vt = uval(i, j, k + 1);
            const double sum = ((uval(i - 1, j, k) + uval(i + 1, j, k)) + (uval(i, j - 1, k) + uval(i, j + 1, k))) + (vb + vt);
            const double fv = __ldg(F + (int64_t)k * plf + (int64_t)j * pf + i);
            const double r = fma(a.inv_h2, fma(-6.0, vc, sum), fv);
            if (a.g0.p) wp<T>(a.g0)[at(a.g0.pitch, n, i, j, k)] = source_store<T>(r, a.scale, a.scale_f);
            rr = fma(r, r, rr);
            if (a.part_f) ff = fma(fv, fv, ff);
            vb = vc;
            vc = vt;
        }
    }
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    double t = block_sum(rr, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part_r[bid] = t;
    if (a.part_f) {
        t = block_sum(ff, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) a.part_f[bid] = t;
    }
}

// Fast lattice-form level change at stride 2 (3-D): a node with p odd indexes takes the mean of the
// 2^p surrounding values of Gc - dl; lattice nodes copy Gc.
template <typename T>
__global__ void __launch_bounds__(J3X * J3Y) k_prolong3_s1(ProlongArgs a, int rows) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.G.n;
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (i >= n || j >= n) return;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    const int I0 = i >> 1, J0 = j >> 1;
    const int ox = i & 1, oy = j & 1;
    const T* C0 = cp<T>(a.Gc);
    const T* D0 = cp<T>(a.dl);
    const int nc = a.Gc.n;
    for (int k = k0; k < k1; ++k) {
        const int K0 = k >> 1, oz = k & 1;
        C v;
        if (!(ox | oy | oz)) {
            v = St<T>::ld(C0 + at(a.Gc.pitch, nc, I0, J0, K0));
        } else {
            C acc = 0;
            for (int dz = 0; dz <= oz; ++dz)
                for (int dy = 0; dy <= oy; ++dy)
                    for (int dx = 0; dx <= ox; ++dx)
                        acc += St<T>::ld(C0 + at(a.Gc.pitch, nc, I0 + dx, J0 + dy, K0 + dz)) -
                               St<T>::ld(D0 + at(a.dl.pitch, a.dl.n, I0 + dx, J0 + dy, K0 + dz));
            v = acc * ((C)1 / (C)(1 << (ox + oy + oz)));
        }
        wp<T>(a.G)[at(a.G.pitch, n, i, j, k)] = St<T>::put(v);
    }
}

// Fast whole-grid iteration at level m >= 1 (2-D): every fine node adds the bilinear interpolant of
// the pending variation (level mp >= 1) unless it lies on the level-mp lattice, and level-m
// lattice nodes relax. Each thread marches one column down JR rows. The interpolant along x at a
// lattice row J, q(J), is formed once per coarse cell: moving down one cell the previous cell's
// upper value becomes the new lower one, so one new q and one difference per cell, and none of
// either in a column on the level-mp lattice (q is then the lattice value itself). A node at
// offset b inside its cell adds q0 + (b 2^-mp)(q1 - q0), the weight assembled from integer bits,
// the addition written as a fused multiply-add by a run-time 1 (the FP64 pipe issues those faster):
// two FMAs per node (one on a lattice row), no conversion on the FP64 pipe.
//
// Columns are dealt to the block's threads by residue class: with L = 2^min(m, 2), the first JX/L
// threads take the columns on the level-min(m, 2) lattice, the next JX/L the next class, and so on,
// so that whether a column relaxes (and, for mp <= 2, whether it lies on the pending lattice) is
// the same for every lane of a warp. Otherwise every warp would issue the relaxation's FP64
// instructions on every lattice row for its few lattice lanes, and GB300's FP64 pipe takes a warp
// instruction's full time whatever the number of active lanes.
template <bool PEND, typename T>
__global__ void __launch_bounds__(JX) k_wholegrid2(IterArgs a) {
    pdl_begin();
    using C = typename St<T>::C;
    const int n = a.e_new.n;
    // (FP64 only: the binary32 arithmetic kernels are memory bound and keep contiguous lanes)
    const int Lp = std::is_same<T, double>::value ? (a.m >= 2 ? 4 : 2) : 1, per = JX / Lp;  // m >= 1 here
    const int cls = threadIdx.x / per;
    const int off = (threadIdx.x % per) * Lp + ((Lp - 1 - cls) & (Lp - 1));
    const int i = blockIdx.x * JX + off + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * JR + 1;
    const int j1 = min(j0 + JR, n);
    const T* __restrict__ E = cp<T>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    T* __restrict__ O = wp<T>(a.e_new);
    const int64_t po = a.e_new.pitch;
    const int m = a.m, l = 1 << m, lm = l - 1;
    const C om = pick<C>(a.omega, a.omega_f);
    const C one = (C)a.one;
    const bool col_on_lattice = (i & lm) == 0;
    const int mp = PEND ? a.mp : 0;
    const int lpm = (1 << mp) - 1;
    const int I0 = i >> mp;
    const C alpha = PEND ? dyadic<C>(i & lpm, mp) : (C)0;
    const T* __restrict__ D = cp<T>(a.dprev);
    const int64_t pd = a.dprev.pitch;
    const bool col_on_prev = (i & lpm) == 0;
    // x-interpolant of the pending variation at lattice row J of this column
    auto qrow = [&](int J) -> C {
        const T* d = D + (int64_t)J * pd + I0;
        const C a0 = St<T>::ld(d);
        return col_on_prev ? a0 : fma(alpha, St<T>::ld(d + 1) - a0, a0);
    };
    int cell = -2;
    C r0 = 0, r1 = 0, dr = 0;
    for (int j = j0; j < j1; ++j) {
        C v = St<T>::ld(E + (int64_t)j * pe + i);
        if (col_on_lattice && (j & lm) == 0) {
            const C sum = (St<T>::ld(E + (int64_t)j * pe + i - l) + St<T>::ld(E + (int64_t)j * pe + i + l)) +
                          (St<T>::ld(E + (int64_t)(j - l) * pe + i) + St<T>::ld(E + (int64_t)(j + l) * pe + i));
            const C g = St<T>::ld(cp<T>(a.g) + (int64_t)(j >> m) * a.g.pitch + (i >> m));
            const C delta = fma(om, fma((C)-4, v, sum), g);
            if (a.dnew.p) wp<T>(a.dnew)[(int64_t)(j >> m) * a.dnew.pitch + (i >> m)] = St<T>::put(delta);
            v += delta;
        }
        if (PEND) {
            const int J0 = j >> mp;
            const int b = j & lpm;
            if (J0 != cell) {
                r0 = (J0 == cell + 1) ? r1 : qrow(J0);
                r1 = qrow(J0 + 1);
                dr = r1 - r0;
                cell = J0;
            }
            if (b == 0) {
                if (!col_on_prev) v = fma(one, v, r0);
            } else {
                v = fma(one, v, fma(dyadic<C>(b, mp), dr, r0));
            }
        }
        O[(int64_t)j * po + i] = St<T>::put(v);
    }
}

// Fast update + residual (2-D): each warp marches a strip of 32 columns along y; every lane forms
// u_new = u_in + e once per node of its column, the 30 inner lanes own their nodes and take the west
// and east neighbours' updated values by shuffle, the two edge lanes only supply theirs. Every
// instruction is issued once per warp and row for 30 nodes, none for an edge lane alone. The
// neighbour sum is formed from shared pairs (one addition per node for the pair, one to join two
// pairs, as in k_jacobi2d): 7 FP64 instructions per node in FP64 cycles, 6 in binary32 and bfloat16
// cycles (the source's multiply in binary32, source_store), one more for the norm of f on the
// initial residual. Widening e and rounding the source to the cycle's storage use the integer
// conversions above. Results are bit-identical to forming every pair locally.
constexpr int RS_OUT = 30;  // nodes per warp strip
template <typename T, bool VC, bool BATCH, bool P>
__device__ __forceinline__ void residual2_fast_body(ResidArgs a, int n, int bx, int by, int bz, int gx) {
    if (BATCH && !batch_view<T>(a, bz)) return;  // uniform over the block
    __shared__ double sh[JX / 32];
    const int lane = threadIdx.x & 31;
    const int strip = bx * (JX / 32) + (threadIdx.x >> 5);
    const int i = strip * RS_OUT + lane;  // this lane's column
    const bool col_in = i >= 1 && i <= n - 1;
    const bool active = col_in && lane >= 1 && lane <= RS_OUT;
    const int j0 = by * JR + 1;
    const int j1 = min(j0 + JR, n);
    const bool upd = a.e.p != nullptr;
    const double* __restrict__ U = a.u_in.p ? a.u_in.p : a.st->u;
    const int64_t pu = a.u_in.p ? a.u_in.pitch : (int64_t)(n + 1);
    const T* __restrict__ Ev = cp<T>(a.e);
    const int64_t pe = a.e.pitch;
    const double* __restrict__ F = a.st->f;
    const int64_t pf = n + 1;
    const bool want_f = a.part_f != nullptr;
    // Additions are written as fused multiply-adds by a run-time 1: the FP64 pipe, which bounds this
    // kernel, issues those faster than additions on GB300 (the results are the same roundings).
    const double one = a.one;
    auto un = [&](int jj) -> double {  // updated iterate at (i, jj); 0 on the boundary and outside
        if (!col_in || jj <= 0 || jj >= n) return 0.0;
        double v = ld64<P>(U + (int64_t)jj * pu + i);
        if (upd) v = fma(one, v, to_d(ldv<T, P>(Ev + (int64_t)jj * pe + i)));
        return v;
    };
    double rr = 0.0, ff = 0.0;
    double vs = un(j0 - 1), vc = un(j0);
    double ks = (VC && active) ? __ldg(a.ky + (int64_t)(j0 - 1) * a.kpitch + i) : 0.0;
    // Poisson: the neighbour pair D(i, j) = v(i+1, j) + v(i, j+1) of every lane, east + north here
    // and west + south of the node (i+1, j+1), taken from the left lane's previous row
    double dp = VC ? 0.0 : fma(one, __shfl_down_sync(0xffffffffu, vs, 1), vc);  // D(i, j0 - 1)
    for (int j = j0; j < j1; ++j) {
        const double vn = un(j + 1);
        const double e = __shfl_down_sync(0xffffffffu, vc, 1);
        const double w = VC ? __shfl_up_sync(0xffffffffu, vc, 1) : 0.0;
        double dh = 0.0, dw = 0.0;
        if constexpr (!VC) {
            dw = __shfl_up_sync(0xffffffffu, dp, 1);  // D(i-1, j-1)
            dh = fma(one, e, vn);                     // D(i, j)
            dp = dh;
        }
        if (active) {
            const double fv = __ldg(F + (int64_t)j * pf + i);
            double r;
            if constexpr (VC) {  // r = f - (D u - sum k_nb u_nb) / h^2, D = sum of the four face coefficients
                const double* kr = a.kx + (int64_t)j * a.kpitch + i;
                const double kw = __ldg(kr - 1), ke = __ldg(kr), kn = __ldg(a.ky + (int64_t)j * a.kpitch + i);
                double t = kw * w;
                t = fma(ke, e, t);
                t = fma(ks, vs, t);
                t = fma(kn, vn, t);
                const double d = fma(one, fma(one, fma(one, kw, ke), ks), kn);
                r = fma(-a.inv_h2, fma(d, vc, -t), fv);
                ks = kn;
            } else {
                r = fma(a.inv_h2, fma(-4.0, vc, fma(one, dh, dw)), fv);
            }
            if (a.u_out.p) a.u_out.p[(int64_t)j * a.u_out.pitch + i] = vc;
            if (a.g0.p) wp<T>(a.g0)[(int64_t)j * a.g0.pitch + i] = source_store<T>(r, a.scale, a.scale_f);
            rr = fma(r, r, rr);
            if (want_f) ff = fma(fv, fv, ff);
        }
        vs = vc;
        vc = vn;
    }
    const int bid = bx + gx * by;
    double t = block_sum(rr, sh);
    if (threadIdx.x == 0) a.part_r[bid] = t;
    if (a.part_f) {
        t = block_sum(ff, sh);
        if (threadIdx.x == 0) a.part_f[bid] = t;
    }
}

template <typename T, bool VC, bool BATCH>
__global__ void __launch_bounds__(JX) k_residual2_fast(ResidArgs a, int n) {
    pdl_begin();
    residual2_fast_body<T, VC, BATCH, false>(a, n, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x);
}

// =============================================================================================
// Power-of-two grids (Sec. 3), whole-grid form.
// =============================================================================================
// Local lattice index of fine index x along one axis for quadrant half qb at level m >= 1, or -1.
__device__ __forceinline__ int p2_local(int N, int m, int qb, int x) {
    const int d = qb ? (N - 1 - x) : x;
    if (d & ((1 << m) - 1)) return -1;
    const int a = d >> m;
    return a <= ((N >> 1) >> m) ? a : -1;
}

// Marked at level m >= 1 (an interior node of one quadrant's lattice): quadrant and local indexes.
// The halves' lattices are disjoint along each axis (N - 1 is odd), so at most one matches.
__device__ __forceinline__ bool p2_marked(int N, int m, int x, int y, int& q, int& a, int& b) {
    const int a0 = p2_local(N, m, 0, x), b0 = p2_local(N, m, 0, y);
    a = a0 >= 0 ? a0 : p2_local(N, m, 1, x);
    b = b0 >= 0 ? b0 : p2_local(N, m, 1, y);
    q = (a0 >= 0 ? 0 : 1) | ((b0 >= 0 ? 0 : 1) << 1);
    return a > 0 && b > 0;
}

// One whole-grid iteration: relax the nodes marked at level m (fast form v' = c1 v + omega sum + g,
// neighbours at distance 2^m, 0 outside the grid), store the variation in the quadrant's array, and
// add the bilinear interpolation of the pending level-mp variation from the node's own quadrant at
// the nodes not marked at level mp.
template <typename T>
__global__ void __launch_bounds__(P2X * P2Y) k_pow2_iterate(Pow2IterArgs a) {
    pdl_begin();
    using C = typename St<T>::C;
    const int N = a.N;
    // Columns by residue class (see k_wholegrid2): with L = min(2^max(m, mp), 4), the block's P2X
    // columns are dealt so that each warp holds one residue of x mod L, the lattice residue first:
    // 0 in the left half, L - 1 in the right half (its lattices are marked from x = N - 1). A block
    // lies in one half when N >= 2 P2X; whether a lane relaxes, or lies on the pending lattice, is
    // then the same for the whole warp on the level-min(m, 2) lattice.
    const int mm = a.m > a.mp ? a.m : a.mp;
    // (FP64 only: the binary32 arithmetic kernels are memory bound and keep contiguous lanes)
    const int L = std::is_same<T, double>::value ? (mm >= 2 ? 4 : 2) : 1, per = P2X / L;
    const int x0 = blockIdx.x * P2X;
    const int rlat = (x0 >= (N >> 1)) ? L - 1 : 0;
    const int u = threadIdx.x, cls = u / per;
    const int x = x0 + (u % per) * L + ((rlat + cls) & (L - 1));
    const int y = blockIdx.y * P2Y + threadIdx.y;
    if (x >= N || y >= N) return;
    T* O = wp<T>(a.e_new);
    const int64_t po = a.e_new.pitch;
    if (x == 0 || y == 0 || x == N - 1 || y == N - 1) {
        O[(int64_t)y * po + x] = St<T>::put((C)0);
        return;
    }
    const T* E = cp<T>(a.e_old);
    const int64_t pe = a.e_old.pitch;
    auto ev = [&](int xx, int yy) -> C {
        if (E == nullptr || xx < 0 || yy < 0 || xx >= N || yy >= N) return (C)0;
        return St<T>::ld(E + (int64_t)yy * pe + xx);
    };
    C v = ev(x, y);
    int q = 0, la = 0, lb = 0;
    if (a.m == 0 || p2_marked(N, a.m, x, y, q, la, lb)) {
        const int l = 1 << a.m;
        const C sum = (ev(x - l, y) + ev(x + l, y)) + (ev(x, y - l) + ev(x, y + l));
        const C g = (a.m == 0) ? St<T>::ld(cp<T>(a.g) + (int64_t)y * a.g.pitch + x)
                               : St<T>::ld(cp<T>(a.g) + (int64_t)q * a.g.bstride + (int64_t)lb * a.g.pitch + la);
        const C om = pick<C>(a.omega, a.omega_f), c1 = pick<C>(a.c1, a.c1_f);
        const C nv = fma(c1, v, fma(om, sum, g));
        if (a.dnew.p) wp<T>(a.dnew)[(int64_t)q * a.dnew.bstride + (int64_t)lb * a.dnew.pitch + la] = St<T>::put(nv - v);
        v = nv;
    }
    int q2, a2, b2;
    if (a.mp >= 1 && !p2_marked(N, a.mp, x, y, q2, a2, b2)) {
        // bilinear as two x-lerps and a y-lerp (7 FP instructions); the dyadic weights f 2^-mp are
        // built from integer bits, so no floating-point work goes into them
        const int H = N >> 1, qx = x >= H, qy = y >= H, lp = 1 << a.mp;
        const int dx = qx ? N - 1 - x : x, dy = qy ? N - 1 - y : y;
        const int A0 = dx >> a.mp, fa = dx & (lp - 1), B0 = dy >> a.mp, fb = dy & (lp - 1);
        const int A1 = fa ? A0 + 1 : A0, B1 = fb ? B0 + 1 : B0;
        const T* D = cp<T>(a.dprev) + (int64_t)(qx | (qy << 1)) * a.dprev.bstride;
        const int64_t pd = a.dprev.pitch;
        const C wx = dyadic<C>(fa, a.mp), wy = dyadic<C>(fb, a.mp);
        const C d00 = St<T>::ld(D + (int64_t)B0 * pd + A0), d10 = St<T>::ld(D + (int64_t)B0 * pd + A1);
        const C d01 = St<T>::ld(D + (int64_t)B1 * pd + A0), d11 = St<T>::ld(D + (int64_t)B1 * pd + A1);
        const C r0 = fma(wx, d10 - d00, d00), r1 = fma(wx, d11 - d01, d01);
        v += fma(wy, r1 - r0, r0);
    }
    O[(int64_t)y * po + x] = St<T>::put(v);
}

// Hat-weighted sum sum_{|d| < l} (l - |d|)/l * f(d) over one stencil line: by one thread (short
// lines) or by a warp (long lines, lanes striding, shuffle reduction).
template <bool WARP, typename F>
__device__ __forceinline__ double hat_sum(int l, F f) {
    double acc = 0.0;
    const double inv = 1.0 / (double)l;  // exact: l is a power of two
    if constexpr (!WARP) {
        for (int d = -(l - 1); d <= l - 1; ++d) acc = fma((double)(l - abs(d)) * inv, f(d), acc);
    } else {
        for (int d = -(l - 1) + (int)(threadIdx.x & 31); d <= l - 1; d += 32) acc = fma((double)(l - abs(d)) * inv, f(d), acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    return acc;
}

// Row pass: tmp[(y*2 + qx)*(n_m+1) + a] = hat sum of g0 along row y around x(qx, a).
template <typename T, bool WARP>
__global__ void k_pow2_rows(Pow2RestrictArgs r) {
    pdl_begin();
    const int N = r.N, m = r.m, l = 1 << m, nm = (N >> 1) >> m;
    const int64_t outs = (int64_t)N * 2 * (nm + 1);
    const int64_t id = WARP ? ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= outs) return;
    const int a = (int)(id % (nm + 1)), qx = (int)((id / (nm + 1)) % 2), y = (int)(id / (2 * (nm + 1)));
    const int x = qx ? N - 1 - a * l : a * l;
    const T* G = cp<T>(r.g0) + (int64_t)y * r.g0.pitch;
    const double s = hat_sum<WARP>(l, [&](int d) -> double {
        const int xx = x + d;
        return (xx < 0 || xx >= N) ? 0.0 : (double)St<T>::ld(G + xx);
    });
    if (!WARP || (threadIdx.x & 31) == 0) r.tmp[id] = s;
}

// Column pass: gm[q][b][a] = hat sum of tmp down column (qx, a) around y(qy, b); 0 on the domain
// boundary (a == 0 or b == 0).
template <typename T, bool WARP>
__global__ void k_pow2_cols(Pow2RestrictArgs r) {
    pdl_begin();
    const int N = r.N, m = r.m, l = 1 << m, nm = (N >> 1) >> m;
    const int64_t outs = (int64_t)4 * (nm + 1) * (nm + 1);
    const int64_t id = WARP ? ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= outs) return;
    const int a = (int)(id % (nm + 1)), b = (int)((id / (nm + 1)) % (nm + 1)), q = (int)(id / ((int64_t)(nm + 1) * (nm + 1)));
    const int qx = q & 1, qy = q >> 1;
    const int y = qy ? N - 1 - b * l : b * l;
    double s = 0.0;
    if (a > 0 && b > 0)
        s = hat_sum<WARP>(l, [&](int d) -> double {
            const int yy = y + d;
            return (yy < 0 || yy >= N) ? 0.0 : r.tmp[((int64_t)yy * 2 + qx) * (nm + 1) + a];
        });
    // times 4^m = l^2 keeps the source pre-scaled by h_m^2: each pass carries a factor l
    if (!WARP || (threadIdx.x & 31) == 0)
        wp<T>(r.gm)[(int64_t)q * r.gm.bstride + (int64_t)b * r.gm.pitch + a] = St<T>::put(St<T>::from_d(s));
}

// Nodes per thread along the march: long columns on large launches (fewer blocks, more reuse),
// short ones on small launches, where a thread's serial chain of loads would otherwise set the
// time. `nb` problems of a batch share the launch.
int march_rows(int ndim, int n, int nb = 1) {
    const double nodes = (double)nb * ((ndim == 2) ? (double)(n - 1) * (n - 1) : (double)(n - 1) * (n - 1) * (n - 1));
    if (nodes >= 8.0e6) return 16;
    if (nodes >= 1.0e6) return 4;
    return 1;
}

dim3 grid_for(int ndim, int n) {
    return dim3((unsigned)((n - 1 + BX - 1) / BX), (unsigned)((n - 1 + BY - 1) / BY), ndim == 3 ? (unsigned)(n - 1) : 1u);
}

// The fast residual kernels use their own grids: 2-D (n-1)/(30 * JX/32) x (n-1)/JR blocks, 3-D
// (n-1)/J3X x (n-1)/J3Y x (n-1)/rows.
dim3 resid_grid(int ndim, bool strict, int n) {
    if (ndim == 2 && !strict)
        return dim3((unsigned)((((n - 1 + RS_OUT - 1) / RS_OUT) + JX / 32 - 1) / (JX / 32)), (unsigned)((n - 1 + JR - 1) / JR));
    if (ndim == 3 && !strict) {
        const int rows = march_rows(3, n);
        return dim3((unsigned)((n - 1 + J3X - 1) / J3X), (unsigned)((n - 1 + J3Y - 1) / J3Y), (unsigned)((n - 1 + rows - 1) / rows));
    }
    return grid_for(ndim, n);
}

// ---- launch templates ----------------------------------------------------------------------
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 g, dim3 b, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g;
    cfg.blockDim = b;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename T>
cudaError_t iterate_t(int ndim, bool strict, const IterArgs& a, cudaStream_t s) {
    const int n = a.e_new.n;
    if (a.kx != nullptr) {  // variable coefficients: 2-D fast lattice form only (checked by the host)
        const bool wd = a.dnew.p != nullptr;
        const int rows = a.rows > 0 ? a.rows : march_rows(2, n, a.nb);
        const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows)), b(JX);
        const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
#define JVC(P, W) launch_k(k_jacobi2_vc<P, W, T>, g, b, s, a, rows)
        if (pend == 0) { if (wd) JVC(0, true); else JVC(0, false); }
        else if (pend == 1) { if (wd) JVC(1, true); else JVC(1, false); }
        else { if (wd) JVC(2, true); else JVC(2, false); }
#undef JVC
        return cudaGetLastError();
    }
    if (!strict && a.m == 0 && a.e_old.p != nullptr) {
        const bool wd = a.dnew.p != nullptr;
        const int rows = a.rows > 0 ? a.rows : march_rows(ndim, n, a.nb);
        if (ndim == 2 && std::is_same<T, double>::value && !a.bst && n >= JD2_MIN_N) {
            constexpr int per_block = JX / 32 * JD2_COLS;
            const dim3 g((unsigned)((n - 1 + per_block - 1) / per_block), (unsigned)((n - 1 + rows - 1) / rows)), b(JX);
            const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
#define JAC2D(P, W) launch_k(k_jacobi2d2<P, W>, g, b, s, a, rows)
            if (pend == 0) { if (wd) JAC2D(0, true); else JAC2D(0, false); }
            else if (pend == 1) { if (wd) JAC2D(1, true); else JAC2D(1, false); }
            else { if (wd) JAC2D(2, true); else JAC2D(2, false); }
#undef JAC2D
        } else if (ndim == 2 && std::is_same<T, double>::value && !a.bst) {
            constexpr int per_block = JX / 32 * JD_COLS;
            const dim3 g((unsigned)((n - 1 + per_block - 1) / per_block), (unsigned)((n - 1 + rows - 1) / rows)), b(JX);
            const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
#define JAC2D(P, W) launch_k(k_jacobi2d<P, W>, g, b, s, a, rows)
            if (pend == 0) { if (wd) JAC2D(0, true); else JAC2D(0, false); }
            else if (pend == 1) { if (wd) JAC2D(1, true); else JAC2D(1, false); }
            else { if (wd) JAC2D(2, true); else JAC2D(2, false); }
#undef JAC2D
        } else if (ndim == 2) {
            const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows), (unsigned)a.nb), b(JX);
            const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
#define JAC2(P, W) (a.bst ? launch_k(k_jacobi2<P, W, T, true>, g, b, s, a, rows) : launch_k(k_jacobi2<P, W, T, false>, g, b, s, a, rows))
            if (pend == 0) { if (wd) JAC2(0, true); else JAC2(0, false); }
            else if (pend == 1) { if (wd) JAC2(1, true); else JAC2(1, false); }
            else { if (wd) JAC2(2, true); else JAC2(2, false); }
#undef JAC2
        } else if (std::is_same<T, double>::value) {
            const bool pend = a.mp >= 0;
            const dim3 g((unsigned)((n - 1 + JD_COLS - 1) / JD_COLS), (unsigned)((n - 1 + J3Y - 1) / J3Y),
                         (unsigned)((n - 1 + rows - 1) / rows)),
                b(J3X, J3Y);
            if (pend && wd) launch_k(k_jacobi3d<true, true>, g, b, s, a, rows);
            else if (pend) launch_k(k_jacobi3d<true, false>, g, b, s, a, rows);
            else if (wd) launch_k(k_jacobi3d<false, true>, g, b, s, a, rows);
            else launch_k(k_jacobi3d<false, false>, g, b, s, a, rows);
        } else {
            const bool pend = a.mp >= 0;
            const dim3 g((unsigned)((n - 1 + J3X - 1) / J3X), (unsigned)((n - 1 + J3Y - 1) / J3Y),
                         (unsigned)((n - 1 + rows - 1) / rows)),
                b(J3X, J3Y);
            if (pend && wd) launch_k(k_jacobi3<true, true, T>, g, b, s, a, rows);
            else if (pend) launch_k(k_jacobi3<true, false, T>, g, b, s, a, rows);
            else if (wd) launch_k(k_jacobi3<false, true, T>, g, b, s, a, rows);
            else launch_k(k_jacobi3<false, false, T>, g, b, s, a, rows);
        }
        return cudaGetLastError();
    }
    if (!strict && ndim == 2 && a.m >= 1 && a.e_old.p != nullptr && a.mp != 0) {
        const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + JR - 1) / JR)), b(JX);
        if (a.mp >= 1) launch_k(k_wholegrid2<true, T>, g, b, s, a);
        else launch_k(k_wholegrid2<false, T>, g, b, s, a);
        return cudaGetLastError();
    }
    dim3 g = grid_for(ndim, n);
    const dim3 b(BX, BY);
    if (ndim == 2) g.z = (unsigned)a.nb;
    if (ndim == 2) {
        if (strict) launch_k(k_iterate<2, true, T>, g, b, s, a);
        else launch_k(k_iterate<2, false, T>, g, b, s, a);
    } else {
        if (strict) launch_k(k_iterate<3, true, T>, g, b, s, a);
        else launch_k(k_iterate<3, false, T>, g, b, s, a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t prolong_t(int ndim, bool strict, const ProlongArgs& a, cudaStream_t s) {
    if (!strict && ndim == 2 && a.s == 1) {
        const int n = a.G.n;
        const int rows = march_rows(2, n, a.nb);
        const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows), (unsigned)a.nb);
        if (a.bst) launch_k(k_prolong2_s1<T, true>, g, dim3(JX), s, a, rows);
        else launch_k(k_prolong2_s1<T, false>, g, dim3(JX), s, a, rows);
        return cudaGetLastError();
    }
    if (!strict && ndim == 3 && a.s == 1) {
        const int n = a.G.n;
        const int rows = march_rows(3, n);
        const dim3 g((unsigned)((n - 1 + J3X - 1) / J3X), (unsigned)((n - 1 + J3Y - 1) / J3Y), (unsigned)((n - 1 + rows - 1) / rows));
        launch_k(k_prolong3_s1<T>, g, dim3(J3X, J3Y), s, a, rows);
        return cudaGetLastError();
    }
    dim3 g = grid_for(ndim, a.G.n);
    const dim3 b(BX, BY);
    if (ndim == 2) g.z = (unsigned)a.nb;
    if (ndim == 2) {
        if (strict) launch_k(k_prolong<2, true, T>, g, b, s, a);
        else launch_k(k_prolong<2, false, T>, g, b, s, a);
    } else {
        if (strict) launch_k(k_prolong<3, true, T>, g, b, s, a);
        else launch_k(k_prolong<3, false, T>, g, b, s, a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t residual_t(int ndim, bool strict, const ResidArgs& a, int n, cudaStream_t s) {
    dim3 g = resid_grid(ndim, strict, n);
    if (ndim == 2) g.z = (unsigned)a.nb;
    if (ndim == 2) {
        if (strict) launch_k(k_residual<2, true, T>, g, dim3(BX, BY), s, a, n);
        else if (a.batch) launch_k(k_residual2_fast<T, false, true>, g, dim3(JX), s, a, n);
        else if (a.kx) launch_k(k_residual2_fast<T, true, false>, g, dim3(JX), s, a, n);
        else launch_k(k_residual2_fast<T, false, false>, g, dim3(JX), s, a, n);
    } else if (strict) {
        launch_k(k_residual<3, true, T>, g, dim3(BX, BY), s, a, n);
    } else {
        const int rows = march_rows(3, n);
        ResidArgs b = a;
        if (a.e.p) {  // update pass first; the residual then reads the updated iterate
            launch_k(k_update3<T>, g, dim3(J3X, J3Y), s, a, n, rows);
            b.u_in = CDGrid{a.u_out.p, a.u_out.pitch, a.u_out.n};
            b.e = CGrid{nullptr, 0, n};
        } else if (a.u_out.p) {  // initial residual: copy the caller's u in, then read the copy
            ResidArgs c = a;
            launch_k(k_copy_in3, g, dim3(J3X, J3Y), s, c, n, rows);
            b.u_in = CDGrid{a.u_out.p, a.u_out.pitch, a.u_out.n};
        }
        launch_k(k_residual3_fast<T>, g, dim3(J3X, J3Y), s, b, n, rows);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t restrict_t(int ndim, bool strict, const RestrictArgs& a, cudaStream_t s) {
    dim3 g = grid_for(ndim, a.gc.n);
    const dim3 b(BX, BY);
    if (ndim == 2) g.z = (unsigned)a.nb;
    if (ndim == 2) {
        if (strict) launch_k(k_restrict<2, true, T>, g, b, s, a);
        else launch_k(k_restrict<2, false, T>, g, b, s, a);
    } else {
        if (strict) launch_k(k_restrict<3, true, T>, g, b, s, a);
        else launch_k(k_restrict<3, false, T>, g, b, s, a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Persistent batch kernel (see PersistArgs): one cooperative launch runs every size group's cycles.
// ---------------------------------------------------------------------------------------------

// Grid barrier with a bounded wait. Thread 0 of each block arrives (release fence, then the arrival
// counter); the last block to arrive resets the counter and advances the generation; the others poll
// the generation until it moves, another block has given up, or timeout_ns has passed, and then
// fence (acquire) so that the next phase sees every block's writes of this one. On timeout the
// block records the failure in *err; false tells the caller to leave the kernel. Every wait is
// bounded, so the launch ends whatever another block does.
__device__ bool grid_barrier(const PersistArgs& P, unsigned int target) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = P.sync + 1;
        const unsigned int g = *gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(P.sync, 1u) + 1u;
        int ok = 1;
        if (arrived == target) {
            atomicExch(P.sync, 0u);
            __threadfence();
            atomicAdd(P.sync + 1, 1u);
        } else {
            const long long t0 = device_clock_ns();
            while (*gen == g) {
                if (*(volatile int*)P.err) { ok = 0; break; }
                if (device_clock_ns() - t0 > P.timeout_ns) { atomicExch(P.err, 1); ok = 0; break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// Convergence test of problem z of a group (the batch finalize's per-problem part); counts the
// problems still running into *running.
__device__ void finalize_problem(const FinalizeArgs& a, int z, unsigned int* running) {
    __shared__ double sh[JX / 32];
    State* st = a.st + z;
    double* hist = a.hist + (int64_t)z * a.hist_bstride;
    const double* pr = a.part_r + (int64_t)z * a.part_bstride;
    const double* pf = a.part_f ? a.part_f + (int64_t)z * a.part_bstride : nullptr;
    const bool skip = a.mode == FIN_CYCLE && st->done;
    if (!skip) {
        double sr = 0.0, sf = 0.0;
        for (int t = threadIdx.x; t < a.nparts; t += blockDim.x) {
            sr += pr[t];
            if (pf) sf += pf[t];
        }
        sr = block_sum(sr, sh);
        if (pf) sf = block_sum(sf, sh);
        if (threadIdx.x == 0) finalize_decide(a, st, hist, sr, sf);
    }
    if (threadIdx.x == 0 && !st->done) atomicAdd(running, 1u);
}

// One block of one op: block r of the op's gx x gy x gz blocks. The marching ops run their own
// kernels' bodies; the tiled ops (BX x BY nodes) take two passes of the JX threads.
template <typename T>
__device__ void run_item(const PersistItem& I, int r, unsigned int* running) {
    const int bx = r % I.gx, by = (r / I.gx) % I.gy, bz = r / (I.gx * I.gy);
    constexpr bool B32 = !std::is_same<T, double>::value;  // fused sweeps: binary32 cycles only
    switch (I.kind) {
        case PK_ITER:
            switch (I.sub) {
                case 0: jacobi2_body<0, false, T, true, true>(I.it, I.rows, bx, by, bz); break;
                case 1: jacobi2_body<0, true, T, true, true>(I.it, I.rows, bx, by, bz); break;
                case 2: jacobi2_body<1, false, T, true, true>(I.it, I.rows, bx, by, bz); break;
                case 3: jacobi2_body<1, true, T, true, true>(I.it, I.rows, bx, by, bz); break;
                case 4: jacobi2_body<2, false, T, true, true>(I.it, I.rows, bx, by, bz); break;
                default: jacobi2_body<2, true, T, true, true>(I.it, I.rows, bx, by, bz); break;
            }
            break;
        case PK_ITER2:
            if constexpr (B32) jacobi2_x2_body<T, true, true>(I.it, I.rows, bx, by, bz);
            break;
        case PK_ITER4:
            if constexpr (B32) jacobi2_xk_body<T, true, 4, true>(I.it, I.rows, bx, by, bz);
            break;
        case PK_PROLONG2: prolong2_s1_body<T, true, true>(I.pr, I.rows, bx, by, bz); break;
        case PK_BLOCK: coarse_block_body<2, T>(I.ops, I.nops, bz); break;
        case PK_RESID: residual2_fast_body<T, false, true, true>(I.ra, I.n, bx, by, bz, I.gx); break;
        case PK_FINAL: finalize_problem(I.fa, bz, running); break;
        default: {  // tiled ops
            IterArgs it = I.it;
            ProlongArgs pr = I.pr;
            RestrictArgs rs = I.rs;
            bool live = true;
            int side = 0;
            if (I.kind == PK_ITERG) { live = batch_view<T>(it, bz); side = it.e_new.n; }
            else if (I.kind == PK_PROLONG) { live = batch_view<T>(pr, bz); side = pr.G.n; }
            else if (I.kind == PK_RESTRICT) { live = batch_view<T>(rs, bz); side = rs.gc.n; }
            else side = I.n;
            if (!live) break;
            for (int pass = 0; pass < BY * BX / JX; ++pass) {
                const int i = bx * BX + (threadIdx.x & (BX - 1)) + 1;
                const int j = by * BY + (threadIdx.x / BX) + pass * (JX / BX) + 1;
                if (i >= side || j >= side) continue;
                if (I.kind == PK_ITERG) iterate_point<2, false, T>(it, i, j, 0);
                else if (I.kind == PK_PROLONG) prolong_point<2, false, T>(pr, i, j, 0);
                else if (I.kind == PK_RESTRICT) restrict_point<2, false, T>(rs, i, j, 0);
                else {  // PK_COPY (see k_copy_out)
                    const State* st = I.co.st;
                    CDGrid u0 = I.co.u0, u1 = I.co.u1;
                    if (I.co.batch) {
                        st += bz;
                        shift(u0, bz);
                        shift(u1, bz);
                    }
                    double v = 0.0;
                    if (!st->zero_u) {
                        const CDGrid src = (st->cycle & 1) ? u1 : u0;
                        v = src.p[at(src.pitch, side, i, j, 0)];
                    }
                    st->u[at(side + 1, side, i, j, 0)] = v;
                }
            }
        }
    }
}

// The work queue of one phase: blocks draw item blocks from the phase's counter until none is left.
template <typename T>
__device__ void run_phase(const PersistArgs& P, const PersistPhase& ph, unsigned int* counter, unsigned int* running) {
    __shared__ int t_sh;
    for (;;) {
        if (threadIdx.x == 0) t_sh = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int t = t_sh;
        __syncthreads();
        if (t >= ph.blocks) return;
        int r = t, q = ph.first;
        for (;; ++q) {
            const int nb = P.items[q].gx * P.items[q].gy * P.items[q].gz;
            if (r < nb) break;
            r -= nb;
        }
        run_item<T>(P.items[q], r, running);
        __syncthreads();  // the bodies' shared memory is reused by the next item
    }
}

// Runs `count` phases from `first`; false when a grid barrier gave up.
template <typename T>
__device__ bool run_segment(const PersistArgs& P, int first, int count, unsigned int& gp, unsigned int target,
                            unsigned int* running) {
    for (int q = 0; q < count; ++q) {
        run_phase<T>(P, P.phases[first + q], P.queue + gp++, running);
        if (!grid_barrier(P, target)) return false;
    }
    return true;
}

template <typename T>
// 10 blocks of JX threads per SM: the union of the bodies then spills to local memory, which
// measured faster than fewer resident blocks without spills (253 ms for the 1024-problem batch
// against 437 ms at 4 blocks and 317 ms at 6).
__global__ void __launch_bounds__(JX, 10) k_batch_persistent(PersistArgs P) {
    const unsigned int target = gridDim.x + (P.stall ? 1u : 0u);
    if (P.stall) {  // self-test: a barrier that cannot complete, before any problem data is touched
        grid_barrier(P, target);
        return;
    }
    unsigned int gp = 0;
    unsigned int* cnt = P.sync + 2;  // running problems after the test of cycle k: cnt[k % 3]
    if (!run_segment<T>(P, P.init_first, P.init_count, gp, target, cnt)) return;
    if (*(volatile unsigned int*)cnt == 0u) P.max_cycles = 0;  // nothing to solve
    for (int k = 1; k <= P.max_cycles; ++k) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(k + 1) % 3] = 0u;  // counter of cycle k + 1
        if (!run_segment<T>(P, P.cyc_first[k & 1], P.cyc_count, gp, target, cnt + k % 3)) return;
        if (*(volatile unsigned int*)(cnt + k % 3) == 0u) break;
    }
    run_segment<T>(P, P.copy_first, P.copy_count, gp, target, cnt);
}

}  // namespace

#define DISPATCH_PREC(prec, CALL)                                    \
    switch (prec) {                                                  \
        case PREC_FP64: { using T = double; return CALL; }           \
        case PREC_FP32: { using T = float; return CALL; }            \
        case PREC_BF16: { using T = __nv_bfloat16; return CALL; }    \
        default: return cudaErrorInvalidValue;                       \
    }

cudaError_t launch_iterate(int ndim, int prec, bool strict, const IterArgs& a, cudaStream_t s) {
    DISPATCH_PREC(prec, iterate_t<T>(ndim, strict, a, s));
}

template <typename T, int K> cudaError_t iterate_k_t(const IterArgs& a, cudaStream_t s) {
    const int n = a.e_new.n;
    constexpr int OUTK = 34 - 2 * K;
    const int xb = (((n - 1 + OUTK - 1) / OUTK) + JX / 32 - 1) / (JX / 32);
    const double nodes = (double)a.nb * (double)(n - 1) * (double)(n - 1);
    const int rows = a.rows > 0 ? a.rows : (nodes >= 1.0e6 ? 32 : 8);
    const dim3 g((unsigned)xb, (unsigned)((n - 1 + rows - 1) / rows), (unsigned)a.nb), b(JX);
    return a.bst ? launch_k(k_jacobi2_xk<T, true, K>, g, b, s, a, rows) : launch_k(k_jacobi2_xk<T, false, K>, g, b, s, a, rows);
}

cudaError_t launch_iterate3_2(int prec, const IterArgs& a, cudaStream_t s) {
    const int n = a.e_new.n;
    const double nodes = (double)(n - 1) * (double)(n - 1) * (double)(n - 1);
    const int rows = a.rows > 0 ? a.rows : (nodes >= 8.0e6 ? 32 : 8);
    const dim3 g((unsigned)((n - 1 + J3X - 3) / (J3X - 2)), (unsigned)((n - 1 + J3Y2 - 3) / (J3Y2 - 2)),
                 (unsigned)((n - 1 + rows - 1) / rows)),
        b(J3X, J3Y2);
    switch (prec) {
        case PREC_FP32: return launch_k(k_jacobi3_x2<float>, g, b, s, a, rows);
        case PREC_BF16: return launch_k(k_jacobi3_x2<__nv_bfloat16>, g, b, s, a, rows);
        default: return cudaErrorInvalidValue;
    }
}

// The packed pair kernel's layout conditions: every row holds the padding column n + 1, and every
// pair load (even column, every problem of a batch) is aligned to two elements.
bool pairs_ok(int prec, const IterArgs& a) {
    if (prec != PREC_FP32 && prec != PREC_BF16) return false;
    const size_t es = (prec == PREC_FP32) ? sizeof(float) : sizeof(__nv_bfloat16);
    const int n = a.e_new.n;
    auto fits = [&](const void* p, int64_t pitch, int64_t bstride) {
        return p != nullptr && pitch >= (int64_t)n + 2 && pitch % 2 == 0 && bstride % 2 == 0 &&
               reinterpret_cast<uintptr_t>(p) % (2 * es) == 0;
    };
    return fits(a.e_old.p, a.e_old.pitch, a.e_old.bstride) && fits(a.g.p, a.g.pitch, a.g.bstride) &&
           fits(a.e_new.p, a.e_new.pitch, a.e_new.bstride);
}

cudaError_t launch_iterate2(int prec, int sweeps, const IterArgs& a, cudaStream_t s) {
    if (sweeps == 4) {
        if (prec == PREC_FP32) return iterate_k_t<float, 4>(a, s);
        if (prec == PREC_BF16) return iterate_k_t<__nv_bfloat16, 4>(a, s);
        return cudaErrorInvalidValue;
    }
    if (sweeps != 2) return cudaErrorInvalidValue;
    const int n = a.e_new.n;
    // each warp also computes the first sweep one row above and one below its own rows: march
    // further than a single sweep does, to keep that overhead small
    const double nodes = (double)a.nb * (double)(n - 1) * (double)(n - 1);
    const int rows = a.rows > 0 ? a.rows : (nodes >= 1.0e6 ? 16 : 8);
    const dim3 b(JX);
    if (prec == PREC_BF16 && n >= X2P_MIN_N && pairs_ok(prec, a)) {
        const int xp = (((n + X2P_OUT - 1) / X2P_OUT) + JX / 32 - 1) / (JX / 32);  // strips cover columns 0 .. n - 1
        const dim3 g((unsigned)xp, (unsigned)((n - 1 + rows - 1) / rows), (unsigned)a.nb);
        return a.bst ? launch_k(k_jacobi2_x2p<__nv_bfloat16, true>, g, b, s, a, rows)
                     : launch_k(k_jacobi2_x2p<__nv_bfloat16, false>, g, b, s, a, rows);
    }
    const int xb = (((n - 1 + X2_OUT - 1) / X2_OUT) + JX / 32 - 1) / (JX / 32);  // blocks across: JX / 32 strips each
    const dim3 g((unsigned)xb, (unsigned)((n - 1 + rows - 1) / rows), (unsigned)a.nb);
    switch (prec) {
        case PREC_FP32:
            return a.bst ? launch_k(k_jacobi2_x2<float, true>, g, b, s, a, rows) : launch_k(k_jacobi2_x2<float, false>, g, b, s, a, rows);
        case PREC_BF16:
            return a.bst ? launch_k(k_jacobi2_x2<__nv_bfloat16, true>, g, b, s, a, rows)
                         : launch_k(k_jacobi2_x2<__nv_bfloat16, false>, g, b, s, a, rows);
        default: return cudaErrorInvalidValue;  // FP64 sweeps are FP64-bound: never paired
    }
}

// TMA two-sweep kernel: RT output rows per block. Measured at 4097² (graph solves, RT from 4 to 32):
// short tiles win, many small blocks per SM overlapping each other's copy with their sweeps;
// bfloat16 8 rows (16 KB of shared memory; four columns per thread: 20.9 us per level-0 pair, 23.0
// at 4 rows, 21.4 at 12), binary32 6 rows (26 KB; 36.8 us, 38.4 at 4 and 8 rows, 45.0 at 32).
template <typename T> constexpr int xt_rows() { return sizeof(T) == 2 ? 8 : 6; }
// Columns per thread: four for bfloat16 (fewer instructions per node), two for binary32.
template <typename T> constexpr int xt_cols() { return sizeof(T) == 2 ? 4 : 2; }
template <typename T> constexpr size_t xt_smem_bytes() {
    return (size_t)((xt_rows<T>() + 4) + 2 * (xt_rows<T>() + 2)) * XT_W * sizeof(T) + 16;
}

// cuTensorMapEncodeTiled, obtained once through the runtime's driver entry-point query.
PFN_cuTensorMapEncodeTiled_v12000 xt_encoder() {
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

// A lattice array of (n + 1) x (n + 1) nodes, rows of `pitch` elements, as a 2-D tensor whose box
// is XT_W columns x `rows` rows; zero outside the lattice.
template <typename T>
cudaError_t xt_map(CUtensorMap* map, const void* base, int n, int64_t pitch, int rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = xt_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)(n + 1), (cuuint64_t)(n + 1)};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(T)};
    const cuuint32_t box[2] = {(cuuint32_t)XT_W, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T> cudaError_t tma_sweep_maps_t(const IterArgs& a, TmaSweepMaps* maps) {
    const int n = a.e_new.n;
    if (!a.e_old.p || !a.g.p || a.bst || n < XT_MIN_N || (a.e_old.pitch * sizeof(T)) % 16 || (a.g.pitch * sizeof(T)) % 16 ||
        reinterpret_cast<uintptr_t>(a.e_old.p) % 16 || reinterpret_cast<uintptr_t>(a.g.p) % 16 || a.e_new.pitch % 2 ||
        reinterpret_cast<uintptr_t>(a.e_new.p) % (2 * sizeof(T)))
        return cudaErrorInvalidValue;
    cudaError_t e = xt_map<T>(&maps->me, a.e_old.p, n, a.e_old.pitch, xt_rows<T>() + 4);
    if (e == cudaSuccess) e = xt_map<T>(&maps->mg, a.g.p, n, a.g.pitch, xt_rows<T>() + 2);
    return e;
}

cudaError_t tma_sweep_maps(int prec, const IterArgs& a, TmaSweepMaps* maps) {
    switch (prec) {
        case PREC_FP32: return tma_sweep_maps_t<float>(a, maps);
        case PREC_BF16: return tma_sweep_maps_t<__nv_bfloat16>(a, maps);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t iterate2_tma_t(const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s) {
    constexpr int RT = xt_rows<T>();
    constexpr int Q = xt_cols<T>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_jacobi2_x2t<T, RT, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)xt_smem_bytes<T>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int n = a.e_new.n;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n - 1) / XT_OUT + 1), (unsigned)((n - 1 + RT - 1) / RT));
    cfg.blockDim = dim3(XT_W / Q);
    cfg.dynamicSmemBytes = xt_smem_bytes<T>();
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_jacobi2_x2t<T, RT, Q>, a, maps.me, maps.mg, fault);
}

// 3-D TMA two-sweep kernel: RY output rows, RZ output planes per block, Q = 2 NP columns per thread.
// Measured at 513³ (level-0 pair inside the solve; RY 2 / 4 / 8, NP 1 / 2): bfloat16 8 rows, four
// columns per thread (414 us against 576 us for the marching k_jacobi3_x2; 409 at 4 rows, 471-569
// at 2), binary32 8 rows, two columns (567 against 598 us; 578 at 4 rows, 666 at 2).
template <typename T> constexpr int x3_rows() { return 8; }
constexpr int X3_PLANES = 32;
template <typename T> constexpr int x3_pairs() { return sizeof(T) == 2 ? 2 : 1; }
template <typename T, int D> constexpr size_t x3_smem_bytes() {
    return (size_t)((D + 3) * (x3_rows<T>() + 4) + (D + 5) * (x3_rows<T>() + 2)) * XT_W * sizeof(T) + 64;
}

// A 3-D lattice array of (n + 1)^3 nodes, rows of `pitch` elements, (n + 1) rows per plane, as a 3-D
// tensor whose box is XT_W columns x `rows` rows x 1 plane; zero outside the lattice.
template <typename T>
cudaError_t xt_map3(CUtensorMap* map, const void* base, int n, int64_t pitch, int rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = xt_encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)(n + 1), (cuuint64_t)(n + 1), (cuuint64_t)(n + 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(T), (cuuint64_t)pitch * (cuuint64_t)(n + 1) * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)XT_W, (cuuint32_t)rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt = sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T> cudaError_t tma_sweep_maps3_t(const IterArgs& a, TmaSweepMaps* maps) {
    const int n = a.e_new.n;
    if (!a.e_old.p || !a.g.p || a.bst || n < XT_MIN_N || (a.e_old.pitch * sizeof(T)) % 16 || (a.g.pitch * sizeof(T)) % 16 ||
        reinterpret_cast<uintptr_t>(a.e_old.p) % 16 || reinterpret_cast<uintptr_t>(a.g.p) % 16 || a.e_new.pitch % 4 ||
        reinterpret_cast<uintptr_t>(a.e_new.p) % 16)
        return cudaErrorInvalidValue;
    cudaError_t e = xt_map3<T>(&maps->me, a.e_old.p, n, a.e_old.pitch, x3_rows<T>() + 4);
    if (e == cudaSuccess) e = xt_map3<T>(&maps->mg, a.g.p, n, a.g.pitch, x3_rows<T>() + 2);
    return e;
}

cudaError_t tma_sweep_maps3(int prec, const IterArgs& a, TmaSweepMaps* maps) {
    switch (prec) {
        case PREC_FP32: return tma_sweep_maps3_t<float>(a, maps);
        case PREC_BF16: return tma_sweep_maps3_t<__nv_bfloat16>(a, maps);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int D>
cudaError_t iterate3_2_tma_d(const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s) {
    constexpr int RY = x3_rows<T>(), NP = x3_pairs<T>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_jacobi3_x2t<T, RY, X3_PLANES, NP, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)x3_smem_bytes<T, D>());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int n = a.e_new.n;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n - 1) / XT_OUT + 1), (unsigned)((n - 1 + RY - 1) / RY),
                       (unsigned)((n - 1 + X3_PLANES - 1) / X3_PLANES));
    cfg.blockDim = dim3(XT_W / (2 * NP));
    cfg.dynamicSmemBytes = x3_smem_bytes<T, D>();
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_jacobi3_x2t<T, RY, X3_PLANES, NP, D>, a, maps.me, maps.mg, fault);
}

// Prefetch distance 1: at 513³ distances 2 and 3 measured slower (binary32 934 / 927 us per level-0
// pair against 588, bfloat16 492 / 611 against 425): their larger rings cost resident blocks per SM.
template <typename T>
cudaError_t iterate3_2_tma_t(const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s) {
    return iterate3_2_tma_d<T, 1>(a, maps, fault, s);
}

cudaError_t launch_iterate3_2_tma(int prec, const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s) {
    switch (prec) {
        case PREC_FP32: return iterate3_2_tma_t<float>(a, maps, fault, s);
        case PREC_BF16: return iterate3_2_tma_t<__nv_bfloat16>(a, maps, fault, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_iterate2_tma(int prec, const IterArgs& a, const TmaSweepMaps& maps, int* fault, cudaStream_t s) {
    switch (prec) {
        case PREC_FP32: return iterate2_tma_t<float>(a, maps, fault, s);
        case PREC_BF16: return iterate2_tma_t<__nv_bfloat16>(a, maps, fault, s);
        default: return cudaErrorInvalidValue;
    }
}

// The library's self-test of the two-sweep kernels: the packed kernel writes into out_packed, the
// per-column kernel into a.e_new, from the same input.
cudaError_t launch_check_sweep_pair(int prec, const IterArgs& a, void* out_packed, cudaStream_t s) {
    IterArgs p = a;
    p.e_new.p = out_packed;
    if (!pairs_ok(prec, a) || !pairs_ok(prec, p)) return cudaErrorInvalidValue;
    const int n = a.e_new.n, rows = a.rows > 0 ? a.rows : 8;
    const dim3 b(JX);
    const dim3 gp((unsigned)((((n + X2P_OUT - 1) / X2P_OUT) + JX / 32 - 1) / (JX / 32)), (unsigned)((n - 1 + rows - 1) / rows));
    const dim3 gc((unsigned)((((n - 1 + X2_OUT - 1) / X2_OUT) + JX / 32 - 1) / (JX / 32)), gp.y);
    cudaError_t e;
    if (prec == PREC_FP32) {
        e = launch_k(k_jacobi2_x2p<float, false>, gp, b, s, p, rows);
        if (e == cudaSuccess) e = launch_k(k_jacobi2_x2<float, false>, gc, b, s, a, rows);
    } else {
        e = launch_k(k_jacobi2_x2p<__nv_bfloat16, false>, gp, b, s, p, rows);
        if (e == cudaSuccess) e = launch_k(k_jacobi2_x2<__nv_bfloat16, false>, gc, b, s, a, rows);
    }
    return e;
}

__global__ void k_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        f_out[k] = narrow_rn(d_in[k]);
        d_out[k] = widen_f32(f_in[k]);
    }
}

cudaError_t launch_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n,
                                     cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256, blocks = want < 152 * 16 ? want : 152 * 16;
    k_check_conversions<<<(unsigned)blocks, 256, 0, s>>>(d_in, f_out, f_in, d_out, n);
    return cudaGetLastError();
}

cudaError_t launch_prolong(int ndim, int prec, bool strict, const ProlongArgs& a, cudaStream_t s) {
    DISPATCH_PREC(prec, prolong_t<T>(ndim, strict, a, s));
}

int residual_blocks(int ndim, bool strict, int n) {
    const dim3 g = resid_grid(ndim, strict, n);
    return (int)(g.x * g.y * g.z);
}

cudaError_t launch_residual(int ndim, int prec, bool strict, const ResidArgs& a, int n, cudaStream_t s) {
    DISPATCH_PREC(prec, residual_t<T>(ndim, strict, a, n, s));
}

cudaError_t launch_restrict(int ndim, int prec, bool strict, const RestrictArgs& a, cudaStream_t s) {
    DISPATCH_PREC(prec, restrict_t<T>(ndim, strict, a, s));
}

cudaError_t launch_pow2_iterate(int prec, const Pow2IterArgs& a, cudaStream_t s) {
    const dim3 g((unsigned)((a.N + P2X - 1) / P2X), (unsigned)((a.N + P2Y - 1) / P2Y)), b(P2X, P2Y);
    DISPATCH_PREC(prec, (launch_k(k_pow2_iterate<T>, g, b, s, a), cudaGetLastError()));
}

cudaError_t launch_pow2_restrict(int prec, const Pow2RestrictArgs& a, cudaStream_t s) {
    const int l = 1 << a.m, nm = (a.N >> 1) >> a.m;
    const bool warp = l > 16;
    const int64_t rows = (int64_t)a.N * 2 * (nm + 1), cols = (int64_t)4 * (nm + 1) * (nm + 1);
    const int64_t tr = warp ? rows * 32 : rows, tc = warp ? cols * 32 : cols;
    const dim3 gr((unsigned)((tr + 255) / 256)), gc((unsigned)((tc + 255) / 256));
    cudaError_t e = cudaSuccess;
    switch (prec) {
        case PREC_FP64:
            e = warp ? launch_k(k_pow2_rows<double, true>, gr, 256, s, a) : launch_k(k_pow2_rows<double, false>, gr, 256, s, a);
            if (e == cudaSuccess) e = warp ? launch_k(k_pow2_cols<double, true>, gc, 256, s, a) : launch_k(k_pow2_cols<double, false>, gc, 256, s, a);
            break;
        case PREC_FP32:
            e = warp ? launch_k(k_pow2_rows<float, true>, gr, 256, s, a) : launch_k(k_pow2_rows<float, false>, gr, 256, s, a);
            if (e == cudaSuccess) e = warp ? launch_k(k_pow2_cols<float, true>, gc, 256, s, a) : launch_k(k_pow2_cols<float, false>, gc, 256, s, a);
            break;
        case PREC_BF16:
            e = warp ? launch_k(k_pow2_rows<__nv_bfloat16, true>, gr, 256, s, a) : launch_k(k_pow2_rows<__nv_bfloat16, false>, gr, 256, s, a);
            if (e == cudaSuccess) e = warp ? launch_k(k_pow2_cols<__nv_bfloat16, true>, gc, 256, s, a) : launch_k(k_pow2_cols<__nv_bfloat16, false>, gc, 256, s, a);
            break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_vc_setup(const double* k, int n, int m, bool dbl, void* kx, void* ky, void* wd, int64_t pitch,
                            double omega_j, int* bad, cudaStream_t s) {
    const int nm = n >> m;
    const dim3 b(32, 8), g((unsigned)((nm + 1 + 31) / 32), (unsigned)((nm + 1 + 7) / 8));
    if (dbl) k_vc_setup<double><<<g, b, 0, s>>>(k, n, m, (double*)kx, (double*)ky, (double*)wd, pitch, omega_j, bad);
    else k_vc_setup<float><<<g, b, 0, s>>>(k, n, m, (float*)kx, (float*)ky, (float*)wd, pitch, omega_j, bad);
    return cudaGetLastError();
}

// Shared memory of the largest level run (set once per device context, outside stream capture).
// Shared memory of a level run on n intervals: iterate (two buffers) and source on the lattice,
// the coarser variation on the coarse lattice.
template <typename T> constexpr size_t run_smem_bytes(int n) {
    return (3 * (size_t)(n + 1) * (size_t)(n + 1) + (size_t)(n / 2 + 1) * (size_t)(n / 2 + 1)) * sizeof(T);
}
static_assert(run_smem_bytes<float>(RUN_MAX_N) <= 232448, "a level run must fit one block's shared memory");

template <typename T> cudaError_t level_run_setup() {
    const int mx = (int)run_smem_bytes<T>(RUN_MAX_N);
    cudaError_t e = cudaFuncSetAttribute(k_level_run2<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_level_run2<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return e;
}

cudaError_t prepare_level_run(int prec) {
    switch (prec) {
        case PREC_FP32: return level_run_setup<float>();
        case PREC_BF16: return level_run_setup<__nv_bfloat16>();
        default: return cudaSuccess;
    }
}

template <typename T>
cudaError_t level_run_t(const ProlongArgs& pr, const IterArgs& it, int sweeps, int nb, cudaStream_t s) {
    const int n = it.e_new.n;
    if (n > RUN_MAX_N || n < 2 || sweeps < 1) return cudaErrorInvalidValue;
    const size_t smem = run_smem_bytes<T>(n);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1, 1, (unsigned)nb);
    cfg.blockDim = dim3((unsigned)n, RUN_Y);  // thread (x, y): column x + 1, band y of rows
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return it.bst ? cudaLaunchKernelEx(&cfg, k_level_run2<T, true>, pr, it, sweeps)
                  : cudaLaunchKernelEx(&cfg, k_level_run2<T, false>, pr, it, sweeps);
}

cudaError_t launch_level_run(int prec, const ProlongArgs& pr, const IterArgs& it, int sweeps, int nb, cudaStream_t s) {
    switch (prec) {
        case PREC_FP32: return level_run_t<float>(pr, it, sweeps, nb, s);
        case PREC_BF16: return level_run_t<__nv_bfloat16>(pr, it, sweeps, nb, s);
        default: return cudaErrorInvalidValue;  // FP64 sweeps are FP64-bound: one SM is too slow for them
    }
}

cudaError_t launch_coarse_block(int ndim, int prec, const BlockOp* ops, int nops, int nb, cudaStream_t s) {
    if (ndim == 2) { DISPATCH_PREC(prec, (launch_k(k_coarse_block<2, T>, dim3(1, 1, nb), 512, s, ops, nops), cudaGetLastError())); }
    DISPATCH_PREC(prec, (launch_k(k_coarse_block<3, T>, 1, 512, s, ops, nops), cudaGetLastError()));
}

template <typename T>
cudaError_t vresid_t(int ndim, bool strict, const VResidArgs& a, cudaStream_t s) {
    if (!strict && ndim == 2 && a.e.p != nullptr) {
        const int n = a.rho.n, rows = march_rows(2, n);
        launch_k(k_vresid2_fast<T>, dim3((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows)),
                 dim3(JX), s, a, rows);
        return cudaGetLastError();
    }
    const dim3 g = grid_for(ndim, a.rho.n), b(BX, BY);
    if (ndim == 2) {
        if (strict) launch_k(k_vresid<2, true, T>, g, b, s, a);
        else launch_k(k_vresid<2, false, T>, g, b, s, a);
    } else {
        if (strict) launch_k(k_vresid<3, true, T>, g, b, s, a);
        else launch_k(k_vresid<3, false, T>, g, b, s, a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t prolong_add_t(int ndim, bool strict, const ProlongAddArgs& a, cudaStream_t s) {
    if (!strict && ndim == 2) {
        const int n = a.e.n, rows = march_rows(2, n);
        launch_k(k_prolong_add2_s1<T>, dim3((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows)),
                 dim3(JX), s, a, rows);
        return cudaGetLastError();
    }
    const dim3 g = grid_for(ndim, a.e.n), b(BX, BY);
    if (ndim == 2) {
        if (strict) launch_k(k_prolong_add<2, true, T>, g, b, s, a);
        else launch_k(k_prolong_add<2, false, T>, g, b, s, a);
    } else {
        if (strict) launch_k(k_prolong_add<3, true, T>, g, b, s, a);
        else launch_k(k_prolong_add<3, false, T>, g, b, s, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_vresid(int ndim, int prec, bool strict, const VResidArgs& a, cudaStream_t s) {
    DISPATCH_PREC(prec, vresid_t<T>(ndim, strict, a, s));
}

cudaError_t launch_prolong_add(int ndim, int prec, bool strict, const ProlongAddArgs& a, cudaStream_t s) {
    DISPATCH_PREC(prec, prolong_add_t<T>(ndim, strict, a, s));
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    launch_k(k_finalize, a.batch ? a.batch : 1, 1024, s, a);
    return cudaGetLastError();
}

void persist_iter(const IterArgs& a, PersistItem& it) {
    const int n = a.e_new.n;
    it.it = a;
    if (a.m == 0 && a.e_old.p != nullptr) {  // as iterate_t: the marching sweep
        const int rows = a.rows > 0 ? a.rows : march_rows(2, n, a.nb);
        const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
        it.kind = PK_ITER;
        it.sub = 2 * pend + (a.dnew.p != nullptr ? 1 : 0);
        it.rows = rows;
        it.gx = (n - 1 + JX - 1) / JX;
        it.gy = (n - 1 + rows - 1) / rows;
    } else {
        it.kind = PK_ITERG;
        it.gx = (n - 1 + BX - 1) / BX;
        it.gy = (n - 1 + BY - 1) / BY;
    }
    it.gz = a.nb;
}

void persist_iter2(int sweeps, const IterArgs& a, PersistItem& it) {
    const int n = a.e_new.n;
    const double nodes = (double)a.nb * (double)(n - 1) * (double)(n - 1);
    const int out = (sweeps == 4) ? 34 - 2 * 4 : X2_OUT;
    const int rows = a.rows > 0 ? a.rows : (nodes >= 1.0e6 ? (sweeps == 4 ? 32 : 16) : 8);
    it.it = a;
    it.kind = (sweeps == 4) ? PK_ITER4 : PK_ITER2;
    it.rows = rows;
    it.gx = (((n - 1 + out - 1) / out) + JX / 32 - 1) / (JX / 32);
    it.gy = (n - 1 + rows - 1) / rows;
    it.gz = a.nb;
}

void persist_prolong(const ProlongArgs& a, PersistItem& it) {
    const int n = a.G.n;
    it.pr = a;
    if (a.s == 1) {
        const int rows = march_rows(2, n, a.nb);
        it.kind = PK_PROLONG2;
        it.rows = rows;
        it.gx = (n - 1 + JX - 1) / JX;
        it.gy = (n - 1 + rows - 1) / rows;
    } else {
        it.kind = PK_PROLONG;
        it.gx = (n - 1 + BX - 1) / BX;
        it.gy = (n - 1 + BY - 1) / BY;
    }
    it.gz = a.nb;
}

void persist_restrict(const RestrictArgs& a, PersistItem& it) {
    it.rs = a;
    it.kind = PK_RESTRICT;
    it.gx = (a.gc.n - 1 + BX - 1) / BX;
    it.gy = (a.gc.n - 1 + BY - 1) / BY;
    it.gz = a.nb;
}

void persist_block(const BlockOp* ops, int nops, int nb, PersistItem& it) {
    it.kind = PK_BLOCK;
    it.ops = ops;
    it.nops = nops;
    it.gx = it.gy = 1;
    it.gz = nb;
}

void persist_resid(const ResidArgs& a, int n, PersistItem& it) {
    const dim3 g = resid_grid(2, false, n);
    it.ra = a;
    it.kind = PK_RESID;
    it.n = n;
    it.gx = (int)g.x;
    it.gy = (int)g.y;
    it.gz = a.nb;
}

void persist_final(const FinalizeArgs& a, PersistItem& it) {
    it.fa = a;
    it.kind = PK_FINAL;
    it.gx = it.gy = 1;
    it.gz = a.batch ? a.batch : 1;
}

void persist_copy(const CopyOutArgs& a, int n, PersistItem& it) {
    it.co = a;
    it.kind = PK_COPY;
    it.n = n;
    it.gx = (n - 1 + BX - 1) / BX;
    it.gy = (n - 1 + BY - 1) / BY;
    it.gz = a.batch ? a.nb : 1;
}

template <typename T>
cudaError_t persistent_t(const PersistArgs& a, int* blocks, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent<T>, JX, 0);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int nb = sms * per;
    if (blocks) *blocks = nb;
    PersistArgs p = a;
    void* args[] = {&p};
    return cudaLaunchCooperativeKernel((const void*)k_batch_persistent<T>, dim3(nb), dim3(JX), args, 0, s);
}

cudaError_t launch_persistent(int prec, const PersistArgs& a, int* blocks, cudaStream_t s) {
    DISPATCH_PREC(prec, persistent_t<T>(a, blocks, s));
}

cudaError_t launch_copy_out(int ndim, const CopyOutArgs& a, int n, cudaStream_t s) {
    dim3 g = grid_for(ndim, n);
    const dim3 b(BX, BY);
    if (ndim == 2) g.z = (unsigned)a.nb;
    if (ndim == 2) launch_k(k_copy_out<2>, g, b, s, a, n);
    else launch_k(k_copy_out<3>, g, b, s, a, n);
    return cudaGetLastError();
}

}  // namespace homg
