// HOMG kernels for sm_103a: the fused relaxation+interpolation iteration, the lattice level change,
// update+residual, full-weighting restriction, the convergence test and the copy-out.
//
// Arithmetic: with STRICT every formula is evaluated in the CPU oracle's canonical operation order
// with round-to-nearest intrinsics (no FMA contraction); otherwise the compiler may contract.
#include <math.h>

#include "../../include/homg.h"
#include "homg_internal.h"

namespace homg {
namespace {

constexpr int BX = 32;
constexpr int BY = 8;

template <bool S> __device__ __forceinline__ double add(double a, double b) { return S ? __dadd_rn(a, b) : a + b; }
template <bool S> __device__ __forceinline__ double sub(double a, double b) { return S ? __dsub_rn(a, b) : a - b; }
template <bool S> __device__ __forceinline__ double mul(double a, double b) { return S ? __dmul_rn(a, b) : a * b; }

// Element (i, j, k) of a grid with `pitch` doubles per row and (n+1) rows per plane.
__device__ __forceinline__ int64_t at(int64_t pitch, int n, int i, int j, int k) {
    return ((int64_t)k * (n + 1) + j) * pitch + i;
}

// Value at (i, j[, k]) of the (bi/tri)linear interpolant of compact array d at stride 2^mp
// (Sec. 2: linear interpolation S; exact dyadic weights). Summation order as in the oracle:
// 2-D (w00 d00 + w10 d10) + (w01 d01 + w11 d11); 3-D x-pairs, then y, then z.
// With DIFF, the interpolated field is d - d2 (the level-change kernel's stale values).
template <int ND, bool S, bool DIFF>
__device__ __forceinline__ double interp(CGrid d, CGrid d2, int mp, int i, int j, int k) {
    const int lp = 1 << mp;
    const double inv = ldexp(1.0, -mp);
    const int I0 = i >> mp, a = i & (lp - 1), I1 = a ? I0 + 1 : I0;
    const int J0 = j >> mp, b = j & (lp - 1), J1 = b ? J0 + 1 : J0;
    const double wx0 = (double)(lp - a) * inv, wx1 = (double)a * inv;
    const double wy0 = (double)(lp - b) * inv, wy1 = (double)b * inv;
    auto val = [&](int I, int J, int K) -> double {
        double v = d.p[at(d.pitch, d.n, I, J, K)];
        if (DIFF) v = sub<S>(v, d2.p[at(d2.pitch, d2.n, I, J, K)]);
        return v;
    };
    if (ND == 2) {
        double t00 = mul<S>(mul<S>(wx0, wy0), val(I0, J0, 0));
        double t10 = mul<S>(mul<S>(wx1, wy0), val(I1, J0, 0));
        double t01 = mul<S>(mul<S>(wx0, wy1), val(I0, J1, 0));
        double t11 = mul<S>(mul<S>(wx1, wy1), val(I1, J1, 0));
        return add<S>(add<S>(t00, t10), add<S>(t01, t11));
    } else {
        const int K0 = k >> mp, c = k & (lp - 1), K1 = c ? K0 + 1 : K0;
        const double wz0 = (double)(lp - c) * inv, wz1 = (double)c * inv;
        const double wx[2] = {wx0, wx1}, wy[2] = {wy0, wy1}, wz[2] = {wz0, wz1};
        const int Ix[2] = {I0, I1}, Jy[2] = {J0, J1}, Kz[2] = {K0, K1};
        double t[2][2][2];
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
template <int ND, bool S>
__global__ void __launch_bounds__(BX * BY) k_iterate(IterArgs a) {
    const int n = a.e_new.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    const bool zero = (a.e_old.p == nullptr);
    auto E = [&](int ii, int jj, int kk) -> double {
        return zero ? 0.0 : a.e_old.p[at(a.e_old.pitch, n, ii, jj, kk)];
    };
    double v = E(i, j, k);
    const int l = 1 << a.m;
    const int lat_mask = l - 1;
    if (((i | j | (ND == 3 ? k : 0)) & lat_mask) == 0) {
        double lap;
        if (ND == 2) {
            lap = mul<S>(4.0, v);
            lap = sub<S>(lap, E(i - l, j, 0));
            lap = sub<S>(lap, E(i + l, j, 0));
            lap = sub<S>(lap, E(i, j - l, 0));
            lap = sub<S>(lap, E(i, j + l, 0));
        } else {
            lap = mul<S>(6.0, v);
            lap = sub<S>(lap, E(i - l, j, k));
            lap = sub<S>(lap, E(i + l, j, k));
            lap = sub<S>(lap, E(i, j - l, k));
            lap = sub<S>(lap, E(i, j + l, k));
            lap = sub<S>(lap, E(i, j, k - l));
            lap = sub<S>(lap, E(i, j, k + l));
        }
        const int I = i >> a.m, J = j >> a.m, K = (ND == 3) ? (k >> a.m) : 0;
        const double g = a.g.p[at(a.g.pitch, a.g.n, I, J, K)];
        // strict: g = h_m^2 F_m, delta = omega (g - lap); fast: g = omega h_m^2 F_m, delta = g - omega lap
        const double delta = S ? mul<S>(a.omega, sub<S>(g, lap)) : fma(-a.omega, lap, g);
        if (a.dnew.p) a.dnew.p[at(a.dnew.pitch, a.dnew.n, I, J, K)] = delta;
        v = add<S>(v, delta);
    }
    if (a.mp >= 0) {
        const int lpm = (1 << a.mp) - 1;
        if (((i | j | (ND == 3 ? k : 0)) & lpm) != 0) v = add<S>(v, interp<ND, S, false>(a.dprev, a.dprev, a.mp, i, j, k));
    }
    a.e_new.p[at(a.e_new.pitch, n, i, j, k)] = v;
}

// ---------------------------------------------------------------------------------------------
// Lattice form, level change (see ProlongArgs): stale values of the finer lattice.
// ---------------------------------------------------------------------------------------------
template <int ND, bool S>
__global__ void __launch_bounds__(BX * BY) k_prolong(ProlongArgs a) {
    const int n = a.G.n;
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    const int sm = (1 << a.s) - 1;
    double v;
    if (((i | j | (ND == 3 ? k : 0)) & sm) == 0)
        v = a.Gc.p[at(a.Gc.pitch, a.Gc.n, i >> a.s, j >> a.s, (ND == 3) ? (k >> a.s) : 0)];
    else
        v = interp<ND, S, true>(a.Gc, a.dl, a.s, i, j, k);
    a.G.p[at(a.G.pitch, n, i, j, k)] = v;
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
// residual equation after each cycle) and the level-0 source of the next cycle.
// ---------------------------------------------------------------------------------------------
template <int ND, bool S>
__global__ void __launch_bounds__(BX * BY) k_residual(ResidArgs a, int n) {
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
        if (a.e.p) v = add<S>(v, a.e.p[at(a.e.pitch, n, ii, jj, kk)]);
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
        if (a.g0.p) a.g0.p[at(a.g0.pitch, n, i, j, k)] = mul<S>(a.scale, r);
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
template <int ND, bool S>
__global__ void __launch_bounds__(BX * BY) k_restrict(RestrictArgs a) {
    const int nc = a.gc.n;
    const int I = blockIdx.x * BX + threadIdx.x + 1;
    const int J = blockIdx.y * BY + threadIdx.y + 1;
    const int K = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (I >= nc || J >= nc) return;
    const int i = 2 * I, j = 2 * J, k = 2 * K;
    auto F = [&](int ii, int jj, int kk) -> double { return a.gf.p[at(a.gf.pitch, a.gf.n, ii, jj, kk)]; };
    double v;
    if (ND == 2) {
        const double c = F(i, j, 0);
        const double edges = add<S>(add<S>(add<S>(F(i - 1, j, 0), F(i + 1, j, 0)), F(i, j - 1, 0)), F(i, j + 1, 0));
        const double corners =
            add<S>(add<S>(add<S>(F(i - 1, j - 1, 0), F(i + 1, j - 1, 0)), F(i - 1, j + 1, 0)), F(i + 1, j + 1, 0));
        v = mul<S>(add<S>(add<S>(mul<S>(4.0, c), mul<S>(2.0, edges)), corners), 0.25);
    } else {
        const double c = F(i, j, k);
        double faces = 0.0, edges = 0.0, corners = 0.0;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nz = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nz == 0) continue;
                    const double x = F(i + dx, j + dy, k + dz);
                    if (nz == 1) faces = add<S>(faces, x);
                    else if (nz == 2) edges = add<S>(edges, x);
                    else corners = add<S>(corners, x);
                }
        v = mul<S>(add<S>(add<S>(add<S>(mul<S>(8.0, c), mul<S>(4.0, faces)), mul<S>(2.0, edges)), corners), 0.0625);
    }
    a.gc.p[at(a.gc.pitch, nc, I, J, K)] = v;
}

// ---------------------------------------------------------------------------------------------
// K3: convergence test (Sec. 2, restart on the residual equation until the desired accuracy).
// One block; partial sums are added in a fixed order so the decision is reproducible. Enables the
// next cycle's conditional graph nodes while the solve continues.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_finalize(FinalizeArgs a) {
    __shared__ double sh[32];
    double sr = 0.0, sf = 0.0;
    for (int t = threadIdx.x; t < a.nparts; t += blockDim.x) {
        sr += a.part_r[t];
        if (a.part_f) sf += a.part_f[t];
    }
    sr = block_sum(sr, sh);
    if (a.part_f) sf = block_sum(sf, sh);
    if (threadIdx.x != 0) return;
    State* st = a.st;
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
        if (fn == 0.0) {
            st->zero_u = 1;
            st->relres = 0.0;
            st->status = HOMG_OK;
            st->done = 1;
            a.hist[0] = 0.0;
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
    a.hist[k] = rel;
    st->relres = rel;
    int status = -1;
    if (rel <= st->tol) status = HOMG_OK;
    else if (!isfinite(rel) || rel > st->div_factor * st->rr0) status = HOMG_DIVERGED;
    else if (k >= st->max_cycles) status = HOMG_NOT_CONVERGED;
    st->status = status;
    st->done = (status >= 0);
    if (status < 0 && k + 1 <= a.nstages) {
        for (int p = 0; p < 3; ++p) cudaGraphSetConditional(a.handles[3 * (k + 1) + p], 1u);
    }
}

// Copy the final iterate into the caller's u (interior nodes); u = 0 when ||f|| = 0.
template <int ND>
__global__ void __launch_bounds__(BX * BY) k_copy_out(CopyOutArgs a, int n) {
    const int i = blockIdx.x * BX + threadIdx.x + 1;
    const int j = blockIdx.y * BY + threadIdx.y + 1;
    const int k = (ND == 3) ? (int)blockIdx.z + 1 : 0;
    if (i >= n || j >= n) return;
    const State* st = a.st;
    double v = 0.0;
    if (!st->zero_u) {
        const CGrid src = (st->cycle & 1) ? a.u1 : a.u0;
        v = src.p[at(src.pitch, n, i, j, k)];
    }
    st->u[at(n + 1, n, i, j, k)] = v;
}


// ---------------------------------------------------------------------------------------------
// Fast level-0 iteration (every iteration of the lattice form, the level-0 iterations of the
// whole-grid form): damped Jacobi on every interior node with the source pre-scaled by omega,
//   v' = (1 - c omega) v + omega * (sum of the 2d neighbours) + omega h^2 F
// = 5 FP64 instructions per node in 2-D (7 in 3-D), plus the pending interpolation on the first
// iteration of a level. Each thread marches one column (2-D: along y; 3-D: along z) keeping the
// centre and its two neighbours along the march in registers; the other neighbours come through
// L1. The FP64 pipe, not DRAM, bounds this kernel on GB300.
// ---------------------------------------------------------------------------------------------
constexpr int JX = 128;  // threads per block along x (2-D)
constexpr int JR = 16;   // nodes per thread along the march

// Pending interpolation at stride 2 (level change m+1 -> m, the common case): nodes with one odd
// index take the mean of two lattice neighbours, nodes with two odd indexes the mean of four.
__device__ __forceinline__ double pend2_s1(const CGrid& d, int i, int j) {
    const int I0 = i >> 1, J0 = j >> 1;
    const double* p = d.p + (int64_t)J0 * d.pitch + I0;
    if ((j & 1) == 0) return 0.5 * (__ldg(p) + __ldg(p + 1));           // i odd
    if ((i & 1) == 0) return 0.5 * (__ldg(p) + __ldg(p + d.pitch));     // j odd
    return 0.25 * ((__ldg(p) + __ldg(p + 1)) + (__ldg(p + d.pitch) + __ldg(p + d.pitch + 1)));
}

template <int PEND, bool WD>
__global__ void __launch_bounds__(JX) k_jacobi2(IterArgs a, int rows) {
    const int n = a.e_new.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const double* __restrict__ E = a.e_old.p;
    const int64_t pe = a.e_old.pitch;
    double* __restrict__ O = a.e_new.p;
    const int64_t po = a.e_new.pitch;
    const double* __restrict__ G = a.g.p;
    const int64_t pg = a.g.pitch;
    const double om = a.omega, c1 = 1.0 - 4.0 * a.omega;
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    double vs = __ldg(E + (int64_t)(j0 - 1) * pe + i);
    double vc = __ldg(E + (int64_t)j0 * pe + i);
#pragma unroll 4
    for (int j = j0; j < j1; ++j) {
        const double* row = E + (int64_t)j * pe + i;
        const double vn = __ldg(row + pe);
        const double w = __ldg(row - 1), e = __ldg(row + 1);
        const double g = __ldg(G + (int64_t)j * pg + i);
        const double sum = (w + e) + (vs + vn);
        double v = fma(c1, vc, fma(om, sum, g));
        if (WD) a.dnew.p[(int64_t)j * a.dnew.pitch + i] = v - vc;
        if (PEND == 1 && ((i | j) & 1)) v += pend2_s1(a.dprev, i, j);
        if (PEND == 2 && ((i | j) & lpm)) v += interp<2, false, false>(a.dprev, a.dprev, a.mp, i, j, 0);
        O[(int64_t)j * po + i] = v;
        vs = vc;
        vc = vn;
    }
}

// Fast lattice-form level change at stride 2 (2-D): lattice nodes copy Gc; the others take the
// mean of the two or four surrounding values of Gc - dl.
__global__ void __launch_bounds__(JX) k_prolong2_s1(ProlongArgs a, int rows) {
    const int n = a.G.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * rows + 1;
    const int j1 = min(j0 + rows, n);
    const int I0 = i >> 1;
    const bool iodd = i & 1;
    const double* __restrict__ C = a.Gc.p;
    const double* __restrict__ D = a.dl.p;
    const int64_t pc = a.Gc.pitch, pd = a.dl.pitch;
    for (int j = j0; j < j1; ++j) {
        const int J0 = j >> 1;
        const double* c = C + (int64_t)J0 * pc + I0;
        const double* d = D + (int64_t)J0 * pd + I0;
        double v;
        if (!(j & 1)) {
            if (!iodd) v = __ldg(c);
            else v = 0.5 * ((__ldg(c) - __ldg(d)) + (__ldg(c + 1) - __ldg(d + 1)));
        } else if (!iodd) {
            v = 0.5 * ((__ldg(c) - __ldg(d)) + (__ldg(c + pc) - __ldg(d + pd)));
        } else {
            v = 0.25 * (((__ldg(c) - __ldg(d)) + (__ldg(c + 1) - __ldg(d + 1))) +
                        ((__ldg(c + pc) - __ldg(d + pd)) + (__ldg(c + pc + 1) - __ldg(d + pd + 1))));
        }
        a.G.p[(int64_t)j * a.G.pitch + i] = v;
    }
}

constexpr int J3X = 32, J3Y = 4;

template <bool PEND, bool WD>
__global__ void __launch_bounds__(J3X * J3Y) k_jacobi3(IterArgs a, int rows) {
    const int n = a.e_new.n;
    const int i = blockIdx.x * J3X + threadIdx.x + 1;
    const int j = blockIdx.y * J3Y + threadIdx.y + 1;
    if (i >= n || j >= n) return;
    const int k0 = blockIdx.z * rows + 1;
    const int k1 = min(k0 + rows, n);
    const double* __restrict__ E = a.e_old.p;
    const int64_t pe = a.e_old.pitch, ple = (int64_t)(n + 1) * pe;
    double* __restrict__ O = a.e_new.p;
    const int64_t po = a.e_new.pitch, plo = (int64_t)(n + 1) * po;
    const double* __restrict__ G = a.g.p;
    const int64_t pg = a.g.pitch, plg = (int64_t)(n + 1) * pg;
    const double om = a.omega, c1 = 1.0 - 6.0 * a.omega;
    const int lpm = PEND ? (1 << a.mp) - 1 : 0;
    const double* col = E + (int64_t)j * pe + i;
    double vb = __ldg(col + (int64_t)(k0 - 1) * ple);
    double vc = __ldg(col + (int64_t)k0 * ple);
#pragma unroll 2
    for (int k = k0; k < k1; ++k) {
        const double* p = col + (int64_t)k * ple;
        const double vt = __ldg(p + ple);
        const double w = __ldg(p - 1), e = __ldg(p + 1), sn = __ldg(p - pe), nn = __ldg(p + pe);
        const double g = __ldg(G + (int64_t)k * plg + (int64_t)j * pg + i);
        const double sum = ((w + e) + (sn + nn)) + (vb + vt);
        double v = fma(c1, vc, fma(om, sum, g));
        if (WD) a.dnew.p[(int64_t)k * (n + 1) * a.dnew.pitch + (int64_t)j * a.dnew.pitch + i] = v - vc;
        if (PEND && ((i | j | k) & lpm)) v += interp<3, false, false>(a.dprev, a.dprev, a.mp, i, j, k);
        O[(int64_t)k * plo + (int64_t)j * po + i] = v;
        vb = vc;
        vc = vt;
    }
}


// ---------------------------------------------------------------------------------------------
// Fast whole-grid iteration at level m >= 1 (2-D): every fine node adds the bilinear interpolant of
// the pending variation (level mp >= 1) unless it lies on the level-mp lattice, and level-m
// lattice nodes relax. Each thread marches one column; the interpolant along x is formed once per
// coarse cell row (r0, r1 at the cell's lower and upper lattice rows) and shared down the column,
// so a node off both lattices costs one FMA and one add.
// ---------------------------------------------------------------------------------------------
template <bool PEND>
__global__ void __launch_bounds__(JX) k_wholegrid2(IterArgs a) {
    const int n = a.e_new.n;
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    if (i >= n) return;
    const int j0 = blockIdx.y * JR + 1;
    const int j1 = min(j0 + JR, n);
    const double* __restrict__ E = a.e_old.p;
    const int64_t pe = a.e_old.pitch;
    double* __restrict__ O = a.e_new.p;
    const int64_t po = a.e_new.pitch;
    const int m = a.m, l = 1 << m, lm = l - 1;
    const double om = a.omega;
    const bool col_on_lattice = (i & lm) == 0;
    // pending interpolation, per column
    const int mp = PEND ? a.mp : 0;
    const int lpm = (1 << mp) - 1;
    const int I0 = i >> mp;
    const double alpha = PEND ? (double)(i & lpm) * ldexp(1.0, -mp) : 0.0;
    const double beta_step = PEND ? ldexp(1.0, -mp) : 0.0;
    const double* __restrict__ D = a.dprev.p;
    const int64_t pd = a.dprev.pitch;
    const bool col_on_prev = (i & lpm) == 0;
    int cell = -1;
    double r0 = 0.0, dr = 0.0;
    for (int j = j0; j < j1; ++j) {
        double v = __ldg(E + (int64_t)j * pe + i);
        if (col_on_lattice && (j & lm) == 0) {
            const double sum = (__ldg(E + (int64_t)j * pe + i - l) + __ldg(E + (int64_t)j * pe + i + l)) +
                               (__ldg(E + (int64_t)(j - l) * pe + i) + __ldg(E + (int64_t)(j + l) * pe + i));
            const double g = __ldg(a.g.p + (int64_t)(j >> m) * a.g.pitch + (i >> m));
            const double delta = fma(om, fma(-4.0, v, sum), g);
            if (a.dnew.p) a.dnew.p[(int64_t)(j >> m) * a.dnew.pitch + (i >> m)] = delta;
            v += delta;
        }
        if (PEND) {
            const int J0 = j >> mp;
            const int b = j & lpm;
            if (!(col_on_prev && b == 0)) {
                if (J0 != cell) {
                    const double* d0 = D + (int64_t)J0 * pd + I0;
                    const double* d1 = d0 + pd;
                    const double a0 = __ldg(d0), a1 = __ldg(d1);
                    const double q0 = fma(alpha, __ldg(d0 + 1) - a0, a0);
                    const double q1 = fma(alpha, __ldg(d1 + 1) - a1, a1);
                    r0 = q0;
                    dr = q1 - q0;
                    cell = J0;
                }
                v += fma((double)b * beta_step, dr, r0);
            }
        }
        O[(int64_t)j * po + i] = v;
    }
}

// ---------------------------------------------------------------------------------------------
// Fast update + residual (2-D): one column per thread marching along y, u_new = u_in + e formed
// once per node for the column and once for each side neighbour; 10 FP64 instructions per node.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(JX) k_residual2_fast(ResidArgs a, int n) {
    __shared__ double sh[JX / 32];
    const int i = blockIdx.x * JX + threadIdx.x + 1;
    const int j0 = blockIdx.y * JR + 1;
    const int j1 = min(j0 + JR, n);
    const bool active = i < n;
    const bool upd = a.e.p != nullptr;
    const double* __restrict__ U = a.u_in.p ? a.u_in.p : a.st->u;
    const int64_t pu = a.u_in.p ? a.u_in.pitch : (int64_t)(n + 1);
    const double* __restrict__ Ev = a.e.p;
    const int64_t pe = a.e.pitch;
    const double* __restrict__ F = a.st->f;
    const int64_t pf = n + 1;
    // u_new at (ii, jj), 0 on the boundary
    auto un = [&](int ii, int jj) -> double {
        if (ii <= 0 || jj <= 0 || ii >= n || jj >= n) return 0.0;
        double v = __ldg(U + (int64_t)jj * pu + ii);
        if (upd) v += __ldg(Ev + (int64_t)jj * pe + ii);
        return v;
    };
    double rr = 0.0, ff = 0.0;
    if (active) {
        double vs = un(i, j0 - 1), vc = un(i, j0);
        for (int j = j0; j < j1; ++j) {
            const double vn = un(i, j + 1);
            const double w = un(i - 1, j), e = un(i + 1, j);
            const double sum = (w + e) + (vs + vn);
            const double fv = __ldg(F + (int64_t)j * pf + i);
            const double r = fma(a.inv_h2, fma(-4.0, vc, sum), fv);
            if (a.u_out.p) a.u_out.p[(int64_t)j * a.u_out.pitch + i] = vc;
            if (a.g0.p) a.g0.p[(int64_t)j * a.g0.pitch + i] = a.scale * r;
            rr = fma(r, r, rr);
            ff = fma(fv, fv, ff);
            vs = vc;
            vc = vn;
        }
    }
    const int bid = blockIdx.x + gridDim.x * blockIdx.y;
    double t = block_sum(rr, sh);
    if (threadIdx.x == 0) a.part_r[bid] = t;
    if (a.part_f) {
        t = block_sum(ff, sh);
        if (threadIdx.x == 0) a.part_f[bid] = t;
    }
}

// Nodes per thread along the march: long columns on large grids (fewer blocks, more reuse), short
// ones on small grids, where a thread's serial chain of loads would otherwise set the time.
int march_rows(int ndim, int n) {
    const double nodes = (ndim == 2) ? (double)(n - 1) * (n - 1) : (double)(n - 1) * (n - 1) * (n - 1);
    if (nodes >= 8.0e6) return 16;
    if (nodes >= 1.0e6) return 4;
    return 1;
}

dim3 grid_for(int ndim, int n) {
    return dim3((unsigned)((n - 1 + BX - 1) / BX), (unsigned)((n - 1 + BY - 1) / BY), ndim == 3 ? (unsigned)(n - 1) : 1u);
}

}  // namespace

cudaError_t launch_iterate(int ndim, bool strict, const IterArgs& a, cudaStream_t s) {
    if (!strict && a.m == 0 && a.e_old.p != nullptr) {
        const bool wd = a.dnew.p != nullptr;
        const int n = a.e_new.n;
        const int rows = march_rows(ndim, n);
        if (ndim == 2) {
            const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows)), b(JX);
            const int pend = a.mp < 0 ? 0 : (a.mp == 1 ? 1 : 2);
#define JAC2(P, W) k_jacobi2<P, W><<<g, b, 0, s>>>(a, rows)
            if (pend == 0) { if (wd) JAC2(0, true); else JAC2(0, false); }
            else if (pend == 1) { if (wd) JAC2(1, true); else JAC2(1, false); }
            else { if (wd) JAC2(2, true); else JAC2(2, false); }
#undef JAC2
        } else {
            const bool pend = a.mp >= 0;
            const dim3 g((unsigned)((n - 1 + J3X - 1) / J3X), (unsigned)((n - 1 + J3Y - 1) / J3Y),
                         (unsigned)((n - 1 + rows - 1) / rows)),
                b(J3X, J3Y);
            if (pend && wd) k_jacobi3<true, true><<<g, b, 0, s>>>(a, rows);
            else if (pend) k_jacobi3<true, false><<<g, b, 0, s>>>(a, rows);
            else if (wd) k_jacobi3<false, true><<<g, b, 0, s>>>(a, rows);
            else k_jacobi3<false, false><<<g, b, 0, s>>>(a, rows);
        }
        return cudaGetLastError();
    }
    if (!strict && ndim == 2 && a.m >= 1 && a.e_old.p != nullptr && a.mp != 0) {
        const int n = a.e_new.n;
        const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + JR - 1) / JR)), b(JX);
        if (a.mp >= 1) k_wholegrid2<true><<<g, b, 0, s>>>(a);
        else k_wholegrid2<false><<<g, b, 0, s>>>(a);
        return cudaGetLastError();
    }
    const dim3 g = grid_for(ndim, a.e_new.n), b(BX, BY);
    if (ndim == 2) {
        if (strict) k_iterate<2, true><<<g, b, 0, s>>>(a);
        else k_iterate<2, false><<<g, b, 0, s>>>(a);
    } else {
        if (strict) k_iterate<3, true><<<g, b, 0, s>>>(a);
        else k_iterate<3, false><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_prolong(int ndim, bool strict, const ProlongArgs& a, cudaStream_t s) {
    if (!strict && ndim == 2 && a.s == 1) {
        const int n = a.G.n;
        const int rows = march_rows(2, n);
        const dim3 g((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + rows - 1) / rows));
        k_prolong2_s1<<<g, dim3(JX), 0, s>>>(a, rows);
        return cudaGetLastError();
    }
    const dim3 g = grid_for(ndim, a.G.n), b(BX, BY);
    if (ndim == 2) {
        if (strict) k_prolong<2, true><<<g, b, 0, s>>>(a);
        else k_prolong<2, false><<<g, b, 0, s>>>(a);
    } else {
        if (strict) k_prolong<3, true><<<g, b, 0, s>>>(a);
        else k_prolong<3, false><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// The fast 2-D residual uses its own grid: (n-1)/JX x (n-1)/JR blocks.
static dim3 resid_grid(int ndim, bool strict, int n) {
    if (ndim == 2 && !strict) return dim3((unsigned)((n - 1 + JX - 1) / JX), (unsigned)((n - 1 + JR - 1) / JR));
    return grid_for(ndim, n);
}

int residual_blocks(int ndim, bool strict, int n) {
    const dim3 g = resid_grid(ndim, strict, n);
    return (int)(g.x * g.y * g.z);
}

cudaError_t launch_residual(int ndim, bool strict, const ResidArgs& a, int n, cudaStream_t s) {
    const dim3 g = resid_grid(ndim, strict, n);
    if (ndim == 2) {
        if (strict) k_residual<2, true><<<g, dim3(BX, BY), 0, s>>>(a, n);
        else k_residual2_fast<<<g, dim3(JX), 0, s>>>(a, n);
    } else {
        if (strict) k_residual<3, true><<<g, dim3(BX, BY), 0, s>>>(a, n);
        else k_residual<3, false><<<g, dim3(BX, BY), 0, s>>>(a, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_restrict(int ndim, bool strict, const RestrictArgs& a, cudaStream_t s) {
    const dim3 g = grid_for(ndim, a.gc.n), b(BX, BY);
    if (ndim == 2) {
        if (strict) k_restrict<2, true><<<g, b, 0, s>>>(a);
        else k_restrict<2, false><<<g, b, 0, s>>>(a);
    } else {
        if (strict) k_restrict<3, true><<<g, b, 0, s>>>(a);
        else k_restrict<3, false><<<g, b, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    k_finalize<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(int ndim, const CopyOutArgs& a, int n, cudaStream_t s) {
    const dim3 g = grid_for(ndim, n), b(BX, BY);
    if (ndim == 2) k_copy_out<2><<<g, b, 0, s>>>(a, n);
    else k_copy_out<3><<<g, b, 0, s>>>(a, n);
    return cudaGetLastError();
}

}  // namespace homg
