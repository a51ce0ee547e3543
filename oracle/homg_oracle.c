/*
 * HOMG CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of the high-occupancy multigrid (HOMG) of
 * Becerra-Sagredo, Malaga and Mandujano, "A novel and scalable Multigrid algorithm for many-core
 * architectures" (arXiv:1108.2045). Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file; the GPU library neither links nor calls it and
 * shares no code with it.
 *
 * Every function follows the paper's steps in the paper's order, one grid node at a time, with no
 * blocking, fusion or reordering. The arithmetic order inside each formula is fixed and written
 * out so a reader can check it by eye ("canonical order").
 *
 * Problem (Sec. 2, Eq. 1; Sec. 4, Eq. "poisson"): A u = f on the unit square (cube) with zero
 * Dirichlet boundary, A = -Laplacian discretised with the 5-point (2-D) or 7-point (3-D) stencil
 * on a node grid of (n+1)^d nodes, n = 2^K, h = 1/n. The paper writes the Poisson equation with
 * the opposite sign, and its relaxation formula, read with that sign, would grow the error for
 * any positive weight; the positive-definite form is used here so that damped Jacobi is stable,
 * and the paper's own test source is passed in with its sign flipped.
 *
 * Layout: node (i, j[, k]) of a grid with n intervals per side lives at
 *   2-D: j*(n+1) + i          3-D: (k*(n+1) + j)*(n+1) + i        (x fastest).
 * Level m (Sec. 2, relaxation formula) is the lattice of interior nodes whose indexes are all
 * multiples of l = 2^m, with spacing h_m = 2^m h. A "compact" level-m array stores one value per
 * node of that lattice (boundary included) as an (n/2^m + 1)^d grid in the same layout.
 *
 * Parity pins (tests/test_oracle_*.py): closed-form discrete eigen-solutions, dense direct solves
 * on tiny grids, the closed form of full weighting on a sine product, the adjoint relation between
 * full weighting and bilinear interpolation, exact reproduction of (tri)linear fields by the
 * interpolation, the damped-Jacobi amplification factor of a single-level cycle, the Fig. 3
 * narrative (spike, stall, pyramid), O(h^2) discretisation error, the residual decrease per cycle,
 * and the Fig. 4 error levels as an order-of-magnitude check. The schedule itself (Fig. 1 is
 * missing) is pinned only by the MFMG rule stated in Sec. 2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HOMG_ORACLE_OK 0
#define HOMG_ORACLE_NOT_CONVERGED 1
#define HOMG_ORACLE_DIVERGED 2
#define HOMG_ORACLE_EINVAL (-1)
#define HOMG_ORACLE_ENOMEM (-4)

static int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

static int log2_exact(int64_t n) {
    int k = 0;
    if (n < 1) return -1;
    while (((int64_t)1 << k) < n) ++k;
    return (((int64_t)1 << k) == n) ? k : -1;
}

/* ------------------------------------------------------------------------------------------ */
/* Schedule (Sec. 2, MFMG paragraph and Fig. 1 caption): levels are visited from the coarsest   */
/* M = levels-1 down to the finest 0; the coarsest gets two iterations and every finer level     */
/* doubles the count until it reaches MaxI.                                                      */
/* ------------------------------------------------------------------------------------------ */
int homg_oracle_mfmg_schedule(int levels, int max_i, int *sched, int cap) {
    int count = 0;
    if (levels < 1 || max_i < 1) return HOMG_ORACLE_EINVAL;
    int M = levels - 1;
    for (int m = M; m >= 0; --m) {
        int64_t nm = 2;
        for (int s = 0; s < M - m && nm < max_i; ++s) nm *= 2;
        if (nm > max_i) nm = max_i;
        for (int64_t t = 0; t < nm; ++t) {
            if (sched && count < cap) sched[count] = m;
            ++count;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------------------------ */
/* Residual r = f - A_h u (Sec. 2, step (b) of the two-grid scheme). Interior nodes only; the     */
/* boundary of r is 0 and boundary values of u are taken as the homogeneous Dirichlet value 0.  */
/* 2-D: A_h u = ((((4u - uW) - uE) - uS) - uN) / h^2                                              */
/* 3-D: A_h u = ((((((6u - uW) - uE) - uS) - uN) - uB) - uT) / h^2                                */
/* ------------------------------------------------------------------------------------------ */
static double u_at2(const double *u, int64_t n, int64_t i, int64_t j) {
    if (i <= 0 || j <= 0 || i >= n || j >= n) return 0.0;
    return u[j * (n + 1) + i];
}

static double u_at3(const double *u, int64_t n, int64_t i, int64_t j, int64_t k) {
    if (i <= 0 || j <= 0 || k <= 0 || i >= n || j >= n || k >= n) return 0.0;
    return u[(k * (n + 1) + j) * (n + 1) + i];
}

void homg_oracle_residual(int ndim, int64_t n, const double *f, const double *u, double *r) {
    const double h = 1.0 / (double)n;
    const double h2 = h * h;
    if (ndim == 2) {
        for (int64_t j = 0; j <= n; ++j)
            for (int64_t i = 0; i <= n; ++i) {
                int64_t p = j * (n + 1) + i;
                if (i == 0 || j == 0 || i == n || j == n) { r[p] = 0.0; continue; }
                double lap = 4.0 * u_at2(u, n, i, j);
                lap = lap - u_at2(u, n, i - 1, j);
                lap = lap - u_at2(u, n, i + 1, j);
                lap = lap - u_at2(u, n, i, j - 1);
                lap = lap - u_at2(u, n, i, j + 1);
                r[p] = f[p] - lap / h2;
            }
    } else {
        for (int64_t k = 0; k <= n; ++k)
            for (int64_t j = 0; j <= n; ++j)
                for (int64_t i = 0; i <= n; ++i) {
                    int64_t p = (k * (n + 1) + j) * (n + 1) + i;
                    if (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n) { r[p] = 0.0; continue; }
                    double lap = 6.0 * u_at3(u, n, i, j, k);
                    lap = lap - u_at3(u, n, i - 1, j, k);
                    lap = lap - u_at3(u, n, i + 1, j, k);
                    lap = lap - u_at3(u, n, i, j - 1, k);
                    lap = lap - u_at3(u, n, i, j + 1, k);
                    lap = lap - u_at3(u, n, i, j, k - 1);
                    lap = lap - u_at3(u, n, i, j, k + 1);
                    r[p] = f[p] - lap / h2;
                }
    }
}

/* Euclidean norm over the interior nodes, summed in layout order (reading A7: relative 2-norm). */
double homg_oracle_norm_interior(int ndim, int64_t n, const double *v) {
    double s = 0.0;
    if (ndim == 2) {
        for (int64_t j = 1; j < n; ++j)
            for (int64_t i = 1; i < n; ++i) { double x = v[j * (n + 1) + i]; s += x * x; }
    } else {
        for (int64_t k = 1; k < n; ++k)
            for (int64_t j = 1; j < n; ++j)
                for (int64_t i = 1; i < n; ++i) { double x = v[(k * (n + 1) + j) * (n + 1) + i]; s += x * x; }
    }
    return sqrt(s);
}

/* ------------------------------------------------------------------------------------------ */
/* Restriction P (Sec. 2: restrictions are linearly weighted averages of neighbouring sources,   */
/* done once per cycle as nested reductions over the mesh; reading A4: full weighting, the       */
/* adjoint of (bi/tri)linear interpolation). Compact level-m array (nf intervals per side) to    */
/* compact level-(m+1) array (nf/2 intervals). Boundary of the coarse array is 0.               */
/* 2-D: Fc = (4c + 2(((w+e)+s)+n) + (((sw+se)+nw)+ne)) / 16                                      */
/* 3-D: Fc = (8c + 4*faces + 2*edges + corners) / 64, each group summed in a fixed order.         */
/* ------------------------------------------------------------------------------------------ */
void homg_oracle_restrict(int ndim, int64_t nf, const double *Ff, double *Fc) {
    const int64_t nc = nf / 2;
    if (ndim == 2) {
#define FF(I, J) Ff[(J) * (nf + 1) + (I)]
        for (int64_t J = 0; J <= nc; ++J)
            for (int64_t I = 0; I <= nc; ++I) {
                int64_t q = J * (nc + 1) + I;
                if (I == 0 || J == 0 || I == nc || J == nc) { Fc[q] = 0.0; continue; }
                int64_t i = 2 * I, j = 2 * J;
                double c = FF(i, j);
                double edges = ((FF(i - 1, j) + FF(i + 1, j)) + FF(i, j - 1)) + FF(i, j + 1);
                double corners = ((FF(i - 1, j - 1) + FF(i + 1, j - 1)) + FF(i - 1, j + 1)) + FF(i + 1, j + 1);
                Fc[q] = (4.0 * c + 2.0 * edges + corners) / 16.0;
            }
#undef FF
    } else {
#define FF(I, J, K) Ff[((K) * (nf + 1) + (J)) * (nf + 1) + (I)]
        for (int64_t K = 0; K <= nc; ++K)
            for (int64_t J = 0; J <= nc; ++J)
                for (int64_t I = 0; I <= nc; ++I) {
                    int64_t q = (K * (nc + 1) + J) * (nc + 1) + I;
                    if (I == 0 || J == 0 || K == 0 || I == nc || J == nc || K == nc) { Fc[q] = 0.0; continue; }
                    int64_t i = 2 * I, j = 2 * J, k = 2 * K;
                    double c = FF(i, j, k);
                    double faces = 0.0, edges = 0.0, corners = 0.0;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int nz = (dx != 0) + (dy != 0) + (dz != 0);
                                double v = FF(i + dx, j + dy, k + dz);
                                if (nz == 1) faces = faces + v;
                                else if (nz == 2) edges = edges + v;
                                else if (nz == 3) corners = corners + v;
                            }
                    Fc[q] = (8.0 * c + 4.0 * faces + 2.0 * edges + corners) / 64.0;
                }
#undef FF
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Interpolation S (Sec. 2: linear interpolation; Sec. 4, Fig. 3 "pyramid"): the value at node   */
/* (i,j[,k]) of the (bi/tri)linear interpolant of the compact level-mp array d (stride           */
/* lp = 2^mp). Weights are the exact dyadic fractions (lp-a)/lp and a/lp per direction.          */
/* 2-D order: (w00*d00 + w10*d10) + (w01*d01 + w11*d11)                                          */
/* ------------------------------------------------------------------------------------------ */
static double interp2(const double *d, int64_t n, int mp, int64_t i, int64_t j) {
    const int64_t lp = (int64_t)1 << mp, nc = n >> mp;
    /* lp is a power of two: i / lp == i >> mp and i % lp == i & (lp - 1) */
    int64_t I0 = i >> mp, a = i & (lp - 1);
    int64_t J0 = j >> mp, b = j & (lp - 1);
    int64_t I1 = (a == 0) ? I0 : I0 + 1, J1 = (b == 0) ? J0 : J0 + 1;
    double wx0 = (double)(lp - a) / (double)lp, wx1 = (double)a / (double)lp;
    double wy0 = (double)(lp - b) / (double)lp, wy1 = (double)b / (double)lp;
    double d00 = d[J0 * (nc + 1) + I0], d10 = d[J0 * (nc + 1) + I1];
    double d01 = d[J1 * (nc + 1) + I0], d11 = d[J1 * (nc + 1) + I1];
    return ((wx0 * wy0) * d00 + (wx1 * wy0) * d10) + ((wx0 * wy1) * d01 + (wx1 * wy1) * d11);
}

/* 3-D order: ((c000 + c100) + (c010 + c110)) + ((c001 + c101) + (c011 + c111)), cXYZ = w*d. */
static double interp3(const double *d, int64_t n, int mp, int64_t i, int64_t j, int64_t k) {
    const int64_t lp = (int64_t)1 << mp, nc = n >> mp;
    int64_t I0 = i >> mp, a = i & (lp - 1);
    int64_t J0 = j >> mp, b = j & (lp - 1);
    int64_t K0 = k >> mp, c = k & (lp - 1);
    int64_t I1 = (a == 0) ? I0 : I0 + 1, J1 = (b == 0) ? J0 : J0 + 1, K1 = (c == 0) ? K0 : K0 + 1;
    double wx[2] = {(double)(lp - a) / (double)lp, (double)a / (double)lp};
    double wy[2] = {(double)(lp - b) / (double)lp, (double)b / (double)lp};
    double wz[2] = {(double)(lp - c) / (double)lp, (double)c / (double)lp};
    int64_t Ix[2] = {I0, I1}, Jy[2] = {J0, J1}, Kz[2] = {K0, K1};
    double t[2][2][2];
    for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y)
            for (int x = 0; x < 2; ++x)
                t[z][y][x] = ((wx[x] * wy[y]) * wz[z]) * d[(Kz[z] * (nc + 1) + Jy[y]) * (nc + 1) + Ix[x]];
    return ((t[0][0][0] + t[0][0][1]) + (t[0][1][0] + t[0][1][1])) +
           ((t[1][0][0] + t[1][0][1]) + (t[1][1][0] + t[1][1][1]));
}

/* ------------------------------------------------------------------------------------------ */
/* One HOMG iteration (Sec. 2: relaxation on the level-m lattice fused with interpolation of the  */
/* previous iteration's variations on the rest of the grid; Sec. 4: the interpolation is         */
/* delayed by one iteration because both run in parallel).                                        */
/*                                                                                              */
/*   for p in L_m:   delta(p) = omega * (h_m^2 F_m(p) - lap_m(e_old)(p))                          */
/*                   (damped Jacobi = explicit Euler of Eq. "heat" at level m, sign-consistent     */
/*                    for A = -Laplacian; lap_m uses neighbours at distance l = 2^m)               */
/*   e_new(p) = e_old(p) + [p in L_m] delta(p) + [p not in L_mprev] (S_mprev dprev)(p)            */
/*                                                                                              */
/* Every term reads only e_old (Jacobi). mprev < 0 means "no pending variation" (first iteration */
/* of a cycle). F_m and d_new are compact level-m arrays; dprev is a compact level-mprev array.   */
/* d_new receives delta on L_m and 0 on the lattice boundary.                                     */
/* ------------------------------------------------------------------------------------------ */
static void iteration2(int64_t n, int m, int mprev, double omega, const double *Fm, const double *dprev,
                       const double *e_old, double *e_new, double *d_new) {
    const int64_t l = (int64_t)1 << m, nm = n >> m, side = n + 1;
    const int64_t lp = (mprev >= 0) ? ((int64_t)1 << mprev) : 1;
    const double h = 1.0 / (double)n;
    const double hm = h * (double)l;
    const double hm2 = hm * hm;
    for (int64_t q = 0; q < (nm + 1) * (nm + 1); ++q) d_new[q] = 0.0;
    for (int64_t j = 0; j <= n; ++j)
        for (int64_t i = 0; i <= n; ++i) {
            int64_t p = j * side + i;
            if (i == 0 || j == 0 || i == n || j == n) { e_new[p] = 0.0; continue; }
            double v = e_old[p];
            if ((i & (l - 1)) == 0 && (j & (l - 1)) == 0) { /* p on the level-m lattice */
                double lap = 4.0 * v;
                lap = lap - e_old[j * side + (i - l)];
                lap = lap - e_old[j * side + (i + l)];
                lap = lap - e_old[(j - l) * side + i];
                lap = lap - e_old[(j + l) * side + i];
                int64_t q = (j >> m) * (nm + 1) + (i >> m);
                double delta = omega * (hm2 * Fm[q] - lap);
                d_new[q] = delta;
                v = v + delta;
            }
            if (mprev >= 0 && !((i & (lp - 1)) == 0 && (j & (lp - 1)) == 0)) v = v + interp2(dprev, n, mprev, i, j);
            e_new[p] = v;
        }
}

static void iteration3(int64_t n, int m, int mprev, double omega, const double *Fm, const double *dprev,
                       const double *e_old, double *e_new, double *d_new) {
    const int64_t l = (int64_t)1 << m, nm = n >> m, side = n + 1;
    const int64_t lp = (mprev >= 0) ? ((int64_t)1 << mprev) : 1;
    const double h = 1.0 / (double)n;
    const double hm = h * (double)l;
    const double hm2 = hm * hm;
    for (int64_t q = 0; q < (nm + 1) * (nm + 1) * (nm + 1); ++q) d_new[q] = 0.0;
    for (int64_t k = 0; k <= n; ++k)
        for (int64_t j = 0; j <= n; ++j)
            for (int64_t i = 0; i <= n; ++i) {
                int64_t p = (k * side + j) * side + i;
                if (i == 0 || j == 0 || k == 0 || i == n || j == n || k == n) { e_new[p] = 0.0; continue; }
                double v = e_old[p];
                if ((i & (l - 1)) == 0 && (j & (l - 1)) == 0 && (k & (l - 1)) == 0) { /* p on the level-m lattice */
                    double lap = 6.0 * v;
                    lap = lap - e_old[(k * side + j) * side + (i - l)];
                    lap = lap - e_old[(k * side + j) * side + (i + l)];
                    lap = lap - e_old[(k * side + (j - l)) * side + i];
                    lap = lap - e_old[(k * side + (j + l)) * side + i];
                    lap = lap - e_old[((k - l) * side + j) * side + i];
                    lap = lap - e_old[((k + l) * side + j) * side + i];
                    int64_t q = ((k >> m) * (nm + 1) + (j >> m)) * (nm + 1) + (i >> m);
                    double delta = omega * (hm2 * Fm[q] - lap);
                    d_new[q] = delta;
                    v = v + delta;
                }
                if (mprev >= 0 && !((i & (lp - 1)) == 0 && (j & (lp - 1)) == 0 && (k & (lp - 1)) == 0)) v = v + interp3(dprev, n, mprev, i, j, k);
                e_new[p] = v;
            }
}

void homg_oracle_iteration(int ndim, int64_t n, int m, int mprev, double omega, const double *Fm,
                           const double *dprev, const double *e_old, double *e_new, double *d_new) {
    if (ndim == 2) iteration2(n, m, mprev, omega, Fm, dprev, e_old, e_new, d_new);
    else iteration3(n, m, mprev, omega, Fm, dprev, e_old, e_new, d_new);
}

/* ------------------------------------------------------------------------------------------ */
/* One HOMG cycle on the residual equation A e = F_0 starting from e = 0 (Sec. 2, steps (a)-(c)  */
/* and the MFMG paragraph). F_0 is the fine residual; F_1..F_{L-1} are built once, before the     */
/* cycle, by nested full-weighting reductions. The schedule lists the level of every iteration   */
/* and must end on the finest level, where no variation is left pending.                         */
/* omega = omega_J / (2 d) is the damped-Jacobi weight per iteration (reading A2).               */
/* ------------------------------------------------------------------------------------------ */
int homg_oracle_cycle(int ndim, int64_t n, int levels, const int *sched, int nsched, double omega_j,
                      const double *F0, double *e) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || nsched < 1) return HOMG_ORACLE_EINVAL;
    for (int t = 0; t < nsched; ++t)
        if (sched[t] < 0 || sched[t] >= levels) return HOMG_ORACLE_EINVAL;
    if (sched[nsched - 1] != 0) return HOMG_ORACLE_EINVAL;
    const double omega = omega_j / (2.0 * ndim);
    const int64_t side = n + 1;
    const int64_t total = ipow(side, ndim);

    double **F = (double **)calloc((size_t)levels, sizeof(double *));
    double *ebuf = (double *)malloc((size_t)total * sizeof(double));
    double *dA = (double *)malloc((size_t)total * sizeof(double));
    double *dB = (double *)malloc((size_t)total * sizeof(double));
    int rc = HOMG_ORACLE_OK;
    if (!F || !ebuf || !dA || !dB) { rc = HOMG_ORACLE_ENOMEM; goto done; }
    F[0] = (double *)F0;
    for (int m = 1; m < levels; ++m) {
        F[m] = (double *)malloc((size_t)ipow((n >> m) + 1, ndim) * sizeof(double));
        if (!F[m]) { rc = HOMG_ORACLE_ENOMEM; goto done; }
        homg_oracle_restrict(ndim, n >> (m - 1), F[m - 1], F[m]);
    }
    for (int64_t p = 0; p < total; ++p) e[p] = 0.0;
    {
        double *e_old = e, *e_new = ebuf, *dprev = dA, *dnew = dB;
        int mprev = -1;
        for (int t = 0; t < nsched; ++t) {
            int m = sched[t];
            homg_oracle_iteration(ndim, n, m, mprev, omega, F[m], dprev, e_old, e_new, dnew);
            double *tmp = e_old; e_old = e_new; e_new = tmp;
            tmp = dprev; dprev = dnew; dnew = tmp;
            mprev = m;
        }
        if (e_old != e) memcpy(e, e_old, (size_t)total * sizeof(double));
    }
done:
    if (F) for (int m = 1; m < levels; ++m) free(F[m]);
    free(F); free(ebuf); free(dA); free(dB);
    return rc;
}

/* ------------------------------------------------------------------------------------------ */
/* Solver (Sec. 2, last paragraph; Sec. 4: after a cycle the residual equation restarts the      */
/* cycles as often as needed). u is the initial guess and the result; only interior nodes are     */
/* read or written. hist[k] (k = 0..cycles) receives ||r_k|| / ||f|| before cycle k+1.            */
/* Stop when the relative residual <= tol (OK), when it is not finite or grows past              */
/* div_factor * hist[0] (DIVERGED), or after max_cycles cycles (NOT_CONVERGED).                  */
/* ||f|| = 0 gives u = 0 (interior), relres = 0, 0 cycles.                                        */
/* ------------------------------------------------------------------------------------------ */
int homg_oracle_solve(int ndim, int64_t n, int levels, const int *sched, int nsched, double omega_j,
                      double div_factor, const double *f, double *u, double tol, int max_cycles,
                      double *hist, int *cycles_out, double *relres_out) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || max_cycles < 0) return HOMG_ORACLE_EINVAL;
    const int64_t side = n + 1;
    const int64_t total = ipow(side, ndim);
    double fnorm = homg_oracle_norm_interior(ndim, n, f);
    if (fnorm == 0.0) {
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, k = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && k > 0 && i < n && j < n && k < n) u[p] = 0.0;
        }
        if (hist) hist[0] = 0.0;
        if (cycles_out) *cycles_out = 0;
        if (relres_out) *relres_out = 0.0;
        return HOMG_ORACLE_OK;
    }
    double *r = (double *)malloc((size_t)total * sizeof(double));
    double *e = (double *)malloc((size_t)total * sizeof(double));
    if (!r || !e) { free(r); free(e); return HOMG_ORACLE_ENOMEM; }
    int status = HOMG_ORACLE_NOT_CONVERGED, k;
    double rr = 0.0, rr0 = 0.0;
    for (k = 0;; ++k) {
        homg_oracle_residual(ndim, n, f, u, r);
        rr = homg_oracle_norm_interior(ndim, n, r) / fnorm;
        if (hist) hist[k] = rr;
        if (k == 0) rr0 = rr;
        if (rr <= tol) { status = HOMG_ORACLE_OK; break; }
        if (!isfinite(rr) || rr > div_factor * rr0) { status = HOMG_ORACLE_DIVERGED; break; }
        if (k == max_cycles) { status = HOMG_ORACLE_NOT_CONVERGED; break; }
        int rc = homg_oracle_cycle(ndim, n, levels, sched, nsched, omega_j, r, e);
        if (rc != HOMG_ORACLE_OK) { free(r); free(e); return rc; }
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, kk = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && kk > 0 && i < n && j < n && kk < n) u[p] = u[p] + e[p];
        }
    }
    free(r); free(e);
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = rr;
    return status;
}

/* ========================================================================================== */
/* Low-precision cycle for mixed-precision solves (Sec. 4: the paper's computations are all in  */
/* single precision). The cycle's values -- restricted sources, iterates and variations -- are  */
/* stored and computed in IEEE binary32 (prec = 1), or computed in binary32 and stored as       */
/* bfloat16 (prec = 2), following exactly the steps and canonical operation order of the FP64   */
/* functions above. The residual that feeds a cycle, the update u += e and the norms stay       */
/* binary64 in homg_oracle_solve_mixed: the restart loop is then iterative refinement.          */
/* ========================================================================================== */

/* bfloat16 keeps the sign, the 8 exponent bits and the top 7 fraction bits of binary32; rounding */
/* to it is round-to-nearest-even on the 16 dropped bits. NaN stays NaN (made quiet).            */
static float bf16_round(float x) {
    uint32_t b;
    memcpy(&b, &x, sizeof(b));
    if ((b & 0x7f800000u) == 0x7f800000u) {
        if (b & 0x007fffffu) b |= 0x00400000u;
        b &= 0xffff0000u;
    } else {
        uint32_t lsb = (b >> 16) & 1u;
        b += 0x7fffu + lsb;
        b &= 0xffff0000u;
    }
    memcpy(&x, &b, sizeof(x));
    return x;
}

static float store_lp(float x, int prec) { return prec == 2 ? bf16_round(x) : x; }

float homg_oracle_bf16_round(float x) { return bf16_round(x); }

static float interp2f(const float *d, int64_t n, int mp, int64_t i, int64_t j) {
    const int64_t lp = (int64_t)1 << mp, nc = n >> mp;
    int64_t I0 = i >> mp, a = i & (lp - 1);
    int64_t J0 = j >> mp, b = j & (lp - 1);
    int64_t I1 = (a == 0) ? I0 : I0 + 1, J1 = (b == 0) ? J0 : J0 + 1;
    float wx0 = (float)(lp - a) / (float)lp, wx1 = (float)a / (float)lp;
    float wy0 = (float)(lp - b) / (float)lp, wy1 = (float)b / (float)lp;
    float d00 = d[J0 * (nc + 1) + I0], d10 = d[J0 * (nc + 1) + I1];
    float d01 = d[J1 * (nc + 1) + I0], d11 = d[J1 * (nc + 1) + I1];
    return ((wx0 * wy0) * d00 + (wx1 * wy0) * d10) + ((wx0 * wy1) * d01 + (wx1 * wy1) * d11);
}

static float interp3f(const float *d, int64_t n, int mp, int64_t i, int64_t j, int64_t k) {
    const int64_t lp = (int64_t)1 << mp, nc = n >> mp;
    int64_t I0 = i >> mp, a = i & (lp - 1);
    int64_t J0 = j >> mp, b = j & (lp - 1);
    int64_t K0 = k >> mp, c = k & (lp - 1);
    int64_t I1 = (a == 0) ? I0 : I0 + 1, J1 = (b == 0) ? J0 : J0 + 1, K1 = (c == 0) ? K0 : K0 + 1;
    float wx[2] = {(float)(lp - a) / (float)lp, (float)a / (float)lp};
    float wy[2] = {(float)(lp - b) / (float)lp, (float)b / (float)lp};
    float wz[2] = {(float)(lp - c) / (float)lp, (float)c / (float)lp};
    int64_t Ix[2] = {I0, I1}, Jy[2] = {J0, J1}, Kz[2] = {K0, K1};
    float t[2][2][2];
    for (int z = 0; z < 2; ++z)
        for (int y = 0; y < 2; ++y)
            for (int x = 0; x < 2; ++x)
                t[z][y][x] = ((wx[x] * wy[y]) * wz[z]) * d[(Kz[z] * (nc + 1) + Jy[y]) * (nc + 1) + Ix[x]];
    return ((t[0][0][0] + t[0][0][1]) + (t[0][1][0] + t[0][1][1])) +
           ((t[1][0][0] + t[1][0][1]) + (t[1][1][0] + t[1][1][1]));
}

/* Full weighting (see homg_oracle_restrict), single precision, result stored at precision prec. */
void homg_oracle_restrict_lp(int ndim, int64_t nf, const float *Ff, float *Fc, int prec) {
    const int64_t nc = nf / 2;
    if (ndim == 2) {
#define FF(I, J) Ff[(J) * (nf + 1) + (I)]
        for (int64_t J = 0; J <= nc; ++J)
            for (int64_t I = 0; I <= nc; ++I) {
                int64_t q = J * (nc + 1) + I;
                if (I == 0 || J == 0 || I == nc || J == nc) { Fc[q] = 0.0f; continue; }
                int64_t i = 2 * I, j = 2 * J;
                float c = FF(i, j);
                float edges = ((FF(i - 1, j) + FF(i + 1, j)) + FF(i, j - 1)) + FF(i, j + 1);
                float corners = ((FF(i - 1, j - 1) + FF(i + 1, j - 1)) + FF(i - 1, j + 1)) + FF(i + 1, j + 1);
                Fc[q] = store_lp((4.0f * c + 2.0f * edges + corners) / 16.0f, prec);
            }
#undef FF
    } else {
#define FF(I, J, K) Ff[((K) * (nf + 1) + (J)) * (nf + 1) + (I)]
        for (int64_t K = 0; K <= nc; ++K)
            for (int64_t J = 0; J <= nc; ++J)
                for (int64_t I = 0; I <= nc; ++I) {
                    int64_t q = (K * (nc + 1) + J) * (nc + 1) + I;
                    if (I == 0 || J == 0 || K == 0 || I == nc || J == nc || K == nc) { Fc[q] = 0.0f; continue; }
                    int64_t i = 2 * I, j = 2 * J, k = 2 * K;
                    float c = FF(i, j, k);
                    float faces = 0.0f, edges = 0.0f, corners = 0.0f;
                    for (int dz = -1; dz <= 1; ++dz)
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int nz = (dx != 0) + (dy != 0) + (dz != 0);
                                float v = FF(i + dx, j + dy, k + dz);
                                if (nz == 1) faces = faces + v;
                                else if (nz == 2) edges = edges + v;
                                else if (nz == 3) corners = corners + v;
                            }
                    Fc[q] = store_lp((8.0f * c + 4.0f * faces + 2.0f * edges + corners) / 64.0f, prec);
                }
#undef FF
    }
}

/* One HOMG iteration (see homg_oracle_iteration), single precision; stored values at prec. */
void homg_oracle_iteration_lp(int ndim, int64_t n, int m, int mprev, float omega, const float *Fm,
                              const float *dprev, const float *e_old, float *e_new, float *d_new, int prec) {
    const int64_t l = (int64_t)1 << m, nm = n >> m, side = n + 1;
    const int64_t lp = (mprev >= 0) ? ((int64_t)1 << mprev) : 1;
    const float h = 1.0f / (float)n;
    const float hm = h * (float)l;
    const float hm2 = hm * hm;
    const int64_t dsize = (ndim == 2) ? (nm + 1) * (nm + 1) : (nm + 1) * (nm + 1) * (nm + 1);
    for (int64_t q = 0; q < dsize; ++q) d_new[q] = 0.0f;
    const int64_t kmax = (ndim == 2) ? 0 : n;
    for (int64_t k = 0; k <= kmax; ++k)
        for (int64_t j = 0; j <= n; ++j)
            for (int64_t i = 0; i <= n; ++i) {
                int64_t p = (k * side + j) * side + i;
                int boundary = i == 0 || j == 0 || i == n || j == n || (ndim == 3 && (k == 0 || k == n));
                if (boundary) { e_new[p] = 0.0f; continue; }
                float v = e_old[p];
                int on = (i & (l - 1)) == 0 && (j & (l - 1)) == 0 && (ndim == 2 || (k & (l - 1)) == 0);
                if (on) { /* p on the level-m lattice */
                    float lap;
                    if (ndim == 2) {
                        lap = 4.0f * v;
                        lap = lap - e_old[j * side + (i - l)];
                        lap = lap - e_old[j * side + (i + l)];
                        lap = lap - e_old[(j - l) * side + i];
                        lap = lap - e_old[(j + l) * side + i];
                    } else {
                        lap = 6.0f * v;
                        lap = lap - e_old[(k * side + j) * side + (i - l)];
                        lap = lap - e_old[(k * side + j) * side + (i + l)];
                        lap = lap - e_old[(k * side + (j - l)) * side + i];
                        lap = lap - e_old[(k * side + (j + l)) * side + i];
                        lap = lap - e_old[((k - l) * side + j) * side + i];
                        lap = lap - e_old[((k + l) * side + j) * side + i];
                    }
                    int64_t q = ((k >> m) * (nm + 1) + (j >> m)) * (nm + 1) + (i >> m);
                    float delta = omega * (hm2 * Fm[q] - lap);
                    d_new[q] = store_lp(delta, prec);
                    v = v + delta;
                }
                if (mprev >= 0) {
                    int on_prev = (i & (lp - 1)) == 0 && (j & (lp - 1)) == 0 && (ndim == 2 || (k & (lp - 1)) == 0);
                    if (!on_prev) v = v + ((ndim == 2) ? interp2f(dprev, n, mprev, i, j) : interp3f(dprev, n, mprev, i, j, k));
                }
                e_new[p] = store_lp(v, prec);
            }
}

/* One low-precision HOMG cycle on A e = F0 (see homg_oracle_cycle); F0 and e are binary64 arrays
 * at the interface, rounded to / widened from the cycle's precision. */
int homg_oracle_cycle_lp(int ndim, int64_t n, int levels, const int *sched, int nsched, double omega_j, int prec,
                         const double *F0, double *e) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || nsched < 1 || (prec != 1 && prec != 2))
        return HOMG_ORACLE_EINVAL;
    for (int t = 0; t < nsched; ++t)
        if (sched[t] < 0 || sched[t] >= levels) return HOMG_ORACLE_EINVAL;
    if (sched[nsched - 1] != 0) return HOMG_ORACLE_EINVAL;
    const float omega = (float)(omega_j / (2.0 * ndim));
    const int64_t total = ipow(n + 1, ndim);
    float **F = (float **)calloc((size_t)levels, sizeof(float *));
    float *ea = (float *)calloc((size_t)total, sizeof(float));
    float *eb = (float *)malloc((size_t)total * sizeof(float));
    float *dA = (float *)malloc((size_t)total * sizeof(float));
    float *dB = (float *)malloc((size_t)total * sizeof(float));
    int rc = HOMG_ORACLE_OK;
    if (!F || !ea || !eb || !dA || !dB) { rc = HOMG_ORACLE_ENOMEM; goto done; }
    for (int m = 0; m < levels; ++m) {
        F[m] = (float *)malloc((size_t)ipow((n >> m) + 1, ndim) * sizeof(float));
        if (!F[m]) { rc = HOMG_ORACLE_ENOMEM; goto done; }
    }
    for (int64_t p = 0; p < total; ++p) F[0][p] = store_lp((float)F0[p], prec);
    for (int m = 1; m < levels; ++m) homg_oracle_restrict_lp(ndim, n >> (m - 1), F[m - 1], F[m], prec);
    {
        float *e_old = ea, *e_new = eb, *dprev = dA, *dnew = dB;
        int mprev = -1;
        for (int t = 0; t < nsched; ++t) {
            int m = sched[t];
            homg_oracle_iteration_lp(ndim, n, m, mprev, omega, F[m], dprev, e_old, e_new, dnew, prec);
            float *tmp = e_old; e_old = e_new; e_new = tmp;
            tmp = dprev; dprev = dnew; dnew = tmp;
            mprev = m;
        }
        for (int64_t p = 0; p < total; ++p) e[p] = (double)e_old[p];
    }
done:
    if (F) for (int m = 0; m < levels; ++m) free(F[m]);
    free(F); free(ea); free(eb); free(dA); free(dB);
    return rc;
}

/* Mixed-precision restarted solve: binary64 residual, update and norms around low-precision     */
/* cycles (prec 1: binary32, prec 2: bfloat16 storage). Same stopping rules as homg_oracle_solve. */
int homg_oracle_solve_mixed(int ndim, int64_t n, int levels, const int *sched, int nsched, double omega_j,
                            double div_factor, int prec, const double *f, double *u, double tol, int max_cycles,
                            double *hist, int *cycles_out, double *relres_out) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || max_cycles < 0 || (prec != 1 && prec != 2))
        return HOMG_ORACLE_EINVAL;
    const int64_t side = n + 1;
    const int64_t total = ipow(side, ndim);
    double fnorm = homg_oracle_norm_interior(ndim, n, f);
    if (fnorm == 0.0) {
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, k = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && k > 0 && i < n && j < n && k < n) u[p] = 0.0;
        }
        if (hist) hist[0] = 0.0;
        if (cycles_out) *cycles_out = 0;
        if (relres_out) *relres_out = 0.0;
        return HOMG_ORACLE_OK;
    }
    double *r = (double *)malloc((size_t)total * sizeof(double));
    double *e = (double *)malloc((size_t)total * sizeof(double));
    if (!r || !e) { free(r); free(e); return HOMG_ORACLE_ENOMEM; }
    int status = HOMG_ORACLE_NOT_CONVERGED, k;
    double rr = 0.0, rr0 = 0.0;
    for (k = 0;; ++k) {
        homg_oracle_residual(ndim, n, f, u, r);
        rr = homg_oracle_norm_interior(ndim, n, r) / fnorm;
        if (hist) hist[k] = rr;
        if (k == 0) rr0 = rr;
        if (rr <= tol) { status = HOMG_ORACLE_OK; break; }
        if (!isfinite(rr) || rr > div_factor * rr0) { status = HOMG_ORACLE_DIVERGED; break; }
        if (k == max_cycles) { status = HOMG_ORACLE_NOT_CONVERGED; break; }
        int rc = homg_oracle_cycle_lp(ndim, n, levels, sched, nsched, omega_j, prec, r, e);
        if (rc != HOMG_ORACLE_OK) { free(r); free(e); return rc; }
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, kk = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && kk > 0 && i < n && j < n && kk < n) u[p] = u[p] + e[p];
        }
    }
    free(r); free(e);
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = rr;
    return status;
}

/* ========================================================================================== */
/* Classic V(nu1, nu2) cycle, the comparator of the benchmark (Sec. 2, the two-grid correction   */
/* scheme (a)-(e) applied recursively): (a) nu1 damped-Jacobi pre-smoothing sweeps, (b) the       */
/* residual restricted to the next coarser grid by full weighting, (c) the coarse residual        */
/* equation solved by the same cycle, (d) the coarse correction interpolated bilinearly and added,*/
/* (e) nu2 post-smoothing sweeps. Coarse operators are rediscretised (5/7-point at spacing 2^m h).*/
/* The coarsest level (reading of this build) is solved by max(1, n_c^2) undamped Jacobi sweeps   */
/* from zero: exact in one sweep when it has a single interior node.                             */
/* ========================================================================================== */

/* (Bi/tri)linear prolongation of a compact coarse array (nc = nf/2 intervals) onto the fine   */
/* compact grid: lattice nodes copy the coarse value, the others interpolate (weights 1/2, 1/4,  */
/* 1/8). Boundary nodes are 0.                                                                  */
void homg_oracle_prolong(int ndim, int64_t nf, const double *Ec, double *Ef) {
    const int64_t side = nf + 1, nc = nf / 2;
    const int64_t kmax = (ndim == 2) ? 0 : nf;
    for (int64_t k = 0; k <= kmax; ++k)
        for (int64_t j = 0; j <= nf; ++j)
            for (int64_t i = 0; i <= nf; ++i) {
                int64_t p = (k * side + j) * side + i;
                int boundary = i == 0 || j == 0 || i == nf || j == nf || (ndim == 3 && (k == 0 || k == nf));
                if (boundary) { Ef[p] = 0.0; continue; }
                int on = (i % 2 == 0) && (j % 2 == 0) && (ndim == 2 || k % 2 == 0);
                if (on) Ef[p] = Ec[((k / 2) * (nc + 1) + j / 2) * (nc + 1) + i / 2];
                else Ef[p] = (ndim == 2) ? interp2(Ec, nf, 1, i, j) : interp3(Ec, nf, 1, i, j, k);
            }
}

static int vcycle_level(int ndim, int64_t n, int m, int M, int nu1, int nu2, double omega, const double *Fm,
                        double *em) {
    const int64_t nm = n >> m;
    const int64_t cnt = ipow(nm + 1, ndim);
    double *tmp = (double *)malloc((size_t)cnt * sizeof(double));
    double *dsc = (double *)malloc((size_t)cnt * sizeof(double));
    int rc = HOMG_ORACLE_OK;
    if (!tmp || !dsc) { free(tmp); free(dsc); return HOMG_ORACLE_ENOMEM; }
    for (int64_t p = 0; p < cnt; ++p) em[p] = 0.0;
    if (m == M) {
        /* coarsest level: undamped Jacobi (omega = 1/(2d)) sweeps from zero */
        int64_t sweeps = nm * nm > 1 ? nm * nm : 1;
        for (int64_t s = 0; s < sweeps; ++s) {
            homg_oracle_iteration(ndim, nm, 0, -1, 1.0 / (2.0 * ndim), Fm, NULL, em, tmp, dsc);
            memcpy(em, tmp, (size_t)cnt * sizeof(double));
        }
        free(tmp); free(dsc);
        return HOMG_ORACLE_OK;
    }
    const int64_t ncm = nm / 2;
    const int64_t ccnt = ipow(ncm + 1, ndim);
    double *r = (double *)malloc((size_t)cnt * sizeof(double));
    double *Fc = (double *)malloc((size_t)ccnt * sizeof(double));
    double *ec = (double *)malloc((size_t)ccnt * sizeof(double));
    double *pe = (double *)malloc((size_t)cnt * sizeof(double));
    if (!r || !Fc || !ec || !pe) { rc = HOMG_ORACLE_ENOMEM; goto done; }
    for (int s = 0; s < nu1; ++s) {                            /* (a) pre-smoothing */
        homg_oracle_iteration(ndim, nm, 0, -1, omega, Fm, NULL, em, tmp, dsc);
        memcpy(em, tmp, (size_t)cnt * sizeof(double));
    }
    homg_oracle_residual(ndim, nm, Fm, em, r);                 /* (b) residual ...       */
    homg_oracle_restrict(ndim, nm, r, Fc);                     /*     ... restricted     */
    rc = vcycle_level(ndim, n, m + 1, M, nu1, nu2, omega, Fc, ec); /* (c) coarse equation */
    if (rc != HOMG_ORACLE_OK) goto done;
    homg_oracle_prolong(ndim, nm, ec, pe);                     /* (d) interpolate ...    */
    for (int64_t p = 0; p < cnt; ++p) em[p] = em[p] + pe[p];   /*     ... and correct    */
    for (int s = 0; s < nu2; ++s) {                            /* (e) post-smoothing */
        homg_oracle_iteration(ndim, nm, 0, -1, omega, Fm, NULL, em, tmp, dsc);
        memcpy(em, tmp, (size_t)cnt * sizeof(double));
    }
done:
    free(tmp); free(dsc); free(r); free(Fc); free(ec); free(pe);
    return rc;
}

/* One V(nu1, nu2) cycle on A e = F0 from e = 0 (levels 0 .. levels-1). */
int homg_oracle_vcycle(int ndim, int64_t n, int levels, int nu1, int nu2, double omega_j, const double *F0, double *e) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || nu1 < 0 || nu2 < 0) return HOMG_ORACLE_EINVAL;
    return vcycle_level(ndim, n, 0, levels - 1, nu1, nu2, omega_j / (2.0 * ndim), F0, e);
}

/* Restarted V-cycle solve: the same loop and stopping rules as homg_oracle_solve. */
int homg_oracle_solve_vcycle(int ndim, int64_t n, int levels, int nu1, int nu2, double omega_j, double div_factor,
                             const double *f, double *u, double tol, int max_cycles, double *hist, int *cycles_out,
                             double *relres_out) {
    int K = log2_exact(n);
    if ((ndim != 2 && ndim != 3) || K < 1 || levels < 1 || levels > K || max_cycles < 0) return HOMG_ORACLE_EINVAL;
    const int64_t side = n + 1;
    const int64_t total = ipow(side, ndim);
    double fnorm = homg_oracle_norm_interior(ndim, n, f);
    if (fnorm == 0.0) {
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, k = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && k > 0 && i < n && j < n && k < n) u[p] = 0.0;
        }
        if (hist) hist[0] = 0.0;
        if (cycles_out) *cycles_out = 0;
        if (relres_out) *relres_out = 0.0;
        return HOMG_ORACLE_OK;
    }
    double *r = (double *)malloc((size_t)total * sizeof(double));
    double *e = (double *)malloc((size_t)total * sizeof(double));
    if (!r || !e) { free(r); free(e); return HOMG_ORACLE_ENOMEM; }
    int status = HOMG_ORACLE_NOT_CONVERGED, k;
    double rr = 0.0, rr0 = 0.0;
    for (k = 0;; ++k) {
        homg_oracle_residual(ndim, n, f, u, r);
        rr = homg_oracle_norm_interior(ndim, n, r) / fnorm;
        if (hist) hist[k] = rr;
        if (k == 0) rr0 = rr;
        if (rr <= tol) { status = HOMG_ORACLE_OK; break; }
        if (!isfinite(rr) || rr > div_factor * rr0) { status = HOMG_ORACLE_DIVERGED; break; }
        if (k == max_cycles) { status = HOMG_ORACLE_NOT_CONVERGED; break; }
        int rc = homg_oracle_vcycle(ndim, n, levels, nu1, nu2, omega_j, r, e);
        if (rc != HOMG_ORACLE_OK) { free(r); free(e); return rc; }
        for (int64_t p = 0; p < total; ++p) {
            int64_t i = p % side, j = (p / side) % side, kk = (ndim == 3) ? p / (side * side) : 1;
            if (i > 0 && j > 0 && kk > 0 && i < n && j < n && kk < n) u[p] = u[p] + e[p];
        }
    }
    free(r); free(e);
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = rr;
    return status;
}

/* ========================================================================================== */
/* Variable-coefficient diffusion (2-D), an extension of the paper's Poisson problem:            */
/*   A u = -div(k grad u) on the unit square, zero Dirichlet boundary,                         */
/* discretised in flux form on the five-point stencil,                                          */
/*   (A u)(p) = sum over the four faces of p of k_f (u(p) - u(nb)) / h^2,                        */
/* with each face coefficient the harmonic mean of the node coefficients at its two ends,       */
/* k_f = 2 k(p) k(nb) / (k(p) + k(nb)), written ((2 a) b) / (a + b) (symmetric in a and b, bit   */
/* for bit). Level m uses the same form between lattice neighbours at spacing h_m, with k taken  */
/* by injection (its values at the lattice nodes). The HOMG relaxation (Sec. 2) becomes damped  */
/* Jacobi with the node's own diagonal D = ((k_W + k_E) + k_S) + k_N:                            */
/*   delta(p) = (omega_J / D) (h_m^2 F_m(p) - (A_m e)(p) h_m^2),                                 */
/* which for k = 1 (D = 4) is the Poisson relaxation with omega = omega_J / 4. Restriction,     */
/* interpolation, schedule and restart loop are the Poisson solver's. k is a node array on the   */
/* (n+1)^2 grid, boundary included: boundary faces use the boundary node values.               */
/* ========================================================================================== */
static double face_coef(double a, double b) { return ((2.0 * a) * b) / (a + b); }

/* Face coefficients of lattice node (i, j) at lattice spacing l (fine-grid index units). */
static void vc_faces(const double *kc, int64_t n, int64_t l, int64_t i, int64_t j, double *kw, double *ke,
                     double *ks, double *kn) {
    const int64_t side = n + 1;
    const double kp = kc[j * side + i];
    *kw = face_coef(kp, kc[j * side + (i - l)]);
    *ke = face_coef(kp, kc[j * side + (i + l)]);
    *ks = face_coef(kp, kc[(j - l) * side + i]);
    *kn = face_coef(kp, kc[(j + l) * side + i]);
}

void homg_oracle_residual_vc(int64_t n, const double *kc, const double *f, const double *u, double *r) {
    const double h = 1.0 / (double)n;
    const double h2 = h * h;
    for (int64_t j = 0; j <= n; ++j)
        for (int64_t i = 0; i <= n; ++i) {
            int64_t p = j * (n + 1) + i;
            if (i == 0 || j == 0 || i == n || j == n) { r[p] = 0.0; continue; }
            double kw, ke, ks, kn;
            vc_faces(kc, n, 1, i, j, &kw, &ke, &ks, &kn);
            const double uc = u_at2(u, n, i, j);
            double au = kw * (uc - u_at2(u, n, i - 1, j));
            au = au + ke * (uc - u_at2(u, n, i + 1, j));
            au = au + ks * (uc - u_at2(u, n, i, j - 1));
            au = au + kn * (uc - u_at2(u, n, i, j + 1));
            r[p] = f[p] - au / h2;
        }
}

/* One HOMG iteration with the variable-coefficient relaxation (see homg_oracle_iteration). */
void homg_oracle_iteration_vc(int64_t n, int m, int mprev, double omega_j, const double *kc, const double *Fm,
                              const double *dprev, const double *e_old, double *e_new, double *d_new) {
    const int64_t l = (int64_t)1 << m, nm = n >> m, side = n + 1;
    const int64_t lp = (mprev >= 0) ? ((int64_t)1 << mprev) : 1;
    const double h = 1.0 / (double)n;
    const double hm = h * (double)l;
    const double hm2 = hm * hm;
    for (int64_t q = 0; q < (nm + 1) * (nm + 1); ++q) d_new[q] = 0.0;
    for (int64_t j = 0; j <= n; ++j)
        for (int64_t i = 0; i <= n; ++i) {
            int64_t p = j * side + i;
            if (i == 0 || j == 0 || i == n || j == n) { e_new[p] = 0.0; continue; }
            double v = e_old[p];
            if ((i & (l - 1)) == 0 && (j & (l - 1)) == 0) { /* p on the level-m lattice */
                double kw, ke, ks, kn;
                vc_faces(kc, n, l, i, j, &kw, &ke, &ks, &kn);
                const double D = ((kw + ke) + ks) + kn;
                double ae = kw * (v - e_old[j * side + (i - l)]);
                ae = ae + ke * (v - e_old[j * side + (i + l)]);
                ae = ae + ks * (v - e_old[(j - l) * side + i]);
                ae = ae + kn * (v - e_old[(j + l) * side + i]);
                int64_t q = (j >> m) * (nm + 1) + (i >> m);
                double delta = (omega_j / D) * (hm2 * Fm[q] - ae);
                d_new[q] = delta;
                v = v + delta;
            }
            if (mprev >= 0 && !((i & (lp - 1)) == 0 && (j & (lp - 1)) == 0)) v = v + interp2(dprev, n, mprev, i, j);
            e_new[p] = v;
        }
}

/* The same iteration in binary32 (stored at prec: 1 binary32, 2 bfloat16). The coefficients are */
/* formed in binary64 as above and rounded once to binary32: k_f, and the weight omega_J / D.    */
void homg_oracle_iteration_vc_lp(int64_t n, int m, int mprev, double omega_j, const double *kc, const float *Fm,
                                 const float *dprev, const float *e_old, float *e_new, float *d_new, int prec) {
    const int64_t l = (int64_t)1 << m, nm = n >> m, side = n + 1;
    const int64_t lp = (mprev >= 0) ? ((int64_t)1 << mprev) : 1;
    const float h = 1.0f / (float)n;
    const float hm = h * (float)l;
    const float hm2 = hm * hm;
    for (int64_t q = 0; q < (nm + 1) * (nm + 1); ++q) d_new[q] = 0.0f;
    for (int64_t j = 0; j <= n; ++j)
        for (int64_t i = 0; i <= n; ++i) {
            int64_t p = j * side + i;
            if (i == 0 || j == 0 || i == n || j == n) { e_new[p] = 0.0f; continue; }
            float v = e_old[p];
            if ((i & (l - 1)) == 0 && (j & (l - 1)) == 0) {
                double kw, ke, ks, kn;
                vc_faces(kc, n, l, i, j, &kw, &ke, &ks, &kn);
                const float wd = (float)(omega_j / (((kw + ke) + ks) + kn));
                float ae = (float)kw * (v - e_old[j * side + (i - l)]);
                ae = ae + (float)ke * (v - e_old[j * side + (i + l)]);
                ae = ae + (float)ks * (v - e_old[(j - l) * side + i]);
                ae = ae + (float)kn * (v - e_old[(j + l) * side + i]);
                int64_t q = (j >> m) * (nm + 1) + (i >> m);
                float delta = wd * (hm2 * Fm[q] - ae);
                d_new[q] = store_lp(delta, prec);
                v = v + delta;
            }
            if (mprev >= 0 && !((i & (lp - 1)) == 0 && (j & (lp - 1)) == 0)) v = v + interp2f(dprev, n, mprev, i, j);
            e_new[p] = store_lp(v, prec);
        }
}

/* One variable-coefficient HOMG cycle on A e = F0 from e = 0 (see homg_oracle_cycle); prec 0:   */
/* binary64, 1: binary32, 2: bfloat16 storage (see homg_oracle_cycle_lp).                        */
int homg_oracle_cycle_vc(int64_t n, int levels, const int *sched, int nsched, double omega_j, int prec,
                         const double *kc, const double *F0, double *e) {
    int K = log2_exact(n);
    if (K < 1 || levels < 1 || levels > K || nsched < 1 || prec < 0 || prec > 2) return HOMG_ORACLE_EINVAL;
    for (int t = 0; t < nsched; ++t)
        if (sched[t] < 0 || sched[t] >= levels) return HOMG_ORACLE_EINVAL;
    if (sched[nsched - 1] != 0) return HOMG_ORACLE_EINVAL;
    const int64_t total = (n + 1) * (n + 1);
    int rc = HOMG_ORACLE_OK;
    if (prec == 0) {
        double **F = (double **)calloc((size_t)levels, sizeof(double *));
        double *ebuf = (double *)malloc((size_t)total * sizeof(double));
        double *dA = (double *)malloc((size_t)total * sizeof(double));
        double *dB = (double *)malloc((size_t)total * sizeof(double));
        if (!F || !ebuf || !dA || !dB) { rc = HOMG_ORACLE_ENOMEM; goto done64; }
        F[0] = (double *)F0;
        for (int m = 1; m < levels; ++m) {
            F[m] = (double *)malloc((size_t)(((n >> m) + 1) * ((n >> m) + 1)) * sizeof(double));
            if (!F[m]) { rc = HOMG_ORACLE_ENOMEM; goto done64; }
            homg_oracle_restrict(2, n >> (m - 1), F[m - 1], F[m]);
        }
        for (int64_t p = 0; p < total; ++p) e[p] = 0.0;
        {
            double *e_old = e, *e_new = ebuf, *dprev = dA, *dnew = dB;
            int mprev = -1;
            for (int t = 0; t < nsched; ++t) {
                int m = sched[t];
                homg_oracle_iteration_vc(n, m, mprev, omega_j, kc, F[m], dprev, e_old, e_new, dnew);
                double *tmp = e_old; e_old = e_new; e_new = tmp;
                tmp = dprev; dprev = dnew; dnew = tmp;
                mprev = m;
            }
            if (e_old != e) memcpy(e, e_old, (size_t)total * sizeof(double));
        }
    done64:
        if (F) for (int m = 1; m < levels; ++m) free(F[m]);
        free(F); free(ebuf); free(dA); free(dB);
        return rc;
    }
    float **F = (float **)calloc((size_t)levels, sizeof(float *));
    float *ea = (float *)calloc((size_t)total, sizeof(float));
    float *eb = (float *)malloc((size_t)total * sizeof(float));
    float *dA = (float *)malloc((size_t)total * sizeof(float));
    float *dB = (float *)malloc((size_t)total * sizeof(float));
    if (!F || !ea || !eb || !dA || !dB) { rc = HOMG_ORACLE_ENOMEM; goto donelp; }
    for (int m = 0; m < levels; ++m) {
        F[m] = (float *)malloc((size_t)(((n >> m) + 1) * ((n >> m) + 1)) * sizeof(float));
        if (!F[m]) { rc = HOMG_ORACLE_ENOMEM; goto donelp; }
    }
    for (int64_t p = 0; p < total; ++p) F[0][p] = store_lp((float)F0[p], prec);
    for (int m = 1; m < levels; ++m) homg_oracle_restrict_lp(2, n >> (m - 1), F[m - 1], F[m], prec);
    {
        float *e_old = ea, *e_new = eb, *dprev = dA, *dnew = dB;
        int mprev = -1;
        for (int t = 0; t < nsched; ++t) {
            int m = sched[t];
            homg_oracle_iteration_vc_lp(n, m, mprev, omega_j, kc, F[m], dprev, e_old, e_new, dnew, prec);
            float *tmp = e_old; e_old = e_new; e_new = tmp;
            tmp = dprev; dprev = dnew; dnew = tmp;
            mprev = m;
        }
        for (int64_t p = 0; p < total; ++p) e[p] = (double)e_old[p];
    }
donelp:
    if (F) for (int m = 0; m < levels; ++m) free(F[m]);
    free(F); free(ea); free(eb); free(dA); free(dB);
    return rc;
}

/* Restarted variable-coefficient solve (see homg_oracle_solve; binary64 residual, update and   */
/* norms around cycles of precision prec).                                                      */
int homg_oracle_solve_vc(int64_t n, int levels, const int *sched, int nsched, double omega_j, double div_factor,
                         int prec, const double *kc, const double *f, double *u, double tol, int max_cycles,
                         double *hist, int *cycles_out, double *relres_out) {
    int K = log2_exact(n);
    if (K < 1 || levels < 1 || levels > K || max_cycles < 0 || prec < 0 || prec > 2) return HOMG_ORACLE_EINVAL;
    const int64_t side = n + 1, total = side * side;
    double fnorm = homg_oracle_norm_interior(2, n, f);
    if (fnorm == 0.0) {
        for (int64_t j = 1; j < n; ++j)
            for (int64_t i = 1; i < n; ++i) u[j * side + i] = 0.0;
        if (hist) hist[0] = 0.0;
        if (cycles_out) *cycles_out = 0;
        if (relres_out) *relres_out = 0.0;
        return HOMG_ORACLE_OK;
    }
    double *r = (double *)malloc((size_t)total * sizeof(double));
    double *e = (double *)malloc((size_t)total * sizeof(double));
    if (!r || !e) { free(r); free(e); return HOMG_ORACLE_ENOMEM; }
    int status = HOMG_ORACLE_NOT_CONVERGED, k;
    double rr = 0.0, rr0 = 0.0;
    for (k = 0;; ++k) {
        homg_oracle_residual_vc(n, kc, f, u, r);
        rr = homg_oracle_norm_interior(2, n, r) / fnorm;
        if (hist) hist[k] = rr;
        if (k == 0) rr0 = rr;
        if (rr <= tol) { status = HOMG_ORACLE_OK; break; }
        if (!isfinite(rr) || rr > div_factor * rr0) { status = HOMG_ORACLE_DIVERGED; break; }
        if (k == max_cycles) { status = HOMG_ORACLE_NOT_CONVERGED; break; }
        int rc = homg_oracle_cycle_vc(n, levels, sched, nsched, omega_j, prec, kc, r, e);
        if (rc != HOMG_ORACLE_OK) { free(r); free(e); return rc; }
        for (int64_t j = 1; j < n; ++j)
            for (int64_t i = 1; i < n; ++i) u[j * side + i] = u[j * side + i] + e[j * side + i];
    }
    free(r); free(e);
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = rr;
    return status;
}

/* ========================================================================================== */
/* Power-of-two grids (Sec. 3), 2-D, whole-grid form. Reading of this build (Fig. 2 is missing): */
/*   the grid has N = 2^K nodes per side, boundary nodes included (h = 1 / (N - 1)); it is split */
/*   into four quadrants of H = N/2 nodes per side. Quadrant q (qx = q & 1, qy = q >> 1) has its */
/*   external corner at (cx, cy), cx = qx ? N-1 : 0, and points inward with sx = qx ? -1 : +1    */
/*   (likewise y). Its level-m lattice (m >= 1) is marked from that corner: local nodes (a, b),  */
/*   0 <= a, b <= n_m = H >> m, at fine node (cx + sx a 2^m, cy + sy b 2^m). The last local row  */
/*   and column (a or b = n_m) lie just outside the quadrant, on the far side of the centre      */
/*   lines, so the coarsest level (m = K-1) holds exactly one point per quadrant: the four        */
/*   central points. Local nodes with a = 0 or b = 0 are domain boundary; all others are marked  */
/*   and relaxed. The four lattices of a level are disjoint (N - 1 is odd).                      */
/*   Restriction: F_m = the m-fold nested full weighting of the fine residual, evaluated at each */
/*   quadrant's lattice nodes as one separable hat stencil (see homg_oracle_pow2_restrict).      */
/*   Relaxation at a marked node p of level m: delta = omega (h_m^2 F - lap_m e)(p), lap_m reading */
/*   the fine iterate at distance 2^m (0 outside the grid).                                       */
/*   Interpolation of the pending level-mp variation at a node not marked at level mp: bilinear  */
/*   from the lattice of the quadrant that contains the node, nothing from other quadrants.      */
/*   Level 0 is the whole fine grid (every interior node marked).                                 */
/* Arrays: the fine iterate and residual are N x N; per level m >= 1 the four quadrants' local    */
/* arrays of (n_m+1)^2 values are stored one after another (quadrant q at q (n_m+1)^2).           */
/* ========================================================================================== */
static int pow2_exponent(int64_t N) {
    int K = 0;
    while (((int64_t)1 << K) < N) ++K;
    return (((int64_t)1 << K) == N) ? K : -1;
}

static double e_at_pow2(const double *e, int64_t N, int64_t x, int64_t y) {
    if (x < 0 || y < 0 || x >= N || y >= N) return 0.0;
    return e[y * N + x];
}

/* Local lattice coordinate of fine index x along one axis for quadrant bit qb, or -1 when x is not  */
/* on the level-m lattice of that quadrant.                                                          */
static int64_t pow2_local(int64_t N, int m, int qb, int64_t x) {
    const int64_t H = N / 2, nm = H >> m, l = (int64_t)1 << m;
    const int64_t d = qb ? (N - 1 - x) : x;  /* distance from the external corner */
    if (d < 0 || (d & (l - 1)) != 0) return -1;
    const int64_t a = d >> m;
    return (a <= nm) ? a : -1;
}

/* quadrant bit of fine index x along one axis */
static int pow2_qbit(int64_t N, int64_t x) { return x >= N / 2; }

/* marked at level m: on some quadrant's lattice, not domain boundary (level 0: every interior node) */
static int pow2_marked(int64_t N, int m, int64_t x, int64_t y, int *q_out, int64_t *a_out, int64_t *b_out) {
    if (x <= 0 || y <= 0 || x >= N - 1 || y >= N - 1) return 0;
    if (m == 0) return 1;
    for (int q = 0; q < 4; ++q) {
        int64_t a = pow2_local(N, m, q & 1, x), b = pow2_local(N, m, q >> 1, y);
        if (a > 0 && b > 0) {
            if (q_out) *q_out = q;
            if (a_out) *a_out = a;
            if (b_out) *b_out = b;
            return 1;
        }
    }
    return 0;
}

/* Level m (>= 1) sources of the four quadrants from the fine N x N residual r: at lattice node p,  */
/* F_m(p) = sum over |dx|, |dy| < 2^m of w(dx) w(dy) r(p + (dx, dy)), w(d) = (2^m - |d|) / 4^m (zero  */
/* outside the grid), the composition of m full weightings at strides 1, 2, ..., 2^(m-1). At nodes   */
/* whose stencils stay inside one quadrant's lattices it equals the nested full weighting; at the    */
/* far row and column it reads the fine residual across the centre lines. Summation: rows of the     */
/* stencil first (dx ascending), then the row sums (dy ascending). Fc holds 4 (n_m+1)^2 values.     */
void homg_oracle_pow2_restrict(int64_t N, int m, const double *r, double *Fc) {
    const int64_t H = N / 2, nm = H >> m, side = nm + 1, l = (int64_t)1 << m;
    const double l2 = (double)l * (double)l;
    for (int q = 0; q < 4; ++q) {
        const int qx = q & 1, qy = q >> 1;
        double *out = Fc + (int64_t)q * side * side;
        for (int64_t b = 0; b <= nm; ++b)
            for (int64_t a = 0; a <= nm; ++a) {
                if (a == 0 || b == 0) { out[b * side + a] = 0.0; continue; }
                const int64_t x = qx ? (N - 1 - a * l) : a * l, y = qy ? (N - 1 - b * l) : b * l;
                double acc = 0.0;
                for (int64_t dy = -(l - 1); dy <= l - 1; ++dy) {
                    double row = 0.0;
                    for (int64_t dx = -(l - 1); dx <= l - 1; ++dx)
                        row = row + ((double)(l - (dx < 0 ? -dx : dx)) / l2) * e_at_pow2(r, N, x + dx, y + dy);
                    acc = acc + ((double)(l - (dy < 0 ? -dy : dy)) / l2) * row;
                }
                out[b * side + a] = acc;
            }
    }
}

/* Bilinear value at fine node (x, y) of quadrant q's level-mp variation (4 local arrays). */
static double pow2_interp(const double *d, int64_t N, int mp, int q, int64_t x, int64_t y) {
    const int64_t H = N / 2, nm = H >> mp, lp = (int64_t)1 << mp, side = nm + 1;
    const int qx = q & 1, qy = q >> 1;
    const int64_t dx = qx ? (N - 1 - x) : x, dy = qy ? (N - 1 - y) : y;
    const int64_t A0 = dx >> mp, fa = dx & (lp - 1), B0 = dy >> mp, fb = dy & (lp - 1);
    const int64_t A1 = fa ? A0 + 1 : A0, B1 = fb ? B0 + 1 : B0;
    const double wx0 = (double)(lp - fa) / (double)lp, wx1 = (double)fa / (double)lp;
    const double wy0 = (double)(lp - fb) / (double)lp, wy1 = (double)fb / (double)lp;
    const double *dq = d + (int64_t)q * side * side;
    const double d00 = dq[B0 * side + A0], d10 = dq[B0 * side + A1];
    const double d01 = dq[B1 * side + A0], d11 = dq[B1 * side + A1];
    return ((wx0 * wy0) * d00 + (wx1 * wy0) * d10) + ((wx0 * wy1) * d01 + (wx1 * wy1) * d11);
}

/* One HOMG iteration on the power-of-two grid (see homg_oracle_iteration): relax the nodes marked  */
/* at level m (source Fm: the fine residual for m = 0, else the four local arrays), and add the      */
/* interpolation of the pending level-mprev variation at the nodes not marked at level mprev.        */
/* d_new receives delta at the marked nodes (level m >= 1: four local arrays; level 0: unused).      */
void homg_oracle_pow2_iteration(int64_t N, int m, int mprev, double omega, const double *Fm, const double *dprev,
                                const double *e_old, double *e_new, double *d_new) {
    const int64_t H = N / 2, l = (int64_t)1 << m;
    const double h = 1.0 / (double)(N - 1);
    const double hm = h * (double)l;
    const double hm2 = hm * hm;
    if (m >= 1) {
        const int64_t side = (H >> m) + 1;
        for (int64_t p = 0; p < 4 * side * side; ++p) d_new[p] = 0.0;
    }
    for (int64_t y = 0; y < N; ++y)
        for (int64_t x = 0; x < N; ++x) {
            const int64_t p = y * N + x;
            if (x == 0 || y == 0 || x == N - 1 || y == N - 1) { e_new[p] = 0.0; continue; }
            double v = e_old[p];
            int q = 0;
            int64_t a = 0, b = 0;
            if (pow2_marked(N, m, x, y, &q, &a, &b)) {
                double lap = 4.0 * v;
                lap = lap - e_at_pow2(e_old, N, x - l, y);
                lap = lap - e_at_pow2(e_old, N, x + l, y);
                lap = lap - e_at_pow2(e_old, N, x, y - l);
                lap = lap - e_at_pow2(e_old, N, x, y + l);
                double F;
                if (m == 0) F = Fm[p];
                else {
                    const int64_t side = (H >> m) + 1;
                    F = Fm[(int64_t)q * side * side + b * side + a];
                }
                const double delta = omega * (hm2 * F - lap);
                if (m >= 1) {
                    const int64_t side = (H >> m) + 1;
                    d_new[(int64_t)q * side * side + b * side + a] = delta;
                }
                v = v + delta;
            }
            if (mprev >= 1 && !pow2_marked(N, mprev, x, y, NULL, NULL, NULL))
                v = v + pow2_interp(dprev, N, mprev, pow2_qbit(N, x) | (pow2_qbit(N, y) << 1), x, y);
            e_new[p] = v;
        }
}

/* One power-of-two HOMG cycle on A e = F0 (N x N fine residual) from e = 0. */
int homg_oracle_pow2_cycle(int64_t N, int levels, const int *sched, int nsched, double omega_j, const double *F0,
                           double *e) {
    const int K = pow2_exponent(N);
    if (K < 2 || levels < 1 || levels > K || nsched < 1) return HOMG_ORACLE_EINVAL;
    for (int t = 0; t < nsched; ++t)
        if (sched[t] < 0 || sched[t] >= levels) return HOMG_ORACLE_EINVAL;
    if (sched[nsched - 1] != 0) return HOMG_ORACLE_EINVAL;
    const double omega = omega_j / 4.0;
    const int64_t total = N * N, H = N / 2;
    double **F = (double **)calloc((size_t)levels, sizeof(double *));
    double **D = (double **)calloc((size_t)2 * levels, sizeof(double *));
    double *ebuf = (double *)malloc((size_t)total * sizeof(double));
    int rc = HOMG_ORACLE_OK;
    if (!F || !D || !ebuf) { rc = HOMG_ORACLE_ENOMEM; goto done; }
    F[0] = (double *)F0;
    for (int m = 1; m < levels; ++m) {
        const int64_t side = (H >> m) + 1;
        F[m] = (double *)malloc((size_t)(4 * side * side) * sizeof(double));
        D[2 * m] = (double *)calloc((size_t)(4 * side * side), sizeof(double));
        D[2 * m + 1] = (double *)calloc((size_t)(4 * side * side), sizeof(double));
        if (!F[m] || !D[2 * m] || !D[2 * m + 1]) { rc = HOMG_ORACLE_ENOMEM; goto done; }
        homg_oracle_pow2_restrict(N, m, F0, F[m]);
    }
    for (int64_t p = 0; p < total; ++p) e[p] = 0.0;
    {
        double *e_old = e, *e_new = ebuf;
        int mprev = -1;
        int par[64] = {0};
        const double *dprev = NULL;
        for (int t = 0; t < nsched; ++t) {
            const int m = sched[t];
            double *dnew = (m >= 1) ? D[2 * m + par[m]] : NULL;
            double dummy = 0.0;
            homg_oracle_pow2_iteration(N, m, mprev, omega, F[m], dprev, e_old, e_new, dnew ? dnew : &dummy);
            if (m >= 1) par[m] ^= 1;
            dprev = dnew;
            double *tmp = e_old; e_old = e_new; e_new = tmp;
            mprev = m;
        }
        if (e_old != e) memcpy(e, e_old, (size_t)total * sizeof(double));
    }
done:
    if (F) for (int m = 1; m < levels; ++m) free(F[m]);
    if (D) for (int m = 0; m < 2 * levels; ++m) free(D[m]);
    free(F); free(D); free(ebuf);
    return rc;
}

/* Restarted solve on the power-of-two grid (see homg_oracle_solve): the residual is the five-point */
/* Poisson residual of the N x N node grid (n = N - 1 intervals, h = 1/(N-1)).                      */
int homg_oracle_pow2_solve(int64_t N, int levels, const int *sched, int nsched, double omega_j, double div_factor,
                           const double *f, double *u, double tol, int max_cycles, double *hist, int *cycles_out,
                           double *relres_out) {
    const int K = pow2_exponent(N);
    if (K < 2 || levels < 1 || levels > K || max_cycles < 0) return HOMG_ORACLE_EINVAL;
    const int64_t n = N - 1, total = N * N;
    double fnorm = homg_oracle_norm_interior(2, n, f);
    if (fnorm == 0.0) {
        for (int64_t y = 1; y < n; ++y)
            for (int64_t x = 1; x < n; ++x) u[y * N + x] = 0.0;
        if (hist) hist[0] = 0.0;
        if (cycles_out) *cycles_out = 0;
        if (relres_out) *relres_out = 0.0;
        return HOMG_ORACLE_OK;
    }
    double *r = (double *)malloc((size_t)total * sizeof(double));
    double *e = (double *)malloc((size_t)total * sizeof(double));
    if (!r || !e) { free(r); free(e); return HOMG_ORACLE_ENOMEM; }
    int status = HOMG_ORACLE_NOT_CONVERGED, k;
    double rr = 0.0, rr0 = 0.0;
    for (k = 0;; ++k) {
        homg_oracle_residual(2, n, f, u, r);
        rr = homg_oracle_norm_interior(2, n, r) / fnorm;
        if (hist) hist[k] = rr;
        if (k == 0) rr0 = rr;
        if (rr <= tol) { status = HOMG_ORACLE_OK; break; }
        if (!isfinite(rr) || rr > div_factor * rr0) { status = HOMG_ORACLE_DIVERGED; break; }
        if (k == max_cycles) { status = HOMG_ORACLE_NOT_CONVERGED; break; }
        int rc = homg_oracle_pow2_cycle(N, levels, sched, nsched, omega_j, r, e);
        if (rc != HOMG_ORACLE_OK) { free(r); free(e); return rc; }
        for (int64_t y = 1; y < n; ++y)
            for (int64_t x = 1; x < n; ++x) u[y * N + x] = u[y * N + x] + e[y * N + x];
    }
    free(r); free(e);
    if (cycles_out) *cycles_out = k;
    if (relres_out) *relres_out = rr;
    return status;
}
