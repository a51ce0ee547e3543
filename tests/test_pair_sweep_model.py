"""A CPU model of k_jacobi2d and k_jacobi2d2 (and of k_jacobi3d in 3-D), the FP64 level iterations
with shared neighbour pairs, restated as the kernels run: blocks of four warps, each warp's 32 lanes
on adjacent columns with lane 0 on the column left of the warp's 31 output columns, lanes past the
last interior column clamped to it, each lane marching `rows` rows and taking the west + south pair
from the left lane's previous row (a shuffle up by one, lane 0 keeping its own value).

For every launch shape it checks:
- every load stays inside the (n+1)^2 array;
- every interior node is written exactly once;
- the result equals the pair formula v' = c1 v + om (D(i, j) + D(i-1, j-1)) + g, with
  D(i, j) = v(i+1, j) + v(i, j+1) formed from the array directly, bit for bit (exact fused
  multiply-adds), so the shuffle hands each lane the right pair;
- the result agrees with the damped-Jacobi update c1 v + om (w + e + s + n) + g to rounding.
The GPU tests check the kernel itself against the oracle.
"""

from fractions import Fraction

import numpy as np
import pytest

JX = 128  # threads per block
COLS = 31  # output columns per warp
COLS2 = 63  # the same, two columns per lane


def fma(a, b, c):
    """a * b + c rounded once to binary64."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


class Grid:
    def __init__(self, E, G, n):
        self.E, self.G, self.n = E, G, n
        self.O = np.zeros_like(E)
        self.written = np.zeros(E.shape, dtype=int)

    def ld(self, A, i, r):
        assert 0 <= i <= self.n and 0 <= r <= self.n, (i, r)
        return float(A[r, i])


def model(E, G, n, rows, om, c1):
    gr = Grid(E, G, n)
    per_block = JX // 32 * COLS
    for bx in range((n - 1 + per_block - 1) // per_block):
        for by in range((n - 1 + rows - 1) // rows):
            for w in range(JX // 32):
                i0 = (bx * (JX // 32) + w) * COLS
                if i0 + 1 > n - 1:
                    continue
                lanes = range(32)
                col = [min(i0 + l, n - 1) for l in lanes]
                out = [l > 0 and i0 + l <= n - 1 for l in lanes]
                j0 = by * rows + 1
                j1 = min(j0 + rows, n)
                vc = [gr.ld(E, col[l], j0) for l in lanes]
                dp = [fma(1.0, gr.ld(E, col[l] + 1, j0 - 1), vc[l]) for l in lanes]
                for j in range(j0, j1):
                    dw = [dp[l - 1] if l > 0 else dp[0] for l in lanes]  # shuffle up by one
                    for l in lanes:
                        i = col[l]
                        vn = gr.ld(E, i, j + 1)
                        e = gr.ld(E, i + 1, j)
                        g = gr.ld(G, i, j)
                        dh = fma(1.0, e, vn)
                        v = fma(om, dh, fma(om, dw[l], fma(c1, vc[l], g)))
                        if out[l]:
                            gr.O[j, i] = v
                            gr.written[j, i] += 1
                        dp[l] = dh
                        vc[l] = vn
    return gr


def model2(E, G, n, rows, om, c1):
    """k_jacobi2d2: two adjacent columns per lane, 63 output columns per warp."""
    gr = Grid(E, G, n)
    per_block = JX // 32 * COLS2
    for bx in range((n - 1 + per_block - 1) // per_block):
        for by in range((n - 1 + rows - 1) // rows):
            for w in range(JX // 32):
                i0 = (bx * (JX // 32) + w) * COLS2
                if i0 + 1 > n - 1:
                    continue
                lanes = range(32)
                cA = [i0 + 2 * l for l in lanes]
                cB = [c + 1 for c in cA]
                iA = [min(c, n) for c in cA]
                iB = [min(c, n) for c in cB]
                iE = [min(c + 1, n) for c in cB]
                outA = [l > 0 and cA[l] <= n - 1 for l in lanes]
                outB = [cB[l] <= n - 1 for l in lanes]
                j0 = by * rows + 1
                j1 = min(j0 + rows, n)
                vcA = [gr.ld(E, iA[l], j0) for l in lanes]
                vcB = [gr.ld(E, iB[l], j0) for l in lanes]
                dpA = [fma(1.0, gr.ld(E, iB[l], j0 - 1), vcA[l]) for l in lanes]
                dpB = [fma(1.0, gr.ld(E, iE[l], j0 - 1), vcB[l]) for l in lanes]
                for j in range(j0, j1):
                    dwA = [dpB[l - 1] if l > 0 else dpB[0] for l in lanes]  # shuffle up by one
                    for l in lanes:
                        vnA, vnB = gr.ld(E, iA[l], j + 1), gr.ld(E, iB[l], j + 1)
                        eB = gr.ld(E, iE[l], j)
                        gA, gB = gr.ld(G, iA[l], j), gr.ld(G, iB[l], j)
                        dhA, dhB = fma(1.0, vcB[l], vnA), fma(1.0, eB, vnB)
                        vA = fma(om, dhA, fma(om, dwA[l], fma(c1, vcA[l], gA)))
                        vB = fma(om, dhB, fma(om, dpA[l], fma(c1, vcB[l], gB)))
                        for out, c, v in ((outA[l], cA[l], vA), (outB[l], cB[l], vB)):
                            if out:
                                gr.O[j, c] = v
                                gr.written[j, c] += 1
                        dpA[l], dpB[l] = dhA, dhB
                        vcA[l], vcB[l] = vnA, vnB
    return gr


def pair_formula(E, G, n, om, c1):
    O = np.zeros_like(E)
    D = lambda i, j: fma(1.0, float(E[j, i + 1]), float(E[j + 1, i]))
    for j in range(1, n):
        for i in range(1, n):
            O[j, i] = fma(om, D(i, j), fma(om, D(i - 1, j - 1), fma(c1, float(E[j, i]), float(G[j, i]))))
    return O


@pytest.mark.parametrize("cols", [1, 2])
@pytest.mark.parametrize("n,rows", [(8, 3), (32, 32), (33, 7), (64, 16), (125, 16), (129, 40), (257, 64)])
def test_pair_sweep_geometry_and_values(n, rows, cols):
    rng = np.random.default_rng(n * 1000 + rows)
    E = rng.standard_normal((n + 1, n + 1))
    E[0, :] = E[n, :] = E[:, 0] = E[:, n] = 0.0
    G = rng.standard_normal((n + 1, n + 1))
    om, c1 = 0.2, 1.0 - 0.8
    gr = (model if cols == 1 else model2)(E, G, n, rows, om, c1)
    assert (gr.written[1:n, 1:n] == 1).all()
    assert gr.written.sum() == (n - 1) ** 2
    ref = pair_formula(E, G, n, om, c1)
    assert np.array_equal(gr.O[1:n, 1:n], ref[1:n, 1:n])
    jac = np.zeros_like(E)
    jac[1:n, 1:n] = c1 * E[1:n, 1:n] + om * (E[1:n, :n - 1] + E[1:n, 2:] + E[:n - 1, 1:n] + E[2:, 1:n]) + G[1:n, 1:n]
    assert np.max(np.abs(gr.O - jac)) <= 1e-14 * np.max(np.abs(jac))


def test_model_catches_a_wrong_shuffle():
    # the pair from the lane's own previous row instead of the left lane's gives other values
    n, rows = 40, 8
    rng = np.random.default_rng(5)
    E = rng.standard_normal((n + 1, n + 1))
    E[0, :] = E[n, :] = E[:, 0] = E[:, n] = 0.0
    G = rng.standard_normal((n + 1, n + 1))
    ref = pair_formula(E, G, n, 0.2, 0.2)
    wrong = np.zeros_like(E)
    for j in range(1, n):
        for i in range(1, n):
            own = fma(1.0, float(E[j - 1, i + 1]), float(E[j, i]))
            dh = fma(1.0, float(E[j, i + 1]), float(E[j + 1, i]))
            wrong[j, i] = fma(0.2, dh, fma(0.2, own, fma(0.2, float(E[j, i]), float(G[j, i]))))
    assert not np.array_equal(wrong[1:n, 1:n], ref[1:n, 1:n])


J3Y = 4  # thread rows of a 3-D block; each row of 32 lanes is one warp


def model3(E, G, n, rows, om, c1):
    """k_jacobi3d: the pair D(i, j, k) = v(i+1, j, k) + v(i, j, k+1) handed to the right lane at the
    next plane; arrays indexed [k, j, i]."""
    O = np.zeros_like(E)
    written = np.zeros(E.shape, dtype=int)

    def ld(A, i, j, k):
        assert 0 <= i <= n and 0 <= j <= n and 0 <= k <= n, (i, j, k)
        return float(A[k, j, i])

    for bx in range((n - 1 + COLS - 1) // COLS):
        if bx * COLS + 1 > n - 1:
            continue
        for by in range((n - 1 + J3Y - 1) // J3Y):
            for bz in range((n - 1 + rows - 1) // rows):
                for ty in range(J3Y):
                    j = by * J3Y + ty + 1
                    if j >= n:
                        continue
                    lanes = range(32)
                    col = [min(bx * COLS + l, n - 1) for l in lanes]
                    out = [l > 0 and bx * COLS + l <= n - 1 for l in lanes]
                    k0 = bz * rows + 1
                    k1 = min(k0 + rows, n)
                    vc = [ld(E, col[l], j, k0) for l in lanes]
                    dp = [fma(1.0, ld(E, col[l] + 1, j, k0 - 1), vc[l]) for l in lanes]
                    for k in range(k0, k1):
                        dw = [dp[l - 1] if l > 0 else dp[0] for l in lanes]
                        for l in lanes:
                            i = col[l]
                            vt = ld(E, i, j, k + 1)
                            e, sn, nn = ld(E, i + 1, j, k), ld(E, i, j - 1, k), ld(E, i, j + 1, k)
                            g = ld(G, i, j, k)
                            dh = fma(1.0, e, vt)
                            v = fma(om, dh, fma(om, dw[l], fma(om, fma(1.0, sn, nn), fma(c1, vc[l], g))))
                            if out[l]:
                                O[k, j, i] = v
                                written[k, j, i] += 1
                            dp[l] = dh
                            vc[l] = vt
    return O, written


@pytest.mark.parametrize("n,rows", [(4, 2), (16, 5), (33, 8)])
def test_pair_sweep_3d_geometry_and_values(n, rows):
    rng = np.random.default_rng(n + rows)
    E = rng.standard_normal((n + 1,) * 3)
    for ax in range(3):
        idx = [slice(None)] * 3
        for b in (0, n):
            idx[ax] = b
            E[tuple(idx)] = 0.0
    G = rng.standard_normal((n + 1,) * 3)
    om, c1 = 0.8 / 6, 1.0 - 0.8
    O, written = model3(E, G, n, rows, om, c1)
    inner = (slice(1, n),) * 3
    assert (written[inner] == 1).all() and written.sum() == (n - 1) ** 3
    ref = np.zeros_like(E)
    for k in range(1, n):
        for j in range(1, n):
            for i in range(1, n):
                dh = fma(1.0, float(E[k, j, i + 1]), float(E[k + 1, j, i]))
                dw = fma(1.0, float(E[k - 1, j, i]), float(E[k, j, i - 1]))
                sn = fma(1.0, float(E[k, j - 1, i]), float(E[k, j + 1, i]))
                ref[k, j, i] = fma(om, dh, fma(om, dw, fma(om, sn, fma(c1, float(E[k, j, i]), float(G[k, j, i])))))
    assert np.array_equal(O[inner], ref[inner])
    jac = c1 * E[inner] + om * (E[1:n, 1:n, :n - 1] + E[1:n, 1:n, 2:] + E[1:n, :n - 1, 1:n] + E[1:n, 2:, 1:n]
                                + E[:n - 1, 1:n, 1:n] + E[2:, 1:n, 1:n]) + G[inner]
    assert np.max(np.abs(O[inner] - jac)) <= 1e-14 * np.max(np.abs(jac))
