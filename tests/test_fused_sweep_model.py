"""A CPU model of the fused-sweep kernels' launch geometry: k_jacobi2_x2 (two sweeps),
k_jacobi2_x2p (two sweeps, two columns per lane) and k_jacobi2_xk (K sweeps), restated step by step
as the kernels march. The model covers warp strips
of 32 lanes with 30 (34 - 2K) owning lanes, blocks of four strips, clamped load columns and rows,
the peeled boundary rows, and the register windows and shuffles.

For every launch shape it checks three things:
- every load stays inside the (n+1)^2 array;
- every interior node is written exactly once;
- the result equals K plain damped-Jacobi sweeps bit for bit.

The arithmetic is binary32 with one helper standing in for the kernels' fused multiply-adds, used
alike by the plain sweeps and the fused model. The GPU tests check the kernels themselves
against the oracle, and batch results (four-sweep launches) bit for bit against single solves
(two-sweep launches).
"""

import numpy as np
import pytest

JX = 128  # threads per block: four warp strips


def fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def step32(c1, vc, om, s, g):
    """v' = fma(c1, vc, fma(om, s, g)) in binary32."""
    return fma32(c1, vc, fma32(om, s, g))


def plain_sweep(E, G, om, c1, n):
    O = np.zeros_like(E)
    for j in range(1, n):
        for i in range(1, n):
            s = np.float32(np.float32(E[j, i - 1] + E[j, i + 1]) + np.float32(E[j - 1, i] + E[j + 1, i]))
            O[j, i] = step32(c1, E[j, i], om, s, G[j, i])
    return O


class Grid:
    """The (n+1)^2 arrays with bounds-checked reads and a write counter."""

    def __init__(self, E, G, n):
        self.E, self.G, self.n = E, G, n
        self.O = np.zeros_like(E)
        self.written = np.zeros(E.shape, dtype=int)

    def ld(self, A, i, r):
        assert 0 <= i <= self.n and 0 <= r <= self.n, (i, r)
        return A[r, i]

    def store(self, i, r, v):
        self.O[r, i] = v
        self.written[r, i] += 1

    def check_coverage(self):
        n = self.n
        assert (self.written[1:n, 1:n] == 1).all()
        assert self.written.sum() == (n - 1) ** 2


def shuffles(vals):
    """__shfl_up_sync / __shfl_down_sync by 1 over a warp (lane 0 / 31 keep their own value)."""
    up = [vals[l - 1] if l > 0 else vals[l] for l in range(32)]
    down = [vals[l + 1] if l < 31 else vals[l] for l in range(32)]
    return up, down


def model_x2(grid, om, c1, rows):
    """k_jacobi2_x2: first sweep one row ahead on 32 columns, second sweep on the 30 inner ones."""
    n, E, G = grid.n, grid.E, grid.G
    out_cols = 30
    xb = (((n - 1 + out_cols - 1) // out_cols) + JX // 32 - 1) // (JX // 32)
    for by in range((n - 1 + rows - 1) // rows):
        j0 = by * rows + 1
        j1 = min(j0 + rows, n)
        r0, ra, rb = j0 - 1, max(j0 - 1, 1), min(j1, n - 1)
        for strip in range(xb * (JX // 32)):
            if strip * out_cols + 1 > n - 1:
                continue  # the whole warp leaves
            lanes = []
            for lane in range(32):
                i = strip * out_cols + lane
                col_in = 1 <= i <= n - 1
                il = min(max(i, 1), n - 1)
                lanes.append(dict(i=i, il=il, col_in=col_in, out=col_in and 1 <= lane <= out_cols, r=ra, ro=j0,
                                  em=grid.ld(E, il, ra - 1), ec=grid.ld(E, il, ra), sp=0.0, sc=0.0, gc=0.0))

            def first(d):
                r, il = d["r"], d["il"]
                assert 1 <= r <= n - 1
                ep = grid.ld(E, il, r + 1)
                s = np.float32(np.float32(grid.ld(E, il - 1, r) + grid.ld(E, il + 1, r)) + np.float32(d["em"] + ep))
                g = grid.ld(G, il, r)
                v = step32(c1, d["ec"], om, s, g)
                d["em"], d["ec"], d["r"] = d["ec"], ep, r + 1
                return (v if d["col_in"] else np.float32(0)), g

            def second(vs):
                up, down = shuffles([d["sc"] for d in lanes])
                for lane, d in enumerate(lanes):
                    if d["out"]:
                        s = np.float32(np.float32(up[lane] + down[lane]) + np.float32(d["sp"] + vs[lane]))
                        grid.store(d["i"], d["ro"], step32(c1, d["sc"], om, s, d["gc"]))
                    d["ro"] += 1

            if r0 >= 1:
                for d in lanes:
                    d["sc"], d["gc"] = first(d)
            for d in lanes:
                v, g = first(d)
                d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            for _ in range(j0 + 1, rb + 1):
                res = [first(d) for d in lanes]
                second([v for v, _ in res])
                for d, (v, g) in zip(lanes, res):
                    d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            if j1 == n:
                second([np.float32(0)] * 32)


def model_x2p(E, G, om, c1, n, rows, pitch):
    """k_jacobi2_x2p: two sweeps with two adjacent columns per lane (one aligned pair load per row of
    e and of g, packed binary32 arithmetic). Lane L of strip s holds columns c0, c0 + 1 with
    c0 = 60 s - 2 + 2 L; the pair is loaded from column min(max(c0, 0), n rounded down to even),
    which may reach the row's padding (column n + 1 < pitch). The first sweep runs on both columns
    of every lane, side neighbours from the lane's own pair or the adjacent lane's (shuffle);
    lanes 1..30 store the second sweep (60 columns). E and G are (n+1) x pitch arrays whose
    padding holds NaN, so that a padding value reaching an unmasked result shows. Returns the
    output and the write counts."""
    O = np.zeros_like(E)
    written = np.zeros(E.shape, dtype=int)
    zero = np.float32(0)
    ne = n & ~1

    def ld2(A, c, r):
        assert c % 2 == 0 and 0 <= c and c + 1 <= pitch - 1 and 0 <= r <= n, (c, r)
        return [A[r, c], A[r, c + 1]]

    strips = (n + 59) // 60
    xb = (strips + JX // 32 - 1) // (JX // 32)
    for by in range((n - 1 + rows - 1) // rows):
        j0 = by * rows + 1
        j1 = min(j0 + rows, n)
        r0, ra, rb = j0 - 1, max(j0 - 1, 1), min(j1, n - 1)
        for strip in range(xb * (JX // 32)):
            if 60 * strip > n - 1:
                continue  # the whole warp leaves
            lanes = []
            for lane in range(32):
                c0 = 60 * strip - 2 + 2 * lane
                cl = min(max(c0, 0), ne)
                m = [1 <= c0 + k <= n - 1 for k in range(2)]
                o = [m[k] and 1 <= lane <= 30 for k in range(2)]
                lanes.append(dict(c0=c0, cl=cl, m=m, o=o, r=ra, ro=j0, em=ld2(E, cl, ra - 1), ec=ld2(E, cl, ra),
                                  sp=[zero, zero], sc=[zero, zero], gc=[zero, zero]))

            def first_all():
                left = [d["ec"][1] for d in lanes]
                right = [d["ec"][0] for d in lanes]
                up, _ = shuffles(left)
                _, down = shuffles(right)
                res = []
                for lane, d in enumerate(lanes):
                    r = d["r"]
                    assert 1 <= r <= n - 1
                    ep = ld2(E, d["cl"], r + 1)
                    g = ld2(G, d["cl"], r)
                    ec, em = d["ec"], d["em"]
                    w = [up[lane], ec[0]]
                    e = [ec[1], down[lane]]
                    v = []
                    for k in range(2):
                        s = np.float32(np.float32(w[k] + e[k]) + np.float32(em[k] + ep[k]))
                        y = step32(c1, ec[k], om, s, g[k])
                        v.append(y if d["m"][k] else zero)
                    d["em"], d["ec"], d["r"] = ec, ep, r + 1
                    res.append((v, g))
                return res

            def second(vs):
                up, _ = shuffles([d["sc"][1] for d in lanes])
                _, down = shuffles([d["sc"][0] for d in lanes])
                for lane, d in enumerate(lanes):
                    sc = d["sc"]
                    sw = [up[lane], sc[0]]
                    se = [sc[1], down[lane]]
                    for k in range(2):
                        s = np.float32(np.float32(sw[k] + se[k]) + np.float32(d["sp"][k] + vs[lane][k]))
                        y = step32(c1, sc[k], om, s, d["gc"][k])
                        if d["o"][k]:
                            O[d["ro"], d["c0"] + k] = y
                            written[d["ro"], d["c0"] + k] += 1
                    d["ro"] += 1

            if r0 >= 1:
                for d, (v, g) in zip(lanes, first_all()):
                    d["sc"], d["gc"] = v, g
            for d, (v, g) in zip(lanes, first_all()):
                d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            for _ in range(j0 + 1, rb + 1):
                res = first_all()
                second([v for v, _ in res])
                for d, (v, g) in zip(lanes, res):
                    d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            if j1 == n:
                second([[zero, zero]] * 32)
    return O, written


def model_xk(grid, om, c1, rows, K):
    """k_jacobi2_xk<K>: sweep l at row r - l + 1 in step r, loads from rows clamped into 0..n, sweep
    values outside rows/columns 1..n-1 replaced by 0, the 34 - 2K inner lanes storing sweep K."""
    n, E, G = grid.n, grid.E, grid.G
    out_cols = 34 - 2 * K
    xb = (((n - 1 + out_cols - 1) // out_cols) + JX // 32 - 1) // (JX // 32)
    clamp = lambda row: min(max(row, 0), n)  # noqa: E731
    zero = np.float32(0)
    for by in range((n - 1 + rows - 1) // rows):
        j0 = by * rows + 1
        j1 = min(j0 + rows, n)
        rf, rl = j0 - (K - 1), j1 + K - 2
        for strip in range(xb * (JX // 32)):
            if strip * out_cols + 1 > n - 1:
                continue
            lanes = []
            for lane in range(32):
                i = strip * out_cols + lane - (K - 2)
                col_in = 1 <= i <= n - 1
                il = min(max(i, 1), n - 1)
                lanes.append(dict(i=i, il=il, col_in=col_in, out=col_in and K - 1 <= lane <= 32 - K,
                                  em=grid.ld(E, il, clamp(rf - 1)), ec=grid.ld(E, il, clamp(rf)),
                                  sp=[zero] * K, sc=[zero] * K, gq=[zero] * K))
            for r in range(rf, rl + 1):
                for d in lanes:
                    il = d["il"]
                    ep = grid.ld(E, il, clamp(r + 1))
                    s = np.float32(np.float32(grid.ld(E, il - 1, clamp(r)) + grid.ld(E, il + 1, clamp(r)))
                                   + np.float32(d["em"] + ep))
                    g = grid.ld(G, il, clamp(r))
                    y = step32(c1, d["ec"], om, s, g)
                    d["v"] = [None, y if (d["col_in"] and 1 <= r <= n - 1) else zero] + [None] * (K - 1)
                    d["em"], d["ec"] = d["ec"], ep
                    d["gq"] = [g] + d["gq"][:-1]
                for level in range(2, K + 1):
                    x = r - level + 1
                    up, down = shuffles([d["sc"][level - 1] for d in lanes])
                    for lane, d in enumerate(lanes):
                        s = np.float32(np.float32(up[lane] + down[lane]) + np.float32(d["sp"][level - 1] + d["v"][level - 1]))
                        y = step32(c1, d["sc"][level - 1], om, s, d["gq"][level - 1])
                        d["v"][level] = zero
                        if level < K:
                            d["v"][level] = y if (d["col_in"] and 1 <= x <= n - 1) else zero
                        elif d["out"] and j0 <= x < j1:
                            grid.store(d["i"], x, y)
                        d["sp"][level - 1] = d["sc"][level - 1]
                        d["sc"][level - 1] = d["v"][level - 1]


def problem(n, seed):
    rng = np.random.default_rng(seed)
    E = np.zeros((n + 1, n + 1), np.float32)
    G = np.zeros_like(E)
    E[1:n, 1:n] = rng.standard_normal((n - 1, n - 1))
    G[1:n, 1:n] = rng.standard_normal((n - 1, n - 1))
    return E, G


OM, C1 = np.float32(0.2), np.float32(0.2)  # fast-form scalars for omega_J = 4/5 in 2-D


@pytest.mark.parametrize("n,rows", [(2, 1), (3, 1), (17, 8), (31, 4), (32, 16), (64, 63), (127, 8), (130, 16), (260, 5)])
def test_two_sweep_model_equals_two_sweeps(n, rows):
    E, G = problem(n, n)
    grid = Grid(E, G, n)
    model_x2(grid, OM, C1, rows)
    grid.check_coverage()
    want = plain_sweep(plain_sweep(E, G, OM, C1, n), G, OM, C1, n)
    assert np.array_equal(grid.O[1:n, 1:n], want[1:n, 1:n])


@pytest.mark.parametrize("n,rows", [(2, 1), (3, 1), (4, 2), (17, 8), (32, 16), (60, 4), (61, 7), (64, 63),
                                    (120, 16), (128, 16), (130, 5), (256, 16)])
def test_packed_pair_model_equals_two_sweeps(n, rows):
    pitch = -(-(n + 1) // 16) * 16
    E, G = problem(n, 200 + n)
    Ep = np.full((n + 1, pitch), np.nan, np.float32)
    Gp = np.full((n + 1, pitch), np.nan, np.float32)
    Ep[:, :n + 1], Gp[:, :n + 1] = E, G
    O, written = model_x2p(Ep, Gp, OM, C1, n, rows, pitch)
    assert (written[1:n, 1:n] == 1).all() and written.sum() == (n - 1) ** 2
    want = plain_sweep(plain_sweep(E, G, OM, C1, n), G, OM, C1, n)
    assert np.array_equal(O[1:n, 1:n], want[1:n, 1:n])


@pytest.mark.parametrize("K", [3, 4])
@pytest.mark.parametrize("n,rows", [(2, 1), (5, 2), (17, 8), (31, 4), (64, 63), (130, 16)])
def test_k_sweep_model_equals_k_sweeps(n, rows, K):
    E, G = problem(n, 100 + n)
    grid = Grid(E, G, n)
    model_xk(grid, OM, C1, rows, K)
    grid.check_coverage()
    want = E
    for _ in range(K):
        want = plain_sweep(want, G, OM, C1, n)
    assert np.array_equal(grid.O[1:n, 1:n], want[1:n, 1:n])


J3X, J3Y2 = 32, 16  # threads of the 3-D pair kernel: a warp along x, J3Y2 warps along y


def plain_sweep3(E, G, om, c1, n):
    O = np.zeros_like(E)
    for k in range(1, n):
        for j in range(1, n):
            for i in range(1, n):
                s = np.float32(np.float32(np.float32(E[k, j, i - 1] + E[k, j, i + 1]) + np.float32(E[k, j - 1, i] + E[k, j + 1, i]))
                               + np.float32(E[k - 1, j, i] + E[k + 1, j, i]))
                O[k, j, i] = step32(c1, E[k, j, i], om, s, G[k, j, i])
    return O


def model_x2_3d(E, G, om, c1, n, rows):
    """k_jacobi3_x2: tiles of 32 x J3Y2 columns marching down z, the first sweep on every thread, the
    second on the inner (32 - 2) x (J3Y2 - 2), x neighbours by shuffle, y neighbours from the
    previous step's plane in (triple-buffered) shared memory. Returns the output and write counts."""
    O = np.zeros_like(E)
    written = np.zeros(E.shape, dtype=int)
    zero = np.float32(0)

    def ld(A, k, j, i):
        assert 0 <= i <= n and 0 <= j <= n and 0 <= k <= n, (k, j, i)
        return A[k, j, i]

    gx, gy, gz = (n - 1 + J3X - 3) // (J3X - 2), (n - 1 + J3Y2 - 3) // (J3Y2 - 2), (n - 1 + rows - 1) // rows
    for bz in range(gz):
        k0 = bz * rows + 1
        k1 = min(k0 + rows, n)
        r0 = k0 - 1
        ra, rb = max(r0, 1), min(k1, n - 1)
        for by in range(gy):
            for bx in range(gx):
                th = {}
                for ty in range(J3Y2):
                    for tx in range(J3X):
                        i, j = bx * (J3X - 2) + tx, by * (J3Y2 - 2) + ty
                        col_in = 1 <= i <= n - 1 and 1 <= j <= n - 1
                        il, jl = min(max(i, 1), n - 1), min(max(j, 1), n - 1)
                        th[ty, tx] = dict(i=i, j=j, il=il, jl=jl, col_in=col_in,
                                          out=col_in and 1 <= tx <= J3X - 2 and 1 <= ty <= J3Y2 - 2,
                                          em=ld(E, ra - 1, jl, il), ec=ld(E, ra, jl, il), sp=zero, sc=zero, gc=zero)
                pl = {}

                def first(d, r):
                    il, jl = d["il"], d["jl"]
                    assert 1 <= r <= n - 1
                    ep = ld(E, r + 1, jl, il)
                    s = np.float32(np.float32(np.float32(ld(E, r, jl, il - 1) + ld(E, r, jl, il + 1))
                                              + np.float32(ld(E, r, jl - 1, il) + ld(E, r, jl + 1, il))) + np.float32(d["em"] + ep))
                    g = ld(G, r, jl, il)
                    y = step32(c1, d["ec"], om, s, g)
                    d["em"], d["ec"] = d["ec"], ep
                    return (y if d["col_in"] else zero), g

                def second(x, vs):
                    for ty in range(J3Y2):
                        for tx in range(J3X):
                            d = th[ty, tx]
                            sw = th[ty, tx - 1]["sc"] if tx > 0 else d["sc"]
                            se = th[ty, tx + 1]["sc"] if tx < J3X - 1 else d["sc"]
                            if d["out"]:
                                ss, sn = pl[x % 3][ty - 1, tx], pl[x % 3][ty + 1, tx]
                                s = np.float32(np.float32(np.float32(sw + se) + np.float32(ss + sn)) + np.float32(d["sp"] + vs[ty, tx]))
                                O[x, d["j"], d["i"]] = step32(c1, d["sc"], om, s, d["gc"])
                                written[x, d["j"], d["i"]] += 1

                if r0 >= 1:
                    for d in th.values():
                        d["sc"], _ = first(d, r0)
                pl[k0 % 3] = {}
                for key, d in th.items():
                    v, g = first(d, k0)
                    pl[k0 % 3][key] = v
                    d["sp"], d["sc"], d["gc"] = d["sc"], v, g
                for r in range(k0 + 1, rb + 1):
                    res = {key: first(d, r) for key, d in th.items()}
                    pl[r % 3] = {key: v for key, (v, _) in res.items()}
                    second(r - 1, {key: v for key, (v, _) in res.items()})
                    for key, (v, g) in res.items():
                        d = th[key]
                        d["sp"], d["sc"], d["gc"] = d["sc"], v, g
                if k1 == n:
                    second(n - 1, {key: zero for key in th})
    return O, written


@pytest.mark.parametrize("n,rows", [(2, 1), (3, 1), (5, 2), (9, 8), (17, 4), (18, 32), (33, 8)])
def test_3d_pair_model_equals_two_sweeps(n, rows):
    rng = np.random.default_rng(300 + n)
    E = np.zeros((n + 1,) * 3, np.float32)
    G = np.zeros_like(E)
    E[1:n, 1:n, 1:n] = rng.standard_normal((n - 1,) * 3)
    G[1:n, 1:n, 1:n] = rng.standard_normal((n - 1,) * 3)
    O, written = model_x2_3d(E, G, OM, C1, n, rows)
    assert (written[1:n, 1:n, 1:n] == 1).all() and written.sum() == (n - 1) ** 3
    want = plain_sweep3(plain_sweep3(E, G, OM, C1, n), G, OM, C1, n)
    assert np.array_equal(O[1:n, 1:n, 1:n], want[1:n, 1:n, 1:n])
