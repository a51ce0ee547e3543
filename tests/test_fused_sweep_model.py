"""A CPU model of the fused-sweep kernels' launch geometry: k_jacobi2_x2 (two sweeps) and
k_jacobi2_xk (K sweeps), restated step by step as the kernels march. The model covers warp strips
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


class PaddedGrid(Grid):
    """Rows padded to a multiple of 16 elements, as the level buffer lays them out: aligned vector
    groups may read the padding (never past it), which holds arbitrary values."""

    def __init__(self, E, G, n, rng):
        super().__init__(E, G, n)
        self.pitch = (n + 1 + 15) // 16 * 16
        pad = lambda A: np.concatenate([A, rng.standard_normal((n + 1, self.pitch - n - 1)).astype(np.float32) * 1e3], 1)  # noqa: E731
        self.Ep, self.Gp = pad(E), pad(G)

    def vld(self, A, c0, r, V):
        assert c0 % V == 0 and 0 <= c0 and c0 + V - 1 <= self.pitch - 1 and 0 <= r <= self.n, (c0, r)
        return [A[r, c0 + k] for k in range(V)]


def model_x2v(grid, om, c1, rows, V):
    """k_jacobi2_x2v: V columns per lane loaded as one aligned group, W output columns per strip."""
    n = grid.n
    W = V * (31 - (V + 2) // V)
    xb = (((n - 1 + W - 1) // W) + JX // 32 - 1) // (JX // 32)
    zero = np.float32(0)
    for by in range((n - 1 + rows - 1) // rows):
        j0 = by * rows + 1
        j1 = min(j0 + rows, n)
        r0, ra, rb = j0 - 1, max(j0 - 1, 1), min(j1, n - 1)
        for strip in range(xb * (JX // 32)):
            base = strip * W
            if base + 1 > n - 1:
                continue
            lanes = []
            for lane in range(32):
                c0 = base - V + V * lane
                cols = [c0 + k for k in range(V)]
                d = dict(c0=c0, grp=0 <= c0 <= n, ein=[0 <= c <= n for c in cols], inn=[1 <= c <= n - 1 for c in cols],
                         out=[1 <= c <= n - 1 and base + 1 <= c <= base + W for c in cols], r=ra, ro=j0)
                d["full"] = all(d["out"])
                lanes.append(d)

            def row(d, A, r):
                x = grid.vld(A, d["c0"], r, V) if d["grp"] else [zero] * V
                return [x[k] if (d["grp"] and d["ein"][k]) else zero for k in range(V)]

            for d in lanes:
                d["em"], d["ec"] = row(d, grid.Ep, d["r"] - 1), row(d, grid.Ep, d["r"])
                d["sp"] = d["sc"] = d["gc"] = [zero] * V

            def first():
                res = []
                left = [lanes[l - 1]["ec"][V - 1] if l > 0 else lanes[l]["ec"][V - 1] for l in range(32)]
                right = [lanes[l + 1]["ec"][0] if l < 31 else lanes[l]["ec"][0] for l in range(32)]
                for l, d in enumerate(lanes):
                    r = d["r"]
                    assert 1 <= r <= n - 1
                    ep, g = row(d, grid.Ep, r + 1), row(d, grid.Gp, r)
                    v = []
                    for k in range(V):
                        w = d["ec"][k - 1] if k > 0 else left[l]
                        e = d["ec"][k + 1] if k < V - 1 else right[l]
                        s = np.float32(np.float32(w + e) + np.float32(d["em"][k] + ep[k]))
                        y = step32(c1, d["ec"][k], om, s, g[k])
                        v.append(y if d["inn"][k] else zero)
                    d["em"], d["ec"], d["r"] = d["ec"], ep, r + 1
                    res.append((v, g))
                return res

            def second(vs):
                left = [lanes[l - 1]["sc"][V - 1] if l > 0 else lanes[l]["sc"][V - 1] for l in range(32)]
                right = [lanes[l + 1]["sc"][0] if l < 31 else lanes[l]["sc"][0] for l in range(32)]
                for l, d in enumerate(lanes):
                    for k in range(V):
                        sw = d["sc"][k - 1] if k > 0 else left[l]
                        se = d["sc"][k + 1] if k < V - 1 else right[l]
                        s = np.float32(np.float32(sw + se) + np.float32(d["sp"][k] + vs[l][k]))
                        o = step32(c1, d["sc"][k], om, s, d["gc"][k])
                        if d["full"] or d["out"][k]:
                            assert d["out"][k] and d["c0"] % V == 0
                            grid.store(d["c0"] + k, d["ro"], o)
                    d["ro"] += 1

            if r0 >= 1:
                for d, (v, _) in zip(lanes, first()):
                    d["sc"] = v
            for d, (v, g) in zip(lanes, first()):
                d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            for _ in range(j0 + 1, rb + 1):
                res = first()
                second([v for v, _ in res])
                for d, (v, g) in zip(lanes, res):
                    d["sp"], d["sc"], d["gc"] = d["sc"], v, g
            if j1 == n:
                second([[zero] * V] * 32)


@pytest.mark.parametrize("V", [2, 4, 8])
@pytest.mark.parametrize("n,rows", [(2, 1), (3, 1), (8, 3), (17, 8), (31, 4), (64, 63), (127, 8), (130, 16), (260, 5), (512, 16)])
def test_vector_pair_model_equals_two_sweeps(n, rows, V):
    E, G = problem(n, 200 + n)
    grid = PaddedGrid(E, G, n, np.random.default_rng(n))
    model_x2v(grid, OM, C1, rows, V)
    grid.check_coverage()
    want = plain_sweep(plain_sweep(E, G, OM, C1, n), G, OM, C1, n)
    assert np.array_equal(grid.O[1:n, 1:n], want[1:n, 1:n])
