"""CPU model of the convolution kernel's tile walk and staged-row ring (k_conv3x3 in
paper_1108_2045_gb300/csrc/homg_net.cu), run without a GPU.

Each CTA walks a contiguous chunk of tiles in column-major order (image, tile column, tile row).
Input row y (-1 .. H) of the current column sits in ring slot (y + 1) mod (2R + 2). A tile that
continues its column gets its R new rows loaded at the start of the previous tile; a tile that starts
a column is loaded whole once the previous tile's products have completed. The model replays that
schedule slot by slot and checks that every tile reads exactly its input rows, that no copy
overwrites a slot a tile still has to read, and that every tile is computed once.
"""

import pytest


def ceil_div(a, b):
    return -(-a // b)


def replay(B, H, W, R, grid, TW=128, nring=None):
    nring = nring or 2 * R + 2
    tx, ty = ceil_div(W, TW), ceil_div(H, R)
    tiles = B * ty * tx
    chunk = ceil_div(tiles, grid)
    seen = []
    for cta in range(grid):
        u0, u1 = cta * chunk, min(cta * chunk + chunk, tiles)
        ring = [None] * nring  # (column, row) held by each slot
        busy = set()           # slots the tile being computed still reads

        def coords(u):
            return u // ty, u % ty  # (column id, tile row)

        def load(u, ya, yb):
            col, _ = coords(u)
            for y in range(ya, yb + 1):
                slot = (y + 1) % nring
                assert slot not in busy, ("copy into a slot still being read", cta, u, y)
                ring[slot] = (col, y)

        if u0 < u1:
            _, yt = coords(u0)
            load(u0, yt * R - 1, yt * R + R)
        for u in range(u0, u1):
            col, yt = coords(u)
            y0 = yt * R
            nxt = u + 1 < u1
            cont = nxt and coords(u + 1)[0] == col
            need = {(y0 + rho) % nring for rho in range(R + 2)}
            if cont:  # issued before this tile's products start
                busy = need
                load(u + 1, y0 + R + 1, y0 + 2 * R)
            for rho in range(R + 2):
                assert ring[(y0 + rho) % nring] == (col, y0 - 1 + rho), (cta, u, rho)
            busy = set()  # products completed
            if nxt and not cont:
                _, yt1 = coords(u + 1)
                load(u + 1, yt1 * R - 1, yt1 * R + R)
            seen.append(u)
    assert sorted(seen) == list(range(tiles))
    return tiles


@pytest.mark.parametrize("R", [4, 8])
@pytest.mark.parametrize("B,H,W,grid", [(1, 2049, 2049, 304), (1, 2049, 2049, 152), (3, 64, 64, 304),
                                        (2, 37, 150, 5), (1, 16, 16, 4), (64, 64, 64, 304), (1, 9, 7, 1),
                                        (5, 130, 300, 7)])
def test_ring_schedule(B, H, W, R, grid):
    tiles = replay(B, H, W, R, grid=min(grid, B * ceil_div(H, R) * ceil_div(W, 128)))
    assert tiles >= 1


@pytest.mark.parametrize("R", [4, 8])
def test_model_catches_a_short_ring(R):
    # with one slot fewer the early copy overwrites a row the current tile still reads
    with pytest.raises(AssertionError, match="still being read"):
        replay(1, 64, 64, R, grid=1, nring=2 * R + 1)
