"""Bookkeeping of the D3Q19 collision pass's next density (host-side check of
the rules k_coll3d implements; no GPU).

The pass collides tiles of 32 columns x bands of 11 rows (ColTiles,
RowBands) and gathers the next density of a node from the populations pushed
into it (Eq. 1: f_i(x + e_i) <- f*_i(x)).  A population reaches its target by
one of five channels: the target's own gather (same tile and band), the sum
for the row beyond a band edge (oacc), the sum for the column beyond a tile
edge (cacc), or the single in-plane diagonal leaving a tile corner.  The
z-direction never crosses a tile (the pass recomputes one plane at each end
of a z-chunk), so the x-y projection of the nine in-plane directions decides
everything.  This test restates the kernel's channel conditions and checks,
over many lattice shapes:

* every (source node, direction) is carried by exactly one channel;
* a node that is not a tile corner receives from at most two (channel, CTA)
  groups, so two float additions onto zero complete it in any order;
* the kernel's choice between a float addition and a fixed-point corner
  accumulator agrees with the geometry, and the corner index it writes names
  the target node.
"""
import itertools
from collections import defaultdict

import pytest


def col_starts(nx):
    """ColTiles: 32-column tiles; a last tile of one column joins the one before."""
    nt = (nx + 31) // 32
    adj = 1 if nt >= 2 and nx - (nt - 1) * 32 == 1 else 0
    return [32 * t - (adj if t == nt - 1 else 0) for t in range(nt)] + [nx]


def row_starts(ny, ry=11):
    """RowBands: bands of 11 rows; a last band of one row joins the one before."""
    nb = (ny + ry - 1) // ry
    adj = 1 if nb >= 2 and ny - (nb - 1) * ry == 1 else 0
    return [b * ry - (adj if b == nb - 1 else 0) for b in range(nb)] + [ny]


DIRS = [(ex, ey) for ex in (-1, 0, 1) for ey in (-1, 0, 1)]


def channels(lx, ly, vw, vh, ex, ey):
    """The channels that carry the population (ex, ey) of the node at
    (lx, ly) of a vw x vh tile, by the kernel's conditions."""
    L, R, T, B = lx == 0, lx == vw - 1, ly == 0, ly == vh - 1
    tx, ty = lx + ex, ly + ey
    out = []

    def excluded_x(tx_):  # the target lane skips what comes across a tile edge
        return (ex > 0 and tx_ == 0) or (ex < 0 and tx_ == vw - 1)

    if ey == 0:
        if ex == 0 or (0 <= tx < vw and not excluded_x(tx)):
            out.append("own")  # register or warp shuffle
        if (ex < 0 and L) or (ex > 0 and R):
            out.append("col")  # edge column, row mover
    elif not ((ey < 0 and T) or (ey > 0 and B)):
        # stored in the staged plane
        tT, tB = ty == 0, ty == vh - 1
        from_band_beyond = (ey > 0 and tT) or (ey < 0 and tB)
        if 0 <= tx < vw and not excluded_x(tx) and not from_band_beyond:
            out.append("own")
        if ((ex < 0 and L) or (ex > 0 and R)) and not from_band_beyond:
            out.append("col")  # edge column, diagonal from the rows above / below
    else:
        # leaving the band
        if 0 <= tx < vw and not excluded_x(tx):
            out.append("row")
        if (ex < 0 and L) or (ex > 0 and R):
            out.append("diag")
    return out


def corner_node(xs, ys, t, b, c):
    return (xs[t + 1] - 1 if c & 1 else xs[t], ys[b + 1] - 1 if c & 2 else ys[b])


SHAPES = [(nx, ny) for nx in list(range(8, 41)) + [63, 64, 65, 66, 68, 96, 97]
          for ny in list(range(8, 25)) + [33, 34, 45]] + [(256, 256), (192, 192), (33, 256)]


@pytest.mark.parametrize("nx,ny", SHAPES[::7] + [(256, 256), (192, 192), (65, 23), (33, 20)])
def test_every_population_reaches_its_target_once(nx, ny):
    xs, ys = col_starts(nx), row_starts(ny)
    ntx, nb = len(xs) - 1, len(ys) - 1
    recv = defaultdict(list)
    corners = set()
    for t, b in itertools.product(range(ntx), range(nb)):
        x0, vw, y0, vh = xs[t], xs[t + 1] - xs[t], ys[b], ys[b + 1] - ys[b]
        assert vw >= 2 and vh >= 2
        for c in range(4):
            corners.add(corner_node(xs, ys, t, b, c))
        for lx, ly in itertools.product(range(vw), range(vh)):
            for ex, ey in DIRS:
                ch = channels(lx, ly, vw, vh, ex, ey)
                assert len(ch) == 1, (nx, ny, t, b, lx, ly, ex, ey, ch)
                recv[((x0 + lx + ex) % nx, (y0 + ly + ey) % ny)].append((ch[0], (t, b)))
    assert len(recv) == nx * ny
    for node, lst in recv.items():
        assert len(lst) == 9
        groups = set(lst)
        assert len(groups) <= (4 if node in corners else 2), (node, groups)


@pytest.mark.parametrize("nx,ny", [(8, 8), (33, 20), (40, 11), (65, 23), (68, 45), (256, 256)])
def test_float_or_fixed_point_and_corner_indices(nx, ny):
    xs, ys = col_starts(nx), row_starts(ny)
    ntx, nb = len(xs) - 1, len(ys) - 1
    corners = {corner_node(xs, ys, t, b, c) for t in range(ntx) for b in range(nb) for c in range(4)}
    for t, b in itertools.product(range(ntx), range(nb)):
        x0, vw, y0, vh = xs[t], xs[t + 1] - xs[t], ys[b], ys[b + 1] - ys[b]
        tm, tp, bm, bp = (t - 1) % ntx, (t + 1) % ntx, (b - 1) % nb, (b + 1) % nb
        for lx, ly in itertools.product(range(vw), range(vh)):
            L, R, T, B = lx == 0, lx == vw - 1, ly == 0, ly == vh - 1
            node = (x0 + lx, y0 + ly)
            assert (node in corners) == ((L or R) and (T or B))
            if (L or R) and (T or B):  # own partial sum of a corner
                assert corner_node(xs, ys, t, b, (1 if R else 0) | (2 if B else 0)) == node
            if T or B:  # row beyond the band edge
                tgt = (x0 + lx, (y0 - 1) % ny if T else (y0 + vh) % ny)
                assert (tgt in corners) == (L or R)
                if L or R:
                    assert corner_node(xs, ys, t, bm if T else bp, (2 if T else 0) | (1 if R else 0)) == tgt
            if L or R:  # column beyond the tile edge
                tgt = ((x0 - 1) % nx if L else (x0 + vw) % nx, y0 + ly)
                assert (tgt in corners) == (T or B)
                if T or B:
                    assert corner_node(xs, ys, tm if L else tp, b, (1 if L else 0) | (2 if B else 0)) == tgt
            if (L or R) and (T or B):  # the diagonal leaving the corner
                tgt = ((x0 + lx + (-1 if L else 1)) % nx, (y0 + ly + (-1 if T else 1)) % ny)
                assert corner_node(xs, ys, tm if L else tp, bm if T else bp, (1 if L else 0) | (2 if T else 0)) == tgt
