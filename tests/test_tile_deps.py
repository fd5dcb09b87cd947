"""The tile exchange rule of the multi-step step launch (configuration 8),
checked by brute force on the CPU.

A tile of configuration 7 has 58 x 26 outputs; tile kx covers domain columns
[58 kx - 1, 58 kx + 57), tile ky rows [26 ky, 26 ky + 26); its TMA box reaches
4 cells further on every side; periodic axes write ghost images of the first
and last 4 rows (columns).  Two tiles must wait for each other's previous
step when one writes a cell the other's box reads (read after write, and
write after read one step later).  The kernel's rule: the two neighbours
along each axis (periodic wrap included), plus tiles 0 and n-2 of an axis
whose last tile is thin; and with tile rows visited in the folded order
0, ty-1, 1, ty-2, ... every dependency lies within 4 tiles_x - 1 work items,
which the host's choice of launch relies on."""
import numpy as np
import pytest

TX, TY, H = 58, 26, 4


def dep_axis(k, c, n, thin):
    if c < 3:
        v = k + c - 1
        return v + n if v < 0 else (v - n if v >= n else v)
    if not thin:
        return -1
    return n - 2 if k == 0 else (0 if k == n - 2 else -1)


def rule(kx, ky, tx, ty, nx, ny):
    thin_x = (tx - 1) * TX + 3 > nx
    thin_y = (ty - 1) * TY + H > ny
    out = set()
    for c in range(16):
        dx = dep_axis(kx, c & 3, tx, thin_x)
        dy = dep_axis(ky, c >> 2, ty, thin_y)
        if dx >= 0 and dy >= 0:
            out.add((dx, dy))
    return out


def footprints(nx, ny, perx, pery):
    tx, ty = (nx + TX) // TX, (ny + TY - 1) // TY
    W, Hh = nx + 2 * H, ny + 2 * H
    reads, writes = {}, {}
    for ky in range(ty):
        for kx in range(tx):
            r = np.zeros((Hh, W), bool)
            c0, c1 = kx * TX - 1 - H, kx * TX - 1 + TX + H
            r0, r1 = ky * TY - H, ky * TY + TY + H
            r[max(r0 + H, 0):min(r1 + H, Hh), max(c0 + H, 0):min(c1 + H, W)] = True
            w = np.zeros((Hh, W), bool)
            xs = np.arange(max(kx * TX - 1, 0), min(kx * TX - 1 + TX, nx))
            ys = np.arange(ky * TY, min(ky * TY + TY, ny))
            for X in [xs] + ([xs[xs < H] + nx, xs[xs >= nx - H] - nx] if perx else []):
                for Y in [ys] + ([ys[ys < H] + ny, ys[ys >= ny - H] - ny] if pery else []):
                    w[np.ix_(Y + H, X + H)] = True
            reads[(kx, ky)], writes[(kx, ky)] = r, w
    return tx, ty, reads, writes


def folded_pos(kx, ky, tx, ty):
    order = [p // 2 if p % 2 == 0 else ty - 1 - p // 2 for p in range(ty)]
    return order.index(ky) * tx + kx


@pytest.mark.parametrize("nx", [5, 59, 61, 117, 119, 175, 178, 301])
@pytest.mark.parametrize("ny", [5, 27, 29, 53, 56, 79, 157])
@pytest.mark.parametrize("per", [(1, 1), (0, 1), (1, 0)])
def test_rule_covers_every_exchange(nx, ny, per):
    tx, ty, reads, writes = footprints(nx, ny, *per)
    for A in reads:
        dA = rule(*A, tx, ty, nx, ny)
        for B in writes:
            if A != B and (writes[B] & reads[A]).any():
                assert B in dA and A in rule(*B, tx, ty, nx, ny), (A, B)
        for B in dA:
            assert abs(folded_pos(*A, tx, ty) - folded_pos(*B, tx, ty)) <= 4 * tx - 1


def test_thin_last_row_needs_the_extra_pair():
    """157 rows = 6 x 26 + 1: tile row 5's box reaches the ghost rows that
    tile row 0 writes, so the plain 3 x 3 neighbourhood would miss it."""
    nx, ny = 301, 157
    tx, ty, reads, writes = footprints(nx, ny, 1, 1)
    assert (writes[(0, 0)] & reads[(0, 5)]).any()
    assert (0, 0) in rule(0, 5, tx, ty, nx, ny)
