"""Index arithmetic of the two-step tile's periodic halo fill, emulated on the CPU.

The two-step kernel (csrc/lbm_fused.cuh, stage 1) loads a tile's region by a
tensor copy, which leaves zeros where the region crosses the lattice's edge.
For a periodic edge it then fetches, with plain loads, the cells of the ring
of width two around the lattice that lie in the region and outside the
lattice: the only cells outside the lattice that a node of the lattice reads
in the two steps.  The kernel enumerates them as rows (across a periodic y
edge) and columns (across a periodic x edge) of a flat index; this test
repeats that enumeration in Python and checks it against the set defined
directly (every region cell within two nodes of the lattice, outside it across
a periodic edge, not beyond a wall): the same cells, each once, every index
inside the region's shared-memory box.
"""
import itertools

import pytest

TX, TY = 64, 16            # the tile (FusedTile)
RW, RH = TX + 4, TY + 4    # the region of the even step: the tile and two nodes around it


def needs_fill(nx, ny, x0, y0, perx, pery):
    """The kernel's test for an edge tile that needs wrapped halo cells."""
    return (perx and (x0 - 2 < 0 or x0 + TX + 2 > nx)) or (pery and (y0 - 2 < 0 or y0 + TY + 2 > ny))


def ring_by_definition(nx, ny, x0, y0, perx, pery):
    """{(rx, ry): (source x, source y)} for the region cells the fill must write."""
    out = {}
    for ry in range(RH):
        for rx in range(RW):
            gx, gy = x0 - 2 + rx, y0 - 2 + ry
            if not (-2 <= gx <= nx + 1 and -2 <= gy <= ny + 1):
                continue                     # no node of the lattice reads it
            outx, outy = not 0 <= gx < nx, not 0 <= gy < ny
            if (outx and not perx) or (outy and not pery):
                continue                     # beyond a wall
            if outx or outy:
                out[(rx, ry)] = (gx % nx, gy % ny)
    return out


def ring_as_enumerated(nx, ny, x0, y0, perx, pery):
    """The kernel's enumeration: rows across a periodic y edge over the ring's
    columns, then columns across a periodic x edge over the rows inside."""
    X0, Y0 = x0 - 2, y0 - 2
    X1, Y1 = min(x0 + TX + 2, nx + 2), min(y0 + TY + 2, ny + 2)
    xi0, xi1 = max(X0, 0), min(X1, nx)
    yi0, yi1 = max(Y0, 0), min(Y1, ny)
    rlo = max(0, min(0, Y1) - Y0) if pery else 0
    rhi = max(0, Y1 - max(ny, Y0)) if pery else 0
    rx0 = X0 if perx else xi0
    rw = max(0, (X1 if perx else xi1) - rx0)
    clo = max(0, min(0, X1) - X0) if perx else 0
    chi = max(0, X1 - max(nx, X0)) if perx else 0
    ch = max(0, yi1 - yi0)
    nrow = (rlo + rhi) * rw
    ncell = nrow + (clo + chi) * ch
    cells = []
    for k in range(ncell):
        if k < nrow:
            r = k // rw
            gx = rx0 + (k - r * rw)
            gy = Y0 + r if r < rlo else max(ny, Y0) + (r - rlo)
        else:
            c = (k - nrow) // ch
            gy = yi0 + (k - nrow - c * ch)
            gx = X0 + c if c < clo else max(nx, X0) + (c - clo)
        cells.append((gx - X0, gy - Y0, ((gx % nx) + nx) % nx, ((gy % ny) + ny) % ny))
    return cells


SIDES_X = [4, 5, 7, 31, 62, 63, 64, 65, 66, 67, 68, 69, 100, 127, 128, 129, 130, 131, 200, 257]
SIDES_Y = [4, 5, 13, 14, 15, 16, 17, 18, 19, 20, 21, 33, 50, 65, 70]


@pytest.mark.parametrize("perx,pery", list(itertools.product([True, False], repeat=2)),
                         ids=["periodic", "x_periodic", "y_periodic", "walled"])
def test_halo_ring_enumeration_matches_its_definition(perx, pery):
    tiles = 0
    for nx in SIDES_X:
        for ny in SIDES_Y:
            for x0 in range(0, nx, TX):
                for y0 in range(0, ny, TY):
                    want = ring_by_definition(nx, ny, x0, y0, perx, pery)
                    if not needs_fill(nx, ny, x0, y0, perx, pery):
                        assert not want, (nx, ny, x0, y0)
                        continue
                    got = ring_as_enumerated(nx, ny, x0, y0, perx, pery)
                    for rx, ry, sx, sy in got:
                        assert 0 <= rx < RW and 0 <= ry < RH, (nx, ny, x0, y0, rx, ry)
                        assert 0 <= sx < nx and 0 <= sy < ny
                    keys = [(rx, ry) for rx, ry, _, _ in got]
                    assert len(keys) == len(set(keys)), ("a cell twice", nx, ny, x0, y0)
                    assert {(rx, ry): (sx, sy) for rx, ry, sx, sy in got} == want, (nx, ny, x0, y0)
                    tiles += 1
    assert tiles > 0 or not (perx or pery)


def test_halo_ring_is_at_most_352_cells_per_plane():
    """Four rows of the region's 68 columns and four columns of its 16 inner
    rows: the bound that makes the fill two rounds of 256 threads at most."""
    worst = 0
    for nx in SIDES_X:
        for ny in SIDES_Y:
            for x0 in range(0, nx, TX):
                for y0 in range(0, ny, TY):
                    if needs_fill(nx, ny, x0, y0, True, True):
                        worst = max(worst, len(ring_as_enumerated(nx, ny, x0, y0, True, True)))
    assert worst <= 4 * RW + 4 * TY
