"""Index rules of the neighbour-synchronised merged sweep (k_nsweep),
restated on the host.

The sweep keeps a tile's odd step of plane k from writing a location before
every tile that reads it has loaded it, by waiting until the tile's eight
neighbours have loaded plane k+1.  That is enough only if every reader of a
location the tile writes is the tile itself or one of those neighbours.  A
tile writes the cells within one cell of it (planes k-1 .. k+1); a tile
reads its own cells and its one-cell halo ring.  Checked here for many
lattice shapes, with the band split of the sweep (32-wide tiles, bands of
near-equal height of at most 14 rows): the readers of every written cell
are among the writer and its neighbours, and the copy box (x from the tile
start minus the 16-byte margin) covers the tile and its halo."""
import pytest

TX, TY = 32, 14


def _bands(ny):
    nty = (ny + TY - 1) // TY
    hb, rem = ny // nty, ny % nty
    out, y = [], 0
    for b in range(nty):
        h = hb + (1 if b < rem else 0)
        out.append((y, h))
        y += h
    assert y == ny
    return out


def _tiles(nx, ny):
    ntx = (nx + TX - 1) // TX
    return [(bx, by, bx * TX, min(TX, nx - bx * TX), y0, th)
            for by, (y0, th) in enumerate(_bands(ny)) for bx in range(ntx)]


def _owner(nx, ny):
    own = {}
    for bx, by, x0, tw, y0, th in _tiles(nx, ny):
        for y in range(y0, y0 + th):
            for x in range(x0, x0 + tw):
                own[(x, y)] = (bx, by)
    return own


@pytest.mark.parametrize("nx", [1, 2, 31, 32, 33, 64, 65, 100, 256])
@pytest.mark.parametrize("ny", [1, 2, 13, 14, 15, 27, 28, 29, 43, 100, 256])
def test_readers_of_written_cells_are_neighbours(nx, ny):
    own = _owner(nx, ny)
    readers = {}
    for bx, by, x0, tw, y0, th in _tiles(nx, ny):
        if len(_bands(ny)) > 1:
            assert th >= 2
        for y in range(y0 - 1, y0 + th + 1):
            for x in range(x0 - 1, x0 + tw + 1):
                if 0 <= x < nx and 0 <= y < ny:
                    readers.setdefault((x, y), set()).add((bx, by))
    for bx, by, x0, tw, y0, th in _tiles(nx, ny):
        nbrs = {(bx + dx, by + dy) for dx in (-1, 0, 1) for dy in (-1, 0, 1)}
        for y in range(y0 - 1, y0 + th + 1):
            for x in range(x0 - 1, x0 + tw + 1):
                if 0 <= x < nx and 0 <= y < ny:
                    assert readers[(x, y)] <= nbrs, ((nx, ny), (bx, by), (x, y))
                    assert own[(x, y)] in nbrs


@pytest.mark.parametrize("elem", [4, 2])
def test_copy_box_covers_tile_and_halo(elem):
    xm = 16 // elem
    bw, bh = TX + 2 * xm, TY + 2
    assert (bw * elem) % 16 == 0
    for bx in range(8):
        x0 = bx * TX
        start = x0 - xm
        assert (start * elem) % 16 == 0          # tiled-copy alignment of the x coordinate
        for tw in (1, 17, 32):
            for lx in range(-1, tw + 1):          # tile columns and the two halo columns
                col = lx + xm
                assert 0 <= col < bw and start + col == x0 + lx
        for th in (2, 13, 14):
            for ly in range(-1, th + 1):
                assert 0 <= ly + 1 < bh
