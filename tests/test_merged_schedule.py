"""Plane sources of the shadow-shell merged sweep split into z chunks (the
index rules of k_merged3 and k_zcopy restated on the host).

Chunk j of nzc covers the odd steps of planes [z0, z1) with z0 = j nz / nzc,
z1 = (j + 1) nz / nzc, and loads planes max(z0 - 1, 0) .. min(z1, nz - 1)
for its even steps.  The planes z - 1 and z next to a boundary z are
written by both chunks during the sweep, so both load them from the copy
(plane 2b + s of the copy holds plane zb - 1 + s of boundary b).  Checked
here: every loaded plane that does not come from the copy is written by no
other chunk, the copy coordinates are in range and name the right plane,
and the chunks' odd steps cover every plane once."""


def _chunks(nz, nzc):
    for j in range(nzc):
        z0, z1 = j * nz // nzc, (j + 1) * nz // nzc
        yield j, z0, z1, (z0 - 1 if z0 > 0 else 0), (z1 if z1 < nz else nz - 1)


def _copy_plane(j, nzc, z0, z1, q):
    if j > 0 and q in (z0 - 1, z0):
        return 2 * (j - 1) + (q - z0 + 1)
    if j < nzc - 1 and q in (z1 - 1, z1):
        return 2 * j + (q - z1 + 1)
    return -1


def test_z_chunk_plane_sources():
    for nz in range(1, 70):
        for nzc in range(1, max(1, nz // 4) + 1):
            chunks = list(_chunks(nz, nzc))
            # planes each chunk's odd steps write: k - 1 .. k + 1 for k in [z0, z1)
            written = {j: set(range(max(z0 - 1, 0), min(z1, nz - 1) + 1)) for j, z0, z1, _, _ in chunks}
            odd = []
            for j, z0, z1, qb, last in chunks:
                assert nzc == 1 or z1 - z0 >= 4
                odd += range(z0, z1)
                for q in range(qb, last + 1):
                    p = _copy_plane(j, nzc, z0, z1, q)
                    if p >= 0:
                        assert 0 <= p < 2 * (nzc - 1)
                        assert ((p >> 1) + 1) * nz // nzc - 1 + (p & 1) == q
                    else:
                        assert all(q not in w for j2, w in written.items() if j2 != j), (nz, nzc, j, q)
            assert odd == list(range(nz))


def _shadow_emulation(C, nx, ny, nz, per, TY):
    """Index rules of k_merged3's shell shadow (z not periodic): every shadow
    entry of every plane is written exactly once per sweep, every ring and
    halo access stays in its buffer, and the cells with shell targets are
    exactly the band cells the odd warps take first."""
    Q, TX, W, H = 19, 32, 34, TY + 2
    NPOS, NS = W * H, 2 * TX + 2 * (TY - 2)
    NSP, NH = (NS + 7) // 8 * 8, 2 * W + 2 * TY
    opp = [0] + [i + 9 for i in range(1, 10)] + [i - 9 for i in range(10, 19)]
    ntx, nty = (nx + 31) // 32, (ny + TY - 1) // TY
    hb, rem = ny // nty, ny % nty
    gplane = ntx * nty * Q * NSP

    def band_of(by):
        return by * hb + min(by, rem), hb + (1 if by < rem else 0)

    def band_at(y):
        big = rem * (hb + 1)
        return y // (hb + 1) if y < big else rem + (y - big) // hb

    def shell_slot(lx, ly, tw, th):
        if ly == 0:
            return lx
        if ly == th - 1:
            return 32 + lx
        if lx == 0:
            return 64 + ly - 1
        if lx == tw - 1:
            return 64 + (TY - 2) + ly - 1
        return -1

    def shell_offset(x, y):
        bx, by = x >> 5, band_at(y)
        y0, th = band_of(by)
        tw = min(32, nx - 32 * bx)
        s = shell_slot(x - 32 * bx, y - y0, tw, th)
        return -1 if s < 0 else (by * ntx + bx) * Q * NSP + s

    def wrap(v, n, p):
        if 0 <= v < n:
            return v, True
        return (v % n, True) if p else (v, False)

    expect = set()
    for y in range(ny):
        for x in range(nx):
            o = shell_offset(x, y)
            if o >= 0:
                for i in range(Q):
                    assert o + i * NSP not in expect and o + i * NSP < gplane
                    expect.add(o + i * NSP)
    written = set()
    for by in range(nty):
        y0, th = band_of(by)
        for bx in range(ntx):
            x0, tw = 32 * bx, min(32, nx - 32 * bx)
            gtab = [-1] * NPOS
            for p in range(NPOS):
                px, py = p % W - 1, p // W - 1
                if px <= tw and py <= th:
                    gx, okx = wrap(x0 + px, nx, per[0])
                    gy, oky = wrap(y0 + py, ny, per[1])
                    if okx and oky:
                        gtab[p] = shell_offset(gx, gy)
            for h in range(32 * ((NH + 31) // 32)):  # halo cells: their shadow rows exist
                if h < W:
                    lx, ly, act = h - 1, -1, h - 1 <= tw
                elif h < 2 * W:
                    lx, ly, act = h - W - 1, th, h - W - 1 <= tw
                elif h < 2 * W + TY:
                    lx, ly, act = -1, h - 2 * W, h - 2 * W < th
                elif h < NH:
                    lx, ly, act = tw, h - 2 * W - TY, h - 2 * W - TY < th
                else:
                    act = False
                if act:
                    _, okx = wrap(x0 + lx, nx, per[0])
                    _, oky = wrap(y0 + ly, ny, per[1])
                    if okx and oky:
                        pos = (ly + 1) * W + lx + 1
                        assert 0 <= pos < NPOS and gtab[pos] >= 0 and gtab[pos] + 18 * NSP < gplane
            for ly in range(th):
                for lx in range(tw):
                    pos, x, y = (ly + 1) * W + lx + 1, x0 + lx, y0 + ly
                    assert (gtab[pos] >= 0) == (lx in (0, tw - 1) or ly in (0, th - 1))
                    has_target = False
                    for i in range(Q):
                        cx_, cy_, cz_ = (int(v) for v in C[i])
                        assert 0 <= pos - cx_ - cy_ * W < NPOS
                        tx, okx = wrap(x + cx_, nx, per[0])
                        ty, oky = wrap(y + cy_, ny, per[1])
                        off = -1
                        if okx and oky:
                            off = gtab[pos + cx_ + cy_ * W]
                            assert off == shell_offset(tx, ty)
                            has_target |= off >= 0
                        for k in range(nz):
                            zt = k + cz_
                            if not (okx and oky) or zt < 0 or zt >= nz:  # wall link: bounce in the own cell
                                zt, off2, d2 = k, gtab[pos], opp[i]
                            else:
                                off2, d2 = off, i
                            if off2 >= 0:
                                key = (zt, off2 + d2 * NSP)
                                assert key not in written
                                written.add(key)
                    if tw >= 4 and th >= 4:
                        band = ly in (0, 1, th - 2, th - 1) or lx in (0, 1, tw - 2, tw - 1)
                        assert has_target == band
    assert written == {(z, e) for z in range(nz) for e in expect}


# The CUDA library's direction numbering (grouped by c_z: rest, then the nine
# vectors whose first non-zero component is -1, then their opposites); the
# ABI test checks that lbm_lattice() reports exactly this table.
GPU_C = [(0, 0, 0), (0, 0, -1), (-1, 0, -1), (0, -1, -1), (-1, 0, 1), (0, -1, 1), (-1, 0, 0), (0, -1, 0),
         (-1, -1, 0), (-1, 1, 0)]
GPU_C += [tuple(-v for v in c) for c in GPU_C[1:]]


def test_shell_shadow_written_once():
    C = GPU_C
    for shape, per, ty in [((16, 16, 4), (0, 0), 14), ((37, 19, 5), (1, 1), 14), ((37, 19, 5), (1, 1), 6),
                           ((33, 40, 4), (0, 1), 14), ((20, 1, 3), (1, 1), 14), ((70, 3, 3), (1, 0), 6),
                           ((64, 30, 3), (0, 0), 4)]:
        _shadow_emulation(C, *shape, per, ty)


def _shell_cell(s, tw, th, TY):
    if s < 32:
        return (s, 0) if s < tw else None
    if s < 64:
        return (s - 32, th - 1) if th > 1 and s - 32 < tw else None
    if s < 64 + (TY - 2):
        return (0, s - 63) if s - 63 < th - 1 else None
    if s < 64 + 2 * (TY - 2):
        ly = s - 64 - (TY - 2) + 1
        return (tw - 1, ly) if tw > 1 and ly < th - 1 else None
    return None


def test_role_maps_cover_each_tile_once():
    """The even warps (shell cells in shadow-slot order, then the inner cells)
    and the odd warps (the two outer rows on either side, the two outer
    columns of the middle rows, then the inner cells; plain rows for tiles
    under 4 x 4) each take every cell of every tile shape exactly once."""
    for TY in (14, 4):
        NS = 64 + 2 * (TY - 2)
        for tw in range(1, 33):
            for th in range(1, TY + 1):
                cells = sorted((x, y) for y in range(th) for x in range(tw))
                even = []
                for t in range(32 * TY):
                    if t < NS:
                        c = _shell_cell(t, tw, th, TY)
                        if c:
                            even.append(c)
                    else:
                        v, w = t - NS, tw - 2
                        if w > 0 and th > 2 and v < w * (th - 2):
                            even.append((1 + v % w, 1 + v // w))
                assert sorted(even) == cells, ("even", TY, tw, th)
                odd = []
                for t in range(32 * TY):
                    if tw < 4 or th < 4:
                        lx, ly = t & 31, t >> 5
                        if lx < tw and ly < th:
                            odd.append((lx, ly))
                        continue
                    nrow, nband = 4 * tw, 4 * tw + 4 * (th - 4)
                    if t >= tw * th:
                        continue
                    if t < nrow:
                        r = t // tw
                        odd.append((t - r * tw, r if r < 2 else th - 4 + r))
                    elif t < nband:
                        u = t - nrow
                        j = u & 3
                        odd.append((j if j < 2 else tw - 4 + j, 2 + (u >> 2)))
                    else:
                        v, w = t - nband, tw - 4
                        odd.append((2 + v % w, 2 + v // w))
                assert sorted(odd) == cells, ("odd", TY, tw, th)
