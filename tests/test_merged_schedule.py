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
