// merged3.cuh -- two collision-streaming steps per sweep with a shadow copy
// of the tile shells (the MERGED schedule on a lattice whose z faces are
// walls).
//
// The paper merges two time steps of a cell as soon as its neighbours have
// done the first one (Sec. 4.1, Alg. 2), and makes the layers where two
// threads' sub-domains meet safe by handling them apart (the intersection
// layers of Alg. 3, Sec. 4.2).  Here:
//
//  * A CTA owns a column of 32 x TH cells (TH <= TY; the rows of the plane
//    are split into bands of near-equal height) and marches it along z.
//    Its warps are specialised: "even" warps (one per tile row) collide
//    plane k+2 and hand the post-collision values to shared-memory rings,
//    "odd" warps (one per tile row) gather plane k from the rings, collide
//    and scatter into f, and halo warps re-collide the one-cell halo ring
//    and stage the inputs.  Even and odd warps work in the same interval
//    between two CTA barriers, two planes apart, so twice as many warps
//    hide each other's latencies.
//  * Inputs of a plane arrive in a two-slot stage: one TMA tensor copy per
//    direction for the 32 x TY tile, and cp.async copies for the tile's own
//    shell cells and its halo cells, all completing on the slot's mbarrier.
//  * Cells on a tile's boundary ring ("shell" cells) are read by up to four
//    CTAs: the owner and the neighbours whose halo they are.  Every shell
//    cell also lives in a double-buffered shadow G: a sweep takes shell and
//    halo inputs from G_cur (never from f, which other CTAs are already
//    overwriting) and writes every post-stream value that lands on a shell
//    cell to G_next as well as to f.  No CTA reads what another CTA writes
//    during the sweep, so tiles need no synchronisation at all, and f stays
//    the complete state after every sweep.
//  * With fewer tiles than SMs the march is split along z into chunks, one
//    CTA per tile and chunk (CHUNK = true).  A chunk also collides the
//    plane beyond each of its ends (even step only); the two planes next to
//    a chunk boundary, which both chunks write, are loaded from a copy made
//    before the sweep (k_zcopy).
//
// HBM traffic per two steps: every population read and written once, plus
// the shell shadow (read once by its owner, written once): 2 x 19 x
// sizeof(T) x (1 + NS / (32 TY)) bytes per cell.
#pragma once

#include "tma.cuh"

namespace lbm {

template <int TY>
struct M3 {
    static constexpr int TX = 32, W = TX + 2, H = TY + 2, NPOS = W * H;
    static constexpr int NT = TX * TY;
    static constexpr int NH = 2 * W + 2 * TY;          // halo ring cells
    static constexpr int NHW = (NH + 31) / 32;          // halo warps
    static constexpr int NHT = 32 * NHW;                // halo threads
    static constexpr int NWARPS = 2 * TY + NHW;
    static constexpr int THREADS = 32 * NWARPS;
    static constexpr int NS = 2 * TX + 2 * (TY - 2);    // shell slots of a full tile
    static constexpr int NSP = (NS + 7) / 8 * 8;
    // ring slots per z-group (planes alive at once with even warps two
    // planes ahead of odd warps) and the small rings of the rest and pure-z
    // populations
    static constexpr int RSM = 3, RS0 = 3, RSP = 4;
    static constexpr int NRING = RSM * NDM + RS0 * ND0 + RSP * NDP;
    static constexpr int SREST = 3, SZP = 4, SZM = 3;
    static constexpr int NTS = 33 * TY;  // small-ring slot size (pitch 33)
    // periodic z: per tile, the values of planes -1 and 0 kept for the end of
    // the march (16 ring directions at every position, rest and pure z)
    static constexpr int NXY = 16;
    static constexpr int ZSAVE = 2 * (NXY * NPOS + 3 * NTS);
    static_assert(TY >= 2, "bands of at least two rows");
    static_assert(THREADS <= 1024, "one CTA");
};

// Shared-memory layout of one CTA for stored type T and compute type R.
template <int TY, class T, class R>
struct M3Smem {
    using L = M3<TY>;
    static constexpr int EPU = sizeof(T) >= 4 ? 1 : 4 / (int)sizeof(T);  // elements per copy unit
    static constexpr int CP = (int)sizeof(T) * EPU;                         // bytes per copy unit
    static constexpr int DST = (L::NT + L::NSP + 128 / (int)sizeof(T) - 1) / (128 / (int)sizeof(T)) *
                               (128 / (int)sizeof(T));                      // tile-block stride per direction
    static constexpr size_t tile_bytes = (size_t)Q * DST * sizeof(T);
    static constexpr size_t halo_bytes = (size_t)Q * L::NHT * CP;
    static constexpr size_t slot_bytes = (tile_bytes + halo_bytes + 127) / 128 * 128;
    static constexpr size_t stage_off = 0;
    static constexpr size_t ring_off = 2 * slot_bytes;
    static constexpr size_t small_off = ring_off + (size_t)L::NRING * L::NPOS * sizeof(R);
    static constexpr size_t gtab_off = small_off + (size_t)(L::SREST + L::SZP + L::SZM) * L::NTS * sizeof(R);
    static constexpr size_t bar_off = (gtab_off + (size_t)L::NPOS * sizeof(int) + 15) / 16 * 16;
    static constexpr size_t flag_off = bar_off + 2 * sizeof(uint64_t);
    static constexpr size_t bytes = flag_off + 16;
    static constexpr unsigned tma_bytes = (unsigned)(Q * L::NT * sizeof(T));
    static constexpr int CHUNKS = L::NSP * (int)sizeof(T) / 16;  // 16-byte chunks of one direction's shell row
    static_assert(L::NSP * sizeof(T) % 16 == 0, "shell rows in 16-byte chunks");
};

// Shell slot of local cell (lx, ly) of a tw x th tile, or -1 inside:
// first row, last row, first column, last column (corners in the rows).
template <int TY>
__host__ __device__ __forceinline__ int shell_slot(int lx, int ly, int tw, int th)
{
    if (ly == 0) return lx;
    if (ly == th - 1) return 32 + lx;
    if (lx == 0) return 64 + ly - 1;
    if (lx == tw - 1) return 64 + (TY - 2) + ly - 1;
    return -1;
}

// Inverse of shell_slot; false when the slot is unused by this tile.
template <int TY>
__host__ __device__ __forceinline__ bool shell_cell(int s, int tw, int th, int &lx, int &ly)
{
    if (s < 32) { lx = s; ly = 0; return lx < tw; }
    if (s < 64) { lx = s - 32; ly = th - 1; return th > 1 && lx < tw; }
    if (s < 64 + (TY - 2)) { lx = 0; ly = s - 63; return ly < th - 1; }
    if (s < 64 + 2 * (TY - 2)) { lx = tw - 1; ly = s - 64 - (TY - 2) + 1; return tw > 1 && ly < th - 1; }
    return false;
}

__host__ __device__ __forceinline__ void band_of(const ShellInfo &si, int by, int &y0, int &th)
{
    y0 = by * si.hb + (by < si.rem ? by : si.rem);
    th = si.hb + (by < si.rem ? 1 : 0);
}
__host__ __device__ __forceinline__ int band_at(const ShellInfo &si, int y)
{
    const int big = si.rem * (si.hb + 1);
    return y < big ? y / (si.hb + 1) : si.rem + (y - big) / si.hb;
}

// Offset inside one z-plane of G of the shell cell (x, y) (in the domain),
// or -1 when it is not on its tile's boundary ring.
template <int TY>
__host__ __device__ __forceinline__ int shell_offset(const ShellInfo &si, int nx, int x, int y)
{
    const int bx = x >> 5, by = band_at(si, y);
    int y0, th;
    band_of(si, by, y0, th);
    const int tw = nx - 32 * bx < 32 ? nx - 32 * bx : 32;
    const int s = shell_slot<TY>(x - 32 * bx, y - y0, tw, th);
    return s < 0 ? -1 : (by * si.ntx + bx) * Q * M3<TY>::NSP + s;
}

// Copies the shell cells of f into G (the state a merged sweep starts from).
template <class S, int TY>
__global__ void __launch_bounds__(256) k_shell_gather(Geom<typename S::R> g, Dirs<const typename S::T> f,
                                                      typename S::T *__restrict__ G, ShellInfo si)
{
    constexpr int NSP = M3<TY>::NSP;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per_plane = (int64_t)si.ntx * si.nty * NSP;
    if (idx >= per_plane * g.nz) return;
    const int z = (int)(idx / per_plane);
    const int r = (int)(idx % per_plane);
    const int tile = r / NSP, s = r % NSP;
    const int bx = tile % si.ntx, by = tile / si.ntx;
    int y0, th, lx, ly;
    band_of(si, by, y0, th);
    const int tw = min(32, g.nx - 32 * bx);
    if (!shell_cell<TY>(s, tw, th, lx, ly)) return;
    const int c = cell32(g, 32 * bx + lx, y0 + ly, z);
    typename S::T *dst = G + z * si.gplane + (int64_t)tile * Q * NSP + s;
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        dst[i * NSP] = f.p[i][c];
    });
}


// Copies the planes zb-1 and zb of every boundary zb = (b+1) nz / nzc between
// z chunks b and b+1 into zc[d][2b + s][y][x] (s = 0, 1), before the sweep
// in which both chunks write them.
template <class S>
__global__ void __launch_bounds__(256) k_zcopy(Geom<typename S::R> g, const typename S::T *__restrict__ f,
                                               typename S::T *__restrict__ zc, int nzc)
{
    const int64_t per_plane = (int64_t)g.ny * g.nxp;
    const int np = 2 * (nzc - 1);
    const int64_t total = (int64_t)Q * np * per_plane;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx % per_plane, t = idx / per_plane;
        const int p = (int)(t % np), d = (int)(t / np);
        const int zb = (int)((int64_t)((p >> 1) + 1) * g.nz / nzc);
        zc[idx] = f[d * g.slot + (int64_t)(zb - 1 + (p & 1)) * per_plane + r];
    }
}

// CTA-wide barrier that the warps may reach from different code locations
// (every thread arrives the same number of times).
__device__ __forceinline__ void cta_barrier() { asm volatile("barrier.sync 0;" ::: "memory"); }

// 16-byte asynchronous copy that bypasses L1.
__device__ __forceinline__ void cp_async_cg16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_mbar_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Directions with c_z = -1 / +1 (wall links on the z = 0 / nz-1 planes).
__host__ __device__ constexpr unsigned z_bits(int sign)
{
    unsigned m = 0u;
    for (int i = 0; i < Q; ++i)
        if (cz(i) == sign) m |= 1u << i;
    return m;
}

// Index of an xy-moving direction among the 16 (ring directions).
__host__ __device__ constexpr int xyidx(int i)
{
    int n = 0;
    for (int j = 0; j < i; ++j)
        if (grp(j) == GRP_M || grp(j) == GRP_0 || grp(j) == GRP_P) ++n;
    return n;
}

template <class S, bool FORCE, int TY, bool PERZ, bool CHUNK>
struct M3Cta {
    using R = typename S::R;
    using T = typename S::T;
    using L = M3<TY>;
    using SM = M3Smem<TY, T, R>;
    static constexpr int W = L::W, NPOS = L::NPOS, NSP = L::NSP, NT = L::NT, NHT = L::NHT;
    static constexpr int DST = SM::DST, EPU = SM::EPU, CP = SM::CP;
    static constexpr unsigned CZM = z_bits(-1), CZP = z_bits(1);
    enum { EVEN = 0, ODD = 1, HALO = 2 };

    const Geom<R> &g;
    const Dirs<T> &fd;
    const Dirs<T> &fo;  // fd.p[i] + noff[i]: the push target of an interior cell
    const Dirs<T> &go;  // Gn + cz(i) gplane + i NSP: the shadow target of direction i
    const T *__restrict__ Gc;
    T *__restrict__ Gn;
    const ShellInfo &si;
    const CUtensorMap *tmap;
    const CUtensorMap *tmapz;  // the z-chunk boundary planes (z split into chunks), else unused
    R *zsave;  // periodic z: this tile's save area (ZSAVE elements), else null
    unsigned char *smem;
    R *ringm, *ring0, *ringp, *srest, *szp, *szm;
    int *gtab;
    uint64_t *bar;
    int *issued;  // shared count of the stages whose copies have been started
    int role, x0, y0, tw, th, lx, ly, x, y, pos, tc, hidx, nx, ny, nz, goff, cxy, inoff, sub;
    // z chunk jc of nzc: odd steps of planes [zc0, zc1), loaded planes from qb
    int jc, nzc, zc0, zc1, qb;
    unsigned gmask, wxy, lxy;
    bool active, perx, pery, xybnd, timed_out;
    static constexpr bool perz = PERZ;

    __device__ __forceinline__ M3Cta(const Geom<R> &g_, const Dirs<T> &fd_, const Dirs<T> &fo_, const Dirs<T> &go_,
                                     const T *Gc_, T *Gn_, const ShellInfo &si_, const CUtensorMap *tmap_, R *zs,
                                     unsigned char *smem_)
        : g(g_), fd(fd_), fo(fo_), go(go_), Gc(Gc_), Gn(Gn_), si(si_), tmap(tmap_), smem(smem_)
    {
        ringm = reinterpret_cast<R *>(smem + SM::ring_off);
        ring0 = ringm + L::RSM * NDM * NPOS;
        ringp = ring0 + L::RS0 * ND0 * NPOS;
        srest = reinterpret_cast<R *>(smem + SM::small_off);
        szp = srest + L::SREST * L::NTS;
        szm = szp + L::SZP * L::NTS;
        gtab = reinterpret_cast<int *>(smem + SM::gtab_off);
        bar = reinterpret_cast<uint64_t *>(smem + SM::bar_off);
        nx = g.nx; ny = g.ny; nz = g.nz;
        perx = g.per[0] != 0; pery = g.per[1] != 0;
        zsave = PERZ ? zs + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * L::ZSAVE : nullptr;
        x0 = 32 * blockIdx.x;
        tw = min(32, nx - x0);
        band_of(si, blockIdx.y, y0, th);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        role = warp < TY ? EVEN : (warp < 2 * TY ? ODD : HALO);
        hidx = 0;
        if (role == HALO) {
            // halo ring: row -1, row th, column -1, column tw
            const int h = (warp - 2 * TY) * 32 + lane;
            hidx = h;
            active = true;
            if (h < W) { lx = h - 1; ly = -1; active = lx <= tw; }
            else if (h < 2 * W) { lx = h - W - 1; ly = th; active = lx <= tw; }
            else if (h < 2 * W + TY) { lx = -1; ly = h - 2 * W; active = ly < th; }
            else if (h < 2 * W + 2 * TY) { lx = tw; ly = h - 2 * W - TY; active = ly < th; }
            else { lx = 0; ly = 0; active = false; }
        } else if (role == EVEN) {
            // even warps: the shell cells in shadow-slot order (their inputs
            // sit side by side in the stage), then the inner cells row by row
            const int t = threadIdx.x;
            if (t < L::NS) {
                active = shell_cell<TY>(t, tw, th, lx, ly);
                if (!active) { lx = 0; ly = 0; }
            } else {
                const int v = t - L::NS, w = tw - 2;
                active = w > 0 && th > 2 && v < w * (th - 2);
                if (active) { ly = 1 + v / w; lx = 1 + v % w; }
                else { lx = 0; ly = 0; }
            }
        } else if (tw < 4 || th < 4) {
            lx = lane;
            ly = warp - TY;
            active = lx < tw && ly < th;
        } else {
            // odd warps take the cells in band order: the two outer rows on
            // either side, then the two outer columns of the middle rows
            // (every cell that can land a value on a shell cell), then the
            // inner cells, so that whole warps skip the shadow stores
            const int t = threadIdx.x - 32 * TY;
            const int nrow = 4 * tw, nband = nrow + 4 * (th - 4);
            active = t < tw * th;
            if (!active) { lx = 0; ly = 0; }
            else if (t < nrow) { const int r = t / tw; lx = t - r * tw; ly = r < 2 ? r : th - 4 + r; }
            else if (t < nband) { const int u = t - nrow, j = u & 3; ly = 2 + (u >> 2); lx = j < 2 ? j : tw - 4 + j; }
            else { const int v = t - nband, w = tw - 4; ly = 2 + v / w; lx = 2 + v % w; }
        }
        pos = (ly + 1) * W + (lx + 1);
        tc = role == HALO ? 0 : ly * 33 + lx;  // pitch 33 spreads a column over the banks
        x = x0 + lx; y = y0 + ly;
        if (role == HALO && active) {  // wrap the halo cell into the domain, or drop it (wall)
            if (x < 0 || x >= nx) { if (perx) x = x < 0 ? x + nx : x - nx; else active = false; }
            if (y < 0 || y >= ny) { if (pery) y = y < 0 ? y + ny : y - ny; else active = false; }
        }
        xybnd = x == 0 || x == nx - 1 || y == 0 || y == ny - 1;
        cxy = active ? y * (int)g.nxp + x : 0;
        goff = -1;
        inoff = 0;
        sub = 0;
        gmask = wxy = lxy = 0u;
        timed_out = false;
        // wall links through the x and y faces, and those ending on a lid
        if (active) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                bool wall = false, lid = false;
                const int tx = x + cx(i), ty = y + cy(i);
                if ((tx < 0 || tx >= nx) && !perx) { wall = true; lid |= g.lid[tx < 0 ? 0 : 1] != 0; }
                if ((ty < 0 || ty >= ny) && !pery) { wall = true; lid |= g.lid[ty < 0 ? 2 : 3] != 0; }
                if (wall) wxy |= 1u << i;
                if (wall && lid) lxy |= 1u << i;
            });
        }
    }

    // Shadow offsets of every ring and halo position (one table per CTA).
    __device__ __forceinline__ void fill_gtab()
    {
        for (int p = threadIdx.x; p < NPOS; p += L::THREADS) {
            const int px = p % W - 1, py = p / W - 1;
            int v = -1;
            if (px <= tw && py <= th) {
                int gx = x0 + px, gy = y0 + py;
                bool in = true;
                if (gx < 0 || gx >= nx) { if (perx) gx = gx < 0 ? gx + nx : gx - nx; else in = false; }
                if (gy < 0 || gy >= ny) { if (pery) gy = gy < 0 ? gy + ny : gy - ny; else in = false; }
                if (in) v = shell_offset<TY>(si, nx, gx, gy);
            }
            gtab[p] = v;
        }
    }

    // After fill_gtab and a barrier.
    __device__ __forceinline__ void setup()
    {
        if (!active) return;
        goff = gtab[pos];
        if (role == EVEN) {
            const int s = shell_slot<TY>(lx, ly, tw, th);
            inoff = s >= 0 ? NT + s : ly * 32 + lx;
        } else if (role == HALO) {
            sub = goff & (EPU - 1);
        } else {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                if (gtab[pos + cx(i) + cy(i) * W] >= 0) gmask |= 1u << i;
            });
        }
    }

    __device__ __forceinline__ static int slot(int plane, int n) { return (plane + n) % n; }
    template <int GG>
    __device__ __forceinline__ R *ring_at(int plane, int gi) const
    {
        if constexpr (GG == GRP_M) return ringm + (slot(plane, L::RSM) * NDM + gi) * NPOS;
        else if constexpr (GG == GRP_0) return ring0 + (slot(plane, L::RS0) * ND0 + gi) * NPOS;
        else return ringp + (slot(plane, L::RSP) * NDP + gi) * NPOS;
    }
    // Planes of the march are virtual: with periodic z they run from the
    // image -1 of plane nz-1 to the image nz of plane 0.  Stage slots count
    // the loaded planes u = q - qb.
    __device__ __forceinline__ int phys(int q) const
    {
        if constexpr (PERZ) return q < 0 ? q + nz : (q >= nz ? q - nz : q);
        else return q;
    }
    __device__ __forceinline__ T *tile_block(int q) const
    {
        return reinterpret_cast<T *>(smem + ((q - qb) & 1) * SM::slot_bytes);
    }
    __device__ __forceinline__ unsigned char *halo_block(int q) const
    {
        return smem + ((q - qb) & 1) * SM::slot_bytes + SM::tile_bytes;
    }

    // z split into chunks: the two planes on either side of a chunk boundary
    // are written by both chunks during the sweep, so both read them from a
    // copy taken before it (planes 2b and 2b+1 of the copy: zb-1 and zb for
    // the boundary zb between chunks b and b+1); -1 for a plane read from f.
    __device__ __forceinline__ int zcopy_plane(int q) const
    {
        if (jc > 0 && (q == zc0 - 1 || q == zc0)) return 2 * (jc - 1) + (q - zc0 + 1);
        if (jc < nzc - 1 && (q == zc1 - 1 || q == zc1)) return 2 * jc + (q - zc1 + 1);
        return -1;
    }

    // Halo warps: start the copies of plane q into its stage slot.
    __device__ __forceinline__ void issue_stage(int q)
    {
        uint64_t *b = &bar[(q - qb) & 1];
        T *tb = tile_block(q);
        const int pz = phys(q);
        if (hidx == 0) {
            mbar_arrive_expect_tx(b, SM::tma_bytes);
            const int zq = CHUNK ? zcopy_plane(q) : -1;
            const CUtensorMap *mp = zq >= 0 ? tmapz : tmap;
            const int zz = zq >= 0 ? zq : pz;
            for (int d = 0; d < Q; ++d) tma_load_4d(tb + d * DST, mp, x0, y0, zz, d, b);
        }
        // the tile's own shell cells: 16-byte chunks of its shadow rows
        const T *gs = Gc + pz * si.gplane + (int64_t)(blockIdx.y * si.ntx + blockIdx.x) * Q * NSP;
        for (int ch = hidx; ch < Q * SM::CHUNKS; ch += NHT) {
            const int d = ch / SM::CHUNKS, j = ch - d * SM::CHUNKS;
            cp_async_cg16(reinterpret_cast<unsigned char *>(tb + d * DST + NT) + 16 * j,
                      reinterpret_cast<const unsigned char *>(gs + d * NSP) + 16 * j);
        }
        // this thread's halo cell: the copy unit holding each direction
        if (active) {
            const T *hs = Gc + pz * si.gplane + (goff - sub);
            unsigned char *hb = halo_block(q) + hidx * CP;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                cp_async<CP>(hb + i * NHT * CP, hs + i * NSP);
            });
        }
        cp_async_mbar_arrive(b);
        if (hidx == 0) ++*issued;  // stages issued so far (read when bailing out)
    }

    __device__ __forceinline__ void wait_stage(int q)
    {
        const int u = q - qb;
        if (!mbar_wait_bounded(&bar[u & 1], (unsigned)((u >> 1) & 1))) timed_out = true;
    }

    // Even step of plane q (even and halo warps): collide, hand every value
    // to its ring.
    __device__ __forceinline__ void produce(int q)
    {
        if (!active) return;
        R s[Q];
        if (role == EVEN) {
            const T *in = tile_block(q) + inoff;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = decode<S, i>(in[i * DST]);
            });
        } else {
            const unsigned char *hb = halo_block(q) + hidx * CP;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = decode<S, i>(reinterpret_cast<const T *>(hb + i * NHT * CP)[sub]);
            });
        }
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, phys(q)), ncanon(g), Fx, Fy, Fz);
        bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
        // value that leaves along c_i as the next step reads it: + L_opp(i)
        // on a wall link that ends on a lid
        const unsigned lm = lxy | (q == 0 && g.lid[4] ? CZM : 0u) | (q == nz - 1 && g.lid[5] ? CZP : 0u);
        if (lm) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                if (lm & (1u << i)) s[i] = radd(s[i], g.L[opp(i)]);
            });
        }
        R *zs = nullptr;
        if constexpr (PERZ)
            if (q <= 0) zs = zsave + (q + 1) * (L::NXY * NPOS + 3 * L::NTS);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            const R v = roundtrip<S, i>(s[i]);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                ring_at<gg>(q, gidx(i))[pos] = v;
                if constexpr (PERZ)
                    if (zs) zs[xyidx(i) * NPOS + pos] = v;
            } else if (role == EVEN) {
                if constexpr (i == 0) srest[slot(q, L::SREST) * L::NTS + tc] = v;
                else if constexpr (i == DIR_ZP) szp[slot(q, L::SZP) * L::NTS + tc] = v;
                else szm[slot(q, L::SZM) * L::NTS + tc] = v;
                if constexpr (PERZ) {
                    constexpr int sm = i == 0 ? 0 : (i == DIR_ZP ? 1 : 2);
                    if (zs) zs[L::NXY * NPOS + sm * L::NTS + tc] = v;
                }
            }
        });
    }

    // Periodic z, planes nz-1 and nz at the end of the march: the values of
    // their images -1 and 0, computed before any odd step wrote into them.
    __device__ __forceinline__ void restore(int q)
    {
        if constexpr (!PERZ) return;
        if (!active) return;
        const R *zs = zsave + (q - nz + 1) * (L::NXY * NPOS + 3 * L::NTS);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                ring_at<gg>(q, gidx(i))[pos] = zs[xyidx(i) * NPOS + pos];
            } else if (role == EVEN) {
                constexpr int sm = i == 0 ? 0 : (i == DIR_ZP ? 1 : 2);
                const R v = zs[L::NXY * NPOS + sm * L::NTS + tc];
                if constexpr (i == 0) srest[slot(q, L::SREST) * L::NTS + tc] = v;
                else if constexpr (i == DIR_ZP) szp[slot(q, L::SZP) * L::NTS + tc] = v;
                else szm[slot(q, L::SZM) * L::NTS + tc] = v;
            }
        });
    }

    // Odd step of plane k (odd warps, active threads): gather and collide;
    // scatter() writes the result one interval later.
    __device__ __forceinline__ void consume(int k, R (&s)[Q]) const
    {
        const bool zlo = !PERZ && k == 0, zhi = !PERZ && k == nz - 1;
        const unsigned wm = wxy | (zlo ? CZM : 0u) | (zhi ? CZP : 0u);
        s[0] = srest[slot(k, L::SREST) * L::NTS + tc];
        s[DIR_ZP] = zlo ? szm[slot(k, L::SZM) * L::NTS + tc] : szp[slot(k - 1, L::SZP) * L::NTS + tc];
        s[DIR_ZM] = zhi ? szp[slot(k, L::SZP) * L::NTS + tc] : szm[slot(k + 1, L::SZM) * L::NTS + tc];
        if (!wm) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                constexpr int gg = grp(i);
                if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P)
                    s[i] = ring_at<gg>(k - cz(i), gidx(i))[pos - cx(i) - cy(i) * W];
            });
        } else {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                constexpr int gg = grp(i);
                if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                    if (wm & (1u << opp(i))) s[i] = ring_at<grp(opp(i))>(k, gidx(opp(i)))[pos];
                    else s[i] = ring_at<gg>(k - cz(i), gidx(i))[pos - cx(i) - cy(i) * W];
                }
            });
        }
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, k), ncanon(g), Fx, Fy, Fz);
        bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
    }

    // Push the odd-step result of plane k into f and, for targets on a
    // shell, into the next shadow.

    __device__ __forceinline__ void scatter(int k, const R (&s)[Q]) const
    {
        const int c = cxy + k * (int)g.plane;
        const int kg = k * (int)si.gplane;  // shadow sizes stay below 2^31 elements
        T *const gk = Gn + kg;
        if (!xybnd && k > 0 && k < nz - 1) {
            if (!gmask) {  // inner cells: no shell target
                static_for<Q>([&](auto K) {
                    constexpr int i = decltype(K)::value;
                    st_no_l1(&fo.p[i][c], encode<S, i>(s[i]));
                });
            } else {
                // shadow offsets of the 3 x 3 neighbourhood, loaded together
                // (19 directions share 9 targets in the plane)
                int gt[9];
#pragma unroll
                for (int j = 0; j < 9; ++j) gt[j] = gtab[pos + (j % 3 - 1) + (j / 3 - 1) * W];
                static_for<Q>([&](auto K) {
                    constexpr int i = decltype(K)::value;
                    const T e = encode<S, i>(s[i]);
                    st_no_l1(&fo.p[i][c], e);
                    if (gmask & (1u << i)) st_no_l1(&go.p[i][kg + gt[(cx(i) + 1) + (cy(i) + 1) * 3]], e);
                });
            }
        } else {
            const Faces fc = faces_of(g, x, y, k);
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                constexpr unsigned m = face_mask(cx(i), cy(i), cz(i));
                if (fc.wall & m) {
                    R v = s[i];
                    if (fc.lid & m) v = radd(v, g.L[opp(i)]);
                    const T e = encode<S, opp(i)>(v);
                    fd.p[opp(i)][c] = e;
                    if (goff >= 0) gk[goff + opp(i) * NSP] = e;
                } else {
                    const T e = encode<S, i>(s[i]);
                    fd.p[i][c + step_offset<cx(i), cy(i), cz(i)>(g, fc)] = e;
                    const int t = gtab[pos + cx(i) + cy(i) * W];
                    if (t >= 0) Gn[phys(k + cz(i)) * si.gplane + t + i * NSP] = e;
                }
            });
        }
    }
};

template <class S, bool FORCE, int TY, bool PERZ, bool CHUNK>
__global__ void __launch_bounds__(M3<TY>::THREADS, 1)
    k_merged3(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmapz,
              Geom<typename S::R> g, Dirs<typename S::T> fd, Dirs<typename S::T> fo, Dirs<typename S::T> go,
              const typename S::T *__restrict__ Gc, typename S::T *__restrict__ Gn, ShellInfo si,
              typename S::R *__restrict__ zsave, int *__restrict__ status)
{
    static_assert(!(PERZ && CHUNK), "a periodic z march is not split");
    using C = M3Cta<S, FORCE, TY, PERZ, CHUNK>;
    using SM = typename C::SM;
    extern __shared__ __align__(128) unsigned char smem[];
    C c(g, fd, fo, go, Gc, Gn, si, &tmap, zsave, smem);
    c.tmapz = &tmapz;
    int *abort_flag = reinterpret_cast<int *>(smem + SM::flag_off);
    c.issued = abort_flag + 1;
    const int nz = g.nz;
    if (threadIdx.x == 0) {
        mbar_init(&c.bar[0], 1 + M3<TY>::NHT);
        mbar_init(&c.bar[1], 1 + M3<TY>::NHT);
        mbar_fence_init();
        *abort_flag = 0;
        *c.issued = 0;
    }
    c.fill_gtab();
    __syncthreads();
    c.setup();
    // z chunk blockIdx.z of si.nzc (one chunk with periodic z): odd steps of
    // planes [zc0, zc1), even steps of the loaded planes qb .. last, one
    // plane beyond the chunk on either side where it has a neighbour.  With
    // periodic z the planes -1 .. nz-2 are loaded and nz-1, nz restored.
    c.nzc = CHUNK ? si.nzc : 1;
    c.jc = CHUNK ? (int)blockIdx.z : 0;
    c.zc0 = CHUNK ? (int)((int64_t)c.jc * nz / c.nzc) : 0;
    c.zc1 = CHUNK ? (int)((int64_t)(c.jc + 1) * nz / c.nzc) : nz;
    c.qb = PERZ ? -1 : (CHUNK && c.zc0 > 0 ? c.zc0 - 1 : 0);
    const int last = PERZ ? nz - 2 : (CHUNK && c.zc1 < nz ? c.zc1 : nz - 1);
    const int kend = CHUNK ? c.zc1 : nz;
    // interval k: even and halo warps collide plane k+2, odd warps plane k;
    // the halo warps start loading plane k+3 into the slot plane k+1 freed.
    // The roles run separate loops over the same intervals (one barrier
    // each); odd warps store plane k-1 at the start of interval k, so that
    // its stores drain while they collide plane k, not at the barrier.
    if (c.role == C::ODD) {
        typename S::R sk[Q];
        bool held = false;
        for (int k = c.qb - 2; k < kend; ++k) {
            if (held) c.scatter(k - 1, sk);
            held = k >= c.zc0 && c.active;
            if (held) c.consume(k, sk);
            cta_barrier();
            if (*abort_flag) goto bail;
        }
        if (held) c.scatter(kend - 1, sk);
        return;
    }
    if (c.role == C::HALO) c.issue_stage(c.qb);
    for (int k = c.qb - 2; k < kend; ++k) {
        const int q = k + 2;
        if (c.role == C::HALO && q + 1 <= last) c.issue_stage(q + 1);
        if (q <= last) {
            c.wait_stage(q);
            if (!c.timed_out) c.produce(q);
        } else if (PERZ && q <= nz) {
            c.restore(q);
        }
        if (c.timed_out) *abort_flag = 1;
        cta_barrier();
        if (*abort_flag) goto bail;
    }
    return;

bail:
    // a stage never completed: record it, drain the copies still in flight
    // (bounded) and leave without touching the lattice again.  Only the last
    // two issued stages can still be in flight; stage u completes phase
    // (u >> 1) & 1 of the mbarrier of slot u & 1, and no later stage has been
    // issued into either slot.  Every thread drains its own cp.async copies,
    // which were never committed to a group (they arrive on the mbarrier).
    if (threadIdx.x == 0) {
        atomicOr(status, 2);
        const int n = *c.issued;
        for (int u = n - 2 > 0 ? n - 2 : 0; u < n; ++u) mbar_wait_bounded(&c.bar[u & 1], (unsigned)((u >> 1) & 1));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace lbm
