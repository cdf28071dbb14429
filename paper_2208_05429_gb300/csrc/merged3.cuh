// merged3.cuh -- two collision-streaming steps per sweep with a shadow copy
// of the tile shells (the MERGED schedule on a lattice whose z faces are
// walls).
//
// The paper merges two time steps of a cell as soon as its neighbours have
// done the first one (Sec. 4.1, Alg. 2), and makes the layers where two
// threads' sub-domains meet safe by handling them apart (the intersection
// layers of Alg. 3, Sec. 4.2).  Here:
//
//  * A CTA owns a column of 32 x TH cells (TH <= TY, the rows of the plane
//    split into bands of near-equal height) and marches it along z.  At
//    iteration k it performs the even (local) half of the AA pair on plane
//    k+1 and the odd half on plane k.  Post-collision values move between
//    threads through shared-memory rings (one per z-group of directions,
//    sized to how long the values live) covering the tile and a one-cell
//    halo ring; the rest population and the pure-z directions stay in
//    registers.  One __syncthreads per plane.
//  * Cells on a tile's boundary ring ("shell" cells) are read by up to four
//    CTAs: the owner and the neighbours whose halo they are.  Every shell
//    cell also lives in a double-buffered shadow G: a sweep takes shell and
//    halo inputs from G_cur (never from f, which other CTAs are already
//    overwriting) and writes every post-stream value that lands on a shell
//    cell to G_next as well as to f.  No CTA reads what another CTA writes
//    during the sweep, so tiles need no synchronisation at all, and f stays
//    the complete state after every sweep.
//  * The halo ring is collided again by dedicated halo warps from G_cur
//    (2 x 34 + 2 x TY cells, three warps for TY = 14), so the tile warps
//    run without divergent halo code.
//  * Inputs are loaded straight into registers one plane ahead (coalesced
//    32-wide rows of f; G rows of the tile's shell slots).
//
// HBM traffic per two steps: every population read and written once, plus
// the shell shadow (read once by its owner, written once): 2 x 19 x
// sizeof(T) x (1 + NS/cells-per-tile) bytes per cell.
#pragma once

#include "merged.cuh"

namespace lbm {

template <int TY>
struct M3 {
    static constexpr int TX = 32, W = TX + 2, H = TY + 2, NPOS = W * H;
    static constexpr int NT = TX * TY;
    static constexpr int NH = 2 * W + 2 * TY;  // halo ring cells
    static constexpr int NHW = (NH + 31) / 32;  // halo warps
    static constexpr int THREADS = NT + 32 * NHW;
    static constexpr int NS = 2 * TX + 2 * (TY - 2);  // shell slots of a full tile
    static constexpr int NSP = (NS + 7) / 8 * 8;
    static constexpr int NRING = SLM * NDM + SL0 * ND0 + SLP * NDP;
    template <class R>
    static constexpr size_t smem() { return (size_t)NRING * NPOS * sizeof(R) + (size_t)NPOS * sizeof(int); }
    static_assert(TY >= 2, "bands of at least two rows");
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

template <class S, bool FORCE, int TY>
struct Merged3Cta {
    using R = typename S::R;
    using T = typename S::T;
    using L = M3<TY>;
    static constexpr int W = L::W, NPOS = L::NPOS, NSP = L::NSP;

    const Geom<R> &g;
    const Dirs<T> &fd;
    const T *__restrict__ Gc;
    T *__restrict__ Gn;
    const ShellInfo &si;
    R *ringm, *ring0, *ringp;
    int *gtab;
    int x0, y0, tw, th, lx, ly, x, y, pos, nx, ny, nz, goff, cxy;
    unsigned gmask;
    bool tile_thr, active, perx, pery, wxl, wxh, wyl, wyh, xybnd;
    R rest_c, rest_n, zp1, zp0, zp_n, zm_prev, zm_n;

    __device__ __forceinline__ Merged3Cta(const Geom<R> &g_, const Dirs<T> &fd_, const T *Gc_, T *Gn_,
                                          const ShellInfo &si_, unsigned char *smem)
        : g(g_), fd(fd_), Gc(Gc_), Gn(Gn_), si(si_)
    {
        ringm = reinterpret_cast<R *>(smem);
        ring0 = ringm + SLM * NDM * NPOS;
        ringp = ring0 + SL0 * ND0 * NPOS;
        gtab = reinterpret_cast<int *>(ringp + SLP * NDP * NPOS);
        nx = g.nx; ny = g.ny; nz = g.nz;
        perx = g.per[0] != 0; pery = g.per[1] != 0;
        x0 = 32 * blockIdx.x;
        tw = min(32, nx - x0);
        band_of(si, blockIdx.y, y0, th);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        tile_thr = warp < TY;
        if (tile_thr) {
            lx = lane; ly = warp;
            active = lx < tw && ly < th;
        } else {
            // halo ring: row -1, row th, column -1, column tw
            const int h = (warp - TY) * 32 + lane;
            active = true;
            if (h < W) { lx = h - 1; ly = -1; active = lx <= tw; }
            else if (h < 2 * W) { lx = h - W - 1; ly = th; active = lx <= tw; }
            else if (h < 2 * W + TY) { lx = -1; ly = h - 2 * W; active = ly < th; }
            else if (h < 2 * W + 2 * TY) { lx = tw; ly = h - 2 * W - TY; active = ly < th; }
            else { lx = 0; ly = 0; active = false; }
        }
        pos = (ly + 1) * W + (lx + 1);
        x = x0 + lx; y = y0 + ly;
        if (!tile_thr && active) {  // wrap the halo cell into the domain, or drop it (wall)
            if (x < 0 || x >= nx) { if (perx) x = x < 0 ? x + nx : x - nx; else active = false; }
            if (y < 0 || y >= ny) { if (pery) y = y < 0 ? y + ny : y - ny; else active = false; }
        }
        wxl = tile_thr && x == 0 && !perx; wxh = tile_thr && x == nx - 1 && !perx;
        wyl = tile_thr && y == 0 && !pery; wyh = tile_thr && y == ny - 1 && !pery;
        xybnd = x == 0 || x == nx - 1 || y == 0 || y == ny - 1;
        cxy = active ? y * (int)g.nxp + x : 0;
        rest_c = rest_n = zp1 = zp0 = zp_n = zm_prev = zm_n = R(0);
        goff = -1;
        gmask = 0u;
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

    // After fill_gtab and a barrier: own shadow offset and, for tile
    // threads, the directions whose (non-wall) target is a shell cell.
    __device__ __forceinline__ void setup_masks()
    {
        if (!active) return;
        goff = gtab[pos];
        if (!tile_thr) return;
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if (gtab[pos + cx(i) + cy(i) * W] >= 0) gmask |= 1u << i;
        });
    }

    __device__ __forceinline__ static int slot(int plane, int n) { return (plane + n) % n; }
    template <int GG>
    __device__ __forceinline__ R *ring_at(int plane, int gi) const
    {
        if constexpr (GG == GRP_M) return ringm + (slot(plane, SLM) * NDM + gi) * NPOS;
        else if constexpr (GG == GRP_0) return ring0 + (slot(plane, SL0) * ND0 + gi) * NPOS;
        else return ringp + (slot(plane, SLP) * NDP + gi) * NPOS;
    }

    // Stored inputs of plane z: the shadow for shell and halo cells, f for
    // the inside of the tile.
    __device__ __forceinline__ void load(int z, T (&raw)[Q]) const
    {
        if (!active) return;
        if (goff >= 0) {
            const T *p = Gc + z * si.gplane + goff;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                raw[i] = p[i * NSP];
            });
        } else {
            const int c = cxy + z * (int)g.plane;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                raw[i] = fd.p[i][c];
            });
        }
    }

    // Even step of plane q: collide and hand every value to its ring.
    __device__ __forceinline__ void produce(int q, const T (&raw)[Q])
    {
        if (!active) return;
        R s[Q];
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            s[i] = decode<S, i>(raw[i]);
        });
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, q), ncanon(g), Fx, Fy, Fz);
        bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
        outgoing_values<S>(g, x, y, q, s);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            s[i] = roundtrip<S, i>(s[i]);
        });
        rest_n = s[0];
        zm_n = s[DIR_ZM];
        zp_n = s[DIR_ZP];
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) ring_at<gg>(q, gidx(i))[pos] = s[i];
        });
    }

    // Odd step of plane k: gather, collide, scatter into f and, for targets
    // on a shell, into the next shadow.
    __device__ __forceinline__ void consume(int k)
    {
        if (!active || !tile_thr) return;
        const bool zlo = k == 0, zhi = k == nz - 1;
        R s[Q];
        s[0] = rest_c;
        s[DIR_ZP] = zlo ? zm_prev : zp1;
        s[DIR_ZM] = zhi ? zp0 : zm_n;
        if (!(wxl || wxh || wyl || wyh || zlo || zhi)) {
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
                    const bool wall = (cx(i) == 1 && wxl) || (cx(i) == -1 && wxh) || (cy(i) == 1 && wyl) ||
                                      (cy(i) == -1 && wyh) || (cz(i) == 1 && zlo) || (cz(i) == -1 && zhi);
                    if (!wall) s[i] = ring_at<gg>(k - cz(i), gidx(i))[pos - cx(i) - cy(i) * W];
                    else s[i] = ring_at<grp(opp(i))>(k, gidx(opp(i)))[pos];
                }
            });
        }
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, k), ncanon(g), Fx, Fy, Fz);
        bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
        scatter(k, s);
    }

    __device__ __forceinline__ T *gnext(int z) const { return Gn + z * si.gplane; }

    __device__ __forceinline__ void scatter(int k, const R (&s)[Q]) const
    {
        const int c = cxy + k * (int)g.plane;
        if (!xybnd && k > 0 && k < nz - 1) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                const T e = encode<S, i>(s[i]);
                fd.p[i][c + g.noff[i]] = e;
                if (gmask & (1u << i)) gnext(k + cz(i))[gtab[pos + cx(i) + cy(i) * W] + i * NSP] = e;
            });
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
                    if (goff >= 0) gnext(k)[goff + opp(i) * NSP] = e;
                } else {
                    const T e = encode<S, i>(s[i]);
                    fd.p[i][c + step_offset<cx(i), cy(i), cz(i)>(g, fc)] = e;
                    const int t = gtab[pos + cx(i) + cy(i) * W];
                    if (t >= 0) gnext(k + cz(i))[t + i * NSP] = e;
                }
            });
        }
    }

    __device__ __forceinline__ void rotate()
    {
        rest_c = rest_n;
        zp1 = zp0;
        zp0 = zp_n;
        zm_prev = zm_n;
    }
};

template <class S, bool FORCE, int TY>
__global__ void __launch_bounds__(M3<TY>::THREADS, 1)
    k_merged3(Geom<typename S::R> g, Dirs<typename S::T> fd, const typename S::T *__restrict__ Gc,
              typename S::T *__restrict__ Gn, ShellInfo si)
{
    using C = Merged3Cta<S, FORCE, TY>;
    using T = typename S::T;
    extern __shared__ __align__(128) unsigned char smem[];
    C c(g, fd, Gc, Gn, si, smem);
    const int nz = g.nz;
    c.fill_gtab();
    __syncthreads();
    c.setup_masks();

    T raw[Q], nxt[Q];
    c.load(0, raw);
    if (nz > 1) c.load(1, nxt);
    c.produce(0, raw);
    c.rotate();
    // iteration k: even step of plane k+1, odd step of plane k
    for (int k = 0; k < nz; ++k) {
        const int q = k + 1;
        if (q < nz) {
#pragma unroll
            for (int i = 0; i < Q; ++i) raw[i] = nxt[i];
            if (q + 1 < nz) c.load(q + 1, nxt);
            c.produce(q, raw);
        }
        __syncthreads();
        c.consume(k);
        c.rotate();
    }
}

}  // namespace lbm
