// merged.cuh -- two collision-streaming steps per sweep (K4) and the shell
// snapshot that makes the in-place sweep safe between tiles.
//
// The paper merges steps t and t+1 of a cell as soon as every neighbour it
// depends on has finished step t (Sec. 4.1, Alg. 2: the second computation
// of cell (iX-1, iY-1, iZ-1)), and protects the layers where two threads'
// sub-domains meet by processing them first (Stage I of Alg. 3, Sec. 4.2).
// On the GPU:
//
//  * A CTA owns a TX x TY column of cells and marches it along z.  At
//    iteration k it performs the even (local) half of the AA pair on plane
//    k+1 and the odd half on plane k, whose inputs -- the post-collision
//    values of the 3x3x3 neighbourhood -- all exist by then.
//  * Plane k+1 arrives through a TMA tensor copy (all 19 directions of the
//    tile in one cp.async.bulk.tensor.4d) issued two iterations ahead into a
//    two-stage shared-memory pipeline guarded by mbarriers.
//  * Post-collision values travel between threads through shared-memory
//    rings indexed by the producing cell (with a one-cell halo ring), one
//    ring per z-group of directions sized to how long its values live:
//    c_z = -1 values are consumed in the iteration that produces them, c_z
//    = 0 one iteration later, c_z = +1 two iterations later.  The rest
//    population and the two pure-z directions stay in registers.  One
//    __syncthreads per plane orders producers and consumers.
//  * Cells on the boundary of a tile are read by two CTAs and written by
//    both.  Before the sweep, k_snapshot stores the post-collision values of
//    every shell cell (tile rows/columns next to another tile, and the
//    planes z = 0, nz-1 when z is periodic) in G.  During the sweep a CTA
//    takes its own shell cells and its neighbours' halo values from G (via
//    cp.async two planes ahead) and never from f, so it cannot see what
//    another CTA has already written there -- the GPU counterpart of the
//    intersection layers of Alg. 3 (Stage I).
//  * Wall links bounce inside the CTA: the value a wall link returns is the
//    producer's own outgoing value (lid term already added), read back from
//    the ring at the producer's own position.
//
// Per two steps the sweep reads and writes every population once (2 x 19 x
// sizeof(T) bytes per cell, the bytes of a single AA step), plus the shell
// traffic of the snapshot.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace lbm {

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the barrier did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ------------------------------------------------- direction groups of K4
enum { GRP_REST = 0, GRP_ZM = 1, GRP_ZP = 2, GRP_M = 3, GRP_0 = 4, GRP_P = 5 };
__host__ __device__ constexpr int grp(int i)
{
    return i == 0 ? GRP_REST
         : (cx(i) == 0 && cy(i) == 0) ? (cz(i) < 0 ? GRP_ZM : GRP_ZP)
         : cz(i) < 0 ? GRP_M : (cz(i) == 0 ? GRP_0 : GRP_P);
}
__host__ __device__ constexpr int gidx(int i)
{
    int n = 0;
    for (int j = 0; j < i; ++j)
        if (grp(j) == grp(i)) ++n;
    return n;
}
constexpr int DIR_ZM = 1, DIR_ZP = 10;  // the pure-z directions in this numbering
static_assert(grp(DIR_ZM) == GRP_ZM && grp(DIR_ZP) == GRP_ZP, "pure-z direction indices");
constexpr int NDM = 4, ND0 = 8, NDP = 4;      // xy-moving directions per z-group
constexpr int SLM = 2, SL0 = 3, SLP = 4;      // ring slots per z-group
constexpr int STAGES = 2;                     // TMA pipeline depth

template <int TX, int TY, class T, class R>
struct MergedSmem {
    static constexpr int NT = TX * TY;
    static constexpr int W = TX + 2, H = TY + 2, NPOS = W * H;
    static constexpr int NE = 2 * TX + 2 * TY;  // edge cells (own-shell staging slots)
    static constexpr size_t stage_off = 0;
    static constexpr size_t stage_bytes = (size_t)STAGES * Q * NT * sizeof(T);
    static constexpr size_t ringm_off = (stage_off + stage_bytes + 127) / 128 * 128;
    static constexpr size_t ring0_off = ringm_off + (size_t)SLM * NDM * NPOS * sizeof(R);
    static constexpr size_t ringp_off = ring0_off + (size_t)SL0 * ND0 * NPOS * sizeof(R);
    static constexpr size_t shell_off = ringp_off + (size_t)SLP * NDP * NPOS * sizeof(R);
    static constexpr size_t bar_off = (shell_off + (size_t)2 * Q * NE * sizeof(R) + 15) / 16 * 16;
    static constexpr size_t flag_off = bar_off + STAGES * sizeof(uint64_t);
    static constexpr size_t bytes = flag_off + 16;
};

// Shell rows / columns: the first and last row of every tile that touches
// another tile (across a periodic face too).  Snapshot buffers (compute type):
//   GY[q][z][2*nty][nx]   rows (side 0 = first row of the tile, 1 = last)
//   GX[q][z][2*ntx][ny]   columns
//   GZ[q][2][ny][nx]      planes z = 0 and z = nz-1 (periodic z only)
template <class R>
__device__ __forceinline__ bool row_is_shell(const Geom<R> &g, const TileInfo &ti, int tile, int side)
{
    return ti.yshell && (side == 0 ? (tile > 0 || g.per[1]) : (tile < ti.nty - 1 || g.per[1]));
}
template <class R>
__device__ __forceinline__ bool col_is_shell(const Geom<R> &g, const TileInfo &ti, int tile, int side)
{
    return ti.xshell && (side == 0 ? (tile > 0 || g.per[0]) : (tile < ti.ntx - 1 || g.per[0]));
}

// Post-collision value that leaves (x,y,z) along c_i, as the next step reads
// it: f*_i, or f*_i + L_opp(i) when the link ends on a moving lid.
template <class S>
__device__ __forceinline__ void outgoing_values(const Geom<typename S::R> &g, int x, int y, int z,
                                                typename S::R (&s)[Q])
{
    if (interior(g, x, y, z)) return;
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        int tx, ty, tz;
        bool lid;
        if (!link(g, x, y, z, cx(i), cy(i), cz(i), tx, ty, tz, lid) && lid) s[i] = radd(s[i], g.L[opp(i)]);
    });
}

template <class S, bool FORCE>
__global__ void __launch_bounds__(256) k_snapshot(Geom<typename S::R> g, const typename S::T *__restrict__ f,
                                                  typename S::R *__restrict__ G, TileInfo ti, int64_t cnt_z,
                                                  int64_t cnt_y, int64_t cnt_x)
{
    using R = typename S::R;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int x, y, z;
    int64_t base, sl;
    if (idx < cnt_z) {
        const int64_t pl = (int64_t)g.ny * g.nx;
        const int zi = (int)(idx / pl);
        const int64_t r = idx % pl;
        y = (int)(r / g.nx);
        x = (int)(r % g.nx);
        z = zi ? g.nz - 1 : 0;
        base = ti.gz_off + idx;
        sl = ti.gz_slot;
    } else if (idx < cnt_z + cnt_y) {
        const int64_t j = idx - cnt_z;
        const int64_t rowlen = 2LL * ti.nty * g.nx;
        z = (int)(j / rowlen);
        const int64_t r = j % rowlen;
        const int row = (int)(r / g.nx);
        x = (int)(r % g.nx);
        const int tile = row >> 1, side = row & 1;
        if (!row_is_shell(g, ti, tile, side)) return;
        y = side ? min(g.ny, (tile + 1) * ti.TY) - 1 : tile * ti.TY;
        base = ti.gy_off + j;
        sl = ti.gy_slot;
    } else if (idx < cnt_z + cnt_y + cnt_x) {
        const int64_t j = idx - cnt_z - cnt_y;
        const int64_t collen = 2LL * ti.ntx * g.ny;
        z = (int)(j / collen);
        const int64_t r = j % collen;
        const int col = (int)(r / g.ny);
        y = (int)(r % g.ny);
        const int tile = col >> 1, side = col & 1;
        if (!col_is_shell(g, ti, tile, side)) return;
        x = side ? min(g.nx, (tile + 1) * ti.TX) - 1 : tile * ti.TX;
        base = ti.gx_off + j;
        sl = ti.gx_slot;
    } else {
        return;
    }
    R s[Q];
    load_natural<S>(g, f, x, y, z, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
    outgoing_values<S>(g, x, y, z, s);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        G[base + i * sl] = roundtrip<S, i>(s[i]);
    });
}

// Per-thread state and the phases of one CTA of the merged sweep.
template <class S, bool FORCE, int TX, int TY>
struct MergedCta {
    using R = typename S::R;
    using T = typename S::T;
    using L = MergedSmem<TX, TY, T, R>;
    static constexpr int NT = L::NT, W = L::W, NPOS = L::NPOS, NE = L::NE;
    static constexpr unsigned STAGE_BYTES = (unsigned)(Q * NT * sizeof(T));

    const CUtensorMap *tmap;
    const Geom<R> &g;
    const Dirs<T> &fd;
    const R *__restrict__ G;
    const TileInfo &ti;
    T *stage;
    R *ringm, *ring0, *ringp, *shellst;
    uint64_t *bar;
    int tx, ty, tid, bxi, byi, x0, y0, x1, y1, x, y, pos, nx, ny, nz, eidx;
    bool active, perx, pery, perz, ysh_lo, ysh_hi, xsh_lo, xsh_hi, own_shell, wxl, wxh, wyl, wyh, xywall, dupx,
        dupy, edge, timed_out;
    R rest_c, rest_n, zp1, zp0, zp_n, zm_prev, zm_n;  // rest and pure-z populations carried in registers

    __device__ __forceinline__ MergedCta(const CUtensorMap *tmap_, const Geom<R> &g_, const Dirs<T> &fd_, const R *G_,
                                         const TileInfo &ti_, unsigned char *smem)
        : tmap(tmap_), g(g_), fd(fd_), G(G_), ti(ti_)
    {
        stage = reinterpret_cast<T *>(smem + L::stage_off);
        ringm = reinterpret_cast<R *>(smem + L::ringm_off);
        ring0 = reinterpret_cast<R *>(smem + L::ring0_off);
        ringp = reinterpret_cast<R *>(smem + L::ringp_off);
        shellst = reinterpret_cast<R *>(smem + L::shell_off);
        bar = reinterpret_cast<uint64_t *>(smem + L::bar_off);
        tx = threadIdx.x; ty = threadIdx.y; tid = ty * TX + tx;
        bxi = blockIdx.x; byi = blockIdx.y;
        x0 = bxi * TX; y0 = byi * TY;
        nx = g.nx; ny = g.ny; nz = g.nz;
        x1 = min(nx, x0 + TX) - 1; y1 = min(ny, y0 + TY) - 1;
        x = x0 + tx; y = y0 + ty;
        active = x <= x1 && y <= y1;
        pos = (ty + 1) * W + (tx + 1);
        perx = g.per[0] != 0; pery = g.per[1] != 0; perz = g.per[2] != 0;
        ysh_lo = active && y == y0 && row_is_shell(g, ti, byi, 0);
        ysh_hi = active && y == y1 && row_is_shell(g, ti, byi, 1);
        xsh_lo = active && x == x0 && col_is_shell(g, ti, bxi, 0);
        xsh_hi = active && x == x1 && col_is_shell(g, ti, bxi, 1);
        own_shell = ysh_lo || ysh_hi || xsh_lo || xsh_hi;
        eidx = ty == 0 ? tx : (y == y1 ? TX + tx : (tx == 0 ? 2 * TX + ty : 2 * TX + TY + ty));
        wxl = active && x == 0 && !perx; wxh = active && x == nx - 1 && !perx;
        wyl = active && y == 0 && !pery; wyh = active && y == ny - 1 && !pery;
        xywall = wxl || wxh || wyl || wyh;
        dupx = active && perx && ti.ntx == 1 && (x == 0 || x == nx - 1);
        dupy = active && pery && ti.nty == 1 && (y == 0 || y == ny - 1);
        edge = active && (x == x0 || x == x1 || y == y0 || y == y1);
        timed_out = false;
        rest_c = rest_n = zp1 = zp0 = zp_n = zm_prev = zm_n = R(0);
    }

    __device__ __forceinline__ static int slot(int plane, int n) { return (plane + n) % n; }
    template <int GG>
    __device__ __forceinline__ R *ring_at(int plane, int gi) const
    {
        if constexpr (GG == GRP_M) return ringm + (slot(plane, SLM) * NDM + gi) * NPOS;
        else if constexpr (GG == GRP_0) return ring0 + (slot(plane, SL0) * ND0 + gi) * NPOS;
        else return ringp + (slot(plane, SLP) * NDP + gi) * NPOS;
    }
    __device__ __forceinline__ bool in_tile(int px, int py) const { return px >= x0 && px <= x1 && py >= y0 && py <= y1; }
    __device__ __forceinline__ static int wrap(int v, int n, bool per, bool &out)
    {
        out = false;
        if (v < 0 || v >= n) {
            if (per) v = v < 0 ? v + n : v - n;
            else out = true;
        }
        return v;
    }

    // ------------------------------------------------------------ TMA
    __device__ __forceinline__ void issue_tma(int plane)  // one thread
    {
        if (plane < 0 || plane >= nz) return;
        const int s = plane % STAGES;
        mbar_arrive_expect_tx(&bar[s], STAGE_BYTES);
        tma_load_4d(stage + (size_t)s * Q * NT, tmap, x0, y0, plane, 0, &bar[s]);
    }
    __device__ __forceinline__ void wait_tma(int plane)
    {
        if (plane < 0 || plane >= nz) return;
        if (!mbar_wait_bounded(&bar[plane % STAGES], (unsigned)((plane / STAGES) & 1))) timed_out = true;
    }

    // ------------------------------------------------- G prefetching
    // Halo values of plane p at halo position (hx, hy): the inward directions
    // of the neighbouring tile's shell cell, from G.
    __device__ __forceinline__ void fill_halo(int p, int pr, int hx, int hy)
    {
        bool ox, oy;
        const int sx = wrap(hx, nx, perx, ox), sy = wrap(hy, ny, pery, oy);
        if (ox || oy || in_tile(sx, sy)) return;  // wall, or an image inside this tile
        // a source in another row of tiles is on that tile's first or last
        // row (row snapshot); otherwise it is on an edge column of the tile
        // beside this one (column snapshot)
        int64_t base, sl;
        if (sy < y0 || sy > y1) {
            base = ti.gy_off + ((int64_t)pr * 2 * ti.nty + 2 * (sy / TY) + (hy < y0 ? 1 : 0)) * nx + sx;
            sl = ti.gy_slot;
        } else {
            base = ti.gx_off + ((int64_t)pr * 2 * ti.ntx + 2 * (sx / TX) + (hx < x0 ? 1 : 0)) * ny + sy;
            sl = ti.gx_slot;
        }
        const int hpos = (hy - y0 + 1) * W + (hx - x0 + 1);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                if ((p < 0 && gg != GRP_P) || (p >= nz && gg != GRP_M)) return;
                if (!in_tile(hx + cx(i), hy + cy(i))) return;
                cp_async<sizeof(R)>(ring_at<gg>(p, gidx(i)) + hpos, G + base + i * sl);
            }
        });
    }
    // Everything plane p needs from G that this thread fetches: its own
    // shell values and the halo positions next to it.
    __device__ __forceinline__ void prefetch(int p)
    {
        if (!edge) return;
        if (p < -1 || p > nz || ((p < 0 || p >= nz) && !perz)) return;
        const int pr = p < 0 ? p + nz : (p >= nz ? p - nz : p);
        const bool zsnap = ti.zshell && (pr == 0 || pr == nz - 1);
        if (own_shell && !zsnap && p >= 0 && p < nz) {
            int64_t base, sl;
            if (ysh_lo || ysh_hi) {
                base = ti.gy_off + ((int64_t)pr * 2 * ti.nty + 2 * byi + (ysh_lo ? 0 : 1)) * nx + x;
                sl = ti.gy_slot;
            } else {
                base = ti.gx_off + ((int64_t)pr * 2 * ti.ntx + 2 * bxi + (xsh_lo ? 0 : 1)) * ny + y;
                sl = ti.gx_slot;
            }
            R *dst = shellst + (size_t)(p & 1) * Q * NE + eidx;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                cp_async<sizeof(R)>(dst + i * NE, G + base + i * sl);
            });
        }
        if (x == x0) fill_halo(p, pr, x0 - 1, y);
        if (x == x1) fill_halo(p, pr, x1 + 1, y);
        if (y == y0) {
            fill_halo(p, pr, x, y0 - 1);
            if (x == x0) fill_halo(p, pr, x0 - 1, y0 - 1);
            if (x == x1) fill_halo(p, pr, x1 + 1, y0 - 1);
        }
        if (y == y1) {
            fill_halo(p, pr, x, y1 + 1);
            if (x == x0) fill_halo(p, pr, x0 - 1, y1 + 1);
            if (x == x1) fill_halo(p, pr, x1 + 1, y1 + 1);
        }
    }

    // ---------------------------------------------------- even step
    // Even step of virtual plane q (q = -1 / nz are the periodic images of
    // nz-1 / 0): collide, then hand every value to the ring of its z-group.
    __device__ __forceinline__ void produce(int q)
    {
        if (!active) return;
        const int zr = q < 0 ? q + nz : (q >= nz ? q - nz : q);
        const bool zsnap = ti.zshell && (zr == 0 || zr == nz - 1);
        R s[Q];
        if (zsnap) {
            const int64_t base = ti.gz_off + ((int64_t)(zr == 0 ? 0 : 1) * ny + y) * nx + x;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = G[base + i * ti.gz_slot];
            });
        } else if (own_shell) {
            const R *src = shellst + (size_t)(q & 1) * Q * NE + eidx;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = src[i * NE];
            });
        } else {
            const T *src = stage + (size_t)(q % STAGES) * Q * NT + tid;
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = decode<S, i>(src[i * NT]);
            });
            R Fx, Fy, Fz;
            force_at<R, FORCE>(g, canon(g, x, y, zr), ncanon(g), Fx, Fy, Fz);
            bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
            outgoing_values<S>(g, x, y, zr, s);
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = roundtrip<S, i>(s[i]);
            });
        }
        rest_n = s[0];
        zm_n = s[DIR_ZM];
        zp_n = s[DIR_ZP];
        const bool vlo = q < 0, vhi = q >= nz;
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                if ((vlo && gg != GRP_P) || (vhi && gg != GRP_M)) return;
                R *r = ring_at<gg>(q, gidx(i));
                r[pos] = s[i];
                if ((cx(i) != 0 && dupx) || (cy(i) != 0 && dupy)) {
                    bool ox, oy;
                    const int tx2 = wrap(x + cx(i), nx, perx, ox), ty2 = wrap(y + cy(i), ny, pery, oy);
                    if (!ox && !oy && (tx2 != x + cx(i) || ty2 != y + cy(i)) && in_tile(tx2, ty2))
                        r[(ty2 - cy(i) - y0 + 1) * W + (tx2 - cx(i) - x0 + 1)] = s[i];
                }
            }
        });
    }

    // ----------------------------------------------------- odd step
    // Odd step of plane k: gather from the rings (own outgoing values for
    // wall links), collide, scatter into f.
    __device__ __forceinline__ void consume(int k)
    {
        if (!active) return;
        const bool zlo = k == 0 && !perz, zhi = k == nz - 1 && !perz;
        R s[Q];
        s[0] = rest_c;
        s[DIR_ZP] = zlo ? zm_prev : zp1;
        s[DIR_ZM] = zhi ? zp0 : zm_n;
        if (!(xywall || zlo || zhi)) {
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
        push_store_d<S>(g, fd, x, y, k, cell32(g, x, y, k), s);
    }

    __device__ __forceinline__ void rotate()
    {
        rest_c = rest_n;
        zp1 = zp0;
        zp0 = zp_n;
        zm_prev = zm_n;
    }
};

template <class S, bool FORCE, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 1) k_merged(const __grid_constant__ CUtensorMap tmap,
                                                       Geom<typename S::R> g, Dirs<typename S::T> fd,
                                                       const typename S::R *__restrict__ G, TileInfo ti,
                                                       int *__restrict__ status)
{
    using C = MergedCta<S, FORCE, TX, TY>;
    extern __shared__ __align__(128) unsigned char smem[];
    int *abort_flag = reinterpret_cast<int *>(smem + C::L::flag_off);
    C c(&tmap, g, fd, G, ti, smem);
    const int nz = g.nz;

    if (c.tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&c.bar[s], 1);
        mbar_fence_init();
        *abort_flag = 0;
    }
    __syncthreads();

    // prologue: planes -1 (periodic z), 0 and 1 in flight, planes -1 and 0
    // collided and distributed
    if (c.tid == 0) {
        c.issue_tma(0);
        c.issue_tma(1);
    }
    if (c.perz) c.prefetch(-1);
    c.prefetch(0);
    c.prefetch(1);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (c.perz) {
        c.produce(-1);
        c.rotate();
    }
    c.wait_tma(0);
    if (c.timed_out) *abort_flag = 1;
    __syncthreads();
    if (*abort_flag) goto bail;
    c.produce(0);
    c.rotate();
    __syncthreads();
    if (c.tid == 0) c.issue_tma(2);

    // z march: iteration k collides plane k+1 (even) and plane k (odd)
    for (int k = 0; k < nz; ++k) {
        const int q = k + 1;
        if (q < nz || c.perz) {
            cp_async_wait_all();
            c.wait_tma(q);
            c.produce(q);
        }
        if (c.timed_out) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) goto bail;
        if (c.tid == 0) c.issue_tma(k + 3);
        c.prefetch(k + 2);
        cp_async_commit();
        c.consume(k);
        c.rotate();
    }
    cp_async_wait_all();
    return;

bail:
    // a TMA copy never completed: record it, drain what is still in flight
    // (bounded) and leave without touching the lattice again
    if (c.tid == 0) {
        atomicOr(status, 2);
        for (int s = 0; s < STAGES; ++s) mbar_wait_bounded(&c.bar[s], 0);
    }
    cp_async_wait_all();
}

}  // namespace lbm
