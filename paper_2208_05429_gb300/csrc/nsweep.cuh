// nsweep.cuh -- two collision-streaming steps per sweep, the column tiles
// kept in step by their neighbours' progress (the MERGED schedule on a
// lattice whose six faces are walls or lids).
//
// The paper merges the two time steps of a cell as soon as every neighbour
// it depends on has done the first one (Sec. 4.1, Alg. 2), and keeps the
// layers where two threads' sub-domains meet safe by ordering the threads'
// work on them (the intersection layers of Alg. 3, Sec. 4.2).  On the GPU:
//
//  * One CTA per 32 x TH column tile (TH <= TY; the rows are split into
//    bands of near-equal height, 152 tiles on a 256^2 plane), all CTAs
//    resident at once (cooperative launch), each marching its tile along z.
//  * Plane p arrives in a two-slot stage by ONE TMA tensor copy: the 19
//    directions of the tile plus its one-cell halo ring, a box of
//    (32 + 2 XM) x (TY + 2) cells whose x start lies 16 bytes before the
//    tile (the alignment rule of tiled copies; the extra columns are not
//    used).  Boxes reaching past the lattice read zeros, which only wall
//    positions see.
//  * Interval k (one CTA barrier): every tile warp first does the odd step
//    of plane k for its row -- gather the post-collision values from
//    shared-memory rings, collide, push into f -- and then the even step of
//    plane k+2 -- collide the staged values and hand them to the rings.  The
//    halo warps do the even step of plane k+2 on the halo ring (recomputed,
//    not exchanged).  The rest and pure-z values of a tile cell never leave
//    its thread's registers.
//  * Why no tile reads what a neighbour already overwrote.  The odd step of
//    plane k writes planes k-1, k, k+1 of the tile and of the cells around
//    it; every other reader of those locations reads them through its TMA
//    copy of that plane.  So before interval k+1 (whose odd step writes up to
//    plane k+2) a CTA waits until each of its eight neighbours has received
//    its copy of plane k+2: a sync warp publishes "plane p loaded" in a
//    global progress word as soon as the copy lands, and polls the
//    neighbours' words while the other warps compute.  Only the pushes into
//    plane k+1 (the five directions with c_z = +1) need the newest word; the
//    tile warps hold them back until after their even step, so the poll has
//    the whole interval to succeed.  This replaces the shell shadow of
//    the other merged sweep: the HBM traffic is the algorithmic 2 x 19 x
//    sizeof(T) bytes per cell per two steps, with the halo columns and rows
//    served from L2 when the neighbours copy them at about the same time.
//  * Every wait is bounded; a CTA whose wait runs out sets status bit 8,
//    drains its copies and leaves, and its neighbours then give up too.
#pragma once

#include "merged3.cuh"

namespace lbm {

template <int TY, class T>
struct NSL {
    static constexpr int TX = 32, W = TX + 2, H = TY + 2, NPOS = W * H;
    static constexpr int XM = 16 / (int)sizeof(T);  // x margin of the copy box
    static constexpr int BW = TX + 2 * XM, BH = TY + 2, BPLANE = BW * BH;
    static constexpr int NH = 2 * W + 2 * TY;       // halo ring cells
    static constexpr int NHW = (NH + 31) / 32;      // halo warps
    static constexpr int SYNCW = TY + NHW;          // the sync warp
    static constexpr int NWARPS = SYNCW + 1;
    static constexpr int THREADS = 32 * NWARPS;
    // ring slots per z-group: in one interval the odd step of plane k reads
    // planes k-1 .. k+1 while the even step of plane k+2 writes
    static constexpr int RSM = 3, RS0 = 3, RSP = 4;
    static constexpr int NRING = RSM * NDM + RS0 * ND0 + RSP * NDP;
    static_assert(THREADS <= 1024, "one CTA");

    // Logical warp (tile row 0 .. TY-1, then the halo warps, then the sync
    // warp) of hardware warp w.  Warps w, w+4, w+8, ... share one of the SM's
    // four schedulers; with 14 tile, 3 halo and 1 sync warp the identity puts
    // four tile warps and a halo warp on one scheduler and three tile warps on
    // another.  The permutation below gives the schedulers 4 tile + sync,
    // 3 tile + 2 halo, 4 tile, and 3 tile + 1 halo warps, closer to equal
    // work (a halo warp does about half a tile warp's).
    __device__ __forceinline__ static int logical(int w)
    {
        if constexpr (TY == 14 && NWARPS == 18) {
            switch (w) {
            case 13: return 14;
            case 14: return 13;
            case 15: return 16;
            case 16: return 17;
            case 17: return 15;
            default: return w;
            }
        } else {
            return w;
        }
    }
};

template <int TY, class T, class R>
struct NSSmem {
    using L = NSL<TY, T>;
    static constexpr size_t stage_bytes = ((size_t)Q * L::BPLANE * sizeof(T) + 127) / 128 * 128;
    static constexpr size_t ring_off = 2 * stage_bytes;
    static constexpr size_t bar_off = ring_off + (size_t)L::NRING * L::NPOS * sizeof(R);
    static constexpr size_t flag_off = bar_off + 2 * sizeof(uint64_t);
    static constexpr size_t bytes = flag_off + 16;
    static constexpr unsigned tma_bytes = (unsigned)(Q * L::BPLANE * sizeof(T));
    static_assert((L::BW * sizeof(T)) % 16 == 0, "copy box rows in 16-byte units");
};

// Waits of the sync warp on a neighbour's progress word: at most
// NS_POLL_LIMIT polls about 64 ns apart (a fraction of a second).
constexpr int NS_POLL_LIMIT = 1 << 21;
constexpr int NS_STATUS_BIT = 8;

template <class S, bool FORCE, int TY, int COLL = COLL_BGK>
struct NSCta {
    using R = typename S::R;
    using T = typename S::T;
    using L = NSL<TY, T>;
    using SM = NSSmem<TY, T, R>;
    static constexpr int W = L::W, NPOS = L::NPOS, BPLANE = L::BPLANE, XM = L::XM;
    static constexpr unsigned CZM = z_bits(-1), CZP = z_bits(1);
    enum { TILE = 0, HALO = 1, SYNC = 2 };

    const Geom<R> &g;
    const Dirs<T> &fd;
    const Dirs<T> &fo;  // fd.p[i] + noff[i]: the push target of an interior cell
    unsigned char *smem;
    R *ringm, *ring0, *ringp;
    uint64_t *bar;
    int role, x0, y0, tw, th, lx, ly, x, y, pos, sidx, nx, ny, nz, cxy;
    unsigned wxy, lxy;  // wall links through the x / y faces; those ending on a lid
    bool active, xybnd, xwall, ywall;

    __device__ __forceinline__ NSCta(const Geom<R> &g_, const Dirs<T> &fd_, const Dirs<T> &fo_,
                                     const ShellInfo &si, unsigned char *smem_)
        : g(g_), fd(fd_), fo(fo_), smem(smem_)
    {
        ringm = reinterpret_cast<R *>(smem + SM::ring_off);
        ring0 = ringm + L::RSM * NDM * NPOS;
        ringp = ring0 + L::RS0 * ND0 * NPOS;
        bar = reinterpret_cast<uint64_t *>(smem + SM::bar_off);
        nx = g.nx; ny = g.ny; nz = g.nz;
        x0 = 32 * blockIdx.x;
        tw = min(32, nx - x0);
        band_of(si, blockIdx.y, y0, th);
        const int warp = L::logical(threadIdx.x >> 5), lane = threadIdx.x & 31;
        role = warp < TY ? TILE : (warp < L::SYNCW ? HALO : SYNC);
        if (role == TILE) {
            lx = lane;
            ly = warp;
            active = lx < tw && ly < th;
        } else if (role == HALO) {
            // halo ring: row -1, row th, column -1, column tw; cells outside
            // the lattice (walls) have nothing to compute
            const int h = (warp - TY) * 32 + lane;
            if (h < W) { lx = h - 1; ly = -1; active = lx <= tw; }
            else if (h < 2 * W) { lx = h - W - 1; ly = th; active = lx <= tw; }
            else if (h < 2 * W + TY) { lx = -1; ly = h - 2 * W; active = ly < th; }
            else if (h < L::NH) { lx = tw; ly = h - 2 * W - TY; active = ly < th; }
            else { lx = 0; ly = 0; active = false; }
            if (active && (x0 + lx < 0 || x0 + lx >= nx || y0 + ly < 0 || y0 + ly >= ny)) active = false;
        } else {
            lx = 0; ly = 0; active = false;
        }
        if (!active) { lx = 0; ly = 0; }
        x = x0 + lx; y = y0 + ly;
        pos = (ly + 1) * W + (lx + 1);
        sidx = (ly + 1) * L::BW + lx + XM;
        xybnd = x == 0 || x == nx - 1 || y == 0 || y == ny - 1;
        xwall = active && (x == 0 || x == nx - 1);
        ywall = active && (y == 0 || y == ny - 1);
        cxy = y * (int)g.nxp + x;
        wxy = lxy = 0u;
        if (active) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                bool wall = false, lid = false;
                const int tx = x + cx(i), ty = y + cy(i);
                if (tx < 0 || tx >= nx) { wall = true; lid |= g.lid[tx < 0 ? 0 : 1] != 0; }
                if (ty < 0 || ty >= ny) { wall = true; lid |= g.lid[ty < 0 ? 2 : 3] != 0; }
                if (wall) wxy |= 1u << i;
                if (wall && lid) lxy |= 1u << i;
            });
        }
    }

    __device__ __forceinline__ static int slot(int plane, int n) { return plane % n; }
    template <int GG>
    __device__ __forceinline__ R *ring_at(int plane, int gi) const
    {
        if constexpr (GG == GRP_M) return ringm + (slot(plane, L::RSM) * NDM + gi) * NPOS;
        else if constexpr (GG == GRP_0) return ring0 + (slot(plane, L::RS0) * ND0 + gi) * NPOS;
        else return ringp + (slot(plane, L::RSP) * NDP + gi) * NPOS;
    }
    // Ring bases at this thread's position for the planes one interval
    // touches, computed once per interval (the slot arithmetic stays out of
    // the unrolled direction loops, whose accesses become base + constant).
    struct Bases {
        R *m0, *m1;  // c_z = -1 group: planes k, k+1
        R *z0;       // c_z = 0 group: plane k
        R *pm, *p0;  // c_z = +1 group: planes k-1, k
    };
    __device__ __forceinline__ Bases bases(int k) const
    {
        const int s3 = k % L::RSM;
        Bases b;
        b.m0 = ringm + s3 * (NDM * NPOS) + pos;
        b.m1 = ringm + (s3 + 1 == L::RSM ? 0 : s3 + 1) * (NDM * NPOS) + pos;
        b.z0 = ring0 + (k % L::RS0) * (ND0 * NPOS) + pos;
        b.pm = ringp + ((k + L::RSP - 1) % L::RSP) * (NDP * NPOS) + pos;
        b.p0 = ringp + (k % L::RSP) * (NDP * NPOS) + pos;
        return b;
    }
    // value gathered for direction I from x - c_I (plane k - c_z), and the
    // cell's own outgoing value along c_opp(I) (plane k)
    template <int I>
    __device__ __forceinline__ static const R *from_neighbour(const Bases &b)
    {
        constexpr int gg = grp(I), off = gidx(I) * NPOS - cx(I) - cy(I) * W;
        if constexpr (gg == GRP_M) return b.m1 + off;
        else if constexpr (gg == GRP_0) return b.z0 + off;
        else return b.pm + off;
    }
    template <int I>
    __device__ __forceinline__ static const R *own_outgoing(const Bases &b)
    {
        constexpr int j = opp(I), gg = grp(j), off = gidx(j) * NPOS;
        if constexpr (gg == GRP_M) return b.m0 + off;
        else if constexpr (gg == GRP_0) return b.z0 + off;
        else return b.p0 + off;
    }
    __device__ __forceinline__ T *stage(int p) const { return reinterpret_cast<T *>(smem + (p & 1) * SM::stage_bytes); }

    // Even step of plane p (tile and halo threads): collide the staged
    // values, hand the xy-moving ones to the rings, return the rest and
    // pure-z values (which only the cell's own thread reads).
    __device__ __forceinline__ void produce(int p, R &rest, R &zp, R &zm) const
    {
        R s[Q];
        const T *in = stage(p) + sidx;
        // FP32 storage of f itself: decode the opposite pairs {i, i+9}
        // (one weight) two lanes at a time -- the same roundings as the
        // scalar decode, half the instructions
        constexpr bool PAIRS = std::is_same<S, StoreF32>::value;
        if constexpr (PAIRS) {
            s[0] = decode<S, 0>(in[0]);
            static_for<9>([&](auto K) {
                constexpr int i = decltype(K)::value + 1;
                const float2 v = p_add(make_float2(in[i * BPLANE], in[(i + 9) * BPLANE]), p_dup(-float(wgt(i))));
                s[i] = v.x;
                s[i + 9] = v.y;
            });
        } else {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = decode<S, i>(in[i * BPLANE]);
            });
        }
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, p), ncanon(g), Fx, Fy, Fz);
        collide_sel<R, FORCE, COLL>(g, s, Fx, Fy, Fz);
        // value that leaves along c_i as the next step reads it: + L_opp(i)
        // on a wall link that ends on a lid (the lid takes precedence)
        const unsigned lm = lxy | (p == 0 && g.lid[4] ? CZM : 0u) | (p == nz - 1 && g.lid[5] ? CZP : 0u);
        if (lm) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                if (lm & (1u << i)) s[i] = radd(s[i], g.L[opp(i)]);
            });
        }
        // the values as the storage holds them (the AA pair stores them
        // between its two steps): the pairs of FP32 storage two lanes at a time
        if constexpr (PAIRS) {
            s[0] = roundtrip<S, 0>(s[0]);
            static_for<9>([&](auto K) {
                constexpr int i = decltype(K)::value + 1;
                const float2 w = p_dup(float(wgt(i)));
                const float2 v = p_add(p_add(make_float2(s[i], s[i + 9]), w), p_neg(w));
                s[i] = v.x;
                s[i + 9] = v.y;
            });
        } else if constexpr (std::is_same<S, StoreF16S>::value || std::is_same<S, StoreBF16S>::value) {
            // 16-bit storage: both lanes of a pair converted down (round to
            // nearest even, as the scalar conversion) and back in one go
            s[0] = roundtrip<S, 0>(s[0]);
            static_for<9>([&](auto K) {
                constexpr int i = decltype(K)::value + 1;
                float2 v;
                if constexpr (std::is_same<S, StoreF16S>::value)
                    v = __half22float2(__float22half2_rn(make_float2(s[i], s[i + 9])));
                else
                    v = __bfloat1622float2(__float22bfloat162_rn(make_float2(s[i], s[i + 9])));
                s[i] = v.x;
                s[i + 9] = v.y;
            });
        } else {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = roundtrip<S, i>(s[i]);
            });
        }
        R *const wm_ = ringm + (p % L::RSM) * (NDM * NPOS) + pos;
        R *const w0_ = ring0 + (p % L::RS0) * (ND0 * NPOS) + pos;
        R *const wp_ = ringp + (p % L::RSP) * (NDP * NPOS) + pos;
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            const R v = s[i];
            if constexpr (gg == GRP_M) wm_[gidx(i) * NPOS] = v;
            else if constexpr (gg == GRP_0) w0_[gidx(i) * NPOS] = v;
            else if constexpr (gg == GRP_P) wp_[gidx(i) * NPOS] = v;
            else if constexpr (i == 0) rest = v;
            else if constexpr (i == DIR_ZP) zp = v;
            else zm = v;
        });
    }

    // Path of a tile warp's odd step, the same for all its lanes (no lane
    // may diverge from the others): no wall link in the warp; wall links
    // through x or y faces only (a lane at an x edge, a y-edge row), handled
    // by selecting addresses; or a z-edge plane (general path).  One select
    // path serves every x/y case: separate variants per face made the kernel
    // larger and every tile slower.
    enum { PATH_FREE = 0, PATH_XYWALL = 3, PATH_XYLID = 5, PATH_WALL = 4 };
    // directions whose links can cross the faces of select set SEL (bit 0:
    // x faces, bit 1: y faces)
    template <int SEL, int I>
    __host__ __device__ static constexpr bool selected() { return ((SEL & 1) && cx(I) != 0) || ((SEL & 2) && cy(I) != 0); }

    template <int SEL>
    __device__ __forceinline__ void gather_sel(const Bases &b, unsigned wm, R (&s)[Q]) const
    {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int gg = grp(i);
            if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                if constexpr (selected<SEL, i>())
                    s[i] = *((wm >> opp(i)) & 1u ? own_outgoing<i>(b) : from_neighbour<i>(b));
                else
                    s[i] = *from_neighbour<i>(b);
            }
        });
    }

    // LID: some lane of the warp has a wall link ending on a lid through an
    // x or y face (else the lid term is left out altogether)
    template <int SEL, bool ZP, bool LID>
    __device__ __forceinline__ void push_sel(int c, const R (&s)[Q]) const
    {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if constexpr ((cz(i) == 1) == ZP) {
                if constexpr (selected<SEL, i>()) {
                    const bool w = (wxy >> i) & 1u;
                    R v = s[i];
                    if constexpr (LID) v = (lxy >> i) & 1u ? radd(s[i], g.L[opp(i)]) : s[i];
                    st_no_l1(w ? &fd.p[opp(i)][c] : &fo.p[i][c], encode<S, i>(v));
                } else {
                    st_no_l1(&fo.p[i][c], encode<S, i>(s[i]));
                }
            }
        });
    }

    // Odd step of plane k (tile threads): gather from the rings and the
    // registers, collide.  rk = rest of plane k; zpm / zp0 = +z values of
    // planes k-1 / k; zm0 / zm1 = -z values of planes k / k+1.
    __device__ __forceinline__ void consume(int k, int path, R (&s)[Q], R rk, R zpm, R zp0, R zm0, R zm1) const
    {
        const bool zlo = k == 0, zhi = k == nz - 1;
        const unsigned wm = wxy | (zlo ? CZM : 0u) | (zhi ? CZP : 0u);
        s[0] = rk;
        s[DIR_ZP] = zlo ? zm0 : zpm;
        s[DIR_ZM] = zhi ? zp0 : zm1;
        const Bases b = bases(k);
        if (path == PATH_FREE) {
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                constexpr int gg = grp(i);
                if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) s[i] = *from_neighbour<i>(b);
            });
        } else if (path == PATH_XYWALL || path == PATH_XYLID) {
            // a link from x - c_i that crosses a wall brings back the cell's
            // own outgoing value along c_opp(i): picked by address
            gather_sel<3>(b, wm, s);
        } else {
            // a link from x - c_i that crosses a wall brings back the cell's
            // own outgoing value along c_opp(i) (lid term already added)
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                constexpr int gg = grp(i);
                if constexpr (gg == GRP_M || gg == GRP_0 || gg == GRP_P) {
                    if (wm & (1u << opp(i))) s[i] = *own_outgoing<i>(b);
                    else s[i] = *from_neighbour<i>(b);
                }
            });
        }
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, k), ncanon(g), Fx, Fy, Fz);
        collide_sel<R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    }

    // Push the odd-step result of plane k: slot i of x + c_i, or (wall link)
    // slot opp(i) of x itself with the lid term.  ZP = false pushes the
    // fourteen directions with c_z <= 0 (targets in planes k-1 and k),
    // ZP = true the five with c_z = +1 (targets in plane k+1, or plane k
    // across the top wall), which wait for the neighbours' copies of k+1.
    template <bool ZP>
    __device__ __forceinline__ void scatter(int k, int path, const R (&s)[Q]) const
    {
        const int c = cxy + k * (int)g.plane;
        if (path == PATH_FREE) {
            if constexpr (std::is_same<S, StoreF32>::value && !ZP) {
                // FP32 storage: the opposite pairs in the plane (c_z = 0, one
                // weight) encoded two lanes at a time, the rest one by one
                static_for<9>([&](auto K) {
                    constexpr int i = decltype(K)::value + 1;
                    if constexpr (cz(i) == 0) {
                        const float2 e = p_add(make_float2(s[i], s[i + 9]), p_dup(float(wgt(i))));
                        st_no_l1(&fo.p[i][c], e.x);
                        st_no_l1(&fo.p[i + 9][c], e.y);
                    }
                });
                static_for<Q>([&](auto K) {
                    constexpr int i = decltype(K)::value;
                    if constexpr (i == 0 || cz(i) == -1) st_no_l1(&fo.p[i][c], encode<S, i>(s[i]));
                });
            } else {
                static_for<Q>([&](auto K) {
                    constexpr int i = decltype(K)::value;
                    if constexpr ((cz(i) == 1) == ZP) st_no_l1(&fo.p[i][c], encode<S, i>(s[i]));
                });
            }
        } else if (path == PATH_XYWALL) {
            // a wall link through an x or y face stores into the cell's own
            // slot opp(i) (same weight, so the same encoding), with the lid
            // term on a lid face
            push_sel<3, ZP, false>(c, s);
        } else if (path == PATH_XYLID) {
            push_sel<3, ZP, true>(c, s);
        } else {
            const Faces fc = faces_of(g, x, y, k);
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                if constexpr ((cz(i) == 1) == ZP) {
                    constexpr unsigned m = face_mask(cx(i), cy(i), cz(i));
                    if (fc.wall & m) {
                        R v = s[i];
                        if (fc.lid & m) v = radd(v, g.L[opp(i)]);
                        st_no_l1(&fd.p[opp(i)][c], encode<S, opp(i)>(v));
                    } else {
                        st_no_l1(&fo.p[i][c], encode<S, i>(s[i]));
                    }
                }
            });
        }
    }
};

// Progress words: one per tile, NS_PROG_INTS apart (each on its own 128-byte
// line, so that the polls of many SMs do not meet on one line).
__device__ __forceinline__ void ns_store_relaxed(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ns_load_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <class S, bool FORCE, int TY, int COLL = COLL_BGK>
__global__ void __launch_bounds__(NSL<TY, typename S::T>::THREADS, 1)
    k_nsweep(const __grid_constant__ CUtensorMap tmap, Geom<typename S::R> g, Dirs<typename S::T> fd,
             Dirs<typename S::T> fo, ShellInfo si, int *__restrict__ prog, int *__restrict__ status)
{
    using C = NSCta<S, FORCE, TY, COLL>;
    using L = typename C::L;
    using SM = typename C::SM;
    using R = typename S::R;
    extern __shared__ __align__(128) unsigned char smem[];
    C c(g, fd, fo, si, smem);
    // abort flags, one per parity of the barrier count: a flag raised before
    // barrier b is read after it, and no thread can raise the other one
    // before every thread has passed barrier b
    int *abort_flag = reinterpret_cast<int *>(smem + SM::flag_off);
    int ph = 0;
    const int nz = g.nz;
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const bool syncw = c.role == C::SYNC;
    const bool cell = c.active;
    if (threadIdx.x == 0) {
        mbar_init(&c.bar[0], 1);
        mbar_init(&c.bar[1], 1);
        mbar_fence_init();
        abort_flag[0] = abort_flag[1] = 0;
    }
    __syncthreads();
    // sync warp: lanes 0..7 watch one neighbouring tile each (-1: none)
    int nb = -1;
    if (syncw && lane < 8) {
        const int d = lane < 4 ? lane : lane + 1;
        const int bx = (int)blockIdx.x + d % 3 - 1, by = (int)blockIdx.y + d / 3 - 1;
        if (bx >= 0 && bx < (int)gridDim.x && by >= 0 && by < (int)gridDim.y) nb = by * (int)gridDim.x + bx;
    }
    int issued = 0;  // planes whose copy has been started (lane 0 of the sync warp)
    auto issue = [&](int p) {
        uint64_t *b = &c.bar[p & 1];
        mbar_arrive_expect_tx(b, SM::tma_bytes);
        tma_load_4d(c.stage(p), &tmap, c.x0 - L::XM, c.y0 - 1, p, 0, b);
        ++issued;
    };
    // plane p is the (p >> 1)-th use of stage slot p & 1
    auto wait_stage = [&](int p) { return mbar_wait_bounded(&c.bar[p & 1], (unsigned)((p >> 1) & 1)); };
    // sync warp, lane 0: the planes 0 .. pub-1 are published as loaded
    int pub = 0;
    auto landed = [&](int p) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(&c.bar[p & 1])), "r"((unsigned)((p >> 1) & 1))
            : "memory");
        return ok != 0;
    };
    // sync warp: publish our copies as they land (at least planes 0 ..
    // must_pub) and wait until every neighbour has loaded plane `need`
    // (need < 0: no condition).  The progress words are read and written
    // relaxed, without fences: a word is written only after the copy it
    // vouches for has completed (its mbarrier phase, data in shared memory),
    // and the CTA's pushes that depend on a neighbour's word are issued only
    // after the load that saw it has returned (the push barrier follows the
    // poll), so no push can reach a location before the copy that reads it.
    // (A fence here would wait for the CTA's whole store stream to drain,
    // several microseconds per interval.)
    auto sync_interval = [&](int need, int must_pub) {
        bool mine = nb < 0 || need < 0;
        bool done = false;
        for (int it = 0; it < NS_POLL_LIMIT; ++it) {
            if (lane == 0) {
                const int before = pub;
                while (pub < issued && landed(pub)) ++pub;
                if (pub != before && tile != si.mute) ns_store_relaxed(prog + NS_PROG_INTS * tile, pub);
            }
            const int pw = __shfl_sync(0xffffffffu, pub, 0);
            if (!mine) mine = ns_load_relaxed(prog + NS_PROG_INTS * nb) >= need + 1;
            done = __all_sync(0xffffffffu, mine) && pw > must_pub;
            if (done) break;
            __nanosleep(64);
        }
        if (!done && lane == 0) abort_flag[ph & 1] = 1;
    };
    // which of the warp's cells have wall links through x or y faces (tile
    // warps; every lane votes)
    const bool warp_x = __any_sync(0xffffffffu, c.xwall), warp_y = __any_sync(0xffffffffu, c.ywall);
    const bool warp_lid = __any_sync(0xffffffffu, c.lxy != 0u);
    const int xy_path = warp_lid ? C::PATH_XYLID : C::PATH_XYWALL;
    // rest of planes k, k+1; +z of planes k-1, k, k+1; -z of planes k, k+1
    R rk = R(0), rk1 = R(0), zpm = R(0), zp0 = R(0), zp1 = R(0), zm0 = R(0), zm1 = R(0);
    // the odd step's pushes into the next plane, held until the next interval
    R held[Q];
    int held_k = -1, held_path = C::PATH_WALL;
    // prologue: even steps of planes 0 and 1; the copy of plane 2 goes into
    // the slot plane 0 leaves; every neighbour must have loaded plane 0
    // before the first pushes
    if (syncw && lane == 0) {
        issue(0);
        if (nz > 1) issue(1);
    }
    if (cell) {
        if (wait_stage(0)) c.produce(0, rk, zp0, zm0);
        else abort_flag[ph & 1] = 1;
    }
    if (syncw) sync_interval(-1, 0);
    cta_barrier();
    if (abort_flag[ph++ & 1]) goto bail;
    if (syncw && lane == 0 && nz > 2) issue(2);
    if (nz > 1 && cell) {
        if (wait_stage(1)) c.produce(1, rk1, zp1, zm1);
        else abort_flag[ph & 1] = 1;
    }
    if (syncw) sync_interval(0, nz > 1 ? 1 : 0);
    cta_barrier();
    if (abort_flag[ph++ & 1]) goto bail;
    // interval k: odd step of plane k and even step of plane k+2 (in either
    // order: tile warps that share a scheduler take them in opposite orders,
    // so that their pushes and collisions interleave); the copy of plane k+3 goes
    // into the slot plane k+1 left in the previous interval.  The pushes
    // into planes k-1 and k need the neighbours' copies of plane k; the
    // pushes of the odd step of plane k into plane k+1 are held in registers
    // and issued at the start of interval k+1, after the sync warp has seen
    // the neighbours' copies of plane k+1 (it polls during interval k, before
    // the barrier that ends it).
    for (int k = 0; k < nz; ++k) {
        R s[Q];
        R rn = R(0), zpn = R(0), zmn = R(0);
        // warps w, w+4, w+8, ... share a scheduler (warp index mod 4): they
        // alternate, so that each scheduler has collisions of one step and
        // memory operations of the other in flight at once
        const bool odd_first = ((threadIdx.x >> 7) & 1) == 0;
        const int path = (k == 0 || k == nz - 1) ? C::PATH_WALL : (warp_x || warp_y ? xy_path : C::PATH_FREE);
        if (c.role == C::SYNC) {
            if (lane == 0 && k + 3 < nz) issue(k + 3);
            sync_interval(k + 1 < nz ? k + 1 : nz - 1, k + 2 < nz ? k + 2 : nz - 1);
        } else {
            const bool tile_cell = c.role == C::TILE && cell;
            if (tile_cell && held_k >= 0) c.template scatter<true>(held_k, held_path, held);
            if (tile_cell && odd_first) {
                c.consume(k, path, s, rk, zpm, zp0, zm0, zm1);
                c.template scatter<false>(k, path, s);
            }
            if (k + 2 < nz && cell) {
                if (wait_stage(k + 2)) c.produce(k + 2, rn, zpn, zmn);
                else abort_flag[ph & 1] = 1;
            }
            if (tile_cell && !odd_first) {
                c.consume(k, path, s, rk, zpm, zp0, zm0, zm1);
                c.template scatter<false>(k, path, s);
            }
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                if constexpr (cz(i) == 1) held[i] = s[i];
            });
            held_k = k;
            held_path = path;
        }
        rk = rk1; rk1 = rn;
        zpm = zp0; zp0 = zp1; zp1 = zpn;
        zm0 = zm1; zm1 = zmn;
        cta_barrier();
        if (abort_flag[ph++ & 1]) goto bail;
    }
    // the last plane's held pushes (the sync warp saw plane nz-1 loaded by
    // every neighbour before the last barrier)
    if (c.role == C::TILE && cell && held_k >= 0) c.template scatter<true>(held_k, held_path, held);
    return;

bail:
    // a wait ran out: record it, wait (bounded) for the copies still in
    // flight -- the last two issued, each the newest use of its slot -- and
    // leave without touching the lattice again
    if (syncw && lane == 0)
        for (int u = issued - 2 > 0 ? issued - 2 : 0; u < issued; ++u)
            mbar_wait_bounded(&c.bar[u & 1], (unsigned)((u >> 1) & 1));
    if (threadIdx.x == 0) atomicOr(status, NS_STATUS_BIT);
}

}  // namespace lbm
