// merged.cuh -- two collision-streaming steps per sweep (K4) and the shell
// snapshot that makes the in-place sweep safe between tiles.
//
// The paper merges the steps t and t+1 of a cell as soon as every neighbour
// it pulls from has finished step t (Sec. 4.1, Alg. 2, "second computation"
// of cell (iX-1, iY-1, iZ-1)), and protects the layers where two threads'
// sub-domains meet by processing them first (Stage I of Alg. 3, Sec. 4.2).
// On the GPU:
//
//  * a CTA owns a TX x TY column of cells and marches it along z; at
//    iteration k it loads plane k+1, performs the even (local) collision of
//    the AA pair on it, and then the odd step of plane k, whose inputs --
//    the post-collision values of the 3x3x3 neighbourhood -- now all exist;
//  * the post-collision values travel between the threads of the CTA through
//    a shared-memory ring of four planes, indexed by the cell and the step
//    that consumes them (the producer scatters, the consumer reads its own
//    slot), so one __syncthreads per plane orders everything;
//  * cells on the boundary of a tile are read by two CTAs and written by
//    both: before the sweep, k_snapshot stores the post-collision values of
//    every shell cell (the tile rows/columns next to another tile, and the
//    planes z = 0, nz-1 when z is periodic) in the buffer G.  During the
//    sweep a CTA reads its own shell and its neighbours' from G and never
//    from f, so it cannot see what another CTA has already written there --
//    the GPU counterpart of the intersection layers of Alg. 3 (Stage I).
//
// Per two steps the sweep reads and writes every population once (the
// 2 x 19 x sizeof(T) bytes per cell of a single AA step), plus the shell
// traffic of the snapshot.
#pragma once

#include "kernels.cuh"

namespace lbm {

// Shell rows / columns: the first and last row of every tile that touches
// another tile (across a periodic face too).  Snapshot buffers:
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
                                                  typename S::T *__restrict__ G, TileInfo ti, int64_t cnt_z,
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
        G[base + i * sl] = encode<S, i>(s[i]);
    });
}

template <class S, bool FORCE, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, 1) k_merged(Geom<typename S::R> g, typename S::T *__restrict__ f,
                                                       const typename S::T *__restrict__ G, TileInfo ti)
{
    using R = typename S::R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *B = reinterpret_cast<R *>(smem_raw);  // [4][Q][TY*TX], slot = consuming plane & 3
    constexpr int NT = TX * TY;

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int bxi = blockIdx.x, byi = blockIdx.y;
    const int x0 = bxi * TX, y0 = byi * TY;
    const int x1 = min(g.nx, x0 + TX) - 1, y1 = min(g.ny, y0 + TY) - 1;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x <= x1 && y <= y1;
    const int pos = ty * TX + tx;
    const int nx = g.nx, ny = g.ny, nz = g.nz;

    const bool ysh_lo = y == y0 && row_is_shell(g, ti, byi, 0);
    const bool ysh_hi = y == y1 && row_is_shell(g, ti, byi, 1);
    const bool xsh_lo = x == x0 && col_is_shell(g, ti, bxi, 0);
    const bool xsh_hi = x == x1 && col_is_shell(g, ti, bxi, 1);
    const bool own_shell = ysh_lo || ysh_hi || xsh_lo || xsh_hi;

    // Even step of virtual plane q (q = -1 / nz are the periodic images of
    // nz-1 / 0), then hand every value to the odd step that consumes it.
    auto produce = [&](int q) {
        if (!active) return;
        const int zr = q < 0 ? q + nz : (q >= nz ? q - nz : q);
        R s[Q];
        const bool zsnap = ti.zshell && (zr == 0 || zr == nz - 1);
        if (zsnap || own_shell) {
            int64_t base, sl;
            if (zsnap) {
                base = ti.gz_off + ((int64_t)(zr == 0 ? 0 : 1) * ny + y) * nx + x;
                sl = ti.gz_slot;
            } else if (ysh_lo || ysh_hi) {
                base = ti.gy_off + ((int64_t)zr * 2 * ti.nty + 2 * byi + (ysh_lo ? 0 : 1)) * nx + x;
                sl = ti.gy_slot;
            } else {
                base = ti.gx_off + ((int64_t)zr * 2 * ti.ntx + 2 * bxi + (xsh_lo ? 0 : 1)) * ny + y;
                sl = ti.gx_slot;
            }
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = decode<S, i>(G[base + i * sl]);
            });
        } else {
            load_natural<S>(g, f, x, y, zr, s);
            R Fx, Fy, Fz;
            force_at<R, FORCE>(g, canon(g, x, y, zr), ncanon(g), Fx, Fy, Fz);
            bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
            outgoing_values<S>(g, x, y, zr, s);
            static_for<Q>([&](auto K) {
                constexpr int i = decltype(K)::value;
                s[i] = roundtrip<S, i>(s[i]);
            });
        }
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            int tx2 = x + cx(i), ty2 = y + cy(i);
            const int tq = q + cz(i);
            bool wall = false;
            if (cx(i) != 0 && (tx2 < 0 || tx2 >= nx)) {
                if (g.per[0]) tx2 = tx2 < 0 ? tx2 + nx : tx2 - nx;
                else wall = true;
            }
            if (cy(i) != 0 && (ty2 < 0 || ty2 >= ny)) {
                if (g.per[1]) ty2 = ty2 < 0 ? ty2 + ny : ty2 - ny;
                else wall = true;
            }
            if (cz(i) != 0 && (tq < 0 || tq >= nz) && !g.per[2]) wall = true;
            if (wall) {
                if (q >= 0 && q < nz) B[((q & 3) * Q + opp(i)) * NT + pos] = s[i];
            } else if (tq >= 0 && tq < nz && tx2 >= x0 && tx2 <= x1 && ty2 >= y0 && ty2 <= y1) {
                B[((tq & 3) * Q + i) * NT + (ty2 - y0) * TX + (tx2 - x0)] = s[i];
            }
        });
    };

    // Odd step of plane k: gather (ring or, across a tile edge, the snapshot),
    // collide, scatter into f.
    auto consume = [&](int k) {
        if (!active) return;
        R s[Q];
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            bool from_g = false;
            if constexpr (cx(i) != 0 || cy(i) != 0) {
                const bool edge = (cx(i) == 1 && x == x0) || (cx(i) == -1 && x == x1) ||
                                  (cy(i) == 1 && y == y0) || (cy(i) == -1 && y == y1);
                if (edge) {
                    int sx = x - cx(i), sy = y - cy(i), sz = k - cz(i);
                    bool wall = false;
                    if (sx < 0 || sx >= nx) {
                        if (g.per[0]) sx = sx < 0 ? sx + nx : sx - nx;
                        else wall = true;
                    }
                    if (sy < 0 || sy >= ny) {
                        if (g.per[1]) sy = sy < 0 ? sy + ny : sy - ny;
                        else wall = true;
                    }
                    if (sz < 0 || sz >= nz) {
                        if (g.per[2]) sz = sz < 0 ? sz + nz : sz - nz;
                        else wall = true;
                    }
                    if (!wall && !(sx >= x0 && sx <= x1 && sy >= y0 && sy <= y1)) {
                        from_g = true;
                        if (sy < y0 || sy > y1) {
                            const int64_t b = ti.gy_off +
                                              ((int64_t)sz * 2 * ti.nty + 2 * (sy / ti.TY) + (cy(i) == 1 ? 1 : 0)) * nx + sx;
                            s[i] = decode<S, i>(G[b + i * ti.gy_slot]);
                        } else {
                            const int64_t b = ti.gx_off +
                                              ((int64_t)sz * 2 * ti.ntx + 2 * (sx / ti.TX) + (cx(i) == 1 ? 1 : 0)) * ny + sy;
                            s[i] = decode<S, i>(G[b + i * ti.gx_slot]);
                        }
                    }
                }
            }
            if (!from_g) s[i] = B[((k & 3) * Q + i) * NT + pos];
        });
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, canon(g, x, y, k), ncanon(g), Fx, Fy, Fz);
        bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
        push_store<S>(g, f, x, y, k, s);
    };

    if (g.per[2]) produce(-1);
    produce(0);
    for (int k = 0; k < nz; ++k) {
        if (k + 1 < nz || g.per[2]) produce(k + 1);
        __syncthreads();
        consume(k);
    }
}

}  // namespace lbm
