// wavefront.cuh -- two collision-streaming steps per HBM round trip by
// marching a plane wavefront through the L2 cache (WAVEFRONT schedule).
//
// The paper gains its speed by reusing a cell's data in cache for the second
// of two merged time steps before it is evicted (Sec. 4.1: the second
// computation of a cell follows its first while both layers are cached;
// Sec. 5.2 shows the drop once two layers no longer fit in L3).  On GB300 the
// cache that can hold whole layers is the 126 MB L2.
//
// One persistent kernel processes the AA pair as work items, each the even
// step (E) or the odd step (O) of one block of rows (all x) of one z-plane.
// Items are handed out by an atomic ticket in the order
//
//     E(0) .. E(L),  E(L+1) O(0),  E(L+2) O(1),  ...,  O(nz-1)
//
// (each entry expanded over its row blocks; with a periodic z axis E(nz-1)
// goes first).  The odd step of rows r of plane p reads and writes rows
// r-1..r+1 of planes p-1..p+1, so it waits until the even steps of those
// nine (plane, row block) pairs are done -- per-pair completion flags set
// with release semantics and read with acquire semantics.  Every item it
// waits for carries a smaller ticket and is therefore held by a CTA that is
// already running, so the wait always ends (bounded anyway: on timeout the
// CTA sets a status bit and stops).  Only about L planes are in flight, so
// the post-collision values written by E(p) are still in L2 when O(p) reads
// them and are overwritten there before eviction: DRAM sees one read and one
// write of every population per two time steps, with no halo or shell
// copies.  Every cell runs exactly the AA even / odd code, so the schedule
// is bit-identical to AA.
#pragma once

#include "kernels.cuh"

namespace lbm {

constexpr int WF_THREADS = 512;

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// L2-only loads: other CTAs of this launch wrote the data.
template <class T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

// Interior stores of the sweep: the 2-byte formats skip L1 allocation (faster
// for them on a 256^3 cavity, slower for FP32).
template <class T>
__device__ __forceinline__ void wf_store(T *p, T v)
{
    if constexpr (sizeof(T) == 2) st_no_l1(p, v);
    else *p = v;
}

template <class S, bool FORCE>
__device__ __forceinline__ void wf_even_cell(const Geom<typename S::R> &g, const Dirs<typename S::T> &f, int x,
                                             int y, int z)
{
    using R = typename S::R;
    const int c = cell32(g, x, y, z);
    R s[Q];
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = decode<S, i>(ldcg(f.p[i] + c));
    });
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            wf_store(&f.p[opp(i)][c], encode<S, opp(i)>(s[i]));
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr unsigned m = face_mask(cx(i), cy(i), cz(i));
            R v = s[i];
            if ((fc.wall & m) && (fc.lid & m)) v = radd(v, g.L[opp(i)]);
            f.p[opp(i)][c] = encode<S, opp(i)>(v);
        });
    }
}

template <class S, bool FORCE>
__device__ __forceinline__ void wf_odd_cell(const Geom<typename S::R> &g, const Dirs<typename S::T> &f,
                                            const Dirs<typename S::T> &fin, const Dirs<typename S::T> &fout, int x,
                                            int y, int z)
{
    using R = typename S::R;
    const int c = cell32(g, x, y, z);
    R s[Q];
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            s[k] = decode<S, k>(ldcg(fin.p[k] + c));
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if (fc.wall & face_mask(-cx(k), -cy(k), -cz(k))) s[k] = decode<S, k>(ldcg(f.p[k] + c));
            else s[k] = decode<S, k>(ldcg(f.p[opp(k)] + (c + step_offset<-cx(k), -cy(k), -cz(k)>(g, fc))));
        });
    }
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            wf_store(&fout.p[i][c], encode<S, i>(s[i]));
        });
    } else {
        push_store_d<S>(g, f, x, y, z, c, s);
    }
}

// Schedule of one launch (host-built, device pointers):
//   entries[e] = 2 * plane + (0 even, 1 odd), e < nentries
//   an item is (entry, row block): rb rows per block, nrb blocks per plane
//   ticket: work counter; done[plane * nrb + block]: that even step is done
//   (both zeroed before the launch); status bit 4 = a wait gave up.
struct WaveSchedule {
    const int *entries;
    int nentries, rb, nrb;
    int *ticket, *done, *status;
};

template <class S, bool FORCE>
__global__ void __launch_bounds__(WF_THREADS) k_wavefront(Geom<typename S::R> g, Dirs<typename S::T> f,
                                                          Dirs<typename S::T> fin, Dirs<typename S::T> fout,
                                                          WaveSchedule ws)
{
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    const int total = ws.nentries * ws.nrb;
    const bool pery = g.per[1] != 0, perz = g.per[2] != 0;
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(ws.ticket, 1);
            s_ok = 1;
        }
        __syncthreads();
        const int t = s_item;
        if (t >= total) break;
        const int code = ws.entries[t / ws.nrb], rblk = t % ws.nrb;
        const int plane = code >> 1;
        const bool odd = (code & 1) != 0;
        if (odd) {
            if (tid < 9) {  // one waiting thread per neighbouring (plane, row block)
                int ok = 1;
                int q = plane + tid / 3 - 1, r = rblk + tid % 3 - 1;
                bool skip = false;
                if (q < 0 || q >= g.nz) {
                    if (perz) q = q < 0 ? q + g.nz : q - g.nz;
                    else skip = true;
                }
                if (r < 0 || r >= ws.nrb) {
                    if (pery) r = r < 0 ? r + ws.nrb : r - ws.nrb;
                    else skip = true;
                }
                if (!skip) {
                    int it = 0;
                    while (ld_acquire(ws.done + q * ws.nrb + r) == 0) {
                        if (++it > (1 << 24)) { ok = 0; break; }
                        __nanosleep(32);
                    }
                    __threadfence();
                }
                if (!ok) s_ok = 0;
            }
            __syncthreads();
            if (!s_ok) {
                if (tid == 0) atomicOr(ws.status, 4);
                break;
            }
        }
        const int y0 = rblk * ws.rb, y1 = min(g.ny, y0 + ws.rb);
        const int ncell = (y1 - y0) * g.nx;
        for (int i = tid; i < ncell; i += WF_THREADS) {
            const int x = i % g.nx, y = y0 + i / g.nx;
            if (odd) wf_odd_cell<S, FORCE>(g, f, fin, fout, x, y, plane);
            else wf_even_cell<S, FORCE>(g, f, x, y, plane);
        }
        __syncthreads();  // the item's writes are done; s_item may be reused
        if (!odd && tid == 0) {
            __threadfence();
            st_release(ws.done + plane * ws.nrb + rblk, 1);
        }
    }
}

}  // namespace lbm
