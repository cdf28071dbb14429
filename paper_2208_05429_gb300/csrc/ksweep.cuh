// ksweep.cuh -- K time steps per sweep (K = 3 or 4) on two lattices: the
// merge of more than two collision-streaming steps that the paper leaves as
// future work for GPUs (Sec. 6).
//
// One CTA per TX x TY column tile marches z and carries a pipeline of K
// levels in shared memory.  Level s (s = 0 .. K-1) holds the post-collision
// populations after s steps in a ring of three planes, on the tile widened
// by a halo of K - s cells on each side (the cells whose values level s + 1
// pulls from).  In pipeline stage t (t = -K .. nz-1+K) level s produces
// plane t - s: level 0 loads and collides the source state, level s > 0
// pulls from level s - 1 (planes t-s-1 .. t-s+1, the previous stage's three
// slots), and level K pulls the K-th post-stream state of the tile into the
// destination lattice.  The halos are recomputed by every tile that needs
// them (overlapped tiles): no tile waits on another, at the price of about
// 1.9 collisions per cell update for K = 3 on 16 x 8 tiles.
//
// Every pulled value passes through the storage format (decode(encode(v)),
// the lid term of a wall link added first) exactly as the two-lattice step
// stores and reloads it, and every collision is bgk_collide() (this sweep
// is built for the BGK collision): the result equals K two-lattice steps bit
// for bit.  Periodic axes are read through
// wrapped coordinates (a halo wider than the lattice holds repeated
// cells); across a wall or lid the pull bounces back half-way.
#pragma once

#include "kernels.cuh"

namespace lbm {

template <int K>
struct KSL {
    static_assert(K == 3 || K == 4, "three or four steps per sweep");
    static constexpr int TX = 16, TY = K == 3 ? 8 : 4, THREADS = 256;
    __host__ __device__ static constexpr int rw(int s) { return TX + 2 * (K - s); }
    __host__ __device__ static constexpr int rh(int s) { return TY + 2 * (K - s); }
    __host__ __device__ static constexpr int cells(int s) { return rw(s) * rh(s); }
    // first compute-type element of level s's ring
    __host__ __device__ static constexpr int base(int s) { return s == 0 ? 0 : base(s - 1) + 3 * Q * cells(s - 1); }
    static constexpr size_t smem_bytes = (size_t)base(K) * sizeof(float);
};

template <class S, bool FORCE, int K>
__global__ void __launch_bounds__(KSL<K>::THREADS, 1)
    k_ksweep(Geom<typename S::R> g, Dirs<const typename S::T> src, Dirs<typename S::T> dst)
{
    using R = typename S::R;
    using LK = KSL<K>;
    static_assert(sizeof(R) == sizeof(float), "FP32 compute");
    extern __shared__ __align__(16) float ks_smem[];
    R *const ring = reinterpret_cast<R *>(ks_smem);
    const int x0 = blockIdx.x * LK::TX, y0 = blockIdx.y * LK::TY;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const bool px = g.per[0] != 0, py = g.per[1] != 0, pz = g.per[2] != 0;
    for (int t = -K; t < nz + K; ++t) {
        for (int s = 0; s <= K; ++s) {
            const int p = t - s;
            const int h = s < K ? K - s : 0;
            bool live;
            if (s < K) live = (p >= 0 && p < nz) || (pz && p >= -h && p < nz + h);
            else live = p >= 0 && p < nz;
            if (live) {
                const int rws = LK::TX + 2 * h, rhs = LK::TY + 2 * h, ncell = rws * rhs;
                int wz = p;
                while (wz < 0) wz += nz;
                while (wz >= nz) wz -= nz;
                // z faces crossed by a pull from plane p (non-periodic z)
                const bool zlo = !pz && p == 0, zhi = !pz && p == nz - 1;
                for (int r = threadIdx.x; r < ncell; r += LK::THREADS) {
                    const int rx = r % rws, ry = r / rws;
                    const int X = x0 - h + rx, Y = y0 - h + ry;
                    if ((!px && (X < 0 || X >= nx)) || (!py && (Y < 0 || Y >= ny))) continue;
                    // periodic axes: wrap (a halo wider than the lattice
                    // wraps more than once)
                    int wx = X, wy = Y;
                    while (wx < 0) wx += nx;
                    while (wx >= nx) wx -= nx;
                    while (wy < 0) wy += ny;
                    while (wy >= ny) wy -= ny;
                    const int64_t c = cell_of(g, wx, wy, wz);
                    R v[Q];
                    if (s == 0) {
                        static_for<Q>([&](auto KK) {
                            constexpr int i = decltype(KK)::value;
                            v[i] = decode<S, i>(src.p[i][c]);
                        });
                    } else {
                        // pull f_i(X) from level s-1: post-collision value of
                        // X - c_i, or (wall link) of X itself along opp(i)
                        // plus the lid term of a lid face
                        const bool xlo = !px && X == 0, xhi = !px && X == nx - 1;
                        const bool ylo = !py && Y == 0, yhi = !py && Y == ny - 1;
                        const int ps = s - 1, pr = LK::TX + 2 * (K - ps);
                        const int pcells = pr * (LK::TY + 2 * (K - ps));
                        const R *lv = ring + LK::base(ps);
                        const int qx = rx + 1, qy = ry + 1;  // X, Y in level s-1's region
                        static_for<Q>([&](auto KK) {
                            constexpr int i = decltype(KK)::value;
                            const bool wl = (cx(i) > 0 && xlo) || (cx(i) < 0 && xhi) || (cy(i) > 0 && ylo) ||
                                            (cy(i) < 0 && yhi) || (cz(i) > 0 && zlo) || (cz(i) < 0 && zhi);
                            R val;
                            if (wl) {
                                const bool lid = (cx(i) > 0 && xlo && g.lid[0]) || (cx(i) < 0 && xhi && g.lid[1]) ||
                                                 (cy(i) > 0 && ylo && g.lid[2]) || (cy(i) < 0 && yhi && g.lid[3]) ||
                                                 (cz(i) > 0 && zlo && g.lid[4]) || (cz(i) < 0 && zhi && g.lid[5]);
                                const int sl = ((p % 3) + 3) % 3;
                                val = lv[(sl * Q + opp(i)) * pcells + qy * pr + qx];
                                if (lid) val = radd(val, g.L[i]);
                            } else {
                                const int sp = p - cz(i);
                                const int sl = ((sp % 3) + 3) % 3;
                                val = lv[(sl * Q + i) * pcells + (qy - cy(i)) * pr + (qx - cx(i))];
                            }
                            v[i] = s == K ? val : roundtrip<S, i>(val);
                        });
                    }
                    if (s == K) {
                        if (X < nx && Y < ny) {
                            static_for<Q>([&](auto KK) {
                                constexpr int i = decltype(KK)::value;
                                dst.p[i][c] = encode<S, i>(v[i]);
                            });
                        }
                    } else {
                        R Fx, Fy, Fz;
                        force_at<R, FORCE>(g, canon(g, wx, wy, wz), ncanon(g), Fx, Fy, Fz);
                        bgk_collide<R, FORCE>(v, g.omega, g.kf, Fx, Fy, Fz);
                        const int sl = ((p % 3) + 3) % 3;
                        R *const out = ring + LK::base(s) + (sl * Q) * ncell + r;
                        static_for<Q>([&](auto KK) {
                            constexpr int i = decltype(KK)::value;
                            out[i * ncell] = v[i];
                        });
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <class S, bool FORCE, int K>
cudaError_t launch_ksweep_k(const Geom<typename S::R> &g, const Dirs<const typename S::T> &a,
                            const Dirs<typename S::T> &b, int nx, int ny, cudaStream_t st)
{
    using LK = KSL<K>;
    static bool attr_set = false;  // once per process: not inside a stream capture
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_ksweep<S, FORCE, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)LK::smem_bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((nx + LK::TX - 1) / LK::TX, (ny + LK::TY - 1) / LK::TY);
    k_ksweep<S, FORCE, K><<<grid, LK::THREADS, LK::smem_bytes, st>>>(g, a, b);
    return cudaGetLastError();
}

// K steps (3 or 4) from src to dst (natural parity, two lattices).
template <class S>
cudaError_t launch_ksweep(const HostGeom &h, int64_t pitch, bool force, int K, const void *src, void *dst,
                          cudaStream_t st)
{
    using T = typename S::T;
    using R = typename S::R;
    const Geom<R> g = make_geom<R>(h, pitch);
    const int64_t slot = pitch * h.ny * h.nz;
    const Dirs<const T> a = make_dirs((const T *)src, slot);
    const Dirs<T> b = make_dirs((T *)dst, slot);
    if (K == 3) return force ? launch_ksweep_k<S, true, 3>(g, a, b, h.nx, h.ny, st)
                             : launch_ksweep_k<S, false, 3>(g, a, b, h.nx, h.ny, st);
    if (K == 4) return force ? launch_ksweep_k<S, true, 4>(g, a, b, h.nx, h.ny, st)
                             : launch_ksweep_k<S, false, 4>(g, a, b, h.nx, h.ny, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
