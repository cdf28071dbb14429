// kernels.cuh -- CUDA kernels of the D3Q19 update and their host launchers.
//
// Population layout in device memory: structure of arrays f[q][z][y][xp],
// x fastest, rows padded to a pitch nxp (a multiple of 16 elements) so that
// every row starts on a 32-byte sector; 64-bit element offsets throughout.
//
// State convention.  "Natural" parity: slot i of cell x holds f_i(x) of the
// post-stream state.  "A" parity (after an AA even step): slot opp(i) of x
// holds the post-collision f*_i(x) -- for a wall link the value that comes
// back, f*_i + L_opp(i), so the next read needs no boundary arithmetic.
//
// Semantics shared by every schedule (TWO_LATTICE, AA, MERGED): each time
// step collides with bgk_collide(), then every post-stream population is
// rounded to the storage format once (encode), the lid term of a wall link
// added before that rounding.  This is what makes the three schedules agree
// bit for bit.
#pragma once

#include "d3q19.cuh"
#include "ops.h"

#include <type_traits>

namespace lbm {

// L2 eviction-priority policies and loads/stores that carry one.  The
// adjoint step streams the recomputed state f^t (evict first) and keeps the
// adjoint fields lambda and dL/dF, re-read every step, in L2 (evict last):
// on the 128 x 64 x 64 channel both lambda buffers and dL/dF (93 MB) fit.
__device__ __forceinline__ uint64_t l2_policy_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
template <class T>
__device__ __forceinline__ T ld_pol(const T *p, uint64_t pol)
{
    T v;
    if constexpr (sizeof(T) == 4) {
        unsigned u;
        asm("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
        v = *reinterpret_cast<T *>(&u);
    } else if constexpr (sizeof(T) == 2) {
        unsigned short u;
        asm("ld.global.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(u) : "l"(p), "l"(pol));
        v = *reinterpret_cast<T *>(&u);
    } else {
        unsigned long long u;
        asm("ld.global.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(u) : "l"(p), "l"(pol));
        v = *reinterpret_cast<T *>(&u);
    }
    return v;
}
template <class T>
__device__ __forceinline__ void st_pol(T *p, T v, uint64_t pol)
{
    if constexpr (sizeof(T) == 4) {
        const unsigned u = *reinterpret_cast<const unsigned *>(&v);
        asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(u), "l"(pol));
    } else if constexpr (sizeof(T) == 2) {
        const unsigned short u = *reinterpret_cast<const unsigned short *>(&v);
        asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;" ::"l"(p), "h"(u), "l"(pol));
    } else {
        const unsigned long long u = *reinterpret_cast<const unsigned long long *>(&v);
        asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(u), "l"(pol));
    }
}

// Global store that allocates no L1 line, for values written once per sweep
// and not read back through the writing SM's L1 (later reads of them go
// through L2: TMA or cp.async copies, ld.global.cg, or the next launch).
template <class T>
__device__ __forceinline__ void st_no_l1(T *p, T v)
{
    static_assert(sizeof(T) == 2 || sizeof(T) == 4 || sizeof(T) == 8, "stored element");
    if constexpr (sizeof(T) == 4) {
        const unsigned u = *reinterpret_cast<const unsigned *>(&v);
        asm volatile("st.global.L1::no_allocate.b32 [%0], %1;" ::"l"(p), "r"(u));
    } else if constexpr (sizeof(T) == 2) {
        const unsigned short u = *reinterpret_cast<const unsigned short *>(&v);
        asm volatile("st.global.L1::no_allocate.b16 [%0], %1;" ::"l"(p), "h"(u));
    } else {
        const unsigned long long u = *reinterpret_cast<const unsigned long long *>(&v);
        asm volatile("st.global.L1::no_allocate.b64 [%0], %1;" ::"l"(p), "l"(u));
    }
}


// ---------------------------------------------------------------------------
// host -> device parameter conversion
// ---------------------------------------------------------------------------
template <class R>
inline Geom<R> make_geom(const HostGeom &h, int64_t pitch)
{
    Geom<R> g;
    g.nx = h.nx; g.ny = h.ny; g.nz = h.nz;
    for (int a = 0; a < 3; ++a) g.per[a] = h.per[a];
    for (int k = 0; k < 6; ++k) g.lid[k] = h.lid[k];
    g.nxp = pitch;
    g.plane = pitch * h.ny;
    g.slot = g.plane * h.nz;
    g.omega = R(h.omega);
    g.kf = R(h.kf);
    g.coll = h.coll;
    g.om = R(h.omega_m);
    g.kfm = R(h.kf_m);
    g.s3 = R(h.mrt_s3);
    g.s4 = R(h.mrt_s4);
    for (int i = 0; i < Q; ++i) g.L[i] = R(h.L[i]);
    for (int a = 0; a < 3; ++a) g.Fu[a] = R(h.Fu[a]);
    g.Ff = h.Ff;
    for (int i = 0; i < Q; ++i) g.noff[i] = (int32_t)(cz(i) * g.plane + cy(i) * pitch + cx(i));
    return g;
}

template <class T>
inline Dirs<T> make_dirs(T *base, int64_t slot)
{
    Dirs<T> d;
    for (int i = 0; i < Q; ++i) d.p[i] = base + (size_t)i * slot;
    return d;
}

template <class R>
__device__ __forceinline__ int64_t canon(const Geom<R> &g, int x, int y, int z)
{
    return ((int64_t)z * g.ny + y) * g.nx + x;
}

template <class R>
__device__ __forceinline__ int64_t ncanon(const Geom<R> &g)
{
    return (int64_t)g.nx * g.ny * g.nz;
}

// Natural post-stream value f_i from a stored element of slot I.
template <class S, int I>
__device__ __forceinline__ typename S::R natural_value(typename S::T v)
{
    using R = typename S::R;
    if constexpr (S::shifted) return radd(S::to_r(v), R(wgt(I)));
    else return S::to_r(v);
}

// Shifted populations of cell (x,y,z) at natural parity.
template <class S>
__device__ __forceinline__ void load_natural(const Geom<typename S::R> &g, const typename S::T *__restrict__ f,
                                             int x, int y, int z, typename S::R (&s)[Q])
{
    const int64_t c = cell_of(g, x, y, z);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = decode<S, i>(f[i * g.slot + c]);
    });
}

// Shifted post-stream populations of cell (x,y,z) from a state at A parity:
// f_k(x) sits in slot opp(k) of x - c_k, or (wall link) in slot k of x.
template <class S>
__device__ __forceinline__ void load_aparity(const Geom<typename S::R> &g, const typename S::T *__restrict__ f,
                                             int x, int y, int z, typename S::R (&s)[Q])
{
    const int64_t c = cell_of(g, x, y, z);
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            const int64_t off = (int64_t)cz(k) * g.plane + (int64_t)cy(k) * g.nxp + cx(k);
            s[k] = decode<S, k>(f[opp(k) * g.slot + c - off]);
        });
    } else {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            int sx, sy, sz;
            bool lid;
            if (link(g, x, y, z, -cx(k), -cy(k), -cz(k), sx, sy, sz, lid))
                s[k] = decode<S, k>(f[opp(k) * g.slot + cell_of(g, sx, sy, sz)]);
            else
                s[k] = decode<S, k>(f[k * g.slot + c]);
        });
    }
}

// Store post-collision populations with the streaming rule of a two-lattice
// push: slot i of x + c_i, or slot opp(i) of x (+ lid term) for a wall link.
template <class S>
__device__ __forceinline__ void push_store(const Geom<typename S::R> &g, typename S::T *__restrict__ dst,
                                           int x, int y, int z, const typename S::R (&s)[Q])
{
    const int64_t c = cell_of(g, x, y, z);
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            const int64_t off = (int64_t)cz(i) * g.plane + (int64_t)cy(i) * g.nxp + cx(i);
            dst[i * g.slot + c + off] = encode<S, i>(s[i]);
        });
    } else {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            int tx, ty, tz;
            bool lid;
            if (link(g, x, y, z, cx(i), cy(i), cz(i), tx, ty, tz, lid)) {
                dst[i * g.slot + cell_of(g, tx, ty, tz)] = encode<S, i>(s[i]);
            } else {
                typename S::R v = s[i];
                if (lid) v = radd(v, g.L[opp(i)]);
                dst[opp(i) * g.slot + c] = encode<S, opp(i)>(v);
            }
        });
    }
}

// ----- the same three access patterns on per-direction base pointers -----

template <class S>
__device__ __forceinline__ void load_natural_d(const Dirs<const typename S::T> &f, int c, typename S::R (&s)[Q])
{
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = decode<S, i>(f.p[i][c]);
    });
}

// A parity: f_k(x) in slot opp(k) of x - c_k, or (wall link) slot k of x.
template <class S>
__device__ __forceinline__ void load_aparity_d(const Geom<typename S::R> &g, const Dirs<const typename S::T> &f,
                                               int x, int y, int z, int c, typename S::R (&s)[Q])
{
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            s[k] = decode<S, k>(f.p[opp(k)][c - g.noff[k]]);
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if (fc.wall & face_mask(-cx(k), -cy(k), -cz(k))) s[k] = decode<S, k>(f.p[k][c]);
            else s[k] = decode<S, k>(f.p[opp(k)][c + step_offset<-cx(k), -cy(k), -cz(k)>(g, fc)]);
        });
    }
}

// Two-lattice push: slot i of x + c_i, or slot opp(i) of x (+ lid term).
template <class S>
__device__ __forceinline__ void push_store_d(const Geom<typename S::R> &g, const Dirs<typename S::T> &dst, int x,
                                             int y, int z, int c, const typename S::R (&s)[Q])
{
    if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            dst.p[i][c + g.noff[i]] = encode<S, i>(s[i]);
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr unsigned m = face_mask(cx(i), cy(i), cz(i));
            if (fc.wall & m) {
                typename S::R v = s[i];
                if (fc.lid & m) v = radd(v, g.L[opp(i)]);
                dst.p[opp(i)][c] = encode<S, opp(i)>(v);
            } else {
                dst.p[i][c + step_offset<cx(i), cy(i), cz(i)>(g, fc)] = encode<S, i>(s[i]);
            }
        });
    }
}

// ---------------------------------------------------------------------------
// K0: equilibrium initialisation (natural parity)
// ---------------------------------------------------------------------------
template <class S>
__global__ void k_init_eq(Geom<typename S::R> g, typename S::T *__restrict__ f, const void *rho, const void *u,
                          int dtype)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    double r = 1.0, ux = 0.0, uy = 0.0, uz = 0.0;
    if (dtype == 1) {
        const double *rp = (const double *)rho, *up = (const double *)u;
        if (rp) r = rp[cc];
        if (up) { ux = up[cc]; uy = up[n + cc]; uz = up[2 * n + cc]; }
    } else {
        const float *rp = (const float *)rho, *up = (const float *)u;
        if (rp) r = rp[cc];
        if (up) { ux = up[cc]; uy = up[n + cc]; uz = up[2 * n + cc]; }
    }
    const double usq = ux * ux + uy * uy + uz * uz;
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const double P = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        if constexpr (S::shifted) {
            const double sv = wgt(i) * ((r - 1.0) + r * P);
            f[i * g.slot + c] = S::from_r((typename S::R)sv);
        } else {
            const double fv = wgt(i) * r * (1.0 + P);
            f[i * g.slot + c] = S::from_r((typename S::R)fv);
        }
    });
}

// The moments (rho, u) of a cell that the adjoint step reads, as
// moments_of computes them: mom[a * slot + c], a = 0 .. 3 (rho, ux, uy, uz),
// compute type.
template <class R>
__device__ __forceinline__ void store_mom(R *__restrict__ mom, int64_t slot, int c, const Mom<R> &m)
{
    mom[c] = m.rho;
    mom[slot + c] = m.ux;
    mom[2 * slot + c] = m.uy;
    mom[3 * slot + c] = m.uz;
}

// Push of a cell in a row inside in y and z (only x faces can be crossed),
// for all lanes of a warp alike: f*_i goes to slot i of x + c_i
// (dout.p[i] = dst.p[i] + noff[i]), or, across an x wall, to slot opp(i) of
// x itself (same weight, same encoding) with the lid term of a lid face;
// across a periodic x face the target wraps by nx.  lo / hi: x is the first /
// last cell of its row.
template <class S>
__device__ __forceinline__ void push_xsel(const Geom<typename S::R> &g, const Dirs<typename S::T> &dst,
                                          const Dirs<typename S::T> &dout, int c, bool lo, bool hi,
                                          const typename S::R (&s)[Q])
{
    using R = typename S::R;
    using T = typename S::T;
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        if constexpr (cx(i) == 0) {
            dout.p[i][c] = encode<S, i>(s[i]);
        } else {
            const bool out = cx(i) > 0 ? hi : lo;
            T *a = dout.p[i] + c;
            R v = s[i];
            if (g.per[0]) {
                a = out ? a + (cx(i) > 0 ? -g.nx : g.nx) : a;
            } else {
                a = out ? dst.p[opp(i)] + c : a;
                if (g.lid[cx(i) > 0 ? 1 : 0]) v = out ? radd(v, g.L[opp(i)]) : v;
            }
            *a = encode<S, i>(v);
        }
    });
}

// A warp whose row is inside in y and z and that holds an x-edge cell (the
// case push_xsel and the odd step's select gather serve).
template <class G>
__device__ __forceinline__ bool xedge_warp(const G &g, int x, int y, int z)
{
    const int wx0 = x - (int)(threadIdx.x & 31);
    return y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1 && (wx0 == 0 || wx0 + 31 >= g.nx - 1);
}

// ---------------------------------------------------------------------------
// K1: two-lattice fused collide-and-push (natural -> natural)
// ---------------------------------------------------------------------------
// dout.p[i] = dst.p[i] + noff[i]: the push address of an interior cell.
// MOM: also store the moments of the input state in mom (the recompute of
// the adjoint's checkpoint segments).
template <class S, bool FORCE, int COLL = COLL_BGK, bool MOM = false>
__global__ void __launch_bounds__(128) k_two_lattice(Geom<typename S::R> g, Dirs<const typename S::T> src,
                                                     Dirs<typename S::T> dst, Dirs<typename S::T> dout,
                                                     typename S::R *__restrict__ mom)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[Q];
    load_natural_d<S>(src, c, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    if constexpr (MOM) store_mom<R>(mom, g.slot, c, moments_of<R, FORCE>(s, Fx, Fy, Fz));
    collide_sel<R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    // x-edge warps of rows inside in y and z: one select path for all lanes
    // (as the AA odd step's push)
    if (xedge_warp(g, x, y, z)) {
        push_xsel<S>(g, dst, dout, c, x == 0, x == g.nx - 1, s);
    } else if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            dout.p[i][c] = encode<S, i>(s[i]);
        });
    } else {
        push_store_d<S>(g, dst, x, y, z, c, s);
    }
}

// ---------------------------------------------------------------------------
// K2: AA even step (natural -> A parity), purely local: collide and write
// f*_i into slot opp(i) of the same cell (the "revert" of Sec. 3).  Planes
// z0 .. z0 + gridDim.z - 1.
// ---------------------------------------------------------------------------
// Post-collision value f*_i of one cell as the even step stores it in slot
// opp(i): + L_opp(i) when the link along c_i is a wall link ending on a lid.
template <class S>
__device__ __forceinline__ void even_outputs(const Geom<typename S::R> &g, int x, int y, int z,
                                             typename S::R (&s)[Q])
{
    if (interior(g, x, y, z)) return;
    const Faces fc = faces_of(g, x, y, z);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        constexpr unsigned m = face_mask(cx(i), cy(i), cz(i));
        if ((fc.wall & m) && (fc.lid & m)) s[i] = radd(s[i], g.L[opp(i)]);
    });
}

template <class S, bool FORCE, int COLL>
__device__ __forceinline__ void aa_even_cell(const Geom<typename S::R> &g, const Dirs<typename S::T> &f, int x, int y,
                                             int z, int c)
{
    using R = typename S::R;
    R s[Q];
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = decode<S, i>(f.p[i][c]);
    });
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    collide_sel<R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    even_outputs<S>(g, x, y, z, s);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        f.p[opp(i)][c] = encode<S, opp(i)>(s[i]);
    });
}

template <class S, bool FORCE, int COLL = COLL_BGK>
__global__ void __launch_bounds__(128) k_aa_even(Geom<typename S::R> g, Dirs<typename S::T> f, int z0)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z + z0;
    if (x >= g.nx) return;
    aa_even_cell<S, FORCE, COLL>(g, f, x, y, z, cell32(g, x, y, z));
}

// The even step for 2-byte storage, two neighbouring cells (x, x+1), x even,
// per thread: every access of the step is to the cells' own slots, so the
// pair moves as one 4-byte word per direction and converts with the packed
// two-element conversions (element-wise the same rounding).
template <class S>
struct Pair2 {
    __device__ static void decode2(uint32_t w, float &a, float &b)
    {
        if constexpr (std::is_same<typename S::T, __half>::value) {
            __half2 h = *reinterpret_cast<__half2 *>(&w);
            const float2 v = __half22float2(h);
            a = v.x; b = v.y;
        } else {
            __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
            const float2 v = __bfloat1622float2(h);
            a = v.x; b = v.y;
        }
    }
    __device__ static uint32_t encode2(float a, float b)
    {
        if constexpr (std::is_same<typename S::T, __half>::value) {
            __half2 h = __floats2half2_rn(a, b);
            return *reinterpret_cast<uint32_t *>(&h);
        } else {
            __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            return *reinterpret_cast<uint32_t *>(&h);
        }
    }
};

template <class S, bool FORCE, int COLL = COLL_BGK>
__global__ void __launch_bounds__(128) k_aa_even_pair(Geom<typename S::R> g, Dirs<typename S::T> f, int z0)
{
    static_assert(sizeof(typename S::T) == 2 && S::shifted, "2-byte shifted storage");
    using R = typename S::R;
    const int x = 2 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y, z = blockIdx.z + z0;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    if (x + 1 >= g.nx) {  // odd nx: the last cell alone
        aa_even_cell<S, FORCE, COLL>(g, f, x, y, z, c);
        return;
    }
    R a[Q], b[Q];
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        Pair2<S>::decode2(*reinterpret_cast<const uint32_t *>(f.p[i] + c), a[i], b[i]);
    });
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    collide_sel<R, FORCE, COLL>(g, a, Fx, Fy, Fz);
    force_at<R, FORCE>(g, canon(g, x + 1, y, z), ncanon(g), Fx, Fy, Fz);
    collide_sel<R, FORCE, COLL>(g, b, Fx, Fy, Fz);
    even_outputs<S>(g, x, y, z, a);
    even_outputs<S>(g, x + 1, y, z, b);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        *reinterpret_cast<uint32_t *>(f.p[opp(i)] + c) = Pair2<S>::encode2(a[i], b[i]);
    });
}

// ---------------------------------------------------------------------------
// K3: AA odd step (A parity -> natural): gather the streamed values, collide,
// scatter to the neighbours (the "swap_stream" of Sec. 3).  Cell x reads
// (x - c_k, opp(k)) and writes (x + c_i, i); no other cell touches those
// locations in this sweep, so the update is race-free in place.  Planes
// z0 .. z0 + gridDim.z - 1.
// ---------------------------------------------------------------------------
template <class S, bool FORCE, int COLL = COLL_BGK>
__global__ void __launch_bounds__(128) k_aa_odd(Geom<typename S::R> g, Dirs<typename S::T> f, Dirs<typename S::T> fin,
                                                Dirs<typename S::T> fout, int z0)
{
    // fin.p[k] = f.p[opp(k)] - noff[k] and fout.p[i] = f.p[i] + noff[i]: the
    // gather and push addresses of an interior cell, one index away
    using R = typename S::R;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z + z0;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[Q];
    // Warps whose row is inside in y and z and that hold an x-edge cell take
    // one branch-free path for all their lanes: links through an x face pick
    // their address (and the lid term) by select, so the warp does not split
    // into an interior and a boundary half.  The gather takes this path for
    // 4- and 8-byte storage only: with 2-byte storage the kernel is
    // instruction-bound and the select gather made it slower (0.31 -> 0.35 ms
    // at 256^3), while the select push helps every format (FP32 +6% with
    // both, 2-byte 0.31 -> 0.29 ms with the push alone).
    constexpr bool XSEL = sizeof(T) >= 4;
    const bool xsel = xedge_warp(g, x, y, z);
    const bool in = interior(g, x, y, z);
    const bool lo = x == 0, hi = x == g.nx - 1;
    if (XSEL && xsel) {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            // f_k(x) sits in slot opp(k) of x - c_k, or, across an x wall, in
            // slot k of x itself
            if constexpr (cx(k) == 0) {
                s[k] = decode<S, k>(fin.p[k][c]);
            } else {
                const bool out = cx(k) > 0 ? lo : hi;
                const T *a = fin.p[k] + c;
                if (g.per[0]) a = out ? a + (cx(k) > 0 ? g.nx : -g.nx) : a;
                else a = out ? f.p[k] + c : a;
                s[k] = decode<S, k>(*a);
            }
        });
    } else if (in) {
        static_for<Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            s[k] = decode<S, k>(fin.p[k][c]);
        });
    } else {
        load_aparity_d<S>(g, reinterpret_cast<const Dirs<const T> &>(f), x, y, z, c, s);
    }
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    collide_sel<R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    if (xsel) {
        push_xsel<S>(g, f, fout, c, lo, hi, s);
    } else if (in) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            fout.p[i][c] = encode<S, i>(s[i]);
        });
    } else {
        push_store_d<S>(g, f, x, y, z, c, s);
    }
}

// ---------------------------------------------------------------------------
// K5: moments, population export/import, raw parity normalisation
// ---------------------------------------------------------------------------
template <class S, bool FORCE, bool APAR>
__global__ void k_moments(Geom<typename S::R> g, const typename S::T *__restrict__ f, void *rho, void *u, int dtype)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    R s[Q];
    if constexpr (APAR) load_aparity<S>(g, f, x, y, z, s);
    else load_natural<S>(g, f, x, y, z, s);
    const int64_t n = ncanon(g), cc = canon(g, x, y, z);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, cc, n, Fx, Fy, Fz);
    const Mom<R> m = moments_of<R, FORCE>(s, Fx, Fy, Fz);
    if (dtype == 1) {
        if (rho) ((double *)rho)[cc] = (double)m.rho;
        if (u) {
            double *up = (double *)u;
            up[cc] = (double)m.ux; up[n + cc] = (double)m.uy; up[2 * n + cc] = (double)m.uz;
        }
    } else {
        if (rho) ((float *)rho)[cc] = (float)m.rho;
        if (u) {
            float *up = (float *)u;
            up[cc] = (float)m.ux; up[n + cc] = (float)m.uy; up[2 * n + cc] = (float)m.uz;
        }
    }
}

template <class S, bool APAR>
__global__ void k_export(Geom<typename S::R> g, const typename S::T *__restrict__ f, void *out, int dtype)
{
    using R = typename S::R;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    const bool in = interior(g, x, y, z);
    static_for<Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        T v;
        if constexpr (APAR) {
            int sx, sy, sz;
            bool lid;
            if (in) v = f[opp(k) * g.slot + c - ((int64_t)cz(k) * g.plane + (int64_t)cy(k) * g.nxp + cx(k))];
            else if (link(g, x, y, z, -cx(k), -cy(k), -cz(k), sx, sy, sz, lid))
                v = f[opp(k) * g.slot + cell_of(g, sx, sy, sz)];
            else v = f[k * g.slot + c];
        } else {
            v = f[k * g.slot + c];
        }
        const R nv = natural_value<S, k>(v);
        if (dtype == 1) ((double *)out)[k * n + cc] = (double)nv;
        else ((float *)out)[k * n + cc] = (float)nv;
    });
}

template <class S>
__global__ void k_import(Geom<typename S::R> g, typename S::T *__restrict__ f, const void *in, int dtype)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    static_for<Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        if (dtype == 1) {
            const double v = ((const double *)in)[k * n + cc];
            f[k * g.slot + c] = S::from_r((R)(S::shifted ? v - wgt(k) : v));
        } else {
            const float v = ((const float *)in)[k * n + cc];
            f[k * g.slot + c] = S::from_r(S::shifted ? (R)rsub(v, float(wgt(k))) : (R)v);
        }
    });
}

// Raw copy of a state into natural parity (no rounding): from A parity this
// is the pure gather, element by element; used for exact checkpoints.
template <class S>
__global__ void k_raw_natural(Geom<typename S::R> g, const typename S::T *__restrict__ f, typename S::T *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t c = cell_of(g, x, y, z);
    static_for<Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        int sx, sy, sz;
        bool lid;
        if (link(g, x, y, z, -cx(k), -cy(k), -cz(k), sx, sy, sz, lid))
            out[k * g.slot + c] = f[opp(k) * g.slot + cell_of(g, sx, sy, sz)];
        else
            out[k * g.slot + c] = f[k * g.slot + c];
    });
}

// ---------------------------------------------------------------------------
// K6: deterministic FP64 reductions (mass, momentum, kinetic energy)
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <class S, bool FORCE, bool APAR>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_partial(Geom<typename S::R> g, const typename S::T *__restrict__ f,
                                                                double *__restrict__ partial, int *__restrict__ flag)
{
    using R = typename S::R;
    const int64_t n = ncanon(g);
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (int64_t cc = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; cc < n; cc += (int64_t)gridDim.x * RED_THREADS) {
        const int x = (int)(cc % g.nx);
        const int64_t r = cc / g.nx;
        const int y = (int)(r % g.ny), z = (int)(r / g.ny);
        R s[Q];
        if constexpr (APAR) load_aparity<S>(g, f, x, y, z, s);
        else load_natural<S>(g, f, x, y, z, s);
        // per-cell moments in the compute type (FP64 for FP64 storage), the
        // sums over cells in FP64; rho = 1 + dr is formed in FP64
        R dr = R(0), jx = R(0), jy = R(0), jz = R(0);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            const R v = s[i];
            dr += v;
            if constexpr (cx(i) != 0) jx = cx(i) > 0 ? jx + v : jx - v;
            if constexpr (cy(i) != 0) jy = cy(i) > 0 ? jy + v : jy - v;
            if constexpr (cz(i) != 0) jz = cz(i) > 0 ? jz + v : jz - v;
        });
        R Fx, Fy, Fz;
        force_at<R, FORCE>(g, cc, n, Fx, Fy, Fz);
        const R rho = R(1) + dr, inv = R(1) / rho;
        const R ux = (jx + R(0.5) * Fx) * inv, uy = (jy + R(0.5) * Fy) * inv, uz = (jz + R(0.5) * Fz) * inv;
        const R ke = R(0.5) * rho * (ux * ux + uy * uy + uz * uz);
        if (!isfinite(rho) || !isfinite(ke)) bad = true;
        acc[0] += 1.0 + (double)dr; acc[1] += (double)jx; acc[2] += (double)jy; acc[3] += (double)jz;
        acc[4] += (double)ke;
    }
    if (bad) atomicOr(flag, 1);
    __shared__ double red[5][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = lane < RED_THREADS / 32 ? red[k][lane] : 0.0;
            v = warp_sum(v);
            if (lane == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = v;
        }
    }
}

static __global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double *__restrict__ partial, int nblocks,
                                                              double *__restrict__ out)
{
    __shared__ double red[RED_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 5; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += RED_THREADS) v += partial[(int64_t)k * nblocks + b];
        v = warp_sum(v);
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (warp == 0) {
            double t = lane < RED_THREADS / 32 ? red[lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) out[k] = t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K4: two steps per sweep: nsweep.cuh (neighbour-synchronised) and
// merged3.cuh (shadow-shell).
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// K8: adjoint of one step (two buffers) and its seed.
// ---------------------------------------------------------------------------
// lam_out(x) = (d f^{t+1}/d f^t)^T lam_in at cell x, gF(x) += (d f^{t+1}/dF(x))^T lam_in.
// f and lam share the geometry g (pitch g.nxp); gF and the force are canonical.
// fd.p[i] = f + i slot; lin.p[i] = lam_in + i slot + noff[i], the gather
// address of an interior cell; lout.p[j] = lam_out + j slot.
// MOMIN: the moments of f^t come from mom (store_mom layout) instead of
// being computed from f^t (fd unused).
template <class S, bool FORCE, bool MOMIN = false>
__global__ void __launch_bounds__(128) k_adjoint(Geom<typename S::R> g, Dirs<const typename S::T> fd,
                                                 Dirs<const typename S::R> lin, Dirs<typename S::R> lout,
                                                 double *__restrict__ gF, const typename S::R *__restrict__ mom)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z);
    const int c = cell32(g, x, y, z);
    const uint64_t pf = l2_policy_first(), pl = l2_policy_last();
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, cc, n, Fx, Fy, Fz);
    Mom<R> m;
    if constexpr (MOMIN) {
        m.rho = ld_pol(mom + c, pf);
        m.ux = ld_pol(mom + g.slot + c, pf);
        m.uy = ld_pol(mom + 2 * g.slot + c, pf);
        m.uz = ld_pol(mom + 3 * g.slot + c, pf);
    } else {
        R s[Q];
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            s[i] = decode<S, i>(ld_pol(fd.p[i] + c, pf));
        });
        m = moments_of<R, FORCE>(s, Fx, Fy, Fz);
    }
    const R usq = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    // mu_i = dL/df*_i: the transpose of streaming
    R mu[Q];
    if (xedge_warp(g, x, y, z)) {
        // x-edge warps of rows inside in y and z: one select path for all
        // lanes (links through an x face only), as in the AA odd step
        const bool lo = x == 0, hi = x == g.nx - 1;
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if constexpr (cx(i) == 0) {
                mu[i] = ld_pol(lin.p[i] + c, pl);
            } else {
                const bool out = cx(i) > 0 ? hi : lo;
                const R *a = lin.p[i] + c;
                if (g.per[0]) a = out ? a + (cx(i) > 0 ? -g.nx : g.nx) : a;
                else a = out ? lin.p[opp(i)] + c + g.noff[i] : a;
                mu[i] = ld_pol(a, pl);
            }
        });
    } else if (interior(g, x, y, z)) {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            mu[i] = ld_pol(lin.p[i] + c, pl);
        });
    } else {
        // lin.p[i][c + wrap] is lam_in_i at the (wrapped) target of the push;
        // lin.p[opp(i)][c + noff[i]] is lam_in_opp(i) of the cell itself
        const Faces fc = faces_of(g, x, y, z);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if (fc.wall & face_mask(cx(i), cy(i), cz(i))) mu[i] = ld_pol(lin.p[opp(i)] + c + g.noff[i], pl);
            else mu[i] = ld_pol(lin.p[i] + c + wrap_adj<cx(i), cy(i), cz(i)>(fc), pl);
        });
    }
    // a = sum mu_i dfeq_i/drho; b = sum mu_i dfeq_i/du; sv = sum mu_i dS_i/du;
    // gv = sum mu_i dS_i/dF|_u.  With wm_i = w_i mu_i and its direction
    // moments M0 = sum wm_i, M1 = sum wm_i c_i, M2 = sum wm_i c_i c_i^T:
    //   a = M0 (1 - 1.5 u.u) + 3 M1.u + 4.5 u.M2 u
    //   gv = 3 M1 + 9 M2 u - 3 u M0,  b = rho gv
    //   sv = 9 M2 F - 3 F M0
    // (the c_i are 0 or +-1, so the moments are sums and differences of wm_i).
    R M0 = R(0), M1x = R(0), M1y = R(0), M1z = R(0);
    R Mxx = R(0), Myy = R(0), Mzz = R(0), Mxy = R(0), Mxz = R(0), Myz = R(0);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        const R wm = R(wgt(i)) * mu[i];
        M0 += wm;
        if constexpr (cx(i) != 0) { M1x += cx(i) > 0 ? wm : -wm; Mxx += wm; }
        if constexpr (cy(i) != 0) { M1y += cy(i) > 0 ? wm : -wm; Myy += wm; }
        if constexpr (cz(i) != 0) { M1z += cz(i) > 0 ? wm : -wm; Mzz += wm; }
        if constexpr (cx(i) * cy(i) != 0) Mxy += cx(i) * cy(i) > 0 ? wm : -wm;
        if constexpr (cx(i) * cz(i) != 0) Mxz += cx(i) * cz(i) > 0 ? wm : -wm;
        if constexpr (cy(i) * cz(i) != 0) Myz += cy(i) * cz(i) > 0 ? wm : -wm;
    });
    const R Mux = Mxx * m.ux + Mxy * m.uy + Mxz * m.uz;
    const R Muy = Mxy * m.ux + Myy * m.uy + Myz * m.uz;
    const R Muz = Mxz * m.ux + Myz * m.uy + Mzz * m.uz;
    const R a = M0 * (R(1) - R(1.5) * usq) + R(3) * (M1x * m.ux + M1y * m.uy + M1z * m.uz) +
                R(4.5) * (m.ux * Mux + m.uy * Muy + m.uz * Muz);
    const R gx = R(3) * M1x + R(9) * Mux - R(3) * m.ux * M0;
    const R gy = R(3) * M1y + R(9) * Muy - R(3) * m.uy * M0;
    const R gz = R(3) * M1z + R(9) * Muz - R(3) * m.uz * M0;
    R sx = R(0), sy = R(0), sz = R(0);
    if constexpr (FORCE) {
        sx = R(9) * (Mxx * Fx + Mxy * Fy + Mxz * Fz) - R(3) * Fx * M0;
        sy = R(9) * (Mxy * Fx + Myy * Fy + Myz * Fz) - R(3) * Fy * M0;
        sz = R(9) * (Mxz * Fx + Myz * Fy + Mzz * Fz) - R(3) * Fz * M0;
    }
    const R ex = g.omega * (m.rho * gx) + g.kf * sx, ey = g.omega * (m.rho * gy) + g.kf * sy,
            ez = g.omega * (m.rho * gz) + g.kf * sz;
    const R inv = R(1) / m.rho;
    // lam_out_j = (1 - omega) mu_j + omega a + e.(c_j - u) / rho
    const R Ex = ex * inv, Ey = ey * inv, Ez = ez * inv;
    const R base = g.omega * a - (Ex * m.ux + Ey * m.uy + Ez * m.uz);
    static_for<Q>([&](auto K) {
        constexpr int j = decltype(K)::value;
        R v = (R(1) - g.omega) * mu[j] + base;
        if constexpr (cx(j) != 0) v = cx(j) > 0 ? v + Ex : v - Ex;
        if constexpr (cy(j) != 0) v = cy(j) > 0 ? v + Ey : v - Ey;
        if constexpr (cz(j) != 0) v = cz(j) > 0 ? v + Ez : v - Ez;
        st_pol(lout.p[j] + c, v, pl);
    });
    if (gF) {
        const R h = R(0.5) * inv;
        st_pol(gF + cc, ld_pol(gF + cc, pl) + (double)(g.kf * gx + ex * h), pl);
        st_pol(gF + n + cc, ld_pol(gF + n + cc, pl) + (double)(g.kf * gy + ey * h), pl);
        st_pol(gF + 2 * n + cc, ld_pol(gF + 2 * n + cc, pl) + (double)(g.kf * gz + ez * h), pl);
    }
}

// The moments of state f (natural parity) into mom (store_mom layout): the
// last state of an adjoint checkpoint segment, which no recompute step reads.
template <class S, bool FORCE>
__global__ void __launch_bounds__(128) k_adj_moments(Geom<typename S::R> g, Dirs<const typename S::T> src,
                                                     typename S::R *__restrict__ mom)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[Q];
    load_natural_d<S>(src, c, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    store_mom<R>(mom, g.slot, c, moments_of<R, FORCE>(s, Fx, Fy, Fz));
}

// lam = dL/df for L(rho, u) of state f (natural parity); gF += dL/du / (2 rho).
template <class S, bool FORCE>
__global__ void k_adjoint_seed(Geom<typename S::R> g, const typename S::T *__restrict__ f, const void *dLdrho,
                               const void *dLdu, int dtype, typename S::R *__restrict__ lam, double *__restrict__ gF)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    R s[Q];
    load_natural<S>(g, f, x, y, z, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, cc, n, Fx, Fy, Fz);
    const Mom<R> m = moments_of<R, FORCE>(s, Fx, Fy, Fz);
    R dr = R(0), dx, dy, dz;
    if (dtype == 1) {
        const double *du = (const double *)dLdu;
        if (dLdrho) dr = (R)((const double *)dLdrho)[cc];
        dx = (R)du[cc]; dy = (R)du[n + cc]; dz = (R)du[2 * n + cc];
    } else {
        const float *du = (const float *)dLdu;
        if (dLdrho) dr = (R)((const float *)dLdrho)[cc];
        dx = (R)du[cc]; dy = (R)du[n + cc]; dz = (R)du[2 * n + cc];
    }
    const R inv = R(1) / m.rho;
    static_for<Q>([&](auto K) {
        constexpr int j = decltype(K)::value;
        lam[j * g.slot + c] = dr + (dx * (R(cx(j)) - m.ux) + dy * (R(cy(j)) - m.uy) + dz * (R(cz(j)) - m.uz)) * inv;
    });
    if (gF) {
        const R h = R(0.5) * inv;
        gF[cc] += (double)(dx * h);
        gF[n + cc] += (double)(dy * h);
        gF[2 * n + cc] += (double)(dz * h);
    }
}

// Cast between a canonical array of dtype and an R array of pitch g.nxp.
template <class R>
__global__ void k_canon_to_pitched(Geom<R> g, const void *in, int dtype, R *__restrict__ out, int ncomp)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    for (int k = 0; k < ncomp; ++k)
        out[k * g.slot + c] = dtype == 1 ? (R)((const double *)in)[k * n + cc] : (R)((const float *)in)[k * n + cc];
}
template <class R>
__global__ void k_pitched_to_canon(Geom<R> g, const R *__restrict__ in, void *out, int dtype, int ncomp)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    for (int k = 0; k < ncomp; ++k) {
        if (dtype == 1) ((double *)out)[k * n + cc] = (double)in[k * g.slot + c];
        else ((float *)out)[k * n + cc] = (float)in[k * g.slot + c];
    }
}

}  // namespace lbm
