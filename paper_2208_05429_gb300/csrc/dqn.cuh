// dqn.cuh -- the single-step update on the D3Q15 and D3Q27 lattices: their
// collision (BGK, TRT or regularised BGK, with Guo forcing), the
// two-lattice step, the AA even / odd pair, moments, population export /
// import and the FP64 reductions, with the same storage formats, layout,
// state convention and boundary rule as the D3Q19 kernels (kernels.cuh):
//
//  * SoA f[q][z][y][xp], pitch xp a multiple of 16 elements;
//  * natural parity: slot i of x holds f_i(x); A parity (after an even
//    step): slot opp(i) of x holds f*_i(x), plus the lid term L_opp(i) when
//    the link along c_i is a wall link that crosses a lid face;
//  * a wall link bounces back half-way: f_opp(i)(x) = f*_i(x) + L_opp(i),
//    L_k = 6 w_k rho_w (c_k . u_lid) on a lid, 0 on a plain wall.
//
// One thread per cell, 128 cells of a row per CTA, every direction slot
// read and written with x fastest (coalesced, the cx = +-1 directions one
// element off).  Arithmetic uses the explicitly rounded operations of
// d3q19.cuh, so the two-lattice and AA schedules agree bit for bit.
#pragma once

#include "kernels.cuh"
#include "lattice.cuh"

#include <string.h>

namespace lbm {

// Lid terms L_k of lattice QN (compute type).
template <class R, int QN>
struct LidQ {
    R L[QN];
};

template <class R, int QN>
inline LidQ<R, QN> make_lidq(const HostGeom &h)
{
    LidQ<R, QN> l;
    for (int k = 0; k < QN; ++k) l.L[k] = R(h.L[k]);
    return l;
}

template <class S>
__device__ __forceinline__ typename S::R dq_decode(typename S::T v, typename S::R w)
{
    if constexpr (S::shifted) return S::to_r(v);
    else return rsub(S::to_r(v), w);
}
template <class S>
__device__ __forceinline__ typename S::T dq_encode(typename S::R s, typename S::R w)
{
    if constexpr (S::shifted) return S::from_r(s);
    else return S::from_r(radd(s, w));
}

// c_i . (ax, ay, az) as a signed sum of the non-zero components.
template <class L, int I, class R>
__device__ __forceinline__ R dq_cdot(R ax, R ay, R az)
{
    R v = R(0);
    bool first = true;
    auto acc = [&](int c, R a) {
        if (c == 0) return;
        if (first) { v = c > 0 ? a : -a; first = false; }
        else v = c > 0 ? radd(v, a) : rsub(v, a);
    };
    acc(L::cx(I), ax);
    acc(L::cy(I), ay);
    acc(L::cz(I), az);
    return v;
}

// ---------------------------------------------------------------------------
// Collision of one cell in the shifted form s_i = f_i - w_i:
//   rho = 1 + sum s_i, u = (sum s_i c_i + F/2) / rho,
//   feq_i - w_i = w_i (rho - 1 + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)),
//   S_i = w_i (3 (c_i - u) + 9 (c_i . u) c_i) . F,
// then BGK  s*_i = s_i - omega (s_i - seq_i) + (1 - omega/2) S_i,
//      TRT  the same on the symmetric parts with omega, on the
//           antisymmetric parts with omega- (g.om, g.kfm),
//      REG  s*_i = seq_i + (1 - omega) w_i (3 c_i . J + 4.5 (c_i c_i - I/3) : Pi)
//           + (1 - omega/2) S_i, J and Pi the first and second moments of
//           s - seq (the regularised BGK form).
// ---------------------------------------------------------------------------
template <class L, class R, bool FORCE, int COLL>
__device__ __forceinline__ void dq_collide(const Geom<R> &g, R (&s)[L::Q], R Fx, R Fy, R Fz)
{
    constexpr int Q = L::Q;
    R drho = s[0];
    static_for<Q - 1>([&](auto K) { drho = radd(drho, s[decltype(K)::value + 1]); });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        if constexpr (L::cx(i) == 1) jx = radd(jx, s[i]);
        if constexpr (L::cx(i) == -1) jx = rsub(jx, s[i]);
        if constexpr (L::cy(i) == 1) jy = radd(jy, s[i]);
        if constexpr (L::cy(i) == -1) jy = rsub(jy, s[i]);
        if constexpr (L::cz(i) == 1) jz = radd(jz, s[i]);
        if constexpr (L::cz(i) == -1) jz = rsub(jz, s[i]);
    });
    const R rho = radd(R(1), drho);
    const R inv = rdiv(R(1), rho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    const R ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const R usq15 = rmul(R(1.5), rfma(ux, ux, rfma(uy, uy, rmul(uz, uz))));
    R uF = R(0);
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    R seq[Q], S[Q];
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        const R w = R(L::wgt(i));
        const R cu = dq_cdot<L, i>(ux, uy, uz);
        const R P = rsub(rmul(cu, rfma(R(4.5), cu, R(3))), usq15);
        seq[i] = rmul(w, rfma(rho, P, drho));
        if constexpr (FORCE) {
            const R cF = dq_cdot<L, i>(Fx, Fy, Fz);
            S[i] = rmul(w, rfma(rmul(R(9), cu), cF, rmul(R(3), rsub(cF, uF))));
        } else {
            S[i] = R(0);
        }
    });
    const R om = g.omega, kf = g.kf;
    if constexpr (COLL == COLL_TRT) {
        const R omm = g.om, kfm = g.kfm;
        {
            R v = rfma(-om, rsub(s[0], seq[0]), s[0]);
            if constexpr (FORCE) v = rfma(kf, S[0], v);
            s[0] = v;
        }
        static_for<L::H>([&](auto K) {
            constexpr int i = decltype(K)::value + 1, j = L::opp(i);
            const R np = rmul(R(0.5), radd(rsub(s[i], seq[i]), rsub(s[j], seq[j])));
            const R nm = rmul(R(0.5), rsub(rsub(s[i], seq[i]), rsub(s[j], seq[j])));
            R a = rfma(-om, np, s[i]), b = rfma(-om, np, s[j]);
            a = rfma(-omm, nm, a);
            b = rfma(omm, nm, b);
            if constexpr (FORCE) {
                const R sp = rmul(R(0.5), radd(S[i], S[j])), sm = rmul(R(0.5), rsub(S[i], S[j]));
                a = rfma(kfm, sm, rfma(kf, sp, a));
                b = rfma(-kfm, sm, rfma(kf, sp, b));
            }
            s[i] = a;
            s[j] = b;
        });
    } else if constexpr (COLL == COLL_REG) {
        R J[3] = {R(0), R(0), R(0)}, Pi[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};  // xx yy zz xy xz yz
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            const R n = rsub(s[i], seq[i]);
            constexpr int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (c[a] == 1) J[a] = radd(J[a], n);
                if (c[a] == -1) J[a] = rsub(J[a], n);
                if (c[a] != 0) Pi[a] = radd(Pi[a], n);
            }
            constexpr int pxy = c[0] * c[1], pxz = c[0] * c[2], pyz = c[1] * c[2];
            if constexpr (pxy == 1) Pi[3] = radd(Pi[3], n);
            if constexpr (pxy == -1) Pi[3] = rsub(Pi[3], n);
            if constexpr (pxz == 1) Pi[4] = radd(Pi[4], n);
            if constexpr (pxz == -1) Pi[4] = rsub(Pi[4], n);
            if constexpr (pyz == 1) Pi[5] = radd(Pi[5], n);
            if constexpr (pyz == -1) Pi[5] = rsub(Pi[5], n);
        });
        const R tr3 = rmul(R(1.0 / 3.0), radd(radd(Pi[0], Pi[1]), Pi[2]));
        const R keep = rsub(R(1), om);
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr int c[3] = {L::cx(i), L::cy(i), L::cz(i)};
            const R cJ = dq_cdot<L, i>(J[0], J[1], J[2]);
            // (c c - I/3) : Pi = sum_a c_a^2 Pi_aa + 2 sum_{a<b} c_a c_b Pi_ab - tr Pi / 3
            R qp = rsub(R(0), tr3);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (c[a] != 0) qp = radd(qp, Pi[a]);
            constexpr int pxy = c[0] * c[1], pxz = c[0] * c[2], pyz = c[1] * c[2];
            if constexpr (pxy != 0) qp = pxy > 0 ? rfma(R(2), Pi[3], qp) : rfma(R(-2), Pi[3], qp);
            if constexpr (pxz != 0) qp = pxz > 0 ? rfma(R(2), Pi[4], qp) : rfma(R(-2), Pi[4], qp);
            if constexpr (pyz != 0) qp = pyz > 0 ? rfma(R(2), Pi[5], qp) : rfma(R(-2), Pi[5], qp);
            const R f1 = rmul(R(L::wgt(i)), rfma(R(3), cJ, rmul(R(4.5), qp)));
            R v = rfma(keep, f1, seq[i]);
            if constexpr (FORCE) v = rfma(kf, S[i], v);
            s[i] = v;
        });
    } else {
        static_for<Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            R v = rfma(-om, rsub(s[i], seq[i]), s[i]);
            if constexpr (FORCE) v = rfma(kf, S[i], v);
            s[i] = v;
        });
    }
}

// Shifted populations of cell (x,y,z) at natural parity.
template <class L, class S>
__device__ __forceinline__ void dq_load_natural(const Geom<typename S::R> &g, const typename S::T *__restrict__ f,
                                                int64_t c, typename S::R (&s)[L::Q])
{
    using R = typename S::R;
    static_for<L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = dq_decode<S>(f[i * g.slot + c], R(L::wgt(i)));
    });
}

// Element index of f_k(x) in a state at A parity: slot opp(k) of x - c_k,
// or (wall link) slot k of x.
template <class L, int K, class R>
__device__ __forceinline__ int64_t dq_aparity_index(const Geom<R> &g, int x, int y, int z, int64_t c, bool in)
{
    if (in) return L::opp(K) * g.slot + c - ((int64_t)L::cz(K) * g.plane + (int64_t)L::cy(K) * g.nxp + L::cx(K));
    int sx, sy, sz;
    bool lid;
    if (link(g, x, y, z, -L::cx(K), -L::cy(K), -L::cz(K), sx, sy, sz, lid))
        return L::opp(K) * g.slot + cell_of(g, sx, sy, sz);
    return K * g.slot + c;
}

template <class L, class S>
__device__ __forceinline__ void dq_load_aparity(const Geom<typename S::R> &g, const typename S::T *__restrict__ f,
                                                int x, int y, int z, int64_t c, typename S::R (&s)[L::Q])
{
    using R = typename S::R;
    const bool in = interior(g, x, y, z);
    static_for<L::Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        s[k] = dq_decode<S>(f[dq_aparity_index<L, k>(g, x, y, z, c, in)], R(L::wgt(k)));
    });
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
template <class L, class S>
__global__ void k_q_init_eq(Geom<typename S::R> g, typename S::T *__restrict__ f, const void *rho, const void *u,
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
    static_for<L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        const double cu = L::cx(i) * ux + L::cy(i) * uy + L::cz(i) * uz;
        const double P = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
        const double v = S::shifted ? L::wgt(i) * ((r - 1.0) + r * P) : L::wgt(i) * r * (1.0 + P);
        f[i * g.slot + c] = S::from_r((typename S::R)v);
    });
}

// Base pointer of every direction slot of lattice QN (kernel parameters, so
// that each access is one 32-bit cell index away from a parameter).
template <class T, int QN>
struct DirsQ {
    T *p[QN];
};

// Cell-index offset of x + c_i from x (no wrap).
template <class L, int I>
inline int64_t dq_noff(int64_t plane, int64_t pitch)
{
    return (int64_t)L::cz(I) * plane + (int64_t)L::cy(I) * pitch + L::cx(I);
}

// Natural-parity loads of cell c from per-direction base pointers.
template <class L, class S>
__device__ __forceinline__ void dq_load_natural_d(const DirsQ<const typename S::T, L::Q> &f, int c,
                                                  typename S::R (&s)[L::Q])
{
    using R = typename S::R;
    static_for<L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        s[i] = dq_decode<S>(f.p[i][c], R(L::wgt(i)));
    });
}

// A-parity gather: f_k(x) from slot opp(k) of x - c_k, or (wall link) from
// slot k of x.  fin.p[k] = slot opp(k) - noff(k): the gather address of an
// interior cell, one index away.  One branch per cell: interior cells take
// a straight run of loads.
template <class L, class S>
__device__ __forceinline__ void dq_gather_aparity_d(const Geom<typename S::R> &g,
                                                    const DirsQ<const typename S::T, L::Q> &f,
                                                    const DirsQ<const typename S::T, L::Q> &fin, int x, int y, int z,
                                                    int c, typename S::R (&s)[L::Q])
{
    using R = typename S::R;
    using T = typename S::T;
    if (interior(g, x, y, z)) {
        static_for<L::Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            s[k] = dq_decode<S>(fin.p[k][c], R(L::wgt(k)));
        });
    } else if (sizeof(T) >= 4 && xedge_warp(g, x, y, z)) {
        // a warp of a row inside in y and z holding an x-edge cell: one
        // path for all its lanes, the links through an x face selecting
        // their address (the wrapped one, or slot k of x across a wall)
        const bool lo = x == 0, hi = x == g.nx - 1;
        static_for<L::Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (L::cx(k) == 0) {
                s[k] = dq_decode<S>(fin.p[k][c], R(L::wgt(k)));
            } else {
                const bool out = L::cx(k) > 0 ? lo : hi;
                const T *ad = fin.p[k] + c;
                if (g.per[0]) ad = out ? ad + (L::cx(k) > 0 ? g.nx : -g.nx) : ad;
                else ad = out ? f.p[k] + c : ad;
                s[k] = dq_decode<S>(*ad, R(L::wgt(k)));
            }
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<L::Q>([&](auto K) {
            constexpr int k = decltype(K)::value;
            constexpr unsigned m = face_mask(-L::cx(k), -L::cy(k), -L::cz(k));
            if (fc.wall & m) s[k] = dq_decode<S>(f.p[k][c], R(L::wgt(k)));
            else s[k] = dq_decode<S>(f.p[L::opp(k)][c + step_offset<-L::cx(k), -L::cy(k), -L::cz(k)>(g, fc)],
                                     R(L::wgt(k)));
        });
    }
}

// Push: f*_i to slot i of x + c_i (dout.p[i] = slot i + noff(i) for an
// interior cell), or (wall link) to slot opp(i) of x with the lid term of a
// lid face; across a periodic face the target wraps.
template <class L, class S>
__device__ __forceinline__ void dq_push_d(const Geom<typename S::R> &g, const LidQ<typename S::R, L::Q> &lq,
                                          const DirsQ<typename S::T, L::Q> &dst,
                                          const DirsQ<typename S::T, L::Q> &dout, int x, int y, int z, int c,
                                          const typename S::R (&s)[L::Q])
{
    using R = typename S::R;
    using T = typename S::T;
    if (interior(g, x, y, z)) {
        static_for<L::Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            dout.p[i][c] = dq_encode<S>(s[i], R(L::wgt(i)));
        });
    } else if (xedge_warp(g, x, y, z)) {
        // x-edge warp of a row inside in y and z: the links through an x face
        // select their target (wrapped, or slot opp(i) of x with the lid term)
        const bool lo = x == 0, hi = x == g.nx - 1;
        static_for<L::Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if constexpr (L::cx(i) == 0) {
                dout.p[i][c] = dq_encode<S>(s[i], R(L::wgt(i)));
            } else {
                const bool out = L::cx(i) > 0 ? hi : lo;
                T *ad = dout.p[i] + c;
                R v = s[i];
                if (g.per[0]) {
                    ad = out ? ad + (L::cx(i) > 0 ? -g.nx : g.nx) : ad;
                } else {
                    ad = out ? dst.p[L::opp(i)] + c : ad;
                    if (g.lid[L::cx(i) > 0 ? 1 : 0]) v = out ? radd(v, lq.L[L::opp(i)]) : v;
                }
                *ad = dq_encode<S>(v, R(L::wgt(i)));
            }
        });
    } else {
        const Faces fc = faces_of(g, x, y, z);
        static_for<L::Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr unsigned m = face_mask(L::cx(i), L::cy(i), L::cz(i));
            if (fc.wall & m) {
                R v = s[i];
                if (fc.lid & m) v = radd(v, lq.L[L::opp(i)]);
                dst.p[L::opp(i)][c] = dq_encode<S>(v, R(L::wgt(i)));
            } else {
                dst.p[i][c + step_offset<L::cx(i), L::cy(i), L::cz(i)>(g, fc)] = dq_encode<S>(s[i], R(L::wgt(i)));
            }
        });
    }
}

template <class L, class S, bool FORCE, int COLL>
__global__ void __launch_bounds__(128) k_q_two_lattice(Geom<typename S::R> g, LidQ<typename S::R, L::Q> lq,
                                                       DirsQ<const typename S::T, L::Q> src,
                                                       DirsQ<typename S::T, L::Q> dst,
                                                       DirsQ<typename S::T, L::Q> dout)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[L::Q];
    dq_load_natural_d<L, S>(src, c, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    dq_collide<L, R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    dq_push_d<L, S>(g, lq, dst, dout, x, y, z, c, s);
}

// AA even step (natural -> A parity): collide, f*_i into slot opp(i) of the
// same cell (+ L_opp(i) across a lid).
template <class L, class S, bool FORCE, int COLL>
__global__ void __launch_bounds__(128) k_q_aa_even(Geom<typename S::R> g, LidQ<typename S::R, L::Q> lq,
                                                   DirsQ<typename S::T, L::Q> f)
{
    using R = typename S::R;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[L::Q];
    dq_load_natural_d<L, S>(reinterpret_cast<const DirsQ<const T, L::Q> &>(f), c, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    dq_collide<L, R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    if (!interior(g, x, y, z)) {
        const Faces fc = faces_of(g, x, y, z);
        static_for<L::Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            constexpr unsigned m = face_mask(L::cx(i), L::cy(i), L::cz(i));
            if ((fc.wall & m) && (fc.lid & m)) s[i] = radd(s[i], lq.L[L::opp(i)]);
        });
    }
    static_for<L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        f.p[L::opp(i)][c] = dq_encode<S>(s[i], R(L::wgt(i)));
    });
}

// AA odd step (A parity -> natural), in place: gather f_k(x) from slot
// opp(k) of x - c_k (slot k of x across a wall), collide, push.  Each
// location is read and written by the same cell only.
template <class L, class S, bool FORCE, int COLL>
__global__ void __launch_bounds__(128) k_q_aa_odd(Geom<typename S::R> g, LidQ<typename S::R, L::Q> lq,
                                                  DirsQ<typename S::T, L::Q> f, DirsQ<const typename S::T, L::Q> fin,
                                                  DirsQ<typename S::T, L::Q> fout)
{
    using R = typename S::R;
    using T = typename S::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int c = cell32(g, x, y, z);
    R s[L::Q];
    dq_gather_aparity_d<L, S>(g, reinterpret_cast<const DirsQ<const T, L::Q> &>(f), fin, x, y, z, c, s);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, canon(g, x, y, z), ncanon(g), Fx, Fy, Fz);
    dq_collide<L, R, FORCE, COLL>(g, s, Fx, Fy, Fz);
    dq_push_d<L, S>(g, lq, f, fout, x, y, z, c, s);
}

// rho and u (with half the force) of the post-stream state.
template <class L, class R, bool FORCE>
__device__ __forceinline__ Mom<R> dq_moments(const R (&s)[L::Q], R Fx, R Fy, R Fz)
{
    R drho = s[0];
    static_for<L::Q - 1>([&](auto K) { drho = radd(drho, s[decltype(K)::value + 1]); });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        if constexpr (L::cx(i) == 1) jx = radd(jx, s[i]);
        if constexpr (L::cx(i) == -1) jx = rsub(jx, s[i]);
        if constexpr (L::cy(i) == 1) jy = radd(jy, s[i]);
        if constexpr (L::cy(i) == -1) jy = rsub(jy, s[i]);
        if constexpr (L::cz(i) == 1) jz = radd(jz, s[i]);
        if constexpr (L::cz(i) == -1) jz = rsub(jz, s[i]);
    });
    Mom<R> m;
    m.drho = drho;
    m.rho = radd(R(1), drho);
    const R inv = rdiv(R(1), m.rho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    m.ux = rmul(jx, inv);
    m.uy = rmul(jy, inv);
    m.uz = rmul(jz, inv);
    return m;
}

template <class L, class S, bool FORCE, bool APAR>
__global__ void k_q_moments(Geom<typename S::R> g, const typename S::T *__restrict__ f, void *rho, void *u, int dtype)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t c = cell_of(g, x, y, z);
    R s[L::Q];
    if constexpr (APAR) dq_load_aparity<L, S>(g, f, x, y, z, c, s);
    else dq_load_natural<L, S>(g, f, c, s);
    const int64_t n = ncanon(g), cc = canon(g, x, y, z);
    R Fx, Fy, Fz;
    force_at<R, FORCE>(g, cc, n, Fx, Fy, Fz);
    const Mom<R> m = dq_moments<L, R, FORCE>(s, Fx, Fy, Fz);
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

// Natural populations f_k = s_k + w_k, canonical [q][nz][ny][nx], FP32 or FP64.
template <class L, class S, bool APAR>
__global__ void k_q_export(Geom<typename S::R> g, const typename S::T *__restrict__ f, void *out, int dtype)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    const bool in = interior(g, x, y, z);
    static_for<L::Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        const int64_t e = APAR ? dq_aparity_index<L, k>(g, x, y, z, c, in) : k * g.slot + c;
        const typename S::T v = f[e];
        const R nv = S::shifted ? radd(S::to_r(v), R(L::wgt(k))) : S::to_r(v);
        if (dtype == 1) ((double *)out)[k * n + cc] = (double)nv;
        else ((float *)out)[k * n + cc] = (float)nv;
    });
}

template <class L, class S>
__global__ void k_q_import(Geom<typename S::R> g, typename S::T *__restrict__ f, const void *in, int dtype)
{
    using R = typename S::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
    if (x >= g.nx) return;
    const int64_t n = ncanon(g), cc = canon(g, x, y, z), c = cell_of(g, x, y, z);
    static_for<L::Q>([&](auto K) {
        constexpr int k = decltype(K)::value;
        if (dtype == 1) {
            const double v = ((const double *)in)[k * n + cc];
            f[k * g.slot + c] = S::from_r((R)(S::shifted ? v - L::wgt(k) : v));
        } else {
            const float v = ((const float *)in)[k * n + cc];
            f[k * g.slot + c] = S::from_r(S::shifted ? (R)rsub(v, float(L::wgt(k))) : (R)v);
        }
    });
}

// FP64 partial sums (mass, momentum, kinetic energy) per block; a
// non-finite rho or KE raises flag.  k_reduce_final adds the partials.
template <class L, class S, bool FORCE, bool APAR>
__global__ void __launch_bounds__(RED_THREADS) k_q_reduce_partial(Geom<typename S::R> g,
                                                                  const typename S::T *__restrict__ f,
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
        const int64_t c = cell_of(g, x, y, z);
        R s[L::Q];
        if constexpr (APAR) dq_load_aparity<L, S>(g, f, x, y, z, c, s);
        else dq_load_natural<L, S>(g, f, c, s);
        R dr = R(0), jx = R(0), jy = R(0), jz = R(0);
        static_for<L::Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            const R v = s[i];
            dr += v;
            if constexpr (L::cx(i) != 0) jx = L::cx(i) > 0 ? jx + v : jx - v;
            if constexpr (L::cy(i) != 0) jy = L::cy(i) > 0 ? jy + v : jy - v;
            if constexpr (L::cz(i) != 0) jz = L::cz(i) > 0 ? jz + v : jz - v;
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

// ---------------------------------------------------------------------------
// Launchers of lattice D3Q<QN> and one storage format, and their table
// (the entries of the two-step sweeps and the adjoint stay null: those are
// built for D3Q19).
// ---------------------------------------------------------------------------
template <int QN, class S>
struct LaunchQ {
    using L = DQ<QN>;
    using R = typename S::R;
    using T = typename S::T;
    static dim3 grid(const HostGeom &h) { return dim3((h.nx + 127) / 128, h.ny, h.nz); }

    // fn(FORCE, COLL) for the collisions built on these lattices
    template <class Fn>
    static void model(bool force, int coll, Fn &&fn)
    {
        auto pick = [&](auto F) {
            if (coll == COLL_TRT) fn(F, std::integral_constant<int, COLL_TRT>{});
            else if (coll == COLL_REG) fn(F, std::integral_constant<int, COLL_REG>{});
            else fn(F, std::integral_constant<int, COLL_BGK>{});
        };
        if (force) pick(std::true_type{});
        else pick(std::false_type{});
    }
    static cudaError_t init_eq(const HostGeom &h, int64_t pitch, void *f, const void *rho, const void *u, int dtype,
                               cudaStream_t st)
    {
        k_q_init_eq<L, S><<<grid(h), 128, 0, st>>>(make_geom<R>(h, pitch), (T *)f, rho, u, dtype);
        return cudaGetLastError();
    }
    // direction base pointers of a state at base: slot i, slot i + noff(i)
    // (push target of an interior cell), slot opp(i) - noff(i) (A-parity
    // gather address of an interior cell)
    template <class P>
    static DirsQ<P, QN> slots(P *base, const HostGeom &h, int64_t pitch, int shift)
    {
        DirsQ<P, QN> d;
        const int64_t plane = pitch * h.ny, slot = plane * h.nz;
        static_for<QN>([&](auto K) {
            constexpr int i = decltype(K)::value;
            if (shift == 0) d.p[i] = base + i * slot;
            else if (shift > 0) d.p[i] = base + i * slot + dq_noff<L, i>(plane, pitch);
            else d.p[i] = base + L::opp(i) * slot - dq_noff<L, i>(plane, pitch);
        });
        return d;
    }
    static cudaError_t two_lattice(const HostGeom &h, int64_t pitch, bool force, const void *src, void *dst,
                                   cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const LidQ<R, QN> lq = make_lidq<R, QN>(h);
        const DirsQ<const T, QN> a = slots((const T *)src, h, pitch, 0);
        const DirsQ<T, QN> b = slots((T *)dst, h, pitch, 0), bo = slots((T *)dst, h, pitch, 1);
        model(force, h.coll, [&](auto F, auto C) {
            k_q_two_lattice<L, S, decltype(F)::value, decltype(C)::value><<<grid(h), 128, 0, st>>>(g, lq, a, b, bo);
        });
        return cudaGetLastError();
    }
    static cudaError_t aa_even(const HostGeom &h, int64_t pitch, bool force, void *f, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const LidQ<R, QN> lq = make_lidq<R, QN>(h);
        const DirsQ<T, QN> d = slots((T *)f, h, pitch, 0);
        model(force, h.coll, [&](auto F, auto C) {
            k_q_aa_even<L, S, decltype(F)::value, decltype(C)::value><<<grid(h), 128, 0, st>>>(g, lq, d);
        });
        return cudaGetLastError();
    }
    static cudaError_t aa_odd(const HostGeom &h, int64_t pitch, bool force, void *f, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const LidQ<R, QN> lq = make_lidq<R, QN>(h);
        const DirsQ<T, QN> d = slots((T *)f, h, pitch, 0), dout = slots((T *)f, h, pitch, 1);
        const DirsQ<const T, QN> din = slots((const T *)f, h, pitch, -1);
        model(force, h.coll, [&](auto F, auto C) {
            k_q_aa_odd<L, S, decltype(F)::value, decltype(C)::value><<<grid(h), 128, 0, st>>>(g, lq, d, din, dout);
        });
        return cudaGetLastError();
    }
    static cudaError_t moments(const HostGeom &h, int64_t pitch, bool force, int parity, const void *f, void *rho,
                               void *u, int dtype, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const T *p = (const T *)f;
        if (force) {
            if (parity) k_q_moments<L, S, true, true><<<grid(h), 128, 0, st>>>(g, p, rho, u, dtype);
            else k_q_moments<L, S, true, false><<<grid(h), 128, 0, st>>>(g, p, rho, u, dtype);
        } else {
            if (parity) k_q_moments<L, S, false, true><<<grid(h), 128, 0, st>>>(g, p, rho, u, dtype);
            else k_q_moments<L, S, false, false><<<grid(h), 128, 0, st>>>(g, p, rho, u, dtype);
        }
        return cudaGetLastError();
    }
    static cudaError_t export_pop(const HostGeom &h, int64_t pitch, int parity, const void *f, void *out, int dtype,
                                  cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        if (parity) k_q_export<L, S, true><<<grid(h), 128, 0, st>>>(g, (const T *)f, out, dtype);
        else k_q_export<L, S, false><<<grid(h), 128, 0, st>>>(g, (const T *)f, out, dtype);
        return cudaGetLastError();
    }
    static cudaError_t import_pop(const HostGeom &h, int64_t pitch, void *f, const void *in, int dtype,
                                  cudaStream_t st)
    {
        k_q_import<L, S><<<grid(h), 128, 0, st>>>(make_geom<R>(h, pitch), (T *)f, in, dtype);
        return cudaGetLastError();
    }
    static cudaError_t reduce(const HostGeom &h, int64_t pitch, bool force, int parity, const void *f,
                              double *partial, int nblocks, int *flag, double *out, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const T *p = (const T *)f;
        if (force) {
            if (parity) k_q_reduce_partial<L, S, true, true><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
            else k_q_reduce_partial<L, S, true, false><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
        } else {
            if (parity) k_q_reduce_partial<L, S, false, true><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
            else k_q_reduce_partial<L, S, false, false><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, RED_THREADS, 0, st>>>(partial, nblocks, out);
        return cudaGetLastError();
    }
    static int no_ns(bool, int) { return 0; }
};

template <int QN, class S>
StorageOps make_ops_q()
{
    using LQ = LaunchQ<QN, S>;
    StorageOps o;
    memset(&o, 0, sizeof(o));
    o.elem_size = sizeof(typename S::T);
    o.real_size = sizeof(typename S::R);
    o.init_eq = &LQ::init_eq;
    o.two_lattice = &LQ::two_lattice;
    o.aa_even = &LQ::aa_even;
    o.aa_odd = &LQ::aa_odd;
    o.moments = &LQ::moments;
    o.export_pop = &LQ::export_pop;
    o.import_pop = &LQ::import_pop;
    o.reduce = &LQ::reduce;
    o.nsweep_ctas_per_sm = &LQ::no_ns;
    return o;
}

}  // namespace lbm
