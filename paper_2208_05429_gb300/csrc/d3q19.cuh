// d3q19.cuh -- device-side lattice, arithmetic, storage codecs and the BGK
// collision shared by every kernel of the library.
//
// The collision (BGK with Guo forcing) is evaluated in the shifted form
// s_i = f_i - w_i: delta_rho = sum s_i, j = sum s_i c_i, and
//   feq_i - w_i = w_i (delta_rho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)),
// which keeps the O(1e-2) deviations from rest at full FP32 precision.  Every
// arithmetic step uses an explicitly rounded intrinsic (__fadd_rn, __fmaf_rn,
// ...), so the compiler can neither contract nor reorder it: all kernels that
// call bgk_collide() produce bit-identical results for the same inputs, which
// is how TWO_LATTICE, AA and MERGED are made to agree bit for bit.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace lbm {

constexpr int Q = 19;

// Collision operators (kernel template argument): BGK, two relaxation times,
// regularised BGK, multiple relaxation times in Hermite moments.
enum { COLL_BGK = 0, COLL_TRT = 1, COLL_REG = 2, COLL_MRT = 3 };

// ---------------------------------------------------------------------------
// D3Q19 velocity set.  Directions 1..9 have -1 as their first non-zero
// component (the half of the neighbours that the swap scheme streams to,
// Sec. 3 of the paper) and i+9 is the opposite of i.  Inside that rule the
// listing is grouped by c_z, which the plane-marching kernel exploits.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i)
{
    return i == 2 || i == 4 || i == 6 || i == 8 || i == 9 ? -1
         : i == 11 || i == 13 || i == 15 || i == 17 || i == 18 ? 1 : 0;
}
__host__ __device__ constexpr int cy(int i)
{
    return i == 3 || i == 5 || i == 7 || i == 8 || i == 18 ? -1
         : i == 12 || i == 14 || i == 16 || i == 17 || i == 9 ? 1 : 0;
}
__host__ __device__ constexpr int cz(int i)
{
    return i == 1 || i == 2 || i == 3 || i == 13 || i == 14 ? -1
         : i == 4 || i == 5 || i == 10 || i == 11 || i == 12 ? 1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
__host__ __device__ constexpr int csq(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
__host__ __device__ constexpr double wgt(int i)
{
    return csq(i) == 0 ? 1.0 / 3.0 : (csq(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..N-1.
template <class F, int... Is>
__host__ __device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, Is...>)
{
    (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic (no contraction, no reassociation).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }

// c_i . (ax, ay, az) as a signed sum of the non-zero components (exact for
// the unit components of D3Q19, no multiplications).
template <int I, class R>
__device__ __forceinline__ R cdot(R ax, R ay, R az)
{
    R v = R(0);
    bool first = true;
    auto acc = [&](int c, R a) {
        if (c == 0) return;
        if (first) { v = c > 0 ? a : -a; first = false; }
        else v = c > 0 ? radd(v, a) : rsub(v, a);
    };
    acc(cx(I), ax);
    acc(cy(I), ay);
    acc(cz(I), az);
    return v;
}

// ---------------------------------------------------------------------------
// Storage codecs.  T = stored element, R = compute type.  decode() returns
// the shifted value s_i = f_i - w_i in R; encode() stores it back.
// ---------------------------------------------------------------------------
struct StoreF64 {
    using T = double; using R = double;
    static constexpr bool shifted = false;
    __device__ static R to_r(T v) { return v; }
    __device__ static T from_r(R v) { return v; }
};
struct StoreF32 {
    using T = float; using R = float;
    static constexpr bool shifted = false;
    __device__ static R to_r(T v) { return v; }
    __device__ static T from_r(R v) { return v; }
};
struct StoreF32S {
    using T = float; using R = float;
    static constexpr bool shifted = true;
    __device__ static R to_r(T v) { return v; }
    __device__ static T from_r(R v) { return v; }
};
struct StoreF16S {
    using T = __half; using R = float;
    static constexpr bool shifted = true;
    __device__ static R to_r(T v) { return __half2float(v); }
    __device__ static T from_r(R v) { return __float2half_rn(v); }
};
struct StoreBF16S {
    using T = __nv_bfloat16; using R = float;
    static constexpr bool shifted = true;
    __device__ static R to_r(T v) { return __bfloat162float(v); }
    __device__ static T from_r(R v) { return __float2bfloat16_rn(v); }
};

template <class S, int I>
__device__ __forceinline__ typename S::R decode(typename S::T v)
{
    using R = typename S::R;
    if constexpr (S::shifted) return S::to_r(v);
    else return rsub(S::to_r(v), R(wgt(I)));
}
template <class S, int I>
__device__ __forceinline__ typename S::T encode(typename S::R s)
{
    using R = typename S::R;
    if constexpr (S::shifted) return S::from_r(s);
    else return S::from_r(radd(s, R(wgt(I))));
}
// The value a later decode() of encode(s) returns (storage rounding).
template <class S, int I>
__device__ __forceinline__ typename S::R roundtrip(typename S::R s)
{
    return decode<S, I>(encode<S, I>(s));
}

// ---------------------------------------------------------------------------
// Moments and collision.
// ---------------------------------------------------------------------------
template <class R>
struct Mom {
    R drho, rho, ux, uy, uz;
};

// delta_rho, rho and u = (j + F/2) / rho from shifted populations.
template <class R, bool FORCE>
__device__ __forceinline__ Mom<R> moments_of(const R (&s)[Q], R Fx, R Fy, R Fz)
{
    R drho = s[0];
    static_for<Q - 1>([&](auto K) { drho = radd(drho, s[decltype(K)::value + 1]); });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        if constexpr (cx(i) == 1) jx = radd(jx, s[i]);
        if constexpr (cx(i) == -1) jx = rsub(jx, s[i]);
        if constexpr (cy(i) == 1) jy = radd(jy, s[i]);
        if constexpr (cy(i) == -1) jy = rsub(jy, s[i]);
        if constexpr (cz(i) == 1) jz = radd(jz, s[i]);
        if constexpr (cz(i) == -1) jz = rsub(jz, s[i]);
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

__device__ __forceinline__ float rrcp(float a) { return __frcp_rn(a); }
__device__ __forceinline__ double rrcp(double a) { return __drcp_rn(a); }

// Packed two-lane FP32 arithmetic (sm_100 and later).  Each lane rounds
// exactly as the scalar round-to-nearest operation does, so a pair of
// results is bit-identical to the two scalar ones.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_dup(float a) { return make_float2(a, a); }

// c_i . (A, B, C) on duplicated pairs, in the order cdot() uses.
template <int I>
__device__ __forceinline__ float2 cdot_pair(float2 A, float2 B, float2 C)
{
    float2 v = make_float2(0.f, 0.f);
    bool first = true;
    auto acc = [&](int c, float2 a) {
        if (c == 0) return;
        if (first) { v = c > 0 ? a : p_neg(a); first = false; }
        else v = p_add(v, c > 0 ? a : p_neg(a));
    };
    acc(cx(I), A);
    acc(cy(I), B);
    acc(cz(I), C);
    return v;
}

// Sum of t[B .. E-1] as a balanced tree (compile-time bounds).
template <int B, int E>
__device__ __forceinline__ float2 pair_tree_sum(const float2 *t)
{
    if constexpr (E - B == 1) return t[B];
    else return p_add(pair_tree_sum<B, (B + E) / 2>(t), pair_tree_sum<(B + E) / 2, E>(t));
}

// Component a of c_i (i = 1..9), and the number of pairs with a non-zero one.
__host__ __device__ constexpr int ccomp(int i, int a) { return a == 0 ? cx(i) : (a == 1 ? cy(i) : cz(i)); }
template <int A>
__host__ __device__ constexpr int n_axis()
{
    int n = 0;
    for (int i = 1; i <= 9; ++i) n += ccomp(i, A) != 0;
    return n;
}
template <int A>
__host__ __device__ constexpr int axis_slot(int i)
{
    int n = 0;
    for (int k = 1; k < i; ++k) n += ccomp(k, A) != 0;
    return n;
}

// S_A = sum_i c_iA P_i over the pairs with c_iA != 0, as a balanced tree.
template <int A>
__device__ __forceinline__ float2 axis_tree_sum(const float2 (&P)[10])
{
    float2 t[n_axis<A>()];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr int c = ccomp(i, A);
        if constexpr (c != 0) t[axis_slot<A>(i)] = c > 0 ? P[i] : p_neg(P[i]);
    });
    return pair_tree_sum<0, n_axis<A>()>(t);
}

// The FP32 collision of bgk_collide() on the pairs P_i = {s_i, s_i+9} of
// opposite directions, two lanes per instruction.
//  * Moments: D = sum_i P_i gives delta_rho = (s_0 + D.x) + D.y, and
//    S_a = sum_i c_ia P_i gives j_a = S_a.x - S_a.y (c_i+9 = -c_i); both
//    sums are balanced trees, which keeps their dependency chains short.
//  * Relaxation: per pair the common part sym and the odd part +-anti of
//    the equilibrium, {a, b} = P + omega ({sym + anti, sym - anti} - P)
//    (plus the Guo source the same way), with exactly the operations, order
//    and rounding of the scalar form.
template <bool FORCE>
__device__ __forceinline__ void bgk_collide_pairs(float (&s)[Q], float omega, float kf, float Fx, float Fy, float Fz)
{
    float2 P[10];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        P[i] = make_float2(s[i], s[i + 9]);
    });
    // balanced sums (depth 4 and 3 instead of chains of 8 and 4 additions)
    const float2 D = pair_tree_sum<1, 10>(P);
    const float2 Sx = axis_tree_sum<0>(P), Sy = axis_tree_sum<1>(P), Sz = axis_tree_sum<2>(P);
    const float drho = radd(radd(s[0], D.x), D.y);
    float jx = rsub(Sx.x, Sx.y), jy = rsub(Sy.x, Sy.y), jz = rsub(Sz.x, Sz.y);
    const float rho = radd(1.f, drho);
    if constexpr (FORCE) {
        jx = rfma(0.5f, Fx, jx);
        jy = rfma(0.5f, Fy, jy);
        jz = rfma(0.5f, Fz, jz);
    }
    const float inv = rrcp(rho);
    const float ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const float ux2 = rmul(ux, ux), uy2 = rmul(uy, uy), uz2 = rmul(uz, uz);
    const float m15 = rmul(-1.5f, radd(radd(ux2, uy2), uz2));
    const float C0 = rfma(rmul(1.f / 3.f, rho), m15, rmul(1.f / 3.f, drho));
    const float A1 = rmul(1.f / 18.f, rho), A2 = rmul(1.f / 36.f, rho);
    const float C1 = rfma(A1, m15, rmul(1.f / 18.f, drho)), C2 = rfma(A2, m15, rmul(1.f / 36.f, drho));
    const float D1 = rmul(4.5f, A1), D2 = rmul(4.5f, A2);
    const float E1 = rmul(3.f, A1), E2 = rmul(3.f, A2);
    float uF = 0.f;
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    s[0] = rfma(omega, rsub(C0, s[0]), s[0]);
    if constexpr (FORCE) s[0] = rfma(kf, -uF, s[0]);
    const float2 UX = p_dup(ux), UY = p_dup(uy), UZ = p_dup(uz);
    const float2 OM = p_dup(omega);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr bool face = csq(i) == 1;
        const float2 CU = cdot_pair<i>(UX, UY, UZ);
        float2 T;
        if constexpr (face) T = p_dup(cx(i) != 0 ? ux2 : (cy(i) != 0 ? uy2 : uz2));
        else T = p_mul(CU, CU);
        const float2 SYM = p_fma(p_dup(face ? D1 : D2), T, p_dup(face ? C1 : C2));
        const float E = face ? E1 : E2;
        const float2 ANTI = p_mul(make_float2(E, -E), CU);
        const float2 V = p_add(SYM, ANTI);
        float2 R2 = p_fma(OM, p_add(V, p_neg(P[i])), P[i]);
        if constexpr (FORCE) {
            constexpr double w = wgt(i);
            const float cF = cdot<i, float>(Fx, Fy, Fz);
            const float ssym = rfma(rmul(float(9 * w), CU.x), cF, rmul(float(-3 * w), uF));
            const float santi = rmul(float(3 * w), cF);
            R2 = p_fma(p_dup(kf), p_add(p_dup(ssym), make_float2(santi, -santi)), R2);
        }
        s[i] = R2.x;
        s[i + 9] = R2.y;
    });
}

// In-place BGK + Guo collision of one cell's shifted populations s_i =
// f_i - w_i.  omega = 1/tau, kf = 1 - omega/2.
//
// Opposite directions i and i+9 (i = 1..9) share w_i and |c_i . u|, so the
// shifted equilibrium seq_i = feq_i - w_i splits into a part common to the
// pair and a part of opposite sign, seq = sym +- anti with
//   sym  = w (rho (4.5 (c.u)^2 - 1.5 u.u) + (rho - 1)),
//   anti = 3 w rho (c.u),
// and likewise the Guo source, S = w (9 (c.u)(c.F) - 3 u.F) +- 3 w c.F.
// The relaxation keeps the form s + omega (seq - s) (the non-equilibrium
// part is formed first, which keeps the rounding relative to it).  Every
// schedule collides through this function, which is what keeps them
// bit-identical to each other.
template <class R, bool FORCE>
__device__ __forceinline__ void bgk_collide(R (&s)[Q], R omega, R kf, R Fx, R Fy, R Fz)
{
    if constexpr (std::is_same<R, float>::value) {
        bgk_collide_pairs<FORCE>(s, omega, kf, Fx, Fy, Fz);
        return;
    }
    // moments from pair sums and differences
    R dif[10];
    R drho = s[0];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        drho = radd(drho, radd(s[i], s[i + 9]));
        dif[i] = rsub(s[i], s[i + 9]);
    });
    R jx = R(0), jy = R(0), jz = R(0);
    bool fx = true, fy = true, fz = true;
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        auto acc = [&](R &j, bool &first, int c) {
            if (c == 0) return;
            if (first) { j = c > 0 ? dif[i] : -dif[i]; first = false; }
            else j = c > 0 ? radd(j, dif[i]) : rsub(j, dif[i]);
        };
        acc(jx, fx, cx(i));
        acc(jy, fy, cy(i));
        acc(jz, fz, cz(i));
    });
    const R rho = radd(R(1), drho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    const R inv = rrcp(rho);
    const R ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const R ux2 = rmul(ux, ux), uy2 = rmul(uy, uy), uz2 = rmul(uz, uz);
    const R m15 = rmul(R(-1.5), radd(radd(ux2, uy2), uz2));
    // per weight class: A = w rho, C = w (rho (-1.5 u.u) + drho)
    const R C0 = rfma(rmul(R(1.0 / 3.0), rho), m15, rmul(R(1.0 / 3.0), drho));
    const R A1 = rmul(R(1.0 / 18.0), rho), A2 = rmul(R(1.0 / 36.0), rho);
    const R C1 = rfma(A1, m15, rmul(R(1.0 / 18.0), drho)), C2 = rfma(A2, m15, rmul(R(1.0 / 36.0), drho));
    const R D1 = rmul(R(4.5), A1), D2 = rmul(R(4.5), A2);
    const R E1 = rmul(R(3), A1), E2 = rmul(R(3), A2);
    R uF = R(0);
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    s[0] = rfma(omega, rsub(C0, s[0]), s[0]);
    if constexpr (FORCE) s[0] = rfma(kf, -uF, s[0]);  // w_0 S_0 = -3 w_0 u.F = -u.F
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr bool face = csq(i) == 1;
        const R cu = cdot<i, R>(ux, uy, uz);
        R t;
        if constexpr (face) t = cx(i) != 0 ? ux2 : (cy(i) != 0 ? uy2 : uz2);
        else t = rmul(cu, cu);
        const R sym = rfma(face ? D1 : D2, t, face ? C1 : C2);
        const R anti = rmul(face ? E1 : E2, cu);
        R a = rfma(omega, rsub(radd(sym, anti), s[i]), s[i]);
        R b = rfma(omega, rsub(rsub(sym, anti), s[i + 9]), s[i + 9]);
        if constexpr (FORCE) {
            constexpr double w = wgt(i);
            const R cF = cdot<i, R>(Fx, Fy, Fz);
            const R ssym = rfma(rmul(R(9 * w), cu), cF, rmul(R(-3 * w), uF));
            const R santi = rmul(R(3 * w), cF);
            a = rfma(kf, radd(ssym, santi), a);
            b = rfma(kf, rsub(ssym, santi), b);
        }
        s[i] = a;
        s[i + 9] = b;
    });
}

// Two-relaxation-time (TRT) collision of one cell's shifted populations
// s_i = f_i - w_i: for each pair of opposite directions the symmetric parts
// of s, of the equilibrium and of the Guo source relax with omega+ = 1/tau
// (kf = 1 - omega+/2), the antisymmetric parts with omega- (kfm = 1 -
// omega-/2), where (1/omega+ - 1/2)(1/omega- - 1/2) = Lambda.  In the
// notation of bgk_collide, per pair i, i+9:
//   n+ = (s_i + s_i+9)/2 - sym,  n- = (s_i - s_i+9)/2 - anti,
//   s_i   <- s_i   - omega+ n+ - omega- n- + kf ssym + kfm santi,
//   s_i+9 <- s_i+9 - omega+ n+ + omega- n- + kf ssym - kfm santi.
template <class R, bool FORCE>
__device__ __forceinline__ void trt_collide(R (&s)[Q], R omega, R kf, R om, R kfm, R Fx, R Fy, R Fz)
{
    R dif[10];
    R drho = s[0];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        drho = radd(drho, radd(s[i], s[i + 9]));
        dif[i] = rsub(s[i], s[i + 9]);
    });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        if constexpr (cx(i) != 0) jx = cx(i) > 0 ? radd(jx, dif[i]) : rsub(jx, dif[i]);
        if constexpr (cy(i) != 0) jy = cy(i) > 0 ? radd(jy, dif[i]) : rsub(jy, dif[i]);
        if constexpr (cz(i) != 0) jz = cz(i) > 0 ? radd(jz, dif[i]) : rsub(jz, dif[i]);
    });
    const R rho = radd(R(1), drho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    const R inv = rrcp(rho);
    const R ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const R m15 = rmul(R(-1.5), radd(radd(rmul(ux, ux), rmul(uy, uy)), rmul(uz, uz)));
    R uF = R(0);
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    // rest: symmetric only, seq_0 = w_0 (rho (-1.5 u.u) + drho), w_0 S_0 = -u.F
    const R C0 = rfma(rmul(R(1.0 / 3.0), rho), m15, rmul(R(1.0 / 3.0), drho));
    s[0] = rsub(s[0], rmul(omega, rsub(s[0], C0)));
    if constexpr (FORCE) s[0] = rfma(kf, -uF, s[0]);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr double w = wgt(i);
        const R cu = cdot<i, R>(ux, uy, uz);
        const R A = rmul(R(w), rho);
        const R sym = rfma(rmul(R(4.5), A), rmul(cu, cu), rfma(A, m15, rmul(R(w), drho)));
        const R anti = rmul(rmul(R(3), A), cu);
        const R np_ = rsub(rmul(R(0.5), radd(s[i], s[i + 9])), sym);
        const R nm = rsub(rmul(R(0.5), rsub(s[i], s[i + 9])), anti);
        R a = rsub(rsub(s[i], rmul(omega, np_)), rmul(om, nm));
        R b = radd(rsub(s[i + 9], rmul(omega, np_)), rmul(om, nm));
        if constexpr (FORCE) {
            const R cF = cdot<i, R>(Fx, Fy, Fz);
            const R ssym = rfma(rmul(R(9 * w), cu), cF, rmul(R(-3 * w), uF));
            const R santi = rmul(R(3 * w), cF);
            a = rfma(kfm, santi, rfma(kf, ssym, a));
            b = rfma(kfm, -santi, rfma(kf, ssym, b));
        }
        s[i] = a;
        s[i + 9] = b;
    });
}

// Regularised BGK on shifted values s_i = f_i - w_i.  The non-equilibrium
// part n_i = s_i - seq_i (seq_i = feq_i - w_i) is replaced by its projection
// on the Hermite polynomials up to second order before relaxing:
//   J = sum_i n_i c_i,  Pi = sum_i n_i c_i c_i,
//   f1_i = w_i (3 c_i . J + 4.5 (c_i . Pi . c_i - tr Pi / 3)),
//   s_i <- seq_i + (1 - omega) f1_i + kf S_i.
// J is -F/2 with a body force (zero without); dropping it would lose part of
// the Guo momentum gain.  Per pair {i, i+9}: seq and S split into the parts
// even and odd in c as in trt_collide; c.Pi.c is even, c.J odd.
template <class R, bool FORCE>
__device__ __forceinline__ void reg_collide(R (&s)[Q], R omega, R kf, R Fx, R Fy, R Fz)
{
    R dif[10];
    R drho = s[0];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        drho = radd(drho, radd(s[i], s[i + 9]));
        dif[i] = rsub(s[i], s[i + 9]);
    });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        if constexpr (cx(i) != 0) jx = cx(i) > 0 ? radd(jx, dif[i]) : rsub(jx, dif[i]);
        if constexpr (cy(i) != 0) jy = cy(i) > 0 ? radd(jy, dif[i]) : rsub(jy, dif[i]);
        if constexpr (cz(i) != 0) jz = cz(i) > 0 ? radd(jz, dif[i]) : rsub(jz, dif[i]);
    });
    const R rho = radd(R(1), drho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    const R inv = rrcp(rho);
    const R ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const R m15 = rmul(R(-1.5), radd(radd(rmul(ux, ux), rmul(uy, uy)), rmul(uz, uz)));
    R uF = R(0);
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    // pass 1: the non-equilibrium moments J and Pi (the rest population has
    // c = 0 and adds to neither)
    R Jx = R(0), Jy = R(0), Jz = R(0);
    R Pxx = R(0), Pyy = R(0), Pzz = R(0), Pxy = R(0), Pxz = R(0), Pyz = R(0);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr double w = wgt(i);
        const R cu = cdot<i, R>(ux, uy, uz);
        const R A = rmul(R(w), rho);
        const R sym = rfma(rmul(R(4.5), A), rmul(cu, cu), rfma(A, m15, rmul(R(w), drho)));
        const R anti = rmul(rmul(R(3), A), cu);
        const R ne = rsub(radd(s[i], s[i + 9]), rmul(R(2), sym));  // n_i + n_i+9
        const R no = rsub(dif[i], rmul(R(2), anti));               // n_i - n_i+9
        if constexpr (cx(i) != 0) { Jx = cx(i) > 0 ? radd(Jx, no) : rsub(Jx, no); Pxx = radd(Pxx, ne); }
        if constexpr (cy(i) != 0) { Jy = cy(i) > 0 ? radd(Jy, no) : rsub(Jy, no); Pyy = radd(Pyy, ne); }
        if constexpr (cz(i) != 0) { Jz = cz(i) > 0 ? radd(Jz, no) : rsub(Jz, no); Pzz = radd(Pzz, ne); }
        if constexpr (cx(i) * cy(i) != 0) Pxy = cx(i) * cy(i) > 0 ? radd(Pxy, ne) : rsub(Pxy, ne);
        if constexpr (cx(i) * cz(i) != 0) Pxz = cx(i) * cz(i) > 0 ? radd(Pxz, ne) : rsub(Pxz, ne);
        if constexpr (cy(i) * cz(i) != 0) Pyz = cy(i) * cz(i) > 0 ? radd(Pyz, ne) : rsub(Pyz, ne);
    });
    const R tr3 = rmul(R(1.0 / 3.0), radd(radd(Pxx, Pyy), Pzz));
    const R om1 = rsub(R(1), omega);
    // rest: seq_0 = w_0 (rho (-1.5 u.u) + drho), f1_0 = -4.5 w_0 tr/3, w_0 S_0 = -u.F
    const R C0 = rfma(rmul(R(1.0 / 3.0), rho), m15, rmul(R(1.0 / 3.0), drho));
    s[0] = rfma(om1, rmul(R(-1.5), tr3), C0);
    if constexpr (FORCE) s[0] = rfma(kf, -uF, s[0]);
    // pass 2: rebuild each pair from seq, the projected f1 and the source
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr double w = wgt(i);
        const R cu = cdot<i, R>(ux, uy, uz);
        const R A = rmul(R(w), rho);
        const R sym = rfma(rmul(R(4.5), A), rmul(cu, cu), rfma(A, m15, rmul(R(w), drho)));
        const R anti = rmul(rmul(R(3), A), cu);
        R cpc = R(0);
        if constexpr (cx(i) != 0) cpc = radd(cpc, Pxx);
        if constexpr (cy(i) != 0) cpc = radd(cpc, Pyy);
        if constexpr (cz(i) != 0) cpc = radd(cpc, Pzz);
        if constexpr (cx(i) * cy(i) != 0) cpc = cx(i) * cy(i) > 0 ? radd(cpc, rmul(R(2), Pxy)) : rsub(cpc, rmul(R(2), Pxy));
        if constexpr (cx(i) * cz(i) != 0) cpc = cx(i) * cz(i) > 0 ? radd(cpc, rmul(R(2), Pxz)) : rsub(cpc, rmul(R(2), Pxz));
        if constexpr (cy(i) * cz(i) != 0) cpc = cy(i) * cz(i) > 0 ? radd(cpc, rmul(R(2), Pyz)) : rsub(cpc, rmul(R(2), Pyz));
        const R f1s = rmul(R(4.5 * w), rsub(cpc, tr3));
        const R f1a = rmul(R(3 * w), cdot<i, R>(Jx, Jy, Jz));
        R a = rfma(om1, radd(f1s, f1a), radd(sym, anti));
        R b = rfma(om1, rsub(f1s, f1a), rsub(sym, anti));
        if constexpr (FORCE) {
            const R cF = cdot<i, R>(Fx, Fy, Fz);
            const R ssym = rfma(rmul(R(9 * w), cu), cF, rmul(R(-3 * w), uF));
            const R santi = rmul(R(3 * w), cF);
            a = rfma(kf, radd(ssym, santi), a);
            b = rfma(kf, rsub(ssym, santi), b);
        }
        s[i] = a;
        s[i + 9] = b;
    });
}

// Multiple relaxation times in Hermite moments, on shifted values.  The
// non-equilibrium part n_i = s_i - seq_i splits into orthogonal parts (in
// sum_i w_i a_i b_i) by Hermite order: f1 (orders 1 and 2, as in
// reg_collide), P3 (order 3) and P4 = n - f1 - P3 (order 4; order 0 is zero),
// relaxed with omega, s3 and s4:
//   s_i <- seq_i + (1 - omega) f1_i + (1 - s3) P3_i + (1 - s4) P4_i + kf S_i.
// On D3Q19 the third-order space is spanned by three orthogonal pairs of odd
// functions (u, v) = (a + b, a - b) of the Hermite polynomials
// a = xxy - y/3, b = yzz - y/3 and their permutations,
//   u1 = y (x^2 + z^2 - 2/3), v1 = y (x^2 - z^2),
//   u2 = z (x^2 + y^2 - 2/3), v2 = z (x^2 - y^2),
//   u3 = x (y^2 + z^2 - 2/3), v3 = x (y^2 - z^2),
// with norms sum_i w_i u^2 = 2/27 and sum_i w_i v^2 = 2/9, so that
// P3_i = w_i sum (b_u u(c_i) 27/2 + b_v v(c_i) 9/2), b_u = sum_j u(c_j) n_j.
template <int I>
__host__ __device__ constexpr double mrt_u(int k)
{
    return k == 1 ? cy(I) * (cx(I) * cx(I) + cz(I) * cz(I) - 2.0 / 3.0)
         : k == 2 ? cz(I) * (cx(I) * cx(I) + cy(I) * cy(I) - 2.0 / 3.0)
                  : cx(I) * (cy(I) * cy(I) + cz(I) * cz(I) - 2.0 / 3.0);
}
template <int I>
__host__ __device__ constexpr double mrt_v(int k)
{
    return k == 1 ? cy(I) * (cx(I) * cx(I) - cz(I) * cz(I))
         : k == 2 ? cz(I) * (cx(I) * cx(I) - cy(I) * cy(I))
                  : cx(I) * (cy(I) * cy(I) - cz(I) * cz(I));
}
template <class R, bool FORCE>
__device__ __forceinline__ void mrt_collide(R (&s)[Q], R omega, R kf, R s3, R s4, R Fx, R Fy, R Fz)
{
    R dif[10];
    R drho = s[0];
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        drho = radd(drho, radd(s[i], s[i + 9]));
        dif[i] = rsub(s[i], s[i + 9]);
    });
    R jx = R(0), jy = R(0), jz = R(0);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        if constexpr (cx(i) != 0) jx = cx(i) > 0 ? radd(jx, dif[i]) : rsub(jx, dif[i]);
        if constexpr (cy(i) != 0) jy = cy(i) > 0 ? radd(jy, dif[i]) : rsub(jy, dif[i]);
        if constexpr (cz(i) != 0) jz = cz(i) > 0 ? radd(jz, dif[i]) : rsub(jz, dif[i]);
    });
    const R rho = radd(R(1), drho);
    if constexpr (FORCE) {
        jx = rfma(R(0.5), Fx, jx);
        jy = rfma(R(0.5), Fy, jy);
        jz = rfma(R(0.5), Fz, jz);
    }
    const R inv = rrcp(rho);
    const R ux = rmul(jx, inv), uy = rmul(jy, inv), uz = rmul(jz, inv);
    const R m15 = rmul(R(-1.5), radd(radd(rmul(ux, ux), rmul(uy, uy)), rmul(uz, uz)));
    R uF = R(0);
    if constexpr (FORCE) uF = rfma(ux, Fx, rfma(uy, Fy, rmul(uz, Fz)));
    // pass 1: J, Pi (orders 1, 2) and the six third-order coefficients
    R Jx = R(0), Jy = R(0), Jz = R(0);
    R Pxx = R(0), Pyy = R(0), Pzz = R(0), Pxy = R(0), Pxz = R(0), Pyz = R(0);
    R bu1 = R(0), bu2 = R(0), bu3 = R(0), bv1 = R(0), bv2 = R(0), bv3 = R(0);
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr double w = wgt(i);
        const R cu = cdot<i, R>(ux, uy, uz);
        const R A = rmul(R(w), rho);
        const R sym = rfma(rmul(R(4.5), A), rmul(cu, cu), rfma(A, m15, rmul(R(w), drho)));
        const R anti = rmul(rmul(R(3), A), cu);
        const R ne = rsub(radd(s[i], s[i + 9]), rmul(R(2), sym));  // n_i + n_i+9
        const R no = rsub(dif[i], rmul(R(2), anti));               // n_i - n_i+9
        if constexpr (cx(i) != 0) { Jx = cx(i) > 0 ? radd(Jx, no) : rsub(Jx, no); Pxx = radd(Pxx, ne); }
        if constexpr (cy(i) != 0) { Jy = cy(i) > 0 ? radd(Jy, no) : rsub(Jy, no); Pyy = radd(Pyy, ne); }
        if constexpr (cz(i) != 0) { Jz = cz(i) > 0 ? radd(Jz, no) : rsub(Jz, no); Pzz = radd(Pzz, ne); }
        if constexpr (cx(i) * cy(i) != 0) Pxy = cx(i) * cy(i) > 0 ? radd(Pxy, ne) : rsub(Pxy, ne);
        if constexpr (cx(i) * cz(i) != 0) Pxz = cx(i) * cz(i) > 0 ? radd(Pxz, ne) : rsub(Pxz, ne);
        if constexpr (cy(i) * cz(i) != 0) Pyz = cy(i) * cz(i) > 0 ? radd(Pyz, ne) : rsub(Pyz, ne);
        if constexpr (mrt_u<i>(1) != 0.0) bu1 = rfma(R(mrt_u<i>(1)), no, bu1);
        if constexpr (mrt_u<i>(2) != 0.0) bu2 = rfma(R(mrt_u<i>(2)), no, bu2);
        if constexpr (mrt_u<i>(3) != 0.0) bu3 = rfma(R(mrt_u<i>(3)), no, bu3);
        if constexpr (mrt_v<i>(1) != 0.0) bv1 = rfma(R(mrt_v<i>(1)), no, bv1);
        if constexpr (mrt_v<i>(2) != 0.0) bv2 = rfma(R(mrt_v<i>(2)), no, bv2);
        if constexpr (mrt_v<i>(3) != 0.0) bv3 = rfma(R(mrt_v<i>(3)), no, bv3);
    });
    const R tr3 = rmul(R(1.0 / 3.0), radd(radd(Pxx, Pyy), Pzz));
    const R om1 = rsub(R(1), omega), o3 = rsub(R(1), s3), o4 = rsub(R(1), s4);
    // rest: seq_0, f1_0 = -1.5 tr/3, P3_0 = 0, P4_0 = n_0 - f1_0, w_0 S_0 = -u.F
    {
        const R C0 = rfma(rmul(R(1.0 / 3.0), rho), m15, rmul(R(1.0 / 3.0), drho));
        const R f10 = rmul(R(-1.5), tr3);
        const R n0 = rsub(s[0], C0);
        s[0] = rfma(o4, rsub(n0, f10), rfma(om1, f10, C0));
        if constexpr (FORCE) s[0] = rfma(kf, -uF, s[0]);
    }
    // pass 2: each pair from seq and the three relaxed parts
    static_for<9>([&](auto K) {
        constexpr int i = decltype(K)::value + 1;
        constexpr double w = wgt(i);
        const R cu = cdot<i, R>(ux, uy, uz);
        const R A = rmul(R(w), rho);
        const R sym = rfma(rmul(R(4.5), A), rmul(cu, cu), rfma(A, m15, rmul(R(w), drho)));
        const R anti = rmul(rmul(R(3), A), cu);
        R cpc = R(0);
        if constexpr (cx(i) != 0) cpc = radd(cpc, Pxx);
        if constexpr (cy(i) != 0) cpc = radd(cpc, Pyy);
        if constexpr (cz(i) != 0) cpc = radd(cpc, Pzz);
        if constexpr (cx(i) * cy(i) != 0) cpc = cx(i) * cy(i) > 0 ? radd(cpc, rmul(R(2), Pxy)) : rsub(cpc, rmul(R(2), Pxy));
        if constexpr (cx(i) * cz(i) != 0) cpc = cx(i) * cz(i) > 0 ? radd(cpc, rmul(R(2), Pxz)) : rsub(cpc, rmul(R(2), Pxz));
        if constexpr (cy(i) * cz(i) != 0) cpc = cy(i) * cz(i) > 0 ? radd(cpc, rmul(R(2), Pyz)) : rsub(cpc, rmul(R(2), Pyz));
        const R f1s = rmul(R(4.5 * w), rsub(cpc, tr3));
        const R f1a = rmul(R(3 * w), cdot<i, R>(Jx, Jy, Jz));
        R q = R(0);  // sum_p b_p H_p(c_i) / N_p over the third-order pairs
        if constexpr (mrt_u<i>(1) != 0.0) q = rfma(R(13.5 * mrt_u<i>(1)), bu1, q);
        if constexpr (mrt_u<i>(2) != 0.0) q = rfma(R(13.5 * mrt_u<i>(2)), bu2, q);
        if constexpr (mrt_u<i>(3) != 0.0) q = rfma(R(13.5 * mrt_u<i>(3)), bu3, q);
        if constexpr (mrt_v<i>(1) != 0.0) q = rfma(R(4.5 * mrt_v<i>(1)), bv1, q);
        if constexpr (mrt_v<i>(2) != 0.0) q = rfma(R(4.5 * mrt_v<i>(2)), bv2, q);
        if constexpr (mrt_v<i>(3) != 0.0) q = rfma(R(4.5 * mrt_v<i>(3)), bv3, q);
        const R p3 = rmul(R(w), q);
        const R na = rsub(s[i], radd(sym, anti)), nb = rsub(s[i + 9], rsub(sym, anti));
        const R f1p = radd(f1s, f1a), f1m = rsub(f1s, f1a);
        R a = rfma(o4, rsub(rsub(na, f1p), p3), rfma(o3, p3, rfma(om1, f1p, radd(sym, anti))));
        R b = rfma(o4, radd(rsub(nb, f1m), p3), rfma(o3, -p3, rfma(om1, f1m, rsub(sym, anti))));
        if constexpr (FORCE) {
            const R cF = cdot<i, R>(Fx, Fy, Fz);
            const R ssym = rfma(rmul(R(9 * w), cu), cF, rmul(R(-3 * w), uF));
            const R santi = rmul(R(3 * w), cF);
            a = rfma(kf, radd(ssym, santi), a);
            b = rfma(kf, rsub(ssym, santi), b);
        }
        s[i] = a;
        s[i + 9] = b;
    });
}

// ---------------------------------------------------------------------------
// Geometry and boundary description passed by value to every kernel.
// ---------------------------------------------------------------------------
template <class R>
struct Geom {
    int nx, ny, nz;
    int per[3];          // axis periodic?
    int lid[6];          // face is a moving lid?  (x-, x+, y-, y+, z-, z+)
    int64_t nxp;         // padded row pitch (elements)
    int64_t plane;       // nxp * ny
    int64_t slot;        // plane * nz: elements per direction
    R omega, kf;         // 1/tau, 1 - omega/2
    int coll;            // collision (COLL_*; AA and two-lattice kernels)
    R om, kfm;           // TRT: omega-, 1 - omega-/2
    R s3, s4;            // MRT: rates of the third- and fourth-order moments
    R L[Q];              // 6 w_k rho_w (c_k . u_lid): added to incoming slot k of a lid link
    R Fu[3];             // uniform force
    const float *Ff;     // per-cell force field [3][N] canonical, or nullptr
    int32_t noff[Q];     // cell-index offset of the neighbour x + c_i (no wrap)
};

// Base pointer of every direction slot, passed by value so that each access
// is one 32-bit cell index away from a kernel-parameter pointer.
template <class T>
struct Dirs {
    T *p[Q];
};

// Per-cell face information: the index correction of a step that wraps
// through a periodic face, and which faces are walls / moving lids.  Bits
// and adj[] entries are ordered x-, x+, y-, y+, z-, z+.
struct Faces {
    int32_t adj[6];
    unsigned wall, lid;
};

// Face bits crossed by a step along (dx, dy, dz) from a cell next to them.
__host__ __device__ constexpr unsigned face_mask(int dx, int dy, int dz)
{
    return (dx < 0 ? 1u : dx > 0 ? 2u : 0u) | (dy < 0 ? 4u : dy > 0 ? 8u : 0u) | (dz < 0 ? 16u : dz > 0 ? 32u : 0u);
}

// Link from (x,y,z) along d: returns true and the wrapped target cell, or
// false for a wall link (and tells whether a lid face is crossed).
template <class R>
__device__ __forceinline__ bool link(const Geom<R> &g, int x, int y, int z, int dx, int dy, int dz,
                                     int &tx, int &ty, int &tz, bool &lid)
{
    bool wall = false;
    lid = false;
    tx = x + dx; ty = y + dy; tz = z + dz;
    if (tx < 0 || tx >= g.nx) {
        if (g.per[0]) tx = tx < 0 ? tx + g.nx : tx - g.nx;
        else { wall = true; lid |= g.lid[tx < 0 ? 0 : 1] != 0; }
    }
    if (ty < 0 || ty >= g.ny) {
        if (g.per[1]) ty = ty < 0 ? ty + g.ny : ty - g.ny;
        else { wall = true; lid |= g.lid[ty < 0 ? 2 : 3] != 0; }
    }
    if (tz < 0 || tz >= g.nz) {
        if (g.per[2]) tz = tz < 0 ? tz + g.nz : tz - g.nz;
        else { wall = true; lid |= g.lid[tz < 0 ? 4 : 5] != 0; }
    }
    return !wall;
}

template <class R>
__device__ __forceinline__ int64_t cell_of(const Geom<R> &g, int x, int y, int z)
{
    return (int64_t)z * g.plane + (int64_t)y * g.nxp + x;
}

// 32-bit cell index inside one direction slot (slot sizes are below 2^31).
template <class R>
__device__ __forceinline__ int cell32(const Geom<R> &g, int x, int y, int z)
{
    return z * (int)g.plane + y * (int)g.nxp + x;
}

template <class R>
__device__ __forceinline__ Faces faces_of(const Geom<R> &g, int x, int y, int z)
{
    Faces fc;
    fc.wall = 0u;
    fc.lid = 0u;
    for (int k = 0; k < 6; ++k) fc.adj[k] = 0;
    const int n[3] = {g.nx, g.ny, g.nz};
    const int p[3] = {x, y, z};
    const int stride[3] = {1, (int)g.nxp, (int)g.plane};
    for (int a = 0; a < 3; ++a) {
        if (p[a] == 0) {
            if (g.per[a]) fc.adj[2 * a] = n[a] * stride[a];
            else { fc.wall |= 1u << (2 * a); if (g.lid[2 * a]) fc.lid |= 1u << (2 * a); }
        }
        if (p[a] == n[a] - 1) {
            if (g.per[a]) fc.adj[2 * a + 1] = -n[a] * stride[a];
            else { fc.wall |= 2u << (2 * a); if (g.lid[2 * a + 1]) fc.lid |= 2u << (2 * a); }
        }
    }
    return fc;
}

// Cell-index offset of the step (DX, DY, DZ) from a cell with faces fc
// (wrapping through periodic faces; meaningless across a wall).
template <int DX, int DY, int DZ, class R>
__device__ __forceinline__ int step_offset(const Geom<R> &g, const Faces &fc)
{
    int o = DZ * (int)g.plane + DY * (int)g.nxp + DX;
    if constexpr (DX < 0) o += fc.adj[0];
    if constexpr (DX > 0) o += fc.adj[1];
    if constexpr (DY < 0) o += fc.adj[2];
    if constexpr (DY > 0) o += fc.adj[3];
    if constexpr (DZ < 0) o += fc.adj[4];
    if constexpr (DZ > 0) o += fc.adj[5];
    return o;
}

// The periodic-wrap part of step_offset: what a step along (DX, DY, DZ) adds
// to the plain neighbour offset (0 unless it leaves through a periodic face).
template <int DX, int DY, int DZ>
__device__ __forceinline__ int wrap_adj(const Faces &fc)
{
    int o = 0;
    if constexpr (DX < 0) o += fc.adj[0];
    if constexpr (DX > 0) o += fc.adj[1];
    if constexpr (DY < 0) o += fc.adj[2];
    if constexpr (DY > 0) o += fc.adj[3];
    if constexpr (DZ < 0) o += fc.adj[4];
    if constexpr (DZ > 0) o += fc.adj[5];
    return o;
}

// True when every neighbour of (x,y,z) is an ordinary, unwrapped cell.
template <class R>
__device__ __forceinline__ bool interior(const Geom<R> &g, int x, int y, int z)
{
    return x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1;
}

// Body force of canonical cell index c.
template <class R, bool FORCE>
__device__ __forceinline__ void force_at(const Geom<R> &g, int64_t c, int64_t n, R &Fx, R &Fy, R &Fz)
{
    if constexpr (FORCE) {
        if (g.Ff) {
            Fx = R(g.Ff[c]);
            Fy = R(g.Ff[n + c]);
            Fz = R(g.Ff[2 * n + c]);
        } else {
            Fx = g.Fu[0]; Fy = g.Fu[1]; Fz = g.Fu[2];
        }
    } else {
        Fx = Fy = Fz = R(0);
    }
}

// The collision a kernel of the AA or two-lattice schedule applies: BGK, or
// TRT, regularised or MRT (a separate kernel instantiation each).
template <class R, bool FORCE, int COLL>
__device__ __forceinline__ void collide_sel(const Geom<R> &g, R (&s)[Q], R Fx, R Fy, R Fz)
{
    if constexpr (COLL == COLL_TRT) trt_collide<R, FORCE>(s, g.omega, g.kf, g.om, g.kfm, Fx, Fy, Fz);
    else if constexpr (COLL == COLL_REG) reg_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
    else if constexpr (COLL == COLL_MRT) mrt_collide<R, FORCE>(s, g.omega, g.kf, g.s3, g.s4, Fx, Fy, Fz);
    else bgk_collide<R, FORCE>(s, g.omega, g.kf, Fx, Fy, Fz);
}

}  // namespace lbm
