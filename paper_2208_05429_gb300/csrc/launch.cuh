// launch.cuh -- host launchers of one storage format, gathered into a
// StorageOps table by make_ops<S>().  Included once per inst_*.cu.
#pragma once

#include "kernels.cuh"
#include "merged3.cuh"
#include "nsweep.cuh"

#include <string.h>

#include <type_traits>

namespace lbm {

constexpr int CELL_BLOCK = 128;

inline dim3 cell_grid(const HostGeom &h) { return dim3((h.nx + CELL_BLOCK - 1) / CELL_BLOCK, h.ny, h.nz); }

// fn(FORCE, COLL) with the runtime force flag and collision operator as
// compile-time constants (std::integral_constant).
template <class Fn>
inline void with_model(bool force, int coll, Fn &&fn)
{
    auto pick = [&](auto F) {
        if (coll == COLL_TRT) fn(F, std::integral_constant<int, COLL_TRT>{});
        else if (coll == COLL_REG) fn(F, std::integral_constant<int, COLL_REG>{});
        else if (coll == COLL_MRT) fn(F, std::integral_constant<int, COLL_MRT>{});
        else fn(F, std::integral_constant<int, COLL_BGK>{});
    };
    if (force) pick(std::true_type{});
    else pick(std::false_type{});
}

template <class S>
struct Launch {
    using R = typename S::R;
    using T = typename S::T;

    static cudaError_t init_eq(const HostGeom &h, int64_t pitch, void *f, const void *rho, const void *u, int dtype,
                               cudaStream_t st)
    {
        k_init_eq<S><<<cell_grid(h), CELL_BLOCK, 0, st>>>(make_geom<R>(h, pitch), (T *)f, rho, u, dtype);
        return cudaGetLastError();
    }
    static int64_t slot_of(const HostGeom &h, int64_t pitch) { return pitch * h.ny * h.nz; }
    static cudaError_t two_lattice(const HostGeom &h, int64_t pitch, bool force, const void *src, void *dst,
                                   cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<const T> a = make_dirs((const T *)src, slot_of(h, pitch));
        const Dirs<T> b = make_dirs((T *)dst, slot_of(h, pitch));
        Dirs<T> bo;  // push addresses of an interior cell, one index away
        for (int i = 0; i < Q; ++i) bo.p[i] = b.p[i] + g.noff[i];
        with_model(force, h.coll, [&](auto F, auto C) {
            k_two_lattice<S, decltype(F)::value, decltype(C)::value>
                <<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, a, b, bo, nullptr);
        });
        return cudaGetLastError();
    }
    // the same (BGK), also storing the moments of src in mom (adjoint recompute)
    static cudaError_t two_lattice_mom(const HostGeom &h, int64_t pitch, bool force, const void *src, void *dst,
                                       void *mom, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<const T> a = make_dirs((const T *)src, slot_of(h, pitch));
        const Dirs<T> b = make_dirs((T *)dst, slot_of(h, pitch));
        Dirs<T> bo;
        for (int i = 0; i < Q; ++i) bo.p[i] = b.p[i] + g.noff[i];
        if (force) k_two_lattice<S, true, COLL_BGK, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, a, b, bo, (R *)mom);
        else k_two_lattice<S, false, COLL_BGK, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, a, b, bo, (R *)mom);
        return cudaGetLastError();
    }
    static cudaError_t adj_moments(const HostGeom &h, int64_t pitch, bool force, const void *f, void *mom,
                                   cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<const T> a = make_dirs((const T *)f, slot_of(h, pitch));
        if (force) k_adj_moments<S, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, a, (R *)mom);
        else k_adj_moments<S, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, a, (R *)mom);
        return cudaGetLastError();
    }
    // planes [z0, z1) only
    static cudaError_t aa_even_range(const HostGeom &h, int64_t pitch, bool force, void *f, int z0, int z1,
                                     cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<T> d = make_dirs((T *)f, slot_of(h, pitch));
        if constexpr (sizeof(T) == 2) {  // two cells per thread (packed 4-byte accesses)
            const dim3 grid((h.nx + 2 * CELL_BLOCK - 1) / (2 * CELL_BLOCK), h.ny, z1 - z0);
            with_model(force, h.coll, [&](auto F, auto C) {
                k_aa_even_pair<S, decltype(F)::value, decltype(C)::value><<<grid, CELL_BLOCK, 0, st>>>(g, d, z0);
            });
        } else {
            const dim3 grid((h.nx + CELL_BLOCK - 1) / CELL_BLOCK, h.ny, z1 - z0);
            with_model(force, h.coll, [&](auto F, auto C) {
                k_aa_even<S, decltype(F)::value, decltype(C)::value><<<grid, CELL_BLOCK, 0, st>>>(g, d, z0);
            });
        }
        return cudaGetLastError();
    }
    static cudaError_t aa_odd_range(const HostGeom &h, int64_t pitch, bool force, void *f, int z0, int z1,
                                    cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<T> d = make_dirs((T *)f, slot_of(h, pitch));
        Dirs<T> din, dout;
        for (int i = 0; i < Q; ++i) {
            din.p[i] = d.p[opp(i)] - g.noff[i];
            dout.p[i] = d.p[i] + g.noff[i];
        }
        const dim3 grid((h.nx + CELL_BLOCK - 1) / CELL_BLOCK, h.ny, z1 - z0);
        with_model(force, h.coll, [&](auto F, auto C) {
            k_aa_odd<S, decltype(F)::value, decltype(C)::value><<<grid, CELL_BLOCK, 0, st>>>(g, d, din, dout, z0);
        });
        return cudaGetLastError();
    }
    static cudaError_t aa_even(const HostGeom &h, int64_t pitch, bool force, void *f, cudaStream_t st)
    {
        return aa_even_range(h, pitch, force, f, 0, h.nz, st);
    }
    static cudaError_t aa_odd(const HostGeom &h, int64_t pitch, bool force, void *f, cudaStream_t st)
    {
        return aa_odd_range(h, pitch, force, f, 0, h.nz, st);
    }
    static cudaError_t moments(const HostGeom &h, int64_t pitch, bool force, int parity, const void *f, void *rho,
                               void *u, int dtype, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const T *p = (const T *)f;
        if (force) {
            if (parity) k_moments<S, true, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, p, rho, u, dtype);
            else k_moments<S, true, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, p, rho, u, dtype);
        } else {
            if (parity) k_moments<S, false, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, p, rho, u, dtype);
            else k_moments<S, false, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, p, rho, u, dtype);
        }
        return cudaGetLastError();
    }
    static cudaError_t export_pop(const HostGeom &h, int64_t pitch, int parity, const void *f, void *out, int dtype,
                                  cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        if (parity) k_export<S, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, (const T *)f, out, dtype);
        else k_export<S, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, (const T *)f, out, dtype);
        return cudaGetLastError();
    }
    static cudaError_t import_pop(const HostGeom &h, int64_t pitch, void *f, const void *in, int dtype,
                                  cudaStream_t st)
    {
        k_import<S><<<cell_grid(h), CELL_BLOCK, 0, st>>>(make_geom<R>(h, pitch), (T *)f, in, dtype);
        return cudaGetLastError();
    }
    static cudaError_t raw_natural(const HostGeom &h, int64_t pitch, const void *f, void *out, cudaStream_t st)
    {
        k_raw_natural<S><<<cell_grid(h), CELL_BLOCK, 0, st>>>(make_geom<R>(h, pitch), (const T *)f, (T *)out);
        return cudaGetLastError();
    }
    static cudaError_t reduce(const HostGeom &h, int64_t pitch, bool force, int parity, const void *f,
                              double *partial, int nblocks, int *flag, double *out, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const T *p = (const T *)f;
        if (force) {
            if (parity) k_reduce_partial<S, true, true><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
            else k_reduce_partial<S, true, false><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
        } else {
            if (parity) k_reduce_partial<S, false, true><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
            else k_reduce_partial<S, false, false><<<nblocks, RED_THREADS, 0, st>>>(g, p, partial, flag);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, RED_THREADS, 0, st>>>(partial, nblocks, out);
        return cudaGetLastError();
    }
    // band height of the shadow-shell sweep: 32 x 14 tiles (one per SM on a
    // 256^2 plane) for 4-byte and 2-byte storage, 32 x 4 for FP64 (shared
    // memory)
    static constexpr int M3_TY = sizeof(R) == 8 ? 4 : 14;
    using M3L = M3Smem<M3_TY, T, R>;
    static_assert(M3L::bytes <= 232448, "shadow-shell sweep shared memory");
    static cudaError_t shell_gather(const HostGeom &h, int64_t pitch, const void *f, void *G, const ShellInfo &si,
                                    cudaStream_t st)
    {
        const int64_t tot = (int64_t)si.ntx * si.nty * M3<M3_TY>::NSP * h.nz;
        const unsigned blocks = (unsigned)((tot + 255) / 256);
        k_shell_gather<S, M3_TY><<<blocks, 256, 0, st>>>(make_geom<R>(h, pitch),
                                                         make_dirs((const T *)f, slot_of(h, pitch)), (T *)G, si);
        return cudaGetLastError();
    }
    template <bool F, bool PZ, bool CH>
    static cudaError_t merged3_f(const HostGeom &h, int64_t pitch, void *f, const void *Gc, void *Gn,
                                 const ShellInfo &si, void *zsave, const void *tmap, const void *tmapz, int *status,
                                 cudaStream_t st)
    {
        constexpr size_t smem = M3L::bytes;
        static bool attr_set = false;  // once per process: not inside a stream capture
        if (!attr_set) {
            const cudaError_t e = cudaFuncSetAttribute(k_merged3<S, F, M3_TY, PZ, CH>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            attr_set = true;
        }
        CUtensorMap map, mapz;
        memcpy(&map, tmap, sizeof(map));
        memcpy(&mapz, si.nzc > 1 ? tmapz : tmap, sizeof(mapz));
        const Geom<R> g = make_geom<R>(h, pitch);
        const Dirs<T> fd = make_dirs((T *)f, slot_of(h, pitch));
        Dirs<T> fo = fd, go;
        for (int i = 0; i < Q; ++i) {
            fo.p[i] = fd.p[i] + g.noff[i];
            go.p[i] = (T *)Gn + cz(i) * si.gplane + (int64_t)i * M3<M3_TY>::NSP;
        }
        k_merged3<S, F, M3_TY, PZ, CH><<<dim3(si.ntx, si.nty, CH ? si.nzc : 1), M3<M3_TY>::THREADS, smem, st>>>(
            map, mapz, g, fd, fo, go, (const T *)Gc, (T *)Gn, si, (R *)zsave, status);
        return cudaGetLastError();
    }
    static cudaError_t merged3(const HostGeom &h, int64_t pitch, bool force, void *f, const void *Gc, void *Gn,
                               const ShellInfo &si, void *zsave, const void *tmap, const void *tmapz, int *status,
                               cudaStream_t st)
    {
        if (h.per[2])
            return force ? merged3_f<true, true, false>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st)
                         : merged3_f<false, true, false>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st);
        if (si.nzc > 1)
            return force ? merged3_f<true, false, true>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st)
                         : merged3_f<false, false, true>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st);
        return force ? merged3_f<true, false, false>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st)
                     : merged3_f<false, false, false>(h, pitch, f, Gc, Gn, si, zsave, tmap, tmapz, status, st);
    }
    static cudaError_t zcopy(const HostGeom &h, int64_t pitch, const void *f, void *zc, const ShellInfo &si,
                             cudaStream_t st)
    {
        if (si.nzc < 2) return cudaSuccess;
        const int64_t total = (int64_t)Q * 2 * (si.nzc - 1) * h.ny * pitch;
        const int64_t nb = (total + 255) / 256;
        k_zcopy<S><<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(make_geom<R>(h, pitch), (const T *)f, (T *)zc,
                                                                      si.nzc);
        return cudaGetLastError();
    }
    // neighbour-synchronised merged sweep: 4- and 2-byte storage, 32 x 14 tiles
    static constexpr int NS_TY = 14;
    static constexpr bool HAS_NS = sizeof(T) < 8;
    template <bool F, int C>
    static cudaError_t nsweep_f(const HostGeom &h, int64_t pitch, void *f, const ShellInfo &si, int *prog,
                                const void *tmap, int *status, cudaStream_t st)
    {
        if constexpr (!HAS_NS) {
            return cudaErrorNotSupported;
        } else {
            using NSM = NSSmem<NS_TY, T, R>;
            static_assert(NSM::bytes <= 232448, "neighbour-synchronised sweep shared memory");
            constexpr size_t smem = NSM::bytes;
            static bool attr_set = false;  // once per process: not inside a stream capture
            if (!attr_set) {
                const cudaError_t e = cudaFuncSetAttribute(k_nsweep<S, F, NS_TY, C>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                attr_set = true;
            }
            CUtensorMap map;
            memcpy(&map, tmap, sizeof(map));
            const Geom<R> g = make_geom<R>(h, pitch);
            const Dirs<T> fd = make_dirs((T *)f, slot_of(h, pitch));
            Dirs<T> fo = fd;
            for (int i = 0; i < Q; ++i) fo.p[i] = fd.p[i] + g.noff[i];
            cudaLaunchConfig_t cfg;
            memset(&cfg, 0, sizeof(cfg));
            cfg.gridDim = dim3(si.ntx, si.nty, 1);
            cfg.blockDim = dim3(NSL<NS_TY, T>::THREADS, 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeCooperative;
            attr[0].val.cooperative = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            return cudaLaunchKernelEx(&cfg, k_nsweep<S, F, NS_TY, C>, map, g, fd, fo, si, prog, status);
        }
    }
    static cudaError_t nsweep(const HostGeom &h, int64_t pitch, bool force, void *f, const ShellInfo &si, int *prog,
                              const void *tmap, int *status, cudaStream_t st)
    {
        cudaError_t e = cudaSuccess;
        with_model(force, h.coll, [&](auto F, auto C) {
            e = nsweep_f<decltype(F)::value, decltype(C)::value>(h, pitch, f, si, prog, tmap, status, st);
        });
        return e;
    }
    // CTAs of the sweep one SM holds (0 where it does not exist or fit)
    static int nsweep_ctas_per_sm(bool force, int coll)
    {
        if constexpr (!HAS_NS) {
            return 0;
        } else {
            constexpr size_t smem = NSSmem<NS_TY, T, R>::bytes;
            decltype(&k_nsweep<S, false, NS_TY, COLL_BGK>) kern = nullptr;
            with_model(force, coll, [&](auto F, auto C) { kern = k_nsweep<S, decltype(F)::value, NS_TY, decltype(C)::value>; });
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, NSL<NS_TY, T>::THREADS, smem) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            return n;
        }
    }
    static cudaError_t adjoint(const HostGeom &h, int64_t pitch, bool force, const void *f, const void *lam_in,
                               void *lam_out, double *gF, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const int64_t sl = slot_of(h, pitch);
        const Dirs<const T> fd = make_dirs((const T *)f, sl);
        const Dirs<R> lout = make_dirs((R *)lam_out, sl);
        Dirs<const R> lin;  // interior gather addresses, one index away
        for (int i = 0; i < Q; ++i) lin.p[i] = (const R *)lam_in + i * sl + g.noff[i];
        if (force) k_adjoint<S, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, fd, lin, lout, gF, nullptr);
        else k_adjoint<S, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, fd, lin, lout, gF, nullptr);
        return cudaGetLastError();
    }
    // the same with the moments of f^t read from mom (adj_moments layout)
    static cudaError_t adjoint_mom(const HostGeom &h, int64_t pitch, bool force, const void *mom,
                                   const void *lam_in, void *lam_out, double *gF, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        const int64_t sl = slot_of(h, pitch);
        const Dirs<const T> fd{};
        const Dirs<R> lout = make_dirs((R *)lam_out, sl);
        Dirs<const R> lin;
        for (int i = 0; i < Q; ++i) lin.p[i] = (const R *)lam_in + i * sl + g.noff[i];
        if (force) k_adjoint<S, true, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, fd, lin, lout, gF, (const R *)mom);
        else k_adjoint<S, false, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, fd, lin, lout, gF, (const R *)mom);
        return cudaGetLastError();
    }
    static cudaError_t adjoint_seed(const HostGeom &h, int64_t pitch, bool force, const void *f, const void *dLdrho,
                                    const void *dLdu, int dtype, void *lam, double *gF, cudaStream_t st)
    {
        const Geom<R> g = make_geom<R>(h, pitch);
        if (force) k_adjoint_seed<S, true><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, (const T *)f, dLdrho, dLdu, dtype, (R *)lam, gF);
        else k_adjoint_seed<S, false><<<cell_grid(h), CELL_BLOCK, 0, st>>>(g, (const T *)f, dLdrho, dLdu, dtype, (R *)lam, gF);
        return cudaGetLastError();
    }
    static cudaError_t canon_to_pitched(const HostGeom &h, int64_t pitch, const void *in, int dtype, void *out,
                                        int ncomp, cudaStream_t st)
    {
        k_canon_to_pitched<R><<<cell_grid(h), CELL_BLOCK, 0, st>>>(make_geom<R>(h, pitch), in, dtype, (R *)out, ncomp);
        return cudaGetLastError();
    }
    static cudaError_t pitched_to_canon(const HostGeom &h, int64_t pitch, const void *in, void *out, int dtype,
                                        int ncomp, cudaStream_t st)
    {
        k_pitched_to_canon<R><<<cell_grid(h), CELL_BLOCK, 0, st>>>(make_geom<R>(h, pitch), (const R *)in, out, dtype, ncomp);
        return cudaGetLastError();
    }
};

template <class S>
StorageOps make_ops()
{
    using L = Launch<S>;
    StorageOps o;
    o.elem_size = sizeof(typename S::T);
    o.real_size = sizeof(typename S::R);
    o.nsweep = L::HAS_NS ? &L::nsweep : nullptr;
    o.nsweep_ctas_per_sm = &L::nsweep_ctas_per_sm;
    o.ns_ty = L::NS_TY;
    o.ns_box_w = 32 + 2 * (16 / (int)sizeof(typename S::T));
    o.ns_margin = 16 / (int)sizeof(typename S::T);
    o.init_eq = &L::init_eq;
    o.two_lattice = &L::two_lattice;
    o.aa_even = &L::aa_even;
    o.aa_odd = &L::aa_odd;
    o.aa_even_range = &L::aa_even_range;
    o.aa_odd_range = &L::aa_odd_range;
    o.moments = &L::moments;
    o.export_pop = &L::export_pop;
    o.import_pop = &L::import_pop;
    o.raw_natural = &L::raw_natural;
    o.reduce = &L::reduce;
    o.m3_ty = L::M3_TY;
    o.m3_nsp = M3<L::M3_TY>::NSP;
    o.m3_zsave = M3<L::M3_TY>::ZSAVE;
    o.shell_gather = &L::shell_gather;
    o.merged3 = &L::merged3;
    o.zcopy = &L::zcopy;
    o.adjoint = &L::adjoint;
    o.adjoint_mom = &L::adjoint_mom;
    o.two_lattice_mom = &L::two_lattice_mom;
    o.adj_moments = &L::adj_moments;
    o.adjoint_seed = &L::adjoint_seed;
    o.canon_to_pitched = &L::canon_to_pitched;
    o.pitched_to_canon = &L::pitched_to_canon;
    return o;
}

}  // namespace lbm
