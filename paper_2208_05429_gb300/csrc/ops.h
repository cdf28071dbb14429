// ops.h -- host-side interface between the C ABI (lbm_api.cu) and the
// per-storage kernel instantiations (inst_*.cu).  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbm {

// Problem description in double precision; converted to the compute type by
// each instantiation.
struct HostGeom {
    int nx, ny, nz;
    int per[3];
    int lid[6];
    double omega, kf;
    int coll;            // collision: 0 BGK, 1 TRT, 2 regularised BGK, 3 MRT
    double omega_m, kf_m;
    double mrt_s3, mrt_s4;
    int q;               // lattice: 15, 19 or 27 velocities
    double L[27];        // 6 w_k rho_w (c_k . u_lid), k < q
    double Fu[3];
    const float *Ff;
};

// Tiles of the shadow-shell merged sweep: 32 cells wide along x, bands of
// near-equal height along y; its shadow G[z][tile][q][nsp] (tile = by * ntx
// + bx) holds the stored populations of every tile-boundary cell.
struct ShellInfo {
    int ntx, nty;      // tiles along x and y
    int hb, rem;       // band heights: hb + 1 for the first rem bands, else hb
    int64_t gplane;    // elements of one z-plane of G
    int nzc;           // z chunks marched by separate CTAs (1 with periodic z)
    int mute;          // neighbour-synchronised sweep: a tile that never
                       // publishes its progress (-1: none; the self-test of
                       // the bounded waits sets it)
};

enum { PARITY_NATURAL = 0, PARITY_A = 1 };

// Launchers of one storage format.  `pitch` is the row pitch (elements) of
// the population arrays passed in; canonical arrays use pitch = nx.
struct StorageOps {
    size_t elem_size;  // bytes of a stored population
    size_t real_size;  // bytes of the compute type
    cudaError_t (*init_eq)(const HostGeom &, int64_t pitch, void *f, const void *rho, const void *u, int dtype,
                           cudaStream_t);
    cudaError_t (*two_lattice)(const HostGeom &, int64_t pitch, bool force, const void *src, void *dst,
                               cudaStream_t);
    cudaError_t (*aa_even)(const HostGeom &, int64_t pitch, bool force, void *f, cudaStream_t);
    cudaError_t (*aa_odd)(const HostGeom &, int64_t pitch, bool force, void *f, cudaStream_t);
    // the same on planes [z0, z1) only
    cudaError_t (*aa_even_range)(const HostGeom &, int64_t pitch, bool force, void *f, int z0, int z1, cudaStream_t);
    cudaError_t (*aa_odd_range)(const HostGeom &, int64_t pitch, bool force, void *f, int z0, int z1, cudaStream_t);
    cudaError_t (*moments)(const HostGeom &, int64_t pitch, bool force, int parity, const void *f, void *rho,
                           void *u, int dtype, cudaStream_t);
    cudaError_t (*export_pop)(const HostGeom &, int64_t pitch, int parity, const void *f, void *out, int dtype,
                              cudaStream_t);
    cudaError_t (*import_pop)(const HostGeom &, int64_t pitch, void *f, const void *in, int dtype, cudaStream_t);
    cudaError_t (*raw_natural)(const HostGeom &, int64_t pitch, const void *f, void *out, cudaStream_t);
    // partial: 5 * nblocks doubles; out: 5 doubles (device)
    cudaError_t (*reduce)(const HostGeom &, int64_t pitch, bool force, int parity, const void *f, double *partial,
                          int nblocks, int *flag, double *out, cudaStream_t);
    // shadow-shell merged sweep: band height limit and shell slots per tile
    // of this storage's instantiation; G* arrays hold stored elements
    int m3_ty, m3_nsp;
    int m3_zsave;  // compute-type elements per tile saved across a periodic-z march
    cudaError_t (*shell_gather)(const HostGeom &, int64_t pitch, const void *f, void *G, const ShellInfo &,
                                cudaStream_t);
    // Tensor maps (tmap, tmapz) are CUtensorMaps in host memory (64 bytes);
    // status receives a bit when a bounded wait of a sweep gave up.
    // tmap: CUtensorMap of f with a box of one direction of a 32 x m3_ty tile;
    // tmapz: the same over the chunk-boundary copy (nzc > 1, else unused);
    // zsave: m3_zsave elements per tile with periodic z (else unused)
    cudaError_t (*merged3)(const HostGeom &, int64_t pitch, bool force, void *f, const void *Gcur, void *Gnext,
                           const ShellInfo &, void *zsave, const void *tmap, const void *tmapz, int *status,
                           cudaStream_t);
    // copy of the planes zb-1 and zb of every z-chunk boundary zb into zc
    // ([19][2 (nzc-1)][ny][pitch], stored elements)
    cudaError_t (*zcopy)(const HostGeom &, int64_t pitch, const void *f, void *zc, const ShellInfo &, cudaStream_t);
    // neighbour-synchronised merged sweep (every face a wall or lid): one
    // cooperative launch of si.ntx x si.nty CTAs, all resident; prog holds
    // NS_PROG_INTS * si.ntx * si.nty ints that must be zero at launch; tmap is the
    // CUtensorMap of f with a box of ns_box_w x (ns_ty + 2) cells and all 19
    // directions.  nsweep is null where the format has no such sweep (FP64).
    cudaError_t (*nsweep)(const HostGeom &, int64_t pitch, bool force, void *f, const ShellInfo &, int *prog,
                          const void *tmap, int *status, cudaStream_t);
    int (*nsweep_ctas_per_sm)(bool force, int coll);  // coll: COLL_* of the kernel variant
    int ns_ty, ns_box_w, ns_margin;
    // lam_* are arrays of the compute type with the given pitch
    cudaError_t (*adjoint)(const HostGeom &, int64_t pitch, bool force, const void *f, const void *lam_in,
                           void *lam_out, double *gF, cudaStream_t);
    // The adjoint's checkpoint segments: mom holds the moments (rho, ux, uy,
    // uz) of one state, 4 * pitch * ny * nz compute-type elements; the
    // recompute step stores those of its input, adj_moments those of f, and
    // adjoint_mom runs the adjoint step from them instead of from f^t.
    cudaError_t (*two_lattice_mom)(const HostGeom &, int64_t pitch, bool force, const void *src, void *dst,
                                   void *mom, cudaStream_t);
    cudaError_t (*adj_moments)(const HostGeom &, int64_t pitch, bool force, const void *f, void *mom, cudaStream_t);
    cudaError_t (*adjoint_mom)(const HostGeom &, int64_t pitch, bool force, const void *mom, const void *lam_in,
                               void *lam_out, double *gF, cudaStream_t);
    cudaError_t (*adjoint_seed)(const HostGeom &, int64_t pitch, bool force, const void *f, const void *dLdrho,
                                const void *dLdu, int dtype, void *lam, double *gF, cudaStream_t);
    cudaError_t (*canon_to_pitched)(const HostGeom &, int64_t pitch, const void *in, int dtype, void *out, int ncomp,
                                    cudaStream_t);
    cudaError_t (*pitched_to_canon)(const HostGeom &, int64_t pitch, const void *in, void *out, int dtype, int ncomp,
                                    cudaStream_t);
};

const StorageOps &ops_f64();
const StorageOps &ops_f32();
const StorageOps &ops_f32s();
const StorageOps &ops_f16s();
const StorageOps &ops_bf16s();
// the D3Q15 / D3Q27 single-step kernels of one storage format (q = 15 or
// 27; null otherwise)
const StorageOps *ops_dq_f64(int q);
const StorageOps *ops_dq_f32(int q);
const StorageOps *ops_dq_f32s(int q);
const StorageOps *ops_dq_f16s(int q);
const StorageOps *ops_dq_bf16s(int q);

constexpr int RED_BLOCKS_MAX = 1024;
// ints per tile of the neighbour-synchronised sweep's progress words (one
// 128-byte line each)
constexpr int NS_PROG_INTS = 32;

}  // namespace lbm
