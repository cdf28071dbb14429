// noalloc.cu -- lbm_reduce_populations(): the FP64 mass / momentum / kinetic
// energy sums of lbm_reduce() for a population field the caller holds, run
// without allocating any device memory.
//
// Who needs this.  lbm_reduce() works on a handle, and a handle owns device
// scratch for the per-block partial sums.  Some callers cannot create one:
// a process whose free device memory is all held by a caching allocator
// (PyTorch's, for instance, where cudaMalloc fails although the pool has
// room), a serving or time-stepping loop that must not take the device-wide
// synchronisation cudaMalloc and cudaFree imply, or code that runs inside an
// allocator's own callback.  This entry point keeps its scratch in one
// fixed-size array in device global memory that exists from the moment the
// library's device code is loaded on a GPU until the process exits.
//
// The kernels are the ones lbm_reduce() launches (k_reduce_partial and
// k_reduce_final, FP64 sums over a fixed summation tree), on the canonical
// layout; only where their scratch lives differs.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "lbm.h"
#include "ops.h"

using namespace lbm;

namespace {

// Layout of the scratch array (in doubles): RED_BLOCKS_MAX partial sums of
// each of the five quantities, the five results, and one word for the
// non-finite flag (an int in the first half of a double).
constexpr int NA_PARTIAL = 0;
constexpr int NA_OUT = 5 * RED_BLOCKS_MAX;
constexpr int NA_FLAG = NA_OUT + 8;
constexpr int NA_DOUBLES = NA_FLAG + 8;  // 41,088 bytes

constexpr int NA_MAX_DEVICES = 64;

}  // namespace

// The scratch itself.  In host code this name is only a host-side stand-in
// for the symbol, never a device address: the address a kernel may use is
// the one cudaGetSymbolAddress() returns for the current device.
static __device__ __align__(256) double lbm_na_scratch[NA_DOUBLES];

namespace {

std::mutex na_mutex;
double *na_addr[NA_MAX_DEVICES];  // device address of the scratch, per device

// Device address of the scratch on the current device, looked up once per
// device (the lookup also loads the library's device code there).
int scratch_of_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return LBM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_addr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, lbm_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LBM_ECUDA;
        }
        na_addr[dev] = p;
    }
    *out = na_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_populations(const lbm_config *cfg, const void *f, int32_t dtype, const float *F,
                                      double *out, void *stream)
{
    // lbm_validate() bounds the lattice at 2^31 - 1 cells; the partial sums
    // never need more than RED_BLOCKS_MAX blocks whatever the size.
    if (!cfg || !f || !out) return LBM_EINVAL;
    if (lbm_validate(cfg) != LBM_OK) return LBM_EINVAL;
    if (cfg->lattice != 0 && cfg->lattice != LBM_LATTICE_D3Q19) return LBM_EUNSUPPORTED;
    if (dtype != LBM_DTYPE_F32 && dtype != LBM_DTYPE_F64) return LBM_EINVAL;
    if (cfg->force_mode == LBM_FORCE_FIELD && !F) return LBM_EINVAL;
    double *scratch = nullptr;
    const int rc = scratch_of_current_device(&scratch);
    if (rc != LBM_OK) return rc;

    // the geometry the reduction reads: sizes and the body force
    HostGeom hg;
    memset(&hg, 0, sizeof(hg));
    hg.nx = (int)cfg->nx;
    hg.ny = (int)cfg->ny;
    hg.nz = (int)cfg->nz;
    for (int a = 0; a < 3; ++a) hg.per[a] = cfg->face_bc[2 * a] == LBM_BC_PERIODIC;
    hg.omega = 1.0 / cfg->tau;
    hg.kf = 1.0 - 0.5 * hg.omega;
    if (cfg->force_mode == LBM_FORCE_UNIFORM)
        for (int a = 0; a < 3; ++a) hg.Fu[a] = cfg->force_uniform[a];
    hg.Ff = cfg->force_mode == LBM_FORCE_FIELD ? F : nullptr;
    const bool force = cfg->force_mode != LBM_FORCE_NONE;

    const int64_t n = cfg->nx * cfg->ny * cfg->nz;
    const int64_t nb = (n + 255) / 256;
    const int nblocks = (int)(nb < RED_BLOCKS_MAX ? nb : RED_BLOCKS_MAX);
    const cudaStream_t st = (cudaStream_t)stream;
    const StorageOps &o = dtype == LBM_DTYPE_F64 ? ops_f64() : ops_f32();
    int *flag = reinterpret_cast<int *>(scratch + NA_FLAG);
    int bad = 0;
    // the flag must start at zero; the partials and results are overwritten
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return LBM_ECUDA;
    if (o.reduce(hg, cfg->nx, force, PARITY_NATURAL, f, scratch + NA_PARTIAL, nblocks, flag, scratch + NA_OUT, st) !=
        cudaSuccess)
        return LBM_ECUDA;
    if (cudaMemcpyAsync(out, scratch + NA_OUT, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return LBM_ECUDA;
    return bad ? LBM_ENONFINITE : LBM_OK;
}
