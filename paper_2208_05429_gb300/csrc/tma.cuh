// tma.cuh -- what the two merged sweeps (merged3.cuh, nsweep.cuh) share:
// inline-PTX helpers for mbarriers, TMA tensor copies and cp.async, and the
// grouping of the 19 directions by their z component, which decides how
// long a post-collision value stays in a shared-memory ring while a tile
// marches along z (the two-step merge of Sec. 4.1, Alg. 2).
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace lbm {

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the barrier did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// ---------------------------------------------- direction groups by c_z
enum { GRP_REST = 0, GRP_ZM = 1, GRP_ZP = 2, GRP_M = 3, GRP_0 = 4, GRP_P = 5 };
__host__ __device__ constexpr int grp(int i)
{
    return i == 0 ? GRP_REST
         : (cx(i) == 0 && cy(i) == 0) ? (cz(i) < 0 ? GRP_ZM : GRP_ZP)
         : cz(i) < 0 ? GRP_M : (cz(i) == 0 ? GRP_0 : GRP_P);
}
__host__ __device__ constexpr int gidx(int i)
{
    int n = 0;
    for (int j = 0; j < i; ++j)
        if (grp(j) == grp(i)) ++n;
    return n;
}
constexpr int DIR_ZM = 1, DIR_ZP = 10;  // the pure-z directions in this numbering
static_assert(grp(DIR_ZM) == GRP_ZM && grp(DIR_ZP) == GRP_ZP, "pure-z direction indices");
constexpr int NDM = 4, ND0 = 8, NDP = 4;      // xy-moving directions per z-group

}  // namespace lbm
