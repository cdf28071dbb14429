// inst_ks.cu -- the K-step sweep (ksweep.cuh) for the FP32-compute storage formats.
#include "ksweep.cuh"
#include "ksweep_api.h"
#include "lbm.h"

namespace lbm {
cudaError_t ksweep_launch(int storage, const HostGeom &h, int64_t pitch, bool force, int K, const void *src,
                          void *dst, cudaStream_t st)
{
    switch (storage) {
    case LBM_STORAGE_F32: return launch_ksweep<StoreF32>(h, pitch, force, K, src, dst, st);
    case LBM_STORAGE_F32S: return launch_ksweep<StoreF32S>(h, pitch, force, K, src, dst, st);
    case LBM_STORAGE_F16S: return launch_ksweep<StoreF16S>(h, pitch, force, K, src, dst, st);
    case LBM_STORAGE_BF16S: return launch_ksweep<StoreBF16S>(h, pitch, force, K, src, dst, st);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace lbm
