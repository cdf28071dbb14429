// ksweep_api.h -- the launcher of the K-step sweep (ksweep.cuh, inst_ks.cu)
// as the C ABI calls it.  Internal to the library.
#pragma once

#include "ops.h"

namespace lbm {

// K time steps per sweep (K = 3 or 4) from src to dst, both natural parity,
// D3Q19 BGK; storage LBM_STORAGE_F32, _F32S, _F16S or _BF16S (else
// cudaErrorInvalidValue).
cudaError_t ksweep_launch(int storage, const HostGeom &h, int64_t pitch, bool force, int K, const void *src,
                          void *dst, cudaStream_t st);

}  // namespace lbm
