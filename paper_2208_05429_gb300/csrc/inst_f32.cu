// inst_f32.cu -- kernels and launchers of the F32 storage format.
#include "launch.cuh"

namespace lbm {
const StorageOps &ops_f32()
{
    static const StorageOps o = make_ops<StoreF32>();
    return o;
}
}  // namespace lbm
