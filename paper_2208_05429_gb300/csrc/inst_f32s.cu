// inst_f32s.cu -- kernels and launchers of the F32S storage format.
#include "launch.cuh"

namespace lbm {
const StorageOps &ops_f32s()
{
    static const StorageOps o = make_ops<StoreF32S>();
    return o;
}
}  // namespace lbm
