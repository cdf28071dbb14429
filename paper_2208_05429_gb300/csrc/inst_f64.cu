// inst_f64.cu -- kernels and launchers of the F64 storage format.
#include "launch.cuh"

namespace lbm {
const StorageOps &ops_f64()
{
    static const StorageOps o = make_ops<StoreF64>();
    return o;
}
}  // namespace lbm
