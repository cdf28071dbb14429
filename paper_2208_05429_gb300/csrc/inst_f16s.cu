// inst_f16s.cu -- kernels and launchers of the F16S storage format.
#include "launch.cuh"

namespace lbm {
const StorageOps &ops_f16s()
{
    static const StorageOps o = make_ops<StoreF16S>();
    return o;
}
}  // namespace lbm
