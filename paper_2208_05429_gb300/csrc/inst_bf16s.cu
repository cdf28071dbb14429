// inst_bf16s.cu -- kernels and launchers of the BF16S storage format.
#include "launch.cuh"

namespace lbm {
const StorageOps &ops_bf16s()
{
    static const StorageOps o = make_ops<StoreBF16S>();
    return o;
}
}  // namespace lbm
