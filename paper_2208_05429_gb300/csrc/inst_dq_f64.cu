// inst_dq_f64.cu -- D3Q15 and D3Q27 kernels and launchers of the F64 storage format.
#include "dqn.cuh"

namespace lbm {
const StorageOps *ops_dq_f64(int q)
{
    static const StorageOps q15 = make_ops_q<15, StoreF64>(), q27 = make_ops_q<27, StoreF64>();
    return q == 15 ? &q15 : (q == 27 ? &q27 : nullptr);
}
}  // namespace lbm
