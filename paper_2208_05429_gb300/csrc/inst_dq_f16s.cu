// inst_dq_f16s.cu -- D3Q15 and D3Q27 kernels and launchers of the F16S storage format.
#include "dqn.cuh"

namespace lbm {
const StorageOps *ops_dq_f16s(int q)
{
    static const StorageOps q15 = make_ops_q<15, StoreF16S>(), q27 = make_ops_q<27, StoreF16S>();
    return q == 15 ? &q15 : (q == 27 ? &q27 : nullptr);
}
}  // namespace lbm
