// inst_dq_f32s.cu -- D3Q15 and D3Q27 kernels and launchers of the F32S storage format.
#include "dqn.cuh"

namespace lbm {
const StorageOps *ops_dq_f32s(int q)
{
    static const StorageOps q15 = make_ops_q<15, StoreF32S>(), q27 = make_ops_q<27, StoreF32S>();
    return q == 15 ? &q15 : (q == 27 ? &q27 : nullptr);
}
}  // namespace lbm
