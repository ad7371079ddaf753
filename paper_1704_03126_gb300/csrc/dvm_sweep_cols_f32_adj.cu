// dvm_sweep_cols_f32_adj.cu -- FP32-storage adjoint (transposed) instantiations of the column sweep (see dvm_sweep_cols.cuh).
#include "dvm_sweep_cols.cuh"

namespace dvm {

cudaError_t launch_sweep_cols_f32_adj(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? cols::launch_v<float, true, true>(L, nblocks, stream)
                       : cols::launch_v<float, true, false>(L, nblocks, stream);
}

}  // namespace dvm
