// dvm_sweep_cols_f64_fwd.cu -- FP64 forward instantiations of the column sweep (see dvm_sweep_cols.cuh).
#include "dvm_sweep_cols.cuh"

namespace dvm {

cudaError_t launch_sweep_cols_f64_fwd(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? cols::launch_v<double, false, true>(L, nblocks, stream)
                       : cols::launch_v<double, false, false>(L, nblocks, stream);
}

}  // namespace dvm
