// dvm_sweep_f32.cu -- FP32-storage instantiations of the sweep kernel (see dvm_sweep.cuh).
#include "dvm_sweep.cuh"

namespace dvm {

size_t sweep_smem_bytes_f32(int warps, int cw, int ntile) { return sweep::layout<float>(warps, cw, ntile).total; }

cudaError_t launch_sweep_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? sweep::launch_cw<float, true, false>(L, nblocks, stream)
                       : sweep::launch_cw<float, false, false>(L, nblocks, stream);
}

cudaError_t launch_sweep_adjoint_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? sweep::launch_cw<float, true, true>(L, nblocks, stream)
                       : sweep::launch_cw<float, false, true>(L, nblocks, stream);
}

}  // namespace dvm
