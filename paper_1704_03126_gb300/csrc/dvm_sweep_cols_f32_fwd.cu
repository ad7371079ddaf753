// dvm_sweep_cols_f32_fwd.cu -- FP32-storage forward instantiations of the column sweep (see dvm_sweep_cols.cuh).
#include "dvm_sweep_cols.cuh"

namespace dvm {

cudaError_t launch_sweep_cols_f32_fwd(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? cols::launch_v<float, false, true>(L, nblocks, stream)
                       : cols::launch_v<float, false, false>(L, nblocks, stream);
}

}  // namespace dvm

namespace dvm {

cudaError_t launch_sweep_cols_f32_adj(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_cols_f64_fwd(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_cols_f64_adj(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);

size_t cols_smem_bytes(bool fp64, int v, int warps) {
  const int ncol = warps * (kLanes / v);
  return cols_smem_layout(v, cols_g(fp64), ncol, fp64 ? 8 : 4).total;
}

cudaError_t launch_sweep_cols_f32(bool uniform_delta, bool adjoint, const LaunchDesc &L, int nblocks,
                                  cudaStream_t stream) {
  return adjoint ? launch_sweep_cols_f32_adj(uniform_delta, L, nblocks, stream)
                 : launch_sweep_cols_f32_fwd(uniform_delta, L, nblocks, stream);
}

cudaError_t launch_sweep_cols_f64(bool uniform_delta, bool adjoint, const LaunchDesc &L, int nblocks,
                                  cudaStream_t stream) {
  return adjoint ? launch_sweep_cols_f64_adj(uniform_delta, L, nblocks, stream)
                 : launch_sweep_cols_f64_fwd(uniform_delta, L, nblocks, stream);
}

}  // namespace dvm
