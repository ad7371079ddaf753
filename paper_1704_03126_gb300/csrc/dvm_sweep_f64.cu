// dvm_sweep_f64.cu -- FP64 instantiations of the sweep kernel (see dvm_sweep.cuh).
#include "dvm_sweep.cuh"

namespace dvm {

size_t sweep_smem_bytes_f64(int warps, int cw, int ntile) { return sweep::layout<double>(warps, cw, ntile).total; }

cudaError_t launch_sweep_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? sweep::launch_cw<double, true, false>(L, nblocks, stream)
                       : sweep::launch_cw<double, false, false>(L, nblocks, stream);
}

cudaError_t launch_sweep_adjoint_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  return uniform_delta ? sweep::launch_cw<double, true, true>(L, nblocks, stream)
                       : sweep::launch_cw<double, false, true>(L, nblocks, stream);
}

size_t sweep_smem_bytes(bool fp64, int warps, int cw, int ntile) {
  return fp64 ? sweep_smem_bytes_f64(warps, cw, ntile) : sweep_smem_bytes_f32(warps, cw, ntile);
}

cudaError_t launch_sweep(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  if (L.cols_v > 0)
    return fp64 ? launch_sweep_cols_f64(uniform_delta, false, L, nblocks, stream)
                : launch_sweep_cols_f32(uniform_delta, false, L, nblocks, stream);
  return fp64 ? launch_sweep_f64(uniform_delta, L, nblocks, stream) : launch_sweep_f32(uniform_delta, L, nblocks, stream);
}

cudaError_t launch_sweep_adjoint(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  if (L.cols_v > 0)
    return fp64 ? launch_sweep_cols_f64(uniform_delta, true, L, nblocks, stream)
                : launch_sweep_cols_f32(uniform_delta, true, L, nblocks, stream);
  return fp64 ? launch_sweep_adjoint_f64(uniform_delta, L, nblocks, stream)
              : launch_sweep_adjoint_f32(uniform_delta, L, nblocks, stream);
}

}  // namespace dvm
