// dvm_kernels.h -- host-side launch wrappers of the libdvm kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "dvm_device.cuh"

namespace dvm {

// Shared-memory layout of the sweep kernel (bytes), identical on host and device: the 3-deep ring of
// R warps x CW cells x ring_stride, the record stages, the staged seam rows (FP32), the 1/denominator
// table, the moment weights and the warps' progress words.
struct SweepSmemLayout {
  size_t ring, stage, seam, inv, wts, prog, total;
};

__host__ __device__ inline SweepSmemLayout sweep_smem_layout(int R, int cw, int tsize, int recsize, int nstage,
                                                             int stage_seams, int ring_stride) {
  SweepSmemLayout L;
  size_t off = 0;
  auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  L.ring = off;
  off = align16(off + (size_t)R * 3 * cw * ring_stride * tsize);
  L.stage = off;
  off = align16(off + (size_t)R * nstage * cw * recsize);
  L.seam = off;
  if (stage_seams) off = align16(off + (size_t)2 * nstage * 2 * cw * kLanes * tsize);
  L.inv = off;
  off = align16(off + (size_t)9 * kLanes * tsize);
  L.wts = off;
  off = align16(off + (size_t)4 * ring_stride * tsize);
  L.prog = off;
  off = align16(off + (size_t)R * sizeof(int));
  L.total = off;
  return L;
}

size_t sweep_smem_bytes(bool fp64, int warps, int cw);

// One source-iteration sweep of every instance in the launch (fused moments and wall fluxes).
cudaError_t launch_sweep(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
size_t sweep_smem_bytes_f32(int warps, int cw);
size_t sweep_smem_bytes_f64(int warps, int cw);
// The transposed sweep of the adjoint iteration (launch over adjoint views of the instances).
cudaError_t launch_sweep_adjoint(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_adjoint_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_adjoint_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
// Adjoint bookkeeping: lagged seam sums, adjoint moments -> next right-hand sides, stopping test;
// records of h = 0; the gradient from the stored forward and adjoint distributions.
cudaError_t launch_adjoint_finalize(const LaunchDesc &L, int fin_blocks, int seam_blocks, bool fp64, cudaStream_t stream);
cudaError_t launch_adjoint_reset(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream);
cudaError_t launch_adjoint_gradient(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream);

// Finalize: mean-density projection, moments, residual, flow rate, next sweep records.
cudaError_t launch_finalize(const LaunchDesc &L, int nblocks, bool fp64, cudaStream_t stream);
// Reset an instance to h = 0 (records, accumulators and state; arrays are cleared by the caller).
cudaError_t launch_reset(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream);
// Arm the stopping test of an instance: tol, absolute sweep limit; clears done and status.
cudaError_t launch_arm(DeviceState *st, double tol, int max_iter_abs, cudaStream_t stream);

}  // namespace dvm
