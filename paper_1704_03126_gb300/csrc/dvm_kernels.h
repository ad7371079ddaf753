// dvm_kernels.h -- host-side launch wrappers of the libdvm kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "dvm_device.cuh"

namespace dvm {

// Shared-memory layout of the sweep kernel (bytes), identical on host and device.
struct SweepSmemLayout {
  size_t ring, stage, seam, inv, wts, total;
};

__host__ __device__ inline SweepSmemLayout sweep_smem_layout(int R, int C, int tsize, int recsize,
                                                             int nstage, int stage_seams) {
  SweepSmemLayout L;
  size_t off = 0;
  L.ring = off;
  off += (size_t)R * 3 * C * kRingPad * tsize;
  off = (off + 15) & ~(size_t)15;
  L.stage = off;
  off += (size_t)R * nstage * C * recsize;
  off = (off + 15) & ~(size_t)15;
  L.seam = off;
  if (stage_seams) off += (size_t)2 * nstage * 2 * C * kLanes * tsize;
  off = (off + 15) & ~(size_t)15;
  L.inv = off;
  off += (size_t)9 * kLanes * tsize;
  L.wts = off;
  off += (size_t)4 * kRingPad * tsize;
  off = (off + 15) & ~(size_t)15;
  L.total = off;
  return L;
}

// Sweep configuration of a precision: stage depth and seam staging.
inline int sweep_nstage(bool fp64) { return fp64 ? 1 : 2; }
inline int sweep_stage_seams(bool fp64) { return fp64 ? 0 : 1; }

size_t sweep_smem_bytes(bool fp64, int warps, int cmax);

// One source-iteration sweep of every instance in the launch (fused moments and wall fluxes).
cudaError_t launch_sweep(bool fp64, bool store_h, bool uniform_delta, const LaunchDesc &L, int nblocks,
                         cudaStream_t stream);
// Finalize: mean-density projection, moments, residual, flow rate, next sweep records.
cudaError_t launch_finalize(const LaunchDesc &L, int nblocks, bool fp64, cudaStream_t stream);
// Reset an instance to h = 0 (records, accumulators and state; arrays are cleared by the caller).
cudaError_t launch_reset(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream);
// Arm the stopping test of an instance: tol, absolute sweep limit; clears done and status.
cudaError_t launch_arm(DeviceState *st, double tol, int max_iter_abs, cudaStream_t stream);

}  // namespace dvm
