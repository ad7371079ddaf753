// dvm_kernels.h -- host-side launch wrappers of the libdvm kernels (internal).
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "dvm_device.cuh"

namespace dvm {

// Shared-memory layout of the sweep kernel (bytes), identical on host and device: the 3-deep ring of
// R warps x CW cells x ring_stride, the record stages, the staged seam rows (FP32), the 1/denominator
// table, the moment weights and the warps' progress words.  A block may sweep `ntile` velocity groups
// side by side (narrow grids): the seam stages, the 1/denominator tables and the weights are per group.
struct SweepSmemLayout {
  size_t ring, stage, seam, inv, wts, prog, total;
};
// rows of the per-group weight table: the four moment weights, then the x and y wall-flux weights
constexpr int kSweepWtsRows = 6;

__host__ __device__ inline SweepSmemLayout sweep_smem_layout(int R, int cw, int tsize, int recsize, int nstage,
                                                             int stage_seams, int ring_stride, int ntile = 1) {
  SweepSmemLayout L;
  size_t off = 0;
  auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  L.ring = off;
  off = align16(off + (size_t)R * 3 * cw * ring_stride * tsize);
  L.stage = off;
  off = align16(off + (size_t)R * nstage * cw * recsize);
  L.seam = off;
  if (stage_seams) off = align16(off + (size_t)ntile * 2 * nstage * 2 * cw * kLanes * tsize);
  L.inv = off;
  off = align16(off + (size_t)ntile * kInvRows * kLanes * tsize);  // rows 0-8: stencil classes, row 9: solid (0)
  L.wts = off;
  off = align16(off + (size_t)ntile * kSweepWtsRows * ring_stride * tsize);
  L.prog = off;
  off = align16(off + (size_t)R * sizeof(int));
  L.total = off;
  return L;
}

size_t sweep_smem_bytes(bool fp64, int warps, int cw, int ntile = 1);

// Paired FP32 row sweep (dvm_sweep_pair.cuh): a warp sweeps two velocity groups of one quadrant, lane l
// holding velocity l of each (entries 2l, 2l+1 of a 64-wide ring row).  Sweep-map entries of paired
// blocks carry kPairFlag; their group field is the first group of the first pair and the 4-bit field the
// number of pairs side by side.  Each paired block lays out its own shared memory for its R warps and
// ntile pairs: the ring (R x 3 x CW cells x kPairRS floats), one record stage per warp, the
// 1/denominator tables and weights of each pair (interleaved like the ring), the weights' tensor-core
// fragments, progress words.
constexpr int kPairFlag = 1 << 30;
constexpr int kPairRS = 68;  // 64 velocities + 16 bytes: ldmatrix rows at 272-byte stride are conflict-free
struct SweepPairSmemLayout {
  size_t ring, stage, inv, wts, bfr, prog, total;
};
__host__ __device__ inline SweepPairSmemLayout sweep_pair_smem_layout(int R, int cw, int ntile) {
  SweepPairSmemLayout L;
  size_t off = 0;
  auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  L.ring = off;
  off = align16(off + (size_t)R * 3 * cw * kPairRS * 4);
  L.stage = off;
  off = align16(off + (size_t)R * cw * 48);
  L.inv = off;
  off = align16(off + (size_t)ntile * kInvRows * 2 * kLanes * 4);
  L.wts = off;
  off = align16(off + (size_t)ntile * kSweepWtsRows * kPairRS * 4);
  L.bfr = off;  // the weights as tensor-core B fragments: [pair][k-step 0-7][lane] x 16 bytes
  off = align16(off + (size_t)ntile * 8 * kLanes * 16);
  L.prog = off;
  off = align16(off + (size_t)R * sizeof(int));
  L.total = off;
  return L;
}

// Column sweep (dvm_sweep_cols.cuh): shared-memory layout -- per-pair velocity constants, the
// 1/denominator table of the block's velocities and the 3-deep ring of column results.
constexpr int kColsMaxThreads = 512;
constexpr int kColsCstFields = 12;  // per-velocity constants of the column sweep (see dvm_sweep_cols.cuh)
struct ColsSmemLayout {
  size_t cst, inv, ring, recs, xseam, yseam, mbar, total;
};
// cell records are staged `depth` steps ahead: 5 (FP32, 48-byte records) or 4 (FP64, 64 bytes); the
// x-seam values of a row sit in a ring of kColsSeamRows rows, the y-seam values of every column are
// staged once at the start
__host__ __device__ inline int cols_depth(int tsize) { return tsize == 4 ? 5 : 4; }
constexpr int kColsSeamRows = 8;
constexpr int kColsSpinLimit = 1 << 22;  // bounded mbarrier waits of the column sweep
__host__ __device__ inline ColsSmemLayout cols_smem_layout(int V, int G, int ncol, int tsize) {
  ColsSmemLayout L;
  size_t off = 0;
  auto align16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const int VB = V * G;
  L.cst = off;
  off = align16(off + (size_t)VB * kColsCstFields * tsize);
  L.inv = off;
  off = align16(off + (size_t)kInvRows * VB * tsize);
  L.ring = off;
  off = align16(off + (size_t)3 * V * G * tsize * ncol);
  L.recs = off;
  off = align16(off + (size_t)cols_depth(tsize) * ncol * (tsize == 4 ? 48 : 64));
  L.xseam = off;
  off = align16(off + (size_t)kColsSeamRows * V * 2 * G * tsize);
  L.yseam = off;
  off = align16(off + (size_t)V * ncol * 2 * G * tsize);
  L.mbar = off;  // one mbarrier per record stage, then the block's abort flag
  off = align16(off + (size_t)cols_depth(tsize) * 8 + 16);
  L.total = off;
  return L;
}
// velocities per thread of the column sweep
inline int cols_g(bool fp64) { return fp64 ? 4 : 8; }
size_t cols_smem_bytes(bool fp64, int v, int warps);

// One source-iteration sweep of every instance in the launch (fused moments and wall fluxes).
cudaError_t launch_sweep(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
size_t sweep_smem_bytes_f32(int warps, int cw, int ntile);
size_t sweep_smem_bytes_f64(int warps, int cw, int ntile);
cudaError_t launch_sweep_cols_f32(bool uniform_delta, bool adjoint, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_cols_f64(bool uniform_delta, bool adjoint, const LaunchDesc &L, int nblocks, cudaStream_t stream);
// The transposed sweep of the adjoint iteration (launch over adjoint views of the instances).
cudaError_t launch_sweep_adjoint(bool fp64, bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_adjoint_f32(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
cudaError_t launch_sweep_adjoint_f64(bool uniform_delta, const LaunchDesc &L, int nblocks, cudaStream_t stream);
// Adjoint bookkeeping: lagged seam sums, adjoint moments -> next right-hand sides, stopping test;
// records of h = 0; the gradient from the stored forward and adjoint distributions.
cudaError_t launch_adjoint_finalize(const LaunchDesc &L, int fin_blocks, int seam_blocks, bool fp64, cudaStream_t stream);
cudaError_t launch_adjoint_reset(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream);
cudaError_t launch_adjoint_gradient(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream);

// The persistent batched launch (dvm_persist.cu): an arming kernel, then up to `sweeps` source
// iterations of every member not done, scheduled on the device (row sweep, plain iteration).
cudaError_t launch_persistent(bool fp64, bool uniform_delta, const LaunchDesc &L, const PersistDesc &P, int blocks,
                              int sweeps, cudaStream_t stream);
int persistent_blocks_per_sm(bool fp64, bool uniform_delta, const LaunchDesc &L);
// One warp polls a scheduler with no work and one active instance: result_dev receives -1 when it gave up.
cudaError_t launch_persist_selftest(const PersistDesc &P, int *result_dev, cudaStream_t stream);
// Finalize: mean-density projection, (Anderson mixing,) moments, residual, flow rate, next sweep records.
cudaError_t launch_finalize(const LaunchDesc &L, int nblocks, bool fp64, cudaStream_t stream);
// Anderson mixing between the projection and the record writer (instances with a mixing state).
cudaError_t launch_anderson(const LaunchDesc &L, bool fp64, cudaStream_t stream);
// Reset an instance to h = 0 (records, accumulators and state; arrays are cleared by the caller).
cudaError_t launch_reset(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream);
// Rebuild an instance's records (both layouts) from its stored state: moments, mass shift, pending shift
// and the last sweep's wall fluxes (the mixed-precision refinement, dvm_refine.cu).
cudaError_t launch_records(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream);
// Mixed-precision refinement (dvm_refine.cu): seam values per instance, and the four steps of a pass.
size_t refine_seam_count(const InstanceDesc &D);
cudaError_t launch_refine_snapshot(const InstanceDesc *d, const InstanceDesc &h, bool fp64, double *snap, void *snap_seam,
                                   double *snap_sc, cudaStream_t s);
cudaError_t launch_refine_load_twin(const InstanceDesc *d, const InstanceDesc *twin, const InstanceDesc &h, bool fp64,
                                    cudaStream_t s);
cudaError_t launch_refine_residual(const InstanceDesc *d, const InstanceDesc *twin, const InstanceDesc &h, bool fp64,
                                   const double *snap, const void *snap_seam, const double *snap_sc, double *rho,
                                   void *rho_seam, cudaStream_t s);
cudaError_t launch_refine_combine(const InstanceDesc *d, const InstanceDesc &h, bool fp64, const double *snap,
                                  const void *snap_seam, const double *snap_sc, const double *rho, double *sums,
                                  cudaStream_t s);
// Rebuild an instance's diagonal-major records from its row-major ones (before column-sweep launches).
cudaError_t launch_sync_diag(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream);
// Arm every instance of a launch for `count` more sweeps (device-relative; one launch).
cudaError_t launch_arm_all(const InstanceDesc *descs, int n, double tol, int count, cudaStream_t stream);
// Arm the stopping test of an instance: tol, absolute sweep limit; clears done and status.
cudaError_t launch_arm(DeviceState *st, double tol, int max_iter_abs, cudaStream_t stream);

}  // namespace dvm
