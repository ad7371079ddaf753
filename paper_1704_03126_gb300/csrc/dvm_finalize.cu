// dvm_finalize.cu -- per-iteration reductions after the sweep (FP64 throughout).
//
// fin1: the mean gas density of the swept state gives the mass shift s = sum_gas rho / (n_gas sum W)
//       that projects the null mode h = const out of the iteration (the constant solves the
//       homogeneous problem: the sweep reproduces constants exactly and the walls conserve mass).
// fin2: shifted moments rho, u1, u2, tau (Sec. II.A), the collision coefficients a = G^{-1} m of the
//       W-orthogonal projection onto (1, v1, v2, |v|^2), the accumulated bordering unknown c += s, the
//       stopping quantities eps_n = sum|u1^n - u1^{n-1}| / sum|u1^n| and the flow rate
//       Q = sum u1 dA / Lx (Sec. III), the diffuse wall values rho_w = incident flux / outgoing
//       normaliser (Eq. diffuse2), and the sweep records of the next iteration.  The last block of
//       each instance applies the stopping test and sets the instance's done flag.
#include <cmath>
#include <cstdint>

#include "dvm_device.cuh"
#include "dvm_finalize.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace {

constexpr int kFinBlock = 256;

// Block sums of N doubles per thread, valid in thread 0.  The values go to shared memory and one warp
// adds them: this part's FP64 pipe is narrow (2 lanes per SM and cycle), so the block does about one
// FP64 add per value instead of the five of a shuffle tree run by every warp.
template <int N>
__device__ __forceinline__ void block_sums(double (&v)[N], double (*sh)[kFinBlock]) {
#pragma unroll
  for (int k = 0; k < N; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double r = sh[k][threadIdx.x];
#pragma unroll
      for (int i = 32; i < kFinBlock; i += 32) r += sh[k][threadIdx.x + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      v[k] = r;
    }
  }
}

__global__ void __launch_bounds__(kFinBlock) fin1_kernel(LaunchDesc L) {
  __shared__ double sh[1][kFinBlock];
  const int map = L.fin_map[blockIdx.x];
  const InstanceDesc *D = L.inst + (map >> 16);
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int cell = (map & 0xffff) * kFinBlock + threadIdx.x;
  double v[1] = {0.0};
  if (cell < D->ncell && !(D->code4[(size_t)cell * 4] & kSolid)) v[0] = D->acc[(size_t)cell * 4];
  block_sums<1>(v, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->mass_acc, v[0]);
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket1, 1u);
    if (t == (unsigned)D->fin_nblocks - 1u) {
      __threadfence();
      const double mass = atomicAdd(&st->mass_acc, 0.0);
      st->s_new = mass / ((double)D->n_gas * D->sumW[0]);
      st->mass_acc = 0.0;
      st->ticket1 = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kFinBlock) fin2_kernel(LaunchDesc L) {
  __shared__ double sh[3][kFinBlock];
  const int map = L.fin_map[blockIdx.x];
  const InstanceDesc *D = L.inst + (map >> 16);
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int ncell = D->ncell;
  const int cell = (map & 0xffff) * kFinBlock + threadIdx.x;
  const double s = st->s_new;
  // correction phase of the refinement: the fixed residual rho is added after the projection
  const double *rho_in = D->rho;
  const double c_new = st->c + s + (rho_in ? rho_in[(size_t)8 * ncell] : 0.0);
  const int parity = (st->iter + 1) & 1;
  const double *fcur = D->facc + (size_t)parity * ncell * 4;
  double *fnext = D->facc + (size_t)(parity ^ 1) * ncell * 4;
  double du = 0.0, ua = 0.0, uq = 0.0, bad = 0.0;
  if (cell < ncell) fin2_cell<T>(D, cell, s, c_new, fcur, fnext, rho_in, L.cols_v != 0, du, ua, uq, bad);
  if (rho_in) seam_inject<T>(D, (size_t)(map & 0xffff) * kFinBlock + threadIdx.x, (size_t)D->fin_nblocks * kFinBlock);
  double sums[3] = {du, ua, uq};
  const bool any_bad = __syncthreads_or(bad > 0.0) != 0;
  block_sums<3>(sums, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->du_acc, sums[0]);
    atomicAdd(&st->u_acc, sums[1]);
    atomicAdd(&st->q_acc, sums[2]);
    if (any_bad) atomicExch(&st->nan_flag, 1);
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket2, 1u);
    if (t == (unsigned)D->fin_nblocks - 1u) {
      __threadfence();
      const double dsum = atomicAdd(&st->du_acc, 0.0);
      const double usum = atomicAdd(&st->u_acc, 0.0);
      const double qsum = atomicAdd(&st->q_acc, 0.0);
      st->ticket2 = 0u;
      stop_test(D, st, dsum, usum, qsum, c_new, s);
    }
  }
}

// h = 0: records with B = F (C = F when the flow is along x2) and everything else zero; state cleared.
template <typename T>
__global__ void reset_kernel(const InstanceDesc *D) {
  const int ncell = D->ncell;
  SweepRec<T> *rec = static_cast<SweepRec<T> *>(D->rec);
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncell; cell += gridDim.x * blockDim.x) {
    const uint32_t code0 = D->code4[(size_t)cell * 4];
    const double d = (code0 & kSolid) ? 0.0 : (D->uniform_delta ? D->delta : D->delta_field[cell]);
    const double F = (code0 & kSolid) ? 0.0 : D->force;
    const double B = D->flow_axis ? 0.0 : F, C = D->flow_axis ? F : 0.0;
    for (int q = 0; q < 4; ++q) {
      store_rec<T>(rec + (size_t)q * ncell + cell, 0.0, B, C, 0.0, 0.0, 0.0, D->code4[(size_t)cell * 4 + q], d);
      if (D->rec_diag)
        store_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                         diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) != 0, (q & 2) != 0),
                     0.0, B, C, 0.0, 0.0, 0.0, D->code4[(size_t)cell * 4 + q], d);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    DeviceState *st = D->state;
    st->iter = 0;
    st->done = 0;
    st->status = 0;
    st->max_iter = 0;
    st->nan_flag = 0;
    st->err_flag = 0;
    st->ticket1 = st->ticket2 = 0u;
    st->tol = 0.0;
    st->c = st->s = st->s_new = 0.0;
    st->eps = st->est = st->Q = 0.0;
    for (int k = 0; k < 4; ++k) st->eps_ring[k] = 0.0;
    st->eps_min = INFINITY;
    st->iter_min = 0;
    st->mass_acc = st->du_acc = st->u_acc = st->q_acc = 0.0;
    st->aa_res = st->aa_est = st->aa_res_min = INFINITY;
    st->aa_rho = 0.0;
    st->aa_iter_min = 0;
  }
}

// Records (both layouts) of every cell from the stored state: moments, st->c, st->s and the fluxes of
// the last sweep (parity st->iter & 1).  Solid cells get zero records.
template <typename T>
__global__ void records_kernel(const InstanceDesc *D) {
  const DeviceState *st = D->state;
  const int ncell = D->ncell;
  const double *fcur = D->facc + (size_t)(st->iter & 1) * ncell * 4;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncell; cell += gridDim.x * blockDim.x) {
    const uint32_t code0 = D->code4[(size_t)cell * 4];
    if (code0 & kSolid) {
      for (int q = 0; q < 4; ++q) {
        store_rec<T>(static_cast<SweepRec<T> *>(D->rec) + (size_t)q * ncell + cell, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
                     D->code4[(size_t)cell * 4 + q], 0.0);
        if (D->rec_diag)
          store_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                           diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) != 0, (q & 2) != 0),
                       0.0, 0.0, 0.0, 0.0, 0.0, 0.0, D->code4[(size_t)cell * 4 + q], 0.0);
      }
      continue;
    }
    const Dbl4 m = reinterpret_cast<const Dbl4 *>(D->mom)[cell];
    write_records<T>(D, cell, m.x, m.y, m.z, m.w, st->c, st->s, fcur, nullptr, true);
  }
}

// Rebuild the diagonal-major records from the row-major ones (all four quadrants).
template <typename T>
__global__ void sync_diag_kernel(const InstanceDesc *D) {
  const int ncell = D->ncell;
  const SweepRec<T> *rec = static_cast<const SweepRec<T> *>(D->rec);
  SweepRec<T> *diag = static_cast<SweepRec<T> *>(D->rec_diag);
  const size_t qs = diag_quadrant_size(D->nx, D->ny);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * ncell; t += gridDim.x * blockDim.x) {
    const int q = t / ncell, cell = t - q * ncell;
    diag[q * qs + diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) != 0, (q & 2) != 0)] =
        rec[(size_t)q * ncell + cell];
  }
}

__global__ void arm_kernel(DeviceState *st, double tol, int max_iter_abs) {
  st->tol = tol;
  st->eps_min = INFINITY;
  st->iter_min = st->iter;
  st->aa_res_min = INFINITY;
  st->aa_iter_min = st->iter;
  st->max_iter = max_iter_abs;
  st->status = 0;
  st->nan_flag = 0;
  st->err_flag = 0;
  st->done = (st->iter >= max_iter_abs) ? 1 : 0;
  if (st->done) st->status = 4;
}

// Arm every instance of a launch for `count` more sweeps, relative to its device-side sweep count
// (no host read of the state: used by asynchronous batch sweeps).
__global__ void arm_all_kernel(const InstanceDesc *descs, int n, double tol, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DeviceState *st = descs[i].state;
  const long long lim = (long long)st->iter + count;
  const int max_iter_abs = lim > 2000000000LL ? 2000000000 : (int)lim;
  st->tol = tol;
  st->eps_min = INFINITY;
  st->iter_min = st->iter;
  st->aa_res_min = INFINITY;
  st->aa_iter_min = st->iter;
  st->max_iter = max_iter_abs;
  st->status = 0;
  st->nan_flag = 0;
  st->err_flag = 0;
  st->done = (st->iter >= max_iter_abs) ? 1 : 0;
  if (st->done) st->status = 4;
}

}  // namespace

cudaError_t launch_arm_all(const InstanceDesc *descs, int n, double tol, int count, cudaStream_t stream) {
  arm_all_kernel<<<(n + 127) / 128, 128, 0, stream>>>(descs, n, tol, count);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const LaunchDesc &L, int nblocks, bool fp64, cudaStream_t stream) {
  fin1_kernel<<<nblocks, kFinBlock, 0, stream>>>(L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (L.anderson) {
    e = launch_anderson(L, fp64, stream);
    if (e != cudaSuccess) return e;
  }
  if (fp64)
    fin2_kernel<double><<<nblocks, kFinBlock, 0, stream>>>(L);
  else
    fin2_kernel<float><<<nblocks, kFinBlock, 0, stream>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_reset(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream) {
  const int blocks = (ncell + 255) / 256 < 1024 ? (ncell + 255) / 256 : 1024;
  if (fp64)
    reset_kernel<double><<<blocks, 256, 0, stream>>>(inst_dev);
  else
    reset_kernel<float><<<blocks, 256, 0, stream>>>(inst_dev);
  return cudaGetLastError();
}

cudaError_t launch_records(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream) {
  const int blocks = (ncell + 255) / 256 < 1024 ? (ncell + 255) / 256 : 1024;
  if (fp64)
    records_kernel<double><<<blocks, 256, 0, stream>>>(inst_dev);
  else
    records_kernel<float><<<blocks, 256, 0, stream>>>(inst_dev);
  return cudaGetLastError();
}

cudaError_t launch_sync_diag(const InstanceDesc *inst_dev, int ncell, bool fp64, cudaStream_t stream) {
  const int blocks = (4 * ncell + 255) / 256 < 1024 ? (4 * ncell + 255) / 256 : 1024;
  if (fp64)
    sync_diag_kernel<double><<<blocks, 256, 0, stream>>>(inst_dev);
  else
    sync_diag_kernel<float><<<blocks, 256, 0, stream>>>(inst_dev);
  return cudaGetLastError();
}

cudaError_t launch_arm(DeviceState *st, double tol, int max_iter_abs, cudaStream_t stream) {
  arm_kernel<<<1, 1, 0, stream>>>(st, tol, max_iter_abs);
  return cudaGetLastError();
}

}  // namespace dvm
