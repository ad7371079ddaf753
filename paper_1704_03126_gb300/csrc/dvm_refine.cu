// dvm_refine.cu -- mixed-precision refinement of the FP32-storage source iteration.
//
// With FP32 storage the sweep rounds h to about 1e-7 relative, and the source iteration of
// Eq. (iteration) amplifies that rounding by 1 / (1 - r) (r its contraction rate): where the plain
// iteration converges slowly (small Kn, long channels) the FP32 fixed point lies 1e-5 to 1e-4 from the
// FP64 one.  Iterative refinement removes that error without sweeping in FP64 more than once per pass.
//
// The iteration maps the state x = (moments, wall values, periodic seam values, mass shift c) to
// G(x) = P S(x): S is the affine sweep (force and moving plate are its constant part), P the mean-
// density projection.  With the FP32 fixed point x~ (G~(x~) = x~, G~ the FP32 map):
//   1. rho = G(x~) - x~, one sweep of an FP64 twin of the instance started from x~ (exact transfer:
//      the FP32 state is a set of FP64 moments and wall values and FP32 seam values);
//   2. d solves d = P S_0(d) + rho (S_0: the sweep without force or plate drift), by the FP32
//      iteration itself: its rounding is now relative to |d|, which is |rho| / (1 - r), not |x|;
//   3. x = x~ + d.
// The error left after a pass is about (1e-7 / (1 - r) + the correction's own tolerance) |d|; passes
// repeat until that estimate (flow velocity, L1 over gas cells, relative to |x|) is below the caller's
// tolerance, usually after one pass.
//
// State buffers per instance (FP64 unless noted), laid out as the correction input rho of
// InstanceDesc: [4 ncell] moments (rho, u1, u2, tau) | [4 ncell] wall values per (cell, side), the
// projected incident flux divided by the outgoing normaliser (what the records use) | [1] c; seam values
// [seam_x | seam_y] in the storage precision.  Wall values are formed with each instance's own
// normalisers, so the transfer between the FP32 instance and its FP64 twin keeps them exactly.
#include <algorithm>

#include <cuda_runtime.h>

#include "dvm_device.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace {

constexpr int kRefBlock = 256;

struct alignas(32) Dbl4r {
  double x, y, z, w;
};

__device__ __forceinline__ size_t seam_x_count(const InstanceDesc *D) {
  return D->periodic_x ? (size_t)D->ngroups * D->ny * 2 * kLanes : 0;
}
__device__ __forceinline__ size_t seam_y_count(const InstanceDesc *D) {
  return D->periodic_y ? (size_t)D->ngroups * D->nx * 2 * kLanes : 0;
}

// x~: moments, wall values, raw seams; scalars [c, s, Q, iter].
template <typename T>
__global__ void snapshot_kernel(const InstanceDesc *D, double *snap, T *snap_seam, double *snap_sc) {
  const DeviceState *st = D->state;
  const int ncell = D->ncell;
  const double s = st->s;
  const double *F = D->facc + (size_t)(st->iter & 1) * ncell * 4;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t cell = tid; cell < (size_t)ncell; cell += stride) {
    reinterpret_cast<Dbl4r *>(snap)[cell] = reinterpret_cast<const Dbl4r *>(D->mom)[cell];
    for (int side = 0; side < 4; ++side)
      snap[(size_t)4 * ncell + cell * 4 + side] = (F[cell * 4 + side] - s * D->ain[side]) / D->nrm[side];
  }
  const size_t nsx = seam_x_count(D), nsy = seam_y_count(D);
  for (size_t e = tid; e < nsx + nsy; e += stride)
    snap_seam[e] = e < nsx ? static_cast<const T *>(D->seam_x)[e] : static_cast<const T *>(D->seam_y)[e - nsx];
  if (tid == 0) {
    snap[(size_t)8 * ncell] = st->c;
    snap_sc[0] = st->c;
    snap_sc[1] = s;
    snap_sc[2] = st->Q;
    snap_sc[3] = (double)st->iter;
  }
}

// Start the FP64 twin Tw from the state of D: the same moments, wall values, seam values and shifts.
template <typename T>
__global__ void load_twin_kernel(const InstanceDesc *D, const InstanceDesc *Tw) {
  const DeviceState *st = D->state;
  const int ncell = D->ncell;
  const double s = st->s;
  const int par = st->iter & 1;
  const double *F = D->facc + (size_t)par * ncell * 4;
  double *Ft = Tw->facc + (size_t)par * ncell * 4;
  double *Fo = Tw->facc + (size_t)(par ^ 1) * ncell * 4;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t cell = tid; cell < (size_t)ncell; cell += stride) {
    reinterpret_cast<Dbl4r *>(Tw->mom)[cell] = reinterpret_cast<const Dbl4r *>(D->mom)[cell];
    reinterpret_cast<Dbl4r *>(Tw->acc)[cell] = Dbl4r{0.0, 0.0, 0.0, 0.0};
    for (int side = 0; side < 4; ++side) {
      const double w = (F[cell * 4 + side] - s * D->ain[side]) / D->nrm[side];
      Ft[cell * 4 + side] = w * Tw->nrm[side] + s * Tw->ain[side];
      Fo[cell * 4 + side] = 0.0;
    }
  }
  const size_t nsx = seam_x_count(D), nsy = seam_y_count(D);
  for (size_t e = tid; e < nsx + nsy; e += stride) {
    if (e < nsx)
      static_cast<double *>(Tw->seam_x)[e] = (double)static_cast<const T *>(D->seam_x)[e];
    else
      static_cast<double *>(Tw->seam_y)[e - nsx] = (double)static_cast<const T *>(D->seam_y)[e - nsx];
  }
  if (tid == 0) {
    DeviceState *t = Tw->state;
    t->iter = st->iter;
    t->done = 0;
    t->status = 0;
    t->nan_flag = 0;
    t->err_flag = 0;
    t->ticket1 = t->ticket2 = 0u;
    t->c = st->c;
    t->s = s;
    t->s_new = 0.0;
    t->mass_acc = t->du_acc = t->u_acc = t->q_acc = 0.0;
  }
}

// rho = G(x~) - x~ from the twin's state after its sweep, in the FP32 instance's units.
template <typename T>
__global__ void residual_kernel(const InstanceDesc *D, const InstanceDesc *Tw, const double *snap, const T *snap_seam,
                                const double *snap_sc, double *rho, T *rho_seam) {
  const DeviceState *tst = Tw->state;
  const int ncell = D->ncell;
  const double st_ = tst->s;
  const double *Ft = Tw->facc + (size_t)(tst->iter & 1) * ncell * 4;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t cell = tid; cell < (size_t)ncell; cell += stride) {
    const Dbl4r a = reinterpret_cast<const Dbl4r *>(Tw->mom)[cell];
    const Dbl4r b = reinterpret_cast<const Dbl4r *>(snap)[cell];
    reinterpret_cast<Dbl4r *>(rho)[cell] = Dbl4r{a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w};
    for (int side = 0; side < 4; ++side) {
      const double wt = (Ft[cell * 4 + side] - st_ * Tw->ain[side]) / Tw->nrm[side];
      // the correction phase adds this to the projected flux of the FP32 instance (fin2)
      rho[(size_t)4 * ncell + cell * 4 + side] = (wt - snap[(size_t)4 * ncell + cell * 4 + side]) * D->nrm[side];
    }
  }
  const size_t nsx = seam_x_count(D), nsy = seam_y_count(D);
  const double s0 = snap_sc[1];
  for (size_t e = tid; e < nsx + nsy; e += stride) {
    const double vt = e < nsx ? static_cast<const double *>(Tw->seam_x)[e] : static_cast<const double *>(Tw->seam_y)[e - nsx];
    rho_seam[e] = (T)((vt - st_) - ((double)snap_seam[e] - s0));
  }
  if (tid == 0) rho[(size_t)8 * ncell] = tst->c - snap_sc[0];
}

// x = x~ + d: d is the state the correction phase left in D's buffers (its wall values include the
// injected rho, its raw seams too).  Stored with no pending shift; sums[0] += |u_d|, sums[1] += |u|
// over the gas cells (flow component).
template <typename T>
__global__ void combine_kernel(const InstanceDesc *D, const double *snap, const T *snap_seam, const double *snap_sc,
                               const double *rho, double *sums) {
  __shared__ double sh[2][kRefBlock / 32];
  const DeviceState *st = D->state;
  const int ncell = D->ncell;
  const double sd = st->s;
  const int par_d = st->iter & 1;
  const long long new_iter = (long long)snap_sc[3] + st->iter;
  const int par = (int)(new_iter & 1);
  const double *Fd = D->facc + (size_t)par_d * ncell * 4;
  double *Fn = D->facc + (size_t)par * ncell * 4;
  double *Fo = D->facc + (size_t)(par ^ 1) * ncell * 4;
  const int comp = D->flow_axis ? 2 : 1;
  double ad = 0.0, ax = 0.0;
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t cell = tid; cell < (size_t)ncell; cell += stride) {
    double w[4];
    for (int side = 0; side < 4; ++side) {
      const double wd = (Fd[cell * 4 + side] - sd * D->ain[side] + rho[(size_t)4 * ncell + cell * 4 + side]) / D->nrm[side];
      w[side] = snap[(size_t)4 * ncell + cell * 4 + side] + wd;
    }
    // Fd and Fn may be the same array: read all four before writing
    for (int side = 0; side < 4; ++side) {
      Fn[cell * 4 + side] = w[side] * D->nrm[side];
      if (Fo != Fn) Fo[cell * 4 + side] = 0.0;
    }
    const Dbl4r a = reinterpret_cast<const Dbl4r *>(snap)[cell];
    const Dbl4r b = reinterpret_cast<const Dbl4r *>(D->mom)[cell];
    const Dbl4r m{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
    reinterpret_cast<Dbl4r *>(D->mom)[cell] = m;
    if (!(D->code4[cell * 4] & kSolid)) {
      const double uf = comp == 1 ? m.y : m.z, ud = comp == 1 ? b.y : b.z;
      D->u1prev[cell] = uf;
      ad += fabs(ud);
      ax += fabs(uf);
    }
  }
  const size_t nsx = seam_x_count(D), nsy = seam_y_count(D);
  const double s0 = snap_sc[1];
  for (size_t e = tid; e < nsx + nsy; e += stride) {
    T *p = e < nsx ? static_cast<T *>(D->seam_x) + e : static_cast<T *>(D->seam_y) + (e - nsx);
    *p = (T)(((double)snap_seam[e] - s0) + ((double)*p - sd));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ad += __shfl_xor_sync(0xffffffffu, ad, o);
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = ad;
    sh[1][threadIdx.x >> 5] = ax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a0 += sh[0][i];
      a1 += sh[1][i];
    }
    atomicAdd(&sums[0], a0);
    atomicAdd(&sums[1], a1);
  }
}

// Scalars of the combined state (after combine_kernel has read d's): c, no pending shift, Q, the sweeps
// of both phases, and the size of the last correction as the error estimate.
__global__ void combine_state_kernel(const InstanceDesc *D, const double *snap_sc, const double *sums) {
  DeviceState *st = D->state;
  st->c = snap_sc[0] + st->c;
  st->s = 0.0;
  st->s_new = 0.0;
  st->Q = snap_sc[2] + st->Q;
  const long long it = (long long)snap_sc[3] + st->iter;
  st->iter = it > 2000000000LL ? 2000000000 : (int)it;
  st->est = sums[1] > 0.0 ? sums[0] / sums[1] : 0.0;
  st->eps = st->est;
  st->status = 0;
  st->done = 1;
}

int grid_for(size_t n) {
  const size_t b = (n + kRefBlock - 1) / kRefBlock;
  return (int)(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

}  // namespace

size_t refine_seam_count(const InstanceDesc &D) {
  return (D.periodic_x ? (size_t)D.ngroups * D.ny * 2 * kLanes : 0) +
         (D.periodic_y ? (size_t)D.ngroups * D.nx * 2 * kLanes : 0);
}

cudaError_t launch_refine_snapshot(const InstanceDesc *d, const InstanceDesc &h, bool fp64, double *snap, void *snap_seam,
                                   double *snap_sc, cudaStream_t s) {
  const int g = grid_for(std::max((size_t)h.ncell, refine_seam_count(h)));
  if (fp64)
    snapshot_kernel<double><<<g, kRefBlock, 0, s>>>(d, snap, static_cast<double *>(snap_seam), snap_sc);
  else
    snapshot_kernel<float><<<g, kRefBlock, 0, s>>>(d, snap, static_cast<float *>(snap_seam), snap_sc);
  return cudaGetLastError();
}

cudaError_t launch_refine_load_twin(const InstanceDesc *d, const InstanceDesc *twin, const InstanceDesc &h, bool fp64,
                                    cudaStream_t s) {
  const int g = grid_for(std::max((size_t)h.ncell, refine_seam_count(h)));
  if (fp64)
    load_twin_kernel<double><<<g, kRefBlock, 0, s>>>(d, twin);
  else
    load_twin_kernel<float><<<g, kRefBlock, 0, s>>>(d, twin);
  return cudaGetLastError();
}

cudaError_t launch_refine_residual(const InstanceDesc *d, const InstanceDesc *twin, const InstanceDesc &h, bool fp64,
                                   const double *snap, const void *snap_seam, const double *snap_sc, double *rho,
                                   void *rho_seam, cudaStream_t s) {
  const int g = grid_for(std::max((size_t)h.ncell, refine_seam_count(h)));
  if (fp64)
    residual_kernel<double><<<g, kRefBlock, 0, s>>>(d, twin, snap, static_cast<const double *>(snap_seam), snap_sc, rho,
                                                     static_cast<double *>(rho_seam));
  else
    residual_kernel<float><<<g, kRefBlock, 0, s>>>(d, twin, snap, static_cast<const float *>(snap_seam), snap_sc, rho,
                                                    static_cast<float *>(rho_seam));
  return cudaGetLastError();
}

cudaError_t launch_refine_combine(const InstanceDesc *d, const InstanceDesc &h, bool fp64, const double *snap,
                                  const void *snap_seam, const double *snap_sc, const double *rho, double *sums,
                                  cudaStream_t s) {
  const int g = grid_for(std::max((size_t)h.ncell, refine_seam_count(h)));
  cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (fp64)
    combine_kernel<double><<<g, kRefBlock, 0, s>>>(d, snap, static_cast<const double *>(snap_seam), snap_sc, rho, sums);
  else
    combine_kernel<float><<<g, kRefBlock, 0, s>>>(d, snap, static_cast<const float *>(snap_seam), snap_sc, rho, sums);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  combine_state_kernel<<<1, 1, 0, s>>>(d, snap_sc, sums);
  return cudaGetLastError();
}

}  // namespace dvm
