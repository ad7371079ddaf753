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
#include "dvm_kernels.h"

namespace dvm {
namespace {

constexpr int kFinBlock = 256;

struct alignas(32) Dbl4 {
  double x, y, z, w;
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__global__ void __launch_bounds__(kFinBlock) fin1_kernel(LaunchDesc L) {
  __shared__ double sh[32];
  const int map = L.fin_map[blockIdx.x];
  const InstanceDesc *D = L.inst + (map >> 16);
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int cell = (map & 0xffff) * kFinBlock + threadIdx.x;
  double v = 0.0;
  if (cell < D->ncell && !(D->code4[(size_t)cell * 4] & kSolid)) v = D->acc[(size_t)cell * 4];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->mass_acc, v);
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

// Write the sweep record of one cell and quadrant: right-hand-side coefficients, the upwind
// coefficients of the cell's stencil classes and the wall terms 2 h_w of wall-class axes.
template <typename T>
__device__ __forceinline__ void store_rec(SweepRec<T> *dst, double A, double B, double C, double Dd, double hwx,
                                          double hwy, uint32_t code, double delta);
template <>
__device__ __forceinline__ void store_rec<float>(SweepRec<float> *dst, double A, double B, double C, double Dd,
                                                 double hwx, double hwy, uint32_t code, double delta) {
  const int clx = (code >> kClsXShift) & 3, cly = (code >> kClsYShift) & 3;
  const bool solid = (code & kSolid) != 0;
  SweepRec<float> r;
  r.A = solid ? 0.f : (float)A;
  r.B = solid ? 0.f : (float)B;
  r.C = solid ? 0.f : (float)C;
  r.D = solid ? 0.f : (float)Dd;
  r.ax1 = solid ? 0.f : class_a1(clx);
  r.ax2 = solid ? 0.f : class_a2(clx);
  r.xw = (!solid && clx == kWall) ? (float)(2.0 * hwx) : 0.f;
  r.ay1 = solid ? 0.f : class_a1(cly);
  r.ay2 = solid ? 0.f : class_a2(cly);
  r.yw = (!solid && cly == kWall) ? (float)(2.0 * hwy) : 0.f;
  r.code = code;
  r.delta = (float)delta;
  *dst = r;
}
template <>
__device__ __forceinline__ void store_rec<double>(SweepRec<double> *dst, double A, double B, double C, double Dd,
                                                  double hwx, double hwy, uint32_t code, double delta) {
  const int clx = (code >> kClsXShift) & 3, cly = (code >> kClsYShift) & 3;
  const bool solid = (code & kSolid) != 0;
  SweepRec<double> r;
  r.A = solid ? 0.0 : A;
  r.B = solid ? 0.0 : B;
  r.C = solid ? 0.0 : C;
  r.D = solid ? 0.0 : Dd;
  r.xw = (!solid && clx == kWall) ? 2.0 * hwx : 0.0;
  r.yw = (!solid && cly == kWall) ? 2.0 * hwy : 0.0;
  r.code = code;
  r.pad = 0u;
  r.delta = delta;
  *dst = r;
}

// The sweep records of gas cell `cell` for all four quadrants from its moments (rho, u1, u2, tau), the
// accumulated mass shift c, the pending shift s of the stored fluxes and the raw incident fluxes fcur
// (with the correction phase's rho added to the projected fluxes when rho_in is set); the diagonal-
// major copy too when `diag`.
template <typename T>
__device__ __forceinline__ void write_records(const InstanceDesc *D, int cell, double rho, double u1, double u2,
                                              double tau, double c, double s, const double *fcur,
                                              const double *rho_in, bool diag) {
  const int ncell = D->ncell;
  const double d = D->uniform_delta ? D->delta : D->delta_field[cell];
  // collision coefficients a = G^{-1} m, m = (rho, u1, u2, rho + tau) = sum W psi h
  const double m[4] = {rho, u1, u2, rho + tau};
  double a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    a[i] = D->ginv[i * 4] * m[0] + D->ginv[i * 4 + 1] * m[1] + D->ginv[i * 4 + 2] * m[2] + D->ginv[i * 4 + 3] * m[3];
  // R = delta (a0 + a1 v1 + a2 v2 + a3 |v|^2 - c) + F v_flow in the basis 1, v1, v2, |v|^2 - 1
  const double A = d * (a[0] + a[3] - c);
  const double B = d * a[1] + (D->flow_axis ? 0.0 : D->force);
  const double Cc = d * a[2] + (D->flow_axis ? D->force : 0.0);
  const double Dd = d * a[3];
  SweepRec<T> *rec = static_cast<SweepRec<T> *>(D->rec);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double hw[2];
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const int src = D->hw_src[(size_t)cell * 8 + q * 2 + ax];
      if (src >= 0) {
        const int side = src & 3;
        // diffuse part alpha rho_w; the specular part (1 - alpha) h(mirror v) is added in the sweep
        const double corr = rho_in ? rho_in[(size_t)4 * ncell + src] : 0.0;
        hw[ax] = D->alpha * (fcur[src] - s * D->ain[side] + corr) / D->nrm[side];
      } else {
        hw[ax] = 0.0;
      }
    }
    store_rec<T>(rec + (size_t)q * ncell + cell, A, B, Cc, Dd, hw[0], hw[1], D->code4[(size_t)cell * 4 + q], d);
    // the diagonal-major copy only feeds the column sweep (rebuilt by sync_diag when a launch
    // switches to it)
    if (diag && D->rec_diag)
      store_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                       diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) != 0, (q & 2) != 0),
                   A, B, Cc, Dd, hw[0], hw[1], D->code4[(size_t)cell * 4 + q], d);
  }
}

template <typename T>
__global__ void __launch_bounds__(kFinBlock) fin2_kernel(LaunchDesc L) {
  __shared__ double sh[32];
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
  if (cell < ncell) {
    const uint32_t code0 = D->code4[(size_t)cell * 4];
    if (!(code0 & kSolid)) {
      Dbl4 *acc4 = reinterpret_cast<Dbl4 *>(D->acc);
      const Dbl4 am = acc4[cell];
      acc4[cell] = Dbl4{0.0, 0.0, 0.0, 0.0};
      double rho = am.x - s * D->sumW[0];
      double u1 = am.y - s * D->sumW[1];
      double u2 = am.z - s * D->sumW[2];
      double tau = (am.w - s * D->sumW[3]) - rho;
      if (rho_in) {
        const Dbl4 r = reinterpret_cast<const Dbl4 *>(rho_in)[cell];
        rho += r.x;
        u1 += r.y;
        u2 += r.z;
        tau += r.w;
      }
      reinterpret_cast<Dbl4 *>(D->mom)[cell] = Dbl4{rho, u1, u2, tau};
      write_records<T>(D, cell, rho, u1, u2, tau, c_new, s, fcur, rho_in, L.cols_v != 0);
      const double uf = D->flow_axis ? u2 : u1;  // velocity along the flow
      du = fabs(uf - D->u1prev[cell]);
      ua = fabs(uf);
      uq = D->xwidth ? uf * D->xwidth[cell % D->nx] : uf;  // area-weighted for unequal columns
      D->u1prev[cell] = uf;
      if (!isfinite(rho) || !isfinite(u1) || !isfinite(u2) || !isfinite(tau)) bad = 1.0;
    }
    reinterpret_cast<Dbl4 *>(fnext)[cell] = Dbl4{0.0, 0.0, 0.0, 0.0};
  }
  if (rho_in) {
    // the seam part of rho goes into the raw seam values the next sweep reads (this sweep has written
    // them; the next one subtracts the pending shift from raw + rho)
    const size_t nsx = D->periodic_x ? (size_t)D->ngroups * D->ny * 2 * kLanes : 0;
    const size_t nsy = D->periodic_y ? (size_t)D->ngroups * D->nx * 2 * kLanes : 0;
    const size_t stride = (size_t)D->fin_nblocks * kFinBlock;
    for (size_t e = (size_t)(map & 0xffff) * kFinBlock + threadIdx.x; e < nsx + nsy; e += stride) {
      T *dst = e < nsx ? static_cast<T *>(D->seam_x) + e : static_cast<T *>(D->seam_y) + (e - nsx);
      const T add = e < nsx ? static_cast<const T *>(D->rho_seam_x)[e] : static_cast<const T *>(D->rho_seam_y)[e - nsx];
      *dst += add;
    }
  }
  du = block_sum(du, sh);
  ua = block_sum(ua, sh);
  uq = block_sum(uq, sh);
  bad = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->du_acc, du);
    atomicAdd(&st->u_acc, ua);
    atomicAdd(&st->q_acc, uq);
    if (bad > 0.0) atomicExch(&st->nan_flag, 1);
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket2, 1u);
    if (t == (unsigned)D->fin_nblocks - 1u) {
      __threadfence();
      const double dsum = atomicAdd(&st->du_acc, 0.0);
      const double usum = atomicAdd(&st->u_acc, 0.0);
      const double qsum = atomicAdd(&st->q_acc, 0.0);
      const int n = st->iter + 1;
      const double eps = usum > 0.0 ? dsum / usum : 0.0;
      const double back = st->eps_ring[n & 3];  // eps_{n-4}
      st->eps_ring[n & 3] = eps;
      double est = INFINITY;
      int done = 0, status = 0;
      if (D->aa) {
        // mixed iterates (FP64 storage only): the estimate from the plain residual (dvm_anderson.cu).
        // Near the rounding floor the residual stops falling while rho keeps the estimate above a
        // tight tol: below tol, 32 sweeps without a 10 % smaller residual also end the iteration.
        est = st->aa_est;
        if (n >= 5 && est < st->tol) done = 1;
        if (st->aa_res < 0.9 * st->aa_res_min) {
          st->aa_res_min = st->aa_res;
          st->aa_iter_min = n;
        }
        if (!done && n >= 5 && st->aa_res < st->tol && n - st->aa_iter_min >= 32) done = 1;
      } else {
        if (n >= 5) {
          double r = back > 0.0 ? pow(eps / back, 0.25) : 0.0;
          if (r > 0.9999) r = 0.9999;
          est = eps / (1.0 - r);
          if (est < st->tol) done = 1;
        }
        // With FP32 storage the change per sweep stalls at the rounding noise floor, where the rate
        // estimate says nothing: below tol, 16 sweeps without a new smallest eps also end the iteration.
        if (eps < st->eps_min) {
          st->eps_min = eps;
          st->iter_min = n;
        }
        if (!done && D->fp32 && n >= 5 && eps < st->tol && n - st->iter_min >= 16) done = 1;
      }
      if (!done && n >= st->max_iter) {
        done = 1;
        status = 4;  // DVM_ENOCONV
      }
      if (atomicAdd(&st->nan_flag, 0) != 0) {
        done = 1;
        status = 6;  // DVM_ENUMERIC
      }
      if (atomicAdd(&st->err_flag, 0) != 0) {
        done = 1;
        status = 5;  // DVM_ETIMEOUT: a sweep block gave up waiting on another warp
      }
      st->iter = n;
      st->c = c_new;
      st->s = s;
      st->eps = eps;
      st->est = est;
      st->Q = qsum * D->dA_over_Lx;
      st->du_acc = 0.0;
      st->u_acc = 0.0;
      st->q_acc = 0.0;
      st->ticket2 = 0u;
      st->status = status;
      __threadfence();
      st->done = done;
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
