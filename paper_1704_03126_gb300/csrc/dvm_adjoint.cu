// dvm_adjoint.cu -- the adjoint of the projected source iteration (gradient of Q with respect to the
// per-cell collision rate delta_c), outside the transposed sweep itself.
//
// One forward iteration is Phi(h, c) = P(S(h, c)): S solves T h~ = delta (M(h) - c) + L(h) + F v1
// (T: the in-sweep upwind operator, L: the lagged wall and seam terms, M: the collision
// projection), and P shifts h~ by s = rho^T h~ (rho = W / (n_gas sum W)) into c.  At the fixed point,
// dQ/d delta = Lambda^T dPhi/d delta with Lambda = J^T Lambda + (g, 0), g = W v1 dA / Lx.  One adjoint
// step, given (lambda, mu):
//     lambda' = lambda + rho (mu - sum lambda)                  (transpose of P)
//     z       = T^{-T} lambda'                                  (the transposed sweep)
//     lambda  = (delta M)^T z + L^T z + g,   mu = mu - sum_c delta_c sum_k z_kc
// and dQ/d delta_c = sum_k z_kc (M_kc - c - h_kc).  The transposed sweep (dvm_sweep.cuh, ADJ) takes
// lambda' as W_k (A + B v1 + C v2 + D (|v|^2 - 1)) + |v1| W TX + |v2| W TY and returns the unweighted
// moments Z = sum_k (1, v1, v2, |v|^2) z_k, the transposed wall reads t_f and the seam values.
// Here: (delta M)^T z = delta W psi(v) . G^{-T} Z, the lagged seam sums, sum lambda, mu, the next
// records, the stopping test and finally the gradient.
#include <cmath>
#include <cstdint>

#include "dvm_device.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace {

constexpr int kBlock = 256;

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
  return r;
}

// Lagged reads across periodic seams: in the next transposed sweep, the first two cells of a line
// (in its visiting order) read the seam values of the last two with weights t1, t2; their sum
// |v_a|/dx (t1(p0) z(slot 1) + t2(p0) z(slot 0) + t2(p1) z(slot 1)) belongs to sum lambda.
// One warp per seam line: group x row (x seams), then group x column (y seams).
template <typename T>
__global__ void __launch_bounds__(kBlock) aseam_kernel(const InstanceDesc *D) {
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nx = D->nx, ny = D->ny, G = D->ngroups;
  const int nxl = D->periodic_x ? G * ny : 0, nyl = D->periodic_y ? G * nx : 0;
  if (gw >= nxl + nyl) return;
  const bool is_x = gw < nxl;
  const int g = is_x ? gw / ny : (gw - nxl) / nx;
  const int line = is_x ? gw % ny : (gw - nxl) % nx;
  const int quad = g / D->groups_per_quadrant;
  const T *vt = static_cast<const T *>(D->vel) + (size_t)g * kNumVelFields * kLanes;
  double val;
  if (is_x) {
    const bool xneg = (quad & 1) == 0;  // transposed order: opposite to the forward one
    const int i0 = xneg ? nx - 1 : 0, i1 = xneg ? nx - 2 : 1;
    const uint32_t c0 = D->code4[((size_t)line * nx + i0) * 4 + quad];
    const uint32_t c1 = D->code4[((size_t)line * nx + i1) * 4 + quad];
    const double t1p0 = (double)((c0 >> kAdjT1XShift) & 3), t2p0 = (c0 & kAdjT2X) ? -0.5 : 0.0;
    const double t2p1 = (c1 & kAdjT2X) ? -0.5 : 0.0;
    const T *sx = static_cast<const T *>(D->seam_x) + ((size_t)g * ny + line) * 2 * kLanes;
    val = (double)vt[kCx * kLanes + lane] * (t1p0 * (double)sx[kLanes + lane] + t2p0 * (double)sx[lane] +
                                             t2p1 * (double)sx[kLanes + lane]);
  } else {
    const bool yneg = (quad & 2) == 0;
    const int j0 = yneg ? ny - 1 : 0, j1 = yneg ? ny - 2 : 1;
    const uint32_t c0 = D->code4[((size_t)j0 * nx + line) * 4 + quad];
    const uint32_t c1 = D->code4[((size_t)j1 * nx + line) * 4 + quad];
    const double t1p0 = (double)((c0 >> kAdjT1YShift) & 3), t2p0 = (c0 & kAdjT2Y) ? -0.5 : 0.0;
    const double t2p1 = (c1 & kAdjT2Y) ? -0.5 : 0.0;
    const T *sy = static_cast<const T *>(D->seam_y) + ((size_t)g * nx + line) * 2 * kLanes;
    val = (double)vt[kCy * kLanes + lane] * (t1p0 * (double)sy[kLanes + lane] + t2p0 * (double)sy[lane] +
                                             t2p1 * (double)sy[kLanes + lane]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
  if (lane == 0) atomicAdd(&st->seam_acc, val);
}

// Adjoint moments -> collision coefficients alpha = delta G^{-T} Z + (0, dA/Lx, 0, 0) per cell, the
// sums for mu and sum lambda, the relative change of Z1 = sum v_flow z (stopping test); v_flow = v1, or
// v2 for an instance stored transposed (then g and Z1 use the second moment).
__global__ void __launch_bounds__(kBlock) afin1_kernel(const InstanceDesc *D) {
  __shared__ double sh[32];
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int ncell = D->ncell;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  const int parity = (st->iter + 1) & 1;
  const double *fcur = D->facc + (size_t)parity * ncell * 4;
  double dz = 0.0, lam = 0.0, du = 0.0, ua = 0.0, bad = 0.0;
  if (cell < ncell && !(D->code4[(size_t)cell * 4] & kSolid)) {
    Dbl4 *acc4 = reinterpret_cast<Dbl4 *>(D->acc);
    const Dbl4 zz = acc4[cell];
    acc4[cell] = Dbl4{0.0, 0.0, 0.0, 0.0};
    const double Z[4] = {zz.x, zz.y, zz.z, zz.w};
    const double d = D->uniform_delta ? D->delta : D->delta_field[cell];
    double al[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      double y = 0.0;
#pragma unroll
      for (int j = 0; j < 4; ++j) y += D->ginv[j * 4 + i] * Z[j];
      al[i] = d * y;
    }
    // g = W v_flow dA / L (dA: the column's width for columns of unequal width)
    (D->flow_axis ? al[2] : al[1]) += D->dA_over_Lx * (D->xwidth ? D->xwidth[cell % D->nx] : 1.0);
    const double zf = D->flow_axis ? Z[2] : Z[1];
    reinterpret_cast<Dbl4 *>(D->mom)[cell] = Dbl4{al[0], al[1], al[2], al[3]};
    dz = d * Z[0];
#pragma unroll
    for (int i = 0; i < 4; ++i) lam += al[i] * D->sumW[i];
    // transposed walls: lambda(j, owner) += alpha t_f |v_j . n| W_j / N over incident j (diffuse part)
    // and (1 - alpha) 2 |v_a|/dx z of the mirrored velocity (specular part, added in the next
    // transposed sweep): their sum over j is t_f (alpha ain / N + 1 - alpha)
    const uint32_t c0 = D->code4[(size_t)cell * 4 + 0], c1 = D->code4[(size_t)cell * 4 + 1],
                   c2 = D->code4[(size_t)cell * 4 + 2];
    const double spec = 1.0 - D->alpha;
    if (c0 & kIncX) lam += fcur[(size_t)cell * 4 + kE] * (D->ain[kE] * D->wnrm[kE] + spec);
    if (c1 & kIncX) lam += fcur[(size_t)cell * 4 + kW] * (D->ain[kW] * D->wnrm[kW] + spec);
    if (c0 & kIncY) lam += fcur[(size_t)cell * 4 + kN] * (D->ain[kN] * D->wnrm[kN] + spec);
    if (c2 & kIncY) lam += fcur[(size_t)cell * 4 + kS] * (D->ain[kS] * D->wnrm[kS] + spec);
    du = fabs(zf - D->u1prev[cell]);
    ua = fabs(zf);
    D->u1prev[cell] = zf;
    if (!isfinite(Z[0]) || !isfinite(Z[1]) || !isfinite(Z[2]) || !isfinite(Z[3])) bad = 1.0;
  }
  dz = block_sum(dz, sh);
  lam = block_sum(lam, sh);
  du = block_sum(du, sh);
  ua = block_sum(ua, sh);
  bad = block_sum(bad, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->dz_acc, dz);
    atomicAdd(&st->lam_acc, lam);
    atomicAdd(&st->du_acc, du);
    atomicAdd(&st->u_acc, ua);
    if (bad > 0.0) atomicExch(&st->nan_flag, 1);
    __threadfence();
    const unsigned t = atomicAdd(&st->ticket1, 1u);
    if (t == gridDim.x - 1u) {
      __threadfence();
      const double dzs = atomicAdd(&st->dz_acc, 0.0);
      const double lams = atomicAdd(&st->lam_acc, 0.0) + atomicAdd(&st->seam_acc, 0.0);
      const double dsum = atomicAdd(&st->du_acc, 0.0);
      const double usum = atomicAdd(&st->u_acc, 0.0);
      const double mu = st->mu - dzs;
      st->mu = mu;
      st->kappa = (mu - lams) / ((double)D->n_gas * D->sumW[0]);
      const int n = st->iter + 1;
      const double eps = usum > 0.0 ? dsum / usum : 0.0;
      const double back = st->eps_ring[n & 3];
      st->eps_ring[n & 3] = eps;
      double est = INFINITY;
      int done = 0, status = 0;
      if (n >= 5 && usum > 0.0) {
        double r = back > 0.0 ? pow(eps / back, 0.25) : 0.0;
        if (r > 0.9999) r = 0.9999;
        est = eps / (1.0 - r);
        if (est < st->tol) done = 1;
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
        status = 5;  // DVM_ETIMEOUT
      }
      st->iter = n;
      st->eps = eps;
      st->est = est;
      st->dz_acc = st->lam_acc = st->seam_acc = st->du_acc = st->u_acc = 0.0;
      st->ticket1 = 0u;
      st->status = status;
      __threadfence();
      st->done = done;
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_adj_rec(SweepRec<T> *dst, const double al[4], double kappa, double tx, double ty,
                                              uint32_t code, double delta);
template <>
__device__ __forceinline__ void store_adj_rec<float>(SweepRec<float> *dst, const double al[4], double kappa, double tx,
                                                     double ty, uint32_t code, double delta) {
  const bool solid = (code & kSolid) != 0;
  SweepRec<float> r;
  r.A = solid ? 0.f : (float)(al[0] + al[3] + kappa);
  r.B = solid ? 0.f : (float)al[1];
  r.C = solid ? 0.f : (float)al[2];
  r.D = solid ? 0.f : (float)al[3];
  r.ax1 = (float)((code >> kAdjT1XShift) & 3);
  r.ax2 = (code & kAdjT2X) ? -0.5f : 0.f;
  r.xw = solid ? 0.f : (float)tx;
  r.ay1 = (float)((code >> kAdjT1YShift) & 3);
  r.ay2 = (code & kAdjT2Y) ? -0.5f : 0.f;
  r.yw = solid ? 0.f : (float)ty;
  r.code = code;
  r.delta = (float)delta;  // the transposed sweep has the forward diagonal delta_c + sum |v_a|/dx kappa_a
  *dst = r;
}
template <>
__device__ __forceinline__ void store_adj_rec<double>(SweepRec<double> *dst, const double al[4], double kappa,
                                                      double tx, double ty, uint32_t code, double delta) {
  const bool solid = (code & kSolid) != 0;
  SweepRec<double> r;
  r.A = solid ? 0.0 : al[0] + al[3] + kappa;
  r.B = solid ? 0.0 : al[1];
  r.C = solid ? 0.0 : al[2];
  r.D = solid ? 0.0 : al[3];
  r.xw = solid ? 0.0 : tx;
  r.yw = solid ? 0.0 : ty;
  r.code = code;
  r.pad = 0u;
  r.delta = delta;
  *dst = r;
}

// Right-hand sides of the next transposed sweep: W (alpha . psi + kappa) plus the incident-wall terms
// TX = alpha t_f / N at cells owning a face that the quadrant's velocities hit (alpha: accommodation).
template <typename T>
__global__ void __launch_bounds__(kBlock) afin2_kernel(const InstanceDesc *D) {
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;
  const int ncell = D->ncell;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  // afin1 advanced iter, so the sweep that just ran accumulated into parity (iter & 1)
  const int parity = st->iter & 1;
  const double *fcur = D->facc + (size_t)parity * ncell * 4;
  double *fnext = D->facc + (size_t)(parity ^ 1) * ncell * 4;
  const Dbl4 a4 = reinterpret_cast<const Dbl4 *>(D->mom)[cell];
  const double al[4] = {a4.x, a4.y, a4.z, a4.w};
  const double kappa = st->kappa;
  const bool solid = (D->code4[(size_t)cell * 4] & kSolid) != 0;
  const double d = solid ? 0.0 : (D->uniform_delta ? D->delta : D->delta_field[cell]);
  SweepRec<T> *rec = static_cast<SweepRec<T> *>(D->rec);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t code = D->code4[(size_t)cell * 4 + q];
    const int sx = (q & 1) ? kW : kE, sy = (q & 2) ? kS : kN;  // wall sides these velocities hit
    const double tx = (code & kIncX) ? fcur[(size_t)cell * 4 + sx] * D->wnrm[sx] : 0.0;
    const double ty = (code & kIncY) ? fcur[(size_t)cell * 4 + sy] * D->wnrm[sy] : 0.0;
    store_adj_rec<T>(rec + (size_t)q * ncell + cell, al, kappa, tx, ty, code, d);
    // the transposed sweep visits cells in the opposite order of the quadrant
    if (D->rec_diag)
      store_adj_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                           diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) == 0, (q & 2) == 0),
                       al, kappa, tx, ty, code, d);
  }
  reinterpret_cast<Dbl4 *>(fnext)[cell] = Dbl4{0.0, 0.0, 0.0, 0.0};
}

// lambda = 0, mu = 0: all-zero right-hand sides; adjoint state cleared.
template <typename T>
__global__ void areset_kernel(const InstanceDesc *D) {
  const int ncell = D->ncell;
  SweepRec<T> *rec = static_cast<SweepRec<T> *>(D->rec);
  const double zero[4] = {0.0, 0.0, 0.0, 0.0};
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncell; cell += gridDim.x * blockDim.x) {
    const bool solid = (D->code4[(size_t)cell * 4] & kSolid) != 0;
    const double d = solid ? 0.0 : (D->uniform_delta ? D->delta : D->delta_field[cell]);
    for (int q = 0; q < 4; ++q) {
      store_adj_rec<T>(rec + (size_t)q * ncell + cell, zero, 0.0, 0.0, 0.0, D->code4[(size_t)cell * 4 + q], d);
      if (D->rec_diag)
        store_adj_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                             diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) == 0, (q & 2) == 0),
                         zero, 0.0, 0.0, 0.0, D->code4[(size_t)cell * 4 + q], d);
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
    st->mu = st->kappa = 0.0;
    st->lam_acc = st->dz_acc = st->seam_acc = 0.0;
  }
}

// dQ/d delta_c = sum_k z_kc (M_kc - c - h_kc), one warp per cell over the groups; M from the forward
// moments through the collision projection, h the stored forward distribution minus its last shift.
// Also Q_identity = F sum z v_flow (equals Q at convergence), accumulated in state->Q.
template <typename T>
__global__ void __launch_bounds__(kBlock) agrad_kernel(const InstanceDesc *D) {
  const int lane = threadIdx.x & 31;
  const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (cell >= D->ncell) return;
  if (D->code4[(size_t)cell * 4] & kSolid) {
    if (lane == 0) D->grad[cell] = 0.0;
    return;
  }
  const DeviceState *sf = D->state_fwd;
  const double c = sf->c, s = sf->s;
  const Dbl4 m4 = reinterpret_cast<const Dbl4 *>(D->mom_fwd)[cell];
  const double m[4] = {m4.x, m4.y, m4.z, m4.x + m4.w};  // (rho, u1, u2, rho + tau)
  double a[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = D->ginv[i * 4] * m[0] + D->ginv[i * 4 + 1] * m[1] + D->ginv[i * 4 + 2] * m[2] + D->ginv[i * 4 + 3] * m[3];
  const size_t ncell = D->ncell;
  double gsum = 0.0, qsum = 0.0;
  for (int g = 0; g < D->ngroups; ++g) {
    const T *vt = static_cast<const T *>(D->vel) + (size_t)g * kNumVelFields * kLanes;
    const double v1 = vt[kV1 * kLanes + lane], v2 = vt[kV2 * kLanes + lane];
    const double vsq = (double)vt[kE2m1 * kLanes + lane] + 1.0;
    const double z = (double)static_cast<const T *>(D->h)[((size_t)g * ncell + cell) * kLanes + lane];
    const double h = (double)static_cast<const T *>(D->h_fwd)[((size_t)g * ncell + cell) * kLanes + lane] - s;
    const double M = a[0] + a[1] * v1 + a[2] * v2 + a[3] * vsq;
    gsum += z * (M - c - h);
    qsum += z * (D->flow_axis ? v2 : v1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gsum += __shfl_xor_sync(0xffffffffu, gsum, o);
    qsum += __shfl_xor_sync(0xffffffffu, qsum, o);
  }
  if (lane == 0) {
    D->grad[cell] = gsum;
    atomicAdd(&D->state->Q, D->force * qsum);
  }
}

}  // namespace

cudaError_t launch_adjoint_finalize(const LaunchDesc &L, int fin_blocks, int seam_blocks, bool fp64, cudaStream_t stream) {
  if (seam_blocks > 0) {
    if (fp64) aseam_kernel<double><<<seam_blocks, kBlock, 0, stream>>>(L.inst);
    else aseam_kernel<float><<<seam_blocks, kBlock, 0, stream>>>(L.inst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  afin1_kernel<<<fin_blocks, kBlock, 0, stream>>>(L.inst);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fp64) afin2_kernel<double><<<fin_blocks, kBlock, 0, stream>>>(L.inst);
  else afin2_kernel<float><<<fin_blocks, kBlock, 0, stream>>>(L.inst);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_reset(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream) {
  const int blocks = (ncell + kBlock - 1) / kBlock < 1024 ? (ncell + kBlock - 1) / kBlock : 1024;
  if (fp64) areset_kernel<double><<<blocks, kBlock, 0, stream>>>(adj_dev);
  else areset_kernel<float><<<blocks, kBlock, 0, stream>>>(adj_dev);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gradient(const InstanceDesc *adj_dev, int ncell, bool fp64, cudaStream_t stream) {
  const int blocks = (int)(((long long)ncell * 32 + kBlock - 1) / kBlock);
  if (fp64) agrad_kernel<double><<<blocks, kBlock, 0, stream>>>(adj_dev);
  else agrad_kernel<float><<<blocks, kBlock, 0, stream>>>(adj_dev);
  return cudaGetLastError();
}

}  // namespace dvm
