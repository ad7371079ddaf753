// dvm_finalize.cuh -- per-cell pieces of the finalize step shared by the per-sweep kernels
// (dvm_finalize.cu) and the persistent batched kernel (dvm_persist.cu).  Loads of data that other
// thread blocks of the same launch write (accumulators, fluxes, the instance state) go through L2
// (__ldcg), so that a persistent kernel never reads a stale L1 line.
#pragma once
#include <cmath>
#include <cstdint>

#include "dvm_device.cuh"

namespace dvm {

struct alignas(32) Dbl4 {
  double x, y, z, w;
};

// Write the sweep record of one cell and quadrant: right-hand-side coefficients (already in the record's
// precision), the upwind coefficients of the cell's stencil classes and the wall terms 2 h_w of
// wall-class axes.
template <typename T>
__device__ __forceinline__ void store_rec(SweepRec<T> *dst, T A, T B, T C, T Dd, double hwx, double hwy,
                                          uint32_t code, T delta);
template <>
__device__ __forceinline__ void store_rec<float>(SweepRec<float> *dst, float A, float B, float C, float Dd,
                                                 double hwx, double hwy, uint32_t code, float delta) {
  const int clx = (code >> kClsXShift) & 3, cly = (code >> kClsYShift) & 3;
  const bool solid = (code & kSolid) != 0;
  SweepRec<float> r;
  r.A = solid ? 0.f : A;
  r.B = solid ? 0.f : B;
  r.C = solid ? 0.f : C;
  r.D = solid ? 0.f : Dd;
  r.ax1 = solid ? 0.f : class_a1(clx);
  r.ax2 = solid ? 0.f : class_a2(clx);
  r.xw = (!solid && clx == kWall) ? (float)(2.0 * hwx) : 0.f;
  r.ay1 = solid ? 0.f : class_a1(cly);
  r.ay2 = solid ? 0.f : class_a2(cly);
  r.yw = (!solid && cly == kWall) ? (float)(2.0 * hwy) : 0.f;
  r.code = code;
  r.delta = delta;
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
  const double *gi = D->ginv;
  double a[4];
  if (D->ginv_sparse) {
    a[0] = gi[0] * m[0] + gi[3] * m[3];
    a[1] = gi[5] * m[1];
    a[2] = gi[10] * m[2];
    a[3] = gi[12] * m[0] + gi[15] * m[3];
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      a[i] = gi[i * 4] * m[0] + gi[i * 4 + 1] * m[1] + gi[i * 4 + 2] * m[2] + gi[i * 4 + 3] * m[3];
  }
  // R = delta (a0 + a1 v1 + a2 v2 + a3 |v|^2 - c) + F v_flow in the basis 1, v1, v2, |v|^2 - 1; the
  // coefficients are shared by the four quadrants and rounded to the record's precision once
  const T A = static_cast<T>(d * (a[0] + a[3] - c));
  const T B = static_cast<T>(d * a[1] + (D->flow_axis ? 0.0 : D->force));
  const T Cc = static_cast<T>(d * a[2] + (D->flow_axis ? D->force : 0.0));
  const T Dd = static_cast<T>(d * a[3]);
  const T dt = static_cast<T>(d);
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
        hw[ax] = (__ldcg(fcur + src) - s * D->ain[side] + corr) * D->wnrm[side];
      } else {
        hw[ax] = 0.0;
      }
    }
    store_rec<T>(rec + (size_t)q * ncell + cell, A, B, Cc, Dd, hw[0], hw[1], D->code4[(size_t)cell * 4 + q], dt);
    // the diagonal-major copy only feeds the column sweep (rebuilt by sync_diag when a launch
    // switches to it)
    if (diag && D->rec_diag)
      store_rec<T>(static_cast<SweepRec<T> *>(D->rec_diag) + q * diag_quadrant_size(D->nx, D->ny) +
                       diag_slot(D->nx, D->ny, cell % D->nx, cell / D->nx, (q & 1) != 0, (q & 2) != 0),
                   A, B, Cc, Dd, hw[0], hw[1], D->code4[(size_t)cell * 4 + q], dt);
  }
}

// The finalize of one gas or solid cell after a sweep: shifted moments (plus the correction phase's
// rho), the records of the next sweep, the cell's terms of the stopping test (|du|, |u|, u dA) and a
// NaN check, and the cleared flux slot of the next sweep.  s = the mass shift of this sweep, c_new the
// accumulated shift, fcur / fnext the flux arrays of this and the next sweep.
template <typename T>
__device__ __forceinline__ void fin2_cell(const InstanceDesc *D, int cell, double s, double c_new, const double *fcur,
                                          double *fnext, const double *rho_in, bool diag, double &du, double &ua,
                                          double &uq, double &bad) {
  const uint32_t code0 = D->code4[(size_t)cell * 4];
  if (!(code0 & kSolid)) {
    Dbl4 *acc4 = reinterpret_cast<Dbl4 *>(D->acc);
    const double *accd = D->acc + (size_t)cell * 4;
    const Dbl4 am{__ldcg(accd), __ldcg(accd + 1), __ldcg(accd + 2), __ldcg(accd + 3)};
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
    write_records<T>(D, cell, rho, u1, u2, tau, c_new, s, fcur, rho_in, diag);
    const double uf = D->flow_axis ? u2 : u1;  // velocity along the flow
    du = fabs(uf - __ldcg(D->u1prev + cell));
    ua = fabs(uf);
    uq = D->xwidth ? uf * D->xwidth[cell % D->nx] : uf;  // area-weighted for unequal columns
    D->u1prev[cell] = uf;
    if (!isfinite(rho) || !isfinite(u1) || !isfinite(u2) || !isfinite(tau)) bad = 1.0;
  }
  reinterpret_cast<Dbl4 *>(fnext)[cell] = Dbl4{0.0, 0.0, 0.0, 0.0};
}

// Correction phase of the refinement: the seam part of rho goes into the raw seam values the next
// sweep reads (this sweep has written them; the next one subtracts the pending shift from raw + rho).
// Elements e0, e0 + stride, ... of [seam_x | seam_y].
template <typename T>
__device__ __forceinline__ void seam_inject(const InstanceDesc *D, size_t e0, size_t stride) {
  const size_t nsx = D->periodic_x ? (size_t)D->ngroups * D->ny * 2 * kLanes : 0;
  const size_t nsy = D->periodic_y ? (size_t)D->ngroups * D->nx * 2 * kLanes : 0;
  for (size_t e = e0; e < nsx + nsy; e += stride) {
    T *dst = e < nsx ? static_cast<T *>(D->seam_x) + e : static_cast<T *>(D->seam_y) + (e - nsx);
    const T add = e < nsx ? static_cast<const T *>(D->rho_seam_x)[e] : static_cast<const T *>(D->rho_seam_y)[e - nsx];
    *dst = __ldcg(dst) + add;
  }
}

// The stopping test after a sweep (one thread, after every cell's terms are summed): eps_n, the rate
// estimate, the FP32 noise-floor exit, the mixed-iteration estimate, limits and failure flags; stores
// the new iteration count, shifts, eps, est, Q, the status and finally the done flag.
__device__ __forceinline__ void stop_test(const InstanceDesc *D, DeviceState *st, double dsum, double usum, double qsum,
                                          double c_new, double s) {
  // (the state is read through L2: in the persistent launch an earlier test may have run on another SM)
  const int n = __ldcg(&st->iter) + 1;
  const double eps = usum > 0.0 ? dsum / usum : 0.0;
  const double back = __ldcg(&st->eps_ring[n & 3]);  // eps_{n-4}
  st->eps_ring[n & 3] = eps;
  double est = INFINITY;
  int done = 0, status = 0;
  if (D->aa) {
    // mixed iterates (FP64 storage only): the estimate from the plain residual (dvm_anderson.cu).
    // Near the rounding floor the residual stops falling while rho keeps the estimate above a
    // tight tol: below tol, 32 sweeps without a 10 % smaller residual also end the iteration.
    est = __ldcg(&st->aa_est);
    const double res = __ldcg(&st->aa_res);
    if (n >= 5 && est < st->tol) done = 1;
    if (res < 0.9 * __ldcg(&st->aa_res_min)) {
      st->aa_res_min = res;
      st->aa_iter_min = n;
    }
    if (!done && n >= 5 && res < st->tol && n - __ldcg(&st->aa_iter_min) >= 32) done = 1;
  } else {
    if (n >= 5) {
      double r = back > 0.0 ? pow(eps / back, 0.25) : 0.0;
      if (r > 0.9999) r = 0.9999;
      est = eps / (1.0 - r);
      if (est < st->tol) done = 1;
    }
    // With FP32 storage the change per sweep stalls at the rounding noise floor, where the rate
    // estimate says nothing: below tol, 16 sweeps without a new smallest eps also end the iteration.
    if (eps < __ldcg(&st->eps_min)) {
      st->eps_min = eps;
      st->iter_min = n;
    }
    if (!done && D->fp32 && n >= 5 && eps < st->tol && n - __ldcg(&st->iter_min) >= 16) done = 1;
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
  st->status = status;
  __threadfence();
  st->done = done;
}

}  // namespace dvm
