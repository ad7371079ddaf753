// dvm_sweep.cu -- the transport sweep of one source iteration (the hot path).
//
// For every discrete velocity, Eq. (iteration) of arXiv:1704.03126 (Sec. II.A) is solved over all
// gas cells with second-order upwind differences:
//     (delta + sum_a |v_a|/dx kappa_a) h = R + sum_a |v_a|/dx combo_a,
//     R = delta (rho + 2 u.v + tau (|v|^2 - 1) - c) + F v1                    (Eq. BGK)
// where along each axis (s = sign v_a, u1 = cell - s, u2 = cell - 2 s)
//     interior            kappa = 3/2, combo = 2 h(u1) - h(u2)/2   (second order)
//     u2 solid            kappa = 1,   combo = h(u1)               (first order)
//     u1 solid            kappa = 2,   combo = 2 h_w(own face)     (linear through the wall value)
// h_w is the diffuse wall value (Eq. diffuse2) of the previous iterate, and upstream cells across a
// periodic seam also take the previous iterate (lagged).
//
// GB300 mapping.  One thread block sweeps one group of 32 velocities of one quadrant (one velocity
// per lane, so every lane walks the cells in the same order and all branches are warp-uniform).
// Its R warps are rows in flight of a skewed wavefront: row q processes column chunk c (C = nx/R
// cells) at step q + c, so rows q-1 and q-2 finished that chunk one and two steps earlier.  Each
// warp writes its row into a 3-deep shared-memory ring that the next two rows read; one block
// barrier per step.  Per-cell records (right-hand-side coefficients, wall values, stencil classes)
// are staged into shared memory with cp.async one step ahead.  Moments are reduced per chunk from
// the ring (FP32 or FP64 sums over the 32 lanes) and accumulated across groups in FP64 atomics;
// incident wall fluxes likewise.  h itself is only written to HBM at the periodic seams (and when
// the distribution is kept).
#include <cstdint>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T kappa_of(int cls) {
  return cls == kFull ? T(1.5) : (cls == kNear ? T(1.0) : T(2.0));
}

template <typename T>
__device__ __forceinline__ T recip(T x) {
  return T(1) / x;
}
template <>
__device__ __forceinline__ double recip<double>(double x) {
  return __drcp_rn(x);
}

template <typename T, bool STORE_H, bool UNIF, int NSTAGE, bool STAGE_SEAM>
__global__ void __launch_bounds__(kMaxWarps * kLanes, 1) sweep_kernel(LaunchDesc L) {
  const int map = L.sweep_map[blockIdx.x];
  const InstanceDesc *__restrict__ D = L.inst + (map >> 16);
  const int g = map & 0xffff;
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;

  const int nx = D->nx, ny = D->ny;
  const bool px = D->periodic_x != 0, py = D->periodic_y != 0;
  const int quad = g / D->groups_per_quadrant;
  const bool xneg = (quad & 1) != 0, yneg = (quad & 2) != 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = L.warps;
  const int C = (nx + R - 1) / R;  // columns per chunk of this instance
  const int Cl = L.cmax;           // layout stride shared by the launch

  extern __shared__ __align__(16) unsigned char smem[];
  const SweepSmemLayout SL = sweep_smem_layout(R, Cl, sizeof(T), sizeof(SweepRec<T>), NSTAGE, STAGE_SEAM);
  T *ring = reinterpret_cast<T *>(smem + SL.ring);
  SweepRec<T> *stage = reinterpret_cast<SweepRec<T> *>(smem + SL.stage);
  T *seamst = reinterpret_cast<T *>(smem + SL.seam);
  T *invt = reinterpret_cast<T *>(smem + SL.inv);
  T *wts = reinterpret_cast<T *>(smem + SL.wts);

  const T *vt = static_cast<const T *>(D->vel) + (size_t)g * kNumVelFields * kLanes;
  const T v1 = vt[kV1 * kLanes + lane], v2 = vt[kV2 * kLanes + lane], em1 = vt[kE2m1 * kLanes + lane];
  const T cx = vt[kCx * kLanes + lane], cy = vt[kCy * kLanes + lane];
  const T wnx = vt[kWnx * kLanes + lane], wny = vt[kWny * kLanes + lane];
  if (UNIF) {
    const T *iv = static_cast<const T *>(D->inv_den) + (size_t)g * 9 * kLanes;
    for (int i = threadIdx.x; i < 9 * kLanes; i += blockDim.x) invt[i] = iv[i];
  }
  for (int i = threadIdx.x; i < 4 * kLanes; i += blockDim.x)
    wts[(i >> 5) * kRingPad + (i & 31)] = vt[(kW0 + (i >> 5)) * kLanes + (i & 31)];

  const T sshift = static_cast<T>(st->s);
  const int ncell = D->ncell;
  const SweepRec<T> *__restrict__ rec = static_cast<const SweepRec<T> *>(D->rec) + (size_t)quad * ncell;
  T *seamx = static_cast<T *>(D->seam_x) + (size_t)g * ny * 2 * kLanes;
  T *seamy = static_cast<T *>(D->seam_y) + (size_t)g * nx * 2 * kLanes;
  T *hout = STORE_H ? static_cast<T *>(D->h) + (size_t)g * ncell * kLanes : nullptr;
  double *acc = D->acc;
  double *facc = D->facc + (size_t)((st->iter + 1) & 1) * ncell * 4;
  const int sidex = xneg ? kW : kE;  // wall side hit by this quadrant's velocities along x
  const int sidey = yneg ? kS : kN;
  __syncthreads();

  // row (in sweep order) and chunk of this warp at step t
  auto row_chunk = [&](int t, int &q, int &c) -> bool {
    const int rel = t - w;
    if (rel < 0) return false;
    q = w + R * (rel / R);
    c = rel % R;
    return q < ny && c * C < nx;
  };

  // stage the records (and wrapped seam rows) of the chunk processed at step t
  auto issue = [&](int t) {
    int q, c;
    if (row_chunk(t, q, c)) {
      const int j = yneg ? ny - 1 - q : q;
      SweepRec<T> *sdst = stage + ((size_t)w * NSTAGE + (t % NSTAGE)) * Cl;
      const int p0 = c * C;
      const int cnt = min(C, nx - p0);
      for (int l = lane; l < cnt; l += kLanes) {
        const int p = p0 + l;
        const int i = xneg ? nx - 1 - p : p;
        const char *src = reinterpret_cast<const char *>(rec + (size_t)j * nx + i);
        char *dst = reinterpret_cast<char *>(sdst + l);
#pragma unroll
        for (int b = 0; b < (int)sizeof(SweepRec<T>); b += 16) cp_async16(dst + b, src + b);
      }
      if (STAGE_SEAM && py && q < 2) {
        // row 0 reads rows ny-1, ny-2 (seam slots 1, 0); row 1 reads row ny-1 (slot 1) as h(u2)
        T *sd = seamst + ((size_t)(w & 1) * NSTAGE + (t % NSTAGE)) * 2 * Cl * kLanes;
        for (int l = 0; l < cnt; ++l) {
          const int p = p0 + l;
          const int i = xneg ? nx - 1 - p : p;
          const T *s0 = seamy + (size_t)i * 2 * kLanes + lane;
          if (q == 0) {
            cp_async_small<sizeof(T)>(sd + (size_t)l * kLanes + lane, s0 + kLanes);
            cp_async_small<sizeof(T)>(sd + (size_t)(Cl + l) * kLanes + lane, s0);
          } else {
            cp_async_small<sizeof(T)>(sd + (size_t)(Cl + l) * kLanes + lane, s0 + kLanes);
          }
        }
      }
    }
    cp_async_commit();
  };

  // sweep one chunk; MODE 0: upstream rows from shared memory (ring or staged seam rows);
  // MODES 1 and 2 (FP64 path, rows 0 and 1 of a periodic y axis): the wrapped upstream rows are read
  // from the global seam buffer (pointers already offset by the lane)
  T hp1 = T(0), hp2 = T(0);
  auto run_chunk = [&](auto mode_tag, int q, int c, const SweepRec<T> *rs, T *myr, const T *pr1, long ps1,
                       const T *pr2, long ps2) {
    constexpr int MODE = decltype(mode_tag)::value;
    const int j = yneg ? ny - 1 - q : q;
    if (c == 0) {
      if (px) {
        const T *sx = seamx + (size_t)j * 2 * kLanes + lane;
        hp1 = sx[kLanes] - sshift;  // column nx-1 in sweep order
        hp2 = sx[0] - sshift;       // column nx-2
      } else {
        hp1 = T(0);
        hp2 = T(0);
      }
    }
    const int p0 = c * C;
    const int cnt = min(C, nx - p0);
    for (int l = 0; l < cnt; ++l) {
      const int p = p0 + l;
      const int i = xneg ? nx - 1 - p : p;
      const SweepRec<T> r = rs[l];
      T h = T(0);
      if (!(r.code & kSolid)) {
        T hq1, hq2;
        if (MODE == 0) {  // both upstream rows in shared memory
          hq1 = pr1[l * ps1 + lane];
          hq2 = pr2[l * ps2 + lane];
        } else if (MODE == 1) {  // both upstream rows across the periodic seam (global, lagged)
          hq1 = pr1[l * ps1] - sshift;
          hq2 = pr2[l * ps2] - sshift;
        } else {  // h(u1) in shared memory, h(u2) across the seam
          hq1 = pr1[l * ps1 + lane];
          hq2 = pr2[l * ps2] - sshift;
        }
        const T Rk = fma(r.D, em1, fma(r.C, v2, fma(r.B, v1, r.A)));
        const int clx = (r.code >> kClsXShift) & 3, cly = (r.code >> kClsYShift) & 3;
        const T bx = clx == kFull ? fma(T(2), hp1, T(-0.5) * hp2) : (clx == kNear ? hp1 : T(2) * r.hwx);
        const T by = cly == kFull ? fma(T(2), hq1, T(-0.5) * hq2) : (cly == kNear ? hq1 : T(2) * r.hwy);
        T inv;
        if (UNIF) {
          inv = invt[(clx * 3 + cly) * kLanes + lane];
        } else {
          inv = recip<T>(r.delta + cx * kappa_of<T>(clx) + cy * kappa_of<T>(cly));
        }
        h = fma(cx, bx, fma(cy, by, Rk)) * inv;
        if (r.code & kIncX) {
          const T f = warp_sum<T>(wnx * h);
          if (lane == 0) atomicAdd(&facc[((size_t)j * nx + i) * 4 + sidex], static_cast<double>(f));
        }
        if (r.code & kIncY) {
          const T f = warp_sum<T>(wny * h);
          if (lane == 0) atomicAdd(&facc[((size_t)j * nx + i) * 4 + sidey], static_cast<double>(f));
        }
        if (STORE_H) hout[((size_t)j * nx + i) * kLanes + lane] = h;
      }
      hp2 = hp1;
      hp1 = h;
      myr[l * kRingPad + lane] = h;
      if (px && p >= nx - 2) seamx[((size_t)j * 2 + (p - (nx - 2))) * kLanes + lane] = h;
      if (py && q >= ny - 2) seamy[((size_t)i * 2 + (q - (ny - 2))) * kLanes + lane] = h;
    }
    // moments of the chunk: pair (cell l, moment m) per lane, sum over the 32 velocities
    __syncwarp();
    for (int pr = lane; pr < cnt * 4; pr += kLanes) {
      const int l = pr >> 2, m = pr & 3;
      if (!(rs[l].code & kSolid)) {
        const T *hr = myr + l * kRingPad;
        const T *wr = wts + m * kRingPad;
        T sum = T(0);
#pragma unroll
        for (int k = 0; k < kLanes; ++k) sum = fma(wr[k], hr[k], sum);
        const int p = p0 + l;
        const int i = xneg ? nx - 1 - p : p;
        atomicAdd(&acc[((size_t)j * nx + i) * 4 + m], static_cast<double>(sum));
      }
    }
  };

  const int nsteps = ny + R - 1;
  if (NSTAGE == 2) issue(0);
  for (int t = 0; t < nsteps; ++t) {
    if (NSTAGE == 2) {
      issue(t + 1);
      cp_async_wait<1>();
    } else {
      issue(t);
      cp_async_wait<0>();
    }
    __syncwarp();
    int q, c;
    if (row_chunk(t, q, c)) {
      const SweepRec<T> *rs = stage + ((size_t)w * NSTAGE + (t % NSTAGE)) * Cl;
      T *myr = ring + ((size_t)w * 3 + (t % 3)) * Cl * kRingPad;
      const T *pr1 = ring + ((size_t)((w + R - 1) % R) * 3 + ((t + 2) % 3)) * Cl * kRingPad;
      const T *pr2 = ring + ((size_t)((w + 2 * R - 2) % R) * 3 + ((t + 1) % 3)) * Cl * kRingPad;
      if (py && q < 2) {
        if (STAGE_SEAM) {
          T *sd = seamst + ((size_t)(w & 1) * NSTAGE + (t % NSTAGE)) * 2 * Cl * kLanes;
          const int cnt = min(C, nx - c * C);
          // the staged seam values are the previous iterate before its mass shift
          if (q == 0)
            for (int l = 0; l < cnt; ++l) sd[(size_t)l * kLanes + lane] -= sshift;
          for (int l = 0; l < cnt; ++l) sd[(size_t)(Cl + l) * kLanes + lane] -= sshift;
          __syncwarp();
          if (q == 0) {
            run_chunk(std::integral_constant<int, 0>(), q, c, rs, myr, sd, kLanes, sd + (size_t)Cl * kLanes,
                      kLanes);
          } else {
            run_chunk(std::integral_constant<int, 0>(), q, c, rs, myr, pr1, kRingPad, sd + (size_t)Cl * kLanes,
                      kLanes);
          }
        } else {
          const int p0 = c * C;
          const int i0 = xneg ? nx - 1 - p0 : p0;
          const long stride = xneg ? -2L * kLanes : 2L * kLanes;
          const T *s0 = seamy + (size_t)i0 * 2 * kLanes + lane;
          if (q == 0) {
            run_chunk(std::integral_constant<int, 1>(), q, c, rs, myr, s0 + kLanes, stride, s0, stride);
          } else {
            // h(u1) is row 0 (shared memory, read with lane offset below), h(u2) the seam row ny-1
            run_chunk(std::integral_constant<int, 2>(), q, c, rs, myr, pr1, kRingPad, s0 + kLanes, stride);
          }
        }
      } else {
        run_chunk(std::integral_constant<int, 0>(), q, c, rs, myr, pr1, kRingPad, pr2, kRingPad);
      }
    }
    __syncthreads();
  }
}

template <typename T, bool STORE_H, bool UNIF>
cudaError_t launch_t(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  constexpr bool F64 = sizeof(T) == 8;
  constexpr int NSTAGE = F64 ? 1 : 2;
  constexpr bool STAGE_SEAM = !F64;
  auto kern = sweep_kernel<T, STORE_H, UNIF, NSTAGE, STAGE_SEAM>;
  const size_t smem = sweep_smem_layout(L.warps, L.cmax, sizeof(T), sizeof(SweepRec<T>), NSTAGE, STAGE_SEAM).total;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, L.warps * kLanes, smem, stream>>>(L);
  return cudaGetLastError();
}

}  // namespace

size_t sweep_smem_bytes(bool fp64, int warps, int cmax) {
  return fp64 ? sweep_smem_layout(warps, cmax, 8, sizeof(SweepRec<double>), 1, 0).total
              : sweep_smem_layout(warps, cmax, 4, sizeof(SweepRec<float>), 2, 1).total;
}

cudaError_t launch_sweep(bool fp64, bool store_h, bool uniform_delta, const LaunchDesc &L, int nblocks,
                         cudaStream_t stream) {
  if (fp64) {
    if (store_h) return uniform_delta ? launch_t<double, true, true>(L, nblocks, stream)
                                      : launch_t<double, true, false>(L, nblocks, stream);
    return uniform_delta ? launch_t<double, false, true>(L, nblocks, stream)
                         : launch_t<double, false, false>(L, nblocks, stream);
  }
  if (store_h) return uniform_delta ? launch_t<float, true, true>(L, nblocks, stream)
                                    : launch_t<float, true, false>(L, nblocks, stream);
  return uniform_delta ? launch_t<float, false, true>(L, nblocks, stream)
                       : launch_t<float, false, false>(L, nblocks, stream);
}

}  // namespace dvm
