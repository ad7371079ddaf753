// dvm_sweep_cols.cuh -- the transport sweep with one thread per grid column (the "column" sweep),
// shared by the FP32 and FP64, forward and adjoint translation units.
//
// It computes exactly the update of the row-wavefront sweep (dvm_sweep.cuh): Eq. (iteration) of
// arXiv:1704.03126 (Sec. II.A) with second-order upwind differences, lagged periodic seams and the
// diffuse wall values of the previous iterate, fused with the moments and incident wall fluxes.
// Only the mapping differs.  A thread owns one column p of the grid (in the quadrant's sweep order)
// and G velocities of the block's velocity set, and walks down its column one row per step: at step S
// it updates cell (p, S - p), so the block advances along the anti-diagonals of the quadrant.  Every
// upstream value is one or two steps old:
//   y: h(p, q-1) and h(p, q-2) are the thread's own last two results (registers);
//   x: h(p-1, q) and h(p-2, q) were written one and two steps ago by threads p-1 and p-2 into a
//      3-deep shared-memory ring; one block barrier per step orders them.
// The G velocities of a thread are independent, so the arithmetic runs on velocity pairs (packed
// FP32x2 FMAs in FP32), and the cell's record is read once for G updates.  The V threads of a block
// that share a column hold different velocities; their moment and wall-flux sums are combined with
// warp shuffles and added to the FP64 accumulators with one atomic per value.  There are no
// spin-waits: the only synchronisation is the per-step barrier, which every thread reaches.
#pragma once
#include <cstdint>

#include "dvm_device.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace cols {

template <typename T>
struct Vec;
template <>
struct Vec<float> {
  using T2 = float2;
  using V16 = float4;  // 16-byte shared-memory vector: two velocity pairs
  __device__ static __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
  __device__ static __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
  __device__ static __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
  __device__ static __forceinline__ float2 splat(float x) { return make_float2(x, x); }
  __device__ static __forceinline__ float2 rcp2(float2 d) { return make_float2(1.0f / d.x, 1.0f / d.y); }
  __device__ static __forceinline__ float2 pair(const float4 &v, int i) {
    return i ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
  }
  __device__ static __forceinline__ float4 pack(const float2 *p) { return make_float4(p[0].x, p[0].y, p[1].x, p[1].y); }
};
template <>
struct Vec<double> {
  using T2 = double2;
  using V16 = double2;  // one velocity pair
  __device__ static __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
  }
  __device__ static __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
  __device__ static __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static __forceinline__ double2 splat(double x) { return make_double2(x, x); }
  __device__ static __forceinline__ double2 rcp2(double2 d) { return make_double2(1.0 / d.x, 1.0 / d.y); }
  __device__ static __forceinline__ double2 pair(const double2 &v, int) { return v; }
  __device__ static __forceinline__ double2 pack(const double2 *p) { return p[0]; }
};

// velocities per thread: 8 in FP32 (4 packed pairs), 4 in FP64
template <typename T>
struct ColsG {
  static constexpr int value = sizeof(T) == 4 ? 8 : 4;
};

// per-pair constant fields in shared memory ([VB / 2][kCstFields] pairs): v1, v2, |v|^2 - 1, |v1|/dx,
// |v2|/dy, the moment weight w (W forward, 1 on real lanes for the adjoint), the adjoint's W, and
// the products w v1, w v2, w (|v|^2 - 1) that let FP64 accumulate each moment with one FMA
enum : int { kCV1 = 0, kCV2, kCE, kCCx, kCCy, kCWm, kCWr, kCWv1, kCWv2, kCWe, kCPad0, kCPad1, kCstFields };
static_assert(kCstFields == kColsCstFields, "shared-memory layout");

template <typename T>
__host__ __device__ inline ColsSmemLayout layout(int V, int ncol) {
  constexpr int G = ColsG<T>::value;
  return cols_smem_layout(V, G, ncol, (int)sizeof(T));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(static_cast<unsigned>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// TMA bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completing on bar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// ADJ = false: the forward sweep.  ADJ = true: the transposed sweep of the adjoint iteration (see
// dvm_sweep.cuh): reversed traversal, transposed weights t1, t2 from the record, right-hand side
// W (A + B v1 + C v2 + D (|v|^2 - 1)) + |v1| W TX + |v2| W TY, unweighted moments, and
// 2 |v_a|/dx z added to the wall adjoint flux of cells whose upstream neighbour is solid.
template <typename T, bool ADJ, bool UNIF, int V, bool SPEC>
__global__ void __launch_bounds__(kColsMaxThreads, 1) cols_kernel(LaunchDesc L) {
  using Q = Vec<T>;
  using T2 = typename Q::T2;
  using V16 = typename Q::V16;
  constexpr int G = ColsG<T>::value;
  constexpr int CPW = kLanes / V;                 // columns per warp
  constexpr int NP = G / 2;                       // velocity pairs per thread
  constexpr int VB = V * G;                       // velocities per block
  constexpr int NQ = G * (int)sizeof(T) / 16;     // 16-byte vectors per thread and column
  constexpr int PPQ = 16 / (2 * (int)sizeof(T));  // pairs per 16-byte vector
  constexpr int DEPTH = sizeof(T) == 4 ? 5 : 4;    // = cols_depth: record stages in flight
  constexpr int SR = kColsSeamRows;                // rows of the staged x-seam ring (> DEPTH + 1)
  static_assert(SR >= DEPTH + 2, "a staged seam row must outlive the two steps that read it");
  static_assert(4 % V == 0, "V divides the four moments");

  const int map = L.sweep_map[blockIdx.x];
  const InstanceDesc *__restrict__ D = L.inst + (map >> 16);
  const int g = map & 0xfff, sub = (map >> 12) & 0xf;
  DeviceState *st = D->state;
  if (*reinterpret_cast<volatile int *>(&st->done)) return;

  const int nx = D->nx, ny = D->ny, ncell = D->ncell;
  const bool px = D->periodic_x != 0, py = D->periodic_y != 0;
  const int quad = g / D->groups_per_quadrant;
  const bool xneg = ((quad & 1) != 0) != ADJ, yneg = ((quad & 2) != 0) != ADJ;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int v = lane / CPW;                       // velocity subset of this thread
  const int p = w * CPW + (lane % CPW);           // column in sweep order
  const int ncol = (blockDim.x >> 5) * CPW;
  const int l0 = sub * VB + v * G;                // first velocity lane (within the group)

  extern __shared__ __align__(16) unsigned char smem[];
  const ColsSmemLayout SL = layout<T>(V, ncol);
  T *cstT = reinterpret_cast<T *>(smem + SL.cst);
  const T2 *cst = reinterpret_cast<const T2 *>(smem + SL.cst);
  T *invt = reinterpret_cast<T *>(smem + SL.inv);
  V16 *ring = reinterpret_cast<V16 *>(smem + SL.ring);
  SweepRec<T> *recs = reinterpret_cast<SweepRec<T> *>(smem + SL.recs);  // [DEPTH][ncol]
  T *xsr = reinterpret_cast<T *>(smem + SL.xseam);  // [SR][2][VB]: seam columns (nx-2, nx-1) of row q
  T *ysr = reinterpret_cast<T *>(smem + SL.yseam);  // [V][ncol][2][G]: seam rows (ny-2, ny-1) of column p
  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + SL.mbar);  // [DEPTH] completion of each record stage
  int *abort_flag = reinterpret_cast<int *>(smem + SL.mbar + DEPTH * sizeof(uint64_t));

  for (size_t b = threadIdx.x; b < SL.total / 16; b += blockDim.x)
    reinterpret_cast<float4 *>(smem)[b] = make_float4(0.f, 0.f, 0.f, 0.f);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // before TMA writes to the same bytes
  __syncthreads();
  {
    const T *vt = static_cast<const T *>(D->vel) + (size_t)g * kNumVelFields * kLanes + sub * VB;
    for (int t = threadIdx.x; t < VB * kCstFields; t += blockDim.x) {
      const int vl = t % VB, f = t / VB;
      const int wm = ADJ ? kZ0 : kW0;
      T val;
      if (f == kCWv1) val = vt[wm * kLanes + vl] * vt[kV1 * kLanes + vl];
      else if (f == kCWv2) val = vt[wm * kLanes + vl] * vt[kV2 * kLanes + vl];
      else if (f == kCWe) val = vt[wm * kLanes + vl] * vt[kE2m1 * kLanes + vl];
      else if (f >= kCPad0) val = T(0);
      else {
        const int fld = f == kCV1 ? kV1 : f == kCV2 ? kV2 : f == kCE ? kE2m1 : f == kCCx ? kCx : f == kCCy ? kCy
                      : f == kCWm ? wm : kW0;
        val = vt[fld * kLanes + vl];
      }
      cstT[((vl >> 1) * kCstFields + f) * 2 + (vl & 1)] = val;
    }
    if (UNIF) {
      const T *iv = static_cast<const T *>(D->inv_den) + (size_t)g * kInvRows * kLanes + sub * VB;
      for (int t = threadIdx.x; t < kInvRows * VB; t += blockDim.x) invt[t] = iv[(t / VB) * kLanes + t % VB];
    }
  }
  __syncthreads();

  const T sshift = ADJ ? T(0) : static_cast<T>(st->s);
  const T dx = static_cast<T>(D->dx), dy = static_cast<T>(D->dy);
  const SweepRec<T> *__restrict__ rec = static_cast<const SweepRec<T> *>(D->rec) + (size_t)quad * ncell;
  T *seamx = static_cast<T *>(D->seam_x) + (size_t)g * ny * 2 * kLanes + l0;
  T *seamy = static_cast<T *>(D->seam_y) + (size_t)g * nx * 2 * kLanes + l0;
  T *hout = D->h ? static_cast<T *>(D->h) + (size_t)g * ncell * kLanes + l0 : nullptr;
  double *acc = D->acc;
  double *facc = D->facc + (size_t)((st->iter + 1) & 1) * ncell * 4;
  const int sidex = xneg ? kW : kE;
  const int sidey = yneg ? kS : kN;
  // accommodation < 1: the wall value of a wall-class cell gains (1 - alpha) times the previous
  // sweep's value of the mirrored velocity at the same face, written by the mirrored quadrant's block
  // at its incident cells; double-buffered by sweep parity.  The transposed sweep swaps the roles:
  // wall-class cells write z, and a cell owning the (forward) downstream face adds (1 - alpha) 2 |v_a|/dx
  // times the mirrored velocity's z of the last transposed sweep to its right-hand side.
  const bool spec = SPEC && D->alpha < 1.0;
  // a moving plate beyond the last row (Couette flow, Eq. diffuse1): its wall value alpha (rho_w +
  // 2 U v1) adds 4 alpha U v1 to the y combination of the cells under it (forward only)
  const T top_term = static_cast<T>(4.0 * D->alpha * D->top_u);
  const T one_m_alpha2 = static_cast<T>(2.0 * (1.0 - D->alpha));
  // Columns of unequal width (the caller's rows of Sec. II.A stored transposed).  The x stencil of a
  // column k is the derivative at its centre of the polynomial through the points the class uses,
  // widths w relative to dx: upstream centre distances d1 = (w_k + w_u1)/2 and d2 = d1 + (w_u1 + w_u2)/2;
  // interior kappa = 1/d1 + 1/d2 with weights d2/(d1 (d2 - d1)) on h(u1) and -d1/(d2 (d2 - d1)) on
  // h(u2); first order kappa = weight = 1/d1; next to a wall (face at w_k/2) kappa = 2/w_k, the wall
  // terms (2 alpha rho_w, the specular part, the plate's drift) times 1/w_k.  The transposed sweep has
  // the same diagonal; its cell c pulls z of the forward-downstream columns d1, d2 with the forward
  // weights of d1 (on its u1 = c) and of d2 (on its u2 = c).
  const bool nux = SPEC && D->xwidth != nullptr;
  T nk_full = T(1.5), na1_full = T(2), na2_full = T(-0.5), nk_near = T(1), nwsc = T(1);
  T ta1_full = T(2), ta1_near = T(1), ta2_full = T(-0.5);
  if (nux && p < nx) {
    const int i = xneg ? nx - 1 - p : p;
    const int sf = (xneg != ADJ) ? -1 : 1;  // forward direction: the forward upstream of column k is k - sf
    // a column beyond a closed x end belongs to a cell whose stencil does not use it: read `k` instead
    auto col = [&](int c, int k) { return (c >= 0 && c < nx) ? c : (px ? ((c % nx) + nx) % nx : k); };
    struct Stencil {
      double k_full, a1, a2, k_near, wsc;
    };
    auto stencil = [&](int k) {
      const double w0 = D->xwidth[k], w1 = D->xwidth[col(k - sf, k)], w2 = D->xwidth[col(k - 2 * sf, k)];
      const double d1 = 0.5 * (w0 + w1), d2 = d1 + 0.5 * (w1 + w2);
      return Stencil{1.0 / d1 + 1.0 / d2, d2 / (d1 * (d2 - d1)), -d1 / (d2 * (d2 - d1)), 1.0 / d1, 1.0 / w0};
    };
    const Stencil s0 = stencil(i);
    nk_full = static_cast<T>(s0.k_full);
    na1_full = static_cast<T>(s0.a1);
    na2_full = static_cast<T>(s0.a2);
    nk_near = static_cast<T>(s0.k_near);
    nwsc = static_cast<T>(s0.wsc);
    if (ADJ) {
      const Stencil s1 = stencil(col(i + sf, i)), s2 = stencil(col(i + 2 * sf, i));
      ta1_full = static_cast<T>(s1.a1);
      ta1_near = static_cast<T>(s1.k_near);
      ta2_full = static_cast<T>(s2.a2);
    }
  }
  const int gi = g % D->groups_per_quadrant, gq = D->groups_per_quadrant;
  T *wbuf_wr = nullptr;
  const T *wbuf_rd = nullptr;
  if (spec) {
    const size_t half = (size_t)D->nwall * 2 * gq * kLanes;
    wbuf_wr = static_cast<T *>(D->wbuf) + (size_t)((st->iter + 1) & 1) * half;
    wbuf_rd = static_cast<const T *>(D->wbuf) + (size_t)(st->iter & 1) * half;
  }
  // face record of (slot, sign of the other velocity component, group within quadrant, lanes)
  auto wface = [&](int slot, int sgn) -> size_t { return ((size_t)(slot * 2 + sgn) * gq + gi) * kLanes + l0; };
  const int nsteps = nx + ny - 1;
  const T2 zero2 = Q::splat(T(0));

  auto ring_at = [&](int slot, int col, int kq) -> V16 * {
    return ring + ((size_t)(slot * V + v) * NQ + kq) * ncol + col;
  };
  auto load_vec = [&](const T *src, T2 (&dst)[NP], T shift) {
#pragma unroll
    for (int kq = 0; kq < NQ; ++kq) {
      const V16 x = *reinterpret_cast<const V16 *>(src + kq * (16 / (int)sizeof(T)));
#pragma unroll
      for (int u = 0; u < PPQ; ++u) dst[kq * PPQ + u] = Q::add2(Q::pair(x, u), Q::splat(-shift));
    }
  };
  auto store_vec = [&](T *dst, const T2 (&src)[NP]) {
#pragma unroll
    for (int kq = 0; kq < NQ; ++kq) *reinterpret_cast<V16 *>(dst + kq * (16 / (int)sizeof(T))) = Q::pack(src + kq * PPQ);
  };

  // Nothing a step reads comes straight from global memory.  The records of the cells the block
  // reaches at step S are contiguous in the diagonal-major record array (one anti-diagonal of the
  // quadrant); one thread copies them, and for a periodic x axis the previous sweep's seam values of
  // row S (read by columns 0 and 1), into stage S % DEPTH with TMA bulk copies that complete on that
  // stage's mbarrier, DEPTH - 1 steps ahead.  At the end of step S the same thread waits for stage
  // S + 1, and the step's block barrier publishes it to every thread.  The y-seam values of every
  // column are copied (cp.async) before the first step.
  constexpr int SEGS = G * (int)sizeof(T) / 16;  // 16-byte pieces of one thread's G values
  const SweepRec<T> *__restrict__ rdiag =
      static_cast<const SweepRec<T> *>(D->rec_diag) + (size_t)quad * diag_quadrant_size(nx, ny);
  const T *seamx_blk = static_cast<const T *>(D->seam_x) + (size_t)g * ny * 2 * kLanes + sub * VB;
  const bool leader = threadIdx.x == 0;
  auto issue = [&](int S, int slot) {  // leader only
    unsigned bytes = 0;
    int p_lo = 0, count = 0;
    if (S < nsteps) {
      p_lo = max(0, S - (ny - 1));
      count = min(nx - 1, S) - p_lo + 1;
      bytes = (unsigned)(count * sizeof(SweepRec<T>));
      if (px && S < ny) bytes += 2u * VB * sizeof(T);
    }
    // the stage's previous contents were read with ordinary loads before the last block barrier
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    mbar_arrive_expect_tx(&mbar[slot], bytes);
    if (count > 0) {
      bulk_g2s(recs + (size_t)slot * ncol + p_lo, rdiag + (size_t)S * nx + p_lo,
               (unsigned)(count * sizeof(SweepRec<T>)), &mbar[slot]);
      if (px && S < ny) {
        const int j = yneg ? ny - 1 - S : S;
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
          bulk_g2s(xsr + (size_t)((S % SR) * 2 + sl) * VB, seamx_blk + (size_t)(j * 2 + sl) * kLanes,
                   (unsigned)(VB * sizeof(T)), &mbar[slot]);
      }
    }
  };
  // bounded wait of the leader for stage S; false if it did not complete
  auto wait_stage = [&](int S, int slot) -> bool {
    const unsigned parity = (unsigned)(S / DEPTH) & 1u;
    for (int spin = 0; spin < kColsSpinLimit; ++spin)
      if (mbar_try_wait(&mbar[slot], parity)) return true;
    return false;
  };
  if (leader) {
    for (int s = 0; s < DEPTH; ++s) mbar_init(&mbar[s], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (py && p < nx) {
    const int i = xneg ? nx - 1 - p : p;
    T *dst = ysr + (size_t)(v * ncol + p) * 2 * G;
#pragma unroll
    for (int sl = 0; sl < 2; ++sl)
#pragma unroll
      for (int b = 0; b < SEGS; ++b)
        cp_async16(dst + sl * G + b * (16 / (int)sizeof(T)),
                   seamy + (size_t)(i * 2 + sl) * kLanes + b * (16 / (int)sizeof(T)));
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  if (leader) {
    for (int s = 0; s < DEPTH - 1; ++s) issue(s, s);
    if (!wait_stage(0, 0)) {
      *abort_flag = 1;
      atomicExch(&st->err_flag, 1);
      for (int s = 1; s < DEPTH - 1; ++s) wait_stage(s, s);
    }
  }
  __syncthreads();
  if (*abort_flag) return;

  // one step: hy1 holds h(p, q-1), hy2 holds h(p, q-2); the new h(p, q) replaces hy2
  // ring slots of steps S, S-1, S-2 and the record stage of step S (rotated, not recomputed)
  int r0 = 0, r1 = 2, r2 = 1, sd = 0;
  auto step = [&](T2 (&hy1)[NP], T2 (&hy2)[NP], const int S) {
    const int q = S - p;
    const bool active = p < nx && q >= 0 && q < ny;
    if (leader) issue(S + DEPTH - 1, sd == 0 ? DEPTH - 1 : sd - 1);  // the stage of step S - 1
    if (__any_sync(0xffffffffu, active)) {
      const int j = yneg ? ny - 1 - q : q, i = xneg ? nx - 1 - p : p;
      const int cell = j * nx + i;
      uint32_t code = kSolid;
      T m0 = T(0), m1 = T(0), m2 = T(0), m3 = T(0);
      if (active) {
        const SweepRec<T> r = recs[sd * ncol + p];
        code = r.code;
        T ax1, ax2, ay1, ay2, xw = T(0), yw = T(0);
        if constexpr (sizeof(T) == 4) {
          ax1 = r.ax1;
          ax2 = r.ax2;
          ay1 = r.ay1;
          ay2 = r.ay2;
        } else if constexpr (!ADJ) {
          const int clx = (code >> kClsXShift) & 3, cly = (code >> kClsYShift) & 3;
          const bool solid = (code & kSolid) != 0;
          ax1 = solid ? T(0) : T(class_a1(clx));
          ax2 = solid ? T(0) : T(class_a2(clx));
          ay1 = solid ? T(0) : T(class_a1(cly));
          ay2 = solid ? T(0) : T(class_a2(cly));
        } else {
          ax1 = T((code >> kAdjT1XShift) & 3);
          ax2 = (code & kAdjT2X) ? T(-0.5) : T(0);
          ay1 = T((code >> kAdjT1YShift) & 3);
          ay2 = (code & kAdjT2Y) ? T(-0.5) : T(0);
        }
        if (!ADJ) {
          xw = r.xw;
          yw = r.yw;
        }
        T xsc = T(1);  // scale of the x wall terms (unequal columns)
        if (ADJ && nux && !(code & kSolid)) {
          const uint32_t t1c = (code >> kAdjT1XShift) & 3u;
          ax1 = t1c == 2u ? ta1_full : (t1c == 1u ? ta1_near : T(0));
          ax2 = (code & kAdjT2X) ? ta2_full : T(0);
          xsc = nwsc;
        } else if (nux && !(code & kSolid)) {
          const int clx = (code >> kClsXShift) & 3;
          if (clx == kFull) {
            ax1 = na1_full;
            ax2 = na2_full;
          } else if (clx == kNear) {
            ax1 = nk_near;
            ax2 = T(0);
          } else {
            ax1 = T(0);
            ax2 = T(0);
            xsc = nwsc;
            xw *= xsc;
          }
        }
        if (q == 0) {
          if (py) {
            const T *ys = ysr + (size_t)(v * ncol + p) * 2 * G;
            load_vec(ys + G, hy1, sshift);
            load_vec(ys, hy2, sshift);
          } else {
#pragma unroll
            for (int k = 0; k < NP; ++k) hy1[k] = hy2[k] = zero2;
          }
        }
        T2 u1[NP], u2[NP];
        const int s0 = r0, s1 = r1, s2 = r2;
        const T *xs = xsr + (size_t)(q % SR) * 2 * VB + v * G;  // staged seam of this row (columns 0, 1)
        if (p >= 2) {
#pragma unroll
          for (int kq = 0; kq < NQ; ++kq) {
            const V16 a = *ring_at(s1, p - 1, kq), b = *ring_at(s2, p - 2, kq);
#pragma unroll
            for (int u = 0; u < PPQ; ++u) {
              u1[kq * PPQ + u] = Q::pair(a, u);
              u2[kq * PPQ + u] = Q::pair(b, u);
            }
          }
        } else {
          // column 0 reads the previous sweep's columns nx-1, nx-2 (slots 1, 0); column 1 reads
          // column 0 of this sweep and slot 1
          if (p == 1) {
#pragma unroll
            for (int kq = 0; kq < NQ; ++kq) {
              const V16 a = *ring_at(s1, 0, kq);
#pragma unroll
              for (int u = 0; u < PPQ; ++u) u1[kq * PPQ + u] = Q::pair(a, u);
            }
          } else if (px) {
            load_vec(xs + VB, u1, sshift);
          } else {
#pragma unroll
            for (int k = 0; k < NP; ++k) u1[k] = zero2;
          }
          if (px) {
            load_vec(xs + p * VB, u2, sshift);
          } else {
#pragma unroll
            for (int k = 0; k < NP; ++k) u2[k] = zero2;
          }
        }
        if (spec && !(code & kSolid)) {
          // forward: wall-class cells read the mirrored velocity's incident value; transposed: cells
          // owning the forward downstream face read the mirrored velocity's z at that face
          const bool rdx = ADJ ? (code & kIncX) != 0 : ((code >> kClsXShift) & 3u) == (uint32_t)kWall;
          const bool rdy = ADJ ? (code & kIncY) != 0 : ((code >> kClsYShift) & 3u) == (uint32_t)kWall;
          if (rdx) {
            const int slot = D->wall_slot[(size_t)cell * 4 + (xneg ? kE : kW)];
            if (slot >= 0) {  // always: every wall-class face has a slot
              load_vec(wbuf_rd + wface(slot, (quad >> 1) & 1), u1, sshift);
              ax1 = one_m_alpha2 * xsc;  // x combination 2 alpha rho_w + 2 (1 - alpha) h(mirror v)
            }
          }
          if (rdy) {
            const int slot = D->wall_slot[(size_t)cell * 4 + (yneg ? kN : kS)];
            if (slot >= 0) {
              // h(p, q-1) lies in a solid cell here, so its register is free; the next cell reads it
              // only with a zero coefficient
              load_vec(wbuf_rd + wface(slot, quad & 1), hy1, sshift);
              ay1 = one_m_alpha2;
            }
          }
        }
        // moving plate (set only on gas cells whose upstream wall along that axis is the plate): the
        // reflected drift 2 U v_t along the plate, v_t = v1 for a plate beyond the last row, v2 for
        // one beyond the last column (an instance stored transposed)
        T mwy = T(0), mwx = T(0);
        if constexpr (SPEC && !ADJ) {
          if (code & kTopWall) mwy = top_term;
          if (code & kTopWallX) mwx = top_term * xsc;
        }
        const T2 smwy = Q::splat(mwy), smwx = Q::splat(mwx);
        const T2 sA = Q::splat(r.A), sB = Q::splat(r.B), sC = Q::splat(r.C), sD = Q::splat(r.D);
        const T2 sax1 = Q::splat(ax1), sax2 = Q::splat(ax2), say1 = Q::splat(ay1), say2 = Q::splat(ay2);
        const T2 sxw = Q::splat(xw), syw = Q::splat(yw);
        const T2 stx = Q::splat(ADJ ? T(r.xw) * dx : T(0)), sty = Q::splat(ADJ ? T(r.yw) * dy : T(0));
        const int irow = (code >> kInvShift) & 15;
        T2 skx = zero2, sky = zero2, sdl = zero2;
        if (!UNIF) {
          const int clx = (code >> kClsXShift) & 3, cly = (code >> kClsYShift) & 3;
          if (nux) skx = Q::splat(clx == kFull ? nk_full : (clx == kNear ? nk_near : T(2) * nwsc));
          else skx = Q::splat(clx == kFull ? T(1.5) : (clx == kNear ? T(1.0) : T(2.0)));
          sky = Q::splat(cly == kFull ? T(1.5) : (cly == kNear ? T(1.0) : T(2.0)));
          sdl = Q::splat(T(r.delta));
        }
        T2 M0 = zero2, M1 = zero2, M2 = zero2, M3 = zero2;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          const T2 *c = cst + (size_t)((v * NP + k) * kCstFields);
          const T2 cv1 = c[kCV1], cv2 = c[kCV2], ce = c[kCE], ccx = c[kCCx], ccy = c[kCCy], cwm = c[kCWm];
          T2 Rk = Q::fma2(sD, ce, Q::fma2(sC, cv2, Q::fma2(sB, cv1, sA)));
          if (ADJ) Rk = Q::mul2(c[kCWr], Q::fma2(ccx, stx, Q::fma2(ccy, sty, Rk)));
          const T2 by = Q::fma2(say1, hy1[k], Q::fma2(say2, hy2[k], (SPEC && !ADJ) ? Q::fma2(smwy, cv1, syw) : syw));
          const T2 bx = Q::fma2(sax1, u1[k], Q::fma2(sax2, u2[k], (SPEC && !ADJ) ? Q::fma2(smwx, cv2, sxw) : sxw));
          T2 iv;
          if (UNIF) iv = *reinterpret_cast<const T2 *>(invt + irow * VB + v * G + 2 * k);
          else iv = Q::rcp2(Q::fma2(ccx, skx, Q::fma2(ccy, sky, sdl)));
          const T2 h = Q::mul2(Q::fma2(ccx, bx, Q::fma2(ccy, by, Rk)), iv);
          hy2[k] = h;
          if constexpr (sizeof(T) == 8) {
            // FP64 is bound by the FMA pipe: one FMA per moment with the premultiplied weights
            M0 = Q::fma2(cwm, h, M0);
            M1 = Q::fma2(c[kCWv1], h, M1);
            M2 = Q::fma2(c[kCWv2], h, M2);
            M3 = Q::fma2(c[kCWe], h, M3);
          } else {
            const T2 wh = Q::mul2(cwm, h);
            M0 = Q::add2(M0, wh);
            M1 = Q::fma2(cv1, wh, M1);
            M2 = Q::fma2(cv2, wh, M2);
            M3 = Q::fma2(ce, wh, M3);
          }
        }
#pragma unroll
        for (int kq = 0; kq < NQ; ++kq) *ring_at(s0, p, kq) = Q::pack(hy2 + kq * PPQ);
        m0 = M0.x + M0.y;
        m1 = M1.x + M1.y;
        m2 = M2.x + M2.y;
        m3 = (M3.x + M3.y) + m0;  // sum w |v|^2 h = sum w (|v|^2 - 1) h + sum w h
        if (hout) store_vec(hout + (size_t)cell * kLanes, hy2);
        if (px && p >= nx - 2) store_vec(seamx + (size_t)(j * 2 + (p - (nx - 2))) * kLanes, hy2);
        if (py && q >= ny - 2) store_vec(seamy + (size_t)(i * 2 + (q - (ny - 2))) * kLanes, hy2);
      }
#pragma unroll
      for (int off = CPW; off < kLanes; off <<= 1) {
        m0 += __shfl_xor_sync(0xffffffffu, m0, off);
        m1 += __shfl_xor_sync(0xffffffffu, m1, off);
        m2 += __shfl_xor_sync(0xffffffffu, m2, off);
        m3 += __shfl_xor_sync(0xffffffffu, m3, off);
      }
      if (active && !(code & kSolid)) {
#pragma unroll
        for (int t = 0; t < 4 / V; ++t) {
          const int mi = v + t * V;
          const T val = mi == 0 ? m0 : (mi == 1 ? m1 : (mi == 2 ? m2 : m3));
          red_add(&acc[(size_t)cell * 4 + mi], static_cast<double>(val));
        }
      }
      // forward: incident flux sum |v_n| W h at cells owning a downstream wall face; adjoint: the
      // transposed wall reads, sum 2 |v_a|/dx z at cells whose upstream neighbour is solid
      bool fxf, fyf;
      if (ADJ) {
        fxf = active && !(code & kSolid) && ((code >> kClsXShift) & 3u) == (uint32_t)kWall;
        fyf = active && !(code & kSolid) && ((code >> kClsYShift) & 3u) == (uint32_t)kWall;
      } else {
        fxf = active && (code & kIncX) != 0;
        fyf = active && (code & kIncY) != 0;
      }
      if (__any_sync(0xffffffffu, fxf || fyf)) {
        T fx = T(0), fy = T(0);
        if (fxf || fyf) {
          T2 ax = zero2, ay = zero2;
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            const T2 *c = cst + (size_t)((v * NP + k) * kCstFields);
            const T2 wh = ADJ ? hy2[k] : Q::mul2(c[kCWm], hy2[k]);
            ax = Q::fma2(c[kCCx], wh, ax);
            ay = Q::fma2(c[kCCy], wh, ay);
          }
          fx = fxf ? (ax.x + ax.y) : T(0);
          fy = fyf ? (ay.x + ay.y) : T(0);
        }
#pragma unroll
        for (int off = CPW; off < kLanes; off <<= 1) {
          fx += __shfl_xor_sync(0xffffffffu, fx, off);
          fy += __shfl_xor_sync(0xffffffffu, fy, off);
        }
        // (|v_a|/d_a) W h summed, times d_a: the incident flux sum |v_a| W h
        const T scx = ADJ ? T(2) * nwsc : dx, scy = ADJ ? T(2) : dy;
        if (v == 0 && fxf) red_add(&facc[(size_t)cell * 4 + sidex], static_cast<double>(fx * scx));
        if (v == 0 && fyf) red_add(&facc[(size_t)cell * 4 + sidey], static_cast<double>(fy * scy));
        if (spec && fxf) {
          const int slot = D->wall_slot[(size_t)cell * 4 + sidex];
          if (slot >= 0) store_vec(wbuf_wr + wface(slot, (quad >> 1) & 1), hy2);
        }
        if (spec && fyf) {
          const int slot = D->wall_slot[(size_t)cell * 4 + sidey];
          if (slot >= 0) store_vec(wbuf_wr + wface(slot, quad & 1), hy2);
        }
      }
    }
    if (leader && S + 1 < nsteps && !wait_stage(S + 1, sd + 1 == DEPTH ? 0 : sd + 1)) *abort_flag = 1;
    __syncthreads();
    const int t = r2;
    r2 = r1;
    r1 = r0;
    r0 = t;
    sd = sd + 1 == DEPTH ? 0 : sd + 1;
  };

  T2 ha[NP], hb[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) ha[k] = hb[k] = zero2;
  int S = 0;
  for (; S < nsteps; S += 2) {
    step(ha, hb, S);  // h -> hb
    if (*abort_flag) break;
    if (S + 1 < nsteps) step(hb, ha, S + 1);
    if (*abort_flag) break;
  }
  if (*abort_flag && leader) {
    // a stage never completed: report it and wait (bounded) for the copies still in flight
    atomicExch(&st->err_flag, 1);
    for (int s2 = S + 1; s2 < min(nsteps, S + DEPTH + 1); ++s2) wait_stage(s2, s2 % DEPTH);
  }
}

template <typename T, bool ADJ, bool UNIF, int V, bool SPEC>
cudaError_t launch(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  auto kern = cols_kernel<T, ADJ, UNIF, V, SPEC>;
  const int ncol = L.warps * (kLanes / V);
  const size_t smem = layout<T>(V, ncol).total;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, L.warps * kLanes, smem, stream>>>(L);
  return cudaGetLastError();
}

template <typename T, bool ADJ, bool UNIF, bool SPEC>
cudaError_t launch_vs(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  switch (L.cols_v) {
    case 1: return launch<T, ADJ, UNIF, 1, SPEC>(L, nblocks, stream);
    case 2: return launch<T, ADJ, UNIF, 2, SPEC>(L, nblocks, stream);
    case 4: return launch<T, ADJ, UNIF, 4, SPEC>(L, nblocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

// SPEC: some instance of the launch has partially specular walls, a moving plate or columns of unequal
// width
template <typename T, bool ADJ, bool UNIF>
cudaError_t launch_v(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  if (L.specular) return launch_vs<T, ADJ, UNIF, true>(L, nblocks, stream);
  return launch_vs<T, ADJ, UNIF, false>(L, nblocks, stream);
}

}  // namespace cols
}  // namespace dvm
