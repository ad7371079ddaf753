// dvm_sweep.cuh -- the transport sweep of one source iteration (the hot path), shared by the FP32
// and FP64 translation units.
//
// For every discrete velocity, Eq. (iteration) of arXiv:1704.03126 (Sec. II.A) is solved over all
// gas cells with upwind differences:
//     (delta + sum_a |v_a|/dx kappa_a) h = R + sum_a |v_a|/dx combo_a,
//     R = delta (a0 + a1 v1 + a2 v2 + a3 |v|^2 - c) + F v1                     (Eq. BGK)
// where along each axis (s = sign v_a, u1 = cell - s, u2 = cell - 2 s)
//     interior            kappa = 3/2, combo = 2 h(u1) - h(u2)/2   (second order)
//     u2 solid            kappa = 1,   combo = h(u1)               (first order)
//     u1 solid            kappa = 2,   combo = 2 h_w(own face)     (linear through the wall value)
// h_w is the diffuse wall value (Eq. diffuse2) of the previous iterate, and upstream cells across a
// periodic seam also take the previous iterate (lagged).
//
// GB300 mapping.  One thread block sweeps one group of 32 velocities of one quadrant (a velocity per
// lane: every lane walks the cells in the same order, so all branches are warp-uniform).  Its R
// warps are rows in flight of a wavefront: row q (in sweep order) goes through column chunks of CW
// cells, chunk c at "step" q + c, and warp w owns rows w, w + R, ...  A warp writes its rows into a
// 3-deep shared-memory ring that the next two rows read.  There is no block-wide barrier: each warp
// publishes the steps it has finished in a shared progress word and waits (bounded spins) only for
//   - the warp of row q-1 to have finished the same chunk (then row q-2 has too), and
//   - the warp of row q+2 to have read the ring slot this step overwrites.
// Per-cell records (right-hand-side coefficients, wall values, stencil classes) are staged into
// shared memory with cp.async one chunk ahead (FP32) or at the start of the chunk (FP64).  The
// moments and incident wall fluxes of each finished chunk are sums over the 32 lanes read back from
// the ring -- an m16n8k8 TF32 tensor-core contraction in FP32, per-lane dot products in FP64 -- and
// are accumulated across groups with FP64 atomics.
// h itself goes to HBM only at the periodic seams (and when the distribution is kept).
#pragma once
#include <climits>
#include <cstdint>
#include <algorithm>
#include <type_traits>

#include "dvm_device.cuh"
#include "dvm_kernels.h"

namespace dvm {
namespace sweep {

constexpr int kSpinLimit = 1 << 22;  // bounded waits: about 0.1-1 s before the kernel gives up

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
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];\n" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.cta.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// All lanes of the warp spin until *p >= need; false when the spin limit ran out.
__device__ __forceinline__ bool wait_at_least(const int *p, int need) {
  int spins = 0;
  while (ld_acquire(p) < need) {
    if (++spins > kSpinLimit) return false;
    if (spins > 64) __nanosleep(32);
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Dot product over the 32 velocities of a group (FP64 sweep): h values of one cell (a ring row) with one
// weight row, both in shared memory.
template <typename T, int RS>
__device__ __forceinline__ T dot32(const T *hr, const T *wr) {
  T sum = T(0);
#pragma unroll
  for (int k = 0; k < kLanes; ++k) sum = fma(wr[k], hr[k], sum);
  return sum;
}

// FP32 per-cell sums on the tensor cores.  The h values of a finished chunk sit in the ring as a
// CW x 32 tile (cell x velocity); the four moments and the two wall fluxes of every cell are that tile
// times a 32 x 6 weight matrix, a small dense contraction: one m16n8k8 TF32 mma per 8 velocities, with
// each FP32 operand split into a TF32 head and a TF32 tail (hi*hi + hi*lo + lo*hi, error a few FP32
// ulps of the products).  ldmatrix reads the tile once (16 cells x 32 velocities = 16 shared-memory
// wavefronts); the weights stay in registers as B fragments.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// B fragments of the weight matrix B[k][n] = weight row n (0-5; 6, 7 zero) at velocity k of the group:
// for k-step s, lane (n = lane / 4, t = lane % 4) holds B[8 s + t][n] and B[8 s + t + 4][n], each as
// TF32 head and tail: bf[s] = {hi0, hi1, lo0, lo1}.
template <int RS>
__device__ __forceinline__ void weight_fragments(const float *wts, int lane, uint32_t (&bf)[4][4]) {
  const int n = lane >> 2, t = lane & 3;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float w = n < kSweepWtsRows ? wts[n * RS + 8 * s + t + 4 * e] : 0.f;
      const uint32_t hi = tf32_rna(w);
      bf[s][e] = hi;
      bf[s][2 + e] = tf32_rna(w - __uint_as_float(hi));
    }
  }
}
// d = the tile times the weights.  `base`: this lane's ldmatrix row address for k-step 0 (lanes
// 8 m .. 8 m + 7 address the rows of matrix m: cells 0-7 / 8-15 of the chunk (rows past the chunk
// repeat its last cell) at velocities 0-3 / 4-7 of the k-step).  Lane (g = lane / 4, t = lane % 4)
// gets columns 2t, 2t+1 of cells g (d0, d1) and g + 8 (d2, d3).
__device__ __forceinline__ void cell_sums_mma(uint32_t base, const uint32_t (&bf)[4][4], float (&d)[4]) {
  d[0] = d[1] = d[2] = d[3] = 0.f;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    uint32_t a[4], ah[4], al[4];
    ldsm_x4(base + s * 32, a);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // head: x rounded to TF32 (round half away from zero on the bit pattern); tail: the exact
      // remainder, which the mma truncates to TF32
      ah[i] = (a[i] + 0x1000u) & 0xffffe000u;
      al[i] = __float_as_uint(__uint_as_float(a[i]) - __uint_as_float(ah[i]));
    }
    mma_tf32(d, al, bf[s][0], bf[s][1]);
    mma_tf32(d, ah, bf[s][2], bf[s][3]);
    mma_tf32(d, ah, bf[s][0], bf[s][1]);
  }
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

template <typename T>
struct Traits;
template <>
struct Traits<float> {
  static constexpr int kStages = 2;       // records staged one chunk ahead
  static constexpr bool kStageSeams = true;
  static constexpr int kRingStride = 36;  // 16-byte rows: vector loads in the moment dot products
};
template <>
struct Traits<double> {
  static constexpr int kStages = 1;       // shared memory is needed by the 8-byte ring
  static constexpr bool kStageSeams = false;
  static constexpr int kRingStride = 33;  // odd stride: conflict-free column reads
};

template <typename T>
__host__ __device__ inline SweepSmemLayout layout(int warps, int cw, int ntile = 1) {
  return sweep_smem_layout(warps, cw, (int)sizeof(T), (int)sizeof(SweepRec<T>), Traits<T>::kStages,
                           Traits<T>::kStageSeams ? 1 : 0, Traits<T>::kRingStride, ntile);
}

// ADJ = false: the forward sweep.  ADJ = true: the transposed sweep of the adjoint iteration --
// cells are visited in the reverse order (the forward order of the opposite quadrant), each pulls
// from its forward-downstream cells with the transposed weights t1, t2, the right-hand side is
// W (A + B v1 + C v2 + D (|v|^2 - 1)) + |v1| W TX + |v2| W TY, the moments are the unweighted sums
// of (1, v1, v2, |v|^2) z, and cells next to a wall add 2 |v_a|/dx z to that wall's adjoint flux.
//
// sweep_tile is one block's share of a sweep: the velocity group(s) named by the sweep-map entry `map`.
// PER = true: called from the persistent batched kernel (dvm_persist.cu), which hands out tiles of
// active instances only and whose blocks run many tiles: data written earlier in the same launch by
// other blocks (seams, the instance state) is read through L2, never from a possibly stale L1 line.
template <typename T, bool UNIF, int CW, bool ADJ, bool PER>
__device__ __forceinline__ void sweep_tile(const LaunchDesc &L, int map, unsigned char *smem, int Rb) {
  constexpr int NSTAGE = Traits<T>::kStages;
  constexpr bool STAGE_SEAM = Traits<T>::kStageSeams;
  constexpr int RS = Traits<T>::kRingStride;
  const InstanceDesc *__restrict__ D = L.inst + (map >> 16);
  DeviceState *st = D->state;
  if (!PER && *reinterpret_cast<volatile int *>(&st->done)) return;

  const int nx = D->nx, ny = D->ny, ncell = D->ncell;
  const bool px = D->periodic_x != 0, py = D->periodic_y != 0;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int R = (nx + CW - 1) / CW;         // rows in flight of this instance (host ensures R <= Rb)
  // A narrow grid leaves warps over: the block sweeps `ntile` consecutive groups side by side, group
  // g0 + j on warps [j R, (j + 1) R) with its own seam stages, 1/denominator table and weights.
  const int g0 = map & 0xfff;
  const int ntile = min(max((map >> 12) & 15, 1), D->ngroups - g0);
  const int wt = w / R, lw = w - wt * R, wb = wt * R;  // sub-tile, warp within it, its first warp
  const int g = g0 + wt;
  const int quad = min(g, D->ngroups - 1) / D->groups_per_quadrant;
  const bool xneg = ((quad & 1) != 0) != ADJ, yneg = ((quad & 2) != 0) != ADJ;

  const SweepSmemLayout SL = layout<T>(Rb, CW, L.row_tiles > 0 ? L.row_tiles : 1);
  T *ring = reinterpret_cast<T *>(smem + SL.ring);
  SweepRec<T> *stage = reinterpret_cast<SweepRec<T> *>(smem + SL.stage);
  T *seamst = reinterpret_cast<T *>(smem + SL.seam);
  T *invt_all = reinterpret_cast<T *>(smem + SL.inv);
  T *wts_all = reinterpret_cast<T *>(smem + SL.wts);
  int *prog = reinterpret_cast<int *>(smem + SL.prog);

  // zero the whole dynamic shared memory: ring slots and staged seam entries that are read before
  // (or without) being written are multiplied by zero coefficients and must not hold NaN patterns
  for (size_t b = threadIdx.x; b < SL.total / 16; b += (size_t)Rb * kLanes)
    reinterpret_cast<float4 *>(smem)[b] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  constexpr int kMom0 = ADJ ? kZ0 : kW0;  // moment weights: (W, W v1, W v2, W |v|^2) or (1, v1, v2, |v|^2)
  for (int j = 0; j < ntile; ++j) {
    const T *vtj = static_cast<const T *>(D->vel) + (size_t)(g0 + j) * kNumVelFields * kLanes;
    if (UNIF) {
      const T *iv = static_cast<const T *>(D->inv_den) + (size_t)(g0 + j) * kInvRows * kLanes;
      for (int i = threadIdx.x; i < kInvRows * kLanes; i += Rb * kLanes) invt_all[j * kInvRows * kLanes + i] = iv[i];
    }
    for (int i = threadIdx.x; i < 4 * kLanes; i += Rb * kLanes)
      wts_all[(j * kSweepWtsRows + (i >> 5)) * RS + (i & 31)] = vtj[(kMom0 + (i >> 5)) * kLanes + (i & 31)];
    // wall-flux weights: forward |v_n| W (incident flux), adjoint 2 |v_a| / dx (transposed wall read)
    for (int i = threadIdx.x; i < 2 * kLanes; i += Rb * kLanes) {
      const int ax = i >> 5, ln = i & 31;
      wts_all[(j * kSweepWtsRows + 4 + ax) * RS + ln] =
          ADJ ? T(2) * vtj[(ax ? kCy : kCx) * kLanes + ln] : vtj[(ax ? kWny : kWnx) * kLanes + ln];
    }
  }
  // progress word of warp w = number of steps known finished; the warp of local row lw starts at step lw
  for (int i = threadIdx.x; i < Rb; i += Rb * kLanes) prog[i] = i % R;
  __syncthreads();
  if (wt >= ntile) return;
  const T *vt = static_cast<const T *>(D->vel) + (size_t)g * kNumVelFields * kLanes;
  const T *invt_lane = invt_all + wt * kInvRows * kLanes + lane;
  const T *wts = wts_all + wt * kSweepWtsRows * RS;

  const T v1 = vt[kV1 * kLanes + lane], v2 = vt[kV2 * kLanes + lane], em1 = vt[kE2m1 * kLanes + lane];
  const T cx = vt[kCx * kLanes + lane], cy = vt[kCy * kLanes + lane];
  const T wnx = vt[kWnx * kLanes + lane], wny = vt[kWny * kLanes + lane];
  const T wl = vt[kW0 * kLanes + lane];
  const T cx2 = T(2) * cx, cxh = T(-0.5) * cx, cy2 = T(2) * cy, cyh = T(-0.5) * cy;  // FP64 class weights
  const T sshift = ADJ ? T(0) : static_cast<T>(__ldcg(&st->s));
  const SweepRec<T> *__restrict__ rec = static_cast<const SweepRec<T> *>(D->rec) + (size_t)quad * ncell;
  T *seamx = static_cast<T *>(D->seam_x) + (size_t)g * ny * 2 * kLanes;
  T *seamy = static_cast<T *>(D->seam_y) + (size_t)g * nx * 2 * kLanes;
  T *hout = D->h ? static_cast<T *>(D->h) + (size_t)g * ncell * kLanes : nullptr;
  double *acc = D->acc;
  double *facc = D->facc + (size_t)((__ldcg(&st->iter) + 1) & 1) * ncell * 4;
  const int sidex = xneg ? kW : kE;  // wall side hit by this quadrant's velocities along x
  const int sidey = yneg ? kS : kN;
  const int wprev = wb + (lw + R - 1) % R, wnext2 = wb + (lw + 2) % R;
  // FP32 per-cell sums (cell_sums_mma): the weight fragments, this lane's ldmatrix row in a ring slot,
  // and where its two result columns go -- lanes t = 0, 1: moments 2t, 2t+1; t = 2: the x and y wall
  // fluxes; t = 3: nothing -- each at the cells whose code satisfies (code & am) == cv
  uint32_t bfr[4][4];
  if constexpr (sizeof(T) == 4) weight_fragments<RS>(reinterpret_cast<const float *>(wts), lane, bfr);
  const int t4 = lane & 3, g4 = lane >> 2;
  const uint32_t ldsm_off =
      (uint32_t)((min((lane & 7) + 8 * ((lane >> 3) & 1), CW - 1) * RS + 4 * (lane >> 4)) * (int)sizeof(T));
  double *const red_base = t4 == 2 ? facc : acc;
  double *const red_p0 = red_base + (t4 == 2 ? sidex : 2 * t4);
  double *const red_p1 = red_base + (t4 == 2 ? sidey : 2 * t4 + 1);
  // moments: gas cells; forward fluxes: the cell owns a downstream wall face; adjoint fluxes: the
  // cell's class is "next to a wall" (upstream neighbour solid); lanes t = 3: never ((code & 0) == 1)
  uint32_t red_am0 = kSolid, red_cv0 = 0u, red_am1 = kSolid, red_cv1 = 0u;
  if (t4 == 2) {
    if (ADJ) {
      red_am0 = kSolid | (3u << kClsXShift);
      red_cv0 = (uint32_t)kWall << kClsXShift;
      red_am1 = kSolid | (3u << kClsYShift);
      red_cv1 = (uint32_t)kWall << kClsYShift;
    } else {
      red_am0 = red_cv0 = kIncX;
      red_am1 = red_cv1 = kIncY;
    }
  } else if (t4 == 3) {
    red_am0 = red_am1 = 0u;
    red_cv0 = red_cv1 = 1u;
  }

  // stage the records of chunk (q, c) into buffer `buf` (and, for rows 0 and 1 of a periodic y
  // axis, the wrapped seam rows); x-seam values of a new row are loaded into registers
  T pf_hp1 = T(0), pf_hp2 = T(0);
  // record staging of a full chunk: piece lane + 32 k (16 bytes) of the chunk's contiguous records goes
  // to byte st_dst[k] of the stage buffer
  constexpr int NPC = (int)sizeof(SweepRec<T>) / 16, NPIECE = NPC * CW, PPL = (NPIECE + kLanes - 1) / kLanes;
  int st_dst[PPL];
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int pc = lane + k * kLanes, r = pc / NPC, l = xneg ? CW - 1 - r : r;
    st_dst[k] = l * (int)sizeof(SweepRec<T>) + 16 * (pc - r * NPC);
  }
  auto issue = [&](int q, int c, int buf) {
    const int j = yneg ? ny - 1 - q : q;
    SweepRec<T> *sdst = stage + ((size_t)w * NSTAGE + buf) * CW;
    const int p0 = c * CW;
    const int cnt = min(CW, nx - p0);
    // the chunk's records are one contiguous run of cnt records in memory (cells i_lo .. i_lo + cnt - 1
    // of row j): the lanes copy consecutive 16-byte pieces of it (coalesced), each into the slot of its
    // record in sweep order
    const char *src = reinterpret_cast<const char *>(rec + j * nx + (xneg ? nx - p0 - cnt : p0));
    if (cnt == CW) {
#pragma unroll
      for (int k = 0; k < PPL; ++k)
        if (NPIECE % kLanes == 0 || lane + k * kLanes < NPIECE)
          cp_async16(reinterpret_cast<char *>(sdst) + st_dst[k], src + 16 * (lane + k * kLanes));
    } else {
      for (int pc = lane; pc < NPC * cnt; pc += kLanes) {
        const int r = pc / NPC, l = xneg ? cnt - 1 - r : r;
        cp_async16(reinterpret_cast<char *>(sdst + l) + 16 * (pc - r * NPC), src + 16 * pc);
      }
      if (lane >= cnt && lane < CW) {
        // past the ragged end of the row: a solid record (zero coefficients) sweeps to h = 0
        float4 *dst = reinterpret_cast<float4 *>(sdst + lane);
#pragma unroll
        for (int b = 0; b < NPC; ++b) dst[b] = make_float4(0.f, 0.f, 0.f, 0.f);
        sdst[lane].code = kSolid | (9u << kInvShift);
      }
    }
    if (STAGE_SEAM && py && q < 2) {
      // row 0 reads rows ny-1, ny-2 (seam slots 1, 0); row 1 reads row ny-1 (slot 1) as h(u2)
      T *sd = seamst + (((size_t)wt * 2 + (lw & 1)) * NSTAGE + buf) * 2 * CW * kLanes;
#pragma unroll
      for (int l = 0; l < CW; ++l) {
        if (l < cnt) {
          const int p = p0 + l;
          const int i = xneg ? nx - 1 - p : p;
          const T *s0 = seamy + i * 2 * kLanes + lane;
          if constexpr (PER) {
            // plain L2 loads (cp.async of 4 bytes would go through L1)
            if (q == 0) {
              sd[l * kLanes + lane] = __ldcg(s0 + kLanes);
              sd[(CW + l) * kLanes + lane] = __ldcg(s0);
            } else {
              sd[(CW + l) * kLanes + lane] = __ldcg(s0 + kLanes);
            }
          } else if (q == 0) {
            cp_async_small<sizeof(T)>(sd + l * kLanes + lane, s0 + kLanes);
            cp_async_small<sizeof(T)>(sd + (CW + l) * kLanes + lane, s0);
          } else {
            cp_async_small<sizeof(T)>(sd + (CW + l) * kLanes + lane, s0 + kLanes);
          }
        }
      }
    }
    if (c == 0 && px) {
      const T *sx = seamx + j * 2 * kLanes + lane;
      pf_hp1 = __ldcg(sx + kLanes);  // column nx-1 in sweep order (before its mass shift)
      pf_hp2 = __ldcg(sx);           // column nx-2
    }
    cp_async_commit();
  };

  // sweep one chunk.  MODE 0: upstream rows from shared memory (ring or staged seam rows);
  // MODES 1 and 2 (FP64, rows 0 and 1 of a periodic y axis): the wrapped upstream rows come from
  // the global seam buffer (pointers already offset by the lane)
  T hp1 = T(0), hp2 = T(0);
  T row_hp1 = T(0), row_hp2 = T(0);  // x-seam values of the current row, latched from pf_*
  auto run_chunk = [&](auto mode_tag, int q, int c, int t, const SweepRec<T> *rs, T *myr, const T *pr1, int ps1,
                       const T *pr2, int ps2) {
    constexpr int MODE = decltype(mode_tag)::value;
    const int j = yneg ? ny - 1 - q : q;
    if (c == 0) {
      hp1 = px ? row_hp1 - sshift : T(0);
      hp2 = px ? row_hp2 - sshift : T(0);
    }
    const int p0 = c * CW;
    const int cnt = min(CW, nx - p0);
    // The FP32 cell loop has no branches: stencil classes are coefficients in the records; solid cells
    // and the cells past a ragged row end have zero coefficients and sweep to h = 0.  Sub-chunks of
    // SUB cells run in two phases: first everything that does not depend on this row's x-recurrence
    // (records, the two upstream rows, the right-hand side, the y combination, 1/denominator) for all
    // SUB cells, so their shared-memory loads overlap; then the recurrence itself and the ring stores.
    // FP64 forward sweep (bound by the FP64 pipe): the stencil weights a_k of a cell's classes are
    // picked as per-lane products |v_a|/dx a_k (selects, no FP64 arithmetic), and the wall terms are
    // added only at wall-class cells (a warp-uniform branch: every lane visits the same cell), so an
    // interior update costs 3 FMA (right-hand side) + 4 FMA (upwind terms) + 1 MUL.
    constexpr bool FAST64 = sizeof(T) == 8 && !ADJ;
    constexpr int SUB = (sizeof(T) == 4) ? (CW < 8 ? CW : 8) : (CW < 2 ? CW : 2);
#pragma unroll
    for (int l0 = 0; l0 < CW; l0 += SUB) {
      T base[SUB], invv[SUB], cax1[SUB], cax2[SUB], cxw[SUB];
#pragma unroll
      for (int u = 0; u < SUB; ++u) {
        const int l = l0 + u;
        const SweepRec<T> r = rs[l];
        T hq1, hq2;
        if (MODE == 0) {
          hq1 = pr1[l * ps1 + lane];
          hq2 = pr2[l * ps2 + lane];
        } else if (MODE == 1) {
          hq1 = l < cnt ? __ldcg(pr1 + l * ps1) - sshift : T(0);
          hq2 = l < cnt ? __ldcg(pr2 + l * ps2) - sshift : T(0);
        } else {
          hq1 = pr1[l * ps1 + lane];
          hq2 = l < cnt ? __ldcg(pr2 + l * ps2) - sshift : T(0);
        }
        T Rk = fma(r.D, em1, fma(r.C, v2, fma(r.B, v1, r.A)));
        if constexpr (FAST64) {
          const int clx = (r.code >> kClsXShift) & 3, cly = (r.code >> kClsYShift) & 3;
          const bool solid = (r.code & kSolid) != 0;
          // class a1 = 2, 1, 0 and a2 = -1/2, 0, 0 (interior, second cell, next to a wall), times |v_a|/dx
          const T y1 = solid ? T(0) : (cly == kFull ? cy2 : (cly == kNear ? cy : T(0)));
          const T y2 = (!solid && cly == kFull) ? cyh : T(0);
          cax1[u] = solid ? T(0) : (clx == kFull ? cx2 : (clx == kNear ? cx : T(0)));
          cax2[u] = (!solid && clx == kFull) ? cxh : T(0);
          T b = fma(y1, hq1, fma(y2, hq2, Rk));
          if (!solid && cly == kWall) b = fma(cy, r.yw, b);
          if (!solid && clx == kWall) b = fma(cx, r.xw, b);
          base[u] = b;
          cxw[u] = T(0);
        } else {
          T ay1, ay2;
          if constexpr (sizeof(T) == 4) {
            cax1[u] = r.ax1;
            cax2[u] = r.ax2;
            ay1 = r.ay1;
            ay2 = r.ay2;
          } else {
            cax1[u] = T((r.code >> kAdjT1XShift) & 3);
            cax2[u] = (r.code & kAdjT2X) ? T(-0.5) : T(0);
            ay1 = T((r.code >> kAdjT1YShift) & 3);
            ay2 = (r.code & kAdjT2Y) ? T(-0.5) : T(0);
          }
          T by;
          if constexpr (ADJ) {
            // the incident-wall terms ride in the xw / yw slots of adjoint records
            Rk = fma(wnx, r.xw, fma(wny, r.yw, wl * Rk));
            cxw[u] = T(0);
            by = fma(ay1, hq1, ay2 * hq2);
          } else {
            cxw[u] = r.xw;
            by = fma(ay1, hq1, fma(ay2, hq2, r.yw));
          }
          base[u] = fma(cy, by, Rk);
        }
        if (UNIF) {
          // row (code >> kInvShift) & 15 of the table, as a byte offset: 128-byte rows (FP32), 256 (FP64)
          const uint32_t boff = (r.code & (15u << kInvShift)) << (sizeof(T) == 8 ? 1 : 0);
          invv[u] = *reinterpret_cast<const T *>(reinterpret_cast<const char *>(invt_lane) + boff);
        } else {
          const int clx = (r.code >> kClsXShift) & 3, cly = (r.code >> kClsYShift) & 3;
          invv[u] = recip<T>(r.delta + cx * kappa_of<T>(clx) + cy * kappa_of<T>(cly));
        }
      }
#pragma unroll
      for (int u = 0; u < SUB; ++u) {
        T h;
        if constexpr (FAST64) {
          h = fma(cax1[u], hp1, fma(cax2[u], hp2, base[u])) * invv[u];
        } else {
          const T bx = fma(cax1[u], hp1, fma(cax2[u], hp2, cxw[u]));
          h = fma(cx, bx, base[u]) * invv[u];
        }
        hp2 = hp1;
        hp1 = h;
        myr[(l0 + u) * RS + lane] = h;
      }
    }
    // The next rows need only the ring: publish this step now, so that the per-chunk passes below
    // (stored h, seams, wall fluxes, moments) stay off the wavefront's critical path.  The ring slot
    // is not rewritten before the consumer two rows down has read it (checked at step t + 3).
    __syncwarp();
    if (lane == 0) st_release(&prog[w], t + 1);
    __syncwarp();
    // per-chunk passes over the ring: stored distribution, seams, incident wall fluxes, moments
    if (hout) {
      for (int l = 0; l < cnt; ++l) {
        const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
        hout[(size_t)(j * nx + i) * kLanes + lane] = myr[l * RS + lane];
      }
    }
    if (px && p0 + cnt > nx - 2) {
      for (int p = max(p0, nx - 2); p < p0 + cnt; ++p)
        seamx[(j * 2 + (p - (nx - 2))) * kLanes + lane] = myr[(p - p0) * RS + lane];
    }
    if (py && q >= ny - 2) {
      for (int l = 0; l < cnt; ++l) {
        const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
        seamy[(i * 2 + (q - (ny - 2))) * kLanes + lane] = myr[l * RS + lane];
      }
    }
    if constexpr (sizeof(T) == 4) {
      // The six sums of every cell of the chunk on the tensor cores (four moments; forward: the
      // incident flux sum |v_n| W h at cells owning a downstream wall face; adjoint: the transposed
      // wall reads, sum 2 |v_a|/dx z at cells whose upstream neighbour is solid), added to the FP64
      // accumulators by the lanes holding them.
      float d[4];
      cell_sums_mma(smem_u32(myr) + ldsm_off, bfr, d);
      // element offset (cell * 4) of this lane's first cell, g, and the step to its second, g + 8
      const int e0 = (j * nx + (xneg ? nx - 1 - p0 - g4 : p0 + g4)) * 4;
      const int de = xneg ? -32 : 32;
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        if ((hf == 0 || CW > 8) && g4 + 8 * hf < cnt) {
          const uint32_t code = rs[g4 + 8 * hf].code;
          const int e = e0 + hf * de;
          if ((code & red_am0) == red_cv0) red_add(red_p0 + e, static_cast<double>(d[2 * hf]));
          if ((code & red_am1) == red_cv1) red_add(red_p1 + e, static_cast<double>(d[2 * hf + 1]));
        }
      }
    } else {
      {
        // forward: incident flux sum |v_n| W h at cells owning a downstream wall face; adjoint: the
        // transposed wall reads, sum 2 |v_a|/dx z at cells whose upstream neighbour is solid
        const uint32_t mycode = lane < cnt ? rs[lane].code : 0u;
        const bool fx = ADJ ? (((mycode >> kClsXShift) & 3u) == (uint32_t)kWall && !(mycode & kSolid)) : (mycode & kIncX) != 0;
        const bool fy = ADJ ? (((mycode >> kClsYShift) & 3u) == (uint32_t)kWall && !(mycode & kSolid)) : (mycode & kIncY) != 0;
        const unsigned incx = __ballot_sync(0xffffffffu, fx);
        const unsigned incy = __ballot_sync(0xffffffffu, fy);
        // one wall face per lane (at most 2 CW faces): the dot product over the velocities read back
        // from the ring, like a moment
        const int nfx = __popc(incx), nf = nfx + __popc(incy);
        for (int e = lane; e < nf; e += kLanes) {
          const bool is_x = e < nfx;
          const int l = (int)__fns(is_x ? incx : incy, 0u, is_x ? e + 1 : e - nfx + 1);
          const T f = dot32<T, RS>(myr + l * RS, wts + (is_x ? 4 : 5) * RS);
          const int i = xneg ? nx - 1 - (p0 + l) : p0 + l;
          red_add(&facc[(j * nx + i) * 4 + (is_x ? sidex : sidey)], static_cast<double>(f));
        }
      }
      // moments of the chunk (FP64, bound by the FP64 pipe): one (cell, moment) pair per lane and pass,
      // dot product over the lanes, skipped for solid cells and rows past the chunk (a pass whose pairs
      // are all skipped costs the warp nothing)
  #pragma unroll
      for (int pass = 0; pass < (CW * 4 + kLanes - 1) / kLanes; ++pass) {
        const int pr = pass * kLanes + lane;
        const int l = pr >> 2, m = pr & 3;
        if (pr < CW * 4 && l < cnt && !(rs[l].code & kSolid)) {
          const T sum = dot32<T, RS>(myr + l * RS, wts + m * RS);
          const int p = p0 + l;
          const int i = xneg ? nx - 1 - p : p;
          red_add(&acc[(j * nx + i) * 4 + m], static_cast<double>(sum));
        }
      }
    }
  };

  auto give_up = [&]() {
    cp_async_wait<0>();
    atomicExch(&st->err_flag, 1);
  };

  int item = 0;
  int s0 = lw % 3;  // ring slot of the current step t: the warp's steps are lw, lw + 1, ...
  T *ring_w = ring + (size_t)w * 3 * CW * RS;
  const T *ring_p1 = ring + (size_t)wprev * 3 * CW * RS;
  const T *ring_p2 = ring + (size_t)(wb + (lw + 2 * R - 2) % R) * 3 * CW * RS;
  if (NSTAGE == 2) issue(lw, 0, 0);
  for (int q = lw; q < ny; q += R) {
    for (int c = 0; c < R; ++c, ++item) {
      const int t = q + c;
      const int buf = (NSTAGE == 2) ? (item & 1) : 0;
      if (NSTAGE == 2) {
        // pf_* hold this row's x-seam values (loaded when this chunk was staged); latch them before
        // staging the next chunk, which may belong to the next row (one chunk per row when R = 1)
        if (c == 0) {
          row_hp1 = pf_hp1;
          row_hp2 = pf_hp2;
        }
        const int nq = (c + 1 < R) ? q : q + R, nc = (c + 1 < R) ? c + 1 : 0;
        if (nq < ny) issue(nq, nc, buf ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();
      } else {
        issue(q, c, 0);
        cp_async_wait<0>();
        if (c == 0) {
          row_hp1 = pf_hp1;
          row_hp2 = pf_hp2;
        }
      }
      __syncwarp();
      // row q-1 finished this chunk, and row q+2 has read the ring slot written three steps ago
      if (R > 1 && !wait_at_least(&prog[wprev], t)) return give_up();
      if (R > 2 && !wait_at_least(&prog[wnext2], t)) return give_up();
      const SweepRec<T> *rs = stage + ((size_t)w * NSTAGE + buf) * CW;
      // ring slots t % 3 (this row), (t - 1) % 3 (row q-1) and (t - 2) % 3 (row q-2)
      const int s1 = s0 == 0 ? 2 : s0 - 1, s2 = s0 == 2 ? 0 : s0 + 1;
      T *myr = ring_w + s0 * (CW * RS);
      const T *pr1 = ring_p1 + s1 * (CW * RS);
      const T *pr2 = ring_p2 + s2 * (CW * RS);
      s0 = s2;
      if (py && q < 2) {
        if (STAGE_SEAM) {
          T *sd = seamst + (((size_t)wt * 2 + (lw & 1)) * NSTAGE + buf) * 2 * CW * kLanes;
          const int cnt = min(CW, nx - c * CW);
          // the staged seam values are the previous iterate before its mass shift (own lane only)
          for (int l = 0; l < cnt; ++l) {
            if (q == 0) sd[l * kLanes + lane] -= sshift;
            sd[(CW + l) * kLanes + lane] -= sshift;
          }
          if (q == 0)
            run_chunk(std::integral_constant<int, 0>(), q, c, t, rs, myr, sd, kLanes, sd + CW * kLanes, kLanes);
          else
            run_chunk(std::integral_constant<int, 0>(), q, c, t, rs, myr, pr1, RS, sd + CW * kLanes, kLanes);
        } else {
          const int p0 = c * CW;
          const int i0 = xneg ? nx - 1 - p0 : p0;
          const int stride = xneg ? -2 * kLanes : 2 * kLanes;
          const T *s0 = seamy + i0 * 2 * kLanes + lane;
          if (q == 0)
            run_chunk(std::integral_constant<int, 1>(), q, c, t, rs, myr, s0 + kLanes, stride, s0, stride);
          else
            run_chunk(std::integral_constant<int, 2>(), q, c, t, rs, myr, pr1, RS, s0 + kLanes, stride);
        }
      } else {
        run_chunk(std::integral_constant<int, 0>(), q, c, t, rs, myr, pr1, RS, pr2, RS);
      }
      __syncwarp();
    }
  }
  if (lane == 0) st_release(&prog[w], INT_MAX / 2);  // no more rows: never wait on this warp again
}

}  // namespace sweep
}  // namespace dvm

#include "dvm_sweep_pair.cuh"

namespace dvm {
namespace sweep {

// One block per sweep-map entry: a tile of one velocity group per warp, or (FP32 forward launches with a
// uniform collision rate) a tile of group pairs when the entry carries kPairFlag.
template <typename T, bool UNIF, int CW, bool ADJ>
__global__ void __launch_bounds__(kMaxSweepWarps * kLanes, 1) sweep_kernel(LaunchDesc L) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int map = L.sweep_map[blockIdx.x];
  if constexpr (sizeof(T) == 4 && UNIF && !ADJ) {
    if (map & kPairFlag) {
      sweep_tile_pair<CW>(L, map, smem, (int)(blockDim.x >> 5));
      return;
    }
  }
  sweep_tile<T, UNIF, CW, ADJ, false>(L, map, smem, (int)(blockDim.x >> 5));
}

template <typename T, bool UNIF, int CW, bool ADJ>
cudaError_t launch(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  auto kern = sweep_kernel<T, UNIF, CW, ADJ>;
  size_t smem = layout<T>(L.warps, CW, L.row_tiles > 0 ? L.row_tiles : 1).total;
  smem = std::max(smem, (size_t)L.pair_smem);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, L.warps * kLanes, smem, stream>>>(L);
  return cudaGetLastError();
}

template <typename T, bool UNIF, bool ADJ>
cudaError_t launch_cw(const LaunchDesc &L, int nblocks, cudaStream_t stream) {
  switch (L.cw) {
    case 1: return launch<T, UNIF, 1, ADJ>(L, nblocks, stream);
    case 2: return launch<T, UNIF, 2, ADJ>(L, nblocks, stream);
    case 4: return launch<T, UNIF, 4, ADJ>(L, nblocks, stream);
    case 8: return launch<T, UNIF, 8, ADJ>(L, nblocks, stream);
    case 16: return launch<T, UNIF, 16, ADJ>(L, nblocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sweep
}  // namespace dvm
