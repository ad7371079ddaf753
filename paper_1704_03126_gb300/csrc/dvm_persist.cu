// dvm_persist.cu -- the persistent batched launch: m source iterations of every member of a batch in
// one kernel, scheduled on the device.
//
// Per sweep the source iteration of an instance has three stages (Eq. iteration: the transport sweep
// with its fused moments and wall fluxes; the mass shift of the projection; the shifted moments,
// records, residual and stopping test), and each stage is a set of independent work items: the
// instance's sweep tiles (velocity groups, row wavefront), then its cell chunks twice.  Each instance
// carries a 64-bit work word (stage counter << 32 | items taken).  A block takes an item by a compare-
// and-swap on the word, runs it with all its threads, and counts it finished; the block that finishes
// the last item of a stage does the stage's scalar work (the mass shift, or the stopping test) and
// publishes the next stage -- or retires the instance when it has converged, failed or run its sweeps
// for this launch.  There is no device-wide barrier: instances advance independently, a converged
// instance drops out at once, and one instance's finalize overlaps the others' sweeps.
//
// Waits.  A block with nothing to take polls the work words.  Every item is run by a block that has
// already started, so no wait depends on a block that is not resident; each poll loop is bounded
// (kPersistSpinLimit polls) and gives up with an error flag that the host reports as DVM_ETIMEOUT.
//
// Coherence.  Items read data that other blocks wrote earlier in the same launch (accumulators, fluxes,
// records, seams, the instance state).  The writer fences before counting its item finished; the
// taker fences after its compare-and-swap; reads of such data go through L2 (cp.async.cg, __ldcg).
#include <algorithm>
#include <climits>

#include "dvm_device.cuh"
#include "dvm_finalize.cuh"
#include "dvm_kernels.h"
#include "dvm_sweep.cuh"

namespace dvm {
namespace {

constexpr unsigned kRetired = 0xffffffffu;  // stage counter of an instance that takes no more items

__device__ __forceinline__ unsigned long long ld_word(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_int(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int items_of(const PersistDesc &P, int i, unsigned stage) {
  return stage == 0 ? P.tile_count[i] : P.fin_items[i];
}

__device__ __forceinline__ double block_sum_p(double v, double *sh) {
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

// Warp 0 takes a work item: finalize items first (they release an instance's next sweep), then
// sweep tiles, instances in P.order (longest sweeps first).  Returns 1 with (inst, stage, idx), 0
// when every instance has retired, -1 when the poll limit ran out.
__device__ int take_item(const PersistDesc &P, int *inst, unsigned *stage, int *idx) {
  const int lane = threadIdx.x & 31;
  for (int spin = 0;; ++spin) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int base = 0; base < P.ninst; base += 32) {
        const int k = base + lane;
        int i = -1;
        unsigned long long w = 0ull;
        bool cand = false;
        if (k < P.ninst) {
          i = P.order[k];
          w = ld_word(P.work + i);
          const unsigned ph = (unsigned)(w >> 32), taken = (unsigned)w;
          if (ph != kRetired) {
            const unsigned st = ph % 3u;
            cand = (pass == 0) == (st != 0u) && taken < (unsigned)items_of(P, i, st);
          }
        }
        unsigned m = __ballot_sync(0xffffffffu, cand);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          int ok = 0;
          if (lane == src) ok = atomicCAS(P.work + i, w, w + 1ull) == w;
          ok = __shfl_sync(0xffffffffu, ok, src);
          if (ok) {
            *inst = __shfl_sync(0xffffffffu, i, src);
            const unsigned long long wv = __shfl_sync(0xffffffffu, w, src);
            *stage = (unsigned)(wv >> 32) % 3u;
            *idx = (int)(unsigned)wv;
            return 1;
          }
        }
      }
    }
    if (ld_int(P.active) <= 0 || ld_int(P.error) != 0) return 0;
    if (spin >= kPersistSpinLimit) return -1;
    if (spin > 32) __nanosleep(256);
  }
}

// Count an item finished (thread 0, after the block's writes are fenced); the last item of a stage
// does that stage's scalar work and publishes the next stage or retires the instance.
__device__ void finish_item(const LaunchDesc &L, const PersistDesc &P, int i, unsigned stage) {
  const unsigned cnt = (unsigned)items_of(P, i, stage);
  if (atomicAdd(P.finished + i, 1u) + 1u != cnt) return;
  __threadfence();
  atomicExch(P.finished + i, 0u);
  const InstanceDesc *D = L.inst + i;
  DeviceState *st = D->state;
  const unsigned long long w = ld_word(P.work + i);
  const unsigned ph = (unsigned)(w >> 32);
  bool retire = false;
  if (stage == 1u) {
    // the mass shift of this sweep (the projection's null mode)
    const double mass = atomicAdd(&st->mass_acc, 0.0);
    st->s_new = mass / ((double)D->n_gas * D->sumW[0]);
    st->mass_acc = 0.0;
  } else if (stage == 2u) {
    const double dsum = atomicAdd(&st->du_acc, 0.0);
    const double usum = atomicAdd(&st->u_acc, 0.0);
    const double qsum = atomicAdd(&st->q_acc, 0.0);
    const double s = __ldcg(&st->s_new);
    const double c_new = __ldcg(&st->c) + s + (D->rho ? D->rho[(size_t)8 * D->ncell] : 0.0);
    stop_test(D, st, dsum, usum, qsum, c_new, s);
    const int left = atomicSub(P.left + i, 1) - 1;
    retire = ld_int(&st->done) != 0 || left <= 0;
  }
  __threadfence();
  if (retire) {
    atomicExch(P.work + i, (unsigned long long)kRetired << 32);
    __threadfence();
    atomicSub(P.active, 1);
  } else {
    atomicExch(P.work + i, (unsigned long long)(ph + 1u) << 32);
  }
}

// Stage 1 item: this chunk's share of sum_gas rho.
__device__ void fin1_item(const InstanceDesc *D, int idx, int chunk, double *sh) {
  DeviceState *st = D->state;
  const int c0 = idx * chunk, c1 = min(c0 + chunk, D->ncell);
  double v = 0.0;
  for (int cell = c0 + threadIdx.x; cell < c1; cell += blockDim.x)
    if (!(D->code4[(size_t)cell * 4] & kSolid)) v += __ldcg(D->acc + (size_t)cell * 4);
  v = block_sum_p(v, sh);
  if (threadIdx.x == 0) atomicAdd(&st->mass_acc, v);
}

// Stage 2 item: shifted moments, records and the stopping-test terms of this chunk's cells.
template <typename T>
__device__ void fin2_item(const InstanceDesc *D, int idx, int chunk, int nitems, double *sh) {
  DeviceState *st = D->state;
  const int ncell = D->ncell;
  const double s = __ldcg(&st->s_new);
  const double *rho_in = D->rho;
  const double c_new = __ldcg(&st->c) + s + (rho_in ? rho_in[(size_t)8 * ncell] : 0.0);
  const int parity = (__ldcg(&st->iter) + 1) & 1;
  const double *fcur = D->facc + (size_t)parity * ncell * 4;
  double *fnext = D->facc + (size_t)(parity ^ 1) * ncell * 4;
  double du = 0.0, ua = 0.0, uq = 0.0, bad = 0.0;
  const int c0 = idx * chunk, c1 = min(c0 + chunk, ncell);
  for (int cell = c0 + threadIdx.x; cell < c1; cell += blockDim.x) {
    double a = 0.0, b = 0.0, q = 0.0, x = 0.0;
    fin2_cell<T>(D, cell, s, c_new, fcur, fnext, rho_in, false, a, b, q, x);
    du += a;
    ua += b;
    uq += q;
    bad += x;
  }
  if (rho_in) seam_inject<T>(D, (size_t)idx * blockDim.x + threadIdx.x, (size_t)nitems * blockDim.x);
  du = block_sum_p(du, sh);
  ua = block_sum_p(ua, sh);
  uq = block_sum_p(uq, sh);
  bad = block_sum_p(bad, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&st->du_acc, du);
    atomicAdd(&st->u_acc, ua);
    atomicAdd(&st->q_acc, uq);
    if (bad > 0.0) atomicExch(&st->nan_flag, 1);
  }
}

template <typename T, bool UNIF, int CW>
__global__ void __launch_bounds__(kMaxSweepWarps * kLanes, 1) persist_kernel(LaunchDesc L, PersistDesc P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int item[4];
  __shared__ double sh[32];
  const int Rb = (int)(blockDim.x >> 5);
  for (;;) {
    if (threadIdx.x < 32) {
      int inst = 0, idx = 0;
      unsigned stage = 0;
      const int r = take_item(P, &inst, &stage, &idx);
      if (threadIdx.x == 0) {
        if (r < 0) atomicExch(P.error, 1);
        item[0] = r;
        item[1] = inst;
        item[2] = (int)stage;
        item[3] = idx;
      }
    }
    __syncthreads();
    const int r = item[0], inst = item[1], stage = item[2], idx = item[3];
    if (r <= 0) break;
    __threadfence();  // order this block's reads after the take
    const InstanceDesc *D = L.inst + inst;
    if (stage == 0) {
      const int map = P.tiles[P.tile_base[inst] + idx];
      bool paired = false;
      if constexpr (sizeof(T) == 4 && UNIF) {
        if (map & kPairFlag) {
          sweep::sweep_tile_pair<CW, true>(L, map, smem, Rb);
          paired = true;
        }
      }
      if (!paired) sweep::sweep_tile<T, UNIF, CW, false, true>(L, map, smem, Rb);
    } else if (stage == 1) {
      fin1_item(D, idx, P.fin_cells, sh);
    } else {
      fin2_item<T>(D, idx, P.fin_cells, P.fin_items[inst], sh);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) finish_item(L, P, inst, (unsigned)stage);
  }
}

// Arm the scheduler for one launch: every member that is not done takes up to `sweeps` sweeps.
__global__ void persist_init_kernel(LaunchDesc L, PersistDesc P, int sweeps) {
  __shared__ int act;
  if (threadIdx.x == 0) act = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < P.ninst; i += blockDim.x) {
    const bool done = L.inst[i].state->done != 0;
    P.work[i] = done ? (unsigned long long)kRetired << 32 : 0ull;
    P.finished[i] = 0u;
    P.left[i] = sweeps;
    if (!done) atomicAdd(&act, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *P.active = act;
    *P.error = 0;
  }
}

// A scheduler whose instances never publish work: the poll loop must give up (failure detection).
__global__ void persist_selftest_kernel(PersistDesc P, int *result) {
  if (threadIdx.x < 32) {
    int inst = 0, idx = 0;
    unsigned stage = 0;
    const int r = take_item(P, &inst, &stage, &idx);
    if (threadIdx.x == 0) *result = r;
  }
}

template <typename T, bool UNIF, int CW>
cudaError_t launch_p(const LaunchDesc &L, const PersistDesc &P, int blocks, cudaStream_t stream) {
  auto kern = persist_kernel<T, UNIF, CW>;
  const size_t smem = std::max(sweep::layout<T>(L.warps, CW, L.row_tiles > 0 ? L.row_tiles : 1).total,
                               (size_t)L.pair_smem);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, L.warps * kLanes, smem, stream>>>(L, P);
  return cudaGetLastError();
}

template <typename T, bool UNIF>
cudaError_t launch_cw(const LaunchDesc &L, const PersistDesc &P, int blocks, cudaStream_t stream) {
  switch (L.cw) {
    case 1: return launch_p<T, UNIF, 1>(L, P, blocks, stream);
    case 2: return launch_p<T, UNIF, 2>(L, P, blocks, stream);
    case 4: return launch_p<T, UNIF, 4>(L, P, blocks, stream);
    case 8: return launch_p<T, UNIF, 8>(L, P, blocks, stream);
    case 16: return launch_p<T, UNIF, 16>(L, P, blocks, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, bool UNIF, int CW>
int occupancy_p(const LaunchDesc &L) {
  int n = 0;
  const size_t smem = std::max(sweep::layout<T>(L.warps, CW, L.row_tiles > 0 ? L.row_tiles : 1).total,
                               (size_t)L.pair_smem);
  auto kern = persist_kernel<T, UNIF, CW>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, L.warps * kLanes, smem) != cudaSuccess) return 0;
  return n;
}

template <typename T, bool UNIF>
int occupancy_cw(const LaunchDesc &L) {
  switch (L.cw) {
    case 1: return occupancy_p<T, UNIF, 1>(L);
    case 2: return occupancy_p<T, UNIF, 2>(L);
    case 4: return occupancy_p<T, UNIF, 4>(L);
    case 8: return occupancy_p<T, UNIF, 8>(L);
    case 16: return occupancy_p<T, UNIF, 16>(L);
    default: return 0;
  }
}

}  // namespace

cudaError_t launch_persistent(bool fp64, bool uniform_delta, const LaunchDesc &L, const PersistDesc &P, int blocks,
                              int sweeps, cudaStream_t stream) {
  persist_init_kernel<<<1, 256, 0, stream>>>(L, P, sweeps);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fp64) return uniform_delta ? launch_cw<double, true>(L, P, blocks, stream) : launch_cw<double, false>(L, P, blocks, stream);
  return uniform_delta ? launch_cw<float, true>(L, P, blocks, stream) : launch_cw<float, false>(L, P, blocks, stream);
}

int persistent_blocks_per_sm(bool fp64, bool uniform_delta, const LaunchDesc &L) {
  if (fp64) return uniform_delta ? occupancy_cw<double, true>(L) : occupancy_cw<double, false>(L);
  return uniform_delta ? occupancy_cw<float, true>(L) : occupancy_cw<float, false>(L);
}

cudaError_t launch_persist_selftest(const PersistDesc &P, int *result_dev, cudaStream_t stream) {
  persist_selftest_kernel<<<1, 32, 0, stream>>>(P, result_dev);
  return cudaGetLastError();
}

}  // namespace dvm
