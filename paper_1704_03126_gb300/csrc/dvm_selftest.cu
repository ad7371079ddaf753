// dvm_selftest.cu -- failure detection without a fault: the sweeps' bounded waits, run on a flag
// that nothing raises, give up after their spin limit and report it as a status.
//
// A sweep block that waits for a neighbour warp (row sweep: an acquire-load of a progress word) or
// for a TMA stage (column sweep: mbarrier try_wait) spins at most a fixed number of times; when the
// limit runs out the block records DVM_ETIMEOUT in the instance state and returns, so the context
// stays usable.  dvm_selftest_wait runs the same wait primitives in a one-block kernel whose flag or
// barrier never completes.
#include <chrono>

#include "dvm.h"
#include "dvm_kernels.h"
#include "dvm_sweep.cuh"
#include "dvm_sweep_cols.cuh"

namespace dvm {
namespace {

// result: 1 when the wait gave up, 0 when the (never raised) flag was seen
__global__ void selftest_wait_kernel(int primitive, int spin_limit, int *result) {
  __shared__ int flag;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    flag = 0;
    if (primitive == 1) cols::mbar_init(&bar, 1);
  }
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  __syncthreads();
  bool seen = false;
  if (primitive == 0) {
    // the row sweep's progress-word wait (all lanes of every warp)
    if (spin_limit <= 0) {
      seen = sweep::wait_at_least(&flag, 1);
    } else {
      for (int spin = 0; spin < spin_limit && !seen; ++spin) seen = sweep::ld_acquire(&flag) >= 1;
    }
  } else if (threadIdx.x == 0) {
    // the column sweep's stage wait: phase 0 of a barrier that expects one arrival that never comes
    const int limit = spin_limit > 0 ? spin_limit : kColsSpinLimit;
    for (int spin = 0; spin < limit && !seen; ++spin) seen = cols::mbar_try_wait(&bar, 0u);
  }
  __syncthreads();
  if (threadIdx.x == 0) *result = seen ? 0 : 1;
}

}  // namespace
}  // namespace dvm

// Primitive 2: the persistent launch's scheduler poll (dvm_persist.cu) on one instance that is active
// but whose only work item is already taken, so no work ever appears; the poll must give up (-1).
static dvm_status selftest_persist(double *seconds) {
  using namespace dvm;
  // work word, finished, left, active, error, order, tile_base, tile_count, fin_items, tiles, result
  int *mem = nullptr;
  if (cudaMalloc(&mem, 64 * sizeof(int)) != cudaSuccess) return DVM_ECUDA;
  int h[64] = {};
  // work word of instance 0: stage 0, one item taken (ints 0-1); active = 1 (int 5)
  h[0] = 1;
  h[5] = 1;
  h[7] = 0;   // order
  h[8] = 0;   // tile_base
  h[9] = 1;   // tile_count
  h[10] = 1;  // fin_items
  h[11] = 0;  // tiles
  PersistDesc P{};
  P.ninst = 1;
  P.fin_cells = 1;
  P.work = reinterpret_cast<unsigned long long *>(mem);
  P.finished = reinterpret_cast<unsigned int *>(mem + 2);
  P.left = mem + 4;
  P.active = mem + 5;
  P.error = mem + 6;
  P.order = mem + 7;
  P.tile_base = mem + 8;
  P.tile_count = mem + 9;
  P.fin_items = mem + 10;
  P.tiles = mem + 11;
  int *result = mem + 12;
  h[12] = 7;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMemcpy(mem, h, sizeof(h), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_persist_selftest(P, result, 0);
  int r = 7;
  if (e == cudaSuccess) e = cudaMemcpy(&r, result, sizeof(int), cudaMemcpyDeviceToHost);
  const auto t1 = std::chrono::steady_clock::now();
  cudaFree(mem);
  if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
  if (e != cudaSuccess) return DVM_ECUDA;
  return r == -1 ? DVM_ETIMEOUT : DVM_OK;
}

extern "C" dvm_status dvm_selftest_wait(int primitive, int spin_limit, double *seconds) {
  if (primitive == 2) return selftest_persist(seconds);
  if (primitive != 0 && primitive != 1) return DVM_EINVAL;
  int *d_result = nullptr;
  if (cudaMalloc(&d_result, sizeof(int)) != cudaSuccess) return DVM_ECUDA;
  const auto t0 = std::chrono::steady_clock::now();
  dvm::selftest_wait_kernel<<<1, 128>>>(primitive, spin_limit, d_result);
  int result = -1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(&result, d_result, sizeof(int), cudaMemcpyDeviceToHost);
  const auto t1 = std::chrono::steady_clock::now();
  cudaFree(d_result);
  if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
  if (e != cudaSuccess) return DVM_ECUDA;
  return result == 1 ? DVM_ETIMEOUT : DVM_OK;
}
