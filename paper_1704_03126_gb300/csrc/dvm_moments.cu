// dvm_moments.cu -- moments and mass flow rate of a distribution held by the caller.
//
// rho = sum_k W_k h_k, u_i = sum_k W_k v_i h_k, tau = sum_k W_k |v_k|^2 h_k - rho (the quadrature
// forms of the moments of Sec. II.A) at every cell, and Q = sum_gas u1 dA / L (Sec. III, Eq. Q).
// One thread per cell walks the velocities (coalesced over cells for the [K][ncell] layout);
// block partial sums of Q go to scratch memory and the last block adds them in block order, so Q
// is deterministic.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "dvm.h"
#include "dvm_tables.h"

namespace dvm {

// Records the message that dvm_last_error(NULL) returns (defined with the other C ABI calls).
void set_moments_error(const std::string &msg);

namespace {

constexpr int kMomBlock = 256;
constexpr int kMomMaxBlocks = 1024;

struct VelTable {
  int n;
  double x[64];
  double w[64];
};

__global__ void __launch_bounds__(kMomBlock) moments_kernel(const double *__restrict__ h, const uint8_t *__restrict__ mask,
                                                            int ncell, VelTable vt, double dA_over_L,
                                                            double *__restrict__ mom, double *__restrict__ Q,
                                                            double *partials, unsigned int *ticket) {
  __shared__ double sh[kMomBlock / 32];
  const int n = vt.n;
  double q_local = 0.0;
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < ncell; cell += gridDim.x * blockDim.x) {
    const bool gas = !mask || !mask[cell];
    double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0;
    if (gas) {
      for (int a = 0; a < n; ++a) {
        const double v1 = vt.x[a], wa = vt.w[a];
        for (int b = 0; b < n; ++b) {
          const double v2 = vt.x[b];
          const double wh = wa * vt.w[b] * h[(size_t)(a * n + b) * ncell + cell];
          m0 += wh;
          m1 += wh * v1;
          m2 += wh * v2;
          m3 += wh * (v1 * v1 + v2 * v2);
        }
      }
      q_local += m1;
    }
    mom[(size_t)cell * 4 + 0] = m0;
    mom[(size_t)cell * 4 + 1] = m1;
    mom[(size_t)cell * 4 + 2] = m2;
    mom[(size_t)cell * 4 + 3] = m3 - m0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q_local += __shfl_xor_sync(0xffffffffu, q_local, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = q_local;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int wi = 0; wi < kMomBlock / 32; ++wi) s += sh[wi];
    partials[blockIdx.x] = s;
    __threadfence();
    const unsigned t = atomicAdd(ticket, 1u);
    if (t == gridDim.x - 1) {
      __threadfence();
      double total = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) total += *((volatile double *)&partials[b]);
      *Q = total * dA_over_L;
      *ticket = 0u;
    }
  }
}

// Validate arguments and build the velocity table; returns DVM_OK or the failure.
dvm_status prepare(const dvm_quad *q, const double *h, int ncell, double *mom, double *Q, VelTable &vt,
                   int &blocks, std::string *why = nullptr) {
  if (!q || !h || !mom || !Q || ncell < 1) {
    if (why) *why = "null pointer argument or ncell < 1";
    return DVM_EINVAL;
  }
  std::vector<double> x, w;
  std::string err;
  if (!quadrature_1d(q->kind, q->n, q->vmax, x, w, err)) {  // n even, 2 <= n <= 64 (VelTable holds 64)
    if (why) *why = err;
    return DVM_EINVAL;
  }
  vt.n = q->n;
  for (int a = 0; a < q->n; ++a) {
    vt.x[a] = x[a];
    vt.w[a] = w[a];
  }
  const long long want = ((long long)ncell + kMomBlock - 1) / kMomBlock;
  blocks = (int)(want < kMomMaxBlocks ? want : kMomMaxBlocks);
  return DVM_OK;
}

}  // namespace
}  // namespace dvm

extern "C" dvm_status dvm_moments(const dvm_quad *q, const double *h, const uint8_t *mask, int ncell,
                                  double dA_over_L, double *mom, double *Q, void *stream) {
  using namespace dvm;
  VelTable vt;
  int blocks = 0;
  dvm_status st = prepare(q, h, ncell, mom, Q, vt, blocks);
  if (st != DVM_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void *scratch = nullptr;  // block partials, then the last-block ticket
  const size_t bytes = sizeof(double) * kMomMaxBlocks + 256;
  if (cudaMalloc(&scratch, bytes) != cudaSuccess) return DVM_ENOMEM;
  double *partials = static_cast<double *>(scratch);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + sizeof(double) * kMomMaxBlocks);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    moments_kernel<<<blocks, kMomBlock, 0, s>>>(h, mask, ncell, vt, dA_over_L, mom, Q, partials, ticket);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  return e == cudaSuccess ? DVM_OK : DVM_ECUDA;
}

// ------------------------------------------------------------------------------------------------
// dvm_moments_noalloc: the same reduction with its scratch in a fixed device array, for callers that
// cannot allocate device memory during a call.  cudaMalloc / cudaFree synchronise the whole device
// and can fail under memory pressure; a caller in a latency-critical loop, a caller whose device
// memory is all reserved by a framework allocator at start-up, or a caller that may not touch the
// allocator while other streams run therefore cannot use dvm_moments, which allocates per call.
//
// The scratch below (block partial sums of Q and the last-block ticket, about 8.3 KB) lives in every
// device that loads this library until the process exits.  Every call shares it and it keeps the
// last call's contents; the ticket, which must start at zero, is cleared at the start of each call.
// Calls on one device that overlap on the GPU (for example on two streams) race on the same array and
// must be serialised by the caller.  The first call in a CUDA context looks up the array's device
// address (cudaGetSymbolAddress, with that context current); make that first call before any stream
// capture.  The address is cached per (device, context): after cudaDeviceReset, or when the primary
// context is released and created again, the module is loaded anew and the next call looks the
// address up again instead of using the stale one.
namespace dvm {
namespace {

constexpr size_t kNoAllocScratchBytes = sizeof(double) * kMomMaxBlocks + 256;
// The grid-stride kernel needs only kMomMaxBlocks partial sums for any cell count, so the scratch does
// not bound ncell; the call accepts at most this many cells (as many as the largest dvm_create grid,
// rounded up to a power of two) so that its cost stays bounded.
constexpr long long kNoAllocMaxCells = 16777216LL;

__device__ __align__(256) unsigned char g_moments_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// The current driver context, read through the runtime's driver entry point (no link against libcuda).
cudaError_t current_context(CUcontext *out) {
  using GetCurrent = CUresult (*)(CUcontext *);
  static GetCurrent fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<GetCurrent>(p);
  }
  return fn(out) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array in the current context, looked up once per (device, context).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  e = cudaFree(nullptr);  // makes the device's primary context current (no allocation, no free)
  if (e != cudaSuccess) return e;
  CUcontext ctx = nullptr;
  e = current_context(&ctx);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_moments_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dvm

extern "C" dvm_status dvm_moments_noalloc(const dvm_quad *q, const double *h, const uint8_t *mask, int ncell,
                                          double dA_over_L, double *mom, double *Q, void *stream) {
  using namespace dvm;
  if ((long long)ncell > kNoAllocMaxCells) {
    set_moments_error("dvm_moments_noalloc: ncell = " + std::to_string(ncell) + " exceeds this call's maximum of " +
                      std::to_string(kNoAllocMaxCells) + " cells; use dvm_moments");
    return DVM_EINVAL;
  }
  VelTable vt;
  int blocks = 0;
  std::string why;
  dvm_status st = prepare(q, h, ncell, mom, Q, vt, blocks, &why);
  if (st != DVM_OK) {
    set_moments_error("dvm_moments_noalloc: " + why);
    return st;
  }
  void *scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_moments_error(std::string("dvm_moments_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return DVM_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *partials = static_cast<double *>(scratch);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + sizeof(double) * kMomMaxBlocks);
  e = cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    moments_kernel<<<blocks, kMomBlock, 0, s>>>(h, mask, ncell, vt, dA_over_L, mom, Q, partials, ticket);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_moments_error(std::string("dvm_moments_noalloc: ") + cudaGetErrorString(e));
    return DVM_ECUDA;
  }
  return DVM_OK;
}
