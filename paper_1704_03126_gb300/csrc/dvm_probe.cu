// dvm_probe.cu -- measured ceilings of this GPU for the roofline of the sweeps: the rate of dependent-
// free FMA chains in FP32, packed FP32x2 and FP64, and the L2 size.
//
// The transport sweep (Eq. iteration) keeps h on chip, so its bound is the SM's arithmetic rate, not
// HBM.  The FP64 rate of this part is a small fraction of its FP32 rate and is not published per
// clock in a form the roofline can use, so it is measured: every thread runs kChains independent FMA
// chains for `iters` steps (no memory traffic inside the loop), and the rate is the FMA count over the
// kernel's CUDA-event time.  The grid fills every SM several times over.
#include <cuda_runtime.h>

#include "dvm.h"

namespace dvm {
namespace {

constexpr int kChains = 8;
constexpr int kProbeBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeBlock) fma_chain_kernel(int iters, T a, T b, T *out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // a store the compiler cannot prove dead (a = 0 never happens for the caller's values)
  if (s == T(-12345)) out[0] = s;
}

// Packed FP32x2: each instruction does two FMAs.
__global__ void __launch_bounds__(kProbeBlock) fma2_chain_kernel(int iters, float a, float b, float *out) {
  float2 x[kChains];
  const float2 av = make_float2(a, a), bv = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = make_float2(float(threadIdx.x + c) * 1e-3f, float(c) * 1e-3f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], av, bv);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
  if (s == -12345.f) out[0] = s;
}

}  // namespace
}  // namespace dvm

extern "C" dvm_status dvm_probe_peaks(int kind, double seconds, double *tflops, int *l2_bytes, int *sms) {
  using namespace dvm;
  if (kind < 0 || kind > 2 || !tflops || !(seconds > 0.0) || seconds > 10.0) return DVM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DVM_ECUDA;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return DVM_ECUDA;
  if (l2_bytes) *l2_bytes = prop.l2CacheSize;
  if (sms) *sms = prop.multiProcessorCount;
  const int blocks = prop.multiProcessorCount * 8;  // 2048 threads per SM
  void *out = nullptr;
  if (cudaMalloc(&out, 16) != cudaSuccess) return DVM_ECUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // one calibration launch, then one launch sized to `seconds`
  auto run = [&](int iters, float *ms) -> cudaError_t {
    cudaError_t r = cudaEventRecord(e0, 0);
    if (r != cudaSuccess) return r;
    if (kind == 0)
      fma_chain_kernel<float><<<blocks, kProbeBlock>>>(iters, 0.999f, 1e-4f, static_cast<float *>(out));
    else if (kind == 1)
      fma2_chain_kernel<<<blocks, kProbeBlock>>>(iters, 0.999f, 1e-4f, static_cast<float *>(out));
    else
      fma_chain_kernel<double><<<blocks, kProbeBlock>>>(iters, 0.999, 1e-4, static_cast<double *>(out));
    r = cudaGetLastError();
    if (r != cudaSuccess) return r;
    r = cudaEventRecord(e1, 0);
    if (r != cudaSuccess) return r;
    r = cudaEventSynchronize(e1);
    if (r != cudaSuccess) return r;
    return cudaEventElapsedTime(ms, e0, e1);
  };
  float ms = 0.f;
  int iters = kind == 2 ? 256 : 4096;
  if (e == cudaSuccess) e = run(iters, &ms);
  if (e == cudaSuccess && ms > 0.f) {
    const double scale = seconds * 1e3 / ms;
    long long want = (long long)(iters * scale);
    if (want < iters) want = iters;
    if (want > (1LL << 30)) want = 1LL << 30;
    iters = (int)want;
    e = run(iters, &ms);
  }
  if (e == cudaSuccess) {
    const double fmas = (double)blocks * kProbeBlock * kChains * (double)iters * (kind == 1 ? 2.0 : 1.0);
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return e == cudaSuccess ? DVM_OK : DVM_ECUDA;
}
