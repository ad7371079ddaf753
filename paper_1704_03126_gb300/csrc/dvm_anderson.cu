// dvm_anderson.cu -- Anderson mixing of the source iteration (an extension: the paper iterates
// Eq. (iteration) plainly).
//
// One source iteration maps the projected state x (what the next sweep starts from: the moments
// rho, u1, u2, rho + tau of every gas cell, the incident fluxes of every wall face, the lagged values
// on the periodic seams and the mass shift c) to g = G(x).  Plain iteration takes x_{k+1} = g_k.  Type-II
// Anderson mixing of depth m (Walker & Ni, SIAM J. Numer. Anal. 49, 2011) keeps the last m differences
// dF_j = f_{j+1} - f_j of the residuals f = g - x and dG_j = g_{j+1} - g_j, and takes
//   gamma = argmin | f_k - dF gamma |_2,   x_{k+1} = g_k - dG gamma.
// Both iterations have the same fixed points.  The three kernels run between the mass projection
// (fin1, which sets the shift s of the sweep's output) and the record writer (fin2):
//   gather  g (the sweep's output shifted by s), f = g - x, the newest difference pair and the dot
//           products dF_new . dF_j and dF_j . f over the state;
//   solve   one thread per instance: the m x m normal equations (Cholesky with a small ridge), the
//           new c, and the shift s' = c_{k+1} - c that fin2 will apply;
//   update  x_{k+1} written back into the sweep's output arrays shifted by s', so that fin2 and the
//           next sweep see exactly x_{k+1}.
#include "dvm_kernels.h"

namespace dvm {
namespace {

constexpr int kAABlock = 256;

// Element e of the state of instance D: its value g (the sweep output after the shift s) and a
// writer that stores x back shifted by s2.
template <typename T>
struct StateView {
  const InstanceDesc *D;
  const AndersonDesc *A;
  double *fcur;
  T *sx, *sy;

  __device__ StateView(const InstanceDesc *d) : D(d), A(d->aa) {
    fcur = D->facc + (size_t)((D->state->iter + 1) & 1) * D->ncell * 4;
    sx = static_cast<T *>(D->seam_x);
    sy = static_cast<T *>(D->seam_y);
  }
  __device__ double g(long long e, double s) const {
    if (e < A->n_mom) {
      const int cell = (int)(e >> 2);
      if (D->code4[(size_t)cell * 4] & kSolid) return 0.0;
      return D->acc[e] - s * D->sumW[e & 3];
    }
    e -= A->n_mom;
    if (e < A->n_wall) return A->wallface[e] ? fcur[e] - s * D->ain[e & 3] : 0.0;
    e -= A->n_wall;
    if (e < A->n_sx) return (double)sx[e] - s;
    e -= A->n_sx;
    if (e < A->n_sy) return (double)sy[e] - s;
    return D->state->c + s;  // the last element: c
  }
  __device__ void put(long long e, double x, double s2) const {
    if (e < A->n_mom) {
      const int cell = (int)(e >> 2);
      if (!(D->code4[(size_t)cell * 4] & kSolid)) D->acc[e] = x + s2 * D->sumW[e & 3];
      return;
    }
    e -= A->n_mom;
    if (e < A->n_wall) {
      if (A->wallface[e]) fcur[e] = x + s2 * D->ain[e & 3];
      return;
    }
    e -= A->n_wall;
    if (e < A->n_sx) {
      sx[e] = static_cast<T>(x + s2);
      return;
    }
    e -= A->n_sx;
    if (e < A->n_sy) sy[e] = static_cast<T>(x + s2);
    // c: fin2 forms c + s2 itself
  }
};

__device__ __forceinline__ bool aa_active(const InstanceDesc *D) {
  return D->aa != nullptr && !*reinterpret_cast<const volatile int *>(&D->state->done);
}

template <typename T>
__global__ void __launch_bounds__(kAABlock) aa_gather_kernel(LaunchDesc L) {
  const InstanceDesc *D = L.inst + blockIdx.y;
  if (!aa_active(D)) return;
  const AndersonDesc *A = D->aa;
  const StateView<T> V(D);
  const int m = A->m;
  const int k = A->meta[2];                       // gathers so far
  const int count = A->meta[0], head = A->meta[1];
  const int ncol = k == 0 ? 0 : (count < m ? count + 1 : m);  // columns once the new one is in
  const double s = D->state->s_new;
  double dn[kAAMaxDepth], df[kAAMaxDepth];
#pragma unroll
  for (int j = 0; j < kAAMaxDepth; ++j) dn[j] = df[j] = 0.0;
  double ex[4] = {0.0, 0.0, 0.0, 0.0};  // |f|^2, |g|^2, |dG_new|^2, |dx_new|^2 over the flow velocity
  const long long n = A->n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double ge = V.g(e, s);
    const double fe = ge - A->x[e];
    if (k > 0) {
      const double dfe = fe - A->fp[e];
      const double dge = ge - A->gp[e];
      A->dF[(size_t)head * n + e] = dfe;
      A->dG[(size_t)head * n + e] = dge;
      if (e < A->n_mom && (int)(e & 3) == A->flow_comp) {
        ex[0] += fe * fe;
        ex[1] += ge * ge;
        ex[2] += dge * dge;
        ex[3] += (dge - dfe) * (dge - dfe);
      }
#pragma unroll
      for (int j = 0; j < kAAMaxDepth; ++j) {
        if (j < ncol) {
          const double dj = j == head ? dfe : A->dF[(size_t)j * n + e];
          dn[j] += dfe * dj;
          df[j] += dj * fe;
        }
      }
    }
    A->fp[e] = fe;
    A->gp[e] = ge;
  }
  if (k == 0) return;
  // block sums of the 2 m dot products, then one atomic each
  __shared__ double sh[kAABlock / 32][kAARed];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    double a = ex[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[wid][2 * kAAMaxDepth + t] = a;
  }
#pragma unroll
  for (int j = 0; j < kAAMaxDepth; ++j) {
    if (j < ncol) {
      double a = dn[j], b = df[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
      if (lane == 0) {
        sh[wid][j] = a;
        sh[wid][kAAMaxDepth + j] = b;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < kAARed) {
    const int j = threadIdx.x < 2 * kAAMaxDepth ? threadIdx.x % kAAMaxDepth : 0;
    if (j < ncol) {
      double t = 0.0;
      for (int w = 0; w < kAABlock / 32; ++w) t += sh[w][threadIdx.x];
      atomicAdd(&A->red[threadIdx.x], t);
    }
  }
}

// One thread per instance: the newest Gram row, the least-squares coefficients, the new c.
__global__ void aa_solve_kernel(LaunchDesc L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.ninst) return;
  const InstanceDesc *D = L.inst + i;
  if (!aa_active(D)) return;
  const AndersonDesc *A = D->aa;
  DeviceState *st = D->state;
  const int m = A->m;
  int *meta = A->meta;
  const int k = meta[2];
  meta[2] = k + 1;
  if (k == 0) {
    for (int j = 0; j < m; ++j) A->gamma[j] = 0.0;
    return;  // x_1 = g_0; s unchanged
  }
  const int count = meta[0], head = meta[1];
  const int ncol = count < m ? count + 1 : m;
  // stopping estimate: the plain residual at x_k over the flow velocity, divided by 1 - rho with
  // rho the largest contraction |G(x_j+1) - G(x_j)| / |x_j+1 - x_j| seen so far
  {
    const double *ex = A->red + 2 * kAAMaxDepth;
    if (ex[3] > 0.0) st->aa_rho = fmax(st->aa_rho, fmin(sqrt(ex[2] / ex[3]), 0.9999));
    st->aa_res = ex[1] > 0.0 ? sqrt(ex[0] / ex[1]) : 0.0;
    st->aa_est = st->aa_res / (1.0 - st->aa_rho);
  }
  double *G = A->gram;
  double rhs[kAAMaxDepth];
  for (int j = 0; j < ncol; ++j) {
    G[head * m + j] = A->red[j];
    G[j * m + head] = A->red[j];
    rhs[j] = A->red[kAAMaxDepth + j];
  }
  for (int j = 0; j < kAARed; ++j) A->red[j] = 0.0;
  meta[0] = ncol;
  meta[1] = (head + 1) % m;
  // (G + lambda I) gamma = rhs by Cholesky.  Differences of late iterates are nearly parallel, so the
  // normal equations are ill-conditioned: the ridge lambda starts at 1e-12 of the largest diagonal
  // entry and grows a hundredfold per failed factorisation (the history is dropped only when even
  // 1e-2 fails).
  double Lc[kAAMaxDepth * kAAMaxDepth];
  double dmax = 0.0;
  for (int j = 0; j < ncol; ++j) dmax = fmax(dmax, G[j * m + j]);
  bool ok = dmax > 0.0 && isfinite(dmax);
  for (double rel = 1e-12; ok && rel <= 1e-2; rel *= 100.0) {
    const double lam = rel * dmax;
    bool fact = true;
    for (int r = 0; r < ncol && fact; ++r) {
      for (int c = 0; c <= r; ++c) {
        double v = G[r * m + c] + (r == c ? lam : 0.0);
        for (int q = 0; q < c; ++q) v -= Lc[r * kAAMaxDepth + q] * Lc[c * kAAMaxDepth + q];
        if (r == c) {
          if (!(v > 0.0)) {
            fact = false;
            break;
          }
          Lc[r * kAAMaxDepth + r] = sqrt(v);
        } else {
          Lc[r * kAAMaxDepth + c] = v / Lc[c * kAAMaxDepth + c];
        }
      }
    }
    if (fact) break;
    if (rel * 100.0 > 1e-2) ok = false;
  }
  double gam[kAAMaxDepth];
  if (ok) {
    for (int r = 0; r < ncol; ++r) {
      double v = rhs[r];
      for (int q = 0; q < r; ++q) v -= Lc[r * kAAMaxDepth + q] * gam[q];
      gam[r] = v / Lc[r * kAAMaxDepth + r];
    }
    for (int r = ncol - 1; r >= 0; --r) {
      double v = gam[r];
      for (int q = r + 1; q < ncol; ++q) v -= Lc[q * kAAMaxDepth + r] * gam[q];
      gam[r] = v / Lc[r * kAAMaxDepth + r];
    }
    for (int r = 0; r < ncol; ++r) ok = ok && isfinite(gam[r]);
  }
  if (!ok) {
    // a degenerate history: drop it and take the plain step
    for (int r = 0; r < ncol; ++r) gam[r] = 0.0;
    meta[0] = 0;
    meta[1] = 0;
  }
  for (int j = 0; j < m; ++j) A->gamma[j] = j < ncol ? gam[j] : 0.0;
  // c_{k+1} = g_c - dG_c gamma; fin2 forms c + s_new, so s_new becomes c_{k+1} - c
  const size_t ec = (size_t)(A->n - 1);
  double xc = A->gp[ec];
  for (int j = 0; j < ncol; ++j) xc -= gam[j] * A->dG[(size_t)j * A->n + ec];
  st->s_new = xc - st->c;
}

template <typename T>
__global__ void __launch_bounds__(kAABlock) aa_update_kernel(LaunchDesc L) {
  const InstanceDesc *D = L.inst + blockIdx.y;
  if (!aa_active(D)) return;
  const AndersonDesc *A = D->aa;
  const StateView<T> V(D);
  const int m = A->m;
  const int ncol = A->meta[2] <= 1 ? 0 : A->meta[0];
  const double s2 = D->state->s_new;
  double gam[kAAMaxDepth];
#pragma unroll
  for (int j = 0; j < kAAMaxDepth; ++j) gam[j] = j < m ? A->gamma[j] : 0.0;
  const long long n = A->n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double x = A->gp[e];
#pragma unroll
    for (int j = 0; j < kAAMaxDepth; ++j)
      if (j < ncol) x -= gam[j] * A->dG[(size_t)j * n + e];
    A->x[e] = x;
    V.put(e, x, s2);
  }
}

}  // namespace

cudaError_t launch_anderson(const LaunchDesc &L, bool fp64, cudaStream_t stream) {
  const dim3 grid(L.aa_blocks, L.ninst);
  if (fp64) aa_gather_kernel<double><<<grid, kAABlock, 0, stream>>>(L);
  else aa_gather_kernel<float><<<grid, kAABlock, 0, stream>>>(L);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  aa_solve_kernel<<<(L.ninst + 63) / 64, 64, 0, stream>>>(L);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (fp64) aa_update_kernel<double><<<grid, kAABlock, 0, stream>>>(L);
  else aa_update_kernel<float><<<grid, kAABlock, 0, stream>>>(L);
  return cudaGetLastError();
}

}  // namespace dvm
