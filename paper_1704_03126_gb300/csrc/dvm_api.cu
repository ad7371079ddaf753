// dvm_api.cu -- the C ABI of libdvm (include/dvm.h): contexts, device tables, the CUDA-graph solve
// loop and batched solves.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dvm.h"
#include "dvm_device.cuh"
#include "dvm_kernels.h"
#include "dvm_tables.h"

using namespace dvm;

namespace dvm {
namespace {
std::string g_create_error;
}  // namespace
// Errors of context-free calls (dvm_create failures, dvm_moments_noalloc) are read with dvm_last_error(NULL).
void set_moments_error(const std::string &msg) { g_create_error = msg; }
}  // namespace dvm

struct dvm_ctx {
  dvm_params P{};
  int nx = 0, ny = 0, ncell = 0, nv = 0, half = 0, gq = 0, ngroups = 0;  // stored (internal) grid
  // tr: the caller's grid (unx x uny, x1 along rows) is stored transposed, so that the sweeps walk
  // the longer axis; the caller's cell (i, j) is stored at (j, i) and its x1 is the stored x2
  bool tr = false;
  int unx = 0, uny = 0;
  double dxs = 0.0, dys = 0.0;     // stored x reference spacing and stored y spacing
  bool nux = false;                // stored x spacing varies by column (the caller's unequal rows)
  double *d_xwidth = nullptr;      // nux: stored column widths / dxs
  // Anderson mixing (dvm_params.anderson_depth > 0): the device descriptor and its buffers
  int aa_m = 0;
  long long aa_n = 0;
  AndersonDesc *d_aa = nullptr;
  double *d_aa_buf = nullptr;      // x, fp, gp [n] | dF, dG [m][n] | red [kAARed] | gram [m][m] | gamma [m]
  int *d_aa_meta = nullptr;
  unsigned char *d_wallface = nullptr;
  bool fp64 = true, store_h = false, uniform = true;
  double delta = 0.0, kn = 0.0;
  std::vector<double> x1, w1;
  Geometry geo;
  cudaStream_t stream = nullptr;     // work stream (user's or own)
  cudaStream_t cap_stream = nullptr; // private stream used for graph capture
  bool own_stream = false;
  int device = 0;
  // device memory
  void *d_vel = nullptr, *d_inv = nullptr, *d_rec = nullptr, *d_rec_diag = nullptr;
  uint32_t *d_code4 = nullptr;
  int *d_hw_src = nullptr;
  double *d_delta_field = nullptr, *d_acc = nullptr, *d_facc = nullptr, *d_mom = nullptr, *d_u1prev = nullptr;
  void *d_seamx = nullptr, *d_seamy = nullptr, *d_h = nullptr;
  DeviceState *d_state = nullptr;
  InstanceDesc hdesc{};
  InstanceDesc *d_desc = nullptr;
  int *d_sweep_map = nullptr, *d_fin_map = nullptr;
  int cw = 0;                      // row sweep: chunk width preferred by this context
  int sched_kind = DVM_SWEEP_AUTO, sched_v = 0;  // sweep kernel requested by dvm_set_schedule
  int *d_adj_map = nullptr;        // sweep map of the adjoint launch
  double alpha = 1.0;              // accommodation
  double top_u = 0.0;              // speed of the plate beyond the last row (Couette flow)
  int nwall = 0;
  int *d_wall_slot = nullptr;      // alpha < 1: [ncell][4] face slots (freed with the context)
  void *d_wbuf = nullptr;          // alpha < 1: incident values at the wall faces, two parities
  dvm_batch *self = nullptr;       // batch of this context alone (built on first use)
  std::vector<dvm_batch *> batches; // every live batch that has this context as a member
  DeviceState *h_state = nullptr;  // pinned
  std::string err;
  // adjoint (allocated by the first dvm_adjoint)
  void *a_rec = nullptr, *a_rec_diag = nullptr, *a_seamx = nullptr, *a_seamy = nullptr, *a_z = nullptr;
  double *a_acc = nullptr, *a_flux = nullptr, *a_alpha = nullptr, *a_z1prev = nullptr, *a_grad = nullptr;
  void *a_wbuf = nullptr;          // accommodation < 1: z at the wall faces, two parities (adjoint)
  DeviceState *a_state = nullptr;
  InstanceDesc *a_desc = nullptr;
  cudaGraphExec_t a_graph = nullptr;
  int a_graph_iters = 0;
  // mixed-precision refinement of FP32 storage (dvm_refine.cu): the caller's inputs (to build the FP64
  // twin), the twin, and the state buffers, all created on first use
  std::vector<uint8_t> mask_user;
  std::vector<double> rows_user, delta_user;
  dvm_ctx *twin = nullptr;
  double *r_state = nullptr;       // snapshot [8 ncell + 1] | rho [8 ncell + 1] | scalars [4] | sums [2]
  void *r_seam = nullptr;          // snapshot seams | rho seams, storage precision
  size_t r_nseam = 0;
  bool refine_unavailable = false;
};

// A set of contexts advanced together: one launch of each kernel per sweep, replayed as CUDA graphs.
struct dvm_batch {
  std::vector<dvm_ctx *> ctxs;
  bool fp64 = true, store_h = false, uniform = true;
  int warps = 0, cw = 0, nsweep = 0, nfin = 0;
  int row_tiles = 1;                 // row sweep: most velocity groups a block sweeps side by side
  int kind = DVM_SWEEP_COLUMNS, cols_v = 1;  // resolved sweep schedule of the launch
  int pairing = DVM_PAIRING_AUTO, pair_blocks = 0;  // paired-group policy and the paired blocks planned
  std::vector<int> single_blocks;  // per member: its blocks with one group per warp (pairing decisions)
  bool tail_unpaired = false;      // AUTO: pairs dropped for the tail of the last solve
  bool fixed_plan = false;         // no re-planning (the refinement's correction phase has edited d_descs)
  InstanceDesc *d_descs = nullptr;
  int *d_smap = nullptr, *d_fmap = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t g_many = nullptr;  // m sweeps
  cudaGraphExec_t g_sweep = nullptr; // one sweep kernel (timed single sweeps)
  cudaGraphExec_t g_fin = nullptr;   // the two finalize kernels of that sweep
  int m = 1;
  bool anderson = false;             // some member mixes its iterates (3 more kernels per sweep)
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  bool timed = false;
  std::vector<InstanceDesc> hdescs;  // the members' descriptors as uploaded to d_descs
  bool detached = false;             // a member was destroyed first: device resources released
  // persistent launch: the device scheduler's arrays (one allocation) and its descriptor
  bool persistent = false;
  void *p_mem = nullptr;
  PersistDesc pdesc{};
  int p_blocks = 0;
};

namespace {

dvm_status fail(dvm_ctx *ctx, dvm_status st, const std::string &msg) {
  if (ctx) ctx->err = msg;
  else g_create_error = msg;
  return st;
}

// Stored cell of the caller's cell index ucell = j unx + i: (j, i) when the grid is stored transposed.
inline size_t stored_cell(const dvm_ctx *c, size_t ucell) {
  if (!c->tr) return ucell;
  return (ucell % c->unx) * (size_t)c->nx + ucell / c->unx;
}

// Features that only the column sweep's special variant implements: accommodation < 1, a moving
// plate, columns of unequal width.
inline bool needs_special(const dvm_ctx *c) { return c->alpha < 1.0 || c->top_u != 0.0 || c->nux; }

#define DVM_CUDA(ctx, call)                                                                     \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(ctx, DVM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

constexpr int kFinBlock = 256;

template <typename T>
void build_velocity_tables(const dvm_ctx *c, std::vector<T> &vel, std::vector<T> &inv) {
  const int half = c->half, gq = c->gq;
  vel.assign((size_t)c->ngroups * kNumVelFields * kLanes, T(0));
  inv.assign((size_t)c->ngroups * kInvRows * kLanes, T(0));  // row 9 stays 0 (solid cells)
  const double kap[3] = {1.5, 1.0, 2.0};  // interior, second cell from a wall, next to a wall
  for (int g = 0; g < c->ngroups; ++g) {
    const int q = g / gq, gi = g % gq;
    const double s1 = (q & 1) ? -1.0 : 1.0, s2 = (q & 2) ? -1.0 : 1.0;
    for (int lane = 0; lane < kLanes; ++lane) {
      const int pos = gi * kLanes + lane;
      const bool valid = pos < half * half;
      const int a = valid ? pos / half : 0, b = valid ? pos % half : 0;
      const double v1 = s1 * c->x1[half + a], v2 = s2 * c->x1[half + b];
      const double W = valid ? c->w1[half + a] * c->w1[half + b] : 0.0;
      const double e = v1 * v1 + v2 * v2 - 1.0;
      const double cx = std::fabs(v1) / c->dxs, cy = std::fabs(v2) / c->dys;
      const double z = valid ? 1.0 : 0.0;
      const double f[kNumVelFields] = {v1, v2, e, cx, cy, W, W * v1, W * v2, W * (v1 * v1 + v2 * v2),
                                       std::fabs(v1) * W, std::fabs(v2) * W,
                                       z, z * v1, z * v2, z * (v1 * v1 + v2 * v2)};
      for (int k = 0; k < kNumVelFields; ++k) vel[((size_t)g * kNumVelFields + k) * kLanes + lane] = (T)f[k];
      for (int clx = 0; clx < 3; ++clx)
        for (int cly = 0; cly < 3; ++cly)
          inv[((size_t)g * kInvRows + clx * 3 + cly) * kLanes + lane] = (T)(1.0 / (c->delta + cx * kap[clx] + cy * kap[cly]));
    }
  }
}

// Quadrature sums of the velocity table exactly as the kernels see it (values rounded to the sweep
// precision): the moment weights w_i = (W, W v1, W v2, W |v|^2), the basis the right-hand side is
// built from psi = (1, v1, v2, (|v|^2 - 1) + 1), and the wall-flux weights |v_n| W.  With
// G_ij = sum_k w_i(v_k) psi_j(v_k) and collision coefficients a = G^{-1} m, the collision operator
// L = delta psi . a is the projection onto span(psi) that conserves the kernel's own moments exactly
// (for FP64 tables and an exact quadrature: the delta [rho + 2 u.v + tau (|v|^2 - 1)] of Eq. BGK).
template <typename T>
bool table_sums(const dvm_ctx *c, const std::vector<T> &vel, InstanceDesc &D) {
  double g[4][8] = {};
  // The moment sums are accumulated per quadrant and the quadrants added last: the four quadrants
  // list mirrored velocities in the same lane order, so sums odd in v1 or v2 cancel exactly.
  double gq[4][4][4] = {}, sq[4][4] = {};
  for (int k = 0; k < 4; ++k) D.sumW[k] = D.ain[k] = D.nrm[k] = 0.0;
  for (int grp = 0; grp < c->ngroups; ++grp) {
    const int quad = grp / c->gq;
    for (int lane = 0; lane < kLanes; ++lane) {
      auto f = [&](int field) { return (double)vel[((size_t)grp * kNumVelFields + field) * kLanes + lane]; };
      const double w[4] = {f(kW0), f(kW1), f(kW2), f(kW3)};
      if (w[0] == 0.0) continue;  // padded lane
      const double psi[4] = {1.0, f(kV1), f(kV2), f(kE2m1) + 1.0};
      for (int i = 0; i < 4; ++i) {
        sq[quad][i] += w[i];
        for (int j = 0; j < 4; ++j) gq[quad][i][j] += w[i] * psi[j];
      }
      const double v1 = f(kV1), v2 = f(kV2), wnx = f(kWnx), wny = f(kWny);
      // side W: inward normal +x, outgoing v1 > 0; E: -x; S: +y; N: -y
      (v1 > 0 ? D.nrm[kW] : D.ain[kW]) += wnx;
      (v1 < 0 ? D.nrm[kE] : D.ain[kE]) += wnx;
      (v2 > 0 ? D.nrm[kS] : D.ain[kS]) += wny;
      (v2 < 0 ? D.nrm[kN] : D.ain[kN]) += wny;
    }
  }
  for (int i = 0; i < 4; ++i) {
    D.sumW[i] = (sq[0][i] + sq[1][i]) + (sq[2][i] + sq[3][i]);
    for (int j = 0; j < 4; ++j) g[i][j] = (gq[0][i][j] + gq[1][i][j]) + (gq[2][i][j] + gq[3][i][j]);
  }
  // Gauss-Jordan inverse with partial pivoting (exact zeros of G stay exact zeros of the inverse)
  for (int i = 0; i < 4; ++i) g[i][4 + i] = 1.0;
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(g[r][col]) > std::fabs(g[piv][col])) piv = r;
    if (g[piv][col] == 0.0) return false;
    if (piv != col)
      for (int j = 0; j < 8; ++j) std::swap(g[piv][j], g[col][j]);
    const double d = g[col][col];
    for (int j = 0; j < 8; ++j) g[col][j] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double fr = g[r][col];
      for (int j = 0; j < 8; ++j) g[r][j] -= fr * g[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) D.ginv[i * 4 + j] = g[i][4 + j];
  return true;
}

// Sweep schedule: the row-wavefront kernel with chunk width v (cells per warp and step; 0 = the
// members' own choice) or the column kernel with v threads per column.
struct Schedule {
  int kind = DVM_SWEEP_COLUMNS;
  int v = 1;
  bool persistent = false;  // row sweep only: the persistent batched launch (dvm_persist.cu)
  int pairing = DVM_PAIRING_AUTO;  // FP32 row sweep: paired velocity groups (dvm_batch_set_pairing)
};

// The column sweep needs nx * v <= kColsMaxThreads (a thread per column and velocity subset); the
// row sweep needs ceil(nx / 16) <= 16 rows in flight, i.e. nx <= 256.
bool resolve_schedule(int nx_max, int kind, int v, Schedule *out, std::string *why, bool specular = false) {
  if (kind == DVM_SWEEP_AUTO) kind = DVM_SWEEP_COLUMNS;
  if (kind == DVM_SWEEP_ROWS) {
    if (nx_max > 16 * kMaxSweepWarps) {
      *why = "the row sweep needs nx <= 256";
      return false;
    }
    if (specular) {
      *why = "the row sweep supports fixed, fully diffuse walls on equal rows only (accommodation = 1, no moving "
             "plate, no row heights)";
      return false;
    }
    if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8 && v != 16) {
      *why = "the row sweep's chunk width must be 1, 2, 4, 8 or 16";
      return false;
    }
    if (v != 0 && (nx_max + v - 1) / v > kMaxSweepWarps) {
      *why = "chunk width too small: more than 16 rows in flight";
      return false;
    }
    out->kind = kind;
    out->v = v;
    return true;
  }
  if (kind != DVM_SWEEP_COLUMNS) {
    *why = "unknown sweep kind";
    return false;
  }
  if (v == 0) {
    v = 4;
    while (v > 1 && nx_max * v > kColsMaxThreads) v >>= 1;
  }
  if (v != 1 && v != 2 && v != 4) {
    *why = "threads per column must be 1, 2 or 4";
    return false;
  }
  if (nx_max * v > kColsMaxThreads) {
    *why = "the column sweep needs nx * threads_per_column <= " + std::to_string(kColsMaxThreads);
    return false;
  }
  out->kind = kind;
  out->v = v;
  return true;
}

// Blocks of the column sweep per velocity group: the group's 32 velocities split into parts of
// v threads x cols_g velocities.
int cols_parts(bool fp64, int v) { return kLanes / (v * cols_g(fp64)); }

// Sweep chunk width: the smallest of 1, 2, 4, 8, 16 cells that keeps ceil(nx / cw) rows in flight
// within max_warps (each row in flight is one warp).
int choose_cw(int nx, int max_warps) {
  for (int cw : {1, 2, 4, 8, 16})
    if ((nx + cw - 1) / cw <= max_warps) return cw;
  return 16;
}

template <typename T>
void free_dev(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

void batch_free(dvm_batch *b);

void release_device(dvm_ctx *c) {
  if (c->self) batch_free(c->self);
  c->self = nullptr;
  free_dev(c->d_vel);
  free_dev(c->d_inv);
  free_dev(c->d_rec);
  free_dev(c->d_rec_diag);
  free_dev(c->d_code4);
  free_dev(c->d_hw_src);
  free_dev(c->d_delta_field);
  free_dev(c->d_acc);
  free_dev(c->d_facc);
  free_dev(c->d_mom);
  free_dev(c->d_u1prev);
  free_dev(c->d_seamx);
  free_dev(c->d_seamy);
  free_dev(c->d_h);
  free_dev(c->d_state);
  free_dev(c->d_desc);
  free_dev(c->d_sweep_map);
  free_dev(c->d_fin_map);
  free_dev(c->d_wall_slot);
  free_dev(c->d_wbuf);
  free_dev(c->d_xwidth);
  free_dev(c->d_aa);
  free_dev(c->d_aa_buf);
  free_dev(c->d_aa_meta);
  free_dev(c->d_wallface);
  if (c->h_state) cudaFreeHost(c->h_state);
  c->h_state = nullptr;
  if (c->a_graph) cudaGraphExecDestroy(c->a_graph);
  c->a_graph = nullptr;
  free_dev(c->a_rec);
  free_dev(c->a_rec_diag);
  free_dev(c->a_seamx);
  free_dev(c->a_seamy);
  free_dev(c->a_z);
  free_dev(c->a_acc);
  free_dev(c->a_flux);
  free_dev(c->a_alpha);
  free_dev(c->a_z1prev);
  free_dev(c->a_wbuf);
  free_dev(c->a_grad);
  free_dev(c->a_state);
  free_dev(c->a_desc);
  if (c->twin) dvm_destroy(c->twin);
  c->twin = nullptr;
  free_dev(c->r_state);
  free_dev(c->r_seam);
}

dvm_status reset_state(dvm_ctx *c) {
  const size_t ts = c->fp64 ? 8 : 4;
  DVM_CUDA(c, cudaMemsetAsync(c->d_acc, 0, sizeof(double) * 4 * c->ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->d_facc, 0, sizeof(double) * 8 * c->ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->d_mom, 0, sizeof(double) * 4 * c->ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->d_u1prev, 0, sizeof(double) * c->ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->d_seamx, 0, ts * c->ngroups * c->ny * 2 * kLanes, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->d_seamy, 0, ts * c->ngroups * c->nx * 2 * kLanes, c->stream));
  if (c->d_h) DVM_CUDA(c, cudaMemsetAsync(c->d_h, 0, ts * c->ngroups * (size_t)c->ncell * kLanes, c->stream));
  if (c->d_wbuf)
    DVM_CUDA(c, cudaMemsetAsync(c->d_wbuf, 0, ts * 2 * (size_t)std::max(c->nwall, 1) * 2 * c->gq * kLanes, c->stream));
  if (c->d_aa) {
    // the mixing restarts from the state of h = 0 (x = 0) with an empty history
    DVM_CUDA(c, cudaMemsetAsync(c->d_aa_buf, 0, sizeof(double) * (size_t)c->aa_n, c->stream));
    DVM_CUDA(c, cudaMemsetAsync(c->d_aa_buf + (size_t)(3 + 2 * c->aa_m) * c->aa_n, 0, sizeof(double) * kAARed,
                                c->stream));
    DVM_CUDA(c, cudaMemsetAsync(c->d_aa_meta, 0, sizeof(int) * 3, c->stream));
  }
  DVM_CUDA(c, launch_reset(c->d_desc, c->ncell, c->fp64, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  return DVM_OK;
}

dvm_status upload_desc(dvm_ctx *c) {
  InstanceDesc &D = c->hdesc;
  D.uniform_delta = c->uniform ? 1 : 0;
  D.delta_field = c->d_delta_field;
  DVM_CUDA(c, cudaMemcpyAsync(c->d_desc, &D, sizeof(InstanceDesc), cudaMemcpyHostToDevice, c->stream));
  return DVM_OK;
}

LaunchDesc make_launch(const InstanceDesc *insts, const int *sweep_map, const int *fin_map, int ninst, int warps,
                       int cw, int cols_v = 0, bool specular = false) {
  LaunchDesc L;
  L.cols_v = cols_v;
  L.specular = specular ? 1 : 0;
  L.inst = insts;
  L.sweep_map = sweep_map;
  L.fin_map = fin_map;
  L.ninst = ninst;
  L.warps = warps;
  L.row_tiles = 1;
  L.cw = cw;
  L.pair_smem = 0;
  L.anderson = 0;
  L.aa_blocks = 0;
  return L;
}

// Capture `iters` sweeps of a launch into a graph: each the sweep kernel (when `sweep`) followed by
// the two finalize kernels (when `fin`).
dvm_status capture_graph(dvm_ctx *err_ctx, cudaStream_t cap, const LaunchDesc &L, int sweep_blocks, int fin_blocks,
                         bool fp64, bool uniform, int iters, bool sweep, bool fin, cudaGraphExec_t *out) {
  cudaGraph_t graph = nullptr;
  DVM_CUDA(err_ctx, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    if (sweep) e = launch_sweep(fp64, uniform, L, sweep_blocks, cap);
    if (e == cudaSuccess && fin) e = launch_finalize(L, fin_blocks, fp64, cap);
  }
  cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(err_ctx, DVM_ECUDA,
                std::string("graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(err_ctx, DVM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return DVM_OK;
}

int iters_per_graph(double updates_per_iter) {
  if (updates_per_iter >= 5e7) return 4;
  if (updates_per_iter >= 5e6) return 8;
  if (updates_per_iter >= 5e5) return 16;
  return 32;
}

// The batch's device resources (graphs, events, launch arrays), not the host struct.
void batch_release(dvm_batch *b) {
  if (b->g_many) cudaGraphExecDestroy(b->g_many);
  if (b->g_sweep) cudaGraphExecDestroy(b->g_sweep);
  if (b->g_fin) cudaGraphExecDestroy(b->g_fin);
  for (auto &e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_smap) cudaFree(b->d_smap);
  if (b->d_fmap) cudaFree(b->d_fmap);
  if (b->p_mem) cudaFree(b->p_mem);
  b->g_many = b->g_sweep = b->g_fin = nullptr;
  for (auto &e : b->ev) e = nullptr;
  b->d_descs = nullptr;
  b->d_smap = b->d_fmap = nullptr;
  b->p_mem = nullptr;
}

// Unregister the batch from its members (each member keeps the list of batches it belongs to).
void batch_unlink(dvm_batch *b) {
  for (dvm_ctx *c : b->ctxs) {
    auto &v = c->batches;
    v.erase(std::remove(v.begin(), v.end(), b), v.end());
  }
}

void batch_free(dvm_batch *b) {
  if (!b) return;
  batch_unlink(b);
  batch_release(b);
  delete b;
}

// A member is being destroyed while the batch lives on: release the batch's device resources now,
// while the member's stream still exists; the batch can then only be destroyed (DVM_ESTATE otherwise).
void batch_detach(dvm_batch *b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_unlink(b);
  batch_release(b);
  b->ctxs.clear();
  b->stream = nullptr;
  b->detached = true;
}

constexpr int kPersistSweeps = 64;     // sweeps per instance per persistent launch (members retire early)
constexpr int kPersistFinCells = 4096; // cells per finalize work item of the persistent launch

// The persistent launch of a row-sweep batch: its scheduler arrays and one graph per sweep count.
dvm_status persist_setup(dvm_batch *b, const std::vector<int> &smap, const std::vector<double> &work,
                         const LaunchDesc &L) {
  const int n = (int)b->ctxs.size();
  dvm_ctx *c0 = b->ctxs[0];
  std::vector<int> order(n), base(n), count(n, 0), fin(n), tiles;
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
  for (int i = 0; i < n; ++i) {
    base[i] = (int)tiles.size();
    for (int e : smap)
      if (((e >> 16) & 0x3fff) == i) {
        tiles.push_back(e);
        ++count[i];
      }
    fin[i] = (b->ctxs[i]->ncell + kPersistFinCells - 1) / kPersistFinCells;
  }
  // one allocation: work words (8-byte aligned first), then the int arrays
  const size_t nint = 5 * (size_t)n + tiles.size() + 2;
  const size_t bytes = 8 * (size_t)n + 4 * (size_t)n + 4 * nint;
  DVM_CUDA(c0, cudaMalloc(&b->p_mem, bytes));
  char *m = static_cast<char *>(b->p_mem);
  PersistDesc &P = b->pdesc;
  P.ninst = n;
  P.fin_cells = kPersistFinCells;
  P.work = reinterpret_cast<unsigned long long *>(m);
  P.finished = reinterpret_cast<unsigned int *>(m + 8 * (size_t)n);
  int *ip = reinterpret_cast<int *>(m + 12 * (size_t)n);
  P.left = ip;
  P.active = ip + n;
  P.error = ip + n + 1;
  int *arrays = ip + n + 2;
  std::vector<int> host;
  host.insert(host.end(), order.begin(), order.end());
  host.insert(host.end(), base.begin(), base.end());
  host.insert(host.end(), count.begin(), count.end());
  host.insert(host.end(), fin.begin(), fin.end());
  host.insert(host.end(), tiles.begin(), tiles.end());
  P.order = arrays;
  P.tile_base = arrays + n;
  P.tile_count = arrays + 2 * n;
  P.fin_items = arrays + 3 * n;
  P.tiles = arrays + 4 * n;
  DVM_CUDA(c0, cudaMemsetAsync(b->p_mem, 0, bytes, b->stream));
  DVM_CUDA(c0, cudaMemcpyAsync(arrays, host.data(), sizeof(int) * host.size(), cudaMemcpyHostToDevice, b->stream));
  DVM_CUDA(c0, cudaStreamSynchronize(b->stream));
  int sms = 0;
  DVM_CUDA(c0, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->device));
  const int per_sm = persistent_blocks_per_sm(b->fp64, b->uniform, L);
  if (per_sm < 1) return fail(c0, DVM_EINVAL, "the persistent launch does not fit an SM");
  b->p_blocks = sms * per_sm;
  return DVM_OK;
}

// Capture the persistent launch (arming kernel + scheduler kernel) for `sweeps` sweeps per member.
dvm_status capture_persistent(dvm_batch *b, const LaunchDesc &L, int sweeps, cudaGraphExec_t *out) {
  dvm_ctx *c0 = b->ctxs[0];
  cudaGraph_t graph = nullptr;
  DVM_CUDA(c0, cudaStreamBeginCapture(c0->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_persistent(b->fp64, b->uniform, L, b->pdesc, b->p_blocks, sweeps, c0->cap_stream);
  cudaError_t e2 = cudaStreamEndCapture(c0->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(c0, DVM_ECUDA, std::string("persistent graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(c0, DVM_ECUDA, std::string("persistent graph instantiate: ") + cudaGetErrorString(e));
  return DVM_OK;
}

// Build a batch over ctxs (errors reported on ctxs[0]) with the given sweep schedule, or with the
// first member's requested one.
// DVM_SWEEP_AUTO: the row sweep where it applies (fully diffuse fixed walls, equal rows, nx <= 256) and the
// launch has velocity groups for at least half the SMs; otherwise the column sweep, which spreads a few
// groups over more threads.
int auto_sweep_kind(dvm_ctx *const *ctxs, int n, int nx_max, bool spec) {
  if (spec || nx_max > 16 * kMaxSweepWarps) return DVM_SWEEP_COLUMNS;
  long long groups = 0;
  for (int i = 0; i < n; ++i) groups += ctxs[i]->ngroups;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctxs[0]->device);
  return 2 * groups >= std::max(nsm, 1) ? DVM_SWEEP_ROWS : DVM_SWEEP_COLUMNS;
}

dvm_status batch_build(dvm_ctx *const *ctxs, int n, dvm_batch **out, const Schedule *force = nullptr) {
  if (!ctxs || n < 1 || !ctxs[0]) return DVM_EINVAL;
  dvm_ctx *c0 = ctxs[0];
  if (n > 32767) return fail(c0, DVM_EINVAL, "too many instances in one batch");
  int nx_max = 0;
  bool spec = false;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(c0, DVM_EINVAL, "null context in batch");
    spec = spec || needs_special(ctxs[i]);
    if (ctxs[i]->fp64 != c0->fp64 || ctxs[i]->store_h != c0->store_h)
      return fail(c0, DVM_EINVAL, "batched contexts must share precision and store_distribution");
    if (ctxs[i]->device != c0->device) return fail(c0, DVM_EINVAL, "batched contexts must share a device");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return fail(c0, DVM_EINVAL, "a context appears twice in the batch");
    nx_max = std::max(nx_max, ctxs[i]->nx);
  }
  Schedule sched;
  if (force) {
    sched = *force;
    if (spec && sched.kind == DVM_SWEEP_ROWS)
      return fail(c0, DVM_EINVAL, "the row sweep supports fixed, fully diffuse walls on equal rows only (accommodation = 1, "
                                  "no moving plate, no row heights)");
  } else {
    std::string why;
    const bool automatic = c0->sched_kind == DVM_SWEEP_AUTO;
    const int kind = automatic ? auto_sweep_kind(ctxs, n, nx_max, spec) : c0->sched_kind;
    if (!resolve_schedule(nx_max, kind, automatic ? 0 : c0->sched_v, &sched, &why, spec))
      return fail(c0, DVM_EINVAL, why);
  }
  const bool cols = sched.kind == DVM_SWEEP_COLUMNS;
  dvm_batch *b = new (std::nothrow) dvm_batch();
  if (!b) return fail(c0, DVM_ENOMEM, "host allocation failed");
  b->ctxs.assign(ctxs, ctxs + n);
  b->fp64 = c0->fp64;
  b->store_h = c0->store_h;
  b->stream = c0->stream;
  b->kind = sched.kind;
  b->cols_v = cols ? sched.v : 0;
  // row sweep: one chunk width for the launch, the widest preferred by a member, keeps every member
  // within kMaxSweepWarps rows in flight; the block has as many warps as the widest member needs.
  // Column sweep: ceil(nx / (32 / v)) warps for the widest member.
  b->cw = 1;
  for (int i = 0; i < n; ++i) {
    b->cw = std::max(b->cw, ctxs[i]->cw);
    // the 1/denominator tables hold one value per stencil class: unequal columns need the per-cell form
    b->uniform = b->uniform && ctxs[i]->uniform && !ctxs[i]->nux;
  }
  if (!cols && sched.v > 0) b->cw = sched.v;
  b->warps = 1;
  std::vector<InstanceDesc> descs(n);
  std::vector<int> smap, fmap;
  std::vector<double> work(n);
  double upd = 0.0;
  const int parts = cols ? cols_parts(b->fp64, b->cols_v) : 1;
  for (int i = 0; i < n; ++i) {
    const int need = cols ? (ctxs[i]->nx + kLanes / b->cols_v - 1) / (kLanes / b->cols_v)
                          : (ctxs[i]->nx + b->cw - 1) / b->cw;
    b->warps = std::max(b->warps, need);
    descs[i] = ctxs[i]->hdesc;
    descs[i].uniform_delta = ctxs[i]->uniform ? 1 : 0;
    descs[i].delta_field = ctxs[i]->d_delta_field;
    for (int blk = 0; blk < ctxs[i]->hdesc.fin_nblocks; ++blk) fmap.push_back((i << 16) | blk);
    work[i] = (double)ctxs[i]->ncell;
    upd += (double)ctxs[i]->geo.n_gas * ctxs[i]->nv * ctxs[i]->nv;
  }
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c0->device);
  // Row sweep: a member whose rows in flight fill only part of the block sweeps several of its velocity
  // groups side by side (at most 8, and as many as the shared memory of the launch allows).
  int row_tiles = 1;
  if (!cols) {
    for (int i = 0; i < n; ++i) {
      const int need = (ctxs[i]->nx + b->cw - 1) / b->cw;
      row_tiles = std::max(row_tiles, std::min(std::min(b->warps / need, 8), ctxs[i]->ngroups));
    }
    while (row_tiles > 1 && sweep_smem_bytes(b->fp64, b->warps, b->cw, row_tiles) > (size_t)smem_optin) --row_tiles;
  }
  // Paired groups (FP32 row sweep with a uniform collision rate, per-kernel launches): a member sweeps two
  // velocity groups of a quadrant per warp, k pairs side by side (as many as fill the block's warps and
  // fit the shared memory), when its paired layout fits at all.  Pairing halves the blocks, so it is used
  // only when the launch has at least three waves of single-group blocks (otherwise the SMs it leaves
  // idle cost more than it saves).
  size_t pair_smem = 0;
  std::vector<int> pair_k(n, 0);
  long long single_blocks = 0;
  b->single_blocks.assign(n, 0);
  if (!cols)
    for (int i = 0; i < n; ++i) {
      const int need = (ctxs[i]->nx + b->cw - 1) / b->cw;
      const int k = std::max(1, std::min(b->warps / need, row_tiles));
      b->single_blocks[i] = (ctxs[i]->ngroups + k - 1) / k;
      single_blocks += b->single_blocks[i];
    }
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c0->device);
  b->pairing = sched.pairing;
  if (!cols && !b->fp64 && b->uniform && !spec && n < (1 << 14) &&
      (sched.pairing == DVM_PAIRING_ON ||
       (sched.pairing == DVM_PAIRING_AUTO && single_blocks >= 3LL * std::max(nsm, 1)))) {
    for (int i = 0; i < n; ++i) {
      const int need = (ctxs[i]->nx + b->cw - 1) / b->cw;
      if (ctxs[i]->gq < 2) continue;
      for (int k = std::min(std::min(b->warps / need, ctxs[i]->gq / 2), 7); k >= 1; --k) {
        const size_t bytes = sweep_pair_smem_layout(k * need, b->cw, k).total;
        if (bytes <= (size_t)smem_optin) {
          pair_k[i] = k;
          pair_smem = std::max(pair_smem, bytes);
          break;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    if (cols) {
      for (int g = 0; g < ctxs[i]->ngroups; ++g)
        for (int part = 0; part < parts; ++part) smap.push_back((i << 16) | (part << 12) | g);
    } else if (pair_k[i] > 0) {
      // pairs (g, g + 1) within each quadrant, pair_k of them per block; an odd group left over at the
      // end of a quadrant is swept alone
      const int gq = ctxs[i]->gq, np = gq / 2;
      for (int q = 0; q < 4; ++q) {
        for (int m = 0; m < np; m += pair_k[i]) {
          const int k = std::min(pair_k[i], np - m);
          smap.push_back(kPairFlag | (i << 16) | (k << 12) | (q * gq + 2 * m));
        }
        if (gq & 1) smap.push_back((i << 16) | (1 << 12) | (q * gq + gq - 1));
      }
    } else {
      const int need = (ctxs[i]->nx + b->cw - 1) / b->cw;
      const int k = std::max(1, std::min(b->warps / need, row_tiles));
      for (int g = 0; g < ctxs[i]->ngroups; g += k) smap.push_back((i << 16) | (k << 12) | g);
    }
  }
  b->pair_blocks = (int)std::count_if(smap.begin(), smap.end(), [](int e) { return (e & kPairFlag) != 0; });
  // longest sweeps first
  std::stable_sort(smap.begin(), smap.end(),
                   [&](int a, int c) { return work[(a >> 16) & 0x3fff] > work[(c >> 16) & 0x3fff]; });
  b->nsweep = (int)smap.size();
  b->nfin = (int)fmap.size();
  b->row_tiles = row_tiles;
  size_t smem = cols ? cols_smem_bytes(b->fp64, b->cols_v, b->warps)
                     : sweep_smem_bytes(b->fp64, b->warps, b->cw, row_tiles);
  smem = std::max(smem, pair_smem);
  if ((!cols && b->warps > kMaxSweepWarps) || (cols && b->warps * kLanes > kColsMaxThreads) || smem > (size_t)smem_optin) {
    batch_free(b);
    return fail(c0, DVM_EINVAL, "batched grids too wide for the sweep's shared memory");
  }
#define BATCH_CUDA(call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      batch_free(b);                                                                             \
      return fail(c0, DVM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    }                                                                                            \
  } while (0)
  b->hdescs = descs;
  BATCH_CUDA(cudaMalloc(&b->d_descs, sizeof(InstanceDesc) * n));
  BATCH_CUDA(cudaMalloc(&b->d_smap, sizeof(int) * smap.size()));
  BATCH_CUDA(cudaMalloc(&b->d_fmap, sizeof(int) * fmap.size()));
  BATCH_CUDA(cudaMemcpyAsync(b->d_descs, descs.data(), sizeof(InstanceDesc) * n, cudaMemcpyHostToDevice, b->stream));
  BATCH_CUDA(cudaMemcpyAsync(b->d_smap, smap.data(), sizeof(int) * smap.size(), cudaMemcpyHostToDevice, b->stream));
  BATCH_CUDA(cudaMemcpyAsync(b->d_fmap, fmap.data(), sizeof(int) * fmap.size(), cudaMemcpyHostToDevice, b->stream));
  // row-sweep launches write only the row-major records: a column-sweep launch starts from a copy
  if (cols)
    for (int i = 0; i < n; ++i) BATCH_CUDA(launch_sync_diag(ctxs[i]->d_desc, ctxs[i]->ncell, b->fp64, b->stream));
  BATCH_CUDA(cudaStreamSynchronize(b->stream));
  for (auto &e : b->ev) BATCH_CUDA(cudaEventCreate(&e));
#undef BATCH_CUDA
  LaunchDesc L = make_launch(b->d_descs, b->d_smap, b->d_fmap, n, b->warps, b->cw, b->cols_v, spec);
  L.row_tiles = b->row_tiles;
  L.pair_smem = (int)pair_smem;
  {
    long long aa_max = 0;
    for (int i = 0; i < n; ++i) aa_max = std::max(aa_max, ctxs[i]->aa_n);
    b->anderson = aa_max > 0;
    L.anderson = b->anderson ? 1 : 0;
    // about 8 elements per thread, at most 1024 blocks per instance
    L.aa_blocks = (int)std::min<long long>(1024, std::max<long long>(1, (aa_max + 2047) / 2048));
  }
  if (sched.persistent) {
    if (cols || b->anderson || spec) {
      batch_free(b);
      return fail(c0, DVM_EINVAL, "the persistent launch runs the row sweep with fully diffuse fixed walls, equal rows "
                                  "and the plain iteration (no mixing)");
    }
    b->persistent = true;
    dvm_status st = persist_setup(b, smap, work, L);
    if (st == DVM_OK) {
      b->m = kPersistSweeps;
      st = capture_persistent(b, L, b->m, &b->g_many);
    }
    if (st == DVM_OK) st = capture_persistent(b, L, 1, &b->g_sweep);
    if (st != DVM_OK) {
      batch_free(b);
      return st;
    }
    for (dvm_ctx *c : b->ctxs) c->batches.push_back(b);
    *out = b;
    return DVM_OK;
  }
  b->m = iters_per_graph(upd);
  dvm_status st = capture_graph(c0, c0->cap_stream, L, b->nsweep, b->nfin, b->fp64, b->uniform, b->m, true, true,
                                &b->g_many);
  if (st == DVM_OK)
    st = capture_graph(c0, c0->cap_stream, L, b->nsweep, b->nfin, b->fp64, b->uniform, 1, true, false, &b->g_sweep);
  if (st == DVM_OK)
    st = capture_graph(c0, c0->cap_stream, L, b->nsweep, b->nfin, b->fp64, b->uniform, 1, false, true, &b->g_fin);
  if (st != DVM_OK) {
    batch_free(b);
    return st;
  }
  for (dvm_ctx *c : b->ctxs) c->batches.push_back(b);
  *out = b;
  return DVM_OK;
}

// Rebuild the launch of an existing batch for another schedule; the members' state is untouched.
dvm_status batch_replan(dvm_batch *b, const Schedule &sched, int pairing_override = -1) {
  dvm_batch *nb = nullptr;
  dvm_ctx *c0 = b->ctxs[0];
  DVM_CUDA(c0, cudaStreamSynchronize(b->stream));
  Schedule s2 = sched;
  // the batch's pairing policy outlives schedule changes (an override plans one launch without
  // changing the policy)
  s2.pairing = pairing_override >= 0 ? pairing_override : b->pairing;
  const int policy = b->pairing;
  dvm_status st = batch_build(b->ctxs.data(), (int)b->ctxs.size(), &nb, &s2);
  if (st == DVM_OK) nb->pairing = policy;
  if (st != DVM_OK) return st;
  std::swap(*b, *nb);
  batch_free(nb);
  return DVM_OK;
}

dvm_status batch_poll(dvm_batch *b, bool *all_done) {
  dvm_ctx *c0 = b->ctxs[0];
  for (dvm_ctx *c : b->ctxs)
    DVM_CUDA(c0, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, b->stream));
  int perr = 0;
  if (b->persistent) DVM_CUDA(c0, cudaMemcpyAsync(&perr, b->pdesc.error, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  DVM_CUDA(c0, cudaStreamSynchronize(b->stream));
  if (perr) return fail(c0, DVM_ETIMEOUT, "persistent launch: an idle block gave up waiting for work");
  bool all = true;
  for (dvm_ctx *c : b->ctxs) all = all && c->h_state->done;
  *all_done = all;
  return DVM_OK;
}

// Arm every member for `count` more sweeps with the given tolerance; returns the start iterations.
dvm_status batch_arm(dvm_batch *b, double tol, int count, std::vector<int> &start) {
  dvm_ctx *c0 = b->ctxs[0];
  for (dvm_ctx *c : b->ctxs)
    if (c->stream != b->stream) DVM_CUDA(c0, cudaStreamSynchronize(c->stream));
  for (dvm_ctx *c : b->ctxs)
    DVM_CUDA(c0, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, b->stream));
  DVM_CUDA(c0, cudaStreamSynchronize(b->stream));
  start.resize(b->ctxs.size());
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    start[i] = b->ctxs[i]->h_state->iter;
    const long long limit = (long long)start[i] + count;
    if (limit > 2000000000LL) return fail(c0, DVM_EINVAL, "iteration limit too large");
    DVM_CUDA(c0, launch_arm(b->ctxs[i]->d_state, tol, (int)limit, b->stream));
  }
  return DVM_OK;
}

// The schedule a batch was planned with (for re-planning it).
Schedule batch_schedule(const dvm_batch *b) {
  Schedule sc;
  sc.kind = b->kind;
  sc.v = b->kind == DVM_SWEEP_ROWS ? b->cw : b->cols_v;
  sc.persistent = b->persistent;
  return sc;
}

// AUTO pairing is planned for every member; once the members still iterating no longer fill three waves
// of single-group blocks, the rest of the solve runs without pairs (re-planned; the state is untouched).
dvm_status batch_unpair_tail(dvm_batch *b) {
  if (b->fixed_plan || b->pairing != DVM_PAIRING_AUTO || b->pair_blocks == 0) return DVM_OK;
  long long active = 0;
  for (size_t i = 0; i < b->ctxs.size(); ++i)
    if (!b->ctxs[i]->h_state->done) active += b->single_blocks[i];
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->ctxs[0]->device);
  if (active >= 3LL * std::max(nsm, 1)) return DVM_OK;
  dvm_status st = batch_replan(b, batch_schedule(b), DVM_PAIRING_OFF);
  if (st == DVM_OK) b->tail_unpaired = true;
  return st;
}

dvm_status batch_run(dvm_batch *b, double tol, int max_iter, dvm_status *per, int *iters, double *est) {
  dvm_ctx *c0 = b->ctxs[0];
  if (max_iter < 1) return fail(c0, DVM_EINVAL, "max_iter must be >= 1");
  if (b->tail_unpaired && !b->fixed_plan) {
    // a new solve starts with every member: plan the pairs again
    dvm_status st = batch_replan(b, batch_schedule(b));
    if (st != DVM_OK) return st;
  }
  std::vector<int> start;
  dvm_status st = batch_arm(b, tol, max_iter, start);
  if (st != DVM_OK) return st;
  // every member is armed to stop after max_iter sweeps, so the loop ends after at most
  // ceil(max_iter / m) replays; the bound below only guards against a flag that is never set
  const long long max_replays = (long long)max_iter / b->m + 3;
  for (long long replay = 0;; ++replay) {
    if (replay >= max_replays) return fail(c0, DVM_ETIMEOUT, "device stop flag not set after max_iter sweeps");
    DVM_CUDA(c0, cudaGraphLaunch(b->g_many, b->stream));
    bool all = false;
    st = batch_poll(b, &all);
    if (st != DVM_OK) return st;
    if (all) break;
    st = batch_unpair_tail(b);
    if (st != DVM_OK) return st;
  }
  dvm_status result = DVM_OK;
  for (size_t i = 0; i < b->ctxs.size(); ++i) {
    const dvm_status si = (dvm_status)b->ctxs[i]->h_state->status;
    if (per) per[i] = si;
    if (si != DVM_OK && result == DVM_OK) result = si;
  }
  if (iters) *iters = c0->h_state->iter - start[0];
  if (est) *est = c0->h_state->est;
  b->timed = false;
  return result;
}

dvm_status batch_iterate(dvm_batch *b, int n) {
  dvm_ctx *c0 = b->ctxs[0];
  if (n < 1) return fail(c0, DVM_EINVAL, "n must be >= 1");
  std::vector<int> start;
  dvm_status st = batch_arm(b, -1.0, n, start);
  if (st != DVM_OK) return st;
  int left = n;
  while (left >= b->m && b->m > 1) {
    DVM_CUDA(c0, cudaGraphLaunch(b->g_many, b->stream));
    left -= b->m;
  }
  for (; left > 0; --left) {
    // single sweeps: stream events around the sweep and the finalize kernels time them
    DVM_CUDA(c0, cudaEventRecord(b->ev[0], b->stream));
    DVM_CUDA(c0, cudaGraphLaunch(b->g_sweep, b->stream));
    DVM_CUDA(c0, cudaEventRecord(b->ev[1], b->stream));
    // (the persistent launch finalizes inside g_sweep)
    if (b->g_fin) DVM_CUDA(c0, cudaGraphLaunch(b->g_fin, b->stream));
    DVM_CUDA(c0, cudaEventRecord(b->ev[2], b->stream));
  }
  bool all = false;
  st = batch_poll(b, &all);
  if (st != DVM_OK) return st;
  for (dvm_ctx *c : b->ctxs) {
    const int s = c->h_state->status;
    if (s != DVM_OK && s != DVM_ENOCONV) return fail(c0, (dvm_status)s, "a batch member failed during iteration");
  }
  b->timed = (n == 1) || (n % b->m != 0) || b->m == 1;
  return DVM_OK;
}

dvm_status ensure_self(dvm_ctx *c) {
  if (c->self) return DVM_OK;
  dvm_ctx *one[1] = {c};
  return batch_build(one, 1, &c->self);
}

// ------------------------------------------------------------------------------------------------
// Mixed-precision refinement of FP32 storage (kernels and the method in dvm_refine.cu).

constexpr double kCorrectionTol = 1e-2;  // relative tolerance of each correction solve (on |d|)

// Doubles per state region of the refinement buffers: 8 ncell + 1 rounded up to a multiple of four.
size_t refine_state_stride(int ncell) { return ((size_t)8 * ncell + 1 + 3) & ~(size_t)3; }

// The FP64 twin of an FP32 context (same grid, walls, drive, collision-rate field) and the state buffers.
dvm_status ensure_refine(dvm_ctx *c) {
  if (c->refine_unavailable) return DVM_EINVAL;
  if (!c->twin) {
    dvm_params P = c->P;
    P.precision = DVM_FP64;
    P.store_distribution = 0;
    P.anderson_depth = 0;
    P.fp32_refine = 0;
    P.row_heights = c->rows_user.empty() ? nullptr : c->rows_user.data();
    const std::string saved = g_create_error;
    dvm_ctx *t = nullptr;
    dvm_status st = dvm_create(c->mask_user.data(), &P, c->stream, &t);
    if (st != DVM_OK) {
      c->refine_unavailable = true;
      c->err = "refinement unavailable: the FP64 twin could not be created (" + g_create_error + ")";
      g_create_error = saved;
      return st;
    }
    if (!c->uniform) {
      st = dvm_set_delta_field(t, c->delta_user.data());
      if (st != DVM_OK) {
        dvm_destroy(t);
        c->refine_unavailable = true;
        return st;
      }
    }
    c->twin = t;
  }
  if (!c->r_state) {
    c->r_nseam = refine_seam_count(c->hdesc);
    DVM_CUDA(c, cudaMalloc(&c->r_state, sizeof(double) * (2 * refine_state_stride(c->ncell) + 8)));
    DVM_CUDA(c, cudaMalloc(&c->r_seam, (c->fp64 ? 8 : 4) * std::max<size_t>(2 * c->r_nseam, 1)));
  }
  return DVM_OK;
}

// After an FP32 batch has converged: up to fp32_refine passes of residual (FP64 twin sweep), correction
// solve (FP32, no drive, residual injected after each projection) and update.  Members whose walls are
// partially specular, or whose twin cannot be built, leave the batch unrefined (DVM_OK).
dvm_status batch_refine(dvm_batch *b, double tol, int max_iter) {
  if (b->fp64 || b->ctxs.empty()) return DVM_OK;
  dvm_ctx *c0 = b->ctxs[0];
  int passes = 0;
  for (dvm_ctx *c : b->ctxs) {
    if (c->alpha < 1.0 || c->P.fp32_refine <= 0) return DVM_OK;
    passes = std::max(passes, c->P.fp32_refine);
  }
  for (dvm_ctx *c : b->ctxs)
    if (ensure_refine(c) != DVM_OK) return DVM_OK;
  const int n = (int)b->ctxs.size();
  std::vector<dvm_ctx *> tw(n);
  for (int i = 0; i < n; ++i) tw[i] = b->ctxs[i]->twin;
  dvm_batch *tb = nullptr;
  dvm_status st = batch_build(tw.data(), n, &tb);
  if (st != DVM_OK) {
    c0->err = "refinement: " + tw[0]->err;
    return st;
  }
  cudaStream_t s = b->stream;
  auto bufs = [&](dvm_ctx *c, double **snap, double **rho, double **sc, double **sums, void **sseam, void **rseam) {
    // the kernels read the moment part of snapshot and rho as 32-byte vectors: every region starts on a
    // multiple of four doubles (the allocation itself is 256-byte aligned)
    const size_t nstate = refine_state_stride(c->ncell);
    *snap = c->r_state;
    *rho = c->r_state + nstate;
    *sc = c->r_state + 2 * nstate;
    *sums = c->r_state + 2 * nstate + 4;
    *sseam = c->r_seam;
    *rseam = static_cast<char *>(c->r_seam) + 4 * c->r_nseam;
  };
  std::vector<double> sums(2 * n), first(n, 0.0);
  dvm_status result = DVM_OK;
  for (int pass = 0; pass < passes && result == DVM_OK; ++pass) {
    for (int i = 0; i < n; ++i) {
      dvm_ctx *c = b->ctxs[i];
      double *snap, *rho, *sc, *sm;
      void *sseam, *rseam;
      bufs(c, &snap, &rho, &sc, &sm, &sseam, &rseam);
      DVM_CUDA(c0, launch_refine_snapshot(b->d_descs + i, b->hdescs[i], false, snap, sseam, sc, s));
      DVM_CUDA(c0, launch_refine_load_twin(b->d_descs + i, tb->d_descs + i, b->hdescs[i], false, s));
      DVM_CUDA(c0, launch_records(tb->d_descs + i, c->ncell, true, s));
    }
    DVM_CUDA(c0, cudaStreamSynchronize(s));
    st = batch_iterate(tb, 1);  // rho = G(x~) - x~ needs one FP64 sweep from x~
    if (st != DVM_OK) {
      c0->err = "refinement residual sweep: " + tw[0]->err;
      result = st;
      break;
    }
    for (int i = 0; i < n; ++i) {
      dvm_ctx *c = b->ctxs[i];
      double *snap, *rho, *sc, *sm;
      void *sseam, *rseam;
      bufs(c, &snap, &rho, &sc, &sm, &sseam, &rseam);
      DVM_CUDA(c0, launch_refine_residual(b->d_descs + i, tb->d_descs + i, b->hdescs[i], false, snap, sseam, sc, rho,
                                          rseam, s));
      // the correction phase: the member's descriptor without drive and with rho, its state d = 0
      InstanceDesc cd = b->hdescs[i];
      cd.force = 0.0;
      cd.top_u = 0.0;
      cd.rho = rho;
      cd.rho_seam_x = rseam;
      cd.rho_seam_y = static_cast<char *>(rseam) + 4 * (cd.periodic_x ? (size_t)c->ngroups * c->ny * 2 * kLanes : 0);
      DVM_CUDA(c0, cudaMemcpyAsync(b->d_descs + i, &cd, sizeof(InstanceDesc), cudaMemcpyHostToDevice, s));
      const size_t ts = 4;
      DVM_CUDA(c0, cudaMemsetAsync(c->d_acc, 0, sizeof(double) * 4 * c->ncell, s));
      DVM_CUDA(c0, cudaMemsetAsync(c->d_facc, 0, sizeof(double) * 8 * c->ncell, s));
      DVM_CUDA(c0, cudaMemsetAsync(c->d_mom, 0, sizeof(double) * 4 * c->ncell, s));
      DVM_CUDA(c0, cudaMemsetAsync(c->d_u1prev, 0, sizeof(double) * c->ncell, s));
      DVM_CUDA(c0, cudaMemsetAsync(c->d_seamx, 0, ts * c->ngroups * c->ny * 2 * kLanes, s));
      DVM_CUDA(c0, cudaMemsetAsync(c->d_seamy, 0, ts * c->ngroups * c->nx * 2 * kLanes, s));
      DVM_CUDA(c0, launch_reset(b->d_descs + i, c->ncell, false, s));
    }
    DVM_CUDA(c0, cudaStreamSynchronize(s));
    std::vector<dvm_status> per(n);
    b->fixed_plan = true;  // the members' descriptors on the device are the correction phase's
    st = batch_run(b, kCorrectionTol, max_iter, per.data(), nullptr, nullptr);
    b->fixed_plan = false;
    // back to the members' own descriptors, then x = x~ + d and the records of x with the full drive
    for (int i = 0; i < n; ++i)
      DVM_CUDA(c0, cudaMemcpyAsync(b->d_descs + i, &b->hdescs[i], sizeof(InstanceDesc), cudaMemcpyHostToDevice, s));
    if (st != DVM_OK && st != DVM_ENOCONV) {
      result = st;
      break;
    }
    for (int i = 0; i < n; ++i) {
      dvm_ctx *c = b->ctxs[i];
      double *snap, *rho, *sc, *sm;
      void *sseam, *rseam;
      bufs(c, &snap, &rho, &sc, &sm, &sseam, &rseam);
      DVM_CUDA(c0, launch_refine_combine(b->d_descs + i, b->hdescs[i], false, snap, sseam, sc, rho, sm, s));
      DVM_CUDA(c0, launch_records(b->d_descs + i, c->ncell, false, s));
      DVM_CUDA(c0, cudaMemcpyAsync(&sums[2 * i], sm, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    DVM_CUDA(c0, cudaStreamSynchronize(s));
    // Error left after this pass: the correction solve's own tolerance and the FP32 rounding it
    // amplifies, both relative to |d|; the rounding part is at most |d_1| / |x| (the first correction
    // carries the whole amplified rounding of the FP32 fixed point).  Stop when, with a factor 10 of
    // margin, that is below tol for every member; the estimate is stored as the solve's est.
    double worst = 0.0;
    std::vector<double> est(n);
    for (int i = 0; i < n; ++i) {
      const double rel = sums[2 * i + 1] > 0.0 ? sums[2 * i] / sums[2 * i + 1] : 0.0;
      if (pass == 0) first[i] = rel;
      est[i] = rel * (kCorrectionTol + first[i]);
      worst = std::max(worst, 10.0 * est[i]);
      DVM_CUDA(c0, cudaMemcpyAsync(&b->ctxs[i]->d_state->est, &est[i], sizeof(double), cudaMemcpyHostToDevice, s));
    }
    DVM_CUDA(c0, cudaStreamSynchronize(s));
    if (worst < tol) break;
  }
  batch_free(tb);
  if (result != DVM_OK) return result;
  if (b->store_h) {
    // the stored distribution: one more (plain) sweep from the refined state, whose own rounding is
    // about 1e-7 relative; the refined estimate is kept
    std::vector<double> est(n);
    for (int i = 0; i < n; ++i)
      DVM_CUDA(c0, cudaMemcpyAsync(&est[i], &b->ctxs[i]->d_state->est, sizeof(double), cudaMemcpyDeviceToHost, s));
    DVM_CUDA(c0, cudaStreamSynchronize(s));
    st = batch_iterate(b, 1);
    if (st != DVM_OK) return st;
    for (int i = 0; i < n; ++i)
      DVM_CUDA(c0, cudaMemcpyAsync(&b->ctxs[i]->d_state->est, &est[i], sizeof(double), cudaMemcpyHostToDevice, s));
    DVM_CUDA(c0, cudaStreamSynchronize(s));
  }
  return DVM_OK;
}

}  // namespace

extern "C" {

dvm_status dvm_params_init(dvm_params *p) {
  if (!p) return DVM_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->nx = 0;
  p->ny = 0;
  p->periodic_x = 1;
  p->periodic_y = 0;
  p->ly = 1.0;
  p->kn = 0.1;
  p->delta = -1.0;
  p->quad.kind = DVM_QUAD_GAUSS_HERMITE;
  p->quad.n = 12;
  p->quad.vmax = 5.0;
  p->accommodation = 1.0;
  p->precision = DVM_FP64;
  p->force = 1.0;
  p->store_distribution = 0;
  p->sweep_warps = 0;
  p->top_wall_u1 = 0.0;
  p->storage = DVM_STORAGE_AUTO;
  p->fp32_refine = 3;
  return DVM_OK;
}

const char *dvm_status_string(dvm_status s) {
  switch (s) {
    case DVM_OK: return "DVM_OK";
    case DVM_EINVAL: return "DVM_EINVAL";
    case DVM_ENOMEM: return "DVM_ENOMEM";
    case DVM_ECUDA: return "DVM_ECUDA";
    case DVM_ENOCONV: return "DVM_ENOCONV";
    case DVM_ETIMEOUT: return "DVM_ETIMEOUT";
    case DVM_ENUMERIC: return "DVM_ENUMERIC";
    case DVM_ESTATE: return "DVM_ESTATE";
  }
  return "DVM_UNKNOWN";
}

const char *dvm_last_error(const dvm_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

dvm_status dvm_create(const uint8_t *mask, const dvm_params *params, void *stream, dvm_ctx **out) {
  if (!mask || !params || !out) return fail(nullptr, DVM_EINVAL, "null argument");
  const dvm_params &P = *params;
  if (P.nx < 2 || P.ny < 2 || P.nx > 65536 || P.ny > 65536)
    return fail(nullptr, DVM_EINVAL, "nx and ny must be in [2, 65536]");
  // the finalize launch maps hold 16 bits of 256-cell blocks per instance
  if ((long long)P.nx * P.ny > 65535LL * 256) return fail(nullptr, DVM_EINVAL, "at most 16,776,960 cells");
  if (!(P.ly > 0.0) || !std::isfinite(P.ly)) return fail(nullptr, DVM_EINVAL, "ly must be positive");
  if (!(P.accommodation >= 0.0 && P.accommodation <= 1.0))
    return fail(nullptr, DVM_EINVAL, "accommodation must be in [0, 1]");
  if (!std::isfinite(P.top_wall_u1)) return fail(nullptr, DVM_EINVAL, "top_wall_u1 must be finite");
  if (P.top_wall_u1 != 0.0 && P.periodic_y)
    return fail(nullptr, DVM_EINVAL, "a moving top plate needs a non-periodic x2 axis");
  if (P.precision != DVM_FP64 && P.precision != DVM_FP32_ACC64) return fail(nullptr, DVM_EINVAL, "bad precision");
  if (!std::isfinite(P.force)) return fail(nullptr, DVM_EINVAL, "force must be finite");
  double delta;
  if (P.kn > 0.0) {
    if (P.delta >= 0.0) return fail(nullptr, DVM_EINVAL, "set exactly one of kn and delta");
    delta = std::isinf(P.kn) ? 0.0 : std::sqrt(M_PI) / (2.0 * P.kn);
  } else if (P.delta >= 0.0 && std::isfinite(P.delta)) {
    delta = P.delta;
  } else {
    return fail(nullptr, DVM_EINVAL, "set exactly one of kn (> 0) and delta (>= 0)");
  }
  if (P.sweep_warps < 0 || P.sweep_warps > kMaxWarps) return fail(nullptr, DVM_EINVAL, "sweep_warps must be 0..32");
  if (P.storage != DVM_STORAGE_AUTO && P.storage != DVM_STORAGE_AS_GIVEN && P.storage != DVM_STORAGE_TRANSPOSED)
    return fail(nullptr, DVM_EINVAL, "storage must be DVM_STORAGE_AUTO, _AS_GIVEN or _TRANSPOSED");
  if (!(P.dx1 >= 0.0) || !std::isfinite(P.dx1)) return fail(nullptr, DVM_EINVAL, "dx1 must be finite and >= 0");
  if (P.anderson_depth < 0 || P.anderson_depth > kAAMaxDepth)
    return fail(nullptr, DVM_EINVAL, "anderson_depth must be 0.." + std::to_string(kAAMaxDepth));
  if (P.fp32_refine < 0 || P.fp32_refine > 8) return fail(nullptr, DVM_EINVAL, "fp32_refine must be 0..8");
  if (P.anderson_depth > 0 && P.accommodation < 1.0)
    return fail(nullptr, DVM_EINVAL, "Anderson mixing needs fully diffuse walls (accommodation = 1)");
  if (P.anderson_depth > 0 && P.precision != DVM_FP64)
    return fail(nullptr, DVM_EINVAL, "Anderson mixing needs FP64 storage (FP32 rounding pollutes its history)");
  double ly = P.ly;
  if (P.row_heights) {
    if (!(P.dx1 > 0.0)) return fail(nullptr, DVM_EINVAL, "row heights need the x1 spacing dx1 > 0");
    if (P.storage == DVM_STORAGE_AS_GIVEN)
      return fail(nullptr, DVM_EINVAL, "row heights need the transposed storage (DVM_STORAGE_AUTO or _TRANSPOSED)");
    ly = 0.0;
    for (int j = 0; j < P.ny; ++j) {
      if (!(P.row_heights[j] > 0.0) || !std::isfinite(P.row_heights[j]))
        return fail(nullptr, DVM_EINVAL, "row heights must be finite and > 0");
      ly += P.row_heights[j];
    }
  }

  dvm_ctx *c = new (std::nothrow) dvm_ctx();
  if (!c) return fail(nullptr, DVM_ENOMEM, "host allocation failed");
  c->P = P;
  c->P.row_heights = nullptr;  // the caller's array is read here only (a copy is kept for the FP64 twin)
  c->mask_user.assign(mask, mask + (size_t)P.nx * P.ny);
  if (P.row_heights) c->rows_user.assign(P.row_heights, P.row_heights + P.ny);
  // the sweeps run along the stored x2 (column sweep: one thread per stored column; row sweep: rows in
  // flight across the stored x1), so a grid wider than tall is stored transposed by default
  // (row heights: the caller's x2 becomes the stored x1, along which every sweep thread owns a column)
  c->tr = P.storage == DVM_STORAGE_TRANSPOSED || (P.storage == DVM_STORAGE_AUTO && (P.nx > P.ny || P.row_heights));
  c->unx = P.nx;
  c->uny = P.ny;
  c->nx = c->tr ? P.ny : P.nx;
  c->ny = c->tr ? P.nx : P.ny;
  c->ncell = P.nx * P.ny;
  {
    // caller's spacings: x1 uniform (dx1, or square cells ly / ny), x2 the mean row height ly / ny
    const double udy = ly / P.ny, udx = P.dx1 > 0.0 ? P.dx1 : udy;
    c->dxs = c->tr ? udy : udx;
    c->dys = c->tr ? udx : udy;
    c->nux = P.row_heights != nullptr;
  }
  c->fp64 = P.precision == DVM_FP64;
  c->store_h = P.store_distribution != 0;
  c->alpha = P.accommodation;
  c->top_u = P.top_wall_u1;
  c->delta = delta;
  c->kn = P.kn > 0.0 ? P.kn : (delta > 0 ? std::sqrt(M_PI) / (2.0 * delta) : INFINITY);
  std::string qerr;
  if (!quadrature_1d(P.quad.kind, P.quad.n, P.quad.vmax, c->x1, c->w1, qerr)) {
    delete c;
    return fail(nullptr, DVM_EINVAL, qerr);
  }
  c->nv = P.quad.n;
  c->half = c->nv / 2;
  c->gq = (c->half * c->half + kLanes - 1) / kLanes;
  c->ngroups = 4 * c->gq;
  const bool spx = (c->tr ? P.periodic_y : P.periodic_x) != 0, spy = (c->tr ? P.periodic_x : P.periodic_y) != 0;
  if (c->tr) {
    std::vector<uint8_t> tmask((size_t)c->ncell);
    for (int j = 0; j < c->uny; ++j)
      for (int i = 0; i < c->unx; ++i) tmask[(size_t)i * c->nx + j] = mask[(size_t)j * c->unx + i];
    build_geometry(tmask.data(), c->nx, c->ny, spx, spy, true, c->geo);
  } else {
    build_geometry(mask, c->nx, c->ny, spx, spy, false, c->geo);
  }
  if (c->geo.n_gas == 0) {
    delete c;
    return fail(nullptr, DVM_EINVAL, "the mask has no gas cell");
  }
  const int max_warps = P.sweep_warps > 0 ? std::min(P.sweep_warps, kMaxSweepWarps) : kMaxSweepWarps;
  c->cw = choose_cw(c->nx, max_warps);
  {
    Schedule sc;
    std::string why;
    if (!resolve_schedule(c->nx, DVM_SWEEP_AUTO, 0, &sc, &why)) {
      delete c;
      return fail(nullptr, DVM_EINVAL, "grid too wide: " + why);
    }
  }
  // the automatic schedule (the column sweep) must fit; the row sweep is checked when chosen
  const size_t smem = cols_smem_bytes(c->fp64, 1, (c->nx + kLanes - 1) / kLanes);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, DVM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  c->device = dev;
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)smem_optin) {
    delete c;
    return fail(nullptr, DVM_EINVAL,
                "grid too wide for the sweep's shared-memory ring (" + std::to_string(smem) + " > " +
                    std::to_string(smem_optin) + " bytes); use fewer columns nx or FP32 storage");
  }
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return fail(nullptr, DVM_ECUDA, "cudaStreamCreate failed");
    }
    c->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return fail(nullptr, DVM_ECUDA, "cudaStreamCreate failed");
  }

  auto cleanup_fail = [&](dvm_status st, const std::string &msg) {
    g_create_error = msg;
    release_device(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    cudaStreamDestroy(c->cap_stream);
    delete c;
    return st;
  };
#define CREATE_CUDA(call)                                                                                   \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess) {                                                                                \
      return cleanup_fail(e_ == cudaErrorMemoryAllocation ? DVM_ENOMEM : DVM_ECUDA,                         \
                          std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                                       \
  } while (0)

  const size_t ts = c->fp64 ? 8 : 4;
  const size_t recsz = c->fp64 ? sizeof(SweepRec<double>) : sizeof(SweepRec<float>);
  const size_t ncell = (size_t)c->ncell;
  CREATE_CUDA(cudaMalloc(&c->d_vel, ts * c->ngroups * kNumVelFields * kLanes));
  CREATE_CUDA(cudaMalloc(&c->d_inv, ts * c->ngroups * kInvRows * kLanes));
  CREATE_CUDA(cudaMalloc(&c->d_rec, recsz * 4 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_rec_diag, recsz * 4 * diag_quadrant_size(c->nx, c->ny)));
  CREATE_CUDA(cudaMalloc(&c->d_code4, sizeof(uint32_t) * 4 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_hw_src, sizeof(int) * 8 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_delta_field, sizeof(double) * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_acc, sizeof(double) * 4 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_facc, sizeof(double) * 8 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_mom, sizeof(double) * 4 * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_u1prev, sizeof(double) * ncell));
  CREATE_CUDA(cudaMalloc(&c->d_seamx, ts * c->ngroups * c->ny * 2 * kLanes));
  CREATE_CUDA(cudaMalloc(&c->d_seamy, ts * c->ngroups * c->nx * 2 * kLanes));
  if (c->store_h) CREATE_CUDA(cudaMalloc(&c->d_h, ts * c->ngroups * ncell * kLanes));
  CREATE_CUDA(cudaMalloc(&c->d_state, sizeof(DeviceState)));
  CREATE_CUDA(cudaMalloc(&c->d_desc, sizeof(InstanceDesc)));
  CREATE_CUDA(cudaMallocHost(&c->h_state, sizeof(DeviceState)));

  // velocity tables and the quadrature sums of exactly those values
  InstanceDesc &D = c->hdesc;
  std::memset(&D, 0, sizeof(D));
  bool sums_ok;
  if (c->fp64) {
    std::vector<double> vel, inv;
    build_velocity_tables<double>(c, vel, inv);
    sums_ok = table_sums<double>(c, vel, D);
    CREATE_CUDA(cudaMemcpy(c->d_vel, vel.data(), vel.size() * sizeof(double), cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(c->d_inv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> vel, inv;
    build_velocity_tables<float>(c, vel, inv);
    sums_ok = table_sums<float>(c, vel, D);
    CREATE_CUDA(cudaMemcpy(c->d_vel, vel.data(), vel.size() * sizeof(float), cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(c->d_inv, inv.data(), inv.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  if (!sums_ok) return cleanup_fail(DVM_EINVAL, "velocity grid moments are degenerate");
  CREATE_CUDA(cudaMemcpy(c->d_code4, c->geo.code4.data(), sizeof(uint32_t) * 4 * ncell, cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemcpy(c->d_hw_src, c->geo.hw_src.data(), sizeof(int) * 8 * ncell, cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemset(c->d_delta_field, 0, sizeof(double) * ncell));
  if (c->alpha < 1.0) {
    // a slot for every wall face a sweep reads (the faces behind wall-class cells)
    std::vector<int> slot(ncell * 4, -1);
    for (size_t k = 0; k < c->geo.hw_src.size(); ++k) {
      const int f = c->geo.hw_src[k];
      if (f >= 0 && slot[f] < 0) slot[f] = c->nwall++;
    }
    CREATE_CUDA(cudaMalloc(&c->d_wall_slot, sizeof(int) * 4 * ncell));
    CREATE_CUDA(cudaMemcpy(c->d_wall_slot, slot.data(), sizeof(int) * 4 * ncell, cudaMemcpyHostToDevice));
    const size_t wbytes = ts * 2 * (size_t)std::max(c->nwall, 1) * 2 * c->gq * kLanes;
    CREATE_CUDA(cudaMalloc(&c->d_wbuf, wbytes));
    CREATE_CUDA(cudaMemset(c->d_wbuf, 0, wbytes));
  }

  if (P.anderson_depth > 0) {
    AndersonDesc A{};
    A.m = c->aa_m = P.anderson_depth;
    A.n_mom = 4 * (long long)ncell;
    A.n_wall = 4 * (long long)ncell;
    const bool spx = c->tr ? P.periodic_y : P.periodic_x, spy = c->tr ? P.periodic_x : P.periodic_y;
    A.n_sx = spx ? (long long)c->ngroups * c->ny * 2 * kLanes : 0;
    A.n_sy = spy ? (long long)c->ngroups * c->nx * 2 * kLanes : 0;
    A.n = c->aa_n = A.n_mom + A.n_wall + A.n_sx + A.n_sy + 1;
    const size_t nbuf = (size_t)(3 + 2 * A.m) * A.n + kAARed + (size_t)A.m * A.m + A.m;
    CREATE_CUDA(cudaMalloc(&c->d_aa_buf, sizeof(double) * nbuf));
    CREATE_CUDA(cudaMemset(c->d_aa_buf, 0, sizeof(double) * nbuf));
    CREATE_CUDA(cudaMalloc(&c->d_aa_meta, sizeof(int) * 3));
    CREATE_CUDA(cudaMemset(c->d_aa_meta, 0, sizeof(int) * 3));
    std::vector<unsigned char> wf(ncell * 4, 0);
    for (size_t k = 0; k < c->geo.hw_src.size(); ++k)
      if (c->geo.hw_src[k] >= 0) wf[c->geo.hw_src[k]] = 1;
    CREATE_CUDA(cudaMalloc(&c->d_wallface, ncell * 4));
    CREATE_CUDA(cudaMemcpy(c->d_wallface, wf.data(), ncell * 4, cudaMemcpyHostToDevice));
    double *b = c->d_aa_buf;
    A.x = b;
    A.fp = b + A.n;
    A.gp = b + 2 * A.n;
    A.dF = b + 3 * A.n;
    A.dG = b + (size_t)(3 + A.m) * A.n;
    A.red = b + (size_t)(3 + 2 * A.m) * A.n;
    A.gram = A.red + kAARed;
    A.flow_comp = c->tr ? 2 : 1;
    A.gamma = A.gram + A.m * A.m;
    A.meta = c->d_aa_meta;
    A.wallface = c->d_wallface;
    CREATE_CUDA(cudaMalloc(&c->d_aa, sizeof(AndersonDesc)));
    CREATE_CUDA(cudaMemcpy(c->d_aa, &A, sizeof(AndersonDesc), cudaMemcpyHostToDevice));
  }

  if (c->nux) {
    // stored column i is the caller's row i: its width relative to the mean row height
    std::vector<double> w(c->nx);
    for (int i = 0; i < c->nx; ++i) w[i] = P.row_heights[i] / c->dxs;
    CREATE_CUDA(cudaMalloc(&c->d_xwidth, sizeof(double) * c->nx));
    CREATE_CUDA(cudaMemcpy(c->d_xwidth, w.data(), sizeof(double) * c->nx, cudaMemcpyHostToDevice));
  }

  // launch maps of a single-instance launch
  std::vector<int> smap(c->ngroups), fmap;
  for (int g = 0; g < c->ngroups; ++g) smap[g] = g;
  const int fin_nblocks = (c->ncell + kFinBlock - 1) / kFinBlock;
  if (fin_nblocks > 65535) return cleanup_fail(DVM_EINVAL, "grid has too many cells");
  fmap.resize(fin_nblocks);
  for (int b = 0; b < fin_nblocks; ++b) fmap[b] = b;
  CREATE_CUDA(cudaMalloc(&c->d_sweep_map, sizeof(int) * smap.size()));
  CREATE_CUDA(cudaMalloc(&c->d_fin_map, sizeof(int) * fmap.size()));
  CREATE_CUDA(cudaMemcpy(c->d_sweep_map, smap.data(), sizeof(int) * smap.size(), cudaMemcpyHostToDevice));
  CREATE_CUDA(cudaMemcpy(c->d_fin_map, fmap.data(), sizeof(int) * fmap.size(), cudaMemcpyHostToDevice));

  D.nx = c->nx;
  D.ny = c->ny;
  D.ncell = c->ncell;
  D.periodic_x = spx;
  D.periodic_y = spy;
  D.ngroups = c->ngroups;
  D.groups_per_quadrant = c->gq;
  D.n_gas = c->geo.n_gas;
  D.fin_nblocks = fin_nblocks;
  D.dx = c->dxs;
  D.dy = c->dys;
  D.flow_axis = c->tr ? 1 : 0;
  // Q = sum u1 dx1 dy / (unx dx1) = sum u1 dy / unx, dy the caller's row height (stored: the column
  // width dxs xwidth[i] when the grid is stored transposed)
  D.dA_over_Lx = (c->tr ? c->dxs : c->dys) / c->unx;
  D.xwidth = c->d_xwidth;
  D.aa = c->d_aa;
  D.delta = delta;
  D.force = P.force;
  D.alpha = c->alpha;
  for (int k = 0; k < 4; ++k) D.wnrm[k] = c->alpha / D.nrm[k];
  {
    // a symmetric velocity set gives a Gram matrix whose only off-diagonal coupling is (1, |v|^2):
    // then the finalize applies its inverse in 6 instead of 16 multiply-adds (the skipped products
    // are exact zeros)
    bool sparse = true;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        const bool kept = i == j || (i == 0 && j == 3) || (i == 3 && j == 0);
        if (!kept && D.ginv[i * 4 + j] != 0.0) sparse = false;
      }
    D.ginv_sparse = sparse ? 1 : 0;
  }
  D.top_u = c->top_u;
  D.nwall = c->nwall;
  D.wall_slot = c->d_wall_slot;
  D.wbuf = c->d_wbuf;
  D.fp32 = c->fp64 ? 0 : 1;
  D.vel = c->d_vel;
  D.inv_den = c->d_inv;
  D.rec = c->d_rec;
  D.rec_diag = c->d_rec_diag;
  D.code4 = c->d_code4;
  D.hw_src = c->d_hw_src;
  D.acc = c->d_acc;
  D.facc = c->d_facc;
  D.mom = c->d_mom;
  D.u1prev = c->d_u1prev;
  D.seam_x = c->d_seamx;
  D.seam_y = c->d_seamy;
  D.h = c->d_h;
  D.state = c->d_state;
  c->uniform = true;
  if (upload_desc(c) != DVM_OK) return cleanup_fail(DVM_ECUDA, c->err);
  if (reset_state(c) != DVM_OK) return cleanup_fail(DVM_ECUDA, c->err);
#undef CREATE_CUDA
  *out = c;
  return DVM_OK;
}

dvm_status dvm_reset(dvm_ctx *ctx) {
  if (!ctx) return DVM_EINVAL;
  return reset_state(ctx);
}

dvm_status dvm_set_delta_field(dvm_ctx *ctx, const double *delta_c) {
  if (!ctx) return DVM_EINVAL;
  if (delta_c) {
    std::vector<double> d((size_t)ctx->ncell, 0.0);
    for (int ucell = 0; ucell < ctx->ncell; ++ucell) {
      const size_t cell = stored_cell(ctx, ucell);
      if (ctx->geo.code4[cell * 4] & kSolid) continue;
      if (!(delta_c[ucell] >= 0.0) || !std::isfinite(delta_c[ucell]))
        return fail(ctx, DVM_EINVAL, "delta field entries must be finite and >= 0 in gas cells");
      d[cell] = delta_c[ucell];
    }
    DVM_CUDA(ctx, cudaMemcpyAsync(ctx->d_delta_field, d.data(), sizeof(double) * ctx->ncell, cudaMemcpyHostToDevice,
                                  ctx->stream));
    DVM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->uniform = false;
    ctx->delta_user.assign(delta_c, delta_c + ctx->ncell);
  } else {
    ctx->uniform = true;
    ctx->delta_user.clear();
  }
  if (ctx->twin) {
    // the FP64 twin of the refinement is rebuilt with the new field when next needed
    dvm_destroy(ctx->twin);
    ctx->twin = nullptr;
  }
  if (ctx->self) {
    batch_free(ctx->self);
    ctx->self = nullptr;
  }
  if (ctx->a_graph) {
    cudaGraphExecDestroy(ctx->a_graph);
    ctx->a_graph = nullptr;
  }
  dvm_status st = upload_desc(ctx);
  if (st != DVM_OK) return st;
  return reset_state(ctx);
}

dvm_status dvm_solve(dvm_ctx *ctx, double tol, int max_iter, int *iters, double *est) {
  if (!ctx) return DVM_EINVAL;
  if (!(tol > 0.0)) return fail(ctx, DVM_EINVAL, "tol must be > 0");
  dvm_status st = ensure_self(ctx);
  if (st != DVM_OK) return st;
  DVM_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, ctx->stream));
  DVM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int start = ctx->h_state->iter;
  st = batch_run(ctx->self, tol, max_iter, nullptr, iters, est);
  if (st != DVM_OK || ctx->fp64) return st;
  st = batch_refine(ctx->self, tol, max_iter);
  if (st != DVM_OK) return st;
  DVM_CUDA(ctx, cudaMemcpyAsync(ctx->h_state, ctx->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, ctx->stream));
  DVM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (iters) *iters = ctx->h_state->iter - start;
  if (est) *est = ctx->h_state->est;
  return DVM_OK;
}

dvm_status dvm_iterate(dvm_ctx *ctx, int n) {
  if (!ctx) return DVM_EINVAL;
  dvm_status st = ensure_self(ctx);
  if (st != DVM_OK) return st;
  return batch_iterate(ctx->self, n);
}

dvm_status dvm_get_info(const dvm_ctx *ctx, dvm_info *info) {
  if (!ctx || !info) return DVM_EINVAL;
  dvm_ctx *c = const_cast<dvm_ctx *>(ctx);
  DVM_CUDA(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  info->iterations = c->h_state->iter;
  info->eps = c->h_state->eps;
  info->est = c->h_state->est;
  info->mass_shift = c->h_state->c;
  info->Q = c->h_state->Q;
  info->status = c->h_state->status;
  info->transposed = c->tr ? 1 : 0;
  return DVM_OK;
}

dvm_status dvm_flowrate(const dvm_ctx *ctx, double *Q, double *k_a) {
  if (!ctx || !Q) return DVM_EINVAL;
  dvm_info info;
  dvm_status st = dvm_get_info(ctx, &info);
  if (st != DVM_OK) return st;
  if (info.iterations < 1) return fail(const_cast<dvm_ctx *>(ctx), DVM_ESTATE, "no sweep has run yet");
  *Q = info.Q;
  if (k_a) *k_a = (ctx->uniform && ctx->delta > 0.0) ? std::sqrt(4.0 / M_PI) * info.Q * ctx->kn : NAN;
  return DVM_OK;
}

dvm_status dvm_fields(const dvm_ctx *ctx, double *rho, double *u1, double *u2, double *tau) {
  if (!ctx) return DVM_EINVAL;
  dvm_ctx *c = const_cast<dvm_ctx *>(ctx);
  std::vector<double> mom((size_t)4 * c->ncell);
  DVM_CUDA(c, cudaMemcpyAsync(mom.data(), c->d_mom, sizeof(double) * 4 * c->ncell, cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  // stored moments (rho, u1, u2, tau) of the stored axes; a transposed grid swaps u1 and u2
  double *outs[4] = {rho, c->tr ? u2 : u1, c->tr ? u1 : u2, tau};
  for (int ucell = 0; ucell < c->ncell; ++ucell) {
    const size_t cell = stored_cell(c, ucell);
    const bool solid = (c->geo.code4[cell * 4] & kSolid) != 0;
    for (int m = 0; m < 4; ++m)
      if (outs[m]) outs[m][ucell] = solid ? NAN : mom[cell * 4 + m];
  }
  return DVM_OK;
}

dvm_status dvm_distribution(const dvm_ctx *ctx, const int *ks, int nk, double *out) {
  if (!ctx || (nk > 0 && (!ks || !out)) || nk < 0) return DVM_EINVAL;
  dvm_ctx *c = const_cast<dvm_ctx *>(ctx);
  if (!c->d_h) return fail(c, DVM_ESTATE, "the distribution is not kept (store_distribution = 0)");
  const size_t ts = c->fp64 ? 8 : 4;
  std::vector<unsigned char> buf(ts * c->ncell);
  // the stored sweep output is the state before its last mass shift s
  DVM_CUDA(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  const double shift = c->h_state->iter > 0 ? c->h_state->s : 0.0;
  for (int m = 0; m < nk; ++m) {
    const int k = ks[m];
    if (k < 0 || k >= c->nv * c->nv) return fail(c, DVM_EINVAL, "velocity index out of range");
    // (a, b): indices of the stored v1 and v2 (the caller's v2 and v1 when the grid is transposed)
    const int a = c->tr ? k % c->nv : k / c->nv, b = c->tr ? k / c->nv : k % c->nv;
    const int s1neg = a < c->half, s2neg = b < c->half;
    const int ap = s1neg ? c->half - 1 - a : a - c->half;
    const int bp = s2neg ? c->half - 1 - b : b - c->half;
    const int q = s1neg + 2 * s2neg;
    const int pos = ap * c->half + bp;
    const int g = q * c->gq + pos / kLanes, lane = pos % kLanes;
    const char *src = static_cast<const char *>(c->d_h) + ((size_t)g * c->ncell * kLanes + lane) * ts;
    DVM_CUDA(c, cudaMemcpy2DAsync(buf.data(), ts, src, ts * kLanes, ts, c->ncell, cudaMemcpyDeviceToHost, c->stream));
    DVM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int ucell = 0; ucell < c->ncell; ++ucell) {
      const size_t cell = stored_cell(c, ucell);
      double v;
      if (c->fp64) std::memcpy(&v, &buf[cell * 8], 8);
      else {
        float f;
        std::memcpy(&f, &buf[cell * 4], 4);
        v = f;
      }
      v = (c->geo.code4[cell * 4] & kSolid) ? 0.0 : v - shift;
      out[(size_t)m * c->ncell + ucell] = v;
    }
  }
  return DVM_OK;
}

dvm_status dvm_quadrature(const dvm_ctx *ctx, double *nodes, double *weights) {
  if (!ctx) return DVM_EINVAL;
  for (int a = 0; a < ctx->nv; ++a) {
    if (nodes) nodes[a] = ctx->x1[a];
    if (weights) weights[a] = ctx->w1[a];
  }
  return DVM_OK;
}

dvm_status dvm_velocity_grid(const dvm_quad *q, double *nodes, double *weights) {
  if (!q || !nodes || !weights) return DVM_EINVAL;
  std::vector<double> x, w;
  std::string err;
  if (!quadrature_1d(q->kind, q->n, q->vmax, x, w, err)) return fail(nullptr, DVM_EINVAL, err);
  for (int a = 0; a < q->n; ++a) {
    nodes[a] = x[a];
    weights[a] = w[a];
  }
  return DVM_OK;
}

// ------------------------------------------------------------------------------------------------
// Adjoint: gradient of Q with respect to the per-cell collision rate (dvm_adjoint).

namespace {

dvm_status adjoint_setup(dvm_ctx *c) {
  const size_t ts = c->fp64 ? 8 : 4;
  const size_t recsz = c->fp64 ? sizeof(SweepRec<double>) : sizeof(SweepRec<float>);
  const size_t ncell = (size_t)c->ncell;
  if (!c->a_state) {
    DVM_CUDA(c, cudaMalloc(&c->a_rec, recsz * 4 * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_rec_diag, recsz * 4 * diag_quadrant_size(c->nx, c->ny)));
    DVM_CUDA(c, cudaMalloc(&c->a_seamx, ts * c->ngroups * c->ny * 2 * kLanes));
    DVM_CUDA(c, cudaMalloc(&c->a_seamy, ts * c->ngroups * c->nx * 2 * kLanes));
    DVM_CUDA(c, cudaMalloc(&c->a_z, ts * c->ngroups * ncell * kLanes));
    DVM_CUDA(c, cudaMalloc(&c->a_acc, sizeof(double) * 4 * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_flux, sizeof(double) * 8 * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_alpha, sizeof(double) * 4 * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_z1prev, sizeof(double) * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_grad, sizeof(double) * ncell));
    DVM_CUDA(c, cudaMalloc(&c->a_state, sizeof(DeviceState)));
    DVM_CUDA(c, cudaMalloc(&c->a_desc, sizeof(InstanceDesc)));
  }
  const size_t wbytes = ts * 2 * (size_t)std::max(c->nwall, 1) * 2 * c->gq * kLanes;
  if (c->alpha < 1.0 && !c->a_wbuf) DVM_CUDA(c, cudaMalloc(&c->a_wbuf, wbytes));
  // the adjoint view: the forward instance with the adjoint buffers in place of the forward ones
  InstanceDesc A = c->hdesc;
  A.wbuf = c->a_wbuf;
  A.uniform_delta = c->uniform ? 1 : 0;
  A.delta_field = c->d_delta_field;
  A.rec = c->a_rec;
  A.rec_diag = c->a_rec_diag;
  A.acc = c->a_acc;
  A.facc = c->a_flux;
  A.mom = c->a_alpha;
  A.u1prev = c->a_z1prev;
  A.seam_x = c->a_seamx;
  A.seam_y = c->a_seamy;
  A.h = c->a_z;
  A.state = c->a_state;
  A.h_fwd = c->d_h;
  A.mom_fwd = c->d_mom;
  A.state_fwd = c->d_state;
  A.grad = c->a_grad;
  A.aa = nullptr;  // the adjoint iteration is not mixed
  DVM_CUDA(c, cudaMemcpyAsync(c->a_desc, &A, sizeof(InstanceDesc), cudaMemcpyHostToDevice, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_acc, 0, sizeof(double) * 4 * ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_flux, 0, sizeof(double) * 8 * ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_alpha, 0, sizeof(double) * 4 * ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_z1prev, 0, sizeof(double) * ncell, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_seamx, 0, ts * c->ngroups * c->ny * 2 * kLanes, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_seamy, 0, ts * c->ngroups * c->nx * 2 * kLanes, c->stream));
  DVM_CUDA(c, cudaMemsetAsync(c->a_z, 0, ts * c->ngroups * ncell * kLanes, c->stream));
  if (c->a_wbuf) DVM_CUDA(c, cudaMemsetAsync(c->a_wbuf, 0, wbytes, c->stream));
  DVM_CUDA(c, launch_adjoint_reset(c->a_desc, c->ncell, c->fp64, c->stream));
  if (!c->a_graph) {
    Schedule sc;
    std::string why;
    if (!resolve_schedule(c->nx, c->sched_kind, c->sched_v, &sc, &why, needs_special(c))) return fail(c, DVM_EINVAL, why);
    const bool cols = sc.kind == DVM_SWEEP_COLUMNS;
    const int parts = cols ? cols_parts(c->fp64, sc.v) : 1;
    std::vector<int> amap;
    for (int g = 0; g < c->ngroups; ++g)
      for (int part = 0; part < parts; ++part) amap.push_back((part << 12) | g);
    free_dev(c->d_adj_map);
    DVM_CUDA(c, cudaMalloc(&c->d_adj_map, sizeof(int) * amap.size()));
    DVM_CUDA(c, cudaMemcpyAsync(c->d_adj_map, amap.data(), sizeof(int) * amap.size(), cudaMemcpyHostToDevice, c->stream));
    DVM_CUDA(c, cudaStreamSynchronize(c->stream));
    const int cw = (!cols && sc.v > 0) ? sc.v : c->cw;
    const int warps = cols ? (c->nx + kLanes / sc.v - 1) / (kLanes / sc.v) : (c->nx + cw - 1) / cw;
    LaunchDesc L = make_launch(c->a_desc, c->d_adj_map, c->d_fin_map, 1, warps, cw, cols ? sc.v : 0,
                               cols && needs_special(c));
    const int sweep_blocks = (int)amap.size();
    const int fin_blocks = c->hdesc.fin_nblocks;
    const int lines = (c->hdesc.periodic_x ? c->ngroups * c->ny : 0) + (c->hdesc.periodic_y ? c->ngroups * c->nx : 0);
    const int seam_blocks = (lines * 32 + 255) / 256;
    const double upd = (double)c->geo.n_gas * c->nv * c->nv;
    c->a_graph_iters = iters_per_graph(upd);
    cudaGraph_t graph = nullptr;
    DVM_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < c->a_graph_iters && e == cudaSuccess; ++it) {
      // columns of unequal width take the per-cell denominators (the uniform table assumes equal columns)
      e = launch_sweep_adjoint(c->fp64, c->uniform && !c->nux, L, sweep_blocks, c->cap_stream);
      if (e == cudaSuccess) e = launch_adjoint_finalize(L, fin_blocks, seam_blocks, c->fp64, c->cap_stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return fail(c, DVM_ECUDA, std::string("adjoint graph capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&c->a_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, DVM_ECUDA, std::string("adjoint graph instantiate: ") + cudaGetErrorString(e));
  }
  return DVM_OK;
}

}  // namespace

dvm_status dvm_adjoint(dvm_ctx *ctx, double tol, int max_iter, double *dQ_ddelta, double *q_identity, int *iters) {
  if (!ctx || !dQ_ddelta) return DVM_EINVAL;
  dvm_ctx *c = ctx;
  if (!(tol > 0.0) || max_iter < 1) return fail(c, DVM_EINVAL, "tol must be > 0 and max_iter >= 1");
  if (!c->d_h) return fail(c, DVM_ESTATE, "dvm_adjoint needs the forward distribution (store_distribution = 1)");
  // a moving plate only adds a constant source: the transposed operator is the one of a plate at rest
  if (c->nux && c->hdesc.periodic_x)
    return fail(c, DVM_EINVAL, "dvm_adjoint: rows of unequal height need a non-periodic x2 axis");
  DVM_CUDA(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->h_state->iter < 1) return fail(c, DVM_ESTATE, "dvm_adjoint needs a forward solve first");
  dvm_status st = adjoint_setup(c);
  if (st != DVM_OK) return st;
  DVM_CUDA(c, launch_arm(c->a_state, tol, max_iter, c->stream));
  const long long max_replays = (long long)max_iter / c->a_graph_iters + 3;
  for (long long replay = 0;; ++replay) {
    if (replay >= max_replays) return fail(c, DVM_ETIMEOUT, "adjoint stop flag not set after max_iter sweeps");
    DVM_CUDA(c, cudaGraphLaunch(c->a_graph, c->stream));
    DVM_CUDA(c, cudaMemcpyAsync(c->h_state, c->a_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, c->stream));
    DVM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->h_state->done) break;
  }
  const dvm_status status = (dvm_status)c->h_state->status;
  const int n = c->h_state->iter;
  if (status != DVM_OK && status != DVM_ENOCONV) return fail(c, status, "adjoint iteration failed");
  DVM_CUDA(c, cudaMemsetAsync(&c->a_state->Q, 0, sizeof(double), c->stream));
  DVM_CUDA(c, launch_adjoint_gradient(c->a_desc, c->ncell, c->fp64, c->stream));
  std::vector<double> g((size_t)c->ncell);
  DVM_CUDA(c, cudaMemcpyAsync(g.data(), c->a_grad, sizeof(double) * c->ncell, cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaMemcpyAsync(c->h_state, c->a_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, c->stream));
  DVM_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int ucell = 0; ucell < c->ncell; ++ucell) {
    const size_t cell = stored_cell(c, ucell);
    dQ_ddelta[ucell] = (c->geo.code4[cell * 4] & kSolid) ? 0.0 : g[cell];
  }
  if (q_identity) *q_identity = c->h_state->Q;
  if (iters) *iters = n;
  return status;
}

dvm_status dvm_batch_create(dvm_ctx *const *ctxs, int n, dvm_batch **out) {
  if (!out) return DVM_EINVAL;
  return batch_build(ctxs, n, out);
}

dvm_status dvm_batch_run(dvm_batch *batch, double tol, int max_iter, dvm_status *per) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  if (!(tol > 0.0)) return fail(batch->ctxs[0], DVM_EINVAL, "tol must be > 0");
  dvm_status st = batch_run(batch, tol, max_iter, per, nullptr, nullptr);
  if (st != DVM_OK || batch->fp64) return st;
  return batch_refine(batch, tol, max_iter);
}

dvm_status dvm_batch_iterate(dvm_batch *batch, int n) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  return batch_iterate(batch, n);
}

dvm_status dvm_batch_enqueue(dvm_batch *batch, int n) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  dvm_batch *b = batch;
  dvm_ctx *c0 = b->ctxs[0];
  if (n < 1 || n > 1000000) return fail(c0, DVM_EINVAL, "n must be in 1..1000000");
  for (dvm_ctx *c : b->ctxs)
    if (c->stream != b->stream) DVM_CUDA(c0, cudaStreamSynchronize(c->stream));
  DVM_CUDA(c0, launch_arm_all(b->d_descs, (int)b->ctxs.size(), -1.0, n, b->stream));
  int left = n;
  while (left >= b->m && b->m > 1) {
    DVM_CUDA(c0, cudaGraphLaunch(b->g_many, b->stream));
    left -= b->m;
  }
  for (; left > 0; --left) {
    DVM_CUDA(c0, cudaEventRecord(b->ev[0], b->stream));
    DVM_CUDA(c0, cudaGraphLaunch(b->g_sweep, b->stream));
    DVM_CUDA(c0, cudaEventRecord(b->ev[1], b->stream));
    // (the persistent launch finalizes inside g_sweep)
    if (b->g_fin) DVM_CUDA(c0, cudaGraphLaunch(b->g_fin, b->stream));
    DVM_CUDA(c0, cudaEventRecord(b->ev[2], b->stream));
  }
  b->timed = (n == 1) || (n % b->m != 0) || b->m == 1;
  return DVM_OK;
}

dvm_status dvm_batch_check(dvm_batch *batch) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  bool all = false;
  dvm_status st = batch_poll(batch, &all);
  if (st != DVM_OK) return st;
  for (dvm_ctx *c : batch->ctxs) {
    const int s = c->h_state->status;
    if (s != DVM_OK && s != DVM_ENOCONV) return fail(batch->ctxs[0], (dvm_status)s, "a batch member failed");
  }
  return DVM_OK;
}

dvm_status dvm_batch_timing(const dvm_batch *batch, float *sweep_ms, float *finalize_ms) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  if (!batch->timed) return fail(batch->ctxs[0], DVM_ESTATE, "no timed single sweep has run on this batch");
  float a = 0.f, b = 0.f;
  DVM_CUDA(batch->ctxs[0], cudaEventElapsedTime(&a, batch->ev[0], batch->ev[1]));
  DVM_CUDA(batch->ctxs[0], cudaEventElapsedTime(&b, batch->ev[1], batch->ev[2]));
  if (sweep_ms) *sweep_ms = a;
  if (finalize_ms) *finalize_ms = b;
  return DVM_OK;
}

int dvm_batch_kernels_per_sweep(const dvm_batch *batch) {
  if (!batch || batch->detached) return 0;
  if (batch->persistent) return 2;  // per launch: the arming kernel and the scheduler kernel
  return batch->anderson ? 6 : 3;
}

dvm_status dvm_batch_set_persistent(dvm_batch *batch, int on) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  Schedule sc;
  sc.kind = batch->kind;
  sc.v = batch->kind == DVM_SWEEP_ROWS ? batch->cw : batch->cols_v;
  sc.persistent = on != 0;
  if (sc.persistent && sc.kind != DVM_SWEEP_ROWS)
    return fail(batch->ctxs[0], DVM_EINVAL, "the persistent launch runs the row sweep: set a row schedule first");
  return batch_replan(batch, sc);
}

dvm_status dvm_batch_set_pairing(dvm_batch *batch, int mode) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  if (mode != DVM_PAIRING_AUTO && mode != DVM_PAIRING_ON && mode != DVM_PAIRING_OFF)
    return fail(batch->ctxs[0], DVM_EINVAL, "pairing mode must be DVM_PAIRING_AUTO, _ON or _OFF");
  Schedule sc;
  sc.kind = batch->kind;
  sc.v = batch->kind == DVM_SWEEP_ROWS ? batch->cw : batch->cols_v;
  sc.persistent = batch->persistent;
  const int old = batch->pairing;
  batch->pairing = mode;
  const dvm_status st = batch_replan(batch, sc);
  if (st != DVM_OK) batch->pairing = old;
  return st;
}

dvm_status dvm_batch_get_pairing(const dvm_batch *batch, int *mode, int *paired_blocks) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;
  if (mode) *mode = batch->pairing;
  if (paired_blocks) *paired_blocks = batch->pair_blocks;
  return DVM_OK;
}

dvm_status dvm_batch_get_persistent(const dvm_batch *batch, int *on, int *blocks) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  if (on) *on = batch->persistent ? 1 : 0;
  if (blocks) *blocks = batch->persistent ? batch->p_blocks : 0;
  return DVM_OK;
}

dvm_status dvm_set_schedule(dvm_ctx *ctx, int kind, int threads_per_column) {
  if (!ctx) return DVM_EINVAL;
  Schedule sc;
  std::string why;
  if (threads_per_column < 0 || !resolve_schedule(ctx->nx, kind, threads_per_column, &sc, &why, needs_special(ctx)))
    return fail(ctx, DVM_EINVAL, why.empty() ? "bad threads_per_column" : why);
  ctx->sched_kind = sc.kind;
  ctx->sched_v = sc.v;
  if (ctx->stream) DVM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (ctx->self) {
    batch_free(ctx->self);
    ctx->self = nullptr;
  }
  if (ctx->a_graph) {
    cudaGraphExecDestroy(ctx->a_graph);
    ctx->a_graph = nullptr;
  }
  return DVM_OK;
}

dvm_status dvm_get_schedule(const dvm_ctx *ctx, int *kind, int *threads_per_column) {
  if (!ctx) return DVM_EINVAL;
  Schedule sc;
  std::string why;
  dvm_ctx *c = const_cast<dvm_ctx *>(ctx);
  const bool automatic = ctx->sched_kind == DVM_SWEEP_AUTO;
  const int k = automatic ? auto_sweep_kind(&c, 1, ctx->nx, needs_special(ctx)) : ctx->sched_kind;
  if (!resolve_schedule(ctx->nx, k, automatic ? 0 : ctx->sched_v, &sc, &why, needs_special(ctx)))
    return fail(c, DVM_EINVAL, why);
  if (kind) *kind = sc.kind;
  if (threads_per_column) *threads_per_column = (sc.kind == DVM_SWEEP_ROWS && sc.v == 0) ? ctx->cw : sc.v;
  return DVM_OK;
}

dvm_status dvm_batch_set_schedule(dvm_batch *batch, int kind, int threads_per_column) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  int nx_max = 0;
  bool spec = false;
  for (dvm_ctx *c : batch->ctxs) {
    nx_max = std::max(nx_max, c->nx);
    spec = spec || needs_special(c);
  }
  Schedule sc;
  std::string why;
  if (threads_per_column < 0 || !resolve_schedule(nx_max, kind, threads_per_column, &sc, &why, spec))
    return fail(batch->ctxs[0], DVM_EINVAL, why.empty() ? "bad threads_per_column" : why);
  return batch_replan(batch, sc);
}

dvm_status dvm_batch_get_schedule(const dvm_batch *batch, int *kind, int *threads_per_column) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  if (kind) *kind = batch->kind;
  if (threads_per_column) *threads_per_column = batch->kind == DVM_SWEEP_ROWS ? batch->cw : batch->cols_v;
  return DVM_OK;
}

dvm_status dvm_batch_autotune(dvm_batch *batch, int sweeps, int *kind, int *threads_per_column, float *sweep_ms) {
  if (!batch) return DVM_EINVAL;
  if (batch->detached) return DVM_ESTATE;  // a member context was destroyed
  dvm_ctx *c0 = batch->ctxs[0];
  if (sweeps < 1 || sweeps > 1000) return fail(c0, DVM_EINVAL, "sweeps must be in 1..1000");
  int nx_max = 0;
  bool spec = false;
  for (dvm_ctx *c : batch->ctxs) {
    nx_max = std::max(nx_max, c->nx);
    spec = spec || needs_special(c);
  }
  std::vector<Schedule> cands;
  {
    // the row kernel at its narrowest chunk (most rows in flight) and two wider ones
    const int cw0 = choose_cw(nx_max, kMaxSweepWarps);
    for (int cw : {cw0, 2 * cw0, 4 * cw0}) {
      Schedule sc;
      std::string why;
      if (cw <= 16 && resolve_schedule(nx_max, DVM_SWEEP_ROWS, cw, &sc, &why, spec)) cands.push_back(sc);
    }
    for (int v : {1, 2, 4}) {
      Schedule sc;
      std::string why;
      if (resolve_schedule(nx_max, DVM_SWEEP_COLUMNS, v, &sc, &why, spec)) cands.push_back(sc);
    }
  }
  Schedule best;
  float best_ms = INFINITY;
  for (const Schedule &sc : cands) {
    if (batch_replan(batch, sc) != DVM_OK) continue;  // e.g. the row sweep's shared memory does not fit
    std::vector<float> t;
    for (int s = 0; s < sweeps + 1; ++s) {
      dvm_status st = batch_iterate(batch, 1);
      if (st != DVM_OK) return st;
      float a = 0.f;
      DVM_CUDA(c0, cudaEventElapsedTime(&a, batch->ev[0], batch->ev[1]));
      if (s > 0) t.push_back(a);  // the first sweep after a re-plan warms the new kernel up
    }
    std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
    const float med = t[t.size() / 2];
    if (med < best_ms) {
      best_ms = med;
      best = sc;
    }
  }
  if (!(best_ms < INFINITY)) return fail(c0, DVM_EINVAL, "no sweep kernel fits the batch");
  dvm_status st = batch_replan(batch, best);
  if (st != DVM_OK) return st;
  if (kind) *kind = best.kind;
  if (threads_per_column) *threads_per_column = best.v;  // rows: the chunk width
  if (sweep_ms) *sweep_ms = best_ms;
  return DVM_OK;
}

void dvm_batch_destroy(dvm_batch *batch) {
  if (!batch) return;
  if (!batch->detached) cudaStreamSynchronize(batch->stream);
  batch_free(batch);
}

dvm_status dvm_batch_solve(dvm_ctx *const *ctxs, int n, double tol, int max_iter, dvm_status *per) {
  if (!ctxs || n < 1 || !(tol > 0.0) || max_iter < 1) return DVM_EINVAL;
  dvm_batch *b = nullptr;
  dvm_status st = batch_build(ctxs, n, &b);
  if (st != DVM_OK) return st;
  st = batch_run(b, tol, max_iter, per, nullptr, nullptr);
  if (st == DVM_OK && !b->fp64) st = batch_refine(b, tol, max_iter);
  batch_free(b);
  return st;
}

void dvm_destroy(dvm_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  // batches still holding this context lose their launches now (their streams may be this context's)
  while (!ctx->batches.empty()) {
    dvm_batch *b = ctx->batches.back();
    if (b == ctx->self) {
      batch_free(b);
      ctx->self = nullptr;
    } else {
      batch_detach(b);
    }
  }
  release_device(ctx);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

}  // extern "C"
