// dvm_device.cuh -- device-side data layout of libdvm (internal; not part of the C ABI).
//
// One "instance" is one geometry + Knudsen number + velocity grid.  The distribution h of an
// instance is split into velocity groups of 32 velocities of one quadrant (sign(v1), sign(v2)).
// The row-wavefront sweep gives one thread block a group (lanes = velocities, warps = rows in
// flight); the column sweep gives a block a group or a part of one (threads = grid columns, each
// with a few velocities).  Several instances can share a launch (batched solves).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dvm {

constexpr int kLanes = 32;       // velocities per group = warp width
constexpr int kRingPad = 33;     // padded row stride (elements) of the shared-memory ring buffer
constexpr int kMaxWarps = 32;
constexpr int kMaxSweepWarps = 16;  // rows in flight per sweep block (512 threads, up to 128 registers)

// Per-cell code bits for one quadrant (static geometry, see dvm_tables.cpp).
enum : uint32_t {
  kSolid = 1u,
  kClsXShift = 1,  // 2 bits: 0 interior (second order), 1 second cell from a wall (first order),
                   //         2 next to a wall (linear through the wall value)
  kClsYShift = 3,
  kIncX = 1u << 5, // the cell owns a wall face on its downstream x side (incident for this quadrant)
  kIncY = 1u << 6,
  kInvShift = 7,   // 4 bits: row of the 1/denominator table, clx * 3 + cly, or 9 (solid: 0); at bit 7
                   // code & (15 << 7) is the row's byte offset in an FP32 table of 32-entry rows
  // Transposed stencil (adjoint sweep): the forward-downstream cells d1 = c + s and d2 = c + 2 s
  // read c with weights t1 in {0, 1, 2} (d1 solid / second cell from a wall / interior) and
  // t2 in {0, -1/2} (d1 or d2 solid / interior).
  kAdjT1XShift = 12,  // 2 bits: t1 along x
  kAdjT2X = 1u << 14, // t2 = -1/2 along x
  kAdjT1YShift = 15,  // 2 bits: t1 along y
  kAdjT2Y = 1u << 17,
  kTopWall = 1u << 18,   // the upstream y wall of this quadrant is the moving plate beyond the last row
  kTopWallX = 1u << 19,  // the upstream x wall is the moving plate beyond the last column (transposed)
};
enum : int { kFull = 0, kNear = 1, kWall = 2 };
// sides of a cell: the solid neighbour lies at -x (W), +x (E), -y (S), +y (N)
enum : int { kW = 0, kE = 1, kS = 2, kN = 3 };
constexpr int kInvRows = 10;

// Sweep record: everything the sweep needs per cell and quadrant, rewritten every iteration by the
// finalize kernel.  R_k = A + B v1 + C v2 + D (|v|^2 - 1) is the right-hand side of Eq. (iteration),
// delta (a0 + a1 v1 + a2 v2 + a3 |v|^2 - c) + F v1 with the collision coefficients a = G^{-1} m
// (for an exact quadrature: delta (rho - c) + (2 delta u1 + F) v1 + 2 delta u2 v2 + delta tau (|v|^2 - 1)).
// The upwind combination along x is ax1 h(u1) + ax2 h(u2) + xw, with (ax1, ax2, xw) = (2, -1/2, 0)
// inside, (1, 0, 0) at the second cell from a wall and (0, 0, 2 h_w) next to a wall; y likewise.
// Solid cells carry all-zero coefficients (and the zero row of the 1/denominator table), so the
// sweep computes h = 0 there without a branch.
template <typename T> struct SweepRec;
template <> struct alignas(16) SweepRec<float> {
  float A, B, C, D;
  float ax1, ax2, xw, ay1;
  float ay2, yw;
  uint32_t code;
  float delta;
};
template <> struct alignas(16) SweepRec<double> {
  double A, B, C, D;
  double xw, yw;
  uint32_t code;   // the FP64 record derives (ax1, ax2, ay1, ay2) from the class bits
  uint32_t pad;
  double delta;
};
static_assert(sizeof(SweepRec<float>) == 48, "record layout");
static_assert(sizeof(SweepRec<double>) == 64, "record layout");

// Slot of cell (i, j) in the diagonal-major record array of one quadrant: with (p, q) the cell's
// column and row in the quadrant's sweep order, cells of one anti-diagonal S = p + q are contiguous.
__host__ __device__ inline size_t diag_slot(int nx, int ny, int i, int j, bool xneg, bool yneg) {
  const int p = xneg ? nx - 1 - i : i, q = yneg ? ny - 1 - j : j;
  return (size_t)(p + q) * nx + p;
}
__host__ __device__ inline size_t diag_quadrant_size(int nx, int ny) { return (size_t)(nx + ny - 1) * nx; }

// Upwind coefficients (a1, a2) of a stencil class: interior (2, -1/2), second cell (1, 0), wall (0, 0).
__host__ __device__ inline float class_a1(int cls) { return cls == kFull ? 2.0f : (cls == kNear ? 1.0f : 0.0f); }
__host__ __device__ inline float class_a2(int cls) { return cls == kFull ? -0.5f : 0.0f; }

// Per-lane velocity table fields ([group][field][lane], in the sweep precision).
enum : int {
  kV1 = 0, kV2, kE2m1, kCx, kCy,   // v1, v2, |v|^2 - 1, |v1|/dx, |v2|/dy
  kW0, kW1, kW2, kW3,              // W, W v1, W v2, W |v|^2 (moment weights; W = 0 on padded lanes)
  kWnx, kWny,                      // |v1| W, |v2| W (incident wall flux weights)
  kZ0, kZ1, kZ2, kZ3,              // 1, v1, v2, |v|^2 (adjoint moments; 0 on padded lanes)
  kNumVelFields
};

// Solver state of one instance (device memory; read back by the host between graph replays).
struct DeviceState {
  int iter;        // sweeps completed
  int done;        // 1 = stop: every kernel of the instance returns immediately
  int status;      // dvm_status of the solve so far
  int max_iter;    // stop with DVM_ENOCONV when iter reaches it
  int nan_flag;
  int iter_min;    // sweep of the smallest eps so far (FP32 stall test)
  int err_flag;    // a bounded device-side wait gave up (reported as DVM_ETIMEOUT)
  int pad0;
  unsigned int ticket1, ticket2;  // last-block counters of the two finalize kernels
  double tol;
  double c;        // accumulated mass shift (bordering unknown)
  double s;        // shift still to subtract from the stored seam values
  double s_new;    // shift of the current iteration
  double eps, est, Q;
  double eps_ring[4];
  double eps_min;  // smallest eps so far
  double mass_acc, du_acc, u_acc, q_acc;
  // adjoint iteration only
  double mu;       // bordering multiplier of the transposed system
  double kappa;    // (mu - sum lambda) / (n_gas sum W), added to the next right-hand side
  double lam_acc, dz_acc, seam_acc;
  // Anderson mixing only: the stopping test uses the plain residual f = G(x) - x at the mixed iterate
  double aa_res;       // |f| / |g| over the flow velocity of the gas cells (L2)
  double aa_rho;       // running estimate of the plain contraction, max |dG| / |dx| over the differences
  double aa_est;       // aa_res / (1 - aa_rho): the distance to the fixed point
  double aa_res_min;   // smallest aa_res since the solve was armed (10 % steps)
  int aa_iter_min;     // sweep of that minimum
};

// Anderson mixing of the source iteration (dvm_anderson.cu), one per instance that uses it.  The
// state vector is [moments 4 ncell | wall-face fluxes 4 ncell | x seam | y seam | c].
constexpr int kAAMaxDepth = 8;
// reduction slots: dF_new . dF_j [kAAMaxDepth], dF_j . f [kAAMaxDepth], then over the flow velocity
// |f|^2, |g|^2, |dG_new|^2, |dG_new - dF_new|^2
constexpr int kAARed = 2 * kAAMaxDepth + 4;
struct AndersonDesc {
  int m;                          // depth: differences kept (1..kAAMaxDepth)
  long long n_mom, n_wall, n_sx, n_sy, n;  // segment lengths (seams 0 on closed axes) and the total
  const unsigned char *wallface;  // [4 ncell] 1 where (cell, side) is a wall face
  double *x;                      // [n] the state the running sweep started from
  double *fp, *gp;                // [n] f = g - x and g of the latest iteration
  double *dF, *dG;                // [m][n] differences of consecutive f and g (a ring)
  double *red;                    // [kAARed] reduction slots
  double *gram;                   // [m][m] dF_i . dF_j
  double *gamma;                  // [m] mixing coefficients
  int *meta;                      // [3] columns held, next ring slot, iterations gathered
  int flow_comp;                  // moment index of the flow velocity (1: u1, 2: u2 when stored transposed)
};

struct InstanceDesc {
  int nx, ny, ncell;
  int periodic_x, periodic_y;
  int ngroups, groups_per_quadrant;
  int n_gas;
  int uniform_delta;
  int fin_nblocks;      // blocks of this instance in the finalize grids
  int fp32;             // 1 = FP32 storage (enables the noise-floor exit of the stopping test)
  int flow_axis;        // 0: the force, the moving plate's drift, Q and the stopping test are along x1;
                        // 1: along x2 (the caller's grid stored transposed: its x1 is this grid's x2)
  double dx;            // cell size along x (the mean column width when columns differ)
  double dy;            // cell size along y
  double dA_over_Lx;    // cell area / length of the grid along the flow axis (times xwidth[i] if set)
  const double *xwidth; // [nx] column widths / dx, or nullptr (equal columns)
  double delta;         // uniform collision rate
  double force;         // F
  double alpha;         // accommodation: wall value alpha rho_w + (1 - alpha) h(mirror v), Eq. (diffuse2)
  double top_u;         // speed of the moving plate (Couette flow), or 0
  int nwall;            // wall faces (gas cell, side) with a solid or outside neighbour across the side
  const int *wall_slot; // [ncell][4] -> face slot or -1 (alpha < 1 only)
  void *wbuf;           // [2 parities][nwall][2][groups_per_quadrant][32] T: incident h at each wall face
                        // from the previous sweep, by the sign of the velocity component along the face
  double sumW[4];       // sum W, sum W v1, sum W v2, sum W |v|^2
  double ginv[16];      // inverse Gram matrix of psi = (1, v1, v2, |v|^2) under the weights W
  double ain[4];        // per side: sum_{v.n<0} |v.n| W  (incident weight of a constant)
  double nrm[4];        // per side: sum_{v.n>0} (v.n) W  (outgoing normaliser)
  double wnrm[4];       // per side: alpha / nrm, the diffuse wall value per unit incident flux
  int ginv_sparse;      // 1: ginv couples only (1, |v|^2) (entries off that pattern are exactly 0)
  const void *vel;      // [ngroups][kNumVelFields][32] T
  const void *inv_den;  // [ngroups][kInvRows][32] T: 1 / (delta + cx kx + cy ky), uniform delta only; row 9 = 0
  void *rec;            // [4][ncell] SweepRec<T>
  void *rec_diag;       // [4][nx + ny - 1][nx] SweepRec<T>: the same records along the anti-diagonals of
                        // each quadrant's sweep order (column sweep), see diag_slot
  const uint32_t *code4;   // [ncell][4]
  const int *hw_src;       // [ncell][8]: (quadrant, axis) -> owner cell * 4 + side, or -1
  const double *delta_field;  // [ncell] or nullptr
  double *acc;          // [ncell][4]   moment accumulators of the running sweep
  double *facc;         // [2][ncell][4] incident wall-flux accumulators (by iteration parity)
  double *mom;          // [ncell][4]   rho, u1, u2, tau of the current state
  double *u1prev;       // [ncell] velocity along the flow axis after the previous sweep
  void *seam_x;         // [ngroups][ny][2][32] T: last two columns of the previous sweep
  void *seam_y;         // [ngroups][nx][2][32] T: last two rows of the previous sweep
  void *h;              // [ngroups][ncell][32] T, or nullptr
  DeviceState *state;
  // adjoint view only: the forward state the gradient is taken at
  const void *h_fwd;           // forward h, [ngroups][ncell][32] T
  const double *mom_fwd;       // forward moments [ncell][4]
  const DeviceState *state_fwd;
  double *grad;                // [ncell] dQ / d delta_c
  AndersonDesc *aa;            // Anderson mixing state (device), or nullptr: plain source iteration
  // Correction phase of the mixed-precision refinement (dvm_refine.cu), or nullptr: the iteration
  // d <- P S(d) + rho with no drive.  rho = [4 ncell] moments (rho, u1, u2, tau) | [4 ncell] projected
  // wall-face fluxes (cell * 4 + side) | [1] mass shift; rho_seam_x / _y have the layout of seam_x / _y.
  const double *rho;
  const void *rho_seam_x, *rho_seam_y;
};

// Launch descriptor shared by the kernels of one (possibly batched) iteration.
struct LaunchDesc {
  const InstanceDesc *inst;  // device array [ninst]
  const int *sweep_map;      // [sweep blocks]: instance << 16 | part << 12 | group; for the row sweep the
                             // 4-bit field is the number of consecutive groups swept side by side (0 = 1)
  const int *fin_map;        // [finalize blocks]: instance << 16 | block within instance
  int ninst;
  int warps;                 // sweep warps per block: max over instances of ceil(nx / cw)
  int row_tiles;             // row sweep: most velocity groups a block sweeps side by side (shared-memory
                             // layout); a sweep-map entry carries its own count
  int cw;                    // chunk width (cells per warp and step) of the sweep: 1, 2, 4, 8 or 16
  int pair_smem;             // FP32 row sweep: shared-memory bytes of the largest paired block's layout (0: the
                             // launch has no paired blocks; their sweep-map entries carry kPairFlag)
  int cols_v;                // 0: row-wavefront sweep; 1, 2, 4: column sweep with that many threads per
                             // column (the block's velocity set is split among them)
  int specular;              // 1: some instance has accommodation < 1 or a moving plate (column sweep only)
  int anderson;              // 1: some instance mixes its iterates (dvm_anderson.cu)
  int aa_blocks;             // blocks per instance of the mixing kernels
};

// Scheduler of the persistent batched launch (dvm_persist.cu).  Instance i's work items per sweep:
// tile_count[i] sweep tiles (sweep-map entries tiles[tile_base[i] ...]), then fin_items[i] chunks of
// fin_cells cells twice (mass shift; moments, records and stopping test).
constexpr int kPersistSpinLimit = 1 << 22;  // polls of an idle block before it gives up (~1 s)
struct PersistDesc {
  int ninst;
  int fin_cells;
  const int *order;            // [ninst] instances in scan order (longest sweeps first)
  const int *tile_base;        // [ninst]
  const int *tile_count;       // [ninst]
  const int *tiles;            // sweep-map entries grouped by instance
  const int *fin_items;        // [ninst]
  unsigned long long *work;    // [ninst] stage counter << 32 | items taken
  unsigned int *finished;      // [ninst] items of the current stage finished
  int *left;                   // [ninst] sweeps left in this launch
  int *active;                 // instances not retired in this launch
  int *error;                  // an idle block's poll limit ran out
};

#ifdef __CUDACC__
// FP64 reduction into global memory without a return value (PTX red): the warp does not wait for the
// L2 round trip that atomicAdd's returned old value would cost.
__device__ __forceinline__ void red_add(double *addr, double v) {
  asm volatile("red.global.add.f64 [%0], %1;\n" ::"l"(__cvta_generic_to_global(addr)), "d"(v) : "memory");
}
#endif

}  // namespace dvm
