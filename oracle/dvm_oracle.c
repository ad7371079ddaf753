/*
 * dvm_oracle.c -- plain FP64 CPU reference for the discrete velocity method (DVM) applied to the
 * steady linearized BGK equation (Lindsay, Su, Liu & Wu, arXiv:1704.03126, Sec. II.A).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is checked against.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (paper notation; the paper's Eq. labels in brackets):
 *   h(x, v)      perturbation of the VDF, f = f_eq (1 + h), f_eq = exp(-|v|^2) / pi  [Sec. II.A]
 *   delta        sqrt(pi) / (2 Kn), the collision rate in front of the BGK operator   [Eq. BGK]
 *   L(rho,u,tau) delta [rho + 2 u.v + tau (|v|^2 - 1)]                               [Eq. BGK]
 *   moments      rho = int h f_eq, u_i = int v_i h f_eq, tau = int |v|^2 h f_eq - rho
 *   iteration    delta h^{n+1} + v . grad h^{n+1} = L(rho^n, u^n, tau^n) + force     [Eq. iteration]
 *   derivatives  second-order upwind finite differences                              [Eq. iteration]
 *   walls        diffuse reflection, h_out = 2 sqrt(pi) int_{v_n<0} |v_n| h f_eq     [Eq. diffuse2]
 *   periodic     inlet/outlet (and for porous media both axes) are periodic           [Sec. II.A, III]
 *   Q            int v1 f dv dx1 dx2 / L  ( = sum u1 dA / L )                          [Sec. III, Eq. Q]
 *   k_a          sqrt(4/pi) Q Kn                                                       [Sec. III, Eq. k_a]
 *
 * Readings where the paper is silent (each one is restated in the design notes):
 *   force     the Poiseuille flow is driven by a unit body force along x1, i.e. a source +F v1.
 *   weights   velocity weights (never printed for Eq. nonuniform_v) are the trapezoid rule in the
 *             uniform parameter s, times exp(-v^2)/sqrt(pi); Newton-Cotes = closed trapezoid on
 *             [-vmax, vmax]; Gauss-Hermite nodes/weights divided by sqrt(pi).
 *   stencil   cell-centred grid, walls on cell faces.  Along one axis, with s = sign(v_a),
 *             u1 = cell - s, u2 = cell - 2 s, the term v_a dh/dx_a is (|v_a|/dx) (kappa h0 - combo):
 *               both upstream cells gas : kappa = 3/2, combo = 2 h(u1) - h(u2)/2  (second order)
 *               u1 gas, u2 solid        : kappa = 1,   combo = h(u1)              (first order)
 *               u1 solid                : kappa = 2,   combo = 2 h_w(face cell|u1)
 *             The last is the linear interpolant through the wall-face value.  Every form is exact
 *             on linear fields.  The quadratic through h0, h(u1) and the wall value would put a
 *             negative weight on the lagged wall value, and the iteration then diverges in narrow
 *             pores (an oscillating mode), so the second cell from a wall is first order.
 *   spacing   x1 spacing dx is uniform; the rows may have heights dy_j (Sec. II.A: the paper puts 60
 *             rows across the rough band and 100 above it).  With upstream centre distances
 *             d1 = (dy_c + dy_u1)/2 and d2 = d1 + (dy_u1 + dy_u2)/2 the three forms become the
 *             derivative at the cell centre of the Lagrange interpolant through the same points:
 *             interior kappa = 1/d1 + 1/d2, combo = d2/(d1 (d2-d1)) h(u1) - d1/(d2 (d2-d1)) h(u2);
 *             first order kappa = 1/d1, combo = h(u1)/d1; next to a wall (face at dy_c/2)
 *             kappa = 2/dy_c, combo = (2/dy_c) h_w -- per unit length, multiplied by |v2|.  For
 *             equal heights they are the forms above divided by dx.  Still exact on linear fields.
 *             Q weights each cell by its area dx dy_j.
 *   moving    the plate beyond the last row (x2 = H, non-periodic x2) may move along x1 with speed
 *             U (Couette flow, Sec. II.A, Eq. diffuse1): its reflected molecules carry the drift
 *             2 U v1 in addition to rho_w; every other wall is at rest (Eq. diffuse2).
 *   wall      h_w = alpha rho_w + (1 - alpha) h(mirror v) at the face's gas cell, where
 *             rho_w = sum_{v.n<0} |v.n| W h / sum_{v.n>0} (v.n) W (discrete zero mass flux).
 *   collision the discrete L is the projection of h onto span{1, v1, v2, |v|^2} in the quadrature
 *             inner product, L = delta sum_i a_i psi_i(v) with a = G^{-1} m, G_ij = sum_k W psi_i psi_j
 *             and m_j = sum_k W psi_j h (psi = 1, v1, v2, |v|^2).  For an exact quadrature this is
 *             delta [rho + 2 u.v + tau (|v|^2 - 1)] of Eq. BGK; for an inexact one it still conserves
 *             the discrete mass, momentum and energy, as the BGK operator does.
 *   lagging   values across a periodic seam and the wall values come from the previous iterate.
 *   mass      h = const solves the homogeneous problem; after every sweep the mean density over
 *             the gas cells is projected to zero by a constant shift s, accumulated in c, and the
 *             source carries -delta c.  The fixed point is the bordered system
 *               (delta + v.D) h - delta M(h) + delta c = F v1,   mean_gas rho(h) = 0.
 *   stop      eps_n = sum|u1^n - u1^{n-1}| / sum|u1^n|; r = (eps_n / eps_{n-4})^{1/4} clamped to
 *             [0, 0.9999]; stop when n >= 5 and eps_n / (1 - r) < tol.
 *
 * Layout: h[k][j][i], k = a * nv + b over the tensor-product velocity grid (v1 = x_a, v2 = x_b),
 * j the x2 (row) index, i the x1 index.  mask[j][i] = 1 marks a solid cell.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENOCONV 4
#define ORC_ENUMERIC 6

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------------------------ */
/* One-dimensional velocity quadratures.  Weights approximate int g(x) exp(-x^2)/sqrt(pi) dx.   */
/* ------------------------------------------------------------------------------------------ */

/* Orthonormal Hermite polynomials for the weight exp(-x^2): returns p_n(x) and
 * sum_{m<n} p_m(x)^2 (the Christoffel function's reciprocal). */
static double hermite_pn(int n, double x, double *sumsq) {
  double p_prev = 0.0, p = pow(M_PI, -0.25), s = 0.0;
  for (int m = 0; m < n; ++m) {
    s += p * p;
    double p_next = x * sqrt(2.0 / (m + 1)) * p - sqrt((double)m / (m + 1)) * p_prev;
    p_prev = p;
    p = p_next;
  }
  if (sumsq) *sumsq = s;
  return p;
}

/* Gauss-Hermite rule with n (even) nodes: roots of p_n bracketed on a fine scan of [0, sqrt(2n+1)]
 * and bisected; weight = 1 / sum_{m<n} p_m(x)^2 (Christoffel), divided by sqrt(pi). */
int orc_quad_gauss_hermite(int n, double *x, double *w) {
  if (n < 2 || (n & 1)) return ORC_EINVAL;
  int half = n / 2, found = 0;
  double L = sqrt(2.0 * n + 1.0) + 1.0;
  double dx = (M_PI / sqrt(2.0 * n + 1.0)) / 64.0;
  double xa = 0.0, pa = hermite_pn(n, xa, NULL);
  while (xa < L && found < half) {
    double xb = xa + dx, pb = hermite_pn(n, xb, NULL);
    if (pa == 0.0 || pa * pb < 0.0) {
      double lo = xa, hi = xb, plo = pa;
      for (int it = 0; it < 200 && hi - lo > 1e-17 * (1.0 + hi); ++it) {
        double mid = 0.5 * (lo + hi), pm = hermite_pn(n, mid, NULL);
        if (plo == 0.0) break;
        if (plo * pm <= 0.0) hi = mid; else { lo = mid; plo = pm; }
      }
      double root = (pa == 0.0) ? xa : 0.5 * (lo + hi);
      double sumsq;
      hermite_pn(n, root, &sumsq);
      x[half + found] = root;
      w[half + found] = 1.0 / sumsq / sqrt(M_PI);
      ++found;
    }
    xa = xb;
    pa = pb;
  }
  if (found != half) return ORC_EINVAL;
  for (int m = 0; m < half; ++m) {
    x[half - 1 - m] = -x[half + m];
    w[half - 1 - m] = w[half + m];
  }
  return ORC_OK;
}

/* Closed trapezoid (degree-1 Newton-Cotes) on n equispaced nodes in [-vmax, vmax]. */
int orc_quad_newton_cotes(int n, double vmax, double *x, double *w) {
  if (n < 2 || (n & 1) || !(vmax > 0.0)) return ORC_EINVAL;
  double hstep = 2.0 * vmax / (n - 1);
  for (int a = 0; a < n; ++a) {
    x[a] = -vmax + a * hstep;
    double end = (a == 0 || a == n - 1) ? 0.5 : 1.0;
    w[a] = hstep * end * exp(-x[a] * x[a]) / sqrt(M_PI);
  }
  return ORC_OK;
}

/* Non-uniform cubic grid of Eq. (nonuniform_v): v = 4 s^3 / (n-1)^3, s = -n+1, -n+3, ..., n-1.
 * Weight: trapezoid rule in s (step 2) applied to g(v(s)) v'(s), v'(s) = 12 s^2 / (n-1)^3. */
int orc_quad_cubic(int n, double *x, double *w) {
  if (n < 2 || (n & 1)) return ORC_EINVAL;
  double d3 = pow((double)(n - 1), 3.0);
  for (int a = 0; a < n; ++a) {
    double s = (double)(-n + 1 + 2 * a);
    x[a] = 4.0 * s * s * s / d3;
    double end = (a == 0 || a == n - 1) ? 0.5 : 1.0;
    w[a] = 2.0 * end * (12.0 * s * s / d3) * exp(-x[a] * x[a]) / sqrt(M_PI);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Problem description and geometry helpers.                                                   */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int nx, ny;                /* cells along x1 and x2 */
  int periodic_x, periodic_y;
  double dx;                 /* square cell size (H / ny) */
  const unsigned char *mask; /* [ny][nx], 1 = solid */
  const double *delta;       /* [ny][nx] rarefaction (collision rate) per cell */
  int nv;                    /* nodes per velocity axis */
  const double *xv, *wv;     /* 1D nodes and weights; velocity k = a*nv + b has v = (x_a, x_b) */
  double alpha;              /* accommodation: 1 = fully diffuse walls */
  double force;              /* body-force source coefficient F (source F v1) */
  double top_u;              /* speed U along x1 of the plate beyond the last row (Couette), or 0 */
  const double *dy;          /* row heights [ny] (x2 spacing), or NULL: square cells of size dx */
  int collision;             /* 0: projection onto the collision invariants (default); 1: Eq. BGK as
                                printed, delta [rho + 2 u.v + tau (|v|^2 - 1)] with quadrature moments */
} orc_problem;

enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* 1 when cell (i, j) is solid or lies outside a non-periodic axis. */
static int solid_at(const orc_problem *p, int i, int j) {
  if (i < 0 || i >= p->nx) {
    if (!p->periodic_x) return 1;
    i = wrap(i, p->nx);
  }
  if (j < 0 || j >= p->ny) {
    if (!p->periodic_y) return 1;
    j = wrap(j, p->ny);
  }
  return p->mask[(size_t)j * p->nx + i] != 0;
}

static size_t cell_id(const orc_problem *p, int i, int j) {
  return (size_t)wrap(j, p->ny) * p->nx + wrap(i, p->nx);
}

/* Component of v_k along the inward normal of a wall on the given side of a gas cell.
 * A solid neighbour on the W side means the wall normal pointing into the gas is +x1. */
static double v_dot_n(const orc_problem *p, int k, int side) {
  double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
  switch (side) {
    case SIDE_W: return v1;
    case SIDE_E: return -v1;
    case SIDE_S: return v2;
    default: return -v2;
  }
}

/* Index of the velocity mirrored across a wall with the given side (reverses the normal part).
 * All grids here are symmetric, x_{nv-1-a} = -x_a. */
static int mirror_velocity(const orc_problem *p, int k, int side) {
  int a = k / p->nv, b = k % p->nv;
  if (side == SIDE_W || side == SIDE_E) a = p->nv - 1 - a;
  else b = p->nv - 1 - b;
  return a * p->nv + b;
}

/* Inverse of the 4 x 4 Gram matrix G_ij = sum_k W_k psi_i(v_k) psi_j(v_k), psi = (1, v1, v2, |v|^2),
 * by Gauss-Jordan elimination with partial pivoting.  Returns 0 when G is singular. */
static int gram_inverse(const orc_problem *p, double ginv[16]) {
  double a[4][8];
  int K = p->nv * p->nv;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = (j - 4 == i) ? 1.0 : 0.0;
  for (int k = 0; k < K; ++k) {
    double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
    double W = p->wv[k / p->nv] * p->wv[k % p->nv];
    double psi[4] = {1.0, v1, v2, v1 * v1 + v2 * v2};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a[i][j] += W * psi[i] * psi[j];
  }
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
    if (a[piv][col] == 0.0) return 0;
    for (int j = 0; j < 8; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
    double d = a[col][col];
    for (int j = 0; j < 8; ++j) a[col][j] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      double f = a[r][col];
      for (int j = 0; j < 8; ++j) a[r][j] -= f * a[col][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) ginv[i * 4 + j] = a[i][j + 4];
  return 1;
}

/* Collision coefficients a of every gas cell in the basis psi = (1, v1, v2, |v|^2), so that
 * L = delta sum_i a_i psi_i(v):
 *   projection (collision = 0): a = G^{-1} m with m = (rho, u1, u2, tau + rho);
 *   literal    (collision = 1): Eq. BGK as printed, rho + 2 u.v + tau (|v|^2 - 1), i.e.
 *                               a = (rho - tau, 2 u1, 2 u2, tau).
 * The two coincide when the quadrature integrates psi_i psi_j f_eq exactly. */
static void collision_coefficients(const orc_problem *p, const double ginv[16], const double *rho,
                                   const double *u1, const double *u2, const double *tau, double *a) {
  size_t ncell = (size_t)p->nx * p->ny;
  for (size_t c = 0; c < ncell; ++c) {
    double m[4] = {rho[c], u1[c], u2[c], tau[c] + rho[c]};
    double lit[4] = {rho[c] - tau[c], 2.0 * u1[c], 2.0 * u2[c], tau[c]};
    for (int i = 0; i < 4; ++i) {
      double s = 0;
      for (int j = 0; j < 4; ++j) s += ginv[i * 4 + j] * m[j];
      if (p->collision == 1) s = lit[i];
      a[c * 4 + i] = p->mask[c] ? 0.0 : s;
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Moments, wall values and one transport sweep.                                              */
/* ------------------------------------------------------------------------------------------ */

/* rho, u1, u2, tau at every gas cell (moments of Sec. II.A); solid cells get 0. */
static void compute_moments(const orc_problem *p, const double *h, double *rho, double *u1,
                            double *u2, double *tau) {
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < (long)ncell; ++c) {
    double r = 0, m1 = 0, m2 = 0, e = 0;
    if (!p->mask[c]) {
      for (int k = 0; k < K; ++k) {
        double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
        double W = p->wv[k / p->nv] * p->wv[k % p->nv];
        double hk = h[(size_t)k * ncell + c];
        r += W * hk;
        m1 += W * v1 * hk;
        m2 += W * v2 * hk;
        e += W * (v1 * v1 + v2 * v2) * hk;
      }
    }
    rho[c] = r;
    u1[c] = m1;
    u2[c] = m2;
    tau[c] = e - r;
  }
}

/* Diffuse wall density rho_w for every (gas cell, side) whose neighbour on that side is solid:
 * incident flux sum_{v.n<0} |v.n| W h over the outgoing normaliser sum_{v.n>0} (v.n) W  [Eq. diffuse2]. */
static void compute_wall_density(const orc_problem *p, const double *h, double *rho_w) {
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
  double norm[4];
  for (int side = 0; side < 4; ++side) {
    norm[side] = 0;
    for (int k = 0; k < K; ++k) {
      double vn = v_dot_n(p, k, side);
      if (vn > 0) norm[side] += vn * p->wv[k / p->nv] * p->wv[k % p->nv];
    }
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < (long)ncell; ++c) {
    int i = (int)(c % p->nx), j = (int)(c / p->nx);
    const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
    for (int side = 0; side < 4; ++side) {
      double val = 0;
      if (!p->mask[c] && solid_at(p, i + di[side], j + dj[side])) {
        double flux = 0;
        for (int k = 0; k < K; ++k) {
          double vn = v_dot_n(p, k, side);
          if (vn < 0) flux += -vn * p->wv[k / p->nv] * p->wv[k % p->nv] * h[(size_t)k * ncell + c];
        }
        val = flux / norm[side];
      }
      rho_w[c * 4 + side] = val;
    }
  }
}

/* Wall value seen by velocity k on the given side of gas cell c: diffuse part from rho_w plus the
 * specular part from the previous iterate at the mirrored velocity. */
static double wall_value(const orc_problem *p, const double *rho_w, const double *h_old, size_t c,
                         int side, int k) {
  size_t ncell = (size_t)p->nx * p->ny;
  double hw = p->alpha * rho_w[c * 4 + side];
  /* the moving plate: the wall Maxwellian drifts with U, rho_w + 2 U v1 (Eq. diffuse1) */
  if (p->top_u != 0.0 && side == SIDE_N && !p->periodic_y && (int)(c / p->nx) == p->ny - 1)
    hw += p->alpha * 2.0 * p->top_u * p->xv[k / p->nv];
  if (p->alpha < 1.0) hw += (1.0 - p->alpha) * h_old[(size_t)mirror_velocity(p, k, side) * ncell + c];
  return hw;
}

/* Upwind contribution along one axis for gas cell (i, j): fills kappa and combo such that
 * v_a dh/dx_a = (|v_a|/dx) (kappa h(i,j) - combo).  (di, dj) is the unit step along the axis and s
 * the sign of v_a.  hk is the velocity's own array, updated in place, so that a wrapped (periodic)
 * upstream cell, visited later in the sweep, still holds the previous iterate. */
static void upwind_axis(const orc_problem *p, const double *hk, const double *rho_w,
                        const double *h_old, int k, int i, int j, int di, int dj, int s,
                        double *kappa, double *combo) {
  int side = (di != 0) ? (s > 0 ? SIDE_W : SIDE_E) : (s > 0 ? SIDE_S : SIDE_N);
  int i1 = i - s * di, j1 = j - s * dj, i2 = i - 2 * s * di, j2 = j - 2 * s * dj;
  if (p->dy && dj != 0) {
    /* rows of unequal height: Lagrange forms per unit length, scaled back by dx for the caller's
     * (|v|/dx) factor */
    double hc = p->dy[j];
    if (solid_at(p, i1, j1)) {
      *kappa = 2.0 / hc * p->dx;
      *combo = 2.0 / hc * p->dx * wall_value(p, rho_w, h_old, cell_id(p, i, j), side, k);
      return;
    }
    double d1 = 0.5 * (hc + p->dy[wrap(j1, p->ny)]);
    if (solid_at(p, i2, j2)) {
      *kappa = p->dx / d1;
      *combo = p->dx / d1 * hk[cell_id(p, i1, j1)];
      return;
    }
    double d2 = d1 + 0.5 * (p->dy[wrap(j1, p->ny)] + p->dy[wrap(j2, p->ny)]);
    *kappa = p->dx * (1.0 / d1 + 1.0 / d2);
    *combo = p->dx * (d2 / (d1 * (d2 - d1)) * hk[cell_id(p, i1, j1)] - d1 / (d2 * (d2 - d1)) * hk[cell_id(p, i2, j2)]);
    return;
  }
  if (solid_at(p, i1, j1)) {
    *kappa = 2.0;
    *combo = 2.0 * wall_value(p, rho_w, h_old, cell_id(p, i, j), side, k);
  } else if (solid_at(p, i2, j2)) {
    *kappa = 1.0;
    *combo = hk[cell_id(p, i1, j1)];
  } else {
    *kappa = 1.5;
    *combo = 2.0 * hk[cell_id(p, i1, j1)] - 0.5 * hk[cell_id(p, i2, j2)];
  }
}

/* Sweep velocity k over all gas cells in its upwind order, in place in hk = h[k]:
 *   (delta + sum_a |v_a|/dx kappa_a) h = R + sum_a |v_a|/dx combo_a,
 *   R = delta (a0 + a1 v1 + a2 v2 + a3 |v|^2 - c) + F v1         [Eq. iteration, Eq. BGK]
 * with the collision coefficients a of each cell (exact quadrature: a0 + a3 |v|^2 + ... =
 * rho + 2 u.v + tau (|v|^2 - 1)). */
static void sweep_velocity(const orc_problem *p, int k, double *hk, const double *acoef,
                           double c_shift, const double *rho_w, const double *h_old) {
  double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
  int s1 = v1 > 0 ? 1 : -1, s2 = v2 > 0 ? 1 : -1;
  double cx = fabs(v1) / p->dx, cy = fabs(v2) / p->dx, vsq = v1 * v1 + v2 * v2;
  for (int jj = 0; jj < p->ny; ++jj) {
    int j = s2 > 0 ? jj : p->ny - 1 - jj;
    for (int ii = 0; ii < p->nx; ++ii) {
      int i = s1 > 0 ? ii : p->nx - 1 - ii;
      size_t c = (size_t)j * p->nx + i;
      if (p->mask[c]) continue;
      double kx, bx, ky, by;
      upwind_axis(p, hk, rho_w, h_old, k, i, j, 1, 0, s1, &kx, &bx);
      upwind_axis(p, hk, rho_w, h_old, k, i, j, 0, 1, s2, &ky, &by);
      double d = p->delta[c];
      const double *a = acoef + c * 4;
      double R = d * (a[0] + a[1] * v1 + a[2] * v2 + a[3] * vsq - c_shift) + p->force * v1;
      hk[c] = (R + cx * bx + cy * by) / (d + cx * kx + cy * ky);
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Source iteration.                                                                           */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int iters;        /* sweeps performed */
  double eps;       /* last relative change of u1 */
  double est;       /* last error estimate eps / (1 - r) */
  double c_shift;   /* accumulated mass shift c */
  double Q;         /* mass flow rate sum u1 dA / Lx */
} orc_result;

static double q_flow(const orc_problem *p, const double *u1) {
  size_t ncell = (size_t)p->nx * p->ny;
  double q = 0;
  for (size_t c = 0; c < ncell; ++c)
    if (!p->mask[c]) q += u1[c] * (p->dy ? p->dy[c / p->nx] : p->dx);
  return q * p->dx / (p->nx * p->dx);
}

/* Solve by source iteration from the state in h (zeros for a cold start) and c_shift.
 * On return h holds the last iterate; rho/u1/u2/tau its moments.  eps_hist (optional, length
 * max_iter) receives eps_n. */
int orc_solve(const orc_problem *p, double tol, int max_iter, double *h, double c_shift,
              double *rho, double *u1, double *u2, double *tau, double *eps_hist,
              orc_result *res) {
  if (p->nx < 2 || p->ny < 2 || p->nv < 2 || (p->nv & 1) || max_iter < 1) return ORC_EINVAL;
  if (p->dy)
    for (int j = 0; j < p->ny; ++j)
      if (!(p->dy[j] > 0.0) || !isfinite(p->dy[j])) return ORC_EINVAL;
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
  long ngas = 0;
  for (size_t c = 0; c < ncell; ++c) ngas += !p->mask[c];
  if (ngas == 0) return ORC_EINVAL;
  double sumW = 0;
  for (int k = 0; k < K; ++k) sumW += p->wv[k / p->nv] * p->wv[k % p->nv];

  double ginv[16];
  if (!gram_inverse(p, ginv)) return ORC_EINVAL;
  double *rho_w = (double *)calloc(ncell * 4, sizeof(double));
  double *u1_prev = (double *)calloc(ncell, sizeof(double));
  double *acoef = (double *)calloc(ncell * 4, sizeof(double));
  double *h_old = (p->alpha < 1.0) ? (double *)malloc((size_t)K * ncell * sizeof(double)) : NULL;
  double eps_ring[4] = {0, 0, 0, 0}; /* slot n % 4 holds eps_{n-4} */
  if (!rho_w || !u1_prev || !acoef || (p->alpha < 1.0 && !h_old)) {
    free(rho_w); free(u1_prev); free(acoef); free(h_old);
    return ORC_ENOMEM;
  }
  compute_moments(p, h, rho, u1, u2, tau);
  memcpy(u1_prev, u1, ncell * sizeof(double));

  int status = ORC_ENOCONV, n;
  double eps = 1.0, est = INFINITY;
  for (n = 1; n <= max_iter; ++n) {
    /* wall values and (for alpha < 1) the specular source from the previous iterate */
    compute_wall_density(p, h, rho_w);
    collision_coefficients(p, ginv, rho, u1, u2, tau, acoef);
    if (h_old) memcpy(h_old, h, (size_t)K * ncell * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < K; ++k)
      sweep_velocity(p, k, h + (size_t)k * ncell, acoef, c_shift, rho_w, h_old);

    /* project the mean gas density to zero: s = sum_gas rho / (n_gas sum W) */
    double mass = 0;
    for (int k = 0; k < K; ++k) {
      double W = p->wv[k / p->nv] * p->wv[k % p->nv], part = 0;
      for (size_t c = 0; c < ncell; ++c)
        if (!p->mask[c]) part += h[(size_t)k * ncell + c];
      mass += W * part;
    }
    double s = mass / ((double)ngas * sumW);
#pragma omp parallel for schedule(static)
    for (long kc = 0; kc < (long)((size_t)K * ncell); ++kc)
      if (!p->mask[kc % ncell]) h[kc] -= s;
    c_shift += s;

    compute_moments(p, h, rho, u1, u2, tau);
    double dsum = 0, usum = 0;
    int finite = isfinite(s);
    for (size_t c = 0; c < ncell; ++c) {
      if (p->mask[c]) continue;
      dsum += fabs(u1[c] - u1_prev[c]);
      usum += fabs(u1[c]);
      finite = finite && isfinite(rho[c]) && isfinite(u1[c]) && isfinite(u2[c]) && isfinite(tau[c]);
    }
    if (!finite) { status = ORC_ENUMERIC; break; }
    memcpy(u1_prev, u1, ncell * sizeof(double));
    eps = usum > 0 ? dsum / usum : 0.0;
    if (eps_hist) eps_hist[n - 1] = eps;
    double eps_back = eps_ring[n % 4];
    eps_ring[n % 4] = eps;
    est = INFINITY;
    if (n >= 5) {
      double r = eps_back > 0 ? pow(eps / eps_back, 0.25) : 0.0;
      if (r > 0.9999) r = 0.9999;
      est = eps / (1.0 - r);
      if (est < tol) { status = ORC_OK; break; }
    }
  }
  if (n > max_iter) n = max_iter;
  res->iters = n;
  res->eps = eps;
  res->est = est;
  res->c_shift = c_shift;
  res->Q = q_flow(p, u1);
  free(rho_w); free(u1_prev); free(acoef); free(h_old);
  return status;
}

/* One source-iteration sweep of the listed velocities from a given state, with no projection:
 * h_in is the full previous iterate [K][ny][nx]; the sweeps of velocities ks[0..nk) are written to
 * out[m][ny][nx].  Used to check single velocities of a large solve one by one. */
int orc_sweep_selected(const orc_problem *p, const double *h_in, double c_shift, const int *ks,
                       int nk, double *out) {
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
  double ginv[16];
  if (!gram_inverse(p, ginv)) return ORC_EINVAL;
  double *rho = (double *)malloc(ncell * sizeof(double) * 8);
  double *rho_w = (double *)calloc(ncell * 4, sizeof(double));
  if (!rho || !rho_w) { free(rho); free(rho_w); return ORC_ENOMEM; }
  double *u1 = rho + ncell, *u2 = rho + 2 * ncell, *tau = rho + 3 * ncell, *acoef = rho + 4 * ncell;
  compute_moments(p, h_in, rho, u1, u2, tau);
  collision_coefficients(p, ginv, rho, u1, u2, tau, acoef);
  compute_wall_density(p, h_in, rho_w);
  int status = ORC_OK;
  for (int m = 0; m < nk; ++m) {
    if (ks[m] < 0 || ks[m] >= K) { status = ORC_EINVAL; break; }
    memcpy(out + (size_t)m * ncell, h_in + (size_t)ks[m] * ncell, ncell * sizeof(double));
    sweep_velocity(p, ks[m], out + (size_t)m * ncell, acoef, c_shift, rho_w, h_in);
  }
  free(rho); free(rho_w);
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint of the projected source iteration: gradient of Q with respect to delta per cell.    */
/* ------------------------------------------------------------------------------------------ */
/*
 * Write one iteration as Phi(h, c) = P(S(h, c)): S solves T h~ = delta (M(h) - c) + L(h) + F v1
 * (T: the in-sweep upwind operator, L: wall and periodic-seam terms taken from h), P shifts
 * h~ by s = rho^T h~ (rho = W / (n_gas sum W)) and adds s to c.  At the fixed point x* = Phi(x*),
 * dQ/d delta = Lambda^T dPhi/d delta with Lambda = J^T Lambda + (g, 0), g = W v1 dA / Lx.
 * One adjoint step, given (lambda, mu):
 *   lambda' = lambda + rho (mu - sum lambda)              (transpose of P)
 *   z       = T^{-T} lambda'                              (reverse-order sweep per velocity)
 *   lambda  = (delta M)^T z + L^T z + g,  mu = mu - sum delta z
 * and dQ/d delta_c = sum_k z_kc (M_kc - c - h_kc), M_kc = a(c) . psi(v_k) the collision part.
 * Identity at convergence: Q = F sum z v1.
 */

/* Coefficients of the forward stencil of gas cell (i, j) along one axis (step (di, dj), sign s), in the
 * normalised form v_a dh/dx_a = (|v_a|/dx) (kap h0 - w1 ref1 - w2 ref2): returns 2 when ref1 is the wall
 * value (u1 solid), 1 for first order (ref1 = h(u1)), 0 for the interior form (ref1 = h(u1), ref2 =
 * h(u2)).  Rows of unequal height give the Lagrange forms of upwind_axis scaled by dx. */
static int stencil_weights(const orc_problem *p, int i, int j, int di, int dj, int s, double *kap, double *w1,
                           double *w2) {
  int i1 = i - s * di, j1 = j - s * dj, i2 = i - 2 * s * di, j2 = j - 2 * s * dj;
  *w2 = 0.0;
  if (p->dy && dj != 0) {
    double hc = p->dy[j];
    if (solid_at(p, i1, j1)) {
      *kap = *w1 = 2.0 / hc * p->dx;
      return 2;
    }
    double d1 = 0.5 * (hc + p->dy[wrap(j1, p->ny)]);
    if (solid_at(p, i2, j2)) {
      *kap = *w1 = p->dx / d1;
      return 1;
    }
    double d2 = d1 + 0.5 * (p->dy[wrap(j1, p->ny)] + p->dy[wrap(j2, p->ny)]);
    *kap = p->dx * (1.0 / d1 + 1.0 / d2);
    *w1 = p->dx * d2 / (d1 * (d2 - d1));
    *w2 = -p->dx * d1 / (d2 * (d2 - d1));
    return 0;
  }
  if (solid_at(p, i1, j1)) {
    *kap = *w1 = 2.0;
    return 2;
  }
  if (solid_at(p, i2, j2)) {
    *kap = *w1 = 1.0;
    return 1;
  }
  *kap = 1.5;
  *w1 = 2.0;
  *w2 = -0.5;
  return 0;
}

/* Push form of the transposed upwind sweep for velocity k: acc holds lambda'_k on entry and is
 * consumed; z (output) gets T_k^{-T} lambda'_k.  Contributions through lagged references (wrapped
 * seam cells and wall values) go to lam_new (the L^T z part). */
static void adjoint_sweep_velocity(const orc_problem *p, int k, double *acc, double *zk,
                                   double *lam_new, const double *norm_side) {
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
  double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
  int s1 = v1 > 0 ? 1 : -1, s2 = v2 > 0 ? 1 : -1;
  double cxy[2] = {fabs(v1) / p->dx, fabs(v2) / p->dx};
  /* reverse of the forward order: forward visits jj = 0..ny-1, ii = 0..nx-1 */
  for (int jj = p->ny - 1; jj >= 0; --jj) {
    int j = s2 > 0 ? jj : p->ny - 1 - jj;
    for (int ii = p->nx - 1; ii >= 0; --ii) {
      int i = s1 > 0 ? ii : p->nx - 1 - ii;
      size_t c = (size_t)j * p->nx + i;
      if (p->mask[c]) continue;
      /* diagonal of the forward row for this cell */
      double diag = p->delta[c];
      double kap[2], w1[2], w2[2];
      int cls[2];
      for (int ax = 0; ax < 2; ++ax) {
        int di = ax == 0, dj = ax == 1, s = ax == 0 ? s1 : s2;
        cls[ax] = stencil_weights(p, i, j, di, dj, s, &kap[ax], &w1[ax], &w2[ax]);
        diag += cxy[ax] * kap[ax];
      }
      double z = acc[c] / diag;
      zk[c] = z;
      /* the forward row reads, with coefficient a, either h_k at an upstream cell or a wall value */
      for (int ax = 0; ax < 2; ++ax) {
        int di = ax == 0, dj = ax == 1, s = ax == 0 ? s1 : s2;
        int side = ax == 0 ? (s > 0 ? SIDE_W : SIDE_E) : (s > 0 ? SIDE_S : SIDE_N);
        int i1 = i - s * di, j1 = j - s * dj, i2 = i - 2 * s * di, j2 = j - 2 * s * dj;
        /* refs: (cell index or -1 for wall, wall owner, coefficient, wrapped flag) */
        size_t ref_cell[2];
        int ref_is_wall[2], ref_wrapped[2], nref = 0;
        double ref_coef[2];
        int wrapped1 = (ax == 0) ? (i1 < 0 || i1 >= p->nx) : (j1 < 0 || j1 >= p->ny);
        int wrapped2 = (ax == 0) ? (i2 < 0 || i2 >= p->nx) : (j2 < 0 || j2 >= p->ny);
        if (cls[ax] == 2) {
          ref_cell[0] = c; ref_is_wall[0] = 1; ref_wrapped[0] = 0; ref_coef[0] = w1[ax]; nref = 1;
        } else if (cls[ax] == 1) {
          ref_cell[0] = cell_id(p, i1, j1); ref_is_wall[0] = 0; ref_wrapped[0] = wrapped1;
          ref_coef[0] = w1[ax];
          nref = 1;
        } else {
          ref_cell[0] = cell_id(p, i1, j1); ref_is_wall[0] = 0; ref_wrapped[0] = wrapped1;
          ref_coef[0] = w1[ax];
          ref_cell[1] = cell_id(p, i2, j2); ref_is_wall[1] = 0; ref_wrapped[1] = wrapped2;
          ref_coef[1] = w2[ax];
          nref = 2;
        }
        for (int r = 0; r < nref; ++r) {
          double t = cxy[ax] * ref_coef[r] * z;
          if (!ref_is_wall[r]) {
            if (ref_wrapped[r]) lam_new[(size_t)k * ncell + ref_cell[r]] += t; /* lagged seam */
            else acc[ref_cell[r]] += t;                                        /* in-sweep */
          } else {
            /* wall value h_w = alpha rho_w(owner, side) + (1 - alpha) h_old[mirror k][owner] */
            size_t owner = ref_cell[r];
            if (p->alpha > 0.0) {
              for (int kk = 0; kk < K; ++kk) {
                double vn = v_dot_n(p, kk, side);
                if (vn < 0)
                  lam_new[(size_t)kk * ncell + owner] +=
                      p->alpha * t * (-vn) * p->wv[kk / p->nv] * p->wv[kk % p->nv] / norm_side[side];
              }
            }
            if (p->alpha < 1.0)
              lam_new[(size_t)mirror_velocity(p, k, side) * ncell + owner] += (1.0 - p->alpha) * t;
          }
        }
      }
    }
  }
}

/* Adjoint solve at a converged forward state (h, c_shift): returns dQ/d delta_c in grad[ny][nx]
 * (0 in solid cells) and Q_adj = F sum z v1 dA-weighted identity value. */
int orc_adjoint(const orc_problem *p, const double *h, double c_shift, double tol, int max_iter,
                double *grad, double *q_identity, int *iters_out) {
  size_t ncell = (size_t)p->nx * p->ny;
  int K = p->nv * p->nv;
  long ngas = 0;
  for (size_t c = 0; c < ncell; ++c) ngas += !p->mask[c];
  /* the transposed collision below is that of the projection (collision = 0) */
  if (ngas == 0 || max_iter < 1 || p->collision != 0) return ORC_EINVAL;
  double sumW = 0;
  for (int k = 0; k < K; ++k) sumW += p->wv[k / p->nv] * p->wv[k % p->nv];
  double norm_side[4];
  for (int side = 0; side < 4; ++side) {
    norm_side[side] = 0;
    for (int k = 0; k < K; ++k) {
      double vn = v_dot_n(p, k, side);
      if (vn > 0) norm_side[side] += vn * p->wv[k / p->nv] * p->wv[k % p->nv];
    }
  }
  size_t N = (size_t)K * ncell;
  double *lam = (double *)calloc(N, sizeof(double));
  double *lam_new = (double *)calloc(N, sizeof(double));
  double *acc = (double *)malloc(N * sizeof(double));
  double *z = (double *)calloc(N, sizeof(double));
  double *mom = (double *)malloc(4 * ncell * sizeof(double));
  double *gprev = (double *)calloc(ncell, sizeof(double));
  if (!lam || !lam_new || !acc || !z || !mom || !gprev) {
    free(lam); free(lam_new); free(acc); free(z); free(mom); free(gprev);
    return ORC_ENOMEM;
  }
  double *rho = mom, *u1 = mom + ncell, *u2 = mom + 2 * ncell, *tau = mom + 3 * ncell;
  compute_moments(p, h, rho, u1, u2, tau);
  double ginv[16];
  double *acoef = (double *)malloc(4 * ncell * sizeof(double));
  if (!acoef || !gram_inverse(p, ginv)) {
    free(lam); free(lam_new); free(acc); free(z); free(mom); free(gprev); free(acoef);
    return acoef ? ORC_EINVAL : ORC_ENOMEM;
  }
  collision_coefficients(p, ginv, rho, u1, u2, tau, acoef);
  /* g = W v1 dA / L per cell: dA = dx dy_j, L = nx dx */
  double mu = 0.0;
  double eps_ring[4] = {0, 0, 0, 0}; /* slot n % 4 holds eps_{n-4} */
  int status = ORC_ENOCONV, n;
  for (n = 1; n <= max_iter; ++n) {
    /* lambda' = lambda + rho (mu - sum lambda) */
    double lsum = 0;
    for (size_t kc = 0; kc < N; ++kc)
      if (!p->mask[kc % ncell]) lsum += lam[kc];
    for (size_t kc = 0; kc < N; ++kc) {
      int k = (int)(kc / ncell);
      double W = p->wv[k / p->nv] * p->wv[k % p->nv];
      acc[kc] = p->mask[kc % ncell] ? 0.0 : lam[kc] + W / ((double)ngas * sumW) * (mu - lsum);
    }
    memset(lam_new, 0, N * sizeof(double));
    /* velocities push into shared lam_new entries through the wall terms: keep this serial */
    for (int k = 0; k < K; ++k)
      adjoint_sweep_velocity(p, k, acc + (size_t)k * ncell, z + (size_t)k * ncell, lam_new, norm_side);
    /* (delta M)^T z + g and mu update */
    double dz = 0;
    for (size_t c = 0; c < ncell; ++c) {
      if (p->mask[c]) continue;
      /* M_k(h) = sum_j W_j psi(v_k)^T G^{-1} psi(v_j) h_j, so (delta M)^T z at velocity j is
       * delta W_j psi(v_j)^T G^{-1} Z with Z = sum_k psi(v_k) z_k */
      double Z[4] = {0, 0, 0, 0}, GZ[4];
      for (int k = 0; k < K; ++k) {
        double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
        double zz = z[(size_t)k * ncell + c];
        Z[0] += zz; Z[1] += v1 * zz; Z[2] += v2 * zz; Z[3] += (v1 * v1 + v2 * v2) * zz;
      }
      for (int i = 0; i < 4; ++i) GZ[i] = ginv[i * 4] * Z[0] + ginv[i * 4 + 1] * Z[1] + ginv[i * 4 + 2] * Z[2] + ginv[i * 4 + 3] * Z[3];
      double d = p->delta[c];
      dz += d * Z[0];
      for (int k = 0; k < K; ++k) {
        double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
        double W = p->wv[k / p->nv] * p->wv[k % p->nv];
        lam_new[(size_t)k * ncell + c] +=
            d * W * (GZ[0] + GZ[1] * v1 + GZ[2] * v2 + GZ[3] * (v1 * v1 + v2 * v2)) +
            W * v1 * (p->dy ? p->dy[c / p->nx] : p->dx) / p->nx;
      }
    }
    mu -= dz;
    double *t = lam; lam = lam_new; lam_new = t;
    /* gradient from z and the forward state; relative change as the stopping test */
    double dsum = 0, gsum = 0;
    for (size_t c = 0; c < ncell; ++c) {
      double g = 0;
      if (!p->mask[c]) {
        for (int k = 0; k < K; ++k) {
          double v1 = p->xv[k / p->nv], v2 = p->xv[k % p->nv];
          const double *a = acoef + c * 4;
          double M = a[0] + a[1] * v1 + a[2] * v2 + a[3] * (v1 * v1 + v2 * v2);
          g += z[(size_t)k * ncell + c] * (M - c_shift - h[(size_t)k * ncell + c]);
        }
      }
      dsum += fabs(g - gprev[c]);
      gsum += fabs(g);
      grad[c] = g;
      gprev[c] = g;
    }
    double eps = gsum > 0 ? dsum / gsum : 0.0;
    double eps_back = eps_ring[n % 4];
    eps_ring[n % 4] = eps;
    if (n >= 5) {
      double r = eps_back > 0 ? pow(eps / eps_back, 0.25) : 0.0;
      if (r > 0.9999) r = 0.9999;
      if (eps / (1.0 - r) < tol) { status = ORC_OK; break; }
    }
  }
  if (n > max_iter) n = max_iter;
  double qid = 0;
  for (size_t kc = 0; kc < N; ++kc) {
    int k = (int)(kc / ncell);
    if (!p->mask[kc % ncell]) qid += p->force * z[kc] * p->xv[k / p->nv];
  }
  *q_identity = qid;
  *iters_out = n;
  free(lam); free(lam_new); free(acc); free(z); free(mom); free(gprev); free(acoef);
  return status;
}
