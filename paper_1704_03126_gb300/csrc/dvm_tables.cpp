// dvm_tables.cpp -- host-side tables of libdvm: velocity quadratures and geometry classes.
#include "dvm_tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace dvm {

namespace {

// Eigen-decomposition of a small symmetric matrix by cyclic Jacobi rotations (Golub & Van Loan,
// Sec. 8.5).  a is n x n row-major and is destroyed; eigenvalues go to lam, eigenvectors to the
// columns of v.
void jacobi_eigen(int n, std::vector<double> &a, std::vector<double> &lam, std::vector<double> &v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = a[(size_t)i * n + i];
}

}  // namespace

bool quadrature_1d(int kind, int n, double vmax, std::vector<double> &x, std::vector<double> &w, std::string &err) {
  if (n < 2 || n > 64 || (n & 1)) {
    err = "velocity grid: n must be even and in [2, 64]";
    return false;
  }
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double rpi = std::sqrt(M_PI);
  if (kind == 0) {
    // Gauss-Hermite by Golub-Welsch: nodes are the eigenvalues of the Jacobi matrix of the Hermite
    // recurrence (zero diagonal, off-diagonal sqrt(k/2)); weight = sqrt(pi) (first eigenvector
    // component)^2, then divided by sqrt(pi) for the normalised Maxwellian.
    std::vector<double> a((size_t)n * n, 0.0), lam, v;
    for (int k = 1; k < n; ++k) a[(size_t)(k - 1) * n + k] = a[(size_t)k * n + k - 1] = std::sqrt(0.5 * k);
    jacobi_eigen(n, a, lam, v);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int p, int q) { return lam[p] < lam[q]; });
    for (int i = 0; i < n; ++i) {
      x[i] = lam[order[i]];
      const double v0 = v[order[i]];  // row 0, column order[i]
      w[i] = v0 * v0;
    }
    // exact symmetry of the rule (the solver relies on x_{n-1-a} = -x_a)
    for (int i = 0; i < n / 2; ++i) {
      const double xs = 0.5 * (x[n - 1 - i] - x[i]), ws = 0.5 * (w[i] + w[n - 1 - i]);
      x[i] = -xs;
      x[n - 1 - i] = xs;
      w[i] = w[n - 1 - i] = ws;
    }
    (void)rpi;
    return true;
  }
  if (kind == 1) {
    if (!(vmax > 0.0)) {
      err = "Newton-Cotes velocity grid needs vmax > 0";
      return false;
    }
    const double step = 2.0 * vmax / (n - 1);
    for (int a = 0; a < n; ++a) {
      // symmetric construction: node a and node n-1-a are exact negatives
      x[a] = (a < n / 2) ? -(vmax - a * step) : (vmax - (n - 1 - a) * step);
      const double half = (a == 0 || a == n - 1) ? 0.5 : 1.0;
      w[a] = step * half * std::exp(-x[a] * x[a]) / rpi;
    }
    return true;
  }
  if (kind == 2) {
    // Eq. (nonuniform_v): v = 4 (s / (n-1))^3, s = -n+1, -n+3, ..., n-1; weights: trapezoid rule in
    // s (spacing 2) of g(v(s)) dv/ds, dv/ds = 12 s^2 / (n-1)^3.
    const double m = (double)(n - 1);
    for (int a = 0; a < n; ++a) {
      const double s = (double)(2 * a - (n - 1));
      const double r = s / m;
      x[a] = 4.0 * r * r * r;
      const double half = (a == 0 || a == n - 1) ? 0.5 : 1.0;
      w[a] = 2.0 * half * 12.0 * r * r / m * std::exp(-x[a] * x[a]) / rpi;
    }
    return true;
  }
  err = "unknown velocity grid kind";
  return false;
}

void build_geometry(const uint8_t *mask, int nx, int ny, bool px, bool py, bool plate_x, Geometry &G) {
  const int ncell = nx * ny;
  G.code4.assign((size_t)ncell * 4, 0u);
  G.hw_src.assign((size_t)ncell * 8, -1);
  G.n_gas = 0;
  auto solid = [&](int i, int j) -> bool {
    if (i < 0 || i >= nx) {
      if (!px) return true;
      i = ((i % nx) + nx) % nx;
    }
    if (j < 0 || j >= ny) {
      if (!py) return true;
      j = ((j % ny) + ny) % ny;
    }
    return mask[(size_t)j * nx + i] != 0;
  };
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) {
      const int cell = j * nx + i;
      if (mask[cell]) {
        for (int q = 0; q < 4; ++q) G.code4[(size_t)cell * 4 + q] = kSolid | (9u << kInvShift);
        continue;
      }
      ++G.n_gas;
      for (int q = 0; q < 4; ++q) {
        const int sx = (q & 1) ? -1 : 1, sy = (q & 2) ? -1 : 1;
        uint32_t code = 0;
        // x axis: upstream side is W for v1 > 0, E for v1 < 0
        {
          const int side = sx > 0 ? kW : kE;
          int cls = kFull, src = -1;
          if (solid(i - sx, j)) {
            cls = kWall;
            src = cell * 4 + side;
          } else if (solid(i - 2 * sx, j)) {
            cls = kNear;  // first order through the gas neighbour: no wall value
          }
          code |= (uint32_t)cls << kClsXShift;
          if (plate_x && !px && i == nx - 1 && sx < 0) code |= kTopWallX;
          G.hw_src[(size_t)cell * 8 + q * 2 + 0] = src;
          if (solid(i + sx, j)) code |= kIncX;
        }
        {
          const int side = sy > 0 ? kS : kN;
          int cls = kFull, src = -1;
          if (solid(i, j - sy)) {
            cls = kWall;
            src = cell * 4 + side;
          } else if (solid(i, j - 2 * sy)) {
            cls = kNear;
          }
          code |= (uint32_t)cls << kClsYShift;
          if (!plate_x && !py && j == ny - 1 && sy < 0) code |= kTopWall;
          G.hw_src[(size_t)cell * 8 + q * 2 + 1] = src;
          if (solid(i, j + sy)) code |= kIncY;
        }
        const uint32_t clx = (code >> kClsXShift) & 3u, cly = (code >> kClsYShift) & 3u;
        code |= (clx * 3u + cly) << kInvShift;
        // transposed stencil: which forward-downstream cells read this one, and with what weight
        {
          const uint32_t t1 = solid(i + sx, j) ? 0u : (solid(i - sx, j) ? 1u : 2u);
          const bool t2 = !solid(i + sx, j) && !solid(i + 2 * sx, j);
          code |= t1 << kAdjT1XShift;
          if (t2) code |= kAdjT2X;
        }
        {
          const uint32_t t1 = solid(i, j + sy) ? 0u : (solid(i, j - sy) ? 1u : 2u);
          const bool t2 = !solid(i, j + sy) && !solid(i, j + 2 * sy);
          code |= t1 << kAdjT1YShift;
          if (t2) code |= kAdjT2Y;
        }
        G.code4[(size_t)cell * 4 + q] = code;
      }
    }
  }
}

}  // namespace dvm
