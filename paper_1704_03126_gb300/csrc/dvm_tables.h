// dvm_tables.h -- host-side tables of libdvm (internal).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "dvm_device.cuh"

namespace dvm {

// 1D nodes (ascending, exactly antisymmetric) and weights approximating
// int g(x) exp(-x^2)/sqrt(pi) dx.  kind: 0 Gauss-Hermite, 1 trapezoid on [-vmax, vmax],
// 2 the cubic grid of Eq. (nonuniform_v).
bool quadrature_1d(int kind, int n, double vmax, std::vector<double> &x, std::vector<double> &w, std::string &err);

// Stencil classes and wall sources of every cell for the four quadrants.
struct Geometry {
  std::vector<uint32_t> code4;  // [ncell][4]
  std::vector<int> hw_src;      // [ncell][8]
  int n_gas = 0;
};
// plate_x: the moving plate (if any) lies beyond the last column instead of beyond the last row
void build_geometry(const uint8_t *mask, int nx, int ny, bool px, bool py, bool plate_x, Geometry &G);

}  // namespace dvm
