// Shared declarations of the hofem CUDA library (host + device).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hofem.h"

namespace hofem {

constexpr int kMaxN = 16;       // largest element order
constexpr int kMaxK = 8192;     // largest elements per axis (power of two)
constexpr int kMaxDims = 3;

// Host copy of one axis' eigen-data and twiddles (FP64), built at plan time.
struct AxisTables {
  int n = 0, K = 0, M = 0;
  double X = 0.0;
  std::vector<double> lam;    // M: 4 h^-2 lambda in spectral order
  std::vector<double> mix;    // (K-1) n n: [k-1][l][s], s = interior 0..n-2, n-1 = nodal
  std::vector<double> evec;   // (n-1)^2: [l][i]
  std::vector<double> tw;     // 2K complex: exp(-i pi t / K)
  std::vector<double> Aloc;   // (n+1)^2 local stiffness, FP64 (high part)
  std::vector<double> AlocLo; // (n+1)^2 remainder A - Aloc (double-double low part)
  std::vector<double> Cloc;   // (n+1)^2 local mass, FP64
};

hofem_status build_axis_tables(int n, int K, double X, AxisTables* out, std::string* err);

}  // namespace hofem
