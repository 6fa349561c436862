// Shared declarations of the hofem CUDA library (host + device).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/hofem.h"

namespace hofem {

constexpr int kMaxN = 16;       // largest element order
constexpr int kMaxK = 8192;     // largest elements per axis
constexpr int kMaxDims = 3;
// Orders whose element stiffness, scaled by the common denominator of its entries, is an
// integer matrix exactly representable in FP64; larger orders carry it as hi + lo.
constexpr int kExactStiffnessMaxN = 9;

// Host copy of one axis' eigen-data and twiddles (FP64), built at plan time.
struct AxisTables {
  int n = 0, K = 0, M = 0;
  double X = 0.0;
  std::vector<double> lam;    // M: 4 h^-2 lambda in spectral order
  std::vector<double> mix;    // (K-1) n n: [k-1][l][s], s = interior 0..n-2, n-1 = nodal
  std::vector<double> evec;   // (n-1)^2: [l][i]
  std::vector<double> tw;     // 2K complex: exp(-i pi t / K)
  // Even/odd folded local matrices (centro-symmetry R M R = M): for h = (n+1)/2 pairs
  // (t, n-t) and, for even n, the middle point, rows r < hr = n/2 + 1:
  //   E[r][t] = (M[r][t] + M[r][n-t]) / 2 (t < h),  E[r][mid] = M[r][mid],
  //   O[r][t] = (M[r][t] - M[r][n-t]) / 2 (r, t < h),
  // so (M w)_r = E_r + O_r and (M w)_{n-r} = E_r - O_r with the folded w.
  std::vector<double> Aloc, Cloc;        // (n+1)^2 local stiffness and mass, FP64
  std::vector<double> CfE, CfO;          // mass, FP64   (hr x hr, h x h)
  // Stiffness: for n <= 9 the integer matrix D A (exact; lo parts zero, a_scale = 1/D),
  // else A as double-double hi + lo (a_scale = 1).
  std::vector<double> AfE, AfO;
  std::vector<double> AfELo, AfOLo;
  double a_scale = 1.0;
};

hofem_status build_axis_tables(int n, int K, double X, AxisTables* out, std::string* err);

// Appends to tw (2K complex DST twiddles, interleaved re/im) the tables of the Bluestein
// form of the K-point DFT (outputs m < H = (K - 1) / 2 + 1) with convolution length NB (a
// power of two >= K - 1 + H) whose NB-point FFTs run the DIF passes of radices
// radix[0..npass): exp(-i pi t / NB) for t < 2 NB; the chirp c_j = exp(-i pi j^2 / K) for
// j < K; the DFT of the filter b_d = conj(c_|d|) (lags -(K-1) <= d < H, indices mod NB),
// divided by NB, at the passes' output slots.
void bluestein_tables(int K, int NB, int npass, const int* radix, std::vector<double>* tw);

// (n+1)-point Gauss-Legendre nodes xi (ascending) and T[a (n+1) + g] = w_g e_a(xi_g).
void element_load_table(int n, std::vector<double>* T, std::vector<double>* xi);
// B[g][a] = e_a(xi_g), D[g][a] = e_a'(xi_g) and the weights w_g of that rule.
void element_basis_tables(int n, std::vector<double>* B, std::vector<double>* D, std::vector<double>* w);

}  // namespace hofem
