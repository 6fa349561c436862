// Launch parameters of the banded per-mode solve of algorithm (b) (banded.cu).
#pragma once
#include "common.cuh"

namespace hofem {

constexpr int kBandTab = (kMaxN + 1) * (kMaxN + 1);

struct BandParams {
  double* u;                  // (outer, M, inner): transformed RHS in, solution out (in place)
  double* scratch;            // outer x inner x (K + 2 ceil(K / 32)) doubles: Thomas multipliers
                              // per node and the chunk-boundary node contributions
  long long outer, inner;
  int K, n, M;
  double sA;                  // 4 h^-2 of the solve axis
  double alpha;
  const double* lamA;         // eigenvalues of the transformed axes by column c of inner:
  const double* lamB;         //   lamA[c / MB] + lamB[c % MB] (lamB may be null)
  long long MB;
  double A[kBandTab], C[kBandTab];   // local stiffness and mass, (n+1) x (n+1)
};

cudaError_t launch_banded(const BandParams& p, cudaStream_t s);

}  // namespace hofem
