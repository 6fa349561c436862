// Plan-time 1D eigen-data of the scaled FEM pencil A v = lambda C v (Eq. eig_glob).
//
// Host (double-double): local matrices A, C of the equispaced order-n Lagrange element
// on [-1, 1] (Sect. 2 par. 1) by (n+1)-point Gauss-Legendre quadrature, exact for the
// polynomial integrands; twiddles exp(-i pi t / N); eta_k = 1 - cos(pi k/K) and
// zeta_k = 1 + cos(pi k/K) from sin^2 series so that neither loses digits.
//
// Device (double-double, one thread per frequency k): for k >= 1 the eigenpairs of
// the n x n symmetric-definite pencil (A_k, C_k), A_k = lead_n(A + theta_k A R),
// C_k = lead_n(C + theta_k C R) (R = reversal of R^{n+1}).  Substituting the ansatz of
// Theorem 1 part 3 -- nodal values c sin(pi k j/K), interior q sin(pi k (j-1)/K) +
// P q sin(pi k j/K) -- into the rows of Eq. eig_glob gives exactly these n equations
// (the interior rows give G~ q = -g c as in Theorem 1, the node rows the theta-equation,
// Eq. theta), so their eigenvalues are lambda_k^(l) and u = (c, q) builds s_k^(l).
// With u^T C_k u = 1 the C-norm of s_k^(l) is K (it equals K u^T (C + theta C R) u).
// For k = 0 the element pencil (A~, C~) of Lemma 1 gives lambda_0^(l), e^(l) with
// C~ e . e = 1 (Theorem 1 part 2), norm K.  Both are solved by Cholesky of the mass
// matrix and cyclic Jacobi on L^{-1} A L^{-T}, all in double-double.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dd.cuh"

namespace hofem {

// ----------------------------------------------------------------- host: series
static const dd DD_PI = {3.141592653589793116, 1.2246467991473532072e-16};

static dd dd_from_int_ratio(long long a, long long b) { return dd_make((double)a) / dd_make((double)b); }

// sin and cos of x in [0, pi/2] by Taylor series in double-double.
static void dd_sincos_small(dd x, dd* s, dd* c) {
  dd x2 = x * x;
  dd term = x, sum = x;
  for (int k = 1; k < 40; ++k) {
    term = (-term * x2) / dd_make((double)((2 * k) * (2 * k + 1)));
    sum = sum + term;
    if (fabs(term.hi) < 1e-40) break;
  }
  *s = sum;
  term = dd_make(1.0);
  sum = dd_make(1.0);
  for (int k = 1; k < 40; ++k) {
    term = (-term * x2) / dd_make((double)((2 * k - 1) * (2 * k)));
    sum = sum + term;
    if (fabs(term.hi) < 1e-40) break;
  }
  *c = sum;
}

// cos and sin of pi t / N for integer t in [0, 2N).
static void dd_sincos_pi_frac(long long t, long long N, dd* s, dd* c) {
  t %= 2 * N;
  if (t < 0) t += 2 * N;
  bool neg = false;
  if (t >= N) { t -= N; neg = true; }            // angle + pi
  bool refl = false;
  if (2 * t > N) { t = N - t; refl = true; }      // pi - angle
  dd x = DD_PI * dd_from_int_ratio(t, N);
  dd ss, cc;
  dd_sincos_small(x, &ss, &cc);
  if (refl) cc = -cc;
  if (neg) { ss = -ss; cc = -cc; }
  *s = ss;
  *c = cc;
}

// ----------------------------------------------------------------- host: element
// Legendre P_G and P_G' at x (three-term recurrence), double-double.
static void legendre(int G, dd x, dd* p, dd* dp) {
  dd p0 = dd_make(1.0), p1 = x;
  if (G == 0) { *p = p0; *dp = dd_make(0.0); return; }
  for (int k = 1; k < G; ++k) {
    dd p2 = (dd_make((double)(2 * k + 1)) * x * p1 - dd_make((double)k) * p0) / dd_make((double)(k + 1));
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = dd_make((double)G) * (x * p1 - p0) / (x * x - dd_make(1.0));
}

static void gauss_legendre(int G, std::vector<dd>& xs, std::vector<dd>& ws) {
  xs.resize(G);
  ws.resize(G);
  for (int i = 0; i < G; ++i) {
    double x = cos(M_PI * (i + 0.75) / (G + 0.5));
    for (int it = 0; it < 100; ++it) {   // FP64 Newton
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < G; ++k) {
        double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      double dp = G * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    dd X = dd_make(x);
    for (int it = 0; it < 3; ++it) {     // double-double Newton
      dd p, dp;
      legendre(G, X, &p, &dp);
      X = X - p / dp;
    }
    dd p, dp;
    legendre(G, X, &p, &dp);
    xs[i] = X;
    ws[i] = dd_make(2.0) / ((dd_make(1.0) - X * X) * dp * dp);
  }
}

// Load-vector quadrature of Sect. 2 par. 5: the (n+1) Gauss-Legendre points xi_g on
// [-1, 1] (ascending) and T[a (n+1) + g] = w_g e_a(xi_g), rounded once from double-double.
void element_load_table(int n, std::vector<double>* T, std::vector<double>* xi) {
  const int m = n + 1, G = n + 1;
  std::vector<dd> xs, ws;
  gauss_legendre(G, xs, ws);
  std::vector<dd> t(m);
  for (int k = 0; k < m; ++k) t[k] = dd_make(-1.0) + dd_from_int_ratio(2 * k, n);
  T->assign(m * G, 0.0);
  xi->assign(G, 0.0);
  // gauss_legendre returns the nodes in descending order (cos of increasing angles)
  for (int g = 0; g < G; ++g) {
    const int gs = G - 1 - g;
    (*xi)[g] = dd_to_double(xs[gs]);
    for (int a = 0; a < m; ++a) {
      dd v = dd_make(1.0);
      for (int q = 0; q < m; ++q)
        if (q != a) v = v * (xs[gs] - t[q]) / (t[a] - t[q]);
      (*T)[a * G + g] = dd_to_double(ws[gs] * v);
    }
  }
}

// Basis and derivative values at the (n+1) Gauss-Legendre points (ascending) and the
// weights: B[g (n+1) + a] = e_a(xi_g), D[g (n+1) + a] = e_a'(xi_g), rounded from double-double.
void element_basis_tables(int n, std::vector<double>* B, std::vector<double>* D, std::vector<double>* w) {
  const int m = n + 1, G = n + 1;
  std::vector<dd> xs, ws;
  gauss_legendre(G, xs, ws);
  std::vector<dd> t(m);
  for (int k = 0; k < m; ++k) t[k] = dd_make(-1.0) + dd_from_int_ratio(2 * k, n);
  B->assign(G * m, 0.0);
  D->assign(G * m, 0.0);
  w->assign(G, 0.0);
  for (int g = 0; g < G; ++g) {
    const int gs = G - 1 - g;                    // gauss_legendre returns descending nodes
    (*w)[g] = dd_to_double(ws[gs]);
    for (int a = 0; a < m; ++a) {
      dd v = dd_make(1.0), d = dd_make(0.0);
      for (int q = 0; q < m; ++q)
        if (q != a) v = v * (xs[gs] - t[q]) / (t[a] - t[q]);
      for (int q = 0; q < m; ++q) {
        if (q == a) continue;
        dd term = dd_make(1.0) / (t[a] - t[q]);
        for (int r = 0; r < m; ++r)
          if (r != a && r != q) term = term * (xs[gs] - t[r]) / (t[a] - t[r]);
        d = d + term;
      }
      (*B)[g * m + a] = dd_to_double(v);
      (*D)[g * m + a] = dd_to_double(d);
    }
  }
}

// A_ab = int e'_a e'_b, C_ab = int e_a e_b on [-1, 1], equispaced Lagrange basis.
void element_matrices_dd(int n, std::vector<dd>& A, std::vector<dd>& C) {
  const int m = n + 1, G = n + 1;
  std::vector<dd> xs, ws;
  gauss_legendre(G, xs, ws);
  std::vector<dd> t(m);
  for (int k = 0; k < m; ++k) t[k] = dd_make(-1.0) + dd_from_int_ratio(2 * k, n);
  std::vector<dd> val(G * m), der(G * m);
  for (int g = 0; g < G; ++g) {
    for (int l = 0; l < m; ++l) {
      dd v = dd_make(1.0);
      for (int q = 0; q < m; ++q)
        if (q != l) v = v * (xs[g] - t[q]) / (t[l] - t[q]);
      dd d = dd_make(0.0);
      for (int q = 0; q < m; ++q) {
        if (q == l) continue;
        dd term = dd_make(1.0) / (t[l] - t[q]);
        for (int r = 0; r < m; ++r)
          if (r != l && r != q) term = term * (xs[g] - t[r]) / (t[l] - t[r]);
        d = d + term;
      }
      val[g * m + l] = v;
      der[g * m + l] = d;
    }
  }
  A.assign(m * m, dd_make(0.0));
  C.assign(m * m, dd_make(0.0));
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      dd sa = dd_make(0.0), sc = dd_make(0.0);
      for (int g = 0; g < G; ++g) {
        sa = sa + ws[g] * der[g * m + a] * der[g * m + b];
        sc = sc + ws[g] * val[g * m + a] * val[g * m + b];
      }
      A[a * m + b] = sa;
      C[a * m + b] = sc;
    }
  // exact symmetries (R A R = A, A = A^T) -- average out the last-bit asymmetry
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      dd s = (A[a * m + b] + A[b * m + a] + A[(n - a) * m + (n - b)] + A[(n - b) * m + (n - a)]) * 0.25;
      dd c = (C[a * m + b] + C[b * m + a] + C[(n - a) * m + (n - b)] + C[(n - b) * m + (n - a)]) * 0.25;
      A[a * m + b] = s;
      C[a * m + b] = c;
    }
}

// Integer form of the element stiffness.  On [-1, 1], A_ab = (n/2) int_0^n N_a' N_b' dx /
// (d_a d_b) with the node polynomials N_a(x) = prod_{c != a} (x - c) (integer coefficients,
// nodes 0..n) and d_a = prod_{c != a} (a - c), |d_a| = a! (n-a)! a divisor of n!; the
// integral of x^k over [0, n] is n^{k+1}/(k+1) with k <= 2n-2.  So D0 = 2 (n!)^2
// lcm(1..2n-1) clears every denominator, and D = D0 / gcd(D0, all D0 A_ab) is the least
// common one.  D0 A_ab is rounded from the double-double entries (their error is far
// below 1/2 for n <= 9).  Returns false unless every D A_ab is below 2^52 in magnitude
// and every row of D A sums to zero exactly (A annihilates constants).
static bool stiffness_integers(int n, const std::vector<dd>& A, std::vector<double>* S, double* inv_D) {
  if (n < 1 || n > kExactStiffnessMaxN) return false;
  typedef __int128 i128;
  auto gcd = [](i128 a, i128 b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b != 0) {
      const i128 t = a % b;
      a = b;
      b = t;
    }
    return a;
  };
  i128 fact = 1, L = 1;
  for (int i = 2; i <= n; ++i) fact *= i;
  for (int i = 2; i <= 2 * n - 1; ++i) L = L / gcd(L, i) * i;
  const i128 D0 = 2 * fact * fact * L;
  const double d_hi = (double)D0;
  const dd Dd = fast_two_sum(d_hi, (double)(D0 - (i128)d_hi));
  const int m1 = n + 1;
  std::vector<i128> Z(m1 * m1);
  i128 g = D0;
  for (int i = 0; i < m1 * m1; ++i) {
    const dd z = A[i] * Dd;
    const double a = nearbyint(z.hi);
    const double rem = (z.hi - a) + z.lo;
    const double b = nearbyint(rem);
    if (fabs(rem - b) > 1e-6) return false;
    Z[i] = (i128)a + (i128)b;
    g = gcd(g, Z[i]);
  }
  const i128 D = D0 / g;
  const i128 lim = (i128)1 << 52;
  if (D >= lim) return false;
  S->assign(m1 * m1, 0.0);
  for (int r = 0; r < m1; ++r) {
    i128 row = 0;
    for (int c = 0; c < m1; ++c) {
      const i128 v = Z[r * m1 + c] / g;
      if (v >= lim || -v >= lim) return false;
      row += v;
      (*S)[r * m1 + c] = (double)v;
    }
    if (row != 0) return false;
  }
  *inv_D = 1.0 / (double)D;
  return true;
}

// ----------------------------------------------------------------- device: eigen
struct EigInput {
  int n, K;
  const dd* base;      // 6 n x n blocks: lead(A+AR), lead(A-AR), lead(AR), same for C
  const dd* elemA;     // (n-1)^2 interior block of A
  const dd* elemC;
  const dd* coef;      // per k: eta_k (k <= K/2) or zeta_k (k > K/2)
  dd scale;            // 4 K^2 / X^2
  double* lam;         // M
  double* mix;         // (K-1) n n
  double* evec;        // (n-1)^2
  int* status;         // 0 ok, else 1 + k of the first failure
};

__global__ void eig_kernel(EigInput in) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= in.K) return;
  const int n = in.n;
  const int m = (k == 0) ? n - 1 : n;
  if (m <= 0) return;
  dd Am[kMaxN][kMaxN], Cm[kMaxN][kMaxN], V[kMaxN][kMaxN];
  if (k == 0) {
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        Am[a][b] = in.elemA[a * m + b];
        Cm[a][b] = in.elemC[a * m + b];
      }
  } else {
    const bool low = 2 * k <= in.K;   // theta >= 0: (M + MR) - eta MR, else (M - MR) + zeta MR
    const dd cf = in.coef[k];
    const int nn = n * n;
    const dd* PA = in.base + (low ? 0 : 1) * nn;
    const dd* RA = in.base + 2 * nn;
    const dd* PC = in.base + (low ? 3 : 4) * nn;
    const dd* RC = in.base + 5 * nn;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        dd ra = cf * RA[a * n + b], rc = cf * RC[a * n + b];
        Am[a][b] = low ? PA[a * n + b] - ra : PA[a * n + b] + ra;
        Cm[a][b] = low ? PC[a * n + b] - rc : PC[a * n + b] + rc;
      }
  }
  // Cholesky C = L L^T (L stored in the lower triangle of Cm)
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      dd s = Cm[i][j];
      for (int q = 0; q < j; ++q) s = s - Cm[i][q] * Cm[j][q];
      if (i == j) {
        if (!(s.hi > 0.0)) { atomicCAS(in.status, 0, 1 + k); return; }
        Cm[i][i] = dd_sqrt(s);
      } else {
        Cm[i][j] = s / Cm[j][j];
      }
    }
  }
  // B = L^{-1} A L^{-T}: first Y = L^{-1} A (in V), then B = L^{-1} Y^T (in Am)
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      dd s = Am[i][c];
      for (int q = 0; q < i; ++q) s = s - Cm[i][q] * V[q][c];
      V[i][c] = s / Cm[i][i];
    }
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      dd s = V[c][i];
      for (int q = 0; q < i; ++q) s = s - Cm[i][q] * Am[q][c];
      Am[i][c] = s / Cm[i][i];
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) {
      dd s = (Am[i][j] + Am[j][i]) * 0.5;
      Am[i][j] = s;
      Am[j][i] = s;
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) V[i][j] = dd_make(i == j ? 1.0 : 0.0);
  // cyclic Jacobi
  bool done = false;
  for (int sweep = 0; sweep < 60 && !done; ++sweep) {
    done = true;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        dd apq = Am[p][q];
        double thr = 1e-33 * sqrt(fabs(Am[p][p].hi * Am[q][q].hi));
        if (fabs(apq.hi) <= thr) continue;
        done = false;
        dd th = (Am[q][q] - Am[p][p]) / (apq * 2.0);
        dd t = dd_make(1.0) / (dd_abs(th) + dd_sqrt(th * th + dd_make(1.0)));
        if (th.hi < 0.0) t = -t;
        dd c = dd_make(1.0) / dd_sqrt(t * t + dd_make(1.0));
        dd s = t * c;
        for (int r = 0; r < m; ++r) {
          dd arp = Am[r][p], arq = Am[r][q];
          Am[r][p] = c * arp - s * arq;
          Am[r][q] = s * arp + c * arq;
        }
        for (int r = 0; r < m; ++r) {
          dd apr = Am[p][r], aqr = Am[q][r];
          Am[p][r] = c * apr - s * aqr;
          Am[q][r] = s * apr + c * aqr;
        }
        Am[p][q] = dd_make(0.0);
        Am[q][p] = dd_make(0.0);
        for (int r = 0; r < m; ++r) {
          dd vrp = V[r][p], vrq = V[r][q];
          V[r][p] = c * vrp - s * vrq;
          V[r][q] = s * vrp + c * vrq;
        }
      }
  }
  if (!done) { atomicCAS(in.status, 0, 1 + k); return; }
  // eigenvectors u = L^{-T} v (overwrite V column by column)
  for (int c = 0; c < m; ++c)
    for (int i = m - 1; i >= 0; --i) {
      dd s = V[i][c];
      for (int q = i + 1; q < m; ++q) s = s - Cm[q][i] * V[q][c];
      V[i][c] = s / Cm[i][i];
    }
  // ascending order
  int ord[kMaxN];
  for (int i = 0; i < m; ++i) ord[i] = i;
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (Am[ord[j]][ord[j]] < Am[ord[i]][ord[i]]) { int tmp = ord[i]; ord[i] = ord[j]; ord[j] = tmp; }
  for (int l = 0; l < m; ++l) {
    const int c = ord[l];
    double sgn = 1.0;
    if (k > 0) {
      sgn = V[0][c].hi < 0.0 ? -1.0 : 1.0;
    } else {
      double mx = 0.0;
      for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(V[i][c].hi));
      for (int i = 0; i < m; ++i)
        if (fabs(V[i][c].hi) >= 1e-3 * mx) { sgn = V[i][c].hi < 0.0 ? -1.0 : 1.0; break; }
    }
    dd lam = Am[c][c] * in.scale;
    if (k > 0) {
      in.lam[(size_t)(k - 1) * n + l] = dd_to_double(lam);
      double* row = in.mix + ((size_t)(k - 1) * n + l) * n;
      for (int s = 0; s < n - 1; ++s) row[s] = sgn * dd_to_double(V[s + 1][c]);
      row[n - 1] = sgn * dd_to_double(V[0][c]);
    } else {
      in.lam[(size_t)(in.K - 1) * n + l] = dd_to_double(lam);
      for (int i = 0; i < m; ++i) in.evec[l * m + i] = sgn * dd_to_double(V[i][c]);
    }
  }
}

// ----------------------------------------------------------------- host driver
hofem_status build_axis_tables(int n, int K, double X, AxisTables* out, std::string* err) {
  const int M = n * K - 1;
  std::vector<dd> A, C;
  element_matrices_dd(n, A, C);
  const int m1 = n + 1;
  std::vector<dd> base(6 * n * n);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      dd ar = A[a * m1 + (n - b)], cr = C[a * m1 + (n - b)];
      base[0 * n * n + a * n + b] = A[a * m1 + b] + ar;
      base[1 * n * n + a * n + b] = A[a * m1 + b] - ar;
      base[2 * n * n + a * n + b] = ar;
      base[3 * n * n + a * n + b] = C[a * m1 + b] + cr;
      base[4 * n * n + a * n + b] = C[a * m1 + b] - cr;
      base[5 * n * n + a * n + b] = cr;
    }
  const int mi = n - 1;
  std::vector<dd> eA(std::max(mi * mi, 1)), eC(std::max(mi * mi, 1));
  for (int a = 0; a < mi; ++a)
    for (int b = 0; b < mi; ++b) {
      eA[a * mi + b] = A[(a + 1) * m1 + (b + 1)];
      eC[a * mi + b] = C[(a + 1) * m1 + (b + 1)];
    }
  std::vector<dd> coef(K);
  for (int k = 0; k < K; ++k) {
    // eta = 1 - cos(pi k/K) = 2 sin^2(pi k/(2K)); zeta = 1 + cos = 2 sin^2(pi (K-k)/(2K))
    long long t = (2 * k <= K) ? k : (K - k);
    dd s, c;
    dd_sincos_pi_frac(t, 2LL * K, &s, &c);
    coef[k] = s * s * 2.0;
  }
  dd Xd = dd_make(X);
  dd scale = dd_make(4.0) * dd_make((double)K) * dd_make((double)K) / (Xd * Xd);

  std::vector<double> lam(M), mix((size_t)(K - 1) * n * n), evec(std::max(mi * mi, 1));
  dd *d_base = nullptr, *d_eA = nullptr, *d_eC = nullptr, *d_coef = nullptr;
  double *d_lam = nullptr, *d_mix = nullptr, *d_evec = nullptr;
  int* d_status = nullptr;
  int h_status = 0;
  hofem_status st = HOFEM_OK;
#define PC_CHECK(x)                                                          \
  do {                                                                       \
    cudaError_t e_ = (x);                                                    \
    if (e_ != cudaSuccess) {                                                 \
      *err = std::string("precompute: ") + cudaGetErrorString(e_);           \
      st = (e_ == cudaErrorMemoryAllocation) ? HOFEM_ERR_OOM : HOFEM_ERR_CUDA; \
      goto cleanup;                                                          \
    }                                                                        \
  } while (0)
  PC_CHECK(cudaMalloc(&d_base, base.size() * sizeof(dd)));
  PC_CHECK(cudaMalloc(&d_eA, eA.size() * sizeof(dd)));
  PC_CHECK(cudaMalloc(&d_eC, eC.size() * sizeof(dd)));
  PC_CHECK(cudaMalloc(&d_coef, coef.size() * sizeof(dd)));
  PC_CHECK(cudaMalloc(&d_lam, lam.size() * sizeof(double)));
  PC_CHECK(cudaMalloc(&d_mix, mix.size() * sizeof(double)));
  PC_CHECK(cudaMalloc(&d_evec, evec.size() * sizeof(double)));
  PC_CHECK(cudaMalloc(&d_status, sizeof(int)));
  PC_CHECK(cudaMemcpy(d_base, base.data(), base.size() * sizeof(dd), cudaMemcpyHostToDevice));
  PC_CHECK(cudaMemcpy(d_eA, eA.data(), eA.size() * sizeof(dd), cudaMemcpyHostToDevice));
  PC_CHECK(cudaMemcpy(d_eC, eC.data(), eC.size() * sizeof(dd), cudaMemcpyHostToDevice));
  PC_CHECK(cudaMemcpy(d_coef, coef.data(), coef.size() * sizeof(dd), cudaMemcpyHostToDevice));
  PC_CHECK(cudaMemset(d_status, 0, sizeof(int)));
  {
    EigInput in{n, K, d_base, d_eA, d_eC, d_coef, scale, d_lam, d_mix, d_evec, d_status};
    const int threads = 32;
    eig_kernel<<<(K + threads - 1) / threads, threads>>>(in);
    PC_CHECK(cudaGetLastError());
  }
  PC_CHECK(cudaMemcpy(&h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_status != 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "precompute: eigen-solve failed at k = %d", h_status - 1);
    *err = buf;
    st = HOFEM_ERR_CUDA;
    goto cleanup;
  }
  PC_CHECK(cudaMemcpy(lam.data(), d_lam, lam.size() * sizeof(double), cudaMemcpyDeviceToHost));
  PC_CHECK(cudaMemcpy(mix.data(), d_mix, mix.size() * sizeof(double), cudaMemcpyDeviceToHost));
  PC_CHECK(cudaMemcpy(evec.data(), d_evec, evec.size() * sizeof(double), cudaMemcpyDeviceToHost));
  out->n = n;
  out->K = K;
  out->M = M;
  out->X = X;
  out->lam = lam;
  out->mix = mix;
  out->evec = evec;
  // twiddles exp(-i pi t / K), t = 0 .. 2K-1 (the 2K-th roots used by the DST)
  out->tw.resize(2 * (size_t)K * 2);
  for (int t = 0; t < 2 * K; ++t) {
    dd s, c;
    dd_sincos_pi_frac(t, K, &s, &c);
    out->tw[2 * t] = dd_to_double(c);
    out->tw[2 * t + 1] = -dd_to_double(s);
  }
  // folded element matrices for the matrix-free operator
  {
    const int h = (n + 1) / 2, hr = n / 2 + 1;
    const bool mid = (n % 2) == 0;
    std::vector<double> S;
    double inv_D = 1.0;
    const bool exact = stiffness_integers(n, A, &S, &inv_D);
    if (n <= kExactStiffnessMaxN && !exact) {
      if (err) *err = "element stiffness is not an exact FP64 integer matrix after scaling";
      st = HOFEM_ERR_UNSUPPORTED;
      goto cleanup;
    }
    out->a_scale = exact ? inv_D : 1.0;
    // full local matrices rounded to FP64 (the banded solve of algorithm (b))
    out->Aloc.resize(m1 * m1);
    out->Cloc.resize(m1 * m1);
    for (int i = 0; i < m1 * m1; ++i) {
      out->Aloc[i] = dd_to_double(A[i]);
      out->Cloc[i] = dd_to_double(C[i]);
    }
    out->CfE.assign(hr * hr, 0.0);
    out->AfE.assign(hr * hr, 0.0);
    out->AfELo.assign(hr * hr, 0.0);
    out->CfO.assign(h * h, 0.0);
    out->AfO.assign(h * h, 0.0);
    out->AfOLo.assign(h * h, 0.0);
    // stiffness entry (r, t) of the folded tables as hi + lo (lo = 0 when exact)
    auto fold = [&](int r, int t, double sign, double w, double* hi, double* lo) {
      if (exact) {
        *hi = (S[r * m1 + t] + sign * S[r * m1 + (n - t)]) * w;   // integers < 2^52: exact
        *lo = 0.0;
      } else {
        const dd a = (A[r * m1 + t] + A[r * m1 + (n - t)] * sign) * w;
        const dd v = fast_two_sum(a.hi, a.lo);
        *hi = v.hi;
        *lo = v.lo;
      }
    };
    for (int r = 0; r < hr; ++r) {
      for (int t = 0; t < h; ++t) {
        out->CfE[r * hr + t] = dd_to_double((C[r * m1 + t] + C[r * m1 + (n - t)]) * 0.5);
        fold(r, t, 1.0, 0.5, &out->AfE[r * hr + t], &out->AfELo[r * hr + t]);
        if (r < h) {
          out->CfO[r * h + t] = dd_to_double((C[r * m1 + t] - C[r * m1 + (n - t)]) * 0.5);
          fold(r, t, -1.0, 0.5, &out->AfO[r * h + t], &out->AfOLo[r * h + t]);
        }
      }
      if (mid) {
        const int t = n / 2;
        out->CfE[r * hr + t] = dd_to_double(C[r * m1 + t]);
        if (exact) {
          out->AfE[r * hr + t] = S[r * m1 + t];
        } else {
          const dd v = fast_two_sum(A[r * m1 + t].hi, A[r * m1 + t].lo);
          out->AfE[r * hr + t] = v.hi;
          out->AfELo[r * hr + t] = v.lo;
        }
      }
    }
  }
cleanup:
  cudaFree(d_base);
  cudaFree(d_eA);
  cudaFree(d_eC);
  cudaFree(d_coef);
  cudaFree(d_lam);
  cudaFree(d_mix);
  cudaFree(d_evec);
  cudaFree(d_status);
#undef PC_CHECK
  return st;
}

void bluestein_tables(int K, int NB, int npass, const int* radix, std::vector<double>* tw) {
  using cd = std::complex<double>;
  std::vector<double> wB(4 * (size_t)NB);
  for (int t = 0; t < 2 * NB; ++t) {
    dd sn, cs;
    dd_sincos_pi_frac(t, NB, &sn, &cs);
    wB[2 * t] = dd_to_double(cs);
    wB[2 * t + 1] = -dd_to_double(sn);
  }
  // chirp: j^2 reduced mod 2K indexes the 2K-th roots already in tw
  std::vector<double> ch(2 * (size_t)K);
  std::vector<cd> b(NB, cd(0.0, 0.0));
  for (int j = 0; j < K; ++j) {
    const long long r = ((long long)j * j) % (2LL * K);
    ch[2 * j] = (*tw)[2 * r];
    ch[2 * j + 1] = (*tw)[2 * r + 1];
    const cd cc(ch[2 * j], -ch[2 * j + 1]);
    if (j <= (K - 1) / 2) b[j] = cc;           // lags 0 .. H-1 (the outputs used)
    if (j > 0) b[NB - j] = cc;                  // lags -(K-1) .. -1
  }
  // B = DFT_NB(b): radix-2, natural order (bit-reversal permutation, then butterflies)
  int lg = 0;
  while ((1 << lg) < NB) ++lg;
  for (int i = 0; i < NB; ++i) {
    int r = 0;
    for (int k = 0; k < lg; ++k) r |= ((i >> k) & 1) << (lg - 1 - k);
    if (r > i) std::swap(b[i], b[r]);
  }
  for (int len = 2; len <= NB; len <<= 1) {
    const int step = 2 * NB / len;            // exp(-2 pi i j / len) = wB[j step]
    for (int s0 = 0; s0 < NB; s0 += len)
      for (int j = 0; j < len / 2; ++j) {
        const cd w(wB[2 * (size_t)j * step], wB[2 * (size_t)j * step + 1]);
        const cd u = b[s0 + j], v = b[s0 + j + len / 2] * w;
        b[s0 + j] = u + v;
        b[s0 + j + len / 2] = u - v;
      }
  }
  // output slot of frequency k after the DIF passes: the low digit of k selects the top
  // digit of the slot
  std::vector<double> filt(2 * (size_t)NB);
  for (int k = 0; k < NB; ++k) {
    int slot = 0, sh = lg, m = k;
    for (int ps = 0; ps < npass; ++ps) {
      int lb = 0;
      while ((1 << lb) < radix[ps]) ++lb;
      sh -= lb;
      slot |= (m & (radix[ps] - 1)) << sh;
      m >>= lb;
    }
    filt[2 * slot] = b[k].real() / NB;
    filt[2 * slot + 1] = b[k].imag() / NB;
  }
  tw->insert(tw->end(), wB.begin(), wB.end());
  tw->insert(tw->end(), ch.begin(), ch.end());
  tw->insert(tw->end(), filt.begin(), filt.end());
}

}  // namespace hofem
