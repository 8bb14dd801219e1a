// coeffs.cpp -- host-side coefficient generation for libcfs (long double arithmetic).
//
// Everything here is derived from the defining conditions of arXiv 2506.03027, not from the
// printed polynomials:
//   * LSERK stage polynomials P_e(z) of Eq. 3 and nu_j^e of Eq. 10 (Table 4 coefficients).
//   * Stage-0 extrapolation weights c(k): the Taylor constraints of Eq. 6 restricted to time
//     (exact for polynomials of degree C-1 in t), Eq. 14-15.
//   * Buffer temporal-derivative weights d^(e)(k): the constraint system of Eq. 13.
//   * Collapsed halo weights W^(m)(k): the buffer recursion of Eq. 8 is linear in the delayed
//     levels and free of dt, so U_buf^(m) = sum_l W^(m)_l(k) U^{n-k-l}.
//   * Tenth-order Pade filter right-side coefficients: T(w) = 1 + O(w^10) and T(pi) = 0.
#include "cfs_internal.h"

#include <cmath>
#include <cstring>

namespace cfs {

typedef long double ld;

// Gaussian elimination with partial pivoting, n <= 8.  A is row-major n x n, b overwritten by x.
static bool solve_small(int n, ld* A, ld* b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0L) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { ld t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
      ld t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      ld f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    ld s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
    b[r] = s / A[r * n + r];
  }
  return true;
}

int lserk_coeffs(int order, double* A, double* B) {
  if (order == 4) {
    // Table 4 (Carpenter & Kennedy five-stage fourth-order, 8 printed digits)
    static const double a[5] = {0.0, -0.4812317, -1.0495626, -1.6025296, -1.7782672};
    static const double b[5] = {0.09761835, 0.41225329, 0.44021696, 1.42631146, 0.19787605};
    std::memcpy(A, a, sizeof(a));
    std::memcpy(B, b, sizeof(b));
    return 5;
  }
  if (order == 2) {  // App. B: A = {0, -1/2}, B = {1/2, 1}
    A[0] = 0.0; A[1] = -0.5;
    B[0] = 0.5; B[1] = 1.0;
    return 2;
  }
  return 0;
}

// Coefficients of the stage polynomial P_e(z) (y' = z y, y^(0) = 1) after e stages.
static void stage_poly(int order, int e, ld* P /* [8] */) {
  double A[5], B[5];
  lserk_coeffs(order, A, B);
  ld Pc[8] = {1.0L, 0, 0, 0, 0, 0, 0, 0}, Qc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = 0; m < e; ++m) {
    ld Qn[8];
    for (int j = 0; j < 8; ++j) Qn[j] = (ld)A[m] * Qc[j] + (j > 0 ? Pc[j - 1] : 0.0L);
    for (int j = 0; j < 8; ++j) { Qc[j] = Qn[j]; Pc[j] += (ld)B[m] * Qc[j]; }
  }
  std::memcpy(P, Pc, sizeof(Pc));
}

static ld factorial(int n) {
  ld f = 1.0L;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Taylor row of level t = -(k + l) (in units of dt): (-(k+l))^theta / theta!
static void taylor_matrix(int C, int k, ld* M) {
  for (int th = 0; th < C; ++th)
    for (int l = 0; l < C; ++l) M[th * C + l] = powl(-(ld)(k + l), th) / factorial(th);
}

bool extrap_weights(int order, int k, ld* c) {
  const int C = order == 4 ? 5 : 3;
  ld M[64];
  taylor_matrix(C, k, M);
  for (int th = 0; th < C; ++th) c[th] = (th == 0) ? 1.0L : 0.0L;
  if (!solve_small(C, M, c)) return false;
  // the exact weights are rationals with denominators dividing 24: snap elimination residue
  // (|w| ~ 1e-19) to zero so that c(0) is exactly the unit vector
  for (int l = 0; l < C; ++l)
    if (fabsl(c[l]) < 1e-12L) c[l] = 0.0L;
  return true;
}

bool buffer_dudt_weights(int order, int e, int k, ld* d) {
  const int C = order == 4 ? 5 : 3;
  ld P[8];
  stage_poly(order, e, P);
  ld M[64];
  taylor_matrix(C, k, M);
  // theta = 0: sum d = 0; theta = j+1 (j = 0..e): nu_j^e; remaining theta up to q/r = C-1: 0
  for (int th = 0; th < C; ++th) d[th] = (th >= 1 && th <= e + 1) ? P[th - 1] : 0.0L;
  return solve_small(C, M, d);
}

int at_weight_table(int order, int kmax, double* W) {
  if ((order != 2 && order != 4) || kmax < 0 || kmax > CFS_MAX_DELAY) return -1;
  const int C = order == 4 ? 5 : 3;
  double A[5], B[5];
  const int s = lserk_coeffs(order, A, B);
  for (int k = 0; k <= kmax; ++k) {
    ld w[5], v[5] = {0, 0, 0, 0, 0};
    if (!extrap_weights(order, k, w)) return -1;
    for (int l = 0; l < C; ++l) W[(k * s + 0) * C + l] = (double)w[l];
    for (int m = 1; m < s; ++m) {
      ld d[5];
      if (!buffer_dudt_weights(order, m - 1, k, d)) return -1;
      for (int l = 0; l < C; ++l) {
        v[l] = (ld)A[m - 1] * v[l] + d[l];
        w[l] += (ld)B[m - 1] * v[l];
        W[(k * s + m) * C + l] = (double)w[l];
      }
    }
  }
  return (kmax + 1) * s * C;
}

int filter_extrap_table(int order, int kmax, double* Wf) {
  const int C = order == 4 ? 5 : 3;
  for (int k = 0; k <= kmax; ++k) {
    ld w[5];
    if (!extrap_weights(order, k + 1, w)) return -1;
    for (int l = 0; l < C; ++l) Wf[k * C + l] = (double)w[l];
  }
  return (kmax + 1) * C;
}

bool pade10_coeffs(double alpha, double* a) {
  // sum_n a_n n^{2j} = (j == 0 ? 1 + 2 alpha : 2 alpha) for j = 0..4 (T = 1 + O(w^10)),
  // sum_n a_n (-1)^n = 0 (T(pi) = 0).
  ld M[36], b[6];
  for (int j = 0; j < 5; ++j) {
    for (int n = 0; n < 6; ++n) M[j * 6 + n] = powl((ld)n, 2 * j);
    b[j] = (j == 0) ? 1.0L + 2.0L * alpha : 2.0L * alpha;
  }
  for (int n = 0; n < 6; ++n) M[5 * 6 + n] = (n % 2 == 0) ? 1.0L : -1.0L;
  b[5] = 0.0L;
  if (!solve_small(6, M, b)) return false;
  for (int n = 0; n < 6; ++n) a[n] = (double)b[n];
  return true;
}

}  // namespace cfs

extern "C" int cfs_at_weights(int order, int kmax, double* W) {
  if (!W) return -1;
  return cfs::at_weight_table(order, kmax, W);
}
