// Host dense linear algebra for the one-time coarse eigendecomposition
// (Algorithm 2 step 1 on V_H): A_H Q = M_H Q Lambda with Q^T M_H Q = I.
//
// Method (textbook, no library): Cholesky M = L L^T, C = L^{-1} A L^{-T},
// cyclic Jacobi on the symmetric C (Golub & Van Loan, "Matrix Computations",
// the cyclic Jacobi algorithm with the symmetric 2x2 Schur decomposition),
// Q = L^{-T} V, eigenvalues sorted ascending.  Jacobi is slow (O(n^3) per
// sweep) but accurate; the coarse dimension is a few hundred.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

namespace pasm {

// In-place lower Cholesky factor of the n x n row-major SPD matrix a.
// Returns false if a pivot is not positive.
static bool cholesky(int n, std::vector<double>& a) {
  for (int j = 0; j < n; ++j) {
    double s = a[(size_t)j * n + j];
    for (int p = 0; p < j; ++p) s -= a[(size_t)j * n + p] * a[(size_t)j * n + p];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    a[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = a[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) t -= a[(size_t)i * n + p] * a[(size_t)j * n + p];
      a[(size_t)i * n + j] = t / ljj;
    }
    for (int i = 0; i < j; ++i) a[(size_t)i * n + j] = 0.0;
  }
  return true;
}

// Solve L x = b in place for each column of B (n x m row-major).
static void lower_solve(int n, int m, const std::vector<double>& L, std::vector<double>& B) {
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < n; ++i) {
      double s = B[(size_t)i * m + c];
      for (int p = 0; p < i; ++p) s -= L[(size_t)i * n + p] * B[(size_t)p * m + c];
      B[(size_t)i * m + c] = s / L[(size_t)i * n + i];
    }
}

// Solve L^T x = b in place for each column of B.
static void upper_solve_t(int n, int m, const std::vector<double>& L, std::vector<double>& B) {
  for (int c = 0; c < m; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = B[(size_t)i * m + c];
      for (int p = i + 1; p < n; ++p) s -= L[(size_t)p * n + i] * B[(size_t)p * m + c];
      B[(size_t)i * m + c] = s / L[(size_t)i * n + i];
    }
}

// Cyclic Jacobi on symmetric C (overwritten); V receives the eigenvectors (columns).
static void jacobi_eig(int n, std::vector<double>& C, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double x : C) fro += x * x;
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += C[(size_t)p * n + q] * C[(size_t)p * n + q];
    if (std::sqrt(2.0 * off) <= 1e-17 * fro) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double cpq = C[(size_t)p * n + q];
        if (cpq == 0.0) continue;
        const double cpp = C[(size_t)p * n + p], cqq = C[(size_t)q * n + q];
        const double tau = (cqq - cpp) / (2.0 * cpq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // C <- J^T C J with J the rotation in the (p, q) plane
        for (int r = 0; r < n; ++r) {
          const double crp = C[(size_t)r * n + p], crq = C[(size_t)r * n + q];
          C[(size_t)r * n + p] = c * crp - s * crq;
          C[(size_t)r * n + q] = s * crp + c * crq;
        }
        for (int r = 0; r < n; ++r) {
          const double cpr = C[(size_t)p * n + r], cqr = C[(size_t)q * n + r];
          C[(size_t)p * n + r] = c * cpr - s * cqr;
          C[(size_t)q * n + r] = s * cpr + c * cqr;
        }
        C[(size_t)p * n + q] = C[(size_t)q * n + p] = 0.0;
        for (int r = 0; r < n; ++r) {
          const double vrp = V[(size_t)r * n + p], vrq = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = c * vrp - s * vrq;
          V[(size_t)r * n + q] = s * vrp + c * vrq;
        }
      }
  }
}

// A, M: n x n row-major symmetric.  lam (n) ascending, Q (n x n row-major,
// column j = eigenvector j).  Returns 0, or 1 if M or A is not SPD.
int coarse_generalized_eig(int n, const double* A, const double* M, double* lam, double* Q) {
  std::vector<double> L(M, M + (size_t)n * n);
  if (!cholesky(n, L)) return 1;
  // C = L^{-1} A L^{-T}: first W = L^{-1} A, then C = (L^{-1} W^T)^T = L^{-1} W^T (symmetric)
  std::vector<double> W(A, A + (size_t)n * n);
  lower_solve(n, n, L, W);
  std::vector<double> Wt((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Wt[(size_t)j * n + i] = W[(size_t)i * n + j];
  lower_solve(n, n, L, Wt);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = 0.5 * (Wt[(size_t)i * n + j] + Wt[(size_t)j * n + i]);
  std::vector<double> V;
  jacobi_eig(n, C, V);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return C[(size_t)x * n + x] < C[(size_t)y * n + y]; });
  for (int j = 0; j < n; ++j) {
    lam[j] = C[(size_t)order[j] * n + order[j]];
    if (!(lam[j] > 0.0)) return 1;
  }
  // Q = L^{-T} V (columns reordered)
  std::vector<double> Vs((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Vs[(size_t)i * n + j] = V[(size_t)i * n + order[j]];
  upper_solve_t(n, n, L, Vs);
  std::copy(Vs.begin(), Vs.end(), Q);
  return 0;
}

}  // namespace pasm
