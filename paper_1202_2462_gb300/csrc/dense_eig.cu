// Small dense eigenproblems of the set-up's second part (Sec. 3), on the host:
//   * harmonic Ritz pairs from an Arnoldi relation A V_m = V_{m+1} Hbar:
//     Hbar^H Hbar y = theta H_m^H y, brought to the standard form
//     (H_m + |h_{m+1,m}|^2 f e_m^T) y = theta y with H_m^H f = e_m (the matrix
//     stays upper Hessenberg), solved by the shifted QR algorithm (Wilkinson
//     shifts, Givens rotations, deflation) with back substitution on the
//     Schur form for the eigenvectors (Golub and Van Loan, Matrix
//     Computations, 4th ed., Sec. 7.5 and 7.6);
//   * the Hermitian (DV)^dagger DV matrix by the cyclic complex Jacobi method
//     (each 2x2 pivot block made real by a diagonal phase, then a real Jacobi
//     rotation; Golub and Van Loan Sec. 8.5).
// Matrices are column-major complex (re, im interleaved).  These run once per
// set-up on matrices of dimension 2N <= 128.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "internal.h"

namespace sapmg {

using cd = std::complex<double>;

namespace {

struct Mat {
  int n = 0;
  std::vector<cd> a;
  explicit Mat(int n_) : n(n_), a((size_t)n_ * n_) {}
  cd& operator()(int i, int j) { return a[(size_t)j * n + i]; }
  cd operator()(int i, int j) const { return a[(size_t)j * n + i]; }
};

// Solve A x = b (A n x n, destroyed) by Gaussian elimination with partial pivoting.
bool solve_linear(Mat A, std::vector<cd>& b) {
  const int n = A.n;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(A(i, k)) > std::abs(A(p, k))) p = i;
    if (A(p, k) == cd(0)) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A(k, j), A(p, j));
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cd l = A(i, k) / A(k, k);
      for (int j = k; j < n; ++j) A(i, j) -= l * A(k, j);
      b[i] -= l * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    cd s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A(k, j) * b[j];
    b[k] = s / A(k, k);
  }
  return true;
}

// Givens rotation [c s; -conj(s) c] (c real) with [c s; -conj(s) c] [a; b] = [r; 0].
void givens(cd a, cd b, double& c, cd& s) {
  const double na = std::abs(a), nb = std::abs(b);
  if (nb == 0.0) { c = 1.0; s = 0.0; return; }
  if (na == 0.0) { c = 0.0; s = std::conj(b) / nb; return; }
  const double r = std::hypot(na, nb);
  c = na / r;
  s = (a / na) * std::conj(b) / r;
}

// Schur form of an upper Hessenberg matrix: H = Q T Q^H, T upper triangular
// (overwrites H with T), Q accumulated.  Returns false if it does not converge.
bool hessenberg_qr(Mat& H, Mat& Q) {
  const int n = H.n;
  const double eps = 2.2e-16;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Q(i, j) = i == j ? cd(1) : cd(0);
  int hi = n - 1, iter = 0;
  while (hi > 0) {
    // deflation: find the lowest small subdiagonal entry in the active block
    int lo = hi;
    while (lo > 0) {
      const double s = std::abs(H(lo - 1, lo - 1)) + std::abs(H(lo, lo));
      if (std::abs(H(lo, lo - 1)) <= eps * (s > 0 ? s : 1.0)) {
        H(lo, lo - 1) = 0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      iter = 0;
      continue;
    }
    if (++iter > 60 * n) return false;
    // Wilkinson shift from the trailing 2x2 block (exceptional shift every 11 steps)
    const cd a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
    cd mu;
    if (iter % 11 == 0) {
      mu = d + cd(std::abs(H(hi, hi - 1)), 0);
    } else {
      const cd tr = 0.5 * (a + d), det = a * d - b * c;
      const cd disc = std::sqrt(tr * tr - det);
      const cd l1 = tr + disc, l2 = tr - disc;
      mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
    }
    // one implicit QR step on rows/columns lo..hi: H - mu I = Q R, H <- R Q + mu I
    for (int k = lo; k <= hi; ++k) H(k, k) -= mu;
    std::vector<double> cs(hi - lo);
    std::vector<cd> sn(hi - lo);
    for (int k = lo; k < hi; ++k) {
      double c1;
      cd s1;
      givens(H(k, k), H(k + 1, k), c1, s1);
      cs[k - lo] = c1;
      sn[k - lo] = s1;
      for (int j = k; j < n; ++j) {
        const cd x = H(k, j), y = H(k + 1, j);
        H(k, j) = c1 * x + s1 * y;
        H(k + 1, j) = -std::conj(s1) * x + c1 * y;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const double c1 = cs[k - lo];
      const cd s1 = sn[k - lo];
      for (int i = 0; i <= std::min(k + 2, hi); ++i) {
        const cd x = H(i, k), y = H(i, k + 1);
        H(i, k) = c1 * x + std::conj(s1) * y;
        H(i, k + 1) = -s1 * x + c1 * y;
      }
      // rows above lo that belong to the already-deflated part see the same rotation
      for (int i = 0; i < n; ++i) {
        const cd x = Q(i, k), y = Q(i, k + 1);
        Q(i, k) = c1 * x + std::conj(s1) * y;
        Q(i, k + 1) = -s1 * x + c1 * y;
      }
    }
    for (int k = lo; k <= hi; ++k) H(k, k) += mu;
  }
  return true;
}

}  // namespace

int harmonic_ritz_host(int m, const double* hbar, double* theta_out, double* y_out) {
  if (m < 1 || !hbar || !theta_out || !y_out) return MG_ERR_ARG;
  const int ld = m + 1;
  auto hb = [&](int i, int j) { return cd(hbar[2 * ((size_t)j * ld + i)], hbar[2 * ((size_t)j * ld + i) + 1]); };
  // M = H_m + |h_{m+1,m}|^2 f e_m^T,  H_m^H f = e_m
  Mat M(m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) M(i, j) = hb(i, j);
  const double h2 = std::norm(hb(m, m - 1));
  if (h2 > 0) {
    Mat HmH(m);
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) HmH(i, j) = std::conj(M(j, i));
    std::vector<cd> f(m, cd(0));
    f[m - 1] = 1.0;
    if (!solve_linear(HmH, f)) return MG_ERR_NONFINITE;
    for (int i = 0; i < m; ++i) M(i, m - 1) += h2 * f[i];
  }
  Mat T = M, Q(m);
  if (!hessenberg_qr(T, Q)) return MG_ERR_NONFINITE;
  // eigenvectors of T by back substitution, then x = Q z
  std::vector<cd> theta(m);
  Mat X(m);
  double tnorm = 0;
  for (int j = 0; j < m; ++j)
    for (int i = 0; i <= j; ++i) tnorm = std::max(tnorm, std::abs(T(i, j)));
  const double small = 1e-14 * (tnorm > 0 ? tnorm : 1.0);
  for (int k = 0; k < m; ++k) {
    theta[k] = T(k, k);
    std::vector<cd> z(m, cd(0));
    z[k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      cd s = 0;
      for (int j = i + 1; j <= k; ++j) s += T(i, j) * z[j];
      cd den = T(i, i) - theta[k];
      if (std::abs(den) < small) den = small;
      z[i] = -s / den;
    }
    double nz = 0;
    std::vector<cd> x(m, cd(0));
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j <= k; ++j) x[i] += Q(i, j) * z[j];
      nz += std::norm(x[i]);
    }
    nz = std::sqrt(nz);
    for (int i = 0; i < m; ++i) X(i, k) = x[i] / nz;
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return std::abs(theta[a]) < std::abs(theta[b]); });
  for (int k = 0; k < m; ++k) {
    const int o = order[k];
    theta_out[2 * k] = theta[o].real();
    theta_out[2 * k + 1] = theta[o].imag();
    for (int i = 0; i < m; ++i) {
      y_out[2 * ((size_t)k * m + i)] = X(i, o).real();
      y_out[2 * ((size_t)k * m + i) + 1] = X(i, o).imag();
    }
  }
  for (int k = 0; k < 2 * m; ++k)
    if (!std::isfinite(theta_out[k])) return MG_ERR_NONFINITE;
  return MG_OK;
}

int eigh_host(int n, const double* a_in, double* w_out, double* v_out) {
  if (n < 1 || !a_in || !w_out || !v_out) return MG_ERR_ARG;
  Mat A(n), V(n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      A(i, j) = cd(a_in[2 * ((size_t)j * n + i)], a_in[2 * ((size_t)j * n + i) + 1]);
      V(i, j) = i == j ? cd(1) : cd(0);
    }
  // symmetrise (the input is Hermitian up to rounding)
  for (int j = 0; j < n; ++j) {
    A(j, j) = cd(A(j, j).real(), 0);
    for (int i = j + 1; i < n; ++i) {
      const cd h = 0.5 * (A(i, j) + std::conj(A(j, i)));
      A(i, j) = h;
      A(j, i) = std::conj(h);
    }
  }
  double fro = 0;
  for (const cd& x : A.a) fro += std::norm(x);
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i)
        if (i != j) off += std::norm(A(i, j));
    if (std::sqrt(off) <= 1e-15 * (fro > 0 ? fro : 1.0)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd apq = A(p, q);
        const double g = std::abs(apq);
        if (g == 0.0) continue;
        const cd ph = apq / g;                     // A(p, q) = g ph
        const double app = A(p, p).real(), aqq = A(q, q).real();
        // real Jacobi rotation for [[app, g], [g, aqq]]
        const double tau = (aqq - app) / (2.0 * g);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        // U = diag(1, conj(ph)) [[c, s], [-s, c]] on columns p, q
        const cd u00 = c, u01 = s, u10 = -s * std::conj(ph), u11 = c * std::conj(ph);
        for (int k = 0; k < n; ++k) {
          const cd x = A(k, p), y = A(k, q);
          A(k, p) = x * u00 + y * u10;
          A(k, q) = x * u01 + y * u11;
        }
        for (int k = 0; k < n; ++k) {
          const cd x = A(p, k), y = A(q, k);
          A(p, k) = std::conj(u00) * x + std::conj(u10) * y;
          A(q, k) = std::conj(u01) * x + std::conj(u11) * y;
        }
        A(p, q) = 0;
        A(q, p) = 0;
        A(p, p) = cd(A(p, p).real(), 0);
        A(q, q) = cd(A(q, q).real(), 0);
        for (int k = 0; k < n; ++k) {
          const cd x = V(k, p), y = V(k, q);
          V(k, p) = x * u00 + y * u10;
          V(k, q) = x * u01 + y * u11;
        }
      }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return A(a, a).real() < A(b, b).real(); });
  for (int k = 0; k < n; ++k) {
    const int o = order[k];
    w_out[k] = A(o, o).real();
    for (int i = 0; i < n; ++i) {
      v_out[2 * ((size_t)k * n + i)] = V(i, o).real();
      v_out[2 * ((size_t)k * n + i) + 1] = V(i, o).imag();
    }
  }
  return MG_OK;
}

}  // namespace sapmg
