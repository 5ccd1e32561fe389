// Small dense complex linear algebra for the Rayleigh-Ritz step of the eigensolver (host).
//
// The subspace eigensolver (ov_eig.cu) keeps its n-vectors on the device and reduces them
// to b x b matrices (b <= 64) there; the b x b eigenproblem, Cholesky factor and inverse of
// those projections are solved here, as GPU eigensolvers commonly do for the projected
// problem. Methods: cyclic Jacobi for Hermitian matrices (Golub and Van Loan, Matrix
// Computations, 4th ed., Sec. 8.5), Householder reduction to Hessenberg form and the
// shifted QR iteration for general complex matrices (ibid., Secs. 7.4-7.5), eigenvectors
// of the triangular Schur factor by back substitution (ibid., Sec. 7.6.4), and the unitary
// factor of a QR factorisation by modified Gram-Schmidt applied twice (ibid., Sec. 5.2.8;
// Giraud, Langou and Rozloznik, Comput. Math. Appl. 50 (2005) for the second pass).
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "ov_internal.h"

namespace ov {
namespace {
using cd = std::complex<double>;

// A (row-major n x n) -> A = Q T Q^dag with T upper triangular; Q row-major. Returns false
// if the QR iteration did not converge.
bool schur(int n, std::vector<cd>& A, std::vector<cd>& Q) {
  auto a = [&](int i, int j) -> cd& { return A[(size_t)i * n + j]; };
  auto q = [&](int i, int j) -> cd& { return Q[(size_t)i * n + j]; };
  Q.assign((size_t)n * n, cd(0.0));
  for (int i = 0; i < n; ++i) q(i, i) = 1.0;
  // Householder reduction to upper Hessenberg form
  std::vector<cd> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double alpha2 = 0.0;
    for (int i = k + 1; i < n; ++i) alpha2 += std::norm(a(i, k));
    const double alpha = sqrt(alpha2);
    if (alpha == 0.0) continue;
    const cd x0 = a(k + 1, k);
    const cd ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0);
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    for (int i = k + 1; i < n; ++i) v[i] = a(i, k);
    v[k + 1] += ph * alpha;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // A = H A H with H = I - 2 v v^dag / |v|^2; Q = Q H
    for (int j = 0; j < n; ++j) {
      cd s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * a(i, j);
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) a(i, j) -= v[i] * s;
    }
    for (int i = 0; i < n; ++i) {
      cd s = 0.0;
      for (int j = k + 1; j < n; ++j) s += a(i, j) * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) a(i, j) -= s * std::conj(v[j]);
    }
    for (int i = 0; i < n; ++i) {
      cd s = 0.0;
      for (int j = k + 1; j < n; ++j) s += q(i, j) * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) q(i, j) -= s * std::conj(v[j]);
    }
    for (int i = k + 2; i < n; ++i) a(i, k) = 0.0;
  }
  // shifted QR on the active block [lo, hi] with Givens rotations (Wilkinson shift)
  int hi = n - 1;
  int iter = 0;
  const double eps = 2.2e-16;
  while (hi > 0) {
    if (++iter > 100 * n) return false;
    // deflate negligible subdiagonals
    int lo = hi;
    while (lo > 0) {
      const double s = std::abs(a(lo, lo)) + std::abs(a(lo - 1, lo - 1));
      if (std::abs(a(lo, lo - 1)) <= eps * (s > 0.0 ? s : 1.0)) {
        a(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      iter = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2 x 2 block
    const cd p = a(hi - 1, hi - 1), r = a(hi - 1, hi), s2 = a(hi, hi - 1), t = a(hi, hi);
    const cd tr = p + t, det = p * t - r * s2;
    const cd disc = std::sqrt(tr * tr * 0.25 - det);
    const cd m1 = tr * 0.5 + disc, m2 = tr * 0.5 - disc;
    cd mu = std::abs(m1 - t) < std::abs(m2 - t) ? m1 : m2;
    if (iter % 11 == 10) mu = t + std::abs(a(hi, hi - 1)) * 0.75;  // exceptional shift
    // QR step on rows/cols lo..hi: (H - mu I) = QR, H <- RQ + mu I, by Givens rotations
    cd x = a(lo, lo) - mu, y = a(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      const double nrm = sqrt(std::norm(x) + std::norm(y));
      cd c = 1.0, s = 0.0;
      if (nrm > 0.0) {
        c = x / nrm;
        s = y / nrm;
      }
      // G = [[conj(c), conj(s)], [-s, c]] applied to rows k, k+1 (columns from k-1 on)
      for (int j = std::max(lo, k - 1); j < n; ++j) {
        const cd u = a(k, j), w = a(k + 1, j);
        a(k, j) = std::conj(c) * u + std::conj(s) * w;
        a(k + 1, j) = -s * u + c * w;
      }
      // columns k, k+1 of A (rows 0..min(k+2, hi)) and of Q multiplied by G^dag
      for (int i = 0; i <= std::min(k + 2, hi); ++i) {
        const cd u = a(i, k), w = a(i, k + 1);
        a(i, k) = c * u + s * w;
        a(i, k + 1) = -std::conj(s) * u + std::conj(c) * w;
      }
      for (int i = 0; i < n; ++i) {
        const cd u = q(i, k), w = q(i, k + 1);
        q(i, k) = c * u + s * w;
        q(i, k + 1) = -std::conj(s) * u + std::conj(c) * w;
      }
      if (k + 1 < hi) {
        x = a(k + 1, k);
        y = a(k + 2, k);
      }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) a(i, j) = 0.0;
  return true;
}

}  // namespace

// Eigenvalues w and right eigenvectors (columns of V, row-major n x n, unit norm) of a
// general complex n x n matrix A (row-major). Returns false if the QR iteration failed.
bool small_eig(int n, const double2* A_in, double2* w, double2* V_out) {
  std::vector<cd> A((size_t)n * n), Q;
  for (size_t e = 0; e < (size_t)n * n; ++e) A[e] = cd(A_in[e].x, A_in[e].y);
  if (!schur(n, A, Q)) return false;
  auto t = [&](int i, int j) { return A[(size_t)i * n + j]; };
  // eigenvectors of T: for each k, solve (T - t_kk) y = 0 with y_k = 1, y_i = 0 for i > k
  std::vector<cd> Y((size_t)n * n, cd(0.0));
  double tnorm = 0.0;
  for (size_t e = 0; e < (size_t)n * n; ++e) tnorm = std::max(tnorm, std::abs(A[e]));
  const double small = 1e-15 * (tnorm > 0.0 ? tnorm : 1.0);
  for (int k = 0; k < n; ++k) {
    const cd lam = t(k, k);
    Y[(size_t)k * n + k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      cd s = 0.0;
      for (int j = i + 1; j <= k; ++j) s += t(i, j) * Y[(size_t)j * n + k];
      cd d = t(i, i) - lam;
      if (std::abs(d) < small) d = small;
      Y[(size_t)i * n + k] = -s / d;
    }
  }
  for (int k = 0; k < n; ++k) {
    w[k] = make_double2(t(k, k).real(), t(k, k).imag());
    double nr = 0.0;
    std::vector<cd> col(n, cd(0.0));
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j <= k; ++j) col[i] += Q[(size_t)i * n + j] * Y[(size_t)j * n + k];
      nr += std::norm(col[i]);
    }
    nr = sqrt(nr);
    for (int i = 0; i < n; ++i) V_out[(size_t)i * n + k] = make_double2(col[i].real() / nr, col[i].imag() / nr);
  }
  return true;
}

// Eigenvalues (real, ascending) and orthonormal eigenvectors (columns of V) of a Hermitian
// n x n matrix by cyclic Jacobi rotations.
bool small_eigh(int n, const double2* A_in, double* w, double2* V_out) {
  std::vector<cd> A((size_t)n * n), V((size_t)n * n, cd(0.0));
  for (size_t e = 0; e < (size_t)n * n; ++e) A[e] = cd(A_in[e].x, A_in[e].y);
  for (int i = 0; i < n; ++i) {
    V[(size_t)i * n + i] = 1.0;
    A[(size_t)i * n + i] = A[(size_t)i * n + i].real();
  }
  auto a = [&](int i, int j) -> cd& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += std::norm(a(i, j));
        if (i != j) off += std::norm(a(i, j));
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd apq = a(p, q);
        const double ab = std::abs(apq);
        if (ab == 0.0) continue;
        const cd ph = apq / ab;  // a_pq = |a_pq| e^{i phi}
        const double app = a(p, p).real(), aqq = a(q, q).real();
        const double theta = 0.5 * atan2(2.0 * ab, aqq - app);
        const double c = cos(theta), s = sin(theta);
        // rotation J = [[c, s ph], [-s conj(ph), c]] on columns p, q: A <- J^dag A J
        for (int k = 0; k < n; ++k) {
          const cd u = a(k, p), v = a(k, q);
          a(k, p) = c * u - s * std::conj(ph) * v;
          a(k, q) = s * ph * u + c * v;
        }
        for (int k = 0; k < n; ++k) {
          const cd u = a(p, k), v = a(q, k);
          a(p, k) = c * u - s * ph * v;
          a(q, k) = s * std::conj(ph) * u + c * v;
        }
        a(p, q) = 0.0;
        a(q, p) = 0.0;
        for (int k = 0; k < n; ++k) {
          const cd u = V[(size_t)k * n + p], v = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * u - s * std::conj(ph) * v;
          V[(size_t)k * n + q] = s * ph * u + c * v;
        }
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return a(x, x).real() < a(y, y).real(); });
  for (int k = 0; k < n; ++k) {
    w[k] = a(idx[k], idx[k]).real();
    for (int i = 0; i < n; ++i) {
      const cd v = V[(size_t)i * n + idx[k]];
      V_out[(size_t)i * n + k] = make_double2(v.real(), v.imag());
    }
  }
  return true;
}

// Upper Cholesky factor R (A = R^dag R) of a Hermitian positive definite n x n matrix and
// its inverse Rinv (both row-major). Returns false if A is not positive definite.
bool small_chol_inv(int n, const double2* A_in, double2* Rinv_out) {
  std::vector<cd> R((size_t)n * n, cd(0.0));
  auto A = [&](int i, int j) { return cd(A_in[(size_t)i * n + j].x, A_in[(size_t)i * n + j].y); };
  for (int j = 0; j < n; ++j) {
    double d = A(j, j).real();
    for (int k = 0; k < j; ++k) d -= std::norm(R[(size_t)k * n + j]);
    if (!(d > 0.0)) return false;
    const double rjj = sqrt(d);
    R[(size_t)j * n + j] = rjj;
    for (int i = j + 1; i < n; ++i) {
      cd s = A(j, i);
      for (int k = 0; k < j; ++k) s -= std::conj(R[(size_t)k * n + j]) * R[(size_t)k * n + i];
      R[(size_t)j * n + i] = s / rjj;
    }
  }
  // inverse of the upper triangular R by back substitution, column by column
  std::vector<cd> X((size_t)n * n, cd(0.0));
  for (int c = 0; c < n; ++c) {
    for (int i = n - 1; i >= 0; --i) {
      cd s = i == c ? cd(1.0) : cd(0.0);
      for (int k = i + 1; k < n; ++k) s -= R[(size_t)i * n + k] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = s / R[(size_t)i * n + i];
    }
  }
  for (size_t e = 0; e < (size_t)n * n; ++e) Rinv_out[e] = make_double2(X[e].real(), X[e].imag());
  return true;
}

// Inverse of a general complex n x n matrix by Gauss-Jordan with partial pivoting.
bool small_inv(int n, const double2* A_in, double2* X_out) {
  std::vector<cd> A((size_t)n * n), X((size_t)n * n, cd(0.0));
  for (size_t e = 0; e < (size_t)n * n; ++e) A[e] = cd(A_in[e].x, A_in[e].y);
  for (int i = 0; i < n; ++i) X[(size_t)i * n + i] = 1.0;
  for (int j = 0; j < n; ++j) {
    int p = j;
    for (int i = j + 1; i < n; ++i)
      if (std::abs(A[(size_t)i * n + j]) > std::abs(A[(size_t)p * n + j])) p = i;
    if (std::abs(A[(size_t)p * n + j]) == 0.0) return false;
    for (int c = 0; c < n; ++c) {
      std::swap(A[(size_t)j * n + c], A[(size_t)p * n + c]);
      std::swap(X[(size_t)j * n + c], X[(size_t)p * n + c]);
    }
    const cd inv = 1.0 / A[(size_t)j * n + j];
    for (int c = 0; c < n; ++c) {
      A[(size_t)j * n + c] *= inv;
      X[(size_t)j * n + c] *= inv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == j) continue;
      const cd f = A[(size_t)i * n + j];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)i * n + c] -= f * A[(size_t)j * n + c];
        X[(size_t)i * n + c] -= f * X[(size_t)j * n + c];
      }
    }
  }
  for (size_t e = 0; e < (size_t)n * n; ++e) X_out[e] = make_double2(X[e].real(), X[e].imag());
  return true;
}

// Q (row-major n x n, unitary) with A = Q R, R upper triangular: the leading j columns of Q
// span those of A for every j. A column that is numerically dependent on the ones before it
// is replaced by the unit vector that keeps the most after projection (Q stays unitary).
bool small_qr_q(int n, const double2* A_in, double2* Q_out) {
  std::vector<cd> Q((size_t)n * n);
  for (size_t i = 0; i < (size_t)n * n; ++i) Q[i] = cd(A_in[i].x, A_in[i].y);
  auto q = [&](int i, int j) -> cd& { return Q[(size_t)i * n + j]; };
  std::vector<cd> u(n);
  auto project = [&](int j) {  // column j minus its components along columns 0 .. j-1
    for (int k = 0; k < j; ++k) {
      cd d = 0.0;
      for (int i = 0; i < n; ++i) d += std::conj(q(i, k)) * q(i, j);
      for (int i = 0; i < n; ++i) q(i, j) -= d * q(i, k);
    }
  };
  auto norm = [&](int j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::norm(q(i, j));
    return sqrt(s);
  };
  for (int j = 0; j < n; ++j) {
    const double n0 = norm(j);
    project(j);
    project(j);
    double nj = norm(j);
    if (!(nj > 1e-10 * n0) || !(nj > 0.0)) {
      int best = -1;
      double keep = -1.0;
      for (int e = 0; e < n; ++e) {
        for (int i = 0; i < n; ++i) q(i, j) = i == e ? 1.0 : 0.0;
        project(j);
        const double r = norm(j);
        if (r > keep) { keep = r; best = e; }
      }
      for (int i = 0; i < n; ++i) q(i, j) = i == best ? 1.0 : 0.0;
      project(j);
      project(j);
      nj = norm(j);
      if (!(nj > 0.5 / sqrt((double)n))) return false;  // some unit vector keeps >= 1/sqrt(n)
    }
    for (int i = 0; i < n; ++i) q(i, j) /= nj;
  }
  for (size_t i = 0; i < (size_t)n * n; ++i) Q_out[i] = make_double2(Q[i].real(), Q[i].imag());
  return true;
}

}  // namespace ov
