#include "linalg.h"

#include <algorithm>
#include <exception>
#include <mutex>
#include <thread>
#include <cmath>
#include <stdexcept>
#include <string>

namespace riesz {

void parallel_for(int n, const std::function<void(int)>& fn) {
  const int nt = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  std::exception_ptr err = nullptr;
  std::mutex mu;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      try {
        for (int i = t; i < n; i += nt) fn(i);
      } catch (...) {
        std::lock_guard<std::mutex> lk(mu);
        if (!err) err = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  if (err) std::rethrow_exception(err);
}

Mat gram_tn(const Mat& A, const std::vector<double>& w, const Mat& B) {
  if (A.m != B.m || (int)w.size() != A.m) throw std::runtime_error("gram_tn: shape mismatch");
  const bool sym = &A == &B;
  const int q = A.m, m = A.n, n = B.n;
  // operands with the summation index contiguous: At [m][q], WBt [n][q] = (diag(w) B)^T
  std::vector<double> At((size_t)m * q), WBt((size_t)n * q);
  for (int k = 0; k < q; ++k) {
    for (int i = 0; i < m; ++i) At[(size_t)i * q + k] = A(k, i);
    for (int j = 0; j < n; ++j) WBt[(size_t)j * q + k] = w[k] * B(k, j);
  }
  Mat C(m, n);
  constexpr int BI = 4, BJ = 4;
  const int nbi = (m + BI - 1) / BI;
  parallel_for(nbi, [&](int bi) {
    const int i0 = bi * BI;
    const int j_start = sym ? i0 : 0;
    for (int j0 = j_start; j0 < n; j0 += BJ) {
      double acc[BI][BJ] = {};
      const double* a[BI];
      const double* b[BJ];
      for (int r = 0; r < BI; ++r) a[r] = &At[(size_t)std::min(i0 + r, m - 1) * q];
      for (int c = 0; c < BJ; ++c) b[c] = &WBt[(size_t)std::min(j0 + c, n - 1) * q];
      for (int k = 0; k < q; ++k) {
        double av[BI], bv[BJ];
        for (int r = 0; r < BI; ++r) av[r] = a[r][k];
        for (int c = 0; c < BJ; ++c) bv[c] = b[c][k];
        for (int r = 0; r < BI; ++r)
          for (int c = 0; c < BJ; ++c) acc[r][c] += av[r] * bv[c];
      }
      for (int r = 0; r < BI && i0 + r < m; ++r)
        for (int c = 0; c < BJ && j0 + c < n; ++c) C(i0 + r, j0 + c) = acc[r][c];
    }
  });
  if (sym)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j) C(i, j) = C(j, i);
  return C;
}

Mat matmul(const Mat& A, const Mat& B) {
  if (A.n != B.m) throw std::runtime_error("matmul: shape mismatch");
  Mat C(A.m, B.n);
  for (int i = 0; i < A.m; ++i) {
    double* c = &C.a[(size_t)i * C.n];
    for (int k = 0; k < A.n; ++k) {
      const double aik = A(i, k);
      if (aik == 0.0) continue;
      const double* b = &B.a[(size_t)k * B.n];
      for (int j = 0; j < B.n; ++j) c[j] += aik * b[j];
    }
  }
  return C;
}

Mat matmul_tn(const Mat& A, const Mat& B) {
  if (A.m != B.m) throw std::runtime_error("matmul_tn: shape mismatch");
  Mat C(A.n, B.n);
  for (int k = 0; k < A.m; ++k) {
    const double* a = &A.a[(size_t)k * A.n];
    const double* b = &B.a[(size_t)k * B.n];
    for (int i = 0; i < A.n; ++i) {
      const double aki = a[i];
      if (aki == 0.0) continue;
      double* c = &C.a[(size_t)i * C.n];
      for (int j = 0; j < B.n; ++j) c[j] += aki * b[j];
    }
  }
  return C;
}

Mat transpose(const Mat& A) {
  Mat T(A.n, A.m);
  for (int i = 0; i < A.m; ++i)
    for (int j = 0; j < A.n; ++j) T(j, i) = A(i, j);
  return T;
}

Mat cols(const Mat& A, int c0, int c1) {
  Mat B(A.m, c1 - c0);
  for (int i = 0; i < A.m; ++i)
    for (int j = c0; j < c1; ++j) B(i, j - c0) = A(i, j);
  return B;
}

// Householder reflector H = I - beta v v^T with v[0] = 1 that maps x to
// (alpha, 0, ..., 0).  Returns beta; writes v and alpha.
static double householder(const double* x, int len, int stride, std::vector<double>& v,
                          double& alpha) {
  double sigma = 0.0;
  for (int i = 1; i < len; ++i) sigma += x[(size_t)i * stride] * x[(size_t)i * stride];
  const double x0 = x[0];
  v.assign(len, 0.0);
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = x[(size_t)i * stride];
  if (sigma == 0.0) {
    alpha = x0;
    return 0.0;
  }
  const double mu = std::sqrt(x0 * x0 + sigma);
  const double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
  const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] /= v0;
  alpha = mu;
  return beta;
}

// Shared worker: QR (with or without column pivoting) of A (m x n).
static void qr_impl(const Mat& A, bool pivot, Mat& Q, std::vector<double>& rdiag) {
  const int m = A.m, n = A.n, K = std::min(m, n);
  // store columns contiguously for speed: W is n x m (column j = row j of W)
  std::vector<double> W((size_t)n * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A(i, j);
  std::vector<std::vector<double>> vs(K);
  std::vector<double> betas(K, 0.0);
  rdiag.assign(K, 0.0);
  std::vector<double> v;
  for (int k = 0; k < K; ++k) {
    if (pivot) {
      int best = k;
      double bn = -1.0;
      for (int j = k; j < n; ++j) {
        const double* c = &W[(size_t)j * m];
        double s = 0.0;
        for (int i = k; i < m; ++i) s += c[i] * c[i];
        if (s > bn) {
          bn = s;
          best = j;
        }
      }
      if (best != k)
        std::swap_ranges(W.begin() + (size_t)k * m, W.begin() + (size_t)(k + 1) * m,
                         W.begin() + (size_t)best * m);
    }
    double alpha;
    double* ck = &W[(size_t)k * m];
    const double beta = householder(ck + k, m - k, 1, v, alpha);
    rdiag[k] = std::fabs(alpha);
    ck[k] = alpha;
    for (int i = k + 1; i < m; ++i) ck[i] = 0.0;
    if (beta != 0.0) {
      for (int j = k + 1; j < n; ++j) {
        double* c = &W[(size_t)j * m];
        double s = 0.0;
        for (int i = 0; i < m - k; ++i) s += v[i] * c[k + i];
        s *= beta;
        for (int i = 0; i < m - k; ++i) c[k + i] -= s * v[i];
      }
    }
    vs[k] = v;
    betas[k] = beta;
  }
  // Q = H_0 H_1 ... H_{K-1}: apply to the identity from the last reflector.
  // Keep Q column-major in a scratch buffer (columns contiguous).
  std::vector<double> Qc((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Qc[(size_t)i * m + i] = 1.0;
  for (int k = K - 1; k >= 0; --k) {
    if (betas[k] == 0.0) continue;
    const std::vector<double>& vk = vs[k];
    for (int j = 0; j < m; ++j) {
      double* c = &Qc[(size_t)j * m];
      double s = 0.0;
      for (int i = 0; i < m - k; ++i) s += vk[i] * c[k + i];
      if (s == 0.0) continue;
      s *= betas[k];
      for (int i = 0; i < m - k; ++i) c[k + i] -= s * vk[i];
    }
  }
  Q = Mat(m, m);
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) Q(i, j) = Qc[(size_t)j * m + i];
}

void qr_colpiv(const Mat& A, Mat& Q, std::vector<double>& rdiag) { qr_impl(A, true, Q, rdiag); }
void qr_square(const Mat& A, Mat& Q, std::vector<double>& rdiag) { qr_impl(A, false, Q, rdiag); }

Mat null_space(const Mat& C, int dim, const char* what) {
  const int n = C.n;
  if (dim == 0) return Mat(n, 0);
  Mat Ct = transpose(C);  // n x mc
  Mat Q;
  std::vector<double> rd;
  qr_colpiv(Ct, Q, rd);
  const int rank = n - dim;
  const double r0 = rd.empty() ? 0.0 : rd[0];
  if (rank > (int)rd.size()) throw std::runtime_error(std::string("null_space: too few constraints: ") + what);
  if (rank > 0 && !(rd[rank - 1] > 1e-8 * r0))
    throw std::runtime_error(std::string("null_space: rank deficient: ") + what);
  if (rank < (int)rd.size() && !(rd[rank] < 1e-10 * r0))
    throw std::runtime_error(std::string("null_space: no rank gap: ") + what);
  return cols(Q, rank, n);
}

Mat range_space(const Mat& S, int rank, const char* what) {
  Mat Q;
  std::vector<double> rd;
  qr_colpiv(S, Q, rd);
  const double r0 = rd[0];
  if (!(rd[rank - 1] > 1e-8 * r0)) throw std::runtime_error(std::string("range_space: rank deficient: ") + what);
  if (rank < (int)rd.size() && !(rd[rank] < 1e-10 * r0))
    throw std::runtime_error(std::string("range_space: no rank gap: ") + what);
  return cols(Q, 0, rank);
}

void sym_eig(const Mat& A0, std::vector<double>& w, Mat& V) {
  const int n = A0.m;
  Mat A = A0;
  V = Mat::eye(n);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double x = A(i, j) * A(i, j);
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A(p, p), aqq = A(q, q);
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A(k, p), akq = A(k, q);
          A(k, p) = c * akp - s * akq;
          A(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A(p, k), aqk = A(q, k);
          A(p, k) = c * apk - s * aqk;
          A(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V(k, p), vkq = V(k, q);
          V(k, p) = c * vkp - s * vkq;
          V(k, q) = s * vkp + c * vkq;
        }
      }
    }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return A(a, a) < A(b, b); });
  w.resize(n);
  Mat Vs(n, n);
  for (int j = 0; j < n; ++j) {
    w[j] = A(idx[j], idx[j]);
    for (int i = 0; i < n; ++i) Vs(i, j) = V(i, idx[j]);
  }
  V = Vs;
}

Mat inverse(const Mat& A, double* cond1) {
  const int n = A.m;
  Mat LU = A;
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(LU(k, k));
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(LU(i, k)) > best) {
        best = std::fabs(LU(i, k));
        p = i;
      }
    if (best == 0.0) throw std::runtime_error("inverse: singular matrix");
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(LU(k, j), LU(p, j));
    for (int i = k + 1; i < n; ++i) {
      const double f = LU(i, k) / LU(k, k);
      LU(i, k) = f;
      if (f == 0.0) continue;
      for (int j = k + 1; j < n; ++j) LU(i, j) -= f * LU(k, j);
    }
  }
  Mat X = Mat::eye(n);
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < n; ++j) std::swap(X(k, j), X(piv[k], j));
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {  // forward (unit lower)
      double s = X(i, j);
      for (int k = 0; k < i; ++k) s -= LU(i, k) * X(k, j);
      X(i, j) = s;
    }
    for (int i = n - 1; i >= 0; --i) {  // backward
      double s = X(i, j);
      for (int k = i + 1; k < n; ++k) s -= LU(i, k) * X(k, j);
      X(i, j) = s / LU(i, i);
    }
  }
  if (cond1) {
    double na = 0.0, ni = 0.0;
    for (int j = 0; j < n; ++j) {
      double sa = 0.0, si = 0.0;
      for (int i = 0; i < n; ++i) {
        sa += std::fabs(A(i, j));
        si += std::fabs(X(i, j));
      }
      na = std::max(na, sa);
      ni = std::max(ni, si);
    }
    *cond1 = na * ni;
  }
  return X;
}

}  // namespace riesz
