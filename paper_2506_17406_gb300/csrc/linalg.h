// Small dense FP64 linear algebra for the host-side reference-element builder.
// Row-major matrices; no external BLAS/LAPACK.
#pragma once
#include <cstddef>
#include <functional>
#include <vector>

namespace riesz {

struct Mat {
  int m = 0, n = 0;
  std::vector<double> a;
  Mat() {}
  Mat(int m_, int n_) : m(m_), n(n_), a((size_t)m_ * n_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * n + j]; }
  double operator()(int i, int j) const { return a[(size_t)i * n + j]; }
  static Mat eye(int n) {
    Mat I(n, n);
    for (int i = 0; i < n; ++i) I(i, i) = 1.0;
    return I;
  }
};

// Run fn(i) for i in [0, n) on up to hardware_concurrency() threads
// (interleaved static schedule; fn must be safe to call concurrently).
void parallel_for(int n, const std::function<void(int)>& fn);

// C = A^T diag(w) B for A [q][m], B [q][n] (blocked, threaded).  With B the
// same object as A only the upper triangle is computed and mirrored.
Mat gram_tn(const Mat& A, const std::vector<double>& w, const Mat& B);

Mat matmul(const Mat& A, const Mat& B);      // A B
Mat matmul_tn(const Mat& A, const Mat& B);   // A^T B
Mat transpose(const Mat& A);
Mat cols(const Mat& A, int c0, int c1);      // columns [c0, c1)

// Householder QR with column pivoting: A P = Q R.  Returns the full orthogonal
// Q (m x m) and |R_kk| for k < min(m, n) (non-increasing up to rounding).
void qr_colpiv(const Mat& A, Mat& Q, std::vector<double>& rdiag);

// Plain Householder QR of a square matrix: A = Q R, returns Q and diag(R).
void qr_square(const Mat& A, Mat& Q, std::vector<double>& rdiag);

// Orthonormal basis of the null space of C (known dimension dim); throws if
// the rank gap is not clean.
Mat null_space(const Mat& C, int dim, const char* what);

// Orthonormal basis of the column space of S (known rank); throws if not clean.
Mat range_space(const Mat& S, int rank, const char* what);

// Symmetric eigen-decomposition by cyclic Jacobi rotations.  Eigenvalues in
// ascending order; eigenvectors are the columns of V.
void sym_eig(const Mat& A, std::vector<double>& w, Mat& V);

// Inverse by LU with partial pivoting; also returns the 1-norm condition estimate.
Mat inverse(const Mat& A, double* cond1 = nullptr);

}  // namespace riesz
