// Host FP64 builder of the reference element of arXiv 2506.17406 (Sections 3-4).
//
// Steps, in the paper's order:
//   1. the local spaces of Eq. (2.5) and, for the H(div) degrees of freedom,
//      the second-kind Nedelec space of Eq. (2.6) (Section 3.4.3);
//   2. bubble spaces on every subsimplex (Section 3.1);
//   3. the augmented eigenproblem of Eq. (3.10) on each bubble space, the kernel
//      of d dropped and the rest rescaled so that Eq. (3.9) holds;
//   4. the degrees of freedom of Eqs. (3.14), (3.16), (3.18);
//   5. the dual (Ciarlet) basis, and from it the reference matrices contracted
//      by the device operator.
//
// Conventions (the paper leaves them open):
//   * equilateral reference simplices of edge length 2, centroid at 0;
//   * a face (edge) of the reference tetrahedron is parametrised by the
//     isometric affine map sending the reference triangle's (interval's)
//     vertices, in order, to the face's (edge's) vertices in increasing order;
//     t = (x_b - x_a)/|.|, n = (x_b - x_a) x (x_c - x_a)/|.|;
//   * in Eq. (3.10) exactly dim d X^{k-1}(S) eigenpairs with the smallest mu
//     are dropped;
//   * eigenvectors are ordered by increasing mu; eigenvalues within a relative
//     spread of 1e-8 form a cluster whose basis is fixed by the echelon rule on
//     probe functionals (vector j of a cluster vanishes on probes 1..j-1 and is
//     positive on probe j);
//   * DOF order: vertices 0..3; edges 01,02,03,12,13,23; faces 012,013,023,123;
//     interior; inside an entity Whitney, type I, type II.
//
// The polynomial expansion is the orthonormal Dubiner (PKD) basis evaluated by
// homogenised Jacobi recurrences, integrated with collapsed Gauss-Jacobi rules.
#include "refelem.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>

namespace riesz {

namespace {

const double S3 = std::sqrt(3.0);
const double S6 = std::sqrt(6.0);
const double TET[4][3] = {{-1.0, -1.0 / S3, -1.0 / S6},
                          {1.0, -1.0 / S3, -1.0 / S6},
                          {0.0, 2.0 / S3, -1.0 / S6},
                          {0.0, 0.0, 3.0 / S6}};
const double TRI[3][2] = {{-1.0, -1.0 / S3}, {1.0, -1.0 / S3}, {0.0, 2.0 / S3}};
const int EDGES[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int FACES[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
const double CLUSTER_RTOL = 1e-8;

int dimP(int dim, int deg) {
  if (deg < 0) return 0;
  if (dim == 1) return deg + 1;
  if (dim == 2) return (deg + 1) * (deg + 2) / 2;
  return (deg + 1) * (deg + 2) * (deg + 3) / 6;
}

// simplex vertex coordinate accessor
double vert(int dim, int i, int c) {
  if (dim == 1) return i == 0 ? -1.0 : 1.0;
  if (dim == 2) return TRI[i][c];
  return TET[i][c];
}

// Barycentric coordinates (and their constant gradients) of a point.
struct Bary {
  int dim;
  double Minv[4][4];  // lambda = Minv * [x; 1]
  explicit Bary(int d) : dim(d) {
    Mat M(d + 1, d + 1);
    for (int i = 0; i <= d; ++i) {
      for (int c = 0; c < d; ++c) M(c, i) = vert(d, i, c);
      M(d, i) = 1.0;
    }
    Mat Mi = inverse(M);
    for (int i = 0; i <= d; ++i)
      for (int j = 0; j <= d; ++j) Minv[i][j] = Mi(i, j);
  }
  void lam(const double* x, double* l) const {
    for (int i = 0; i <= dim; ++i) {
      double s = Minv[i][dim];
      for (int c = 0; c < dim; ++c) s += Minv[i][c] * x[c];
      l[i] = s;
    }
  }
  double grad(int i, int c) const { return Minv[i][c]; }
};

// Homogenised Jacobi recurrence for P_n^{(alpha,0)} written as a polynomial in
// g1 = t*u and u: H_n = P_n(t) u^n.  Values and gradients (dim components).
void jacobi_h(int alpha, int nmax, double g1, const double* dg1, double u, const double* du, int dim,
              double* P, double* dP) {
  P[0] = 1.0;
  for (int c = 0; c < dim; ++c) dP[c] = 0.0;
  if (nmax == 0) return;
  P[1] = 0.5 * ((alpha + 2) * g1 + alpha * u);
  for (int c = 0; c < dim; ++c) dP[dim + c] = 0.5 * ((alpha + 2) * dg1[c] + alpha * du[c]);
  for (int n = 1; n < nmax; ++n) {
    const double s = 2.0 * n + alpha;
    const double den = 2.0 * (n + 1) * (n + alpha + 1) * s;
    const double c1 = (s + 1.0) * (s + 2.0) * s / den;
    const double c2 = (s + 1.0) * (double)alpha * alpha / den;
    const double c3 = 2.0 * (n + alpha) * n * (s + 2.0) / den;
    const double a = c1 * g1 + c2 * u;
    P[n + 1] = a * P[n] - c3 * u * u * P[n - 1];
    for (int c = 0; c < dim; ++c) {
      const double da = c1 * dg1[c] + c2 * du[c];
      dP[(n + 1) * dim + c] = da * P[n] + a * dP[n * dim + c] -
                              c3 * (2.0 * u * du[c] * P[n - 1] + u * u * dP[(n - 1) * dim + c]);
    }
  }
}

// Gauss-Jacobi nodes/weights for weight (1-x)^alpha on [-1,1] (Golub-Welsch).
void gauss_jacobi(int n, int alpha, std::vector<double>& x, std::vector<double>& w) {
  Mat T(n, n);
  const double a = alpha, b = 0.0;
  for (int k = 0; k < n; ++k) {
    const double s = 2.0 * k + a + b;
    T(k, k) = (k == 0) ? (b - a) / (a + b + 2.0) : (b * b - a * a) / (s * (s + 2.0));
    if (k >= 1) {
      const double num = 4.0 * k * (k + a) * (k + b) * (k + a + b);
      const double den = s * s * (s + 1.0) * (s - 1.0);
      T(k, k - 1) = T(k - 1, k) = std::sqrt(num / den);
    }
  }
  std::vector<double> ev;
  Mat V;
  sym_eig(T, ev, V);
  const double mu0 = std::pow(2.0, a + 1.0) / (a + 1.0);
  x = ev;
  w.resize(n);
  for (int k = 0; k < n; ++k) w[k] = mu0 * V(0, k) * V(0, k);
}

}  // namespace

// ---------------------------------------------------------------------------
// quadrature
// ---------------------------------------------------------------------------
Rule simplex_rule(int dim, int n) {
  Rule R;
  R.dim = dim;
  std::vector<double> x0, w0, x1, w1, x2, w2;
  gauss_jacobi(n, 0, x0, w0);
  if (dim == 1) {
    R.x = x0;
    R.w = w0;
    return R;
  }
  gauss_jacobi(n, 1, x1, w1);
  if (dim == 2) {
    const double area_scale = S3 / 2.0;  // biunit triangle (area 2) -> reference (sqrt 3)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double r1 = 0.5 * (1.0 + x0[i]) * (1.0 - x1[j]) - 1.0, r2 = x1[j];
        const double l1 = 0.5 * (r1 + 1.0), l2 = 0.5 * (r2 + 1.0);
        for (int c = 0; c < 2; ++c)
          R.x.push_back(TRI[0][c] + l1 * (TRI[1][c] - TRI[0][c]) + l2 * (TRI[2][c] - TRI[0][c]));
        R.w.push_back(0.5 * w0[i] * w1[j] * area_scale);
      }
    return R;
  }
  gauss_jacobi(n, 2, x2, w2);
  const double vol_scale = std::sqrt(2.0) / 2.0;  // biunit tet (4/3) -> reference (2 sqrt2 / 3)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        const double r1 = 0.25 * (1.0 + x0[i]) * (1.0 - x1[j]) * (1.0 - x2[k]) - 1.0;
        const double r2 = 0.5 * (1.0 + x1[j]) * (1.0 - x2[k]) - 1.0;
        const double r3 = x2[k];
        const double l1 = 0.5 * (r1 + 1.0), l2 = 0.5 * (r2 + 1.0), l3 = 0.5 * (r3 + 1.0);
        for (int c = 0; c < 3; ++c)
          R.x.push_back(TET[0][c] + l1 * (TET[1][c] - TET[0][c]) + l2 * (TET[2][c] - TET[0][c]) +
                        l3 * (TET[3][c] - TET[0][c]));
        R.w.push_back(0.125 * w0[i] * w1[j] * w2[k] * vol_scale);
      }
  return R;
}

// ---------------------------------------------------------------------------
// Dubiner expansion
// ---------------------------------------------------------------------------
static void pkd_raw(int dim, int deg, const std::vector<int>& order, const Bary& B, const double* x,
                    double* val, double* grad) {
  double lam[4];
  B.lam(x, lam);
  // biunit coordinates rho_k = -1 + 2 lambda_k (k = 1..dim) and d rho_k / dx_c
  double rho[3] = {0, 0, 0}, drho[3][3] = {{0}};
  for (int k = 0; k < dim; ++k) {
    rho[k] = -1.0 + 2.0 * lam[k + 1];
    for (int c = 0; c < dim; ++c) drho[k][c] = 2.0 * B.grad(k + 1, c);
  }
  const int nfun = dimP(dim, deg);
  std::vector<double> gr((size_t)nfun * 3, 0.0);  // gradient wrt rho
  std::vector<double> P(deg + 2), dP((deg + 2) * 3);
  if (dim == 1) {
    const double g1 = rho[0], dg1[1] = {1.0}, u = 1.0, du[1] = {0.0};
    jacobi_h(0, deg, g1, dg1, u, du, 1, P.data(), dP.data());
    for (int k = 0; k < nfun; ++k) {
      val[k] = P[order[k * 3]];
      gr[k * 3] = dP[order[k * 3]];
    }
  } else if (dim == 2) {
    const double X = rho[0], Y = rho[1];
    std::vector<double> A(deg + 2), dA((deg + 2) * 2);
    {
      const double g1 = 0.5 * (1.0 + 2.0 * X + Y), dg1[2] = {1.0, 0.5};
      const double u = 0.5 * (1.0 - Y), du[2] = {0.0, -0.5};
      jacobi_h(0, deg, g1, dg1, u, du, 2, A.data(), dA.data());
    }
    std::map<int, std::pair<std::vector<double>, std::vector<double>>> Bp;
    for (int k = 0; k < nfun; ++k) {
      const int p = order[k * 3], q = order[k * 3 + 1];
      auto it = Bp.find(p);
      if (it == Bp.end()) {
        std::vector<double> Bv(deg + 2), dB((deg + 2) * 2);
        const double g1 = Y, dg1[2] = {0.0, 1.0}, u = 1.0, du[2] = {0.0, 0.0};
        jacobi_h(2 * p + 1, deg - p, g1, dg1, u, du, 2, Bv.data(), dB.data());
        it = Bp.emplace(p, std::make_pair(Bv, dB)).first;
      }
      const double a = A[p], b = it->second.first[q];
      val[k] = a * b;
      for (int c = 0; c < 2; ++c) gr[k * 3 + c] = dA[p * 2 + c] * b + a * it->second.second[q * 2 + c];
    }
  } else {
    const double X = rho[0], Y = rho[1], Z = rho[2];
    std::vector<double> A(deg + 2), dA((deg + 2) * 3);
    {
      const double g1 = 0.5 * (2.0 + 2.0 * X + Y + Z), dg1[3] = {1.0, 0.5, 0.5};
      const double u = -0.5 * (Y + Z), du[3] = {0.0, -0.5, -0.5};
      jacobi_h(0, deg, g1, dg1, u, du, 3, A.data(), dA.data());
    }
    std::vector<std::vector<double>> Bv(deg + 1), dB(deg + 1);
    for (int p = 0; p <= deg; ++p) {
      Bv[p].resize(deg + 2);
      dB[p].resize((deg + 2) * 3);
      const double g1 = 0.5 * (1.0 + 2.0 * Y + Z), dg1[3] = {0.0, 1.0, 0.5};
      const double u = 0.5 * (1.0 - Z), du[3] = {0.0, 0.0, -0.5};
      jacobi_h(2 * p + 1, deg - p, g1, dg1, u, du, 3, Bv[p].data(), dB[p].data());
    }
    std::vector<double> C(deg + 2), dC((deg + 2) * 3);
    for (int k = 0; k < nfun; ++k) {
      const int p = order[k * 3], q = order[k * 3 + 1], r = order[k * 3 + 2];
      const double g1 = Z, dg1[3] = {0.0, 0.0, 1.0}, u = 1.0, du[3] = {0.0, 0.0, 0.0};
      jacobi_h(2 * p + 2 * q + 2, r, g1, dg1, u, du, 3, C.data(), dC.data());
      const double a = A[p], b = Bv[p][q], c = C[r];
      val[k] = a * b * c;
      for (int d = 0; d < 3; ++d)
        gr[k * 3 + d] = dA[p * 3 + d] * b * c + a * dB[p][q * 3 + d] * c + a * b * dC[r * 3 + d];
    }
  }
  if (grad)
    for (int k = 0; k < nfun; ++k)
      for (int c = 0; c < dim; ++c) {
        double s = 0.0;
        for (int m = 0; m < dim; ++m) s += gr[k * 3 + m] * drho[m][c];
        grad[k * dim + c] = s;
      }
}

static const Bary& bary(int dim) {
  static const Bary b1(1), b2(2), b3(3);
  return dim == 1 ? b1 : (dim == 2 ? b2 : b3);
}

Expansion::Expansion(int dim_, int deg_) : dim(dim_), deg(deg_) {
  n = dimP(dim, deg);
  for (int d = 0; d <= deg; ++d) {
    if (dim == 1) {
      order.insert(order.end(), {d, 0, 0});
    } else if (dim == 2) {
      for (int p = 0; p <= d; ++p) order.insert(order.end(), {p, d - p, 0});
    } else {
      for (int p = 0; p <= d; ++p)
        for (int q = 0; q <= d - p; ++q) order.insert(order.end(), {p, q, d - p - q});
    }
  }
  norm.assign(n, 1.0);
  Rule R = simplex_rule(dim, deg + 2);
  std::vector<double> v(n), acc(n, 0.0);
  for (int i = 0; i < R.npt(); ++i) {
    pkd_raw(dim, deg, order, bary(dim), &R.x[(size_t)i * dim], v.data(), nullptr);
    for (int k = 0; k < n; ++k) acc[k] += R.w[i] * v[k] * v[k];
  }
  for (int k = 0; k < n; ++k) norm[k] = 1.0 / std::sqrt(acc[k]);
}

void Expansion::eval(int npt, const double* x, double* values, double* grads) const {
  std::vector<double> g((size_t)n * dim);
  for (int i = 0; i < npt; ++i) {
    double* v = values + (size_t)i * n;
    pkd_raw(dim, deg, order, bary(dim), x + (size_t)i * dim, v, grads ? g.data() : nullptr);
    for (int k = 0; k < n; ++k) v[k] *= norm[k];
    if (grads)
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < dim; ++c) grads[((size_t)i * n + k) * dim + c] = g[k * dim + c] * norm[k];
  }
}

// ---------------------------------------------------------------------------
// Tabulated fields: a field space is a coefficient matrix over a scalar
// expansion repeated ncomp times (index comp * E.n + k).
// ---------------------------------------------------------------------------
namespace {

struct Tab {  // tabulation of the (vector) expansion at points
  int npt, nexp, ncomp, dim;
  std::vector<double> v, g;  // scalar expansion values (npt x nexp) and grads (npt x nexp x dim)
};

Tab tabulate_expansion(const Expansion& E, int ncomp, int npt, const double* x) {
  Tab T{npt, E.n, ncomp, E.dim, {}, {}};
  T.v.resize((size_t)npt * E.n);
  T.g.resize((size_t)npt * E.n * E.dim);
  E.eval(npt, x, T.v.data(), T.g.data());
  return T;
}

// value of field coefficient column y (length ncomp*nexp) at point i, component c
inline double field_val(const Tab& T, const double* y, int i, int c) {
  const double* v = &T.v[(size_t)i * T.nexp];
  const double* yc = y + (size_t)c * T.nexp;
  double s = 0.0;
  for (int k = 0; k < T.nexp; ++k) s += v[k] * yc[k];
  return s;
}
// derivative d f_c / d x_d at point i
inline double field_jac(const Tab& T, const double* y, int i, int c, int d) {
  const double* g = &T.g[(size_t)i * T.nexp * T.dim];
  const double* yc = y + (size_t)c * T.nexp;
  double s = 0.0;
  for (int k = 0; k < T.nexp; ++k) s += g[k * T.dim + d] * yc[k];
  return s;
}

// Exterior derivative of expansion element (comp c, fn k) at point i.
// family: 0 grad (scalar), 1 curl (vector, 3D) / scalar curl (2D), 2 div.
void d_of_basis(const Tab& T, int family, int i, int c, int k, double* out, int& nout) {
  const double* g = &T.g[((size_t)i * T.nexp + k) * T.dim];
  if (family == 0) {
    nout = T.dim;
    for (int d = 0; d < T.dim; ++d) out[d] = g[d];
  } else if (family == 1) {
    if (T.dim == 3) {  // curl(psi e_c) = grad psi x e_c
      nout = 3;
      double e[3] = {0, 0, 0};
      e[c] = 1.0;
      out[0] = g[1] * e[2] - g[2] * e[1];
      out[1] = g[2] * e[0] - g[0] * e[2];
      out[2] = g[0] * e[1] - g[1] * e[0];
    } else {  // d f2/dx - d f1/dy
      nout = 1;
      out[0] = (c == 1) ? g[0] : -g[1];
    }
  } else {
    nout = 1;
    out[0] = g[c];
  }
}

Mat d_gram(const Expansion& E, int ncomp, int family) {
  Rule R = simplex_rule(E.dim, E.deg + 2);
  Tab T = tabulate_expansion(E, ncomp, R.npt(), R.x.data());
  const int N = ncomp * E.n;
  Mat G(N, N);
  std::vector<double> D((size_t)N * 3);
  for (int i = 0; i < R.npt(); ++i) {
    int nd = 0;
    for (int c = 0; c < ncomp; ++c)
      for (int k = 0; k < E.n; ++k) d_of_basis(T, family, i, c, k, &D[(size_t)(c * E.n + k) * 3], nd);
    for (int a = 0; a < N; ++a)
      for (int b = a; b < N; ++b) {
        double s = 0.0;
        for (int d = 0; d < nd; ++d) s += D[(size_t)a * 3 + d] * D[(size_t)b * 3 + d];
        G(a, b) += R.w[i] * s;
      }
  }
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < a; ++b) G(a, b) = G(b, a);
  return G;
}

// --- local spaces ----------------------------------------------------------
enum Family { CG = 0, N1 = 1, N2 = 2, RT = 3, BDM = 4 };  // BDM: P_p^3 with normal-trace bubbles

struct FieldSpace {
  Expansion E;
  int ncomp;
  Mat U;  // (ncomp * E.n) x dim, L2-orthonormal columns
};

FieldSpace make_space(int fam, int p, int dim) {
  FieldSpace S;
  S.E = Expansion(dim, p);
  S.ncomp = (fam == CG) ? 1 : dim;
  const int N = S.ncomp * S.E.n;
  if (fam == CG || fam == N2 || fam == BDM) {  // the full P_p (P_p^dim) of Eq. (2.6)
    S.U = Mat::eye(N);
    return S;
  }
  const int nlow = dimP(dim, p - 1), nlow2 = dimP(dim, p - 2);
  Rule R = simplex_rule(dim, p + 2);
  Tab T = tabulate_expansion(S.E, S.ncomp, R.npt(), R.x.data());
  std::vector<std::vector<double>> span;
  for (int c = 0; c < dim; ++c)
    for (int k = 0; k < nlow; ++k) {
      std::vector<double> y(N, 0.0);
      y[c * S.E.n + k] = 1.0;
      span.push_back(y);
    }
  // the extra fields x-dependent times degree-(p-1) expansion functions
  auto project = [&](auto fieldfun) {
    std::vector<double> y(N, 0.0);
    for (int i = 0; i < R.npt(); ++i) {
      double f[3];
      fieldfun(&R.x[(size_t)i * dim], i, f);
      const double* v = &T.v[(size_t)i * S.E.n];
      for (int c = 0; c < dim; ++c)
        for (int k = 0; k < S.E.n; ++k) y[c * S.E.n + k] += R.w[i] * f[c] * v[k];
    }
    return y;
  };
  int rank = 0;
  for (int k = nlow2; k < nlow; ++k) {
    auto psi = [&](int i) { return T.v[(size_t)i * S.E.n + k]; };
    if (fam == N1 && dim == 3) {
      for (int m = 0; m < 3; ++m)
        span.push_back(project([&](const double* x, int i, double* f) {
          double e[3] = {0, 0, 0};
          e[m] = psi(i);  // (psi e_m) x x
          f[0] = e[1] * x[2] - e[2] * x[1];
          f[1] = e[2] * x[0] - e[0] * x[2];
          f[2] = e[0] * x[1] - e[1] * x[0];
        }));
    } else if (fam == N1 && dim == 2) {
      span.push_back(project([&](const double* x, int i, double* f) {
        f[0] = -x[1] * psi(i);
        f[1] = x[0] * psi(i);
      }));
    } else if (fam == RT) {
      span.push_back(project([&](const double* x, int i, double* f) {
        for (int c = 0; c < 3; ++c) f[c] = x[c] * psi(i);
      }));
    }
  }
  if (fam == N1 && dim == 3) rank = p * (p + 2) * (p + 3) / 2;
  if (fam == N1 && dim == 2) rank = p * (p + 2);
  if (fam == RT) rank = p * (p + 1) * (p + 3) / 2;
  Mat Sp(N, (int)span.size());
  for (size_t j = 0; j < span.size(); ++j)
    for (int i = 0; i < N; ++i) Sp(i, (int)j) = span[j][i];
  S.U = range_space(Sp, rank, "local space");
  return S;
}

// --- bubbles ---------------------------------------------------------------
int bubble_dim(int fam, int p, int dim) {
  if (fam == CG) return dimP(dim, p - dim - 1);
  if (fam == N1) return dim == 2 ? p * (p - 1) : p * (p + 2) * (p + 3) / 2 - 6 * p - 4 * p * (p - 1);
  if (fam == N2) {
    const int n = 3 * dimP(3, p);
    return dim == 2 ? (p + 1) * (p - 1) : n - 6 * (p + 1) - 4 * (p + 1) * (p - 1);
  }
  if (fam == BDM) return 3 * dimP(3, p) - 4 * dimP(2, p);  // P_p^3 minus the degree-p normal traces
  return p * (p + 1) * (p - 1) / 2;  // RT, 3D
}

int kernel_dim(int fam, int p, int dim) {
  if (fam == CG) return 0;
  if (fam == N1) return dimP(dim, p - dim - 1);  // grad of CG_p bubbles
  if (fam == N2) return dimP(dim, p + 1 - dim - 1);  // grad of CG_{p+1} bubbles
  // RT / BDM bubbles minus their divergences, the mean-free P_{p-1}
  return bubble_dim(fam, p, 3) - (dimP(3, p - 1) - 1);
}

// Columns: L2-orthonormal bubble basis in the space's coefficients.
Mat bubble_basis(const FieldSpace& S, int fam, int p, int dim) {
  const int N = S.ncomp * S.E.n;
  const int bdim = bubble_dim(fam, p, dim);
  if (bdim == 0) return Mat(N, 0);
  if (fam == CG) {  // product of barycentrics times P_{p-dim-1}, orthonormalised
    Rule R = simplex_rule(dim, p + 2);
    Tab T = tabulate_expansion(S.E, 1, R.npt(), R.x.data());
    Expansion Elow(dim, p - dim - 1);
    std::vector<double> lv((size_t)R.npt() * Elow.n);
    Elow.eval(R.npt(), R.x.data(), lv.data(), nullptr);
    Mat Sp(N, Elow.n);
    for (int i = 0; i < R.npt(); ++i) {
      double lam[4];
      bary(dim).lam(&R.x[(size_t)i * dim], lam);
      double b = 1.0;
      for (int j = 0; j <= dim; ++j) b *= lam[j];
      for (int j = 0; j < Elow.n; ++j) {
        const double f = R.w[i] * b * lv[(size_t)i * Elow.n + j];
        for (int k = 0; k < N; ++k) Sp(k, j) += f * T.v[(size_t)i * N + k];
      }
    }
    return range_space(Sp, bdim, "CG bubbles");
  }
  // trace-moment constraints on the boundary (edges in 2D, faces in 3D)
  std::vector<std::vector<double>> rows;
  if (dim == 2) {
    const int mdeg = (fam == N1) ? p - 1 : p;
    Rule G = simplex_rule(1, p + 2);
    Expansion L(1, mdeg);
    std::vector<double> lv((size_t)G.npt() * L.n);
    L.eval(G.npt(), G.x.data(), lv.data(), nullptr);
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b) {
        double t[2] = {0.5 * (TRI[b][0] - TRI[a][0]), 0.5 * (TRI[b][1] - TRI[a][1])};
        std::vector<double> X;
        for (int i = 0; i < G.npt(); ++i)
          for (int c = 0; c < 2; ++c) X.push_back(0.5 * (TRI[a][c] + TRI[b][c]) + G.x[i] * t[c]);
        Tab T = tabulate_expansion(S.E, 2, G.npt(), X.data());
        for (int j = 0; j < L.n; ++j) {
          std::vector<double> row(N, 0.0);
          for (int i = 0; i < G.npt(); ++i) {
            const double f = G.w[i] * lv[(size_t)i * L.n + j];
            for (int c = 0; c < 2; ++c)
              for (int k = 0; k < S.E.n; ++k) row[c * S.E.n + k] += f * t[c] * T.v[(size_t)i * S.E.n + k];
          }
          rows.push_back(row);
        }
      }
  } else {
    Rule F = simplex_rule(2, p + 2);
    Expansion E2(2, p);
    std::vector<double> fv((size_t)F.npt() * E2.n);
    E2.eval(F.npt(), F.x.data(), fv.data(), nullptr);
    Mat Rm(2, 2);
    Rm(0, 0) = TRI[1][0] - TRI[0][0];
    Rm(1, 0) = TRI[1][1] - TRI[0][1];
    Rm(0, 1) = TRI[2][0] - TRI[0][0];
    Rm(1, 1) = TRI[2][1] - TRI[0][1];
    Mat Rinv = inverse(Rm);
    for (int f = 0; f < 4; ++f) {
      const int a = FACES[f][0], b = FACES[f][1], c3 = FACES[f][2];
      double B[3][2], nrm[3];
      for (int c = 0; c < 3; ++c) {
        const double e0 = TET[b][c] - TET[a][c], e1 = TET[c3][c] - TET[a][c];
        B[c][0] = e0 * Rinv(0, 0) + e1 * Rinv(1, 0);
        B[c][1] = e0 * Rinv(0, 1) + e1 * Rinv(1, 1);
      }
      nrm[0] = B[1][0] * B[2][1] - B[2][0] * B[1][1];
      nrm[1] = B[2][0] * B[0][1] - B[0][0] * B[2][1];
      nrm[2] = B[0][0] * B[1][1] - B[1][0] * B[0][1];
      std::vector<double> X;
      for (int i = 0; i < F.npt(); ++i) {
        const double xi0 = F.x[i * 2] - TRI[0][0], xi1 = F.x[i * 2 + 1] - TRI[0][1];
        for (int c = 0; c < 3; ++c) X.push_back(TET[a][c] + B[c][0] * xi0 + B[c][1] * xi1);
      }
      Tab T = tabulate_expansion(S.E, 3, F.npt(), X.data());
      const bool normal = fam == RT || fam == BDM;
      const int nproj = normal ? 1 : 2;
      for (int m = 0; m < nproj; ++m)
        for (int j = 0; j < E2.n; ++j) {
          std::vector<double> row(N, 0.0);
          for (int i = 0; i < F.npt(); ++i) {
            const double f2 = F.w[i] * fv[(size_t)i * E2.n + j];
            for (int c = 0; c < 3; ++c) {
              const double dirc = normal ? nrm[c] : B[c][m];
              for (int k = 0; k < S.E.n; ++k) row[c * S.E.n + k] += f2 * dirc * T.v[(size_t)i * S.E.n + k];
            }
          }
          rows.push_back(row);
        }
    }
  }
  // constraints on the space's coefficients: C = rows * U
  Mat Cx((int)rows.size(), N);
  for (size_t r = 0; r < rows.size(); ++r)
    for (int k = 0; k < N; ++k) Cx((int)r, k) = rows[r][k];
  Mat C = matmul(Cx, S.U);
  Mat Z = null_space(C, bdim, "bubbles");
  return matmul(S.U, Z);
}

// --- probes and canonical eigenbases -----------------------------------------
void probe(int dim, int i, double* pt, double* dir) {
  double b[4], sb = 0.0;
  for (int j = 0; j <= dim; ++j) {
    b[j] = 1.0 + 0.5 * std::sin(1.7 * (i + 1) * (j + 1) + 0.3 * (j + 1) * (j + 1));
    sb += b[j];
  }
  for (int c = 0; c < dim; ++c) {
    pt[c] = 0.0;
    for (int j = 0; j <= dim; ++j) pt[c] += b[j] / sb * vert(dim, j, c);
  }
  double nd = 0.0;
  for (int l = 0; l < dim; ++l) {
    dir[l] = std::cos(0.9 * (i + 1) * (l + 1) + 0.5 * l + 0.25);
    nd += dir[l] * dir[l];
  }
  nd = std::sqrt(nd);
  for (int l = 0; l < dim; ++l) dir[l] /= nd;
}

struct EigenBasis {
  FieldSpace S;
  Mat Y;                    // coefficients of psi_j (columns)
  std::vector<double> lam;  // lambda_j = 1 / mu_j
};

EigenBasis eigenbasis(int fam, int p, int dim) {
  EigenBasis EB;
  EB.S = make_space(fam, p, dim);
  Mat Z = bubble_basis(EB.S, fam, p, dim);
  const int nb = Z.n;
  const int N = EB.S.ncomp * EB.S.E.n;
  if (nb == 0) {
    EB.Y = Mat(N, 0);
    return EB;
  }
  const int dfam = (fam == CG) ? 0 : ((fam == RT || fam == BDM) ? 2 : 1);
  Mat G = d_gram(EB.S.E, EB.S.ncomp, dfam);
  Mat K = matmul_tn(Z, matmul(G, Z));
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < i; ++j) K(i, j) = K(j, i) = 0.5 * (K(i, j) + K(j, i));
  std::vector<double> mu;
  Mat V;
  sym_eig(K, mu, V);
  const int nk = kernel_dim(fam, p, dim);
  const double mumax = mu[nb - 1];
  if (nk > 0 && !(mu[nk - 1] < 1e-9 * mumax)) throw std::runtime_error("eigenbasis: kernel not found");
  if (!(mu[nk] > 1e-7 * mumax)) throw std::runtime_error("eigenbasis: no spectral gap");
  const int ne = nb - nk;
  Mat Y = matmul(Z, cols(V, nk, nb));
  std::vector<double> m(ne);
  for (int j = 0; j < ne; ++j) {
    m[j] = mu[nk + j];
    const double s = 1.0 / std::sqrt(m[j]);
    for (int i = 0; i < N; ++i) Y(i, j) *= s;
  }
  // clusters of (numerically) equal mu, made unique by the echelon rule
  int i0 = 0;
  while (i0 < ne) {
    int i1 = i0 + 1;
    while (i1 < ne && (m[i1] - m[i1 - 1]) <= CLUSTER_RTOL * std::fabs(m[i1])) ++i1;
    const int sz = i1 - i0;
    std::vector<double> pts((size_t)sz * dim), dirs((size_t)sz * dim);
    for (int q = 0; q < sz; ++q) probe(dim, q, &pts[(size_t)q * dim], &dirs[(size_t)q * dim]);
    Tab T = tabulate_expansion(EB.S.E, EB.S.ncomp, sz, pts.data());
    Mat Gm(sz, sz);
    for (int q = 0; q < sz; ++q)
      for (int j = 0; j < sz; ++j) {
        const double* y = &Y.a[0];
        std::vector<double> col(N);
        for (int r = 0; r < N; ++r) col[r] = Y(r, i0 + j);
        double s = 0.0;
        if (EB.S.ncomp == 1)
          s = field_val(T, col.data(), q, 0);
        else
          for (int c = 0; c < EB.S.ncomp; ++c) s += dirs[(size_t)q * dim + c] * field_val(T, col.data(), q, c);
        (void)y;
        Gm(q, j) = s;
      }
    Mat Q;
    std::vector<double> rd;
    qr_square(transpose(Gm), Q, rd);
    Mat Rfull = matmul_tn(Q, transpose(Gm));  // = R (upper triangular)
    double gmax = 0.0;
    for (double x : Gm.a) gmax = std::max(gmax, std::fabs(x));
    for (int j = 0; j < sz; ++j) {
      if (!(std::fabs(Rfull(j, j)) > 1e-8 * gmax)) throw std::runtime_error("eigenbasis: singular probe matrix");
      if (Rfull(j, j) < 0)
        for (int r = 0; r < sz; ++r) Q(r, j) = -Q(r, j);
    }
    Mat Yc = matmul(cols(Y, i0, i1), Q);
    for (int r = 0; r < N; ++r)
      for (int j = 0; j < sz; ++j) Y(r, i0 + j) = Yc(r, j);
    i0 = i1;
  }
  EB.Y = Y;
  EB.lam.resize(ne);
  for (int j = 0; j < ne; ++j) EB.lam[j] = 1.0 / m[j];
  return EB;
}

// cache of eigenbases
// Build-once cache: the global lock only guards the map; each entry is built
// under its own once-flag, so different keys build concurrently and a build
// may look up other keys.
template <typename K, typename V>
struct OnceCache {
  struct Entry {
    std::once_flag once;
    std::shared_ptr<V> val;
  };
  std::mutex mu;
  std::map<K, std::shared_ptr<Entry>> m;
  template <typename F>
  const V& get(const K& k, F&& make) {
    std::shared_ptr<Entry> e;
    {
      std::lock_guard<std::mutex> lk(mu);
      auto& slot = m[k];
      if (!slot) slot = std::make_shared<Entry>();
      e = slot;
    }
    std::call_once(e->once, [&] { e->val = make(); });
    return *e->val;
  }
};

OnceCache<std::tuple<int, int, int>, EigenBasis> g_eig;

const EigenBasis& eig_cached(int fam, int p, int dim) {
  return g_eig.get(std::make_tuple(fam, p, dim),
                   [&] { return std::make_shared<EigenBasis>(eigenbasis(fam, p, dim)); });
}

// Tabulate an eigenbasis at points: values (npt x ne x ncomp), d (npt x ne x nd)
void eig_tab(const EigenBasis& EB, int dfam, int npt, const double* x, std::vector<double>& val,
             std::vector<double>& dv, int& nd) {
  const int dim = EB.S.E.dim, nc = EB.S.ncomp, ne = EB.Y.n, nE = EB.S.E.n;
  Tab T = tabulate_expansion(EB.S.E, nc, npt, x);
  val.assign((size_t)npt * ne * nc, 0.0);
  nd = (dfam == 0) ? dim : ((dfam == 1 && dim == 3) ? 3 : 1);
  dv.assign((size_t)npt * ne * nd, 0.0);
  double D[3];
  int ndo;
  for (int i = 0; i < npt; ++i)
    for (int c = 0; c < nc; ++c)
      for (int k = 0; k < nE; ++k) {
        const double vk = T.v[(size_t)i * nE + k];
        d_of_basis(T, dfam, i, c, k, D, ndo);
        for (int j = 0; j < ne; ++j) {
          const double y = EB.Y(c * nE + k, j);
          if (y == 0.0) continue;
          val[((size_t)i * ne + j) * nc + c] += vk * y;
          for (int d = 0; d < nd; ++d) dv[((size_t)i * ne + j) * nd + d] += D[d] * y;
        }
      }
}

}  // namespace

// ---------------------------------------------------------------------------
// the reference element
// ---------------------------------------------------------------------------
// kind 1: CG_p, Ned1_p, RT_p (Eq. (2.5)); kind 2: NedTwo_p, BDM_p (Eq. (2.6)).  The H(curl) gradient
// moments use the CG eigenbasis of degree p0 (p, or p + 1 for NedTwo_p: its X^0 is CG_{p+1}); the H(div)
// face and curl moments use the NedTwo eigenbasis of degree p1 (p, or p + 1 for BDM_p), Section 3.4.
static void build_element(RefElement& R, int space, int p, int kind) {
  R.space = space;
  R.p = p;
  R.kind = kind;
  const bool second = kind == 2 && space != H1;
  const int fam = space == H1 ? CG : (space == HCURL ? (second ? N2 : N1) : (second ? BDM : RT));
  const int p0 = (space == HCURL && second) ? p + 1 : p;
  const int p1 = (space == HDIV && second) ? p + 1 : p;
  FieldSpace S = make_space(fam, p, 3);
  R.E = S.E;
  R.ncomp = S.ncomp;
  R.dcomp = (space == HDIV) ? 1 : 3;
  const int N = S.ncomp * S.E.n;
  std::vector<std::vector<double>> L;  // functionals on expansion coefficients
  int counts[4] = {0, 0, 0, 0};
  auto add_rows = [&](int dimkey, const Mat& rows) {
    for (int r = 0; r < rows.m; ++r) {
      std::vector<double> row(rows.n);
      for (int k = 0; k < rows.n; ++k) row[k] = rows(r, k);
      L.push_back(row);
    }
    counts[dimkey] += rows.m;
  };
  Rule G = simplex_rule(1, p + 2), F = simplex_rule(2, p + 2), C = simplex_rule(3, p + 2);
  // ----- vertices (H1 only): point evaluation
  if (space == H1) {
    for (int a = 0; a < 4; ++a) {
      Tab T = tabulate_expansion(S.E, 1, 1, TET[a]);
      Mat row(1, N);
      for (int k = 0; k < N; ++k) row(0, k) = T.v[k];
      add_rows(0, row);
    }
  }
  // ----- edges
  if (space != HDIV) {
    const EigenBasis& EE = eig_cached(CG, space == HCURL ? p0 : p, 1);
    std::vector<double> ev, ed;
    int nd;
    eig_tab(EE, 0, G.npt(), G.x.data(), ev, ed, nd);
    const int ne = EE.Y.n;
    for (int e = 0; e < 6; ++e) {
      const int a = EDGES[e][0], b = EDGES[e][1];
      double t[3], X[64 * 3];
      for (int c = 0; c < 3; ++c) t[c] = 0.5 * (TET[b][c] - TET[a][c]);
      std::vector<double> Xv;
      for (int i = 0; i < G.npt(); ++i)
        for (int c = 0; c < 3; ++c) Xv.push_back(0.5 * (TET[a][c] + TET[b][c]) + G.x[i] * t[c]);
      (void)X;
      Tab T = tabulate_expansion(S.E, S.ncomp, G.npt(), Xv.data());
      const int nE = S.E.n;
      if (space == H1) {  // (d psi/ds, t . grad v)
        Mat rows(ne, N);
        for (int i = 0; i < G.npt(); ++i)
          for (int k = 0; k < nE; ++k) {
            double tg = 0.0;
            for (int c = 0; c < 3; ++c) tg += t[c] * T.g[((size_t)i * nE + k) * 3 + c];
            for (int j = 0; j < ne; ++j) rows(j, k) += G.w[i] * ed[(size_t)i * ne + j] * tg;
          }
        add_rows(1, rows);
      } else {  // Whitney (1, t.v) then type II (d psi/ds, t.v)
        Mat rows(1 + ne, N);
        for (int i = 0; i < G.npt(); ++i)
          for (int c = 0; c < 3; ++c)
            for (int k = 0; k < nE; ++k) {
              const double tv = t[c] * T.v[(size_t)i * nE + k];
              rows(0, c * nE + k) += G.w[i] * tv;
              for (int j = 0; j < ne; ++j) rows(1 + j, c * nE + k) += G.w[i] * ed[(size_t)i * ne + j] * tv;
            }
        add_rows(1, rows);
      }
    }
  }
  // ----- faces
  {
    Mat Rm(2, 2);
    Rm(0, 0) = TRI[1][0] - TRI[0][0];
    Rm(1, 0) = TRI[1][1] - TRI[0][1];
    Rm(0, 1) = TRI[2][0] - TRI[0][0];
    Rm(1, 1) = TRI[2][1] - TRI[0][1];
    Mat Rinv = inverse(Rm);
    std::vector<double> av, ad, bv, bd;
    int nda = 0, ndb = 0, na = 0, nb = 0;
    if (space == H1) {
      const EigenBasis& A = eig_cached(CG, p, 2);
      eig_tab(A, 0, F.npt(), F.x.data(), av, ad, nda);
      na = A.Y.n;
    } else if (space == HCURL) {
      const EigenBasis& A = eig_cached(fam, p, 2);
      eig_tab(A, 1, F.npt(), F.x.data(), av, ad, nda);
      na = A.Y.n;
      const EigenBasis& B = eig_cached(CG, p0, 2);
      eig_tab(B, 0, F.npt(), F.x.data(), bv, bd, ndb);
      nb = B.Y.n;
    } else {
      const EigenBasis& A = eig_cached(N2, p1, 2);
      eig_tab(A, 1, F.npt(), F.x.data(), av, ad, nda);
      na = A.Y.n;
    }
    const int nE = S.E.n;
    for (int f = 0; f < 4; ++f) {
      const int a = FACES[f][0], b = FACES[f][1], c3 = FACES[f][2];
      double B[3][2], nrm[3];
      for (int c = 0; c < 3; ++c) {
        const double e0 = TET[b][c] - TET[a][c], e1 = TET[c3][c] - TET[a][c];
        B[c][0] = e0 * Rinv(0, 0) + e1 * Rinv(1, 0);
        B[c][1] = e0 * Rinv(0, 1) + e1 * Rinv(1, 1);
      }
      nrm[0] = B[1][0] * B[2][1] - B[2][0] * B[1][1];
      nrm[1] = B[2][0] * B[0][1] - B[0][0] * B[2][1];
      nrm[2] = B[0][0] * B[1][1] - B[1][0] * B[0][1];
      std::vector<double> Xv;
      for (int i = 0; i < F.npt(); ++i) {
        const double xi0 = F.x[i * 2] - TRI[0][0], xi1 = F.x[i * 2 + 1] - TRI[0][1];
        for (int c = 0; c < 3; ++c) Xv.push_back(TET[a][c] + B[c][0] * xi0 + B[c][1] * xi1);
      }
      Tab T = tabulate_expansion(S.E, S.ncomp, F.npt(), Xv.data());
      if (space == H1) {  // (grad_F psi, B^T grad v)
        Mat rows(na, N);
        for (int i = 0; i < F.npt(); ++i)
          for (int k = 0; k < nE; ++k) {
            const double* g = &T.g[((size_t)i * nE + k) * 3];
            const double tg0 = B[0][0] * g[0] + B[1][0] * g[1] + B[2][0] * g[2];
            const double tg1 = B[0][1] * g[0] + B[1][1] * g[1] + B[2][1] * g[2];
            for (int j = 0; j < na; ++j)
              rows(j, k) += F.w[i] * (ad[((size_t)i * na + j) * 2] * tg0 + ad[((size_t)i * na + j) * 2 + 1] * tg1);
          }
        add_rows(2, rows);
      } else if (space == HCURL) {  // type I (curl_F Psi, n.curl v); type II (grad_F psi, B^T v)
        Mat rows(na + nb, N);
        for (int i = 0; i < F.npt(); ++i)
          for (int c = 0; c < 3; ++c)
            for (int k = 0; k < nE; ++k) {
              const double* g = &T.g[((size_t)i * nE + k) * 3];
              // n . curl(psi e_c) = n . (grad psi x e_c)
              double e[3] = {0, 0, 0};
              e[c] = 1.0;
              const double cr[3] = {g[1] * e[2] - g[2] * e[1], g[2] * e[0] - g[0] * e[2], g[0] * e[1] - g[1] * e[0]};
              const double nc = nrm[0] * cr[0] + nrm[1] * cr[1] + nrm[2] * cr[2];
              const double vk = T.v[(size_t)i * nE + k];
              for (int j = 0; j < na; ++j) rows(j, c * nE + k) += F.w[i] * ad[(size_t)i * na + j] * nc;
              for (int j = 0; j < nb; ++j)
                rows(na + j, c * nE + k) +=
                    F.w[i] * (bd[((size_t)i * nb + j) * 2] * B[c][0] + bd[((size_t)i * nb + j) * 2 + 1] * B[c][1]) * vk;
            }
        add_rows(2, rows);
      } else {  // Whitney (1, n.v); type II (curl_F Psi, n.v)
        Mat rows(1 + na, N);
        for (int i = 0; i < F.npt(); ++i)
          for (int c = 0; c < 3; ++c)
            for (int k = 0; k < nE; ++k) {
              const double nv = nrm[c] * T.v[(size_t)i * nE + k];
              rows(0, c * nE + k) += F.w[i] * nv;
              for (int j = 0; j < na; ++j) rows(1 + j, c * nE + k) += F.w[i] * ad[(size_t)i * na + j] * nv;
            }
        add_rows(2, rows);
      }
    }
  }
  // ----- interior
  {
    Tab T = tabulate_expansion(S.E, S.ncomp, C.npt(), C.x.data());
    const int nE = S.E.n;
    std::vector<double> v1, d1, v2, d2;
    int nd1 = 0, nd2 = 0, n1 = 0, n2 = 0;
    if (space == H1) {
      const EigenBasis& A = eig_cached(CG, p, 3);
      n1 = A.Y.n;
      if (n1) eig_tab(A, 0, C.npt(), C.x.data(), v1, d1, nd1);
    } else if (space == HCURL) {
      const EigenBasis& A = eig_cached(fam, p, 3);
      n1 = A.Y.n;
      if (n1) eig_tab(A, 1, C.npt(), C.x.data(), v1, d1, nd1);
      const EigenBasis& B = eig_cached(CG, p0, 3);
      n2 = B.Y.n;
      if (n2) eig_tab(B, 0, C.npt(), C.x.data(), v2, d2, nd2);
    } else {
      const EigenBasis& A = eig_cached(fam, p, 3);
      n1 = A.Y.n;
      if (n1) eig_tab(A, 2, C.npt(), C.x.data(), v1, d1, nd1);
      const EigenBasis& B = eig_cached(N2, p1, 3);
      n2 = B.Y.n;
      if (n2) eig_tab(B, 1, C.npt(), C.x.data(), v2, d2, nd2);
    }
    Mat rows(n1 + n2, N);
    const int dfam = space == H1 ? 0 : (space == HCURL ? 1 : 2);
    double D[3];
    int nd;
    for (int i = 0; i < C.npt(); ++i)
      for (int c = 0; c < S.ncomp; ++c)
        for (int k = 0; k < nE; ++k) {
          d_of_basis(T, dfam, i, c, k, D, nd);
          const double vk = T.v[(size_t)i * nE + k];
          for (int j = 0; j < n1; ++j) {  // type I: (d psi, d v)
            double s = 0.0;
            for (int d = 0; d < nd; ++d) s += d1[((size_t)i * n1 + j) * nd1 + d] * D[d];
            rows(j, c * nE + k) += C.w[i] * s;
          }
          for (int j = 0; j < n2; ++j)  // type II: (d psi^{k-1}, v)
            rows(n1 + j, c * nE + k) += C.w[i] * d2[((size_t)i * n2 + j) * nd2 + c] * vk;
        }
    add_rows(3, rows);
    R.ninterior = n1 + n2;
  }
  const int nref = (int)L.size();
  if (nref != S.U.n) throw std::runtime_error("reference element: DOF count mismatch");
  R.nref = nref;
  R.per_entity[0] = counts[0] / 4;
  R.per_entity[1] = counts[1] / 6;
  R.per_entity[2] = counts[2] / 4;
  R.per_entity[3] = counts[3];
  Mat Lm(nref, N);
  for (int i = 0; i < nref; ++i)
    for (int k = 0; k < N; ++k) Lm(i, k) = L[i][k];
  Mat D = matmul(Lm, S.U);
  Mat Dinv = inverse(D, &R.dof_cond);
  R.Phi = matmul(S.U, Dinv);

  // ----- reference matrices for the device contraction
  Rule Q = simplex_rule(3, p + 2);
  std::vector<double> v((size_t)Q.npt() * nref * R.ncomp), d((size_t)Q.npt() * nref * R.dcomp);
  R.tabulate(Q.npt(), Q.x.data(), v.data(), d.data());
  const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
  auto component = [&](const std::vector<double>& t, int nc, int a) {  // [q][i] = t_i^a(x_q)
    Mat T(Q.npt(), nref);
    for (int q = 0; q < Q.npt(); ++q)
      for (int i = 0; i < nref; ++i) T(q, i) = t[((size_t)q * nref + i) * nc + a];
    return T;
  };
  auto comp_matrix = [&](const std::vector<double>& t, int nc, int a, int b, double* out) {
    // out[i][j] = sum_q w t_i^a t_j^b (+ the transposed term when a != b)
    const Mat Ta = component(t, nc, a);
    if (a == b) {
      const Mat G = gram_tn(Ta, Q.w, Ta);
      std::copy(G.a.begin(), G.a.end(), out);
    } else {
      const Mat G = gram_tn(Ta, Q.w, component(t, nc, b));
      for (int i = 0; i < nref; ++i)
        for (int j = 0; j < nref; ++j) out[(size_t)i * nref + j] = G(i, j) + G(j, i);
    }
  };
  const size_t nn = (size_t)nref * nref;
  if (space == H1) {
    R.Q = 7;
    R.R.assign(7 * nn, 0.0);
    comp_matrix(v, 1, 0, 0, &R.R[0]);
    for (int q = 0; q < 6; ++q) comp_matrix(d, 3, pairs[q][0], pairs[q][1], &R.R[(1 + q) * nn]);
  } else if (space == HCURL) {
    R.Q = 12;
    R.R.assign(12 * nn, 0.0);
    for (int q = 0; q < 6; ++q) comp_matrix(v, 3, pairs[q][0], pairs[q][1], &R.R[q * nn]);
    for (int q = 0; q < 6; ++q) comp_matrix(d, 3, pairs[q][0], pairs[q][1], &R.R[(6 + q) * nn]);
  } else {
    R.Q = 7;
    R.R.assign(7 * nn, 0.0);
    for (int q = 0; q < 6; ++q) comp_matrix(v, 3, pairs[q][0], pairs[q][1], &R.R[q * nn]);
    comp_matrix(d, 1, 0, 0, &R.R[6 * nn]);
  }
}

void RefElement::tabulate(int npt, const double* x, double* vals, double* dvals) const {
  Tab T = tabulate_expansion(E, ncomp, npt, x);
  const int nE = E.n;
  const int dfam = space == H1 ? 0 : (space == HCURL ? 1 : 2);
  parallel_for(npt, [&](int i) {
    double D[3];
    int nd;
    if (vals) std::fill(vals + (size_t)i * nref * ncomp, vals + (size_t)(i + 1) * nref * ncomp, 0.0);
    if (dvals) std::fill(dvals + (size_t)i * nref * dcomp, dvals + (size_t)(i + 1) * nref * dcomp, 0.0);
    for (int c = 0; c < ncomp; ++c)
      for (int k = 0; k < nE; ++k) {
        const double vk = T.v[(size_t)i * nE + k];
        d_of_basis(T, dfam, i, c, k, D, nd);
        const double* ph = &Phi.a[(size_t)(c * nE + k) * nref];
        for (int j = 0; j < nref; ++j) {
          const double y = ph[j];
          if (vals) vals[((size_t)i * nref + j) * ncomp + c] += vk * y;
          if (dvals)
            for (int dd = 0; dd < nd; ++dd) dvals[((size_t)i * nref + j) * dcomp + dd] += D[dd] * y;
        }
      }
  });
}

static void build_cross(RefElement& R, const RefElement& cg) {
  Rule Q = simplex_rule(3, R.p + 2);
  std::vector<double> v((size_t)Q.npt() * R.nref * R.ncomp), c((size_t)Q.npt() * cg.nref);
  R.tabulate(Q.npt(), Q.x.data(), v.data(), nullptr);
  cg.tabulate(Q.npt(), Q.x.data(), c.data(), nullptr);
  R.ncg = cg.nref;
  R.Xcross.assign((size_t)R.ncomp * cg.nref * R.nref, 0.0);
  // Xcross[l][a][i] = sum_q w_q c_a(x_q) v_i^l(x_q)
  Mat Cm(Q.npt(), cg.nref), Vl(Q.npt(), R.nref);
  for (int q = 0; q < Q.npt(); ++q)
    for (int a = 0; a < cg.nref; ++a) Cm(q, a) = c[(size_t)q * cg.nref + a];
  for (int l = 0; l < R.ncomp; ++l) {
    for (int q = 0; q < Q.npt(); ++q)
      for (int i = 0; i < R.nref; ++i) Vl(q, i) = v[((size_t)q * R.nref + i) * R.ncomp + l];
    const Mat X = gram_tn(Cm, Q.w, Vl);
    std::copy(X.a.begin(), X.a.end(), R.Xcross.begin() + (size_t)l * cg.nref * R.nref);
  }
}

const RefElement& reference_element(int space, int p, int kind) {
  static OnceCache<std::tuple<int, int, int>, RefElement> cache;
  if (p < 1 || p > 12 || space < 0 || space > 2 || kind < 1 || kind > 2)
    throw std::runtime_error("reference_element: unsupported (space, p, kind)");
  if (space == H1) kind = 1;  // CG_p is both kinds
  return cache.get(std::make_tuple(space, p, kind), [&] {
    auto R = std::make_shared<RefElement>();
    build_element(*R, space, p, kind);
    const RefElement& cg = (space == H1) ? *R : reference_element(H1, p);
    build_cross(*R, cg);
    return R;
  });
}

int dg_dim(int p) { return p * (p + 1) * (p + 2) / 6; }

void dg_tabulate(int p, int npt, const double* x, double* vals) {
  const EigenBasis& A = eig_cached(RT, p, 3);
  const int n1 = A.Y.n, n = 1 + n1;
  if (n != dg_dim(p)) throw std::runtime_error("DG basis: dimension mismatch");
  double E[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) E[r][c] = vert(3, r + 1, c) - vert(3, 0, c);
  const double det = E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) - E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                     E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
  const double vol = std::fabs(det) / 6.0;
  std::vector<double> v1, d1;
  int nd1 = 0;
  if (n1) eig_tab(A, 2, npt, x, v1, d1, nd1);
  for (int i = 0; i < npt; ++i) {
    vals[(size_t)i * n] = 1.0 / vol;  // dual to the mean (1, v)_T
    for (int j = 0; j < n1; ++j) vals[(size_t)i * n + 1 + j] = d1[(size_t)i * n1 + j];  // div Phi_{C,j}
  }
}

const std::vector<double>& mixed_reference_tables(int k, int p) {
  static OnceCache<std::pair<int, int>, std::vector<double>> cache;
  if (k < 1 || k > 3) throw std::runtime_error("mixed_reference_tables: k must be 1, 2 or 3");
  if (k == 3)
    return cache.get(std::make_pair(k, p), [&] {
      const RefElement& R0 = reference_element(HDIV, p);
      const int n0 = R0.nref, n1 = dg_dim(p);
      Rule Q = simplex_rule(3, p + 2);
      const int np = Q.npt();
      std::vector<double> d0((size_t)np * n0), v1((size_t)np * n1);
      R0.tabulate(np, Q.x.data(), nullptr, d0.data());
      dg_tabulate(p, np, Q.x.data(), v1.data());
      Mat D(np, n0), V(np, n1);
      for (int q = 0; q < np; ++q) {
        for (int j = 0; j < n0; ++j) D(q, j) = d0[(size_t)q * n0 + j];
        for (int i = 0; i < n1; ++i) V(q, i) = v1[(size_t)q * n1 + i];
      }
      const Mat G = gram_tn(D, Q.w, V);  // [j][i] = sum w div phi^RT_j psi^DG_i
      return std::make_shared<std::vector<double>>(G.a);
    });
  return cache.get(std::make_pair(k, p), [&] {
    const RefElement& R0 = reference_element(k - 1, p);  // X^{k-1}: CG_p or Ned1_p
    const RefElement& R1 = reference_element(k, p);      // X^k: Ned1_p or RT_p
    const int n0 = R0.nref, n1 = R1.nref;
    Rule Q = simplex_rule(3, p + 2);
    const int np = Q.npt();
    std::vector<double> v1((size_t)np * n1 * 3), d0((size_t)np * n0 * 3);
    R1.tabulate(np, Q.x.data(), v1.data(), nullptr);
    R0.tabulate(np, Q.x.data(), nullptr, d0.data());
    auto comp = [&](const std::vector<double>& t, int n, int a) {  // [q][i] = t_i^a(x_q)
      Mat T(np, n);
      for (int q = 0; q < np; ++q)
        for (int i = 0; i < n; ++i) T(q, i) = t[((size_t)q * n + i) * 3 + a];
      return T;
    };
    const int pairs[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
    auto out = std::make_shared<std::vector<double>>((size_t)6 * n0 * n1, 0.0);
    for (int q = 0; q < 6; ++q) {
      const int a = pairs[q][0], b = pairs[q][1];
      const Mat G = gram_tn(comp(d0, n0, b), Q.w, comp(v1, n1, a));  // [j][i] = sum w (d phi0_j)_b (phi1_i)_a
      const Mat H = (a == b) ? Mat() : gram_tn(comp(d0, n0, a), Q.w, comp(v1, n1, b));
      double* o = out->data() + (size_t)q * n0 * n1;
      for (int j = 0; j < n0; ++j)
        for (int i = 0; i < n1; ++i) o[(size_t)j * n1 + i] = G(j, i) + (a == b ? 0.0 : H(j, i));
    }
    return out;
  });
}

}  // namespace riesz
