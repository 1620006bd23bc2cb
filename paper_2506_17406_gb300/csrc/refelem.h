// Host FP64 builder of the paper's orthogonality-promoting reference element
// (arXiv 2506.17406, Sections 3-4) and of the reference tables the device
// kernels contract against.
#pragma once
#include <vector>

#include "linalg.h"

namespace riesz {

enum Space { H1 = 0, HCURL = 1, HDIV = 2 };

// Orthonormal (Dubiner / PKD) polynomial expansion of total degree <= deg on
// the equilateral reference simplex of dimension dim (edge length 2).
struct Expansion {
  int dim = 0, deg = 0, n = 0;
  std::vector<double> norm;  // normalisation of each raw PKD function
  std::vector<int> order;    // (p, q, r) triples flattened
  Expansion() {}
  Expansion(int dim, int deg);
  // values[npt][n], grads[npt][n][dim]
  void eval(int npt, const double* x, double* values, double* grads) const;
};

struct Rule {  // quadrature on a reference simplex
  int dim = 0;
  std::vector<double> x, w;  // x: npt*dim
  int npt() const { return (int)w.size(); }
};
Rule simplex_rule(int dim, int npts_per_dir);

// A reference element: the dual basis of the paper's DOFs and its tables.
struct RefElement {
  int space = 0, p = 0, nref = 0, ninterior = 0;
  int kind = 1;                      // 1: first kind (Eq. (2.5)), 2: second kind (Eq. (2.6))
  int ncomp = 1, dcomp = 3;  // value / exterior-derivative components
  int per_entity[4] = {0, 0, 0, 0};  // DOFs per vertex, edge, face, interior
  Expansion E;                       // expansion (scalar for H1, vector otherwise)
  Mat Phi;                           // (ncomp * E.n) x nref coefficients
  double dof_cond = 0.0;
  // Reference matrices R_q (Q x nref x nref), see geometric_factor_kind below.
  int Q = 0;
  std::vector<double> R;
  // Cross tables for the right-hand side of an [CG_p]^3 (or CG_p) source:
  // X[l][a][i] = int phi^CG_a v_i^l (l < ncomp), a < ncg.
  int ncg = 0;
  std::vector<double> Xcross;
  // tabulate values (npt x nref x ncomp) and d (npt x nref x dcomp) at points
  void tabulate(int npt, const double* x, double* vals, double* dvals) const;
};

// Cached per (space, p, kind).  space H1, HCURL or HDIV; kind 1 gives CG_p, Ned1_p, RT_p
// (Eq. (2.5)), kind 2 NedTwo_p and BDM_p (Eq. (2.6); CG_p for H1).  Throws std::runtime_error on failure.
const RefElement& reference_element(int space, int p, int kind = 1);

// Reference tables of the coupling (d phi^{k-1}_j, phi^k_i) of the Hodge-Laplace
// problem (k = 1: CG_p -> Ned1_p, k = 2: Ned1_p -> RT_p): 6 matrices [j][i]
// (n_{k-1} x n_k), one per symmetric metric entry (00, 11, 22, 01, 02, 12), the
// off-diagonal ones holding both orderings; contracted against the X^k mass
// factors of a cell (|det J| J^{-1}J^{-T} for k = 1, J^T J / |det J| for k = 2).
// k = 3 (RT_p -> DG_{p-1}): one matrix [j][i] (n_RT x n_DG) of
// (div phi^RT_j, psi^DG_i), contracted with the single factor 1 / |det J|.
const std::vector<double>& mixed_reference_tables(int k, int p);

// X^3 = DG_{p-1} of the complex ending in RT_p: the dual basis of the paper's
// cell DOFs at k = d, (1, v)_T and (div Phi_{C,j}, v)_T with Phi the RT_p
// interior type-I eigenbasis normalised by (div Phi_i, div Phi_j) = delta_ij;
// it is {1 / |T|} followed by {div Phi_{C,j}}, L2-orthogonal.
int dg_dim(int p);
void dg_tabulate(int p, int npt, const double* x, double* vals);  // vals [npt][dg_dim(p)]

}  // namespace riesz
