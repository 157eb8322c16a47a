// Host-side finite element model: quadrature rules on the reference
// tetrahedron, the equispaced Lagrange basis, and the tables that the device
// kernels read (basis values and reference gradients at quadrature points,
// pre-evaluated reference tensors of Algorithm 2).
#pragma once
#include <cstdint>
#include <vector>

namespace fea {

enum Form { MASS = 0, HELMHOLTZ = 1, ELASTICITY = 2, NEOHOOKEAN = 3 };

inline int nbasis(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }
inline bool vector_form(int form) { return form == ELASTICITY || form == NEOHOOKEAN; }
inline int local_dim(int form, int p) { return vector_form(form) ? 3 * nbasis(p) : nbasis(p); }
int coeff_len(int form, int p);

// Rule index used for a form and degree: 0 = the 4-point degree-2 rule,
// m >= 1 = collapsed Gauss-Jacobi rule with m^3 points (exact to degree 2m-1).
int rule_index(int form, int p);
inline int rule_points(int m) { return m == 0 ? 4 : m * m * m; }

struct Rule {
  int Q = 0;
  std::vector<double> X;  // [Q][3]
  std::vector<double> W;  // [Q]
};
Rule make_rule(int m);

// Lagrange basis of degree p as coefficients over the monomials x^a y^b z^c,
// a+b+c <= p, obtained by inverting the Vandermonde matrix at the nodes.
struct Basis {
  int p = 0, n = 0;
  std::vector<int> mono;      // [n][3] exponents
  std::vector<double> nodes;  // [n][3]
  std::vector<double> coef;   // [n][n]: phi_i = sum_m coef[i][m] X^mono[m]
  void eval(const double* X, double* phi, double* dphi) const;  // phi[n], dphi[n][3]
};
Basis make_basis(int p);

// Number of pre-evaluated reference tensors r and whether the form admits
// pre-evaluation (its integrand is a polynomial in reference coordinates).
int pre_terms(int form, int p);

// Tables of one (form, degree): all in FP64, converted by the caller.
struct Tables {
  int form = 0, p = 0, ns = 0, Q = 0, r = 0;
  std::vector<double> W;      // [Q]
  std::vector<double> phi;    // [Q][ns]
  std::vector<double> dphi;   // [Q][ns][3]
  std::vector<double> phi1;   // [Q][4] P1 basis (elasticity coefficients)
  std::vector<double> R;      // [r][ns][ns] pre-evaluated reference tensors
};
Tables make_tables(int form, int p);

}  // namespace fea
