// Host-side finite element model (see host_model.h).
//
// Quadrature: Golub-Welsch -- the nodes of a Gauss-Jacobi rule are the
// eigenvalues of the symmetric tridiagonal Jacobi matrix of the orthogonal
// polynomials, the weights are mu_0 times the squared first components of the
// normalised eigenvectors.  The eigenproblem is solved with cyclic Jacobi
// rotations.  The collapsed (conical-product) rule maps [0,1]^3 onto the
// reference tetrahedron: X = (t(1-s)(1-r), s(1-r), r), with weight (1-r)^2
// (Gauss-Jacobi alpha=2), (1-s) (alpha=1) and 1 (Gauss-Legendre).
//
// Basis: equispaced Lagrange nodes; the coefficients over monomials come from
// inverting the Vandermonde matrix with Gauss-Jordan elimination.
#include "host_model.h"

#include <cmath>
#include <stdexcept>

namespace fea {

int coeff_len(int form, int p) {
  switch (form) {
    case MASS: return 0;
    case HELMHOLTZ: return nbasis(p);
    case ELASTICITY: return 8;
    case NEOHOOKEAN: return 3 * nbasis(p);
  }
  return -1;
}

int rule_index(int form, int p) {
  switch (form) {
    case MASS: return p == 1 ? 0 : p + 1;        // integrand degree 2p
    case HELMHOLTZ: return (3 * p + 2) / 2;      // degree 3p: m = ceil((3p+1)/2)
    case ELASTICITY: return p;                   // degree 2(p-1) + 1
    case NEOHOOKEAN: return p + 1;               // not polynomial: one point more than P_p
  }
  return -1;
}

// Symmetric eigenproblem by cyclic Jacobi rotations: A (n x n, row-major) is
// overwritten; on return its diagonal holds the eigenvalues and V's columns
// the eigenvectors.
static void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-60) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A G (columns p, q)
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- G^T A (rows p, q)
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b on [-1,1] by Golub-Welsch.
static void golub_welsch(int m, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> T(m * m, 0.0), V;
  for (int k = 0; k < m; ++k) {
    double s = 2.0 * k + a + b;
    T[k * m + k] = (k == 0 && std::fabs(a + b) < 1e-300) ? (b - a) / (a + b + 2.0)
                                                          : (b * b - a * a) / (s * (s + 2.0));
    if (k + 1 < m) {
      double j = k + 1, sj = 2.0 * j + a + b;
      double beta = 4.0 * j * (j + a) * (j + b) * (j + a + b) / (sj * sj * (sj + 1.0) * (sj - 1.0));
      T[k * m + k + 1] = T[(k + 1) * m + k] = std::sqrt(beta);
    }
  }
  jacobi_eigen(m, T, V);
  double mu0 = std::pow(2.0, a + b + 1.0) * std::tgamma(a + 1.0) * std::tgamma(b + 1.0) / std::tgamma(a + b + 2.0);
  std::vector<std::pair<double, double>> nw(m);
  for (int k = 0; k < m; ++k) nw[k] = {T[k * m + k], mu0 * V[k] * V[k]};  // V[0][k]
  for (int i = 1; i < m; ++i)  // sort ascending
    for (int j = i; j > 0 && nw[j].first < nw[j - 1].first; --j) std::swap(nw[j], nw[j - 1]);
  x.resize(m);
  w.resize(m);
  for (int k = 0; k < m; ++k) {
    x[k] = nw[k].first;
    w[k] = nw[k].second;
  }
}

Rule make_rule(int m) {
  Rule r;
  if (m == 0) {  // 4-point rule: barycentric (a, b, b, b) and permutations
    const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
    r.Q = 4;
    for (int k = 0; k < 4; ++k) {
      double l[4] = {b, b, b, b};
      l[k] = a;
      r.X.push_back(l[1]);
      r.X.push_back(l[2]);
      r.X.push_back(l[3]);
      r.W.push_back(1.0 / 24.0);
    }
    return r;
  }
  if (m < 1 || m > 16) throw std::invalid_argument("rule index");
  std::vector<double> xr, wr, xs, ws, xt, wt;
  golub_welsch(m, 2.0, 0.0, xr, wr);
  golub_welsch(m, 1.0, 0.0, xs, ws);
  golub_welsch(m, 0.0, 0.0, xt, wt);
  r.Q = m * m * m;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < m; ++k) {
        double R = 0.5 * (1.0 + xr[i]), S = 0.5 * (1.0 + xs[j]), T = 0.5 * (1.0 + xt[k]);
        r.X.push_back(T * (1.0 - S) * (1.0 - R));
        r.X.push_back(S * (1.0 - R));
        r.X.push_back(R);
        r.W.push_back(wr[i] / 8.0 * ws[j] / 4.0 * wt[k] / 2.0);
      }
  return r;
}

// Barycentric indices of the P_p nodes in DOF order.
static std::vector<int> node_multi_indices(int p) {
  std::vector<int> out;
  auto push = [&](int b0, int b1, int b2, int b3) {
    out.push_back(b0); out.push_back(b1); out.push_back(b2); out.push_back(b3);
  };
  for (int v = 0; v < 4; ++v) {
    int b[4] = {0, 0, 0, 0};
    b[v] = p;
    push(b[0], b[1], b[2], b[3]);
  }
  const int edge[6][2] = {{2, 3}, {1, 3}, {1, 2}, {0, 3}, {0, 2}, {0, 1}};
  for (auto& e : edge)
    for (int m = 1; m < p; ++m) {
      int b[4] = {0, 0, 0, 0};
      b[e[0]] = p - m;
      b[e[1]] = m;
      push(b[0], b[1], b[2], b[3]);
    }
  for (int v = 0; v < 4; ++v) {
    int f[3], k = 0;
    for (int c = 0; c < 4; ++c)
      if (c != v) f[k++] = c;
    for (int i2 = 1; i2 < p; ++i2)      // last face vertex slowest
      for (int i1 = 1; i1 < p; ++i1) {
        int i0 = p - i1 - i2;
        if (i0 < 1) continue;
        int b[4] = {0, 0, 0, 0};
        b[f[0]] = i0; b[f[1]] = i1; b[f[2]] = i2;
        push(b[0], b[1], b[2], b[3]);
      }
  }
  for (int i3 = 1; i3 < p; ++i3)
    for (int i2 = 1; i2 < p; ++i2)
      for (int i1 = 1; i1 < p; ++i1) {
        int i0 = p - i1 - i2 - i3;
        if (i0 >= 1) push(i0, i1, i2, i3);
      }
  return out;
}

Basis make_basis(int p) {
  Basis B;
  B.p = p;
  for (int a = 0; a <= p; ++a)
    for (int b = 0; a + b <= p; ++b)
      for (int c = 0; a + b + c <= p; ++c) {
        B.mono.push_back(a); B.mono.push_back(b); B.mono.push_back(c);
      }
  B.n = (int)B.mono.size() / 3;
  int n = B.n;
  std::vector<int> beta = node_multi_indices(p);
  if ((int)beta.size() != 4 * n) throw std::logic_error("node count");
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) B.nodes.push_back((double)beta[4 * i + k + 1] / p);
  // Gauss-Jordan inverse of V[i][m] = node_i^mono_m
  std::vector<double> V(n * n), I(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    I[i * n + i] = 1.0;
    for (int m = 0; m < n; ++m)
      V[i * n + m] = std::pow(B.nodes[3 * i], B.mono[3 * m]) * std::pow(B.nodes[3 * i + 1], B.mono[3 * m + 1]) *
                     std::pow(B.nodes[3 * i + 2], B.mono[3 * m + 2]);
  }
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(V[r * n + col]) > std::fabs(V[piv * n + col])) piv = r;
    for (int k = 0; k < n; ++k) {
      std::swap(V[col * n + k], V[piv * n + k]);
      std::swap(I[col * n + k], I[piv * n + k]);
    }
    double d = V[col * n + col];
    for (int k = 0; k < n; ++k) { V[col * n + k] /= d; I[col * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = V[r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { V[r * n + k] -= f * V[col * n + k]; I[r * n + k] -= f * I[col * n + k]; }
    }
  }
  // phi_i(x_j) = delta_ij  <=>  coef V^T = I  <=>  coef = (V^-1)^T
  B.coef.resize(n * n);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < n; ++m) B.coef[i * n + m] = I[m * n + i];
  return B;
}

void Basis::eval(const double* X, double* phi, double* dphi) const {
  std::vector<double> pw(3 * (p + 1));
  for (int k = 0; k < 3; ++k) {
    pw[k * (p + 1)] = 1.0;
    for (int e = 1; e <= p; ++e) pw[k * (p + 1) + e] = pw[k * (p + 1) + e - 1] * X[k];
  }
  auto P = [&](int k, int e) { return e < 0 ? 0.0 : pw[k * (p + 1) + e]; };
  for (int i = 0; i < n; ++i) {
    double v = 0, g0 = 0, g1 = 0, g2 = 0;
    for (int m = 0; m < n; ++m) {
      int a = mono[3 * m], b = mono[3 * m + 1], c = mono[3 * m + 2];
      double cf = coef[i * n + m];
      v += cf * P(0, a) * P(1, b) * P(2, c);
      if (a) g0 += cf * a * P(0, a - 1) * P(1, b) * P(2, c);
      if (b) g1 += cf * b * P(0, a) * P(1, b - 1) * P(2, c);
      if (c) g2 += cf * c * P(0, a) * P(1, b) * P(2, c - 1);
    }
    phi[i] = v;
    dphi[3 * i] = g0;
    dphi[3 * i + 1] = g1;
    dphi[3 * i + 2] = g2;
  }
}

int pre_terms(int form, int p) {
  switch (form) {
    case MASS: return 1;
    case HELMHOLTZ: return 6 + nbasis(p);
    case ELASTICITY: return 36;
    default: return 0;
  }
}

Tables make_tables(int form, int p) {
  Tables t;
  t.form = form;
  t.p = p;
  Basis B = make_basis(p), B1 = make_basis(1);
  int ns = B.n;
  t.ns = ns;
  Rule rule = make_rule(rule_index(form, p));
  int Q = rule.Q;
  t.Q = Q;
  t.W = rule.W;
  t.phi.resize(Q * ns);
  t.dphi.resize(Q * ns * 3);
  t.phi1.resize(Q * 4);
  std::vector<double> d1(12);
  for (int q = 0; q < Q; ++q) {
    B.eval(&rule.X[3 * q], &t.phi[q * ns], &t.dphi[q * ns * 3]);
    B1.eval(&rule.X[3 * q], &t.phi1[q * 4], d1.data());
  }
  t.r = pre_terms(form, p);
  t.R.assign((size_t)t.r * ns * ns, 0.0);
  auto R = [&](int r, int a, int b) -> double& { return t.R[((size_t)r * ns + a) * ns + b]; };
  // Pre-evaluation (Algorithm 2): sum the reduction over q once, on the host.
  for (int q = 0; q < Q; ++q) {
    const double w = t.W[q];
    const double* ph = &t.phi[q * ns];
    const double* dp = &t.dphi[q * ns * 3];
    for (int a = 0; a < ns; ++a)
      for (int b = 0; b < ns; ++b) {
        if (form == MASS) {
          R(0, a, b) += w * ph[a] * ph[b];
        } else if (form == HELMHOLTZ) {
          for (int al = 0; al < 3; ++al) R(al, a, b) += w * dp[3 * a + al] * dp[3 * b + al];
          R(3, a, b) += w * (dp[3 * a + 0] * dp[3 * b + 1] + dp[3 * a + 1] * dp[3 * b + 0]);
          R(4, a, b) += w * (dp[3 * a + 0] * dp[3 * b + 2] + dp[3 * a + 2] * dp[3 * b + 0]);
          R(5, a, b) += w * (dp[3 * a + 1] * dp[3 * b + 2] + dp[3 * a + 2] * dp[3 * b + 1]);
          for (int k = 0; k < ns; ++k) R(6 + k, a, b) += w * ph[k] * ph[a] * ph[b];
        } else if (form == ELASTICITY) {
          for (int k = 0; k < 4; ++k)
            for (int al = 0; al < 3; ++al)
              for (int be = 0; be < 3; ++be)
                R((k * 3 + al) * 3 + be, a, b) += w * t.phi1[q * 4 + k] * dp[3 * a + al] * dp[3 * b + be];
        }
      }
  }
  return t;
}

}  // namespace fea
