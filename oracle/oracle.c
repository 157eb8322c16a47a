/*
 * Oracle for element-local assembly on tetrahedra: a plain, slow FP64 CPU
 * loop nest that evaluates the quadrature-mode definition of each element
 * matrix (Section 2.2, equation "quadrature") with no factorisation, no code
 * motion and no pre-evaluation.
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, table
 * or constant generator with the CUDA library: it has its own quadrature
 * (Newton iteration on Jacobi polynomials), its own Lagrange basis (Silvester's
 * product formula in barycentric coordinates) and writes every integrand out
 * from the weak form.
 *
 * Conventions (interfaces shared with the library by definition, not by code):
 *   reference tet  T = {X >= 0, X0+X1+X2 <= 1}, vertices v0=(0,0,0), v1=e0,
 *                  v2=e1, v3=e2; barycentrics l0 = 1-X0-X1-X2, l{k+1} = Xk.
 *   element map    x = x0 + J X,  J[r][c] = x_{c+1}[r] - x_0[r].
 *   DOF order      vertices 0..3; edges (2,3),(1,3),(1,2),(0,3),(0,2),(0,1)
 *                  with nodes running from the lower to the higher vertex;
 *                  faces opposite vertices 0..3; then the interior.  Inside a
 *                  face / the interior nodes are ordered by their barycentric
 *                  indices on the entity's vertices, last vertex slowest.
 *   vector DOFs    row/column index 3*a + c (scalar node a, component c).
 *   output         A[e][i][j] row-major, i = test, j = trial.
 *
 * The Bernstein-Bezier basis (the variant computed by sum factorisation on
 * the device) is evaluated here from its definition, for the same two forms.
 *
 * Parity of the Neo-Hookean tangent is pinned by finite differences of this
 * file's own residual and energy (both written from the strain energy), not by
 * a closed form; every other form has closed-form or invariant pins in tests/.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_MASS = 0, OR_HELMHOLTZ = 1, OR_ELASTICITY = 2, OR_NEOHOOKEAN = 3 };

/* ------------------------------------------------------------------------ */
/* Jacobi polynomials P_n^{(a,b)} on [-1,1] by the three-term recurrence.    */
/* ------------------------------------------------------------------------ */
static double jacobi_p(int n, double a, double b, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0;
  double p1 = 0.5 * ((a - b) + (a + b + 2.0) * x);
  for (int k = 1; k < n; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * (k + 1) * (k + a + b + 1) * s;
    double c2 = (s + 1) * ((s + 2) * s * x + a * a - b * b);
    double c3 = 2.0 * (k + a) * (k + b) * (s + 2);
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* d/dx P_n^{(a,b)} = (n+a+b+1)/2 * P_{n-1}^{(a+1,b+1)} */
static double jacobi_dp(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + a + b + 1) * jacobi_p(n - 1, a + 1, b + 1, x);
}

/* Gauss-Jacobi nodes by Newton iteration with deflation against the roots
 * already found, and the classical weight formula
 *   w_k = 2^{a+b+1} G(n+a+1) G(n+b+1) / (G(n+a+b+1) n!) / ((1-x_k^2) P'_n(x_k)^2)
 * for the weight (1-x)^a (1+x)^b on [-1,1]. */
static void gauss_jacobi(int n, double a, double b, double *x, double *w) {
  for (int k = 0; k < n; ++k) {
    double r = -cos((2.0 * k + 1.0) * M_PI / (2.0 * n));
    if (k > 0) r = 0.5 * (r + x[k - 1]);
    for (int it = 0; it < 200; ++it) {
      double s = 0.0;
      for (int i = 0; i < k; ++i) s += 1.0 / (r - x[i]);
      double p = jacobi_p(n, a, b, r);
      double dp = jacobi_dp(n, a, b, r);
      double delta = -p / (dp - s * p);
      r += delta;
      if (fabs(delta) < 1e-17) break;
    }
    x[k] = r;
  }
  /* sort ascending (deflated Newton may return them in any order) */
  for (int i = 1; i < n; ++i) {
    double v = x[i];
    int j = i - 1;
    while (j >= 0 && x[j] > v) { x[j + 1] = x[j]; --j; }
    x[j + 1] = v;
  }
  double c = pow(2.0, a + b + 1) * tgamma(n + a + 1) * tgamma(n + b + 1) /
             (tgamma(n + a + b + 1) * tgamma(n + 1.0));
  for (int k = 0; k < n; ++k) {
    double dp = jacobi_dp(n, a, b, x[k]);
    w[k] = c / ((1.0 - x[k] * x[k]) * dp * dp);
  }
}

/* Number of points of rule m: m = 0 is the 4-point degree-2 rule, m >= 1 is
 * the collapsed (conical-product) Gauss-Jacobi rule with m^3 points. */
int oracle_rule_size(int m) { return m == 0 ? 4 : m * m * m; }

/* Quadrature on the reference tet.  X is [Q][3], W is [Q]; the weights sum to
 * the reference volume 1/6.  Collapsed rule: r from Gauss-Jacobi(2,0),
 * s from Gauss-Jacobi(1,0), t from Gauss-Legendre, all mapped to [0,1];
 * X = (t(1-s)(1-r), s(1-r), r), point order r slowest, t fastest. */
int oracle_quad_rule(int m, double *X, double *W) {
  if (m == 0) {
    const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0;
    const double b = (5.0 - sqrt(5.0)) / 20.0;
    for (int k = 0; k < 4; ++k) {
      double lam[4] = {b, b, b, b};
      lam[k] = a;
      X[3 * k + 0] = lam[1];
      X[3 * k + 1] = lam[2];
      X[3 * k + 2] = lam[3];
      W[k] = 1.0 / 24.0;
    }
    return 4;
  }
  if (m < 1 || m > 16) return -1;
  double xr[16], wr[16], xs[16], ws[16], xt[16], wt[16];
  gauss_jacobi(m, 2.0, 0.0, xr, wr);
  gauss_jacobi(m, 1.0, 0.0, xs, ws);
  gauss_jacobi(m, 0.0, 0.0, xt, wt);
  int q = 0;
  for (int i = 0; i < m; ++i) {
    double r = 0.5 * (1.0 + xr[i]);
    for (int j = 0; j < m; ++j) {
      double s = 0.5 * (1.0 + xs[j]);
      for (int k = 0; k < m; ++k) {
        double t = 0.5 * (1.0 + xt[k]);
        X[3 * q + 0] = t * (1.0 - s) * (1.0 - r);
        X[3 * q + 1] = s * (1.0 - r);
        X[3 * q + 2] = r;
        /* (1-r)^2 dr -> w/8, (1-s) ds -> w/4, dt -> w/2 */
        W[q] = (wr[i] / 8.0) * (ws[j] / 4.0) * (wt[k] / 2.0);
        ++q;
      }
    }
  }
  return q;
}

/* Rule used for each form and degree (a convention both sides implement). */
int oracle_default_rule(int form, int p) {
  switch (form) {
    case OR_MASS: return p == 1 ? 0 : p + 1;
    case OR_HELMHOLTZ: return (3 * p + 2) / 2; /* ceil((3p+1)/2) */
    case OR_ELASTICITY: return p;
    case OR_NEOHOOKEAN: return p + 1;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Lagrange basis on equispaced nodes: Silvester's product formula.          */
/* ------------------------------------------------------------------------ */
int oracle_nbasis(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

/* Barycentric multi-indices of the nodes of P_p in DOF order. beta is [n][4]. */
int oracle_node_indices(int p, int *beta) {
  int n = 0;
  for (int v = 0; v < 4; ++v) {
    for (int c = 0; c < 4; ++c) beta[4 * n + c] = (c == v) ? p : 0;
    ++n;
  }
  static const int edges[6][2] = {{2, 3}, {1, 3}, {1, 2}, {0, 3}, {0, 2}, {0, 1}};
  for (int e = 0; e < 6; ++e) {
    for (int m = 1; m < p; ++m) {
      for (int c = 0; c < 4; ++c) beta[4 * n + c] = 0;
      beta[4 * n + edges[e][0]] = p - m;
      beta[4 * n + edges[e][1]] = m;
      ++n;
    }
  }
  for (int v = 0; v < 4; ++v) {
    int f[3], k = 0;
    for (int c = 0; c < 4; ++c)
      if (c != v) f[k++] = c;
    for (int b2 = 1; b2 < p; ++b2)
      for (int b1 = 1; b1 < p; ++b1) {
        int b0 = p - b1 - b2;
        if (b0 < 1) continue;
        for (int c = 0; c < 4; ++c) beta[4 * n + c] = 0;
        beta[4 * n + f[0]] = b0;
        beta[4 * n + f[1]] = b1;
        beta[4 * n + f[2]] = b2;
        ++n;
      }
  }
  for (int b3 = 1; b3 < p; ++b3)
    for (int b2 = 1; b2 < p; ++b2)
      for (int b1 = 1; b1 < p; ++b1) {
        int b0 = p - b1 - b2 - b3;
        if (b0 < 1) continue;
        beta[4 * n + 0] = b0;
        beta[4 * n + 1] = b1;
        beta[4 * n + 2] = b2;
        beta[4 * n + 3] = b3;
        ++n;
      }
  return n;
}

/* One factor of Silvester's formula: prod_{m<k} (p*l - m)/(m+1) and its
 * derivative with respect to l. */
static void silvester_factor(int p, int k, double l, double *val, double *der) {
  double v = 1.0, d = 0.0;
  for (int m = 0; m < k; ++m) {
    double f = (p * l - m) / (m + 1.0);
    double df = p / (m + 1.0);
    d = d * f + v * df;
    v = v * f;
  }
  *val = v;
  *der = d;
}

/* Values phi[n] and reference gradients dphi[n][3] of the P_p basis at X. */
static void basis_eval(int p, int n, const int *beta, const double *X,
                       double *phi, double *dphi) {
  double lam[4] = {1.0 - X[0] - X[1] - X[2], X[0], X[1], X[2]};
  for (int a = 0; a < n; ++a) {
    double v[4], d[4];
    for (int c = 0; c < 4; ++c) silvester_factor(p, beta[4 * a + c], lam[c], &v[c], &d[c]);
    double val = v[0] * v[1] * v[2] * v[3];
    double dl[4];
    for (int c = 0; c < 4; ++c) {
      double prod = d[c];
      for (int o = 0; o < 4; ++o)
        if (o != c) prod *= v[o];
      dl[c] = prod;
    }
    phi[a] = val;
    /* dl0/dX_k = -1, dl_{k+1}/dX_k = +1 */
    for (int k = 0; k < 3; ++k) dphi[3 * a + k] = dl[k + 1] - dl[0];
  }
}

/* Public: tabulate the basis at Q points.  phi is [Q][n], dphi is [Q][n][3]. */
int oracle_basis(int p, int Q, const double *X, double *phi, double *dphi) {
  int n = oracle_nbasis(p);
  int *beta = (int *)malloc(sizeof(int) * 4 * n);
  oracle_node_indices(p, beta);
  for (int q = 0; q < Q; ++q) basis_eval(p, n, beta, X + 3 * q, phi + (size_t)q * n, dphi + (size_t)q * n * 3);
  free(beta);
  return n;
}

/* Reference coordinates of the nodes, [n][3]. */
int oracle_nodes(int p, double *X) {
  int n = oracle_nbasis(p);
  int *beta = (int *)malloc(sizeof(int) * 4 * n);
  oracle_node_indices(p, beta);
  for (int a = 0; a < n; ++a)
    for (int k = 0; k < 3; ++k) X[3 * a + k] = (double)beta[4 * a + k + 1] / p;
  free(beta);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
/* J[r][c] = x_{c+1}[r] - x_0[r]; returns det J and writes Jinv[a][b] = dX_a/dx_b. */
static double geometry(const double *x, double J[3][3], double Jinv[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = x[3 * (c + 1) + r] - x[r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  /* inverse = transpose of the cofactor matrix over det */
  Jinv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  Jinv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Jinv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Jinv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  Jinv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Jinv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Jinv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  Jinv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Jinv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return det;
}

/* Physical gradient of one basis function: g_b = sum_a dX_a/dx_b dPhi/dX_a. */
static void phys_grad(double Jinv[3][3], const double *dref, double *g) {
  for (int b = 0; b < 3; ++b) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += Jinv[a][b] * dref[a];
    g[b] = s;
  }
}

static double det3(double F[3][3]) {
  return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
         F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}

static void inv3(double F[3][3], double d, double Fi[3][3]) {
  Fi[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) / d;
  Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) / d;
  Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) / d;
  Fi[1][0] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) / d;
  Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) / d;
  Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) / d;
  Fi[2][0] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) / d;
  Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) / d;
  Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) / d;
}

int oracle_local_dim(int form, int p) {
  int n = oracle_nbasis(p);
  return (form == OR_ELASTICITY || form == OR_NEOHOOKEAN) ? 3 * n : n;
}

/* Deformation gradient F = I + grad u at one point (Neo-Hookean). */
static void deformation(int n, const double *u, double Jinv[3][3], const double *dphi_q, double F[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) F[i][j] = (i == j) ? 1.0 : 0.0;
  for (int a = 0; a < n; ++a) {
    double g[3];
    phys_grad(Jinv, dphi_q + 3 * a, g);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) F[i][j] += u[3 * a + i] * g[j];
  }
}

/* ------------------------------------------------------------------------ */
/* Element matrices.                                                         */
/*   mass        : int phi_i phi_j                                           */
/*   helmholtz   : int grad phi_i . grad phi_j + f phi_i phi_j, f in P_p      */
/*   elasticity  : int 2 mu eps(u):eps(v) + lam div u div v, mu, lam in P_1   */
/*   neohookean  : tangent of W = mu/2 (tr C - 3) - mu ln J + lam/2 (ln J)^2  */
/* coeffs per element: helmholtz f[n]; elasticity mu[4], lam[4];             */
/* neohookean u[n][3] with the constants mu, lam passed separately.          */
/* ------------------------------------------------------------------------ */
int oracle_assemble(int form, int p, int m, int64_t E, const double *coords,
                    const double *coeffs, double mu_c, double lam_c,
                    double *out, int nthreads) {
  if (form < 0 || form > 3 || p < 1 || p > 4) return -1;
  int n = oracle_nbasis(p);
  int nd = oracle_local_dim(form, p);
  int Q = oracle_rule_size(m);
  double *X = (double *)malloc(sizeof(double) * 3 * Q);
  double *W = (double *)malloc(sizeof(double) * Q);
  if (oracle_quad_rule(m, X, W) < 0) { free(X); free(W); return -2; }
  double *phi = (double *)malloc(sizeof(double) * Q * n);
  double *dphi = (double *)malloc(sizeof(double) * Q * n * 3);
  oracle_basis(p, Q, X, phi, dphi);
  double *phi1 = (double *)malloc(sizeof(double) * Q * 4);
  double *dphi1 = (double *)malloc(sizeof(double) * Q * 4 * 3);
  oracle_basis(1, Q, X, phi1, dphi1);
  int clen = form == OR_HELMHOLTZ ? n : form == OR_ELASTICITY ? 8 : form == OR_NEOHOOKEAN ? 3 * n : 0;
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int64_t e = 0; e < E; ++e) {
    const double *x = coords + 12 * e;
    const double *c = coeffs ? coeffs + (size_t)clen * e : NULL;
    double *A = out + (size_t)nd * nd * e;
    double J[3][3], Jinv[3][3];
    double det = geometry(x, J, Jinv);
    if (!(det != 0.0)) bad += 1;
    double adet = fabs(det);
    for (int i = 0; i < nd * nd; ++i) A[i] = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double *ph = phi + (size_t)q * n;
      const double *dph = dphi + (size_t)q * n * 3;
      double wq = W[q] * adet;
      if (form == OR_MASS) {
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) A[i * nd + j] += wq * ph[i] * ph[j];
      } else if (form == OR_HELMHOLTZ) {
        double fq = 0.0;
        for (int k = 0; k < n; ++k) fq += c[k] * ph[k];
        for (int i = 0; i < n; ++i)
          for (int j = 0; j < n; ++j) {
            double gi[3], gj[3];
            phys_grad(Jinv, dph + 3 * i, gi);
            phys_grad(Jinv, dph + 3 * j, gj);
            double dot = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
            A[i * nd + j] += wq * (dot + fq * ph[i] * ph[j]);
          }
      } else if (form == OR_ELASTICITY) {
        double muq = 0.0, lamq = 0.0;
        for (int k = 0; k < 4; ++k) {
          muq += c[k] * phi1[4 * q + k];
          lamq += c[4 + k] * phi1[4 * q + k];
        }
        for (int a = 0; a < n; ++a)
          for (int cc = 0; cc < 3; ++cc)
            for (int b = 0; b < n; ++b)
              for (int d = 0; d < 3; ++d) {
                double ga[3], gb[3];
                phys_grad(Jinv, dph + 3 * a, ga);
                phys_grad(Jinv, dph + 3 * b, gb);
                /* grad v = e_cc (x) ga, grad u = e_d (x) gb */
                double gv[3][3] = {{0}}, gu[3][3] = {{0}};
                for (int k = 0; k < 3; ++k) {
                  gv[cc][k] = ga[k];
                  gu[d][k] = gb[k];
                }
                double epsv[3][3], epsu[3][3];
                for (int r = 0; r < 3; ++r)
                  for (int s = 0; s < 3; ++s) {
                    epsv[r][s] = 0.5 * (gv[r][s] + gv[s][r]);
                    epsu[r][s] = 0.5 * (gu[r][s] + gu[s][r]);
                  }
                double contr = 0.0;
                for (int r = 0; r < 3; ++r)
                  for (int s = 0; s < 3; ++s) contr += epsu[r][s] * epsv[r][s];
                double divv = epsv[0][0] + epsv[1][1] + epsv[2][2];
                double divu = epsu[0][0] + epsu[1][1] + epsu[2][2];
                A[(3 * a + cc) * nd + 3 * b + d] += wq * (2.0 * muq * contr + lamq * divu * divv);
              }
      } else { /* OR_NEOHOOKEAN */
        double F[3][3], Fi[3][3];
        deformation(n, c, Jinv, dph, F);
        double JF = det3(F);
        if (!(JF > 0.0)) bad += 1;
        inv3(F, JF, Fi);
        double lnJ = log(JF);
        for (int a = 0; a < n; ++a)
          for (int cc = 0; cc < 3; ++cc)
            for (int b = 0; b < n; ++b)
              for (int d = 0; d < 3; ++d) {
                double ga[3], gb[3];
                phys_grad(Jinv, dph + 3 * a, ga);
                phys_grad(Jinv, dph + 3 * b, gb);
                double s = 0.0;
                for (int I = 0; I < 3; ++I)
                  for (int JJ = 0; JJ < 3; ++JJ) {
                    /* dP_{cc I} / dF_{d JJ} */
                    double tang = mu_c * ((cc == d) && (I == JJ) ? 1.0 : 0.0) +
                                  (mu_c - lam_c * lnJ) * Fi[JJ][cc] * Fi[I][d] +
                                  lam_c * Fi[I][cc] * Fi[JJ][d];
                    s += ga[I] * tang * gb[JJ];
                  }
                A[(3 * a + cc) * nd + 3 * b + d] += wq * s;
              }
      }
    }
  }
  free(X); free(W); free(phi); free(dphi); free(phi1); free(dphi1);
  return bad;
}

/* Neo-Hookean residual R_{(a,c)} = int P(F)_{cI} d phi_a/dx_I with
 * P = dW/dF = mu (F - F^{-T}) + lam ln J F^{-T}; out is [E][3n]. */
int oracle_neohookean_residual(int p, int m, int64_t E, const double *coords,
                               const double *u, double mu_c, double lam_c, double *out) {
  int n = oracle_nbasis(p);
  int Q = oracle_rule_size(m);
  double *X = (double *)malloc(sizeof(double) * 3 * Q);
  double *W = (double *)malloc(sizeof(double) * Q);
  oracle_quad_rule(m, X, W);
  double *phi = (double *)malloc(sizeof(double) * Q * n);
  double *dphi = (double *)malloc(sizeof(double) * Q * n * 3);
  oracle_basis(p, Q, X, phi, dphi);
  for (int64_t e = 0; e < E; ++e) {
    double J[3][3], Jinv[3][3];
    double adet = fabs(geometry(coords + 12 * e, J, Jinv));
    const double *ue = u + (size_t)3 * n * e;
    double *R = out + (size_t)3 * n * e;
    for (int i = 0; i < 3 * n; ++i) R[i] = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double *dph = dphi + (size_t)q * n * 3;
      double F[3][3], Fi[3][3];
      deformation(n, ue, Jinv, dph, F);
      double JF = det3(F);
      inv3(F, JF, Fi);
      double lnJ = log(JF);
      double P[3][3];
      for (int i = 0; i < 3; ++i)
        for (int I = 0; I < 3; ++I) P[i][I] = mu_c * (F[i][I] - Fi[I][i]) + lam_c * lnJ * Fi[I][i];
      for (int a = 0; a < n; ++a) {
        double g[3];
        phys_grad(Jinv, dph + 3 * a, g);
        for (int cc = 0; cc < 3; ++cc) {
          double s = 0.0;
          for (int I = 0; I < 3; ++I) s += P[cc][I] * g[I];
          R[3 * a + cc] += W[q] * adet * s;
        }
      }
    }
  }
  free(X); free(W); free(phi); free(dphi);
  return 0;
}

/* Load vector of the Helmholtz form's right-hand side (its linear
 * counterpart, Section 2: a form of arity 1): b_i = int f phi_i dx with f in
 * the same P_p space as the basis, f = sum_k f_k phi_k; out is [E][n]. */
int oracle_load_vector(int p, int m, int64_t E, const double *coords, const double *f, double *out) {
  int n = oracle_nbasis(p);
  int Q = oracle_rule_size(m);
  double *X = (double *)malloc(sizeof(double) * 3 * Q);
  double *W = (double *)malloc(sizeof(double) * Q);
  oracle_quad_rule(m, X, W);
  double *phi = (double *)malloc(sizeof(double) * Q * n);
  double *dphi = (double *)malloc(sizeof(double) * Q * n * 3);
  oracle_basis(p, Q, X, phi, dphi);
  for (int64_t e = 0; e < E; ++e) {
    double J[3][3], Jinv[3][3];
    double adet = fabs(geometry(coords + 12 * e, J, Jinv));
    const double *fe = f + (size_t)n * e;
    double *b = out + (size_t)n * e;
    for (int i = 0; i < n; ++i) b[i] = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double *ph = phi + (size_t)q * n;
      double fq = 0.0;
      for (int k = 0; k < n; ++k) fq += fe[k] * ph[k];
      for (int i = 0; i < n; ++i) b[i] += W[q] * adet * fq * ph[i];
    }
  }
  free(X); free(W); free(phi); free(dphi);
  return 0;
}

/* Neo-Hookean stored energy int W(F) dx per element; out is [E]. */
int oracle_neohookean_energy(int p, int m, int64_t E, const double *coords,
                             const double *u, double mu_c, double lam_c, double *out) {
  int n = oracle_nbasis(p);
  int Q = oracle_rule_size(m);
  double *X = (double *)malloc(sizeof(double) * 3 * Q);
  double *W = (double *)malloc(sizeof(double) * Q);
  oracle_quad_rule(m, X, W);
  double *phi = (double *)malloc(sizeof(double) * Q * n);
  double *dphi = (double *)malloc(sizeof(double) * Q * n * 3);
  oracle_basis(p, Q, X, phi, dphi);
  for (int64_t e = 0; e < E; ++e) {
    double J[3][3], Jinv[3][3];
    double adet = fabs(geometry(coords + 12 * e, J, Jinv));
    const double *ue = u + (size_t)3 * n * e;
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) {
      double F[3][3];
      deformation(n, ue, Jinv, dphi + (size_t)q * n * 3, F);
      double JF = det3(F);
      double trC = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) trC += F[i][j] * F[i][j];
      double lnJ = log(JF);
      double Wd = 0.5 * mu_c * (trC - 3.0) - mu_c * lnJ + 0.5 * lam_c * lnJ * lnJ;
      acc += W[q] * adet * Wd;
    }
    out[e] = acc;
  }
  free(X); free(W); free(phi); free(dphi);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Bernstein-Bezier basis (the sum-factorised variant): the definition.      */
/* ------------------------------------------------------------------------ */
/* B_a = p! / (a0! a1! a2! a3!) l0^a0 l1^a1 l2^a2 l3^a3 over |a| = p, ordered
 * a3 = 0..p (slowest), then a2 = 0..p-a3, then a1 = 0..p-a3-a2 (fastest),
 * a0 = p - a1 - a2 - a3.  The order is an interface convention; the values
 * here come from the definition only. */
int oracle_bernstein_indices(int p, int *alpha) {
  int k = 0;
  for (int a3 = 0; a3 <= p; ++a3)
    for (int a2 = 0; a2 <= p - a3; ++a2)
      for (int a1 = 0; a1 <= p - a3 - a2; ++a1) {
        alpha[4 * k + 0] = p - a1 - a2 - a3;
        alpha[4 * k + 1] = a1;
        alpha[4 * k + 2] = a2;
        alpha[4 * k + 3] = a3;
        ++k;
      }
  return k;
}

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= (double)i;
  return f;
}

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/* B [Q][n] and dB/dX [Q][n][3] at reference points X [Q][3]. */
int oracle_bernstein_basis(int p, int Q, const double *X, double *B, double *dB) {
  const int n = oracle_nbasis(p);
  int *al = (int *)malloc(sizeof(int) * 4 * n);
  oracle_bernstein_indices(p, al);
  for (int q = 0; q < Q; ++q) {
    const double l[4] = {1.0 - X[3 * q] - X[3 * q + 1] - X[3 * q + 2], X[3 * q], X[3 * q + 1], X[3 * q + 2]};
    for (int k = 0; k < n; ++k) {
      const int *a = al + 4 * k;
      const double c = factorial(p) / (factorial(a[0]) * factorial(a[1]) * factorial(a[2]) * factorial(a[3]));
      double v = c;
      for (int j = 0; j < 4; ++j) v *= ipow(l[j], a[j]);
      B[(size_t)q * n + k] = v;
      /* dB/dl_j = c a_j l^(a - e_j); dB/dX_i = dB/dl_{i+1} - dB/dl_0 */
      double dl[4];
      for (int j = 0; j < 4; ++j) {
        if (a[j] == 0) {
          dl[j] = 0.0;
          continue;
        }
        double t = c * (double)a[j];
        for (int i = 0; i < 4; ++i) t *= ipow(l[i], a[i] - (i == j ? 1 : 0));
        dl[j] = t;
      }
      for (int i = 0; i < 3; ++i) dB[((size_t)q * n + k) * 3 + i] = dl[i + 1] - dl[0];
    }
  }
  free(al);
  return n;
}

/* Element matrices in the Bernstein basis by the plain quadrature nest:
 * mass A_ij = sum_q w_q |det J| B_i B_j; Helmholtz
 * A_ij = sum_q w_q |det J| (G_i . G_j + f_q B_i B_j) with f_q = sum_k c_k B_k(X_q)
 * (c: the Bernstein coefficients of f, [E][n]) and G = J^-T grad_X B. */
int oracle_assemble_bernstein(int form, int p, int m, int64_t E, const double *coords, const double *c,
                              double *out, int nthreads) {
  if ((form != OR_MASS && form != OR_HELMHOLTZ) || p < 1 || p > 4) return -1;
  const int n = oracle_nbasis(p);
  const int Q = oracle_rule_size(m);
  double *X = (double *)malloc(sizeof(double) * 3 * Q);
  double *W = (double *)malloc(sizeof(double) * Q);
  if (oracle_quad_rule(m, X, W) < 0) {
    free(X);
    free(W);
    return -2;
  }
  double *B = (double *)malloc(sizeof(double) * Q * n);
  double *dB = (double *)malloc(sizeof(double) * Q * n * 3);
  oracle_bernstein_basis(p, Q, X, B, dB);
  int bad = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(+ : bad)
#endif
  for (int64_t e = 0; e < E; ++e) {
    const double *x = coords + 12 * e;
    double *A = out + (size_t)n * n * e;
    double J[3][3], Jinv[3][3];
    const double det = geometry(x, J, Jinv);
    if (!(det != 0.0)) bad += 1;
    const double adet = fabs(det);
    for (int i = 0; i < n * n; ++i) A[i] = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double *b = B + (size_t)q * n;
      const double *db = dB + (size_t)q * n * 3;
      const double wq = W[q] * adet;
      double fq = 1.0;
      if (form == OR_HELMHOLTZ) {
        fq = 0.0;
        for (int k = 0; k < n; ++k) fq += c[(size_t)n * e + k] * b[k];
      }
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double v = fq * b[i] * b[j];
          if (form == OR_HELMHOLTZ) {
            double gi[3], gj[3];
            phys_grad(Jinv, db + 3 * i, gi);
            phys_grad(Jinv, db + 3 * j, gj);
            v += gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
          }
          A[i * n + j] += wq * v;
        }
    }
  }
  free(X);
  free(W);
  free(B);
  free(dB);
  return bad;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
