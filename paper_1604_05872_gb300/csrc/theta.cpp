// The cost function theta of Section 4.2 for the library's forms, and the
// C ABI entry points of the planner's operation-count algorithm.
//
// theta_se(m): Algorithm 1 applied to the monomial's normal-form expression
//   over the loop nest (e, q, j, k), counted per element; pointwise
//   coefficient values at a point (f(z_0, z_1, ...) of Figure "poisson") are
//   opaque symbols whose evaluation cost is added per (e, q).
// theta_pre(m): rho * iota tables (Section 4.2) give 2 rho iota - 1 operations
//   per (j, k) entry, plus forming the rho * iota geometry coefficients.
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fea.h"
#include "host_model.h"
#include "opcount.h"

namespace fea {

int set_error(int code, const char* msg);

namespace {

std::string G(int x, const std::string& L) {  // physical gradient component x of the basis on loop L
  std::string s = "(";
  for (int a = 0; a < 3; ++a) {
    if (a) s += " + ";
    s += "Ji" + std::to_string(a) + std::to_string(x) + "[e]*D" + std::to_string(a) + "[q," + L + "]";
  }
  return s + ")";
}

struct Mono {
  std::string name;
  std::vector<std::string> blocks;  // one bilinear expression per nonzero (c, d) block
  int64_t pointwise;                // operations per (e, q) outside the nest
  bool pre_ok;
  int64_t rho, n_coef_basis, k_coef;  // pre-evaluation: rho, iota = C(n + k - 1, k)
  int64_t geo_pre;                  // operations forming the geometry tensor per element
};

std::vector<Mono> form_monomials(int form, int p) {
  const int64_t ns = nbasis(p);
  std::vector<Mono> m;
  const std::string wd = "*W[q]*det[e]";
  if (form == MASS) {
    m.push_back({"mass", {"P[q,j]*P[q,k]" + wd}, 0, true, 1, 1, 0, 0});
  } else if (form == HELMHOLTZ) {
    std::string st = "(" + G(0, "j") + "*" + G(0, "k") + " + " + G(1, "j") + "*" + G(1, "k") + " + " + G(2, "j") + "*" +
                     G(2, "k") + ")" + wd;
    m.push_back({"stiffness", {st}, 0, true, 6, 1, 0, 36});
    m.push_back({"f-mass", {"fq[e,q]*P[q,j]*P[q,k]" + wd}, 2 * ns - 1, true, 1, ns, 1, ns});
  } else if (form == ELASTICITY) {
    Mono e{"elastic", {}, 14, true, 9, 4, 1, 324 * 8};
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        std::string s = "(mu[e,q]*(";
        if (c == d) s += G(0, "j") + "*" + G(0, "k") + " + " + G(1, "j") + "*" + G(1, "k") + " + " + G(2, "j") + "*" + G(2, "k") + " + ";
        s += G(d, "j") + "*" + G(c, "k") + ") + lam[e,q]*" + G(c, "j") + "*" + G(d, "k") + ")" + wd;
        e.blocks.push_back(s);
      }
    m.push_back(e);
  } else {
    Mono t{"tangent", {}, ns * 33 + 60 + 81 * 6, false, 0, 0, 0, 0};
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) {
        std::string s = "(";
        for (int I = 0; I < 3; ++I)
          for (int J = 0; J < 3; ++J) {
            if (I || J) s += " + ";
            s += G(I, "j") + "*A" + std::to_string(c) + std::to_string(I) + std::to_string(d) + std::to_string(J) +
                 "[e,q]*" + G(J, "k");
          }
        s += ")" + wd;
        t.blocks.push_back(s);
      }
    m.push_back(t);
  }
  return m;
}

}  // namespace

struct Theta {
  int64_t se, pre, table_words;
};

// theta_se and theta_pre (per element) of monomial `mi` of a form.
Theta theta_of(int form, int p, int mi) {
  auto ms = form_monomials(form, p);
  if (mi < 0 || mi >= (int)ms.size()) throw std::invalid_argument("monomial index");
  const Mono& m = ms[mi];
  const int64_t ns = nbasis(p), Q = rule_points(rule_index(form, p));
  std::map<std::string, int64_t> ext{{"e", 1}, {"q", Q}, {"j", ns}, {"k", ns}};
  std::string prog;
  for (size_t b = 0; b < m.blocks.size(); ++b) {
    oc::SEResult r = oc::sharing_elimination("A" + std::to_string(b) + "[e,j,k]", m.blocks[b], {"e", "q", "j", "k"}, ext,
                                             "b" + std::to_string(b) + "_");
    prog += (prog.empty() ? "" : "; ") + r.program;
  }
  Theta t;
  t.se = oc::count_program(oc::parse_program(prog), ext) + Q * m.pointwise;
  if (m.pre_ok) {
    const int64_t iota = oc::increase_factor(m.n_coef_basis, m.k_coef);
    const int64_t terms = m.rho * iota;
    t.pre = (int64_t)m.blocks.size() * ns * ns * (2 * terms - 1) + m.geo_pre;
    t.table_words = terms * ns * ns;
  } else {
    t.pre = -1;
    t.table_words = 0;
  }
  return t;
}

int num_monomials(int form, int p) { return (int)form_monomials(form, p).size(); }

}  // namespace fea

using namespace fea;

extern "C" {

int fea_opcount_program(const char* program, const char* extents, int64_t* ops) {
  if (!program || !extents || !ops) return set_error(FEA_EINVAL, "NULL argument");
  try {
    *ops = oc::count_program(oc::parse_program(program), oc::parse_extents(extents));
  } catch (const std::exception& e) {
    return set_error(FEA_EINVAL, e.what());
  }
  return FEA_OK;
}

int fea_sharing_elimination(const char* lhs, const char* expr, const char* loops, const char* extents, char* program,
                            size_t cap, int64_t* ops, int* cover) {
  if (!lhs || !expr || !loops || !extents) return set_error(FEA_EINVAL, "NULL argument");
  try {
    std::vector<std::string> ls;
    std::string cur;
    for (const char* c = loops;; ++c) {
      if (*c == ',' || *c == 0) {
        size_t b = cur.find_first_not_of(' '), e = cur.find_last_not_of(' ');
        if (b != std::string::npos) ls.push_back(cur.substr(b, e - b + 1));
        cur.clear();
        if (!*c) break;
      } else {
        cur += *c;
      }
    }
    oc::SEResult r = oc::sharing_elimination(lhs, expr, ls, oc::parse_extents(extents));
    if (ops) *ops = r.ops;
    if (cover) *cover = r.cover;
    if (program && cap) {
      if (r.program.size() + 1 > cap) return set_error(FEA_EINVAL, "program buffer too small");
      std::memcpy(program, r.program.c_str(), r.program.size() + 1);
    }
  } catch (const std::exception& e) {
    return set_error(FEA_EINVAL, e.what());
  }
  return FEA_OK;
}

int fea_vertex_cover(int nl, int nr, const int* edges, int nedges, int* cover_size) {
  if (nl < 0 || nr < 0 || nedges < 0 || (nedges && !edges) || !cover_size) return set_error(FEA_EINVAL, "bad graph");
  std::vector<std::pair<int, int>> E;
  for (int k = 0; k < nedges; ++k) {
    int u = edges[2 * k], v = edges[2 * k + 1];
    if (u < 0 || u >= nl || v < 0 || v >= nr) return set_error(FEA_EINVAL, "edge out of range");
    E.push_back({u, v});
  }
  *cover_size = (int)oc::min_vertex_cover(nl, nr, E).size();
  return FEA_OK;
}

int64_t fea_increase_factor(int n, int k) {
  if (n < 1 || k < 0) return -1;
  return oc::increase_factor(n, k);
}

int fea_theta(int form, int degree, int monomial, int64_t* theta_se, int64_t* theta_pre, int64_t* table_words) {
  if (form < 0 || form > 3 || degree < 1 || degree > 4) return set_error(FEA_EINVAL, "unsupported form/degree");
  if (monomial < 0 || monomial >= num_monomials(form, degree)) return set_error(FEA_EINVAL, "monomial index");
  Theta t = theta_of(form, degree, monomial);
  if (theta_se) *theta_se = t.se;
  if (theta_pre) *theta_pre = t.pre;
  if (table_words) *table_words = t.table_words;
  return FEA_OK;
}

int fea_num_monomials(int form, int degree) {
  if (form < 0 || form > 3 || degree < 1 || degree > 4) return -1;
  return num_monomials(form, degree);
}

}  // extern "C"
