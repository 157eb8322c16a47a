// Host planner (see planner.h).
//
// Operation counts follow Definition 8's convention (additions and products;
// a fused multiply-add counts as two; divisions, square roots and logarithms
// are not counted).  They are the counts of the loop nests the kernels run:
//
//   naive  plain quadrature nest in normal form: everything inside (q, i, j)
//   SE     quadrature nest after sharing elimination (Algorithm 1): physical
//          gradients hoisted per (q, a), pointwise kernels per q, left
//          operands per (q, a, c), and 2 x (#products) flops per entry
//   PRE    pre-evaluated reference tensors (Algorithm 2): geometry tensor per
//          element, then 2 r flops per output entry
//
// Algorithm 3 enumerates the bipartitions of the pre-evaluable monomials,
// drops those whose pre-evaluated tables do not fit T_H (Constraint 2) and
// takes the cheapest by theta = theta_se(S u b_S) + theta_pre(b_P).
#include "planner.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/fea.h"
#include "host_model.h"

namespace fea {

// Flops of one monomial of a form under each schedule, per element.
struct MonoCost {
  int64_t se, pre;       // pre < 0: not pre-evaluable
  int64_t table_bytes4;  // pre-evaluated table size in 4-byte words
};

static std::vector<MonoCost> monomials(int form, int p) {
  const int64_t ns = nbasis(p), Q = rule_points(rule_index(form, p));
  const int64_t n = vector_form(form) ? 3 * ns : ns, nn = n * n;
  const int64_t grad = 15 * ns;  // physical gradients per point: 3 x (3 mul + 2 add) per basis function
  std::vector<MonoCost> m;
  switch (form) {
    case MASS:
      // SE: s = w|det| (1), t_a = s phi_a (ns), entry += t_a phi_b (2)
      m.push_back({Q * (1 + ns + 2 * nn), 2 * nn, ns * ns});
      break;
    case HELMHOLTZ:
      // stiffness: SE needs the gradients, 3 scaled copies and 3 FMA per entry;
      // PRE: K (6 x 6 flops) + 6 terms per entry
      m.push_back({Q * (grad + 1 + 3 * ns + 6 * nn), 36 + 12 * nn, 6 * ns * ns});
      // f-mass: SE needs f_q (2 ns), s f_q phi_a (ns + 1), 1 FMA per entry; PRE: |det| f_k (ns) + ns terms
      m.push_back({Q * (2 * ns + ns + 1 + 2 * nn), ns + 2 * ns * nn, ns * ns * ns});
      break;
    case ELASTICITY:
      // SE (factorised tangent): gradients, mu_q/lam_q (18), 24 FMA per (a, b) block
      // PRE followed by sharing elimination: M (54), then per (a, b) X and L (72 FMA),
      // tr(M X) (9), X^T + L (9), adj^T Z adj (54) and the scaling (9)
      m.push_back({Q * (grad + 18 + 48 * ns * ns), 54 + 306 * ns * ns, 36 * ns * ns});
      break;
    case NEOHOOKEAN:
      // SE: gradients twice (F and contraction), F (18 ns), Y = F^-T G (15 ns), 24 FMA per (a, b) block
      m.push_back({Q * (2 * grad + 18 * ns + 15 * ns + 6 + 48 * ns * ns), -1, 0});
      break;
  }
  return m;
}

OpCounts op_counts(int form, int p) {
  const int64_t ns = nbasis(p), Q = rule_points(rule_index(form, p));
  const int64_t n = vector_form(form) ? 3 * ns : ns, nn = n * n;
  const int64_t geo = 9 + 27 + 5;  // J, adjugate (9 x (mul + fma)), det
  OpCounts oc;
  // naive: per (q, i, j) normal-form integrand, plus per-(e, q) coefficient values
  int64_t per_entry = 0, per_point = 0;
  switch (form) {
    case MASS: per_entry = 4; per_point = 0; break;
    case HELMHOLTZ: per_entry = 41; per_point = 2 * ns; break;
    case ELASTICITY: per_entry = 39 + 2; per_point = 16; break;  // + 5 on the 1/3 diagonal entries
    case NEOHOOKEAN: per_entry = 141; per_point = 33 * ns + 60; break;
  }
  oc.naive = geo + Q * (per_point + per_entry * nn);
  int64_t se = geo, pre = geo;
  bool pre_ok = true;
  for (const MonoCost& m : monomials(form, p)) {
    se += m.se;
    if (m.pre < 0) pre_ok = false;
    else pre += m.pre;
  }
  if (form == HELMHOLTZ) se -= Q * (1 + 3 * ns + 2 * ns);  // shared s and left-operand build counted once
  oc.se = se;
  oc.pre = pre_ok ? pre : -1;
  return oc;
}

static std::mutex g_tmu;
static std::map<std::tuple<int, int, int>, std::pair<int, int>> g_tuned;
static int g_tuned_gen = 0;

int tuned_generation() {
  std::lock_guard<std::mutex> lk(g_tmu);
  return g_tuned_gen;
}

void set_tuned(int form, int p, int prec, int variant, int tile) {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_tuned[std::make_tuple(form, p, prec)] = {variant, tile};
  ++g_tuned_gen;
}
bool get_tuned(int form, int p, int prec, int* variant, int* tile) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_tuned.find(std::make_tuple(form, p, prec));
  if (it == g_tuned.end()) return false;
  *variant = it->second.first;
  *tile = it->second.second;
  return true;
}
void clear_tuned() {
  std::lock_guard<std::mutex> lk(g_tmu);
  g_tuned.clear();
  ++g_tuned_gen;
}

struct Theta {
  int64_t se, pre, table_words;
};
Theta theta_of(int form, int p, int mi);
int num_monomials(int form, int p);

// Algorithm 3: returns a bitmask of the monomials to pre-evaluate.
unsigned algorithm3(int form, int p, int prec, size_t budget, int64_t* best_cost) {
  const int nm = num_monomials(form, p);
  std::vector<Theta> th;
  for (int i = 0; i < nm; ++i) th.push_back(theta_of(form, p, i));
  // step 1: S = {m : theta(m) = theta_pre - theta_se > 0} stays with sharing elimination
  std::vector<int> P;
  for (int i = 0; i < nm; ++i)
    if (th[i].pre >= 0 && th[i].pre - th[i].se <= 0) P.push_back(i);
  const size_t word = prec == 0 ? 8 : 4;
  unsigned best = 0;
  int64_t bestc = INT64_MAX;
  // steps 2-4: every bipartition (b_S, b_P) of P, Constraint 2 filter, argmin
  for (unsigned b = 0; b < (1u << P.size()); ++b) {
    size_t mem = 0;
    int64_t cost = 0;
    unsigned mask = 0;
    for (size_t k = 0; k < P.size(); ++k)
      if (b >> k & 1u) mask |= 1u << P[k];
    for (int i = 0; i < nm; ++i) {
      if (mask >> i & 1u) {
        mem += (size_t)th[i].table_words * word;
        cost += th[i].pre;
      } else {
        cost += th[i].se;
      }
    }
    if (mem > budget) continue;
    if (cost < bestc) {
      bestc = cost;
      best = mask;
    }
  }
  if (best_cost) *best_cost = bestc;
  return best;
}

int choose_variant(int form, int p, int prec, size_t budget, bool use_tuned) {
  int v = 0, t = 0;
  if (use_tuned && get_tuned(form, p, prec, &v, &t) && v != FEA_VARIANT_AUTO) return v;
  if (form == NEOHOOKEAN) return FEA_VARIANT_SE;
  const unsigned mask = algorithm3(form, p, prec, budget, nullptr);
  const int nm = num_monomials(form, p);
  if (mask == (1u << nm) - 1) return FEA_VARIANT_PRE;
  if (mask == 0) return FEA_VARIANT_SE;
  // A mixed bipartition: the kernels implement whole-form variants, so take
  // the cheaper of the two.
  OpCounts oc = op_counts(form, p);
  return (oc.pre >= 0 && oc.pre <= oc.se) ? FEA_VARIANT_PRE : FEA_VARIANT_SE;
}

int default_tile(int variant, int form, int p, int prec, int max_tile, size_t budget, int Q,
                 size_t (*smem)(int, int), bool use_tuned, int pref_tile) {
  int v = 0, t = 0;
  if (use_tuned && get_tuned(form, p, prec, &v, &t) && t > 0 && t <= max_tile && smem(t, Q) <= budget) return t;
  if (pref_tile > 0) {  // the kernel's thread layout is built for this tile
    int te = std::min(pref_tile, max_tile);
    while (te > 1 && smem(te, Q) > budget) --te;
    return te;
  }
  // target a few resident CTAs per SM: about 48 KB of shared memory per tile
  const size_t target = std::min<size_t>(budget, 48 * 1024);
  int best = 1;
  for (int te = 1; te <= max_tile; ++te)
    if (smem(te, Q) <= target) best = te;
  // whole warps for the per-element FP64 geometry (one lane per element): an
  // FP64 instruction holds the FP64 unit for the full warp whatever its lanes
  if (best >= 32) best = best / 32 * 32;
  (void)variant;
  return best;
}

int set_error(int code, const char* msg);

}  // namespace fea

extern "C" int fea_algorithm3(int form, int degree, int precision, size_t smem_budget, unsigned* premask,
                              int64_t* cost) {
  using namespace fea;
  if (form < 0 || form > 3 || degree < 1 || degree > 4) return set_error(FEA_EINVAL, "unsupported form/degree");
  const unsigned m = algorithm3(form, degree, precision == FEA_PREC_FP64 ? 0 : 1,
                                smem_budget ? smem_budget : 232448, cost);
  if (premask) *premask = m;
  return FEA_OK;
}

extern "C" int fea_tune_set(int form, int degree, int precision, int variant, int tile) {
  using namespace fea;
  if (form < 0 || form > 3 || degree < 1 || degree > 4) return set_error(FEA_EINVAL, "unsupported form/degree");
  if (precision != FEA_PREC_FP64 && precision != FEA_PREC_FP32) return set_error(FEA_EINVAL, "unsupported precision");
  if (variant != FEA_VARIANT_AUTO && variant != FEA_VARIANT_SE && variant != FEA_VARIANT_PRE)
    return set_error(FEA_EINVAL, "a tuned variant is SE, PRE or AUTO");
  if (variant == FEA_VARIANT_PRE && form == NEOHOOKEAN) return set_error(FEA_EINVAL, "no pre-evaluated Neo-Hookean form");
  if (tile < 0) return set_error(FEA_EINVAL, "negative tile");
  set_tuned(form, degree, precision == FEA_PREC_FP64 ? 0 : 1, variant, tile);
  return FEA_OK;
}

extern "C" void fea_tune_clear(void) { fea::clear_tuned(); }
