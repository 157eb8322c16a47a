// Operation counting, sharing elimination (Algorithm 1) and the increase
// factor of pre-evaluation (Section 4.2) on the planner's expression language
// (see opcount.h).
#include "opcount.h"

#include <algorithm>
#include <cctype>
#include <functional>
#include <sstream>
#include <stdexcept>

namespace fea {
namespace oc {

// ------------------------------------------------------------------ parsing
namespace {
struct Parser {
  const std::string& s;
  size_t p = 0;
  Expr e;
  explicit Parser(const std::string& src) : s(src) {}
  void ws() {
    while (p < s.size() && std::isspace((unsigned char)s[p])) ++p;
  }
  bool eat(char c) {
    ws();
    if (p < s.size() && s[p] == c) {
      ++p;
      return true;
    }
    return false;
  }
  std::string ident() {
    ws();
    size_t b = p;
    while (p < s.size() && (std::isalnum((unsigned char)s[p]) || s[p] == '_' || s[p] == '.')) ++p;
    if (b == p) throw std::invalid_argument("expected a name at: " + s.substr(b));
    return s.substr(b, p - b);
  }
  int add(Node n) {
    e.n.push_back(std::move(n));
    return (int)e.n.size() - 1;
  }
  int atom() {
    if (eat('(')) {
      int r = expr();
      if (!eat(')')) throw std::invalid_argument("missing ')'");
      return r;
    }
    Node n;
    n.name = ident();
    if (std::isdigit((unsigned char)n.name[0])) {
      n.kind = Node::NUM;
      return add(n);
    }
    n.kind = Node::SYM;
    if (eat('[')) {
      do {
        n.idx.push_back(ident());
      } while (eat(','));
      if (!eat(']')) throw std::invalid_argument("missing ']'");
    }
    return add(n);
  }
  int term() {
    std::vector<int> f{atom()};
    while (eat('*')) f.push_back(atom());
    if (f.size() == 1) return f[0];
    Node n;
    n.kind = Node::MUL;
    n.ch = f;
    return add(n);
  }
  int expr() {
    std::vector<int> t{term()}, neg{0};
    for (;;) {
      if (eat('+')) {
        t.push_back(term());
        neg.push_back(0);
      } else if (eat('-')) {
        t.push_back(term());
        neg.push_back(1);
      } else {
        break;
      }
    }
    if (t.size() == 1) return t[0];
    Node n;
    n.kind = Node::ADD;
    n.ch = t;
    n.neg = neg;
    return add(n);
  }
};

std::vector<std::string> split(const std::string& s, char c) {
  std::vector<std::string> out;
  std::string cur;
  for (char ch : s) {
    if (ch == c) {
      out.push_back(cur);
      cur.clear();
    } else {
      cur += ch;
    }
  }
  out.push_back(cur);
  return out;
}

std::string trim(const std::string& s) {
  size_t b = s.find_first_not_of(" \t\n"), e = s.find_last_not_of(" \t\n");
  return b == std::string::npos ? "" : s.substr(b, e - b + 1);
}
}  // namespace

Expr parse_expr(const std::string& s) {
  Parser ps(s);
  ps.e.root = ps.expr();
  ps.ws();
  if (ps.p != s.size()) throw std::invalid_argument("trailing text: " + s.substr(ps.p));
  return ps.e;
}

std::string Expr::str(int i) const {
  const Node& x = n[i];
  if (x.kind == Node::SYM) {
    std::string r = x.name;
    if (!x.idx.empty()) {
      r += "[";
      for (size_t k = 0; k < x.idx.size(); ++k) r += (k ? "," : "") + x.idx[k];
      r += "]";
    }
    return r;
  }
  if (x.kind == Node::NUM) return x.name;
  std::string r = "(";
  for (size_t k = 0; k < x.ch.size(); ++k) {
    if (k) r += x.kind == Node::MUL ? "*" : (x.neg[k] ? "-" : "+");
    r += str(x.ch[k]);
  }
  return r + ")";
}

std::set<std::string> Expr::deps(int i) const {
  const Node& x = n[i];
  if (x.kind == Node::SYM) return std::set<std::string>(x.idx.begin(), x.idx.end());
  std::set<std::string> d;
  for (int c : x.ch) {
    auto s = deps(c);
    d.insert(s.begin(), s.end());
  }
  return d;
}

int64_t Expr::ops(int i) const {
  const Node& x = n[i];
  if (x.kind == Node::SYM || x.kind == Node::NUM) return 0;
  int64_t k = (int64_t)x.ch.size() - 1;
  for (int c : x.ch) k += ops(c);
  return k;
}

std::vector<Stmt> parse_program(const std::string& s) {
  std::vector<Stmt> prog;
  for (const std::string& raw : split(s, ';')) {
    std::string t = trim(raw);
    if (t.empty()) continue;
    size_t colon = t.find(':');
    if (colon == std::string::npos) throw std::invalid_argument("statement without loops: " + t);
    Stmt st;
    for (const std::string& l : split(t.substr(0, colon), ',')) {
      std::string lt = trim(l);
      if (!lt.empty()) st.loops.push_back(lt);
    }
    std::string rest = t.substr(colon + 1);
    size_t pe = rest.find("+=");
    size_t eq = pe != std::string::npos ? pe : rest.find('=');
    if (eq == std::string::npos) throw std::invalid_argument("statement without '=': " + t);
    st.accum = pe != std::string::npos;
    st.lhs = trim(rest.substr(0, eq));
    st.rhs = parse_expr(trim(rest.substr(eq + (st.accum ? 2 : 1))));
    prog.push_back(std::move(st));
  }
  return prog;
}

std::map<std::string, int64_t> parse_extents(const std::string& s) {
  std::map<std::string, int64_t> m;
  for (const std::string& kv : split(s, ',')) {
    std::string t = trim(kv);
    if (t.empty()) continue;
    size_t c = t.find(':');
    if (c == std::string::npos) throw std::invalid_argument("extent without ':'");
    m[trim(t.substr(0, c))] = std::stoll(trim(t.substr(c + 1)));
  }
  return m;
}

int64_t count_program(const std::vector<Stmt>& prog, const std::map<std::string, int64_t>& ext) {
  // group statements by loop body; count distinct non-trivial sub-expressions once per body
  std::map<std::vector<std::string>, std::pair<std::set<std::string>, int64_t>> body;
  for (const Stmt& st : prog) {
    auto& b = body[st.loops];
    std::function<void(int)> visit = [&](int i) {
      const Node& x = st.rhs.n[i];
      if (x.kind == Node::SYM || x.kind == Node::NUM) return;
      std::string key = st.rhs.str(i);
      if (b.first.insert(key).second) {
        b.second += (int64_t)x.ch.size() - 1;
        for (int c : x.ch) visit(c);
      }
    };
    visit(st.rhs.root);
    if (st.accum) b.second += 1;
  }
  int64_t total = 0;
  for (auto& kv : body) {
    int64_t trips = 1;
    for (const std::string& l : kv.first) {
      auto it = ext.find(l);
      if (it == ext.end()) throw std::invalid_argument("no extent for loop " + l);
      trips *= it->second;
    }
    total += trips * kv.second.second;
  }
  return total;
}

// ------------------------------------------------------------ vertex cover
std::vector<std::pair<int, int>> min_vertex_cover(int nl, int nr, const std::vector<std::pair<int, int>>& edges) {
  std::vector<std::vector<int>> adj(nl);
  for (auto& e : edges) adj[e.first].push_back(e.second);
  std::vector<int> ml(nl, -1), mr(nr, -1);
  std::function<bool(int, std::vector<char>&)> augment = [&](int u, std::vector<char>& seen) {
    for (int v : adj[u]) {
      if (seen[v]) continue;
      seen[v] = 1;
      if (mr[v] < 0 || augment(mr[v], seen)) {
        ml[u] = v;
        mr[v] = u;
        return true;
      }
    }
    return false;
  };
  for (int u = 0; u < nl; ++u) {
    std::vector<char> seen(nr, 0);
    augment(u, seen);
  }
  // Koenig: Z = vertices reachable from free left vertices by alternating paths
  std::vector<char> zl(nl, 0), zr(nr, 0);
  std::function<void(int)> walk = [&](int u) {
    if (zl[u]) return;
    zl[u] = 1;
    for (int v : adj[u]) {
      if (zr[v] || ml[u] == v) continue;
      zr[v] = 1;
      if (mr[v] >= 0) walk(mr[v]);
    }
  };
  for (int u = 0; u < nl; ++u)
    if (ml[u] < 0) walk(u);
  std::vector<std::pair<int, int>> cover;
  for (int u = 0; u < nl; ++u)
    if (!zl[u] && !adj[u].empty()) cover.push_back({0, u});
  for (int v = 0; v < nr; ++v)
    if (zr[v]) cover.push_back({1, v});
  return cover;
}

int64_t increase_factor(int64_t n, int64_t k) {
  // C(n + k - 1, k)
  int64_t r = 1;
  for (int64_t i = 1; i <= k; ++i) r = r * (n + i - 1) / i;
  return r;
}

// ------------------------------------------------------- sharing elimination
namespace {
// One term of the expanded expression: product of scalar factors, one
// operand per linear loop (strings: canonical text of sub-expressions).
struct Term {
  std::vector<std::string> coef;
  std::vector<std::string> a, b;  // operands on the first / second linear loop
  bool neg = false;
};

struct Ctx {
  const Expr& e;
  std::string L1, L2;
  int side(int i) const {
    auto d = e.deps(i);
    bool h1 = d.count(L1), h2 = d.count(L2);
    return h1 && h2 ? 3 : h1 ? 1 : h2 ? 2 : 0;
  }
  std::vector<Term> expand(int i) const {
    const Node& x = e.n[i];
    int s = side(i);
    if (s != 3) {
      Term t;
      (s == 0 ? t.coef : s == 1 ? t.a : t.b).push_back(e.str(i));
      return {t};
    }
    if (x.kind == Node::ADD) {
      std::vector<Term> out;
      for (size_t k = 0; k < x.ch.size(); ++k)
        for (Term t : expand(x.ch[k])) {
          t.neg ^= (bool)x.neg[k];
          out.push_back(t);
        }
      return out;
    }
    if (x.kind == Node::MUL) {
      std::vector<Term> acc{Term{}};
      for (int c : x.ch) {
        std::vector<Term> nxt;
        for (const Term& l : acc)
          for (const Term& r : expand(c)) {
            Term t = l;
            t.coef.insert(t.coef.end(), r.coef.begin(), r.coef.end());
            t.a.insert(t.a.end(), r.a.begin(), r.a.end());
            t.b.insert(t.b.end(), r.b.begin(), r.b.end());
            t.neg = l.neg ^ r.neg;
            nxt.push_back(t);
          }
        acc = nxt;
      }
      return acc;
    }
    throw std::invalid_argument("a symbol depends on both linear loops: not a multilinear nest");
  }
};

std::string join(const std::vector<std::string>& v, const std::string& sep) {
  std::string r;
  for (size_t k = 0; k < v.size(); ++k) r += (k ? sep : "") + v[k];
  return r;
}

// multilinear symbols of an operand (symbols that depend on its loop)
std::set<std::string> ml_symbols(const Expr& e, int i, const std::string& L) {
  std::set<std::string> s;
  const Node& x = e.n[i];
  if (x.kind == Node::SYM) {
    if (std::find(x.idx.begin(), x.idx.end(), L) != x.idx.end()) s.insert(e.str(i));
    return s;
  }
  for (int c : x.ch) {
    auto t = ml_symbols(e, c, L);
    s.insert(t.begin(), t.end());
  }
  return s;
}

// Expand an operand linear in its multilinear symbols into (coefficient, symbol) pairs.
bool linear_split(const Expr& e, int i, const std::string& L, std::vector<std::pair<std::string, std::string>>& out,
                  std::string coef) {
  const Node& x = e.n[i];
  auto d = e.deps(i);
  if (!d.count(L)) return false;
  if (x.kind == Node::SYM) {
    out.push_back({coef, e.str(i)});
    return true;
  }
  if (x.kind == Node::ADD) {
    for (size_t k = 0; k < x.ch.size(); ++k) {
      std::string c = coef;
      if (x.neg[k]) c = c.empty() ? "(0-1)" : "(0-1)*" + c;
      if (!linear_split(e, x.ch[k], L, out, c)) return false;
    }
    return true;
  }
  if (x.kind == Node::MUL) {
    int lin = -1;
    std::vector<std::string> sc;
    for (int c : x.ch) {
      if (e.deps(c).count(L)) {
        if (lin >= 0) return false;  // product of two multilinear factors
        lin = c;
      } else {
        sc.push_back(e.str(c));
      }
    }
    std::string c = coef;
    for (auto& s : sc) c = c.empty() ? s : c + "*" + s;
    return linear_split(e, lin, L, out, c);
  }
  return false;
}
}  // namespace

SEResult sharing_elimination(const std::string& lhs, const std::string& expr, const std::vector<std::string>& loops,
                             const std::map<std::string, int64_t>& ext, const std::string& prefix) {
  if (loops.size() < 2) throw std::invalid_argument("need two linear loops");
  const std::string L1 = loops[loops.size() - 2], L2 = loops.back();
  std::vector<std::string> outer(loops.begin(), loops.end() - 2);
  auto with = [&](const std::string& L) {
    std::vector<std::string> v = outer;
    v.push_back(L);
    return v;
  };
  auto lstr = [](const std::vector<std::string>& v) { return join(v, ","); };
  Expr e = parse_expr(expr);
  Ctx cx{e, L1, L2};
  std::vector<Term> terms = cx.expand(e.root);

  // operands: merge several factors of one side into one product
  std::map<std::string, int> opnode;  // canonical text -> node id in e
  std::function<void(int)> index_nodes = [&](int i) {
    opnode.emplace(e.str(i), i);
    for (int c : e.n[i].ch) index_nodes(c);
  };
  index_nodes(e.root);
  for (Term& t : terms) {
    for (auto* side : {&t.a, &t.b}) {
      if (side->size() > 1) {
        std::string prod = "(" + join(*side, "*") + ")";
        side->assign(1, prod);
      }
    }
  }
  SEResult res;
  std::vector<std::string> prog;  // statements
  std::map<std::string, std::string> temp_of;  // operand text -> vertex name
  int ntemp = 0;

  // Step 1: partition the operands of each side by their multilinear symbols.
  for (int sd = 0; sd < 2; ++sd) {
    const std::string& L = sd == 0 ? L1 : L2;
    std::map<std::set<std::string>, std::vector<std::string>> parts;
    for (const Term& t : terms) {
      const auto& v = sd == 0 ? t.a : t.b;
      if (v.empty()) continue;
      Expr oe = parse_expr(v[0]);
      auto syms = ml_symbols(oe, oe.root, L);
      auto& P = parts[syms];
      if (std::find(P.begin(), P.end(), v[0]) == P.end()) P.push_back(v[0]);
    }
    for (auto& kv : parts) {
      const auto& P = kv.second;
      if (P.size() <= kv.first.size()) {
        // Strategy 1: generalised code motion; a bare symbol needs no temporary
        ++res.strategy1;
        for (const std::string& op : P) {
          Expr oe = parse_expr(op);
          if (oe.n[oe.root].kind == Node::SYM) {
            temp_of[op] = op;
          } else {
            std::string t = prefix + "t" + std::to_string(ntemp++) + "[" + L + "]";
            prog.push_back(lstr(with(L)) + ": " + t + " = " + op);
            temp_of[op] = t;
          }
        }
      } else {
        // Strategy 2: expand the operands and factorise by the multilinear symbols
        ++res.strategy2;
        for (const std::string& op : P) temp_of[op] = "";  // marker: expand
      }
    }
  }
  // rewrite terms onto vertices (Strategy 2 operands expand into symbol terms)
  std::vector<Term> vt;
  for (const Term& t : terms) {
    std::vector<std::pair<std::string, std::string>> ea{{"", t.a.empty() ? "1" : t.a[0]}};
    std::vector<std::pair<std::string, std::string>> eb{{"", t.b.empty() ? "1" : t.b[0]}};
    for (int sd = 0; sd < 2; ++sd) {
      auto& ex = sd == 0 ? ea : eb;
      const std::string op = ex[0].second;
      if (op == "1") continue;
      if (temp_of[op].empty()) {
        Expr oe = parse_expr(op);
        std::vector<std::pair<std::string, std::string>> lin;
        if (!linear_split(oe, oe.root, sd == 0 ? L1 : L2, lin, ""))
          throw std::invalid_argument("operand is not linear in its symbols: " + op);
        ex = lin;
      } else {
        ex[0].second = temp_of[op];
      }
    }
    for (auto& pa : ea)
      for (auto& pb : eb) {
        Term n;
        n.coef = t.coef;
        if (!pa.first.empty()) n.coef.push_back(pa.first);
        if (!pb.first.empty()) n.coef.push_back(pb.first);
        n.a = {pa.second};
        n.b = {pb.second};
        n.neg = t.neg;
        vt.push_back(n);
      }
  }
  // Steps 3-4: sharing graph on distinct vertices, merged edges
  std::vector<std::string> left, right;
  auto vid = [](std::vector<std::string>& v, const std::string& s) {
    auto it = std::find(v.begin(), v.end(), s);
    if (it != v.end()) return (int)(it - v.begin());
    v.push_back(s);
    return (int)v.size() - 1;
  };
  std::map<std::pair<int, int>, std::vector<std::string>> edge_coef;  // summed coefficients
  for (const Term& t : vt) {
    int u = vid(left, t.a[0]), w = vid(right, t.b[0]);
    std::string c = t.coef.empty() ? "1" : join(t.coef, "*");
    if (t.neg) c = "(0-1)*" + c;
    edge_coef[{u, w}].push_back(c);
  }
  std::vector<std::pair<int, int>> edges;
  for (auto& kv : edge_coef) edges.push_back(kv.first);
  // Step 5: the ILP is a minimum vertex cover of the bipartite sharing graph.
  // Among minimum covers prefer the larger loop's side: the partner sums (and
  // their coefficient products) then run over the smaller loop.
  auto extent = [&](const std::string& L) {
    auto it = ext.find(L);
    return it == ext.end() ? (int64_t)1 : it->second;
  };
  std::vector<std::pair<int, int>> cover;
  if (extent(L1) >= extent(L2)) {
    cover = min_vertex_cover((int)left.size(), (int)right.size(), edges);
  } else {
    std::vector<std::pair<int, int>> flipped;
    for (auto& ed : edges) flipped.push_back({ed.second, ed.first});
    for (auto& c : min_vertex_cover((int)right.size(), (int)left.size(), flipped)) cover.push_back({1 - c.first, c.second});
  }
  res.cover = (int)cover.size();
  // coefficient temporaries at the outer level (hoisted, shared)
  std::map<std::string, std::string> ctemp;
  int nc = 0;
  auto coef_name = [&](const std::vector<std::string>& cs) -> std::string {
    std::string sum = cs.size() == 1 ? cs[0] : "(" + join(cs, "+") + ")";
    if (sum == "1") return "1";
    Expr ce = parse_expr(sum);
    if (ce.n[ce.root].kind == Node::SYM || ce.n[ce.root].kind == Node::NUM) return sum;
    auto it = ctemp.find(sum);
    if (it != ctemp.end()) return it->second;
    std::string nm = prefix + "c" + std::to_string(nc++);
    if (!outer.empty()) nm += "[" + join(outer, ",") + "]";
    prog.push_back((outer.empty() ? std::string("") : lstr(outer)) + ": " + nm + " = " + sum);
    ctemp[sum] = nm;
    return nm;
  };
  // Step 6 / factorisation: each edge goes to a cover endpoint; T_s sums the partners
  std::vector<char> inL(left.size(), 0), inR(right.size(), 0);
  for (auto& c : cover) (c.first == 0 ? inL : inR)[c.second] = 1;
  std::map<std::pair<int, int>, std::vector<std::string>> sums;  // (side, v) -> partner terms
  for (auto& kv : edge_coef) {
    int u = kv.first.first, w = kv.first.second;
    std::string cn = coef_name(kv.second);
    if (inL[u]) sums[{0, u}].push_back(cn == "1" ? right[w] : cn + "*" + right[w]);
    else sums[{1, w}].push_back(cn == "1" ? left[u] : cn + "*" + left[u]);
  }
  std::vector<std::string> inner;
  int nt = 0;
  for (auto& kv : sums) {
    const bool onL = kv.first.first == 0;
    const std::string s = onL ? left[kv.first.second] : right[kv.first.second];
    const std::string Lo = onL ? L2 : L1;
    std::string T;
    if (kv.second.size() == 1 && parse_expr(kv.second[0]).n.size() == 1) {
      T = kv.second[0];
    } else {
      T = prefix + "T" + std::to_string(nt++) + "[" + Lo + "]";
      prog.push_back(lstr(with(Lo)) + ": " + T + " = " + join(kv.second, " + "));
    }
    inner.push_back(s == "1" ? T : (T == "1" ? s : s + "*" + T));
  }
  prog.push_back(lstr(loops) + ": " + lhs + " += " + join(inner, " + "));
  res.program = join(prog, "; ");
  res.ops = count_program(parse_program(res.program), ext);
  return res;
}

}  // namespace oc
}  // namespace fea
