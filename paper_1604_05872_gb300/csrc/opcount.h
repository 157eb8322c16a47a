// Operation counting and the transformation algorithms of Sections 3-4 on a
// small expression language (the planner's IR).
//
//   program   := stmt (';' stmt)*
//   stmt      := loops ':' lhs ('=' | '+=') expr
//   loops     := index (',' index)*          enclosing loops, outermost first
//   expr      := term (('+' | '-') term)*
//   term      := atom ('*' atom)*
//   atom      := symbol ('[' index (',' index)* ']')? | number | '(' expr ')'
//
// Counting (Definition 8): every binary + - * is one operation, '+=' adds one;
// a statement costs its operations times the product of its loop extents; a
// non-trivial sub-expression that occurs more than once among the statements
// of one loop body is counted once (the convention of Figure "poisson").
#pragma once
#include <cstdint>
#include <map>
#include <set>
#include <string>
#include <vector>

namespace fea {
namespace oc {

struct Node {
  enum Kind { SYM, NUM, ADD, MUL } kind = SYM;
  std::string name;              // SYM: symbol name, NUM: literal
  std::vector<std::string> idx;  // SYM: indices
  std::vector<int> ch;           // ADD/MUL operands (n-ary, >= 2)
  std::vector<int> neg;          // ADD: operand is subtracted
};

struct Expr {
  std::vector<Node> n;
  int root = -1;
  std::string str(int i) const;             // canonical text of a sub-expression
  std::string str() const { return str(root); }
  std::set<std::string> deps(int i) const;  // indices a sub-expression depends on
  int64_t ops(int i) const;                 // operations without any sharing
};

Expr parse_expr(const std::string& s);

struct Stmt {
  std::vector<std::string> loops;
  std::string lhs;
  bool accum = false;
  Expr rhs;
};
std::vector<Stmt> parse_program(const std::string& s);
std::map<std::string, int64_t> parse_extents(const std::string& s);  // "e:1,i:64,j:10,k:10"

int64_t count_program(const std::vector<Stmt>& prog, const std::map<std::string, int64_t>& ext);

// Minimum vertex cover of a bipartite graph (left vertices 0..nl-1, right
// 0..nr-1) by maximum matching and Koenig's theorem.  Returns the cover as
// (side, vertex) pairs with side 0 = left.
std::vector<std::pair<int, int>> min_vertex_cover(int nl, int nr, const std::vector<std::pair<int, int>>& edges);

// Algorithm 1 (sharing elimination) on `A[...] += expr` inside the loop nest
// `loops` (outermost first; the last two are the linear test/trial loops, the
// others order-free or reduction loops).  Returns the transformed program as
// text (same language, executable) and its operation count.
struct SEResult {
  std::string program;
  int64_t ops = 0;
  int cover = 0;        // size of the vertex cover = products per innermost iteration
  int strategy1 = 0;    // operand partitions scheduled by code motion only
  int strategy2 = 0;    // operand partitions expanded and factorised
};
SEResult sharing_elimination(const std::string& lhs, const std::string& expr, const std::vector<std::string>& loops,
                             const std::map<std::string, int64_t>& ext, const std::string& prefix = "");

// Section 4.2: increase factor iota = C(n + k - 1, k) of pre-evaluation.
int64_t increase_factor(int64_t n, int64_t k);

}  // namespace oc
}  // namespace fea
