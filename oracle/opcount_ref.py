"""Reference checks for the planner's operation-count algorithm.

Test infrastructure: brute force and direct execution, sharing no code with
the library's C++ planner.

* ``execute``: runs a loop-nest program of the planner's expression language
  on numbers, tallying every executed + - * (a '+=' adds one) with the
  convention of Figure "poisson": inside one iteration of a loop body a
  sub-expression already evaluated is reused, not recounted.  The tally is
  measured, not derived from the program text.
* ``min_vertex_cover_bruteforce``: the ILP of Algorithm 1 step 5 by
  enumerating every vertex subset.
* ``algorithm3_bruteforce``: the cheapest admissible set of pre-evaluated
  monomials by enumerating every subset (Section 4.1).
"""
import itertools
import re

_TOK = re.compile(r"\s*([A-Za-z_][A-Za-z0-9_.]*|[0-9][0-9.]*|\+=|[-+*()=\[\],:;])")


def _tokens(s):
    pos, out = 0, []
    s = s.strip()
    while pos < len(s):
        m = _TOK.match(s, pos)
        if not m:
            raise ValueError("bad character at %r" % s[pos:])
        out.append(m.group(1))
        pos = m.end()
    return out


class _P:
    def __init__(self, toks):
        self.t, self.i = toks, 0

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else None

    def take(self, x=None):
        v = self.peek()
        if x is not None and v != x:
            raise ValueError("expected %r got %r" % (x, v))
        self.i += 1
        return v

    def expr(self):
        node = ["+", [(1, self.term())]]
        while self.peek() in ("+", "-"):
            sgn = 1 if self.take() == "+" else -1
            node[1].append((sgn, self.term()))
        return node if len(node[1]) > 1 else node[1][0][1]

    def term(self):
        fs = [self.atom()]
        while self.peek() == "*":
            self.take()
            fs.append(self.atom())
        return ["*", fs] if len(fs) > 1 else fs[0]

    def atom(self):
        if self.peek() == "(":
            self.take()
            e = self.expr()
            self.take(")")
            return e
        name = self.take()
        if name[0].isdigit():
            return ["num", float(name)]
        idx = []
        if self.peek() == "[":
            self.take()
            idx.append(self.take())
            while self.peek() == ",":
                self.take()
                idx.append(self.take())
            self.take("]")
        return ["sym", name, tuple(idx)]


def _key(n):
    if n[0] == "num":
        return repr(n[1])
    if n[0] == "sym":
        return n[1] + "[" + ",".join(n[2]) + "]"
    if n[0] == "*":
        return "(" + "*".join(_key(c) for c in n[1]) + ")"
    return "(" + "".join(("+" if s > 0 else "-") + _key(c) for s, c in n[1]) + ")"


def parse_program(text):
    prog = []
    for st in text.split(";"):
        st = st.strip()
        if not st:
            continue
        loops, rest = st.split(":", 1)
        loops = [x.strip() for x in loops.split(",") if x.strip()]
        accum = "+=" in rest
        lhs, rhs = rest.split("+=" if accum else "=", 1)
        p = _P(_tokens(rhs))
        e = p.expr()
        lp = _P(_tokens(lhs))
        tgt = lp.atom()
        prog.append((loops, tgt, accum, e))
    return prog


def _nest(prog):
    """Group consecutive statements into a loop tree (shared outer loops)."""
    def build(stmts, depth):
        items, k = [], 0
        while k < len(stmts):
            loops = stmts[k][0]
            if len(loops) == depth:
                items.append(("stmt", stmts[k]))
                k += 1
                continue
            l = loops[depth]
            j = k
            while j < len(stmts) and len(stmts[j][0]) > depth and stmts[j][0][depth] == l:
                j += 1
            items.append(("loop", l, build(stmts[k:j], depth + 1)))
            k = j
        return items
    return build(prog, 0)


def execute(text, extents, env):
    """Run a program; env maps symbol name -> function(index tuple) -> float.
    Returns (store of assigned arrays, operation tally)."""
    prog = parse_program(text)
    store = {}
    tally = [0]
    idx = {}

    def val(n, memo):
        k = _key(n)
        if n[0] == "num":
            return n[1]
        if n[0] == "sym":
            key = (n[1], tuple(idx[i] for i in n[2]))
            if key in store:
                return store[key]
            return env[n[1]](tuple(idx[i] for i in n[2]))
        if k in memo:
            return memo[k]
        if n[0] == "*":
            v = 1.0
            for c in n[1]:
                v *= val(c, memo)
            tally[0] += len(n[1]) - 1
        else:
            v = 0.0
            for s, c in n[1]:
                v += s * val(c, memo)
            tally[0] += len(n[1]) - 1
        memo[k] = v
        return v

    def run(items):
        body = [it for it in items if it[0] == "stmt"]
        memo = {}
        for it in items:
            if it[0] == "stmt":
                loops, tgt, accum, e = it[1]
                v = val(e, memo)
                key = (tgt[1], tuple(idx[i] for i in tgt[2]))
                if accum:
                    store[key] = store.get(key, 0.0) + v
                    tally[0] += 1
                else:
                    store[key] = v
            else:
                _, l, inner = it
                for x in range(extents[l]):
                    idx[l] = x
                    run(inner)
                del idx[l]
        return body

    run(_nest(prog))
    return store, tally[0]


def min_vertex_cover_bruteforce(nl, nr, edges):
    verts = [(0, u) for u in range(nl)] + [(1, v) for v in range(nr)]
    for k in range(len(verts) + 1):
        for sub in itertools.combinations(verts, k):
            s = set(sub)
            if all((0, u) in s or (1, v) in s for (u, v) in edges):
                return k
    return len(verts)


def algorithm3_bruteforce(thetas, budget_words_bytes):
    """thetas: [(se, pre, table_bytes)] per monomial (pre < 0: not admissible).
    Returns the minimal cost over every admissible subset pre-evaluated."""
    best = None
    n = len(thetas)
    for mask in range(1 << n):
        cost, mem, ok = 0, 0, True
        for i, (se, pre, tb) in enumerate(thetas):
            if mask >> i & 1:
                if pre < 0:
                    ok = False
                    break
                cost += pre
                mem += tb
            else:
                cost += se
        if ok and mem <= budget_words_bytes and (best is None or cost < best):
            best = cost
    return best
