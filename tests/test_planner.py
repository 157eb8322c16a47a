"""Pins for the planner's operation-count algorithm (host logic, no GPU):

* the paper's worked examples: Figure "multi_loopnest" (4 JI -> 3 JI -> I + 2 JI),
  Figure "poisson" (18 IJK naive, I(9J + 6K + 4JK) after sharing elimination),
  Figure "loopnest_rednored", the increase factor iota (3 and 6, Section 4.2);
* every count equals the tally of executing the program (oracle/opcount_ref);
* sharing elimination preserves the value of the expression (executed);
* the vertex cover of step 5 equals brute force on random bipartite graphs;
* Algorithm 3 equals brute force over every subset of monomials.
"""
import random

import numpy as np
import pytest

import paper_1604_05872_gb300 as fea
from oracle import opcount_ref as ref
from paper_1604_05872_gb300 import build as fbuild


@pytest.fixture(scope="module", autouse=True)
def lib():
    fbuild.build()
    return fea.load()


def rand_env(seed=0):
    rng = random.Random(seed)
    cache = {}

    def make(name):
        def f(ix):
            key = (name, ix)
            if key not in cache:
                cache[key] = rng.uniform(-1, 1)
            return cache[key]
        return f

    class Env(dict):
        def __missing__(self, k):
            self[k] = make(k)
            return self[k]
    return Env()


def check_tally(program, ext):
    n = fea.opcount_program(program, ext)
    _, tally = ref.execute(program, ext, rand_env())
    assert n == tally, (program, n, tally)
    return n


# ------------------------------------------------------------ Figure multi_loopnest
def test_multi_loopnest_counts():
    J, I = 7, 5
    ext = {"j": J, "i": I}
    assert check_tally("j,i: a[j,i] += b[j]*c[i] + b[j]*d[i]", ext) == 4 * J * I
    assert check_tally("j,i: a[j,i] += b[j]*(c[i] + d[i])", ext) == 3 * J * I
    assert check_tally("i: t[i] = c[i] + d[i]; j,i: a[j,i] += b[j]*t[i]", ext) == I + 2 * J * I


def test_multi_loopnest_sharing_elimination_reaches_optimal_form():
    J, I = 7, 5
    ext = {"j": J, "i": I}
    prog, ops, cover = fea.sharing_elimination("a[j,i]", "b[j]*c[i] + b[j]*d[i]", ["j", "i"], ext)
    assert ops == I + 2 * J * I and cover == 1
    check_tally(prog, ext)
    env = rand_env(1)
    a0, _ = ref.execute("j,i: a[j,i] += b[j]*c[i] + b[j]*d[i]", ext, env)
    a1, _ = ref.execute(prog, ext, env)
    for j in range(J):
        for i in range(I):
            assert abs(a0[("a", (j, i))] - a1[("a", (j, i))]) < 1e-12


# ------------------------------------------------------------------- Figure poisson
POISSON = ("((z0[e]*a[i,k] + z2[e]*b[i,k])*(z0[e]*c[i,j] + z2[e]*d[i,j]) + "
           "(z1[e]*a[i,k] + z3[e]*b[i,k])*(z1[e]*c[i,j] + z3[e]*d[i,j]))*W[i]*det[e]")
POISSON_B = ("e,i,k: t0[k] = z0[e]*a[i,k] + z2[e]*b[i,k]; e,i,k: t1[k] = z1[e]*a[i,k] + z3[e]*b[i,k]; "
             "e,i,j: t2[j] = (z0[e]*c[i,j] + z2[e]*d[i,j])*(W[i]*det[e]); "
             "e,i,j: t3[j] = (z1[e]*c[i,j] + z3[e]*d[i,j])*(W[i]*det[e]); "
             "e,i,j,k: A[e,j,k] += t0[k]*t2[j] + t1[k]*t3[j]")


def paper_values():
    """Values the paper prints (tests/golden/paper_values.json, each with its citation)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("E,I,J,K", [(1, 3, 3, 3), (2, 4, 3, 5), (1, 6, 6, 6)])
def test_poisson_counts(E, I, J, K):
    g = paper_values()["poisson_2d"]
    ext = {"e": E, "i": I, "j": J, "k": K}
    assert check_tally("e,i,j,k: A[e,j,k] += " + POISSON, ext) == E * I * J * K * g["naive_ops_per_eijk"]
    # the listing of Figure "poisson" (b): 6 per k, 9 per j (W_i det counted once), 4 per (j, k)
    c = g["se_coefficients_of_the_listing"]
    assert check_tally(POISSON_B, ext) == E * I * (c["K"] * K + c["J"] * J + c["JK"] * J * K)
    # the caption's printed count, with its J and K labels swapped back, is the same polynomial
    pr = g["se_coefficients_as_printed"]
    assert (pr["J"], pr["K"], pr["JK"]) == (c["K"], c["J"], c["JK"])
    if J == K:  # where the example lives, the printed count holds as printed
        assert check_tally(POISSON_B, ext) == E * I * (pr["J"] * J + pr["K"] * K + pr["JK"] * J * K)


@pytest.mark.parametrize("E,I,J,K", [(1, 3, 3, 3), (2, 4, 3, 5), (1, 2, 6, 4)])
def test_poisson_sharing_elimination(E, I, J, K):
    ext = {"e": E, "i": I, "j": J, "k": K}
    prog, ops, cover = fea.sharing_elimination("A[e,j,k]", POISSON, ["e", "i", "j", "k"], ext)
    assert cover == paper_values()["poisson_2d"]["vertex_cover"]  # two products per innermost iteration
    assert ops == check_tally(prog, ext)
    # generalized code motion hoists W_i det to the i loop (1 per i) and the
    # coefficient products run over the smaller linear loop
    assert ops == E * I * (1 + 6 * max(J, K) + 8 * min(J, K) + 4 * J * K)
    assert ops <= E * I * (6 * K + 9 * J + 4 * J * K) + E * I
    assert ops < E * I * J * K * 18
    env = rand_env(2)
    a0, _ = ref.execute("e,i,j,k: A[e,j,k] += " + POISSON, ext, env)
    a1, _ = ref.execute(prog, ext, env)
    for key, v in a0.items():
        assert abs(v - a1[key]) < 1e-10 * max(1.0, abs(v))


# ------------------------------------------------------- Figure loopnest_rednored
def test_reduction_pre_evaluation_counts():
    E, I, K = 10, 6, 4
    ext = {"e": E, "i": I, "k": K}
    red = "e,i,k: a[e,k] += d[e]*b[i,k]*c[i] + d[e]*b[i,k]*d2[i]"
    pre = "i,k: t[k] += b[i,k]*(c[i] + d2[i]); e,k: a[e,k] = d[e]*t[k]"
    n_red, n_pre = check_tally(red, ext), check_tally(pre, ext)
    assert n_pre == I * K * 3 + E * K and n_pre < n_red
    env = rand_env(3)
    s0, _ = ref.execute(red, ext, env)
    s1, _ = ref.execute(pre, ext, env)
    for e in range(E):
        for k in range(K):
            assert abs(s0[("a", (e, k))] - s1[("a", (e, k))]) < 1e-10


def test_increase_factor():
    # Section 4.2: iota = 3 for n = 3, k = 1 and iota = 6 for k = 2
    for ex in paper_values()["increase_factor"]["examples"]:
        assert fea.increase_factor(ex["n"], ex["k"]) == ex["iota"]
    assert fea.increase_factor(10, 1) == 10 and fea.increase_factor(4, 0) == 1
    from math import comb
    for n in range(1, 9):
        for k in range(0, 4):
            assert fea.increase_factor(n, k) == comb(n + k - 1, k)


# ------------------------------------------------------------------ vertex cover
def test_vertex_cover_equals_bruteforce():
    rng = random.Random(7)
    for trial in range(300):
        nl, nr = rng.randint(1, 6), rng.randint(1, 6)
        edges = sorted({(rng.randrange(nl), rng.randrange(nr)) for _ in range(rng.randint(0, nl * nr))})
        assert fea.vertex_cover(nl, nr, edges) == ref.min_vertex_cover_bruteforce(nl, nr, edges), (nl, nr, edges)


# --------------------------------------------------------- forms and Algorithm 3
@pytest.mark.parametrize("form", [0, 1, 2, 3])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_algorithm3_equals_bruteforce(form, p):
    th = fea.theta(form, p)
    for budget in (0, 256 * 1024, 96 * 1024, 16 * 1024, 1024):
        for prec in (fea.PREC_FP32, fea.PREC_FP64):
            word = 4 if prec == fea.PREC_FP32 else 8
            mask, cost = fea.algorithm3(form, p, prec, budget)
            b = budget or 232448
            best = ref.algorithm3_bruteforce([(se, pre, tw * word) for (se, pre, tw) in th], b)
            assert cost == best, (form, p, budget, prec)
            assert sum(th[i][2] * word for i in range(len(th)) if mask >> i & 1) <= b


def test_theta_pre_structure():
    # Helmholtz P2: stiffness rho = 6 (symmetric 3x3 geometry, 3 in 2-D), iota = 1;
    # f-mass rho = 1, iota = n = 10; tables = 6 + 10 = the kernel's reference terms
    th = fea.theta(1, 2)
    assert th[0][2] == 6 * 100 and th[1][2] == 10 * 100
    # the paper's rho: 1 for a mass monomial (Helmholtz's f-mass term above: one table per coefficient
    # DOF), 3 for the 2-D Poisson geometry tensor (d (d + 1) / 2 with d = 2; 6 for d = 3 here)
    rho = paper_values()["rho"]
    for p in (1, 2, 3):
        nn = fea.local_dim(0, p) ** 2
        assert fea.theta(0, p)[0][2] == rho["mass_monomial"] * nn  # mass: one table
    # stiffness: one table per entry of the symmetric d x d geometry tensor, d (d + 1) / 2:
    # the paper's 3 in two dimensions, 6 here in three
    assert rho["poisson_2d"] == 2 * 3 // 2 and th[0][2] == (3 * 4 // 2) * 100
    assert fea.plan(1, 2)["ref_terms"] == 16
    # iota >= Q makes pre-evaluation unprofitable: elasticity P1 (iota = 4, Q = 1)
    se, pre, _ = fea.theta(2, 1)[0]
    assert pre > se
    # Neo-Hookean has no pre-evaluated form
    assert fea.theta(3, 2)[0][1] == -1


def test_form_programs_count_equals_execution():
    """The sharing-elimination program of a real monomial, on tiny extents."""
    ext = {"e": 1, "q": 2, "j": 3, "k": 3}
    G = lambda x, L: "(" + " + ".join("Ji%d%d[e]*D%d[q,%s]" % (a, x, a, L) for a in range(3)) + ")"
    stiff = "(" + " + ".join(G(x, "j") + "*" + G(x, "k") for x in range(3)) + ")*W[q]*det[e]"
    prog, ops, cover = fea.sharing_elimination("A[e,j,k]", stiff, ["e", "q", "j", "k"], ext)
    assert ops == check_tally(prog, ext)
    assert cover == 3  # G_j . G_k: three products per entry
    env = rand_env(4)
    a0, _ = ref.execute("e,q,j,k: A[e,j,k] += " + stiff, ext, env)
    a1, _ = ref.execute(prog, ext, env)
    for key, v in a0.items():
        assert abs(v - a1[key]) < 1e-10 * max(1.0, abs(v))


def test_variant_choice_follows_algorithm3():
    for form in (0, 1, 2):
        for p in range(1, 5):
            mask, _ = fea.algorithm3(form, p)
            n = len(fea.theta(form, p))
            v = fea.plan(form, p)["variant"]
            if mask == (1 << n) - 1:
                assert v == fea.VARIANT_PRE
            elif mask == 0:
                assert v == fea.VARIANT_SE
    assert fea.plan(3, 2)["variant"] == fea.VARIANT_SE
