"""Test-side polynomial machinery for pinning the oracle.

Builds the equispaced Lagrange basis on the reference tetrahedron by inverting
the monomial Vandermonde matrix (a construction independent of the oracle's
Silvester product formula) and integrates products of basis functions exactly
with the closed form  int_T x^a y^b z^c = a! b! c! / (a+b+c+3)!.
"""
import itertools
from fractions import Fraction
from math import factorial

import numpy as np

EDGES = [(2, 3), (1, 3), (1, 2), (0, 3), (0, 2), (0, 1)]


def monomial_integral(a, b, c):
    return Fraction(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))


def node_multi_indices(p):
    """Barycentric indices of the P_p nodes in the DOF convention: vertices,
    edges (2,3),(1,3),(1,2),(0,3),(0,2),(0,1) running low -> high vertex,
    faces opposite vertices 0..3, interior; inside an entity the index of the
    entity's last vertex varies slowest."""
    out = []
    for v in range(4):
        b = [0, 0, 0, 0]
        b[v] = p
        out.append(tuple(b))
    for (v0, v1) in EDGES:
        for m in range(1, p):
            b = [0, 0, 0, 0]
            b[v0], b[v1] = p - m, m
            out.append(tuple(b))
    for v in range(4):
        f = [c for c in range(4) if c != v]
        cand = []
        for b0 in range(1, p):
            for b1 in range(1, p):
                b2 = p - b0 - b1
                if b2 >= 1:
                    cand.append((b2, b1, b0))
        for (b2, b1, b0) in sorted(cand):
            b = [0, 0, 0, 0]
            b[f[0]], b[f[1]], b[f[2]] = b0, b1, b2
            out.append(tuple(b))
    cand = []
    for b in itertools.product(range(1, p), repeat=4):
        if sum(b) == p:
            cand.append(b[::-1])
    for key in sorted(cand):
        out.append(tuple(key[::-1]))
    return out


def monomials(d):
    return [(a, b, c) for a in range(d + 1) for b in range(d + 1 - a) for c in range(d + 1 - a - b)]


class Basis:
    """Lagrange basis of degree p as coefficient vectors over monomials."""

    def __init__(self, p):
        self.p = p
        self.mons = monomials(p)
        beta = node_multi_indices(p)
        self.nodes = np.array([[b[1] / p, b[2] / p, b[3] / p] for b in beta])
        V = np.array([[x ** a * y ** b * z ** c for (a, b, c) in self.mons] for (x, y, z) in self.nodes])
        self.C = np.linalg.solve(V, np.eye(len(self.mons))).T  # C[i] = coefficients of phi_i
        self.n = len(self.mons)

    def grad(self, k):
        """Coefficients of d phi_i / dX_k over the same monomial list."""
        idx = {m: i for i, m in enumerate(self.mons)}
        G = np.zeros_like(self.C)
        for j, m in enumerate(self.mons):
            if m[k] == 0:
                continue
            mm = list(m)
            mm[k] -= 1
            G[:, idx[tuple(mm)]] += m[k] * self.C[:, j]
        return G

    def eval(self, X):
        X = np.atleast_2d(X)
        M = np.array([[x ** a * y ** b * z ** c for (a, b, c) in self.mons] for (x, y, z) in X])
        return M @ self.C.T


def moment_matrix(mons_a, mons_b):
    return np.array([[float(monomial_integral(a[0] + b[0], a[1] + b[1], a[2] + b[2])) for b in mons_b]
                     for a in mons_a])


def moment_tensor(mons_a, mons_b, mons_c):
    T = np.zeros((len(mons_a), len(mons_b), len(mons_c)))
    for i, a in enumerate(mons_a):
        for j, b in enumerate(mons_b):
            for k, c in enumerate(mons_c):
                T[i, j, k] = float(monomial_integral(a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]))
    return T


def reference_mass(B):
    M = moment_matrix(B.mons, B.mons)
    return B.C @ M @ B.C.T


def reference_stiffness(B):
    """S[a][b][i][j] = int dphi_i/dX_a dphi_j/dX_b."""
    M = moment_matrix(B.mons, B.mons)
    G = [B.grad(k) for k in range(3)]
    S = np.zeros((3, 3, B.n, B.n))
    for a in range(3):
        for b in range(3):
            S[a, b] = G[a] @ M @ G[b].T
    return S


def reference_triple(Bk, B):
    """T[k][i][j] = int psi_k phi_i phi_j (psi from basis Bk)."""
    T = moment_tensor(Bk.mons, B.mons, B.mons)
    return np.einsum("km,mab,ia,jb->kij", Bk.C, T, B.C, B.C)


def reference_weighted_stiffness(Bk, B):
    """R[k][a][b][i][j] = int psi_k dphi_i/dX_a dphi_j/dX_b."""
    T = moment_tensor(Bk.mons, B.mons, B.mons)
    G = [B.grad(k) for k in range(3)]
    R = np.zeros((Bk.n, 3, 3, B.n, B.n))
    for a in range(3):
        for b in range(3):
            R[:, a, b] = np.einsum("km,mxy,ix,jy->kij", Bk.C, T, G[a], G[b])
    return R


def geometry(coords):
    """(det J [E], Jinv [E,3,3]) with J[:, r, c] = x_{c+1,r} - x_{0,r}."""
    J = np.transpose(coords[:, 1:, :] - coords[:, :1, :], (0, 2, 1))
    return np.linalg.det(J), np.linalg.inv(J)
