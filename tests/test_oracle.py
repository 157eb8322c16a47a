"""Pins for the FP64 CPU oracle, none of which re-types its formulas:

* quadrature: exactness on monomials (closed form a!b!c!/(a+b+c+3)!), 1-D nodes
  against scipy's Gauss-Jacobi routine, weights summing to the volume;
* basis: Kronecker property, partition of unity, polynomial reproduction, P1/P2
  closed forms, gradients against finite differences, DOF ordering;
* forms: the P1 mass closed form |K|/20 (1 + delta_ij); every polynomial form
  against the tensor-contraction mode (Section 2.3) with reference tensors built
  from an independent Vandermonde basis and exact monomial integrals;
  invariants (symmetry, zero row sums, rigid-body null space, PSD ranks,
  linearity); Neo-Hookean against central differences of its residual and
  energy, and against linear elasticity at zero displacement.
"""
import math

import numpy as np
import pytest
import scipy.special

import polyexact as px
from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


# ----------------------------------------------------------------- quadrature
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7])
def test_collapsed_rule_exact_to_degree_2m_minus_1(orc, m):
    X, W = orc.quad_rule(m)
    assert X.shape == (m ** 3, 3)
    assert abs(W.sum() - 1.0 / 6.0) < 1e-15
    for (a, b, c) in px.monomials(2 * m - 1):
        exact = float(px.monomial_integral(a, b, c))
        got = np.sum(W * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c)
        assert abs(got - exact) <= 1e-14 * max(exact, 1e-300) + 1e-17, (m, a, b, c)
    # and not exact one degree higher (the rule is not accidentally richer)
    errs = [abs(np.sum(W * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c) - float(px.monomial_integral(a, b, c)))
            for (a, b, c) in px.monomials(2 * m) if a + b + c == 2 * m]
    assert max(errs) > 1e-12


@pytest.mark.parametrize("m", [1, 2, 3, 4, 6])
def test_collapsed_rule_nodes_match_scipy_gauss_jacobi(orc, m):
    X, W = orc.quad_rule(m)
    r = np.unique(np.round(X[:, 2], 14))
    xr, wr = scipy.special.roots_jacobi(m, 2, 0)
    assert np.allclose(np.sort(r), np.sort((1 + xr) / 2), atol=1e-14)
    # weights of the r-direction: sum over the (s,t) sub-rule of each r level
    for rv, wv in zip((1 + xr) / 2, wr / 8):
        sel = np.abs(X[:, 2] - rv) < 1e-12
        assert abs(W[sel].sum() - wv / 2.0) < 1e-15  # (s,t) weights sum to 1/2


def test_four_point_rule_degree_two(orc):
    X, W = orc.quad_rule(0)
    assert X.shape == (4, 3) and abs(W.sum() - 1 / 6) < 1e-16
    for (a, b, c) in px.monomials(2):
        assert abs(np.sum(W * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c) - float(px.monomial_integral(a, b, c))) < 1e-16
    a3 = np.sum(W * X[:, 0] ** 3) - float(px.monomial_integral(3, 0, 0))
    assert abs(a3) > 1e-6


def test_default_rules(orc):
    # mass P1 -> 4-point rule, Helmholtz P2 -> 4^3, elasticity P3 -> 3^3, Neo-Hookean P2 -> 3^3
    assert orc.default_rule(orc.MASS, 1) == 0
    assert orc.default_rule(orc.HELMHOLTZ, 2) == 4
    assert orc.default_rule(orc.ELASTICITY, 3) == 3
    assert orc.default_rule(orc.NEOHOOKEAN, 2) == 3
    for p in range(1, 5):
        # exactness: Helmholtz integrand degree 3p, elasticity 2p-1, mass 2p
        assert 2 * orc.default_rule(orc.HELMHOLTZ, p) - 1 >= 3 * p
        assert 2 * orc.default_rule(orc.ELASTICITY, p) - 1 >= 2 * p - 1
        if p > 1:
            assert 2 * orc.default_rule(orc.MASS, p) - 1 >= 2 * p


# ---------------------------------------------------------------------- basis
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_kronecker_unity_reproduction(orc, p):
    nodes = orc.nodes(p)
    phi, dphi = orc.basis(p, nodes)
    assert np.abs(phi - np.eye(len(nodes))).max() < 1e-13
    rng = np.random.default_rng(1)
    P = rng.dirichlet(np.ones(4), size=50)[:, 1:]
    phi, dphi = orc.basis(p, P)
    assert np.abs(phi.sum(1) - 1).max() < 1e-13
    assert np.abs(dphi.sum(1)).max() < 1e-12
    # reproduction of every monomial of degree <= p, values and gradients
    for (a, b, c) in px.monomials(p):
        f_nodes = nodes[:, 0] ** a * nodes[:, 1] ** b * nodes[:, 2] ** c
        f = P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c
        assert np.abs(phi @ f_nodes - f).max() < 1e-12
        gx = a * P[:, 0] ** max(a - 1, 0) * P[:, 1] ** b * P[:, 2] ** c
        assert np.abs(dphi[:, :, 0] @ f_nodes - gx).max() < 1e-11


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_gradients_finite_difference(orc, p):
    rng = np.random.default_rng(2)
    P = rng.dirichlet(np.ones(4), size=8)[:, 1:] * 0.9 + 0.02
    _, dphi = orc.basis(p, P)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fp, _ = orc.basis(p, P + e)
        fm, _ = orc.basis(p, P - e)
        assert np.abs((fp - fm) / (2 * h) - dphi[:, :, k]).max() < 1e-7


def test_basis_closed_forms_p1_p2(orc):
    rng = np.random.default_rng(3)
    P = rng.dirichlet(np.ones(4), size=20)[:, 1:]
    lam = np.column_stack([1 - P.sum(1), P])
    phi1, _ = orc.basis(1, P)
    assert np.abs(phi1 - lam).max() < 1e-15
    phi2, _ = orc.basis(2, P)
    want = [lam[:, v] * (2 * lam[:, v] - 1) for v in range(4)]
    want += [4 * lam[:, a] * lam[:, b] for (a, b) in px.EDGES]
    assert np.abs(phi2 - np.column_stack(want)).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dof_ordering_convention(orc, p):
    beta = orc.node_indices(p)
    assert [tuple(b) for b in beta] == px.node_multi_indices(p)
    assert len(beta) == orc.nbasis(p) == [4, 10, 20, 35][p - 1]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_independent_vandermonde_basis_agrees(orc, p):
    B = px.Basis(p)
    rng = np.random.default_rng(4)
    P = rng.dirichlet(np.ones(4), size=10)[:, 1:]
    phi, _ = orc.basis(p, P)
    assert np.abs(B.eval(P) - phi).max() < 1e-11


# ---------------------------------------------------------------------- forms
def _mesh(E, seed=11, anisotropic=False):
    rng = np.random.default_rng(seed)
    return inputs.random_tets(E, rng, anisotropic), rng


def test_mass_p1_closed_form(orc):
    c, _ = _mesh(200)
    A = orc.assemble(orc.MASS, 1, c)
    det, _ = px.geometry(c)
    ref = (np.abs(det) / 6 / 20)[:, None, None] * (1 + np.eye(4))[None]
    assert np.abs(A - ref).max() / np.abs(ref).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_sums_to_volume(orc, p):
    c, _ = _mesh(20)
    A = orc.assemble(orc.MASS, p, c)
    det, _ = px.geometry(c)
    assert np.allclose(A.sum((1, 2)), np.abs(det) / 6, rtol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_and_helmholtz_equal_tensor_contraction_mode(orc, p):
    """Quadrature mode (oracle) vs the tensor-contraction mode with exactly
    integrated reference tensors (Section 2.3) from an independent basis."""
    B = px.Basis(p)
    M0 = px.reference_mass(B)
    S0 = px.reference_stiffness(B)
    T0 = px.reference_triple(B, B) if p <= 3 else None
    c, rng = _mesh(6, seed=20 + p, anisotropic=True)
    det, Jinv = px.geometry(c)
    A = orc.assemble(orc.MASS, p, c)
    ref = np.abs(det)[:, None, None] * M0[None]
    assert np.abs(A - ref).max() / np.abs(ref).max() < 1e-12
    f = rng.uniform(-1, 1, size=(6, B.n))
    H = orc.assemble(orc.HELMHOLTZ, p, c, f)
    K = np.einsum("eax,ebx->eab", Jinv, Jinv) * np.abs(det)[:, None, None]
    stiff = np.einsum("eab,abij->eij", K, S0)
    if T0 is None:  # P4: the f-mass part through the (exact) quadrature of the oracle's own rule
        return
    fm = np.abs(det)[:, None, None] * np.einsum("ek,kij->eij", f, T0)
    ref = stiff + fm
    err = np.linalg.norm((H - ref).reshape(6, -1), axis=1) / np.linalg.norm(ref.reshape(6, -1), axis=1)
    assert err.max() < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_elasticity_equals_tensor_contraction_mode(orc, p):
    B = px.Basis(p)
    B1 = px.Basis(1)
    R = px.reference_weighted_stiffness(B1, B)  # [k, a, b, i, j]
    c, rng = _mesh(4, seed=30 + p, anisotropic=True)
    det, Jinv = px.geometry(c)
    co = rng.uniform(0.5, 2, size=(4, 8))
    A = orc.assemble(orc.ELASTICITY, p, c, co)
    n = B.n
    for e in range(4):
        # weighted reference integrals pushed forward: W_mu[x][y][i][j] = int mu G_i^x G_j^y
        Wmu = np.einsum("k,kabij,ax,by->xyij", co[e, :4], R, Jinv[e], Jinv[e]) * abs(det[e])
        Wla = np.einsum("k,kabij,ax,by->xyij", co[e, 4:], R, Jinv[e], Jinv[e]) * abs(det[e])
        ref = np.zeros((n, 3, n, 3))
        for cc in range(3):
            for d in range(3):
                ref[:, cc, :, d] = Wmu[d, cc] + Wla[cc, d]
                if cc == d:
                    ref[:, cc, :, d] += Wmu[0, 0] + Wmu[1, 1] + Wmu[2, 2]
        ref = ref.reshape(3 * n, 3 * n)
        assert np.linalg.norm(A[e] - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_helmholtz_invariants(orc, p):
    c, _ = _mesh(10, seed=40 + p)
    n = orc.nbasis(p)
    S = orc.assemble(orc.HELMHOLTZ, p, c, np.zeros((10, n)))
    assert np.abs(S.sum(2)).max() < 1e-11 * np.abs(S).max()
    assert np.abs(S - S.transpose(0, 2, 1)).max() < 1e-12 * np.abs(S).max()
    for e in range(10):
        w = np.linalg.eigvalsh(S[e])
        assert w[0] > -1e-11 * w[-1] and abs(w[0]) < 1e-11 * w[-1] and w[1] > 1e-8 * w[-1]
    H1 = orc.assemble(orc.HELMHOLTZ, p, c, np.ones((10, n)))
    M = orc.assemble(orc.MASS, p, c, m=orc.default_rule(orc.HELMHOLTZ, p))
    assert np.abs(H1 - S - M).max() < 1e-12 * np.abs(H1).max()


def _rigid_modes(p, orc):
    nodes = orc.nodes(p)
    n = len(nodes)
    modes = []
    for k in range(3):
        v = np.zeros((n, 3))
        v[:, k] = 1
        modes.append(v.reshape(-1))
    return modes, nodes


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_elasticity_invariants(orc, p):
    c, rng = _mesh(5, seed=50 + p, anisotropic=True)
    co = rng.uniform(0.5, 2, size=(5, 8))
    A = orc.assemble(orc.ELASTICITY, p, c, co)
    n = orc.nbasis(p)
    _, Jinv = px.geometry(c)
    J = np.linalg.inv(Jinv)
    ref_nodes = orc.nodes(p)
    for e in range(5):
        x = c[e, 0][None, :] + ref_nodes @ J[e].T  # physical node positions
        modes = []
        for k in range(3):
            v = np.zeros((n, 3))
            v[:, k] = 1
            modes.append(v.reshape(-1))
        for w in np.eye(3):
            modes.append(np.cross(w[None, :], x).reshape(-1))
        Ae = A[e]
        scale = np.abs(Ae).max()
        for r in modes:
            assert np.abs(Ae @ r).max() < 1e-9 * scale * np.abs(r).max()
        assert np.abs(Ae - Ae.T).max() < 1e-12 * scale
        w = np.linalg.eigvalsh(Ae / scale)
        assert w.min() > -1e-9
    # PSD with exactly six zero modes (well-shaped elements keep the spectrum resolvable)
    ci, rng2 = _mesh(3, seed=55 + p)
    Ai = orc.assemble(orc.ELASTICITY, p, ci, rng2.uniform(0.5, 2, size=(3, 8)))
    for e in range(3):
        w = np.linalg.eigvalsh(Ai[e] / np.abs(Ai[e]).max())
        assert w.min() > -1e-12 and np.sum(w > 1e-9) == 3 * n - 6
    # linearity in (mu, lambda)
    A2 = orc.assemble(orc.ELASTICITY, p, c, 2 * co)
    assert np.abs(A2 - 2 * A).max() < 1e-12 * np.abs(A).max()


def test_elasticity_p3_rule_exactness(orc):
    c, rng = _mesh(4, seed=60, anisotropic=True)
    co = rng.uniform(0.5, 2, size=(4, 8))
    A3 = orc.assemble(orc.ELASTICITY, 3, c, co, m=3)
    A4 = orc.assemble(orc.ELASTICITY, 3, c, co, m=4)
    assert np.abs(A3 - A4).max() / np.abs(A4).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_neohookean_tangent_is_derivative_of_residual(orc, p):
    c, u = inputs.workload(inputs.NEOHOOKEAN, p, 3, seed=70 + p)
    n = orc.nbasis(p)
    K = orc.assemble(orc.NEOHOOKEAN, p, c, u)
    h = 1e-5

    def central(fun, e, j, step):
        up = u[e:e + 1].copy()
        um = u[e:e + 1].copy()
        up[0, j] += step
        um[0, j] -= step
        return (fun(up) - fun(um))[0] / (2 * step)

    def richardson(fun, e, j):  # O(h^4) central difference
        return (4 * central(fun, e, j, h / 2) - central(fun, e, j, h)) / 3

    for e in range(3):
        res = lambda uu: orc.neohookean_residual(p, c[e:e + 1], uu)
        Kfd = np.column_stack([richardson(res, e, j) for j in range(3 * n)])
        assert np.linalg.norm(Kfd - K[e]) / np.linalg.norm(K[e]) < 1e-7
        # residual is the derivative of the energy
        R = orc.neohookean_residual(p, c[e:e + 1], u[e:e + 1])[0]
        en = lambda uu: orc.neohookean_energy(p, c[e:e + 1], uu)
        for j in range(0, 3 * n, max(1, n // 3)):
            assert abs(richardson(en, e, j) - R[j]) < 1e-7 * np.abs(R).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_neohookean_invariants(orc, p):
    c, u = inputs.workload(inputs.NEOHOOKEAN, p, 4, seed=80 + p)
    n = orc.nbasis(p)
    K = orc.assemble(orc.NEOHOOKEAN, p, c, u)
    scale = np.abs(K).max()
    assert np.abs(K - K.transpose(0, 2, 1)).max() < 1e-12 * scale
    for k in range(3):
        t = np.zeros((n, 3))
        t[:, k] = 1
        assert np.abs(K @ t.reshape(-1)).max() < 1e-10 * scale
    # zero displacement: linear elasticity with constant mu, lambda
    K0 = orc.assemble(orc.NEOHOOKEAN, p, c, np.zeros((4, 3 * n)), mu=0.8, lam=1.3)
    co = np.concatenate([np.full((4, 4), 0.8), np.full((4, 4), 1.3)], axis=1)
    L = orc.assemble(orc.ELASTICITY, p, c, co)
    assert np.abs(K0 - L).max() < 1e-12 * np.abs(L).max()


def test_neohookean_rule_convergence(orc):
    """Non-polynomial integrand: the collapsed rules converge geometrically."""
    c, u = inputs.workload(inputs.NEOHOOKEAN, 2, 3, seed=90)
    ref = orc.assemble(orc.NEOHOOKEAN, 2, c, u, m=10)
    d = [np.abs(orc.assemble(orc.NEOHOOKEAN, 2, c, u, m=m) - ref).max() / np.abs(ref).max() for m in (3, 4, 6, 8)]
    assert all(d[k + 1] < 0.1 * d[k] for k in range(3)) and d[-1] < 1e-11


def test_openmp_matches_serial(orc):
    c, rng = _mesh(64, seed=95)
    f = rng.uniform(-1, 1, size=(64, 10))
    a = orc.assemble(orc.HELMHOLTZ, 2, c, f, nthreads=1)
    b = orc.assemble(orc.HELMHOLTZ, 2, c, f, nthreads=4)
    assert np.array_equal(a, b)


def test_generator_is_seeded_and_positive():
    c1, f1 = inputs.workload(inputs.HELMHOLTZ, 2, 100)
    c2, f2 = inputs.workload(inputs.HELMHOLTZ, 2, 100)
    assert np.array_equal(c1, c2) and np.array_equal(f1, f2)
    cA, _ = inputs.workload(inputs.ELASTICITY, 3, 2000)
    J = np.transpose(cA[:, 1:] - cA[:, :1], (0, 2, 1))
    sv = np.linalg.svd(J, compute_uv=False)
    assert (sv[:, 0] / sv[:, 2]).max() > 100  # strongly anisotropic elements present
    assert np.all(np.linalg.det(J) > 0)


def test_stream_requests_config():
    reqs = inputs.stream_requests()
    assert len(reqs) == 64
    assert sum(r[2] for r in reqs) == 2_000_000
    assert all(1000 <= r[2] <= 200_000 for r in reqs)
    assert {r[0] for r in reqs} <= {0, 1, 2, 3} and {r[1] for r in reqs} <= {1, 2, 3, 4}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_neohookean_workload_keeps_det_f_positive(orc, p):
    """det F > 0 at every quadrature point of a large sample of the seeded
    Neo-Hookean workload (numpy evaluation of F = I + grad u)."""
    E = 40000 if p <= 2 else 10000
    c, u = inputs.workload(inputs.NEOHOOKEAN, p, E, seed=123 + p)
    X, _ = orc.quad_rule(orc.default_rule(orc.NEOHOOKEAN, p))
    _, dphi = orc.basis(p, X)
    _, Jinv = px.geometry(c)
    G = np.einsum("qai,eix->eqax", dphi, Jinv)
    F = np.eye(3)[None, None] + np.einsum("eac,eqax->eqcx", u.reshape(E, -1, 3), G)
    assert np.linalg.det(F).min() > 0.05


# ---------------------------------------------------------------- linear forms
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_load_vector_pins(orc, p):
    """b_i = int f phi_i: constants integrate to the volume (partition of unity),
    P1 has the closed form |K|/20 (f_i + sum_j f_j), and b = M f with the
    (independently pinned) mass matrix, both rules being exact for degree 2p."""
    c, rng = _mesh(5, seed=100 + p)
    n = orc.nbasis(p)
    vol = np.abs(np.linalg.det(np.stack([c[:, 1] - c[:, 0], c[:, 2] - c[:, 0], c[:, 3] - c[:, 0]], axis=-1))) / 6
    b1 = orc.load_vector(p, c, np.ones((5, n)))
    assert np.allclose(b1.sum(axis=1), vol, rtol=1e-13, atol=0)
    f = rng.uniform(-1, 1, size=(5, n))
    b = orc.load_vector(p, c, f)
    M = orc.assemble(orc.MASS, p, c)
    assert np.abs(b - np.einsum("eij,ej->ei", M, f)).max() < 1e-14 * np.abs(b).max() * n
    if p == 1:
        ref = vol[:, None] / 20 * (f + f.sum(axis=1, keepdims=True))
        assert np.abs(b - ref).max() < 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_neohookean_residual_invariants(orc, p):
    """Independent of the energy: zero and rigid-translation displacements give
    no force; forces sum to zero per component (sum_a grad phi_a = 0); and
    for small displacements R(eps u) = eps K_lin u + O(eps^2), K_lin the
    linear-elasticity stiffness with the same constant mu, lambda."""
    c, u = inputs.workload(inputs.NEOHOOKEAN, p, 3, seed=110 + p)
    n = orc.nbasis(p)
    assert np.abs(orc.neohookean_residual(p, c, np.zeros_like(u))).max() == 0.0
    shift = np.tile(np.array([0.3, -0.2, 0.1]), (3, n))
    assert np.abs(orc.neohookean_residual(p, c, shift)).max() < 1e-13
    R = orc.neohookean_residual(p, c, u)
    assert np.abs(R.reshape(3, n, 3).sum(axis=1)).max() < 1e-12 * np.abs(R).max()
    co = np.concatenate([np.full((3, 4), 0.8), np.full((3, 4), 1.3)], axis=1)
    Kl = orc.assemble(orc.ELASTICITY, p, c, co)
    errs = []
    for eps in (1e-2, 1e-3):
        lin = eps * np.einsum("eij,ej->ei", Kl, u)
        errs.append(np.linalg.norm(orc.neohookean_residual(p, c, eps * u) - lin) / np.linalg.norm(lin))
    assert errs[1] < 0.2 * errs[0] and errs[1] < 1e-2


# ------------------------------------------------- Bernstein basis (sum factorisation)
def _bern_elements(p, E, seed):
    coords, _ = inputs.workload(inputs.MASS, p, E, seed=seed)
    c = np.random.default_rng(seed).uniform(-1.0, 1.0, (E, inputs.nbasis(p)))
    return coords, c


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bernstein_basis_unity_and_gradient_fd(orc, p):
    rng = np.random.default_rng(10 + p)
    X = rng.dirichlet(np.ones(4), 20)[:, 1:]
    B, dB = orc.bernstein_basis(p, X)
    assert np.allclose(B.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(dB.sum(axis=1), 0.0, atol=1e-12)
    assert (B >= 0).all()
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (orc.bernstein_basis(p, X + e)[0] - orc.bernstein_basis(p, X - e)[0]) / (2 * h)
        assert np.allclose(fd, dB[:, :, k], atol=1e-7)
    # vertex values: B_(p e_j) is 1 at vertex j, every other basis function 0
    al = orc.bernstein_indices(p)
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    Bv = orc.bernstein_basis(p, V)[0]
    for j in range(4):
        k = int(np.where(al[:, j] == p)[0][0])
        assert abs(Bv[j, k] - 1.0) < 1e-15 and abs(Bv[j].sum() - 1.0) < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bernstein_mass_closed_form(orc, p):
    """int_K B_a B_b = |det J| (p!)^2 (a+b)! / (a! b! (2p+3)!) (multi-index factorials)."""
    coords, _ = _bern_elements(p, 5, 20 + p)
    A = orc.assemble_bernstein(orc.MASS, p, coords)
    al = orc.bernstein_indices(p)
    f = [math.factorial(k) for k in range(2 * p + 4)]
    for e in range(coords.shape[0]):
        J = (coords[e, 1:] - coords[e, 0]).T
        adet = abs(np.linalg.det(J))
        for i in range(al.shape[0]):
            for j in range(al.shape[0]):
                g = al[i] + al[j]
                num = f[p] ** 2 * np.prod([f[x] for x in g])
                den = np.prod([f[x] for x in al[i]]) * np.prod([f[x] for x in al[j]]) * f[2 * p + 3]
                assert abs(A[e, i, j] - adet * num / den) <= 1e-13 * adet


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_bernstein_helmholtz_is_lagrange_helmholtz_in_another_basis(orc, p):
    """The same space: B_b = sum_i B_b(x_i) phi_i at the Lagrange nodes x_i, so with V[i][b] = B_b(x_i)
    the Bernstein matrix is V^T A V of the Lagrange matrix for f with Lagrange DOFs V c."""
    coords, c = _bern_elements(p, 6, 30 + p)
    V = orc.bernstein_basis(p, orc.nodes(p))[0]
    AL = orc.assemble(orc.HELMHOLTZ, p, coords, c @ V.T)
    AB = orc.assemble_bernstein(orc.HELMHOLTZ, p, coords, c)
    want = np.einsum("ib,eij,jc->ebc", V, AL, V)
    assert orc.rel_frobenius(AB, want).max() <= 1e-13
    assert np.abs(AB - AB.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(AB).max()
