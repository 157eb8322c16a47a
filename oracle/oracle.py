"""ctypes front-end of the FP64 CPU oracle (oracle.c).

Test infrastructure: only tests/, the smoke check and the CPU-baseline leg of
the benchmark load this module.  It compiles oracle.c with the host C compiler
on first use (``build()``), so it works unchanged on x86 and on Arm hosts.

Every function evaluates the quadrature-mode definition of the element matrix
(Section 2.2, equation "quadrature") literally; see oracle.c for the loop nest.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

MASS, HELMHOLTZ, ELASTICITY, NEOHOOKEAN = 0, 1, 2, 3
FORM_NAMES = {MASS: "mass", HELMHOLTZ: "helmholtz", ELASTICITY: "elasticity", NEOHOOKEAN: "neohookean"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile oracle.c into liboracle.so (gcc, OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", "-std=c11",
            "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            lib.oracle_rule_size.argtypes = [ctypes.c_int]
            lib.oracle_quad_rule.argtypes = [ctypes.c_int, D, D]
            lib.oracle_default_rule.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_nbasis.argtypes = [ctypes.c_int]
            lib.oracle_node_indices.argtypes = [ctypes.c_int, I]
            lib.oracle_basis.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D]
            lib.oracle_nodes.argtypes = [ctypes.c_int, D]
            lib.oracle_local_dim.argtypes = [ctypes.c_int, ctypes.c_int]
            lib.oracle_bernstein_indices.argtypes = [ctypes.c_int, I]
            lib.oracle_bernstein_basis.argtypes = [ctypes.c_int, ctypes.c_int, D, D, D]
            lib.oracle_assemble_bernstein.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, D, D,
                                                      D, ctypes.c_int]
            lib.oracle_assemble.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, D, D,
                                            ctypes.c_double, ctypes.c_double, D, ctypes.c_int]
            lib.oracle_neohookean_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, D, D,
                                                       ctypes.c_double, ctypes.c_double, D]
            lib.oracle_neohookean_energy.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, D, D,
                                                     ctypes.c_double, ctypes.c_double, D]
            lib.oracle_load_vector.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, D, D, D]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nbasis(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def local_dim(form, p):
    return 3 * nbasis(p) if form in (ELASTICITY, NEOHOOKEAN) else nbasis(p)


def coeff_len(form, p):
    """Doubles per element in the coefficient array."""
    return {MASS: 0, HELMHOLTZ: nbasis(p), ELASTICITY: 8, NEOHOOKEAN: 3 * nbasis(p)}[form]


def default_rule(form, p):
    """Rule index m (0 = 4-point degree-2 rule, m >= 1 = m^3-point collapsed rule)."""
    return _load().oracle_default_rule(form, p)


def quad_rule(m):
    """(X [Q,3], W [Q]) of rule m on the reference tetrahedron."""
    lib = _load()
    Q = lib.oracle_rule_size(m)
    X = np.zeros((Q, 3))
    W = np.zeros(Q)
    if lib.oracle_quad_rule(m, _ptr(X), _ptr(W)) < 0:
        raise ValueError("bad rule %d" % m)
    return X, W


def node_indices(p):
    n = nbasis(p)
    beta = np.zeros((n, 4), dtype=np.int32)
    _load().oracle_node_indices(p, beta.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return beta


def nodes(p):
    n = nbasis(p)
    X = np.zeros((n, 3))
    _load().oracle_nodes(p, _ptr(X))
    return X


def basis(p, X):
    """(phi [Q,n], dphi [Q,n,3]) of the P_p Lagrange basis at points X [Q,3]."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    Q = X.shape[0]
    n = nbasis(p)
    phi = np.zeros((Q, n))
    dphi = np.zeros((Q, n, 3))
    _load().oracle_basis(p, Q, _ptr(X), _ptr(phi), _ptr(dphi))
    return phi, dphi


def assemble(form, p, coords, coeffs=None, mu=0.8, lam=1.3, m=None, nthreads=1):
    """Element matrices A [E, n, n] (FP64) by the plain quadrature loop nest.

    coords [E,4,3]; coeffs [E, coeff_len] (helmholtz f, elasticity mu[4] lam[4],
    neohookean u[n][3]); mu, lam are the Neo-Hookean constants."""
    lib = _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 12)
    E = coords.shape[0]
    if m is None:
        m = default_rule(form, p)
    cl = coeff_len(form, p)
    if cl:
        coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(E, cl)
        cptr = _ptr(coeffs)
    else:
        cptr = None
    n = local_dim(form, p)
    out = np.zeros((E, n, n))
    bad = lib.oracle_assemble(form, p, m, E, _ptr(coords), cptr, float(mu), float(lam), _ptr(out), int(nthreads))
    if bad < 0:
        raise ValueError("oracle_assemble rejected form=%d p=%d" % (form, p))
    return out


def neohookean_residual(p, coords, u, mu=0.8, lam=1.3, m=None):
    lib = _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 12)
    E = coords.shape[0]
    n = nbasis(p)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(E, 3 * n)
    if m is None:
        m = default_rule(NEOHOOKEAN, p)
    out = np.zeros((E, 3 * n))
    lib.oracle_neohookean_residual(p, m, E, _ptr(coords), _ptr(u), float(mu), float(lam), _ptr(out))
    return out


def load_vector(p, coords, f, m=None):
    """Helmholtz right-hand side b_i = int f phi_i, f in P_p given by its DOFs [E, n]; [E, n]."""
    lib = _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 12)
    E = coords.shape[0]
    n = nbasis(p)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(E, n)
    if m is None:
        m = default_rule(HELMHOLTZ, p)
    out = np.zeros((E, n))
    lib.oracle_load_vector(p, m, E, _ptr(coords), _ptr(f), _ptr(out))
    return out


def neohookean_energy(p, coords, u, mu=0.8, lam=1.3, m=None):
    lib = _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 12)
    E = coords.shape[0]
    n = nbasis(p)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(E, 3 * n)
    if m is None:
        m = default_rule(NEOHOOKEAN, p)
    out = np.zeros(E)
    lib.oracle_neohookean_energy(p, m, E, _ptr(coords), _ptr(u), float(mu), float(lam), _ptr(out))
    return out


def bernstein_indices(p):
    """Multi-indices (a0, a1, a2, a3), |a| = p, of the Bernstein basis in its DOF order [n, 4]."""
    n = nbasis(p)
    a = np.zeros((n, 4), dtype=np.int32)
    _load().oracle_bernstein_indices(p, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return a


def bernstein_basis(p, X):
    """(B [Q,n], dB/dX [Q,n,3]) of the degree-p Bernstein basis at points X [Q,3]."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    Q = X.shape[0]
    n = nbasis(p)
    B = np.zeros((Q, n))
    dB = np.zeros((Q, n, 3))
    _load().oracle_bernstein_basis(p, Q, _ptr(X), _ptr(B), _ptr(dB))
    return B, dB


def assemble_bernstein(form, p, coords, c=None, m=None, nthreads=1):
    """Mass or Helmholtz element matrices [E, n, n] in the Bernstein basis; c [E, n]
    holds the Bernstein coefficients of f (Helmholtz)."""
    lib = _load()
    coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1, 12)
    E = coords.shape[0]
    n = nbasis(p)
    if m is None:
        m = default_rule(HELMHOLTZ, p)
    cptr = None
    if form == HELMHOLTZ:
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(E, n)
        cptr = _ptr(c)
    out = np.zeros((E, n, n))
    if lib.oracle_assemble_bernstein(form, p, m, E, _ptr(coords), cptr, _ptr(out), int(nthreads)) < 0:
        raise ValueError("oracle_assemble_bernstein rejected form=%d p=%d" % (form, p))
    return out


def max_threads():
    return _load().oracle_max_threads()


def rel_frobenius(A, Aref):
    """Per-element relative Frobenius error ||A - Aref||_F / ||Aref||_F."""
    A = np.asarray(A, dtype=np.float64).reshape(Aref.shape[0], -1)
    R = np.asarray(Aref, dtype=np.float64).reshape(Aref.shape[0], -1)
    return np.linalg.norm(A - R, axis=1) / np.linalg.norm(R, axis=1)
