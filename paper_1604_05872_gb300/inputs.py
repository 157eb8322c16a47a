"""Seeded synthetic workloads (random affine tetrahedra and coefficient DOFs).

This module only draws random numbers; it holds none of the assembly
arithmetic, so the CUDA path and the CPU oracle can both be fed from it.

Element recipe (stands in for the paper's 4374-tet Firedrake mesh, Section 7,
which is not available here):
  1. unit tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1), each vertex jittered by
     U[-0.1, 0.1]^3;
  2. uniform scale U[0.5, 2] (Neo-Hookean displacements scale with it);
  3. optionally an anisotropic squeeze diag(1, 1, 10^-U[0,3]) (aspect ratio up
     to 1e3);
  4. a Haar-random rotation (normalised Gaussian quaternion);
  5. a translation U[-10, 10]^3.
The jitter moves a vertex by at most 0.17 while the smallest height of the unit
tetrahedron is 0.577, so det J > 0 for every element (asserted).
"""
import math

import numpy as np

SEED = 160405872

MASS, HELMHOLTZ, ELASTICITY, NEOHOOKEAN = 0, 1, 2, 3
FORMS = {"mass": MASS, "helmholtz": HELMHOLTZ, "elasticity": ELASTICITY, "neohookean": NEOHOOKEAN}
NEO_MU, NEO_LAMBDA = 0.8, 1.3


def nbasis(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


def coeff_len(form, p):
    """Doubles per element of the coefficient array."""
    return {MASS: 0, HELMHOLTZ: nbasis(p), ELASTICITY: 8, NEOHOOKEAN: 3 * nbasis(p)}[form]


def _rotations(rng, E):
    q = rng.standard_normal((E, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((E, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_tets(E, rng, anisotropic=False):
    """coords [E, 4, 3] float64 of E random positively oriented tetrahedra."""
    return _tets(E, rng, anisotropic)[0]


def _tets(E, rng, anisotropic):
    base = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    v = base[None, :, :] + rng.uniform(-0.1, 0.1, size=(E, 4, 3))
    scale = rng.uniform(0.5, 2.0, size=(E, 1, 1))
    v *= scale
    if anisotropic:
        v[:, :, 2] *= 10.0 ** (-rng.uniform(0.0, 3.0, size=(E, 1)))
    R = _rotations(rng, E)
    v = np.einsum("eij,ekj->eki", R, v)
    v += rng.uniform(-10.0, 10.0, size=(E, 1, 3))
    d = v[:, 1:, :] - v[:, :1, :]
    det = np.einsum("ei,ei->e", d[:, 0], np.cross(d[:, 1], d[:, 2]))
    assert np.all(det > 0), "generator produced an inverted tetrahedron"
    return np.ascontiguousarray(v), scale.reshape(E)


def random_coeffs(form, p, E, rng, scale=None):
    """Coefficient DOFs [E, coeff_len] for one form (None for mass).

    Neo-Hookean displacements are U[-0.05, 0.05] times the element's scale
    factor (and times (2/p)^3 above P2), so that the displacement gradient has
    the same distribution on every element size and J = det F stays positive."""
    if form == MASS:
        return None
    if form == HELMHOLTZ:
        return rng.uniform(-1.0, 1.0, size=(E, nbasis(p)))
    if form == ELASTICITY:
        return rng.uniform(0.5, 2.0, size=(E, 8))
    if form == NEOHOOKEAN:
        amp = 0.05 * min(1.0, (2.0 / p) ** 3)
        u = rng.uniform(-amp, amp, size=(E, 3 * nbasis(p)))
        if scale is not None:
            u *= np.asarray(scale).reshape(E, 1)
        return u
    raise ValueError(form)


def workload(form, p, E, seed=SEED, anisotropic=None):
    """(coords [E,4,3], coeffs [E,clen] or None) for one form/degree.

    Elasticity uses the anisotropic (aspect ratio up to 1e3) elements by
    default, as its benchmark configuration asks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if anisotropic is None:
        anisotropic = form == ELASTICITY
    coords, scale = _tets(E, rng, anisotropic)
    coeffs = random_coeffs(form, p, E, rng, scale)
    return coords, coeffs


def coeff_array(form, p, coeffs, mu=NEO_MU, lam=NEO_LAMBDA):
    """Flat float64 coefficient buffer as the library expects it: the
    per-element DOFs, and for Neo-Hookean the two material constants
    (mu, lambda) appended after the last element."""
    if form == MASS:
        return np.zeros(0)
    flat = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(-1)
    if form == NEOHOOKEAN:
        flat = np.concatenate([flat, [mu, lam]])
    return flat


def stream_requests(seed=SEED, nreq=64, total=2_000_000, lo=1_000, hi=200_000):
    """Config of the uneven batch: list of (form, degree, E) with log-uniform
    sizes in [lo, hi] summing to `total`, forms and degrees uniform."""
    rng = np.random.Generator(np.random.PCG64(seed + 5))
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), size=nreq))
    sizes = sizes / sizes.sum() * total
    for _ in range(100):
        sizes = np.clip(sizes, lo, hi)
        resid = total - sizes.sum()
        if abs(resid) < 0.5:
            break
        free = (sizes < hi) if resid > 0 else (sizes > lo)
        sizes[free] += resid * sizes[free] / sizes[free].sum()
    sizes = np.floor(sizes).astype(np.int64)
    sizes[np.argmax(sizes)] += total - int(sizes.sum())
    forms = rng.integers(0, 4, size=nreq)
    degrees = rng.integers(1, 5, size=nreq)
    return [(int(f), int(d), int(s)) for f, d, s in zip(forms, degrees, sizes)]


def shard(E, rank, world):
    """Contiguous element range [start, start + count) of one rank: the element
    loop is order-free (Definition 6), so ranks assemble disjoint ranges with no
    exchange; the first E % world ranks take one element more."""
    base, extra = divmod(E, world)
    start = rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def box_mesh(k, p, jitter=0.0, seed=SEED):
    """Conforming tetrahedral mesh of the unit cube: k^3 cubes, each cut into the
    6 tetrahedra of the path subdivision (one per ordering of the axes, all
    sharing the cube's main diagonal), positively oriented.  Returns
    (coords [E, 4, 3], dofs [E, n_p] int32 global DOF of each local DOF for
    p = 1 or 2 in the library's local order -- vertices, then the edges
    (2,3), (1,3), (1,2), (0,3), (0,2), (0,1) -- and the DOF count).  `jitter`
    moves interior vertices by U[-jitter, jitter] / k per axis."""
    import itertools
    if p not in (1, 2):
        raise ValueError("box_mesh numbers P1 and P2 DOFs")
    m = k + 1
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), axis=-1).reshape(-1, 3)
    pts = g.astype(np.float64) / k
    if jitter:
        rng = np.random.Generator(np.random.PCG64(seed))
        inner = np.all((g > 0) & (g < k), axis=1)
        pts[inner] += rng.uniform(-jitter, jitter, size=(int(inner.sum()), 3)) / k
    cube = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), axis=-1).reshape(-1, 1, 3)
    paths = []
    for perm in itertools.permutations(range(3)):  # one tetrahedron per ordering of the axes
        steps = np.zeros((4, 3), dtype=np.int64)
        for t, ax in enumerate(perm):
            steps[t + 1:, ax] += 1
        paths.append(steps)
    corner = cube + np.stack(paths)[None, :, :, :].reshape(1, 6 * 4, 3)  # [cubes, 6 * 4, 3]
    tets = ((corner[..., 0] * m + corner[..., 1]) * m + corner[..., 2]).reshape(-1, 4).astype(np.int64)
    d = pts[tets[:, 1:]] - pts[tets[:, :1]]
    neg = np.einsum("ei,ei->e", d[:, 0], np.cross(d[:, 1], d[:, 2])) < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    coords = np.ascontiguousarray(pts[tets])
    nv = pts.shape[0]
    if p == 1:
        return coords, tets.astype(np.int32), nv
    pairs = [(2, 3), (1, 3), (1, 2), (0, 3), (0, 2), (0, 1)]
    ends = np.stack([np.sort(np.stack([tets[:, a], tets[:, b]], axis=1), axis=1) for a, b in pairs], axis=1)
    key = ends[..., 0] * nv + ends[..., 1]
    uniq, inv = np.unique(key.reshape(-1), return_inverse=True)
    dofs = np.concatenate([tets, nv + inv.reshape(-1, 6)], axis=1).astype(np.int32)
    return coords, dofs, nv + uniq.size


def vector_dofs(dofs):
    """Global DOFs of a vector field: local 3 a + c -> global 3 dof[a] + c."""
    d = np.asarray(dofs, dtype=np.int64)
    return (3 * d[:, :, None] + np.arange(3)[None, None, :]).reshape(d.shape[0], -1).astype(np.int32)
