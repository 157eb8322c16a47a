"""GPU parity of the split-BF16 tensor-core contraction (FEA_PREC_BF16X2) against
the FP64 CPU oracle: the Neo-Hookean tangent on tcgen05 tensor cores, at P2 (one
product per tile of 14 elements with the reference tables as the shared operand)
and at P3 (one product per element, tiles of 4).

Tolerance: per-element relative Frobenius error <= 1e-5, max over elements (the
same bound as the FP32 contraction).  Sizes give every CTA of the persistent
launch several tiles (so every accumulator buffer and pointwise-data slot is
reused) and end in a ragged tail.
"""
import numpy as np
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
TC = 2  # FEA_PREC_BF16X2


def to_dev(coords, coeffs, form, p):
    c = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    f = None if form == inputs.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


def ref_of(orc, form, p, coords, coeffs):
    return orc.assemble(form, p, coords, coeffs, mu=inputs.NEO_MU, lam=inputs.NEO_LAMBDA, nthreads=8)


TILE = {2: 14, 3: 4}
SIZES = {2: [1, 13, 14, 15, 29, 20011], 3: [1, 3, 4, 5, 9, 2333, 20011]}


@pytest.mark.parametrize("p", [2, 3])
def test_plan_selects_tensor_core_kernel(fea, p):
    pl = fea.plan(3, p, precision=TC)
    assert pl["tile"] == TILE[p] and pl["threads"] > 256 and pl["threads"] % 32 == 0
    # a tile other than the kernel's own is refused
    with pytest.raises(fea.FeaError) as e:
        fea.plan(3, p, precision=TC, tile=8)
    assert e.value.code == fea.EINVAL


@pytest.mark.parametrize("p,E", [(p, E) for p in (2, 3) for E in SIZES[p]])
def test_neohookean_matches_oracle(fea, orc, p, E):
    coords, coeffs = inputs.workload(3, p, E, seed=3100 + 100 * p + E)
    c, f = to_dev(coords, coeffs, 3, p)
    out = fea.assemble(3, p, c, f, precision=TC)
    fea.sync()
    o = out.cpu().numpy()
    ref = ref_of(orc, 3, p, coords, coeffs)
    err = orc.rel_frobenius(o, ref)
    assert np.isfinite(o).all()
    assert err.max() <= TOL, (p, E, err.max(), int(err.argmax()))


@pytest.mark.parametrize("p", [2, 3])
def test_neohookean_symmetric_and_float_output(fea, orc, p):
    E = 4000
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    coords, coeffs = inputs.workload(3, p, E, seed=3200 + p)
    c, f = to_dev(coords, coeffs, 3, p)
    o64 = fea.assemble(3, p, c, f, precision=TC)
    o32 = fea.assemble(3, p, c, f, precision=TC, out_f32=True)
    fea.sync()
    # both outputs come from the same FP32 staging: the double output is the float one widened
    assert torch.equal(o64.float(), o32)
    a = o64.cpu().numpy()
    if p == 2:
        # the off-diagonal blocks are written as a pair's block and its transpose
        blocks_equal = np.abs(a - a.transpose(0, 2, 1))
        diag = np.zeros((3 * ns, 3 * ns), dtype=bool)
        for b in range(ns):
            diag[3 * b:3 * b + 3, 3 * b:3 * b + 3] = True
        assert blocks_equal[:, ~diag].max() == 0.0
    else:
        # every entry is computed: symmetric up to the split-BF16 rounding
        scale = np.abs(a).max(axis=(1, 2), keepdims=True)
        assert (np.abs(a - a.transpose(0, 2, 1)) / scale).max() <= 1e-5
    # deterministic: a second launch gives the same bits
    again = fea.assemble(3, p, c, f, precision=TC)
    fea.sync()
    assert torch.equal(again, o64)


@pytest.mark.parametrize("p", [2, 3])
def test_neohookean_large_deformation(fea, orc, p):
    """Displacements twice the benchmark's (det F further from 1, larger ln det F), keeping
    the elements whose det F stays above 0.05 at every quadrature point."""
    ns = (p + 1) * (p + 2) * (p + 3) // 6
    coords, coeffs = inputs.workload(3, p, 4000, seed=3300 + p)
    coeffs = coeffs * 2.0
    X, _ = orc.quad_rule(orc.default_rule(3, p))
    _, dphi = orc.basis(p, X)
    Ji = np.linalg.inv(np.transpose(coords[:, 1:] - coords[:, :1], (0, 2, 1)))
    grad_u = np.einsum("eai,qak,ekx->eqix", coeffs.reshape(-1, ns, 3), dphi, Ji)
    detF = np.linalg.det(np.eye(3) + grad_u).min(axis=1)
    keep = detF > 0.05
    assert keep.sum() > 3000 and detF.min() < 0.7
    coords, coeffs = np.ascontiguousarray(coords[keep]), np.ascontiguousarray(coeffs[keep])
    c, f = to_dev(coords, coeffs, 3, p)
    out = fea.assemble(3, p, c, f, precision=TC)
    fea.sync()
    err = orc.rel_frobenius(out.cpu().numpy(), ref_of(orc, 3, p, coords, coeffs))
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("p", [2, 3])
def test_degenerate_element_flags_and_writes_nan(fea, orc, p):
    E = 40
    coords, coeffs = inputs.workload(3, p, E, seed=3400 + p)
    coords = coords.copy()
    coords[17, 2] = coords[17, 0]  # collapsed edge: det J = 0
    coeffs = coeffs.copy()
    # u = -2 (x - x_0) on element 30 (linear, so its nodal values are exact): F = -I, det F = -1
    v = coords[30]
    nodes = v[0] + orc.nodes(p) @ (v[1:] - v[0])
    coeffs[30] = (-2.0 * (nodes - v[0])).reshape(-1)
    c, f = to_dev(coords, coeffs, 3, p)
    fea.sync()
    out = fea.assemble(3, p, c, f, precision=TC)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[17]).all()
    assert np.isnan(o[30]).all()
    keep = np.delete(o, [17, 30], axis=0)
    assert np.isfinite(keep).all()
    fea.sync()


def test_other_forms_run_the_fp32_contraction(fea):
    """In the split-BF16 mode the (form, degree) without a tensor-core kernel run the FP32 kernels."""
    for form, p in [(0, 2), (1, 2), (2, 3), (3, 1), (3, 4)]:
        E = 100
        coords, coeffs = inputs.workload(form, p, E, seed=3500 + 10 * form + p)
        c, f = to_dev(coords, coeffs, form, p)
        a = fea.assemble(form, p, c, f, precision=TC)
        b = fea.assemble(form, p, c, f, precision=fea.PREC_FP32)
        fea.sync()
        assert torch.equal(a, b), (form, p)


def test_batch_with_tensor_core_requests(fea, orc):
    reqs = [(3, 2, 1000), (1, 2, 333), (3, 2, 15), (2, 2, 120), (3, 1, 64), (3, 3, 501), (3, 3, 6)]
    built = []
    for k, (form, p, E) in enumerate(reqs):
        coords, coeffs = inputs.workload(form, p, E, seed=3600 + k)
        c, f = to_dev(coords, coeffs, form, p)
        built.append((form, p, c, f, fea.empty_out(form, p, E), coords, coeffs))
    for _ in range(2):  # capture, then replay
        fea.assemble_batch([(form, p, c, f, o) for (form, p, c, f, o, _, _) in built], precision=TC)
    fea.sync()
    for (form, p, c, f, o, coords, coeffs) in built:
        single = fea.assemble(form, p, c, f, precision=TC)
        fea.sync()
        assert torch.equal(single, o), (form, p)
        assert orc.rel_frobenius(o.cpu().numpy(), ref_of(orc, form, p, coords, coeffs)).max() <= TOL
