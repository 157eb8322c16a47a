"""GPU parity of the split-BF16 tensor-core contraction (FEA_PREC_BF16X2) against
the FP64 CPU oracle: the Neo-Hookean tangent at P2 on tcgen05 tensor cores.

Tolerance: per-element relative Frobenius error <= 1e-5, max over elements (the
same bound as the FP32 contraction).  Sizes give every CTA of the persistent
launch several tiles of 14 elements (so both accumulator buffers and both
pointwise-data slots are reused) and end in a ragged tail.
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


def test_plan_selects_tensor_core_kernel(fea):
    pl = fea.plan(3, 2, precision=TC)
    assert pl["tile"] == 14 and pl["threads"] > 256 and pl["threads"] % 32 == 0
    # a tile other than the kernel's own is refused
    with pytest.raises(fea.FeaError) as e:
        fea.plan(3, 2, precision=TC, tile=8)
    assert e.value.code == fea.EINVAL


@pytest.mark.parametrize("E", [1, 13, 14, 15, 29, 20011])
def test_neohookean_p2_matches_oracle(fea, orc, E):
    coords, coeffs = inputs.workload(3, 2, E, seed=3100 + E)
    c, f = to_dev(coords, coeffs, 3, 2)
    out = fea.assemble(3, 2, c, f, precision=TC)
    fea.sync()
    o = out.cpu().numpy()
    ref = ref_of(orc, 3, 2, coords, coeffs)
    err = orc.rel_frobenius(o, ref)
    assert np.isfinite(o).all()
    assert err.max() <= TOL, (E, err.max(), int(err.argmax()))


def test_neohookean_p2_symmetric_and_float_output(fea, orc):
    E = 4000
    coords, coeffs = inputs.workload(3, 2, E, seed=3200)
    c, f = to_dev(coords, coeffs, 3, 2)
    o64 = fea.assemble(3, 2, c, f, precision=TC)
    o32 = fea.assemble(3, 2, c, f, precision=TC, out_f32=True)
    fea.sync()
    # both outputs come from the same FP32 staging: the double output is the float one widened
    assert torch.equal(o64.float(), o32)
    # the off-diagonal blocks are written as a pair's block and its transpose
    a = o64.cpu().numpy()
    blocks_equal = np.abs(a - a.transpose(0, 2, 1))
    diag = np.zeros((30, 30), dtype=bool)
    for b in range(10):
        diag[3 * b:3 * b + 3, 3 * b:3 * b + 3] = True
    assert blocks_equal[:, ~diag].max() == 0.0
    # deterministic: a second launch gives the same bits
    again = fea.assemble(3, 2, c, f, precision=TC)
    fea.sync()
    assert torch.equal(again, o64)


def test_neohookean_p2_large_deformation(fea, orc):
    """Displacements twice the benchmark's (det F further from 1, larger ln det F), keeping
    the elements whose det F stays above 0.05 at every quadrature point."""
    coords, coeffs = inputs.workload(3, 2, 4000, seed=3300)
    coeffs = coeffs * 2.0
    X, _ = orc.quad_rule(orc.default_rule(3, 2))
    _, dphi = orc.basis(2, X)
    Ji = np.linalg.inv(np.transpose(coords[:, 1:] - coords[:, :1], (0, 2, 1)))
    grad_u = np.einsum("eai,qak,ekx->eqix", coeffs.reshape(-1, 10, 3), dphi, Ji)
    detF = np.linalg.det(np.eye(3) + grad_u).min(axis=1)
    keep = detF > 0.05
    assert keep.sum() > 3000 and detF.min() < 0.5
    coords, coeffs = np.ascontiguousarray(coords[keep]), np.ascontiguousarray(coeffs[keep])
    c, f = to_dev(coords, coeffs, 3, 2)
    out = fea.assemble(3, 2, c, f, precision=TC)
    fea.sync()
    err = orc.rel_frobenius(out.cpu().numpy(), ref_of(orc, 3, 2, coords, coeffs))
    assert err.max() <= TOL, err.max()


def test_degenerate_element_flags_and_writes_nan(fea):
    E = 40
    coords, coeffs = inputs.workload(3, 2, E, seed=3400)
    coords = coords.copy()
    coords[17, 2] = coords[17, 0]  # collapsed edge: det J = 0
    coeffs = coeffs.copy()
    # u = -2 (x - x_0) on element 30 (linear, so its P2 nodal values are exact): F = -I, det F = -1
    v = coords[30]
    edges = [(2, 3), (1, 3), (1, 2), (0, 3), (0, 2), (0, 1)]
    nodes = np.vstack([v, [(v[i] + v[j]) / 2 for i, j in edges]])
    coeffs[30] = (-2.0 * (nodes - v[0])).reshape(-1)
    c, f = to_dev(coords, coeffs, 3, 2)
    fea.sync()
    out = fea.assemble(3, 2, c, f, precision=TC)
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
    for form, p in [(0, 2), (1, 2), (2, 3), (3, 1), (3, 3)]:
        E = 100
        coords, coeffs = inputs.workload(form, p, E, seed=3500 + 10 * form + p)
        c, f = to_dev(coords, coeffs, form, p)
        a = fea.assemble(form, p, c, f, precision=TC)
        b = fea.assemble(form, p, c, f, precision=fea.PREC_FP32)
        fea.sync()
        assert torch.equal(a, b), (form, p)


def test_batch_with_tensor_core_requests(fea, orc):
    reqs = [(3, 2, 1000), (1, 2, 333), (3, 2, 15), (2, 2, 120), (3, 1, 64)]
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
