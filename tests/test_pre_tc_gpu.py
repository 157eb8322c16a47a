"""GPU parity of the pre-evaluated mass and Helmholtz matrices on the tcgen05 tensor
cores (FEA_PREC_BF16X2 with FP32 output, P1-P2) against the FP64 CPU oracle.

Tolerance: per-element relative Frobenius error <= 1e-5, max over elements (the
bound of the FP32 contraction), including elements of aspect ratio 10^3.  Sizes
span several 128-element tiles per CTA of the persistent launch and end in a
ragged tail.  With FP64 output the same precision keeps the FP32 contraction
(bit for bit), which is bound by HBM there.
"""
import numpy as np
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
TC = 2  # FEA_PREC_BF16X2
CASES = [(0, 1), (0, 2), (1, 1), (1, 2)]


def to_dev(coords, coeffs, form, p):
    c = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    f = None if form == inputs.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


@pytest.mark.parametrize("form,p", CASES)
def test_plan_selects_the_tensor_cores_with_fp32_output_only(fea, form, p):
    tc = fea.plan(form, p, precision=TC, out_f32=True)
    assert tc["tile"] == 128 and tc["threads"] == 256 and tc["variant"] == fea.VARIANT_PRE
    assert tc != fea.plan(form, p, precision=fea.PREC_FP32, out_f32=True)
    # FP64 output: the FP32 contraction
    assert fea.plan(form, p, precision=TC) == fea.plan(form, p, precision=fea.PREC_FP32)


@pytest.mark.parametrize("form,p", CASES)
@pytest.mark.parametrize("E", [1, 127, 128, 129, 1000, 40011])
def test_matches_oracle(fea, orc, form, p, E):
    coords, coeffs = inputs.workload(form, p, E, seed=5100 + 10 * form + p + E)
    c, f = to_dev(coords, coeffs, form, p)
    out = fea.assemble(form, p, c, f, precision=TC, out_f32=True)
    fea.sync()
    o = out.cpu().numpy()
    assert out.dtype == torch.float32 and np.isfinite(o).all()
    err = orc.rel_frobenius(o, orc.assemble(form, p, coords, coeffs, nthreads=8))
    assert err.max() <= TOL, (form, p, E, err.max(), int(err.argmax()))
    again = fea.assemble(form, p, c, f, precision=TC, out_f32=True)  # deterministic
    fea.sync()
    assert torch.equal(again, out)


@pytest.mark.parametrize("form,p", [(0, 2), (1, 2)])
def test_anisotropic_elements(fea, orc, form, p):
    E = 5000
    coords, coeffs = inputs.workload(form, p, E, seed=5300 + form, anisotropic=True)
    c, f = to_dev(coords, coeffs, form, p)
    out = fea.assemble(form, p, c, f, precision=TC, out_f32=True)
    fea.sync()
    err = orc.rel_frobenius(out.cpu().numpy(), orc.assemble(form, p, coords, coeffs, nthreads=8))
    assert err.max() <= TOL, (form, p, err.max())


def test_fp64_output_keeps_the_fp32_contraction(fea):
    coords, coeffs = inputs.workload(1, 2, 3000, seed=5400)
    c, f = to_dev(coords, coeffs, 1, 2)
    a = fea.assemble(1, 2, c, f, precision=TC)
    b = fea.assemble(1, 2, c, f, precision=fea.PREC_FP32)
    fea.sync()
    assert torch.equal(a, b)


def test_degenerate_element_flags_and_writes_nan(fea):
    coords, coeffs = inputs.workload(1, 2, 300, seed=5500)
    coords = coords.copy()
    coords[200, 3] = coords[200, 0]  # collapsed edge: det J = 0 exactly, in the second tile
    c, f = to_dev(coords, coeffs, 1, 2)
    fea.sync()
    out = fea.assemble(1, 2, c, f, precision=TC, out_f32=True)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[200]).all() and np.isfinite(np.delete(o, 200, axis=0)).all()
    fea.sync()  # cleared
