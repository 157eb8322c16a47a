"""Element vectors of the linear forms (fea_assemble_vector): the Helmholtz
load vector and the Neo-Hookean residual against the FP64 oracle, element by
element, at sizes spanning several tiles with a ragged tail; FP32 (1e-5) and
FP64 (1e-12) paths; FP32 output; the empty and degenerate cases."""
import numpy as np
import pytest

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(x, ref):
    """Per-element relative 2-norm error, max over elements."""
    num = np.linalg.norm(x - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return float((num / den).max())


def _data(form, p, E, seed):
    import torch
    coords, coeffs = inputs.workload(form, p, E, seed=seed)
    c = torch.from_numpy(coords).cuda()
    f = torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return coords, coeffs, c, f


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (0, 1e-12)])
def test_load_vector_parity(fea, orc, p, prec, tol):
    E = 333  # three tiles of 128 and a ragged tail
    coords, f, c, fd = _data(inputs.HELMHOLTZ, p, E, seed=200 + p)
    out = fea.assemble_vector(fea.HELMHOLTZ, p, c, fd, precision=prec)
    fea.sync()
    ref = orc.load_vector(p, coords, f)
    assert out.shape == (E, orc.nbasis(p))
    assert _rel(out.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (0, 1e-12)])
def test_neohookean_residual_parity(fea, orc, p, prec, tol):
    E = {1: 77, 2: 77, 3: 37, 4: 19}[p]  # several tiles and a ragged tail
    coords, u, c, ud = _data(inputs.NEOHOOKEAN, p, E, seed=210 + p)
    out = fea.assemble_vector(fea.NEOHOOKEAN, p, c, ud, precision=prec)
    fea.sync()
    ref = orc.neohookean_residual(p, coords, u)
    assert out.shape == (E, 3 * orc.nbasis(p))
    assert _rel(out.cpu().numpy(), ref) <= tol


def test_vector_f32_output_empty_and_errors(fea, orc):
    import torch
    coords, f, c, fd = _data(inputs.HELMHOLTZ, 2, 200, seed=220)
    o32 = fea.assemble_vector(fea.HELMHOLTZ, 2, c, fd, out_f32=True)
    fea.sync()
    assert o32.dtype == torch.float32
    assert _rel(o32.cpu().numpy().astype(np.float64), orc.load_vector(2, coords, f)) <= 1e-5
    empty = fea.assemble_vector(fea.HELMHOLTZ, 2, c[:0], fd[:0])
    assert empty.shape == (0, 10)
    for form in (fea.MASS, fea.ELASTICITY):
        with pytest.raises(fea.FeaError):
            fea.assemble_vector(form, 2, c, fd)
    with pytest.raises(fea.FeaError):
        fea.assemble_vector(fea.HELMHOLTZ, 2, c.cpu(), fd.cpu())  # host pointers: no CPU fallback


def test_vector_degenerate_element_is_nan(fea):
    import torch
    coords, u = inputs.workload(inputs.NEOHOOKEAN, 2, 40, seed=230)
    coords[7, 3] = coords[7, 0]  # collapsed element: det J = 0
    c = torch.from_numpy(coords).cuda()
    ud = torch.from_numpy(inputs.coeff_array(inputs.NEOHOOKEAN, 2, u)).cuda()
    out = fea.assemble_vector(fea.NEOHOOKEAN, 2, c, ud)
    with pytest.raises(fea.FeaError) as ei:
        fea.sync()
    assert ei.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[7]).all() and np.isfinite(np.delete(o, 7, axis=0)).all()


def test_load_vector_many_tiles_per_cta_and_degenerate(fea, orc):
    """More tiles than resident CTAs (each CTA streams several, double-buffered), a ragged tail and
    one collapsed element: its row is NaN and flagged, every other row matches the oracle."""
    import torch
    E = 152 * 8 * 128 + 77
    coords, f, c, fd = _data(inputs.HELMHOLTZ, 2, E, seed=240)
    coords[E - 5, 2] = coords[E - 5, 0]
    c = torch.from_numpy(coords).cuda()
    out = fea.assemble_vector(fea.HELMHOLTZ, 2, c, fd)
    with pytest.raises(fea.FeaError) as ei:
        fea.sync()
    assert ei.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[E - 5]).all()
    keep = np.ones(E, dtype=bool)
    keep[E - 5] = False
    assert _rel(o[keep], orc.load_vector(2, coords[keep], f[keep])) <= 1e-5
