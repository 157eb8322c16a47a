"""GPU parity of the sum-factorised Bernstein-Bezier Helmholtz variant
(fea_assemble_bernstein) against the FP64 CPU oracle's plain quadrature nest in
the same basis (pinned in test_oracle.py against the Lagrange oracle).

Tolerance: per-element relative Frobenius error <= 1e-5, max over elements
(FP64 geometry, FP32 arithmetic after it).  Sizes span several tiles of 32
elements and end in ragged tails.
"""
import numpy as np
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _data(p, E, seed):
    coords, _ = inputs.workload(inputs.HELMHOLTZ, p, E, seed=seed)
    c = np.random.default_rng(seed).uniform(-1.0, 1.0, (E, inputs.nbasis(p)))
    return coords, c, torch.from_numpy(coords).cuda(), torch.from_numpy(c).cuda()


@pytest.mark.parametrize("p,E", [(p, E) for p in (1, 2, 3, 4) for E in (1, 31, 33, 777)])
def test_bernstein_matches_oracle(fea, orc, p, E):
    coords, c, dc, dcoef = _data(p, E, 7000 + 10 * p + E)
    out = fea.assemble_bernstein(fea.HELMHOLTZ, p, dc, dcoef)
    fea.sync()
    o = out.cpu().numpy()
    ref = orc.assemble_bernstein(orc.HELMHOLTZ, p, coords, c, nthreads=8)
    err = orc.rel_frobenius(o, ref)
    assert np.isfinite(o).all()
    assert err.max() <= TOL, (p, E, err.max(), int(err.argmax()))


@pytest.mark.parametrize("p", [2, 4])
def test_bernstein_float_output_and_determinism(fea, p):
    coords, c, dc, dcoef = _data(p, 5000, 7100 + p)
    o64 = fea.assemble_bernstein(fea.HELMHOLTZ, p, dc, dcoef)
    o32 = fea.assemble_bernstein(fea.HELMHOLTZ, p, dc, dcoef, out_f32=True)
    again = fea.assemble_bernstein(fea.HELMHOLTZ, p, dc, dcoef)
    fea.sync()
    assert o32.dtype == torch.float32
    assert torch.equal(o64.float(), o32)  # the FP64 output is the FP32 result widened exactly
    assert torch.equal(again, o64)


def test_bernstein_full_size_sampled(fea, orc):
    """P4 at 2e5 elements: a sample of elements (first, last, random) against the oracle."""
    p, E = 4, 200_000
    coords, c, dc, dcoef = _data(p, E, 7200)
    out = fea.assemble_bernstein(fea.HELMHOLTZ, p, dc, dcoef)
    fea.sync()
    idx = np.unique(np.concatenate([np.arange(40), np.arange(E - 40, E),
                                    np.random.default_rng(1).choice(E, 1000, replace=False)]))
    ref = orc.assemble_bernstein(orc.HELMHOLTZ, p, coords[idx], c[idx], nthreads=16)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    assert orc.rel_frobenius(got, ref).max() <= TOL
    assert torch.isfinite(out).all()


def test_bernstein_degenerate_element(fea):
    coords, c, dc, dcoef = _data(3, 70, 7300)
    coords = coords.copy()
    coords[41, 3] = coords[41, 0]  # collapsed edge: det J = 0
    dc = torch.from_numpy(coords).cuda()
    fea.sync()
    out = fea.assemble_bernstein(fea.HELMHOLTZ, 3, dc, dcoef)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[41]).all() and np.isfinite(np.delete(o, 41, axis=0)).all()
    fea.sync()


def test_bernstein_refusals(fea):
    coords, c, dc, dcoef = _data(2, 10, 7400)
    with pytest.raises(fea.FeaError) as e:
        fea.assemble_bernstein(fea.HELMHOLTZ, 2, torch.from_numpy(coords), dcoef)  # host coords
    assert e.value.code == fea.EINVAL
    empty = fea.assemble_bernstein(fea.HELMHOLTZ, 2, dc[:0], dcoef[:0])
    fea.sync()
    assert empty.shape == (0, 10, 10)
