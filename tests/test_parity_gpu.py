"""GPU parity: the CUDA path against the FP64 CPU oracle, element by element.

Tolerances (per-element relative Frobenius error, max over elements):
  FP64 path (plain and flop-reduced)  <= 1e-12
  FP32 contraction, FP64 geometry     <= 1e-5
  split-BF16 tensor-core contraction  <= 1e-5 (Neo-Hookean P2; the other forms run FP32 in that mode)
Sizes span several tiles and end in a ragged tail; the full benchmark sizes are
checked on sampled elements in test_fullsize_gpu.py.
"""
import numpy as np
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-5}
FORMS = [0, 1, 2, 3]
DEGREES = [1, 2, 3, 4]


def to_dev(coords, coeffs, form, p):
    c = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    f = None
    if form != inputs.MASS:
        f = torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


def oracle_ref(orc, form, p, coords, coeffs):
    return orc.assemble(form, p, coords, coeffs, mu=inputs.NEO_MU, lam=inputs.NEO_LAMBDA, nthreads=8)


def sizes_for(fea, form, p, variant, prec):
    t = fea.plan(form, p, precision=prec, variant=variant)["tile"]
    nn = fea.local_dim(form, p) ** 2
    # several tiles and a ragged tail, bounded by the oracle's cost
    cap = max(3, int(3e5 // nn)) if p < 4 else max(3, int(6e4 // nn))
    return max(1, min(2 * t + 3, cap))


def variants(form):
    return [1, 2] if form != 3 else [1]


@pytest.mark.parametrize("prec", [1, 0, 2])
@pytest.mark.parametrize("p", DEGREES)
@pytest.mark.parametrize("form", FORMS)
def test_flop_reduced_variants_match_oracle(fea, orc, form, p, prec):
    for variant in variants(form):
        E = sizes_for(fea, form, p, variant, prec)
        coords, coeffs = inputs.workload(form, p, E, seed=1000 + 10 * form + p)
        c, f = to_dev(coords, coeffs, form, p)
        out = fea.assemble(form, p, c, f, precision=prec, variant=variant)
        fea.sync()
        ref = oracle_ref(orc, form, p, coords, coeffs)
        err = orc.rel_frobenius(out.cpu().numpy(), ref)
        assert err.max() <= TOL[prec], (form, p, variant, prec, err.max())


@pytest.mark.parametrize("form,p", [(2, 1), (2, 2), (3, 1), (3, 2), (3, 3)])
def test_vector_se_smaller_tile(fea, orc, form, p):
    """The sharing-elimination tile kernel at a tile below the one its thread layout is built for
    (runtime tile sizes instead of compile-time ones), several tiles and a ragged tail."""
    t = fea.plan(form, p, variant=1)["tile"]
    small = max(1, t - 1) if t > 1 else 1
    E = 3 * small + 1
    coords, coeffs = inputs.workload(form, p, E, seed=1500 + 10 * form + p)
    c, f = to_dev(coords, coeffs, form, p)
    out = fea.assemble(form, p, c, f, variant=1, tile=small)
    fea.sync()
    err = orc.rel_frobenius(out.cpu().numpy(), oracle_ref(orc, form, p, coords, coeffs))
    assert err.max() <= TOL[1], (form, p, small, err.max())


@pytest.mark.parametrize("p", DEGREES)
@pytest.mark.parametrize("form", FORMS)
def test_plain_fp64_kernel_matches_oracle(fea, orc, form, p):
    E = sizes_for(fea, form, p, fea.VARIANT_NAIVE, 0)
    coords, coeffs = inputs.workload(form, p, E, seed=2000 + 10 * form + p)
    c, f = to_dev(coords, coeffs, form, p)
    out = fea.assemble(form, p, c, f, precision=fea.PREC_FP64, variant=fea.VARIANT_NAIVE)
    fea.sync()
    ref = oracle_ref(orc, form, p, coords, coeffs)
    assert orc.rel_frobenius(out.cpu().numpy(), ref).max() <= 1e-12


def test_anisotropic_elasticity_fp32_within_tolerance(fea, orc):
    """Aspect ratios up to 1e3 with the FP32 contraction: FP64 geometry keeps 1e-5."""
    coords, coeffs = inputs.workload(2, 3, 300, seed=77, anisotropic=True)
    c, f = to_dev(coords, coeffs, 2, 3)
    for variant in (1, 2):
        out = fea.assemble(2, 3, c, f, precision=1, variant=variant)
        fea.sync()
        ref = oracle_ref(orc, 2, 3, coords, coeffs)
        assert orc.rel_frobenius(out.cpu().numpy(), ref).max() <= 1e-5


def test_float_output_and_default_call(fea, orc):
    coords, coeffs = inputs.workload(1, 2, 1001, seed=5)
    c, f = to_dev(coords, coeffs, 1, 2)
    ref = oracle_ref(orc, 1, 2, coords, coeffs)
    o32 = fea.assemble(1, 2, c, f, out_f32=True)
    o64 = fea.empty_out(1, 2, 1001)
    fea.assemble_default(1, 2, c, f, o64)
    fea.sync()
    assert o32.dtype == torch.float32
    assert orc.rel_frobenius(o32.double().cpu().numpy(), ref).max() <= 1e-5
    assert orc.rel_frobenius(o64.cpu().numpy(), ref).max() <= 1e-5
    # the double output is the float result widened exactly
    assert torch.equal(o64.float(), o32)


@pytest.mark.parametrize("form,p", [(0, 1), (0, 2), (0, 3), (1, 1), (1, 3), (2, 1), (2, 2), (2, 3), (3, 2)])
def test_float_output_every_streaming_kernel(fea, orc, form, p):
    """FP32 output equals the FP64 output rounded (both come from the same FP32
    contraction), on ragged sizes, for the kernels with their own FP32 store path."""
    E = 777
    coords, coeffs = inputs.workload(form, p, E, seed=40 + 4 * form + p)
    c, f = to_dev(coords, coeffs, form, p)
    o32 = fea.assemble(form, p, c, f, out_f32=True)
    o64 = fea.assemble(form, p, c, f)
    fea.sync()
    assert torch.equal(o64.float(), o32)
    ref = oracle_ref(orc, form, p, coords, coeffs)
    assert orc.rel_frobenius(o32.double().cpu().numpy(), ref).max() <= 1e-5


def test_host_buffer_call_equals_device_call(fea):
    for form, p in [(1, 2), (3, 2), (2, 3)]:
        E = 777
        coords, coeffs = inputs.workload(form, p, E, seed=9)
        c, f = to_dev(coords, coeffs, form, p)
        dev = fea.assemble(form, p, c, f)
        hc = torch.from_numpy(coords).pin_memory()
        hf = None if f is None else f.cpu().pin_memory()
        ho = torch.empty((E,) + dev.shape[1:], dtype=torch.float64).pin_memory()
        fea.assemble_host(form, p, hc, hf, ho)
        torch.cuda.synchronize()
        assert torch.equal(ho, dev.cpu())


def test_edge_cases(fea, orc):
    coords, coeffs = inputs.workload(1, 2, 3, seed=3)
    c, f = to_dev(coords, coeffs, 1, 2)
    # E = 0 is a no-op
    out = torch.full((0, 10, 10), 7.0, dtype=torch.float64, device="cuda")
    fea.assemble(1, 2, c[:0], f[:0], out=out)
    # E = 1 and odd counts
    for E in (1, 2, 3):
        o = fea.assemble(1, 2, c[:E], f[:10 * E])
        fea.sync()
        ref = oracle_ref(orc, 1, 2, coords[:E], coeffs[:E])
        assert orc.rel_frobenius(o.cpu().numpy(), ref).max() <= 1e-5
    # host pointers are rejected: no CPU fallback
    with pytest.raises(fea.FeaError) as e:
        fea.assemble(1, 2, torch.from_numpy(coords), f, out=torch.empty((3, 10, 10), dtype=torch.float64, device="cuda"))
    assert e.value.code == fea.EINVAL
    # bad form / degree
    with pytest.raises(fea.FeaError):
        fea.assemble(9, 2, c, f)
    with pytest.raises(fea.FeaError):
        fea.assemble(1, 5, c, f)
    # misaligned output pointer
    big = torch.empty(3 * 100 + 1, dtype=torch.float64, device="cuda")
    rc = fea.load().fea_assemble(1, 2, 3, c.data_ptr(), f.data_ptr(), big.data_ptr() + 4, None)
    assert rc == fea.EINVAL


def test_degenerate_element_flags_and_writes_nan(fea):
    coords, coeffs = inputs.workload(1, 2, 8, seed=4)
    coords = coords.copy()
    coords[5, 3] = coords[5, 0]  # collapsed edge: det J = 0 exactly
    c, f = to_dev(coords, coeffs, 1, 2)
    fea.sync()
    out = fea.assemble(1, 2, c, f)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EDEGENERATE
    o = out.cpu().numpy()
    assert np.isnan(o[5]).all() and np.isfinite(np.delete(o, 5, axis=0)).all()
    fea.sync()  # cleared


@pytest.mark.parametrize("fused", [False, True])
def test_batch_matches_standalone(fea, orc, fused):
    reqs = [(0, 1, 50), (1, 2, 333), (2, 3, 17), (3, 2, 41), (1, 4, 9), (2, 2, 120), (3, 1, 64), (0, 4, 11)]
    built = []
    for k, (form, p, E) in enumerate(reqs):
        coords, coeffs = inputs.workload(form, p, E, seed=50 + k)
        c, f = to_dev(coords, coeffs, form, p)
        built.append((form, p, c, f, fea.empty_out(form, p, E), coords, coeffs))
    fea.assemble_batch([(form, p, c, f, o) for (form, p, c, f, o, _, _) in built], fused=fused)
    fea.assemble_batch([(form, p, c, f, o) for (form, p, c, f, o, _, _) in built], fused=fused)  # graph replay
    fea.sync()
    for (form, p, c, f, o, coords, coeffs) in built:
        single = fea.assemble(form, p, c, f)
        fea.sync()
        assert torch.equal(single, o), (form, p)
        ref = oracle_ref(orc, form, p, coords, coeffs)
        assert orc.rel_frobenius(o.cpu().numpy(), ref).max() <= 1e-5
