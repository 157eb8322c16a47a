"""CPU checks of the C ABI: the library builds, loads, exports every symbol that
include/fea.h declares, and its host-side logic (sizes, rules, planner, op
counts) answers without a GPU.  No assembly is launched here."""
import ctypes
import os
import re

import pytest

import paper_1604_05872_gb300 as fea
from paper_1604_05872_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fea.load()


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fea_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "fea_assemble" in names and len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    assert set(fea.EXPORTS) <= set(names)


def test_sizes(lib):
    assert [fea.local_dim(0, p) for p in range(1, 5)] == [4, 10, 20, 35]
    assert [fea.local_dim(2, p) for p in range(1, 5)] == [12, 30, 60, 105]
    assert fea.coeff_len(1, 2) == 10 and fea.coeff_len(2, 3) == 8 and fea.coeff_len(3, 2) == 30
    assert fea.coeffs_size(3, 2, 100) == 3002 and fea.coeffs_size(0, 1, 5) == 0
    assert fea.local_dim(4, 1) == -1 and fea.local_dim(0, 5) == -1 and fea.coeffs_size(1, 1, -1) == -1


def test_quadrature_points_match_oracle_rules(lib, orc):
    for form in range(4):
        for p in range(1, 5):
            m = orc.default_rule(form, p)
            assert fea.quad_points(form, p) == (4 if m == 0 else m ** 3)


def test_plan_without_gpu(lib):
    info = fea.plan(fea.HELMHOLTZ, 2)
    assert info["variant"] == fea.VARIANT_PRE and info["quad_points"] == 64 and info["ref_terms"] == 16
    assert info["flops_pre"] < info["flops_se"] < info["flops_naive"]
    assert info["bytes"] == 96 + 80 + 800
    nh = fea.plan(fea.NEOHOOKEAN, 2)
    assert nh["variant"] == fea.VARIANT_SE and nh["flops_pre"] == -1
    with pytest.raises(fea.FeaError) as e:
        fea.plan(fea.NEOHOOKEAN, 2, variant=fea.VARIANT_PRE)
    assert e.value.code == fea.EINVAL
    with pytest.raises(fea.FeaError):
        fea.plan(fea.MASS, 1, precision=fea.PREC_FP32, variant=fea.VARIANT_NAIVE)
    with pytest.raises(fea.FeaError):
        fea.plan(7, 1)
    with pytest.raises(fea.FeaError):
        fea.plan(fea.HELMHOLTZ, 2, tile=100000)


def test_op_counts_decrease(lib):
    for form in range(4):
        for p in range(1, 5):
            naive, best = fea.op_count(form, p)
            assert 0 < best < naive, (form, p)


def test_shared_memory_budget_is_constraint_two(lib):
    # a tiny T_H forces small tiles, then rejection
    small = fea.plan(fea.ELASTICITY, 3, smem_budget=60 * 1024)
    assert small["smem_bytes"] <= 60 * 1024
    with pytest.raises(fea.FeaError):
        fea.plan(fea.ELASTICITY, 4, smem_budget=4 * 1024)


def test_scatter_argument_checks_without_gpu(lib):
    # argument errors are answered before any device access
    nul = ctypes.c_void_p(0)
    assert lib.fea_csr_scatter_map(10, 4, nul, 5, nul, nul, 2 ** 31, 0, nul, 0, nul) == fea.EINVAL
    assert "int64 map" in lib.fea_last_error().decode()
    assert lib.fea_csr_scatter_map(10, 4, nul, 5, nul, nul, 100, 0, nul, 2, nul) == fea.EINVAL
    assert lib.fea_csr_scatter_map(10, 4, nul, 5, nul, nul, 100, 3, nul, 0, nul) == fea.EINVAL
    assert lib.fea_scatter_add_csr_mapped(10, 4, nul, 3, nul, 0, 100, nul, nul) == fea.EINVAL
    assert lib.fea_scatter_add_csr_mapped(-1, 4, nul, 0, nul, 0, 100, nul, nul) == fea.EINVAL


def test_one_pass_global_assembly_argument_checks_without_gpu(lib):
    nul = ctypes.c_void_p(0)
    for form, p, nnz, w in ((2, 1, 100, 0), (3, 2, 100, 0), (0, 4, 100, 0), (1, 1, 2 ** 31, 0), (0, 1, 100, 3),
                            (0, 1, -1, 0)):
        assert lib.fea_assemble_csr(form, p, 10, nul, nul, nul, w, nnz, nul, nul) == fea.EINVAL, (form, p, nnz, w)
    lib.fea_assemble_csr(2, 1, 10, nul, nul, nul, 0, 100, nul, nul)
    assert "one-pass" in lib.fea_last_error().decode()


def test_log_and_pattern_argument_checks_without_gpu(lib):
    nul = ctypes.c_void_p(0)
    assert lib.fea_log_f64(nul, nul, -1, nul) == fea.EINVAL
    assert lib.fea_log_f64(nul, nul, 0, nul) == 0  # nothing to do
    nnz = ctypes.c_int64(0)
    assert lib.fea_csr_pattern(1, 4, nul, 10, 2, nul, nul, ctypes.byref(nnz)) == fea.EINVAL  # upper not 0/1


def test_bernstein_argument_checks_on_cpu(lib):
    """The Bernstein entry point refuses other forms, degrees, negative sizes and bad
    out_f32 flags before it touches a device."""
    import paper_1604_05872_gb300 as fea
    nul = None
    assert lib.fea_assemble_bernstein(fea.MASS, 2, 10, nul, nul, nul, 0, nul) == fea.EINVAL
    assert lib.fea_assemble_bernstein(fea.NEOHOOKEAN, 2, 10, nul, nul, nul, 0, nul) == fea.EINVAL
    assert lib.fea_assemble_bernstein(fea.HELMHOLTZ, 5, 10, nul, nul, nul, 0, nul) == fea.EINVAL
    assert lib.fea_assemble_bernstein(fea.HELMHOLTZ, 2, -1, nul, nul, nul, 0, nul) == fea.EINVAL
    assert lib.fea_assemble_bernstein(fea.HELMHOLTZ, 2, 10, nul, nul, nul, 2, nul) == fea.EINVAL


def test_split_bf16_plan_selection_without_gpu(lib):
    """The split-BF16 precision takes the tensor cores where the contraction is compute-bound: the
    Neo-Hookean tangent (P2, P3) always, the pre-evaluated mass and Helmholtz matrices (P1, P2) only
    with FP32 output; everything else keeps its FP32 plan."""
    TC = fea.PREC_BF16X2
    for form, p in [(fea.MASS, 1), (fea.MASS, 2), (fea.HELMHOLTZ, 1), (fea.HELMHOLTZ, 2)]:
        tc = fea.plan(form, p, precision=TC, out_f32=True)
        assert tc["tile"] == 128 and tc["threads"] == 256 and tc["variant"] == fea.VARIANT_PRE
        assert tc != fea.plan(form, p, precision=fea.PREC_FP32, out_f32=True)
        assert fea.plan(form, p, precision=TC) == fea.plan(form, p, precision=fea.PREC_FP32)
        with pytest.raises(fea.FeaError):  # the tensor-core layout fixes its tile
            fea.plan(form, p, precision=TC, out_f32=True, tile=96)
    for form, p in [(fea.MASS, 3), (fea.HELMHOLTZ, 3), (fea.HELMHOLTZ, 4), (fea.ELASTICITY, 2)]:
        assert fea.plan(form, p, precision=TC, out_f32=True) == fea.plan(form, p, precision=fea.PREC_FP32, out_f32=True)
    for p in (2, 3):
        assert fea.plan(fea.NEOHOOKEAN, p, precision=TC)["threads"] > 256


def test_combined_global_assembly_argument_checks_without_gpu(lib):
    """Host-side refusals of fea_assemble_csr_combined (no device memory touched)."""
    for form, p in [(fea.ELASTICITY, 1), (fea.NEOHOOKEAN, 2), (fea.MASS, 4)]:
        assert lib.fea_assemble_csr_combined(form, p, 10, None, None, None, 100, 10, None, None) == fea.EINVAL
    # a plan shorter than its header for E elements
    assert lib.fea_assemble_csr_combined(fea.MASS, 1, 1000, None, None, None, 5, 10, None, None) == fea.EINVAL
    assert lib.fea_assemble_csr_combined(fea.MASS, 1, -1, None, None, None, 100, 10, None, None) == fea.EINVAL
