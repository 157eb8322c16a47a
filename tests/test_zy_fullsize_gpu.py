"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (default options, same inputs and seeds): the element matrices (or
vectors) of a sample of elements -- random ones, the first and last, and the
worst-shaped ones -- against the FP64 oracle computed element by element, and
invariants that hold for every element (finiteness, symmetry) on the whole
output.  Collected after the other parity tests (large device allocations)."""
import numpy as np
import pytest

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 contraction, relative Frobenius error per element


def _worst_shaped(coords, k):
    """Indices of the k elements with the smallest |det J| / (longest edge)^3."""
    d = coords[:, 1:, :] - coords[:, :1, :]
    det = np.abs(np.einsum("ei,ei->e", d[:, 0], np.cross(d[:, 1], d[:, 2])))
    edges = [coords[:, i] - coords[:, j] for i in range(4) for j in range(i)]
    longest = np.max(np.stack([np.linalg.norm(x, axis=1) for x in edges]), axis=0)
    return np.argsort(det / longest ** 3)[:k]


def _sample(coords, n, seed):
    E = coords.shape[0]
    rng = np.random.default_rng(seed)
    idx = np.concatenate([[0, E - 1], rng.choice(E, size=min(n, E), replace=False), _worst_shaped(coords, 50)])
    return np.unique(idx)


def _rows(out, idx):
    import torch
    return out.index_select(0, torch.from_numpy(idx).to(out.device)).cpu().numpy()


@pytest.mark.parametrize("name,form,p,E,aniso,prec", [
    ("helmholtz_p2_1M", 1, 2, 1_000_000, False, 1),
    ("mass_p1_10k", 0, 1, 10_000, False, 1),
    ("elasticity_p3_200k", 2, 3, 200_000, True, 1),
    ("neohookean_p2_500k", 3, 2, 500_000, False, 1),
    ("neohookean_p2_500k", 3, 2, 500_000, False, 2),  # split-BF16 tensor cores, as bench.py runs it
])
def test_benchmark_workload_full_size(fea, orc, name, form, p, E, aniso, prec):
    import torch
    coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED, anisotropic=aniso)
    c = torch.from_numpy(coords).cuda()
    f = None if form == 0 else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    out = fea.assemble(form, p, c, f, precision=prec)
    fea.sync()
    idx = np.arange(E) if E <= 10_000 else _sample(coords, 1500, seed=E)
    got = _rows(out, idx)
    ref = orc.assemble(form, p, coords[idx], None if coeffs is None else coeffs[idx], nthreads=orc.max_threads())
    assert orc.rel_frobenius(got, ref).max() <= TOL, name
    # every element: finite and (all four forms) symmetric up to the FP32 contraction's rounding
    assert bool(torch.isfinite(out).all())
    step = max(1, E // 20000)
    sub = out[::step]
    asym = (sub - sub.transpose(1, 2)).abs().amax(dim=(1, 2)) / sub.abs().amax(dim=(1, 2))
    assert float(asym.max()) <= 1e-5, name
    del out, c, f
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fused,prec", [(False, 1), (True, 1), (False, 2)])
def test_stream_64_requests_full_size(fea, orc, fused, prec):
    """The 2M-element, 64-request stream exactly as bench.py builds it."""
    import torch
    reqs = inputs.stream_requests()
    built, host = [], []
    for k, (form, p, E) in enumerate(reqs):
        coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED + 100 + k, anisotropic=(form == 2))
        c = torch.from_numpy(coords).cuda()
        f = None if form == 0 else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
        built.append((form, p, c, f, fea.empty_out(form, p, E)))
        host.append((coords, coeffs))
    fea.assemble_batch(built, fused=fused, precision=prec)
    fea.sync()
    worst = 0.0
    for k, ((form, p, c, f, o), (coords, coeffs)) in enumerate(zip(built, host)):
        idx = _sample(coords, 40 if form == 3 and p >= 3 else 100, seed=k)
        got = _rows(o, idx)
        ref = orc.assemble(form, p, coords[idx], None if coeffs is None else coeffs[idx], nthreads=orc.max_threads())
        worst = max(worst, float(orc.rel_frobenius(got, ref).max()))
        assert bool(torch.isfinite(o).all()), (k, form, p)
    assert worst <= TOL
    del built
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name,form,p,E", [
    ("helmholtz_load_p2_1M", 1, 2, 1_000_000),
    ("neohookean_residual_p2_500k", 3, 2, 500_000),
])
def test_element_vector_workload_full_size(fea, orc, name, form, p, E):
    import torch
    coords, coeffs = inputs.workload(form, p, E, seed=inputs.SEED)
    c = torch.from_numpy(coords).cuda()
    f = torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    out = fea.assemble_vector(form, p, c, f)
    fea.sync()
    idx = _sample(coords, 3000, seed=E + 1)
    got = _rows(out, idx)
    if form == 1:
        ref = orc.load_vector(p, coords[idx], coeffs[idx])
    else:
        ref = orc.neohookean_residual(p, coords[idx], coeffs[idx])
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= TOL, name
    assert bool(torch.isfinite(out).all())
    if form == 3:  # force balance on every element: sum over nodes of each component is zero
        bal = out.view(E, -1, 3).sum(dim=1).abs().amax(dim=1) / out.abs().amax(dim=1)
        assert float(bal.max()) <= 1e-5
    del out, c, f
    torch.cuda.empty_cache()


def test_global_assembly_full_size(fea, orc):
    """The global assembly workload at its full size (Helmholtz P2 on the 55^3-cube mesh, 998 250
    elements), in bench.py's launch configuration: the row sums of the assembled matrix are the
    assembled load vector (the stiffness rows sum to zero, the f-mass rows to int f phi_i), checked
    against the oracle's element load vectors summed at the global DOFs, to the FP32 contraction's
    tolerance relative to each row's absolute sum; symmetric storage holds the upper triangle of the
    full matrix; the combining kernel gives both up to the order of the FP64 additions."""
    import torch
    coords, dofs, nd = inputs.box_mesh(55, 2, jitter=0.1, seed=inputs.SEED)
    E = coords.shape[0]
    f = inputs.random_coeffs(1, 2, E, np.random.Generator(np.random.PCG64(inputs.SEED + 7)))
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    c = torch.from_numpy(coords).cuda()
    fc = torch.from_numpy(inputs.coeff_array(1, 2, f)).cuda()
    dd = torch.from_numpy(dofs).cuda()
    smap = fea.csr_scatter_map(dd, torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col_idx).cuda())
    vals = fea.assemble_csr(1, 2, c, fc, smap, torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda"))
    fea.sync()
    v = vals.cpu().numpy()
    assert np.isfinite(v).all()
    rows = np.add.reduceat(v, row_ptr[:-1])
    absrows = np.add.reduceat(np.abs(v), row_ptr[:-1])
    b = orc.load_vector(2, coords, f)
    ref = np.bincount(dofs.ravel(), weights=b.ravel(), minlength=nd)
    assert np.all(np.abs(rows - ref) <= TOL * absrows)
    # symmetric storage: the upper triangle of the same matrix
    ur, uc = fea.csr_pattern(dofs, nd, upper=True)
    umap = fea.csr_scatter_map(dd, torch.from_numpy(ur).cuda(), torch.from_numpy(uc).cuda(), upper=True)
    uv = fea.assemble_csr(1, 2, c, fc, umap, torch.zeros(uc.shape[0], dtype=torch.float64, device="cuda"))
    fea.sync()
    r = np.repeat(np.arange(nd), np.diff(row_ptr))
    keep = col_idx >= r
    assert np.allclose(uv.cpu().numpy(), v[keep], rtol=0, atol=1e-12 * np.abs(v).max())
    # the combining kernel that bench.py times (a tile's entries summed per CSR position): the same
    # matrix up to the order of the FP64 additions, full and symmetric storage
    plan = torch.from_numpy(fea.csr_combine_plan(smap, col_idx.shape[0])).cuda()
    cv = fea.assemble_csr_combined(1, 2, c, fc, plan, torch.zeros_like(vals))
    uplan = torch.from_numpy(fea.csr_combine_plan(umap, uc.shape[0])).cuda()
    cu = fea.assemble_csr_combined(1, 2, c, fc, uplan, torch.zeros_like(uv))
    fea.sync()
    assert np.allclose(cv.cpu().numpy(), v, rtol=0, atol=1e-12 * np.abs(v).max())
    assert np.allclose(cu.cpu().numpy(), uv.cpu().numpy(), rtol=0, atol=1e-12 * np.abs(v).max())
