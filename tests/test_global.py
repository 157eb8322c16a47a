"""Global assembly: the CSR pattern builder (host, C ABI) against a library
sparse sum, the reference global matrices against closed forms on the unit
cube, and the GPU scatter-add against the reference."""
import numpy as np
import pytest

from oracle import global_ref
from paper_1604_05872_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1604_05872_gb300 import build as fbuild
    import paper_1604_05872_gb300 as fea
    fbuild.build()
    return fea.load()


@pytest.mark.parametrize("p", [1, 2])
def test_csr_pattern_matches_library_sparse_sum(p):
    import paper_1604_05872_gb300 as fea
    coords, dofs, nd = inputs.box_mesh(3, p, jitter=0.2)
    for d, nrows in ((dofs, nd), (inputs.vector_dofs(dofs), 3 * nd)):
        row_ptr, col_idx = fea.csr_pattern(d, nrows)
        n = d.shape[1]
        indptr, indices, _ = global_ref.assemble_csr(d, np.ones((d.shape[0], n, n)), nrows)
        assert np.array_equal(row_ptr, indptr) and np.array_equal(col_idx, indices)
    with pytest.raises(fea.FeaError):
        fea.csr_pattern(dofs, nd - 1)  # a DOF outside [0, nrows)


@pytest.mark.parametrize("p", [1, 2])
def test_upper_pattern_is_the_upper_triangle(p):
    """Symmetric storage: the pattern with upper=True is the upper triangle (diagonal included) of
    the full pattern, row by row, and holds (nnz + nrows) / 2 entries."""
    import paper_1604_05872_gb300 as fea
    coords, dofs, nd = inputs.box_mesh(3, p, jitter=0.2)
    rp, ci = fea.csr_pattern(dofs, nd)
    ur, uc = fea.csr_pattern(dofs, nd, upper=True)
    indptr, indices, _ = global_ref.assemble_csr(dofs, np.ones((dofs.shape[0],) + (dofs.shape[1],) * 2), nd, upper=True)
    assert np.array_equal(ur, indptr) and np.array_equal(uc, indices)
    assert 2 * uc.shape[0] == ci.shape[0] + nd
    for r in range(nd):
        row = ci[rp[r]:rp[r + 1]]
        assert np.array_equal(uc[ur[r]:ur[r + 1]], row[row >= r])


@pytest.mark.parametrize("p", [1, 2])
def test_reference_global_matrices_on_the_unit_cube(orc, p):
    """Mass: the entries sum to the volume (1).  Laplacian (Helmholtz with
    f = 0): zero row sums, and u^T K u = int |grad u|^2 = 1 for u = x, exact
    for P1 and P2; both symmetric."""
    coords, dofs, nd = inputs.box_mesh(3, p, jitter=0.2)
    E, n = dofs.shape
    M = orc.assemble(orc.MASS, p, coords)
    K = orc.assemble(orc.HELMHOLTZ, p, coords, np.zeros((E, n)))
    _, _, mdata = global_ref.assemble_csr(dofs, M, nd)
    assert abs(mdata.sum() - 1.0) < 1e-13
    import scipy.sparse as sp
    indptr, indices, kdata = global_ref.assemble_csr(dofs, K, nd)
    Kg = sp.csr_matrix((kdata, indices, indptr), shape=(nd, nd))
    assert np.abs(Kg @ np.ones(nd)).max() < 1e-12
    assert abs(Kg - Kg.T).max() < 1e-13
    # nodal values of u = x at every global DOF (vertices, and edge midpoints for P2)
    x = np.zeros(nd)
    nodes = {1: [0, 1, 2, 3], 2: list(range(10))}[p]
    pos = np.concatenate([coords, 0.5 * (coords[:, [2, 1, 1, 0, 0, 0]] + coords[:, [3, 3, 2, 3, 2, 1]])], axis=1)
    x[dofs.reshape(-1)] = pos[:, nodes, 0].reshape(-1)
    assert abs(x @ (Kg @ x) - 1.0) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("form,p", [(0, 1), (1, 2), (2, 1), (2, 2), (3, 2)])
def test_gpu_global_assembly_matches_reference(fea, orc, form, p):
    import torch
    coords, dofs, nd = inputs.box_mesh(8, p, jitter=0.1)  # 3072 elements
    E = coords.shape[0]
    rng = np.random.default_rng(7)
    scale = np.full(E, 1.0 / 8)  # element size: displacement gradients as on the unit-size workloads
    coeffs = inputs.random_coeffs(form, p, E, rng, scale)
    d = dofs if form < 2 else inputs.vector_dofs(dofs)
    nrows = nd if form < 2 else 3 * nd
    row_ptr, col_idx = fea.csr_pattern(d, nrows)
    c = torch.from_numpy(coords).cuda()
    f = None if form == 0 else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    elem = fea.assemble(form, p, c, f)
    dd = torch.from_numpy(d).cuda()
    rp = torch.from_numpy(row_ptr).cuda()
    ci = torch.from_numpy(col_idx).cuda()
    vals = torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda")
    fea.scatter_add_csr(dd, elem, rp, ci, vals)
    fea.sync()
    got = vals.cpu().numpy()
    # the same element matrices summed by the library sparse sum: summation order only
    _, _, same = global_ref.assemble_csr(d, elem.cpu().numpy(), nrows)
    assert np.abs(got - same).max() <= 1e-12 * np.abs(same).max()
    # against the oracle's element matrices: the FP32 contraction's tolerance
    ref_elem = orc.assemble(form, p, coords, coeffs)
    _, _, ref = global_ref.assemble_csr(d, ref_elem, nrows)
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    # the two-step form (positions once, then search-free scatter) gives the same sums, with
    # 4- and 8-byte maps holding the same positions
    smap = fea.csr_scatter_map(dd, rp, ci)
    smap64 = fea.csr_scatter_map(dd, rp, ci, index_dtype=torch.int64)
    assert smap.dtype == torch.int32 and torch.equal(smap.long(), smap64)
    for m in (smap, smap64):
        vals_m = fea.scatter_add_csr_mapped(m, elem, torch.zeros_like(vals))
        fea.sync()
        assert torch.allclose(vals_m, vals, rtol=0, atol=1e-12 * float(vals.abs().max()))
    # FP32 element input gives the same sums of the rounded values
    vals32 = torch.zeros_like(vals)
    fea.scatter_add_csr(dd, fea.assemble(form, p, c, f, out_f32=True), rp, ci, vals32)
    fea.sync()
    assert torch.allclose(vals32, vals, rtol=0, atol=1e-12 * float(vals.abs().max()))


@pytest.mark.gpu
def test_gpu_scatter_outside_pattern_is_flagged(fea):
    import torch
    coords, dofs, nd = inputs.box_mesh(2, 1)
    row_ptr, col_idx = fea.csr_pattern(np.arange(nd, dtype=np.int32).reshape(-1, 1), nd)  # diagonal only
    c = torch.from_numpy(coords).cuda()
    elem = fea.assemble(0, 1, c)
    vals = torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda")
    fea.scatter_add_csr(torch.from_numpy(dofs).cuda(), elem, torch.from_numpy(row_ptr).cuda(),
                        torch.from_numpy(col_idx).cuda(), vals)
    with pytest.raises(fea.FeaError) as ei:
        fea.sync()
    assert ei.value.code == fea.EINVAL
    # the mapped form: missing entries map to -1 and are flagged at both steps
    dd = torch.from_numpy(dofs).cuda()
    smap = fea.csr_scatter_map(dd, torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col_idx).cuda())
    with pytest.raises(fea.FeaError):
        fea.sync()
    assert int((smap < 0).sum()) == smap.numel() - dofs.size  # only the diagonal entries are in the pattern
    fea.scatter_add_csr_mapped(smap, elem, vals)
    with pytest.raises(fea.FeaError):
        fea.sync()
    bad = dofs.copy()
    bad[3, 2] = nd + 5  # a DOF outside the rows: skipped on the device, flagged
    fea.scatter_add_csr(torch.from_numpy(bad).cuda(), elem, torch.from_numpy(row_ptr).cuda(),
                        torch.from_numpy(col_idx).cuda(), vals)
    with pytest.raises(fea.FeaError):
        fea.sync()


def random_dof_map(E, n, ndofs, rng):
    """An element-to-DOF map with distinct DOFs per element (any degree; no mesh needed)."""
    return np.stack([rng.choice(ndofs, size=n, replace=False) for _ in range(E)]).astype(np.int32)


@pytest.mark.gpu
@pytest.mark.parametrize("form,p,mesh", [(0, 1, True), (1, 1, True), (1, 2, True), (0, 2, True),
                                         (1, 3, False), (0, 3, False)])
@pytest.mark.parametrize("index_dtype", ["int32", "int64"])
def test_gpu_one_pass_global_assembly(fea, orc, form, p, mesh, index_dtype):
    """fea_assemble_csr (element matrices added into the CSR values, never stored) against the
    two-pass form on the same inputs (summation order only) and against the reference global
    matrix of the oracle's element matrices (the FP32 contraction's tolerance)."""
    import torch
    rng = np.random.default_rng(11 + p)
    if mesh:
        coords, dofs, nd = inputs.box_mesh(6, p, jitter=0.1)  # 1296 elements, a ragged last tile
    else:
        E, n = 1111, fea.local_dim(form, p)
        coords, _ = inputs.workload(form, p, E, seed=inputs.SEED + 31)
        nd = 3000
        dofs = random_dof_map(E, n, nd, rng)
    E = coords.shape[0]
    coeffs = None if form == 0 else inputs.random_coeffs(form, p, E, rng)
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    c = torch.from_numpy(coords).cuda()
    f = None if coeffs is None else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    dd, rp, ci = (torch.from_numpy(x).cuda() for x in (dofs, row_ptr, col_idx))
    smap = fea.csr_scatter_map(dd, rp, ci, index_dtype=getattr(torch, index_dtype))
    vals = fea.assemble_csr(form, p, c, f, smap, torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda"))
    two = fea.scatter_add_csr_mapped(smap, fea.assemble(form, p, c, f), torch.zeros_like(vals))
    fea.sync()
    assert torch.allclose(vals, two, rtol=0, atol=1e-12 * float(two.abs().max()))
    ref_elem = orc.assemble(form, p, coords, coeffs)
    _, _, ref = global_ref.assemble_csr(dofs, ref_elem, nd)
    got = vals.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    # accumulation: a second pass doubles the matrix
    fea.assemble_csr(form, p, c, f, smap, vals)
    fea.sync()
    assert torch.allclose(vals, 2 * two, rtol=0, atol=1e-12 * float(two.abs().max()))


@pytest.mark.gpu
def test_gpu_one_pass_rejects_and_flags(fea):
    import torch
    coords, dofs, nd = inputs.box_mesh(2, 1)
    c = torch.from_numpy(coords).cuda()
    dd = torch.from_numpy(dofs).cuda()
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    smap = fea.csr_scatter_map(dd, torch.from_numpy(row_ptr).cuda(), torch.from_numpy(col_idx).cuda())
    vals = torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda")
    fea.sync()
    with pytest.raises(fea.FeaError) as e:  # no one-pass kernel for the vector forms
        fea.assemble_csr(2, 1, c, torch.zeros(c.shape[0] * 8, dtype=torch.float64, device="cuda"), smap, vals)
    assert e.value.code == fea.EINVAL
    with pytest.raises(fea.FeaError):  # nor for P4
        fea.assemble_csr(0, 4, c, None, smap, vals)
    bad = smap.clone()
    bad[5, 1, 2] = col_idx.shape[0] + 7  # a position outside the values: skipped, flagged
    bad[9, 0, 0] = -3
    fea.assemble_csr(0, 1, c, None, bad, vals)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EINVAL
    # every other entry was added: the sum of all element entries (the cube's volume up to the
    # FP32 contraction's rounding) minus the two skipped ones
    m = fea.assemble(0, 1, c).cpu().numpy()
    assert abs(m.sum() - 1.0) < 1e-6
    assert abs(float(vals.sum()) - (m.sum() - m[5, 1, 2] - m[9, 0, 0])) < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("form,p", [(0, 1), (1, 2)])
def test_gpu_symmetric_storage(fea, orc, form, p):
    """Upper-triangle pattern and map: the one-pass and the mapped scatter both give the upper
    triangle of the full global matrix; entries below the diagonal are passed over without an error."""
    import torch
    rng = np.random.default_rng(17)
    coords, dofs, nd = inputs.box_mesh(6, p, jitter=0.1)
    E = coords.shape[0]
    coeffs = None if form == 0 else inputs.random_coeffs(form, p, E, rng)
    c = torch.from_numpy(coords).cuda()
    f = None if coeffs is None else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    dd = torch.from_numpy(dofs).cuda()
    ur, uc = fea.csr_pattern(dofs, nd, upper=True)
    umap = fea.csr_scatter_map(dd, torch.from_numpy(ur).cuda(), torch.from_numpy(uc).cuda(), upper=True)
    fea.sync()  # no entry is missing: the lower ones are marked, not flagged
    assert int((umap == -2).sum()) == int((dofs[:, None, :] < dofs[:, :, None]).sum())
    assert int((umap == -1).sum()) == 0
    one = fea.assemble_csr(form, p, c, f, umap, torch.zeros(uc.shape[0], dtype=torch.float64, device="cuda"))
    two = fea.scatter_add_csr_mapped(umap, fea.assemble(form, p, c, f), torch.zeros_like(one))
    fea.sync()
    full_r, full_c = fea.csr_pattern(dofs, nd)
    fmap = fea.csr_scatter_map(dd, torch.from_numpy(full_r).cuda(), torch.from_numpy(full_c).cuda())
    full = fea.assemble_csr(form, p, c, f, fmap, torch.zeros(full_c.shape[0], dtype=torch.float64, device="cuda"))
    fea.sync()
    import scipy.sparse as sp
    A = sp.csr_matrix((full.cpu().numpy(), full_c, full_r), shape=(nd, nd))
    U = sp.triu(A, k=0, format="csr")
    U.sort_indices()
    assert np.array_equal(U.indptr, ur) and np.array_equal(U.indices, uc)
    scale = float(np.abs(U.data).max())
    assert np.abs(one.cpu().numpy() - U.data).max() <= 1e-12 * scale
    assert np.abs(two.cpu().numpy() - U.data).max() <= 1e-12 * scale
    # against the oracle's element matrices
    _, _, ref = global_ref.assemble_csr(dofs, orc.assemble(form, p, coords, coeffs), nd, upper=True)
    assert np.linalg.norm(one.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)


# ---- combining plan (host builder, checked on the CPU) and the combined one-pass kernel ----

def host_scatter_map(dofs, row_ptr, col_idx, upper=False):
    """Positions of every (e, i, j) in the CSR values, by a per-entry search (numpy); -2 below
    the diagonal under symmetric storage."""
    E, n = dofs.shape
    m = np.empty((E, n, n), dtype=np.int64)
    for e in range(E):
        for i in range(n):
            r = dofs[e, i]
            seg = col_idx[row_ptr[r]:row_ptr[r + 1]]
            for j in range(n):
                c = dofs[e, j]
                m[e, i, j] = -2 if (upper and c < r) else row_ptr[r] + int(np.searchsorted(seg, c))
    return m


def decode_combine_plan(plan, E, n):
    """Tiles of the plan as lists of (position, [tile entries]) in stored order, after checking
    the layout rules the kernel relies on."""
    T = min(128, max(2, (3200 // (n * n)) & ~1))
    assert plan[0] == 0x46435031 and plan[1] == n and plan[2] == T
    ntiles = (E + T - 1) // T
    off = plan[4:4 + 2 * (ntiles + 1)].view(np.int64)
    assert off[0] >= 4 + 2 * (ntiles + 1) and off[-1] == plan.shape[0]
    tiles = []
    for t in range(ntiles):
        a, b = int(off[t]), int(off[t + 1])
        assert a % 4 == 0 and a < b
        U, R, L = (int(x) for x in plan[a:a + 3])
        cw, pw, iw = (R + 3) & ~3, (U + 3) & ~3, ((L + 1) // 2 + 3) & ~3
        assert a + 4 + cw + pw + iw == b
        cnt = plan[a + 4:a + 4 + R]
        assert (R == 0 and U == 0) or (cnt[0] == U and np.all(np.diff(cnt) <= 0) and cnt[-1] > 0)
        assert int(cnt.sum()) == L
        pos = plan[a + 4 + cw:a + 4 + cw + U]
        idx = plan[a + 4 + cw + pw:b].view(np.uint16)[:L]
        groups = [[] for _ in range(U)]
        o = 0
        for r in range(R):
            for s in range(int(cnt[r])):
                groups[s].append(int(idx[o + s]))
            o += int(cnt[r])
        tiles.append(list(zip(pos.tolist(), groups)))
    return T, tiles


@pytest.mark.parametrize("p,upper,ragged", [(1, False, False), (2, False, True), (2, True, False), (3, False, True)])
def test_combine_plan_groups_every_entry_at_its_position(p, upper, ragged):
    """Every stored entry of a tile appears exactly once, under the position the map gives it;
    positions are distinct within a tile and ordered by their number of entries; entries below
    the diagonal (symmetric storage) are left out."""
    import paper_1604_05872_gb300 as fea
    rng = np.random.default_rng(5 + p)
    if p < 3:
        coords, dofs, nd = inputs.box_mesh(3 if p == 2 else 5, p, jitter=0.1)
        if ragged:
            dofs = dofs[:-7]
    else:
        nd = 400
        dofs = random_dof_map(75, 20, nd, rng)
    E, n = dofs.shape
    row_ptr, col_idx = fea.csr_pattern(dofs, nd, upper=upper)
    m = host_scatter_map(dofs, row_ptr, col_idx, upper=upper)
    for dt in (np.int32, np.int64):
        plan = fea.csr_combine_plan(m.astype(dt), col_idx.shape[0])
        T, tiles = decode_combine_plan(plan, E, n)
        nn = n * n
        for t, slots in enumerate(tiles):
            flat = m[t * T:(t + 1) * T].reshape(-1)
            seen = np.zeros(flat.shape[0], dtype=np.int64)
            for pos, ks in slots:
                for k in ks:
                    assert flat[k] == pos
                    seen[k] += 1
            assert np.array_equal(seen, (flat != -2).astype(np.int64))
            assert len({pos for pos, _ in slots}) == len(slots)
            mult = [len(ks) for _, ks in slots]
            assert mult == sorted(mult, reverse=True)
            assert all(k < nn * min(T, E - t * T) for _, ks in slots for k in ks)


@pytest.mark.parametrize("form,p", [(0, 1), (1, 2)])
def test_combined_sums_give_the_reference_global_matrix(orc, form, p):
    """Summing the oracle's element matrices tile by tile as the plan groups them, one addition
    per distinct position, reproduces the reference global matrix (a library sparse sum)."""
    import paper_1604_05872_gb300 as fea
    rng = np.random.default_rng(23)
    coords, dofs, nd = inputs.box_mesh(3, p, jitter=0.1)
    E, n = dofs.shape
    coeffs = None if form == 0 else inputs.random_coeffs(form, p, E, rng)
    elem = orc.assemble(form, p, coords, coeffs)
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    plan = fea.csr_combine_plan(host_scatter_map(dofs, row_ptr, col_idx), col_idx.shape[0])
    T, tiles = decode_combine_plan(plan, E, n)
    vals = np.zeros(col_idx.shape[0])
    adds = 0
    for t, slots in enumerate(tiles):
        flat = elem[t * T:(t + 1) * T].reshape(-1)
        for pos, ks in slots:
            vals[pos] += flat[ks].sum()
            adds += 1
    _, _, ref = global_ref.assemble_csr(dofs, elem, nd)
    assert np.abs(vals - ref).max() <= 1e-13 * np.abs(ref).max()
    assert adds < E * n * n  # entries of a tile that meet were combined


def test_combine_plan_rejects_bad_maps():
    import ctypes
    import paper_1604_05872_gb300 as fea
    _, dofs, nd = inputs.box_mesh(2, 1)
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    m = host_scatter_map(dofs, row_ptr, col_idx)
    nnz = col_idx.shape[0]
    for bad_value in (nnz, -1, -3):
        bad = m.copy()
        bad[3, 1, 2] = bad_value
        with pytest.raises(fea.FeaError) as e:
            fea.csr_combine_plan(bad, nnz)
        assert e.value.code == fea.EINVAL
    with pytest.raises(fea.FeaError):  # 32-bit positions only
        fea.csr_combine_plan(m, 2 ** 31)
    with pytest.raises(fea.FeaError):  # 16-bit tile entries: n^2 T <= 65536
        fea.csr_combine_plan(np.zeros((1, 182, 182), dtype=np.int32), 1)
    # a buffer smaller than the size query is refused
    words = ctypes.c_int64(0)
    lib = fea.load()
    mm = np.ascontiguousarray(m)
    assert lib.fea_csr_combine_plan(mm.shape[0], 4, mm.ctypes.data, 1, nnz, None, ctypes.byref(words)) == 0
    buf = np.zeros(words.value, dtype=np.int32)
    small = ctypes.c_int64(words.value - 1)
    assert lib.fea_csr_combine_plan(mm.shape[0], 4, mm.ctypes.data, 1, nnz, buf.ctypes.data,
                                    ctypes.byref(small)) == fea.EINVAL
    # an empty mesh: a header and one offset
    plan = fea.csr_combine_plan(np.zeros((0, 4, 4), dtype=np.int32), 0)
    assert plan.shape[0] == 8 and plan[0] == 0x46435031


@pytest.mark.gpu
@pytest.mark.parametrize("form,p,mesh", [(0, 1, True), (1, 1, True), (1, 2, True), (0, 2, True),
                                         (1, 3, False), (0, 3, False)])
@pytest.mark.parametrize("upper", [False, True])
def test_gpu_combined_global_assembly(fea, orc, form, p, mesh, upper):
    """fea_assemble_csr_combined against the two-pass assembly on the same inputs (the order of the
    FP64 additions only) and against the reference global matrix of the oracle's element
    matrices (the FP32 contraction's tolerance); full and symmetric storage; ragged last tile."""
    import torch
    rng = np.random.default_rng(41 + p)
    if mesh:
        coords, dofs, nd = inputs.box_mesh(6, p, jitter=0.1)  # 1296 elements, a ragged last tile
    else:
        E, n = 1111, fea.local_dim(form, p)
        coords, _ = inputs.workload(form, p, E, seed=inputs.SEED + 37)
        nd = 3000
        dofs = random_dof_map(E, n, nd, rng)
    E = coords.shape[0]
    coeffs = None if form == 0 else inputs.random_coeffs(form, p, E, rng)
    row_ptr, col_idx = fea.csr_pattern(dofs, nd, upper=upper)
    c = torch.from_numpy(coords).cuda()
    f = None if coeffs is None else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    dd, rp, ci = (torch.from_numpy(x).cuda() for x in (dofs, row_ptr, col_idx))
    smap = fea.csr_scatter_map(dd, rp, ci, upper=upper)
    plan = torch.from_numpy(fea.csr_combine_plan(smap, col_idx.shape[0])).cuda()
    vals = fea.assemble_csr_combined(form, p, c, f, plan,
                                     torch.zeros(col_idx.shape[0], dtype=torch.float64, device="cuda"))
    two = fea.scatter_add_csr_mapped(smap, fea.assemble(form, p, c, f), torch.zeros_like(vals))
    fea.sync()
    assert torch.allclose(vals, two, rtol=0, atol=1e-12 * float(two.abs().max()))
    _, _, ref = global_ref.assemble_csr(dofs, orc.assemble(form, p, coords, coeffs), nd, upper=upper)
    got = vals.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
    fea.assemble_csr_combined(form, p, c, f, plan, vals)  # accumulates
    fea.sync()
    assert torch.allclose(vals, 2 * two, rtol=0, atol=1e-12 * float(two.abs().max()))


@pytest.mark.gpu
def test_gpu_combined_rejects_and_flags(fea):
    """Wrong form or degree, a short or misaligned plan: refused on the host.  A plan of another
    tile size or with a position outside the values: flagged (FEA_EINVAL at the next sync), the
    offending tile or position skipped, every other position added."""
    import torch
    coords, dofs, nd = inputs.box_mesh(2, 1)  # 48 elements: one tile of 128 at P1
    c = torch.from_numpy(coords).cuda()
    row_ptr, col_idx = fea.csr_pattern(dofs, nd)
    nnz = col_idx.shape[0]
    smap = fea.csr_scatter_map(torch.from_numpy(dofs).cuda(), torch.from_numpy(row_ptr).cuda(),
                               torch.from_numpy(col_idx).cuda())
    host = fea.csr_combine_plan(smap, nnz)
    plan = torch.from_numpy(host).cuda()
    vals = torch.zeros(nnz, dtype=torch.float64, device="cuda")
    fea.sync()
    with pytest.raises(fea.FeaError) as e:  # no combined kernel for the vector forms
        fea.assemble_csr_combined(2, 1, c, torch.zeros(c.shape[0] * 8, dtype=torch.float64, device="cuda"), plan, vals)
    assert e.value.code == fea.EINVAL
    with pytest.raises(fea.FeaError):  # nor for P4
        fea.assemble_csr_combined(0, 4, c, None, plan, vals)
    with pytest.raises(fea.FeaError):  # shorter than its header for this many elements
        fea.assemble_csr_combined(0, 1, c, None, plan[:5], vals)
    with pytest.raises(fea.FeaError):  # not 16-byte aligned
        fea.assemble_csr_combined(0, 1, c, None, plan[1:], vals)
    # a plan for the P2 tile size used at P1: the kernel refuses it whole
    other = host.copy()
    other[2] = 64
    fea.assemble_csr_combined(0, 1, c, None, torch.from_numpy(other).cuda(), vals)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EINVAL
    assert float(vals.abs().sum()) == 0.0
    # one position outside the values: that position is skipped, the rest added
    a = int(host[4:6].view(np.int64)[0])
    R, U = int(host[a + 1]), int(host[a])
    pos_at = a + 4 + ((R + 3) & ~3)
    bad = host.copy()
    bad[pos_at + U - 1] = nnz + 5
    fea.assemble_csr_combined(0, 1, c, None, torch.from_numpy(bad).cuda(), vals)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.EINVAL
    full = fea.assemble_csr_combined(0, 1, c, None, plan, torch.zeros_like(vals))
    fea.sync()
    skipped = int(host[pos_at + U - 1])
    diff = (full - vals).cpu().numpy()
    assert diff[skipped] == float(full[skipped]) and np.delete(diff, skipped).max() == 0.0
