"""The allocation-free batched entry point against the regular one.

fea_assemble_batch_noalloc is for callers that cannot allocate device memory
at the moment they assemble (code inside another framework's memory pool, or a
latency-critical loop where an allocation may block or fail): its scratch is a
fixed device array inside the library.  Here it must give the same element
matrices as fea_assemble_batch on two calls in a row (the second call reuses
the array the first one left behind), allocate nothing while it runs, and
refuse the two cases its documentation names.  This file is collected last so
that a stop at the first failure has run every other test.
"""
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu

REQS = [(0, 1, 300), (1, 2, 1234), (2, 3, 37), (3, 2, 91), (1, 4, 13), (2, 2, 250), (3, 1, 77), (0, 3, 45)]


def build(fea, seed):
    out = []
    for k, (form, p, E) in enumerate(REQS):
        coords, coeffs = inputs.workload(form, p, E, seed=seed + k)
        c = torch.from_numpy(coords).cuda()
        f = None if form == inputs.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
        out.append((form, p, c, f))
    return out


def rel_err(a, b):
    a = a.reshape(a.shape[0], -1).double()
    b = b.reshape(b.shape[0], -1).double()
    return ((a - b).norm(dim=1) / b.norm(dim=1)).max().item()


def test_noalloc_batch_matches_regular_batch_twice(fea):
    data = build(fea, 900)
    ref = [fea.empty_out(form, p, c.shape[0]) for (form, p, c, f) in data]
    # the regular entry point (it also makes the tables resident on this device)
    fea.assemble_batch([(form, p, c, f, o) for (form, p, c, f), o in zip(data, ref)])
    fea.sync()
    for call in range(2):
        outs = [torch.full_like(o, float("nan")) for o in ref]
        torch.cuda.synchronize()
        before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        fea.assemble_batch_noalloc([(form, p, c, f, o) for (form, p, c, f), o in zip(data, outs)])
        fea.sync()
        after = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        if call == 1:  # the first call may still load the library's kernels; the second allocates nothing
            assert after == before, (before, after)
        for (form, p, c, f), o, r in zip(data, outs, ref):
            assert torch.isfinite(o).all(), (call, form, p)
            assert rel_err(o, r) <= 1e-5, (call, form, p)


def test_noalloc_batch_rejects_too_many_requests(fea):
    form, p, c, f = build(fea, 950)[0]
    o = fea.empty_out(form, p, c.shape[0])
    with pytest.raises(fea.FeaError) as e:
        fea.assemble_batch_noalloc([(form, p, c, f, o)] * 513)
    assert e.value.code == fea.EINVAL


def test_noalloc_batch_refuses_without_state_or_tables(fea):
    data = build(fea, 970)
    form, p, c, f = data[1]    # Helmholtz P2
    form2, p2, c2, f2 = data[2]  # elasticity P3
    o = fea.empty_out(form, p, c.shape[0])
    o2 = fea.empty_out(form2, p2, c2.shape[0])
    fea.finalize()  # no library state on this device any more
    with pytest.raises(fea.FeaError) as e:
        fea.assemble_batch_noalloc([(form, p, c, f, o)])
    assert e.value.code == fea.EINVAL
    # an allocating call makes the state and the Helmholtz P2 tables, not the elasticity P3 ones
    ref = fea.assemble(form, p, c, f)
    fea.sync()
    with pytest.raises(fea.FeaError) as e:
        fea.assemble_batch_noalloc([(form2, p2, c2, f2, o2)])
    assert e.value.code == fea.EINVAL
    fea.assemble_batch_noalloc([(form, p, c, f, o)])
    fea.sync()
    assert rel_err(o, ref) <= 1e-5
