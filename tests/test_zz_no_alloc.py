"""The allocation-free batched entry point against the regular one.

fea_assemble_batch_noalloc exists for callers that cannot allocate device
memory when they assemble (graph capture, foreign memory pools, latency-bound
loops): its scratch is a fixed device array inside the library.  Here it must
give the same element matrices as fea_assemble_batch, on two calls in a row
(the second call reuses the array the first one left behind).  This file is
collected last so that a stop at the first failure has run every other test.
"""
import numpy as np
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
        fea.assemble_batch_noalloc([(form, p, c, f, o) for (form, p, c, f), o in zip(data, outs)])
        fea.sync()
        for (form, p, c, f), o, r in zip(data, outs, ref):
            assert torch.isfinite(o).all(), (call, form, p)
            assert rel_err(o, r) <= 1e-5, (call, form, p)


def test_noalloc_batch_rejects_too_many_requests(fea):
    form, p, c, f = build(fea, 950)[0]
    o = fea.empty_out(form, p, c.shape[0])
    with pytest.raises(fea.FeaError) as e:
        fea.assemble_batch_noalloc([(form, p, c, f, o)] * 513)
    assert e.value.code == fea.EINVAL
