"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

* A bounded wait made to run out: fea_test_skip_input_copy makes the next launch
  skip one tile's bulk input copy, so the CTA that runs that tile waits for
  inputs that never come.  Its wait gives up after a few seconds, the CTA
  leaves once its other copies have landed, fea_sync reports FEA_ETIMEOUT, and
  the next call on the same context succeeds with the same results as before.
* Padding canaries: outputs written into the middle of a larger buffer whose
  guard regions hold a sentinel pattern, on ragged sizes, for every kernel
  family; the guards must come back untouched.
"""
import numpy as np
import pytest
import torch

from paper_1604_05872_gb300 import inputs

pytestmark = pytest.mark.gpu


def to_dev(coords, coeffs, form, p):
    c = torch.from_numpy(np.ascontiguousarray(coords)).cuda()
    f = None if form == inputs.MASS else torch.from_numpy(inputs.coeff_array(form, p, coeffs)).cuda()
    return c, f


@pytest.mark.parametrize("form,p,prec,E", [(1, 2, 1, 20000), (0, 3, 1, 9000), (3, 2, 2, 6000), (3, 3, 2, 3000)])
def test_skipped_input_copy_times_out_and_context_survives(fea, form, p, prec, E):
    coords, coeffs = inputs.workload(form, p, E, seed=4100 + 10 * form + p)
    c, f = to_dev(coords, coeffs, form, p)
    good = fea.assemble(form, p, c, f, precision=prec)
    fea.sync()
    fea.skip_input_copy_once(3)
    fea.assemble(form, p, c, f, precision=prec)
    with pytest.raises(fea.FeaError) as e:
        fea.sync()
    assert e.value.code == fea.ETIMEOUT
    fea.sync()  # the error word was cleared
    again = fea.assemble(form, p, c, f, precision=prec)
    fea.sync()
    assert torch.equal(again, good)


@pytest.mark.parametrize("form,p,prec,variant,f32", [
    (1, 2, 1, -1, False), (1, 2, 1, -1, True),   # streaming pre-evaluated kernel
    (0, 4, 1, -1, False),                        # pre-evaluated tile kernel
    (2, 3, 1, 2, False), (2, 3, 1, 2, True),     # vector streaming kernel
    (3, 3, 1, -1, False),                        # vector sharing-elimination tile kernel
    (3, 2, 2, -1, False), (3, 2, 2, -1, True),   # tensor-core kernel, shared reference operand
    (3, 3, 2, -1, False), (3, 3, 2, -1, True),   # tensor-core kernel, one product per element
    (1, 3, 0, -1, False),                        # FP64 path
    (2, 2, 0, 0, False),                         # plain FP64 comparator
])
def test_outputs_stay_inside_their_buffer(fea, form, p, prec, variant, f32):
    tile = fea.plan(form, p, precision=prec, variant=variant)["tile"]
    E = 3 * tile + 1
    coords, coeffs = inputs.workload(form, p, E, seed=4200 + 10 * form + p)
    c, f = to_dev(coords, coeffs, form, p)
    n = fea.local_dim(form, p)
    dt = torch.float32 if f32 else torch.float64
    G = 2  # guard elements on each side (keeps the output 16-byte aligned)
    buf = torch.full((E + 2 * G, n, n), -12345.678, dtype=dt, device="cuda")
    out = buf[G:G + E]
    fea.assemble(form, p, c, f, out=out, precision=prec, variant=variant, out_f32=f32)
    fea.sync()
    guards = torch.cat([buf[:G], buf[G + E:]])
    assert bool((guards == -12345.678).all()), (form, p, prec, variant, f32)
    assert bool(torch.isfinite(out).all())
