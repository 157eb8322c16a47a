"""GB300 (sm_103a) batched element-local assembly.

Thin Python binding of the C ABI declared in include/fea.h: argument
marshalling only.  Every step of the assembly runs in the CUDA library
libfea.so (built in-tree by ``build.py``); there is no CPU fallback, and every
call raises ``FeaError`` if the library is missing or a call fails.

Tensors are torch tensors (device memory and streams come from PyTorch):
coords float64 [E, 4, 3], coefficients float64 (flat, ``coeffs_size``
doubles), output float64 or float32 [E, n, n].
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfea.so")

MASS, HELMHOLTZ, ELASTICITY, NEOHOOKEAN = 0, 1, 2, 3
FORMS = {"mass": MASS, "helmholtz": HELMHOLTZ, "elasticity": ELASTICITY, "neohookean": NEOHOOKEAN}
OK, EINVAL, ENOMEM, ECUDA, EDEGENERATE, ETIMEOUT = 0, 1, 2, 3, 4, 5
PREC_FP64, PREC_FP32, PREC_BF16X2 = 0, 1, 2
VARIANT_AUTO, VARIANT_NAIVE, VARIANT_SE, VARIANT_PRE = -1, 0, 1, 2
VARIANT_NAMES = {VARIANT_NAIVE: "naive", VARIANT_SE: "se", VARIANT_PRE: "pre"}

EXPORTS = ["fea_local_dim", "fea_coeff_len", "fea_coeffs_size", "fea_quad_points", "fea_assemble",
           "fea_assemble_vector", "fea_csr_pattern", "fea_scatter_add_csr",
           "fea_csr_scatter_map", "fea_scatter_add_csr_mapped", "fea_assemble_csr", "fea_csr_combine_plan",
           "fea_assemble_csr_combined", "fea_log_f64",
           "fea_assemble_ex", "fea_assemble_host", "fea_assemble_batch", "fea_assemble_batch_fused",
           "fea_assemble_batch_noalloc",
           "fea_sync", "fea_test_skip_input_copy", "fea_plan", "fea_plan_flop",
           "fea_op_count", "fea_opcount_program", "fea_sharing_elimination", "fea_vertex_cover",
           "fea_increase_factor", "fea_num_monomials", "fea_theta", "fea_algorithm3",
           "fea_tune_set", "fea_tune_clear", "fea_mlp_num_params", "fea_mlp_scratch_floats",
           "fea_mlp_forward", "fea_mlp_loss_grad", "fea_mlp_adam",
           "fea_last_error", "fea_finalize"]


class FeaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fea error %d: %s" % (code, msg))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("out_f32", ctypes.c_int), ("variant", ctypes.c_int),
                ("tile", ctypes.c_int), ("smem_budget", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("degree", ctypes.c_int), ("E", ctypes.c_int64),
                ("coords", ctypes.c_void_p), ("coeffs", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("tile", ctypes.c_int), ("threads", ctypes.c_int),
                ("quad_points", ctypes.c_int), ("ref_terms", ctypes.c_int), ("smem_bytes", ctypes.c_size_t),
                ("flops_naive", ctypes.c_int64), ("flops_se", ctypes.c_int64), ("flops_pre", ctypes.c_int64),
                ("flops_run", ctypes.c_int64), ("bytes", ctypes.c_int64)]


_lib = None


def load(path=None):
    """Load libfea.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise FeaError(ECUDA, "CUDA library %s is missing: run __graft_entry__.build() first" % path)
    lib = ctypes.CDLL(path)
    i, i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    P = ctypes.POINTER
    lib.fea_local_dim.argtypes = [i, i]
    lib.fea_coeff_len.argtypes = [i, i]
    lib.fea_coeffs_size.argtypes = [i, i, i64]
    lib.fea_coeffs_size.restype = i64
    lib.fea_quad_points.argtypes = [i, i]
    lib.fea_assemble.argtypes = [i, i, i64, vp, vp, vp, vp]
    lib.fea_assemble_bernstein.argtypes = [i, i, i64, vp, vp, vp, i, vp]
    lib.fea_assemble_ex.argtypes = [i, i, i64, vp, vp, vp, P(Options), vp]
    lib.fea_assemble_host.argtypes = [i, i, i64, vp, vp, vp, P(Options), vp]
    lib.fea_assemble_batch.argtypes = [P(Request), i, P(Options), vp]
    lib.fea_assemble_batch_fused.argtypes = [P(Request), i, P(Options), vp]
    lib.fea_assemble_vector.argtypes = [i, i, i64, vp, vp, vp, P(Options), vp]
    lib.fea_csr_pattern.argtypes = [i64, i, vp, i64, i, vp, vp, P(i64)]
    lib.fea_scatter_add_csr.argtypes = [i64, i, vp, vp, i, i64, vp, vp, i64, vp, vp]
    lib.fea_csr_scatter_map.argtypes = [i64, i, vp, i64, vp, vp, i64, i, vp, i, vp]
    lib.fea_log_f64.argtypes = [vp, vp, i64, vp]
    lib.fea_assemble_csr.argtypes = [i, i, i64, vp, vp, vp, i, i64, vp, vp]
    lib.fea_csr_combine_plan.argtypes = [i64, i, vp, i, i64, vp, P(i64)]
    lib.fea_assemble_csr_combined.argtypes = [i, i, i64, vp, vp, vp, i64, i64, vp, vp]
    lib.fea_scatter_add_csr_mapped.argtypes = [i64, i, vp, i, vp, i, i64, vp, vp]
    lib.fea_assemble_batch_noalloc.argtypes = [P(Request), i, P(Options), vp]
    lib.fea_sync.argtypes = [vp]
    lib.fea_test_skip_input_copy.argtypes = [i64]
    lib.fea_plan.argtypes = [i, i, P(Options), P(PlanInfo)]
    lib.fea_plan_flop.argtypes = [i, i, P(Options), P(PlanInfo)]
    lib.fea_op_count.argtypes = [i, i, i, P(i64), P(i64)]
    cp = ctypes.c_char_p
    lib.fea_opcount_program.argtypes = [cp, cp, P(i64)]
    lib.fea_sharing_elimination.argtypes = [cp, cp, cp, cp, ctypes.c_char_p, ctypes.c_size_t, P(i64), P(i)]
    lib.fea_vertex_cover.argtypes = [i, i, P(i), i, P(i)]
    lib.fea_increase_factor.argtypes = [i, i]
    lib.fea_increase_factor.restype = i64
    lib.fea_num_monomials.argtypes = [i, i]
    lib.fea_theta.argtypes = [i, i, i, P(i64), P(i64), P(i64)]
    lib.fea_algorithm3.argtypes = [i, i, i, ctypes.c_size_t, P(ctypes.c_uint), P(i64)]
    lib.fea_tune_set.argtypes = [i, i, i, i, i]
    lib.fea_tune_clear.argtypes = []
    lib.fea_tune_clear.restype = None
    lib.fea_mlp_num_params.argtypes = [i, i]
    lib.fea_mlp_scratch_floats.argtypes = [i, i]
    lib.fea_mlp_scratch_floats.restype = i64
    lib.fea_mlp_forward.argtypes = [vp, i, i, vp, i, vp, vp]
    lib.fea_mlp_loss_grad.argtypes = [vp, i, i, vp, vp, i, vp, vp, vp, vp]
    lib.fea_mlp_adam.argtypes = [vp, vp, vp, vp, i, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, i, vp]
    lib.fea_last_error.restype = ctypes.c_char_p
    lib.fea_finalize.argtypes = []
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        raise FeaError(rc, load().fea_last_error().decode())


def options(precision=PREC_FP32, out_f32=False, variant=VARIANT_AUTO, tile=0, smem_budget=0):
    return Options(int(precision), int(bool(out_f32)), int(variant), int(tile), int(smem_budget))


def local_dim(form, degree):
    return load().fea_local_dim(form, degree)


def coeff_len(form, degree):
    return load().fea_coeff_len(form, degree)


def coeffs_size(form, degree, E):
    return load().fea_coeffs_size(form, degree, E)


def quad_points(form, degree):
    return load().fea_quad_points(form, degree)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def empty_out(form, degree, E, out_f32=False, device="cuda"):
    import torch
    n = local_dim(form, degree)
    if n < 0:
        raise FeaError(EINVAL, "unsupported form/degree (%r, %r)" % (form, degree))
    return torch.empty((E, n, n), dtype=torch.float32 if out_f32 else torch.float64, device=device)


def assemble(form, degree, coords, coeffs=None, out=None, precision=PREC_FP32, out_f32=False,
             variant=VARIANT_AUTO, tile=0, smem_budget=0, stream=None):
    """Element matrices of E elements (device tensors); returns `out`."""
    E = coords.shape[0]
    if out is None:
        out = empty_out(form, degree, E, out_f32, coords.device)
    o = options(precision, out_f32, variant, tile, smem_budget)
    _check(load().fea_assemble_ex(form, degree, E, _ptr(coords), _ptr(coeffs), _ptr(out), ctypes.byref(o),
                                  _stream_ptr(stream)))
    return out


def assemble_default(form, degree, coords, coeffs, out, stream=None):
    """fea_assemble: the 5-argument call with default options."""
    _check(load().fea_assemble(form, degree, coords.shape[0], _ptr(coords), _ptr(coeffs), _ptr(out),
                               _stream_ptr(stream)))
    return out


def assemble_host(form, degree, coords, coeffs, out, precision=PREC_FP32, out_f32=False, variant=VARIANT_AUTO,
                  tile=0, stream=None):
    """Same with HOST tensors (pinned for full bandwidth); copies inside the call."""
    o = options(precision, out_f32, variant, tile, 0)
    _check(load().fea_assemble_host(form, degree, coords.shape[0], _ptr(coords), _ptr(coeffs), _ptr(out),
                                    ctypes.byref(o), _stream_ptr(stream)))
    return out


def assemble_vector(form, degree, coords, coeffs, out=None, precision=PREC_FP32, out_f32=False, tile=0,
                    smem_budget=0, stream=None):
    """Element vectors of the linear forms (fea_assemble_vector): the Helmholtz
    load vector [E, n_p] or the Neo-Hookean residual [E, 3 n_p]; returns `out`."""
    import torch
    E = coords.shape[0]
    n = local_dim(form, degree)
    if n < 0:
        raise FeaError(1, "unsupported form/degree")
    if out is None:
        out = torch.empty((E, n), dtype=torch.float32 if out_f32 else torch.float64, device=coords.device)
    o = options(precision, out_f32, VARIANT_AUTO, tile, smem_budget)
    _check(load().fea_assemble_vector(form, degree, E, _ptr(coords), _ptr(coeffs), _ptr(out), ctypes.byref(o),
                                      _stream_ptr(stream)))
    return out


def assemble_bernstein(form, degree, coords, coeffs, out=None, out_f32=False, stream=None):
    """Helmholtz element matrices [E, n_p, n_p] in the Bernstein-Bezier basis by sum
    factorisation (fea_assemble_bernstein); coeffs [E, n_p]: Bernstein coefficients of f."""
    import torch
    E = coords.shape[0]
    n = local_dim(form, degree)
    if n < 0:
        raise FeaError(1, "unsupported form/degree")
    if out is None:
        out = torch.empty((E, n, n), dtype=torch.float32 if out_f32 else torch.float64, device=coords.device)
    _check(load().fea_assemble_bernstein(form, degree, E, _ptr(coords), _ptr(coeffs), _ptr(out), int(bool(out_f32)),
                                         _stream_ptr(stream)))
    return out


def csr_pattern(dofs, nrows, upper=False):
    """CSR pattern (row_ptr int64 [nrows + 1], col_idx int32 [nnz]) of the element-to-DOF map
    `dofs` (host int32 array [E, n]); upper=True keeps columns >= row only (symmetric storage);
    fea_csr_pattern, built on the host."""
    import numpy as np
    d = np.ascontiguousarray(dofs, dtype=np.int32)
    E, n = d.shape
    nnz = ctypes.c_int64(0)
    _check(load().fea_csr_pattern(E, n, d.ctypes.data, nrows, int(bool(upper)), None, None, ctypes.byref(nnz)))
    row_ptr = np.empty(nrows + 1, dtype=np.int64)
    col_idx = np.empty(max(1, nnz.value), dtype=np.int32)
    _check(load().fea_csr_pattern(E, n, d.ctypes.data, nrows, int(bool(upper)), row_ptr.ctypes.data,
                                  col_idx.ctypes.data, ctypes.byref(nnz)))
    return row_ptr, col_idx[:nnz.value]


def scatter_add_csr(dofs, elem, row_ptr, col_idx, values, stream=None):
    """values += the element matrices `elem` [E, n, n] (device, double or float) at the global DOFs
    `dofs` [E, n] (device int32) of the CSR pattern (row_ptr int64, col_idx int32, values double;
    device); fea_scatter_add_csr.  Returns `values`."""
    import torch
    E, n = dofs.shape
    f32 = elem.dtype == torch.float32
    _check(load().fea_scatter_add_csr(E, n, _ptr(dofs), _ptr(elem), int(f32), row_ptr.shape[0] - 1, _ptr(row_ptr),
                                      _ptr(col_idx), col_idx.shape[0], _ptr(values), _stream_ptr(stream)))
    return values


def csr_scatter_map(dofs, row_ptr, col_idx, stream=None, index_dtype=None, upper=False):
    """CSR position of every (element, i, j) [E, n, n] (device); fea_csr_scatter_map.  int32
    when the pattern has fewer than 2^31 entries (index_dtype=None), else int64; upper=True for a
    pattern of the upper triangle (entries below the diagonal map to -2, not stored)."""
    import torch
    E, n = dofs.shape
    nnz = col_idx.shape[0]
    if index_dtype is None:
        index_dtype = torch.int32 if nnz < 2 ** 31 else torch.int64
    m = torch.empty((E, n, n), dtype=index_dtype, device=dofs.device)
    _check(load().fea_csr_scatter_map(E, n, _ptr(dofs), row_ptr.shape[0] - 1, _ptr(row_ptr), _ptr(col_idx),
                                      nnz, int(bool(upper)), _ptr(m), int(index_dtype == torch.int64),
                                      _stream_ptr(stream)))
    return m


def assemble_csr(form, degree, coords, coeffs, scatter_map, values, stream=None):
    """Local and global assembly in one pass (mass, Helmholtz P1-P3): values[map] += A_e, the
    element matrices never stored; fea_assemble_csr.  Returns `values`."""
    import torch
    if scatter_map.dtype not in (torch.int32, torch.int64):
        raise TypeError("scatter map must be int32 or int64")
    _check(load().fea_assemble_csr(form, degree, coords.shape[0], _ptr(coords), _ptr(coeffs),
                                   _ptr(scatter_map), int(scatter_map.dtype == torch.int64), values.shape[0],
                                   _ptr(values), _stream_ptr(stream)))
    return values


def csr_combine_plan(scatter_map, nnz):
    """Combining plan of the one-pass global assembly (int32 words, numpy) from a position map
    [E, n, n] (int32 or int64; numpy, or a tensor, copied to the host); fea_csr_combine_plan.
    For every tile of elements: the distinct CSR positions its entries fall on and which
    entries meet at each."""
    import numpy as np
    m = scatter_map.cpu().numpy() if hasattr(scatter_map, "cpu") else scatter_map
    if m.dtype not in (np.int32, np.int64) or m.ndim != 3 or m.shape[1] != m.shape[2]:
        raise TypeError("scatter map must be an int32 or int64 array [E, n, n]")
    m = np.ascontiguousarray(m)
    E, n = m.shape[0], m.shape[1]
    words = ctypes.c_int64(0)
    lib = load()
    _check(lib.fea_csr_combine_plan(E, n, m.ctypes.data, int(m.dtype == np.int64), nnz, None, ctypes.byref(words)))
    plan = np.zeros(words.value, dtype=np.int32)
    _check(lib.fea_csr_combine_plan(E, n, m.ctypes.data, int(m.dtype == np.int64), nnz, plan.ctypes.data,
                                    ctypes.byref(words)))
    return plan[:words.value]


def assemble_csr_combined(form, degree, coords, coeffs, plan, values, stream=None):
    """fea_assemble_csr with a tile's entries combined per CSR position before the FP64 atomics:
    values += the global matrix (mass, Helmholtz P1-P3); `plan` is the device copy (int32 tensor)
    of csr_combine_plan.  Returns `values`."""
    import torch
    if plan.dtype != torch.int32:
        raise TypeError("plan must be int32")
    _check(load().fea_assemble_csr_combined(form, degree, coords.shape[0], _ptr(coords), _ptr(coeffs), _ptr(plan),
                                            plan.numel(), values.shape[0], _ptr(values), _stream_ptr(stream)))
    return values


def log_f64(x, stream=None):
    """ln x of a float64 device tensor by the kernels' table-driven FP64 logarithm; fea_log_f64."""
    import torch
    x = x.contiguous()
    if x.dtype != torch.float64:
        raise TypeError("log_f64 takes float64")
    y = torch.empty_like(x)
    _check(load().fea_log_f64(_ptr(x), _ptr(y), x.numel(), _stream_ptr(stream)))
    return y


def scatter_add_csr_mapped(scatter_map, elem, values, stream=None):
    """values[map] += elem (device); fea_scatter_add_csr_mapped.  Returns `values`."""
    import torch
    E, n, _ = scatter_map.shape
    if scatter_map.dtype not in (torch.int32, torch.int64):
        raise TypeError("scatter map must be int32 or int64")
    _check(load().fea_scatter_add_csr_mapped(E, n, _ptr(scatter_map), int(scatter_map.dtype == torch.int64),
                                             _ptr(elem), int(elem.dtype == torch.float32),
                                             values.shape[0], _ptr(values), _stream_ptr(stream)))
    return values


def assemble_batch(requests, out_f32=False, stream=None, fused=False, precision=PREC_FP32):
    """requests: list of (form, degree, coords, coeffs, out) device tensors, one CUDA graph launch
    (fea_assemble_batch: one persistent kernel per request; fused=True: fea_assemble_batch_fused,
    one persistent kernel over a work list of all requests' tiles, FP32 only)."""
    arr = (Request * len(requests))()
    for k, (form, degree, coords, coeffs, out) in enumerate(requests):
        arr[k] = Request(form, degree, coords.shape[0], coords.data_ptr(),
                         None if coeffs is None else coeffs.data_ptr(), out.data_ptr())
    o = options(precision, out_f32)
    fn = load().fea_assemble_batch_fused if fused else load().fea_assemble_batch
    _check(fn(arr, len(requests), ctypes.byref(o), _stream_ptr(stream)))


def assemble_batch_noalloc(requests, out_f32=False, stream=None):
    """fea_assemble_batch_noalloc: the batched launch without device allocations
    (for callers that cannot allocate; see include/fea.h for its limits)."""
    arr = (Request * max(1, len(requests)))()
    for k, (form, degree, coords, coeffs, out) in enumerate(requests):
        arr[k] = Request(form, degree, coords.shape[0], coords.data_ptr(),
                         None if coeffs is None else coeffs.data_ptr(), out.data_ptr())
    o = options(PREC_FP32, out_f32)
    _check(load().fea_assemble_batch_noalloc(arr, len(requests), ctypes.byref(o), _stream_ptr(stream)))


def skip_input_copy_once(tile):
    """Fault injection for tests: the next standalone launch skips the input copy of global tile
    `tile` (-1 clears); its bounded wait runs out and the next sync raises FeaError(ETIMEOUT)."""
    _check(load().fea_test_skip_input_copy(tile))


def sync(stream=None):
    """Wait for the stream; raises FeaError(EDEGENERATE) after a degenerate element."""
    _check(load().fea_sync(_stream_ptr(stream)))


def plan(form, degree, precision=PREC_FP32, out_f32=False, variant=VARIANT_AUTO, tile=0, smem_budget=0):
    info = PlanInfo()
    o = options(precision, out_f32, variant, tile, smem_budget)
    _check(load().fea_plan(form, degree, ctypes.byref(o), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def plan_flop(form, degree, precision=PREC_FP32, out_f32=False, smem_budget=0):
    """The plan without tuned choices: Algorithm 3's variant and the default tile."""
    info = PlanInfo()
    o = options(precision, out_f32, VARIANT_AUTO, 0, smem_budget)
    _check(load().fea_plan_flop(form, degree, ctypes.byref(o), ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


def op_count(form, degree, variant=VARIANT_AUTO):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().fea_op_count(form, degree, variant, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def opcount_program(program, extents):
    """Operation count of a loop-nest program (see include/fea.h)."""
    ops = ctypes.c_int64()
    _check(load().fea_opcount_program(program.encode(), _ext(extents), ctypes.byref(ops)))
    return ops.value


def _ext(extents):
    if isinstance(extents, dict):
        extents = ",".join("%s:%d" % kv for kv in extents.items())
    return extents.encode()


def sharing_elimination(lhs, expr, loops, extents):
    """Algorithm 1 on `lhs += expr`: (program text, operation count, vertex-cover size)."""
    buf = ctypes.create_string_buffer(1 << 20)
    ops, cover = ctypes.c_int64(), ctypes.c_int()
    _check(load().fea_sharing_elimination(lhs.encode(), expr.encode(), ",".join(loops).encode(), _ext(extents),
                                          buf, len(buf), ctypes.byref(ops), ctypes.byref(cover)))
    return buf.value.decode(), ops.value, cover.value


def vertex_cover(nl, nr, edges):
    flat = (ctypes.c_int * (2 * len(edges)))(*[x for e in edges for x in e])
    k = ctypes.c_int()
    _check(load().fea_vertex_cover(nl, nr, flat, len(edges), ctypes.byref(k)))
    return k.value


def increase_factor(n, k):
    return load().fea_increase_factor(n, k)


def theta(form, degree):
    """[(theta_se, theta_pre, table_words)] per monomial of the form."""
    out = []
    for m in range(load().fea_num_monomials(form, degree)):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().fea_theta(form, degree, m, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        out.append((a.value, b.value, c.value))
    return out


def algorithm3(form, degree, precision=PREC_FP32, smem_budget=0):
    """(bitmask of pre-evaluated monomials, cost) chosen by Algorithm 3."""
    m, c = ctypes.c_uint(), ctypes.c_int64()
    _check(load().fea_algorithm3(form, degree, precision, smem_budget, ctypes.byref(m), ctypes.byref(c)))
    return m.value, c.value


def tune_set(form, degree, variant=VARIANT_AUTO, tile=0, precision=PREC_FP32):
    _check(load().fea_tune_set(form, degree, precision, variant, tile))


def tune_clear():
    load().fea_tune_clear()


def mlp_num_params(d_in, hidden):
    return load().fea_mlp_num_params(d_in, hidden)


def mlp_forward(params, X, hidden, out=None, stream=None):
    """Predictions of the MLP for rows X [n, d_in] (float32 device tensors)."""
    import torch
    n, d = X.shape
    y = out if out is not None else torch.empty(n, dtype=torch.float32, device=X.device)
    _check(load().fea_mlp_forward(_ptr(params), d, hidden, _ptr(X), n, _ptr(y), _stream_ptr(stream)))
    return y


def mlp_loss_grad(params, X, y, hidden, grad=None, loss=None, scratch=None, stream=None):
    """(loss [1], grad [nparam]) of the mean squared error, on the device."""
    import torch
    n, d = X.shape
    dev = X.device
    grad = grad if grad is not None else torch.empty_like(params)
    loss = loss if loss is not None else torch.empty(1, dtype=torch.float32, device=dev)
    if scratch is None:
        scratch = torch.empty(load().fea_mlp_scratch_floats(n, hidden), dtype=torch.float32, device=dev)
    _check(load().fea_mlp_loss_grad(_ptr(params), d, hidden, _ptr(X), _ptr(y), n, _ptr(grad), _ptr(loss),
                                    _ptr(scratch), _stream_ptr(stream)))
    return loss, grad


def mlp_adam(params, grad, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().fea_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), lr, beta1, beta2, eps,
                               step, _stream_ptr(stream)))


def finalize():
    if _lib is not None:
        _lib.fea_finalize()
