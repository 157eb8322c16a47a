/*
 * fea.h -- C ABI of the GB300 (sm_103a) batched element-local assembly library.
 *
 * For every tetrahedron e of a batch the library computes the local element
 * matrix  A_e[i][j] = sum_q w_q |det J_e| F(phi_i, phi_j, coefficients, J_e^-1)(X_q)
 * (Section 2.2, equation "quadrature"; the statement of local assembly is in
 * Section 2), in the flop-reduced forms that the paper's transformation
 * algorithm selects between: sharing elimination (Section 3.2, Algorithm 1)
 * and pre-evaluation of the quadrature reduction (Section 3.3, Algorithm 2),
 * coordinated by the cost function theta and Algorithm 3 (Section 4).
 *
 * Forms (Section 7 names them Mass, Helmholtz, Elasticity, Hyperelasticity):
 *   FEA_MASS        int u v
 *   FEA_HELMHOLTZ   int grad u . grad v + f u v,        f in P_p
 *   FEA_ELASTICITY  int 2 mu eps(u):eps(v) + lam div u div v,  mu, lam in P_1
 *   FEA_NEOHOOKEAN  tangent stiffness of W = mu/2 (tr C - 3) - mu ln J + lam/2 (ln J)^2
 * Degrees p = 1..4 (Lagrange, equispaced nodes) on tetrahedra.
 *
 * Data layout (all arrays are C-contiguous, little-endian IEEE):
 *   coords  double [E][4][3]  vertex coordinates; J[r][c] = x_{c+1}[r] - x_0[r].
 *   coeffs  double, per element (fea_coeff_len doubles each):
 *             mass: none (may be NULL);  helmholtz: f DOFs [n_p];
 *             elasticity: mu DOFs [4] then lambda DOFs [4] (P_1 vertex values);
 *             neohookean: displacement DOFs [n_p][3] (component fastest), and
 *             after the last element two doubles: the constants mu, lambda.
 *           fea_coeffs_size() gives the total length.
 *   out     [E][n][n] row-major, n = fea_local_dim(); test index = row, trial
 *           index = column; vector forms use DOF index 3*a + c.  double by
 *           default, float when fea_options.out_f32 = 1.
 *   DOF order of P_p: vertices 0..3; edges (2,3),(1,3),(1,2),(0,3),(0,2),(0,1)
 *           with nodes running from the lower to the higher vertex; faces
 *           opposite vertices 0..3; interior.  Inside a face or the interior,
 *           nodes are ordered by barycentric index with the entity's last
 *           vertex varying slowest.
 *
 * Ownership: the caller owns coords, coeffs and out.  In fea_assemble /
 * fea_assemble_ex / fea_assemble_batch they are DEVICE pointers of the current
 * CUDA device (16-byte aligned); host pointers are rejected with FEA_EINVAL --
 * there is no CPU fallback.  fea_assemble_host takes HOST pointers and does the
 * copies itself.  The library owns only its plan cache, its device-resident
 * basis/reference tables and a reusable staging workspace; fea_finalize frees
 * them.
 *
 * Errors: every call returns an fea_status and never aborts.  Device calls are
 * asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy
 * default stream).  A degenerate element (det J == 0, or det F <= 0 for the
 * Neo-Hookean form) writes NaN into that element's matrix and sets a device
 * error word; fea_sync() returns FEA_EDEGENERATE once for it.
 * fea_last_error() returns a message for the last failing call of this thread.
 */
#ifndef FEA_H
#define FEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FEA_MASS = 0, FEA_HELMHOLTZ = 1, FEA_ELASTICITY = 2, FEA_NEOHOOKEAN = 3 } fea_form;

typedef enum {
  FEA_OK = 0,
  FEA_EINVAL = 1,       /* bad argument (form, degree, size, pointer kind, alignment, option) */
  FEA_ENOMEM = 2,       /* table or workspace allocation failed */
  FEA_ECUDA = 3,        /* a CUDA runtime call failed (message in fea_last_error) */
  FEA_EDEGENERATE = 4,  /* a degenerate element was met (NaN written for it) */
  FEA_ETIMEOUT = 5      /* a bounded wait in the batch work queue gave up */
} fea_status;

/* Arithmetic of the contraction.  Geometry (J, det J and the adjugate of J,
 * i.e. det J * J^-1) and the Neo-Hookean det F, F^-1, ln det F are FP64 in
 * every mode. */
typedef enum {
  FEA_PREC_FP64 = 0,   /* everything FP64 (parity path, <= 1e-12 relative) */
  FEA_PREC_FP32 = 1,   /* FP32 contraction and pointwise work, FP64 geometry */
  FEA_PREC_BF16X2 = 2  /* split-BF16 tensor-core contraction where the contraction is dense and
                        * compute-bound (the Neo-Hookean tangent at P2): both operands as
                        * hi + lo BF16 pairs, all four products on tcgen05 tensor cores with
                        * FP32 accumulation (<= 1e-5 relative); the per-point kinematics as
                        * in FEA_PREC_FP32.  With FP32 output (out_f32 = 1) the
                        * pre-evaluated mass and Helmholtz matrices at P1-P2 also run on the
                        * tensor cores (one [128 elements x r] x [r x n^2] product per tile,
                        * both operands split the same way), since without the FP64 stores
                        * their contraction, not HBM, bounds them.  Every other (form,
                        * degree, output) runs the FP32 contraction in this mode (bound by
                        * HBM, not by the contraction).  fea_assemble_batch accepts it; the
                        * fused batch does not. */
} fea_precision;

/* Loop-nest variant (Section 4, Figure "loopnest-opt"). */
typedef enum {
  FEA_VARIANT_AUTO = -1, /* Algorithm 3 choice, refined by the tuner when enabled */
  FEA_VARIANT_NAIVE = 0, /* plain quadrature nest in normal form, FP64 (the comparator) */
  FEA_VARIANT_SE = 1,    /* quadrature nest after sharing elimination (Algorithm 1) */
  FEA_VARIANT_PRE = 2    /* pre-evaluated reference tensors (Algorithm 2) */
} fea_variant;

typedef struct {
  int precision;       /* fea_precision (default FEA_PREC_FP32) */
  int out_f32;         /* 0: out is double, 1: out is float */
  int variant;         /* fea_variant (default FEA_VARIANT_AUTO) */
  int tile;            /* elements per CTA tile, 0 = planner default */
  size_t smem_budget;  /* T_H of Constraint 2 in bytes of shared memory, 0 = device limit */
} fea_options;

/* One request of a batch (fea_assemble_batch): device pointers as above. */
typedef struct {
  int form;
  int degree;
  int64_t E;
  const double* coords;
  const double* coeffs;
  void* out;
} fea_request;

/* Plan summary (fea_plan). */
typedef struct {
  int variant;          /* variant that will run */
  int tile;             /* elements per CTA tile */
  int threads;          /* threads per CTA */
  int quad_points;      /* Q of the rule */
  int ref_terms;        /* r: reference tensors (pre-evaluation) */
  size_t smem_bytes;    /* dynamic shared memory per CTA */
  int64_t flops_naive;  /* per element, plain quadrature nest (normal form) */
  int64_t flops_se;     /* per element, after sharing elimination */
  int64_t flops_pre;    /* per element, after pre-evaluation (-1: not applicable) */
  int64_t flops_run;    /* per element, variant that will run */
  int64_t bytes;        /* per element, algorithmic HBM bytes (inputs + output) */
} fea_plan_info;

/* Sizes.  Return -1 for an unsupported (form, degree). */
int fea_local_dim(int form, int degree);                /* n: n_p or 3 n_p */
int fea_coeff_len(int form, int degree);                /* doubles per element */
int64_t fea_coeffs_size(int form, int degree, int64_t E); /* total doubles in coeffs */
int fea_quad_points(int form, int degree);              /* Q of the rule used */

/* Assemble E element matrices on `stream` (device pointers).  fea_assemble
 * uses default options (FP32 contraction, double output, variant AUTO). */
int fea_assemble(int form, int degree, int64_t E, const double* coords,
                 const double* coeffs, void* out, void* stream);
int fea_assemble_ex(int form, int degree, int64_t E, const double* coords,
                    const double* coeffs, void* out, const fea_options* opt, void* stream);

/* Same, with HOST buffers: copies coords/coeffs to the device, assembles and
 * copies the result back, then synchronises `stream`.  Pinned host memory
 * gives the full copy bandwidth; work is pipelined over chunks. */
int fea_assemble_host(int form, int degree, int64_t E, const double* coords_host,
                      const double* coeffs_host, void* out_host, const fea_options* opt,
                      void* stream);

/* Element VECTORS of the linear forms (arity 1, Section 2), E of them, on
 * `stream` (device pointers, 16-byte aligned):
 *   FEA_HELMHOLTZ:   the load vector b_i = int f phi_i, f in P_degree given by
 *                    its DOFs; coeffs as for the Helmholtz matrix ([E][n_p]);
 *                    out [E][n_p].
 *   FEA_NEOHOOKEAN:  the residual R_(a,c) = int P(F)_{cx} dphi_a/dx_x with
 *                    P = mu (F - F^-T) + lam ln det F F^-T; coeffs as for the
 *                    tangent ([E][n_p][3] displacements, then mu, lam);
 *                    out [E][3 n_p], index 3 a + c.
 * Other forms return FEA_EINVAL.  opt: precision (FP32 contraction with FP64
 * geometry and FP64 det F / ln det F, or FP64), out_f32, tile (0 = default),
 * smem_budget; variant must be AUTO.  Degenerate elements give NaN entries
 * and FEA_EDEGENERATE at the next fea_sync. */
int fea_assemble_vector(int form, int degree, int64_t E, const double* coords,
                        const double* coeffs, void* out, const fea_options* opt, void* stream);

/* Helmholtz element matrices in the Bernstein-Bezier basis, computed by sum
 * factorisation over the collapsed quadrature rule (the paper names sum
 * factorisation as future work, Section 8 "Limitations and future work"; the
 * weak form is that of Section 2, the pre-evaluated stiffness that of
 * Section 3.3).  The same finite element space as FEA_HELMHOLTZ at `degree`
 * (1..4), in another basis:
 *   B_a = p!/a! l^a over the multi-indices a = (a0, a1, a2, a3), |a| = p, of the
 *   barycentric coordinates l0 = 1 - X0 - X1 - X2, l_{k+1} = X_k; DOF order a3
 *   slowest, then a2, then a1 (a0 = p - a1 - a2 - a3).
 * coeffs [E][n_p] (DEVICE, doubles): the Bernstein coefficients of f,
 * f = sum_k c_k B_k; coords as for fea_assemble; out [E][n_p][n_p] (row = test,
 * column = trial), double, or float with out_f32 = 1.  FP64 geometry, FP32
 * arithmetic after it (<= 1e-5 relative Frobenius error).  The variable-
 * coefficient term int f B_a B_b = C(a+b, a) / C(2p, p) int f B^2p_(a+b) takes
 * the moments of f in six one-dimensional passes (O(p^4) per element instead
 * of n_p^3).  Asynchronous on `stream`; FEA_EINVAL for another form or
 * degree, a negative E or host pointers; degenerate elements give NaN and
 * FEA_EDEGENERATE at the next fea_sync.  The library keeps one table per
 * degree, freed by fea_finalize. */
int fea_assemble_bernstein(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                           void* out, int out_f32, void* stream);

/* The natural logarithm the Neo-Hookean kernels evaluate ln det F with (FP64
 * arithmetic, table-driven: Tang, ACM TOMS 16(4), 1990; 13 FP64 operations),
 * applied to n doubles: y[i] = ln x[i] (DEVICE arrays, on `stream`).  A few
 * units in the last place for finite x > 0; unspecified for other x.  Exposed
 * so that its accuracy can be checked against other implementations. */
int fea_log_f64(const double* x, double* y, int64_t n, void* stream);

/* Global assembly (the sum over elements of the element matrices at their
 * global degrees of freedom).
 *
 * fea_csr_pattern (HOST arrays): the CSR sparsity pattern of a mesh whose
 * element e has global DOFs dofs[e][0..n) (int32, row-major [E][n]; vector
 * forms number DOF 3 a + c of a node a as the caller's global map says), with
 * sorted unique columns per row; upper = 1 keeps only columns >= row (the
 * symmetric storage of a symmetric matrix), upper = 0 all.  Two calls: first
 * with col_idx = NULL to get *nnz (row_ptr may be NULL too), then with row_ptr
 * [nrows + 1] and col_idx [*nnz] to fill them.  FEA_EINVAL for a DOF outside
 * [0, nrows), upper not 0 or 1, or a col_idx smaller than *nnz.
 *
 * fea_scatter_add_csr (DEVICE arrays, on `stream`; full patterns): values[k]
 * += elem[e][i][j] for k the position of column dofs[e][j] in row dofs[e][i];
 * elem is [E][n][n] double (elem_f32 = 0) or float (1), as fea_assemble writes
 * it; values is [nnz] double and is accumulated into (zero it first for a
 * fresh matrix).  FP64 atomics: the sum order, and so the last bits, vary
 * between runs.  A DOF, row segment or column outside the pattern is skipped
 * and makes the next fea_sync return FEA_EINVAL. */
int fea_csr_pattern(int64_t E, int n, const int32_t* dofs, int64_t nrows, int upper, int64_t* row_ptr,
                    int32_t* col_idx, int64_t* nnz);
int fea_scatter_add_csr(int64_t E, int n, const int32_t* dofs, const void* elem, int elem_f32,
                        int64_t nrows, const int64_t* row_ptr, const int32_t* col_idx, int64_t nnz,
                        double* values, void* stream);

/* The same scatter split in two for repeated assembly on one mesh:
 * fea_csr_scatter_map writes once, for every (e, i, j), the CSR position of
 * column dofs[e][j] in row dofs[e][i] into map [E][n][n] (device; int32 when
 * map_i64 = 0, which needs nnz < 2^31, else FEA_EINVAL; int64 when map_i64 = 1;
 * -1 and FEA_EINVAL at the next fea_sync where the pattern has no entry; with
 * upper = 1, for a pattern built with upper = 1, -2 for the entries below the
 * diagonal, which are not stored and raise no error);
 * fea_scatter_add_csr_mapped then does values[map[e][i][j]] += elem[e][i][j]
 * with coalesced reads and no search (map_i64 as the map was written; -2
 * entries are passed over; any other position outside [0, nnz) is skipped and
 * flagged like a missing entry). */
int fea_csr_scatter_map(int64_t E, int n, const int32_t* dofs, int64_t nrows, const int64_t* row_ptr,
                        const int32_t* col_idx, int64_t nnz, int upper, void* map, int map_i64, void* stream);
int fea_scatter_add_csr_mapped(int64_t E, int n, const void* map, int map_i64, const void* elem, int elem_f32,
                               int64_t nnz, double* values, void* stream);

/* Local and global assembly in one pass: for mass and Helmholtz P1-P3 the
 * streaming pre-evaluated kernel adds every element matrix entry into the CSR
 * values at its position instead of storing the matrix: values[map[e][i][j]]
 * += A_e[i][j] (DEVICE arrays, on `stream`; coords and coeffs as for
 * fea_assemble; map [E][n][n] from fea_csr_scatter_map, int32 when map_i64 = 0
 * (nnz < 2^31) or int64; values [nnz] double, accumulated into; a map of an
 * upper-triangle pattern assembles the symmetric storage).  FP32
 * contraction, FP64 atomics (the last bits of the sums vary between runs).
 * FEA_EINVAL for other forms and degrees (use fea_assemble, then
 * fea_scatter_add_csr_mapped); a position outside [0, nnz) is skipped and
 * makes the next fea_sync return FEA_EINVAL; a degenerate element adds NaN and
 * makes it return FEA_EDEGENERATE. */
int fea_assemble_csr(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                     const void* map, int map_i64, int64_t nnz, double* values, void* stream);

/* Combining plan of the one-pass global assembly (HOST arrays, no GPU needed),
 * computed once per mesh from the position map of fea_csr_scatter_map (copied
 * to the host; [E][n][n], int32 when map_i64 = 0, else int64): for every tile of
 * T = min(128, 3200 / n^2 rounded down to even) consecutive elements, the
 * distinct CSR positions the tile's entries fall on and, per position, which of
 * the tile's entries add to it (Section 2: the global matrix is the sum of the
 * element matrices at their global DOFs; entries of one tile meeting at one
 * position are summed before they reach the global values).  Layout (32-bit
 * words, documented in csrc/pre_combine.cuh): a header (magic, n, T), int64
 * offsets of the tile records, then per tile the number of distinct positions,
 * the positions ordered by how many entries meet there (largest first) and the
 * 16-bit tile-local entry indices round by round.  Map entries -2 (lower
 * triangle under symmetric storage) are left out.  Call with plan = NULL to get
 * the size in *plan_words, then with a buffer of that many words; the call
 * writes the size used into *plan_words.  FEA_EINVAL: a position outside
 * [0, nnz) other than -2, nnz >= 2^31, n^2 T > 65536, or a buffer smaller than
 * needed. */
int fea_csr_combine_plan(int64_t E, int n, const void* map, int map_i64, int64_t nnz, int32_t* plan,
                         int64_t* plan_words);

/* fea_assemble_csr with the plan above (DEVICE copy, 16-byte aligned,
 * plan_words 32-bit words) in place of the map: the element entries of a tile
 * are staged in shared memory, every distinct position of the tile is summed
 * from them in FP64 (each FP32 entry widened exactly) and added to values [nnz]
 * with one FP64 atomic.  The result equals the two-pass assembly's up to the
 * order of the FP64 additions.  Mass and Helmholtz P1-P3 (FEA_EINVAL for
 * others, or a plan too short for E elements or not 16-byte aligned).  A plan
 * that is not for this local dimension and tile size, or breaks a bound of its
 * layout, is flagged: the next fea_sync returns FEA_EINVAL and the offending
 * tiles or positions are skipped; a degenerate element adds NaN and makes it
 * return FEA_EDEGENERATE. */
int fea_assemble_csr_combined(int form, int degree, int64_t E, const double* coords, const double* coeffs,
                              const int32_t* plan, int64_t plan_words, int64_t nnz, double* values, void* stream);

/* Uneven batch of requests (forms, degrees and sizes mixed) in one CUDA graph
 * launch, captured once per distinct batch and replayed: each request runs the
 * persistent kernel it would run alone (its own tile, registers and shared
 * memory), the requests spread over concurrent graph branches, largest first.
 * All requests use the same options (FP32 contraction). */
int fea_assemble_batch(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);

/* The same batch as ONE persistent kernel launch (also graph-captured): the
 * tiles of all requests form a work list that CTAs pull with an atomic
 * counter, dispatching on (variant, form, degree) to the FP32 tile functions;
 * one register and shared-memory budget serves every request.  Same results
 * as fea_assemble_batch. */
int fea_assemble_batch_fused(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);

/* The batched launch above, for callers that cannot allocate device memory at
 * the moment they assemble: code that lives inside another framework's memory
 * pool and may not allocate outside it, or a latency-critical loop where an
 * allocation may block, fail or cost more than the assembly itself.  The
 * paper has no counterpart.  The work-list counter and the request list live in
 * a file-scope device array of the library (256 B + 512 request slots, about
 * 37 KB, held by every GPU that loads the library until exit) instead of
 * allocations; the request list reaches it as kernel parameters of a small
 * copy kernel, and the batched kernel is launched directly on `stream`.  The
 * call allocates nothing, on the device or on the host.  Limits: at most 512
 * requests per call (FEA_EINVAL beyond); FP32 contraction only; the library's
 * state and the tables of each requested (form, degree) must already exist on
 * the current device -- any earlier allocating call there makes them -- else
 * FEA_EINVAL.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All
 * calls share the array and each restarts its counter at zero, so calls whose
 * kernels overlap on the GPU race: keep them ordered (one stream). */
int fea_assemble_batch_noalloc(const fea_request* reqs, int nreq, const fea_options* opt, void* stream);

/* Wait for `stream`, then report (and clear) the device error word. */
int fea_sync(void* stream);

/* Fault injection for tests of the failure path (the paper has no
 * counterpart): the next standalone launch skips the input copy of its global
 * tile `tile` (-1 clears; other values below -1 give FEA_EINVAL).  The kernels
 * that stream their inputs by bulk copies (mass and Helmholtz P1-P3 FP32, the
 * one-pass global assembly, the split-BF16 Neo-Hookean kernel) honour it: the
 * CTA that runs that tile waits for inputs that never arrive, its bounded wait
 * gives up (after a few seconds), the CTA leaves after its copies in flight have
 * landed, the outputs of that tile and of that CTA's later tiles are left
 * unwritten, and the next fea_sync returns FEA_ETIMEOUT.  Other kernels ignore
 * it.  The setting applies to one launch and then clears itself. */
int fea_test_skip_input_copy(int64_t tile);

/* Plan for (form, degree, options) without launching anything. */
int fea_plan(int form, int degree, const fea_options* opt, fea_plan_info* info);

/* The same plan ignoring tuned choices: the paper's choice by operation count
 * (Algorithm 3's variant and the shared-memory tile rule). */
int fea_plan_flop(int form, int degree, const fea_options* opt, fea_plan_info* info);

/* Operation counts per element (Definition 8 counting: adds and products, an
 * FMA counts 2) of the plain nest and of `variant` (AUTO = Algorithm 3 pick). */
int fea_op_count(int form, int degree, int variant, int64_t* naive_flops, int64_t* opt_flops);

/* ---- the planner's operation-count algorithm (host only, no GPU needed) ----
 * Expression language: program := stmt (';' stmt)*, stmt := loops ':' lhs
 * ('=' | '+=') expr, loops := index (',' index)*, expr over + - * and
 * parentheses, symbols name[i,j,...].  Extents: "e:1,i:64,j:10,k:10". */

/* Operation count of a loop-nest program (Definition 8 with the convention of
 * Figure "poisson": adds and products, '+=' counts one, a sub-expression that
 * occurs more than once in one loop body is counted once). */
int fea_opcount_program(const char* program, const char* extents, int64_t* ops);

/* Algorithm 1 (sharing elimination, Section 3.2) on `lhs += expr` inside the
 * loops (comma separated, outermost first; the last two are the linear
 * test/trial loops).  Writes the transformed program (same language) into
 * `program` (capacity `cap` bytes, may be NULL), its operation count and the
 * size of the minimum vertex cover of the sharing graph (step 5's ILP). */
int fea_sharing_elimination(const char* lhs, const char* expr, const char* loops, const char* extents,
                            char* program, size_t cap, int64_t* ops, int* cover);

/* Minimum vertex cover of a bipartite graph (the ILP of Algorithm 1, step 5):
 * left vertices 0..nl-1, right 0..nr-1, edges[2k], edges[2k+1]. */
int fea_vertex_cover(int nl, int nr, const int* edges, int nedges, int* cover_size);

/* Increase factor iota = C(n + k - 1, k) of pre-evaluation (Section 4.2);
 * -1 for n < 1 or k < 0. */
int64_t fea_increase_factor(int n, int k);

/* Monomials of a form (Section 2.1) and their costs per element: theta_se
 * (Algorithm 1), theta_pre (rho * iota tables, Section 4.2; -1 when the
 * integrand is not polynomial) and the pre-evaluated table size in words. */
int fea_num_monomials(int form, int degree);
int fea_theta(int form, int degree, int monomial, int64_t* theta_se, int64_t* theta_pre, int64_t* table_words);

/* Algorithm 3 (Section 4.1): bitmask of the monomials to pre-evaluate under
 * the memory threshold T_H = smem_budget bytes (0 = 227 KB), and its cost. */
int fea_algorithm3(int form, int degree, int precision, size_t smem_budget, unsigned* premask, int64_t* cost);

/* ---- tuning and the learned cost model (the paper has no counterpart; it asks
 * for "a more sophisticated cost model" in Section 8) ----
 * Install / clear a tuned (variant, tile) for (form, degree, precision): used by
 * FEA_VARIANT_AUTO and tile 0 in every later call (tile 0 keeps the default
 * tile; variant FEA_VARIANT_AUTO keeps Algorithm 3's variant). */
int fea_tune_set(int form, int degree, int precision, int variant, int tile);
void fea_tune_clear(void);

/* MLP cost model y = w3 . tanh(W2 tanh(W1 x + b1) + b2) + b3 with d_in <= 32
 * inputs and hidden in {16, 32, 64}; parameters (float, device) laid out as
 * W1[hidden][d_in] b1 W2[hidden][hidden] b2 w3 b3.  All pointers are device
 * pointers; calls are asynchronous on `stream`. */
int fea_mlp_num_params(int d_in, int hidden);                 /* -1 if unsupported */
int64_t fea_mlp_scratch_floats(int n, int hidden);            /* workspace of fea_mlp_loss_grad */
int fea_mlp_forward(const float* params, int d_in, int hidden, const float* X, int n, float* y, void* stream);
/* Mean squared error over n rows and its gradient (deterministic, no atomics);
 * `scratch` holds fea_mlp_scratch_floats(n, hidden) floats. */
int fea_mlp_loss_grad(const float* params, int d_in, int hidden, const float* X, const float* y, int n,
                      float* grad, float* loss, float* scratch, void* stream);
/* One Adam step (bias-corrected; step counts from 1). */
int fea_mlp_adam(float* params, const float* grad, float* m, float* v, int nparam, float lr, float beta1,
                 float beta2, float eps, int step, void* stream);

const char* fea_last_error(void);
void fea_finalize(void);

#ifdef __cplusplus
}
#endif
#endif /* FEA_H */
