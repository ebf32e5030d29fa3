/*
 * bta.h -- C ABI of the GB300 library for the INLA hyperparameter objective
 * f(theta) and its exact reverse-mode gradient on block-tridiagonal-
 * arrowhead (BTA) precision matrices (ADELIA, Sections II-III).
 *
 * All pointers are plain host or device pointers as stated per argument;
 * no C++ or framework types cross this boundary.  Device pointers must be
 * allocated on the current CUDA device.  Every call is stream-ordered on the
 * given stream; only inla_value_and_grad() synchronises (it returns host
 * scalars).  No call traps: failures come back as a status code.
 *
 * Latent ordering: x = [x_1 .. x_n, beta]; x_t is one time step of b values
 * (k variables stacked, each over ns grid nodes, node s = iy*nx + ix).
 */
#ifndef BTA_H
#define BTA_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BTA_OK = 0,
  BTA_ERR_ARG = -1,      /* bad argument, NaN/Inf theta, size out of range  */
  BTA_ERR_NOT_SPD = -2,  /* a pivot was not positive; see fail_block         */
  BTA_ERR_CUDA = -3,     /* a CUDA runtime call failed                       */
  BTA_ERR_NOMEM = -4,    /* device allocation failed                         */
  BTA_ERR_TIMEOUT = -5,  /* a bounded device wait gave up                    */
  BTA_ERR_STATE = -6     /* descriptor is not in the state the call needs    */
} bta_status;

/* Descriptor states, checked by every call that takes a descriptor. */
enum { BTA_STATE_EMPTY = 0, BTA_STATE_ASSEMBLED = 1, BTA_STATE_FACTORED = 2,
       BTA_STATE_SELINV = 3 };

/*
 * BTA matrix (Section II-B): n diagonal blocks D_i, n-1 sub-diagonal blocks
 * B_i = Q[i+1, i], n arrow blocks C_i = Q[T, i] (a x b) and the tip T (a x a).
 * Layout (all device memory, caller-owned, column-major FP64):
 *   D: n blocks of ld x ld, block i at D + i*ld*ld; lower triangle referenced.
 *   B: n-1 blocks of ld x ld, block i at B + i*ld*ld.
 *   C: n blocks of a x ld (leading dimension a), block i at C + i*a*ld.
 *   T: a x a (leading dimension a).  a may be 0 (block-tridiagonal), then C, T
 *      may be NULL.
 * ld is b rounded up to a multiple of 32.  Rows/columns b..ld-1 are padding:
 * D holds the identity there and B, C hold zeros (bta_assemble writes this).
 * The padding adds log 1 = 0 to log-determinants and leaves every result on
 * the first b rows/columns exact.
 *
 * After bta_factor the same memory holds the factor (Algorithm 1):
 *   D_i <- L_Di^{-1} (lower triangle; the inverse of the diagonal Cholesky
 *          factor, which is what the solves and the selected inversion use),
 *   B_i <- L_Bi = B_i L_Di^{-T},  C_i <- L_Ci,  T <- L_T (lower).
 * After bta_selinv it holds the selected inverse Z = Q^{-1} on the BTA pattern:
 *   D_i <- Z_Di (full symmetric), B_i <- Z_Bi, C_i <- Z_Ci, T <- Z_T (full).
 */
typedef struct {
  int32_t n, b, a, ld;
  double *D, *B, *C, *T;
  int32_t state;
} bta_desc;

/*
 * Model description (Section II-A, Eq. 1; Section III-B, Eq. 10), host arrays,
 * copied by inla_model_create.  The prior precision of variable m is the
 * Kronecker form  M0 (x) K0 + 2 kappa gamma M1 (x) K1 + M2 (x) Cm,
 * K0 = kappa^4 Cm + 2 kappa^2 G + GG, K1 = kappa^2 Cm + G, scaled by e^{theta_1}
 * (k == 1) or combined through the coregionalisation weights
 * W_pq^(m) = (Lambda^{-1})_{mp} (Lambda^{-1})_{mq} (k > 1).
 *   Spatial matrices: one CSR pattern over ns nodes (row_ptr[ns+1], col[nnz],
 *   sorted columns, symmetric pattern) with the values of Cm, G and GG on it.
 *   Temporal matrices Mj (nt x nt, tridiagonal): m_diag[j*nt + t] = Mj[t,t],
 *   m_sub[j*(nt-1) + t] = Mj[t+1,t].
 *   Observations: row r touches latent (obs_t[r], obs_v[r], obs_s[r]) with
 *   weight 1 and fixed effects obs_v[r]*a_r .. +a_r-1 with obs_cov[r*a_r + c];
 *   a_r = a / k.
 */
typedef struct {
  int32_t k, ns, nt, a;
  int32_t nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val_C;
  const double* val_G;
  const double* val_GG;
  const double* m_diag;      /* 3 * nt     */
  const double* m_sub;       /* 3 * (nt-1) */
  int64_t n_obs;
  const int32_t* obs_t;
  const int32_t* obs_s;
  const int32_t* obs_v;
  const double* obs_cov;     /* n_obs * (a/k) */
  const double* y;           /* n_obs */
  double tip_prior;          /* prior precision of each fixed effect (1e-3) */
  double theta_prior_var;    /* log p(theta) = -sum theta^2 / (2 var)  (100) */
  int32_t low_memory;        /* 1: the model's evaluations keep only the diagonal
                                factors L_Di^{-1} (and the arrow) between the
                                forward and the reverse pass; every step that
                                needs an off-diagonal factor re-assembles B_i
                                and recomputes L_Bi = B_i L_Di^{-T} (the
                                carry-based variant of Algorithm 1, Section
                                III-A): about half the device memory, one more
                                b x b product per block.  Precision 1 (mixed)
                                is refused (BTA_ERR_ARG) on such a model.  0:
                                both factors kept whole.                       */
} inla_model_spec;

typedef struct inla_model inla_model;

/* Options for inla_value_and_grad. */
typedef struct {
  int32_t precision;   /* 0: FP64 everywhere.  1: mixed -- the b x b
                          off-diagonal Schur products of both factorisations
                          and the selected-inversion products in split TF32
                          on the tensor cores (FP32 accumulation); diagonal
                          block factorisation to FP64 accuracy (FP64 pivots;
                          blocks above 512 rows split 2 x 2, their inner
                          products and the 32 x 32 tile products of the
                          leaves emulated as in mode 2), log-determinants,
                          arrow and tip in FP64; one FP64 refinement step on
                          x*.
                          2: emulated FP64 -- the same b x b products as in
                          mode 1, with the arrow's rows and rank-a terms
                          carried along, and the diagonal factor's inner and
                          tile products, computed to FP64 accuracy on the
                          BF16 tensor cores (8 slices, as bta_gemm_emulated;
                          products with K > 5120 fall back to FP64);
                          everything else as in mode 0                        */
  int32_t use_graph;   /* 1: capture the evaluation in a CUDA graph, replay */
  int32_t streams;     /* thetas evaluated together for batch > 1 (1..16): their
                          matrices are swept in the same batched launches;
                          each needs its own device buffers                 */
  int32_t reserved;
} inla_opts;

/* Create / destroy a model.  Uploads the theta-independent pieces (counts of
 * observations per latent node, covariate sums, A^T y, covariate Gram
 * blocks) and allocates the library-owned workspaces. */
bta_status inla_model_create(const inla_model_spec* spec, inla_model** out);
void inla_model_destroy(inla_model* m);

/* Number of hyperparameters d = 4k + k(k-1)/2, block size b, padded ld, N. */
bta_status inla_model_dims(const inla_model* m, int32_t* d, int32_t* b, int32_t* ld,
                           int32_t* n, int32_t* a);

/*
 * bta_assemble -- Section II-A computational structure / Eq. 10: write the
 * dense BTA blocks of Q_p(theta) (which = 0, block-tridiagonal, a of the
 * descriptor must be 0) or Q_c(theta) = Q_p + sum_m tau_m A_m^T A_m
 * (which = 1, arrowhead a = model a) into out (device memory, caller-owned,
 * sized as documented for bta_desc with the model's n, b, ld).  theta is a
 * host array of d values.  rhs (device, n*ld + a, may be NULL) receives
 * r = sum_m tau_m A_m^T y_m (zero on padding) when which = 1.
 * Errors: BTA_ERR_ARG (NaN/Inf theta, shape mismatch).  Sets state ASSEMBLED.
 */
bta_status bta_assemble(inla_model* m, const double* theta, int32_t which,
                        bta_desc* out, double* rhs, cudaStream_t stream);

/*
 * bta_factor -- Algorithm 1 (Section III-A): block Cholesky of an ASSEMBLED
 * BTA matrix, in place, fused with the lower solve L z = r when rhs_inout !=
 * NULL (device, n*ld + a; overwritten by z).  logdet (device scalar)
 * receives log|Q| = 2 sum log diag(L).  fail_block (device int32) receives
 *   -1               the factor is complete,
 *   i >= 0           the index of the first diagonal block (n for the tip)
 *                    whose pivot was not positive,
 *   BTA_ERR_TIMEOUT  (-5) a bounded device wait of the factor expired;
 * in both failure cases the factor is not usable.  The call does not
 * synchronise, so it cannot itself return BTA_ERR_NOT_SPD or
 * BTA_ERR_TIMEOUT: read fail_block.
 * precision: as inla_opts.precision.  0: FP64.  1: mixed -- the b x b
 * Schur-complement products (D_i -= L_B L_B^T, L_B = B L_D^{-T}) in split TF32
 * on the tensor cores, the diagonal factors (FP64 pivots, emulated-FP64 inner
 * products), log-determinant, arrow and tip in FP64 (relative error ~1e-9 in
 * log|Q|, ~1e-6 in the factor; refine the solve with bta_solve(refine = 1)).
 * 2: emulated FP64 -- the same products, the arrow's carried along, to FP64
 * accuracy on the BF16 tensor cores.  Modes 1 and 2 allocate their
 * operand copies with cudaMallocAsync on the stream, as the workspace of
 * every mode.  Sets state FACTORED.
 */
bta_status bta_factor(bta_desc* q, double* rhs_inout, double* logdet, int32_t* fail_block,
                      int32_t precision, cudaStream_t stream);

/*
 * bta_factor_noalloc -- the same factorisation as bta_factor (same arguments,
 * same results, precision fixed to FP64), for callers that cannot allocate
 * device memory during the call: a process that has handed the device to its
 * own allocator or a fixed memory budget, a framework that forbids allocation
 * on its hot path, or code that cannot take the device-wide synchronisation a
 * free may imply.  The paper has no counterpart; this is a library-level
 * variant.  Its temporary blocks come from a fixed array in the library's
 * device memory (2.4 MB per device, held until the process exits), so:
 *   - sizes are limited to ld <= 256, a <= 32 and n * (ld / 32) + 1 <= 16384;
 *     beyond that it returns BTA_ERR_ARG without doing any work;
 *   - all calls on a device share the array: calls that overlap on the GPU
 *     race and give wrong results, so order them on one stream;
 *   - under CUDA's lazy module loading the array is reserved on a device by
 *     the first call there (which loads the library's device code for it, and
 *     may allocate and synchronise): make one call at set-up time, before any
 *     stream capture.  Every call looks the array's address up again, so a
 *     device reset leaves no stale address.
 * Apart from that first reservation it calls no cudaMalloc, cudaFree or
 * allocating library routine.
 */
bta_status bta_factor_noalloc(bta_desc* q, double* rhs_inout, double* logdet,
                              int32_t* fail_block, cudaStream_t stream);

/*
 * bta_solve -- Eqs. 3-5: given a FACTORED descriptor and z (device, from the
 * fused lower solve), overwrite z by x = Q^{-1} r.  With lower = 1 the lower
 * solve L z = r is done first (so z_inout may hold r).
 * refine = 1 adds one step of iterative refinement in FP64, x += L^{-T} L^{-1}
 * (r - Q x), the step the mixed-precision mode applies to x*: it needs
 * lower = 1 (z_inout holds r on entry) and Q_or_null, a separate ASSEMBLED
 * descriptor of the same matrix (same n, b, a, ld; D and T lower triangles
 * referenced), which is read, not changed.  refine = 0 ignores Q_or_null.
 * Errors: BTA_ERR_ARG (refine without lower or Q, shape mismatch),
 * BTA_ERR_STATE (L not FACTORED, Q not ASSEMBLED).  Allocates its workspace
 * with cudaMallocAsync on the stream.
 */
bta_status bta_solve(const bta_desc* L, double* z_inout, int32_t lower, int32_t refine,
                     const bta_desc* Q_or_null, cudaStream_t stream);

/*
 * bta_selinv -- selected inversion of a FACTORED descriptor in place
 * (Section III-A, Phase A), Z = Q^{-1} on the BTA pattern.  When m and
 * trace_terms (device, d doubles) are given, the traces of Eq. 7 against the
 * model's block Jacobians at theta (host, d) are fused into the sweep:
 * trace_terms[k] = tr(Q^{-1} dQ/dtheta_k) for the matrix given by which
 * (0 = Q_p, 1 = Q_c).  Sets state SELINV.
 */
bta_status bta_selinv(bta_desc* L, inla_model* m, const double* theta, int32_t which,
                      double* trace_terms, cudaStream_t stream);

/*
 * inla_value_and_grad -- Eq. 1 and Eq. 6.  theta: host, batch x d.  f: host,
 * batch values.  grad: host, batch x d, or NULL for the value-only path
 * (the finite-difference baseline's evaluation).  opts may be NULL.
 * Synchronises stream.  Returns BTA_ERR_NOT_SPD if a factor met a
 * non-positive pivot and BTA_ERR_TIMEOUT if a bounded device wait expired
 * (f and grad are then not usable; the model stays usable).
 * log l omits the -(n/2) log 2 pi constant and const = 0 in Eq. 1.
 */
bta_status inla_value_and_grad(inla_model* m, const double* theta, int32_t batch, double* f,
                               double* grad, const inla_opts* opts, cudaStream_t stream);

/*
 * inla_backward -- the reverse pass alone (Eq. 6, Phases A-C via the two
 * in-place selected inversions) for the theta of the immediately preceding
 * value-only inla_value_and_grad call (batch 1), reusing the factors that
 * call left in the model.  grad: host, d values.  BTA_ERR_STATE if there is
 * no such value-only call (the factors are consumed: a second call fails).
 */
bta_status inla_backward(inla_model* m, double* grad, int32_t use_graph, cudaStream_t stream);

/*
 * inla_hessian -- Section III-D, Eq. 13: the posterior Hessian at theta as
 * central differences of exact gradients, H[:, j] = (grad f(theta + h e_j) -
 * grad f(theta - h e_j)) / 2h, i.e. 2d + 1 calls of the gradient instead of
 * 2d^2 + 1 objective evaluations (the paper uses h = 5e-3).  H: host, d x d
 * row-major (H[i*d + j] = dgrad_i / dtheta_j, not symmetrised); grad0: host,
 * d values of the gradient at theta, or NULL.  opts as for
 * inla_value_and_grad (opts->streams > 1 evaluates that many gradients
 * together).  Synchronises stream.
 */
bta_status inla_hessian(inla_model* m, const double* theta, double h, double* H, double* grad0,
                        const inla_opts* opts, cudaStream_t stream);

/*
 * Several independent models -- e.g. the thetas of a finite-difference
 * stencil or of a line search on models of different block sizes -- evaluated
 * by ONE CUDA graph launch: each model's whole evaluation (theta upload,
 * both factorisations, solve, optional selected inversions, result download)
 * is a branch of the graph on that model's own streams, so the branches of
 * uneven size run concurrently and fill each other's idle SMs.
 *   inla_batch_create: the models (distinct, each used by at most one batch
 *     at a time) are borrowed, not copied.
 *   inla_batch_value_and_grad: theta row i (host, leading dimension ldt >=
 *     every model's d) goes to model i; f[i], grad row i (ldt stride, or
 *     grad = NULL for values only).  opts->precision as for
 *     inla_value_and_grad.  The graph is captured on the first call per
 *     (value/gradient, precision) and replayed after.  Synchronises stream.
 */
typedef struct inla_batch inla_batch;
bta_status inla_batch_create(inla_model* const* models, int32_t count, inla_batch** out);
void inla_batch_destroy(inla_batch* b);
bta_status inla_batch_value_and_grad(inla_batch* b, const double* theta, int32_t ldt, double* f,
                                     double* grad, const inla_opts* opts, cudaStream_t stream);

/*
 * inla_last_parts -- diagnostics of the last single evaluation (host):
 * parts[0..7] = log|Q_p|, log|Q_c|, x^T Q_p x, log l, log p, f, (unused) x2;
 * phases (may be NULL): 4 x d values Phase A, Phase B, Phase C, explicit.
 */
bta_status inla_last_parts(const inla_model* m, double* parts, double* phases);

/* inla_copy_mode -- copy the last conditional mode x* (device, n*ld + a,
 * padded layout) into dst (device). */
bta_status inla_copy_mode(const inla_model* m, double* dst, cudaStream_t stream);

/*
 * bta_gemm -- the FP64 tile contraction every sweep step is built from
 * (Algorithm 1 and the selected inversion are sequences of these products):
 * C = alpha op(A) op(B) + beta C, column-major, device pointers, op = transpose
 * when the flag is 1; op(A) is M x K, op(B) is K x N.  Stream-ordered.
 */
bta_status bta_gemm(int32_t M, int32_t N, int32_t K, double alpha, const double* A, int32_t lda,
                    int32_t transA, const double* B, int32_t ldb, int32_t transB, double beta,
                    double* C, int32_t ldc, cudaStream_t stream);

/*
 * bta_gemm_mixed -- the same product as bta_gemm, computed in split
 * precision on the tensor cores (the off-diagonal Schur-complement products
 * of the mixed-precision mode): each FP64 operand is carried as a pair of
 * TF32 values hi + lo, three TF32 products (hi*hi, hi*lo, lo*hi) accumulate
 * in FP32, the result is combined with alpha and beta in FP64.  Relative
 * error per entry ~1e-6 of sum |A||B|.  status (device int32, may be NULL)
 * receives BTA_ERR_TIMEOUT if a bounded wait in the kernel expired (0 is
 * never written: initialise it).  Allocates its operand copies with
 * cudaMallocAsync on the stream.
 */
bta_status bta_gemm_mixed(int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                          int32_t lda, int32_t transA, const double* B, int32_t ldb,
                          int32_t transB, double beta, double* C, int32_t ldc, int32_t* status,
                          cudaStream_t stream);

/*
 * bta_gemm_emulated -- the same product as bta_gemm to FP64 accuracy on the
 * BF16 tensor cores (the products of the emulated-FP64 mode, the Ozaki
 * error-free splitting; no counterpart in the paper, whose GPUs have FP64
 * tensor cores): each row of op(A) and column of op(B) is scaled by a power
 * of two and written as `slices` (6..8) signed base-128 digits (7 bits
 * each: 8 slices carry 56 bits, more than FP64's 53), the slice products
 * of the leading levels accumulate exactly in FP32 and are summed in 64-bit
 * integers, and the result is rounded once to FP64.  Error per entry at most
 * (slices + 4) 2^(-7 slices) K max_k|a_ik| max_k|b_kn| plus the final
 * rounding (slices = 8: the order of an FP64 GEMM's rounding bound).  Requires 1 <= K <= 5120.  status as for
 * bta_gemm_mixed.  Allocates its operand slices with cudaMallocAsync on
 * the stream.
 */
bta_status bta_gemm_emulated(int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                             int32_t lda, int32_t transA, const double* B, int32_t ldb,
                             int32_t transB, double beta, double* C, int32_t ldc,
                             int32_t slices, int32_t* status, cudaStream_t stream);

/*
 * bta_gemm_emulated_timed -- bta_gemm_emulated (same arguments and result)
 * that also writes to kernel_ms (host float) the duration of its tensor-core
 * product kernel alone, from CUDA events recorded on the stream around that
 * launch (the exponent, split and compose kernels excluded): the measurement
 * behind the emulated product's roofline.  Synchronises the stream.  The
 * paper has no counterpart.
 */
bta_status bta_gemm_emulated_timed(int32_t M, int32_t N, int32_t K, double alpha,
                                   const double* A, int32_t lda, int32_t transA, const double* B,
                                   int32_t ldb, int32_t transB, double beta, double* C,
                                   int32_t ldc, int32_t slices, int32_t* status,
                                   float* kernel_ms, cudaStream_t stream);

/*
 * inla_grid_stencil -- spatial base matrices of an nx x ny grid model
 * (Section II-A): Cm = I, G = 5-point graph Laplacian with natural boundary,
 * GG = G G, all on GG's 13-point pattern, CSR with sorted columns (host
 * arrays, caller-owned).  Call once with row_ptr = NULL to get *nnz, then with
 * arrays of ns+1 and *nnz entries.  Host-only, no device work.
 */
bta_status inla_grid_stencil(int32_t nx, int32_t ny, int32_t* nnz, int32_t* row_ptr,
                             int32_t* col, double* val_C, double* val_G, double* val_GG);

/*
 * bta_set_wait_limit -- test hook for the bounded device waits of the
 * diagonal-block factor (the task graph of bta_factor and of every
 * evaluation): limit_ns bounds each wait (1 ms .. 60 s; 0 restores the 2 s
 * default); stall = 1 makes the factor's chain wait on a counter that nothing
 * sets, so that its waits run out and the factor reports BTA_ERR_TIMEOUT
 * (fail_block, or the status of inla_value_and_grad) without a fault.  The
 * paper has no counterpart.  Process-wide; applies to launches recorded after
 * the call (a CUDA graph captured before keeps its settings).  Host-only.
 */
bta_status bta_set_wait_limit(int64_t limit_ns, int32_t stall);

/*
 * bta_pivot_reciprocals -- the two scalar functions the diagonal-block
 * factor applies to every pivot d (Algorithm 1's POTRF leaf), exposed so
 * they can be checked against CUDA's own: recip_out[i] = 1 / v[i] (relative
 * error within 2^-52 of the correctly rounded value for |v| in 2^-100 ..
 * 2^100; the division elsewhere) and rsqrt_out[i] = v[i]^{-1/2} (within
 * 2^-51 relative for positive v in that range; 1 / sqrt(v) elsewhere).
 * v, recip_out, rsqrt_out: device arrays of n doubles; either output may be
 * NULL.  Stream-ordered.  The paper has no counterpart.
 */
bta_status bta_pivot_reciprocals(const double* v, int64_t n, double* recip_out,
                                 double* rsqrt_out, cudaStream_t stream);

/* Number of kernels inla_value_and_grad ran for this model (CUDA-graph
 * replays counted kernel by kernel); NULL: kernels the library launched. */
int64_t inla_kernel_launches(const inla_model* m);

/* Human-readable text for a status. */
const char* bta_status_string(bta_status s);

#ifdef __cplusplus
}
#endif
#endif /* BTA_H */
