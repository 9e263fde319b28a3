/*
 * eda.h - C ABI of the GB300 (sm_103a) library for exponential discriminant
 * analysis (EDA): the t dominant eigenpairs of the pencil
 *     exp(c^2 S_B) x = lambda exp(c^2 S_W) x                       (Eq. (1.7))
 * solved in the symmetric form M y = lambda y with
 *     M = exp(-c^2 S_W / 2) exp(c^2 S_B) exp(-c^2 S_W / 2)        (Eqs. (3.13), (3.15))
 * by block Lanczos (Algorithm 3), where S_W = H_W H_W^T and S_B = H_B H_B^T
 * (Eqs. (1.1), (1.2)) are never formed: every exponential is applied through
 * Theorem 3.1 as
 *     exp(alpha H H^T) X = X + H K(alpha) (H^T X),
 *     K(alpha) = alpha phi(alpha H^T H),  phi(z) = (e^z - 1) / z.
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers unless a comment says otherwise. The caller
 *    owns every input and output buffer; the library owns the handle and the
 *    device memory behind it (factors, Gram matrices, operators, workspaces).
 *  - Matrices are column-major. A d x n sample block has one sample per
 *    column, each sample contiguous, leading dimension ld >= d.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is issued on it in order. Calls that return results to the
 *    host (eda_build, eda_solve) synchronise that stream before returning.
 *  - Every call returns an eda_status; no call aborts, traps or exits. On a
 *    CUDA error the code is EDA_ERR_CUDA and eda_last_cuda_error() tells which.
 *  - Handles are not thread-safe: one handle is used by one host thread at a time.
 */
#ifndef EDA_GB300_H
#define EDA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EDA_OK = 0,
    EDA_ERR_INVALID_ARG = -1,    /* a size, pointer, enum or tolerance is out of range      */
    EDA_ERR_BAD_LABELS = -2,     /* a label outside [0, k) or a class with no sample          */
    EDA_ERR_NONFINITE = -3,      /* NaN/Inf in the input, a Gram matrix or a residual         */
    EDA_ERR_OOM = -4,            /* device allocation failed                                 */
    EDA_ERR_CUDA = -5,           /* a CUDA call failed; see eda_last_cuda_error()              */
    EDA_ERR_TIMEOUT = -6,        /* a bounded device wait (grid barrier) gave up              */
    EDA_ERR_BREAKDOWN = -7,      /* Krylov block lost rank and could not be refilled          */
    EDA_ERR_NOT_CONVERGED = -8   /* outputs hold the best Ritz pairs; see eda_solve_info      */
} eda_status;

typedef enum {
    EDA_F64 = 0,                 /* IEEE double                                              */
    EDA_F32 = 1,                 /* IEEE single                                              */
    EDA_BF16 = 2,                /* bfloat16 storage, FP32 accumulation                      */
    EDA_BF16X2 = 3,              /* hi + lo bfloat16 split of an FP32 value (not accepted)   */
    EDA_F64_TC = 4               /* FP64-accurate products on the bf16 tensor cores: each    */
                                 /* operand split exactly into 7 bf16 digit planes with a   */
                                 /* power-of-two scale per row, 28 plane products with exact */
                                 /* integer accumulation (error-free splitting)             */
} eda_prec;

typedef enum {
    EDA_OP_SW = 0,               /* Y = exp(alpha S_W) X                                     */
    EDA_OP_SB = 1,               /* Y = exp(alpha S_B) X                                     */
    EDA_OP_M = 2,                /* Y = M X with the handle's c^2 (alpha ignored)            */
    EDA_OP_N = 3                 /* Y = exp(-c^2 S_W) exp(c^2 S_B) X, the nonsymmetric form  */
                                 /* of Eq. (3.1) (alpha ignored; FP64 io only)               */
} eda_op;

typedef struct {
    int32_t prec;                /* eda_prec of the Krylov sweeps: EDA_F64 (plain FP64),      */
                                 /* EDA_F64_TC (FP64 solver whose M-apply sweeps over        */
                                 /* [H_W H_B] run as FP64-accurate tensor-core products),    */
                                 /* EDA_F32 (single-precision H, basis and sweeps) or         */
                                 /* EDA_BF16 (bf16 H on the tensor cores, single-precision    */
                                 /* basis); the last two end with FP64 refinement to tol      */
    int32_t block_b;             /* block size b of block Lanczos (>= 1)                     */
    int32_t m_max;               /* max basis columns; <= 0 selects n + k + b (exact end)    */
    int32_t check_every;         /* Rayleigh-Ritz convergence check every this many blocks   */
    double tau;                  /* scale target: c^2 = tau / max(lmax(G_W), lmax(G_B))      */
    double c2;                   /* explicit c^2 when > 0 (tau is then ignored)              */
    uint64_t seed;               /* seed of the counter-based start block / refill vectors  */
    int32_t true_residuals;      /* 1: eda_solve also reports true FP64 residuals            */
    int32_t m_form;              /* FP64 M-apply: 0 = the three products of the symmetric     */
                                 /* form one after another (Eq. (3.16)); 1 = their composed  */
                                 /* form M = I + Z C Z^T, Z = [H_W H_B] (Theorem 3.1 for each  */
                                 /* factor; two sweeps over Z instead of six over H_W, H_B)   */
    int32_t wait_limit;          /* polls of a grid-wide barrier wait (the cooperative        */
                                 /* symmetric eigensolver, n > 512) before it gives up and    */
                                 /* the call returns EDA_ERR_TIMEOUT; <= 0: the default,      */
                                 /* 20,000,000 (about 1-2 s)                                  */
    int32_t tc_min_mi;           /* EDA_F64_TC: the size of Z = [H_W H_B], d (n + k), in units  */
                                 /* of 2^20 entries, from which the tensor-core products are  */
                                 /* used; below it the FP64 ones (the two agree to FP64       */
                                 /* rounding; the splitting launches cost more than they save */
                                 /* on small factors); 0: the default, 4; < 0: always         */
    int32_t tc_fused;            /* EDA_BF16: >= 0 (default 0) applies exp(alpha H H^T) in one  */
                                 /* resident launch when the factor fits the SMs' shared      */
                                 /* memory (d <= 128 x resident CTAs, n <= 768): bf16 of      */
                                 /* B = H R^T with sign(alpha) K = R^T R, read once; < 0: the */
                                 /* four-launch sweeps of bf16 H and bf16 H K                 */
    int32_t reserved[3];
} eda_config;

typedef struct {
    int32_t converged;           /* number of the t wanted pairs with rel-res <= tol          */
    int32_t iters;               /* block Lanczos steps taken                                */
    int32_t mapplies;            /* M-applies, counted in d x b blocks                       */
    int32_t basis_cols;          /* final basis width m                                      */
    int32_t refills;             /* rank-deficient columns replaced by fresh random vectors  */
    int32_t checks;              /* Rayleigh-Ritz checks performed                            */
    int32_t refine_iters;        /* FP64 refinement rounds: mixed precision, or FP64 after refills */
    int32_t reserved0;
    double c2, lmax_w, lmax_b;   /* scale and the two largest Gram eigenvalues               */
    double max_relres_est;       /* max_i ||B_{m+1} S_{m,i}|| / theta_i over the t pairs      */
    double max_relres_true;      /* max_i ||M y_i - theta_i y_i|| / theta_i (if requested)   */
    double ms_solve;             /* device time of the whole eda_solve call                   */
    double* relres;              /* HOST pointer, t entries, filled when non-NULL            */
} eda_solve_info;

typedef struct eda_ctx* eda_handle;

/* Fill *cfg with defaults: F64, b = 8, m_max = 0 (n + k + b), check_every = 1,
 * tau = 10, c2 = 0, seed = 1, true_residuals = 0, m_form = 0, wait_limit = 0. */
int eda_config_default(eda_config* cfg);

/* Build a handle from labelled samples (Section 1; Algorithm 2 step 1 with the
 * Gram form of steps 2-4).
 *   X       : d x n samples, x_dtype EDA_F64 or EDA_F32, leading dimension ldx >= d.
 *   labels  : n int32 class ids in [0, k).
 * Steps on the device: stable class segmentation; centroids mu_j, mu in a
 * fixed order (bit-exact FP64); H_W (d x n, class-major columns, input order
 * within a class) and H_B (d x k, columns sqrt(n_j)(mu_j - mu)); Gram
 * matrices G_W = H_W^T H_W, G_B = H_B^T H_B in FP64; their largest eigenvalues
 * and c^2 (the scale of the samples' spread, A1: c^2 = tau / max lambda_max); and
 * K(alpha) = alpha phi(alpha G) for alpha = -c^2/2 (W) and +c^2 (B) (Theorem 3.1). When n and
 * k are at most 256, lambda_max comes from a Lanczos run whose error bound is checked (the
 * symmetric eigensolver when the bound fails) and K from G by scaling and squaring; beyond,
 * both come from the Grams' symmetric eigendecompositions.
 * Errors: INVALID_ARG (d < 1, n < 2, k < 1, k > n, ldx < d), BAD_LABELS,
 * NONFINITE (X has NaN/Inf), OOM, CUDA. *out is set only on EDA_OK.
 * X and labels are read only during the call (stream-ordered). */
int eda_build(const void* X, int32_t x_dtype, int64_t d, int64_t n, int64_t ldx,
              const int32_t* labels, int32_t k, const eda_config* cfg, void* stream,
              eda_handle* out);

/* Build a handle from given factors (H_W: d x n, H_B: d x kb, FP64, ld = d).
 * No segmentation or centroid step; everything from the Gram on is as in
 * eda_build. Used for closed-form checks (commuting diagonal factors). */
int eda_build_from_factors(const double* HW, int64_t n, const double* HB, int64_t kb, int64_t d,
                           const eda_config* cfg, void* stream, eda_handle* out);

/* Y = exp(alpha H H^T) X for op SW (H = H_W) or SB (H = H_B), or Y = M X for
 * op M (Theorem 3.1; Algorithm 2 steps 6L-12L for M). X, Y: d x b, leading
 * dimension ldx. io_dtype EDA_F64 uses the FP64 factors (any handle, any alpha);
 * io_dtype EDA_F32 uses the handle's working precision (prec EDA_F32: single-
 * precision sweeps; prec EDA_BF16: bf16 H on the tensor cores) and accepts only the
 * stored alphas (-c^2/2 for SW, c^2 for SB). X and Y must not overlap. An FP64 alpha other
 * than the stored one needs the Gram's eigenpairs: the first such call computes them
 * (symmetric eigensolver, with host synchronisation) if the build did not. */
int eda_apply_exp(eda_handle h, int32_t op, double alpha, const void* X, void* Y,
                  int64_t ldx, int32_t b, int32_t io_dtype, void* stream);

/* The t dominant eigenpairs (Algorithm 3, steps 5-6).
 *   V0     : optional d x b0 start block (NULL: seeded counter-based Gaussian block).
 *   V      : d x t output, orthonormal basis of the t generalized eigenvectors
 *            x_i = exp(-c^2 S_W / 2) y_i (Eq. (3.14)), orthonormalised.
 *   lambda : t output eigenvalues, descending.
 *   Y      : optional d x t output, the orthonormal Ritz vectors y_i of M.
 * tol is the relative residual ||M y - theta y|| <= tol * theta of each of the t
 * pairs (Remark 3.4). Returns EDA_ERR_NOT_CONVERGED (outputs still written)
 * when the basis limit is reached first. When the Krylov phase replaced lost directions by fresh
 * ones (refills > 0), the FP64 solver ends with a Rayleigh-Ritz / residual-expansion phase on true
 * FP64 residuals (refine_iters rounds), as the residual estimate cannot see such losses. */
int eda_solve(eda_handle h, int32_t t, double tol, const double* V0, int32_t b0,
              double* V, double* lambda, double* Y, eda_solve_info* info, void* stream);

/* The t dominant eigenpairs of the nonsymmetric form of the pencil, Eq. (3.1):
 *     exp(-c^2 S_W) exp(c^2 S_B) x = lambda x,
 * by block Arnoldi (Section 3.1; Algorithm 2 steps 6A-10A for the products; Algorithm 3 step 5, Arnoldi
 * form). Each step applies the operator once (two Theorem 3.1 products, as two sweeps over [H_W H_B]);
 * the basis is kept orthonormal by full reorthogonalisation (as for eda_solve). The Ritz pairs are the
 * real eigenpairs of the Galerkin condition with test space exp(c^2 S_W) V on the Arnoldi subspace V
 * (a symmetric-definite projected pencil). There is no recovery step: the Ritz vectors are the
 * generalized eigenvectors x themselves.
 *   V      : d x t output, orthonormal basis of the t generalized eigenvectors.
 *   lambda : t output eigenvalues, descending.
 * tol bounds ||N x - theta x|| / (theta ||x||) for each pair (from the Arnoldi relation; when directions
 * were refilled, from true residuals, one N-apply of the Ritz vectors, once the relation's estimates are
 * within a factor 100 of tol or the basis is full: info->max_relres_true >= 0 and info->refine_iters counts
 * those verifications). The handle's
 * prec selects FP64 or tensor-core FP64 sweeps (EDA_F64, EDA_F64_TC); block size, basis limit, check
 * schedule and seed come from its configuration. Errors as for eda_solve. */
int eda_solve_arnoldi(eda_handle h, int32_t t, double tol, double* V, double* lambda, eda_solve_info* info,
                      void* stream);

/* The t dominant eigenpairs of the symmetric form solved exactly in the span of Z = [H_W H_B], without
 * Krylov iteration: a cross-check of eda_solve at the cost of two small dense eigenproblems.
 * Theorem 3.1 for each factor of M (Eq. (3.15)) gives M = I + Z C Z^T with C built from K_W, K_B and the
 * Grams, so every eigenvector of M whose eigenvalue is not 1 lies in range(Z) (Theorem 3.7). Z has k + 1
 * known dependent columns (each class's columns of H_W sum to zero; so do the sqrt(n_j)-weighted columns
 * of H_B); without them the Gram of the other n - 1 columns is Cholesky-factored, the (n - 1) x (n - 1)
 * symmetric matrix I + P^T C P (P = Z^T Q, Q the orthonormal basis this gives) is solved for its t
 * largest eigenpairs, and the recovery x = exp(-c^2 S_W / 2) y (Eq. (3.14)) and orth (Algorithm 3 step 6)
 * are done in the coordinates of Z, followed by one pass over Z for V and one CholQR pass on V.
 *   t      : 1 <= t <= n - 1 (the eigenvalues above 1 are k - 1 of the n - 1 nontrivial ones).
 *   V      : d x t output, orthonormal basis of the t generalized eigenvectors (ld d).
 *   lambda : t output eigenvalues, descending.
 *   info   : optional; converged = t, basis_cols = n - 1, ms_solve = device time of the call.
 * Needs a handle from eda_build (the class structure), prec EDA_F64 or EDA_F64_TC (tensor-core FP64
 * products for the n x n operators and the pass over Z when the handle has them); INVALID_ARG otherwise.
 * BREAKDOWN when the n - 1 kept columns are numerically dependent (samples not affinely independent).
 * Other errors as for eda_solve. Synchronises the stream. */
int eda_solve_direct(eda_handle h, int32_t t, double* V, double* lambda, eda_solve_info* info, void* stream);

/* P = V^T Xq (t x m, column-major, ld t): the projected samples of the
 * nearest-neighbour classifier (Section 3.3, d_ij = ||V^T (x_i - y_j)||).
 * V: d x t (ld d); Xq: d x m (EDA_F64 or EDA_F32, ld ldq). */
int eda_project(eda_handle h, const double* V, int32_t t, const void* Xq, int32_t xq_dtype,
                int64_t m, int64_t ldq, double* P, void* stream);

/* Y = X + H K (H^T X) for a caller-supplied operator, allocating no device memory.
 * The paper has no counterpart: this is for callers that must not allocate, such as code
 * embedded in a host framework that owns a fixed device-memory budget, or latency-critical
 * loops where cudaMalloc/cudaFree (which may synchronise the device) cannot be used.
 *   H : d x m, K : m x m (for exp(alpha H H^T) pass K = alpha phi(alpha H^T H), e.g. the KW or
 *       KB matrices returned by eda_get_factors), X, Y : d x b, all FP64, leading dimension ld
 *       (H uses ld = d). Y must not overlap X, H or K (EDA_ERR_INVALID_ARG otherwise).
 * Temporaries live in one fixed 4 MiB device array inside the library (held on every GPU that
 * loads it until the process exits): m * b must not exceed 174762 (2^19 / 3 doubles), larger
 * sizes return EDA_ERR_INVALID_ARG before any device work. The first call on a device looks up
 * that array's device address with the device current; make that first call before any stream
 * capture. The address is kept together with the identity of the device's context and looked up
 * again when that context changes (after cudaDeviceReset the module, and with it the array, is
 * loaded anew; the next call on that device is again a first call). All calls share the array,
 * so calls whose work overlaps on the GPU (different streams, or other host threads) race and
 * must be serialised by the caller. Nothing carries over between calls: every scratch value
 * read is written earlier in the same call. */
int eda_lowrank_exp_apply_noalloc(const double* H, int64_t d, int32_t m, const double* K,
                                  const double* X, double* Y, int64_t ld, int32_t b, void* stream);

/* One problem of a batched solve (all pointers device pointers except info.relres).
 * Inputs as for eda_build / eda_solve; block_b = 0 uses the batch configuration's block size,
 * or the tuned one when that is 0 as well. Outputs: V (d x t, orthonormal basis of the
 * generalized eigenvectors), lambda (t, descending), status (eda_status of this problem) and info
 * (info.relres is not filled). */
typedef struct {
    const void* X;               /* d x n samples, x_dtype EDA_F64 or EDA_F32, leading dim ldx  */
    int32_t x_dtype;
    int32_t k;                   /* classes                                                   */
    int64_t d, n, ldx;
    const int32_t* labels;       /* n class ids in [0, k)                                     */
    int32_t t;                   /* wanted eigenpairs                                         */
    int32_t block_b;             /* 0: batch default / tuned                                  */
    double tol;                  /* relative residual of every wanted pair                    */
    double* V;                   /* out: d x t                                                */
    double* lambda;              /* out: t                                                    */
    int32_t status;              /* out                                                       */
    int32_t reserved;
    eda_solve_info info;         /* out                                                       */
} eda_problem;

/* Solve nprob independent problems of uneven d, n, k (random training splits, class subsets): the
 * single-problem path of eda_build and eda_solve for each, run side by side by `workers` host
 * threads (<= 0: 16), each with its own CUDA stream, largest problems first. When cfg->block_b is
 * 0, each problem shape gets the block size that minimises the measured time of one M-apply of
 * width b times the ceil(t / b) + 2 blocks of a solve (b in {4, 8, 16, 32}). The batch starts after
 * the work already queued on `stream` and `stream` waits for all of it; the call returns when every
 * problem is done. Returns EDA_OK when every problem converged, else the first hard error of a
 * problem, else EDA_ERR_NOT_CONVERGED; per-problem results are in probs[i].status. The paper has
 * no batched counterpart: its experiments solve one split at a time. */
int eda_solve_batched(eda_problem* probs, int32_t nprob, const eda_config* cfg, int32_t workers,
                      void* stream);

/* Copy out build results into caller device buffers (any pointer may be NULL):
 * HW d x n, HB d x k, counts k, perm n, GW n x n, GB k x k, KW n x n
 * (alpha = -c^2/2), KB k x k (alpha = c^2), evals_w n, evals_b k (ascending). The
 * eigenvalues are computed by the first call that asks for them when the build did not
 * need them (symmetric eigensolver on the stream, with host synchronisation). */
int eda_get_factors(eda_handle h, double* HW, double* HB, int32_t* counts, int32_t* perm,
                    double* GW, double* GB, double* KW, double* KB, double* evals_w,
                    double* evals_b, void* stream);

/* Host-side scalars of a built handle. Any pointer may be NULL. */
int eda_get_dims(eda_handle h, int64_t* d, int64_t* n, int32_t* k, double* c2,
                 double* lmax_w, double* lmax_b);

void eda_destroy(eda_handle h);
const char* eda_strerror(int status);
/* The last CUDA error code seen by any call of this thread (0 = none), and its name with the
 * library source location that saw it (a static per-thread string). */
int eda_last_cuda_error(void);
const char* eda_last_cuda_error_string(void);

/* Number of this library's kernels launched so far by the calling process. */
uint64_t eda_kernel_launches(void);

/* Region timers (off by default). When enabled, the library records a CUDA event pair on the
 * launching stream around each call of a named region: "exp_apply_w" / "exp_apply_b" (one
 * Theorem 3.1 product with H_W / H_B),
 * "m_apply" (three products), "tridiag" (Householder reduction), "symeig" (a full small
 * eigensolve), "gram" (the two Gram products of the build), "rr" (one Rayleigh-Ritz check),
 * "reorth" (one CGS2 pass pair). eda_profile_read synchronises the pending events of a region
 * and returns its accumulated device time in ms and its call count (0, 0 for unknown names). */
int eda_profile_enable(int on);
int eda_profile_reset(void);
int eda_profile_read(const char* region, double* total_ms, int64_t* calls);
/* Algorithmic work counted by the library for the calls of a region while timing was on: FLOPs
 * and bytes by the definition of the operation, not by the kernels' actual traffic ("tridiag":
 * 4/3 n^3 flops; "exp_apply_w"/"exp_apply_b": 4 d m b + 2 m^2 b flops and 2 |H| + 3 |X| bytes
 * in the storage type of the sweeps; 0, 0 for regions without a count or unknown names). */
int eda_profile_work(const char* region, double* flops, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* EDA_GB300_H */
