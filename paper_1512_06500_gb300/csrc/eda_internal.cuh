// Internal declarations shared by the CUDA translation units of the EDA library.
#pragma once

#include <cuda.h>            // CUtensorMap (types only; the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include <atomic>
#include <mutex>

#include "../../include/eda.h"

namespace eda {

// ---------------------------------------------------------------- errors
void note_cuda_error(cudaError_t e, const char* file = nullptr, int line = 0);
std::atomic<uint64_t>& launch_counter();   // kernels launched by this process (all threads)

#define EDA_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t e__ = (expr);                                 \
        if (e__ != cudaSuccess) {                                 \
            ::eda::note_cuda_error(e__, __FILE__, __LINE__);      \
            return e__ == cudaErrorMemoryAllocation ? EDA_ERR_OOM \
                                                    : EDA_ERR_CUDA; \
        }                                                         \
    } while (0)

#define EDA_TRY(expr)                    \
    do {                                 \
        int s__ = (expr);                \
        if (s__ != EDA_OK) return s__;   \
    } while (0)

// After a kernel launch: count it and surface launch-configuration errors.
#define EDA_LAUNCHED()                                \
    do {                                              \
        ::eda::launch_counter()++;                    \
        EDA_CUDA_TRY(cudaPeekAtLastError());          \
    } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Device status word bits (written by kernels, read by the host).
enum : int {
    ST_TIMEOUT = 1,       // a bounded grid-barrier wait gave up
    ST_NONFINITE = 2,     // NaN/Inf met
    ST_BADLABEL = 4,      // a label outside [0, k)
    ST_EMPTYCLASS = 8,    // a class without samples
    ST_RANKLOSS = 16,     // Cholesky pivot below the rank threshold
};

// ---------------------------------------------------------------- region timers
// Records a CUDA event pair around its scope on stream s when profiling is enabled.
class ProfScope {
  public:
    // flops, bytes: algorithmic work of this call, accumulated per region while timing is on
    ProfScope(const char* name, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t e0_ = nullptr;
};

// ---------------------------------------------------------------- workspace
// A stream-ordered bump allocator over one device block owned by the handle.
struct Arena {
    char* base = nullptr;
    size_t cap = 0, used = 0;
    template <class T> T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        if (off + count * sizeof(T) > cap) return nullptr;
        used = off + count * sizeof(T);
        return reinterpret_cast<T*>(base + off);
    }
    void reset() { used = 0; }
};

// Grid barrier state in device memory (zeroed at allocation) and the number of polls a wait makes
// before it gives up (ST_TIMEOUT).
constexpr long long kGridSpinDefault = 20000000;   // about 1-2 s of polling
struct GridBarrier {
    unsigned int* count;
    unsigned int* gen;
    long long spin_limit = kGridSpinDefault;
};

// ---------------------------------------------------------------- dense FP64 ops
// C (m x p) = alpha * A^T B (+ beta * C), A: d x m (lda), B: d x p (ldb), reduction over d split
// across CTAs with a fixed-order second pass (deterministic). partial: >= splits * m * p doubles.
int gemm_tn_f64(int64_t d, int m, int p, double alpha, const double* A, int64_t lda,
                const double* B, int64_t ldb, double beta, double* C, int ldc,
                double* partial, size_t partial_cap, cudaStream_t s);
// Symmetric C (m x m) = alpha * A^T A (+ beta * C), A: d x m: only the tiles of the lower triangle are
// computed and each result is written to both triangles (bitwise symmetric).
int syrk_f64(int64_t d, int m, double alpha, const double* A, int64_t lda, double beta, double* C, int ldc,
             double* partial, size_t partial_cap, cudaStream_t s);
// Streaming multiprocessors of the current device (queried once per process).
int sm_count();
// C (d x p) = beta * C0 + alpha * A B, A: d x m (lda), B: m x p (ldb); C may equal C0 (same ld).
int gemm_nn_f64(int64_t d, int m, int p, double alpha, const double* A, int64_t lda,
                const double* B, int ldb, double beta, const double* C0, int64_t ldc0,
                double* C, int64_t ldc, cudaStream_t s);
// Small dense C (m x p) = alpha * op(A) op(B) + beta * C with op = N or T (all column-major).
int gemm_small_f64(bool ta, bool tb, int m, int p, int kk, double alpha, const double* A, int lda,
                   const double* B, int ldb, double beta, double* C, int ldc, cudaStream_t s);
// In-place upper Cholesky of a b x b SPD matrix G = R^T R (R stored in the upper triangle, the
// strict lower triangle zeroed) and Rinv = R^{-1} (b x b, ld b). A pivot (squared) at or below
// max(rank_tol * max diag, piv_min2) marks rank loss: that row of R and of Rinv is set to zero
// and ST_RANKLOSS is or-ed into *status; lost pivots are listed in lost[0..], lost[b] = count.
int chol_inv_small(int b, double* G, int ldg, double* Rinv, double rank_tol, double piv_min2,
                   int* status, int* lost, cudaStream_t s);
// The same factorisation for any m, blocked: one-CTA factorisations of kCholBlock x kCholBlock diagonal
// blocks and multi-CTA products for the panels, trailing updates and the inverse. Rank detection
// (rank_tol) applies within each diagonal block; no lost list. work: chol_inv_blocked_doubles(m) doubles;
// partial: split-K partials (at least m * m doubles).
constexpr int kCholBlock = 64;
size_t chol_inv_blocked_doubles(int m);
int chol_inv_blocked(int m, double* G, int ldg, double* Rinv, int ldr, double rank_tol, int* status, double* work,
                     double* partial, size_t pcap, cudaStream_t s);
// chol_inv_small (one CTA) up to b = 90, chol_inv_blocked beyond (Rinv with ld b); no lost list, no pivot floor.
int chol_inv_auto(int b, double* G, int ldg, double* Rinv, double rank_tol, int* status, double* work, double* partial,
                  size_t pcap, cudaStream_t s);
// Copy / scale / symmetrise helpers.
int copy_mat_f64(int64_t rows, int cols, const double* A, int64_t lda, double* B, int64_t ldb,
                 cudaStream_t s);
int symmetrize_f64(int m, double* A, int lda, cudaStream_t s);
int fill_gaussian_f64(int64_t rows, int cols, double* A, int64_t lda, uint64_t seed,
                      uint64_t stream_id, cudaStream_t s);
int col_norms_f64(int64_t rows, int cols, const double* A, int64_t lda, double* out, cudaStream_t s);

// Templated tall-skinny products on the storage type T (double or float). T = float computes
// each split in single precision and sums the splits in double; the small outputs/operands
// (C of gemm_tn, B of gemm_nn) are always double. partial_buf holds splits * m * p values of T.
template <class T>
int gemm_tn(int64_t d, int m, int p, double alpha, const T* A, int64_t lda, const T* B, int64_t ldb, double beta,
            double* C, int ldc, void* partial_buf, size_t partial_cap, cudaStream_t s);
template <class T>
int syrk_tn(int64_t d, int m, double alpha, const T* A, int64_t lda, double beta, double* C, int ldc,
            void* partial_buf, size_t partial_cap, cudaStream_t s);
// b_upper: B is upper triangular with its zeros stored (B[l, c] = 0 for l > c, as R^{-1} from
// chol_inv_small); the product then skips rows of B that are zero for a whole column slice (exact zero
// terms, so the result is bit-for-bit that of the full product for finite A).
template <class T>
int gemm_nn(int64_t d, int m, int p, double alpha, const T* A, int64_t lda, const double* B, int ldb, double beta,
            const T* C0, int64_t ldc0, T* C, int64_t ldc, cudaStream_t s, bool b_upper = false);
template <class Ti, class To>
int copy_mat(int64_t rows, int cols, const Ti* A, int64_t lda, To* B, int64_t ldb, cudaStream_t s);
template <class T>
int fill_gaussian(int64_t rows, int cols, T* A, int64_t lda, uint64_t seed, uint64_t stream_id, cudaStream_t s);
template <class T>
int col_norms(int64_t rows, int cols, const T* A, int64_t lda, double* out, cudaStream_t s);

// ---------------------------------------------------------------- symmetric eigensolver
struct SymEigWork {
    double* A;        // n x n copy (destroyed)
    double* dgl;      // n diagonal
    double* eoff;     // n off-diagonal
    double* tau;      // n Householder scalars
    double* vbuf;     // 4 * n scratch vectors for the tridiagonal reduction
    double* partial;  // per-CTA partial sums (2 * max_ctas)
    double* lu;       // 5 * n * nv inverse-iteration factors
    GridBarrier bar;
    int max_ctas;
};
size_t symeig_work_bytes(int n, int nv);
int symeig_work_carve(Arena& a, int n, int nv, GridBarrier bar, SymEigWork* w);
// Eigenpairs with ascending indices il..iu (0-based) of the symmetric n x n A (lda). Eigenvalues go
// to w (iu-il+1, ascending), eigenvectors to Z (n x (iu-il+1), ldz) when Z != NULL. Runs of
// eigenvalues whose gaps are <= cluster_rel * max|w| get explicit Gram-Schmidt.
int symeig_f64(int n, const double* A, int lda, int il, int iu, double* w, double* Z, int ldz,
               SymEigWork* ws, int* status, uint64_t seed, double cluster_rel, cudaStream_t s);
// The two halves of symeig_f64: reduction + eigenvalues, then eigenvectors of nv eigenvalues w
// (any subset, ascending) reusing the reduction left in ws.
// Calling thread shares the GPU with other problems' kernels (or runs two eigensolves side by side):
// avoid grid-wide software barriers. Returns the previous setting.
bool symeig_set_shared_gpu(bool on);
int symeig_values(int n, const double* A, int lda, int il, int iu, double* w, SymEigWork* ws,
                  int* status, cudaStream_t s);
int symeig_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, uint64_t seed,
                   double cluster_rel, cudaStream_t s);
// Lanczos estimate of the largest eigenvalue of a symmetric positive semidefinite n x n matrix A
// (n <= kLanczosMaxN: in one thread-block cluster with the matrix in shared memory; beyond: two
// launches per step, the matrix read from global memory): m steps of the three-term recurrence, then the
// two largest eigenvalues of the m x m tridiagonal and the last entry of the unit eigenvector of the
// largest. out (device, 4 doubles): theta_1, theta_2 (-DBL_MAX when m = 1), |z_m|, beta_m; the
// distance from theta_1 to an eigenvalue of A is at most beta_m |z_m|, and at most
// (beta_m z_m)^2 / (theta_1 - theta_2 - beta_m |z_m|) when that gap is positive. ws: carved for n.
constexpr int kLanczosMaxN = 256;
constexpr int kOzSmallMinN = 512;     // n from which K_W and G_W products run on the tensor cores
int lanczos_top(int n, const double* A, int lda, int m, uint64_t seed, SymEigWork* ws, double* out,
                cudaStream_t s);
// Orthonormalise the columns of Z (n x nv) against each other by Newton-Schulz steps
// Z <- Z (3 I - Z^T Z) / 2; tmp holds 2 * nv * nv + n * nv doubles.
int newton_schulz_f64(int n, int nv, double* Z, int ldz, int steps, double* tmp, double* partial,
                      size_t partial_cap, cudaStream_t s);

// ---------------------------------------------------------------- build kernels
int segment_labels(const int32_t* labels, int n, int k, int32_t* counts, int32_t* offsets,
                   int32_t* perm, int* status, cudaStream_t s);
int build_factors(const void* X, int x_dtype, int64_t d, int n, int64_t ldx, int k,
                  const int32_t* labels, const int32_t* counts, const int32_t* offsets,
                  const int32_t* perm, double* mu_j, double* mu, double* HW, double* HB,
                  int* status, cudaStream_t s);
int check_finite_f64(int64_t rows, int cols, const double* A, int64_t lda, int* status, cudaStream_t s);
// K = alpha I + W_s diag(alpha (phi(alpha lam_s) - 1)) W_s^T over the ns significant eigenpairs
// (lam_s, W_s) of the Gram; equal to alpha W diag(phi(alpha lam)) W^T because sum_i w_i w_i^T = I
// and phi(0) = 1. tmp: n * ns doubles.
int phi_operator(int n, int ns, const double* lam, const double* W, int ldw, double alpha,
                 double* K, double* tmp, cudaStream_t s);

// ---------------------------------------------------------------- exp-apply
struct ExpOp {
    const double* H;  // d x m (ld d)
    const double* K;  // m x m
    int m;
    const char* tag;  // region-timer name
};
// Y = X + H K (H^T X) for a d x b block with H and X in storage type T (double or float).
template <class T>
int exp_apply(int64_t d, const T* H, const double* K, int m, const char* tag, int b, const T* X, int64_t ldx, T* Y,
              int64_t ldy, double* P, double* Q, void* partial, size_t partial_cap, cudaStream_t s);
// Y = X + H K (H^T X) for a d x b block (FP64 sweeps).
int exp_apply_f64(int64_t d, const ExpOp& op, int b, const double* X, int64_t ldx, double* Y,
                  int64_t ldy, double* P, double* Q, double* partial, size_t partial_cap,
                  cudaStream_t s);

// ---------------------------------------------------------------- tensor-core exp-apply (bf16 H)
// One factor H (d x m) in the two pre-tiled bf16 layouts the tensor-core sweeps read: 128-row x
// 64-element tiles, each a contiguous 16 KB block in the 128-byte-swizzled shared-memory image.
struct TcFactor {
    const __nv_bfloat16* A1 = nullptr;    // bf16(H): tile rows = columns of H, K along d (sweep 1)
    const __nv_bfloat16* A2 = nullptr;    // bf16(H K(alpha)): tile rows = rows of H, K along m (sweep 2)
    int64_t d = 0, ldh = 0;               // ldh = d rounded up to 64
    int m = 0, ldm = 0;                   // ldm = m rounded up to 64
    // one-pass form (when bf16 B = H R^T, sign(alpha) K = R^T R, fits in the SMs' shared memory):
    // exp(alpha H H^T) X = X + fsign B (B^T X), B tiled for the resident kernel, fgrid CTAs
    const __nv_bfloat16* F = nullptr;
    float fsign = 0.f;
    int fgrid = 0;
};
// Per-handle staging buffers of the sweeps (bf16 hi/lo pairs of X and of P = H^T X, 32 columns
// each) with their tensor maps for N = 16 ([0]) and N = 32 ([1]) column boxes.
struct TcBuffers {
    CUtensorMap mapXh[2], mapXl[2], mapQh[2], mapQl[2];
    float* partial = nullptr;             // split-K partials of sweep 1
    size_t partial_cap = 0;               // in floats
    __nv_bfloat16 *Xhi = nullptr, *Xlo = nullptr, *Qhi = nullptr, *Qlo = nullptr;
    int64_t ldh = 0;
    int ldq = 0;
    // one-pass form: per-CTA partials of B^T X (fgrid x m x 32 floats), its grid barrier (arrival count
    // at fbar[0], the launch base at fbar[32], zeroed once) and the barrier's poll limit
    float* fpartial = nullptr;
    unsigned* fbar = nullptr;
    long long fspin = 0;
};
inline int64_t tc_pad_rows(int64_t d) { return (d + 63) / 64 * 64; }
inline int tc_pad_cols(int m) { return (m + 63) / 64 * 64; }
// Element counts of the two tiled layouts of a d x m factor.
int64_t tc_tiles_sweep1(int64_t d, int m);
int64_t tc_tiles_sweep2(int64_t d, int m);
// Tile an FP64 factor H (d x m, ld d) as bf16 for sweep 1 and form the tiled bf16(H K) for sweep 2 from
// K (m x m, FP64) on the tensor cores. Synchronises the stream (temporaries).
int tc_factor_make(const double* H, int64_t d, int m, const double* K, __nv_bfloat16* A1, __nv_bfloat16* A2,
                   TcFactor* f, int* status, cudaStream_t s);
// Floats of split-K partials needed for factors with at most m_max columns (two CTAs per SM).
size_t tc_partial_floats(int m_max);
int tc_buffers_make(int64_t ldh, int ldq, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, __nv_bfloat16* Qhi,
                    __nv_bfloat16* Qlo, float* partial, size_t partial_cap, TcBuffers* b);
// exp_apply_tc flags: the staging pair already holds the split of X (skip the split step); write the
// split of Y into the staging pair (for the next exp-apply). Both apply only when b <= 32.
enum : int { TC_X_SPLIT_READY = 1, TC_EMIT_SPLIT = 2 };
// One-pass form: CTAs of the resident kernel for a d x m factor (0 when it does not fit: m > 768, or more
// 128-row chunks than CTAs that can be resident at once); elements of its tiled image; floats of its
// partials for factors up to m_max columns; the image of B = H R^T for sign(alpha) K = R^T R (synchronises
// the stream); the product X + fsign B (B^T X) itself (b columns, in launches of at most 32).
int tc_fused_grid(int64_t d, int m);
int64_t tc_fused_elems(int64_t d, int m);
size_t tc_fused_partial_floats(int64_t d, int m_max);
int tc_fused_make(const double* H, int64_t d, int m, const double* K, double alpha, __nv_bfloat16* img, TcFactor* f,
                  int* status, cudaStream_t s);
int exp_apply_tc_fused(const TcFactor& f, const TcBuffers& bufs, int b, const float* X, int64_t ldx, float* Y,
                       int64_t ldy, int* status, cudaStream_t s);
// Y = X + H K (H^T X) with bf16 H on the tensor cores; X, Y single precision, Y may alias X. Uses the
// one-pass form when the factor has it.
int exp_apply_tc(const TcFactor& f, const TcBuffers& bufs, const char* tag, int b, const float* X, int64_t ldx,
                 float* Y, int64_t ldy, int flags, int* status, cudaStream_t s);

// ---------------------------------------------------------------- FP64-accurate products on the tensor cores
// An FP64 operand split once into kOzSlices bf16 digit planes with a power-of-two scale per M row
// (error-free splitting), each plane in the pre-tiled swizzled layout: M rows are the columns of the
// source matrix (operand of A^T B) or its rows (operand of A B), K runs along the reduction index.
constexpr int kOzSlices = 7;
struct OzOperand {
    __nv_bfloat16* tiles = nullptr;   // plane q at tiles + q * slice
    int64_t slice = 0;                // elements between planes
    int* exps = nullptr;              // M scale exponents
    int64_t M = 0, K = 0;
    int kbs = 0, mtiles = 0;          // 64-wide K tiles per 128-row band; bands
};
// Staging of the narrow operand (at most 32 columns, split on every call), its tensor map, and the
// split-K partial sums.
struct OzNarrow {
    CUtensorMap map;
    __nv_bfloat16* planes = nullptr;  // [7][32][ldmax]
    int* exps = nullptr;              // 32
    double* partial = nullptr;
    size_t pcap = 0;                  // doubles
    int64_t ldmax = 0, map_ld = 0;
};
size_t oz_operand_bytes(int64_t M, int64_t K);
// Split A (lda) into the operand: rows_are_cols = true: M = columns of A (d x M matrix, K = d rows);
// false: M = rows of A (M x K matrix). mem: oz_operand_bytes(M, K) bytes, 256-byte aligned.
// Splitting flags ST_NONFINITE in *status when it meets Inf or NaN.
int oz_operand_make(const double* A, int64_t lda, int64_t M, int64_t K, bool rows_are_cols, void* mem,
                    OzOperand* op, int* status, cudaStream_t s);
// A growing operand (the Krylov basis): room for Mcap rows and Kcap reduction values, planes zeroed.
// oz_append_cols: split columns i0 .. i1 of A (d x ., lda) as rows i0 .. i1 of a column-scaled operand
// (K = d). oz_resplit_rows: split all of A (M x K) afresh as a row-scaled operand (row scales over the K
// columns present).
int oz_operand_init(int64_t Mcap, int64_t Kcap, void* mem, OzOperand* op, cudaStream_t s);
int oz_append_cols(const double* A, int64_t lda, int i0, int i1, int64_t K, OzOperand* op, int* status,
                   cudaStream_t s);
int oz_resplit_rows(const double* A, int64_t lda, int64_t M, int64_t K, OzOperand* op, int* status, cudaStream_t s);
// Grow a row-scaled operand (made by oz_operand_init, grown only by this call) from k0 to k1 columns of A:
// new digits for the rows whose scale the new columns leave unchanged, a full re-split of the others.
// list: M + 1 ints of scratch.
int oz_grow_rows(const double* A, int64_t lda, int64_t M, int64_t k0, int64_t k1, OzOperand* op, int* list,
                 int* status, cudaStream_t s);
size_t oz_narrow_bytes(int64_t Kmax, int max_splits, int64_t Mmax);
int oz_narrow_make(int64_t Kmax, int max_splits, int64_t Mmax, void* mem, OzNarrow* nb);
// D (M x p, ldd) = alpha * op(A) B + beta * C0 (ldc0), op(A) the M x K split operand, B: K x p (ldb),
// p <= 32, in FP64 accuracy on the bf16 tensor cores. D may equal C0 (same ld).
int oz_gemm(const OzOperand& A, OzNarrow& nb, int p, const double* B, int64_t ldb, double alpha, double beta,
            const double* C0, int64_t ldc0, double* D, int64_t ldd, int* status, cudaStream_t s);

// D (A.M x B.M, ldd) = alpha A B^T + beta C0 for two split operands over the same K (both in the
// column-scaled layout: D_ij = sum_k A_ik B_jk), one launch over (128-row band of A, 32-row block of B).
// upper (A and B the same operand, beta = 0): only the blocks meeting the upper triangle are computed and
// the others mirrored; the product of an operand with itself is exactly symmetric. part (pcap doubles,
// optional): K-split partials, used when the output grid alone leaves SMs idle (not with upper).
int oz_gemm_tiled(const OzOperand& A, const OzOperand& B, double alpha, double beta, const double* C0, int64_t ldc0,
                  double* D, int64_t ldd, bool upper, int* status, cudaStream_t s, double* part = nullptr,
                  size_t pcap = 0);

// K(alpha) = alpha phi(alpha G) from G itself by scaling and squaring (dense products only), given
// lmax >= the largest eigenvalue of G. work: 6 m^2 doubles. With oz the m x m products run on the
// tensor cores: abuf and bbuf hold oz_operand_bytes(m, m) bytes each (the two factors' splits).
struct OzSquare {
    void* abuf = nullptr;
    void* bbuf = nullptr;
    int* status = nullptr;
};
int phi_by_squaring(int m, const double* G, double alpha, double lmax, double* K, double* work,
                    cudaStream_t s, const OzSquare* oz = nullptr);

}  // namespace eda

// The handle.
struct eda_ctx {
    int64_t d = 0, n = 0;
    int32_t k = 0;          // number of columns of H_B
    eda_config cfg{};
    double c2 = 0, lmax_w = 0, lmax_b = 0;
    double lmax_w_bound = 0;   // an upper bound of lambda_max(G_W) (lmax_w itself unless only estimated)
    // owned device memory
    void* block = nullptr;  // one allocation for everything below
    size_t block_bytes = 0;
    double *HW = nullptr, *HB = nullptr;   // adjacent: [H_W H_B] is one d x (n + k) matrix (ld d)
    int32_t *counts = nullptr, *offsets = nullptr, *perm = nullptr;
    double *mu_j = nullptr, *mu = nullptr;
    double *GW = nullptr, *GB = nullptr;
    double *evals_w = nullptr, *evals_b = nullptr;
    double *evecs_w = nullptr, *evecs_b = nullptr;
    double *KW = nullptr, *KB = nullptr;   // K(-c^2/2) for H_W, K(c^2) for H_B
    // single-precision copies of H_W, H_B for the mixed-precision solver (prec = EDA_F32), and
    // bf16 copies in the two tensor-core layouts (prec = EDA_BF16)
    void* block32 = nullptr;
    float *HW32 = nullptr, *HB32 = nullptr;
    eda::TcFactor tcW, tcB;
    eda::TcBuffers tcbuf;
    void* fblock = nullptr;                // the one-pass images of both factors, their partials, barrier
    int* status = nullptr;                 // device status word
    eda::GridBarrier bar{};
    size_t build_arena_off = 0;            // start of the build scratch inside `block`
    int nsig_first = 0;                    // scratch result of the last Gram eigensolve
    int nsig_w = 0, nsig_b = 0;            // significant eigenpairs kept for K_W, K_B
    bool eig_ready = false;                // evals / evecs hold the Grams' eigenpairs (computed on
                                           // demand when K came from scaling and squaring)
    // K(alpha) for an alpha other than the stored ones (allocated on first use)
    void* kblock = nullptr;
    double *Kalpha = nullptr, *Kalpha_tmp = nullptr;
    // cross Grams G_WB = H_W^T H_B (n x k) and G_BW = its transpose, for the composed FP64 M-apply of
    // the mixed-precision refinement (allocated on first use)
    void* xblock = nullptr;
    double *GWB = nullptr, *GBW = nullptr;
    // prec = EDA_F64_TC: Z = [H_W H_B] split for Z^T Y (ozT) and for Z U (ozN), and the narrow staging
    void* ozblock = nullptr;
    eda::OzOperand ozT, ozN;
    eda::OzNarrow oznb;
    // prec = EDA_F64_TC and n >= kOzSmallMinN: the left-factor split of the scaling and squaring that
    // forms K_W (and, for the nonsymmetric form, K(-c^2) and K(+c^2)), then K_W and G_W split for
    // their products with the n x p coordinates inside the composed M-apply and the recovery
    void* ozsmall = nullptr;
    eda::OzOperand ozKW, ozGW;
    // K(-c^2) and K(+c^2) for H_W, the operators of the nonsymmetric form exp(-c^2 S_W) exp(c^2 S_B) and of
    // exp(c^2 S_W) (allocated on first use by the Arnoldi solver)
    void* nblock = nullptr;
    double *KWm = nullptr, *KWp = nullptr;
    // solve workspace (grown on demand)
    void* ws = nullptr;
    size_t ws_bytes = 0;
};

namespace eda {
// Grow the handle's solve workspace to at least `bytes` (contents are not preserved).
int ensure_workspace(eda_ctx* h, size_t bytes);
// The two sweeps over Z = [H_W H_B] of a composed product (FP64, or the tensor-core FP64 products when the
// handle was built with EDA_F64_TC): PQ = Z^T Y, and OUT = Y + Z U.
int sweep_zt(eda_ctx* h, int p, const double* Y, int64_t ldy, double* PQ, double* part, size_t pcap, cudaStream_t s);
int sweep_z(eda_ctx* h, int p, const double* U, const double* Y, int64_t ldy, double* OUT, int64_t ldo,
            cudaStream_t s);
// The nonsymmetric operator of Eq. (3.1): NY = exp(-c^2 S_W) exp(c^2 S_B) Y in composed form; PQ, U: (n + k) x p;
// ZtY ((n + k) x p, optional) receives Z^T Y.
int n_apply_composed(eda_ctx* h, int p, const double* Y, int64_t ldy, double* NY, int64_t ldn, double* PQ, double* U,
                     double* ZtY, double* part, size_t pcap, cudaStream_t s);
// K(-c^2) and K(+c^2) of H_W (and the cross Grams) for the nonsymmetric form.
int ensure_n_operators(eda_ctx* h, cudaStream_t s);
// Form the cross Grams G_WB, G_BW of the handle if they are not there yet.
int ensure_cross_gram(eda_ctx* h, double* part, size_t pcap, cudaStream_t s);
}  // namespace eda
