// Build step: class segmentation, centroids and the scatter factors H_W, H_B (Eqs. (1.1), (1.2)),
// finite checks, and the small operator K(alpha) = alpha phi(alpha G) of Theorem 3.1.
#include "eda_internal.cuh"

#include <algorithm>
#include <cmath>
#include <utility>

namespace eda {

namespace {

// Counts, offsets and a stable class-major permutation. One CTA; the scatter is done by warp 0
// in input order, 32 samples at a time, with equal labels ranked by lane order.
__global__ void k_segment(const int32_t* __restrict__ labels, int n, int k, int32_t* counts, int32_t* offsets,
                          int32_t* perm, int* status) {
    extern __shared__ int cnt[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) cnt[j] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = labels[i];
        if (l < 0 || l >= k) atomicOr(status, ST_BADLABEL);
        else atomicAdd(&cnt[l], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int off = 0;
        for (int j = 0; j < k; ++j) {
            offsets[j] = off;
            counts[j] = cnt[j];
            if (cnt[j] == 0) atomicOr(status, ST_EMPTYCLASS);
            off += cnt[j];
        }
        offsets[k] = off;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = lane; j < k; j += 32) cnt[j] = offsets[j];
        __syncwarp();
        const unsigned lt = (1u << lane) - 1u;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            int l = (i < n) ? labels[i] : -1;
            if (l < 0 || l >= k) l = -1;
            const unsigned mask = __match_any_sync(0xffffffffu, l);
            const int leader = __ffs(mask) - 1;
            const int rank = __popc(mask & lt);
            int b0 = 0;
            if (lane == leader && l >= 0) b0 = cnt[l];
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (l >= 0) perm[b0 + rank] = i;
            __syncwarp();
            if (lane == leader && l >= 0) cnt[l] = b0 + __popc(mask);
            __syncwarp();
        }
    }
}

template <class T>
__device__ __forceinline__ double ld_sample(const T* X, int64_t ldx, int i, int64_t p) {
    return (double)X[(int64_t)i * ldx + p];
}

// mu_j[j][p] = (sum over class-j samples in input order) / n_j, single IEEE operations only.
template <class T>
__global__ void k_class_means(const T* __restrict__ X, int64_t d, int64_t ldx, const int32_t* __restrict__ counts,
                              const int32_t* __restrict__ offsets, const int32_t* __restrict__ perm,
                              double* __restrict__ mu_j) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= d) return;
    double acc = 0.0;
    for (int q = offsets[j]; q < offsets[j + 1]; ++q) acc = __dadd_rn(acc, ld_sample(X, ldx, perm[q], p));
    mu_j[(int64_t)j * d + p] = __ddiv_rn(acc, (double)counts[j]);
}

template <class T>
__global__ void k_global_mean(const T* __restrict__ X, int64_t d, int64_t ldx, int n, double* __restrict__ mu) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= d) return;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc = __dadd_rn(acc, ld_sample(X, ldx, i, p));
    mu[p] = __ddiv_rn(acc, (double)n);
}

// H_W[:, q] = chi_{perm[q]} - mu_{label}
template <class T>
__global__ void k_build_hw(const T* __restrict__ X, int64_t d, int64_t ldx, int n, const int32_t* __restrict__ labels,
                           const int32_t* __restrict__ perm, const double* __restrict__ mu_j, double* __restrict__ HW) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (p >= d) return;
    const int i = perm[q];
    const int l = labels[i];
    HW[(int64_t)q * d + p] = __dsub_rn(ld_sample(X, ldx, i, p), mu_j[(int64_t)l * d + p]);
}

// H_B[:, j] = sqrt(n_j) (mu_j - mu)
__global__ void k_build_hb(int64_t d, const int32_t* __restrict__ counts, const double* __restrict__ mu_j,
                           const double* __restrict__ mu, double* __restrict__ HB) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= d) return;
    const double s = __dsqrt_rn((double)counts[j]);
    HB[(int64_t)j * d + p] = __dmul_rn(s, __dsub_rn(mu_j[(int64_t)j * d + p], mu[p]));
}

template <class T>
__global__ void k_check_finite(int64_t rows, int cols, const T* __restrict__ A, int64_t lda, int* status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = rows * cols;
    bool bad = false;
    for (int64_t x = e; x < tot; x += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)A[(x / rows) * lda + (x % rows)];
        if (!isfinite(v)) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// tmp[:, s] = coef_s W[:, first + s],  coef_s = alpha (phi(alpha lam_s) - 1),  phi(z) = expm1(z) / z.
__global__ void k_phi_scale(int n, int ns, const double* __restrict__ lam, const double* __restrict__ W, int ldw,
                            double alpha, double* __restrict__ tmp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * ns) return;
    const int i = (int)(e % n), s = (int)(e / n);
    const double z = alpha * fmax(lam[s], 0.0);
    const double phim1 = (z == 0.0) ? 0.0 : expm1(z) / z - 1.0;
    tmp[(int64_t)s * n + i] = alpha * phim1 * W[(int64_t)s * ldw + i];
}

__global__ void k_add_diag(int n, double alpha, double* K) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) K[(int64_t)i * n + i] += alpha;
}

// D = c0 I + c1 P1 + c2 P2 + c3 P3 (m x m, ld m); a null P contributes nothing.
__global__ void k_lincomb4(int m, double c0, double c1, const double* P1, double c2, const double* P2, double c3,
                           const double* P3, double* D) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    double v = (i == j) ? c0 : 0.0;
    if (P1) v = fma(c1, P1[e], v);
    if (P2) v = fma(c2, P2[e], v);
    if (P3) v = fma(c3, P3[e], v);
    D[e] = v;
}

// D = a S (m x m)
__global__ void k_scale_sq(int m, double a, const double* S, double* D) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)m * m) D[e] = a * S[e];
}

}  // namespace

int segment_labels(const int32_t* labels, int n, int k, int32_t* counts, int32_t* offsets, int32_t* perm,
                   int* status, cudaStream_t s) {
    const size_t smem = (size_t)k * sizeof(int);
    if (smem > 48 * 1024) return EDA_ERR_INVALID_ARG;
    k_segment<<<1, 1024, smem, s>>>(labels, n, k, counts, offsets, perm, status);
    EDA_LAUNCHED();
    return EDA_OK;
}

int build_factors(const void* X, int x_dtype, int64_t d, int n, int64_t ldx, int k, const int32_t* labels,
                  const int32_t* counts, const int32_t* offsets, const int32_t* perm, double* mu_j, double* mu,
                  double* HW, double* HB, int* status, cudaStream_t s) {
    const int tb = 256;
    const dim3 gk(ceil_div(d, tb), k), g1(ceil_div(d, tb)), gn(ceil_div(d, tb), n);
    if (x_dtype == EDA_F64) {
        const double* x = static_cast<const double*>(X);
        k_check_finite<<<std::min(ceil_div(d * n, tb), 4096), tb, 0, s>>>(d, n, x, ldx, status);
        EDA_LAUNCHED();
        k_class_means<<<gk, tb, 0, s>>>(x, d, ldx, counts, offsets, perm, mu_j);
        EDA_LAUNCHED();
        k_global_mean<<<g1, tb, 0, s>>>(x, d, ldx, n, mu);
        EDA_LAUNCHED();
        k_build_hw<<<gn, tb, 0, s>>>(x, d, ldx, n, labels, perm, mu_j, HW);
        EDA_LAUNCHED();
    } else if (x_dtype == EDA_F32) {
        const float* x = static_cast<const float*>(X);
        k_check_finite<<<std::min(ceil_div(d * n, tb), 4096), tb, 0, s>>>(d, n, x, ldx, status);
        EDA_LAUNCHED();
        k_class_means<<<gk, tb, 0, s>>>(x, d, ldx, counts, offsets, perm, mu_j);
        EDA_LAUNCHED();
        k_global_mean<<<g1, tb, 0, s>>>(x, d, ldx, n, mu);
        EDA_LAUNCHED();
        k_build_hw<<<gn, tb, 0, s>>>(x, d, ldx, n, labels, perm, mu_j, HW);
        EDA_LAUNCHED();
    } else {
        return EDA_ERR_INVALID_ARG;
    }
    k_build_hb<<<gk, tb, 0, s>>>(d, counts, mu_j, mu, HB);
    EDA_LAUNCHED();
    return EDA_OK;
}

int check_finite_f64(int64_t rows, int cols, const double* A, int64_t lda, int* status, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return EDA_OK;
    k_check_finite<<<std::min(ceil_div(rows * cols, 256), 4096), 256, 0, s>>>(rows, cols, A, lda, status);
    EDA_LAUNCHED();
    return EDA_OK;
}

int phi_operator(int n, int ns, const double* lam, const double* W, int ldw, double alpha, double* K, double* tmp,
                 cudaStream_t s) {
    if (ns > 0) {
        k_phi_scale<<<ceil_div((int64_t)n * ns, 256), 256, 0, s>>>(n, ns, lam, W, ldw, alpha, tmp);
        EDA_LAUNCHED();
        EDA_TRY(gemm_small_f64(false, true, n, n, ns, 1.0, tmp, n, W, ldw, 0.0, K, n, s));
    } else {
        EDA_CUDA_TRY(cudaMemsetAsync(K, 0, (size_t)n * n * sizeof(double), s));
    }
    k_add_diag<<<ceil_div(n, 256), 256, 0, s>>>(n, alpha, K);
    EDA_LAUNCHED();
    return EDA_OK;
}


// K(alpha) = alpha phi(alpha G) of a symmetric positive semidefinite Gram G (m x m) without its
// eigenvectors, for matrices small enough that a few dense products cost less than the eigensolver's
// sequential steps. With B = alpha G / 2^s, s the least integer with |alpha| lambda_max / 2^s <= 1:
// phi(B) = sum_{k=0}^{17} B^k / (k+1)! (the first omitted term is below 1/19! < 2^-56 for ||B|| <= 1),
// evaluated in Paterson-Stockmeyer form in the powers B, B^2, B^3 and B^4; e^B = I + B phi(B); then s
// doublings phi(2B) = phi(B) (I + e^B) / 2 and e^(2B) = (e^B)^2. Every factor is a polynomial in G, so
// all products commute in exact arithmetic; the result is symmetrised. 7 + 2 s dense m x m x m
// products, on the FP64 pipe or, given oz, as FP64-accurate tensor-core products (both factors split, by
// columns: D_ij = sum_k A_ki B_kj, and A is symmetric, so this is (A B)_ij). work: 6 m^2 doubles.
int phi_by_squaring(int m, const double* G, double alpha, double lmax, double* K, double* work, cudaStream_t s,
                    const OzSquare* oz) {
    if (m <= 0) return EDA_OK;
    const size_t mm = (size_t)m * m;
    const int eb = ceil_div((int64_t)mm, 256);
    const double rho = fabs(alpha) * std::max(lmax, 0.0);
    int sq = 0;
    while (sq < 60 && std::ldexp(rho, -sq) > 1.0) ++sq;
    double c[20];
    {
        double f = 1.0;
        for (int k = 0; k < 20; ++k) {
            f *= (double)(k + 1);
            c[k] = 1.0 / f;                          // 1 / (k+1)!
        }
    }
    double* P1 = work;
    double* P2 = work + mm;
    double* P3 = work + 2 * mm;
    double* P4 = work + 3 * mm;
    double* F = work + 4 * mm;
    double* T = work + 5 * mm;
    // C = alpha A B + beta C
    auto mulab = [&](double alpha_, const double* A, const double* B, double beta, double* C) -> int {
        if (!oz) return gemm_small_f64(false, false, m, m, m, alpha_, A, m, B, m, beta, C, m, s);
        OzOperand oa, ob;
        EDA_TRY(oz_operand_make(A, m, m, m, true, oz->abuf, &oa, oz->status, s));
        EDA_TRY(oz_operand_make(B, m, m, m, true, oz->bbuf, &ob, oz->status, s));
        return oz_gemm_tiled(oa, ob, alpha_, beta, beta != 0.0 ? C : nullptr, m, C, m, false, oz->status, s);
    };
    auto mul = [&](const double* A, const double* B, double beta, double* C) { return mulab(1.0, A, B, beta, C); };
    k_scale_sq<<<eb, 256, 0, s>>>(m, std::ldexp(alpha, -sq), G, P1);
    EDA_LAUNCHED();
    EDA_TRY(mul(P1, P1, 0.0, P2));
    EDA_TRY(mul(P2, P1, 0.0, P3));
    EDA_TRY(mul(P3, P1, 0.0, P4));
    // Horner in B^4 over the blocks c_{4i} .. c_{4i+3}, i = 4 (c_16, c_17) down to 0
    k_lincomb4<<<eb, 256, 0, s>>>(m, c[16], c[17], P1, 0.0, nullptr, 0.0, nullptr, F);
    EDA_LAUNCHED();
    for (int i = 3; i >= 0; --i) {
        k_lincomb4<<<eb, 256, 0, s>>>(m, c[4 * i], c[4 * i + 1], P1, c[4 * i + 2], P2, c[4 * i + 3], P3, T);
        EDA_LAUNCHED();
        EDA_TRY(mul(F, P4, 1.0, T));               // T = F B^4 + Q_i
        std::swap(F, T);
    }
    // E = I + B phi(B) (in P2; B^2 and B^3 are no longer needed)
    double* E = P2;
    double* E2 = P3;
    k_lincomb4<<<eb, 256, 0, s>>>(m, 1.0, 0.0, nullptr, 0.0, nullptr, 0.0, nullptr, E);
    EDA_LAUNCHED();
    EDA_TRY(mul(P1, F, 1.0, E));
    for (int q = 0; q < sq; ++q) {
        k_scale_sq<<<eb, 256, 0, s>>>(m, 0.5, F, T);
        EDA_LAUNCHED();
        EDA_TRY(mulab(0.5, F, E, 1.0, T));                                                 // phi(2B)
        std::swap(F, T);
        if (q + 1 < sq) {
            EDA_TRY(mul(E, E, 0.0, E2));                                                   // e^(2B)
            std::swap(E, E2);
        }
    }
    k_scale_sq<<<eb, 256, 0, s>>>(m, alpha, F, K);
    EDA_LAUNCHED();
    return symmetrize_f64(m, K, m, s);
}

}  // namespace eda
