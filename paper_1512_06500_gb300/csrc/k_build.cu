// Build step: class segmentation, centroids and the scatter factors H_W, H_B (Eq. eqn1, eqn2),
// finite checks, and the small operator K(alpha) = alpha phi(alpha G) of Theorem 3.1.
#include "eda_internal.cuh"

#include <cmath>

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

}  // namespace eda
