// FP64 dense building blocks of the Krylov solver: tall-skinny products with a deterministic
// split-K reduction, small products, Cholesky with inverse, and seeded Gaussian blocks.
#include "eda_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>

namespace eda {

namespace {

constexpr int TN_KB = 32;       // rows of A/B staged per pass
constexpr int TN_TM = 32;       // output tile rows
constexpr int TN_THREADS = 256;

// Tile (bx, by) with bx >= by of the lower triangle of a T x T tile grid from its index
// q = bx (bx + 1) / 2 + by (row by row).
__device__ __forceinline__ void tri_tile(int q, int& bx, int& by) {
    int x = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
    while ((x + 1) * (x + 2) / 2 <= q) ++x;
    while (x * (x + 1) / 2 > q) --x;
    bx = x;
    by = q - x * (x + 1) / 2;
}

// partial[s][j][i] = sum over rows r of split s of A[r, i0+i] * B[r, j0+j]. SYM (A = B, m = p, TP = TN_TM):
// only the tiles with i0 >= j0 are launched (blockIdx.x runs over the lower triangle of the tile grid);
// a diagonal tile computes entries (i, j) and (j, i) from the same products in the same order, so it is
// exactly symmetric.
template <int TP, class T, bool SYM = false>
__global__ void __launch_bounds__(TN_THREADS) k_gemm_tn_partial(int64_t d, int m, int p, const T* __restrict__ A,
                                                                int64_t lda, const T* __restrict__ B, int64_t ldb,
                                                                int64_t rows_per_split, T* __restrict__ partial) {
    __shared__ T As[TN_KB][TN_TM + 1];
    __shared__ T Bs[TN_KB][TP + 1];
    int bx = blockIdx.x, by = blockIdx.y;
    if (SYM) tri_tile(blockIdx.x, bx, by);
    const int i0 = bx * TN_TM;
    const int j0 = by * TP;
    const int s = blockIdx.z;
    const int64_t r_begin = (int64_t)s * rows_per_split;
    const int64_t r_end = min(d, r_begin + rows_per_split);
    // thread -> outputs: TM*TP outputs over 256 threads
    constexpr int OUT = TN_TM * TP / TN_THREADS;      // 1 (TP=8), 2 (TP=16), 4 (TP=32)
    constexpr int TPT = (TP >= 16) ? 2 : 1;           // columns per thread
    constexpr int TMT = OUT / TPT;                    // rows per thread
    const int tx = threadIdx.x % (TN_TM / TMT);       // row group
    const int ty = threadIdx.x / (TN_TM / TMT);       // column group
    T acc[TMT][TPT];
#pragma unroll
    for (int a = 0; a < TMT; ++a)
#pragma unroll
        for (int b = 0; b < TPT; ++b) acc[a][b] = T(0);

    // the next chunk of rows is read into registers while the current one is multiplied, so the
    // global-memory latency overlaps the FP64 work (the products and their order are unchanged)
    constexpr int PA = TN_KB * TN_TM / TN_THREADS;                  // A elements per thread and chunk
    constexpr int PB = (TN_KB * TP + TN_THREADS - 1) / TN_THREADS;  // B elements per thread and chunk
    T ra[PA], rb[PB];
    auto fetch = [&](int64_t r0) {
#pragma unroll
        for (int q = 0; q < PA; ++q) {
            const int e = threadIdx.x + q * TN_THREADS;
            const int rr = e % TN_KB, cc = e / TN_KB;
            const int64_t r = r0 + rr;
            const int c = i0 + cc;
            ra[q] = (r < r_end && c < m) ? A[(int64_t)c * lda + r] : T(0);
        }
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int e = threadIdx.x + q * TN_THREADS;
            const int rr = e % TN_KB, cc = e / TN_KB;
            const int64_t r = r0 + rr;
            const int c = j0 + cc;
            rb[q] = (e < TN_KB * TP && r < r_end && c < p) ? B[(int64_t)c * ldb + r] : T(0);
        }
    };
    if (r_begin < r_end) fetch(r_begin);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += TN_KB) {
        // stage A rows r0..r0+KB of columns i0..i0+TM and the matching rows of B
#pragma unroll
        for (int q = 0; q < PA; ++q) {
            const int e = threadIdx.x + q * TN_THREADS;
            As[e % TN_KB][e / TN_KB] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < PB; ++q) {
            const int e = threadIdx.x + q * TN_THREADS;
            if (e < TN_KB * TP) Bs[e % TN_KB][e / TN_KB] = rb[q];
        }
        __syncthreads();
        if (r0 + TN_KB < r_end) fetch(r0 + TN_KB);
#pragma unroll 8
        for (int rr = 0; rr < TN_KB; ++rr) {
            T av[TMT], bv[TPT];
#pragma unroll
            for (int a = 0; a < TMT; ++a) av[a] = As[rr][tx + a * (TN_TM / TMT)];
#pragma unroll
            for (int b = 0; b < TPT; ++b) bv[b] = Bs[rr][ty + b * (TP / TPT)];
#pragma unroll
            for (int a = 0; a < TMT; ++a)
#pragma unroll
                for (int b = 0; b < TPT; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    T* out = partial + (int64_t)s * m * p;
#pragma unroll
    for (int a = 0; a < TMT; ++a)
#pragma unroll
        for (int b = 0; b < TPT; ++b) {
            const int i = i0 + tx + a * (TN_TM / TMT);
            const int j = j0 + ty + b * (TP / TPT);
            if (i < m && j < p) out[(int64_t)j * m + i] = acc[a][b];
        }
}

// C[i, j] = alpha * sum_s partial[s][j][i] + beta * C[i, j]. Small split counts: one thread per
// output, splits summed in order. Large split counts: one warp per output, lane l sums splits
// l, l + 32, ... in order, then a fixed butterfly across lanes (deterministic either way).
// SYM: only entries with i >= j are summed; each is written to (i, j) and mirrored to (j, i).
__device__ __forceinline__ void tn_store(double* C, int ldc, int i, int j, double acc, double alpha, double beta,
                                         bool sym) {
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, C[(int64_t)j * ldc + i], v);
    C[(int64_t)j * ldc + i] = v;
    if (sym && i != j) {
        double w = alpha * acc;
        if (beta != 0.0) w = fma(beta, C[(int64_t)i * ldc + j], w);
        C[(int64_t)i * ldc + j] = w;
    }
}

template <class T>
__global__ void k_gemm_tn_reduce(int m, int p, int splits, const T* __restrict__ partial, double alpha,
                                 double beta, double* __restrict__ C, int ldc, bool sym) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * p) return;
    const int i = (int)(e % m), j = (int)(e / m);
    if (sym && i < j) return;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)partial[(int64_t)s * m * p + e];
    tn_store(C, ldc, i, j, acc, alpha, beta, sym);
}

template <class T>
__global__ void k_gemm_tn_reduce_warp(int m, int p, int splits, const T* __restrict__ partial, double alpha,
                                      double beta, double* __restrict__ C, int ldc, bool sym) {
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= (int64_t)m * p) return;
    const int i = (int)(e % m), j = (int)(e / m);
    if (sym && i < j) return;
    const int64_t mp = (int64_t)m * p;
    double a0 = 0.0, a1 = 0.0;
    int s = lane;
    for (; s + 32 < splits; s += 64) {
        a0 += (double)partial[(int64_t)s * mp + e];
        a1 += (double)partial[(int64_t)(s + 32) * mp + e];
    }
    if (s < splits) a0 += (double)partial[(int64_t)s * mp + e];
    double acc = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) tn_store(C, ldc, i, j, acc, alpha, beta, sym);
}

// C[r, c] = beta * C0[r, c] + alpha * sum_l A[r, l] B[l, c] for tall A (d x m) and small B
// (m x p). A CTA owns 32 rows and NC columns; its eight warps (two per SM sub-partition, so that
// one issues FP64 work while the other waits on a load) split the inner dimension into eighths,
// each thread keeps NC independent accumulators, the slice of B sits in shared memory, and the
// partial sums of the eighths are added in a fixed pairwise order at the end. For an upper
// triangular B (ub) each warp stops at row c0 + NC of B, below which the CTA's columns are zero: the
// partition of the inner dimension is unchanged and only exact zero terms are left out.
template <int NC, class T>
__global__ void __launch_bounds__(256) k_gemm_nn(int64_t d, int m, int p, double alpha, const T* __restrict__ A,
                                                 int64_t lda, const double* __restrict__ B, int ldb, double beta,
                                                 const T* C0, int64_t ldc0, T* C, int64_t ldc, int ub) {
    constexpr int LCH = 256;                 // rows of B staged per pass
    __shared__ T Bs[LCH][NC];
    __shared__ T red[7][32][NC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * 32 + lane;
    const int c0 = blockIdx.y * NC;
    const int nc = min(NC, p - c0);
    const int lim = ub ? min(m, c0 + NC) : m;   // rows of B that can be nonzero in these columns
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    const bool live = r < d;
    const T* Ar = A + (live ? r : 0);
    for (int l0 = 0; l0 < m; l0 += LCH) {
        const int lc = min(LCH, m - l0);
        __syncthreads();
        for (int e = threadIdx.x; e < lc * NC; e += blockDim.x) {
            const int l = e / NC, c = e % NC;
            Bs[l][c] = (c < nc) ? (T)B[(int64_t)(c0 + c) * ldb + l0 + l] : T(0);
        }
        __syncthreads();
        const int q = (lc + 7) / 8;
        const int lb = w * q, le = min(min(lc, lb + q), lim - l0);
        int l = lb;
        // groups of four rows of A, the next group read while the current one is multiplied
        T a[4];
        if (l + 3 < le) {
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = live ? Ar[(int64_t)(l0 + l + u) * lda] : T(0);
        }
        for (; l + 3 < le; l += 4) {
            T an[4];
            const bool more = l + 7 < le;
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; ++u) an[u] = live ? Ar[(int64_t)(l0 + l + 4 + u) * lda] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < NC; ++c) acc[c] = fma(a[u], Bs[l + u][c], acc[c]);
            if (more) {
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = an[u];
            }
        }
        for (; l < le; ++l) {
            const T a0 = live ? Ar[(int64_t)(l0 + l) * lda] : T(0);
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fma(a0, Bs[l][c], acc[c]);
        }
    }
    if (w > 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) red[w - 1][lane][c] = acc[c];
    }
    __syncthreads();
    if (w > 0 || !live) return;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c >= nc) break;
        const T sum = ((acc[c] + red[0][lane][c]) + (red[1][lane][c] + red[2][lane][c])) +
                      ((red[3][lane][c] + red[4][lane][c]) + (red[5][lane][c] + red[6][lane][c]));
        T v = (T)alpha * sum;
        if (beta != 0.0) v = fma((T)beta, C0[(int64_t)(c0 + c) * ldc0 + r], v);
        C[(int64_t)(c0 + c) * ldc + r] = v;
    }
}

// Small C (m x p) = alpha A B + beta C (both operands untransposed) with a long inner dimension:
// CTA = 8 warps for one (32-row block, column); warp w sums its eighth of the inner dimension with
// eight independent chains (eight loads of A in flight per lane: at these sizes the product is bound
// by load latency, then by the FP64 pipe), and the eighths are added in a fixed order through shared
// memory.
constexpr int kSplitkWarps = 8;
__global__ void __launch_bounds__(32 * kSplitkWarps) k_gemm_small_nn_splitk(int m, int p, int kk, double alpha,
                                                                           const double* __restrict__ A, int lda,
                                                                           const double* __restrict__ B, int ldb,
                                                                           double beta, double* __restrict__ C,
                                                                           int ldc) {
    __shared__ double part[kSplitkWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y;
    const int q = (kk + kSplitkWarps - 1) / kSplitkWarps;
    const int lb = w * q, le = min(kk, lb + q);
    double a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) a[u] = 0.0;
    if (i < m) {
        const double* Bj = B + (int64_t)j * ldb;
        int l = lb;
        for (; l + 7 < le; l += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = fma(A[(int64_t)(l + u) * lda + i], Bj[l + u], a[u]);
        }
        for (; l < le; ++l) a[0] = fma(A[(int64_t)l * lda + i], Bj[l], a[0]);
    }
    part[w][lane] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    __syncthreads();
    if (w == 0 && i < m) {
        const double acc = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                           ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
        double v = alpha * acc;
        if (beta != 0.0) v = fma(beta, C[(int64_t)j * ldc + i], v);
        C[(int64_t)j * ldc + i] = v;
    }
}

__global__ void k_gemm_small(bool ta, bool tb, int m, int p, int kk, double alpha, const double* __restrict__ A,
                             int lda, const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
                             int ldc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= m || j >= p) return;
    double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
    int l = 0;
    for (; l + 3 < kk; l += 4) {
        if (ta) {
            acc0 = fma(A[(int64_t)i * lda + l], tb ? B[(int64_t)l * ldb + j] : B[(int64_t)j * ldb + l], acc0);
            acc1 = fma(A[(int64_t)i * lda + l + 1], tb ? B[(int64_t)(l + 1) * ldb + j] : B[(int64_t)j * ldb + l + 1], acc1);
            acc2 = fma(A[(int64_t)i * lda + l + 2], tb ? B[(int64_t)(l + 2) * ldb + j] : B[(int64_t)j * ldb + l + 2], acc2);
            acc3 = fma(A[(int64_t)i * lda + l + 3], tb ? B[(int64_t)(l + 3) * ldb + j] : B[(int64_t)j * ldb + l + 3], acc3);
        } else {
            acc0 = fma(A[(int64_t)l * lda + i], tb ? B[(int64_t)l * ldb + j] : B[(int64_t)j * ldb + l], acc0);
            acc1 = fma(A[(int64_t)(l + 1) * lda + i], tb ? B[(int64_t)(l + 1) * ldb + j] : B[(int64_t)j * ldb + l + 1], acc1);
            acc2 = fma(A[(int64_t)(l + 2) * lda + i], tb ? B[(int64_t)(l + 2) * ldb + j] : B[(int64_t)j * ldb + l + 2], acc2);
            acc3 = fma(A[(int64_t)(l + 3) * lda + i], tb ? B[(int64_t)(l + 3) * ldb + j] : B[(int64_t)j * ldb + l + 3], acc3);
        }
    }
    for (; l < kk; ++l) {
        const double a = ta ? A[(int64_t)i * lda + l] : A[(int64_t)l * lda + i];
        const double b = tb ? B[(int64_t)l * ldb + j] : B[(int64_t)j * ldb + l];
        acc0 = fma(a, b, acc0);
    }
    double v = alpha * ((acc0 + acc1) + (acc2 + acc3));
    if (beta != 0.0) v = fma(beta, C[(int64_t)j * ldc + i], v);
    C[(int64_t)j * ldc + i] = v;
}

// Single-CTA right-looking upper Cholesky G = R^T R with rank detection, then R^{-1}.
// The same factorisation for b <= 32 by one warp with the matrix in shared memory: lane c owns
// column c; one reciprocal per pivot; warp-level synchronisation only. Rank decisions (threshold,
// lost list in pivot order, status bits) are those of k_chol_inv.
__global__ void __launch_bounds__(32) k_chol_inv_warp(int b, double* G, int ldg, double* Rinv, double rank_tol,
                                                      double piv_min2, int* status, int* lost) {
    __shared__ double sg[32][33];   // sg[c][r] = G[r, c]
    __shared__ double sx[32][33];   // sx[c][i] = Rinv[i, c]
    __shared__ double inv[32];
    const int lane = threadIdx.x;
    const bool live = lane < b;
    if (live)
        for (int r = 0; r <= lane; ++r) sg[lane][r] = G[(int64_t)lane * ldg + r];
    double dg = live ? G[(int64_t)lane * ldg + lane] : 0.0;
    const bool bad = live && !isfinite(dg);
    double mx = fabs(dg);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_NONFINITE);
    const double thr = fmax(rank_tol * mx, piv_min2);
    int nlost = 0;
    __syncwarp();
    for (int j = 0; j < b; ++j) {
        const double g = sg[j][j];
        const bool lost_j = !(g > thr) || mx == 0.0;
        const double piv = lost_j ? 0.0 : sqrt(g);
        const double ip = lost_j ? 0.0 : 1.0 / piv;
        __syncwarp();   // every lane has read the pivot before lane 0 overwrites it
        if (lane == 0) {
            if (lost_j) {
                if (lost) lost[nlost] = j;
                atomicOr(status, ST_RANKLOSS);
            }
            sg[j][j] = piv;
            inv[j] = ip;
        }
        nlost += lost_j ? 1 : 0;
        // row j of R (entries (j, c) for c > j), then the trailing update of column c
        if (live && lane > j) sg[lane][j] *= ip;
        __syncwarp();
        if (live && lane > j) {
            const double rjc = sg[lane][j];
            for (int c1 = j + 1; c1 <= lane; ++c1) sg[lane][c1] -= sg[c1][j] * rjc;
        }
        __syncwarp();
    }
    // Rinv = R^{-1} (upper triangular): lane c solves R x = e_c from the bottom up
    if (live) {
        const int c = lane;
        for (int i = b - 1; i > c; --i) sx[c][i] = 0.0;
        for (int i = c; i >= 0; --i) {
            double a0 = (i == c) ? 1.0 : 0.0, a1 = 0.0;
            int l = i + 1;
            for (; l + 1 <= c; l += 2) {
                a0 -= sg[l][i] * sx[c][l];
                a1 -= sg[l + 1][i] * sx[c][l + 1];
            }
            if (l <= c) a0 -= sg[l][i] * sx[c][l];
            sx[c][i] = (a0 + a1) * inv[i];
        }
    }
    __syncwarp();
    if (live) {
        for (int r = 0; r < b; ++r) {
            G[(int64_t)lane * ldg + r] = (r <= lane) ? sg[lane][r] : 0.0;
            Rinv[(int64_t)lane * b + r] = sx[lane][r];
        }
    }
    if (lane == 0 && lost) lost[b] = nlost;
}

__global__ void k_chol_inv(int b, double* G, int ldg, double* Rinv, double rank_tol, double piv_min2, int* status,
                           int* lost) {
    __shared__ double maxdiag;
    __shared__ int nlost;
    __shared__ double piv;
    if (threadIdx.x == 0) {
        double mx = 0.0;
        bool bad = false;
        for (int j = 0; j < b; ++j) {
            const double g = G[(int64_t)j * ldg + j];
            if (!isfinite(g)) bad = true;
            mx = fmax(mx, fabs(g));
        }
        maxdiag = mx;
        nlost = 0;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    __syncthreads();
    const double thr = fmax(rank_tol * maxdiag, piv_min2);
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            const double g = G[(int64_t)j * ldg + j];
            if (!(g > thr) || maxdiag == 0.0) {
                piv = 0.0;
                if (lost) lost[nlost] = j;
                nlost++;
                atomicOr(status, ST_RANKLOSS);
            } else {
                piv = sqrt(g);
            }
            G[(int64_t)j * ldg + j] = piv;
        }
        __syncthreads();
        const double rjj = piv;
        // row j of R: G[j, c] / r_jj for c > j (upper triangle, column-major: G[c*ldg + j])
        for (int c = j + 1 + threadIdx.x; c < b; c += blockDim.x) {
            const double v = (rjj > 0.0) ? G[(int64_t)c * ldg + j] / rjj : 0.0;
            G[(int64_t)c * ldg + j] = v;
        }
        __syncthreads();
        // trailing update of the upper triangle: G[c1, c2] -= R[j, c1] R[j, c2], j < c1 <= c2
        const int rem = b - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int c1 = j + 1 + e % rem, c2 = j + 1 + e / rem;
            if (c1 <= c2) G[(int64_t)c2 * ldg + c1] -= G[(int64_t)c1 * ldg + j] * G[(int64_t)c2 * ldg + j];
        }
        __syncthreads();
    }
    // zero the strict lower triangle
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e % b, c = e / b;
        if (r > c) G[(int64_t)c * ldg + r] = 0.0;
    }
    __syncthreads();
    // Rinv by back substitution, one column per thread
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        for (int i = b - 1; i >= 0; --i) {
            double v = (i == c) ? 1.0 : 0.0;
            if (i > c) v = 0.0;
            else {
                for (int l = i + 1; l <= c; ++l) v -= G[(int64_t)l * ldg + i] * Rinv[(int64_t)c * b + l];
                const double rii = G[(int64_t)i * ldg + i];
                v = (rii > 0.0) ? v / rii : 0.0;
            }
            Rinv[(int64_t)c * b + i] = v;
        }
    }
    if (threadIdx.x == 0 && lost) lost[b] = nlost;
}

// The factorisation of k_chol_inv for 32 < b <= kCholSmemMax with G and R^{-1} held in shared memory
// (the same pivot order, rank threshold, lost list and status bits): one reciprocal per pivot
// scales its row of R, and the back substitution for R^{-1} multiplies by the stored reciprocal
// pivots and splits each inner product over two accumulators, halving its dependent FMA chain.
constexpr int kCholSmemMax = 90;

__global__ void __launch_bounds__(256) k_chol_inv_smem(int b, double* G, int ldg, double* Rinv, double rank_tol,
                                                       double piv_min2, int* status, int* lost) {
    extern __shared__ double smc[];
    double* sg = smc;              // sg[c * b + r] = G[r, c]
    double* sx = smc + b * b;      // sx[c * b + i] = Rinv[i, c]
    __shared__ double inv[kCholSmemMax];
    __shared__ double maxdiag;
    __shared__ int nlost;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) sg[e] = G[(int64_t)(e / b) * ldg + e % b];
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        bool bad = false;
        for (int j = 0; j < b; ++j) {
            const double g = sg[j * b + j];
            if (!isfinite(g)) bad = true;
            mx = fmax(mx, fabs(g));
        }
        maxdiag = mx;
        nlost = 0;
        if (bad) atomicOr(status, ST_NONFINITE);
    }
    __syncthreads();
    const double thr = fmax(rank_tol * maxdiag, piv_min2);
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            const double g = sg[j * b + j];
            double piv = 0.0;
            if (!(g > thr) || maxdiag == 0.0) {
                if (lost) lost[nlost] = j;
                nlost++;
                atomicOr(status, ST_RANKLOSS);
            } else {
                piv = sqrt(g);
            }
            sg[j * b + j] = piv;
            inv[j] = piv > 0.0 ? 1.0 / piv : 0.0;
        }
        __syncthreads();
        const double ip = inv[j];
        for (int c = j + 1 + threadIdx.x; c < b; c += blockDim.x) sg[c * b + j] *= ip;
        __syncthreads();
        const int rem = b - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int c1 = j + 1 + e % rem, c2 = j + 1 + e / rem;
            if (c1 <= c2) sg[c2 * b + c1] -= sg[c1 * b + j] * sg[c2 * b + j];
        }
        __syncthreads();
    }
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        for (int i = b - 1; i > c; --i) sx[c * b + i] = 0.0;
        for (int i = c; i >= 0; --i) {
            double a0 = (i == c) ? 1.0 : 0.0, a1 = 0.0;
            int l = i + 1;
            for (; l + 1 <= c; l += 2) {
                a0 -= sg[l * b + i] * sx[c * b + l];
                a1 -= sg[(l + 1) * b + i] * sx[c * b + l + 1];
            }
            if (l <= c) a0 -= sg[l * b + i] * sx[c * b + l];
            sx[c * b + i] = (a0 + a1) * inv[i];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
        const int r = e % b, c = e / b;
        G[(int64_t)c * ldg + r] = (r > c) ? 0.0 : sg[e];
        Rinv[e] = sx[e];
    }
    if (threadIdx.x == 0 && lost) lost[b] = nlost;
}

template <class Ti, class To>
__global__ void k_copy(int64_t rows, int cols, const Ti* __restrict__ A, int64_t lda, To* __restrict__ B,
                       int64_t ldb) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e % rows, c = e / rows;
    B[c * ldb + r] = (To)A[c * lda + r];
}

__global__ void k_symmetrize(int m, double* A, int lda) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int r = (int)(e % m), c = (int)(e / m);
    if (r < c) {
        const double v = 0.5 * (A[(int64_t)c * lda + r] + A[(int64_t)r * lda + c]);
        A[(int64_t)c * lda + r] = v;
        A[(int64_t)r * lda + c] = v;
    }
}

// splitmix64 finaliser (Steele, Lea and Flood, 2014) as a counter-based generator.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <class T>
__global__ void k_fill_gaussian(int64_t rows, int cols, T* A, int64_t lda, uint64_t seed, uint64_t sid) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e % rows, c = e / rows;
    const uint64_t h1 = mix64(seed ^ mix64(sid * 0x100000001B3ull + (uint64_t)e));
    const uint64_t h2 = mix64(h1 + 0x632BE59BD9B4E019ull);
    const double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);   // (0, 1]
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);         // [0, 1)
    A[c * lda + r] = (T)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));       // Box-Muller
}

template <class T>
__global__ void k_col_norms(int64_t rows, const T* __restrict__ A, int64_t lda, double* out) {
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
        const double v = (double)A[(int64_t)c * lda + r];
        acc = fma(v, v, acc);
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        out[c] = sqrt(s);
    }
}

}  // namespace

namespace {

int g_sm_count = 0;   // streaming multiprocessors of the device the split counts are sized for

template <class T>
int gemm_tn_impl(int64_t d, int m, int p, double alpha, const T* A, int64_t lda, const T* B, int64_t ldb,
                 double beta, double* C, int ldc, void* partial_buf, size_t partial_cap, bool sym, cudaStream_t s) {
    if (m <= 0 || p <= 0) return EDA_OK;
    T* partial = static_cast<T*>(partial_buf);
    const int TP = sym ? TN_TM : (p <= 8 ? 8 : (p <= 16 ? 16 : 32));
    const int tm = ceil_div(m, TN_TM);
    const int tiles = sym ? tm * (tm + 1) / 2 : tm * ceil_div(p, TP);
    const int nsm = sm_count();
    // algorithmic work of this product, by the definition (one triangle for the symmetric case):
    // flops 2 d m p (SYRK: d m (m + 1)), bytes: A and B read once, C written once, in the storage type
    const double flops = sym ? (double)d * m * (m + 1.0) : 2.0 * (double)d * m * p;
    const double bytes = (double)sizeof(T) * (double)d * (sym ? m : (double)m + p) + 8.0 * m * p;
    ProfScope prof(std::is_same<T, double>::value ? "tn_f64" : "tn_f32", s, flops, bytes);
    // Split count: the kernel is FP64- or bandwidth-bound per SM, so an SM holding one CTA more than
    // the others sets the time. Among counts giving 1.8 to 4 CTAs per SM (after rounding the split
    // rows to TN_KB), take the one that fills the SMs most evenly, tiles * splits over
    // nsm * ceil(tiles * splits / nsm), preferring fewer splits unless another fills 2 % better.
    int splits = 1;
    {
        const int smax = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(4 * nsm, tiles), (d + 63) / 64));
        const int smin = std::min(smax, std::max(1, (int)std::ceil(1.8 * nsm / tiles)));
        double best = -1.0;
        for (int s0 = smin; s0 <= smax; ++s0) {
            int64_t rw = (d + s0 - 1) / s0;
            rw = (rw + TN_KB - 1) / TN_KB * TN_KB;
            const int sc = (int)std::max<int64_t>(1, (d + rw - 1) / rw);
            const int64_t ctas = (int64_t)tiles * sc;
            const double fill = (double)ctas / ((double)nsm * (double)((ctas + nsm - 1) / nsm));
            if (fill > best + 0.02) {
                best = fill;
                splits = sc;
            }
        }
    }
    while (splits > 1 && (size_t)splits * m * p > partial_cap) --splits;
    if ((size_t)splits * m * p > partial_cap) return EDA_ERR_INVALID_ARG;
    int64_t rows = (d + splits - 1) / splits;
    rows = (rows + TN_KB - 1) / TN_KB * TN_KB;
    splits = (int)std::max<int64_t>(1, (d + rows - 1) / rows);
    if (d > 0) {
        if (sym) {
            dim3 grid(tiles, 1, splits);
            k_gemm_tn_partial<32, T, true><<<grid, TN_THREADS, 0, s>>>(d, m, p, A, lda, B, ldb, rows, partial);
        } else {
            dim3 grid(tm, ceil_div(p, TP), splits);
            if (TP == 8) k_gemm_tn_partial<8, T><<<grid, TN_THREADS, 0, s>>>(d, m, p, A, lda, B, ldb, rows, partial);
            else if (TP == 16) k_gemm_tn_partial<16, T><<<grid, TN_THREADS, 0, s>>>(d, m, p, A, lda, B, ldb, rows, partial);
            else k_gemm_tn_partial<32, T><<<grid, TN_THREADS, 0, s>>>(d, m, p, A, lda, B, ldb, rows, partial);
        }
        EDA_LAUNCHED();
    } else {
        splits = 0;
    }
    const int64_t tot = (int64_t)m * p;
    if (splits >= 16 && tot <= 65536)
        k_gemm_tn_reduce_warp<T><<<ceil_div(tot * 32, 256), 256, 0, s>>>(m, p, splits, partial, alpha, beta, C, ldc,
                                                                          sym);
    else
        k_gemm_tn_reduce<T><<<ceil_div(tot, 256), 256, 0, s>>>(m, p, splits, partial, alpha, beta, C, ldc, sym);
    EDA_LAUNCHED();
    return EDA_OK;
}

}  // namespace

int sm_count() {
    // queried once per process for the current device (every handle of a process uses one GPU type)
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            g_sm_count = n;
        else
            g_sm_count = 148;
        cudaGetLastError();
    });
    return g_sm_count;
}

template <class T>
int gemm_tn(int64_t d, int m, int p, double alpha, const T* A, int64_t lda, const T* B, int64_t ldb, double beta,
            double* C, int ldc, void* partial_buf, size_t partial_cap, cudaStream_t s) {
    return gemm_tn_impl<T>(d, m, p, alpha, A, lda, B, ldb, beta, C, ldc, partial_buf, partial_cap, false, s);
}

template <class T>
int syrk_tn(int64_t d, int m, double alpha, const T* A, int64_t lda, double beta, double* C, int ldc,
            void* partial_buf, size_t partial_cap, cudaStream_t s) {
    return gemm_tn_impl<T>(d, m, m, alpha, A, lda, A, lda, beta, C, ldc, partial_buf, partial_cap, true, s);
}

template <class T>
int gemm_nn(int64_t d, int m, int p, double alpha, const T* A, int64_t lda, const double* B, int ldb, double beta,
            const T* C0, int64_t ldc0, T* C, int64_t ldc, cudaStream_t s, bool b_upper) {
    if (d <= 0 || p <= 0) return EDA_OK;
    // algorithmic work: 2 d m p flops (2 d sum_c min(m, c + 1) for an upper triangular B); A read once,
    // C0 read (beta != 0) and C written once
    double terms = (double)m * p;
    if (b_upper) {
        terms = 0.0;
        for (int c = 0; c < p; ++c) terms += std::min(m, c + 1);
    }
    ProfScope prof(std::is_same<T, double>::value ? "nn_f64" : "nn_f32", s, 2.0 * (double)d * terms,
                   (double)sizeof(T) * (double)d * (m + (beta != 0.0 ? 2.0 : 1.0) * p) + 8.0 * m * p);
    const int ub = b_upper ? 1 : 0;
    const int rowblocks = ceil_div(d, 32);
    // columns per thread: as many as possible while at least ~one CTA per SM stays busy
    if (p >= 6 && (int64_t)rowblocks * ceil_div(p, 8) >= 120) {
        k_gemm_nn<8, T><<<dim3(rowblocks, ceil_div(p, 8)), 256, 0, s>>>(d, m, p, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc, ub);
    } else if (p >= 3 && (int64_t)rowblocks * ceil_div(p, 4) >= 120) {
        k_gemm_nn<4, T><<<dim3(rowblocks, ceil_div(p, 4)), 256, 0, s>>>(d, m, p, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc, ub);
    } else if (p >= 2) {
        k_gemm_nn<2, T><<<dim3(rowblocks, ceil_div(p, 2)), 256, 0, s>>>(d, m, p, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc, ub);
    } else {
        k_gemm_nn<1, T><<<dim3(rowblocks, p), 256, 0, s>>>(d, m, p, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc, ub);
    }
    EDA_LAUNCHED();
    return EDA_OK;
}

template <class Ti, class To>
int copy_mat(int64_t rows, int cols, const Ti* A, int64_t lda, To* B, int64_t ldb, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return EDA_OK;
    k_copy<Ti, To><<<ceil_div(rows * cols, 256), 256, 0, s>>>(rows, cols, A, lda, B, ldb);
    EDA_LAUNCHED();
    return EDA_OK;
}

template <class T>
int fill_gaussian(int64_t rows, int cols, T* A, int64_t lda, uint64_t seed, uint64_t stream_id, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return EDA_OK;
    k_fill_gaussian<T><<<ceil_div(rows * cols, 256), 256, 0, s>>>(rows, cols, A, lda, seed, stream_id);
    EDA_LAUNCHED();
    return EDA_OK;
}

template <class T>
int col_norms(int64_t rows, int cols, const T* A, int64_t lda, double* out, cudaStream_t s) {
    if (cols <= 0) return EDA_OK;
    k_col_norms<T><<<cols, 256, 0, s>>>(rows, A, lda, out);
    EDA_LAUNCHED();
    return EDA_OK;
}

template int gemm_tn<double>(int64_t, int, int, double, const double*, int64_t, const double*, int64_t, double,
                             double*, int, void*, size_t, cudaStream_t);
template int gemm_tn<float>(int64_t, int, int, double, const float*, int64_t, const float*, int64_t, double,
                            double*, int, void*, size_t, cudaStream_t);
template int syrk_tn<double>(int64_t, int, double, const double*, int64_t, double, double*, int, void*, size_t,
                             cudaStream_t);
template int syrk_tn<float>(int64_t, int, double, const float*, int64_t, double, double*, int, void*, size_t,
                            cudaStream_t);
template int gemm_nn<double>(int64_t, int, int, double, const double*, int64_t, const double*, int, double,
                             const double*, int64_t, double*, int64_t, cudaStream_t, bool);
template int gemm_nn<float>(int64_t, int, int, double, const float*, int64_t, const double*, int, double,
                            const float*, int64_t, float*, int64_t, cudaStream_t, bool);
template int copy_mat<double, double>(int64_t, int, const double*, int64_t, double*, int64_t, cudaStream_t);
template int copy_mat<float, float>(int64_t, int, const float*, int64_t, float*, int64_t, cudaStream_t);
template int copy_mat<double, float>(int64_t, int, const double*, int64_t, float*, int64_t, cudaStream_t);
template int copy_mat<float, double>(int64_t, int, const float*, int64_t, double*, int64_t, cudaStream_t);
template int fill_gaussian<double>(int64_t, int, double*, int64_t, uint64_t, uint64_t, cudaStream_t);
template int fill_gaussian<float>(int64_t, int, float*, int64_t, uint64_t, uint64_t, cudaStream_t);
template int col_norms<double>(int64_t, int, const double*, int64_t, double*, cudaStream_t);
template int col_norms<float>(int64_t, int, const float*, int64_t, double*, cudaStream_t);

int gemm_tn_f64(int64_t d, int m, int p, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                double beta, double* C, int ldc, double* partial, size_t partial_cap, cudaStream_t s) {
    return gemm_tn<double>(d, m, p, alpha, A, lda, B, ldb, beta, C, ldc, partial, partial_cap, s);
}

int syrk_f64(int64_t d, int m, double alpha, const double* A, int64_t lda, double beta, double* C, int ldc,
             double* partial, size_t partial_cap, cudaStream_t s) {
    return syrk_tn<double>(d, m, alpha, A, lda, beta, C, ldc, partial, partial_cap, s);
}

int gemm_nn_f64(int64_t d, int m, int p, double alpha, const double* A, int64_t lda, const double* B, int ldb,
                double beta, const double* C0, int64_t ldc0, double* C, int64_t ldc, cudaStream_t s) {
    return gemm_nn<double>(d, m, p, alpha, A, lda, B, ldb, beta, C0, ldc0, C, ldc, s);
}

int gemm_small_f64(bool ta, bool tb, int m, int p, int kk, double alpha, const double* A, int lda, const double* B,
                   int ldb, double beta, double* C, int ldc, cudaStream_t s) {
    if (m <= 0 || p <= 0) return EDA_OK;
    if (!ta && !tb && kk >= 64) {
        k_gemm_small_nn_splitk<<<dim3(ceil_div(m, 32), p), 32 * kSplitkWarps, 0, s>>>(m, p, kk, alpha, A, lda, B, ldb,
                                                                                  beta, C, ldc);
        EDA_LAUNCHED();
        return EDA_OK;
    }
    // one warp per CTA (32 rows of one column): FP64 work spreads over all SMs
    dim3 blk(32, 1), grid(ceil_div(m, 32), p);
    k_gemm_small<<<grid, blk, 0, s>>>(ta, tb, m, p, kk, alpha, A, lda, B, ldb, beta, C, ldc);
    EDA_LAUNCHED();
    return EDA_OK;
}

int chol_inv_small(int b, double* G, int ldg, double* Rinv, double rank_tol, double piv_min2, int* status, int* lost,
                   cudaStream_t s) {
    if (b <= 32) {
        k_chol_inv_warp<<<1, 32, 0, s>>>(b, G, ldg, Rinv, rank_tol, piv_min2, status, lost);
    } else if (b <= kCholSmemMax) {
        static std::once_flag once;
        static cudaError_t attr_rc = cudaSuccess;
        std::call_once(once, [] {
            attr_rc = cudaFuncSetAttribute(k_chol_inv_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(2 * sizeof(double) * kCholSmemMax * kCholSmemMax));
        });
        EDA_CUDA_TRY(attr_rc);
        k_chol_inv_smem<<<1, 256, 2 * sizeof(double) * b * b, s>>>(b, G, ldg, Rinv, rank_tol, piv_min2, status, lost);
    } else {
        k_chol_inv<<<1, 256, 0, s>>>(b, G, ldg, Rinv, rank_tol, piv_min2, status, lost);
    }
    EDA_LAUNCHED();
    return EDA_OK;
}

namespace {
// B (rows x cols, ldb) = 0 below the diagonal (strict lower triangle of a square or tall block)
__global__ void k_zero_lower(int m, double* A, int lda) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int r = (int)(e % m), c = (int)(e / m);
    if (r > c) A[(int64_t)c * lda + r] = 0.0;
}
__global__ void k_zero_all(int m, double* A, int lda) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    A[(int64_t)(e / m) * lda + e % m] = 0.0;
}
}  // namespace

size_t chol_inv_blocked_doubles(int m) { return (size_t)kCholBlock * m + (size_t)kCholBlock * kCholBlock; }

// Right-looking blocked Cholesky G = R^T R (R upper, in place, strict lower triangle zeroed) and R^{-1}, in
// blocks of kCholBlock: the diagonal block by the one-CTA factorisation (with its rank detection), the row
// panel R12 = R11^{-T} G12 and the trailing update G22 -= R12^T R12 as multi-CTA products; then R^{-1} block
// column by block column, X[:j, j] = -X[:j, :j] R[:j, j] R_jj^{-1}. work: chol_inv_blocked_doubles(m);
// partial: split-K partials of at least m * m doubles.
int chol_inv_blocked(int m, double* G, int ldg, double* Rinv, int ldr, double rank_tol, int* status, double* work,
                     double* partial, size_t pcap, cudaStream_t s) {
    constexpr int NB = kCholBlock;
    double* T = work;                          // NB x m
    double* Dinv = work + (size_t)NB * m;      // NB x NB
    // R^{-1} starts as zero: its blocks below the block diagonal are never written and are read as zeros
    k_zero_all<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, Rinv, ldr);
    EDA_LAUNCHED();
    for (int j0 = 0; j0 < m; j0 += NB) {
        const int nb = std::min(NB, m - j0);
        double* G11 = G + (int64_t)j0 * ldg + j0;
        EDA_TRY(chol_inv_small(nb, G11, ldg, Dinv, rank_tol, 0.0, status, nullptr, s));
        // R^{-1} diagonal block
        EDA_TRY(copy_mat_f64(nb, nb, Dinv, nb, Rinv + (int64_t)j0 * ldr + j0, ldr, s));
        const int r = m - j0 - nb;
        if (r > 0) {
            double* G12 = G + (int64_t)(j0 + nb) * ldg + j0;
            double* G22 = G + (int64_t)(j0 + nb) * ldg + j0 + nb;
            // R12 = R11^{-T} G12
            EDA_TRY(gemm_small_f64(true, false, nb, r, nb, 1.0, Dinv, nb, G12, ldg, 0.0, T, nb, s));
            EDA_TRY(copy_mat_f64(nb, r, T, nb, G12, ldg, s));
            // G22 -= R12^T R12 (a product reduced over the nb rows of R12)
            EDA_TRY(gemm_tn_f64(nb, r, r, -1.0, G12, ldg, G12, ldg, 1.0, G22, ldg, partial, pcap, s));
        }
    }
    k_zero_lower<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, G, ldg);
    EDA_LAUNCHED();
    // off-diagonal blocks of R^{-1}: X[:j0, j-block] = -X[:j0, :j0] (R[:j0, j-block] R_jj^{-1})
    for (int j0 = NB; j0 < m; j0 += NB) {
        const int nb = std::min(NB, m - j0);
        const double* Rj = G + (int64_t)j0 * ldg;                       // R[:j0, j-block]
        const double* Xjj = Rinv + (int64_t)j0 * ldr + j0;              // R_jj^{-1}
        EDA_TRY(gemm_small_f64(false, false, j0, nb, nb, 1.0, Rj, ldg, Xjj, ldr, 0.0, T, j0, s));
        EDA_TRY(gemm_small_f64(false, false, j0, nb, j0, -1.0, Rinv, ldr, T, j0, 0.0, Rinv + (int64_t)j0 * ldr, ldr,
                               s));
    }
    return EDA_OK;
}

int chol_inv_auto(int b, double* G, int ldg, double* Rinv, double rank_tol, int* status, double* work, double* partial,
                  size_t pcap, cudaStream_t s) {
    if (b <= 90) return chol_inv_small(b, G, ldg, Rinv, rank_tol, 0.0, status, nullptr, s);
    return chol_inv_blocked(b, G, ldg, Rinv, b, rank_tol, status, work, partial, pcap, s);
}

int copy_mat_f64(int64_t rows, int cols, const double* A, int64_t lda, double* B, int64_t ldb, cudaStream_t s) {
    return copy_mat<double, double>(rows, cols, A, lda, B, ldb, s);
}

int symmetrize_f64(int m, double* A, int lda, cudaStream_t s) {
    if (m <= 1) return EDA_OK;
    k_symmetrize<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>(m, A, lda);
    EDA_LAUNCHED();
    return EDA_OK;
}

int fill_gaussian_f64(int64_t rows, int cols, double* A, int64_t lda, uint64_t seed, uint64_t stream_id,
                      cudaStream_t s) {
    return fill_gaussian<double>(rows, cols, A, lda, seed, stream_id, s);
}

int col_norms_f64(int64_t rows, int cols, const double* A, int64_t lda, double* out, cudaStream_t s) {
    return col_norms<double>(rows, cols, A, lda, out, s);
}

}  // namespace eda
