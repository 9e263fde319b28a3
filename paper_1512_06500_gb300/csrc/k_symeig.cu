// FP64 symmetric eigensolver for the small matrices of the method: the Gram matrices
// G = H^T H (the spectra D = Sigma^2 of Eqs. (3.4)-(3.6)) and the block-tridiagonal Lanczos
// matrix T of the Rayleigh-Ritz step.
//
// Route: Householder reduction to tridiagonal form (from n = 288 a cooperative grid with the columns
// resident in its CTAs' shared memory; below that, or when the GPU is shared, one thread-block cluster;
// beyond what shared memory holds, a cooperative grid streaming the matrix through L2; all with bounded
// barriers) -> eigenvalues by 33-way
// multisection on Sturm counts (one warp per eigenvalue) -> eigenvectors of the tridiagonal
// by inverse iteration with partial pivoting (one thread per eigenvector) -> modified
// Gram-Schmidt inside tight clusters (one warp per cluster) -> back-transformation with the
// stored reflectors. Callers add a Newton-Schulz step for orthogonality across near clusters.
#include "eda_internal.cuh"
#include "grid_bar.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cfloat>
#include <cmath>

namespace eda {

namespace {

constexpr int TRI_THREADS = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid-wide barrier for a cooperative launch. On timeout it records ST_TIMEOUT and
// returns; the kernel then runs to completion with stale data and the host reports the error.
__device__ void grid_sync(GridBarrier bar, int* status) {
    if (gridDim.x == 1) {
        __syncthreads();
        return;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_u32(bar.gen);
        __threadfence();
        const unsigned ticket = atomicAdd(bar.count, 1u);
        if (ticket == gridDim.x - 1) {
            atomicExch(bar.count, 0u);
            __threadfence();
            atomicAdd(bar.gen, 1u);
        } else {
            long long it = 0;
            while (ld_acquire_u32(bar.gen) == g) {
                if (++it > bar.spin_limit) {
                    atomicOr(status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    // pairwise tree over the warps: the same fixed order in every thread and every CTA
    const int nw = blockDim.x >> 5;
    if (nw == 4) return (red[0] + red[1]) + (red[2] + red[3]);
    if (nw == 8) return ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    double sacc = 0.0;
    for (int i = 0; i < nw; ++i) sacc += red[i];
    return sacc;
}

// Householder tridiagonalisation of the full symmetric n x n matrix A (ld n), in place.
// HV[j * n + i] receives reflector j (u_j[j+1] = 1, zero above), tau[j] its scalar.
// vbuf: 2n doubles (p vector and a copy of the current column).
__global__ void __launch_bounds__(TRI_THREADS) k_tridiag(int n, double* A, double* HV, double* dgl, double* eoff,
                                                         double* tau, double* pglob, GridBarrier bar, int* status) {
    extern __shared__ double sm[];
    double* v = sm;          // n
    double* w = sm + n;      // n
    __shared__ double red[32];
    const int C = gridDim.x, cta = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;

    for (int j = 0; j + 2 < n; ++j) {
        const int i0 = j + 1;                // trailing block starts here
        // ---- Householder vector of column j (computed redundantly by every CTA) ----
        double ss = 0.0;
        for (int i = i0 + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double x = A[(int64_t)j * n + i];
            ss = fma(x, x, ss);
        }
        ss = block_sum(ss, red);
        const double alpha = A[(int64_t)j * n + i0];
        double beta, tj, scal;
        if (ss == 0.0) {
            beta = alpha;
            tj = 0.0;
            scal = 0.0;
        } else {
            beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
            tj = (beta - alpha) / beta;
            scal = 1.0 / (alpha - beta);
        }
        for (int i = i0 + threadIdx.x; i < n; i += blockDim.x)
            v[i] = (i == i0) ? 1.0 : A[(int64_t)j * n + i] * scal;
        __syncthreads();
        if (cta == 0) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) HV[(int64_t)j * n + i] = (i >= i0) ? v[i] : 0.0;
            if (threadIdx.x == 0) {
                eoff[j] = beta;
                tau[j] = tj;
            }
        }
        if (tj == 0.0) {
            grid_sync(bar, status);   // keep every CTA on the same barrier count
            grid_sync(bar, status);
            continue;
        }
        // ---- p[r] = tau * sum_c A[c, r] v[c] for owned rows r (column r is contiguous) ----
        for (int r = i0 + cta + C * warp; r < n; r += C * nwarps) {
            double acc = 0.0;
            const double* col = A + (int64_t)r * n;
            for (int c = i0 + lane; c < n; c += 32) acc = fma(col[c], v[c], acc);
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) pglob[r] = tj * acc;
        }
        grid_sync(bar, status);
        // ---- w = p - (tau/2)(p^T v) v, then A22 -= v w^T + w v^T on owned columns ----
        double pv = 0.0;
        for (int i = i0 + threadIdx.x; i < n; i += blockDim.x) {
            const double pi = pglob[i];
            w[i] = pi;
            pv = fma(pi, v[i], pv);
        }
        pv = block_sum(pv, red);
        const double kk = 0.5 * tj * pv;
        for (int i = i0 + threadIdx.x; i < n; i += blockDim.x) w[i] = fma(-kk, v[i], w[i]);
        __syncthreads();
        for (int r = i0 + cta + C * warp; r < n; r += C * nwarps) {
            double* col = A + (int64_t)r * n;
            const double vr = v[r], wr = w[r];
            for (int c = i0 + lane; c < n; c += 32) col[c] -= fma(v[c], wr, w[c] * vr);
        }
        grid_sync(bar, status);
    }
    if (cta == 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            dgl[i] = A[(int64_t)i * n + i];
            if (i + 2 >= n) {
                if (i + 1 < n) eoff[i] = A[(int64_t)i * n + i + 1];
                tau[i] = 0.0;
                for (int r = 0; r < n; ++r) HV[(int64_t)i * n + r] = 0.0;
            }
        }
        if (threadIdx.x == 0) eoff[n - 1] = 0.0;
    }
}

constexpr int CT_THREADS = 128;

// Reflector of column j (entries a[i], i > j) formed by the CTA that owns the column and
// published in its shared memory: vpub[i] for i > j, vpub[n] = tau, vpub[n + 1] = beta.
__device__ void make_reflector(int j, int n, const double* a, double* vpub, double* HV, double* eoff, double* tau,
                               double* red) {
    const int tid = threadIdx.x, bd = blockDim.x;
    const int i0 = j + 1;
    double ss = 0.0;
    for (int i = i0 + 1 + tid; i < n; i += bd) ss = fma(a[i], a[i], ss);
    ss = block_sum(ss, red);
    const double alpha = a[i0];
    double beta, tj, scal;
    if (ss == 0.0) {
        beta = alpha;
        tj = 0.0;
        scal = 0.0;
    } else {
        // beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta, scal = 1 / (alpha - beta)
        const double nrm2 = fma(alpha, alpha, ss);
        const double rn = rsqrt(nrm2);
        const double sg = (alpha >= 0.0) ? 1.0 : -1.0;
        beta = -sg * nrm2 * rn;
        tj = fma(sg * alpha, rn, 1.0);
        scal = 1.0 / (alpha - beta);
    }
    for (int i = tid; i < n; i += bd) {
        const double val = (i < i0) ? 0.0 : ((i == i0) ? 1.0 : a[i] * scal);
        if (i >= i0) vpub[i] = val;
        HV[(int64_t)j * n + i] = val;
    }
    if (tid == 0) {
        vpub[n] = tj;
        vpub[n + 1] = beta;
        eoff[j] = beta;
        tau[j] = tj;
    }
}

// Householder tridiagonalisation on one thread-block cluster (C <= 16 CTAs). Column c of the
// symmetric matrix is owned by CTA c % C and kept in its shared memory (or, for large n, in a
// global slab of that CTA). Per column j: after a cluster barrier every CTA reads the reflector
// that the owner of column j published, forms its partial p over the columns it owns; after a
// second barrier every CTA sums the partials of all CTAs (distributed shared memory, fixed
// pairwise order), forms w and updates its columns. The owner of column j + 1 updates that
// column first and publishes reflector j + 1 while the other CTAs are still updating
// (look-ahead), so the reflector's FP64 latency chain is off the critical path.
template <int C>
__global__ void __launch_bounds__(CT_THREADS) k_tridiag_cluster(int n, const double* __restrict__ Ain, int lda,
                                                                double* Aglob, int in_smem, double* HV, double* dgl,
                                                                double* eoff, double* tau) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    extern __shared__ double sm[];
    __shared__ double red[32];
    const int ncl = (n + C - 1) / C;
    double* vbuf = sm;                 // n: reflector (local copy)
    double* vpub = sm + n;             // n + 2: reflector published by the owner, then tau, beta
    double* ppart = sm + 2 * n + 2;    // n: this CTA's partial p
    double* pw = sm + 3 * n + 2;       // n: full p, then w
    double* Aloc = in_smem ? (sm + 4 * n + 2) : (Aglob + (size_t)rank * ncl * n);
    const int tid = threadIdx.x, bd = blockDim.x;

    for (int q = 0; q < ncl; ++q) {
        const int c = q * C + rank;
        if (c >= n) break;
        for (int i = tid; i < n; i += bd)
            Aloc[(size_t)q * n + i] = 0.5 * (Ain[(int64_t)c * lda + i] + Ain[(int64_t)i * lda + c]);
    }
    __syncthreads();
    if (n >= 3 && rank == 0) make_reflector(0, n, Aloc, vpub, HV, eoff, tau, red);

    for (int j = 0; j + 2 < n; ++j) {
        const int i0 = j + 1;
        const int owner = j % C;
        const int next = j + 1;
        const bool own_next = (next + 2 < n) && (next % C == rank);
        cluster.sync();                                   // reflector j published
        const double* rv = cluster.map_shared_rank(vpub, owner);
        const double tj = rv[n];
        if (tj == 0.0) {                                  // same decision in every CTA
            __syncthreads();
            if (own_next) make_reflector(next, n, Aloc + (size_t)(next / C) * n, vpub, HV, eoff, tau, red);
            continue;
        }
        for (int i = i0 + tid; i < n; i += bd) vbuf[i] = rv[i];
        __syncthreads();
        const int q0 = (i0 - rank + C - 1) / C;           // first owned column >= i0
        for (int i = i0 + tid; i < n; i += bd) {
            double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
            int q = q0;
            for (; q + 3 < ncl; q += 4) {
                const int c0 = q * C + rank;
                if (c0 + 3 * C >= n) break;
                const double* a = Aloc + (size_t)q * n + i;
                acc0 = fma(a[0], vbuf[c0], acc0);
                acc1 = fma(a[n], vbuf[c0 + C], acc1);
                acc2 = fma(a[2 * n], vbuf[c0 + 2 * C], acc2);
                acc3 = fma(a[3 * n], vbuf[c0 + 3 * C], acc3);
            }
            for (; q < ncl; ++q) {
                const int c = q * C + rank;
                if (c >= n) break;
                acc0 = fma(Aloc[(size_t)q * n + i], vbuf[c], acc0);
            }
            ppart[i] = (acc0 + acc1) + (acc2 + acc3);
        }
        cluster.sync();                                   // partial products published
        for (int i = i0 + tid; i < n; i += bd) {
            double t[C];
#pragma unroll
            for (int r = 0; r < C; ++r) t[r] = cluster.map_shared_rank(ppart, r)[i];
#pragma unroll
            for (int wd = 1; wd < C; wd <<= 1)
#pragma unroll
                for (int r = 0; r + wd < C; r += 2 * wd) t[r] += t[r + wd];
            pw[i] = tj * t[0];
        }
        __syncthreads();
        double pv = 0.0;
        for (int i = i0 + tid; i < n; i += bd) pv = fma(pw[i], vbuf[i], pv);
        pv = block_sum(pv, red);
        const double kk = 0.5 * tj * pv;
        for (int i = i0 + tid; i < n; i += bd) pw[i] = fma(-kk, vbuf[i], pw[i]);
        __syncthreads();
        if (own_next) {
            double* col = Aloc + (size_t)(next / C) * n;
            const double vc = vbuf[next], wc = pw[next];
            for (int i = i0 + tid; i < n; i += bd) col[i] -= fma(vbuf[i], wc, pw[i] * vc);
            __syncthreads();
            make_reflector(next, n, col, vpub, HV, eoff, tau, red);
        }
        {
            const int qskip = own_next ? next / C : -1;
            int qend = ncl;
            while (qend > q0 && (qend - 1) * C + rank >= n) --qend;
            for (int i = i0 + tid; i < n; i += bd) {
                const double vi = vbuf[i], wi = pw[i];
                int q = q0;
                for (; q + 3 < qend; q += 4) {
                    double* c0 = Aloc + (size_t)q * n + i;
                    const int cc = q * C + rank;
                    const double a0 = c0[0], a1 = c0[n], a2 = c0[2 * n], a3 = c0[3 * n];
                    const double r0 = a0 - fma(vi, pw[cc], wi * vbuf[cc]);
                    const double r1 = a1 - fma(vi, pw[cc + C], wi * vbuf[cc + C]);
                    const double r2 = a2 - fma(vi, pw[cc + 2 * C], wi * vbuf[cc + 2 * C]);
                    const double r3 = a3 - fma(vi, pw[cc + 3 * C], wi * vbuf[cc + 3 * C]);
                    if (q != qskip) c0[0] = r0;
                    if (q + 1 != qskip) c0[n] = r1;
                    if (q + 2 != qskip) c0[2 * n] = r2;
                    if (q + 3 != qskip) c0[3 * n] = r3;
                }
                for (; q < qend; ++q) {
                    if (q == qskip) continue;
                    const int cc = q * C + rank;
                    double* c0 = Aloc + (size_t)q * n + i;
                    c0[0] -= fma(vi, pw[cc], wi * vbuf[cc]);
                }
            }
        }
        __syncthreads();
    }
    for (int q = 0; q < ncl; ++q) {
        const int c = q * C + rank;
        if (c >= n) break;
        if (tid == 0) {
            dgl[c] = Aloc[(size_t)q * n + c];
            if (c == n - 2) eoff[c] = Aloc[(size_t)q * n + c + 1];
        }
    }
    if (rank == 0) {
        for (int jj = (n >= 2 ? n - 2 : 0); jj < n; ++jj) {
            if (tid == 0) tau[jj] = 0.0;
            for (int i = tid; i < n; i += bd) HV[(int64_t)jj * n + i] = 0.0;
        }
        if (tid == 0) eoff[n - 1] = 0.0;
    }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// Householder tridiagonalisation on a cooperative grid of G CTAs with the matrix resident in shared
// memory: column c is owned by CTA c % G (slot c / G, n doubles). Per column j, after the grid barrier
// that publishes reflector j (global memory, read through L2): every CTA copies it into shared memory,
// forms p[r] = tau v^T A[:, r] for its own columns r and its share of p^T v (its columns in increasing
// order), publishes both; after a second barrier every CTA reads p and the G shares (summed in CTA
// order: the same value everywhere), forms w = p - (tau / 2)(p^T v) v and updates its columns
// (A -= v w^T + w v^T). The owner of column j + 1 updates that column first and publishes reflector
// j + 1 while the others update theirs (look-ahead). Two bounded grid barriers per column on the
// monotonic arrival counter; the columns never leave shared memory.
__global__ void __launch_bounds__(TRI_THREADS) k_tridiag_res(int n, const double* __restrict__ Ain, int lda,
                                                             double* vglob, double* pglob, double* pshare, double* HV,
                                                             double* dgl, double* eoff, double* tau, GridBarWords bw,
                                                             int* status) {
    extern __shared__ double sm[];
    __shared__ double red[32];
    __shared__ double s_pv;
    const int G = gridDim.x, cta = blockIdx.x;
    const int ncl = (n + G - 1) / G;
    double* vs = sm;             // n: reflector j
    double* ws = sm + n;         // n: p, then w
    double* Aloc = sm + 2 * n;   // ncl x n: the owned columns
    double* shs = Aloc + (size_t)ncl * n;   // G: the CTAs' shares of p^T v
    const int tid = threadIdx.x, bd = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = bd >> 5;
    const unsigned base = gb_base(bw);
    unsigned nb = 0;

    for (int q = 0; q < ncl; ++q) {
        const int c = q * G + cta;
        if (c >= n) break;
        for (int i = tid; i < n; i += bd)
            Aloc[(size_t)q * n + i] = 0.5 * (Ain[(int64_t)c * lda + i] + Ain[(int64_t)i * lda + c]);
    }
    __syncthreads();
    if (n >= 3 && cta == 0) make_reflector(0, n, Aloc, vglob, HV, eoff, tau, red);
    gb_sync(bw, base, ++nb, status);

    for (int j = 0; j + 2 < n; ++j) {
        const int i0 = j + 1;
        const int next = j + 1;
        const bool own_next = (next + 2 < n) && (next % G == cta);
        const int q0 = (i0 - cta + G - 1) / G;   // first owned slot with a column >= i0
        const double tj = __ldcg(vglob + n);
        if (tj == 0.0) {
            // no reflection at this column: every CTA has read tau before the owner of j + 1 overwrites it
            gb_sync(bw, base, ++nb, status);
            if (own_next) make_reflector(next, n, Aloc + (size_t)(next / G) * n, vglob, HV, eoff, tau, red);
            gb_sync(bw, base, ++nb, status);
            continue;
        }
        for (int i = i0 + tid; i < n; i += bd) vs[i] = __ldcg(vglob + i);
        __syncthreads();
        // p over the owned columns, one warp per column (lane-strided dot, fixed shuffle tree)
        for (int q = q0 + warp; q < ncl; q += nw) {
            const int r = q * G + cta;
            if (r >= n) break;
            const double* col = Aloc + (size_t)q * n;
            double a0 = 0.0, a1 = 0.0;
            int c = i0 + lane;
            for (; c + 32 < n; c += 64) {
                a0 = fma(col[c], vs[c], a0);
                a1 = fma(col[c + 32], vs[c + 32], a1);
            }
            if (c < n) a0 = fma(col[c], vs[c], a0);
            double acc = a0 + a1;
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                const double p = tj * acc;
                pglob[r] = p;
                ws[r] = p;
            }
        }
        __syncthreads();
        if (tid == 0) {
            double sh = 0.0;
            for (int q = q0; q < ncl; ++q) {
                const int r = q * G + cta;
                if (r >= n) break;
                sh = fma(ws[r], vs[r], sh);
            }
            pshare[cta] = sh;
        }
        gb_sync(bw, base, ++nb, status);
        // w = p - (tau / 2)(p^T v) v
        for (int i = i0 + tid; i < n; i += bd) ws[i] = __ldcg(pglob + i);
        for (int g = tid; g < G; g += bd) shs[g] = __ldcg(pshare + g);
        __syncthreads();
        if (warp == 0) {
            // the G shares in a fixed order (lane-strided runs, then a shuffle tree): the same value in every CTA
            double pv = 0.0;
            for (int g = lane; g < G; g += 32) pv += shs[g];
            for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
            if (lane == 0) s_pv = pv;
        }
        __syncthreads();
        const double kk = 0.5 * tj * s_pv;
        for (int i = i0 + tid; i < n; i += bd) ws[i] = fma(-kk, vs[i], ws[i]);
        __syncthreads();
        if (own_next) {
            double* col = Aloc + (size_t)(next / G) * n;
            const double vc = vs[next], wc = ws[next];
            for (int i = i0 + tid; i < n; i += bd) col[i] -= fma(vs[i], wc, ws[i] * vc);
            __syncthreads();
            make_reflector(next, n, col, vglob, HV, eoff, tau, red);
        }
        for (int q = q0; q < ncl; ++q) {
            const int c = q * G + cta;
            if (c >= n) break;
            if (own_next && c == next) continue;
            double* col = Aloc + (size_t)q * n;
            const double vc = vs[c], wc = ws[c];
            for (int i = i0 + tid; i < n; i += bd) col[i] -= fma(vs[i], wc, ws[i] * vc);
        }
        gb_sync(bw, base, ++nb, status);
    }
    for (int q = 0; q < ncl; ++q) {
        const int c = q * G + cta;
        if (c >= n) break;
        if (tid == 0) {
            dgl[c] = Aloc[(size_t)q * n + c];
            if (c == n - 2) eoff[c] = Aloc[(size_t)q * n + c + 1];
        }
    }
    if (cta == 0) {
        for (int jj = (n >= 2 ? n - 2 : 0); jj < n; ++jj) {
            if (tid == 0) tau[jj] = 0.0;
            for (int i = tid; i < n; i += bd) HV[(int64_t)jj * n + i] = 0.0;
        }
        if (tid == 0) eoff[n - 1] = 0.0;
    }
    gb_finish(bw, base, nb);
}

// Number of eigenvalues below x of the tridiagonal with diagonal d and squared off-diagonal e2, in
// single precision (ratio form q_i = (d_i - x) - e2_{i-1} / q_{i-1}, small pivots replaced).
__device__ __forceinline__ int sturm_count_f32(int n, const float* d, const float* e2, float x, float pivmin) {
    int cnt = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += (q < 0.f);
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - __fdividef(e2[i - 1], q);
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += (q < 0.f);
    }
    return cnt;
}

// The same count in double precision without divisions: the leading principal minors
// p_i = det(T_i - x I) obey
// p_i = (d_{i-1} - x) p_{i-1} - e2_{i-2} p_{i-2}, and the number of sign changes along
// p_0 = 1, p_1, ..., p_n is the number of eigenvalues below x (Sturm). Sign tests use the sign
// bit (integer pipe); an exact zero takes the sign opposite to its predecessor (a sign change,
// as a zero pivot does in the ratio form); every fourth step the pair (p_{i-1}, p_i) is rescaled
// by a power of two when its exponent drifts, which keeps every sign and ratio exact.
__device__ __forceinline__ double fix_zero(double p, double prev) {
    const int hi = __double2hiint(p), lo = __double2loint(p);
    if (((hi & 0x7fffffff) | lo) != 0) return p;
    return __hiloint2double((~__double2hiint(prev) & 0x80000000) | 0x00100000, 0);   // -sign(prev) * DBL_MIN
}

__device__ __forceinline__ void rescale_pair(double& pc, double& pm) {
    const int ex = (__double2hiint(pc) >> 20) & 0x7ff;
    if (ex > 1023 + 480 || ex < 1023 - 480) {
        const double sc = __hiloint2double((2046 - ex) << 20, 0);   // 2^(1023 - ex)
        pc *= sc;
        pm *= sc;
    }
}

// The number of eigenvalues below x0 by that recurrence (one shift per thread).
__device__ __forceinline__ int sturm_count1_f64(int n, const double* d, const double* e2, double x0) {
    double pm0 = 1.0;
    double pc0 = fix_zero(d[0] - x0, 1.0);
    int c0 = (int)((unsigned)__double2hiint(pc0) >> 31);
    for (int i = 1; i < n; ++i) {
        const double di = d[i], ei = e2[i - 1];
        const double pn0 = fix_zero(fma(di - x0, pc0, -ei * pm0), pc0);
        c0 += (int)(((unsigned)__double2hiint(pn0) ^ (unsigned)__double2hiint(pc0)) >> 31);
        pm0 = pc0;
        pc0 = pn0;
        if ((i & 3) == 0) rescale_pair(pc0, pm0);
    }
    return c0;
}

// One CTA of two warps per wanted eigenvalue (ascending index il + blockIdx.x). The tridiagonal is
// scaled by 1 / ||T||; 33-way multisection first on single-precision counts (fast; both warps run it
// alike) until the interval is 1e-5 wide, then, after widening it by that margin (far above the
// single-precision backward error of the count, about 1e-6), 65-way multisection on double-precision
// counts down to ~eps: lane l of warp 0 counts at the shift 2 l + 1 of the 65-way split and lane l of
// warp 1 at 2 l + 2, so each warp's FP64 chain carries one shift (the FP64 pipe of a sub-partition
// holds a warp instruction for ~64 cycles, so two warps on two sub-partitions halve the time).
__global__ void __launch_bounds__(64) k_bisect(int n, const double* __restrict__ dgl, const double* __restrict__ eoff,
                                                int il, int nw, double* w) {
    extern __shared__ double smb[];
    double* d64 = smb;                                     // n
    double* e264 = smb + n;                                // n
    float* d32 = reinterpret_cast<float*>(smb + 2 * n);    // n
    float* e232 = d32 + n;                                 // n
    __shared__ double s_tnorm;
    __shared__ unsigned s_ball[2];
    __shared__ int s_cnt[2];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    // ||T||_inf by warp 0
    if (threadIdx.x < 32) {
        double m = 0.0;
        for (int i = lane; i < n; i += 32) {
            const double r = fabs(dgl[i]) + ((i > 0) ? fabs(eoff[i - 1]) : 0.0) + ((i + 1 < n) ? fabs(eoff[i]) : 0.0);
            m = fmax(m, r);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_tnorm = (m > 0.0) ? m : 1.0;
    }
    __syncthreads();
    const double tn = s_tnorm, itn = 1.0 / tn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double di = dgl[i] * itn;
        const double ei = (i + 1 < n) ? eoff[i] * itn : 0.0;
        d64[i] = di;
        e264[i] = ei * ei;
        d32[i] = (float)di;
        e232[i] = (float)(ei * ei);
    }
    __syncthreads();
    const int gw = blockIdx.x;
    if (gw >= nw) return;                                   // uniform over the CTA
    const int idx = il + gw;
    // scaled Gershgorin interval is inside [-1, 1]
    float lo = -1.0f - 1e-6f, hi = 1.0f + 1e-6f;
    const float piv32 = 1e-30f;
    for (int round = 0; round < 8 && hi - lo > 1e-5f; ++round) {
        const float step = (hi - lo) / 33.f;
        const float x = lo + (lane + 1) * step;
        const int cnt = sturm_count_f32(n, d32, e232, x, piv32);
        const unsigned above = __ballot_sync(0xffffffffu, cnt > idx);
        if (above == 0u) {
            lo = __shfl_sync(0xffffffffu, x, 31);
        } else {
            const int l = __ffs(above) - 1;
            const float xl = __shfl_sync(0xffffffffu, x, l);
            const float xp = __shfl_sync(0xffffffffu, x, l > 0 ? l - 1 : 0);
            if (l > 0) lo = xp;
            hi = xl;
        }
    }
    double dlo = (double)lo - 1e-5, dhi = (double)hi + 1e-5;
    // confirm the bracket in double precision (warp 0 at dlo, warp 1 at dhi); fall back to the full
    // interval if it fails
    {
        if (lane == 0) s_cnt[wp] = sturm_count1_f64(n, d64, e264, wp == 0 ? dlo : dhi);
        __syncthreads();
        const int clo = s_cnt[0], chi = s_cnt[1];
        if (!(clo <= idx && chi > idx)) {
            dlo = -1.0 - 1e-12;
            dhi = 1.0 + 1e-12;
        }
        __syncthreads();
    }
    for (int round = 0; round < 24; ++round) {
        const double width = dhi - dlo;
        if (width <= 2.0 * DBL_EPSILON * fmax(fabs(dlo), fabs(dhi)) || width <= 0.5 * DBL_EPSILON) break;
        const double step = width / 65.0;
        const double x = dlo + (2 * lane + 1 + wp) * step;   // warp 0: shifts 2 l + 1, warp 1: 2 l + 2
        const int c = sturm_count1_f64(n, d64, e264, x);
        const unsigned b = __ballot_sync(0xffffffffu, c > idx);
        if (lane == 0) s_ball[wp] = b;
        __syncthreads();
        const unsigned b0 = s_ball[0], b1 = s_ball[1];
        __syncthreads();
        const unsigned above = b0 | b1;
        if (above == 0u) {
            dlo = dlo + (2 * 31 + 2) * step;
        } else {
            const int l = __ffs(above) - 1;
            const bool first = (b0 >> l) & 1u;
            const double a0 = dlo + (2 * l + 1) * step;
            const double a1 = dlo + (2 * l + 2) * step;
            const double pl = dlo + (2 * (l > 0 ? l - 1 : 0) + 2) * step;
            if (first) {
                if (l > 0) dlo = pl;
                dhi = a0;
            } else {
                dlo = a0;
                dhi = a1;
            }
        }
    }
    if (threadIdx.x == 0) w[gw] = 0.5 * (dlo + dhi) * tn;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Inverse iteration, one thread per eigenvector; factor arrays laid out [array][i][q] so that
// the threads of a warp touch consecutive addresses. Gaussian elimination with partial pivoting
// of T - lambda I takes one reciprocal per row (of the pivot); the two triangular solves carry
// the running entries in registers. Every pass over the stored arrays reads IV_U rows at a time
// into registers before it uses them, so one memory latency is paid per IV_U rows instead of per
// row (the loads of a pass never depend on its stores: row i + 1 is read before row i is written,
// and the values read are the ones the previous pass left).
// Output: Zt[i][q] (n x nv, row stride nv).
constexpr int IV_U = 16;

__global__ void k_invit(int n, int nv, const double* __restrict__ dgl, const double* __restrict__ eoff,
                        const double* __restrict__ lam, double* lu, double* Zt, uint64_t seed) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nv) return;
    const int64_t S = nv;
    double* DL = lu;                           // multipliers
    double* RD = lu + (int64_t)n * S;          // reciprocal pivots
    double* DU = lu + 2 * (int64_t)n * S;      // first superdiagonal of U
    double* DU2 = lu + 3 * (int64_t)n * S;     // second superdiagonal of U
    double* PIV = lu + 4 * (int64_t)n * S;     // 1.0 where rows i and i+1 were interchanged
    double* x = Zt;
    const double l = lam[q];
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i)
        tnorm = fmax(tnorm, fabs(dgl[i]) + ((i > 0) ? fabs(eoff[i - 1]) : 0.0) + ((i + 1 < n) ? fabs(eoff[i]) : 0.0));
    const double tiny = fmax(DBL_EPSILON * tnorm, DBL_MIN);
    double dcur = dgl[0] - l;
    double ucur = (n > 1) ? eoff[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double sub = eoff[i];                    // T[i+1, i]
        const double dnext = dgl[i + 1] - l;
        const double unext = (i + 2 < n) ? eoff[i + 1] : 0.0;
        const bool swap = fabs(dcur) < fabs(sub);
        const double piv = swap ? sub : ((dcur == 0.0) ? tiny : dcur);
        const double r = 1.0 / piv;
        const double f = (swap ? dcur : sub) * r;
        RD[i * S + q] = r;
        DL[i * S + q] = f;
        DU[i * S + q] = swap ? dnext : ucur;
        DU2[i * S + q] = swap ? unext : 0.0;
        PIV[i * S + q] = swap ? 1.0 : 0.0;
        const double nd = swap ? (ucur - f * dnext) : (dnext - f * ucur);
        ucur = swap ? -f * unext : unext;
        dcur = nd;
    }
    RD[(int64_t)(n - 1) * S + q] = 1.0 / ((dcur == 0.0) ? tiny : dcur);
    // random start in [-1, 1]
    for (int i = 0; i < n; ++i) {
        const uint64_t h = mix64(seed ^ mix64(((uint64_t)q << 32) + (uint64_t)i + 0x5851F42D4C957F2Dull));
        x[i * S + q] = 2.0 * ((h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    double sc = 1.0;   // scale of the previous pass, applied to x as it is read
    for (int it = 0; it < 2; ++it) {
        // forward: L^{-1} P b, the running entry carried in a register
        double carry = x[q];
        if (it > 0) carry *= sc;
        for (int i0 = 0; i0 + 1 < n; i0 += IV_U) {
            double f[IV_U], nx[IV_U], pv[IV_U];
#pragma unroll
            for (int u = 0; u < IV_U; ++u) {
                const int i = i0 + u;
                if (i + 1 < n) {
                    f[u] = DL[i * S + q];
                    pv[u] = PIV[i * S + q];
                    nx[u] = x[(i + 1) * S + q];
                    if (it > 0) nx[u] *= sc;
                }
            }
#pragma unroll
            for (int u = 0; u < IV_U; ++u) {
                const int i = i0 + u;
                if (i + 1 < n) {
                    if (pv[u] != 0.0) {
                        x[i * S + q] = nx[u];
                        carry = carry - f[u] * nx[u];
                    } else {
                        x[i * S + q] = carry;
                        carry = nx[u] - f[u] * carry;
                    }
                }
            }
        }
        x[(int64_t)(n - 1) * S + q] = carry;
        // back: U^{-1}, carrying the two previous solution entries
        double v1 = 0.0, v2 = 0.0, mx = 0.0;
        for (int i0 = n - 1; i0 >= 0; i0 -= IV_U) {
            double xv[IV_U], du[IV_U], du2[IV_U], rd[IV_U];
#pragma unroll
            for (int u = 0; u < IV_U; ++u) {
                const int i = i0 - u;
                if (i >= 0) {
                    xv[u] = x[i * S + q];
                    du[u] = (i + 1 < n) ? DU[i * S + q] : 0.0;
                    du2[u] = (i + 2 < n) ? DU2[i * S + q] : 0.0;
                    rd[u] = RD[i * S + q];
                }
            }
#pragma unroll
            for (int u = 0; u < IV_U; ++u) {
                const int i = i0 - u;
                if (i >= 0) {
                    double v = xv[u];
                    if (i + 1 < n) v -= du[u] * v1;
                    if (i + 2 < n) v -= du2[u] * v2;
                    v *= rd[u];
                    x[i * S + q] = v;
                    mx = fmax(mx, fabs(v));
                    v2 = v1;
                    v1 = v;
                }
            }
        }
        sc = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 0.0;
    }
    // the last pass's scale, then the norm and the normalisation
    double nrm = 0.0;
    for (int i0 = 0; i0 < n; i0 += IV_U) {
        double xv[IV_U];
#pragma unroll
        for (int u = 0; u < IV_U; ++u)
            if (i0 + u < n) xv[u] = x[(i0 + u) * S + q] * sc;
#pragma unroll
        for (int u = 0; u < IV_U; ++u)
            if (i0 + u < n) nrm = fma(xv[u], xv[u], nrm);
    }
    const double sn = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
    for (int i0 = 0; i0 < n; i0 += IV_U) {
        double xv[IV_U];
#pragma unroll
        for (int u = 0; u < IV_U; ++u)
            if (i0 + u < n) xv[u] = x[(i0 + u) * S + q];
#pragma unroll
        for (int u = 0; u < IV_U; ++u)
            if (i0 + u < n) x[(i0 + u) * S + q] = (xv[u] * sc) * sn;
    }
}

// Zt (row-major n x nv) -> Z (column-major, ldz)
__global__ void k_transpose_out(int n, int nv, const double* Zt, double* Z, int ldz) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nv) return;
    const int i = (int)(e % n), q = (int)(e / n);
    Z[(int64_t)q * ldz + i] = Zt[(int64_t)i * nv + q];
}

// Z <- H_0 H_1 ... H_{n-3} Z, one warp per column of Z; reflector j is read from HV (row j,
// contiguous, zero above j + 1) through the read-only cache.
__global__ void k_backtransform(int n, int nv, const double* __restrict__ HV, const double* __restrict__ tau,
                                double* Z, int ldz) {
    const int lane = threadIdx.x & 31;
    const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (col >= nv) return;
    double* z = Z + (int64_t)col * ldz;
    for (int j = n - 3; j >= 0; --j) {
        const double tj = __ldg(tau + j);
        if (tj == 0.0) continue;
        const double* u = HV + (int64_t)j * n;
        double dot = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fma(__ldg(u + i), z[i], dot);
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double f = tj * dot;
        for (int i = j + 1 + lane; i < n; i += 32) z[i] = fma(-f, __ldg(u + i), z[i]);
    }
}

// The same with the column held in the registers of four warps (n <= 128 NPL), one warp per SM
// sub-partition: carried by a single warp, the chain of reflectors is bound by the FP64 issue rate of one
// sub-partition. Rows are dealt in 32-row stripes, row 32 (4 k + w) + lane in register k of warp w; a
// warp skips the stripes that lie wholly at or above reflector j's first nonzero row j + 1 (exact zero
// terms), the four partial dot products are added in a fixed order through shared memory (one barrier
// per reflector, the partials double-buffered), and reflector j - 1 and its scalar are read while
// reflector j is applied.
template <int NPL>
__global__ void __launch_bounds__(128) k_backtransform_w4(int n, int nv, const double* __restrict__ HV,
                                                          const double* __restrict__ tau, double* Z, int ldz) {
    __shared__ double red[2][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int col = blockIdx.x;
    if (col >= nv) return;   // uniform over the CTA
    double* zc = Z + (int64_t)col * ldz;
    double z[NPL];
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = 32 * (4 * k + w) + lane;
        z[k] = (i < n) ? zc[i] : 0.0;
    }
    // stripe k of this warp holds a row below j exactly when its last row 32 (4 k + w) + 31 exceeds j
    double un[NPL];
    double tn = 0.0;
    if (n >= 3) {
        const int j = n - 3;
        const double* u = HV + (int64_t)j * n;
        tn = __ldg(tau + j);
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            const int i = 32 * (4 * k + w) + lane;
            un[k] = (i < n && 32 * (4 * k + w) + 31 > j) ? __ldg(u + i) : 0.0;
        }
    }
    int par = 0;
    for (int j = n - 3; j >= 0; --j) {
        double uu[NPL];
#pragma unroll
        for (int k = 0; k < NPL; ++k) uu[k] = un[k];
        const double tj = tn;
        if (j > 0) {
            const double* u = HV + (int64_t)(j - 1) * n;
            tn = __ldg(tau + j - 1);
#pragma unroll
            for (int k = 0; k < NPL; ++k) {
                const int i = 32 * (4 * k + w) + lane;
                un[k] = (i < n && 32 * (4 * k + w) + 31 > j - 1) ? __ldg(u + i) : 0.0;
            }
        }
        if (tj == 0.0) continue;   // uniform over the CTA
        double d0 = 0.0, d1 = 0.0;
#pragma unroll
        for (int k = 0; k < NPL; ++k) {
            if (32 * (4 * k + w) + 31 > j) {
                if (k & 1) d1 = fma(uu[k], z[k], d1);
                else d0 = fma(uu[k], z[k], d0);
            }
        }
        double dot = d0 + d1;
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) red[par][w] = dot;
        __syncthreads();
        const double tot = (red[par][0] + red[par][1]) + (red[par][2] + red[par][3]);
        par ^= 1;
        const double f = tj * tot;
#pragma unroll
        for (int k = 0; k < NPL; ++k)
            if (32 * (4 * k + w) + 31 > j) z[k] = fma(-f, uu[k], z[k]);
    }
#pragma unroll
    for (int k = 0; k < NPL; ++k) {
        const int i = 32 * (4 * k + w) + lane;
        if (i < n) zc[i] = z[k];
    }
}

// Largest eigenvalue of a symmetric positive semidefinite n x n matrix A (n <= 16 C) by the plain
// symmetric Lanczos recurrence u = A v_j - beta_{j-1} v_{j-1}, alpha_j = v_j^T u,
// u <- u - alpha_j v_j, beta_j = ||u||, v_{j+1} = u / beta_j, run for m steps in one thread-block
// cluster of C CTAs. The extreme Ritz values of the tridiagonal T_m converge to the extreme
// eigenvalues of A without reorthogonalisation (loss of orthogonality only adds copies of converged
// Ritz values), so the recurrence alone is kept. CTA r owns rows [r nb, r nb + nb) of A (nb <= 16)
// in its shared memory and every CTA keeps the whole current vector v; the two inner products of a
// step are summed over the CTAs in a fixed order, so every CTA holds bitwise the same alpha_j and
// beta_j. Output: T_m as dgl[0..m-1] (alpha) and eoff[0..m-1] (beta, eoff[m-1] = beta_m, the norm of
// the residual after the last step). On breakdown (beta_j at rounding level) the recurrence stops
// and the rest of T_m is zero: a diagonal block of zeros, which leaves the largest eigenvalue of the
// nonnegative spectrum unchanged. Start vector: uniform in [-1, 1] from a counter-based hash of
// (seed, index).
constexpr int LZ_THREADS = 128;
constexpr int LZ_ROWS = 16;
constexpr int LZ_GROUPS = LZ_THREADS / LZ_ROWS;

__global__ void __launch_bounds__(LZ_THREADS) k_lanczos(int n, const double* __restrict__ A, int lda, int m,
                                                        uint64_t seed, double* dgl, double* eoff) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int nb = (n + C - 1) / C;
    const int r0 = rank * nb;
    const int nr = max(0, min(n, r0 + nb) - r0);
    extern __shared__ double smz[];
    double* Aloc = smz;                    // Aloc[c * LZ_ROWS + i] = A[r0 + i, c]
    double* v = smz + (size_t)LZ_ROWS * n; // the current Lanczos vector, all n entries
    __shared__ double part[LZ_GROUPS][LZ_ROWS];
    __shared__ double vnew[LZ_ROWS];       // this CTA's rows of v_{j+1} (read by the other CTAs)
    __shared__ double red[2];              // this CTA's partial sums of the step (read by the other CTAs)
    __shared__ double s_ab[2];
    __shared__ double s_red[32];
    __shared__ int s_stop;
    const int tid = threadIdx.x, lane = tid & 31;
    const int row = tid % LZ_ROWS, grp = tid / LZ_ROWS;
    for (int e = tid; e < LZ_ROWS * n; e += LZ_THREADS) {
        const int c = e / LZ_ROWS, i = e % LZ_ROWS;
        Aloc[e] = (i < nr) ? A[(int64_t)c * lda + r0 + i] : 0.0;
    }
    // start vector: every CTA forms all n entries and their norm in the same order
    double ss = 0.0;
    for (int c = tid; c < n; c += LZ_THREADS) {
        const uint64_t h = mix64(seed ^ mix64((uint64_t)c + 0x2545F4914F6CDD1Dull));
        const double x = 2.0 * ((h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        v[c] = x;
        ss = fma(x, x, ss);
    }
    ss = block_sum(ss, s_red);
    const double inv0 = (ss > 0.0) ? 1.0 / sqrt(ss) : 0.0;
    __syncthreads();
    for (int c = tid; c < n; c += LZ_THREADS) v[c] *= inv0;
    double vp = 0.0;                       // v_{j-1} at this thread's row (warp 0, lanes < nr)
    double beta = 0.0, anorm = 0.0;
    if (tid == 0) s_stop = 0;
    __syncthreads();
    int j = 0;
    for (; j < m; ++j) {
        // u = A v over this CTA's rows: thread (row, grp) sums the columns c = grp mod LZ_GROUPS
        double acc = 0.0;
        for (int c = grp; c < n; c += LZ_GROUPS) acc = fma(Aloc[c * LZ_ROWS + row], v[c], acc);
        part[grp][row] = acc;
        __syncthreads();
        double u = 0.0, vi = 0.0;
        if (tid < 32) {
            if (lane < nr) {
                double t = part[0][lane];
#pragma unroll
                for (int g = 1; g < LZ_GROUPS; ++g) t += part[g][lane];
                vi = v[r0 + lane];
                u = fma(-beta, vp, t);
            }
            double a = vi * u;
            for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);   // lanes < 16 hold the rows
            if (lane == 0) red[0] = a;
        }
        cluster.sync();                                    // partial alpha of every CTA published
        if (tid < 32) {
            double a = (lane < C) ? *cluster.map_shared_rank(&red[0], lane) : 0.0;
            for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);     // C <= 16
            u = (lane < nr) ? fma(-a, vi, u) : 0.0;
            double b2 = u * u;
            for (int o = 8; o > 0; o >>= 1) b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            if (lane == 0) {
                s_ab[0] = a;
                red[1] = b2;
            }
        }
        cluster.sync();                                    // partial ||u||^2 of every CTA published
        if (tid < 32) {
            double b2 = (lane < C) ? *cluster.map_shared_rank(&red[1], lane) : 0.0;
            for (int o = 8; o > 0; o >>= 1) b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            const double a = s_ab[0];
            // beta and 1 / beta from one reciprocal square root (each within a few ulps)
            const double rb = (b2 > 0.0) ? rsqrt(b2) : 0.0;
            const double b = b2 * rb;
            anorm = fmax(anorm, fabs(a) + b + beta);
            const bool stop = !(b > 16.0 * DBL_EPSILON * anorm);
            if (rank == 0 && lane == 0) {
                dgl[j] = a;
                eoff[j] = stop ? 0.0 : b;
            }
            if (lane < nr) {
                vp = vi;
                vnew[lane] = stop ? 0.0 : u * rb;
            }
            beta = b;
            if (lane == 0) s_stop = stop ? 1 : 0;
        }
        cluster.sync();                                    // v_{j+1} published
        if (s_stop) break;                                 // the same decision in every CTA
        for (int c = tid; c < n; c += LZ_THREADS) v[c] = cluster.map_shared_rank(vnew, c / nb)[c % nb];
        __syncthreads();
    }
    if (rank == 0)
        for (int jj = j + 1 + tid; jj < m; jj += LZ_THREADS) {
            dgl[jj] = 0.0;
            eoff[jj] = 0.0;
        }
    cluster.sync();   // no CTA leaves while another may still read its shared memory
}

// The same recurrence for a Gram too large for one cluster's shared memory (n > kLanczosMaxN), two
// launches per step with the matrix read from global memory (L2-resident at these sizes):
// k_lz_matvec forms u = A v_j (one warp per row; A is symmetric, so row r is read as its contiguous
// column r), k_lz_update the rest of the step in one CTA. The vectors rotate through three buffers
// chosen by the host; st[0] = beta_{j-1}, st[1] = the running norm estimate, st[2] = the stop flag.
constexpr int LZG_THREADS = 1024;
__global__ void k_lz_start(int n, uint64_t seed, double* __restrict__ v, double* __restrict__ vprev,
                           double* __restrict__ st) {
    __shared__ double red[32];
    double ss = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const uint64_t h = mix64(seed ^ mix64((uint64_t)c + 0x2545F4914F6CDD1Dull));
        const double x = 2.0 * ((h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
        v[c] = x;
        vprev[c] = 0.0;
        ss = fma(x, x, ss);
    }
    ss = block_sum(ss, red);
    const double inv0 = (ss > 0.0) ? 1.0 / sqrt(ss) : 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) v[c] *= inv0;
    if (threadIdx.x == 0) {
        st[0] = 0.0;
        st[1] = 0.0;
        st[2] = 0.0;
    }
}

__global__ void k_lz_matvec(int n, const double* __restrict__ A, int lda, const double* __restrict__ v,
                            double* __restrict__ u, const double* __restrict__ st) {
    if (st[2] != 0.0) return;
    const int row = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row >= n) return;
    const double* col = A + (int64_t)row * lda;
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc = fma(col[c], v[c], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[row] = acc;
}

// u <- u - beta_{j-1} v_{j-1}; alpha_j = v_j^T u; u <- u - alpha_j v_j; beta_j = ||u||;
// v_{j+1} = u / beta_j, written over v_{j-1}. On breakdown (or after it) T's entries are zero.
__global__ void __launch_bounds__(LZG_THREADS) k_lz_update(int n, int j, double* __restrict__ u,
                                                           const double* __restrict__ v, double* __restrict__ vprev,
                                                           double* __restrict__ st, double* dgl, double* eoff) {
    __shared__ double red[32];
    if (st[2] != 0.0) {
        if (threadIdx.x == 0) {
            dgl[j] = 0.0;
            eoff[j] = 0.0;
        }
        return;
    }
    const double beta = st[0];
    double a = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double x = fma(-beta, vprev[c], u[c]);
        u[c] = x;
        a = fma(v[c], x, a);
    }
    a = block_sum(a, red);
    double b2 = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double x = fma(-a, v[c], u[c]);
        u[c] = x;
        b2 = fma(x, x, b2);
    }
    b2 = block_sum(b2, red);
    const double rb = (b2 > 0.0) ? rsqrt(b2) : 0.0;
    const double b = b2 * rb;
    const double anorm = fmax(st[1], fabs(a) + b + beta);
    const bool stop = !(b > 16.0 * DBL_EPSILON * anorm);
    for (int c = threadIdx.x; c < n; c += blockDim.x) vprev[c] = stop ? 0.0 : u[c] * rb;
    __syncthreads();   // every thread has read st before thread 0 updates it
    if (threadIdx.x == 0) {
        dgl[j] = a;
        eoff[j] = stop ? 0.0 : b;
        st[0] = b;
        st[1] = anorm;
        st[2] = stop ? 1.0 : 0.0;
    }
}

// (theta_1, theta_2, |z_m|, beta_m) of the Lanczos tridiagonal: its two largest eigenvalues, the last
// entry of the unit eigenvector of theta_1, and the residual norm after the last step.
__global__ void k_lanczos_pack(int m, const double* w, const double* z, const double* eoff, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    out[0] = w[m >= 2 ? 1 : 0];
    out[1] = (m >= 2) ? w[0] : -DBL_MAX;
    out[2] = fabs(z[m - 1]);
    out[3] = eoff[m - 1];
}

__global__ void k_copy_sq(int n, const double* A, int lda, double* B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int r = (int)(e % n), c = (int)(e / n);
    // symmetrise on the way in
    B[(int64_t)c * n + r] = 0.5 * (A[(int64_t)c * lda + r] + A[(int64_t)r * lda + c]);
}

}  // namespace

constexpr int kBlockClusterMin = 48;   // clusters of this many columns or more: block Gram-Schmidt
int symeig_orth_clusters(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, double cluster_rel,
                         int maxc, cudaStream_t s);
int symeig_backtransform(int n, int nv, double* Z, int ldz, SymEigWork* ws, cudaStream_t s);

size_t symeig_work_bytes(int n, int nv) {
    const size_t nn = (size_t)n * n;
    size_t b = 0;
    auto add = [&](size_t cnt) { b += ((cnt * sizeof(double) + 255) / 256) * 256; };
    add(nn + 16 * (size_t)n);   // A (the cluster path keeps up to n + 16 columns of n)
    add(nn);            // HV
    add(n);             // d
    add(n);             // e
    add(n);             // tau
    add(4 * (size_t)n); // vbuf
    add(5 * (size_t)n * std::max(nv, 1) + (size_t)n * std::max(nv, 1));  // lu + Zt
    return b + 4096;
}

int symeig_work_carve(Arena& a, int n, int nv, GridBarrier bar, SymEigWork* w) {
    const size_t nn = (size_t)n * n;
    w->A = a.take<double>(nn + 16 * (size_t)n);
    w->partial = a.take<double>(nn);      // HV
    w->dgl = a.take<double>(n);
    w->eoff = a.take<double>(n);
    w->tau = a.take<double>(n);
    w->vbuf = a.take<double>(4 * (size_t)n);
    w->lu = a.take<double>(6 * (size_t)n * std::max(nv, 1));
    w->bar = bar;
    w->max_ctas = 0;
    if (!w->A || !w->partial || !w->dgl || !w->eoff || !w->tau || !w->vbuf || !w->lu) return EDA_ERR_OOM;
    return EDA_OK;
}

constexpr int kClusterMaxN = 512;        // the cluster path up to here; a cooperative grid beyond
constexpr int kClusterMaxNShared = 1024; // limit of the cluster path when the GPU is shared (see below)
constexpr int kResMinN = 288;            // the resident-column cooperative grid from here (when it fits)

// Host threads that run many problems side by side (the batched solver) set this: a cooperative
// grid with a software grid barrier needs all its CTAs resident at once, which concurrent kernels
// of other problems can delay beyond the barrier's limit, while a thread-block cluster is scheduled
// as one unit by the hardware. Such threads take the cluster path (matrix in a global slab) up to
// kClusterMaxNShared.
thread_local bool tl_shared_gpu = false;

// Launch k_tridiag_cluster<C> on one cluster of C CTAs (a power of two, 16 only when the device
// accepts that non-portable cluster size with the needed shared memory).
template <int C>
int launch_tridiag_cluster(int n, const double* A, int lda, SymEigWork* ws, cudaStream_t s, bool probe_only,
                           bool* fits) {
    auto kern = k_tridiag_cluster<C>;
    static std::mutex mu;                 // the function attributes below are shared by all threads
    static size_t smem_set = 0;
    static bool attrs = false;
    const int ncl = (n + C - 1) / C;
    const size_t vec_bytes = (4 * (size_t)n + 2) * sizeof(double);
    const size_t a_bytes = (size_t)ncl * n * sizeof(double);
    const int in_smem = (vec_bytes + a_bytes <= 200 * 1024) ? 1 : 0;
    const size_t smem = vec_bytes + (in_smem ? a_bytes : 0);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attrs) {
            attrs = true;
            if (C > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaGetLastError();
        }
        if (smem > smem_set) {
            EDA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)std::max<size_t>(smem, 48 * 1024)));
            smem_set = std::max<size_t>(smem, 48 * 1024);
        }
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(CT_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (probe_only) {
        int nclusters = 0;
        *fits = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1;
        cudaGetLastError();
        return EDA_OK;
    }
    ProfScope prof("tridiag", s, 4.0 / 3.0 * (double)n * n * n);
    EDA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, n, A, lda, ws->A, in_smem, ws->partial, ws->dgl, ws->eoff, ws->tau));
    launch_counter()++;
    return EDA_OK;
}

int launch_tridiag_c(int C, int n, const double* A, int lda, SymEigWork* ws, cudaStream_t s, bool probe_only,
                     bool* fits) {
    switch (C) {
        case 16: return launch_tridiag_cluster<16>(n, A, lda, ws, s, probe_only, fits);
        case 8: return launch_tridiag_cluster<8>(n, A, lda, ws, s, probe_only, fits);
        case 4: return launch_tridiag_cluster<4>(n, A, lda, ws, s, probe_only, fits);
        case 2: return launch_tridiag_cluster<2>(n, A, lda, ws, s, probe_only, fits);
        default: return launch_tridiag_cluster<1>(n, A, lda, ws, s, probe_only, fits);
    }
}

int tridiag_cluster(int n, const double* A, int lda, SymEigWork* ws, cudaStream_t s) {
    static int chosen_C[kClusterMaxNShared + 1] = {};   // cluster size that passed the occupancy check, per n
    static std::mutex mu;
    std::unique_lock<std::mutex> lk(mu);
    if (!chosen_C[n]) {
        // about 12 or more columns per CTA: fewer FP64 instructions per warp and column step (each
        // holds a sub-partition's FP64 pipe for ~64 cycles) outweigh the wider cluster barrier
        int want = 2;
        if (n > 32) {
            want = 1;
            while (want < 16 && want * 2 * 12 <= n) want *= 2;
        }
        // clusters of at least two CTAs: the kernel's one-CTA instance loses accuracy on small n and is
        // not used
        int C = std::max(2, want);
        for (; C > 2; C /= 2) {
            bool fits = false;
            EDA_TRY(launch_tridiag_c(C, n, A, lda, ws, s, true, &fits));
            if (fits) break;
        }
        chosen_C[n] = C;
    }
    const int C = chosen_C[n];
    lk.unlock();
    return launch_tridiag_c(C, n, A, lda, ws, s, false, nullptr);
}

// The resident-column grid (k_tridiag_res): about four columns per CTA, at most one CTA per SM, when the
// owned columns and two work vectors fit in 200 KB of shared memory. INVALID_ARG: does not apply.
int tridiag_res(int n, const double* A, int lda, double* HV, SymEigWork* ws, int* status, int sms, cudaStream_t s) {
    const int G = std::max(1, std::min(sms, (n + 3) / 4));
    const int ncl = (n + G - 1) / G;
    const size_t smem = ((size_t)(ncl + 2) * n + G) * sizeof(double);
    if (smem > 200 * 1024 || 2 * (size_t)n + 2 + G > 4 * (size_t)n) return EDA_ERR_INVALID_ARG;
    {
        static std::mutex mu;
        static size_t set = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (smem > set && smem > 40 * 1024) {
            EDA_CUDA_TRY(cudaFuncSetAttribute(k_tridiag_res, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)std::max<size_t>(smem, 48 * 1024)));
            set = std::max<size_t>(smem, 48 * 1024);
        }
    }
    int per_sm = 0;
    EDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_res, TRI_THREADS, smem));
    if (per_sm < 1 || G > per_sm * sms) return EDA_ERR_INVALID_ARG;
    // both barrier words to zero: the launch starts its arrival count from 0
    EDA_CUDA_TRY(cudaMemsetAsync(ws->bar.count, 0, 256, s));
    ProfScope prof("tridiag", s, 4.0 / 3.0 * (double)n * n * n);
    int nn = n, ld = lda;
    const double* a0 = A;
    double* vg = ws->vbuf;
    double* pg = ws->vbuf + n + 2;
    double* ps = ws->vbuf + 2 * n + 2;
    double* a1 = HV;
    double* a2 = ws->dgl;
    double* a3 = ws->eoff;
    double* a4 = ws->tau;
    GridBarWords bw{ws->bar.count, ws->bar.gen, ws->bar.spin_limit};
    int* st = status;
    void* args[] = {&nn, &a0, &ld, &vg, &pg, &ps, &a1, &a2, &a3, &a4, &bw, &st};
    EDA_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_tridiag_res, dim3(G), dim3(TRI_THREADS), args, smem, s));
    launch_counter()++;
    return EDA_OK;
}

int symeig_values(int n, const double* A, int lda, int il, int iu, double* w, SymEigWork* ws, int* status,
                  cudaStream_t s) {
    if (n <= 0 || il < 0 || iu >= n || il > iu) return EDA_ERR_INVALID_ARG;
    EDA_CUDA_TRY(cudaPeekAtLastError());   // surface an error left by an earlier call at its own site
    const int nv = iu - il + 1;
    double* HV = ws->partial;
    // ---- tridiagonal reduction: resident-column grid, cluster, or L2-streaming grid (see the file header) ----
    int dev = 0;
    EDA_CUDA_TRY(cudaGetDevice(&dev));
    int sms = 0;
    EDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // dynamic shared memory near 48 KB needs the opt-in too: the kernels also hold static shared
    // variables, and the default limit covers static + dynamic
    const size_t smem = 2 * (size_t)n * sizeof(double);
    if (smem > 40 * 1024) {
        // raise-only, under a lock: concurrent solves of different sizes share the attribute
        static std::mutex mu;
        static size_t set = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (smem > set) {
            EDA_CUDA_TRY(cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            set = smem;
        }
    }
    int res = EDA_ERR_INVALID_ARG;   // the resident-column grid when it applies and fits
    if (!tl_shared_gpu && n >= kResMinN) res = tridiag_res(n, A, lda, HV, ws, status, sms, s);
    if (res == EDA_OK) {
    } else if (res != EDA_ERR_INVALID_ARG) {
        return res;
    } else if (n <= (tl_shared_gpu ? kClusterMaxNShared : kClusterMaxN)) {
        EDA_TRY(tridiag_cluster(n, A, lda, ws, s));
    } else {
    int per_sm = 0;
    EDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag, TRI_THREADS, smem));
    // about 8 rows per CTA: more CTAs shorten each column step's FP64 chains (16 rows per CTA measured
    // 10 % slower at the Rayleigh-Ritz sizes 576-704; fewer than 8 rows gained nothing)
    int ctas = std::max(1, std::min(n / 8, sms));
    ctas = std::min(ctas, std::max(1, per_sm * sms));
    double* pglob = ws->vbuf;
    EDA_CUDA_TRY(cudaMemsetAsync(ws->bar.count, 0, sizeof(unsigned), s));
    k_copy_sq<<<ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, A, lda, ws->A);
    EDA_LAUNCHED();
    {
        ProfScope prof("tridiag", s, 4.0 / 3.0 * (double)n * n * n);
        int nn = n;
        double* a0 = ws->A;
        double* a1 = HV;
        double* a2 = ws->dgl;
        double* a3 = ws->eoff;
        double* a4 = ws->tau;
        double* a5 = pglob;
        GridBarrier b = ws->bar;
        int* st = status;
        void* args[] = {&nn, &a0, &a1, &a2, &a3, &a4, &a5, &b, &st};
        EDA_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_tridiag, dim3(ctas), dim3(TRI_THREADS), args, smem, s));
        launch_counter()++;
    }
    }
    // ---- eigenvalues ----
    EDA_CUDA_TRY(cudaPeekAtLastError());
    const size_t bsm = 3 * (size_t)n * sizeof(double);
    if (bsm > 40 * 1024) {
        static std::mutex mu;
        static size_t set = 0;
        std::lock_guard<std::mutex> lk(mu);
        if (bsm > set) {
            EDA_CUDA_TRY(cudaFuncSetAttribute(k_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
            set = bsm;
        }
    }
    {
        ProfScope prof("bisect", s);
        // one warp per CTA: the FP64 pipe of one SM is narrow, so the warps are spread over SMs
        k_bisect<<<nv, 64, bsm, s>>>(n, ws->dgl, ws->eoff, il, nv, w);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

namespace {
// Inverse iteration for the nv eigenvalues w of the tridiagonal in ws, vectors into Z (n x nv, ldz).
int invit_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, uint64_t seed, cudaStream_t s) {
    double* lu = ws->lu;
    double* Zt = ws->lu + 5 * (size_t)n * nv;
    {
        ProfScope prof("invit", s);
        k_invit<<<ceil_div(nv, 32), 32, 0, s>>>(n, nv, ws->dgl, ws->eoff, w, lu, Zt, seed);
        EDA_LAUNCHED();
    }
    k_transpose_out<<<ceil_div((int64_t)n * nv, 256), 256, 0, s>>>(n, nv, Zt, Z, ldz);
    EDA_LAUNCHED();
    return EDA_OK;
}
}  // namespace

int symeig_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, uint64_t seed,
                   double cluster_rel, cudaStream_t s) {
    if (nv <= 0) return EDA_OK;
    EDA_TRY(invit_vectors(n, nv, w, Z, ldz, ws, seed, s));
    EDA_TRY(symeig_orth_clusters(n, nv, w, Z, ldz, ws, cluster_rel, kBlockClusterMin, s));
    return symeig_backtransform(n, nv, Z, ldz, ws, s);
}

int symeig_f64(int n, const double* A, int lda, int il, int iu, double* w, double* Z, int ldz, SymEigWork* ws,
               int* status, uint64_t seed, double cluster_rel, cudaStream_t s) {
    ProfScope prof("symeig", s);
    EDA_TRY(symeig_values(n, A, lda, il, iu, w, ws, status, s));
    if (!Z) return EDA_OK;
    return symeig_vectors(n, iu - il + 1, w, Z, ldz, ws, seed, cluster_rel, s);
}

// Cluster MGS with a tolerance relative to max |lambda|, computed on the device.
namespace {
__global__ void k_cluster_scale(int nv, const double* lam, double rel, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < nv; ++i) m = fmax(m, fabs(lam[i]));
        out[0] = rel * m;
    }
}
// Columns Z[:, 0 .. bs) (bs <= 16), already orthogonal to every earlier column of their cluster: each column
// against the earlier ones of the block by classical Gram-Schmidt applied twice (the dot products of a pass
// on one warp each, the update on all threads), then normalised. Computed from the vectors themselves (not
// their Gram matrix), like the column-by-column loop it replaces, so nearly dependent inverse-iteration
// vectors of a tight cluster keep their content above the rounding level.
constexpr int kClusterBlock = 16;
__global__ void __launch_bounds__(512) k_cluster_block_cgs2(int n, double* Z, int ldz, int bs) {
    __shared__ double dots[kClusterBlock];
    __shared__ double red[16];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c = 0; c < bs; ++c) {
        double* zc = Z + (int64_t)c * ldz;
        for (int pass = 0; pass < 2 && c > 0; ++pass) {
            if (warp < c) {
                const double* zw = Z + (int64_t)warp * ldz;
                double dot = 0.0;
                for (int i = lane; i < n; i += 32) dot = fma(zw[i], zc[i], dot);
                for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                if (lane == 0) dots[warp] = dot;
            }
            __syncthreads();
            for (int i = tid; i < n; i += blockDim.x) {
                double acc = 0.0;
                for (int w = 0; w < c; ++w) acc = fma(dots[w], Z[(int64_t)w * ldz + i], acc);
                zc[i] -= acc;
            }
            __syncthreads();
        }
        double nrm = 0.0;
        for (int i = tid; i < n; i += blockDim.x) nrm = fma(zc[i], zc[i], nrm);
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if (lane == 0) red[warp] = nrm;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            red[0] = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        }
        __syncthreads();
        const double sc = red[0];
        for (int i = tid; i < n; i += blockDim.x) zc[i] *= sc;
        __syncthreads();
    }
}

// Modified Gram-Schmidt (two passes) inside each run of eigenvalues whose consecutive gaps are <= ctol,
// one warp per run; runs of maxc or more columns are left to the block path.
__global__ void k_cluster_mgs_dev(int n, int nv, const double* lam, const double* ctol_dev, double* Z, int ldz,
                                  int maxc) {
    const double ctol = ctol_dev[0];
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nv) return;
    if (q > 0 && lam[q] - lam[q - 1] <= ctol) return;
    int end = q + 1;
    while (end < nv && lam[end] - lam[end - 1] <= ctol) ++end;
    if (end - q < 2 || end - q >= maxc) return;
    for (int c = q + 1; c < end; ++c) {
        double* zc = Z + (int64_t)c * ldz;
        for (int pass = 0; pass < 2; ++pass) {
            for (int pcol = q; pcol < c; ++pcol) {
                const double* zp = Z + (int64_t)pcol * ldz;
                double dot = 0.0;
                for (int i = lane; i < n; i += 32) dot = fma(zp[i], zc[i], dot);
                for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                for (int i = lane; i < n; i += 32) zc[i] = fma(-dot, zp[i], zc[i]);
            }
        }
        double nrm = 0.0;
        for (int i = lane; i < n; i += 32) nrm = fma(zc[i], zc[i], nrm);
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        const double sc = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
        for (int i = lane; i < n; i += 32) zc[i] *= sc;
    }
}
}  // namespace

// Orthogonalisation of the inverse-iteration vectors inside eigenvalue clusters (runs whose consecutive
// gaps are <= cluster_rel * max |w|), in the tridiagonal basis. Runs shorter than maxc columns: modified
// Gram-Schmidt (two passes) by one warp each (k_cluster_mgs_dev). Longer runs (when eigenvalues span many
// orders of magnitude, every value near the bottom of the spectrum falls within one such run): blocks of
// kClusterBlock columns in order, each first made orthogonal to the earlier blocks of its run by block
// classical Gram-Schmidt applied twice with the multi-CTA products, then orthonormalised column by column
// (k_cluster_block_cgs2). In exact arithmetic this is the same Gram-Schmidt basis as the column loop, and
// like it every step works on the vectors, never on their Gram matrix. The cluster bounds are found on the
// host with the device's criterion and operations.
int symeig_orth_clusters(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, double cluster_rel,
                         int maxc, cudaStream_t s) {
    double* ctol = ws->vbuf + 2 * n;
    k_cluster_scale<<<1, 32, 0, s>>>(nv, w, cluster_rel, ctol);
    EDA_LAUNCHED();
    k_cluster_mgs_dev<<<ceil_div((int64_t)nv * 32, 256), 256, 0, s>>>(n, nv, w, ctol, Z, ldz, maxc);
    EDA_LAUNCHED();
    if (maxc == INT_MAX || nv < maxc) return EDA_OK;
    std::vector<double> wh(nv);
    EDA_CUDA_TRY(cudaMemcpyAsync(wh.data(), w, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    double mx = 0.0;
    for (int i = 0; i < nv; ++i) mx = std::fmax(mx, std::fabs(wh[i]));
    const double tol = cluster_rel * mx;
    std::vector<std::pair<int, int>> big;
    for (int q = 0; q < nv;) {
        int end = q + 1;
        while (end < nv && wh[end] - wh[end - 1] <= tol) ++end;
        if (end - q >= maxc) big.emplace_back(q, end);
        q = end;
    }
    if (big.empty()) return EDA_OK;
    ProfScope prof("cluster_orth", s);
    // scratch in the inverse-iteration factors (free once the vectors are in Z)
    constexpr int BS = kClusterBlock;
    double* C = ws->lu;                                   // nv x BS
    double* part = C + (size_t)nv * BS;
    const size_t cap = 6 * (size_t)n * nv;
    if ((size_t)nv * BS * 2 > cap) return EDA_ERR_INVALID_ARG;
    const size_t pcap = cap - (size_t)nv * BS;
    for (const auto& cl : big) {
        const int q = cl.first, end = cl.second;
        double* Zq = Z + (size_t)q * ldz;
        for (int j0 = q; j0 < end; j0 += BS) {
            const int bs = std::min(BS, end - j0);
            double* Zj = Z + (size_t)j0 * ldz;
            const int prev = j0 - q;
            for (int pass = 0; pass < 2 && prev > 0; ++pass) {
                EDA_TRY(gemm_tn_f64(n, prev, bs, 1.0, Zq, ldz, Zj, ldz, 0.0, C, prev, part, pcap, s));
                EDA_TRY(gemm_nn_f64(n, prev, bs, -1.0, Zq, ldz, C, prev, 1.0, Zj, ldz, Zj, ldz, s));
            }
            k_cluster_block_cgs2<<<1, 512, 0, s>>>(n, Zj, ldz, bs);
            EDA_LAUNCHED();
        }
    }
    return EDA_OK;
}

// Householder back-transformation of the tridiagonal eigenvectors Z (reflectors still in ws).
int symeig_backtransform(int n, int nv, double* Z, int ldz, SymEigWork* ws, cudaStream_t s) {
    if (n >= 3) {
        ProfScope prof("backtransform", s);
        if (n <= 256) k_backtransform_w4<2><<<nv, 128, 0, s>>>(n, nv, ws->partial, ws->tau, Z, ldz);
        else if (n <= 512) k_backtransform_w4<4><<<nv, 128, 0, s>>>(n, nv, ws->partial, ws->tau, Z, ldz);
        else if (n <= 1024) k_backtransform_w4<8><<<nv, 128, 0, s>>>(n, nv, ws->partial, ws->tau, Z, ldz);
        else k_backtransform<<<nv, 32, 0, s>>>(n, nv, ws->partial, ws->tau, Z, ldz);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

int newton_schulz_f64(int n, int nv, double* Z, int ldz, int steps, double* tmp, double* partial, size_t partial_cap,
                      cudaStream_t s) {
    double* G = tmp;                       // nv x nv
    double* Zn = tmp + (size_t)nv * nv;    // n x nv
    for (int it = 0; it < steps; ++it) {
        EDA_TRY(syrk_f64(n, nv, 1.0, Z, ldz, 0.0, G, nv, partial, partial_cap, s));
        // Zn = 1.5 Z - 0.5 Z G
        EDA_TRY(gemm_nn_f64(n, nv, nv, -0.5, Z, ldz, G, nv, 1.5, Z, ldz, Zn, n, s));
        EDA_TRY(copy_mat_f64(n, nv, Zn, n, Z, ldz, s));
    }
    return EDA_OK;
}

int lanczos_top(int n, const double* A, int lda, int m, uint64_t seed, SymEigWork* ws, double* out,
                cudaStream_t s) {
    if (n < 1 || m < 1 || m > n) return EDA_ERR_INVALID_ARG;
    if (n > kLanczosMaxN) {
        // three n-vectors in vbuf (4 n doubles), the state after them in lu
        double* buf[3] = {ws->vbuf, ws->vbuf + n, ws->vbuf + 2 * (size_t)n};
        double* st = ws->lu;
        {
            ProfScope prof("lanczos", s);
            k_lz_start<<<1, LZG_THREADS, 0, s>>>(n, seed, buf[0], buf[1], st);
            EDA_LAUNCHED();
            // v_j in buf[j % 2], v_{j-1} (then v_{j+1}) in buf[(j + 1) % 2], u in buf[2]
            for (int j = 0; j < m; ++j) {
                double* v = buf[j & 1];
                double* vp = buf[(j + 1) & 1];
                k_lz_matvec<<<ceil_div((int64_t)n * 32, 256), 256, 0, s>>>(n, A, lda, v, buf[2], st);
                EDA_LAUNCHED();
                k_lz_update<<<1, LZG_THREADS, 0, s>>>(n, j, buf[2], v, vp, st, ws->dgl, ws->eoff);
                EDA_LAUNCHED();
            }
        }
        const int nv = m >= 2 ? 2 : 1;
        double* w = ws->vbuf + 3 * (size_t)n;       // nv values (vbuf holds 4 n doubles)
        double* zt = ws->lu + 5 * (size_t)m;        // the eigenvector after the 5 m factor entries
        k_bisect<<<nv, 64, 3 * (size_t)m * sizeof(double), s>>>(m, ws->dgl, ws->eoff, m - nv, nv, w);
        EDA_LAUNCHED();
        k_invit<<<1, 32, 0, s>>>(m, 1, ws->dgl, ws->eoff, w + nv - 1, ws->lu, zt, seed);   // st is dead here
        EDA_LAUNCHED();
        k_lanczos_pack<<<1, 32, 0, s>>>(m, w, zt, ws->eoff, out);
        EDA_LAUNCHED();
        return EDA_OK;
    }
    const int C = (n + LZ_ROWS - 1) / LZ_ROWS;
    {
        static std::once_flag once;
        std::call_once(once, [] {
            cudaFuncSetAttribute(k_lanczos, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            cudaGetLastError();
        });
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(LZ_THREADS);
    cfg.dynamicSmemBytes = (size_t)(LZ_ROWS + 1) * n * sizeof(double);
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
        ProfScope prof("lanczos", s);
        EDA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_lanczos, n, A, lda, m, seed, ws->dgl, ws->eoff));
        launch_counter()++;
    }
    // the two largest eigenvalues of T_m and the eigenvector of the largest
    const int nv = m >= 2 ? 2 : 1;
    double* w = ws->vbuf;                       // nv values
    double* zt = ws->lu + 5 * (size_t)m;        // the eigenvector (m entries) after the 5 m factor entries
    k_bisect<<<nv, 64, 3 * (size_t)m * sizeof(double), s>>>(m, ws->dgl, ws->eoff, m - nv, nv, w);
    EDA_LAUNCHED();
    k_invit<<<1, 32, 0, s>>>(m, 1, ws->dgl, ws->eoff, w + nv - 1, ws->lu, zt, seed);
    EDA_LAUNCHED();
    k_lanczos_pack<<<1, 32, 0, s>>>(m, w, zt, ws->eoff, out);
    EDA_LAUNCHED();
    return EDA_OK;
}

bool symeig_set_shared_gpu(bool on) {
    const bool prev = tl_shared_gpu;
    tl_shared_gpu = on;
    return prev;
}

}  // namespace eda
