// FP64 symmetric eigensolver for the small matrices of the method: the Gram matrices
// G = H^T H (the spectra D = Sigma^2 of Eq. 3.11-3.13) and the block-tridiagonal Lanczos
// matrix T of the Rayleigh-Ritz step.
//
// Route: Householder reduction to tridiagonal form (one cooperative launch, rows owned
// cyclically by CTAs, two bounded grid barriers per column) -> eigenvalues by 33-way
// multisection on Sturm counts (one warp per eigenvalue) -> eigenvectors of the tridiagonal
// by inverse iteration with partial pivoting (one thread per eigenvector) -> modified
// Gram-Schmidt inside tight clusters (one warp per cluster) -> back-transformation with the
// stored reflectors. Callers add a Newton-Schulz step for orthogonality across near clusters.
#include "eda_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>

namespace eda {

namespace {

constexpr int TRI_THREADS = 256;
constexpr long long SPIN_LIMIT = 20000000;   // ~1-2 s of polling before a barrier gives up

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
                if (++it > SPIN_LIMIT) {
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
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    const int nw = blockDim.x >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];   // same fixed order in every thread and CTA
    return s;
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

// Number of eigenvalues of the tridiagonal (dgl, e2 = squared off-diagonal) below x.
__device__ int sturm_count(int n, const double* dgl, const double* e2, double x, double pivmin) {
    int cnt = 0;
    double q = dgl[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += (q < 0.0);
    for (int i = 1; i < n; ++i) {
        q = (dgl[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += (q < 0.0);
    }
    return cnt;
}

// One warp per wanted eigenvalue (ascending index il + warp id): 33-way multisection.
__global__ void k_bisect(int n, const double* dgl, const double* eoff, double* e2, int il, int nw, double* w) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nw) return;
    const int idx = il + gw;
    // Gershgorin interval and pivmin, computed by the warp
    double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double el = (i > 0) ? fabs(eoff[i - 1]) : 0.0;
        const double er = (i + 1 < n) ? fabs(eoff[i]) : 0.0;
        lo = fmin(lo, dgl[i] - el - er);
        hi = fmax(hi, dgl[i] + el + er);
        if (i + 1 < n) emax = fmax(emax, er * er);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    }
    const double tnorm = fmax(fabs(lo), fabs(hi));
    const double pivmin = DBL_MIN * fmax(1.0, emax);
    lo -= 2.0 * DBL_EPSILON * tnorm + pivmin;
    hi += 2.0 * DBL_EPSILON * tnorm + pivmin;
    for (int round = 0; round < 24; ++round) {
        const double width = hi - lo;
        if (width <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) || width <= 0.05 * DBL_EPSILON * tnorm) break;
        const double x = lo + (lane + 1) * (width / 33.0);
        const int cnt = sturm_count(n, dgl, e2, x, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, cnt > idx);
        if (above == 0u) {
            lo = __shfl_sync(0xffffffffu, x, 31);
        } else {
            const int l = __ffs(above) - 1;
            const double xl = __shfl_sync(0xffffffffu, x, l);
            const double xp = __shfl_sync(0xffffffffu, x, l > 0 ? l - 1 : 0);
            if (l > 0) lo = xp;
            hi = xl;
        }
    }
    if (lane == 0) w[gw] = 0.5 * (lo + hi);
}

__global__ void k_square_off(int n, const double* eoff, double* e2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) e2[i] = (i + 1 < n) ? eoff[i] * eoff[i] : 0.0;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Inverse iteration, one thread per eigenvector; factor arrays laid out [array][i][q] so that
// the threads of a warp touch consecutive addresses. Output: Zt[i][q] (n x nv, row stride nv).
__global__ void k_invit(int n, int nv, const double* dgl, const double* eoff, const double* lam, double* lu,
                        double* Zt, uint64_t seed) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nv) return;
    const int64_t S = nv;
    double* DL = lu;
    double* D = lu + (int64_t)n * S;
    double* DU = lu + 2 * (int64_t)n * S;
    double* DU2 = lu + 3 * (int64_t)n * S;
    double* PIV = lu + 4 * (int64_t)n * S;     // 0 / 1 flags stored as doubles
    double* x = Zt;
    const double l = lam[q];
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i)
        tnorm = fmax(tnorm, fabs(dgl[i]) + ((i > 0) ? fabs(eoff[i - 1]) : 0.0) + ((i + 1 < n) ? fabs(eoff[i]) : 0.0));
    const double tiny = fmax(DBL_EPSILON * tnorm, DBL_MIN);
    for (int i = 0; i < n; ++i) {
        D[i * S + q] = dgl[i] - l;
        if (i + 1 < n) {
            DL[i * S + q] = eoff[i];
            DU[i * S + q] = eoff[i];
        }
        DU2[i * S + q] = 0.0;
        PIV[i * S + q] = 0.0;
    }
    // Gaussian elimination with partial pivoting on T - lambda I
    for (int i = 0; i + 1 < n; ++i) {
        const double di = D[i * S + q], dli = DL[i * S + q];
        if (fabs(di) >= fabs(dli)) {
            const double dd = (di == 0.0) ? tiny : di;
            D[i * S + q] = dd;
            const double f = dli / dd;
            DL[i * S + q] = f;
            D[(i + 1) * S + q] -= f * DU[i * S + q];
        } else {
            const double f = di / dli;
            D[i * S + q] = dli;
            DL[i * S + q] = f;
            const double tmp = DU[i * S + q];
            DU[i * S + q] = D[(i + 1) * S + q];
            D[(i + 1) * S + q] = tmp - f * D[(i + 1) * S + q];
            if (i + 2 < n) {
                DU2[i * S + q] = DU[(i + 1) * S + q];
                DU[(i + 1) * S + q] = -f * DU[(i + 1) * S + q];
            }
            PIV[i * S + q] = 1.0;
        }
    }
    if (D[(int64_t)(n - 1) * S + q] == 0.0) D[(int64_t)(n - 1) * S + q] = tiny;
    // random start in [-1, 1]
    for (int i = 0; i < n; ++i) {
        const uint64_t h = mix64(seed ^ mix64(((uint64_t)q << 32) + (uint64_t)i + 0x5851F42D4C957F2Dull));
        x[i * S + q] = 2.0 * ((h >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    for (int it = 0; it < 3; ++it) {
        // forward: L^{-1} P b
        for (int i = 0; i + 1 < n; ++i) {
            const double f = DL[i * S + q];
            if (PIV[i * S + q] == 0.0) {
                x[(i + 1) * S + q] -= f * x[i * S + q];
            } else {
                const double t0 = x[i * S + q];
                x[i * S + q] = x[(i + 1) * S + q];
                x[(i + 1) * S + q] = t0 - f * x[i * S + q];
            }
        }
        // back: U^{-1}
        double mx = 0.0;
        for (int i = n - 1; i >= 0; --i) {
            double v = x[i * S + q];
            if (i + 1 < n) v -= DU[i * S + q] * x[(i + 1) * S + q];
            if (i + 2 < n) v -= DU2[i * S + q] * x[(i + 2) * S + q];
            v /= D[i * S + q];
            x[i * S + q] = v;
            mx = fmax(mx, fabs(v));
        }
        const double sc = (mx > 0.0 && isfinite(mx)) ? 1.0 / mx : 0.0;
        for (int i = 0; i < n; ++i) x[i * S + q] *= sc;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm = fma(x[i * S + q], x[i * S + q], nrm);
    const double sc = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
    for (int i = 0; i < n; ++i) x[i * S + q] *= sc;
}

// Zt (row-major n x nv) -> Z (column-major, ldz)
__global__ void k_transpose_out(int n, int nv, const double* Zt, double* Z, int ldz) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * nv) return;
    const int i = (int)(e % n), q = (int)(e / n);
    Z[(int64_t)q * ldz + i] = Zt[(int64_t)i * nv + q];
}

// Z <- H_0 H_1 ... H_{n-3} Z; each CTA owns 8 columns, the reflector is staged in shared memory.
__global__ void k_backtransform(int n, int nv, const double* HV, const double* tau, double* Z, int ldz) {
    extern __shared__ double u[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = blockIdx.x * (blockDim.x >> 5) + warp;
    for (int j = n - 3; j >= 0; --j) {
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) u[i] = HV[(int64_t)j * n + i];
        __syncthreads();
        const double tj = tau[j];
        if (col >= nv || tj == 0.0) continue;
        double* z = Z + (int64_t)col * ldz;
        double dot = 0.0;
        for (int i = j + 1 + lane; i < n; i += 32) dot = fma(u[i], z[i], dot);
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double f = tj * dot;
        for (int i = j + 1 + lane; i < n; i += 32) z[i] = fma(-f, u[i], z[i]);
    }
}

__global__ void k_copy_sq(int n, const double* A, int lda, double* B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int r = (int)(e % n), c = (int)(e / n);
    // symmetrise on the way in
    B[(int64_t)c * n + r] = 0.5 * (A[(int64_t)c * lda + r] + A[(int64_t)r * lda + c]);
}

}  // namespace

int symeig_finish_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, double cluster_rel,
                          cudaStream_t s);

size_t symeig_work_bytes(int n, int nv) {
    const size_t nn = (size_t)n * n;
    size_t b = 0;
    auto add = [&](size_t cnt) { b += ((cnt * sizeof(double) + 255) / 256) * 256; };
    add(nn);            // A
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
    w->A = a.take<double>(nn);
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

int symeig_values(int n, const double* A, int lda, int il, int iu, double* w, SymEigWork* ws, int* status,
                  cudaStream_t s) {
    if (n <= 0 || il < 0 || iu >= n || il > iu) return EDA_ERR_INVALID_ARG;
    const int nv = iu - il + 1;
    double* HV = ws->partial;
    k_copy_sq<<<ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, A, lda, ws->A);
    EDA_LAUNCHED();
    // ---- tridiagonal reduction: cooperative launch ----
    int dev = 0;
    EDA_CUDA_TRY(cudaGetDevice(&dev));
    int sms = 0;
    EDA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = 2 * (size_t)n * sizeof(double);
    if (smem > 48 * 1024) {
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int per_sm = 0;
    EDA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag, TRI_THREADS, smem));
    int ctas = std::max(1, std::min(n / 16, sms));
    ctas = std::min(ctas, std::max(1, per_sm * sms));
    double* pglob = ws->vbuf;
    EDA_CUDA_TRY(cudaMemsetAsync(ws->bar.count, 0, sizeof(unsigned), s));
    {
        ProfScope prof("tridiag", s);
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
    // ---- eigenvalues ----
    double* e2 = ws->vbuf + n;
    k_square_off<<<ceil_div(n, 256), 256, 0, s>>>(n, ws->eoff, e2);
    EDA_LAUNCHED();
    k_bisect<<<ceil_div((int64_t)nv * 32, 256), 256, 0, s>>>(n, ws->dgl, ws->eoff, e2, il, nv, w);
    EDA_LAUNCHED();
    return EDA_OK;
}

int symeig_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, uint64_t seed,
                   double cluster_rel, cudaStream_t s) {
    if (nv <= 0) return EDA_OK;
    double* lu = ws->lu;
    double* Zt = ws->lu + 5 * (size_t)n * nv;
    k_invit<<<ceil_div(nv, 64), 64, 0, s>>>(n, nv, ws->dgl, ws->eoff, w, lu, Zt, seed);
    EDA_LAUNCHED();
    k_transpose_out<<<ceil_div((int64_t)n * nv, 256), 256, 0, s>>>(n, nv, Zt, Z, ldz);
    EDA_LAUNCHED();
    return symeig_finish_vectors(n, nv, w, Z, ldz, ws, cluster_rel, s);
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
__global__ void k_cluster_mgs_dev(int n, int nv, const double* lam, const double* ctol_dev, double* Z, int ldz) {
    const double ctol = ctol_dev[0];
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nv) return;
    if (q > 0 && lam[q] - lam[q - 1] <= ctol) return;
    int end = q + 1;
    while (end < nv && lam[end] - lam[end - 1] <= ctol) ++end;
    if (end - q < 2) return;
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

// Cluster orthogonalisation (tridiagonal basis) and back-transformation; call after symeig_f64
// with the same workspace while the reflectors are still in it.
int symeig_finish_vectors(int n, int nv, const double* w, double* Z, int ldz, SymEigWork* ws, double cluster_rel,
                          cudaStream_t s) {
    double* ctol = ws->vbuf + 2 * n;
    k_cluster_scale<<<1, 32, 0, s>>>(nv, w, cluster_rel, ctol);
    EDA_LAUNCHED();
    k_cluster_mgs_dev<<<ceil_div((int64_t)nv * 32, 256), 256, 0, s>>>(n, nv, w, ctol, Z, ldz);
    EDA_LAUNCHED();
    if (n >= 3) {
        const size_t smem = (size_t)n * sizeof(double);
        if (smem > 48 * 1024) {
            EDA_CUDA_TRY(cudaFuncSetAttribute(k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        }
        k_backtransform<<<ceil_div(nv, 8), 256, smem, s>>>(n, nv, ws->partial, ws->tau, Z, ldz);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

int newton_schulz_f64(int n, int nv, double* Z, int ldz, int steps, double* tmp, double* partial, size_t partial_cap,
                      cudaStream_t s) {
    double* G = tmp;                       // nv x nv
    double* Zn = tmp + (size_t)nv * nv;    // n x nv
    for (int it = 0; it < steps; ++it) {
        EDA_TRY(gemm_tn_f64(n, nv, nv, 1.0, Z, ldz, Z, ldz, 0.0, G, nv, partial, partial_cap, s));
        // Zn = 1.5 Z - 0.5 Z G
        EDA_TRY(gemm_nn_f64(n, nv, nv, -0.5, Z, ldz, G, nv, 1.5, Z, ldz, Zn, n, s));
        EDA_TRY(copy_mat_f64(n, nv, Zn, n, Z, ldz, s));
    }
    return EDA_OK;
}

}  // namespace eda
