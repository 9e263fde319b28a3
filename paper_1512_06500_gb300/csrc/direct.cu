// Exact solve of the symmetric form in the span of [H_W H_B] (no Krylov iteration).
//
// Theorem 3.1 applied to each of the three factors of M = exp(-c^2 S_W / 2) exp(c^2 S_B) exp(-c^2 S_W / 2)
// (Eq. (3.15)) gives M = I + Z C Z^T with Z = [H_W H_B] and the symmetric (n + k) x (n + k) matrix
//     C = [ 2 K + K G_W K + (K G_WB) K_B (K G_WB)^T    (K G_WB) K_B ]      K = K_W(-c^2 / 2),
//         [ ((K G_WB) K_B)^T                            K_B          ]      K_B = K_B(c^2),
// so every eigenvector of M with an eigenvalue other than 1 lies in range(Z) (Theorem 3.7: the rest of
// the spectrum is 1). The problem restricted to range(Z) is solved in the coordinates of Z alone, from the
// Gram G = Z^T Z, with no further pass over the d-long data until the final vectors:
//
//   basis    Z has exactly k + 1 known dependencies: the columns of class j in H_W sum to zero
//            (chi_i - mu_j over the class), and sum_j sqrt(n_j) H_B[:, j] = sum_j n_j (mu_j - mu) = 0.
//            Dropping the last column of every class from H_W and the last column of H_B leaves
//            Z' = Z S with n - 1 columns and range(Z') = range(Z) (full column rank for affinely
//            independent samples, Section 3.2's rank count). G' = S^T G S = R^T R (Cholesky);
//            Q = Z' R^{-1} is an orthonormal basis of range(Z) and P = Z^T Q = G S R^{-1}.
//   matrix   Q^T M Q = I + P^T C P: its t largest eigenpairs (1 + mu_i, w_i) are the t largest of M
//            (the eigenvalues above 1, Theorem 3.7), y_i = Z a_i with a = S R^{-1} w.
//   recovery x_i = exp(-c^2 S_W / 2) y_i (Eq. (3.14)) = Z (a + [K (H_W^T Z a); 0]) with H_W^T Z = G[:n, :].
//   orth     V = orth(X_t) (Algorithm 3 step 6): the t x t Gram of the coordinates b = a + [...] is
//            b^T G b, so X_t R_v^{-1} = Z (b R_v^{-1}); one sweep over Z forms V, and one CholQR pass
//            on V itself removes the rounding the coordinates leave in its orthogonality.
// C P is formed by the same chain of n x n and n x k products as the composed M-apply (u1 = K p, ...),
// on all n - 1 columns at once.
#include "eda_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace eda {

namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// Out[i, j] = A[rows ? rows[i] : i, cols[j]] for i < m, j < c (Out ld m; A ld lda).
__global__ void k_gather(int m, int c, const double* __restrict__ A, int64_t lda, const int* __restrict__ rows,
                         const int* __restrict__ cols, double* __restrict__ Out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * c) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const int r = rows ? rows[i] : i;
    Out[e] = A[(int64_t)cols[j] * lda + r];
}

// Out (nk x t, zero outside the kept rows): Out[keep[i], j] = A[i, j] for i < r (A ld r).
__global__ void k_scatter_rows(int nk, int r, int t, const double* __restrict__ A, const int* __restrict__ keep,
                               double* __restrict__ Out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)r * t) return;
    const int i = (int)(e % r), j = (int)(e / r);
    Out[(int64_t)j * nk + keep[i]] = A[e];
}

// Columns in reverse order: Out[:, j] = A[:, t - 1 - j] (ld rows each).
__global__ void k_reverse_cols(int64_t rows, int t, const double* __restrict__ A, double* __restrict__ Out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * t) return;
    const int64_t r = e % rows;
    const int j = (int)(e / rows);
    Out[(int64_t)j * rows + r] = A[(int64_t)(t - 1 - j) * rows + r];
}

// Rank check of the Cholesky factor R (upper, ld r) of the kept columns' Gram: a pivot R_jj^2 at or below
// 1e-13 of the largest (or not finite) means the kept columns are dependent (samples not affinely independent).
__global__ void k_rank_check(int r, const double* __restrict__ R, int* status) {
    __shared__ double smax;
    double mx = 0.0;
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double v = R[(int64_t)j * r + j];
        mx = fmax(mx, v * v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) smax = 0.0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned long long*>(&smax), __double_as_longlong(mx));
    __syncthreads();
    const double thr = 1e-13 * smax;
    bool bad = false;
    for (int j = threadIdx.x; j < r; j += blockDim.x) {
        const double v = R[(int64_t)j * r + j];
        bad |= !(v * v > thr) || !isfinite(v);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ST_RANKLOSS);
}

// lambda[j] = 1 + mu[t - 1 - j] (descending; mu ascending)
__global__ void k_lambda_desc(int t, const double* __restrict__ mu, double* __restrict__ lam) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < t) lam[j] = 1.0 + mu[t - 1 - j];
}

struct DirectWs {
    double *G, *Gs, *Ri, *P, *PQ, *U, *B, *mu, *Wv, *As, *a, *T1, *T2, *Ga, *Gv, *Rv, *Rvi, *bco, *brev, *X;
    double *CW, *part;
    size_t pcap;
    int* keep;
    SymEigWork eig;
};

// D (n x p, ld ldd) = M X (+ D when acc) for the symmetric n x n K_W or G_W (X ld ldx): on the tensor cores
// from the handle's split when it has one, else as the FP64 product M^T X.
int sym_nn(eda_ctx* h, const OzOperand* oz, const double* M, int n, int p, const double* X, int ldx, bool acc,
           double* D, int ldd, DirectWs& w, cudaStream_t s) {
    if (oz) {
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(*oz, h->oznb, std::min(32, p - c0), X + (size_t)c0 * ldx, ldx, 1.0, acc ? 1.0 : 0.0,
                            acc ? D + (size_t)c0 * ldd : nullptr, ldd, D + (size_t)c0 * ldd, ldd, h->status, s));
        return EDA_OK;
    }
    return gemm_tn_f64(n, n, p, 1.0, M, n, X, ldx, acc ? 1.0 : 0.0, D, ldd, w.part, w.pcap, s);
}

// U = C PQ for p columns (both (n + k) x p, ld nk); PQ is overwritten (the chain of the composed M-apply).
int apply_c(eda_ctx* h, int p, double* PQ, double* U, DirectWs& w, cudaStream_t s) {
    const int n = (int)h->n, k = h->k, nk = n + k;
    const OzOperand* okw = h->ozsmall ? &h->ozKW : nullptr;
    const OzOperand* ogw = h->ozsmall ? &h->ozGW : nullptr;
    double* Pw = PQ;
    double* Qb = PQ + n;
    double* Uw = U;
    double* Ub = U + n;
    EDA_TRY(sym_nn(h, okw, h->KW, n, p, Pw, nk, false, Uw, nk, w, s));                            // u1 = K p
    EDA_TRY(gemm_tn_f64(n, k, p, 1.0, h->GWB, n, Uw, nk, 1.0, Qb, nk, w.part, w.pcap, s));       // q + G_BW u1
    EDA_TRY(sym_nn(h, ogw, h->GW, n, p, Uw, nk, true, Pw, nk, w, s));                             // p + G_W u1
    EDA_TRY(gemm_tn_f64(k, k, p, 1.0, h->KB, k, Qb, nk, 0.0, Ub, nk, w.part, w.pcap, s));        // v = K_B q'
    EDA_TRY(gemm_tn_f64(k, n, p, 1.0, h->GBW, k, Ub, nk, 1.0, Pw, nk, w.part, w.pcap, s));       // p' + G_WB v
    return sym_nn(h, okw, h->KW, n, p, Pw, nk, true, Uw, nk, w, s);                               // u1 + K p''
}

// OUT (d x p) = Z U for U ((n + k) x p, ld nk): one sweep over Z (tensor-core FP64 when the handle has Z split).
int z_times(eda_ctx* h, int p, const double* U, double* OUT, cudaStream_t s) {
    const int nk = (int)h->n + h->k;
    if (h->cfg.prec == EDA_F64_TC && h->ozblock) {
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(h->ozN, h->oznb, std::min(32, p - c0), U + (size_t)c0 * nk, nk, 1.0, 0.0, nullptr, 0,
                            OUT + (size_t)c0 * h->d, h->d, h->status, s));
        return EDA_OK;
    }
    return gemm_nn_f64(h->d, nk, p, 1.0, h->HW, h->d, U, nk, 0.0, nullptr, 0, OUT, h->d, s);
}

}  // namespace

int direct_impl(eda_ctx* h, int t, double* Vout, double* lambda, eda_solve_info* info, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k, r = n - 1;
    if (!h->counts || !h->offsets) return EDA_ERR_INVALID_ARG;   // the class structure is needed
    if (r < 1 || t > r || t > d) return EDA_ERR_INVALID_ARG;

    // kept columns of Z: all but the last column of each class in H_W and the last column of H_B
    std::vector<int32_t> offs(k + 1);
    EDA_CUDA_TRY(cudaMemcpyAsync(offs.data(), h->offsets, (k + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> keep;
    keep.reserve(r);
    for (int j = 0; j < k; ++j)
        for (int p = offs[j]; p < offs[j + 1] - 1; ++p) keep.push_back(p);
    for (int j = 0; j + 1 < k; ++j) keep.push_back(n + j);
    if ((int)keep.size() != r) return EDA_ERR_BAD_LABELS;

    // ---- workspace ----
    DirectWs w{};
    w.pcap = std::max<size_t>({size_t(1) << 20, 2 * (size_t)nk * nk, (size_t)64 * t * t});
    size_t need = 0;
    auto add = [&](size_t cnt) { need += a256(cnt * 8); };
    add((size_t)nk * nk);                       // G
    add((size_t)r * r * 3);                     // Gs, Ri, B
    add((size_t)nk * r * 3);                    // P, PQ, U
    add((size_t)r + (size_t)r * t * 2);         // mu, Wv, As
    add((size_t)nk * t * 6);                    // a, T1, T2, Ga, bco, brev
    add((size_t)t * t * 3);                     // Gv, Rv, Rvi
    add((size_t)d * t);                         // X
    add(chol_inv_blocked_doubles(std::max(r, t)));
    add(w.pcap);
    add(r + 64);                                // keep (ints)
    need += symeig_work_bytes(r, t) + 16384;
    EDA_TRY(ensure_workspace(h, need));
    Arena a{static_cast<char*>(h->ws), h->ws_bytes, 0};
    w.G = a.take<double>((size_t)nk * nk);
    w.Gs = a.take<double>((size_t)r * r);
    w.Ri = a.take<double>((size_t)r * r);
    w.B = a.take<double>((size_t)r * r);
    w.P = a.take<double>((size_t)nk * r);
    w.PQ = a.take<double>((size_t)nk * r);
    w.U = a.take<double>((size_t)nk * r);
    w.mu = a.take<double>(r);
    w.Wv = a.take<double>((size_t)r * t);
    w.As = a.take<double>((size_t)r * t);
    w.a = a.take<double>((size_t)nk * t);
    w.T1 = a.take<double>((size_t)nk * t);
    w.T2 = a.take<double>((size_t)nk * t);
    w.Ga = a.take<double>((size_t)nk * t);
    w.bco = a.take<double>((size_t)nk * t);
    w.brev = a.take<double>((size_t)nk * t);
    w.Gv = a.take<double>((size_t)t * t);
    w.Rv = a.take<double>((size_t)t * t);
    w.Rvi = a.take<double>((size_t)t * t);
    w.X = a.take<double>((size_t)d * t);
    w.CW = a.take<double>(chol_inv_blocked_doubles(std::max(r, t)));
    w.part = a.take<double>(w.pcap);
    w.keep = a.take<int>(r + 64);
    EDA_TRY(symeig_work_carve(a, r, t, h->bar, &w.eig));
    if (!w.keep) return EDA_ERR_OOM;

    cudaEvent_t ev0, ev1;
    EDA_CUDA_TRY(cudaEventCreate(&ev0));
    EDA_CUDA_TRY(cudaEventCreate(&ev1));
    int rc = EDA_OK;
    do {
        if (cudaEventRecord(ev0, s) != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
        ProfScope prof("direct", s);
        if (cudaMemsetAsync(h->status, 0, sizeof(int), s) != cudaSuccess ||
            cudaMemcpyAsync(w.keep, keep.data(), r * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = EDA_ERR_CUDA;
            break;
        }
        if (!h->GWB) {
            if ((rc = ensure_cross_gram(h, w.part, w.pcap, s)) != EDA_OK) break;
        }
        // G = Z^T Z from the handle's blocks
        if ((rc = copy_mat_f64(n, n, h->GW, n, w.G, nk, s)) != EDA_OK) break;
        if ((rc = copy_mat_f64(k, n, h->GBW, k, w.G + n, nk, s)) != EDA_OK) break;
        if ((rc = copy_mat_f64(n, k, h->GWB, n, w.G + (size_t)n * nk, nk, s)) != EDA_OK) break;
        if ((rc = copy_mat_f64(k, k, h->GB, k, w.G + (size_t)n * nk + n, nk, s)) != EDA_OK) break;
        // G' = S^T G S = R^T R, F = G S
        k_gather<<<ceil_div((int64_t)r * r, 256), 256, 0, s>>>(r, r, w.G, nk, w.keep, w.keep, w.Gs);
        launch_counter()++;
        k_gather<<<ceil_div((int64_t)nk * r, 256), 256, 0, s>>>(nk, r, w.G, nk, nullptr, w.keep, w.PQ);
        launch_counter()++;
        if ((rc = chol_inv_blocked(r, w.Gs, r, w.Ri, r, 1e-13, h->status, w.CW, w.part, w.pcap, s)) != EDA_OK) break;
        k_rank_check<<<1, 256, 0, s>>>(r, w.Gs, h->status);
        launch_counter()++;
        // P = F R^{-1} = Z^T Q
        if ((rc = gemm_nn_f64(nk, r, r, 1.0, w.PQ, nk, w.Ri, r, 0.0, nullptr, 0, w.P, nk, s)) != EDA_OK) break;
        // B = P^T C P
        if ((rc = copy_mat_f64(nk, r, w.P, nk, w.PQ, nk, s)) != EDA_OK) break;
        if ((rc = apply_c(h, r, w.PQ, w.U, w, s)) != EDA_OK) break;
        if ((rc = gemm_tn_f64(nk, r, r, 1.0, w.P, nk, w.U, nk, 0.0, w.B, r, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = symmetrize_f64(r, w.B, r, s)) != EDA_OK) break;
        // the t largest eigenpairs of P^T C P (ascending)
        if ((rc = symeig_f64(r, w.B, r, r - t, r - 1, w.mu, w.Wv, r, &w.eig, h->status, h->cfg.seed + 29, 1e-7, s)) !=
            EDA_OK)
            break;
        // y = Z a, a = S R^{-1} w
        if ((rc = gemm_nn_f64(r, r, t, 1.0, w.Ri, r, w.Wv, r, 0.0, nullptr, 0, w.As, r, s)) != EDA_OK) break;
        if (cudaMemsetAsync(w.a, 0, (size_t)nk * t * 8, s) != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
        k_scatter_rows<<<ceil_div((int64_t)r * t, 256), 256, 0, s>>>(nk, r, t, w.As, w.keep, w.a);
        launch_counter()++;
        // x = exp(-c^2 S_W / 2) y: coordinates a + [K (G_W a_W + G_WB a_B); 0]
        if ((rc = sym_nn(h, nullptr, h->GW, n, t, w.a, nk, false, w.T1, n, w, s)) != EDA_OK) break;
        if ((rc = gemm_tn_f64(k, n, t, 1.0, h->GBW, k, w.a + n, nk, 1.0, w.T1, n, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = sym_nn(h, nullptr, h->KW, n, t, w.T1, n, true, w.a, nk, w, s)) != EDA_OK) break;
        // orth: Gram of the coordinates b^T G b = R_v^T R_v, coefficients b R_v^{-1}
        if ((rc = gemm_tn_f64(nk, nk, t, 1.0, w.G, nk, w.a, nk, 0.0, w.Ga, nk, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = gemm_tn_f64(nk, t, t, 1.0, w.a, nk, w.Ga, nk, 0.0, w.Gv, t, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = symmetrize_f64(t, w.Gv, t, s)) != EDA_OK) break;
        if ((rc = chol_inv_auto(t, w.Gv, t, w.Rvi, 1e-28, h->status, w.CW, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = gemm_nn_f64(nk, t, t, 1.0, w.a, nk, w.Rvi, t, 0.0, nullptr, 0, w.bco, nk, s)) != EDA_OK) break;
        // descending order, then V = Z b R_v^{-1}
        k_reverse_cols<<<ceil_div((int64_t)nk * t, 256), 256, 0, s>>>(nk, t, w.bco, w.brev);
        launch_counter()++;
        if ((rc = z_times(h, t, w.brev, w.X, s)) != EDA_OK) break;
        // one CholQR pass on V itself
        if ((rc = syrk_f64(d, t, 1.0, w.X, d, 0.0, w.Rv, t, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = chol_inv_auto(t, w.Rv, t, w.Rvi, 1e-28, h->status, w.CW, w.part, w.pcap, s)) != EDA_OK) break;
        if ((rc = gemm_nn_f64(d, t, t, 1.0, w.X, d, w.Rvi, t, 0.0, nullptr, 0, Vout, d, s)) != EDA_OK) break;
        k_lambda_desc<<<ceil_div(t, 128), 128, 0, s>>>(t, w.mu, lambda);
        launch_counter()++;
        if (cudaPeekAtLastError() != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
    } while (false);
    float ms = 0.f;
    if (rc == EDA_OK) {
        if (cudaEventRecord(ev1, s) != cudaSuccess || cudaEventSynchronize(ev1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess)
            rc = EDA_ERR_CUDA;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (rc != EDA_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    int st = 0;
    EDA_CUDA_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (st & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (st & ST_RANKLOSS) return EDA_ERR_BREAKDOWN;   // dependent samples: Z' is rank deficient
    if (info) {
        info->converged = t;
        info->iters = 0;
        info->mapplies = 0;
        info->basis_cols = r;
        info->refills = 0;
        info->checks = 0;
        info->refine_iters = 0;
        info->c2 = h->c2;
        info->lmax_w = h->lmax_w;
        info->lmax_b = h->lmax_b;
        info->max_relres_est = 0.0;
        info->max_relres_true = -1.0;
        info->ms_solve = ms;
        if (info->relres)
            for (int i = 0; i < t; ++i) info->relres[i] = 0.0;
    }
    return EDA_OK;
}

}  // namespace eda
