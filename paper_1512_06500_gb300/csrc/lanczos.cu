// Block Lanczos for the t dominant eigenpairs of M (Algorithm 3, step 5, Lanczos form) with
// full CGS2 reorthogonalisation, CholQR2 block normalisation, Rayleigh-Ritz on the block
// tridiagonal T and the residual test of Remark 3.4; then recovery x = exp(-c^2 S_W / 2) y
// (Eq. eqn311) and orthonormalisation (Algorithm 3, step 6).
//
// M - I has rank at most n - 1 (Theorem 3.1: it maps into span[H_W, H_B]), so the block Krylov
// space is exhausted after about (n - 1) / b + 1 blocks. With the basis sized to n + k + b
// columns no restart is needed: the loop ends by convergence or by exact termination (the new
// block has no component outside the basis).
#include "eda_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

namespace eda {

namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void k_set_block(double* T, int ldt, int r0, int c0, int b, const double* Bm, int ldb, bool transpose) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e % b, j = e / b;
    const double v = transpose ? Bm[(int64_t)i * ldb + j] : Bm[(int64_t)j * ldb + i];
    T[(int64_t)(c0 + j) * ldt + (r0 + i)] = v;
}

// diagonal block: symmetrised
__global__ void k_set_diag_block(double* T, int ldt, int r0, int b, const double* A, int lda) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e % b, j = e / b;
    const double v = 0.5 * (A[(int64_t)j * lda + i] + A[(int64_t)i * lda + j]);
    T[(int64_t)(r0 + j) * ldt + (r0 + i)] = v;
}

// relres[i] = ||B S[rlast:rlast+b, i]|| / |theta_i| for the t Ritz pairs (theta ascending).
__global__ void k_ritz_residuals(int t, int b, const double* Bm, int ldb, const double* S, int lds, int rlast,
                                 const double* theta, double* relres) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t) return;
    double acc = 0.0;
    for (int r = 0; r < b; ++r) {
        double v = 0.0;
        for (int c = 0; c < b; ++c) v = fma(Bm[(int64_t)c * ldb + r], S[(int64_t)i * lds + rlast + c], v);
        acc = fma(v, v, acc);
    }
    const double th = fabs(theta[i]);
    relres[i] = th > 0.0 ? sqrt(acc) / th : INFINITY;
}

// out[:, i] = in[:, t-1-i]  (descending order of the Ritz values)
__global__ void k_reverse_cols(int64_t rows, int t, const double* in, int64_t ldi, double* out, int64_t ldo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * t) return;
    const int64_t r = e % rows;
    const int c = (int)(e / rows);
    out[(int64_t)c * ldo + r] = in[(int64_t)(t - 1 - c) * ldi + r];
}

__global__ void k_reverse_vec(int t, const double* in, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t) out[i] = in[t - 1 - i];
}

// R = M Y - Y diag(theta) in place of MY, column by column
__global__ void k_sub_scaled(int64_t d, int t, double* MY, int64_t ldm, const double* Y, int64_t ldy,
                             const double* theta) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d * t) return;
    const int64_t r = e % d;
    const int c = (int)(e / d);
    MY[(int64_t)c * ldm + r] = fma(-theta[c], Y[(int64_t)c * ldy + r], MY[(int64_t)c * ldm + r]);
}

struct SolveWs {
    double *V, *W, *W1, *tmp, *T, *C, *Gb, *R1, *R1i, *R2, *R2i, *Bm, *P, *Q, *part;
    double *theta, *S, *relres, *Ydesc, *Xt, *Gt, *Rt, *Rti, *lamd;
    int* lost;
    size_t pcap;
    SymEigWork eig;
};

// CholQR of X (d x b) in place: X <- X R^{-1}; R returned in Rm (b x b). Rank loss marks lost pivots.
int cholqr_pass(int64_t d, int b, double* X, int64_t ldx, double* Rm, double* Rinv, double* out, double piv_min2,
                int* status, int* lost, SolveWs& w, cudaStream_t s) {
    EDA_TRY(gemm_tn_f64(d, b, b, 1.0, X, ldx, X, ldx, 0.0, Rm, b, w.part, w.pcap, s));
    EDA_TRY(chol_inv_small(b, Rm, b, Rinv, 1e-28, piv_min2, status, lost, s));
    EDA_TRY(gemm_nn_f64(d, b, b, 1.0, X, ldx, Rinv, b, 0.0, nullptr, 0, out, ldx, s));
    return EDA_OK;
}

// CGS2: X <- X - V (V^T X), twice; the first coefficients are left in Cfirst (cols x b).
int cgs2(int64_t d, int cols, int b, const double* V, double* X, int64_t ldx, double* Cfirst, double* C2,
         SolveWs& w, cudaStream_t s) {
    if (cols <= 0) return EDA_OK;
    ProfScope prof("reorth", s);
    EDA_TRY(gemm_tn_f64(d, cols, b, 1.0, V, d, X, ldx, 0.0, Cfirst, cols, w.part, w.pcap, s));
    EDA_TRY(gemm_nn_f64(d, cols, b, -1.0, V, d, Cfirst, cols, 1.0, X, ldx, X, ldx, s));
    EDA_TRY(gemm_tn_f64(d, cols, b, 1.0, V, d, X, ldx, 0.0, C2, cols, w.part, w.pcap, s));
    EDA_TRY(gemm_nn_f64(d, cols, b, -1.0, V, d, C2, cols, 1.0, X, ldx, X, ldx, s));
    return EDA_OK;
}

}  // namespace

// Y = M X = E_W^{-1/2} E_B E_W^{-1/2} X, the three products (iii)-(v) of Eq. (320).
int m_apply(eda_ctx* h, int b, const double* X, int64_t ldx, double* Y, int64_t ldy, double* tmp, double* P,
            double* Q, double* partial, size_t partial_cap, cudaStream_t s) {
    ProfScope prof("m_apply", s);
    const int64_t d = h->d;
    const ExpOp W{h->HW, h->KW, (int)h->n, "exp_apply_w"};
    const ExpOp B{h->HB, h->KB, h->k, "exp_apply_b"};
    EDA_TRY(exp_apply_f64(d, W, b, X, ldx, tmp, d, P, Q, partial, partial_cap, s));
    EDA_TRY(exp_apply_f64(d, B, b, tmp, d, Y, ldy, P, Q, partial, partial_cap, s));
    EDA_TRY(exp_apply_f64(d, W, b, Y, ldy, tmp, d, P, Q, partial, partial_cap, s));
    EDA_TRY(copy_mat_f64(d, b, tmp, d, Y, ldy, s));
    return EDA_OK;
}

int solve_impl(eda_ctx* h, int t, double tol, const double* V0, int b0, double* Vout, double* lambda, double* Yout,
               eda_solve_info* info, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k;
    const int b = h->cfg.block_b;
    if (t > d || t > n + k) return EDA_ERR_INVALID_ARG;
    int m_max = h->cfg.m_max > 0 ? h->cfg.m_max : n + k + b;
    m_max = (m_max + b - 1) / b * b;
    m_max = (int)std::min<int64_t>(m_max, d / b * b);
    if (m_max < t + b || m_max < 2 * b || m_max > (1 << 16)) return EDA_ERR_INVALID_ARG;
    const int N = std::max(n, k);
    const int tw = std::max(t, b);   // width of the final blocks

    cudaEvent_t ev0, ev1;
    EDA_CUDA_TRY(cudaEventCreate(&ev0));
    EDA_CUDA_TRY(cudaEventCreate(&ev1));
    EDA_CUDA_TRY(cudaEventRecord(ev0, s));

    // ---- workspace ----
    SolveWs w{};
    w.pcap = std::max<size_t>({size_t(1) << 19, (size_t)m_max * tw, (size_t)N * tw, (size_t)t * t});
    size_t need = 0;
    auto add = [&](size_t cnt) { need += a256(cnt * 8); };
    add((size_t)d * m_max);            // V
    add((size_t)d * tw);               // W
    add((size_t)d * tw);               // W1
    add((size_t)d * tw);               // tmp
    add((size_t)m_max * m_max);        // T
    add((size_t)m_max * tw * 2);       // C (two)
    for (int i = 0; i < 6; ++i) add((size_t)b * b);
    add((size_t)N * tw * 2);           // P, Q
    add(w.pcap);
    add(t);                            // theta
    add((size_t)m_max * t);            // S
    add(t);                            // relres
    add((size_t)d * t);                // Ydesc
    add((size_t)d * t);                // Xt
    add((size_t)t * t * 3);            // Gt, Rt, Rti
    add(t);                            // lamd
    add(b + 64);                       // lost (ints)
    need += symeig_work_bytes(m_max, t) + 8192;
    EDA_TRY(ensure_workspace(h, need));
    Arena a{static_cast<char*>(h->ws), h->ws_bytes, 0};
    w.V = a.take<double>((size_t)d * m_max);
    w.W = a.take<double>((size_t)d * tw);
    w.W1 = a.take<double>((size_t)d * tw);
    w.tmp = a.take<double>((size_t)d * tw);
    w.T = a.take<double>((size_t)m_max * m_max);
    w.C = a.take<double>((size_t)m_max * tw * 2);
    w.Gb = a.take<double>((size_t)b * b);
    w.R1 = a.take<double>((size_t)b * b);
    w.R1i = a.take<double>((size_t)b * b);
    w.R2 = a.take<double>((size_t)b * b);
    w.R2i = a.take<double>((size_t)b * b);
    w.Bm = a.take<double>((size_t)b * b);
    w.P = a.take<double>((size_t)N * tw);
    w.Q = a.take<double>((size_t)N * tw);
    w.part = a.take<double>(w.pcap);
    w.theta = a.take<double>(t);
    w.S = a.take<double>((size_t)m_max * t);
    w.relres = a.take<double>(t);
    w.Ydesc = a.take<double>((size_t)d * t);
    w.Xt = a.take<double>((size_t)d * t);
    w.Gt = a.take<double>((size_t)t * t);
    w.Rt = a.take<double>((size_t)t * t);
    w.Rti = a.take<double>((size_t)t * t);
    w.lamd = a.take<double>(t);
    w.lost = a.take<int>(b + 64);
    EDA_TRY(symeig_work_carve(a, m_max, t, h->bar, &w.eig));
    if (!w.lost) return EDA_ERR_OOM;
    EDA_CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    EDA_CUDA_TRY(cudaMemsetAsync(w.T, 0, (size_t)m_max * m_max * 8, s));

    // rank threshold on squared pivots: relative to the bound lambda_1(M) <= exp(c^2 lmax(G_B))
    // of Theorem 3.3 (nu_d = 0)
    const double normM = std::exp(std::min(700.0, h->c2 * h->lmax_b));
    const double piv_min2 = (1e-12 * normM) * (1e-12 * normM);
    int refills = 0;

    // ---- start block ----
    if (V0) {
        const int cp = std::min(b0, b);
        EDA_TRY(copy_mat_f64(d, cp, V0, d, w.V, d, s));
        if (cp < b) EDA_TRY(fill_gaussian_f64(d, b - cp, w.V + (size_t)cp * d, d, h->cfg.seed, 0, s));
    } else {
        EDA_TRY(fill_gaussian_f64(d, b, w.V, d, h->cfg.seed, 0, s));
    }
    EDA_TRY(cholqr_pass(d, b, w.V, d, w.R1, w.R1i, w.W1, 0.0, h->status, w.lost, w, s));
    EDA_TRY(cholqr_pass(d, b, w.W1, d, w.R2, w.R2i, w.V, 0.0, h->status, w.lost, w, s));
    {
        int lostc = 0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&lostc, w.lost + b, sizeof(int), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        if (lostc) return EDA_ERR_BREAKDOWN;   // the start block itself is rank deficient
    }

    int cols = b;            // basis columns filled
    int iters = 0, checks = 0, mapplies = 0;
    bool converged = false, exhausted = false;
    std::vector<double> relres_h(t), theta_h(t);
    double max_rel = INFINITY;
    int conv_count = 0;
    // Rayleigh-Ritz schedule: the first check once the basis has t + b columns; later checks at
    // the basis width where the geometric rate seen between the last two checks predicts
    // convergence (never sooner than check_every blocks, always at the last block).
    int next_check = t + b;
    int prev_check_cols = 0;
    double prev_check_rel = 0.0;
    int rr_cols = 0;         // size of T used by the last Rayleigh-Ritz

    while (true) {
        const int j0 = cols - b;     // first column of the current block V_j
        const double* Vj = w.V + (size_t)j0 * d;
        // W = M V_j
        EDA_TRY(m_apply(h, b, Vj, d, w.W, d, w.tmp, w.P, w.Q, w.part, w.pcap, s));
        ++mapplies;
        ++iters;
        // CGS2 against the whole basis; A_j = rows j0..j0+b of the first coefficient block
        double* C1 = w.C;
        double* C2 = w.C + (size_t)m_max * tw;
        EDA_TRY(cgs2(d, cols, b, w.V, w.W, d, C1, C2, w, s));
        k_set_diag_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.T, m_max, j0, b, C1 + j0, cols);
        EDA_LAUNCHED();
        // CholQR2 of W with rank detection: W = V_{j+1} B_{j+1}
        EDA_CUDA_TRY(cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s));
        EDA_TRY(cholqr_pass(d, b, w.W, d, w.R1, w.R1i, w.W1, piv_min2, h->status, w.lost, w, s));
        int lostc = 0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&lostc, w.lost + b, sizeof(int), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        const bool room = cols + b <= m_max;
        if (lostc == b) {
            exhausted = true;    // no direction outside the basis: T is exact (B_{j+1} = 0)
        } else if (room) {
            if (lostc > 0) {
                // replace the lost columns by fresh random directions orthogonal to the basis
                refills += lostc;
                std::vector<int> lost_h(b + 1);
                EDA_CUDA_TRY(cudaMemcpyAsync(lost_h.data(), w.lost, (b + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
                EDA_CUDA_TRY(cudaStreamSynchronize(s));
                for (int q = 0; q < lostc; ++q)
                    EDA_TRY(fill_gaussian_f64(d, 1, w.W1 + (size_t)lost_h[q] * d, d, h->cfg.seed,
                                              1000 + (uint64_t)iters * 64 + q, s));
                EDA_TRY(cgs2(d, cols, b, w.V, w.W1, d, C2, C2 + (size_t)cols * b, w, s));
            }
            double* Vn = w.V + (size_t)cols * d;
            EDA_CUDA_TRY(cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s));
            EDA_TRY(cholqr_pass(d, b, w.W1, d, w.R2, w.R2i, Vn, 0.0, h->status, w.lost, w, s));
            // B_{j+1} = R2 R1
            EDA_TRY(gemm_small_f64(false, false, b, b, b, 1.0, w.R2, b, w.R1, b, 0.0, w.Bm, b, s));
        } else {
            // basis full: keep B_{j+1} = R1 for the residual estimate only
            EDA_TRY(copy_mat_f64(b, b, w.R1, b, w.Bm, b, s));
        }
        // Rayleigh-Ritz on the leading cols x cols block when due
        const bool last = exhausted || !room;
        if ((cols >= next_check && cols >= t + 1) || (last && cols >= t)) {
            ++checks;
            rr_cols = cols;
            ProfScope prof("rr", s);
            EDA_TRY(symeig_f64(cols, w.T, m_max, cols - t, cols - 1, w.theta, w.S, cols, &w.eig, h->status,
                               h->cfg.seed + 7, 1e-7, s));
            if (exhausted) {
                EDA_CUDA_TRY(cudaMemsetAsync(w.relres, 0, t * sizeof(double), s));
            } else {
                k_ritz_residuals<<<ceil_div(t, 128), 128, 0, s>>>(t, b, w.Bm, b, w.S, cols, cols - b, w.theta,
                                                                 w.relres);
                EDA_LAUNCHED();
            }
            EDA_CUDA_TRY(cudaMemcpyAsync(relres_h.data(), w.relres, t * sizeof(double), cudaMemcpyDeviceToHost, s));
            EDA_CUDA_TRY(cudaStreamSynchronize(s));
            max_rel = 0.0;
            conv_count = 0;
            for (int i = 0; i < t; ++i) {
                if (relres_h[i] <= tol) ++conv_count;
                max_rel = std::max(max_rel, relres_h[i]);
            }
            if (conv_count == t) converged = true;
            // schedule the next check
            int gap = b * h->cfg.check_every;
            if (prev_check_cols > 0 && max_rel > 0.0 && prev_check_rel > 0.0 && max_rel < prev_check_rel &&
                std::isfinite(max_rel)) {
                const double blocks = (double)(cols - prev_check_cols) / b;
                const double rate = std::pow(max_rel / prev_check_rel, 1.0 / blocks);   // per block
                const double need = std::log(tol / max_rel) / std::log(rate);           // blocks to go
                if (std::isfinite(need) && need > 1.0) gap = std::max(gap, b * (int)std::floor(0.8 * need));
            }
            prev_check_cols = cols;
            prev_check_rel = max_rel;
            next_check = cols + gap;
        }
        if (converged || last) break;
        // T gets the off-diagonal block B_{j+1} (rows cols.., columns j0..)
        k_set_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.T, m_max, cols, j0, b, w.Bm, b, false);
        EDA_LAUNCHED();
        k_set_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.T, m_max, j0, cols, b, w.Bm, b, true);
        EDA_LAUNCHED();
        cols += b;
    }
    int st = 0;
    EDA_CUDA_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (st & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (rr_cols == 0) return EDA_ERR_NOT_CONVERGED;

    // ---- Ritz vectors (descending), recovery and orthonormalisation ----
    // Y = V_{:rr} S, columns reversed so that theta is descending
    EDA_TRY(gemm_nn_f64(d, rr_cols, t, 1.0, w.V, d, w.S, rr_cols, 0.0, nullptr, 0, w.Xt, d, s));
    k_reverse_cols<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, w.Xt, d, w.Ydesc, d);
    EDA_LAUNCHED();
    k_reverse_vec<<<ceil_div(t, 128), 128, 0, s>>>(t, w.theta, w.lamd);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemcpyAsync(lambda, w.lamd, t * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (Yout) EDA_CUDA_TRY(cudaMemcpyAsync(Yout, w.Ydesc, (size_t)d * t * 8, cudaMemcpyDeviceToDevice, s));
    // x = exp(-c^2 S_W / 2) y
    const ExpOp Wop{h->HW, h->KW, n, "exp_apply_w"};
    EDA_TRY(exp_apply_f64(d, Wop, t, w.Ydesc, d, w.Xt, d, w.P, w.Q, w.part, w.pcap, s));
    // V = orth(X_t): CholQR2
    {
        EDA_TRY(gemm_tn_f64(d, t, t, 1.0, w.Xt, d, w.Xt, d, 0.0, w.Rt, t, w.part, w.pcap, s));
        EDA_TRY(chol_inv_small(t, w.Rt, t, w.Rti, 1e-28, 0.0, h->status, nullptr, s));
        EDA_TRY(gemm_nn_f64(d, t, t, 1.0, w.Xt, d, w.Rti, t, 0.0, nullptr, 0, Vout, d, s));
        EDA_TRY(gemm_tn_f64(d, t, t, 1.0, Vout, d, Vout, d, 0.0, w.Rt, t, w.part, w.pcap, s));
        EDA_TRY(chol_inv_small(t, w.Rt, t, w.Rti, 1e-28, 0.0, h->status, nullptr, s));
        EDA_TRY(gemm_nn_f64(d, t, t, 1.0, Vout, d, w.Rti, t, 0.0, nullptr, 0, w.Xt, d, s));
        EDA_TRY(copy_mat_f64(d, t, w.Xt, d, Vout, d, s));
    }
    double true_max = -1.0;
    if (h->cfg.true_residuals) {
        // R = M Y - Y diag(theta), in blocks of at most tw columns
        double* MY = w.Xt;
        for (int c0 = 0; c0 < t; c0 += tw) {
            const int cb = std::min(tw, t - c0);
            EDA_TRY(m_apply(h, cb, w.Ydesc + (size_t)c0 * d, d, MY + (size_t)c0 * d, d, w.tmp, w.P, w.Q, w.part,
                            w.pcap, s));
        }
        k_sub_scaled<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, MY, d, w.Ydesc, d, w.lamd);
        EDA_LAUNCHED();
        EDA_TRY(col_norms_f64(d, t, MY, d, w.relres, s));
        std::vector<double> rn(t), lam_h(t);
        EDA_CUDA_TRY(cudaMemcpyAsync(rn.data(), w.relres, t * 8, cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaMemcpyAsync(lam_h.data(), w.lamd, t * 8, cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        true_max = 0.0;
        for (int i = 0; i < t; ++i) true_max = std::max(true_max, rn[i] / std::fabs(lam_h[i]));
    }
    EDA_CUDA_TRY(cudaEventRecord(ev1, s));
    EDA_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    EDA_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    EDA_CUDA_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (st & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (info) {
        info->converged = conv_count;
        info->iters = iters;
        info->mapplies = mapplies;
        info->basis_cols = rr_cols;
        info->refills = refills;
        info->checks = checks;
        info->c2 = h->c2;
        info->lmax_w = h->lmax_w;
        info->lmax_b = h->lmax_b;
        info->max_relres_est = max_rel;
        info->max_relres_true = true_max;
        info->ms_solve = ms;
        if (info->relres) {
            // relres_h is ascending in theta; report in descending order
            for (int i = 0; i < t; ++i) info->relres[i] = relres_h[t - 1 - i];
        }
    }
    return converged ? EDA_OK : EDA_ERR_NOT_CONVERGED;
}

}  // namespace eda
