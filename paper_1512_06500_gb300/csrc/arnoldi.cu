// Arnoldi-EDA: the t dominant eigenpairs of the nonsymmetric form of the pencil (Eq. (3.1))
//     N x = exp(-c^2 S_W) exp(c^2 S_B) x = lambda x
// by block Arnoldi (Section 3.1; Algorithm 3 step 5 in its Arnoldi form). Each step applies N once: two
// Theorem 3.1 products (Algorithm 2 steps 6A-10A), here in composed form
//     N Y = Y + Z [v; u],  [p; q] = Z^T Y,  u = K_B q,  v = K_W(-c^2) (p + G_WB u),   Z = [H_W H_B],
// i.e. two sweeps over Z. The Ritz vectors are generalized eigenvectors of the pencil directly: there is
// no recovery step x = exp(-c^2 S_W / 2) y as in the symmetric form.
//
// Basis: V orthonormal (full CGS2 reorthogonalisation, CholQR2 block normalisation with rank detection
// and refills, as in the Lanczos solver); H = V^T N V is kept in full (upper block Hessenberg). Ritz
// extraction on span(V): eigenpairs of the Galerkin condition with the test space exp(c^2 S_W) V,
//     (V^T exp(c^2 S_B) V) s = theta (V^T exp(c^2 S_W) V) s,
// a symmetric-definite pencil (so theta is real, as the eigenvalues of Eq. (3.1) are), formed from the
// coordinates Z^T V that every N-apply produces anyway: V^T exp(c^2 S_B) V = I + (H_B^T V)^T K_B (H_B^T V) and
// V^T exp(c^2 S_W) V = I + (H_W^T V)^T K_W(c^2) (H_W^T V). (With y = exp(c^2 S_W / 2) x this is the Rayleigh-Ritz
// step of the symmetric form on span(exp(c^2 S_W / 2) V).) The residual r = N x - theta x of a Ritz pair
// (theta, x = V s) follows from the Arnoldi relation N V = V H + W E^T (W the reorthogonalised remainder of the
// last block): r = V (H s - theta s) + W s_last. It is measured in the exp(c^2 S_W) norm, the norm in which it
// equals the symmetric form's residual M y - theta y (so tol means the same for eda_solve and this solver):
// ||r||^2 = ||H s - theta s||^2 + ||W s_last||^2 + (H_W^T r)^T K_W(c^2) (H_W^T r), with H_W^T r from the
// coordinates Z^T V and one sweep Z^T W at each check, and ||y|| = 1 (s = R^{-1} y, y a unit eigenvector of
// the projected symmetric matrix).
#include "eda_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

namespace eda {

namespace {

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

// H[i, j0 + jj] = C1[i, jj] + C2[i, jj] for i < cols (the full coefficients V^T N V_j of the new block)
__global__ void k_arn_set_hcol(double* H, int ldh, int cols, int j0, int b, const double* C1, const double* C2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cols * b) return;
    const int i = e % cols, jj = e / cols;
    H[(int64_t)(j0 + jj) * ldh + i] = C1[(int64_t)jj * cols + i] + C2[(int64_t)jj * cols + i];
}

// H[r0 + i, c0 + jj] = B[i, jj] (the sub-diagonal block: W = V_{j+1} B)
__global__ void k_arn_set_block(double* H, int ldh, int r0, int c0, int b, const double* Bm) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e % b, jj = e / b;
    H[(int64_t)(c0 + jj) * ldh + r0 + i] = Bm[(int64_t)jj * b + i];
}

__global__ void k_arn_add_identity(int m, double* A, int lda) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) A[(int64_t)i * lda + i] += 1.0;
}

// R[:, c] -= theta[c] S[:, c]
__global__ void k_arn_sub_scaled(int rows, int t, double* R, int ldr, const double* S, int lds, const double* theta) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * t) return;
    const int r = (int)(e % rows), c = (int)(e / rows);
    R[(int64_t)c * ldr + r] = fma(-theta[c], S[(int64_t)c * lds + r], R[(int64_t)c * ldr + r]);
}

// relres[i] = sqrt(a[i]^2 + b[i]^2 + q[i]) / |theta[i]|
__global__ void k_arn_relres(int t, const double* a, const double* b, const double* q, const double* theta,
                             double* relres) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= t) return;
    const double den = fabs(theta[i]);
    relres[i] = den > 0.0 ? sqrt(fmax(0.0, fma(a[i], a[i], fma(b[i], b[i], q[i])))) / den : INFINITY;
}

// q[c] = sum_r X[r, c] Y[r, c] (one warp per column)
__global__ void k_arn_coldot(int rows, int t, const double* X, int ldx, const double* Y, int ldy, double* q) {
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    double acc = 0.0;
    for (int r = lane; r < rows; r += 32) acc = fma(X[(int64_t)c * ldx + r], Y[(int64_t)c * ldy + r], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) q[c] = acc;
}

__global__ void k_arn_reverse_cols(int64_t rows, int t, const double* in, int64_t ldi, double* out, int64_t ldo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * t) return;
    const int64_t r = e % rows;
    const int c = (int)(e / rows);
    out[(int64_t)c * ldo + r] = in[(int64_t)(t - 1 - c) * ldi + r];
}

__global__ void k_arn_reverse_vec(int t, const double* in, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t) out[i] = in[t - 1 - i];
}

struct ArnWs {
    double *V, *W, *W1, *X, *X2, *Wz, *H, *C, *R1, *R1i, *R2, *R2i, *Bm, *PQ, *U;
    double *AW, *AB, *Cm, *Ri, *T1, *S, *HS, *theta, *relres, *n1, *n2, *sn, *lamd;
    double *ZW, *T2, *T3;   // Z^T W of the last block; n x t temporaries of the residual
    double* CW;             // blocked Cholesky work
    double* part;
    size_t pcap;
    int* lost;
    SymEigWork eig;
};

// X <- orth(X) in place by CholQR (one pass); X2: d x p scratch; R, Ri: p x p.
int cholqr_once(int64_t d, int p, double* X, double* X2, double* R, double* Ri, double piv_min2, int* status, int* lost,
                ArnWs& w, cudaStream_t s) {
    EDA_TRY(syrk_f64(d, p, 1.0, X, d, 0.0, R, p, w.part, w.pcap, s));
    if (lost || piv_min2 > 0.0) EDA_TRY(chol_inv_small(p, R, p, Ri, 1e-28, piv_min2, status, lost, s));
    else EDA_TRY(chol_inv_auto(p, R, p, Ri, 1e-28, status, w.CW, w.part, w.pcap, s));
    EDA_TRY(gemm_nn_f64(d, p, p, 1.0, X, d, Ri, p, 0.0, nullptr, 0, X2, d, s));
    return EDA_OK;
}

// CGS2 of the d x b block X against the first cols columns of V; coefficients of the passes in C1, C2 (cols x b).
int cgs2_f64(int64_t d, int cols, int b, const double* V, double* X, double* C1, double* C2, ArnWs& w, cudaStream_t s) {
    ProfScope prof("reorth", s);
    for (int pass = 0; pass < 2; ++pass) {
        double* C = pass == 0 ? C1 : C2;
        EDA_TRY(gemm_tn_f64(d, cols, b, 1.0, V, d, X, d, 0.0, C, cols, w.part, w.pcap, s));
        EDA_TRY(gemm_nn_f64(d, cols, b, -1.0, V, d, C, cols, 1.0, X, d, X, d, s));
    }
    return EDA_OK;
}

// Z^T W for the reorthogonalised remainder W of the block just applied, by one sweep over Z. (Forming it
// from Z^T N V_j - (Z^T V) H[:, j] cancels: both terms are of size ||N|| ~ e^tau while W is small, and the
// cancellation leaves an error far above the residuals the solver must resolve.)
int arn_ztw(eda_ctx* h, ArnWs& w, int b, cudaStream_t s) {
    return sweep_zt(h, b, w.W, h->d, w.ZW, w.part, w.pcap, s);
}

// Rayleigh-Ritz on span(V[:, :m]) with the E_W-Galerkin condition: theta (t, ascending), S (m x t), and the
// relative residuals (device relres, host copy).
int arn_ritz(eda_ctx* h, int m, int ldh, int t, int b, ArnWs& w, std::vector<double>& relres_h, cudaStream_t s) {
    ProfScope prof("rr", s);
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k;
    const double* QW = w.Wz;        // H_W^T V: rows 0 .. n of the coordinates (ld nk)
    const double* QB = w.Wz + n;    // H_B^T V: rows n .. nk
    // A_W = I + Q_W^T K_W(c^2) Q_W,  A_B = I + Q_B^T K_B Q_B
    EDA_TRY(gemm_small_f64(false, false, n, m, n, 1.0, h->KWp, n, QW, nk, 0.0, w.T1, n, s));
    EDA_TRY(gemm_tn_f64(n, m, m, 1.0, QW, nk, w.T1, n, 0.0, w.AW, m, w.part, w.pcap, s));
    EDA_TRY(gemm_small_f64(false, false, k, m, k, 1.0, h->KB, k, QB, nk, 0.0, w.T1, k, s));
    EDA_TRY(gemm_tn_f64(k, m, m, 1.0, QB, nk, w.T1, k, 0.0, w.AB, m, w.part, w.pcap, s));
    k_arn_add_identity<<<ceil_div(m, 128), 128, 0, s>>>(m, w.AW, m);
    EDA_LAUNCHED();
    k_arn_add_identity<<<ceil_div(m, 128), 128, 0, s>>>(m, w.AB, m);
    EDA_LAUNCHED();
    EDA_TRY(symmetrize_f64(m, w.AW, m, s));
    EDA_TRY(symmetrize_f64(m, w.AB, m, s));
    // A_W = R^T R; the symmetric C = R^{-T} A_B R^{-1} has the pencil's eigenvalues; s = R^{-1} y
    EDA_TRY(chol_inv_auto(m, w.AW, m, w.Ri, 1e-28, h->status, w.CW, w.part, w.pcap, s));
    EDA_TRY(gemm_small_f64(false, false, m, m, m, 1.0, w.AB, m, w.Ri, m, 0.0, w.T1, m, s));
    EDA_TRY(gemm_small_f64(true, false, m, m, m, 1.0, w.Ri, m, w.T1, m, 0.0, w.Cm, m, s));
    EDA_TRY(symmetrize_f64(m, w.Cm, m, s));
    EDA_TRY(symeig_f64(m, w.Cm, m, m - t, m - 1, w.theta, w.T1, m, &w.eig, h->status, h->cfg.seed + 17, 1e-7, s));
    EDA_TRY(gemm_small_f64(false, false, m, t, m, 1.0, w.Ri, m, w.T1, m, 0.0, w.S, m, s));
    // residuals in the exp(c^2 S_W) norm: ||H s - theta s||^2 + ||W s_last||^2 + (H_W^T r)^T K_W(c^2) (H_W^T r)
    EDA_TRY(gemm_small_f64(false, false, m, t, m, 1.0, w.H, ldh, w.S, m, 0.0, w.HS, m, s));
    k_arn_sub_scaled<<<ceil_div((int64_t)m * t, 256), 256, 0, s>>>(m, t, w.HS, m, w.S, m, w.theta);
    EDA_LAUNCHED();
    EDA_TRY(col_norms_f64(m, t, w.HS, m, w.n1, s));
    EDA_TRY(gemm_nn_f64(d, b, t, 1.0, w.W, d, w.S + (m - b), m, 0.0, nullptr, 0, w.X, d, s));
    EDA_TRY(col_norms_f64(d, t, w.X, d, w.n2, s));
    // H_W^T r = Q_W (H s - theta s) + (H_W^T W) s_last
    EDA_TRY(gemm_small_f64(false, false, n, t, m, 1.0, QW, nk, w.HS, m, 0.0, w.T2, n, s));
    EDA_TRY(gemm_small_f64(false, false, n, t, b, 1.0, w.ZW, nk, w.S + (m - b), m, 1.0, w.T2, n, s));
    EDA_TRY(gemm_small_f64(false, false, n, t, n, 1.0, h->KWp, n, w.T2, n, 0.0, w.T3, n, s));
    k_arn_coldot<<<t, 32, 0, s>>>(n, t, w.T2, n, w.T3, n, w.sn);
    EDA_LAUNCHED();
    k_arn_relres<<<ceil_div(t, 128), 128, 0, s>>>(t, w.n1, w.n2, w.sn, w.theta, w.relres);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemcpyAsync(relres_h.data(), w.relres, t * sizeof(double), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    return EDA_OK;
}

// True residuals of the Ritz pairs (theta, x = V[:, :m] S) in the exp(c^2 S_W) norm, in which every x has
// unit norm: ||r||^2 = ||r||_2^2 + (H_W^T r)^T K_W(c^2) (H_W^T r), r = N x - theta x, with N x by the composed
// N-apply (two sweeps over Z per block of columns) and H_W^T r by one more sweep. The residuals the Arnoldi
// relation gives miss what a dropped (refilled) direction left behind: about 64 eps ||N|| per refill, which
// at tau = 20 lies above tol = 1e-6 however good the subspace is; these do not. X holds the Ritz vectors on
// return, X2 the residual block.
int arn_true_residuals(eda_ctx* h, int m, int t, int b, ArnWs& w, std::vector<double>& relres_h, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, nk = n + h->k;
    EDA_TRY(gemm_nn_f64(d, m, t, 1.0, w.V, d, w.S, m, 0.0, nullptr, 0, w.X, d, s));
    for (int c0 = 0; c0 < t; c0 += b) {
        const int cb = std::min(b, t - c0);
        EDA_TRY(n_apply_composed(h, cb, w.X + (size_t)c0 * d, d, w.X2 + (size_t)c0 * d, d, w.PQ, w.U, nullptr, w.part,
                                 w.pcap, s));
    }
    k_arn_sub_scaled<<<ceil_div(d * t, 256), 256, 0, s>>>((int)d, t, w.X2, (int)d, w.X, (int)d, w.theta);
    EDA_LAUNCHED();
    EDA_TRY(col_norms_f64(d, t, w.X2, d, w.n1, s));
    EDA_TRY(sweep_zt(h, t, w.X2, d, w.T1, w.part, w.pcap, s));   // Z^T r: its first n rows are H_W^T r
    EDA_TRY(gemm_tn_f64(n, n, t, 1.0, h->KWp, n, w.T1, nk, 0.0, w.T2, n, w.part, w.pcap, s));
    k_arn_coldot<<<t, 32, 0, s>>>(n, t, w.T1, nk, w.T2, n, w.sn);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemsetAsync(w.n2, 0, t * sizeof(double), s));
    k_arn_relres<<<ceil_div(t, 128), 128, 0, s>>>(t, w.n1, w.n2, w.sn, w.theta, w.relres);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemcpyAsync(relres_h.data(), w.relres, t * sizeof(double), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    return EDA_OK;
}

}  // namespace

int ensure_n_operators(eda_ctx* h, cudaStream_t s) {
    if (h->KWm) return EDA_OK;
    const int n = (int)h->n, k = h->k;
    // cross Grams (their split-K partials in the solve workspace)
    if (!h->GWB) {
        const size_t pcap = std::max<size_t>(1u << 19, (size_t)n * k);
        EDA_TRY(ensure_workspace(h, pcap * 8 + 4096));
        EDA_TRY(ensure_cross_gram(h, static_cast<double*>(h->ws), pcap, s));
    }
    const size_t nn = a256((size_t)n * n * 8);
    void* p = nullptr;
    EDA_CUDA_TRY(cudaMalloc(&p, 2 * nn + a256(6 * (size_t)n * n * 8)));
    h->nblock = p;
    h->KWm = static_cast<double*>(p);
    h->KWp = reinterpret_cast<double*>(static_cast<char*>(p) + nn);
    double* work = reinterpret_cast<double*>(static_cast<char*>(p) + 2 * nn);
    const double c2 = h->c2;
    if (h->eig_ready) {
        // from the Gram's significant eigenpairs (the build's eigenpair route)
        const int ns = h->nsig_w;
        const double* lam = h->evals_w + (n - ns);
        EDA_TRY(phi_operator(n, ns, lam, h->evecs_w, n, -c2, h->KWm, work, s));
        EDA_TRY(phi_operator(n, ns, lam, h->evecs_w, n, c2, h->KWp, work, s));
    } else {
        // by scaling and squaring of G_W (the build's route for small Grams)
        const size_t b1 = (oz_operand_bytes(n, n) + 255) / 256 * 256;
        const OzSquare oz{h->ozsmall, static_cast<char*>(h->ozsmall) + b1, h->status};
        const OzSquare* pz = h->ozsmall ? &oz : nullptr;
        EDA_TRY(phi_by_squaring(n, h->GW, -c2, h->lmax_w_bound, h->KWm, work, s, pz));
        EDA_TRY(phi_by_squaring(n, h->GW, c2, h->lmax_w_bound, h->KWp, work, s, pz));
    }
    return EDA_OK;
}

int n_apply_composed(eda_ctx* h, int p, const double* Y, int64_t ldy, double* NY, int64_t ldn, double* PQ, double* U,
                     double* ZtY, double* part, size_t pcap, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k;
    ProfScope prof("n_apply", s, 4.0 * d * nk * p + 2.0 * p * ((double)n * n + 2.0 * n * k + (double)k * k),
                   8.0 * (2.0 * d * nk + 3.0 * d * p));
    EDA_TRY(sweep_zt(h, p, Y, ldy, PQ, part, pcap, s));
    if (ZtY) EDA_TRY(copy_mat_f64(nk, p, PQ, nk, ZtY, nk, s));
    double* Pw = PQ;
    double* Qb = PQ + n;
    double* Uw = U;
    double* Ub = U + n;
    EDA_TRY(gemm_small_f64(false, false, k, p, k, 1.0, h->KB, k, Qb, nk, 0.0, Ub, nk, s));     // u = K_B q
    EDA_TRY(gemm_small_f64(false, false, n, p, k, 1.0, h->GWB, n, Ub, nk, 1.0, Pw, nk, s));    // p + G_WB u
    EDA_TRY(gemm_small_f64(false, false, n, p, n, 1.0, h->KWm, n, Pw, nk, 0.0, Uw, nk, s));    // v
    return sweep_z(h, p, U, Y, ldy, NY, ldn, s);
}

int arnoldi_impl(eda_ctx* h, int t, double tol, double* Vout, double* lambda, eda_solve_info* info, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k;
    const int b = h->cfg.block_b;
    if (t > d || t > nk) return EDA_ERR_INVALID_ARG;
    int m_max = h->cfg.m_max > 0 ? h->cfg.m_max : nk + b;
    m_max = (m_max + b - 1) / b * b;
    m_max = (int)std::min<int64_t>(m_max, d / b * b);
    if (m_max < t + b || m_max < 2 * b || m_max > (1 << 16)) return EDA_ERR_INVALID_ARG;
    EDA_TRY(ensure_n_operators(h, s));

    cudaEvent_t ev0, ev1;
    EDA_CUDA_TRY(cudaEventCreate(&ev0));
    EDA_CUDA_TRY(cudaEventCreate(&ev1));
    EDA_CUDA_TRY(cudaEventRecord(ev0, s));

    ArnWs w{};
    const int tw = std::max(t, b);
    w.pcap = std::max<size_t>({size_t(1) << 19, (size_t)m_max * tw, (size_t)nk * tw, (size_t)m_max * m_max});
    size_t need = 0;
    auto add = [&](size_t cnt) { need += a256(cnt * 8); };
    add((size_t)d * m_max);            // V
    add((size_t)d * b * 2);            // W, W1
    add((size_t)d * tw * 2);           // X, X2
    add((size_t)nk * m_max);           // Wz
    add((size_t)m_max * m_max);        // H
    add((size_t)m_max * b * 4);        // C: the two passes' coefficients, and those of a refill
    for (int i = 0; i < 5; ++i) add((size_t)b * b);
    add((size_t)nk * b * 2);           // PQ, U
    for (int i = 0; i < 4; ++i) add((size_t)m_max * m_max);   // AW, AB, Cm, Ri
    add((size_t)std::max<size_t>((size_t)m_max * m_max, (size_t)n * m_max));   // T1
    add((size_t)m_max * t * 2);        // S, HS
    add((size_t)nk * b + 2 * (size_t)n * t);   // ZW, T2, T3
    add(chol_inv_blocked_doubles(m_max));        // CW
    for (int i = 0; i < 6; ++i) add(t);
    add(w.pcap);
    add(b + 64);                       // lost (ints)
    need += symeig_work_bytes(m_max, t) + 16384;
    EDA_TRY(ensure_workspace(h, need));
    Arena a{static_cast<char*>(h->ws), h->ws_bytes, 0};
    w.V = a.take<double>((size_t)d * m_max);
    w.W = a.take<double>((size_t)d * b);
    w.W1 = a.take<double>((size_t)d * b);
    w.X = a.take<double>((size_t)d * tw);
    w.X2 = a.take<double>((size_t)d * tw);
    w.Wz = a.take<double>((size_t)nk * m_max);
    w.H = a.take<double>((size_t)m_max * m_max);
    w.C = a.take<double>((size_t)m_max * b * 4);
    w.R1 = a.take<double>((size_t)b * b);
    w.R1i = a.take<double>((size_t)b * b);
    w.R2 = a.take<double>((size_t)b * b);
    w.R2i = a.take<double>((size_t)b * b);
    w.Bm = a.take<double>((size_t)b * b);
    w.PQ = a.take<double>((size_t)nk * b);
    w.U = a.take<double>((size_t)nk * b);
    w.AW = a.take<double>((size_t)m_max * m_max);
    w.AB = a.take<double>((size_t)m_max * m_max);
    w.Cm = a.take<double>((size_t)m_max * m_max);
    w.Ri = a.take<double>((size_t)m_max * m_max);
    w.T1 = a.take<double>(std::max<size_t>((size_t)m_max * m_max, (size_t)n * m_max));
    w.S = a.take<double>((size_t)m_max * t);
    w.HS = a.take<double>((size_t)m_max * t);
    w.ZW = a.take<double>((size_t)nk * b);
    w.T2 = a.take<double>((size_t)n * t);
    w.T3 = a.take<double>((size_t)n * t);
    w.CW = a.take<double>(chol_inv_blocked_doubles(m_max));
    w.theta = a.take<double>(t);
    w.relres = a.take<double>(t);
    w.n1 = a.take<double>(t);
    w.n2 = a.take<double>(t);
    w.sn = a.take<double>(t);
    w.lamd = a.take<double>(t);
    w.part = a.take<double>(w.pcap);
    w.lost = a.take<int>(b + 64);
    EDA_TRY(symeig_work_carve(a, m_max, t, h->bar, &w.eig));
    if (!w.lost) return EDA_ERR_OOM;
    EDA_CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    EDA_CUDA_TRY(cudaMemsetAsync(w.H, 0, (size_t)m_max * m_max * 8, s));

    int rc = EDA_OK;
    int iters = 0, mapplies = 0, checks = 0, refills = 0, rr_cols = 0, conv = 0, verifies = 0;
    bool true_res = false;   // relres_h holds true residuals (the last check verified its pairs)
    const size_t t1_cap = std::max<size_t>((size_t)m_max * m_max, (size_t)n * m_max);
    double max_rel = INFINITY;
    std::vector<double> relres_h(t, INFINITY);
    do {
        // rank threshold of a new direction: 64 eps ||N|| with ||N|| <= exp(c^2 lmax(G_B)) (||exp(-c^2 S_W)|| <= 1)
        const double normN = std::exp(std::min(700.0, h->c2 * h->lmax_b));
        const double piv_min2 = (64.0 * DBL_EPSILON * normN) * (64.0 * DBL_EPSILON * normN);
        if ((rc = fill_gaussian_f64(d, b, w.V, d, h->cfg.seed, 0, s)) != EDA_OK) break;
        if ((rc = cholqr_once(d, b, w.V, w.W1, w.R1, w.R1i, 0.0, h->status, w.lost, w, s)) != EDA_OK) break;
        if ((rc = cholqr_once(d, b, w.W1, w.V, w.R2, w.R2i, 0.0, h->status, w.lost, w, s)) != EDA_OK) break;
        int cols = b;
        int next_check = t + 2 * b, prev_cols = 0;
        double prev_rel = 0.0;
        while (true) {
            const int j0 = cols - b;
            const double* Vj = w.V + (size_t)j0 * d;
            if ((rc = n_apply_composed(h, b, Vj, d, w.W, d, w.PQ, w.U, w.Wz + (size_t)j0 * nk, w.part, w.pcap, s)) !=
                EDA_OK)
                break;
            ++mapplies;
            ++iters;
            double* C1 = w.C;
            double* C2 = w.C + (size_t)m_max * b;
            if ((rc = cgs2_f64(d, cols, b, w.V, w.W, C1, C2, w, s)) != EDA_OK) break;
            k_arn_set_hcol<<<ceil_div(cols * b, 256), 256, 0, s>>>(w.H, m_max, cols, j0, b, C1, C2);
            launch_counter()++;
            if (cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s) != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
            // W1 = W R1^{-1} (the remainder W itself stays for the residuals)
            if ((rc = cholqr_once(d, b, w.W, w.W1, w.R1, w.R1i, piv_min2, h->status, w.lost, w, s)) != EDA_OK) break;
            int lostc = 0;
            if (cudaMemcpyAsync(&lostc, w.lost + b, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                rc = EDA_ERR_CUDA;
                break;
            }
            const bool room = cols + b <= m_max;
            if (room) {
                if (lostc > 0) {
                    refills += lostc;
                    std::vector<int> lost_h(b + 1);
                    cudaMemcpyAsync(lost_h.data(), w.lost, (b + 1) * sizeof(int), cudaMemcpyDeviceToHost, s);
                    cudaStreamSynchronize(s);
                    for (int q = 0; q < lostc && rc == EDA_OK; ++q)
                        rc = fill_gaussian_f64(d, 1, w.W1 + (size_t)lost_h[q] * d, d, h->cfg.seed,
                                               1000 + (uint64_t)iters * 64 + q, s);
                    // refilled directions against the basis (their coefficients are not part of H)
                    double* C3 = w.C + 2 * (size_t)m_max * b;
                    if (rc == EDA_OK) rc = cgs2_f64(d, cols, b, w.V, w.W1, C3, C3 + (size_t)m_max * b, w, s);
                    if (rc != EDA_OK) break;
                }
                double* Vn = w.V + (size_t)cols * d;
                if (cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s) != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
                if ((rc = cholqr_once(d, b, w.W1, Vn, w.R2, w.R2i, 0.0, h->status, w.lost, w, s)) != EDA_OK) break;
                if ((rc = gemm_small_f64(false, false, b, b, b, 1.0, w.R2, b, w.R1, b, 0.0, w.Bm, b, s)) != EDA_OK)
                    break;
                k_arn_set_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.H, m_max, cols, j0, b, w.Bm);
                launch_counter()++;
            }
            const bool last = !room;
            if ((cols >= next_check && cols >= t + 1) || (last && cols >= t)) {
                ++checks;
                rr_cols = cols;
                if ((rc = arn_ztw(h, w, b, s)) != EDA_OK) break;
                if ((rc = arn_ritz(h, cols, m_max, t, b, w, relres_h, s)) != EDA_OK) break;
                max_rel = 0.0;
                conv = 0;
                for (int i = 0; i < t; ++i) {
                    if (relres_h[i] <= tol) ++conv;
                    max_rel = std::max(max_rel, relres_h[i]);
                }
                // after refills the relation's estimates carry what the dropped directions left behind: once they
                // are within a factor 100 of tol, or the basis is full, the pairs are judged by true residuals
                if (conv < t && refills > 0 && (max_rel <= 100.0 * tol || last) && (size_t)nk * t <= t1_cap) {
                    ++verifies;
                    if ((rc = arn_true_residuals(h, cols, t, b, w, relres_h, s)) != EDA_OK) break;
                    max_rel = 0.0;
                    conv = 0;
                    for (int i = 0; i < t; ++i) {
                        if (relres_h[i] <= tol) ++conv;
                        max_rel = std::max(max_rel, relres_h[i]);
                    }
                    true_res = true;
                }
                // no usable rate (no progress since the last check): wait an eighth of the basis width
                int gap = (prev_cols > 0 && !(max_rel < prev_rel)) ? std::max(b * h->cfg.check_every, (cols / 8) / b * b)
                                                                   : b * h->cfg.check_every;
                if (prev_cols > 0 && max_rel > 0.0 && prev_rel > 0.0 && max_rel < prev_rel && std::isfinite(max_rel)) {
                    const double rate = std::pow(max_rel / prev_rel, 1.0 / ((double)(cols - prev_cols) / b));
                    const double need_b = std::log(tol / max_rel) / std::log(rate);
                    if (std::isfinite(need_b) && need_b > 1.0) gap = std::max(gap, b * (int)std::floor(0.8 * need_b));
                }
                gap = std::min(gap, std::max(b * h->cfg.check_every, (cols / 4) / b * b));
                prev_cols = cols;
                prev_rel = max_rel;
                next_check = cols + gap;
            }
            if (conv == t || last) break;
            cols += b;
        }
        if (rc != EDA_OK) break;
        if (rr_cols == 0) {
            rc = EDA_ERR_NOT_CONVERGED;
            break;
        }
        // Ritz vectors X = V S (the generalized eigenvectors, ascending theta), V = orth(X) by CholQR2
        if ((rc = gemm_nn_f64(d, rr_cols, t, 1.0, w.V, d, w.S, rr_cols, 0.0, nullptr, 0, w.X, d, s)) != EDA_OK) break;
        for (int pass = 0; pass < 2 && rc == EDA_OK; ++pass) {
            rc = cholqr_once(d, t, w.X, w.X2, w.AW, w.Ri, 0.0, h->status, nullptr, w, s);
            if (rc == EDA_OK) rc = copy_mat_f64(d, t, w.X2, d, w.X, d, s);
        }
        if (rc != EDA_OK) break;
        k_arn_reverse_cols<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, w.X, d, Vout, d);
        launch_counter()++;
        k_arn_reverse_vec<<<ceil_div(t, 128), 128, 0, s>>>(t, w.theta, w.lamd);
        launch_counter()++;
        if (cudaMemcpyAsync(lambda, w.lamd, t * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            rc = EDA_ERR_CUDA;
    } while (false);
    if (rc != EDA_OK && rc != EDA_ERR_NOT_CONVERGED) {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        return rc;
    }
    EDA_CUDA_TRY(cudaEventRecord(ev1, s));
    EDA_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    EDA_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    int stw = 0;
    EDA_CUDA_TRY(cudaMemcpyAsync(&stw, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (stw & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (stw & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (info) {
        info->converged = conv;
        info->iters = iters;
        info->mapplies = mapplies;
        info->basis_cols = rr_cols;
        info->refills = refills;
        info->checks = checks;
        info->c2 = h->c2;
        info->lmax_w = h->lmax_w;
        info->lmax_b = h->lmax_b;
        info->max_relres_est = max_rel;
        info->max_relres_true = true_res ? max_rel : -1.0;
        info->refine_iters = verifies;
        info->ms_solve = ms;
        if (info->relres)
            for (int i = 0; i < t; ++i) info->relres[i] = relres_h[t - 1 - i];
    }
    return (rc == EDA_OK && conv == t) ? EDA_OK : EDA_ERR_NOT_CONVERGED;
}

}  // namespace eda
