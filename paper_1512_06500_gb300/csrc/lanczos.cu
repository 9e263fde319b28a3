// Block Lanczos for the t dominant eigenpairs of M (Algorithm 3, step 5, Lanczos form) with
// full CGS2 reorthogonalisation, CholQR2 block normalisation, Rayleigh-Ritz on the block
// tridiagonal T and the residual test of Remark 3.4; then recovery x = exp(-c^2 S_W / 2) y
// (Eq. (3.14)) and orthonormalisation (Algorithm 3, step 6).
//
// M - I has rank at most n - 1 (Theorem 3.1: it maps into span[H_W, H_B]), so the block Krylov
// space is exhausted after about (n - 1) / b + 1 blocks. With the basis sized to n + k + b
// columns no restart is needed: the loop ends by convergence or by exact termination (the new
// block has no component outside the basis).
//
// Precision: the Krylov sweeps and the basis use the storage type T. With T = double this is
// the plain FP64 solver. With T = float (single-precision H, basis and sweeps; the small
// matrices stay FP64) the loop stops at a loose tolerance and the Ritz vectors are refined in
// FP64: Rayleigh-Ritz on span(Y) with FP64 M-applies, then subspace iteration Y <- M Y, until
// the true FP64 relative residual of every pair is at most tol.
#include "eda_internal.cuh"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>
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

// Column block j0..j0+b-1 of the projected matrix T = V^T M V from the full reorthogonalisation
// coefficients (C1 + C2 = V^T (M V_j), cols x b, ld cols), mirrored into the row block; the diagonal
// block symmetrised. Keeping every coupling (not only the block-tridiagonal ones) makes the
// Rayleigh-Ritz step exact on span(V) even after lost directions were replaced by fresh ones.
__global__ void k_set_col_block(double* T, int ldt, int cols, int j0, int b, const double* C1, const double* C2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cols * b) return;
    const int i = e % cols, jj = e / cols;
    const double v = C1[(int64_t)jj * cols + i] + C2[(int64_t)jj * cols + i];
    if (i < j0) {
        T[(int64_t)(j0 + jj) * ldt + i] = v;
        T[(int64_t)i * ldt + (j0 + jj)] = v;
    } else {
        const int ii = i - j0;
        const double w = C1[(int64_t)ii * cols + (j0 + jj)] + C2[(int64_t)ii * cols + (j0 + jj)];
        T[(int64_t)(j0 + jj) * ldt + i] = 0.5 * (v + w);
    }
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

// out[:, i] = in[:, t-1-i] (descending order of the Ritz values)
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

// R = MY - Y diag(theta), written over MY
__global__ void k_sub_scaled(int64_t d, int t, double* MY, int64_t ldm, const double* Y, int64_t ldy,
                             const double* theta) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d * t) return;
    const int64_t r = e % d;
    const int c = (int)(e / d);
    MY[(int64_t)c * ldm + r] = fma(-theta[c], Y[(int64_t)c * ldy + r], MY[(int64_t)c * ldm + r]);
}

__global__ void k_divide(int t, double* num, const double* den) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t) num[i] = fabs(den[i]) > 0.0 ? num[i] / fabs(den[i]) : INFINITY;
}

// Workspace of one solve: Krylov state in T, small matrices and the FP64 finish.
template <class T>
struct SolveWs {
    T *V, *W, *W1, *tmp, *Yt;
    double *Tm, *C, *R1, *R1i, *R2, *R2i, *Bm, *P, *Q, *theta, *S, *relres;
    double *Y, *Z, *Y2, *Z2, *Xt, *Gt, *Rt, *Rti, *lamd, *tmp64;
    double *R, *MR, *A2, *PQ, *Uc;   // refinement: [Y R] and [MY MR] adjacent; (2t)^2; (n + k) x t twice
    double* ZY;                      // refinement: Z^T [Y R], (n + k) x 2t
    double* CW;                      // blocked Cholesky work (t > 90)
    int* idx;                        // refinement: unconverged columns
    void* part;
    int* lost;
    size_t pcap;
    SymEigWork eig;
    // prec = EDA_F64_TC: the basis split for V^T X (column scales, appended block by block) and for V C (row
    // scales over the current columns, split afresh whenever a block is added)
    bool oz = false;
    OzOperand VT, VN;
    int oz_cap = 0;                  // columns the basis operands hold (m_max)
    int* olist = nullptr;            // d + 1 ints: rows of VN to split afresh
};

// tc products with the split basis, 32 columns at a time: C (cols x p, ldc) = V^T X, and X -= V C
template <class T>
int oz_basis_tn(eda_ctx* h, SolveWs<T>& w, int cols, int p, const double* X, int64_t ldx, double* C, int ldc,
                cudaStream_t s) {
    OzOperand A = w.VT;
    A.M = cols;
    A.mtiles = ceil_div(cols, 128);
    for (int c0 = 0; c0 < p; c0 += 32)
        EDA_TRY(oz_gemm(A, h->oznb, std::min(32, p - c0), X + (size_t)c0 * ldx, ldx, 1.0, 0.0, nullptr, 0,
                        C + (size_t)c0 * ldc, ldc, h->status, s));
    return EDA_OK;
}
template <class T>
int oz_basis_nn(eda_ctx* h, SolveWs<T>& w, int cols, int p, const double* C, int ldc, double alpha, double beta,
                const double* X0, int64_t ldx0, double* X, int64_t ldx, cudaStream_t s) {
    OzOperand A = w.VN;
    A.K = cols;
    for (int c0 = 0; c0 < p; c0 += 32)
        EDA_TRY(oz_gemm(A, h->oznb, std::min(32, p - c0), C + (size_t)c0 * ldc, ldc, alpha, beta,
                        X0 ? X0 + (size_t)c0 * ldx0 : nullptr, ldx0, X + (size_t)c0 * ldx, ldx, h->status, s));
    return EDA_OK;
}

// The basis has grown from cols0 to cols1 columns: append their column-scaled digit planes and split the
// whole basis afresh with row scales over all its columns.
template <class T>
int oz_basis_grow(SolveWs<T>& w, int64_t d, int cols0, int cols1, int* status, cudaStream_t s) {
    if (!w.oz) return EDA_OK;
    const double* V = reinterpret_cast<const double*>(w.V);
    EDA_TRY(oz_append_cols(V, d, cols0, cols1, d, &w.VT, status, s));
    // row scales over all columns so far: only rows whose scale the new block raises are split afresh
    return oz_grow_rows(V, d, d, cols0, cols1, &w.VN, w.olist, status, s);
}

template <class T>
int cholqr_pass(int64_t d, int b, T* X, int64_t ldx, double* Rm, double* Rinv, T* out, double piv_min2, int* status,
                int* lost, SolveWs<T>& w, cudaStream_t s) {
    EDA_TRY(syrk_tn<T>(d, b, 1.0, X, ldx, 0.0, Rm, b, w.part, w.pcap, s));
    EDA_TRY(chol_inv_small(b, Rm, b, Rinv, 1e-28, piv_min2, status, lost, s));
    // R^{-1} is upper triangular with its zeros stored: the product skips the zero rows of each column slice
    EDA_TRY(gemm_nn<T>(d, b, b, 1.0, X, ldx, Rinv, b, 0.0, nullptr, 0, out, ldx, s, true));
    return EDA_OK;
}

// CGS2: X <- X - V (V^T X), twice; the first coefficients are left in Cfirst (cols x b). With the split
// basis (tensor-core FP64 mode) both products of each pass run on the tensor cores.
template <class T>
int cgs2(int64_t d, int cols, int b, const T* V, T* X, int64_t ldx, double* Cfirst, double* C2, SolveWs<T>& w,
         cudaStream_t s, eda_ctx* h = nullptr) {
    if (cols <= 0) return EDA_OK;
    ProfScope prof("reorth", s);
    if (w.oz && h) {
        double* Xd = reinterpret_cast<double*>(X);
        for (int pass = 0; pass < 2; ++pass) {
            double* C = pass == 0 ? Cfirst : C2;
            EDA_TRY(oz_basis_tn(h, w, cols, b, Xd, ldx, C, cols, s));
            EDA_TRY(oz_basis_nn(h, w, cols, b, C, cols, -1.0, 1.0, Xd, ldx, Xd, ldx, s));
        }
        return EDA_OK;
    }
    EDA_TRY(gemm_tn<T>(d, cols, b, 1.0, V, d, X, ldx, 0.0, Cfirst, cols, w.part, w.pcap, s));
    EDA_TRY(gemm_nn<T>(d, cols, b, -1.0, V, d, Cfirst, cols, 1.0, X, ldx, X, ldx, s));
    EDA_TRY(gemm_tn<T>(d, cols, b, 1.0, V, d, X, ldx, 0.0, C2, cols, w.part, w.pcap, s));
    EDA_TRY(gemm_nn<T>(d, cols, b, -1.0, V, d, C2, cols, 1.0, X, ldx, X, ldx, s));
    return EDA_OK;
}

template <class T> struct HStore;
template <> struct HStore<double> {
    static const double* W(eda_ctx* h) { return h->HW; }
    static const double* B(eda_ctx* h) { return h->HB; }
};
template <> struct HStore<float> {
    static const float* W(eda_ctx* h) { return h->HW32; }
    static const float* B(eda_ctx* h) { return h->HB32; }
};

}  // namespace

int m_apply_composed(eda_ctx* h, int p, const double* Y, int64_t ldy, double* MY, int64_t ldm, double* PQ,
                     double* U, double* ZtY, double* part, size_t pcap, cudaStream_t s);

// Y = M X = E_W^{-1/2} E_B E_W^{-1/2} X, the three products (iii)-(v) of Eq. (3.16); in FP64 with
// m_form = 1 (and allow_composed) their composed form instead. P and Q hold (n + k) x b doubles.
template <class T>
int m_apply_t(eda_ctx* h, int b, const T* X, int64_t ldx, T* Y, int64_t ldy, T* tmp, double* P, double* Q,
              void* partial, size_t partial_cap, cudaStream_t s, bool allow_composed = true) {
    ProfScope prof("m_apply", s);
    if (std::is_same<T, double>::value && allow_composed && (h->cfg.m_form == 1 || h->cfg.prec == EDA_F64_TC) &&
        h->GWB)
        return m_apply_composed(h, b, reinterpret_cast<const double*>(X), ldx, reinterpret_cast<double*>(Y), ldy, P,
                                Q, nullptr, static_cast<double*>(partial), partial_cap, s);
    const int64_t d = h->d;
    const T* HW = HStore<T>::W(h);
    const T* HB = HStore<T>::B(h);
    const int n = (int)h->n;
    if (std::is_same<T, float>::value && h->cfg.prec == EDA_BF16) {
        // bf16 H on the tensor cores (the basis stays single precision); the three products chain
        // through the bf16 staging pair and run in place on Y
        const float* Xf = reinterpret_cast<const float*>(X);
        float* Yf = reinterpret_cast<float*>(Y);
        (void)tmp;
        EDA_TRY(exp_apply_tc(h->tcW, h->tcbuf, "exp_apply_w", b, Xf, ldx, Yf, ldy, TC_EMIT_SPLIT, h->status, s));
        EDA_TRY(exp_apply_tc(h->tcB, h->tcbuf, "exp_apply_b", b, Yf, ldy, Yf, ldy, TC_X_SPLIT_READY | TC_EMIT_SPLIT,
                             h->status, s));
        EDA_TRY(exp_apply_tc(h->tcW, h->tcbuf, "exp_apply_w", b, Yf, ldy, Yf, ldy, TC_X_SPLIT_READY, h->status, s));
        return EDA_OK;
    }
    EDA_TRY(exp_apply<T>(d, HW, h->KW, n, "exp_apply_w", b, X, ldx, tmp, d, P, Q, partial, partial_cap, s));
    EDA_TRY(exp_apply<T>(d, HB, h->KB, h->k, "exp_apply_b", b, tmp, d, Y, ldy, P, Q, partial, partial_cap, s));
    EDA_TRY(exp_apply<T>(d, HW, h->KW, n, "exp_apply_w", b, Y, ldy, tmp, d, P, Q, partial, partial_cap, s));
    EDA_TRY((copy_mat<T, T>(d, b, tmp, d, Y, ldy, s)));
    return EDA_OK;
}

int m_apply(eda_ctx* h, int b, const double* X, int64_t ldx, double* Y, int64_t ldy, double* tmp, double* P,
            double* Q, double* partial, size_t partial_cap, cudaStream_t s) {
    return m_apply_t<double>(h, b, X, ldx, Y, ldy, tmp, P, Q, partial, partial_cap, s);
}

int m_apply_f32(eda_ctx* h, int b, const float* X, int64_t ldx, float* Y, int64_t ldy, float* tmp, double* P,
                double* Q, double* partial, size_t partial_cap, cudaStream_t s) {
    return m_apply_t<float>(h, b, X, ldx, Y, ldy, tmp, P, Q, partial, partial_cap, s);
}

namespace {

struct LanczosStats {
    int iters = 0, mapplies = 0, checks = 0, refills = 0, rr_cols = 0, conv_count = 0;
    bool converged = false;
    double max_rel = INFINITY;
    std::vector<double> relres;   // ascending theta order
};

// Block Lanczos in storage type T. On return w.theta holds the t Ritz values (ascending) and
// w.Yt the Ritz vectors V_{:rr} S (d x t, same order).
template <class T>
int run_lanczos(eda_ctx* h, int t, double tol, const double* V0, int b0, int m_max, SolveWs<T>& w, LanczosStats& st,
                cudaStream_t s) {
    const int64_t d = h->d;
    const int b = h->cfg.block_b;
    const int tw = std::max(t, b);
    // rank threshold on squared pivots: relative to the bound lambda_1(M) <= exp(c^2 lmax(G_B))
    // of Theorem 3.3 (nu_d = 0). A new direction is lost when its norm after full
    // reorthogonalisation is at the rounding level of the product, 64 eps ||M|| in the basis precision:
    // above that level it carries real spectral content even when it is tiny against ||M||.
    const double normM = std::exp(std::min(700.0, h->c2 * h->lmax_b));
    const double eta = 64.0 * (std::is_same<T, double>::value ? 2.220446049250313e-16 : 1.1920928955078125e-7);
    const double piv_min2 = (eta * normM) * (eta * normM);

    // ---- start block ----
    if (V0) {
        const int cp = std::min(b0, b);
        EDA_TRY((copy_mat<double, T>(d, cp, V0, d, w.V, d, s)));
        if (cp < b) EDA_TRY(fill_gaussian<T>(d, b - cp, w.V + (size_t)cp * d, d, h->cfg.seed, 0, s));
    } else {
        EDA_TRY(fill_gaussian<T>(d, b, w.V, d, h->cfg.seed, 0, s));
    }
    EDA_TRY(cholqr_pass<T>(d, b, w.V, d, w.R1, w.R1i, w.W1, 0.0, h->status, w.lost, w, s));
    EDA_TRY(cholqr_pass<T>(d, b, w.W1, d, w.R2, w.R2i, w.V, 0.0, h->status, w.lost, w, s));
    EDA_TRY(oz_basis_grow<T>(w, d, 0, b, h->status, s));
    {
        int lostc = 0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&lostc, w.lost + b, sizeof(int), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        if (lostc) return EDA_ERR_BREAKDOWN;   // the start block itself is rank deficient
    }

    int cols = b;
    st.relres.assign(t, INFINITY);
    // Rayleigh-Ritz schedule: the first check once the basis has t + 2b columns (block Lanczos needs
    // about two blocks beyond the t wanted directions; an earlier check costs a small eigensolve and
    // rarely succeeds); later checks at the basis width where the geometric rate seen between the last
    // two checks predicts convergence (never sooner than check_every blocks, never more than a quarter of
    // the current basis width later, always at the last block).
    int next_check = t + 2 * b;
    int prev_check_cols = 0;
    double prev_check_rel = 0.0;

    while (true) {
        const int j0 = cols - b;
        const T* Vj = w.V + (size_t)j0 * d;
        EDA_TRY(m_apply_t<T>(h, b, Vj, d, w.W, d, w.tmp, w.P, w.Q, w.part, w.pcap, s));
        ++st.mapplies;
        ++st.iters;
        double* C1 = w.C;
        double* C2 = w.C + (size_t)m_max * tw;
        EDA_TRY(cgs2<T>(d, cols, b, w.V, w.W, d, C1, C2, w, s, h));
        k_set_col_block<<<ceil_div(cols * b, 256), 256, 0, s>>>(w.Tm, m_max, cols, j0, b, C1, C2);
        EDA_LAUNCHED();
        // CholQR2 of W with rank detection: W = V_{j+1} B_{j+1}
        EDA_CUDA_TRY(cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s));
        EDA_TRY(cholqr_pass<T>(d, b, w.W, d, w.R1, w.R1i, w.W1, piv_min2, h->status, w.lost, w, s));
        int lostc = 0;
        EDA_CUDA_TRY(cudaMemcpyAsync(&lostc, w.lost + b, sizeof(int), cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        const bool room = cols + b <= m_max;
        if (room) {
            if (lostc > 0) {
                // replace the lost columns by fresh random directions orthogonal to the basis
                st.refills += lostc;
                std::vector<int> lost_h(b + 1);
                EDA_CUDA_TRY(cudaMemcpyAsync(lost_h.data(), w.lost, (b + 1) * sizeof(int), cudaMemcpyDeviceToHost, s));
                EDA_CUDA_TRY(cudaStreamSynchronize(s));
                for (int q = 0; q < lostc; ++q)
                    EDA_TRY(fill_gaussian<T>(d, 1, w.W1 + (size_t)lost_h[q] * d, d, h->cfg.seed,
                                             1000 + (uint64_t)st.iters * 64 + q, s));
                // the refilled directions against the basis (their coefficients are not part of T)
                double* C3 = w.C + (size_t)m_max * tw * 2;
                EDA_TRY(cgs2<T>(d, cols, b, w.V, w.W1, d, C3, C3 + (size_t)m_max * b, w, s, h));
            }
            T* Vn = w.V + (size_t)cols * d;
            EDA_CUDA_TRY(cudaMemsetAsync(w.lost, 0, (b + 1) * sizeof(int), s));
            EDA_TRY(cholqr_pass<T>(d, b, w.W1, d, w.R2, w.R2i, Vn, 0.0, h->status, w.lost, w, s));
            EDA_TRY(oz_basis_grow<T>(w, d, cols, cols + b, h->status, s));
            EDA_TRY(gemm_small_f64(false, false, b, b, b, 1.0, w.R2, b, w.R1, b, 0.0, w.Bm, b, s));   // B = R2 R1
        } else {
            EDA_TRY(copy_mat_f64(b, b, w.R1, b, w.Bm, b, s));   // basis full: residual estimate only
        }
        const bool last = !room;
        // a block lost entirely means span(V) is invariant to working precision: check at once (for a
        // single-precision basis at most every fourth block: on a wide spectrum it may lose every block)
        const bool full_loss = lostc == b && cols >= t &&
                               (std::is_same<T, double>::value || cols - prev_check_cols >= 4 * b);
        if ((cols >= next_check && cols >= t + 1) || (last && cols >= t) || full_loss) {
            ++st.checks;
            st.rr_cols = cols;
            ProfScope prof("rr", s);
            // residual estimates of the t Ritz pairs in S: from the last block row of S, or from W when
            // directions of W below the rank threshold were dropped from B (||W s_last|| / |theta|, W the
            // reorthogonalised remainder of M V_j)
            auto estimate = [&]() -> int {
                if (lostc > 0) {
                    EDA_TRY(gemm_nn<T>(d, b, t, 1.0, w.W, d, w.S + (cols - b), cols, 0.0, nullptr, 0, w.Yt, d, s));
                    EDA_TRY(col_norms<T>(d, t, w.Yt, d, w.relres, s));
                    k_divide<<<ceil_div(t, 128), 128, 0, s>>>(t, w.relres, w.theta);
                    EDA_LAUNCHED();
                } else {
                    k_ritz_residuals<<<ceil_div(t, 128), 128, 0, s>>>(t, b, w.Bm, b, w.S, cols, cols - b, w.theta,
                                                                     w.relres);
                    EDA_LAUNCHED();
                }
                EDA_CUDA_TRY(
                    cudaMemcpyAsync(st.relres.data(), w.relres, t * sizeof(double), cudaMemcpyDeviceToHost, s));
                EDA_CUDA_TRY(cudaStreamSynchronize(s));
                st.max_rel = 0.0;
                st.conv_count = 0;
                for (int i = 0; i < t; ++i) {
                    if (st.relres[i] <= tol) ++st.conv_count;
                    st.max_rel = std::max(st.max_rel, st.relres[i]);
                }
                return EDA_OK;
            };
            // A check that will not stop the iteration only needs the estimates, for which each inverse
            // iteration vector serves alone: the Gram-Schmidt inside clusters of close Ritz values (here
            // the many just above 1, close in units of 1e-7 theta_1) is done only when the estimates say
            // converged, or at the basis limit, and the estimates are then taken again from the
            // orthogonalised vectors, which the Ritz vectors are formed from.
            EDA_TRY(symeig_f64(cols, w.Tm, m_max, cols - t, cols - 1, w.theta, w.S, cols, &w.eig, h->status,
                               h->cfg.seed + 7, last ? 1e-7 : 0.0, s));
            EDA_TRY(estimate());
            if (!last && st.conv_count == t) {
                EDA_TRY(symeig_vectors(cols, t, w.theta, w.S, cols, &w.eig, h->cfg.seed + 7, 1e-7, s));
                EDA_TRY(estimate());
            }
            if (st.conv_count == t) st.converged = true;
            // no usable rate (no progress since the last check): wait a quarter of the basis width (the
            // largest residual of a slow cluster can stall for many blocks and then fall fast: at d = 65536,
            // t = 199 it stays near 2e-3 from 288 to 576 columns and reaches 1e-7 at 704)
            int gap = (prev_check_cols > 0 && !(st.max_rel < prev_check_rel))
                          ? std::max(b * h->cfg.check_every, (cols / 4) / b * b)
                          : b * h->cfg.check_every;
            if (prev_check_cols > 0 && st.max_rel > 0.0 && prev_check_rel > 0.0 && st.max_rel < prev_check_rel &&
                std::isfinite(st.max_rel)) {
                const double blocks = (double)(cols - prev_check_cols) / b;
                const double rate = std::pow(st.max_rel / prev_check_rel, 1.0 / blocks);   // per block
                const double need = std::log(tol / st.max_rel) / std::log(rate);           // blocks to go
                if (std::isfinite(need) && need > 1.0) gap = std::max(gap, b * (int)std::floor(0.8 * need));
            }
            // the rate comes from residual estimates that refilled directions make noisy: never let it push the
            // next check further than a quarter of the basis built so far (an extra check costs one small
            // eigensolve, a missed one whole blocks of M-applies and reorthogonalisation)
            gap = std::min(gap, std::max(b * h->cfg.check_every, (cols / 4) / b * b));
            prev_check_cols = cols;
            prev_check_rel = st.max_rel;
            next_check = cols + gap;
        }
        if (st.converged || last) break;
        k_set_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.Tm, m_max, cols, j0, b, w.Bm, b, false);
        EDA_LAUNCHED();
        k_set_block<<<ceil_div(b * b, 256), 256, 0, s>>>(w.Tm, m_max, j0, cols, b, w.Bm, b, true);
        EDA_LAUNCHED();
        cols += b;
    }
    if (st.rr_cols == 0) return EDA_ERR_NOT_CONVERGED;
    // Ritz vectors Y = V_{:rr} S (ascending theta)
    if (w.oz)
        return oz_basis_nn(h, w, st.rr_cols, t, w.S, st.rr_cols, 1.0, 0.0, nullptr, 0, reinterpret_cast<double*>(w.Yt),
                           d, s);
    EDA_TRY(gemm_nn<T>(d, st.rr_cols, t, 1.0, w.V, d, w.S, st.rr_cols, 0.0, nullptr, 0, w.Yt, d, s));
    return EDA_OK;
}

}  // namespace

// M Y in FP64 for p columns through the composed form of the three products of Eq. (3.16): with
// Theorem 3.1 for each factor and the Grams G_W, G_WB = H_W^T H_B, only two sweeps over
// Z = [H_W H_B] remain:
//     [p; q] = Z^T y
//     u1 = K_W p                 y1 = y + H_W u1,   H_B^T y1 = q + G_BW u1,   H_W^T y1 = p + G_W u1
//     v  = K_B (H_B^T y1)        y2 = y1 + H_B v,   H_W^T y2 = H_W^T y1 + G_WB v
//     u3 = K_W (H_W^T y2)        M y = y2 + H_W u3 = y + Z [u1 + u3; v]
// (the same operator as m_apply_t, in a third of the sweeps).
int m_apply_composed(eda_ctx* h, int p, const double* Y, int64_t ldy, double* MY, int64_t ldm, double* PQ,
                     double* U, double* ZtY, double* part, size_t pcap, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k, nk = n + k;
    // bytes: Z read once per sweep (FP64, or its seven bf16 digit planes on the tensor-core path), Y read
    // twice and MY written
    const double zbytes = (h->cfg.prec == EDA_F64_TC && h->ozblock) ? 14.0 : 8.0;
    ProfScope prof("m_apply_composed", s, 4.0 * d * nk * p + 2.0 * p * (3.0 * n * n + 2.0 * n * k + k * k),
                   2.0 * zbytes * d * nk + 8.0 * 3.0 * d * p);
    EDA_TRY(sweep_zt(h, p, Y, ldy, PQ, part, pcap, s));
    if (ZtY) EDA_TRY(copy_mat_f64(nk, p, PQ, nk, ZtY, nk, s));   // keep Z^T y (coordinates) for the caller
    double* Pw = PQ;
    double* Qb = PQ + n;
    double* Uw = U;
    double* Ub = U + n;
    // the n x n products with K_W and G_W: on the tensor cores from their splits when the handle has them
    auto nn = [&](const OzOperand* oz, const double* M, const double* X, double beta, const double* C0,
                  double* D) -> int {
        if (!oz) return gemm_small_f64(false, false, n, p, n, 1.0, M, n, X, nk, beta, D, nk, s);
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(*oz, h->oznb, std::min(32, p - c0), X + (size_t)c0 * nk, nk, 1.0, beta,
                            C0 ? C0 + (size_t)c0 * nk : nullptr, nk, D + (size_t)c0 * nk, nk, h->status, s));
        return EDA_OK;
    };
    const OzOperand* okw = h->ozsmall ? &h->ozKW : nullptr;
    const OzOperand* ogw = h->ozsmall ? &h->ozGW : nullptr;
    EDA_TRY(nn(okw, h->KW, Pw, 0.0, nullptr, Uw));                                               // u1
    EDA_TRY(gemm_small_f64(false, false, k, p, n, 1.0, h->GBW, k, Uw, nk, 1.0, Qb, nk, s));  // H_B^T y1
    EDA_TRY(nn(ogw, h->GW, Uw, 1.0, Pw, Pw));                                                    // H_W^T y1
    EDA_TRY(gemm_small_f64(false, false, k, p, k, 1.0, h->KB, k, Qb, nk, 0.0, Ub, nk, s));   // v
    EDA_TRY(gemm_small_f64(false, false, n, p, k, 1.0, h->GWB, n, Ub, nk, 1.0, Pw, nk, s));  // H_W^T y2
    EDA_TRY(nn(okw, h->KW, Pw, 1.0, Uw, Uw));                                                    // u1 + u3
    return sweep_z(h, p, U, Y, ldy, MY, ldm, s);
}

// PQ ((n + k) x p) = Z^T Y, Z = [H_W H_B]: the first sweep of a composed product; FP64-accurate tensor-core
// products (error-free splitting, 32 columns at a time) for prec EDA_F64_TC, FP64 otherwise.
int sweep_zt(eda_ctx* h, int p, const double* Y, int64_t ldy, double* PQ, double* part, size_t pcap, cudaStream_t s) {
    const int nk = (int)h->n + h->k;
    if (h->cfg.prec == EDA_F64_TC && h->ozblock) {
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(h->ozT, h->oznb, std::min(32, p - c0), Y + (size_t)c0 * ldy, ldy, 1.0, 0.0, nullptr, 0,
                            PQ + (size_t)c0 * nk, nk, h->status, s));
        return EDA_OK;
    }
    return gemm_tn_f64(h->d, nk, p, 1.0, h->HW, h->d, Y, ldy, 0.0, PQ, nk, part, pcap, s);
}

// OUT (d x p) = Y + Z U, U ((n + k) x p, ld n + k): the second sweep of a composed product.
int sweep_z(eda_ctx* h, int p, const double* U, const double* Y, int64_t ldy, double* OUT, int64_t ldo,
            cudaStream_t s) {
    const int nk = (int)h->n + h->k;
    if (h->cfg.prec == EDA_F64_TC && h->ozblock) {
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(h->ozN, h->oznb, std::min(32, p - c0), U + (size_t)c0 * nk, nk, 1.0, 1.0,
                            Y + (size_t)c0 * ldy, ldy, OUT + (size_t)c0 * ldo, ldo, h->status, s));
        return EDA_OK;
    }
    return gemm_nn_f64(h->d, nk, p, 1.0, h->HW, h->d, U, nk, 1.0, Y, ldy, OUT, ldo, s);
}

namespace {

// Products of the FP64 finish (refinement, final CholQR2) with d-long operands. With the tensor-core
// FP64 mode they run as FP64-accurate digit-plane products, the d-long operand split afresh into the
// solve's basis-operand buffers (free once the Krylov phase has ended); otherwise on the FP64 pipe.
// C (m x p, ldc) = A^T B, A d x m (ld d), B d x p (ldb).
template <class T>
int fin_tn(eda_ctx* h, SolveWs<T>& w, int m, int p, const double* A, const double* B, int64_t ldb, double* C,
           int ldc, cudaStream_t s) {
    const int64_t d = h->d;
    if (w.oz && m <= w.oz_cap) {
        OzOperand op;
        EDA_TRY(oz_operand_make(A, d, m, d, true, w.VT.tiles, &op, h->status, s));
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(op, h->oznb, std::min(32, p - c0), B + (size_t)c0 * ldb, ldb, 1.0, 0.0, nullptr, 0,
                            C + (size_t)c0 * ldc, ldc, h->status, s));
        return EDA_OK;
    }
    return gemm_tn_f64(d, m, p, 1.0, A, d, B, ldb, 0.0, C, ldc, static_cast<double*>(w.part), w.pcap, s);
}
// OUT (d x p, ld d) = alpha A Bs + beta X0, A d x m (ld d), Bs m x p (ldbs), X0 ld d (may be OUT).
template <class T>
int fin_nn(eda_ctx* h, SolveWs<T>& w, int m, int p, double alpha, const double* A, const double* Bs, int ldbs,
           double beta, const double* X0, double* OUT, cudaStream_t s) {
    const int64_t d = h->d;
    if (w.oz && m <= w.oz_cap) {
        OzOperand op;
        EDA_TRY(oz_operand_make(A, d, d, m, false, w.VN.tiles, &op, h->status, s));
        for (int c0 = 0; c0 < p; c0 += 32)
            EDA_TRY(oz_gemm(op, h->oznb, std::min(32, p - c0), Bs + (size_t)c0 * ldbs, ldbs, alpha, beta,
                            X0 ? X0 + (size_t)c0 * d : nullptr, d, OUT + (size_t)c0 * d, d, h->status, s));
        return EDA_OK;
    }
    return gemm_nn_f64(d, m, p, alpha, A, d, Bs, ldbs, beta, X0, d, OUT, d, s);
}

// X (d x p) <- orth(X) by CholQR in FP64, `passes` times (columns at the rank threshold come out
// zero). One pass suffices for an input that is orthonormal to single precision.
template <class T>
int cholqr_f64(eda_ctx* h, int p, double* X, double* tmpX, SolveWs<T>& w, int passes, cudaStream_t s) {
    const int64_t d = h->d;
    double* part = static_cast<double*>(w.part);
    for (int q = 0; q < passes; ++q) {
        if (w.oz && p <= w.oz_cap)
            EDA_TRY(fin_tn(h, w, p, p, X, X, d, w.Rt, p, s));
        else
            EDA_TRY(syrk_f64(d, p, 1.0, X, d, 0.0, w.Rt, p, part, w.pcap, s));
        EDA_TRY(chol_inv_auto(p, w.Rt, p, w.Rti, 1e-28, h->status, w.CW, part, w.pcap, s));
        EDA_TRY(fin_nn(h, w, p, p, 1.0, X, w.Rti, p, 0.0, nullptr, tmpX, s));
        EDA_TRY(copy_mat_f64(d, p, tmpX, d, X, d, s));
    }
    return EDA_OK;
}

__global__ void k_gather_cols(int64_t d, int r, const int* idx, const double* src, int64_t lds, double* dst,
                              int64_t ldd) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d * r) return;
    const int64_t i = e % d;
    const int j = (int)(e / d);
    dst[(int64_t)j * ldd + i] = src[(int64_t)idx[j] * lds + i];
}

// Residuals R = MY - Y diag(theta) and relres_i = ||R_i|| / |theta_i| (host copy, max in *max_rel).
template <class T>
int ritz_residuals(int64_t d, int t, SolveWs<T>& w, std::vector<double>& relres_h, double* max_rel, cudaStream_t s) {
    EDA_TRY(copy_mat_f64(d, t, w.Z, d, w.R, d, s));
    k_sub_scaled<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, w.R, d, w.Y, d, w.theta);
    EDA_LAUNCHED();
    EDA_TRY(col_norms_f64(d, t, w.R, d, w.relres, s));
    k_divide<<<ceil_div(t, 128), 128, 0, s>>>(t, w.relres, w.theta);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemcpyAsync(relres_h.data(), w.relres, t * sizeof(double), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    *max_rel = 0.0;
    for (int i = 0; i < t; ++i) *max_rel = std::max(*max_rel, relres_h[i]);
    return EDA_OK;
}

// FP64 refinement of t approximate eigenvectors Y (d x t, in w.Y) from the single-precision phase:
// Rayleigh-Ritz on span(Y), then, while some relative residual exceeds tol, Rayleigh-Ritz on
// span([Y, R_u]) with R_u the residual columns of the unconverged pairs orthogonalised against Y
// (each round one FP64 M-apply of those columns, in the composed form). Leaves Y (orthonormal Ritz
// vectors, ascending theta) with w.Z = M Y, theta, the residuals, and the coordinates Z^T Y in
// w.ZY (first t columns), from which the recovery step needs one sweep instead of two.
template <class T>
int refine_f64(eda_ctx* h, int t, double tol, SolveWs<T>& w, int max_iter, int* iters_out, int* mapplies,
               std::vector<double>& relres_h, double* max_rel, cudaStream_t s) {
    ProfScope prof("refine", s);
    const int64_t d = h->d;
    const int b = h->cfg.block_b;
    const int nk = (int)h->n + h->k;
    double* part = static_cast<double*>(w.part);
    if (!h->GWB) return EDA_ERR_INVALID_ARG;   // cross Grams are formed at build for mixed handles
    // span(Y): orthonormalise (Y is orthonormal to single precision: one CholQR pass), M Y, Rayleigh-Ritz
    EDA_TRY(cholqr_f64<T>(h, t, w.Y, w.Y2, w, 1, s));
    EDA_TRY(m_apply_composed(h, t, w.Y, d, w.Z, d, w.PQ, w.Uc, w.ZY, part, w.pcap, s));
    *mapplies += (t + b - 1) / b;
    EDA_TRY(fin_tn(h, w, t, t, w.Y, w.Z, d, w.Gt, t, s));
    EDA_TRY(symmetrize_f64(t, w.Gt, t, s));
    EDA_TRY(symeig_f64(t, w.Gt, t, 0, t - 1, w.theta, w.S, t, &w.eig, h->status, h->cfg.seed + 11, 1e-7, s));
    EDA_TRY(fin_nn(h, w, t, t, 1.0, w.Y, w.S, t, 0.0, nullptr, w.Y2, s));
    EDA_TRY(fin_nn(h, w, t, t, 1.0, w.Z, w.S, t, 0.0, nullptr, w.Z2, s));
    EDA_TRY(copy_mat_f64(d, t, w.Y2, d, w.Y, d, s));
    EDA_TRY(copy_mat_f64(d, t, w.Z2, d, w.Z, d, s));
    EDA_TRY(gemm_small_f64(false, false, nk, t, t, 1.0, w.ZY, nk, w.S, t, 0.0, w.PQ, nk, s));
    EDA_TRY(copy_mat_f64(nk, t, w.PQ, nk, w.ZY, nk, s));
    EDA_TRY(ritz_residuals<T>(d, t, w, relres_h, max_rel, s));
    int it = 0;
    std::vector<int> idx;
    while (*max_rel > tol && it < max_iter) {
        ++it;
        idx.clear();
        for (int i = 0; i < t; ++i)
            if (relres_h[i] > 0.5 * tol) idx.push_back(i);
        const int r = (int)idx.size();
        const int tr = t + r;
        // R_u: the unconverged residual columns, packed right after Y ([Y R_u] adjacent)
        EDA_CUDA_TRY(cudaMemcpyAsync(w.idx, idx.data(), r * sizeof(int), cudaMemcpyHostToDevice, s));
        k_gather_cols<<<ceil_div(d * r, 256), 256, 0, s>>>(d, r, w.idx, w.R, d, w.Y2, d);
        EDA_LAUNCHED();
        EDA_TRY(copy_mat_f64(d, r, w.Y2, d, w.R, d, s));
        for (int pass = 0; pass < 2; ++pass) {
            EDA_TRY(fin_tn(h, w, t, r, w.Y, w.R, d, w.Gt, t, s));
            EDA_TRY(fin_nn(h, w, t, r, -1.0, w.Y, w.Gt, t, 1.0, w.R, w.R, s));
        }
        EDA_TRY(cholqr_f64<T>(h, r, w.R, w.Y2, w, 2, s));
        // M R_u, then Rayleigh-Ritz on [Y R_u] (adjacent in memory, as are [MY M R_u] and their coordinates)
        EDA_TRY(m_apply_composed(h, r, w.R, d, w.MR, d, w.PQ, w.Uc, w.ZY + (size_t)nk * t, part, w.pcap, s));
        *mapplies += (r + b - 1) / b;
        EDA_TRY(fin_tn(h, w, tr, tr, w.Y, w.Z, d, w.A2, tr, s));
        EDA_TRY(symmetrize_f64(tr, w.A2, tr, s));
        EDA_TRY(symeig_f64(tr, w.A2, tr, r, tr - 1, w.theta, w.S, tr, &w.eig, h->status, h->cfg.seed + 13 + it,
                           1e-7, s));
        EDA_TRY(fin_nn(h, w, tr, t, 1.0, w.Y, w.S, tr, 0.0, nullptr, w.Y2, s));
        EDA_TRY(fin_nn(h, w, tr, t, 1.0, w.Z, w.S, tr, 0.0, nullptr, w.Z2, s));
        EDA_TRY(copy_mat_f64(d, t, w.Y2, d, w.Y, d, s));
        EDA_TRY(copy_mat_f64(d, t, w.Z2, d, w.Z, d, s));
        EDA_TRY(gemm_small_f64(false, false, nk, t, tr, 1.0, w.ZY, nk, w.S, tr, 0.0, w.PQ, nk, s));
        EDA_TRY(copy_mat_f64(nk, t, w.PQ, nk, w.ZY, nk, s));
        EDA_TRY(ritz_residuals<T>(d, t, w, relres_h, max_rel, s));
    }
    *iters_out = it + 1;
    return EDA_OK;
}

template <class T>
int solve_t(eda_ctx* h, int t, double tol, const double* V0, int b0, double* Vout, double* lambda, double* Yout,
            eda_solve_info* info, cudaStream_t s) {
    const int64_t d = h->d;
    const int n = (int)h->n, k = h->k;
    const int b = h->cfg.block_b;
    const bool mixed = !std::is_same<T, double>::value;
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
    SolveWs<T> w{};
    w.pcap = std::max<size_t>({size_t(1) << 19, (size_t)m_max * tw, (size_t)N * tw, (size_t)4 * t * t,
                               (size_t)(n + k) * t, (size_t)n * k});
    const int eig_n = std::max(m_max, 2 * t);
    size_t need = 0;
    auto addT = [&](size_t cnt) { need += a256(cnt * sizeof(T)); };
    auto add = [&](size_t cnt) { need += a256(cnt * 8); };
    addT((size_t)d * m_max);           // V
    addT((size_t)d * tw);              // W
    addT((size_t)d * tw);              // W1
    addT((size_t)d * tw);              // tmp
    addT((size_t)d * t);               // Yt
    add((size_t)m_max * m_max);        // Tm
    add((size_t)m_max * tw * 2 + (size_t)m_max * b * 2);   // C: both passes, and a refill's coefficients
    for (int i = 0; i < 7; ++i) add((size_t)b * b);
    add((size_t)(n + k) * tw * 2);     // P, Q (also the (n + k) x b coordinates of the composed M-apply)
    add(w.pcap);                       // partial (double-sized slots hold either type)
    add(t);                            // theta
    add((size_t)eig_n * t);            // S
    add(t);                            // relres
    for (int i = 0; i < 7; ++i) add((size_t)d * t);   // Y, R (adjacent), Z, MR (adjacent), Y2, Z2, Xt
    add((size_t)4 * t * t);            // A2
    add((size_t)(n + k) * t * 4);      // PQ, Uc, ZY
    add(t + 64);                       // idx (ints)
    add((size_t)d * tw);               // tmp64
    add((size_t)t * t * 4);            // Gt, Rt, Rti
    add(t);                            // lamd
    add(b + 64);                       // lost (ints)
    add(chol_inv_blocked_doubles(std::max(t, b)));   // CW
    need += symeig_work_bytes(eig_n, t) + 16384;
    const bool oz = !mixed && h->cfg.prec == EDA_F64_TC && h->ozblock;
    const size_t ozT_bytes = oz ? a256(oz_operand_bytes(m_max, d)) : 0, ozN_bytes = oz ? a256(oz_operand_bytes(d, m_max)) : 0;
    const size_t olist_bytes = oz ? a256((size_t)(d + 64) * sizeof(int)) : 0;
    need += ozT_bytes + ozN_bytes + olist_bytes;
    EDA_TRY(ensure_workspace(h, need));
    Arena a{static_cast<char*>(h->ws), h->ws_bytes, 0};
    w.V = a.take<T>((size_t)d * m_max);
    w.W = a.take<T>((size_t)d * tw);
    w.W1 = a.take<T>((size_t)d * tw);
    w.tmp = a.take<T>((size_t)d * tw);
    w.Yt = a.take<T>((size_t)d * t);
    w.Tm = a.take<double>((size_t)m_max * m_max);
    w.C = a.take<double>((size_t)m_max * tw * 2 + (size_t)m_max * b * 2);
    w.R1 = a.take<double>((size_t)b * b);
    w.R1i = a.take<double>((size_t)b * b);
    w.R2 = a.take<double>((size_t)b * b);
    w.R2i = a.take<double>((size_t)b * b);
    w.Bm = a.take<double>((size_t)b * b);
    (void)a.take<double>((size_t)b * b);
    (void)a.take<double>((size_t)b * b);
    w.P = a.take<double>((size_t)(n + k) * tw);
    w.Q = a.take<double>((size_t)(n + k) * tw);
    w.part = a.take<double>(w.pcap);
    w.theta = a.take<double>(t);
    w.S = a.take<double>((size_t)eig_n * t);
    w.relres = a.take<double>(t);
    w.Y = a.take<double>((size_t)2 * d * t);
    w.R = w.Y + (size_t)d * t;
    w.Z = a.take<double>((size_t)2 * d * t);
    w.MR = w.Z + (size_t)d * t;
    w.A2 = a.take<double>((size_t)4 * t * t);
    w.PQ = a.take<double>((size_t)(n + k) * t);
    w.Uc = a.take<double>((size_t)(n + k) * t);
    w.ZY = a.take<double>((size_t)(n + k) * t * 2);
    w.idx = a.take<int>(t + 64);
    w.Y2 = a.take<double>((size_t)d * t);
    w.Z2 = a.take<double>((size_t)d * t);
    w.Xt = a.take<double>((size_t)d * t);
    w.tmp64 = a.take<double>((size_t)d * tw);
    w.Gt = a.take<double>((size_t)t * t);
    w.Rt = a.take<double>((size_t)t * t);
    w.Rti = a.take<double>((size_t)t * t);
    (void)a.take<double>((size_t)t * t);
    w.lamd = a.take<double>(t);
    w.lost = a.take<int>(b + 64);
    w.CW = a.take<double>(chol_inv_blocked_doubles(std::max(t, b)));
    EDA_TRY(symeig_work_carve(a, eig_n, t, h->bar, &w.eig));
    if (!w.lost) return EDA_ERR_OOM;
    if (oz) {
        char* mT = a.take<char>(ozT_bytes);
        char* mN = a.take<char>(ozN_bytes);
        if (!mT || !mN) return EDA_ERR_OOM;
        EDA_TRY(oz_operand_init(m_max, d, mT, &w.VT, s));
        EDA_TRY(oz_operand_init(d, m_max, mN, &w.VN, s));
        w.olist = a.take<int>((size_t)d + 64);
        if (!w.olist) return EDA_ERR_OOM;
        w.oz = true;
        w.oz_cap = m_max;
    }
    EDA_CUDA_TRY(cudaMemsetAsync(h->status, 0, sizeof(int), s));
    EDA_CUDA_TRY(cudaMemsetAsync(w.Tm, 0, (size_t)m_max * m_max * 8, s));

    // ---- Krylov phase ----
    LanczosStats st;
    const double tol_k = mixed ? std::max(tol, 1e-4) : tol;
    int rc = run_lanczos<T>(h, t, tol_k, V0, b0, m_max, w, st, s);
    if (rc != EDA_OK && rc != EDA_ERR_NOT_CONVERGED) return rc;
    if (rc == EDA_ERR_NOT_CONVERGED && st.rr_cols == 0) return rc;
    EDA_TRY((copy_mat<T, double>(d, t, w.Yt, d, w.Y, d, s)));
    bool converged = st.converged;
    double max_rel = st.max_rel;
    std::vector<double> relres_h = st.relres;
    int refine_iters = 0;
    // FP64 phase: always for the mixed-precision solver; for the FP64 solver when directions were
    // dropped and replaced by fresh ones during the Krylov phase. The Ritz residual estimate only sees
    // the last block, while a direction dropped earlier (its size lost in the rounding of the block's
    // Gram) leaves a residual no later block measures; so the pairs are verified, and refined if
    // needed, with true FP64 residuals.
    if (mixed || st.refills > 0) {
        if (!mixed) EDA_TRY(ensure_cross_gram(h, static_cast<double*>(w.part), w.pcap, s));
        int mapp = 0;
        EDA_TRY(refine_f64<T>(h, t, tol, w, 6, &refine_iters, &mapp, relres_h, &max_rel, s));
        st.mapplies += mapp;
        converged = max_rel <= tol;
        st.conv_count = 0;
        for (int i = 0; i < t; ++i) st.conv_count += relres_h[i] <= tol;
    }
    int stw = 0;
    EDA_CUDA_TRY(cudaMemcpyAsync(&stw, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (stw & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (stw & ST_NONFINITE) return EDA_ERR_NONFINITE;

    // ---- descending order, recovery and orthonormalisation (FP64) ----
    k_reverse_cols<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, w.Y, d, w.Y2, d);
    EDA_LAUNCHED();
    k_reverse_vec<<<ceil_div(t, 128), 128, 0, s>>>(t, w.theta, w.lamd);
    EDA_LAUNCHED();
    EDA_CUDA_TRY(cudaMemcpyAsync(lambda, w.lamd, t * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (Yout) EDA_CUDA_TRY(cudaMemcpyAsync(Yout, w.Y2, (size_t)d * t * 8, cudaMemcpyDeviceToDevice, s));
    // x = exp(-c^2 S_W / 2) y = y + H_W K_W (H_W^T y)
    if (mixed) {
        // H_W^T Y is already known (the first n rows of the tracked coordinates Z^T Y): one sweep
        EDA_TRY(gemm_small_f64(false, false, n, t, n, 1.0, h->KW, n, w.ZY, n + k, 0.0, w.PQ, n, s));
        EDA_TRY(gemm_nn_f64(d, n, t, 1.0, h->HW, d, w.PQ, n, 1.0, w.Y, d, w.Z2, d, s));
        k_reverse_cols<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, w.Z2, d, w.Xt, d);
        EDA_LAUNCHED();
    } else if (h->cfg.prec == EDA_F64_TC && h->ozblock) {
        // the same product with the FP64-accurate tensor-core sweeps: H_W is the first n columns of the
        // split Z (the first n rows of its column-scaled operand, the first n of the reduction index of the
        // row-scaled one; the digits beyond meet zero rows of the narrow operand)
        ProfScope prof("exp_apply_w", s, 4.0 * d * n * t + 2.0 * (double)n * n * t, 8.0 * (2.0 * d * n + 3.0 * d * t));
        OzOperand AT = h->ozT, AN = h->ozN;
        AT.M = n;
        AT.mtiles = ceil_div(n, 128);
        AN.K = n;
        for (int c0 = 0; c0 < t; c0 += 32)
            EDA_TRY(oz_gemm(AT, h->oznb, std::min(32, t - c0), w.Y2 + (size_t)c0 * d, d, 1.0, 0.0, nullptr, 0,
                            w.P + (size_t)c0 * n, n, h->status, s));
        if (h->ozsmall) {
            for (int c0 = 0; c0 < t; c0 += 32)
                EDA_TRY(oz_gemm(h->ozKW, h->oznb, std::min(32, t - c0), w.P + (size_t)c0 * n, n, 1.0, 0.0, nullptr,
                                0, w.Q + (size_t)c0 * n, n, h->status, s));
        } else {
            EDA_TRY(gemm_small_f64(false, false, n, t, n, 1.0, h->KW, n, w.P, n, 0.0, w.Q, n, s));
        }
        for (int c0 = 0; c0 < t; c0 += 32)
            EDA_TRY(oz_gemm(AN, h->oznb, std::min(32, t - c0), w.Q + (size_t)c0 * n, n, 1.0, 1.0,
                            w.Y2 + (size_t)c0 * d, d, w.Xt + (size_t)c0 * d, d, h->status, s));
    } else {
        EDA_TRY(exp_apply<double>(d, h->HW, h->KW, n, "exp_apply_w", t, w.Y2, d, w.Xt, d, w.P, w.Q, w.part, w.pcap,
                                  s));
    }
    // V = orth(X_t): CholQR2 (leaves V in both)
    EDA_TRY(cholqr_f64<T>(h, t, w.Xt, Vout, w, 2, s));
    double true_max = -1.0;
    if (h->cfg.true_residuals) {
        // R = M Y - Y diag(theta) in FP64, in blocks of at most tw columns
        double* MY = w.Xt;
        for (int c0 = 0; c0 < t; c0 += tw) {
            const int cb = std::min(tw, t - c0);
            EDA_TRY(m_apply_t<double>(h, cb, w.Y2 + (size_t)c0 * d, d, MY + (size_t)c0 * d, d, w.tmp64, w.P, w.Q,
                                      w.part, w.pcap, s, /*allow_composed=*/false));
        }
        k_sub_scaled<<<ceil_div((int64_t)d * t, 256), 256, 0, s>>>(d, t, MY, d, w.Y2, d, w.lamd);
        EDA_LAUNCHED();
        EDA_TRY(col_norms_f64(d, t, MY, d, w.relres, s));
        std::vector<double> rn(t), lam_h(t);
        EDA_CUDA_TRY(cudaMemcpyAsync(rn.data(), w.relres, t * 8, cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaMemcpyAsync(lam_h.data(), w.lamd, t * 8, cudaMemcpyDeviceToHost, s));
        EDA_CUDA_TRY(cudaStreamSynchronize(s));
        true_max = 0.0;
        for (int i = 0; i < t; ++i) true_max = std::max(true_max, rn[i] / std::fabs(lam_h[i]));
        // the estimates must not claim more than an independent FP64 evaluation confirms
        if (true_max > 10.0 * tol) converged = false;
    }
    EDA_CUDA_TRY(cudaEventRecord(ev1, s));
    EDA_CUDA_TRY(cudaEventSynchronize(ev1));
    float ms = 0.f;
    EDA_CUDA_TRY(cudaEventElapsedTime(&ms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    EDA_CUDA_TRY(cudaMemcpyAsync(&stw, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    EDA_CUDA_TRY(cudaStreamSynchronize(s));
    if (stw & ST_TIMEOUT) return EDA_ERR_TIMEOUT;
    if (stw & ST_NONFINITE) return EDA_ERR_NONFINITE;
    if (info) {
        info->converged = st.conv_count;
        info->iters = st.iters;
        info->mapplies = st.mapplies;
        info->basis_cols = st.rr_cols;
        info->refills = st.refills;
        info->checks = st.checks;
        info->refine_iters = refine_iters;
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

}  // namespace

int solve_impl(eda_ctx* h, int t, double tol, const double* V0, int b0, double* Vout, double* lambda, double* Yout,
               eda_solve_info* info, cudaStream_t s) {
    if (h->cfg.prec == EDA_F64 || h->cfg.prec == EDA_F64_TC)
        return solve_t<double>(h, t, tol, V0, b0, Vout, lambda, Yout, info, s);
    if (h->cfg.prec == EDA_F32 || h->cfg.prec == EDA_BF16)
        return solve_t<float>(h, t, tol, V0, b0, Vout, lambda, Yout, info, s);
    return EDA_ERR_INVALID_ARG;
}

}  // namespace eda
