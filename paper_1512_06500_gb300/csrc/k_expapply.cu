// Matrix exponential-vector products of Theorem 3.1 in the form
//     exp(alpha H H^T) X = X + H K(alpha) (H^T X),   K(alpha) = alpha phi(alpha H^T H),
// with H tall (d x m, m = n or k) and X a d x b block. Two sweeps over H: the reduction
// P = H^T X over all d rows must finish before any row of Y = X + H (K P) is written.
// The sweeps run in the storage type T of H and X (double, or float for the mixed solver);
// P, Q = K P and K stay in double.
#include "eda_internal.cuh"

namespace eda {

template <class T>
int exp_apply(int64_t d, const T* H, const double* K, int m, const char* tag, int b, const T* X, int64_t ldx, T* Y,
              int64_t ldy, double* P, double* Q, void* partial, size_t partial_cap, cudaStream_t s) {
    ProfScope prof(tag, s, 4.0 * d * m * b + 2.0 * m * m * b, (double)sizeof(T) * (2.0 * d * m + 3.0 * d * b));
    // sweep 1: P = H^T X (m x b), split over d with a fixed-order reduction
    EDA_TRY(gemm_tn<T>(d, m, b, 1.0, H, d, X, ldx, 0.0, P, m, partial, partial_cap, s));
    // Q = K P (m x b)
    EDA_TRY(gemm_small_f64(false, false, m, b, m, 1.0, K, m, P, m, 0.0, Q, m, s));
    // sweep 2: Y = X + H Q
    EDA_TRY(gemm_nn<T>(d, m, b, 1.0, H, d, Q, m, 1.0, X, ldx, Y, ldy, s));
    return EDA_OK;
}

template int exp_apply<double>(int64_t, const double*, const double*, int, const char*, int, const double*, int64_t,
                               double*, int64_t, double*, double*, void*, size_t, cudaStream_t);
template int exp_apply<float>(int64_t, const float*, const double*, int, const char*, int, const float*, int64_t,
                              float*, int64_t, double*, double*, void*, size_t, cudaStream_t);

int exp_apply_f64(int64_t d, const ExpOp& op, int b, const double* X, int64_t ldx, double* Y, int64_t ldy,
                  double* P, double* Q, double* partial, size_t partial_cap, cudaStream_t s) {
    return exp_apply<double>(d, op.H, op.K, op.m, op.tag ? op.tag : "exp_apply", b, X, ldx, Y, ldy, P, Q, partial,
                             partial_cap, s);
}

}  // namespace eda
