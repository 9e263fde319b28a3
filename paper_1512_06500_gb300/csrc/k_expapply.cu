// Matrix exponential-vector products of Theorem 3.1 in the form
//     exp(alpha H H^T) X = X + H K(alpha) (H^T X),   K(alpha) = alpha phi(alpha H^T H),
// with H tall (d x m, m = n or k) and X a d x b block. Two sweeps over H: the reduction
// P = H^T X over all d rows must finish before any row of Y = X + H (K P) is written.
#include "eda_internal.cuh"

namespace eda {

int exp_apply_f64(int64_t d, const ExpOp& op, int b, const double* X, int64_t ldx, double* Y, int64_t ldy,
                  double* P, double* Q, double* partial, size_t partial_cap, cudaStream_t s) {
    ProfScope prof(op.tag ? op.tag : "exp_apply", s);
    const int m = op.m;
    // sweep 1: P = H^T X (m x b), split over d with a fixed-order reduction
    EDA_TRY(gemm_tn_f64(d, m, b, 1.0, op.H, d, X, ldx, 0.0, P, m, partial, partial_cap, s));
    // Q = K P (m x b)
    EDA_TRY(gemm_small_f64(false, false, m, b, m, 1.0, op.K, m, P, m, 0.0, Q, m, s));
    // sweep 2: Y = X + H Q
    EDA_TRY(gemm_nn_f64(d, m, b, 1.0, op.H, d, Q, m, 1.0, X, ldx, Y, ldy, s));
    return EDA_OK;
}

}  // namespace eda
