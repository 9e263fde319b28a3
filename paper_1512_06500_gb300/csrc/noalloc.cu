// Exp-vector product for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc/cudaFree: code embedded in a host framework that owns a
// fixed device-memory budget and forbids allocations outside its own pool, or latency-critical
// loops where an allocation (which may synchronise the device) is not acceptable. This entry
// point takes the operator (H, K) and the blocks X, Y from the caller and keeps its temporaries
// (the split-K partial sums of H^T X, P = H^T X and Q = K P) in one fixed device array defined
// in this file. It allocates nothing.
#include "eda_internal.cuh"

#include <mutex>

namespace {

// Fixed scratch: 2^19 doubles (4 MiB). Every GPU that loads the library holds it until exit.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 19;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of the scratch array, looked up once per device. In host code the array's
// name is only a host-side stand-in and must never be handed to a kernel.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        eda::note_cuda_error(e);
        return EDA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return EDA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // with device `dev` current
        if (e != cudaSuccess || p == nullptr) {
            eda::note_cuda_error(e);
            return EDA_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return EDA_OK;
}

}  // namespace

extern "C" int eda_lowrank_exp_apply_noalloc(const double* H, int64_t d, int32_t m, const double* K,
                                             const double* X, double* Y, int64_t ld, int32_t b, void* stream) {
    if (!H || !K || !X || !Y || d < 1 || m < 1 || b < 1 || ld < d) return EDA_ERR_INVALID_ARG;
    const size_t mb = (size_t)m * (size_t)b;
    // P and Q take m*b doubles each; the partial sums need at least one more m*b slice.
    if (mb > kNoAllocScratchDoubles / 3) return EDA_ERR_INVALID_ARG;
    const char* xb = reinterpret_cast<const char*>(X);
    const char* yb = reinterpret_cast<const char*>(Y);
    const size_t span = ((size_t)(b - 1) * ld + d) * sizeof(double);
    if (xb < yb + span && yb < xb + span) return EDA_ERR_INVALID_ARG;
    double* scratch = nullptr;
    if (int rc = scratch_address(&scratch)) return rc;
    double* P = scratch;
    double* Q = scratch + mb;
    double* partial = scratch + 2 * mb;
    const size_t cap = kNoAllocScratchDoubles - 2 * mb;
    // Every scratch element read in this call is written earlier in the same call, so nothing
    // has to be cleared between calls.
    const eda::ExpOp op{H, K, m, "exp_apply_noalloc"};
    return eda::exp_apply_f64(d, op, b, X, ld, Y, ld, P, Q, partial, cap, static_cast<cudaStream_t>(stream));
}
