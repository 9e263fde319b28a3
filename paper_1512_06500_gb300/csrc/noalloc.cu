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

// Device address of the scratch array, looked up with the device current and kept per device
// together with the identity of the context it was looked up in. In host code the array's name
// is only a host-side stand-in and must never be handed to a kernel. A device reset (or a
// primary context released and created again) reloads the module, and the array may then sit
// at another address: the lookup is repeated whenever the current context is not the one the
// cached address belongs to.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id = 0;   // 0: nothing cached
    double* addr = nullptr;
};
ScratchSlot g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Identity of the calling thread's current context (0 when there is none or the driver does not
// offer context identities, in which case nothing is cached and every call looks the address up).
unsigned long long current_ctx_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        eda::note_cuda_error(e, __FILE__, __LINE__);
        return EDA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return EDA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchSlot& slot = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (id != 0 && slot.ctx_id == id && slot.addr) {
        *out = slot.addr;
        return EDA_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // with device `dev` current
    if (e != cudaSuccess || p == nullptr) {
        eda::note_cuda_error(e, __FILE__, __LINE__);
        return EDA_ERR_CUDA;
    }
    slot.addr = static_cast<double*>(p);
    slot.ctx_id = current_ctx_id();   // the lookup has made the device's primary context current
    *out = slot.addr;
    return EDA_OK;
}

// True when the byte ranges [a, a + na) and [b, b + nb) intersect.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" int eda_lowrank_exp_apply_noalloc(const double* H, int64_t d, int32_t m, const double* K,
                                             const double* X, double* Y, int64_t ld, int32_t b, void* stream) {
    if (!H || !K || !X || !Y || d < 1 || m < 1 || b < 1 || ld < d) return EDA_ERR_INVALID_ARG;
    const size_t mb = (size_t)m * (size_t)b;
    // P and Q take m*b doubles each; the partial sums need at least one more m*b slice.
    if (mb > kNoAllocScratchDoubles / 3) return EDA_ERR_INVALID_ARG;
    // Y is written while X, H and K are still being read (by other CTAs, and K after sweep 1):
    // it may overlap none of them.
    const size_t yspan = ((size_t)(b - 1) * ld + d) * sizeof(double);
    if (overlaps(Y, yspan, X, yspan) || overlaps(Y, yspan, H, (size_t)d * m * sizeof(double)) ||
        overlaps(Y, yspan, K, (size_t)m * m * sizeof(double)))
        return EDA_ERR_INVALID_ARG;
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
