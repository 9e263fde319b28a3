// Tensor-core exp-vector product for H stored in bfloat16 (5th-generation tensor cores: tcgen05.mma
// with the accumulator in tensor memory):
//     sweep 1   P = H^T X      M = m (columns of H), N = b, K = d, split over d across CTAs
//     small     Q = K P        (FP64, shared code)
//     sweep 2   Y = X + H Q    M = d, N = b, K = m
// X and Y are single precision. Each X (and Q) value enters the MMA as a bfloat16 hi + lo pair
// (hi = bf16(x), lo = bf16(x - hi)), two MMAs per K step, so the product error is set by the
// bfloat16 rounding of H alone; accumulation is FP32 in tensor memory, split sums are added in
// FP64. Operands are staged in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix) with two stages: cp.async fills stage s + 1 while the MMAs
// of stage s run; a tcgen05.commit to an mbarrier per stage tells the loaders when a buffer is free.
// Every mbarrier wait is bounded; on timeout the kernel records ST_TIMEOUT and finishes.
#include "eda_internal.cuh"

#include <cuda_bf16.h>

namespace eda {

namespace {

constexpr int TC_M = 128;        // MMA rows (TMEM lanes)
constexpr int TC_KS = 64;        // K per shared-memory stage (4 MMAs of K = 16)
constexpr long long TC_SPIN = 1LL << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok;
}
// bounded wait; returns false (and records the timeout) when it gives up
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, int* status) {
    long long it = 0;
    while (!mbar_try_wait(mbar, parity)) {
        if (++it > TC_SPIN) {
            atomicOr(status, ST_TIMEOUT);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension byte offset (between
// core matrices along K), stride-dimension byte offset (between 8-row groups along M/N), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of row r (of R rows) and 16-byte K chunk c inside a K-major no-swizzle stage
__device__ __forceinline__ int core_off(int r, int c, int R) { return (c * (R / 8) + r / 8) * 128 + (r % 8) * 16; }

__device__ __forceinline__ void split8(const float (&x)[8], uint4& hi, uint4& lo) {
    __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        h[u] = __float2bfloat16_rn(x[u]);
        l[u] = __float2bfloat16_rn(x[u] - __bfloat162float(h[u]));
    }
    hi = *reinterpret_cast<const uint4*>(h);
    lo = *reinterpret_cast<const uint4*>(l);
}

template <int N>
struct TcSmem {
    __nv_bfloat16 A[2][TC_M * TC_KS];   // 2 x 16 KB
    __nv_bfloat16 Bh[2][N * TC_KS];
    __nv_bfloat16 Bl[2][N * TC_KS];
    uint64_t mbar[2];
    uint32_t tbase;
};

// Issue the 4 K-steps of one stage: D += A Bh^T + A Bl^T.
template <int N>
__device__ __forceinline__ void issue_stage(TcSmem<N>& sm, int buf, uint32_t tmem, bool first) {
    const uint32_t a0 = smem_u32(sm.A[buf]), bh = smem_u32(sm.Bh[buf]), bl = smem_u32(sm.Bl[buf]);
    constexpr uint32_t LA = (TC_M / 8) * 128, LB = (N / 8) * 128;
    constexpr uint32_t id = idesc_bf16(TC_M, N);
#pragma unroll
    for (int ks = 0; ks < TC_KS / 16; ++ks) {
        const uint64_t ad = smem_desc(a0 + ks * 2 * LA, LA, 128);
        mma_bf16(tmem, ad, smem_desc(bh + ks * 2 * LB, LB, 128), id, (first && ks == 0) ? 0u : 1u);
        mma_bf16(tmem, ad, smem_desc(bl + ks * 2 * LB, LB, 128), id, 1u);
    }
}

// ---- sweep 1: partial[split][j][i] = sum_{k in split} H[k, i] X[k, j] --------------------------------
// H: bf16, column-major, leading dimension ldh (multiple of 8, zero padded up to a multiple of TC_KS).
template <int N>
__global__ void __launch_bounds__(128) k_tc_sweep1(const __nv_bfloat16* __restrict__ H, int64_t ldh, int m,
                                                    const float* __restrict__ X, int64_t ldx, int64_t d, int b,
                                                    int64_t rows_per_split, float* __restrict__ partial, int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    TcSmem<N>& sm = *reinterpret_cast<TcSmem<N>*>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int i0 = blockIdx.x * TC_M;
    const int split = blockIdx.y;
    const int64_t k_begin = (int64_t)split * rows_per_split;
    const int64_t k_end = min(ldh, k_begin + rows_per_split);          // ldh: padded rows, zeros beyond d
    const int nst = (int)((k_end - k_begin + TC_KS - 1) / TC_KS);
    if (warp == 0) {
        tmem_alloc(&sm.tbase, 32);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tbase;

    auto load = [&](int s, int buf) {
        const int64_t k0 = k_begin + (int64_t)s * TC_KS;
        char* A = reinterpret_cast<char*>(sm.A[buf]);
        for (int e = tid; e < TC_M * 8; e += 128) {
            const int i = e >> 3, c = e & 7;
            const int col = i0 + i;
            char* dst = A + core_off(i, c, TC_M);
            if (col < m && k0 + 8 * c < k_end) cp_async16(dst, H + (int64_t)col * ldh + k0 + 8 * c);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
        }
        char* Bh = reinterpret_cast<char*>(sm.Bh[buf]);
        char* Bl = reinterpret_cast<char*>(sm.Bl[buf]);
        for (int e = tid; e < N * 8; e += 128) {
            const int j = e >> 3, c = e & 7;
            float x[8];
            const int64_t k = k0 + 8 * c;
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (j < b && k + u < d) ? X[(int64_t)j * ldx + k + u] : 0.f;
            uint4 hi, lo;
            split8(x, hi, lo);
            *reinterpret_cast<uint4*>(Bh + core_off(j, c, N)) = hi;
            *reinterpret_cast<uint4*>(Bl + core_off(j, c, N)) = lo;
        }
        cp_async_commit();
    };

    bool ok = true;
    if (nst > 0) load(0, 0);
    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        if (s + 1 < nst) {
            if (s >= 1) ok = mbar_wait(&sm.mbar[buf ^ 1], ((s - 1) >> 1) & 1, status) && ok;   // stage s-1 done
            load(s + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_stage<N>(sm, buf, tmem, s == 0);
            mma_commit(&sm.mbar[buf]);
        }
    }
    if (nst > 0) ok = mbar_wait(&sm.mbar[(nst - 1) & 1], ((nst - 1) >> 1) & 1, status) && ok;
    tc_fence_after();
    // epilogue: warp w owns TMEM lanes 32w..32w+31 (rows i0 + 32w + lane)
    const int i = i0 + 32 * warp + (tid & 31);
    float* out = partial + (int64_t)split * m * b;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int j = c0 + c;
            if (ok && nst > 0 && i < m && j < b) out[(int64_t)j * m + i] = __uint_as_float(r[c]);
            else if (i < m && j < b) out[(int64_t)j * m + i] = 0.f;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// ---- sweep 2: Y[r, j] = X[r, j] + sum_l H[r, l] Q[l, j] ----------------------------------------------------
// Hrm: bf16, row-major d x ldm (ldm multiple of TC_KS, zero columns beyond m). Q: double, m x b (ld ldq).
template <int N>
__global__ void __launch_bounds__(128) k_tc_sweep2(const __nv_bfloat16* __restrict__ Hrm, int64_t d, int ldm, int m,
                                                    const double* __restrict__ Q, int ldq, int b,
                                                    const float* __restrict__ X, int64_t ldx, float* __restrict__ Y,
                                                    int64_t ldy, int* status) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    TcSmem<N>& sm = *reinterpret_cast<TcSmem<N>*>(smraw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * TC_M;
    const int nst = ldm / TC_KS;
    if (warp == 0) {
        tmem_alloc(&sm.tbase, 32);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&sm.mbar[0], 1);
        mbar_init(&sm.mbar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tbase;

    auto load = [&](int s, int buf) {
        const int l0 = s * TC_KS;
        char* A = reinterpret_cast<char*>(sm.A[buf]);
        for (int e = tid; e < TC_M * 8; e += 128) {
            const int i = e >> 3, c = e & 7;
            const int64_t row = r0 + i;
            char* dst = A + core_off(i, c, TC_M);
            if (row < d) cp_async16(dst, Hrm + row * ldm + l0 + 8 * c);
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
        }
        char* Bh = reinterpret_cast<char*>(sm.Bh[buf]);
        char* Bl = reinterpret_cast<char*>(sm.Bl[buf]);
        for (int e = tid; e < N * 8; e += 128) {
            const int j = e >> 3, c = e & 7;
            float x[8];
            const int l = l0 + 8 * c;
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (j < b && l + u < m) ? (float)Q[(int64_t)j * ldq + l + u] : 0.f;
            uint4 hi, lo;
            split8(x, hi, lo);
            *reinterpret_cast<uint4*>(Bh + core_off(j, c, N)) = hi;
            *reinterpret_cast<uint4*>(Bl + core_off(j, c, N)) = lo;
        }
        cp_async_commit();
    };

    bool ok = true;
    if (nst > 0) load(0, 0);
    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        if (s + 1 < nst) {
            if (s >= 1) ok = mbar_wait(&sm.mbar[buf ^ 1], ((s - 1) >> 1) & 1, status) && ok;
            load(s + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            issue_stage<N>(sm, buf, tmem, s == 0);
            mma_commit(&sm.mbar[buf]);
        }
    }
    if (nst > 0) ok = mbar_wait(&sm.mbar[(nst - 1) & 1], ((nst - 1) >> 1) & 1, status) && ok;
    tc_fence_after();
    const int64_t row = r0 + 32 * warp + (tid & 31);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int j = c0 + c;
            if (row < d && j < b) {
                const float acc = (ok && nst > 0) ? __uint_as_float(r[c]) : 0.f;
                Y[(int64_t)j * ldy + row] = X[(int64_t)j * ldx + row] + acc;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// P[i, j] = sum_s partial[s][j][i] (FP64 sums of the FP32 split results, fixed order)
__global__ void k_reduce_f32(int m, int b, int splits, const float* __restrict__ partial, double* __restrict__ P,
                             int ldp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * b) return;
    const int i = (int)(e % m), j = (int)(e / m);
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)partial[(int64_t)s * m * b + e];
    P[(int64_t)j * ldp + i] = acc;
}

// column-major FP64 d x m -> column-major bf16 with leading dimension ldh (zero rows beyond d)
__global__ void k_to_bf16_cm(int64_t d, int m, const double* __restrict__ H, int64_t ld, __nv_bfloat16* out,
                             int64_t ldh) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ldh * m) return;
    const int64_t r = e % ldh;
    const int64_t c = e / ldh;
    out[e] = __float2bfloat16_rn(r < d ? (float)H[c * ld + r] : 0.f);
}
// column-major FP64 d x m -> row-major bf16 d x ldm (zero columns beyond m)
__global__ void k_to_bf16_rm(int64_t d, int m, const double* __restrict__ H, int64_t ld, __nv_bfloat16* out, int ldm) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d * ldm) return;
    const int64_t r = e / ldm;
    const int c = (int)(e % ldm);
    out[e] = __float2bfloat16_rn(c < m ? (float)H[(int64_t)c * ld + r] : 0.f);
}

template <int N>
int launch_tc(const TcFactor& f, const double* K, int b, const float* X, int64_t ldx, float* Y, int64_t ldy, double* P,
              double* Q, float* partial, size_t partial_cap, int* status, cudaStream_t s) {
    const size_t smem = sizeof(TcSmem<N>) + 1024;
    static bool attr = false;
    if (!attr) {
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int m = f.m;
    const int tiles = ceil_div(m, TC_M);
    int splits = std::max(1, ceil_div(2 * 152, tiles));
    splits = (int)std::min<int64_t>(splits, std::max<int64_t>(1, f.ldh / TC_KS));
    while (splits > 1 && (size_t)splits * m * b > partial_cap) --splits;
    if ((size_t)splits * m * b > partial_cap) return EDA_ERR_INVALID_ARG;
    int64_t rows = (f.ldh + splits - 1) / splits;
    rows = (rows + TC_KS - 1) / TC_KS * TC_KS;
    splits = (int)std::max<int64_t>(1, (f.ldh + rows - 1) / rows);
    {
        ProfScope prof("tc_sweep1", s);
        k_tc_sweep1<N><<<dim3(tiles, splits), 128, smem, s>>>(f.Hcm, f.ldh, m, X, ldx, f.d, b, rows, partial, status);
        EDA_LAUNCHED();
    }
    k_reduce_f32<<<ceil_div((int64_t)m * b, 256), 256, 0, s>>>(m, b, splits, partial, P, m);
    EDA_LAUNCHED();
    EDA_TRY(gemm_small_f64(false, false, m, b, m, 1.0, K, m, P, m, 0.0, Q, m, s));
    {
        ProfScope prof("tc_sweep2", s);
        k_tc_sweep2<N><<<ceil_div(f.d, TC_M), 128, smem, s>>>(f.Hrm, f.d, f.ldm, m, Q, m, b, X, ldx, Y, ldy, status);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

}  // namespace

int tc_factor_make(const double* H, int64_t d, int m, __nv_bfloat16* Hcm, __nv_bfloat16* Hrm, TcFactor* f,
                   cudaStream_t s) {
    f->d = d;
    f->m = m;
    f->ldh = tc_pad_rows(d);
    f->ldm = tc_pad_cols(m);
    f->Hcm = Hcm;
    f->Hrm = Hrm;
    k_to_bf16_cm<<<ceil_div(f->ldh * m, 256), 256, 0, s>>>(d, m, H, d, Hcm, f->ldh);
    EDA_LAUNCHED();
    k_to_bf16_rm<<<ceil_div(d * f->ldm, 256), 256, 0, s>>>(d, m, H, d, Hrm, f->ldm);
    EDA_LAUNCHED();
    return EDA_OK;
}

int exp_apply_tc(const TcFactor& f, const double* K, const char* tag, int b, const float* X, int64_t ldx, float* Y,
                 int64_t ldy, double* P, double* Q, void* partial, size_t partial_cap, int* status, cudaStream_t s) {
    ProfScope prof(tag, s);
    if (b <= 16) return launch_tc<16>(f, K, b, X, ldx, Y, ldy, P, Q, static_cast<float*>(partial), partial_cap, status, s);
    if (b <= 32) return launch_tc<32>(f, K, b, X, ldx, Y, ldy, P, Q, static_cast<float*>(partial), partial_cap, status, s);
    // wider blocks: column slices of 32
    for (int c0 = 0; c0 < b; c0 += 32) {
        const int cb = std::min(32, b - c0);
        EDA_TRY(launch_tc<32>(f, K, cb, X + (int64_t)c0 * ldx, ldx, Y + (int64_t)c0 * ldy, ldy, P, Q,
                              static_cast<float*>(partial), partial_cap, status, s));
    }
    return EDA_OK;
}

}  // namespace eda
