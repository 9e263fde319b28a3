// Tensor-core exp-vector product for H stored in bfloat16 (5th-generation tensor cores: tcgen05.mma
// with the accumulator in tensor memory, operands brought in by the Tensor Memory Accelerator):
//     split     X -> (Xhi, Xlo) bf16 pair          (hi = bf16(x), lo = bf16(x - hi))
//     sweep 1   P = H^T X      M = m (columns of H), N = b, K = d, split over d across CTAs
//     small     Q = K P        (FP32, written directly as a bf16 hi/lo pair)
//     sweep 2   Y = X + H Q    M = d, N = b, K = m, from a row-major bf16 copy of H
// Every product is bf16 x (bf16 hi + bf16 lo) with FP32 accumulation, so the error is set by the
// bf16 rounding of H; split sums are added in FP64.
//
// Each CTA runs a 4-stage shared-memory ring: one thread issues cp.async.bulk.tensor loads (a box of
// 8 elements x rows lands exactly in the no-swizzle K-major core-matrix layout: row r of 16-byte
// chunk c at c * rows * 16 + r * 16), one thread issues tcgen05.mma (4 K-steps of 16, hi and lo per
// step) and commits each stage to the stage's "empty" mbarrier; the four warps read the 128 x N FP32
// accumulator out of tensor memory at the end. Every wait is bounded (ST_TIMEOUT on give-up).
#include "eda_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

namespace eda {

namespace {

constexpr int TC_M = 128;        // MMA rows (tensor-memory lanes)
constexpr int TC_KS = 64;        // K per stage (4 MMAs of K = 16)
constexpr int TC_STAGES = 4;
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
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
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
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}
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

template <int N>
struct TcRing {
    __nv_bfloat16 A[TC_STAGES][TC_M * TC_KS];   // 16 KB per stage
    __nv_bfloat16 Bh[TC_STAGES][N * TC_KS];
    __nv_bfloat16 Bl[TC_STAGES][N * TC_KS];
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t done;
    uint32_t tbase;
};

// Main loop shared by both sweeps: K stages [0, nst) starting at element k_begin; A rows from
// a_row0 (tensor map tmA), B rows 0..N-1 (tmBh, tmBl, same K coordinates). Returns false on timeout.
template <int N>
__device__ bool tc_mainloop(TcRing<N>& sm, const CUtensorMap* tmA, const CUtensorMap* tmBh, const CUtensorMap* tmBl,
                            int a_row0, int k_begin, int nst, uint32_t tmem, int* status, bool maps3d) {
    const int tid = threadIdx.x;
    bool ok = true;
    if (tid == 0) {
        // producer: one thread issues all bulk tensor loads
        constexpr uint32_t bytes = TC_M * TC_KS * 2 + 2 * N * TC_KS * 2;
        for (int s = 0; s < nst && ok; ++s) {
            const int slot = s % TC_STAGES;
            if (s >= TC_STAGES) ok = mbar_wait(&sm.empty[slot], ((s / TC_STAGES) - 1) & 1, status);
            if (!ok) break;
            mbar_expect_tx(&sm.full[slot], bytes);
            const int k0 = k_begin + s * TC_KS;
            char* A = reinterpret_cast<char*>(sm.A[slot]);
            char* Bh = reinterpret_cast<char*>(sm.Bh[slot]);
            char* Bl = reinterpret_cast<char*>(sm.Bl[slot]);
            if (maps3d) {
                // (element-in-chunk, row, chunk) boxes land directly in the core-matrix layout
                tma_load_3d(A, tmA, 0, a_row0, k0 / 8, &sm.full[slot]);
                tma_load_3d(Bh, tmBh, 0, 0, k0 / 8, &sm.full[slot]);
                tma_load_3d(Bl, tmBl, 0, 0, k0 / 8, &sm.full[slot]);
            } else {
#pragma unroll
                for (int c = 0; c < TC_KS / 8; ++c) {
                    tma_load_2d(A + c * TC_M * 16, tmA, k0 + 8 * c, a_row0, &sm.full[slot]);
                    tma_load_2d(Bh + c * N * 16, tmBh, k0 + 8 * c, 0, &sm.full[slot]);
                    tma_load_2d(Bl + c * N * 16, tmBl, k0 + 8 * c, 0, &sm.full[slot]);
                }
            }
        }
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t LA = TC_M * 16, LB = N * 16;   // byte stride between 16-byte K chunks
        constexpr uint32_t id = idesc_bf16(TC_M, N);
        for (int s = 0; s < nst; ++s) {
            const int slot = s % TC_STAGES;
            if (!mbar_wait(&sm.full[slot], (s / TC_STAGES) & 1, status)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sm.A[slot]), bh = smem_u32(sm.Bh[slot]), bl = smem_u32(sm.Bl[slot]);
#pragma unroll
            for (int ks = 0; ks < TC_KS / 16; ++ks) {
                const uint64_t ad = smem_desc(a0 + ks * 2 * LA, LA, 128);
                mma_bf16(tmem, ad, smem_desc(bh + ks * 2 * LB, LB, 128), id, (s == 0 && ks == 0) ? 0u : 1u);
                mma_bf16(tmem, ad, smem_desc(bl + ks * 2 * LB, LB, 128), id, 1u);
            }
            mma_commit(&sm.empty[slot]);
        }
        mma_commit(&sm.done);
    }
    // one thread waits for the accumulator; the others rest on the CTA barrier instead of spinning
    __shared__ int s_ok;
    if (tid == 0) s_ok = (mbar_wait(&sm.done, 0, status) && ok) ? 1 : 0;
    if (tid == 32 && !ok) atomicOr(status, ST_TIMEOUT);
    __syncthreads();
    const bool fin = s_ok != 0;
    tc_fence_after();
    return fin;
}

template <int N>
__device__ void tc_setup(TcRing<N>& sm) {
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        tmem_alloc(&sm.tbase, 32);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(&sm.done, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

template <int N>
__device__ void tc_teardown(TcRing<N>& sm, uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 32);
}

// ---- sweep 1: partial[split][j][i] = sum_{k in split} H[k, i] X[k, j] ---------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_tc_sweep1(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmBh,
                                                    const __grid_constant__ CUtensorMap tmBl, int m, int b,
                                                    int rows_per_split, int ldh, float* __restrict__ partial,
                                                    int* status, int maps3d) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    TcRing<N>& sm = *reinterpret_cast<TcRing<N>*>(smraw);
    tc_setup<N>(sm);
    const uint32_t tmem = sm.tbase;
    const int i0 = blockIdx.x * TC_M;
    const int split = blockIdx.y;
    const int k_begin = split * rows_per_split;
    const int nst = (min(ldh, k_begin + rows_per_split) - k_begin) / TC_KS;
    const bool ok = tc_mainloop<N>(sm, &tmA, &tmBh, &tmBl, i0, k_begin, nst, tmem, status, maps3d != 0);
    const int warp = threadIdx.x >> 5;
    const int i = i0 + 32 * warp + (threadIdx.x & 31);
    float* out = partial + (int64_t)split * m * b;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + c0, r);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int j = c0 + c;
            if (i < m && j < b) out[(int64_t)j * m + i] = (ok && nst > 0) ? __uint_as_float(r[c]) : 0.f;
        }
    }
    tc_teardown<N>(sm, tmem);
}

// ---- sweep 2: Y[r, j] = X[r, j] + sum_l H[r, l] Q[l, j] -------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_tc_sweep2(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmBh,
                                                    const __grid_constant__ CUtensorMap tmBl, int64_t d, int ldm, int b,
                                                    const float* __restrict__ X, int64_t ldx, float* __restrict__ Y,
                                                    int64_t ldy, int* status, int maps3d) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    TcRing<N>& sm = *reinterpret_cast<TcRing<N>*>(smraw);
    tc_setup<N>(sm);
    const uint32_t tmem = sm.tbase;
    const int r0 = blockIdx.x * TC_M;
    const int nst = ldm / TC_KS;
    const bool ok = tc_mainloop<N>(sm, &tmA, &tmBh, &tmBl, r0, 0, nst, tmem, status, maps3d != 0);
    const int warp = threadIdx.x >> 5;
    const int64_t row = r0 + 32 * warp + (threadIdx.x & 31);
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
    tc_teardown<N>(sm, tmem);
}

// X (d x b, ld ldx) -> Xhi, Xlo (bf16, column-major ld ldh, rows >= d zero)
__global__ void k_split_x(int64_t d, int b, const float* __restrict__ X, int64_t ldx, int64_t ldh,
                          __nv_bfloat16* Xhi, __nv_bfloat16* Xlo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ldh * b) return;
    const int64_t r = e % ldh;
    const int64_t j = e / ldh;
    const float x = r < d ? X[j * ldx + r] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    Xhi[e] = h;
    Xlo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// P[i, j] = sum_s partial[s][j][i] in FP64 (fixed order), stored as float
__global__ void k_reduce_f32(int m, int b, int splits, const float* __restrict__ partial, float* __restrict__ P) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * b) return;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += (double)partial[(int64_t)s * m * b + e];
    P[e] = (float)acc;
}

// Q = K P (m x m times m x b, FP32) written as bf16 hi/lo, column-major ld ldq (rows m..ldq-1 zero).
// CTA = 4 warps for one 32-row block and NB columns; warp w sums a quarter of the inner dimension
// (K is read once per NB columns); quarters are added in a fixed order through shared memory.
template <int NB>
__global__ void __launch_bounds__(128) k_kp_split(int m, int b, const float* __restrict__ K, const float* __restrict__ P,
                                                  int ldq, __nv_bfloat16* Qhi, __nv_bfloat16* Qlo) {
    __shared__ float part[3][32][NB + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int j0 = blockIdx.y * NB;
    P += (int64_t)j0 * m;
    Qhi += (int64_t)j0 * ldq;
    Qlo += (int64_t)j0 * ldq;
    b = min(NB, b - j0);
    const int q = (m + 3) / 4;
    const int lb = w * q, le = min(m, lb + q);
    float acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = 0.f;
    if (i < m) {
        for (int l = lb; l < le; ++l) {
            const float kv = K[(int64_t)l * m + i];
#pragma unroll
            for (int j = 0; j < NB; ++j)
                if (j < b) acc[j] = fmaf(kv, __ldg(P + (int64_t)j * m + l), acc[j]);
        }
    }
    if (w > 0) {
#pragma unroll
        for (int j = 0; j < NB; ++j) part[w - 1][lane][j] = acc[j];
    }
    __syncthreads();
    if (w == 0 && i < ldq) {
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (j >= b) break;
            const float qv = (i < m) ? (acc[j] + part[0][lane][j]) + (part[1][lane][j] + part[2][lane][j]) : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(qv);
            Qhi[(int64_t)j * ldq + i] = h;
            Qlo[(int64_t)j * ldq + i] = __float2bfloat16_rn(qv - __bfloat162float(h));
        }
    }
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
__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ o) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) o[e] = (float)a[e];
}

// ---- tensor maps ------------------------------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3-D view of the same bf16 matrix: (element within a 16-byte chunk, row, chunk) with strides
// (2 B, ld * 2 B, 16 B) and a box of 8 x box_rows x 8, i.e. one whole 64-element K stage whose
// chunks land box_rows * 16 bytes apart: the no-swizzle core-matrix layout. Returns false when
// the encoder does not accept this view (the caller then uses 2-D boxes).
bool make_map3(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows) {
    EncodeTiledFn enc = encoder();
    if (!enc || inner % 8) return false;
    const cuuint64_t dims[3] = {8, outer, inner / 8};
    const cuuint64_t strides[2] = {ld * 2, 16};
    const cuuint32_t box[3] = {8, box_rows, 8};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2-D bf16 tensor: inner extent `inner` (contiguous), `outer` rows of stride `ld` elements; box of
// 8 inner elements x `box_rows` rows (16 bytes x rows); reads outside the extents return zeros.
int make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows) {
    EncodeTiledFn enc = encoder();
    if (!enc) return EDA_ERR_CUDA;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {8, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? EDA_OK : EDA_ERR_CUDA;
}

template <int N>
int launch_tc(const TcFactor& f, const TcBuffers& bufs, int b, const float* X, int64_t ldx, float* Y, int64_t ldy,
              float* partial, size_t partial_cap, int* status, cudaStream_t s) {
    const size_t smem = sizeof(TcRing<N>) + 1024;
    static bool attr = false;
    if (!attr) {
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int m = f.m;
    const int nb = N == 16 ? 0 : 1;
    // split X into its bf16 pair
    k_split_x<<<ceil_div(f.ldh * b, 256), 256, 0, s>>>(f.d, b, X, ldx, f.ldh, bufs.Xhi, bufs.Xlo);
    EDA_LAUNCHED();
    // sweep 1 over split ranges of whole stages
    const int tiles = ceil_div(m, TC_M);
    const int kst = (int)(f.ldh / TC_KS);
    int splits = std::max(1, std::min(kst, ceil_div(2 * 152, tiles)));
    while (splits > 1 && (size_t)splits * m * b > partial_cap) --splits;
    if ((size_t)splits * m * b > partial_cap) return EDA_ERR_INVALID_ARG;
    const int rows = ceil_div(kst, splits) * TC_KS;
    splits = ceil_div(f.ldh, rows);
    {
        ProfScope prof("tc_sweep1", s);
        const int m3 = (f.maps3d && bufs.maps3d) ? 1 : 0;
        k_tc_sweep1<N><<<dim3(tiles, splits), 128, smem, s>>>(m3 ? f.mapA1_3 : f.mapA1, m3 ? bufs.mapXh3[nb] : bufs.mapXh[nb],
                                                            m3 ? bufs.mapXl3[nb] : bufs.mapXl[nb], m, b, rows,
                                                            (int)f.ldh, partial, status, m3);
        EDA_LAUNCHED();
    }
    k_reduce_f32<<<ceil_div((int64_t)m * b, 256), 256, 0, s>>>(m, b, splits, partial, bufs.P);
    EDA_LAUNCHED();
    k_kp_split<8><<<dim3(ceil_div(f.ldm, 32), ceil_div(b, 8)), 128, 0, s>>>(m, b, f.K32, bufs.P, bufs.ldq, bufs.Qhi,
                                                                            bufs.Qlo);
    EDA_LAUNCHED();
    {
        ProfScope prof("tc_sweep2", s);
        const int m3 = (f.maps3d && bufs.maps3d) ? 1 : 0;
        k_tc_sweep2<N><<<ceil_div(f.d, TC_M), 128, smem, s>>>(m3 ? f.mapA2_3 : f.mapA2, m3 ? bufs.mapQh3[nb] : bufs.mapQh[nb],
                                                            m3 ? bufs.mapQl3[nb] : bufs.mapQl[nb], f.d, f.ldm, b, X, ldx,
                                                            Y, ldy, status, m3);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

}  // namespace

int tc_factor_make(const double* H, int64_t d, int m, const double* K, __nv_bfloat16* Hcm, __nv_bfloat16* Hrm,
                   float* K32, TcFactor* f, cudaStream_t s) {
    f->d = d;
    f->m = m;
    f->ldh = tc_pad_rows(d);
    f->ldm = tc_pad_cols(m);
    f->Hcm = Hcm;
    f->Hrm = Hrm;
    f->K32 = K32;
    k_to_bf16_cm<<<ceil_div(f->ldh * m, 256), 256, 0, s>>>(d, m, H, d, Hcm, f->ldh);
    EDA_LAUNCHED();
    k_to_bf16_rm<<<ceil_div(d * f->ldm, 256), 256, 0, s>>>(d, m, H, d, Hrm, f->ldm);
    EDA_LAUNCHED();
    k_to_f32<<<ceil_div((int64_t)m * m, 256), 256, 0, s>>>((int64_t)m * m, K, K32);
    EDA_LAUNCHED();
    // sweep 1 reads columns of H (K = d contiguous), sweep 2 reads rows (K = m contiguous)
    EDA_TRY(make_map(&f->mapA1, Hcm, (uint64_t)f->ldh, (uint64_t)m, (uint64_t)f->ldh, TC_M));
    EDA_TRY(make_map(&f->mapA2, Hrm, (uint64_t)f->ldm, (uint64_t)d, (uint64_t)f->ldm, TC_M));
    f->maps3d = make_map3(&f->mapA1_3, Hcm, (uint64_t)f->ldh, (uint64_t)m, (uint64_t)f->ldh, TC_M) &&
                make_map3(&f->mapA2_3, Hrm, (uint64_t)f->ldm, (uint64_t)d, (uint64_t)f->ldm, TC_M);
    return EDA_OK;
}

int tc_buffers_make(int64_t ldh, int ldq, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, __nv_bfloat16* Qhi,
                    __nv_bfloat16* Qlo, float* P, TcBuffers* b) {
    b->Xhi = Xhi;
    b->Xlo = Xlo;
    b->Qhi = Qhi;
    b->Qlo = Qlo;
    b->P = P;
    b->ldh = ldh;
    b->ldq = ldq;
    for (int i = 0; i < 2; ++i) {
        const uint32_t rows = i == 0 ? 16 : 32;
        EDA_TRY(make_map(&b->mapXh[i], Xhi, (uint64_t)ldh, 32, (uint64_t)ldh, rows));
        EDA_TRY(make_map(&b->mapXl[i], Xlo, (uint64_t)ldh, 32, (uint64_t)ldh, rows));
        EDA_TRY(make_map(&b->mapQh[i], Qhi, (uint64_t)ldq, 32, (uint64_t)ldq, rows));
        EDA_TRY(make_map(&b->mapQl[i], Qlo, (uint64_t)ldq, 32, (uint64_t)ldq, rows));
    }
    b->maps3d = true;
    for (int i = 0; i < 2; ++i) {
        const uint32_t rows = i == 0 ? 16 : 32;
        b->maps3d = b->maps3d && make_map3(&b->mapXh3[i], Xhi, (uint64_t)ldh, 32, (uint64_t)ldh, rows) &&
                    make_map3(&b->mapXl3[i], Xlo, (uint64_t)ldh, 32, (uint64_t)ldh, rows) &&
                    make_map3(&b->mapQh3[i], Qhi, (uint64_t)ldq, 32, (uint64_t)ldq, rows) &&
                    make_map3(&b->mapQl3[i], Qlo, (uint64_t)ldq, 32, (uint64_t)ldq, rows);
    }
    return EDA_OK;
}

int exp_apply_tc(const TcFactor& f, const TcBuffers& bufs, const char* tag, int b, const float* X, int64_t ldx,
                 float* Y, int64_t ldy, void* partial, size_t partial_cap, int* status, cudaStream_t s) {
    ProfScope prof(tag, s);
    float* part = static_cast<float*>(partial);
    if (b <= 16) return launch_tc<16>(f, bufs, b, X, ldx, Y, ldy, part, partial_cap, status, s);
    for (int c0 = 0; c0 < b; c0 += 32) {
        const int cb = std::min(32, b - c0);
        EDA_TRY(launch_tc<32>(f, bufs, cb, X + (int64_t)c0 * ldx, ldx, Y + (int64_t)c0 * ldy, ldy, part, partial_cap,
                              status, s));
    }
    return EDA_OK;
}

}  // namespace eda
