// Tensor-core exp-vector product for H stored in bfloat16 (5th-generation tensor cores: tcgen05.mma
// with the accumulator in tensor memory, operands brought in by the Tensor Memory Accelerator).
// Theorem 3.1 gives exp(alpha H H^T) X = X + (H K) (H^T X) with K = alpha phi(alpha H^T H); the
// d x m product H K is formed once per factor (it is itself a sweep-2 product, below), so one
// exp-apply is
//     split     X -> (Xhi, Xlo) bf16 pair          (hi = bf16(x), lo = bf16(x - hi))
//     sweep 1   P = H^T X      M = m (columns of H), N = b, K = d, split over d across CTAs
//     reduce    P = sum of the split partials in FP64, written as a bf16 (hi, lo) pair
//     sweep 2   Y = X + (H K) P   M = d, N = b, K = m, from a row-major bf16 copy of H K
// Every product is bf16 x (bf16 hi + bf16 lo) with FP32 accumulation, so the error is set by the
// bf16 rounding of H and of H K; split sums are added in FP64. Sweep 2 can also write the bf16 pair
// of Y, which is the split step of the next exp-apply in a chain, and Y may alias X.
//
// Each CTA runs a 4-stage shared-memory ring: one thread issues cp.async.bulk.tensor loads of
// 64-element (128-byte) K slices in the 128-byte-swizzled layout (row r of a tile at r * 128 bytes,
// its 16-byte chunk c at chunk c ^ (r mod 8)); one thread issues tcgen05.mma (4 K-steps of 16,
// hi and lo per step, each K-step a 32-byte advance of the descriptor start inside the swizzle
// atom) and commits each stage to the stage's "empty" mbarrier; the four warps read the 128 x N
// FP32 accumulator out of tensor memory at the end. Every wait is bounded (ST_TIMEOUT on give-up).
//
// A factor small enough to stay in the SMs' shared memory has a one-pass form (k_tc_fused.cu):
// exp_apply_tc uses it whenever the handle built it.
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

namespace eda {

using namespace tc;

// ---- tensor maps ------------------------------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
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

// 2-D bf16 tensor: inner extent `inner` (contiguous, a multiple of 64), `outer` rows of stride `ld`
// elements; box of 64 inner elements (128 bytes) x `box_rows` rows, 128-byte swizzle; reads outside
// the extents return zeros.
namespace tc {
int make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_rows) {
    EncodeTiledFn enc = encoder();
    if (!enc) return EDA_ERR_CUDA;
    if (inner % TC_KS || ld % TC_KS || (reinterpret_cast<uintptr_t>(base) & 15)) return EDA_ERR_INVALID_ARG;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {TC_KS, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? EDA_OK : EDA_ERR_CUDA;
}
}  // namespace tc

namespace {

// The ring; every tile starts on a 1024-byte boundary (the swizzle pattern repeats every 8 rows of
// 128 bytes), which holds because the struct is placed on such a boundary and every member size is a
// multiple of 1024.
template <int N>
struct TcRing {
    __nv_bfloat16 A[TC_STAGES][TC_M * TC_KS];   // 16 KB per stage: 128 rows x 128 bytes
    __nv_bfloat16 Bh[TC_STAGES][N * TC_KS];     // N rows x 128 bytes
    __nv_bfloat16 Bl[TC_STAGES][N * TC_KS];
    uint64_t full[TC_STAGES];
    uint64_t empty[TC_STAGES];
    uint64_t done;
    uint32_t tbase;
    int fail;                                    // a role thread gave up on a wait
};
template <int N>
constexpr size_t tc_smem_bytes() {
    return sizeof(TcRing<N>) + 1024;
}
template <int N>
__device__ __forceinline__ TcRing<N>& tc_ring(unsigned char* raw) {
    const uint32_t mis = smem_u32(raw) & 1023u;
    return *reinterpret_cast<TcRing<N>*>(raw + ((1024u - mis) & 1023u));
}

// Main loop shared by both sweeps: K stages [0, nst); A stage s is the contiguous 16 KB tile image at
// Atiles + s * 8192 (already in the swizzled layout), B rows 0..N-1 come from tmBh, tmBl at K
// coordinate k_begin + 64 s. Returns false on timeout.
template <int N>
__device__ bool tc_mainloop(TcRing<N>& sm, const __nv_bfloat16* Atiles, const CUtensorMap* tmBh,
                            const CUtensorMap* tmBl, int k_begin, int nst, uint32_t tmem, int* status) {
    const int tid = threadIdx.x;
    bool ok = true;
    int issued = 0;   // producer: stages whose copies have been requested
    if (tid == 0) {
        // producer: one thread issues all loads (one bulk copy and two tensor boxes per stage). The A
        // tiles (H or H K) do not depend on earlier kernels: the first ring's worth is requested before
        // waiting on the preceding grid, whose outputs (the B pair) are loaded after the wait.
        constexpr uint32_t abytes = TC_M * TC_KS * 2;
        constexpr uint32_t bytes = abytes + 2 * N * TC_KS * 2;
        const int pre = min(nst, TC_STAGES);
        for (int s = 0; s < pre; ++s) {
            mbar_expect_tx(&sm.full[s], bytes);
            bulk_load(sm.A[s], Atiles + (int64_t)s * (TC_M * TC_KS), abytes, &sm.full[s]);
        }
        pdl_wait();
        for (int s = 0; s < pre; ++s) {
            tma_load_2d(sm.Bh[s], tmBh, k_begin + s * TC_KS, 0, &sm.full[s]);
            tma_load_2d(sm.Bl[s], tmBl, k_begin + s * TC_KS, 0, &sm.full[s]);
        }
        issued = pre;
        for (int s = pre; s < nst && ok; ++s) {
            const int slot = s % TC_STAGES;
            ok = mbar_wait(&sm.empty[slot], ((s / TC_STAGES) - 1) & 1, status);
            if (!ok) break;
            mbar_expect_tx(&sm.full[slot], bytes);
            bulk_load(sm.A[slot], Atiles + (int64_t)s * (TC_M * TC_KS), abytes, &sm.full[slot]);
            tma_load_2d(sm.Bh[slot], tmBh, k_begin + s * TC_KS, 0, &sm.full[slot]);
            tma_load_2d(sm.Bl[slot], tmBl, k_begin + s * TC_KS, 0, &sm.full[slot]);
            issued = s + 1;
        }
    } else if (tid == 32) {
        // MMA issuer
        constexpr uint32_t id = idesc_bf16(TC_M, N);
        for (int s = 0; s < nst; ++s) {
            const int slot = s % TC_STAGES;
            if (!mbar_wait(&sm.full[slot], (s / TC_STAGES) & 1, status)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sm.A[slot]), bh = smem_u32(sm.Bh[slot]), bl = smem_u32(sm.Bl[slot]);
            // four independent accumulators (hi/lo x even/odd K-step) so consecutive MMAs do not wait
            // on one another's accumulation; they are added in the epilogue
#pragma unroll
            for (int ks = 0; ks < TC_KS / 16; ++ks) {
                const uint64_t ad = smem_desc_sw128(a0 + ks * 32);
                const uint32_t acc = (s == 0 && ks < 2) ? 0u : 1u;
                const uint32_t col = (uint32_t)((ks & 1) * N);
                mma_bf16(tmem + col, ad, smem_desc_sw128(bh + ks * 32), id, acc);
                mma_bf16(tmem + 2 * N + col, ad, smem_desc_sw128(bl + ks * 32), id, acc);
            }
            mma_commit(&sm.empty[slot]);
        }
        mma_commit(&sm.done);
    }
    // one thread waits for the accumulator; the others rest on the CTA barrier instead of spinning
    __shared__ int s_ok;
    if ((tid == 0 || tid == 32) && !ok) sm.fail = 1;
    if (tid == 0) s_ok = (mbar_wait(&sm.done, 0, status) && ok) ? 1 : 0;
    if (tid == 32 && !ok) atomicOr(status, ST_TIMEOUT);
    __syncthreads();
    const bool fin = s_ok != 0 && sm.fail == 0;
    if (tid == 0 && !fin) {
        // after a give-up, wait (bounded again) for this CTA's copies of the last ring that may still
        // be in flight, so that none lands after the CTA's shared memory is released
        for (int st = max(0, issued - TC_STAGES); st < issued; ++st)
            mbar_wait(&sm.full[st % TC_STAGES], (st / TC_STAGES) & 1, status);
    }
    tc_fence_after();
    pdl_wait();   // returns at once by now (the producer has waited); orders this thread's epilogue
    return fin;
}

template <int N>
__device__ void tc_setup(TcRing<N>& sm) {
    const int tid = threadIdx.x;
    if ((tid >> 5) == 0) {
        tmem_alloc(&sm.tbase, 4 * N);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&sm.full[i], 1);
            mbar_init(&sm.empty[i], 1);
        }
        mbar_init(&sm.done, 1);
        fence_mbar_init();
        sm.fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Columns c0 .. c0+15 of the accumulator of this thread's lane (TMEM lane = row within the tile):
// the sum of the four partial accumulators.
template <int N>
__device__ __forceinline__ void tc_read16(uint32_t tmem, int warp, int c0, float (&v)[16]) {
    uint32_t r[4][16];
    const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + c0;
#pragma unroll
    for (int a = 0; a < 4; ++a) tmem_ld16(base + a * N, r[a]);
    tmem_wait_ld();
#pragma unroll
    for (int c = 0; c < 16; ++c)
        v[c] = (__uint_as_float(r[0][c]) + __uint_as_float(r[1][c])) +
               (__uint_as_float(r[2][c]) + __uint_as_float(r[3][c]));
}

template <int N>
__device__ void tc_teardown(TcRing<N>& sm, uint32_t tmem) {
    tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 4 * N);
}

// ---- sweep 1: partial[split][j][i] = sum_{k in split} H[k, i] X[k, j] ---------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_tc_sweep1(const __nv_bfloat16* __restrict__ A1, int kbs,
                                                    const __grid_constant__ CUtensorMap tmBh,
                                                    const __grid_constant__ CUtensorMap tmBl, int m, int b,
                                                    int rows_per_split, int ldh, float* __restrict__ partial,
                                                    int* status) {
    extern __shared__ unsigned char smraw[];
    TcRing<N>& sm = tc_ring<N>(smraw);
    tc_setup<N>(sm);
    pdl_trigger();
    const uint32_t tmem = sm.tbase;
    const int i0 = blockIdx.x * TC_M;
    const int split = blockIdx.y;
    const int k_begin = split * rows_per_split;
    const int nst = (min(ldh, k_begin + rows_per_split) - k_begin) / TC_KS;
    const __nv_bfloat16* At = A1 + ((int64_t)blockIdx.x * kbs + k_begin / TC_KS) * (TC_M * TC_KS);
    const bool ok = tc_mainloop<N>(sm, At, &tmBh, &tmBl, k_begin, nst, tmem, status);
    const int warp = threadIdx.x >> 5;
    const int i = i0 + 32 * warp + (threadIdx.x & 31);
    float* out = partial + (int64_t)split * m * b;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tc_read16<N>(tmem, warp, c0, v);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const int j = c0 + c;
            if (i < m && j < b) out[(int64_t)j * m + i] = (ok && nst > 0) ? v[c] : 0.f;
        }
    }
    tc_teardown<N>(sm, tmem);
}

// ---- sweep 2 -------------------------------------------------------------------------------------------------
// acc[r, j] = sum_l A[r, l] B[l, j] over the full K range (ldm), A row-major bf16, B a bf16 (hi, lo) pair.
//   MODE 0: Y[r, j] = X[r, j] + acc (Y may alias X); when Yhi is not null also the bf16 pair of Y
//           (column-major, leading dimension ldh), for the next exp-apply's sweep 1.
//   MODE 1: O[r * ldo + j] = bf16(acc) (row-major bf16 store of a 32-column slice of H K).
template <int N, int MODE>
__global__ void __launch_bounds__(128) k_tc_sweep2(const __nv_bfloat16* __restrict__ A2,
                                                    const __grid_constant__ CUtensorMap tmBh,
                                                    const __grid_constant__ CUtensorMap tmBl, int64_t d, int ldm, int b,
                                                    const float* X, int64_t ldx, float* Y, int64_t ldy,
                                                    __nv_bfloat16* Yhi, __nv_bfloat16* Ylo, int64_t ldh,
                                                    __nv_bfloat16* O, int ldo_kbs, int o_col0, int* status) {
    extern __shared__ unsigned char smraw[];
    TcRing<N>& sm = tc_ring<N>(smraw);
    tc_setup<N>(sm);
    pdl_trigger();
    const uint32_t tmem = sm.tbase;
    const int r0 = blockIdx.x * TC_M;
    const int nst = ldm / TC_KS;
    const __nv_bfloat16* At = A2 + (int64_t)blockIdx.x * nst * (TC_M * TC_KS);
    const bool ok = tc_mainloop<N>(sm, At, &tmBh, &tmBl, 0, nst, tmem, status);
    const int warp = threadIdx.x >> 5;
    const int64_t row = r0 + 32 * warp + (threadIdx.x & 31);
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float r[16];
        tc_read16<N>(tmem, warp, c0, r);
        if (MODE == 0) {
            // all loads of this thread's X row segment before any store: Y may alias X, but only
            // element for element within this thread, so the reordering is safe and lets the 16
            // loads overlap instead of paying one round trip each
            float xv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = c0 + c;
                xv[c] = (row < d && j < b) ? X[(int64_t)j * ldx + row] : 0.f;
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const int j = c0 + c;
                if (row < d && j < b) {
                    const float acc = (ok && nst > 0) ? r[c] : 0.f;
                    const float y = xv[c] + acc;
                    Y[(int64_t)j * ldy + row] = y;
                    if (Yhi) {
                        const __nv_bfloat16 hv = __float2bfloat16_rn(y);
                        Yhi[(int64_t)j * ldh + row] = hv;
                        Ylo[(int64_t)j * ldh + row] = __float2bfloat16_rn(y - __bfloat162float(hv));
                    }
                }
            }
        } else if (row < d) {
            // 16 consecutive K columns o_col0 + c0 .. +15 of row `row` in the tiled layout: two
            // 8-element chunks, each one 16-byte store
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = o_col0 + c0 + 8 * h;
                __align__(16) __nv_bfloat162 v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float a0 = (ok && nst > 0) ? r[8 * h + 2 * q] : 0.f;
                    const float a1 = (ok && nst > 0) ? r[8 * h + 2 * q + 1] : 0.f;
                    v[q] = __floats2bfloat162_rn(a0, a1);
                }
                *reinterpret_cast<uint4*>(O + tile_off(row, col, ldo_kbs)) = *reinterpret_cast<const uint4*>(v);
            }
        }
    }
    tc_teardown<N>(sm, tmem);
}

// X (d x b, ld ldx) -> Xhi, Xlo (bf16, column-major ld ldh, rows >= d zero). One thread per 8 rows of
// one column: two 16-byte stores; 16-byte loads when X allows them (vec), else eight scalar loads.
__global__ void k_split_x(int64_t d, int b, const float* __restrict__ X, int64_t ldx, int64_t ldh,
                          __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, int vec) {
    pdl_trigger();   // the next sweep may start its H prefetch; it waits for this grid before reading X
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t groups = ldh / 8;
    if (g >= groups * b) return;
    const int64_t r = (g % groups) * 8;
    const int64_t j = g / groups;
    const float* src = X + j * ldx + r;
    float x[8];
    if (vec && r + 8 <= d) {
        const float4 a = *reinterpret_cast<const float4*>(src);
        const float4 c = *reinterpret_cast<const float4*>(src + 4);
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        x[4] = c.x; x[5] = c.y; x[6] = c.z; x[7] = c.w;
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = (r + u < d) ? src[u] : 0.f;
    }
    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        hi[u] = __float2bfloat16_rn(x[u]);
        lo[u] = __float2bfloat16_rn(x[u] - __bfloat162float(hi[u]));
    }
    *reinterpret_cast<uint4*>(Xhi + j * ldh + r) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(Xlo + j * ldh + r) = *reinterpret_cast<const uint4*>(lo);
}

// P[i, j] = sum_s partial[s][j][i], written as the bf16 pair (Phi, Plo), column-major with leading
// dimension ldq; rows m..ldq-1 are zero. CTA = 32 rows (lanes) of one column j (blockIdx.y); warp w
// sums the split range [w q, (w + 1) q) in order, then warp 0 adds the eight warp sums in order: a
// fixed summation order independent of timing. Single precision: the partials are FP32 tensor-core
// accumulators and the product is bf16-accurate, while FP64 adds cost ~30x more issue slots here.
__global__ void __launch_bounds__(256) k_reduce_split(int m, int b, int splits, const float* __restrict__ partial,
                                                      int ldq, __nv_bfloat16* Phi, __nv_bfloat16* Plo) {
    __shared__ float part[8][33];
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    const int j = blockIdx.y;
    const int q = (splits + 7) / 8;
    const int s0 = w * q, s1 = min(splits, s0 + q);
    float acc = 0.f;
    if (i < m) {
        const int64_t stride = (int64_t)m * b;
        const float* src = partial + (int64_t)j * m + i;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (s0 + u < s1) ? src[(s0 + u) * stride] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
        for (int s = s0 + 8; s < s1; ++s) acc += src[s * stride];
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w == 0 && i < ldq) {
        float t = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) t += part[u][lane];
        const float p = (i < m) ? t : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(p);
        Phi[(int64_t)j * ldq + i] = h;
        Plo[(int64_t)j * ldq + i] = __float2bfloat16_rn(p - __bfloat162float(h));
    }
}

// Columns c0 .. c0+31 of the symmetric FP64 K (m x m, ld m) as 32 rows of a bf16 pair with
// leading dimension ldq (entry (l, j) = K[l, c0 + j]); entries outside K are zero.
__global__ void k_kslice_split(int m, int c0, const double* __restrict__ K, int ldq, __nv_bfloat16* Khi,
                               __nv_bfloat16* Klo) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ldq * 32) return;
    const int l = (int)(e % ldq);
    const int c = c0 + (int)(e / ldq);
    const float v = (l < m && c < m) ? (float)K[(int64_t)c * m + l] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Khi[e] = h;
    Klo[e] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// bf16 tiled image of an FP64 factor H (d x m, column-major, ld d). by_column = 1: tile rows are the
// columns of H and K runs along d (sweep 1 operand); by_column = 0: tile rows are the rows of H and
// K runs along m (sweep 2 operand, and the build-time H of H K). Entries outside H are zero.
__global__ void k_tile_bf16(int64_t d, int m, const double* __restrict__ H, int by_column, int kbs, int64_t total,
                            __nv_bfloat16* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t tile = e >> 13;
    const int within = (int)(e & 8191);
    const int rr = within >> 6, pc = (within >> 3) & 7, el = within & 7;
    const int c = pc ^ (rr & 7);
    const int64_t r = (tile / kbs) * TC_M + rr;
    const int64_t kk = (tile % kbs) * TC_KS + c * 8 + el;
    double v = 0.0;
    if (by_column) {
        if (r < m && kk < d) v = H[r * d + kk];
    } else {
        if (r < d && kk < m) v = H[kk * d + r];
    }
    out[e] = __float2bfloat16_rn((float)v);
}

// Launch with programmatic stream serialisation: the kernel may start while the preceding kernel of
// the stream drains; it orders its dependent reads with griddepcontrol.wait.
template <class... KArgs, class... Args>
int launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    EDA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
    launch_counter()++;
    return EDA_OK;
}

template <int N, int MODE>
int set_smem_attr() {
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (!done) {
        EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep2<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_smem_bytes<N>()));
        if (MODE == 0)
            EDA_CUDA_TRY(cudaFuncSetAttribute(k_tc_sweep1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)tc_smem_bytes<N>()));
        done = true;
    }
    return EDA_OK;
}

template <int N>
int launch_tc(const TcFactor& f, const TcBuffers& bufs, int b, const float* X, int64_t ldx, float* Y, int64_t ldy,
              bool x_split_ready, bool emit_split, int* status, cudaStream_t s) {
    float* partial = bufs.partial;
    const size_t partial_cap = bufs.partial_cap;
    EDA_TRY((set_smem_attr<N, 0>()));
    constexpr size_t smem = tc_smem_bytes<N>();
    const int m = f.m;
    const int nb = N == 16 ? 0 : 1;
    if (!x_split_ready) {
        const int vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0 && ldx % 4 == 0) ? 1 : 0;
        k_split_x<<<ceil_div(f.ldh / 8 * b, 256), 256, 0, s>>>(f.d, b, X, ldx, f.ldh, bufs.Xhi, bufs.Xlo, vec);
        EDA_LAUNCHED();
    }
    // sweep 1 over split ranges of whole stages
    const int tiles = ceil_div(m, TC_M);
    const int kst = (int)(f.ldh / TC_KS);
    int splits = std::max(1, std::min(kst, ceil_div(2 * sm_count(), tiles)));
    while (splits > 1 && (size_t)splits * m * b > partial_cap) --splits;
    if ((size_t)splits * m * b > partial_cap) return EDA_ERR_INVALID_ARG;
    const int rows = ceil_div(kst, splits) * TC_KS;
    splits = ceil_div(f.ldh, rows);
    EDA_TRY(launch_pdl(k_tc_sweep1<N>, dim3(tiles, splits), dim3(128), smem, s, f.A1, (int)(f.ldh / TC_KS),
                       bufs.mapXh[nb], bufs.mapXl[nb], m, b, rows, (int)f.ldh, partial, status));
    EDA_TRY(launch_pdl(k_reduce_split, dim3(ceil_div(bufs.ldq, 32), b), dim3(256), 0, s, m, b, splits,
                       (const float*)partial, bufs.ldq, bufs.Qhi, bufs.Qlo));
    EDA_TRY(launch_pdl(k_tc_sweep2<N, 0>, dim3(ceil_div(f.d, TC_M)), dim3(128), smem, s, f.A2, bufs.mapQh[nb],
                       bufs.mapQl[nb], f.d, f.ldm, b, X, ldx, Y, ldy, emit_split ? bufs.Xhi : nullptr,
                       emit_split ? bufs.Xlo : nullptr, f.ldh, (__nv_bfloat16*)nullptr, 0, 0, status));
    return EDA_OK;
}

}  // namespace

int64_t tc_tiles_sweep1(int64_t d, int m) { return (int64_t)ceil_div(m, TC_M) * TC_M * tc_pad_rows(d); }
int64_t tc_tiles_sweep2(int64_t d, int m) { return (int64_t)ceil_div(d, TC_M) * TC_M * tc_pad_cols(m); }

int tc_factor_make(const double* H, int64_t d, int m, const double* K, __nv_bfloat16* A1, __nv_bfloat16* A2,
                   TcFactor* f, int* status, cudaStream_t s) {
    f->d = d;
    f->m = m;
    f->ldh = tc_pad_rows(d);
    f->ldm = tc_pad_cols(m);
    f->A1 = A1;
    f->A2 = A2;
    const int ldm = f->ldm;
    const int kbs1 = (int)(f->ldh / TC_KS), kbs2 = ldm / TC_KS;
    {
        const int64_t tot = tc_tiles_sweep1(d, m);
        k_tile_bf16<<<ceil_div(tot, 256), 256, 0, s>>>(d, m, H, 1, kbs1, tot, A1);
        EDA_LAUNCHED();
    }
    // H K (tiled like the sweep-2 operand) as sweep-2 products: A = tiled bf16(H) by rows, B = 32-column
    // slices of K as bf16 pairs. Temporaries are freed before returning (the stream is synchronised).
    const int64_t tot2 = tc_tiles_sweep2(d, m);
    __nv_bfloat16* Hr = nullptr;
    const size_t hbytes = ((size_t)tot2 * 2 + 255) / 256 * 256;
    const size_t kbytes = (size_t)ldm * 32 * 2;
    if (cudaMalloc(&Hr, hbytes + 2 * kbytes) != cudaSuccess) {
        cudaGetLastError();
        return EDA_ERR_OOM;
    }
    __nv_bfloat16* Khi = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(Hr) + hbytes);
    __nv_bfloat16* Klo = Khi + (size_t)ldm * 32;
    int rc = EDA_OK;
    do {
        k_tile_bf16<<<ceil_div(tot2, 256), 256, 0, s>>>(d, m, H, 0, kbs2, tot2, Hr);
        launch_counter()++;
        if (cudaPeekAtLastError() != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
        CUtensorMap mKh, mKl;
        if ((rc = make_map(&mKh, Khi, (uint64_t)ldm, 32, (uint64_t)ldm, 32)) != EDA_OK) break;
        if ((rc = make_map(&mKl, Klo, (uint64_t)ldm, 32, (uint64_t)ldm, 32)) != EDA_OK) break;
        if ((rc = set_smem_attr<32, 1>()) != EDA_OK) break;
        for (int c0 = 0; c0 < ldm && rc == EDA_OK; c0 += 32) {
            k_kslice_split<<<ceil_div((int64_t)ldm * 32, 256), 256, 0, s>>>(m, c0, K, ldm, Khi, Klo);
            k_tc_sweep2<32, 1><<<ceil_div(d, TC_M), 128, tc_smem_bytes<32>(), s>>>(
                Hr, mKh, mKl, d, ldm, 32, nullptr, 0, nullptr, 0, nullptr, nullptr, 0, A2, kbs2, c0, status);
            launch_counter() += 2;
            if (cudaPeekAtLastError() != cudaSuccess) rc = EDA_ERR_CUDA;
        }
        if (rc == EDA_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = EDA_ERR_CUDA;
    } while (false);
    if (rc != EDA_OK) cudaStreamSynchronize(s);
    cudaFree(Hr);
    return rc;
}

size_t tc_partial_floats(int m_max) { return (size_t)(2 * sm_count() + ceil_div(m_max, TC_M)) * TC_M * 32; }

int tc_buffers_make(int64_t ldh, int ldq, __nv_bfloat16* Xhi, __nv_bfloat16* Xlo, __nv_bfloat16* Qhi,
                    __nv_bfloat16* Qlo, float* partial, size_t partial_cap, TcBuffers* b) {
    b->partial = partial;
    b->partial_cap = partial_cap;
    b->Xhi = Xhi;
    b->Xlo = Xlo;
    b->Qhi = Qhi;
    b->Qlo = Qlo;
    b->ldh = ldh;
    b->ldq = ldq;
    for (int i = 0; i < 2; ++i) {
        const uint32_t rows = i == 0 ? 16 : 32;
        EDA_TRY(make_map(&b->mapXh[i], Xhi, (uint64_t)ldh, 32, (uint64_t)ldh, rows));
        EDA_TRY(make_map(&b->mapXl[i], Xlo, (uint64_t)ldh, 32, (uint64_t)ldh, rows));
        EDA_TRY(make_map(&b->mapQh[i], Qhi, (uint64_t)ldq, 32, (uint64_t)ldq, rows));
        EDA_TRY(make_map(&b->mapQl[i], Qlo, (uint64_t)ldq, 32, (uint64_t)ldq, rows));
    }
    return EDA_OK;
}

int exp_apply_tc(const TcFactor& f, const TcBuffers& bufs, const char* tag, int b, const float* X, int64_t ldx,
                 float* Y, int64_t ldy, int flags, int* status, cudaStream_t s) {
    if (f.F && bufs.fpartial) {
        // one pass: B read once from HBM (its bf16 image), X read twice, Y written once
        ProfScope prof(tag, s, 4.0 * f.d * f.m * b, 2.0 * f.d * f.m + 3.0 * 4.0 * f.d * b);
        return exp_apply_tc_fused(f, bufs, b, X, ldx, Y, ldy, status, s);
    }
    ProfScope prof(tag, s, 4.0 * f.d * f.m * b, 2.0 * 2.0 * f.d * f.m + 3.0 * 4.0 * f.d * b);
    // the split pair lives in one 32-column staging buffer: chaining needs a single slice
    const bool chain = b <= 32;
    const bool ready = chain && (flags & TC_X_SPLIT_READY);
    const bool emit = chain && (flags & TC_EMIT_SPLIT);
    if (b <= 16) return launch_tc<16>(f, bufs, b, X, ldx, Y, ldy, ready, emit, status, s);
    for (int c0 = 0; c0 < b; c0 += 32) {
        const int cb = std::min(32, b - c0);
        EDA_TRY(launch_tc<32>(f, bufs, cb, X + (int64_t)c0 * ldx, ldx, Y + (int64_t)c0 * ldy, ldy, ready, emit,
                              status, s));
    }
    return EDA_OK;
}

}  // namespace eda
