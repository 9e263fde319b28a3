// One-pass exp-vector product on the tensor cores with the factor resident in shared memory.
//
// Theorem 3.1: exp(alpha H H^T) X = X + H K (H^T X) with K = alpha phi(alpha H^T H). K is definite
// (phi > 0; alpha K > 0), so sigma K = R^T R (Cholesky, sigma = sign(alpha)) and with B = H R^T (d x m)
//     exp(alpha H H^T) X = X + sigma B (B^T X):
// both sweeps read the same matrix B. When bf16(B) fits in the shared memory of the GPU's SMs
// (128 rows of B per CTA, m <= 768: 192 KB), one persistent launch does the whole product, reading B
// from HBM once instead of twice and replacing four launches:
//     load     CTA c copies rows [128 c, 128 c + 128) of bf16(B) into shared memory (one bulk copy per
//              128-column band, each with its own mbarrier) and splits its rows of X into bf16 hi + lo
//              pairs while the copies are in flight
//     sweep 1  P_c = B_c^T X_c (tcgen05.mma, M = 128 columns of B per band, K = 128 rows of the chunk,
//              N = 2 b: the hi and lo rows of X stacked into one operand), written as FP32 partials
//     barrier  bounded grid barrier (cooperative launch: every CTA is resident)
//     reduce   P = sum_c P_c, each CTA a slice of the m x b entries, the partials added in a fixed
//              order (eight ranges of c, each in increasing c, then the eight range sums in turn),
//              independent of timing, written as a bf16 (hi, lo) pair
//     barrier
//     sweep 2  Y_c = X_c + sigma B_c P (M = 128 rows of the chunk, K = m): the same shared-memory
//              image read as an MN-major operand (its 128-byte rows hold 64 consecutive rows of B for
//              one column), P streamed by TMA through a ring of 8 (b <= 16) or 4 slices
// The tile image is the 128-byte-swizzled layout of the sweep-1 operand (row = a column of B, 64 rows
// of B per 128-byte row; 16-byte chunk c of image row r at chunk c ^ (r mod 8)). As a K-major operand
// (sweep 1) its core matrices are 8 columns x 16 bytes with 8-row groups 1024 bytes apart; as an
// MN-major operand (sweep 2) a swizzle atom is 64 rows of B (one 128-byte row) x 8 columns, atoms along
// the rows of B 16 KB apart (the next 64-row tile), 8-column groups 1024 bytes apart.
#include "grid_bar.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace eda {

using namespace tc;

namespace {

constexpr int FU_THREADS = 256;   // 8 warps: warps 0-3 also read the accumulators (one 32-lane quarter each)
constexpr int FU_ROWS = 128;      // rows of B and X per CTA
// sweep-2 ring depth: every P slice of a 768-column factor in flight at once would need 12; the shared memory
// left beside the 192 KB image holds 8 slices of a 16-column P pair, 4 of a 32-column one
template <int N>
__host__ __device__ constexpr int fu_ring() {
    return N == 16 ? 8 : 4;
}
constexpr int FU_RED = 128;       // entries per reduction chunk (4 per lane)

__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// MN-major descriptor of the resident image (128-byte swizzle): atoms of 64 rows of B x 8 columns, the
// next 64 rows at +16 KB (leading-dimension offset), the next 8 columns at +1024 B (stride offset).
__device__ __forceinline__ uint64_t smem_desc_sw128_mn(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16384 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

struct FusedArgs {
    const __nv_bfloat16* img;   // tiled bf16(B): band bd, 64-row slice ks at ((bd * kbs + ks) << 13), kbs = 2 G
    const float* X;
    float* Y;
    float* partial;             // G x m x b
    __nv_bfloat16 *Phi, *Plo;   // b x ldq (column j of P at j * ldq)
    GridBarWords bar;           // two barriers per launch
    int* status;
    int64_t d, ldx, ldy;
    int m, b, bands, ldq;
    float sigma;
};

template <int N>
__global__ void __launch_bounds__(FU_THREADS, 1) k_tc_apply_fused(const __grid_constant__ CUtensorMap tmPh,
                                                                 const __grid_constant__ CUtensorMap tmPl,
                                                                 const FusedArgs a) {
    extern __shared__ unsigned char smraw[];
    const uint32_t mis = smem_u32(smraw) & 1023u;
    unsigned char* base = smraw + ((1024u - mis) & 1023u);
    constexpr uint32_t TILE = TC_M * TC_KS * 2;          // 16 KB
    constexpr uint32_t BROW = N * TC_KS * 2;             // one B-operand slice (N rows x 128 B)
    constexpr int FU_RING = fu_ring<N>();
    const int bands = a.bands;
    __nv_bfloat16* img = reinterpret_cast<__nv_bfloat16*>(base);
    unsigned char* un = base + (size_t)bands * 2 * TILE;   // union: X split | reduction scratch | P ring
    // X split: slice ks holds 2 N operand rows, hi of column j in row j, lo in row N + j
    __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(un);              // [2][2 N * 64]
    float* red = reinterpret_cast<float*>(un);                             // [8][FU_RED]
    // P ring: slot s holds the hi box (N rows) then the lo box (N rows), one 2 N-row operand
    __nv_bfloat16* pr = reinterpret_cast<__nv_bfloat16*>(un);              // [FU_RING][2 N * 64]
    uint64_t* bars = reinterpret_cast<uint64_t*>(un + 2 * FU_RING * BROW);
    uint64_t* band_full = bars;                 // [6]
    uint64_t* ring_full = bars + 6;             // [FU_RING]
    uint64_t* ring_empty = bars + 6 + FU_RING;  // [FU_RING]
    uint64_t* done1 = bars + 6 + 2 * FU_RING;
    uint64_t* done2 = done1 + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done2 + 1);
    int* fail = reinterpret_cast<int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int c = blockIdx.x;
    const int64_t r0 = (int64_t)c * FU_ROWS;
    const unsigned gbase = gb_base(a.bar);
    constexpr uint32_t TCOLS = (N == 32) ? 512u : 256u;   // >= 2 N per band (6 bands) and 4 N

    // ---- set-up: tensor memory, barriers; the image copies go out first ----
    if (warp == 0) {
        tmem_alloc(tslot, TCOLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < 6 + 2 * FU_RING + 2; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        *fail = 0;
        for (int bd = 0; bd < bands; ++bd) {
            mbar_expect_tx(&band_full[bd], 2 * TILE);
            bulk_load(img + (size_t)bd * 2 * (TILE / 2), a.img + (((int64_t)bd * 2 * gridDim.x + 2 * c) << 13), 2 * TILE,
                      &band_full[bd]);
        }
    }
    // X rows of this chunk as bf16 hi/lo in the 128-byte-swizzled K-major layout of the sweep-1 B operand:
    // slice ks holds rows 64 ks .. 64 ks + 63 of the chunk, image row j = column j of X
    for (int it = tid; it < N * 16; it += FU_THREADS) {
        const int j = it / 16, q = it % 16;          // column, 8-row group of the chunk
        const int ks = q >> 3, ch = q & 7;
        float v[8];
        const int64_t rr = r0 + 8 * q;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (j < a.b && rr + u < a.d) ? a.X[(int64_t)j * a.ldx + rr + u] : 0.f;
        __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            hi[u] = __float2bfloat16_rn(v[u]);
            lo[u] = __float2bfloat16_rn(v[u] - __bfloat162float(hi[u]));
        }
        const size_t off = (size_t)ks * (2 * N * TC_KS) + (size_t)j * TC_KS + (size_t)((ch ^ (j & 7)) * 8);
        *reinterpret_cast<uint4*>(xs + off) = *reinterpret_cast<const uint4*>(hi);
        *reinterpret_cast<uint4*>(xs + off + (size_t)N * TC_KS) = *reinterpret_cast<const uint4*>(lo);
    }
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // ---- sweep 1: P_c = B_c^T X_c, band bd into accumulator columns [2 N bd, 2 N bd + 2 N): the first N
    // against the hi rows of X, the next N against the lo rows (one MMA of width 2 N reads the band once)
    if (tid == 32) {
        constexpr uint32_t id = idesc_bf16(TC_M, 2 * N);
        bool ok = true;
        for (int bd = 0; bd < bands && ok; ++bd) {
            if (!mbar_wait(&band_full[bd], 0, a.status)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t acc_b = tmem + (uint32_t)(2 * N * bd);
            for (int ks = 0; ks < 2; ++ks) {
                const uint32_t a0 = smem_u32(img + ((size_t)bd * 2 + ks) * (TILE / 2));
                const uint32_t b0 = smem_u32(xs + (size_t)ks * (2 * N * TC_KS));
#pragma unroll
                for (int kk = 0; kk < TC_KS / 16; ++kk) {
                    const uint32_t acc = (ks == 0 && kk == 0) ? 0u : 1u;
                    mma_bf16(acc_b, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), id, acc);
                }
            }
        }
        if (!ok) *fail = 1;
        mma_commit(done1);
    }
    __syncthreads();
    bool good = *fail == 0;
    if (tid == 0 && !mbar_wait(done1, 0, a.status)) *fail = 1;
    if (tid == 0 && !good) {
        // a band copy did not arrive in time: wait (bounded again) for the copies still in flight
        for (int bd = 0; bd < bands; ++bd) mbar_wait(&band_full[bd], 0, a.status);
    }
    __syncthreads();
    good = *fail == 0;
    tc_fence_after();
    // epilogue 1: warps 0-3 read their 32 lanes (columns of B) of every band, hi + lo, into the partials
    if (warp < 4) {
        float* out = a.partial + (int64_t)c * a.m * a.b;
        for (int bd = 0; bd < bands; ++bd) {
            const int i = bd * TC_M + 32 * warp + lane;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t rh[16], rl[16];
                const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(2 * N * bd + c0);
                tmem_ld16(tb, rh);
                tmem_ld16(tb + N, rl);
                tmem_wait_ld();
                if (i < a.m) {
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int j = c0 + u;
                        if (j < a.b) out[(int64_t)j * a.m + i] = good ? __uint_as_float(rh[u]) + __uint_as_float(rl[u]) : 0.f;
                    }
                }
            }
        }
    }
    tc_fence_before();
    gb_sync(a.bar, gbase, 1, a.status);

    // ---- reduce: entries e = j m + i of this CTA's slice, P[e] = sum over c of partial[c][e] (fixed order) ----
    {
        const int64_t E = (int64_t)a.m * a.b;
        const int G = gridDim.x;
        const int64_t e0 = E * c / G, e1 = E * (c + 1) / G;
        const int cw0 = (int)((int64_t)G * warp / 8), cw1 = (int)((int64_t)G * (warp + 1) / 8);
        for (int64_t ch0 = e0; ch0 < e1; ch0 += FU_RED) {
            float s[4] = {0.f, 0.f, 0.f, 0.f};
            // sixteen partials at a time: all 64 loads of a round are issued before any is added
            for (int cb = cw0; cb < cw1; cb += 16) {
                float v[16][4];
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const float* src = a.partial + (int64_t)(cb + u) * E;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int64_t e = ch0 + lane + 32 * q;
                        v[u][q] = (cb + u < cw1 && e < e1) ? __ldcg(src + e) : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 16; ++u)
#pragma unroll
                    for (int q = 0; q < 4; ++q) s[q] += v[u][q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) red[warp * FU_RED + lane + 32 * q] = s[q];
            __syncthreads();
            if (tid < FU_RED) {
                const int64_t e = ch0 + tid;
                if (e < e1) {
                    float t = 0.f;
#pragma unroll
                    for (int w = 0; w < 8; ++w) t += red[w * FU_RED + tid];
                    const int j = (int)(e / a.m), i = (int)(e % a.m);
                    const __nv_bfloat16 hv = __float2bfloat16_rn(t);
                    a.Phi[(int64_t)j * a.ldq + i] = hv;
                    a.Plo[(int64_t)j * a.ldq + i] = __float2bfloat16_rn(t - __bfloat162float(hv));
                }
            }
            __syncthreads();
        }
        // rows m .. (m rounded up to 64) of P read as zeros by sweep 2
        const int mp = (a.m + 63) / 64 * 64;
        if (c == 0)
            for (int e = tid; e < (mp - a.m) * a.b; e += FU_THREADS) {
                const int j = e / (mp - a.m), i = a.m + e % (mp - a.m);
                a.Phi[(int64_t)j * a.ldq + i] = __float2bfloat16_rn(0.f);
                a.Plo[(int64_t)j * a.ldq + i] = __float2bfloat16_rn(0.f);
            }
    }
    fence_proxy_async_global();
    fence_proxy_async_shared();
    gb_sync(a.bar, gbase, 2, a.status);
    gb_finish(a.bar, gbase, 2);

    // ---- sweep 2: Y_c = X_c + sigma B_c P, K = m in stages of 64 ----
    const int nst = (a.m + 63) / 64;
    bool ok2 = true;
    int issued = 0;
    if (tid == 0) {
        fence_proxy_async_global();
        constexpr uint32_t bytes = 2 * BROW;
        const int pre = min(nst, FU_RING);
        for (int s = 0; s < pre; ++s) {
            mbar_expect_tx(&ring_full[s], bytes);
            tma_load_2d(pr + (size_t)s * (2 * N * TC_KS), &tmPh, s * TC_KS, 0, &ring_full[s]);
            tma_load_2d(pr + (size_t)s * (2 * N * TC_KS) + N * TC_KS, &tmPl, s * TC_KS, 0, &ring_full[s]);
        }
        issued = pre;
        for (int s = pre; s < nst && ok2; ++s) {
            const int slot = s % FU_RING;
            ok2 = mbar_wait(&ring_empty[slot], ((s / FU_RING) - 1) & 1, a.status);
            if (!ok2) break;
            mbar_expect_tx(&ring_full[slot], bytes);
            tma_load_2d(pr + (size_t)slot * (2 * N * TC_KS), &tmPh, s * TC_KS, 0, &ring_full[slot]);
            tma_load_2d(pr + (size_t)slot * (2 * N * TC_KS) + N * TC_KS, &tmPl, s * TC_KS, 0, &ring_full[slot]);
            issued = s + 1;
        }
    } else if (tid == 32) {
        // MN-major A (the resident image) against the stacked (hi, lo) operand of width 2 N, two accumulators
        // (even, odd K-step) of 2 N columns each
        constexpr uint32_t id = idesc_bf16(TC_M, 2 * N) | (1u << 15);
        const uint32_t ib = smem_u32(img);
        for (int s = 0; s < nst; ++s) {
            const int slot = s % FU_RING;
            if (!mbar_wait(&ring_full[slot], (s / FU_RING) & 1, a.status)) {
                ok2 = false;
                break;
            }
            tc_fence_after();
            const uint32_t b0 = smem_u32(pr + (size_t)slot * (2 * N * TC_KS));
#pragma unroll
            for (int kk = 0; kk < TC_KS / 16; ++kk) {
                const int i0 = s * TC_KS + kk * 16;           // first column of B of this K-step
                const uint32_t aaddr = ib + (uint32_t)(i0 >> 7) * (2 * TILE) + (uint32_t)(i0 & 127) * 128u;
                const uint32_t acc = (s == 0 && kk < 2) ? 0u : 1u;
                const uint32_t col = (uint32_t)((kk & 1) * 2 * N);
                mma_bf16(tmem + col, smem_desc_sw128_mn(aaddr), smem_desc_sw128(b0 + kk * 32), id, acc);
            }
            mma_commit(&ring_empty[slot]);
        }
        mma_commit(done2);
    }
    if ((tid == 0 || tid == 32) && !ok2) *fail = 1;
    __syncthreads();
    if (tid == 0) {
        if (!mbar_wait(done2, 0, a.status)) *fail = 1;
        if (*fail) {
            // after a give-up, the ring copies still in flight land before the shared memory is released
            for (int st = max(0, issued - FU_RING); st < issued; ++st)
                mbar_wait(&ring_full[st % FU_RING], (st / FU_RING) & 1, a.status);
        }
    }
    __syncthreads();
    good = *fail == 0;
    tc_fence_after();
    // epilogue 2: warps 0-3, row r0 + 32 w + lane of Y
    if (warp < 4) {
        const int64_t row = r0 + 32 * warp + lane;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t q[4][16];
            const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
#pragma unroll
            for (int u = 0; u < 4; ++u) tmem_ld16(tb + u * N, q[u]);
            tmem_wait_ld();
            if (row < a.d) {
                float xv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) xv[u] = (c0 + u < a.b) ? a.X[(int64_t)(c0 + u) * a.ldx + row] : 0.f;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const int j = c0 + u;
                    if (j < a.b) {
                        const float acc = (__uint_as_float(q[0][u]) + __uint_as_float(q[1][u])) +
                                          (__uint_as_float(q[2][u]) + __uint_as_float(q[3][u]));
                        a.Y[(int64_t)j * a.ldy + row] = xv[u] + (good ? a.sigma * acc : 0.f);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

template <int N>
size_t fused_smem_bytes(int bands) {
    constexpr size_t BROW = (size_t)N * TC_KS * 2;
    constexpr int FU_RING = fu_ring<N>();
    return (size_t)bands * 2 * TC_M * TC_KS * 2 + 2 * FU_RING * BROW + (6 + 2 * FU_RING + 2) * 8 + 16 + 1024;
}

// B (d x m, ld d) = H R^T for sigma K = R^T R; R^T is passed as a dense lower-triangular m x m matrix.
__global__ void k_upper_transpose(int m, const double* __restrict__ R, double* __restrict__ RT) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);   // RT[i, j] = R[j, i] (upper R: zero when j > i)
    RT[e] = (j <= i) ? R[(int64_t)i * m + j] : 0.0;
}

__global__ void k_scaled_copy(int64_t n, double sc, const double* __restrict__ A, double* __restrict__ B) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) B[e] = sc * A[e];
}

// bf16 tiled image of B (d x m, ld d): tile (band, slice) holds columns 128 band .. + 127 (image rows) and rows
// 64 slice .. + 63 of B (K), kbs slices per band, zero outside B.
__global__ void k_tile_fused(int64_t d, int m, const double* __restrict__ B, int kbs, int64_t total,
                             __nv_bfloat16* __restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t tile = e >> 13;
    const int within = (int)(e & 8191);
    const int rr = within >> 6, pc = (within >> 3) & 7, el = within & 7;
    const int ch = pc ^ (rr & 7);
    const int64_t col = (tile / kbs) * TC_M + rr;
    const int64_t row = (tile % kbs) * TC_KS + ch * 8 + el;
    const double v = (col < m && row < d) ? B[col * d + row] : 0.0;
    out[e] = __float2bfloat16_rn((float)v);
}

std::once_flag g_fused_attr_once;
int g_fused_attr_rc = EDA_OK;

int fused_set_attrs() {
    std::call_once(g_fused_attr_once, [] {
        if (cudaFuncSetAttribute(k_tc_apply_fused<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<16>(6)) != cudaSuccess ||
            cudaFuncSetAttribute(k_tc_apply_fused<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fused_smem_bytes<32>(6)) != cudaSuccess) {
            cudaGetLastError();
            g_fused_attr_rc = EDA_ERR_CUDA;
        }
    });
    return g_fused_attr_rc;
}

template <int N>
int launch_fused(const TcFactor& f, const TcBuffers& bufs, int b, const float* X, int64_t ldx, float* Y, int64_t ldy,
                 int* status, cudaStream_t s) {
    EDA_TRY(fused_set_attrs());
    const int nb = N == 16 ? 0 : 1;
    FusedArgs a{};
    a.img = f.F;
    a.X = X;
    a.Y = Y;
    a.partial = bufs.fpartial;
    a.Phi = bufs.Qhi;
    a.Plo = bufs.Qlo;
    a.bar = GridBarWords{bufs.fbar, bufs.fbar + 32, bufs.fspin};
    a.status = status;
    a.d = f.d;
    a.ldx = ldx;
    a.ldy = ldy;
    a.m = f.m;
    a.b = b;
    a.bands = (f.m + TC_M - 1) / TC_M;
    a.ldq = bufs.ldq;
    a.sigma = f.fsign;
    const int G = f.fgrid;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(FU_THREADS);
    cfg.dynamicSmemBytes = fused_smem_bytes<N>(a.bands);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    EDA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_apply_fused<N>, bufs.mapQh[nb], bufs.mapQl[nb], a));
    launch_counter()++;
    return EDA_OK;
}

}  // namespace

int tc_fused_grid(int64_t d, int m) {
    if (m < 1 || m > 6 * TC_M || d < 1) return 0;
    const int G = ceil_div(d, FU_ROWS);
    int dev = 0, nsm = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || fused_set_attrs() != EDA_OK) {
        cudaGetLastError();
        return 0;
    }
    const int bands = ceil_div(m, TC_M);
    // the larger instance (N = 32) sets the residency: one CTA per SM, every CTA resident at once
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tc_apply_fused<32>, FU_THREADS,
                                                      fused_smem_bytes<32>(bands)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (per >= 1 && G <= per * nsm) ? G : 0;
}

int64_t tc_fused_elems(int64_t d, int m) { return (int64_t)ceil_div(m, TC_M) * TC_M * (int64_t)ceil_div(d, FU_ROWS) * FU_ROWS; }

size_t tc_fused_partial_floats(int64_t d, int m_max) { return (size_t)ceil_div(d, FU_ROWS) * m_max * 32; }

int tc_fused_make(const double* H, int64_t d, int m, const double* K, double alpha, __nv_bfloat16* img, TcFactor* f,
                  int* status, cudaStream_t s) {
    const int G = tc_fused_grid(d, m);
    if (G == 0 || alpha == 0.0) return EDA_ERR_INVALID_ARG;
    const double sigma = alpha > 0.0 ? 1.0 : -1.0;
    // sigma K = R^T R, B = H R^T (FP64), then the bf16 tiled image; temporaries freed before returning
    const size_t mm = (size_t)m * m;
    const size_t pcap = std::max<size_t>(mm, 1u << 16);
    double* tmp = nullptr;
    const size_t bytes = (3 * mm + (size_t)d * m + chol_inv_blocked_doubles(m) + pcap) * 8 + 1024;
    if (cudaMalloc(&tmp, bytes) != cudaSuccess) {
        cudaGetLastError();
        return EDA_ERR_OOM;
    }
    double* R = tmp;
    double* Ri = R + mm;
    double* RT = Ri + mm;
    double* Bf = RT + mm;
    double* work = Bf + (size_t)d * m;
    double* part = work + chol_inv_blocked_doubles(m);
    int rc = EDA_OK;
    do {
        k_scaled_copy<<<ceil_div((int64_t)mm, 256), 256, 0, s>>>((int64_t)mm, sigma, K, R);
        launch_counter()++;
        if ((rc = chol_inv_auto(m, R, m, Ri, 1e-30, status, work, part, pcap, s)) != EDA_OK) break;
        k_upper_transpose<<<ceil_div((int64_t)mm, 256), 256, 0, s>>>(m, R, RT);
        launch_counter()++;
        if ((rc = gemm_nn_f64(d, m, m, 1.0, H, d, RT, m, 0.0, nullptr, 0, Bf, d, s)) != EDA_OK) break;
        const int kbs = 2 * G;
        const int64_t total = (int64_t)ceil_div(m, TC_M) * kbs * (TC_M * TC_KS);
        k_tile_fused<<<ceil_div(total, 256), 256, 0, s>>>(d, m, Bf, kbs, total, img);
        launch_counter()++;
        if (cudaPeekAtLastError() != cudaSuccess) { rc = EDA_ERR_CUDA; break; }
        if (cudaStreamSynchronize(s) != cudaSuccess) rc = EDA_ERR_CUDA;
    } while (false);
    if (rc != EDA_OK) cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (rc != EDA_OK) return rc;
    f->F = img;
    f->fsign = (float)sigma;
    f->fgrid = G;
    return EDA_OK;
}

int exp_apply_tc_fused(const TcFactor& f, const TcBuffers& bufs, int b, const float* X, int64_t ldx, float* Y,
                       int64_t ldy, int* status, cudaStream_t s) {
    if (b <= 16) return launch_fused<16>(f, bufs, b, X, ldx, Y, ldy, status, s);
    for (int c0 = 0; c0 < b; c0 += 32)
        EDA_TRY(launch_fused<32>(f, bufs, std::min(32, b - c0), X + (int64_t)c0 * ldx, ldx, Y + (int64_t)c0 * ldy, ldy,
                                 status, s));
    return EDA_OK;
}

}  // namespace eda
