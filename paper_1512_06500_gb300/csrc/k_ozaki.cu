// FP64-accurate tall-skinny products on the bf16 tensor cores by error-free splitting of the operands
// into integer digit planes (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications", Numerical
// Algorithms 59, 2012), arranged for tcgen05.
//
// Splitting. Each row i of an operand (the rows of the MMA's M or N side; the reduction index k runs
// along it) gets a power-of-two scale 2^{e_i} with |a_ik| < 2^{e_i}. Then
//     a_ik = 2^{e_i - 7} (s_0 + 2^-8 s_1 + ... + 2^-48 s_6) + tail,   |tail| <= 2^{e_i - 56},
// with integer digits s_q in [-128, 128]: the balanced base-256 digits of the integer nearest to
// a 2^{55 - e}, extracted with integer operations from the bits of a. A digit is exact in bf16 (8
// significant bits).
//
// Products. For D = A B^T over the reduction index (A: M x K, B: N x K, both split),
//     D_ij = 2^{e_i + f_j - 14} sum_q 2^{-8q} L_q,    L_q = sum_{a + b = q} sum_k s^A_{a,ik} s^B_{b,jk},
// truncated at q <= 6 (28 digit-plane products; the dropped terms and both tails are below 2^-53 of
// max_k |a_ik| sum_k |b_jk|). A level L_q summed over a chunk of 128 values of k is an integer below
// (q + 1) 128 2^14 < 2^24, so the tensor cores' FP32 accumulation of a chunk is exact. Each chunk's
// seven levels are read out of tensor memory, converted to integers and folded into two 64-bit
// integer sums per output (G_0 = L_0 2^16 + L_1 2^8 + L_2 and G_1 = L_3 2^24 + L_4 2^16 + L_5 2^8 + L_6),
// so the reduction over k is exact as well; the only roundings are the final conversion to FP64 and the
// 2^-56 truncation of the digits.
//
// Kernel. One CTA per (128-row band of M, split of K), 256 threads: thread 0 issues the bulk copies of
// the pre-tiled digit planes of A (one contiguous 16 KB swizzled tile per K stage of 64 and plane) and
// the TMA boxes of the seven planes of B; thread 32 issues tcgen05.mma (M = 128, K = 16, N = 32 (7 - a) for
// digit plane a of A against planes 0 .. 6 - a of B at once) into one of two accumulator sets of seven
// levels in tensor memory (7 x 32 columns each), switching sets every chunk of two K stages; warps 4-7
// drain a finished set (tcgen05.ld, integer fold) while the tensor cores fill the other. Every wait is
// bounded (ST_TIMEOUT on give-up).
#include "tc_ptx.cuh"

#include <algorithm>
#include <mutex>

namespace eda {

using namespace tc;

namespace {

constexpr int OZ_S = kOzSlices;       // digit planes
constexpr int OZ_N = 32;              // N of every MMA: the narrow operand's columns per launch
constexpr int OZ_AST = 8;             // A ring slots (one 16 KB tile of one plane each)
constexpr int OZ_BST = 2;             // B ring slots (the seven 32 x 64 planes of one K stage)
constexpr int OZ_THREADS = 256;
constexpr int OZ_SET_COLS = 256;      // tensor-memory columns of one accumulator set (7 levels x 32)

struct OzRing {
    __nv_bfloat16 A[OZ_AST][TC_M * TC_KS];            // 8 x 16 KB
    __nv_bfloat16 B[OZ_BST][OZ_S][OZ_N * TC_KS];      // 2 x 7 x 4 KB
    uint64_t fullA[OZ_AST], emptyA[OZ_AST];
    uint64_t fullB[OZ_BST], emptyB[OZ_BST];
    uint64_t accFull[2], accEmpty[2];
    uint32_t tbase;
    int fail;
};
constexpr size_t oz_smem_bytes() { return sizeof(OzRing) + 1024; }

__device__ __forceinline__ OzRing& oz_ring(unsigned char* raw) {
    const uint32_t mis = smem_u32(raw) & 1023u;
    return *reinterpret_cast<OzRing*>(raw + ((1024u - mis) & 1023u));
}

// B from a pre-tiled split operand (BT mode): its planes at tiles + q * slice, the same K tiling as A; the
// product's 32-column block z (blockIdx.z) is the quarter z % 4 of B's 128-row band z / 4, one contiguous
// 4 KB image per plane and stage. upper: skip the blocks wholly below the diagonal (z 32 + 32 <= band 128).
struct OzBTiles {
    const __nv_bfloat16* tiles = nullptr;
    int64_t slice = 0;
    int upper = 0;
};

// D[i, j] (i < M, j < N) = alpha * sum_k A_ik B_jk + beta * C0[i, j]; D, C0 column-major (ld ldd, ldc0),
// the split-th slice of D at D + split * split_stride. A: digit planes at At + q * aslice, pre-tiled
// (128-row bands, kbs tiles of 64 along K per band), row scales expA. B: digit planes read through tmB
// (inner = K, outer = 7 x 32 rows: plane q is rows 32 q .. 32 q + 31), or in BT mode from bt (N rows, the
// CTA's 32 of them chosen by blockIdx.z), row scales expB. K stages [split * kps, min(kst, (split + 1) * kps)).
template <bool BT>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_gemm(const __nv_bfloat16* __restrict__ At, int64_t aslice, int kbs, const __grid_constant__ CUtensorMap tmB,
              const OzBTiles bt, const int* __restrict__ expA, const int* __restrict__ expB, int M, int N, int kst,
              int kps, double alpha, double beta, const double* C0, int64_t ldc0, double* D, int64_t ldd,
              int64_t split_stride, int* status) {
    extern __shared__ unsigned char smraw[];
    OzRing& sm = oz_ring(smraw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int band = blockIdx.x, split = blockIdx.y;
    const int blk = BT ? (int)blockIdx.z : 0;
    if (BT) {
        if (bt.upper && blk * OZ_N + OZ_N <= band * TC_M) return;   // the whole CTA: a uniform exit
        expB += blk * OZ_N;
        N -= blk * OZ_N;
        D += (int64_t)blk * OZ_N * ldd;
        if (C0) C0 += (int64_t)blk * OZ_N * ldc0;
    }
    const int ks0 = split * kps;
    const int nks = max(0, min(kst, ks0 + kps) - ks0);
    const int nchunks = (nks + 1) >> 1;
    if (warp == 0) {
        tmem_alloc(&sm.tbase, 2 * OZ_SET_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < OZ_AST; ++i) {
            mbar_init(&sm.fullA[i], 1);
            mbar_init(&sm.emptyA[i], 1);
        }
        for (int i = 0; i < OZ_BST; ++i) {
            mbar_init(&sm.fullB[i], 1);
            mbar_init(&sm.emptyB[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&sm.accFull[i], 1);
            mbar_init(&sm.accEmpty[i], 128);
        }
        fence_mbar_init();
        sm.fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tbase;

    int issuedA = 0, issuedB = 0;   // producer: copies requested (for the drain after a give-up)
    bool ok = true;
    if (tid == 0) {
        // ---- producer ----
        constexpr uint32_t abytes = TC_M * TC_KS * 2;
        constexpr uint32_t bbytes = OZ_S * OZ_N * TC_KS * 2;
        for (int s = 0; s < nks && ok; ++s) {
            const int kstage = ks0 + s;
            const int bslot = s % OZ_BST;
            if (s >= OZ_BST && !(ok = mbar_wait(&sm.emptyB[bslot], ((s / OZ_BST) - 1) & 1, status))) break;
            mbar_expect_tx(&sm.fullB[bslot], bbytes);
            if (BT) {
                const __nv_bfloat16* src =
                    bt.tiles + ((((int64_t)(blk >> 2)) * kbs + kstage) << 13) + (int64_t)(blk & 3) * (OZ_N * TC_KS);
#pragma unroll
                for (int q = 0; q < OZ_S; ++q)
                    bulk_load(sm.B[bslot][q], src + q * bt.slice, OZ_N * TC_KS * 2, &sm.fullB[bslot]);
            } else {
#pragma unroll
                for (int q = 0; q < OZ_S; ++q)
                    tma_load_2d(sm.B[bslot][q], &tmB, kstage * TC_KS, q * OZ_N, &sm.fullB[bslot]);
            }
            issuedB = s + 1;
            for (int a = 0; a < OZ_S; ++a) {
                const int idx = s * OZ_S + a;
                const int slot = idx % OZ_AST;
                if (idx >= OZ_AST && !(ok = mbar_wait(&sm.emptyA[slot], ((idx / OZ_AST) - 1) & 1, status))) break;
                mbar_expect_tx(&sm.fullA[slot], abytes);
                bulk_load(sm.A[slot], At + a * aslice + ((int64_t)((int64_t)band * kbs + kstage) << 13), abytes,
                          &sm.fullA[slot]);
                issuedA = idx + 1;
            }
        }
    } else if (tid == 32) {
        // ---- MMA issuer ----
        for (int s = 0; s < nks && ok; ++s) {
            const int chunk = s >> 1, set = chunk & 1;
            const bool first = (s & 1) == 0;
            if (first && chunk >= 2 && !(ok = mbar_wait(&sm.accEmpty[set], ((chunk >> 1) - 1) & 1, status))) break;
            const int bslot = s % OZ_BST;
            if (!(ok = mbar_wait(&sm.fullB[bslot], (s / OZ_BST) & 1, status))) break;
            // descriptors differ only in their start-address field (address / 16): a K step of 16 elements
            // is +2; computed once per stage and tile
            const uint64_t bdesc = smem_desc_sw128(smem_u32(sm.B[bslot][0]));
            const uint32_t dset = tmem + (uint32_t)(set * OZ_SET_COLS);
#pragma unroll
            for (int a = 0; a < OZ_S; ++a) {
                const int idx = s * OZ_S + a;
                const int slot = idx % OZ_AST;
                if (!(ok = mbar_wait(&sm.fullA[slot], (idx / OZ_AST) & 1, status))) break;
                tc_fence_after();
                const uint64_t adesc = smem_desc_sw128(smem_u32(sm.A[slot]));
                // A plane a against B planes 0 .. 6 - a in one MMA per K step: those planes are consecutive
                // in shared memory, one operand of N = 32 (7 - a) rows, and the product with plane b lands
                // 32 b columns into the accumulator, so starting it at level column 32 a puts it in level
                // a + b. A is read from shared memory once per K step instead of once per B plane.
                const uint32_t idesc = idesc_bf16(TC_M, OZ_N * (OZ_S - a));
                const uint32_t dcol = dset + (uint32_t)(a * OZ_N);
#pragma unroll
                for (int kk = 0; kk < TC_KS / 16; ++kk) {
                    // the chunk's first MMA (a = 0, first K step) covers all seven levels and overwrites
                    const uint32_t acc = (a == 0 && kk == 0 && first) ? 0u : 1u;
                    mma_bf16(dcol, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, acc);
                }
                mma_commit(&sm.emptyA[slot]);
            }
            if (!ok) break;
            mma_commit(&sm.emptyB[bslot]);
            if ((s & 1) || s == nks - 1) mma_commit(&sm.accFull[set]);
        }
    }
    // ---- epilogue: warps 4-7 fold each finished chunk into exact 64-bit integer sums ----
    long long g0[OZ_N], g1[OZ_N];
#pragma unroll
    for (int c = 0; c < OZ_N; ++c) g0[c] = g1[c] = 0;
    bool eok = true;
    if (warp >= 4) {
        const int ew = warp - 4;
        const uint32_t lanebase = tmem + ((uint32_t)(32 * ew) << 16);
        for (int ch = 0; ch < nchunks; ++ch) {
            const int set = ch & 1;
            if (!(eok = mbar_wait(&sm.accFull[set], (ch >> 1) & 1, status))) break;
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < OZ_N; c0 += 8) {
                uint32_t r[OZ_S][8];
#pragma unroll
                for (int q = 0; q < OZ_S; ++q) tmem_ld8(lanebase + set * OZ_SET_COLS + q * OZ_N + c0, r[q]);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    long long L[OZ_S];
#pragma unroll
                    for (int q = 0; q < OZ_S; ++q) L[q] = (long long)__float2int_rn(__uint_as_float(r[q][c]));
                    g0[c0 + c] += L[0] * 65536LL + L[1] * 256LL + L[2];
                    g1[c0 + c] += ((L[3] * 256LL + L[4]) * 256LL + L[5]) * 256LL + L[6];
                }
            }
            tc_fence_before();
            mbar_arrive(&sm.accEmpty[set]);
        }
    }
    __shared__ int s_ok;
    if ((tid == 0 || tid == 32) && !ok) sm.fail = 1;
    if (warp >= 4 && !eok) sm.fail = 1;
    __syncthreads();
    if (tid == 0) s_ok = sm.fail == 0 ? 1 : 0;
    if (tid == 0 && sm.fail) {
        // after a give-up, wait (bounded again) for this CTA's copies that may still be in flight, so
        // that none lands after the CTA's shared memory is released
        for (int i = max(0, issuedA - OZ_AST); i < issuedA; ++i)
            mbar_wait(&sm.fullA[i % OZ_AST], (i / OZ_AST) & 1, status);
        for (int i = max(0, issuedB - OZ_BST); i < issuedB; ++i)
            mbar_wait(&sm.fullB[i % OZ_BST], (i / OZ_BST) & 1, status);
    }
    __syncthreads();
    if (warp >= 4) {
        const int i = band * TC_M + 32 * (warp - 4) + lane;
        if (i < M) {
            const int ea = expA[i];
            double* Ds = D + (int64_t)split * split_stride;
#pragma unroll
            for (int c = 0; c < OZ_N; ++c) {
                if (c >= N) break;
                const int e = ea + expB[c];
                double v = (s_ok && nks > 0) ? ldexp((double)g0[c], e - 30) + ldexp((double)g1[c], e - 62) : 0.0;
                if (!s_ok) v = nan("");
                double out = alpha * v;
                if (beta != 0.0) out = fma(beta, C0[(int64_t)c * ldc0 + i], out);
                Ds[(int64_t)c * ldd + i] = out;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 2 * OZ_SET_COLS);
}

// frexp exponent of |v| (|v| = f 2^e, f in [0.5, 1)) read from the bits of v; kOzExpZero for v = 0.
// Inf and NaN give 1025.
constexpr int kOzExpZero = -1061109568;   // every byte 0xC0: the fill of a scale array before its maxima
__device__ __forceinline__ int oz_frexp_exp(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
    if (b == 0) return kOzExpZero;
    const int ef = (int)(b >> 52);
    return ef ? ef - 1022 : -1010 - __clzll((long long)b);   // subnormal: b is the mantissa
}

// Digits of x_0 = v 2^{7 - e} (|v| < 2^e). N = v 2^{55 - e} rounded to an integer (|N| <= 2^55, the
// rounding error at most half a unit of 2^{e - 55}), written in balanced base 256: s_6 .. s_1 are its
// low bytes taken as residues in [-128, 127] from the low end, s_0 what remains (|s_0| <= 128, since
// the low digits sum to less than 2^47 in magnitude). Then x_0 = sum_q 2^{-8q} s_q up to 2^{-49}, the
// same precision as the rounding recurrence x_{q+1} = 256 (x_q - rint(x_q)). Integer operations only
// (the mantissa and exponent come from the bits of v), so the split runs at memory speed rather than
// at the FP64 rate. Returns false for Inf or NaN (digits zero).
__device__ __forceinline__ bool oz_digits(double v, int e, __nv_bfloat16 (&s)[OZ_S]) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    long long N = 0;
    if (ef != 0x7FF) {
        int ex = -1074;                       // |v| = m 2^ex
        if (ef) {
            m |= 1ull << 52;
            ex = ef - 1075;
        }
        const int sh = ex + 55 - e;           // <= 2 whenever |v| < 2^e
        if (m != 0) {
            if (sh >= 0)
                N = (long long)(m << sh);
            else if (sh > -56)
                N = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
        }
        if (bits >> 63) N = -N;
    }
#pragma unroll
    for (int q = OZ_S - 1; q >= 1; --q) {
        const int dq = (int)((N + 128) & 255) - 128;
        s[q] = __float2bfloat16_rn((float)dq);
        N = (N - dq) >> 8;                    // exact: N - dq is a multiple of 256
    }
    s[0] = __float2bfloat16_rn((float)N);
    return ef != 0x7FF;
}

// Column scales: e[c] = max over rows r of the frexp exponent of A[r, c] (d x ncols, lda), kOzExpZero for
// a zero column. One CTA per (column, chunk of kOzExpChunk rows); each thread issues its eight loads
// before it reduces them (the scan is bound by the number of loads in flight), and the CTA's maximum is
// merged by one atomicMax into e, which the host fills with kOzExpZero first.
constexpr int kOzExpThreads = 256;
constexpr int kOzExpPer = 8;
constexpr int kOzExpChunk = kOzExpThreads * kOzExpPer;
__global__ void __launch_bounds__(kOzExpThreads) k_oz_exp_cols(int64_t rows, const double* __restrict__ A,
                                                              int64_t lda, int* __restrict__ e) {
    __shared__ int wmax[kOzExpThreads / 32];
    const int c = blockIdx.x;
    const double* col = A + (int64_t)c * lda;
    const int64_t r0 = (int64_t)blockIdx.y * kOzExpChunk + threadIdx.x;
    double v[kOzExpPer];
#pragma unroll
    for (int u = 0; u < kOzExpPer; ++u) {
        const int64_t r = r0 + (int64_t)u * kOzExpThreads;
        v[u] = r < rows ? col[r] : 0.0;
    }
    int mx = kOzExpZero;
#pragma unroll
    for (int u = 0; u < kOzExpPer; ++u) mx = max(mx, oz_frexp_exp(v[u]));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kOzExpThreads / 32; ++w) mx = max(mx, wmax[w]);
        if (mx != kOzExpZero) atomicMax(&e[c], mx);
    }
}

// Row scales of a split operand whose M rows are the ROWS of A (d x m, lda): thread per row, 0 for a
// zero row.
__global__ void k_oz_exp_rows(int64_t rows, int cols, const double* __restrict__ A, int64_t lda,
                              int* __restrict__ e) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int mx = kOzExpZero;
    for (int c = 0; c < cols; ++c) mx = max(mx, oz_frexp_exp(A[(int64_t)c * lda + r]));
    e[r] = mx == kOzExpZero ? 0 : mx;
}

// The seven digit planes of a narrow operand B (K x p, ldb; its columns are the N rows of the product),
// planes [7][32][ld] (plane q, row j at (32 q + j) ld), zero for j >= p or k >= K. Eight consecutive k per
// thread: one 64-byte read and one 16-byte store per plane.
__global__ void k_oz_split_narrow(int64_t K, int p, const double* __restrict__ B, int64_t ldb,
                                  const int* __restrict__ e, int64_t ld, __nv_bfloat16* __restrict__ out,
                                  int* __restrict__ status) {
    const int64_t groups = ld / 8;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)OZ_N * groups) return;
    const int j = (int)(t / groups);
    const int64_t k0 = (t % groups) * 8;
    const int ex = j < p ? e[j] : 0;
    __align__(16) __nv_bfloat16 dg[OZ_S][8];
    bool fin = true;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const double v = (j < p && k0 + u < K) ? B[(int64_t)j * ldb + k0 + u] : 0.0;
        __nv_bfloat16 sq[OZ_S];
        fin &= oz_digits(v, ex, sq);
#pragma unroll
        for (int q = 0; q < OZ_S; ++q) dg[q][u] = sq[q];
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q)
        *reinterpret_cast<uint4*>(out + ((int64_t)q * OZ_N + j) * ld + k0) = *reinterpret_cast<const uint4*>(dg[q]);
}

// Digit planes of the columns i0 .. i1 of A (d x m, lda) as M rows of a split operand whose K index runs down
// the columns (rows_are_cols layout), 8 consecutive k per thread: one 64-byte read of A and one 16-byte
// store per plane. e: the scales of those columns (e[i - i0]). Rows at or beyond Mvalid (the padding of
// the last 128-row band) are written as zeros.
__global__ void k_oz_split_cols8(const double* __restrict__ A, int64_t lda, int i0, int i1, int Mvalid, int64_t K,
                                 const int* __restrict__ e, int kbs, int64_t ld, __nv_bfloat16* __restrict__ out,
                                 int64_t slice, int* __restrict__ status) {
    const int64_t groups = ld / 8;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)(i1 - i0) * groups) return;
    const int i = i0 + (int)(t / groups);
    const int64_t k0 = (t % groups) * 8;
    const bool row = i < Mvalid;
    const int ex = row ? e[i - i0] : 0;
    __align__(16) __nv_bfloat16 dg[OZ_S][8];
    bool fin = true;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const double v = (row && k0 + u < K) ? A[(int64_t)i * lda + k0 + u] : 0.0;
        __nv_bfloat16 sq[OZ_S];
        fin &= oz_digits(v, ex, sq);
#pragma unroll
        for (int q = 0; q < OZ_S; ++q) dg[q][u] = sq[q];
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
    const int64_t off = tile_off(i, k0, kbs);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q)
        *reinterpret_cast<uint4*>(out + q * slice + off) = *reinterpret_cast<const uint4*>(dg[q]);
}

// Digit planes of the rows of A (M x K, lda; M rows = rows of A, K along its columns k0 .. k1, k0 a multiple
// of 8), 8 consecutive k per thread: eight reads, each coalesced across the threads of a warp (consecutive
// rows), and one 16-byte store per plane. Columns at or beyond Kvalid, and rows at or beyond M, are zero.
__global__ void k_oz_split_rows8(const double* __restrict__ A, int64_t lda, int64_t M, int64_t k0, int64_t k1,
                                 int64_t Kvalid, const int* __restrict__ e, int kbs, __nv_bfloat16* __restrict__ out,
                                 int64_t slice, int* __restrict__ status) {
    const int64_t mpad = (M + TC_M - 1) / TC_M * TC_M;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t groups = (k1 - k0 + 7) / 8;
    if (t >= mpad * groups) return;
    const int64_t i = t % mpad;
    const int64_t kg = k0 + (t / mpad) * 8;
    const int ex = i < M ? e[i] : 0;
    __align__(16) __nv_bfloat16 dg[OZ_S][8];
    bool fin = true;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t k = kg + u;
        const double v = (i < M && k < Kvalid) ? A[k * lda + i] : 0.0;
        __nv_bfloat16 sq[OZ_S];
        fin &= oz_digits(v, ex, sq);
#pragma unroll
        for (int q = 0; q < OZ_S; ++q) dg[q][u] = sq[q];
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
    const int64_t off = tile_off(i, kg, kbs);
#pragma unroll
    for (int q = 0; q < OZ_S; ++q)
        *reinterpret_cast<uint4*>(out + q * slice + off) = *reinterpret_cast<const uint4*>(dg[q]);
}

// Growing a row-scaled operand (the Krylov basis, M = d rows, K = the columns so far) from k0 to k1 columns:
// thread per row. A row whose scale is unchanged by the new columns gets the digits of its new 8-groups
// [k0 rounded down to 8, k1) (the part of a group below k0 rewritten with identical digits); a row whose
// scale grows records the new scale and joins list (count in list[0]) for a full re-split by
// k_oz_resplit_listed. Zero rows keep the scale kOzExpZero.
__global__ void k_oz_grow_rows(const double* __restrict__ A, int64_t lda, int64_t M, int64_t k0, int64_t k1,
                               int* __restrict__ e, int kbs, __nv_bfloat16* __restrict__ out, int64_t slice,
                               int* __restrict__ list, int* __restrict__ status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    int mnew = kOzExpZero;
    for (int64_t k = k0; k < k1; ++k) mnew = max(mnew, oz_frexp_exp(A[k * lda + i]));
    int eold = k0 == 0 ? mnew : e[i];
    if (k0 == 0) {
        e[i] = mnew;   // the first columns: their digits below, with their own scale
    } else if (mnew > eold) {
        e[i] = mnew;
        list[1 + atomicAdd(&list[0], 1)] = (int)i;
        return;
    }
    bool fin = true;
    for (int64_t kg = k0 & ~(int64_t)7; kg < k1; kg += 8) {
        __align__(16) __nv_bfloat16 dg[OZ_S][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t k = kg + u;
            const double v = k < k1 ? A[k * lda + i] : 0.0;
            __nv_bfloat16 sq[OZ_S];
            fin &= oz_digits(v, eold, sq);
#pragma unroll
            for (int q = 0; q < OZ_S; ++q) dg[q][u] = sq[q];
        }
        const int64_t off = tile_off(i, kg, kbs);
#pragma unroll
        for (int q = 0; q < OZ_S; ++q)
            *reinterpret_cast<uint4*>(out + q * slice + off) = *reinterpret_cast<const uint4*>(dg[q]);
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
}

// Full re-split, columns 0 .. K, of the rows in list (count list[0]), one (row, 8-group) per thread step.
__global__ void k_oz_resplit_listed(const double* __restrict__ A, int64_t lda, int64_t K, const int* __restrict__ e,
                                    int kbs, __nv_bfloat16* __restrict__ out, int64_t slice,
                                    const int* __restrict__ list, int* __restrict__ status) {
    const int64_t groups = (K + 7) / 8;
    const int64_t total = (int64_t)list[0] * groups;
    bool fin = true;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = list[1 + t % list[0]];
        const int64_t kg = (t / list[0]) * 8;
        const int ex = e[i];
        __align__(16) __nv_bfloat16 dg[OZ_S][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t k = kg + u;
            const double v = k < K ? A[k * lda + i] : 0.0;
            __nv_bfloat16 sq[OZ_S];
            fin &= oz_digits(v, ex, sq);
#pragma unroll
            for (int q = 0; q < OZ_S; ++q) dg[q][u] = sq[q];
        }
        const int64_t off = tile_off(i, kg, kbs);
#pragma unroll
        for (int q = 0; q < OZ_S; ++q)
            *reinterpret_cast<uint4*>(out + q * slice + off) = *reinterpret_cast<const uint4*>(dg[q]);
    }
    if (!fin) atomicOr(status, ST_NONFINITE);
}

// D[i, j] = alpha * sum_s P[s][j][i] + beta * D[i, j], splits added in order (deterministic).
__global__ void k_oz_reduce(int M, int N, int splits, const double* __restrict__ P, int64_t sstride, double alpha,
                            double beta, const double* C0, int64_t ldc0, double* D, int64_t ldd) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * N) return;
    const int i = (int)(t % M), j = (int)(t / M);
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += P[(int64_t)s * sstride + (int64_t)j * M + i];
    double v = alpha * acc;
    if (beta != 0.0) v = fma(beta, C0[(int64_t)j * ldc0 + i], v);
    D[(int64_t)j * ldd + i] = v;
}

int oz_attr() {
    static std::once_flag once;
    static cudaError_t rc = cudaSuccess;
    std::call_once(once, [] {
        rc = cudaFuncSetAttribute(k_oz_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes());
        if (rc == cudaSuccess)
            rc = cudaFuncSetAttribute(k_oz_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)oz_smem_bytes());

    });
    EDA_CUDA_TRY(rc);
    return EDA_OK;
}

}  // namespace

size_t oz_operand_bytes(int64_t M, int64_t K) {
    const int64_t mt = (M + TC_M - 1) / TC_M, kb = (K + TC_KS - 1) / TC_KS;
    const size_t plane = (size_t)mt * kb * TC_M * TC_KS * 2;
    return OZ_S * ((plane + 255) / 256 * 256) + ((size_t)M * 4 + 255) / 256 * 256;
}

// Column scales of columns 0 .. ncols of A (K x ncols, lda) into e.
static int oz_col_exps(int64_t K, const double* A, int64_t lda, int ncols, int* e, cudaStream_t s) {
    if (ncols <= 0) return EDA_OK;
    EDA_CUDA_TRY(cudaMemsetAsync(e, 0xC0, (size_t)ncols * sizeof(int), s));   // kOzExpZero in every entry
    const dim3 grid((unsigned)ncols, (unsigned)ceil_div(std::max<int64_t>(K, 1), kOzExpChunk));
    k_oz_exp_cols<<<grid, kOzExpThreads, 0, s>>>(K, A, lda, e);
    EDA_LAUNCHED();
    return EDA_OK;
}

int oz_operand_make(const double* A, int64_t lda, int64_t M, int64_t K, bool rows_are_cols, void* mem,
                    OzOperand* op, int* status, cudaStream_t s) {
    const int64_t mt = (M + TC_M - 1) / TC_M, kb = (K + TC_KS - 1) / TC_KS;
    const int64_t plane = mt * kb * TC_M * TC_KS;
    const int64_t slice = ((plane * 2 + 255) / 256 * 256) / 2;
    op->tiles = static_cast<__nv_bfloat16*>(mem);
    op->slice = slice;
    op->exps = reinterpret_cast<int*>(static_cast<char*>(mem) + OZ_S * slice * 2);
    op->M = M;
    op->K = K;
    op->kbs = (int)kb;
    op->mtiles = (int)mt;
    const int64_t ld = kb * TC_KS, mpad = mt * TC_M;
    if (rows_are_cols) {
        EDA_TRY(oz_col_exps(K, A, lda, (int)M, op->exps, s));
        k_oz_split_cols8<<<ceil_div(mpad * (ld / 8), 256), 256, 0, s>>>(A, lda, 0, (int)mpad, (int)M, K, op->exps,
                                                                        (int)kb, ld, op->tiles, slice, status);
    } else {
        k_oz_exp_rows<<<ceil_div(M, 256), 256, 0, s>>>(M, (int)K, A, lda, op->exps);
        EDA_LAUNCHED();
        k_oz_split_rows8<<<ceil_div(mpad * (ld / 8), 256), 256, 0, s>>>(A, lda, M, 0, ld, K, op->exps, (int)kb,
                                                                         op->tiles, slice, status);
    }
    EDA_LAUNCHED();
    return EDA_OK;
}

// A split operand with room for Mcap rows (columns of a d x Mcap matrix, K = d) or for Kcap values of K
// (rows_are_cols = false: M = d rows, K up to Kcap columns), planes zeroed, no row filled yet.
int oz_operand_init(int64_t Mcap, int64_t Kcap, void* mem, OzOperand* op, cudaStream_t s) {
    const int64_t mt = (Mcap + TC_M - 1) / TC_M, kb = (Kcap + TC_KS - 1) / TC_KS;
    const int64_t plane = mt * kb * TC_M * TC_KS;
    const int64_t slice = ((plane * 2 + 255) / 256 * 256) / 2;
    op->tiles = static_cast<__nv_bfloat16*>(mem);
    op->slice = slice;
    op->exps = reinterpret_cast<int*>(static_cast<char*>(mem) + OZ_S * slice * 2);
    op->M = 0;
    op->K = 0;
    op->kbs = (int)kb;
    op->mtiles = 0;
    EDA_CUDA_TRY(cudaMemsetAsync(mem, 0, (size_t)OZ_S * slice * 2, s));
    return EDA_OK;
}

int oz_append_cols(const double* A, int64_t lda, int i0, int i1, int64_t K, OzOperand* op, int* status,
                   cudaStream_t s) {
    if (i1 <= i0) return EDA_OK;
    EDA_TRY(oz_col_exps(K, A + (int64_t)i0 * lda, lda, i1 - i0, op->exps + i0, s));
    const int64_t ld = (int64_t)op->kbs * TC_KS;
    k_oz_split_cols8<<<ceil_div((int64_t)(i1 - i0) * (ld / 8), 256), 256, 0, s>>>(
        A, lda, i0, i1, i1, K, op->exps + i0, op->kbs, ld, op->tiles, op->slice, status);
    EDA_LAUNCHED();
    op->M = i1;
    op->K = K;
    op->mtiles = ceil_div(i1, TC_M);
    return EDA_OK;
}

int oz_resplit_rows(const double* A, int64_t lda, int64_t M, int64_t K, OzOperand* op, int* status, cudaStream_t s) {
    k_oz_exp_rows<<<ceil_div(M, 256), 256, 0, s>>>(M, (int)K, A, lda, op->exps);
    EDA_LAUNCHED();
    const int64_t kpad = (K + TC_KS - 1) / TC_KS * TC_KS;
    const int64_t mpad = (M + TC_M - 1) / TC_M * TC_M;
    k_oz_split_rows8<<<ceil_div(mpad * (kpad / 8), 256), 256, 0, s>>>(A, lda, M, 0, kpad, K, op->exps, op->kbs,
                                                                      op->tiles, op->slice, status);
    EDA_LAUNCHED();
    op->M = M;
    op->K = K;
    op->mtiles = ceil_div(M, TC_M);
    return EDA_OK;
}

int oz_grow_rows(const double* A, int64_t lda, int64_t M, int64_t k0, int64_t k1, OzOperand* op, int* list,
                 int* status, cudaStream_t s) {
    if (k1 <= k0) return EDA_OK;
    EDA_CUDA_TRY(cudaMemsetAsync(list, 0, sizeof(int), s));
    k_oz_grow_rows<<<ceil_div(M, 256), 256, 0, s>>>(A, lda, M, k0, k1, op->exps, op->kbs, op->tiles, op->slice, list,
                                                    status);
    EDA_LAUNCHED();
    k_oz_resplit_listed<<<2 * sm_count(), 256, 0, s>>>(A, lda, k1, op->exps, op->kbs, op->tiles, op->slice, list,
                                                        status);
    EDA_LAUNCHED();
    op->M = M;
    op->K = k1;
    op->mtiles = ceil_div(M, TC_M);
    return EDA_OK;
}

size_t oz_narrow_bytes(int64_t Kmax, int max_splits, int64_t Mmax) {
    const int64_t ld = (Kmax + TC_KS - 1) / TC_KS * TC_KS;
    return ((size_t)OZ_S * OZ_N * ld * 2 + 255) / 256 * 256 + 256 +
           ((size_t)max_splits * OZ_N * Mmax * 8 + 255) / 256 * 256;
}

int oz_narrow_make(int64_t Kmax, int max_splits, int64_t Mmax, void* mem, OzNarrow* nb) {
    const int64_t ld = (Kmax + TC_KS - 1) / TC_KS * TC_KS;
    char* p = static_cast<char*>(mem);
    nb->planes = reinterpret_cast<__nv_bfloat16*>(p);
    p += ((size_t)OZ_S * OZ_N * ld * 2 + 255) / 256 * 256;
    nb->exps = reinterpret_cast<int*>(p);
    p += 256;
    nb->partial = reinterpret_cast<double*>(p);
    nb->pcap = (size_t)max_splits * OZ_N * Mmax;
    nb->ldmax = ld;
    nb->map_ld = 0;
    return EDA_OK;
}

int oz_gemm(const OzOperand& A, OzNarrow& nb, int p, const double* B, int64_t ldb, double alpha, double beta,
            const double* C0, int64_t ldc0, double* D, int64_t ldd, int* status, cudaStream_t s) {
    if (p < 1 || p > OZ_N) return EDA_ERR_INVALID_ARG;
    const int64_t ld = (A.K + TC_KS - 1) / TC_KS * TC_KS;
    if (ld > nb.ldmax) return EDA_ERR_INVALID_ARG;
    EDA_TRY(oz_attr());
    if (nb.map_ld != ld) {
        EDA_TRY(make_map(&nb.map, nb.planes, (uint64_t)ld, (uint64_t)OZ_S * OZ_N, (uint64_t)ld, OZ_N));
        nb.map_ld = ld;
    }
    // algorithmic work, as for the FP64 product it replaces: 2 M K p flops; A read once (seven bf16
    // digit planes), B read and D written once in FP64
    ProfScope prof("oz_gemm", s, 2.0 * (double)A.M * A.K * p,
                   2.0 * OZ_S * (double)A.M * A.K + 8.0 * (double)A.K * p + 8.0 * (double)A.M * p);
    EDA_TRY(oz_col_exps(A.K, B, ldb, p, nb.exps, s));
    k_oz_split_narrow<<<ceil_div((int64_t)OZ_N * (ld / 8), 256), 256, 0, s>>>(A.K, p, B, ldb, nb.exps, ld, nb.planes,
                                                                            status);
    EDA_LAUNCHED();
    const int kst = (int)(ld / TC_KS);
    // K splits: fill the SMs with one CTA each (the kernel holds all of an SM's tensor memory)
    const int nsm = sm_count();
    int splits = std::max(1, std::min(kst / 2, nsm / std::max(1, A.mtiles)));
    while (splits > 1 && (size_t)splits * p * A.M > nb.pcap) --splits;
    const int kps = ceil_div(kst, splits);
    splits = ceil_div(kst, kps);
    const dim3 grid((unsigned)A.mtiles, (unsigned)splits);
    const int64_t sstride = splits == 1 ? 0 : (int64_t)p * A.M;
    {
        // the tensor-core kernel alone: it must read the seven digit planes of A and of B once and write D
        // tensor work: the 28 digit-plane products of 2 M K p flops each
        ProfScope kprof("oz_kernel", s, 56.0 * (double)A.M * A.K * p,
                        2.0 * OZ_S * ((double)A.M * A.K + (double)A.K * p) + 8.0 * (double)A.M * p);
        const OzBTiles none{};
        if (splits == 1)
            k_oz_gemm<false><<<grid, OZ_THREADS, oz_smem_bytes(), s>>>(A.tiles, A.slice, A.kbs, nb.map, none, A.exps,
                                                                       nb.exps, (int)A.M, p, kst, kps, alpha, beta, C0,
                                                                       ldc0, D, ldd, 0, status);
        else
            k_oz_gemm<false><<<grid, OZ_THREADS, oz_smem_bytes(), s>>>(A.tiles, A.slice, A.kbs, nb.map, none, A.exps,
                                                                       nb.exps, (int)A.M, p, kst, kps, 1.0, 0.0,
                                                                       nullptr, 0, nb.partial, A.M, sstride, status);
        EDA_LAUNCHED();
    }
    if (splits == 1) return EDA_OK;
    k_oz_reduce<<<ceil_div((int64_t)A.M * p, 256), 256, 0, s>>>((int)A.M, p, splits, nb.partial, sstride, alpha,
                                                                 beta, C0, ldc0, D, ldd);
    EDA_LAUNCHED();
    return EDA_OK;
}

// D[i, j] = alpha sum_k A_ik B_jk + beta C0[i, j] for two split operands with the same K (i < A.M, j < B.M):
// one launch over (A band, B 32-row block); upper: only the blocks meeting the upper triangle i <= j, the
// rest filled by the mirror image (A and B the same operand: the product is then exactly symmetric).
__global__ void k_oz_mirror_lower(int n, double* D, int64_t ldd) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * n) return;
    const int i = (int)(t % n), j = (int)(t / n);
    if (i > j && (j + OZ_N) / OZ_N * OZ_N <= (i / TC_M) * TC_M) D[(int64_t)j * ldd + i] = D[(int64_t)i * ldd + j];
}

int oz_gemm_tiled(const OzOperand& A, const OzOperand& B, double alpha, double beta, const double* C0, int64_t ldc0,
                  double* D, int64_t ldd, bool upper, int* status, cudaStream_t s, double* part, size_t pcap) {
    if (A.K != B.K || A.kbs != B.kbs || A.M < 1 || B.M < 1) return EDA_ERR_INVALID_ARG;
    if (upper && (A.tiles != B.tiles || beta != 0.0)) return EDA_ERR_INVALID_ARG;
    EDA_TRY(oz_attr());
    const int kst = A.kbs;
    const int nblk = ceil_div(B.M, OZ_N);
    // K splits only when the (band, block) grid leaves SMs idle and a partial buffer is given
    int splits = 1;
    if (part && !upper) {
        splits = std::max(1, std::min(kst / 8, sm_count() / std::max(1, A.mtiles * nblk)));
        while (splits > 1 && (size_t)splits * A.M * B.M > pcap) --splits;
    }
    const int kps = ceil_div(kst, splits);
    splits = ceil_div(kst, kps);
    const dim3 grid((unsigned)A.mtiles, (unsigned)splits, (unsigned)nblk);
    OzBTiles bt;
    bt.tiles = B.tiles;
    bt.slice = B.slice;
    bt.upper = upper ? 1 : 0;
    // tensor work of the computed blocks: 28 digit-plane products of 2 x 128 x 32 x K flops per (band, block)
    double blocks = 0.0;
    for (int b = 0; b < A.mtiles; ++b)
        for (int z = 0; z < nblk; ++z) blocks += (upper && z * OZ_N + OZ_N <= b * TC_M) ? 0.0 : 1.0;
    {
        ProfScope kprof("oz_tiled", s, 56.0 * TC_M * OZ_N * (double)kst * TC_KS * blocks,
                        2.0 * OZ_S * ((double)A.M * A.K + (double)A.K * B.M) + 8.0 * (double)A.M * B.M);
        // tmB is not read in this mode; the operand's planes are passed in bt
        static const CUtensorMap unused{};
        if (splits == 1)
            k_oz_gemm<true><<<grid, OZ_THREADS, oz_smem_bytes(), s>>>(A.tiles, A.slice, A.kbs, unused, bt, A.exps,
                                                                      B.exps, (int)A.M, (int)B.M, kst, kps, alpha, beta,
                                                                      C0, ldc0, D, ldd, 0, status);
        else
            k_oz_gemm<true><<<grid, OZ_THREADS, oz_smem_bytes(), s>>>(A.tiles, A.slice, A.kbs, unused, bt, A.exps,
                                                                      B.exps, (int)A.M, (int)B.M, kst, kps, 1.0, 0.0,
                                                                      nullptr, 0, part, A.M, (int64_t)A.M * B.M, status);
        EDA_LAUNCHED();
    }
    if (splits > 1) {
        k_oz_reduce<<<ceil_div((int64_t)A.M * B.M, 256), 256, 0, s>>>((int)A.M, (int)B.M, splits, part,
                                                                     (int64_t)A.M * B.M, alpha, beta, C0, ldc0, D, ldd);
        EDA_LAUNCHED();
    }
    if (upper) {
        k_oz_mirror_lower<<<ceil_div((int64_t)A.M * A.M, 256), 256, 0, s>>>((int)A.M, D, ldd);
        EDA_LAUNCHED();
    }
    return EDA_OK;
}

}  // namespace eda
