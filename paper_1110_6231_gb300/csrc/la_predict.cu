// Learned warm start: column statistics, a set-encoder price predictor and
// its training step.
//
// Refine's initialisation makes any price vector eps-optimal (Sect. 5.2,
// Algorithm 5.2), so a solve may start from predicted prices and from a small
// eps0 instead of p = 0 and eps0 = C~ (Algorithm 5.0): the result is the same
// exact optimum, only the work changes. The predictor estimates the optimal
// column duals v(y) (paper sign: p(y) = (n+1) v(y) on scaled costs) from
// per-column cost statistics.
//
// Network (per instance; columns are a set):
//   h1_j  = relu(W1^T f_j + b1)                 f_j: 8 features, padded to 16
//   c     = mean_j h1_j                         set pooling
//   h2_j  = relu(W2^T [h1_j ; c] + b2)
//   y_j   = W3^T h2_j + b3                      predicted (v(j) - mean v) / T
// Every matrix product runs on the Blackwell tensor cores (tcgen05): the
// operands are BF16 in global memory (activations written in BF16 by the
// kernel that produces them, the weights converted to BF16 once per call),
// loaded by TMA into shared memory with the 128-byte swizzle, multiplied by
// tcgen05.mma into FP32 accumulators in tensor memory and read back by
// tcgen05.ld in the epilogue (bias, ReLU, FP32 and BF16 stores, split-K
// atomics). The master weights and the optimiser state stay FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "la.h"
#include "la_device.cuh"
#include "la_tc.cuh"

namespace {

namespace tc = la::tc;

constexpr int F = LA_PRED_FEATURES_PADDED;   // 16
constexpr int H = LA_PRED_WIDTH;             // 128
// parameter offsets (floats) after the header
constexpr int OFF_W1 = LA_PRED_HEADER;
constexpr int OFF_B1 = OFF_W1 + F * H;
constexpr int OFF_W2 = OFF_B1 + H;
constexpr int OFF_B2 = OFF_W2 + 2 * H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H * 8;
constexpr int NPARAM = OFF_B3 + 8;
static_assert(NPARAM == LA_PRED_PARAMS, "parameter layout");

// ------------------------------------------------------------ features

// Row pass: row minimum (for the row-reduced column statistics) and the
// argmin column of each row (column popularity). One warp per row.
__global__ void k_row_stats(const int32_t *__restrict__ C, int n, float *__restrict__ rowmin,
                            int *__restrict__ pop) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= n) return;
    const int32_t *r = C + (size_t)row * n;
    int best = INT_MAX, arg = INT_MAX;
    for (int y = lane; y < n; y += 32) {
        const int c = r[y];
        if (c < best) { best = c; arg = y; }
    }
    for (int o = 16; o; o >>= 1) {
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob < best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    if (lane == 0) {
        rowmin[row] = (float)best;
        atomicAdd(pop + arg, 1);
    }
}

constexpr int kColBlocks = 16;   // row blocks of the column pass (partials merged by k_features)

// Column pass over a block of rows: per column, min and second min of C and
// of the row-reduced C - rowmin, and the sum. Partials [rb][n][5].
__global__ void k_col_stats(const int32_t *__restrict__ C, int n, const float *__restrict__ rowmin,
                            float *__restrict__ part, int rows_per_block) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y >= n) return;
    const int r0 = blockIdx.y * rows_per_block;
    const int r1 = min(n, r0 + rows_per_block);
    float a1 = INFINITY, a2 = INFINITY, q1 = INFINITY, q2 = INFINITY, sum = 0.f;
    for (int x = r0; x < r1; ++x) {
        const float c = (float)C[(size_t)x * n + y];
        const float q = c - rowmin[x];
        sum += c;
        if (c < a1) { a2 = a1; a1 = c; } else if (c < a2) a2 = c;
        if (q < q1) { q2 = q1; q1 = q; } else if (q < q2) q2 = q;
    }
    float *p = part + ((size_t)blockIdx.y * n + y) * 5;
    p[0] = a1; p[1] = a2; p[2] = q1; p[3] = q2; p[4] = sum;
}

// Merge partials, then the instance scale and the normalised features
// (one block). Writes feats [n][16] and inst[0] = T (cost units per target
// unit), inst[1] = mean of the column minima.
__global__ void __launch_bounds__(1024)
k_features(int n, int rb, const float *__restrict__ part, const int *__restrict__ pop,
           float *__restrict__ colbuf, float *__restrict__ feats, float *__restrict__ inst,
           __nv_bfloat16 *__restrict__ xb) {
    __shared__ float red[4][32];
    __shared__ float s_mean[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float s_a = 0, s_gap = 0, s_q = 0, s_m = 0;
    for (int y = tid; y < n; y += blockDim.x) {
        float a1 = INFINITY, a2 = INFINITY, q1 = INFINITY, q2 = INFINITY, sum = 0;
        for (int b = 0; b < rb; ++b) {
            const float *p = part + ((size_t)b * n + y) * 5;
            const float pa1 = p[0], pa2 = p[1], pq1 = p[2], pq2 = p[3];
            if (pa1 < a1) { a2 = fminf(a1, pa2); a1 = pa1; } else a2 = fminf(a2, pa1);
            if (pq1 < q1) { q2 = fminf(q1, pq2); q1 = pq1; } else q2 = fminf(q2, pq1);
            sum += p[4];
        }
        if (n == 1) { a2 = a1; q2 = q1; }
        const float m = sum / (float)n;
        float *cb = colbuf + (size_t)y * 5;
        cb[0] = a1; cb[1] = a2; cb[2] = q1; cb[3] = q2; cb[4] = m;
        s_a += a1; s_gap += a2 - a1; s_q += q1; s_m += m;
    }
    float v[4] = {s_a, s_gap, s_q, s_m};
    for (int k = 0; k < 4; ++k) {
        for (int o = 16; o; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) red[k][warp] = v[k];
    }
    __syncthreads();
    if (tid < 4) {
        float t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[tid][w];
        s_mean[tid] = t / (float)n;
    }
    __syncthreads();
    const float abar = s_mean[0], T = 1.0f + s_mean[1], qbar = s_mean[2], mbar = s_mean[3];
    // spread of the column means
    float s2 = 0;
    for (int y = tid; y < n; y += blockDim.x) {
        const float d = colbuf[(size_t)y * 5 + 4] - mbar;
        s2 += d * d;
    }
    for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    __syncthreads();
    if (lane == 0) red[0][warp] = s2;
    __syncthreads();
    if (tid == 0) {
        float t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[0][w];
        s_mean[0] = sqrtf(t / (float)n) + 1.0f;
        inst[0] = T;
        inst[1] = abar;
    }
    __syncthreads();
    const float msd = s_mean[0];
    const float lt = logf(T) * 0.1f, ln = logf((float)n) * 0.1f;
    for (int y = tid; y < n; y += blockDim.x) {
        const float *cb = colbuf + (size_t)y * 5;
        float *f = feats + (size_t)y * F;
        f[0] = (cb[0] - abar) / T;
        f[1] = (cb[1] - cb[0]) / T;
        f[2] = (cb[2] - qbar) / T;
        f[3] = (cb[3] - cb[2]) / T;
        f[4] = log1pf((float)pop[y]);
        f[5] = (cb[4] - mbar) / msd;
        f[6] = lt;
        f[7] = ln;
        for (int k = 8; k < F; ++k) f[k] = 0.f;
    }
    if (xb) {   // layer 1's operand: BF16, rows padded to the 64-wide TMA box (coalesced)
        __syncthreads();
        for (int e = tid; e < n * 64; e += blockDim.x) {
            const int y = e >> 6, k = e & 63;
            xb[e] = __float2bfloat16_rn(k < 8 ? feats[(size_t)y * F + k] : 0.f);
        }
    }
}

// ------------------------------------------------------------ GEMM on tcgen05

// C[M x N] = A[M x K] * B[N x K]^T. A and B are K-major BF16 in global
// memory, described by TMA tensor maps with 64-element (128-byte) boxes and
// the 128-byte swizzle. One CTA of 128 threads computes 128 rows of C
// (TMEM lanes) by BN columns over the K range of its split (gridDim.y):
// thread 0 streams K in chunks of 64 through two shared-memory stages (TMA
// completes on a per-stage mbarrier) and issues four 128 x BN x 16 MMAs
// per chunk (fewer in a last, partial chunk); tcgen05.commit frees a stage
// once its MMAs are done and signals the end. Then every warp reads its 32
// TMEM lanes (rows) back 16 columns at a time for the epilogue. Every wait
// is bounded (1 s): on a timeout the kernel sets *err and still frees its
// TMEM.
constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128;
enum { EP_BIAS = 1, EP_RELU = 2, EP_ATOMIC = 4, EP_BF16 = 8, EP_TRANS = 16, EP_NOSTORE = 32 };

template <int BN>
constexpr int tc_stage_bytes() { return TC_BM * TC_BK * 2 + BN * TC_BK * 2; }
template <int BN>
constexpr int tc_smem_bytes() { return 1024 + 2 * tc_stage_bytes<BN>() + 64; }
template <int BN>
constexpr uint32_t tc_tmem_cols() { return BN <= 32 ? 32u : (uint32_t)BN; }

template <int BN>
__global__ void __launch_bounds__(TC_THREADS)
k_tc_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int M, int K,
          int k_per_split, float *__restrict__ out, int ldo, int ncols, __nv_bfloat16 *__restrict__ outb, int ldb,
          const float *__restrict__ bias, int ep, int *__restrict__ err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "N of a 128-row tcgen05 MMA");
    extern __shared__ uint8_t tc_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = tc::smem_addr(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;      // the swizzled tiles need 1024-byte alignment
    uint8_t *sm = tc_raw + (base - raw);
    constexpr int SA = TC_BM * TC_BK * 2, ST = tc_stage_bytes<BN>();
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + 2 * ST);   // [2] a stage's TMA bytes landed
    uint64_t *freed = full + 2;                                    // [2] a stage's MMAs are done
    uint64_t *done = full + 4;                                     // every MMA is done
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 5);
    const int m0 = blockIdx.x * TC_BM;
    const int k0 = blockIdx.y * k_per_split;
    const int k1 = min(K, k0 + k_per_split);
    const int nk = k1 > k0 ? (k1 - k0 + TC_BK - 1) / TC_BK : 0;
    constexpr unsigned long long kLimit = 1000000000ull;

    if (warp == 0) tc::tmem_alloc(tslot, tc_tmem_cols<BN>());
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) tc::mbar_init(full + i, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16(TC_BM, BN);
        int issued = 0, consumed = 0;
        bool ok = true;
        for (; issued < nk && issued < 2; ++issued) {
            const int s = issued & 1;
            tc::mbar_expect_tx(full + s, ST);
            tc::tma_load_2d(sm + s * ST, &mapA, full + s, k0 + issued * TC_BK, m0);
            tc::tma_load_2d(sm + s * ST + SA, &mapB, full + s, k0 + issued * TC_BK, 0);
        }
        for (int c = 0; c < nk; ++c) {
            const int s = c & 1;
            if (!(ok = tc::mbar_wait(full + s, (c >> 1) & 1, kLimit))) break;
            consumed = c + 1;
            tc::fence_after_sync();
            const int ksteps = (min(TC_BK, k1 - (k0 + c * TC_BK)) + 15) / 16;
            const uint32_t sa = base + s * ST, sb = sa + SA;
            for (int kk = 0; kk < ksteps; ++kk)
                tc::mma_bf16(tmem, tc::desc_k128(sa + 32 * kk), tc::desc_k128(sb + 32 * kk), idesc,
                             (c > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(freed + s);
            if (issued < nk) {   // refill this stage once its MMAs have read it
                if (!(ok = tc::mbar_wait(freed + s, (c >> 1) & 1, kLimit))) break;
                tc::mbar_expect_tx(full + s, ST);
                tc::tma_load_2d(sm + s * ST, &mapA, full + s, k0 + issued * TC_BK, m0);
                tc::tma_load_2d(sm + s * ST + SA, &mapB, full + s, k0 + issued * TC_BK, 0);
                ++issued;
            }
        }
        tc::mma_commit(done);
        if (!ok) {
            atomicExch(err, 1);
            // let copies still in flight land before the CTA leaves (bounded)
            for (int c = consumed; c < issued; ++c) (void)tc::mbar_wait(full + (c & 1), (c >> 1) & 1, kLimit);
        }
    }
    const bool fin = tc::mbar_wait(done, 0, kLimit);
    tc::fence_after_sync();
    if (!fin) {
        if (lane == 0) atomicExch(err, 2);
    } else if (nk > 0) {
        __syncwarp();   // tcgen05.ld is warp-collective
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row >= M) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = c0 + i;
                if (col >= ncols) break;
                float x = v[i];
                if (ep & EP_BIAS) x += bias[col];
                if (ep & EP_RELU) x = fmaxf(x, 0.f);
                const size_t o = (ep & EP_TRANS) ? (size_t)col * ldo + row : (size_t)row * ldo + col;
                if (ep & EP_ATOMIC) atomicAdd(out + o, x);
                else if (!(ep & EP_NOSTORE)) out[o] = x;
                if (ep & EP_BF16) outb[(size_t)row * ldb + col] = __float2bfloat16_rn(x);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, tc_tmem_cols<BN>());
}

// ------------------------------------------------------------ BF16 operands

// X [N x 16] FP32 -> Xb [N x 64] BF16 (columns 16..63 zero: the TMA box is
// 64 wide) and its transpose XT [16 x ldt].
__global__ void k_conv_x(const float *__restrict__ X, int N, __nv_bfloat16 *__restrict__ Xb) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)N * 64) return;
    const int r = (int)(e / 64), k = (int)(e % 64);
    Xb[e] = __float2bfloat16_rn(k < F ? X[(size_t)r * F + k] : 0.f);
}

// dst[c][r] = bf16(src[r][c]) for an FP32 [rows x cols] source (leading
// dimension lds) into a BF16 [cols x ldd] destination, through 32 x 32
// shared-memory tiles so that both sides are coalesced.
__global__ void k_transpose_bf16(const float *__restrict__ src, int lds, int rows, int cols,
                                 __nv_bfloat16 *__restrict__ dst, int ldd) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * lds + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[(size_t)c * ldd + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
    }
}

// FP32 [rows x cols] -> BF16, same layout
__global__ void k_to_bf16(const float *__restrict__ src, size_t count, __nv_bfloat16 *__restrict__ dst) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < count) dst[e] = __float2bfloat16_rn(src[e]);
}

// BF16 copies of the weights, in the K-major layouts the products read:
//   W1t [128 x 64]  = W1^T, K padded from 16 to 64 with zeros (layer 1)
//   W2t [128 x 256] = W2^T                                      (layer 2)
//   W2n [256 x 128] = W2                                        (dZ = dH2 W2^T)
//   W3t [16 x 128]  = W3^T, rows 8..15 zero                     (layer 3)
constexpr int WB_W1T = 0, WB_W2T = WB_W1T + H * 64, WB_W2N = WB_W2T + H * 2 * H, WB_W3T = WB_W2N + 2 * H * H,
              WB_TOTAL = WB_W3T + 16 * H;
__global__ void k_weights_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ wb) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < WB_TOTAL; e += gridDim.x * blockDim.x) {
        float v;
        if (e < WB_W2T) {
            const int j = (e - WB_W1T) / 64, f = (e - WB_W1T) % 64;
            v = f < F ? P[OFF_W1 + f * H + j] : 0.f;
        } else if (e < WB_W2N) {
            const int j = (e - WB_W2T) / (2 * H), i = (e - WB_W2T) % (2 * H);
            v = P[OFF_W2 + i * H + j];
        } else if (e < WB_W3T) {
            v = P[OFF_W2 + (e - WB_W2N)];
        } else {
            const int o = (e - WB_W3T) / H, k = (e - WB_W3T) % H;
            v = o < 8 ? P[OFF_W3 + k * 8 + o] : 0.f;
        }
        wb[e] = __float2bfloat16_rn(v);
    }
}

// ------------------------------------------------------------ fused inference

// The whole network for one instance in one launch: a cluster of up to
// eight CTAs of 128 threads (co-scheduled, with distributed shared memory),
// CTA r taking the 128-row tiles r, r + 8, ... Every product is a tcgen05
// MMA with operands in shared memory and FP32 accumulators in TMEM:
//   pass 1, per tile: X (TMA) * W1^T -> relu(+ b1) = H1; only the column
//     sums of H1 are kept (shared memory);
//   the cluster adds its CTAs' column sums (DSMEM) into the pooled context
//     c, which enters layer 2 as a bias: [H1 ; c] W2 = H1 W2_top +
//     c W2_bottom, so b2' = b2 + c W2_bottom is formed once per CTA (CUDA
//     cores, BF16 operands and FP32 sums, as the products round them);
//   pass 2, per tile: layer 1 again (one MMA), H1 written in BF16 into
//     shared memory in the swizzled K-major layout the next MMA reads;
//     H1 * W2_top^T -> relu(+ b2') = H2, written the same way;
//     H2 * W3^T + b3 = y (TMEM columns 128..143);
//   the cluster's largest y (DSMEM), then p_j = round((n+1) T (y_j - max y)):
//     the paper's sign with max 0 (a uniform shift changes no reduced cost).
// Shared memory (1024-aligned): W1^T 16 KB, W2_top^T 2 x 16 KB, W3^T
// 2 x 2 KB, X tile 16 KB, H1 tile 2 x 16 KB, H2 tile 2 x 16 KB. Every wait
// is bounded; on a timeout the kernel still passes every cluster barrier,
// frees its TMEM and sets *err.
constexpr int INF_W1 = 0, INF_W2 = INF_W1 + 16384, INF_W3 = INF_W2 + 32768, INF_X = INF_W3 + 4096,
              INF_H1 = INF_X + 16384, INF_H2 = INF_H1 + 32768, INF_BYTES = INF_H2 + 32768;
constexpr int INF_SMEM = 1024 + INF_BYTES + 2048;
constexpr int INF_CLUSTER = 8;

__device__ __forceinline__ int float_order(float x) {   // order-preserving float -> int
    const int i = __float_as_int(x);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float order_float(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// 16 BF16 values of row r (0..127), columns c0..c0+15 (c0 a multiple of
// 16), into a [128 x 128] K-major tile with the 128-byte swizzle: two
// 64-column halves of 16 KB; within a half, row r is 128 bytes and its
// 16-byte unit u sits at unit u ^ (r % 8).
__device__ __forceinline__ void store_swizzled(uint8_t *tile, int r, int c0, const uint32_t (&p)[8]) {
    const int half = c0 / 64, u = (c0 % 64) / 8;
    uint8_t *rowp = tile + half * 16384 + r * 128;
    *reinterpret_cast<uint4 *>(rowp + ((u ^ (r & 7)) * 16)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4 *>(rowp + (((u + 1) ^ (r & 7)) * 16)) = make_uint4(p[4], p[5], p[6], p[7]);
}

__global__ void __launch_bounds__(TC_THREADS)
k_infer(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW1,
        const __grid_constant__ CUtensorMap mapW2, const __grid_constant__ CUtensorMap mapW3,
        const float *__restrict__ P, const __nv_bfloat16 *__restrict__ wb, int n, const float *__restrict__ inst,
        float *__restrict__ Y, long long *__restrict__ prices, int *__restrict__ err) {
    extern __shared__ uint8_t in_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t raw = tc::smem_addr(in_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sm = in_raw + (base - raw);
    float *colsum = reinterpret_cast<float *>(sm + INF_BYTES);           // [128]
    float *bias2 = colsum + H;                                            // [128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(bias2 + H);             // weights, X, MMA
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 3);
    int *ymax = reinterpret_cast<int *>(tslot + 1);
    int *s_ok = ymax + 1;
    constexpr unsigned long long kLimit = 1000000000ull;
    const int rank = (int)tc::cluster_rank(), csize = (int)tc::cluster_size();
    const int tiles = (n + TC_BM - 1) / TC_BM;

    if (warp == 0) tc::tmem_alloc(tslot, 256);
    colsum[tid] = 0.f;
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) tc::mbar_init(bars + i, 1);
        *ymax = float_order(-INFINITY);
        *s_ok = 1;
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    bool ok = true;                 // thread 0's view
    uint32_t mph = 0, xph = 0;      // phases of the MMA and X barriers
    if (tid == 0) {
        tc::mbar_expect_tx(bars + 0, 16384 + 32768 + 4096);
        tc::tma_load_2d(sm + INF_W1, &mapW1, bars + 0, 0, 0);
        tc::tma_load_2d(sm + INF_W2, &mapW2, bars + 0, 0, 0);
        tc::tma_load_2d(sm + INF_W2 + 16384, &mapW2, bars + 0, 64, 0);
        tc::tma_load_2d(sm + INF_W3, &mapW3, bars + 0, 0, 0);
        tc::tma_load_2d(sm + INF_W3 + 2048, &mapW3, bars + 0, 64, 0);
        ok = tc::mbar_wait(bars + 0, 0, kLimit);
    }
    const float *b1 = P + OFF_B1, *b2 = P + OFF_B2, *b3 = P + OFF_B3;
    constexpr uint32_t id128 = tc::idesc_bf16(TC_BM, H), id16 = tc::idesc_bf16(TC_BM, 16);
    // thread 0: X tile t into shared memory, then layer 1 into TMEM columns 0..127
    auto layer1 = [&](int t) {
        if (ok) {
            tc::mbar_expect_tx(bars + 1, 16384);
            tc::tma_load_2d(sm + INF_X, &mapX, bars + 1, 0, t * TC_BM);
            ok = tc::mbar_wait(bars + 1, xph, kLimit);
            xph ^= 1;
        }
        if (ok) {
            tc::fence_after_sync();
            tc::mma_bf16(tmem, tc::desc_k128(base + INF_X), tc::desc_k128(base + INF_W1), id128, 0u);
        }
        tc::mma_commit(bars + 2);   // arrives at once when nothing was issued
    };
    // everyone: the MMAs committed last are done (bounded)
    auto wait_mma = [&]() {
        if (!tc::mbar_wait(bars + 2, mph, kLimit)) atomicExch(s_ok, 0);
        mph ^= 1;
        tc::fence_after_sync();
        __syncwarp();
    };
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;

    // pass 1: layer 1 and the column sums of H1
    for (int t = rank; t < tiles; t += csize) {
        if (tid == 0) layer1(t);
        wait_mma();
        const int row = t * TC_BM + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lanes + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = row < n ? fmaxf(v[i] + b1[c0 + i], 0.f) : 0.f;
            // sums of the 16 columns over the warp's 32 rows in 16 shuffles: each
            // step keeps half of the columns and adds the partner lane's sums of
            // them; lane l ends with column (l >> 1) & 15, twice
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const int off = 16 >> st, half = 8 >> st;
                const bool up = (lane & off) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const float send = up ? v[i] : v[i + half];
                    const float keep = up ? v[i + half] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            if ((lane & 1) == 0) atomicAdd(colsum + c0 + ((lane >> 1) & 15), v[0]);
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    // W2's bottom rows (c's weights, 32 KB) into the H1 buffer, which pass 2
    // fills only after they are used; completes on the X barrier
    if (tid == 0 && ok) {
        tc::mbar_expect_tx(bars + 1, (uint32_t)(H * H * 2));
        tc::bulk_load(sm + INF_H1, wb + WB_W2N + (size_t)H * H, (uint32_t)(H * H * 2), bars + 1);
    }
    // the pooled context: the cluster's column sums over n
    tc::cluster_sync();
    float c = 0.f;
    for (int q = 0; q < csize; ++q) c += tc::ld_cluster_f32(colsum + tid, (uint32_t)q);
    bias2[tid] = __bfloat162float(__float2bfloat16_rn(c / (float)n));   // c_i, as layer 2 rounds it
    __syncthreads();
    {   // b2'[j] = b2[j] + sum_i c_i W2[128 + i][j], W2's bottom rows staged in the H1 buffer
        if (tid == 0) {
            if (ok) ok = tc::mbar_wait(bars + 1, xph, kLimit);   // the bulk copy issued after pass 1
            xph ^= 1;
        }
        __syncthreads();
        const __nv_bfloat16 *w2s = reinterpret_cast<const __nv_bfloat16 *>(sm + INF_H1);
        float acc = b2[tid];
#pragma unroll 8
        for (int i = 0; i < H; ++i) acc += bias2[i] * __bfloat162float(w2s[i * H + tid]);
        __syncthreads();
        bias2[tid] = acc;
    }
    __syncthreads();

    // pass 2: layer 1 again, then layers 2 and 3
    for (int t = rank; t < tiles; t += csize) {
        if (tid == 0) layer1(t);
        wait_mma();
        const int r = warp * 32 + lane;   // row within the tile
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lanes + (uint32_t)c0, v);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 pr = __floats2bfloat162_rn(fmaxf(v[2 * i] + b1[c0 + 2 * i], 0.f),
                                                                 fmaxf(v[2 * i + 1] + b1[c0 + 2 * i + 1], 0.f));
                p[i] = *reinterpret_cast<const uint32_t *>(&pr);
            }
            store_swizzled(sm + INF_H1, r, c0, p);
        }
        tc::fence_proxy_async();   // written by this thread, read next by the MMA (async proxy)
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            if (ok)
                for (int ch = 0; ch < 2; ++ch)
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem, tc::desc_k128(base + INF_H1 + ch * 16384 + 32 * kk),
                                     tc::desc_k128(base + INF_W2 + ch * 16384 + 32 * kk), id128, (ch | kk) ? 1u : 0u);
            tc::mma_commit(bars + 2);
        }
        wait_mma();
#pragma unroll 1
        for (int c0 = 0; c0 < H; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lanes + (uint32_t)c0, v);
            uint32_t p[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 pr = __floats2bfloat162_rn(fmaxf(v[2 * i] + bias2[c0 + 2 * i], 0.f),
                                                                 fmaxf(v[2 * i + 1] + bias2[c0 + 2 * i + 1], 0.f));
                p[i] = *reinterpret_cast<const uint32_t *>(&pr);
            }
            store_swizzled(sm + INF_H2, r, c0, p);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            if (ok)
                for (int ch = 0; ch < 2; ++ch)
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem + 128, tc::desc_k128(base + INF_H2 + ch * 16384 + 32 * kk),
                                     tc::desc_k128(base + INF_W3 + ch * 2048 + 32 * kk), id16, (ch | kk) ? 1u : 0u);
            tc::mma_commit(bars + 2);
        }
        wait_mma();
        {
            float v[16];
            tc::tmem_ld16(tmem + lanes + 128u, v);
            const int row = t * TC_BM + r;
            const float y = v[0] + b3[0];
            int m = row < n ? float_order(y) : float_order(-INFINITY);
            if (row < n) Y[row] = y;
            m = __reduce_max_sync(0xffffffffu, m);
            if (lane == 0) atomicMax(ymax, m);
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    // the cluster's largest y, then the prices of this CTA's rows
    tc::cluster_sync();
    int mx = float_order(-INFINITY);
    for (int q = 0; q < csize; ++q) mx = max(mx, tc::ld_cluster_s32(ymax, (uint32_t)q));
    const double top = (double)order_float(mx), T = inst[0];
    for (int t = rank; t < tiles; t += csize) {
        const int row = t * TC_BM + tid;
        if (row < n) prices[row] = (long long)llround(((double)Y[row] - top) * T * (double)(n + 1));
    }
    if (tid == 0 && !ok) *s_ok = 0;
    __syncthreads();
    if (tid == 0 && !*s_ok) atomicExch(err, 1);
    // no CTA leaves while another may still read its shared memory
    tc::cluster_sync();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_free(tmem, 256);
}

// ------------------------------------------------------------ set pooling and glue

// ctx[i][:] = mean over the rows of segment i of H1 (seg: [I+1] row offsets).
__global__ void k_segment_mean(const float *__restrict__ Hm, const int *__restrict__ seg, float *__restrict__ ctx) {
    const int i = blockIdx.x, k = threadIdx.x;   // blockDim = H
    const int r0 = seg[i], r1 = seg[i + 1];
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += Hm[(size_t)r * H + k];
    ctx[(size_t)i * H + k] = r1 > r0 ? s / (float)(r1 - r0) : 0.f;
}

// Z[r] = [H1[r] ; ctx[segment of r]], in FP32 and in BF16 (layer 2's operand)
__global__ void k_concat(const float *__restrict__ H1, const float *__restrict__ ctx, const int *__restrict__ rowseg,
                         int N, float *__restrict__ Z, __nv_bfloat16 *__restrict__ Zb) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)N * 2 * H) return;
    const int r = (int)(e / (2 * H)), k = (int)(e % (2 * H));
    const float v = k < H ? H1[(size_t)r * H + k] : ctx[(size_t)rowseg[r] * H + (k - H)];
    Z[e] = v;
    Zb[e] = __float2bfloat16_rn(v);
}

// row -> segment index
__global__ void k_rowseg(const int *__restrict__ seg, int I, int *__restrict__ rowseg) {
    const int i = blockIdx.x;
    for (int r = seg[i] + threadIdx.x; r < seg[i + 1]; r += blockDim.x) rowseg[r] = i;
}

// Loss of one batch and dL/dy: per instance, the variance of the error
// d = y - t, L = (1/I) sum_i (1/n_i) sum_j (d_j - mean_i d)^2 (blind to a
// shift of y or t, as prices are); dL/dy_j = 2 (d_j - mean_i d) / (I n_i).
__global__ void k_loss_grad(const float *__restrict__ Y, int ldy, const float *__restrict__ tgt,
                            const int *__restrict__ seg, int I, float *__restrict__ dY, int lddy,
                            float *__restrict__ loss) {
    __shared__ float red[32];
    __shared__ float s_mean;
    const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = seg[i], r1 = seg[i + 1], n = r1 - r0;
    if (n == 0) return;
    float s = 0.f;
    for (int r = r0 + tid; r < r1; r += blockDim.x) s += Y[(size_t)r * ldy] - tgt[r];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (tid == 0) {
        float tt = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[w];
        s_mean = tt / (float)n;
    }
    __syncthreads();
    const float dbar = s_mean;
    float l = 0.f;
    for (int r = r0 + tid; r < r1; r += blockDim.x) {
        const float e = Y[(size_t)r * ldy] - tgt[r] - dbar;
        l += e * e;
        if (dY) dY[(size_t)r * lddy] = 2.f * e / ((float)I * (float)n);
    }
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    __syncthreads();
    if (lane == 0) red[warp] = l;
    __syncthreads();
    if (tid == 0 && loss) {
        float tt = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[w];
        atomicAdd(loss, tt / ((float)I * (float)n));
    }
}

// dH2 = (dy W3^T) * [h2 > 0]
__global__ void k_dh2(const float *__restrict__ dY, int lddy, const float *__restrict__ W3,
                      const float *__restrict__ H2, int N, float *__restrict__ dH2) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)N * H) return;
    const int r = (int)(e / H), k = (int)(e % H);
    dH2[e] = H2[e] > 0.f ? dY[(size_t)r * lddy] * W3[k * 8] : 0.f;
}

// dH1 = (dZ[:, :H] + (1/n_i) sum_{rows of i} dZ[:, H:]) * [h1 > 0]
__global__ void k_dh1(const float *__restrict__ dZ, const float *__restrict__ H1, const int *__restrict__ seg,
                      float *__restrict__ dH1) {
    const int i = blockIdx.x, k = threadIdx.x;   // blockDim = H
    const int r0 = seg[i], r1 = seg[i + 1];
    float s = 0.f;
    for (int r = r0; r < r1; ++r) s += dZ[(size_t)r * 2 * H + H + k];
    const float c = r1 > r0 ? s / (float)(r1 - r0) : 0.f;
    for (int r = r0; r < r1; ++r) {
        const size_t e = (size_t)r * H + k;
        dH1[e] = H1[e] > 0.f ? dZ[(size_t)r * 2 * H + k] + c : 0.f;
    }
}

// column sums of X [N x W] (ldx) accumulated into out[W] (bias gradients)
__global__ void k_colsum(const float *__restrict__ X, int ldx, int N, int W, float *__restrict__ out) {
    const int k = blockIdx.x * blockDim.y + threadIdx.y;
    if (k >= W) return;
    float s = 0.f;
    for (int r = threadIdx.x; r < N; r += blockDim.x) s += X[(size_t)r * ldx + k];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out + k, s);
}

// Adam on the parameter block (header entries are left alone).
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int count, float lr, float b1, float b2, float eps,
                       float c1, float c2, float wd) {
    const int i = LA_PRED_HEADER + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i] + wd * p[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------ host side

constexpr int kMaxDevices = 64;

struct PredWorkspace {
    size_t cap_n = 0;       // columns (features rows) capacity
    size_t cap_i = 0;       // instances capacity
    float *feats = nullptr, *H1 = nullptr, *Z = nullptr, *H2 = nullptr, *Y = nullptr;
    float *ctx = nullptr, *dY = nullptr, *dH2 = nullptr, *dZ = nullptr, *dH1 = nullptr;
    float *grad = nullptr, *loss = nullptr, *rowmin = nullptr, *part = nullptr, *colbuf = nullptr, *inst = nullptr;
    int *pop = nullptr, *seg = nullptr, *rowseg = nullptr;
    long long *prices = nullptr;   // la_solve_warm's predicted prices
    float *h_loss = nullptr;
    // BF16 operands of the tensor-core products (row-major [rows x K], or
    // transposed [K-dim x ldt] with ldt = cap_n rounded up to 64)
    __nv_bfloat16 *Xb = nullptr, *Zb = nullptr, *H2b = nullptr, *dH2b = nullptr;
    __nv_bfloat16 *XT = nullptr, *ZT = nullptr, *H2T = nullptr, *dYT = nullptr, *dH2T = nullptr, *dH1T = nullptr;
    __nv_bfloat16 *wb = nullptr;   // BF16 weight copies (k_weights_bf16)
    int *err = nullptr;            // set by a tensor-core kernel whose wait timed out
    int *h_err = nullptr;
    size_t ldt = 0;
    int num_sms = 0;
};

std::mutex g_pmu;
PredWorkspace g_pws[kMaxDevices];

template <class T>
bool grow(T *&p, size_t count) {
    cudaFree(p);
    p = nullptr;
    return cudaMalloc(&p, sizeof(T) * std::max<size_t>(count, 1)) == cudaSuccess;
}

la_status ensure_pws(PredWorkspace &w, size_t nrows, size_t ninst, int nmat) {
    if (!w.h_loss && cudaMallocHost(&w.h_loss, sizeof(float)) != cudaSuccess) return LA_ERR_NOMEM;
    if (!w.h_err && cudaMallocHost(&w.h_err, sizeof(int)) != cudaSuccess) return LA_ERR_NOMEM;
    if (!w.grad && !grow(w.grad, NPARAM)) return LA_ERR_NOMEM;
    if (!w.loss && !grow(w.loss, 1)) return LA_ERR_NOMEM;
    if (!w.inst && !grow(w.inst, 4)) return LA_ERR_NOMEM;
    if (!w.err && !grow(w.err, 1)) return LA_ERR_NOMEM;
    if (!w.wb && !grow(w.wb, WB_TOTAL)) return LA_ERR_NOMEM;
    if (nrows > w.cap_n) {
        const size_t c = std::max(nrows, (size_t)1024);
        const size_t t = (c + 63) / 64 * 64;
        if (!grow(w.feats, c * F) || !grow(w.H1, c * H) || !grow(w.Z, c * 2 * H) || !grow(w.H2, c * H) ||
            !grow(w.Y, c * 8) || !grow(w.dY, c * 8) || !grow(w.dH2, c * H) || !grow(w.dZ, c * 2 * H) ||
            !grow(w.dH1, c * H) || !grow(w.rowseg, c) || !grow(w.rowmin, c) || !grow(w.pop, c) ||
            !grow(w.colbuf, c * 5) || !grow(w.prices, c) || !grow(w.Xb, c * 64) || !grow(w.Zb, c * 2 * H) ||
            !grow(w.H2b, c * H) || !grow(w.dH2b, c * H) || !grow(w.XT, F * t) || !grow(w.ZT, 2 * H * t) ||
            !grow(w.H2T, H * t) || !grow(w.dYT, 8 * t) || !grow(w.dH2T, H * t) || !grow(w.dH1T, H * t))
            return LA_ERR_NOMEM;
        w.cap_n = c;
        w.ldt = t;
        // column-pass partials for a single matrix of this size
        if (!grow(w.part, c * 5 * (size_t)kColBlocks)) return LA_ERR_NOMEM;
    }
    if (ninst + 1 > w.cap_i) {
        const size_t c = std::max(ninst + 1, (size_t)64);
        if (!grow(w.ctx, c * H) || !grow(w.seg, c)) return LA_ERR_NOMEM;
        w.cap_i = c;
    }
    (void)nmat;
    return LA_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tensor map of a K-major BF16 matrix [rows x k] with row pitch ld
// elements (a multiple of 8): boxes of 64 x box_rows, 128-byte swizzle,
// zeros outside the matrix.
bool kmajor_map(CUtensorMap *m, const __nv_bfloat16 *ptr, int k, int rows, size_t ld, int box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || k <= 0 || rows <= 0 || (ld * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M x N] = A[M x K] * B[N x K]^T on the tensor cores (k_tc_gemm): A with
// row pitch lda, B with row pitch ldbm (elements), split over K in `splits`
// parts (EP_ATOMIC then adds the partial products).
template <int BN>
cudaError_t tc_gemm(cudaStream_t s, const __nv_bfloat16 *A, size_t lda, const __nv_bfloat16 *B, size_t ldbm,
                    int bn_rows, int M, int K, int splits, float *out, int ldo, int ncols, __nv_bfloat16 *outb,
                    int ldb, const float *bias, int ep, int *err, int kext = 0) {
    // kext: the stored K extent when the rows are padded beyond K (zeros)
    CUtensorMap ma, mb;
    const int ke = std::max(K, kext);
    if (!kmajor_map(&ma, A, ke, M, lda, TC_BM) || !kmajor_map(&mb, B, ke, bn_rows, ldbm, BN))
        return cudaErrorInvalidValue;
    const int chunks = (K + TC_BK - 1) / TC_BK;
    splits = std::max(1, std::min(splits, chunks));
    const int cps = (chunks + splits - 1) / splits;   // chunks per split; no split is left empty
    splits = (chunks + cps - 1) / cps;
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc_smem_bytes<BN>());
    if (e != cudaSuccess) return e;
    dim3 grid((M + TC_BM - 1) / TC_BM, splits);
    k_tc_gemm<BN><<<grid, TC_THREADS, tc_smem_bytes<BN>(), s>>>(ma, mb, M, K, cps * TC_BK, out, ldo, ncols, outb, ldb,
                                                                 bias, ep, err);
    return cudaGetLastError();
}

// split count for a product whose K is the row count N (weight gradients)
int k_splits(int N, int mtiles, int num_sms) {
    return std::max(1, std::min((N + TC_BK - 1) / TC_BK / 2, 2 * num_sms / std::max(1, mtiles)));
}

inline void transpose(cudaStream_t s, const float *src, int lds, int rows, int cols, __nv_bfloat16 *dst, size_t ldd) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(src, lds, rows, cols, dst, (int)ldd);
}

// features of one n x n matrix into feats (n rows of F) and inst
la_status features_one(cudaStream_t s, const int32_t *C, int n, PredWorkspace &w, float *feats, float *inst,
                       __nv_bfloat16 *xb = nullptr) {
    if (cudaMemsetAsync(w.pop, 0, sizeof(int) * n, s) != cudaSuccess) return LA_ERR_CUDA;
    k_row_stats<<<(n * 32 + 255) / 256, 256, 0, s>>>(C, n, w.rowmin, w.pop);
    const int rpb = std::max(16, (n + kColBlocks - 1) / kColBlocks);   // at most kColBlocks row blocks
    const int rb = (n + rpb - 1) / rpb;
    dim3 grid((n + 127) / 128, rb);
    k_col_stats<<<grid, 128, 0, s>>>(C, n, w.rowmin, w.part, rpb);
    k_features<<<1, 1024, 0, s>>>(n, rb, w.part, w.pop, w.colbuf, feats, inst, xb);
    return cudaGetLastError() == cudaSuccess ? LA_OK : LA_ERR_CUDA;
}

// forward over N rows in I segments; Y [N x 8] (column 0 is the output)
cudaError_t forward(cudaStream_t s, const float *P, const float *X, int N, int I, const int *seg, PredWorkspace &w) {
    cudaError_t e;
    k_weights_bf16<<<64, 256, 0, s>>>(P, w.wb);
    k_conv_x<<<(unsigned)(((size_t)N * 64 + 255) / 256), 256, 0, s>>>(X, N, w.Xb);
    k_rowseg<<<I, 256, 0, s>>>(seg, I, w.rowseg);
    // layer 1: H1 = relu(X W1 + b1)   (K = 16 real features)
    if ((e = tc_gemm<128>(s, w.Xb, 64, w.wb + WB_W1T, 64, H, N, F, 1, w.H1, H, H, nullptr, 0, P + OFF_B1,
                          EP_BIAS | EP_RELU, w.err, 64)) != cudaSuccess)
        return e;
    k_segment_mean<<<I, H, 0, s>>>(w.H1, seg, w.ctx);
    k_concat<<<(unsigned)(((size_t)N * 2 * H + 255) / 256), 256, 0, s>>>(w.H1, w.ctx, w.rowseg, N, w.Z, w.Zb);
    // layer 2: H2 = relu(Z W2 + b2), also in BF16 for layer 3
    if ((e = tc_gemm<128>(s, w.Zb, 2 * H, w.wb + WB_W2T, 2 * H, H, N, 2 * H, 1, w.H2, H, H, w.H2b, H, P + OFF_B2,
                          EP_BIAS | EP_RELU | EP_BF16, w.err)) != cudaSuccess)
        return e;
    // layer 3: Y = H2 W3 + b3 (8 outputs; the MMA's N is 16)
    if ((e = tc_gemm<16>(s, w.H2b, H, w.wb + WB_W3T, H, 16, N, H, 1, w.Y, 8, 8, nullptr, 0, P + OFF_B3, EP_BIAS,
                         w.err)) != cudaSuccess)
        return e;
    return cudaGetLastError();
}

// backward from dY into w.grad (zeroed here)
cudaError_t backward(cudaStream_t s, const float *P, const float *X, int N, int I, const int *seg, PredWorkspace &w,
                     int num_sms) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.grad, 0, sizeof(float) * NPARAM, s)) != cudaSuccess) return e;
    const size_t ldt = w.ldt;
    // layer 3: dW3 = H2^T dY, db3 = sum dY
    transpose(s, w.H2, H, N, H, w.H2T, ldt);
    transpose(s, w.dY, 8, N, 8, w.dYT, ldt);
    if ((e = tc_gemm<16>(s, w.H2T, ldt, w.dYT, ldt, 8, H, N, k_splits(N, 1, num_sms), w.grad + OFF_W3, 8, 8,
                         nullptr, 0, nullptr, EP_ATOMIC, w.err)) != cudaSuccess)
        return e;
    k_colsum<<<1, dim3(32, 8), 0, s>>>(w.dY, 8, N, 8, w.grad + OFF_B3);
    k_dh2<<<(unsigned)(((size_t)N * H + 255) / 256), 256, 0, s>>>(w.dY, 8, P + OFF_W3, w.H2, N, w.dH2);
    // layer 2: dW2 = Z^T dH2, db2, dZ = dH2 W2^T
    transpose(s, w.Z, 2 * H, N, 2 * H, w.ZT, ldt);
    transpose(s, w.dH2, H, N, H, w.dH2T, ldt);
    k_to_bf16<<<(unsigned)(((size_t)N * H + 255) / 256), 256, 0, s>>>(w.dH2, (size_t)N * H, w.dH2b);
    if ((e = tc_gemm<128>(s, w.ZT, ldt, w.dH2T, ldt, H, 2 * H, N, k_splits(N, 2, num_sms), w.grad + OFF_W2, H, H,
                          nullptr, 0, nullptr, EP_ATOMIC, w.err)) != cudaSuccess)
        return e;
    k_colsum<<<H / 8, dim3(32, 8), 0, s>>>(w.dH2, H, N, H, w.grad + OFF_B2);
    if ((e = tc_gemm<256>(s, w.dH2b, H, w.wb + WB_W2N, H, 2 * H, N, H, 1, w.dZ, 2 * H, 2 * H, nullptr, 0, nullptr, 0,
                          w.err)) != cudaSuccess)
        return e;
    // pooling and layer 1: dW1^T = dH1^T X (stored transposed into W1's slots)
    k_dh1<<<I, H, 0, s>>>(w.dZ, w.H1, seg, w.dH1);
    transpose(s, w.dH1, H, N, H, w.dH1T, ldt);
    transpose(s, X, F, N, F, w.XT, ldt);
    if ((e = tc_gemm<16>(s, w.dH1T, ldt, w.XT, ldt, F, H, N, k_splits(N, 1, num_sms), w.grad + OFF_W1, H, F, nullptr,
                         0, nullptr, EP_ATOMIC | EP_TRANS, w.err)) != cudaSuccess)
        return e;
    k_colsum<<<H / 8, dim3(32, 8), 0, s>>>(w.dH1, H, N, H, w.grad + OFF_B1);
    return cudaGetLastError();
}

bool header_ok(const float *h_params_head) {
    return h_params_head[0] == LA_PRED_MAGIC && h_params_head[1] == 1.0f && h_params_head[2] == (float)F &&
           h_params_head[3] == (float)H;
}

}  // namespace

#define LA_PCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

static la_status get_ws(PredWorkspace *&w, size_t nrows, size_t ninst) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    w = &g_pws[dev];
    if (!w->num_sms && cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return LA_ERR_CUDA;
    if (!encode_tiled()) return LA_ERR_CUDA;   // the driver offers no TMA tensor maps
    return ensure_pws(*w, nrows, ninst, 1);
}

// The tensor-core kernels' error flag: cleared before a call's kernels,
// read after them (LA_ERR_INTERNAL if a bounded wait gave up).
static la_status clear_err(PredWorkspace &w, cudaStream_t s) {
    return cudaMemsetAsync(w.err, 0, sizeof(int), s) == cudaSuccess ? LA_OK : LA_ERR_CUDA;
}
static la_status read_err(PredWorkspace &w, cudaStream_t s) {
    if (cudaMemcpyAsync(w.h_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LA_ERR_CUDA;
    return *w.h_err ? LA_ERR_INTERNAL : LA_OK;
}

static la_status check_header(const float *params, cudaStream_t s) {
    float head[4];
    if (cudaMemcpyAsync(head, params, sizeof(head), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LA_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LA_ERR_CUDA;
    return header_ok(head) ? LA_OK : LA_ERR_INVALID;
}

extern "C" {

int32_t la_predictor_param_count(void) { return NPARAM; }

la_status la_features(const int32_t *cost, int32_t n, void *stream, float *feats_out, float *inst_out) {
    if (n <= 0 || !cost || !feats_out) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_pmu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PredWorkspace *w = nullptr;
    if (la_status e = get_ws(w, n, 1)) return e;
    if (la_status e = features_one(s, cost, n, *w, feats_out, inst_out ? inst_out : w->inst)) return e;
    LA_PCK(cudaStreamSynchronize(s));
    return LA_OK;
}

la_status la_predictor_forward(const float *params, const float *feats, const int32_t *seg, int32_t I, int32_t N,
                               void *stream, float *y_out) {
    if (!params || !feats || !seg || !y_out || I <= 0 || N <= 0) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_pmu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PredWorkspace *w = nullptr;
    if (la_status e = get_ws(w, N, I)) return e;
    if (la_status e = clear_err(*w, s)) return e;
    LA_PCK(forward(s, params, feats, N, I, seg, *w));
    LA_PCK(cudaMemcpy2DAsync(y_out, sizeof(float), w->Y, 8 * sizeof(float), sizeof(float), N,
                             cudaMemcpyDeviceToDevice, s));
    return read_err(*w, s);
}

la_status la_predictor_train_step(float *params, float *adam_m, float *adam_v, const float *feats,
                                  const float *targets, const int32_t *seg, int32_t I, int32_t N, int32_t step,
                                  float lr, float weight_decay, void *stream, float *grad_out,
                                  float *loss_out) {
    if (!params || !feats || !targets || !seg || I <= 0 || N <= 0 || step < 1) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_pmu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PredWorkspace *w = nullptr;
    if (la_status e = get_ws(w, N, I)) return e;
    if (la_status e = clear_err(*w, s)) return e;
    LA_PCK(cudaMemsetAsync(w->loss, 0, sizeof(float), s));
    LA_PCK(forward(s, params, feats, N, I, seg, *w));
    LA_PCK(cudaMemsetAsync(w->dY, 0, sizeof(float) * 8 * (size_t)N, s));
    k_loss_grad<<<I, 256, 0, s>>>(w->Y, 8, targets, seg, I, w->dY, 8, w->loss);
    LA_PCK(backward(s, params, feats, N, I, seg, *w, w->num_sms));
    if (grad_out) LA_PCK(cudaMemcpyAsync(grad_out, w->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s));
    if (adam_m && adam_v && lr > 0.f) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, w->grad, adam_m, adam_v, NPARAM, lr, b1, b2, 1e-8f,
                                                   c1, c2, weight_decay);
    }
    LA_PCK(cudaMemcpyAsync(w->h_loss, w->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    if (la_status e = read_err(*w, s)) return e;
    if (loss_out) *loss_out = *w->h_loss;
    return LA_OK;
}

la_status la_predict_prices_ex(const int32_t *cost, int32_t n, const void *weights, void *stream,
                               int64_t *prices_out, int64_t *eps0_out) {
    if (n < 0 || !weights || !prices_out || (n > 0 && !cost)) return LA_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float *P = static_cast<const float *>(weights);
    if (la_status e = check_header(P, s)) return e;
    if (n == 0) {
        if (eps0_out) *eps0_out = 1;
        return LA_OK;
    }
    std::lock_guard<std::mutex> lock(g_pmu);
    PredWorkspace *w = nullptr;
    if (la_status e = get_ws(w, n, 1)) return e;
    if (la_status e = clear_err(*w, s)) return e;
    // features (three launches; the last also writes layer 1's BF16 operand),
    // the BF16 weights, then the whole network and the price rounding in one
    // launch (k_infer)
    if (la_status e = features_one(s, cost, n, *w, w->feats, w->inst, w->Xb)) return e;
    k_weights_bf16<<<64, 256, 0, s>>>(P, w->wb);
    CUtensorMap mx, mw1, mw2, mw3;
    if (!kmajor_map(&mx, w->Xb, 64, n, 64, TC_BM) || !kmajor_map(&mw1, w->wb + WB_W1T, 64, H, 64, TC_BM) ||
        !kmajor_map(&mw2, w->wb + WB_W2T, 2 * H, H, 2 * H, TC_BM) || !kmajor_map(&mw3, w->wb + WB_W3T, H, 16, H, 16))
        return LA_ERR_CUDA;
    LA_PCK(cudaFuncSetAttribute(k_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, INF_SMEM));
    {   // one cluster: up to eight CTAs, each taking every eighth 128-row tile
        const int tiles = (n + TC_BM - 1) / TC_BM;
        const unsigned cl = (unsigned)std::min(INF_CLUSTER, tiles);
        cudaLaunchConfig_t cfg;
        std::memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = INF_SMEM;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        LA_PCK(cudaLaunchKernelEx(&cfg, k_infer, mx, mw1, mw2, mw3, P, (const __nv_bfloat16 *)w->wb, n,
                                  (const float *)w->inst, w->Y, reinterpret_cast<long long *>(prices_out), w->err));
    }
    float inst_h[2] = {0, 0}, calib[2] = {0, 0};
    LA_PCK(cudaMemcpyAsync(inst_h, w->inst, sizeof(inst_h), cudaMemcpyDeviceToHost, s));
    LA_PCK(cudaMemcpyAsync(calib, P + 4, sizeof(calib), cudaMemcpyDeviceToHost, s));
    if (la_status e = read_err(*w, s)) return e;
    if (eps0_out) {
        // eps0 = (n+1) * T * (calibrated error quantile), at least 1
        const double e = (double)(n + 1) * (double)inst_h[0] * (double)calib[0];
        *eps0_out = (int64_t)std::max(1.0, std::ceil(e));
    }
    return LA_OK;
}

la_status la_predict_prices(const int32_t *cost, int32_t n, const void *weights, void *stream,
                            int64_t *prices_out) {
    return la_predict_prices_ex(cost, n, weights, stream, prices_out, nullptr);
}

la_status la_solve_warm(const int32_t *cost, int32_t n, const void *weights, void *stream, int32_t *match_out,
                        int64_t *cost_out, la_stats *stats_out) {
    if (n < 0 || !weights || !cost_out || (n > 0 && !cost)) return LA_ERR_INVALID;
    if (n <= 1) return la_solve_ex(cost, n, nullptr, stream, match_out, cost_out, stats_out);
    int64_t *prices = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        std::lock_guard<std::mutex> lock(g_pmu);
        PredWorkspace *w = nullptr;
        if (la_status e = get_ws(w, n, 1)) return e;
        prices = reinterpret_cast<int64_t *>(w->prices);
    }
    int64_t eps0 = 0;
    if (la_status e = la_predict_prices_ex(cost, n, weights, stream, prices, &eps0)) return e;
    la_options opt;
    std::memset(&opt, 0, sizeof(opt));
    opt.init_prices = prices;
    opt.eps0 = eps0;
    // From predicted prices the phases that remain are the ones below a cost
    // unit, where bids fight over equal costs; on large instances smaller eps
    // steps there measured faster (geometric n = 8192: alpha 4 about 1.25x
    // faster than 10), on small ones the default is (n = 1024: 1.3x).
    opt.alpha = n >= 4096 ? 4 : 0;
    (void)s;
    return la_solve_ex(cost, n, &opt, stream, match_out, cost_out, stats_out);
}

}  // extern "C"
