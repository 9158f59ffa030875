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
// Every matrix product runs on the tensor cores: BF16 operands staged in
// shared memory, mma.sync m16n8k16, FP32 accumulation and FP32 storage.
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

namespace {

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
           float *__restrict__ colbuf, float *__restrict__ feats, float *__restrict__ inst) {
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
}

// ------------------------------------------------------------ GEMM on tensor cores

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

enum { EPI_STORE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_ATOMIC = 3 };

// C[M x N] (op)= op(A)[M x K] * op(B)[K x N], FP32 in global memory.
// op(A)[m][k] = transA ? A[k * lda + m] : A[m * lda + k]; same for B.
// Block tile 64 x 64, K step 32, 4 warps (each 16 rows x 64 columns).
// Operands are rounded to BF16 when staged; accumulation is FP32.
// gridDim.z splits K (EPI_ATOMIC adds partial products into C).
constexpr int TM = 64, TN = 64, TK = 32;

__global__ void __launch_bounds__(128)
k_gemm(const float *__restrict__ A, int lda, int transA, const float *__restrict__ B, int ldb, int transB,
       float *__restrict__ Cout, int ldc, int M, int N, int K, int epi, const float *__restrict__ bias,
       int k_per_split) {
    __shared__ uint32_t sA[TM][TK / 2 + 4];     // bf16 pairs along k
    __shared__ uint32_t sB[TN][TK / 2 + 4];     // B stored n-major: pairs along k
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int kbeg = blockIdx.z * k_per_split;
    const int kend = min(K, kbeg + k_per_split);
    const int g = lane >> 2, t = lane & 3;
    float acc[8][4];
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        // stage A tile [64 x 32] and B tile [32 x 64] as bf16 pairs
        for (int e = tid; e < TM * (TK / 2); e += 128) {
            const int r = e / (TK / 2), kp = e % (TK / 2);
            const int m = m0 + r, k = k0 + 2 * kp;
            float x0 = 0.f, x1 = 0.f;
            if (m < M) {
                if (k < kend) x0 = transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
                if (k + 1 < kend) x1 = transA ? A[(size_t)(k + 1) * lda + m] : A[(size_t)m * lda + k + 1];
            }
            sA[r][kp] = pack_bf16x2(x0, x1);
        }
        for (int e = tid; e < TN * (TK / 2); e += 128) {
            const int c = e / (TK / 2), kp = e % (TK / 2);
            const int nn = n0 + c, k = k0 + 2 * kp;
            float x0 = 0.f, x1 = 0.f;
            if (nn < N) {
                if (k < kend) x0 = transB ? B[(size_t)nn * ldb + k] : B[(size_t)k * ldb + nn];
                if (k + 1 < kend) x1 = transB ? B[(size_t)nn * ldb + k + 1] : B[(size_t)(k + 1) * ldb + nn];
            }
            sB[c][kp] = pack_bf16x2(x0, x1);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TK / 16; ++ks) {
            const int kb = ks * 8;   // in pairs
            uint32_t a[4];
            const int r = warp * 16 + g;
            a[0] = sA[r][kb + t];
            a[1] = sA[r + 8][kb + t];
            a[2] = sA[r][kb + 4 + t];
            a[3] = sA[r + 8][kb + 4 + t];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2];
                b[0] = sB[nt * 8 + g][kb + t];
                b[1] = sB[nt * 8 + g][kb + 4 + t];
                mma_bf16(acc[nt], a, b);
            }
        }
        __syncthreads();
    }
    // epilogue: acc[nt][0..1] -> row g, cols 2t, 2t+1; acc[nt][2..3] -> row g+8
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int m = m0 + warp * 16 + g + 8 * h;
            if (m >= M) continue;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int nn = n0 + nt * 8 + 2 * t + c;
                if (nn >= N) continue;
                float v = acc[nt][2 * h + c];
                float *dst = Cout + (size_t)m * ldc + nn;
                if (epi == EPI_ATOMIC) {
                    atomicAdd(dst, v);
                } else {
                    if (epi == EPI_BIAS_RELU || epi == EPI_BIAS) v += bias[nn];
                    if (epi == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
                    *dst = v;
                }
            }
        }
    }
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

// Z[r] = [H1[r] ; ctx[segment of r]]
__global__ void k_concat(const float *__restrict__ H1, const float *__restrict__ ctx, const int *__restrict__ rowseg,
                         int N, float *__restrict__ Z) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)N * 2 * H) return;
    const int r = (int)(e / (2 * H)), k = (int)(e % (2 * H));
    Z[e] = k < H ? H1[(size_t)r * H + k] : ctx[(size_t)rowseg[r] * H + (k - H)];
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

// prices_out[j] = round(-(n+1) * (T * y_j)) shifted so that max = 0 (paper
// sign; a uniform shift of all prices changes nothing).
__global__ void k_prices(const float *__restrict__ Y, int ldy, int n, const float *__restrict__ inst,
                         long long *__restrict__ prices) {
    __shared__ float red[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float mx = -INFINITY;
    for (int j = tid; j < n; j += blockDim.x) mx = fmaxf(mx, Y[(size_t)j * ldy]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        float t = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
        red[0] = t;
    }
    __syncthreads();
    const double T = inst[0], top = red[0];
    for (int j = tid; j < n; j += blockDim.x) {
        const double v = ((double)Y[(size_t)j * ldy] - top) * T;   // <= 0, cost units
        prices[j] = (long long)llround(v * (double)(n + 1));
    }
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
    if (!w.grad && !grow(w.grad, NPARAM)) return LA_ERR_NOMEM;
    if (!w.loss && !grow(w.loss, 1)) return LA_ERR_NOMEM;
    if (!w.inst && !grow(w.inst, 4)) return LA_ERR_NOMEM;
    if (nrows > w.cap_n) {
        const size_t c = std::max(nrows, (size_t)1024);
        if (!grow(w.feats, c * F) || !grow(w.H1, c * H) || !grow(w.Z, c * 2 * H) || !grow(w.H2, c * H) ||
            !grow(w.Y, c * 8) || !grow(w.dY, c * 8) || !grow(w.dH2, c * H) || !grow(w.dZ, c * 2 * H) ||
            !grow(w.dH1, c * H) || !grow(w.rowseg, c) || !grow(w.rowmin, c) || !grow(w.pop, c) ||
            !grow(w.colbuf, c * 5) || !grow(w.prices, c))
            return LA_ERR_NOMEM;
        w.cap_n = c;
        // column-pass partials for a single matrix of this size
        if (!grow(w.part, c * 5 * (size_t)((c + 255) / 256))) return LA_ERR_NOMEM;
    }
    if (ninst + 1 > w.cap_i) {
        const size_t c = std::max(ninst + 1, (size_t)64);
        if (!grow(w.ctx, c * H) || !grow(w.seg, c)) return LA_ERR_NOMEM;
        w.cap_i = c;
    }
    (void)nmat;
    return LA_OK;
}

cudaError_t gemm(cudaStream_t s, const float *A, int lda, int transA, const float *B, int ldb, int transB,
                 float *C, int ldc, int M, int N, int K, int epi, const float *bias, int splits = 1) {
    splits = std::max(1, std::min(splits, (K + TK - 1) / TK));
    int kps = (K + splits - 1) / splits;
    kps = ((kps + TK - 1) / TK) * TK;
    splits = (K + kps - 1) / kps;
    dim3 grid((M + TM - 1) / TM, (N + TN - 1) / TN, splits);
    k_gemm<<<grid, 128, 0, s>>>(A, lda, transA, B, ldb, transB, C, ldc, M, N, K, epi, bias, kps);
    return cudaGetLastError();
}

// features of one n x n matrix into feats (n rows of F) and inst
la_status features_one(cudaStream_t s, const int32_t *C, int n, PredWorkspace &w, float *feats, float *inst) {
    if (cudaMemsetAsync(w.pop, 0, sizeof(int) * n, s) != cudaSuccess) return LA_ERR_CUDA;
    k_row_stats<<<(n * 32 + 255) / 256, 256, 0, s>>>(C, n, w.rowmin, w.pop);
    const int rpb = 256;
    const int rb = (n + rpb - 1) / rpb;
    dim3 grid((n + 127) / 128, rb);
    k_col_stats<<<grid, 128, 0, s>>>(C, n, w.rowmin, w.part, rpb);
    k_features<<<1, 1024, 0, s>>>(n, rb, w.part, w.pop, w.colbuf, feats, inst);
    return cudaGetLastError() == cudaSuccess ? LA_OK : LA_ERR_CUDA;
}

// forward over N rows in I segments; Y [N x 8] (column 0 is the output)
cudaError_t forward(cudaStream_t s, const float *P, const float *X, int N, int I, const int *seg, PredWorkspace &w) {
    cudaError_t e;
    k_rowseg<<<I, 256, 0, s>>>(seg, I, w.rowseg);
    if ((e = gemm(s, X, F, 0, P + OFF_W1, H, 0, w.H1, H, N, H, F, EPI_BIAS_RELU, P + OFF_B1)) != cudaSuccess) return e;
    k_segment_mean<<<I, H, 0, s>>>(w.H1, seg, w.ctx);
    k_concat<<<(unsigned)(((size_t)N * 2 * H + 255) / 256), 256, 0, s>>>(w.H1, w.ctx, w.rowseg, N, w.Z);
    if ((e = gemm(s, w.Z, 2 * H, 0, P + OFF_W2, H, 0, w.H2, H, N, H, 2 * H, EPI_BIAS_RELU, P + OFF_B2)) != cudaSuccess) return e;
    if ((e = gemm(s, w.H2, H, 0, P + OFF_W3, 8, 0, w.Y, 8, N, 8, H, EPI_BIAS, P + OFF_B3)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// backward from dY into w.grad (zeroed here)
cudaError_t backward(cudaStream_t s, const float *P, const float *X, int N, int I, const int *seg, PredWorkspace &w) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.grad, 0, sizeof(float) * NPARAM, s)) != cudaSuccess) return e;
    const int splits = std::max(1, std::min(64, N / 1024));
    // layer 3: dW3 = H2^T dY, db3 = sum dY
    if ((e = gemm(s, w.H2, H, 1, w.dY, 8, 0, w.grad + OFF_W3, 8, H, 8, N, EPI_ATOMIC, nullptr, splits)) != cudaSuccess) return e;
    k_colsum<<<1, dim3(32, 8), 0, s>>>(w.dY, 8, N, 8, w.grad + OFF_B3);
    k_dh2<<<(unsigned)(((size_t)N * H + 255) / 256), 256, 0, s>>>(w.dY, 8, P + OFF_W3, w.H2, N, w.dH2);
    // layer 2: dW2 = Z^T dH2, db2, dZ = dH2 W2^T
    if ((e = gemm(s, w.Z, 2 * H, 1, w.dH2, H, 0, w.grad + OFF_W2, H, 2 * H, H, N, EPI_ATOMIC, nullptr, splits)) != cudaSuccess) return e;
    k_colsum<<<H / 8, dim3(32, 8), 0, s>>>(w.dH2, H, N, H, w.grad + OFF_B2);
    if ((e = gemm(s, w.dH2, H, 0, P + OFF_W2, H, 1, w.dZ, 2 * H, N, 2 * H, H, EPI_STORE, nullptr)) != cudaSuccess) return e;
    // pooling and layer 1
    k_dh1<<<I, H, 0, s>>>(w.dZ, w.H1, seg, w.dH1);
    if ((e = gemm(s, X, F, 1, w.dH1, H, 0, w.grad + OFF_W1, H, F, H, N, EPI_ATOMIC, nullptr, splits)) != cudaSuccess) return e;
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
    return ensure_pws(*w, nrows, ninst, 1);
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
    LA_PCK(forward(s, params, feats, N, I, seg, *w));
    LA_PCK(cudaMemcpy2DAsync(y_out, sizeof(float), w->Y, 8 * sizeof(float), sizeof(float), N,
                             cudaMemcpyDeviceToDevice, s));
    LA_PCK(cudaStreamSynchronize(s));
    return LA_OK;
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
    LA_PCK(cudaMemsetAsync(w->loss, 0, sizeof(float), s));
    LA_PCK(forward(s, params, feats, N, I, seg, *w));
    LA_PCK(cudaMemsetAsync(w->dY, 0, sizeof(float) * 8 * (size_t)N, s));
    k_loss_grad<<<I, 256, 0, s>>>(w->Y, 8, targets, seg, I, w->dY, 8, w->loss);
    LA_PCK(backward(s, params, feats, N, I, seg, *w));
    if (grad_out) LA_PCK(cudaMemcpyAsync(grad_out, w->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s));
    if (adam_m && adam_v && lr > 0.f) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, w->grad, adam_m, adam_v, NPARAM, lr, b1, b2, 1e-8f,
                                                   c1, c2, weight_decay);
    }
    LA_PCK(cudaMemcpyAsync(w->h_loss, w->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    LA_PCK(cudaStreamSynchronize(s));
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
    if (la_status e = features_one(s, cost, n, *w, w->feats, w->inst)) return e;
    const int seg_h[2] = {0, n};
    LA_PCK(cudaMemcpyAsync(w->seg, seg_h, sizeof(seg_h), cudaMemcpyHostToDevice, s));
    LA_PCK(forward(s, P, w->feats, n, 1, w->seg, *w));
    k_prices<<<1, 1024, 0, s>>>(w->Y, 8, n, w->inst, reinterpret_cast<long long *>(prices_out));
    LA_PCK(cudaGetLastError());
    float inst_h[2] = {0, 0}, calib[2] = {0, 0};
    LA_PCK(cudaMemcpyAsync(inst_h, w->inst, sizeof(inst_h), cudaMemcpyDeviceToHost, s));
    LA_PCK(cudaMemcpyAsync(calib, P + 4, sizeof(calib), cudaMemcpyDeviceToHost, s));
    LA_PCK(cudaStreamSynchronize(s));
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
    (void)s;
    return la_solve_ex(cost, n, &opt, stream, match_out, cost_out, stats_out);
}

}  // extern "C"
