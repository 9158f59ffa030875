// la_maxflow_grid: maximum s-t flow and a minimum cut of a 4-connected grid
// graph with terminal arcs (the graph-cut form of the paper's Sect. 4
// problem), by the lock-free push-relabel method of Hong (Algorithm 4.5)
// run in cycles with a global relabel between them (Algorithm 4.8, the
// hybrid scheme of Hong and He, with the gap step of the paper's own
// implementation).
//
//  * Init (Algorithm 4.7): every source arc s -> x is saturated, so e(x) =
//    u(s, x); heights start at 0; the residual capacities are the arc
//    capacities, the sink arcs x -> t included (t has height 0).
//  * Push-relabel cycles (Algorithm 4.8, lines 1-19): the thread that owns
//    node x finds its lowest neighbour y over residual arcs; if h(x) > h(y)
//    it pushes min(e(x), c_f(x, y)) with atomics on c_f(x, y), c_f(y, x),
//    e(x), e(y), else it relabels h(x) <- h(y) + 1 (only x's thread writes
//    h(x)). A node x with no residual arc gets h(x) = |V| = N + 2.
//  * Global relabel between cycles, on the device instead of the host: the
//    exact distance of every node to t in the residual graph (the backwards
//    BFS of Algorithm 4.8), by relaxation h(x) <- min(h(x), 1 + min over
//    residual arcs (x, y) of h(y)) from h = 1 on nodes with a residual sink
//    arc, in passes over 32 x 32 tiles relaxed in shared memory; nodes that
//    are never reached keep h = |V| (the gap step: their excess can never
//    reach t). Exact
//    distances are a valid labelling, so no arc violates h(x) <= h(y) + 1
//    and no flow has to be cancelled first.
//  * The solve stops when, after a global relabel, no node with excess can
//    reach t: the preflow is then maximum, e(t) is the maximum flow value,
//    and the nodes that cannot reach t (with s) are the source side of a
//    minimum cut, every arc of which is saturated.
// Pushes to s are never needed: an active node has h < |V| = h(s).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "la.h"
#include "la_device.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kBlock = 256;
constexpr int kSweepBatch = 8;           // relabel passes between two host checks
constexpr int kTile = 32;                // relabel tile side (in nodes)
constexpr int kTileIters = 4 * kTile;    // relaxation rounds inside a tile per pass
constexpr int kFirstCycle = 32;          // push-relabel passes per launch, at first
constexpr int kMaxCycle = 4096;          // ... doubled up to this while a round leaves
                                         // more than half of the active nodes
constexpr int kDefaultMaxRounds = 1 << 16;
constexpr int kMaxCap = (1 << 30) - 1;   // c_f(x, y) + c_f(y, x) stays within int32

struct MfCtrl {
    unsigned long long e_t;       // flow into t
    unsigned long long total;     // excess put on the nodes by the source arcs
    unsigned long long active;    // nodes with excess that can reach t
    unsigned long long cut_excess;  // excess stranded on nodes that cannot reach t
    int status;
    int changed[kSweepBatch];     // relabel pass k of a batch lowered a height
};

__device__ __forceinline__ void mf_status(MfCtrl *c, int s) { atomicCAS(&c->status, 0, s); }

// neighbour of u in direction d (0: (i, j+1), 1: (i, j-1), 2: (i+1, j), 3: (i-1, j))
__device__ __forceinline__ int nbr(int u, int d, int W) {
    return d == 0 ? u + 1 : d == 1 ? u - 1 : d == 2 ? u + W : u - W;
}

// Init (Algorithm 4.7) and argument checks: capacities >= 0, arcs that
// would leave the grid have capacity 0.
__global__ void k_mf_init(const int32_t *__restrict__ cap, const int32_t *__restrict__ src,
                          const int32_t *__restrict__ snk, int H, int W, long long *__restrict__ e,
                          int *__restrict__ h, int *__restrict__ cf, int *__restrict__ rt, MfCtrl *c) {
    const int N = H * W;
    unsigned long long tot = 0;
    bool bad = false;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const int i = u / W, j = u - i * W;
        const int s0 = src[u], t0 = snk[u];
        bad |= s0 < 0 || t0 < 0 || s0 > kMaxCap || t0 > kMaxCap;
        e[u] = s0;
        tot += (unsigned long long)(s0 > 0 ? s0 : 0);
        h[u] = 0;
        rt[u] = t0;
        const bool out[4] = {j + 1 >= W, j == 0, i + 1 >= H, i == 0};
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int x = cap[(size_t)d * N + u];
            bad |= x < 0 || x > kMaxCap || (out[d] && x != 0);
            cf[(size_t)d * N + u] = x;
        }
    }
    if (bad) mf_status(c, LA_ERR_INVALID);
    for (int o = 16; o; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&c->total, tot);
}

// Lock-free push-relabel (Algorithm 4.5 / 4.8), `cycle` passes over the
// thread's nodes. Loads of state other threads write go to L2 (.cg), so a
// thread reads some recent value, as the lock-free argument assumes.
__global__ void __launch_bounds__(kBlock)
k_mf_push(int H, int W, long long *__restrict__ e, int *__restrict__ h, int *__restrict__ cf,
          int *__restrict__ rt, MfCtrl *c, int cycle) {
    const int N = H * W, NV = N + 2;               // |V|: the pixels, s and t
    const int stride = gridDim.x * blockDim.x;
    for (int it = 0; it < cycle; ++it) {
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += stride) {
            const long long eu = (long long)__ldcg(reinterpret_cast<const unsigned long long *>(e) + u);
            const int hu = h[u];                       // only this thread writes h[u]
            if (eu <= 0 || hu >= NV) continue;
            // the lowest neighbour over residual arcs (Algorithm 4.5, lines 4-9)
            int hmin = INT_MAX, dmin = -1, cmin = 0;
            const int r = rt[u];                       // only this thread writes rt[u]
            if (r > 0) {
                hmin = 0;                              // t
                dmin = 4;
                cmin = r;
            }
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                const int cd = __ldcg(cf + (size_t)d * N + u);
                if (cd > 0) {
                    const int hv = __ldcg(h + nbr(u, d, W));
                    if (hv < hmin) {
                        hmin = hv;
                        dmin = d;
                        cmin = cd;
                    }
                }
            }
            if (dmin < 0) {                            // no residual arc: t is out of reach
                h[u] = NV;
                continue;
            }
            if (hu > hmin) {                           // PUSH (lines 10-15)
                const long long delta = eu < (long long)cmin ? eu : (long long)cmin;
                if (dmin == 4) {
                    rt[u] = r - (int)delta;
                    atomicAdd(&c->e_t, (unsigned long long)delta);
                } else {
                    const int v = nbr(u, dmin, W);
                    atomicSub(cf + (size_t)dmin * N + u, (int)delta);
                    atomicAdd(cf + (size_t)(dmin ^ 1) * N + v, (int)delta);   // the reverse arc
                    atomicAdd(reinterpret_cast<unsigned long long *>(e) + v, (unsigned long long)delta);
                }
                atomicAdd(reinterpret_cast<unsigned long long *>(e) + u, (unsigned long long)(-delta));
            } else {                                   // RELABEL (line 17)
                h[u] = hmin + 1;
            }
        }
    }
}

// Global relabel, step 1: distance 1 for nodes with a residual sink arc,
// |V| = N + 2 (not reached yet) for the others. A distance to t is at most
// N (a path through every pixel), so |V| never stands for a real one.
__global__ void k_mf_relabel_init(int N, int *__restrict__ h, const int *__restrict__ rt, MfCtrl *c) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x)
        h[u] = rt[u] > 0 ? 1 : N + 2;
    if (blockIdx.x == 0 && threadIdx.x < kSweepBatch) c->changed[threadIdx.x] = 0;
}

// Global relabel, step 2: one relaxation pass over 32 x 32 tiles. A CTA
// loads its tile's heights with a one-node halo and its residual-arc flags
// into shared memory, relaxes h(x) <- min(h(x), 1 + h(y)) over the residual
// arcs inside the tile until nothing falls (at most kTileIters rounds), and
// writes the tile back, so one pass carries a distance across a whole tile.
// Distances only fall and are always lengths of real residual paths, so the
// passes reach the exact distances; they repeat until one changes nothing.
__global__ void __launch_bounds__(kTile * 8)
k_mf_relabel_tiles(int H, int W, int *__restrict__ h, const int *__restrict__ cf, MfCtrl *c, int slot) {
    __shared__ int sh[kTile + 2][kTile + 2];
    __shared__ unsigned char arcs[kTile][kTile];
    const int N = H * W, INF = N + 2;
    const int tiles_x = (W + kTile - 1) / kTile, tiles = tiles_x * ((H + kTile - 1) / kTile);
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;     // kTile x 8 threads
    bool any = false;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int i0 = (t / tiles_x) * kTile, j0 = (t % tiles_x) * kTile;
        for (int k = threadIdx.x; k < (kTile + 2) * (kTile + 2); k += blockDim.x) {
            const int li = k / (kTile + 2), lj = k % (kTile + 2);
            const int i = i0 + li - 1, j = j0 + lj - 1;
            sh[li][lj] = (i >= 0 && i < H && j >= 0 && j < W) ? __ldcg(h + (size_t)i * W + j) : INF;
        }
        for (int r = ty; r < kTile; r += 8) {
            const int i = i0 + r, j = j0 + tx;
            unsigned a = 0;
            if (i < H && j < W) {
                const size_t u = (size_t)i * W + j;
#pragma unroll
                for (int d = 0; d < 4; ++d) a |= (cf[(size_t)d * N + u] > 0 ? 1u : 0u) << d;
            }
            arcs[r][tx] = (unsigned char)a;
        }
        __syncthreads();
        bool tile_changed = false;
        for (int iter = 0; iter < kTileIters; ++iter) {
            bool ch = false;
            for (int r = ty; r < kTile; r += 8) {
                const unsigned a = arcs[r][tx];
                const int cur = sh[r + 1][tx + 1];
                if (!a || cur <= 1) continue;
                int best = cur;
                if (a & 1u) best = min(best, sh[r + 1][tx + 2] + 1);   // (i, j+1)
                if (a & 2u) best = min(best, sh[r + 1][tx] + 1);       // (i, j-1)
                if (a & 4u) best = min(best, sh[r + 2][tx + 1] + 1);   // (i+1, j)
                if (a & 8u) best = min(best, sh[r][tx + 1] + 1);       // (i-1, j)
                if (best < cur) {
                    sh[r + 1][tx + 1] = best;
                    ch = true;
                }
            }
            if (!__syncthreads_or(ch)) break;
            tile_changed = true;
        }
        if (tile_changed) {
            for (int r = ty; r < kTile; r += 8) {
                const int i = i0 + r, j = j0 + tx;
                if (i < H && j < W) h[(size_t)i * W + j] = sh[r + 1][tx + 1];
            }
            any = true;
        }
        __syncthreads();
    }
    if (any && threadIdx.x == 0) c->changed[slot] = 1;
}

// Nodes with excess that can still reach t, and excess that cannot.
__global__ void k_mf_count(int N, const long long *__restrict__ e, const int *__restrict__ h, MfCtrl *c) {
    unsigned long long act = 0, stranded = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x) {
        const long long eu = e[u];
        if (eu > 0) {
            if (h[u] < N + 2) ++act;
            else stranded += (unsigned long long)eu;
        }
    }
    for (int o = 16; o; o >>= 1) {
        act += __shfl_xor_sync(0xffffffffu, act, o);
        stranded += __shfl_xor_sync(0xffffffffu, stranded, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (act) atomicAdd(&c->active, act);
        if (stranded) atomicAdd(&c->cut_excess, stranded);
    }
}

__global__ void k_mf_cut(int N, const int *__restrict__ h, uint8_t *__restrict__ side) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < N; u += gridDim.x * blockDim.x)
        side[u] = h[u] >= N + 2 ? 1 : 0;
}

struct MfWorkspace {
    int64_t cap = 0;
    long long *e = nullptr;
    int *h = nullptr;
    int *cf = nullptr;
    int *rt = nullptr;
    MfCtrl *ctrl = nullptr;
    MfCtrl *h_ctrl = nullptr;
    int num_sms = 0;
    int occ = 0;
};

std::mutex g_mmu;
MfWorkspace g_mws[kMaxDevices];

la_status ensure_mws(MfWorkspace &w, int64_t N) {
    if (!w.ctrl) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
        if (cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return LA_ERR_CUDA;
        if (cudaMalloc(&w.ctrl, sizeof(MfCtrl)) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMallocHost(&w.h_ctrl, sizeof(MfCtrl)) != cudaSuccess) return LA_ERR_NOMEM;
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_mf_push, kBlock, 0);
        w.occ = std::max(1, o);
    }
    if (w.cap < N) {
        cudaFree(w.e);
        cudaFree(w.h);
        cudaFree(w.cf);
        cudaFree(w.rt);
        w.e = nullptr;
        w.h = w.cf = w.rt = nullptr;
        w.cap = 0;
        if (cudaMalloc(&w.e, sizeof(long long) * N) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.h, sizeof(int) * N) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.cf, sizeof(int) * 4 * N) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.rt, sizeof(int) * N) != cudaSuccess) return LA_ERR_NOMEM;
        w.cap = N;
    }
    return LA_OK;
}

}  // namespace

#define LA_MCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

static la_status maxflow_locked(const int32_t *cap, const int32_t *src, const int32_t *snk, int32_t H, int32_t W,
                                const la_maxflow_options *opt, cudaStream_t s, int64_t *flow_out,
                                uint8_t *cut_out, la_maxflow_stats *st) {
    const bool fixed_cycle = opt && opt->cycle > 0;
    int cycle = fixed_cycle ? opt->cycle : kFirstCycle;
    const int max_rounds = (opt && opt->max_rounds > 0) ? opt->max_rounds : kDefaultMaxRounds;
    la_maxflow_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    const int64_t N = (int64_t)H * W;
    int dev = 0;
    LA_MCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    MfWorkspace &w = g_mws[dev];
    if (la_status e = ensure_mws(w, N)) return e;
    const int n = (int)N;
    const int grid = std::max(1, std::min((n + kBlock - 1) / kBlock, w.num_sms * w.occ));
    const int tiles = ((H + kTile - 1) / kTile) * ((W + kTile - 1) / kTile);
    const int tgrid = std::max(1, std::min(tiles, 8 * w.num_sms));
    LA_MCK(cudaMemsetAsync(w.ctrl, 0, sizeof(MfCtrl), s));
    k_mf_init<<<grid, kBlock, 0, s>>>(cap, src, snk, H, W, w.e, w.h, w.cf, w.rt, w.ctrl);
    int64_t launches = 1;
    LA_MCK(cudaGetLastError());
    // nothing reads a neighbour before the capacities are known to stay inside the grid
    LA_MCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, s));
    LA_MCK(cudaStreamSynchronize(s));
    if (w.h_ctrl->status) return (la_status)w.h_ctrl->status;

    // global relabel: init, then batches of sweeps until a batch's last sweep changes nothing
    auto global_relabel = [&]() -> la_status {
        k_mf_relabel_init<<<grid, kBlock, 0, s>>>(n, w.h, w.rt, w.ctrl);
        ++launches;
        for (int b = 0; b * kSweepBatch <= n; ++b) {
            for (int k = 0; k < kSweepBatch; ++k) {
                k_mf_relabel_tiles<<<tgrid, kTile * 8, 0, s>>>(H, W, w.h, w.cf, w.ctrl, k);
                ++launches;
            }
            stats.relabel_sweeps += kSweepBatch;
            LA_MCK(cudaGetLastError());
            LA_MCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, s));
            LA_MCK(cudaStreamSynchronize(s));
            if (!w.h_ctrl->changed[kSweepBatch - 1]) break;
            LA_MCK(cudaMemsetAsync(w.ctrl->changed, 0, sizeof(int) * kSweepBatch, s));
        }
        ++stats.global_relabels;
        return LA_OK;
    };

    if (la_status e = global_relabel()) return e;
    if (w.h_ctrl->status) return (la_status)w.h_ctrl->status;
    stats.excess_total = (int64_t)w.h_ctrl->total;
    la_status rc = LA_ERR_ITER_LIMIT;
    unsigned long long last_active = ~0ull;
    for (int round = 0; round < max_rounds; ++round) {
        LA_MCK(cudaMemsetAsync(&w.ctrl->active, 0, 2 * sizeof(unsigned long long), s));
        k_mf_count<<<grid, kBlock, 0, s>>>(n, w.e, w.h, w.ctrl);
        ++launches;
        LA_MCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(MfCtrl), cudaMemcpyDeviceToHost, s));
        LA_MCK(cudaStreamSynchronize(s));
        if (w.h_ctrl->status) return (la_status)w.h_ctrl->status;
        const unsigned long long active = w.h_ctrl->active;
        if (active == 0) {                // every node with excess is cut off from t
            rc = LA_OK;
            break;
        }
        // long augmenting paths need more passes between two global relabels
        if (!fixed_cycle && round > 0 && 2 * active > last_active) cycle = std::min(2 * cycle, kMaxCycle);
        last_active = active;
        k_mf_push<<<grid, kBlock, 0, s>>>(H, W, w.e, w.h, w.cf, w.rt, w.ctrl, cycle);
        ++launches;
        ++stats.rounds;
        if (la_status e = global_relabel()) return e;
    }
    if (rc != LA_OK) return rc;
    const MfCtrl c1 = *w.h_ctrl;
    // every unit of excess is in t or stranded on the source side
    if (c1.e_t + c1.cut_excess != c1.total) return LA_ERR_INTERNAL;
    LA_MCK(cudaMemcpyAsync(flow_out, &w.ctrl->e_t, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (cut_out) {
        k_mf_cut<<<grid, kBlock, 0, s>>>(n, w.h, cut_out);
        ++launches;
    }
    LA_MCK(cudaGetLastError());
    LA_MCK(cudaStreamSynchronize(s));
    stats.flow = (int64_t)c1.e_t;
    stats.launches = launches;
    if (st) *st = stats;
    return LA_OK;
}

extern "C" {

la_status la_maxflow_grid_ex(const int32_t *cap, const int32_t *src, const int32_t *snk, int32_t H, int32_t W,
                             const la_maxflow_options *opt, void *stream, int64_t *flow_out, uint8_t *cut_out,
                             la_maxflow_stats *stats_out) {
    if (H < 1 || W < 1 || (int64_t)H * W >= (1ll << 30) || !cap || !src || !snk || !flow_out) return LA_ERR_INVALID;
    if (opt && (opt->cycle < 0 || opt->max_rounds < 0)) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mmu);
    return maxflow_locked(cap, src, snk, H, W, opt, static_cast<cudaStream_t>(stream), flow_out, cut_out,
                          stats_out);
}

la_status la_maxflow_grid(const int32_t *cap, const int32_t *src, const int32_t *snk, int32_t H, int32_t W,
                          void *stream, int64_t *flow_out, uint8_t *cut_out) {
    return la_maxflow_grid_ex(cap, src, snk, H, W, nullptr, stream, flow_out, cut_out, nullptr);
}

}  // extern "C"
