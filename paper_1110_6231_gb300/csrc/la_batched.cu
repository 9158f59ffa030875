// la_solve_batched: many independent dense assignments in one persistent
// launch (captured in a CUDA graph and replayed).
//
// Each CTA claims instances from a device work queue, largest first, and
// runs the whole cost-scaling solve of an instance (Sect. 5.1, Algorithm
// 5.0's epsilon loop; refine initialisation of Algorithm 5.2; the push /
// relabel of Algorithm 5.4 as a double push) with the instance's column keys
// in shared memory:
//   * one 64-bit key per column, (price, mate) packed as in la_solve, so a
//     bid is one shared-memory atomicMin;
//   * the CTA's warps are the instance's parallel bidders ("rows per CTA" =
//     warps per CTA): each takes a free row from a shared counter, scans its
//     cost row from global memory against the shared prices, bids, and
//     continues with the row it displaced;
//   * a phase ends at a CTA barrier once the queue is empty and every warp's
//     row is matched.
// Prices stay exact integers; per instance, costs are scaled by n + 1 and
// the last phase runs at eps = 1, so every instance's cost is exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "la.h"
#include "la_device.cuh"

using namespace la;

namespace {

constexpr int kPrepThreads = 1024;
constexpr int kMaxDevices = 64;

struct BatchCtrl {
    unsigned long long scan_bytes;   // 4 n bytes of cost per row scan
    unsigned long long scans;
    unsigned long long wins;
    unsigned long long displaced;
    unsigned long long phases;
    int next;       // work-queue head
    int status;     // first failing instance's status
    int failed;     // failing instances
    int max_n;      // largest n in the batch (prep)
};

struct BatchParams {
    int alpha[LA_ALPHA_BUCKETS];   // per floor(log2 n)
    int budget_factor;             // scans per row per phase before LA_ERR_ITER_LIMIT
};

__device__ __forceinline__ int log2_bucket(int n) {
    return min(LA_ALPHA_BUCKETS - 1, 31 - __clz(max(n, 1)));
}

// Exclusive scan of one value per thread across the block (blockDim = kPrepThreads).
__device__ long long block_exclusive_scan(long long v, long long *sh, long long *total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (kPrepThreads / 32) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    const long long before = (warp ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[kPrepThreads / 32 - 1];
    __syncthreads();
    return before;
}

// Plan of a batch (one block): match offsets = exclusive prefix sums of n,
// and a work order with the largest instances first (counting sort on n).
__global__ void __launch_bounds__(kPrepThreads)
k_batch_prep(const int *__restrict__ ns, int B, int max_n, long long *__restrict__ moff,
             int *__restrict__ order, int *__restrict__ hist, BatchCtrl *ctrl) {
    __shared__ long long sh[32];
    const int tid = threadIdx.x;
    const int nb = max_n + 2;                   // bin 0: invalid, bin 1 + (max_n - n) otherwise
    for (int b = tid; b < nb; b += kPrepThreads) hist[b] = 0;
    __syncthreads();
    const int chunk = (B + kPrepThreads - 1) / kPrepThreads;
    const int i0 = min(B, tid * chunk), i1 = min(B, i0 + chunk);
    long long local = 0;
    int mx = 0;
    for (int i = i0; i < i1; ++i) {
        const int n = ns[i];
        const bool ok = n >= 0 && n <= max_n;
        local += ok ? n : 0;
        if (n > mx) mx = n;
        atomicAdd(&hist[ok ? 1 + (max_n - n) : 0], 1);
    }
    long long run = block_exclusive_scan(local, sh, nullptr);
    for (int i = i0; i < i1; ++i) {
        moff[i] = run;
        const int n = ns[i];
        run += (n >= 0 && n <= max_n) ? n : 0;
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if ((tid & 31) == 0) atomicMax(&ctrl->max_n, mx);
    __syncthreads();
    // exclusive scan of the histogram, in chunks
    const int hchunk = (nb + kPrepThreads - 1) / kPrepThreads;
    const int b0 = min(nb, tid * hchunk), b1 = min(nb, b0 + hchunk);
    long long hs = 0;
    for (int b = b0; b < b1; ++b) hs += hist[b];
    long long hrun = block_exclusive_scan(hs, sh, nullptr);
    for (int b = b0; b < b1; ++b) {
        const int c = hist[b];
        hist[b] = (int)hrun;
        hrun += c;
    }
    __syncthreads();
    for (int i = i0; i < i1; ++i) {
        const int n = ns[i];
        const bool ok = n >= 0 && n <= max_n;
        order[atomicAdd(&hist[ok ? 1 + (max_n - n) : 0], 1)] = i;
    }
}

// One refine phase of one instance by one warp (all warps of the CTA run it
// concurrently on the shared keys).
template <bool WIDE>
__device__ __forceinline__ void warp_refine(const int32_t *__restrict__ Ci, int n, int cmin, uint32_t np1,
                                            unsigned long long eps, unsigned long long qlim,
                                            unsigned long long *skey, int *s_next_row,
                                            unsigned long long *s_scans, int *s_status,
                                            unsigned long long budget, bool vec, int lane,
                                            unsigned long long &wins, unsigned long long &displaced) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    const volatile unsigned long long *vkey = skey;
    int row = -1;
    for (;;) {
        if (row < 0) {
            int r = 0;
            if (lane == 0) r = atomicAdd(s_next_row, 1);
            row = __shfl_sync(0xffffffffu, r, 0);
            if (row >= n) break;
        }
        unsigned long long s = 0;
        int st = 0;
        if (lane == 0) {
            s = atomicAdd(s_scans, 1ull);
            st = *reinterpret_cast<volatile int *>(s_status);
        }
        s = __shfl_sync(0xffffffffu, s, 0);
        st = __shfl_sync(0xffffffffu, st, 0);
        if (st != 0) break;
        if (s >= budget) {
            if (lane == 0) atomicCAS(s_status, 0, (int)LA_ERR_ITER_LIMIT);
            break;
        }
        const int32_t *crow = Ci + (size_t)row * n;
        Lane2<V> t;
        lane2_init(t);
        if (vec) {
            const int4 *r4 = reinterpret_cast<const int4 *>(crow);
            const int nv = n >> 2;
#pragma unroll 2
            for (int j = lane; j < nv; j += 32) {
                const int4 c = ld_row4(r4 + j);
                const int y = j << 2;
                lane2_push<V>(t, (V)(uint32_t)(c.x - cmin) * np1 + (V)key_q(vkey[y]), y);
                lane2_push<V>(t, (V)(uint32_t)(c.y - cmin) * np1 + (V)key_q(vkey[y + 1]), y + 1);
                lane2_push<V>(t, (V)(uint32_t)(c.z - cmin) * np1 + (V)key_q(vkey[y + 2]), y + 2);
                lane2_push<V>(t, (V)(uint32_t)(c.w - cmin) * np1 + (V)key_q(vkey[y + 3]), y + 3);
            }
        } else {
#pragma unroll 4
            for (int y = lane; y < n; y += 32) {
                const int c = ld_row1(crow + y);
                lane2_push<V>(t, (V)(uint32_t)(c - cmin) * np1 + (V)key_q(vkey[y]), y);
            }
        }
        const V c1 = t.w1 >= 0 ? (V)(uint32_t)(ld_row1(crow + t.w1) - cmin) * np1 : (V)0;
        ScanResult<V> r{t.b1, t.b2, c1, t.w1 < 0 ? INT_MAX : t.w1};
        warp_merge(r);
        const unsigned long long nq = (unsigned long long)(r.b1 - r.c1) + (r.b2 - r.b1) + eps;
        if (r.w >= n || nq > qlim) {
            if (lane == 0) atomicCAS(s_status, 0, (int)(r.w >= n ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW));
            break;
        }
        const unsigned long long nk = pack_key(nq, (uint32_t)row);
        unsigned long long old = 0;
        if (lane == 0) old = atomicMin(skey + r.w, nk);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old > nk) {
            ++wins;
            const uint32_t m = key_mate(old);
            if (m != kNone) {
                ++displaced;
                row = (int)m;
            } else {
                row = -1;
            }
        }
    }
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
k_batch_solve(const int32_t *__restrict__ C, const long long *__restrict__ offsets,
              const int *__restrict__ ns, const int *__restrict__ order,
              const long long *__restrict__ moff, int B, int max_n, BatchParams P,
              int32_t *__restrict__ match_out, long long *__restrict__ cost_out,
              int *__restrict__ inst_status, BatchCtrl *ctrl, long long *__restrict__ prices_out) {
    extern __shared__ unsigned long long skey[];
    __shared__ int s_k, s_next_row, s_cmin, s_cmax, s_status;
    __shared__ unsigned long long s_qmin, s_scans, s_cost;
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned long long wins = 0, displaced = 0, phases_run = 0;
    for (;;) {
        if (tid == 0) s_k = atomicAdd(&ctrl->next, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= B) break;
        const int i = order[k];
        const int n = ns[i];
        if (tid == 0) {
            s_cmin = INT_MAX;
            s_cmax = INT_MIN;
            s_status = 0;
            s_scans = 0;
            s_cost = 0;
        }
        __syncthreads();
        if (n < 0 || n > max_n || n == 0) {
            if (tid == 0) {
                const int st = n == 0 ? 0 : (int)LA_ERR_INVALID;
                if (cost_out) cost_out[i] = 0;
                if (inst_status) inst_status[i] = st;
                if (st) {
                    atomicAdd(&ctrl->failed, 1);
                    atomicCAS(&ctrl->status, 0, st);
                }
            }
            __syncthreads();
            continue;
        }
        const int32_t *Ci = C + offsets[i];
        int32_t *Mi = match_out ? match_out + moff[i] : nullptr;
        // min and max cost of the instance
        {
            int lo = INT_MAX, hi = INT_MIN;
            const long long tot = (long long)n * n;
            for (long long e = tid; e < tot; e += BLOCK) {
                const int c = ld_row1(Ci + e);
                lo = min(lo, c);
                hi = max(hi, c);
            }
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if (lane == 0) {
                atomicMin(&s_cmin, lo);
                atomicMax(&s_cmax, hi);
            }
        }
        for (int y = tid; y < n; y += BLOCK) skey[y] = ~0ull;   // q = 0, no mate
        __syncthreads();
        const int cmin = s_cmin;
        const unsigned long long np1 = (unsigned long long)n + 1;
        const unsigned long long Ct = np1 * (unsigned long long)((long long)s_cmax - (long long)cmin);
        const int alpha = max(2, P.alpha[log2_bucket(n)]);
        int nph = 0;
        {
            unsigned long long e = Ct;
            do {
                e = max(1ull, e / (unsigned long long)alpha);
                ++nph;
            } while (e > 1);
        }
        const unsigned long long eps1 = max(1ull, Ct / (unsigned long long)alpha);
        const bool wide = 4 * Ct + 2 * eps1 + 16 >= (1ull << 32);
        const unsigned long long qlim = wide ? (kQMax - 1) : ((1ull << 32) - 2 - Ct);
        const bool vec = ((offsets[i] & 3) == 0) && (n % 4 == 0) &&
                         ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
        const unsigned long long budget = (unsigned long long)P.budget_factor * n * nph + 65536;
        if (Ct >= (1ull << 40)) {
            if (tid == 0) s_status = LA_ERR_OVERFLOW;
        } else if (n == 1) {
            if (tid == 0) {
                if (Mi) Mi[0] = 0;
                s_cost = (unsigned long long)(long long)Ci[0];
            }
        } else {
            unsigned long long eps = Ct;
            for (int ph = 0; ph < nph; ++ph) {
                eps = max(1ull, eps / (unsigned long long)alpha);
                // refine initialisation: shift prices so that min q = 0,
                // clear every mate, reset the row queue
                if (tid == 0) s_qmin = ~0ull;
                __syncthreads();
                unsigned long long m = ~0ull;
                for (int y = tid; y < n; y += BLOCK) m = min(m, key_q(skey[y]));
                for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) atomicMin(&s_qmin, m);
                __syncthreads();
                const unsigned long long qmin = s_qmin;
                for (int y = tid; y < n; y += BLOCK) skey[y] = pack_key(key_q(skey[y]) - qmin, kNone);
                if (tid == 0) s_next_row = 0;
                __syncthreads();
                if (wide)
                    warp_refine<true>(Ci, n, cmin, (uint32_t)np1, eps, qlim, skey, &s_next_row, &s_scans,
                                      &s_status, budget, vec, lane, wins, displaced);
                else
                    warp_refine<false>(Ci, n, cmin, (uint32_t)np1, eps, qlim, skey, &s_next_row, &s_scans,
                                       &s_status, budget, vec, lane, wins, displaced);
                __syncthreads();
                ++phases_run;
                if (s_status) break;
            }
            if (!s_status) {
                long long sum = 0;
                for (int y = tid; y < n; y += BLOCK) {
                    const uint32_t mm = key_mate(skey[y]);
                    if (mm >= (uint32_t)n) {
                        atomicCAS(&s_status, 0, (int)LA_ERR_INTERNAL);
                        continue;
                    }
                    if (Mi) Mi[mm] = y;
                    if (prices_out) prices_out[moff[i] + y] = -(long long)key_q(skey[y]);
                    sum += Ci[(size_t)mm * n + y];
                }
                for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                if (lane == 0 && sum) atomicAdd(&s_cost, (unsigned long long)sum);
            }
        }
        __syncthreads();
        if (tid == 0) {
            const int st = s_status;
            if (cost_out) cost_out[i] = (long long)s_cost;
            if (inst_status) inst_status[i] = st;
            atomicAdd(&ctrl->scans, s_scans);
            atomicAdd(&ctrl->scan_bytes, s_scans * 4ull * (unsigned long long)n);
            if (st) {
                atomicAdd(&ctrl->failed, 1);
                atomicCAS(&ctrl->status, 0, st);
            }
        }
        __syncthreads();
    }
    if (lane == 0) {
        atomicAdd(&ctrl->wins, wins);
        atomicAdd(&ctrl->displaced, displaced);
    }
    if (tid == 0) atomicAdd(&ctrl->phases, phases_run);
}

// ---------------------------------------------------------------- host side

struct GraphKey {
    const void *cost, *offsets, *ns, *match, *costout, *status, *prices;
    int B, block, max_n;
    cudaStream_t stream;
    BatchParams P;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct BatchWorkspace {
    int64_t capB = 0;
    int max_n_cap = 0;
    long long *moff = nullptr;
    int *order = nullptr;
    int *hist = nullptr;
    int *status = nullptr;
    BatchCtrl *ctrl = nullptr;
    BatchCtrl *h_ctrl = nullptr;
    int num_sms = 0;
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    bool have_key = false;
};

std::mutex g_bmu;
BatchWorkspace g_bws[kMaxDevices];

void drop_graph(BatchWorkspace &w) {
    if (w.exec) cudaGraphExecDestroy(w.exec);
    w.exec = nullptr;
    w.have_key = false;
}

la_status ensure_bws(BatchWorkspace &w, int64_t B, int max_n) {
    if (!w.ctrl) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
        if (cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return LA_ERR_CUDA;
        if (cudaMalloc(&w.ctrl, sizeof(BatchCtrl)) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMallocHost(&w.h_ctrl, sizeof(BatchCtrl)) != cudaSuccess) return LA_ERR_NOMEM;
    }
    if (w.capB < B || w.max_n_cap < max_n) {
        drop_graph(w);
        cudaFree(w.moff);
        cudaFree(w.order);
        cudaFree(w.hist);
        cudaFree(w.status);
        w.moff = nullptr;
        w.order = nullptr;
        w.hist = nullptr;
        w.status = nullptr;
        const int64_t cap = std::max<int64_t>(std::max(B, w.capB), 1024);
        const int mcap = std::max(max_n, w.max_n_cap);
        if (cudaMalloc(&w.moff, sizeof(long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.order, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.status, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.hist, sizeof(int) * (mcap + 2)) != cudaSuccess) return LA_ERR_NOMEM;
        w.capB = cap;
        w.max_n_cap = mcap;
    }
    return LA_OK;
}

template <int BLOCK>
cudaError_t launch_solve(cudaStream_t s, int grid, size_t smem, const int32_t *cost, const int64_t *offsets,
                         const int32_t *ns, const BatchWorkspace &w, int B, int max_n, const BatchParams &P,
                         int32_t *match_out, int64_t *cost_out, int *status, int64_t *prices) {
    k_batch_solve<BLOCK><<<grid, BLOCK, smem, s>>>(cost, reinterpret_cast<const long long *>(offsets), ns,
                                                   w.order, w.moff, B, max_n, P, match_out,
                                                   reinterpret_cast<long long *>(cost_out), status, w.ctrl,
                                                   reinterpret_cast<long long *>(prices));
    return cudaGetLastError();
}

template <int BLOCK>
int solve_grid(int num_sms, size_t smem) {
    static int occ[2] = {0, 0};
    static size_t occ_smem[2] = {0, 0};
    const int slot = 0;
    if (!occ[slot] || occ_smem[slot] != smem) {
        int o = 0;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_batch_solve<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch_solve<BLOCK>, BLOCK, smem);
        occ[slot] = std::max(1, o);
        occ_smem[slot] = smem;
    }
    return num_sms * occ[slot];
}

cudaError_t enqueue(cudaStream_t s, int block, int grid, size_t smem, const int32_t *cost,
                    const int64_t *offsets, const int32_t *ns, BatchWorkspace &w, int B, int max_n,
                    const BatchParams &P, int32_t *match_out, int64_t *cost_out, int *status, int64_t *prices) {
    cudaError_t e = cudaMemsetAsync(w.ctrl, 0, sizeof(BatchCtrl), s);
    if (e != cudaSuccess) return e;
    k_batch_prep<<<1, kPrepThreads, 0, s>>>(ns, B, max_n, w.moff, w.order, w.hist, w.ctrl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    switch (block) {
    case 64: return launch_solve<64>(s, grid, smem, cost, offsets, ns, w, B, max_n, P, match_out, cost_out, status, prices);
    case 128: return launch_solve<128>(s, grid, smem, cost, offsets, ns, w, B, max_n, P, match_out, cost_out, status, prices);
    case 256: return launch_solve<256>(s, grid, smem, cost, offsets, ns, w, B, max_n, P, match_out, cost_out, status, prices);
    default: return launch_solve<512>(s, grid, smem, cost, offsets, ns, w, B, max_n, P, match_out, cost_out, status, prices);
    }
}

}  // namespace

#define LA_BCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

static la_status batched_locked(const int32_t *cost, const int64_t *offsets, const int32_t *ns, int32_t B,
                                const la_batch_options *opt, cudaStream_t s, int32_t *match_out,
                                int64_t *cost_out, int32_t *status_out, la_batch_stats *st) {
    const int block = (opt && opt->block_threads) ? opt->block_threads : 128;
    const int max_n = (opt && opt->max_n) ? opt->max_n : LA_BATCH_MAX_N;
    const bool graph = !(opt && opt->no_graph);
    int64_t *prices = opt ? opt->prices_out : nullptr;
    if (block != 64 && block != 128 && block != 256 && block != 512) return LA_ERR_INVALID;
    if (max_n < 1 || max_n > LA_BATCH_MAX_N) return LA_ERR_INVALID;
    BatchParams P;
    for (int k = 0; k < LA_ALPHA_BUCKETS; ++k) {
        const int a = opt ? opt->alpha[k] : 0;
        if (a != 0 && a < 2) return LA_ERR_INVALID;
        P.alpha[k] = a ? a : 10;
    }
    P.budget_factor = (opt && opt->budget_factor > 0) ? opt->budget_factor : 256;
    if (st) std::memset(st, 0, sizeof(*st));
    if (B == 0) return LA_OK;

    int dev = 0;
    LA_BCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    BatchWorkspace &w = g_bws[dev];
    if (la_status e = ensure_bws(w, B, max_n)) return e;
    int *status = status_out ? status_out : w.status;
    const size_t smem = sizeof(unsigned long long) * (size_t)max_n;
    int grid = 0;
    switch (block) {
    case 64: grid = solve_grid<64>(w.num_sms, smem); break;
    case 128: grid = solve_grid<128>(w.num_sms, smem); break;
    case 256: grid = solve_grid<256>(w.num_sms, smem); break;
    default: grid = solve_grid<512>(w.num_sms, smem); break;
    }
    grid = std::max(1, std::min(grid, (int)B));

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool profile = opt && opt->profile;
    if (profile) {
        LA_BCK(cudaEventCreate(&e0));
        LA_BCK(cudaEventCreate(&e1));
        LA_BCK(cudaEventRecord(e0, s));
    }
    bool launched_graph = false;
    if (graph) {
        GraphKey key;
        std::memset(&key, 0, sizeof(key));
        key.cost = cost;
        key.offsets = offsets;
        key.ns = ns;
        key.match = match_out;
        key.costout = cost_out;
        key.status = status;
        key.prices = prices;
        key.B = B;
        key.block = block;
        key.max_n = max_n;
        key.stream = s;
        key.P = P;
        if (!(w.have_key && w.key == key && w.exec)) {
            drop_graph(w);
            cudaStream_t cs = nullptr;
            LA_BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                const cudaError_t le = enqueue(cs, block, grid, smem, cost, offsets, ns, w, B, max_n, P,
                                               match_out, cost_out, status, prices);
                ce = cudaStreamEndCapture(cs, &g);
                if (le != cudaSuccess) ce = le;
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&w.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess) {
                w.exec = nullptr;
                return LA_ERR_CUDA;
            }
            w.key = key;
            w.have_key = true;
        }
        LA_BCK(cudaGraphLaunch(w.exec, s));
        launched_graph = true;
    } else {
        LA_BCK(enqueue(s, block, grid, smem, cost, offsets, ns, w, B, max_n, P, match_out, cost_out, status,
                       prices));
    }
    if (profile) LA_BCK(cudaEventRecord(e1, s));
    LA_BCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, s));
    LA_BCK(cudaStreamSynchronize(s));
    const BatchCtrl c = *w.h_ctrl;
    if (st) {
        st->instances = B;
        st->failed = c.failed;
        st->scans = (int64_t)c.scans;
        st->scan_bytes = (int64_t)c.scan_bytes;
        st->wins = (int64_t)c.wins;
        st->displaced = (int64_t)c.displaced;
        st->phases = (int64_t)c.phases;
        st->max_n = c.max_n;
        st->grid = grid;
        st->block_threads = block;
        st->graph = launched_graph;
        if (profile) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            st->device_ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (c.max_n > max_n && c.status == 0) return LA_ERR_INVALID;
    return (la_status)c.status;
}

extern "C" {

la_status la_solve_batched_ex(const int32_t *cost, const int64_t *offsets, const int32_t *ns, int32_t B,
                              const la_batch_options *opt, void *stream, int32_t *match_out,
                              int64_t *cost_out, int32_t *status_out, la_batch_stats *stats_out) {
    if (B < 0 || (B > 0 && (!cost || !offsets || !ns || !cost_out))) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_bmu);
    return batched_locked(cost, offsets, ns, B, opt, static_cast<cudaStream_t>(stream), match_out, cost_out,
                          status_out, stats_out);
}

la_status la_solve_batched(const int32_t *cost, const int64_t *offsets, const int32_t *ns, int32_t B,
                           void *stream, int32_t *match_out, int64_t *cost_out) {
    return la_solve_batched_ex(cost, offsets, ns, B, nullptr, stream, match_out, cost_out, nullptr, nullptr);
}

}  // extern "C"
