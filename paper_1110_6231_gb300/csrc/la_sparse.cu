// la_solve_sparse: exact minimum-cost perfect matching of a sparse bipartite
// graph (arcs in CSR form) by the same cost scaling as la_solve.
//
// The paper's implementation takes arbitrary bipartite graphs (Sect. 1 and
// Sect. 6); Sect. 5 reduces assignment to min-cost flow with u(x,y) = 1 on
// the graph's arcs. Here a free row's warp scans only its own arcs
// (coalesced loads of columns and costs, prices gathered at L2) for the best
// and second-best part-reduced cost, and commits the Goldberg-Kennedy double
// push with the same packed 64-bit atomicMin on the column key as the dense
// refine (Algorithm 5.4 as a double push, Algorithm 5.2's initialisation,
// Algorithm 5.0's eps loop on costs scaled by n + 1).
//
// Readings for graphs that are not complete:
//  * A row with one arc (or whose arcs all lead to one column) has no second
//    best: any price drop >= eps keeps it eps-optimal, since eps-CS compares
//    only the row's own arcs. It bids as on a tie (drop = eps).
//  * Parallel arcs x -> y are allowed; a matching uses the cheaper one, and
//    a bid against the other copy keeps eps-CS (it only shrinks the drop).
//  * Feasibility. A graph may have no perfect matching. A first refine
//    phase runs with every arc cost taken as 0 and eps = 1 from zero prices:
//    if a perfect matching M' exists it is 0-optimal there, and the
//    price-drop bound of cost scaling (the path argument behind Lemma 5.6's
//    use of eps-optimality: a column relabelled while it holds excess lies on
//    an alternating path to a free column, of at most 2n - 1 arcs) keeps every
//    price within (eps + 0)(2n - 1) of its start. A drop beyond 4n + 4 in that
//    phase therefore proves that no perfect matching exists
//    (LA_ERR_INFEASIBLE); otherwise prices are reset and the cost phases run
//    on a graph known to be feasible.
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

constexpr int kMaxDevices = 64;
constexpr int kBlock = 256;

__device__ __forceinline__ void sp_set_status(Ctrl *ctrl, int s) { atomicCAS(&ctrl->status, 0, s); }

// Structure of the CSR arrays, min / max cost, rows and columns without arcs.
__global__ void k_sp_validate(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ cols,
                              const int32_t *__restrict__ costs, int n, int nnz, int *__restrict__ colseen,
                              Ctrl *ctrl) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    bool bad = false, empty_row = false;
    for (int x = tid; x < n; x += stride) {
        const int b = row_ptr[x], e = row_ptr[x + 1];
        bad |= e < b || b < 0 || e > nnz;
        empty_row |= e == b;
    }
    if (tid == 0) bad |= row_ptr[0] != 0 || row_ptr[n] != nnz;
    int lo = INT_MAX, hi = INT_MIN;
    for (int k = tid; k < nnz; k += stride) {
        const int y = cols[k];
        if (y < 0 || y >= n) {
            bad = true;
            continue;
        }
        colseen[y] = 1;
        const int c = costs[k];
        lo = min(lo, c);
        hi = max(hi, c);
    }
    if (bad) sp_set_status(ctrl, LA_ERR_INVALID);
    if (empty_row) atomicExch(&ctrl->colseen_missing, 1);
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ctrl->cmin, lo);
        atomicMax(&ctrl->cmax, hi);
    }
}

__global__ void k_sp_colcheck(const int *__restrict__ colseen, int n, Ctrl *ctrl) {
    bool miss = false;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) miss |= colseen[y] == 0;
    if (miss) atomicExch(&ctrl->colseen_missing, 1);
}

__global__ void k_sp_qmin(const unsigned long long *__restrict__ key, int n, Ctrl *ctrl, int slot) {
    unsigned long long m = ~0ull;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x)
        m = min(m, key_q(__ldcg(key + y)));
    m = warp_min(m);
    if ((threadIdx.x & 31) == 0) atomicMin(&ctrl->qmin[slot], m);
}

// Refine initialisation (Algorithm 5.2): every row free, prices kept and
// shifted so that min q = 0, the price mirror refreshed, the queue reset.
// zero = 1 restarts from zero prices (after the feasibility phase).
__global__ void k_sp_reset(unsigned long long *__restrict__ key, unsigned long long *__restrict__ qm, int n,
                           unsigned long long qlim, Ctrl *ctrl, int slot, int phase, int zero) {
    const unsigned long long qmin = zero ? 0ull : ctrl->qmin[slot];
    bool bad = false;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const unsigned long long q = zero ? 0ull : key_q(key[y]) - qmin;
        bad |= q > qlim;
        key[y] = pack_key(q, kNone);
        qm[y] = q;
    }
    if (bad) sp_set_status(ctrl, LA_ERR_OVERFLOW);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->next_row = 0;
        ctrl->qmin[slot ^ 1] = ~0ull;
        ctrl->phase_start_scans[phase & 63] = ctrl->scans;
    }
}

// One refine phase over the arcs: persistent grid, one warp per free row.
// ZERO: the feasibility phase (every arc cost taken as 0; a price drop past
// qinf proves that no perfect matching exists).
template <bool ZERO>
__global__ void __launch_bounds__(kBlock)
k_sp_refine(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ cols,
            const int32_t *__restrict__ costs, int n, int cmin, uint32_t np1, unsigned long long eps,
            unsigned long long qlim, unsigned long long qinf, unsigned long long *__restrict__ key,
            unsigned long long *__restrict__ qm, Ctrl *__restrict__ ctrl, unsigned long long budget) {
    constexpr unsigned kFlush = 8;
    const int lane = threadIdx.x & 31;
    using V = unsigned long long;
    const V inf = ~0ull;
    if (*reinterpret_cast<volatile int *>(&ctrl->status) != 0) return;   // an earlier phase failed
    int row = -1;
    unsigned long long wins = 0, displaced = 0, total = 0;
    unsigned pending = 0;
    for (;;) {
        if (row < 0) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&ctrl->next_row, 1);
            row = __shfl_sync(0xffffffffu, r, 0);
            if (row >= n) break;
        }
        if (pending == kFlush) {
            unsigned long long s = 0;
            int st = 0;
            if (lane == 0) {
                s = atomicAdd(&ctrl->scans, (unsigned long long)kFlush);
                st = *reinterpret_cast<volatile int *>(&ctrl->status);
            }
            s = __shfl_sync(0xffffffffu, s, 0);
            st = __shfl_sync(0xffffffffu, st, 0);
            pending = 0;
            if (st != 0) break;
            if (s + kFlush > budget) {
                if (lane == 0) sp_set_status(ctrl, LA_ERR_ITER_LIMIT);
                break;
            }
        }
        ++pending;
        ++total;
        // best and second best of v(x,y) = (C - cmin)(n+1) + q(y) over the row's arcs
        const int b = __ldg(row_ptr + row), e = __ldg(row_ptr + row + 1);
        ScanResult<V> r{inf, inf, 0, INT_MAX};
        for (int k = b + lane; k < e; k += 32) {
            const int y = __ldg(cols + k);
            const V cs = ZERO ? 0ull : (V)(uint32_t)(__ldg(costs + k) - cmin) * np1;
            const V v = cs + __ldcg(qm + y);
            const bool better = v < r.b1 || (v == r.b1 && (unsigned)y < (unsigned)r.w);
            const V hi = better ? r.b1 : v;
            r.b2 = hi < r.b2 ? hi : r.b2;
            r.c1 = better ? cs : r.c1;
            r.w = better ? y : r.w;
            r.b1 = better ? v : r.b1;
        }
        warp_merge(r);
        if (r.b2 == inf) r.b2 = r.b1;     // a single arc: bid as on a tie
        const unsigned long long nq = (r.b1 - r.c1) + (r.b2 - r.b1) + eps;
        if (r.w >= n || nq > qlim || nq > qinf) {
            if (lane == 0)
                sp_set_status(ctrl, r.w >= n ? LA_ERR_INTERNAL : (nq > qinf ? LA_ERR_INFEASIBLE : LA_ERR_OVERFLOW));
            break;
        }
        const unsigned long long nk = pack_key(nq, (uint32_t)row);
        unsigned long long old = 0;
        if (lane == 0) {
            old = atomicMin(key + r.w, nk);
            atomicMax(qm + r.w, old > nk ? nq : key_q(old));
        }
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
    if (lane == 0 && total) {
        atomicAdd(&ctrl->scans, (unsigned long long)pending);
        atomicAdd(&ctrl->wins, wins);
        atomicAdd(&ctrl->displaced, displaced);
        atomicAdd(&ctrl->full_scans, total);
        atomicMax(&ctrl->max_chain, total);
    }
}

// The matching from the column keys; the exact cost sums the cheapest arc of
// every matched pair.
__global__ void k_sp_finalize(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ cols,
                              const int32_t *__restrict__ costs, int n, const unsigned long long *__restrict__ key,
                              int32_t *match, long long *cost, long long *prices, Ctrl *ctrl, int slot) {
    long long sum = 0;
    const unsigned long long qmin = prices ? ctrl->qmin[slot] : 0;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const unsigned long long k = key[y];
        const uint32_t m = key_mate(k);
        if (m >= (uint32_t)n) {
            sp_set_status(ctrl, LA_ERR_INTERNAL);
            continue;
        }
        if (match) match[m] = y;
        int best = INT_MAX;
        bool found = false;
        for (int a = row_ptr[m]; a < row_ptr[m + 1]; ++a)
            if (cols[a] == y) {
                best = min(best, costs[a]);
                found = true;
            }
        if (!found) sp_set_status(ctrl, LA_ERR_INTERNAL);
        sum += best;
        if (prices) prices[y] = -(long long)(key_q(k) - qmin);
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(cost), (unsigned long long)sum);
}

struct SparseWorkspace {
    int64_t cap = 0;
    unsigned long long *key = nullptr;
    unsigned long long *qm = nullptr;
    int *colseen = nullptr;
    Ctrl *ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;
    int num_sms = 0;
    int occ = 0;
    bool events = false;
    cudaEvent_t ev[2];
};

std::mutex g_smu;
SparseWorkspace g_sws[kMaxDevices];

la_status ensure_sws(SparseWorkspace &w, int64_t n) {
    if (!w.ctrl) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
        if (cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return LA_ERR_CUDA;
        if (cudaMalloc(&w.ctrl, sizeof(Ctrl)) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMallocHost(&w.h_ctrl, sizeof(Ctrl)) != cudaSuccess) return LA_ERR_NOMEM;
        for (auto &e : w.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return LA_ERR_CUDA;
        w.events = true;
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_sp_refine<false>, kBlock, 0);
        w.occ = std::max(1, o);
    }
    if (w.cap < n) {
        cudaFree(w.key);
        cudaFree(w.qm);
        cudaFree(w.colseen);
        w.key = nullptr;
        w.qm = nullptr;
        w.colseen = nullptr;
        w.cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1024);
        if (cudaMalloc(&w.key, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.qm, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.colseen, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        w.cap = cap;
    }
    return LA_OK;
}

}  // namespace

#define LA_SCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

static la_status sparse_locked(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs, int32_t n,
                               int32_t nnz, const la_options *opt, cudaStream_t s, int32_t *match_out,
                               int64_t *cost_out, la_stats *st) {
    const int alpha = (opt && opt->alpha) ? opt->alpha : 10;
    const int64_t eps0 = opt ? opt->eps0 : 0;
    int64_t *prices_out = opt ? opt->prices_out : nullptr;
    const bool profile = opt && opt->profile;
    if (alpha < 2 || eps0 < 0 || (opt && opt->scan_budget < 0) || (opt && opt->init_prices)) return LA_ERR_INVALID;
    la_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    stats.n = n;
    stats.wide = 1;
    if (n == 0) {
        LA_SCK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
        LA_SCK(cudaStreamSynchronize(s));
        if (st) *st = stats;
        return LA_OK;
    }
    int dev = 0;
    LA_SCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    SparseWorkspace &w = g_sws[dev];
    if (la_status e = ensure_sws(w, n)) return e;

    Ctrl init;
    std::memset(&init, 0, sizeof(init));
    init.cmin = INT_MAX;
    init.cmax = INT_MIN;
    init.qmin[0] = init.qmin[1] = ~0ull;
    *w.h_ctrl = init;
    LA_SCK(cudaMemcpyAsync(w.ctrl, w.h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    LA_SCK(cudaMemsetAsync(w.colseen, 0, sizeof(int) * n, s));
    int64_t launches = 0;
    const int vg = std::max(1, std::min((std::max(n, nnz) + kBlock - 1) / kBlock, 8 * w.num_sms));
    k_sp_validate<<<vg, kBlock, 0, s>>>(row_ptr, cols, costs, n, nnz, w.colseen, w.ctrl);
    const int sg = std::max(1, std::min((n + kBlock - 1) / kBlock, 4 * w.num_sms));
    k_sp_colcheck<<<sg, kBlock, 0, s>>>(w.colseen, n, w.ctrl);
    launches += 2;
    LA_SCK(cudaGetLastError());
    LA_SCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_SCK(cudaStreamSynchronize(s));
    const Ctrl c0 = *w.h_ctrl;
    if (c0.status) return (la_status)c0.status;
    if (c0.colseen_missing) {   // a row or a column without arcs: Hall's condition fails
        if (st) *st = stats;
        return LA_ERR_INFEASIBLE;
    }
    const unsigned long long np1 = (unsigned long long)n + 1;
    const unsigned long long Ct = np1 * (unsigned long long)((long long)c0.cmax - (long long)c0.cmin);
    stats.scaled_range = (int64_t)Ct;
    if (Ct >= (1ull << 40)) return LA_ERR_OVERFLOW;
    std::vector<unsigned long long> sched;
    {
        unsigned long long e = eps0 > 0 ? (unsigned long long)eps0 : Ct;
        do {
            e = std::max<unsigned long long>(1, e / (unsigned long long)alpha);
            sched.push_back(e);
        } while (e > 1 && sched.size() < 64);
        if (sched.back() != 1) return LA_ERR_INVALID;
    }
    stats.eps_first = (int64_t)sched[0];
    const unsigned long long qlim = kQMax - 1;
    const unsigned long long budget = opt && opt->scan_budget ? (unsigned long long)opt->scan_budget
                                                              : 256ull * n * (sched.size() + 1) + (1ull << 22);
    const int grid = std::max(1, std::min(w.num_sms * w.occ, (n + kBlock / 32 - 1) / (kBlock / 32)));
    if (profile) LA_SCK(cudaEventRecord(w.ev[0], s));
    // feasibility phase: zero costs, eps = 1, prices from 0
    k_sp_reset<<<sg, kBlock, 0, s>>>(w.key, w.qm, n, qlim, w.ctrl, 0, 0, 1);
    k_sp_refine<true><<<grid, kBlock, 0, s>>>(row_ptr, cols, costs, n, c0.cmin, (uint32_t)np1, 1ull, qlim,
                                              4ull * (unsigned long long)n + 4, w.key, w.qm, w.ctrl, budget);
    launches += 2;
    // cost phases (Algorithm 5.0), from zero prices again
    int ph = 0;
    for (; ph < (int)sched.size(); ++ph) {
        const int slot = ph & 1;
        if (ph > 0) {
            k_sp_qmin<<<sg, kBlock, 0, s>>>(w.key, n, w.ctrl, slot);
            ++launches;
        }
        k_sp_reset<<<sg, kBlock, 0, s>>>(w.key, w.qm, n, qlim, w.ctrl, slot, ph + 1, ph == 0);
        k_sp_refine<false><<<grid, kBlock, 0, s>>>(row_ptr, cols, costs, n, c0.cmin, (uint32_t)np1, sched[ph],
                                                   qlim, ~0ull, w.key, w.qm, w.ctrl, budget);
        launches += 2;
    }
    if (profile) LA_SCK(cudaEventRecord(w.ev[1], s));
    const int fslot = ph & 1;
    if (prices_out) {
        k_sp_qmin<<<sg, kBlock, 0, s>>>(w.key, n, w.ctrl, fslot);
        ++launches;
    }
    LA_SCK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
    k_sp_finalize<<<sg, kBlock, 0, s>>>(row_ptr, cols, costs, n, w.key, match_out,
                                        reinterpret_cast<long long *>(cost_out),
                                        reinterpret_cast<long long *>(prices_out), w.ctrl, fslot);
    ++launches;
    LA_SCK(cudaGetLastError());
    LA_SCK(cudaMemcpyAsync(w.h_ctrl, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_SCK(cudaStreamSynchronize(s));
    const Ctrl c1 = *w.h_ctrl;
    stats.phases = (int64_t)sched.size();
    stats.scans = (int64_t)c1.scans;
    stats.wins = (int64_t)c1.wins;
    stats.displaced = (int64_t)c1.displaced;
    stats.launches = launches;
    stats.refine_launches = (int64_t)sched.size() + 1;
    stats.max_chain = (int64_t)c1.max_chain;
    stats.full_scans = (int64_t)c1.full_scans;
    for (int k = 0; k <= ph && k < LA_STATS_PHASES; ++k) {
        // phase 0 of the counters is the feasibility phase
        const unsigned long long end = (k < ph) ? c1.phase_start_scans[k + 1] : c1.scans;
        stats.phase_scans[k] = (int64_t)(end - c1.phase_start_scans[k]);
    }
    if (profile) {
        float t = 0;
        LA_SCK(cudaEventElapsedTime(&t, w.ev[0], w.ev[1]));
        stats.refine_ms = t;
    }
    if (st) *st = stats;
    return (la_status)c1.status;
}

extern "C" {

la_status la_solve_sparse_ex(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs, int32_t n,
                             int32_t nnz, const la_options *opt, void *stream, int32_t *match_out,
                             int64_t *cost_out, la_stats *stats_out) {
    if (n < 0 || n > LA_MAX_N || nnz < 0 || !cost_out || (n > 0 && (!row_ptr || (nnz > 0 && (!cols || !costs)))))
        return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_smu);
    return sparse_locked(row_ptr, cols, costs, n, nnz, opt, static_cast<cudaStream_t>(stream), match_out, cost_out,
                         stats_out);
}

la_status la_solve_sparse(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs, int32_t n,
                          int32_t nnz, void *stream, int32_t *match_out, int64_t *cost_out) {
    return la_solve_sparse_ex(row_ptr, cols, costs, n, nnz, nullptr, stream, match_out, cost_out, nullptr);
}

}  // extern "C"
