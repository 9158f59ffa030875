// la_solve / la_solve_ex: dense assignment by cost scaling with a lock-free
// parallel refine on one GPU.
//
// Outer loop (Sect. 5.1, Algorithm 5.0): eps starts at C~ = (n+1)(max C -
// min C) and every phase runs refine at eps <- max(1, floor(eps / alpha));
// the phase at eps = 1 is the last. Costs are scaled by n + 1 so that an
// eps = 1 optimal assignment is exactly optimal.
//
// Refine (Algorithm 5.2's initialisation + Algorithm 5.4's push/relabel as a
// Goldberg-Kennedy double push), one phase per launch of k_refine:
//   * f <- 0: every column's mate is cleared, its price is kept; the row
//     prices are implicit, p(x) = -min_y (c'_p(x,y) + eps).
//   * each warp of a persistent grid takes a free row x from a device queue
//     and scans its cost row with 128-bit loads for the best (b1 at w) and
//     second best (b2) part-reduced cost v(x,y) = c~(x,y) - p(y);
//   * it bids q(w) <- q_read(w) + (b2 - b1) + eps (that is, p(w) drops by
//     second - best + eps) with one 64-bit atomicMin on the column key that
//     packs (price, mate): a win is the push x -> w, the relabel of w and the
//     push of w's old mate back, all at once. The displaced mate becomes
//     the warp's next row; a lost bid rescans the same row.
//   * the phase ends when the queue is empty and every warp's row is
//     matched; no host round trip inside a phase.
// A row is scanned through its exact candidate list when the list decides
// its bid (la_lists.cuh), and once a phase is down to a few free rows, the
// refine hands them to k_tail, which finishes their displacement chains on
// one CTA with the keys in shared memory; a second refine launch takes any
// rows the tail kernel gives back.
// Lemma 5.2 (prices never increase) makes stale price reads safe: they can
// only make a bid lose, and a row holding a column keeps its
// eps-complementary slackness while other prices fall.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "la.h"
#include "la_device.cuh"
#include "la_lists.cuh"

using namespace la;

namespace {

constexpr int kMaxPhases = 64;
constexpr int kMaxDevices = 64;
constexpr int kDefaultBlock = 256;
constexpr unsigned long long kRangeLimit = 1ull << 40;  // C~ limit (LA_ERR_OVERFLOW)
constexpr int kTailMaxN = 16384;      // shared-memory keys of the tail kernel (128 KB)
// Threads of the one-CTA tail kernel: 64-bit values run four insertion
// chains per full scan and need the registers of a 512-thread CTA.
template <bool WIDE>
constexpr int tail_threads() { return WIDE ? 512 : 1024; }
constexpr int kDefaultTailRows = 32;
constexpr unsigned kTailGiveUpFull = 16;   // full scans before the tail kernel may give its rows back
constexpr int kDefaultPuRounds = 0;   // global price updates per phase (off unless asked)

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ void set_status(Ctrl *ctrl, int s) {
    atomicCAS(&ctrl->status, 0, s);
}

// min / max of the cost matrix (one pass).
__global__ void k_minmax(const int32_t *__restrict__ C, long long total, Ctrl *ctrl) {
    int lo = INT_MAX, hi = INT_MIN;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(C) & 15) == 0) {
        const long long nv = total >> 2;
        const int4 *C4 = reinterpret_cast<const int4 *>(C);
        for (long long i = tid; i < nv; i += stride) {
            const int4 c = ld_row4(C4 + i);
            lo = min(lo, min(min(c.x, c.y), min(c.z, c.w)));
            hi = max(hi, max(max(c.x, c.y), max(c.z, c.w)));
        }
        for (long long i = (nv << 2) + tid; i < total; i += stride) {
            const int c = C[i];
            lo = min(lo, c);
            hi = max(hi, c);
        }
    } else {
        for (long long i = tid; i < total; i += stride) {
            const int c = C[i];
            lo = min(lo, c);
            hi = max(hi, c);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&ctrl->cmin, lo);
        atomicMax(&ctrl->cmax, hi);
    }
}

// n == 1: the only matching.
__global__ void k_single(const int32_t *C, int32_t *match, long long *cost, long long *prices) {
    if (match) match[0] = 0;
    *cost = C[0];
    if (prices) prices[0] = 0;
}

// Warm start, step 1: max of the given prices.
__global__ void k_warm_pmax(const long long *__restrict__ p, int n, Ctrl *ctrl) {
    long long m = LLONG_MIN;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x)
        m = max(m, p[y]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ctrl->pmax, m);
}

// Warm start, step 2: q(y) = max p - p(y) >= 0 (a uniform shift), keys with
// no mate, and the spread max q for the range check.
__global__ void k_warm_init(const long long *__restrict__ p, int n, unsigned long long *key, Ctrl *ctrl) {
    unsigned long long spread = 0;
    const long long pm = ctrl->pmax;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        unsigned long long q = (unsigned long long)(pm - p[y]);
        if (pm - p[y] < 0) q = kQMax;       // wrapped difference: far out of range
        spread = max(spread, q);
        key[y] = pack_key(min(q, kQMax - 1), kNone);
    }
    for (int o = 16; o; o >>= 1) spread = max(spread, __shfl_xor_sync(0xffffffffu, spread, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ctrl->qspread, spread);
}

// Smallest q over the columns (for the per-phase shift).
__global__ void k_qmin(const unsigned long long *__restrict__ key, int n, Ctrl *ctrl, int slot) {
    unsigned long long m = ~0ull;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x)
        m = min(m, key_q(__ldcg(key + y)));
    for (int o = 16; o; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(&ctrl->qmin[slot], m);
}

// Phase initialisation (Algorithm 5.2, refine initialisation): clear every
// mate (f <- 0), keep prices shifted so that min q = 0, refresh the price
// mirror and reset the row queue.
template <bool WIDE>
__global__ void k_reset(unsigned long long *__restrict__ key, void *__restrict__ qmv, int n,
                        unsigned long long qlim, Ctrl *ctrl, int slot, int phase, int pu_rounds) {
    const unsigned long long qmin = ctrl->qmin[slot];
    bool bad = false;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const unsigned long long q = key_q(key[y]) - qmin;
        bad |= q > qlim;
        key[y] = pack_key(q, kNone);
        if (WIDE) static_cast<unsigned long long *>(qmv)[y] = q;
        else static_cast<uint32_t *>(qmv)[y] = (uint32_t)q;
    }
    if (bad) set_status(ctrl, LA_ERR_OVERFLOW);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->next_row = 0;
        ctrl->qmin[slot ^ 1] = ~0ull;
        ctrl->phase_start_scans[phase & 63] = ctrl->scans;
        ctrl->phase_start_full[phase & 63] = ctrl->full_scans;
        ctrl->phase_start_tail[phase & 63] = ctrl->tail_scans;
        if (*reinterpret_cast<volatile int *>(&ctrl->status) == 0) ctrl->phase_now = phase;
        ctrl->rebase_total += qmin;
        ctrl->free_rows = n;
        ctrl->handoff = 0;
        ctrl->tail_count = 0;
        ctrl->ph_full = 0;
        ctrl->ph_hits = 0;
        ctrl->qmode = 0;
        ctrl->qlen = n;
        ctrl->pu_left = pu_rounds;
        ctrl->pu_mark = ctrl->scans;
    }
}

// The refine phase: persistent grid, one warp per free row.
//
// With mode 1, the launch is the phase's bulk sweep: every row of the
// queue bids once, and the row its bid leaves free (the displaced mate, or
// the row itself after a lost bid) is queued for the next launch instead of
// bidding at once. The last block to finish makes that queue the current
// one. The sweep is the bandwidth part of a phase (each row's first scan,
// all rows in flight); the launch after it carries the displacement chains.
// Mode 2 is a chain launch that hands its rows to the team refine (k_team)
// once at most ctrl->team_T rows are free; mode 0 a chain launch without.
template <bool WIDE, bool VEC>
__global__ void __launch_bounds__(256)
k_refine(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long eps,
         unsigned long long qlim, unsigned long long *__restrict__ key, void *__restrict__ qmv,
         Ctrl *__restrict__ ctrl, unsigned long long budget, RowLists L, int tail_T,
         int *__restrict__ tail_rows, int pu_T, int *__restrict__ qlist0,
         int *__restrict__ qlist1, int stop_free, int mode) {
    constexpr unsigned kFlush = 8;       // scans between budget / status / hand-off checks
    const bool sweep = mode == 1;
    int miss = 0;                        // this warp's consecutive scans that the lists did not answer
    const int lane = threadIdx.x & 31;
    const unsigned long long R = ctrl->rebase_total;
    const int qmode = ctrl->qmode, qlen = ctrl->qlen;
    const int *qlist = ctrl->qsel ? qlist1 : qlist0;
    int *pend_list = ctrl->qsel ? qlist0 : qlist1;     // sweep: rows left free by its bids
    const bool pu_on = pu_T > 0 && ctrl->pu_left > 0;
    int row = -1;
    unsigned long long wins = 0, displaced = 0, total = 0, full = 0, hits = 0;
    unsigned long long full_pub = 0, hits_pub = 0;   // already added to the phase counters
    unsigned pending = 0;
    for (;;) {
        if (row < 0) {
            int r = 0;
            if (lane == 0) {
                r = atomicAdd(&ctrl->next_row, 1);
                if (qmode) r = r < qlen ? __ldcg(qlist + r) : n;
            }
            row = __shfl_sync(0xffffffffu, r, 0);
            if (row >= n) break;
        }
        if (pending == kFlush) {
            unsigned long long s = 0;
            int st = 0, ho = 0;
            if (lane == 0) {
                s = atomicAdd(&ctrl->scans, (unsigned long long)kFlush);
                st = *reinterpret_cast<volatile int *>(&ctrl->status);
                ho = *reinterpret_cast<volatile int *>(&ctrl->handoff);
                if (tail_T > 0) {
                    atomicAdd(&ctrl->ph_full, full - full_pub);
                    atomicAdd(&ctrl->ph_hits, hits - hits_pub);
                }
                // Few free rows and a stretch of bidding since the last update:
                // stop here for a global price update (Alg. 5.3).
                if (!ho && pu_on) {
                    const int fr = *reinterpret_cast<volatile int *>(&ctrl->free_rows);
                    const unsigned long long mark = *reinterpret_cast<volatile unsigned long long *>(&ctrl->pu_mark);
                    if (fr <= pu_T && s >= mark + 8ull * (unsigned long long)pu_T + 256ull) {
                        atomicCAS(&ctrl->handoff, 0, 2);
                        ho = 2;
                    }
                }
            }
            full_pub = full;
            hits_pub = hits;
            s = __shfl_sync(0xffffffffu, s, 0);
            st = __shfl_sync(0xffffffffu, st, 0);
            ho = __shfl_sync(0xffffffffu, ho, 0);
            pending = 0;
            if (st != 0) break;
            if (s + kFlush > budget) {
                if (lane == 0) set_status(ctrl, LA_ERR_ITER_LIMIT);
                break;
            }
            if (ho == 3) break;   // the phase was cut short: its last rows stay free
            if (ho) {   // few free rows left: the tail kernel takes this one
                if (lane == 0) tail_rows[atomicAdd(&ctrl->tail_count, 1)] = row;
                break;
            }
        }
        ++pending;
        ++total;
        bool was_full = false;
        // After three misses in a row the lists are stale for this stretch
        // of the phase (a large eps moves prices past theta after a bid or
        // two): go straight to a full scan for the best two only, trying the
        // list again every 8th scan. A full scan first asks L2 for the whole
        // row, so that a lone warp's dependent loads do not wait on HBM.
        const bool try_list = miss < 3 || (total & 7) == 0;
        const auto t = scan_for_bid<WIDE, VEC, false, 1>(C, row, n, cmin, np1, MirrorPrices<WIDE>{qmv}, lane, L, R, was_full,
                                                           ListAhead{-1, 0ull, {}}, try_list, true, true);
        if (was_full) {
            ++full;
            ++miss;
        } else {
            ++hits;
            miss = 0;
        }
        __syncwarp();
        // double push: x -> w, relabel w, w's old mate becomes free
        const unsigned long long qw = (unsigned long long)(t.b1 - t.c1);
        const unsigned long long nq = qw + (t.b2 - t.b1) + eps;
        if (t.w >= n || nq > qlim) {
            if (lane == 0) set_status(ctrl, t.w >= n ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW);
            break;
        }
        const unsigned long long nk = pack_key(nq, (uint32_t)row);
        unsigned long long old = 0;
        if (lane == 0) {
            old = atomicMin(key + t.w, nk);
            const unsigned long long qnow = old > nk ? nq : key_q(old);
            if (WIDE) atomicMax(static_cast<unsigned long long *>(qmv) + t.w, qnow);
            else atomicMax(static_cast<uint32_t *>(qmv) + t.w, (uint32_t)qnow);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        if (sweep) {   // one bid per row: the row left free waits for the chain launch
            int left = -1;
            if (old > nk) {
                ++wins;
                const uint32_t m = key_mate(old);
                if (m != kNone) {
                    ++displaced;
                    left = (int)m;
                } else if (lane == 0) {
                    atomicSub(&ctrl->free_rows, 1);
                }
            } else {
                left = row;
            }
            if (lane == 0 && left >= 0) pend_list[atomicAdd(&ctrl->pend, 1)] = left;
            row = -1;
            continue;
        }
        if (old > nk) {
            ++wins;
            const uint32_t m = key_mate(old);
            if (m != kNone) {
                ++displaced;
                row = (int)m;
            } else {
                row = -1;
                // Hand the last rows to the one-CTA tail kernel only while
                // the candidate lists answer most scans (>= 3 of 4): its
                // single SM is then spent on cheap list scans, not rescans.
                if (lane == 0 && (tail_T > 0 || mode == 2 || pu_on || stop_free > 0)) {
                    const int fr = atomicSub(&ctrl->free_rows, 1) - 1;
                    // An intermediate phase only prepares prices for the next
                    // one, whose initialisation makes any prices eps-optimal
                    // (Alg. 5.2): it may stop with a few rows still free.
                    if (stop_free > 0 && fr <= stop_free) atomicCAS(&ctrl->handoff, 0, 3);
                    if (mode == 2 && fr <= ctrl->team_T) {
                        // at most one free row per team CTA: the team refine takes over
                        if (atomicCAS(&ctrl->handoff, 0, 4) == 0) ctrl->team_go = 1;
                    } else if (!pu_on && tail_T > 0 && fr <= tail_T) {
                        const unsigned long long pf = *reinterpret_cast<volatile unsigned long long *>(&ctrl->ph_full);
                        const unsigned long long ph = *reinterpret_cast<volatile unsigned long long *>(&ctrl->ph_hits);
                        if (ph >= 3 * pf) atomicCAS(&ctrl->handoff, 0, 1);
                    }
                }
            }
        }
        // else: a lower price got there first; rescan this row
    }
    if (lane == 0 && total) {
        atomicAdd(&ctrl->scans, (unsigned long long)pending);
        atomicAdd(&ctrl->wins, wins);
        atomicAdd(&ctrl->displaced, displaced);
        atomicAdd(&ctrl->full_scans, full);
        atomicAdd(&ctrl->list_scans, hits);
        atomicMax(&ctrl->max_chain, total);
        if (sweep) {
            atomicAdd(&ctrl->sweep_scans, total);
            atomicAdd(&ctrl->sweep_full, full);
        }
    }
    if (sweep) {
        // The last block to finish makes the rows left free the current
        // queue (the next launch reads it; the launch boundary orders the
        // writes). Every warp of every block reaches this point.
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&ctrl->sweep_done, 1u) == gridDim.x - 1) {
                __threadfence();
                ctrl->qsel ^= 1;
                ctrl->qmode = 1;
                ctrl->qlen = *reinterpret_cast<volatile int *>(&ctrl->pend);
                ctrl->next_row = 0;
                ctrl->pend = 0;
                ctrl->sweep_done = 0;
            }
        }
    }
}

// Team refine (on unless LA_FLAG_NO_TEAM_REFINE). Once at most one row per CTA of its
// grid is free, the refine's chains are latency bound, and where the lists
// keep failing each step is a lone warp's full scan: n / 32 values ranked
// per lane behind n / 1024 dependent rounds of loads. Here a CTA of
// kTeamWarps warps carries one chain and every warp ranks its own slice of
// the row: the best two only once the lists keep failing, as the refine
// does, else the lanes' best kListK, merged into the row's new list;
// thread 0 merges the slices and commits the same double push. A list scan
// is warp 0's alone. The rows are a refine launch's hand-off (tail_rows and the
// rest of the queue). When at most tail_T rows are free and the lists
// answer (as for the refine's own hand-off), or when a price update is due
// (pu_T, as in the refine), the rows still held and those never claimed
// become the queue of the next kernel (the one-CTA tail kernel, or k_pu and
// the refine launch after it); the last CTA to finish sets it up.
constexpr int kTeamWarps = 8;

template <bool WIDE, bool VEC>
__global__ void __launch_bounds__(32 * kTeamWarps)
k_team(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long eps,
       unsigned long long qlim, unsigned long long *__restrict__ key, void *__restrict__ qmv,
       Ctrl *__restrict__ ctrl, unsigned long long budget, RowLists L, int tail_T,
       const int *__restrict__ tail_rows, int *__restrict__ qlist0, int *__restrict__ qlist1, int stop_free,
       int pu_T) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    constexpr unsigned kFlush = 8;
    __shared__ ScanResult<V> s_part[kTeamWarps];
    __shared__ V s_kv[kTeamWarps][kListK][32];     // list rebuild: each warp's lane lists
    __shared__ int s_kw[kTeamWarps][kListK][32];
    __shared__ int s_kc[kTeamWarps][32];
    __shared__ int s_row, s_exit, s_try, s_ok;
    // team_go stays set for the whole launch (handoff may move on from 4),
    // so every CTA takes part and the last one to finish is seen
    if (*reinterpret_cast<volatile int *>(&ctrl->team_go) == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long R = ctrl->rebase_total;
    const int qmode = ctrl->qmode, qlen = ctrl->qlen, qsel = ctrl->qsel, tc = ctrl->tail_count;
    const int *qold = qsel ? qlist1 : qlist0;
    int *qnew = qsel ? qlist0 : qlist1;   // the tail kernel's queue, if it takes over
    const int qend = qmode ? qlen : n;
    const int q0 = min(ctrl->next_row, qend);
    const int items = tc + (qend - q0);
    // this warp's slice of a row (16-byte aligned when VEC)
    int y0, y1;
    if (VEC) {
        const int g = ((n >> 2) + kTeamWarps - 1) / kTeamWarps;
        y0 = min(n, 4 * g * warp);
        y1 = min(n, 4 * g * (warp + 1));
    } else {
        const int g = (n + kTeamWarps - 1) / kTeamWarps;
        y0 = min(n, g * warp);
        y1 = min(n, g * (warp + 1));
    }
    const MirrorPrices<WIDE> prices{qmv};
    const V inf = (V)~(V)0;
    // thread 0's state
    int row = -1, miss = 0, fail = 0;
    unsigned pending = 0;
    unsigned long long wins = 0, displaced = 0, total = 0, full = 0, hits = 0, chain = 0, longest = 0;
    unsigned long long full_pub = 0, hits_pub = 0;
    for (;;) {
        __syncthreads();   // the last step's shared results have been read
        if (tid == 0) {
            int ex = fail ? 2 : 0;
            if (!ex && row < 0) {
                longest = max(longest, chain);
                chain = 0;
                const int k = atomicAdd(&ctrl->team_next, 1);
                if (k >= items) ex = 1;
                else row = k < tc ? __ldcg(tail_rows + k) : (qmode ? __ldcg(qold + q0 + (k - tc)) : q0 + (k - tc));
            }
            if (!ex && pending >= kFlush) {
                const unsigned long long sc = atomicAdd(&ctrl->scans, (unsigned long long)pending);
                atomicAdd(&ctrl->ph_full, full - full_pub);
                atomicAdd(&ctrl->ph_hits, hits - hits_pub);
                full_pub = full;
                hits_pub = hits;
                pending = 0;
                const int st = *reinterpret_cast<volatile int *>(&ctrl->status);
                int ho = *reinterpret_cast<volatile int *>(&ctrl->handoff);
                // few free rows and a stretch of bidding since the last update:
                // stop for a global price update, as the refine does
                if (ho == 4 && pu_T > 0 && *reinterpret_cast<volatile int *>(&ctrl->pu_left) > 0) {
                    const int fr = *reinterpret_cast<volatile int *>(&ctrl->free_rows);
                    const unsigned long long mark = *reinterpret_cast<volatile unsigned long long *>(&ctrl->pu_mark);
                    if (fr <= pu_T && sc >= mark + 8ull * (unsigned long long)pu_T + 256ull) {
                        atomicCAS(&ctrl->handoff, 4, 2);
                        ho = *reinterpret_cast<volatile int *>(&ctrl->handoff);
                    }
                }
                if (st != 0 || ho == 3) {
                    ex = 2;
                } else if (sc + kFlush > budget) {
                    set_status(ctrl, LA_ERR_ITER_LIMIT);
                    ex = 2;
                } else if (ho == 1 || ho == 2) {   // the tail kernel or the price update takes this row
                    qnew[atomicAdd(&ctrl->team_back, 1)] = row;
                    row = -1;
                    ex = 3;
                }
            }
            s_row = row;
            s_exit = ex;
            s_try = L.cols && (miss < 3 || (total & 7) == 0);
            s_ok = 0;
        }
        __syncthreads();
        if (s_exit) break;
        const int r = s_row;
        const int32_t *crow = C + (size_t)r * n;
        if (s_try && warp == 0) {   // uniform across the CTA
            unsigned long long th = 0;
            const auto t = list_scan<WIDE, false>(r, n, cmin, np1, prices, lane, L, ListAhead{-1, 0ull, {}}, th);
            // exact when the list's second best does not exceed theta (see scan_for_bid)
            const bool ok = th != 0 && (th == ~0ull || (unsigned long long)t.b2 + R + 1 <= th);
            if (lane == 0) {
                s_ok = ok;
                if (ok) s_part[0] = t;
            }
        }
        if (s_try) __syncthreads();
        const bool ok = s_ok != 0;
        // A list that was tried and failed is rebuilt, as the refine does:
        // every warp keeps its lanes' kListK best pairs over its slice, and
        // lane l of warp 0 merges the eight lists of lane l (columns outside
        // them lost kListK times within that lane's columns, so theta keeps
        // its meaning). In a stretch of failing lists (no try) the best two
        // of each slice are enough.
        const bool build = !ok && s_try;
        if (build) {
            LaneK<V, kListK> t;
            int cnt;
            scan_topk_range<WIDE, VEC>(crow, y0, y1, cmin, np1, prices, lane, t, cnt);
#pragma unroll
            for (int k = 0; k < kListK; ++k) {
                s_kv[warp][k][lane] = t.b[k];
                s_kw[warp][k][lane] = t.w[k];
            }
            s_kc[warp][lane] = cnt;
            __syncthreads();
            if (warp == 0) {
                LaneK<V, kListK> m;
                lanek_init(m);
                int c = 0;
                for (int w = 0; w < kTeamWarps; ++w) {
                    c += s_kc[w][lane];
#pragma unroll
                    for (int k = 0; k < kListK; ++k)   // an empty entry (~0, -1) inserts nothing
                        lanek_insert<V, kListK>(m, s_kv[w][k][lane], s_kw[w][k][lane]);
                }
                int craw[kListK];
#pragma unroll
                for (int k = 0; k < kListK; ++k) craw[k] = m.w[k] >= 0 ? ld_row1(crow + m.w[k]) : 0;
                const size_t base = (size_t)r * kListLen + kListK * lane;
#pragma unroll
                for (int g = 0; g < kListK / 4; ++g) {
                    reinterpret_cast<int4 *>(L.cols + base)[g] =
                        make_int4(m.w[4 * g], m.w[4 * g + 1], m.w[4 * g + 2], m.w[4 * g + 3]);
                    reinterpret_cast<int4 *>(L.costs + base)[g] =
                        make_int4(craw[4 * g], craw[4 * g + 1], craw[4 * g + 2], craw[4 * g + 3]);
                }
                const V th = warp_min<V>(c > kListK ? m.b[kListK - 1] : inf);
                if (lane == 0) L.theta[r] = th == inf ? ~0ull : (unsigned long long)th + R + 1;
                __threadfence();   // the list is complete before this row can change hands
                ScanResult<V> res{m.b[0], m.b[1], m.w[0] >= 0 ? (V)(uint32_t)(craw[0] - cmin) * np1 : (V)0,
                                  m.w[0] < 0 ? INT_MAX : m.w[0]};
                warp_merge(res);
                if (lane == 0) s_part[0] = res;
            }
            __syncthreads();
        } else if (!ok) {
            const auto t = scan_top2_range<WIDE, VEC>(crow, y0, y1, cmin, np1, prices, lane);
            if (lane == 0) s_part[warp] = t;
            __syncthreads();
        }
        if (tid == 0) {
            ScanResult<V> m = s_part[0];
            if (!ok && !build) {   // lowest value, then lowest column; the second best over every slice
                for (int k = 1; k < kTeamWarps; ++k) {
                    const ScanResult<V> p = s_part[k];
                    if (p.b1 < m.b1 || (p.b1 == m.b1 && (unsigned)p.w < (unsigned)m.w)) {
                        m.b2 = min(m.b1, p.b2);
                        m.b1 = p.b1;
                        m.c1 = p.c1;
                        m.w = p.w;
                    } else {
                        m.b2 = min(m.b2, p.b1);
                    }
                }
                if (m.b2 == inf) m.b2 = m.b1;
            }
            ++pending;
            ++total;
            ++chain;
            if (ok) {
                ++hits;
                miss = 0;
            } else {
                ++full;
                ++miss;
            }
            // double push: x -> w, relabel w, w's old mate becomes free
            const unsigned long long nq = (unsigned long long)(m.b1 - m.c1) + (m.b2 - m.b1) + eps;
            if (m.w < 0 || m.w >= n || nq > qlim) {
                set_status(ctrl, (m.w < 0 || m.w >= n) ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW);
                fail = 1;
            } else {
                const unsigned long long nk = pack_key(nq, (uint32_t)r);
                const unsigned long long old = atomicMin(key + m.w, nk);
                const unsigned long long qnow = old > nk ? nq : key_q(old);
                if (WIDE) atomicMax(static_cast<unsigned long long *>(qmv) + m.w, qnow);
                else atomicMax(static_cast<uint32_t *>(qmv) + m.w, (uint32_t)qnow);
                if (old > nk) {
                    ++wins;
                    const uint32_t mate = key_mate(old);
                    if (mate != kNone) {
                        ++displaced;
                        row = (int)mate;
                    } else {
                        row = -1;
                        const int fr = atomicSub(&ctrl->free_rows, 1) - 1;
                        if (stop_free > 0 && fr <= stop_free) atomicCAS(&ctrl->handoff, 4, 3);
                        if (pu_T == 0 && tail_T > 0 && fr <= tail_T) {   // no update left in this phase
                            const unsigned long long pf = *reinterpret_cast<volatile unsigned long long *>(&ctrl->ph_full);
                            const unsigned long long ph = *reinterpret_cast<volatile unsigned long long *>(&ctrl->ph_hits);
                            if (ph >= 3 * pf) atomicCAS(&ctrl->handoff, 4, 1);
                        }
                    }
                }
                // else: a lower price got there first; rescan this row
            }
        }
    }
    if (tid == 0) {
        longest = max(longest, chain);
        atomicAdd(&ctrl->scans, (unsigned long long)pending);
        atomicAdd(&ctrl->ph_full, full - full_pub);
        atomicAdd(&ctrl->ph_hits, hits - hits_pub);
        if (total) {
            atomicAdd(&ctrl->wins, wins);
            atomicAdd(&ctrl->displaced, displaced);
            atomicAdd(&ctrl->full_scans, full);
            atomicAdd(&ctrl->list_scans, hits);
            atomicAdd(&ctrl->team_scans, total);
            atomicAdd(&ctrl->team_full, full);
            atomicMax(&ctrl->max_chain, longest);
        }
        __threadfence();
        if (atomicAdd(&ctrl->team_done, 1u) == gridDim.x - 1) {   // every CTA has finished
            __threadfence();
            const int ho = *reinterpret_cast<volatile int *>(&ctrl->handoff);
            if (ho == 1 || ho == 2) {
                // rows never claimed go to the next kernel too
                int back = *reinterpret_cast<volatile int *>(&ctrl->team_back);
                for (int k = min(*reinterpret_cast<volatile int *>(&ctrl->team_next), items); k < items; ++k)
                    qnew[back++] = k < tc ? __ldcg(tail_rows + k) : (qmode ? __ldcg(qold + q0 + (k - tc)) : q0 + (k - tc));
                ctrl->qsel = qsel ^ 1;
                ctrl->qlen = back;
            } else {
                if (ho == 4) ctrl->handoff = 0;   // the phase ended here
                ctrl->qlen = 0;
            }
            ctrl->qmode = 1;
            ctrl->next_row = 0;
            ctrl->tail_count = 0;
            ctrl->team_next = 0;
            ctrl->team_back = 0;
            ctrl->team_done = 0;
            ctrl->team_go = 0;
            ctrl->team_phases += 1;
        }
    }
}

constexpr unsigned kMaxPuLevel = 2048;
// Labels are kept clamped at kLabelTop: every update truncates them at a
// level K <= kMaxPuLevel, and the fixed point of the clamped relaxation is
// min(exact label, kLabelTop), so the truncated labels are the same.
constexpr unsigned kLabelTop = kMaxPuLevel + 1;

// min(floor(t / e), kLabelTop) for e >= 1: an estimate from the FP32
// reciprocal inv of e, corrected to the exact floor by one step either way.
// Below 2^12 the estimate's relative error (three FP32 roundings, under
// 2^-22) keeps it within one of t / e; FP32 because this part's FP64 rate
// is a small fraction of it. Since floor is monotone, a row's min over its
// arcs of label(y) + floor(d_y / e) is label_quot(min over its arcs of
// label(y) * e + d_y): one quotient per row instead of one per arc.
__device__ __forceinline__ unsigned label_quot(unsigned long long t, unsigned long long e, float inv) {
    if ((t >> 12) >= e) return kLabelTop;   // the quotient is at least 2^12
    unsigned q = (unsigned)(__ull2float_rz(t) * inv);
    const unsigned long long p = (unsigned long long)q * e;
    if (p > t) --q;
    else if (t - p >= e) ++q;
    return min(q, kLabelTop);
}

// The global price update (Sect. 5.2, Algorithm 5.3) on the tail kernel's
// own CTA, before its chains start: the same labels as k_pu (below), with
// the labels in shared memory and CTA barriers between the Bellman-Ford
// sweeps instead of grid barriers. Labels are distances in units of eps to
// the nearest free column over the residual graph of the candidate lists
// (a matched row's label capped by the bound theta on its unlisted
// columns), run to a fixed point (the last free row's bucket finished, as
// Algorithm 5.3 requires), truncated at one more than the largest label of
// a free row; every price then falls by eps * label (q grows).
//
// One SM has to hide L2 latency alone, so the work is indexed by column:
// a matched column's row is the mate in its shared-memory key, its
// v(x, M(x)) and cap are kept per column (vref, cap: global scratch of n
// entries), and a warp relaxes kPuBatch columns at a time with their lists'
// loads all in flight. Only the lists are read in a sweep; a column whose
// label is 0 is skipped. The matched rows are marked in a bitmap of n bits
// after the labels (mark).
constexpr int kPuBatch = 4;

// Shared memory of the update beyond the n keys: labels, and the row marks.
inline int tail_pu_smem(int n) { return (int)(sizeof(unsigned) * ((size_t)n + (n + 31) / 32)); }

template <bool WIDE>
__device__ void tail_price_update(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1,
                                  unsigned long long eps, unsigned long long qlim, unsigned long long *skey,
                                  unsigned *lab, unsigned *mark, const RowLists &L, unsigned long long R,
                                  unsigned long long *vref, unsigned *cap, Ctrl *ctrl) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const float inv = 1.0f / (float)eps;
    const unsigned long long t0 = tid == 0 ? global_timer_ns() : 0ull;
    __shared__ unsigned s_last;
    __shared__ unsigned long long s_qmax;
    for (int i = tid; i < (n + 31) / 32; i += blockDim.x) mark[i] = 0;
    if (tid == 0) {
        s_last = 0;
        s_qmax = 0;
    }
    __syncthreads();
    // per column: the start label, the matched row's mark, v(x, M(x)) and the
    // cap from theta (thread per column, the loads of a thread independent)
    unsigned long long qmx = 0;
    for (int y = tid; y < n; y += blockDim.x) {
        const unsigned long long k = skey[y];
        const uint32_t x = key_mate(k);
        qmx = max(qmx, key_q(k));
        unsigned l = 0;
        if (x < (uint32_t)n) {
            atomicOr(mark + (x >> 5), 1u << (x & 31));
            const unsigned long long th = __ldca(L.theta + x);
            const unsigned long long vr =
                (unsigned long long)(uint32_t)(ld_row1(C + (size_t)x * n + y) - cmin) * np1 + key_q(k);
            if (th == 0) {
                l = 0;                                   // no list: label 0 is always safe
            } else if (th == ~0ull) {
                l = kLabelTop;                           // every arc is listed
            } else {
                const unsigned long long tf = th > R + 1 ? th - R - 1 : 0;
                l = tf + eps >= vr ? label_quot(tf + eps - vr, eps, inv) : 0u;
            }
            vref[y] = vr;
            cap[y] = l;
        }
        lab[y] = l;
    }
    qmx = warp_max_u64(qmx);
    if (lane == 0) atomicMax(&s_qmax, qmx);
    __syncthreads();
    // Bellman-Ford sweeps until no label falls
    bool settled = false;
    int sweeps = 0;
    while (sweeps < 256) {
        ++sweeps;
        int changed = 0;
        for (int base = warp * kPuBatch; base < n; base += nwarps * kPuBatch) {
            LaneList e[kPuBatch];
            unsigned long long vr[kPuBatch];
            unsigned cur[kPuBatch];
            bool act[kPuBatch];
#pragma unroll
            for (int j = 0; j < kPuBatch; ++j) {
                const int w = base + j;
                act[j] = false;
                if (w < n) {
                    cur[j] = lab[w];
                    const uint32_t x = key_mate(skey[w]);
                    act[j] = cur[j] != 0 && x < (uint32_t)n;   // a label of 0 cannot fall
                    if (act[j]) {
                        e[j] = load_lane_list<true>(L, (int)x, lane);
                        vr[j] = __ldcg(vref + w);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kPuBatch; ++j) {
                if (!act[j]) continue;
                const int w = base + j;
                unsigned long long t = ~0ull;   // min of label(y) * eps + (v(x,y) + eps - v(x,w))
#pragma unroll
                for (int k = 0; k < kListK; ++k) {
                    const int y = e[j].y[k];
                    if (y < 0 || y >= n || y == w) continue;
                    const unsigned long long vy = (unsigned long long)(uint32_t)(e[j].c[k] - cmin) * np1 + key_q(skey[y]);
                    const unsigned long long d = vy + eps >= vr[j] ? vy + eps - vr[j] : 0;
                    t = min(t, (unsigned long long)lab[y] * eps + d);
                }
                t = warp_min(t);
                const unsigned best = min(__ldcg(cap + w), label_quot(t, eps, inv));
                if (lane == 0 && best < cur[j]) {
                    atomicMin(lab + w, best);
                    changed = 1;
                }
            }
        }
        if (!__syncthreads_or(changed)) {
            settled = true;
            break;
        }
    }
    // the free rows' labels set the truncation level
    unsigned mx = 0;
    for (int x = warp; x < n; x += nwarps) {
        if (mark[x >> 5] & (1u << (x & 31))) continue;
        const unsigned long long th = __ldca(L.theta + x);
        unsigned long long best = 0;
        if (th != 0) {
            const LaneList e = load_lane_list<true>(L, x, lane);
            unsigned long long m = ~0ull;
#pragma unroll
            for (int j = 0; j < kListK; ++j)
                if (e.y[j] >= 0 && e.y[j] < n)
                    m = min(m, (unsigned long long)(uint32_t)(e.c[j] - cmin) * np1 + key_q(skey[e.y[j]]));
            m = warp_min(m);
            const unsigned long long tf = th == ~0ull ? ~0ull : (th > R + 1 ? th - R - 1 : 0);
            const unsigned long long vr = min(m, tf);   // <= the row's best value
            unsigned long long t = ~0ull;
#pragma unroll
            for (int j = 0; j < kListK; ++j) {
                const int y = e.y[j];
                if (y < 0 || y >= n) continue;
                const unsigned long long vy = (unsigned long long)(uint32_t)(e.c[j] - cmin) * np1 + key_q(skey[y]);
                t = min(t, (unsigned long long)lab[y] * eps + (vy >= vr ? vy - vr : 0));
            }
            t = warp_min(t);
            best = min(th == ~0ull ? kLabelTop : label_quot(tf - vr, eps, inv), label_quot(t, eps, inv));
        }
        mx = max(mx, (unsigned)best);
    }
    if (lane == 0) atomicMax(&s_last, mx);
    __syncthreads();
    unsigned long long K = settled ? (unsigned long long)s_last + 1 : 0;
    K = min(K, (unsigned long long)kMaxPuLevel);
    K = min(K, qlim > s_qmax ? (qlim - s_qmax) / eps : 0ull);
    for (int y = tid; y < n && K > 0; y += blockDim.x) {
        const unsigned long long lb = min((unsigned long long)lab[y], K);
        if (lb == 0) continue;
        const unsigned long long k = skey[y];
        skey[y] = pack_key(key_q(k) + eps * lb, key_mate(k));
    }
    __syncthreads();
    if (tid == 0) {
        atomicAdd(&ctrl->pu_tail_ns, global_timer_ns() - t0);
        atomicAdd(&ctrl->pu_iters, (unsigned long long)sweeps);
        if (K > 0) {
            atomicAdd(&ctrl->pu_updates, 1ull);
            atomicAdd(&ctrl->pu_levels, K);
        }
    }
    __syncthreads();
}

// The end of a refine phase on one CTA. Once few rows are free (the refine
// kernel's hand-off), every step of their displacement chains is latency
// bound; here the column keys live in shared memory, so a step's price reads
// and its commit (the same packed atomicMin) stay on the SM. The rows handed
// over, and any still in the queue, are finished by the CTA's warps, then
// the keys go back to global memory.
//
// One SM is the right place for chains of list scans, not for full scans:
// when the lists stop answering (more than a quarter of the tail's scans,
// after kTailGiveUpFull of them, read whole rows), the CTA stops, and every
// row still free goes back to the row queue for a refine launch over the
// whole grid that follows the tail kernel in every phase (and hands the rows
// on to the team refine, whose CTAs share each full scan among 8 warps).
template <bool WIDE, bool VEC>
__global__ void __launch_bounds__(tail_threads<WIDE>())
k_tail(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long eps,
       unsigned long long qlim, unsigned long long *__restrict__ key, void *__restrict__ qmv,
       Ctrl *__restrict__ ctrl, unsigned long long budget, RowLists L, const int *__restrict__ tail_rows,
       int *__restrict__ qlist0, int *__restrict__ qlist1, int pu_tail, unsigned long long *__restrict__ pu_vref,
       unsigned *__restrict__ pu_cap, unsigned long long yield_scans) {
    extern __shared__ unsigned long long skey[];
    __shared__ int s_next, s_tc, s_q0, s_count, s_back, s_stop, s_status;
    __shared__ unsigned s_full, s_hits;
    __shared__ unsigned long long s_scans;
    if (*reinterpret_cast<volatile int *>(&ctrl->handoff) != 1) return;
    const int qmode = ctrl->qmode, qlen = ctrl->qlen, qsel = ctrl->qsel;
    const int *qlist = qsel ? qlist1 : qlist0;
    int *qback = qsel ? qlist0 : qlist1;       // rows handed back to the grid
    constexpr unsigned kFlush = 8;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int y = tid; y < n; y += blockDim.x) skey[y] = __ldcg(key + y);
    if (tid == 0) {
        const int qend = qmode ? qlen : n;
        s_next = 0;
        s_tc = ctrl->tail_count;
        s_q0 = min(ctrl->next_row, qend);
        s_count = s_tc + (qend - s_q0);
        s_back = 0;
        s_stop = 0;
        s_full = 0;
        s_hits = 0;
        s_status = 0;
        s_scans = 0;
        if (*reinterpret_cast<volatile int *>(&ctrl->status) != 0) s_count = 0;   // the phase has failed
    }
    __syncthreads();
    // No other kernel runs during this one: the scan budget and the status
    // are kept in shared memory and published at the end.
    const unsigned long long scans0 = ctrl->scans;
    const unsigned long long R = ctrl->rebase_total;
    if (pu_tail && L.cols && s_count > 0)   // labels, then the row marks, after the n keys in shared memory
        tail_price_update<WIDE>(C, n, cmin, np1, eps, qlim, skey, reinterpret_cast<unsigned *>(skey + n),
                                reinterpret_cast<unsigned *>(skey + n) + n, L, R, pu_vref, pu_cap, ctrl);
    const SharedKeyPrices<WIDE> prices{skey};
    volatile int *stop = &s_stop;
    int row = -1;
    ListAhead ahead;
    ahead.row = -1;
    unsigned long long wins = 0, displaced = 0, total = 0, full = 0, hits = 0;
    unsigned pending = 0;
    for (;;) {
        if (row < 0) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= s_count) break;
            if (k < s_tc) row = __ldcg(tail_rows + k);
            else row = qmode ? __ldcg(qlist + s_q0 + (k - s_tc)) : s_q0 + (k - s_tc);
        }
        if (*stop) {   // the lists no longer answer: this free row goes back to the grid
            if (lane == 0) qback[atomicAdd(&s_back, 1)] = row;
            break;
        }
        if (pending == kFlush) {
            unsigned long long s = 0;
            int st = 0;
            if (lane == 0) {
                s = atomicAdd(&s_scans, (unsigned long long)kFlush);
                st = *reinterpret_cast<volatile int *>(&s_status);
            }
            s = __shfl_sync(0xffffffffu, s, 0);
            st = __shfl_sync(0xffffffffu, st, 0);
            pending = 0;
            if (st != 0) break;
            if (scans0 + s + kFlush > budget) {
                if (lane == 0) atomicCAS(&s_status, 0, (int)LA_ERR_ITER_LIMIT);
                break;
            }
            // a stretch of bidding: stop for a global price update (the rows
            // go back, and k_pu runs next)
            if (yield_scans > 0 && s + kFlush > yield_scans && lane == 0) atomicCAS(&s_stop, 0, 2);
        }
        ++pending;
        ++total;
        bool was_full = false;
        const auto t = scan_for_bid<WIDE, VEC, true, (WIDE ? 4 : 2)>(C, row, n, cmin, np1, prices, lane, L, R, was_full,
                                                                    ahead);
        if (was_full) ++full;
        else ++hits;
        if (lane == 0) {   // the share of full scans can only pass 1/4 when a full scan is counted
            if (was_full) {
                const unsigned f = atomicAdd(&s_full, 1u) + 1;
                const unsigned h = *reinterpret_cast<volatile unsigned *>(&s_hits);
                if (f >= kTailGiveUpFull && 3 * f > h) *stop = 1;
            } else {
                atomicAdd(&s_hits, 1u);
            }
        }
        __syncwarp();
        const unsigned long long nq = (unsigned long long)(t.b1 - t.c1) + (t.b2 - t.b1) + eps;
        if (t.w >= n || nq > qlim) {
            if (lane == 0) atomicCAS(&s_status, 0, (int)(t.w >= n ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW));
            break;
        }
        const unsigned long long nk = pack_key(nq, (uint32_t)row);
        // The row this bid displaces, as far as the column's key tells now:
        // its list is loaded here, so that the load overlaps the commit. It
        // is used only if the commit finds the same key (then that row stayed
        // matched throughout, and no warp can have been rewriting its list).
        // Only the 512-thread (64-bit) kernel has the registers for it.
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long *>(skey + t.w);
        ahead.row = -1;
        if (WIDE && L.cols && cur > nk && key_mate(cur) != kNone)
            load_ahead<true>(ahead, L, (int)key_mate(cur), lane);
        unsigned long long old = 0;
        if (lane == 0) old = atomicMin(skey + t.w, nk);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old != cur) ahead.row = -1;
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
    __syncthreads();
    if (*stop) {   // rows never claimed go back too
        for (int k = min(s_next, s_count) + tid; k < s_count; k += blockDim.x) {
            const int r = k < s_tc ? __ldcg(tail_rows + k) : (qmode ? __ldcg(qlist + s_q0 + (k - s_tc)) : s_q0 + (k - s_tc));
            qback[atomicAdd(&s_back, 1)] = r;
        }
    }
    for (int y = tid; y < n; y += blockDim.x) {
        const unsigned long long k = skey[y];
        key[y] = k;
        if (WIDE) static_cast<unsigned long long *>(qmv)[y] = key_q(k);
        else static_cast<uint32_t *>(qmv)[y] = (uint32_t)key_q(k);
    }
    if (lane == 0 && total) {
        atomicAdd(&ctrl->scans, total);
        atomicAdd(&ctrl->tail_scans, total);
        atomicAdd(&ctrl->tail_full, full);
        atomicAdd(&ctrl->wins, wins);
        atomicAdd(&ctrl->displaced, displaced);
        atomicAdd(&ctrl->full_scans, full);
        atomicAdd(&ctrl->list_scans, hits);
    }
    __syncthreads();
    if (tid == 0) {
        if (s_status) set_status(ctrl, s_status);
        // the queue the follow-up refine launch reads: the rows given back, or none
        ctrl->qsel = *stop ? qsel ^ 1 : qsel;
        ctrl->qmode = 1;
        ctrl->qlen = *stop ? s_back : 0;
        ctrl->next_row = 0;
        ctrl->tail_count = 0;                 // the hand-off list has been taken
        ctrl->handoff = *stop == 2 ? 2 : 0;   // 2: a price update takes the rows first
        ctrl->tail_phases += 1;
        ctrl->tail_giveups += *stop == 1 ? 1 : 0;
    }
}

// ------------------------------------------------------------------------
// Small instances: the whole solve on one CTA, the cost matrix in shared
// memory. For n up to a few hundred a solve is a few thousand bids, most of
// them in sequence (the chains that end each phase), and in the grid path
// every bid pays a round trip to global memory for its row and its prices.
// Here the matrix is copied once into shared memory, as C - min C in 16 bits
// when the cost range allows it (else 32), the column keys live there too,
// and every phase runs in the same launch:
//   * phase initialisation (Alg. 5.2): the least q is taken out of every
//     price (a uniform shift), every mate is cleared;
//   * the bidding (Alg. 5.4 as the double push): each warp takes the next
//     row of the phase's queue and carries its displacement chain to its
//     end (a bid that lands on an unassigned column); a lost bid is retried.
//     When the queue is empty and every warp's chain has ended, every row is
//     matched: the CTA barrier that follows ends the phase.
// The bid itself is the grid refine's: exact best and second best over the
// whole row (from shared memory), one atomicMin on the packed key, stale
// price reads only ever making a bid lose (Lemma 5.2). The keys go back to
// global memory at the end for k_finalize.
constexpr int kSmallThreads = 1024;
constexpr int kSmallMaxN16 = 300;    // 2 n^2 + 8 n bytes of shared memory
constexpr int kSmallMaxN32 = 224;    // 4 n^2 + 8 n bytes

template <bool WIDE, bool C16>
__global__ void __launch_bounds__(kSmallThreads)
k_small(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, const unsigned long long *__restrict__ sched,
        int nph, unsigned long long qlim, unsigned long long *__restrict__ key, Ctrl *__restrict__ ctrl,
        unsigned long long budget) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    using CT = typename std::conditional<C16, uint16_t, uint32_t>::type;
    extern __shared__ unsigned long long small_smem[];
    unsigned long long *skey = small_smem;                        // [n]
    CT *cs = reinterpret_cast<CT *>(skey + n);                    // [n][n], C - cmin
    __shared__ int s_head, s_status;
    __shared__ unsigned long long s_scans, s_qmin;
    const int tid = threadIdx.x, lane = tid & 31;
    const size_t nn = (size_t)n * n;
    for (size_t e = tid; e < nn; e += blockDim.x) cs[e] = (CT)(uint32_t)(C[e] - cmin);
    for (int y = tid; y < n; y += blockDim.x) skey[y] = key[y];
    if (tid == 0) {
        s_status = 0;
        s_scans = 0;
    }
    __syncthreads();
    const volatile unsigned long long *vkey = skey;
    unsigned long long wins = 0, displaced = 0, chain_max = 0;
    for (int ph = 0; ph < nph; ++ph) {
        const unsigned long long eps = sched[ph];
        // phase initialisation: shift the prices so that min q = 0, clear the mates
        if (tid == 0) s_qmin = ~0ull;
        __syncthreads();
        unsigned long long m = ~0ull;
        for (int y = tid; y < n; y += blockDim.x) m = min(m, key_q(skey[y]));
        m = warp_min(m);
        if (lane == 0) atomicMin(&s_qmin, m);
        __syncthreads();
        const unsigned long long qmin = s_qmin;
        bool bad = false;
        for (int y = tid; y < n; y += blockDim.x) {
            const unsigned long long q = key_q(skey[y]) - qmin;
            bad |= q > qlim;
            skey[y] = pack_key(q, kNone);
        }
        if (bad) atomicCAS(&s_status, 0, (int)LA_ERR_OVERFLOW);
        if (tid == 0) {
            s_head = 0;
            ctrl->phase_start_scans[ph & 63] = s_scans;
            if (*reinterpret_cast<volatile int *>(&ctrl->status) == 0) ctrl->phase_now = ph;
        }
        __syncthreads();
        // the bidding: a warp carries each row it takes to the end of its chain
        int row = -1;
        unsigned long long chain = 0;
        unsigned pending = 0;
        for (;;) {
            if (*reinterpret_cast<volatile int *>(&s_status) != 0) break;
            if (row < 0) {
                int r = 0;
                if (lane == 0) r = atomicAdd(&s_head, 1);
                row = __shfl_sync(0xffffffffu, r, 0);
                if (row >= n) break;
            }
            if (++pending == 8) {   // the scan budget, 8 scans at a time
                pending = 0;
                unsigned long long sc = 0;
                if (lane == 0) sc = atomicAdd(&s_scans, 8ull);
                sc = __shfl_sync(0xffffffffu, sc, 0);
                if (sc + 8 > budget) {
                    if (lane == 0) atomicCAS(&s_status, 0, (int)LA_ERR_ITER_LIMIT);
                    break;
                }
            }
            ++chain;
            // best and second best of v(x,y) = (C[x][y] - cmin)(n+1) + q(y) over the row
            const CT *crow = cs + (size_t)row * n;
            Lane2<V> t;
            lane2_init(t);
            for (int y = lane; y < n; y += 32) lane2_push<V>(t, (V)crow[y] * np1 + (V)key_q(vkey[y]), y);
            const V c1 = t.w1 >= 0 ? (V)crow[t.w1] * np1 : (V)0;
            ScanResult<V> r{t.b1, t.b2, c1, t.w1 < 0 ? INT_MAX : t.w1};
            warp_merge(r);
            if (r.b2 == (V)~(V)0) r.b2 = r.b1;   // n = 1 cannot reach here; a lone column bids by eps
            // double push: x -> w, relabel w (its price drops by second - best + eps)
            const unsigned long long nq = (unsigned long long)(r.b1 - r.c1) + (r.b2 - r.b1) + eps;
            if (r.w >= n || nq > qlim) {
                if (lane == 0) atomicCAS(&s_status, 0, (int)(r.w >= n ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW));
                break;
            }
            const unsigned long long nk = pack_key(nq, (uint32_t)row);
            unsigned long long old = 0;
            if (lane == 0) old = atomicMin(skey + r.w, nk);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old > nk) {
                ++wins;
                const uint32_t mate = key_mate(old);
                if (mate != kNone) {
                    ++displaced;
                    row = (int)mate;
                } else {
                    row = -1;
                }
            }
            // else: a lower price got there first; rescan this row
        }
        chain_max = max(chain_max, chain);
        if (lane == 0 && pending) atomicAdd(&s_scans, (unsigned long long)pending);
        __syncthreads();   // every row is matched (or the solve has stopped)
        if (s_status != 0) break;
    }
    for (int y = tid; y < n; y += blockDim.x) key[y] = skey[y];
    if (lane == 0) {
        atomicAdd(&ctrl->wins, wins);
        atomicAdd(&ctrl->displaced, displaced);
        atomicMax(&ctrl->max_chain, chain_max);
    }
    __syncthreads();
    if (tid == 0) {
        ctrl->scans += s_scans;
        ctrl->full_scans += s_scans;
        if (s_status) set_status(ctrl, s_status);
    }
}

// ------------------------------------------------------------------------
// Global price update (Sect. 5.2, Algorithm 5.3), run when a phase is down
// to a few free rows. It labels every node with its distance, in units of
// eps, to the nearest free column (a node with negative excess) over the
// residual graph, then lowers p(y) by eps * label (q grows), which keeps
// every matched row eps-optimal and lines up admissible paths from the free
// rows to the free columns, so their displacement chains become short.
//
// Arc lengths keep the version-2 eps-optimality (Sect. 5.1): with the row
// price p(x) = eps - v(x, M(x)) of a matched row x (v = c~ - p), the arc
// x -> y (y != M(x)) has length floor((v(x,y) - v(x,M(x)) + eps) / eps) and
// the matched arc M(x) -> x has length 0, so the label of a matched column
// is that of its row. Only the kListLen arcs of x's candidate list are relaxed;
// every other column has v >= theta (see RowLists), so the row's label is
// also capped at floor((theta - v(x,M(x)) + eps) / eps), which keeps the
// required inequality label(x) <= label(y) + length(x,y) on those arcs
// (labels are >= 0). Labels are truncated at one more than the largest label
// of a free row, as Algorithm 5.3 does for unscanned nodes (the whole last
// bucket is included). Bellman-Ford sweeps run to a fixed point between grid
// barriers of a cooperatively launched (co-resident) grid; if they do not
// settle within the sweep limit, no price changes.

// Barrier of a co-resident grid. A wait longer than 2 s sets
// LA_ERR_INTERNAL and returns false instead of spinning on.
__device__ bool pu_grid_sync(Ctrl *ctrl, int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctrl->pu_bar[1];
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(&ctrl->pu_bar[0], 1u) + 1 == gridDim.x) {
            atomicExch(&ctrl->pu_bar[0], 0u);
            __threadfence();
            atomicAdd(&ctrl->pu_bar[1], 1u);
        } else {
            const unsigned long long t0 = global_timer_ns();
            while (*gen == g) {
                __nanosleep(64);
                if (global_timer_ns() - t0 > 2000000000ull) {
                    atomicCAS(&ctrl->status, 0, (int)LA_ERR_INTERNAL);
                    *s_ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *s_ok != 0;
}

template <bool WIDE>
__global__ void __launch_bounds__(256, 2)
k_pu(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long eps,
     unsigned long long qlim, unsigned long long *__restrict__ key, void *__restrict__ qmv,
     Ctrl *__restrict__ ctrl, RowLists L, const int *__restrict__ tail_rows, int *__restrict__ qlist0,
     int *__restrict__ qlist1, unsigned *__restrict__ lab, unsigned long long *__restrict__ vref,
     unsigned *__restrict__ cap, int *__restrict__ rowcol, int max_sweeps) {
    __shared__ int s_ok;
    if (*reinterpret_cast<volatile int *>(&ctrl->handoff) != 2) return;
    if (threadIdx.x == 0) s_ok = 1;
    const int tid = threadIdx.x, lane = tid & 31;
    const int gtid = blockIdx.x * blockDim.x + tid, gthreads = gridDim.x * blockDim.x;
    const int gwarp = gtid >> 5, nwarps = gthreads >> 5;
    const unsigned long long R = ctrl->rebase_total;
    const float inv = 1.0f / (float)eps;
    // A0: clear the row -> column map and the sweep flags
    for (int x = gtid; x < n; x += gthreads) rowcol[x] = -1;
    if (gtid == 0) {
        ctrl->pu_changed[0] = 0;
        ctrl->pu_changed[1] = 0;
        ctrl->pu_changed[2] = 0;
    }
    if (!pu_grid_sync(ctrl, &s_ok)) return;
    // A1: per column, the largest q, the row map, and for a matched column
    // v(x, M(x)) and the cap from theta (kept per column: vref, cap), which is
    // its start label; a free column starts at 0
    unsigned long long qmx = 0;
    for (int y = gtid; y < n; y += gthreads) {
        const unsigned long long k = key[y];
        const uint32_t x = key_mate(k);
        qmx = max(qmx, key_q(k));
        unsigned l = 0;
        if (x < (uint32_t)n) {
            rowcol[x] = y;
            const unsigned long long th = L.cols ? __ldcg(L.theta + x) : 0ull;
            const unsigned long long vr =
                (unsigned long long)(uint32_t)(ld_row1(C + (size_t)x * n + y) - cmin) * np1 + key_q(k);
            if (th == 0) {
                l = 0;                                   // no list: label 0 is always safe
            } else if (th == ~0ull) {
                l = kLabelTop;                           // every column is listed
            } else {
                const unsigned long long tf = th > R + 1 ? th - R - 1 : 0;
                l = tf + eps >= vr ? label_quot(tf + eps - vr, eps, inv) : 0u;
            }
            vref[y] = vr;
            cap[y] = l;
        }
        lab[y] = l;
    }
    for (int o = 16; o; o >>= 1) qmx = max(qmx, __shfl_xor_sync(0xffffffffu, qmx, o));
    if (lane == 0) atomicMax(&ctrl->pu_qmax, qmx);
    if (!pu_grid_sync(ctrl, &s_ok)) return;
    // B: Bellman-Ford sweeps over the matched columns until no label falls;
    // a warp relaxes kPuBatch columns at a time, their rows' lists loaded
    // together (the mate read from the column's key, which no kernel changes
    // during the update); a label of 0 cannot fall
    int it = 0;
    bool settled = false;
    for (; it < max_sweeps; ++it) {
        // Flag of this sweep; the next sweep's flag was last read after the
        // barrier two sweeps ago, which every block has passed, so it can be
        // cleared now.
        const int par = it % 3;
        bool changed = false;
        for (int base = gwarp * kPuBatch; base < n; base += nwarps * kPuBatch) {
            LaneList e[kPuBatch];
            unsigned long long vr[kPuBatch];
            unsigned cur[kPuBatch];
            bool act[kPuBatch];
#pragma unroll
            for (int j = 0; j < kPuBatch; ++j) {
                const int w = base + j;
                act[j] = false;
                if (w < n) {
                    cur[j] = __ldcg(lab + w);
                    const uint32_t x = key_mate(__ldcg(key + w));
                    act[j] = cur[j] != 0 && x < (uint32_t)n;
                    if (act[j]) {
                        e[j] = load_lane_list(L, (int)x, lane);
                        vr[j] = __ldcg(vref + w);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kPuBatch; ++j) {
                if (!act[j]) continue;
                const int w = base + j;
                unsigned long long t = ~0ull;   // min of label(y) * eps + (v(x,y) + eps - v(x,w))
#pragma unroll
                for (int k = 0; k < kListK; ++k) {
                    const int y = e[j].y[k];
                    if (y < 0 || y >= n || y == w) continue;
                    const unsigned long long vy = (unsigned long long)(uint32_t)(e[j].c[k] - cmin) * np1 + key_q(__ldcg(key + y));
                    const unsigned long long d = vy + eps >= vr[j] ? vy + eps - vr[j] : 0;
                    t = min(t, (unsigned long long)__ldcg(lab + y) * eps + d);
                }
                t = warp_min(t);
                const unsigned b = min(__ldcg(cap + w), label_quot(t, eps, inv));
                if (lane == 0 && b < cur[j]) {
                    lab[w] = b;
                    changed = true;
                }
            }
        }
        if (changed) ctrl->pu_changed[par] = 1;
        if (gtid == 0) ctrl->pu_changed[(it + 1) % 3] = 0;
        if (!pu_grid_sync(ctrl, &s_ok)) return;
        if (*reinterpret_cast<volatile int *>(&ctrl->pu_changed[par]) == 0) {
            settled = true;
            break;
        }
    }
    // C: the free rows' labels set the truncation level (a free row's value
    // bound: the least listed value, or theta if that is lower)
    unsigned mx = 0;
    for (int x = gwarp; x < n; x += nwarps) {
        if (rowcol[x] >= 0) continue;
        const unsigned long long th = L.cols ? __ldcg(L.theta + x) : 0ull;
        unsigned best = 0;
        if (th != 0) {
            const LaneList e = load_lane_list(L, x, lane);
            unsigned long long m = ~0ull;
#pragma unroll
            for (int k = 0; k < kListK; ++k)
                if (e.y[k] >= 0 && e.y[k] < n)
                    m = min(m, (unsigned long long)(uint32_t)(e.c[k] - cmin) * np1 + key_q(__ldcg(key + e.y[k])));
            m = warp_min(m);
            const unsigned long long tf = th == ~0ull ? ~0ull : (th > R + 1 ? th - R - 1 : 0);
            const unsigned long long vr = min(m, tf);
            unsigned long long t = ~0ull;
#pragma unroll
            for (int k = 0; k < kListK; ++k) {
                const int y = e.y[k];
                if (y < 0 || y >= n) continue;
                const unsigned long long vy = (unsigned long long)(uint32_t)(e.c[k] - cmin) * np1 + key_q(__ldcg(key + y));
                t = min(t, (unsigned long long)__ldcg(lab + y) * eps + (vy >= vr ? vy - vr : 0));
            }
            t = warp_min(t);
            best = min(th == ~0ull ? kLabelTop : label_quot(tf - vr, eps, inv), label_quot(t, eps, inv));
        }
        mx = max(mx, best);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) atomicMax(&ctrl->pu_last, mx);
    if (!pu_grid_sync(ctrl, &s_ok)) return;
    // D: lower the prices, q += eps * min(label, K), and queue the free rows
    const unsigned long long qmax = ctrl->pu_qmax;
    unsigned long long K = settled ? (unsigned long long)ctrl->pu_last + 1 : 0;
    K = min(K, (unsigned long long)kMaxPuLevel);   // keeps the price spread near its usual bound
    K = min(K, qlim > qmax ? (qlim - qmax) / eps : 0ull);
    for (int y = gtid; y < n && K > 0; y += gthreads) {
        const unsigned long long lb = min((unsigned long long)lab[y], K);
        if (lb == 0) continue;
        const unsigned long long k = key[y];
        const unsigned long long q = key_q(k) + eps * lb;
        key[y] = pack_key(q, key_mate(k));
        if (WIDE) static_cast<unsigned long long *>(qmv)[y] = q;
        else static_cast<uint32_t *>(qmv)[y] = (uint32_t)q;
    }
    const int qmode = ctrl->qmode, qlen = ctrl->qlen, qsel = ctrl->qsel, tc = ctrl->tail_count;
    const int *qold = qsel ? qlist1 : qlist0;
    int *qnew = qsel ? qlist0 : qlist1;
    const int qend = qmode ? qlen : n;
    const int q0 = min(ctrl->next_row, qend);
    const int total = tc + (qend - q0);
    for (int k = gtid; k < total; k += gthreads)
        qnew[k] = k < tc ? tail_rows[k] : (qmode ? qold[q0 + (k - tc)] : q0 + (k - tc));
    if (!pu_grid_sync(ctrl, &s_ok)) return;
    if (gtid == 0) {
        ctrl->qsel = qsel ^ 1;
        ctrl->qmode = 1;
        ctrl->qlen = total;
        ctrl->next_row = 0;
        ctrl->tail_count = 0;
        ctrl->pu_left -= 1;
        ctrl->pu_mark = ctrl->scans;
        ctrl->pu_iters += (unsigned long long)(it + 1);
        if (K > 0) {
            ctrl->pu_updates += 1;
            ctrl->pu_levels += K;
        }
        ctrl->pu_qmax = 0;
        ctrl->pu_last = 0;
        __threadfence();
        ctrl->handoff = 0;
    }
}

// Arc fixing (Sect. 5.2), run when a phase other than the last has ended
// with an eps-optimal flow. Sect. 5.2 drops every arc whose reduced cost
// c_p(x,y) exceeds 2 n eps: its flow stays zero in every later phase, so no
// optimal assignment uses it. With the row price of Algorithm 5.2,
// c_p(x,y) = v(x,y) - min_z v(x,z) - eps, the rule drops y from x's arcs when
// v(x,y) - min_z v(x,z) > T = (2n+1) eps. Any upper bound m of the row's
// minimum may stand in for it: the test then keeps more arcs, never fewer.
//
// A row is fixed when everything outside its candidate list can go: its
// list then holds exactly its remaining arcs and theta = ~0 ("every arc is
// listed"), so each later bid of the row is a list scan and none reads the
// row again. One warp per row:
//   * a fixed row drops the listed arcs that the rule removes;
//   * a row with a list is fixed when its unlisted columns, all worth at
//     least theta (see RowLists), are beyond the least listed value m by T;
//   * otherwise, if `full_pass`, the row is read whole (the exact minimum,
//     then its arcs within T of it); if no more than kListLen remain, they
//     become the row's list.
// Rows that are not fixed keep every arc. The kernel runs between the
// phase's last refine launch and the next phase's initialisation, so no
// other kernel reads the lists meanwhile.
template <bool VEC>
__global__ void __launch_bounds__(256)
k_fix(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long T,
      const unsigned long long *__restrict__ key, RowLists L, Ctrl *__restrict__ ctrl, int full_pass, int phase) {
    if (*reinterpret_cast<volatile int *>(&ctrl->status) != 0) return;
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    const unsigned long long R = ctrl->rebase_total;
    unsigned long long rows = 0, arcs = 0;
    for (int x = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); x < n; x += warps) {
        const unsigned long long th = __ldcg(L.theta + x);
        if (th == 0) continue;
        const size_t base = (size_t)x * kListLen + kListK * lane;
        const LaneList e = load_lane_list<false>(L, x, lane);
        unsigned long long v[kListK], m = ~0ull;
#pragma unroll
        for (int k = 0; k < kListK; ++k) {
            const bool ok = e.y[k] >= 0 && e.y[k] < n;
            v[k] = ok ? (unsigned long long)(uint32_t)(e.c[k] - cmin) * np1 + key_q(__ldcg(key + e.y[k])) : ~0ull;
            m = min(m, v[k]);
        }
        m = warp_min(m);
        // every unlisted value is >= this (0: no bound left after the shifts)
        const unsigned long long unlisted = th > R + 1 ? th - R - 1 : 0;
        if (th == ~0ull || (unlisted > m && unlisted - m > T)) {
            int keep[kListK];
            int kept = 0;
#pragma unroll
            for (int k = 0; k < kListK; ++k) {
                keep[k] = (v[k] != ~0ull && v[k] - m <= T) ? e.y[k] : -1;
                kept += keep[k] >= 0;
            }
#pragma unroll
            for (int g = 0; g < kListK / 4; ++g)
                reinterpret_cast<int4 *>(L.cols + base)[g] =
                    make_int4(keep[4 * g], keep[4 * g + 1], keep[4 * g + 2], keep[4 * g + 3]);
            kept = __reduce_add_sync(0xffffffffu, kept);
            if (lane == 0) {
                L.theta[x] = ~0ull;
                ++rows;
                arcs += (unsigned long long)kept;
            }
            continue;
        }
        if (!full_pass) continue;
        // the whole row: exact minimum, then the arcs within T of it
        const int32_t *crow = C + (size_t)x * n;
        unsigned long long mn = ~0ull;
        if (VEC) {
            const int4 *r4 = reinterpret_cast<const int4 *>(crow);
            for (int j = lane; j < (n >> 2); j += 32) {
                const int4 c = ld_row4(r4 + j);
                const int y = j << 2;
                mn = min(mn, (unsigned long long)(uint32_t)(c.x - cmin) * np1 + key_q(__ldcg(key + y)));
                mn = min(mn, (unsigned long long)(uint32_t)(c.y - cmin) * np1 + key_q(__ldcg(key + y + 1)));
                mn = min(mn, (unsigned long long)(uint32_t)(c.z - cmin) * np1 + key_q(__ldcg(key + y + 2)));
                mn = min(mn, (unsigned long long)(uint32_t)(c.w - cmin) * np1 + key_q(__ldcg(key + y + 3)));
            }
        } else {
            for (int y = lane; y < n; y += 32)
                mn = min(mn, (unsigned long long)(uint32_t)(ld_row1(crow + y) - cmin) * np1 + key_q(__ldcg(key + y)));
        }
        mn = warp_min(mn);
        int cnt = 0;
        for (int y = lane; y < n; y += 32)
            cnt += (unsigned long long)(uint32_t)(ld_row1(crow + y) - cmin) * np1 + key_q(__ldcg(key + y)) - mn <= T;
        const int total = __reduce_add_sync(0xffffffffu, cnt);
        if (total > kListLen) continue;
        // lane l writes its arcs at the flat positions after lanes 0..l-1's
        int off = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += t;
        }
        off -= cnt;
        int *cols = L.cols + (size_t)x * kListLen;
        int *costs = L.costs + (size_t)x * kListLen;
        for (int y = lane; y < n; y += 32) {
            const int c = ld_row1(crow + y);
            if ((unsigned long long)(uint32_t)(c - cmin) * np1 + key_q(__ldcg(key + y)) - mn <= T) {
                cols[off] = y;
                costs[off] = c;
                ++off;
            }
        }
        for (int k = total + lane; k < kListLen; k += 32) cols[k] = -1;
        if (lane == 0) {
            L.theta[x] = ~0ull;
            ++rows;
            arcs += (unsigned long long)total;
        }
    }
    if (lane == 0 && rows) {
        atomicAdd(&ctrl->fix_rows[phase & 63], rows);
        atomicAdd(&ctrl->fix_arcs[phase & 63], arcs);
    }
}

// Read the matching out of the column keys; exact int64 cost.
__global__ void k_finalize(const int32_t *__restrict__ C, int n, const unsigned long long *__restrict__ key,
                           int32_t *match, long long *cost, long long *prices, Ctrl *ctrl, int slot) {
    long long sum = 0;
    const unsigned long long qmin = prices ? ctrl->qmin[slot] : 0;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const unsigned long long k = key[y];
        const uint32_t m = key_mate(k);
        // prices first: after a stop (the scan budget) they are the state to resume from
        if (prices) prices[y] = -(long long)(key_q(k) - qmin);
        if (m >= (uint32_t)n) {
            set_status(ctrl, LA_ERR_INTERNAL);
            continue;
        }
        if (match) match[m] = y;
        sum += C[(size_t)m * n + y];
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum != 0)
        atomicAdd(reinterpret_cast<unsigned long long *>(cost), (unsigned long long)sum);
}

// Debug mode (LA_FLAG_CHECK_PHASES). The prices q(y) at the start of a phase,
// after its rebase.
__global__ void k_check_snapshot(const unsigned long long *__restrict__ key, int n, unsigned long long *q0) {
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) q0[y] = key_q(key[y]);
}

// Debug mode, at the end of a phase: one warp per column y checks that y
// has a holder x (if `perfect`), that x holds no other column, that x is
// eps-optimal, (n+1)(C[x][y] - cmin) + q(y) <= min_z ((n+1)(C[x][z] - cmin)
// + q(z)) + eps (version-2 eps-CS, Sect. 5.1), and that q(y) did not fall
// during the phase (prices only decrease, Lemma 5.2). Plain 64-bit
// arithmetic, independent of the refine's narrow and list paths. For a row
// that arc fixing cut down to its list (theta = ~0), z ranges over the
// listed columns, its remaining arcs, with the costs read from C.
__global__ void k_check_phase(const int32_t *__restrict__ C, int n, int cmin, unsigned long long np1,
                              const unsigned long long *__restrict__ key, const unsigned long long *__restrict__ q0,
                              unsigned long long eps, int perfect, int *__restrict__ seen, Ctrl *ctrl,
                              RowLists L) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int y = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); y < n; y += warps) {
        const unsigned long long k = key[y];
        const uint32_t x = key_mate(k);
        unsigned long long bad = key_q(k) < q0[y] ? 1 : 0;
        if (x >= (uint32_t)n) {
            bad += (x != kNone || perfect) ? 1 : 0;
        } else {
            if (lane == 0 && atomicAdd(&seen[x], 1) != 0) ++bad;
            const int32_t *row = C + (size_t)x * n;
            unsigned long long mn = ~0ull;
            if (L.cols && L.theta[x] == ~0ull) {
                for (int k = lane; k < kListLen; k += 32) {
                    const int z = L.cols[(size_t)x * kListLen + k];
                    if (z < 0 || z >= n) continue;
                    const unsigned long long v = (unsigned long long)(uint32_t)(row[z] - cmin) * np1 + key_q(key[z]);
                    mn = v < mn ? v : mn;
                }
            } else {
                for (int z = lane; z < n; z += 32) {
                    const unsigned long long v = (unsigned long long)(uint32_t)(row[z] - cmin) * np1 + key_q(key[z]);
                    mn = v < mn ? v : mn;
                }
            }
            mn = warp_min(mn);
            const unsigned long long mine = (unsigned long long)(uint32_t)(row[y] - cmin) * np1 + key_q(k);
            if (mine > mn + eps) ++bad;
        }
        if (lane == 0 && bad) atomicAdd(&ctrl->check_violations, bad);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctrl->checked_phases, 1);
}

// ---------------------------------------------------------------- host side

struct Workspace {
    int64_t cap = 0;
    unsigned long long *key = nullptr;
    void *qm = nullptr;
    int *lcols = nullptr;                 // candidate lists
    int *lcosts = nullptr;
    unsigned long long *ltheta = nullptr;
    int *tail_rows = nullptr;             // rows handed to the tail kernel / price update
    int *qlist[2] = {nullptr, nullptr};   // row queues after a price update
    unsigned *pu_lab = nullptr;           // price-update labels, caps, row data
    unsigned *pu_cap = nullptr;
    unsigned long long *pu_vref = nullptr;
    int *pu_rowcol = nullptr;
    int pu_grid = 0;
    Ctrl *ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;
    int num_sms = 0;
    bool events = false;
    cudaEvent_t ev[5 * kMaxPhases];   // per phase: start, sweep end, tail start, tail end, end
};

std::mutex g_mu;
Workspace g_ws[kMaxDevices];

void free_ws(Workspace &ws) {
    cudaFree(ws.key);
    cudaFree(ws.qm);
    cudaFree(ws.lcols);
    cudaFree(ws.lcosts);
    cudaFree(ws.ltheta);
    cudaFree(ws.tail_rows);
    cudaFree(ws.qlist[0]);
    cudaFree(ws.qlist[1]);
    cudaFree(ws.pu_lab);
    cudaFree(ws.pu_cap);
    cudaFree(ws.pu_vref);
    cudaFree(ws.pu_rowcol);
    cudaFree(ws.ctrl);
    cudaFreeHost(ws.h_ctrl);
    if (ws.events)
        for (auto &e : ws.ev) cudaEventDestroy(e);
    ws = Workspace();
}

la_status ensure_ws(Workspace &ws, int64_t n) {
    if (!ws.ctrl) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
        if (cudaDeviceGetAttribute(&ws.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return LA_ERR_CUDA;
        if (cudaMalloc(&ws.ctrl, sizeof(Ctrl)) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMallocHost(&ws.h_ctrl, sizeof(Ctrl)) != cudaSuccess) return LA_ERR_NOMEM;
        for (auto &e : ws.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return LA_ERR_CUDA;
        ws.events = true;
    }
    if (ws.cap < n) {
        cudaFree(ws.key);
        cudaFree(ws.qm);
        cudaFree(ws.lcols);
        cudaFree(ws.lcosts);
        cudaFree(ws.ltheta);
        cudaFree(ws.tail_rows);
        cudaFree(ws.qlist[0]);
        cudaFree(ws.qlist[1]);
        cudaFree(ws.pu_lab);
        cudaFree(ws.pu_cap);
        cudaFree(ws.pu_vref);
        cudaFree(ws.pu_rowcol);
        ws.qlist[0] = ws.qlist[1] = nullptr;
        ws.pu_lab = ws.pu_cap = nullptr;
        ws.pu_vref = nullptr;
        ws.pu_rowcol = nullptr;
        ws.key = nullptr;
        ws.qm = nullptr;
        ws.lcols = nullptr;
        ws.lcosts = nullptr;
        ws.ltheta = nullptr;
        ws.tail_rows = nullptr;
        ws.cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1024);
        if (cudaMalloc(&ws.key, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.qm, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.lcols, sizeof(int) * kListLen * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.lcosts, sizeof(int) * kListLen * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.ltheta, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.tail_rows, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.qlist[0], sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.qlist[1], sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.pu_lab, sizeof(unsigned) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.pu_cap, sizeof(unsigned) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.pu_vref, sizeof(unsigned long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&ws.pu_rowcol, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        ws.cap = cap;
    }
    return LA_OK;
}

template <bool WIDE, bool VEC>
int refine_grid(int num_sms, int block, int n) {
    static int occ[kMaxDevices][5];   // per device and block size / 64 (cached; calls are serialised)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    const int slot = std::min(4, block / 64);
    if (!occ[dev][slot]) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_refine<WIDE, VEC>, block, 0);
        occ[dev][slot] = std::max(1, o);
    }
    const int warps_per_block = block / 32;
    const int need = (n + warps_per_block - 1) / warps_per_block;
    return std::max(1, std::min(num_sms * occ[dev][slot], need));
}

template <bool WIDE>
cudaError_t launch_pu(cudaStream_t s, const int32_t *C, int n, int cmin, uint32_t np1, unsigned long long eps,
                      unsigned long long qlim, Workspace &ws, const RowLists &L) {
    if (!ws.pu_grid) {
        int o = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_pu<WIDE>, 256, 0);
        ws.pu_grid = std::max(1, o) * ws.num_sms;
    }
    int max_sweeps = 256;
    void *args[] = {(void *)&C, (void *)&n, (void *)&cmin, (void *)&np1, (void *)&eps, (void *)&qlim,
                    (void *)&ws.key, (void *)&ws.qm, (void *)&ws.ctrl, (void *)&L, (void *)&ws.tail_rows,
                    (void *)&ws.qlist[0], (void *)&ws.qlist[1], (void *)&ws.pu_lab, (void *)&ws.pu_vref,
                    (void *)&ws.pu_cap, (void *)&ws.pu_rowcol, (void *)&max_sweeps};
    return cudaLaunchCooperativeKernel((const void *)k_pu<WIDE>, dim3(ws.pu_grid), dim3(256), args, 0, s);
}

template <bool WIDE, bool VEC>
cudaError_t launch_refine(cudaStream_t s, int grid, int block, const int32_t *C, int n, int cmin, uint32_t np1,
                          unsigned long long eps, unsigned long long qlim, Workspace &ws,
                          unsigned long long budget, const RowLists &L, int tail_T, int pu_T, int pu_rounds,
                          int64_t &launches, int stop_free, cudaEvent_t ev_sweep, cudaEvent_t ev_tail,
                          cudaEvent_t ev_fin, bool sweep, bool tail_pu, int team_T, int tail_updates) {
    if (sweep) {   // the phase's bulk sweep: every row bids once
        k_refine<WIDE, VEC><<<grid, block, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl, budget, L,
                                                   0, ws.tail_rows, 0, ws.qlist[0], ws.qlist[1], 0, 1);
        ++launches;
    }
    if (ev_sweep) {
        cudaError_t e = cudaEventRecord(ev_sweep, s);
        if (e != cudaSuccess) return e;
    }
    for (int r = 0; r <= pu_rounds; ++r) {
        if (r > 0) {
            cudaError_t e = launch_pu<WIDE>(s, C, n, cmin, np1, eps, qlim, ws, L);
            if (e != cudaSuccess) return e;
            ++launches;
        }
        // the last refine of a phase never stops for a price update
        k_refine<WIDE, VEC><<<grid, block, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl, budget, L,
                                                   tail_T, ws.tail_rows, r < pu_rounds ? pu_T : 0,
                                                   ws.qlist[0], ws.qlist[1], stop_free, team_T > 0 ? 2 : 0);
        ++launches;
        if (team_T > 0) {   // one CTA per row the refine hands over (at most team_T)
            k_team<WIDE, VEC><<<team_T, 32 * kTeamWarps, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl,
                                                                 budget, L, tail_T, ws.tail_rows, ws.qlist[0],
                                                                 ws.qlist[1], stop_free, r < pu_rounds ? pu_T : 0);
            ++launches;
        }
    }
    if (ev_tail) {
        cudaError_t e = cudaEventRecord(ev_tail, s);
        if (e != cudaSuccess) return e;
    }
    if (tail_T > 0) {
        ++launches;
        // the column keys, and with the in-tail price update its labels and row marks
        const int smem = (int)(sizeof(unsigned long long) * n + (tail_pu ? tail_pu_smem(n) : 0));
        {   // A per-device attribute, set on every launch (a host call, no GPU work). Without it the
            // kernel's static shared memory and `smem` together may not pass 48 KB (n near 6144).
            cudaError_t e = cudaFuncSetAttribute(k_tail<WIDE, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        // Each tail launch but the last may stop after 2n scans for a grid
        // price update; the refine (and team refine) launch after the update
        // hands the rows straight back to the next tail launch.
        const unsigned long long yield = 2ull * (unsigned long long)n;
        for (int r = 0; r <= tail_updates; ++r) {
            if (r > 0) {
                cudaError_t e = launch_pu<WIDE>(s, C, n, cmin, np1, eps, qlim, ws, L);
                if (e != cudaSuccess) return e;
                k_refine<WIDE, VEC><<<grid, block, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl, budget,
                                                           L, tail_T, ws.tail_rows, 0, ws.qlist[0], ws.qlist[1],
                                                           stop_free, team_T > 0 ? 2 : 0);
                launches += 2;
                if (team_T > 0) {
                    k_team<WIDE, VEC><<<team_T, 32 * kTeamWarps, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm,
                                                                         ws.ctrl, budget, L, tail_T, ws.tail_rows,
                                                                         ws.qlist[0], ws.qlist[1], stop_free, 0);
                    ++launches;
                }
                ++launches;
            }
            k_tail<WIDE, VEC><<<1, tail_threads<WIDE>(), smem, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl,
                                                                   budget, L, ws.tail_rows, ws.qlist[0], ws.qlist[1],
                                                                   tail_pu ? 1 : 0, ws.pu_vref, ws.pu_cap,
                                                                   r < tail_updates ? yield : 0ull);
        }
        if (ev_fin) {
            cudaError_t e = cudaEventRecord(ev_fin, s);
            if (e != cudaSuccess) return e;
        }
        // rows the tail kernel gave back, if any (an empty queue otherwise):
        // the lists stopped answering, so the team refine takes them at once,
        // and no tail kernel follows
        k_refine<WIDE, VEC><<<grid, block, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl, budget, L,
                                                   0, ws.tail_rows, 0, ws.qlist[0], ws.qlist[1], stop_free,
                                                   team_T > 0 ? 2 : 0);
        ++launches;
        if (team_T > 0) {
            k_team<WIDE, VEC><<<team_T, 32 * kTeamWarps, 0, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.qm, ws.ctrl,
                                                                 budget, L, 0, ws.tail_rows, ws.qlist[0], ws.qlist[1],
                                                                 stop_free, 0);
            ++launches;
        }
    } else if (ev_fin) {
        cudaError_t e = cudaEventRecord(ev_fin, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

inline int small_grid(int n, int block, int num_sms) {
    return std::max(1, std::min((n + block - 1) / block, 4 * num_sms));
}

}  // namespace

#define LA_CK(call)                                   \
    do {                                              \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

// ------------------------------------------------------------------------
// la_debug_price_update: one global price update (Algorithm 5.3, the same
// k_pu the refine launches) on a mid-phase state given by the caller, so
// that its labels and new prices can be checked one by one.

// Mates of the given partial matching, and the price mirror.
template <bool WIDE>
__global__ void k_dbg_state(const int32_t *__restrict__ row_match, int n, unsigned long long *__restrict__ key,
                            void *__restrict__ qmv, Ctrl *ctrl) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const int y = row_match[x];
        if (y < 0) continue;
        if (y >= n) {
            set_status(ctrl, LA_ERR_INVALID);
            continue;
        }
        const unsigned long long k = key[y];
        // a column claimed by two rows is an invalid state
        if (atomicCAS(key + y, k, pack_key(key_q(k), (uint32_t)x)) != k || key_mate(k) != kNone)
            set_status(ctrl, LA_ERR_INVALID);
    }
}

template <bool WIDE>
__global__ void k_dbg_mirror(const unsigned long long *__restrict__ key, int n, void *__restrict__ qmv, Ctrl *ctrl) {
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const unsigned long long q = key_q(key[y]);
        if (WIDE) static_cast<unsigned long long *>(qmv)[y] = q;
        else static_cast<uint32_t *>(qmv)[y] = (uint32_t)q;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // the state k_pu starts from: no queue, one update
        ctrl->handoff = 2;
        ctrl->qmode = 1;
        ctrl->qlen = 0;
        ctrl->qsel = 0;
        ctrl->next_row = 0;
        ctrl->tail_count = 0;
        ctrl->rebase_total = 0;
        ctrl->pu_left = 1;
    }
}

// Candidate lists of every row at the given prices (one full scan each).
template <bool WIDE, bool VEC>
__global__ void __launch_bounds__(256)
k_dbg_lists(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, const void *__restrict__ qmv, RowLists L) {
    const int lane = threadIdx.x & 31;
    const int warps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int x = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); x < n; x += warps)
        (void)full_scan<WIDE, VEC, 1>(C + (size_t)x * n, x, n, cmin, np1, MirrorPrices<WIDE>{qmv}, lane, L, 0ull);
}

// The one-CTA update of the tail kernel on the same state: keys and labels
// in shared memory, written back for k_dbg_out.
template <bool WIDE>
__global__ void __launch_bounds__(tail_threads<WIDE>())
k_dbg_tail_pu(const int32_t *__restrict__ C, int n, int cmin, uint32_t np1, unsigned long long eps,
              unsigned long long qlim, unsigned long long *__restrict__ key, Ctrl *__restrict__ ctrl, RowLists L,
              unsigned long long *__restrict__ vref, unsigned *__restrict__ cap, unsigned *__restrict__ lab_out) {
    extern __shared__ unsigned long long skey[];
    unsigned *lab = reinterpret_cast<unsigned *>(skey + n);
    for (int y = threadIdx.x; y < n; y += blockDim.x) skey[y] = key[y];
    __syncthreads();
    tail_price_update<WIDE>(C, n, cmin, np1, eps, qlim, skey, lab, lab + n, L, 0ull, vref, cap, ctrl);
    for (int y = threadIdx.x; y < n; y += blockDim.x) {
        key[y] = skey[y];
        lab_out[y] = lab[y];
    }
}

// Truncated labels and the new prices in the caller's sign and units.
__global__ void k_dbg_out(const unsigned long long *__restrict__ key, const unsigned *__restrict__ lab, int n,
                          const Ctrl *ctrl, int32_t *labels_out, int64_t *prices_out) {
    const unsigned long long K = ctrl->pu_levels;   // the truncation level applied (0: no update)
    const long long pm = ctrl->pmax;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        labels_out[y] = (int32_t)min((unsigned long long)lab[y], K);
        prices_out[y] = pm - (long long)key_q(key[y]);
    }
}

template <bool WIDE>
cudaError_t launch_dbg_tail_pu(cudaStream_t s, const int32_t *C, int n, int cmin, uint32_t np1, unsigned long long eps,
                               unsigned long long qlim, Workspace &ws, const RowLists &L) {
    const int smem = (int)(sizeof(unsigned long long) * n + tail_pu_smem(n));
    cudaError_t e = cudaFuncSetAttribute(k_dbg_tail_pu<WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_dbg_tail_pu<WIDE><<<1, tail_threads<WIDE>(), smem, s>>>(C, n, cmin, np1, eps, qlim, ws.key, ws.ctrl, L,
                                                              ws.pu_vref, ws.pu_cap, ws.pu_lab);
    return cudaGetLastError();
}

static la_status debug_price_update_locked(const int32_t *cost, int32_t n, const int64_t *prices,
                                           const int32_t *row_match, int64_t eps, cudaStream_t s,
                                           int32_t *labels_out, int64_t *prices_out, int32_t kernel) {
    int dev = 0;
    LA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    Workspace &ws = g_ws[dev];
    if (kernel == 1 && n > kTailMaxN) return LA_ERR_INVALID;   // the keys and labels must fit one SM
    if (la_status e = ensure_ws(ws, n)) return e;
    Ctrl init;
    std::memset(&init, 0, sizeof(init));
    init.cmin = INT_MAX;
    init.cmax = INT_MIN;
    init.qmin[0] = init.qmin[1] = ~0ull;
    init.pmax = LLONG_MIN;
    *ws.h_ctrl = init;
    LA_CK(cudaMemcpyAsync(ws.ctrl, ws.h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    const long long total = (long long)n * n;
    const int mm_grid = (int)std::max<long long>(1, std::min<long long>((total / 4 + 255) / 256, 8LL * ws.num_sms));
    const int sg = small_grid(n, 256, ws.num_sms);
    k_minmax<<<mm_grid, 256, 0, s>>>(cost, total, ws.ctrl);
    k_warm_pmax<<<sg, 256, 0, s>>>(reinterpret_cast<const long long *>(prices), n, ws.ctrl);
    k_warm_init<<<sg, 256, 0, s>>>(reinterpret_cast<const long long *>(prices), n, ws.key, ws.ctrl);
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));
    const Ctrl c0 = *ws.h_ctrl;
    const unsigned long long np1 = (unsigned long long)n + 1;
    const unsigned long long Ct = np1 * (unsigned long long)((long long)c0.cmax - (long long)c0.cmin);
    if (Ct >= kRangeLimit || c0.qspread >= (1ull << 42)) return LA_ERR_OVERFLOW;
    // the solver's choice of value width, for a phase at this eps
    const bool wide = c0.qspread + 4 * Ct + 2 * (unsigned long long)eps + 16 >= (1ull << 32);
    const unsigned long long qlim = wide ? (kQMax - 1) : ((1ull << 32) - 2 - Ct);
    const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(cost) & 15) == 0);
    const RowLists L{ws.lcols, ws.lcosts, ws.ltheta};
    const int lg = std::max(1, std::min((n + 7) / 8, 8 * ws.num_sms));   // 8 warps per block
    if (wide) {
        k_dbg_state<true><<<sg, 256, 0, s>>>(row_match, n, ws.key, ws.qm, ws.ctrl);
        k_dbg_mirror<true><<<sg, 256, 0, s>>>(ws.key, n, ws.qm, ws.ctrl);
        if (vec) k_dbg_lists<true, true><<<lg, 256, 0, s>>>(cost, n, c0.cmin, (uint32_t)np1, ws.qm, L);
        else k_dbg_lists<true, false><<<lg, 256, 0, s>>>(cost, n, c0.cmin, (uint32_t)np1, ws.qm, L);
        if (kernel == 1) LA_CK(launch_dbg_tail_pu<true>(s, cost, n, c0.cmin, (uint32_t)np1, (unsigned long long)eps, qlim, ws, L));
        else LA_CK(launch_pu<true>(s, cost, n, c0.cmin, (uint32_t)np1, (unsigned long long)eps, qlim, ws, L));
    } else {
        k_dbg_state<false><<<sg, 256, 0, s>>>(row_match, n, ws.key, ws.qm, ws.ctrl);
        k_dbg_mirror<false><<<sg, 256, 0, s>>>(ws.key, n, ws.qm, ws.ctrl);
        if (vec) k_dbg_lists<false, true><<<lg, 256, 0, s>>>(cost, n, c0.cmin, (uint32_t)np1, ws.qm, L);
        else k_dbg_lists<false, false><<<lg, 256, 0, s>>>(cost, n, c0.cmin, (uint32_t)np1, ws.qm, L);
        if (kernel == 1) LA_CK(launch_dbg_tail_pu<false>(s, cost, n, c0.cmin, (uint32_t)np1, (unsigned long long)eps, qlim, ws, L));
        else LA_CK(launch_pu<false>(s, cost, n, c0.cmin, (uint32_t)np1, (unsigned long long)eps, qlim, ws, L));
    }
    k_dbg_out<<<sg, 256, 0, s>>>(ws.key, ws.pu_lab, n, ws.ctrl, labels_out, prices_out);
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));
    return (la_status)ws.h_ctrl->status;
}



static la_status solve_locked(const int32_t *cost, int32_t n, const la_options *opt, cudaStream_t s,
                              int32_t *match_out, int64_t *cost_out, la_stats *st) {
    const int alpha = (opt && opt->alpha) ? opt->alpha : 10;
    const int64_t eps0 = opt ? opt->eps0 : 0;
    const int block = (opt && opt->block_threads) ? opt->block_threads : kDefaultBlock;
    const int64_t *init_prices = opt ? opt->init_prices : nullptr;
    int64_t *prices_out = opt ? opt->prices_out : nullptr;
    const bool profile = opt && opt->profile;
    const bool lists = !(opt && (opt->flags & LA_FLAG_NO_CANDIDATE_LISTS));
    int tail_T = (opt && opt->tail_threshold) ? opt->tail_threshold : kDefaultTailRows;
    if (tail_T < 0 || n > kTailMaxN) tail_T = 0;
    int pu_rounds = (opt && opt->price_updates) ? opt->price_updates : kDefaultPuRounds;
    if (pu_rounds < 0 || !lists) pu_rounds = 0;
    const int pu_T = std::max(16, n / 128);
    // grid price updates the tail kernel may stop for in each phase
    const int tail_updates = (lists && tail_T > 0 && opt && opt->tail_updates > 0) ? opt->tail_updates : 0;
    // intermediate phases stop at this many free rows (the last phase never does)
    // (off unless asked: see la_options.phase_cutoff)
    const int stop_free = (opt && opt->phase_cutoff > 0) ? opt->phase_cutoff : 0;
    const bool sweep = true;   // every phase opens with its bulk sweep
    const bool tail_pu = lists && opt && (opt->flags & LA_FLAG_TAIL_PRICE_UPDATE);
    // arc fixing needs an eps-optimal flow at every phase end (no cutoff);
    // the final prices certify only the arcs kept, so not with prices_out
    const bool arcfix = lists && !(opt && (opt->flags & LA_FLAG_NO_ARC_FIXING)) && stop_free == 0 &&
                        !(opt && opt->prices_out);
    if (alpha < 2 || eps0 < 0 || block < 32 || block > 256 || block % 32) return LA_ERR_INVALID;
    if (opt && opt->scan_budget < 0) return LA_ERR_INVALID;

    la_stats stats;
    std::memset(&stats, 0, sizeof(stats));
    stats.n = n;
    if (n == 0) {
        LA_CK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
        LA_CK(cudaStreamSynchronize(s));
        if (st) *st = stats;
        return LA_OK;
    }
    int dev = 0;
    LA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    Workspace &ws = g_ws[dev];
    if (la_status e = ensure_ws(ws, n)) return e;
    // team refine: one CTA of kTeamWarps warps per free row once at most 2
    // per SM are free (every variant of k_team fits 2 CTAs per SM)
    const int team_T = (lists && !(opt && (opt->flags & LA_FLAG_NO_TEAM_REFINE)))
                           ? std::max(1, std::min((opt && opt->team_threshold > 0) ? opt->team_threshold : 2 * ws.num_sms, n / 2))
                           : 0;

    Ctrl init;
    std::memset(&init, 0, sizeof(init));
    init.cmin = INT_MAX;
    init.cmax = INT_MIN;
    init.qmin[0] = init.qmin[1] = ~0ull;
    init.pmax = LLONG_MIN;
    init.team_T = team_T;
    *ws.h_ctrl = init;
    LA_CK(cudaMemcpyAsync(ws.ctrl, ws.h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    int64_t launches = 0;

    const long long total = (long long)n * n;
    const int mm_grid = (int)std::max<long long>(1, std::min<long long>((total / 4 + 255) / 256, 8LL * ws.num_sms));
    k_minmax<<<mm_grid, 256, 0, s>>>(cost, total, ws.ctrl);
    ++launches;
    if (n == 1) {
        k_single<<<1, 1, 0, s>>>(cost, match_out, reinterpret_cast<long long *>(cost_out),
                                 reinterpret_cast<long long *>(prices_out));
        ++launches;
        LA_CK(cudaGetLastError());
        LA_CK(cudaStreamSynchronize(s));
        stats.launches = launches;
        if (st) *st = stats;
        return LA_OK;
    }
    const int sg = small_grid(n, 256, ws.num_sms);
    if (init_prices) {
        k_warm_pmax<<<sg, 256, 0, s>>>(reinterpret_cast<const long long *>(init_prices), n, ws.ctrl);
        k_warm_init<<<sg, 256, 0, s>>>(reinterpret_cast<const long long *>(init_prices), n, ws.key, ws.ctrl);
        launches += 2;
    } else {
        LA_CK(cudaMemsetAsync(ws.key, 0xff, sizeof(unsigned long long) * n, s));  // q = 0, no mate
    }
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));
    const Ctrl c0 = *ws.h_ctrl;

    const unsigned long long np1 = (unsigned long long)n + 1;
    const unsigned long long range = (unsigned long long)((long long)c0.cmax - (long long)c0.cmin);
    const unsigned long long Ct = np1 * range;
    const unsigned long long S = init_prices ? c0.qspread : 0;
    stats.scaled_range = (int64_t)Ct;
    if (Ct >= kRangeLimit || S >= (1ull << 42)) return LA_ERR_OVERFLOW;

    // epsilon schedule (Algorithm 5.0): eps <- max(1, eps / alpha) until 1,
    // with alpha_fine (if set) once eps is down to sixteen cost units
    std::vector<unsigned long long> sched;
    {
        const int alpha_fine = (opt && opt->alpha_fine >= 2) ? opt->alpha_fine : alpha;
        unsigned long long e = eps0 > 0 ? (unsigned long long)eps0 : Ct;
        do {
            const int a = e <= 16ull * np1 ? alpha_fine : alpha;
            e = std::max<unsigned long long>(1, e / (unsigned long long)a);
            sched.push_back(e);
        } while (e > 1 && (int)sched.size() < kMaxPhases);
        if (sched.back() != 1) return LA_ERR_INVALID;
    }
    stats.eps_first = (int64_t)sched[0];
    // 32-bit reduced costs when every v = c~ + q provably fits: a phase from
    // spread S' keeps q <= S' + 2 C~ + 2 eps and ends with S' <= C~ + eps.
    const unsigned long long need32 = S + 4 * Ct + 2 * sched[0] + 16;
    const bool wide = need32 >= (1ull << 32);
    const unsigned long long qlim = wide ? (kQMax - 1) : ((1ull << 32) - 2 - Ct);
    const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(cost) & 15) == 0);
    stats.wide = wide;
    stats.vector_loads = vec;

    RowLists L{nullptr, nullptr, nullptr};
    if (lists) {
        L = RowLists{ws.lcols, ws.lcosts, ws.ltheta};
        LA_CK(cudaMemsetAsync(ws.ltheta, 0, sizeof(unsigned long long) * n, s));
    }
    unsigned long long budget = opt && opt->scan_budget ? (unsigned long long)opt->scan_budget
                                                        : 256ull * n * sched.size() + (1ull << 22);
    int grid = 0;
    if (wide) grid = vec ? refine_grid<true, true>(ws.num_sms, block, n) : refine_grid<true, false>(ws.num_sms, block, n);
    else grid = vec ? refine_grid<false, true>(ws.num_sms, block, n) : refine_grid<false, false>(ws.num_sms, block, n);

    const int cmin = c0.cmin;
    // debug mode: scratch for the phase-end checks (allocated per call)
    const bool check = opt && (opt->flags & LA_FLAG_CHECK_PHASES);
    unsigned long long *chk_q0 = nullptr;
    int *chk_seen = nullptr;
    struct ChkFree {
        unsigned long long *&q0;
        int *&seen;
        ~ChkFree() {
            cudaFree(q0);
            cudaFree(seen);
        }
    } chk_free{chk_q0, chk_seen};
    if (check) {
        if (cudaMalloc(&chk_q0, sizeof(unsigned long long) * n) != cudaSuccess ||
            cudaMalloc(&chk_seen, sizeof(int) * n) != cudaSuccess)
            return LA_ERR_NOMEM;
    }
    // small instances: the whole solve on one CTA with the matrix in shared memory
    const bool c16 = range <= 65535 && n <= kSmallMaxN16;
    const bool small = !check && stop_free == 0 && pu_rounds == 0 && !(opt && (opt->flags & LA_FLAG_NO_SMALL_KERNEL)) &&
                       (c16 || n <= kSmallMaxN32) && (int)sched.size() <= kMaxPhases;
    int ph = 0;
    if (small) {
        unsigned long long *dsched = reinterpret_cast<unsigned long long *>(ws.tail_rows);   // n >= 2 ints: room for
        if (ws.cap < (int64_t)(2 * sched.size())) return LA_ERR_INTERNAL;                   // the eps schedule
        LA_CK(cudaMemcpyAsync(dsched, sched.data(), sizeof(unsigned long long) * sched.size(), cudaMemcpyHostToDevice, s));
        const int smem = (int)(sizeof(unsigned long long) * n + (size_t)n * n * (c16 ? 2 : 4));
        if (profile) LA_CK(cudaEventRecord(ws.ev[0], s));
        const int nph = (int)sched.size();
        if (wide) {
            if (c16) {
                LA_CK(cudaFuncSetAttribute(k_small<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_small<true, true><<<1, kSmallThreads, smem, s>>>(cost, n, cmin, (uint32_t)np1, dsched, nph, qlim, ws.key, ws.ctrl, budget);
            } else {
                LA_CK(cudaFuncSetAttribute(k_small<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_small<true, false><<<1, kSmallThreads, smem, s>>>(cost, n, cmin, (uint32_t)np1, dsched, nph, qlim, ws.key, ws.ctrl, budget);
            }
        } else {
            if (c16) {
                LA_CK(cudaFuncSetAttribute(k_small<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_small<false, true><<<1, kSmallThreads, smem, s>>>(cost, n, cmin, (uint32_t)np1, dsched, nph, qlim, ws.key, ws.ctrl, budget);
            } else {
                LA_CK(cudaFuncSetAttribute(k_small<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
                k_small<false, false><<<1, kSmallThreads, smem, s>>>(cost, n, cmin, (uint32_t)np1, dsched, nph, qlim, ws.key, ws.ctrl, budget);
            }
        }
        if (profile) LA_CK(cudaEventRecord(ws.ev[4], s));
        LA_CK(cudaGetLastError());
        launches += 1;
        ph = nph;
    }
    for (; !small && ph < (int)sched.size(); ++ph) {
        const int slot = ph & 1;
        k_qmin<<<sg, 256, 0, s>>>(ws.key, n, ws.ctrl, slot);
        if (wide) k_reset<true><<<sg, 256, 0, s>>>(ws.key, ws.qm, n, qlim, ws.ctrl, slot, ph, pu_rounds + tail_updates);
        else k_reset<false><<<sg, 256, 0, s>>>(ws.key, ws.qm, n, qlim, ws.ctrl, slot, ph, pu_rounds + tail_updates);
        launches += 2;
        if (check) {
            k_check_snapshot<<<sg, 256, 0, s>>>(ws.key, n, chk_q0);
            ++launches;
        }
        if (profile) LA_CK(cudaEventRecord(ws.ev[5 * ph], s));
        const int sf = ph + 1 < (int)sched.size() ? stop_free : 0;
        cudaEvent_t evs = profile ? ws.ev[5 * ph + 1] : nullptr;
        cudaEvent_t evt = profile ? ws.ev[5 * ph + 2] : nullptr;
        cudaEvent_t evf = profile ? ws.ev[5 * ph + 3] : nullptr;
        if (wide) {
            if (vec) LA_CK((launch_refine<true, true>(s, grid, block, cost, n, cmin, (uint32_t)np1, sched[ph], qlim, ws, budget, L, tail_T, pu_T, pu_rounds, launches, sf, evs, evt, evf, sweep, tail_pu, team_T, tail_updates)));
            else LA_CK((launch_refine<true, false>(s, grid, block, cost, n, cmin, (uint32_t)np1, sched[ph], qlim, ws, budget, L, tail_T, pu_T, pu_rounds, launches, sf, evs, evt, evf, sweep, tail_pu, team_T, tail_updates)));
        } else {
            if (vec) LA_CK((launch_refine<false, true>(s, grid, block, cost, n, cmin, (uint32_t)np1, sched[ph], qlim, ws, budget, L, tail_T, pu_T, pu_rounds, launches, sf, evs, evt, evf, sweep, tail_pu, team_T, tail_updates)));
            else LA_CK((launch_refine<false, false>(s, grid, block, cost, n, cmin, (uint32_t)np1, sched[ph], qlim, ws, budget, L, tail_T, pu_T, pu_rounds, launches, sf, evs, evt, evf, sweep, tail_pu, team_T, tail_updates)));
        }
        if (profile) LA_CK(cudaEventRecord(ws.ev[5 * ph + 4], s));
        if (check) {
            LA_CK(cudaMemsetAsync(chk_seen, 0, sizeof(int) * n, s));
            const int cg = std::max(1, std::min((n + 7) / 8, 8 * ws.num_sms));   // 8 warps per block
            k_check_phase<<<cg, 256, 0, s>>>(cost, n, cmin, np1, ws.key, chk_q0, sched[ph],
                                             (sf == 0) ? 1 : 0, chk_seen, ws.ctrl, L);
            ++launches;
            LA_CK(cudaGetLastError());
        }
        if (arcfix && ph + 1 < (int)sched.size()) {
            const unsigned long long T = (2ull * (unsigned long long)n + 1) * sched[ph];
            // T <= C~ / 16 leaves rows with a few arcs each: worth a full pass
            const int full_pass = T <= Ct / 16 ? 1 : 0;
            if (T < Ct) {   // otherwise no arc can go
                const int fg = std::max(1, std::min((n + 7) / 8, 8 * ws.num_sms));   // 8 warps per block
                if (vec) k_fix<true><<<fg, 256, 0, s>>>(cost, n, cmin, (uint32_t)np1, T, ws.key, L, ws.ctrl, full_pass, ph);
                else k_fix<false><<<fg, 256, 0, s>>>(cost, n, cmin, (uint32_t)np1, T, ws.key, L, ws.ctrl, full_pass, ph);
                ++launches;
                LA_CK(cudaGetLastError());
            }
        }
    }
    const int fslot = ph & 1;
    if (prices_out) {
        k_qmin<<<sg, 256, 0, s>>>(ws.key, n, ws.ctrl, fslot);
        ++launches;
    }
    LA_CK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
    k_finalize<<<sg, 256, 0, s>>>(cost, n, ws.key, match_out, reinterpret_cast<long long *>(cost_out),
                                  reinterpret_cast<long long *>(prices_out), ws.ctrl, fslot);
    ++launches;
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(ws.h_ctrl, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));
    const Ctrl c1 = *ws.h_ctrl;

    stats.phases = (int64_t)sched.size();
    stats.scans = (int64_t)c1.scans;
    stats.wins = (int64_t)c1.wins;
    stats.displaced = (int64_t)c1.displaced;
    stats.launches = launches;
    stats.refine_launches = small ? 1 : (int64_t)sched.size() * (1 + pu_rounds + (tail_T > 0 ? 1 : 0) + (sweep ? 1 : 0) + (team_T > 0 ? 1 + pu_rounds + (tail_T > 0 ? 1 : 0) : 0) +
                                                      tail_updates * (team_T > 0 ? 2 : 1));
    stats.small_kernel = small ? 1 : 0;
    stats.tail_price_update_ms = 1e-6 * (double)c1.pu_tail_ns;
    stats.team_phases = c1.team_phases;
    stats.team_scans = (int64_t)c1.team_scans;
    stats.team_full_scans = (int64_t)c1.team_full;
    stats.price_updates = (int64_t)c1.pu_updates;
    stats.price_update_sweeps = (int64_t)c1.pu_iters;
    stats.price_update_levels = (int64_t)c1.pu_levels;
    stats.max_chain = (int64_t)c1.max_chain;
    stats.full_scans = (int64_t)c1.full_scans;
    stats.list_scans = (int64_t)c1.list_scans;
    stats.tail_scans = (int64_t)c1.tail_scans;
    stats.tail_full_scans = (int64_t)c1.tail_full;
    stats.tail_giveups = c1.tail_giveups;
    stats.sweep_scans = (int64_t)c1.sweep_scans;
    stats.sweep_full_scans = (int64_t)c1.sweep_full;
    stats.tail_phases = c1.tail_phases;
    for (int k = 0; k < ph && k < LA_STATS_PHASES; ++k) {
        const bool last = k + 1 >= ph;
        stats.phase_scans[k] = (int64_t)((last ? c1.scans : c1.phase_start_scans[k + 1]) - c1.phase_start_scans[k]);
        stats.phase_full_scans[k] =
            (int64_t)((last ? c1.full_scans : c1.phase_start_full[k + 1]) - c1.phase_start_full[k]);
        stats.phase_tail_scans[k] =
            (int64_t)((last ? c1.tail_scans : c1.phase_start_tail[k + 1]) - c1.phase_start_tail[k]);
        stats.phase_fixed_rows[k] = (int64_t)c1.fix_rows[k];
        if (c1.fix_rows[k]) {
            stats.fixed_rows = (int64_t)c1.fix_rows[k];
            stats.fixed_arcs = (int64_t)c1.fix_arcs[k];
        }
    }
    stats.list_entries = lists ? kListLen : 0;
    stats.checked_phases = c1.checked_phases;
    stats.stop_phase = c1.status ? c1.phase_now : -1;
    stats.stop_eps = c1.status ? (int64_t)sched[std::min<int>(std::max(c1.phase_now, 0), (int)sched.size() - 1)] : 0;
    stats.check_violations = (int64_t)c1.check_violations;
    if (profile && small) {   // one launch for every phase
        float t = 0;
        LA_CK(cudaEventElapsedTime(&t, ws.ev[0], ws.ev[4]));
        stats.refine_ms = t;
    } else if (profile) {
        double ms = 0, tail_ms = 0, sweep_ms = 0;
        for (int k = 0; k < ph; ++k) {
            float t = 0, tt = 0;
            float ts = 0;
            LA_CK(cudaEventElapsedTime(&t, ws.ev[5 * k], ws.ev[5 * k + 4]));
            LA_CK(cudaEventElapsedTime(&tt, ws.ev[5 * k + 2], ws.ev[5 * k + 3]));
            LA_CK(cudaEventElapsedTime(&ts, ws.ev[5 * k], ws.ev[5 * k + 1]));
            sweep_ms += ts;
            ms += t;
            tail_ms += tt;
            if (k < LA_STATS_PHASES) {
                stats.phase_ms[k] = t;
                stats.phase_tail_ms[k] = tt;
            }
        }
        stats.refine_ms = ms;
        stats.tail_ms = tail_ms;
        stats.sweep_ms = sweep_ms;
    }
    if (st) *st = stats;
    if (c1.status == 0 && check && (c1.check_violations != 0 || c1.checked_phases != ph)) return LA_ERR_INTERNAL;
    return (la_status)c1.status;
}

extern "C" {

la_status la_solve_ex(const int32_t *cost, int32_t n, const la_options *opt, void *stream,
                      int32_t *match_out, int64_t *cost_out, la_stats *stats_out) {
    if (n < 0 || n > LA_MAX_N || !cost_out || (n > 0 && !cost)) return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mu);
    return solve_locked(cost, n, opt, static_cast<cudaStream_t>(stream), match_out, cost_out, stats_out);
}

la_status la_solve(const int32_t *cost, int32_t n, void *stream, int32_t *match_out, int64_t *cost_out) {
    return la_solve_ex(cost, n, nullptr, stream, match_out, cost_out, nullptr);
}

const char *la_status_string(la_status s) {
    switch (s) {
    case LA_OK: return "LA_OK";
    case LA_ERR_INVALID: return "LA_ERR_INVALID: invalid argument";
    case LA_ERR_CUDA: return "LA_ERR_CUDA: a CUDA runtime call failed";
    case LA_ERR_OVERFLOW: return "LA_ERR_OVERFLOW: cost range too large for the exact price field";
    case LA_ERR_ITER_LIMIT: return "LA_ERR_ITER_LIMIT: row-scan budget exhausted";
    case LA_ERR_NOMEM: return "LA_ERR_NOMEM: device workspace allocation failed";
    case LA_ERR_INTERNAL: return "LA_ERR_INTERNAL: device consistency check failed";
    case LA_ERR_TOO_LARGE: return "LA_ERR_TOO_LARGE: n exceeds the fixed scratch size";
    case LA_ERR_INFEASIBLE: return "LA_ERR_INFEASIBLE: the graph has no perfect matching";
    }
    return "unknown la_status";
}

la_status la_debug_price_update(const int32_t *cost, int32_t n, const int64_t *prices, const int32_t *row_match,
                                int64_t eps, void *stream, int32_t *labels_out, int64_t *prices_out,
                                int32_t kernel) {
    if (n < 2 || n > LA_MAX_N || eps < 1 || !cost || !prices || !row_match || !labels_out || !prices_out ||
        (kernel != 0 && kernel != 1))
        return LA_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mu);
    return debug_price_update_locked(cost, n, prices, row_match, eps, static_cast<cudaStream_t>(stream),
                                     labels_out, prices_out, kernel);
}

la_status la_release_workspace(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LA_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    if (cudaDeviceSynchronize() != cudaSuccess) return LA_ERR_CUDA;
    free_ws(g_ws[dev]);
    return LA_OK;
}

int32_t la_version(void) { return 100; }

}  // extern "C"

// ------------------------------------------------------------------------
// la_solve_noalloc: the same solve for callers that cannot allocate.
//
// The column keys, the price mirror and the control block live in one
// fixed array in device memory, declared below, instead of the per-device
// workspace. Kernels receive the array's device address; host code obtains
// it once per device with cudaGetSymbolAddress (in host code the symbol
// itself is only a host-side stand-in, not a device address).
// ------------------------------------------------------------------------

namespace {
constexpr size_t kNoallocKeyOff = 0;
constexpr size_t kNoallocQmOff = sizeof(unsigned long long) * LA_NOALLOC_MAX_N;
constexpr size_t kNoallocCtrlOff = 2 * sizeof(unsigned long long) * LA_NOALLOC_MAX_N;
constexpr size_t kNoallocBytes = kNoallocCtrlOff + ((sizeof(Ctrl) + 255) / 256) * 256;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch
    int num_sms = 0;
};
NoallocDevice g_noalloc[kMaxDevices];

// Once per device, with that device current.
la_status noalloc_setup(int dev, NoallocDevice &d) {
    if (d.ready) return LA_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return LA_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LA_ERR_CUDA;
    d.base = static_cast<unsigned char *>(p);
    d.num_sms = sms;
    d.ready = true;
    return LA_OK;
}

la_status solve_noalloc_locked(const int32_t *cost, int32_t n, cudaStream_t s, int32_t *match_out,
                               int64_t *cost_out) {
    if (n == 0) {
        LA_CK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
        LA_CK(cudaStreamSynchronize(s));
        return LA_OK;
    }
    int dev = 0;
    LA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    NoallocDevice &d = g_noalloc[dev];
    if (la_status e = noalloc_setup(dev, d)) return e;
    unsigned long long *key = reinterpret_cast<unsigned long long *>(d.base + kNoallocKeyOff);
    void *qm = d.base + kNoallocQmOff;
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(d.base + kNoallocCtrlOff);

    // the array keeps the previous call's contents: start the control block clean
    Ctrl h;
    std::memset(&h, 0, sizeof(h));
    h.cmin = INT_MAX;
    h.cmax = INT_MIN;
    h.qmin[0] = h.qmin[1] = ~0ull;
    h.pmax = LLONG_MIN;
    LA_CK(cudaMemcpyAsync(ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, s));

    const long long total = (long long)n * n;
    const int mm_grid = (int)std::max<long long>(1, std::min<long long>((total / 4 + 255) / 256, 8LL * d.num_sms));
    k_minmax<<<mm_grid, 256, 0, s>>>(cost, total, ctrl);
    if (n == 1) {
        k_single<<<1, 1, 0, s>>>(cost, match_out, reinterpret_cast<long long *>(cost_out), nullptr);
        LA_CK(cudaGetLastError());
        LA_CK(cudaStreamSynchronize(s));
        return LA_OK;
    }
    LA_CK(cudaMemsetAsync(key, 0xff, sizeof(unsigned long long) * n, s));  // q = 0, no mate
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));

    const unsigned long long np1 = (unsigned long long)n + 1;
    const unsigned long long Ct = np1 * (unsigned long long)((long long)h.cmax - (long long)h.cmin);
    if (Ct >= kRangeLimit) return LA_ERR_OVERFLOW;
    std::vector<unsigned long long> sched;
    unsigned long long e = Ct;
    do {
        e = std::max<unsigned long long>(1, e / 10);
        sched.push_back(e);
    } while (e > 1);
    const bool wide = 4 * Ct + 2 * sched[0] + 16 >= (1ull << 32);
    const unsigned long long qlim = wide ? (kQMax - 1) : ((1ull << 32) - 2 - Ct);
    const bool vec = (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(cost) & 15) == 0);
    const unsigned long long budget = 256ull * n * sched.size() + (1ull << 22);
    const int block = kDefaultBlock;
    int grid = 0;
    if (wide) grid = vec ? refine_grid<true, true>(d.num_sms, block, n) : refine_grid<true, false>(d.num_sms, block, n);
    else grid = vec ? refine_grid<false, true>(d.num_sms, block, n) : refine_grid<false, false>(d.num_sms, block, n);
    const int sg = small_grid(n, 256, d.num_sms);
    const int cmin = h.cmin;
    int ph = 0;
    for (; ph < (int)sched.size(); ++ph) {
        const int slot = ph & 1;
        k_qmin<<<sg, 256, 0, s>>>(key, n, ctrl, slot);
        if (wide) k_reset<true><<<sg, 256, 0, s>>>(key, qm, n, qlim, ctrl, slot, ph, 0);
        else k_reset<false><<<sg, 256, 0, s>>>(key, qm, n, qlim, ctrl, slot, ph, 0);
        if (wide) {
            if (vec) k_refine<true, true><<<grid, block, 0, s>>>(cost, n, cmin, (uint32_t)np1, sched[ph], qlim, key, qm, ctrl, budget, RowLists{nullptr, nullptr, nullptr}, 0, nullptr, 0, nullptr, nullptr, 0, 0);
            else k_refine<true, false><<<grid, block, 0, s>>>(cost, n, cmin, (uint32_t)np1, sched[ph], qlim, key, qm, ctrl, budget, RowLists{nullptr, nullptr, nullptr}, 0, nullptr, 0, nullptr, nullptr, 0, 0);
        } else {
            if (vec) k_refine<false, true><<<grid, block, 0, s>>>(cost, n, cmin, (uint32_t)np1, sched[ph], qlim, key, qm, ctrl, budget, RowLists{nullptr, nullptr, nullptr}, 0, nullptr, 0, nullptr, nullptr, 0, 0);
            else k_refine<false, false><<<grid, block, 0, s>>>(cost, n, cmin, (uint32_t)np1, sched[ph], qlim, key, qm, ctrl, budget, RowLists{nullptr, nullptr, nullptr}, 0, nullptr, 0, nullptr, nullptr, 0, 0);
        }
    }
    LA_CK(cudaMemsetAsync(cost_out, 0, sizeof(int64_t), s));
    k_finalize<<<sg, 256, 0, s>>>(cost, n, key, match_out, reinterpret_cast<long long *>(cost_out), nullptr,
                                  ctrl, ph & 1);
    LA_CK(cudaGetLastError());
    LA_CK(cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    LA_CK(cudaStreamSynchronize(s));
    return (la_status)h.status;
}

}  // namespace

extern "C" la_status la_solve_noalloc(const int32_t *cost, int32_t n, void *stream, int32_t *match_out,
                                      int64_t *cost_out) {
    if (n < 0 || !cost_out || (n > 0 && !cost)) return LA_ERR_INVALID;
    if (n > LA_NOALLOC_MAX_N) return LA_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lock(g_mu);
    return solve_noalloc_locked(cost, n, static_cast<cudaStream_t>(stream), match_out, cost_out);
}
