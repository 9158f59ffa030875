// la_solve_batched: many independent dense assignments in one persistent
// launch (captured in a CUDA graph and replayed).
//
// Each CTA keeps up to S instances resident ("slots") and runs the whole
// cost-scaling solve of each (Sect. 5.1, Algorithm 5.0's epsilon loop;
// refine initialisation of Algorithm 5.2; the push / relabel of Algorithm
// 5.4 as a double push) with the instance's column keys in shared memory:
//   * one 64-bit key per column, (price, mate) packed as in la_solve, so a
//     bid is one shared-memory atomicMin;
//   * the CTA's warps take free rows from any resident instance (one
//     shared-memory atomicAdd on the slot's claim word), scan the row against
//     the shared prices, bid, and continue with the row they displaced;
//   * a row is read into the warp's shared-memory buffer by one bulk copy
//     (cp.async.bulk on a per-warp mbarrier), or, for large instances,
//     through its exact candidate list as in la_solve;
//   * an instance's phase ends when its last row is matched, with no CTA
//     barrier; the warp that matched it starts the next phase or writes the
//     instance's results and loads the next instance (largest first) from
//     the device work queue.
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
#include "la_lists.cuh"

using namespace la;

namespace {

constexpr int kPrepThreads = 1024;
constexpr int kDefaultSlots = 4;                 // instances resident per CTA
constexpr size_t kSlotSmemBudget = 192 * 1024;   // shared memory for their column keys
constexpr int kMaxDevices = 64;
constexpr int kAutoListsN = 2048;                       // default: lists when max_n is at least this
constexpr size_t kAutoListsBytes = 4ull << 30;          // ... and they fit in this
constexpr bool kStageRows = true;                       // bulk-copy row staging in the list-free kernel
constexpr size_t kStageSmemBudget = 200 * 1024;         // its shared memory (keys + row buffers) at most

struct BatchCtrl {
    unsigned long long scan_bytes;   // 4 n bytes per full row scan, kListLen * 8 + 8 per list scan
    unsigned long long scans;
    unsigned long long full_scans;
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

// Per-instance min and max cost (a bandwidth-bound pass over the whole
// batch before the solve): block b reduces instances b, b + gridDim.x, ...
__global__ void __launch_bounds__(256)
k_batch_minmax(const int32_t *__restrict__ C, const long long *__restrict__ offsets,
               const int *__restrict__ ns, int B, int max_n, int2 *__restrict__ cminmax) {
    __shared__ int s_lo[8], s_hi[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = blockIdx.x; i < B; i += gridDim.x) {
        const int n = ns[i];
        int lo = INT_MAX, hi = INT_MIN;
        if (n > 0 && n <= max_n) {
            const int32_t *Ci = C + offsets[i];
            const long long tot = (long long)n * n;
            if ((reinterpret_cast<uintptr_t>(Ci) & 15) == 0) {
                const int4 *C4 = reinterpret_cast<const int4 *>(Ci);
                const long long nv = tot >> 2;
                for (long long e = tid; e < nv; e += 256) {
                    const int4 c = ld_row4(C4 + e);
                    lo = min(lo, min(min(c.x, c.y), min(c.z, c.w)));
                    hi = max(hi, max(max(c.x, c.y), max(c.z, c.w)));
                }
                for (long long e = (nv << 2) + tid; e < tot; e += 256) {
                    const int c = ld_row1(Ci + e);
                    lo = min(lo, c);
                    hi = max(hi, c);
                }
            } else {
                for (long long e = tid; e < tot; e += 256) {
                    const int c = ld_row1(Ci + e);
                    lo = min(lo, c);
                    hi = max(hi, c);
                }
            }
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) {
            s_lo[warp] = lo;
            s_hi[warp] = hi;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < 8; ++w) {
                lo = min(lo, s_lo[w]);
                hi = max(hi, s_hi[w]);
            }
            cminmax[i] = make_int2(lo, hi);
        }
        __syncthreads();
    }
}

// Row staging by the bulk-copy engine (list-free kernel): a warp asks for
// its whole cost row with one cp.async.bulk into its own shared-memory
// buffer and waits on its own mbarrier, instead of having every lane load
// its part of the row from L2 in several dependent rounds.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Lane 0: expect `bytes` on the barrier and start the copy (global src and
// shared dst 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_row(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    unsigned long long g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Every lane waits for the phase `parity` of the barrier to complete; false
// after 1 s (the copy is then treated as lost).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const unsigned long long t0 = global_timer_ns();
    for (unsigned it = 0;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 255) == 255 && global_timer_ns() - t0 > 1000000000ull) return false;
    }
}
// Ints per warp buffer: a row of max_n ints starting at any 4-byte offset,
// widened to 16-byte boundaries at both ends.
__host__ __device__ __forceinline__ int stage_stride(int max_n) { return (max_n + 8 + 3) & ~3; }
// The keys of S slots in u64 words, rounded up so that the row buffers start 16-byte aligned.
__host__ __device__ __forceinline__ size_t stage_key_words(int S, int max_n) {
    return ((size_t)S * (size_t)max_n + 1) & ~(size_t)1;
}
__host__ __device__ __forceinline__ size_t stage_smem(int S, int max_n, int warps) {
    return stage_key_words(S, max_n) * 8 + (size_t)warps * stage_stride(max_n) * 4 + (size_t)warps * 8;
}

// Key formats. 64-bit instances, and every instance of the lists kernel, use
// la_solve's packing, (2^44 - 1 - q) << 20 | mate. 32-bit instances of the
// list-free kernel use (2^32 - 1 - q) << 32 | mate: a scan then reads a
// column's price as the key's high word, one 32-bit load and no shifts.
// Both order keys by price, then holder, so a bid is the same atomicMin.
constexpr uint32_t kNone32 = 0xFFFFFFFFu;
__device__ __forceinline__ unsigned long long bkey_pack(bool k32, unsigned long long q, uint32_t mate) {
    return k32 ? (((0xFFFFFFFFull - q) << 32) | mate) : pack_key(q, mate);
}
__device__ __forceinline__ unsigned long long bkey_q(bool k32, unsigned long long k) {
    return k32 ? (0xFFFFFFFFull - (k >> 32)) : key_q(k);
}
__device__ __forceinline__ uint32_t bkey_mate(bool k32, unsigned long long k) {
    return k32 ? (uint32_t)k : key_mate(k);
}
__device__ __forceinline__ uint32_t bkey_none(bool k32) { return k32 ? kNone32 : kNone; }

// v(y) = (c - cmin)(n + 1) + q(y) for a scanned cost c. With 32-bit keys,
// q(y) = 2^32 - 1 - hi(key(y)) and the constant folds into k2 =
// -cmin (n + 1) - 1 (mod 2^32): v = c (n + 1) + k2 - hi, exact because a
// 32-bit instance's values fit in 32 bits.
template <bool WIDE, bool K32, typename V>
__device__ __forceinline__ V bval(int c, int y, int cmin, uint32_t np1, uint32_t k2,
                                  const volatile unsigned long long *vkey) {
    if (K32) {
        const volatile uint32_t *hi = reinterpret_cast<const volatile uint32_t *>(vkey);
        return (V)((uint32_t)c * np1 + k2 - hi[2 * y + 1]);
    } else {
        return (V)(uint32_t)(c - cmin) * np1 + (V)key_q(vkey[y]);
    }
}

// One instance resident in a CTA. Rows are claimed with one atomicAdd on
// `claim` = (n << 32) | next row: a claim is valid exactly when the returned
// index is below the returned n, so no claim can land between two phases or
// two instances (the slot is republished by one atomicExch after its fields
// are written).
struct Slot {
    unsigned long long claim;
    unsigned long long eps, qlim, budget, scans;
    unsigned long long full;     // full row scans (all of them without lists)
    unsigned long long rebase;   // sum of the per-phase price shifts (candidate-list bounds)
    long long off;       // element offset of the instance's matrix
    long long moff;      // offset of its rows in match_out / prices_out
    int inst;            // instance index, -1 = empty
    int n, cmin, phase, nph, alpha, wide, vec;
    int k32;             // keys in the 32-bit-price format (bkey_*)
    int unmatched;       // rows not yet matched (or given up) in this phase
    int status;
};
constexpr int kMaxSlots = 8;

struct BatchArgs {
    const int32_t *C;
    const long long *offsets;
    const int *ns;
    const int *order;
    const long long *moff;
    const int2 *cminmax;
    int B, max_n;
    BatchParams P;
    int32_t *match_out;
    long long *cost_out;
    int *inst_status;
    BatchCtrl *ctrl;
    long long *prices_out;
    RowLists lists;   // candidate lists, row g = moff[i] + x of instance i (cols == nullptr: off)
};

__device__ __forceinline__ void finish_trivial(const BatchArgs &a, int i, int st, long long cost, int ctrl_failed) {
    if (a.cost_out) a.cost_out[i] = cost;
    if (a.inst_status) a.inst_status[i] = st;
    if (st && ctrl_failed) {
        atomicAdd(&a.ctrl->failed, 1);
        atomicCAS(&a.ctrl->status, 0, st);
    }
}

// Loads the next instance of the work queue (largest first) into a slot
// (one warp). Instances that need no refine (n = 0 or 1, an invalid n, a
// cost range beyond the exact price field) are finished on the spot. The
// slot is left empty once the queue is drained.
__device__ void load_next(const BatchArgs &a, Slot &sl, unsigned long long *keys, int lane) {
    volatile Slot &v = sl;
    for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&a.ctrl->next, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= a.B) {
            if (lane == 0) {
                v.inst = -1;
                v.claim = 0ull;
            }
            __syncwarp();
            return;
        }
        const int i = a.order[k];
        const int n = a.ns[i];
        if (n < 0 || n > a.max_n || n == 0) {
            if (lane == 0) finish_trivial(a, i, n == 0 ? 0 : (int)LA_ERR_INVALID, 0, 1);
            continue;
        }
        const int2 mm = a.cminmax[i];
        const unsigned long long np1 = (unsigned long long)n + 1;
        const unsigned long long Ct = np1 * (unsigned long long)((long long)mm.y - (long long)mm.x);
        if (Ct >= (1ull << 40)) {
            if (lane == 0) finish_trivial(a, i, (int)LA_ERR_OVERFLOW, 0, 1);
            continue;
        }
        if (n == 1) {
            if (lane == 0) {
                if (a.match_out) a.match_out[a.moff[i]] = 0;
                if (a.prices_out) a.prices_out[a.moff[i]] = 0;
                finish_trivial(a, i, 0, (long long)a.C[a.offsets[i]], 0);
            }
            continue;
        }
        const int alpha = max(2, a.P.alpha[log2_bucket(n)]);
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
        for (int y = lane; y < n; y += 32) keys[y] = ~0ull;   // q = 0, no mate
        if (a.lists.cols) {   // no row of this instance has a list yet
            const long long mo = a.moff[i];
            for (int y = lane; y < n; y += 32) a.lists.theta[mo + y] = 0ull;
        }
        if (lane == 0) {
            v.inst = i;
            v.n = n;
            v.cmin = mm.x;
            v.off = a.offsets[i];
            v.moff = a.moff[i];
            v.alpha = alpha;
            v.nph = nph;
            v.phase = 0;
            v.eps = eps1;
            v.wide = wide;
            v.k32 = !wide && !a.lists.cols;
            v.qlim = wide ? (kQMax - 1) : ((1ull << 32) - 2 - Ct);
            v.vec = ((a.offsets[i] & 3) == 0) && (n % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15) == 0);
            v.budget = (unsigned long long)a.P.budget_factor * n * nph + 4096;
            v.scans = 0;
            v.full = 0;
            v.rebase = 0;
            v.status = 0;
            v.unmatched = n;
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) atomicExch(&sl.claim, (unsigned long long)n << 32);
        __syncwarp();
        return;
    }
}

// The displacement chain of one claimed row (one warp): scan, double push
// (one shared-memory atomicMin on the column key), continue with the row it
// displaced, until a bid lands on a column nobody held. Returns true when
// that made the slot's last row matched: the phase is over and the caller
// runs the next one.
//
// With LISTS, a row is scanned through its candidate list when the list
// decides its bid, else in full (rebuilding the list), exactly as in the
// single solve; every warp of the instance runs on this CTA's SM, so the
// lists may be read through L1.
template <bool WIDE, bool LISTS, bool STAGE>
__device__ bool run_chain(Slot &sl, unsigned long long *keys, const int32_t *__restrict__ Ci, int row, int n,
                          int cmin, unsigned long long eps, unsigned long long qlim, unsigned long long budget,
                          bool vec, int lane, unsigned long long &wins, unsigned long long &displaced,
                          const RowLists &Li, unsigned long long R, int *sbuf, unsigned long long *sbar,
                          unsigned &spar, bool &sok) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    constexpr bool K32 = !WIDE && !LISTS;
    const volatile unsigned long long *vkey = keys;
    const uint32_t np1 = (uint32_t)n + 1;
    const uint32_t k2 = (0u - (uint32_t)cmin) * np1 - 1u;
    for (;;) {
        unsigned long long s = 0;
        int st = 0;
        if (lane == 0) {
            s = atomicAdd(&sl.scans, 1ull);
            st = *reinterpret_cast<volatile int *>(&sl.status);
        }
        s = __shfl_sync(0xffffffffu, s, 0);
        st = __shfl_sync(0xffffffffu, st, 0);
        bool give_up = st != 0 || s >= budget;
        if (give_up && st == 0 && lane == 0) atomicCAS(&sl.status, 0, (int)LA_ERR_ITER_LIMIT);
        ScanResult<V> r{0, 0, 0, 0};
        if (!give_up && LISTS) {
            bool full = false;
            const SharedKeyPrices<WIDE> prices{keys};
            const ListAhead none{-1, 0ull, {}};
            // two interleaved insertion chains in a full scan (measured 27 % faster than one
            // on 304 n = 4096 instances; four were no better)
            r = vec ? scan_for_bid<WIDE, true, true, 2>(Ci, row, n, cmin, np1, prices, lane, Li, R, full, none)
                    : scan_for_bid<WIDE, false, true, 1>(Ci, row, n, cmin, np1, prices, lane, Li, R, full, none);
            if (full && lane == 0) atomicAdd(&sl.full, 1ull);
        } else if (!give_up) {
            if (lane == 0) atomicAdd(&sl.full, 1ull);
            const int32_t *crow = Ci + (size_t)row * n;
            Lane2<V> t;
            lane2_init(t);
            bool staged = false;
            int d = 0;
            if (STAGE && sok) {
                // the row widened to 16-byte boundaries, if that stays inside the instance
                const uintptr_t a0 = reinterpret_cast<uintptr_t>(crow), a1 = a0 + 4ull * (unsigned)n;
                const uintptr_t w0 = a0 & ~(uintptr_t)15, w1 = (a1 + 15) & ~(uintptr_t)15;
                const uintptr_t lo = reinterpret_cast<uintptr_t>(Ci), hi = lo + 4ull * (unsigned)n * (unsigned)n;
                if (w0 >= lo && w1 <= hi) {
                    __syncwarp();   // every lane is done with the previous row in the buffer
                    if (lane == 0) {
                        fence_proxy_async();
                        bulk_row(sbuf, reinterpret_cast<const void *>(w0), (unsigned)(w1 - w0), sbar);
                    }
                    const bool ok = __all_sync(0xffffffffu, mbar_wait(sbar, spar));
                    spar ^= 1u;
                    if (ok) {
                        staged = true;
                        d = (int)((a0 - w0) >> 2);
                    } else {   // the copy never completed: stop staging on this warp, report it
                        sok = false;
                        if (lane == 0) atomicCAS(&sl.status, 0, (int)LA_ERR_INTERNAL);
                    }
                }
            }
            if (STAGE && staged) {
                const volatile int *rb = sbuf + d;
                if (d == 0 && (n & 3) == 0) {
                    const int4 *r4 = reinterpret_cast<const int4 *>(sbuf);
                    const int nv = n >> 2;
#pragma unroll 2
                    for (int j = lane; j < nv; j += 32) {
                        const int4 c = r4[j];
                        const int y = j << 2;
                        lane2_push<V>(t, bval<WIDE, K32, V>(c.x, y, cmin, np1, k2, vkey), y);
                        lane2_push<V>(t, bval<WIDE, K32, V>(c.y, y + 1, cmin, np1, k2, vkey), y + 1);
                        lane2_push<V>(t, bval<WIDE, K32, V>(c.z, y + 2, cmin, np1, k2, vkey), y + 2);
                        lane2_push<V>(t, bval<WIDE, K32, V>(c.w, y + 3, cmin, np1, k2, vkey), y + 3);
                    }
                } else {
#pragma unroll 4
                    for (int y = lane; y < n; y += 32)
                        lane2_push<V>(t, bval<WIDE, K32, V>(rb[y], y, cmin, np1, k2, vkey), y);
                }
                const V c1 = t.w1 >= 0 ? (V)(uint32_t)(rb[t.w1] - cmin) * np1 : (V)0;
                r = ScanResult<V>{t.b1, t.b2, c1, t.w1 < 0 ? INT_MAX : t.w1};
                warp_merge(r);
            } else {
            prefetch_row_l2(crow, n, lane);
            if (vec) {
                const int4 *r4 = reinterpret_cast<const int4 *>(crow);
                const int nv = n >> 2;
#pragma unroll 2
                for (int j = lane; j < nv; j += 32) {
                    const int4 c = ld_row4(r4 + j);
                    const int y = j << 2;
                    lane2_push<V>(t, bval<WIDE, K32, V>(c.x, y, cmin, np1, k2, vkey), y);
                    lane2_push<V>(t, bval<WIDE, K32, V>(c.y, y + 1, cmin, np1, k2, vkey), y + 1);
                    lane2_push<V>(t, bval<WIDE, K32, V>(c.z, y + 2, cmin, np1, k2, vkey), y + 2);
                    lane2_push<V>(t, bval<WIDE, K32, V>(c.w, y + 3, cmin, np1, k2, vkey), y + 3);
                }
            } else {
#pragma unroll 4
                for (int y = lane; y < n; y += 32) {
                    const int c = ld_row1(crow + y);
                    lane2_push<V>(t, bval<WIDE, K32, V>(c, y, cmin, np1, k2, vkey), y);
                }
            }
            const V c1 = t.w1 >= 0 ? (V)(uint32_t)(ld_row1(crow + t.w1) - cmin) * np1 : (V)0;
            r = ScanResult<V>{t.b1, t.b2, c1, t.w1 < 0 ? INT_MAX : t.w1};
            warp_merge(r);
            }
        }
        const unsigned long long nq = give_up ? 0ull : (unsigned long long)(r.b1 - r.c1) + (r.b2 - r.b1) + eps;
        if (!give_up && (r.w >= n || nq > qlim)) {
            if (lane == 0) atomicCAS(&sl.status, 0, (int)(r.w >= n ? LA_ERR_INTERNAL : LA_ERR_OVERFLOW));
            give_up = true;
        }
        if (give_up) {
            // The instance has failed: its rows are given up one by one, so
            // the phase still ends (and the slot is released) once every row
            // is matched or given up.
            int left = 1;
            if (lane == 0) left = atomicSub(&sl.unmatched, 1) - 1;
            left = __shfl_sync(0xffffffffu, left, 0);
            return left == 0;
        }
        const unsigned long long nk = bkey_pack(K32, nq, (uint32_t)row);
        unsigned long long old = 0;
        int left = 1;
        if (lane == 0) {
            old = atomicMin(keys + r.w, nk);
            if (old > nk && bkey_mate(K32, old) == bkey_none(K32)) {
                __threadfence_block();   // the commit is visible before the count can reach 0
                left = atomicSub(&sl.unmatched, 1) - 1;
            }
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        left = __shfl_sync(0xffffffffu, left, 0);
        if (old > nk) {
            ++wins;
            const uint32_t m = bkey_mate(K32, old);
            if (m == bkey_none(K32)) return left == 0;
            ++displaced;
            row = (int)m;
        }
        // else: a lower price got there first; rescan this row
    }
}

// After a slot's last row was matched (one warp; no other warp can touch the
// slot: none of its rows is free and every claim fails): the next phase's
// refine initialisation (Algorithm 5.2: keep prices shifted so that min q =
// 0, clear every mate, all rows free), or, after the eps = 1 phase, the
// instance's outputs and the next instance.
__device__ void end_phase(const BatchArgs &a, Slot &sl, unsigned long long *keys, int lane,
                          unsigned long long &phases_run) {
    volatile Slot &v = sl;
    __threadfence_block();
    ++phases_run;
    const int n = v.n;
    const int st = v.status;
    if (st == 0 && v.phase + 1 < v.nph) {
        unsigned long long m = ~0ull;
        const bool k32 = v.k32 != 0;
        for (int y = lane; y < n; y += 32) m = min(m, bkey_q(k32, keys[y]));
        m = warp_min(m);
        for (int y = lane; y < n; y += 32) keys[y] = bkey_pack(k32, bkey_q(k32, keys[y]) - m, bkey_none(k32));
        if (lane == 0) {
            v.rebase = v.rebase + m;
            v.eps = max(1ull, v.eps / (unsigned long long)v.alpha);
            v.phase = v.phase + 1;
            v.unmatched = n;
        }
        __syncwarp();
        __threadfence_block();
        if (lane == 0) atomicExch(&sl.claim, (unsigned long long)n << 32);
        __syncwarp();
        return;
    }
    const int i = v.inst;
    const int32_t *Ci = a.C + v.off;
    const long long mo = v.moff;
    int fst = st;
    long long sum = 0;
    if (fst == 0) {
        bool bad = false;
        for (int y = lane; y < n; y += 32) {
            const uint32_t mm = bkey_mate(v.k32 != 0, keys[y]);
            if (mm >= (uint32_t)n) {
                bad = true;
                continue;
            }
            if (a.match_out) a.match_out[mo + mm] = y;
            if (a.prices_out) a.prices_out[mo + y] = -(long long)bkey_q(v.k32 != 0, keys[y]);
            sum += Ci[(size_t)mm * n + y];
        }
        if (__any_sync(0xffffffffu, bad)) fst = LA_ERR_INTERNAL;
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
        const unsigned long long sc = v.scans, fu = v.full;
        if (a.cost_out) a.cost_out[i] = fst == 0 ? sum : 0;
        if (a.inst_status) a.inst_status[i] = fst;
        atomicAdd(&a.ctrl->scans, sc);
        atomicAdd(&a.ctrl->full_scans, fu);
        atomicAdd(&a.ctrl->scan_bytes, fu * 4ull * (unsigned long long)n +
                                           (sc > fu ? sc - fu : 0ull) * (unsigned long long)(8 * kListLen + 8));
        if (fst) {
            atomicAdd(&a.ctrl->failed, 1);
            atomicCAS(&a.ctrl->status, 0, fst);
        }
    }
    __syncwarp();
    load_next(a, sl, keys, lane);
}

// The batched solve: a persistent grid; each CTA keeps up to S instances
// resident in shared memory (one slot each: column keys and state), and
// every warp takes free rows from any slot. A phase of an instance ends when
// its last row is matched, with no CTA barrier, so warps never wait for
// another instance's displacement chains.
// Without lists the kernel keeps 64 registers (72 below 256 threads) for two
// or more CTAs per SM; with lists, the list scan's insertion network gets
// the registers of one CTA per SM.
template <int BLOCK, bool LISTS, bool STAGE>
__global__ void __launch_bounds__(BLOCK, LISTS ? 1 : (BLOCK >= 256 ? 1024 / BLOCK : 7 * 128 / BLOCK))
k_batch_solve(BatchArgs a, int S) {
    static_assert(!(LISTS && STAGE), "row staging is for the list-free kernel");
    extern __shared__ __align__(16) unsigned long long skey[];
    __shared__ Slot s_slot[kMaxSlots];
    constexpr int kWarps = BLOCK / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long wins = 0, displaced = 0, phases_run = 0;
    // with STAGE: after the keys, one row buffer per warp, then one mbarrier per warp
    int *sbuf = nullptr;
    unsigned long long *sbar = nullptr;
    unsigned spar = 0;
    bool sok = true;
    if (STAGE) {
        int *rows = reinterpret_cast<int *>(skey + stage_key_words(S, a.max_n));
        sbuf = rows + (size_t)warp * stage_stride(a.max_n);
        sbar = reinterpret_cast<unsigned long long *>(rows + (size_t)kWarps * stage_stride(a.max_n)) + warp;
        if (lane == 0) {
            mbar_init(sbar);
            fence_mbar_init();
        }
        __syncwarp();
    }
    for (int s = warp; s < S; s += kWarps) load_next(a, s_slot[s], skey + (size_t)s * a.max_n, lane);
    __syncthreads();
    int s0 = warp % S;
    unsigned long long t_idle = 0, p_idle = 0;
    for (;;) {
        int row = -1, sl = -1;
        bool live = false;
        unsigned long long progress = 0;
        if (lane == 0) {
            for (int k = 0; k < S; ++k) {
                const int s = s0 + k < S ? s0 + k : s0 + k - S;
                volatile Slot &t = s_slot[s];
                if (t.inst < 0) continue;
                live = true;
                progress += t.scans + (unsigned long long)t.inst;
                const unsigned long long w = t.claim;
                if ((uint32_t)w >= (uint32_t)(w >> 32)) continue;
                const unsigned long long old = atomicAdd(&s_slot[s].claim, 1ull);
                if ((uint32_t)old < (uint32_t)(old >> 32)) {
                    row = (int)(uint32_t)old;
                    sl = s;
                    break;
                }
            }
        }
        row = __shfl_sync(0xffffffffu, row, 0);
        sl = __shfl_sync(0xffffffffu, sl, 0);
        live = __shfl_sync(0xffffffffu, (int)live, 0) != 0;
        if (row < 0) {
            if (!live) break;
            // Nothing to claim: the other warps are running this CTA's
            // chains. A CTA that makes no progress at all for 10 s has
            // broken its own bookkeeping: stop with an error, never spin.
            int stop = 0;
            if (lane == 0) {
                const unsigned long long now = global_timer_ns();
                if (t_idle == 0 || progress != p_idle) {
                    t_idle = now;
                    p_idle = progress;
                } else if (now - t_idle > 10000000000ull) {
                    atomicCAS(&a.ctrl->status, 0, (int)LA_ERR_INTERNAL);
                    stop = 1;
                }
                __nanosleep(256);
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            continue;
        }
        t_idle = 0;
        __threadfence_block();
        Slot &t = s_slot[sl];
        volatile Slot &v = t;
        unsigned long long *keys = skey + (size_t)sl * a.max_n;
        const int n = v.n;
        RowLists Li{nullptr, nullptr, nullptr};
        if (LISTS) {
            const long long mo = v.moff;
            Li = RowLists{a.lists.cols + mo * kListLen, a.lists.costs + mo * kListLen, a.lists.theta + mo};
        }
        const unsigned long long R = v.rebase;
        const bool done = v.wide
            ? run_chain<true, LISTS, STAGE>(t, keys, a.C + v.off, row, n, v.cmin, v.eps, v.qlim, v.budget,
                                            v.vec != 0, lane, wins, displaced, Li, R, sbuf, sbar, spar, sok)
            : run_chain<false, LISTS, STAGE>(t, keys, a.C + v.off, row, n, v.cmin, v.eps, v.qlim, v.budget,
                                             v.vec != 0, lane, wins, displaced, Li, R, sbuf, sbar, spar, sok);
        if (done) end_phase(a, t, keys, lane, phases_run);
        s0 = sl;
    }
    if (STAGE && !sok) mbar_wait(sbar, spar ^ 1u);   // a copy that timed out: wait once more before exiting
    if (lane == 0) {
        atomicAdd(&a.ctrl->wins, wins);
        atomicAdd(&a.ctrl->displaced, displaced);
        atomicAdd(&a.ctrl->phases, phases_run);
    }
}

// ---------------------------------------------------------------- host side

struct GraphKey {
    const void *cost, *offsets, *ns, *match, *costout, *status, *prices;
    int B, block, max_n, slots, lists;
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
    int2 *cminmax = nullptr;
    BatchCtrl *ctrl = nullptr;
    BatchCtrl *h_ctrl = nullptr;
    int num_sms = 0;
    size_t list_rows = 0;   // rows the candidate lists have room for
    RowLists lists{nullptr, nullptr, nullptr};
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

// Candidate lists for `rows` rows (B * max_n bounds the rows of a batch).
la_status ensure_lists(BatchWorkspace &w, size_t rows) {
    if (w.list_rows >= rows) return LA_OK;
    drop_graph(w);
    cudaFree(w.lists.cols);
    cudaFree(w.lists.costs);
    cudaFree(w.lists.theta);
    w.lists = RowLists{nullptr, nullptr, nullptr};
    w.list_rows = 0;
    if (cudaMalloc(&w.lists.cols, sizeof(int) * kListLen * rows) != cudaSuccess ||
        cudaMalloc(&w.lists.costs, sizeof(int) * kListLen * rows) != cudaSuccess ||
        cudaMalloc(&w.lists.theta, sizeof(unsigned long long) * rows) != cudaSuccess) {
        cudaFree(w.lists.cols);
        cudaFree(w.lists.costs);
        cudaFree(w.lists.theta);
        w.lists = RowLists{nullptr, nullptr, nullptr};
        return LA_ERR_NOMEM;
    }
    w.list_rows = rows;
    return LA_OK;
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
        cudaFree(w.cminmax);
        w.cminmax = nullptr;
        w.moff = nullptr;
        w.order = nullptr;
        w.hist = nullptr;
        w.status = nullptr;
        const int64_t cap = std::max<int64_t>(std::max(B, w.capB), 1024);
        const int mcap = std::max(max_n, w.max_n_cap);
        if (cudaMalloc(&w.moff, sizeof(long long) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.order, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.status, sizeof(int) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.cminmax, sizeof(int2) * cap) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.hist, sizeof(int) * (mcap + 2)) != cudaSuccess) return LA_ERR_NOMEM;
        w.capB = cap;
        w.max_n_cap = mcap;
    }
    return LA_OK;
}

// Persistent grid size on the current device (the shared-memory attribute is
// per device, so it is set on every call; both are host calls, no GPU work).
template <int BLOCK, bool LISTS, bool STAGE>
int solve_grid(int num_sms, size_t smem) {
    // Always set: the kernel's static shared memory (the slot records) and
    // `smem` together must fit, and 48 KB is the limit without it.
    cudaFuncSetAttribute(k_batch_solve<BLOCK, LISTS, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int o = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_batch_solve<BLOCK, LISTS, STAGE>, BLOCK, smem);
    return num_sms * std::max(1, o);
}

template <bool LISTS, bool STAGE>
int solve_grid_for(int block, int num_sms, size_t smem) {
    switch (block) {
    case 64: return solve_grid<64, LISTS, STAGE>(num_sms, smem);
    case 128: return solve_grid<128, LISTS, STAGE>(num_sms, smem);
    case 256: return solve_grid<256, LISTS, STAGE>(num_sms, smem);
    case 512: return solve_grid<512, LISTS, STAGE>(num_sms, smem);
    default: return solve_grid<1024, LISTS, STAGE>(num_sms, smem);
    }
}

template <bool LISTS, bool STAGE>
void launch_solve(cudaStream_t s, int block, int grid, size_t smem, int slots, const BatchArgs &args) {
    switch (block) {
    case 64: k_batch_solve<64, LISTS, STAGE><<<grid, 64, smem, s>>>(args, slots); break;
    case 128: k_batch_solve<128, LISTS, STAGE><<<grid, 128, smem, s>>>(args, slots); break;
    case 256: k_batch_solve<256, LISTS, STAGE><<<grid, 256, smem, s>>>(args, slots); break;
    case 512: k_batch_solve<512, LISTS, STAGE><<<grid, 512, smem, s>>>(args, slots); break;
    default: k_batch_solve<1024, LISTS, STAGE><<<grid, 1024, smem, s>>>(args, slots); break;
    }
}

cudaError_t enqueue(cudaStream_t s, int block, int grid, size_t smem, int slots, bool stage, const BatchArgs &args,
                    int *hist, int num_sms) {
    cudaError_t e = cudaMemsetAsync(args.ctrl, 0, sizeof(BatchCtrl), s);
    if (e != cudaSuccess) return e;
    k_batch_prep<<<1, kPrepThreads, 0, s>>>(args.ns, args.B, args.max_n, const_cast<long long *>(args.moff),
                                            const_cast<int *>(args.order), hist, args.ctrl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int mm_grid = std::max(1, std::min(args.B, 8 * num_sms));
    k_batch_minmax<<<mm_grid, 256, 0, s>>>(args.C, args.offsets, args.ns, args.B, args.max_n,
                                           const_cast<int2 *>(args.cminmax));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (args.lists.cols) launch_solve<true, false>(s, block, grid, smem, slots, args);
    else if (stage) launch_solve<false, true>(s, block, grid, smem, slots, args);
    else launch_solve<false, false>(s, block, grid, smem, slots, args);
    return cudaGetLastError();
}

}  // namespace

#define LA_BCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

static la_status batched_locked(const int32_t *cost, const int64_t *offsets, const int32_t *ns, int32_t B,
                                const la_batch_options *opt, cudaStream_t s, int32_t *match_out,
                                int64_t *cost_out, int32_t *status_out, la_batch_stats *st) {
    const int block = (opt && opt->block_threads) ? opt->block_threads : 512;
    const int max_n = (opt && opt->max_n) ? opt->max_n : LA_BATCH_MAX_N;
    const bool graph = !(opt && opt->no_graph);
    int64_t *prices = opt ? opt->prices_out : nullptr;
    if (block != 64 && block != 128 && block != 256 && block != 512 && block != 1024) return LA_ERR_INVALID;
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
    // instances resident per CTA, bounded by the shared memory their keys take
    int slots = (opt && opt->slots > 0) ? opt->slots : kDefaultSlots;
    slots = std::min(slots, kMaxSlots);
    slots = std::max(1, std::min(slots, (int)(kSlotSmemBudget / (sizeof(unsigned long long) * (size_t)max_n))));
    size_t smem = sizeof(unsigned long long) * (size_t)max_n * slots;
    // Candidate lists: asked for (lists > 0), or by default when instances may
    // be large (max_n >= kAutoListsN) and lists for B * max_n rows fit in
    // kAutoListsBytes.
    const int lists_opt = opt ? opt->lists : 0;
    const size_t list_row_bytes = sizeof(int) * 2 * kListLen + sizeof(unsigned long long);
    const size_t rows = (size_t)B * (size_t)max_n;
    const bool use_lists = lists_opt > 0 ||
                           (lists_opt == 0 && max_n >= kAutoListsN && rows * list_row_bytes <= kAutoListsBytes);
    if (use_lists)
        if (la_status e = ensure_lists(w, rows)) return e;
    // Row staging (list-free kernel) when the warps' row buffers fit beside the keys.
    const bool stage = kStageRows && !use_lists && stage_smem(slots, max_n, block / 32) <= kStageSmemBudget;
    if (stage) smem = stage_smem(slots, max_n, block / 32);
    const int grid_all = use_lists ? solve_grid_for<true, false>(block, w.num_sms, smem)
                                   : (stage ? solve_grid_for<false, true>(block, w.num_sms, smem)
                                            : solve_grid_for<false, false>(block, w.num_sms, smem));
    int grid = grid_all;
    grid = std::max(1, std::min(grid, (int)((B + slots - 1) / slots)));
    BatchArgs args;
    args.C = cost;
    args.offsets = reinterpret_cast<const long long *>(offsets);
    args.ns = ns;
    args.order = w.order;
    args.moff = w.moff;
    args.cminmax = w.cminmax;
    args.B = B;
    args.max_n = max_n;
    args.P = P;
    args.match_out = match_out;
    args.cost_out = reinterpret_cast<long long *>(cost_out);
    args.inst_status = status;
    args.ctrl = w.ctrl;
    args.prices_out = reinterpret_cast<long long *>(prices);
    args.lists = use_lists ? w.lists : RowLists{nullptr, nullptr, nullptr};

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
        key.slots = slots;
        key.lists = use_lists ? 1 : 0;
        key.stream = s;
        key.P = P;
        if (!(w.have_key && w.key == key && w.exec)) {
            drop_graph(w);
            cudaStream_t cs = nullptr;
            LA_BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                const cudaError_t le = enqueue(cs, block, grid, smem, slots, stage, args, w.hist, w.num_sms);
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
        LA_BCK(enqueue(s, block, grid, smem, slots, stage, args, w.hist, w.num_sms));
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
        st->full_scans = (int64_t)c.full_scans;
        st->lists = use_lists ? 1 : 0;
        st->wins = (int64_t)c.wins;
        st->displaced = (int64_t)c.displaced;
        st->phases = (int64_t)c.phases;
        st->max_n = c.max_n;
        st->grid = grid;
        st->block_threads = block;
        st->slots = slots;
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
