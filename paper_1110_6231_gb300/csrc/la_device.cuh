// Device-side building blocks of the refine: the packed column key, the
// row scan (best / second-best part-reduced cost) and the warp reduction.
//
// Notation (Sect. 3 and Sect. 5 of the paper): rows x in X, columns y in Y,
// scaled cost c~(x,y) = (n+1) C[x][y]. Column prices p(y) are kept as
// q(y) = -p(y) >= 0 after a per-phase shift (a uniform shift of all prices
// leaves every reduced cost c_p(x,y) = c(x,y) + p(x) - p(y) unchanged).
// The part-reduced cost c'_p(x,y) = c~(x,y) - p(y) then reads
//   v(x,y) = (C[x][y] - min C) * (n+1) + q(y)  >= 0,
// the same value up to the constant (n+1) min C.
#pragma once

#include <cstdint>
#include <climits>

namespace la {

constexpr int kMateBits = 20;
constexpr unsigned long long kMateMask = (1ull << kMateBits) - 1;
constexpr uint32_t kNone = (uint32_t)kMateMask;          // "no mate"
constexpr int kPriceBits = 64 - kMateBits;               // 44
constexpr unsigned long long kQMax = (1ull << kPriceBits) - 1;

// A column's state in one 64-bit word: (kQMax - q) in the high 44 bits and
// the mate row in the low 20. A smaller key means a lower price p(y) = -q,
// and at equal price the lower row index. One atomicMin therefore decides
// both the new price and the new holder of the column (the double push's
// push x -> w and relabel of w commit together).
__host__ __device__ __forceinline__ unsigned long long pack_key(unsigned long long q, uint32_t mate) {
    return ((kQMax - q) << kMateBits) | (unsigned long long)mate;
}
__host__ __device__ __forceinline__ unsigned long long key_q(unsigned long long k) {
    return kQMax - (k >> kMateBits);
}
__host__ __device__ __forceinline__ uint32_t key_mate(unsigned long long k) {
    return (uint32_t)(k & kMateMask);
}

// Solver control block in device memory.
struct Ctrl {
    unsigned long long scans;       // row scans (all phases)
    unsigned long long wins;        // successful double pushes
    unsigned long long displaced;   // wins that displaced a mate
    int next_row;                   // head of this phase's row queue
    int status;                     // la_status of the device side, 0 = ok
    int cmin, cmax;                 // min / max cost
    unsigned long long qmin[2];     // per-phase rebase, double buffered
    unsigned long long qspread;     // max q after the warm-start shift
    long long pmax;                 // max of warm-start prices
    unsigned long long max_chain;   // most scans by one warp in one phase
    unsigned long long phase_start_scans[64];
    unsigned long long rebase_total; // sum of the per-phase shifts of q
    unsigned long long full_scans;   // row scans over all n columns
    unsigned long long list_scans;   // row scans answered by the candidate list
    unsigned long long tail_scans;   // row scans made by the tail kernel
    int free_rows;                   // rows still unmatched in this phase
    int handoff;                     // 1: the refine handed its rows to the tail kernel
    int tail_count;                  // rows the refine handed over
    int tail_phases;                 // phases that used the tail kernel
    unsigned long long ph_full;      // this phase's full scans so far (refine kernel)
    unsigned long long ph_hits;      // this phase's candidate-list scans so far
    // row queue: qmode 0 = rows 0..n-1 by index, 1 = rows qlist[qsel][0..qlen)
    int qmode, qlen, qsel;
    int pu_left;                     // price updates still allowed in this phase
    unsigned long long pu_mark;      // scans at the phase start or the last update
    unsigned long long pu_updates;   // price updates applied (all phases)
    unsigned long long pu_iters;     // relaxation sweeps they took
    unsigned long long pu_tail_ns;   // time in the tail kernel's own updates
    unsigned long long pu_levels;    // sum of their truncation levels
    unsigned long long pu_qmax;      // largest q before an update
    unsigned pu_bar[2];              // grid barrier: arrivals, generation
    int pu_changed[3];               // a label fell in this sweep (triple buffered)
    unsigned pu_last;                // largest label of a free row
    int pu_abort;                    // sweeps did not settle: no update
    int colseen_missing;             // sparse graphs: columns without an arc
    unsigned long long tail_full;    // full row scans made by the tail kernel
    int tail_giveups;                // phases whose tail kernel gave its rows back
    unsigned long long check_violations;   // debug mode: failed phase-end checks
    int checked_phases;                    // debug mode: phases checked
    int phase_now;                         // the running phase, frozen when the status is set
    unsigned long long phase_start_full[64];   // full_scans at each phase start
    unsigned long long phase_start_tail[64];   // tail_scans at each phase start
    unsigned long long fix_rows[64];           // arc fixing after phase k: rows fixed
    unsigned long long fix_arcs[64];           // ... and the arcs those rows keep
    int pend;                                  // sweep: rows queued for the chain launch
    unsigned sweep_done;                       // sweep: blocks finished (last one switches the queue)
    unsigned long long sweep_scans;            // row scans made by the sweep launches
    unsigned long long sweep_full;             // ... of which full row scans
    int team_T;                                // team refine: free rows at the hand-off (0: off)
    int team_go;                               // team refine: the refine handed its rows to it
    int team_next;                             // team refine: next hand-off item to claim
    int team_back;                             // team refine: rows queued for the tail kernel
    unsigned team_done;                        // team refine: CTAs finished (the last sets the queue)
    int team_phases;                           // phases the team refine took over
    unsigned long long team_scans;             // row scans made by the team refine
    unsigned long long team_full;              // ... of which full row scans
};

// Global nanosecond timer (bounds every wait in the kernels).
__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// --- loads ---------------------------------------------------------------

// Cost rows are read once per scan and never written: non-coherent path,
// no L1 allocation (the row will not be reused by this SM soon), default L2
// policy (a matrix that fits in L2 stays there across phases).
__device__ __forceinline__ int4 ld_row4(const int4 *p) {
    int4 r;
    asm("ld.global.nc.L1::no_allocate.v4.s32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ int ld_row1(const int *p) {
    int r;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// Asks L2 for every 128-byte line of an n-int row (one line per 32 ints,
// spread over the warp's lanes), so that the scan's own dependent loads
// wait on L2 rather than on HBM. A hint: nothing is read into registers.
__device__ __forceinline__ void prefetch_row_l2(const int32_t *crow, int n, int lane) {
    for (int b = lane * 32; b < n; b += 32 * 32) asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + b));
    if (lane == 0 && n > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(crow + n - 1));
}

// Prices are written by other SMs during the scan. Reading them at L2
// (.cg) keeps the view at most one in-flight update old; an older price is
// higher (prices only decrease, Lemma 5.2), which can only make a bid lose,
// never break eps-optimality. L1 must not serve stale lines repeatedly.
__device__ __forceinline__ uint4 ld_q4(const uint32_t *p) {
    return __ldcg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ ulonglong2 ld_q2(const unsigned long long *p) {
    return __ldcg(reinterpret_cast<const ulonglong2 *>(p));
}

// --- best / second best ---------------------------------------------------

template <typename V>
struct ScanResult {
    V b1, b2;      // best and second-best value over the row
    V c1;          // scaled cost of the best column
    int w;         // best column
};

// Lane-local top two of a stream of (value, column) pairs.
template <typename V>
struct Lane2 {
    V b1, b2;
    int w1, w2;
};

template <typename V>
__device__ __forceinline__ void lane2_init(Lane2<V> &t) {
    t.b1 = (V)~(V)0;
    t.b2 = (V)~(V)0;
    t.w1 = -1;
    t.w2 = -1;
}

template <typename V>
__device__ __forceinline__ void lane2_push(Lane2<V> &t, V v, int y) {
    const bool better = v < t.b1;       // strict: keeps the earliest column
    const bool second = v < t.b2;
    const V hi = better ? t.b1 : v;
    t.b2 = second ? hi : t.b2;
    t.w2 = better ? t.w1 : (second ? y : t.w2);
    t.w1 = better ? y : t.w1;
    t.b1 = better ? v : t.b1;
}

// Lane-local K smallest of a stream of (value, column) pairs, kept sorted
// (b[0] <= b[1] <= ...). Equal values keep the earlier column first, so
// b[0] / w[0] is the lane's best in the same sense as Lane2. A
// predicated insertion network: every element costs the same, whatever
// the data, so the lanes of a warp never diverge.
template <typename V, int K>
struct LaneK {
    V b[K];
    int w[K];
};

template <typename V, int K>
__device__ __forceinline__ void lanek_init(LaneK<V, K> &t) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        t.b[k] = (V)~(V)0;
        t.w[k] = -1;
    }
}

template <typename V, int K>
__device__ __forceinline__ void lanek_push(LaneK<V, K> &t, V v, int y) {
    bool lt[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lt[k] = v < t.b[k];    // strict: keeps the earlier column first
#pragma unroll
    for (int k = K - 1; k > 0; --k) {
        t.b[k] = lt[k - 1] ? t.b[k - 1] : (lt[k] ? v : t.b[k]);
        t.w[k] = lt[k - 1] ? t.w[k - 1] : (lt[k] ? y : t.w[k]);
    }
    t.b[0] = lt[0] ? v : t.b[0];
    t.w[0] = lt[0] ? y : t.w[0];
}

// Insert (v, y) ordering equal values by column: merges lists that were
// built from interleaved streams, so that the result is the K least pairs in
// (value, column) order, as one stream in column order would have kept.
template <typename V, int K>
__device__ __forceinline__ void lanek_insert(LaneK<V, K> &t, V v, int y) {
    bool lt[K];
#pragma unroll
    for (int k = 0; k < K; ++k) lt[k] = v < t.b[k] || (v == t.b[k] && (unsigned)y < (unsigned)t.w[k]);
#pragma unroll
    for (int k = K - 1; k > 0; --k) {
        t.b[k] = lt[k - 1] ? t.b[k - 1] : (lt[k] ? v : t.b[k]);
        t.w[k] = lt[k - 1] ? t.w[k - 1] : (lt[k] ? y : t.w[k]);
    }
    t.b[0] = lt[0] ? v : t.b[0];
    t.w[0] = lt[0] ? y : t.w[0];
}

__device__ __forceinline__ unsigned lane_id() {
    unsigned l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

// Warp-wide minimum of an unsigned value by the hardware reduction
// (redux.sync, 32-bit): a 64-bit value is reduced on its high word, then on
// its low word over the lanes that hold the least high word. Two or three
// instructions replace a five-round shuffle butterfly, which matters in the
// dependent chain of one warp's bid when no other warp hides the latency.
template <typename V>
__device__ __forceinline__ V warp_min(V v) {
    static_assert(sizeof(V) == 4 || sizeof(V) == 8, "32- or 64-bit unsigned values");
    if constexpr (sizeof(V) == 4) {
        return (V)__reduce_min_sync(0xffffffffu, (unsigned)v);
    } else {
        const unsigned hi = __reduce_min_sync(0xffffffffu, (unsigned)(v >> 32));
        const unsigned lo = __reduce_min_sync(0xffffffffu, (unsigned)(v >> 32) == hi ? (unsigned)v : 0xffffffffu);
        return ((V)hi << 32) | (V)lo;
    }
}

// Warp-wide maximum of a 64-bit unsigned value (high word, then low word).
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    const unsigned hi = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32));
    const unsigned lo = __reduce_max_sync(0xffffffffu, (unsigned)(v >> 32) == hi ? (unsigned)v : 0u);
    return ((unsigned long long)hi << 32) | (unsigned long long)lo;
}

// Merge of the lanes' (b1, w, c1, b2): every lane ends with the row's best
// value, its column (the lowest index among equal minima), that column's
// scaled cost and the second-best value, i.e. the least of all the lanes'
// values once one copy of the best is taken out: the winning lane offers
// its own second best, every other lane its best.
template <typename V>
__device__ __forceinline__ void warp_merge(ScanResult<V> &r) {
    const V m1 = warp_min<V>(r.b1);
    const unsigned w = __reduce_min_sync(0xffffffffu, r.b1 == m1 ? (unsigned)r.w : 0xffffffffu);
    const unsigned own = __ballot_sync(0xffffffffu, r.b1 == m1 && (unsigned)r.w == w);
    const int src = __ffs(own) - 1;
    const V c1 = __shfl_sync(0xffffffffu, r.c1, src);
    const V m2 = warp_min<V>((int)lane_id() == src ? r.b2 : r.b1);
    r.b1 = m1;
    r.b2 = m2;
    r.c1 = c1;
    r.w = (int)w;
}

}  // namespace la
