// Exact candidate lists and the row scans that use them, shared by the
// single-instance refine (la_solve.cu) and the batched solver
// (la_batched.cu). Notation as in la_device.cuh.
#pragma once

#include <cstdint>
#include <climits>
#include <type_traits>

#include "la_device.cuh"

namespace la {

// Candidate lists (exact lazy scans). A full scan leaves, for row x, the
// kListK lane-local best columns of each of the 32 lanes (kListLen entries:
// column and raw cost C[x][y]) and the bound
//   theta = min over lanes of the lane's kListK-th best value.
// Every column outside the list was beaten kListK times within its lane, so
// its value was >= theta then; prices only fall (Lemma 5.2), so its value
// stays >= theta, up to the uniform per-phase shift R that is tracked in the
// control block. A later scan of x may therefore gather only the listed
// prices: when the list's second best is <= theta, its best and second best
// are those of the whole row, and the bid is the same as a full scan's.
// A longer list raises theta (the kListK-th order statistic of each lane
// instead of the second), so it stays exact through more price changes.
constexpr int kListK = 4;                 // entries per lane (int4 groups of columns and of costs)
constexpr int kListLen = 32 * kListK;     // entries per row
static_assert(kListK % 4 == 0, "a lane's list entries are loaded and stored as int4 groups");

struct RowLists {
    int *cols;                  // [n][32][kListK] column, -1 = empty
    int *costs;                 // [n][32][kListK] raw cost C[x][y]
    unsigned long long *theta;  // [n]: 0 = no list, ~0 = unbounded, else theta + R + 1
};

// One lane's list entries of row x (two 128-bit loads). Lists are written
// by whichever SM scans the row, so a kernel that runs on many SMs reads
// them at L2 (.cg). A kernel whose every warp runs on one SM (ONE_SM) may
// cache them in L1 (.ca): the SM's own stores keep its L1 coherent, and L1
// holds nothing from earlier kernels, so the rows that its chains keep
// revisiting are read at L1 latency.
struct LaneList {
    int y[kListK];
    int c[kListK];
};
template <bool ONE_SM>
__device__ __forceinline__ int4 ld_list4(const int *p) {
    return ONE_SM ? __ldca(reinterpret_cast<const int4 *>(p)) : __ldcg(reinterpret_cast<const int4 *>(p));
}
template <bool ONE_SM = false>
__device__ __forceinline__ LaneList load_lane_list(const RowLists &L, int row, int lane) {
    const size_t base = (size_t)row * kListLen + kListK * lane;
    LaneList e;
#pragma unroll
    for (int g = 0; g < kListK / 4; ++g) {
        const int4 yy = ld_list4<ONE_SM>(L.cols + base + 4 * g);
        const int4 cc = ld_list4<ONE_SM>(L.costs + base + 4 * g);
        e.y[4 * g] = yy.x; e.y[4 * g + 1] = yy.y; e.y[4 * g + 2] = yy.z; e.y[4 * g + 3] = yy.w;
        e.c[4 * g] = cc.x; e.c[4 * g + 1] = cc.y; e.c[4 * g + 2] = cc.z; e.c[4 * g + 3] = cc.w;
    }
    return e;
}

// A row's list loaded ahead of its scan (row = -1: nothing loaded).
struct ListAhead {
    int row;
    unsigned long long theta;
    LaneList e;
};
template <bool ONE_SM>
__device__ __forceinline__ void load_ahead(ListAhead &a, const RowLists &L, int row, int lane) {
    a.row = row;
    a.theta = ONE_SM ? __ldca(L.theta + row) : __ldcg(L.theta + row);
    a.e = load_lane_list<ONE_SM>(L, row, lane);
}

template <bool WIDE>
__device__ __forceinline__ auto load_q(const void *qmv, int y) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    if (WIDE) return (V)__ldcg(static_cast<const unsigned long long *>(qmv) + y);
    else return (V)__ldcg(static_cast<const uint32_t *>(qmv) + y);
}

// Where a scan reads the column prices q(y) from.
// The global mirror of the refine kernel (read at L2, see ld_q4).
template <bool WIDE>
struct MirrorPrices {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    const void *qm;
    __device__ __forceinline__ V q(int y) const { return load_q<WIDE>(qm, y); }
    __device__ __forceinline__ void q4(int y, V &a, V &b, V &c, V &d) const {
        if (WIDE) {
            const unsigned long long *p = static_cast<const unsigned long long *>(qm) + y;
            const ulonglong2 u = ld_q2(p), w = ld_q2(p + 2);
            a = (V)u.x; b = (V)u.y; c = (V)w.x; d = (V)w.y;
        } else {
            const uint4 u = ld_q4(static_cast<const uint32_t *>(qm) + y);
            a = (V)u.x; b = (V)u.y; c = (V)u.z; d = (V)u.w;
        }
    }
};
// The column keys held in shared memory by the tail kernel.
template <bool WIDE>
struct SharedKeyPrices {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    const volatile unsigned long long *k;
    __device__ __forceinline__ V q(int y) const { return (V)key_q(k[y]); }
    __device__ __forceinline__ void q4(int y, V &a, V &b, V &c, V &d) const {
        a = (V)key_q(k[y]); b = (V)key_q(k[y + 1]); c = (V)key_q(k[y + 2]); d = (V)key_q(k[y + 3]);
    }
};

// Full scan of row x: v(x,y) = (C[x][y] - cmin)(n+1) + q(y) for every y.
// Writes x's candidate list when lists are on.
//
// NCH independent insertion chains per lane take interleaved columns of each
// int4 group (chain c the components c, c + NCH, ...) and are merged at the
// end in (value, column) order, which gives the same lists as one chain. In
// the one-CTA tail kernel, where a warp often scans alone on its SM, four
// chains (two on 32-bit values) measured faster; the grid refine and the
// batched kernel use one, which needs fewer registers.
template <bool WIDE, bool VEC, int NCH, class P>
__device__ __forceinline__ auto full_scan(const int32_t *__restrict__ crow, int row, int n, int cmin,
                                          uint32_t np1, const P &prices, int lane,
                                          const RowLists &L, unsigned long long R) {
    static_assert(NCH == 1 || NCH == 2 || NCH == 4, "one, two or four chains");
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    LaneK<V, kListK> ch[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) lanek_init(ch[c]);
    LaneK<V, kListK> &t = ch[0];
    int cnt;
    if (VEC) {
        const int4 *r4 = reinterpret_cast<const int4 *>(crow);
        const int nv = n >> 2;
        cnt = lane < nv ? 4 * ((nv - lane + 31) >> 5) : 0;
#pragma unroll 8
        for (int j = lane; j < nv; j += 32) {
            const int4 c = ld_row4(r4 + j);
            const int y = j << 2;
            V qa, qb, qc, qd;
            prices.q4(y, qa, qb, qc, qd);
            lanek_push<V, kListK>(ch[0], (V)(uint32_t)(c.x - cmin) * np1 + qa, y);
            lanek_push<V, kListK>(ch[1 % NCH], (V)(uint32_t)(c.y - cmin) * np1 + qb, y + 1);
            lanek_push<V, kListK>(ch[2 % NCH], (V)(uint32_t)(c.z - cmin) * np1 + qc, y + 2);
            lanek_push<V, kListK>(ch[3 % NCH], (V)(uint32_t)(c.w - cmin) * np1 + qd, y + 3);
        }
#pragma unroll
        for (int c = 1; c < NCH; ++c)
#pragma unroll
            for (int k = 0; k < kListK; ++k)   // an empty entry (~0, -1) inserts nothing
                lanek_insert<V, kListK>(t, ch[c].b[k], ch[c].w[k]);
    } else {
        cnt = lane < n ? ((n - lane + 31) >> 5) : 0;
        for (int y = lane; y < n; y += 32) {
            const int c = ld_row1(crow + y);
            lanek_push<V, kListK>(t, (V)(uint32_t)(c - cmin) * np1 + prices.q(y), y);
        }
    }
    // raw costs of the lane's listed columns (the row was just read: L2 hits)
    int craw[kListK];
#pragma unroll
    for (int k = 0; k < kListK; ++k)
        craw[k] = (t.w[k] >= 0 && (k == 0 || L.cols)) ? ld_row1(crow + t.w[k]) : 0;
    const V c1 = t.w[0] >= 0 ? (V)(uint32_t)(craw[0] - cmin) * np1 : (V)0;
    if (L.cols) {
        const size_t base = (size_t)row * kListLen + kListK * lane;
#pragma unroll
        for (int g = 0; g < kListK / 4; ++g) {
            reinterpret_cast<int4 *>(L.cols + base)[g] =
                make_int4(t.w[4 * g], t.w[4 * g + 1], t.w[4 * g + 2], t.w[4 * g + 3]);
            reinterpret_cast<int4 *>(L.costs + base)[g] =
                make_int4(craw[4 * g], craw[4 * g + 1], craw[4 * g + 2], craw[4 * g + 3]);
        }
        const V th = warp_min<V>(cnt > kListK ? t.b[kListK - 1] : (V)~(V)0);
        if (lane == 0)
            L.theta[row] = th == (V)~(V)0 ? ~0ull : (unsigned long long)th + R + 1;
        __threadfence();   // the list is complete before this row can change hands
    }
    ScanResult<V> r{t.b[0], t.b[1], c1, t.w[0] < 0 ? INT_MAX : t.w[0]};
    warp_merge(r);
    return r;
}

// Full scan of row x for the best and second best only, without rebuilding
// its candidate list: for stretches where the lists keep failing (a large
// eps moves prices past theta after a bid or two), the top-4 insertion
// network and the list write would be wasted. The list is left as it was
// (its bound stays a valid lower bound: prices only fall). scan_top2_range
// ranks columns [y0, y1) only (the team refine splits a row among warps).
template <bool WIDE, bool VEC, class P>
__device__ __forceinline__ auto scan_top2_range(const int32_t *__restrict__ crow, int y0, int y1, int cmin,
                                                uint32_t np1, const P &prices, int lane) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    Lane2<V> t;
    lane2_init(t);
    if (VEC) {   // y0 and y1 are multiples of 4
        const int4 *r4 = reinterpret_cast<const int4 *>(crow);
        const int j1 = y1 >> 2;
#pragma unroll 8
        for (int j = (y0 >> 2) + lane; j < j1; j += 32) {
            const int4 c = ld_row4(r4 + j);
            const int y = j << 2;
            V qa, qb, qc, qd;
            prices.q4(y, qa, qb, qc, qd);
            lane2_push<V>(t, (V)(uint32_t)(c.x - cmin) * np1 + qa, y);
            lane2_push<V>(t, (V)(uint32_t)(c.y - cmin) * np1 + qb, y + 1);
            lane2_push<V>(t, (V)(uint32_t)(c.z - cmin) * np1 + qc, y + 2);
            lane2_push<V>(t, (V)(uint32_t)(c.w - cmin) * np1 + qd, y + 3);
        }
    } else {
        for (int y = y0 + lane; y < y1; y += 32)
            lane2_push<V>(t, (V)(uint32_t)(ld_row1(crow + y) - cmin) * np1 + prices.q(y), y);
    }
    const V c1 = t.w1 >= 0 ? (V)(uint32_t)(ld_row1(crow + t.w1) - cmin) * np1 : (V)0;
    ScanResult<V> r{t.b1, t.b2, c1, t.w1 < 0 ? INT_MAX : t.w1};
    warp_merge(r);
    return r;
}

// The lane's kListK best (value, column) pairs over columns [y0, y1) of a
// row (y0, y1 multiples of 4 when VEC) and how many columns the lane saw:
// one warp's share of a list rebuilt by the team refine, which merges the
// warps' pairs lane by lane.
template <bool WIDE, bool VEC, class P>
__device__ __forceinline__ void scan_topk_range(const int32_t *__restrict__ crow, int y0, int y1, int cmin,
                                                uint32_t np1, const P &prices, int lane,
                                                LaneK<typename std::conditional<WIDE, unsigned long long, uint32_t>::type,
                                                      kListK> &t,
                                                int &cnt) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    lanek_init(t);
    if (VEC) {
        const int4 *r4 = reinterpret_cast<const int4 *>(crow);
        const int j0 = y0 >> 2, j1 = y1 >> 2;
        cnt = j0 + lane < j1 ? 4 * ((j1 - j0 - lane + 31) >> 5) : 0;
#pragma unroll 4
        for (int j = j0 + lane; j < j1; j += 32) {
            const int4 c = ld_row4(r4 + j);
            const int y = j << 2;
            V qa, qb, qc, qd;
            prices.q4(y, qa, qb, qc, qd);
            lanek_push<V, kListK>(t, (V)(uint32_t)(c.x - cmin) * np1 + qa, y);
            lanek_push<V, kListK>(t, (V)(uint32_t)(c.y - cmin) * np1 + qb, y + 1);
            lanek_push<V, kListK>(t, (V)(uint32_t)(c.z - cmin) * np1 + qc, y + 2);
            lanek_push<V, kListK>(t, (V)(uint32_t)(c.w - cmin) * np1 + qd, y + 3);
        }
    } else {
        cnt = y0 + lane < y1 ? ((y1 - y0 - lane + 31) >> 5) : 0;
        for (int y = y0 + lane; y < y1; y += 32)
            lanek_push<V, kListK>(t, (V)(uint32_t)(ld_row1(crow + y) - cmin) * np1 + prices.q(y), y);
    }
}

template <bool WIDE, bool VEC, class P>
__device__ __forceinline__ auto full_scan_top2(const int32_t *__restrict__ crow, int n, int cmin, uint32_t np1,
                                               const P &prices, int lane) {
    return scan_top2_range<WIDE, VEC>(crow, 0, n, cmin, np1, prices, lane);
}

// Short scan of row x over its candidate list (kListK entries per lane).
// The list entries and the row's bound theta are loaded in the same round
// trip, or were loaded ahead (ahead.row == x); the prices are gathered only
// when a list exists (theta != 0).
template <bool WIDE, bool ONE_SM, class P>
__device__ __forceinline__ auto list_scan(int row, int n, int cmin, uint32_t np1, const P &prices, int lane,
                                          const RowLists &L, const ListAhead &ahead,
                                          unsigned long long &theta) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    LaneList e;
    if (ahead.row == row) {   // uniform across the warp
        theta = ahead.theta;
        e = ahead.e;
    } else {
        theta = ONE_SM ? __ldca(L.theta + row) : __ldcg(L.theta + row);
        e = load_lane_list<ONE_SM>(L, row, lane);
    }
    const V inf = (V)~(V)0;
    ScanResult<V> r{inf, inf, 0, INT_MAX};
    if (theta == 0) return r;            // no list for this row yet (uniform across the warp)
    V v[kListK], cs[kListK];
#pragma unroll
    for (int k = 0; k < kListK; ++k) {
        const bool ok = e.y[k] >= 0 && e.y[k] < n;
        cs[k] = (V)(uint32_t)(e.c[k] - cmin) * np1;
        const V q = prices.q(ok ? e.y[k] : 0);
        v[k] = ok ? cs[k] + q : inf;
    }
#pragma unroll
    for (int k = 0; k < kListK; ++k) {
        const bool ok = v[k] != inf;
        // lowest value, then lowest column; the second best is the minimum
        // over the other entries
        const bool better = ok && (v[k] < r.b1 || (v[k] == r.b1 && (unsigned)e.y[k] < (unsigned)r.w));
        const V hi = better ? r.b1 : v[k];
        r.b2 = hi < r.b2 ? hi : r.b2;
        r.c1 = better ? cs[k] : r.c1;
        r.w = better ? e.y[k] : r.w;
        r.b1 = better ? v[k] : r.b1;
    }
    warp_merge(r);
    // A row whose arcs were cut down to one (arc fixing) has no second
    // best: any price drop keeps it eps-optimal, and the bid drops by eps.
    if (r.b2 == inf) r.b2 = r.b1;
    return r;
}

// Best and second best of row x for its next bid: from the candidate list
// when it decides the row (see RowLists), else from a full scan that also
// rebuilds the list. The second best may be the lower bound theta.
template <bool WIDE, bool VEC, bool ONE_SM, int NCH, class P>
__device__ __forceinline__ auto scan_for_bid(const int32_t *__restrict__ C, int row, int n, int cmin,
                                             uint32_t np1, const P &prices, int lane,
                                             const RowLists &L, unsigned long long R, bool &full,
                                             const ListAhead &ahead, bool try_list = true,
                                             bool prefetch = false, bool top2 = false) {
    using V = typename std::conditional<WIDE, unsigned long long, uint32_t>::type;
    ScanResult<V> t;
    bool ok = false;
    if (prefetch && !try_list) prefetch_row_l2(C + (size_t)row * n, n, lane);
    if (L.cols && !try_list && top2) {
        full = true;
        return full_scan_top2<WIDE, VEC>(C + (size_t)row * n, n, cmin, np1, prices, lane);
    }
    if (L.cols && try_list) {
        unsigned long long th = 0;
        t = list_scan<WIDE, ONE_SM>(row, n, cmin, np1, prices, lane, L, ahead, th);
        if (th != 0) {
            // Exact when the list's second best does not exceed theta: every
            // other column is >= theta, so the list holds the row's best and
            // second best. (Bidding with theta as a lower bound of the
            // second best would also keep x eps-optimal, but as a list runs
            // out its price drops shrink towards eps, and at eps = 1 two
            // such rows can trade a column for a very long time.)
            ok = th == ~0ull || (unsigned long long)t.b2 + R + 1 <= th;
        }
    }
    full = !ok;
    if (!ok) {
        if (prefetch && try_list) prefetch_row_l2(C + (size_t)row * n, n, lane);
        t = full_scan<WIDE, VEC, NCH>(C + (size_t)row * n, row, n, cmin, np1, prices, lane, L, R);
    }
    return t;
}

}  // namespace la
