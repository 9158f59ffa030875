/*
 * CPU emulation of the lock-free parallel refine, for the tests: host
 * threads play the GPU's bidding warps, with C11 atomics in place of the
 * device atomics, so that ThreadSanitizer can check the protocol for data
 * races and the result can be checked for exactness. It shares no code with
 * the CUDA path or with the oracle.
 *
 * The protocol (Sect. 5.1-5.3: cost scaling, refine initialisation of
 * Algorithm 5.2, push/relabel of Algorithm 5.4 taken as the Goldberg-Kennedy
 * double push), on costs scaled by n + 1:
 *   - one 64-bit word per column, key = (QMAX - q) << 20 | mate, where
 *     q = -p(y) only grows; a bid is a compare-and-swap loop that lowers the
 *     key (an atomic minimum), so price and holder change together;
 *   - a free row reads the keys it needs without locks, finds its best value
 *     b1 at column w and second best b2 (values c~(x,y) + q(y) relative to
 *     the matrix's minimum cost), and bids q'(w) = q(w) + (b2 - b1) + eps;
 *   - a winning bid that displaced a holder continues with that row; a bid
 *     on a free column ends the chain and counts one matched row; a losing
 *     bid rescans the same row;
 *   - a phase ends when every row is matched (a barrier); the next phase
 *     keeps the prices, shifted so that min q = 0, and frees every row.
 *
 * Candidate lists (optional; the exact form of arc fixing the GPU uses):
 *   - a full scan of row x also keeps, for each of `lanes` column classes
 *     (y mod lanes), the `per_lane` best (value, column) pairs it saw, with
 *     their raw costs, and theta = the least per_lane-th best value over the
 *     classes that saw more than per_lane columns (none: every column is
 *     listed); it records the sum R of the price shifts made so far;
 *   - a later bid by x ranks only its listed columns at their current prices.
 *     Values only grow inside a phase (Lemma 5.2) and fall by the shift at a
 *     phase change, so an unlisted column is still >= theta - (R_now - R).
 *     When the list's second best is within that bound the list holds the
 *     row's best and exact second best; otherwise the row is scanned in full
 *     and the list rebuilt;
 *   - only the thread that holds row x writes its list; the next holder reads
 *     it after the compare-and-swap (or the phase barrier) that passed x on.
 *
 * Price mirror (optional; the single-solve refine's read path): scans read
 * column prices from a separate array instead of the keys. After every
 * commit attempt on column w the bidder raises mirror[w] (an atomic
 * maximum) to the price its compare-and-swap left in the key: its own bid
 * when it won, the key's price when it lost. So the mirror never exceeds
 * the key's price, and a scan that reads a stale (lower) price still bids
 * within eps of every column (prices only grow inside a phase, Lemma 5.2).
 * At a phase change the mirror is rewritten from the shifted keys.
 *
 * Usage: lockfree_emulation <in> <out>
 *   in:  int32 n, int32 alpha, int32 threads, int32 lanes, int32 per_lane
 *        (lanes = 0: no lists), int32 mirror (0: prices read from the keys),
 *        then n*n int32 costs (row-major)
 *   out: int64 cost, int64 phases, int64 bids, n int32 matches, n int64
 *        prices (p = -q, paper sign, units of (n+1) C), int64 list scans,
 *        int64 full scans
 * Exit status 0 on success, 1 on a bad input, 2 on an internal error, 3
 * when a price bound that the GPU's 32-bit path relies on is broken: within
 * a phase every q stays <= S + 2 C~ + 2 eps (S = the largest q after the
 * phase's shift), and after a phase the spread max q - min q is <= C~ + eps.
 * Compiling with -DLIST_MUTANT=1 (the shift ignored) or 2 (theta taken as the
 * largest bound instead of the least) plants a mistake in the list rule, so
 * that the tests can show that they would see one.
 */
#define _POSIX_C_SOURCE 200809L   /* pthread barriers under -std=c11 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#ifndef LIST_MUTANT
#define LIST_MUTANT 0
#endif

#define MATE_BITS 20
#define NONE ((1ull << MATE_BITS) - 1)
#define QMAX ((1ull << 44) - 1)

static int n, alpha, nthreads;
static int32_t *C;
static int32_t cmin;
static _Atomic uint64_t *key;
static _Atomic int next_row;      /* queue of the phase's free rows */
static _Atomic int unmatched;     /* rows not matched yet in this phase */
static _Atomic int64_t bids;
static uint64_t eps;
static pthread_barrier_t bar;
static int phases_total;
static uint64_t eps_first;
/* candidate lists: E = lanes * per_lane entries per row */
static int lanes, per_lane, E;
static int32_t *lcol, *lcost;     /* [n][E], column -1 = empty */
static uint64_t *ltheta, *lrb;    /* bound (UINT64_MAX: all listed), shift sum at build */
static unsigned char *lvalid;
static uint64_t R_total;          /* sum of the per-phase shifts */
static _Atomic int64_t list_scans, full_scans;
static _Atomic uint64_t qpeak;     /* the largest q committed in this phase */
static int use_mirror;
static _Atomic uint64_t *mirror;   /* per column: a price <= the key's */

static uint64_t pack(uint64_t q, uint64_t mate) { return ((QMAX - q) << MATE_BITS) | mate; }
static uint64_t key_q(uint64_t k) { return QMAX - (k >> MATE_BITS); }
static uint64_t key_mate(uint64_t k) { return k & NONE; }

/* the price of column y as a scan reads it */
static uint64_t price(int y) {
    return use_mirror ? atomic_load_explicit(&mirror[y], memory_order_relaxed)
                      : key_q(atomic_load_explicit(&key[y], memory_order_relaxed));
}

typedef struct {
    uint64_t b1, b2, c1;
    int w;
} Bid;

/* Ranks row x's listed columns; returns 0 when the list cannot decide. */
static int list_scan(int x, Bid *r) {
    const uint64_t np1 = (uint64_t)n + 1;
    uint64_t b1 = UINT64_MAX, b2 = UINT64_MAX, c1 = 0;
    int w = -1;
    for (int k = 0; k < E; ++k) {
        const int y = lcol[(size_t)x * E + k];
        if (y < 0) continue;
        const uint64_t cs = (uint64_t)(uint32_t)(lcost[(size_t)x * E + k] - cmin) * np1;
        const uint64_t v = cs + price(y);
        if (v < b1 || (v == b1 && y < w)) {
            b2 = b1;
            b1 = v;
            c1 = cs;
            w = y;
        } else if (v < b2) {
            b2 = v;
        }
    }
    if (n == 1) b2 = b1;
    if (w < 0 || b2 == UINT64_MAX) return 0;
#if LIST_MUTANT == 1
    const uint64_t dR = 0;
#else
    const uint64_t dR = R_total - lrb[x];
#endif
    if (ltheta[x] != UINT64_MAX && b2 + dR > ltheta[x]) return 0;
    atomic_fetch_add_explicit(&list_scans, 1, memory_order_relaxed);
    r->b1 = b1;
    r->b2 = b2;
    r->c1 = c1;
    r->w = w;
    return 1;
}

/* Ranks every column of row x and, with lists on, rebuilds x's list. */
static void full_scan(int x, Bid *r, uint64_t *tv, int *ty, int32_t *tc, int *seen) {
    const uint64_t np1 = (uint64_t)n + 1;
    const int32_t *row = C + (size_t)x * n;
    uint64_t b1 = UINT64_MAX, b2 = UINT64_MAX, c1 = 0;
    int w = -1;
    for (int l = 0; l < lanes; ++l) seen[l] = 0;
    for (int y = 0; y < n; ++y) {
        const uint64_t cs = (uint64_t)(uint32_t)(row[y] - cmin) * np1;
        const uint64_t v = cs + price(y);
        if (v < b1) {           /* strict: the lowest column wins ties */
            b2 = b1;
            b1 = v;
            c1 = cs;
            w = y;
        } else if (v < b2) {
            b2 = v;
        }
        if (E > 0) {            /* the class's best per_lane, in (value, column) order */
            const int l = y % lanes;
            uint64_t *lv = tv + (size_t)l * per_lane;
            int *ly = ty + (size_t)l * per_lane;
            int32_t *lc = tc + (size_t)l * per_lane;
            int m = seen[l] < per_lane ? seen[l] : per_lane;
            ++seen[l];
            if (m == per_lane && v >= lv[per_lane - 1]) continue;   /* y is larger: same value, later column */
            int k = m == per_lane ? per_lane - 1 : m;
            while (k > 0 && lv[k - 1] > v) {
                lv[k] = lv[k - 1];
                ly[k] = ly[k - 1];
                lc[k] = lc[k - 1];
                --k;
            }
            lv[k] = v;
            ly[k] = y;
            lc[k] = row[y];
        }
    }
    if (n == 1) b2 = b1;
    atomic_fetch_add_explicit(&full_scans, 1, memory_order_relaxed);
    if (E > 0) {
        uint64_t theta = UINT64_MAX;
#if LIST_MUTANT == 2
        uint64_t worst = 0;
        int any = 0;
#endif
        for (int l = 0; l < lanes; ++l) {
            const int m = seen[l] < per_lane ? seen[l] : per_lane;
            for (int k = 0; k < per_lane; ++k) {
                lcol[(size_t)x * E + (size_t)l * per_lane + k] = k < m ? ty[(size_t)l * per_lane + k] : -1;
                lcost[(size_t)x * E + (size_t)l * per_lane + k] = k < m ? tc[(size_t)l * per_lane + k] : 0;
            }
            if (seen[l] > per_lane) {
                const uint64_t t = tv[(size_t)l * per_lane + per_lane - 1];
#if LIST_MUTANT == 2
                if (t > worst) worst = t;
                any = 1;
#else
                if (t < theta) theta = t;
#endif
            }
        }
#if LIST_MUTANT == 2
        if (any) theta = worst;
#endif
        ltheta[x] = theta;
        lrb[x] = R_total;
        lvalid[x] = 1;
    }
    r->b1 = b1;
    r->b2 = b2;
    r->c1 = c1;
    r->w = w;
}

/* one displacement chain starting at row x */
static void chain(int x, uint64_t *tv, int *ty, int32_t *tc, int *seen) {
    for (;;) {
        Bid bid;
        if (!(E > 0 && lvalid[x] && list_scan(x, &bid))) full_scan(x, &bid, tv, ty, tc, seen);
        const uint64_t b1 = bid.b1, b2 = bid.b2, c1 = bid.c1;
        const int w = bid.w;
        atomic_fetch_add_explicit(&bids, 1, memory_order_relaxed);
        const uint64_t nq = (b1 - c1) + (b2 - b1) + eps;
        if (nq >= QMAX) exit(2);   /* the price field would overflow */
        const uint64_t nk = pack(nq, (uint64_t)x);
        uint64_t cur = atomic_load_explicit(&key[w], memory_order_relaxed);
        int won = 0;
        while (nk < cur) {
            if (atomic_compare_exchange_weak_explicit(&key[w], &cur, nk, memory_order_acq_rel,
                                                      memory_order_relaxed)) {
                won = 1;
                break;
            }
        }
        if (use_mirror) {     /* raise the mirror to the price the key now holds */
            const uint64_t qnow = won ? nq : key_q(cur);
            uint64_t mq = atomic_load_explicit(&mirror[w], memory_order_relaxed);
            while (qnow > mq && !atomic_compare_exchange_weak_explicit(&mirror[w], &mq, qnow, memory_order_relaxed,
                                                                       memory_order_relaxed)) {
            }
        }
        if (!won) continue;   /* a lower price got there first: rescan x */
        uint64_t pk = atomic_load_explicit(&qpeak, memory_order_relaxed);
        while (nq > pk && !atomic_compare_exchange_weak_explicit(&qpeak, &pk, nq, memory_order_relaxed,
                                                                 memory_order_relaxed)) {
        }
        const uint64_t m = key_mate(cur);
        if (m == NONE) {
            atomic_fetch_sub_explicit(&unmatched, 1, memory_order_acq_rel);
            return;
        }
        x = (int)m;
    }
}

static void *worker(void *arg) {
    const int id = (int)(intptr_t)arg;
    /* this thread's scratch for building a list */
    const size_t e = E > 0 ? (size_t)E : 1;
    uint64_t *tv = malloc(sizeof(uint64_t) * e);
    int *ty = malloc(sizeof(int) * e);
    int32_t *tc = malloc(sizeof(int32_t) * e);
    int *seen = malloc(sizeof(int) * (size_t)(lanes > 0 ? lanes : 1));
    if (!tv || !ty || !tc || !seen) exit(2);
    for (;;) {
        pthread_barrier_wait(&bar);   /* phase start (thread 0 set it up) */
        if (eps == 0) {               /* no more phases */
            free(tv);
            free(ty);
            free(tc);
            free(seen);
            return NULL;
        }
        for (;;) {
            const int x = atomic_fetch_add_explicit(&next_row, 1, memory_order_acq_rel);
            if (x >= n) break;
            chain(x, tv, ty, tc, seen);
        }
        while (atomic_load_explicit(&unmatched, memory_order_acquire) > 0) sched_yield();
        pthread_barrier_wait(&bar);   /* phase end */
        (void)id;
    }
}

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int32_t hdr[6];
    if (fread(hdr, sizeof(int32_t), 6, f) != 6) return 1;
    n = hdr[0];
    alpha = hdr[1];
    nthreads = hdr[2];
    lanes = hdr[3];
    per_lane = hdr[4];
    use_mirror = hdr[5] != 0;
    if (n < 1 || n >= (int)NONE || alpha < 2 || nthreads < 1 || nthreads > 64) return 1;
    if (lanes < 0 || lanes > 64 || (lanes > 0 && (per_lane < 1 || per_lane > 16))) return 1;
    E = lanes * (lanes > 0 ? per_lane : 0);
    C = malloc(sizeof(int32_t) * (size_t)n * n);
    key = malloc(sizeof(*key) * (size_t)n);
    mirror = malloc(sizeof(*mirror) * (size_t)n);
    if (!C || !key || !mirror) return 2;
    if (E > 0) {
        lcol = malloc(sizeof(int32_t) * (size_t)n * E);
        lcost = malloc(sizeof(int32_t) * (size_t)n * E);
        ltheta = malloc(sizeof(uint64_t) * (size_t)n);
        lrb = malloc(sizeof(uint64_t) * (size_t)n);
        lvalid = calloc((size_t)n, 1);
        if (!lcol || !lcost || !ltheta || !lrb || !lvalid) return 2;
    }
    if (fread(C, sizeof(int32_t), (size_t)n * n, f) != (size_t)n * n) return 1;
    fclose(f);
    int32_t cmax = C[0];
    cmin = C[0];
    for (size_t i = 0; i < (size_t)n * n; ++i) {
        if (C[i] < cmin) cmin = C[i];
        if (C[i] > cmax) cmax = C[i];
    }
    const uint64_t Ct = ((uint64_t)n + 1) * (uint64_t)((int64_t)cmax - cmin);
    if (Ct >= (1ull << 40)) return 1;
    for (int y = 0; y < n; ++y) {
        atomic_init(&key[y], pack(0, NONE));
        atomic_init(&mirror[y], 0);
    }
    pthread_barrier_init(&bar, NULL, (unsigned)nthreads + 1);
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return 2;
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, (void *)(intptr_t)t);

    uint64_t e = Ct;
    do {
        e = e / (uint64_t)alpha;
        if (e < 1) e = 1;
        if (phases_total == 0) eps_first = e;
        /* refine initialisation: keep prices (shifted to min q = 0), free every row */
        uint64_t qmin = UINT64_MAX;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&key[y]));
            if (q < qmin) qmin = q;
        }
        for (int y = 0; y < n; ++y) atomic_store(&key[y], pack(key_q(atomic_load(&key[y])) - qmin, NONE));
        R_total += qmin;
        for (int y = 0; y < n; ++y) atomic_store(&mirror[y], key_q(atomic_load(&key[y])));
        uint64_t S = 0;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&key[y]));
            if (q > S) S = q;
        }
        atomic_store(&qpeak, S);
        atomic_store(&next_row, 0);
        atomic_store(&unmatched, n);
        eps = e;
        ++phases_total;
        pthread_barrier_wait(&bar);   /* start */
        pthread_barrier_wait(&bar);   /* end */
        uint64_t lo = UINT64_MAX, hi = 0;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&key[y]));
            if (q < lo) lo = q;
            if (q > hi) hi = q;
        }
        if (atomic_load(&qpeak) > S + 2 * Ct + 2 * e || hi - lo > Ct + e) return 3;
    } while (e > 1);
    eps = 0;
    pthread_barrier_wait(&bar);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);

    int32_t *match = malloc(sizeof(int32_t) * (size_t)n);
    int64_t *prices = malloc(sizeof(int64_t) * (size_t)n);
    if (!match || !prices) return 2;
    for (int x = 0; x < n; ++x) match[x] = -1;
    int64_t cost = 0;
    for (int y = 0; y < n; ++y) {
        const uint64_t k = atomic_load(&key[y]);
        const uint64_t m = key_mate(k);
        if (m >= (uint64_t)n || match[m] != -1) return 2;
        match[m] = y;
        prices[y] = -(int64_t)key_q(k);
        cost += C[(size_t)m * n + y];
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    const int64_t out[3] = {cost, phases_total, atomic_load(&bids)};
    fwrite(out, sizeof(int64_t), 3, o);
    fwrite(match, sizeof(int32_t), (size_t)n, o);
    fwrite(prices, sizeof(int64_t), (size_t)n, o);
    const int64_t scans[2] = {atomic_load(&list_scans), atomic_load(&full_scans)};
    fwrite(scans, sizeof(int64_t), 2, o);
    fclose(o);
    (void)eps_first;
    return 0;
}
