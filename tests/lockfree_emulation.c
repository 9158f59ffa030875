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
 * Usage: lockfree_emulation <in> <out>
 *   in:  int32 n, int32 alpha, int32 threads, then n*n int32 costs (row-major)
 *   out: int64 cost, int64 phases, int64 bids, n int32 matches, n int64
 *        prices (p = -q, paper sign, units of (n+1) C)
 * Exit status 0 on success, 1 on a bad input, 2 on an internal error.
 */
#define _POSIX_C_SOURCE 200809L   /* pthread barriers under -std=c11 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

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

static uint64_t pack(uint64_t q, uint64_t mate) { return ((QMAX - q) << MATE_BITS) | mate; }
static uint64_t key_q(uint64_t k) { return QMAX - (k >> MATE_BITS); }
static uint64_t key_mate(uint64_t k) { return k & NONE; }

/* one displacement chain starting at row x */
static void chain(int x) {
    const uint64_t np1 = (uint64_t)n + 1;
    for (;;) {
        const int32_t *row = C + (size_t)x * n;
        uint64_t b1 = UINT64_MAX, b2 = UINT64_MAX, c1 = 0;
        int w = -1;
        for (int y = 0; y < n; ++y) {
            const uint64_t cs = (uint64_t)(uint32_t)(row[y] - cmin) * np1;
            const uint64_t v = cs + key_q(atomic_load_explicit(&key[y], memory_order_relaxed));
            if (v < b1) {           /* strict: the lowest column wins ties */
                b2 = b1;
                b1 = v;
                c1 = cs;
                w = y;
            } else if (v < b2) {
                b2 = v;
            }
        }
        if (n == 1) b2 = b1;
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
        if (!won) continue;   /* a lower price got there first: rescan x */
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
    for (;;) {
        pthread_barrier_wait(&bar);   /* phase start (thread 0 set it up) */
        if (eps == 0) return NULL;    /* no more phases */
        for (;;) {
            const int x = atomic_fetch_add_explicit(&next_row, 1, memory_order_acq_rel);
            if (x >= n) break;
            chain(x);
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
    int32_t hdr[3];
    if (fread(hdr, sizeof(int32_t), 3, f) != 3) return 1;
    n = hdr[0];
    alpha = hdr[1];
    nthreads = hdr[2];
    if (n < 1 || n >= (int)NONE || alpha < 2 || nthreads < 1 || nthreads > 64) return 1;
    C = malloc(sizeof(int32_t) * (size_t)n * n);
    key = malloc(sizeof(*key) * (size_t)n);
    if (!C || !key) return 2;
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
    for (int y = 0; y < n; ++y) atomic_init(&key[y], pack(0, NONE));
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
        atomic_store(&next_row, 0);
        atomic_store(&unmatched, n);
        eps = e;
        ++phases_total;
        pthread_barrier_wait(&bar);   /* start */
        pthread_barrier_wait(&bar);   /* end */
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
    fclose(o);
    (void)eps_first;
    return 0;
}
