/*
 * CPU emulation of the hand-off protocol at the end of a refine phase, for
 * the tests: host threads play the grid refine's warps, the team refine's
 * CTAs and the tail kernel's warps, with C11 atomics in place of the GPU's
 * global atomics, so that ThreadSanitizer can check the protocol for data
 * races and the results can be checked for exactness. Thread joins stand
 * for kernel boundaries. It shares no code with the CUDA path or with the
 * oracle.
 *
 * Each phase of the cost scaling (Algorithm 5.0's eps loop on costs scaled
 * by n + 1, Algorithm 5.2's initialisation, the double push of Algorithm
 * 5.4 committed by one packed-key minimum) runs as three stages:
 *   1. refine: threads claim rows from the phase's queue (rows 0..n-1) and
 *      carry their displacement chains; a bid that leaves at most team_T
 *      rows free moves the hand-off word from 0 to 4 and raises team_go;
 *      a thread that sees 4 parks its row in the hand-off list and stops;
 *   2. team refine (only if team_go): the hand-off items are the parked
 *      rows, then the queue rows never claimed; threads claim items with one
 *      fetch-add and carry chains; a bid that leaves at most tail_T rows free
 *      moves the word from 4 to 1; a thread that sees 1 parks its row in the
 *      tail's queue; the thread that finishes last (a fetch-add on a done
 *      counter) appends the items never claimed and publishes the queue's
 *      length, or, if no hand-off happened, clears the word;
 *   3. tail (only if the word is 1): threads claim the tail's queue and
 *      finish the phase.
 * After each phase every row must be matched and eps-optimal in the
 * version-2 sense (scaled cost + q(M(x)) <= min_y (scaled cost + q(y)) + eps).
 *
 * Usage: team_emulation <in> <out>
 *   in:  int32 n, alpha, refine threads, team threads, tail threads, team_T,
 *        tail_T, then the n x n row-major int32 costs
 *   out: int64 cost, int32 phases the team refine took over, int32 phases
 *        the tail took over, then the matching (int32 per row)
 * Exit status 0 on success, 1 on a bad input, 2 on an internal error, 3
 * when a phase ends without a complete eps-optimal assignment.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#define MATE_BITS 20
#define NONE ((1ull << MATE_BITS) - 1)
#define QMAX ((1ull << 44) - 1)

static uint64_t pack(uint64_t q, uint64_t mate) { return ((QMAX - q) << MATE_BITS) | mate; }
static uint64_t key_q(uint64_t k) { return QMAX - (k >> MATE_BITS); }
static uint64_t key_mate(uint64_t k) { return k & NONE; }

/* the problem and the phase, written between stages only */
static int n;
static int64_t *cs;        /* scaled costs (C - min C)(n + 1) */
static uint64_t eps;
static int team_T, tail_T;

static _Atomic uint64_t *key;
static _Atomic int next_row, free_rows, handoff, team_go;
static _Atomic int tail_count, team_next, team_back, team_done, qlen, tail_next;
static int *tail_rows, *tail_queue;
static _Atomic int bad;

static uint64_t atomic_min_u64(_Atomic uint64_t *p, uint64_t v) {
    uint64_t old = atomic_load(p);
    while (v < old && !atomic_compare_exchange_weak(p, &old, v)) {
    }
    return old;
}

/* One double push of row x at the current prices; returns the row it
   leaves free (x after a lost bid, the displaced mate, or -1). */
static int bid(int x, int *matched) {
    const int64_t *row = cs + (int64_t)x * n;
    uint64_t b1 = UINT64_MAX, b2 = UINT64_MAX;
    int w = -1;
    for (int y = 0; y < n; ++y) {
        const uint64_t v = (uint64_t)row[y] + key_q(atomic_load(&key[y]));
        if (v < b1) {
            b2 = b1;
            b1 = v;
            w = y;
        } else if (v < b2) {
            b2 = v;
        }
    }
    if (b2 == UINT64_MAX) b2 = b1;   /* n = 1 */
    const uint64_t nq = (b1 - (uint64_t)row[w]) + (b2 - b1) + eps;
    if (nq >= QMAX) {
        atomic_store(&bad, 2);
        *matched = 0;
        return -1;
    }
    const uint64_t nk = pack(nq, (uint64_t)x);
    const uint64_t old = atomic_min_u64(&key[w], nk);
    if (old <= nk) {   /* a lower price got there first: bid again */
        *matched = 0;
        return x;
    }
    const uint64_t m = key_mate(old);
    *matched = m == NONE;
    return m == NONE ? -1 : (int)m;
}

/* stage 1: the grid refine */
static void *refine_thread(void *arg) {
    (void)arg;
    int row = -1;
    for (unsigned step = 0;; ++step) {
        if (atomic_load(&bad)) return NULL;
        if (row < 0) {
            const int r = atomic_fetch_add(&next_row, 1);
            if (r >= n) return NULL;
            row = r;
        }
        if (atomic_load(&handoff) == 4) {   /* the team refine takes this row */
            tail_rows[atomic_fetch_add(&tail_count, 1)] = row;
            return NULL;
        }
        int matched;
        const int left = bid(row, &matched);
        if (matched) {
            const int fr = atomic_fetch_sub(&free_rows, 1) - 1;
            int expect = 0;
            if (team_T > 0 && fr <= team_T && atomic_compare_exchange_strong(&handoff, &expect, 4))
                atomic_store(&team_go, 1);
        }
        row = left;
        if ((step & 15) == 15) sched_yield();
    }
}

/* stage 2: the team refine */
static int g_tc, g_q0, g_items, g_team_threads, g_qlen;

static int item_row(int k) { return k < g_tc ? tail_rows[k] : g_q0 + (k - g_tc); }

static void *team_thread(void *arg) {
    (void)arg;
    int row = -1;
    for (unsigned step = 0;; ++step) {
        if (atomic_load(&bad)) break;
        if (row < 0) {
            const int k = atomic_fetch_add(&team_next, 1);
            if (k >= g_items) break;
            row = item_row(k);
        }
        if (atomic_load(&handoff) == 1) {   /* the tail kernel takes this row */
            tail_queue[atomic_fetch_add(&team_back, 1)] = row;
            break;
        }
        int matched;
        const int left = bid(row, &matched);
        if (matched) {
            const int fr = atomic_fetch_sub(&free_rows, 1) - 1;
            int expect = 4;
            if (tail_T > 0 && fr <= tail_T) atomic_compare_exchange_strong(&handoff, &expect, 1);
        }
        row = left;
        if ((step & 15) == 15) sched_yield();
    }
    if (atomic_fetch_add(&team_done, 1) == g_team_threads - 1) {   /* every other thread has finished */
        if (atomic_load(&handoff) == 1) {
            int back = atomic_load(&team_back);
            int k0 = atomic_load(&team_next);
            if (k0 > g_items) k0 = g_items;
            for (int k = k0; k < g_items; ++k) tail_queue[back++] = item_row(k);
            atomic_store(&qlen, back);
        } else {
            int expect = 4;
            atomic_compare_exchange_strong(&handoff, &expect, 0);   /* the phase ended here */
            atomic_store(&qlen, 0);
        }
    }
    return NULL;
}

/* stage 3: the tail */
static void *tail_thread(void *arg) {
    (void)arg;
    int row = -1;
    for (;;) {
        if (atomic_load(&bad)) return NULL;
        if (row < 0) {
            const int k = atomic_fetch_add(&tail_next, 1);
            if (k >= g_qlen) return NULL;
            row = tail_queue[k];
        }
        int matched;
        row = bid(row, &matched);
        if (matched) atomic_fetch_sub(&free_rows, 1);
    }
}

static int run_stage(void *(*fn)(void *), int threads) {
    pthread_t *t = malloc(sizeof(pthread_t) * (size_t)threads);
    if (!t) return 2;
    for (int i = 0; i < threads; ++i)
        if (pthread_create(&t[i], NULL, fn, NULL) != 0) return 2;
    for (int i = 0; i < threads; ++i) pthread_join(t[i], NULL);
    free(t);
    return 0;
}

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int32_t hdr[7];
    if (fread(hdr, sizeof(int32_t), 7, f) != 7) return 1;
    n = hdr[0];
    const int alpha = hdr[1], P = hdr[2], T = hdr[3], Q = hdr[4];
    team_T = hdr[5];
    tail_T = hdr[6];
    if (n < 1 || n >= (int)NONE || alpha < 2 || P < 1 || T < 1 || Q < 1) return 1;
    int32_t *C = malloc(sizeof(int32_t) * (size_t)n * (size_t)n);
    cs = malloc(sizeof(int64_t) * (size_t)n * (size_t)n);
    key = malloc(sizeof(_Atomic uint64_t) * (size_t)n);
    tail_rows = malloc(sizeof(int) * (size_t)n);
    tail_queue = malloc(sizeof(int) * (size_t)n);
    if (!C || !cs || !key || !tail_rows || !tail_queue) return 2;
    if (fread(C, sizeof(int32_t), (size_t)n * (size_t)n, f) != (size_t)n * (size_t)n) return 1;
    fclose(f);
    int32_t cmin = C[0], cmax = C[0];
    for (int64_t i = 0; i < (int64_t)n * n; ++i) {
        if (C[i] < cmin) cmin = C[i];
        if (C[i] > cmax) cmax = C[i];
    }
    for (int64_t i = 0; i < (int64_t)n * n; ++i) cs[i] = ((int64_t)C[i] - cmin) * (n + 1);
    const uint64_t Ct = (uint64_t)((int64_t)cmax - cmin) * (uint64_t)(n + 1);
    for (int y = 0; y < n; ++y) atomic_init(&key[y], pack(0, NONE));
    int team_phases = 0, tail_phases = 0;
    eps = Ct;
    do {
        eps = eps / (uint64_t)alpha > 1 ? eps / (uint64_t)alpha : 1;
        /* phase initialisation (Algorithm 5.2): every row free, prices kept,
           shifted so that the least q is 0 */
        uint64_t qmin = UINT64_MAX;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&key[y]));
            if (q < qmin) qmin = q;
        }
        for (int y = 0; y < n; ++y) atomic_store(&key[y], pack(key_q(atomic_load(&key[y])) - qmin, NONE));
        atomic_store(&next_row, 0);
        atomic_store(&free_rows, n);
        atomic_store(&handoff, 0);
        atomic_store(&team_go, 0);
        atomic_store(&tail_count, 0);
        atomic_store(&team_next, 0);
        atomic_store(&team_back, 0);
        atomic_store(&team_done, 0);
        atomic_store(&qlen, 0);
        atomic_store(&tail_next, 0);
        if (run_stage(refine_thread, P)) return 2;
        if (atomic_load(&team_go)) {
            ++team_phases;
            g_tc = atomic_load(&tail_count);
            const int nr = atomic_load(&next_row);
            g_q0 = nr < n ? nr : n;
            g_items = g_tc + (n - g_q0);
            g_team_threads = T;
            if (run_stage(team_thread, T)) return 2;
            if (atomic_load(&handoff) == 1) {
                ++tail_phases;
                g_qlen = atomic_load(&qlen);
                if (run_stage(tail_thread, Q)) return 2;
            }
        }
        if (atomic_load(&bad)) return 2;
        /* the phase must end with a complete eps-optimal assignment */
        if (atomic_load(&free_rows) != 0) return 3;
        int *seen = calloc((size_t)n, sizeof(int));
        if (!seen) return 2;
        for (int y = 0; y < n; ++y) {
            const uint64_t k = atomic_load(&key[y]);
            const uint64_t x = key_mate(k);
            if (x >= (uint64_t)n || seen[x]) return 3;
            seen[x] = 1;
            uint64_t best = UINT64_MAX;
            for (int z = 0; z < n; ++z) {
                const uint64_t v = (uint64_t)cs[(int64_t)x * n + z] + key_q(atomic_load(&key[z]));
                if (v < best) best = v;
            }
            if ((uint64_t)cs[(int64_t)x * n + y] + key_q(k) > best + eps) return 3;
        }
        free(seen);
    } while (eps > 1);
    int32_t *match = malloc(sizeof(int32_t) * (size_t)n);
    if (!match) return 2;
    int64_t cost = 0;
    for (int y = 0; y < n; ++y) {
        const int x = (int)key_mate(atomic_load(&key[y]));
        match[x] = y;
        cost += C[(int64_t)x * n + y];
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    int32_t counts[2] = {team_phases, tail_phases};
    fwrite(&cost, sizeof(int64_t), 1, o);
    fwrite(counts, sizeof(int32_t), 2, o);
    fwrite(match, sizeof(int32_t), (size_t)n, o);
    fclose(o);
    return 0;
}
