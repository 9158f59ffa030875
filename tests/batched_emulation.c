/*
 * CPU emulation of the batched solver's slot protocol, for the tests: host
 * threads play the warps of one CTA that keeps S instances resident, with
 * C11 atomics in place of the shared-memory atomics, so that
 * ThreadSanitizer can check the protocol for data races and the results can
 * be checked for exactness. It shares no code with the CUDA path or with
 * the oracle.
 *
 * The protocol (the bidding itself is the refine of Sect. 5.1-5.3, as in
 * lockfree_emulation.c):
 *   - a slot's claim word is n << 32 | next free row; a thread claims a row
 *     with one fetch-add and owns it exactly when the returned row is below
 *     the returned n, so no claim can land between two phases or two
 *     instances: a transition first makes every claim fail (next >= n), then
 *     writes the slot's fields, then republishes the word with one exchange;
 *   - a slot's phase ends when its count of unmatched rows reaches 0; the
 *     thread whose bid did that runs the transition: the next phase's
 *     refine initialisation (prices shifted to min q = 0, every mate
 *     cleared), or the instance's results and the next instance from the
 *     shared queue (largest first is the caller's order);
 *   - a thread with nothing to claim yields; all threads stop once every
 *     slot is empty and the queue is drained.
 *
 * Usage: batched_emulation <in> <out>
 *   in:  int32 B, int32 S, int32 threads, int32 alpha, then B int32 sizes n_i,
 *        then the B row-major int32 matrices back to back
 *   out: B int64 costs, then the B matchings back to back (int32 per row)
 * Exit status 0 on success, 1 on a bad input, 2 on an internal error, 3
 * when a price bound that the GPU's 32-bit keys rely on is broken: within a
 * phase every q stays <= S + 2 C~ + 2 eps (S = the largest q after the
 * phase's shift), and after it the spread max q - min q is <= C~ + eps.
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
#define MAXN 1024

static uint64_t pack(uint64_t q, uint64_t mate) { return ((QMAX - q) << MATE_BITS) | mate; }
static uint64_t key_q(uint64_t k) { return QMAX - (k >> MATE_BITS); }
static uint64_t key_mate(uint64_t k) { return k & NONE; }

typedef struct {
    _Atomic uint64_t claim;     /* n << 32 | next row */
    _Atomic int unmatched;
    _Atomic int inst;           /* -1: empty */
    /* written by the transition owner before the claim word is republished;
       read only by threads that hold a valid claim */
    int n, phase, nph, cmin;
    uint64_t eps, Ct, S;
    _Atomic uint64_t qpeak;     /* the largest q committed in this phase */
    const int32_t *C;
    _Atomic uint64_t key[MAXN];
} Slot;

static int B, S, T, alpha;
static int32_t *ns;
static const int32_t **mats;
static int64_t *costs;
static int32_t **matches;
static Slot *slots;
static _Atomic int next_inst;

/* Loads the next instance of the queue into slot s (the caller owns it). */
static void load_next(Slot *sl) {
    for (;;) {
        const int i = atomic_fetch_add(&next_inst, 1);
        if (i >= B) {
            atomic_store(&sl->inst, -1);
            atomic_store(&sl->claim, 0);
            return;
        }
        const int n = ns[i];
        const int32_t *C = mats[i];
        if (n == 1) {
            costs[i] = C[0];
            matches[i][0] = 0;
            continue;
        }
        int32_t cmin = C[0], cmax = C[0];
        for (int k = 0; k < n * n; ++k) {
            if (C[k] < cmin) cmin = C[k];
            if (C[k] > cmax) cmax = C[k];
        }
        const uint64_t Ct = ((uint64_t)n + 1) * (uint64_t)((int64_t)cmax - cmin);
        int nph = 0;
        uint64_t e = Ct;
        do {
            e /= (uint64_t)alpha;
            if (e < 1) e = 1;
            ++nph;
        } while (e > 1);
        for (int y = 0; y < n; ++y) atomic_store(&sl->key[y], pack(0, NONE));
        sl->Ct = Ct;
        sl->S = 0;
        atomic_store(&sl->qpeak, 0);
        sl->n = n;
        sl->C = C;
        sl->cmin = cmin;
        sl->phase = 0;
        sl->nph = nph;
        sl->eps = Ct / (uint64_t)alpha > 1 ? Ct / (uint64_t)alpha : 1;
        atomic_store(&sl->unmatched, n);
        atomic_store(&sl->inst, i);
        atomic_exchange_explicit(&sl->claim, (uint64_t)n << 32, memory_order_release);
        return;
    }
}

/* After the slot's last row was matched: the next phase, or the results and the next instance. */
static void end_phase(Slot *sl) {
    const int n = sl->n;
    {
        uint64_t lo = UINT64_MAX, hi = 0;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&sl->key[y]));
            if (q < lo) lo = q;
            if (q > hi) hi = q;
        }
        if (atomic_load(&sl->qpeak) > sl->S + 2 * sl->Ct + 2 * sl->eps || hi - lo > sl->Ct + sl->eps) exit(3);
    }
    if (sl->phase + 1 < sl->nph) {
        uint64_t m = UINT64_MAX;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&sl->key[y]));
            if (q < m) m = q;
        }
        for (int y = 0; y < n; ++y) atomic_store(&sl->key[y], pack(key_q(atomic_load(&sl->key[y])) - m, NONE));
        uint64_t S = 0;
        for (int y = 0; y < n; ++y) {
            const uint64_t q = key_q(atomic_load(&sl->key[y]));
            if (q > S) S = q;
        }
        sl->S = S;
        atomic_store(&sl->qpeak, S);
        sl->eps = sl->eps / (uint64_t)alpha > 1 ? sl->eps / (uint64_t)alpha : 1;
        sl->phase += 1;
        atomic_store(&sl->unmatched, n);
        atomic_exchange_explicit(&sl->claim, (uint64_t)n << 32, memory_order_release);
        return;
    }
    const int i = atomic_load(&sl->inst);
    int64_t sum = 0;
    for (int y = 0; y < n; ++y) {
        const uint64_t mm = key_mate(atomic_load(&sl->key[y]));
        if (mm >= (uint64_t)n) exit(2);
        matches[i][mm] = y;
        sum += sl->C[(size_t)mm * n + y];
    }
    costs[i] = sum;
    load_next(sl);
}

/* The displacement chain of a claimed row; returns 1 if it matched the slot's last row. */
static int chain(Slot *sl, int x) {
    const int n = sl->n;
    const uint64_t np1 = (uint64_t)n + 1, eps = sl->eps;
    const int32_t *C = sl->C;
    const int32_t cmin = sl->cmin;
    for (;;) {
        const int32_t *row = C + (size_t)x * n;
        uint64_t b1 = UINT64_MAX, b2 = UINT64_MAX, c1 = 0;
        int w = -1;
        for (int y = 0; y < n; ++y) {
            const uint64_t cs = (uint64_t)(uint32_t)(row[y] - cmin) * np1;
            const uint64_t v = cs + key_q(atomic_load_explicit(&sl->key[y], memory_order_relaxed));
            if (v < b1) {
                b2 = b1;
                b1 = v;
                c1 = cs;
                w = y;
            } else if (v < b2) {
                b2 = v;
            }
        }
        const uint64_t nq = (b1 - c1) + (b2 - b1) + eps;
        if (nq >= QMAX) exit(2);
        const uint64_t nk = pack(nq, (uint64_t)x);
        uint64_t cur = atomic_load_explicit(&sl->key[w], memory_order_relaxed);
        int won = 0;
        while (nk < cur) {
            if (atomic_compare_exchange_weak_explicit(&sl->key[w], &cur, nk, memory_order_acq_rel,
                                                      memory_order_relaxed)) {
                won = 1;
                break;
            }
        }
        if (!won) continue;
        uint64_t pk = atomic_load_explicit(&sl->qpeak, memory_order_relaxed);
        while (nq > pk && !atomic_compare_exchange_weak_explicit(&sl->qpeak, &pk, nq, memory_order_relaxed,
                                                                 memory_order_relaxed)) {
        }
        const uint64_t m = key_mate(cur);
        if (m == NONE) return atomic_fetch_sub_explicit(&sl->unmatched, 1, memory_order_acq_rel) == 1;
        x = (int)m;
    }
}

static void *worker(void *arg) {
    int s0 = (int)(intptr_t)arg % S;
    for (;;) {
        int got = 0, live = 0;
        for (int k = 0; k < S && !got; ++k) {
            const int s = (s0 + k) % S;
            Slot *sl = &slots[s];
            if (atomic_load(&sl->inst) < 0) continue;
            live = 1;
            const uint64_t wv = atomic_load_explicit(&sl->claim, memory_order_acquire);
            if ((uint32_t)wv >= (uint32_t)(wv >> 32)) continue;
            const uint64_t old = atomic_fetch_add_explicit(&sl->claim, 1, memory_order_acq_rel);
            if ((uint32_t)old < (uint32_t)(old >> 32)) {
                got = 1;
                s0 = s;
                if (chain(sl, (int)(uint32_t)old)) end_phase(sl);
            }
        }
        if (!got) {
            if (!live) return NULL;
            sched_yield();
        }
    }
}

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int32_t hdr[4];
    if (fread(hdr, sizeof(int32_t), 4, f) != 4) return 1;
    B = hdr[0];
    S = hdr[1];
    T = hdr[2];
    alpha = hdr[3];
    if (B < 1 || S < 1 || S > 16 || T < 1 || T > 64 || alpha < 2) return 1;
    ns = malloc(sizeof(int32_t) * (size_t)B);
    mats = malloc(sizeof(*mats) * (size_t)B);
    costs = calloc((size_t)B, sizeof(int64_t));
    matches = malloc(sizeof(*matches) * (size_t)B);
    slots = calloc((size_t)S, sizeof(Slot));
    if (!ns || !mats || !costs || !matches || !slots) return 2;
    if (fread(ns, sizeof(int32_t), (size_t)B, f) != (size_t)B) return 1;
    for (int i = 0; i < B; ++i) {
        if (ns[i] < 1 || ns[i] > MAXN) return 1;
        int32_t *m = malloc(sizeof(int32_t) * (size_t)ns[i] * ns[i]);
        matches[i] = malloc(sizeof(int32_t) * (size_t)ns[i]);
        if (!m || !matches[i]) return 2;
        if (fread(m, sizeof(int32_t), (size_t)ns[i] * ns[i], f) != (size_t)ns[i] * ns[i]) return 1;
        mats[i] = m;
    }
    fclose(f);
    for (int s = 0; s < S; ++s) load_next(&slots[s]);
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)T);
    if (!th) return 2;
    for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, worker, (void *)(intptr_t)t);
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    fwrite(costs, sizeof(int64_t), (size_t)B, o);
    for (int i = 0; i < B; ++i) fwrite(matches[i], sizeof(int32_t), (size_t)ns[i], o);
    fclose(o);
    return 0;
}
