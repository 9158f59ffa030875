/*
 * CPU emulation of the grid max-flow's lock-free push-relabel, for the
 * tests: host threads play the GPU threads that own the pixels, with C11
 * atomics in place of the device atomics, so that ThreadSanitizer can check
 * the protocol for data races and the flow can be checked against the
 * oracle. It shares no code with the CUDA path or with the oracle.
 *
 * The protocol (Sect. 4: Hong's lock-free push-relabel, Algorithm 4.5, run
 * in cycles with a global relabel between them, Algorithm 4.8):
 *   - init (Algorithm 4.7): every source arc is saturated, e(x) = u(s, x);
 *   - a thread owns the pixels x = t, t + T, ...; in a pass it takes each
 *     owned x with e(x) > 0 and h(x) < |V|, finds the lowest neighbour y over
 *     residual arcs (t at height 0 through the sink arc), and either pushes
 *     d = min(e(x), c_f(x, y)) with atomics on c_f(x, y), c_f(y, x), e(x),
 *     e(y), or relabels h(x) <- h(y) + 1 (only x's owner writes h(x) and the
 *     sink arc of x); x without residual arcs gets h(x) = |V|;
 *   - after `cycle` passes (threads do not wait for one another inside a
 *     cycle) a barrier, then one thread computes the exact distances to t
 *     over the residual graph (a backwards breadth-first search, the global
 *     relabel; unreached pixels get |V|) and counts the pixels with excess
 *     that can reach t; the solve ends when there are none.
 *
 * Usage: maxflow_emulation <in> <out>
 *   in:  int32 H, W, threads, cycle, then int32 cap[4][H*W] (directions
 *        right, left, down, up), src[H*W], snk[H*W]
 *   out: int64 flow, int64 rounds, int64 total excess (the sum of the source
 *        arcs), int64 stranded excess (held by pixels that cannot reach t
 *        after the last global relabel), then uint8 side[H*W]: 1 for a pixel
 *        that cannot reach t (the source side of a minimum cut), else 0
 * Exit status 0 on success, 1 on a bad input, 2 on an internal error.
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

static int H, W, N, NV, T, cycle;
static _Atomic int64_t *e;
static _Atomic int *h;
static _Atomic int *cf;     /* [4][N] */
static _Atomic int *rt;     /* residual sink arcs */
static _Atomic int64_t e_t;
static pthread_barrier_t bar;
static _Atomic int done;

static int nbr(int u, int d) { return d == 0 ? u + 1 : d == 1 ? u - 1 : d == 2 ? u + W : u - W; }

static void *worker(void *arg) {
    const int id = (int)(intptr_t)arg;
    for (;;) {
        pthread_barrier_wait(&bar);   /* a cycle starts (or the solve ends) */
        if (atomic_load(&done)) return NULL;
        for (int it = 0; it < cycle; ++it) {
            for (int u = id; u < N; u += T) {
                const int64_t eu = atomic_load_explicit(&e[u], memory_order_relaxed);
                const int hu = atomic_load_explicit(&h[u], memory_order_relaxed);
                if (eu <= 0 || hu >= NV) continue;
                int hmin = 0x7fffffff, dmin = -1, cmin = 0;
                const int r = atomic_load_explicit(&rt[u], memory_order_relaxed);
                if (r > 0) {
                    hmin = 0;
                    dmin = 4;
                    cmin = r;
                }
                for (int d = 0; d < 4; ++d) {
                    const int cd = atomic_load_explicit(&cf[(size_t)d * N + u], memory_order_relaxed);
                    if (cd > 0) {
                        const int hv = atomic_load_explicit(&h[nbr(u, d)], memory_order_relaxed);
                        if (hv < hmin) {
                            hmin = hv;
                            dmin = d;
                            cmin = cd;
                        }
                    }
                }
                if (dmin < 0) {
                    atomic_store_explicit(&h[u], NV, memory_order_relaxed);
                    continue;
                }
                if (hu > hmin) {   /* push */
                    const int64_t delta = eu < (int64_t)cmin ? eu : (int64_t)cmin;
                    if (dmin == 4) {
                        atomic_store_explicit(&rt[u], r - (int)delta, memory_order_relaxed);
                        atomic_fetch_add(&e_t, delta);
                    } else {
                        const int v = nbr(u, dmin);
                        atomic_fetch_sub(&cf[(size_t)dmin * N + u], (int)delta);
                        atomic_fetch_add(&cf[(size_t)(dmin ^ 1) * N + v], (int)delta);
                        atomic_fetch_add(&e[v], delta);
                    }
                    atomic_fetch_sub(&e[u], delta);
                } else {           /* relabel */
                    atomic_store_explicit(&h[u], hmin + 1, memory_order_relaxed);
                }
            }
        }
        pthread_barrier_wait(&bar);   /* the cycle ends */
    }
}

/* exact distances to t over residual arcs; returns the active pixels that can reach t */
static long global_relabel(int *queue) {
    int head = 0, tail = 0;
    for (int u = 0; u < N; ++u) {
        if (atomic_load(&rt[u]) > 0) {
            atomic_store(&h[u], 1);
            queue[tail++] = u;
        } else {
            atomic_store(&h[u], NV);
        }
    }
    while (head < tail) {
        const int v = queue[head++];
        const int hv = atomic_load(&h[v]);
        for (int d = 0; d < 4; ++d) {
            /* x = neighbour of v with a residual arc x -> v: x's arc in direction d ^ 1 */
            const int i = v / W, j = v % W;
            const int inside = d == 0 ? j + 1 < W : d == 1 ? j > 0 : d == 2 ? i + 1 < H : i > 0;
            if (!inside) continue;
            const int x = nbr(v, d);
            if (atomic_load(&cf[(size_t)(d ^ 1) * N + x]) > 0 && atomic_load(&h[x]) == NV) {
                atomic_store(&h[x], hv + 1);
                queue[tail++] = x;
            }
        }
    }
    long active = 0;
    for (int u = 0; u < N; ++u) active += atomic_load(&e[u]) > 0 && atomic_load(&h[u]) < NV;
    return active;
}

int main(int argc, char **argv) {
    if (argc != 3) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 1;
    int32_t hdr[4];
    if (fread(hdr, sizeof(int32_t), 4, f) != 4) return 1;
    H = hdr[0];
    W = hdr[1];
    T = hdr[2];
    cycle = hdr[3];
    if (H < 1 || W < 1 || (int64_t)H * W > (1 << 22) || T < 1 || T > 64 || cycle < 1) return 1;
    N = H * W;
    NV = N + 2;
    int32_t *buf = malloc(sizeof(int32_t) * (size_t)N * 6);
    e = malloc(sizeof(*e) * (size_t)N);
    h = malloc(sizeof(*h) * (size_t)N);
    cf = malloc(sizeof(*cf) * (size_t)N * 4);
    rt = malloc(sizeof(*rt) * (size_t)N);
    int *queue = malloc(sizeof(int) * (size_t)N);
    if (!buf || !e || !h || !cf || !rt || !queue) return 2;
    if (fread(buf, sizeof(int32_t), (size_t)N * 6, f) != (size_t)N * 6) return 1;
    fclose(f);
    for (int u = 0; u < N; ++u) {
        const int i = u / W, j = u % W;
        const int out[4] = {j + 1 >= W, j == 0, i + 1 >= H, i == 0};
        for (int d = 0; d < 4; ++d) {
            const int c = buf[(size_t)d * N + u];
            if (c < 0 || (out[d] && c != 0)) return 1;
            atomic_init(&cf[(size_t)d * N + u], c);
        }
        if (buf[(size_t)4 * N + u] < 0 || buf[(size_t)5 * N + u] < 0) return 1;
        atomic_init(&e[u], buf[(size_t)4 * N + u]);
        atomic_init(&rt[u], buf[(size_t)5 * N + u]);
        atomic_init(&h[u], 0);
    }
    pthread_barrier_init(&bar, NULL, (unsigned)T + 1);
    pthread_t *th = malloc(sizeof(pthread_t) * (size_t)T);
    if (!th) return 2;
    for (int t = 0; t < T; ++t) pthread_create(&th[t], NULL, worker, (void *)(intptr_t)t);
    int64_t rounds = 0;
    for (;;) {
        if (global_relabel(queue) == 0) break;
        if (++rounds > 1000000) return 2;
        pthread_barrier_wait(&bar);   /* start a cycle */
        pthread_barrier_wait(&bar);   /* its end */
    }
    atomic_store(&done, 1);
    pthread_barrier_wait(&bar);
    for (int t = 0; t < T; ++t) pthread_join(th[t], NULL);
    int64_t total = 0, stranded = 0;
    unsigned char *side = malloc((size_t)N);
    if (!side) return 2;
    for (int u = 0; u < N; ++u) {
        total += buf[(size_t)4 * N + u];
        side[u] = atomic_load(&h[u]) >= NV;
        if (side[u]) stranded += atomic_load(&e[u]);
        else if (atomic_load(&e[u]) != 0) return 2;   /* excess left where t is reachable */
    }
    FILE *o = fopen(argv[2], "wb");
    if (!o) return 2;
    const int64_t out[4] = {atomic_load(&e_t), rounds, total, stranded};
    fwrite(out, sizeof(int64_t), 4, o);
    fwrite(side, 1, (size_t)N, o);
    fclose(o);
    return 0;
}
