/*
 * Oracle for the assignment problem (dense and sparse) and for maximum flow:
 * plain, sequential, slow and obviously correct CPU code.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py load this library. The CUDA product path shares
 * no code, header, table or helper with it and never calls it.
 *
 * Problem (Sect. 3, definitions of matching, perfect matching, assignment and
 * cost; Sect. 5, reduction of the assignment problem to min-cost flow with
 * u(x,y)=1, c(x,y)=w(x,y)): given an n x n integer matrix C (row x = left
 * vertex, column y = right vertex), find a perfect matching M minimising
 * sum_x C[x][M(x)]. The paper states assignment as a maximum-weight problem
 * but its reduction sets c = w and runs a min-cost flow; this oracle
 * minimises, and a maximising caller passes a negated or offset matrix.
 *
 * Three independent computations of the same optimum:
 *   or_brute_force  - the definition itself, all n! permutations (n <= 10).
 *   or_hungarian    - the shortest-augmenting-path Hungarian method with
 *                     integer dual potentials (Kuhn 1955, Munkres 1957, with
 *                     the potentials of Edmonds and Karp 1972). Not from the
 *                     paper: an independent ground truth that certifies itself
 *                     by LP duality.
 *   or_cost_scaling - the paper's sequential cost-scaling method: the outer
 *                     epsilon loop of Algorithm 5.0, the refine initialisation
 *                     of Algorithm 5.2 (unmatch all, p(x) implicit), and the
 *                     push/relabel step of Algorithm 5.4 taken as the
 *                     Goldberg-Kennedy double push (the paper's reference [9]).
 *   or_cost_scaling_arcfix - the same, with Sect. 5.2's arc fixing: after
 *                     every phase but the last, arcs whose reduced cost
 *                     exceeds 2 n eps are deleted for good.
 * and certificate checkers for any claimed matching, among them
 * or_certify_optimal, which proves a matching optimal at any size with no
 * duals given (Klein's negative-cycle criterion). The same problem on
 * sparse bipartite graphs (arcs in CSR form) has its own brute force,
 * successive-shortest-path solver and checkers (or_sparse_*, below), and
 * the paper's first problem, maximum s-t flow (Sect. 4), has Dinic's
 * algorithm, a brute-force minimum cut and a cut-capacity checker
 * (or_maxflow_dinic, or_min_cut_brute, or_cut_capacity, at the end).
 *
 * All arithmetic is exact int64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_INVALID 1
#define OR_INVARIANT 2
#define OR_OVERFLOW 3
#define OR_NOMEM 4

#define OR_INF (INT64_MAX / 4)

/* ------------------------------------------------------------------ */
/* Brute force: enumerate every permutation (Heap's algorithm).        */
/* ------------------------------------------------------------------ */
int or_brute_force(const int32_t *C, int32_t n, int32_t *match, int64_t *cost)
{
    if (n < 0 || n > 10 || (n > 0 && (!C || !match)) || !cost)
        return OR_INVALID;
    if (n == 0) { *cost = 0; return OR_OK; }
    int32_t perm[10], cnt[10];
    for (int i = 0; i < n; ++i) { perm[i] = i; cnt[i] = 0; }
    int64_t best = 0;
    for (int x = 0; x < n; ++x) best += C[(int64_t)x * n + perm[x]];
    memcpy(match, perm, sizeof(int32_t) * n);
    int i = 1;
    while (i < n) {
        if (cnt[i] < i) {
            int j = (i % 2 == 0) ? 0 : cnt[i];
            int32_t t = perm[j]; perm[j] = perm[i]; perm[i] = t;
            int64_t s = 0;
            for (int x = 0; x < n; ++x) s += C[(int64_t)x * n + perm[x]];
            if (s < best) { best = s; memcpy(match, perm, sizeof(int32_t) * n); }
            cnt[i]++;
            i = 1;
        } else {
            cnt[i] = 0;
            i++;
        }
    }
    *cost = best;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Hungarian method, shortest augmenting paths, O(n^3).                */
/*                                                                     */
/* Rows enter one at a time. For the entering row a Dijkstra search    */
/* over columns, with reduced costs C[i][j] - u[i] - v[j] >= 0, finds  */
/* the cheapest alternating path to a free column; the duals move by   */
/* the search distances so that every tree edge stays tight, then the  */
/* path is flipped. Invariants: u[i] + v[j] <= C[i][j] for all i, j,   */
/* with equality on matched pairs. Column index n is a virtual column  */
/* that holds the entering row.                                        */
/* ------------------------------------------------------------------ */
int or_hungarian(const int32_t *C, int32_t n, int32_t *match, int64_t *cost,
                 int64_t *u_out, int64_t *v_out)
{
    if (n < 0 || (n > 0 && (!C || !match)) || !cost) return OR_INVALID;
    if (n == 0) { *cost = 0; return OR_OK; }
    const int N = n + 1;
    int64_t *u = calloc((size_t)n, sizeof(int64_t));
    int64_t *v = calloc((size_t)N, sizeof(int64_t));
    int64_t *dist = malloc(sizeof(int64_t) * N);
    int32_t *owner = malloc(sizeof(int32_t) * N);   /* row holding column j */
    int32_t *from = malloc(sizeof(int32_t) * N);    /* previous column on path */
    char *intree = malloc((size_t)N);
    if (!u || !v || !dist || !owner || !from || !intree) {
        free(u); free(v); free(dist); free(owner); free(from); free(intree);
        return OR_NOMEM;
    }
    for (int j = 0; j < N; ++j) owner[j] = -1;

    for (int32_t r = 0; r < n; ++r) {
        int32_t jcur = n;
        owner[n] = r;
        for (int j = 0; j < N; ++j) { dist[j] = OR_INF; intree[j] = 0; }
        for (;;) {
            intree[jcur] = 1;
            const int32_t i = owner[jcur];
            const int32_t *row = C + (int64_t)i * n;
            int64_t delta = OR_INF;
            int32_t jnext = -1;
            for (int32_t j = 0; j < n; ++j) {
                if (intree[j]) continue;
                int64_t red = (int64_t)row[j] - u[i] - v[j];
                if (red < dist[j]) { dist[j] = red; from[j] = jcur; }
                if (dist[j] < delta) { delta = dist[j]; jnext = j; }
            }
            for (int j = 0; j < N; ++j) {
                if (intree[j]) { u[owner[j]] += delta; v[j] -= delta; }
                else dist[j] -= delta;
            }
            jcur = jnext;
            if (owner[jcur] < 0) break;
        }
        while (jcur != n) {            /* flip the augmenting path */
            int32_t jprev = from[jcur];
            owner[jcur] = owner[jprev];
            jcur = jprev;
        }
    }
    int64_t total = 0;
    for (int32_t j = 0; j < n; ++j) {
        match[owner[j]] = j;
        total += C[(int64_t)owner[j] * n + j];
    }
    *cost = total;
    if (u_out) memcpy(u_out, u, sizeof(int64_t) * n);
    if (v_out) memcpy(v_out, v, sizeof(int64_t) * n);
    free(u); free(v); free(dist); free(owner); free(from); free(intree);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Sequential cost scaling (Sect. 5.1-5.3).                            */
/*                                                                     */
/* Costs are scaled by (n+1): c~ = (n+1) C. Column prices p(y) use the */
/* paper's sign (c_p(x,y) = c(x,y) + p(x) - p(y), c'_p = c - p(y)) and */
/* start at 0 (Alg. 5.0) or at init_prices. Row prices are implicit:   */
/* p(x) = -min_y (c'_p(x,y) + eps) (Alg. 5.2, refine initialisation).  */
/*                                                                     */
/* Outer loop (Alg. 5.0): eps <- eps0 (default C~ = (n+1)(max C -      */
/* min C)); repeat refine with eps <- max(1, floor(eps / alpha)) until */
/* the refine run at eps <= final_eps has finished. With final_eps = 1 */
/* the result is optimal: summing the eps-complementary slackness of   */
/* every row over the matching gives (n+1) cost <= (n+1) OPT + n.      */
/*                                                                     */
/* Refine (Alg. 5.2 + Alg. 5.4): f <- 0 (every row unmatched, prices    */
/* kept). While an unmatched row x exists (FIFO order): scan all        */
/* columns for the smallest c'_p(x,y) (best, at w; lowest index on     */
/* ties) and the second smallest over y != w (second). Push x -> w     */
/* (admissible under the implicit p(x)); then w is relabelled to        */
/* p(w) <- p(w) - (second - best + eps) and pushes the unit of its old */
/* mate back, which becomes unmatched (double push).                   */
/*                                                                     */
/* stats (optional, 4 entries): phases, row scans, displacements,      */
/* eps of the first phase. check != 0 verifies after every phase that  */
/* no price rose (Lemma 5.2) and that every row is eps-optimal          */
/* (Lemma 5.6); a violation returns OR_INVARIANT.                       */
/* ------------------------------------------------------------------ */
int or_cost_scaling(const int32_t *C, int32_t n, int32_t alpha, int64_t eps0,
                    const int64_t *init_prices, int64_t final_eps, int32_t check,
                    int32_t *match, int64_t *cost, int64_t *prices_out,
                    int64_t *stats)
{
    if (n < 0 || alpha < 2 || final_eps < 1 || (n > 0 && (!C || !match)) || !cost)
        return OR_INVALID;
    if (stats) for (int k = 0; k < 4; ++k) stats[k] = 0;
    if (n == 0) { *cost = 0; return OR_OK; }
    if (n == 1) {
        match[0] = 0; *cost = C[0];
        if (prices_out) prices_out[0] = init_prices ? init_prices[0] : 0;
        return OR_OK;
    }
    const int64_t np1 = (int64_t)n + 1;
    int32_t cmin = C[0], cmax = C[0];
    for (int64_t k = 0; k < (int64_t)n * n; ++k) {
        if (C[k] < cmin) cmin = C[k];
        if (C[k] > cmax) cmax = C[k];
    }
    const int64_t Ct = np1 * ((int64_t)cmax - (int64_t)cmin);
    int64_t eps = eps0 > 0 ? eps0 : Ct;

    int64_t *p = malloc(sizeof(int64_t) * n);
    int64_t *p_start = check ? malloc(sizeof(int64_t) * n) : NULL;
    int32_t *holder = malloc(sizeof(int32_t) * n);   /* row matched to column y */
    int32_t *col = malloc(sizeof(int32_t) * n);      /* column matched to row x */
    int32_t *queue = malloc(sizeof(int32_t) * n);
    if (!p || (check && !p_start) || !holder || !col || !queue) {
        free(p); free(p_start); free(holder); free(col); free(queue);
        return OR_NOMEM;
    }
    for (int32_t y = 0; y < n; ++y) p[y] = init_prices ? init_prices[y] : 0;

    int rc = OR_OK;
    int64_t phases = 0, scans = 0, displaced = 0, eps_first = 0;
    do {
        eps = eps / alpha;
        if (eps < 1) eps = 1;
        if (phases == 0) eps_first = eps;
        if (check) memcpy(p_start, p, sizeof(int64_t) * n);
        for (int32_t y = 0; y < n; ++y) holder[y] = -1;
        for (int32_t x = 0; x < n; ++x) { col[x] = -1; queue[x] = x; }
        int64_t head = 0, tail = n;               /* ring buffer of n slots */
        while (head != tail) {
            const int32_t x = queue[head % n];
            head++;
            const int32_t *row = C + (int64_t)x * n;
            int64_t best = OR_INF, second = OR_INF;
            int32_t w = -1;
            for (int32_t y = 0; y < n; ++y) {
                const int64_t cp = np1 * (int64_t)row[y] - p[y];   /* c'_p(x,y) */
                if (cp < best) { second = best; best = cp; w = y; }
                else if (cp < second) second = cp;
            }
            scans++;
            p[w] -= (second - best) + eps;
            if (p[w] < -(INT64_MAX / 8)) { rc = OR_OVERFLOW; goto done; }
            const int32_t old = holder[w];
            holder[w] = x;
            col[x] = w;
            if (old >= 0) {
                col[old] = -1;
                queue[tail % n] = old;
                tail++;
                displaced++;
            }
        }
        phases++;
        if (check) {
            for (int32_t y = 0; y < n; ++y)
                if (p[y] > p_start[y]) { rc = OR_INVARIANT; goto done; }
            for (int32_t x = 0; x < n; ++x) {
                const int32_t *row = C + (int64_t)x * n;
                int64_t mn = OR_INF;
                for (int32_t y = 0; y < n; ++y) {
                    const int64_t cp = np1 * (int64_t)row[y] - p[y];
                    if (cp < mn) mn = cp;
                }
                const int64_t mine = np1 * (int64_t)row[col[x]] - p[col[x]];
                if (mine > mn + eps) { rc = OR_INVARIANT; goto done; }
            }
        }
    } while (eps > final_eps);

    {
        int64_t total = 0;
        for (int32_t x = 0; x < n; ++x) {
            match[x] = col[x];
            total += C[(int64_t)x * n + col[x]];
        }
        *cost = total;
        if (prices_out) memcpy(prices_out, p, sizeof(int64_t) * n);
    }
done:
    if (stats) { stats[0] = phases; stats[1] = scans; stats[2] = displaced; stats[3] = eps_first; }
    free(p); free(p_start); free(holder); free(col); free(queue);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Sequential cost scaling with arc fixing (Sect. 5.2, the arc          */
/* heuristic taken from the paper's reference [8]).                     */
/*                                                                     */
/* The same loop as or_cost_scaling (Alg. 5.0, Alg. 5.2, Alg. 5.4 as a  */
/* double push), on a graph that loses arcs. When a phase other than   */
/* the last has ended, f is an eps-optimal flow: a perfect matching,    */
/* every row x eps-optimal with respect to the column prices p and the  */
/* row price of Alg. 5.2, p(x) = -min over x's remaining arcs of        */
/* (c'_p(x,y) + eps). Sect. 5.2: an arc whose reduced cost             */
/* c_p(x,y) = c~(x,y) + p(x) - p(y) exceeds 2 n eps keeps its flow in   */
/* every later phase, so it is deleted for good. Later phases scan only */
/* the remaining arcs of a row. A row left with one arc has no second   */
/* best; its bid lowers the column's price by eps.                      */
/*                                                                     */
/* Why no optimal assignment loses an arc (the reading the paper does  */
/* not spell out): an optimal assignment M* that used a deleted arc a   */
/* would differ from f on an alternating cycle through a with k <= n    */
/* rows. Taken along f's residual arcs, the cycle costs at least        */
/* c_p(a) - (k-1) eps (prices cancel around a cycle; f's other          */
/* unmatched arcs have c_p >= -eps and its reversed matched arcs        */
/* c_p >= 0). Taken the other way it is a cycle of M*'s residual graph, */
/* which has no negative cycle, so the first direction costs <= 0.      */
/* Hence c_p(a) <= (k-1) eps < 2 n eps. (An eps-optimal M* in place of  */
/* the optimum gives c_p(a) <= (2k-1) eps, the paper's 2 n eps bound.)  */
/*                                                                     */
/* Arguments as or_cost_scaling (no check mode). fixed_out (optional,  */
/* n*n bytes) gets 1 for every deleted arc. stats (optional, 5         */
/* entries): phases, row scans, displacements, eps of the first phase, */
/* arcs deleted.                                                       */
/* ------------------------------------------------------------------ */
int or_cost_scaling_arcfix(const int32_t *C, int32_t n, int32_t alpha, int64_t eps0,
                           const int64_t *init_prices, int32_t *match, int64_t *cost,
                           int64_t *prices_out, uint8_t *fixed_out, int64_t *stats)
{
    if (n < 0 || alpha < 2 || (n > 0 && (!C || !match)) || !cost) return OR_INVALID;
    if (stats) for (int k = 0; k < 5; ++k) stats[k] = 0;
    if (n == 0) { *cost = 0; return OR_OK; }
    const int64_t np1 = (int64_t)n + 1;
    int32_t cmin = C[0], cmax = C[0];
    for (int64_t k = 0; k < (int64_t)n * n; ++k) {
        if (C[k] < cmin) cmin = C[k];
        if (C[k] > cmax) cmax = C[k];
    }
    int64_t eps = eps0 > 0 ? eps0 : np1 * ((int64_t)cmax - (int64_t)cmin);

    int64_t *p = malloc(sizeof(int64_t) * n);
    int32_t *holder = malloc(sizeof(int32_t) * n);
    int32_t *col = malloc(sizeof(int32_t) * n);
    int32_t *queue = malloc(sizeof(int32_t) * n);
    uint8_t *gone = calloc((size_t)n * n, 1);         /* 1: arc deleted */
    if (!p || !holder || !col || !queue || !gone) {
        free(p); free(holder); free(col); free(queue); free(gone);
        return OR_NOMEM;
    }
    for (int32_t y = 0; y < n; ++y) p[y] = init_prices ? init_prices[y] : 0;

    int rc = OR_OK;
    int64_t phases = 0, scans = 0, displaced = 0, eps_first = 0, deleted = 0;
    for (;;) {
        eps = eps / alpha;
        if (eps < 1) eps = 1;
        if (phases == 0) eps_first = eps;
        for (int32_t y = 0; y < n; ++y) holder[y] = -1;
        for (int32_t x = 0; x < n; ++x) { col[x] = -1; queue[x] = x; }
        int64_t head = 0, tail = n;
        while (head != tail) {
            const int32_t x = queue[head % n];
            head++;
            const int32_t *row = C + (int64_t)x * n;
            const uint8_t *dead = gone + (int64_t)x * n;
            int64_t best = OR_INF, second = OR_INF;
            int32_t w = -1;
            for (int32_t y = 0; y < n; ++y) {
                if (dead[y]) continue;
                const int64_t cp = np1 * (int64_t)row[y] - p[y];   /* c'_p(x,y) */
                if (cp < best) { second = best; best = cp; w = y; }
                else if (cp < second) second = cp;
            }
            if (w < 0) { rc = OR_INVARIANT; goto done; }      /* a row lost every arc */
            if (second == OR_INF) second = best;               /* one arc left */
            scans++;
            p[w] -= (second - best) + eps;
            if (p[w] < -(INT64_MAX / 8)) { rc = OR_OVERFLOW; goto done; }
            const int32_t old = holder[w];
            holder[w] = x;
            col[x] = w;
            if (old >= 0) {
                col[old] = -1;
                queue[tail % n] = old;
                tail++;
                displaced++;
            }
        }
        phases++;
        if (eps <= 1) break;
        /* arc fixing on the eps-optimal flow this phase produced */
        for (int32_t x = 0; x < n; ++x) {
            const int32_t *row = C + (int64_t)x * n;
            uint8_t *dead = gone + (int64_t)x * n;
            int64_t mn = OR_INF;
            for (int32_t y = 0; y < n; ++y)
                if (!dead[y] && np1 * (int64_t)row[y] - p[y] < mn) mn = np1 * (int64_t)row[y] - p[y];
            const int64_t px = -(mn + eps);                    /* Alg. 5.2's row price */
            for (int32_t y = 0; y < n; ++y) {
                if (dead[y]) continue;
                const int64_t cp = np1 * (int64_t)row[y] + px - p[y];   /* c_p(x,y) */
                if (cp > 2 * (int64_t)n * eps) { dead[y] = 1; deleted++; }
            }
        }
    }
    {
        int64_t total = 0;
        for (int32_t x = 0; x < n; ++x) {
            match[x] = col[x];
            total += C[(int64_t)x * n + col[x]];
        }
        *cost = total;
        if (prices_out) memcpy(prices_out, p, sizeof(int64_t) * n);
        if (fixed_out) memcpy(fixed_out, gone, (size_t)n * n);
    }
done:
    if (stats) {
        stats[0] = phases; stats[1] = scans; stats[2] = displaced; stats[3] = eps_first; stats[4] = deleted;
    }
    free(p); free(holder); free(col); free(queue); free(gone);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Certificates.                                                       */
/* ------------------------------------------------------------------ */

/* 0: match is a permutation of 0..n-1 and sum C[x][match[x]] equals
 * claimed_cost; 10: not a permutation; 11: cost differs. */
int or_check_matching(const int32_t *C, int32_t n, const int32_t *match,
                      int64_t claimed_cost)
{
    if (n < 0) return OR_INVALID;
    if (n == 0) return claimed_cost == 0 ? OR_OK : 11;
    char *seen = calloc((size_t)n, 1);
    if (!seen) return OR_NOMEM;
    int64_t total = 0;
    int rc = OR_OK;
    for (int32_t x = 0; x < n; ++x) {
        int32_t y = match[x];
        if (y < 0 || y >= n || seen[y]) { rc = 10; break; }
        seen[y] = 1;
        total += C[(int64_t)x * n + y];
    }
    free(seen);
    if (rc == OR_OK && total != claimed_cost) rc = 11;
    return rc;
}

/* LP duality certificate for a matching and integer duals (u, v):
 * 12: u[x] + v[y] > C[x][y] somewhere (infeasible dual);
 * 13: a matched pair is not tight; 14: sum u + sum v != cost of the matching. */
int or_check_duals(const int32_t *C, int32_t n, const int32_t *match,
                   const int64_t *u, const int64_t *v)
{
    if (n < 0) return OR_INVALID;
    int64_t dual = 0, primal = 0;
    for (int32_t x = 0; x < n; ++x) {
        const int32_t *row = C + (int64_t)x * n;
        for (int32_t y = 0; y < n; ++y)
            if (u[x] + v[y] > (int64_t)row[y]) return 12;
        if (u[x] + v[match[x]] != (int64_t)row[match[x]]) return 13;
        dual += u[x] + v[x];          /* x also runs over every column */
        primal += row[match[x]];
    }
    return dual == primal ? OR_OK : 14;
}

/* eps-complementary slackness of a matching with column prices p (paper's
 * sign) on costs scaled by (n+1): for every row x,
 *   (n+1)C[x][M(x)] - p(M(x)) <= min_y ((n+1)C[x][y] - p(y)) + eps.
 * With eps = 1 this implies optimality. 15: violated. */
int or_check_eps_cs(const int32_t *C, int32_t n, const int32_t *match,
                    const int64_t *p, int64_t eps)
{
    if (n < 0) return OR_INVALID;
    const int64_t np1 = (int64_t)n + 1;
    for (int32_t x = 0; x < n; ++x) {
        const int32_t *row = C + (int64_t)x * n;
        int64_t mn = OR_INF;
        for (int32_t y = 0; y < n; ++y) {
            const int64_t cp = np1 * (int64_t)row[y] - p[y];
            if (cp < mn) mn = cp;
        }
        const int64_t mine = np1 * (int64_t)row[match[x]] - p[match[x]];
        if (mine > mn + eps) return 15;
    }
    return OR_OK;
}

/* Optimality of a perfect matching with no duals given (the negative-cycle
 * criterion of Klein 1967: an optimal flow admits no residual cycle of
 * negative cost, which is the eps = 0 end of the eps-optimality of Sect. 5).
 * In the assignment problem a residual cycle moves rows x_1..x_k each from
 * its column M(x_i) to the next row's column, so M is optimal iff the graph
 * on columns with an arc M(x) -> y of length C[x][y] - C[x][M(x)] for every
 * row x and column y has no negative cycle. Bellman-Ford from a virtual
 * source joined to every column by a zero-length arc: n + 1 vertices, so
 * the distances settle within n sweeps unless a negative cycle exists.
 * The settled distances d give LP duals v(y) = d(y) and
 * u(x) = C[x][M(x)] - d(M(x)), tight on M and feasible (that is the
 * fixpoint), written when u_out / v_out are not NULL.
 * 0: optimal; 10: not a permutation; 16: a negative cycle (not optimal). */
int or_certify_optimal(const int32_t *C, int32_t n, const int32_t *match,
                       int64_t *u_out, int64_t *v_out)
{
    if (n < 0) return OR_INVALID;
    if (n == 0) return OR_OK;
    char *seen = calloc((size_t)n, 1);
    int64_t *d = calloc((size_t)n, sizeof(int64_t));
    if (!seen || !d) { free(seen); free(d); return OR_NOMEM; }
    int rc = OR_OK;
    for (int32_t x = 0; x < n && rc == OR_OK; ++x) {
        const int32_t y = match[x];
        if (y < 0 || y >= n || seen[y]) rc = 10;
        else seen[y] = 1;
    }
    int changed = rc == OR_OK;
    for (int32_t sweep = 0; changed && sweep <= n; ++sweep) {
        changed = 0;
        for (int32_t x = 0; x < n; ++x) {
            const int32_t *row = C + (int64_t)x * n;
            const int64_t from = d[match[x]] - (int64_t)row[match[x]];
            for (int32_t y = 0; y < n; ++y)
                if (from + (int64_t)row[y] < d[y]) { d[y] = from + (int64_t)row[y]; changed = 1; }
        }
    }
    if (rc == OR_OK && changed) rc = 16;   /* still relaxing after n + 1 sweeps */
    if (rc == OR_OK) {
        for (int32_t x = 0; x < n; ++x) {
            if (u_out) u_out[x] = (int64_t)C[(int64_t)x * n + match[x]] - d[match[x]];
            if (v_out) v_out[x] = d[x];
        }
    }
    free(seen);
    free(d);
    return rc;
}

/* ================================================================== */
/* Sparse bipartite graphs.                                            */
/*                                                                     */
/* The paper's implementation takes arbitrary bipartite graphs (Sect.  */
/* 1 and Sect. 6), not only complete ones. A graph on rows 0..n-1 and  */
/* columns 0..n-1 is given by its arcs in CSR form: row x's arcs are   */
/* k = row_ptr[x] .. row_ptr[x+1]-1, to column cols[k] at cost         */
/* costs[k]. A row may list the same column twice (parallel arcs: the  */
/* cheaper one is the one a matching would use). The problem: a        */
/* perfect matching that uses arcs only and minimises its total cost,  */
/* or OR_INFEASIBLE when the graph has no perfect matching.            */
/* ================================================================== */
#define OR_INFEASIBLE 5

static int sp_valid(int32_t n, const int32_t *row_ptr, const int32_t *cols)
{
    if (n < 0 || (n > 0 && (!row_ptr || row_ptr[0] != 0))) return 0;
    for (int32_t x = 0; x < n; ++x) {
        if (row_ptr[x + 1] < row_ptr[x]) return 0;
        for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k)
            if (cols[k] < 0 || cols[k] >= n) return 0;
    }
    return 1;
}

/* Cheapest arc x -> y, or OR_INF when there is none. */
static int64_t sp_arc(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs,
                      int32_t x, int32_t y)
{
    int64_t best = OR_INF;
    for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k)
        if (cols[k] == y && costs[k] < best) best = costs[k];
    return best;
}

/* Brute force: every permutation of the columns, kept only if each of its
 * pairs is an arc (n <= 10). */
int or_sparse_brute_force(int32_t n, const int32_t *row_ptr, const int32_t *cols,
                          const int32_t *costs, int32_t *match, int64_t *cost)
{
    if (n < 0 || n > 10 || !cost || (n > 0 && !match) || !sp_valid(n, row_ptr, cols)) return OR_INVALID;
    if (n == 0) { *cost = 0; return OR_OK; }
    int32_t perm[10], cnt[10];
    int64_t w[10][10];
    for (int x = 0; x < n; ++x)
        for (int y = 0; y < n; ++y) w[x][y] = sp_arc(row_ptr, cols, costs, x, y);
    for (int i = 0; i < n; ++i) { perm[i] = i; cnt[i] = 0; }
    int64_t best = OR_INF;
    for (;;) {
        int64_t s = 0;
        for (int x = 0; x < n && s < OR_INF; ++x) s = w[x][perm[x]] >= OR_INF ? OR_INF : s + w[x][perm[x]];
        if (s < best) { best = s; for (int x = 0; x < n; ++x) match[x] = perm[x]; }
        int i = 1;                      /* next permutation (Heap's algorithm) */
        while (i < n && cnt[i] >= i) { cnt[i] = 0; ++i; }
        if (i >= n) break;
        int j = (i % 2 == 0) ? 0 : cnt[i];
        int32_t t = perm[j]; perm[j] = perm[i]; perm[i] = t;
        cnt[i]++;
    }
    if (best >= OR_INF) return OR_INFEASIBLE;
    *cost = best;
    return OR_OK;
}

/* Successive shortest augmenting paths on the arcs (the sparse form of
 * or_hungarian; not from the paper, an independent ground truth). Rows
 * enter one at a time; a Dijkstra search over columns with reduced costs
 * c(x,y) - u(x) - v(y) >= 0 on arcs finds the cheapest alternating path
 * from the entering row to a free column; the duals move by the search
 * distances and the path is flipped. If no free column can be reached the
 * graph has no perfect matching (the search has found a set of rows whose
 * arcs reach fewer columns: Hall's condition fails). Integer duals u, v
 * (optional) certify the result: u(x) + v(y) <= c(x,y) on every arc, with
 * equality on the matching. */
int or_sparse_ssp(int32_t n, const int32_t *row_ptr, const int32_t *cols, const int32_t *costs,
                  int32_t *match, int64_t *cost, int64_t *u_out, int64_t *v_out)
{
    if (!cost || (n > 0 && !match) || !sp_valid(n, row_ptr, cols)) return OR_INVALID;
    if (n == 0) { *cost = 0; return OR_OK; }
    int64_t *u = calloc((size_t)n, sizeof(int64_t));
    int64_t *v = calloc((size_t)n, sizeof(int64_t));
    int64_t *dist = malloc(sizeof(int64_t) * n);
    int32_t *owner = malloc(sizeof(int32_t) * n);   /* row matched to column y */
    int32_t *from = malloc(sizeof(int32_t) * n);    /* column before y on the path, -1 = root row */
    char *done = malloc((size_t)n);
    if (!u || !v || !dist || !owner || !from || !done) {
        free(u); free(v); free(dist); free(owner); free(from); free(done);
        return OR_NOMEM;
    }
    for (int32_t y = 0; y < n; ++y) owner[y] = -1;
    int rc = OR_OK;
    for (int32_t r = 0; r < n && rc == OR_OK; ++r) {
        for (int32_t y = 0; y < n; ++y) { dist[y] = OR_INF; done[y] = 0; from[y] = -1; }
        /* the entering row's arcs; u(r) = 0 before the search */
        u[r] = 0;
        for (int32_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            const int64_t red = (int64_t)costs[k] - u[r] - v[cols[k]];
            if (red < dist[cols[k]]) { dist[cols[k]] = red; from[cols[k]] = -1; }
        }
        int32_t yfree = -1;
        int64_t dfree = 0;
        for (;;) {
            int32_t y = -1;
            int64_t dmin = OR_INF;
            for (int32_t j = 0; j < n; ++j)
                if (!done[j] && dist[j] < dmin) { dmin = dist[j]; y = j; }
            if (y < 0) { rc = OR_INFEASIBLE; break; }
            done[y] = 1;
            if (owner[y] < 0) { yfree = y; dfree = dmin; break; }
            const int32_t x = owner[y];          /* continue through y's row */
            for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k) {
                const int32_t j = cols[k];
                if (done[j]) continue;
                const int64_t red = dmin + (int64_t)costs[k] - u[x] - v[j];
                if (red < dist[j]) { dist[j] = red; from[j] = y; }
            }
        }
        if (rc != OR_OK) break;
        /* dual update: settled columns move by (dfree - dist), their rows too */
        u[r] += dfree;
        for (int32_t j = 0; j < n; ++j) {
            if (!done[j] || j == yfree) continue;
            const int64_t d = dfree - dist[j];
            v[j] -= d;
            u[owner[j]] += d;
        }
        /* flip the path: yfree <- ... <- root row r */
        int32_t y = yfree;
        while (from[y] >= 0) {
            const int32_t yp = from[y];
            owner[y] = owner[yp];
            y = yp;
        }
        owner[y] = r;
    }
    if (rc == OR_OK) {
        int64_t total = 0;
        for (int32_t y = 0; y < n; ++y) {
            match[owner[y]] = y;
            total += sp_arc(row_ptr, cols, costs, owner[y], y);
        }
        *cost = total;
        if (u_out) memcpy(u_out, u, sizeof(int64_t) * n);
        if (v_out) memcpy(v_out, v, sizeof(int64_t) * n);
    }
    free(u); free(v); free(dist); free(owner); free(from); free(done);
    return rc;
}

/* match is a permutation made of arcs and its cost (cheapest parallel arc)
 * equals claimed. */
int or_sparse_check_matching(int32_t n, const int32_t *row_ptr, const int32_t *cols,
                             const int32_t *costs, const int32_t *match, int64_t claimed)
{
    if (!sp_valid(n, row_ptr, cols)) return OR_INVALID;
    char *seen = calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return OR_NOMEM;
    int64_t total = 0;
    int rc = OR_OK;
    for (int32_t x = 0; x < n && rc == OR_OK; ++x) {
        const int32_t y = match[x];
        if (y < 0 || y >= n || seen[y]) { rc = 11; break; }
        seen[y] = 1;
        const int64_t c = sp_arc(row_ptr, cols, costs, x, y);
        if (c >= OR_INF) { rc = 12; break; }
        total += c;
    }
    free(seen);
    if (rc == OR_OK && total != claimed) rc = 13;
    return rc;
}

/* LP duality certificate on the arcs: u(x) + v(y) <= c(x,y) on every arc,
 * equality on the matching; then sum u + sum v = cost(match) is optimal. */
int or_sparse_check_duals(int32_t n, const int32_t *row_ptr, const int32_t *cols,
                          const int32_t *costs, const int32_t *match,
                          const int64_t *u, const int64_t *v)
{
    if (!sp_valid(n, row_ptr, cols)) return OR_INVALID;
    for (int32_t x = 0; x < n; ++x)
        for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k)
            if (u[x] + v[cols[k]] > (int64_t)costs[k]) return 14;
    for (int32_t x = 0; x < n; ++x)
        if (u[x] + v[match[x]] != sp_arc(row_ptr, cols, costs, x, match[x])) return 16;
    return OR_OK;
}

/* eps-complementary slackness of every row on costs scaled by n + 1, over
 * its arcs: (n+1) c(x,M(x)) - p(M(x)) <= min over arcs (n+1) c(x,y) - p(y)
 * + eps. At eps = 1 it proves the matching optimal (Sect. 5.1, Lemma 5.6:
 * summed over the rows, (n+1) cost <= (n+1) OPT + n). */
int or_sparse_check_eps_cs(int32_t n, const int32_t *row_ptr, const int32_t *cols,
                           const int32_t *costs, const int32_t *match, const int64_t *p, int64_t eps)
{
    if (!sp_valid(n, row_ptr, cols)) return OR_INVALID;
    const int64_t np1 = (int64_t)n + 1;
    for (int32_t x = 0; x < n; ++x) {
        int64_t mn = OR_INF;
        for (int32_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k) {
            const int64_t cp = np1 * (int64_t)costs[k] - p[cols[k]];
            if (cp < mn) mn = cp;
        }
        const int64_t c = sp_arc(row_ptr, cols, costs, x, match[x]);
        if (c >= OR_INF) return 12;
        if (np1 * c - p[match[x]] > mn + eps) return 15;
    }
    return OR_OK;
}

/* ================================================================== */
/* Maximum s-t flow (Sect. 4, the paper's first problem).              */
/*                                                                     */
/* A directed graph on nodes 0..nn-1 given by its arcs (tail, head,    */
/* capacity >= 0); parallel and opposite arcs allowed. The maximum     */
/* flow value from s to t, and a minimum cut: the nodes still reachable */
/* from s in the final residual graph (by the max-flow min-cut theorem  */
/* the arcs leaving that set carry exactly the flow value).            */
/* ================================================================== */

/* Brute force over every s-t cut (nn <= 20): the minimum cut capacity,
 * which equals the maximum flow value. side_out[v] = 1 on the source side
 * of one minimum cut. */
int or_min_cut_brute(int32_t nn, int32_t na, const int32_t *tail, const int32_t *head,
                     const int64_t *cap, int32_t s, int32_t t, int64_t *value, uint8_t *side_out)
{
    if (nn < 2 || nn > 20 || s < 0 || t < 0 || s >= nn || t >= nn || s == t || !value) return OR_INVALID;
    for (int32_t a = 0; a < na; ++a)
        if (tail[a] < 0 || tail[a] >= nn || head[a] < 0 || head[a] >= nn || cap[a] < 0) return OR_INVALID;
    int64_t best = -1;
    uint32_t best_mask = 0;
    for (uint32_t mask = 0; mask < (1u << nn); ++mask) {
        if (!(mask >> s & 1u) || (mask >> t & 1u)) continue;      /* s inside, t outside */
        int64_t c = 0;
        for (int32_t a = 0; a < na; ++a)
            if ((mask >> tail[a] & 1u) && !(mask >> head[a] & 1u)) c += cap[a];
        if (best < 0 || c < best) { best = c; best_mask = mask; }
    }
    *value = best;
    if (side_out)
        for (int32_t v = 0; v < nn; ++v) side_out[v] = (uint8_t)(best_mask >> v & 1u);
    return OR_OK;
}

/* Dinic's algorithm (Dinic 1970): BFS levels from s in the residual graph,
 * then blocking flows along level-increasing arcs (iterative DFS with a
 * per-node arc pointer), until t is unreachable. Not from the paper: an
 * independent ground truth for its push-relabel method. */
int or_maxflow_dinic(int32_t nn, int32_t na, const int32_t *tail, const int32_t *head,
                     const int64_t *cap, int32_t s, int32_t t, int64_t *value, uint8_t *side_out)
{
    if (nn < 2 || s < 0 || t < 0 || s >= nn || t >= nn || s == t || na < 0 || !value) return OR_INVALID;
    for (int32_t a = 0; a < na; ++a)
        if (tail[a] < 0 || tail[a] >= nn || head[a] < 0 || head[a] >= nn || cap[a] < 0) return OR_INVALID;
    /* residual arcs 2a (forward) and 2a+1 (backward), adjacency in CSR */
    const int64_t m = 2 * (int64_t)na;
    int64_t *res = malloc(sizeof(int64_t) * (m > 0 ? m : 1));
    int32_t *to = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
    int32_t *start = calloc((size_t)nn + 1, sizeof(int32_t));
    int32_t *order = malloc(sizeof(int32_t) * (m > 0 ? m : 1));
    int32_t *level = malloc(sizeof(int32_t) * nn);
    int32_t *queue = malloc(sizeof(int32_t) * nn);
    int32_t *ptr = malloc(sizeof(int32_t) * nn);
    int32_t *stack_v = malloc(sizeof(int32_t) * nn);     /* DFS path: nodes */
    int32_t *stack_a = malloc(sizeof(int32_t) * nn);     /* DFS path: arcs into them */
    if (!res || !to || !start || !order || !level || !queue || !ptr || !stack_v || !stack_a) {
        free(res); free(to); free(start); free(order); free(level); free(queue); free(ptr);
        free(stack_v); free(stack_a);
        return OR_NOMEM;
    }
    for (int32_t a = 0; a < na; ++a) {
        res[2 * a] = cap[a];  to[2 * a] = head[a];
        res[2 * a + 1] = 0;   to[2 * a + 1] = tail[a];
        start[tail[a] + 1]++;
        start[head[a] + 1]++;
    }
    for (int32_t v = 0; v < nn; ++v) start[v + 1] += start[v];
    {
        int32_t *fill = malloc(sizeof(int32_t) * nn);
        if (!fill) { free(res); free(to); free(start); free(order); free(level); free(queue); free(ptr);
                     free(stack_v); free(stack_a); return OR_NOMEM; }
        for (int32_t v = 0; v < nn; ++v) fill[v] = start[v];
        for (int32_t a = 0; a < na; ++a) {
            order[fill[tail[a]]++] = 2 * a;
            order[fill[head[a]]++] = 2 * a + 1;
        }
        free(fill);
    }
    int64_t flow = 0;
    for (;;) {
        for (int32_t v = 0; v < nn; ++v) level[v] = -1;
        int32_t qh = 0, qt = 0;
        level[s] = 0;
        queue[qt++] = s;
        while (qh < qt) {
            const int32_t v = queue[qh++];
            for (int32_t k = start[v]; k < start[v + 1]; ++k) {
                const int32_t e = order[k];
                if (res[e] > 0 && level[to[e]] < 0) { level[to[e]] = level[v] + 1; queue[qt++] = to[e]; }
            }
        }
        if (level[t] < 0) break;
        for (int32_t v = 0; v < nn; ++v) ptr[v] = start[v];
        /* blocking flow: advance / retreat along level-increasing arcs */
        int32_t depth = 0;
        stack_v[0] = s;
        while (depth >= 0) {
            const int32_t v = stack_v[depth];
            if (v == t) {
                int64_t d = INT64_MAX;
                for (int32_t i = 1; i <= depth; ++i) if (res[stack_a[i]] < d) d = res[stack_a[i]];
                for (int32_t i = 1; i <= depth; ++i) { res[stack_a[i]] -= d; res[stack_a[i] ^ 1] += d; }
                flow += d;
                depth = 0;                 /* restart from s; saturated arcs are skipped below */
                continue;
            }
            int advanced = 0;
            for (; ptr[v] < start[v + 1]; ++ptr[v]) {
                const int32_t e = order[ptr[v]];
                const int32_t w = to[e];
                if (res[e] > 0 && level[w] == level[v] + 1) {
                    stack_v[++depth] = w;
                    stack_a[depth] = e;
                    advanced = 1;
                    break;
                }
            }
            if (!advanced) {               /* dead end: v leaves the level graph */
                level[v] = -1;
                --depth;
                if (depth >= 0) ++ptr[stack_v[depth]];
            }
        }
    }
    *value = flow;
    if (side_out)                          /* reachable from s in the residual graph */
        for (int32_t v = 0; v < nn; ++v) side_out[v] = 0;
    if (side_out) {
        int32_t qh = 0, qt = 0;
        side_out[s] = 1;
        queue[qt++] = s;
        while (qh < qt) {
            const int32_t v = queue[qh++];
            for (int32_t k = start[v]; k < start[v + 1]; ++k) {
                const int32_t e = order[k];
                if (res[e] > 0 && !side_out[to[e]]) { side_out[to[e]] = 1; queue[qt++] = to[e]; }
            }
        }
    }
    free(res); free(to); free(start); free(order); free(level); free(queue); free(ptr);
    free(stack_v); free(stack_a);
    return OR_OK;
}

/* Capacity of the cut whose source side is side[v] = 1 (s inside, t outside). */
int or_cut_capacity(int32_t nn, int32_t na, const int32_t *tail, const int32_t *head, const int64_t *cap,
                    int32_t s, int32_t t, const uint8_t *side, int64_t *value)
{
    if (nn < 2 || !side || !value || s < 0 || t < 0 || s >= nn || t >= nn) return OR_INVALID;
    if (!side[s] || side[t]) return 17;
    int64_t c = 0;
    for (int32_t a = 0; a < na; ++a) {
        if (tail[a] < 0 || tail[a] >= nn || head[a] < 0 || head[a] >= nn) return OR_INVALID;
        if (side[tail[a]] && !side[head[a]]) c += cap[a];
    }
    *value = c;
    return OR_OK;
}
