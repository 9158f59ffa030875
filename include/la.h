/*
 * la.h -- C ABI of the GB300 dense assignment solver.
 *
 * Problem. Given an n x n int32 cost matrix C (row x = left vertex of X,
 * column y = right vertex of Y of a complete bipartite graph), find a perfect
 * matching M that minimises sum_x C[x][M(x)] (Sect. 3 of the paper defines
 * matchings, perfect matchings and the assignment problem; Sect. 5 reduces the
 * assignment problem to a min-cost flow with u(x,y) = 1, c(x,y) = w(x,y), and
 * this library solves that minimisation; a maximising caller passes
 * max_w - w or -w).
 *
 * Method. Cost scaling (Sect. 5.1, Algorithm 5.0's epsilon loop) on costs
 * scaled by n + 1, with a lock-free parallel refine (Sect. 5.3, Algorithm 5.4)
 * whose push/relabel step is taken as the Goldberg-Kennedy double push: a
 * free row x scans its row for the best and second-best part-reduced cost
 * c'_p(x,y) = (n+1) C[x][y] - p(y), takes the best column w and lowers p(w)
 * by (second - best + eps), displacing w's previous mate. All arithmetic is
 * exact integer arithmetic, so the returned cost is the exact optimum.
 *
 * Conventions shared by every entry point:
 *  - Pointers named "device" must point to memory the current CUDA device can
 *    read or write (cudaMalloc, cudaMallocAsync, managed memory). They are
 *    owned by the caller; the library never frees them.
 *  - Matrices are row-major: C[x][y] is element x * n + y.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is ordered on that stream.
 *  - The library keeps a per-device workspace (allocated on first use and
 *    grown on demand, freed by la_release_workspace or at exit). Calls from
 *    several host threads are serialised by an internal lock.
 *  - Argument errors return LA_ERR_INVALID before anything is enqueued.
 *  - The la_solve* calls block the calling host thread until the result is
 *    in place (they read a few scalars back from the device), so outputs are
 *    valid when the call returns LA_OK.
 */
#ifndef LA_H
#define LA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LA_OK = 0,
    LA_ERR_INVALID = 1,     /* bad argument (n < 0, NULL pointer, n > LA_MAX_N) */
    LA_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    LA_ERR_OVERFLOW = 3,    /* cost range too large for the exact integer
                               price field: (n+1)(max C - min C) >= 2^40 */
    LA_ERR_ITER_LIMIT = 4,  /* the row-scan budget ran out before the
                               refine finished (see la_options.scan_budget) */
    LA_ERR_NOMEM = 5,       /* device workspace allocation failed */
    LA_ERR_INTERNAL = 6,    /* a device-side consistency check failed */
    LA_ERR_TOO_LARGE = 7,   /* n exceeds a fixed scratch size
                               (la_solve_noalloc: LA_NOALLOC_MAX_N) */
    LA_ERR_INFEASIBLE = 8   /* la_solve_sparse: the graph has no perfect
                               matching */
} la_status;

/* Largest n accepted by the solver (the mate field of a column key is 20
 * bits wide, with one value reserved for "no mate"). */
#define LA_MAX_N ((1 << 20) - 1)

/* Options for la_solve_ex. Zero-initialise and set what you need. */
typedef struct {
    /* Divisor of eps between refine phases (Algorithm 5.0; the paper uses
       alpha = 10). 0 selects 10. Must be >= 2 otherwise. */
    int32_t alpha;
    /* Starting eps. 0 selects C~ = (n+1)(max C - min C) (Algorithm 5.0
       starts at the largest cost). The first phase runs at
       max(1, eps0 / alpha); the last phase always runs at eps = 1. */
    int64_t eps0;
    /* Device int64[n] or NULL: starting column prices, in the paper's sign
       (c_p(x,y) = c(x,y) + p(x) - p(y)) and in units of the scaled costs
       (n+1) C. NULL starts from p = 0 (Algorithm 5.0). Any values give the
       same optimal cost; good ones need fewer row scans. */
    const int64_t *init_prices;
    /* Device int64[n] or NULL: receives the final column prices in the same
       units and sign, shifted so that max_y p(y) = 0. With them every row
       satisfies (n+1)C[x][M(x)] - p(M(x)) <= min_y((n+1)C[x][y] - p(y)) + 1. */
    int64_t *prices_out;
    /* Maximum number of row scans over the whole solve; 0 selects
       256 * n * phases + 2^22. Exhausting it returns LA_ERR_ITER_LIMIT with
       the matching and cost unspecified; prices_out then holds the prices
       reached, to resume from (see la_stats.stop_eps). */
    int64_t scan_budget;
    /* Nonzero: record CUDA events around every refine launch and report
       their summed duration in la_stats.refine_ms. */
    int32_t profile;
    /* Tuning: threads per block of the refine kernel (0 = default 256). */
    int32_t block_threads;
    /* Bit set of LA_FLAG_* values (0 = defaults). */
    int32_t flags;
    /* When a phase is down to this many free rows, the refine hands them to
       a one-CTA kernel that finishes the phase with the column keys in
       shared memory (n <= 16384). 0 selects 32; negative disables it. If the
       candidate lists stop answering there (more than a quarter of its scans,
       after 64, read whole rows), the rows go back to a refine launch over
       the whole grid. */
    int32_t tail_threshold;
    /* Global price updates (Sect. 5.2, Algorithm 5.3) per phase, each run
       when the phase is down to max(16, n/128) free rows after a stretch of
       bidding. 0 or negative: none (the default; on the measured workloads
       their sweeps cost about what they save). */
    int32_t price_updates;
    /* Intermediate phases (all but the last, eps = 1) stop once this many
       rows or fewer are free; 0 or a negative value runs every phase to a
       complete assignment (Algorithm 5.2 as written; the default). Only the
       last phase must end with an eps-optimal flow: the next phase's
       initialisation makes any prices eps-optimal, so the optimum is
       unchanged. Large values make the next phase pay for the unresolved
       conflicts (small eps, long price wars); keep it small. */
    int32_t phase_cutoff;
    /* Free rows at which the team refine takes a phase over (see
       LA_FLAG_NO_TEAM_REFINE); 0 means 2 per SM, capped at n / 2. */
    int32_t team_threshold;
    /* Global price updates (Sect. 5.2, Algorithm 5.3) the one-CTA tail
       kernel may stop for in each phase, after 2n row scans of its own each;
       0 (the default) or negative: none. */
    int32_t tail_updates;
    /* alpha for the phases that start from eps <= 16 (n + 1), sixteen cost
       units (the eps steps near and below a cost unit, where bids fight over
       equal costs); 0 (the default): alpha throughout. */
    int32_t alpha_fine;
} la_options;

/* la_options.flags: scan every row in full on every bid instead of using
   the exact candidate lists (for measurement and testing). */
#define LA_FLAG_NO_CANDIDATE_LISTS 1
/* la_options.flags, a debug mode: at the end of every phase a device pass
   over C checks the invariants of the refine (Sect. 5.1-5.2): every column
   has a holder and no row holds two (a perfect assignment; with a phase
   cutoff, only at the last phase), every holder x of a column y is
   eps-optimal for the phase's eps (version-2 eps-CS on costs scaled by n+1:
   c~(x,y) - p(y) <= min_z (c~(x,z) - p(z)) + eps), and no column's price
   rose during the phase (Lemma 5.2). Violations are counted in
   la_stats.check_violations and make the solve return LA_ERR_INTERNAL. */
#define LA_FLAG_CHECK_PHASES 2
/* la_options.flags: no arc fixing. By default, after every phase but the
   last, arc fixing (Sect. 5.2) drops every arc (x,y) whose reduced cost
   c_p(x,y) = c~(x,y) + p(x) - p(y), with the row price of Algorithm 5.2,
   exceeds 2 n eps: such an arc keeps its zero flow in every later phase, so
   no optimal assignment uses it (an alternating cycle through it would
   have negative cost in the optimum's residual graph). A row whose
   remaining arcs fit in its candidate list (128 columns) keeps only those
   and is never scanned in full again. The optimal cost is unchanged; the
   final prices certify optimality only over the arcs kept, so arc fixing
   is off whenever prices_out is requested, and with a phase cutoff (whose
   intermediate phases do not end with an eps-optimal flow). With
   LA_FLAG_CHECK_PHASES the eps-CS check of a fixed row covers its kept
   arcs. */
#define LA_FLAG_NO_ARC_FIXING 4
/* la_options.flags: solve small instances through the general path as well.
   By default an instance with n <= 300 and max C - min C <= 65535 (16-bit
   costs), or n <= 224 (32-bit), is solved by one CTA with the whole matrix
   and the column keys in shared memory, every phase in one launch (no
   candidate lists, tail kernel, arc fixing or sweep launch: each bid scans
   its row from shared memory). LA_FLAG_CHECK_PHASES, a phase cutoff and
   price updates also select the general path. */
#define LA_FLAG_NO_SMALL_KERNEL 8
/* la_options.flags: when the one-CTA tail kernel takes a phase over, it
   first runs one global price update (Sect. 5.2, Algorithm 5.3) on its own
   CTA: the labels of la_options.price_updates' grid update, computed with
   the labels in shared memory and CTA barriers between sweeps. */
#define LA_FLAG_TAIL_PRICE_UPDATE 16
/* la_options.flags: by default, once at most 2 rows per SM are free (and
   candidate lists are on), a phase is carried on by one CTA of 8 warps per
   free row, its warps sharing each full row scan (best and second best,
   Sect. 5.3, and the row's candidate list), then by the tail kernel as
   usual. This flag keeps one warp per row throughout. The optimum is the
   same either way. */
#define LA_FLAG_NO_TEAM_REFINE 32

/* Phases whose counters la_stats records one by one. */
#define LA_STATS_PHASES 32

/* Counters of one solve (filled by la_solve_ex when stats_out != NULL). */
typedef struct {
    int64_t n;
    int64_t phases;          /* refine phases run */
    int64_t scans;           /* row scans (one per double push attempt) */
    int64_t wins;            /* successful double pushes */
    int64_t displaced;       /* wins that displaced a previous mate */
    int64_t eps_first;       /* eps of the first phase */
    int64_t scaled_range;    /* C~ = (n+1)(max C - min C) */
    int32_t wide;            /* 1 if the 64-bit reduced-cost path ran */
    int32_t vector_loads;    /* 1 if the 128-bit row-load path ran */
    int64_t launches;        /* kernels this call launched */
    int64_t refine_launches; /* of which refine kernels */
    double refine_ms;        /* summed time of each phase's refine, price-update
                                and tail kernels (profile != 0) */
    int64_t max_chain;       /* most row scans one warp made within a phase
                                (the length of the longest displacement chain
                                plus lost bids: the refine's critical path) */
    int64_t phase_scans[LA_STATS_PHASES];  /* row scans of each phase */
    double phase_ms[LA_STATS_PHASES];      /* refine time of each phase
                                              (profile != 0) */
    int64_t full_scans;      /* scans that read the whole cost row */
    int64_t list_scans;      /* scans answered exactly by the row's candidate
                                list (128 columns) without reading the row */
    int64_t tail_scans;      /* scans made by the one-CTA tail kernel */
    int32_t tail_phases;     /* phases that handed their last rows to it */
    int64_t price_updates;   /* global price updates applied */
    int64_t price_update_sweeps;  /* relaxation sweeps they took */
    int64_t price_update_levels;  /* sum of their truncation levels */
    int32_t list_entries;    /* candidate-list entries per row (0: lists off) */
    double tail_ms;          /* of refine_ms, the time from the end of each
                                phase's refine kernel to the end of its
                                one-CTA tail kernel (profile != 0) */
    int64_t tail_full_scans; /* of tail_scans, those that read the whole row */
    int32_t tail_giveups;    /* phases whose tail kernel handed its rows back to
                                the grid (its lists stopped answering) */
    int32_t checked_phases;  /* LA_FLAG_CHECK_PHASES: phases checked */
    int64_t check_violations; /* LA_FLAG_CHECK_PHASES: failed checks (0 = all held) */
    /* After a non-OK status: the phase it stopped in and that phase's eps
       (-1 and 0 after a success). A solve stopped by its scan budget can be
       resumed: pass the prices it wrote to opt->prices_out (written whenever
       the phases ran, LA_ERR_ITER_LIMIT included) as opt->init_prices, and
       stop_eps * alpha as opt->eps0, so that the resumed solve starts at the
       phase that did not finish; any start prices give the exact optimum. */
    int32_t stop_phase;
    int64_t stop_eps;
    /* Per phase (profile != 0 for the times): the one-CTA tail kernel's
       share of phase_ms, and the phase's full row scans and tail scans. */
    double phase_tail_ms[LA_STATS_PHASES];
    int64_t phase_full_scans[LA_STATS_PHASES];
    int64_t phase_tail_scans[LA_STATS_PHASES];
    /* Arc fixing (Sect. 5.2; see LA_FLAG_NO_ARC_FIXING): rows whose arcs
       were cut down to their candidate list after each phase, and after the
       last fixing pass those rows and the arcs they keep. */
    int64_t phase_fixed_rows[LA_STATS_PHASES];
    int64_t fixed_rows;
    int64_t fixed_arcs;
    /* The bulk sweep that opens every phase (each row's first bid, all rows
       in flight; the displacement chains run in the launches after it): its
       summed time (profile != 0), row scans and full row scans. */
    double sweep_ms;
    int64_t sweep_scans;
    int64_t sweep_full_scans;
    /* 1 if the solve ran on the one-CTA shared-memory kernel for small
       instances (see LA_FLAG_NO_SMALL_KERNEL): every scan is a full scan of
       the row in shared memory, refine_ms is that launch's time. */
    int32_t small_kernel;
    /* Time the tail kernel spent in its own price updates
       (LA_FLAG_TAIL_PRICE_UPDATE), summed over phases, read from the GPU's
       global timer. */
    double tail_price_update_ms;
    /* Phases the team refine took over (see LA_FLAG_NO_TEAM_REFINE), its
       row scans and, of those, full row scans. */
    int32_t team_phases;
    int64_t team_scans;
    int64_t team_full_scans;
} la_stats;

/*
 * la_solve -- exact minimum-cost perfect matching of a dense n x n matrix:
 * the assignment problem of Sect. 3 (as minimisation, see above), solved by
 * the cost scaling of Sect. 5.1 (Algorithm 5.0's eps loop, Algorithm 5.2's
 * initialisation) with the lock-free refine of Sect. 5.3 (Algorithm 5.4).
 *   cost      device const int32[n*n], row-major, read only.
 *   n         0 <= n <= LA_MAX_N. n = 0 writes *cost_out = 0.
 *   stream    cudaStream_t as void*.
 *   match_out device int32[n] or NULL: match_out[x] = column matched to x.
 *   cost_out  device int64[1]: the optimal total cost sum_x C[x][match[x]].
 * Returns LA_OK, or an error code with outputs unspecified.
 */
la_status la_solve(const int32_t *cost, int32_t n, void *stream,
                   int32_t *match_out, int64_t *cost_out);

/* la_solve with options (opt may be NULL) and counters (stats_out may be
 * NULL; it is host memory). */
la_status la_solve_ex(const int32_t *cost, int32_t n, const la_options *opt,
                      void *stream, int32_t *match_out, int64_t *cost_out,
                      la_stats *stats_out);

/* Human-readable name of a status code (static storage). */
const char *la_status_string(la_status s);

/* Frees the calling device's workspace (the next solve reallocates it). */
la_status la_release_workspace(void);

/*
 * la_debug_price_update -- one global price update (Sect. 5.2, Algorithm
 * 5.3) on a mid-phase state given by the caller: a test hook for the update
 * the refine runs with la_options.price_updates, through the same kernel.
 * The state is a phase at scale eps: column prices, a partial matching in
 * which every matched row x is eps-optimal in the version-2 sense of Sect.
 * 5.1 ((n+1)C[x][M(x)] - p(M(x)) <= min_y ((n+1)C[x][y] - p(y)) + eps), and
 * the free rows.
 *   cost        device const int32[n*n], row-major; 2 <= n <= LA_MAX_N.
 *   prices      device const int64[n]: p(y), the paper's sign, units of
 *               (n+1) C.
 *   row_match   device const int32[n]: the column of row x, or -1 if x is
 *               free; no column may appear twice (else LA_ERR_INVALID).
 *   eps         the phase's eps, >= 1.
 *   labels_out  device int32[n]: each column's label, its distance in
 *               units of eps to the nearest free column over the residual
 *               graph, truncated at one more than the largest label of a
 *               free row (Algorithm 5.3's last + 1), as applied.
 *   prices_out  device int64[n]: p(y) - eps * label(y).
 * Each row's arcs are those of its candidate list built at the given
 * prices (the best 4 columns of each of the 32 lanes; all n columns when
 * n <= 128); a matched row's label is capped by the bound on its unlisted
 * columns, which keeps it eps-optimal over every arc. For n <= 128 the
 * labels are therefore the exact truncated distances.
 *   kernel      0: the grid update of la_options.price_updates; 1: the
 *               one-CTA update of LA_FLAG_TAIL_PRICE_UPDATE (labels and
 *               keys in shared memory; n <= 16384, else LA_ERR_INVALID).
 *               Both compute the same labels. Any other value is
 *               LA_ERR_INVALID.
 * Uses the per-device workspace. Blocks until done.
 */
la_status la_debug_price_update(const int32_t *cost, int32_t n, const int64_t *prices, const int32_t *row_match,
                                int64_t eps, void *stream, int32_t *labels_out, int64_t *prices_out,
                                int32_t kernel);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t la_version(void);

/*
 * Batched solves. B independent instances packed back to back; instance i
 * is the n_i x n_i row-major matrix at cost + offsets[i]. One persistent
 * launch (replayed from a CUDA graph) solves them all: each CTA claims
 * instances from a device work queue, largest first, and runs the complete
 * cost-scaling solve of one instance (Sect. 5.1, Algorithm 5.0's epsilon
 * loop with the refine of Algorithms 5.2 and 5.4, costs scaled by n_i + 1)
 * with that instance's column keys in shared memory.
 *   cost       device const int32, all instances.
 *   offsets    device const int64[B]: element offset of each instance.
 *   ns         device const int32[B]: 0 <= n_i <= max_n (see options).
 *   match_out  device int32[sum n_i] or NULL: instance i's matching (row ->
 *              column, 0-based within the instance) at the exclusive prefix
 *              sum of n_0 .. n_{i-1}.
 *   cost_out   device int64[B]: exact optimal cost of each instance.
 *   status_out device int32[B] or NULL: la_status of each instance.
 * Returns LA_OK when every instance succeeded, else the status of one that
 * failed (instances are independent: the others are still solved). Blocks
 * until the results are in place.
 */
#define LA_ALPHA_BUCKETS 16   /* alpha by size: bucket k holds 2^k <= n < 2^(k+1) */
#define LA_BATCH_MAX_N 8192   /* largest instance of a batched solve */

typedef struct {
    /* Threads per CTA (64, 128, 256, 512 or 1024; 0 selects 512): the warps
       that share the CTA's resident instances (see slots). */
    int32_t block_threads;
    /* Largest n the launch must hold in shared memory (0 = LA_BATCH_MAX_N);
       smaller values let more CTAs share an SM. Instances with n > max_n
       fail with LA_ERR_INVALID. */
    int32_t max_n;
    /* alpha for each size bucket (0 = 10). */
    int32_t alpha[LA_ALPHA_BUCKETS];
    /* Row scans per row and phase before LA_ERR_ITER_LIMIT (0 = 256): an
       instance may make budget_factor * n_i * phases + 4096 row scans. */
    int32_t budget_factor;
    /* Nonzero: launch directly instead of capturing and replaying a CUDA
       graph (a graph is captured once per distinct argument set). */
    int32_t no_graph;
    /* Nonzero: time the launch with CUDA events (la_batch_stats.device_ms). */
    int32_t profile;
    /* Device int64[sum n_i] or NULL: final column prices of every instance,
       packed like match_out (paper sign, units of (n_i+1) C, up to a
       constant per instance). */
    int64_t *prices_out;
    /* Instances resident per CTA (1..8, 0 selects 4; fewer when their keys,
       8 max_n bytes each, would exceed 192 KB of shared memory). The CTA's
       warps take free rows from any resident instance. */
    int32_t slots;
    /* Candidate lists (the exact lazy scans of la_solve) for the rows of
       every instance: > 0 on, < 0 off, 0 on when max_n >= 2048 and lists for
       B * max_n rows (1032 bytes each) fit in 4 GB. They cut the bytes of
       most row scans of large instances from 4 n to 1032. */
    int32_t lists;
} la_batch_options;

typedef struct {
    int64_t instances;
    int64_t failed;
    int64_t scans;          /* row scans over all instances */
    int64_t scan_bytes;     /* bytes those scans read: 4 n_i per full scan, 1032 per list scan */
    int64_t wins;
    int64_t displaced;
    int64_t phases;         /* refine phases over all instances */
    int32_t max_n;          /* largest n seen */
    int32_t grid;           /* persistent CTAs launched */
    int32_t block_threads;
    int32_t graph;          /* 1 if the launch was a CUDA graph replay */
    double device_ms;       /* launch time (profile != 0) */
    int32_t slots;          /* instances resident per CTA */
    int32_t lists;          /* candidate lists used */
    int64_t full_scans;     /* scans that read the whole row (all of them without lists) */
} la_batch_stats;

la_status la_solve_batched(const int32_t *cost, const int64_t *offsets, const int32_t *ns,
                           int32_t B, void *stream, int32_t *match_out, int64_t *cost_out);

la_status la_solve_batched_ex(const int32_t *cost, const int64_t *offsets, const int32_t *ns,
                              int32_t B, const la_batch_options *opt, void *stream,
                              int32_t *match_out, int64_t *cost_out, int32_t *status_out,
                              la_batch_stats *stats_out);

/*
 * la_dual_certificate -- exact integer LP duals of an optimal assignment.
 * Given a perfect matching M (device int32[n], row -> column), returns the
 * duals tight on M: v (device int64[n], cost units) is the largest
 * potential with v <= 0 and v(y) <= v(M(x)) + C[x][y] - C[x][M(x)] for all
 * x, y (shortest paths, Bellman-Ford sweeps over the columns), and u
 * (device int64[n] or NULL) is u(x) = C[x][M(x)] - v(M(x)). Then
 * u(x) + v(y) <= C[x][y] everywhere, equality holds on M and
 * sum u + sum v = cost(M), which proves M optimal (LP duality). These are
 * the paper's prices at eps = 0 (c_p(x,y) = c(x,y) + p(x) - p(y) >= 0 with
 * p(y) = v(y), p(x) = -u(x); Sect. 3, eps-optimality).
 * Returns LA_ERR_INVALID if M is not a permutation and LA_ERR_INTERNAL if
 * M is not optimal (no such duals exist). Blocks until done.
 */
la_status la_dual_certificate(const int32_t *cost, int32_t n, const int32_t *match, void *stream,
                              int64_t *u_out, int64_t *v_out);

/*
 * Learned warm start. Refine's initialisation makes any price vector
 * eps-optimal (Sect. 5.2, Algorithm 5.2), so a solve may start from
 * predicted column prices and a small eps0 instead of p = 0 and eps0 = C~
 * (Algorithm 5.0) and still returns the exact optimum. A set encoder
 * predicts the optimal column duals from per-column cost statistics:
 *   f_j   8 features of column j (LA_PRED_FEATURES, padded to 16): column
 *         minimum and gap to the second minimum, the same on the row-reduced
 *         matrix C - rowmin, the number of rows whose minimum is in column j,
 *         the column mean, log T and log n (location features centred and
 *         divided by T = 1 + mean column gap);
 *   h1_j  = relu(W1^T f_j + b1), c = mean_j h1_j,
 *   h2_j  = relu(W2^T [h1_j ; c] + b2), y_j = W3^T h2_j + b3 (width 128),
 *   p(j)  = round((n+1) T (y_j - max y)).
 * Matrix products run on the tensor cores with BF16 operands and FP32
 * accumulation. The weights are one device float array of LA_PRED_PARAMS
 * entries: a 16-float header (LA_PRED_MAGIC, version 1, 16, 128, then the
 * calibrated eps0 factor q: eps0 = ceil((n+1) T q)), followed by W1 [16x128],
 * b1 [128], W2 [256x128], b2 [128], W3 [128x8] (column 0 used), b3 [8].
 */
#define LA_PRED_FEATURES 8
#define LA_PRED_FEATURES_PADDED 16
#define LA_PRED_WIDTH 128
#define LA_PRED_HEADER 16
#define LA_PRED_PARAMS 36120
#define LA_PRED_MAGIC 4242.0f

/* Number of floats in a weight array (LA_PRED_PARAMS). */
int32_t la_predictor_param_count(void);

/* Column features of one n x n matrix: feats_out device float[n][16],
 * inst_out device float[2] or NULL: (T, mean column minimum). */
la_status la_features(const int32_t *cost, int32_t n, void *stream, float *feats_out,
                      float *inst_out);

/* Forward pass over N feature rows forming I instances (seg: device
 * int32[I+1] row offsets): y_out device float[N]. */
la_status la_predictor_forward(const float *params, const float *feats, const int32_t *seg,
                               int32_t I, int32_t N, void *stream, float *y_out);

/* One training step: forward, loss
 *   L = (1/I) sum_i (1/n_i) sum_j (d_j - mean_i d)^2,  d = y - t
 * (targets t: device float[N]; the loss ignores a per-instance shift of y or
 * t, as prices do), backward, and an Adam
 * update of params with moments adam_m / adam_v (device float[LA_PRED_PARAMS],
 * zero at step 1; lr <= 0 or NULL moments skip the update). grad_out (device
 * float[LA_PRED_PARAMS] or NULL) receives dL/dparams; loss_out (host) the loss. */
la_status la_predictor_train_step(float *params, float *adam_m, float *adam_v, const float *feats,
                                  const float *targets, const int32_t *seg, int32_t I, int32_t N,
                                  int32_t step, float lr, float weight_decay, void *stream,
                                  float *grad_out, float *loss_out);

/* Predicted column prices of one matrix (device int64[n], paper sign, units of
 * the scaled costs (n+1) C, max = 0). weights: device float[LA_PRED_PARAMS];
 * a bad header returns LA_ERR_INVALID. _ex also returns the calibrated eps0
 * (host int64). */
la_status la_predict_prices(const int32_t *cost, int32_t n, const void *weights, void *stream,
                            int64_t *prices_out);
la_status la_predict_prices_ex(const int32_t *cost, int32_t n, const void *weights, void *stream,
                               int64_t *prices_out, int64_t *eps0_out);

/* Warm-started exact solve: la_predict_prices_ex, then la_solve_ex from the
 * predicted prices and eps0, with alpha = 4 for n >= 4096 and the default
 * alpha (10) below: from predicted prices the smaller eps steps measured
 * faster on large instances. Same results as la_solve. */
la_status la_solve_warm(const int32_t *cost, int32_t n, const void *weights, void *stream,
                        int32_t *match_out, int64_t *cost_out, la_stats *stats_out);

/*
 * la_solve_sparse -- exact minimum-cost perfect matching of a sparse
 * bipartite graph. The paper's implementation takes arbitrary bipartite
 * graphs (Sect. 1 and Sect. 6), and Sect. 5 reduces the assignment problem
 * to a min-cost flow on the graph's arcs (u(x,y) = 1, c(x,y) = w(x,y)); the
 * method is the same cost scaling as la_solve (Algorithm 5.0's eps loop on
 * costs scaled by n + 1, Algorithm 5.2's initialisation, Algorithm 5.4's
 * push/relabel as a double push), each free row scanning only its own arcs.
 *   row_ptr   device const int32[n+1]: row x's arcs are k = row_ptr[x] ..
 *             row_ptr[x+1] - 1; row_ptr[0] = 0, row_ptr[n] = nnz,
 *             non-decreasing.
 *   cols      device const int32[nnz]: column of arc k, 0 <= cols[k] < n.
 *             Order within a row is free; a row may list a column twice
 *             (the cheaper arc is the one a matching uses).
 *   costs     device const int32[nnz]: cost of arc k.
 *   n, nnz    0 <= n <= LA_MAX_N, 0 <= nnz < 2^31.
 *   match_out device int32[n] or NULL: match_out[x] = column of x's arc in
 *             the matching.
 *   cost_out  device int64[1]: the optimal total cost.
 * Returns LA_OK; LA_ERR_INVALID for malformed CSR arrays (checked on the
 * device before any solving); LA_ERR_INFEASIBLE when no perfect matching
 * exists (a row or column without arcs, or a price drop in a first refine
 * phase on zero costs beyond what a feasible graph allows: 4n + 4, against
 * the bound (2n - 1) eps of cost scaling); else as la_solve. Blocks until
 * the result is in place. Uses the same la_options / la_stats as
 * la_solve_ex: alpha, eps0, prices_out, scan_budget (0 = 256 n (phases + 1)
 * + 2^22) and profile are honoured; init_prices must be NULL. phase_scans[0]
 * counts the feasibility phase.
 */
la_status la_solve_sparse(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs,
                          int32_t n, int32_t nnz, void *stream, int32_t *match_out,
                          int64_t *cost_out);
la_status la_solve_sparse_ex(const int32_t *row_ptr, const int32_t *cols, const int32_t *costs,
                             int32_t n, int32_t nnz, const la_options *opt, void *stream,
                             int32_t *match_out, int64_t *cost_out, la_stats *stats_out);

/*
 * la_maxflow_grid -- maximum s-t flow and a minimum cut of a 4-connected
 * H x W grid graph with terminal arcs (the graph-cut form of the paper's
 * Sect. 4 problem), by Hong's lock-free push-relabel (Algorithm 4.5) run in
 * cycles with a global relabel between them (Algorithm 4.8, plus the gap
 * step of the paper's implementation), all on the device.
 *   cap      device const int32[4][H][W]: cap[d][i][j] is the capacity of
 *            the arc from pixel (i, j) to its neighbour in direction d
 *            (0: (i, j+1), 1: (i, j-1), 2: (i+1, j), 3: (i-1, j)); arcs that
 *            would leave the grid must be 0.
 *   src, snk device const int32[H][W]: capacities s -> (i, j), (i, j) -> t.
 *            Every capacity is in [0, 2^30 - 1].
 *   flow_out device int64[1]: the maximum flow value.
 *   cut_out  device uint8[H][W] or NULL: 1 for the pixels on the source side
 *            of a minimum cut (those that cannot reach t in the final
 *            residual graph), 0 for the others; the capacity of the arcs
 *            from the source side to the sink side equals the flow value.
 * Returns LA_OK; LA_ERR_INVALID for bad sizes or capacities (checked on the
 * device before any push); LA_ERR_ITER_LIMIT after max_rounds cycles.
 * Blocks until the result is in place. H * W < 2^30.
 */
typedef struct {
    int32_t cycle;        /* push-relabel passes per launch between two
                             global relabels (the paper's CYCLE); 0 = adaptive:
                             32 at first, doubled (up to 4096) after every
                             round that leaves more than half of the active
                             nodes active */
    int32_t max_rounds;   /* cycles before LA_ERR_ITER_LIMIT; 0 = 65536 */
} la_maxflow_options;

typedef struct {
    int64_t flow;             /* the maximum flow value */
    int64_t excess_total;     /* sum of the source arcs' capacities */
    int64_t rounds;           /* push-relabel launches */
    int64_t global_relabels;
    int64_t relabel_sweeps;   /* tiled relaxation passes over the grid they took */
    int64_t launches;         /* kernels launched */
} la_maxflow_stats;

la_status la_maxflow_grid(const int32_t *cap, const int32_t *src, const int32_t *snk,
                          int32_t H, int32_t W, void *stream, int64_t *flow_out,
                          uint8_t *cut_out);
la_status la_maxflow_grid_ex(const int32_t *cap, const int32_t *src, const int32_t *snk,
                             int32_t H, int32_t W, const la_maxflow_options *opt,
                             void *stream, int64_t *flow_out, uint8_t *cut_out,
                             la_maxflow_stats *stats_out);

/*
 * la_solve_noalloc -- la_solve for callers that must not allocate memory.
 *
 * The paper has no counterpart: this entry point exists for deployments
 * that cannot let a library call cudaMalloc, for example a process whose
 * device memory is already claimed in full by another allocator (a
 * framework's caching pool), a real-time loop that cannot afford the
 * latency and implicit device synchronisation of an allocation, or a
 * certified system that forbids dynamic allocation after start-up.
 *
 * Same arguments, exact optimal cost and blocking behaviour as la_solve
 * (every call returns only once its result is in place), but not the same
 * configuration: it runs the refine without candidate lists and without the
 * one-CTA tail kernel, so every bid reads its whole cost row (a full row
 * scan) in every phase, at alpha = 10 from zero prices. That is la_solve_ex
 * with LA_FLAG_NO_CANDIDATE_LISTS and tail_threshold = -1; its speed, and the
 * default scan budget at which it returns LA_ERR_ITER_LIMIT, are that
 * configuration's. Instead of the per-device workspace it uses one fixed
 * scratch array that the library declares in device memory: 16 bytes per
 * column for LA_NOALLOC_MAX_N columns (the column keys and the price mirror)
 * plus a control block, about 257 KB in all. Every GPU that loads the
 * library holds that array until the process exits. The call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *   - n must be <= LA_NOALLOC_MAX_N; larger n returns LA_ERR_TOO_LARGE with
 *     nothing enqueued.
 *   - CUDA loads the array, and each kernel, on a device when they are first
 *     used there (lazy module loading), which takes a little device memory
 *     once. A caller whose device memory will later be claimed in full by
 *     another allocator should therefore make a first call at start-up, on
 *     an instance of the kind it will solve, or run with
 *     CUDA_MODULE_LOADING=EAGER.
 *   - The first call on a device also looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture on that device.
 *   - All calls on a device share the one array, which keeps the last
 *     call's contents; each call re-initialises what must start clean.
 *     Calls whose GPU work overlaps race on the array. A call waits for its
 *     own GPU work before it returns and calls from different host threads
 *     are serialised, so overlap can only follow a call that returned
 *     LA_ERR_CUDA with work still queued: synchronise that stream before
 *     the next call. (Each process has its own copy of the array.)
 */
#define LA_NOALLOC_MAX_N 16384
la_status la_solve_noalloc(const int32_t *cost, int32_t n, void *stream,
                           int32_t *match_out, int64_t *cost_out);

/*
 * la_probe_read -- read-bandwidth probe (a measurement utility; no solve
 * uses it). It supplies the measured peak of the cache level a scan's data
 * comes from: a 64 MiB cost matrix (n = 4096) stays in the 129 MB L2 across
 * the phases of a solve, so the refine's arc-scan rate is compared with the
 * L2 read rate, which no vendor figure states.
 *   buf    device buffer of `bytes` bytes, 16-byte aligned; read only.
 *   bytes  a multiple of 16, > 0.
 *   reps   passes over the buffer in one launch (>= 1); every thread of a
 *          grid-stride kernel (4 CTAs of 512 threads per SM) reads the same
 *          addresses in every pass with 128-bit loads cached at L2 only
 *          (.cg), so passes after the first hit L2 whenever the buffer fits.
 *   stream a cudaStream_t (NULL: the legacy default stream).
 *   ms_out host float: the launch's duration by CUDA events on `stream`.
 * The achieved rate is bytes * reps / time. Blocks until done (it
 * synchronises on its events). Returns LA_ERR_INVALID on a bad argument
 * (nothing enqueued) and LA_ERR_CUDA on a CUDA error.
 */
la_status la_probe_read(const void *buf, size_t bytes, int32_t reps, void *stream, float *ms_out);

#ifdef __cplusplus
}
#endif

#endif /* LA_H */
