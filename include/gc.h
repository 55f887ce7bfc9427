/*
 * gc.h - C ABI of libgc, GB300-native speculative First-Fit graph colouring.
 *
 * Method: Rokos, Gorman, Kelly, "A Fast and Scalable Graph Coloring
 * Algorithm for Multi-core and Many-core Architectures", arXiv 1505.04086.
 *   - Problem (Sec. 2.1, Algorithm 1): given an undirected graph G(V,E),
 *     assign every vertex the smallest colour not used by its coloured
 *     neighbours; colours are 1..d+1 for maximum degree d.
 *   - GC_ALG_RSOC (Sec. 3, Algorithm 3): round 0 colours all of V
 *     tentatively; every later round inspects the vertices recoloured in the
 *     round before, recolours at once those still in conflict and collects
 *     them for the next round (one barrier per round).
 *   - GC_ALG_TWO_PHASE (Sec. 2.2, Algorithm 2): tentative colouring of the
 *     worklist, barrier, separate conflict detection, barrier.
 *
 * Graph format (all entry points): symmetric CSR, int32 row pointers
 * (n+1 entries, row_ptr[0] == 0, row_ptr[n] == nnz) and int32 column indices
 * (nnz entries).  Rows sorted strictly ascending; no self-loops; every entry
 * (v,u) has its mirror (u,v).  nnz counts directed entries (2|E|).
 * GC_VALIDATE checks all of this on the device; without it a malformed
 * graph gives an unspecified (but memory-safe for in-range indices)
 * colouring.
 *
 * Colours: int32, 1-based, in 1..deg(v)+1 on success (1..|D2(v)|+1 with
 * GC_DIST2); 0 is "uncoloured" and never appears in a successful result.
 *
 * Ownership: the caller owns every array it passes; the library never
 * frees or keeps them past the call (the server copies what it needs).
 * Errors are returned as negative status codes; nothing throws across the
 * ABI.  A gc_ctx is not thread-safe; use one per host thread.  The server
 * entry points are thread-safe.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
    GC_OK = 0,
    GC_PENDING = 1,              /* server: request not finished yet */
    GC_ERR_ARG = -1,             /* bad argument (null pointer, size, flag) */
    GC_ERR_GRAPH = -2,           /* GC_VALIDATE found a malformed CSR */
    GC_ERR_OOM = -3,             /* device or host allocation failed */
    GC_ERR_BUDGET = -4,          /* server: request larger than the budget */
    GC_ERR_NO_CONVERGENCE = -5,  /* round cap reached with conflicts left */
    GC_ERR_TIMEOUT = -6,         /* a bounded device wait gave up */
    GC_ERR_CUDA = -7,            /* a CUDA runtime call failed */
    GC_ERR_OVERFLOW = -8,        /* internal worklist capacity exceeded */
    GC_ERR_CHECK = -9,           /* GC_CHECKED found an invalid colouring */
    GC_ERR_NOT_FOUND = -10,      /* server: unknown ticket */
    GC_ERR_TOO_LARGE = -11       /* gc_color_noalloc: n > GC_NOALLOC_MAX_N */
};

/* ---- mode bits ------------------------------------------------------- */
enum {
    GC_ALG_RSOC = 0,             /* Algorithm 3 (default) */
    GC_ALG_TWO_PHASE = 1,        /* Algorithm 2 */
    GC_SCHED_DET = 0,            /* every read of a round sees the colours of
                                    the end of the previous round: results are
                                    deterministic (default) */
    GC_SCHED_ASYNC = 2,          /* colours are updated in place while other
                                    threads read them (the paper's form) */
    GC_TIE_LOWER_KEEPS = 0,      /* of two equal-coloured neighbours the
                                    higher id is recoloured (default) */
    GC_TIE_HIGHER_KEEPS = 4,     /* the lower id is recoloured, as the test
                                    "V_j > V_i" of Algorithms 2 and 3 reads */
    GC_VALIDATE = 8,             /* check the CSR on the device first */
    GC_CHECKED = 16,             /* verify the result on the device after */
    GC_DEBUG_NO_TIEBREAK = 32,   /* symmetric conflict test: both endpoints
                                    recolour (the Sec. 5 / Fig. 7 livelock);
                                    only meaningful with a small max_rounds */
    GC_NO_COLOR_STATS = 64,      /* skip the max/distinct colour reduction */
    GC_REPAIR_SNAPSHOT = 128,    /* with GC_SCHED_ASYNC and GC_ALG_RSOC: round 0
                                    runs in place, every later round reads the
                                    colours of the end of the round before
                                    (fewer colours on dense cores, more rounds) */
    GC_TIERS = 256,              /* with GC_SCHED_ASYNC and GC_ALG_RSOC: colour
                                    the vertices of degree > t2, then those of
                                    degree > t1, then the rest, each tier taken
                                    through round 0 and its repair rounds before
                                    the next (later tiers are uncoloured while
                                    an earlier one is repaired).  Close to
                                    largest-first order: on power-law graphs
                                    fewer colours than the plain asynchronous
                                    schedule (t2 defaults to 4096 here) */
    GC_FF_KEEPERS = 512,         /* with GC_SCHED_ASYNC, GC_ALG_RSOC and
                                    GC_TIE_LOWER_KEEPS only (else GC_ERR_ARG;
                                    not with GC_REPAIR_SNAPSHOT): a vertex's
                                    First-Fit choice, in round 0 and in every
                                    repair, avoids only the colours of its lower
                                    neighbours (those that keep their colour on
                                    a tie), as sequential First-Fit in id order
                                    sees them; a higher neighbour that then
                                    holds the chosen colour joins the next
                                    round's worklist.  Not the recolouring step
                                    of Algorithm 3 (which avoids every
                                    neighbour): colour counts stay close to
                                    sequential First-Fit under heavy
                                    concurrency.  conflicts counts those
                                    handed-on neighbours too. */
    GC_DIST2 = 1024              /* distance-2 colouring (Sec. 6 names it as the
                                    next target of the method): two vertices
                                    joined by a path of one or two edges get
                                    different colours, i.e. the colouring of
                                    G^2 without building it.  Algorithm 3 with
                                    "neighbour" read as "vertex of D2(v)" (the
                                    neighbours u of v and every w != v adjacent
                                    to such a u).  Single graph only
                                    (gc_color, gc_color_async, and the host
                                    form gc_host_color; GC_ERR_ARG in
                                    the batch, plan, server, no-alloc,
                                    recolour and autotune calls) and only with
                                    GC_ALG_RSOC, either schedule, either
                                    tie-break, GC_VALIDATE, GC_CHECKED (checks
                                    distance 2) and GC_NO_COLOR_STATS.
                                    GC_SCHED_DET: round 0 gives every vertex
                                    colour 1, then every round inspects U
                                    against the colours of the end of the
                                    round before (bit-exact replay).
                                    GC_SCHED_ASYNC: round 0 is First-Fit over
                                    D2(v) in place for every vertex, then
                                    rounds over U = V, L, ... in place.
                                    Colours lie in 1..|D2(v)|+1.  opts: only
                                    max_rounds, blocks_per_sm and d2_heavy
                                    apply. */
};

/* Every mode bit above. */
#define GC_MODE_MASK 2047u

/* ---- device error word bits (gc_stats.error_word) ---------------------- */
enum {
    GC_EW_TIMEOUT = 1,
    GC_EW_NO_CONVERGENCE = 2,
    GC_EW_OVERFLOW = 4,
    GC_EW_GRAPH = 8,
    GC_EW_CHECK = 16
};

typedef struct {
    const int32_t *row_ptr;      /* n+1 entries */
    const int32_t *col_idx;      /* nnz entries */
} gc_csr;

typedef struct {
    int32_t rounds;              /* while-loop iterations (the last one, which
                                    finds no conflict, included; RSOC's round 0
                                    not counted) */
    int32_t colors;              /* largest colour used (-1 if not computed) */
    int64_t conflicts;           /* sum over iterations of |L| */
    int32_t distinct_colors;     /* number of distinct colours (-1 if not computed) */
    int32_t error_word;          /* GC_EW_* bits raised on the device */
    int64_t model_bytes;         /* algorithmic bytes the executed rounds must
                                    move: per inspected vertex 8 for its row
                                    pointers, 4 for its worklist entry (not in
                                    a pass over all of V), 4 for its own colour
                                    (detection passes); 8 per adjacency entry
                                    read (index + colour): all entries for a
                                    (re)colouring, the tie side for a clean
                                    detection; 4 (index only) for a neighbour
                                    the asynchronous round 0 knows to be
                                    uncoloured (in a tile not yet claimed);
                                    in the first asynchronous repair of one
                                    graph, a thread-path vertex reads 8 for
                                    its round-0 mask and 8 per neighbour it
                                    read as uncoloured there; 4 per colour
                                    written and per worklist push;
                                    4 per vertex for a pass in which nothing
                                    is coloured yet.  GC_DIST2:
                                    per inspected vertex 4 (worklist entry,
                                    not in a pass over all of V) + 8 + 4 (own
                                    colour; not in the asynchronous round 0)
                                    + 16 per neighbour u (index, colour, two
                                    row pointers) + 8 per entry of u's row,
                                    + 4 + 4 when recoloured (+ 4 for the
                                    colour written in the asynchronous round
                                    0); the deterministic round 0 moves 4n */
    float elapsed_ms;            /* device time of the colouring kernel(s) */
    int32_t *round_sizes;        /* optional caller-owned HOST array; receives
                                    |L| of each iteration */
    int32_t round_sizes_cap;     /* its capacity (entries) */
    int64_t *round_ns;           /* optional caller-owned HOST array: [0] = ns
                                    from kernel start to the end of round 0
                                    (the prologue for deterministic runs),
                                    [k] = to the end of iteration k (device
                                    clock; first 255 iterations) */
    int32_t round_ns_cap;        /* its capacity (entries) */
} gc_stats;

/* Tuning knobs; zero-initialise for defaults. */
typedef struct {
    int32_t max_rounds;          /* iteration cap; 0 = n+1 */
    int32_t t1;                  /* degree <= t1: thread per vertex (<= 62); 0 = 32 */
    int32_t t2;                  /* t1 < degree <= t2: warp per vertex; above:
                                    block per vertex (<= 4096); 0 = 2048
                                    (4096 with GC_TIERS) */
    int32_t tile;                /* worklist entries a warp claims at once
                                    (multiple of 32, <= 4096); 0 = 64 */
    int32_t blocks_per_sm;       /* resident blocks per SM; 0 = occupancy max */
    int32_t tail;                /* once a worklist has at most this many
                                    vertices (and at most 16x as many adjacency
                                    entries) a single block finishes the
                                    colouring; 0 = 2048, -1 = never */
    int32_t window;              /* GC_SCHED_ASYNC round 0 (and the first
                                    tentative phase of Algorithm 2): which
                                    graphs are coloured strictly in id order
                                    (each vertex once its lower neighbours are,
                                    higher ones unread: sequential First-Fit).
                                    0 = automatic: graphs of at most 16384
                                    vertices, graphs whose edges mostly join
                                    nearby ids (a naturally numbered mesh) and
                                    graphs of at most 262144 vertices with no
                                    vertex of degree > 62 or > t2; one warp
                                    each, or a group of warps for a big one
                                    without such vertices.  1 = every graph;
                                    -1 = none (pure speculation); k > 1 = none,
                                    and at most k tiles in flight */
    int32_t d2_heavy;            /* GC_DIST2: a vertex whose two-hop
                                    neighbourhood has more entries (sum of its
                                    neighbours' degrees) than this is inspected
                                    by a whole block, the others by one warp;
                                    0 = 4096 */
    int32_t core_deg;            /* GC_SCHED_ASYNC (every colouring call
                                    except recolouring; not with GC_TIERS,
                                    GC_FF_KEEPERS or GC_DIST2): in each graph
                                    the vertices of degree above max(core_deg,
                                    t2) -- if there are at most 4096 of them --
                                    form its core, coloured before round 0 one
                                    at a time in decreasing degree (ties:
                                    increasing id) by First-Fit among
                                    themselves; they keep those colours, so
                                    the repair rounds never rescan their rows
                                    and a dense core of hubs (R-MAT) does not
                                    drive the colour count up.  The cores of a
                                    batch are coloured side by side, one block
                                    each.  0 = 4096, -1 = no core */
} gc_opts;

typedef struct gc_ctx gc_ctx;

/* ---- library --------------------------------------------------------- */

/* Static string for a status code.  Never NULL. */
const char *gc_strerror(int status);

/* Library version: major*10000 + minor*100 + patch. */
int gc_version(void);

/* Create a context bound to CUDA device `device`: it owns the scratch
 * memory (second colour buffer, worklists, counters) reused across calls
 * and grown on demand.  Returns GC_OK and sets *ctx, or an error. */
int gc_ctx_create(gc_ctx **ctx, int device);

/* Free the context and its device memory (after its work finishes). */
void gc_ctx_destroy(gc_ctx *ctx);

/* ---- single graph ---------------------------------------------------- */

/*
 * Colour one graph (Sec. 3 Algorithm 3 or Sec. 2.2 Algorithm 2, per mode)
 * and wait for the result.  row_ptr, col_idx and colors_out may each be
 * host or device memory (host arrays are staged through the device).
 * Uses a per-host-thread default context on the current device.
 * colors_out: n int32 entries, written on success and on
 * GC_ERR_NO_CONVERGENCE (the colouring at the cap); after any other error
 * raised by the colouring its contents are unspecified.
 * stats_out may be NULL.
 */
int gc_color(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode,
             int32_t *colors_out, gc_stats *stats_out);

/*
 * Enqueue the colouring of one graph on `stream` (a cudaStream_t, NULL for
 * the legacy default stream) and return without waiting.  All pointers must
 * be device memory that stays valid until the work completes; colors_out
 * (n entries) also serves as the first colour buffer.  opts may be NULL.
 * Finish with gc_ctx_stats(), which waits for the work and reports status.
 * Returns GC_OK if the work was enqueued.
 */
int gc_color_async(gc_ctx *ctx, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode,
                   const gc_opts *opts, int32_t *colors_out, void *stream);

/*
 * Incremental recolouring (no counterpart call in the paper; Sec. 1's
 * adaptivity loops change a mesh locally): repair the colouring
 * colors_inout (DEVICE, n entries, updated in place) of the graph csr
 * after an edit, by Algorithm 3's while-loop started from those colours with
 * the first worklist = touched (DEVICE int32[n_touched]; repeats are
 * ignored; an id outside 0..n-1 gives GC_ERR_GRAPH) instead of round 0 and
 * U = V.  A vertex inspected is defective if it is uncoloured (0) or a
 * neighbour on its tie side shares its colour.  List every uncoloured
 * vertex and both endpoints of every inserted edge; only listed vertices
 * can change colour (with GC_FF_KEEPERS, also the higher neighbours a
 * recoloured vertex clashes with).  GC_ALG_RSOC only (GC_SCHED_DET: bit-exact as the
 * oracle's replay; GC_SCHED_ASYNC, GC_FF_KEEPERS allowed); no GC_TIERS or
 * GC_REPAIR_SNAPSHOT.  Enqueued on `stream`; finish with gc_ctx_stats().
 */
int gc_recolor_async(gc_ctx *ctx, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, const gc_opts *opts,
                     int32_t *colors_inout, const int32_t *touched, int32_t n_touched, void *stream);

/*
 * Wait for the context's last enqueued colouring and report it.  Returns
 * that colouring's status (GC_OK, GC_ERR_NO_CONVERGENCE, GC_ERR_TIMEOUT,
 * GC_ERR_GRAPH, GC_ERR_CHECK, GC_ERR_OVERFLOW or GC_ERR_CUDA).  stats may
 * be NULL.
 */
int gc_ctx_stats(gc_ctx *ctx, gc_stats *stats);

/* ---- many graphs in one launch ------------------------------------------ */

/*
 * A batch of G independent graphs in one set of device arrays:
 *   vtx_off[G+1], edge_off[G+1]: int64 prefix sums of n_g and nnz_g
 *   row_ptr: graph g's local row pointers (n_g+1 entries, starting at 0)
 *            begin at row_ptr + vtx_off[g] + g
 *   col_idx: graph g's local (0-based) neighbour ids begin at
 *            col_idx + edge_off[g]
 * total_n = vtx_off[G] and total_nnz = edge_off[G] must be given on the
 * host as well (total_n < 2^31, total_nnz < 2^33).  Graph g's colours land
 * at colors_out + vtx_off[g].
 */
typedef struct {
    int32_t G;
    int64_t total_n;             /* < 2^31 */
    int64_t total_nnz;
    const int64_t *vtx_off;      /* device */
    const int64_t *edge_off;     /* device */
    const int32_t *row_ptr;      /* device */
    const int32_t *col_idx;      /* device */
} gc_batch;

/*
 * Colour every graph of the batch in one persistent launch (the graphs form
 * one disjoint union; each graph's colouring, iteration count and conflict
 * count equal those of colouring it alone in GC_SCHED_DET mode).  Per-graph
 * results go to the optional device arrays rounds_out[G] and
 * conflicts_out[G].  Enqueued on `stream`; finish with gc_ctx_stats().
 */
int gc_color_batch(gc_ctx *ctx, const gc_batch *batch, uint32_t mode, const gc_opts *opts,
                   int32_t *colors_out, int32_t *rounds_out, int64_t *conflicts_out,
                   void *stream);

/* ---- batch plans: one batch colouring captured in a CUDA graph ---------- */

typedef struct gc_plan gc_plan;

/*
 * Capture one gc_color_batch call (its memsets, kernels, event records and
 * statistics read-back) into a CUDA graph on `device`, to be replayed by
 * gc_plan_launch with no host-side planning or allocation per launch.  The
 * plan owns a private context whose scratch memory is sized here and never
 * moves.  Every launch colours the same arrays: the batch's device arrays,
 * colors_out and the optional rounds_out/conflicts_out must stay allocated
 * and in place until gc_plan_destroy.  Returns GC_ERR_CUDA if the device
 * cannot capture the launch.
 */
int gc_plan_create(const gc_batch *batch, int device, uint32_t mode, const gc_opts *opts,
                   int32_t *colors_out, int32_t *rounds_out, int64_t *conflicts_out, gc_plan **plan);

/* Replay the captured colouring on `stream` (asynchronous). */
int gc_plan_launch(gc_plan *plan, void *stream);

/* Wait for the last launch and report it (as gc_ctx_stats). */
int gc_plan_stats(gc_plan *plan, gc_stats *stats);

/* Wait for the last launch and free the plan. */
void gc_plan_destroy(gc_plan *plan);

/* ---- autotuning the options of a batch ---------------------------------- */

typedef struct {
    gc_opts best;                /* fastest option set found */
    float best_ms;               /* its median device time */
    float default_ms;            /* median device time with default options */
    int32_t evaluated;           /* option sets timed */
} gc_tune_result;

/*
 * Choose gc_opts for colouring this batch in `mode` by timing it: coordinate
 * descent from the defaults over t1 (largest degree coloured by one
 * thread), t2 (largest degree coloured by one warp; above it a block per
 * vertex), tile and blocks_per_sm (searched as pairs: they interact) and
 * tail (window, which changes which graphs are coloured in id order and so
 * the colour counts, stays automatic); each candidate's cost is the median
 * of `reps` (1..64) runs' device time (CUDA events), and at most three
 * sweeps are made.  In GC_SCHED_ASYNC the
 * options change the colouring as well: a candidate is taken only if none of
 * its runs used more colours than the default options' runs did (unless
 * GC_NO_COLOR_STATS is set).  Synchronous (legacy
 * default stream); colors_out (device, total_n entries) receives the
 * colourings while it runs.  In GC_SCHED_DET mode every option set gives
 * the same colouring, so only speed is at stake.  Returns the first error
 * of any run.
 *
 * Cache: when the environment variable GC_TUNE_CACHE names a file, results
 * are kept there (one text line each, appended) under a key of the library
 * version, the call, the mode, the graph's shape (total vertices, entries,
 * graphs), the device's SM count and reps.  A call whose key is in the file
 * searches nothing: it colours once with the cached options (colors_out
 * receives that colouring) and returns them with evaluated = 0 and the
 * cached times.
 */
int gc_autotune_batch(gc_ctx *ctx, const gc_batch *batch, uint32_t mode, int32_t reps, int32_t *colors_out,
                      gc_tune_result *result);

/* As gc_autotune_batch for one graph (device pointers; gc_color_async
 * semantics): colors_out (n entries) receives the colourings. */
int gc_autotune(gc_ctx *ctx, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, int32_t reps,
                int32_t *colors_out, gc_tune_result *result);

/* ---- colour classes --------------------------------------------------- */

/*
 * The colour classes of a colouring: its vertices grouped by colour, each
 * group in increasing id (a stable counting sort).  Sec. 1: the vertices of
 * one colour are an independent set, so a consumer processes them
 * concurrently, class after class.
 *   colors:         DEVICE int32[n], every value in 1..num_colors
 *                   (GC_ERR_ARG otherwise; the outputs are then unspecified)
 *   class_ptr:      DEVICE int32[num_colors + 2]: the vertices of colour c
 *                   are class_vertices[class_ptr[c] .. class_ptr[c+1]);
 *                   class_ptr[0] = class_ptr[1] = 0
 *   class_vertices: DEVICE int32[n]
 * num_colors <= GC_CLASSES_MAX_COLORS.  Scratch comes from the context
 * (about num_colors * n / 64 bytes, at most 256 MB).
 * Enqueued on `stream`, then waited for; returns the status.
 */
#define GC_CLASSES_MAX_COLORS (1 << 20)
int gc_color_classes(gc_ctx *ctx, const int32_t *colors, int32_t n, int32_t num_colors, int32_t *class_ptr,
                     int32_t *class_vertices, void *stream);

/* ---- serving: continuous batching of colouring requests ------------------ */

/*
 * A colouring server on one device.  Requests (graphs in host memory) are
 * queued; a worker thread admits them in arrival order while their CSR fits
 * the device-memory budget (and at most max_slots are resident), uploading
 * them on a copy stream, and colours the uploaded requests in batched
 * launches ("waves", gc_color_batch semantics, every graph independent) on
 * two compute lanes: a wave starts as soon as a lane is free, so requests
 * that arrive while a wave runs are coloured in the next wave on the other
 * lane, beside it.  Each wave's grid takes its share of the SMs (opts
 * blocks_per_sm, by default half the kernel's resident blocks per SM).
 * Thread-safe.
 *
 * Memory: the budget is one device allocation holding the resident graphs'
 * row pointers and column indices ((n+1+nnz)*4 bytes each, 256-byte
 * granules).  Per-batch working memory (about 32 bytes per vertex of the
 * batch) comes on top of it, as does a pinned host pool of 2*budget bytes
 * that holds submitted graphs and their results until they are polled
 * (requests that do not fit it get pinned blocks of their own).
 * In GC_SCHED_DET mode every request's colouring is exactly the colouring
 * gc_color would return for it alone.
 */
typedef struct gc_server gc_server;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t waves;              /* batched launches so far */
    int64_t budget_bytes;        /* device bytes for resident graphs */
    int64_t in_use_bytes;        /* of which held now */
    int64_t peak_bytes;          /* most ever held (never above the budget) */
    int32_t queued;              /* waiting for admission */
    int32_t resident;            /* admitted and not finished */
    int32_t max_wave_graphs;     /* largest batch launched */
    int32_t lanes;               /* waves that can be on the GPU at once */
    uint64_t cancelled;          /* requests dropped by gc_server_cancel */
    uint64_t overlapped_waves;   /* waves whose GPU interval (event timestamps
                                    around the colouring) overlapped another
                                    lane's wave */
    int64_t overlap_us;          /* total time two waves were on the GPU at
                                    once (same timestamps) */
} gc_server_info;

/* Create a server on `device` with a device-memory budget and a slot limit;
 * mode and opts apply to every request (opts may be NULL). */
int gc_server_create(gc_server **s, int device, size_t device_budget_bytes, int max_slots, uint32_t mode,
                     const gc_opts *opts);

/* Queue a graph given by HOST arrays; they are copied (to pinned memory)
 * before the call returns, and the call does not wait for the GPU.  *ticket
 * identifies the request.  GC_ERR_BUDGET if the graph alone can never fit
 * the budget.  Results stay in pinned memory until polled. */
int gc_server_submit(gc_server *s, const gc_csr *host_csr, int32_t n, int64_t nnz, uint64_t *ticket);

/* GC_PENDING while the request runs; once done, copies its colours to the
 * HOST array colors_out (n entries, may be NULL), fills stats_out (may be
 * NULL; elapsed_ms = submit-to-completion latency, colors and
 * distinct_colors counted on the host) and returns the request's status;
 * the ticket is then released (GC_ERR_NOT_FOUND afterwards). */
int gc_server_poll(gc_server *s, uint64_t ticket, int32_t *colors_out, gc_stats *stats_out);

/* As gc_server_poll, waiting up to timeout_ms (< 0: no limit) for the
 * request to finish; GC_PENDING if it has not. */
int gc_server_wait(gc_server *s, uint64_t ticket, int32_t *colors_out, gc_stats *stats_out, int32_t timeout_ms);

/* Drop a request: a queued one is removed before any GPU work, one already
 * uploading or being coloured is discarded when its work ends, a finished one
 * is discarded unpolled.  The ticket is released at once (poll and wait then
 * return GC_ERR_NOT_FOUND).  GC_OK, or GC_ERR_NOT_FOUND for an unknown
 * ticket. */
int gc_server_cancel(gc_server *s, uint64_t ticket);

/* Counters and memory use of the server. */
int gc_server_query(gc_server *s, gc_server_info *out);

/* Stop the worker, wait for work in flight and free everything; requests
 * not yet polled are dropped. */
void gc_server_destroy(gc_server *s);

/* ---- colouring without any allocation ---------------------------------- */

/* Largest graph (vertices) gc_color_noalloc accepts. */
#define GC_NOALLOC_MAX_N 262144

/*
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate memory while they run: code whose device memory is
 * owned by another allocator under a hard budget, or latency-critical loops
 * that cannot afford a cudaMalloc/cudaFree (either may synchronise the
 * device).  Colours one graph as gc_color_async + gc_ctx_stats do, but no
 * context is needed and nothing is allocated: all working memory comes from
 * one fixed array of about 7 MB compiled into the library, which every GPU
 * that loads the library holds until the process exits.  Differences from
 * gc_color_async: GC_DIST2 is rejected (GC_ERR_ARG) and d2_heavy is
 * ignored; asynchronous RSOC keeps no round-0 suspect masks, so its first
 * repair reads whole tie sides and its work counters (model_bytes) can
 * differ from the allocating call's.  Deterministic modes give exactly the
 * allocating call's colouring and statistics.
 *
 *   csr, colors_out: DEVICE pointers (host pointers give GC_ERR_ARG: staging
 *                    them would need memory); the caller owns them.
 *   n > GC_NOALLOC_MAX_N returns GC_ERR_TOO_LARGE before touching the GPU.
 *   stream: a cudaStream_t (NULL = legacy default stream).  The call enqueues
 *           its work there and waits for it, then fills stats_out (may be
 *           NULL; elapsed_ms is 0: no timing is recorded).
 *   Returns the colouring's status, as gc_ctx_stats would.
 *
 * The first call on each device looks up the fixed array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * previous call's contents (the parts that must start at zero are cleared at
 * the start of each call), so calls whose GPU work overlaps -- on different
 * streams or host threads without ordering between them -- race and give
 * undefined results.  Serialise them.
 */
int gc_color_noalloc(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, const gc_opts *opts,
                     int32_t *colors_out, gc_stats *stats_out, void *stream);

/* ---- the paper's own form on the host cores ---------------------------- */

/*
 * Algorithms 2 and 3 as the paper runs them (Sec. 3, measured in Sec. 4):
 * OpenMP threads over the CPU cores, every loop over U a parallel for with
 * dynamic scheduling.  A separate host implementation for comparison beside
 * the GPU calls: no GPU call ever runs it, and it touches no GPU.
 *
 *   csr, colors_out: HOST pointers (n+1, nnz and n int32 entries).
 *   mode: GC_ALG_RSOC or GC_ALG_TWO_PHASE, GC_SCHED_ASYNC (colours read and
 *         written in place by all threads, the paper's form; round 0 of RSOC
 *         is First-Fit over V in place) or GC_SCHED_DET (every read of an
 *         iteration sees the colours of the end of the iteration before:
 *         the same colouring, iterations, conflicts and round sizes as
 *         gc_color in GC_SCHED_DET, whatever the thread count), either
 *         tie-break, GC_VALIDATE (check the CSR on the host first, as
 *         gc_color does on the device: GC_ERR_GRAPH if malformed),
 *         GC_CHECKED (verify the result on the host;
 *         GC_ERR_CHECK if invalid), GC_NO_COLOR_STATS and GC_DIST2 (the same
 *         algorithms over two-hop neighbourhoods: deterministic forms equal
 *         the distance-2 replay of gc_color); any other bit gives
 *         GC_ERR_ARG.
 *   num_threads: OpenMP threads (0 = the OpenMP default).  With one thread
 *         GC_SCHED_ASYNC RSOC is sequential First-Fit in id order.
 *   stats_out (may be NULL): rounds, conflicts, colors, distinct_colors,
 *         round_sizes (as for gc_ctx_stats), elapsed_ms = host wall time of
 *         the colouring; model_bytes and error_word are 0.
 * Returns GC_OK, GC_ERR_ARG, GC_ERR_OOM, GC_ERR_GRAPH, GC_ERR_NO_CONVERGENCE
 * (n+1 iterations with conflicts left; colors_out holds the colouring at the
 * cap) or GC_ERR_CHECK.  Without GC_VALIDATE a malformed graph is not
 * detected: unsorted rows give an invalid colouring and out-of-range
 * indices are read out of bounds.
 */
int gc_host_color(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, int32_t num_threads,
                  int32_t *colors_out, gc_stats *stats_out);

/* Threads gc_host_color uses with num_threads = 0 (1 if the library was
 * built without OpenMP). */
int gc_host_threads(void);

/* ---- failure path ------------------------------------------------------ */

/*
 * Check of the bounded wait that every persistent kernel's grid barrier
 * uses: a cooperative launch on `device` (2 blocks) whose barrier waits for
 * one block more than the grid holds, an arrival that never comes.  After
 * timeout_ms (1..10000) the wait gives up, the device error word receives
 * GC_EW_TIMEOUT (copied to *error_word_out if not NULL) and the kernel
 * returns; the CUDA context stays usable.  Synchronous.  Returns
 * GC_ERR_TIMEOUT when the wait ran out as it should, GC_OK if it did not,
 * GC_ERR_ARG or GC_ERR_CUDA.  The colouring calls report the same failure
 * as GC_ERR_TIMEOUT after a 10 s wait.
 */
int gc_debug_barrier_timeout(int device, int32_t timeout_ms, int32_t *error_word_out);

/* The bounded waits of the colouring kernel that gc_debug_wait_timeout can
 * run out. */
enum {
    GC_WAIT_GRID_BARRIER = 0,    /* the grid barrier between rounds (10 s) */
    GC_WAIT_TILE_DONE = 1,       /* asynchronous round 0 with gc_opts.window >
                                    1: a tile waits until the tile `window`
                                    places before it is published (10 s) */
    GC_WAIT_PIPE_CHUNK = 2,      /* round 0 of a graph coloured in id order by
                                    a group of warps: a vertex waits until its
                                    lower neighbours are coloured (2 s) */
    GC_WAIT_STAGE_COPY = 3       /* a staged adjacency copy (TMA bulk copy)
                                    completing on its mbarrier (2 s, then as
                                    long again for the copy to land) */
};

/*
 * Check of one bounded wait of the colouring kernel, as
 * gc_debug_barrier_timeout does for the grid barrier: a one-warp launch on
 * `device` runs that wait against a flag nobody publishes (GC_WAIT_TILE_DONE),
 * a lower neighbour nobody colours (GC_WAIT_PIPE_CHUNK; a 64-vertex graph
 * whose vertex 32 is adjacent to vertex 0) or an mbarrier no copy completes
 * (GC_WAIT_STAGE_COPY), with the limit timeout_ms (1..10000) instead of the
 * one given above.  The wait gives up, the device error word receives
 * GC_EW_TIMEOUT (copied to *error_word_out if not NULL) and the kernel
 * returns; the CUDA context stays usable.  GC_WAIT_STAGE_COPY waits twice the
 * limit (the second wait lets a copy in flight land).  Synchronous.  Returns
 * GC_ERR_TIMEOUT when the wait ran out as it should, GC_OK if it did not,
 * GC_ERR_ARG or GC_ERR_CUDA.  GC_WAIT_GRID_BARRIER is
 * gc_debug_barrier_timeout.
 */
int gc_debug_wait_timeout(int device, int32_t wait, int32_t timeout_ms, int32_t *error_word_out);

/* ---- measurement ------------------------------------------------------- */

/*
 * Random 4-byte gathers per second from an array of `array_bytes` bytes
 * (4 KB .. 1 GB, rounded down to a power of two) on `device`: the ceiling
 * of the colouring kernels' neighbour-colour reads, which are random 4-byte
 * loads from the colour array (8 MB for 2^21 vertices, resident in L2).
 * The paper has no counterpart; it serves the roofline analysis only.
 * One launch of SMs x blocks_per_sm (1..8) blocks of 256 threads after one
 * warm-up launch, timed with CUDA events.  dependent = 0: every thread
 * issues independent loads at hashed positions (eight in flight);
 * dependent = 1: every thread follows a chain in which each loaded value is
 * the next position (one load in flight), like the kernels' row pointer ->
 * column index -> colour chains.  The array is allocated, filled on the
 * device and freed by the call.  Synchronous.  Writes the loads per second
 * to *gloads_per_s_out (in units of 1e9).  Returns GC_OK, GC_ERR_ARG,
 * GC_ERR_OOM or GC_ERR_CUDA.
 */
int gc_measure_gather_rate(int device, int64_t array_bytes, int32_t blocks_per_sm, int32_t dependent,
                           double *gloads_per_s_out);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */
