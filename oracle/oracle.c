/*
 * CPU oracle for speculative First-Fit graph colouring.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA path (no headers, helpers or tables) and is deliberately plain,
 * slow and single-threaded so that each function can be checked against the
 * paper by eye.
 *
 * Paper: Rokos, Gorman, Kelly, "A Fast and Scalable Graph Coloring
 * Algorithm for Multi-core and Many-core Architectures" (arXiv 1505.04086).
 *
 *   oracle_ff          Algorithm 1 (sequential greedy / First-Fit), Sec. 2.1
 *   oracle_rsoc_det    Algorithm 3 (RSOC), Sec. 3, every round reading the
 *                      colours as they stood at the end of the previous round
 *   oracle_2p_det      Algorithm 2 (Catalyurek et al.), Sec. 2.2, same
 *                      snapshot reading; written independently of the above
 *   oracle_check       validity + the d+1 bound of Sec. 2.1
 *   oracle_chi         exact chromatic number by exhaustive search (n <= 12)
 *   oracle_csr_check   input well-formedness (symmetric, sorted, simple)
 *   oracle_rsoc_det_from  incremental recolouring: Algorithm 3's while-loop
 *                      (snapshot reading) started from a given colouring
 *                      and the vertices an edit touched
 *   oracle_ff_d2, oracle_rsoc_det_d2
 *                      distance-2 colouring (Sec. 6 names it as the variant
 *                      that gains most): Algorithm 1 and the Algorithm 3
 *                      replay with "neighbour" read as "within two hops"
 *   oracle_classes     colour classes: the vertices grouped by colour, each
 *                      group in increasing id (the independent sets a
 *                      colouring is computed for, Sec. 1)
 *
 * Colours are 1-based; 0 means "not coloured" (Sec. 2.1 numbers colours
 * 1..d+1 and Algorithm 1 forbids only the colours of *coloured* neighbours).
 *
 * Tie-break (which endpoint of a conflicting edge is recoloured):
 *   ORACLE_TIE_LOWER_KEEPS   v is defective iff some neighbour u < v shares
 *                            its colour (the lower id keeps its colour)
 *   ORACLE_TIE_HIGHER_KEEPS  v is defective iff some neighbour u > v shares
 *                            its colour (the test printed in Algorithms 2, 3)
 *   ORACLE_TIE_NONE          v is defective iff any neighbour shares its
 *                            colour; this is the symmetric test whose
 *                            lock-step livelock Section 5 / Fig. 7 describes
 *
 * Iterations count executions of the while-loop body, the last one (which
 * finds no defect) included; RSOC's round 0 is not counted.  Conflicts are
 * the sum over iterations of the number of vertices found defective.
 *
 * Byte model (reported beside the results; the GPU path counts the same
 * quantity so both can be compared): per vertex inspected in a round,
 *   4  if the round reads an explicit worklist (not the first pass over V)
 *   8  for its two row pointers
 *   4  for its own colour (detection passes only)
 *   8  per adjacency entry the step must read (column index + colour):
 *        tentative colouring / recolouring: all deg(v) entries
 *        clean vertex under detection: its tie-side entries only
 *   4  per colour written, 4 per worklist push
 * A tentative pass over a snapshot in which nothing is coloured needs no
 * reads (every vertex gets colour 1) and is counted as 4 bytes per vertex.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORACLE_TIE_LOWER_KEEPS = 0, ORACLE_TIE_HIGHER_KEEPS = 1, ORACLE_TIE_NONE = 2 };
enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_OOM = 2, ORACLE_ERR_NO_CONVERGENCE = 3 };

typedef struct {
    int64_t iterations;
    int64_t conflicts;
    int64_t model_bytes;
    int32_t colors;          /* max colour */
    int32_t distinct_colors;
    int32_t *round_sizes;    /* optional, caller-owned: |L| per iteration */
    int64_t round_sizes_cap;
} oracle_stats;

/* ------------------------------------------------------------------ */
/* First-Fit step (Alg. 1 body)                                        */
/* ------------------------------------------------------------------ */

/*
 * Smallest colour k >= 1 that no coloured neighbour of v has, with the
 * neighbours' colours taken from `col`.  `mark` is scratch of at least
 * maxdeg+2 entries; mark[k] == stamp means "colour k is taken".  Colours
 * above deg(v)+1 cannot change the answer (Sec. 2.1: one of 1..d+1 is
 * always free) and are skipped.
 */
static int32_t first_fit(int32_t v, const int32_t *row_ptr, const int32_t *col_idx,
                         const int32_t *col, int64_t *mark, int64_t stamp)
{
    int32_t deg = row_ptr[v + 1] - row_ptr[v];
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        int32_t c = col[col_idx[k]];
        if (c >= 1 && c <= deg + 1) mark[c] = stamp;
    }
    int32_t k = 1;
    while (mark[k] == stamp) ++k;
    return k;
}

static int32_t max_degree(int32_t n, const int32_t *row_ptr)
{
    int32_t d = 0;
    for (int32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] - row_ptr[v] > d) d = row_ptr[v + 1] - row_ptr[v];
    return d;
}

static void colour_counts(int32_t n, const int32_t *c, oracle_stats *st)
{
    if (!st) return;
    int32_t mx = 0;
    for (int32_t v = 0; v < n; ++v)
        if (c[v] > mx) mx = c[v];
    st->colors = mx;
    char *seen = (char *)calloc((size_t)mx + 1, 1);
    int32_t d = 0;
    if (seen) {
        for (int32_t v = 0; v < n; ++v)
            if (c[v] > 0 && !seen[c[v]]) { seen[c[v]] = 1; ++d; }
        free(seen);
    }
    st->distinct_colors = d;
}

/*
 * Algorithm 1: visit v = 0..n-1 in natural order and give each the
 * smallest colour not used by its already-coloured neighbours.
 * Returns the number of colours used (max colour), or -1 on OOM.
 */
int32_t oracle_ff(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *c)
{
    if (n < 0) return -1;
    int32_t dmax = max_degree(n, row_ptr);
    int64_t *mark = (int64_t *)malloc(((size_t)dmax + 2) * sizeof(int64_t));
    if (!mark) return -1;
    for (int32_t k = 0; k < dmax + 2; ++k) mark[k] = -1;
    for (int32_t v = 0; v < n; ++v) c[v] = 0;
    int32_t used = 0;
    for (int32_t v = 0; v < n; ++v) {
        c[v] = first_fit(v, row_ptr, col_idx, c, mark, v);
        if (c[v] > used) used = c[v];
    }
    free(mark);
    return used;
}

/* ------------------------------------------------------------------ */
/* Algorithm 3 (RSOC), snapshot replay                                 */
/* ------------------------------------------------------------------ */

/* Does the tie-break make v the endpoint that must change when its
 * neighbour u has the same colour? */
static int loses_to(int32_t v, int32_t u, int tie)
{
    if (tie == ORACLE_TIE_LOWER_KEEPS) return u < v;
    if (tie == ORACLE_TIE_HIGHER_KEEPS) return u > v;
    return 1;
}

/*
 * Algorithm 3 with every read of round i seeing the colours as they stood
 * at the end of round i-1 (the deterministic, round-synchronous reading):
 *
 *   round 0: every vertex takes First-Fit over the (all-uncoloured)
 *            snapshot;
 *   U <- V;
 *   while U is not empty:
 *       for v in U: if some neighbour u that v loses to has c(u) == c(v),
 *                   v takes First-Fit over the snapshot (all neighbours'
 *                   colours forbidden, whether or not they are defective
 *                   themselves) and joins L;
 *       U <- L.
 *
 * max_iters bounds the loop; hitting it returns ORACLE_ERR_NO_CONVERGENCE
 * with the colouring as it stands.
 */
int oracle_rsoc_det(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int tie,
                    int64_t max_iters, int32_t *c, oracle_stats *st)
{
    if (n < 0 || !c) return ORACLE_ERR_ARG;
    int32_t dmax = max_degree(n, row_ptr);
    int32_t *snap = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *U = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *L = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t *mark = (int64_t *)malloc(((size_t)dmax + 2) * sizeof(int64_t));
    if (!snap || !U || !L || !mark) {
        free(snap); free(U); free(L); free(mark);
        return ORACLE_ERR_OOM;
    }
    for (int32_t k = 0; k < dmax + 2; ++k) mark[k] = -1;
    int64_t stamp = 0, bytes = 0, iters = 0, conflicts = 0;

    /* Round 0: tentative First-Fit of every vertex over the snapshot in
     * which no vertex is coloured yet. */
    for (int32_t v = 0; v < n; ++v) snap[v] = 0;
    for (int32_t v = 0; v < n; ++v) c[v] = first_fit(v, row_ptr, col_idx, snap, mark, stamp++);
    bytes += 4 * (int64_t)n;

    /* U^0 <- V */
    int64_t nu = n;
    for (int32_t v = 0; v < n; ++v) U[v] = v;
    int first_pass = 1;
    int rc = ORACLE_OK;

    while (nu > 0) {
        if (iters >= max_iters) { rc = ORACLE_ERR_NO_CONVERGENCE; break; }
        ++iters;
        memcpy(snap, c, (size_t)n * sizeof(int32_t));
        int64_t nl = 0;
        for (int64_t i = 0; i < nu; ++i) {
            int32_t v = U[i];
            int defective = 0;
            int64_t tie_side = 0;
            for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                int32_t u = col_idx[k];
                if (!loses_to(v, u, tie)) continue;
                ++tie_side;
                if (snap[u] == snap[v]) defective = 1;
            }
            int32_t deg = row_ptr[v + 1] - row_ptr[v];
            bytes += (first_pass ? 0 : 4) + 8 + 4;
            if (defective) {
                c[v] = first_fit(v, row_ptr, col_idx, snap, mark, stamp++);
                L[nl++] = v;
                bytes += 8 * (int64_t)deg + 4 + 4;
            } else {
                bytes += 8 * tie_side;
            }
        }
        if (st && st->round_sizes && iters - 1 < st->round_sizes_cap)
            st->round_sizes[iters - 1] = (int32_t)nl;
        conflicts += nl;
        int32_t *t = U; U = L; L = t;
        nu = nl;
        first_pass = 0;
    }
    if (st) {
        st->iterations = iters;
        st->conflicts = conflicts;
        st->model_bytes = bytes;
        colour_counts(n, c, st);
    }
    free(snap); free(U); free(L); free(mark);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 (two-phase), snapshot replay                            */
/* ------------------------------------------------------------------ */

/*
 * Algorithm 2 with the same round-synchronous reading:
 *
 *   U <- V
 *   while U is not empty:
 *       phase 1: for v in U, new(v) = First-Fit of v over the colours as
 *                they stood before this phase; then all new colours land;
 *       phase 2: L = { v in U : some neighbour u that v loses to has
 *                c(u) == c(v) } over the colours after phase 1;
 *       U <- L.
 *
 * Written without reference to oracle_rsoc_det; the two replays are
 * expected to agree (the phase-1 recolouring of iteration k+1 equals the
 * fused recolouring of RSOC iteration k), which the tests check.
 */
int oracle_2p_det(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int tie,
                  int64_t max_iters, int32_t *c, oracle_stats *st)
{
    if (n < 0 || !c) return ORACLE_ERR_ARG;
    int32_t *before = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *work = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *next = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t dmax = max_degree(n, row_ptr);
    int32_t *taken = (int32_t *)malloc(((size_t)dmax + 2) * sizeof(int32_t));
    if (!before || !work || !next || !taken) {
        free(before); free(work); free(next); free(taken);
        return ORACLE_ERR_OOM;
    }
    for (int32_t v = 0; v < n; ++v) c[v] = 0;
    int64_t w = 0;
    for (int32_t v = 0; v < n; ++v) work[w++] = v;
    int64_t iters = 0, conflicts = 0, bytes = 0;
    int rc = ORACLE_OK;
    int first = 1;
    while (w > 0) {
        if (iters >= max_iters) { rc = ORACLE_ERR_NO_CONVERGENCE; break; }
        ++iters;
        /* Phase 1: tentative colouring from the colours before this phase. */
        memcpy(before, c, (size_t)n * sizeof(int32_t));
        int any_coloured = 0;
        for (int32_t v = 0; v < n && !any_coloured; ++v) any_coloured = before[v] != 0;
        for (int64_t i = 0; i < w; ++i) {
            int32_t v = work[i];
            int32_t deg = row_ptr[v + 1] - row_ptr[v];
            for (int32_t k = 0; k <= deg + 1; ++k) taken[k] = 0;
            for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                int32_t cu = before[col_idx[k]];
                if (cu > 0 && cu <= deg + 1) taken[cu] = 1;
            }
            int32_t pick = 1;
            while (taken[pick]) ++pick;
            c[v] = pick;
            if (any_coloured)
                bytes += (first ? 0 : 4) + 8 + 8 * (int64_t)deg + 4;
            else
                bytes += 4;
        }
        /* Phase 2: conflict detection on the colours after phase 1. */
        int64_t nl = 0;
        for (int64_t i = 0; i < w; ++i) {
            int32_t v = work[i];
            int bad = 0;
            int64_t seen = 0;
            for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                int32_t u = col_idx[k];
                int counts = tie == ORACLE_TIE_NONE ||
                             (tie == ORACLE_TIE_LOWER_KEEPS && u < v) ||
                             (tie == ORACLE_TIE_HIGHER_KEEPS && u > v);
                if (!counts) continue;
                ++seen;
                if (c[u] == c[v]) bad = 1;
            }
            bytes += (first ? 0 : 4) + 8 + 4 + 8 * seen;
            if (bad) { next[nl++] = v; bytes += 4; }
        }
        if (st && st->round_sizes && iters - 1 < st->round_sizes_cap)
            st->round_sizes[iters - 1] = (int32_t)nl;
        conflicts += nl;
        memcpy(work, next, (size_t)nl * sizeof(int32_t));
        w = nl;
        first = 0;
    }
    if (st) {
        st->iterations = iters;
        st->conflicts = conflicts;
        st->model_bytes = bytes;
        colour_counts(n, c, st);
    }
    free(before); free(work); free(next); free(taken);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Checker                                                             */
/* ------------------------------------------------------------------ */

/*
 * Returns 0 if c is a proper colouring (no entry (v,u) with c[v] == c[u])
 * and every colour lies in 1..deg(v)+1 (the Sec. 2.1 bound).  Otherwise it
 * names the first offending vertex v: -(v+1) if c[v] is out of bounds,
 * v+1 if v shares its colour with a neighbour.  The max colour and the
 * number of distinct colours go to *colors / *distinct when given.
 */
int64_t oracle_check(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *c,
                     int32_t *colors, int32_t *distinct)
{
    int64_t bad = 0;
    for (int32_t v = 0; v < n && !bad; ++v) {
        int32_t deg = row_ptr[v + 1] - row_ptr[v];
        if (c[v] < 1 || c[v] > deg + 1) { bad = -((int64_t)v + 1); break; }
        for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k)
            if (c[col_idx[k]] == c[v]) { bad = (int64_t)v + 1; break; }
    }
    if (colors || distinct) {
        oracle_stats st;
        memset(&st, 0, sizeof st);
        colour_counts(n, c, &st);
        if (colors) *colors = st.colors;
        if (distinct) *distinct = st.distinct_colors;
    }
    return bad;
}

/*
 * 0 if the CSR is symmetric, rows strictly increasing (sorted, no repeats),
 * indices in range and no self-loops; otherwise 1 + offending vertex.
 */
int64_t oracle_csr_check(int32_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col_idx)
{
    if (n < 0 || row_ptr[0] != 0 || row_ptr[n] != nnz) return 1;
    for (int32_t v = 0; v < n; ++v) {
        if (row_ptr[v + 1] < row_ptr[v]) return (int64_t)v + 1;
        for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int32_t u = col_idx[k];
            if (u < 0 || u >= n || u == v) return (int64_t)v + 1;
            if (k > row_ptr[v] && col_idx[k - 1] >= u) return (int64_t)v + 1;
            /* u's row must contain v */
            int found = 0;
            for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j)
                if (col_idx[j] == v) { found = 1; break; }
            if (!found) return (int64_t)v + 1;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Exact chromatic number (small graphs)                               */
/* ------------------------------------------------------------------ */

static int try_colour(int32_t n, const uint32_t *adj, int32_t v, int32_t k, int32_t *c)
{
    if (v == n) return 1;
    for (int32_t col = 1; col <= k; ++col) {
        int ok = 1;
        for (int32_t u = 0; u < v; ++u)
            if (((adj[v] >> u) & 1u) && c[u] == col) { ok = 0; break; }
        if (!ok) continue;
        c[v] = col;
        if (try_colour(n, adj, v + 1, k, c)) return 1;
    }
    c[v] = 0;
    return 0;
}

/* Smallest k such that the graph has a proper k-colouring, found by trying
 * every assignment in order; n <= 12.  Returns -1 for bad input. */
int32_t oracle_chi(int32_t n, const int32_t *row_ptr, const int32_t *col_idx)
{
    if (n < 0 || n > 12) return -1;
    if (n == 0) return 0;
    uint32_t adj[12] = {0};
    for (int32_t v = 0; v < n; ++v)
        for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) adj[v] |= 1u << col_idx[k];
    int32_t c[12];
    for (int32_t k = 1; k <= n; ++k) {
        memset(c, 0, sizeof c);
        if (try_colour(n, adj, 0, k, c)) return k;
    }
    return n;
}

/*
 * Colour classes (Sec. 1: a colouring partitions V into independent sets
 * whose vertices can be processed concurrently).  A stable counting sort by
 * colour: count every colour, turn the counts into start offsets, then walk
 * the vertices in increasing id and append each one to its colour's group.
 *   colors[v] in 1..k for every v (else returns 1 + the first bad vertex)
 *   ptr[0..k+1]: the vertices of colour c are verts[ptr[c] .. ptr[c+1])
 *   (ptr[0] = ptr[1] = 0: there is no colour 0)
 * Returns 0 on success.
 */
int64_t oracle_classes(int32_t n, const int32_t *colors, int32_t k, int32_t *ptr, int32_t *verts)
{
    for (int32_t v = 0; v < n; ++v)
        if (colors[v] < 1 || colors[v] > k) return (int64_t)v + 1;
    for (int32_t c = 0; c <= k + 1; ++c) ptr[c] = 0;
    for (int32_t v = 0; v < n; ++v) ptr[colors[v] + 1] += 1;   /* count colour c at ptr[c+1] */
    for (int32_t c = 1; c <= k + 1; ++c) ptr[c] += ptr[c - 1];  /* now ptr[c] = vertices of colour < c */
    int32_t *next = (int32_t *)malloc(((size_t)k + 2) * sizeof(int32_t));
    if (!next) return -1;
    for (int32_t c = 0; c <= k + 1; ++c) next[c] = ptr[c];
    for (int32_t v = 0; v < n; ++v) verts[next[colors[v]]++] = v;
    free(next);
    return 0;
}

/*
 * Incremental recolouring.  Sec. 1 motivates colouring with meshes that an
 * adaptivity loop keeps changing; after a local edit only the touched part
 * needs repair.  This is the while-loop of Algorithm 3 with snapshot reads
 * (as oracle_rsoc_det) started from the colouring c (updated in place) and
 * U = the touched vertices (each listed once; repeats are ignored) instead
 * of round 0 and U = V.  A vertex of U is defective if it is uncoloured (0)
 * or a neighbour on its tie side shares its colour.  The caller lists every
 * uncoloured vertex and both endpoints of every inserted edge (a removed
 * edge creates no conflict).  Every round reads an explicit worklist.
 */
int oracle_rsoc_det_from(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int tie, int64_t max_iters,
                         const int32_t *touched, int32_t n_touched, int32_t *c, oracle_stats *st)
{
    if (n < 0 || n_touched < 0 || !c || (n_touched > 0 && !touched)) return ORACLE_ERR_ARG;
    int32_t dmax = max_degree(n, row_ptr);
    int32_t *snap = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *U = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *L = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    char *seen = (char *)calloc((size_t)n + 1, 1);
    int64_t *mark = (int64_t *)malloc(((size_t)dmax + 2) * sizeof(int64_t));
    if (!snap || !U || !L || !seen || !mark) {
        free(snap); free(U); free(L); free(seen); free(mark);
        return ORACLE_ERR_OOM;
    }
    for (int32_t k = 0; k < dmax + 2; ++k) mark[k] = -1;
    int64_t nu = 0;
    for (int32_t i = 0; i < n_touched; ++i) {
        int32_t v = touched[i];
        if (v < 0 || v >= n) {
            free(snap); free(U); free(L); free(seen); free(mark);
            return ORACLE_ERR_ARG;
        }
        if (!seen[v]) {
            seen[v] = 1;
            U[nu++] = v;
        }
    }
    int64_t stamp = 0, bytes = 0, iters = 0, conflicts = 0;
    int rc = ORACLE_OK;
    while (nu > 0) {
        if (iters >= max_iters) { rc = ORACLE_ERR_NO_CONVERGENCE; break; }
        ++iters;
        memcpy(snap, c, (size_t)n * sizeof(int32_t));
        int64_t nl = 0;
        for (int64_t i = 0; i < nu; ++i) {
            int32_t v = U[i];
            int defective = snap[v] == 0;
            int64_t tie_side = 0;
            for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
                int32_t u = col_idx[k];
                if (!loses_to(v, u, tie)) continue;
                ++tie_side;
                if (snap[u] == snap[v]) defective = 1;
            }
            int32_t deg = row_ptr[v + 1] - row_ptr[v];
            bytes += 4 + 8 + 4;
            if (defective) {
                c[v] = first_fit(v, row_ptr, col_idx, snap, mark, stamp++);
                L[nl++] = v;
                bytes += 8 * (int64_t)deg + 4 + 4;
            } else {
                bytes += 8 * tie_side;
            }
        }
        if (st && st->round_sizes && iters - 1 < st->round_sizes_cap)
            st->round_sizes[iters - 1] = (int32_t)nl;
        conflicts += nl;
        int32_t *t = U; U = L; L = t;
        nu = nl;
    }
    if (st) {
        st->iterations = iters;
        st->conflicts = conflicts;
        st->model_bytes = bytes;
        colour_counts(n, c, st);
    }
    free(snap); free(U); free(L); free(seen); free(mark);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Distance-2 colouring                                                 */
/* ------------------------------------------------------------------ */

/*
 * Distance-2 colouring asks two vertices joined by a path of one or two
 * edges to differ in colour: the colouring of G^2, whose edges are those
 * paths.  G^2 is not built: the two-hop neighbourhood D2(v) of v is read as
 * "every u adjacent to v, and every w != v adjacent to such a u" (a vertex
 * may be seen more than once; that changes nothing).
 *
 * Byte model of the distance-2 replay, per vertex inspected in a round:
 *   4 for its worklist entry (every round after the first), 8 for its two
 *   row pointers, 4 for its own colour, 16 per neighbour u (column index,
 *   colour, and u's two row pointers), 8 per entry of u's row (column index
 *   and colour), and 4 + 4 for the colour written and the push when it is
 *   recoloured.  The conflict test and the First-Fit set come from one scan
 *   of D2(v).  Round 0 colours every vertex 1: 4 bytes per vertex.
 */

/* Smallest colour >= 1 held by no coloured vertex of D2(v) in col, and
 * whether a vertex of D2(v) on v's tie side holds colour cv (cv = 0: no
 * test).  mark: scratch of at least d2max+2 entries. */
static int32_t d2_scan(int32_t v, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *col, int tie,
                       int32_t cv, int32_t d2max, int64_t *mark, int64_t stamp, int *conflict, int64_t *bytes)
{
    int c2 = 0;
    int64_t b = 16 * (int64_t)(row_ptr[v + 1] - row_ptr[v]);
    for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
        int32_t u = col_idx[k];
        int32_t cu = col[u];
        if (cu >= 1 && cu <= d2max + 1) mark[cu] = stamp;
        if (cv && cu == cv && loses_to(v, u, tie)) c2 = 1;
        b += 8 * (int64_t)(row_ptr[u + 1] - row_ptr[u]);
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t w = col_idx[j];
            if (w == v) continue;
            int32_t cw = col[w];
            if (cw >= 1 && cw <= d2max + 1) mark[cw] = stamp;
            if (cv && cw == cv && loses_to(v, w, tie)) c2 = 1;
        }
    }
    int32_t k = 1;
    while (mark[k] == stamp) ++k;
    if (conflict) *conflict = c2;
    if (bytes) *bytes += b;
    return k;
}

/* An upper bound of |D2(v)| over v: sum of the neighbours' degrees. */
static int32_t d2_bound(int32_t n, const int32_t *row_ptr, const int32_t *col_idx)
{
    int64_t best = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t s = 0;
        for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) s += row_ptr[col_idx[k] + 1] - row_ptr[col_idx[k]];
        if (s > best) best = s;
    }
    return best > INT32_MAX - 2 ? INT32_MAX - 2 : (int32_t)best;
}

/* Algorithm 1 over two-hop neighbourhoods, natural order. */
int32_t oracle_ff_d2(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t *c)
{
    if (n < 0) return -1;
    int32_t d2max = d2_bound(n, row_ptr, col_idx);
    int64_t *mark = (int64_t *)malloc(((size_t)d2max + 2) * sizeof(int64_t));
    if (!mark) return -1;
    for (int32_t k = 0; k < d2max + 2; ++k) mark[k] = -1;
    for (int32_t v = 0; v < n; ++v) c[v] = 0;
    int32_t used = 0;
    for (int32_t v = 0; v < n; ++v) {
        c[v] = d2_scan(v, row_ptr, col_idx, c, ORACLE_TIE_LOWER_KEEPS, 0, d2max, mark, v, NULL, NULL);
        if (c[v] > used) used = c[v];
    }
    free(mark);
    return used;
}

/* Algorithm 3 with snapshot reads over two-hop neighbourhoods (as
 * oracle_rsoc_det, "neighbour" meaning "vertex of D2(v)"). */
int oracle_rsoc_det_d2(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int tie, int64_t max_iters,
                       int32_t *c, oracle_stats *st)
{
    if (n < 0 || !c) return ORACLE_ERR_ARG;
    int32_t d2max = d2_bound(n, row_ptr, col_idx);
    int32_t *snap = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *U = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t *L = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t *mark = (int64_t *)malloc(((size_t)d2max + 2) * sizeof(int64_t));
    if (!snap || !U || !L || !mark) {
        free(snap); free(U); free(L); free(mark);
        return ORACLE_ERR_OOM;
    }
    for (int32_t k = 0; k < d2max + 2; ++k) mark[k] = -1;
    int64_t stamp = 0, bytes = 4 * (int64_t)n, iters = 0, conflicts = 0;
    for (int32_t v = 0; v < n; ++v) c[v] = 1;  /* round 0 over an uncoloured snapshot */
    int64_t nu = n;
    for (int32_t v = 0; v < n; ++v) U[v] = v;
    int first_pass = 1, rc = ORACLE_OK;
    while (nu > 0) {
        if (iters >= max_iters) { rc = ORACLE_ERR_NO_CONVERGENCE; break; }
        ++iters;
        memcpy(snap, c, (size_t)n * sizeof(int32_t));
        int64_t nl = 0;
        for (int64_t i = 0; i < nu; ++i) {
            int32_t v = U[i];
            int defective = 0;
            bytes += (first_pass ? 0 : 4) + 8 + 4;
            int32_t k = d2_scan(v, row_ptr, col_idx, snap, tie, snap[v], d2max, mark, stamp++, &defective, &bytes);
            if (defective) {
                c[v] = k;
                L[nl++] = v;
                bytes += 4 + 4;
            }
        }
        if (st && st->round_sizes && iters - 1 < st->round_sizes_cap)
            st->round_sizes[iters - 1] = (int32_t)nl;
        conflicts += nl;
        int32_t *t = U; U = L; L = t;
        nu = nl;
        first_pass = 0;
    }
    if (st) {
        st->iterations = iters;
        st->conflicts = conflicts;
        st->model_bytes = bytes;
        colour_counts(n, c, st);
    }
    free(snap); free(U); free(L); free(mark);
    return rc;
}

/* Validity at distance 2: 0, or 1 + the first vertex sharing its colour
 * with a vertex of D2(v) (or uncoloured). */
int64_t oracle_check_d2(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *c)
{
    for (int32_t v = 0; v < n; ++v) {
        if (c[v] < 1) return (int64_t)v + 1;
        for (int32_t k = row_ptr[v]; k < row_ptr[v + 1]; ++k) {
            int32_t u = col_idx[k];
            if (c[u] == c[v]) return (int64_t)v + 1;
            for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j)
                if (col_idx[j] != v && c[col_idx[j]] == c[v]) return (int64_t)v + 1;
        }
    }
    return 0;
}
