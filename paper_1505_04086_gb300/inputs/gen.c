/*
 * Seeded synthetic graph generators (input side only).
 *
 * This file builds the undirected test graphs that stand in for the paper's
 * benchmark inputs (Section 4: a 2D anisotropic CFD mesh, two 3D meshes from
 * the UF collection and 16M-vertex R-MAT graphs with shuffled ids).  None of
 * those files exist here, so every input is generated from a seed:
 *
 *   tri2d   structured 2D triangular mesh, one diagonal per cell
 *   jtri2d  jittered 2D triangular mesh (each cell cut along its shorter
 *           diagonal after the vertices are perturbed)
 *   kuhn3d  Kuhn/Freudenthal tetrahedralisation of an N^3 lattice
 *   rmat    R-MAT edge draws (Chakrabarti et al.), ids permuted
 *   rgg     random geometric graph in the unit square
 *
 * Output is always a symmetric CSR with int32 row pointers and column
 * indices, rows sorted ascending, no self-loops and no duplicate entries.
 *
 * The file holds no colouring arithmetic: it is shared by the tests, the
 * benchmark and (through the arrays it returns) both the CUDA path and the
 * CPU oracle, which never see each other.
 *
 * Random numbers come from the splitmix64 finaliser evaluated at a counter,
 * so every value depends only on (seed, counter) and not on call order or
 * thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The i-th output of a splitmix64 stream started at `seed`. */
uint64_t gcgen_rand_at(uint64_t seed, uint64_t i)
{
    return mix64(seed + (i + 1) * GOLDEN);
}

/* Uniform double in [0,1) from 53 random bits. */
static inline double u01(uint64_t seed, uint64_t i)
{
    return (double)(gcgen_rand_at(seed, i) >> 11) * (1.0 / 9007199254740992.0);
}

typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t *row_ptr; /* n+1 */
    int32_t *col_idx; /* nnz */
} gcgen_csr;

void gcgen_free(gcgen_csr *g)
{
    if (!g) return;
    free(g->row_ptr);
    free(g->col_idx);
    free(g);
}

/* ------------------------------------------------------------------ */
/* Edge list -> symmetric, sorted, de-duplicated CSR.                  */
/* ------------------------------------------------------------------ */

/*
 * Builds the CSR of the undirected graph with the given m edge pairs.
 * Self-loops are dropped, each edge is stored in both directions and
 * repeated entries are removed.  Rows come out sorted because the entries
 * are placed by a counting sort on the destination followed by a stable
 * scatter on the source.  Returns NULL on allocation failure.
 */
static gcgen_csr *csr_from_pairs(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev)
{
    gcgen_csr *g = (gcgen_csr *)calloc(1, sizeof(gcgen_csr));
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!g || !cnt) goto fail;

    /* Directed entries (a -> b) with a != b: count by destination. */
    int64_t nd = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (eu[e] == ev[e]) continue;
        cnt[ev[e] + 1]++;
        cnt[eu[e] + 1]++;
        nd += 2;
    }
    for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];

    /* by_dst[k] = source of the k-th entry in destination order */
    int32_t *by_dst = (int32_t *)malloc((size_t)(nd > 0 ? nd : 1) * sizeof(int32_t));
    int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!by_dst || !pos) { free(by_dst); free(pos); goto fail; }
    memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = eu[e], b = ev[e];
        if (a == b) continue;
        by_dst[pos[b]++] = a; /* entry a -> b */
        by_dst[pos[a]++] = b; /* entry b -> a */
    }

    /* Out-degree (with duplicates) of each source equals its in-degree by symmetry. */
    int64_t *rp = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t *col = (int32_t *)malloc((size_t)(nd > 0 ? nd : 1) * sizeof(int32_t));
    if (!rp || !col) { free(by_dst); free(pos); free(rp); free(col); goto fail; }
    memcpy(rp, cnt, ((size_t)n + 1) * sizeof(int64_t));
    memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
    /* Walk destinations in increasing order; each source row receives its
     * destinations in increasing order, so rows are sorted. */
    for (int32_t d = 0; d < n; ++d)
        for (int64_t k = cnt[d]; k < cnt[d + 1]; ++k) {
            int32_t s = by_dst[k];
            col[pos[s]++] = d;
        }
    free(by_dst);

    /* Remove repeats inside each (sorted) row and compact. */
    g->row_ptr = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!g->row_ptr) { free(pos); free(rp); free(col); goto fail; }
    int64_t w = 0;
    g->row_ptr[0] = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t b = rp[v], e = rp[v + 1];
        for (int64_t k = b; k < e; ++k)
            if (k == b || col[k] != col[k - 1]) col[w++] = col[k];
        if (w > INT32_MAX) { free(pos); free(rp); free(col); goto fail; }
        g->row_ptr[v + 1] = (int32_t)w;
    }
    free(pos);
    free(rp);
    g->n = n;
    g->nnz = w;
    /* shrink to the deduplicated size; on failure keep the larger block */
    int32_t *shrunk = (int32_t *)realloc(col, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
    g->col_idx = shrunk ? shrunk : col;
    free(cnt);
    return g;
fail:
    free(cnt);
    gcgen_free(g);
    return NULL;
}

/* Seeded Fisher-Yates permutation of 0..n-1 (perm[old] = new). */
static int32_t *make_perm(int32_t n, uint64_t seed)
{
    int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return NULL;
    for (int32_t i = 0; i < n; ++i) p[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        uint64_t r = gcgen_rand_at(seed ^ 0x5045524DULL, (uint64_t)i);
        int32_t j = (int32_t)(r % (uint64_t)(i + 1));
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
    return p;
}

void gcgen_perm(int32_t n, uint64_t seed, int32_t *out)
{
    int32_t *p = make_perm(n, seed);
    if (!p) return;
    memcpy(out, p, (size_t)n * sizeof(int32_t));
    free(p);
}

static void apply_perm(int64_t m, int32_t *eu, int32_t *ev, const int32_t *perm)
{
    for (int64_t e = 0; e < m; ++e) { eu[e] = perm[eu[e]]; ev[e] = perm[ev[e]]; }
}

/* ------------------------------------------------------------------ */
/* 2D structured / jittered triangular meshes                          */
/* ------------------------------------------------------------------ */

/*
 * rows x cols lattice, vertex (i,j) has id i*cols+j.  Horizontal and
 * vertical lattice edges plus one diagonal per cell.  diag selects it:
 *   0: every cell split by (i,j)-(i+1,j+1)
 *   1: vertices jittered by up to +-jitter (seeded) and each cell split by
 *      its shorter diagonal (ties go to (i,j)-(i+1,j+1)); topology then
 *      varies from cell to cell like an unstructured mesher's output.
 */
gcgen_csr *gcgen_tri2d(int32_t rows, int32_t cols, int diag, double jitter, uint64_t seed)
{
    if (rows < 1 || cols < 1 || (int64_t)rows * cols > INT32_MAX) return NULL;
    int32_t n = rows * cols;
    int64_t mmax = (int64_t)rows * (cols - 1) + (int64_t)(rows - 1) * cols + (int64_t)(rows - 1) * (cols - 1);
    int32_t *eu = (int32_t *)malloc((size_t)(mmax > 0 ? mmax : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(mmax > 0 ? mmax : 1) * sizeof(int32_t));
    double *x = NULL, *y = NULL;
    if (diag == 1) {
        x = (double *)malloc((size_t)n * sizeof(double));
        y = (double *)malloc((size_t)n * sizeof(double));
    }
    if (!eu || !ev || (diag == 1 && (!x || !y))) { free(eu); free(ev); free(x); free(y); return NULL; }
    if (diag == 1)
        for (int32_t v = 0; v < n; ++v) {
            int32_t i = v / cols, j = v % cols;
            x[v] = j + jitter * (2.0 * u01(seed, 2 * (uint64_t)v) - 1.0);
            y[v] = i + jitter * (2.0 * u01(seed, 2 * (uint64_t)v + 1) - 1.0);
        }
    int64_t m = 0;
    for (int32_t i = 0; i < rows; ++i)
        for (int32_t j = 0; j < cols; ++j) {
            int32_t v = i * cols + j;
            if (j + 1 < cols) { eu[m] = v; ev[m] = v + 1; ++m; }
            if (i + 1 < rows) { eu[m] = v; ev[m] = v + cols; ++m; }
            if (i + 1 < rows && j + 1 < cols) {
                int32_t a = v, b = v + cols + 1;     /* main diagonal */
                int32_t c = v + 1, d = v + cols;     /* anti diagonal */
                int use_anti = 0;
                if (diag == 1) {
                    double dm = (x[a] - x[b]) * (x[a] - x[b]) + (y[a] - y[b]) * (y[a] - y[b]);
                    double da = (x[c] - x[d]) * (x[c] - x[d]) + (y[c] - y[d]) * (y[c] - y[d]);
                    use_anti = da < dm;
                }
                if (use_anti) { eu[m] = c; ev[m] = d; }
                else { eu[m] = a; ev[m] = b; }
                ++m;
            }
        }
    free(x);
    free(y);
    gcgen_csr *g = csr_from_pairs(n, m, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/* ------------------------------------------------------------------ */
/* 3D Kuhn (Freudenthal) tetrahedralisation                            */
/* ------------------------------------------------------------------ */

/*
 * Lattice points (x,y,z) in [0,N)^3; each point is joined to p + e_S for
 * the seven non-empty S subset of {x,y,z} that stay inside the box.  These
 * are exactly the edges of the Kuhn subdivision of every unit cube into six
 * tetrahedra along the (1,1,1) diagonal.  Interior degree is 14.  If
 * permute is set, ids are relabelled by a seeded Fisher-Yates permutation.
 */
gcgen_csr *gcgen_kuhn3d(int32_t N, int permute, uint64_t seed)
{
    if (N < 1 || (int64_t)N * N * N > INT32_MAX) return NULL;
    int64_t n64 = (int64_t)N * N * N;
    int32_t n = (int32_t)n64;
    int64_t L = N, Lm = N - 1;
    int64_t mmax = 3 * Lm * L * L + 3 * Lm * Lm * L + Lm * Lm * Lm;
    int32_t *eu = (int32_t *)malloc((size_t)(mmax > 0 ? mmax : 1) * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)(mmax > 0 ? mmax : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return NULL; }
    static const int D[7][3] = {{1,0,0},{0,1,0},{0,0,1},{1,1,0},{1,0,1},{0,1,1},{1,1,1}};
    int64_t m = 0;
    for (int32_t x = 0; x < N; ++x)
        for (int32_t y = 0; y < N; ++y)
            for (int32_t z = 0; z < N; ++z) {
                int32_t v = (x * N + y) * N + z;
                for (int d = 0; d < 7; ++d) {
                    int32_t X = x + D[d][0], Y = y + D[d][1], Z = z + D[d][2];
                    if (X >= N || Y >= N || Z >= N) continue;
                    eu[m] = v;
                    ev[m] = (X * N + Y) * N + Z;
                    ++m;
                }
            }
    if (permute) {
        int32_t *p = make_perm(n, seed);
        if (!p) { free(eu); free(ev); return NULL; }
        apply_perm(m, eu, ev, p);
        free(p);
    }
    gcgen_csr *g = csr_from_pairs(n, m, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/* ------------------------------------------------------------------ */
/* R-MAT                                                               */
/* ------------------------------------------------------------------ */

/*
 * ef * 2^scale edge draws.  Edge e descends `scale` levels; at each level a
 * uniform 32-bit draw picks quadrant a (0,0), b (0,1), c (1,0) or d (1,1),
 * which fixes one bit of the source and destination.  Draw l of edge e is
 * half of the splitmix64 value at counter e*ceil(scale/2) + l/2.  No noise
 * is added.  Ids are relabelled by a seeded permutation when permute is set
 * (the paper shuffles its R-MAT vertex indices), then the edge set is
 * symmetrised with self-loops and repeats removed.  The draws run on up to
 * 16 POSIX threads; the result does not depend on the thread count.
 */
typedef struct {
    int64_t e0, e1;
    int32_t scale;
    uint32_t ta, tab, tabc;
    uint64_t seed;
    int32_t *eu, *ev;
} rmat_job;

static void *rmat_worker(void *arg)
{
    rmat_job *J = (rmat_job *)arg;
    const uint64_t per = (uint64_t)(J->scale + 1) / 2;
    for (int64_t e = J->e0; e < J->e1; ++e) {
        uint32_t s = 0, d = 0;
        uint64_t r = 0;
        for (int32_t l = 0; l < J->scale; ++l) {
            if ((l & 1) == 0) r = gcgen_rand_at(J->seed, (uint64_t)e * per + (uint64_t)(l >> 1));
            uint32_t x = (l & 1) ? (uint32_t)(r >> 32) : (uint32_t)r;
            uint32_t sb = x >= J->tab, db = (x >= J->ta && x < J->tab) || x >= J->tabc;
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        J->eu[e] = (int32_t)s;
        J->ev[e] = (int32_t)d;
    }
    return NULL;
}

static uint32_t prob_to_u32(double p)
{
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 0xFFFFFFFFu;
    return (uint32_t)(p * 4294967296.0);
}

gcgen_csr *gcgen_rmat(int32_t scale, int32_t ef, double a, double b, double c, uint64_t seed, int permute)
{
    if (scale < 1 || scale > 30 || ef < 1) return NULL;
    int32_t n = (int32_t)1 << scale;
    int64_t m = (int64_t)ef * n;
    int32_t *eu = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return NULL; }
    enum { NT = 16 };
    rmat_job jobs[NT];
    pthread_t th[NT];
    int started[NT];
    for (int t = 0; t < NT; ++t) {
        jobs[t].e0 = m * t / NT;
        jobs[t].e1 = m * (t + 1) / NT;
        jobs[t].scale = scale;
        jobs[t].ta = prob_to_u32(a);
        jobs[t].tab = prob_to_u32(a + b);
        jobs[t].tabc = prob_to_u32(a + b + c);
        jobs[t].seed = seed;
        jobs[t].eu = eu;
        jobs[t].ev = ev;
        started[t] = pthread_create(&th[t], NULL, rmat_worker, &jobs[t]) == 0;
        if (!started[t]) rmat_worker(&jobs[t]);
    }
    for (int t = 0; t < NT; ++t)
        if (started[t]) pthread_join(th[t], NULL);
    if (permute) {
        int32_t *p = make_perm(n, seed);
        if (!p) { free(eu); free(ev); return NULL; }
        apply_perm(m, eu, ev, p);
        free(p);
    }
    gcgen_csr *g = csr_from_pairs(n, m, eu, ev);
    free(eu);
    free(ev);
    return g;
}

/* ------------------------------------------------------------------ */
/* Random geometric graph                                              */
/* ------------------------------------------------------------------ */

/*
 * n points uniform in the unit square; u~v iff their distance is below
 * r = sqrt(mean_deg / (pi n)), which gives the requested mean degree away
 * from the boundary.  Neighbour search uses a uniform cell grid of side >= r.
 */
gcgen_csr *gcgen_rgg(int32_t n, double mean_deg, uint64_t seed)
{
    if (n < 1) return NULL;
    double r = sqrt(mean_deg / (M_PI * (double)n));
    double r2 = r * r;
    int32_t G = (int32_t)floor(1.0 / r);
    if (G < 1) G = 1;
    if (G > 65536) G = 65536;
    double *px = (double *)malloc((size_t)n * sizeof(double));
    double *py = (double *)malloc((size_t)n * sizeof(double));
    int64_t ncell = (int64_t)G * G;
    int32_t *cstart = (int32_t *)calloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t *cell_of = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *sorted = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!px || !py || !cstart || !cell_of || !sorted) goto oom;
    for (int32_t v = 0; v < n; ++v) {
        px[v] = u01(seed, 2 * (uint64_t)v);
        py[v] = u01(seed, 2 * (uint64_t)v + 1);
        int32_t cx = (int32_t)(px[v] * G), cy = (int32_t)(py[v] * G);
        if (cx >= G) cx = G - 1;
        if (cy >= G) cy = G - 1;
        cell_of[v] = cy * G + cx;
        cstart[cell_of[v] + 1]++;
    }
    for (int64_t k = 0; k < ncell; ++k) cstart[k + 1] += cstart[k];
    {
        int32_t *fill = (int32_t *)malloc((size_t)ncell * sizeof(int32_t));
        if (!fill) goto oom;
        memcpy(fill, cstart, (size_t)ncell * sizeof(int32_t));
        for (int32_t v = 0; v < n; ++v) sorted[fill[cell_of[v]]++] = v;
        free(fill);
    }
    int64_t cap = (int64_t)n * 8 + 16, m = 0;
    int32_t *eu = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    int32_t *ev = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); goto oom; }
    for (int32_t v = 0; v < n; ++v) {
        int32_t cx = cell_of[v] % G, cy = cell_of[v] / G;
        for (int32_t dy = -1; dy <= 1; ++dy)
            for (int32_t dx = -1; dx <= 1; ++dx) {
                int32_t X = cx + dx, Y = cy + dy;
                if (X < 0 || Y < 0 || X >= G || Y >= G) continue;
                int64_t cc = (int64_t)Y * G + X;
                for (int32_t k = cstart[cc]; k < cstart[cc + 1]; ++k) {
                    int32_t u = sorted[k];
                    if (u <= v) continue;
                    double ddx = px[u] - px[v], ddy = py[u] - py[v];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (m == cap) {
                            cap *= 2;
                            int32_t *nu = (int32_t *)realloc(eu, (size_t)cap * sizeof(int32_t));
                            if (!nu) { free(eu); free(ev); goto oom; }
                            eu = nu;
                            int32_t *nv = (int32_t *)realloc(ev, (size_t)cap * sizeof(int32_t));
                            if (!nv) { free(eu); free(ev); goto oom; }
                            ev = nv;
                        }
                        eu[m] = v;
                        ev[m] = u;
                        ++m;
                    }
                }
            }
    }
    free(px); free(py); free(cstart); free(cell_of); free(sorted);
    gcgen_csr *g = csr_from_pairs(n, m, eu, ev);
    free(eu);
    free(ev);
    return g;
oom:
    free(px); free(py); free(cstart); free(cell_of); free(sorted);
    return NULL;
}

/* ------------------------------------------------------------------ */
/* Batch of uneven graphs                                              */
/* ------------------------------------------------------------------ */

/*
 * G graphs with vertex counts log-uniform in [nmin, nmax]; each is, with
 * equal odds, a jittered triangular mesh (rows*cols ~ n) or a random
 * geometric graph of mean degree `rgg_deg`.  Graph g's parameters depend
 * only on (seed, g).  Generated on `threads` POSIX threads.
 *
 * Output layout (all caller-visible through gcgen_batch_*):
 *   vtx_off[G+1], edge_off[G+1] (int64 prefix sums of n_g and nnz_g)
 *   row_ptr: graph g's local row pointers (n_g+1 entries) start at
 *            vtx_off[g] + g
 *   col_idx: graph g's local column indices start at edge_off[g]
 *   kind[g]: 0 mesh, 1 rgg
 */
typedef struct {
    int32_t G;
    int64_t *vtx_off;
    int64_t *edge_off;
    int32_t *row_ptr;
    int32_t *col_idx;
    int32_t *kind;
} gcgen_batch;

typedef struct {
    int32_t G, nmin, nmax, next;
    double rgg_deg, jitter;
    uint64_t seed;
    gcgen_csr **parts;
    int32_t *kind;
    pthread_mutex_t mu;
    int failed;
} batch_job;

static void batch_one(batch_job *J, int32_t g)
{
    uint64_t gs = mix64(J->seed ^ (0xBA7C4ULL + (uint64_t)g * GOLDEN));
    double lo = log((double)J->nmin), hi = log((double)J->nmax);
    int32_t n = (int32_t)floor(exp(lo + (hi - lo) * u01(gs, 0)));
    if (n < J->nmin) n = J->nmin;
    if (n > J->nmax) n = J->nmax;
    int k = (int)(gcgen_rand_at(gs, 1) & 1);
    gcgen_csr *c;
    if (k == 0) {
        int32_t rows = (int32_t)floor(sqrt((double)n) + 0.5);
        if (rows < 1) rows = 1;
        int32_t cols = (n + rows / 2) / rows;
        if (cols < 1) cols = 1;
        c = gcgen_tri2d(rows, cols, 1, J->jitter, gs);
    } else {
        c = gcgen_rgg(n, J->rgg_deg, gs);
    }
    J->parts[g] = c;
    J->kind[g] = k;
    if (!c) J->failed = 1;
}

static void *batch_worker(void *arg)
{
    batch_job *J = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int32_t g = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (g >= J->G) break;
        batch_one(J, g);
    }
    return NULL;
}

void gcgen_batch_free(gcgen_batch *b)
{
    if (!b) return;
    free(b->vtx_off); free(b->edge_off); free(b->row_ptr); free(b->col_idx); free(b->kind);
    free(b);
}

gcgen_batch *gcgen_batch_make(int32_t G, int32_t nmin, int32_t nmax, double rgg_deg, double jitter,
                              uint64_t seed, int32_t threads)
{
    if (G < 1 || nmin < 1 || nmax < nmin) return NULL;
    batch_job J;
    memset(&J, 0, sizeof J);
    J.G = G; J.nmin = nmin; J.nmax = nmax; J.rgg_deg = rgg_deg; J.jitter = jitter; J.seed = seed;
    J.parts = (gcgen_csr **)calloc((size_t)G, sizeof(gcgen_csr *));
    J.kind = (int32_t *)calloc((size_t)G, sizeof(int32_t));
    gcgen_batch *b = (gcgen_batch *)calloc(1, sizeof(gcgen_batch));
    if (!J.parts || !J.kind || !b) { free(J.parts); free(J.kind); free(b); return NULL; }
    pthread_mutex_init(&J.mu, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < threads; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &J) == 0) ++started;
    if (started == 0) batch_worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);

    b->G = G;
    b->kind = J.kind;
    b->vtx_off = (int64_t *)malloc(((size_t)G + 1) * sizeof(int64_t));
    b->edge_off = (int64_t *)malloc(((size_t)G + 1) * sizeof(int64_t));
    if (J.failed || !b->vtx_off || !b->edge_off) goto fail;
    b->vtx_off[0] = 0;
    b->edge_off[0] = 0;
    for (int32_t g = 0; g < G; ++g) {
        b->vtx_off[g + 1] = b->vtx_off[g] + J.parts[g]->n;
        b->edge_off[g + 1] = b->edge_off[g] + J.parts[g]->nnz;
    }
    b->row_ptr = (int32_t *)malloc(((size_t)b->vtx_off[G] + (size_t)G) * sizeof(int32_t));
    b->col_idx = (int32_t *)malloc((size_t)(b->edge_off[G] > 0 ? b->edge_off[G] : 1) * sizeof(int32_t));
    if (!b->row_ptr || !b->col_idx) goto fail;
    for (int32_t g = 0; g < G; ++g) {
        gcgen_csr *c = J.parts[g];
        memcpy(b->row_ptr + b->vtx_off[g] + g, c->row_ptr, ((size_t)c->n + 1) * sizeof(int32_t));
        memcpy(b->col_idx + b->edge_off[g], c->col_idx, (size_t)c->nnz * sizeof(int32_t));
        gcgen_free(c);
        J.parts[g] = NULL;
    }
    free(J.parts);
    return b;
fail:
    for (int32_t g = 0; g < G; ++g) gcgen_free(J.parts[g]);
    free(J.parts);
    gcgen_batch_free(b);
    return NULL;
}

/* Accessors, so that the Python side needs no struct layout. */
int32_t gcgen_n(const gcgen_csr *g) { return g->n; }
int64_t gcgen_nnz(const gcgen_csr *g) { return g->nnz; }
const int32_t *gcgen_row_ptr(const gcgen_csr *g) { return g->row_ptr; }
const int32_t *gcgen_col_idx(const gcgen_csr *g) { return g->col_idx; }
int32_t gcgen_batch_G(const gcgen_batch *b) { return b->G; }
const int64_t *gcgen_batch_vtx_off(const gcgen_batch *b) { return b->vtx_off; }
const int64_t *gcgen_batch_edge_off(const gcgen_batch *b) { return b->edge_off; }
const int32_t *gcgen_batch_row_ptr(const gcgen_batch *b) { return b->row_ptr; }
const int32_t *gcgen_batch_col_idx(const gcgen_batch *b) { return b->col_idx; }
const int32_t *gcgen_batch_kind(const gcgen_batch *b) { return b->kind; }
