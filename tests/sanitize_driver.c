/*
 * Host sanitizer run of the CPU oracle and the input generators: built by
 * tests/test_sanitizers.py with AddressSanitizer and UndefinedBehavior-
 * Sanitizer, it runs every oracle routine on generated and hand-made graphs
 * (and the CSR check on malformed ones) and exits non-zero on any failed
 * expectation; the sanitizers abort on any memory or UB error.
 */
#include "oracle.c"

#include <stdio.h>

typedef struct gcgen_csr gcgen_csr;
typedef struct gcgen_batch gcgen_batch;
gcgen_csr *gcgen_tri2d(int32_t rows, int32_t cols, int diag, double jitter, uint64_t seed);
gcgen_csr *gcgen_kuhn3d(int32_t N, int permute, uint64_t seed);
gcgen_csr *gcgen_rmat(int32_t scale, int32_t ef, double a, double b, double c, uint64_t seed, int permute);
gcgen_csr *gcgen_rgg(int32_t n, double mean_deg, uint64_t seed);
void gcgen_free(gcgen_csr *g);
int32_t gcgen_n(const gcgen_csr *g);
int64_t gcgen_nnz(const gcgen_csr *g);
const int32_t *gcgen_row_ptr(const gcgen_csr *g);
const int32_t *gcgen_col_idx(const gcgen_csr *g);
gcgen_batch *gcgen_batch_make(int32_t G, int32_t nmin, int32_t nmax, double rgg_deg, double jitter,
                              uint64_t seed, int32_t threads);
void gcgen_batch_free(gcgen_batch *b);
int32_t gcgen_batch_G(const gcgen_batch *b);
const int64_t *gcgen_batch_vtx_off(const gcgen_batch *b);
const int64_t *gcgen_batch_edge_off(const gcgen_batch *b);
const int32_t *gcgen_batch_row_ptr(const gcgen_batch *b);
const int32_t *gcgen_batch_col_idx(const gcgen_batch *b);

static int failures = 0;

#define EXPECT(cond, what)                                                  \
    do {                                                                    \
        if (!(cond)) {                                                      \
            fprintf(stderr, "FAILED: %s (%s:%d)\n", what, __FILE__, __LINE__); \
            ++failures;                                                     \
        }                                                                   \
    } while (0)

static int64_t two_hop(int32_t n, const int32_t *rp, const int32_t *ci)
{
    int64_t s = 0;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t k = rp[v]; k < rp[v + 1]; ++k) s += rp[ci[k] + 1] - rp[ci[k]];
    return s;
}

static void exercise(const char *name, int32_t n, const int32_t *rp, const int32_t *ci)
{
    int32_t *a = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *b = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *all = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    int32_t mx = 0, dist = 0;
    int32_t rs1[4096], rs2[4096];
    oracle_stats s1 = {0}, s2 = {0};
    fprintf(stderr, "graph %s: n=%d nnz=%d\n", name, n, n ? rp[n] : 0);
    EXPECT(oracle_csr_check(n, n ? rp[n] : 0, rp, ci) == 0, "well-formed input accepted");
    EXPECT(oracle_ff(n, rp, ci, a) >= 0, "first fit");
    EXPECT(oracle_check(n, rp, ci, a, &mx, &dist) == 0, "first fit valid");
    for (int tie = 0; tie < 2; ++tie) {
        s1.round_sizes = rs1;
        s1.round_sizes_cap = 4096;
        s2.round_sizes = rs2;
        s2.round_sizes_cap = 4096;
        EXPECT(oracle_rsoc_det(n, rp, ci, tie, (int64_t)n + 1, a, &s1) == ORACLE_OK, "rsoc replay");
        EXPECT(oracle_check(n, rp, ci, a, &mx, &dist) == 0, "rsoc replay valid");
        EXPECT(oracle_2p_det(n, rp, ci, tie, (int64_t)n + 1, b, &s2) == ORACLE_OK, "two-phase replay");
        EXPECT(memcmp(a, b, (size_t)n * sizeof(int32_t)) == 0, "rsoc and two-phase replays agree");
        EXPECT(s1.iterations == s2.iterations && s1.conflicts == s2.conflicts, "same iterations and conflicts");
        for (int32_t v = 0; v < n; ++v) all[v] = v;
        for (int32_t v = 0; v < n; ++v) b[v] = 1;
        EXPECT(oracle_rsoc_det_from(n, rp, ci, tie, (int64_t)n + 1, all, n, b, &s2) == ORACLE_OK,
               "replay from all ones");
        EXPECT(memcmp(a, b, (size_t)n * sizeof(int32_t)) == 0, "replay from all ones equals the replay");
    }
    int rc = oracle_rsoc_det(n, rp, ci, ORACLE_TIE_NONE, 5, b, NULL);
    EXPECT(rc == ORACLE_OK || rc == ORACLE_ERR_NO_CONVERGENCE, "no tie-break under a cap");
    {
        int32_t *ptr = (int32_t *)calloc((size_t)mx + 2, sizeof(int32_t));
        int32_t *verts = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
        EXPECT(oracle_classes(n, a, mx, ptr, verts) >= 0, "colour classes");
        free(ptr);
        free(verts);
    }
    if (n <= 12) EXPECT(oracle_chi(n, rp, ci) >= 0, "chromatic number");
    if (two_hop(n, rp, ci) <= 2000000) {
        EXPECT(oracle_ff_d2(n, rp, ci, a) >= 0, "distance-2 first fit");
        EXPECT(oracle_check_d2(n, rp, ci, a) == 0, "distance-2 first fit valid");
        if (n <= 4096)
            for (int tie = 0; tie < 2; ++tie) {
                EXPECT(oracle_rsoc_det_d2(n, rp, ci, tie, (int64_t)n + 1, b, NULL) == ORACLE_OK,
                       "distance-2 replay");
                EXPECT(oracle_check_d2(n, rp, ci, b) == 0, "distance-2 replay valid");
            }
    }
    free(a);
    free(b);
    free(all);
}

static void exercise_gen(const char *name, gcgen_csr *g)
{
    EXPECT(g != NULL, "generator");
    if (!g) return;
    exercise(name, gcgen_n(g), gcgen_row_ptr(g), gcgen_col_idx(g));
    gcgen_free(g);
}

int main(void)
{
    exercise_gen("tri2d", gcgen_tri2d(10, 12, 1, 0.3, 7));
    exercise_gen("kuhn3d", gcgen_kuhn3d(6, 1, 8));
    exercise_gen("rmat", gcgen_rmat(9, 16, 0.57, 0.19, 0.19, 9, 1));
    exercise_gen("rgg", gcgen_rgg(500, 12.0, 10));
    {
        gcgen_batch *bt = gcgen_batch_make(8, 16, 2048, 12.0, 0.3, 11, 4);
        EXPECT(bt != NULL, "batch generator");
        if (bt) {
            const int64_t *vo = gcgen_batch_vtx_off(bt), *eo = gcgen_batch_edge_off(bt);
            const int32_t *rp = gcgen_batch_row_ptr(bt), *ci = gcgen_batch_col_idx(bt);
            for (int32_t g = 0; g < gcgen_batch_G(bt); ++g)
                exercise("batch graph", (int32_t)(vo[g + 1] - vo[g]), rp + vo[g] + g, ci + eo[g]);
            gcgen_batch_free(bt);
        }
    }
    {
        const int32_t rp0[1] = {0};
        exercise("empty", 0, rp0, rp0);
        const int32_t rp1[2] = {0, 0};
        exercise("one vertex", 1, rp1, rp1);
        /* star K_{1,5} and the clique K_5 */
        const int32_t srp[7] = {0, 5, 6, 7, 8, 9, 10};
        const int32_t sci[10] = {1, 2, 3, 4, 5, 0, 0, 0, 0, 0};
        exercise("star", 6, srp, sci);
        int32_t krp[6], kci[20];
        for (int v = 0, k = 0; v < 5; ++v) {
            krp[v] = k;
            for (int u = 0; u < 5; ++u)
                if (u != v) kci[k++] = u;
            krp[v + 1] = k;
        }
        exercise("clique", 5, krp, kci);
    }
    {
        /* malformed inputs the CSR check must reject */
        const int32_t rp[4] = {0, 1, 2, 2};
        const int32_t out_of_range[2] = {1, 7};
        const int32_t self_loop[2] = {0, 0};
        const int32_t asym[2] = {1, 2};
        EXPECT(oracle_csr_check(3, 2, rp, out_of_range) != 0, "out-of-range index rejected");
        EXPECT(oracle_csr_check(3, 2, rp, self_loop) != 0, "self loop rejected");
        EXPECT(oracle_csr_check(3, 2, rp, asym) != 0, "asymmetric entry rejected");
        const int32_t rp2[3] = {0, 2, 4};
        const int32_t unsorted[4] = {1, 1, 0, 0};
        EXPECT(oracle_csr_check(2, 4, rp2, unsorted) != 0, "repeated entry rejected");
    }
    if (failures) fprintf(stderr, "%d expectation(s) failed\n", failures);
    else fprintf(stderr, "all expectations met\n");
    return failures ? 1 : 0;
}
