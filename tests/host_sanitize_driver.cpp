// Host AddressSanitizer / UndefinedBehaviorSanitizer run of the paper's
// OpenMP form (gc_host_color): every mode on generated graphs (distance 2
// too, on the small meshes), several thread counts, the library's own check
// of each result (GC_CHECKED).
#include <cstdio>
#include <cstdint>
#include <initializer_list>

#include "gc.h"

extern "C" {
struct gcgen_csr;
gcgen_csr *gcgen_tri2d(int32_t rows, int32_t cols, int diag, double jitter, uint64_t seed);
gcgen_csr *gcgen_kuhn3d(int32_t N, int permute, uint64_t seed);
gcgen_csr *gcgen_rmat(int32_t scale, int32_t ef, double a, double b, double c, uint64_t seed, int permute);
gcgen_csr *gcgen_rgg(int32_t n, double mean_deg, uint64_t seed);
void gcgen_free(gcgen_csr *g);
int32_t gcgen_n(const gcgen_csr *g);
int64_t gcgen_nnz(const gcgen_csr *g);
const int32_t *gcgen_row_ptr(const gcgen_csr *g);
const int32_t *gcgen_col_idx(const gcgen_csr *g);
}

int main()
{
    int failures = 0;
    gcgen_csr *gs[] = {gcgen_tri2d(30, 30, 1, 0.3, 3), gcgen_kuhn3d(10, 1, 4), gcgen_rmat(11, 16, 0.57, 0.19, 0.19, 5, 1),
                       gcgen_rgg(3000, 12.0, 6)};
    const uint32_t modes[] = {0, GC_ALG_TWO_PHASE, GC_SCHED_ASYNC, GC_SCHED_ASYNC | GC_ALG_TWO_PHASE,
                              GC_SCHED_ASYNC | GC_TIE_HIGHER_KEEPS, GC_TIE_HIGHER_KEEPS};
    for (gcgen_csr *g : gs) {
        if (!g) {
            ++failures;
            continue;
        }
        const int32_t n = gcgen_n(g);
        gc_csr csr{gcgen_row_ptr(g), gcgen_col_idx(g)};
        int32_t *col = new int32_t[n > 0 ? n : 1];
        int32_t rs[256];
        const bool small = n <= 1100;  // distance 2 on the small meshes only
        for (uint32_t m : modes)
            for (uint32_t d2 : {0u, (uint32_t)GC_DIST2})
                for (int t : {1, 3, 8}) {
                    if (d2 && !small) continue;
                    gc_stats st{};
                    st.round_sizes = rs;
                    st.round_sizes_cap = 256;
                    const int rc = gc_host_color(&csr, n, gcgen_nnz(g), m | d2 | GC_CHECKED, t, col, &st);
                    if (rc != GC_OK) {
                        std::fprintf(stderr, "FAILED: mode %u threads %d status %d\n", m | d2, t, rc);
                        ++failures;
                    }
                }
        delete[] col;
        gcgen_free(g);
    }
    gc_csr none{nullptr, nullptr};
    if (gc_host_color(&none, 4, 0, 0, 2, nullptr, nullptr) != GC_ERR_ARG) ++failures;  // null arrays
    std::fprintf(stderr, failures ? "%d failure(s)\n" : "all expectations met\n", failures);
    return failures ? 1 : 0;
}
