// The method in the paper's own form: OpenMP threads on the host cores
// (Sec. 3; the paper measures it on multicore CPUs in Sec. 4).  Every loop
// over the worklist U is a parallel for with dynamic scheduling; the end of
// each loop is the barrier of Algorithms 2 and 3.
//
//   asynchronous RSOC (Algorithm 3): round 0 colours V by First-Fit in
//     place, then every iteration inspects U in place: a vertex that shares
//     its colour with a neighbour on its tie side is recoloured at once
//     (First-Fit over all its neighbours' current colours) and joins L.
//   asynchronous two-phase (Algorithm 2): every iteration recolours all of
//     U in place (tentative phase), then, after the barrier, puts on L the
//     vertices of U that share a colour with a neighbour on their tie side.
//   deterministic forms: the same steps, each loop reading the colours of
//     the end of the loop before (new colours are kept per worklist entry
//     and written after the loop), so the result does not depend on the
//     thread count or the schedule.
//
// Colours are read and written with relaxed atomics: in the asynchronous
// forms threads race on them by design, as the paper's threads do.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "gc.h"
#include "gc_nvtx.h"

namespace {

constexpr uint32_t kHostModes = GC_ALG_TWO_PHASE | GC_SCHED_ASYNC | GC_TIE_HIGHER_KEEPS | GC_VALIDATE | GC_CHECKED |
                                GC_NO_COLOR_STATS | GC_DIST2;

// GC_VALIDATE: the input format every loop relies on -- row pointers from 0
// to nnz without decreasing, indices in 0..n-1, rows strictly ascending
// (the tie-side scans read a prefix or suffix), no self-loops, and every
// entry (v,u) mirrored by (u,v).  Reads row pointers before the entries
// they bound, so malformed input is never read out of bounds.
bool valid_csr(const int32_t *rp, const int32_t *ci, int32_t n, int64_t nnz)
{
    if (rp[0] != 0 || rp[n] != nnz) return false;
    for (int32_t v = 0; v < n; ++v)
        if (rp[v + 1] < rp[v]) return false;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
            const int32_t u = ci[k];
            if (u < 0 || u >= n || u == v) return false;
            if (k > rp[v] && ci[k - 1] >= u) return false;
        }
    for (int32_t v = 0; v < n; ++v)
        for (int32_t k = rp[v]; k < rp[v + 1]; ++k) {
            const int32_t u = ci[k];
            if (!std::binary_search(ci + rp[u], ci + rp[u + 1], v)) return false;
        }
    return true;
}

inline int32_t ld(const int32_t *p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
inline void st(int32_t *p, int32_t v) { __atomic_store_n(p, v, __ATOMIC_RELAXED); }

struct Graph {
    const int32_t *rp;
    const int32_t *ci;
    int32_t n;
    bool higher_keeps;
    bool dist2;  // neighbourhood = two-hop neighbourhood D2(v) (GC_DIST2)
    // whether a clash of v with u is v's to repair
    bool tie_side(int32_t u, int32_t v) const { return higher_keeps ? u > v : u < v; }
};

// Per-thread forbidden-colour marks: stamp[c] == cur means colour c is taken.
struct Marks {
    std::vector<int64_t> stamp;
    int64_t cur = 0;
};

// Smallest colour >= 1 held by no neighbour of v in col (with dist2: by no
// vertex of D2(v), the neighbours u of v and every w != v adjacent to one).
int32_t first_fit(const Graph &g, int32_t v, const int32_t *col, Marks &m)
{
    const int64_t top = (int64_t)m.stamp.size() - 1;  // a free colour lies in 1..top
    ++m.cur;
    for (int32_t k = g.rp[v]; k < g.rp[v + 1]; ++k) {
        const int32_t u = g.ci[k];
        const int32_t c = ld(col + u);
        if (c >= 1 && c <= top) m.stamp[c] = m.cur;
        if (!g.dist2) continue;
        for (int32_t j = g.rp[u]; j < g.rp[u + 1]; ++j) {
            const int32_t w = g.ci[j];
            if (w == v) continue;
            const int32_t cw = ld(col + w);
            if (cw >= 1 && cw <= top) m.stamp[cw] = m.cur;
        }
    }
    int32_t k = 1;
    while (m.stamp[k] == m.cur) ++k;
    return k;
}

// Whether a neighbour (dist2: a vertex of D2(v)) of v on its tie side holds
// colour cv in col.
bool clashes(const Graph &g, int32_t v, int32_t cv, const int32_t *col)
{
    if (!g.dist2) {
        // rows are sorted: the tie side is a prefix (lower ids) or a suffix
        if (!g.higher_keeps) {
            for (int32_t k = g.rp[v]; k < g.rp[v + 1] && g.ci[k] < v; ++k)
                if (ld(col + g.ci[k]) == cv) return true;
        } else {
            for (int32_t k = g.rp[v + 1] - 1; k >= g.rp[v] && g.ci[k] > v; --k)
                if (ld(col + g.ci[k]) == cv) return true;
        }
        return false;
    }
    for (int32_t k = g.rp[v]; k < g.rp[v + 1]; ++k) {
        const int32_t u = g.ci[k];
        if (g.tie_side(u, v) && ld(col + u) == cv) return true;
        if (!g.dist2) continue;
        for (int32_t j = g.rp[u]; j < g.rp[u + 1]; ++j) {
            const int32_t w = g.ci[j];
            if (w != v && g.tie_side(w, v) && ld(col + w) == cv) return true;
        }
    }
    return false;
}

int threads_for(int32_t req)
{
#ifdef _OPENMP
    return req > 0 ? req : omp_get_max_threads();
#else
    (void)req;
    return 1;
#endif
}

int thread_id()
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

// Concatenate the threads' pushes into L (thread order).
int64_t gather(std::vector<std::vector<int32_t>> &local, std::vector<int32_t> &L)
{
    size_t total = 0;
    for (auto &x : local) total += x.size();
    L.resize(total);
    size_t o = 0;
    for (auto &x : local) {
        if (!x.empty()) memcpy(L.data() + o, x.data(), x.size() * sizeof(int32_t));
        o += x.size();
        x.clear();
    }
    return (int64_t)total;
}

struct Run {
    int64_t iters = 0, conflicts = 0;
    std::vector<int32_t> sizes;
    bool capped = false;
};

// top: the largest colour First-Fit can return (the largest neighbourhood
// + 1).
void color_host(const Graph &g, uint32_t mode, int T, int32_t *c, int64_t top, Run &r)
{
    const int32_t n = g.n;
    const bool async = mode & GC_SCHED_ASYNC;
    const bool twop = mode & GC_ALG_TWO_PHASE;
    std::vector<Marks> marks(T);
    for (auto &m : marks) m.stamp.assign((size_t)top + 1, 0);
    std::vector<std::vector<int32_t>> local(T);
    std::vector<int32_t> U, L, fresh;  // fresh: deterministic forms, new colour per worklist entry
    std::vector<char> flag;
    bool all = true;                   // U = V (not materialised)
    int64_t nu = n;

    // RSOC round 0 (two-phase starts uncoloured: its first tentative phase
    // is the same First-Fit over V)
#pragma omp parallel for num_threads(T) schedule(static)
    for (int32_t v = 0; v < n; ++v) st(c + v, (!twop && !async) ? 1 : 0);
    if (!twop && async) {
#pragma omp parallel for num_threads(T) schedule(dynamic, 256)
        for (int32_t v = 0; v < n; ++v) st(c + v, first_fit(g, v, c, marks[thread_id()]));
    }

    const int64_t cap = (int64_t)n + 1;
    while (nu > 0) {
        if (r.iters >= cap) {
            r.capped = true;
            break;
        }
        ++r.iters;
        if (!async) fresh.resize((size_t)nu);
        if (twop) {
            // tentative phase over U
#pragma omp parallel for num_threads(T) schedule(dynamic, 256)
            for (int64_t i = 0; i < nu; ++i) {
                const int32_t v = all ? (int32_t)i : U[i];
                const int32_t k = first_fit(g, v, c, marks[thread_id()]);
                if (async) st(c + v, k);
                else fresh[i] = k;
            }
            if (!async) {
#pragma omp parallel for num_threads(T) schedule(static)
                for (int64_t i = 0; i < nu; ++i) st(c + (all ? (int32_t)i : U[i]), fresh[i]);
            }
            // detection phase over U
#pragma omp parallel for num_threads(T) schedule(dynamic, 256)
            for (int64_t i = 0; i < nu; ++i) {
                const int32_t v = all ? (int32_t)i : U[i];
                if (clashes(g, v, ld(c + v), c)) local[thread_id()].push_back(v);
            }
        } else {
            // fused detect-and-recolour over U
            if (!async) flag.assign((size_t)nu, 0);
#pragma omp parallel for num_threads(T) schedule(dynamic, 256)
            for (int64_t i = 0; i < nu; ++i) {
                const int32_t v = all ? (int32_t)i : U[i];
                if (!clashes(g, v, ld(c + v), c)) continue;
                const int32_t k = first_fit(g, v, c, marks[thread_id()]);
                if (async) {
                    st(c + v, k);
                    local[thread_id()].push_back(v);
                } else {
                    fresh[i] = k;
                    flag[i] = 1;
                }
            }
            if (!async) {
                for (int64_t i = 0; i < nu; ++i)
                    if (flag[i]) {
                        const int32_t v = all ? (int32_t)i : U[i];
                        st(c + v, fresh[i]);
                        local[0].push_back(v);
                    }
            }
        }
        const int64_t nl = gather(local, L);
        r.sizes.push_back((int32_t)nl);
        r.conflicts += nl;
        U.swap(L);
        nu = nl;
        all = false;
    }
}

}  // namespace

extern "C" int gc_host_threads(void) { return threads_for(0); }

extern "C" int gc_host_color(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, int32_t num_threads,
                             int32_t *colors_out, gc_stats *stats_out)
{
    gc::NvtxRange nvtx_range("gc_host_color");
    if (!csr || n < 0 || nnz < 0 || nnz > INT32_MAX || num_threads < 0 || (mode & ~kHostModes)) return GC_ERR_ARG;
    if (n > 0 && (!csr->row_ptr || !colors_out)) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    if ((mode & GC_VALIDATE) && n > 0 && !valid_csr(csr->row_ptr, csr->col_idx, n, nnz)) return GC_ERR_GRAPH;
    const Graph g{csr->row_ptr, csr->col_idx, n, (mode & GC_TIE_HIGHER_KEEPS) != 0, (mode & GC_DIST2) != 0};
    // the largest neighbourhood: degree, or two-hop entries (sum of the
    // neighbours' degrees) with GC_DIST2
    int64_t widest = 0;
    for (int32_t v = 0; v < n; ++v) {
        int64_t w = g.rp[v + 1] - g.rp[v];
        if (g.dist2) {
            w = 0;
            for (int32_t k = g.rp[v]; k < g.rp[v + 1]; ++k) w += g.rp[g.ci[k] + 1] - g.rp[g.ci[k]];
        }
        widest = std::max(widest, w);
    }
    if (widest > INT32_MAX - 2) return GC_ERR_ARG;
    const int T = threads_for(num_threads);
    Run r;
    const auto t0 = std::chrono::steady_clock::now();
    try {
        // colours never exceed the neighbourhood size + 1, nor n
        if (n > 0) color_host(g, mode, T, colors_out, std::min<int64_t>(widest, n) + 1, r);
    } catch (const std::bad_alloc &) {
        return GC_ERR_OOM;
    }
    const auto t1 = std::chrono::steady_clock::now();
    int status = r.capped ? GC_ERR_NO_CONVERGENCE : GC_OK;
    if (status == GC_OK && (mode & GC_CHECKED)) {
        for (int32_t v = 0; v < n && status == GC_OK; ++v) {
            const int32_t cv = colors_out[v];
            if (cv < 1 || (!g.dist2 && cv > g.rp[v + 1] - g.rp[v] + 1)) status = GC_ERR_CHECK;
            for (int32_t k = g.rp[v]; k < g.rp[v + 1] && status == GC_OK; ++k) {
                const int32_t u = g.ci[k];
                if (colors_out[u] == cv) status = GC_ERR_CHECK;
                if (g.dist2)
                    for (int32_t j = g.rp[u]; j < g.rp[u + 1] && status == GC_OK; ++j)
                        if (g.ci[j] != v && colors_out[g.ci[j]] == cv) status = GC_ERR_CHECK;
            }
        }
    }
    if (stats_out) {
        int32_t *rs = stats_out->round_sizes;
        const int32_t rcap = stats_out->round_sizes_cap;
        int64_t *rn = stats_out->round_ns;
        const int32_t ncap = stats_out->round_ns_cap;
        gc_stats s;
        memset(&s, 0, sizeof s);
        s.rounds = (int32_t)r.iters;
        s.conflicts = r.conflicts;
        s.colors = -1;
        s.distinct_colors = -1;
        if (!(mode & GC_NO_COLOR_STATS)) {
            int32_t mx = 0;
            for (int32_t v = 0; v < n; ++v) mx = std::max(mx, colors_out[v]);
            std::vector<char> seen((size_t)mx + 1, 0);
            int32_t d = 0;
            for (int32_t v = 0; v < n; ++v)
                if (colors_out[v] >= 1 && !seen[colors_out[v]]) {
                    seen[colors_out[v]] = 1;
                    ++d;
                }
            s.colors = mx;
            s.distinct_colors = d;
        }
        s.elapsed_ms = std::chrono::duration<float, std::milli>(t1 - t0).count();
        if (rs && rcap > 0)
            for (int32_t i = 0; i < rcap && i < (int32_t)r.sizes.size(); ++i) rs[i] = r.sizes[i];
        s.round_sizes = rs;
        s.round_sizes_cap = rcap;
        s.round_ns = rn;
        s.round_ns_cap = ncap;
        if (rn && ncap > 0) memset(rn, 0, (size_t)ncap * sizeof(int64_t));
        *stats_out = s;
    }
    return status;
}
