// Batch plans (one gc_color_batch call captured into a CUDA graph and
// replayed) and the option autotuner: the extern "C" entry points gc_plan_*,
// gc_autotune_batch and gc_autotune of include/gc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "gc.h"
#include "gc_ctx.h"
#include "gc_internal.h"
#include "gc_nvtx.h"

struct gc_plan {
    gc_ctx *ctx = nullptr;               // private: its scratch never moves under the graph
    cudaStream_t cap = nullptr;          // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    gc::LastCall launched;               // host fields of the captured call
};

namespace {

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return GC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
}

bool batch_ok(const gc_batch *b)
{
    if (!b || b->G < 0 || b->total_n < 0 || b->total_n > INT32_MAX || b->total_nnz < 0 ||
        b->total_nnz >= (1ll << gc::kWorkBits))
        return false;
    if (b->G > 0 && (!b->vtx_off || !b->edge_off)) return false;
    if (b->total_n > 0 && !b->row_ptr) return false;
    if (b->total_nnz > 0 && !b->col_idx) return false;
    return true;
}

int run_batch(gc_ctx *c, const gc_batch *b, uint32_t mode, const gc_opts *o, int32_t *colors_out, cudaStream_t s)
{
    return gc::color_batch_impl(c, b->G, b->total_n, b->total_nnz, b->vtx_off, b->edge_off, nullptr, b->row_ptr,
                                b->col_idx, mode, o, colors_out, nullptr, nullptr, s);
}

// On-disk cache of tuning results, used when the environment variable
// GC_TUNE_CACHE names a file: one text line per tuned problem,
//   <key> t1 t2 tile blocks_per_sm tail window best_ms default_ms
// where the key names the library version, the call (one graph or a batch),
// the mode, the graph's shape (vertices, entries, graphs), the SM count and
// the repetitions.  Lines are appended; the last line of a key wins.
std::mutex g_cache_mu;

std::string cache_key(const char *kind, uint32_t mode, int64_t n, int64_t nnz, int64_t G, int sms, int reps)
{
    char buf[192];
    snprintf(buf, sizeof buf, "gc%d:%s:mode=%u:n=%lld:nnz=%lld:G=%lld:sms=%d:reps=%d", gc_version(), kind, mode,
             (long long)n, (long long)nnz, (long long)G, sms, reps);
    return buf;
}

bool cache_lookup(const std::string &key, gc_tune_result *out)
{
    const char *path = getenv("GC_TUNE_CACHE");
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool hit = false;
    while (fgets(line, sizeof line, f)) {
        char k[256];
        gc_opts o;
        memset(&o, 0, sizeof o);
        float best = 0.f, def = 0.f;
        if (sscanf(line, "%255s %d %d %d %d %d %d %f %f", k, &o.t1, &o.t2, &o.tile, &o.blocks_per_sm, &o.tail,
                   &o.window, &best, &def) != 9 || key != k)
            continue;
        out->best = o;
        out->best_ms = best;
        out->default_ms = def;
        hit = true;
    }
    fclose(f);
    return hit;
}

void cache_store(const std::string &key, const gc_tune_result &r)
{
    const char *path = getenv("GC_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lk(g_cache_mu);
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %.6f %.6f\n", key.c_str(), r.best.t1, r.best.t2, r.best.tile,
            r.best.blocks_per_sm, r.best.tail, r.best.window, r.best_ms, r.default_ms);
    fclose(f);
}

// A cached result: one colouring with its options (colors_out receives it);
// evaluated = 0 tells the caller nothing was searched.
template <class Run>
int from_cache(gc_ctx *ctx, const std::string &key, gc_tune_result *out, Run run)
{
    memset(out, 0, sizeof *out);
    if (!cache_lookup(key, out)) return GC_ERR_NOT_FOUND;
    int rc = run(out->best);
    gc_stats st;
    memset(&st, 0, sizeof st);
    if (rc == GC_OK) rc = gc_ctx_stats(ctx, &st);
    return rc;
}

// Coordinate descent over the option knobs (see gc_autotune_batch in gc.h):
// run(o) enqueues one colouring with options o on the legacy stream.
template <class Run>
int tune(gc_ctx *ctx, int reps, uint32_t mode, gc_tune_result *out, Run run)
{
    memset(out, 0, sizeof *out);
    // Device time of one option set (median over reps runs) and the most
    // colours any of the runs used.
    auto measure = [&](const gc_opts &o, float &ms, int &colors) -> int {
        std::vector<float> t;
        colors = 0;
        for (int r = 0; r < reps; ++r) {
            int rc = run(o);
            gc_stats st;
            memset(&st, 0, sizeof st);
            if (rc == GC_OK) rc = gc_ctx_stats(ctx, &st);
            if (rc != GC_OK) return rc;
            t.push_back(st.elapsed_ms);
            colors = std::max(colors, st.colors);
        }
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        ++out->evaluated;
        return GC_OK;
    };
    // In the asynchronous modes the options change the colouring too: a
    // candidate is taken only if it uses no more colours than the defaults
    // did (colour statistics off: time alone).
    const bool guard = (mode & GC_SCHED_ASYNC) && !(mode & GC_NO_COLOR_STATS);
    // The knobs (only those that leave the method's result alone: window,
    // which decides which graphs are coloured in id order, changes colour
    // counts and is not tuned), each with its candidate settings.  Tile and
    // blocks per SM are searched jointly: the work a warp claims at once and
    // the number of warps resident trade against each other, so one often
    // pays off only together with the other.
    using Setting = std::vector<std::pair<int32_t gc_opts::*, int32_t>>;
    std::vector<std::vector<Setting>> knobs;
    knobs.push_back({});
    for (int32_t v : {8, 16, 24, 32, 48, 62}) knobs.back().push_back({{&gc_opts::t1, v}});
    knobs.push_back({});
    for (int32_t v : {128, 256, 512, 1024, 2048, 4096}) knobs.back().push_back({{&gc_opts::t2, v}});
    knobs.push_back({});
    for (int32_t t : {32, 64, 128, 256, 512})
        for (int32_t b : {1, 2, 0}) knobs.back().push_back({{&gc_opts::tile, t}, {&gc_opts::blocks_per_sm, b}});
    knobs.push_back({});
    for (int32_t v : {-1, 256, 2048, 8192}) knobs.back().push_back({{&gc_opts::tail, v}});
    gc_opts best;  // the library defaults, spelled out
    memset(&best, 0, sizeof best);
    best.t1 = 32;
    best.t2 = gc::default_t2(mode);
    best.tile = 64;
    best.tail = 2048;
    float best_ms = 0.f;
    int default_colors = 0;
    int rc = measure(best, best_ms, default_colors);
    if (rc != GC_OK) return rc;
    out->default_ms = best_ms;
    // Coordinate descent from the defaults: up to three sweeps over the
    // knobs, each knob set to its fastest setting with the others held.
    for (int sweep = 0; sweep < 3; ++sweep) {
        bool moved = false;
        for (const auto &knob : knobs) {
            const gc_opts start = best;
            for (const Setting &st : knob) {
                gc_opts o = start;
                bool same = true;
                for (const auto &fv : st) {
                    same = same && (o.*(fv.first) == fv.second);
                    o.*(fv.first) = fv.second;
                }
                if (same) continue;
                if (o.t1 > o.t2) continue;  // thread bin above the warp bin
                float ms = 0.f;
                int colors = 0;
                if ((rc = measure(o, ms, colors)) != GC_OK) return rc;
                if (ms < best_ms && (!guard || colors <= default_colors)) {
                    best_ms = ms;
                    best = o;
                    moved = true;
                }
            }
        }
        if (!moved) break;
    }
    out->best = best;
    out->best_ms = best_ms;
    return GC_OK;
}

}  // namespace

extern "C" {

int gc_plan_create(const gc_batch *b, int device, uint32_t mode, const gc_opts *opts, int32_t *colors_out,
                   int32_t *rounds_out, int64_t *conflicts_out, gc_plan **out)
{
    gc::NvtxRange nvtx_range("gc_plan_create");
    if (!out) return GC_ERR_ARG;
    *out = nullptr;
    if (!batch_ok(b) || !gc::dist1_mode_ok(mode) || (b->total_n > 0 && !colors_out)) return GC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    gc_plan *pl = new (std::nothrow) gc_plan();
    if (!pl) return GC_ERR_OOM;
    int rc = gc_ctx_create(&pl->ctx, device);
    if (rc == GC_OK && cudaSetDevice(device) != cudaSuccess) rc = GC_ERR_CUDA;
    if (rc == GC_OK) rc = gc::reserve_batch(pl->ctx, b->G, b->total_n, mode);
    if (rc == GC_OK) rc = cuda_rc(cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking));
    if (rc == GC_OK) rc = cuda_rc(cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
    if (rc == GC_OK) {
        pl->ctx->capturing = true;
        rc = gc::color_batch_impl(pl->ctx, b->G, b->total_n, b->total_nnz, b->vtx_off, b->edge_off, nullptr,
                                  b->row_ptr, b->col_idx, mode, opts, colors_out, rounds_out, conflicts_out,
                                  pl->cap);
        pl->ctx->capturing = false;
        // End the capture whatever happened, so that the stream is usable.
        const cudaError_t e = cudaStreamEndCapture(pl->cap, &pl->graph);
        if (rc == GC_OK) rc = cuda_rc(e);
        else cudaGetLastError();
    }
    if (rc == GC_OK) rc = cuda_rc(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    if (rc == GC_OK) {
        pl->launched = pl->ctx->last;
        pl->ctx->last.pending = false;  // nothing ran yet
        *out = pl;
    } else {
        gc_plan_destroy(pl);
    }
    cudaSetDevice(prev);
    return rc;
}

int gc_plan_launch(gc_plan *pl, void *stream)
{
    gc::NvtxRange nvtx_range("gc_plan_launch");
    if (!pl || !pl->exec) return GC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(pl->ctx->device) != cudaSuccess) return GC_ERR_CUDA;
    int rc = GC_OK;
    if (pl->launched.empty) {
        pl->ctx->last = pl->launched;  // empty batch: nothing was captured to run
    } else {
        rc = cuda_rc(cudaGraphLaunch(pl->exec, (cudaStream_t)stream));
        if (rc == GC_OK) pl->ctx->last = pl->launched;
        else {
            pl->ctx->last.pending = false;
            pl->ctx->last.launch_status = rc;
        }
    }
    cudaSetDevice(prev);
    return rc;
}

int gc_plan_stats(gc_plan *pl, gc_stats *stats)
{
    if (!pl) return GC_ERR_ARG;
    return gc_ctx_stats(pl->ctx, stats);
}

void gc_plan_destroy(gc_plan *pl)
{
    if (!pl) return;
    if (pl->ctx) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(pl->ctx->device);
        if (pl->cap) cudaStreamSynchronize(pl->cap);
        if (pl->exec) cudaGraphExecDestroy(pl->exec);
        if (pl->graph) cudaGraphDestroy(pl->graph);
        if (pl->cap) cudaStreamDestroy(pl->cap);
        cudaGetLastError();
        gc_ctx_destroy(pl->ctx);  // waits for the last replay
        cudaSetDevice(prev);
    }
    delete pl;
}

int gc_autotune_batch(gc_ctx *ctx, const gc_batch *b, uint32_t mode, int32_t reps, int32_t *colors_out,
                      gc_tune_result *out)
{
    gc::NvtxRange nvtx_range("gc_autotune_batch");
    if (!ctx || !out || !batch_ok(b) || !gc::dist1_mode_ok(mode) || (b->total_n > 0 && !colors_out) || reps < 1 ||
        reps > 64)
        return GC_ERR_ARG;
    auto run = [&](const gc_opts &o) { return run_batch(ctx, b, mode, &o, colors_out, nullptr); };
    const std::string key = cache_key("batch", mode, b->total_n, b->total_nnz, b->G, ctx->num_sms, reps);
    int rc = from_cache(ctx, key, out, run);
    if (rc != GC_ERR_NOT_FOUND) return rc;
    rc = tune(ctx, reps, mode, out, run);
    if (rc == GC_OK) cache_store(key, *out);
    return rc;
}

int gc_autotune(gc_ctx *ctx, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, int32_t reps,
                int32_t *colors_out, gc_tune_result *out)
{
    gc::NvtxRange nvtx_range("gc_autotune");
    if (!ctx || !out || !csr || n < 0 || nnz < 0 || nnz > INT32_MAX || !gc::dist1_mode_ok(mode) ||
        (n > 0 && (!csr->row_ptr || !colors_out)) || (nnz > 0 && !csr->col_idx) || reps < 1 || reps > 64)
        return GC_ERR_ARG;
    auto run = [&](const gc_opts &o) { return gc_color_async(ctx, csr, n, nnz, mode, &o, colors_out, nullptr); };
    const std::string key = cache_key("graph", mode, n, nnz, 1, ctx->num_sms, reps);
    int rc = from_cache(ctx, key, out, run);
    if (rc != GC_ERR_NOT_FOUND) return rc;
    rc = tune(ctx, reps, mode, out, run);
    if (rc == GC_OK) cache_store(key, *out);
    return rc;
}

}  // extern "C"
