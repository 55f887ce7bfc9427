// Host side of libgc: contexts, argument checks, launch orchestration and
// the extern "C" entry points declared in include/gc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>

#include "gc.h"
#include "gc_ctx.h"
#include "gc_internal.h"
#include "gc_nvtx.h"

using gc::Buf;
using gc::DevState;
using gc::KParams;
using gc::kRoundSizesDev;

namespace {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return GC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Resolved {
    int32_t max_rounds, t1, t2, tile, tail, blocks_per_sm, window, d2_heavy, core_deg;
};

int resolve_opts(const gc_opts *o, int64_t n, uint32_t mode, Resolved &r)
{
    gc_opts d;
    memset(&d, 0, sizeof d);
    if (!o) o = &d;
    r.max_rounds = o->max_rounds > 0 ? o->max_rounds : (int32_t)std::min<int64_t>(n + 1, INT32_MAX);
    r.t1 = o->t1 > 0 ? o->t1 : 32;
    r.t2 = o->t2 > 0 ? o->t2 : gc::default_t2(mode);
    r.tile = o->tile > 0 ? o->tile : 64;
    r.tail = o->tail > 0 ? o->tail : (o->tail < 0 ? -1 : 2048);
    r.blocks_per_sm = o->blocks_per_sm;
    r.window = o->window;
    if (r.window < -1) return GC_ERR_ARG;
    if (o->d2_heavy < 0) return GC_ERR_ARG;
    r.d2_heavy = o->d2_heavy > 0 ? o->d2_heavy : 4096;
    if (o->core_deg < -1) return GC_ERR_ARG;
    r.core_deg = o->core_deg > 0 ? o->core_deg : (o->core_deg < 0 ? 0 : gc::kCoreDeg);
    if (r.t1 > gc::kT1Max || r.t2 > gc::kT2Max || r.t1 > r.t2) return GC_ERR_ARG;
    if (r.tile % 32 != 0 || r.tile > 4096) return GC_ERR_ARG;
    if (r.blocks_per_sm < 0) return GC_ERR_ARG;
    return GC_OK;
}

int ensure_graph_tables(gc_ctx *c, int64_t G)
{
    const size_t g = (size_t)std::max<int64_t>(G, 1);
    if (!c->gstat.reserve(g * sizeof(gc::GraphStat)) || !c->uofs.reserve((g + 1) * sizeof(int64_t)) ||
        !c->olist.reserve(g * sizeof(int32_t)))
        return GC_ERR_OOM;
    return GC_OK;
}

int ensure_scratch(gc_ctx *c, int64_t n, bool need_b, bool batch, int64_t lut_entries)
{
    const size_t vb = (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t);
    if (need_b && !c->cB.reserve(vb)) return GC_ERR_OOM;
    if (!c->wl0.reserve(vb) || !c->wl1.reserve(vb)) return GC_ERR_OOM;
    if (!c->hb0.reserve(vb) || !c->hb1.reserve(vb) || !c->hub_all.reserve(vb)) return GC_ERR_OOM;
    if (!c->mid_all.reserve(vb)) return GC_ERR_OOM;
    if (!batch && !c->r0mask.reserve((size_t)std::max<int64_t>(n, 1) * sizeof(uint64_t))) return GC_ERR_OOM;
    if (batch && !c->lut.reserve((size_t)std::max<int64_t>(lut_entries, 1) * sizeof(int32_t))) return GC_ERR_OOM;
    if (!c->done.reserve(((size_t)std::max<int64_t>(n, 1) / 32 + 2) * sizeof(int32_t))) return GC_ERR_OOM;
    return GC_OK;
}

int grid_for(gc_ctx *c, bool async, bool batch, bool dist2, const Resolved &r, int64_t n)
{
    int occ = dist2 ? c->occ_d2[async] : c->occ[async][batch];
    int bps = r.blocks_per_sm > 0 ? std::min(r.blocks_per_sm, occ) : occ;
    long long grid = (long long)bps * c->num_sms;
    // Never more blocks than there are vertices to share out.
    long long useful = (n + gc::kBlock - 1) / gc::kBlock;
    if (r.tail > 0 && n <= r.tail) useful = 1;  // small graph: one block from the start
    grid = std::max(1ll, std::min(grid, std::max(useful, 1ll)));
    return (int)grid;
}

// The device state, then (single graphs) the graph's statistics.
constexpr size_t kStateHead = (sizeof(DevState) + 255) / 256 * 256;
constexpr size_t kStateBytes = kStateHead + sizeof(gc::GraphStat);

// Event record on s; while a CUDA graph is being captured the record
// becomes a node of the graph, so timing and completion work on replays.
cudaError_t record(gc_ctx *c, cudaEvent_t ev, cudaStream_t s)
{
    return c->capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

// Enqueue the colouring described by p (single graph or batch) on s.
int enqueue(gc_ctx *c, KParams &p, bool batch, uint32_t mode, const Resolved &r, cudaStream_t s)
{
    const bool async = (mode & GC_SCHED_ASYNC) != 0;
    const int64_t n = p.n;
    const int aux_grid = std::max(1, std::min<int>((int)((n + 255) / 256), c->num_sms * 8));
    cudaError_t e;

    p.st = c->st.as<DevState>();
    p.round_sizes = c->round_sizes.as<int32_t>();
    p.round_sizes_cap = kRoundSizesDev;
    p.mode = mode;
    p.tie = (mode & GC_DEBUG_NO_TIEBREAK) ? gc::TIE_NONE
                                          : ((mode & GC_TIE_HIGHER_KEEPS) ? gc::TIE_HIGHER : gc::TIE_LOWER);
    p.max_rounds = r.max_rounds;
    p.t1 = r.t1;
    p.t2 = r.t2;
    p.tile = r.tile;
    p.tail = r.tail;
    p.window = r.window;
    p.d2_heavy = r.d2_heavy;
    // Round-0 suspect masks: asynchronous RSOC on one graph whose first
    // repair follows a round 0 over all of V with in-place repairs.
    const bool masks = async && !batch && !(mode & (GC_ALG_TWO_PHASE | GC_TIERS | GC_FF_KEEPERS | GC_REPAIR_SNAPSHOT |
                                                     GC_DIST2)) && p.touched == nullptr;
    p.r0mask = masks ? c->r0mask.as<uint64_t>() : nullptr;
    p.core_deg = gc::core_applies(mode, p.touched != nullptr) ? r.core_deg : 0;
    p.done = c->done.as<int32_t>();
    // one graph: its statistics sit right after the state, so that one
    // memset clears both
    p.gstat = p.G <= 1 ? reinterpret_cast<gc::GraphStat *>(c->st.as<char>() + kStateHead)
                       : c->gstat.as<gc::GraphStat>();
    p.uofs = c->uofs.as<int64_t>();
    p.olist = c->olist.as<int32_t>();
    p.pitems = c->pitems.as<int64_t>();
    p.pitems_cap = c->pitems_cap;
    p.cB = c->cB.as<int32_t>();
    p.mark = (mode & GC_FF_KEEPERS) ? p.cB : nullptr;
    p.wl[0] = c->wl0.as<int32_t>();
    p.wl[1] = c->wl1.as<int32_t>();
    p.hub[0] = c->hb0.as<int32_t>();
    p.hub[1] = c->hb1.as<int32_t>();
    p.hub_all = c->hub_all.as<int32_t>();
    p.mid_all = c->mid_all.as<int32_t>();
    p.hub_cap = (int32_t)n;

    if (p.G <= 1) {
        if ((e = cudaMemsetAsync(c->st.p, 0, kStateBytes, s)) != cudaSuccess) return cuda_status(e);
    } else {
        if ((e = cudaMemsetAsync(c->st.p, 0, sizeof(DevState), s)) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemsetAsync(c->gstat.p, 0, (size_t)p.G * sizeof(gc::GraphStat), s)) != cudaSuccess)
            return cuda_status(e);
    }
    const bool stats = !(mode & GC_NO_COLOR_STATS);
    p.stats_bitmap = stats ? c->bitmap.as<uint32_t>() : nullptr;  // computed at the end of the colouring kernel
    if (batch && (e = gc::launch_build_lut(p.vtx_off, p.G, p.n, c->lut.as<int32_t>(), s)) != cudaSuccess)
        return cuda_status(e);
    if ((mode & GC_VALIDATE) && (e = gc::launch_validate(p, batch, aux_grid, s)) != cudaSuccess)
        return cuda_status(e);
    const bool dist2 = (mode & GC_DIST2) != 0;  // single graph only (checked by the callers)
    const int grid = grid_for(c, async, batch, dist2, r, n);
    if ((e = record(c, c->ev0, s)) != cudaSuccess) return cuda_status(e);
    e = dist2 ? gc::launch_color_d2(p, async, grid, s) : gc::launch_color(p, async, batch, grid, s);
    if (e != cudaSuccess) return cuda_status(e);
    if ((e = record(c, c->ev1, s)) != cudaSuccess) return cuda_status(e);
    if (mode & GC_CHECKED) {
        e = dist2 ? gc::launch_check_d2(p, aux_grid, s) : gc::launch_check(p, batch, aux_grid, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if ((e = cudaMemcpyAsync(c->st_host, c->st.p, sizeof(DevState), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return cuda_status(e);
    c->last.rounds_copied = gc::kStamps;  // DevState::round_head
    if ((e = record(c, c->ev_done, s)) != cudaSuccess) return cuda_status(e);
    c->last.stats = stats;
    return GC_OK;
}

int status_from_error_word(int ew)
{
    if (ew & GC_EW_TIMEOUT) return GC_ERR_TIMEOUT;
    if (ew & GC_EW_OVERFLOW) return GC_ERR_OVERFLOW;
    if (ew & GC_EW_GRAPH) return GC_ERR_GRAPH;
    if (ew & GC_EW_CHECK) return GC_ERR_CHECK;
    if (ew & GC_EW_NO_CONVERGENCE) return GC_ERR_NO_CONVERGENCE;
    return GC_OK;
}

thread_local std::unordered_map<int, gc_ctx *> *t_default = nullptr;

gc_ctx *default_ctx()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (!t_default) t_default = new std::unordered_map<int, gc_ctx *>();
    auto it = t_default->find(dev);
    if (it != t_default->end()) return it->second;
    gc_ctx *c = nullptr;
    if (gc_ctx_create(&c, dev) != GC_OK) return nullptr;
    (*t_default)[dev] = c;
    return c;
}

}  // namespace

namespace gc {

int reserve_batch(gc_ctx *c, int32_t G, int64_t total_n, uint32_t mode)
{
    const int64_t lut_entries = (total_n + (1 << kLutShift) - 1) >> kLutShift;
    int rc = ensure_scratch(c, total_n, needs_second_buffer(mode), true, lut_entries);
    if (rc == GC_OK) rc = ensure_graph_tables(c, G);
    return rc;
}

int color_batch_impl(gc_ctx *c, int32_t G, int64_t total_n, int64_t total_nnz, const int64_t *vtx_off,
                     const int64_t *edge_off, const int64_t *rp_off, const int32_t *row_ptr, const int32_t *col_idx,
                     uint32_t mode, const gc_opts *opts, int32_t *colors_out, int32_t *rounds_out,
                     int64_t *conflicts_out, cudaStream_t s)
{
    if (!gc::dist1_mode_ok(mode)) return GC_ERR_ARG;
    if (total_n > 0 && !colors_out) return GC_ERR_ARG;
    Resolved r;
    // The cap applies per graph; every graph's own bound is below total_n + 1.
    int rc = resolve_opts(opts, total_n, mode, r);
    if (rc != GC_OK) return rc;
    c->last.pending = false;
    c->last.n = (int32_t)total_n;
    c->last.mode = mode;
    c->last.empty = (total_n == 0);
    c->last.launch_status = GC_OK;
    if (cudaSetDevice(c->device) != cudaSuccess) return GC_ERR_CUDA;
    if (G > 0 && rounds_out) {
        cudaError_t e = cudaMemsetAsync(rounds_out, 0, (size_t)G * sizeof(int32_t), s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (G > 0 && conflicts_out) {
        cudaError_t e = cudaMemsetAsync(conflicts_out, 0, (size_t)G * sizeof(int64_t), s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    if (total_n == 0) {
        c->last.pending = true;
        return GC_OK;
    }
    const int64_t n = total_n;
    if ((rc = reserve_batch(c, G, n, mode)) != GC_OK) return rc;
    KParams p;
    memset(&p, 0, sizeof p);
    p.row_ptr = row_ptr;
    p.col_idx = col_idx;
    p.vtx_off = vtx_off;
    p.edge_off = edge_off;
    p.rp_off = rp_off;
    p.gid_lut = c->lut.as<int32_t>();
    p.G = G;
    p.n = (int32_t)n;
    p.nnz = total_nnz;
    p.cA = colors_out;
    p.g_rounds = rounds_out;
    p.g_conflicts = reinterpret_cast<unsigned long long *>(conflicts_out);
    rc = enqueue(c, p, true, mode, r, s);
    if (rc == GC_OK) c->last.pending = true;
    c->last.launch_status = rc;
    return rc;
}

int color_batch_offsets(gc_ctx *ctx, int32_t G, int64_t total_n, int64_t col_extent, const int64_t *vtx_off,
                        const int64_t *edge_off, const int64_t *rp_off, const int32_t *base, uint32_t mode,
                        const gc_opts *opts, int32_t *colors_out, int32_t *rounds_out, int64_t *conflicts_out,
                        cudaStream_t stream)
{
    if (!ctx || G < 0 || total_n < 0 || total_n > INT32_MAX || col_extent < 0 ||
        col_extent >= (1ll << kWorkBits) || (G > 0 && (!vtx_off || !edge_off || !rp_off || !base)))
        return GC_ERR_ARG;
    return color_batch_impl(ctx, G, total_n, col_extent, vtx_off, edge_off, rp_off, base, base, mode, opts,
                            colors_out, rounds_out, conflicts_out, stream);
}

}  // namespace gc

extern "C" {

const char *gc_strerror(int s)
{
    switch (s) {
    case GC_OK: return "ok";
    case GC_PENDING: return "pending";
    case GC_ERR_ARG: return "invalid argument";
    case GC_ERR_GRAPH: return "malformed graph (CSR validation failed)";
    case GC_ERR_OOM: return "out of memory";
    case GC_ERR_BUDGET: return "request exceeds the device-memory budget";
    case GC_ERR_NO_CONVERGENCE: return "round cap reached with conflicts left";
    case GC_ERR_TIMEOUT: return "a bounded device wait timed out";
    case GC_ERR_CUDA: return "CUDA runtime error";
    case GC_ERR_OVERFLOW: return "internal worklist overflow";
    case GC_ERR_CHECK: return "result check failed (invalid colouring)";
    case GC_ERR_NOT_FOUND: return "unknown ticket";
    case GC_ERR_TOO_LARGE: return "graph larger than the fixed scratch of gc_color_noalloc";
    default: return "unknown status";
    }
}

int gc_version(void) { return 100; }

int gc_ctx_create(gc_ctx **out, int device)
{
    if (!out) return GC_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return GC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return GC_ERR_CUDA;
    gc_ctx *c = new (std::nothrow) gc_ctx();
    if (!c) return GC_ERR_OOM;
    c->device = device;
    int rc = GC_OK;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    for (int a = 0; a < 2 && e == cudaSuccess; ++a)
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = gc::query_occupancy(a, b, &c->occ[a][b]);
    for (int a = 0; a < 2 && e == cudaSuccess; ++a) e = gc::query_occupancy_d2(a, &c->occ_d2[a]);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->st_host, sizeof(DevState));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->rs_host, kRoundSizesDev * sizeof(int32_t));
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc == GC_OK && (!c->st.reserve(kStateBytes) ||
                        !c->bitmap.reserve(gc::kStatBitmapWords * sizeof(uint32_t)) ||
                        !c->round_sizes.reserve(kRoundSizesDev * sizeof(int32_t))))
        rc = GC_ERR_OOM;
    // the colour-statistics kernel leaves the bitmap zero after every use
    if (rc == GC_OK && cudaMemset(c->bitmap.p, 0, gc::kStatBitmapWords * sizeof(uint32_t)) != cudaSuccess)
        rc = GC_ERR_CUDA;
    for (int a = 0; a < 2; ++a) {
        for (int b = 0; b < 2; ++b)
            if (rc == GC_OK && c->occ[a][b] < 1) rc = GC_ERR_CUDA;
        if (rc == GC_OK && c->occ_d2[a] < 1) rc = GC_ERR_CUDA;
    }
    if (rc == GC_OK) {
        // one warp-group item per warp of the largest grid
        const int occ = std::max(std::max(c->occ[0][0], c->occ[0][1]), std::max(c->occ[1][0], c->occ[1][1]));
        c->pitems_cap = c->num_sms * occ * gc::kWarps;
        if (!c->pitems.reserve((size_t)c->pitems_cap * sizeof(int64_t))) rc = GC_ERR_OOM;
    }
    cudaSetDevice(prev);
    if (rc != GC_OK) {
        gc_ctx_destroy(c);
        return rc;
    }
    *out = c;
    return GC_OK;
}

void gc_ctx_destroy(gc_ctx *c)
{
    if (!c) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    if (c->ev_done) cudaEventSynchronize(c->ev_done);
    for (Buf *b : {&c->r0mask, &c->cB, &c->wl0, &c->wl1, &c->hb0, &c->hb1, &c->hub_all, &c->mid_all, &c->lut, &c->bitmap,
                   &c->round_sizes, &c->st, &c->done, &c->gstat, &c->uofs, &c->olist, &c->pitems, &c->cls, &c->stage_rp,
                   &c->stage_ci,
                   &c->stage_col})
        b->release();
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->rs_host) cudaFreeHost(c->rs_host);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev_done) cudaEventDestroy(c->ev_done);
    cudaGetLastError();
    cudaSetDevice(prev);
    delete c;
}

int gc_color_async(gc_ctx *c, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, const gc_opts *opts,
                   int32_t *colors_out, void *stream)
{
    gc::NvtxRange nvtx_range("gc_color_async");
    if (!c || !csr || n < 0 || nnz < 0 || nnz > INT32_MAX) return GC_ERR_ARG;
    if (!gc::mode_ok(mode)) return GC_ERR_ARG;
    if (n > 0 && (!csr->row_ptr || !colors_out)) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    Resolved r;
    int rc = resolve_opts(opts, n, mode, r);
    if (rc != GC_OK) return rc;
    c->last.pending = false;
    c->last.n = n;
    c->last.mode = mode;
    c->last.empty = (n == 0);
    c->last.launch_status = GC_OK;
    if (n == 0) {
        c->last.pending = true;
        return GC_OK;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return GC_ERR_CUDA;
    const bool need_b = gc::needs_second_buffer(mode);
    if ((rc = ensure_scratch(c, n, need_b, false, 0)) != GC_OK) return rc;
    if ((rc = ensure_graph_tables(c, 1)) != GC_OK) return rc;
    KParams p;
    memset(&p, 0, sizeof p);
    p.row_ptr = csr->row_ptr;
    p.col_idx = csr->col_idx;
    p.G = 1;
    p.n = n;
    p.nnz = nnz;
    p.cA = colors_out;
    rc = enqueue(c, p, false, mode, r, (cudaStream_t)stream);
    if (rc == GC_OK) c->last.pending = true;
    c->last.launch_status = rc;
    return rc;
}

int gc_recolor_async(gc_ctx *c, const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, const gc_opts *opts,
                     int32_t *colors_inout, const int32_t *touched, int32_t n_touched, void *stream)
{
    gc::NvtxRange nvtx_range("gc_recolor_async");
    if (!c || !csr || n < 0 || nnz < 0 || nnz > INT32_MAX || n_touched < 0) return GC_ERR_ARG;
    if (!gc::dist1_mode_ok(mode) || (mode & (GC_ALG_TWO_PHASE | GC_TIERS | GC_REPAIR_SNAPSHOT))) return GC_ERR_ARG;
    if (n > 0 && (!csr->row_ptr || !colors_inout)) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    if (n_touched > 0 && !touched) return GC_ERR_ARG;
    Resolved r;
    int rc = resolve_opts(opts, n, mode, r);
    if (rc != GC_OK) return rc;
    c->last.pending = false;
    c->last.n = n;
    c->last.mode = mode;
    c->last.empty = (n == 0);
    c->last.launch_status = GC_OK;
    if (n == 0) {
        c->last.pending = true;
        return GC_OK;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return GC_ERR_CUDA;
    if ((rc = ensure_scratch(c, n, gc::needs_second_buffer(mode), false, 0)) != GC_OK) return rc;
    if ((rc = ensure_graph_tables(c, 1)) != GC_OK) return rc;
    KParams p;
    memset(&p, 0, sizeof p);
    p.row_ptr = csr->row_ptr;
    p.col_idx = csr->col_idx;
    p.G = 1;
    p.n = n;
    p.nnz = nnz;
    p.cA = colors_inout;
    static const int32_t kNoTouched = 0;
    p.touched = n_touched > 0 ? touched : &kNoTouched;  // non-null marks the incremental run
    p.n_touched = n_touched;
    rc = enqueue(c, p, false, mode, r, (cudaStream_t)stream);
    if (rc == GC_OK) c->last.pending = true;
    c->last.launch_status = rc;
    return rc;
}

int gc_ctx_stats(gc_ctx *c, gc_stats *out)
{
    gc::NvtxRange nvtx_range("gc_ctx_stats");
    if (!c) return GC_ERR_ARG;
    if (!c->last.pending) return c->last.launch_status != GC_OK ? c->last.launch_status : GC_ERR_ARG;
    gc_stats s;
    memset(&s, 0, sizeof s);
    s.colors = -1;
    s.distinct_colors = -1;
    int status = GC_OK;
    if (c->last.empty) {
        s.colors = 0;
        s.distinct_colors = 0;
    } else {
        cudaError_t e = cudaEventSynchronize(c->ev_done);
        if (e != cudaSuccess) return cuda_status(e);
        const DevState &d = *c->st_host;
        s.rounds = d.rounds;
        s.conflicts = (int64_t)d.conflicts;
        s.model_bytes = (int64_t)d.model_bytes;
        s.error_word = d.error;
        if (c->last.stats) {
            s.colors = d.max_color;
            s.distinct_colors = d.distinct;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) s.elapsed_ms = ms;
        cudaGetLastError();
        status = status_from_error_word(d.error);
    }
    if (out) {
        int32_t *rs = out->round_sizes;
        int32_t cap = out->round_sizes_cap;
        if (rs && cap > 0) {
            int32_t k = std::min<int32_t>(std::min<int32_t>(s.rounds, cap), kRoundSizesDev);
            if (k > c->last.rounds_copied) {
                // more than the head copied back with the state: fetch synchronously
                if (cudaMemcpy(c->rs_host, c->round_sizes.p, (size_t)k * sizeof(int32_t),
                               cudaMemcpyDeviceToHost) != cudaSuccess) {
                    cudaGetLastError();
                    k = 0;
                }
                memcpy(rs, c->rs_host, (size_t)std::max(k, 0) * sizeof(int32_t));
            } else {
                memcpy(rs, c->st_host->round_head, (size_t)std::max(k, 0) * sizeof(int32_t));
            }
        }
        s.round_sizes = rs;
        s.round_sizes_cap = cap;
        s.round_ns = out->round_ns;
        s.round_ns_cap = out->round_ns_cap;
        if (s.round_ns && s.round_ns_cap > 0) {
            const DevState &d = *c->st_host;
            const int k = std::min<int>(std::min<int>(s.rounds + 1, s.round_ns_cap), gc::kStamps);
            for (int i = 0; i < k; ++i)
                s.round_ns[i] = (c->last.empty || d.stamp[i] == 0) ? 0 : (int64_t)(d.stamp[i] - d.t_start);
        }
        *out = s;
    }
    return status;
}

int gc_color(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, int32_t *colors_out, gc_stats *stats_out)
{
    gc::NvtxRange nvtx_range("gc_color");
    if (!csr || n < 0 || nnz < 0 || nnz > INT32_MAX) return GC_ERR_ARG;
    if (n > 0 && (!csr->row_ptr || !colors_out)) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    gc_ctx *c = default_ctx();
    if (!c) return GC_ERR_CUDA;
    if (n == 0) {
        int rc = gc_color_async(c, csr, 0, 0, mode, nullptr, colors_out, nullptr);
        return rc != GC_OK ? rc : gc_ctx_stats(c, stats_out);
    }
    const bool rp_dev = is_device_ptr(csr->row_ptr);
    const bool ci_dev = nnz == 0 || is_device_ptr(csr->col_idx);
    const bool out_dev = is_device_ptr(colors_out);
    gc_csr d = *csr;
    cudaStream_t s = nullptr;
    cudaError_t e;
    // Uploads, colouring and the download of the colours are enqueued on
    // one stream and waited for once (from pinned host memory the copies
    // run without blocking the host).
    if (!rp_dev) {
        if (!c->stage_rp.reserve(((size_t)n + 1) * sizeof(int32_t))) return GC_ERR_OOM;
        if ((e = cudaMemcpyAsync(c->stage_rp.p, csr->row_ptr, ((size_t)n + 1) * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_status(e);
        d.row_ptr = c->stage_rp.as<int32_t>();
    }
    if (!ci_dev) {
        if (!c->stage_ci.reserve((size_t)nnz * sizeof(int32_t))) return GC_ERR_OOM;
        if ((e = cudaMemcpyAsync(c->stage_ci.p, csr->col_idx, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice,
                                 s)) != cudaSuccess)
            return cuda_status(e);
        d.col_idx = c->stage_ci.as<int32_t>();
    }
    int32_t *out = colors_out;
    if (!out_dev) {
        if (!c->stage_col.reserve((size_t)n * sizeof(int32_t))) return GC_ERR_OOM;
        out = c->stage_col.as<int32_t>();
    }
    int rc = gc_color_async(c, &d, n, nnz, mode, nullptr, out, s);
    if (rc != GC_OK) {
        cudaStreamSynchronize(s);  // the uploads read the caller's arrays
        return rc;
    }
    if (!out_dev && (e = cudaMemcpyAsync(colors_out, out, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s)) !=
                        cudaSuccess) {
        cudaStreamSynchronize(s);
        return cuda_status(e);
    }
    rc = gc_ctx_stats(c, stats_out);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess && rc == GC_OK) rc = cuda_status(e);
    return rc;
}

int gc_color_batch(gc_ctx *c, const gc_batch *b, uint32_t mode, const gc_opts *opts, int32_t *colors_out,
                   int32_t *rounds_out, int64_t *conflicts_out, void *stream)
{
    gc::NvtxRange nvtx_range("gc_color_batch");
    if (!c || !b || b->G < 0 || b->total_n < 0 || b->total_n > INT32_MAX || b->total_nnz < 0 ||
        b->total_nnz >= (1ll << gc::kWorkBits))
        return GC_ERR_ARG;
    if (b->G > 0 && (!b->vtx_off || !b->edge_off)) return GC_ERR_ARG;
    if (b->total_n > 0 && !b->row_ptr) return GC_ERR_ARG;
    if (b->total_nnz > 0 && !b->col_idx) return GC_ERR_ARG;
    return gc::color_batch_impl(c, b->G, b->total_n, b->total_nnz, b->vtx_off, b->edge_off, nullptr, b->row_ptr,
                                b->col_idx, mode, opts, colors_out, rounds_out, conflicts_out, (cudaStream_t)stream);
}

}  // extern "C"
