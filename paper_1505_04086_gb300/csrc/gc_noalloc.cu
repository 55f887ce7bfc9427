// gc_color_noalloc: single-graph colouring that never allocates memory.
//
// Who needs this: callers that may not allocate device memory while they
// run -- for example a host loop whose device memory is owned by another
// allocator with a hard budget, or a latency-critical loop in which a
// cudaMalloc/cudaFree (which can synchronise the whole device) is not
// acceptable.  Such callers pass their own input and output arrays; every
// other buffer the colouring needs (second colour buffer, worklists, flags,
// counters) comes from one fixed array that is part of the library image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds kNoAllocBytes of it until the process exits.  Host code may
// not use its name as an address (on the host it is only a stand-in), so the
// first call on each device looks the real address up with
// cudaGetSymbolAddress while that device is current, and caches it.
//
// All calls share the array, and it keeps whatever the previous call left
// in it; the parts that must start at zero are cleared on the stream at the
// start of every call.  Two calls whose GPU work overlaps (different streams
// or host threads without ordering between them) race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "gc.h"
#include "gc_ctx.h"
#include "gc_internal.h"
#include "gc_nvtx.h"

namespace {

constexpr int64_t kMaxN = GC_NOALLOC_MAX_N;
constexpr int kRoundSizes = 4096;

// Byte offsets of the pieces inside the fixed array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kVec = align256((size_t)kMaxN * sizeof(int32_t));
constexpr size_t kOffState = 0;
constexpr size_t kOffBitmap = align256(sizeof(gc::DevState));
constexpr size_t kOffRounds = kOffBitmap + align256(gc::kStatBitmapWords * sizeof(uint32_t));
constexpr size_t kOffDone = kOffRounds + align256(kRoundSizes * sizeof(int32_t));
constexpr size_t kOffGstat = kOffDone + align256(((size_t)kMaxN / 32 + 2) * sizeof(int32_t));
constexpr size_t kOffUofs = kOffGstat + align256(sizeof(gc::GraphStat));
constexpr size_t kOffOlist = kOffUofs + align256(2 * sizeof(int64_t));
constexpr size_t kOffB = kOffOlist + align256(sizeof(int32_t));
constexpr size_t kOffWl0 = kOffB + kVec;
constexpr size_t kOffWl1 = kOffWl0 + kVec;
constexpr size_t kOffHb0 = kOffWl1 + kVec;
constexpr size_t kOffHb1 = kOffHb0 + kVec;
constexpr size_t kOffHubAll = kOffHb1 + kVec;
constexpr size_t kOffMidAll = kOffHubAll + kVec;
constexpr int32_t kPitems = 8192;  // round-0 warp groups: items for grids of up to 8192 warps
constexpr size_t kOffPitems = kOffMidAll + kVec;
constexpr size_t kNoAllocBytes = kOffPitems + align256(kPitems * sizeof(int64_t));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
    int occ[2] = {0, 0};               // blocks per SM: [det, async]
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: find the device address of the
// fixed array and the launch geometry.  Returns GC_OK or GC_ERR_CUDA.
int setup_device(int dev, DeviceSetup **out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return GC_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            gc::query_occupancy(false, false, &d.occ[0]) != cudaSuccess ||
            gc::query_occupancy(true, false, &d.occ[1]) != cudaSuccess || d.occ[0] < 1 || d.occ[1] < 1) {
            cudaGetLastError();
            return GC_ERR_CUDA;
        }
        d.scratch = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    *out = &d;
    return GC_OK;
}

bool device_accessible(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int gc_color_noalloc(const gc_csr *csr, int32_t n, int64_t nnz, uint32_t mode, const gc_opts *opts,
                                int32_t *colors_out, gc_stats *stats_out, void *stream)
{
    gc::NvtxRange nvtx_range("gc_color_noalloc");
    if (!csr || n < 0 || nnz < 0 || nnz > INT32_MAX) return GC_ERR_ARG;
    if (!gc::dist1_mode_ok(mode)) return GC_ERR_ARG;
    if (n > kMaxN) return GC_ERR_TOO_LARGE;
    if (n > 0 && (!csr->row_ptr || !colors_out)) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    gc_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    const int32_t max_rounds = o.max_rounds > 0 ? o.max_rounds : n + 1;
    const int32_t t1 = o.t1 > 0 ? o.t1 : 32, t2 = o.t2 > 0 ? o.t2 : gc::default_t2(mode), tile = o.tile > 0 ? o.tile : 64;
    const int32_t tail = o.tail > 0 ? o.tail : (o.tail < 0 ? -1 : 2048);
    if (t1 > gc::kT1Max || t2 > gc::kT2Max || t1 > t2 || tile % 32 != 0 || tile > 4096 ||
        o.blocks_per_sm < 0 || o.window < -1 || o.core_deg < -1)
        return GC_ERR_ARG;
    gc_stats s;
    memset(&s, 0, sizeof s);
    if (n == 0) {
        if (stats_out) {
            s.round_sizes = stats_out->round_sizes;
            s.round_sizes_cap = stats_out->round_sizes_cap;
            s.round_ns = stats_out->round_ns;
            s.round_ns_cap = stats_out->round_ns_cap;
            *stats_out = s;
        }
        return GC_OK;
    }
    if (!device_accessible(csr->row_ptr) || !device_accessible(colors_out) ||
        (nnz > 0 && !device_accessible(csr->col_idx)))
        return GC_ERR_ARG;  // no staging here: that would need memory

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    DeviceSetup *d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc != GC_OK) return rc;

    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = d->scratch;
    gc::KParams p;
    memset(&p, 0, sizeof p);
    p.row_ptr = csr->row_ptr;
    p.col_idx = csr->col_idx;
    p.G = 1;
    p.n = n;
    p.nnz = nnz;
    p.cA = colors_out;
    p.cB = reinterpret_cast<int32_t *>(base + kOffB);
    p.mark = (mode & GC_FF_KEEPERS) ? p.cB : nullptr;
    p.wl[0] = reinterpret_cast<int32_t *>(base + kOffWl0);
    p.wl[1] = reinterpret_cast<int32_t *>(base + kOffWl1);
    p.hub[0] = reinterpret_cast<int32_t *>(base + kOffHb0);
    p.hub[1] = reinterpret_cast<int32_t *>(base + kOffHb1);
    p.hub_all = reinterpret_cast<int32_t *>(base + kOffHubAll);
    p.mid_all = reinterpret_cast<int32_t *>(base + kOffMidAll);
    p.hub_cap = n;
    p.done = reinterpret_cast<int32_t *>(base + kOffDone);
    p.gstat = reinterpret_cast<gc::GraphStat *>(base + kOffGstat);
    p.uofs = reinterpret_cast<int64_t *>(base + kOffUofs);
    p.olist = reinterpret_cast<int32_t *>(base + kOffOlist);
    p.pitems = reinterpret_cast<int64_t *>(base + kOffPitems);
    p.pitems_cap = kPitems;
    p.st = reinterpret_cast<gc::DevState *>(base + kOffState);
    p.round_sizes = reinterpret_cast<int32_t *>(base + kOffRounds);
    p.round_sizes_cap = kRoundSizes;
    p.mode = mode;
    p.tie = (mode & GC_DEBUG_NO_TIEBREAK) ? gc::TIE_NONE
                                          : ((mode & GC_TIE_HIGHER_KEEPS) ? gc::TIE_HIGHER : gc::TIE_LOWER);
    p.max_rounds = max_rounds;
    p.t1 = t1;
    p.t2 = t2;
    p.tile = tile;
    p.tail = tail;
    p.window = o.window;
    p.core_deg = gc::core_applies(mode, false) ? (o.core_deg > 0 ? o.core_deg : (o.core_deg < 0 ? 0 : gc::kCoreDeg))
                                                      : 0;

    const bool async = (mode & GC_SCHED_ASYNC) != 0;
    const int occ = d->occ[async ? 1 : 0];
    const int bps = o.blocks_per_sm > 0 && o.blocks_per_sm < occ ? o.blocks_per_sm : occ;
    long long grid = (long long)bps * d->num_sms;
    long long useful = ((long long)n + gc::kBlock - 1) / gc::kBlock;
    if (tail > 0 && n <= tail) useful = 1;
    if (grid > useful) grid = useful;
    if (grid < 1) grid = 1;
    const int aux_grid = (int)(useful < (long long)d->num_sms * 8 ? (useful > 0 ? useful : 1) : d->num_sms * 8);
    const bool stats = !(mode & GC_NO_COLOR_STATS);
    p.stats_bitmap = stats ? reinterpret_cast<uint32_t *>(base + kOffBitmap) : nullptr;

    // Clear what must start at zero: the launch state (the colour bitmap is
    // zero from load time and left zero by every statistics pass).
    cudaError_t e = cudaMemsetAsync(p.st, 0, sizeof(gc::DevState), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.gstat, 0, sizeof(gc::GraphStat), st);
    if (e == cudaSuccess && (mode & GC_VALIDATE)) e = gc::launch_validate(p, false, aux_grid, st);
    if (e == cudaSuccess) e = gc::launch_color(p, async, false, (int)grid, st);
    if (e == cudaSuccess && (mode & GC_CHECKED)) e = gc::launch_check(p, false, aux_grid, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    gc::DevState h;
    if (e == cudaSuccess) e = cudaMemcpy(&h, p.st, sizeof h, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
    }
    s.rounds = h.rounds;
    s.conflicts = (int64_t)h.conflicts;
    s.model_bytes = (int64_t)h.model_bytes;
    s.error_word = h.error;
    s.colors = stats ? h.max_color : -1;
    s.distinct_colors = stats ? h.distinct : -1;
    s.elapsed_ms = 0.f;  // no events: this entry point records no timing
    if (stats_out) {
        s.round_sizes = stats_out->round_sizes;
        s.round_sizes_cap = stats_out->round_sizes_cap;
        if (s.round_sizes && s.round_sizes_cap > 0) {
            int k = s.rounds < s.round_sizes_cap ? s.rounds : s.round_sizes_cap;
            if (k > kRoundSizes) k = kRoundSizes;
            if (k > 0 && cudaMemcpy(s.round_sizes, p.round_sizes, (size_t)k * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost) != cudaSuccess) {
                cudaGetLastError();
                return GC_ERR_CUDA;
            }
        }
        s.round_ns = stats_out->round_ns;
        s.round_ns_cap = stats_out->round_ns_cap;
        if (s.round_ns && s.round_ns_cap > 0) {
            int k = s.rounds + 1 < s.round_ns_cap ? s.rounds + 1 : s.round_ns_cap;
            if (k > gc::kStamps) k = gc::kStamps;
            for (int i = 0; i < k; ++i) s.round_ns[i] = h.stamp[i] ? (int64_t)(h.stamp[i] - h.t_start) : 0;
        }
        *stats_out = s;
    }
    if (h.error & GC_EW_TIMEOUT) return GC_ERR_TIMEOUT;
    if (h.error & GC_EW_OVERFLOW) return GC_ERR_OVERFLOW;
    if (h.error & GC_EW_GRAPH) return GC_ERR_GRAPH;
    if (h.error & GC_EW_CHECK) return GC_ERR_CHECK;
    if (h.error & GC_EW_NO_CONVERGENCE) return GC_ERR_NO_CONVERGENCE;
    return GC_OK;
}
