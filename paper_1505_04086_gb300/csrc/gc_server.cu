// Serving runtime: a request queue with continuous batching.
//
// Requests (host CSR graphs) are copied into a pinned host pool at submit
// time.  A worker thread admits them in arrival order into a fixed device
// arena (the memory budget), uploading on a copy stream, and colours every
// uploaded request in one batched persistent launch (a "wave") on one of
// kLanes compute lanes (stream + context + wave buffers).  A wave starts as
// soon as a lane is free and a request is uploaded: requests that arrive
// while a wave runs go into the next wave, which runs on the other lane
// beside it, each wave's grid sized to its share of the SMs.  Results are
// copied back to the pinned pool and handed out by gc_server_poll /
// gc_server_wait; gc_server_cancel drops a request.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gc.h"
#include "gc_ctx.h"
#include "gc_internal.h"
#include "gc_nvtx.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) in 256-byte units (offsets only).
class Arena {
  public:
    void reset(int64_t size)
    {
        free_.clear();
        size_ = size;
        if (size > 0) free_[0] = size;
    }
    int64_t alloc(int64_t bytes)
    {
        bytes = (bytes + 255) & ~int64_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                const int64_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest > 0) free_[off + bytes] = rest;
                used_ += bytes;
                return off;
            }
        return -1;
    }
    void release(int64_t off, int64_t bytes)
    {
        bytes = (bytes + 255) & ~int64_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t used() const { return used_; }
    int64_t size() const { return size_; }

  private:
    std::map<int64_t, int64_t> free_;
    int64_t size_ = 0, used_ = 0;
};

enum ReqState { QUEUED, UPLOADING, IN_WAVE, DONE };

struct Request {
    uint64_t ticket = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int64_t pin_off = -1, pin_bytes = 0;  // host pool: row_ptr, col_idx, colours
    int64_t dev_off = -1, dev_bytes = 0;  // device arena: row_ptr, col_idx
    cudaEvent_t uploaded = nullptr;
    ReqState state = QUEUED;
    int status = GC_OK;
    int32_t rounds = 0;
    int64_t conflicts = 0;
    Clock::time_point t_submit, t_done;
    int32_t *h_rp = nullptr, *h_ci = nullptr, *h_col = nullptr;
    unsigned char *own_pinned = nullptr;  // host block of its own when the pool was full
    bool cancelled = false;               // ticket released; dropped when its GPU work ends
};

constexpr int kLanes = 2;      // waves that can be on the GPU at once
constexpr int kHistory = 64;   // completed wave intervals kept for the overlap count

// One compute lane: a stream, a context (scratch), the wave tables and
// colours, and the wave it runs.
struct Lane {
    gc_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int64_t *h_tab = nullptr;  // vtx_off[G+1] | edge_off[G+1] | rp_off[G+1] (pinned)
    int64_t *d_tab = nullptr;
    int32_t *d_rounds = nullptr, *h_rounds = nullptr;
    int64_t *d_confl = nullptr, *h_confl = nullptr;
    int32_t *d_colors = nullptr;
    int64_t colors_cap = 0;
    cudaEvent_t done = nullptr;                   // wave finished (results on the host)
    cudaEvent_t t_start = nullptr, t_end = nullptr;  // timing: around the colouring
    std::vector<Request *> wave;
    bool inflight = false;
};

struct Interval {
    int lane;
    float start_ms, end_ms;  // since the server's epoch event
};

int64_t dev_footprint(int32_t n, int64_t nnz) { return ((int64_t)n + 1 + nnz) * 4; }
int64_t pin_footprint(int32_t n, int64_t nnz) { return ((int64_t)n + 1 + nnz + n) * 4 + 64; }

}  // namespace

struct gc_server {
    int device = 0;
    uint32_t mode = 0;
    gc_opts opts;
    bool have_opts = false;
    int max_slots = 0;
    cudaStream_t copy = nullptr;
    // device arena (the budget) and pinned host pool
    unsigned char *arena = nullptr;
    Arena arena_alloc;
    unsigned char *pinned = nullptr;
    Arena pinned_alloc;
    Lane lanes[kLanes];
    cudaEvent_t epoch = nullptr;  // timing origin of the wave intervals
    Interval history[kHistory];
    int nhistory = 0;
    // queues and bookkeeping
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::deque<Request *> queue;
    std::vector<Request *> uploading;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::vector<cudaEvent_t> event_pool;
    gc_server_info info;
};

namespace {

cudaEvent_t take_event(gc_server *s)
{
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void release_device(gc_server *s, Request *r)
{
    if (r->dev_off >= 0) {
        s->arena_alloc.release(r->dev_off, r->dev_bytes);
        r->dev_off = -1;
    }
    if (r->uploaded) {
        s->event_pool.push_back(r->uploaded);
        r->uploaded = nullptr;
    }
}

void destroy_request(gc_server *s, Request *r);

void finish(gc_server *s, Request *r, int status)
{
    r->status = status;
    r->state = DONE;
    r->t_done = Clock::now();
    release_device(s, r);
    if (r->cancelled) {  // nobody will poll it
        destroy_request(s, r);
        return;
    }
    if (status == GC_OK || status == GC_ERR_NO_CONVERGENCE) s->info.completed++;
    else s->info.failed++;
}

// The GPU interval of a completed wave (event timestamps, ms since the
// epoch): add its overlap with the earlier completed waves of other lanes.
void account_overlap(gc_server *s, int lane)
{
    const Lane &L = s->lanes[lane];
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, s->epoch, L.t_start) != cudaSuccess ||
        cudaEventElapsedTime(&b, s->epoch, L.t_end) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    bool overlapped = false;
    const int k = std::min(s->nhistory, kHistory);
    for (int i = 0; i < k; ++i) {
        const Interval &h = s->history[i];
        if (h.lane == lane) continue;
        const float ov = std::min(b, h.end_ms) - std::max(a, h.start_ms);
        if (ov > 0.f) {
            s->info.overlap_us += (int64_t)(ov * 1000.f);
            overlapped = true;
        }
    }
    if (overlapped) s->info.overlapped_waves++;
    s->history[s->nhistory % kHistory] = Interval{lane, a, b};
    s->nhistory++;
}

// Complete the wave of a lane (its event has fired).
void complete_wave(gc_server *s, int lane)
{
    Lane &L = s->lanes[lane];
    gc_stats st;
    memset(&st, 0, sizeof st);
    const int rc = gc_ctx_stats(L.ctx, &st);
    account_overlap(s, lane);
    for (size_t g = 0; g < L.wave.size(); ++g) {
        Request *r = L.wave[g];
        r->rounds = L.h_rounds[g];
        r->conflicts = L.h_confl[g];
        finish(s, r, rc);
    }
    L.wave.clear();
    L.inflight = false;
    s->cv_done.notify_all();
}

int resident_count(const gc_server *s)
{
    int k = (int)s->uploading.size();
    for (const Lane &L : s->lanes) k += (int)L.wave.size();
    return k;
}

// Admit queued requests (in order) while arena space and slots allow.
bool admit(gc_server *s)
{
    bool any = false;
    int room = s->max_slots - resident_count(s);
    while (!s->queue.empty() && room > 0) {
        Request *r = s->queue.front();
        const int64_t off = s->arena_alloc.alloc(r->dev_bytes);
        if (off < 0) break;  // wait for memory to come back
        r->dev_off = off;
        r->uploaded = take_event(s);
        int32_t *d = reinterpret_cast<int32_t *>(s->arena + off);
        cudaError_t e = cudaMemcpyAsync(d, r->h_rp, ((size_t)r->n + 1) * 4, cudaMemcpyHostToDevice, s->copy);
        if (e == cudaSuccess && r->nnz > 0)
            e = cudaMemcpyAsync(d + r->n + 1, r->h_ci, (size_t)r->nnz * 4, cudaMemcpyHostToDevice, s->copy);
        if (e == cudaSuccess && r->uploaded) e = cudaEventRecord(r->uploaded, s->copy);
        s->queue.pop_front();
        if (e != cudaSuccess || !r->uploaded) {
            cudaGetLastError();
            finish(s, r, GC_ERR_CUDA);
            s->cv_done.notify_all();
            continue;
        }
        r->state = UPLOADING;
        s->uploading.push_back(r);
        s->info.peak_bytes = std::max<int64_t>(s->info.peak_bytes, s->arena_alloc.used());
        --room;
        any = true;
    }
    return any;
}

bool ensure_wave_colors(Lane &L, int64_t n)
{
    if (n <= L.colors_cap) return true;
    if (L.d_colors) cudaFree(L.d_colors);
    L.d_colors = nullptr;
    L.colors_cap = 0;
    const int64_t cap = std::max<int64_t>(n, 1 << 20);
    if (cudaMalloc(&L.d_colors, (size_t)cap * 4) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    L.colors_cap = cap;
    return true;
}

// Launch one wave on an idle lane over every request whose upload has
// completed (cancelled ones are dropped here).
bool launch_wave(gc_server *s, int lane)
{
    Lane &L = s->lanes[lane];
    std::vector<Request *> ready, waiting;
    bool dropped = false;
    for (Request *r : s->uploading) {
        const cudaError_t q = cudaEventQuery(r->uploaded);
        if (q == cudaSuccess) {
            if (r->cancelled) {
                destroy_request(s, r);
                dropped = true;
            } else {
                ready.push_back(r);
            }
        } else {
            if (q != cudaErrorNotReady) cudaGetLastError();
            waiting.push_back(r);
        }
    }
    s->uploading = waiting;
    if (ready.empty()) return dropped;
    const int G = (int)ready.size();
    int64_t *vtx = L.h_tab, *edge = L.h_tab + (G + 1), *rpo = L.h_tab + 2 * (G + 1);
    vtx[0] = 0;
    for (int g = 0; g < G; ++g) {
        Request *r = ready[g];
        const int64_t base = r->dev_off / 4;  // int32 units from the arena start
        vtx[g + 1] = vtx[g] + r->n;
        rpo[g] = base;
        edge[g] = base + r->n + 1;
    }
    edge[G] = edge[G - 1];
    rpo[G] = 0;
    const int64_t total_n = vtx[G];
    int rc = GC_OK;
    if (!ensure_wave_colors(L, total_n)) rc = GC_ERR_OOM;
    cudaError_t e = cudaSuccess;
    if (rc == GC_OK)
        e = cudaMemcpyAsync(L.d_tab, L.h_tab, (size_t)3 * (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                            L.stream);
    if (rc == GC_OK && e == cudaSuccess) e = cudaEventRecord(L.t_start, L.stream);
    if (rc == GC_OK && e == cudaSuccess)
        rc = gc::color_batch_offsets(L.ctx, G, total_n, s->arena_alloc.size() / 4, L.d_tab, L.d_tab + (G + 1),
                                     L.d_tab + 2 * (G + 1), reinterpret_cast<const int32_t *>(s->arena), s->mode,
                                     &s->opts, L.d_colors, L.d_rounds, L.d_confl, L.stream);
    if (rc == GC_OK && e == cudaSuccess) e = cudaEventRecord(L.t_end, L.stream);
    if (e != cudaSuccess) rc = GC_ERR_CUDA;
    for (int g = 0; g < G && rc == GC_OK; ++g) {
        Request *r = ready[g];
        if (r->n > 0 && cudaMemcpyAsync(r->h_col, L.d_colors + vtx[g], (size_t)r->n * 4, cudaMemcpyDeviceToHost,
                                        L.stream) != cudaSuccess)
            rc = GC_ERR_CUDA;
    }
    if (rc == GC_OK &&
        (cudaMemcpyAsync(L.h_rounds, L.d_rounds, (size_t)G * 4, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
         cudaMemcpyAsync(L.h_confl, L.d_confl, (size_t)G * 8, cudaMemcpyDeviceToHost, L.stream) != cudaSuccess ||
         cudaEventRecord(L.done, L.stream) != cudaSuccess))
        rc = GC_ERR_CUDA;
    if (rc != GC_OK) {
        cudaGetLastError();
        for (Request *r : ready) finish(s, r, rc);
        s->cv_done.notify_all();
        return true;
    }
    for (Request *r : ready) r->state = IN_WAVE;
    L.wave = ready;
    L.inflight = true;
    s->info.waves++;
    s->info.max_wave_graphs = std::max<int32_t>(s->info.max_wave_graphs, G);
    return true;
}

void worker_main(gc_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        for (int l = 0; l < kLanes; ++l) {
            Lane &L = s->lanes[l];
            if (!L.inflight) continue;
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaSuccess) {
                complete_wave(s, l);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                complete_wave(s, l);
                progress = true;
            }
        }
        if (admit(s)) progress = true;
        for (int l = 0; l < kLanes && !s->uploading.empty(); ++l)
            if (!s->lanes[l].inflight && launch_wave(s, l)) progress = true;
        if (!progress) {
            bool busy = !s->uploading.empty();
            for (const Lane &L : s->lanes) busy = busy || L.inflight;
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
    }
}

void fill_stats(const Request *r, gc_stats *st)
{
    if (!st) return;
    int32_t *rs = st->round_sizes;
    const int32_t rcap = st->round_sizes_cap;
    int64_t *rn = st->round_ns;
    const int32_t ncap = st->round_ns_cap;
    memset(st, 0, sizeof *st);
    st->round_sizes = rs;
    st->round_sizes_cap = rcap;
    st->round_ns = rn;
    st->round_ns_cap = ncap;
    st->rounds = r->rounds;
    st->conflicts = r->conflicts;
    int32_t mx = 0;
    std::vector<char> seen;
    for (int32_t v = 0; v < r->n; ++v) mx = std::max(mx, r->h_col[v]);
    seen.assign((size_t)mx + 1, 0);
    int32_t d = 0;
    for (int32_t v = 0; v < r->n; ++v)
        if (r->h_col[v] > 0 && !seen[r->h_col[v]]) {
            seen[r->h_col[v]] = 1;
            ++d;
        }
    st->colors = mx;
    st->distinct_colors = d;
    st->elapsed_ms = (float)std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
}

void destroy_request(gc_server *s, Request *r)
{
    release_device(s, r);
    if (r->pin_off >= 0) {
        s->pinned_alloc.release(r->pin_off, r->pin_bytes);
        r->pin_off = -1;
    }
    if (r->own_pinned) {
        cudaFreeHost(r->own_pinned);
        r->own_pinned = nullptr;
    }
    delete r;
}

}  // namespace

extern "C" {

int gc_server_create(gc_server **out, int device, size_t budget, int max_slots, uint32_t mode, const gc_opts *opts)
{
    if (!out || budget < 4096 || max_slots < 1 || !gc::dist1_mode_ok(mode)) return GC_ERR_ARG;
    *out = nullptr;
    gc_server *s = new (std::nothrow) gc_server();
    if (!s) return GC_ERR_OOM;
    memset(&s->info, 0, sizeof s->info);
    s->device = device;
    s->mode = mode | GC_NO_COLOR_STATS;  // per-request colour counts are taken on the host
    s->max_slots = max_slots;
    memset(&s->opts, 0, sizeof s->opts);
    if (opts) s->opts = *opts;
    int rc = GC_OK;
    for (int l = 0; l < kLanes && rc == GC_OK; ++l) rc = gc_ctx_create(&s->lanes[l].ctx, device);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSuccess;
    if (rc == GC_OK) {
        e = cudaSetDevice(device);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&s->arena, budget);
        if (e == cudaSuccess) e = cudaMallocHost(&s->pinned, 2 * budget);
        if (e == cudaSuccess) e = cudaEventCreate(&s->epoch);
        const size_t tab = (size_t)3 * (max_slots + 1) * sizeof(int64_t);
        for (int l = 0; l < kLanes && e == cudaSuccess; ++l) {
            Lane &L = s->lanes[l];
            e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaMallocHost(&L.h_tab, tab);
            if (e == cudaSuccess) e = cudaMalloc(&L.d_tab, tab);
            if (e == cudaSuccess) e = cudaMalloc(&L.d_rounds, (size_t)max_slots * 4);
            if (e == cudaSuccess) e = cudaMallocHost(&L.h_rounds, (size_t)max_slots * 4);
            if (e == cudaSuccess) e = cudaMalloc(&L.d_confl, (size_t)max_slots * 8);
            if (e == cudaSuccess) e = cudaMallocHost(&L.h_confl, (size_t)max_slots * 8);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreate(&L.t_start);
            if (e == cudaSuccess) e = cudaEventCreate(&L.t_end);
        }
        if (e == cudaSuccess) e = cudaEventRecord(s->epoch, s->copy);
        if (e == cudaSuccess) e = cudaEventSynchronize(s->epoch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
        }
    }
    cudaSetDevice(prev);
    if (rc != GC_OK) {
        gc_server_destroy(s);
        return rc;
    }
    // Each wave takes its share of the SMs, so that the waves of the lanes
    // run side by side (unless the caller chose the blocks per SM).
    if (s->opts.blocks_per_sm == 0) {
        const bool async = (mode & GC_SCHED_ASYNC) != 0;
        s->opts.blocks_per_sm = std::max(1, s->lanes[0].ctx->occ[async][1] / kLanes);
    }
    s->arena_alloc.reset((int64_t)budget);
    s->pinned_alloc.reset((int64_t)(2 * budget));
    s->info.budget_bytes = (int64_t)budget;
    s->info.lanes = kLanes;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GC_OK;
}

int gc_server_submit(gc_server *s, const gc_csr *csr, int32_t n, int64_t nnz, uint64_t *ticket)
{
    gc::NvtxRange nvtx_range("gc_server_submit");
    if (!s || !csr || !ticket || n < 0 || nnz < 0 || nnz > INT32_MAX) return GC_ERR_ARG;
    if (n > 0 && !csr->row_ptr) return GC_ERR_ARG;
    if (nnz > 0 && !csr->col_idx) return GC_ERR_ARG;
    const int64_t dev = dev_footprint(n, nnz), pin = pin_footprint(n, nnz);
    if (dev > s->arena_alloc.size() || pin > s->pinned_alloc.size()) return GC_ERR_BUDGET;
    Request *r = new (std::nothrow) Request();
    if (!r) return GC_ERR_OOM;
    r->n = n;
    r->nnz = nnz;
    r->dev_bytes = dev;
    r->pin_bytes = pin;
    r->t_submit = Clock::now();
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) {
        delete r;
        return GC_ERR_ARG;
    }
    // Host copy: from the pinned pool, or (pool full) a pinned block of its own.
    unsigned char *host = nullptr;
    r->pin_off = s->pinned_alloc.alloc(pin);
    if (r->pin_off >= 0) {
        host = s->pinned + r->pin_off;
    } else {
        lk.unlock();
        if (cudaMallocHost(&r->own_pinned, (size_t)pin) != cudaSuccess) {
            cudaGetLastError();
            delete r;
            return GC_ERR_OOM;
        }
        host = r->own_pinned;
        lk.lock();
    }
    r->h_rp = reinterpret_cast<int32_t *>(host);
    r->h_ci = r->h_rp + n + 1;
    r->h_col = r->h_ci + nnz;
    r->ticket = s->next_ticket++;
    lk.unlock();
    // Copy the caller's arrays (the caller may free them after this call).
    if (n > 0) memcpy(r->h_rp, csr->row_ptr, ((size_t)n + 1) * 4);
    else r->h_rp[0] = 0;
    if (nnz > 0) memcpy(r->h_ci, csr->col_idx, (size_t)nnz * 4);
    lk.lock();
    s->all[r->ticket] = r;
    s->info.submitted++;
    if (n == 0) {
        r->state = UPLOADING;  // trivially coloured: nothing to do
        finish(s, r, GC_OK);
    } else {
        s->queue.push_back(r);
        s->cv_work.notify_one();
    }
    *ticket = r->ticket;
    return GC_OK;
}

int gc_server_poll(gc_server *s, uint64_t ticket, int32_t *colors_out, gc_stats *stats_out)
{
    if (!s) return GC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GC_ERR_NOT_FOUND;
    Request *r = it->second;
    if (r->state != DONE) return GC_PENDING;
    const int status = r->status;
    if (colors_out && r->n > 0 && (status == GC_OK || status == GC_ERR_NO_CONVERGENCE))
        memcpy(colors_out, r->h_col, (size_t)r->n * 4);
    fill_stats(r, stats_out);
    s->all.erase(it);
    destroy_request(s, r);
    return status;
}

int gc_server_wait(gc_server *s, uint64_t ticket, int32_t *colors_out, gc_stats *stats_out, int32_t timeout_ms)
{
    gc::NvtxRange nvtx_range("gc_server_wait");
    if (!s) return GC_ERR_ARG;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
        for (;;) {
            auto it = s->all.find(ticket);
            if (it == s->all.end()) return GC_ERR_NOT_FOUND;
            if (it->second->state == DONE) break;
            if (timeout_ms >= 0 && Clock::now() >= deadline) return GC_PENDING;
            s->cv_done.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
    return gc_server_poll(s, ticket, colors_out, stats_out);
}

int gc_server_cancel(gc_server *s, uint64_t ticket)
{
    if (!s) return GC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GC_ERR_NOT_FOUND;
    Request *r = it->second;
    s->all.erase(it);
    s->info.cancelled++;
    if (r->state == QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
        destroy_request(s, r);
    } else if (r->state == DONE) {
        destroy_request(s, r);
    } else {
        r->cancelled = true;  // on the GPU: dropped when its upload or wave ends
    }
    s->cv_done.notify_all();
    return GC_OK;
}

int gc_server_query(gc_server *s, gc_server_info *out)
{
    if (!s || !out) return GC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    *out = s->info;
    out->in_use_bytes = s->arena_alloc.used();
    out->queued = (int32_t)s->queue.size();
    out->resident = (int32_t)resident_count(s);
    return GC_OK;
}

void gc_server_destroy(gc_server *s)
{
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (Lane &L : s->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    // cancelled requests still held by the worker's lists, then the rest
    for (Request *r : s->uploading)
        if (r->cancelled) destroy_request(s, r);
    for (Lane &L : s->lanes)
        for (Request *r : L.wave)
            if (r->cancelled) destroy_request(s, r);
    for (auto &kv : s->all) {
        release_device(s, kv.second);
        if (kv.second->own_pinned) cudaFreeHost(kv.second->own_pinned);
        delete kv.second;
    }
    s->all.clear();
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    for (Lane &L : s->lanes) {
        if (L.done) cudaEventDestroy(L.done);
        if (L.t_start) cudaEventDestroy(L.t_start);
        if (L.t_end) cudaEventDestroy(L.t_end);
        if (L.ctx) gc_ctx_destroy(L.ctx);
        if (L.h_tab) cudaFreeHost(L.h_tab);
        if (L.d_tab) cudaFree(L.d_tab);
        if (L.d_rounds) cudaFree(L.d_rounds);
        if (L.h_rounds) cudaFreeHost(L.h_rounds);
        if (L.d_confl) cudaFree(L.d_confl);
        if (L.h_confl) cudaFreeHost(L.h_confl);
        if (L.d_colors) cudaFree(L.d_colors);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    if (s->epoch) cudaEventDestroy(s->epoch);
    if (s->arena) cudaFree(s->arena);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->copy) cudaStreamDestroy(s->copy);
    cudaGetLastError();
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
