// Host-side context of libgc (shared by the host translation units; not
// part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "gc_internal.h"

namespace gc {

constexpr int kRoundSizesDev = 65536;  // per-iteration |L| kept on the device

// Default warp/block degree split.  With GC_TIERS it is also the first
// tier's boundary: fewer, larger hubs coloured together keep a dense core's
// concurrent First-Fit choices (and so the colour count) down.
inline int32_t default_t2(uint32_t mode) { return (mode & GC_TIERS) ? 4096 : 2048; }

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    // Grow-only device buffer.  Returns false on allocation failure.
    bool reserve(size_t need)
    {
        if (need <= bytes) return true;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bytes = need;
        return true;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Host fields describing the context's last enqueued colouring (what
// gc_ctx_stats reports on).
struct LastCall {
    bool pending = false;
    int launch_status = GC_OK;
    int32_t n = 0;
    uint32_t mode = 0;
    bool empty = false;
    bool stats = false;
    int32_t rounds_copied = 0;
};

// Enqueue the batch colouring on s (the body of gc_color_batch); see
// color_batch_offsets for the arguments.
int color_batch_impl(gc_ctx *c, int32_t G, int64_t total_n, int64_t total_nnz, const int64_t *vtx_off,
                     const int64_t *edge_off, const int64_t *rp_off, const int32_t *row_ptr, const int32_t *col_idx,
                     uint32_t mode, const gc_opts *opts, int32_t *colors_out, int32_t *rounds_out,
                     int64_t *conflicts_out, cudaStream_t s);

// Allocate everything a batch colouring of this size and mode needs, so
// that a later color_batch_impl call allocates nothing (stream capture).
int reserve_batch(gc_ctx *c, int32_t G, int64_t total_n, uint32_t mode);

}  // namespace gc

struct gc_ctx {
    int device = 0;
    int num_sms = 0;
    int occ[2][2] = {{0, 0}, {0, 0}};       // colouring kernel blocks per SM [async][batch]
    int occ_d2[2] = {0, 0};                 // distance-2 kernel blocks per SM [async]
    // scratch
    gc::Buf cB, wl0, wl1, hb0, hb1, hub_all, mid_all, lut, bitmap, round_sizes, st, done, gstat, uofs, olist;
    gc::Buf pitems;                         // round-0 warp groups: one item per warp of the grid
    gc::Buf cls;                            // gc_color_classes: count matrix and scan sums
    gc::Buf r0mask;                         // round-0 suspect masks (one graph, asynchronous RSOC)
    int32_t pitems_cap = 0;
    gc::Buf stage_rp, stage_ci, stage_col;  // gc_color host staging
    gc::DevState *st_host = nullptr;        // pinned
    int32_t *rs_host = nullptr;             // pinned round sizes
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
    // while a CUDA graph is captured, events are recorded as graph nodes
    bool capturing = false;
    gc::LastCall last;                      // last enqueued call
};
