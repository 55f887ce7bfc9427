// Internal declarations shared by the kernel and host translation units of
// libgc.  Not part of the public ABI (include/gc.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gc.h"

namespace gc {

constexpr int kBlock = 256;             // threads per block of the colouring kernel
constexpr int kWarps = kBlock / 32;
constexpr int kT1Max = 62;              // thread path keeps colours in a 64-bit mask
constexpr int kT2Max = 4096;            // warp path bitmap covers colours 0..kT2Max+1
constexpr int kWarpBmWords = (kT2Max + 2) / 32 + 1;
constexpr int kHubBmWords = 256;        // block path: 8192-colour window per pass
constexpr int kSegCap = 512;            // staged adjacency entries per buffer (2 per warp)
constexpr int kRingIds = 1024;          // ordered graphs: colours of the last ids, per warp
constexpr int kLutShift = 10;           // batch: graph lookup per 1024 vertices
constexpr int kRing = 4;                // round-counter ring depth
constexpr int kStatBitmapWords = 1 << 15;  // distinct-colour bitmap: colours < 2^20
constexpr int kStamps = 256;            // per-iteration end times kept in DevState
constexpr int kWorkBits = 33;           // pushed-degree sum field of wl_packed (< 2^33 entries)
constexpr int kTailWorkPerVertex = 16;  // tail hand-off: at most tail*16 entries left
constexpr int kNearIds = 2048;          // locality: "near" lower neighbour id distance
constexpr int kOrderedSmall = 16384;    // graphs this small are coloured in id order (round 0)
constexpr int kLocalitySample = 64;     // locality: every 64th vertex is sampled
constexpr int kLocalitySampleEntries = 8;   // locality: entries read per sampled vertex
constexpr int kOrderedGroup = 1 << 18;  // graphs this small without hubs or wide rows are ordered (round 0)
constexpr int kPipeMaxK = 512;          // largest warp group colouring one graph in id order
constexpr int kPipeMinChunks = 8;       // fewest chunks per warp of a group
constexpr int kTargetSteps = 32;        // candidate chunk shares per grouped warp (x1.1 apart)
constexpr int kCoreDeg = 4096;          // asynchronous single graph: default degree above which a vertex is in the core
constexpr int kCoreMax = 4096;          // largest core coloured one vertex at a time before round 0
constexpr int kCoreSeg = 1024;          // adjacency entries per task of the core's adjacency build

enum Op : int { OP_TENT = 0, OP_RSOC = 1, OP_DETECT = 2 };

// Mode bits a single-graph colouring accepts: GC_FF_KEEPERS only with
// asynchronous RSOC, lower-keeps ties and in-place repairs; GC_DIST2 only
// with RSOC and neither of the repair variants.
inline bool mode_ok(uint32_t mode)
{
    if (mode & ~GC_MODE_MASK) return false;
    if ((mode & GC_FF_KEEPERS) &&
        (!(mode & GC_SCHED_ASYNC) ||
         (mode & (GC_ALG_TWO_PHASE | GC_TIE_HIGHER_KEEPS | GC_REPAIR_SNAPSHOT | GC_DEBUG_NO_TIEBREAK))))
        return false;
    if ((mode & GC_DIST2) &&
        (mode & (GC_ALG_TWO_PHASE | GC_DEBUG_NO_TIEBREAK | GC_REPAIR_SNAPSHOT | GC_TIERS | GC_FF_KEEPERS)))
        return false;
    return true;
}

// Mode bits of the calls that colour with the distance-1 kernel only
// (batches, plans, the server, the no-alloc and recolour calls, autotuning).
inline bool dist1_mode_ok(uint32_t mode) { return mode_ok(mode) && !(mode & GC_DIST2); }

// Whether a colouring in this mode colours each graph's core of high-degree
// vertices first (asynchronous, a full colouring, the plain First-Fit
// choices of Algorithm 2 or 3 and one stage for all degrees).
inline bool core_applies(uint32_t mode, bool recolor)
{
    return (mode & GC_SCHED_ASYNC) && !recolor && !(mode & (GC_TIERS | GC_FF_KEEPERS | GC_DIST2));
}

// The second n-entry buffer holds colours (deterministic mode, snapshot
// repairs) or, with GC_FF_KEEPERS, the round a vertex was last queued for.
inline bool needs_second_buffer(uint32_t mode)
{
    return !(mode & GC_SCHED_ASYNC) || ((mode & GC_REPAIR_SNAPSHOT) && !(mode & GC_ALG_TWO_PHASE)) ||
           (mode & GC_FF_KEEPERS);
}
enum Tie : int { TIE_LOWER = 0, TIE_HIGHER = 1, TIE_NONE = 2 };

// Per-graph state of one launch (a single graph is graph 0).  Zeroed
// before each launch.
struct GraphStat {
    unsigned long long near_lower;  // locality sample: lower neighbours within kNearIds
    unsigned long long all_lower;   // locality sample: all lower neighbours
    unsigned int hubs;              // vertices of degree > t2
    unsigned int ordered;           // coloured in id order in round 0
    unsigned int wide;              // nonzero: some vertex has kT1Max < degree <= t2
    unsigned int group;             // warps colouring it in id order together (0: one)
    int core_cnt;                   // its hubs of degree > core_deg (core candidates)
    int core_fill;                  // candidates listed so far
    int core_on;                    // nonzero: its core is coloured before round 0
    int core_off;                   // first entry of its core in the core list
    int core_bofs;                  // first word of its core's bit matrix
};

// Device-resident state of one colouring launch.  Zeroed before each launch.
struct DevState {
    unsigned int bar_count;
    unsigned int bar_gen;
    int error;
    int rounds;
    int hub_all_count;
    int mid_all_count;
    int max_color;
    unsigned long long conflicts;
    unsigned long long model_bytes;
    int pass_tile[kRing];      // per-pass claim counters (tiles)
    int pass_hub[kRing];       // per-pass claim counters (hubs)
    int hub_count[kRing];      // per-iteration push counters (hub list)
    // per-iteration tile-list pushes: count << kWorkBits | sum of pushed
    // degrees (tile and hub lists), one atomic per push
    unsigned long long wl_packed[kRing];
    int distinct;
    int seq_claim;                   // round 0: next ordered graph to claim
    int n_ordered;                   // number of ordered graphs coloured by one warp
    int n_pitems;                    // warps of the groups colouring one graph in id order
    long long n_uchunks;             // chunks of the graphs that are not ordered
    int window;                      // number of graphs coloured in id order in round 0
    unsigned long long t_start;      // globaltimer at kernel start (ns)
    unsigned long long stamp[kStamps];  // [0]: end of round 0, [k]: end of iteration k
    int round_head[kStamps];         // |L| of iterations 1..kStamps (copied back with the state)
    unsigned int stats_done;         // colour-statistics blocks finished
    int d2_hcount[kRing];            // distance-2: heavy vertices pushed per iteration
    int d2_hclaim[kRing];            // distance-2: heavy vertices claimed per iteration
    int d2_hclaim0;                  // distance-2: heavy vertices claimed in round 0
    int core_count;                  // entries of the core list (all graphs' cores)
    int core_n;                      // core sorting: next graph to claim
    int core_task;                   // core adjacency build: next task
    int core_colors;                 // core colouring: next graph to claim
    long long core_words;            // words of the cores' bit matrices
};

struct KParams {
    // graph (single graph: G == 1, vtx_off/edge_off/gid_lut null)
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *vtx_off;
    const int64_t *edge_off;
    const int32_t *gid_lut;
    const int64_t *rp_off;     // batch: graph g's row pointers start at row_ptr + rp_off[g]
                               // (null: at row_ptr + vtx_off[g] + g)
    int32_t G;
    int32_t n;                 // total vertices
    int64_t nnz;               // total entries
    // colour buffers
    int32_t *cA;               // caller's output; first buffer
    int32_t *cB;               // second buffer (deterministic mode)
    // worklists (capacity n each; hub lists capacity hub_cap)
    int32_t *wl[2];
    int32_t *hub[2];
    int32_t *hub_all;
    int32_t *mid_all;          // tiered mode: all vertices with t1 < deg <= t2
    int32_t hub_cap;
    DevState *st;
    int32_t *round_sizes;      // device, round_sizes_cap entries
    int32_t round_sizes_cap;
    int32_t *g_rounds;         // batch: per-graph iterations (device, optional)
    unsigned long long *g_conflicts;  // batch: per-graph conflicts (device, optional)
    uint32_t mode;
    int32_t tie;
    int32_t max_rounds;
    int32_t t1, t2;
    int32_t tile;
    int32_t tail;
    int32_t window;            // asynchronous round 0: tiles in flight (0 auto, -1 unlimited)
    int32_t *done;             // per-tile completion flags of the ordered round-0 pass
    GraphStat *gstat;          // G entries (1 for a single graph)
    int64_t *uofs;             // G+1: prefix sums of the unordered graphs' chunk counts
    int32_t *olist;            // G: the ordered graphs
    int32_t *mark;             // GC_FF_KEEPERS: n entries, last iteration a vertex was queued in + 1
    uint32_t *stats_bitmap;    // colour statistics at the end of the launch (null: none); zero on entry
    const int32_t *touched;    // incremental recolouring: the first worklist (null: normal colouring)
    int32_t n_touched;
    int64_t *pitems;           // round 0: (graph, warp, group size) of each grouped warp
    int32_t pitems_cap;        // its capacity (>= the grid's warps)
    int32_t d2_heavy;          // distance 2: two-hop entries above which a block inspects a vertex
    uint64_t *r0mask;          // asynchronous round 0 of one graph: per suspect, the row positions of the
                               // tie-side neighbours read as uncoloured (null: not kept)
    int32_t core_deg;          // asynchronous: each graph's vertices of degree > core_deg (and > t2) are
                               // coloured first, one at a time in decreasing degree (0: no core)
    int32_t round_blocks;      // blocks of the rounds kernel (set by the launcher; the prologue may run on
                               // more, and plans round 0 for these)
};

// Batched colouring with per-graph row-pointer offsets (the server's waves:
// every graph's arrays sit at its own offset in one device arena).
// base: arena start (row pointers and column indices are read relative to
// it); col_extent: int32 entries readable from base.  Same contract as
// gc_color_batch otherwise; finish with gc_ctx_stats.
int color_batch_offsets(gc_ctx *ctx, int32_t G, int64_t total_n, int64_t col_extent, const int64_t *vtx_off,
                        const int64_t *edge_off, const int64_t *rp_off, const int32_t *base, uint32_t mode,
                        const gc_opts *opts, int32_t *colors_out, int32_t *rounds_out, int64_t *conflicts_out,
                        cudaStream_t stream);

// Launchers (gc_kernels.cu).  All return cudaSuccess or the launch error.
cudaError_t launch_color(const KParams &p, bool async, bool batch, int grid, cudaStream_t s);
cudaError_t query_occupancy(bool async, bool batch, int *blocks_per_sm);
size_t color_smem_bytes();
cudaError_t prepare_color_kernels();  // opt in to the kernel's dynamic shared memory
cudaError_t launch_validate(const KParams &p, bool batch, int grid, cudaStream_t s);
cudaError_t launch_check(const KParams &p, bool batch, int grid, cudaStream_t s);
// Distance-2 colouring (gc_d2.cu): the persistent kernel and the check.
cudaError_t launch_color_d2(const KParams &p, bool async, int grid, cudaStream_t s);
cudaError_t query_occupancy_d2(bool async, int *blocks_per_sm);
cudaError_t launch_check_d2(const KParams &p, int grid, cudaStream_t s);
// Failure-path probe (gc_kernels.cu): one bounded wait (GC_WAIT_TILE_DONE,
// GC_WAIT_PIPE_CHUNK or GC_WAIT_STAGE_COPY) run out against p's state.
cudaError_t launch_wait_probe(const KParams &p, int which, unsigned long long timeout_ns, cudaStream_t s);
cudaError_t launch_build_lut(const int64_t *vtx_off, int32_t G, int32_t n, int32_t *lut,
                             cudaStream_t s);

}  // namespace gc
