// Distance-2 colouring on the device: Algorithm 3 (RSOC, Sec. 3) with the
// neighbourhood of a vertex read as its two-hop neighbourhood D2(v) (the
// neighbours u of v and every w != v adjacent to such a u), the colouring
// of G^2 that Sec. 6 names as the method's next target, without building
// G^2.
//
// One persistent, cooperatively launched kernel runs round 0 and every
// while-loop iteration, separated by the bounded grid barrier.  A warp
// inspects one vertex at a time (tiles of 32 worklist entries claimed
// dynamically, as Sec. 5 proposes for SIMT): lanes own neighbours u, and
// the entries of all their rows are then spread evenly over the lanes
// (prefix sum of the row lengths, each lane finding the row of its entry by
// a 5-step shuffle search), so a hub next to low-degree vertices does not
// serialise one lane.  The colours of D2(v) are marked in a 2048-colour
// shared-memory window per warp, the conflict test is taken in the same
// scan, and First-Fit is the first clear bit (the window moves on and D2(v)
// is read again only when 2048 colours are all taken).  A vertex whose
// two-hop neighbourhood has more than d2_heavy entries is flagged in the
// prologue and inspected by a whole block (32768-colour window) after the
// warps' share of each pass.
//
// GC_SCHED_DET: round 0 colours every vertex 1; iteration i reads the
// colours of the end of iteration i-1 from one buffer and writes every
// inspected vertex's colour into the other (the buffers swap each
// iteration; a vertex not inspected in iteration i kept its colour in
// iteration i-1, so both buffers agree on it).  GC_SCHED_ASYNC: round 0 is
// First-Fit over D2(v) for every vertex in place, then iterations over V,
// L, ... read and write one buffer in place.
#include <climits>

#include "gc_device.cuh"

namespace gc {
namespace {

#ifndef GC_D2_UNROLL
#define GC_D2_UNROLL 8
#endif
#ifndef GC_D2_MIN_BLOCKS
#define GC_D2_MIN_BLOCKS 4
#endif
constexpr int kD2Window = 2048;             // colours per First-Fit window of a warp
constexpr int kD2Words = kD2Window / 32;    // window words per warp (2 per lane)
constexpr int kD2Unroll = GC_D2_UNROLL;     // batches of 32 two-hop entries in flight
constexpr int kHeavyWindow = 32768;         // colours per First-Fit window of a block
constexpr int kHeavyWords = kHeavyWindow / 32;

struct D2Shared {
    uint32_t warp_bm[kWarps][kD2Words];
    uint32_t block_bm[kHeavyWords];
    int first_free;
    int item;
};

// Mark colour c in the window of colours [base, base + window): the first
// 64 colours of the window in the lane's register mask `low` (OR-reduced
// over the warp afterwards), the rest in the shared-memory bitmap bm.
__device__ __forceinline__ void d2_mark(uint32_t *bm, unsigned long long &low, int c, int base, int window)
{
    const unsigned o = (unsigned)(c - base);
    if (o < 64u) low |= 1ull << o;
    else if (o < (unsigned)window) atomicOr(bm + (o >> 5), 1u << (o & 31));
}

// One read of this warp's share of D2(v) in the colour buffer R: the
// neighbours at entries kfirst, kfirst + kstride, ... (chunks of 32) of v's
// row, which ends at `end`, and their rows.  Marks every colour in the
// window [base, base + window) (its first 64 colours in the lane's mask
// low); returns (per lane) whether a vertex read on v's tie side holds
// colour cv (only if test).  entries: the lane's share of the two-hop
// entries read (the byte model's 8 per entry of a neighbour's row).
template <bool ASYNC>
__device__ bool d2_read(const KParams &p, const int32_t *R, int32_t v, int64_t kfirst, int64_t end, int kstride,
                        int cv, bool test, int base, int window, uint32_t *bm, unsigned long long &low, int lane,
                        long long &entries)
{
    bool hit = false;
    for (int64_t k0 = kfirst; k0 < end; k0 += kstride) {
        const int64_t k = k0 + lane;
        int ub = 0, du = 0;
        if (k < end) {
            const int32_t u = __ldg(p.col_idx + k);
            ub = __ldg(p.row_ptr + u);
            du = __ldg(p.row_ptr + u + 1) - ub;
            const int cu = ld_color<ASYNC>(R + u);
            d2_mark(bm, low, cu, base, window);
            if (test && cu == cv && on_tie_side(p.tie, u, v)) hit = true;
        }
        entries += du;
        // The rows of this chunk's neighbours laid end to end.  Distinct
        // neighbours have disjoint rows, so the sum fits in 32 bits for any
        // well-formed graph; a malformed one can only misplace entries, and
        // the index check below keeps every load inside col_idx.
        int incl = du;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(FULL_MASK, incl, 31);
        const int excl = incl - du;
        for (int t0 = 0; t0 < total; t0 += 32 * kD2Unroll) {
            int32_t w[kD2Unroll];
#pragma unroll
            for (int j = 0; j < kD2Unroll; ++j) {
                const int t = t0 + j * 32 + lane;
                const int tc = t < total ? t : total - 1;
                // owner lane: the number of lanes whose rows end at or before tc
                int pos = 0;
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const int x = __shfl_sync(FULL_MASK, incl, pos + s - 1);
                    if (x <= tc) pos += s;
                }
                const unsigned idx = (unsigned)__shfl_sync(FULL_MASK, ub, pos) +
                                     (unsigned)(tc - __shfl_sync(FULL_MASK, excl, pos));
                w[j] = (t < total && idx < (unsigned long long)p.nnz) ? __ldg(p.col_idx + idx) : -1;
            }
#pragma unroll
            for (int j = 0; j < kD2Unroll; ++j) {
                if (w[j] >= 0 && w[j] != v) {
                    const int cw = ld_color<ASYNC>(R + w[j]);
                    d2_mark(bm, low, cw, base, window);
                    if (test && cw == cv && on_tie_side(p.tie, w[j], v)) hit = true;
                }
            }
        }
    }
    return hit;
}

// Inspect v (warp-uniform) against R with one warp.  test: v holds colour
// cv and is defective if a vertex of D2(v) on its tie side holds cv too; a
// clean v returns cv.  Otherwise (and always without test) returns the
// smallest colour >= 1 held by no vertex of D2(v).  mb: per-lane byte
// model, 8 per two-hop entry of the first read.
template <bool ASYNC>
__device__ int d2_vertex(const KParams &p, const int32_t *R, int32_t v, int64_t beg, int64_t end, int cv, bool test,
                         uint32_t *bm, int lane, bool &defective, long long &mb)
{
    defective = false;
    for (int base = 1;; base += kD2Window) {
        __syncwarp();
        bm[lane] = 0u;
        bm[lane + 32] = 0u;
        __syncwarp();
        const bool first = base == 1;
        long long e = 0;
        unsigned long long low = 0;
        const bool hit =
            d2_read<ASYNC>(p, R, v, beg, end, 32, cv, test && first, base, kD2Window, bm, low, lane, e);
        if (first) {
            mb += 8 * e;
            defective = __any_sync(FULL_MASK, hit);
            if (test && !defective) return cv;
        }
        const unsigned lo = __reduce_or_sync(FULL_MASK, (unsigned)low);
        const unsigned hi = __reduce_or_sync(FULL_MASK, (unsigned)(low >> 32));
        __syncwarp();
        const uint32_t w0 = bm[lane] | (lane == 0 ? lo : (lane == 1 ? hi : 0u)), w1 = bm[lane + 32];
        unsigned m = __ballot_sync(FULL_MASK, w0 != 0xffffffffu);
        if (m) {
            const int l = __ffs(m) - 1;
            const uint32_t w = __shfl_sync(FULL_MASK, w0, l);
            return base + 32 * l + __ffs(~w) - 1;
        }
        m = __ballot_sync(FULL_MASK, w1 != 0xffffffffu);
        if (m) {
            const int l = __ffs(m) - 1;
            const uint32_t w = __shfl_sync(FULL_MASK, w1, l);
            return base + 32 * (32 + l) + __ffs(~w) - 1;
        }
    }
}

// The same inspection of a heavy vertex by the whole block (block-uniform
// v): warp w reads neighbour chunks w, w + kWarps, ... into one
// kHeavyWindow-colour window.
template <bool ASYNC>
__device__ int d2_vertex_block(const KParams &p, const int32_t *R, int32_t v, int64_t beg, int64_t end, int cv,
                               bool test, D2Shared &sh, int lane, bool &defective, long long &mb)
{
    const int wid = threadIdx.x >> 5;
    defective = false;
    for (int base = 1;; base += kHeavyWindow) {
        __syncthreads();
        for (int w = threadIdx.x; w < kHeavyWords; w += blockDim.x) sh.block_bm[w] = 0u;
        if (threadIdx.x == 0) sh.first_free = INT_MAX;
        __syncthreads();
        const bool first = base == 1;
        long long e = 0;
        unsigned long long low = 0;
        const bool hit = d2_read<ASYNC>(p, R, v, beg + 32 * wid, end, 32 * kWarps, cv, test && first, base,
                                        kHeavyWindow, sh.block_bm, low, lane, e);
        const unsigned lo = __reduce_or_sync(FULL_MASK, (unsigned)low);
        const unsigned hi = __reduce_or_sync(FULL_MASK, (unsigned)(low >> 32));
        if (lane == 0 && lo) atomicOr(&sh.block_bm[0], lo);
        if (lane == 0 && hi) atomicOr(&sh.block_bm[1], hi);
        if (first) {
            mb += 8 * e;
            defective = __syncthreads_or(hit) != 0;
            if (test && !defective) return cv;
        } else {
            __syncthreads();
        }
        for (int w = threadIdx.x; w < kHeavyWords; w += blockDim.x) {
            const uint32_t x = sh.block_bm[w];
            if (x != 0xffffffffu) {
                atomicMin(&sh.first_free, w * 32 + __ffs(~x) - 1);
                break;  // this thread's later words hold larger colours
            }
        }
        __syncthreads();
        const int f = sh.first_free;
        if (f != INT_MAX) return base + f;
    }
}

enum D2Op : int { D2_FF = 0, D2_RSOC = 1 };

// Warps' share of one pass over cnt worklist entries (in == null: the ids
// 0..cnt-1, heavy vertices skipped: the blocks take them), tiles of 32
// entries claimed per warp from *claim.  D2_FF: round 0 of the asynchronous
// schedule, First-Fit for every vertex.  D2_RSOC: one iteration of
// Algorithm 3's while-loop; defective vertices are recoloured and pushed
// onto out (count in *pushed).  mb: the byte model, per lane.
template <bool ASYNC, int OP>
__device__ void d2_pass(const KParams &p, const int32_t *in, int cnt, const int32_t *R, int32_t *W, int32_t *out,
                        int *claim, int *pushed, uint32_t *bm, int lane, long long &mb)
{
    const uint32_t *heavy = reinterpret_cast<const uint32_t *>(p.done);
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(claim, 32);
        t0 = __shfl_sync(FULL_MASK, t0, 0);
        if ((unsigned)t0 >= (unsigned)cnt) break;  // (a wrapped counter reads as past the end)
        const long long i = (long long)t0 + lane;
        int32_t mine = i < cnt ? (in ? __ldcg(in + i) : (int32_t)i) : -1;
        if (!in && mine >= 0 && ((__ldcg(heavy + (mine >> 5)) >> (mine & 31)) & 1u)) mine = -1;
        // the tile's row bounds and own colours, one vertex per lane (a
        // vertex's colour changes only when its own warp recolours it)
        int my_beg = 0, my_end = 0, my_cv = 0;
        if (mine >= 0) {
            my_beg = __ldg(p.row_ptr + mine);
            my_end = __ldg(p.row_ptr + mine + 1);
            if (OP == D2_RSOC) my_cv = ld_color<ASYNC>(R + mine);
        }
        bool my_def = false;
        unsigned todo = __ballot_sync(FULL_MASK, mine >= 0);
        while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t v = __shfl_sync(FULL_MASK, mine, j);
            const int64_t beg = __shfl_sync(FULL_MASK, my_beg, j), end = __shfl_sync(FULL_MASK, my_end, j);
            bool d = false;
            if (OP == D2_FF) {
                const int k = d2_vertex<ASYNC>(p, R, v, beg, end, 0, false, bm, lane, d, mb);
                if (lane == 0) {
                    st_color<ASYNC>(W + v, k);
                    mb += 8 + 16 * (end - beg) + 4;
                }
            } else {
                const int cv = __shfl_sync(FULL_MASK, my_cv, j);
                const int k = d2_vertex<ASYNC>(p, R, v, beg, end, cv, true, bm, lane, d, mb);
                if (lane == 0) {
                    if (!ASYNC || d) st_color<ASYNC>(W + v, k);  // deterministic: every inspected vertex
                    mb += (in ? 4 : 0) + 8 + 4 + 16 * (end - beg) + (d ? 8 : 0);
                }
                if (lane == j) my_def = d;
            }
        }
        if (OP == D2_RSOC) {
            const unsigned dm = __ballot_sync(FULL_MASK, my_def);
            if (dm) {
                int pos = 0;
                if (lane == 0) pos = atomicAdd(pushed, __popc(dm));
                pos = __shfl_sync(FULL_MASK, pos, 0);
                if (my_def) __stcg(out + pos + __popc(dm & ((1u << lane) - 1u)), mine);
            }
        }
    }
}

// Blocks' share of the same pass: the heavy vertices hin[0..hcnt), one
// block each, claimed from *claim.  listed: the entries come from a
// worklist (the byte model's 4 per entry).  Defective vertices go onto hout
// (count in *hpushed): they stay heavy.
template <bool ASYNC, int OP>
__device__ void d2_heavy_pass(const KParams &p, const int32_t *hin, int hcnt, bool listed, const int32_t *R,
                              int32_t *W, int32_t *hout, int *claim, int *hpushed, D2Shared &sh, int lane,
                              long long &mb)
{
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) sh.item = atomicAdd(claim, 1);
        __syncthreads();
        const int it = sh.item;
        if ((unsigned)it >= (unsigned)hcnt) break;
        const int32_t v = __ldcg(hin + it);
        const int64_t beg = __ldg(p.row_ptr + v), end = __ldg(p.row_ptr + v + 1);
        bool d = false;
        if (OP == D2_FF) {
            const int k = d2_vertex_block<ASYNC>(p, R, v, beg, end, 0, false, sh, lane, d, mb);
            if (threadIdx.x == 0) {
                st_color<ASYNC>(W + v, k);
                mb += 8 + 16 * (end - beg) + 4;
            }
        } else {
            const int cv = ld_color<ASYNC>(R + v);
            const int k = d2_vertex_block<ASYNC>(p, R, v, beg, end, cv, true, sh, lane, d, mb);
            if (threadIdx.x == 0) {
                if (!ASYNC || d) st_color<ASYNC>(W + v, k);
                mb += (listed ? 4 : 0) + 8 + 4 + 16 * (end - beg) + (d ? 8 : 0);
                if (d) __stcg(hout + atomicAdd(hpushed, 1), v);
            }
        }
    }
}

// Heavy vertices: two-hop entries (sum of the neighbours' degrees) above
// p.d2_heavy.  One thread per vertex, a warp per 32 consecutive ids writes
// one word of the flag bitmap (p.done) and appends its heavy vertices to
// p.hub_all.
__device__ void d2_find_heavy(const KParams &p, DevState *st, int lane)
{
    uint32_t *flags = reinterpret_cast<uint32_t *>(p.done);
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x; b < p.n; b += gthreads) {
        const long long vi = b + threadIdx.x;
        bool heavy = false;
        if (vi < p.n) {
            const int32_t v = (int32_t)vi;
            const int beg = __ldg(p.row_ptr + v), end = __ldg(p.row_ptr + v + 1);
            if (end - beg > p.d2_heavy) {
                heavy = true;
            } else {
                long long s = 0;
#pragma unroll 4
                for (int k = beg; k < end; ++k) {
                    const int32_t u = __ldg(p.col_idx + k);
                    s += __ldg(p.row_ptr + u + 1) - __ldg(p.row_ptr + u);
                    if (s > p.d2_heavy) {
                        heavy = true;
                        break;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(FULL_MASK, heavy);
        const long long w0 = vi - lane;  // first id of this warp's 32 (a multiple of 32)
        if (lane == 0 && w0 < p.n) flags[w0 >> 5] = m;
        if (m) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(&st->hub_all_count, __popc(m));
            pos = __shfl_sync(FULL_MASK, pos, 0);
            if (heavy) __stcg(p.hub_all + pos + __popc(m & ((1u << lane) - 1u)), (int32_t)vi);
        }
    }
}

template <bool ASYNC>
__global__ void __launch_bounds__(kBlock, GC_D2_MIN_BLOCKS) color_d2_kernel(KParams p)
{
    __shared__ D2Shared sh;
    DevState *st = p.st;
    const int lane = threadIdx.x & 31;
    uint32_t *bm = sh.warp_bm[threadIdx.x >> 5];
    const unsigned nbl = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const long long gthreads = (long long)gridDim.x * blockDim.x;
    long long mb = 0;
    if (lead) st->t_start = global_timer();

    // prologue: heavy vertices; round 0: every vertex colour 1
    // (deterministic), or uncoloured and then First-Fit over D2(v) in place
    // (asynchronous)
    d2_find_heavy(p, st, lane);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gthreads)
        __stcg(p.cA + i, ASYNC ? 0 : 1);
    if (!ASYNC && lead) mb += 4ll * p.n;
    grid_sync(st, nbl);
    const int nheavy = ld_volatile(&st->hub_all_count);
    if (ASYNC && !(ld_volatile(&st->error) & GC_EW_TIMEOUT)) {
        d2_pass<true, D2_FF>(p, nullptr, p.n, p.cA, p.cA, nullptr, &st->pass_hub[0], nullptr, bm, lane, mb);
        d2_heavy_pass<true, D2_FF>(p, p.hub_all, nheavy, false, p.cA, p.cA, nullptr, &st->d2_hclaim0, nullptr, sh,
                                   lane, mb);
        grid_sync(st, nbl);
    }
    if (lead) st->stamp[0] = global_timer();

    // iteration 1: U = V (warps take the light vertices, blocks the heavy
    // list); later: the light and heavy vertices recoloured the iteration
    // before
    const int32_t *in = nullptr, *hin = p.hub_all;
    int cnt = p.n, hcnt = nheavy;
    for (int it = 1; !(ld_volatile(&st->error) & GC_EW_TIMEOUT); ++it) {
        const int r = it & (kRing - 1);
        const int32_t *R = (ASYNC || (it & 1)) ? p.cA : p.cB;
        int32_t *W = (ASYNC || !(it & 1)) ? p.cA : p.cB;
        d2_pass<ASYNC, D2_RSOC>(p, in, cnt, R, W, p.wl[it & 1], &st->pass_tile[r], &st->hub_count[r], bm, lane, mb);
        if (hcnt > 0)
            d2_heavy_pass<ASYNC, D2_RSOC>(p, hin, hcnt, in != nullptr, R, W, p.hub[it & 1], &st->d2_hclaim[r],
                                          &st->d2_hcount[r], sh, lane, mb);
        // counters of iteration it+2: their last readers passed the barrier
        // that ended iteration it-1
        if (lead) {
            const int r2 = (it + 2) & (kRing - 1);
            st->pass_tile[r2] = 0;
            st->hub_count[r2] = 0;
            st->d2_hcount[r2] = 0;
            st->d2_hclaim[r2] = 0;
        }
        grid_sync(st, nbl);
        if (ld_volatile(&st->error) & GC_EW_TIMEOUT) break;
        const int light = ld_volatile(&st->hub_count[r]);
        const int hvy = ld_volatile(&st->d2_hcount[r]);
        const int size = light + hvy;
        if (lead) {
            st->rounds = it;
            st->conflicts += (unsigned long long)size;
            if (it - 1 < p.round_sizes_cap) p.round_sizes[it - 1] = size;
            if (it - 1 < kStamps) st->round_head[it - 1] = size;
            if (it < kStamps) st->stamp[it] = global_timer();
        }
        if (size == 0) break;
        if (it >= p.max_rounds) {
            if (lead) atomicOr(&st->error, GC_EW_NO_CONVERGENCE);
            // the colouring at the cap is the one iteration it wrote
            if (W != p.cA)
                for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += gthreads)
                    __stcg(p.cA + i, __ldcg(W + i));
            break;
        }
        in = p.wl[it & 1];
        cnt = light;
        hin = p.hub[it & 1];
        hcnt = hvy;
    }

    if (p.stats_bitmap) {
        grid_sync(st, nbl);
        colour_stats(p.cA, p.n, st, p.stats_bitmap);
    }
    for (int o = 16; o > 0; o >>= 1) mb += __shfl_down_sync(FULL_MASK, mb, o);
    if (lane == 0 && mb) atomicAdd(&st->model_bytes, (unsigned long long)mb);
}

// Distance-2 validity: every vertex coloured within 1..(two-hop entries)+1
// and no vertex of D2(v) sharing v's colour.  Warp per vertex.
__global__ void check_d2_kernel(KParams p)
{
    const int lane = threadIdx.x & 31;
    bool bad = false;
    for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < p.n;
         v += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int64_t beg = __ldg(p.row_ptr + v), end = __ldg(p.row_ptr + v + 1);
        const int cv = __ldcg(p.cA + v);
        long long reach = 0;
        for (int64_t k = beg + lane; k < end; k += 32) {
            const int32_t u = __ldg(p.col_idx + k);
            if (__ldcg(p.cA + u) == cv) bad = true;
            const int64_t ub = __ldg(p.row_ptr + u), ue = __ldg(p.row_ptr + u + 1);
            reach += ue - ub;
            for (int64_t j = ub; j < ue; ++j) {
                const int32_t w = __ldg(p.col_idx + j);
                if (w != v && __ldcg(p.cA + w) == cv) bad = true;
            }
        }
        for (int o = 16; o > 0; o >>= 1) reach += __shfl_xor_sync(FULL_MASK, reach, o);
        if (cv < 1 || (long long)cv > reach + 1) bad = true;
    }
    if (bad) atomicOr(&p.st->error, GC_EW_CHECK);
}

template <bool A>
cudaError_t launch_d2(const KParams &p, int grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, color_d2_kernel<A>, p);
}

}  // namespace

cudaError_t launch_color_d2(const KParams &p, bool async, int grid, cudaStream_t s)
{
    return async ? launch_d2<true>(p, grid, s) : launch_d2<false>(p, grid, s);
}

cudaError_t query_occupancy_d2(bool async, int *blocks_per_sm)
{
    const void *k = async ? (const void *)color_d2_kernel<true> : (const void *)color_d2_kernel<false>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kBlock, 0);
}

cudaError_t launch_check_d2(const KParams &p, int grid, cudaStream_t s)
{
    check_d2_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace gc
