// Device code of libgc: speculative First-Fit colouring for sm_103a.
//
// One persistent, cooperatively launched kernel runs every round of a
// colouring (Algorithm 3, RSOC, Sec. 3; or Algorithm 2, two-phase, Sec. 2.2)
// with a bounded grid barrier where the paper has "#pragma omp barrier".
// Work inside a round is claimed dynamically from atomic counters in vertex
// order (the remedy Sec. 5 proposes for SIMT lock-step: dynamic assignment of
// vertices to threads) and split by degree:
//   deg <= t1        one thread per vertex, forbidden colours in a 64-bit mask
//   t1 < deg <= t2   one warp per vertex, shared-memory bitmap + ballot/ffs
//   deg > t2         one block per vertex ("hub"), windowed shared bitmap
// Deterministic mode keeps two colour buffers: round i reads one and writes
// every inspected vertex's colour into the other, so each read sees the
// colours of the end of round i-1 exactly, with one barrier per round.
// Asynchronous mode updates one buffer in place, as the paper's threads do.
//
// Conflict rule (tie-break): with rows sorted, the neighbours a vertex can
// lose to form a prefix (lower ids keep their colour) or a suffix (higher ids
// keep theirs), so a clean vertex reads only that side of its row.
#include <climits>

#include "gc_device.cuh"

namespace gc {

// Tile-list pushes of iteration `it` (read after the barrier that ends it).
__device__ __forceinline__ int packed_count(DevState *st, int it)
{
    return (int)(*(volatile unsigned long long *)&st->wl_packed[it & (kRing - 1)] >> kWorkBits);
}

// mbarrier + 1-D bulk (TMA) copy helpers for staging adjacency segments.
__device__ __forceinline__ uint32_t smem_addr(const void *ptr)
{
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred done;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 done, [%1], %2;\n"
        " selp.u32 %0, 1, 0, done;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of
// 16; completion is signalled on `bar` as transaction bytes.  The copied
// column indices are read once per pass: their L2 lines are marked first to
// evict, so that the stream does not push the colour array out of L2.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    unsigned long long policy;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void fence_mbarrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// ------------------------------------------------------------------------
// graph access
// ------------------------------------------------------------------------

// Row of global vertex v: entries [beg, end) of col_idx, neighbour ids are
// nbase + col_idx[k].  For a batch, g is v's graph.
template <bool BATCH>
__device__ __forceinline__ void row_of(const KParams &p, int32_t v, int64_t &beg, int64_t &end,
                                       int32_t &nbase, int32_t &g)
{
    if (!BATCH) {
        beg = __ldg(p.row_ptr + v);
        end = __ldg(p.row_ptr + v + 1);
        nbase = 0;
        g = 0;
    } else {
        // lookup table per 2^kLutShift ids: -(g+1) if the whole block of ids
        // lies in graph g, else g = the graph of its first id (step on)
        const int e = __ldg(p.gid_lut + (v >> kLutShift));
        int gg = e < 0 ? -e - 1 : e;
        if (e >= 0)
            while (gg + 1 < p.G && __ldg(p.vtx_off + gg + 1) <= (int64_t)v) ++gg;
        const int64_t vo = __ldg(p.vtx_off + gg);
        const int64_t eo = __ldg(p.edge_off + gg);
        const int32_t *rp = p.row_ptr + (p.rp_off ? __ldg(p.rp_off + gg) : vo + gg);
        const int32_t lv = v - (int32_t)vo;
        beg = eo + __ldg(rp + lv);
        end = eo + __ldg(rp + lv + 1);
        nbase = (int32_t)vo;
        g = gg;
    }
}

// ------------------------------------------------------------------------
// thread per vertex (deg <= t1 <= 62)
// ------------------------------------------------------------------------

constexpr int kUnroll = 8;     // adjacency entries per thread in flight (thread path)
constexpr int kMinBlocks = 3;  // launch bound: resident blocks per SM the register budget allows

// Adjacency entry k (a global CSR index) of the row being processed: read
// from col_idx, or from the warp's staged copy of the chunk's segment.
// row(beg) gives a cursor over the entries from beg on, indexed with 32-bit
// offsets (rows hold at most 2^31 entries).
struct GlobalEnts {
    const int32_t *col;
    __device__ __forceinline__ int32_t operator()(int64_t k) const { return __ldg(col + k); }
    struct Row {
        const int32_t *p;
        __device__ __forceinline__ int32_t operator[](int i) const { return __ldg(p + i); }
    };
    __device__ __forceinline__ Row row(int64_t beg) const { return Row{col + beg}; }
};
struct StagedEnts {
    const int32_t *buf;        // shared memory: entry k is buf[k - off]
    int64_t off;
    __device__ __forceinline__ int32_t operator()(int64_t k) const { return buf[k - off]; }
    struct Row {
        const int32_t *p;
        __device__ __forceinline__ int32_t operator[](int i) const { return p[i]; }
    };
    __device__ __forceinline__ Row row(int64_t beg) const { return Row{buf + (beg - off)}; }
};

// Smallest colour >= 1 not held by a neighbour u <= vmax (Algorithm 1 body;
// vmax = INT32_MAX takes every neighbour, v - 1 only the lower ones, and the
// sorted row is then read up to v).  With deg <= 62 the answer is <= 63, so
// a 64-bit mask of colours 1..64 suffices.  t = entries read.
template <bool ASYNC, class E>
__device__ __forceinline__ int ff_thread(const E &ent, int64_t beg, int deg, int32_t nbase, const int32_t *R,
                                         int32_t vmax, int &t)
{
    unsigned long long mask = 0;
    t = 0;
    const auto row = ent.row(beg);
    for (int i = 0; i < deg; i += kUnroll) {
        int u[kUnroll];
        bool take[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            const bool in = i + q < deg;
            u[q] = in ? nbase + row[i + q] : 0;
            take[q] = in && u[q] <= vmax;
        }
        int c[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) c[q] = take[q] ? ld_color<ASYNC>(R + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            t += take[q];
            unsigned b = (unsigned)(c[q] - 1);
            if (b < 64u) mask |= 1ull << b;
        }
        if (!take[kUnroll - 1]) break;  // row ended, or passed vmax
    }
    return __ffsll((long long)~mask);
}

// The neighbour bound of a tentative (round-0) First-Fit choice: with degree
// tiers, higher neighbours may hold final colours of an earlier tier that no
// later round inspects, so GC_FF_KEEPERS reads them there.
__device__ __forceinline__ int32_t tent_vmax(const KParams &p, int32_t vmax)
{
    return (p.mode & GC_TIERS) ? INT32_MAX : vmax;
}

template <bool BATCH>
__device__ __forceinline__ void note_push_graph(const KParams &p, int32_t g, int it)
{
    if (BATCH) {
        if (p.g_conflicts) atomicAdd(p.g_conflicts + g, 1ull);
        if (p.g_rounds) atomicMax(p.g_rounds + g, it + 1);
    }
}

// GC_FF_KEEPERS: claim w for the worklist of iteration `it` (mark[w] holds
// the last iteration w was queued in, plus one).  False: already queued.
__device__ __forceinline__ bool claim_push(const KParams &p, int32_t w, int it)
{
    return atomicExch(p.mark + w, it + 1) != it + 1;
}

// GC_FF_KEEPERS: queue w (a higher neighbour that now holds the colour a
// lower neighbour just took) for the next round, in the hub or tile list by
// its degree.
template <bool BATCH>
__device__ __noinline__ void push_one(const KParams &p, int32_t w, int it)
{
    if (!claim_push(p, w, it)) return;
    int64_t beg, end;
    int32_t nbase, g;
    row_of<BATCH>(p, w, beg, end, nbase, g);
    const unsigned long long deg = (unsigned long long)(end - beg);
    DevState *st = p.st;
    if (deg > (unsigned long long)p.t2) {
        atomicAdd(&st->wl_packed[it & (kRing - 1)], deg);
        const int idx = atomicAdd(&st->hub_count[it & (kRing - 1)], 1);
        if (idx < p.hub_cap) __stcg(p.hub[it & 1] + idx, w);
        else atomicOr(&st->error, GC_EW_OVERFLOW);
    } else {
        const int o =
            (int)(atomicAdd(&st->wl_packed[it & (kRing - 1)], (1ull << kWorkBits) + deg) >> kWorkBits);
        if (o < p.n) __stcg(p.wl[it & 1] + o, w);
        else atomicOr(&st->error, GC_EW_OVERFLOW);
    }
    note_push_graph<BATCH>(p, g, it);
}

// GC_FF_KEEPERS: v (lower-keeps ties) just took colour k; every higher
// neighbour holding k now loses the tie to v and is queued.  Reads the part
// of the sorted row above v, from its end.
template <bool ASYNC, bool BATCH, class E>
__device__ __forceinline__ void push_clashes_thread(const KParams &p, const E &ent, int32_t v, int64_t beg,
                                                    int64_t end, int32_t nbase, const int32_t *R, int k, int it)
{
    const int deg = (int)(end - beg);
    const auto row = ent.row(beg);
    for (int i = 0; i < deg; i += kUnroll) {
        int u[kUnroll];
        bool side[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            const bool in = i + q < deg;
            u[q] = in ? nbase + row[deg - 1 - (i + q)] : 0;
            side[q] = in && u[q] > v;
        }
        int c[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < kUnroll; ++q)
            if (side[q] && c[q] == k) push_one<BATCH>(p, u[q], it);
        if (!side[kUnroll - 1]) break;
    }
}

// Is some neighbour on v's tie side coloured cv?  t = tie-side entries seen
// (the whole tie side unless stop_early ended the scan at a conflict).
template <bool ASYNC, class E>
__device__ __forceinline__ bool detect_thread(const E &ent, int tie, int32_t v, int64_t beg, int64_t end,
                                              int32_t nbase, const int32_t *R, int cv, bool stop_early, int &t)
{
    const int deg = (int)(end - beg);
    bool def = false;
    t = 0;
    const auto row = ent.row(beg);
    for (int i = 0; i < deg; i += kUnroll) {
        int u[kUnroll];
        bool side[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            const int ii = i + q;
            const bool in = ii < deg;
            u[q] = in ? nbase + row[(tie == TIE_HIGHER) ? deg - 1 - ii : ii] : 0;
            side[q] = in && on_tie_side(tie, u[q], v);
        }
        int c[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : -1;
#pragma unroll
        for (int q = 0; q < kUnroll; ++q)
            if (side[q]) {
                ++t;
                def |= (c[q] == cv);
            }
        if (tie != TIE_NONE && !side[kUnroll - 1]) break;  // sorted: tie side ended
        if (def && stop_early) break;
    }
    return def;
}

// One vertex, one thread.  Returns true if v must join the next worklist.
// Byte model accounting goes to mb (see gc.h, gc_stats.model_bytes).
template <bool ASYNC, bool BATCH, class E>
__device__ __forceinline__ bool vertex_thread(const KParams &p, const E &ent, int op, int32_t v, int64_t beg,
                                              int64_t end, int32_t nbase, const int32_t *R, int32_t *W,
                                              bool implicit, long long &mb, int it)
{
    const int deg = (int)(end - beg);
    const bool keep = ASYNC && (p.mode & GC_FF_KEEPERS);
    const int32_t vmax = keep ? v - 1 : INT32_MAX;
    mb += (implicit ? 0 : 4) + 8;
    int t;
    if (op == OP_TENT) {
        st_color<ASYNC>(W + v, ff_thread<ASYNC>(ent, beg, deg, nbase, R, tent_vmax(p, vmax), t));
        mb += 8ll * t + 4;
        return false;
    }
    const int cv = ld_color<ASYNC>(R + v);
    mb += 4;
    bool d;
    if (ASYNC && !BATCH && op == OP_RSOC && it == 1 && p.r0mask && !implicit) {  // (masks: one graph only)
        // First repair after round 0: only the neighbours this vertex read
        // as uncoloured there can share its colour (see chunk_tent_ordered).
        unsigned long long m = __ldcg(reinterpret_cast<const unsigned long long *>(p.r0mask) + v);
        const auto row = ent.row(beg);
        bool def = cv == 0;
        t = 0;
        while (m) {
            // four named positions at a time: their entries, then their
            // colours, loaded together
            constexpr int kQ = 4;
            int pos[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                pos[q] = m ? __ffsll((long long)m) - 1 : -1;
                m &= m - 1;
            }
            int32_t u[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) u[q] = pos[q] >= 0 ? nbase + row[pos[q]] : 0;
            int c[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) c[q] = pos[q] >= 0 ? ld_color<ASYNC>(R + u[q]) : -1;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                t += pos[q] >= 0;
                def |= c[q] == cv;
            }
        }
        d = def;
        mb += 8;  // the mask
    } else {
        d = detect_thread<ASYNC>(ent, p.tie, v, beg, end, nbase, R, cv, op == OP_RSOC, t) || cv == 0;
    }
    if (op == OP_DETECT) {
        if (!ASYNC) st_color<false>(p.cA + v, cv);  // two-phase: bring buffer A up to date
        mb += 8ll * t + (d ? 4 : 0);
        return d;
    }
    if (d) {
        int tf;
        const int k = ff_thread<ASYNC>(ent, beg, deg, nbase, R, vmax, tf);
        st_color<ASYNC>(W + v, k);
        if (keep) push_clashes_thread<ASYNC, BATCH>(p, ent, v, beg, end, nbase, R, k, it);
        mb += 8ll * deg + 8;
    } else {
        if (W != R) st_color<ASYNC>(W + v, cv);  // snapshot rounds: carry the colour over
        mb += 8ll * t;
    }
    return d;
}

// ------------------------------------------------------------------------
// warp per vertex (t1 < deg <= t2 <= kT2Max)
// ------------------------------------------------------------------------

// Warp-wide First-Fit over the neighbours u <= vmax (see ff_thread);
// t_total = entries read.
template <bool ASYNC>
__device__ int ff_warp(const KParams &p, int64_t beg, int deg, int32_t nbase, const int32_t *R, int32_t vmax,
                       uint32_t *bm, int lane, int &t_total)
{
    int t = 0;
    const int nwords = (deg + 1) / 32 + 1;  // bits for colours 0..deg+1
    __syncwarp();
    for (int w = lane; w < nwords; w += 32) bm[w] = (w == 0) ? 1u : 0u;  // colour 0 is not a colour
    __syncwarp();
    for (int i0 = 0; i0 < deg; i0 += 32 * 4) {
        int c[4];
        bool take[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * 32 + lane;
            const int32_t u = (i < deg) ? nbase + __ldg(p.col_idx + beg + i) : 0;
            take[q] = i < deg && u <= vmax;
            c[q] = take[q] ? ld_color<ASYNC>(R + u) : 0;
            t += take[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if ((unsigned)c[q] <= (unsigned)(deg + 1)) atomicOr(&bm[c[q] >> 5], 1u << (c[q] & 31));
        if (!(__ballot_sync(FULL_MASK, take[3]) >> 31)) break;  // row ended, or passed vmax
    }
    t_total = __reduce_add_sync(FULL_MASK, t);
    __syncwarp();
    for (int w0 = 0; w0 < nwords; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t freeb = (w < nwords) ? ~bm[w] : 0u;
        const unsigned bal = __ballot_sync(FULL_MASK, freeb != 0u);
        if (bal) {
            const int src = __ffs(bal) - 1;
            const uint32_t fb = __shfl_sync(FULL_MASK, freeb, src);
            return (w0 + src) * 32 + __ffs(fb) - 1;
        }
    }
    return deg + 1;  // not reached: one of 1..deg+1 is always free
}

// Warp-wide push_clashes_thread: queue v's higher neighbours that hold k.
template <bool ASYNC, bool BATCH>
__device__ void push_clashes_warp(const KParams &p, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                                  const int32_t *R, int k, int it, int lane)
{
    const int deg = (int)(end - beg);
    for (int i0 = 0; i0 < deg; i0 += 32 * 4) {
        int32_t u[4];
        bool side[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + q * 32 + lane;
            u[q] = (i < deg) ? nbase + __ldg(p.col_idx + end - 1 - i) : 0;
            side[q] = i < deg && u[q] > v;
        }
        int c[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (side[q] && c[q] == k) push_one<BATCH>(p, u[q], it);
        if (!(__ballot_sync(FULL_MASK, side[3]) >> 31)) break;
    }
}

constexpr int kWarpUnroll = 4;   // entries per lane in flight (warp path)
constexpr int kBlockUnroll = 4;  // entries per thread in flight (block path)
constexpr int kSusBuf = 64;      // round 0: suspects a warp collects before one append

template <bool ASYNC>
__device__ bool detect_warp(const KParams &p, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                            const int32_t *R, int cv, bool stop_early, int lane, int &t_total)
{
    const int deg = (int)(end - beg);
    const int tie = p.tie;
    bool def = false;
    int t = 0;
    for (int i0 = 0; i0 < deg; i0 += 32 * kWarpUnroll) {
        int32_t u[kWarpUnroll];
        bool side[kWarpUnroll];
#pragma unroll
        for (int q = 0; q < kWarpUnroll; ++q) {
            const int ii = i0 + q * 32 + lane;
            const bool in = ii < deg;
            const int64_t k = (tie == TIE_HIGHER) ? end - 1 - ii : beg + ii;
            u[q] = in ? nbase + __ldg(p.col_idx + k) : 0;
            side[q] = in && on_tie_side(tie, u[q], v);
        }
        int c[kWarpUnroll];
#pragma unroll
        for (int q = 0; q < kWarpUnroll; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : -1;
#pragma unroll
        for (int q = 0; q < kWarpUnroll; ++q)
            if (side[q]) {
                ++t;
                def |= (c[q] == cv);
            }
        const unsigned more = __ballot_sync(FULL_MASK, side[kWarpUnroll - 1]);
        const bool any_def = __any_sync(FULL_MASK, def);
        if (tie != TIE_NONE && !(more >> 31)) break;
        if (any_def && stop_early) break;
    }
    t_total = __reduce_add_sync(FULL_MASK, t);
    return __any_sync(FULL_MASK, def);
}

template <bool ASYNC, bool BATCH>
__device__ __noinline__ bool vertex_warp(const KParams &p, int op, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                            const int32_t *R, int32_t *W, bool implicit, long long &mb, uint32_t *bm,
                            int lane, int it)
{
    const int deg = (int)(end - beg);
    const bool keep = ASYNC && (p.mode & GC_FF_KEEPERS);
    const int32_t vmax = keep ? v - 1 : INT32_MAX;
    long long add = (implicit ? 0 : 4) + 8;
    bool d = false;
    int tf;
    if (op == OP_TENT) {
        const int c = ff_warp<ASYNC>(p, beg, deg, nbase, R, tent_vmax(p, vmax), bm, lane, tf);
        if (lane == 0) st_color<ASYNC>(W + v, c);
        add += 8ll * tf + 4;
    } else {
        const int cv = ld_color<ASYNC>(R + v);
        add += 4;
        int t;
        d = detect_warp<ASYNC>(p, v, beg, end, nbase, R, cv, op == OP_RSOC, lane, t) || cv == 0;
        if (op == OP_DETECT) {
            if (!ASYNC && lane == 0) st_color<false>(p.cA + v, cv);
            add += 8ll * t + (d ? 4 : 0);
        } else if (d) {
            const int c = ff_warp<ASYNC>(p, beg, deg, nbase, R, vmax, bm, lane, tf);
            if (lane == 0) st_color<ASYNC>(W + v, c);
            if (keep) push_clashes_warp<ASYNC, BATCH>(p, v, beg, end, nbase, R, c, it, lane);
            add += 8ll * deg + 8;
        } else {
            if (W != R && lane == 0) st_color<ASYNC>(W + v, cv);
            add += 8ll * t;
        }
    }
    if (lane == 0) mb += add;
    return d;
}

// ------------------------------------------------------------------------
// block per vertex (deg > t2)
// ------------------------------------------------------------------------

struct Shared {
    int32_t seg[kWarps][2][kSegCap];         // staged adjacency segments (double buffer per warp)
    uint16_t ring[kWarps][kRingIds];         // ordered graphs: colours of the warp's last ids
    unsigned long long mbar[kWarps][2];      // their completion barriers
    struct SlotInfo {
        long long cb;                        // first id of the chunk; -1: none
        long long cend;                      // ids of the chunk stop here
        long long soff;                      // entry index held by seg[..][0]; -1: not staged
        int tile, kin;                       // claimed tile and chunk index inside it
    } slot[kWarps][2];
    uint32_t warp_bm[kWarps][kWarpBmWords];
    uint32_t hub_bm[kHubBmWords];
    int32_t sus[kWarps][kSusBuf];            // round 0: suspects of the warp not yet appended
    int found;                               // detect_block: a conflict was seen
    int first;
    int tcount;
    int claim;
};

// Block-wide First-Fit over the neighbours u <= vmax (see ff_thread), in
// windows of kHubBmWords*32 colours; t_total = entries read.
template <bool ASYNC>
__device__ int ff_block(const KParams &p, int64_t beg, int deg, int32_t nbase, const int32_t *R, int32_t vmax,
                        Shared &sh, int &t_total)
{
    constexpr int kWin = kHubBmWords * 32;
    if (threadIdx.x == 0) sh.tcount = 0;
    for (int base = 0;; base += kWin) {
        for (int w = threadIdx.x; w < kHubBmWords; w += kBlock) sh.hub_bm[w] = 0u;
        if (threadIdx.x == 0) sh.first = INT_MAX;
        __syncthreads();
        int t = 0;
        for (int i0 = 0; i0 < deg; i0 += kBlock * kBlockUnroll) {
            int c[kBlockUnroll];
            bool take[kBlockUnroll];
#pragma unroll
            for (int q = 0; q < kBlockUnroll; ++q) {
                const int i = i0 + q * kBlock + threadIdx.x;
                const int32_t u = (i < deg) ? nbase + __ldg(p.col_idx + beg + i) : 0;
                take[q] = i < deg && u <= vmax;
                c[q] = take[q] ? ld_color<ASYNC>(R + u) : -1;
                t += take[q];
            }
#pragma unroll
            for (int q = 0; q < kBlockUnroll; ++q) {
                const int d = c[q] - base;
                if (c[q] >= 0 && d >= 0 && d < kWin) atomicOr(&sh.hub_bm[d >> 5], 1u << (d & 31));
            }
            // A thread's entries rise with i in a sorted row: once one is
            // past the row's end or vmax, so are all its later ones.  No
            // barrier: every thread runs ahead on its own entries.
            if (!take[kBlockUnroll - 1]) break;
        }
        if (base == 0 && t) atomicAdd(&sh.tcount, t);
        __syncthreads();
        for (int w = threadIdx.x; w < kHubBmWords; w += kBlock) {
            uint32_t f = ~sh.hub_bm[w];
            if (w == 0 && base == 0) f &= ~1u;  // colour 0 is not a colour
            if (f) atomicMin(&sh.first, w * 32 + __ffs(f) - 1);
        }
        __syncthreads();
        const int first = sh.first;
        t_total = sh.tcount;
        __syncthreads();
        if (first != INT_MAX) return base + first;
        if (base > deg + 1) return deg + 1;  // not reached
    }
}

// Block-wide push_clashes_thread: queue v's higher neighbours that hold k.
template <bool ASYNC, bool BATCH>
__device__ void push_clashes_block(const KParams &p, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                                   const int32_t *R, int k, int it)
{
    const int deg = (int)(end - beg);
    for (int i0 = 0; i0 < deg; i0 += kBlock * kBlockUnroll) {
        int32_t u[kBlockUnroll];
        bool side[kBlockUnroll];
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q) {
            const int i = i0 + q * kBlock + threadIdx.x;
            u[q] = (i < deg) ? nbase + __ldg(p.col_idx + end - 1 - i) : 0;
            side[q] = i < deg && u[q] > v;
        }
        int c[kBlockUnroll];
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q)
            if (side[q] && c[q] == k) push_one<BATCH>(p, u[q], it);
        if (!side[kBlockUnroll - 1]) break;  // this thread's entries fell to v or below
    }
}

template <bool ASYNC>
__device__ bool detect_block(const KParams &p, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                             const int32_t *R, int cv, bool stop_early, Shared &sh, int &t_total)
{
    const int deg = (int)(end - beg);
    const int tie = p.tie;
    bool def = false;
    int t = 0;
    if (threadIdx.x == 0) {
        sh.tcount = 0;
        sh.found = 0;
    }
    __syncthreads();
    for (int i0 = 0; i0 < deg; i0 += kBlock * kBlockUnroll) {
        int32_t u[kBlockUnroll];
        bool side[kBlockUnroll];
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q) {
            const int ii = i0 + q * kBlock + threadIdx.x;
            const bool in = ii < deg;
            const int64_t k = (tie == TIE_HIGHER) ? end - 1 - ii : beg + ii;
            u[q] = in ? nbase + __ldg(p.col_idx + k) : 0;
            side[q] = in && on_tie_side(tie, u[q], v);
        }
        int c[kBlockUnroll];
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q) c[q] = side[q] ? ld_color<ASYNC>(R + u[q]) : -1;
#pragma unroll
        for (int q = 0; q < kBlockUnroll; ++q)
            if (side[q]) {
                ++t;
                def |= (c[q] == cv);
            }
        // No barrier per step: a thread's entries move away from v in a
        // sorted row (up from the row start, or down from its end with
        // higher-keeps ties), so once one leaves the tie side all its later
        // ones do; a conflict found by any thread ends the others' scans
        // through a shared flag.
        if (def && stop_early) *(volatile int *)&sh.found = 1;
        if (tie != TIE_NONE && !side[kBlockUnroll - 1]) break;
        if (stop_early && *(volatile int *)&sh.found) break;
    }
    if (t) atomicAdd(&sh.tcount, t);
    const int any = __syncthreads_or((int)def);
    t_total = sh.tcount;
    __syncthreads();
    return any != 0;
}

template <bool ASYNC, bool BATCH>
__device__ __noinline__ bool vertex_block(const KParams &p, int op, int32_t v, int64_t beg, int64_t end, int32_t nbase,
                             const int32_t *R, int32_t *W, bool implicit, long long &mb, Shared &sh, int it)
{
    const int deg = (int)(end - beg);
    const bool keep = ASYNC && (p.mode & GC_FF_KEEPERS);
    const int32_t vmax = keep ? v - 1 : INT32_MAX;
    long long add = (implicit ? 0 : 4) + 8;
    bool d = false;
    int tf;
    if (op == OP_TENT) {
        const int c = ff_block<ASYNC>(p, beg, deg, nbase, R, tent_vmax(p, vmax), sh, tf);
        if (threadIdx.x == 0) st_color<ASYNC>(W + v, c);
        add += 8ll * tf + 4;
    } else {
        const int cv = ld_color<ASYNC>(R + v);
        add += 4;
        int t;
        d = detect_block<ASYNC>(p, v, beg, end, nbase, R, cv, op == OP_RSOC, sh, t) || cv == 0;
        if (op == OP_DETECT) {
            if (!ASYNC && threadIdx.x == 0) st_color<false>(p.cA + v, cv);
            add += 8ll * t + (d ? 4 : 0);
        } else if (d) {
            const int c = ff_block<ASYNC>(p, beg, deg, nbase, R, vmax, sh, tf);
            if (threadIdx.x == 0) st_color<ASYNC>(W + v, c);
            if (keep) push_clashes_block<ASYNC, BATCH>(p, v, beg, end, nbase, R, c, it);
            add += 8ll * deg + 8;
        } else {
            if (W != R && threadIdx.x == 0) st_color<ASYNC>(W + v, cv);
            add += 8ll * t;
        }
    }
    if (threadIdx.x == 0) mb += add;
    return d;
}

// ------------------------------------------------------------------------
// ordered tentative colouring of a chunk of 32 consecutive ids (round 0)
// ------------------------------------------------------------------------

// The 32 lanes colour ids cbase..cbase+31 as sequential First-Fit would:
// lane k sees the final colours of every lower lane it is adjacent to (they
// are resolved in lane order through shuffles) and the current colours of
// every neighbour outside the chunk.  This removes the lock-step tie of
// Sec. 5 / Fig. 7 inside a warp.  Hub ids (coloured before the tiles) count
// as outside; warp-path ids are coloured afterwards and see all lanes.
// Returns true on lanes whose vertex may end round 0 in conflict with a
// neighbour it can lose to (see `suspect` below); such vertices form the
// first repair worklist instead of all of V.
constexpr uint16_t kRingGlobal = 0xFFFFu;  // ring entry: read this id's colour from memory

// The colours the 32 lanes of a chunk take when they are coloured in lane
// (id) order: ext = colours of a lane's neighbours outside the chunk (bit
// c-1 for colour c), low = the lower lanes it is adjacent to, act = the lane
// has a vertex to colour.  Lanes in no lane's `low` and with act false do not
// take part; their result is 0.
__device__ __forceinline__ int resolve_in_order(unsigned long long ext, unsigned low, bool act, int lane)
{
    int mine = act ? __ffsll((long long)~ext) : 0;
    // In-chunk dependencies: walk only the lanes between the first lane some
    // lane depends on and the last dependent lane, in id order.  Branch-free:
    // every lane recomputes its candidate each step and lane k's is taken.
    const unsigned dependent = __ballot_sync(FULL_MASK, low != 0u);
    if (dependent) {
        const unsigned needed = __reduce_or_sync(FULL_MASK, low);
        const int k0 = __ffs(needed) - 1;
        const int k1 = 31 - __clz(dependent);
        // 32-bit masks suffice when every lane keeps a free colour in 1..31
        // whatever its in-chunk neighbours pick.
        const bool narrow = __all_sync(FULL_MASK, (ext >> 31) == 0ull &&
                                                      __popc((uint32_t)ext) + __popc(low) <= 30);
        // Chain: every lane depends on nothing in the chunk or on the lane
        // just below it (consecutive ids along a mesh row).  Lane k's colour
        // is then F_k(colour of lane k-1) with F_k(c) = (c == A) ? X : Y
        // (A, Y its first free colour, X its second), a form closed under
        // composition, so an inclusive scan of the F's over the lanes gives
        // every colour in five shuffle steps.
        const bool chain = __all_sync(FULL_MASK, low == 0u || low == (1u << ((lane + 31) & 31)));
        if (chain) {
            const int a = __ffsll((long long)~ext);
            int A = 0, X = a, Y = a;  // low == 0: constant a
            if (low) {
                A = a;
                X = __ffsll((long long)~(ext | (1ull << (a - 1))));
            }
            for (int d = 1; d < 32; d <<= 1) {
                const int A2 = __shfl_up_sync(FULL_MASK, A, d);
                const int X2 = __shfl_up_sync(FULL_MASK, X, d);
                const int Y2 = __shfl_up_sync(FULL_MASK, Y, d);
                if (lane >= d) {  // compose: this lane's function after lane-d's
                    const int nX = (X2 == A) ? X : Y;
                    const int nY = (Y2 == A) ? X : Y;
                    A = A2;
                    X = nX;
                    Y = nY;
                }
            }
            mine = X;  // lane 0's function is constant, so the composition is too
        } else if (narrow) {
            uint32_t e32 = (uint32_t)ext;
            for (int k = k0; k <= k1; ++k) {
                const int cand = __ffs(~e32);
                const int ck = __shfl_sync(FULL_MASK, cand, k);
                mine = (lane == k) ? cand : mine;
                e32 |= ((low >> k) & 1u) << (ck - 1);
            }
            if (lane > k1) mine = __ffs(~e32);
        } else {
            for (int k = k0; k <= k1; ++k) {
                const int cand = __ffsll((long long)~ext);
                const int ck = __shfl_sync(FULL_MASK, cand, k);
                mine = (lane == k) ? cand : mine;
                ext |= (unsigned long long)((low >> k) & 1u) << (ck - 1);
            }
            if (lane > k1) mine = __ffsll((long long)~ext);
        }
        if (!act) mine = 0;
    }
    return mine;
}

// RING: the chunk belongs to an ordered graph that this warp colours in id
// order from v0; ids in [max(v0, cbase - kRingIds), cbase) were coloured by
// this warp and their colours sit in `ring`; with skip_higher no id above
// the chunk is coloured yet (the graph has no vertex coloured elsewhere).
// LEAN: the caller has checked that every vertex of the chunk takes the
// thread path (no hub, no warp-path lane), that lower ids keep their colours
// and that GC_FF_KEEPERS is off; the checks for those cases drop out of the
// per-entry work.
// What a lean chunk's lane read as uncoloured on its tie side: the first
// two such neighbours (u0, u1), how many there were (zc) and the colour the
// lane took (cv), so that the suspect can be checked again a chunk later.
struct SusHint {
    int32_t u0, u1;
    int zc;
    int cv;
};

template <class E, bool RING, bool LEAN = false>
__device__ bool chunk_tent_ordered(const KParams &p, const E &ent, long long cbase, int32_t v, int64_t beg,
                                   int64_t end, int32_t nbase, int32_t *C, long long &mb, uint32_t *bm, int lane,
                                   int dmax, uint16_t *ring = nullptr, long long v0 = 0, bool skip_higher = false,
                                   int32_t unclaimed = INT32_MAX, SusHint *hint = nullptr)
{
    if (LEAN && hint) hint->zc = 0;
    const int deg = (int)(end - beg);
    const int tie = LEAN ? (int)TIE_LOWER : p.tie;
    const bool hub = !LEAN && v >= 0 && deg > dmax;  // coloured before this pass
    const bool mid = !LEAN && v >= 0 && !hub && deg > p.t1;
    const bool thr = v >= 0 && !hub && !mid;
    const unsigned hubmask = LEAN ? 0u : __ballot_sync(FULL_MASK, hub);
    const unsigned midmask = LEAN ? 0u : __ballot_sync(FULL_MASK, mid);
    unsigned long long ext = 0;
    unsigned low = 0;
    const int32_t cb32 = (int32_t)cbase;  // ids are below 2^31
    const int32_t v032 = (int32_t)v0;
    // Every vertex is written once in round 0, so a non-zero colour read
    // for a neighbour is that neighbour's final round-0 colour and the
    // First-Fit choice avoids it.  Lanes inside the chunk are resolved in
    // id order (a higher or warp-path lane sees this lane's final colour).
    // So an edge can end round 0 monochromatic only if one endpoint read the
    // other as uncoloured: that endpoint is the suspect when the tie-break
    // makes it the one to recolour.
    bool suspect = mid;
    // Row positions of the neighbours on the tie side read as uncoloured:
    // the only ones that can clash with this lane after round 0 (the others
    // were read with their final round-0 colours, which First-Fit avoided).
    unsigned long long zmask = 0;
    // GC_FF_KEEPERS: only lower neighbours count, and the sorted row is read
    // up to v.
    // With degree tiers the higher neighbours read here may be final
    // colours of an earlier tier, which no later round inspects: read them.
    const bool keepers = !LEAN && (p.mode & GC_FF_KEEPERS) != 0 && !(p.mode & GC_TIERS);
    // An ordered graph whose higher ids are all uncoloured (skip_higher)
    // gains nothing from the part of a row above v either.
    const bool keep = keepers || (RING && skip_higher);
    int nread = 0, nskip = 0;
    if (thr) {
        const auto row = ent.row(beg);
        for (int i = 0; i < deg; i += kUnroll) {
            int u[kUnroll];
            bool outside[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                u[q] = (i + q < deg) ? nbase + row[i + q] : -1;
                if (keep && u[q] > v) u[q] = -1;
                nread += u[q] >= 0;
                const uint32_t d = (uint32_t)(u[q] - cb32);  // in-chunk offset (wraps when outside)
                const bool inside = u[q] >= 0 && d < 32u && !((hubmask >> d) & 1u);
                if (inside && u[q] < v && !((midmask >> d) & 1u)) low |= 1u << d;
                // A lower warp-path lane is coloured after this one and, with
                // keepers, without looking at it: the pair is not checked
                // unless this lane is.
                if (keepers && inside && u[q] < v && ((midmask >> d) & 1u)) suspect = true;
                outside[q] = u[q] >= 0 && !inside;
            }
            int c[kUnroll];
            if (RING) {
                bool glob[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    glob[q] = outside[q];
                    c[q] = 0;
                    if (outside[q] && u[q] < cb32 && u[q] >= v032 && cb32 - u[q] <= kRingIds) {
                        const uint16_t r = ring[u[q] & (kRingIds - 1)];
                        glob[q] = r == kRingGlobal;
                        c[q] = r;
                    } else if (outside[q] && skip_higher && u[q] >= cb32 + 32) {
                        glob[q] = false;  // not coloured yet in id order
                    }
                }
#pragma unroll
                for (int q = 0; q < kUnroll; ++q)
                    if (glob[q]) c[q] = ld_color<true>(C + u[q]);
            } else {
                // Ids from `unclaimed` on belong to tiles no warp has claimed
                // yet: uncoloured, so their colours are not read (what the
                // read would return, taken a moment earlier).
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    const bool skip = outside[q] && u[q] >= unclaimed;
                    nskip += skip;
                    c[q] = (outside[q] && !skip) ? ld_color<true>(C + u[q]) : 0;
                }
            }
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const unsigned b = (unsigned)(c[q] - 1);
                if (b < 64u) ext |= 1ull << b;
                if (outside[q] && c[q] == 0 && on_tie_side(tie, u[q], v)) {
                    suspect = true;
                    zmask |= 1ull << (i + q);  // i + q < deg <= t1 <= 62
                    if (LEAN && hint) {
                        if (hint->zc == 0) hint->u0 = u[q];
                        else if (hint->zc == 1) hint->u1 = u[q];
                        ++hint->zc;
                    }
                }
            }
            if (keep && u[kUnroll - 1] < 0) break;  // row ended, or passed v
        }
    }
    __syncwarp();
    const int mine = resolve_in_order(ext, low, thr, lane);
    if (LEAN && hint) hint->cv = mine;
    if (thr) {
        st_color<true>(C + v, mine);
        mb += 8 + 8ll * nread - 4ll * nskip + 4;  // index only for the unread colours
        if (zmask && p.r0mask) __stcg(reinterpret_cast<unsigned long long *>(p.r0mask) + v, zmask);
    }
    __syncwarp();
    unsigned mm = midmask;
    while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const int32_t vv = __shfl_sync(FULL_MASK, v, src);
        const int64_t bb = __shfl_sync(FULL_MASK, beg, src);
        const int64_t ee = __shfl_sync(FULL_MASK, end, src);
        const int32_t nb = __shfl_sync(FULL_MASK, nbase, src);
        vertex_warp<true, false>(p, OP_TENT, vv, bb, ee, nb, C, C, true, mb, bm, lane, 0);
    }
    if (RING) {
        __syncwarp();
        if (v >= 0) {
            uint16_t r = kRingGlobal;
            if (thr) r = (uint16_t)mine;
            else if (mid) {
                const int cm = ld_color<true>(C + v);
                r = cm < (int)kRingGlobal ? (uint16_t)cm : kRingGlobal;
            }
            ring[v & (kRingIds - 1)] = r;
        }
        __syncwarp();
    }
    return suspect;
}

// Wait (bounded: timeout_ns, 10 s by default) until tile t of the ordered
// pass has been published.
__device__ void wait_tile_done(const KParams &p, long long t, int lane,
                               unsigned long long timeout_ns = kBarrierTimeoutNs)
{
    if (lane == 0) {
        const unsigned *f = reinterpret_cast<const unsigned *>(p.done + t);
        unsigned long long t0 = global_timer();
        unsigned polls = 0;
        while (ld_acquire_u32(f) == 0u) {
            __nanosleep(32);
            if (++polls > kBarrierMaxPolls || global_timer() - t0 > timeout_ns) {
                atomicOr(&p.st->error, GC_EW_TIMEOUT);
                break;
            }
        }
    }
    __syncwarp();
}

__device__ void publish_tile_done(const KParams &p, long long t, int lane)
{
    __syncwarp();
    if (lane == 0) {
        __threadfence();
        st_release_u32(reinterpret_cast<unsigned *>(p.done + t), 1u);
    }
}

// ------------------------------------------------------------------------
// one pass over a worklist
// ------------------------------------------------------------------------

struct PassIn {
    bool implicit;             // worklist is all of V (ids 0..n-1)
    const int32_t *wl;         // explicit tile worklist
    int32_t n;                 // its length (or n for implicit)
    const int32_t *hub;        // hub worklist
    int32_t hn;
    int32_t dmax;              // implicit passes skip vertices of higher degree
};

// Warp-aggregated append of the lanes with d set to the tile worklist of
// iteration `it` (one atomic per warp); their degrees feed the tail test.
// `stats`: count them as conflicts of their graph (batch statistics).
template <bool BATCH>
__device__ __forceinline__ void push_lanes(const KParams &p, bool d, int32_t v, int deg, int32_t g, int it,
                                           int lane, bool stats)
{
    DevState *st = p.st;
    if (d && (p.mode & GC_FF_KEEPERS)) d = claim_push(p, v, it);  // not queued yet by a lower neighbour
    const unsigned m = __ballot_sync(FULL_MASK, d);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long work = d ? (unsigned long long)deg : 0ull;
    for (int o = 16; o > 0; o >>= 1) work += __shfl_xor_sync(FULL_MASK, work, o);
    int ob = 0;
    if (lane == leader)
        ob = (int)(atomicAdd(&st->wl_packed[it & (kRing - 1)], ((unsigned long long)__popc(m) << kWorkBits) + work) >>
                   kWorkBits);
    ob = __shfl_sync(FULL_MASK, ob, leader);
    if (d) {
        const int o = ob + __popc(m & ((1u << lane) - 1u));
        if (o < p.n) __stcg(p.wl[it & 1] + o, v);
        else atomicOr(&st->error, GC_EW_OVERFLOW);
        if (stats) note_push_graph<BATCH>(p, g, it);
    }
}

// Round 0's suspects of one warp, collected in shared memory and appended to
// the worklist of iteration `it` kSusBuf at a time: one atomic per flush
// instead of one per chunk, off the chunk's critical path.
struct SusBuf {
    int n = 0;                       // entries held (warp-uniform)
    unsigned long long work = 0;     // their degree sum (warp-uniform)
};

__device__ __forceinline__ void sus_flush(const KParams &p, Shared &sh, SusBuf &b, int it, int lane, int wid)
{
    if (b.n == 0) return;
    DevState *st = p.st;
    int ob = 0;
    if (lane == 0)
        ob = (int)(atomicAdd(&st->wl_packed[it & (kRing - 1)], ((unsigned long long)b.n << kWorkBits) + b.work) >>
                   kWorkBits);
    ob = __shfl_sync(FULL_MASK, ob, 0);
    for (int i = lane; i < b.n; i += 32) {
        const int o = ob + i;
        if (o < p.n) __stcg(p.wl[it & 1] + o, sh.sus[wid][i]);
        else atomicOr(&st->error, GC_EW_OVERFLOW);
    }
    __syncwarp();
    b.n = 0;
    b.work = 0;
}

// Add the lanes with d set (keepers: those not queued yet) to the buffer.
__device__ __forceinline__ void sus_push(const KParams &p, Shared &sh, SusBuf &b, bool d, int32_t v, int deg, int it,
                                         int lane, int wid)
{
    if (d && (p.mode & GC_FF_KEEPERS)) d = claim_push(p, v, it);
    const unsigned m = __ballot_sync(FULL_MASK, d);
    if (!m) return;
    const int k = __popc(m);
    if (b.n + k > kSusBuf) sus_flush(p, sh, b, it, lane, wid);
    if (d) sh.sus[wid][b.n + __popc(m & ((1u << lane) - 1u))] = v;
    b.work += (unsigned long long)__reduce_add_sync(FULL_MASK, d ? (unsigned)deg : 0u);
    b.n += k;
    __syncwarp();
}

// One chunk of up to 32 worklist entries, one per lane (v = -1: none):
// thread-path lanes run `op` with adjacency entries from `ent`, the warp
// takes the mid-degree lanes one by one, and defective vertices are
// appended to the worklist of iteration `it` (warp-aggregated).
template <bool ASYNC, bool BATCH, class E>
__device__ __forceinline__ void chunk_ops(const KParams &p, Shared &sh, const E &ent, int op, int it,
                                          bool implicit, int dmax, int32_t v, int64_t beg, int64_t end,
                                          int32_t nbase, int32_t g, const int32_t *R, int32_t *W, bool push,
                                          long long &mb, int lane, int wid)
{
    const int deg = (int)(end - beg);
    if (implicit && deg > dmax) v = -1;  // coloured in another phase / stage
    const bool mid = v >= 0 && deg > p.t1;
    bool d = false;
    if (v >= 0 && !mid) d = vertex_thread<ASYNC, BATCH>(p, ent, op, v, beg, end, nbase, R, W, implicit, mb, it);
    unsigned mm = __ballot_sync(FULL_MASK, mid);
    while (mm) {
        const int src = __ffs(mm) - 1;
        mm &= mm - 1;
        const int32_t vv = __shfl_sync(FULL_MASK, v, src);
        const int64_t bb = __shfl_sync(FULL_MASK, beg, src);
        const int64_t ee = __shfl_sync(FULL_MASK, end, src);
        const int32_t nb = __shfl_sync(FULL_MASK, nbase, src);
        const bool dd =
            vertex_warp<ASYNC, BATCH>(p, op, vv, bb, ee, nb, R, W, implicit, mb, sh.warp_bm[wid], lane, it);
        if (lane == src) d = dd;
    }
    // A tentative pass over an explicit list (the degree tiers' round 0)
    // keeps every vertex it coloured for the first repair pass, as the hub
    // pass does: it did not track which ones read an uncoloured neighbour.
    if (push) {
        if (op == OP_TENT) push_lanes<BATCH>(p, v >= 0, v, deg, g, it, lane, false);
        else push_lanes<BATCH>(p, d, v, deg, g, it, lane, true);
    }
}

// A chunk of 32 consecutive ids in a pass over V: its uniform description
// lives in Shared::slot, each lane's row in a LaneRow register set.
struct LaneRow {
    int64_t beg;               // lane's row starts here (entry index)
    int32_t deg;               // and holds deg entries; -1: no vertex on this lane
    int32_t nbase, g;          // batch: graph offset and graph (0 otherwise)
};

constexpr unsigned long long kStageTimeoutNs = 2000000000ull;  // 2 s for one staged copy

// Load the lanes' row pointers of chunk [cb, min(cb+32, cend)) into `r`,
// record the chunk in Shared::slot[wid][slot] and start the 1-D TMA copy of
// its contiguous adjacency segment into seg[wid][slot].  The copy runs
// 16-byte aligned; a segment that does not fit, or whose aligned end would
// pass the last full 16 bytes of col_idx, is read from global memory instead.
template <bool BATCH>
__device__ __forceinline__ void stage_chunk(const KParams &p, Shared &sh, long long cb, long long cend, int tile,
                                            int kin, int slot, int lane, int wid, long long lim16, LaneRow &r)
{
    r.beg = 0;
    r.deg = -1;
    r.nbase = 0;
    r.g = 0;
    long long soff = -1;
    if (cb >= 0) {
        const long long vi = cb + lane;
        if (vi < cend) {
            int64_t end;
            row_of<BATCH>(p, (int32_t)vi, r.beg, end, r.nbase, r.g);
            r.deg = (int32_t)(end - r.beg);
        }
        const int last = (int)min(31ll, cend - 1 - cb);
        const long long s0 = __shfl_sync(FULL_MASK, (long long)r.beg, 0);
        const long long e0 = __shfl_sync(FULL_MASK, (long long)(r.beg + (r.deg > 0 ? r.deg : 0)), last);
        const long long a0 = (s0 * 4) & ~15ll;
        const long long a1 = (e0 * 4 + 15) & ~15ll;
        if (e0 > s0 && a1 - a0 <= (long long)kSegCap * 4 && a1 <= lim16) {
            soff = a0 >> 2;
            if (lane == 0) {
                fence_proxy_async_smem();  // earlier reads of this buffer precede the copy
                mbar_arrive_expect_tx(&sh.mbar[wid][slot], (uint32_t)(a1 - a0));
                bulk_copy_g2s(sh.seg[wid][slot], reinterpret_cast<const char *>(p.col_idx) + a0, (uint32_t)(a1 - a0),
                              &sh.mbar[wid][slot]);
            }
        }
    }
    if (lane == 0) {
        Shared::SlotInfo &si = sh.slot[wid][slot];
        si.cb = cb;
        si.cend = cend;
        si.soff = soff;
        si.tile = tile;
        si.kin = kin;
    }
    __syncwarp();
}

// Bounded wait for phase `par` of mbarrier `bar` (the completion of a
// staged copy): gives up after timeout_ns, setting GC_EW_TIMEOUT, and then
// waits once more, as long again, so that a copy still in flight does not
// land after the caller has moved on.  False on timeout.
__device__ __forceinline__ bool wait_mbar(const KParams &p, unsigned long long *bar, uint32_t par,
                                          unsigned long long timeout_ns)
{
    if (mbar_try_wait(bar, par)) return true;
    const unsigned long long t0 = global_timer();
    while (!mbar_try_wait(bar, par)) {
        if (global_timer() - t0 > timeout_ns) {
            atomicOr(&p.st->error, GC_EW_TIMEOUT);
            const unsigned long long t1 = global_timer();
            while (!mbar_try_wait(bar, par) && global_timer() - t1 <= timeout_ns) {
            }
            return false;
        }
    }
    return true;
}

// Wait for the copy into seg[wid][slot] (see wait_mbar).
__device__ __forceinline__ bool wait_stage(const KParams &p, Shared &sh, int slot, uint32_t &phase, int wid)
{
    const uint32_t par = (phase >> slot) & 1u;
    phase ^= 1u << slot;
    return wait_mbar(p, &sh.mbar[wid][slot], par, kStageTimeoutNs);
}

// Round 0 of an ordered graph (ids v0..v1-1): one warp colours it chunk by
// chunk in id order, each chunk's lanes in id order, which is exactly
// sequential First-Fit (Algorithm 1) on the graph apart from vertices
// coloured elsewhere (hubs, earlier tiers).  Chunk j+1's segment is staged
// while chunk j is worked on; recent colours are read from the warp's ring.
template <bool BATCH>
__device__ __noinline__ void seq_graph(const KParams &p, Shared &sh, int32_t g, long long v0, long long v1,
                                       int32_t *C, long long &mb, uint32_t &phase, int lane, int wid, int dmax,
                                       bool skip_higher, int it, bool push)
{
    const long long lim16 = (p.nnz * 4) & ~15ll;
    uint16_t *ring = sh.ring[wid];
    // The graph's row pointers and column indices (local ids + nbase).
    const int32_t *rp = p.row_ptr;
    int64_t eo = 0;
    int32_t nbase = 0;
    if (BATCH) {
        rp = p.row_ptr + (p.rp_off ? __ldg(p.rp_off + g) : v0 + g);
        eo = __ldg(p.edge_off + g);
        nbase = (int32_t)v0;
    }
    const long long ng = v1 - v0;
    // Row pointers are loaded two chunks ahead, the segment copy one ahead.
    auto load_rows = [&](long long k, int32_t &b, int32_t &e) {
        const long long lv = k * 32 + lane;
        b = e = 0;
        if (k >= 0 && lv < ng) {
            b = __ldg(rp + lv);
            e = __ldg(rp + lv + 1);
        }
    };
    auto issue = [&](long long k, int slot, int32_t b, int32_t e) -> long long {
        // start the copy of chunk k's segment; returns soff (-1: not staged)
        long long soff = -1;
        if (k * 32 < ng) {
            const int last = (int)min(31ll, ng - 1 - k * 32);
            const long long s0 = eo + __shfl_sync(FULL_MASK, b, 0);
            const long long e0 = eo + __shfl_sync(FULL_MASK, e, last);
            const long long a0 = (s0 * 4) & ~15ll, a1 = (e0 * 4 + 15) & ~15ll;
            if (e0 > s0 && a1 - a0 <= (long long)kSegCap * 4 && a1 <= lim16) {
                soff = a0 >> 2;
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&sh.mbar[wid][slot], (uint32_t)(a1 - a0));
                    bulk_copy_g2s(sh.seg[wid][slot], reinterpret_cast<const char *>(p.col_idx) + a0,
                                  (uint32_t)(a1 - a0), &sh.mbar[wid][slot]);
                }
            }
        }
        return soff;
    };
    const long long nck = (ng + 31) / 32;
    int32_t b0, e0, b1, e1, b2, e2;
    load_rows(0, b0, e0);
    load_rows(1, b1, e1);
    int slot = 0;
    long long soff0 = nck > 0 ? issue(0, 0, b0, e0) : -1;
    for (long long k = 0; k < nck; ++k) {
        load_rows(k + 2, b2, e2);
        const long long soff1 = k + 1 < nck ? issue(k + 1, slot ^ 1, b1, e1) : -1;
        bool staged = soff0 >= 0;
        if (staged && !wait_stage(p, sh, slot, phase, wid)) staged = false;
        const long long cb = v0 + k * 32;
        const int32_t v = k * 32 + lane < ng ? (int32_t)(cb + lane) : -1;
        const int64_t beg = eo + b0, end = eo + e0;
        bool sus;
        if (staged)
            sus = chunk_tent_ordered<StagedEnts, true>(p, StagedEnts{sh.seg[wid][slot], soff0}, cb, v, beg, end,
                                                       nbase, C, mb, sh.warp_bm[wid], lane, dmax, ring, v0,
                                                       skip_higher);
        else
            sus = chunk_tent_ordered<GlobalEnts, true>(p, GlobalEnts{p.col_idx}, cb, v, beg, end, nbase, C, mb,
                                                       sh.warp_bm[wid], lane, dmax, ring, v0, skip_higher);
        if (push) push_lanes<BATCH>(p, sus, v, e0 - b0, g, it, lane, false);
        __syncwarp();
        b0 = b1;
        e0 = e1;
        b1 = b2;
        e1 = e2;
        soff0 = soff1;
        slot ^= 1;
    }
}

// Chunk vc of a pass: direct (ids 32*vc.., up to n) or, in the round-0
// tentative pass, numbered over the graphs that are not ordered (uofs holds
// their prefix sums of chunk counts).
// ------------------------------------------------------------------------
// ordered round 0 by a group of warps (pipelined id order)
// ------------------------------------------------------------------------

constexpr unsigned long long kPipeTimeoutNs = 2000000000ull;  // 2 s per chunk

// One chunk of a graph that a group of warps colours in id order: a lane
// is coloured once every lower neighbour is (those outside the chunk are
// polled in memory, where other warps of the group write them; those inside
// are resolved here), from those colours only.  Nothing above a vertex is
// read, so the result is exactly sequential First-Fit (Algorithm 1), while
// the chunks of the group's warps overlap wherever they do not depend on
// each other (along a mesh, a wavefront over its rows).  Lanes whose lower
// neighbours are all coloured go first, in id order; the others wait.
// Returns false if a wait timed out (error word set).
template <class E>
__device__ bool chunk_pipe(const KParams &p, const E &ent, int32_t cb, int32_t v, int64_t beg, int deg,
                           int32_t nbase, int32_t *C, long long &mb, int lane,
                           unsigned long long timeout_ns = kPipeTimeoutNs)
{
    const bool act = v >= 0;
    unsigned done = __ballot_sync(FULL_MASK, !act);
    int mine = 0;
    unsigned long long t0 = 0;
    unsigned backoff = 32;
    while (done != FULL_MASK) {
        const bool todo = !((done >> lane) & 1u);
        unsigned long long ext = 0;
        unsigned low = 0;
        bool pend = false;
        int nlo = 0;
        if (todo) {
            const auto row = ent.row(beg);
            for (int i = 0; i < deg; i += kUnroll) {
                int u[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    u[q] = (i + q < deg) ? nbase + row[i + q] : -1;
                    if (u[q] > v) u[q] = -1;  // higher neighbours are not looked at
                }
                int c[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    const uint32_t d = (uint32_t)(u[q] - cb);
                    const bool inside = u[q] >= 0 && d < 32u;
                    if (inside) low |= 1u << d;
                    c[q] = (u[q] >= 0 && !inside) ? ld_color<true>(C + u[q]) : 0;
                    if (u[q] >= 0 && !inside && c[q] == 0) pend = true;
                    nlo += u[q] >= 0;
                }
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    const unsigned b = (unsigned)(c[q] - 1);
                    if (b < 64u) ext |= 1ull << b;
                }
                if (u[kUnroll - 1] < 0) break;  // row ended, or passed v (rows are sorted)
            }
        }
        // colours of lower lanes finished earlier in this call
        const unsigned need = __reduce_or_sync(FULL_MASK, todo ? (low & done) : 0u);
        for (unsigned m = need; m; m &= m - 1) {
            const int j = __ffs(m) - 1;
            const int cj = __shfl_sync(FULL_MASK, mine, j);
            if (todo && ((low >> j) & 1u)) ext |= 1ull << (cj - 1);
        }
        low &= ~done;
        // the lanes that can go now: no uncoloured neighbour outside, and every
        // lower lane they depend on goes too
        unsigned S = __ballot_sync(FULL_MASK, todo && !pend);
        for (;;) {
            const unsigned S2 = __ballot_sync(FULL_MASK, ((S >> lane) & 1u) && (low & ~S) == 0u);
            if (S2 == S) break;
            S = S2;
        }
        if (S) {
            const bool in = (S >> lane) & 1u;
            const int m = resolve_in_order(ext, in ? low : 0u, in, lane);
            if (in) {
                mine = m;
                st_color<true>(C + v, mine);
                mb += 8 + 8ll * nlo + 4;
            }
            done |= S;
            continue;
        }
        // nothing can go: the group's other warps still colour lower ids
        if (t0 == 0) {
            t0 = global_timer();
        } else if (global_timer() - t0 > timeout_ns) {
            if (lane == 0) atomicOr(&p.st->error, GC_EW_TIMEOUT);
            return false;
        }
        __nanosleep(backoff);
        backoff = min(backoff * 2u, 1024u);
    }
    return true;
}

// Warp j of a group of K colours chunks j, j+K, j+2K, ... of graph g (ids
// v0..v1-1) with chunk_pipe, staging each chunk's adjacency segment one
// chunk ahead.  Only graphs without hubs and without vertices of degree
// above kT1Max are grouped: every lane colours its vertex alone, whatever t1.
template <bool BATCH>
__device__ __noinline__ void pipe_graph(const KParams &p, Shared &sh, int32_t g, long long v0, long long v1, int j,
                                        int K, int32_t *C, long long &mb, uint32_t &phase, int lane, int wid)
{
    const long long lim16 = (p.nnz * 4) & ~15ll;
    const int32_t *rp = p.row_ptr;
    int64_t eo = 0;
    int32_t nbase = 0;
    if (BATCH) {
        rp = p.row_ptr + (p.rp_off ? __ldg(p.rp_off + g) : v0 + g);
        eo = __ldg(p.edge_off + g);
        nbase = (int32_t)v0;
    }
    const long long ng = v1 - v0;
    const long long nck = (ng + 31) / 32;
    auto load_rows = [&](long long k, int32_t &b, int32_t &e) {
        const long long lv = k * 32 + lane;
        b = e = 0;
        if (k < nck && lv < ng) {
            b = __ldg(rp + lv);
            e = __ldg(rp + lv + 1);
        }
    };
    auto issue = [&](long long k, int slot, int32_t b, int32_t e) -> long long {
        long long soff = -1;
        if (k < nck) {
            const int last = (int)min(31ll, ng - 1 - k * 32);
            const long long s0 = eo + __shfl_sync(FULL_MASK, b, 0);
            const long long e0 = eo + __shfl_sync(FULL_MASK, e, last);
            const long long a0 = (s0 * 4) & ~15ll, a1 = (e0 * 4 + 15) & ~15ll;
            if (e0 > s0 && a1 - a0 <= (long long)kSegCap * 4 && a1 <= lim16) {
                soff = a0 >> 2;
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&sh.mbar[wid][slot], (uint32_t)(a1 - a0));
                    bulk_copy_g2s(sh.seg[wid][slot], reinterpret_cast<const char *>(p.col_idx) + a0,
                                  (uint32_t)(a1 - a0), &sh.mbar[wid][slot]);
                }
            }
        }
        return soff;
    };
    int32_t b0, e0, b1, e1;
    load_rows(j, b0, e0);
    int slot = 0;
    long long soff0 = issue(j, 0, b0, e0);
    for (long long k = j; k < nck; k += K) {
        load_rows(k + K, b1, e1);
        const long long soff1 = issue(k + K, slot ^ 1, b1, e1);
        bool staged = soff0 >= 0;
        bool ok = true;
        if (staged && !wait_stage(p, sh, slot, phase, wid)) staged = ok = false;
        const int32_t cb = (int32_t)(v0 + k * 32);
        const int32_t v = k * 32 + lane < ng ? cb + lane : -1;
        if (ok) {
            if (staged)
                ok = chunk_pipe(p, StagedEnts{sh.seg[wid][slot], soff0}, cb, v, eo + b0, e0 - b0, nbase, C, mb,
                                lane);
            else
                ok = chunk_pipe(p, GlobalEnts{p.col_idx}, cb, v, eo + b0, e0 - b0, nbase, C, mb, lane);
        }
        __syncwarp();
        if (!ok) {  // let the copy in flight land before leaving
            if (soff1 >= 0) wait_stage(p, sh, slot ^ 1, phase, wid);
            return;
        }
        b0 = b1;
        e0 = e1;
        soff0 = soff1;
        slot ^= 1;
    }
}

template <bool BATCH>
__device__ __forceinline__ void chunk_of(const KParams &p, long long vc, bool virt, long long n, long long &cb,
                                         long long &cend)
{
    if (!virt) {
        cb = vc * 32;
        cend = n;
        return;
    }
    if (!BATCH) {
        cb = vc * 32;
        cend = p.n;
        return;
    }
    int lo = 0, hi = p.G - 1;  // largest g with uofs[g] <= vc
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldcg(p.uofs + mid) <= vc) lo = mid;
        else hi = mid - 1;
    }
    cb = __ldg(p.vtx_off + lo) + (vc - __ldcg(p.uofs + lo)) * 32;
    cend = __ldg(p.vtx_off + lo + 1);
}

// Pass over all of V (implicit worklist): each warp walks the chunks of the
// tiles it claims in id order, staging chunk j+1 while it works on chunk j.
// The asynchronous tentative pass resolves lanes in id order and keeps at
// most `window` tiles in flight (window <= 0: no limit).
template <bool ASYNC, bool BATCH, bool WIDE>
__device__ __forceinline__ void implicit_staged(const KParams &p, Shared &sh, int op, int q, int it, const PassIn &in,
                                const int32_t *R, int32_t *W, bool push, long long &mb, int window,
                                uint32_t &phase)
{
    DevState *st = p.st;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    int *claim = &st->pass_tile[q & (kRing - 1)];
    const long long n = in.n;
    const int cpt = p.tile >> 5;
    const bool ordered = ASYNC && op == OP_TENT;
    const long long lim16 = (p.nnz * 4) & ~15ll;

    if (ordered) {
        // Phase A: ordered graphs.  Warp w < n_pitems belongs to a group
        // colouring one graph together (all of a group's warps are resident
        // and start at once); then one warp per remaining ordered graph.
        const int gw = blockIdx.x * kWarps + wid;
        if (gw < ld_volatile(&st->n_pitems)) {
            const long long item = __ldcg(p.pitems + gw);
            const int32_t g = (int32_t)(item >> 20);
            const int j = (int)((item >> 10) & 1023), K = (int)(item & 1023) + 1;
            const long long v0 = BATCH ? __ldg(p.vtx_off + g) : 0;
            const long long v1 = BATCH ? __ldg(p.vtx_off + g + 1) : p.n;
            pipe_graph<BATCH>(p, sh, g, v0, v1, j, K, W, mb, phase, lane, wid);
        }
        const int nord = ld_volatile(&st->n_ordered);
        const bool tiered = (p.mode & GC_TIERS) != 0;
        for (;;) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&st->seq_claim, 1);
            k = __shfl_sync(FULL_MASK, k, 0);
            if (k >= nord) break;
            const int g = __ldcg(p.olist + k);
            const long long v0 = BATCH ? __ldg(p.vtx_off + g) : 0;
            const long long v1 = BATCH ? __ldg(p.vtx_off + g + 1) : p.n;
            const bool skip_higher = !tiered && __ldcg(&p.gstat[g].hubs) == 0;
            seq_graph<BATCH>(p, sh, g, v0, v1, W, mb, phase, lane, wid, in.dmax, skip_higher, it, push);
        }
    }
    // Phase B: chunks claimed tile by tile (the unordered graphs only, in the
    // round-0 tentative pass).
    const long long nchunks = ordered ? *(volatile long long *)&st->n_uchunks : (n + 31) / 32;
    const long long ntiles = (nchunks + cpt - 1) / cpt;
    // One graph, tiles claimed in id order, lower ids keep their colour, no
    // vertex coloured before the tiles (hubs, earlier tiers): every id past
    // the claimed tiles is uncoloured, and as a higher neighbour its colour
    // is not needed for the suspect test either.
    const bool skip_unclaimed = ordered && !BATCH && p.tie == TIE_LOWER &&
                                !(p.mode & (GC_TIERS | GC_FF_KEEPERS)) && window <= 0 &&
                                __ldcg(&p.gstat[0].hubs) == 0u;

    // One graph with no hub and no vertex of degree above kT1Max, lower ids
    // keep, no keepers: its round-0 chunks take the lean colouring whenever
    // all their lanes are on the thread path.  (Graphs with wider rows keep
    // the one general form: alternating between the two made R-MAT's round
    // 0 slower.)  Only in the build for at most two blocks per SM (WIDE: 128
    // registers); in the three-block build, at 80 registers, the extra code
    // made every graph's round 0 slower through more spilling.
    const bool lean_graph = WIDE && !BATCH && ordered && p.tie == TIE_LOWER && !(p.mode & GC_FF_KEEPERS) &&
                            __ldcg(&p.gstat[0].hubs) == 0u && __ldcg(&p.gstat[0].wide) == 0u;
    int t = 0;
    if (lane == 0) t = atomicAdd(claim, 1);
    t = __shfl_sync(FULL_MASK, t, 0);
    LaneRow cur, nxt;
    SusBuf sbuf;
    int slot = 0;
    // The suspects of a lean chunk wait one chunk: by then the tie-side
    // neighbours each read as uncoloured (at most two are kept) have almost
    // always been coloured, and a round-0 colour is final for the round, so
    // a suspect whose such neighbours all hold colours other than its own
    // has no clash on its tie side and is dropped from the first repair.
    bool pend = false;  // warp-uniform: the previous chunk's suspects wait
    bool psus = false;
    int32_t pv = -1;
    int pdeg = 0;
    SusHint ph{0, 0, 0, 0};
    auto push_pending = [&]() {
        bool still = psus;
        if (psus && ph.zc <= 2) {
            const int c0 = ld_color<true>(W + ph.u0);
            const int c1 = ph.zc == 2 ? ld_color<true>(W + ph.u1) : -1;
            mb += 4ll * ph.zc;
            still = c0 == 0 || c0 == ph.cv || (ph.zc == 2 && (c1 == 0 || c1 == ph.cv));
        }
        sus_push(p, sh, sbuf, still, pv, pdeg, it, lane, wid);
        pend = false;
    };
    {
        long long cb = -1, cend = 0;
        if (t < ntiles) chunk_of<BATCH>(p, (long long)t * cpt, ordered, n, cb, cend);
        stage_chunk<BATCH>(p, sh, cb, cend, t, 0, slot, lane, wid, lim16, cur);
    }
    for (;;) {
        const long long cb = sh.slot[wid][slot].cb;
        if (cb < 0) {
            if (ordered && push) {
                if (pend) push_pending();
                sus_flush(p, sh, sbuf, it, lane, wid);
            }
            break;
        }
        const long long soff = sh.slot[wid][slot].soff;
        const int tile = sh.slot[wid][slot].tile;
        const int kin = sh.slot[wid][slot].kin;
        int ntile = tile, nkin = kin + 1;
        long long vc = (long long)ntile * cpt + nkin;
        const bool last_of_tile = nkin >= cpt || vc >= nchunks;
        if (last_of_tile) {
            int t2 = 0;
            if (lane == 0) t2 = atomicAdd(claim, 1);
            ntile = __shfl_sync(FULL_MASK, t2, 0);
            nkin = 0;
            vc = (long long)ntile * cpt;
        }
        {
            long long ncb = -1, ncend = 0;
            if (vc < nchunks) chunk_of<BATCH>(p, vc, ordered, n, ncb, ncend);
            stage_chunk<BATCH>(p, sh, ncb, ncend, ntile, nkin, slot ^ 1, lane, wid, lim16, nxt);
        }

        bool staged = soff >= 0;
        if (staged && !wait_stage(p, sh, slot, phase, wid)) staged = false;
        if (ordered && window > 0 && kin == 0 && tile >= window) wait_tile_done(p, tile - window, lane);
        const int32_t v = cur.deg >= 0 ? (int32_t)(cb + lane) : -1;
        const int64_t end = cur.beg + (cur.deg > 0 ? cur.deg : 0);
        int32_t unclaimed = INT32_MAX;
        if (skip_unclaimed) {
            // the tiles past this warp's latest claim were unclaimed when it
            // made that claim
            const long long first_free = ((long long)ntile + 1) * cpt * 32;
            if (first_free < n) unclaimed = (int32_t)first_free;
        }
        bool sus = false;
        bool lean = false;
        SusHint hint{0, 0, 0, 0};
        if (staged) {
            const StagedEnts ent{sh.seg[wid][slot], soff};
            // every lane on the thread path (checked per chunk in a graph
            // of uniform low degree)
            lean = lean_graph && !__any_sync(FULL_MASK, v >= 0 && (cur.deg > in.dmax || cur.deg > p.t1));
            if (lean)
                sus = chunk_tent_ordered<StagedEnts, false, WIDE && !BATCH>(p, ent, cb, v, cur.beg, end, cur.nbase, W, mb,
                                                                    sh.warp_bm[wid], lane, in.dmax, nullptr, 0, false,
                                                                    unclaimed, &hint);
            else if (ordered)
                sus = chunk_tent_ordered<StagedEnts, false>(p, ent, cb, v, cur.beg, end, cur.nbase, W, mb,
                                                            sh.warp_bm[wid], lane, in.dmax, nullptr, 0, false,
                                                            unclaimed);
            else
                chunk_ops<ASYNC, BATCH>(p, sh, ent, op, it, true, in.dmax, v, cur.beg, end, cur.nbase, cur.g, R, W,
                                        push, mb, lane, wid);
        } else {
            const GlobalEnts ent{p.col_idx};
            if (ordered)
                sus = chunk_tent_ordered<GlobalEnts, false>(p, ent, cb, v, cur.beg, end, cur.nbase, W, mb,
                                                            sh.warp_bm[wid], lane, in.dmax, nullptr, 0, false,
                                                            unclaimed);
            else
                chunk_ops<ASYNC, BATCH>(p, sh, ent, op, it, true, in.dmax, v, cur.beg, end, cur.nbase, cur.g, R, W,
                                        push, mb, lane, wid);
        }
        // Round 0 with push: the suspects form the first repair worklist.
        if (ordered && push) {
            if (pend) push_pending();
            if (WIDE && lean && p.r0mask) {
                pend = true;
                psus = sus;
                pv = v;
                pdeg = cur.deg;
                ph = hint;
            } else {
                sus_push(p, sh, sbuf, sus, v, cur.deg, it, lane, wid);
            }
        }
        if (ordered && window > 0 && last_of_tile) publish_tile_done(p, tile, lane);
        __syncwarp();  // every lane is done with seg[slot] before it is refilled
        cur = nxt;
        slot ^= 1;
    }
}

// Runs `op` over the hubs (block per vertex) and then the tiles (warp per
// 32 entries) of `in`.  Vertices found defective are appended to the
// worklists of iteration `it` when `push` is set.
// The first hub of block b and the first tile of warp w are fixed (b and w;
// nbl blocks take part), the rest are claimed, so a pass whose work fits
// the grid makes no claim at all.
template <bool ASYNC, bool BATCH, bool WIDE>
__device__ void run_pass(const KParams &p, Shared &sh, int op, int q, int it, const PassIn &in,
                         const int32_t *R, int32_t *W, bool push, long long &mb, uint32_t &phase, unsigned nbl,
                         int window = -1)
{
    DevState *st = p.st;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->pass_tile[(q + 2) & (kRing - 1)] = 0;
        st->pass_hub[(q + 2) & (kRing - 1)] = 0;
    }
    int *out_hub = p.hub[it & 1];
    const bool keep = ASYNC && (p.mode & GC_FF_KEEPERS);

    // hubs: one block per vertex
    if (in.hn > 0) {
        int *claim = &st->pass_hub[q & (kRing - 1)];
        for (int h = (int)blockIdx.x;;) {
            if (h >= in.hn) break;
            const int32_t v = __ldcg(in.hub + h);
            int64_t beg, end;
            int32_t nbase, g;
            row_of<BATCH>(p, v, beg, end, nbase, g);
            // a core was coloured before round 0 and never changes
            if (!(p.core_deg > 0 && end - beg > p.core_deg && __ldcg(&p.gstat[g].core_on))) {
                const bool d =
                    vertex_block<ASYNC, BATCH>(p, op, v, beg, end, nbase, R, W, in.implicit, mb, sh, it) ||
                    op == OP_TENT;  // round 0: hubs are kept for the first repair pass
                if (push && d && threadIdx.x == 0 && (!keep || claim_push(p, v, it))) {
                    atomicAdd(&st->wl_packed[it & (kRing - 1)], (unsigned long long)(end - beg));
                    const int idx = atomicAdd(&st->hub_count[it & (kRing - 1)], 1);
                    if (idx < p.hub_cap) __stcg(out_hub + idx, v);
                    else atomicOr(&st->error, GC_EW_OVERFLOW);
                    if (op != OP_TENT) note_push_graph<BATCH>(p, g, it);
                }
            }
            if (in.hn <= (int)nbl) break;  // every hub had a block of its own
            __syncthreads();
            if (threadIdx.x == 0) sh.claim = (int)nbl + atomicAdd(claim, 1);
            __syncthreads();
            h = sh.claim;
        }
    }

    // tiles: one warp per group of `tile` consecutive worklist entries
    if (in.implicit) {
        implicit_staged<ASYNC, BATCH, WIDE>(p, sh, op, q, it, in, R, W, push, mb, window, phase);
        return;
    }
    int *claim = &st->pass_tile[q & (kRing - 1)];
    const long long nwarps = (long long)nbl * kWarps;
    const long long ntiles = ((long long)in.n + p.tile - 1) / p.tile;
    for (long long t = (long long)blockIdx.x * kWarps + wid;;) {
        const long long base = t * p.tile;
        if (base >= in.n) break;
        for (int j = 0; j < p.tile && base + j < in.n; j += 32) {
            const long long idx = base + j + lane;
            int32_t v = -1;
            if (idx < in.n) v = __ldcg(in.wl + idx);
            int64_t beg = 0, end = 0;
            int32_t nbase = 0, g = 0;
            if (v >= 0) row_of<BATCH>(p, v, beg, end, nbase, g);
            chunk_ops<ASYNC, BATCH>(p, sh, GlobalEnts{p.col_idx}, op, it, false, in.dmax, v, beg, end, nbase, g, R,
                                    W, push, mb, lane, wid);
        }
        if (ntiles <= nwarps) break;  // every tile had a warp of its own
        int c = 0;
        if (lane == 0) c = atomicAdd(claim, 1);
        t = nwarps + __shfl_sync(FULL_MASK, c, 0);
    }
}

// Sum of x over the block (every thread gets it).  Uses sh.hub_bm as
// scratch; all threads must call it.
__device__ long long block_sum(long long x, Shared &sh)
{
    long long *red = reinterpret_cast<long long *>(sh.hub_bm);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    __syncthreads();
    if (lane == 0) red[wid] = x;
    __syncthreads();
    long long t = 0;
    for (int w = 0; w < kWarps; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Block 0: decide which graphs are coloured in id order in round 0 of the
// asynchronous mode (window 1: every graph; 0: graphs of at most
// kOrderedSmall vertices, graphs whose sampled lower neighbours mostly lie
// within kNearIds ids, and graphs of at most kOrderedGroup vertices without
// hubs or vertices of degree above kT1Max; else none), and how: a graph without hubs or vertices
// of degree above kT1Max whose chunks exceed the per-warp share of all ordered
// chunks gets a group of warps (pipe_graph; the groups together take at
// most three quarters of the grid's warps), any other ordered graph one
// warp.  Also numbers the chunks of the graphs that are not ordered
// (prefix sums in uofs).
template <bool BATCH>
__device__ __noinline__ void plan_ordering(const KParams &p, Shared &sh)
{
    DevState *st = p.st;
    const int window = p.window;
    const bool tiers = (p.mode & GC_TIERS) != 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // the warps of the rounds kernel, which run the plan
    const long long warps = (long long)(p.round_blocks > 0 ? p.round_blocks : (int)gridDim.x) * kWarps;
    const long long budget = min(warps, (long long)p.pitems_cap) * 7 / 8;
    auto graph_n = [&](int g) -> long long {
        return BATCH ? __ldg(p.vtx_off + g + 1) - __ldg(p.vtx_off + g) : (long long)p.n;
    };
    auto groupable = [&](int g) -> bool {
        return !tiers && p.gstat[g].hubs == 0 && p.gstat[g].wide == 0;
    };
    auto is_ordered = [&](int g, long long ng) -> bool {
        const GraphStat &gs = p.gstat[g];
        // Small graphs are ordered too: coloured all at once they would be
        // coloured almost simultaneously, whatever their numbering.  So are
        // graphs a warp group can take (up to kOrderedGroup vertices).
        return ng > 0 && (window == 1 || (window == 0 && (ng <= kOrderedSmall ||
                                                          (gs.all_lower > 0 && 2 * gs.near_lower >= gs.all_lower) ||
                                                          (ng <= kOrderedGroup && groupable(g)))));
    };
    if (p.G == 1) {
        // One graph: the same decisions as below, by one thread with rolled
        // loops (the general form's per-graph loops over the candidates are
        // unrolled: long straight-line code that a single graph does not
        // need to fetch).
        if (threadIdx.x == 0) {
            const long long ng = graph_n(0);
            const bool ord = is_ordered(0, ng);
            const long long c = (ng + 31) / 32;
            int K = 1;
            if (ord && groupable(0)) {
                long long cand = max((c + warps - 1) / max(warps, 1ll), (long long)kPipeMinChunks);
                long long target = cand;
                for (int i = 0; i < kTargetSteps; ++i) {
                    target = cand;  // the last candidate if none fits
                    const bool grp = c > cand;
                    const long long wg = grp ? min((c + cand - 1) / cand, (long long)kPipeMaxK) : 0;
                    if (wg <= budget && (grp ? 0 : c) <= cand * (warps - wg)) break;
                    cand += cand / 10 + 1;
                }
                if (c > target) K = (int)min((c + target - 1) / target, (long long)kPipeMaxK);
            }
            p.gstat[0].ordered = ord;
            p.gstat[0].group = K > 1 ? K : 0;
            const long long uch = ord ? 0 : c;
            if (ord && K == 1) p.olist[0] = 0;
            st->n_ordered = (ord && K == 1) ? 1 : 0;
            st->n_pitems = (ord && K > 1) ? K : 0;
            p.uofs[0] = 0;
            p.uofs[1] = uch;
            st->n_uchunks = uch;
            sh.claim = (ord && K > 1) ? K : 0;
        }
        __syncthreads();
        const int K = sh.claim;
        for (int j = threadIdx.x; j < K; j += kBlock) p.pitems[j] = ((long long)j << 10) | (long long)(K - 1);
        __syncthreads();
        return;
    }
    // Ordered chunks in all.
    long long T = 0;
    for (int g0 = 0; g0 < p.G; g0 += kBlock) {
        const int g = g0 + threadIdx.x;
        long long c = 0;
        if (g < p.G) {
            const long long ng = graph_n(g);
            if (is_ordered(g, ng)) c = (ng + 31) / 32;
        }
        T += block_sum(c, sh);
    }
    // The chunks per grouped warp, `target`: the smallest of kTargetSteps
    // candidates (from the even share of all ordered chunks upwards, x1.1
    // each) at which the groups fit the budget and the graphs left to single
    // warps fit on the remaining warps at `target` chunks each.
    long long cand[kTargetSteps];
    cand[0] = max((T + warps - 1) / max(warps, 1ll), (long long)kPipeMinChunks);
    for (int i = 1; i < kTargetSteps; ++i) cand[i] = cand[i - 1] + cand[i - 1] / 10 + 1;
    long long *acc = reinterpret_cast<long long *>(sh.hub_bm);  // [2 * kTargetSteps], block-local scratch
    for (int i = threadIdx.x; i < 2 * kTargetSteps; i += kBlock) acc[i] = 0;
    __syncthreads();
    {
        long long wg[kTargetSteps], single[kTargetSteps];
#pragma unroll
        for (int i = 0; i < kTargetSteps; ++i) wg[i] = single[i] = 0;
        for (int g = threadIdx.x; g < p.G; g += kBlock) {
            const long long ng = graph_n(g);
            if (!is_ordered(g, ng)) continue;
            const long long c = (ng + 31) / 32;
            const bool gr = groupable(g);
#pragma unroll
            for (int i = 0; i < kTargetSteps; ++i) {
                if (gr && c > cand[i]) wg[i] += min((c + cand[i] - 1) / cand[i], (long long)kPipeMaxK);
                else single[i] += c;
            }
        }
#pragma unroll
        for (int i = 0; i < kTargetSteps; ++i) {
            if (wg[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&acc[2 * i]), (unsigned long long)wg[i]);
            if (single[i]) atomicAdd(reinterpret_cast<unsigned long long *>(&acc[2 * i + 1]), (unsigned long long)single[i]);
        }
    }
    __syncthreads();
    long long target = cand[kTargetSteps - 1];
    for (int i = 0; i < kTargetSteps; ++i) {
        const long long wgi = acc[2 * i], si = acc[2 * i + 1];
        if (wgi <= budget && si <= cand[i] * (warps - wgi)) {
            target = cand[i];
            break;
        }
    }
    __syncthreads();
    auto group_of = [&](long long chunks) -> int {
        return chunks > target ? (int)min((chunks + target - 1) / target, (long long)kPipeMaxK) : 1;
    };
    // Graphs left to single warps are listed largest first (by powers of two
    // of their chunk counts), so that the longest start first.
    int *bucket = reinterpret_cast<int *>(sh.hub_bm);  // [64]: counts, then fill positions
    for (int i = threadIdx.x; i < 64; i += kBlock) bucket[i] = 0;
    __syncthreads();
    auto bucket_of = [&](long long chunks) -> int { return 63 - __clzll((unsigned long long)chunks | 1ull); };
    for (int g = threadIdx.x; g < p.G; g += kBlock) {
        const long long ng = graph_n(g);
        if (is_ordered(g, ng) && (!groupable(g) || group_of((ng + 31) / 32) == 1))
            atomicAdd(&bucket[bucket_of((ng + 31) / 32)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 31; b >= 0; --b) {  // largest first
            const int c = bucket[b];
            bucket[32 + b] = run;
            run += c;
        }
        st->n_ordered = run;
    }
    __syncthreads();
    long long carry = 0;
    long long *warp_tot = reinterpret_cast<long long *>(sh.hub_bm) + 32;  // block-local scratch after bucket[]
    for (int g0 = 0; g0 < p.G; g0 += kBlock) {
        const int g = g0 + threadIdx.x;
        long long chunks = 0;
        if (g < p.G) {
            const long long ng = graph_n(g);
            const bool ord = is_ordered(g, ng);
            int K = 1;
            if (ord && groupable(g)) K = group_of((ng + 31) / 32);
            p.gstat[g].ordered = ord;
            p.gstat[g].group = K > 1 ? K : 0;
            if (ord && K > 1) {
                const int base = atomicAdd(&st->n_pitems, K);
                for (int j = 0; j < K; ++j)
                    p.pitems[base + j] = ((long long)g << 20) | ((long long)j << 10) | (long long)(K - 1);
            } else if (ord) {
                p.olist[atomicAdd(&bucket[32 + bucket_of((ng + 31) / 32)], 1)] = g;
            } else {
                chunks = (ng + 31) / 32;
            }
        }
        // block-wide exclusive scan of chunks
        long long x = chunks;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(FULL_MASK, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        long long before = carry;
        for (int w = 0; w < wid; ++w) before += warp_tot[w];
        if (g < p.G) p.uofs[g] = before + x - chunks;
        long long tile_total = 0;
        for (int w = 0; w < kWarps; ++w) tile_total += warp_tot[w];
        __syncthreads();
        carry += tile_total;
    }
    if (threadIdx.x == 0) {
        p.uofs[p.G] = carry;
        st->n_uchunks = carry;
    }
}


// ------------------------------------------------------------------------
// the core: the highest-degree vertices of one graph, coloured first
// ------------------------------------------------------------------------
//
// In the asynchronous mode a graph with very high-degree vertices (R-MAT's
// hubs, which form a dense core) gets them coloured before round 0 of the
// rest, one vertex at a time in decreasing degree (ties: increasing id), by
// First-Fit among themselves: the interleaving of Algorithm 3's round 0 in
// which the threads holding the core run first and one after the other.
// They then hold final colours that no later round changes (every other
// vertex avoids them), so the repair rounds never rescan a hub row, and the
// colour count stays close to sequential First-Fit (the core decides it).
//
// Every graph of a launch has its own core (a batch's R-MAT requests as
// much as a single R-MAT graph).  Data: p.mid_all lists the cores, graph
// after graph (GraphStat::core_off), each in rank order after core_sort, and
// p.hub[0] the graph of each entry; while the cores are built, a core
// vertex's colour slot holds -(rank + 1); p.wl[1] holds each core's adjacency
// as a bit matrix from word GraphStat::core_bofs on, word w of rank r at
// w * Hp + r, Hp = H rounded up to a multiple of 32 (column-major: the 32
// ranks of a colouring batch are one coalesced read); p.hub[1][i] is the
// first adjacency-build task of entry i (one entry more at the end).

// Exclusive prefix sum over the block of one value per thread (all threads
// call it); `scratch` holds kWarps ints of shared memory.
__device__ __forceinline__ int block_exclusive_scan(int x, int *scratch, int &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) scratch[wid] = incl;
    __syncthreads();
    int before = 0;
    total = 0;
    for (int w = 0; w < kWarps; ++w) {
        const int t = scratch[w];
        if (w < wid) before += t;
        total += t;
    }
    __syncthreads();
    return before + incl - x;
}

// One block: sort a core (list, H entries) by (degree descending, id
// ascending), write it back in rank order, mark the colour slots with the
// ranks and store each entry's number of build tasks in tasks[].
template <bool BATCH>
__device__ __noinline__ void core_sort(const KParams &p, Shared &sh, int32_t *list, int H, int32_t *tasks)
{
    unsigned long long *key = reinterpret_cast<unsigned long long *>(&sh.seg[0][0][0]);  // kCoreMax keys
    static_assert(sizeof(sh.seg) >= kCoreMax * sizeof(unsigned long long), "core keys fit the staging area");
    int P = 1;
    while (P < H) P <<= 1;
    for (int i = threadIdx.x; i < P; i += kBlock) {
        unsigned long long k = ~0ull;
        if (i < H) {
            const int32_t v = __ldcg(list + i);
            int64_t beg, end;
            int32_t nbase, g;
            row_of<BATCH>(p, v, beg, end, nbase, g);
            k = ((unsigned long long)(~(uint32_t)(end - beg)) << 32) | (uint32_t)v;
        }
        key[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)  // bitonic sort, ascending keys
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += kBlock) {
                const int lo = 2 * i - (i & (stride - 1));
                const int hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long a = key[lo], b = key[hi];
                if ((a > b) == up) {
                    key[lo] = b;
                    key[hi] = a;
                }
            }
            __syncthreads();
        }
    for (int r = threadIdx.x; r < H; r += kBlock) {
        const int32_t v = (int32_t)(uint32_t)key[r];
        const int d = (int)~(uint32_t)(key[r] >> 32);
        __stcg(list + r, v);
        __stcg(tasks + r, (d + kCoreSeg - 1) / kCoreSeg);
        st_color<true>(p.cA + v, -(r + 1));
    }
    __syncthreads();
}

// One block: exclusive prefix sum of x[0..T) in place, x[T] = the total.
__device__ __noinline__ void block_scan_inplace(int32_t *x, int T, Shared &sh)
{
    int carry = 0;
    for (int i0 = 0; i0 < T; i0 += kBlock) {
        const int i = i0 + threadIdx.x;
        const int v = i < T ? __ldcg(x + i) : 0;
        int total;
        const int before = block_exclusive_scan(v, reinterpret_cast<int *>(sh.warp_bm), total);
        if (i < T) __stcg(x + i, carry + before);
        carry += total;
    }
    if (threadIdx.x == 0) __stcg(x + T, carry);
    __syncthreads();
}

// All blocks: the cores' adjacency bit matrices, from the core vertices'
// rows (a neighbour is in its graph's core when its colour slot holds a rank
// mark).  Tasks of kCoreSeg entries are claimed warp by warp.
template <bool BATCH>
__device__ __noinline__ void core_build(const KParams &p, int T, long long &mb)
{
    const int lane = threadIdx.x & 31;
    const int32_t *tpfx = p.hub[1];
    const int ntask = __ldcg(tpfx + T);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&p.st->core_task, 1);
        t = __shfl_sync(FULL_MASK, t, 0);
        if (t >= ntask) break;
        int lo = 0, hi = T - 1;  // the entry whose tasks hold t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldcg(tpfx + mid) <= t) lo = mid;
            else hi = mid - 1;
        }
        const int i = lo;
        const int k = t - __ldcg(tpfx + i);
        const int32_t v = __ldcg(p.mid_all + i);
        const int gg = BATCH ? __ldcg(p.hub[0] + i) : 0;
        const GraphStat &gs = p.gstat[gg];
        const int r = i - gs.core_off;
        const int Hp = (gs.core_cnt + 31) & ~31;  // column stride: word w of rank r at w * Hp + r
        uint32_t *bits = reinterpret_cast<uint32_t *>(p.wl[1]) + gs.core_bofs;
        int64_t rb, re;
        int32_t nbase, g;
        row_of<BATCH>(p, v, rb, re, nbase, g);
        const int64_t beg = rb + (int64_t)k * kCoreSeg;
        const int64_t end = min(re, beg + kCoreSeg);
        for (int64_t i0 = beg; i0 < end; i0 += 32 * kUnroll) {
            int32_t u[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) {
                const int64_t e = i0 + q * 32 + lane;
                u[q] = e < end ? nbase + __ldg(p.col_idx + e) : -1;
            }
            int c[kUnroll];
#pragma unroll
            for (int q = 0; q < kUnroll; ++q) c[q] = u[q] >= 0 ? __ldcg(p.cA + u[q]) : 0;
#pragma unroll
            for (int q = 0; q < kUnroll; ++q)
                if (c[q] < 0) {
                    const int j = -c[q] - 1;
                    atomicOr(bits + (size_t)(j >> 5) * Hp + r, 1u << (j & 31));
                }
        }
        // First-Fit of a core vertex reads its row (index + colour), its row
        // pointers and writes its colour.
        if (lane == 0) mb += 8ll * (end - beg) + (k == 0 ? 12 : 0);
    }
}

// First colour >= 1 not in the forbidden set Fl; warp-wide (every lane
// gets it).
__device__ __forceinline__ int first_free_warp(const uint32_t *Fl, int Fw, int lane)
{
    for (int w0 = 0; w0 < Fw; w0 += 32) {
        const int w = w0 + lane;
        uint32_t fr = w < Fw ? ~Fl[w] : 0u;
        if (w == 0) fr &= ~1u;  // colour 0 is not a colour
        const unsigned bal = __ballot_sync(FULL_MASK, fr != 0u);
        if (bal) {
            const int src = __ffs(bal) - 1;
            const uint32_t fb = __shfl_sync(FULL_MASK, fr, src);
            return (w0 + src) * 32 + __ffs(fb) - 1;
        }
    }
    return Fw * 32;  // not reached: Fw words cover colours up to H+1
}

// The bytes of w that differ from the tag byte (t4 = tag in all four), as
// bits 0..3: the high bit of ((v & 0x7f..) + 0x7f..) | v is set exactly in the
// non-zero bytes of v (no carry crosses a byte), and the multiply gathers
// bits 7, 15, 23, 31 into bits 28..31 (the four partial products land on
// distinct bits).
__device__ __forceinline__ uint32_t untagged4(uint32_t w, uint32_t t4)
{
    const uint32_t v = w ^ t4;
    const uint32_t nz = (((v & 0x7f7f7f7fu) + 0x7f7f7f7fu) | v) & 0x80808080u;
    return (nz * 0x00204081u) >> 28;
}

constexpr int kMarkColours = 1024;              // colours the byte rows cover
constexpr int kMarkStride = kMarkColours + 16;  // bytes per row (16-byte aligned, rows on different banks)
__device__ __noinline__ int core_colour(const KParams &p, Shared &sh, const int32_t *list, const uint32_t *bits, int H,
                                       int32_t *also)
{
    static_assert(offsetof(Shared, ring) == sizeof(sh.seg), "staging area and ring are contiguous");
    unsigned char *area = reinterpret_cast<unsigned char *>(&sh.seg[0][0][0]);
    constexpr int kArea = (int)(sizeof(sh.seg) + sizeof(sh.ring));
    uint16_t *col16 = reinterpret_cast<uint16_t *>(area);                    // colour of each rank
    unsigned char *mark = area + kCoreMax * 2;                               // 32 byte rows
    uint32_t *F = reinterpret_cast<uint32_t *>(area + kCoreMax * 2);         // or 32 bitset rows of Fw words
    const int Fw = (H + 2 + 31) / 32;                                        // colours 0..H+1
    static_assert(kCoreMax * 2 + 32 * kMarkStride <= kArea, "byte rows fit");
    static_assert(kCoreMax * 2 + 32 * ((kCoreMax + 2 + 31) / 32) * 4 <= kArea, "bitset rows fit");
    static_assert((kCoreMax * 2) % 16 == 0 && kMarkStride % 16 == 0, "byte rows are 16-byte aligned");
    constexpr int kWordsPerThread = (kCoreMax / 32 + kWarps - 1) / kWarps;
    const int Hp = (H + 31) & ~31;  // column stride of the bit matrix
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 32 * kMarkStride / 4; i += kBlock) reinterpret_cast<uint32_t *>(mark)[i] = 0u;
    bool bitset = false;  // block-uniform: colours may reach kMarkColours
    int M = 0;
    uint32_t xs[kWordsPerThread];
#pragma unroll
    for (int q = 0; q < kWordsPerThread; ++q) xs[q] = 0u;  // batch 0 has no earlier batch
    uint32_t inb = 0u;
    int32_t vid = -1;
    if (wid == 0 && lane < min(32, H)) {
        inb = __ldcg(bits + lane);  // word 0 of rank lane
        vid = __ldcg(list + lane);
    }
    __syncthreads();
    for (int b = 0; 32 * b < H; ++b) {
        const int nb = min(32, H - 32 * b);
        const unsigned tag = (unsigned)b + 1;  // b < 128: one tag per batch
        if (lane < nb) {
            unsigned char *row = mark + lane * kMarkStride;
            uint32_t *Fl = F + lane * Fw;
#pragma unroll
            for (int q = 0; q < kWordsPerThread; ++q) {
                uint32_t x = xs[q];
                const int base = 32 * (wid + q * kWarps);
                if (!bitset) {
                    while (x) {  // four bits at a time (a missing bit repeats the first)
                        const int j0 = __ffs(x) - 1;
                        x &= x - 1;
                        const int j1 = x ? __ffs(x) - 1 : j0;
                        x &= x - 1;
                        const int j2 = x ? __ffs(x) - 1 : j0;
                        x &= x - 1;
                        const int j3 = x ? __ffs(x) - 1 : j0;
                        x &= x - 1;
                        const int c0 = col16[base + j0], c1 = col16[base + j1];
                        const int c2 = col16[base + j2], c3 = col16[base + j3];
                        row[c0] = (unsigned char)tag;
                        row[c1] = (unsigned char)tag;
                        row[c2] = (unsigned char)tag;
                        row[c3] = (unsigned char)tag;
                    }
                } else {
                    while (x) {
                        const int c = col16[base + __ffs(x) - 1];
                        x &= x - 1;
                        atomicOr(Fl + (c >> 5), 1u << (c & 31));
                    }
                }
            }
        }
        // the next batch's words (they do not depend on colours)
        const int b1 = b + 1, r1 = 32 * b1 + lane;
#pragma unroll
        for (int q = 0; q < kWordsPerThread; ++q) {
            const int w = wid + q * kWarps;
            xs[q] = (w < b1 && r1 < H) ? __ldcg(bits + (size_t)w * Hp + r1) : 0u;
        }
        __syncthreads();
        if (wid == 0) {
            int mine = 0;
            if (!bitset) {
                const uint32_t t4 = tag * 0x01010101u;
                for (int k = 0; k < nb; ++k) {
                    unsigned char *rowk = mark + k * kMarkStride;
                    if (lane < k && ((inb >> k) & 1u)) rowk[mine] = (unsigned char)tag;
                    __syncwarp();
                    int c = 0;
                    for (int c0 = 0; c == 0 && c0 < kMarkColours; c0 += 512) {  // colours c0 + 16*lane .. +15
                        const uint4 w4 = *reinterpret_cast<const uint4 *>(rowk + c0 + 16 * lane);
                        uint32_t fm = untagged4(w4.x, t4) | (untagged4(w4.y, t4) << 4) | (untagged4(w4.z, t4) << 8) |
                                      (untagged4(w4.w, t4) << 12);  // bit i: colour c0 + 16*lane + i untagged
                        if (c0 == 0 && lane == 0) fm &= ~1u;  // colour 0 is not a colour
                        const unsigned bal = __ballot_sync(FULL_MASK, fm != 0u);
                        if (bal) {
                            const int src = __ffs(bal) - 1;
                            const uint32_t fb = __shfl_sync(FULL_MASK, fm, src);
                            c = c0 + 16 * src + __ffs(fb) - 1;
                        }
                    }
                    if (lane == k) mine = c;
                }
            } else {
                for (int k = 0; k < nb; ++k) {
                    if (lane < k && ((inb >> k) & 1u)) atomicOr(F + k * Fw + (mine >> 5), 1u << (mine & 31));
                    __syncwarp();
                    const int c = first_free_warp(F + k * Fw, Fw, lane);
                    if (lane == k) mine = c;
                }
            }
            if (lane < nb) {
                col16[32 * b + lane] = (uint16_t)mine;
                st_color<true>(p.cA + vid, mine);
                if (also) st_color<true>(also + vid, mine);
            }
            const int bm = __reduce_max_sync(FULL_MASK, mine);
            // the next batch's in-batch word and vertices
            inb = r1 < H ? __ldcg(bits + (size_t)b1 * Hp + r1) : 0u;
            vid = r1 < H ? __ldcg(list + r1) : -1;
            if (lane == 0) sh.claim = max(M, bm);
        }
        __syncthreads();
        const int Mprev = M;
        M = sh.claim;
        if (!bitset && M + 32 >= kMarkColours) {
            // the next batch could reach kMarkColours: bitset rows from here on
            bitset = true;
            for (int i = threadIdx.x; i < 32 * Fw; i += kBlock) F[i] = 0u;
        } else if (bitset) {
            // every set bit is a colour <= M: clear those words
            const int fw = min(Fw, (max(M, Mprev) >> 5) + 1);
            for (int i = threadIdx.x; i < 32 * fw; i += kBlock) F[(i / fw) * Fw + (i % fw)] = 0u;
        }
        __syncthreads();
    }
    return M;
}


// The core phase of the asynchronous mode (all blocks; block 0 has just run
// plan_ordering).  Each graph's hubs of degree > core_deg are counted; a
// graph with 1..kCoreMax of them whose bit matrix still fits the buffer gets
// a core: its candidates are listed, one block sorts them, all blocks build
// the bit matrices, and one block per graph colours its core (the hub pass
// then skips them); the others stay ordinary hubs.  Ends with a grid barrier.
template <bool BATCH>
__device__ __noinline__ void core_stage(const KParams &p, Shared &sh)
{
    DevState *st = p.st;
    const unsigned nbl = gridDim.x;
    const int lane = threadIdx.x & 31;
    const bool snap = (p.mode & GC_REPAIR_SNAPSHOT) && !(p.mode & GC_ALG_TWO_PHASE);
    long long mb = 0;
    const int nh = ld_volatile(&st->hub_all_count);
    // each graph's candidates
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < nh; i += nbl * kBlock) {
        const int32_t v = __ldcg(p.hub_all + i);
        int64_t beg, end;
        int32_t nbase, g;
        row_of<BATCH>(p, v, beg, end, nbase, g);
        if (end - beg > p.core_deg) atomicAdd(&p.gstat[g].core_cnt, 1);
    }
    grid_sync(st, nbl);
    // block 0: which graphs get a core (those with 1..kCoreMax candidates, in
    // graph order while their lists and bit matrices fit: the prefix sums
    // only grow, so the graphs with a core come before the first that does
    // not fit), their list offsets and bit-matrix words
    if (blockIdx.x == 0) {
        long long carry_c = 0, carry_w = 0;
        for (int g0 = 0; g0 < p.G; g0 += kBlock) {
            const int g = g0 + threadIdx.x;
            int H = 0;
            if (g < p.G) {
                H = __ldcg(&p.gstat[g].core_cnt);
                if (H > kCoreMax) H = 0;
            }
            const int W = (H + 31) / 32;
            int tot_c, tot_w;
            const int before_c = block_exclusive_scan(H, reinterpret_cast<int *>(sh.warp_bm), tot_c);
            const int before_w = block_exclusive_scan(W * W, reinterpret_cast<int *>(sh.warp_bm), tot_w);
            if (g < p.G) {
                const long long off = carry_c + before_c, bofs = carry_w + 32ll * before_w;
                const bool on = H > 0 && off + H < (long long)p.n && bofs + 32ll * W * W <= (long long)p.n;
                p.gstat[g].core_on = on;
                p.gstat[g].core_off = (int)off;
                p.gstat[g].core_bofs = (int)bofs;
                p.gstat[g].core_cnt = on ? H : 0;
                if (on) {
                    atomicMax(&st->core_count, (int)(off + H));          // entries listed
                    atomicMax(&st->core_words, bofs + 32ll * W * W);     // words to clear
                }
            }
            carry_c += tot_c;
            carry_w += 32ll * tot_w;
        }
        __syncthreads();
    }
    grid_sync(st, nbl);
    // the candidates of the graphs with a core, listed graph by graph; their
    // bit matrices cleared
    const long long words_all = *(volatile long long *)&st->core_words;
    const int T = ld_volatile(&st->core_count);
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < nh; i += nbl * kBlock) {
        const int32_t v = __ldcg(p.hub_all + i);
        int64_t beg, end;
        int32_t nbase, g;
        row_of<BATCH>(p, v, beg, end, nbase, g);
        if (end - beg > p.core_deg && __ldcg(&p.gstat[g].core_on)) {
            const int o = __ldcg(&p.gstat[g].core_off) + atomicAdd(&p.gstat[g].core_fill, 1);
            __stcg(p.mid_all + o, v);
            if (BATCH) __stcg(p.hub[0] + o, g);
        }
    }
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < words_all; i += (long long)nbl * kBlock)
        __stcg(p.wl[1] + i, 0);
    grid_sync(st, nbl);
    // one block per core: sort, rank marks, task counts
    for (;;) {
        if (threadIdx.x == 0) sh.claim = atomicAdd(&st->core_n, 1);
        __syncthreads();
        const int g = sh.claim;
        __syncthreads();
        if (g >= p.G) break;
        const int H = __ldcg(&p.gstat[g].core_cnt);
        if (H == 0) continue;
        const int off = __ldcg(&p.gstat[g].core_off);
        core_sort<BATCH>(p, sh, p.mid_all + off, H, p.hub[1] + off);
    }
    grid_sync(st, nbl);
    if (T > 0) {
        if (blockIdx.x == 0) block_scan_inplace(p.hub[1], T, sh);
        grid_sync(st, nbl);
        core_build<BATCH>(p, T, mb);
        grid_sync(st, nbl);
        // one block per core: colour it
        for (;;) {
            if (threadIdx.x == 0) sh.claim = atomicAdd(&st->core_colors, 1);
            __syncthreads();
            const int g = sh.claim;
            __syncthreads();
            if (g >= p.G) break;
            const GraphStat &gs = p.gstat[g];
            const int H = __ldcg(&gs.core_cnt);
            if (H == 0) continue;
            core_colour(p, sh, p.mid_all + __ldcg(&gs.core_off),
                        reinterpret_cast<const uint32_t *>(p.wl[1]) + __ldcg(&gs.core_bofs), H,
                        snap ? p.cB : nullptr);
        }
        grid_sync(st, nbl, kBarrierTimeoutNs, 1024);  // the grid waits for the cores' serial work
    }
    for (int o = 16; o > 0; o >>= 1) mb += __shfl_down_sync(FULL_MASK, mb, o);
    if (lane == 0 && mb) atomicAdd(&st->model_bytes, (unsigned long long)mb);
}

// The prologue of a colouring launch (all blocks): degree binning of V (hub lists),
// colour initialisation, per-graph statistics, the ordered round-0 plan
// and the core (asynchronous), or the first worklist of an incremental
// recolouring.  Ends with a grid barrier; its byte-model count goes to the
// launch state directly.
template <bool ASYNC, bool BATCH>
__device__ __forceinline__ void prologue(const KParams &p, Shared &sh)
{
    DevState *st = p.st;
    const int lane = threadIdx.x & 31;
    const bool twop = (p.mode & GC_ALG_TWO_PHASE) != 0;
    const bool tiers = ASYNC && !twop && (p.mode & GC_TIERS) != 0;
    const bool keep = ASYNC && (p.mode & GC_FF_KEEPERS) != 0;
    const bool recolor = p.touched != nullptr;
    const unsigned nbl = gridDim.x;
    long long mb = 0;
    {
        // Prologue: degree binning of V (hub list) and colour initialisation.
        // Deterministic round 0 colours every vertex from a snapshot in which
        // nothing is coloured yet, so every vertex gets colour 1.
        const long long stride = (long long)gridDim.x * kBlock;
        if (recolor && (!ASYNC || keep)) {
            // Incremental recolouring needs no binning (no round 0): only the
            // second snapshot buffer or the keepers marks are initialised.
            for (long long v = (long long)blockIdx.x * kBlock + threadIdx.x; v < p.n; v += stride) {
                if (!ASYNC) st_color<false>(p.cB + v, __ldcg(p.cA + v));  // both snapshot buffers start equal
                if (keep) p.mark[v] = 0;
            }
        }
        // One graph, asynchronous, 16-byte aligned row pointers and colours:
        // groups of four consecutive vertices, their row pointers read as one
        // 16-byte load (plus the next group's first), four groups per thread
        // per step (16 vertices: one step covers a 2^21-vertex graph), the
        // colours cleared with 16-byte stores.
        const bool vec = !BATCH && ASYNC && !recolor && !keep &&
                         (reinterpret_cast<uintptr_t>(p.row_ptr) & 15u) == 0 &&
                         (reinterpret_cast<uintptr_t>(p.cA) & 15u) == 0;
        if (vec) {
            auto append = [&](bool hub, bool midv, int32_t v) {  // every lane of the warp calls it
                const unsigned m = __ballot_sync(FULL_MASK, hub);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int ob = 0;
                    if (lane == leader) ob = atomicAdd(&st->hub_all_count, __popc(m));
                    ob = __shfl_sync(FULL_MASK, ob, leader);
                    if (hub) {
                        const int o = ob + __popc(m & ((1u << lane) - 1u));
                        if (o < p.hub_cap) __stcg(p.hub_all + o, v);
                        else atomicOr(&st->error, GC_EW_OVERFLOW);
                    }
                }
                const unsigned mm = __ballot_sync(FULL_MASK, midv);
                if (mm) {
                    const int leader = __ffs(mm) - 1;
                    int ob = 0;
                    if (lane == leader) ob = atomicAdd(&st->mid_all_count, __popc(mm));
                    ob = __shfl_sync(FULL_MASK, ob, leader);
                    if (midv) {
                        const int o = ob + __popc(mm & ((1u << lane) - 1u));
                        if (o < p.n) __stcg(p.mid_all + o, v);
                        else atomicOr(&st->error, GC_EW_OVERFLOW);
                    }
                }
            };
            auto classify = [&](bool valid, int32_t v, int64_t deg) {
                bool hub = false, midv = false;
                if (valid) {
                    hub = deg > p.t2;
                    midv = tiers && !hub && deg > p.t1;
                    if (hub) atomicAdd(&p.gstat[0].hubs, 1u);
                    if (!hub && deg > kT1Max && __ldcg(&p.gstat[0].wide) == 0u) atomicOr(&p.gstat[0].wide, 1u);
                }
                append(hub, midv, v);
            };
            constexpr int kG = 4;
            const long long n4 = (long long)p.n / 4;
            const long long tid = (long long)blockIdx.x * kBlock + threadIdx.x;
            const int4 *rp4 = reinterpret_cast<const int4 *>(p.row_ptr);
            int4 *c4 = reinterpret_cast<int4 *>(p.cA);
            for (long long base = 0; base < n4; base += kG * stride) {
                int4 r[kG];
                int32_t nx[kG];
#pragma unroll
                for (int q = 0; q < kG; ++q) {
                    const long long gi = base + q * stride + tid;
                    r[q] = make_int4(0, 0, 0, 0);
                    nx[q] = 0;
                    if (gi < n4) {
                        r[q] = __ldg(rp4 + gi);
                        nx[q] = __ldg(p.row_ptr + 4 * gi + 4);  // <= row_ptr[n]
                    }
                }
#pragma unroll
                for (int q = 0; q < kG; ++q) {
                    const long long gi = base + q * stride + tid;
                    const bool ok = gi < n4;
                    const int32_t v = (int32_t)(4 * gi);
                    classify(ok, v, (int64_t)r[q].y - r[q].x);
                    classify(ok, v + 1, (int64_t)r[q].z - r[q].y);
                    classify(ok, v + 2, (int64_t)r[q].w - r[q].z);
                    classify(ok, v + 3, (int64_t)nx[q] - r[q].w);
                    if (ok) __stcg(c4 + gi, make_int4(0, 0, 0, 0));
                }
            }
            // the last n % 4 vertices, one per thread (every lane of a warp
            // takes part in the appends)
            {
                const long long vi = 4 * n4 + tid;
                const bool ok = vi < p.n;
                int64_t deg = 0;
                if (ok) {
                    deg = (int64_t)__ldg(p.row_ptr + vi + 1) - __ldg(p.row_ptr + vi);
                    st_color<false>(p.cA + vi, 0);
                }
                if (tid < 32) classify(ok, (int32_t)vi, deg);  // n % 4 < 32: block 0, warp 0
            }
        }
        // Eight vertices per thread per step, their row lookups issued together
        // (each is a chain of dependent loads in a batch).
        constexpr int kProU = 8;
        for (long long b0 = (long long)blockIdx.x * kBlock; b0 < ((recolor || vec) ? 0ll : (long long)p.n);
             b0 += kProU * stride) {
            int64_t degs[kProU];
            int32_t gs[kProU];
            if (BATCH && !p.rp_off) {
                // Graph g's row pointers start at row_ptr + vtx_off[g] + g, so
                // vertex v's are row_ptr[v + g], row_ptr[v + g + 1]: only g is
                // looked up, and the loads of the four vertices are issued
                // stage by stage so that they overlap.
                int e[kProU];
#pragma unroll
                for (int u = 0; u < kProU; ++u) {
                    const long long vi = b0 + u * stride + threadIdx.x;
                    e[u] = vi < p.n ? __ldg(p.gid_lut + (vi >> kLutShift)) : -1;
                }
#pragma unroll
                for (int u = 0; u < kProU; ++u) {
                    const long long vi = b0 + u * stride + threadIdx.x;
                    int gg = e[u] < 0 ? -e[u] - 1 : e[u];
                    if (e[u] >= 0 && vi < p.n)  // the block of ids spans graphs (rare)
                        while (gg + 1 < p.G && __ldg(p.vtx_off + gg + 1) <= vi) ++gg;
                    gs[u] = gg;
                }
                int32_t r0[kProU], r1[kProU];
#pragma unroll
                for (int u = 0; u < kProU; ++u) {
                    const long long vi = b0 + u * stride + threadIdx.x;
                    r0[u] = r1[u] = 0;
                    if (vi < p.n) {
                        r0[u] = __ldg(p.row_ptr + vi + gs[u]);
                        r1[u] = __ldg(p.row_ptr + vi + gs[u] + 1);
                    }
                }
#pragma unroll
                for (int u = 0; u < kProU; ++u) degs[u] = (int64_t)r1[u] - r0[u];
            } else {
#pragma unroll
                for (int u = 0; u < kProU; ++u) {
                    const long long vi = b0 + u * stride + threadIdx.x;
                    degs[u] = -1;
                    gs[u] = 0;
                    if (vi < p.n) {
                        int64_t beg, end;
                        int32_t nbase;
                        row_of<BATCH>(p, (int32_t)vi, beg, end, nbase, gs[u]);
                        degs[u] = end - beg;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kProU; ++u) {
                const long long vi = b0 + u * stride + threadIdx.x;
                bool hub = false, midv = false;
                const int32_t v = (int32_t)vi;
                if (vi < p.n) {
                    const int64_t deg = degs[u];
                    const int32_t g = gs[u];
                    hub = deg > p.t2;
                    midv = tiers && !hub && deg > p.t1;
                    if (hub && ASYNC) atomicAdd(&p.gstat[g].hubs, 1u);
                    if (ASYNC && !hub && deg > kT1Max && __ldcg(&p.gstat[g].wide) == 0u)
                        atomicOr(&p.gstat[g].wide, 1u);
                    st_color<false>(p.cA + v, ASYNC ? 0 : 1);
                    if (!ASYNC && twop) st_color<false>(p.cB + v, 1);
                    if (!ASYNC) mb += 4;
                    if (keep) p.mark[v] = 0;
                }
                const unsigned m = __ballot_sync(FULL_MASK, hub);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int ob = 0;
                    if (lane == leader) ob = atomicAdd(&st->hub_all_count, __popc(m));
                    ob = __shfl_sync(FULL_MASK, ob, leader);
                    if (hub) {
                        const int o = ob + __popc(m & ((1u << lane) - 1u));
                        if (o < p.hub_cap) __stcg(p.hub_all + o, v);
                        else atomicOr(&st->error, GC_EW_OVERFLOW);
                    }
                }
                const unsigned mm = __ballot_sync(FULL_MASK, midv);
                if (mm) {
                    const int leader = __ffs(mm) - 1;
                    int ob = 0;
                    if (lane == leader) ob = atomicAdd(&st->mid_all_count, __popc(mm));
                    ob = __shfl_sync(FULL_MASK, ob, leader);
                    if (midv) {
                        const int o = ob + __popc(mm & ((1u << lane) - 1u));
                        if (o < p.n) __stcg(p.mid_all + o, v);
                        else atomicOr(&st->error, GC_EW_OVERFLOW);
                    }
                }
            }
        }
        if (BATCH && p.g_rounds)
            for (long long g = (long long)blockIdx.x * kBlock + threadIdx.x; g < p.G; g += stride)
                p.g_rounds[g] = (__ldg(p.vtx_off + g + 1) > __ldg(p.vtx_off + g)) ? 1 : 0;
        if (ASYNC && !recolor) {
            // Flags of the ordered round-0 pass, and (automatic window) a
            // sample of how far lower neighbours sit in id from their vertex.
            const long long ntiles = ((long long)p.n + p.tile - 1) / p.tile;
            for (long long t = (long long)blockIdx.x * kBlock + threadIdx.x; t < ntiles; t += stride)
                p.done[t] = 0;
            if (p.window == 0) {
                // Per graph: how many sampled lower neighbours sit within
                // kNearIds ids of their vertex.
                for (long long b1 = (long long)blockIdx.x * kBlock * kLocalitySample; b1 < p.n;
                     b1 += stride * kLocalitySample) {
                    const long long vi = b1 + (long long)threadIdx.x * kLocalitySample;
                    unsigned long long near = 0, all = 0;
                    int32_t g = -1;
                    if (vi < p.n) {
                        int64_t beg, end;
                        int32_t nbase;
                        row_of<BATCH>(p, (int32_t)vi, beg, end, nbase, g);
                        // the first kLocalitySampleEntries entries of the row, loaded
                        // together; the lower neighbours among them (a prefix: rows are
                        // sorted) are the sample
                        int32_t u[kLocalitySampleEntries];
#pragma unroll
                        for (int q = 0; q < kLocalitySampleEntries; ++q)
                            u[q] = beg + q < end ? nbase + __ldg(p.col_idx + beg + q) : INT32_MAX;
#pragma unroll
                        for (int q = 0; q < kLocalitySampleEntries; ++q) {
                            const bool lower = u[q] < (int32_t)vi;
                            all += lower;
                            near += lower && ((int32_t)vi - u[q]) < kNearIds;
                        }
                    }
                    const int g0 = __shfl_sync(FULL_MASK, g, 0);
                    if (__all_sync(FULL_MASK, g == g0 || g < 0)) {
                        for (int o = 16; o > 0; o >>= 1) {
                            near += __shfl_down_sync(FULL_MASK, near, o);
                            all += __shfl_down_sync(FULL_MASK, all, o);
                        }
                        if (lane == 0 && all) {
                            atomicAdd(&p.gstat[g0].near_lower, near);
                            atomicAdd(&p.gstat[g0].all_lower, all);
                        }
                    } else if (g >= 0 && all) {
                        atomicAdd(&p.gstat[g].near_lower, near);
                        atomicAdd(&p.gstat[g].all_lower, all);
                    }
                }
            }
        }
        if (recolor)  // repeat filter of the touched list
            for (long long w = (long long)blockIdx.x * kBlock + threadIdx.x; w < (long long)p.n / 32 + 1; w += stride)
                p.done[w] = 0;
        grid_sync(st, nbl);
        if (recolor) {
            // Incremental recolouring: the touched vertices (each once) form
            // the worklist of the first iteration; there is no round 0.
            for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < p.n_touched; i += stride) {
                const int32_t v = __ldg(p.touched + i);
                if (v < 0 || v >= p.n) {
                    atomicOr(&st->error, GC_EW_GRAPH);
                    continue;
                }
                const unsigned bit = 1u << (v & 31);
                if (atomicOr((unsigned *)p.done + (v >> 5), bit) & bit) continue;
                int64_t beg, end;
                int32_t nbase, g;
                row_of<BATCH>(p, v, beg, end, nbase, g);
                const unsigned long long deg = (unsigned long long)(end - beg);
                if (deg > (unsigned long long)p.t2) {
                    atomicAdd(&st->wl_packed[0], deg);
                    const int idx = atomicAdd(&st->hub_count[0], 1);
                    if (idx < p.hub_cap) __stcg(p.hub[0] + idx, v);
                    else atomicOr(&st->error, GC_EW_OVERFLOW);
                } else {
                    const int o = (int)(atomicAdd(&st->wl_packed[0], (1ull << kWorkBits) + deg) >> kWorkBits);
                    if (o < p.n) __stcg(p.wl[0] + o, v);
                    else atomicOr(&st->error, GC_EW_OVERFLOW);
                }
            }
            grid_sync(st, nbl);
        }

        if (ASYNC && ld_volatile(&st->error) == 0 && !recolor) {
            // Ids of a naturally numbered mesh are local: neighbours would be
            // coloured concurrently unless the graph goes strictly in id order.
            if (blockIdx.x == 0) plan_ordering<BATCH>(p, sh);
            // The core of one graph (see core_sort); its first barrier also
            // ends plan_ordering (without a core, the end of this launch does).
            if (p.core_deg > 0 && ld_volatile(&st->hub_all_count) > 0) core_stage<BATCH>(p, sh);
            if (blockIdx.x == 0 && threadIdx.x == 0) st->window = ld_volatile(&st->n_ordered);
        }

    }
    for (int o = 16; o > 0; o >>= 1) mb += __shfl_down_sync(FULL_MASK, mb, o);
    if (lane == 0 && mb) atomicAdd(&st->model_bytes, (unsigned long long)mb);
}


// The prologue of a colouring as a launch of its own (degree binning,
// colour initialisation, the round-0 plan and the core), so that the
// rounds' kernel below is compiled without the core's code and calls.
template <bool ASYNC, bool BATCH>
__global__ void __launch_bounds__(kBlock, kMinBlocks) prologue_kernel(KParams p)
{
    extern __shared__ __align__(128) unsigned char gc_smem[];
    Shared &sh = *reinterpret_cast<Shared *>(gc_smem);
    DevState *st = p.st;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_start = global_timer();
    if (ld_volatile(&st->error) == 0) prologue<ASYNC, BATCH>(p, sh);
}

// All rounds of a colouring (after prologue_kernel on the same stream).
// MINB: the resident blocks per SM it is compiled for (kMinBlocks, or 2 for
// grids of at most two blocks per SM, which then get more registers per
// thread).
template <bool ASYNC, bool BATCH, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) color_kernel(KParams p)
{
    extern __shared__ __align__(128) unsigned char gc_smem[];
    Shared &sh = *reinterpret_cast<Shared *>(gc_smem);
    DevState *st = p.st;
    const int lane = threadIdx.x & 31;
    const bool twop = (p.mode & GC_ALG_TWO_PHASE) != 0;
    // Snapshot rounds: deterministic mode, or asynchronous round 0 followed
    // by round-synchronous repair rounds (GC_REPAIR_SNAPSHOT, RSOC only).
    const bool snap = !twop && (!ASYNC || (p.mode & GC_REPAIR_SNAPSHOT) != 0);
    // Degree tiers (asynchronous RSOC): hubs, then mid-degree, then the rest.
    const bool tiers = ASYNC && !twop && (p.mode & GC_TIERS) != 0;
    const bool recolor = p.touched != nullptr;  // incremental: start from the given colours
    unsigned nbl = gridDim.x;
    long long mb = 0;
    uint32_t phase = 0;  // parity bits of this warp's two staging barriers
    if (lane == 0) {
        mbar_init(&sh.mbar[threadIdx.x >> 5][0], 1);
        mbar_init(&sh.mbar[threadIdx.x >> 5][1], 1);
        fence_mbarrier_init();
    }
    __syncwarp();

    if (ld_volatile(&st->error) == 0) {
        bool alive = true;
        const int hub_all_n = ld_volatile(&st->hub_all_count);
        const int mid_all_n = ld_volatile(&st->mid_all_count);
        int q = 0;
        // Tile window for the round-0 pass over the graphs that are not
        // coloured in id order by one warp (window > 1 only).
        const int window = p.window > 1 ? p.window : -1;

        // Stages: one (all of V), or, with tiers, hubs -> mid degree -> low
        // degree, each taken through round 0 and its repair rounds before the
        // next starts (vertices of later stages are still uncoloured then).
        PassIn stages[3];
        int nstages = 1;
        if (recolor) {
            stages[0] = PassIn{false, p.wl[0], packed_count(st, 0), p.hub[0], ld_volatile(&st->hub_count[0]), p.t2};
        } else if (tiers) {
            stages[0] = PassIn{false, nullptr, 0, p.hub_all, hub_all_n, 0};
            stages[1] = PassIn{false, p.mid_all, mid_all_n, nullptr, 0, 0};
            stages[2] = PassIn{true, nullptr, p.n, nullptr, 0, p.t1};
            nstages = 3;
        } else {
            stages[0] = PassIn{true, nullptr, p.n, p.hub_all, hub_all_n, p.t2};
        }

        int32_t *R = p.cA;
        int32_t *W = snap ? p.cB : p.cA;
        int32_t *last_written = p.cA;
        bool copy_back = false;
        int it = 0;
        for (int sg = 0; sg < nstages && alive; ++sg) {
            PassIn in = stages[sg];
            if (in.n == 0 && in.hn == 0) continue;
            const bool last_stage = sg == nstages - 1;
            // Asynchronous round 0 (Algorithm 3): tentative colouring of the
            // stage's vertices, in place on the current colours.  Without
            // snapshot rounds it also lists the vertices that can be in
            // conflict afterwards, and the first repair round inspects only
            // those (every other vertex of U^0 = V is provably clean).
            if (ASYNC && !twop && !recolor) {
                const bool suspects = !snap;
                run_pass<ASYNC, BATCH, (MINB <= 2)>(p, sh, OP_TENT, q++, it, in, R, R, suspects, mb, phase, nbl, window);
                grid_sync(st, nbl);
                if (blockIdx.x == 0 && threadIdx.x == 0 && it < kStamps) st->stamp[it] = global_timer();
                if (ld_volatile(&st->error)) {
                    alive = false;
                    break;
                }
                if (suspects)
                    in = PassIn{false, p.wl[it & 1], packed_count(st, it), p.hub[it & 1],
                                ld_volatile(&st->hub_count[it & (kRing - 1)]), p.t2};
            }
            for (;;) {
                ++it;
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    st->hub_count[(it + 2) & (kRing - 1)] = 0;
                    st->wl_packed[(it + 2) & (kRing - 1)] = 0;
                }
                if (twop) {
                    // Algorithm 2: phase 1 tentative colouring of U (in
                    // deterministic mode iteration 1's phase 1 is the fill of
                    // the prologue), barrier, phase 2 detection, barrier.
                    if (ASYNC || it > 1) {
                        run_pass<ASYNC, BATCH, (MINB <= 2)>(p, sh, OP_TENT, q++, it, in, p.cA, ASYNC ? p.cA : p.cB, false,
                                               mb, phase, nbl, window);
                        grid_sync(st, nbl);
                        if (ld_volatile(&st->error)) {
                            alive = false;
                            break;
                        }
                    }
                    run_pass<ASYNC, BATCH, (MINB <= 2)>(p, sh, OP_DETECT, q++, it, in, ASYNC ? p.cA : p.cB, p.cA, true, mb,
                                           phase, nbl);
                } else {
                    // Algorithm 3: fused detect-and-recolour over U.
                    run_pass<ASYNC, BATCH, (MINB <= 2)>(p, sh, OP_RSOC, q++, it, in, R, W, true, mb, phase, nbl);
                    last_written = W;
                }
                grid_sync(st, nbl);
                if (ld_volatile(&st->error)) {
                    copy_back = true;
                    break;
                }
                const int nl = packed_count(st, it);
                const int nh = ld_volatile(&st->hub_count[it & (kRing - 1)]);
                const int tot = nl + nh;
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    if (it < kStamps) st->stamp[it] = global_timer();
                    st->rounds = it;
                    st->conflicts += (unsigned long long)tot;
                    if (p.round_sizes && it - 1 < p.round_sizes_cap) p.round_sizes[it - 1] = tot;
                    if (it - 1 < kStamps) st->round_head[it - 1] = tot;
                }
                if (snap) {
                    int32_t *t = R;
                    R = W;
                    W = t;
                }
                if (tot == 0) break;
                if (it >= p.max_rounds) {
                    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&st->error, GC_EW_NO_CONVERGENCE);
                    copy_back = true;
                    break;
                }
                in = PassIn{false, p.wl[it & 1], nl, p.hub[it & 1], nh, p.t2};
                const unsigned long long work =
                    *(volatile unsigned long long *)&st->wl_packed[it & (kRing - 1)] & ((1ull << kWorkBits) - 1);
                if (last_stage && nbl > 1 && tot <= p.tail && work <= (unsigned long long)p.tail * kTailWorkPerVertex) {
                    // Few vertices left: block 0 finishes alone with block-local
                    // barriers; the others leave.
                    if (blockIdx.x != 0) {
                        alive = false;
                        break;
                    }
                    nbl = 1;
                }
            }
            if (copy_back) break;
        }
        // Deterministic RSOC stopped early (cap or error): the latest colours
        // may sit in the second buffer.  On normal termination both buffers
        // hold the final colouring.
        if (alive && copy_back && snap && last_written != p.cA) {
            const long long s2 = (long long)nbl * kBlock;
            for (long long v = (long long)blockIdx.x * kBlock + threadIdx.x; v < p.n; v += s2)
                __stcg(p.cA + v, __ldcg(p.cB + v));
        }
    }

    // Colour statistics of the result in the same launch: every block,
    // those that left the rounds early included, meets at one more grid
    // barrier and scans its share of the colours.
    if (p.stats_bitmap) {
        grid_sync(st, gridDim.x);
        colour_stats(p.cA, p.n, st, p.stats_bitmap);
    }

    // flush the byte-model counter
    for (int o = 16; o > 0; o >>= 1) mb += __shfl_down_sync(FULL_MASK, mb, o);
    if (lane == 0 && mb) atomicAdd(&st->model_bytes, (unsigned long long)mb);
}

// ------------------------------------------------------------------------
// auxiliary kernels
// ------------------------------------------------------------------------

template <bool BATCH>
__global__ void validate_kernel(KParams p)
{
    bool bad = false;
    for (long long vi = (long long)blockIdx.x * blockDim.x + threadIdx.x; vi < p.n && !bad;
         vi += (long long)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)vi;
        int64_t beg, end;
        int32_t nbase, g;
        row_of<BATCH>(p, v, beg, end, nbase, g);
        int64_t gn = p.n, lo_e = 0, hi_e = LLONG_MAX;
        if (BATCH) {
            gn = __ldg(p.vtx_off + g + 1) - __ldg(p.vtx_off + g);
            lo_e = __ldg(p.edge_off + g);
            hi_e = __ldg(p.edge_off + g + 1);
            const int64_t rpo = p.rp_off ? __ldg(p.rp_off + g) : (int64_t)nbase + g;
            if (v == nbase && __ldg(p.row_ptr + rpo) != 0) bad = true;
        }
        if (!BATCH) {
            hi_e = p.nnz;
            if (v == 0 && beg != 0) bad = true;
        }
        if (beg > end || beg < lo_e || end > hi_e) { bad = true; break; }
        if (v - nbase == gn - 1 && end != hi_e) { bad = true; break; }  // last row ends at nnz
        for (int64_t k = beg; k < end && !bad; ++k) {
            const int32_t lu = __ldg(p.col_idx + k);
            if (lu < 0 || lu >= gn) { bad = true; break; }
            const int32_t u = nbase + lu;
            if (u == v) bad = true;
            if (k > beg && __ldg(p.col_idx + k - 1) >= lu) bad = true;
            if (bad) break;
            int64_t ub, ue;
            int32_t unb, ug;
            row_of<BATCH>(p, u, ub, ue, unb, ug);
            const int32_t lv = v - nbase;
            int64_t lo = ub, hi = ue;  // binary search for v in u's row
            bool found = false;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int32_t x = __ldg(p.col_idx + mid);
                if (x == lv) { found = true; break; }
                if (x < lv) lo = mid + 1; else hi = mid;
            }
            if (!found) bad = true;
        }
    }
    if (bad) atomicOr(&p.st->error, GC_EW_GRAPH);
}

// Result check: 1 <= c(v) <= deg(v)+1 and no neighbour shares c(v).
template <bool BATCH>
__global__ void check_kernel(KParams p)
{
    bool bad = false;
    for (long long vi = (long long)blockIdx.x * blockDim.x + threadIdx.x; vi < p.n && !bad;
         vi += (long long)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)vi;
        int64_t beg, end;
        int32_t nbase, g;
        row_of<BATCH>(p, v, beg, end, nbase, g);
        const int cv = __ldcg(p.cA + v);
        if (cv < 1 || cv > (int)(end - beg) + 1) bad = true;
        for (int64_t k = beg; k < end && !bad; ++k)
            if (__ldcg(p.cA + nbase + __ldg(p.col_idx + k)) == cv) bad = true;
    }
    if (bad) atomicOr(&p.st->error, GC_EW_CHECK);
}

// Batch: graph of the first vertex of every 2^kLutShift-vertex chunk.
__global__ void build_lut_kernel(const int64_t *vtx_off, int32_t G, int32_t n, int32_t *lut)
{
    const long long chunks = ((long long)n + (1 << kLutShift) - 1) >> kLutShift;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (long long)gridDim.x * blockDim.x) {
        const int64_t x = c << kLutShift;
        int lo = 0, hi = G - 1;  // largest g with vtx_off[g] <= x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (vtx_off[mid] <= x) lo = mid; else hi = mid - 1;
        }
        const int64_t block_end = x + (1ll << kLutShift) < (int64_t)n ? x + (1ll << kLutShift) : (int64_t)n;
        lut[c] = (lo + 1 >= G || vtx_off[lo + 1] >= block_end) ? -lo - 1 : lo;  // negative: one graph only
    }
}

// ------------------------------------------------------------------------
// failure-path probes (gc_debug_wait_timeout)
// ------------------------------------------------------------------------

// One bounded wait of the colouring kernel run against something that never
// happens, with a short limit; the wait must give up, set GC_EW_TIMEOUT and
// return.  One warp.
//   GC_WAIT_TILE_DONE:  an ordered round-0 tile flag nobody publishes (p.done
//                       zeroed);
//   GC_WAIT_PIPE_CHUNK: a warp-group chunk whose lane 0 (vertex 32) has a
//                       lower neighbour (vertex 0) that no warp colours
//                       (p.row_ptr/p.col_idx: that graph, p.cA zeroed);
//   GC_WAIT_STAGE_COPY: a staged-copy barrier that no copy completes (an
//                       mbarrier expecting one arrival that never comes).
__global__ void wait_probe_kernel(KParams p, int which, unsigned long long timeout_ns)
{
    __shared__ unsigned long long bar;
    const int lane = threadIdx.x & 31;
    if (which == GC_WAIT_TILE_DONE) {
        wait_tile_done(p, 0, lane, timeout_ns);
    } else if (which == GC_WAIT_PIPE_CHUNK) {
        const int32_t v = 32 + lane;
        const int32_t beg = __ldg(p.row_ptr + v), end = __ldg(p.row_ptr + v + 1);
        long long mb = 0;
        chunk_pipe(p, GlobalEnts{p.col_idx}, 32, v, beg, end - beg, 0, p.cA, mb, lane, timeout_ns);
    } else if (which == GC_WAIT_STAGE_COPY) {
        if (lane == 0) {
            mbar_init(&bar, 1);
            fence_mbarrier_init();
        }
        __syncwarp();
        if (lane == 0) wait_mbar(p, &bar, 0, timeout_ns);
        __syncwarp();
    }
}

cudaError_t launch_wait_probe(const KParams &p, int which, unsigned long long timeout_ns, cudaStream_t s)
{
    wait_probe_kernel<<<1, 32, 0, s>>>(p, which, timeout_ns);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------

// SMs of the current device.
static int sm_count()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

template <bool A, bool B>
static cudaError_t launch_one(const KParams &p, int grid, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = sizeof(Shared);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // The prologue (a streaming pass over V, the core's bit matrices) runs
    // on as many resident blocks as it can hold when the rounds kernel has
    // at least two per SM; it plans round 0 for the rounds kernel's grid.
    static int prologue_occ = 0;  // resident prologue blocks per SM (the same on every sm_103a device)
    const int sms = sm_count();
    if (prologue_occ == 0) {
        int a = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, prologue_kernel<A, B>, kBlock, sizeof(Shared)) ==
            cudaSuccess)
            prologue_occ = a;
        else
            cudaGetLastError();
    }
    KParams q = p;
    q.round_blocks = grid;
    cudaLaunchConfig_t pcfg = cfg;
    if (sms > 0 && grid >= 2 * sms && prologue_occ * sms > grid) pcfg.gridDim = dim3((unsigned)(prologue_occ * sms));
    cudaError_t e = cudaLaunchKernelEx(&pcfg, prologue_kernel<A, B>, q);
    if (e != cudaSuccess) return e;
    if constexpr (A) {
        if (grid <= 2 * sms) return cudaLaunchKernelEx(&cfg, color_kernel<A, B, 2>, q);
    }
    return cudaLaunchKernelEx(&cfg, color_kernel<A, B, kMinBlocks>, q);
}

cudaError_t launch_color(const KParams &p, bool async, bool batch, int grid, cudaStream_t s)
{
    if (async) return batch ? launch_one<true, true>(p, grid, s) : launch_one<true, false>(p, grid, s);
    return batch ? launch_one<false, true>(p, grid, s) : launch_one<false, false>(p, grid, s);
}

static const void *color_kernel_ptr(bool async, bool batch, bool two = false)
{
    if (two) return batch ? (const void *)color_kernel<true, true, 2> : (const void *)color_kernel<true, false, 2>;
    return async ? (batch ? (const void *)color_kernel<true, true, kMinBlocks>
                          : (const void *)color_kernel<true, false, kMinBlocks>)
                 : (batch ? (const void *)color_kernel<false, true, kMinBlocks>
                          : (const void *)color_kernel<false, false, kMinBlocks>);
}

static const void *prologue_kernel_ptr(bool async, bool batch)
{
    return async ? (batch ? (const void *)prologue_kernel<true, true> : (const void *)prologue_kernel<true, false>)
                 : (batch ? (const void *)prologue_kernel<false, true> : (const void *)prologue_kernel<false, false>);
}

cudaError_t prepare_color_kernels()
{
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (const void *f : {color_kernel_ptr(a, b), color_kernel_ptr(a, b, a != 0), prologue_kernel_ptr(a, b)}) {
                const cudaError_t e =
                    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
                if (e != cudaSuccess) return e;
            }
    return cudaSuccess;
}

// Blocks per SM both launches of a colouring can hold (the grid of each is
// cooperative: all its blocks resident at once).
cudaError_t query_occupancy(bool async, bool batch, int *blocks_per_sm)
{
    cudaError_t e = prepare_color_kernels();
    if (e != cudaSuccess) return e;
    int a = 0, b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, color_kernel_ptr(async, batch), kBlock, sizeof(Shared));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, prologue_kernel_ptr(async, batch), kBlock,
                                                          sizeof(Shared));
    *blocks_per_sm = a < b ? a : b;
    return e;
}

size_t color_smem_bytes() { return sizeof(Shared); }

cudaError_t launch_validate(const KParams &p, bool batch, int grid, cudaStream_t s)
{
    if (batch) validate_kernel<true><<<grid, 256, 0, s>>>(p);
    else validate_kernel<false><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_check(const KParams &p, bool batch, int grid, cudaStream_t s)
{
    if (batch) check_kernel<true><<<grid, 256, 0, s>>>(p);
    else check_kernel<false><<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_build_lut(const int64_t *vtx_off, int32_t G, int32_t n, int32_t *lut, cudaStream_t s)
{
    const long long chunks = ((long long)n + (1 << kLutShift) - 1) >> kLutShift;
    long long blocks = (chunks + 255) / 256;
    const int grid = (int)(blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks));
    build_lut_kernel<<<grid, 256, 0, s>>>(vtx_off, G, n, lut);
    return cudaGetLastError();
}

}  // namespace gc
