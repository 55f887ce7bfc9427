// Device primitives shared by the kernel translation units of libgc:
// ordered loads and stores, colour accesses, the bounded grid barrier of
// the persistent kernels and the colour statistics taken at their end.
// Each .cu file compiles its own copy (no relocatable device code).
#pragma once

#include "gc_internal.h"

namespace gc {

#define FULL_MASK 0xffffffffu

constexpr unsigned long long kBarrierTimeoutNs = 10000000000ull;  // 10 s
constexpr unsigned kBarrierMaxPolls = 1u << 28;

// ------------------------------------------------------------------------
// memory helpers
// ------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long global_timer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

// Colour loads/stores.  Asynchronous mode reads colours that other threads
// are writing in the same round: relaxed gpu-scope accesses, which are
// coherent (never served from a stale L1 line).  Deterministic mode never
// reads a buffer that is written in the same round; it still bypasses L1
// (.cg) because the buffer was written in an earlier round of this launch.
template <bool ASYNC>
__device__ __forceinline__ int ld_color(const int32_t *p)
{
    if (ASYNC) {
        int v;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
        return v;
    }
    return __ldcg(p);
}

template <bool ASYNC>
__device__ __forceinline__ void st_color(int32_t *p, int v)
{
    if (ASYNC)
        asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
    else
        __stcg(p, v);
}

// ------------------------------------------------------------------------
// grid barrier (bounded)
// ------------------------------------------------------------------------

// All nblocks blocks must be co-resident (cooperative launch).  A block that
// waits longer than timeout_ns (default 10 s) sets GC_EW_TIMEOUT and leaves; the
// caller checks the error word after every barrier.
// sleep_ns: pause between polls; a long one where the grid waits for one
// block's serial work keeps the polls from crowding that block's L2 traffic.
static __device__ void grid_sync(DevState *st, unsigned nblocks, unsigned long long timeout_ns = kBarrierTimeoutNs,
                                 unsigned sleep_ns = 64)
{
    // Arrival is a release (the block's writes, ordered before thread 0 by
    // the block barrier, become visible with it) and the wait an acquire;
    // the last block resets the count before it releases the next
    // generation, so no block arrives at the next barrier before the reset.
    __syncthreads();
    if (threadIdx.x == 0) {
        if (nblocks > 1) {
            const unsigned gen = ld_acquire_u32(&st->bar_gen);
            unsigned arrived;
            asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&st->bar_count) : "memory");
            if (arrived + 1u == nblocks) {
                asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&st->bar_count) : "memory");
                st_release_u32(&st->bar_gen, gen + 1u);
            } else {
                unsigned long long t0 = global_timer();
                unsigned polls = 0;
                while (ld_acquire_u32(&st->bar_gen) == gen) {
                    __nanosleep(sleep_ns);
                    if (++polls > kBarrierMaxPolls || global_timer() - t0 > timeout_ns) {
                        atomicOr(&st->error, GC_EW_TIMEOUT);
                        break;
                    }
                }
            }
        }
    }
    __syncthreads();
}

// Whether a clash of v with u is v's to repair: u keeps its colour (lower
// ids keep by default, higher ids with GC_TIE_HIGHER_KEEPS; no tie-break:
// both repair).
__device__ __forceinline__ bool on_tie_side(int tie, int32_t u, int32_t v)
{
    return tie == TIE_LOWER ? u < v : (tie == TIE_HIGHER ? u > v : true);
}

// ------------------------------------------------------------------------
// colour statistics
// ------------------------------------------------------------------------

// Largest colour and presence bitmap of colours over the grid; the last
// block to finish counts the distinct colours and clears the bitmap for the
// next call (it must be zero on entry).
static __device__ void colour_stats(const int32_t *c, int32_t n, DevState *st, uint32_t *bitmap)
{
    constexpr int kSmemWords = 32;  // colours below 1024 are collected per block first
    __shared__ int acc;
    __shared__ bool last;
    __shared__ int smax;
    __shared__ uint32_t sbm[kSmemWords];
    if (threadIdx.x < kSmemWords) sbm[threadIdx.x] = 0u;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    int mx = 0;
    unsigned long long low = 0;  // colours 0..63, OR-reduced per warp
    bool wrote = false;          // this thread updated the global bitmap
    auto note = [&](int x) {
        mx = max(mx, x);
        if (x >= 0 && x < 64) {
            low |= 1ull << x;
        } else if (x >= 64 && x < kSmemWords * 32) {
            atomicOr(&sbm[x >> 5], 1u << (x & 31));
        } else if (x >= kSmemWords * 32 && x < kStatBitmapWords * 32) {
            atomicOr(&bitmap[x >> 5], 1u << (x & 31));
            wrote = true;
        }
    };
    // eight independent loads in flight per thread (16-byte vectors when the
    // array is 16-byte aligned), then the remainder
    constexpr int kU = 8;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long i = tid;
    if ((reinterpret_cast<uintptr_t>(c) & 15u) == 0) {
        const int4 *c4 = reinterpret_cast<const int4 *>(c);
        const long long n4 = n / 4;
        for (; i + (kU - 1) * stride < n4; i += kU * stride) {
            int4 x[kU];
#pragma unroll
            for (int q = 0; q < kU; ++q) x[q] = __ldcg(c4 + i + q * stride);
#pragma unroll
            for (int q = 0; q < kU; ++q) {
                note(x[q].x);
                note(x[q].y);
                note(x[q].z);
                note(x[q].w);
            }
        }
        for (; i < n4; i += stride) {
            const int4 x = __ldcg(c4 + i);
            note(x.x);
            note(x.y);
            note(x.z);
            note(x.w);
        }
        if (n4 * 4 + tid < n) note(__ldcg(c + n4 * 4 + tid));  // the last n % 4
    } else {
        for (; i + (kU - 1) * stride < n; i += kU * stride) {
            int x[kU];
#pragma unroll
            for (int q = 0; q < kU; ++q) x[q] = __ldcg(c + i + q * stride);
#pragma unroll
            for (int q = 0; q < kU; ++q) note(x[q]);
        }
        for (; i < n; i += stride) note(__ldcg(c + i));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_down_sync(FULL_MASK, mx, o));
        low |= __shfl_down_sync(FULL_MASK, low, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (mx) atomicMax(&smax, mx);
        if (low & 0xffffffffull) atomicOr(&sbm[0], (uint32_t)low);
        if (low >> 32) atomicOr(&sbm[1], (uint32_t)(low >> 32));
    }
    __syncthreads();
    // one warp publishes the block's words and maximum; every thread's own
    // global updates (colours >= 1024) land before the block reports done
    if (threadIdx.x < kSmemWords) {
        if (sbm[threadIdx.x]) atomicOr(&bitmap[threadIdx.x], sbm[threadIdx.x]);
        if (threadIdx.x == 0 && smax) atomicMax(&st->max_color, smax);
    }
    if (wrote || threadIdx.x < kSmemWords) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        last = atomicAdd(&st->stats_done, 1u) == gridDim.x - 1;
        acc = 0;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // Every set bit is a colour <= the largest colour: only the words up to
    // it are read (and cleared).
    const int top = ld_volatile(&st->max_color);
    const int words4 = min(kStatBitmapWords, (top >> 5) + 1 + 3) / 4;
    int s = 0;
    uint4 *bm4 = reinterpret_cast<uint4 *>(bitmap);
#pragma unroll 8
    for (int w = threadIdx.x; w < words4; w += blockDim.x) {  // independent 16-byte loads in flight
        uint4 x = __ldcg(bm4 + w);
        if (x.x | x.y | x.z | x.w) bm4[w] = make_uint4(0u, 0u, 0u, 0u);
        if (w == 0) x.x &= ~1u;  // colour 0 is not a colour
        s += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w);
    }
    atomicAdd(&acc, s);
    __syncthreads();
    if (threadIdx.x == 0) st->distinct = acc;
}

}  // namespace gc
