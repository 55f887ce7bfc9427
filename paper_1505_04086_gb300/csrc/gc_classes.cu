// Colour classes: the vertices of a colouring grouped by colour, each group
// in increasing id (a stable counting sort).  Sec. 1 of the paper motivates
// colouring by exactly this use: the vertices of one colour form an
// independent set and can be processed concurrently.
//
// Three steps, all HBM streams: (1) every warp counts the colours of its
// tile of consecutive vertices into a colour-major count matrix
// (count[c-1][tile]); (2) an exclusive scan of that matrix turns it into
// each (colour, tile) pair's first output slot; (3) every warp walks its
// tile again in id order and writes each vertex to its slot, lanes of the
// same colour ranked by lane (warp match), so the order inside a class is
// the id order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gc.h"
#include "gc_ctx.h"
#include "gc_internal.h"
#include "gc_nvtx.h"

namespace gc {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 8;
constexpr int kScanSeg = kScanThreads * kScanPerThread;  // matrix entries per scan block
constexpr long long kMaxMatrix = 1ll << 26;              // count-matrix entries (256 MB)

// (1) count[(c-1) * T + t] = vertices of colour c in tile t (tile = tv
// consecutive ids, one warp per tile).  A colour outside 1..k sets *err.
__global__ void classes_count_kernel(const int32_t *colors, int32_t n, int32_t k, long long T, int tv,
                                     int32_t *count, int *err)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = warp; t < T; t += nwarps) {
        for (int i = 0; i < tv; i += 32) {
            const long long v = t * tv + i + lane;
            int c = v < n ? __ldg(colors + v) : 0;
            if (v < n && (c < 1 || c > k)) {
                atomicOr(err, 1);
                c = 0;
            }
            const unsigned peers = __match_any_sync(kFull, c);
            if (c > 0 && lane == __ffs(peers) - 1) atomicAdd(count + (long long)(c - 1) * T + t, __popc(peers));
        }
    }
}

// Block-wide inclusive scan of one value per thread (kScanThreads threads).
__device__ int block_scan_incl(int x, int *warp_sums)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const int before = wid > 0 ? warp_sums[wid - 1] : 0;
    __syncthreads();
    return x + before;
}

// (2a) sums[b] = sum of matrix segment b.
__global__ void __launch_bounds__(kScanThreads) classes_seg_sum_kernel(const int32_t *m, long long len, int32_t *sums)
{
    __shared__ int warp_sums[32];
    const long long base = (long long)blockIdx.x * kScanSeg + (long long)threadIdx.x * kScanPerThread;
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) s += base + j < len ? m[base + j] : 0;
    const int tot = block_scan_incl(s, warp_sums);
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = tot;
}

// (2b) exclusive scan of the segment sums, in place (one block).
__global__ void __launch_bounds__(kScanThreads) classes_sums_scan_kernel(int32_t *sums, long long nseg)
{
    __shared__ int warp_sums[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b0 = 0; b0 < nseg; b0 += kScanThreads) {
        const long long b = b0 + threadIdx.x;
        const int x = b < nseg ? sums[b] : 0;
        const int incl = block_scan_incl(x, warp_sums);
        const int c0 = carry;
        if (b < nseg) sums[b] = c0 + incl - x;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c0 + incl;
        __syncthreads();
    }
}

// (2c) exclusive scan of the matrix in place; the slot of (colour c, tile
// 0) is where class c starts: class_ptr[c].
__global__ void __launch_bounds__(kScanThreads)
    classes_seg_scan_kernel(int32_t *m, long long len, const int32_t *sums, long long T, int32_t *class_ptr)
{
    __shared__ int warp_sums[32];
    const long long base = (long long)blockIdx.x * kScanSeg + (long long)threadIdx.x * kScanPerThread;
    int v[kScanPerThread];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        v[j] = base + j < len ? m[base + j] : 0;
        s += v[j];
    }
    int run = block_scan_incl(s, warp_sums) - s + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        const long long idx = base + j;
        if (idx < len) {
            m[idx] = run;
            if (idx % T == 0) class_ptr[idx / T + 1] = run;
        }
        run += v[j];
    }
}

// (3) every vertex to its slot, tiles walked in id order by their warp.
__global__ void classes_scatter_kernel(const int32_t *colors, int32_t n, int32_t k, long long T, int tv,
                                       int32_t *slot, int32_t *verts)
{
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long t = warp; t < T; t += nwarps) {
        for (int i = 0; i < tv; i += 32) {
            const long long v = t * tv + i + lane;
            int c = v < n ? __ldg(colors + v) : 0;
            if (c < 1 || c > k) c = 0;  // counted as an error in step (1); written nowhere
            const unsigned peers = __match_any_sync(kFull, c);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (c > 0 && lane == leader) base = atomicAdd(slot + (long long)(c - 1) * T + t, __popc(peers));
            base = __shfl_sync(kFull, base, leader);
            if (c > 0) verts[base + __popc(peers & ((1u << lane) - 1u))] = (int32_t)v;
        }
    }
}

__global__ void classes_bounds_kernel(int32_t *class_ptr, int32_t k, int32_t n)
{
    class_ptr[0] = 0;
    class_ptr[k + 1] = n;
    if (k == 0) class_ptr[1] = n;
}

}  // namespace
}  // namespace gc

extern "C" int gc_color_classes(gc_ctx *c, const int32_t *colors, int32_t n, int32_t num_colors, int32_t *class_ptr,
                                int32_t *class_vertices, void *stream)
{
    gc::NvtxRange nvtx_range("gc_color_classes");
    if (!c || n < 0 || num_colors < 0 || num_colors > GC_CLASSES_MAX_COLORS || !class_ptr ||
        (n > 0 && (!colors || !class_vertices)) || (n > 0 && num_colors < 1))
        return GC_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(c->device) != cudaSuccess) return GC_ERR_CUDA;
    // Tiles of tv vertices (a multiple of 32), wide enough that the count
    // matrix holds at most kMaxMatrix entries.
    long long tv = 256;
    while ((long long)num_colors * ((n + tv - 1) / tv) > gc::kMaxMatrix) tv *= 2;
    const long long T = std::max<long long>((n + tv - 1) / tv, 1);
    const long long len = (long long)num_colors * T;
    const long long nseg = std::max<long long>((len + gc::kScanSeg - 1) / gc::kScanSeg, 1);
    if (!c->cls.reserve((size_t)(len + nseg + 1) * sizeof(int32_t))) return GC_ERR_OOM;
    int32_t *m = c->cls.as<int32_t>();
    int32_t *sums = m + len;
    int *err = sums + nseg;
    cudaError_t e = cudaMemsetAsync(m, 0, (size_t)(len + nseg + 1) * sizeof(int32_t), s);
    const int warps_needed = (int)std::min<long long>(T, (long long)c->num_sms * 64);
    const int grid = std::max(1, (warps_needed * 32 + 255) / 256);
    if (e == cudaSuccess && n > 0) {
        gc::classes_count_kernel<<<grid, 256, 0, s>>>(colors, n, num_colors, T, (int)tv, m, err);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            gc::classes_seg_sum_kernel<<<(unsigned)nseg, gc::kScanThreads, 0, s>>>(m, len, sums);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            gc::classes_sums_scan_kernel<<<1, gc::kScanThreads, 0, s>>>(sums, nseg);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            gc::classes_seg_scan_kernel<<<(unsigned)nseg, gc::kScanThreads, 0, s>>>(m, len, sums, T, class_ptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            gc::classes_scatter_kernel<<<grid, 256, 0, s>>>(colors, n, num_colors, T, (int)tv, m, class_vertices);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && n > 0) {
        gc::classes_bounds_kernel<<<1, 1, 0, s>>>(class_ptr, num_colors, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n == 0) e = cudaMemsetAsync(class_ptr, 0, ((size_t)num_colors + 2) * sizeof(int32_t), s);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
    }
    return herr ? GC_ERR_ARG : GC_OK;
}
