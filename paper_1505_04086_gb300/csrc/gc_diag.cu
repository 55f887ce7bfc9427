// Failure-path checks of the colouring kernels' bounded waits, and the
// gather-rate measurement behind their roofline.  The checks run without
// any GPU fault: the grid barrier (a cooperative launch whose blocks wait for
// one block more than the grid holds, an arrival nothing makes) and, through
// the probe kernel of gc_kernels.cu, the ordered pass's tile wait, the warp
// groups' chunk wait and the staged-copy wait, each against a flag, a
// colour or a copy that never comes.  Every wait must run out, set
// GC_EW_TIMEOUT in the error word and return with the context usable.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "gc.h"
#include "gc_device.cuh"

namespace gc {
namespace {

__global__ void barrier_probe_kernel(DevState *st, unsigned long long timeout_ns)
{
    grid_sync(st, gridDim.x + 1, timeout_ns);
}

// A bijection of [0, mask]: odd multipliers and xor-shifts, each invertible
// modulo a power of two.
__device__ __forceinline__ uint32_t scatter_bits(uint32_t x, uint32_t mask, int half)
{
    x = (x * 0x9E3779B1u) & mask;
    x ^= x >> half;
    x = (x * 0x85EBCA77u) & mask;
    x ^= x >> (half / 2 + 1);
    return x;
}

__global__ void gather_fill_kernel(int32_t *a, uint32_t mask, int half)
{
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x <= mask; x += gridDim.x * blockDim.x)
        a[x] = (int32_t)scatter_bits(x, mask, half);
}

// Independent gathers: positions from a per-thread xorshift32 sequence
// (Marsaglia, 2003), eight loads in flight per thread.
__global__ void gather_indep_kernel(const int32_t *a, uint32_t mask, int rounds, int32_t *sink)
{
    uint32_t h = ((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B9u) | 1u;
    int32_t acc = 0;
    for (int r = 0; r < rounds; ++r) {
        int32_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            h ^= h << 13;
            h ^= h >> 17;
            h ^= h << 5;
            v[q] = __ldcg(a + (h & mask));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += v[q];
    }
    if (acc == 0x7fffffff) *sink = acc;
}

// Dependent gathers: each loaded value (a position, every a[x] <= mask) is
// the next position.
__global__ void gather_chase_kernel(const int32_t *a, uint32_t mask, int steps, int32_t *sink)
{
    uint32_t x = ((blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B1u) & mask;
    for (int s = 0; s < steps; ++s) x = (uint32_t)__ldcg(a + x);
    if (x == 0xffffffffu) *sink = (int32_t)x;
}

}  // namespace
}  // namespace gc

extern "C" int gc_debug_barrier_timeout(int device, int32_t timeout_ms, int32_t *error_word_out)
{
    if (timeout_ms < 1 || timeout_ms > 10000) return GC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    gc::DevState *st = nullptr;
    int word = 0;
    cudaError_t e = cudaMalloc(&st, sizeof(gc::DevState));
    if (e == cudaSuccess) e = cudaMemset(st, 0, sizeof(gc::DevState));
    if (e == cudaSuccess) {
        unsigned long long ns = (unsigned long long)timeout_ms * 1000000ull;
        void *args[] = {&st, &ns};
        e = cudaLaunchCooperativeKernel((const void *)gc::barrier_probe_kernel, dim3(2), dim3(32), args, 0, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&word, &st->error, sizeof(int), cudaMemcpyDeviceToHost);
    if (st) cudaFree(st);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    if (error_word_out) *error_word_out = word;
    return (word & GC_EW_TIMEOUT) ? GC_ERR_TIMEOUT : GC_OK;
}

extern "C" int gc_debug_wait_timeout(int device, int32_t wait, int32_t timeout_ms, int32_t *error_word_out)
{
    if (timeout_ms < 1 || timeout_ms > 10000) return GC_ERR_ARG;
    if (wait == GC_WAIT_GRID_BARRIER) return gc_debug_barrier_timeout(device, timeout_ms, error_word_out);
    if (wait != GC_WAIT_TILE_DONE && wait != GC_WAIT_PIPE_CHUNK && wait != GC_WAIT_STAGE_COPY) return GC_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    // state, a zeroed tile flag, and the 64-vertex graph of the chunk probe:
    // vertex 32's only neighbour is vertex 0 (and back); colours all zero
    constexpr int kN = 64;
    struct Mem {
        gc::DevState st;
        int32_t done[4];
        int32_t row_ptr[kN + 1];
        int32_t col_idx[2];
        int32_t colors[kN];
    };
    Mem h;
    memset(&h, 0, sizeof h);
    for (int v = 0; v <= kN; ++v) h.row_ptr[v] = v == 0 ? 0 : (v <= 32 ? 1 : 2);
    h.col_idx[0] = 32;  // row of vertex 0
    h.col_idx[1] = 0;   // row of vertex 32
    Mem *d = nullptr;
    int word = 0;
    cudaError_t e = cudaMalloc(&d, sizeof(Mem));
    if (e == cudaSuccess) e = cudaMemcpy(d, &h, sizeof(Mem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        gc::KParams p;
        memset(&p, 0, sizeof p);
        p.st = &d->st;
        p.done = d->done;
        p.row_ptr = d->row_ptr;
        p.col_idx = d->col_idx;
        p.cA = d->colors;
        p.n = kN;
        p.nnz = 2;
        p.G = 1;
        p.t1 = 32;
        p.tie = gc::TIE_LOWER;
        e = gc::launch_wait_probe(p, wait, (unsigned long long)timeout_ms * 1000000ull, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&word, &d->st.error, sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    if (error_word_out) *error_word_out = word;
    return (word & GC_EW_TIMEOUT) ? GC_ERR_TIMEOUT : GC_OK;
}

extern "C" int gc_measure_gather_rate(int device, int64_t array_bytes, int32_t blocks_per_sm, int32_t dependent,
                                      double *gloads_per_s_out)
{
    if (array_bytes < 4096 || array_bytes > (1ll << 30) || blocks_per_sm < 1 || blocks_per_sm > 8 ||
        (dependent != 0 && dependent != 1) || !gloads_per_s_out)
        return GC_ERR_ARG;
    int k = 0;  // log2 of the element count
    while ((4ll << (k + 1)) <= array_bytes) ++k;
    const uint32_t mask = (1u << k) - 1u;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_CUDA;
    }
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int32_t *a = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&a, ((size_t)mask + 2) * sizeof(int32_t));  // + the sink
    const bool oom = e == cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    const int grid = sms * blocks_per_sm, threads = 256;
    const long long nthreads = (long long)grid * threads;
    // about 2^28 loads: independent ~1 ms, dependent 2000 steps per thread
    const int rounds = (int)std::max(1ll, (1ll << 28) / (nthreads * 8));
    const int steps = 2000;
    double loads = 0.0;
    float ms = 0.f;
    if (e == cudaSuccess) {
        gc::gather_fill_kernel<<<sms * 4, 256>>>(a, mask, (k + 1) / 2);
        e = cudaGetLastError();
    }
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // warm-up, then the timed launch
        if (rep == 1) e = cudaEventRecord(ev0, 0);
        if (e != cudaSuccess) break;
        if (dependent) gc::gather_chase_kernel<<<grid, threads>>>(a, mask, steps, a + mask + 1);
        else gc::gather_indep_kernel<<<grid, threads>>>(a, mask, rounds, a + mask + 1);
        e = cudaGetLastError();
        if (e == cudaSuccess && rep == 1) e = cudaEventRecord(ev1, 0);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    loads = dependent ? (double)nthreads * steps : (double)nthreads * rounds * 8.0;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (a) cudaFree(a);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return oom ? GC_ERR_OOM : GC_ERR_CUDA;
    }
    *gloads_per_s_out = ms > 0.f ? loads / (ms * 1e-3) / 1e9 : 0.0;
    return GC_OK;
}
