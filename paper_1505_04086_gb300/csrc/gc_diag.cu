// Failure-path checks of the colouring kernels' bounded waits, run without
// any GPU fault: the grid barrier (a cooperative launch whose blocks wait for
// one block more than the grid holds, an arrival nothing makes) and, through
// the probe kernel of gc_kernels.cu, the ordered pass's tile wait, the warp
// groups' chunk wait and the staged-copy wait, each against a flag, a
// colour or a copy that never comes.  Every wait must run out, set
// GC_EW_TIMEOUT in the error word and return with the context usable.
#include <cuda_runtime.h>

#include <cstring>

#include "gc.h"
#include "gc_device.cuh"

namespace gc {
namespace {

__global__ void barrier_probe_kernel(DevState *st, unsigned long long timeout_ns)
{
    grid_sync(st, gridDim.x + 1, timeout_ns);
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
