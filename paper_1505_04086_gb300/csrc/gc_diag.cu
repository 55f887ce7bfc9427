// Failure-path check of the persistent kernels' bounded grid barrier: a
// cooperative launch whose blocks wait for one block more than the grid
// holds (an arrival nothing makes), so the wait runs out, the error word
// gets GC_EW_TIMEOUT and the kernel returns with the context usable.
#include <cuda_runtime.h>

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
