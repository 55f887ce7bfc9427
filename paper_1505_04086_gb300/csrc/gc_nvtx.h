// NVTX range around an entry point of libgc: named spans on the timeline of
// Nsight Systems / Nsight Compute (header-only NVTX 3; without a tool
// attached a push/pop is a couple of branches).
// A host-only compile without the CUDA headers (the sanitizer build of the
// host form) gets empty ranges.
#pragma once

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GC_HAVE_NVTX 1
#endif

namespace gc {

struct NvtxRange {
#ifdef GC_HAVE_NVTX
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else
    explicit NvtxRange(const char *) {}
#endif
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace gc
