// A named NVTX range over a C++ scope, for the host-side stages of the library
// (sources, stencil time steps, Jacobian / Hessian reduction, log-det and sum, a
// served request).  It brackets the enqueueing of a stage, which a profiler's
// timeline lines up with the stage's kernels.  NVTX v3 is header-only: without a
// profiler attached, push and pop return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace oed {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace oed
