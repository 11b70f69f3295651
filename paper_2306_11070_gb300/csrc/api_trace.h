// Tracing of the C ABI: one NVTX range per call that launches work, free
// unless a profiler is attached (which then shows the calls on the host
// timeline beside the kernels they launch).
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace huff {

struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};

}  // namespace huff

#define HUFF_API_RANGE(name) ::huff::ApiRange huff_api_range_(name)
