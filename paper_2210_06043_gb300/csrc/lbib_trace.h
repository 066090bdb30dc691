// lbib_trace.h -- NVTX ranges around the library's entry points (host side).
//
// Each C-ABI call that does work opens a named range for its duration, so a
// profiler that records NVTX (Nsight Systems; ncu with --nvtx and
// --nvtx-include "lbib_advance/") shows which call enqueued which kernels.
// The header-only NVTX v3 API costs a branch per range when no tool is
// attached; without the toolkit's nvtx3 headers the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define LBIB_HAVE_NVTX 1
#endif
#endif

namespace lbib_trace {

struct Range {
    explicit Range(const char* name)
    {
#ifdef LBIB_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range()
    {
#ifdef LBIB_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace lbib_trace

// a range named after the enclosing entry point, closed when it returns
#define LBIB_TRACE(name) const lbib_trace::Range lbib_trace_range_(name)
