// nx_trace.h -- NVTX ranges of libnavixgb (header-only NVTX 3: a call costs
// a branch on a null function pointer unless a tool such as ncu --nvtx is
// attached).  Calls of the C ABI and their chunk launches are pushed as
// nested ranges on the calling thread; a serving request is one start/end
// range from its admission to its retirement (opened and closed by the
// server's worker thread).
#pragma once
#include <nvtx3/nvToolsExt.h>

struct nx_range {
    explicit nx_range(const char* name) { nvtxRangePushA(name); }
    ~nx_range() { nvtxRangePop(); }
    nx_range(const nx_range&) = delete;
    nx_range& operator=(const nx_range&) = delete;
};
