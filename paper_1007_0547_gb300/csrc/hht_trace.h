// NVTX ranges for profilers (Nsight Systems / Compute timelines): one range
// per detection job, per level of the level loop and per kernel launch of the
// host code.  The NVTX calls do nothing unless a tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace hht {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// "level 1" .. "level 24" without formatting at run time.
inline const char* level_name(int s) {
    static const char* const names[] = {"level 0",  "level 1",  "level 2",  "level 3",  "level 4",  "level 5",
                                        "level 6",  "level 7",  "level 8",  "level 9",  "level 10", "level 11",
                                        "level 12", "level 13", "level 14", "level 15", "level 16", "level 17",
                                        "level 18", "level 19", "level 20", "level 21", "level 22", "level 23",
                                        "level 24"};
    return (s >= 0 && s <= 24) ? names[s] : "level";
}

}  // namespace hht
