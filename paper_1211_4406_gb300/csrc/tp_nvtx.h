// tp_nvtx.h -- host-side profiler annotations of the library's phases.
#pragma once
#include <nvtx3/nvToolsExt.h>

// NVTX ranges around the phases, named after the rows of the paper's Table I
// ("tree construction", "tree traversal", "force calculation") so that a
// profiler's timeline shows them; with no tool attached a range costs a few
// nanoseconds on the host.
struct NvtxRange {
    bool on = true;
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    void end()
    {
        if (on) nvtxRangePop();
        on = false;
    }
    ~NvtxRange() { end(); }
};
