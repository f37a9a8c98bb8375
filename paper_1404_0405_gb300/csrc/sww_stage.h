// Persistent RK stage (sww_stage.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"

namespace sww {

// Arguments of one persistent stage: levels (device array of jmax + 1 records),
// the all-level work list, patch area P, the levels, the constants, the stage
// coefficients and the time step, and the barrier state: STAGE_BAR_WORDS words, zero
// before the first launch (generation word and arrival counters, each in its own
// 128-byte line), err set on a timed-out wait.
constexpr int STAGE_BAR_WORDS = 32 * 18;

template <class R>
struct StageArgs {
    const DevLevelT<R>* lvs;
    const int32_t* all_list;
    const int32_t* all_count;
    int P;
    int jmin, jtop, jmax;
    double H, g;
    RKStage st;
    const double* dt;
    unsigned* bar;
    int* err;
};

// co-resident blocks of the stage kernel on nsm SMs (0 when it cannot run)
template <class R>
unsigned stage_grid(int nsm);
template <class R>
cudaError_t launch_stage(const StageArgs<R>& a, unsigned grid, cudaStream_t s);

}  // namespace sww
