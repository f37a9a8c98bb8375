// List-based mask construction (sww_mask.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"

namespace sww {

// Arguments of the mask over levels ja..jb (ja = Jmin) from the active list of the
// grid before it: candidate lists are built into the levels' cand/gcand arrays
// and concatenated into cand/gcand (device arrays of max_entries entries).
template <class R>
struct MaskListArgs {
    const DevLevelT<R>* lvs;           // device array of levels
    const DevLevelT<R>* host;          // the same levels on the host
    const unsigned* grid_lv;           // per-level fixed grids (host)
    int ja, jb, hops, rings, P;
    unsigned grid;                     // fixed grid of multi-level list launches
    int64_t max_entries;               // patches (+ pole entries) of levels ja..jb
    const int32_t* active;             // all-level active list of the grid before the mask
    const int32_t* active_count;
    const double* thr;                 // eps_h, eps_u
    int32_t* sig_any;
    Span patches;                      // levels ja..jb: patches + pole entry
    int32_t *cand, *cand_count, *gcand, *gcand_count;
    unsigned long long* lstat;         // learned-proposal counters or null
};

template <class R>
void launch_mask_lists(const MaskListArgs<R>& a, cudaStream_t s);

}  // namespace sww
