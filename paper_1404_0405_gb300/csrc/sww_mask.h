// List-based mask construction (sww_mask.cu), for one handle or for every member
// of an ensemble in the same launches.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_learn.h"

namespace sww {

// One member's mask: its levels, the all-level active list of the grid before the
// mask, the candidate lists (built into the levels' cand/gcand arrays and
// concatenated into cand/gcand), the rebuilt all-level and irregular lists, its
// thresholds and counters.  Levels Jmin..jb take part (jb = min(top + 1, jmax)).
template <class R>
struct MaskMember {
    const DevLevelT<R>* lvs;             // device array of levels 0..jmax
    const int32_t* active;               // all-level active list before the mask
    const int32_t* active_count;
    int32_t *cand, *cand_count, *gcand, *gcand_count;
    int32_t *all, *all_count, *irr, *irr_count;
    const double* thr;                   // eps_h, eps_u
    int32_t* sig_any;                    // [jmax + 2] per level: a significant point or a proposed patch
    unsigned long long* lstat;           // learned-proposal counters (misses, over, proposed) or null
    const MlpWeights* net;               // device weights of the proposal (learn == 2)
    float logit_tau;                     // proposal threshold on the logit
    int learn;                           // 0 off, 1 features only, 2 features and proposal
    int jb, jmax;
};

// The members of one mask launch sequence (by value in every launch: CAP members
// at most) and what they share: patch area P, Jmin, the largest jb and jmax, the
// ghost band's hops, candidate rings, and the patch spans of the levels (the
// members share one grid): levels ja..jb_max, ja+1..jb_max, ja+1..jmax_max.
template <class R, int CAP>
struct MaskBatch {
    int nm, P, ja, jb_max, jmax_max, hops, rings;
    Span patches, patches_f, props;
    MaskMember<R> m[CAP];
};

constexpr int MASK_BATCH_MAX = 128;

// significance, proposal, candidates, closure, live flags, ghost band, covered
// nodes, patch flags and lists, and the all-level and irregular lists of every
// member (grid: blocks per member of the list launches)
template <class R, int CAP>
void launch_mask_batch(const MaskBatch<R, CAP>& b, unsigned grid, cudaStream_t s);
// the learned proposal's features and proposal (members with learn > 0) and the
// proposal roll before a mask (post 0) or after it (post 1)
template <class R, int CAP>
void launch_proposal_batch(const MaskBatch<R, CAP>& b, unsigned grid, int post, cudaStream_t s);
// the all-level and irregular lists of every member from its level lists, and the
// levels' point work lists (grid: blocks per member of the list launch)
template <class R, int CAP>
void launch_concat_batch(const MaskBatch<R, CAP>& b, unsigned grid, cudaStream_t s);

}  // namespace sww
