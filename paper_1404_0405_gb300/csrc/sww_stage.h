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
    const int32_t* irr_list;    // entries of all_list whose tile is not regular
    const int32_t* irr_count;
    int P;
    int jmin, jtop, jmax;
    double H, g;
    RKStage st;
    const double* dt;
    unsigned* bar;
    int* err;
    // bounded barrier waits: a wait gives up after `spin` clock cycles (<= 0: the
    // default, about 2 s); block `skip` (fault injection for tests, -1: none) leaves
    // at the first barrier without arriving, so the others' waits run out
    long long spin = 0;
    int skip = -1;
};

// One member of an ensemble stage: its level records (contiguous, levels 0..jmax),
// its all-level active list, its time step and its top level.
template <class R>
struct MemberRef {
    const DevLevelT<R>* lvs;
    const int32_t* all_list;
    const int32_t* all_count;
    double* dt;
    int jtop;
    unsigned long long* red;   // [RED_WORDS] reduction words (CFL step, live maxima; see RED_WORDS)
    double cfl;
    // adaptation (batched phases around the members' own masks)
    double* thr;               // [2] thresholds eps_h, eps_u
    double eps_c;              // relative coefficient tolerance (eps, or eps^{3/2})
    int advect;                // prescribed velocity: no velocity threshold
    int j1;                    // top level of the inverse transform (min(jtop + 1, jmax))
    int jmax;
    int* err;                  // error flag of the member's bounded waits (barriers, bulk copies)
    const int32_t* irr_list;   // entries of all_list whose tile is not regular
    const int32_t* irr_count;
};

// One RK stage of nm members (m: device array of nm refs, nm <= 128) with a common
// patch area P, Jmin, mean depth H and gravity g.
template <class R>
struct BatchArgs {
    const MemberRef<R>* m;
    int nm, P, jmin, jtop_max;
    double H, g;
    RKStage st;
    unsigned* bar;
    int* err;
    double dt_given;   // phases before the stages: > 0 sets every member's time step
    void* out;         // read-back records, one per member (BatchOut, below)
};

// Read-back record of one member after a batched step: dt, the error flag, and the
// active patch count and the live nodes of each level 0..15.
struct BatchOut {
    double dt;
    int32_t err;
    int32_t counts[16];
    int32_t live[16];   // live nodes of each level
    int32_t pad;
};
static_assert(sizeof(BatchOut) == 144, "read-back record size (the Python binding's BATCH_OUT_BYTES)");

// co-resident blocks of the stage kernel for patch area P on nsm SMs (0 when it
// cannot run)
template <class R>
unsigned stage_grid(int P, int nsm);
template <class R>
cudaError_t launch_stage(const StageArgs<R>& a, unsigned grid, cudaStream_t s);
// words of the geometry block of one tile of side `side` (4, 8 or 16; 0 otherwise)
template <class R>
size_t tile_geo_words(int side);
// the geometry blocks of L's regular patches into out ([npatch * words], zeroed by
// the caller), for tiles of side `side` (sww_tile.cu)
template <class R>
cudaError_t build_tile_geo(const DevLevelT<R>& L, int side, R* out, cudaStream_t s);
// The trend of a stage over all members (sww_tile.cu): the structured kernel over
// every active patch (parts bit 0), then the tabulated node and Coriolis bodies
// over the irregular patches (bit 1).  entries and irr_entries bound the members'
// all-level and irregular list entries in total.
template <class R>
cudaError_t launch_tile_trend(const BatchArgs<R>& a, int64_t entries, int64_t irr_entries, int nsm, int parts,
                              cudaStream_t s);
// One RK stage as one regular launch per phase over all members (level-serial
// phases once per level); level_entries[j] bounds the members' level-j list
// entries in total, irr_entries their irregular entries (for the grid sizes).
template <class R>
cudaError_t launch_stage_batch_phases(const BatchArgs<R>& a, const int64_t* level_entries, int64_t irr_entries, int nsm,
                                      cudaStream_t s);
// The same stage in parts: 0 the ghosts, 1 the structured trend, 2 the irregular
// patches, 3 the restrictions and divergences level by level, 4 the update.
template <class R>
cudaError_t launch_stage_batch_part(const BatchArgs<R>& a, const int64_t* level_entries, int64_t irr_entries, int nsm,
                                    int part, cudaStream_t s);
// Before the stages of a step, over all members: the RK base copy and the time
// step (dt > 0 for every member, else each member's CFL step).
template <class R>
cudaError_t launch_batch_pre(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, double dt, cudaStream_t s);
// After the stages: the partial height transform (top-1 down to Jmin) and the
// ghosts (Jmin+1 up to the top) of every member.
template <class R>
cudaError_t launch_batch_post(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, cudaStream_t s);
// Before the members' masks: wavelet coefficients, live maxima and thresholds.
template <class R>
cudaError_t launch_batch_adapt_pre(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, cudaStream_t s);
// After them: the inverse transform and ghosts, level by level up to each
// member's j1 (level_entries up to the largest j1).
template <class R>
cudaError_t launch_batch_adapt_post(const BatchArgs<R>& a, const int64_t* level_entries, int j1_max, int nsm,
                                    cudaStream_t s);
// The read-back records (BatchOut) of every member into a.out.
template <class R>
cudaError_t launch_batch_out(const BatchArgs<R>& a, cudaStream_t s);

}  // namespace sww
