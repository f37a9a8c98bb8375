// Host-side launchers of the kernels in sww_kernels.cu.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "sww_core.cuh"

namespace sww {

// One Runge-Kutta stage: y <- a*y0 + b*y + (cdt*dt)*k + (ddt*dt)*acc, acc <- al*acc + be*k.
// apply == 0 only stores the trend k.
struct RKStage {
    int apply;
    double a, b, cdt, ddt, al, be;
};

// A work list on the device: entries (level-tagged patches), their count, the
// device array of levels (for multi-level lists; null for a single level's list),
// threads per entry S (the configured patch area) and the fixed grid size.
struct Work {
    const DevLevel* lvs;
    const int32_t* list;
    const int32_t* count;
    int S;
    unsigned grid;
};

// Levels ja..jb of a multi-level dense launch; off[j - ja] is the first thread of
// level j and off[jb + 1 - ja] the total.
struct Span {
    int ja, jb;
    int64_t off[14];
};

// Arguments of the mask construction over levels ja..jb (ja = Jmin).
struct MaskArgs {
    const DevLevel* lvs;    // device array of levels
    const DevLevel* host;   // the same levels on the host
    int ja, jb, hops;
    const double* thr;      // eps_h, eps_u on the device
    Span nodes_f, edges_f;  // levels ja+1..jb: nodes, edges
    Span nodes, edges;      // levels ja..jb
    Span nodes_c;           // levels ja..jb-1: nodes
    Span patches;           // levels ja..jb: patches
    int32_t* sig_any;       // [sig_any_len] per level: any significant point (device)
    int sig_any_len;
    int skip;               // level above the top live level (-1: none)
};

// list kernels (FP64, active patches)
void launch_pv_flux(const Work& W, double H, cudaStream_t s);
void launch_node_coriolis(const Work& W, double g, cudaStream_t s);
void launch_update(const Work& W, const RKStage& st, const double* dt, cudaStream_t s);
void launch_save_base(const Work& W, cudaStream_t s);
void launch_fill(const DevLevel& F, const DevLevel& C, const Work& W, cudaStream_t s);
void launch_restrict(const DevLevel& C, const DevLevel& F, const Work& W, cudaStream_t s);
void launch_partial(const DevLevel& C, const DevLevel& F, const Work& W, cudaStream_t s);
void launch_details(const Work& W, int jmin, cudaStream_t s);
void launch_inverse(const DevLevel& F, const DevLevel& C, const Work& W, cudaStream_t s);
void launch_maxabs(const Work& W, unsigned long long* red, cudaStream_t s);
void launch_dt(const Work& W, double H, double g, unsigned long long* red, cudaStream_t s);
void launch_dt_final(const unsigned long long* red, double cfl, double* dt, cudaStream_t s);
void launch_thresholds(const unsigned long long* red, double eps, double eh, double eu, double* thr, cudaStream_t s);

// dense level kernels (masks, initialisation, diagnostics)
void launch_restrict_full(const DevLevel& C, const DevLevel& F, cudaStream_t s);
// significance, adjacency, closure, live flags, ghost band, covered nodes and
// patch lists of levels a.ja..a.jb
void launch_mask(const MaskArgs& a, cudaStream_t s);
// every point of levels nodes.ja..nodes.jb live; covered flags; patch lists
void launch_live_all(const DevLevel* lvs, const Span& nodes, const Span& edges, cudaStream_t s);
void launch_covered_all(const DevLevel* lvs, const Span& nodes_c, cudaStream_t s);
void launch_patches_all(const DevLevel* lvs, const Span& patches, cudaStream_t s);
void launch_concat(const DevLevel* lvs, int jmin, int jmax, int32_t* all, int32_t* count, cudaStream_t s);
int sums_blocks(const DevLevel& L);
void launch_sums(const DevLevel& L, double H, double g, double* part, double* out, cudaStream_t s);
void launch_count(const DevLevel& L, unsigned long long* cnt, cudaStream_t s);

// Process-wide number of library kernel launches (count_launch adds launches made
// outside the launchers above).
int64_t kernel_launches();
void count_launch(int64_t n);

}  // namespace sww
