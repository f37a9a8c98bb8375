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
template <class R>
struct WorkT {
    const DevLevelT<R>* lvs;
    const int32_t* list;
    const int32_t* count;
    int S;
    unsigned grid;
};

// Levels ja..jb of a multi-level dense launch; off[j - ja] is the first thread of
// level j and off[jb + 1 - ja] the total.  Level tail_j (-1: none; only ever jb) is a
// tail level of tail_n items covered by a fixed number of striding threads.
struct Span {
    int ja, jb;
    int64_t off[14];
    int tail_j;
    int64_t tail_n;
};

// Arguments of the mask construction over levels ja..jb (ja = Jmin).
template <class R>
struct MaskArgsT {
    const DevLevelT<R>* lvs;    // device array of levels
    const DevLevelT<R>* host;   // the same levels on the host
    int ja, jb, hops;
    const double* thr;          // eps_h, eps_u on the device
    Span nodes_f, edges_f;      // levels ja+1..jb: nodes, edges
    Span nodes, edges;          // levels ja..jb
    Span nodes_c;               // levels ja..jb-1: nodes
    Span patches;               // levels ja..jb: patches
    int32_t* sig_any;           // [sig_any_len] per level: any significant point (device)
    int sig_any_len;
    unsigned tail_blocks;       // blocks of a per-level launch on the tail level
    unsigned long long* lstat;  // learned-proposal counters (misses, over, proposed) or null
};

// Launchers; R = double (FP64 form) or float (FP32 form), instantiated for both.
// list kernels (active patches)
template <class R> void launch_update(const WorkT<R>& W, const RKStage& st, const double* dt, cudaStream_t s);
template <class R> void launch_save_base(const WorkT<R>& W, cudaStream_t s);
template <class R> void launch_fill(const DevLevelT<R>& F, const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s);
// restriction of B, F, q F^perp from level j+1 (F) to level j (C); then the
// divergence of the restricted fluxes at C's nodes
template <class R> void launch_restrict(const DevLevelT<R>& C, const DevLevelT<R>& F, const WorkT<R>& W, cudaStream_t s);
template <class R> void launch_div(const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s);
template <class R> void launch_partial(const DevLevelT<R>& C, const DevLevelT<R>& F, const WorkT<R>& W, cudaStream_t s);
template <class R> void launch_details(const WorkT<R>& W, int jmin, cudaStream_t s);
template <class R> void launch_inverse(const DevLevelT<R>& F, const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s);
template <class R> void launch_maxabs(const WorkT<R>& W, unsigned long long* red, cudaStream_t s);
template <class R> void launch_dt(const WorkT<R>& W, double H, double g, unsigned long long* red, cudaStream_t s);
template <class R>
void launch_dt_final(const DevLevelT<R>* lvs, const unsigned long long* red, double cfl, double* dt, cudaStream_t s);
void launch_thresholds(const unsigned long long* red, double eps, double eh, double eu, int advect, double* thr,
                       cudaStream_t s);

// dense level kernels (masks, initialisation, diagnostics)
template <class R> void launch_restrict_full(const DevLevelT<R>& C, const DevLevelT<R>& F, cudaStream_t s);
// full level F from the full level below (zero coefficients away from live points)
template <class R>
void launch_uniform(const DevLevelT<R>& F, const DevLevelT<R>& C, const R* cdh, const R* cu, R* odh, R* ou,
                    cudaStream_t s);
// WASLIVE := LIVE on the listed patches (inverse transform of the stored coefficients)
template <class R> void launch_mark_support(const WorkT<R>& W, cudaStream_t s);
// significance, adjacency, closure, live flags, ghost band, covered nodes and
// patch lists of levels a.ja..a.jb
template <class R> void launch_mask(const MaskArgsT<R>& a, cudaStream_t s);
// every point of levels nodes.ja..nodes.jb live; covered flags; patch lists
template <class R> void launch_live_all(const DevLevelT<R>* lvs, const Span& nodes, const Span& edges, cudaStream_t s);
template <class R> void launch_covered_all(const DevLevelT<R>* lvs, const Span& nodes_c, cudaStream_t s);
template <class R> void launch_patches_all(const DevLevelT<R>* lvs, const Span& patches, cudaStream_t s);
// the all-level active list from the levels' lists, its entries whose tile is not
// regular (irregular list, same order), and the levels' point work lists (patch
// area P; grid: blocks of the list launch)
template <class R>
void launch_concat(const DevLevelT<R>* lvs, int jmin, int jmax, int32_t* all, int32_t* count, int32_t* irr,
                   int32_t* irr_count, int P, unsigned grid, cudaStream_t s);
template <class R> int sums_blocks(const DevLevelT<R>& L);
template <class R>
void launch_sums(const DevLevelT<R>& L, double H, double g, double* part, double* out, cudaStream_t s);
template <class R> void launch_count(const DevLevelT<R>& L, unsigned long long* cnt, cudaStream_t s);
// y[i] = B(x[i]) (double <-> float)
template <class A, class B> void launch_convert(const A* x, B* y, int64_t n, cudaStream_t s);

// Process-wide number of library kernel launches (count_launch adds launches made
// outside the launchers above).
int64_t kernel_launches();
void count_launch(int64_t n);

}  // namespace sww
