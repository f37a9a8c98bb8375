// Device-side data of one level and the launch helpers shared by the kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace sww {

// Node/edge flag bits (WASLIVE: live before the adaptation that set the flags).
constexpr uint8_t LIVE = 1, GHOST = 2, COVERED = 4, WASLIVE = 8;
constexpr uint8_t AVAIL = LIVE | GHOST;

// Learned refinement proposal: NF features per patch, NH hidden units; NB
// same-level neighbour patches at most.
constexpr int NF = 8, NH = 32, NB = 24;
constexpr int MLP_PARAMS = NF * NH + NH + NH + 1;   // W1[NF][NH], b1[NH], w2[NH], b2

// Work lists of a level (DevLevelT::wl): ghost nodes, ghost edges, covered nodes,
// edges with a covered end, nodes whose divergence the restriction changes; and the
// level's live-node count, taken in the same pass (wl_n[WL_LIVE]).
constexpr int WL_GN = 0, WL_GE = 1, WL_CN = 2, WL_RE = 3, WL_DN = 4, WL_KINDS = 5, WL_LIVE = 5, WL_WORDS = 6;

// Work-list entry: (level << LVL_SHIFT) | patch; patch == npatch stands for the two poles.
constexpr int LVL_SHIFT = 27;
constexpr int32_t PATCH_MASK = (1 << LVL_SHIFT) - 1;

// Reduction words of a handle: [0] the largest squared CFL frequency (bits of a
// non-negative double), [1] unused, [2] and [3] max |dh| and max |u| over live
// points (bits of non-negative doubles), [RED_LEVEL + j] the largest |u| over the
// live edges of level j (abs_key of the field type), for levels 0..11.
constexpr int RED_LEVEL = 4, RED_WORDS = RED_LEVEL + 12;

// One level on the device, with fields in the working precision R (double, or
// float for the FP32 form).  The spherical geometry (areas, lengths, kites, the
// Coriolis parameter and the TRiSK reconstruction weights) is FP64 in both forms:
// the FP32 form reads the FP64 tables and rounds each value as it enters FP32
// arithmetic.  The transform weights (lifting, velocity prediction, flux
// restriction) are in R (the FP64 tables rounded once for the FP32 form).  All
// arrays are dense over the level (see grid.h for the element layout); slot-major
// tables store slot s of item i at s*count + i.

template <class R>
struct DevLevelT {
    int J;
    int64_t n, p, np, nelem, N, E, T, npatch;
    double dx;                     // Table 1 spacing of the level (m)
    double kx2;                    // (pi / dx)^2, the squared wavenumber of the CFL bound
    double nu;                     // viscosity (m^2/s) of the viscous form; 0: inviscid
    int advect;                    // 1: prescribed velocity (advection test case): u never changes
    // topology
    const int32_t *en, *et;        // [2*E] origin/end node, left/right triangle
    const int32_t *tn, *te;        // [3*T] nodes, side edges (2e + against)
    const uint8_t* deg;            // [N]
    const int32_t *ring_e;         // [6*N] (2e + edge points into the node), -1 padded
    const int32_t* ring_n;         // [6*N] the neighbour across ring edge k, -1 padded
    const int32_t* f2c;            // [N] coarse node at the same place (-1: odd node)
    // geometry (FP64 in every precision form)
    const double *A_i, *A_v, *kite, *d_e, *l_e, *f_v, *f_n;
    const int32_t* cor_i;          // [10*E]
    const double* cor_w;           // [10*E]
    // fine side of the pair (J-1, J)
    const int32_t* par;            // [4*N] prediction parents of odd nodes (fine ids)
    const R* ptw;                  // [4*N] s~_km
    const int8_t* fe_kind;         // [E] 0/1 half of a coarse edge, 2 interior
    const int32_t* fe_ce;          // [E] coarse edge of a half
    const int32_t* vst;            // [12*E] coarse stencil
    const R* vw;                   // [12*E]
    // coarse side of the pair (J, J+1)
    const int32_t *c2f, *mid, *half;  // [N], [E], [2*E]
    const int32_t* mk_i;           // [12*N]
    const R* mk_w;                 // [12*N]
    const int32_t *rf_fi, *rf_ci;  // [12*E], [11*E]
    const R *rf_fw, *rf_cw;
    // patch graph (index npatch is the two poles)
    const int32_t* ppar;           // [npatch+1] patch of level J-1 under each patch (-1 on the coarsest level)
    const int32_t* pnbr;           // [NB*(npatch+1)] patches with a node within two hops, -1 padded
    const int32_t* pchild;         // [4*(npatch+1)] patches of level J+1 over each patch, -1 padded
    // tiles of the structured trend (tile.h): halo ids per patch (null without
    // tiles) and the irregular flag of each patch (index npatch: the poles, 1)
    const int32_t* thalo;          // [npatch * halo]
    const uint8_t* tirr;           // [npatch + 1]
    const R* tgeo;                 // [npatch * geometry block words]: geometry blocks of the regular patches
    // state and work arrays
    R *dh, *u, *dh0, *u0, *dha, *ua, *dht, *ut;
    R *F, *q, *B, *c, *Q;
    R *Fd, *zeta;                  // [E] diffusive height flux, [T] relative vorticity (nu > 0)
    uint8_t *nflag, *eflag, *sig, *tmask, *band0, *band1;
    R *hdet, *ue, *ui;             // [N], [E of level J-1], [E]
    uint8_t* pflag;                // [npatch]
    // learned refinement proposal (per patch)
    float* pfeat;                  // [NF*(npatch+1)] features of the last adaptation
    uint8_t *prop, *prop_prev;     // [npatch+1] proposal for the next / used by the last mask
    uint8_t* pexact;               // [npatch+1] patch holds a point of the exact rules' set
    int32_t* patches;              // [npatch + 1] active patch list (+ pole entry), level-tagged
    int32_t* npatches;             // [1]
    // work lists of the stage's point-wise phases, rebuilt with the active lists
    // (after every adaptation): ghost nodes [N], ghost edges [E], covered nodes [N],
    // edges with a covered end [E], available nodes with a covered node among them and
    // their neighbours [N], at offsets 0, N, N+E, 2N+E, 2N+2E of wl; their counts in
    // wl_n[0..4]; wl_n[WL_LIVE] the level's live nodes
    int32_t* wl;
    int32_t* wl_n;
    // candidate patches of the list-based mask (index npatch: the two poles)
    uint8_t *zflag, *sflag, *cflag, *lflag, *gflag;   // [npatch+1] seeds, significance, candidates,
                                                      //   live nodes, ghost candidates
    int32_t *cand, *ncand;         // [npatch + 1] candidates of the live set (level-tagged), [1]
    int32_t *gcand, *ngcand;       // [npatch + 1] candidates of the ghost band, [1]
};

using DevLevel = DevLevelT<double>;

inline unsigned blocks_for(int64_t n, int t) { return unsigned((n + t - 1) / t); }

}  // namespace sww
