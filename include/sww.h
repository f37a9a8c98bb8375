/*
 * sww.h -- C ABI of the GB300 adaptive wavelet TRiSK shallow-water library.
 *
 * Aechtner, Kevlahan & Dubos, "A conservative adaptive wavelet method for the
 * shallow water equations on the sphere" (arXiv:1404.0405).  The library holds
 * one dynamically adapted, staggered hexagonal C-grid on the icosahedral sphere
 * (levels Jmin..Jmax, Sec. 2.2, Table 1) and advances the rotating shallow-water
 * equations (Sec. 3.1, Eqs. height and velo) with the TRiSK discretisation, the
 * lifting wavelet transforms (Eqs. 1, 2, Rh), the conservative flux restriction
 * (Sec. 4.2-4.3, Eqs. restr_flux, ho_flux, kml) and the threshold-plus-neighbour
 * grid adaptation (Sec. 2.3).  All arithmetic runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *   - Each level j holds N_j = 10*4^j + 2 nodes, E_j = 30*4^j edges and
 *     T_j = 20*4^j triangles in the library's own order (query it with
 *     sww_get_grid).  Heights are the perturbation dh = h - H at nodes (m);
 *     velocities are the component along each edge from its origin node to its
 *     end node (m/s).
 *   - Host arrays are owned by the caller and only read/written during the
 *     call.  Pointers flagged as device pointers must be device memory of the
 *     handle's GPU; they are read in the caller's stream order.
 *   - Every call returns SWW_OK (0) or a negative error code; sww_last_error
 *     gives a message for the last failure on the calling thread.  A failed
 *     call leaves the handle usable unless it returns SWW_E_CUDA.
 *   - A handle is not thread-safe.  Every call is ordered after the work
 *     already queued on the stream given to sww_create, and later work on that
 *     stream is ordered after the call (the library runs its kernels on a stream
 *     of its own, joined to the caller's stream with events).  Calls that
 *     return host data, and sww_step, wait for their own work to finish.
 *   - sww_step replays one CUDA graph per step (captured on first use for each
 *     top level and time-step mode); it reads the new time step and the work-list
 *     sizes back to the host once per step.
 */
#ifndef SWW_H
#define SWW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SWW_OK = 0,
    SWW_E_ARG = -1,      /* invalid argument (bad level, null pointer, bad config) */
    SWW_E_CUDA = -2,     /* a CUDA call failed; the handle should be destroyed */
    SWW_E_POOL = -3,     /* device memory exhausted at creation */
    SWW_E_TIMEOUT = -4,  /* a bounded device wait (a grid barrier of a persistent stage, or a tile's bulk copy) gave up */
    SWW_E_STATE = -5,    /* call out of order (e.g. step before set_state) */
    SWW_E_NUMERIC = -6   /* non-finite value detected in the state */
};

enum { SWW_RK4 = 0, SWW_SSP43 = 1 };

/* Quantities readable per level with sww_get_level (element type in brackets). */
enum {
    SWW_DH = 0,        /* [double N_j]  depth perturbation at nodes                      */
    SWW_U = 1,         /* [double E_j]  velocity along edges                              */
    SWW_DH_T = 2,      /* [double N_j]  last trend d(dh)/dt (valid at live nodes)         */
    SWW_U_T = 3,       /* [double E_j]  last trend du/dt (valid at live edges)            */
    SWW_NODE_FLAGS = 4,/* [uint8 N_j]   bit0 live, bit1 ghost, bit2 covered (R_h applies) */
    SWW_EDGE_FLAGS = 5,/* [uint8 E_j]   bit0 live, bit1 ghost                              */
    SWW_HDET = 6,      /* [double N_j]  height coefficient at odd nodes of level j (0 elsewhere) */
    SWW_UDET_E = 7,    /* [double E_{j-1}] velocity coefficient per coarse edge           */
    SWW_UDET_I = 8,    /* [double E_j]  velocity coefficient at interior fine edges (0 elsewhere) */
    SWW_SIG = 9        /* [uint8 N_j]   significance set of the last adaptation          */
};

enum { SWW_FP64 = 0, SWW_FP32 = 1 };

typedef struct {
    int jmin, jmax;    /* coarsest and finest level, 1 <= jmin <= jmax <= 11           */
    double radius;     /* sphere radius (m)                                            */
    double omega;      /* rotation rate (1/s)                                          */
    double g;          /* gravity (m/s^2)                                              */
    double H;          /* mean depth (m)                                               */
    int patch;         /* patch side p: 4, 8 or 16; levels with 2^j < p use 2^j        */
    int rk;            /* SWW_RK4 or SWW_SSP43                                         */
    double cfl;        /* dt = cfl * min(1/omega_max, min dx/|u|) when dt <= 0         */
    double eps;        /* relative threshold: eps_h = eps*max|dh|, eps_u = eps*max|u| (see regime); 0 keeps every point */
    int blocks_per_sm; /* work-list launches: blocks of 256 threads per SM (0: 4)           */
    int precision;     /* SWW_FP64: fields and arithmetic in FP64.  SWW_FP32: fields,
                          stencils and transforms in FP32; the spherical geometry
                          (areas, lengths, kite areas, Coriolis parameter, TRiSK
                          weights) stays FP64 on the device and is rounded as it
                          enters FP32 arithmetic, the transform weights are the FP64
                          tables rounded once; thresholds, time step and the
                          compensated mass/energy sums in FP64 on the FP32 values.
                          The ABI's double arrays are converted at the boundary.     */
    int persistent;    /* RK stages.  0: one cooperative launch per stage (all phases of
                          the trend and the update, grid barriers between them) for a
                          handle stepping alone, one launch per phase inside
                          sww_step_ensemble (the members' steps then overlap); 3:
                          inside sww_step_ensemble, one regular launch per phase of
                          the step over all members, each member's mask on its own
                          stream (see sww_step_ensemble); -1: one launch per phase
                          always.  Falls back to -1 where the cooperative launch
                          cannot run.  Other values give SWW_E_ARG.                  */
    int mask;          /* 0: mask passes over candidate patches (near the active grid);
                          1: dense passes over every point of the levels (same mask)    */
    double nu;         /* viscosity (m^2/s) of the viscous form (Sec. 3.1): nu div grad dh
                          on the height, nu (grad div u - grad^perp curl u) on the velocity;
                          0: inviscid.  The time step rule has no viscous bound.      */
    int advect;        /* 1: prescribed velocity (the advection test case of Sec. 7.1): the
                          velocity set by sww_set_state (restricted to every level) never
                          changes; the depth h = H + dh is carried by the flux h_e u_e
                          through the same flux restriction, transforms and adaptation.
                          The velocity takes no part in the significance test (eps_u
                          infinite unless passed to sww_adapt), the time step is
                          cfl * min dx/|u| (no gravity waves), and H may be 0.  0: the
                          full shallow-water equations.                                */
    int regime;        /* how eps sets the coefficient thresholds.  0: eps_h = eps max|dh|,
                          eps_u = eps max|u|.  1: eps is the trend tolerance of Sec. 2.3
                          and the thresholds scale as eps^{3/2} (eps*sqrt(eps) in place of
                          eps above), the scaling both regimes of the paper share.     */
} sww_config;

typedef struct {
    double t;                 /* model time (s)                                        */
    double dt;                /* last time step (s)                                    */
    double mass;              /* sum over Jmin of A_k (H + dh_k) (m^3), compensated   */
    double energy;            /* Sec. 7.2 energy on Jmin (m^5/s^2 ... as printed)      */
    double eps_h, eps_u;      /* thresholds of the last adaptation                     */
    int64_t steps;
    int64_t live_nodes[16];   /* per level j (index j), live nodes                     */
    int64_t ghost_nodes[16];
    int64_t live_edges[16];
    int64_t active_patches[16];
    int64_t kernel_launches;  /* library kernel launches so far in this process            */
} sww_stats;

typedef struct sww_handle sww_handle;

/* Build the grid and its geometry for levels Jmin..Jmax (host FP64, uploaded).
 * stream: a cudaStream_t (may be NULL for the default stream).  *out receives
 * the handle, owned by the library until sww_destroy. */
int sww_create(const sww_config* cfg, void* stream, sww_handle** out);
int sww_destroy(sww_handle* h);

/* Ensemble member sharing the grid of `share` (Sec. 2.2: the grid depends only on
 * the levels, the radius and the rotation rate): same as sww_create but the
 * grid and all geometric tables of `share` are reused instead of rebuilt, so a
 * member costs only its state arrays.  cfg must have share's jmin, patch, radius
 * and omega and jmax <= share's jmax; g, H, rk, cfl, eps, blocks_per_sm and
 * precision are free.  Coarse-level areas are those of the shared hierarchy
 * (built up from its finest level, Sec. 4.1), so a member with a smaller jmax
 * matches a grid of its own to rounding, not bit for bit.  The tables stay alive
 * while any handle uses them.  SWW_E_ARG otherwise. */
int sww_create_shared(const sww_config* cfg, void* stream, const sww_handle* share, sww_handle** out);

/* Sizes of level j: nodes, edges, triangles, patches. */
int sww_level_sizes(const sww_handle* h, int level, int64_t* n_nodes, int64_t* n_edges,
                    int64_t* n_tris, int64_t* n_patches);

/* Geometry of level j into host arrays: node_xyz[3*N] unit vectors,
 * edge_nodes[2*E] (origin, end) node ids.  Either pointer may be NULL. */
int sww_get_grid(const sww_handle* h, int level, double* node_xyz, int32_t* edge_nodes);

/* Fields on the full finest level Jmax (dh[N_Jmax], u[E_Jmax]); every coarser
 * level receives their restriction (R_h for height, the mean of the two half
 * edges for velocity) and every point becomes live (Sec. 3.1 initialisation).
 * device_ptrs != 0: dh, u are device pointers. */
int sww_set_state(sww_handle* h, const double* dh, const double* u, int device_ptrs);

/* The same from fields on a full level J in Jmin..Jmax (dh[N_J], u[E_J]): levels
 * Jmin..J receive them and their restrictions and are all live; the levels above
 * J hold no point until adaptation refines into them.  With a prescribed
 * velocity (advect) J must be Jmax (SWW_E_ARG otherwise).  Host fields with a
 * non-finite value are refused (SWW_E_NUMERIC) before the handle's state
 * changes (they are copied into the handle's FP64 staging buffer and checked
 * there); device fields are taken as given. */
int sww_set_state_level(sww_handle* h, int level, const double* dh, const double* u, int device_ptrs);

/* Adapt the grid (Sec. 2.3): wavelet coefficients at live points, thresholds
 * (eps_h, eps_u > 0 given explicitly, else eps times the live maxima),
 * significance, neighbours in space and scale, graded closure, ghost band,
 * patch lists, and the inverse transform of the retained coefficients. */
int sww_adapt(sww_handle* h, double eps_h, double eps_u);

/* Same mask construction from caller-provided coefficients: hdet[N_j] per
 * level j (values at odd nodes), udet_e[E_{j-1}], udet_i[E_j] (interior fine
 * edges), for j = Jmin+1..Jmax in order, host arrays concatenated by level,
 * with explicit thresholds.  Significance uses the current live flags; the new
 * flags, patch lists and the inverse transform of these coefficients onto the
 * new live set replace the current ones (the state changes accordingly). */
int sww_mask_from_coeffs(sww_handle* h, const double* hdet, const double* udet_e,
                         const double* udet_i, double eps_h, double eps_u);

/* Evaluate the trend of the current state (ghosts refreshed, restrictions
 * applied, Sec. 3.1) into the SWW_DH_T / SWW_U_T buffers. */
int sww_rhs(sww_handle* h);

/* Advance nsteps RK steps.  dt <= 0 uses the CFL step of the current state.
 * adapt != 0 runs the partial height transform and sww_adapt after each step;
 * adapt == 0 runs only the partial height transform. */
int sww_step(sww_handle* h, double dt, int nsteps, int adapt);

/* nsteps steps of each of n independent ensemble members (distinct handles, each
 * as sww_step alone would advance it, bit for bit).  By default every member's
 * step runs on the member's own stream, so the members' kernels overlap on the
 * GPU and each member waits only for its own previous step; with more than one
 * member the RK stages then run as one launch per phase (cooperative launches of
 * different streams do not overlap).  When every member has persistent = 3 and
 * they share precision, Jmin, patch, H, g and scheme (at most 128 members),
 * every phase of the step but the mask (time step, RK base, stage phases,
 * partial transform, ghosts, coefficients, thresholds, inverse transform,
 * read-back) is one regular launch over all members on the first member's
 * stream; each member's mask runs on its own stream in between.
 * On entry each member's work is ordered after its caller stream, and on return
 * each caller stream waits for its member.  Returns the first error; members
 * then stand at different step counts (sww_stats_get tells which). */
int sww_step_ensemble(sww_handle* const* hs, int n, double dt, int nsteps, int adapt);

/* Copy one per-level quantity (SWW_DH ... SWW_SIG) to the host. */
int sww_get_level(const sww_handle* h, int level, int what, void* out);

/* The adapted grid of level j (Sec. 2.3): node flags nodes[N_j] and edge flags
 * edges[E_j] as in SWW_NODE_FLAGS / SWW_EDGE_FLAGS (bit 0 live, bit 1 ghost,
 * bit 2 covered); either pointer may be null. */
int sww_get_mask(const sww_handle* h, int level, uint8_t* nodes, uint8_t* edges);

/* Write the depth perturbation and velocity of level j (host arrays). */
int sww_set_level(sww_handle* h, int level, const double* dh, const double* u);

/* Forward wavelet transform of the active grid (Eqs. 1-2 and the velocity
 * transform of Sec. 4.1): the coefficients of every live point above Jmin into
 * the coefficient buffers (h~ at odd nodes, the pair coefficient per coarse edge,
 * u~ at interior fine edges), read with sww_get_coeffs.  The state is unchanged. */
int sww_forward(sww_handle* h);

/* Inverse wavelet transform onto the current live set, coarse to fine: the live
 * points of each level above Jmin are rebuilt from the level below and the
 * stored coefficients of live points (set by sww_forward, sww_adapt or
 * sww_set_coeffs), ghosts refilled.  Inverse after forward returns the state to
 * rounding.  A prescribed velocity (advect) is left as set. */
int sww_inverse(sww_handle* h);

/* Coefficients of level j > Jmin: hdet[N_j] (values at odd nodes, 0 elsewhere),
 * udet_e[E_{j-1}], udet_i[E_j] (interior fine edges); any pointer may be null.
 * sww_get_coeffs copies them to the host, sww_set_coeffs writes them for the
 * next sww_inverse.  SWW_E_ARG for j = Jmin. */
int sww_get_coeffs(const sww_handle* h, int level, double* hdet, double* udet_e, double* udet_i);
int sww_set_coeffs(sww_handle* h, int level, const double* hdet, const double* udet_e, const double* udet_i);

/* The state on the full level j (dh[N_j], u[E_j], host arrays; either may be
 * null): live points keep their values, every other point is the inverse
 * transform with zero coefficients of the full level j-1, recursively from Jmin
 * (Sec. 2.2).  Uses the RK base arrays as scratch, so it runs between steps only
 * (as every call does). */
int sww_get_state(sww_handle* h, int level, double* dh, double* u);

/* Checkpoint / resume.  sww_save writes the model time, step count, last dt and
 * thresholds, and per level the depth, velocity (working precision, ghosts
 * included) and node/edge flags to a binary file (little-endian as written by
 * this host: "SWWCKPT1", a fixed header, the levels Jmin..Jmax, "SWWCKEND").
 * sww_load reads one into a handle of the same Jmin, Jmax, patch, radius, omega
 * and precision (else SWW_E_ARG; other settings are the handle's own), clears
 * the per-adaptation scratch and rebuilds the patch lists; stepping then
 * continues as the saved handle would, bit for bit.  A truncated or foreign file
 * is SWW_E_ARG and leaves the handle unchanged. */
int sww_save(const sww_handle* h, const char* path);
int sww_load(sww_handle* h, const char* path);

/* Active patch list of level j (ascending patch ids) into out[n_patches];
 * *count receives its length. */
int sww_get_patches(const sww_handle* h, int level, int32_t* out, int32_t* count);

/* Live nodes over every level (the adapted grid's size, Sec. 2.3), as of the
 * handle's last call that set its mask (sww_set_state, sww_set_state_level,
 * sww_adapt, sww_mask_from_coeffs, sww_step, sww_step_ensemble, sww_load): the
 * count those calls already brought back with their read-back, so this call does
 * no device work and does not synchronise.  *total is 0 before the first state is
 * set.  SWW_E_ARG for a null argument. */
int sww_live_nodes(const sww_handle* h, int64_t* total);

/* Diagnostics (synchronises the stream). */
int sww_stats_get(sww_handle* h, sww_stats* st);

/* Kernel classes timed by the tracing hook below. */
enum {
    SWW_K_TREND = 0,     /* the structured trend of every active patch: F, q, div F,
                            K, B, q F^perp of the regular tiles, F and q elsewhere   */
    SWW_K_IRREG = 1,     /* div F, K, B and q F^perp at the irregular patches        */
    SWW_K_NODE = 2,      /* divergence of the restricted fluxes at coarse nodes      */
    SWW_K_RESERVED = 3,  /* (no launches)                                            */
    SWW_K_RESTRICT = 4,  /* restriction of B, F and q F^perp                         */
    SWW_K_UPDATE = 5,    /* trends and Runge-Kutta stage combination                 */
    SWW_K_FILL = 6,      /* ghost prolongation                                       */
    SWW_K_PARTIAL = 7,   /* partial height transform                                 */
    SWW_K_COEFF = 8,     /* wavelet coefficients                                     */
    SWW_K_MASK = 9,      /* thresholds, significance, closure, ghosts, patches       */
    SWW_K_INVERSE = 10,  /* inverse transform onto the new mask                      */
    SWW_K_DT = 11,       /* CFL time step reduction                                  */
    SWW_K_STAGE = 12,    /* persistent RK stage (trend and update in one launch)     */
    SWW_K_NCLASS = 13
};

/* Tracing: from now on record a pair of CUDA events on the library's stream
 * around every launch group of the kernel classes whose bit is set in class_mask
 * (bit k for class k); 0 stops recording.  Previous records are discarded.  While
 * any class is traced, sww_step runs its kernels directly instead of replaying
 * the captured graph.  In sww_step_ensemble with batched stages (persistent 3)
 * the first member's records cover the batched launches of all members
 * (SWW_K_STAGE per RK stage, SWW_K_DT for the time step and RK base,
 * SWW_K_PARTIAL for the partial transform and ghosts after the stages). */
int sww_profile(sww_handle* h, uint32_t class_mask);

/* Fault injection for tests of the bounded grid barrier of the persistent RK
 * stage (no counterpart in the paper).  Every barrier wait of the handle's later
 * persistent stages (and their waits for a patch's geometry copy) gives up after
 * spin_cycles SM clock cycles (0: the default, about 2 s),
 * sets the handle's error flag and lets the stage kernel return; the step then
 * returns SWW_E_TIMEOUT without advancing t, and the barrier state is reset so
 * that the next step runs normally.  skip_block >= 0 makes that block of each
 * persistent stage leave at its first barrier without arriving, so that the other
 * blocks' waits run out (-1: no block skips).  Synchronises the handle's stream and
 * drops its captured steps.  SWW_E_ARG for a null handle or spin_cycles < 0. */
int sww_barrier_fault(sww_handle* h, long long spin_cycles, int skip_block);

/* Sum of the recorded durations (ms[SWW_K_NCLASS]) and of the kernel launches
 * inside the records (launches[SWW_K_NCLASS]) per class since sww_profile;
 * synchronises the stream and clears the records (recording continues). */
int sww_profile_read(sww_handle* h, double* ms, int64_t* launches);

/* Mass and energy of the Jmin level (the same two numbers sww_stats_get reports)
 * computed without allocating any device memory.  The paper has no counterpart
 * for this call: it exists for callers that cannot allocate device memory when
 * they ask for the diagnostics -- code inside a framework whose caching
 * allocator owns the device heap, real-time loops where the implicit
 * synchronisation of cudaMalloc/cudaFree is not allowed, or hosts that hand the
 * library only the buffers it may touch.
 *   dh[N_Jmin], u[E_Jmin]: device arrays (caller-owned) of the Jmin depth
 *     perturbation and velocity, in the library's order.
 *   out[2]: device array (caller-owned) that receives mass (m^3) and energy.
 * The per-block partial sums go to a fixed 128 KiB device array inside the
 * library (resident on every GPU that loads it, until the process exits), which
 * bounds N_Jmin to 1,048,576 nodes (Jmin <= 8); larger levels return SWW_E_ARG.
 * dh, u and out must be device or managed memory (checked with
 * cudaPointerGetAttributes; SWW_E_ARG otherwise); their lengths cannot be seen
 * here, so the caller guarantees N_Jmin, E_Jmin and 2 values.
 * The call is asynchronous on the caller's stream given to sww_create (dh, u
 * and out are read and written in that stream's order) and makes no cudaMalloc,
 * cudaFree or other allocating call.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the process;
 * make that first call before any stream capture, and do not use the call on a
 * device after a cudaDeviceReset of it.  Every call reuses the same array:
 * calls whose work may overlap on the GPU (other streams, other handles on the
 * same device) race.  A CUDA error already pending when the call starts gives
 * SWW_E_CUDA before any launch. */
int sww_mass_energy_static(sww_handle* h, const double* dh, const double* u, double* out);

/* ---------------------------------------------------------------------------
 * Learned refinement proposal (an extension: the paper's criterion is the
 * threshold rule of Sec. 2.3, which keeps the last word).
 *
 * After the coefficients and thresholds of an adaptation, each patch of the
 * levels above Jmin that hold active patches gets SWW_MLP_FEATURES features:
 *   0 log2(1 + max|h~|/eps_h) over its live odd nodes
 *   1 log2(1 + max|u~|/eps_u) over its live interior edges and the pair
 *     coefficients of the coarse edges under its even nodes
 *   2, 3  features 0, 1 of the coarse patch under it (0 on the level above Jmin)
 *   4, 5  maxima of features 0, 1 over its neighbour patches
 *   6 fraction of its nodes that are live
 *   7 (level - Jmin) / (Jmax - Jmin)
 * A two-layer perceptron (SWW_MLP_HIDDEN ReLU units; BF16 weights, FP32
 * accumulation) maps them to the probability that the exact rules will need the
 * patch at the next adaptation; a patch that is not active yet and scores above
 * tau is proposed (a refinement ahead of the exact rules), and all its nodes
 * join the set T of the mask (Sec. 2.3) before the graded closure, so the mask is
 * the exact one plus the proposed patches.  Parameters (FP32 masters, rounded to
 * BF16 for use): W1[F][H] row-major, b1[H], w2[H], b2. */
enum { SWW_MLP_FEATURES = 8, SWW_MLP_HIDDEN = 32, SWW_MLP_PARAMS = 8 * 32 + 32 + 32 + 1 };
enum { SWW_MLP_WORK = 256 * (SWW_MLP_PARAMS + 1) };   /* floats of the gradient work buffer */
enum { SWW_P_FEATURES = 0, SWW_P_EXACT = 1, SWW_P_PROPOSAL = 2, SWW_P_ACTIVE = 3 };

/* mode 0: off; 1: compute the features at every adaptation (for training data);
 * 2: features and proposal with params (host [SWW_MLP_PARAMS]) and 0 < tau < 1.
 * Drops the handle's captured step graphs. */
int sww_set_learned(sww_handle* h, int mode, const float* params, float tau);

/* Explicit proposal for the next adaptation only: flags[n_patches + 1] (host; the
 * last entry is the two poles) of level j > Jmin.  A learned proposal (mode 2)
 * replaces it on the levels the perceptron covers. */
int sww_propose(sww_handle* h, int level, const uint8_t* flags);

/* Per-patch data of level j into host memory:
 *   SWW_P_FEATURES float[SWW_MLP_FEATURES * (n_patches + 1)], feature-major
 *                  (feature f of patch P at f * (n_patches + 1) + P), last adaptation;
 *   SWW_P_EXACT    uint8[n_patches + 1]: the patch holds a point of the exact
 *                  rules' set T of the last mask;
 *   SWW_P_PROPOSAL uint8[n_patches + 1]: proposal applied by the last mask;
 *   SWW_P_ACTIVE   uint8[n_patches]: active patches (live or ghost point). */
int sww_get_patch_data(const sww_handle* h, int level, int what, void* out);

/* Cumulative counts since the last reset, over all levels above Jmin:
 * out[0] misses: patches the exact set reached that were not active during the
 * step before (late refinements); out[1] over-refined: patches the previous
 * proposal named that hold none of the exact set; out[2] proposed patches. */
int sww_learn_stats(sww_handle* h, int64_t* out, int reset);

/* Training kernels on device arrays (stream: the caller's).  X[n][F] features, y[n]
 * labels in {0, 1}, params[SWW_MLP_PARAMS] FP32 masters.  loss_grad writes the mean
 * weighted binary cross-entropy (positive class weight pos_weight) and its gradient:
 * out[0..SWW_MLP_PARAMS) = d loss / d params (through the BF16 rounding, passed
 * straight through), out[SWW_MLP_PARAMS] = loss; work holds SWW_MLP_WORK floats.
 * adam: one Adam update (beta 0.9, 0.999, eps 1e-8) of params with step count t >= 1
 * and moments m, v.  predict: p[n] = sigmoid(logit). */
int sww_mlp_loss_grad(const float* X, const float* y, int64_t n, const float* params, float pos_weight, float* work,
                      float* out, void* stream);
int sww_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, void* stream);
int sww_mlp_predict(const float* X, int64_t n, const float* params, float* p, void* stream);

/* Message of the last error on the calling thread. */
int sww_last_error(char* buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif
