// C ABI (include/sww.h): handle lifetime, upload of the host-built grid, and the
// sequencing of kernels for one trend evaluation, one RK step and one adaptation.
//
// The library issues its work on a stream of its own, joined to the caller's
// stream with events at the start and end of every call.  A step is captured once
// as a CUDA graph per (top level, time-step mode) and replayed; the only host
// round trip per step reads the new time step and the per-level work-list sizes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <tuple>
#include <type_traits>
#include <vector>

#include "grid.h"
#include "sww.h"
#include "sww_core.cuh"
#include "sww_internal.h"
#include "sww_kernels.h"
#include "sww_learn.h"
#include "sww_stage.h"
#include "sww_mask.h"

using namespace sww;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

struct CudaError : std::runtime_error {
    using std::runtime_error::runtime_error;
};

void ck(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw CudaError(std::string(what) + ": " + cudaGetErrorString(e));
}

__global__ void k_set(double* p, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// reduction words of the time step (see RED_WORDS): the maxima start at zero
__global__ void k_reset_red(unsigned long long* red) {
    if (blockIdx.x == 0 && threadIdx.x < RED_WORDS) red[threadIdx.x] = 0ull;
}

// per level: the active patch list's size at out[j], the live nodes at
// out[jmax + 1 + j]
template <class R>
__global__ void k_gather_counts(const DevLevelT<R>* lvs, int jmin, int jmax, int32_t* out) {
    int j = jmin + int(threadIdx.x);
    if (j <= jmax) {
        out[j] = *lvs[j].npatches;
        out[jmax + 1 + j] = lvs[j].wl_n[WL_LIVE];
    }
}

// active patches of levels jmin..jmax for the statistics (the pole entry, the
// largest index of an ascending list, left out), one thread per level
template <class R>
__global__ void k_stat_patches(const DevLevelT<R>* lvs, int jmin, int jmax, unsigned long long* out) {
    const int j = jmin + int(threadIdx.x);
    if (j > jmax) return;
    const DevLevelT<R>& L = lvs[j];
    const int32_t n = *L.npatches;
    const bool pole = n > 0 && int64_t(L.patches[n - 1] & PATCH_MASK) == L.npatch;
    out[j] = static_cast<unsigned long long>(n - (pole ? 1 : 0));
}

// sets *flag when a value of x[0..n) is not finite (exponent bits all ones)
__global__ void k_nonfinite(const double* __restrict__ x, int64_t n, unsigned* flag) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    bool bad = false;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
        bad = bad || ((static_cast<unsigned long long>(__double_as_longlong(x[i])) >> 52) & 0x7ffull) == 0x7ffull;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// statistics words of a handle: live nodes, ghost nodes and live edges of level j
// at 3 j .. 3 j + 2, active patches of level j at STAT_PATCHES + j (levels 0..15)
constexpr int STAT_PATCHES = 48, STAT_WORDS = 64;

constexpr int GHOST_HOPS = 5;

template <typename T>
T* dev_alloc(std::vector<void*>& allocs, size_t n) {
    void* p = nullptr;
    ck(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc");
    allocs.push_back(p);
    return static_cast<T*>(p);
}

// The grid and every geometric table of levels jmin..jmax on the device (read-only
// after construction).  Handles with the same jmin, patch size, radius and rotation
// rate share one Geometry; a handle uses the levels up to its own jmax.
struct Geometry {
    int jmin = 0, jmax = 0, patch = 0;
    double radius = 0, omega = 0;
    std::vector<DevLevel> lv;                 // geometry pointers only (FP64 tables)
    std::vector<DevLevelT<float>> lvf;        // the same with FP32 transform weights (on demand)
    std::vector<int64_t> n_irr;               // entries per level whose tile is not regular (poles included)
    std::mutex mu;
    std::vector<std::vector<double>> xyz;     // host node positions per level (flattened)
    std::vector<std::vector<int32_t>> edges;  // host edge (origin, end) pairs per level
    std::vector<void*> allocs;

    template <typename T>
    T* up(const std::vector<T>& v) {
        T* p = dev_alloc<T>(allocs, v.size());
        ck(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
        return p;
    }
    template <typename T, int K>
    T* up_slots(const std::vector<T> (&v)[K], int count) {
        size_t n = v[0].size();
        std::vector<T> flat(n * count);
        for (int k = 0; k < count; ++k) std::memcpy(flat.data() + k * n, v[k].data(), n * sizeof(T));
        return up(flat);
    }
    // FP32 copies of the transform weights (rounded once from the FP64 tables); the
    // geometry and the TRiSK weights stay FP64
    void ensure_fp32() {
        std::lock_guard<std::mutex> lock(mu);
        if (!lvf.empty()) return;
        std::vector<DevLevelT<float>> out(lv.size());
        for (int j = jmin; j <= jmax; ++j) {
            const DevLevel& D = lv[j];
            DevLevelT<float>& F = out[j];
            F.J = D.J, F.n = D.n, F.p = D.p, F.np = D.np, F.nelem = D.nelem, F.N = D.N, F.E = D.E, F.T = D.T;
            F.npatch = D.npatch, F.dx = D.dx, F.kx2 = D.kx2;
            F.en = D.en, F.et = D.et, F.tn = D.tn, F.te = D.te, F.deg = D.deg, F.ring_e = D.ring_e, F.ring_n = D.ring_n, F.f2c = D.f2c;
            F.cor_i = D.cor_i, F.par = D.par, F.fe_kind = D.fe_kind, F.fe_ce = D.fe_ce, F.vst = D.vst;
            F.c2f = D.c2f, F.mid = D.mid, F.half = D.half, F.mk_i = D.mk_i, F.rf_fi = D.rf_fi, F.rf_ci = D.rf_ci;
            F.ppar = D.ppar, F.pnbr = D.pnbr, F.pchild = D.pchild;
            F.thalo = D.thalo, F.tirr = D.tirr;
            // the geometry stays FP64 (no FP32 copies)
            F.A_i = D.A_i, F.A_v = D.A_v, F.kite = D.kite, F.d_e = D.d_e, F.l_e = D.l_e, F.f_v = D.f_v;
            F.f_n = D.f_n, F.cor_w = D.cor_w;
            auto cv = [&](const double* x, int64_t n) -> const float* {
                if (!x) return nullptr;
                float* y = dev_alloc<float>(allocs, n);
                launch_convert(x, y, n, cudaStream_t(0));
                return y;
            };
            F.ptw = cv(D.ptw, 4 * D.N);
            F.vw = cv(D.vw, int64_t(VST) * D.E);
            F.mk_w = cv(D.mk_w, 12 * D.N);
            F.rf_fw = cv(D.rf_fw, int64_t(RF_F) * D.E);
            F.rf_cw = cv(D.rf_cw, int64_t(RF_C) * D.E);
        }
        ck(cudaDeviceSynchronize(), "fp32 tables");
        lvf.swap(out);
    }
    // geometry blocks of the structured trend in precision R (on demand): the
    // FP64 tables rounded once, as the stencils round them on use
    bool tgeo_f64 = false, tgeo_f32 = false;
    template <class R>
    void ensure_tile_geo() {
        std::lock_guard<std::mutex> lock(mu);
        constexpr bool f32 = std::is_same<R, float>::value;
        bool& done = f32 ? tgeo_f32 : tgeo_f64;
        if (done) return;
        for (int j = jmin; j <= jmax; ++j) {
            DevLevelT<R>& D = *level_rec<R>(j);
            if (!D.thalo) continue;
            const size_t words = tile_geo_words<R>(patch);
            if (!words || D.p != patch) throw std::runtime_error("tile geometry: patch side");
            R* out = dev_alloc<R>(allocs, size_t(D.npatch) * words);
            ck(cudaMemset(out, 0, size_t(D.npatch) * words * sizeof(R)), "memset");
            ck(build_tile_geo<R>(D, patch, out, cudaStream_t(0)), "tile geometry");
            D.tgeo = out;
        }
        ck(cudaDeviceSynchronize(), "tile geometry");
        done = true;
    }
    template <class R>
    DevLevelT<R>* level_rec(int j) {
        if constexpr (std::is_same<R, float>::value)
            return &lvf[j];
        else
            return &lv[j];
    }
    ~Geometry() {
        for (void* p : allocs) cudaFree(p);
    }
};

}  // namespace

struct sww_handle {
    sww_config cfg{};
    cudaStream_t user = nullptr;    // the caller's stream
    cudaStream_t stream = nullptr;  // the library's own stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::shared_ptr<Geometry> geo;  // shared grid and tables
    // geometry of geo plus this handle's state arrays, in the handle's precision
    std::vector<DevLevelT<double>> lv;
    std::vector<DevLevelT<float>> lvf;
    void* d_lvs = nullptr;          // device copy of lv or lvf
    double* stage = nullptr;        // FP64 staging buffer of host or FP32 input (set_state; N + E of Jmax)
    // learned refinement proposal: 0 off, 1 features only, 2 features and proposal
    int learn_mode = 0;
    float tau = 0.5f;
    MlpWeights net{};
    MlpWeights* d_net = nullptr;   // device copy of net (the mask kernels read it)
    unsigned long long* lstat = nullptr;   // [3] misses, over-refined, proposed (cumulative)
    // persistent RK stages: blocks of the cooperative launch (0: one launch per phase),
    // barrier state and the error flag of a timed-out barrier (device and pinned copy)
    unsigned stage_blocks = 0, stage_cap = 0;
    // bounded barrier waits of the persistent stage: spin limit in clock cycles
    // (0: the default) and a block that skips its arrival (fault injection, -1: none)
    long long spin_cycles = 0;
    int skip_block = -1;
    // buffers of ensemble steps led by this handle (allocated on first use)
    struct {
        uint8_t* refs = nullptr;    // device MemberRef array
        uint8_t* h_refs = nullptr;  // pinned staging of the refs
        unsigned* bar = nullptr;
        int* err = nullptr;
        int* h_err = nullptr;
        cudaEvent_t ev = nullptr;
        unsigned grid = 0;
        uint8_t* out = nullptr;     // device read-back records (BatchOut per member)
        uint8_t* h_out = nullptr;   // pinned copy
    } ens;
    unsigned* bar = nullptr;
    int* err = nullptr;
    int* h_err = nullptr;
    std::vector<void*> allocs;
    unsigned long long *red = nullptr, *cnt = nullptr;
    double *thr = nullptr, *dt = nullptr, *part = nullptr, *sums = nullptr;
    int32_t *all_list = nullptr, *all_count = nullptr, *d_counts = nullptr, *sig_any = nullptr;
    // entries of all_list whose tile is not regular, and a bound on their number
    int32_t *irr_list = nullptr, *irr_count = nullptr;
    int64_t irr_bound = 0;
    uint8_t* self_ref = nullptr;    // device MemberRef of this handle (its own trend launches)
    // candidate lists of the list-based mask (all levels)
    int32_t *cand = nullptr, *cand_count = nullptr, *gcand = nullptr, *gcand_count = nullptr;
    int64_t total_entries = 0;
    int32_t* h_counts = nullptr;    // pinned: per-level list sizes, then live nodes, after each step
    double* h_dt = nullptr;         // pinned: time step of the last step
    int S = 64, jtop = 0, nsm = 152;
    unsigned grid_all = 1;
    std::vector<unsigned> grid_lv;
    double t = 0, last_dt = 0;
    int64_t steps = 0;
    bool has_state = false;
    // captured steps: (part, top level, adapt, dt, stage blocks) -> graph and its kernel count
    std::map<std::tuple<int, int, int, double, unsigned>, std::pair<cudaGraphExec_t, int64_t>> graphs;
    // tracing: per-class event pairs
    uint32_t prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        int64_t launches;   // kernel launches between the two events
    };
    std::vector<Rec> recs;
    cudaEvent_t take_event() {
        if (!ev_pool.empty()) {
            cudaEvent_t e = ev_pool.back();
            ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        ck(cudaEventCreate(&e), "cudaEventCreate");
        return e;
    }

    template <typename T>
    T* alloc(size_t n) {
        return dev_alloc<T>(allocs, n);
    }
    void drop_graphs() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second.first);
        graphs.clear();
    }
    ~sww_handle() {
        if (stream) cudaStreamSynchronize(stream);
        drop_graphs();
        for (auto& r : recs) cudaEventDestroy(r.a), cudaEventDestroy(r.b);
        for (auto e : ev_pool) cudaEventDestroy(e);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (h_counts) cudaFreeHost(h_counts);
        if (h_err) cudaFreeHost(h_err);
        if (ens.h_refs) cudaFreeHost(ens.h_refs);
        if (ens.h_err) cudaFreeHost(ens.h_err);
        if (ens.h_out) cudaFreeHost(ens.h_out);
        if (ens.ev) cudaEventDestroy(ens.ev);
        if (h_dt) cudaFreeHost(h_dt);
        for (void* p : allocs) cudaFree(p);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

template <class R>
std::vector<DevLevelT<R>>& lvl(sww_handle* h);
template <>
std::vector<DevLevelT<double>>& lvl<double>(sww_handle* h) {
    return h->lv;
}
template <>
std::vector<DevLevelT<float>>& lvl<float>(sww_handle* h) {
    return h->lvf;
}
template <class R>
const std::vector<DevLevelT<R>>& lvl(const sww_handle* h) {
    return lvl<R>(const_cast<sww_handle*>(h));
}
template <class R>
DevLevelT<R>* dlv(const sww_handle* h) {
    return static_cast<DevLevelT<R>*>(h->d_lvs);
}
// sizes of level j (any precision)
const DevLevel& meta(const sww_handle* h, int j) { return h->geo->lv[j]; }

// Calls f(R()) with R the handle's working precision.
template <class F>
int by_prec(const sww_handle* h, F&& f) {
    return h->cfg.precision == SWW_FP32 ? f(float(0)) : f(double(0));
}

// geometry of one level (fine-side tables when a coarser level exists, coarse-side
// tables when a finer one does)
void upload_geometry(Geometry& G, HostLevel& L, bool fine_side, bool coarse_side) {
    DevLevel D{};
    D.J = L.J, D.n = L.n, D.p = L.p, D.np = L.np, D.nelem = L.nelem, D.N = L.N, D.E = L.E, D.T = L.T, D.npatch = L.npatch;
    D.dx = nominal_spacing(L.J, G.radius);
    D.kx2 = (M_PI / D.dx) * (M_PI / D.dx);
    D.en = G.up_slots(L.en, 2);
    D.et = G.up_slots(L.et, 2);
    D.tn = G.up_slots(L.tn, 3);
    D.te = G.up_slots(L.te, 3);
    D.deg = G.up(L.deg);
    D.ring_e = G.up_slots(L.ring_e, 6);
    D.ring_n = G.up_slots(L.ring_n, 6);
    D.A_i = G.up(L.A_i), D.A_v = G.up(L.A_v), D.kite = G.up_slots(L.kite, 3);
    D.d_e = G.up(L.d_e), D.l_e = G.up(L.l_e), D.f_v = G.up(L.f_v), D.f_n = G.up(L.f_n);
    D.cor_i = G.up_slots(L.cor_i, COR);
    D.cor_w = G.up_slots(L.cor_w, COR);
    D.thalo = L.tile_halo.empty() ? nullptr : G.up(L.tile_halo);
    D.tirr = G.up(L.tile_irr);
    {
        int64_t n = 0;
        for (uint8_t f : L.tile_irr) n += f;
        if (int64_t(G.n_irr.size()) <= L.J) G.n_irr.resize(L.J + 1, 0);
        G.n_irr[L.J] = n;
    }
    if (fine_side) {
        D.par = G.up_slots(L.par, 4);
        D.ptw = G.up_slots(L.ptw, 4);
        D.fe_kind = G.up(L.fe_kind);
        D.fe_ce = G.up(L.fe_ce);
        D.vst = G.up_slots(L.vst, VST);
        D.vw = G.up_slots(L.vw, VST);
    }
    if (coarse_side) {
        D.c2f = G.up(L.c2f), D.mid = G.up(L.mid), D.half = G.up_slots(L.half, 2);
        D.mk_i = G.up_slots(L.mk_i, 12);
        D.mk_w = G.up_slots(L.mk_w, 12);
        D.rf_fi = G.up_slots(L.rf_fi, RF_F);
        D.rf_fw = G.up_slots(L.rf_fw, RF_F);
        D.rf_ci = G.up_slots(L.rf_ci, RF_C);
        D.rf_cw = G.up_slots(L.rf_cw, RF_C);
    }
    // f2c of this level: coarse node at the same place (-1 for odd nodes)
    {
        std::vector<int32_t> f2c(L.N, -1);
        if (fine_side) {
            // even element (2i, 2j) <-> coarse element (i, j); poles map to poles
            int64_t n = L.n, p = L.p, np = L.np;
            int64_t cn = n / 2, cp = std::min<int64_t>(L.p, cn), cnp = cn / cp;
            for (int64_t e = 0; e < L.nelem; ++e) {
                int64_t pp = p * p, pid = e / pp, loc = e % pp;
                int64_t pj = pid % np, pi = (pid / np) % np, d = pid / (np * np);
                int64_t i = pi * p + loc / p, j = pj * p + loc % p;
                if ((i & 1) || (j & 1)) continue;
                int64_t ci = i / 2, cj = j / 2;
                f2c[e] = int32_t(((d * cnp + ci / cp) * cnp + cj / cp) * cp * cp + (ci % cp) * cp + (cj % cp));
            }
            f2c[L.nelem] = int32_t(10 * cn * cn);
            f2c[L.nelem + 1] = int32_t(10 * cn * cn + 1);
        }
        D.f2c = G.up(f2c);
        // patch graph: same-level neighbour patches (a node of one within two hops of
        // a node of the other, so that every patch around P within p hops is one),
        // the coarse patch under each patch, and the fine patches over it
        const int64_t pp = L.p * L.p, np1 = L.npatch + 1;
        auto patch_of = [&](int64_t v) { return v < L.nelem ? v / pp : L.npatch; };
        std::vector<int32_t> nbr(NB * np1, -1), par(np1, -1), child(4 * np1, -1);
        std::vector<int> cnt(np1, 0);
        auto add = [&](std::vector<int32_t>& tab, std::vector<int>& c, int cap, int64_t P, int64_t Q) {
            for (int q = 0; q < c[P]; ++q)
                if (tab[q * np1 + P] == Q) return;
            if (c[P] >= cap) throw std::runtime_error("patch table overflow");
            tab[c[P]++ * np1 + P] = int32_t(Q);
        };
        for (int64_t v = 0; v < L.N; ++v) {
            const int64_t P = patch_of(v);
            for (int k = 0; k < L.deg[v]; ++k) {
                const int64_t w = L.ring_n[k][v];
                if (patch_of(w) != P) add(nbr, cnt, NB, P, patch_of(w));
                for (int k2 = 0; k2 < L.deg[w]; ++k2) {
                    const int64_t Q = patch_of(L.ring_n[k2][w]);
                    if (Q != P) add(nbr, cnt, NB, P, Q);
                }
            }
        }
        if (fine_side) {
            const int64_t cp = std::min<int64_t>(L.p, L.n / 2), cpp = cp * cp, cnelem = 10 * (L.n / 2) * (L.n / 2);
            for (int64_t v = 0; v < L.N; ++v) {
                int64_t P = patch_of(v);
                if (par[P] >= 0) continue;
                int64_t k = f2c[v] >= 0 ? f2c[v] : f2c[L.par[0][v]];
                par[P] = int32_t(k < cnelem ? k / cpp : cnelem / cpp);
            }
        }
        if (coarse_side) {
            const int64_t fn = 2 * L.n, fp = std::min<int64_t>(G.patch, fn), fpp = fp * fp, fnelem = 10 * fn * fn;
            std::vector<int> cc(np1, 0);
            for (int64_t v = 0; v < L.N; ++v) {
                const int64_t x = L.c2f[v];
                add(child, cc, 4, patch_of(v), x < fnelem ? x / fpp : fnelem / fpp);
            }
        }
        D.pchild = G.up(child);
        D.pnbr = G.up(nbr);
        D.ppar = G.up(par);
    }
    G.lv[L.J] = D;
}

std::shared_ptr<Geometry> build_geometry(int jmin, int jmax, int patch, double radius, double omega) {
    auto G = std::make_shared<Geometry>();
    G->jmin = jmin, G->jmax = jmax, G->patch = patch, G->radius = radius, G->omega = omega;
    Hierarchy H;
    build_hierarchy(H, jmin, jmax, patch, radius, omega);
    // every id a kernel gathers through must lie in its array (the kernels do not
    // check them again)
    std::string what;
    if (!validate_tables(H, &what)) throw std::runtime_error("grid table out of bounds: " + what);
    G->lv.assign(jmax + 1, DevLevel{});
    G->xyz.assign(jmax + 1, {});
    G->edges.assign(jmax + 1, {});
    for (int j = jmin; j <= jmax; ++j) {
        HostLevel& L = H.lv[j];
        upload_geometry(*G, L, j > jmin, j < jmax);
        G->xyz[j].resize(3 * L.N);
        for (int64_t v = 0; v < L.N; ++v)
            G->xyz[j][3 * v] = L.xyz[v].x, G->xyz[j][3 * v + 1] = L.xyz[v].y, G->xyz[j][3 * v + 2] = L.xyz[v].z;
        G->edges[j].resize(2 * L.E);
        for (int64_t e = 0; e < L.E; ++e) G->edges[j][2 * e] = L.en[0][e], G->edges[j][2 * e + 1] = L.en[1][e];
    }
    return G;
}

// state and work arrays of one level of a handle (zeroed)
template <class R>
void alloc_state(sww_handle* h, int j) {
    DevLevelT<R> D;
    if constexpr (std::is_same<R, float>::value)
        D = h->geo->lvf[j];
    else
        D = h->geo->lv[j];
    // a level with tiles has its geometry blocks (the structured trend copies them)
    if (D.thalo && !D.tgeo) throw std::runtime_error("tile geometry blocks missing");
    const int64_t N = D.N, E = D.E, T = D.T;
    const int64_t coarse_E = j > h->cfg.jmin ? h->geo->lv[j - 1].E : 1;
    R** dN[] = {&D.dh, &D.dh0, &D.dha, &D.dht, &D.B, &D.c, &D.hdet};
    for (auto p : dN) *p = h->alloc<R>(N);
    R** dE[] = {&D.u, &D.u0, &D.ua, &D.ut, &D.F, &D.Q, &D.ui, &D.Fd};
    for (auto p : dE) *p = h->alloc<R>(E);
    D.q = h->alloc<R>(T);
    D.zeta = h->alloc<R>(T);
    ck(cudaMemset(D.zeta, 0, T * sizeof(R)), "memset");
    D.nu = h->cfg.nu;
    D.advect = h->cfg.advect;
    D.ue = h->alloc<R>(coarse_E);
    // byte arrays padded to a multiple of 16 bytes (zeroed): the structured trend
    // copies the aligned 32-bit word holding a flag
    const int64_t N16 = (N + 15) / 16 * 16, E16 = (E + 15) / 16 * 16;
    uint8_t** bN[] = {&D.nflag, &D.sig, &D.tmask, &D.band0, &D.band1};
    for (auto p : bN) *p = h->alloc<uint8_t>(N16);
    D.eflag = h->alloc<uint8_t>(E16);
    D.pflag = h->alloc<uint8_t>(D.npatch);
    ck(cudaMemset(D.pflag, 0, D.npatch), "memset");
    D.pfeat = h->alloc<float>(NF * (D.npatch + 1));
    D.prop = h->alloc<uint8_t>(D.npatch + 1);
    D.prop_prev = h->alloc<uint8_t>(D.npatch + 1);
    D.pexact = h->alloc<uint8_t>(D.npatch + 1);
    uint8_t* pz[] = {D.prop, D.prop_prev, D.pexact};
    for (uint8_t* p : pz) ck(cudaMemset(p, 0, D.npatch + 1), "memset");
    ck(cudaMemset(D.pfeat, 0, NF * (D.npatch + 1) * sizeof(float)), "memset");
    D.patches = h->alloc<int32_t>(D.npatch + 1);
    D.npatches = h->alloc<int32_t>(1);
    D.wl = h->alloc<int32_t>(3 * N + 2 * E);
    D.wl_n = h->alloc<int32_t>(WL_WORDS);
    ck(cudaMemset(D.wl_n, 0, WL_WORDS * sizeof(int32_t)), "memset");
    uint8_t** cf[] = {&D.zflag, &D.sflag, &D.cflag, &D.lflag, &D.gflag};
    for (auto p : cf) {
        *p = h->alloc<uint8_t>(D.npatch + 1);
        ck(cudaMemset(*p, 0, D.npatch + 1), "memset");
    }
    int32_t** cl[] = {&D.cand, &D.ncand, &D.gcand, &D.ngcand};
    for (auto p : cl) {
        *p = h->alloc<int32_t>(D.npatch + 1);
        ck(cudaMemset(*p, 0, (D.npatch + 1) * sizeof(int32_t)), "memset");
    }
    for (auto p : dN) ck(cudaMemset(*p, 0, N * sizeof(R)), "memset");
    for (auto p : dE) ck(cudaMemset(*p, 0, E * sizeof(R)), "memset");
    ck(cudaMemset(D.q, 0, T * sizeof(R)), "memset");
    for (auto p : bN) ck(cudaMemset(*p, 0, N16), "memset");
    ck(cudaMemset(D.eflag, 0, E16), "memset");
    ck(cudaMemset(D.ue, 0, coarse_E * sizeof(R)), "memset");
    ck(cudaMemset(D.npatches, 0, sizeof(int32_t)), "memset");
    lvl<R>(h)[j] = D;
}

void check_launch() { ck(cudaGetLastError(), "kernel launch"); }

// host FP64 values -> device array of the working precision (on the handle's
// stream; the caller synchronises before the host data goes away)
template <class R>
void to_device(sww_handle* h, R* dst, const double* src, int64_t n) {
    if constexpr (std::is_same<R, double>::value) {
        ck(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "to_device");
    } else {
        std::vector<R> tmp(src, src + n);
        ck(cudaMemcpyAsync(dst, tmp.data(), n * sizeof(R), cudaMemcpyHostToDevice, h->stream), "to_device");
        ck(cudaStreamSynchronize(h->stream), "to_device");   // tmp lives on this frame
    }
}

// device array of the working precision -> host FP64 values (synchronous)
template <class R>
void from_device(sww_handle* h, double* dst, const R* src, int64_t n) {
    std::vector<R> tmp;
    void* host = dst;
    if constexpr (!std::is_same<R, double>::value) {
        tmp.resize(n);
        host = tmp.data();
    }
    ck(cudaEventRecord(h->ev_in, h->user), "join in");
    ck(cudaStreamWaitEvent(h->stream, h->ev_in, 0), "join in");
    ck(cudaMemcpyAsync(host, src, n * sizeof(R), cudaMemcpyDeviceToHost, h->stream), "from_device");
    ck(cudaStreamSynchronize(h->stream), "from_device");
    if constexpr (!std::is_same<R, double>::value)
        for (int64_t i = 0; i < n; ++i) dst[i] = double(tmp[i]);
}

// Orders the library's stream after the caller's stream on entry and the caller's
// stream after the library's stream on exit.
struct Join {
    sww_handle* h;
    explicit Join(sww_handle* h_) : h(h_) {
        ck(cudaEventRecord(h->ev_in, h->user), "join in");
        ck(cudaStreamWaitEvent(h->stream, h->ev_in, 0), "join in");
    }
    ~Join() {
        if (cudaEventRecord(h->ev_out, h->stream) == cudaSuccess) cudaStreamWaitEvent(h->user, h->ev_out, 0);
    }
};

// Records a pair of events around the launches made during its lifetime when the
// handle traces class `cls` (eager execution only).
struct Trace {
    sww_handle* h;
    int cls;
    cudaEvent_t a = nullptr;
    int64_t l0 = 0;
    Trace(sww_handle* h_, int c) : h(h_), cls(c) {
        if (h->prof_mask & (1u << cls)) {
            a = h->take_event();
            ck(cudaEventRecord(a, h->stream), "cudaEventRecord");
            l0 = kernel_launches();
        }
    }
    ~Trace() {
        if (!a) return;
        cudaEvent_t b = h->take_event();
        cudaEventRecord(b, h->stream);
        h->recs.push_back({cls, a, b, kernel_launches() - l0});
    }
};

template <class R>
WorkT<R> work_all(const sww_handle* h) {
    return WorkT<R>{dlv<R>(h), h->all_list, h->all_count, h->S, h->grid_all};
}
template <class R>
WorkT<R> work_level(const sww_handle* h, int j) {
    const DevLevelT<R>& L = lvl<R>(h)[j];
    return WorkT<R>{nullptr, L.patches, L.npatches, h->S, h->grid_lv[j]};
}

// ------------------------------------------------------------------ sequences

template <class R>
void fill_ghosts(sww_handle* h) {
    auto& lv = lvl<R>(h);
    for (int j = h->cfg.jmin + 1; j <= h->jtop; ++j) {
        Trace t(h, SWW_K_FILL);
        launch_fill(lv[j], lv[j - 1], work_level<R>(h, j), h->stream);
    }
}

// one trend evaluation (Sec. 3.1): ghosts, q/K/B/F/qF^perp on every level, then the
// restriction of B, F and q F^perp from the top level down to Jmin
template <class R>
void trend(sww_handle* h) {
    const int j0 = h->cfg.jmin;
    cudaStream_t s = h->stream;
    auto& lv = lvl<R>(h);
    fill_ghosts<R>(h);
    {
        // the structured trend of every active patch, then the irregular patches'
        // node and Coriolis terms (one member: this handle)
        BatchArgs<R> a{reinterpret_cast<const MemberRef<R>*>(h->self_ref), 1, h->S, j0, h->jtop, h->cfg.H, h->cfg.g,
                       RKStage{}, nullptr, nullptr, 0.0, nullptr};
        { Trace t(h, SWW_K_TREND); ck(launch_tile_trend(a, h->total_entries, h->irr_bound, h->nsm, 1, s), "trend"); }
        { Trace t(h, SWW_K_IRREG); ck(launch_tile_trend(a, h->total_entries, h->irr_bound, h->nsm, 2, s), "trend"); }
    }
    for (int j = h->jtop - 1; j >= j0; --j) {
        { Trace t(h, SWW_K_RESTRICT); launch_restrict(lv[j], lv[j + 1], work_level<R>(h, j), s); }
        { Trace t(h, SWW_K_NODE); launch_div(lv[j], work_level<R>(h, j), s); }
    }
}

template <class R>
void update(sww_handle* h, const RKStage& st) {
    Trace t(h, SWW_K_UPDATE);
    launch_update(work_all<R>(h), st, h->dt, h->stream);
}

// trend and RK stage: one persistent cooperative launch, or one launch per phase
template <class R>
void stage(sww_handle* h, const RKStage& st) {
    if (!h->stage_blocks) {
        trend<R>(h);
        update<R>(h, st);
        return;
    }
    Trace t(h, SWW_K_STAGE);
    StageArgs<R> a{dlv<R>(h), h->all_list, h->all_count, h->irr_list, h->irr_count, h->S, h->cfg.jmin, h->jtop,
                   h->cfg.jmax, h->cfg.H, h->cfg.g, st, h->dt, h->bar, h->err, h->spin_cycles, h->skip_block};
    ck(launch_stage(a, h->stage_blocks, h->stream), "persistent stage launch");
}

// SWW_E_TIMEOUT (and the flag cleared) when a persistent stage's barrier or a tile's
// bulk copy timed out
int barrier_status(sww_handle* h) {
    if (!*h->h_err) return SWW_OK;
    *h->h_err = 0;
    ck(cudaMemset(h->err, 0, sizeof(int)), "reset err");
    ck(cudaMemset(h->bar, 0, STAGE_BAR_WORDS * sizeof(unsigned)), "reset barrier");
    return fail(SWW_E_TIMEOUT, "a bounded wait of the RK stage (grid barrier or bulk copy) timed out");
}

template <class R>
void compute_dt(sww_handle* h) {
    Trace t(h, SWW_K_DT);
    count_launch(1);
    k_reset_red<<<1, 32, 0, h->stream>>>(h->red);
    launch_dt(work_all<R>(h), h->cfg.H, h->cfg.g, h->red, h->stream);
    launch_dt_final<R>(dlv<R>(h), h->red, h->cfg.cfl, h->dt, h->stream);
}

// list sizes of every level into pinned host memory (read after the next sync)
template <class R>
void read_counts(sww_handle* h) {
    count_launch(1);
    k_gather_counts<R><<<1, 32, 0, h->stream>>>(dlv<R>(h), h->cfg.jmin, h->cfg.jmax, h->d_counts);
    ck(cudaMemcpyAsync(h->h_counts, h->d_counts, sizeof(int32_t) * 2 * (h->cfg.jmax + 1), cudaMemcpyDeviceToHost,
                       h->stream),
       "counts");
}

// top level with any live or ghost point (after the stream has synchronised)
void update_top(sww_handle* h) {
    int top = h->cfg.jmin;
    for (int j = h->cfg.jmin; j <= h->cfg.jmax; ++j)
        if (h->h_counts[j] > 0) top = j;
    h->jtop = top;
}

// Thread ranges of levels ja..jb for a multi-level dense launch.
template <typename Count>
Span span_of(const sww_handle* h, int ja, int jb, Count count, int tail_j = -1, int64_t tail_threads = 0) {
    Span sp{};
    sp.ja = ja, sp.jb = jb;
    sp.tail_j = -1;
    int64_t t = 0;
    for (int j = ja; j <= jb; ++j) {
        sp.off[j - ja] = t;
        int64_t n = count(meta(h, j));
        if (j == tail_j) {
            sp.tail_j = j, sp.tail_n = n;
            n = std::min(n, tail_threads);
        }
        t += n;
    }
    sp.off[jb + 1 - ja] = t;
    return sp;
}

// The level above the top live level (j1 > top) is a tail level of the mask spans:
// a fixed number of striding threads that leave at once unless the level below holds
// a significant point.
template <class R>
MaskArgsT<R> mask_args(const sww_handle* h, int j0, int j1, bool allow_tail = true) {
    MaskArgsT<R> a{};
    a.lvs = dlv<R>(h), a.host = lvl<R>(h).data(), a.ja = j0, a.jb = j1, a.hops = GHOST_HOPS, a.thr = h->thr;
    auto N = [](const DevLevel& L) { return L.N; };
    auto E = [](const DevLevel& L) { return L.E; };
    auto P = [](const DevLevel& L) { return L.npatch; };
    const int tail = (allow_tail && j1 > h->jtop) ? j1 : -1;
    const int64_t tt = int64_t(h->grid_all) * 256;
    int jf = std::min(j0 + 1, j1);
    a.nodes_f = span_of(h, jf, j1, N, tail, tt);
    a.edges_f = span_of(h, jf, j1, E, tail, tt);
    if (j1 == j0) a.nodes_f.off[1] = 0, a.edges_f.off[1] = 0;   // no level above Jmin
    a.nodes = span_of(h, j0, j1, N, tail, tt);
    a.edges = span_of(h, j0, j1, E, tail, tt);
    a.nodes_c = span_of(h, j0, std::max(j0, j1 - 1), N);
    a.patches = span_of(h, j0, j1, P, tail, int64_t(h->grid_all));
    a.sig_any = h->sig_any;
    a.sig_any_len = h->cfg.jmax + 2;
    a.tail_blocks = h->grid_all;
    a.lstat = h->lstat;
    return a;
}

// Mask construction and inverse transform.  Levels above top + 1 hold no live point
// and can gain none in one adaptation, so the byte-wide passes stop there.
// significance, proposal, mask, patch lists (Sec. 2.3), from the stored
// coefficients and thresholds
// The member record of a handle's mask (levels Jmin..min(top + 1, jmax)).
template <class R>
MaskMember<R> mask_member(const sww_handle* h) {
    MaskMember<R> m{};
    m.lvs = dlv<R>(h);
    m.active = h->all_list, m.active_count = h->all_count;
    m.cand = h->cand, m.cand_count = h->cand_count, m.gcand = h->gcand, m.gcand_count = h->gcand_count;
    m.all = h->all_list, m.all_count = h->all_count, m.irr = h->irr_list, m.irr_count = h->irr_count;
    m.thr = h->thr, m.sig_any = h->sig_any, m.lstat = h->lstat, m.net = h->d_net;
    m.logit_tau = std::log(h->tau / (1.f - h->tau));
    m.learn = h->learn_mode;
    m.jb = std::min(h->jtop + 1, h->cfg.jmax), m.jmax = h->cfg.jmax;
    return m;
}

// The shared part of a mask batch over members whose largest jb and jmax are
// given (their grids are the same as h's).
template <class R, int CAP>
void mask_batch_head(MaskBatch<R, CAP>& b, const sww_handle* h, int nm, int jb_max, int jmax_max) {
    const int j0 = h->cfg.jmin;
    auto np1 = [](const DevLevel& L) { return L.npatch + 1; };
    auto empty = [&]() {
        Span sp{};
        sp.ja = sp.jb = j0, sp.tail_j = -1;
        return sp;
    };
    b.nm = nm, b.P = h->S, b.ja = j0, b.jb_max = jb_max, b.jmax_max = jmax_max;
    b.hops = GHOST_HOPS, b.rings = h->cfg.patch >= 8 ? 1 : 2;
    b.patches = span_of(h, j0, jb_max, np1);
    b.patches_f = jb_max > j0 ? span_of(h, j0 + 1, jb_max, np1) : empty();
    b.props = jmax_max > j0 ? span_of(h, j0 + 1, jmax_max, np1) : empty();
}

// the candidate lists need patches of at least 4 x 4 (one or two rings reach the
// five hops of the ghost band)
bool list_mask(const sww_handle* h) { return h->cfg.mask == 0 && h->cfg.patch >= 4; }

// Significance, proposal, mask, patch lists (Sec. 2.3), from the stored
// coefficients and thresholds: the learned proposal for this mask (features of the
// current coefficients on the levels above Jmin up to the mask's top level, then
// the perceptron), the mask, and the all-level and irregular lists.
template <class R>
void mask_only(sww_handle* h) {
    const int j0 = h->cfg.jmin, j1 = std::min(h->jtop + 1, h->cfg.jmax);
    cudaStream_t s = h->stream;
    Trace tm(h, SWW_K_MASK);
    MaskBatch<R, 1> b{};
    mask_batch_head(b, h, 1, j1, h->cfg.jmax);
    b.m[0] = mask_member<R>(h);
    launch_proposal_batch(b, h->grid_all, 0, s);
    if (list_mask(h))
        launch_mask_batch(b, h->grid_all, s);
    else
        launch_mask(mask_args<R>(h, j0, j1), s);
    launch_proposal_batch(b, h->grid_all, 1, s);
    launch_concat_batch(b, h->grid_all, s);
}

template <class R>
void mask_and_inverse(sww_handle* h) {
    const int j0 = h->cfg.jmin, j1 = std::min(h->jtop + 1, h->cfg.jmax);
    cudaStream_t s = h->stream;
    auto& lv = lvl<R>(h);
    mask_only<R>(h);
    // inverse transform of the retained coefficients, coarse to fine, ghosts per level
    for (int j = j0 + 1; j <= j1; ++j) {
        { Trace t(h, SWW_K_INVERSE); launch_inverse(lv[j], lv[j - 1], work_level<R>(h, j), s); }
        { Trace t(h, SWW_K_FILL); launch_fill(lv[j], lv[j - 1], work_level<R>(h, j), s); }
    }
}

// relative coefficient tolerance: eps, or eps^{3/2} when eps is read as the trend
// tolerance of Sec. 2.3 (both regimes of the paper scale the thresholds by eps^{3/2})
double eps_coeff(const sww_config& c) { return c.regime == 1 ? c.eps * std::sqrt(c.eps) : c.eps; }

template <class R>
void adapt(sww_handle* h, double eh, double eu) {
    cudaStream_t s = h->stream;
    { Trace t(h, SWW_K_COEFF); launch_details(work_all<R>(h), h->cfg.jmin, s); }
    {
        Trace t(h, SWW_K_MASK);
        ck(cudaMemsetAsync(h->red + 2, 0, 2 * sizeof(unsigned long long), s), "memset red");
        launch_maxabs(work_all<R>(h), h->red, s);
        launch_thresholds(h->red, eps_coeff(h->cfg), eh, eu, h->cfg.advect, h->thr, s);
    }
    mask_and_inverse<R>(h);
}

const RKStage* stages(int rk, int& n) {
    // classical RK4 (acc holds k1 + 2 k2 + 2 k3) and the 4-stage, third-order SSP
    // scheme of Spiteri & Ruuth (Sec. 3.1)
    static const RKStage rk4[4] = {
        {1, 1.0, 0.0, 0.5, 0.0, 0.0, 1.0},
        {1, 1.0, 0.0, 0.5, 0.0, 1.0, 2.0},
        {1, 1.0, 0.0, 1.0, 0.0, 1.0, 2.0},
        {1, 1.0, 0.0, 1.0 / 6.0, 1.0 / 6.0, 1.0, 0.0},
    };
    static const RKStage ssp[4] = {
        {1, 0.0, 1.0, 0.5, 0.0, 0.0, 0.0},
        {1, 0.0, 1.0, 0.5, 0.0, 0.0, 0.0},
        {1, 2.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0, 0.0, 0.0, 0.0},
        {1, 0.0, 1.0, 0.5, 0.0, 0.0, 0.0},
    };
    n = 4;
    return rk == SWW_SSP43 ? ssp : rk4;
}

// One RK step with its partial transform and (optionally) adaptation; ends with the
// device-to-host copies of the time step and the list sizes.  part 1 is what comes
// before the RK stages (time step, RK base), part 2 what follows them; part 0 is the
// whole step.
// part 0: the whole step; 1: time step and RK base only; 2: after the stages
// (partial transform, ghosts, adaptation, read-backs); 3: adaptation and
// read-backs only (the rest ran batched over an ensemble); 4: the mask only
template <class R>
void one_step(sww_handle* h, double dt, bool do_adapt, int part = 0) {
    const int j0 = h->cfg.jmin;
    auto& lv = lvl<R>(h);
    if (part == 4) {   // the mask alone (coefficients, thresholds and inverse batched)
        mask_only<R>(h);
        return;
    }
    if (part == 0 || part == 1) {
        if (dt > 0) {
            count_launch(1);
            k_set<<<1, 32, 0, h->stream>>>(h->dt, dt);
        } else {
            compute_dt<R>(h);
        }
        { Trace t(h, SWW_K_UPDATE); launch_save_base(work_all<R>(h), h->stream); }
    }
    if (part == 0) {
        int ns;
        const RKStage* st = stages(h->cfg.rk, ns);
        for (int k = 0; k < ns; ++k) stage<R>(h, st[k]);
    }
    if (part == 1) return;
    if (part != 3) {
        for (int j = h->jtop - 1; j >= j0; --j) {
            Trace t(h, SWW_K_PARTIAL);
            launch_partial(lv[j], lv[j + 1], work_level<R>(h, j), h->stream);
        }
        fill_ghosts<R>(h);
    }
    if (do_adapt) adapt<R>(h, -1.0, -1.0);
    read_counts<R>(h);
    ck(cudaMemcpyAsync(h->h_dt, h->dt, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "dt");
    ck(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "err");
}

// Run one step (or part of one) through a captured graph (eager when tracing).
template <class R>
void run_step_t(sww_handle* h, double dt, bool do_adapt, int part = 0) {
    if (h->prof_mask) {
        one_step<R>(h, dt, do_adapt, part);
        return;
    }
    const unsigned mode = h->stage_blocks;
    auto key = std::make_tuple(part, h->jtop, int(do_adapt), dt > 0 ? dt : -1.0, mode);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        if (h->graphs.size() >= 24) h->drop_graphs();
        int64_t before = kernel_launches();
        ck(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            one_step<R>(h, dt, do_adapt, part);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        cudaGraph_t g = nullptr;
        ck(cudaStreamEndCapture(h->stream, &g), "end capture");
        int64_t n = kernel_launches() - before;
        count_launch(-n);
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        ck(e, "graph instantiate");
        it = h->graphs.emplace(key, std::make_pair(ex, n)).first;
    }
    ck(cudaGraphLaunch(it->second.first, h->stream), "graph launch");
    count_launch(it->second.second);
}

void run_step(sww_handle* h, double dt, bool do_adapt, int part = 0) {
    by_prec(h, [&](auto r) {
        run_step_t<decltype(r)>(h, dt, do_adapt, part);
        return 0;
    });
}

// The member record of a handle (its top level and j1 as of the last step).
template <class R>
MemberRef<R> member_ref(const sww_handle* h) {
    const int j1 = std::min(h->jtop + 1, h->cfg.jmax);
    return MemberRef<R>{dlv<R>(h), h->all_list, h->all_count, h->dt, h->jtop, h->red, h->cfg.cfl, h->thr,
                        eps_coeff(h->cfg), h->cfg.advect, j1, h->cfg.jmax, h->err, h->irr_list, h->irr_count};
}

// Device buffers of ensemble steps led by `lead` (allocated on first use).
template <class R>
void ensure_ensemble(sww_handle* lead) {
    auto& E = lead->ens;
    if (E.refs) return;
    E.refs = lead->alloc<uint8_t>(sizeof(MemberRef<double>) * 128);
    E.bar = lead->alloc<unsigned>(STAGE_BAR_WORDS);
    E.err = lead->alloc<int>(1);
    E.out = lead->alloc<uint8_t>(sizeof(BatchOut) * 128);
    ck(cudaMemset(E.bar, 0, STAGE_BAR_WORDS * sizeof(unsigned)), "memset");
    ck(cudaMemset(E.err, 0, sizeof(int)), "memset");
    ck(cudaMallocHost(&E.h_refs, sizeof(MemberRef<double>) * 128), "cudaMallocHost");
    ck(cudaMallocHost(&E.h_err, sizeof(int)), "cudaMallocHost");
    ck(cudaMallocHost(&E.h_out, sizeof(BatchOut) * 128), "cudaMallocHost");
    *E.h_err = 0;
    ck(cudaEventCreateWithFlags(&E.ev, cudaEventDisableTiming), "cudaEventCreate");
}

// Member refs of this step on the lead's stream (after every member's previous
// work: the members' streams are joined into the lead's), the largest top level
// and j1, and the bounds of the members' level-j list entries.
template <class R>
BatchArgs<R> ensemble_refs(sww_handle* const* hs, int n, std::vector<int64_t>& entries, int& j1_max,
                           int64_t& irr_entries) {
    sww_handle* lead = hs[0];
    auto& E = lead->ens;
    MemberRef<R>* refs = reinterpret_cast<MemberRef<R>*>(E.h_refs);
    int jtop = 0;
    j1_max = 0;
    for (int i = 0; i < n; ++i) {
        sww_handle* h = hs[i];
        const int j1 = std::min(h->jtop + 1, h->cfg.jmax);
        refs[i] = member_ref<R>(h);
        refs[i].jtop = h->jtop;
        refs[i].j1 = j1;
        jtop = std::max(jtop, h->jtop);
        j1_max = std::max(j1_max, j1);
        if (i > 0) {
            ck(cudaEventRecord(h->ev_out, h->stream), "ensemble join");
            ck(cudaStreamWaitEvent(lead->stream, h->ev_out, 0), "ensemble join");
        }
    }
    ck(cudaMemcpyAsync(E.refs, refs, sizeof(MemberRef<R>) * n, cudaMemcpyHostToDevice, lead->stream), "refs");
    entries.assign(j1_max + 1, 0);
    irr_entries = 0;
    for (int i = 0; i < n; ++i) irr_entries += hs[i]->irr_bound;
    for (int i = 0; i < n; ++i)
        for (int j = lead->cfg.jmin; j <= std::min(j1_max, hs[i]->cfg.jmax); ++j)
            entries[j] += meta(hs[i], j).npatch + 1;
    int ns;
    const RKStage* st = stages(lead->cfg.rk, ns);
    return BatchArgs<R>{reinterpret_cast<const MemberRef<R>*>(E.refs), n, lead->S, lead->cfg.jmin, jtop,
                        lead->cfg.H, lead->cfg.g, st[0], E.bar, E.err, 0.0, E.out};
}

// One step of every member with the work batched over members (persistent = 3), on
// the first member's stream: time step and RK base, the stage phases, the partial
// transform and ghosts, the coefficients and thresholds; each member's mask on its
// own stream; then the inverse transform and ghosts and the read-back records of
// all members (copied to pinned memory; the caller synchronises the first
// member's stream).  The records cover all members.
template <class R>
void ensemble_phased(sww_handle* const* hs, int n, double dt, bool do_adapt) {
    sww_handle* lead = hs[0];
    ensure_ensemble<R>(lead);
    auto& E = lead->ens;
    cudaStream_t s = lead->stream;
    std::vector<int64_t> entries;
    int j1_max = 0;
    int64_t irr_entries = 0;
    BatchArgs<R> a = ensemble_refs<R>(hs, n, entries, j1_max, irr_entries);
    int ns;
    const RKStage* st = stages(lead->cfg.rk, ns);
    {
        Trace t(lead, SWW_K_DT);
        ck(launch_batch_pre(a, entries.data(), lead->nsm, dt, s), "batched ensemble step");
    }
    static const int part_cls[5] = {SWW_K_FILL, SWW_K_TREND, SWW_K_IRREG, SWW_K_RESTRICT, SWW_K_UPDATE};
    for (int k = 0; k < ns; ++k) {
        Trace t(lead, SWW_K_STAGE);
        a.st = st[k];
        for (int part = 0; part < 5; ++part) {
            Trace tp(lead, part_cls[part]);
            ck(launch_stage_batch_part(a, entries.data(), irr_entries, lead->nsm, part, s), "batched ensemble stage");
        }
    }
    {
        Trace t(lead, SWW_K_PARTIAL);
        ck(launch_batch_post(a, entries.data(), lead->nsm, s), "batched ensemble step");
    }
    if (do_adapt) {
        {
            Trace t(lead, SWW_K_COEFF);
            ck(launch_batch_adapt_pre(a, entries.data(), lead->nsm, s), "batched ensemble step");
        }
        bool lists = true;
        for (int i = 0; i < n; ++i) lists = lists && list_mask(hs[i]);
        if (lists) {
            // every member's mask in the same launches on the lead's stream
            Trace tm(lead, SWW_K_MASK);
            auto b = std::make_unique<MaskBatch<R, MASK_BATCH_MAX>>();
            int jb_max = lead->cfg.jmin, jmax_max = lead->cfg.jmin;
            for (int i = 0; i < n; ++i) {
                b->m[i] = mask_member<R>(hs[i]);
                jb_max = std::max(jb_max, b->m[i].jb);
                jmax_max = std::max(jmax_max, hs[i]->cfg.jmax);
            }
            mask_batch_head(*b, lead, n, jb_max, jmax_max);
            // blocks per member of the list passes: two waves of 8 blocks of 256 per SM
            // over all members (measured 8 % faster than one wave on the 64-member jet)
            const unsigned grid = unsigned(std::max(1, std::min<int>(int(lead->grid_all), 16 * lead->nsm / n)));
            launch_proposal_batch(*b, grid, 0, s);
            launch_mask_batch(*b, grid, s);
            launch_proposal_batch(*b, grid, 1, s);
            launch_concat_batch(*b, grid, s);
        } else {
            // each member's mask on its own stream, then back to the lead's
            ck(cudaEventRecord(E.ev, s), "ensemble fork");
            for (int i = 1; i < n; ++i) ck(cudaStreamWaitEvent(hs[i]->stream, E.ev, 0), "ensemble fork");
            for (int i = 0; i < n; ++i) run_step(hs[i], dt, true, 4);
            for (int i = 1; i < n; ++i) {
                ck(cudaEventRecord(hs[i]->ev_out, hs[i]->stream), "ensemble join");
                ck(cudaStreamWaitEvent(s, hs[i]->ev_out, 0), "ensemble join");
            }
        }
        Trace t(lead, SWW_K_INVERSE);
        ck(launch_batch_adapt_post(a, entries.data(), j1_max, lead->nsm, s), "batched ensemble step");
    }
    ck(launch_batch_out(a, s), "batched ensemble step");
    ck(cudaMemcpyAsync(E.h_out, E.out, sizeof(BatchOut) * n, cudaMemcpyDeviceToHost, s), "read-back");
}

int check_level(const sww_handle* h, int level) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (level < h->cfg.jmin || level > h->cfg.jmax) return fail(SWW_E_ARG, "level out of range");
    return SWW_OK;
}

template <typename F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const CudaError& e) {
        return fail(SWW_E_CUDA, e.what());
    } catch (const std::bad_alloc&) {
        return fail(SWW_E_POOL, "host allocation failed");
    } catch (const std::exception& e) {
        return fail(SWW_E_ARG, e.what());
    }
}

int check_config(const sww_config* cfg) {
    if (cfg->jmin < 1 || cfg->jmax < cfg->jmin || cfg->jmax > 11) return fail(SWW_E_ARG, "need 1 <= jmin <= jmax <= 11");
    if (cfg->advect != 0 && cfg->advect != 1) return fail(SWW_E_ARG, "advect must be 0 or 1");
    if (cfg->regime != 0 && cfg->regime != 1) return fail(SWW_E_ARG, "regime must be 0 or 1");
    // a prescribed velocity never divides by the depth, so it may vanish (h = dh)
    const bool depth_ok = cfg->advect ? cfg->H >= 0 : cfg->H > 0;
    if (!(cfg->radius > 0) || !(cfg->g > 0) || !depth_ok || !(cfg->cfl > 0))
        return fail(SWW_E_ARG, "radius, g and cfl must be positive, H positive (>= 0 with advect)");
    if (!(cfg->eps >= 0)) return fail(SWW_E_ARG, "eps must be >= 0 (0: every point significant, no compression)");
    if (cfg->patch != 4 && cfg->patch != 8 && cfg->patch != 16) return fail(SWW_E_ARG, "patch must be 4, 8 or 16");
    if (cfg->rk != SWW_RK4 && cfg->rk != SWW_SSP43) return fail(SWW_E_ARG, "rk must be SWW_RK4 or SWW_SSP43");
    if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32) return fail(SWW_E_ARG, "blocks_per_sm must be 0..32");
    if (cfg->precision != SWW_FP64 && cfg->precision != SWW_FP32)
        return fail(SWW_E_ARG, "precision must be SWW_FP64 or SWW_FP32");
    if (cfg->mask != 0 && cfg->mask != 1) return fail(SWW_E_ARG, "mask must be 0 (candidate lists) or 1 (dense)");
    if (cfg->persistent != -1 && cfg->persistent != 0 && cfg->persistent != 3)
        return fail(SWW_E_ARG, "persistent must be -1, 0 or 3");
    if (!(cfg->nu >= 0)) return fail(SWW_E_ARG, "nu must be >= 0");
    return SWW_OK;
}

// A handle over levels cfg->jmin..cfg->jmax of `geo` (built here when null).
int create_handle(const sww_config* cfg, void* stream, std::shared_ptr<Geometry> geo, sww_handle** out) {
    sww_handle* h = new (std::nothrow) sww_handle();
    if (!h) return fail(SWW_E_POOL, "host allocation failed");
    int rc = guarded([&]() -> int {
        h->cfg = *cfg;
        h->user = static_cast<cudaStream_t>(stream);
        ck(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        ck(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "cudaEventCreate");
        ck(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming), "cudaEventCreate");
        int dev = 0;
        ck(cudaGetDevice(&dev), "cudaGetDevice");
        ck(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev), "device attribute");
        h->geo = geo ? geo : build_geometry(cfg->jmin, cfg->jmax, cfg->patch, cfg->radius, cfg->omega);
        const bool fp32 = cfg->precision == SWW_FP32;
        if (fp32) {
            h->geo->ensure_fp32();
            h->geo->ensure_tile_geo<float>();
        } else {
            h->geo->ensure_tile_geo<double>();
        }
        h->lv.assign(fp32 ? 0 : cfg->jmax + 1, DevLevelT<double>{});
        h->lvf.assign(fp32 ? cfg->jmax + 1 : 0, DevLevelT<float>{});
        h->grid_lv.assign(cfg->jmax + 1, 1);
        h->S = cfg->patch * cfg->patch;
        int64_t total = 0;
        // grid-stride launches: blocks_per_sm blocks of 256 per SM
        const int64_t cap = int64_t(h->nsm) * (cfg->blocks_per_sm > 0 ? cfg->blocks_per_sm : 4);
        for (int j = cfg->jmin; j <= cfg->jmax; ++j) {
            if (fp32)
                alloc_state<float>(h, j);
            else
                alloc_state<double>(h, j);
            int64_t items = (meta(h, j).npatch + 1) * h->S;
            h->grid_lv[j] = unsigned(std::min<int64_t>(blocks_for(items, 256), cap));
            total += meta(h, j).npatch + 1;
        }
        h->grid_all = unsigned(std::min<int64_t>(blocks_for(total * h->S, 256), cap));
        if (fp32) {
            h->d_lvs = h->alloc<DevLevelT<float>>(cfg->jmax + 1);
            ck(cudaMemcpy(h->d_lvs, h->lvf.data(), sizeof(DevLevelT<float>) * (cfg->jmax + 1), cudaMemcpyHostToDevice),
               "levels");
        } else {
            h->d_lvs = h->alloc<DevLevelT<double>>(cfg->jmax + 1);
            ck(cudaMemcpy(h->d_lvs, h->lv.data(), sizeof(DevLevelT<double>) * (cfg->jmax + 1), cudaMemcpyHostToDevice),
               "levels");
        }
        h->all_list = h->alloc<int32_t>(total);
        h->all_count = h->alloc<int32_t>(1);
        h->irr_list = h->alloc<int32_t>(total);
        h->irr_count = h->alloc<int32_t>(1);
        ck(cudaMemset(h->irr_count, 0, sizeof(int32_t)), "memset");
        h->total_entries = total;
        h->irr_bound = 0;
        for (int j = cfg->jmin; j <= cfg->jmax; ++j)
            h->irr_bound += (cfg->nu != 0.0 || cfg->advect) ? meta(h, j).npatch + 1 : h->geo->n_irr[j];
        h->cand = h->alloc<int32_t>(total);
        h->gcand = h->alloc<int32_t>(total);
        h->cand_count = h->alloc<int32_t>(1);
        h->gcand_count = h->alloc<int32_t>(1);
        ck(cudaMemset(h->cand_count, 0, sizeof(int32_t)), "memset");
        ck(cudaMemset(h->gcand_count, 0, sizeof(int32_t)), "memset");
        h->d_counts = h->alloc<int32_t>(2 * (cfg->jmax + 1));
        ck(cudaMemset(h->d_counts, 0, sizeof(int32_t) * 2 * (cfg->jmax + 1)), "memset");
        h->sig_any = h->alloc<int32_t>(cfg->jmax + 2);
        ck(cudaMemset(h->sig_any, 0, sizeof(int32_t) * (cfg->jmax + 2)), "memset");
        ck(cudaMallocHost(&h->h_counts, sizeof(int32_t) * 2 * (cfg->jmax + 1)), "cudaMallocHost");
        ck(cudaMallocHost(&h->h_dt, sizeof(double)), "cudaMallocHost");
        std::memset(h->h_counts, 0, sizeof(int32_t) * 2 * (cfg->jmax + 1));
        *h->h_dt = 0;
        h->red = h->alloc<unsigned long long>(RED_WORDS);
        ck(cudaMemset(h->red, 0, RED_WORDS * sizeof(unsigned long long)), "memset");
        h->d_net = h->alloc<MlpWeights>(1);
        ck(cudaMemset(h->d_net, 0, sizeof(MlpWeights)), "memset");
        h->lstat = h->alloc<unsigned long long>(4);
        ck(cudaMemset(h->lstat, 0, 4 * sizeof(unsigned long long)), "memset");
        h->bar = h->alloc<unsigned>(STAGE_BAR_WORDS);
        h->err = h->alloc<int>(1);
        ck(cudaMemset(h->bar, 0, STAGE_BAR_WORDS * sizeof(unsigned)), "memset");
        ck(cudaMemset(h->err, 0, sizeof(int)), "memset");
        ck(cudaMallocHost(&h->h_err, sizeof(int)), "cudaMallocHost");
        *h->h_err = 0;
        if (cfg->persistent >= 0 && cfg->jmax + 1 <= 12) {
            int coop = 0;
            ck(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev), "device attribute");
            if (coop) h->stage_cap = fp32 ? stage_grid<float>(h->S, h->nsm) : stage_grid<double>(h->S, h->nsm);
            h->stage_blocks = h->stage_cap;
        }
        h->cnt = h->alloc<unsigned long long>(STAT_WORDS);
        h->thr = h->alloc<double>(2);
        h->dt = h->alloc<double>(1);
        h->sums = h->alloc<double>(2);
        h->part = h->alloc<double>(4 * size_t(sums_blocks(meta(h, cfg->jmin))));
        ck(cudaMemset(h->thr, 0, 2 * sizeof(double)), "memset");
        ck(cudaMemset(h->dt, 0, sizeof(double)), "memset");
        ck(cudaMemset(h->all_count, 0, sizeof(int32_t)), "memset");
        h->jtop = cfg->jmax;
        // the handle's own member record (the fields its trend launches read are fixed)
        h->self_ref = h->alloc<uint8_t>(sizeof(MemberRef<double>));
        if (fp32) {
            MemberRef<float> r = member_ref<float>(h);
            ck(cudaMemcpy(h->self_ref, &r, sizeof(r), cudaMemcpyHostToDevice), "member record");
        } else {
            MemberRef<double> r = member_ref<double>(h);
            ck(cudaMemcpy(h->self_ref, &r, sizeof(r), cudaMemcpyHostToDevice), "member record");
        }
        ck(cudaDeviceSynchronize(), "create");
        return SWW_OK;
    });
    if (rc != SWW_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return SWW_OK;
}

}  // namespace

extern "C" {

int sww_create(const sww_config* cfg, void* stream, sww_handle** out) {
    if (!cfg || !out) return fail(SWW_E_ARG, "null argument");
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc) return rc;
    return create_handle(cfg, stream, nullptr, out);
}

int sww_create_shared(const sww_config* cfg, void* stream, const sww_handle* share, sww_handle** out) {
    if (!cfg || !out || !share) return fail(SWW_E_ARG, "null argument");
    *out = nullptr;
    int rc = check_config(cfg);
    if (rc) return rc;
    const Geometry& G = *share->geo;
    if (cfg->jmin != G.jmin || cfg->patch != G.patch || cfg->radius != G.radius || cfg->omega != G.omega)
        return fail(SWW_E_ARG, "shared grid needs the same jmin, patch, radius and omega");
    if (cfg->jmax > G.jmax) return fail(SWW_E_ARG, "shared grid has fewer levels than jmax");
    return create_handle(cfg, stream, share->geo, out);
}

int sww_destroy(sww_handle* h) {
    if (!h) return SWW_OK;
    delete h;
    return SWW_OK;
}

int sww_level_sizes(const sww_handle* h, int level, int64_t* nn, int64_t* ne, int64_t* nt, int64_t* np) {
    int rc = check_level(h, level);
    if (rc) return rc;
    const DevLevel& L = meta(h, level);
    if (nn) *nn = L.N;
    if (ne) *ne = L.E;
    if (nt) *nt = L.T;
    if (np) *np = L.npatch;
    return SWW_OK;
}

int sww_get_grid(const sww_handle* h, int level, double* node_xyz, int32_t* edge_nodes) {
    int rc = check_level(h, level);
    if (rc) return rc;
    const Geometry& G = *h->geo;
    if (node_xyz) std::memcpy(node_xyz, G.xyz[level].data(), G.xyz[level].size() * sizeof(double));
    if (edge_nodes) std::memcpy(edge_nodes, G.edges[level].data(), G.edges[level].size() * sizeof(int32_t));
    return SWW_OK;
}

// Fields on the full level J; coarser levels get their restriction, every point
// of levels Jmin..J becomes live and the levels above J are empty.
static int set_state_at(sww_handle* h, const double* dh, const double* u, int J, int device_ptrs) {
    return guarded([&]() -> int {
        const int j0 = h->cfg.jmin, j1 = h->cfg.jmax;
        cudaStream_t s = h->stream;
        const int64_t NJ = meta(h, J).N, EJ = meta(h, J).E;
        // host fields: both copied into the FP64 staging buffer and checked there for
        // a non-finite value (one kernel, one read-back), refused before the state
        // changes; the state is then filled from the staging buffer
        const bool staged = !device_ptrs;
        if (staged) {
            if (!h->stage) h->stage = h->alloc<double>(meta(h, j1).N + meta(h, j1).E);
            unsigned bad = 0;
            {
                Join jn(h);
                ck(cudaMemcpyAsync(h->stage, dh, NJ * sizeof(double), cudaMemcpyHostToDevice, s), "set_state dh");
                ck(cudaMemcpyAsync(h->stage + NJ, u, EJ * sizeof(double), cudaMemcpyHostToDevice, s), "set_state u");
                unsigned* flag = reinterpret_cast<unsigned*>(h->cnt);
                ck(cudaMemsetAsync(flag, 0, sizeof(unsigned), s), "memset flag");
                count_launch(1);
                k_nonfinite<<<unsigned(std::min<int64_t>((NJ + EJ + 255) / 256, 4 * int64_t(h->nsm))), 256, 0, s>>>(
                    h->stage, NJ + EJ, flag);
                ck(cudaMemcpyAsync(&bad, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "flag");
                check_launch();
            }
            ck(cudaStreamSynchronize(s), "set_state check");
            if (bad) return fail(SWW_E_NUMERIC, "non-finite value in the initial fields");
            dh = h->stage;
            u = h->stage + NJ;
        }
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            auto& lv = lvl<R>(h);
            DevLevelT<R>& F = lv[J];
            if constexpr (std::is_same<R, double>::value) {
                ck(cudaMemcpyAsync(F.dh, dh, F.N * sizeof(double), cudaMemcpyDeviceToDevice, s), "set_state dh");
                ck(cudaMemcpyAsync(F.u, u, F.E * sizeof(double), cudaMemcpyDeviceToDevice, s), "set_state u");
            } else if (staged) {
                // FP64 input rounded once to the working precision
                launch_convert(dh, F.dh, F.N, s);
                launch_convert(u, F.u, F.E, s);
            } else {
                if (!h->stage) h->stage = h->alloc<double>(meta(h, j1).N + meta(h, j1).E);
                ck(cudaMemcpyAsync(h->stage, dh, F.N * sizeof(double), cudaMemcpyDeviceToDevice, s), "set_state dh");
                launch_convert(h->stage, F.dh, F.N, s);
                ck(cudaMemcpyAsync(h->stage, u, F.E * sizeof(double), cudaMemcpyDeviceToDevice, s), "set_state u");
                launch_convert(h->stage, F.u, F.E, s);
            }
            for (int j = J; j > j0; --j) launch_restrict_full(lv[j - 1], lv[j], s);
            MaskArgsT<R> a = mask_args<R>(h, j0, J, false);
            launch_live_all(dlv<R>(h), a.nodes, a.edges, s);
            for (int j = J + 1; j <= j1; ++j) {
                const DevLevelT<R>& L = lv[j];
                ck(cudaMemsetAsync(L.nflag, 0, L.N, s), "memset flags");
                ck(cudaMemsetAsync(L.eflag, 0, L.E, s), "memset flags");
                ck(cudaMemsetAsync(L.dh, 0, L.N * sizeof(R), s), "memset state");
                ck(cudaMemsetAsync(L.u, 0, L.E * sizeof(R), s), "memset state");
            }
            // the list-based mask expects the band bytes zero away from its candidates
            for (int j = j0; j <= j1; ++j) {
                ck(cudaMemsetAsync(lv[j].band0, 0, lv[j].N, s), "memset band");
                ck(cudaMemsetAsync(lv[j].band1, 0, lv[j].N, s), "memset band");
            }
            if (J > j0) launch_covered_all(dlv<R>(h), a.nodes_c, s);
            MaskArgsT<R> b = mask_args<R>(h, j0, j1, false);
            launch_patches_all(dlv<R>(h), b.patches, s);
            launch_concat(dlv<R>(h), j0, j1, h->all_list, h->all_count, h->irr_list, h->irr_count, h->S, h->grid_all, s);
            read_counts<R>(h);
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(s), "set_state");
        update_top(h);
        h->has_state = true;
        h->t = 0;
        h->steps = 0;
        return SWW_OK;
    });
}

int sww_set_state(sww_handle* h, const double* dh, const double* u, int device_ptrs) {
    if (!h || !dh || !u) return fail(SWW_E_ARG, "null argument");
    return sww_set_state_level(h, h->cfg.jmax, dh, u, device_ptrs);
}

int sww_set_state_level(sww_handle* h, int level, const double* dh, const double* u, int device_ptrs) {
    if (!h || !dh || !u) return fail(SWW_E_ARG, "null argument");
    int rc = check_level(h, level);
    if (rc) return rc;
    if (h->cfg.advect && level != h->cfg.jmax)
        return fail(SWW_E_ARG, "a prescribed velocity is set on Jmax (it holds on every level)");
    return set_state_at(h, dh, u, level, device_ptrs);
}

int sww_adapt(sww_handle* h, double eps_h, double eps_u) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            adapt<R>(h, eps_h, eps_u);
            read_counts<R>(h);
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(h->stream), "adapt");
        update_top(h);
        return SWW_OK;
    });
}

int sww_mask_from_coeffs(sww_handle* h, const double* hdet, const double* udet_e, const double* udet_i, double eps_h,
                         double eps_u) {
    if (!h || !hdet || !udet_e || !udet_i) return fail(SWW_E_ARG, "null argument");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    if (!(eps_h > 0) || !(eps_u > 0)) return fail(SWW_E_ARG, "explicit positive thresholds required");
    return guarded([&]() -> int {
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            auto& lv = lvl<R>(h);
            size_t oh = 0, oe = 0, oi = 0;
            for (int j = h->cfg.jmin + 1; j <= h->cfg.jmax; ++j) {
                DevLevelT<R>& F = lv[j];
                int64_t ce = lv[j - 1].E;
                to_device(h, F.hdet, hdet + oh, F.N);
                to_device(h, F.ue, udet_e + oe, ce);
                to_device(h, F.ui, udet_i + oi, F.E);
                oh += F.N, oe += ce, oi += F.E;
            }
            double th[2] = {eps_h, eps_u};
            ck(cudaMemcpyAsync(h->thr, th, sizeof(th), cudaMemcpyHostToDevice, h->stream), "thr");
            ck(cudaStreamSynchronize(h->stream), "thr");   // th lives on this host stack frame
            mask_and_inverse<R>(h);
            read_counts<R>(h);
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(h->stream), "mask");
        update_top(h);
        return SWW_OK;
    });
}

int sww_rhs(sww_handle* h) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            RKStage none{0, 0, 0, 0, 0, 0, 0};
            stage<R>(h, none);
            ck(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "err");
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(h->stream), "rhs");
        return barrier_status(h);
    });
}

int sww_step(sww_handle* h, double dt, int nsteps, int do_adapt) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    if (nsteps < 0) return fail(SWW_E_ARG, "nsteps < 0");
    return guarded([&]() -> int {
        for (int s = 0; s < nsteps; ++s) {
            {
                Join jn(h);
                run_step(h, dt, do_adapt != 0);
                check_launch();
            }
            ck(cudaStreamSynchronize(h->stream), "step");
            if (int rc = barrier_status(h)) return rc;
            double d = *h->h_dt;
            if (!std::isfinite(d) || !(d > 0)) return fail(SWW_E_NUMERIC, "non-finite or non-positive time step");
            h->t += d;
            h->last_dt = d;
            h->steps += 1;
            update_top(h);
        }
        return SWW_OK;
    });
}

int sww_step_ensemble(sww_handle* const* hs, int n, double dt, int nsteps, int do_adapt) {
    if (!hs || n < 0 || nsteps < 0) return fail(SWW_E_ARG, "bad argument");
    for (int i = 0; i < n; ++i) {
        if (!hs[i]) return fail(SWW_E_ARG, "null handle");
        if (!hs[i]->has_state) return fail(SWW_E_STATE, "sww_set_state first");
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return fail(SWW_E_ARG, "a handle appears twice");
    }
    if (n == 0 || nsteps == 0) return SWW_OK;
    // the whole step batched over the members but their masks, one regular launch
    // per phase over all members, when every member asks for it (persistent = 3)
    // and they share precision, Jmin, patch side, depth, gravity and scheme;
    // otherwise the members' whole steps overlap on their own streams
    bool batched = n > 1 && n <= 128 && hs[0]->cfg.persistent == 3;
    for (int i = 0; i < n && batched; ++i) {
        const sww_config &a = hs[0]->cfg, &b = hs[i]->cfg;
        batched = b.persistent == 3 && a.precision == b.precision && a.jmin == b.jmin && a.patch == b.patch &&
                  a.H == b.H && a.g == b.g && a.rk == b.rk;
    }
    return guarded([&]() -> int {
        for (int i = 0; i < n; ++i) {
            sww_handle* h = hs[i];
            ck(cudaEventRecord(h->ev_in, h->user), "join in");
            ck(cudaStreamWaitEvent(h->stream, h->ev_in, 0), "join in");
        }
        auto finish = [&](sww_handle* h) -> int {
            ck(cudaStreamSynchronize(h->stream), "step");
            if (int rc = barrier_status(h)) return rc;
            double d = *h->h_dt;
            if (!std::isfinite(d) || !(d > 0)) return fail(SWW_E_NUMERIC, "non-finite or non-positive time step");
            h->t += d;
            h->last_dt = d;
            h->steps += 1;
            update_top(h);
            return SWW_OK;
        };
        auto join_out = [&]() {
            for (int i = 0; i < n; ++i) {
                sww_handle* h = hs[i];
                ck(cudaEventRecord(h->ev_out, h->stream), "join out");
                ck(cudaStreamWaitEvent(h->user, h->ev_out, 0), "join out");
            }
        };
        int rc = SWW_OK;
        if (batched) {
            for (int s = 0; s < nsteps && rc == SWW_OK; ++s) {
                by_prec(hs[0], [&](auto r) {
                    ensemble_phased<decltype(r)>(hs, n, dt, do_adapt != 0);
                    return 0;
                });
                check_launch();
                ck(cudaStreamSynchronize(hs[0]->stream), "step");
                const BatchOut* o = reinterpret_cast<const BatchOut*>(hs[0]->ens.h_out);
                for (int i = 0; i < n && rc == SWW_OK; ++i) {
                    sww_handle* h = hs[i];
                    *h->h_dt = o[i].dt;
                    *h->h_err = o[i].err;
                    for (int j = 0; j <= h->cfg.jmax && j < 16; ++j) {
                        h->h_counts[j] = o[i].counts[j];
                        h->h_counts[h->cfg.jmax + 1 + j] = o[i].live[j];
                    }
                    rc = finish(h);
                }
            }
            join_out();
            return rc;
        }
        // otherwise every member's step is one graph launch on the member's own
        // stream, the members advancing in turn, each waiting only for its own
        // previous step.  Cooperative launches of different streams do not overlap,
        // so a member's RK stage runs as one launch per phase
        std::vector<unsigned> own(n);
        for (int i = 0; i < n; ++i) {
            own[i] = hs[i]->stage_blocks;
            if (n > 1) hs[i]->stage_blocks = 0;
        }
        struct Restore {
            sww_handle* const* hs;
            std::vector<unsigned>& own;
            ~Restore() {
                for (size_t i = 0; i < own.size(); ++i) hs[i]->stage_blocks = own[i];
            }
        } restore{hs, own};
        auto launch = [&](sww_handle* h) {
            run_step(h, dt, do_adapt != 0);
            check_launch();
        };
        for (int i = 0; i < n; ++i) launch(hs[i]);
        for (int s = 1; s < nsteps && rc == SWW_OK; ++s)
            for (int i = 0; i < n && rc == SWW_OK; ++i) {
                rc = finish(hs[i]);
                if (rc == SWW_OK) launch(hs[i]);
            }
        for (int i = 0; i < n; ++i) {
            int r = finish(hs[i]);
            if (rc == SWW_OK) rc = r;
        }
        join_out();
        return rc;
    });
}

int sww_get_level(const sww_handle* h, int level, int what, void* out) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!out) return fail(SWW_E_ARG, "null output");
    if (what == SWW_UDET_E && level == h->cfg.jmin) return fail(SWW_E_ARG, "no coefficients on Jmin");
    if (what < SWW_DH || what > SWW_SIG) return fail(SWW_E_ARG, "unknown quantity");
    sww_handle* hh = const_cast<sww_handle*>(h);
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            const DevLevelT<R>& L = lvl<R>(h)[level];
            const R* field = nullptr;
            int64_t n = 0;
            const uint8_t* bytes = nullptr;
            switch (what) {
                case SWW_DH: field = L.dh, n = L.N; break;
                case SWW_U: field = L.u, n = L.E; break;
                case SWW_DH_T: field = L.dht, n = L.N; break;
                case SWW_U_T: field = L.ut, n = L.E; break;
                case SWW_HDET: field = L.hdet, n = L.N; break;
                case SWW_UDET_E: field = L.ue, n = meta(h, level - 1).E; break;
                case SWW_UDET_I: field = L.ui, n = L.E; break;
                case SWW_NODE_FLAGS: bytes = L.nflag, n = L.N; break;
                case SWW_EDGE_FLAGS: bytes = L.eflag, n = L.E; break;
                case SWW_SIG: bytes = L.sig, n = L.N; break;
            }
            if (bytes) {
                {
                    Join jn(hh);
                    ck(cudaMemcpyAsync(out, bytes, n, cudaMemcpyDeviceToHost, hh->stream), "get_level");
                }
                ck(cudaStreamSynchronize(hh->stream), "get_level");
            } else {
                from_device(hh, static_cast<double*>(out), field, n);
            }
            return SWW_OK;
        });
    });
}

int sww_get_mask(const sww_handle* h, int level, uint8_t* nodes, uint8_t* edges) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (nodes && (rc = sww_get_level(h, level, SWW_NODE_FLAGS, nodes))) return rc;
    if (edges && (rc = sww_get_level(h, level, SWW_EDGE_FLAGS, edges))) return rc;
    return SWW_OK;
}

int sww_set_level(sww_handle* h, int level, const double* dh, const double* u) {
    int rc = check_level(h, level);
    if (rc) return rc;
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            const DevLevelT<R>& L = lvl<R>(h)[level];
            {
                Join jn(h);
                if (dh) to_device(h, L.dh, dh, L.N);
                if (u) to_device(h, L.u, u, L.E);
            }
            ck(cudaStreamSynchronize(h->stream), "set_level");
            return SWW_OK;
        });
    });
}

int sww_forward(sww_handle* h) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            Trace t(h, SWW_K_COEFF);
            launch_details(work_all<R>(h), h->cfg.jmin, h->stream);
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(h->stream), "forward");
        return SWW_OK;
    });
}

int sww_inverse(sww_handle* h) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        by_prec(h, [&](auto r) {
            using R = decltype(r);
            Join jn(h);
            auto& lv = lvl<R>(h);
            cudaStream_t s = h->stream;
            launch_mark_support(work_all<R>(h), s);
            for (int j = h->cfg.jmin + 1; j <= h->jtop; ++j) {
                { Trace t(h, SWW_K_INVERSE); launch_inverse(lv[j], lv[j - 1], work_level<R>(h, j), s); }
                { Trace t(h, SWW_K_FILL); launch_fill(lv[j], lv[j - 1], work_level<R>(h, j), s); }
            }
            check_launch();
            return 0;
        });
        ck(cudaStreamSynchronize(h->stream), "inverse");
        return SWW_OK;
    });
}

int sww_get_coeffs(const sww_handle* h, int level, double* hdet, double* udet_e, double* udet_i) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (level == h->cfg.jmin) return fail(SWW_E_ARG, "no coefficients on Jmin");
    if (hdet && (rc = sww_get_level(h, level, SWW_HDET, hdet))) return rc;
    if (udet_e && (rc = sww_get_level(h, level, SWW_UDET_E, udet_e))) return rc;
    if (udet_i && (rc = sww_get_level(h, level, SWW_UDET_I, udet_i))) return rc;
    return SWW_OK;
}

int sww_set_coeffs(sww_handle* h, int level, const double* hdet, const double* udet_e, const double* udet_i) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (level == h->cfg.jmin) return fail(SWW_E_ARG, "no coefficients on Jmin");
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            const DevLevelT<R>& L = lvl<R>(h)[level];
            {
                Join jn(h);
                if (hdet) to_device(h, L.hdet, hdet, L.N);
                if (udet_e) to_device(h, L.ue, udet_e, meta(h, level - 1).E);
                if (udet_i) to_device(h, L.ui, udet_i, L.E);
            }
            ck(cudaStreamSynchronize(h->stream), "set_coeffs");
            return SWW_OK;
        });
    });
}

int sww_get_state(sww_handle* h, int level, double* dh, double* u) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            auto& lv = lvl<R>(h);
            const int j0 = h->cfg.jmin;
            // the full levels above Jmin go to the RK base arrays, which hold nothing
            // between steps; Jmin is always full
            {
                Join jn(h);
                for (int j = j0 + 1; j <= level; ++j) {
                    const R* cdh = j - 1 == j0 ? lv[j0].dh : lv[j - 1].dh0;
                    const R* cu = j - 1 == j0 ? lv[j0].u : lv[j - 1].u0;
                    launch_uniform(lv[j], lv[j - 1], cdh, cu, lv[j].dh0, lv[j].u0, h->stream);
                }
                check_launch();
            }
            const DevLevelT<R>& L = lv[level];
            if (dh) from_device(h, dh, level == j0 ? L.dh : L.dh0, L.N);
            if (u) from_device(h, u, level == j0 ? L.u : L.u0, L.E);
            ck(cudaStreamSynchronize(h->stream), "get_state");
            return SWW_OK;
        });
    });
}

// ---------------------------------------------------------------- checkpoints
// File: "SWWCKPT1", then the header below, then per level Jmin..Jmax the depth,
// velocity (working precision), node flags and edge flags, then "SWWCKEND".
namespace {
struct CkptHeader {
    uint32_t version, precision;
    int32_t jmin, jmax, patch, reserved;
    double radius, omega, t, dt, eps_h, eps_u;
    int64_t steps;
};
const char CKPT_MAGIC[8] = {'S', 'W', 'W', 'C', 'K', 'P', 'T', '1'};
const char CKPT_END[8] = {'S', 'W', 'W', 'C', 'K', 'E', 'N', 'D'};

struct File {
    FILE* f;
    File(const char* path, const char* mode) : f(std::fopen(path, mode)) {}
    ~File() {
        if (f) std::fclose(f);
    }
    bool put(const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
    bool get(void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
};
}  // namespace

int sww_save(const sww_handle* hc, const char* path) {
    if (!hc || !path) return fail(SWW_E_ARG, "null argument");
    if (!hc->has_state) return fail(SWW_E_STATE, "nothing to save before sww_set_state");
    sww_handle* h = const_cast<sww_handle*>(hc);
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            File out(path, "wb");
            if (!out.f) return fail(SWW_E_ARG, std::string("cannot open ") + path);
            double thr[2];
            {
                Join jn(h);
                ck(cudaMemcpyAsync(thr, h->thr, sizeof(thr), cudaMemcpyDeviceToHost, h->stream), "save thr");
            }
            ck(cudaStreamSynchronize(h->stream), "save");
            CkptHeader hd{1u, uint32_t(h->cfg.precision), h->cfg.jmin, h->cfg.jmax, h->cfg.patch, 0,
                          h->cfg.radius, h->cfg.omega, h->t, h->last_dt, thr[0], thr[1], h->steps};
            bool ok = out.put(CKPT_MAGIC, 8) && out.put(&hd, sizeof(hd));
            std::vector<R> buf;
            std::vector<uint8_t> bytes;
            for (int j = h->cfg.jmin; ok && j <= h->cfg.jmax; ++j) {
                const DevLevelT<R>& L = lvl<R>(h)[j];
                const int64_t ne[2] = {L.N, L.E};
                ok = out.put(ne, sizeof(ne));
                const R* fields[2] = {L.dh, L.u};
                const uint8_t* flags[2] = {L.nflag, L.eflag};
                for (int k = 0; ok && k < 2; ++k) {
                    buf.resize(size_t(ne[k]));
                    ck(cudaMemcpyAsync(buf.data(), fields[k], ne[k] * sizeof(R), cudaMemcpyDeviceToHost, h->stream),
                       "save field");
                    ck(cudaStreamSynchronize(h->stream), "save field");
                    ok = out.put(buf.data(), ne[k] * sizeof(R));
                }
                for (int k = 0; ok && k < 2; ++k) {
                    bytes.resize(size_t(ne[k]));
                    ck(cudaMemcpyAsync(bytes.data(), flags[k], ne[k], cudaMemcpyDeviceToHost, h->stream), "save flags");
                    ck(cudaStreamSynchronize(h->stream), "save flags");
                    ok = out.put(bytes.data(), ne[k]);
                }
            }
            ok = ok && out.put(CKPT_END, 8);
            if (!ok) return fail(SWW_E_ARG, std::string("write failed: ") + path);
            return SWW_OK;
        });
    });
}

int sww_load(sww_handle* h, const char* path) {
    if (!h || !path) return fail(SWW_E_ARG, "null argument");
    return guarded([&]() -> int {
        return by_prec(h, [&](auto r) -> int {
            using R = decltype(r);
            File in(path, "rb");
            if (!in.f) return fail(SWW_E_ARG, std::string("cannot open ") + path);
            char magic[8];
            CkptHeader hd{};
            if (!in.get(magic, 8) || std::memcmp(magic, CKPT_MAGIC, 8) || !in.get(&hd, sizeof(hd)) || hd.version != 1)
                return fail(SWW_E_ARG, "not a checkpoint of this library");
            if (hd.precision != uint32_t(h->cfg.precision) || hd.jmin != h->cfg.jmin || hd.jmax != h->cfg.jmax ||
                hd.patch != h->cfg.patch || hd.radius != h->cfg.radius || hd.omega != h->cfg.omega)
                return fail(SWW_E_ARG, "checkpoint grid or precision differs from the handle's");
            // read everything before touching the device state
            const int j0 = h->cfg.jmin, j1 = h->cfg.jmax;
            std::vector<std::vector<R>> fld(2 * (j1 + 1));
            std::vector<std::vector<uint8_t>> flg(2 * (j1 + 1));
            for (int j = j0; j <= j1; ++j) {
                const DevLevelT<R>& L = lvl<R>(h)[j];
                int64_t ne[2];
                if (!in.get(ne, sizeof(ne)) || ne[0] != L.N || ne[1] != L.E)
                    return fail(SWW_E_ARG, "checkpoint level sizes differ");
                for (int k = 0; k < 2; ++k) {
                    fld[2 * j + k].resize(size_t(ne[k]));
                    if (!in.get(fld[2 * j + k].data(), ne[k] * sizeof(R))) return fail(SWW_E_ARG, "truncated checkpoint");
                }
                for (int k = 0; k < 2; ++k) {
                    flg[2 * j + k].resize(size_t(ne[k]));
                    if (!in.get(flg[2 * j + k].data(), ne[k])) return fail(SWW_E_ARG, "truncated checkpoint");
                }
            }
            if (!in.get(magic, 8) || std::memcmp(magic, CKPT_END, 8)) return fail(SWW_E_ARG, "truncated checkpoint");
            cudaStream_t s = h->stream;
            {
                Join jn(h);
                auto& lv = lvl<R>(h);
                for (int j = j0; j <= j1; ++j) {
                    const DevLevelT<R>& L = lv[j];
                    ck(cudaMemcpyAsync(L.dh, fld[2 * j].data(), L.N * sizeof(R), cudaMemcpyHostToDevice, s), "load");
                    ck(cudaMemcpyAsync(L.u, fld[2 * j + 1].data(), L.E * sizeof(R), cudaMemcpyHostToDevice, s), "load");
                    ck(cudaMemcpyAsync(L.nflag, flg[2 * j].data(), L.N, cudaMemcpyHostToDevice, s), "load");
                    ck(cudaMemcpyAsync(L.eflag, flg[2 * j + 1].data(), L.E, cudaMemcpyHostToDevice, s), "load");
                    // per-mask scratch starts clean (the list mask expects it zero away
                    // from its candidates)
                    uint8_t* nbytes[] = {L.sig, L.tmask, L.band0, L.band1};
                    for (auto p : nbytes) ck(cudaMemsetAsync(p, 0, L.N, s), "load scratch");
                    uint8_t* pbytes[] = {L.zflag, L.sflag, L.cflag, L.lflag, L.gflag, L.prop, L.prop_prev, L.pexact};
                    for (auto p : pbytes) ck(cudaMemsetAsync(p, 0, L.npatch + 1, s), "load scratch");
                }
                ck(cudaMemsetAsync(h->cand_count, 0, sizeof(int32_t), s), "load scratch");
                ck(cudaMemsetAsync(h->gcand_count, 0, sizeof(int32_t), s), "load scratch");
                const double thr[2] = {hd.eps_h, hd.eps_u};
                ck(cudaMemcpyAsync(h->thr, thr, sizeof(thr), cudaMemcpyHostToDevice, s), "load thr");
                MaskArgsT<R> a = mask_args<R>(h, j0, j1, false);
                launch_patches_all(dlv<R>(h), a.patches, s);
                launch_concat(dlv<R>(h), j0, j1, h->all_list, h->all_count, h->irr_list, h->irr_count, h->S, h->grid_all, s);
                read_counts<R>(h);
                check_launch();
                ck(cudaStreamSynchronize(s), "load");   // host buffers live on this frame
            }
            update_top(h);
            h->has_state = true;
            h->t = hd.t;
            h->last_dt = hd.dt;
            h->steps = hd.steps;
            return SWW_OK;
        });
    });
}

int sww_live_nodes(const sww_handle* h, int64_t* total) {
    if (!h || !total) return fail(SWW_E_ARG, "null argument");
    int64_t n = 0;
    for (int j = h->cfg.jmin; j <= h->cfg.jmax; ++j) n += h->h_counts[h->cfg.jmax + 1 + j];
    *total = h->has_state ? n : 0;
    return SWW_OK;
}

int sww_get_patches(const sww_handle* h, int level, int32_t* out, int32_t* count) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!count) return fail(SWW_E_ARG, "null count");
    sww_handle* hh = const_cast<sww_handle*>(h);
    return guarded([&]() -> int {
        const int32_t* patches = nullptr;
        const int32_t* npatches = nullptr;
        by_prec(h, [&](auto r) {
            const auto& L = lvl<decltype(r)>(h)[level];
            patches = L.patches, npatches = L.npatches;
            return 0;
        });
        const DevLevel& L = meta(h, level);
        int32_t n = 0;
        std::vector<int32_t> tmp(L.npatch + 1);
        {
            Join jn(hh);
            ck(cudaMemcpyAsync(&n, npatches, sizeof(int32_t), cudaMemcpyDeviceToHost, hh->stream), "npatches");
            ck(cudaMemcpyAsync(tmp.data(), patches, tmp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, hh->stream),
               "patches");
        }
        ck(cudaStreamSynchronize(hh->stream), "patches");
        int32_t c = 0;
        for (int32_t i = 0; i < n; ++i) {
            int32_t p = tmp[i] & PATCH_MASK;
            if (p == L.npatch) continue;   // pole entry
            if (out) out[c] = p;
            ++c;
        }
        *count = c;
        return SWW_OK;
    });
}

int sww_stats_get(sww_handle* h, sww_stats* st) {
    if (!h || !st) return fail(SWW_E_ARG, "null argument");
    return guarded([&]() -> int {
        std::memset(st, 0, sizeof(*st));
        const int j0 = h->cfg.jmin, j1 = std::min(h->cfg.jmax, 15);
        // every level's counts, the active patch counts, the Jmin sums and the
        // thresholds on the handle's stream, read back with one synchronisation
        unsigned long long c[STAT_WORDS];
        double s[2], th[2];
        {
            Join jn(h);
            ck(cudaMemsetAsync(h->cnt, 0, STAT_WORDS * sizeof(unsigned long long), h->stream), "memset cnt");
            by_prec(h, [&](auto r) {
                using R = decltype(r);
                for (int j = j0; j <= j1; ++j) launch_count(lvl<R>(h)[j], h->cnt + 3 * j, h->stream);
                count_launch(1);
                k_stat_patches<R><<<1, 32, 0, h->stream>>>(dlv<R>(h), j0, j1, h->cnt + STAT_PATCHES);
                launch_sums(lvl<R>(h)[j0], h->cfg.H, h->cfg.g, h->part, h->sums, h->stream);
                return 0;
            });
            ck(cudaMemcpyAsync(c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "cnt");
            ck(cudaMemcpyAsync(s, h->sums, sizeof(s), cudaMemcpyDeviceToHost, h->stream), "sums");
            ck(cudaMemcpyAsync(th, h->thr, sizeof(th), cudaMemcpyDeviceToHost, h->stream), "thr");
            check_launch();
        }
        ck(cudaStreamSynchronize(h->stream), "stats");
        for (int j = j0; j <= j1; ++j) {
            st->live_nodes[j] = int64_t(c[3 * j]);
            st->ghost_nodes[j] = int64_t(c[3 * j + 1]);
            st->live_edges[j] = int64_t(c[3 * j + 2]);
            st->active_patches[j] = int64_t(c[STAT_PATCHES + j]);
        }
        double AS = 4.0 * M_PI * h->cfg.radius * h->cfg.radius;
        double c2 = h->cfg.g * s[0] / AS;
        st->mass = s[0];
        st->energy = s[1] - 0.5 * c2 * c2 * AS;
        st->eps_h = th[0];
        st->eps_u = th[1];
        st->t = h->t;
        st->dt = h->last_dt;
        st->steps = h->steps;
        st->kernel_launches = kernel_launches();
        return SWW_OK;
    });
}

int sww_set_learned(sww_handle* h, int mode, const float* params, float tau) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (mode < 0 || mode > 2) return fail(SWW_E_ARG, "mode must be 0, 1 or 2");
    if (mode == 2 && (!params || !(tau > 0.f) || !(tau < 1.f))) return fail(SWW_E_ARG, "mode 2 needs params and 0 < tau < 1");
    return guarded([&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "set_learned");
        h->learn_mode = mode;
        h->tau = tau;
        if (params) {
            h->net = mlp_weights(params);
            ck(cudaMemcpy(h->d_net, &h->net, sizeof(MlpWeights), cudaMemcpyHostToDevice), "weights");
        }
        h->drop_graphs();
        return SWW_OK;
    });
}

int sww_propose(sww_handle* h, int level, const uint8_t* flags) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!flags) return fail(SWW_E_ARG, "null flags");
    if (level == h->cfg.jmin) return fail(SWW_E_ARG, "Jmin is always complete");
    return guarded([&]() -> int {
        uint8_t* prop = nullptr;
        by_prec(h, [&](auto r) {
            prop = lvl<decltype(r)>(h)[level].prop;
            return 0;
        });
        {
            Join jn(h);
            ck(cudaMemcpyAsync(prop, flags, meta(h, level).npatch + 1, cudaMemcpyHostToDevice, h->stream), "propose");
        }
        ck(cudaStreamSynchronize(h->stream), "propose");
        return SWW_OK;
    });
}

int sww_get_patch_data(const sww_handle* h, int level, int what, void* out) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!out) return fail(SWW_E_ARG, "null output");
    sww_handle* hh = const_cast<sww_handle*>(h);
    return guarded([&]() -> int {
        const void* src = nullptr;
        size_t bytes = 0;
        const int64_t np1 = meta(h, level).npatch + 1;
        by_prec(h, [&](auto r) {
            const auto& L = lvl<decltype(r)>(h)[level];
            switch (what) {
                case SWW_P_FEATURES: src = L.pfeat, bytes = NF * np1 * sizeof(float); break;
                case SWW_P_EXACT: src = L.pexact, bytes = np1; break;
                case SWW_P_PROPOSAL: src = L.prop_prev, bytes = np1; break;
                case SWW_P_ACTIVE: src = L.pflag, bytes = np1 - 1; break;
            }
            return 0;
        });
        if (!src) return fail(SWW_E_ARG, "unknown patch quantity");
        {
            Join jn(hh);
            ck(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, hh->stream), "patch data");
        }
        ck(cudaStreamSynchronize(hh->stream), "patch data");
        return SWW_OK;
    });
}

int sww_learn_stats(sww_handle* h, int64_t* out, int reset) {
    if (!h || !out) return fail(SWW_E_ARG, "null argument");
    return guarded([&]() -> int {
        unsigned long long c[3] = {0, 0, 0};
        {
            Join jn(h);
            ck(cudaMemcpyAsync(c, h->lstat, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "learn stats");
            if (reset) ck(cudaMemsetAsync(h->lstat, 0, sizeof(c), h->stream), "learn stats");
        }
        ck(cudaStreamSynchronize(h->stream), "learn stats");
        for (int k = 0; k < 3; ++k) out[k] = int64_t(c[k]);
        return SWW_OK;
    });
}

int sww_barrier_fault(sww_handle* h, long long spin_cycles, int skip_block) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (spin_cycles < 0) return fail(SWW_E_ARG, "spin_cycles < 0");
    return guarded([&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "barrier fault");
        h->spin_cycles = spin_cycles;
        h->skip_block = skip_block < 0 ? -1 : skip_block;
        h->drop_graphs();   // captured steps hold the stage arguments
        return SWW_OK;
    });
}

int sww_profile(sww_handle* h, uint32_t class_mask) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    return guarded([&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "profile");
        for (auto& r : h->recs) h->ev_pool.push_back(r.a), h->ev_pool.push_back(r.b);
        h->recs.clear();
        h->prof_mask = class_mask;
        return SWW_OK;
    });
}

int sww_profile_read(sww_handle* h, double* ms, int64_t* launches) {
    if (!h || !ms || !launches) return fail(SWW_E_ARG, "null argument");
    return guarded([&]() -> int {
        ck(cudaStreamSynchronize(h->stream), "profile_read");
        for (int k = 0; k < SWW_K_NCLASS; ++k) ms[k] = 0, launches[k] = 0;
        for (auto& r : h->recs) {
            float t = 0;
            ck(cudaEventElapsedTime(&t, r.a, r.b), "cudaEventElapsedTime");
            ms[r.cls] += t;
            launches[r.cls] += r.launches;
            h->ev_pool.push_back(r.a), h->ev_pool.push_back(r.b);
        }
        h->recs.clear();
        return SWW_OK;
    });
}

int sww_last_error(char* buf, size_t len) {
    if (!buf || len == 0) return SWW_E_ARG;
    std::snprintf(buf, len, "%s", g_err.c_str());
    return SWW_OK;
}

}  // extern "C"

namespace sww {

bool handle_view(const sww_handle* h, HandleView* v) {
    if (!h || !v) return false;
    v->jmin_level = &h->geo->lv[h->cfg.jmin];   // FP64 geometry of Jmin
    v->stream = h->user;
    v->radius = h->cfg.radius;
    v->g = h->cfg.g;
    v->H = h->cfg.H;
    return true;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

}  // namespace sww
