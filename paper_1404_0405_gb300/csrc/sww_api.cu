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
#include <new>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "grid.h"
#include "sww.h"
#include "sww_core.cuh"
#include "sww_internal.h"
#include "sww_kernels.h"

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

__global__ void k_reset_red(unsigned long long* red) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        red[0] = 0ull;
        red[1] = ~0ull;
    }
}

__global__ void k_gather_counts(const DevLevel* lvs, int jmin, int jmax, int32_t* out) {
    int j = jmin + int(threadIdx.x);
    if (j <= jmax) out[j] = *lvs[j].npatches;
}

constexpr int GHOST_HOPS = 5;

}  // namespace

struct sww_handle {
    sww_config cfg{};
    cudaStream_t user = nullptr;    // the caller's stream
    cudaStream_t stream = nullptr;  // the library's own stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::vector<DevLevel> lv;
    DevLevel* d_lvs = nullptr;
    std::vector<std::vector<double>> xyz;     // host node positions per level (flattened)
    std::vector<std::vector<int32_t>> edges;  // host edge (origin, end) pairs per level
    std::vector<void*> allocs;
    unsigned long long *red = nullptr, *cnt = nullptr;
    double *thr = nullptr, *dt = nullptr, *part = nullptr, *sums = nullptr;
    int32_t *all_list = nullptr, *all_count = nullptr, *d_counts = nullptr, *sig_any = nullptr;
    int32_t* h_counts = nullptr;    // pinned: per-level list sizes after each step
    double* h_dt = nullptr;         // pinned: time step of the last step
    int S = 64, jtop = 0, nsm = 152;
    unsigned grid_all = 1;
    std::vector<unsigned> grid_lv;
    double t = 0, last_dt = 0;
    int64_t steps = 0;
    bool has_state = false;
    // captured steps: (top level, adapt, dt) -> graph and its kernel count
    std::map<std::tuple<int, int, double>, std::pair<cudaGraphExec_t, int64_t>> graphs;
    // tracing: per-class event pairs
    uint32_t prof_mask = 0;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
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
        void* p = nullptr;
        ck(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc");
        allocs.push_back(p);
        return static_cast<T*>(p);
    }
    template <typename T>
    T* up(const std::vector<T>& v) {
        T* p = alloc<T>(v.size());
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
        if (h_dt) cudaFreeHost(h_dt);
        for (void* p : allocs) cudaFree(p);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

void upload_level(sww_handle* h, HostLevel& L, bool fine_side, bool coarse_side, int64_t coarse_E) {
    DevLevel D{};
    D.J = L.J, D.n = L.n, D.p = L.p, D.np = L.np, D.nelem = L.nelem, D.N = L.N, D.E = L.E, D.T = L.T, D.npatch = L.npatch;
    D.dx = nominal_spacing(L.J, h->cfg.radius);
    D.en = h->up_slots(L.en, 2);
    D.et = h->up_slots(L.et, 2);
    D.tn = h->up_slots(L.tn, 3);
    D.te = h->up_slots(L.te, 3);
    D.deg = h->up(L.deg);
    D.ring_e = h->up_slots(L.ring_e, 6);
    D.A_i = h->up(L.A_i), D.A_v = h->up(L.A_v), D.kite = h->up_slots(L.kite, 3);
    D.d_e = h->up(L.d_e), D.l_e = h->up(L.l_e), D.f_v = h->up(L.f_v), D.f_n = h->up(L.f_n);
    D.cor_i = h->up_slots(L.cor_i, COR);
    D.cor_w = h->up_slots(L.cor_w, COR);
    if (fine_side) {
        D.par = h->up_slots(L.par, 4);
        D.ptw = h->up_slots(L.ptw, 4);
        D.fe_kind = h->up(L.fe_kind);
        D.fe_ce = h->up(L.fe_ce);
        D.vst = h->up_slots(L.vst, VST);
        D.vw = h->up_slots(L.vw, VST);
    }
    if (coarse_side) {
        D.c2f = h->up(L.c2f), D.mid = h->up(L.mid), D.half = h->up_slots(L.half, 2);
        D.mk_i = h->up_slots(L.mk_i, 12);
        D.mk_w = h->up_slots(L.mk_w, 12);
        D.rf_fi = h->up_slots(L.rf_fi, RF_F);
        D.rf_fw = h->up_slots(L.rf_fw, RF_F);
        D.rf_ci = h->up_slots(L.rf_ci, RF_C);
        D.rf_cw = h->up_slots(L.rf_cw, RF_C);
    }
    const int64_t N = L.N, E = L.E, T = L.T;
    double** dN[] = {&D.dh, &D.dh0, &D.dha, &D.dht, &D.B, &D.c, &D.hdet};
    for (auto p : dN) *p = h->alloc<double>(N);
    double** dE[] = {&D.u, &D.u0, &D.ua, &D.ut, &D.F, &D.Q, &D.ui};
    for (auto p : dE) *p = h->alloc<double>(E);
    D.q = h->alloc<double>(T);
    D.ue = h->alloc<double>(coarse_E > 0 ? coarse_E : 1);
    uint8_t** bN[] = {&D.nflag, &D.sig, &D.tmask, &D.band0, &D.band1};
    for (auto p : bN) *p = h->alloc<uint8_t>(N);
    D.eflag = h->alloc<uint8_t>(E);
    D.pflag = h->alloc<uint8_t>(L.npatch);
    D.patches = h->alloc<int32_t>(L.npatch + 1);
    D.npatches = h->alloc<int32_t>(1);
    // f2c of this level: coarse node at the same place (-1 for odd nodes)
    {
        std::vector<int32_t> f2c(N, -1);
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
        D.f2c = h->up(f2c);
    }
    for (double* p : {D.dh, D.dh0, D.dha, D.dht, D.B, D.c, D.hdet}) ck(cudaMemset(p, 0, N * sizeof(double)), "memset");
    for (double* p : {D.u, D.u0, D.ua, D.ut, D.F, D.Q, D.ui}) ck(cudaMemset(p, 0, E * sizeof(double)), "memset");
    ck(cudaMemset(D.q, 0, T * sizeof(double)), "memset");
    for (uint8_t* p : {D.nflag, D.sig, D.tmask, D.band0, D.band1}) ck(cudaMemset(p, 0, N), "memset");
    ck(cudaMemset(D.eflag, 0, E), "memset");
    ck(cudaMemset(D.ue, 0, (coarse_E > 0 ? coarse_E : 1) * sizeof(double)), "memset");
    ck(cudaMemset(D.npatches, 0, sizeof(int32_t)), "memset");
    h->lv[L.J] = D;
}

void check_launch() { ck(cudaGetLastError(), "kernel launch"); }

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
    Trace(sww_handle* h_, int c) : h(h_), cls(c) {
        if (h->prof_mask & (1u << cls)) {
            a = h->take_event();
            ck(cudaEventRecord(a, h->stream), "cudaEventRecord");
        }
    }
    ~Trace() {
        if (!a) return;
        cudaEvent_t b = h->take_event();
        cudaEventRecord(b, h->stream);
        h->recs.push_back({cls, a, b});
    }
};

Work work_all(const sww_handle* h) { return Work{h->d_lvs, h->all_list, h->all_count, h->S, h->grid_all}; }
Work work_level(const sww_handle* h, int j) {
    return Work{nullptr, h->lv[j].patches, h->lv[j].npatches, h->S, h->grid_lv[j]};
}

// ------------------------------------------------------------------ sequences

void fill_ghosts(sww_handle* h) {
    for (int j = h->cfg.jmin + 1; j <= h->jtop; ++j) {
        Trace t(h, SWW_K_FILL);
        launch_fill(h->lv[j], h->lv[j - 1], work_level(h, j), h->stream);
    }
}

// one trend evaluation (Sec. 3.1): ghosts, q/K/B/F/qF^perp on every level, then the
// restriction of B, F and q F^perp from the top level down to Jmin
void trend(sww_handle* h) {
    const int j0 = h->cfg.jmin;
    cudaStream_t s = h->stream;
    Work W = work_all(h);
    fill_ghosts(h);
    { Trace t(h, SWW_K_PV); launch_pv_flux(W, h->cfg.H, s); }
    { Trace t(h, SWW_K_CORIOLIS); launch_node_coriolis(W, h->cfg.g, s); }
    for (int j = h->jtop - 1; j >= j0; --j) {
        Trace t(h, SWW_K_RESTRICT);
        launch_restrict(h->lv[j], h->lv[j + 1], work_level(h, j), s);
    }
}

void update(sww_handle* h, const RKStage& st) {
    Trace t(h, SWW_K_UPDATE);
    launch_update(work_all(h), st, h->dt, h->stream);
}

void compute_dt(sww_handle* h) {
    Trace t(h, SWW_K_DT);
    count_launch(1);
    k_reset_red<<<1, 32, 0, h->stream>>>(h->red);
    launch_dt(work_all(h), h->cfg.H, h->cfg.g, h->red, h->stream);
    launch_dt_final(h->red, h->cfg.cfl, h->dt, h->stream);
}

// list sizes of every level into pinned host memory (read after the next sync)
void read_counts(sww_handle* h) {
    count_launch(1);
    k_gather_counts<<<1, 32, 0, h->stream>>>(h->d_lvs, h->cfg.jmin, h->cfg.jmax, h->d_counts);
    ck(cudaMemcpyAsync(h->h_counts, h->d_counts, sizeof(int32_t) * (h->cfg.jmax + 1), cudaMemcpyDeviceToHost, h->stream),
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
Span span_of(const sww_handle* h, int ja, int jb, Count count) {
    Span sp{};
    sp.ja = ja, sp.jb = jb;
    int64_t t = 0;
    for (int j = ja; j <= jb; ++j) {
        sp.off[j - ja] = t;
        t += count(h->lv[j]);
    }
    sp.off[jb + 1 - ja] = t;
    return sp;
}

MaskArgs mask_args(const sww_handle* h, int j0, int j1) {
    MaskArgs a{};
    a.lvs = h->d_lvs, a.host = h->lv.data(), a.ja = j0, a.jb = j1, a.hops = GHOST_HOPS, a.thr = h->thr;
    auto N = [](const DevLevel& L) { return L.N; };
    auto E = [](const DevLevel& L) { return L.E; };
    auto P = [](const DevLevel& L) { return L.npatch; };
    int jf = std::min(j0 + 1, j1);
    a.nodes_f = span_of(h, jf, j1, N);
    a.edges_f = span_of(h, jf, j1, E);
    if (j1 == j0) a.nodes_f.off[1] = 0, a.edges_f.off[1] = 0;   // no level above Jmin
    a.nodes = span_of(h, j0, j1, N);
    a.edges = span_of(h, j0, j1, E);
    a.nodes_c = span_of(h, j0, std::max(j0, j1 - 1), N);
    a.patches = span_of(h, j0, j1, P);
    a.sig_any = h->sig_any;
    a.sig_any_len = h->cfg.jmax + 2;
    a.skip = j1 > h->jtop ? j1 : -1;
    return a;
}

// Mask construction and inverse transform.  Levels above top + 1 hold no live point
// and can gain none in one adaptation, so the byte-wide passes stop there.
void mask_and_inverse(sww_handle* h) {
    const int j0 = h->cfg.jmin, j1 = std::min(h->jtop + 1, h->cfg.jmax);
    cudaStream_t s = h->stream;
    {
        Trace tm(h, SWW_K_MASK);
        MaskArgs a = mask_args(h, j0, j1);
        launch_mask(a, s);
        launch_concat(h->d_lvs, j0, h->cfg.jmax, h->all_list, h->all_count, s);
    }
    // inverse transform of the retained coefficients, coarse to fine, ghosts per level
    for (int j = j0 + 1; j <= j1; ++j) {
        { Trace t(h, SWW_K_INVERSE); launch_inverse(h->lv[j], h->lv[j - 1], work_level(h, j), s); }
        { Trace t(h, SWW_K_FILL); launch_fill(h->lv[j], h->lv[j - 1], work_level(h, j), s); }
    }
}

void adapt(sww_handle* h, double eh, double eu) {
    cudaStream_t s = h->stream;
    { Trace t(h, SWW_K_COEFF); launch_details(work_all(h), h->cfg.jmin, s); }
    {
        Trace t(h, SWW_K_MASK);
        ck(cudaMemsetAsync(h->red, 0, 2 * sizeof(unsigned long long), s), "memset red");
        launch_maxabs(work_all(h), h->red, s);
        launch_thresholds(h->red, h->cfg.eps, eh, eu, h->thr, s);
    }
    mask_and_inverse(h);
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
// device-to-host copies of the time step and the list sizes.
void one_step(sww_handle* h, double dt, bool do_adapt) {
    const int j0 = h->cfg.jmin;
    if (dt > 0) {
        count_launch(1);
        k_set<<<1, 32, 0, h->stream>>>(h->dt, dt);
    } else {
        compute_dt(h);
    }
    { Trace t(h, SWW_K_UPDATE); launch_save_base(work_all(h), h->stream); }
    int ns;
    const RKStage* st = stages(h->cfg.rk, ns);
    for (int k = 0; k < ns; ++k) {
        trend(h);
        update(h, st[k]);
    }
    for (int j = h->jtop - 1; j >= j0; --j) {
        Trace t(h, SWW_K_PARTIAL);
        launch_partial(h->lv[j], h->lv[j + 1], work_level(h, j), h->stream);
    }
    fill_ghosts(h);
    if (do_adapt) adapt(h, -1.0, -1.0);
    read_counts(h);
    ck(cudaMemcpyAsync(h->h_dt, h->dt, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "dt");
}

// Run one step through a captured graph (eager when tracing).
void run_step(sww_handle* h, double dt, bool do_adapt) {
    if (h->prof_mask) {
        one_step(h, dt, do_adapt);
        return;
    }
    auto key = std::make_tuple(h->jtop, int(do_adapt), dt > 0 ? dt : -1.0);
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        if (h->graphs.size() >= 16) h->drop_graphs();
        int64_t before = kernel_launches();
        ck(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        try {
            one_step(h, dt, do_adapt);
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

}  // namespace

extern "C" {

int sww_create(const sww_config* cfg, void* stream, sww_handle** out) {
    if (!cfg || !out) return fail(SWW_E_ARG, "null argument");
    *out = nullptr;
    if (cfg->jmin < 1 || cfg->jmax < cfg->jmin || cfg->jmax > 11) return fail(SWW_E_ARG, "need 1 <= jmin <= jmax <= 11");
    if (!(cfg->radius > 0) || !(cfg->g > 0) || !(cfg->H > 0) || !(cfg->cfl > 0))
        return fail(SWW_E_ARG, "radius, g, H and cfl must be positive");
    if (!(cfg->eps >= 0)) return fail(SWW_E_ARG, "eps must be >= 0 (0: every point significant, no compression)");
    if (cfg->patch < 1 || (cfg->patch & (cfg->patch - 1)) || cfg->patch > 16)
        return fail(SWW_E_ARG, "patch must be a power of two <= 16");
    if (cfg->rk != SWW_RK4 && cfg->rk != SWW_SSP43) return fail(SWW_E_ARG, "rk must be SWW_RK4 or SWW_SSP43");
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
        Hierarchy H;
        build_hierarchy(H, cfg->jmin, cfg->jmax, cfg->patch, cfg->radius, cfg->omega);
        h->lv.assign(cfg->jmax + 1, DevLevel{});
        h->grid_lv.assign(cfg->jmax + 1, 1);
        h->xyz.assign(cfg->jmax + 1, {});
        h->edges.assign(cfg->jmax + 1, {});
        h->S = cfg->patch * cfg->patch;
        int64_t total = 0;
        const int64_t cap = int64_t(h->nsm) * 4;   // grid-stride launches: 4 blocks of 256 per SM
        for (int j = cfg->jmin; j <= cfg->jmax; ++j) {
            HostLevel& L = H.lv[j];
            upload_level(h, L, j > cfg->jmin, j < cfg->jmax, j > cfg->jmin ? H.lv[j - 1].E : 0);
            h->xyz[j].resize(3 * L.N);
            for (int64_t v = 0; v < L.N; ++v) h->xyz[j][3 * v] = L.xyz[v].x, h->xyz[j][3 * v + 1] = L.xyz[v].y, h->xyz[j][3 * v + 2] = L.xyz[v].z;
            h->edges[j].resize(2 * L.E);
            for (int64_t e = 0; e < L.E; ++e) h->edges[j][2 * e] = L.en[0][e], h->edges[j][2 * e + 1] = L.en[1][e];
            int64_t items = (L.npatch + 1) * h->S;
            h->grid_lv[j] = unsigned(std::min<int64_t>(blocks_for(items, 256), cap));
            total += L.npatch + 1;
        }
        h->grid_all = unsigned(std::min<int64_t>(blocks_for(total * h->S, 256), cap));
        h->d_lvs = h->alloc<DevLevel>(cfg->jmax + 1);
        ck(cudaMemcpy(h->d_lvs, h->lv.data(), sizeof(DevLevel) * (cfg->jmax + 1), cudaMemcpyHostToDevice), "levels");
        h->all_list = h->alloc<int32_t>(total);
        h->all_count = h->alloc<int32_t>(1);
        h->d_counts = h->alloc<int32_t>(cfg->jmax + 1);
        h->sig_any = h->alloc<int32_t>(cfg->jmax + 2);
        ck(cudaMemset(h->sig_any, 0, sizeof(int32_t) * (cfg->jmax + 2)), "memset");
        ck(cudaMallocHost(&h->h_counts, sizeof(int32_t) * (cfg->jmax + 1)), "cudaMallocHost");
        ck(cudaMallocHost(&h->h_dt, sizeof(double)), "cudaMallocHost");
        std::memset(h->h_counts, 0, sizeof(int32_t) * (cfg->jmax + 1));
        *h->h_dt = 0;
        h->red = h->alloc<unsigned long long>(4);
        h->cnt = h->alloc<unsigned long long>(4);
        h->thr = h->alloc<double>(2);
        h->dt = h->alloc<double>(1);
        h->sums = h->alloc<double>(2);
        h->part = h->alloc<double>(4 * size_t(sums_blocks(h->lv[cfg->jmin])));
        ck(cudaMemset(h->thr, 0, 2 * sizeof(double)), "memset");
        ck(cudaMemset(h->dt, 0, sizeof(double)), "memset");
        ck(cudaMemset(h->all_count, 0, sizeof(int32_t)), "memset");
        ck(cudaDeviceSynchronize(), "create");
        h->jtop = cfg->jmax;
        return SWW_OK;
    });
    if (rc != SWW_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return SWW_OK;
}

int sww_destroy(sww_handle* h) {
    if (!h) return SWW_OK;
    delete h;
    return SWW_OK;
}

int sww_level_sizes(const sww_handle* h, int level, int64_t* nn, int64_t* ne, int64_t* nt, int64_t* np) {
    int rc = check_level(h, level);
    if (rc) return rc;
    const DevLevel& L = h->lv[level];
    if (nn) *nn = L.N;
    if (ne) *ne = L.E;
    if (nt) *nt = L.T;
    if (np) *np = L.npatch;
    return SWW_OK;
}

int sww_get_grid(const sww_handle* h, int level, double* node_xyz, int32_t* edge_nodes) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (node_xyz) std::memcpy(node_xyz, h->xyz[level].data(), h->xyz[level].size() * sizeof(double));
    if (edge_nodes) std::memcpy(edge_nodes, h->edges[level].data(), h->edges[level].size() * sizeof(int32_t));
    return SWW_OK;
}

int sww_set_state(sww_handle* h, const double* dh, const double* u, int device_ptrs) {
    if (!h || !dh || !u) return fail(SWW_E_ARG, "null argument");
    return guarded([&]() -> int {
        const int j0 = h->cfg.jmin, j1 = h->cfg.jmax;
        cudaStream_t s = h->stream;
        {
            Join jn(h);
            DevLevel& F = h->lv[j1];
            cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
            ck(cudaMemcpyAsync(F.dh, dh, F.N * sizeof(double), kind, s), "set_state dh");
            ck(cudaMemcpyAsync(F.u, u, F.E * sizeof(double), kind, s), "set_state u");
            for (int j = j1; j > j0; --j) launch_restrict_full(h->lv[j - 1], h->lv[j], s);
            MaskArgs a = mask_args(h, j0, j1);
            launch_live_all(h->d_lvs, a.nodes, a.edges, s);
            if (j1 > j0) launch_covered_all(h->d_lvs, a.nodes_c, s);
            launch_patches_all(h->d_lvs, a.patches, s);
            launch_concat(h->d_lvs, j0, j1, h->all_list, h->all_count, s);
            read_counts(h);
            check_launch();
        }
        ck(cudaStreamSynchronize(s), "set_state");
        update_top(h);
        h->has_state = true;
        h->t = 0;
        h->steps = 0;
        return SWW_OK;
    });
}

int sww_adapt(sww_handle* h, double eps_h, double eps_u) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        {
            Join jn(h);
            adapt(h, eps_h, eps_u);
            read_counts(h);
            check_launch();
        }
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
        {
            Join jn(h);
            size_t oh = 0, oe = 0, oi = 0;
            for (int j = h->cfg.jmin + 1; j <= h->cfg.jmax; ++j) {
                DevLevel& F = h->lv[j];
                int64_t ce = h->lv[j - 1].E;
                ck(cudaMemcpyAsync(F.hdet, hdet + oh, F.N * sizeof(double), cudaMemcpyHostToDevice, h->stream), "hdet");
                ck(cudaMemcpyAsync(F.ue, udet_e + oe, ce * sizeof(double), cudaMemcpyHostToDevice, h->stream), "ue");
                ck(cudaMemcpyAsync(F.ui, udet_i + oi, F.E * sizeof(double), cudaMemcpyHostToDevice, h->stream), "ui");
                oh += F.N, oe += ce, oi += F.E;
            }
            double th[2] = {eps_h, eps_u};
            ck(cudaMemcpyAsync(h->thr, th, sizeof(th), cudaMemcpyHostToDevice, h->stream), "thr");
            ck(cudaStreamSynchronize(h->stream), "thr");   // th lives on this host stack frame
            mask_and_inverse(h);
            read_counts(h);
            check_launch();
        }
        ck(cudaStreamSynchronize(h->stream), "mask");
        update_top(h);
        return SWW_OK;
    });
}

int sww_rhs(sww_handle* h) {
    if (!h) return fail(SWW_E_ARG, "null handle");
    if (!h->has_state) return fail(SWW_E_STATE, "sww_set_state first");
    return guarded([&]() -> int {
        {
            Join jn(h);
            trend(h);
            RKStage none{0, 0, 0, 0, 0, 0, 0};
            update(h, none);
            check_launch();
        }
        ck(cudaStreamSynchronize(h->stream), "rhs");
        return SWW_OK;
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

int sww_get_level(const sww_handle* h, int level, int what, void* out) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!out) return fail(SWW_E_ARG, "null output");
    const DevLevel& L = h->lv[level];
    const void* src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case SWW_DH: src = L.dh, bytes = L.N * sizeof(double); break;
        case SWW_U: src = L.u, bytes = L.E * sizeof(double); break;
        case SWW_DH_T: src = L.dht, bytes = L.N * sizeof(double); break;
        case SWW_U_T: src = L.ut, bytes = L.E * sizeof(double); break;
        case SWW_NODE_FLAGS: src = L.nflag, bytes = L.N; break;
        case SWW_EDGE_FLAGS: src = L.eflag, bytes = L.E; break;
        case SWW_HDET: src = L.hdet, bytes = L.N * sizeof(double); break;
        case SWW_UDET_E:
            if (level == h->cfg.jmin) return fail(SWW_E_ARG, "no coefficients on Jmin");
            src = L.ue, bytes = h->lv[level - 1].E * sizeof(double);
            break;
        case SWW_UDET_I: src = L.ui, bytes = L.E * sizeof(double); break;
        case SWW_SIG: src = L.sig, bytes = L.N; break;
        default: return fail(SWW_E_ARG, "unknown quantity");
    }
    sww_handle* hh = const_cast<sww_handle*>(h);
    return guarded([&]() -> int {
        {
            Join jn(hh);
            ck(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, hh->stream), "get_level");
        }
        ck(cudaStreamSynchronize(hh->stream), "get_level");
        return SWW_OK;
    });
}

int sww_set_level(sww_handle* h, int level, const double* dh, const double* u) {
    int rc = check_level(h, level);
    if (rc) return rc;
    return guarded([&]() -> int {
        const DevLevel& L = h->lv[level];
        {
            Join jn(h);
            if (dh) ck(cudaMemcpyAsync(L.dh, dh, L.N * sizeof(double), cudaMemcpyHostToDevice, h->stream), "set dh");
            if (u) ck(cudaMemcpyAsync(L.u, u, L.E * sizeof(double), cudaMemcpyHostToDevice, h->stream), "set u");
        }
        ck(cudaStreamSynchronize(h->stream), "set_level");
        return SWW_OK;
    });
}

int sww_get_patches(const sww_handle* h, int level, int32_t* out, int32_t* count) {
    int rc = check_level(h, level);
    if (rc) return rc;
    if (!count) return fail(SWW_E_ARG, "null count");
    sww_handle* hh = const_cast<sww_handle*>(h);
    return guarded([&]() -> int {
        const DevLevel& L = h->lv[level];
        int32_t n = 0;
        std::vector<int32_t> tmp(L.npatch + 1);
        {
            Join jn(hh);
            ck(cudaMemcpyAsync(&n, L.npatches, sizeof(int32_t), cudaMemcpyDeviceToHost, hh->stream), "npatches");
            ck(cudaMemcpyAsync(tmp.data(), L.patches, tmp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, hh->stream),
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
        for (int j = h->cfg.jmin; j <= h->cfg.jmax && j < 16; ++j) {
            unsigned long long c[3] = {0, 0, 0};
            {
                Join jn(h);
                ck(cudaMemsetAsync(h->cnt, 0, 3 * sizeof(unsigned long long), h->stream), "memset cnt");
                launch_count(h->lv[j], h->cnt, h->stream);
                ck(cudaMemcpyAsync(c, h->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream), "cnt");
            }
            ck(cudaStreamSynchronize(h->stream), "stats");
            st->live_nodes[j] = int64_t(c[0]);
            st->ghost_nodes[j] = int64_t(c[1]);
            st->live_edges[j] = int64_t(c[2]);
            int32_t np = 0;
            int rc = sww_get_patches(h, j, nullptr, &np);
            if (rc) return rc;
            st->active_patches[j] = np;
        }
        double s[2], th[2];
        {
            Join jn(h);
            const DevLevel& L0 = h->lv[h->cfg.jmin];
            launch_sums(L0, h->cfg.H, h->cfg.g, h->part, h->sums, h->stream);
            ck(cudaMemcpyAsync(s, h->sums, sizeof(s), cudaMemcpyDeviceToHost, h->stream), "sums");
            ck(cudaMemcpyAsync(th, h->thr, sizeof(th), cudaMemcpyDeviceToHost, h->stream), "thr");
            check_launch();
        }
        ck(cudaStreamSynchronize(h->stream), "stats");
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
            launches[r.cls] += 1;
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
    v->jmin_level = &h->lv[h->cfg.jmin];
    v->stream = h->user;
    v->radius = h->cfg.radius;
    v->g = h->cfg.g;
    v->H = h->cfg.H;
    return true;
}

int set_error(int code, const char* msg) { return fail(code, msg); }

}  // namespace sww
