// Allocation-free mass and energy sums: a variant of the compensated reduction
// behind sww_stats_get whose per-block partial sums live in a fixed device array
// of this library instead of memory allocated at handle creation.
//
// It serves callers that must not allocate device memory when they ask for the
// diagnostics: code running inside a framework whose caching allocator owns the
// whole device heap, real-time loops where an allocation (and the implicit
// synchronisation of cudaMalloc/cudaFree) is not allowed, and hosts that hand
// the library only the buffers it reads and writes.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "sww.h"
#include "sww_core.cuh"
#include "sww_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4096;   // partial sums for up to 4096 * 256 = 1,048,576 nodes

// Four doubles per block (mass sum and its compensation, energy sum and its
// compensation); 128 KiB, resident on every GPU that loads the library.
__device__ __align__(256) double g_partials[4 * kMaxBlocks];

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

__global__ void k_sums_static(sww::DevLevel L, const double* __restrict__ dh, const double* __restrict__ u, double H,
                              double g, double* part) {
    __shared__ double sh[2][kThreads];
    int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double m = 0.0, en = 0.0;
    if (v < L.N) {
        double h = H + dh[v], A = L.A_i[v], ke = 0.0;
        for (int k = 0; k < L.deg[v]; ++k) {
            int64_t e = L.ring_e[k * L.N + v] >> 1;
            ke += 0.25 * L.l_e[e] * L.d_e[e] * u[e] * u[e];
        }
        m = A * h;
        en = g * h * (0.5 * g * h * A + ke);
    }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = en;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
        for (int k = 0; k < blockDim.x; ++k) neumaier_add(s0, c0, sh[0][k]), neumaier_add(s1, c1, sh[1][k]);
        part[4 * blockIdx.x + 0] = s0;
        part[4 * blockIdx.x + 1] = c0;
        part[4 * blockIdx.x + 2] = s1;
        part[4 * blockIdx.x + 3] = c1;
    }
}

// Reduces the partials; out[0] = mass, out[1] = energy of Sec. 7.2 (with the
// resting state c^4 A_S / 2 removed, as in sww_stats_get).
__global__ void k_sums_static_final(const double* part, int nblk, double g, double area, double* out) {
    if (threadIdx.x || blockIdx.x) return;
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
    for (int b = 0; b < nblk; ++b) {
        neumaier_add(s0, c0, part[4 * b]);
        neumaier_add(s0, c0, part[4 * b + 1]);
        neumaier_add(s1, c1, part[4 * b + 2]);
        neumaier_add(s1, c1, part[4 * b + 3]);
    }
    // the same roundings as the host's resting-state subtraction in sww_stats_get
    // (no fused multiply-adds), so that both report the same bits
    const double mass = s0 + c0;
    const double c2 = __ddiv_rn(__dmul_rn(g, mass), area);
    out[0] = mass;
    out[1] = __dsub_rn(s1 + c1, __dmul_rn(__dmul_rn(__dmul_rn(0.5, c2), c2), area));
}

// Device address of g_partials per device, looked up once per device (a
// cudaDeviceReset of that device ends the library's use of it, as it ends every
// handle there).
std::mutex g_mu;
double* g_addr[64] = {nullptr};

int partials_address(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return sww::set_error(SWW_E_CUDA, "sww_mass_energy_static: no current CUDA device");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess || !p) return sww::set_error(SWW_E_CUDA, "sww_mass_energy_static: cudaGetSymbolAddress failed");
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return SWW_OK;
}

}  // namespace

extern "C" int sww_mass_energy_static(sww_handle* h, const double* dh, const double* u, double* out) {
    sww::HandleView v{};
    if (!sww::handle_view(h, &v)) return sww::set_error(SWW_E_ARG, "sww_mass_energy_static: null handle");
    if (!dh || !u || !out) return sww::set_error(SWW_E_ARG, "sww_mass_energy_static: null pointer");
    const sww::DevLevel& L = *v.jmin_level;
    int64_t nblk = (L.N + kThreads - 1) / kThreads;
    if (nblk > kMaxBlocks)
        return sww::set_error(SWW_E_ARG, "sww_mass_energy_static: Jmin level has more than 1,048,576 nodes "
                                         "(the static scratch holds 4096 blocks of 256)");
    // the three arrays must be device (or managed) memory: a host address would
    // reach the kernels (cudaPointerGetAttributes allocates nothing)
    for (const void* p : {static_cast<const void*>(dh), static_cast<const void*>(u), static_cast<const void*>(out)}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return sww::set_error(SWW_E_ARG, "sww_mass_energy_static: a pointer is not known to CUDA");
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
            return sww::set_error(SWW_E_ARG, "sww_mass_energy_static: dh, u and out must be device memory");
    }
    // an error left pending by earlier work is reported as such, not as this call's
    if (cudaError_t pending = cudaPeekAtLastError(); pending != cudaSuccess)
        return sww::set_error(SWW_E_CUDA, "sww_mass_energy_static: an earlier CUDA error is pending");
    double* part = nullptr;
    int rc = partials_address(&part);
    if (rc != SWW_OK) return rc;
    k_sums_static<<<unsigned(nblk), kThreads, 0, v.stream>>>(L, dh, u, v.H, v.g, part);
    double area = 4.0 * M_PI * v.radius * v.radius;
    k_sums_static_final<<<1, 32, 0, v.stream>>>(part, int(nblk), v.g, area, out);
    if (cudaGetLastError() != cudaSuccess) return sww::set_error(SWW_E_CUDA, "sww_mass_energy_static: launch failed");
    return SWW_OK;
}
