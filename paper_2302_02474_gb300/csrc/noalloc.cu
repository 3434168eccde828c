// Allocation-free density spread (tild_spread_density_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs while a framework's
// caching allocator owns all device memory, plug-ins held to a fixed memory
// budget, and real-time loops where an allocation (which may synchronise the
// device) is not acceptable. This entry point needs no context and allocates
// nothing: its 64-bit fixed-point scratch grid is a file-scope __device__
// array that every GPU loading this library holds until the process exits.
// Under CUDA's lazy module loading (the default) that array, with this file's
// device code, is placed on a device when the first call there looks up its
// address; that first call should therefore run during set-up.
#include <cmath>
#include <cstring>
#include <string>

#include "bead_kernels.cuh"
#include "engine_api.h"

namespace tild {
namespace {

constexpr int kNoAllocMaxN = 64;
constexpr size_t kNoAllocMaxPoints = (size_t)kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN;

// Two species of int64 fixed-point sums (2^22 per unit weight), 4 MiB.
static __device__ __align__(256) unsigned long long g_noalloc_rho[2 * kNoAllocMaxPoints];

template <int P>
__global__ void noalloc_spread(int64_t n_beads, const float* __restrict__ xyz, const unsigned char* __restrict__ species,
                               float L, float inv_L, float inv_dx, int n, unsigned long long* __restrict__ rho) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const float x = wrap_coord(xyz[3 * (size_t)i + 0], L, inv_L);
    const float y = wrap_coord(xyz[3 * (size_t)i + 1], L, inv_L);
    const float z = wrap_coord(xyz[3 * (size_t)i + 2], L, inv_L);
    Stencil<P, float> st;
    st.set(x, y, z, inv_dx);
    const int K = species[i] ? 1 : 0;
    const int nm = n - 1;
    const size_t M = (size_t)n * n * n;
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const float wyz = st.wy[b] * st.wz[c];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const size_t g = ((size_t)((st.jz + c) & nm) * n + ((st.jy + b) & nm)) * n + ((st.jx + a) & nm);
                atomicAdd(rho + K * M + g, FixedPoint<float>::to_grid(st.wx[a] * wyz));
            }
        }
}

__global__ void noalloc_convert(size_t count, const unsigned long long* __restrict__ rho, double scale,
                                float* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (float)((double)(long long)rho[i] * scale);
}

tild_status fail(tild_status st, const std::string& msg) {
    set_global_error(msg);
    return st;
}

}  // namespace
}  // namespace tild

using namespace tild;

extern "C" {

tild_status tild_spread_density_noalloc(const float* xyz, const unsigned char* species, int64_t n_beads, double L,
                                        int n, int pmeorder, float* rho_out, void* stream) {
    if (!xyz || !species || !rho_out) return fail(TILD_EINVAL, "spread_density_noalloc: NULL pointer");
    if (n_beads < 0 || n_beads >= ((int64_t)1 << 31)) return fail(TILD_EINVAL, "spread_density_noalloc: bad n_beads");
    if (!(L > 0) || !std::isfinite(L)) return fail(TILD_EINVAL, "spread_density_noalloc: L must be > 0");
    if (n < 8 || n > kNoAllocMaxN || (n & (n - 1)) != 0)
        return fail(TILD_EINVAL, "spread_density_noalloc: n must be a power of two in [8, 64] (static scratch of 64^3 points)");
    if (pmeorder < 1 || pmeorder > 4) return fail(TILD_EINVAL, "spread_density_noalloc: pmeorder must be in 1..4");
    // the device address of the scratch array on the current device: the
    // host-side name of a __device__ array is not a device address. Looked up
    // on every call (a host-side table lookup once the module is loaded), so
    // no cached address outlives a device reset.
    void* scratch = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_rho);
    if (e != cudaSuccess) return fail(TILD_EDEVICE, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* rho = (unsigned long long*)scratch;
    const size_t M = (size_t)n * n * n;
    // the scratch keeps the previous call's sums: clear what this call uses
    e = cudaMemsetAsync(rho, 0, 2 * M * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return fail(TILD_EDEVICE, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const float Lf = (float)L, inv_L = (float)(1.0 / L), inv_dx = (float)((double)n / L);
    const int64_t nb = n_beads;
    const unsigned grid = (unsigned)((nb + 255) / 256);  // nb < 2^31: at most 2^23 blocks
    if (nb > 0) {
        switch (pmeorder + 1) {
            case 2: noalloc_spread<2><<<grid, 256, 0, s>>>(nb, xyz, species, Lf, inv_L, inv_dx, n, rho); break;
            case 3: noalloc_spread<3><<<grid, 256, 0, s>>>(nb, xyz, species, Lf, inv_L, inv_dx, n, rho); break;
            case 4: noalloc_spread<4><<<grid, 256, 0, s>>>(nb, xyz, species, Lf, inv_L, inv_dx, n, rho); break;
            default: noalloc_spread<5><<<grid, 256, 0, s>>>(nb, xyz, species, Lf, inv_L, inv_dx, n, rho); break;
        }
    }
    const double dV = L * L * L / (double)M;
    noalloc_convert<<<(unsigned)((2 * M + 255) / 256), 256, 0, s>>>(2 * M, rho, 1.0 / FixedPoint<float>::scale / dV,
                                                                       rho_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TILD_EDEVICE, std::string("launch: ") + cudaGetErrorString(e));
    return TILD_OK;
}

}  // extern "C"
