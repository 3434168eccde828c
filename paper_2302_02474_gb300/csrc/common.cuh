// Shared device helpers of the TILD step: complex arithmetic, the
// Philox4x32-10 generator, Deserno-Holm assignment weights and the implicit
// chain topology.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tild {

// ---------------------------------------------------------------- types

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx_of<T>::type;

template <class V> __device__ __forceinline__ V c_add(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <class V> __device__ __forceinline__ V c_sub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
template <class V> __device__ __forceinline__ V c_mul(V a, V b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class V> __device__ __forceinline__ V c_conj(V a) { return {a.x, -a.y}; }
template <class V, typename T> __device__ __forceinline__ V c_scale(V a, T s) { return {a.x * s, a.y * s}; }
// multiply by -i (forward-transform quarter turn) or +i
template <class V> __device__ __forceinline__ V c_mul_negi(V a) { return {a.y, -a.x}; }
template <class V> __device__ __forceinline__ V c_mul_posi(V a) { return {-a.y, a.x}; }

// Deterministic density accumulation: every bead weight w in [0, 1] is
// rounded once to an integer, round(w * 2^F), and all sums are integer sums,
// which are associative: the grids are bit-identical for any order of
// contributions, blocks or re-binning.
//   FP32 path: F = 22. A tile's shared-memory patch holds 32-bit sums; a tile
//     of at most 1023 beads cannot overflow (1023 * 2^22 < 2^32), larger tiles
//     spread straight into the 64-bit grid. Quantisation <= 2^-23 per
//     contribution, comparable to the FP32 rounding of the weights.
//   FP64 path: F = 44, 64-bit patch sums; quantisation <= 2^-45.
// The global grid is 64-bit in both cases.
template <typename T> struct FixedPoint;
// FP32: one 32-bit shared word per patch point and species.
template <> struct FixedPoint<float> {
    using patch_t = unsigned int;
    static constexpr double scale = 4194304.0;  // 2^22
    static constexpr int max_tile_beads = 1023;
    static __device__ __forceinline__ unsigned int to_patch(float w) { return __float2uint_rn(w * 4194304.0f); }
    static __device__ __forceinline__ unsigned long long to_grid(float w) { return to_patch(w); }
};
// FP64: one 64-bit shared word per point and species.
template <> struct FixedPoint<double> {
    using patch_t = unsigned long long;
    static constexpr double scale = 17592186044416.0;  // 2^44
    static constexpr int max_tile_beads = 0x7fffffff;
    static __device__ __forceinline__ unsigned long long to_patch(double w) {
        return (unsigned long long)__double2ll_rn(w * scale);
    }
    static __device__ __forceinline__ unsigned long long to_grid(double w) { return to_patch(w); }
};
// Fixed point -> density (scale = 2^-F / dV); no FP64 in the FP32 path.
__device__ __forceinline__ float from_fixed(long long v, float scale) { return __ll2float_rn(v) * scale; }
__device__ __forceinline__ double from_fixed(long long v, double scale) { return (double)v * scale; }

// Tiles of the bead kernel: beads are binned by 8x8x8 grid cells.
constexpr int kTile = 8;
constexpr int kTileCells = kTile * kTile * kTile;

// ---------------------------------------------------------------- Philox

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = {hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals for (bead id, step) from one Philox block:
// u_j = (x_j + 1/2) 2^-32, Box-Muller on (u0, u1) gives two normals and
// sqrt(-2 ln u2) cos(2 pi u3) the third.
template <typename T> struct normal3 {
    T a, b, c;
};

__device__ __forceinline__ normal3<float> gaussian3(uint32_t id, uint64_t step, uint64_t seed, float) {
    const u32x4 r = philox4x32_10({id, (uint32_t)step, (uint32_t)(step >> 32), 0u}, (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const float s = 2.3283064365386963e-10f;  // 2^-32
    const float u0 = fmaf((float)r.x, s, 0.5f * s);
    const float u1 = fmaf((float)r.y, s, 0.5f * s);
    const float u2 = fmaf((float)r.z, s, 0.5f * s);
    const float u3 = fmaf((float)r.w, s, 0.5f * s);
    // CUDA's fast log and sine/cosine intrinsics (absolute errors near
    // 1e-6); the angle 2 pi u - pi lies in their accurate range [-pi, pi],
    // and sin, cos of 2 pi u are minus those of 2 pi u - pi
    const float m1 = sqrtf(fmaxf(-2.0f * __logf(u0), 0.0f));
    const float m2 = sqrtf(fmaxf(-2.0f * __logf(u2), 0.0f));
    float s1, c1, s3, c3;
    __sincosf(fmaf(6.28318530717958648f, u1, -3.14159265358979324f), &s1, &c1);
    __sincosf(fmaf(6.28318530717958648f, u3, -3.14159265358979324f), &s3, &c3);
    return {-m1 * c1, -m1 * s1, -m2 * c3};
}

__device__ __forceinline__ normal3<double> gaussian3(uint32_t id, uint64_t step, uint64_t seed, double) {
    const u32x4 r = philox4x32_10({id, (uint32_t)step, (uint32_t)(step >> 32), 0u}, (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const double s = 2.3283064365386962890625e-10;  // 2^-32
    const double u0 = ((double)r.x + 0.5) * s;
    const double u1 = ((double)r.y + 0.5) * s;
    const double u2 = ((double)r.z + 0.5) * s;
    const double u3 = ((double)r.w + 0.5) * s;
    const double m1 = sqrt(-2.0 * log(u0));
    const double m2 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    return {m1 * c1, m1 * s1, m2 * c3};
}

// Periodic grid index for j in [-n, 2n) (any n; stencils and patches never
// reach further than one period).
__host__ __device__ __forceinline__ int pwrap(int j, int n) { return j < 0 ? j + n : (j >= n ? j - n : j); }

// ------------------------------------------------- assignment weights

// Charge-assignment weights of order P (P points per dimension), the
// closed-form polynomials of Deserno & Holm (J. Chem. Phys. 109, 7678,
// 1998, appendix) cited by the paper for its spline weights. s is the
// position in grid units; j0 receives the first grid point (not wrapped).
// Even P: t = s - floor(s) in [0, 1), points floor(s)-P/2+1 .. floor(s)+P/2.
// Odd P:  t = s - floor(s + 1/2) in [-1/2, 1/2), points centred on the
//         nearest grid point.
template <int P, typename T> __device__ __forceinline__ void dh_weights(T s, int& j0, T (&w)[P]) {
    if constexpr (P == 2) {
        const T f = floor(s);
        const T t = s - f;
        j0 = (int)f;
        w[0] = T(1) - t;
        w[1] = t;
    } else if constexpr (P == 3) {
        const T f = floor(s + T(0.5));
        const T t = s - f;
        j0 = (int)f - 1;
        w[0] = T(0.5) * (T(0.5) - t) * (T(0.5) - t);
        w[1] = T(0.75) - t * t;
        w[2] = T(0.5) * (T(0.5) + t) * (T(0.5) + t);
    } else if constexpr (P == 4) {
        const T f = floor(s);
        const T t = s - f;
        const T t2 = t * t, t3 = t2 * t, u = T(1) - t;
        j0 = (int)f - 1;
        w[0] = u * u * u * T(1.0 / 6.0);
        w[1] = (T(4) - T(6) * t2 + T(3) * t3) * T(1.0 / 6.0);
        w[2] = (T(1) + T(3) * t + T(3) * t2 - T(3) * t3) * T(1.0 / 6.0);
        w[3] = t3 * T(1.0 / 6.0);
    } else {
        static_assert(P == 5, "orders 1..4 (P = 2..5)");
        const T f = floor(s + T(0.5));
        const T t = s - f;
        const T t2 = t * t, t3 = t2 * t, t4 = t2 * t2;
        const T a = T(1) - T(2) * t, b = T(1) + T(2) * t;
        j0 = (int)f - 2;
        w[0] = a * a * a * a * T(1.0 / 384.0);
        w[1] = (T(19) - T(44) * t + T(24) * t2 + T(16) * t3 - T(16) * t4) * T(1.0 / 96.0);
        w[2] = (T(115) - T(120) * t2 + T(48) * t4) * T(1.0 / 192.0);
        w[3] = (T(19) + T(44) * t + T(24) * t2 - T(16) * t3 - T(16) * t4) * T(1.0 / 96.0);
        w[4] = b * b * b * b * T(1.0 / 384.0);
    }
}

// d/ds of the weights of dh_weights (same points).
template <int P, typename T> __device__ __forceinline__ void dh_weight_derivs(T s, T (&dw)[P]) {
    if constexpr (P == 2) {
        dw[0] = T(-1);
        dw[1] = T(1);
    } else if constexpr (P == 3) {
        const T t = s - floor(s + T(0.5));
        dw[0] = t - T(0.5);
        dw[1] = T(-2) * t;
        dw[2] = T(0.5) + t;
    } else if constexpr (P == 4) {
        const T t = s - floor(s);
        const T u = T(1) - t;
        dw[0] = T(-0.5) * u * u;
        dw[1] = T(-2) * t + T(1.5) * t * t;
        dw[2] = T(0.5) + t - T(1.5) * t * t;
        dw[3] = T(0.5) * t * t;
    } else {
        const T t = s - floor(s + T(0.5));
        const T t2 = t * t, t3 = t2 * t;
        const T a = T(1) - T(2) * t, b = T(1) + T(2) * t;
        dw[0] = -a * a * a * T(1.0 / 48.0);
        dw[1] = (T(-44) + T(48) * t + T(48) * t2 - T(64) * t3) * T(1.0 / 96.0);
        dw[2] = T(-1.25) * t + t3;
        dw[3] = (T(44) + T(48) * t - T(48) * t2 - T(64) * t3) * T(1.0 / 96.0);
        dw[4] = b * b * b * T(1.0 / 48.0);
    }
}

// Stencil extent relative to the cell floor(s): points floor(s)+lo ..
// floor(s)+hi can receive weight.
template <int P> struct stencil_extent {
    static constexpr int lo = (P % 2 == 0) ? -(P / 2 - 1) : -((P - 1) / 2);
    static constexpr int hi = (P % 2 == 0) ? (P / 2) : ((P - 1) / 2 + 1);
};

// ------------------------------------------------------ chain topology

constexpr int kMaxTypes = 8;

// Linear chains numbered type by type (see tild.h). Passed by value to the
// kernels that need species or bonded neighbours of a bead id.
struct Topology {
    int n_types;
    int start[kMaxTypes + 1];  // first bead id of each type (n_beads < 2^31)
    int N[kMaxTypes];
    int n_a[kMaxTypes];
};

struct BeadInfo {
    int species;
    int prev;  // id of the bonded predecessor or -1
    int next;  // id of the bonded successor or -1
};

__host__ __device__ __forceinline__ BeadInfo bead_info(const Topology& t, int id) {
    int k = 0;
    while (k + 1 < t.n_types && id >= t.start[k + 1]) ++k;
    const int s = (id - t.start[k]) % t.N[k];
    BeadInfo b;
    b.species = s < t.n_a[k] ? 0 : 1;
    b.prev = s > 0 ? id - 1 : -1;
    b.next = s < t.N[k] - 1 ? id + 1 : -1;
    return b;
}

// Error flags raised by kernels (read by the host on demand).
constexpr unsigned kErrNonFinite = 1u;
constexpr unsigned kErrBounds = 2u;  // a bounds check of the debug build failed

// Debug build (compiled with -DTILD_DEBUG=1, `_build.build(debug=True)`):
// the bead kernels check slot and grid indices before they use them; a
// failed check records kErrBounds in the context's error word and the access
// is skipped (no trap), and the next synchronising call returns
// TILD_EDEVICE. In the normal build every check is the constant true.
#ifndef TILD_DEBUG
#define TILD_DEBUG 0
#endif
__device__ __forceinline__ bool debug_check(bool ok, unsigned int* err) {
#if TILD_DEBUG
    if (!ok) atomicOr(err, kErrBounds);
    return ok;
#else
    (void)err;
    return true;
#endif
}

}  // namespace tild
