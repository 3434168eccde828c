// Grid stages of the TILD step (Eq. PMM evaluated by FFT):
//   forward:  int64 fixed-point densities -> Z = DFT_xy(rho_A + i rho_B)
//   z pass:   DFT_z, spectral multiply with the smeared chi/kappa kernel and
//             i k (one CTA per pencil tile), inverse DFT_z -> H_d
//   inverse:  H_d -> IDFT_xy -> (d w_A/dr_d, d w_B/dr_d) on the grid
//
// Two real species are carried as one complex field Z = rho_A + i rho_B.
// Their spectra are separated in the z pass with Hermitian symmetry:
//   rho~_A(k) = (Z(k) + conj Z(-k)) / 2,  rho~_B(k) = (Z(k) - conj Z(-k)) / (2i),
// and the three gradient spectra are packed back as
//   H_d(k) = i k~_d (w~_A(k) + i w~_B(k)),
// whose inverse transform is real part d w_A/dr_d, imaginary part
// d w_B/dr_d (both gradient fields are real).
//
// Memory layouts (n^3 points, index g = (z n + y) n + x):
//   rho_fx  int64 [2][M]             fixed-point densities (2^44 per bead weight)
//   Zxy     complex [z][ky][kx]       after the forward x and y transforms
//   H       complex [3][z][ky][kx]    after the z pass (z back in real space)
//   grad    complex [3][z][y][x]      (d w_A, d w_B) per point and direction
#pragma once

#include "fft.cuh"

namespace tild {

template <typename T> struct SpectralParams {
    T two_pi_over_L;   // 2 pi / L
    T eAA, eAB, eBB;   // eps matrix / M (the 1/M of the inverse DFT folded in)
    const T* kernel1d; // exp(-a^2 k_m^2) per 1-D frequency index m (FP64 on the host)
};

// Pitch (in complex elements) of a row of n elements in shared memory: odd
// so that threads on consecutive rows hit distinct banks.
__host__ __device__ constexpr int row_pitch(int n) { return n + 1; }

template <class V> __device__ __forceinline__ void load_twiddles(V* s_tw, const V* g_tw, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) s_tw[i] = g_tw[i];
}

// Units of stage B per thread for `lines` lines of length N with THREADS threads.
template <int N, int THREADS> __host__ __device__ constexpr int upt_for(int lines) {
    return (lines * fft_split<N>::N1 + THREADS - 1) / THREADS;
}

// Load ROWS rows of N fixed-point densities of both species (16-byte
// vectors), optionally zero them, and store rho_A + i rho_B to shared rows of
// pitch PITCH. Loads are issued in batches before any store so that the
// zeroing stores do not serialise them.
template <int N, int PITCH, int ROWS, int NTHR, class V, typename T>
__device__ __forceinline__ void load_fixed_rows(unsigned long long* __restrict__ ga, unsigned long long* __restrict__ gb,
                                                V* rows, T scale, int zero_after) {
    constexpr int PAIRS = ROWS * N / 2;
    constexpr int ITER = (PAIRS + NTHR - 1) / NTHR;
    constexpr int BATCH = ITER < 4 ? ITER : 4;
    longlong2* pa = reinterpret_cast<longlong2*>(ga);
    longlong2* pb = reinterpret_cast<longlong2*>(gb);
#pragma unroll 1
    for (int k0 = 0; k0 < ITER; k0 += BATCH) {
        longlong2 a[BATCH], b[BATCH];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (i < PAIRS) {
                a[k] = __ldcs(pa + i);
                b[k] = __ldcs(pb + i);
            }
        }
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (i < PAIRS) {
                if (zero_after) {
                    pa[i] = make_longlong2(0, 0);
                    pb[i] = make_longlong2(0, 0);
                }
                const int r = (2 * i) / N, x = (2 * i) % N;
                rows[r * PITCH + x] = V{from_fixed(a[k].x, scale), from_fixed(b[k].x, scale)};
                rows[r * PITCH + x + 1] = V{from_fixed(a[k].y, scale), from_fixed(b[k].y, scale)};
            }
        }
    }
}

// --------------------------------------------------------------------------
// Forward xy pass on whole z-planes (plane fits in shared memory).
// grid = n (one CTA per z-plane), block = 512.
// --------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(512) xy_forward_plane(unsigned long long* __restrict__ rho_fx,
                                                         cplx_t<T>* __restrict__ Zxy,
                                                         const cplx_t<T>* __restrict__ tw_g, T scale,
                                                         int zero_after, unsigned long long* step_ctr) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* plane = tw + N;
    load_twiddles(tw, tw_g, N);
    // a step's first kernel advances the noise counter to n+1
    if (step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *step_ctr += 1ull;

    const int z = blockIdx.x;
    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)z * N * N;
    // load + convert: pairs of x so that global accesses are 16-byte vectors
    load_fixed_rows<N, PITCH, N, 512>(rho_fx + base, rho_fx + M + base, plane, scale, zero_after);
    __syncthreads();
    smem_fft_lines<N, -1, N, 512>(plane, StridedLines<PITCH>{}, 1, tw);  // along x
    smem_fft_lines<N, -1, N, 512>(plane, StridedLines<1>{}, PITCH, tw);  // along y
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const int y = i / N, x = i % N;
        Zxy[base + i] = plane[y * PITCH + x];
    }
}

// --------------------------------------------------------------------------
// Inverse xy pass on whole z-planes: grid = (n, 3), block = 512.
// --------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(512) xy_inverse_plane(const cplx_t<T>* __restrict__ H,
                                                         cplx_t<T>* __restrict__ grad,
                                                         const cplx_t<T>* __restrict__ tw_g) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* plane = tw + N;
    load_twiddles(tw, tw_g, N);

    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)blockIdx.y * M + (size_t)blockIdx.x * N * N;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) plane[(i / N) * PITCH + i % N] = H[base + i];
    __syncthreads();
    smem_fft_lines<N, +1, N, 512>(plane, StridedLines<1>{}, PITCH, tw);  // along y
    smem_fft_lines<N, +1, N, 512>(plane, StridedLines<PITCH>{}, 1, tw);  // along x
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) grad[base + i] = plane[(i / N) * PITCH + i % N];
}

// --------------------------------------------------------------------------
// Split passes for planes that do not fit in shared memory.
// Row pass along x: CTA handles R consecutive rows (row r = z n + y).
// --------------------------------------------------------------------------
template <typename T, int N, int R>
__global__ void __launch_bounds__(256) x_forward_rows(unsigned long long* __restrict__ rho_fx,
                                                       cplx_t<T>* __restrict__ Zxy,
                                                       const cplx_t<T>* __restrict__ tw_g, T scale,
                                                       int zero_after, unsigned long long* step_ctr) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* rows = tw + N;
    load_twiddles(tw, tw_g, N);
    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)blockIdx.x * R * N;
    if (step_ctr && blockIdx.x == 0 && threadIdx.x == 0) *step_ctr += 1ull;
    load_fixed_rows<N, PITCH, R, 256>(rho_fx + base, rho_fx + M + base, rows, scale, zero_after);
    __syncthreads();
    smem_fft_lines<N, -1, R, 256>(rows, StridedLines<PITCH>{}, 1, tw);
    for (int i = threadIdx.x; i < R * N; i += blockDim.x) Zxy[base + i] = rows[(i / N) * PITCH + i % N];
}

template <typename T, int N, int R>
__global__ void __launch_bounds__(256) x_inverse_rows(const cplx_t<T>* __restrict__ H, cplx_t<T>* __restrict__ grad,
                                                       const cplx_t<T>* __restrict__ tw_g) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* rows = tw + N;
    load_twiddles(tw, tw_g, N);
    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)blockIdx.y * M + (size_t)blockIdx.x * R * N;
    for (int i = threadIdx.x; i < R * N; i += blockDim.x) rows[(i / N) * PITCH + i % N] = H[base + i];
    __syncthreads();
    smem_fft_lines<N, +1, R, 256>(rows, StridedLines<PITCH>{}, 1, tw);
    for (int i = threadIdx.x; i < R * N; i += blockDim.x) grad[base + i] = rows[(i / N) * PITCH + i % N];
}

// Column pass along y, in place: CTA (x tile, z, field) handles C columns.
template <typename T, int N, int C, int DIR>
__global__ void __launch_bounds__(256) y_columns(cplx_t<T>* __restrict__ data, const cplx_t<T>* __restrict__ tw_g) {
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* tile = tw + N;  // [y][c]
    load_twiddles(tw, tw_g, N);
    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)blockIdx.z * M + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * C;
    for (int i = threadIdx.x; i < N * C; i += blockDim.x) tile[i] = data[base + (size_t)(i / C) * N + i % C];
    __syncthreads();
    smem_fft_lines<N, DIR, C, 256>(tile, StridedLines<1>{}, C, tw);
    for (int i = threadIdx.x; i < N * C; i += blockDim.x) data[base + (size_t)(i / C) * N + i % C] = tile[i];
}

// --------------------------------------------------------------------------
// z pass: forward DFT along z, spectral multiply + gradient, inverse DFT
// along z. CTA (kx tile of C columns, ky). Loads its own tile and the
// mirror tile (-kx, -ky) that Hermitian separation needs.
// --------------------------------------------------------------------------
template <int C, int STRIDE> struct TileAddr {  // buffer b of a tile set starts at b * STRIDE
    __device__ __forceinline__ int operator()(int l) const { return (l / C) * STRIDE + l % C; }
};

template <typename T> __device__ __forceinline__ int freq_index(int i, int n) { return i < n / 2 ? i : i - n; }

template <typename T, int N, int C>
__global__ void __launch_bounds__(256) z_spectral(const cplx_t<T>* __restrict__ Zxy, cplx_t<T>* __restrict__ H,
                                                  const cplx_t<T>* __restrict__ tw_g, SpectralParams<T> sp,
                                                  double* __restrict__ energy_partials,
                                                  cplx_t<T>* __restrict__ spectrum_out) {
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* buf = tw + N;          // 3 buffers [N][C]: own, mirror, third
    const int TS = N * C;     // tile size
    __shared__ double red[2][32];
    __shared__ T e1[N];       // separable Gaussian kernel: u_hat = e1[kx] e1[ky] e1[kz]
    load_twiddles(tw, tw_g, N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) e1[i] = sp.kernel1d[i];

    const int c0 = blockIdx.x * C;
    const int ky = blockIdx.y;
    const int kym = (N - ky) & (N - 1);
    const size_t NN = (size_t)N * N;
    for (int i = threadIdx.x; i < TS; i += blockDim.x) {
        const int z = i / C, c = i % C;
        const int kx = c0 + c;
        const int kxm = (N - kx) & (N - 1);
        buf[i] = Zxy[z * NN + (size_t)ky * N + kx];
        buf[TS + i] = Zxy[z * NN + (size_t)kym * N + kxm];
    }
    __syncthreads();
    smem_fft_lines<N, -1, 2 * C, 256>(buf, TileAddr<C, N * C>{}, C, tw);

    if (spectrum_out) {
        for (int i = threadIdx.x; i < TS; i += blockDim.x)
            spectrum_out[(i / C) * NN + (size_t)ky * N + c0 + i % C] = buf[i];
    }

    const int my = freq_index<T>(ky, N);
    const T kyv = sp.two_pi_over_L * (T)my;
    const T kyg = (ky == N / 2) ? T(0) : kyv;
    double e_chi = 0.0, e_kap = 0.0;
    // pairs (kz, -kz): each thread owns both so in-place writes are safe
    for (int p = threadIdx.x; p < C * (N / 2 + 1); p += blockDim.x) {
        const int c = p % C, kz = p / C;
        const int kzm = (N - kz) & (N - 1);
        const int kx = c0 + c;
        const int mx = freq_index<T>(kx, N);
        const T kxv = sp.two_pi_over_L * (T)mx;
        const T kxg = (kx == N / 2) ? T(0) : kxv;
        const V Zk = buf[kz * C + c], Zkm = buf[kzm * C + c];
        const V Mk = buf[TS + kz * C + c], Mkm = buf[TS + kzm * C + c];
        V out[2][3];
        const int nsel = (kzm == kz) ? 1 : 2;
        for (int s = 0; s < nsel; ++s) {
            const int kzs = s == 0 ? kz : kzm;
            const V Z = s == 0 ? Zk : Zkm;   // Z(k)
            const V Zm = s == 0 ? Mkm : Mk;  // Z(-k)
            const T kzv = sp.two_pi_over_L * (T)freq_index<T>(kzs, N);
            const T kzg = (kzs == N / 2) ? T(0) : kzv;
            const T uh = e1[kx] * e1[ky] * e1[kzs];
            // rho~_A = (Z + conj Zm)/2, rho~_B = -i (Z - conj Zm)/2
            const V A = {T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y)};
            const V B = {T(0.5) * (Z.y + Zm.y), -T(0.5) * (Z.x - Zm.x)};
            if (energy_partials) {
                const double ar = A.x, ai = A.y, br = B.x, bi = B.y;
                e_chi += (double)uh * (ar * br + ai * bi);
                if (!(kx == 0 && ky == 0 && kzs == 0))
                    e_kap += (double)uh * ((ar + br) * (ar + br) + (ai + bi) * (ai + bi));
            }
            const V wA = {uh * (sp.eAA * A.x + sp.eAB * B.x), uh * (sp.eAA * A.y + sp.eAB * B.y)};
            const V wB = {uh * (sp.eAB * A.x + sp.eBB * B.x), uh * (sp.eAB * A.y + sp.eBB * B.y)};
            const V Q = {wA.x - wB.y, wA.y + wB.x};      // w~_A + i w~_B
            const V iQ = {-Q.y, Q.x};                     // i Q
            out[s][0] = {kxg * iQ.x, kxg * iQ.y};
            out[s][1] = {kyg * iQ.x, kyg * iQ.y};
            out[s][2] = {kzg * iQ.x, kzg * iQ.y};
        }
        for (int s = 0; s < nsel; ++s) {
            const int kzs = s == 0 ? kz : kzm;
            for (int d = 0; d < 3; ++d) buf[d * TS + kzs * C + c] = out[s][d];
        }
    }
    if (energy_partials) {
        // block reduction in a fixed order (deterministic)
        for (int o = 16; o > 0; o >>= 1) {
            e_chi += __shfl_down_sync(0xffffffffu, e_chi, o);
            e_kap += __shfl_down_sync(0xffffffffu, e_kap, o);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            red[0][wid] = e_chi;
            red[1][wid] = e_kap;
        }
    }
    __syncthreads();
    if (energy_partials && threadIdx.x == 0) {
        double s0 = 0, s1 = 0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        energy_partials[2 * b] = s0;
        energy_partials[2 * b + 1] = s1;
    }
    smem_fft_lines<N, +1, 3 * C, 256>(buf, TileAddr<C, N * C>{}, C, tw);
    const size_t M = NN * N;
    for (int i = threadIdx.x; i < 3 * TS; i += blockDim.x) {
        const int d = i / TS, r = i % TS;
        H[d * M + (r / C) * NN + (size_t)ky * N + c0 + r % C] = buf[i];
    }
}

}  // namespace tild
