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
// With more than two species (up to four) the species go in pairs: pair p
// carries species 2p and 2p+1 exactly as A and B above, and every array
// below gains a leading pair index; only the z pass sees all pairs at once
// (the spectral multiply couples every species).
//
// Memory layouts (n^3 points, index g = (z n + y) n + x; NP pairs):
//   rho_fx  int64 [2 NP][M]           fixed-point densities (2^22 or 2^44 per bead weight)
//   Zxy     complex [NP][z][ky][pos(kx)]  after the forward x and y transforms
//   H       complex [NP][3][z][ky][pos(kx)] after the z pass (z back in real space)
// (pos(kx): mirror-paired column order, see kx_of_pos)
//   grad    complex [NP][4][z][y][x]  (d w_2p, d w_2p+1) per point and direction,
//                                     then the potentials i (w_2p + i w_2p+1)
#pragma once

#include "fft.cuh"

namespace tild {

template <typename T> struct SpectralParams {
    T two_pi_over_L;   // 2 pi / L
    T eAA, eAB, eBB;   // eps matrix / M (the 1/M of the inverse DFT folded in)
    T eps4[4][4];      // more than two species: eps_KK' / M
    T chi4[4][4];      // more than two species: chi_KK' (the energy sum of the z pass weights by it)
    const T* kernel1d; // exp(-a^2 k_m^2) per 1-D frequency index m (FP64 on the host)
    // smeared-charge electrostatics: w_K += q_K c(k) (q_A rho~_A + q_B rho~_B) with
    // c(k) = el_scale exp(-a_e^2 |k|^2) / |k|^2 (0 at k = 0); el_scale = 4 pi l_B / M
    // (0: no charges); kernel1d_el = exp(-a_e^2 k_m^2)
    T el_scale, qA, qB;
    const T* kernel1d_el;
};

template <int N> __host__ __device__ __forceinline__ int kx_of_pos(int p);
template <int C, int STRIDE> struct TileAddr;

// Wavenumber 2 pi m / L of FFT index i (m = i or i - n; the Nyquist index
// n/2 counts as -n/2).
template <typename T, int N> __device__ __forceinline__ T raw_k(int i, T two_pi_over_L) {
    return two_pi_over_L * (T)(i < N / 2 ? i : i - N);
}

// Wavenumber used for spectral differentiation at FFT index i: 2 pi m / L
// with m = i (i < n/2) or i - n, and 0 at the Nyquist index n/2.
template <typename T, int N> __device__ __forceinline__ T grad_k(int i, T two_pi_over_L) {
    return i == N / 2 ? T(0) : two_pi_over_L * (T)(i < N / 2 ? i : i - N);
}

// 1/x: the correctly rounded reciprocal intrinsic in FP32 (no division
// slow path), a plain division in FP64.
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

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

// Copy COUNT elements from global to shared memory with up to 16
// independent loads in flight per thread: dst(i, value) stores element i.
// Accesses are guarded by i < COUNT unless every thread's batches are full
// (COUNT a multiple of NTHR and PER a multiple of the batch); otherwise the
// last batch of a thread may be partial.
template <int COUNT, int NTHR, class V, class Src, class Dst>
__device__ __forceinline__ void batched_load(Src src, Dst dst) {
    constexpr int PER = (COUNT + NTHR - 1) / NTHR;
    constexpr int B = PER < 16 ? PER : 16;
    constexpr bool kFull = COUNT % NTHR == 0 && PER % B == 0;
#pragma unroll 1
    for (int k0 = 0; k0 < PER; k0 += B) {
        V v[B];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (kFull || i < COUNT) v[k] = src(i);
        }
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (kFull || i < COUNT) dst(i, v[k]);
        }
    }
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
    constexpr int BATCH = ITER < 8 ? ITER : 8;
    constexpr bool kFull = PAIRS % NTHR == 0 && ITER % BATCH == 0;  // no partial batch
    longlong2* pa = reinterpret_cast<longlong2*>(ga);
    longlong2* pb = reinterpret_cast<longlong2*>(gb);
#pragma unroll 1
    for (int k0 = 0; k0 < ITER; k0 += BATCH) {
        longlong2 a[BATCH], b[BATCH];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (kFull || i < PAIRS) {
                a[k] = __ldcs(pa + i);
                b[k] = __ldcs(pb + i);
            }
        }
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int i = threadIdx.x + (k0 + k) * NTHR;
            if (kFull || i < PAIRS) {
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
// grid = n (one CTA per z-plane), block = NT (512, or 128/256 for small
// planes, where several CTAs then share an SM).
// --------------------------------------------------------------------------
template <typename T> struct ForwardArgs {
    unsigned long long* rho_fx;
    cplx_t<T>* Zxy;
    const cplx_t<T>* tw;
    T scale;
    int zero_after;
    unsigned long long* step_ctr;
};

template <typename T, int N, int NT = 512>
__device__ __forceinline__ void xy_forward_plane_body(const ForwardArgs<T>& args, int bx) {
    using V = cplx_t<T>;
    unsigned long long* __restrict__ rho_fx = args.rho_fx;
    cplx_t<T>* __restrict__ Zxy = args.Zxy;
    const cplx_t<T>* __restrict__ tw_g = args.tw;
    const T scale = args.scale;
    const int zero_after = args.zero_after;
    unsigned long long* step_ctr = args.step_ctr;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* plane = tw + N;
    load_twiddles(tw, tw_g, N);
    // a step's first kernel advances the noise counter to n+1
    if (step_ctr && bx == 0 && threadIdx.x == 0) *step_ctr += 1ull;

    const int z = bx;
    const size_t M = (size_t)N * N * N;
    const size_t base = (size_t)z * N * N;
    // load + convert: pairs of x so that global accesses are 16-byte vectors
    load_fixed_rows<N, PITCH, N, NT>(rho_fx + base, rho_fx + M + base, plane, scale, zero_after);
    __syncthreads();
    smem_fft_lines<N, -1, N, NT>(plane, StridedLines<PITCH>{}, 1, tw);  // along x
    smem_fft_lines<N, -1, N, NT>(plane, StridedLines<1>{}, PITCH, tw);  // along y
    for (int i = threadIdx.x; i < N * N; i += NT) {
        const int y = i / N, x = i % N;
        Zxy[base + i] = plane[y * PITCH + kx_of_pos<N>(x)];  // mirror-paired column order
    }
}

// grid = (n, NP): species pair blockIdx.y
template <typename T, int N, int NT = 512>
__global__ void __launch_bounds__(NT) xy_forward_plane(unsigned long long* __restrict__ rho_fx,
                                                         cplx_t<T>* __restrict__ Zxy,
                                                         const cplx_t<T>* __restrict__ tw_g, T scale,
                                                         int zero_after, unsigned long long* step_ctr) {
    const size_t M = (size_t)N * N * N;
    const int pr = blockIdx.y;
    xy_forward_plane_body<T, N, NT>(
        ForwardArgs<T>{rho_fx + 2 * pr * M, Zxy + pr * M, tw_g, scale, zero_after, pr == 0 ? step_ctr : nullptr},
        blockIdx.x);
}

// Batched form: replica blockIdx.y of a table of replicas with the same grid.
template <typename T, int N, int NT = 512>
__global__ void __launch_bounds__(NT) xy_forward_plane_batched(const ForwardArgs<T>* __restrict__ args) {
    xy_forward_plane_body<T, N, NT>(args[blockIdx.y], blockIdx.x);
}

// --------------------------------------------------------------------------
// Inverse xy pass on whole z-planes: grid = (n, 3), block = NT.
// --------------------------------------------------------------------------
template <typename T> struct InverseArgs {
    const cplx_t<T>* H;
    cplx_t<T>* grad;
    const cplx_t<T>* tw;
    T two_pi_over_L;
    int d0;  // first direction (blockIdx.y + d0); 3 alone: the potentials only
};

template <typename T, int N, int NT = 512>
__device__ __forceinline__ void xy_inverse_plane_body(const InverseArgs<T>& args, int bx, int by) {
    using V = cplx_t<T>;
    const cplx_t<T>* __restrict__ H = args.H;
    cplx_t<T>* __restrict__ grad = args.grad;
    const cplx_t<T>* __restrict__ tw_g = args.tw;
    const T two_pi_over_L = args.two_pi_over_L;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* plane = tw + N;
    load_twiddles(tw, tw_g, N);

    // direction d: x from i k_x G, y from i k_y G, z from G_z (field 2);
    // d = 3 (optional): the potentials themselves, i (w_A + i w_B), from G
    const int d = by + args.d0;
    const size_t M = (size_t)N * N * N;
    const size_t src = (d == 2 ? 2 * M : 0) + (size_t)bx * N * N;
    batched_load<N * N, NT, V>([&](int i) { return H[src + i]; },
                                [&](int i, V v) {
                                    const int ky = i / N;
                                    if (d == 1) v = c_scale(v, grad_k<T, N>(ky, two_pi_over_L));
                                    plane[ky * PITCH + kx_of_pos<N>(i % N)] = v;
                                });
    __syncthreads();
    smem_fft_lines<N, +1, N, NT>(plane, StridedLines<1>{}, PITCH, tw);  // along y
    if (d == 0) {
        for (int i = threadIdx.x; i < N * N; i += NT) {
            const int y = i / N, kx = i % N;
            plane[y * PITCH + kx] = c_scale(plane[y * PITCH + kx], grad_k<T, N>(kx, two_pi_over_L));
        }
        __syncthreads();
    }
    smem_fft_lines<N, +1, N, NT>(plane, StridedLines<PITCH>{}, 1, tw);  // along x
    const size_t dst = (size_t)d * M + (size_t)bx * N * N;
    for (int i = threadIdx.x; i < N * N; i += NT) grad[dst + i] = plane[(i / N) * PITCH + i % N];
}

// grid = (n, directions, NP): species pair blockIdx.z
template <typename T, int N, int NT = 512>
__global__ void __launch_bounds__(NT) xy_inverse_plane(const cplx_t<T>* __restrict__ H,
                                                         cplx_t<T>* __restrict__ grad,
                                                         const cplx_t<T>* __restrict__ tw_g, T two_pi_over_L, int d0) {
    const size_t M = (size_t)N * N * N;
    const int pr = blockIdx.z;
    xy_inverse_plane_body<T, N, NT>(InverseArgs<T>{H + 3 * pr * M, grad + 4 * pr * M, tw_g, two_pi_over_L, d0},
                                    blockIdx.x, blockIdx.y);
}

// Batched form: replica blockIdx.z.
template <typename T, int N, int NT = 512>
__global__ void __launch_bounds__(NT) xy_inverse_plane_batched(const InverseArgs<T>* __restrict__ args) {
    xy_inverse_plane_body<T, N, NT>(args[blockIdx.z], blockIdx.x, blockIdx.y);
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
    const int pr = blockIdx.y;  // species pair
    rho_fx += 2 * pr * M;
    Zxy += pr * M;
    if (step_ctr && blockIdx.x == 0 && pr == 0 && threadIdx.x == 0) *step_ctr += 1ull;
    load_fixed_rows<N, PITCH, R, 256>(rho_fx + base, rho_fx + M + base, rows, scale, zero_after);
    __syncthreads();
    smem_fft_lines<N, -1, R, 256>(rows, StridedLines<PITCH>{}, 1, tw);
    for (int i = threadIdx.x; i < R * N; i += blockDim.x) Zxy[base + i] = rows[(i / N) * PITCH + kx_of_pos<N>(i % N)];
}

template <typename T, int N, int R>
__global__ void __launch_bounds__(256) x_inverse_rows(const cplx_t<T>* __restrict__ H, cplx_t<T>* __restrict__ grad,
                                                       const cplx_t<T>* __restrict__ tw_g, T two_pi_over_L, int d0) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* rows = tw + N;
    load_twiddles(tw, tw_g, N);
    const size_t M = (size_t)N * N * N;
    const int d = (int)blockIdx.y + d0;
    H += 3 * (size_t)blockIdx.z * M;  // species pair blockIdx.z
    grad += 4 * (size_t)blockIdx.z * M;
    const size_t base = (size_t)d * M + (size_t)blockIdx.x * R * N;
    // field 3 (optional, the potentials) is the plain transform of field 0
    const size_t src = (size_t)(d == 3 ? 0 : d) * M + (size_t)blockIdx.x * R * N;
    const bool kx_mult = d == 0;  // d_x: multiply by k_x before the x transform
    batched_load<R * N, 256, V>([&](int i) { return H[src + i]; },
                                [&](int i, V v) {
                                    const int kx = kx_of_pos<N>(i % N);
                                    if (kx_mult) v = c_scale(v, grad_k<T, N>(kx, two_pi_over_L));
                                    rows[(i / N) * PITCH + kx] = v;
                                });
    __syncthreads();
    smem_fft_lines<N, +1, R, 256>(rows, StridedLines<PITCH>{}, 1, tw);
    for (int i = threadIdx.x; i < R * N; i += blockDim.x) grad[base + i] = rows[(i / N) * PITCH + i % N];
}

// Column pass along y: CTA (x tile, z plane, part) handles C columns.
// Forward (DIR = -1): Zxy in place; blockIdx.z = species pair.
// Inverse (DIR = +1) on H: part 0 loads a tile of G (field 0) and writes
// the transforms of G (field 0) and of i k_y G (field 1) from the same
// load; part 1 transforms G_z (field 2) in place; blockIdx.z = 2 pair +
// part. With only_g, one part transforms G alone (blockIdx.z = pair).
template <typename T, int N, int C, int DIR>
__global__ void __launch_bounds__(256) y_columns(cplx_t<T>* __restrict__ data, const cplx_t<T>* __restrict__ tw_g,
                                                 T two_pi_over_L, int only_g) {
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* tile = tw + N;  // [2][y][c]
    constexpr int TS = N * C;
    load_twiddles(tw, tw_g, N);
    const size_t M = (size_t)N * N * N;
    const int part = (DIR < 0 || only_g) ? 0 : (int)(blockIdx.z & 1);
    const int pr = (DIR < 0 || only_g) ? (int)blockIdx.z : (int)(blockIdx.z >> 1);
    data += (DIR < 0 ? 1 : 3) * (size_t)pr * M;
    const bool two = DIR > 0 && part == 0 && !only_g;  // only_g: G alone (one part)
    const size_t off = (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * C;
    const size_t src = (DIR > 0 && part == 1 ? 2 * M : 0) + off;
    batched_load<TS, 256, V>([&](int i) { return data[src + (size_t)(i / C) * N + i % C]; },
                             [&](int i, V v) {
                                 tile[i] = v;
                                 if (two) tile[TS + i] = c_scale(v, grad_k<T, N>(i / C, two_pi_over_L));
                             });
    __syncthreads();
    if (two) {
        smem_fft_lines<N, DIR, 2 * C, 256>(tile, TileAddr<C, TS>{}, C, tw);
        for (int i = threadIdx.x; i < TS; i += blockDim.x) {
            data[off + (size_t)(i / C) * N + i % C] = tile[i];
            data[M + off + (size_t)(i / C) * N + i % C] = tile[TS + i];
        }
    } else {
        smem_fft_lines<N, DIR, C, 256>(tile, StridedLines<1>{}, C, tw);
        for (int i = threadIdx.x; i < TS; i += blockDim.x) data[src + (size_t)(i / C) * N + i % C] = tile[i];
    }
}

// --------------------------------------------------------------------------
// Column order of the xy-transformed arrays (Zxy and H): mirror pairs
// (kx, -kx) are adjacent so that a tile of an even number of positions is
// closed under kx -> -kx. Position 0 holds kx = 0, position 1 kx = n/2, and
// positions 2k, 2k+1 hold kx = k and n - k (k = 1 .. n/2 - 1).
// --------------------------------------------------------------------------
template <int N> __host__ __device__ __forceinline__ int kx_of_pos(int p) {
    return p == 0 ? 0 : p == 1 ? N / 2 : (p & 1) ? N - (p >> 1) : (p >> 1);
}
__host__ __device__ __forceinline__ int mirror_pos(int p) { return p < 2 ? p : (p ^ 1); }

template <int C, int STRIDE> struct TileAddr {  // buffer b of a tile set starts at b * STRIDE
    __device__ __forceinline__ int operator()(int l) const { return (l / C) * STRIDE + l % C; }
};

template <typename T> __device__ __forceinline__ int freq_index(int i, int n) { return i < n / 2 ? i : i - n; }

// --------------------------------------------------------------------------
// z pass: forward DFT along z, spectral multiply + gradient, inverse DFT
// along z. CTA (tile of C column positions, ky pair {ky, -ky}); the tile
// holds every column's mirror, so each CTA has Z(k) and Z(-k) for all of its
// elements and transforms each input line once.
//   R = 1 row when ky = -ky (ky = 0 or n/2), else 2 rows.
// Outputs (linearity: k_x and k_y are constant along a z line):
//   G   = IDFT_z[ i Q ]       (field 0; d_x and d_y follow in the xy pass)
//   G_z = IDFT_z[ i k_z Q ]   (field 2)
// with Q = w~_A + i w~_B. Buffers [2R][N][C]: G of row r in buffer r
// (overwriting the input), G_z in buffer R + r.
// --------------------------------------------------------------------------
// out(b, c, z, v): output element z of column c of buffer b (the inverse
// transforms' results, handed over as their last stage produces them).
template <typename T, int N, int C, int R, bool G_ONLY, bool EL, class Out>
__device__ __forceinline__ void z_tile(cplx_t<T>* buf, const cplx_t<T>* tw, const T* e1, const SpectralParams<T>& sp,
                                       int p0, const int (&ky)[2], bool want_e, double (&acc)[5], const T* e2, Out out) {
    using V = cplx_t<T>;
    constexpr int TS = N * C;
    static_assert(256 % C == 0, "a thread keeps one column");
    constexpr int rB = R - 1;
    // column constants of element A (row 0, column c) and its mirror B (row
    // rB, column cB)
    struct Col {
        int cB;
        T exyA, exyB, exy2A, exy2B;
        bool zeroA, zeroB;
        double kxy2A, kxy2B;  // |k_x|^2 + |k_y|^2 (the Nyquist index counts as -n/2)
    };
    auto col_of = [&](int c) {
        Col cl;
        cl.cB = mirror_pos(p0 + c) - p0;
        const int kxA = kx_of_pos<N>(p0 + c), kxB = kx_of_pos<N>(p0 + cl.cB);
        cl.exyA = e1[kxA] * e1[ky[0]];
        cl.exyB = e1[kxB] * e1[ky[rB]];
        cl.zeroA = (kxA == 0 && ky[0] == 0);
        cl.zeroB = (kxB == 0 && ky[rB] == 0);
        const T qxA = raw_k<T, N>(kxA, sp.two_pi_over_L), qyA = raw_k<T, N>(ky[0], sp.two_pi_over_L);
        const T qxB = raw_k<T, N>(kxB, sp.two_pi_over_L), qyB = raw_k<T, N>(ky[rB], sp.two_pi_over_L);
        cl.kxy2A = (double)qxA * qxA + (double)qyA * qyA;
        cl.kxy2B = (double)qxB * qxB + (double)qyB * qyB;
        cl.exy2A = EL ? e2[kxA] * e2[ky[0]] : T(0);
        cl.exy2B = EL ? e2[kxB] * e2[ky[rB]] : T(0);
        return cl;
    };
    // the spectral multiply of one mirror pair: ZA = Z(k) at (row 0, c, kz),
    // ZB = Z(-k) at (row rB, cB, kzB); out[s][d]: s = 0 for A, 1 for B,
    // d = 0 for iQ (G), 1 for i k_z Q (G_z)
    struct Mult {
        V g[2], gz[2];  // iQ and i k_z Q of A (0) and B (1)
    };
    auto mult = [&](const Col& cl, V ZA, V ZB, int kz, int kzB, bool same) {
        Mult out;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && same) break;
            const V Z = s == 0 ? ZA : ZB;   // Z(k)
            const V Zm = s == 0 ? ZB : ZA;  // Z(-k)
            const int kzi = s == 0 ? kz : kzB;
            const T kzv = grad_k<T, N>(kzi, sp.two_pi_over_L);
            const T uh = (s == 0 ? cl.exyA : cl.exyB) * e1[kzi];
            // rho~_A = (Z + conj Zm)/2, rho~_B = -i (Z - conj Zm)/2
            const V A = {T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y)};
            const V B = {T(0.5) * (Z.y + Zm.y), -T(0.5) * (Z.x - Zm.x)};
            if (want_e) {
                // energy sums and their |k|^2-weighted versions (d u_hat / d a = -2 a |k|^2 u_hat)
                const double ar = A.x, ai = A.y, br = B.x, bi = B.y;
                const double qz = (double)raw_k<T, N>(kzi, sp.two_pi_over_L);
                const double k2 = (s == 0 ? cl.kxy2A : cl.kxy2B) + qz * qz;
                const double fchi = (double)uh * (ar * br + ai * bi);
                acc[0] += fchi;
                acc[2] += k2 * fchi;
                if (!((s == 0 ? cl.zeroA : cl.zeroB) && kzi == 0)) {
                    const double fkap = (double)uh * ((ar + br) * (ar + br) + (ai + bi) * (ai + bi));
                    acc[1] += fkap;
                    acc[3] += k2 * fkap;
                }
            }
            V wA = {uh * (sp.eAA * A.x + sp.eAB * B.x), uh * (sp.eAA * A.y + sp.eAB * B.y)};
            V wB = {uh * (sp.eAB * A.x + sp.eBB * B.x), uh * (sp.eAB * A.y + sp.eBB * B.y)};
            if (EL) {
                // w_K += q_K c(k) rho~_q with rho~_q = q_A rho~_A + q_B rho~_B
                const T qzv = raw_k<T, N>(kzi, sp.two_pi_over_L);
                const T k2 = (T)(s == 0 ? cl.kxy2A : cl.kxy2B) + qzv * qzv;
                const T g = k2 > T(0) ? (s == 0 ? cl.exy2A : cl.exy2B) * e2[kzi] * recip(k2) : T(0);
                const V rq = {sp.qA * A.x + sp.qB * B.x, sp.qA * A.y + sp.qB * B.y};
                const T c = sp.el_scale * g;
                wA.x += c * sp.qA * rq.x;
                wA.y += c * sp.qA * rq.y;
                wB.x += c * sp.qB * rq.x;
                wB.y += c * sp.qB * rq.y;
                if (want_e) acc[4] += (double)g * ((double)rq.x * rq.x + (double)rq.y * rq.y);
            }
            const V iQ = {-(wA.y + wB.x), wA.x - wB.y};  // i (w~_A + i w~_B)
            out.g[s] = iQ;                                // x, y: k_x, k_y applied in the xy pass
            out.gz[s] = {kzv * iQ.x, kzv * iQ.y};         // z
        }
        return out;
    };
    auto store = [&](const Mult& out, int c, int cB, int kz, int kzB, bool same) {
        buf[kz * C + c] = out.g[0];
        if (!same) buf[rB * TS + kzB * C + cB] = out.g[1];
        if (!G_ONLY) {
            buf[R * TS + kz * C + c] = out.gz[0];
            if (!same) buf[(R + rB) * TS + kzB * C + cB] = out.gz[1];
        }
    };
    constexpr int N1 = fft_split<N>::N1, N2 = fft_split<N>::N2;
    if constexpr (R == 2 && !EL && N2 > 1 && C * N1 == 256) {
        // two rows: the forward transform's second stage and the multiply in
        // registers (tiles where every thread has one pair of units). Thread q
        // takes stage-B unit (row 0, column c, k1)
        // and the unit holding the mirrors of its outputs, (row 1, column cB,
        // (N1 - k1) mod N1); the outputs X[k1 + N1 k2] of the first meet
        // their mirrors X[-(k1 + N1 k2)] in the second, so each pair is
        // multiplied where the transform left it (same operations as the
        // transform followed by the loop below).
        smem_fft_stage_a<N, -1, R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
        const int q = threadIdx.x;
        const bool active = q < C * N1;
        const int c = q % C, k1 = q / C;
        const int k1B = (N1 - k1) % N1;
        const Col cl = col_of(c);
        V va[N2], vb[N2];
        if (active) {
            const V* pa = buf + c + k1 * N2 * C;             // line c of row 0: positions k1 N2 + j2
            const V* pb = buf + TS + cl.cB + k1B * N2 * C;   // line cB of row 1
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) {
                va[j2] = pa[j2 * C];
                vb[j2] = pb[j2 * C];
            }
        }
        __syncthreads();  // every stage-B input is read before any output is written
        if (active) {
            reg_dft<N2, -1, V>::run(va);
            reg_dft<N2, -1, V>::run(vb);
            // the mirror of output k2: (N2 - k2) mod N2 when k1 = 0, else N2 - 1 - k2
            // (selected with constant indices, so the arrays stay in registers)
            V vm[N2];
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) vm[k2] = k1 == 0 ? vb[(N2 - k2) % N2] : vb[N2 - 1 - k2];
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int kz = k1 + N1 * k2;
                const int kzB = kz == 0 ? 0 : N - kz;
                store(mult(cl, va[k2], vm[k2], kz, kzB, false), c, cl.cB, kz, kzB, false);
            }
        }
    } else {
        smem_fft_lines<N, -1, R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
        const int c = threadIdx.x % C;
        const Col cl = col_of(c);
        for (int kz = threadIdx.x / C; kz < N; kz += 256 / C) {
            const int kzB = kz == 0 ? 0 : N - kz;
            if (R == 1 && kzB * C + cl.cB < kz * C + c) continue;  // the mirror element owns this pair
            const bool same = (R == 1) && (kzB == kz) && (cl.cB == c);
            store(mult(cl, buf[kz * C + c], buf[rB * TS + kzB * C + cl.cB], kz, kzB, same), c, cl.cB, kz, kzB, same);
        }
    }
    __syncthreads();
    constexpr int NB = (G_ONLY ? 1 : 2) * R;  // output buffers
    if constexpr (N2 > 1) {
        smem_fft_lines_out<N, +1, NB * C, 256>(buf, TileAddr<C, TS>{}, C, tw,
                                                [&](int l, int z, V v) { out(l / C, l % C, z, v); });
    } else {
        smem_fft_lines<N, +1, NB * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
        for (int i = threadIdx.x; i < NB * TS; i += blockDim.x) out(i / TS, i % C, (i % TS) / C, buf[i]);
    }
}

template <typename T> struct ZArgs {
    const cplx_t<T>* Zxy;
    cplx_t<T>* H;
    const cplx_t<T>* tw;
    SpectralParams<T> sp;
    double* energy_partials;
    cplx_t<T>* spectrum_out;
};

template <typename T, int N, int C, bool G_ONLY = false, bool EL = false>
__device__ __forceinline__ void z_spectral_body(const ZArgs<T>& args, int bx, int by, int gdx) {
    using V = cplx_t<T>;
    const cplx_t<T>* __restrict__ Zxy = args.Zxy;
    cplx_t<T>* __restrict__ H = args.H;
    const cplx_t<T>* __restrict__ tw_g = args.tw;
    const SpectralParams<T> sp = args.sp;
    double* __restrict__ energy_partials = args.energy_partials;
    cplx_t<T>* __restrict__ spectrum_out = args.spectrum_out;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* buf = tw + N;
    constexpr int TS = N * C;
    __shared__ double red[5][8];
    __shared__ T e1[N];  // separable Gaussian kernel: u_hat = e1[kx] e1[ky] e1[kz]
    __shared__ T e2[N];  // charge smearing exp(-a_e^2 k_m^2), when charges are on
    load_twiddles(tw, tw_g, N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) e1[i] = sp.kernel1d[i];
    if (EL)
        for (int i = threadIdx.x; i < N; i += blockDim.x) e2[i] = sp.kernel1d_el[i];

    const int p0 = bx * C;
    const int ky[2] = {by, by == 0 ? 0 : N - by};
    const int R = (ky[0] == ky[1]) ? 1 : 2;
    const size_t NN = (size_t)N * N;
    auto zsrc = [&](int i) {
        const int r = i / TS, rem = i % TS;
        const int z = rem / C, c = rem % C;
        return Zxy[z * NN + (size_t)ky[r] * N + p0 + c];
    };
    auto zdst = [&](int i, V v) { buf[i] = v; };
    if (R == 1)
        batched_load<TS, 256, V>(zsrc, zdst);
    else
        batched_load<2 * TS, 256, V>(zsrc, zdst);
    __syncthreads();
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const bool want_e = energy_partials != nullptr;
    if (spectrum_out) {
        // forward transform only, written out in natural kx order
        if (R == 1)
            smem_fft_lines<N, -1, C, 256>(buf, TileAddr<C, TS>{}, C, tw);
        else
            smem_fft_lines<N, -1, 2 * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
        for (int i = threadIdx.x; i < R * TS; i += blockDim.x) {
            const int r = i / TS, rem = i % TS;
            const int z = rem / C, c = rem % C;
            spectrum_out[z * NN + (size_t)ky[r] * N + kx_of_pos<N>(p0 + c)] = buf[i];
        }
        return;
    }
    const size_t M = NN * N;
    // G of row r to field 0, G_z to field 2, at (z, ky[r], p0 + c)
    auto store_h = [&](int rr, int b, int c, int z, V v) {
        const int f = (b / rr) * 2, r = b % rr;
        H[f * M + z * NN + (size_t)ky[r] * N + p0 + c] = v;
    };
    if (R == 1)
        z_tile<T, N, C, 1, G_ONLY, EL>(buf, tw, e1, sp, p0, ky, want_e, acc, e2,
                                       [&](int b, int c, int z, V v) { store_h(1, b, c, z, v); });
    else
        z_tile<T, N, C, 2, G_ONLY, EL>(buf, tw, e1, sp, p0, ky, want_e, acc, e2,
                                       [&](int b, int c, int z, V v) { store_h(2, b, c, z, v); });
    if (want_e) {
        // block reduction in a fixed order (deterministic)
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double sum = 0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) sum += red[threadIdx.x][w];
            const size_t b = (size_t)by * gdx + bx;
            energy_partials[5 * b + threadIdx.x] = sum;
        }
    }
}

// G_ONLY: write G alone (the potentials' path of the analytic force).
// EL: add the smeared-charge Coulomb term (charges on).
template <typename T, int N, int C, bool G_ONLY = false, bool EL = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (C <= 8 ? 4 : 3) : 1) z_spectral(const cplx_t<T>* __restrict__ Zxy, cplx_t<T>* __restrict__ H,
                                                  const cplx_t<T>* __restrict__ tw_g, SpectralParams<T> sp,
                                                  double* __restrict__ energy_partials,
                                                  cplx_t<T>* __restrict__ spectrum_out) {
    z_spectral_body<T, N, C, G_ONLY, EL>(ZArgs<T>{Zxy, H, tw_g, sp, energy_partials, spectrum_out}, blockIdx.x,
                                     blockIdx.y, gridDim.x);
}

// Batched form: replica blockIdx.z.
template <typename T, int N, int C, bool EL = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) z_spectral_batched(const ZArgs<T>* __restrict__ args) {
    z_spectral_body<T, N, C, false, EL>(args[blockIdx.z], blockIdx.x, blockIdx.y, gridDim.x);
}

// --------------------------------------------------------------------------
// z pass with two species pairs (three or four species): as z_spectral, on
// both pairs' columns at once. Buffers [2 NP R][N][C]: the input (then G) of
// pair p, row r in buffer p R + r; G_z in buffer NP R + p R + r. The
// species spectra of pair p are rho~_2p = (Z_p(k) + conj Z_p(-k))/2 and
// rho~_2p+1 = -i (Z_p(k) - conj Z_p(-k))/2; w~_K = u_hat sum_K' eps_KK'
// rho~_K'; Q_p = w~_2p + i w~_2p+1. Energy partials: [0] sum_k u_hat
// sum_{K<K'} chi_KK' Re[conj(rho~_K) rho~_K'], [1] sum_{k != 0} u_hat
// |sum_K rho~_K|^2, [2], [3] the same weighted by |k|^2, [4] 0.
// --------------------------------------------------------------------------
template <typename T, int N, int C, int R, bool G_ONLY>
__device__ __forceinline__ void z_tile_pairs(cplx_t<T>* buf, const cplx_t<T>* tw, const T* e1, const SpectralParams<T>& sp,
                                             int p0, const int (&ky)[2], bool want_e, double (&acc)[5]) {
    using V = cplx_t<T>;
    constexpr int TS = N * C;
    constexpr int NP = 2;
    smem_fft_lines<N, -1, NP * R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
    static_assert(256 % C == 0, "a thread keeps one column");
    constexpr int rB = R - 1;
    const int c = threadIdx.x % C;
    const int cB = mirror_pos(p0 + c) - p0;
    const int kxA = kx_of_pos<N>(p0 + c), kxB = kx_of_pos<N>(p0 + cB);
    const T exyA = e1[kxA] * e1[ky[0]], exyB = e1[kxB] * e1[ky[rB]];
    const bool zeroA = (kxA == 0 && ky[0] == 0), zeroB = (kxB == 0 && ky[rB] == 0);
    const T qxA = raw_k<T, N>(kxA, sp.two_pi_over_L), qyA = raw_k<T, N>(ky[0], sp.two_pi_over_L);
    const T qxB = raw_k<T, N>(kxB, sp.two_pi_over_L), qyB = raw_k<T, N>(ky[rB], sp.two_pi_over_L);
    const double kxy2A = (double)qxA * qxA + (double)qyA * qyA, kxy2B = (double)qxB * qxB + (double)qyB * qyB;
    for (int kz = threadIdx.x / C; kz < N; kz += 256 / C) {
        const int kzB = kz == 0 ? 0 : N - kz;
        if (R == 1 && kzB * C + cB < kz * C + c) continue;  // the mirror element owns this pair
        const bool same = (R == 1) && (kzB == kz) && (cB == c);
        V ZA[NP], ZB[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            ZA[q] = buf[(q * R) * TS + kz * C + c];
            ZB[q] = buf[(q * R + rB) * TS + kzB * C + cB];
        }
        V out[2][NP][2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && same) break;
            const int kzi = s == 0 ? kz : kzB;
            const T kzv = grad_k<T, N>(kzi, sp.two_pi_over_L);
            const T uh = (s == 0 ? exyA : exyB) * e1[kzi];
            V A[2 * NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const V Z = s == 0 ? ZA[q] : ZB[q];
                const V Zm = s == 0 ? ZB[q] : ZA[q];
                A[2 * q] = {T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y)};
                A[2 * q + 1] = {T(0.5) * (Z.y + Zm.y), -T(0.5) * (Z.x - Zm.x)};
            }
            if (want_e) {
                const double qz = (double)raw_k<T, N>(kzi, sp.two_pi_over_L);
                const double k2 = (s == 0 ? kxy2A : kxy2B) + qz * qz;
                double fchi = 0.0;
#pragma unroll
                for (int K = 0; K < 2 * NP; ++K)
#pragma unroll
                    for (int K2 = K + 1; K2 < 2 * NP; ++K2)
                        fchi += (double)sp.chi4[K][K2] * ((double)A[K].x * A[K2].x + (double)A[K].y * A[K2].y);
                fchi *= (double)uh;
                acc[0] += fchi;
                acc[2] += k2 * fchi;
                if (!((s == 0 ? zeroA : zeroB) && kzi == 0)) {
                    double tr = 0.0, ti = 0.0;
#pragma unroll
                    for (int K = 0; K < 2 * NP; ++K) {
                        tr += A[K].x;
                        ti += A[K].y;
                    }
                    const double fkap = (double)uh * (tr * tr + ti * ti);
                    acc[1] += fkap;
                    acc[3] += k2 * fkap;
                }
            }
            V w[2 * NP];
#pragma unroll
            for (int K = 0; K < 2 * NP; ++K) {
                T wr = 0, wi = 0;
#pragma unroll
                for (int K2 = 0; K2 < 2 * NP; ++K2) {
                    wr += sp.eps4[K][K2] * A[K2].x;
                    wi += sp.eps4[K][K2] * A[K2].y;
                }
                w[K] = {uh * wr, uh * wi};
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const V iQ = {-(w[2 * q].y + w[2 * q + 1].x), w[2 * q].x - w[2 * q + 1].y};  // i (w~_2q + i w~_2q+1)
                out[s][q][0] = iQ;
                out[s][q][1] = {kzv * iQ.x, kzv * iQ.y};
            }
        }
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            if (d == 1 && G_ONLY) break;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                buf[(d * NP * R + q * R) * TS + kz * C + c] = out[0][q][d];
                if (!same) buf[(d * NP * R + q * R + rB) * TS + kzB * C + cB] = out[1][q][d];
            }
        }
    }
    __syncthreads();
    smem_fft_lines<N, +1, (G_ONLY ? 1 : 2) * NP * R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
}

template <typename T, int N, int C, bool G_ONLY = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) z_spectral_pairs(const cplx_t<T>* __restrict__ Zxy,
                                                                                cplx_t<T>* __restrict__ H,
                                                                                const cplx_t<T>* __restrict__ tw_g,
                                                                                SpectralParams<T> sp,
                                                                                double* __restrict__ energy_partials) {
    using V = cplx_t<T>;
    constexpr int NP = 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* buf = tw + N;
    constexpr int TS = N * C;
    __shared__ double red[5][8];
    __shared__ T e1[N];
    load_twiddles(tw, tw_g, N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) e1[i] = sp.kernel1d[i];
    const int bx = blockIdx.x, by = blockIdx.y;
    const int p0 = bx * C;
    const int ky[2] = {by, by == 0 ? 0 : N - by};
    const int R = (ky[0] == ky[1]) ? 1 : 2;
    const size_t NN = (size_t)N * N, M = NN * N;
    // buffer b = q R + r (pair q, row r)
    auto zsrc = [&](int i) {
        const int b = i / TS, rem = i % TS;
        const int q = b / R, r = b % R;
        const int z = rem / C, c = rem % C;
        return Zxy[q * M + z * NN + (size_t)ky[r] * N + p0 + c];
    };
    auto zdst = [&](int i, V v) { buf[i] = v; };
    if (R == 1)
        batched_load<NP * TS, 256, V>(zsrc, zdst);
    else
        batched_load<NP * 2 * TS, 256, V>(zsrc, zdst);
    __syncthreads();
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const bool want_e = energy_partials != nullptr;
    if (R == 1)
        z_tile_pairs<T, N, C, 1, G_ONLY>(buf, tw, e1, sp, p0, ky, want_e, acc);
    else
        z_tile_pairs<T, N, C, 2, G_ONLY>(buf, tw, e1, sp, p0, ky, want_e, acc);
    if (want_e) {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double sum = 0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) sum += red[threadIdx.x][w];
            energy_partials[5 * ((size_t)by * gridDim.x + bx) + threadIdx.x] = sum;
        }
    }
    // buffer b = (d NP + q) R + r: field 0 (G) or 2 (G_z) of pair q, row r
    const int nbuf = (G_ONLY ? 1 : 2) * NP * R * TS;
    for (int i = threadIdx.x; i < nbuf; i += blockDim.x) {
        const int b = i / TS, rem = i % TS;
        const int d = b / (NP * R), q = (b / R) % NP, r = b % R;
        const int z = rem / C, c = rem % C;
        H[(3 * q + 2 * d) * M + z * NN + (size_t)ky[r] * N + p0 + c] = buf[i];
    }
}

}  // namespace tild
