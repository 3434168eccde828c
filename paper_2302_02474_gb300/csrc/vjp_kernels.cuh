// Differentiable form: the vector-Jacobian product of the ik particle-mesh +
// bond force (Eq. PMM with the gradient taken by i k differentiation; Eq.
// bonds), J^T lam = d/dr of sum_i lam_i . F_i, and the derivatives of
// sum_i lam_i . F_i with respect to chi, kappa and a.
//
// With W_i(g) = W(r_i - g), mu_K(g) = sum_{i in K} W_i(g) lam_i, C the
// convolution with the smeared kernel (u_hat, plus the Coulomb term with
// charges), D the i k~ derivative (anti-self-adjoint) and
// psi_K = sum_K' eps_KK' C (D . mu_K'):
//   (J^T lam)_j = sum_g grad W_j(g) [psi_{K_j}(g) / dV - (lam_j . D w_{K_j})(g)]
//                 - (3/b^2) sum_{i ~ j} (lam_j - lam_i).
// The pipeline: spread mu in fixed point (three grids of int64 pairs:
// component d of mu_A and of mu_B), xy transforms into three complex grids
// (mu_A in the real, mu_B in the imaginary part), a z pass
// that forms D . mu per species, psi and the parameter sums, the inverse
// transforms of psi (the potential slot of the gradient buffer), and a
// per-bead gather with the derivatives of the assignment weights.
#pragma once

#include "bead_kernels.cuh"
#include "grid_kernels.cuh"

namespace tild {

// The spread of lam is accumulated in 64-bit fixed point, so that J^T lam is
// independent of the order of the atomic adds (bitwise reproducible, as the
// forward density is). Each grid sum is bounded by n_beads * max|lam| since
// every assignment weight is at most 1; the scale is the power of two s with
// max|lam| * s < 2^S and S = min(S_max, 62 - ceil(log2 n_beads)), so no sum
// can overflow. S_max is 40 for FP32 (below the FP32 rounding of w * lam)
// and 52 for FP64. A non-finite lam makes the scale 0 and the inverse scale
// NaN: every output is then NaN.
template <typename T> struct AdjointFixed;
template <> struct AdjointFixed<float> {
    using bits_t = unsigned int;
    static constexpr int s_max = 40;
    static __device__ __forceinline__ bits_t abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }
    static __device__ __forceinline__ void scales(bits_t b, int S, float& s, float& inv) {
        const int E = (int)(b >> 23);
        if (E >= 255) {
            s = 0.f;
            inv = __int_as_float(0x7fc00000);
            return;
        }
        const int e = E == 0 ? -127 : E - 127;  // max|lam| < 2^(e+1)
        const int k = min(S - e - 1, 120);
        s = __int_as_float((k + 127) << 23);
        inv = __int_as_float((127 - k) << 23);
    }
    static __device__ __forceinline__ long long to_fixed(float x) { return __float2ll_rn(x); }
};
template <> struct AdjointFixed<double> {
    using bits_t = unsigned long long;
    static constexpr int s_max = 52;
    static __device__ __forceinline__ bits_t abs_bits(double x) {
        return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    }
    static __device__ __forceinline__ void scales(bits_t b, int S, double& s, double& inv) {
        const int E = (int)(b >> 52);
        if (E >= 2047) {
            s = 0.0;
            inv = __longlong_as_double(0x7ff8000000000000ll);
            return;
        }
        const int e = E == 0 ? -1023 : E - 1023;
        const int k = min(S - e - 1, 1000);
        s = __longlong_as_double((long long)(k + 1023) << 52);
        inv = __longlong_as_double((long long)(1023 - k) << 52);
    }
    static __device__ __forceinline__ long long to_fixed(double x) { return __double2ll_rn(x); }
};

// *bits = max over the n values of lam of the bit pattern of |lam| (for
// non-negative IEEE values the order of the bit patterns is the order of the
// values, NaN above infinity); *bits must be 0 on entry.
// (256 threads per block.)
template <typename T>
__global__ void __launch_bounds__(256) lam_absmax(size_t n, const T* __restrict__ lam,
                                                  typename AdjointFixed<T>::bits_t* bits) {
    using B = typename AdjointFixed<T>::bits_t;
    B m = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += 8 * stride) {
        B v[8];  // eight independent loads in flight
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = i0 + k * stride < n ? AdjointFixed<T>::abs_bits(lam[i0 + k * stride]) : B(0);
#pragma unroll
        for (int k = 0; k < 8; ++k) m = max(m, v[k]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = max(m, (B)__shfl_xor_sync(0xffffffffu, m, o));
    __shared__ B s_m[8];
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 1; w < 8; ++w) m = max(m, s_m[w]);
        if (m) atomicMax(bits, m);
    }
}

// mu_d += W_i lam_{i,d} in fixed point; lam by bead id ([N][3]); fx as
// int64 pairs [3][M][2] (species A, B), zero on entry.
template <int P, typename T>
__global__ void __launch_bounds__(256) vjp_spread(BeadParams<T> p, BeadBuffers<T> bf, const T* __restrict__ lam,
                                                  unsigned long long* __restrict__ fx,
                                                  const typename AdjointFixed<T>::bits_t* __restrict__ bits, int S) {
    using FX = AdjointFixed<T>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_beads) return;
    T sc, inv;
    FX::scales(*bits, S, sc, inv);
    const int tag = bf.id[i];
    const int bid = slot_bead_id(tag), K = slot_species(tag);
    const T l0 = lam[3 * (size_t)bid] * sc, l1 = lam[3 * (size_t)bid + 1] * sc, l2 = lam[3 * (size_t)bid + 2] * sc;
    Stencil<P, T> st;
    st.set(bf.px[i], bf.py[i], bf.pz[i], p.inv_dx);
    const int n = p.n;
    const size_t M = (size_t)n * n * n;
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const T wyz = st.wy[b] * st.wz[c];
            const size_t row = ((size_t)pwrap(st.jz + c, n) * n + pwrap(st.jy + b, n)) * n;
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const size_t g = row + pwrap(st.jx + a, n);
                const T w = st.wx[a] * wyz;
                atomicAdd(fx + 2 * g + K, (unsigned long long)FX::to_fixed(w * l0));
                atomicAdd(fx + 2 * (M + g) + K, (unsigned long long)FX::to_fixed(w * l1));
                atomicAdd(fx + 2 * (2 * M + g) + K, (unsigned long long)FX::to_fixed(w * l2));
            }
        }
}

// Forward DFT along x and y of plane blockIdx.x of field blockIdx.y: reads
// the fixed-point spread fx ([3][M] int64 pairs), converts it with the
// inverse scale, and writes the complex [3][M] array `data` in mirror-paired
// column order.
template <typename T, int N>
__global__ void __launch_bounds__(512) xy_forward_cplx(const longlong2* __restrict__ fx,
                                                       const typename AdjointFixed<T>::bits_t* __restrict__ bits, int S,
                                                       cplx_t<T>* __restrict__ data, const cplx_t<T>* __restrict__ tw_g) {
    using V = cplx_t<T>;
    constexpr int PITCH = row_pitch(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* plane = tw + N;
    load_twiddles(tw, tw_g, N);
    T sc, inv;
    AdjointFixed<T>::scales(*bits, S, sc, inv);
    const size_t base = (size_t)blockIdx.y * N * N * N + (size_t)blockIdx.x * N * N;
    batched_load<N * N, 512, longlong2>([&](int i) { return fx[base + i]; },
                                        [&](int i, longlong2 v) {
                                            plane[(i / N) * PITCH + i % N] = V{from_fixed(v.x, inv), from_fixed(v.y, inv)};
                                        });
    __syncthreads();
    smem_fft_lines<N, -1, N, 512>(plane, StridedLines<PITCH>{}, 1, tw);  // along x
    smem_fft_lines<N, -1, N, 512>(plane, StridedLines<1>{}, PITCH, tw);  // along y
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) data[base + i] = plane[(i / N) * PITCH + kx_of_pos<N>(i % N)];
}

// z pass of the VJP. CTA (C column positions, rows ky and -ky) as in
// z_spectral. Buffers [4R][N][C]: sets 0..2 = the xy-transformed mu_d rows,
// set 3 = the xy-transformed density rows (Zxy). Writes i (psi~_A + i psi~_B)
// transformed back along z into field 0 of H, and per block the sums
//   0: sum_k Re[conj(s_A) u_hat rho~_B + conj(s_B) u_hat rho~_A]
//   1: sum_k Re[(conj(s_A) + conj(s_B)) u_hat (rho~_A + rho~_B)]
//   2: sum_k Re[sum_K conj(s_K) |k|^2 u_hat sum_K' (eps_KK'/M) rho~_K']
// with s_K = (D . mu_K)~.
template <typename T, int N, int C, int R>
__device__ __forceinline__ void z_vjp_tile(cplx_t<T>* buf, const cplx_t<T>* tw, const T* e1, const T* e2,
                                           const SpectralParams<T>& sp, bool el, int p0, const int (&ky)[2],
                                           double (&acc)[3]) {
    using V = cplx_t<T>;
    constexpr int TS = N * C;
    smem_fft_lines<N, -1, 4 * R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
    constexpr int rB = R - 1;
    const int c = threadIdx.x % C;
    const int cB = mirror_pos(p0 + c) - p0;
    const int kxA = kx_of_pos<N>(p0 + c), kxB = kx_of_pos<N>(p0 + cB);
    const T exyA = e1[kxA] * e1[ky[0]], exyB = e1[kxB] * e1[ky[rB]];
    const T exy2A = el ? e2[kxA] * e2[ky[0]] : T(0), exy2B = el ? e2[kxB] * e2[ky[rB]] : T(0);
    const T tp = sp.two_pi_over_L;
    const T qxA = raw_k<T, N>(kxA, tp), qyA = raw_k<T, N>(ky[0], tp);
    const T qxB = raw_k<T, N>(kxB, tp), qyB = raw_k<T, N>(ky[rB], tp);
    const T gxA = grad_k<T, N>(kxA, tp), gyA = grad_k<T, N>(ky[0], tp);
    const T gxB = grad_k<T, N>(kxB, tp), gyB = grad_k<T, N>(ky[rB], tp);
    // per-thread partial sums in T (a few terms each; FP64 arithmetic is slow
    // on this part), added to the FP64 block sums after the loop
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int kz = threadIdx.x / C; kz < N; kz += 256 / C) {
        const int kzB = kz == 0 ? 0 : N - kz;
        if (R == 1 && kzB * C + cB < kz * C + c) continue;  // the mirror element owns this pair
        const bool same = (R == 1) && (kzB == kz) && (cB == c);
        V zA[4], zB[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            zA[d] = buf[(d * R) * TS + kz * C + c];
            zB[d] = buf[(d * R + rB) * TS + kzB * C + cB];
        }
        V out[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (s == 1 && same) break;
            const int kzi = s == 0 ? kz : kzB;
            const T kd[3] = {s == 0 ? gxA : gxB, s == 0 ? gyA : gyB, grad_k<T, N>(kzi, tp)};
            // s_K = sum_d i k~_d mu~_{K,d}, mu~_A = (Z + conj Zm)/2, mu~_B = -i (Z - conj Zm)/2
            V sA = {T(0), T(0)}, sB = {T(0), T(0)};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const V Z = s == 0 ? zA[d] : zB[d];
                const V Zm = s == 0 ? zB[d] : zA[d];
                const V mA = {T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y)};
                const V mB = {T(0.5) * (Z.y + Zm.y), -T(0.5) * (Z.x - Zm.x)};
                sA.x -= kd[d] * mA.y;
                sA.y += kd[d] * mA.x;
                sB.x -= kd[d] * mB.y;
                sB.y += kd[d] * mB.x;
            }
            const V Z = s == 0 ? zA[3] : zB[3];
            const V Zm = s == 0 ? zB[3] : zA[3];
            const V rA = {T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y)};
            const V rBv = {T(0.5) * (Z.y + Zm.y), -T(0.5) * (Z.x - Zm.x)};
            const T uh = (s == 0 ? exyA : exyB) * e1[kzi];
            V pA = {uh * (sp.eAA * sA.x + sp.eAB * sB.x), uh * (sp.eAA * sA.y + sp.eAB * sB.y)};
            V pB = {uh * (sp.eAB * sA.x + sp.eBB * sB.x), uh * (sp.eAB * sA.y + sp.eBB * sB.y)};
            const T qz = raw_k<T, N>(kzi, tp);
            const T k2 = (s == 0 ? qxA * qxA + qyA * qyA : qxB * qxB + qyB * qyB) + qz * qz;
            if (el) {
                const T g = k2 > T(0) ? (s == 0 ? exy2A : exy2B) * e2[kzi] * recip(k2) : T(0);
                const T cq = sp.el_scale * g;
                const V sq = {sp.qA * sA.x + sp.qB * sB.x, sp.qA * sA.y + sp.qB * sB.y};
                pA.x += cq * sp.qA * sq.x;
                pA.y += cq * sp.qA * sq.y;
                pB.x += cq * sp.qB * sq.x;
                pB.y += cq * sp.qB * sq.y;
            }
            out[s] = {-(pA.y + pB.x), pA.x - pB.y};  // i (psi~_A + i psi~_B)
            a0 += uh * ((sA.x * rBv.x + sA.y * rBv.y) + (sB.x * rA.x + sB.y * rA.y));
            a1 += uh * ((sA.x + sB.x) * (rA.x + rBv.x) + (sA.y + sB.y) * (rA.y + rBv.y));
            const T wAr = sp.eAA * rA.x + sp.eAB * rBv.x, wAi = sp.eAA * rA.y + sp.eAB * rBv.y;
            const T wBr = sp.eAB * rA.x + sp.eBB * rBv.x, wBi = sp.eAB * rA.y + sp.eBB * rBv.y;
            a2 += uh * k2 * ((sA.x * wAr + sA.y * wAi) + (sB.x * wBr + sB.y * wBi));
        }
        buf[kz * C + c] = out[0];
        if (!same) buf[rB * TS + kzB * C + cB] = out[1];
    }
    acc[0] += (double)a0;
    acc[1] += (double)a1;
    acc[2] += (double)a2;
    __syncthreads();
    smem_fft_lines<N, +1, R * C, 256>(buf, TileAddr<C, TS>{}, C, tw);
}

template <typename T, int N, int C>
__global__ void __launch_bounds__(256) z_vjp(cplx_t<T>* __restrict__ H, const cplx_t<T>* __restrict__ Zxy,
                                             const cplx_t<T>* __restrict__ tw_g, SpectralParams<T> sp,
                                             double* __restrict__ partials, int el) {
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    V* buf = tw + N;
    constexpr int TS = N * C;
    __shared__ double red[3][8];
    __shared__ T e1[N];
    __shared__ T e2[N];
    load_twiddles(tw, tw_g, N);
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        e1[i] = sp.kernel1d[i];
        if (el) e2[i] = sp.kernel1d_el[i];
    }
    const int p0 = blockIdx.x * C;
    const int ky[2] = {(int)blockIdx.y, blockIdx.y == 0 ? 0 : N - (int)blockIdx.y};
    const int R = (ky[0] == ky[1]) ? 1 : 2;
    const size_t NN = (size_t)N * N, M = NN * N;
    // buffer i = (set, row, z, c): sets 0..2 from H (mu), set 3 from Zxy (rho)
    auto src = [&](int i) {
        const int set = i / (R * TS), rem = i % (R * TS);
        const int r = rem / TS, zc = rem % TS;
        const size_t off = (zc / C) * NN + (size_t)ky[r] * N + p0 + zc % C;
        return set < 3 ? H[set * M + off] : Zxy[off];
    };
    auto dst = [&](int i, V v) { buf[i] = v; };
    if (R == 1)
        batched_load<4 * TS, 256, V>(src, dst);
    else
        batched_load<8 * TS, 256, V>(src, dst);
    __syncthreads();
    double acc[3] = {0.0, 0.0, 0.0};
    if (R == 1)
        z_vjp_tile<T, N, C, 1>(buf, tw, e1, e2, sp, el != 0, p0, ky, acc);
    else
        z_vjp_tile<T, N, C, 2>(buf, tw, e1, e2, sp, el != 0, p0, ky, acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double sum = 0;
        for (int w = 0; w < (int)blockDim.x / 32; ++w) sum += red[threadIdx.x][w];
        partials[3 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x) + threadIdx.x] = sum;
    }
    for (int i = threadIdx.x; i < R * TS; i += blockDim.x) {
        const int r = i / TS, zc = i % TS;
        const int z = zc / C, cc = zc % C;
        H[z * NN + (size_t)ky[r] * N + p0 + cc] = buf[i];
    }
}

// Per bead: sum_g grad W_j(g) [psi_{K_j}(g)/dV - lam_j . D w_{K_j}(g)] and the
// bond term. fields = the gradient buffer: [0..2] (d_x, d_y, d_z)(w_A, w_B),
// [3] i (psi_A + i psi_B). lam and out by bead id ([N][3]).
template <int P, typename T>
__global__ void __launch_bounds__(256) vjp_beads(BeadParams<T> p, BeadBuffers<T> bf, const cplx_t<T>* __restrict__ fields,
                                                 const T* __restrict__ lam, T inv_dV, T* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_beads) return;
    const T x = bf.px[i], y = bf.py[i], z = bf.pz[i];
    const int tag = bf.id[i];
    const int bid = slot_bead_id(tag), K = slot_species(tag);
    const T l0 = lam[3 * (size_t)bid], l1 = lam[3 * (size_t)bid + 1], l2 = lam[3 * (size_t)bid + 2];
    Stencil<P, T> st;
    st.set(x, y, z, p.inv_dx);
    T dwx[P], dwy[P], dwz[P];
    dh_weight_derivs<P>(x * p.inv_dx, dwx);
    dh_weight_derivs<P>(y * p.inv_dx, dwy);
    dh_weight_derivs<P>(z * p.inv_dx, dwz);
    const int n = p.n;
    const size_t M = (size_t)n * n * n;
    T ox = 0, oy = 0, oz = 0;
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const size_t row = ((size_t)pwrap(st.jz + c, n) * n + pwrap(st.jy + b, n)) * n;
            const T wyz = st.wy[b] * st.wz[c], dyz = dwy[b] * st.wz[c], ydz = st.wy[b] * dwz[c];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const size_t g = row + pwrap(st.jx + a, n);
                const cplx_t<T> f0 = fields[g], f1 = fields[M + g], f2 = fields[2 * M + g], f3 = fields[3 * M + g];
                const T ldw = l0 * (K ? f0.y : f0.x) + l1 * (K ? f1.y : f1.x) + l2 * (K ? f2.y : f2.x);
                const T psi = K ? -f3.x : f3.y;
                const T val = psi * inv_dV - ldw;
                ox += dwx[a] * wyz * val;
                oy += st.wx[a] * dyz * val;
                oz += st.wx[a] * ydz * val;
            }
        }
    ox *= p.inv_dx;
    oy *= p.inv_dx;
    oz *= p.inv_dx;
    const int2 nb = bf.nbr[i];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k == 0 ? nb.x : nb.y;
        if (s >= 0) {
            const int nid = slot_bead_id(bf.id[s]);
            ox -= p.k_bond * (l0 - lam[3 * (size_t)nid]);
            oy -= p.k_bond * (l1 - lam[3 * (size_t)nid + 1]);
            oz -= p.k_bond * (l2 - lam[3 * (size_t)nid + 2]);
        }
    }
    for_each_extra_bond(nb, bf.ext, [&](int s) {
        const int nid = slot_bead_id(bf.id[s]);
        ox -= p.k_bond * (l0 - lam[3 * (size_t)nid]);
        oy -= p.k_bond * (l1 - lam[3 * (size_t)nid + 1]);
        oz -= p.k_bond * (l2 - lam[3 * (size_t)nid + 2]);
    });
    out[3 * (size_t)bid] = ox;
    out[3 * (size_t)bid + 1] = oy;
    out[3 * (size_t)bid + 2] = oz;
}

// Vector-Jacobian product of the density assignment (Eq. rhohat with the
// weights differentiated): for per-species grid adjoints psi_K(g) =
// dL/drho_K(g) ([S][M], real), the derivative of sum_{K,g} psi_K(g)
// rho_K(g) with respect to bead i's position,
//   out_i = (1/dV) sum_g grad_r W(r_i - g) psi_{K_i}(g),
// by bead id ([N][3]).
template <int P, typename T>
__global__ void __launch_bounds__(256) density_vjp_kernel(BeadParams<T> p, BeadBuffers<T> bf, const T* __restrict__ psi,
                                                          T inv_dV, T* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_beads) return;
    const T x = bf.px[i], y = bf.py[i], z = bf.pz[i];
    const int tag = bf.id[i];
    const int bid = slot_bead_id(tag), K = slot_species(tag);
    Stencil<P, T> st;
    st.set(x, y, z, p.inv_dx);
    T dwx[P], dwy[P], dwz[P];
    dh_weight_derivs<P>(x * p.inv_dx, dwx);
    dh_weight_derivs<P>(y * p.inv_dx, dwy);
    dh_weight_derivs<P>(z * p.inv_dx, dwz);
    const int n = p.n;
    const T* f = psi + (size_t)K * n * n * n;
    T ox = 0, oy = 0, oz = 0;
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
        for (int b = 0; b < P; ++b) {
            const size_t row = ((size_t)pwrap(st.jz + c, n) * n + pwrap(st.jy + b, n)) * n;
            const T wyz = st.wy[b] * st.wz[c], dyz = dwy[b] * st.wz[c], ydz = st.wy[b] * dwz[c];
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const T v = f[row + pwrap(st.jx + a, n)];
                ox += dwx[a] * wyz * v;
                oy += st.wx[a] * dyz * v;
                oz += st.wx[a] * ydz * v;
            }
        }
    const T s = p.inv_dx * inv_dV;  // d/dr = (1/dx) d/ds
    out[3 * (size_t)bid] = ox * s;
    out[3 * (size_t)bid + 1] = oy * s;
    out[3 * (size_t)bid + 2] = oz * s;
}

// acc[k] += sum_b partials[3 b + k] (k = 0..2), in a fixed order: strided
// sums per thread, then a tree in shared memory. One block of 256 threads.
static __global__ void __launch_bounds__(256) accumulate_partials(const double* __restrict__ partials, int n_blocks,
                                                                  double* __restrict__ acc) {
    __shared__ double s[3][256];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < n_blocks; b += 256) v += partials[3 * b + k];
        s[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 3; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 3) acc[threadIdx.x] += s[threadIdx.x][0];
}

// Reverse sweep through K steps of the update shared by every scheme
// (state: positions r and carried velocity u; F = F(r); xi fixed normals):
//   h = su u + sf F + sg xi,   r' = r + sd h + se xi,   u' = sh h + sk xi,
// with the velocity of a state v = vu u + vf F + vg xi and the initial
// u^0 = wu v^0 + wf F(r^0) + wg xi. Adjoint vectors rb, ub (FP64) belong to
// the state being left; lam is the adjoint of F at the next state reached.
//
// Start (state K): ub = vu vb (vb = dL/dv^K), lam = vf vb, plus wf ub when
// K = 0 (then r^0 also enters through u^0).
template <typename T>
__global__ void adjoint_init(size_t n3, double* __restrict__ ub, T* __restrict__ lam, double vu, double vf, double wf,
                             int at_start) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const double v = ub[i], u = vu * v;
    ub[i] = u;
    lam[i] = (T)(vf * v + (at_start ? wf * u : 0.0));
}

// One step back, from state j+1 to state j, after the force VJP at r^{j+1}
// (jt = J^T lam):  rb += jt;  hb = sd rb + sh ub;  ub = su hb;
// lam = sf hb (+ wf ub when j = 0), the adjoint of F(r^j).
template <typename T>
__global__ void adjoint_step(size_t n3, const T* __restrict__ jt, double* __restrict__ rb, double* __restrict__ ub,
                             T* __restrict__ lam, double sd, double sh, double su, double sf, double wf, int at_start) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n3) return;
    const double r = rb[i] + (double)jt[i];
    const double hb = sd * r + sh * ub[i], u = su * hb;
    rb[i] = r;
    ub[i] = u;
    lam[i] = (T)(sf * hb + (at_start ? wf * u : 0.0));
}

// y = (T)(a x)
template <typename T>
__global__ void scale_copy(size_t n, const double* __restrict__ x, double a, T* __restrict__ y) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (T)(a * x[i]);
}

// the device step counter (noise counters of the following steps)
static __global__ void set_counter(unsigned long long* counter, unsigned long long value) { *counter = value; }

// out = a + b (FP64)
template <typename T>
__global__ void add_into(size_t n, const double* __restrict__ a, const T* __restrict__ b, double* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + (double)b[i];
}

}  // namespace tild
