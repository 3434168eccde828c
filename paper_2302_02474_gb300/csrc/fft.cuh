// Hand-written FFT building blocks for lengths 8..256 that split as
// N = N1 * N2 with N1 in {4, 8, 16} and N2 in {1, 3, 4, 5, 8, 16}
// (powers of two, 24, 40, 48, 80).
//
// A length-N transform is split N = N1 * N2 (four-step / Cooley-Tukey):
//   input index  j = j2 + N2 * j1,  output index k = k1 + N1 * k2,
//   X[k1 + N1 k2] = sum_j2 W_N^{j2 k1} W_N2^{j2 k2} sum_j1 x[j2 + N2 j1] W_N1^{j1 k1}.
// Stage A does the N1-point DFTs over j1 in registers and applies the
// twiddle W_N^{j2 k1}; stage B does the N2-point DFTs over j2 in registers
// and writes the result in natural order. Lines live in shared memory; the
// thread-to-data mapping puts consecutive threads on consecutive lines so
// that every shared-memory access of a warp touches consecutive lines at
// the same offset (conflict-free when the line stride is odd in 8-byte
// words, or 1).
//
// Sign convention: forward (DIR = -1) uses exp(-2 pi i jk/N), inverse
// (DIR = +1) exp(+2 pi i jk/N); neither is normalised.
#pragma once

#include "common.cuh"

namespace tild {

// ------------------------------------------------------------- radices

template <int N> struct fft_split;
template <> struct fft_split<8> { static constexpr int N1 = 8, N2 = 1; };
template <> struct fft_split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct fft_split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct fft_split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct fft_split<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct fft_split<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct fft_split<24> { static constexpr int N1 = 8, N2 = 3; };
template <> struct fft_split<40> { static constexpr int N1 = 8, N2 = 5; };
template <> struct fft_split<48> { static constexpr int N1 = 16, N2 = 3; };
template <> struct fft_split<80> { static constexpr int N1 = 16, N2 = 5; };

// Multiply v by W_16^m = exp(DIR * 2 pi i m / 16); m is a compile-time
// constant after unrolling, so the branches fold away.
template <int DIR, class V> __device__ __forceinline__ V w16_mul(int m, V v) {
    using T = decltype(v.x);
    const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);  // cos, sin(pi/8)
    const T h = T(0.70710678118654752440);                                    // cos(pi/4)
    m &= 15;
    // value of exp(-2 pi i m / 16) = (cr, ci); inverse uses the conjugate
    T cr, ci;
    switch (m) {
        case 0: return v;
        case 4: return DIR < 0 ? c_mul_negi(v) : c_mul_posi(v);
        case 8: return {-v.x, -v.y};
        case 12: return DIR < 0 ? c_mul_posi(v) : c_mul_negi(v);
        case 1: cr = c1; ci = -s1; break;
        case 2: cr = h; ci = -h; break;
        case 3: cr = s1; ci = -c1; break;
        case 5: cr = -s1; ci = -c1; break;
        case 6: cr = -h; ci = -h; break;
        case 7: cr = -c1; ci = -s1; break;
        case 9: cr = -c1; ci = s1; break;
        case 10: cr = -h; ci = h; break;
        case 11: cr = -s1; ci = c1; break;
        case 13: cr = s1; ci = c1; break;
        case 14: cr = h; ci = h; break;
        default: cr = c1; ci = s1; break;  // 15
    }
    if (DIR > 0) ci = -ci;
    return {v.x * cr - v.y * ci, v.x * ci + v.y * cr};
}

// In-register DFT of R points (R = 1, 2, 4, 8, 16 by radix-2 decimation in
// time; 3 and 5 directly), natural order in and out.
template <int R, int DIR, class V> struct reg_dft {
    static __device__ __forceinline__ void run(V (&v)[R]) {
        V e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        reg_dft<R / 2, DIR, V>::run(e);
        reg_dft<R / 2, DIR, V>::run(o);
#pragma unroll
        for (int k = 0; k < R / 2; ++k) {
            const V t = w16_mul<DIR>(k * (16 / R), o[k]);
            v[k] = c_add(e[k], t);
            v[k + R / 2] = c_sub(e[k], t);
        }
    }
};
template <int DIR, class V> struct reg_dft<1, DIR, V> {
    static __device__ __forceinline__ void run(V (&)[1]) {}
};

// 3 points: X1,2 = x0 + cos(2pi/3)(x1 + x2) +/- i DIR' sin(2pi/3)(x1 - x2),
// with the sign of the exponent DIR.
template <int DIR, class V> struct reg_dft<3, DIR, V> {
    static __device__ __forceinline__ void run(V (&v)[3]) {
        using T = decltype(v[0].x);
        const T c = T(-0.5), s = T(DIR) * T(0.86602540378443864676);  // DIR sin(2 pi / 3)
        const V t1 = c_add(v[1], v[2]), t3 = c_sub(v[1], v[2]);
        const V m = {v[0].x + c * t1.x, v[0].y + c * t1.y};
        const V it = {-s * t3.y, s * t3.x};  // i s (x1 - x2)
        v[0] = c_add(v[0], t1);
        v[1] = c_add(m, it);
        v[2] = c_sub(m, it);
    }
};

// 5 points with t1 = x1 + x4, t2 = x2 + x3, t3 = x1 - x4, t4 = x2 - x3:
// X1,4 = x0 + c1 t1 + c2 t2 +/- i (s1 t3 + s2 t4), X2,3 = x0 + c2 t1 + c1 t2
// +/- i (s2 t3 - s1 t4), c_k = cos(2 pi k / 5), s_k = DIR sin(2 pi k / 5).
template <int DIR, class V> struct reg_dft<5, DIR, V> {
    static __device__ __forceinline__ void run(V (&v)[5]) {
        using T = decltype(v[0].x);
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
        const T s1 = T(DIR) * T(0.95105651629515357212), s2 = T(DIR) * T(0.58778525229247312917);
        const V t1 = c_add(v[1], v[4]), t2 = c_add(v[2], v[3]);
        const V t3 = c_sub(v[1], v[4]), t4 = c_sub(v[2], v[3]);
        const V a = {v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
        const V b = {v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
        const V p = {s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
        const V q = {s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
        const V ip = {-p.y, p.x}, iq = {-q.y, q.x};
        v[0] = {v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y};
        v[1] = c_add(a, ip);
        v[4] = c_sub(a, ip);
        v[2] = c_add(b, iq);
        v[3] = c_sub(b, iq);
    }
};

// Twiddle table W_N^m = exp(-2 pi i m / N), m in [0, N), computed on the
// host in FP64 and rounded to T; copied to shared memory by each CTA.
template <int DIR, class V> __device__ __forceinline__ V twiddle(const V* tw, int m) {
    const V w = tw[m];
    return DIR < 0 ? w : c_conj(w);
}

// ----------------------------------------------------- line transforms

// FFT of NLINES lines of length N held in shared memory. Element e of
// line l lives at buf[addr(l) + e * es]. All NTHR threads of the CTA call
// this; it ends with __syncthreads(). Stage B keeps all of its work units
// in registers (UPT per thread), so one round covers every line.
// Stage A of smem_fft_lines alone (ends with __syncthreads()): unit
// (line, j2) transforms x[j2 + N2 j1] over j1 and applies W_N^{j2 k1}.
template <int N, int DIR, int NLINES, int NTHR, class V, class Addr>
__device__ __forceinline__ void smem_fft_stage_a(V* buf, Addr addr, int es, const V* tw) {
    constexpr int N1 = fft_split<N>::N1;
    constexpr int N2 = fft_split<N>::N2;
    // Stage A: unit (line, j2); reads and writes only its own positions.
    for (int u = threadIdx.x; u < NLINES * N2; u += NTHR) {
        const int l = u % NLINES;
        const int j2 = u / NLINES;
        V* p = buf + addr(l) + j2 * es;
        V v[N1];
#pragma unroll
        for (int j1 = 0; j1 < N1; ++j1) v[j1] = p[j1 * N2 * es];
        reg_dft<N1, DIR, V>::run(v);
        if (N2 > 1) {
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = c_mul(v[k1], twiddle<DIR>(tw, j2 * k1));
        }
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) p[k1 * N2 * es] = v[k1];
    }
    __syncthreads();
}

template <int N, int DIR, int NLINES, int NTHR, class V, class Addr>
__device__ __forceinline__ void smem_fft_lines(V* buf, Addr addr, int es, const V* tw) {
    constexpr int N1 = fft_split<N>::N1;
    constexpr int N2 = fft_split<N>::N2;
    constexpr int nthr = NTHR;
    constexpr int UPT = (NLINES * N1 + NTHR - 1) / NTHR;
    const int tid = threadIdx.x;

    smem_fft_stage_a<N, DIR, NLINES, NTHR>(buf, addr, es, tw);
    if (N2 == 1) return;

    // Stage B: unit (line, k1) reads the N2 positions j2 + N2 k1 and writes
    // X[k1 + N1 k2]; positions overlap other units, so every unit of a
    // round is loaded before any is stored.
    {
        constexpr int l0 = 0;
        constexpr int nl = NLINES;
        V v[UPT][N2];
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int u = tid + r * nthr;
            if (u < nl * N1) {
                const int l = l0 + u % nl;
                const int k1 = u / nl;
                const V* p = buf + addr(l) + k1 * N2 * es;
#pragma unroll
                for (int j2 = 0; j2 < N2; ++j2) v[r][j2] = p[j2 * es];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int u = tid + r * nthr;
            if (u < nl * N1) {
                const int l = l0 + u % nl;
                const int k1 = u / nl;
                reg_dft<N2, DIR, V>::run(v[r]);
                V* p = buf + addr(l) + k1 * es;
#pragma unroll
                for (int k2 = 0; k2 < N2; ++k2) p[k2 * N1 * es] = v[r][k2];
            }
        }
        __syncthreads();
    }
}

template <int LS> struct StridedLines {
    __device__ __forceinline__ int operator()(int l) const { return l * LS; }
};

}  // namespace tild

namespace tild {

// smem_fft_lines whose second stage hands each output to out(l, k, X_l[k])
// instead of writing it back to shared memory (the caller's last use of the
// lines, e.g. a store to global memory); no barrier at the end. N2 > 1.
template <int N, int DIR, int NLINES, int NTHR, class V, class Addr, class Out>
__device__ __forceinline__ void smem_fft_lines_out(V* buf, Addr addr, int es, const V* tw, Out out) {
    constexpr int N1 = fft_split<N>::N1;
    constexpr int N2 = fft_split<N>::N2;
    static_assert(N2 > 1, "two-stage lengths only");
    constexpr int UPT = (NLINES * N1 + NTHR - 1) / NTHR;
    smem_fft_stage_a<N, DIR, NLINES, NTHR>(buf, addr, es, tw);
    V v[UPT][N2];
#pragma unroll
    for (int r = 0; r < UPT; ++r) {
        const int u = threadIdx.x + r * NTHR;
        if (u < NLINES * N1) {
            const int l = u % NLINES, k1 = u / NLINES;
            const V* p = buf + addr(l) + k1 * N2 * es;
#pragma unroll
            for (int j2 = 0; j2 < N2; ++j2) v[r][j2] = p[j2 * es];
        }
    }
#pragma unroll
    for (int r = 0; r < UPT; ++r) {
        const int u = threadIdx.x + r * NTHR;
        if (u < NLINES * N1) {
            const int l = u % NLINES, k1 = u / NLINES;
            reg_dft<N2, DIR, V>::run(v[r]);
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) out(l, k1 + N1 * k2, v[r][k2]);
        }
    }
}

}  // namespace tild
