// Grid and bead kernels for any grid size and for two-dimensional boxes
// (Sec. "TILD Branch": periodic boxes in two or three dimensions; Listing
// infile runs D = 2 on a 65 x 65 grid). The same method as the tiled path,
// organised for generality rather than speed:
//   - beads: one thread per bead (no tiles or shared patches); the density
//     is accumulated with 64-bit fixed-point global atomics, so it is as
//     bit-reproducible as the tiled path's;
//   - FFT: one kernel per axis on tiles of lines held in shared memory, each
//     line transformed in two factors n = n1 n2 (Cooley-Tukey) with direct
//     DFTs of lengths n1 and n2 and one twiddle table of length n, so odd
//     sizes (65 = 5 x 13, 45, 75, primes) need no special radix;
//   - spectral multiply: one thread per wavevector over the whole spectrum.
// Grids are [..][nz][n][n] with nz = n (D = 3) or 1 (D = 2); spectra are
// complex, species pairs packed as in the tiled path (rho_2p + i rho_2p+1).
#pragma once

#include "bead_kernels.cuh"
#include "grid_kernels.cuh"

namespace tild {

// ---------------------------------------------------------------- FFT

// Twiddle W_n^m for any m >= 0 (the table holds exp(-2 pi i m/n), m < n).
template <int DIR, class V> __device__ __forceinline__ V gtw(const V* tw, int m) {
    const V w = tw[m];
    return DIR < 0 ? w : c_conj(w);
}

// Transform the lines of one tile along `axis` (0 = x, 1 = y, 2 = z) of
// `fields` complex arrays [F][nz][n][n]. A CTA takes C lines that are
// adjacent in x (axis y or z) or adjacent rows (axis x) and keeps them in
// shared memory as buf[line][j] (pitch n + 1), with a second buffer for the
// intermediate of the two-factor transform:
//   t[j2 + n2 k1] = W_n^{j2 k1} sum_j1 x[j2 + n2 j1] W_n^{n2 j1 k1},
//   X[k1 + n1 k2] = sum_j2 t[j2 + n2 k1] W_n^{n1 j2 k2}.
// grid.x = tiles of lines per field, grid.y = field.
template <typename T, int DIR>
__global__ void __launch_bounds__(256) generic_axis_fft(cplx_t<T>* __restrict__ data, int n, int nz, int axis, int C,
                                                        int n1, int n2, const cplx_t<T>* __restrict__ tw_g) {
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tw = reinterpret_cast<V*>(smem_raw);
    const int pitch = n + 1;
    V* buf = tw + n;
    V* tmp = buf + (size_t)C * pitch;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = tw_g[i];
    const size_t M = (size_t)nz * n * n;
    V* f = data + (size_t)blockIdx.y * M;
    // line l of this tile: start offset and element stride
    const size_t stride = axis == 0 ? 1 : axis == 1 ? (size_t)n : (size_t)n * n;
    const int lines_per_field = (int)(M / n);
    const int l0 = blockIdx.x * C;
    auto line_start = [&](int l) -> size_t {
        // lines are numbered so that consecutive numbers are adjacent in x
        // (axes y, z) or consecutive rows (axis x)
        if (axis == 0) return (size_t)l * n;
        if (axis == 1) {
            const int x = l % n, z = l / n;
            return (size_t)z * n * n + x;
        }
        return (size_t)l;  // axis 2: l = y n + x
    };
    const int nl = min(C, lines_per_field - l0);
    for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
        // consecutive threads: consecutive lines (axes y, z) or consecutive elements (axis x)
        int l, j;
        if (axis == 0) {
            l = i / n;
            j = i % n;
        } else {
            l = i % nl;
            j = i / nl;
        }
        buf[l * pitch + j] = f[line_start(l0 + l) + (size_t)j * stride];
    }
    __syncthreads();
    // stage A
    for (int u = threadIdx.x; u < nl * n; u += blockDim.x) {
        const int l = u % nl, r = u / nl;
        const int k1 = r % n1, j2 = r / n1;
        const V* x = buf + l * pitch;
        V acc = {T(0), T(0)};
        int m = 0;
        const int step = (n2 * k1) % n;
        for (int j1 = 0; j1 < n1; ++j1) {
            acc = c_add(acc, c_mul(x[j2 + n2 * j1], gtw<DIR>(tw, m)));
            m += step;
            if (m >= n) m -= n;
        }
        tmp[l * pitch + j2 + n2 * k1] = c_mul(acc, gtw<DIR>(tw, (j2 * k1) % n));
    }
    __syncthreads();
    // stage B
    for (int u = threadIdx.x; u < nl * n; u += blockDim.x) {
        const int l = u % nl, r = u / nl;
        const int k1 = r % n1, k2 = r / n1;
        const V* t = tmp + l * pitch;
        V acc = {T(0), T(0)};
        int m = 0;
        const int step = (n1 * k2) % n;
        for (int j2 = 0; j2 < n2; ++j2) {
            acc = c_add(acc, c_mul(t[j2 + n2 * k1], gtw<DIR>(tw, m)));
            m += step;
            if (m >= n) m -= n;
        }
        buf[l * pitch + k1 + n1 * k2] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nl * n; i += blockDim.x) {
        int l, j;
        if (axis == 0) {
            l = i / n;
            j = i % n;
        } else {
            l = i % nl;
            j = i / nl;
        }
        f[line_start(l0 + l) + (size_t)j * stride] = buf[l * pitch + j];
    }
}

// Fixed-point densities [2 NP][M] -> complex pairs Z_p = rho_2p + i rho_2p+1
// ([NP][M]); zero the fixed-point grid when asked. A step's first kernel
// advances the noise counter.
template <typename T>
__global__ void generic_load_density(size_t M, int np, unsigned long long* __restrict__ rho_fx, cplx_t<T>* __restrict__ Z,
                                     T scale, int zero_after, unsigned long long* step_ctr) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (step_ctr && i == 0) *step_ctr += 1ull;
    if (i >= (size_t)np * M) return;
    const size_t p = i / M, g = i % M;
    unsigned long long* a = rho_fx + 2 * p * M + g;
    unsigned long long* b = a + M;
    const long long va = (long long)*a, vb = (long long)*b;
    if (zero_after) {
        *a = 0ull;
        *b = 0ull;
    }
    Z[i] = cplx_t<T>{from_fixed(va, scale), from_fixed(vb, scale)};
}

// Spectral multiply over the whole spectrum, one thread per wavevector k:
// species spectra from the packed pairs (Hermitian separation with Z(-k)),
// w~_K = u_hat(k) sum_K' eps_KK' rho~_K', and per pair
//   out[p][d] = i k~_d Q_p (d < D; k~ with the Nyquist index zeroed),
//   out[p][3] = i Q_p (the potentials), Q_p = w~_2p + i w~_2p+1.
// Energy partials per block as in the z pass: [0] sum u_hat Re[conj(rho~_0)
// rho~_1] (one pair) or the chi-weighted sum over species pairs (two
// pairs), [1] sum_{k != 0} u_hat |sum_K rho~_K|^2, [2], [3] the same times
// |k|^2, [4] 0. u_hat = e1[kx] e1[ky] (e1[kz]).
template <typename T, int NP>
__global__ void __launch_bounds__(256) generic_spectral(const cplx_t<T>* __restrict__ Z, cplx_t<T>* __restrict__ out,
                                                        int n, int nz, SpectralParams<T> sp,
                                                        double* __restrict__ partials) {
    using V = cplx_t<T>;
    const size_t M = (size_t)nz * n * n;
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double acc[5] = {0, 0, 0, 0, 0};
    if (g < M) {
        const int x = (int)(g % n), y = (int)((g / n) % n), z = (int)(g / ((size_t)n * n));
        const int mx = x == 0 ? 0 : n - x, my = y == 0 ? 0 : n - y, mz = z == 0 ? 0 : nz - z;
        const size_t gm = ((size_t)mz * n + my) * n + mx;
        auto freq = [&](int i, int len) { return (T)(2 * i < len ? i : i - len); };  // 2 i == len: -len/2
        auto kgrad = [&](int i, int len) { return (len % 2 == 0 && 2 * i == len) ? T(0) : sp.two_pi_over_L * freq(i, len); };
        const T qx = sp.two_pi_over_L * freq(x, n), qy = sp.two_pi_over_L * freq(y, n);
        const T qz = nz > 1 ? sp.two_pi_over_L * freq(z, nz) : T(0);
        const T kd[3] = {kgrad(x, n), kgrad(y, n), nz > 1 ? kgrad(z, nz) : T(0)};
        const T uh = sp.kernel1d[x] * sp.kernel1d[y] * (nz > 1 ? sp.kernel1d[z] : T(1));
        V A[2 * NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const V Zk = Z[p * M + g], Zm = Z[p * M + gm];
            A[2 * p] = {T(0.5) * (Zk.x + Zm.x), T(0.5) * (Zk.y - Zm.y)};
            A[2 * p + 1] = {T(0.5) * (Zk.y + Zm.y), -T(0.5) * (Zk.x - Zm.x)};
        }
        if (partials) {
            const double k2 = (double)qx * qx + (double)qy * qy + (double)qz * qz;
            double fchi;
            if (NP == 1) {
                fchi = (double)uh * ((double)A[0].x * A[1].x + (double)A[0].y * A[1].y);
            } else {
                fchi = 0.0;
#pragma unroll
                for (int K = 0; K < 2 * NP; ++K)
#pragma unroll
                    for (int K2 = K + 1; K2 < 2 * NP; ++K2)
                        fchi += (double)sp.chi4[K][K2] * ((double)A[K].x * A[K2].x + (double)A[K].y * A[K2].y);
                fchi *= (double)uh;
            }
            acc[0] = fchi;
            acc[2] = k2 * fchi;
            if (g != 0) {
                double tr = 0, ti = 0;
#pragma unroll
                for (int K = 0; K < 2 * NP; ++K) {
                    tr += A[K].x;
                    ti += A[K].y;
                }
                acc[1] = (double)uh * (tr * tr + ti * ti);
                acc[3] = k2 * acc[1];
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            V w[2];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int K = 2 * p + s;
                T wr = 0, wi = 0;
                if (NP == 1) {
                    const T e0 = s == 0 ? sp.eAA : sp.eAB, e1v = s == 0 ? sp.eAB : sp.eBB;
                    wr = e0 * A[0].x + e1v * A[1].x;
                    wi = e0 * A[0].y + e1v * A[1].y;
                } else {
#pragma unroll
                    for (int K2 = 0; K2 < 2 * NP; ++K2) {
                        wr += sp.eps4[K][K2] * A[K2].x;
                        wi += sp.eps4[K][K2] * A[K2].y;
                    }
                }
                w[s] = {uh * wr, uh * wi};
            }
            const V iQ = {-(w[0].y + w[1].x), w[0].x - w[1].y};
            V* o = out + (size_t)4 * p * M;
            o[g] = {kd[0] * iQ.x, kd[0] * iQ.y};
            o[M + g] = {kd[1] * iQ.x, kd[1] * iQ.y};
            if (nz > 1) o[2 * M + g] = {kd[2] * iQ.x, kd[2] * iQ.y};
            o[3 * M + g] = iQ;
        }
    }
    if (partials) {
        __shared__ double red[5][8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double s = 0;
            for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
            partials[5 * (size_t)blockIdx.x + threadIdx.x] = s;
        }
    }
}

// ---------------------------------------------------------------- beads

// One thread per bead slot: the bead modes of the tiled kernel (spread,
// force and observables, set velocity, step) with D = 2 or 3 and any n.
// grad: [NS/2][4][M] (d_x, d_y, d_z, potentials) per species pair.
template <int P, int MODE, typename T, int D>
__global__ void __launch_bounds__(256) generic_bead_kernel(BeadParams<T> p, BeadBuffers<T> bf, int nz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < p.n_beads;
    double acc[5] = {0, 0, 0, 0, 0};
    if (active) {
        const int n = p.n;
        const size_t M = (size_t)nz * n * n;
        T x = bf.px[i], y = bf.py[i], z = D == 3 ? bf.pz[i] : T(0);
        const int tag = bf.id[i];
        const int bid = slot_bead_id(tag), species = slot_species(tag);
        Stencil<P, T> st;
        st.set(x, y, z, p.inv_dx);
        constexpr int PZ = D == 3 ? P : 1;
        if (MODE != kModeSpread) {
            // field force: -sum_g W(r - g) grad w_K(g)
            const cplx_t<T>* gp = bf.grad + (size_t)(species >> 1) * 4 * M;
            const int comp = species & 1;
            T gx = 0, gy = 0, gz = 0;
#pragma unroll
            for (int c = 0; c < PZ; ++c) {
                const size_t oz = D == 3 ? (size_t)pwrap(st.jz + c, n) * n * n : 0;
                const T wz = D == 3 ? st.wz[c] : T(1);
#pragma unroll
                for (int b = 0; b < P; ++b) {
                    const size_t oy = oz + (size_t)pwrap(st.jy + b, n) * n;
                    const T wyz = st.wy[b] * wz;
#pragma unroll
                    for (int a = 0; a < P; ++a) {
                        const size_t g = oy + pwrap(st.jx + a, n);
                        const T w = st.wx[a] * wyz;
                        const cplx_t<T> vx = __ldg(gp + g), vy = __ldg(gp + M + g);
                        gx += w * (comp ? vx.y : vx.x);
                        gy += w * (comp ? vy.y : vy.x);
                        if (D == 3) {
                            const cplx_t<T> vz = __ldg(gp + 2 * M + g);
                            gz += w * (comp ? vz.y : vz.x);
                        }
                    }
                }
            }
            T fx = -gx, fy = -gy, fz = -gz;
            const int2 nb = bf.nbr[i];
            auto bond = [&](int s) {
                const T dx = min_image(x - bf.px[s], p.L, p.inv_L);
                const T dy = min_image(y - bf.py[s], p.L, p.inv_L);
                const T dz = D == 3 ? min_image(z - bf.pz[s], p.L, p.inv_L) : T(0);
                fx -= p.k_bond * dx;
                fy -= p.k_bond * dy;
                fz -= p.k_bond * dz;
                if (MODE == kModeForce && slot_bead_id(bf.id[s]) > bid)
                    acc[0] += 0.5 * (double)p.k_bond * ((double)dx * dx + (double)dy * dy + (double)dz * dz);
            };
            if (nb.x >= 0) bond(nb.x);
            if (nb.y >= 0) bond(nb.y);
            for_each_extra_bond(nb, bf.ext, bond);
            if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(bf.err, kErrNonFinite);
            T ux = 0, uy = 0, uz = 0;
            if (MODE != kModeSetVel) {
                ux = bf.ux[i];
                uy = bf.uy[i];
                uz = D == 3 ? bf.uz[i] : T(0);
            }
            if (MODE == kModeForce) {
                normal3<T> g = {T(0), T(0), T(0)};
                if (p.vg != T(0)) g = gaussian3((uint32_t)bid, *bf.step, p.seed, T(0));
                const T vx = p.vu * ux + p.vf * fx + p.vg * g.a;
                const T vy = p.vu * uy + p.vf * fy + p.vg * g.b;
                const T vz = D == 3 ? p.vu * uz + p.vf * fz + p.vg * g.c : T(0);
                acc[1] = 0.5 * (double)p.mass * ((double)vx * vx + (double)vy * vy + (double)vz * vz);
                acc[2] = fx;
                acc[3] = fy;
                acc[4] = fz;
                if (bf.f_out) {
                    bf.f_out[3 * (size_t)bid + 0] = fx;
                    bf.f_out[3 * (size_t)bid + 1] = fy;
                    bf.f_out[3 * (size_t)bid + 2] = fz;
                }
                if (bf.v_out) {
                    bf.v_out[3 * (size_t)bid + 0] = vx;
                    bf.v_out[3 * (size_t)bid + 1] = vy;
                    bf.v_out[3 * (size_t)bid + 2] = vz;
                }
            } else if (MODE == kModeSetVel) {
                T vx, vy, vz;
                if (bf.v_in) {
                    vx = bf.v_in[3 * (size_t)bid + 0];
                    vy = bf.v_in[3 * (size_t)bid + 1];
                    vz = bf.v_in[3 * (size_t)bid + 2];
                } else {
                    const normal3<T> g = gaussian3((uint32_t)bid, ~0ull, p.seed, T(0));
                    vx = p.sigma_v * g.a;
                    vy = p.sigma_v * g.b;
                    vz = p.sigma_v * g.c;
                }
                normal3<T> g = {T(0), T(0), T(0)};
                if (p.wg != T(0)) g = gaussian3((uint32_t)bid, *bf.step, p.seed, T(0));
                bf.ux[i] = p.wu * vx + p.wf * fx + p.wg * g.a;
                bf.uy[i] = p.wu * vy + p.wf * fy + p.wg * g.b;
                bf.uz[i] = D == 3 ? p.wu * vz + p.wf * fz + p.wg * g.c : T(0);
            } else {  // step
                const normal3<T> g = gaussian3((uint32_t)bid, *bf.step - (uint64_t)p.noise_lag, p.seed, T(0));
                const T hx = p.su * ux + p.sf * fx + p.sg * g.a;
                const T hy = p.su * uy + p.sf * fy + p.sg * g.b;
                const T hz = p.su * uz + p.sf * fz + p.sg * g.c;
                x = wrap_coord(x + p.sd * hx + p.se * g.a, p.L, p.inv_L);
                y = wrap_coord(y + p.sd * hy + p.se * g.b, p.L, p.inv_L);
                z = D == 3 ? wrap_coord(z + p.sd * hz + p.se * g.c, p.L, p.inv_L) : T(0);
                bf.qx[i] = x;
                bf.qy[i] = y;
                bf.qz[i] = z;
                bf.ux[i] = p.sh * hx + p.sk * g.a;
                bf.uy[i] = p.sh * hy + p.sk * g.b;
                bf.uz[i] = D == 3 ? p.sh * hz + p.sk * g.c : T(0);
                st.set(x, y, z, p.inv_dx);
            }
        }
        if (MODE == kModeSpread || MODE == kModeStep) {
            using FP = FixedPoint<T>;
            unsigned long long* rk = bf.rho_fx + (size_t)species * M;
#pragma unroll
            for (int c = 0; c < PZ; ++c) {
                const size_t oz = D == 3 ? (size_t)pwrap(st.jz + c, n) * n * n : 0;
                const T wz = D == 3 ? st.wz[c] : T(1);
#pragma unroll
                for (int b = 0; b < P; ++b) {
                    const size_t oy = oz + (size_t)pwrap(st.jy + b, n) * n;
                    const T wyz = st.wy[b] * wz;
#pragma unroll
                    for (int a = 0; a < P; ++a) atomicAdd(rk + oy + pwrap(st.jx + a, n), FP::to_grid(st.wx[a] * wyz));
                }
            }
        }
    }
    if (MODE == kModeForce) {
        __shared__ double red[5][8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double v = acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[k][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < 5) {
            double s = 0;
            for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
            bf.partials[5 * (size_t)blockIdx.x + threadIdx.x] = s;
        }
    }
}

}  // namespace tild
