// Bead stages of the TILD step: one CTA per 8x8x8-cell tile of beads.
//
//   gather  F_i = -sum_g W(r_i - g) grad w_K(g)   (same weights as the
//           assignment, caption of Fig. pmm; Eq. PMM)
//   bonds   F_i -= (3/b^2) sum_{j bonded to i} mic(r_i - r_j)   (Eq. bonds)
//   GJF     Gronbech-Jensen-Farago update in carried-velocity form
//   spread  rho_K(g) += W(r_i - g)/dV at the new positions (Eq. rhohat),
//           accumulated as 64-bit fixed point: first in a shared-memory
//           patch covering the tile (integer shared atomics), then flushed
//           with 64-bit global atomic adds. Integer sums make the grid
//           bit-identical for any order of beads or blocks.
//
// Carried velocity: the state between steps is r^n and
//   u^n = a v^{n-1} + (dt/2m) a F^{n-1} + (b/m) beta^n,
// so that v^n = u^n + (dt/2m) F^n once F^n is known, and one pass gives
//   r^{n+1} = r^n + b dt (v^n + (dt/2m) F^n + beta^{n+1}/(2m)),
//   u^{n+1} = a (v^n + (dt/2m) F^n) + (b/m) beta^{n+1},
// which is the GJF update with a = (1 - alpha dt/2m)/(1 + alpha dt/2m),
// b = 1/(1 + alpha dt/2m), beta ~ N(0, 2 alpha kT dt).
//
// The other integrators of Sec. "Integrator Class":
//   EM (overdamped Langevin, Euler-Maruyama): r^{n+1} = r^n + (dt/alpha) F^n
//       + sqrt(2 kT dt/alpha) xi^{n+1}; no velocity (u = 0).
//   VV (velocity-Verlet with the Langevin thermostat force): u^n = v^{n-1/2},
//       F^n = F_c^n - alpha u^n + sqrt(2 alpha kT/dt) xi^n, v^n = u^n + (dt/2m) F^n,
//       u^{n+1} = v^{n+1/2} = u^n + (dt/m) F^n, r^{n+1} = r^n + dt u^{n+1}.
//
// Bead arrays are SoA in "slot" order: beads binned by tile every few steps
// (within a tile: interior beads first, each group in bank-group rounds; see
// bin_count_fine). Slot -> bead id and species in `id`; bonded neighbours by
// slot in `nbr` (and `ext` for beads with more than two bonds). All results
// are independent of the slot order.
//
// Species: up to four. The kernels carry them in pairs (species 2p and
// 2p+1 as the real and imaginary parts of one complex field), so the density
// has NS = 2 or 4 species slots and the gradient fields NS/2 pairs.
#pragma once

#include "common.cuh"

namespace tild {

enum BeadMode : int { kModeSpread = 0, kModeForce = 1, kModeSetVel = 2, kModeStep = 3 };
// Integrators of Sec. "Integrator Class" (values as TILD_SCHEME_* in tild.h).
enum Scheme : int { kSchemeGJF = 0, kSchemeEM = 1, kSchemeVV = 2 };

template <typename T> struct BeadParams {
    int n_beads;
    int n;            // grid points per edge (power of two)
    int tiles;        // tiles per edge
    T L, inv_L, inv_dx;
    T k_bond;         // 3 / b^2
    // Integrator (scheme-specific constants, see integrator_constants):
    //   step   h = su u + sf F + sg xi,  r' = r + sd h + se xi,  u' = sh h + sk xi
    //          with xi the normals of counter (n+1) - noise_lag;
    //   report v^n = vu u + vf F + vg xi^n;  set u from v^n: u = wu v + wf F + wg xi^n.
    T su, sf, sg, sd, se, sh, sk;
    T vu, vf, vg, wu, wf, wg;
    int noise_lag;
    T sigma_v;        // sqrt(kT / m) (initial velocities)
    T mass;
    uint64_t seed;
    Topology topo;
};

template <typename T> struct BeadBuffers {
    const T* __restrict__ px;
    const T* __restrict__ py;
    const T* __restrict__ pz;
    T* __restrict__ qx;  // new positions (STEP)
    T* __restrict__ qy;
    T* __restrict__ qz;
    T* __restrict__ ux;  // carried velocity (read/write in place)
    T* __restrict__ uy;
    T* __restrict__ uz;
    const int* __restrict__ id;
    const int2* __restrict__ nbr;
    const int* __restrict__ ext;  // neighbour lists of beads with more than two bonds (see for_each_extra_bond)
    const int* __restrict__ tile_start;  // [tiles^3 + 1] first slot of each tile
    const cplx_t<T>* __restrict__ grad;  // [NS/2][4][M]: per species pair (d_x, d_y, d_z, potentials)
    unsigned long long* __restrict__ rho_fx;  // [NS][M]
    const unsigned long long* step;  // device step counter: n+1 while step n -> n+1 runs
    unsigned int* err;
    T* __restrict__ f_out;        // FORCE: [n_beads][3] by id (may be null)
    T* __restrict__ v_out;        // FORCE: velocities by id (may be null)
    const T* __restrict__ v_in;   // SETVEL: velocities by id (null: Maxwell-Boltzmann)
    double* __restrict__ partials;  // FORCE: [blocks][5]
};

template <typename T> __device__ __forceinline__ T wrap_coord(T x, T L, T inv_L) {
    const T y = x - L * floor(x * inv_L);
    // rounding can give exactly L (mapped to 0) or a tiny negative value
    // (kept); anything else out of range, i.e. a non-finite or huge input,
    // maps to 0 so that no grid index derived from it leaves the grid
    return (y >= L || !(y >= T(-0.5) * L)) ? T(0) : y;
}

template <typename T> __device__ __forceinline__ T min_image(T d, T L, T inv_L) { return d - L * rint(d * inv_L); }

// Bead slots carry the bead id in bits 0..28 and the species in bits 29..31.
constexpr int kSpeciesShift = 29;
__host__ __device__ __forceinline__ int slot_bead_id(int v) { return v & 0x1fffffff; }
__host__ __device__ __forceinline__ int slot_species(int v) { return (int)((unsigned)v >> kSpeciesShift); }

// Bonded neighbours of a slot: nbr = (first, second), -1 for none. A bead
// with more than two bonds has nbr.y = -2 - off and its neighbours after the
// first in ext[off + 1 .. off + ext[off]] (slots, rewritten at every
// re-binning; see bin_neighbours_explicit).
template <class F> __device__ __forceinline__ void for_each_extra_bond(int2 nb, const int* __restrict__ ext, F&& f) {
    if (nb.y < -1) {
        const int off = -2 - nb.y;
        const int cnt = ext[off];
        for (int j = 1; j <= cnt; ++j) f(ext[off + j]);
    }
}

// Shared-memory patch of one tile: grid points [org, org + W) per dimension
// with W = 8 cells + stencil reach (+ an optional drift margin of kMargin
// cells). Beads are re-binned every few steps and move a small fraction of
// a cell per step, so nearly every bead's stencil lies inside its tile's
// patch; the others take the global-memory path.
constexpr int kMargin = 0;
template <int P> struct Patch {
    static constexpr int W = kTile + stencil_extent<P>::hi - stencil_extent<P>::lo + 2 * kMargin;
    static constexpr int W3 = W * W * W;
    static constexpr int lo = stencil_extent<P>::lo - kMargin;  // org = tile origin + lo
};

template <int P, typename T> struct Stencil {
    T wx[P], wy[P], wz[P];
    int jx, jy, jz;
    __device__ __forceinline__ void set(T x, T y, T z, T inv_dx) {
        dh_weights<P>(x * inv_dx, jx, wx);
        dh_weights<P>(y * inv_dx, jy, wy);
        dh_weights<P>(z * inv_dx, jz, wz);
    }
};

template <typename T> struct vec4_of;
template <> struct vec4_of<float> { using type = float4; };
template <> struct vec4_of<double> { using type = double4_16a; };

// -grad w_K interpolated at a bead, from the staged patch (in_patch: one
// (gx, gy, gz) record per point and species) or from global memory.
template <int P, typename T>
__device__ __forceinline__ void gather_force(const Stencil<P, T>& st, bool in_patch, int3 l,
                                             const typename vec4_of<T>::type* s_grad,
                                             const cplx_t<T>* __restrict__ grad, int n, int species, T& fx, T& fy,
                                             T& fz) {
    // grad: the gradient fields of species pair species/2 (global path)
    using PT = Patch<P>;
    T gx = 0, gy = 0, gz = 0;
    if (in_patch) {
        const typename vec4_of<T>::type* sg = s_grad + species * PT::W3;
#pragma unroll
        for (int c = 0; c < P; ++c)
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T wyz = st.wy[b] * st.wz[c];
                const int row = ((l.z + c) * PT::W + (l.y + b)) * PT::W + l.x;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const T w = st.wx[a] * wyz;
                    const typename vec4_of<T>::type g = sg[row + a];
                    gx += w * g.x;
                    gy += w * g.y;
                    gz += w * g.z;
                }
            }
    } else {
        const size_t M = (size_t)n * n * n;
        const int comp = species & 1;
        grad += (size_t)(species >> 1) * 4 * M;
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const size_t oz = (size_t)pwrap(st.jz + c, n) * n * n;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const size_t oy = oz + (size_t)pwrap(st.jy + b, n) * n;
                const T wyz = st.wy[b] * st.wz[c];
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const size_t g = oy + pwrap(st.jx + a, n);
                    const T w = st.wx[a] * wyz;
                    const cplx_t<T> vx = __ldg(grad + g);
                    const cplx_t<T> vy = __ldg(grad + M + g);
                    const cplx_t<T> vz = __ldg(grad + 2 * M + g);
                    gx += w * (comp ? vx.y : vx.x);
                    gy += w * (comp ? vy.y : vy.x);
                    gz += w * (comp ? vz.y : vz.x);
                }
            }
        }
    }
    fx = -gx;
    fy = -gy;
    fz = -gz;
}

// Analytic-differentiation force: F_i = -sum_g grad_r W(r_i - g) w_K(g),
// the exact gradient of the gridded energy. The potentials come from the
// staged patch (in_patch: one value per point and species) or from the
// global field pot = i (w_2p + i w_2p+1) of the species pair p = species/2
// (pot points at pair 0; pairs are 4 n^3 values apart). dw*: d/ds of the
// weights (s = x/dx).
template <int P, typename T>
__device__ __forceinline__ void gather_force_an(const Stencil<P, T>& st, const T (&dwx)[P], const T (&dwy)[P],
                                                const T (&dwz)[P], bool in_patch, int3 l, const T* s_pot,
                                                const cplx_t<T>* __restrict__ pot, int n, int species, T inv_dx,
                                                T& fx, T& fy, T& fz) {
    using PT = Patch<P>;
    T gx = 0, gy = 0, gz = 0;
    if (in_patch) {
        const T* sp = s_pot + species * PT::W3;
#pragma unroll
        for (int c = 0; c < P; ++c)
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T wyz = st.wy[b] * st.wz[c], dyz = dwy[b] * st.wz[c], ydz = st.wy[b] * dwz[c];
                const int row = ((l.z + c) * PT::W + (l.y + b)) * PT::W + l.x;
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const T w = sp[row + a];
                    gx += dwx[a] * wyz * w;
                    gy += st.wx[a] * dyz * w;
                    gz += st.wx[a] * ydz * w;
                }
            }
    } else {
        const int comp = species & 1;
        pot += (size_t)(species >> 1) * 4 * ((size_t)n * n * n);
#pragma unroll
        for (int c = 0; c < P; ++c) {
            const size_t oz = (size_t)pwrap(st.jz + c, n) * n * n;
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const size_t oy = oz + (size_t)pwrap(st.jy + b, n) * n;
                const T wyz = st.wy[b] * st.wz[c], dyz = dwy[b] * st.wz[c], ydz = st.wy[b] * dwz[c];
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const cplx_t<T> v = __ldg(pot + oy + pwrap(st.jx + a, n));
                    const T w = comp ? -v.x : v.y;
                    gx += dwx[a] * wyz * w;
                    gy += st.wx[a] * dyz * w;
                    gz += st.wx[a] * ydz * w;
                }
            }
        }
    }
    fx = -gx * inv_dx;
    fy = -gy * inv_dx;
    fz = -gz * inv_dx;
}

// Spread one bead of species K into the fixed-point patch (in_patch) or
// straight into the global grid.
template <int P, typename T>
__device__ __forceinline__ void spread_bead(const Stencil<P, T>& st, bool in_patch, int3 l,
                                            typename FixedPoint<T>::patch_t* patch,
                                            unsigned long long* __restrict__ rho_fx, int n, int K,
                                            unsigned int* err = nullptr) {
    using PT = Patch<P>;
    using FP = FixedPoint<T>;
    if (in_patch) {
        typename FP::patch_t* base = patch + K * PT::W3;
#pragma unroll
        for (int c = 0; c < P; ++c)
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T wyz = st.wy[b] * st.wz[c];
                const int row = ((l.z + c) * PT::W + (l.y + b)) * PT::W + l.x;
#pragma unroll
                for (int a = 0; a < P; ++a) atomicAdd(base + row + a, FP::to_patch(st.wx[a] * wyz));
            }
    } else {
        const size_t M = (size_t)n * n * n;
#pragma unroll
        for (int c = 0; c < P; ++c)
#pragma unroll
            for (int b = 0; b < P; ++b) {
                const T wyz = st.wy[b] * st.wz[c];
#pragma unroll
                for (int a = 0; a < P; ++a) {
                    const size_t g = ((size_t)pwrap(st.jz + c, n) * n + pwrap(st.jy + b, n)) * n + pwrap(st.jx + a, n);
                    if (debug_check(g < M, err)) atomicAdd(rho_fx + K * M + g, FP::to_grid(st.wx[a] * wyz));
                }
            }
    }
}

template <int P, typename T> __device__ __forceinline__ bool patch_local(const Stencil<P, T>& st, int3 org, int3& l) {
    using PT = Patch<P>;
    l = make_int3(st.jx - org.x, st.jy - org.y, st.jz - org.z);
    return (unsigned)l.x <= (unsigned)(PT::W - P) && (unsigned)l.y <= (unsigned)(PT::W - P) &&
           (unsigned)l.z <= (unsigned)(PT::W - P);
}

// Beads of a tile are staged in shared memory in chunks of up to kBeadChunk.
constexpr int kBeadChunk = 512;

template <int P, typename T, bool AN = false, int NS = 2> struct BeadSmem {
    using patch_t = typename FixedPoint<T>::patch_t;
    static constexpr int W3 = Patch<P>::W3;
    // the force patch is staged when it is small (else gathered from global
    // memory): [NS species][W3] of (gx, gy, gz, -) records, or with the
    // analytic force [NS species][W3] potentials
    static constexpr size_t field_bytes = AN ? NS * W3 * sizeof(T) : NS * W3 * sizeof(typename vec4_of<T>::type);
    static constexpr bool stage_grad = field_bytes <= 48 * 1024;
    static constexpr int patches = NS;
    static constexpr size_t patch_off = 0;                                                       // patch_t [patches][W3]
    static constexpr size_t grad_off = (patch_off + patches * W3 * sizeof(patch_t) + 31) / 32 * 32;
    static constexpr size_t pos_off = grad_off + (stage_grad ? (field_bytes + 15) / 16 * 16 : 0);
    static constexpr size_t nbr_off = pos_off + 3 * kBeadChunk * sizeof(T);                       // int2 [chunk]
    static constexpr size_t tag_off = nbr_off + kBeadChunk * sizeof(int2);                        // int [chunk]
    static constexpr size_t bytes = tag_off + kBeadChunk * sizeof(int);
};

template <int P, typename T, bool AN = false, int NS = 2> constexpr size_t bead_smem_bytes() {
    return BeadSmem<P, T, AN, NS>::bytes;
}

template <int P, int MODE, typename T, bool AN = false, int NS = 2>
__device__ __forceinline__ void bead_kernel_body(const BeadParams<T>& p, const BeadBuffers<T>& bf, int t) {
    using PT = Patch<P>;
    using SM = BeadSmem<P, T, AN, NS>;
    using FP = FixedPoint<T>;
    using patch_t = typename FP::patch_t;
    using V = cplx_t<T>;
    constexpr int W = PT::W;
    constexpr bool kSpread = (MODE == kModeSpread || MODE == kModeStep);
    constexpr bool kForce = (MODE != kModeSpread);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    patch_t* patch = reinterpret_cast<patch_t*>(smem_raw + SM::patch_off);
    using V4 = typename vec4_of<T>::type;
    V4* s_grad = reinterpret_cast<V4*>(smem_raw + SM::grad_off);
    T* s_pot = reinterpret_cast<T*>(smem_raw + SM::grad_off);  // analytic force: [2][W3] potentials
    T* s_pos = reinterpret_cast<T*>(smem_raw + SM::pos_off);
    int2* s_nbr = reinterpret_cast<int2*>(smem_raw + SM::nbr_off);
    int* s_tag = reinterpret_cast<int*>(smem_raw + SM::tag_off);

    const int tx = t % p.tiles, ty = (t / p.tiles) % p.tiles, tz = t / (p.tiles * p.tiles);
    const int3 org = {tx * kTile + PT::lo, ty * kTile + PT::lo, tz * kTile + PT::lo};
    const size_t M = (size_t)p.n * p.n * p.n;
    // patch rows of W points: RPW rows per warp, lane -> (row offset, x)
    constexpr int RPW = 32 / W;
    const int lane = threadIdx.x & 31;
    const int rsub = lane / W, lx = lane - rsub * W;
    const bool row_lane = rsub < RPW;
    const int row0 = (threadIdx.x >> 5) * RPW + rsub;
    const int rstride = (blockDim.x >> 5) * RPW;
    const int gx = pwrap(org.x + lx, p.n);
    // grid offset of the first point of every patch row (lz, ly), computed
    // once per CTA for the staging and the flush (n^3 < 2^31)
    __shared__ int s_rowbase[W * W];
    for (int i = threadIdx.x; i < W * W; i += blockDim.x) {
        const int lz = i / W, ly = i - lz * W;
        s_rowbase[i] = (pwrap(org.z + lz, p.n) * p.n + pwrap(org.y + ly, p.n)) * p.n;
    }
    if (kSpread) {
        for (int i = threadIdx.x; i < SM::patches * PT::W3; i += blockDim.x) patch[i] = 0;
    }
    __syncthreads();
    if (AN && kForce && row_lane) {
        // stage w_2p, w_2p+1 of the patch from pot = i (w_2p + i w_2p+1)
        // (field 3 of pair p)
        constexpr int NWARP = 8;
        constexpr int ROWS_PER_LANE = (W * W + NWARP * RPW - 1) / (NWARP * RPW);
#pragma unroll
        for (int pr = 0; pr < NS / 2; ++pr) {
            V v[ROWS_PER_LANE];
#pragma unroll
            for (int k = 0; k < ROWS_PER_LANE; ++k) {
                const int row = row0 + k * rstride;
                if (row < W * W) {
                    v[k] = __ldg(bf.grad + (4 * pr + 3) * M + s_rowbase[row] + gx);
                }
            }
#pragma unroll
            for (int k = 0; k < ROWS_PER_LANE; ++k) {
                const int row = row0 + k * rstride;
                if (row < W * W) {
                    s_pot[2 * pr * PT::W3 + row * W + lx] = v[k].y;
                    s_pot[(2 * pr + 1) * PT::W3 + row * W + lx] = -v[k].x;
                }
            }
        }
    }
    if (!AN && kForce && SM::stage_grad && row_lane) {
        // stage the gradient fields of the patch as per-species (gx, gy, gz);
        // every row's loads are issued before any is used
        constexpr int NWARP = 8;  // 256 threads
        constexpr int ROWS_PER_LANE = (W * W + NWARP * RPW - 1) / (NWARP * RPW);
#pragma unroll
        for (int pr = 0; pr < NS / 2; ++pr) {
            const V* gp = bf.grad + (size_t)pr * 4 * M;
            V v[ROWS_PER_LANE][3];
#pragma unroll
            for (int k = 0; k < ROWS_PER_LANE; ++k) {
                const int row = row0 + k * rstride;
                if (row < W * W) {
                    const size_t g = (size_t)s_rowbase[row] + gx;
                    v[k][0] = __ldg(gp + g);
                    v[k][1] = __ldg(gp + M + g);
                    v[k][2] = __ldg(gp + 2 * M + g);
                }
            }
#pragma unroll
            for (int k = 0; k < ROWS_PER_LANE; ++k) {
                const int row = row0 + k * rstride;
                if (row < W * W) {
                    s_grad[2 * pr * PT::W3 + row * W + lx] = V4{v[k][0].x, v[k][1].x, v[k][2].x, T(0)};
                    s_grad[(2 * pr + 1) * PT::W3 + row * W + lx] = V4{v[k][0].y, v[k][1].y, v[k][2].y, T(0)};
                }
            }
        }
    }
    const int start = bf.tile_start[t];
    const int end = bf.tile_start[t + 1];
    // noise counter n+1 of this step (advanced by the first kernel of the step)
    const uint64_t step_next = (MODE == kModeStep) ? *bf.step : 0ull;
    // 32-bit patch sums cannot overflow below this many beads per tile
    const bool patch_ok = end - start <= FP::max_tile_beads;
    double acc[5] = {0, 0, 0, 0, 0};

    for (int c0 = start; c0 < end; c0 += kBeadChunk) {
        const int cnt = min(kBeadChunk, end - c0);
        if (c0 != start) __syncthreads();  // the previous chunk is done with the staged beads
        {
            // all loads of the chunk in flight before the shared stores
            constexpr int PER = kBeadChunk / 256;
            T vx[PER], vy[PER], vz[PER];
            int vt[PER];
            int2 vn[PER];
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int j = threadIdx.x + k * 256;
                if (j < cnt) {
                    vx[k] = bf.px[c0 + j];
                    vy[k] = bf.py[c0 + j];
                    vz[k] = bf.pz[c0 + j];
                    vt[k] = bf.id[c0 + j];
                    if (kForce) vn[k] = bf.nbr[c0 + j];
                }
            }
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int j = threadIdx.x + k * 256;
                if (j < cnt) {
                    s_pos[j] = vx[k];
                    s_pos[kBeadChunk + j] = vy[k];
                    s_pos[2 * kBeadChunk + j] = vz[k];
                    s_tag[j] = vt[k];
                    if (kForce) s_nbr[j] = vn[k];
                }
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
            const int i = c0 + j;
            T x = s_pos[j], y = s_pos[kBeadChunk + j], z = s_pos[2 * kBeadChunk + j];
            const int tag = s_tag[j];
            const int bid = slot_bead_id(tag);
            const int species = slot_species(tag);
            Stencil<P, T> st;
            st.set(x, y, z, p.inv_dx);
            int3 l;
            bool inside = patch_local(st, org, l);
            if (kForce) {
                T ux = 0, uy = 0, uz = 0;
                const bool staged = SM::stage_grad && inside;
                if (MODE != kModeSetVel) {
                    ux = bf.ux[i];
                    uy = bf.uy[i];
                    uz = bf.uz[i];
                }
                // bonded neighbours: from the staged chunk when they are in it
                const int2 nb = s_nbr[j];
                T nx[2], ny[2], nz[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int s = k == 0 ? nb.x : nb.y;
                    if (s >= c0 && s < c0 + cnt) {
                        nx[k] = s_pos[s - c0];
                        ny[k] = s_pos[kBeadChunk + s - c0];
                        nz[k] = s_pos[2 * kBeadChunk + s - c0];
                    } else if (s >= 0 && debug_check(s < p.n_beads, bf.err)) {
                        nx[k] = bf.px[s];
                        ny[k] = bf.py[s];
                        nz[k] = bf.pz[s];
                    } else {
                        nx[k] = ny[k] = nz[k] = T(0);
                    }
                }
                T fx, fy, fz;
                if (AN) {
                    T dwx[P], dwy[P], dwz[P];
                    dh_weight_derivs<P>(x * p.inv_dx, dwx);
                    dh_weight_derivs<P>(y * p.inv_dx, dwy);
                    dh_weight_derivs<P>(z * p.inv_dx, dwz);
                    gather_force_an<P>(st, dwx, dwy, dwz, inside, l, s_pot, bf.grad + 3 * M, p.n, species, p.inv_dx, fx,
                                       fy, fz);
                } else {
                    gather_force<P>(st, staged, l, s_grad, bf.grad, p.n, species, fx, fy, fz);
                }
                // the bond energy counts each bond once, at its end with the smaller bead id
                auto nid_of = [&](int s) { return slot_bead_id(s >= c0 && s < c0 + cnt ? s_tag[s - c0] : bf.id[s]); };
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int s = k == 0 ? nb.x : nb.y;
                    if (s >= 0) {
                        const T dx = min_image(x - nx[k], p.L, p.inv_L);
                        const T dy = min_image(y - ny[k], p.L, p.inv_L);
                        const T dz = min_image(z - nz[k], p.L, p.inv_L);
                        fx -= p.k_bond * dx;
                        fy -= p.k_bond * dy;
                        fz -= p.k_bond * dz;
                        if (MODE == kModeForce && nid_of(s) > bid)
                            acc[0] += 0.5 * (double)p.k_bond * ((double)dx * dx + (double)dy * dy + (double)dz * dz);
                    }
                }
                for_each_extra_bond(nb, bf.ext, [&](int s) {
                    if (!debug_check(s >= 0 && s < p.n_beads, bf.err)) return;
                    const T dx = min_image(x - bf.px[s], p.L, p.inv_L);
                    const T dy = min_image(y - bf.py[s], p.L, p.inv_L);
                    const T dz = min_image(z - bf.pz[s], p.L, p.inv_L);
                    fx -= p.k_bond * dx;
                    fy -= p.k_bond * dy;
                    fz -= p.k_bond * dz;
                    if (MODE == kModeForce && nid_of(s) > bid)
                        acc[0] += 0.5 * (double)p.k_bond * ((double)dx * dx + (double)dy * dy + (double)dz * dz);
                });
                if (!(isfinite(fx) && isfinite(fy) && isfinite(fz))) atomicOr(bf.err, kErrNonFinite);
                if (MODE == kModeForce) {
                    // v^n = vu u + vf F + vg xi^n (the integrator's total force enters)
                    normal3<T> g = {T(0), T(0), T(0)};
                    if (p.vg != T(0)) g = gaussian3((uint32_t)bid, *bf.step, p.seed, T(0));
                    const T vx = p.vu * ux + p.vf * fx + p.vg * g.a;
                    const T vy = p.vu * uy + p.vf * fy + p.vg * g.b;
                    const T vz = p.vu * uz + p.vf * fz + p.vg * g.c;
                    acc[1] += 0.5 * (double)p.mass * ((double)vx * vx + (double)vy * vy + (double)vz * vz);
                    acc[2] += fx;
                    acc[3] += fy;
                    acc[4] += fz;
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
                    bf.uz[i] = p.wu * vz + p.wf * fz + p.wg * g.c;
                } else if (MODE == kModeStep) {
                    const normal3<T> g = gaussian3((uint32_t)bid, step_next - (uint64_t)p.noise_lag, p.seed, T(0));
                    const T hx = p.su * ux + p.sf * fx + p.sg * g.a;
                    const T hy = p.su * uy + p.sf * fy + p.sg * g.b;
                    const T hz = p.su * uz + p.sf * fz + p.sg * g.c;
                    x = wrap_coord(x + p.sd * hx + p.se * g.a, p.L, p.inv_L);
                    y = wrap_coord(y + p.sd * hy + p.se * g.b, p.L, p.inv_L);
                    z = wrap_coord(z + p.sd * hz + p.se * g.c, p.L, p.inv_L);
                    bf.qx[i] = x;
                    bf.qy[i] = y;
                    bf.qz[i] = z;
                    bf.ux[i] = p.sh * hx + p.sk * g.a;
                    bf.uy[i] = p.sh * hy + p.sk * g.b;
                    bf.uz[i] = p.sh * hz + p.sk * g.c;
                    st.set(x, y, z, p.inv_dx);
                    inside = patch_local(st, org, l);
                }
            }
            if (kSpread && debug_check(species < NS, bf.err))
                spread_bead<P>(st, inside && patch_ok, l, patch, bf.rho_fx, p.n, species, bf.err);
        }
    }

    if (kSpread) {
        __syncthreads();
        if (row_lane) {
#pragma unroll 1
            for (int K = 0; K < SM::patches; ++K) {
                unsigned long long* rk = bf.rho_fx + K * M + gx;
                for (int row = row0; row < W * W; row += rstride) {
                    const unsigned long long v = patch[(K * W * W + row) * W + lx];
                    if (v != 0ull) atomicAdd(rk + s_rowbase[row], v);
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
            for (int w = 0; w < (int)blockDim.x / 32; ++w) s += red[threadIdx.x][w];
            bf.partials[5 * (size_t)t + threadIdx.x] = s;
        }
    }
}

template <int P, int MODE, typename T, bool AN = false, int NS = 2>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && P <= 3 && NS == 2) ? 4 : 2)
    bead_kernel(BeadParams<T> p, BeadBuffers<T> bf) {
    bead_kernel_body<P, MODE, T, AN, NS>(p, bf, blockIdx.x);
}

// Batched form: blocks [r * tiles^3, (r + 1) * tiles^3) serve replica r.
template <typename T> struct BeadArgs {
    BeadParams<T> p;
    BeadBuffers<T> bf;
};
template <int P, int MODE, typename T>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && P <= 3) ? 4 : 2)
    bead_kernel_batched(const BeadArgs<T>* __restrict__ args, int tiles3) {
    const int r = blockIdx.x / tiles3;
    bead_kernel_body<P, MODE, T>(args[r].p, args[r].bf, blockIdx.x - r * tiles3);
}

// Exact gradient of the gridded energy with respect to the bead positions:
//   dU/dr_i = sum_g grad_r W(r_i - g) w_K(g) + (3/b^2) sum_j mic(r_i - r_j),
// i.e. the adjoint of the spread (the same weights, differentiated) applied
// to the potential field w_K, plus the bond term. `pot` holds
// i (w_A + i w_B) per grid point. Output by bead id.
template <int P, typename T>
__global__ void __launch_bounds__(256) adjoint_kernel(BeadParams<T> p, BeadBuffers<T> bf, const cplx_t<T>* __restrict__ pot,
                                                      T* __restrict__ grad_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n_beads) return;
    const T x = bf.px[i], y = bf.py[i], z = bf.pz[i];
    const int tag = bf.id[i];
    const int bid = slot_bead_id(tag);
    const int species = slot_species(tag);
    Stencil<P, T> st;
    st.set(x, y, z, p.inv_dx);
    T dx[P], dy[P], dz[P];
    dh_weight_derivs<P>(x * p.inv_dx, dx);
    dh_weight_derivs<P>(y * p.inv_dx, dy);
    dh_weight_derivs<P>(z * p.inv_dx, dz);
    T gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
        for (int b = 0; b < P; ++b)
#pragma unroll
            for (int a = 0; a < P; ++a) {
                const size_t g = ((size_t)pwrap(st.jz + c, p.n) * p.n + pwrap(st.jy + b, p.n)) * p.n + pwrap(st.jx + a, p.n);
                const cplx_t<T> v = pot[(size_t)(species >> 1) * 4 * ((size_t)p.n * p.n * p.n) + g];
                const T w = (species & 1) ? -v.x : v.y;  // w_2p = Im, w_2p+1 = -Re of i (w_2p + i w_2p+1)
                gx += dx[a] * st.wy[b] * st.wz[c] * w;
                gy += st.wx[a] * dy[b] * st.wz[c] * w;
                gz += st.wx[a] * st.wy[b] * dz[c] * w;
            }
    gx *= p.inv_dx;
    gy *= p.inv_dx;
    gz *= p.inv_dx;
    const int2 nb = bf.nbr[i];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int s = k == 0 ? nb.x : nb.y;
        if (s >= 0) {
            gx += p.k_bond * min_image(x - bf.px[s], p.L, p.inv_L);
            gy += p.k_bond * min_image(y - bf.py[s], p.L, p.inv_L);
            gz += p.k_bond * min_image(z - bf.pz[s], p.L, p.inv_L);
        }
    }
    for_each_extra_bond(nb, bf.ext, [&](int s) {
        gx += p.k_bond * min_image(x - bf.px[s], p.L, p.inv_L);
        gy += p.k_bond * min_image(y - bf.py[s], p.L, p.inv_L);
        gz += p.k_bond * min_image(z - bf.pz[s], p.L, p.inv_L);
    });
    grad_out[3 * (size_t)bid + 0] = gx;
    grad_out[3 * (size_t)bid + 1] = gy;
    grad_out[3 * (size_t)bid + 2] = gz;
}

// ------------------------------------------------------------- binning

// Tile of a position: index of the 8x8x8-cell tile holding floor(r/dx).
template <typename T> __device__ __forceinline__ int tile_key(T x, T y, T z, T inv_dx, int n, int tiles) {
    const int cx = min(max((int)floor(x * inv_dx), 0), n - 1);
    const int cy = min(max((int)floor(y * inv_dx), 0), n - 1);
    const int cz = min(max((int)floor(z * inv_dx), 0), n - 1);
    return ((cz / kTile) * tiles + cy / kTile) * tiles + cx / kTile;
}

// atomicAdd(counter + key, 1) for every active lane with one atomic per
// distinct key in the warp; returns this lane's value before its increment.
__device__ __forceinline__ int warp_aggregated_inc(int* counter, int key) {
    const unsigned active = __activemask();
    const unsigned peers = __match_any_sync(active, key);
    const int leader = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    const int rank = __popc(peers & ((1u << lane) - 1));
    int base = 0;
    if (lane == leader) base = atomicAdd(counter + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + rank;
}

// Re-binning in one counting sort over fine bins: 16 per tile, (edge class,
// bank group). Class 0 holds beads more than half a cell from every tile
// face, class 1 the others: those drift out of the tile's patch before the
// next re-binning and take the global-memory paths, so they go last and
// share as few warps as possible. The bank group is the 16-byte bank group
// of the bead's first gather record in the staged patch, (l + K W^3) mod 8
// with l the patch record of its cell and K its species. Within a class the
// slots go round by round: round r takes the r-th bead of every group that
// has one, in group order, so that consecutive beads (the eight lanes of a
// shared-memory access phase) read records in distinct bank groups.
constexpr int kFineBins = 16;

template <typename T>
__global__ void bin_count_fine(int n_beads, const T* __restrict__ px, const T* __restrict__ py,
                               const T* __restrict__ pz, T inv_dx, int n, int nz, int tiles, int patch_w, int patch_lo,
                               Topology topo, const unsigned char* __restrict__ species_of_id,
                               const int* __restrict__ id_src, int* __restrict__ fkey, int* __restrict__ frank,
                               int* __restrict__ fcount) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const T x = px[i], y = py[i], z = pz[i];
    const int cx = min(max((int)floor(x * inv_dx), 0), n - 1);
    const int cy = min(max((int)floor(y * inv_dx), 0), n - 1);
    const int cz = min(max((int)floor(z * inv_dx), 0), nz - 1);
    const int tx = cx / kTile, ty = cy / kTile, tz = cz / kTile;
    const int tile = (tz * tiles + ty) * tiles + tx;
    const T lx = x * inv_dx - (T)(tx * kTile), ly = y * inv_dx - (T)(ty * kTile), lz = z * inv_dx - (T)(tz * kTile);
    const T dmin = min(min(min(lx, T(kTile) - lx), min(ly, T(kTile) - ly)), min(lz, T(kTile) - lz));
    const int edge = dmin < T(0.5) ? 1 : 0;
    const int b = slot_bead_id(id_src[i]);
    const int K = species_of_id ? (int)species_of_id[b] : bead_info(topo, b).species;
    const int rec = ((cz - tz * kTile - patch_lo) * patch_w + (cy - ty * kTile - patch_lo)) * patch_w +
                    (cx - tx * kTile - patch_lo);
    const int grp = (rec + K * patch_w * patch_w * patch_w) & 7;
    const int f = tile * kFineBins + edge * 8 + grp;
    fkey[i] = f;
    frank[i] = warp_aggregated_inc(fcount, f);
}

// tile_start[t] = fine_start[16 t] for t = 0 .. tiles^3 (the last: n_beads)
static __global__ void bin_tile_start(const int* __restrict__ fine_start, int n_tiles, int* __restrict__ tile_start) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= n_tiles) tile_start[t] = fine_start[(size_t)t * kFineBins];
}

// Move every bead (positions, carried velocities, id with species bits) to
// its slot: the start of its (tile, class) block, plus the beads of earlier
// rounds, plus those of its round in lower groups.
template <typename T>
__global__ void bin_scatter_fine(int n_beads, Topology topo, const unsigned char* __restrict__ species_of_id,
                                 const int* __restrict__ fkey, const int* __restrict__ frank,
                                 const int* __restrict__ fcount, const int* __restrict__ fine_start,
                                 const T* __restrict__ pos_src /*[3][N]*/, T* __restrict__ pos_dst,
                                 const T* __restrict__ u_src /*[3][N]*/, T* __restrict__ u_dst,
                                 const int* __restrict__ id_src, int* __restrict__ id_dst, int* __restrict__ slot_of_id) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const int f = fkey[i], r = frank[i];
    const int base = f & ~7, g = f & 7;
    int s = fine_start[base];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int c = fcount[base + q];
        s += min(c, r) + ((q < g && c > r) ? 1 : 0);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pos_dst[(size_t)c * n_beads + s] = pos_src[(size_t)c * n_beads + i];
        u_dst[(size_t)c * n_beads + s] = u_src[(size_t)c * n_beads + i];
    }
    const int b = slot_bead_id(id_src[i]);
    const int K = species_of_id ? (int)species_of_id[b] : bead_info(topo, b).species;
    id_dst[s] = b | (K << kSpeciesShift);
    slot_of_id[b] = s;
}

static __global__ void bin_neighbours(int n_beads, Topology topo, const int* __restrict__ id, const int* __restrict__ slot_of_id,
                               int2* __restrict__ nbr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const BeadInfo b = bead_info(topo, slot_bead_id(id[i]));
    nbr[i] = make_int2(b.prev >= 0 ? slot_of_id[b.prev] : -1, b.next >= 0 ? slot_of_id[b.next] : -1);
}

// Neighbour slots from an explicit bond list: adj[b] holds the first two
// neighbour ids of bead b in increasing order (-1: none), or for a bead with
// more than two bonds the first neighbour and -2 - off, with the count and
// the remaining ids in ext_ids[off], ext_ids[off + 1 ..]. ext_slots (same
// layout) receives the slots of those ids.
static __global__ void bin_neighbours_explicit(int n_beads, const int* __restrict__ id, const int* __restrict__ slot_of_id,
                                               const int2* __restrict__ adj, const int* __restrict__ ext_ids,
                                               int* __restrict__ ext_slots, int2* __restrict__ nbr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const int2 a = adj[slot_bead_id(id[i])];
    int2 r = make_int2(a.x >= 0 ? slot_of_id[a.x] : -1, a.y >= 0 ? slot_of_id[a.y] : -1);
    if (a.y < -1) {
        const int off = -2 - a.y;
        const int cnt = ext_ids[off];
        ext_slots[off] = cnt;
        for (int j = 1; j <= cnt; ++j) ext_slots[off + j] = slot_of_id[ext_ids[off + j]];
        r.y = a.y;
    }
    nbr[i] = r;
}

// Exclusive scan of `count` ints in blocks of 1024 (three kernels).
static __global__ void scan_blocks(const int* __restrict__ in, int* __restrict__ out, int* __restrict__ block_sums, int count) {
    __shared__ int s[1024];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int v = i < count ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < count) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) block_sums[blockIdx.x] = s[1023];
}

static __global__ void scan_top(int* __restrict__ block_sums, int nblocks) {
    // single CTA of 1024 threads; sequential over chunks of 1024
    __shared__ int s[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nblocks ? block_sums[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblocks) block_sums[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += s[1023];
        __syncthreads();
    }
}

static __global__ void scan_add(int* __restrict__ out, const int* __restrict__ block_sums, int count) {
    const int i = blockIdx.x * 1024 + threadIdx.x;
    if (i < count) out[i] += block_sums[blockIdx.x];
}

// -------------------------------------------------------------- I/O

// In: AoS [n][3] by bead id (type TI). Out: SoA slot order = id order.
template <typename T, typename TI>
__global__ void load_positions(int n_beads, const TI* __restrict__ in, T L, T inv_L, T* __restrict__ pos /*[3][N]*/,
                               int* __restrict__ id, unsigned int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const T x = (T)in[3 * (size_t)i + d];
        if (!isfinite(x)) atomicOr(err, kErrNonFinite);
        pos[(size_t)d * n_beads + i] = wrap_coord(x, L, inv_L);
    }
    id[i] = i;
}

// SoA slot order -> AoS by id (type TO).
template <typename T, typename TO>
__global__ void store_by_id(int n_beads, const T* __restrict__ src /*[3][N]*/, const int* __restrict__ id,
                            TO* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const int b = slot_bead_id(id[i]);
#pragma unroll
    for (int d = 0; d < 3; ++d) out[3 * (size_t)b + d] = (TO)src[(size_t)d * n_beads + i];
}

// AoS by id (type TI) -> SoA slot order.
template <typename T, typename TI>
__global__ void load_by_id(int n_beads, const TI* __restrict__ in, const int* __restrict__ id, T* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_beads) return;
    const int b = slot_bead_id(id[i]);
#pragma unroll
    for (int d = 0; d < 3; ++d) dst[(size_t)d * n_beads + i] = (T)in[3 * (size_t)b + d];
}

// [n][3] <-> [3][n] (to_aos: from SoA to AoS).
template <typename TV>
__global__ void transpose_vec3(size_t n, const TV* __restrict__ in, TV* __restrict__ out, bool to_aos) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    // i indexes the output
    if (to_aos)
        out[i] = in[(i % 3) * n + i / 3];
    else
        out[i] = in[3 * (i % n) + i / n];
}

template <typename TO>
__global__ void density_out(size_t count, const unsigned long long* __restrict__ rho_fx, double scale, TO* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (TO)((double)(long long)rho_fx[i] * scale);
}

template <typename TI, typename TO>
__global__ void convert_copy(size_t count, const TI* __restrict__ in, TO* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = (TO)in[i];
}

}  // namespace tild
