// Host engine of the TILD step: owns device buffers, launches the kernels
// of one step in stream order and replays whole re-binning cycles as CUDA
// graphs. Instantiated once per precision (engine_f32.cu, engine_f64.cu).
#pragma once

#include <algorithm>
#include <unordered_map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bead_kernels.cuh"
#include "vjp_kernels.cuh"
#include "engine_api.h"
#include "grid_kernels.cuh"
#include "generic_kernels.cuh"

namespace tild {

#define TILD_CUDA(call)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            err = std::string(#call) + ": " + cudaGetErrorString(e_);                          \
            return e_ == cudaErrorMemoryAllocation ? TILD_ENOMEM : TILD_EDEVICE;               \
        }                                                                                      \
    } while (0)

constexpr uint64_t kStateMagic = 0x54494c4453544154ull;  // "TILDSTAT"

template <typename T> class BatchEngine;

template <typename T> class Engine final : public EngineBase {
    using V = cplx_t<T>;
    friend class BatchEngine<T>;

   public:
    ~Engine() override { release(); }

    tild_status init(HostConfig* cfg) override {
        cfg_ = cfg;
        n_ = cfg->n;
        generic_ = cfg->generic;
        nz_ = cfg->dim == 2 ? 1 : n_;
        M_ = (size_t)nz_ * n_ * n_;
        tiles_ = (n_ + kTile - 1) / kTile;
        P_ = cfg->pmeorder + 1;
        plane_fits_ = plane_smem() <= 200 * 1024;
        C_ = std::min(n_, (int)(128 / sizeof(V)));  // y-column tiles of the split passes
        CZ_ = zpass_cols(n_);                          // column tiles of the z pass
        TILD_CUDA(cudaGetDevice(&device_));
        TILD_CUDA(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking));
        stream_ = own_stream_;
        tild_status gst = alloc_grids(1);
        if (gst) return gst;
        TILD_CUDA(dev_malloc((void**)&tw_, n_ * sizeof(V)));
        TILD_CUDA(dev_malloc((void**)&kernel1d_, 2 * n_ * sizeof(T)));  // exp(-a^2 k_m^2), then exp(-a_e^2 k_m^2)
        TILD_CUDA(dev_malloc((void**)&counters_, 4 * sizeof(unsigned long long)));
        TILD_CUDA(cudaMemset(counters_, 0, 4 * sizeof(unsigned long long)));
        // tiles of 8^3 cells (one layer of tiles on a 2D grid)
        n_tiles_ = tiles_ * tiles_ * ((nz_ + kTile - 1) / kTile);
        n_fine_ = (size_t)kFineBins * n_tiles_ + 1;  // re-binning bins (tile, edge class, bank group)
        TILD_CUDA(dev_malloc((void**)&counts_, n_fine_ * sizeof(int)));
        TILD_CUDA(dev_malloc((void**)&tile_start_, (n_tiles_ + 1) * sizeof(int)));
        TILD_CUDA(dev_malloc((void**)&fine_start_, n_fine_ * sizeof(int)));
        scan_blocks_ = (int)((n_fine_ + 1023) / 1024);
        TILD_CUDA(dev_malloc((void**)&block_sums_, scan_blocks_ * sizeof(int)));
        n_z_blocks_ = generic_ ? (size_t)blocks(M_) : (size_t)(n_ / CZ_) * (n_ / 2 + 1);  // two species pairs: twice as many (zpass_cols2)
        n_partials_ = std::max(10 * n_z_blocks_, 5 * (size_t)tiles_ * tiles_ * tiles_);
        n_partials_ = std::max(n_partials_, 3 * (size_t)(n_ / vjp_cols(n_)) * (n_ / 2 + 1));
        TILD_CUDA(dev_malloc((void**)&partials_, n_partials_ * sizeof(double)));
        partials_bytes_ = n_partials_ * sizeof(double);
        // twiddles W_n^m = exp(-2 pi i m / n) in FP64, rounded to T
        std::vector<V> tw(n_);
        for (int m = 0; m < n_; ++m) {
            const double ang = -2.0 * 3.14159265358979323846 * (double)m / (double)n_;
            tw[m] = V{(T)std::cos(ang), (T)std::sin(ang)};
        }
        TILD_CUDA(cudaMemcpy(tw_, tw.data(), n_ * sizeof(V), cudaMemcpyHostToDevice));
        if (generic_) {
            TILD_CUDA(cudaFuncSetAttribute(generic_axis_fft<T, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gaxis_smem()));
            TILD_CUDA(cudaFuncSetAttribute(generic_axis_fft<T, +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gaxis_smem()));
            // the two factors of the line length: the most balanced split n = n1 n2
            gn1_ = 1;
            for (int f = 1; f * f <= n_; ++f)
                if (n_ % f == 0) gn1_ = f;
            gn2_ = n_ / gn1_;
            return TILD_OK;
        }
        return set_kernel_attributes();
    }

    tild_status set_chains() override {
        invalidate_graph();
        free_beads();
        if (NP_ != 1) {
            tild_status gst = alloc_grids(1);  // the chains give two species
            if (gst) return gst;
        }
        const size_t N = (size_t)cfg_->n_beads;
        for (int k = 0; k < 2; ++k) {
            TILD_CUDA(dev_malloc((void**)&pos_[k], 3 * N * sizeof(T)));
            TILD_CUDA(dev_malloc((void**)&u_[k], 3 * N * sizeof(T)));
            TILD_CUDA(dev_malloc((void**)&id_[k], N * sizeof(int)));
            TILD_CUDA(cudaMemset(u_[k], 0, 3 * N * sizeof(T)));
        }
        TILD_CUDA(dev_malloc((void**)&nbr_, N * sizeof(int2)));
        TILD_CUDA(dev_malloc((void**)&slot_of_id_, N * sizeof(int)));
        TILD_CUDA(dev_malloc((void**)&keys_, N * sizeof(int)));
        TILD_CUDA(dev_malloc((void**)&ranks_, N * sizeof(int)));
        have_pos_ = have_vel_ = false;
        return upload_topology();
    }

    // Species count, per-bead species and bond list from the HostConfig:
    // grids for the species pairs, the device topology arrays, and (with
    // positions) a re-binning and a fresh density.
    tild_status set_topology() override {
        invalidate_graph();
        tild_status st;
        const int np = cfg_->n_species > 2 ? 2 : 1;  // pairs of species on the grids
        if (np != NP_ && (st = alloc_grids(np))) return st;
        if ((st = upload_topology())) return st;
        if (have_pos_) {
            if ((st = enqueue_sort()) || (st = respread())) return st;
            TILD_CUDA(cudaStreamSynchronize(stream_));
        }
        return TILD_OK;
    }

    tild_status io_scratch(size_t bytes, void** ptr) override {
        tild_status st;
        if ((st = device_buffer(&io_, io_bytes_, bytes))) return st;
        *ptr = io_;
        return TILD_OK;
    }

    tild_status transpose3(const void* in, void* out, size_t n, int dtype, bool to_aos) override {
        if (dtype == TILD_DTYPE_F32)
            transpose_vec3<float><<<blocks(3 * n), 256, 0, stream_>>>(n, (const float*)in, (float*)out, to_aos);
        else
            transpose_vec3<double><<<blocks(3 * n), 256, 0, stream_>>>(n, (const double*)in, (double*)out, to_aos);
        TILD_CUDA(cudaGetLastError());
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    tild_status set_stream(cudaStream_t s) override {
        invalidate_graph();
        stream_ = s ? s : own_stream_;
        return TILD_OK;
    }
    cudaStream_t stream() const override { return stream_; }

    tild_status set_positions(const void* xyz, int dtype, int where) override {
        const int N = cfg_->n_beads;
        const void* src = xyz;
        tild_status st = stage_in(&src, xyz, (size_t)3 * N, dtype, where);
        if (st) return st;
        cur_pos_ = cur_u_ = cur_id_ = 0;
        const T L = (T)cfg_->L;
        if (dtype == TILD_DTYPE_F32)
            load_positions<T, float><<<blocks(N), 256, 0, stream_>>>(N, (const float*)src, L, (T)(1.0 / cfg_->L), pos_[0], id_[0], err_ptr());
        else
            load_positions<T, double><<<blocks(N), 256, 0, stream_>>>(N, (const double*)src, L, (T)(1.0 / cfg_->L), pos_[0], id_[0], err_ptr());
        TILD_CUDA(cudaGetLastError());
        if ((st = zero_z())) return st;
        if ((st = enqueue_sort())) return st;
        if ((st = respread())) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if ((st = check_err())) return st;
        have_pos_ = true;
        have_vel_ = false;
        return TILD_OK;
    }

    tild_status set_velocities(const void* v, int dtype, int where) override {
        const int N = cfg_->n_beads;
        tild_status st;
        const T* vin = nullptr;
        if (v) {
            // bring to device in precision T (AoS by id)
            const void* src = v;
            if ((st = stage_in(&src, v, (size_t)3 * N, dtype, where))) return st;
            if ((st = ensure_aux((size_t)3 * N * sizeof(T)))) return st;
            if (dtype == TILD_DTYPE_F32)
                convert_copy<float, T><<<blocks(3 * (size_t)N), 256, 0, stream_>>>((size_t)3 * N, (const float*)src, (T*)aux_);
            else
                convert_copy<double, T><<<blocks(3 * (size_t)N), 256, 0, stream_>>>((size_t)3 * N, (const double*)src, (T*)aux_);
            TILD_CUDA(cudaGetLastError());
            vin = (const T*)aux_;
        }
        if ((st = enqueue_fields(false, nullptr, nullptr))) return st;
        BeadBuffers<T> bf = bead_buffers();
        bf.v_in = vin;
        if ((st = launch_bead(kModeSetVel, bf))) return st;
        TILD_CUDA(cudaMemsetAsync(counters_, 0, 4 * sizeof(unsigned long long), stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        host_step_ = 0;
        steps_since_sort_ = 0;
        have_vel_ = true;
        return TILD_OK;
    }

    tild_status step(int64_t n) override {
        tild_status st;
        const int K = cfg_->sort_every;
        while (n > 0) {
            if (steps_since_sort_ >= K && n >= 2 * (int64_t)K) {
                // a full cycle (sort, K steps, sort, K steps) as one graph
                if ((st = run_cycle_graph())) return st;
                n -= 2 * (int64_t)K;
                host_step_ += 2 * (int64_t)K;
                continue;
            }
            if (steps_since_sort_ >= K) {
                if ((st = enqueue_sort())) return st;
            }
            if ((st = enqueue_step())) return st;
            --n;
            ++host_step_;
        }
        return TILD_OK;
    }

    tild_status synchronize() override {
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return check_err();
    }

    tild_status compute(unsigned what, tild_energy* e, void* f, int dtype, int where) override {
        tild_status st;
        const bool want_e = (what & TILD_COMPUTE_ENERGY) != 0;
        if ((st = ensure_partials())) return st;
        if ((st = enqueue_fields(want_e, partials_, nullptr))) return st;
        std::vector<double> zpart;
        if (want_e) {
            zpart.resize(5 * z_blocks());
            TILD_CUDA(cudaMemcpyAsync(zpart.data(), partials_, zpart.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
        }
        BeadBuffers<T> bf = bead_buffers();
        T* fdev = nullptr;
        if (f) {
            if ((st = ensure_aux((size_t)3 * cfg_->n_beads * sizeof(T)))) return st;
            fdev = (T*)aux_;
            bf.f_out = fdev;
        }
        if ((st = launch_bead(kModeForce, bf))) return st;
        std::vector<double> bpart(5 * bead_blocks());
        TILD_CUDA(cudaMemcpyAsync(bpart.data(), partials_, bpart.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
        if (f && (st = stage_out_vec(fdev, (size_t)3 * cfg_->n_beads, f, dtype, where))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if ((st = check_err())) return st;
        if (want_e && e) {
            double s0 = 0, s1 = 0, s4 = 0;
            for (size_t b = 0; b < z_blocks(); ++b) {
                s0 += zpart[5 * b];
                s1 += zpart[5 * b + 1];
                s4 += zpart[5 * b + 4];
            }
            const double V = volume();
            const double dV = V / (double)M_;
            const double rho0 = cfg_->n_beads / V;
            // one pair: the z pass sums Re[conj(rho_A) rho_B]; two pairs: chi-weighted sums
            e->e_chi = (NP_ == 1 ? cfg_->chi : 1.0) / rho0 * dV * dV / V * s0;
            e->e_kappa = cfg_->kappa / (2.0 * rho0) * dV * dV / V * s1;
            e->e_elec = e_elec_from(s4);
        }
        if (e) {
            double acc[5] = {0, 0, 0, 0, 0};
            for (size_t b = 0; b < bpart.size() / 5; ++b)
                for (int k = 0; k < 5; ++k) acc[k] += bpart[5 * b + k];
            e->e_bond = acc[0];
            e->kinetic = acc[1];
            for (int d = 0; d < 3; ++d) e->net_force[d] = acc[2 + d];
            if (!want_e) e->e_chi = e->e_kappa = e->e_elec = 0.0;
        }
        return TILD_OK;
    }

    tild_status energy_gradient(tild_energy_grad* g, void* dUdr, int dtype, int where) override {
        tild_status st;
        if (generic_) {
            err = "energy_gradient: implemented for the 3D grid sizes of the tiled kernels";
            return TILD_EUNSUPPORTED;
        }
        if (NP_ != 1) {
            err = "energy_gradient: implemented for one or two species";
            return TILD_EUNSUPPORTED;
        }
        if ((st = enqueue_fields(true, partials_, nullptr, kInvGradPot))) return st;
        std::vector<double> zpart(5 * n_z_blocks_);
        TILD_CUDA(cudaMemcpyAsync(zpart.data(), partials_, zpart.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
        BeadBuffers<T> bf = bead_buffers();
        if ((st = launch_bead(kModeForce, bf))) return st;  // bond energy partials
        std::vector<double> bpart(5 * (size_t)tiles_ * tiles_ * tiles_);
        TILD_CUDA(cudaMemcpyAsync(bpart.data(), partials_, bpart.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_));
        if (dUdr) {
            const size_t N = cfg_->n_beads;
            if ((st = ensure_aux(3 * N * sizeof(T)))) return st;
            const BeadParams<T> p = bead_params();
            const V* pot = grad_ + 3 * M_;
            tild_status s2 = dispatch_p([&](auto pp) -> tild_status {
                adjoint_kernel<decltype(pp)::value, T><<<blocks(N), 256, 0, stream_>>>(p, bf, pot, (T*)aux_);
                return TILD_OK;
            });
            if (s2) return s2;
            TILD_CUDA(cudaGetLastError());
            if ((st = stage_out_vec((T*)aux_, 3 * N, dUdr, dtype, where))) return st;
        }
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if ((st = check_err())) return st;
        double s[5] = {0, 0, 0, 0, 0};
        for (size_t b = 0; b < n_z_blocks_; ++b)
            for (int k = 0; k < 5; ++k) s[k] += zpart[5 * b + k];
        double eb = 0;
        for (size_t b = 0; b < bpart.size() / 5; ++b) eb += bpart[5 * b];
        const double V = cfg_->L * cfg_->L * cfg_->L;
        const double dV = V / (double)M_;
        const double rho0 = cfg_->n_beads / V;
        const double f = dV * dV / V;
        // E_chi = chi/rho0 f S0, E_kappa = kappa/(2 rho0) f S1; d u_hat/d a = -2 a |k|^2 u_hat
        g->e_bond = eb;
        g->e_chi = cfg_->chi / rho0 * f * s[0];
        g->e_kappa = cfg_->kappa / (2.0 * rho0) * f * s[1];
        g->e_elec = e_elec_from(s[4]);
        g->energy = g->e_bond + g->e_chi + g->e_kappa + g->e_elec;
        g->dU_dchi = f * s[0] / rho0;
        g->dU_dkappa = f * s[1] / (2.0 * rho0);
        g->dU_da = -2.0 * cfg_->a * (cfg_->chi / rho0 * f * s[2] + cfg_->kappa / (2.0 * rho0) * f * s[3]);
        return TILD_OK;
    }

    tild_status vjp_supported() {
        if (generic_) {
            err = "force_vjp: implemented for the 3D grid sizes of the tiled kernels";
            return TILD_EUNSUPPORTED;
        }
        if (NP_ != 1) {
            err = "force_vjp: implemented for one or two species";
            return TILD_EUNSUPPORTED;
        }
        if (analytic()) {
            err = "force_vjp: implemented for the ik force";
            return TILD_EUNSUPPORTED;
        }
        if (!plane_fits_) {
            err = "force_vjp: the grid must fit the single-plane xy passes (FP32 up to 128^3, FP64 up to 64^3)";
            return TILD_EUNSUPPORTED;
        }
        return TILD_OK;
    }
    size_t vjp_blocks() const { return (size_t)(n_ / vjp_cols(n_)) * (n_ / 2 + 1); }
    // fixed-point bits of the adjoint spread: S = min(S_max, 62 - ceil(log2 n_beads))
    int vjp_fixed_bits() const {
        int lg = 0;
        while ((1ull << lg) < (unsigned long long)cfg_->n_beads) ++lg;
        return std::min(AdjointFixed<T>::s_max, 62 - lg);
    }
    // the fixed-point spread [3][M] int64 pairs and the max|lam| bits
    size_t vjp_fx_need() const { return 6 * M_ * sizeof(unsigned long long) + 16; }
    tild_status vjp_prepare() {
        tild_status st;
        if ((st = vjp_supported())) return st;
        return device_buffer(&vjp_fx_, vjp_fx_bytes_, vjp_fx_need());
    }

    // J^T lam at the current positions into out_d (T, by id), and the
    // parameter sums added to theta_acc (device, 3 doubles); stream-ordered,
    // no host synchronisation (see vjp_kernels.cuh).
    // fields_ready: D w (grad_ fields 0..2) and Zxy of the current positions
    // are already in place, as a step starting from them leaves them.
    tild_status vjp_core(const T* lam_d, T* out_d, double* theta_acc, bool fields_ready = false) {
        const size_t N = cfg_->n_beads;
        tild_status st;
        if (!fields_ready && (st = enqueue_fields(false, nullptr, nullptr, kInvGrad))) return st;  // D w at r; Zxy = xy(rho)
        using Bits = typename AdjointFixed<T>::bits_t;
        unsigned long long* fx = (unsigned long long*)vjp_fx_;
        Bits* bits = (Bits*)(fx + 6 * M_);
        const int S = vjp_fixed_bits();
        TILD_CUDA(cudaMemsetAsync(fx, 0, vjp_fx_need(), stream_));
        lam_absmax<T><<<(int)std::min<size_t>(blocks(3 * N), 2 * 152), 256, 0, stream_>>>(3 * N, lam_d, bits);
        const BeadParams<T> p = bead_params();
        const BeadBuffers<T> bf = bead_buffers();
        if ((st = dispatch_p([&](auto pp) -> tild_status {
                 vjp_spread<decltype(pp)::value, T><<<blocks(N), 256, 0, stream_>>>(p, bf, lam_d, fx, bits, S);
                 return TILD_OK;
             })))
            return st;
        const SpectralParams<T> sp = spectral_params();
        const int el = c_el_on() ? 1 : 0;
        if ((st = dispatch_n([&](auto nn) -> tild_status {
                 constexpr int NN = decltype(nn)::value;
                 if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                     constexpr int CV = vjp_cols(NN);
                     xy_forward_cplx<T, NN><<<dim3(NN, 3), 512, plane_smem(), stream_>>>((const longlong2*)fx, bits, S, H_, tw_);
                     z_vjp<T, NN, CV><<<dim3(NN / CV, NN / 2 + 1), 256, vjp_smem(), stream_>>>(H_, Zxy_, tw_, sp, partials_, el);
                 }
                 return TILD_OK;
             })))
            return st;
        TILD_CUDA(cudaGetLastError());
        accumulate_partials<<<1, 256, 0, stream_>>>(partials_, (int)vjp_blocks(), theta_acc);
        if ((st = enqueue_inverse(kInvPot))) return st;  // psi into the potential slot
        const double dV = cfg_->L * cfg_->L * cfg_->L / (double)M_;
        if ((st = dispatch_p([&](auto pp) -> tild_status {
                 vjp_beads<decltype(pp)::value, T><<<blocks(N), 256, 0, stream_>>>(p, bf, grad_, lam_d, (T)(1.0 / dV), out_d);
                 return TILD_OK;
             })))
            return st;
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    // d(lam . F)/d(chi, kappa, a) from the accumulated sums
    void theta_from_sums(const double* s, double* dtheta) const {
        const double rho0 = cfg_->n_beads / (cfg_->L * cfg_->L * cfg_->L);
        dtheta[0] = s[0] / (rho0 * (double)M_);
        dtheta[1] = s[1] / (rho0 * (double)M_);
        dtheta[2] = -2.0 * cfg_->a * s[2];
    }
    // a device scratch of `bytes` that lives as long as the context
    template <class P> tild_status device_buffer(P** ptr, size_t& have, size_t bytes) {
        if (have >= bytes) return TILD_OK;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        dev_free(*ptr);
        *ptr = nullptr;
        have = 0;
        TILD_CUDA(dev_malloc((void**)ptr, bytes));
        have = bytes;
        return TILD_OK;
    }

    // J^T lam of the ik force at the current positions; dtheta (optional):
    // d(lam . F)/d(chi, kappa, a).
    tild_status force_vjp(const void* lam, void* out, int dtype, int where, double* dtheta) override {
        tild_status st;
        if ((st = vjp_prepare())) return st;
        const size_t N = cfg_->n_beads;
        const void* src = lam;
        if ((st = stage_in(&src, lam, 3 * N, dtype, where))) return st;
        if ((st = ensure_aux(6 * N * sizeof(T)))) return st;
        if ((st = device_buffer(&theta_, theta_bytes_, 3 * sizeof(double)))) return st;
        T* lam_d = (T*)aux_;
        T* out_d = lam_d + 3 * N;
        if (dtype == TILD_DTYPE_F32)
            convert_copy<float, T><<<blocks(3 * N), 256, 0, stream_>>>(3 * N, (const float*)src, lam_d);
        else
            convert_copy<double, T><<<blocks(3 * N), 256, 0, stream_>>>(3 * N, (const double*)src, lam_d);
        TILD_CUDA(cudaGetLastError());
        TILD_CUDA(cudaMemsetAsync(theta_, 0, 3 * sizeof(double), stream_));
        if ((st = vjp_core(lam_d, out_d, theta_))) return st;
        double s[3];
        TILD_CUDA(cudaMemcpyAsync(s, theta_, sizeof(s), cudaMemcpyDeviceToHost, stream_));
        if ((st = stage_out_vec(out_d, 3 * N, out, dtype, where))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if ((st = check_err())) return st;
        if (dtheta) theta_from_sums(s, dtheta);
        return TILD_OK;
    }

    // d/dr_i of sum_{K,g} psi_K(g) rho_K(g) for a grid adjoint psi [S][M]
    // (dtype/where), by bead id ([N][3], dtype/where).
    tild_status density_vjp(const void* psi, void* out, int dtype, int where) override {
        if (cfg_->dim != 3) {
            err = "density_vjp: three-dimensional boxes";
            return TILD_EUNSUPPORTED;
        }
        tild_status st;
        const size_t N = cfg_->n_beads, G = (size_t)cfg_->n_species * M_;
        const void* src = psi;
        if ((st = stage_in(&src, psi, G, dtype, where))) return st;
        if ((st = ensure_aux((G + 3 * N) * sizeof(T)))) return st;
        T* psi_d = (T*)aux_;
        T* out_d = psi_d + G;
        if (dtype == TILD_DTYPE_F32)
            convert_copy<float, T><<<blocks(G), 256, 0, stream_>>>(G, (const float*)src, psi_d);
        else
            convert_copy<double, T><<<blocks(G), 256, 0, stream_>>>(G, (const double*)src, psi_d);
        TILD_CUDA(cudaGetLastError());
        const BeadParams<T> p = bead_params();
        const BeadBuffers<T> bf = bead_buffers();
        const T inv_dV = (T)((double)M_ / volume());
        if ((st = dispatch_p([&](auto pp) -> tild_status {
                 density_vjp_kernel<decltype(pp)::value, T><<<blocks(N), 256, 0, stream_>>>(p, bf, psi_d, inv_dV, out_d);
                 return TILD_OK;
             })))
            return st;
        TILD_CUDA(cudaGetLastError());
        if ((st = stage_out_vec(out_d, 3 * N, out, dtype, where))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return check_err();
    }

    // positions and carried velocities by id ([2][N][3] T) <-> the context
    void store_state(T* dst) {
        const int N = cfg_->n_beads;
        store_by_id<T, T><<<blocks(N), 256, 0, stream_>>>(N, pos_[cur_pos_], id_[cur_id_], dst);
        store_by_id<T, T><<<blocks(N), 256, 0, stream_>>>(N, u_[cur_u_], id_[cur_id_], dst + 3 * (size_t)N);
    }
    tild_status restore_state(const T* src, int64_t step) {
        const int N = cfg_->n_beads;
        invalidate_graph();
        cur_pos_ = cur_u_ = cur_id_ = 0;
        load_positions<T, T><<<blocks(N), 256, 0, stream_>>>(N, src, (T)cfg_->L, (T)(1.0 / cfg_->L), pos_[0], id_[0], err_ptr());
        if (zero_z()) return TILD_EDEVICE;
        load_by_id<T, T><<<blocks(N), 256, 0, stream_>>>(N, src + 3 * (size_t)N, id_[0], u_[0]);
        TILD_CUDA(cudaGetLastError());
        tild_status st;
        if ((st = enqueue_sort()) || (st = respread())) return st;
        set_counter<<<1, 1, 0, stream_>>>(counters_, (unsigned long long)step);
        TILD_CUDA(cudaGetLastError());
        host_step_ = step;
        steps_since_sort_ = 0;
        return TILD_OK;
    }

    // A binned snapshot of the current positions, what the force VJP reads:
    // positions in slot order, slot tags, neighbour slots, tile starts and the
    // fixed-point density of those positions (after a step it holds the
    // spread of the new positions). Restoring one needs no re-binning.
    static size_t snap_part(size_t b) { return (b + 255) / 256 * 256; }
    // (with beads of more than two bonds, their neighbour slots as well)
    void snapshot_parts(void* (&ptr)[6], size_t (&bytes)[6]) {
        const size_t N = cfg_->n_beads;
        void* p[6] = {pos_[cur_pos_], id_[cur_id_], nbr_, tile_start_, rho_fx_, ext_slots_};
        const size_t b[6] = {3 * N * sizeof(T), N * sizeof(int), N * sizeof(int2), (n_tiles_ + 1) * sizeof(int),
                             2 * M_ * sizeof(unsigned long long), n_ext_ * sizeof(int)};
        for (int k = 0; k < 6; ++k) {
            ptr[k] = p[k];
            bytes[k] = b[k];
        }
    }
    size_t snapshot_bytes() {
        void* p[6];
        size_t b[6], total = 0;
        snapshot_parts(p, b);
        for (int k = 0; k < 6; ++k) total += snap_part(b[k]);
        return total;
    }
    tild_status snapshot(unsigned char* s, bool store) {
        void* p[6];
        size_t b[6];
        snapshot_parts(p, b);
        for (int k = 0; k < 6; ++k) {
            if (b[k] == 0) continue;
            if (store)
                TILD_CUDA(cudaMemcpyAsync(s, p[k], b[k], cudaMemcpyDeviceToDevice, stream_));
            else
                TILD_CUDA(cudaMemcpyAsync(p[k], s, b[k], cudaMemcpyDeviceToDevice, stream_));
            s += snap_part(b[k]);
        }
        return TILD_OK;
    }

    // The fields a step computes from its starting positions (D w, grad_
    // fields 0..2, and the xy-transformed density Zxy), what the force VJP at
    // those positions recomputes otherwise.
    size_t field_snapshot_bytes() const { return snap_part(3 * M_ * sizeof(V)) + snap_part(M_ * sizeof(V)); }
    tild_status field_snapshot(unsigned char* s, bool store) {
        const size_t b0 = 3 * M_ * sizeof(V), b1 = M_ * sizeof(V);
        unsigned char* s1 = s + snap_part(b0);
        if (store) {
            TILD_CUDA(cudaMemcpyAsync(s, grad_, b0, cudaMemcpyDeviceToDevice, stream_));
            TILD_CUDA(cudaMemcpyAsync(s1, Zxy_, b1, cudaMemcpyDeviceToDevice, stream_));
        } else {
            TILD_CUDA(cudaMemcpyAsync(grad_, s, b0, cudaMemcpyDeviceToDevice, stream_));
            TILD_CUDA(cudaMemcpyAsync(Zxy_, s1, b1, cudaMemcpyDeviceToDevice, stream_));
        }
        return TILD_OK;
    }

    // Reverse-mode derivatives of L(r^K, v^K) through K steps of the context's
    // scheme with the noise held fixed, checkpoints every C steps; the
    // recursion is that of the scheme's update form (scheme_coeffs; the
    // kernels adjoint_init and adjoint_step). Leaves the context at step K.
    tild_status trajectory_vjp(int64_t K, int C, const void* rbar, const void* vbar, int dtype, int where, void* r0,
                               void* v0, double* dtheta) override {
        tild_status st;
        if ((st = vjp_prepare())) return st;
        const size_t N = cfg_->n_beads, n3 = 3 * N, sb = 6 * N;  // one state: sb values of T
        if (C > K) C = K > 0 ? (int)K : 1;  // no snapshot beyond the trajectory
        const int64_t n_ckpt = K / C + 1;
        const size_t bsnap = snapshot_bytes(), snap = bsnap + field_snapshot_bytes();
        const size_t head = snap_part(sizeof(T) * (sb * ((size_t)n_ckpt + 1) + 2 * n3));
        const size_t need = head + snap * (size_t)C + sizeof(double) * (3 * n3 + 3);
        if ((st = device_buffer(&traj_, traj_bytes_, need))) return st;
        T* ckpt = (T*)traj_;                        // [n_ckpt][sb] by id
        T* fin = ckpt + sb * n_ckpt;                // [sb]
        T* lam = fin + sb;                          // [n3]
        T* jt = lam + n3;                           // [n3]
        unsigned char* seg = (unsigned char*)traj_ + head;  // [C] binned snapshots + fields (256-byte aligned)
        double* rb = (double*)(seg + snap * (size_t)C);
        double* ub = rb + n3;  // dL/dv^K on entry, then the adjoint of u
        double* vout = ub + n3;
        double* acc = vout + n3;
        const SchemeCoeffs q = scheme_coeffs(*cfg_);
        const int64_t step0 = host_step_;
        // forward with checkpoints
        store_state(ckpt);
        for (int64_t s = 0; s < K; ++s) {
            if ((st = step(1))) return st;
            if ((s + 1) % C == 0) store_state(ckpt + sb * ((s + 1) / C));
        }
        store_state(fin);
        // adjoint vectors
        const void* src = rbar;
        if ((st = stage_in(&src, rbar, n3, dtype, where))) return st;
        if (dtype == TILD_DTYPE_F32)
            convert_copy<float, double><<<blocks(n3), 256, 0, stream_>>>(n3, (const float*)src, rb);
        else
            convert_copy<double, double><<<blocks(n3), 256, 0, stream_>>>(n3, (const double*)src, rb);
        if (vbar) {
            src = vbar;
            if ((st = stage_in(&src, vbar, n3, dtype, where))) return st;
            if (dtype == TILD_DTYPE_F32)
                convert_copy<float, double><<<blocks(n3), 256, 0, stream_>>>(n3, (const float*)src, ub);
            else
                convert_copy<double, double><<<blocks(n3), 256, 0, stream_>>>(n3, (const double*)src, ub);
        } else {
            TILD_CUDA(cudaMemsetAsync(ub, 0, n3 * sizeof(double), stream_));
        }
        TILD_CUDA(cudaMemsetAsync(acc, 0, 3 * sizeof(double), stream_));
        adjoint_init<T><<<blocks(n3), 256, 0, stream_>>>(n3, ub, lam, q.vu, q.vf, q.wf, K == 0 ? 1 : 0);
        TILD_CUDA(cudaGetLastError());
        for (int64_t s0 = ((K - 1) / C) * C; K > 0 && s0 >= 0; s0 -= C) {
            const int64_t s1 = std::min<int64_t>(s0 + C, K);
            if ((st = restore_state(ckpt + sb * (s0 / C), step0 + s0))) return st;
            for (int64_t j = s0; j < s1; ++j) {
                if ((st = step(1))) return st;
                // step j started from r^j: its fields belong to state j (snapshot j - 1 - s0)
                if (j > s0 && (st = field_snapshot(seg + snap * (size_t)(j - 1 - s0) + bsnap, true))) return st;
                if ((st = snapshot(seg + snap * (size_t)(j - s0), true))) return st;
            }
            for (int64_t j = s1 - 1; j >= s0; --j) {
                // r^{j+1}, binned as the recomputation left it, with its fields
                // when step j+1 was recomputed
                const bool fields = j + 1 < s1;
                if ((st = snapshot(seg + snap * (size_t)(j - s0), false))) return st;
                if (fields && (st = field_snapshot(seg + snap * (size_t)(j - s0) + bsnap, false))) return st;
                if ((st = vjp_core(lam, jt, acc, fields))) return st;
                adjoint_step<T><<<blocks(n3), 256, 0, stream_>>>(n3, jt, rb, ub, lam, q.sd, q.sh, q.su, q.sf, q.wf,
                                                                  j == 0 ? 1 : 0);
                TILD_CUDA(cudaGetLastError());
            }
        }
        // the force at r^0; dL/dv^0 = wu ub
        if ((st = restore_state(ckpt, step0)) || (st = vjp_core(lam, jt, acc))) return st;
        add_into<T><<<blocks(n3), 256, 0, stream_>>>(n3, rb, jt, rb);
        scale_copy<double><<<blocks(n3), 256, 0, stream_>>>(n3, ub, q.wu, vout);
        TILD_CUDA(cudaGetLastError());
        if ((st = restore_state(fin, step0 + K))) return st;
        if ((st = stage_out_double(rb, n3, r0, dtype, where)) || (st = stage_out_double(vout, n3, v0, dtype, where)))
            return st;
        double s[3];
        TILD_CUDA(cudaMemcpyAsync(s, acc, sizeof(s), cudaMemcpyDeviceToHost, stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if ((st = check_err())) return st;
        if (dtheta) theta_from_sums(s, dtheta);
        return TILD_OK;
    }

    // Device FP64 array -> caller buffer (dtype, host or device).
    tild_status stage_out_double(const double* src, size_t count, void* out, int dtype, int where) {
        tild_status st;
        void* dst = out;
        if (where == TILD_HOST) {
            if ((st = ensure_stage(count * dtype_size(dtype)))) return st;
            dst = stage_;
        }
        if (dtype == TILD_DTYPE_F32)
            convert_copy<double, float><<<blocks(count), 256, 0, stream_>>>(count, src, (float*)dst);
        else
            convert_copy<double, double><<<blocks(count), 256, 0, stream_>>>(count, src, (double*)dst);
        TILD_CUDA(cudaGetLastError());
        if (where == TILD_HOST) {
            TILD_CUDA(cudaMemcpyAsync(out, stage_, count * dtype_size(dtype), cudaMemcpyDeviceToHost, stream_));
            TILD_CUDA(cudaStreamSynchronize(stream_));
        }
        return TILD_OK;
    }

    tild_status get_positions(void* out, int dtype, int where) override {
        return out_by_id(pos_[cur_pos_], out, dtype, where);
    }

    tild_status get_velocities(void* out, int dtype, int where) override {
        tild_status st;
        if ((st = enqueue_fields(false, nullptr, nullptr))) return st;
        if ((st = ensure_aux((size_t)3 * cfg_->n_beads * sizeof(T)))) return st;
        BeadBuffers<T> bf = bead_buffers();
        bf.v_out = (T*)aux_;
        if ((st = launch_bead(kModeForce, bf))) return st;
        if ((st = stage_out_vec((T*)aux_, (size_t)3 * cfg_->n_beads, out, dtype, where))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return check_err();
    }

    tild_status get_density(void* out, int dtype, int where) override {
        const double scale = 1.0 / FixedPoint<T>::scale / (volume() / (double)M_);
        const size_t count = (size_t)cfg_->n_species * M_;
        tild_status st;
        void* dst = out;
        if (where == TILD_HOST) {
            if ((st = ensure_aux(count * 8))) return st;
            dst = aux_;
        }
        if (dtype == TILD_DTYPE_F32)
            density_out<float><<<blocks(count), 256, 0, stream_>>>(count, rho_fx_, scale, (float*)dst);
        else
            density_out<double><<<blocks(count), 256, 0, stream_>>>(count, rho_fx_, scale, (double*)dst);
        TILD_CUDA(cudaGetLastError());
        if (where == TILD_HOST)
            TILD_CUDA(cudaMemcpyAsync(out, dst, count * dtype_size(dtype), cudaMemcpyDeviceToHost, stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    tild_status get_spectrum(void* out, int dtype, int where) override {
        tild_status st;
        if ((st = device_buffer(&spec_, spec_bytes_, NP_ * M_ * sizeof(V)))) return st;
        if ((st = enqueue_fields(false, nullptr, spec_))) return st;
        if ((st = stage_out_vec((T*)spec_, 2 * NP_ * M_, out, dtype, where))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    tild_status get_field_gradient(void* out, int dtype, int where) override {
        tild_status st;
        if ((st = enqueue_fields(false, nullptr, nullptr, kInvGrad))) return st;
        const int D = cfg_->dim;
        for (int q = 0; q < NP_; ++q) {
            char* o = (char*)out + (size_t)q * 2 * D * M_ * dtype_size(dtype);
            if ((st = stage_out_vec((T*)(grad_ + 4 * q * M_), 2 * D * M_, o, dtype, where))) return st;
            if (where == TILD_HOST) TILD_CUDA(cudaStreamSynchronize(stream_));  // the staging buffer is reused
        }
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    int64_t host_step() const override { return host_step_; }
    // blocks of the z pass (energy partials): twice as many column tiles with two species pairs
    size_t z_blocks() const { return NP_ == 2 ? (size_t)(n_ / zpass_cols2(n_)) * (n_ / 2 + 1) : n_z_blocks_; }

    // blob: magic, n_beads, sizeof(T), step, seed | pos[N][3] | u[N][3] (by id, T)
    size_t state_bytes() const override { return 5 * sizeof(uint64_t) + 6 * (size_t)cfg_->n_beads * sizeof(T); }

    // blob: 5 uint64 (magic, beads, sizeof(T), step, seed), then positions
    // and carried velocities by bead id ([2][N][3] T); in host or device memory
    tild_status get_state(void* blob, int where) override {
        const size_t N = cfg_->n_beads;
        uint64_t h[5] = {kStateMagic, N, sizeof(T), (uint64_t)host_step_, cfg_->seed};
        tild_status st;
        T* d;
        if (where == TILD_DEVICE) {
            TILD_CUDA(cudaMemcpyAsync(blob, h, sizeof(h), cudaMemcpyHostToDevice, stream_));
            d = (T*)((char*)blob + sizeof(h));
        } else {
            std::memcpy(blob, h, sizeof(h));
            if ((st = ensure_aux(6 * N * sizeof(T)))) return st;
            d = (T*)aux_;
        }
        store_by_id<T, T><<<blocks(N), 256, 0, stream_>>>((int)N, pos_[cur_pos_], id_[cur_id_], d);
        store_by_id<T, T><<<blocks(N), 256, 0, stream_>>>((int)N, u_[cur_u_], id_[cur_id_], d + 3 * N);
        TILD_CUDA(cudaGetLastError());
        if (where != TILD_DEVICE)
            TILD_CUDA(cudaMemcpyAsync((char*)blob + sizeof(h), d, 6 * N * sizeof(T), cudaMemcpyDeviceToHost, stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    tild_status set_state(const void* blob, int where) override {
        const size_t N = cfg_->n_beads;
        uint64_t h[5];
        if (where == TILD_DEVICE) {
            TILD_CUDA(cudaMemcpyAsync(h, blob, sizeof(h), cudaMemcpyDeviceToHost, stream_));
            TILD_CUDA(cudaStreamSynchronize(stream_));
        } else {
            std::memcpy(h, blob, sizeof(h));
        }
        if (h[0] != kStateMagic || h[1] != N || h[2] != sizeof(T) || h[4] != cfg_->seed) {
            err = "state blob does not match this context (beads, precision or seed)";
            return TILD_EINVAL;
        }
        invalidate_graph();
        tild_status st;
        const T* d;
        if (where == TILD_DEVICE) {
            d = (const T*)((const char*)blob + sizeof(h));
        } else {
            if ((st = ensure_aux(6 * N * sizeof(T)))) return st;
            TILD_CUDA(cudaMemcpyAsync(aux_, (const char*)blob + sizeof(h), 6 * N * sizeof(T), cudaMemcpyHostToDevice,
                                      stream_));
            d = (const T*)aux_;
        }
        cur_pos_ = cur_u_ = cur_id_ = 0;
        load_positions<T, T><<<blocks(N), 256, 0, stream_>>>((int)N, d, (T)cfg_->L, (T)(1.0 / cfg_->L), pos_[0], id_[0], err_ptr());
        if ((st = zero_z())) return st;
        load_by_id<T, T><<<blocks(N), 256, 0, stream_>>>((int)N, d + 3 * N, id_[0], u_[0]);
        TILD_CUDA(cudaGetLastError());
        if ((st = enqueue_sort())) return st;
        if ((st = respread())) return st;
        host_step_ = (int64_t)h[3];
        const unsigned long long dstep = h[3];
        TILD_CUDA(cudaMemcpyAsync(counters_, &dstep, sizeof(dstep), cudaMemcpyHostToDevice, stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        steps_since_sort_ = 0;
        have_pos_ = have_vel_ = true;
        return TILD_OK;
    }

    tild_status profile(int nsteps, double* ms) override {
        tild_status st;
        cudaEvent_t ev[6];
        for (auto& e : ev) TILD_CUDA(cudaEventCreate(&e));
        double acc[5] = {0, 0, 0, 0, 0};
        const int K = cfg_->sort_every;
        for (int s = 0; s < nsteps; ++s) {
            TILD_CUDA(cudaEventRecord(ev[0], stream_));
            if (steps_since_sort_ >= K) {
                if ((st = enqueue_sort())) return st;
            }
            TILD_CUDA(cudaEventRecord(ev[1], stream_));
            if ((st = enqueue_forward(true))) return st;
            TILD_CUDA(cudaEventRecord(ev[2], stream_));
            if ((st = enqueue_zpass(nullptr, nullptr, analytic()))) return st;
            TILD_CUDA(cudaEventRecord(ev[3], stream_));
            if ((st = enqueue_inverse(force_fields()))) return st;
            TILD_CUDA(cudaEventRecord(ev[4], stream_));
            BeadBuffers<T> bf = bead_buffers();
            bf.qx = pos_[1 - cur_pos_];
            bf.qy = bf.qx + cfg_->n_beads;
            bf.qz = bf.qy + cfg_->n_beads;
            if ((st = launch_bead(kModeStep, bf))) return st;
            TILD_CUDA(cudaEventRecord(ev[5], stream_));
            cur_pos_ = 1 - cur_pos_;
            ++steps_since_sort_;
            ++host_step_;
            TILD_CUDA(cudaEventSynchronize(ev[5]));
            float t;
            TILD_CUDA(cudaEventElapsedTime(&t, ev[1], ev[2])); acc[0] += t;
            TILD_CUDA(cudaEventElapsedTime(&t, ev[2], ev[3])); acc[1] += t;
            TILD_CUDA(cudaEventElapsedTime(&t, ev[3], ev[4])); acc[2] += t;
            TILD_CUDA(cudaEventElapsedTime(&t, ev[4], ev[5])); acc[3] += t;
            TILD_CUDA(cudaEventElapsedTime(&t, ev[0], ev[1])); acc[4] += t;
        }
        for (auto& e : ev) cudaEventDestroy(e);
        for (int k = 0; k < 5; ++k) ms[k] = nsteps > 0 ? acc[k] / nsteps : 0.0;
        return check_err();
    }

    int64_t launches(int64_t n) const override {
        const int D = cfg_->dim;
        const int64_t per_step = generic_ ? (1 + D) + 1 + (int64_t)NP_ * D + 1 : (use_planes() ? 2 : 4) + 2;
        const int64_t per_sort = 8;
        const int K = cfg_->sort_every;
        int64_t since = steps_since_sort_, sorts = 0;
        for (int64_t s = 0; s < n; ++s) {
            if (since >= K) {
                ++sorts;
                since = 0;
            }
            ++since;
        }
        return n * per_step + sorts * per_sort;
    }

    bool has_positions() const override { return have_pos_; }
    bool has_velocities() const override { return have_vel_; }

    tild_status save_velocities() override {
        const size_t N = cfg_->n_beads;
        if (!vsave_) TILD_CUDA(dev_malloc((void**)&vsave_, 3 * N * sizeof(T)));
        tild_status st;
        if ((st = enqueue_fields(false, nullptr, nullptr))) return st;
        BeadBuffers<T> bf = bead_buffers();
        bf.v_out = vsave_;
        if ((st = launch_bead(kModeForce, bf))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    tild_status restore_velocities() override {
        invalidate_graph();
        tild_status st;
        if ((st = enqueue_fields(false, nullptr, nullptr))) return st;
        BeadBuffers<T> bf = bead_buffers();
        bf.v_in = vsave_;
        if ((st = launch_bead(kModeSetVel, bf))) return st;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    void params_changed() override { invalidate_graph(); }

    // Launch shapes: plane threads (128, 256 or 512 where the grid allows)
    // and the z pass's column tile (the default or the alternative).
    void launch_shapes(int* plane_threads, int* z_cols, int* z_default, int* z_alt) const override {
        *plane_threads = plane_nt_;
        const int cdef = dispatch_cols(false), calt = dispatch_cols(true);
        *z_cols = zalt_ ? calt : cdef;
        if (z_default) *z_default = cdef;
        if (z_alt) *z_alt = calt;
    }
    tild_status set_launch_shapes(int plane_threads, int z_cols) override {
        if (generic_) {
            err = "launch shapes: the any-size kernels have none";
            return TILD_EUNSUPPORTED;
        }
        bool ok = false;
        dispatch_n([&](auto nn) {
            constexpr int NN = decltype(nn)::value;
            ok = plane_threads == 512 || (plane_fits_ && ((plane_threads == 256 && plane_nt_ok(NN, 256)) ||
                                                         (plane_threads == 128 && plane_nt_ok(NN, 128)) ||
                                                         (plane_threads == 1024 && plane_nt_ok(NN, 1024)) ||
                                                         (plane_threads == 0 && split_ok(NN))));
            return TILD_OK;
        });
        const int cdef = dispatch_cols(false), calt = dispatch_cols(true);
        if (!ok || (z_cols != cdef && z_cols != calt)) {
            err = "launch shapes: plane threads must be 512 (or 128/256/1024 where the grid allows, or 0 for the row "
                  "and column passes) and the z columns the default or the alternative tile";
            return TILD_EINVAL;
        }
        invalidate_graph();
        plane_nt_ = plane_threads;
        zalt_ = z_cols != cdef;
        return TILD_OK;
    }
    int dispatch_cols(bool alt) const {
        int c = 0;
        const_cast<Engine*>(this)->dispatch_n([&](auto nn) {
            c = alt ? zpass_cols_alt(decltype(nn)::value) : zpass_cols(decltype(nn)::value);
            return TILD_OK;
        });
        return c;
    }

   private:
    T* vsave_ = nullptr;
    HostConfig* cfg_ = nullptr;
    // species pairs of the grids (1: up to two species, 2: three or four) and
    // species slots of the bead kernels (2 NP)
    int NP_ = 1, NS_ = 2;
    // launch shapes of the step (tild_set_launch_shapes, tild_autotune):
    // threads of the xy plane CTAs and the z pass's column tile
    int plane_nt_ = 512;
    bool zalt_ = false;
    // any-size / 2D kernels: grid planes along z, the two factors of n
    bool generic_ = false;
    int nz_ = 0, gn1_ = 1, gn2_ = 1;
    size_t partials_bytes_ = 0;
    // explicit topology (by bead id): species, first two neighbours, and the
    // extra neighbour lists of beads with more than two bonds (ids and slots)
    unsigned char* sp_of_id_ = nullptr;
    int2* adj_ = nullptr;
    int* ext_ids_ = nullptr;
    int* ext_slots_ = nullptr;
    size_t n_ext_ = 0;
    void* io_ = nullptr;  // per-bead vectors in the other layout
    size_t io_bytes_ = 0;
    size_t spec_bytes_ = 0;
    std::unordered_map<void*, size_t> live_;  // blocks from the caller's allocator
    int device_ = 0;
    int n_ = 0, tiles_ = 0, P_ = 2, C_ = 16, CZ_ = 8;
    size_t M_ = 0;
    bool plane_fits_ = true;
    cudaStream_t own_stream_ = nullptr, stream_ = nullptr;
    // grids
    unsigned long long* rho_fx_ = nullptr;
    V* Zxy_ = nullptr;
    V* H_ = nullptr;
    V* grad_ = nullptr;
    V* tw_ = nullptr;
    T* kernel1d_ = nullptr;
    double kernel_a_ = -1.0, kernel_ae_ = -1.0;
    V* spec_ = nullptr;
    unsigned long long* counters_ = nullptr;  // [0] noise step counter, [1] error flags
    double* partials_ = nullptr;
    size_t n_partials_ = 0, n_z_blocks_ = 0;
    // beads
    T* pos_[2] = {nullptr, nullptr};
    T* u_[2] = {nullptr, nullptr};
    int* id_[2] = {nullptr, nullptr};
    int2* nbr_ = nullptr;
    int* slot_of_id_ = nullptr;
    int* keys_ = nullptr;   // re-binning: fine bin of each bead
    int* ranks_ = nullptr;  // and its rank in the bin
    int* counts_ = nullptr;  // [n_fine_] bead counts of the fine bins
    size_t n_fine_ = 0;
    int* tile_start_ = nullptr;
    int n_tiles_ = 0;
    int* fine_start_ = nullptr;  // [n_fine_] exclusive scan of counts_
    int* block_sums_ = nullptr;
    int scan_blocks_ = 0;
    int cur_pos_ = 0, cur_u_ = 0, cur_id_ = 0;
    int steps_since_sort_ = 0;
    int64_t host_step_ = 0;
    bool have_pos_ = false, have_vel_ = false;
    // staging
    void* aux_ = nullptr;
    size_t aux_bytes_ = 0;
    double* theta_ = nullptr;  // force-VJP parameter sums
    size_t theta_bytes_ = 0;
    void* traj_ = nullptr;     // trajectory derivatives: checkpoints and adjoint vectors
    size_t traj_bytes_ = 0;
    void* vjp_fx_ = nullptr;   // force VJP: fixed-point spread of lam
    size_t vjp_fx_bytes_ = 0;
    void* stage_ = nullptr;
    size_t stage_bytes_ = 0;
    // graph cache
    cudaGraphExec_t graph_ = nullptr;
    int graph_key_ = -1;

    unsigned int* err_ptr() const { return reinterpret_cast<unsigned int*>(counters_ + 1) + 1; }

    static unsigned blocks(size_t count) { return (unsigned)((count + 255) / 256); }
    static size_t dtype_size(int dtype) { return dtype == TILD_DTYPE_F32 ? 4 : 8; }

    size_t plane_smem() const { return ((size_t)n_ + (size_t)n_ * row_pitch(n_)) * sizeof(V); }
    // two dimensions: z stays 0
    tild_status zero_z() {
        if (cfg_->dim == 2)
            TILD_CUDA(cudaMemsetAsync(pos_[0] + 2 * (size_t)cfg_->n_beads, 0, (size_t)cfg_->n_beads * sizeof(T), stream_));
        return TILD_OK;
    }
    double volume() const { return cfg_->dim == 2 ? cfg_->L * cfg_->L : cfg_->L * cfg_->L * cfg_->L; }
    // lines per CTA of the any-size axis transform: about 96 KB of shared memory
    int gaxis_lines() const {
        const long c = ((long)(96 * 1024 / sizeof(V)) - n_) / (2L * (n_ + 1));
        return (int)std::max(1L, std::min(32L, c));
    }
    size_t gaxis_smem() const { return ((size_t)n_ + 2 * (size_t)gaxis_lines() * (n_ + 1)) * sizeof(V); }
    // blocks of the bead kernel (its FP64 partial sums)
    size_t bead_blocks() const { return generic_ ? (size_t)blocks(cfg_->n_beads) : (size_t)tiles_ * tiles_ * tiles_; }
    tild_status ensure_partials() {
        const size_t need = 5 * std::max(bead_blocks(), z_blocks()) * sizeof(double);
        return device_buffer(&partials_, partials_bytes_, need);
    }
    // the any-size transforms of `count` contiguous fields at f along every axis
    tild_status generic_fft(V* f, int count, int dir) {
        const int C = gaxis_lines();
        const unsigned tiles = (unsigned)((M_ / n_ + C - 1) / C);
        for (int axis = 0; axis < cfg_->dim; ++axis) {
            if (dir < 0)
                generic_axis_fft<T, -1><<<dim3(tiles, count), 256, gaxis_smem(), stream_>>>(f, n_, nz_, axis, C, gn1_, gn2_, tw_);
            else
                generic_axis_fft<T, +1><<<dim3(tiles, count), 256, gaxis_smem(), stream_>>>(f, n_, nz_, axis, C, gn1_, gn2_, tw_);
        }
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    size_t rows_smem() const { return ((size_t)n_ + (size_t)16 * row_pitch(n_)) * sizeof(V); }
    size_t ycol_smem() const { return ((size_t)n_ + 2 * (size_t)n_ * C_) * sizeof(V); }
    size_t zpass_smem() const { return ((size_t)n_ + 4 * (size_t)n_ * CZ_) * sizeof(V); }
    bool analytic() const { return cfg_->force_method == TILD_FORCE_ANALYTIC; }
    bool c_el_on() const { return cfg_->bjerrum > 0 && (cfg_->q_a != 0 || cfg_->q_b != 0); }
    // E_el = (4 pi l_B) dV^2 / (2 V) sum_k exp(-a_e^2 k^2)/k^2 |q_A rho^_A + q_B rho^_B|^2
    double e_elec_from(double s4) const {
        const double V = cfg_->L * cfg_->L * cfg_->L, dV = V / (double)M_;
        return c_el_on() ? 4.0 * 3.14159265358979323846 * cfg_->bjerrum * dV * dV / (2.0 * V) * s4 : 0.0;
    }
    size_t bead_smem() const { return bead_smem(analytic(), NS_); }
    // width and first stencil offset of the bead kernels' shared patch
    void patch_geometry(int* w, int* lo) const {
        switch (P_) {
            case 2: *w = Patch<2>::W; *lo = Patch<2>::lo; break;
            case 3: *w = Patch<3>::W; *lo = Patch<3>::lo; break;
            case 4: *w = Patch<4>::W; *lo = Patch<4>::lo; break;
            default: *w = Patch<5>::W; *lo = Patch<5>::lo; break;
        }
    }
    template <int P> static size_t bead_smem_p(bool an, int ns) {
        if (ns == 4) return an ? bead_smem_bytes<P, T, true, 4>() : bead_smem_bytes<P, T, false, 4>();
        return an ? bead_smem_bytes<P, T, true>() : bead_smem_bytes<P, T>();
    }
    size_t bead_smem(bool an, int ns) const {
        switch (P_) {
            case 2: return bead_smem_p<2>(an, ns);
            case 3: return bead_smem_p<3>(an, ns);
            case 4: return bead_smem_p<4>(an, ns);
            default: return bead_smem_p<5>(an, ns);
        }
    }

    // Device memory through the caller's allocator when one was given.
    cudaError_t dev_malloc(void** p, size_t bytes) {
        const tild_allocator& a = cfg_->allocator;
        if (!a.alloc) return cudaMalloc(p, bytes);
        *p = bytes ? a.alloc(bytes, a.user) : nullptr;
        if (bytes && !*p) return cudaErrorMemoryAllocation;
        if (*p) live_[*p] = bytes;
        return cudaSuccess;
    }
    void dev_free(void* p) {
        if (!p) return;
        const tild_allocator& a = cfg_->allocator;
        if (!a.alloc) {
            cudaFree(p);
            return;
        }
        auto it = live_.find(p);
        const size_t bytes = it == live_.end() ? 0 : it->second;
        if (it != live_.end()) live_.erase(it);
        if (a.free) a.free(p, bytes, a.user);
    }

    // Density, spectrum and field grids for np species pairs.
    tild_status alloc_grids(int np) {
        if (stream_) TILD_CUDA(cudaStreamSynchronize(stream_));
        void* old[] = {rho_fx_, Zxy_, H_, grad_};
        for (void* q : old) dev_free(q);
        rho_fx_ = nullptr;
        Zxy_ = H_ = grad_ = nullptr;
        NP_ = np;
        NS_ = 2 * np;
        TILD_CUDA(dev_malloc((void**)&rho_fx_, 2 * np * M_ * sizeof(unsigned long long)));
        TILD_CUDA(dev_malloc((void**)&Zxy_, np * M_ * sizeof(V)));
        TILD_CUDA(dev_malloc((void**)&H_, 3 * np * M_ * sizeof(V)));
        TILD_CUDA(dev_malloc((void**)&grad_, 4 * np * M_ * sizeof(V)));  // per pair: 3 gradients + (optional) potentials
        TILD_CUDA(cudaMemset(rho_fx_, 0, 2 * np * M_ * sizeof(unsigned long long)));
        return TILD_OK;
    }

    // Device copies of the explicit species and bonds (none: the chains'
    // pattern and linear bonds).
    tild_status upload_topology() {
        TILD_CUDA(cudaStreamSynchronize(stream_));
        dev_free(sp_of_id_);
        dev_free(adj_);
        dev_free(ext_ids_);
        dev_free(ext_slots_);
        sp_of_id_ = nullptr;
        adj_ = nullptr;
        ext_ids_ = ext_slots_ = nullptr;
        n_ext_ = 0;
        const size_t N = cfg_->n_beads;
        if (N == 0) return TILD_OK;
        if (!cfg_->species_of_bead.empty()) {
            TILD_CUDA(dev_malloc((void**)&sp_of_id_, N));
            TILD_CUDA(cudaMemcpy(sp_of_id_, cfg_->species_of_bead.data(), N, cudaMemcpyHostToDevice));
        }
        if (cfg_->explicit_bonds) {
            // adjacency by id, neighbours in increasing id order
            std::vector<std::vector<int>> nb(N);
            const std::vector<int>& bp = cfg_->bond_pairs;
            for (size_t k = 0; k + 1 < bp.size(); k += 2) {
                nb[bp[k]].push_back(bp[k + 1]);
                nb[bp[k + 1]].push_back(bp[k]);
            }
            std::vector<int2> adj(N, make_int2(-1, -1));
            std::vector<int> ext;
            for (size_t b = 0; b < N; ++b) {
                std::vector<int>& v = nb[b];
                std::sort(v.begin(), v.end());
                if (v.size() >= 1) adj[b].x = v[0];
                if (v.size() == 2) adj[b].y = v[1];
                if (v.size() > 2) {
                    adj[b].y = -2 - (int)ext.size();
                    ext.push_back((int)v.size() - 1);
                    ext.insert(ext.end(), v.begin() + 1, v.end());
                }
            }
            TILD_CUDA(dev_malloc((void**)&adj_, N * sizeof(int2)));
            TILD_CUDA(cudaMemcpy(adj_, adj.data(), N * sizeof(int2), cudaMemcpyHostToDevice));
            if (!ext.empty()) {
                n_ext_ = ext.size();
                TILD_CUDA(dev_malloc((void**)&ext_ids_, n_ext_ * sizeof(int)));
                TILD_CUDA(dev_malloc((void**)&ext_slots_, n_ext_ * sizeof(int)));
                TILD_CUDA(cudaMemcpy(ext_ids_, ext.data(), n_ext_ * sizeof(int), cudaMemcpyHostToDevice));
            }
        }
        return TILD_OK;
    }

    void free_beads() {
        for (int k = 0; k < 2; ++k) {
            dev_free(pos_[k]);
            dev_free(u_[k]);
            dev_free(id_[k]);
            pos_[k] = u_[k] = nullptr;
            id_[k] = nullptr;
        }
        dev_free(nbr_);
        dev_free(slot_of_id_);
        dev_free(keys_);
        dev_free(ranks_);
        dev_free(vsave_);
        vsave_ = nullptr;
        nbr_ = nullptr;
        slot_of_id_ = keys_ = ranks_ = nullptr;
    }

    void release() {
        invalidate_graph();
        if (stream_) cudaStreamSynchronize(stream_);  // no kernel may still use a block handed back
        free_beads();
        void* ptrs[] = {rho_fx_, Zxy_, H_, grad_, tw_, kernel1d_, spec_, counters_, partials_, counts_,
                        tile_start_, fine_start_, block_sums_, aux_, stage_, theta_, traj_, vjp_fx_,
                        sp_of_id_, adj_, ext_ids_, ext_slots_, io_};
        for (void* p : ptrs) dev_free(p);
        rho_fx_ = nullptr;
        if (own_stream_) cudaStreamDestroy(own_stream_);
        own_stream_ = nullptr;
    }

    void invalidate_graph() {
        if (graph_) cudaGraphExecDestroy(graph_);
        graph_ = nullptr;
        graph_key_ = -1;
    }

    tild_status check_err() {
        unsigned int h = 0;
        TILD_CUDA(cudaMemcpy(&h, err_ptr(), sizeof(h), cudaMemcpyDeviceToHost));
        if (h & kErrBounds) {
            TILD_CUDA(cudaMemset(err_ptr(), 0, sizeof(unsigned int)));
            err = "a bounds check of the debug build failed on the device (the access was skipped)";
            return TILD_EDEVICE;
        }
        if (h & kErrNonFinite) {
            TILD_CUDA(cudaMemset(err_ptr(), 0, sizeof(unsigned int)));
            err = "non-finite position or force detected on the device";
            return TILD_ENAN;
        }
        return TILD_OK;
    }

    tild_status ensure_aux(size_t bytes) {
        if (aux_bytes_ >= bytes) return TILD_OK;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        dev_free(aux_);
        aux_ = nullptr;
        aux_bytes_ = 0;
        TILD_CUDA(dev_malloc(&aux_, bytes));
        aux_bytes_ = bytes;
        return TILD_OK;
    }

    tild_status ensure_stage(size_t bytes) {
        if (stage_bytes_ >= bytes) return TILD_OK;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        dev_free(stage_);
        stage_ = nullptr;
        stage_bytes_ = 0;
        TILD_CUDA(dev_malloc(&stage_, bytes));
        stage_bytes_ = bytes;
        return TILD_OK;
    }

    // Host input -> device staging buffer (same dtype); device input as is.
    tild_status stage_in(const void** dev, const void* src, size_t count, int dtype, int where) {
        if (where == TILD_DEVICE) {
            *dev = src;
            return TILD_OK;
        }
        tild_status st;
        if ((st = ensure_stage(count * dtype_size(dtype)))) return st;
        TILD_CUDA(cudaMemcpyAsync(stage_, src, count * dtype_size(dtype), cudaMemcpyHostToDevice, stream_));
        *dev = stage_;
        return TILD_OK;
    }

    // Device array of T -> caller buffer (dtype, host or device).
    tild_status stage_out_vec(const T* src, size_t count, void* out, int dtype, int where) {
        tild_status st;
        void* dst = out;
        if (where == TILD_HOST) {
            if ((st = ensure_stage(count * dtype_size(dtype)))) return st;
            dst = stage_;
        }
        if (dtype == TILD_DTYPE_F32)
            convert_copy<T, float><<<blocks(count), 256, 0, stream_>>>(count, src, (float*)dst);
        else
            convert_copy<T, double><<<blocks(count), 256, 0, stream_>>>(count, src, (double*)dst);
        TILD_CUDA(cudaGetLastError());
        if (where == TILD_HOST)
            TILD_CUDA(cudaMemcpyAsync(out, dst, count * dtype_size(dtype), cudaMemcpyDeviceToHost, stream_));
        return TILD_OK;
    }

    tild_status out_by_id(const T* src, void* out, int dtype, int where) {
        const int N = cfg_->n_beads;
        tild_status st;
        void* dst = out;
        if (where == TILD_HOST) {
            if ((st = ensure_stage((size_t)3 * N * dtype_size(dtype)))) return st;
            dst = stage_;
        }
        if (dtype == TILD_DTYPE_F32)
            store_by_id<T, float><<<blocks(N), 256, 0, stream_>>>(N, src, id_[cur_id_], (float*)dst);
        else
            store_by_id<T, double><<<blocks(N), 256, 0, stream_>>>(N, src, id_[cur_id_], (double*)dst);
        TILD_CUDA(cudaGetLastError());
        if (where == TILD_HOST)
            TILD_CUDA(cudaMemcpyAsync(out, dst, (size_t)3 * N * dtype_size(dtype), cudaMemcpyDeviceToHost, stream_));
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    // ---------------------------------------------------------- kernels

    template <int NN> tild_status attrs_n() {
        if (plane_fits_) {
            if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                if constexpr (plane_nt_ok(NN, 256)) {
                    TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane<T, NN, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                    TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane<T, NN, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                }
                if constexpr (plane_nt_ok(NN, 128)) {
                    TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane<T, NN, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                    TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane<T, NN, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                }
                if constexpr (plane_nt_ok(NN, 1024)) {
                    TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane<T, NN, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                    TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane<T, NN, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                }
                TILD_CUDA(cudaFuncSetAttribute(xy_forward_cplx<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plane_smem()));
                TILD_CUDA(cudaFuncSetAttribute(z_vjp<T, NN, vjp_cols(NN)>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vjp_smem()));
            }
        }
        if (!plane_fits_ || split_ok(NN)) {
            TILD_CUDA(cudaFuncSetAttribute(x_forward_rows<T, NN, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem()));
            TILD_CUDA(cudaFuncSetAttribute(x_inverse_rows<T, NN, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem()));
            TILD_CUDA(cudaFuncSetAttribute(y_columns<T, NN, 128 / sizeof(V), -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ycol_smem()));
            TILD_CUDA(cudaFuncSetAttribute(y_columns<T, NN, 128 / sizeof(V), +1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ycol_smem()));
        }
        constexpr int CC = zpass_cols(NN);
        constexpr int C2 = zpass_cols2(NN);
        TILD_CUDA(cudaFuncSetAttribute(z_spectral_pairs<T, NN, C2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass2_smem()));
        TILD_CUDA(cudaFuncSetAttribute(z_spectral_pairs<T, NN, C2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass2_smem()));
        TILD_CUDA(cudaFuncSetAttribute(z_spectral<T, NN, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass_smem()));
        if constexpr (zpass_cols_alt(NN) != CC)
            TILD_CUDA(cudaFuncSetAttribute(z_spectral<T, NN, zpass_cols_alt(NN)>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)zpass_smem_cols(zpass_cols_alt(NN))));
        TILD_CUDA(cudaFuncSetAttribute(z_spectral<T, NN, CC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass_smem()));
        TILD_CUDA(cudaFuncSetAttribute(z_spectral<T, NN, CC, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass_smem()));
        TILD_CUDA(cudaFuncSetAttribute(z_spectral<T, NN, CC, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zpass_smem()));
        return TILD_OK;
    }

    template <int P> tild_status attrs_p() {
        const int s4 = (int)bead_smem(false, 4), sa4 = (int)bead_smem(true, 4);
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSpread, T, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeForce, T, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSetVel, T, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeStep, T, false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeForce, T, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSetVel, T, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa4));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeStep, T, true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa4));
        const int s = (int)bead_smem(false, 2);
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSpread, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeForce, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSetVel, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeStep, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
        const int sa = (int)bead_smem(true, 2);
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeForce, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeSetVel, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
        TILD_CUDA(cudaFuncSetAttribute(bead_kernel<P, kModeStep, T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sa));
        return TILD_OK;
    }

    tild_status set_kernel_attributes() {
        tild_status st = dispatch_n([&](auto nn) { return this->template attrs_n<decltype(nn)::value>(); });
        if (st) return st;
        return dispatch_p([&](auto pp) { return this->template attrs_p<decltype(pp)::value>(); });
    }

    template <int V_> struct ic { static constexpr int value = V_; };


    template <class F> tild_status dispatch_n(F&& f) {
        switch (n_) {
            case 8: return f(ic<8>{});
            case 16: return f(ic<16>{});
            case 32: return f(ic<32>{});
            case 64: return f(ic<64>{});
            case 128: return f(ic<128>{});
            case 24: return f(ic<24>{});
            case 40: return f(ic<40>{});
            case 48: return f(ic<48>{});
            case 80: return f(ic<80>{});
            case 256: return dispatch_256(f);
        }
        err = "unsupported grid size";
        return TILD_EUNSUPPORTED;
    }
    template <class F> tild_status dispatch_256(F&& f) {
        if constexpr (sizeof(T) == 4) return f(ic<256>{});
        err = "FP64 grids are limited to 128^3";
        return TILD_EUNSUPPORTED;
    }
    template <class F> tild_status dispatch_p(F&& f) {
        switch (P_) {
            case 2: return f(ic<2>{});
            case 3: return f(ic<3>{});
            case 4: return f(ic<4>{});
            case 5: return f(ic<5>{});
        }
        err = "unsupported pmeorder";
        return TILD_EUNSUPPORTED;
    }

    T density_scale() const {
        const double dV = volume() / (double)M_;
        return (T)(1.0 / FixedPoint<T>::scale / dV);
    }

    template <int NN> tild_status forward_n(bool zero_after) {
        if (use_planes()) {
            if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                with_nt<NN>([&](auto nt) {
                    constexpr int NT = decltype(nt)::value;
                    xy_forward_plane<T, NN, NT><<<dim3(NN, NP_), NT, plane_smem(), stream_>>>(
                        rho_fx_, Zxy_, tw_, density_scale(), zero_after ? 1 : 0, zero_after ? counters_ : nullptr);
                });
            }
        } else {
            constexpr int CC = 128 / sizeof(V);
            if constexpr (NN >= 16 && NN >= CC) {
                x_forward_rows<T, NN, 16><<<dim3((unsigned)((size_t)NN * NN / 16), NP_), 256, rows_smem(), stream_>>>(
                    rho_fx_, Zxy_, tw_, density_scale(), zero_after ? 1 : 0, zero_after ? counters_ : nullptr);
                y_columns<T, NN, CC, -1><<<dim3(NN / CC, NN, NP_), 256, ycol_smem(), stream_>>>(Zxy_, tw_, two_pi_L(), 0);
            }
        }
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    tild_status enqueue_forward(bool zero_after) {
        if (generic_) {
            generic_load_density<T><<<blocks((size_t)NP_ * M_), 256, 0, stream_>>>(
                M_, NP_, rho_fx_, Zxy_, density_scale(), zero_after ? 1 : 0, zero_after ? counters_ : nullptr);
            TILD_CUDA(cudaGetLastError());
            return generic_fft(Zxy_, NP_, -1);
        }
        return dispatch_n([&](auto nn) { return this->template forward_n<decltype(nn)::value>(zero_after); });
    }

    // z-pass column tile: 128 bytes of complex values, or the largest power of
    // two dividing n when that is smaller
    // force-VJP z pass column tile: the z pass's up to 64^3 (shared memory
    // 8 n C elements), half of it above, at least 2
    static constexpr int vjp_cols(int n) {
        return n <= 64 ? zpass_cols(n) : (zpass_cols(n) / 2 < 2 ? 2 : zpass_cols(n) / 2);
    }
    size_t vjp_smem() const { return ((size_t)n_ + 8 * (size_t)n_ * vjp_cols(n_)) * sizeof(V); }

    static constexpr int zpass_cols(int n) {
        int c = (int)(128 / sizeof(V));
        while (c > 1 && (n % c) != 0) c /= 2;
        return c < n ? c : n;
    }
    // two species pairs: half the columns (twice the buffers), at least 2
    static constexpr int zpass_cols2(int n) { return zpass_cols(n) / 2 < 2 ? 2 : zpass_cols(n) / 2; }
    // the alternative column tile of the z pass (launch shapes): half the
    // default, at least 2
    static constexpr int zpass_cols_alt(int n) { return zpass_cols2(n); }
    size_t zpass_smem_cols(int c) const { return ((size_t)n_ + 4 * (size_t)n_ * c) * sizeof(V); }
    // plane kernels with NT threads: stage B of the line transform keeps
    // ceil(n N1 / NT) units of N2 values per thread; at most 32 complex.
    // 1024 threads where every thread has a stage-B unit (n N1 >= 1024).
    static constexpr bool plane_nt_ok(int n, int nt) {
        if (nt == 512) return true;
        const int n1 = n == 8 ? 8 : n == 16 ? 4 : (n == 48 || n == 80 || n == 128 || n == 256) ? 16 : 8;
        const int n2 = n / n1;
        if (nt == 1024) return sizeof(V) == 8 && n * n1 >= 1024 && n <= 128;
        if (n > 80 || (nt != 128 && nt != 256)) return false;
        return (n * n1 + nt - 1) / nt * n2 <= 32;
    }
    // The row and column passes (x rows, then y columns, through global
    // memory) serve grids whose planes do not fit shared memory, and are the
    // launch shape plane_threads = 0 for those that do.
    static constexpr bool split_ok(int n) {
        return n >= 16 && n % (int)(128 / sizeof(V)) == 0;  // whole column tiles (and rows in blocks of 16)
    }
    bool use_planes() const { return plane_fits_ && plane_nt_ != 0; }
    // runtime forms for the batch's groups
    static bool plane_nt_allowed(int n, int nt) { return plane_nt_ok(n, nt) && n * (n + 1) * (int)sizeof(V) <= 200 * 1024; }
    static int zpass_cols_n(int n) { return zpass_cols(n); }
    static int zpass_cols_alt_n(int n) { return zpass_cols_alt(n); }
    template <int NN, class F> void with_nt(F&& f) {
        if constexpr (plane_nt_ok(NN, 1024))
            if (plane_nt_ == 1024) return f(ic<1024>{});
        if constexpr (plane_nt_ok(NN, 128))
            if (plane_nt_ == 128) return f(ic<128>{});
        if constexpr (plane_nt_ok(NN, 256))
            if (plane_nt_ == 256) return f(ic<256>{});
        return f(ic<512>{});
    }
    size_t zpass2_smem() const { return ((size_t)n_ + 8 * (size_t)n_ * zpass_cols2(n_)) * sizeof(V); }

    T two_pi_L() const { return (T)(2.0 * 3.14159265358979323846 / cfg_->L); }

    SpectralParams<T> spectral_params() const {
        const double V = volume();
        const double rho0 = cfg_->n_beads / V;
        SpectralParams<T> sp;
        sp.two_pi_over_L = (T)(2.0 * 3.14159265358979323846 / cfg_->L);
        sp.eAA = (T)(cfg_->kappa / rho0 / (double)M_);
        sp.eBB = sp.eAA;
        sp.eAB = (T)((cfg_->chi + cfg_->kappa) / rho0 / (double)M_);
        for (int K = 0; K < 4; ++K)
            for (int K2 = 0; K2 < 4; ++K2) {
                const double chi = K == K2 ? 0.0 : cfg_->chi_mat[K][K2];
                sp.eps4[K][K2] = (T)((chi + cfg_->kappa) / rho0 / (double)M_);
                sp.chi4[K][K2] = (T)chi;
            }
        sp.kernel1d = kernel1d_;
        const bool charged = c_el_on();
        sp.el_scale = charged ? (T)(4.0 * 3.14159265358979323846 * cfg_->bjerrum / (double)M_) : T(0);
        sp.qA = (T)cfg_->q_a;
        sp.qB = (T)cfg_->q_b;
        sp.kernel1d_el = kernel1d_ + n_;
        return sp;
    }

    template <int NN> tild_status zpass_n(double* partials, V* spec_out, bool g_only) {
        constexpr int CC = zpass_cols(NN);
        const dim3 grid(NN / CC, NN / 2 + 1);
        const SpectralParams<T> sp = spectral_params();
        const bool el = c_el_on();
        if (NP_ == 2) {
            if (spec_out) {
                // the spectra alone: each pair's forward z transform (no coupling)
                for (int q = 0; q < 2; ++q)
                    z_spectral<T, NN, CC><<<grid, 256, zpass_smem(), stream_>>>(Zxy_ + q * M_, H_, tw_, sp, nullptr,
                                                                              spec_out + q * M_);
            } else {
                constexpr int C2 = zpass_cols2(NN);
                const dim3 grid2(NN / C2, NN / 2 + 1);
                if (g_only)
                    z_spectral_pairs<T, NN, C2, true><<<grid2, 256, zpass2_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials);
                else
                    z_spectral_pairs<T, NN, C2><<<grid2, 256, zpass2_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials);
            }
            TILD_CUDA(cudaGetLastError());
            return TILD_OK;
        }
        if (g_only && el)
            z_spectral<T, NN, CC, true, true><<<grid, 256, zpass_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials, spec_out);
        else if (g_only)
            z_spectral<T, NN, CC, true><<<grid, 256, zpass_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials, spec_out);
        else if (el)
            z_spectral<T, NN, CC, false, true><<<grid, 256, zpass_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials, spec_out);
        else if (zalt_ && !partials && !spec_out) {
            // the step's z pass with the alternative column tile (launch shapes)
            constexpr int CA = zpass_cols_alt(NN);
            z_spectral<T, NN, CA><<<dim3(NN / CA, NN / 2 + 1), 256, zpass_smem_cols(CA), stream_>>>(Zxy_, H_, tw_, sp,
                                                                                                 nullptr, nullptr);
        } else
            z_spectral<T, NN, CC><<<grid, 256, zpass_smem(), stream_>>>(Zxy_, H_, tw_, sp, partials, spec_out);
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    // separable Gaussian tables exp(-s^2 k_m^2), k_m = 2 pi m / L, m in FFT
    // index order: the pair kernel's (s = a) and, with charges, the charge
    // smearing's (s = a_e); rebuilt when the parameter changes
    tild_status refresh_tables() {
        auto refresh = [&](double s, double& cached, T* dst) -> tild_status {
            if (cached == s) return TILD_OK;
            std::vector<T> e(n_);
            for (int i = 0; i < n_; ++i) {
                const double m = 2 * i < n_ ? i : i - n_;  // odd n: frequencies -(n-1)/2 .. (n-1)/2
                const double k = 2.0 * 3.14159265358979323846 * m / cfg_->L;
                e[i] = (T)std::exp(-s * s * k * k);
            }
            TILD_CUDA(cudaStreamSynchronize(stream_));  // no z pass may still read the old table
            TILD_CUDA(cudaMemcpy(dst, e.data(), n_ * sizeof(T), cudaMemcpyHostToDevice));
            cached = s;
            return TILD_OK;
        };
        tild_status st;
        if ((st = refresh(cfg_->a, kernel_a_, kernel1d_))) return st;
        if (c_el_on() && (st = refresh(cfg_->charge_smear, kernel_ae_, kernel1d_ + n_))) return st;
        return TILD_OK;
    }
    tild_status enqueue_zpass(double* partials, V* spec_out, bool g_only = false) {
        tild_status st;
        if ((st = refresh_tables())) return st;
        if (generic_) {
            if (spec_out) {  // the spectrum is complete after the forward transforms
                TILD_CUDA(cudaMemcpyAsync(spec_out, Zxy_, NP_ * M_ * sizeof(V), cudaMemcpyDeviceToDevice, stream_));
                return TILD_OK;
            }
            const SpectralParams<T> sp = spectral_params();
            if (NP_ == 2)
                generic_spectral<T, 2><<<blocks(M_), 256, 0, stream_>>>(Zxy_, grad_, n_, nz_, sp, partials);
            else
                generic_spectral<T, 1><<<blocks(M_), 256, 0, stream_>>>(Zxy_, grad_, n_, nz_, sp, partials);
            TILD_CUDA(cudaGetLastError());
            return TILD_OK;
        }
        return dispatch_n([&](auto nn) { return this->template zpass_n<decltype(nn)::value>(partials, spec_out, g_only); });
    }

    // what the inverse xy pass produces
    static constexpr int kInvGrad = 0, kInvGradPot = 1, kInvPot = 2;
    template <int NN> tild_status inverse_n(int what) {
        const unsigned nd = what == kInvGrad ? 3 : what == kInvGradPot ? 4 : 1;
        const int d0 = what == kInvPot ? 3 : 0;
        if (use_planes()) {
            if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                with_nt<NN>([&](auto nt) {
                    constexpr int NT = decltype(nt)::value;
                    xy_inverse_plane<T, NN, NT><<<dim3(NN, nd, NP_), NT, plane_smem(), stream_>>>(H_, grad_, tw_, two_pi_L(), d0);
                });
            }
        } else {
            constexpr int CC = 128 / sizeof(V);
            if constexpr (NN >= 16 && NN >= CC) {
                y_columns<T, NN, CC, +1><<<dim3(NN / CC, NN, (what == kInvPot ? 1 : 2) * NP_), 256, ycol_smem(), stream_>>>(
                    H_, tw_, two_pi_L(), what == kInvPot ? 1 : 0);
                x_inverse_rows<T, NN, 16><<<dim3((unsigned)((size_t)NN * NN / 16), nd, NP_), 256, rows_smem(), stream_>>>(
                    H_, grad_, tw_, two_pi_L(), d0);
            }
        }
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    tild_status enqueue_inverse(int what) {
        if (generic_) {
            tild_status st;
            for (int q = 0; q < NP_; ++q) {
                if (what != kInvPot && (st = generic_fft(grad_ + 4 * q * M_, cfg_->dim, +1))) return st;
                if (what != kInvGrad && (st = generic_fft(grad_ + (4 * q + 3) * M_, 1, +1))) return st;
            }
            return TILD_OK;
        }
        return dispatch_n([&](auto nn) { return this->template inverse_n<decltype(nn)::value>(what); });
    }
    // the fields the bead kernel's force needs: ik gradients or the potentials
    int force_fields() const { return analytic() ? kInvPot : kInvGrad; }

    tild_status enqueue_fields(bool energy, double* partials, V* spec_out, int what = -1) {
        if (what < 0) what = force_fields();
        tild_status st;
        if (!have_pos_) {
            err = "positions have not been set";
            return TILD_ESTATE;
        }
        if ((st = enqueue_forward(false))) return st;
        if ((st = enqueue_zpass(energy ? partials : nullptr, spec_out, what == kInvPot))) return st;
        return enqueue_inverse(what);
    }

    // Constants of the integrator update (see BeadParams), from FP64.
    // The update of every scheme in one form (state: positions r and carried
    // velocity u; F = F(r); xi the step's normals):
    //   h = su u + sf F + sg xi,  r' = r + sd h + se xi,  u' = sh h + sk xi,
    // the velocity of a state v = vu u + vf F + vg xi, and u from (r, v):
    // u = wu v + wf F + wg xi.
    struct SchemeCoeffs {
        double su, sf, sg, sd, se, sh, sk, vu, vf, vg, wu, wf, wg;
        int lag;
    };
    static SchemeCoeffs scheme_coeffs(const HostConfig& c) {
        const double dt = c.dt, m = c.mass, al = c.friction, kT = c.kT;
        const double hdm = dt / (2.0 * m);
        SchemeCoeffs k{1, 2 * hdm, 0, dt, 0, 1, 0, 1, hdm, 0, 1, -hdm, 0, 0};
        if (c.scheme == kSchemeGJF) {
            // GJF: a = (1 - alpha dt/2m)/(1 + alpha dt/2m), b = 1/(1 + alpha dt/2m), beta = sigma xi
            const double den = 1.0 + al * hdm, ga = (1.0 - al * hdm) / den, gb = 1.0 / den;
            const double sb = std::sqrt(2.0 * al * kT * dt);
            k.sd = gb * dt;
            k.se = gb * dt * sb / (2.0 * m);
            k.sh = ga;
            k.sk = gb * sb / m;
        } else if (c.scheme == kSchemeEM) {
            // r' = r + (dt/alpha) F + sqrt(2 kT dt/alpha) xi; no velocity
            k.su = 0;
            k.sf = al > 0 ? dt / al : 0;
            k.sg = al > 0 ? std::sqrt(2.0 * kT * dt / al) : 0;
            k.sd = 1;
            k.sh = 0;
            k.vu = k.vf = k.wu = k.wf = 0;
        } else {
            // VV: F = F_c - alpha u + s xi^n (s = sqrt(2 alpha kT/dt)), h = u + (dt/m) F
            const double sv = std::sqrt(2.0 * al * kT / dt), inv = 1.0 / (1.0 - al * hdm);
            k.su = 1.0 - 2.0 * hdm * al;
            k.sg = 2.0 * hdm * sv;
            k.lag = 1;
            k.vu = 1.0 - hdm * al;
            k.vg = hdm * sv;
            k.wu = inv;
            k.wf = -inv * hdm;
            k.wg = -inv * hdm * sv;
        }
        return k;
    }
    static void integrator_constants(const HostConfig& c, BeadParams<T>& p) {
        const SchemeCoeffs k = scheme_coeffs(c);
        p.su = (T)k.su; p.sf = (T)k.sf; p.sg = (T)k.sg; p.sd = (T)k.sd; p.se = (T)k.se; p.sh = (T)k.sh; p.sk = (T)k.sk;
        p.vu = (T)k.vu; p.vf = (T)k.vf; p.vg = (T)k.vg; p.wu = (T)k.wu; p.wf = (T)k.wf; p.wg = (T)k.wg;
        p.noise_lag = k.lag;
    }

    BeadParams<T> bead_params() const {
        BeadParams<T> p;
        const HostConfig& c = *cfg_;
        p.n_beads = c.n_beads;
        p.n = n_;
        p.tiles = tiles_;
        p.L = (T)c.L;
        p.inv_L = (T)(1.0 / c.L);
        p.inv_dx = (T)((double)n_ / c.L);
        p.k_bond = (T)(3.0 / (c.b * c.b));
        integrator_constants(c, p);
        p.sigma_v = (T)std::sqrt(c.kT / c.mass);
        p.mass = (T)c.mass;
        p.seed = c.seed;
        p.topo = c.topo;
        return p;
    }

    BeadBuffers<T> bead_buffers() const {
        BeadBuffers<T> b;
        const size_t N = cfg_->n_beads;
        b.px = pos_[cur_pos_];
        b.py = b.px + N;
        b.pz = b.py + N;
        b.qx = b.qy = b.qz = nullptr;
        b.ux = u_[cur_u_];
        b.uy = b.ux + N;
        b.uz = b.uy + N;
        b.id = id_[cur_id_];
        b.nbr = nbr_;
        b.ext = ext_slots_;
        b.tile_start = tile_start_;
        b.grad = grad_;
        b.rho_fx = rho_fx_;
        b.step = counters_;
        b.err = err_ptr();
        b.f_out = nullptr;
        b.v_out = nullptr;
        b.v_in = nullptr;
        b.partials = partials_;
        return b;
    }

    template <int P, int NS> tild_status bead_pn(int mode, const BeadBuffers<T>& bf) {
        const unsigned grid = (unsigned)tiles_ * tiles_ * tiles_;
        const BeadParams<T> p = bead_params();
        if (analytic() && mode != kModeSpread) {
            const size_t sm = bead_smem(true, NS);
            switch (mode) {
                case kModeForce: bead_kernel<P, kModeForce, T, true, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
                case kModeSetVel: bead_kernel<P, kModeSetVel, T, true, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
                default: bead_kernel<P, kModeStep, T, true, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
            }
        } else {
            const size_t sm = bead_smem(false, NS);
            switch (mode) {
                case kModeSpread: bead_kernel<P, kModeSpread, T, false, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
                case kModeForce: bead_kernel<P, kModeForce, T, false, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
                case kModeSetVel: bead_kernel<P, kModeSetVel, T, false, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
                default: bead_kernel<P, kModeStep, T, false, NS><<<grid, 256, sm, stream_>>>(p, bf); break;
            }
        }
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    template <int P, int D> tild_status bead_generic(int mode, const BeadBuffers<T>& bf) {
        const BeadParams<T> p = bead_params();
        const unsigned g = blocks(cfg_->n_beads);
        switch (mode) {
            case kModeSpread: generic_bead_kernel<P, kModeSpread, T, D><<<g, 256, 0, stream_>>>(p, bf, nz_); break;
            case kModeForce: generic_bead_kernel<P, kModeForce, T, D><<<g, 256, 0, stream_>>>(p, bf, nz_); break;
            case kModeSetVel: generic_bead_kernel<P, kModeSetVel, T, D><<<g, 256, 0, stream_>>>(p, bf, nz_); break;
            default: generic_bead_kernel<P, kModeStep, T, D><<<g, 256, 0, stream_>>>(p, bf, nz_); break;
        }
        TILD_CUDA(cudaGetLastError());
        return TILD_OK;
    }
    template <int P> tild_status bead_p(int mode, const BeadBuffers<T>& bf) {
        if (generic_) return cfg_->dim == 2 ? bead_generic<P, 2>(mode, bf) : bead_generic<P, 3>(mode, bf);
        return NS_ == 4 ? bead_pn<P, 4>(mode, bf) : bead_pn<P, 2>(mode, bf);
    }
    tild_status launch_bead(int mode, const BeadBuffers<T>& bf) {
        return dispatch_p([&](auto pp) { return this->template bead_p<decltype(pp)::value>(mode, bf); });
    }

    tild_status respread() {
        TILD_CUDA(cudaMemsetAsync(rho_fx_, 0, 2 * NP_ * M_ * sizeof(unsigned long long), stream_));
        return launch_bead(kModeSpread, bead_buffers());
    }

    // NVTX range on the host thread for profilers (no cost without one attached)
    struct Range {
        explicit Range(const char* name) { nvtxRangePushA(name); }
        ~Range() { nvtxRangePop(); }
    };

    tild_status enqueue_step() {
        Range range("tild step: forward, z pass, inverse, beads");
        tild_status st;
        if ((st = enqueue_forward(true))) return st;
        if ((st = enqueue_zpass(nullptr, nullptr, analytic()))) return st;
        if ((st = enqueue_inverse(force_fields()))) return st;
        BeadBuffers<T> bf = bead_buffers();
        bf.qx = pos_[1 - cur_pos_];
        bf.qy = bf.qx + cfg_->n_beads;
        bf.qz = bf.qy + cfg_->n_beads;
        if ((st = launch_bead(kModeStep, bf))) return st;
        cur_pos_ = 1 - cur_pos_;
        ++steps_since_sort_;
        return TILD_OK;
    }

    tild_status enqueue_sort(cudaStream_t on = nullptr) {
        Range range("tild re-binning");
        cudaStream_t stream_ = on ? on : this->stream_;  // the batch re-bins on its own stream
        const int N = cfg_->n_beads;
        const size_t N3 = N;
        TILD_CUDA(cudaMemsetAsync(counts_, 0, n_fine_ * sizeof(int), stream_));
        const T* p = pos_[cur_pos_];
        int pw = 0, plo = 0;
        patch_geometry(&pw, &plo);
        bin_count_fine<T><<<blocks(N), 256, 0, stream_>>>(N, p, p + N3, p + 2 * N3, (T)((double)n_ / cfg_->L), n_,
                                                           nz_, tiles_, pw, plo, cfg_->topo, sp_of_id_, id_[cur_id_],
                                                           keys_, ranks_, counts_);
        scan_blocks<<<scan_blocks_, 1024, 0, stream_>>>(counts_, fine_start_, block_sums_, (int)n_fine_);
        scan_top<<<1, 1024, 0, stream_>>>(block_sums_, scan_blocks_);
        scan_add<<<scan_blocks_, 1024, 0, stream_>>>(fine_start_, block_sums_, (int)n_fine_);
        bin_tile_start<<<blocks((size_t)n_tiles_ + 1), 256, 0, stream_>>>(fine_start_, n_tiles_, tile_start_);
        bin_scatter_fine<T><<<blocks(N), 256, 0, stream_>>>(N, cfg_->topo, sp_of_id_, keys_, ranks_, counts_,
                                                             fine_start_, pos_[cur_pos_], pos_[1 - cur_pos_], u_[cur_u_],
                                                             u_[1 - cur_u_], id_[cur_id_], id_[1 - cur_id_], slot_of_id_);
        if (adj_)
            bin_neighbours_explicit<<<blocks(N), 256, 0, stream_>>>(N, id_[1 - cur_id_], slot_of_id_, adj_, ext_ids_,
                                                                    ext_slots_, nbr_);
        else
            bin_neighbours<<<blocks(N), 256, 0, stream_>>>(N, cfg_->topo, id_[1 - cur_id_], slot_of_id_, nbr_);
        TILD_CUDA(cudaGetLastError());
        cur_pos_ = 1 - cur_pos_;
        cur_u_ = 1 - cur_u_;
        cur_id_ = 1 - cur_id_;
        steps_since_sort_ = 0;
        return TILD_OK;
    }

    tild_status run_cycle_graph() {
        Range range("tild re-binning cycles (graph)");
        const int key = cur_pos_ | (cur_u_ << 1) | (cur_id_ << 2);
        tild_status st;
        if (!graph_ || graph_key_ != key) {
            invalidate_graph();
            const int sp = cur_pos_, su = cur_u_, si = cur_id_, ss = steps_since_sort_;
            cudaGraph_t g;
            TILD_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            for (int half = 0; half < 2; ++half) {
                st = enqueue_sort();
                for (int s = 0; !st && s < cfg_->sort_every; ++s) st = enqueue_step();
                if (st) break;
            }
            cudaError_t e = cudaStreamEndCapture(stream_, &g);
            if (st) return st;
            TILD_CUDA(e);
            e = cudaGraphInstantiate(&graph_, g, 0);
            cudaGraphDestroy(g);
            TILD_CUDA(e);
            graph_key_ = key;
            // capture only recorded the launches; restore the host-side state
            cur_pos_ = sp;
            cur_u_ = su;
            cur_id_ = si;
            steps_since_sort_ = ss;
        }
        TILD_CUDA(cudaGraphLaunch(graph_, stream_));
        // two sorts and 2K steps flip every double buffer an even number of
        // times, so the parities are those the graph was captured with
        steps_since_sort_ = cfg_->sort_every;
        return TILD_OK;
    }
};

}  // namespace tild
