// Batched form: many independent TILD systems (replicas with their own
// bead counts, boxes, grids, chi, kappa and seeds) stepped together.
//
// Persistent path (FP32, pmeorder 1, ik force, no charges, two species,
// grids 24, 32, 40, 48 or 64): the K steps between two re-binnings of all
// replicas are one cooperative launch (batch_persistent.cuh) walking a table
// of work items of every replica, stage by stage. Otherwise replicas are
// grouped by (grid size, assignment order) and every step issues four
// launches per group (forward xy, z pass, inverse xy, bead kernel) whose
// blocks look up their replica in device tables of per-replica arguments.
// Re-binning runs per replica. Whole re-binning cycles (re-bin, K steps,
// re-bin, K steps for every replica) are captured once as one CUDA graph and
// replayed. Each replica's results are bit-identical to stepping its context
// alone: the kernels and their arguments are the same.
#pragma once

#include <map>
#include <tuple>
#include <utility>

#include "engine.cuh"
#include "batch_persistent.cuh"

namespace tild {

template <typename T> class BatchEngine final : public BatchBase {
    using V = cplx_t<T>;
    using E = Engine<T>;

    struct Group {
        int n = 0, P = 2, C = 16, tiles3 = 0;
        int nt = 512;      // plane CTA threads (launch shapes of the group's first context)
        bool zalt = false;  // the z pass's alternative column tile
        bool el = false;  // charges on (z pass with the Coulomb term)
        std::vector<E*> reps;
        cudaStream_t s = nullptr;   // the group's stream (forked from the batch stream)
        cudaEvent_t done = nullptr;
        ForwardArgs<T>* d_fwd = nullptr;
        ZArgs<T>* d_z = nullptr;
        InverseArgs<T>* d_inv = nullptr;
        BeadArgs<T>* d_bead[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [pos parity][u, id parity]
    };

   public:
    ~BatchEngine() override {
        if (stream_) cudaStreamSynchronize(stream_);
        if (graph_) cudaGraphExecDestroy(graph_);
        for (void* q : pbufs_) cudaFree(q);
        for (auto& g : groups_) {
            if (g.s) cudaStreamDestroy(g.s);
            if (g.done) cudaEventDestroy(g.done);
            cudaFree(g.d_fwd);
            cudaFree(g.d_z);
            cudaFree(g.d_inv);
            for (auto& row : g.d_bead)
                for (auto* q : row) cudaFree(q);
        }
        for (auto& st : sort_streams_) cudaStreamDestroy(st.first), cudaEventDestroy(st.second);
        if (fork_) cudaEventDestroy(fork_);
        if (stream_) cudaStreamDestroy(stream_);
    }

    tild_status init(const std::vector<EngineBase*>& engines) {
        if (engines.empty()) {
            err = "batch: no replicas";
            return TILD_EINVAL;
        }
        int dev0 = -1;
        for (EngineBase* b : engines) {
            E* e = static_cast<E*>(b);
            if (!e->has_velocities()) {
                err = "batch: every replica needs positions and velocities";
                return TILD_ESTATE;
            }
            if (dev0 < 0) dev0 = e->device_;
            if (e->device_ != dev0) {
                err = "batch: replicas must share one device";
                return TILD_EINVAL;
            }
            if (e->generic_) {
                err = "batch: replicas need the 3D grid sizes of the tiled kernels";
                return TILD_EUNSUPPORTED;
            }
            if (e->NP_ != 1) {
                err = "batch: replicas with more than two species are not batched";
                return TILD_EUNSUPPORTED;
            }
            if (!e->plane_fits_) {
                err = "batch: replica grids must fit the single-plane xy passes";
                return TILD_EUNSUPPORTED;
            }
            reps_.push_back(e);
        }
        K_ = reps_[0]->cfg_->sort_every;
        TILD_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
        tild_status sst = sync_replicas();
        if (sst) return sst;
        // groups by (grid, order, charges on)
        std::map<std::tuple<int, int, bool>, size_t> index;
        for (E* e : reps_) {
            const auto key = std::make_tuple(e->n_, e->P_, e->c_el_on());
            if (!index.count(key)) {
                index[key] = groups_.size();
                Group g;
                g.n = e->n_;
                g.P = e->P_;
                g.el = e->c_el_on();
                g.C = E::zpass_cols(e->n_);
                g.tiles3 = e->n_tiles_;
                g.nt = e->plane_nt_;
                g.zalt = e->zalt_ && !g.el;
                groups_.push_back(g);
            }
            groups_[index[key]].reps.push_back(e);
        }
        for (Group& g : groups_) {
            tild_status st = build_tables(g);
            if (st) return st;
            TILD_CUDA(cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking));
            TILD_CUDA(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
        }
        for (int k = 0; k < kSortStreams; ++k) {
            std::pair<cudaStream_t, cudaEvent_t> st;
            TILD_CUDA(cudaStreamCreateWithFlags(&st.first, cudaStreamNonBlocking));
            TILD_CUDA(cudaEventCreateWithFlags(&st.second, cudaEventDisableTiming));
            sort_streams_.push_back(st);
        }
        TILD_CUDA(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
        tild_status pst = init_persistent();
        if (pst) return pst;
        TILD_CUDA(cudaStreamSynchronize(stream_));
        return TILD_OK;
    }

    // Bring every replica to a common state: work on its stream done,
    // freshly re-binned, current buffers in slot 0.
    tild_status sync_replicas() {
        for (E* e : reps_) {
            TILD_CUDA(cudaStreamSynchronize(e->stream_));
            tild_status st = e->enqueue_sort(stream_);
            if (st) return fail_from(e);
            const size_t N = e->cfg_->n_beads;
            if (e->cur_pos_ != 0) {
                TILD_CUDA(cudaMemcpyAsync(e->pos_[0], e->pos_[1], 3 * N * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
                e->cur_pos_ = 0;
            }
            if (e->cur_u_ != 0) {
                TILD_CUDA(cudaMemcpyAsync(e->u_[0], e->u_[1], 3 * N * sizeof(T), cudaMemcpyDeviceToDevice, stream_));
                TILD_CUDA(cudaMemcpyAsync(e->id_[0], e->id_[1], N * sizeof(int), cudaMemcpyDeviceToDevice, stream_));
                e->cur_u_ = e->cur_id_ = 0;
            }
            e->invalidate_graph();
        }
        cur_pos_ = cur_uid_ = 0;
        steps_since_sort_ = 0;
        invalidate_graph();
        return TILD_OK;
    }

    // Batch autotuner: times whole re-binning cycles of the batch for the
    // persistent kernel (when the replicas allow it) and for the per-group
    // launches at plane thread counts 512, 256, 128 (each group falls back to
    // the largest its grid allows) with the default and the alternative z
    // column tile, from the same saved states, and keeps the fastest. The
    // replicas' states are restored afterwards; results do not depend on the
    // choice. ms (may be NULL) receives 9 timings in candidate order (the
    // persistent kernel compiled for 2, 3 and 4 CTAs per SM, then the group
    // launches; -1 where a candidate is unavailable).
    tild_status autotune(int64_t trial, double* ms, int* choice) override {
        std::vector<void*> saved(reps_.size(), nullptr);
        auto free_saved = [&]() {
            for (void* q : saved) cudaFree(q);
        };
        for (size_t k = 0; k < reps_.size(); ++k) {
            cudaError_t ce = cudaMalloc(&saved[k], reps_[k]->state_bytes());
            if (ce != cudaSuccess) {
                free_saved();
                err = "batch autotune: cannot allocate the replica checkpoints";
                return TILD_ENOMEM;
            }
            tild_status st = reps_[k]->get_state(saved[k], TILD_DEVICE);
            if (st) {
                free_saved();
                return fail_from(reps_[k]);
            }
        }
        struct Cand {
            bool pers;
            int nt;  // plane threads, or the persistent variant
            bool zalt;
        };
        std::vector<Cand> cands = {{true, 0, false}, {true, 1, false}, {true, 2, false}};
        for (int nt : {512, 256, 128})
            for (bool za : {false, true}) cands.push_back({false, nt, za});
        const bool can_persist = p_grids_[0] > 0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        TILD_CUDA(cudaEventCreate(&e0));
        TILD_CUDA(cudaEventCreate(&e1));
        const int64_t n = std::max<int64_t>(2 * K_, ((trial + 2 * K_ - 1) / (2 * K_)) * (2 * K_));
        double best = 1e300;
        int best_i = can_persist ? 0 : 3;
        tild_status st = TILD_OK;
        for (size_t i = 0; i < cands.size() && !st; ++i) {
            if (ms) ms[i] = -1.0;
            if (cands[i].pers && (!can_persist || p_grids_[cands[i].nt] < 1)) continue;
            apply_config(cands[i].pers, cands[i].nt, cands[i].zalt);
            for (size_t k = 0; k < reps_.size() && !st; ++k) st = reps_[k]->set_state(saved[k], TILD_DEVICE);
            if (st || (st = sync_replicas()) || (st = step(2 * K_))) break;
            if (cudaEventRecord(e0, stream_) != cudaSuccess) { st = TILD_EDEVICE; break; }
            if ((st = step(n))) break;
            if (cudaEventRecord(e1, stream_) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = TILD_EDEVICE; break; }
            if ((st = synchronize())) break;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            const double per = t / (double)n;
            if (ms) ms[i] = per;
            if (per < best) {
                best = per;
                best_i = (int)i;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (!st) {
            apply_config(cands[best_i].pers, cands[best_i].nt, cands[best_i].zalt);
            for (size_t k = 0; k < reps_.size() && !st; ++k) st = reps_[k]->set_state(saved[k], TILD_DEVICE);
            if (!st) st = sync_replicas();
        }
        free_saved();
        if (st) return st;
        if (choice) *choice = best_i;
        return TILD_OK;
    }

    // persistent kernel or per-group launches (plane threads nt where a
    // group's grid allows it, else 512; the alternative z tile if zalt)
    void apply_config(bool pers, int nt, bool zalt) {
        persistent_ = pers && p_grids_[0] > 0;
        if (persistent_) {
            p_var_ = nt;
            p_grid_ = p_grids_[nt];
            plan_.expected = (unsigned)(p_grid_ + p_extra_);
            invalidate_graph();
            return;
        }
        for (Group& g : groups_) {
            g.nt = E::plane_nt_allowed(g.n, nt) ? nt : 512;
            g.zalt = zalt && !g.el && E::zpass_cols_alt_n(g.n) != E::zpass_cols_n(g.n);
        }
        invalidate_graph();
    }

    tild_status set_path(bool pers) override {
        if (pers && p_grids_[0] <= 0) {
            err = "batch: these replicas cannot take the persistent kernel";
            return TILD_EUNSUPPORTED;
        }
        persistent_ = pers;
        invalidate_graph();
        return TILD_OK;
    }

    // The time limit of the persistent kernel's barrier waits and, for tests,
    // arrivals the barrier waits for beyond the grid (each extra one makes
    // every wait run out). Returns TILD_EUNSUPPORTED without the persistent path.
    tild_status set_wait(int64_t wait_ns, int extra) override {
        if (!persistent_) {
            err = "batch: these replicas are stepped without the persistent kernel";
            return TILD_EUNSUPPORTED;
        }
        invalidate_graph();
        plan_.wait_ns = wait_ns;
        p_extra_ = extra;
        plan_.expected = (unsigned)(p_grid_ + extra);
        return TILD_OK;
    }
    bool persistent() const override { return persistent_; }

    tild_status step(int64_t n) override {
        tild_status st;
        const int64_t n0 = n;
        while (persistent_ && n > 0) {
            if (steps_since_sort_ >= K_ && n >= 2 * (int64_t)K_ && graph_ok_) {
                if ((st = run_cycle_graph())) return st;
                if (graph_ok_) {  // (else the cycle could not be captured and nothing ran)
                    n -= 2 * (int64_t)K_;
                    continue;
                }
            }
            if (steps_since_sort_ >= K_ && (st = sort_all())) return st;
            const int m = (int)std::min<int64_t>(n, (int64_t)(K_ - steps_since_sort_));
            if ((st = launch_persistent(m))) return st;
            n -= m;
        }
        while (n > 0) {
            if (steps_since_sort_ >= K_ && n >= 2 * (int64_t)K_) {
                if ((st = run_cycle_graph())) return st;
                n -= 2 * (int64_t)K_;
                continue;
            }
            if (steps_since_sort_ >= K_ && (st = sort_all())) return st;
            if ((st = step_all())) return st;
            --n;
        }
        for (E* e : reps_) {
            e->host_step_ += n0;
            e->steps_since_sort_ = steps_since_sort_;
        }
        return TILD_OK;
    }

    tild_status synchronize() override {
        TILD_CUDA(cudaStreamSynchronize(stream_));
        if (persistent_) {
            unsigned h = 0;
            TILD_CUDA(cudaMemcpy(&h, plan_.status, sizeof(h), cudaMemcpyDeviceToHost));
            if (h & kStatusTimeout) {
                TILD_CUDA(cudaMemset(plan_.status, 0, sizeof(unsigned)));
                TILD_CUDA(cudaMemset(plan_.bar_count, 0, sizeof(unsigned)));
                err = "batch: a grid barrier of the persistent kernel waited past its limit; the replicas' states are "
                      "undefined";
                return TILD_ETIMEOUT;
            }
        }
        for (E* e : reps_) {
            const tild_status st = e->check_err();
            if (st) return fail_from(e);
        }
        return TILD_OK;
    }

    int64_t launches(int64_t n) const override {
        int64_t since = steps_since_sort_, sorts = 0;
        for (int64_t s = 0; s < n; ++s) {
            if (since >= K_) {
                ++sorts;
                since = 0;
            }
            ++since;
        }
        if (persistent_) {
            // one launch per run of steps between re-binnings
            int64_t since2 = steps_since_sort_, runs = 0;
            bool open = false;
            for (int64_t s = 0; s < n; ++s) {
                if (since2 >= K_) {
                    since2 = 0;
                    open = false;
                }
                if (!open) {
                    ++runs;
                    open = true;
                }
                ++since2;
            }
            return runs + sorts * 8 * (int64_t)reps_.size();
        }
        return n * 4 * (int64_t)groups_.size() + sorts * 8 * (int64_t)reps_.size();
    }

   private:
    std::vector<E*> reps_;
    std::vector<Group> groups_;
    // persistent path
    bool persistent_ = false, graph_ok_ = true;
    PersistentPlan<T> plan_{};
    const BeadArgs<T>* p_bead_[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [pos parity][u, id parity]
    int p_grid_ = 0;             // CTAs of the chosen variant (0: no persistent path)
    int p_grids_[3] = {0, 0, 0};  // CTAs of the variants for 2, 3, 4 CTAs per SM
    int p_var_ = 0;              // chosen variant
    int p_extra_ = 0;            // arrivals a barrier waits for beyond the grid (tests)
    size_t p_smem_ = 0;
    std::vector<void*> pbufs_;

    void invalidate_graph() {
        if (graph_) cudaGraphExecDestroy(graph_);
        graph_ = nullptr;
    }

    template <class A> tild_status upload_p(const A** dst, const std::vector<A>& v) {
        void* d = nullptr;
        TILD_CUDA(cudaMalloc(&d, std::max<size_t>(1, v.size()) * sizeof(A)));
        pbufs_.push_back(d);
        if (!v.empty()) TILD_CUDA(cudaMemcpy(d, v.data(), v.size() * sizeof(A), cudaMemcpyHostToDevice));
        *dst = (const A*)d;
        return TILD_OK;
    }

    // Work tables and the barrier words of the persistent kernel, when every
    // replica can take it.
    tild_status init_persistent() {
        if (sizeof(T) != 4) return TILD_OK;
        for (E* e : reps_)
            if (e->P_ != 2 || e->c_el_on() || e->analytic() || e->NP_ != 1 || e->generic_ || !e->plane_fits_ ||
                !persistent_grid(e->n_))
                return TILD_OK;
        std::vector<E*> order(reps_);
        std::stable_sort(order.begin(), order.end(), [](E* a, E* b) { return a->n_ < b->n_; });
        const int R = (int)order.size();
        std::vector<ForwardArgs<T>> f;
        std::vector<ZArgs<T>> z;
        std::vector<InverseArgs<T>> inv;
        std::vector<int> nn;
        std::vector<int> start[4];
        for (auto& s : start) s.push_back(0);
        for (E* e : order) {
            f.push_back(ForwardArgs<T>{e->rho_fx_, e->Zxy_, e->tw_, e->density_scale(), 1, e->counters_});
            if (e->refresh_tables()) return fail_from(e);
            z.push_back(ZArgs<T>{e->Zxy_, e->H_, e->tw_, e->spectral_params(), nullptr, nullptr});
            inv.push_back(InverseArgs<T>{e->H_, e->grad_, e->tw_, e->two_pi_L(), 0});
            const int n = e->n_, C = persistent_zcols<T>(n);
            nn.push_back(n);
            start[0].push_back(start[0].back() + n);
            start[1].push_back(start[1].back() + (n / C) * (n / 2 + 1));
            start[2].push_back(start[2].back() + 3 * n);
            start[3].push_back(start[3].back() + e->n_tiles_);
        }
        tild_status st;
        if ((st = upload_p(&plan_.fwd, f)) || (st = upload_p(&plan_.z, z)) || (st = upload_p(&plan_.inv, inv)) ||
            (st = upload_p(&plan_.n, nn)))
            return st;
        for (int s = 0; s < 4; ++s)
            if ((st = upload_p(&plan_.start[s], start[s]))) return st;
        for (int pp = 0; pp < 2; ++pp)
            for (int q = 0; q < 2; ++q) {
                std::vector<BeadArgs<T>> bv;
                for (E* e : order) {
                    const size_t N = e->cfg_->n_beads;
                    BeadArgs<T> a;
                    a.p = e->bead_params();
                    a.bf = e->bead_buffers();
                    a.bf.px = e->pos_[pp];
                    a.bf.py = a.bf.px + N;
                    a.bf.pz = a.bf.py + N;
                    a.bf.qx = e->pos_[1 - pp];
                    a.bf.qy = a.bf.qx + N;
                    a.bf.qz = a.bf.qy + N;
                    a.bf.ux = e->u_[q];
                    a.bf.uy = a.bf.ux + N;
                    a.bf.uz = a.bf.uy + N;
                    a.bf.id = e->id_[q];
                    bv.push_back(a);
                }
                if ((st = upload_p(&p_bead_[pp][q], bv))) return st;
            }
        void* words = nullptr;
        TILD_CUDA(cudaMalloc(&words, 4 * sizeof(unsigned)));
        pbufs_.push_back(words);
        TILD_CUDA(cudaMemset(words, 0, 4 * sizeof(unsigned)));
        plan_.bar_count = (unsigned*)words;
        plan_.bar_gen = plan_.bar_count + 1;
        plan_.status = plan_.bar_count + 2;
        plan_.R = R;
        // shared memory: the largest stage body (bead tile, plane or z tile of 64^3)
        const size_t plane64 = (64 + 64 * 65) * sizeof(V);
        const size_t z64 = (64 + 4 * 64 * persistent_zcols<T>(64)) * sizeof(V);
        p_smem_ = std::max(bead_smem_bytes<2, T>(), std::max(plane64, z64));
        int sms = 0, dev = 0;
        TILD_CUDA(cudaGetDevice(&dev));
        TILD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int per_sm[3] = {0, 0, 0};
        TILD_CUDA(cudaFuncSetAttribute(batch_persistent<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem_));
        TILD_CUDA(cudaFuncSetAttribute(batch_persistent<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem_));
        TILD_CUDA(cudaFuncSetAttribute(batch_persistent<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p_smem_));
        TILD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], batch_persistent<T, 2>, 256, p_smem_));
        TILD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], batch_persistent<T, 3>, 256, p_smem_));
        TILD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], batch_persistent<T, 4>, 256, p_smem_));
        for (int v = 0; v < 3; ++v) p_grids_[v] = per_sm[v] * sms;
        if (per_sm[0] < 1) return TILD_OK;  // cannot be resident: keep the per-kernel path
        // the variant with the most resident CTAs until the autotuner says otherwise
        p_var_ = per_sm[2] >= 1 ? 2 : per_sm[1] >= 1 ? 1 : 0;
        p_grid_ = p_grids_[p_var_];
        plan_.expected = (unsigned)p_grid_;
        plan_.wait_ns = 2000000000ll;  // 2 s
        persistent_ = true;
        return TILD_OK;
    }

    // m steps of every replica in one cooperative launch
    tild_status launch_persistent(int m) {
        PersistentPlan<T> pl = plan_;
        pl.bead[0] = p_bead_[0][cur_uid_];
        pl.bead[1] = p_bead_[1][cur_uid_];
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)p_grid_);
        lc.blockDim = dim3(256);
        lc.dynamicSmemBytes = p_smem_;
        lc.stream = stream_;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        if (p_var_ == 2)
            TILD_CUDA(cudaLaunchKernelEx(&lc, batch_persistent<T, 4>, pl, m, cur_pos_));
        else if (p_var_ == 1)
            TILD_CUDA(cudaLaunchKernelEx(&lc, batch_persistent<T, 3>, pl, m, cur_pos_));
        else
            TILD_CUDA(cudaLaunchKernelEx(&lc, batch_persistent<T, 2>, pl, m, cur_pos_));
        if (m & 1) {
            cur_pos_ ^= 1;
            for (E* e : reps_) e->cur_pos_ ^= 1;
        }
        steps_since_sort_ += m;
        return TILD_OK;
    }
    cudaStream_t stream_ = nullptr;
    int K_ = 20;
    int cur_pos_ = 0, cur_uid_ = 0, steps_since_sort_ = 0;
    cudaGraphExec_t graph_ = nullptr;
    static constexpr int kSortStreams = 16;
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> sort_streams_;
    cudaEvent_t fork_ = nullptr;

    // fork: every group stream waits for the batch stream
    tild_status fork_groups() {
        TILD_CUDA(cudaEventRecord(fork_, stream_));
        for (Group& g : groups_) TILD_CUDA(cudaStreamWaitEvent(g.s, fork_, 0));
        return TILD_OK;
    }
    // join: the batch stream waits for every group stream
    tild_status join_groups() {
        for (Group& g : groups_) {
            TILD_CUDA(cudaEventRecord(g.done, g.s));
            TILD_CUDA(cudaStreamWaitEvent(stream_, g.done, 0));
        }
        return TILD_OK;
    }

    tild_status fail_from(E* e) {
        err = e->err;
        return TILD_EDEVICE;
    }

    template <class A> tild_status upload(A** dst, const std::vector<A>& v) {
        TILD_CUDA(cudaMalloc(dst, v.size() * sizeof(A)));
        TILD_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(A), cudaMemcpyHostToDevice));
        return TILD_OK;
    }

    tild_status build_tables(Group& g) {
        std::vector<ForwardArgs<T>> f;
        std::vector<ZArgs<T>> z;
        std::vector<InverseArgs<T>> inv;
        for (E* e : g.reps) {
            f.push_back(ForwardArgs<T>{e->rho_fx_, e->Zxy_, e->tw_, e->density_scale(), 1, e->counters_});
            // the z pass needs the kernel tables of the replica's current a (and a_e)
            if (e->refresh_tables()) return fail_from(e);
            z.push_back(ZArgs<T>{e->Zxy_, e->H_, e->tw_, e->spectral_params(), nullptr, nullptr});
            inv.push_back(InverseArgs<T>{e->H_, e->grad_, e->tw_, e->two_pi_L(), 0});
        }
        tild_status st;
        if ((st = upload(&g.d_fwd, f)) || (st = upload(&g.d_z, z)) || (st = upload(&g.d_inv, inv))) return st;
        for (int pp = 0; pp < 2; ++pp)
            for (int q = 0; q < 2; ++q) {
                std::vector<BeadArgs<T>> b;
                for (E* e : g.reps) {
                    const size_t N = e->cfg_->n_beads;
                    BeadArgs<T> a;
                    a.p = e->bead_params();
                    a.bf = e->bead_buffers();
                    a.bf.px = e->pos_[pp];
                    a.bf.py = a.bf.px + N;
                    a.bf.pz = a.bf.py + N;
                    a.bf.qx = e->pos_[1 - pp];
                    a.bf.qy = a.bf.qx + N;
                    a.bf.qz = a.bf.qy + N;
                    a.bf.ux = e->u_[q];
                    a.bf.uy = a.bf.ux + N;
                    a.bf.uz = a.bf.uy + N;
                    a.bf.id = e->id_[q];
                    b.push_back(a);
                }
                if ((st = upload(&g.d_bead[pp][q], b))) return st;
            }
        // kernel attributes (same dynamic shared memory as the single path)
        E* e0 = g.reps[0];
        return dispatch_group(g, [&](auto nn, auto pp) -> tild_status {
            constexpr int NN = decltype(nn)::value, PP = decltype(pp)::value;
            if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                constexpr int CC = E::zpass_cols(NN);
                constexpr int CA = E::zpass_cols_alt(NN);
                TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane_batched<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)e0->plane_smem()));
                TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane_batched<T, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)e0->plane_smem()));
                if constexpr (E::plane_nt_ok(NN, 256)) {
                    TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane_batched<T, NN, 256>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->plane_smem()));
                    TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane_batched<T, NN, 256>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->plane_smem()));
                }
                if constexpr (E::plane_nt_ok(NN, 128)) {
                    TILD_CUDA(cudaFuncSetAttribute(xy_forward_plane_batched<T, NN, 128>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->plane_smem()));
                    TILD_CUDA(cudaFuncSetAttribute(xy_inverse_plane_batched<T, NN, 128>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->plane_smem()));
                }
                if constexpr (CA != CC)
                    TILD_CUDA(cudaFuncSetAttribute(z_spectral_batched<T, NN, CA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)e0->zpass_smem_cols(CA)));
                TILD_CUDA(cudaFuncSetAttribute(z_spectral_batched<T, NN, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)e0->zpass_smem()));
                TILD_CUDA(cudaFuncSetAttribute(z_spectral_batched<T, NN, CC, true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->zpass_smem()));
                TILD_CUDA(cudaFuncSetAttribute(bead_kernel_batched<PP, kModeStep, T>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e0->bead_smem()));
            }
            return TILD_OK;
        });
    }

    template <int V_> struct ic {
        static constexpr int value = V_;
    };
    template <int NN, class F> void with_group_nt(const Group& g, F&& f) {
        if constexpr (E::plane_nt_ok(NN, 128))
            if (g.nt == 128) return f(ic<128>{});
        if constexpr (E::plane_nt_ok(NN, 256))
            if (g.nt == 256) return f(ic<256>{});
        return f(ic<512>{});
    }

    template <class F> tild_status dispatch_p(int P, F&& f) {
        switch (P) {
            case 2: return f(ic<2>{});
            case 3: return f(ic<3>{});
            case 4: return f(ic<4>{});
            default: return f(ic<5>{});
        }
    }

    template <class F> tild_status dispatch_group(const Group& g, F&& f) {
        auto with_n = [&](auto nn) { return dispatch_p(g.P, [&](auto pp) { return f(nn, pp); }); };
        switch (g.n) {
            case 8: return with_n(ic<8>{});
            case 16: return with_n(ic<16>{});
            case 24: return with_n(ic<24>{});
            case 32: return with_n(ic<32>{});
            case 40: return with_n(ic<40>{});
            case 48: return with_n(ic<48>{});
            case 64: return with_n(ic<64>{});
            case 80: return with_n(ic<80>{});
            case 128: return with_n(ic<128>{});
        }
        err = "batch: unsupported replica grid";
        return TILD_EUNSUPPORTED;
    }

    // one step of every group, each on its own stream (after fork_groups)
    tild_status step_groups() {
        for (Group& g : groups_) {
            const unsigned R = (unsigned)g.reps.size();
            E* e0 = g.reps[0];
            tild_status st = dispatch_group(g, [&](auto nn, auto pp) -> tild_status {
                constexpr int NN = decltype(nn)::value, PP = decltype(pp)::value;
                if constexpr ((size_t)NN * (NN + 1) * sizeof(V) <= 200 * 1024) {
                    constexpr int CC = E::zpass_cols(NN);
                    constexpr int CA = E::zpass_cols_alt(NN);
                    with_group_nt<NN>(g, [&](auto nt) {
                        constexpr int NT = decltype(nt)::value;
                        xy_forward_plane_batched<T, NN, NT><<<dim3(NN, R), NT, e0->plane_smem(), g.s>>>(g.d_fwd);
                    });
                    if (g.el)
                        z_spectral_batched<T, NN, CC, true><<<dim3(NN / CC, NN / 2 + 1, R), 256, e0->zpass_smem(), g.s>>>(g.d_z);
                    else if (g.zalt)
                        z_spectral_batched<T, NN, CA><<<dim3(NN / CA, NN / 2 + 1, R), 256, e0->zpass_smem_cols(CA), g.s>>>(g.d_z);
                    else
                        z_spectral_batched<T, NN, CC><<<dim3(NN / CC, NN / 2 + 1, R), 256, e0->zpass_smem(), g.s>>>(g.d_z);
                    with_group_nt<NN>(g, [&](auto nt) {
                        constexpr int NT = decltype(nt)::value;
                        xy_inverse_plane_batched<T, NN, NT><<<dim3(NN, 3, R), NT, e0->plane_smem(), g.s>>>(g.d_inv);
                    });
                    bead_kernel_batched<PP, kModeStep, T><<<(unsigned)g.tiles3 * R, 256, e0->bead_smem(), g.s>>>(
                        g.d_bead[cur_pos_][cur_uid_], g.tiles3);
                }
                return TILD_OK;
            });
            if (st) return st;
        }
        TILD_CUDA(cudaGetLastError());
        cur_pos_ ^= 1;
        for (E* e : reps_) e->cur_pos_ ^= 1;
        ++steps_since_sort_;
        return TILD_OK;
    }

    tild_status step_all() {
        tild_status st;
        if ((st = fork_groups()) || (st = step_groups())) return st;
        return join_groups();
    }

    // re-bin every replica, spread over a pool of streams (forked from and
    // joined back into the batch stream)
    tild_status sort_all() {
        TILD_CUDA(cudaEventRecord(fork_, stream_));
        for (auto& ss : sort_streams_) TILD_CUDA(cudaStreamWaitEvent(ss.first, fork_, 0));
        for (size_t k = 0; k < reps_.size(); ++k) {
            E* e = reps_[k];
            if (e->enqueue_sort(sort_streams_[k % sort_streams_.size()].first)) return fail_from(e);
        }
        for (auto& ss : sort_streams_) {
            TILD_CUDA(cudaEventRecord(ss.second, ss.first));
            TILD_CUDA(cudaStreamWaitEvent(stream_, ss.second, 0));
        }
        cur_pos_ ^= 1;
        cur_uid_ ^= 1;
        steps_since_sort_ = 0;
        return TILD_OK;
    }

    tild_status run_cycle_graph() {
        if (!graph_) {
            // host-side parities return to their values after a full cycle
            struct Snap {
                int p, u, i, s;
            };
            std::vector<Snap> snap;
            for (E* e : reps_) snap.push_back({e->cur_pos_, e->cur_u_, e->cur_id_, e->steps_since_sort_});
            const int bp = cur_pos_, bu = cur_uid_, bs = steps_since_sort_;
            cudaGraph_t g;
            TILD_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            tild_status st = TILD_OK;
            for (int half = 0; half < 2 && !st; ++half) {
                st = sort_all();
                if (persistent_) {
                    if (!st) st = launch_persistent(K_);
                    continue;
                }
                if (!st) st = fork_groups();
                for (int s = 0; s < K_ && !st; ++s) st = step_groups();
                if (!st) st = join_groups();
            }
            cudaError_t e = cudaStreamEndCapture(stream_, &g);
            if (persistent_ && (st || e != cudaSuccess)) {
                // a cooperative launch that cannot be captured: run cycles
                // without a graph from now on
                cudaGetLastError();
                if (e == cudaSuccess) cudaGraphDestroy(g);
                graph_ok_ = false;
                for (size_t k = 0; k < reps_.size(); ++k) {
                    reps_[k]->cur_pos_ = snap[k].p;
                    reps_[k]->cur_u_ = snap[k].u;
                    reps_[k]->cur_id_ = snap[k].i;
                    reps_[k]->steps_since_sort_ = snap[k].s;
                }
                cur_pos_ = bp;
                cur_uid_ = bu;
                steps_since_sort_ = bs;
                return TILD_OK;
            }
            if (st) return st;
            TILD_CUDA(e);
            e = cudaGraphInstantiate(&graph_, g, 0);
            cudaGraphDestroy(g);
            if (persistent_ && e != cudaSuccess) {
                cudaGetLastError();
                graph_ = nullptr;
                graph_ok_ = false;
                for (size_t k = 0; k < reps_.size(); ++k) {
                    reps_[k]->cur_pos_ = snap[k].p;
                    reps_[k]->cur_u_ = snap[k].u;
                    reps_[k]->cur_id_ = snap[k].i;
                    reps_[k]->steps_since_sort_ = snap[k].s;
                }
                cur_pos_ = bp;
                cur_uid_ = bu;
                steps_since_sort_ = bs;
                return TILD_OK;
            }
            TILD_CUDA(e);
            for (size_t k = 0; k < reps_.size(); ++k) {
                reps_[k]->cur_pos_ = snap[k].p;
                reps_[k]->cur_u_ = snap[k].u;
                reps_[k]->cur_id_ = snap[k].i;
                reps_[k]->steps_since_sort_ = snap[k].s;
            }
            cur_pos_ = bp;
            cur_uid_ = bu;
            steps_since_sort_ = bs;
        }
        TILD_CUDA(cudaGraphLaunch(graph_, stream_));
        steps_since_sort_ = K_;
        return TILD_OK;
    }
};

template <typename T> BatchBase* make_batch(const std::vector<EngineBase*>& engines, std::string& err) {
    BatchEngine<T>* b = new BatchEngine<T>();
    if (b->init(engines) != TILD_OK) {
        err = b->err;
        delete b;
        return nullptr;
    }
    return b;
}

}  // namespace tild
