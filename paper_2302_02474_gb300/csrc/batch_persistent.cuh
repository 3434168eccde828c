// Persistent form of the batched step: one cooperative launch runs K steps
// of every replica. Each step walks four stages (forward xy pass, z pass,
// inverse xy pass, bead kernel) over a table of work items of all replicas;
// the CTAs, all resident at once (cooperative launch), take items in
// round-robin order and meet at a grid-wide barrier between stages. The
// stage bodies are those of the per-kernel path (same arithmetic, so every
// replica's trajectory is bit-identical to stepping its context alone).
//
// Every barrier wait is bounded: a CTA that has waited longer than the
// plan's limit sets the timeout bit of the status word and returns, and the
// others leave at their next check; the host reads the word and reports
// TILD_ETIMEOUT.
#pragma once

#include "bead_kernels.cuh"
#include "grid_kernels.cuh"

namespace tild {

constexpr unsigned kStatusTimeout = 1u;

template <typename T> struct PersistentPlan {
    const ForwardArgs<T>* fwd;   // [R]
    const ZArgs<T>* z;           // [R]
    const InverseArgs<T>* inv;   // [R]
    const BeadArgs<T>* bead[2];  // [position parity][R]
    const int* n;                // [R] grid points per edge
    const int* start[4];         // [R + 1] first work item of each replica, per stage
    int R;
    unsigned* bar_count;         // barrier arrivals
    unsigned* bar_gen;           // barrier generation
    unsigned* status;            // kStatusTimeout when a wait ran out
    unsigned expected;           // arrivals a barrier waits for (the grid size)
    long long wait_ns;           // limit of one barrier wait
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait; false when a wait ran out here or
// anywhere else (then the caller returns).
template <typename T> __device__ __forceinline__ bool persistent_barrier(const PersistentPlan<T>& pl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = pl.bar_gen;
        volatile unsigned* status = pl.status;
        int ok = 1;
        const unsigned g = *gen;
        __threadfence();  // this CTA's writes before its arrival
        if (atomicAdd(pl.bar_count, 1u) + 1u == pl.expected) {
            atomicExch(pl.bar_count, 0u);
            __threadfence();
            atomicAdd(pl.bar_gen, 1u);
        } else {
            const long long t0 = global_ns();
            while (*gen == g) {
                if (*status) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > pl.wait_ns) {
                    atomicOr(pl.status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(200);
            }
        }
        __threadfence();  // the other CTAs' writes after the barrier
        s_ok = ok && *status == 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// z pass column tile of the persistent kernel (the default tile)
template <typename T> __host__ __device__ constexpr int persistent_zcols(int n) {
    int c = (int)(128 / sizeof(cplx_t<T>));
    while (c > 1 && (n % c) != 0) c /= 2;
    return c < n ? c : n;
}

// One work item. Each (grid size, stage) body is a separate, non-inlined
// function, so that each gets its own register allocation instead of one
// allocation for all twenty bodies at once.
template <typename T, int N, int STAGE>
__device__ __noinline__ void persistent_body(const PersistentPlan<T>& pl, int r, int local, int pp) {
    if constexpr (STAGE == 0) {
        xy_forward_plane_body<T, N, 256>(pl.fwd[r], local);
    } else if constexpr (STAGE == 1) {
        constexpr int C = persistent_zcols<T>(N);
        z_spectral_body<T, N, C>(pl.z[r], local % (N / C), local / (N / C), N / C);
    } else if constexpr (STAGE == 2) {
        xy_inverse_plane_body<T, N, 256>(pl.inv[r], local % N, local / N);
    } else {
        bead_kernel_body<2, kModeStep, T>(pl.bead[pp][r].p, pl.bead[pp][r].bf, local);
    }
}

template <typename T, int N>
__device__ __forceinline__ void persistent_item(int stage, const PersistentPlan<T>& pl, int r, int local, int pp) {
    switch (stage) {
        case 0: persistent_body<T, N, 0>(pl, r, local, pp); break;
        case 1: persistent_body<T, N, 1>(pl, r, local, pp); break;
        case 2: persistent_body<T, N, 2>(pl, r, local, pp); break;
        default: persistent_body<T, N, 3>(pl, r, local, pp); break;
    }
}

// n_steps steps of every replica; the first uses position parity pp0.
// MINB: CTAs per SM the register allocation is made for (2, 3 or 4; the
// batch autotuner picks one).
template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB) batch_persistent(PersistentPlan<T> pl, int n_steps, int pp0) {
    for (int s = 0; s < n_steps; ++s) {
        const int pp = (pp0 + s) & 1;
        for (int stage = 0; stage < 4; ++stage) {
            const int* st = pl.start[stage];
            const int total = st[pl.R];
            int r = 0;
            for (int i = blockIdx.x; i < total; i += gridDim.x) {
                while (st[r + 1] <= i) ++r;  // items are in replica order
                const int local = i - st[r];
                switch (pl.n[r]) {
                    case 24: persistent_item<T, 24>(stage, pl, r, local, pp); break;
                    case 32: persistent_item<T, 32>(stage, pl, r, local, pp); break;
                    case 40: persistent_item<T, 40>(stage, pl, r, local, pp); break;
                    case 48: persistent_item<T, 48>(stage, pl, r, local, pp); break;
                    default: persistent_item<T, 64>(stage, pl, r, local, pp); break;
                }
                __syncthreads();  // the next item reuses the shared memory
            }
            if (!persistent_barrier(pl)) return;
        }
    }
}

// Grid sizes the persistent kernel is compiled for.
__host__ __forceinline__ bool persistent_grid(int n) { return n == 24 || n == 32 || n == 40 || n == 48 || n == 64; }

}  // namespace tild
