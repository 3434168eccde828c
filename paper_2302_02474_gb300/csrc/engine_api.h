// Interface between the C ABI layer and the per-precision engines.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "tild.h"
#include "common.cuh"

namespace tild {

// Everything the ABI layer validates and the engines read.
struct HostConfig {
    double L;
    int n;
    int dim = 3;         // 2: a square box and n x n grid (Listing infile's "Dim 2")
    bool generic = false;  // grid served by the any-size kernels (odd sizes, D = 2)
    int pmeorder;
    int precision;
    uint64_t seed;
    int sort_every;
    // chains
    Topology topo;
    int n_beads = 0;
    double b = 1.0;
    // species (1..4) and, when set explicitly, the species of every bead;
    // bonds: empty = the chains' linear bonds, else an explicit list of
    // bead-id pairs (tild_set_bonds)
    int n_species = 2;
    std::vector<unsigned char> species_of_bead;
    bool explicit_bonds = false;
    std::vector<int> bond_pairs;  // [n_bonds][2]
    // interactions; chi_mat[K][K'] is the Flory matrix (chi = chi_mat[0][1])
    double chi = 0.0, kappa = 0.0, a = 0.5;
    double chi_mat[4][4] = {{0}};
    bool have_interactions = false;
    // integrator
    double dt = 0.005, friction = 1.0, kT = 1.0, mass = 1.0;
    int scheme = 0;  // TILD_SCHEME_*
    int force_method = 0;  // TILD_FORCE_*
    // electrostatics: charge per species, Bjerrum length (0: off), charge spreading length
    double q_a = 0.0, q_b = 0.0, bjerrum = 0.0, charge_smear = 0.5;
    // device memory: the caller's allocator (tild_create_with_allocator) or cudaMalloc
    tild_allocator allocator = {nullptr, nullptr, nullptr};
};

class EngineBase {
   public:
    virtual ~EngineBase() {}
    std::string err;
    virtual tild_status init(HostConfig* cfg) = 0;
    virtual tild_status set_chains() = 0;
    // species count / per-bead species / bond list of the HostConfig changed
    virtual tild_status set_topology() = 0;
    virtual tild_status set_stream(cudaStream_t s) = 0;
    virtual cudaStream_t stream() const = 0;
    virtual tild_status set_positions(const void* xyz, int dtype, int where) = 0;
    virtual tild_status set_velocities(const void* v, int dtype, int where) = 0;  // v == NULL: Maxwell-Boltzmann
    virtual tild_status step(int64_t n) = 0;
    virtual tild_status synchronize() = 0;
    virtual tild_status compute(unsigned what, tild_energy* e, void* f, int dtype, int where) = 0;
    virtual tild_status energy_gradient(tild_energy_grad* g, void* dUdr, int dtype, int where) = 0;
    virtual tild_status get_positions(void* out, int dtype, int where) = 0;
    virtual tild_status get_velocities(void* out, int dtype, int where) = 0;
    virtual tild_status get_density(void* out, int dtype, int where) = 0;
    virtual tild_status get_spectrum(void* out, int dtype, int where) = 0;
    virtual tild_status get_field_gradient(void* out, int dtype, int where) = 0;
    virtual int64_t host_step() const = 0;
    virtual size_t state_bytes() const = 0;
    virtual tild_status get_state(void* blob, int where) = 0;
    virtual tild_status set_state(const void* blob, int where) = 0;
    virtual tild_status profile(int n, double* ms) = 0;
    virtual int64_t launches(int64_t n) const = 0;
    virtual bool has_positions() const = 0;
    virtual bool has_velocities() const = 0;
    // Parameter changes: keep v^n while F^n changes (u = v - dt/2m F).
    virtual tild_status force_vjp(const void* lam, void* out, int dtype, int where, double* dtheta) = 0;
    virtual tild_status density_vjp(const void* psi, void* out, int dtype, int where) = 0;
    virtual tild_status trajectory_vjp(int64_t K, int C, const void* rbar, const void* vbar, int dtype, int where,
                                       void* r0, void* v0, double* dtheta) = 0;
    virtual tild_status save_velocities() = 0;
    virtual tild_status restore_velocities() = 0;
    virtual void params_changed() = 0;
    virtual void launch_shapes(int* plane_threads, int* z_cols, int* z_default, int* z_alt) const = 0;
    virtual tild_status set_launch_shapes(int plane_threads, int z_cols) = 0;
    // per-bead vector arrays in the other layout: a device scratch of the
    // context and an [n][3] <-> [3][n] transpose on its stream (synchronised)
    virtual tild_status io_scratch(size_t bytes, void** ptr) = 0;
    virtual tild_status transpose3(const void* in, void* out, size_t n, int dtype, bool to_aos) = 0;
};

// Several contexts stepped together (batched form).
class BatchBase {
   public:
    virtual ~BatchBase() {}
    std::string err;
    virtual tild_status step(int64_t n) = 0;
    virtual tild_status synchronize() = 0;
    virtual int64_t launches(int64_t n) const = 0;
    virtual tild_status set_wait(int64_t wait_ns, int extra) = 0;
    virtual tild_status autotune(int64_t trial, double* ms, int* choice) = 0;
    virtual tild_status set_path(bool persistent) = 0;
    virtual bool persistent() const = 0;
};

// Error text returned by tild_last_error(NULL).
void set_global_error(const std::string& msg);

EngineBase* make_engine_f32();
EngineBase* make_engine_f64();
// Engines must all be of the factory's precision, with positions and
// velocities set; on failure returns nullptr and sets err.
BatchBase* make_batch_f32(const std::vector<EngineBase*>& engines, std::string& err);
BatchBase* make_batch_f64(const std::vector<EngineBase*>& engines, std::string& err);

}  // namespace tild
