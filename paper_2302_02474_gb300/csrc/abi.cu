// extern "C" boundary of the TILD engine: argument validation, error text,
// and dispatch to the FP32 or FP64 engine.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include <memory>
#include <string>

#include "engine_api.h"

using namespace tild;

struct tild_ctx {
    HostConfig cfg;
    std::unique_ptr<EngineBase> eng;
    bool have_chains = false;
    int layout = TILD_LAYOUT_AOS;
    std::string err;
};

struct tild_batch {
    std::unique_ptr<BatchBase> b;
};

namespace {

std::string g_create_error = "no error";

tild_status fail(tild_ctx* c, tild_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

tild_status from_engine(tild_ctx* c, tild_status st) {
    if (st != TILD_OK) c->err = c->eng->err.empty() ? "engine error" : c->eng->err;
    return st;
}

// Grid sizes with a hand-written FFT: powers of two 8..256 and 24, 40, 48, 80.
bool supported_n(int n) {
    if (n >= 8 && n <= 256 && (n & (n - 1)) == 0) return true;
    return n == 24 || n == 40 || n == 48 || n == 80;
}

bool valid_io(int dtype, int where) {
    return (dtype == TILD_DTYPE_F32 || dtype == TILD_DTYPE_F64) && (where == TILD_HOST || where == TILD_DEVICE);
}

template <typename TV> void host_transpose3(const TV* in, TV* out, size_t n, bool to_aos) {
    for (size_t i = 0; i < n; ++i)
        for (size_t d = 0; d < 3; ++d) {
            if (to_aos)
                out[3 * i + d] = in[d * n + i];
            else
                out[d * n + i] = in[3 * i + d];
        }
}

// Per-bead vector arrays of one call in the context's layout: SoA arrays are
// transposed to the AoS arrays the engine reads and writes (host arrays on
// the host, device arrays through slots of the context's device scratch).
struct LayoutIO {
    tild_ctx* c;
    int dtype, where;
    size_t n;
    std::vector<std::vector<unsigned char>> host;
    unsigned char* dev = nullptr;
    tild_status st = TILD_OK;
    LayoutIO(tild_ctx* ctx, int dt, int wh, int slots)
        : c(ctx), dtype(dt), where(wh), n((size_t)ctx->cfg.n_beads), host(slots) {
        if (soa() && where == TILD_DEVICE) {
            void* p = nullptr;
            st = c->eng->io_scratch(slots * bytes(), &p);
            dev = (unsigned char*)p;
            if (st) c->err = c->eng->err;
        }
    }
    bool soa() const { return c->layout == TILD_LAYOUT_SOA; }
    size_t bytes() const { return 3 * n * (dtype == TILD_DTYPE_F32 ? 4 : 8); }
    void transpose(const void* in, void* out, bool to_aos) {
        if (where == TILD_HOST) {
            if (dtype == TILD_DTYPE_F32)
                host_transpose3((const float*)in, (float*)out, n, to_aos);
            else
                host_transpose3((const double*)in, (double*)out, n, to_aos);
        } else if (!st) {
            st = c->eng->transpose3(in, out, n, dtype, to_aos);
            if (st) c->err = c->eng->err;
        }
    }
    void* slot(int k) {
        if (where == TILD_HOST) {
            host[k].resize(bytes());
            return host[k].data();
        }
        return dev + k * bytes();
    }
    // an input array -> the AoS pointer for the engine
    const void* in(const void* p, int k) {
        if (!soa() || !p || st) return p;
        void* a = slot(k);
        transpose(p, a, true);
        return a;
    }
    // an output array -> the AoS buffer the engine writes (then done())
    void* out(void* p, int k) { return (!soa() || !p || st) ? p : slot(k); }
    void done(void* p, int k) {
        if (soa() && p && !st) transpose(slot(k), p, false);
    }
};

}  // namespace

void tild::set_global_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

static tild_status create_ctx(const tild_params* p, const tild_allocator* a, tild_ctx** out);

tild_status tild_create(const tild_params* p, tild_ctx** out) { return create_ctx(p, nullptr, out); }

tild_status tild_create_with_allocator(const tild_params* p, const tild_allocator* a, tild_ctx** out) {
    if (a && a->alloc && !a->free) {
        g_create_error = "tild_create_with_allocator: an allocator needs both alloc and free";
        return TILD_EINVAL;
    }
    return create_ctx(p, a, out);
}

static tild_status create_ctx(const tild_params* p, const tild_allocator* a, tild_ctx** out) {
    if (!p || !out) {
        g_create_error = "tild_create: NULL argument";
        return TILD_EINVAL;
    }
    *out = nullptr;
    const bool two_d = p->n[2] == 1;  // Listing infile's "Dim 2": an n x n grid, z unused
    if (!(p->L[0] > 0) || p->L[0] != p->L[1] || (!two_d && p->L[0] != p->L[2]) || !std::isfinite(p->L[0])) {
        g_create_error = two_d ? "tild_create: a 2D box must be square with L > 0" : "tild_create: the box must be cubic with L > 0";
        return TILD_EUNSUPPORTED;
    }
    const int n = p->n[0];
    const bool fast = !two_d && p->n[1] == n && p->n[2] == n && supported_n(n) && (p->precision != TILD_FP64 || n <= 128);
    const int n_max = two_d ? 2048 : (p->precision == TILD_FP64 ? 128 : 256);
    if (p->n[1] != n || (!two_d && p->n[2] != n) || n < 4 || n > n_max) {
        g_create_error = two_d ? "tild_create: a 2D grid is n x n x 1 with 4 <= n <= 2048"
                               : "tild_create: the grid must be cubic with 4 <= n <= 256 (FP64: 128)";
        return TILD_EUNSUPPORTED;
    }
    if (p->pmeorder < 1 || p->pmeorder > 4) {
        g_create_error = "tild_create: pmeorder must be in 1..4";
        return TILD_EINVAL;
    }
    if (p->precision != TILD_FP32 && p->precision != TILD_FP64) {
        g_create_error = "tild_create: precision must be TILD_FP32 or TILD_FP64";
        return TILD_EINVAL;
    }

    if (p->sort_every < 0) {
        g_create_error = "tild_create: sort_every must be >= 0";
        return TILD_EINVAL;
    }
    std::unique_ptr<tild_ctx> c(new tild_ctx());
    c->cfg.L = p->L[0];
    c->cfg.n = p->n[0];
    c->cfg.dim = two_d ? 2 : 3;
    c->cfg.generic = !fast;
    c->cfg.pmeorder = p->pmeorder;
    c->cfg.precision = p->precision;
    c->cfg.seed = p->seed;
    c->cfg.sort_every = p->sort_every == 0 ? 20 : p->sort_every;
    std::memset(&c->cfg.topo, 0, sizeof(c->cfg.topo));
    if (a && a->alloc) c->cfg.allocator = *a;
    c->eng.reset(p->precision == TILD_FP32 ? make_engine_f32() : make_engine_f64());
    const tild_status st = c->eng->init(&c->cfg);
    if (st != TILD_OK) {
        g_create_error = "tild_create: " + c->eng->err;
        return st;
    }
    *out = c.release();
    return TILD_OK;
}

tild_status tild_destroy(tild_ctx* ctx) {
    delete ctx;
    return TILD_OK;
}

tild_status tild_set_chains(tild_ctx* c, int n_types, const tild_moltype* t, double b) {
    if (!c) return TILD_EINVAL;
    if (!t || n_types < 1 || n_types > kMaxTypes) return fail(c, TILD_EINVAL, "set_chains: 1..8 molecule types required");
    if (!(b > 0) || !std::isfinite(b)) return fail(c, TILD_EINVAL, "set_chains: b must be > 0");
    Topology topo;
    std::memset(&topo, 0, sizeof(topo));
    int64_t total = 0;
    for (int k = 0; k < n_types; ++k) {
        if (t[k].n_chains < 0 || t[k].N < 1 || t[k].n_a < 0 || t[k].n_a > t[k].N)
            return fail(c, TILD_EINVAL, "set_chains: need n_chains >= 0, N >= 1, 0 <= n_a <= N");
        topo.start[k] = (int)total;
        topo.N[k] = t[k].N;
        topo.n_a[k] = t[k].n_a;
        total += t[k].n_chains * (int64_t)t[k].N;
        if (total >= (int64_t)1 << 29) return fail(c, TILD_EUNSUPPORTED, "set_chains: at most 2^29-1 beads");
    }
    if (total < 1) return fail(c, TILD_EINVAL, "set_chains: no beads");
    topo.start[n_types] = (int)total;
    topo.n_types = n_types;
    c->cfg.topo = topo;
    c->cfg.n_beads = (int)total;
    c->cfg.b = b;
    c->cfg.n_species = 2;  // the chains' A/B pattern and linear bonds
    c->cfg.species_of_bead.clear();
    c->cfg.explicit_bonds = false;
    c->cfg.bond_pairs.clear();
    const tild_status st = c->eng->set_chains();
    if (st) return from_engine(c, st);
    c->have_chains = true;
    return TILD_OK;
}

// Parameter limits of the integrator schemes (NULL: acceptable).
static const char* scheme_limits(const HostConfig& h) {
    if (h.scheme == TILD_SCHEME_EM && !(h.friction > 0)) return "Euler-Maruyama needs friction > 0";
    if (h.scheme == TILD_SCHEME_VV && !(h.friction * h.dt / (2.0 * h.mass) < 1.0))
        return "velocity-Verlet with the Langevin force needs friction * dt / (2 mass) < 1";
    return nullptr;
}

static tild_status reparam(tild_ctx* c, const HostConfig& next) {
    // keep v^n = u^n + (dt/2m) F^n across the change
    const bool keep = c->eng->has_velocities();
    tild_status st;
    if (keep && (st = c->eng->save_velocities())) return from_engine(c, st);
    c->cfg = next;
    c->eng->params_changed();
    if (keep && (st = c->eng->restore_velocities())) return from_engine(c, st);
    return TILD_OK;
}

// Topology change (species or bonds): v^n kept across it as for parameters.
static tild_status retopo(tild_ctx* c, const HostConfig& next) {
    const bool keep = c->eng->has_velocities();
    tild_status st;
    if (keep && (st = c->eng->save_velocities())) return from_engine(c, st);
    c->cfg = next;
    if ((st = c->eng->set_topology())) return from_engine(c, st);
    c->eng->params_changed();
    if (keep && (st = c->eng->restore_velocities())) return from_engine(c, st);
    return TILD_OK;
}

tild_status tild_set_species(tild_ctx* c, int n_species, const int32_t* species) {
    if (!c) return TILD_EINVAL;
    if (!c->have_chains) return fail(c, TILD_ESTATE, "set_species: call tild_set_chains first");
    if (n_species < 1 || n_species > 4) return fail(c, TILD_EINVAL, "set_species: 1..4 species");
    if (!species && n_species != 2)
        return fail(c, TILD_EINVAL, "set_species: without a species array the chains' A/B pattern gives two species");
    HostConfig next = c->cfg;
    next.n_species = n_species;
    next.species_of_bead.clear();
    if (species) {
        next.species_of_bead.resize(next.n_beads);
        for (int i = 0; i < next.n_beads; ++i) {
            if (species[i] < 0 || species[i] >= n_species)
                return fail(c, TILD_EINVAL, "set_species: species values must lie in [0, n_species)");
            next.species_of_bead[i] = (unsigned char)species[i];
        }
    }
    if (n_species > 2 && next.bjerrum > 0 && (next.q_a != 0 || next.q_b != 0))
        return fail(c, TILD_EUNSUPPORTED, "set_species: electrostatics are implemented for up to two species");
    for (int K = n_species; K < 4; ++K)
        for (int K2 = 0; K2 < 4; ++K2) next.chi_mat[K][K2] = next.chi_mat[K2][K] = 0.0;
    return retopo(c, next);
}

tild_status tild_set_bonds(tild_ctx* c, int64_t n_bonds, const int32_t* pairs) {
    if (!c) return TILD_EINVAL;
    if (!c->have_chains) return fail(c, TILD_ESTATE, "set_bonds: call tild_set_chains first");
    if (n_bonds < 0 || (n_bonds > 0 && !pairs)) return fail(c, TILD_EINVAL, "set_bonds: need n_bonds >= 0 and pairs");
    const int N = c->cfg.n_beads;
    std::vector<int64_t> keys((size_t)n_bonds);
    for (int64_t k = 0; k < n_bonds; ++k) {
        const int i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= N || j >= N || i == j)
            return fail(c, TILD_EINVAL, "set_bonds: bead ids out of range or a self-bond");
        keys[k] = (int64_t)std::min(i, j) * N + std::max(i, j);
    }
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
        return fail(c, TILD_EINVAL, "set_bonds: a bond is listed twice");
    HostConfig next = c->cfg;
    next.explicit_bonds = true;
    next.bond_pairs.assign(pairs, pairs + 2 * n_bonds);
    return retopo(c, next);
}

tild_status tild_set_chi_matrix(tild_ctx* c, const double* chi) {
    if (!c) return TILD_EINVAL;
    if (!chi) return fail(c, TILD_EINVAL, "set_chi_matrix: NULL matrix");
    const int S = c->cfg.n_species;
    for (int K = 0; K < S; ++K)
        for (int K2 = 0; K2 < S; ++K2) {
            const double v = chi[K * S + K2];
            if (!std::isfinite(v) || v != chi[K2 * S + K] || (K == K2 && v != 0.0))
                return fail(c, TILD_EINVAL, "set_chi_matrix: need a finite symmetric matrix with a zero diagonal");
        }
    HostConfig next = c->cfg;
    for (int K = 0; K < S; ++K)
        for (int K2 = 0; K2 < S; ++K2) next.chi_mat[K][K2] = chi[K * S + K2];
    next.chi = S >= 2 ? next.chi_mat[0][1] : 0.0;
    next.have_interactions = true;
    return reparam(c, next);
}

tild_status tild_set_layout(tild_ctx* c, int layout) {
    if (!c) return TILD_EINVAL;
    if (layout != TILD_LAYOUT_AOS && layout != TILD_LAYOUT_SOA) return fail(c, TILD_EINVAL, "set_layout: unknown layout");
    c->layout = layout;
    return TILD_OK;
}

tild_status tild_set_interactions(tild_ctx* c, double chi_ab, double kappa, double a) {
    if (!c) return TILD_EINVAL;
    if (!std::isfinite(chi_ab) || !std::isfinite(kappa) || !(kappa >= 0) || !(a > 0) || !std::isfinite(a))
        return fail(c, TILD_EINVAL, "set_interactions: need finite chi, kappa >= 0, a > 0");
    HostConfig next = c->cfg;
    next.chi = chi_ab;
    next.chi_mat[0][1] = next.chi_mat[1][0] = chi_ab;
    next.kappa = kappa;
    next.a = a;
    next.have_interactions = true;
    return reparam(c, next);
}

tild_status tild_set_integrator(tild_ctx* c, double dt, double friction, double kT, double mass) {
    if (!c) return TILD_EINVAL;
    if (!(dt > 0) || !(friction >= 0) || !(kT >= 0) || !(mass > 0) || !std::isfinite(dt) || !std::isfinite(friction) ||
        !std::isfinite(kT) || !std::isfinite(mass))
        return fail(c, TILD_EINVAL, "set_integrator: need dt > 0, friction >= 0, kT >= 0, mass > 0");
    HostConfig next = c->cfg;
    next.dt = dt;
    next.friction = friction;
    next.kT = kT;
    next.mass = mass;
    if (const char* why = scheme_limits(next)) return fail(c, TILD_EINVAL, why);
    return reparam(c, next);
}

tild_status tild_set_electrostatics(tild_ctx* c, double q_a, double q_b, double bjerrum, double smear) {
    if (!c) return TILD_EINVAL;
    if (!std::isfinite(q_a) || !std::isfinite(q_b) || !std::isfinite(bjerrum) || !std::isfinite(smear) ||
        !(bjerrum >= 0) || !(smear > 0))
        return fail(c, TILD_EINVAL, "set_electrostatics: need finite charges, bjerrum >= 0 and smear > 0");
    if (c->cfg.n_species > 2 && bjerrum > 0 && (q_a != 0 || q_b != 0))
        return fail(c, TILD_EUNSUPPORTED, "set_electrostatics: implemented for up to two species");
    if (c->cfg.generic && bjerrum > 0 && (q_a != 0 || q_b != 0))
        return fail(c, TILD_EUNSUPPORTED, "set_electrostatics: implemented for the 3D grid sizes of the tiled kernels");
    HostConfig next = c->cfg;
    next.q_a = q_a;
    next.q_b = q_b;
    next.bjerrum = bjerrum;
    next.charge_smear = smear;
    return reparam(c, next);
}

tild_status tild_set_force_method(tild_ctx* c, int method) {
    if (!c) return TILD_EINVAL;
    if (method != TILD_FORCE_IK && method != TILD_FORCE_ANALYTIC)
        return fail(c, TILD_EINVAL, "set_force_method: unknown method");
    if (method == TILD_FORCE_ANALYTIC && c->cfg.generic)
        return fail(c, TILD_EUNSUPPORTED, "set_force_method: the analytic force is implemented for the 3D grid sizes of the tiled kernels");
    HostConfig next = c->cfg;
    next.force_method = method;
    return reparam(c, next);
}

tild_status tild_set_integrator_scheme(tild_ctx* c, int scheme) {
    if (!c) return TILD_EINVAL;
    if (scheme != TILD_SCHEME_GJF && scheme != TILD_SCHEME_EM && scheme != TILD_SCHEME_VV)
        return fail(c, TILD_EINVAL, "set_integrator_scheme: unknown scheme");
    HostConfig next = c->cfg;
    next.scheme = scheme;
    if (const char* why = scheme_limits(next)) return fail(c, TILD_EINVAL, why);
    return reparam(c, next);
}

tild_status tild_set_stream(tild_ctx* c, void* stream) {
    if (!c) return TILD_EINVAL;
    return from_engine(c, c->eng->set_stream((cudaStream_t)stream));
}

tild_status tild_set_positions(tild_ctx* c, const void* xyz, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!xyz || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "set_positions: bad pointer, dtype or where");
    if (!c->have_chains) return fail(c, TILD_ESTATE, "set_positions: call tild_set_chains first");
    LayoutIO io(c, dtype, where, 1);
    const void* a = io.in(xyz, 0);
    if (io.st) return io.st;
    return from_engine(c, c->eng->set_positions(a, dtype, where));
}

tild_status tild_init_velocities(tild_ctx* c) {
    if (!c) return TILD_EINVAL;
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "init_velocities: positions not set");
    return from_engine(c, c->eng->set_velocities(nullptr, TILD_DTYPE_F64, TILD_DEVICE));
}

tild_status tild_set_velocities(tild_ctx* c, const void* v, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!v || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "set_velocities: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "set_velocities: positions not set");
    LayoutIO io(c, dtype, where, 1);
    const void* a = io.in(v, 0);
    if (io.st) return io.st;
    return from_engine(c, c->eng->set_velocities(a, dtype, where));
}

tild_status tild_step(tild_ctx* c, int64_t n_steps) {
    if (!c) return TILD_EINVAL;
    if (n_steps < 0) return fail(c, TILD_EINVAL, "step: n_steps < 0");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "step: velocities not set");
    return from_engine(c, c->eng->step(n_steps));
}

tild_status tild_synchronize(tild_ctx* c) {
    if (!c) return TILD_EINVAL;
    return from_engine(c, c->eng->synchronize());
}

tild_status tild_compute(tild_ctx* c, unsigned what, tild_energy* e, void* forces_out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (what & ~(TILD_COMPUTE_ENERGY | TILD_COMPUTE_FORCES)) return fail(c, TILD_EINVAL, "compute: unknown flags");
    if ((what & TILD_COMPUTE_ENERGY) && !e) return fail(c, TILD_EINVAL, "compute: energy requested with e == NULL");
    if ((what & TILD_COMPUTE_FORCES) && (!forces_out || !valid_io(dtype, where)))
        return fail(c, TILD_EINVAL, "compute: forces requested with a bad buffer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "compute: positions not set");
    void* f = (what & TILD_COMPUTE_FORCES) ? forces_out : nullptr;
    LayoutIO io(c, dtype, where, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->compute(what, e, io.out(f, 0), dtype, where);
    if (st) return from_engine(c, st);
    io.done(f, 0);
    return io.st;
}

tild_status tild_energy_gradient(tild_ctx* c, tild_energy_grad* g, void* dU_dr, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!g) return fail(c, TILD_EINVAL, "energy_gradient: g == NULL");
    if (dU_dr && !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "energy_gradient: bad dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "energy_gradient: positions not set");
    LayoutIO io(c, dtype, where, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->energy_gradient(g, io.out(dU_dr, 0), dtype, where);
    if (st) return from_engine(c, st);
    io.done(dU_dr, 0);
    return io.st;
}

tild_status tild_force_vjp(tild_ctx* c, const void* lam, void* out, int dtype, int where, double* dtheta) {
    if (!c) return TILD_EINVAL;
    if (!lam || !out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "force_vjp: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "force_vjp: positions not set");
    LayoutIO io(c, dtype, where, 2);
    const void* l = io.in(lam, 0);
    if (io.st) return io.st;
    tild_status st = c->eng->force_vjp(l, io.out(out, 1), dtype, where, dtheta);
    if (st) return from_engine(c, st);
    io.done(out, 1);
    return io.st;
}

tild_status tild_density_vjp(tild_ctx* c, const void* dL_drho, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!dL_drho || !out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "density_vjp: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "density_vjp: positions not set");
    LayoutIO io(c, dtype, where, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->density_vjp(dL_drho, io.out(out, 0), dtype, where);
    if (st) return from_engine(c, st);
    io.done(out, 0);
    return io.st;
}

tild_status tild_get_positions(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_positions: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "get_positions: positions not set");
    LayoutIO io(c, dtype, where, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->get_positions(io.out(out, 0), dtype, where);
    if (st) return from_engine(c, st);
    io.done(out, 0);
    return io.st;
}

tild_status tild_get_velocities(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_velocities: bad pointer, dtype or where");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "get_velocities: velocities not set");
    LayoutIO io(c, dtype, where, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->get_velocities(io.out(out, 0), dtype, where);
    if (st) return from_engine(c, st);
    io.done(out, 0);
    return io.st;
}

tild_status tild_get_density(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_density: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "get_density: positions not set");
    return from_engine(c, c->eng->get_density(out, dtype, where));
}

tild_status tild_get_spectrum(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_spectrum: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "get_spectrum: positions not set");
    return from_engine(c, c->eng->get_spectrum(out, dtype, where));
}

tild_status tild_get_field_gradient(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_field_gradient: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "get_field_gradient: positions not set");
    return from_engine(c, c->eng->get_field_gradient(out, dtype, where));
}

tild_status tild_get_step(tild_ctx* c, int64_t* step) {
    if (!c || !step) return fail(c, TILD_EINVAL, "get_step: NULL argument");
    *step = c->eng->host_step();
    return TILD_OK;
}

tild_status tild_state_bytes(tild_ctx* c, size_t* bytes) {
    if (!c || !bytes) return fail(c, TILD_EINVAL, "state_bytes: NULL argument");
    if (!c->have_chains) return fail(c, TILD_ESTATE, "state_bytes: chains not set");
    *bytes = c->eng->state_bytes();
    return TILD_OK;
}

tild_status tild_get_state(tild_ctx* c, void* blob, size_t bytes, int where) {
    if (!c) return TILD_EINVAL;
    if (!blob) return fail(c, TILD_EINVAL, "get_state: NULL blob");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "get_state: velocities not set");
    if (bytes < c->eng->state_bytes()) return fail(c, TILD_EINVAL, "get_state: blob too small");
    if (where != TILD_HOST && where != TILD_DEVICE) return fail(c, TILD_EINVAL, "get_state: bad where");
    return from_engine(c, c->eng->get_state(blob, where));
}

tild_status tild_set_state(tild_ctx* c, const void* blob, size_t bytes, int where) {
    if (!c) return TILD_EINVAL;
    if (!blob) return fail(c, TILD_EINVAL, "set_state: NULL blob");
    if (!c->have_chains) return fail(c, TILD_ESTATE, "set_state: chains not set");
    if (bytes < c->eng->state_bytes()) return fail(c, TILD_EINVAL, "set_state: blob too small");
    if (where != TILD_HOST && where != TILD_DEVICE) return fail(c, TILD_EINVAL, "set_state: bad where");
    return from_engine(c, c->eng->set_state(blob, where));
}

tild_status tild_profile_steps(tild_ctx* c, int n_steps, double* ms) {
    if (!c) return TILD_EINVAL;
    if (!ms || n_steps < 1) return fail(c, TILD_EINVAL, "profile_steps: need ms[5] and n_steps >= 1");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "profile_steps: velocities not set");
    return from_engine(c, c->eng->profile(n_steps, ms));
}

tild_status tild_trajectory_vjp(tild_ctx* c, int64_t n_steps, int checkpoint_every, const void* r_bar,
                                const void* v_bar, int dtype, int where, void* r0_bar, void* v0_bar, double* dtheta) {
    if (!c) return TILD_EINVAL;
    if (n_steps < 0 || checkpoint_every < 1 || !r_bar || !r0_bar || !v0_bar || !valid_io(dtype, where))
        return fail(c, TILD_EINVAL, "trajectory_vjp: bad argument");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "trajectory_vjp: positions and velocities must be set");
    LayoutIO io(c, dtype, where, 4);
    const void* rb = io.in(r_bar, 0);
    const void* vb = io.in(v_bar, 1);
    if (io.st) return io.st;
    tild_status st = c->eng->trajectory_vjp(n_steps, checkpoint_every, rb, vb, dtype, where, io.out(r0_bar, 2),
                                            io.out(v0_bar, 3), dtheta);
    if (st) return from_engine(c, st);
    io.done(r0_bar, 2);
    io.done(v0_bar, 3);
    return io.st;
}

// Time n steps from the saved state after one untimed re-binning cycle;
// ms per step in *ms.
static tild_status time_steps(tild_ctx* c, void* saved, int64_t n, int K, cudaEvent_t e0, cudaEvent_t e1, double* ms) {
    tild_status st;
    if ((st = c->eng->set_state(saved, TILD_DEVICE)) || (st = c->eng->step(2 * (int64_t)K))) return st;
    cudaStream_t s = c->eng->stream();
    if (cudaEventRecord(e0, s) != cudaSuccess) return TILD_EDEVICE;
    if ((st = c->eng->step(n))) return st;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return TILD_EDEVICE;
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (double)n;
    return TILD_OK;
}

tild_status tild_autotune(tild_ctx* c, int64_t trial_steps, int* sort_every, double* ms_per_step) {
    if (!c) return TILD_EINVAL;
    if (trial_steps < 1) return fail(c, TILD_EINVAL, "autotune: trial_steps must be >= 1");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "autotune: positions and velocities must be set");
    static const int kCandidates[4] = {5, 10, 20, 40};
    const size_t nb = c->eng->state_bytes();
    void* saved = nullptr;
    if (cudaMalloc(&saved, nb) != cudaSuccess) return fail(c, TILD_ENOMEM, "autotune: cannot allocate the checkpoint");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    tild_status st = c->eng->get_state(saved, TILD_DEVICE);
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = TILD_EDEVICE;
    const int original = c->cfg.sort_every;
    int best = original;
    double best_ms = 1e300;
    for (int k = 0; k < 4 && !st; ++k) {
        const int K = kCandidates[k];
        c->cfg.sort_every = K;
        c->eng->params_changed();
        // whole re-binning cycles, after one untimed cycle
        const int64_t n = ((trial_steps + 2 * K - 1) / (2 * K)) * (2 * K);
        double ms = 0;
        if ((st = time_steps(c, saved, n, K, e0, e1, &ms))) break;
        if (ms_per_step) ms_per_step[k] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            best = K;
        }
    }
    c->cfg.sort_every = st ? original : best;
    c->eng->params_changed();
    // launch shapes (plane threads, z column tile) at the chosen period;
    // results do not depend on them either
    int pt0, zc0, zdef, zalt;
    c->eng->launch_shapes(&pt0, &zc0, &zdef, &zalt);
    if (!st && !c->cfg.generic) {
        const int K = c->cfg.sort_every;
        const int64_t n = ((trial_steps + 2 * K - 1) / (2 * K)) * (2 * K);
        int best_pt = pt0, best_zc = zc0;
        double best_sh = 1e300;
        const int pts[5] = {512, 1024, 256, 128, 0};  // 0: row and column passes
        const int zcs[2] = {zdef, zalt};
        for (int a = 0; a < 5 && !st; ++a)
            for (int z = 0; z < (zalt != zdef ? 2 : 1) && !st; ++z) {
                if (c->eng->set_launch_shapes(pts[a], zcs[z]) != TILD_OK) continue;  // not available for this grid
                double ms = 0;
                if ((st = time_steps(c, saved, n, K, e0, e1, &ms))) break;
                if (ms < best_sh) {
                    best_sh = ms;
                    best_pt = pts[a];
                    best_zc = zcs[z];
                }
            }
        c->eng->set_launch_shapes(st ? pt0 : best_pt, st ? zc0 : best_zc);
    }
    // keep the fastest choices and the original state (results do not depend on them)
    if (!st) st = c->eng->set_state(saved, TILD_DEVICE);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(saved);
    if (st) return from_engine(c, st);
    if (sort_every) *sort_every = best;
    return TILD_OK;
}

tild_status tild_get_launch_shapes(tild_ctx* c, int* plane_threads, int* z_columns) {
    if (!c || !plane_threads || !z_columns) return fail(c, TILD_EINVAL, "get_launch_shapes: NULL argument");
    c->eng->launch_shapes(plane_threads, z_columns, nullptr, nullptr);
    return TILD_OK;
}

tild_status tild_set_launch_shapes(tild_ctx* c, int plane_threads, int z_columns) {
    if (!c) return TILD_EINVAL;
    return from_engine(c, c->eng->set_launch_shapes(plane_threads, z_columns));
}

tild_status tild_launches_per_steps(tild_ctx* c, int64_t n_steps, int64_t* launches) {
    if (!c || !launches || n_steps < 0) return fail(c, TILD_EINVAL, "launches_per_steps: bad argument");
    if (!c->have_chains) return fail(c, TILD_ESTATE, "launches_per_steps: chains not set");
    *launches = c->eng->launches(n_steps);
    return TILD_OK;
}

tild_status tild_batch_create(int n, tild_ctx* const* ctxs, tild_batch** out) {
    if (!out || !ctxs || n < 1) {
        g_create_error = "batch_create: need n >= 1 contexts and an output pointer";
        return TILD_EINVAL;
    }
    *out = nullptr;
    std::vector<EngineBase*> engines;
    const int prec = ctxs[0] ? ctxs[0]->cfg.precision : -1;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) {
            g_create_error = "batch_create: NULL context";
            return TILD_EINVAL;
        }
        if (ctxs[i]->cfg.precision != prec) {
            g_create_error = "batch_create: all contexts must have the same precision";
            return TILD_EINVAL;
        }
        if (ctxs[i]->cfg.force_method != TILD_FORCE_IK) {
            g_create_error = "batch_create: batched steps use the ik force only";
            return TILD_EUNSUPPORTED;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                g_create_error = "batch_create: a context appears twice";
                return TILD_EINVAL;
            }
        engines.push_back(ctxs[i]->eng.get());
    }
    std::string err;
    BatchBase* b = prec == TILD_FP32 ? make_batch_f32(engines, err) : make_batch_f64(engines, err);
    if (!b) {
        g_create_error = "batch_create: " + err;
        return TILD_EINVAL;
    }
    *out = new tild_batch{std::unique_ptr<BatchBase>(b)};
    return TILD_OK;
}

tild_status tild_batch_step(tild_batch* b, int64_t n_steps) {
    if (!b || n_steps < 0) {
        g_create_error = "batch_step: bad argument";
        return TILD_EINVAL;
    }
    const tild_status st = b->b->step(n_steps);
    if (st) g_create_error = "batch_step: " + b->b->err;
    return st;
}

tild_status tild_batch_synchronize(tild_batch* b) {
    if (!b) return TILD_EINVAL;
    const tild_status st = b->b->synchronize();
    if (st) g_create_error = "batch_synchronize: " + b->b->err;
    return st;
}

tild_status tild_batch_launches_per_steps(tild_batch* b, int64_t n_steps, int64_t* launches) {
    if (!b || !launches || n_steps < 0) return TILD_EINVAL;
    *launches = b->b->launches(n_steps);
    return TILD_OK;
}

tild_status tild_batch_is_persistent(tild_batch* b, int* persistent) {
    if (!b || !persistent) return TILD_EINVAL;
    *persistent = b->b->persistent() ? 1 : 0;
    return TILD_OK;
}

tild_status tild_batch_set_wait_limit(tild_batch* b, int64_t wait_ns, int extra) {
    if (!b || wait_ns < 1 || extra < 0) {
        g_create_error = "batch_set_wait_limit: bad argument";
        return TILD_EINVAL;
    }
    const tild_status st = b->b->set_wait(wait_ns, extra);
    if (st) g_create_error = "batch_set_wait_limit: " + b->b->err;
    return st;
}

tild_status tild_batch_autotune(tild_batch* b, int64_t trial_steps, double* ms, int* choice) {
    if (!b || trial_steps < 1) {
        g_create_error = "batch_autotune: bad argument";
        return TILD_EINVAL;
    }
    const tild_status st = b->b->autotune(trial_steps, ms, choice);
    if (st) g_create_error = "batch_autotune: " + b->b->err;
    return st;
}

tild_status tild_batch_set_persistent(tild_batch* b, int persistent) {
    if (!b) return TILD_EINVAL;
    const tild_status st = b->b->set_path(persistent != 0);
    if (st) g_create_error = "batch_set_persistent: " + b->b->err;
    return st;
}

tild_status tild_batch_destroy(tild_batch* b) {
    delete b;  // waits for the batch's stream
    return TILD_OK;
}

const char* tild_last_error(tild_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

}  // extern "C"
