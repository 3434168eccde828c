// extern "C" boundary of the TILD engine: argument validation, error text,
// and dispatch to the FP32 or FP64 engine.
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include "engine_api.h"

using namespace tild;

struct tild_ctx {
    HostConfig cfg;
    std::unique_ptr<EngineBase> eng;
    bool have_chains = false;
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

}  // namespace

void tild::set_global_error(const std::string& msg) { g_create_error = msg; }

extern "C" {

tild_status tild_create(const tild_params* p, tild_ctx** out) {
    if (!p || !out) {
        g_create_error = "tild_create: NULL argument";
        return TILD_EINVAL;
    }
    *out = nullptr;
    if (!(p->L[0] > 0) || p->L[0] != p->L[1] || p->L[0] != p->L[2] || !std::isfinite(p->L[0])) {
        g_create_error = "tild_create: the box must be cubic with L > 0";
        return TILD_EUNSUPPORTED;
    }
    if (p->n[0] != p->n[1] || p->n[0] != p->n[2] || !supported_n(p->n[0])) {
        g_create_error = "tild_create: the grid must be cubic with n a power of two in [8, 256] or 24, 40, 48, 80";
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
    if (p->precision == TILD_FP64 && p->n[0] > 128) {
        g_create_error = "tild_create: FP64 grids are limited to 128^3";
        return TILD_EUNSUPPORTED;
    }
    if (p->sort_every < 0) {
        g_create_error = "tild_create: sort_every must be >= 0";
        return TILD_EINVAL;
    }
    std::unique_ptr<tild_ctx> c(new tild_ctx());
    c->cfg.L = p->L[0];
    c->cfg.n = p->n[0];
    c->cfg.pmeorder = p->pmeorder;
    c->cfg.precision = p->precision;
    c->cfg.seed = p->seed;
    c->cfg.sort_every = p->sort_every == 0 ? 20 : p->sort_every;
    std::memset(&c->cfg.topo, 0, sizeof(c->cfg.topo));
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
        if (total >= (int64_t)1 << 31) return fail(c, TILD_EUNSUPPORTED, "set_chains: at most 2^31-1 beads");
    }
    if (total < 1) return fail(c, TILD_EINVAL, "set_chains: no beads");
    topo.start[n_types] = (int)total;
    topo.n_types = n_types;
    c->cfg.topo = topo;
    c->cfg.n_beads = (int)total;
    c->cfg.b = b;
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

tild_status tild_set_interactions(tild_ctx* c, double chi_ab, double kappa, double a) {
    if (!c) return TILD_EINVAL;
    if (!std::isfinite(chi_ab) || !std::isfinite(kappa) || !(kappa >= 0) || !(a > 0) || !std::isfinite(a))
        return fail(c, TILD_EINVAL, "set_interactions: need finite chi, kappa >= 0, a > 0");
    HostConfig next = c->cfg;
    next.chi = chi_ab;
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
    return from_engine(c, c->eng->set_positions(xyz, dtype, where));
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
    return from_engine(c, c->eng->set_velocities(v, dtype, where));
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
    return from_engine(c, c->eng->compute(what, e, (what & TILD_COMPUTE_FORCES) ? forces_out : nullptr, dtype, where));
}

tild_status tild_energy_gradient(tild_ctx* c, tild_energy_grad* g, void* dU_dr, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!g) return fail(c, TILD_EINVAL, "energy_gradient: g == NULL");
    if (dU_dr && !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "energy_gradient: bad dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "energy_gradient: positions not set");
    return from_engine(c, c->eng->energy_gradient(g, dU_dr, dtype, where));
}

tild_status tild_force_vjp(tild_ctx* c, const void* lam, void* out, int dtype, int where, double* dtheta) {
    if (!c) return TILD_EINVAL;
    if (!lam || !out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "force_vjp: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "force_vjp: positions not set");
    return from_engine(c, c->eng->force_vjp(lam, out, dtype, where, dtheta));
}

tild_status tild_get_positions(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_positions: bad pointer, dtype or where");
    if (!c->eng->has_positions()) return fail(c, TILD_ESTATE, "get_positions: positions not set");
    return from_engine(c, c->eng->get_positions(out, dtype, where));
}

tild_status tild_get_velocities(tild_ctx* c, void* out, int dtype, int where) {
    if (!c) return TILD_EINVAL;
    if (!out || !valid_io(dtype, where)) return fail(c, TILD_EINVAL, "get_velocities: bad pointer, dtype or where");
    if (!c->eng->has_velocities()) return fail(c, TILD_ESTATE, "get_velocities: velocities not set");
    return from_engine(c, c->eng->get_velocities(out, dtype, where));
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
    return from_engine(c, c->eng->trajectory_vjp(n_steps, checkpoint_every, r_bar, v_bar, dtype, where, r0_bar, v0_bar,
                                                 dtheta));
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
        if ((st = c->eng->set_state(saved, TILD_DEVICE)) || (st = c->eng->step(2 * K))) break;
        cudaStream_t s = c->eng->stream();
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = TILD_EDEVICE; break; }
        if ((st = c->eng->step(n))) break;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) { st = TILD_EDEVICE; break; }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_per_step) ms_per_step[k] = ms / (double)n;
        if (ms / (double)n < best_ms) {
            best_ms = ms / (double)n;
            best = K;
        }
    }
    // keep the fastest period and the original state (results do not depend on the period)
    c->cfg.sort_every = st ? original : best;
    c->eng->params_changed();
    if (!st) st = c->eng->set_state(saved, TILD_DEVICE);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(saved);
    if (st) return from_engine(c, st);
    if (sort_every) *sort_every = best;
    return TILD_OK;
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

tild_status tild_batch_destroy(tild_batch* b) {
    delete b;  // waits for the batch's stream
    return TILD_OK;
}

const char* tild_last_error(tild_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

}  // extern "C"
