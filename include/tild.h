/*
 * tild.h — C ABI of a GB300 (sm_103a) implementation of the
 * theoretically-informed Langevin (TILD) timestep of MATILDA.FT
 * (arXiv 2302.02474).
 *
 * One call of tild_step advances a coarse-grained polymer system by one or
 * more steps of the particle-mesh method the paper describes:
 *   1. assign bead densities to a periodic grid with the spline weights of
 *      order pmeorder (Eq. rhohat; Sec. "Long-range interactions", weights
 *      from the appendix of Deserno & Holm 1998; Fig. pmm);
 *   2. Fourier-transform the species densities;
 *   3. multiply by the Fourier transform of the Gaussian-smeared Flory (chi,
 *      Eq. fh) and Helfand (kappa, Eq. HelfandP) pair kernel and by i k
 *      (the convolution of Eq. PMM);
 *   4. inverse-transform the field gradients;
 *   5. interpolate the forces back to the beads with the same weights
 *      (caption of Fig. pmm), add harmonic bond forces (Eq. bonds);
 *   6. advance positions and velocities with the Gronbech-Jensen-Farago
 *      Langevin integrator (GJF; Sec. "Integrator Class", Listing infile),
 *      or with Euler-Maruyama or velocity-Verlet + Langevin force, the other
 *      integrators that section lists (tild_set_integrator_scheme).
 *
 * Around the step: observables (tild_compute), the analytic-gradient force
 * variant (tild_set_force_method), smeared-charge electrostatics
 * (tild_set_electrostatics), batches of uneven replicas (tild_batch_*) and
 * the differentiable form: the energy gradient (tild_energy_gradient), the
 * force vector-Jacobian product (tild_force_vjp) and derivatives through
 * trajectories (tild_trajectory_vjp).
 *
 * Units are the paper's reduced units (Sec. "Units"): energy kT, mass m of
 * a monomer, length b.
 *
 * Conventions shared by every call:
 *   - Every function returns a tild_status: TILD_OK (0) or a negative error.
 *     On error the context is unchanged unless stated otherwise, and
 *     tild_last_error() returns a one-line description.
 *   - Beads are numbered 0..n_beads-1 chain by chain, in the order of the
 *     molecule types given to tild_set_chains (bead s of chain c of type t
 *     has id start_t + c*N_t + s).
 *   - Arrays of per-bead vectors are AoS, [n_beads][3], in bead-id order,
 *     unless tild_set_layout selects SoA, [3][n_beads].
 *     Their element type is given by a tild_dtype; `where` says whether the
 *     pointer is host or device memory (TILD_HOST / TILD_DEVICE). The caller
 *     owns every buffer it passes; the library copies in or out and keeps no
 *     pointer after the call returns.
 *   - Grid arrays are C-ordered [z][y][x] (x fastest) with n^3 points.
 *   - All device work is ordered on the context's stream. Calls that return
 *     data to the caller synchronise that stream before returning; tild_step
 *     does not (use tild_synchronize).
 *   - The library owns its device state (bead arrays, grids, spectra),
 *     allocated by tild_create / tild_set_chains / tild_set_species (and
 *     scratch by the calls that say so) and freed by tild_destroy, through
 *     cudaMalloc/cudaFree or the allocator given to
 *     tild_create_with_allocator.
 *   - A context is bound to the CUDA device that was current when it was
 *     created; calls on it must be made with that device current.
 *   - Not thread-safe: one host thread at a time per context.
 */
#ifndef TILD_H
#define TILD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tild_status;

#define TILD_OK 0
#define TILD_EINVAL (-1)        /* bad argument (NULL, out of range, wrong size) */
#define TILD_ENOMEM (-2)        /* device or host allocation failed */
#define TILD_EUNSUPPORTED (-3)  /* valid request outside what this build implements */
#define TILD_EDEVICE (-4)       /* a CUDA call failed; see tild_last_error */
#define TILD_ENAN (-5)          /* a non-finite position or force was detected on the device */
#define TILD_ESTATE (-6)        /* call made before the state it needs exists */
#define TILD_ETIMEOUT (-7)      /* a device-side wait ran past its time limit (batches; see tild_batch_set_wait_limit) */

typedef enum { TILD_FP32 = 0, TILD_FP64 = 1 } tild_precision;
typedef enum { TILD_DTYPE_F32 = 0, TILD_DTYPE_F64 = 1 } tild_dtype;
typedef enum { TILD_HOST = 0, TILD_DEVICE = 1 } tild_where;

typedef struct tild_ctx tild_ctx;

/*
 * Box, grid and numerics (Listing infile: box and grid size, pmeorder).
 *   L[3]        box edges; this build requires a cubic box (L[0]=L[1]=L[2] > 0).
 *   n[3]        grid points per edge; cubic: a power of two in [8, 256]
 *               (FP64 grids up to 128) or one of the 5-smooth sizes 24,
 *               40, 48, 80. Others give TILD_EUNSUPPORTED.
 *   pmeorder    assignment order p in 1..4: p+1 grid points per dimension
 *               (order 1 = the two nearest points, Fig. pmm).
 *   precision   TILD_FP32 (grids, FFT and bead state in FP32; energies in
 *               FP64) or TILD_FP64 (everything FP64).
 *   seed        64-bit key of the Philox4x32-10 stream of the thermal noise.
 *   sort_every  re-bin beads by grid tile every this many steps (>= 1;
 *               0 selects the default of 20). Results do not depend on it.
 */
typedef struct {
    double L[3];
    int n[3];
    int pmeorder;
    int precision;
    uint64_t seed;
    int sort_every;
} tild_params;

/*
 * One molecule type (Sec. "Structure of ... models": chains of N_A + N_B = N
 * beads joined by harmonic bonds, Eq. bonds): n_chains linear chains of N
 * beads whose first n_a beads are species A (0) and the rest species B (1).
 */
typedef struct {
    int64_t n_chains;
    int N;
    int n_a;
} tild_moltype;

/* Energies in kT (Eqs. bonds, fh, HelfandP) and diagnostics of the current
 * configuration. e_chi keeps the k=0 Fourier term of Eq. fh; e_kappa drops
 * the k=0 term, which cancels the -rho_0 shift of Eq. HelfandP exactly.
 * kinetic = sum_i m |v_i|^2 / 2. net_force = sum_i F_i. e_elec is the
 * smeared-charge electrostatic energy (0 without charges; see
 * tild_set_electrostatics). */
typedef struct {
    double e_bond;
    double e_chi;
    double e_kappa;
    double kinetic;
    double net_force[3];
    double e_elec;
} tild_energy;

/* Energy of the current configuration and its derivatives with respect to
 * the interaction parameters (the model's energy U = E_bond + E_chi +
 * E_kappa of Eqs. bonds, fh and HelfandP, on the grid):
 *   dU/dchi   = (1/rho_0) int int rho_A u_G rho_B          (Eq. fh)
 *   dU/dkappa = (1/2rho_0) int int (rho_+ - rho_0) u_G (rho_+ - rho_0)
 *   dU/da     = sum over k of (d u_hat/d a) (...), d u_hat/d a = -2 a |k|^2 u_hat
 * (sigma^2 = 2 a^2, Eqs. fhF, HelfandF), all reduced in FP64 on the device. */
typedef struct {
    double energy;
    double e_bond;
    double e_chi;
    double e_kappa;
    double dU_dchi;
    double dU_dkappa;
    double dU_da;
    double e_elec;  /* included in energy; a does not enter it */
} tild_energy_grad;

#define TILD_COMPUTE_ENERGY 1u
#define TILD_COMPUTE_FORCES 2u

/* Create a context for the box/grid in *p on the current CUDA device. On
 * success *out owns device memory for the grids. */
tild_status tild_create(const tild_params* p, tild_ctx** out);

/* Device-memory allocator of a context (for instance a framework's caching
 * allocator). alloc returns `bytes` of device memory on the context's device,
 * aligned to at least 256 bytes, or NULL on failure (the calling tild_*
 * function then returns TILD_ENOMEM). free releases a block that alloc
 * returned, with its size. The library frees every block before
 * tild_destroy returns and calls alloc/free only from the thread making the
 * tild_* call. `user` is passed through. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, size_t bytes, void* user);
    void* user;
} tild_allocator;

/* tild_create with every device allocation of the context (grids, bead
 * arrays, scratch) made through *a. a == NULL or a->alloc == NULL is
 * tild_create. Batches (tild_batch_*) and tild_autotune's checkpoint still
 * use cudaMalloc for their own small tables. */
tild_status tild_create_with_allocator(const tild_params* p, const tild_allocator* a, tild_ctx** out);

/* Free everything the context owns. NULL is accepted. */
tild_status tild_destroy(tild_ctx* ctx);

/* Define the chains (and so the number of beads, the species and the bond
 * topology). b is the statistical segment length of Eq. bonds (bond force
 * -(3/b^2)(r_i - r_j)). At most 8 types, 1 <= N, 0 <= n_a <= N, at least one
 * bead, fewer than 2^29 beads. The chains give two species (A, B) and linear
 * bonds; tild_set_species and tild_set_bonds replace either. Allocates the
 * bead arrays; existing positions are discarded, as are species and bonds
 * set before. */
tild_status tild_set_chains(tild_ctx* ctx, int n_types, const tild_moltype* types, double b);

/* Species of the beads (Sec. "Input file": each atom of the data file has a
 * type; Eq. fh couples every pair of types through chi). n_species in 1..4.
 * species (host, [n_beads] int32 in bead-id order, values in
 * [0, n_species)) gives every bead's species; NULL keeps the chains' A/B
 * pattern (then n_species must be 2). Flory parameters of the new species
 * pairs start at 0 (tild_set_chi_matrix). Three or four species allocate a
 * second pair of density and field grids. With more than two species,
 * electrostatics, tild_energy_gradient, tild_force_vjp, tild_trajectory_vjp
 * and batches return TILD_EUNSUPPORTED. Requires chains; existing positions
 * are re-binned and velocities are kept (as for tild_set_interactions). */
tild_status tild_set_species(tild_ctx* ctx, int n_species, const int32_t* species);

/* Bond topology (Eq. bonds; Sec. "Input file": the data file lists the
 * bonds): n_bonds >= 0 harmonic bonds between bead ids pairs[2k] and
 * pairs[2k+1] (host int32), each pair once, no self-bonds, no repeats; any
 * topology (rings, branches, networks) and any number of bonds per bead.
 * Replaces the chains' linear bonds (pairs == NULL with n_bonds == 0 removes
 * every bond). Forces and energies are independent of the order of the list.
 * Requires chains; positions are re-binned and velocities kept. */
tild_status tild_set_bonds(tild_ctx* ctx, int64_t n_bonds, const int32_t* pairs);

/* Interactions (Eqs. fh, HelfandP; sigma^2 = 2 a^2 per Eqs. fhF, HelfandF):
 * chi_ab = Flory chi between A and B, kappa = Helfand compressibility,
 * a = smearing width of h (the pair kernel's Fourier transform is
 * exp(-|k|^2 a^2)). a > 0, kappa >= 0. rho_0 = n_beads / V.
 * Defaults before the first call: chi_ab = 0, kappa = 0, a = 0.5. If
 * velocities exist, v^n is kept and the carried state is updated to the
 * new forces. */
tild_status tild_set_interactions(tild_ctx* ctx, double chi_ab, double kappa, double a);

/* Flory matrix for more than two species (Eq. fh over every species pair):
 * chi, host [n_species][n_species] doubles, symmetric, finite, zero
 * diagonal. The pair potential matrix becomes eps_KK' = (chi_KK' + kappa) /
 * rho_0. chi[0][1] is the chi_ab of tild_set_interactions (each call sets
 * it). Velocities are kept. */
tild_status tild_set_chi_matrix(tild_ctx* ctx, const double* chi);

/* Integrator parameters (Sec. "Integrator Class"): time step dt > 0,
 * friction alpha >= 0, temperature kT >= 0, bead mass > 0. Defaults:
 * dt = 0.005, alpha = 1, kT = 1, mass = 1. If velocities exist, v^n is
 * kept. The scheme in use may add limits (see tild_set_integrator_scheme);
 * values it cannot take return TILD_EINVAL and change nothing. */
tild_status tild_set_integrator(tild_ctx* ctx, double dt, double friction, double kT, double mass);

/* The three integrators of Sec. "Integrator Class". Random numbers of all
 * three come from the same Philox stream (counter = bead id and step).
 *   TILD_SCHEME_GJF  Gronbech-Jensen-Farago Langevin (the default).
 *   TILD_SCHEME_EM   Euler-Maruyama for overdamped Langevin (Brownian)
 *                    dynamics: r^{n+1} = r^n + (dt/alpha) F^n
 *                    + sqrt(2 kT dt/alpha) xi^{n+1}. Needs alpha > 0. There
 *                    is no velocity: velocities read back as 0 and the
 *                    kinetic energy is 0.
 *   TILD_SCHEME_VV   velocity-Verlet with the Langevin thermostat force
 *                    -alpha v^{n-1/2} + sqrt(2 alpha kT/dt) xi^n acting on the
 *                    half-step velocity (alpha = 0: plain NVE). Needs
 *                    alpha dt / 2m < 1.
 * Forces reported by tild_compute are the field and bond forces only.
 * Switching keeps v^n (zero when leaving EM). Unknown schemes return
 * TILD_EINVAL. */
#define TILD_SCHEME_GJF 0
#define TILD_SCHEME_EM 1
#define TILD_SCHEME_VV 2
tild_status tild_set_integrator_scheme(tild_ctx* ctx, int scheme);

/* How the particle-mesh force is taken from the potentials (Sec. "Long-range
 * interactions", Eq. PMM):
 *   TILD_FORCE_IK        the default: the field gradient by spectral (i k)
 *                        differentiation, interpolated back with the
 *                        assignment weights (three inverse transforms).
 *   TILD_FORCE_ANALYTIC  F_i = -sum_g grad W(r_i - g) w_K(g): the exact
 *                        gradient of the gridded energy, from the potentials
 *                        (one inverse transform) and the derivatives of the
 *                        assignment weights. Not momentum conserving.
 * If velocities exist, v^n is kept. Batches (tild_batch_create) take
 * TILD_FORCE_IK contexts only. Unknown methods return TILD_EINVAL. */
#define TILD_FORCE_IK 0
#define TILD_FORCE_ANALYTIC 1
tild_status tild_set_force_method(tild_ctx* ctx, int method);

/* Electrostatics (Sec. "Long-range interactions": charged monomers interact
 * through Coulomb forces computed with the same particle-mesh scheme;
 * charges are spread over a unit Gaussian with a charge spreading length,
 * and the Bjerrum length sets the strength). q_a, q_b = charge of every A
 * and every B bead (units of e); bjerrum = l_B in units of length (0 turns
 * electrostatics off); smear = a_e > 0. The pair kernel of two smeared
 * charges is 4 pi l_B exp(-|k|^2 a_e^2) / |k|^2 in Fourier space (k = 0
 * dropped: a neutralising background), so w_K gains q_K phi and
 * E_elec = (1/2) int rho_q phi. Applies to both force methods and to
 * tild_energy_gradient. If velocities exist, v^n is kept. Non-finite values,
 * bjerrum < 0 or smear <= 0 return TILD_EINVAL. */
tild_status tild_set_electrostatics(tild_ctx* ctx, double q_a, double q_b, double bjerrum, double smear);

/* Layout of every per-bead vector array this context reads or writes
 * (positions, velocities, forces, dU/dr, adjoint vectors):
 *   TILD_LAYOUT_AOS  [n_beads][3] (the default);
 *   TILD_LAYOUT_SOA  [3][n_beads]: all x, then all y, then all z.
 * Device arrays in SoA pass through a context-owned device scratch of
 * 3 n_beads doubles (allocated on first use). Unknown layouts return
 * TILD_EINVAL. */
#define TILD_LAYOUT_AOS 0
#define TILD_LAYOUT_SOA 1
tild_status tild_set_layout(tild_ctx* ctx, int layout);

/* Order all work of this context on `stream` (a cudaStream_t; NULL = the
 * context's own stream). The stream must belong to the context's device and
 * outlive its use by the context. */
tild_status tild_set_stream(tild_ctx* ctx, void* stream);

/* Copy in positions [n_beads][3] (wrapped into [0, L)). Requires chains.
 * Invalidates velocities: call tild_init_velocities or tild_set_velocities
 * before stepping. A non-finite coordinate returns TILD_ENAN (the bead is
 * placed at 0 on that axis). */
tild_status tild_set_positions(tild_ctx* ctx, const void* xyz, int dtype, int where);

/* Draw Maxwell-Boltzmann velocities (each component N(0, kT/m), Philox
 * counter (bead id, 2^64-1)) and evaluate the forces at the current
 * positions. Resets the step counter to 0. */
tild_status tild_init_velocities(tild_ctx* ctx);

/* Copy in velocities [n_beads][3] and evaluate the forces at the current
 * positions. Resets the step counter to 0. */
tild_status tild_set_velocities(tild_ctx* ctx, const void* v, int dtype, int where);

/* Advance n_steps >= 0 GJF steps, asynchronously on the context's stream.
 * The thermal noise of step n -> n+1 for bead i is drawn from Philox counter
 * (i, n+1). Launch errors are reported here; a non-finite force raised by
 * a step is reported by the next tild_synchronize or tild_compute. */
tild_status tild_step(tild_ctx* ctx, int64_t n_steps);

/* Wait for the context's stream. Returns TILD_ENAN if any step flagged a
 * non-finite force since the last check (the flag is then cleared). */
tild_status tild_synchronize(tild_ctx* ctx);

/* Evaluate at the current positions: `what` = TILD_COMPUTE_ENERGY and/or
 * TILD_COMPUTE_FORCES. Energies go to *e (may be NULL if not requested);
 * total forces (field + bonds) to forces_out [n_beads][3] (may be NULL if
 * not requested). Does not change the state. */
tild_status tild_compute(tild_ctx* ctx, unsigned what, tild_energy* e, void* forces_out, int dtype, int where);

/* Energy and its gradients at the current positions: *g receives U and
 * dU/dchi, dU/dkappa, dU/da; dU_dr (may be NULL) receives dU/dr_i,
 * [n_beads][3], the exact gradient of the gridded energy: the adjoint of the
 * density assignment (the assignment weights differentiated, Sec.
 * "Long-range interactions") applied to the potential fields w_K, plus the
 * bond term of Eq. bonds. (The forces of tild_compute use the spectral
 * gradient instead, as the method does; the two agree as the grid is
 * refined.) Does not change the state. */
tild_status tild_energy_gradient(tild_ctx* ctx, tild_energy_grad* g, void* dU_dr, int dtype, int where);

/* Vector-Jacobian product of the force (differentiable form): for an
 * adjoint vector lam [n_beads][3] (by bead id, dtype/where as for
 * positions), out [n_beads][3] receives sum_i lam_i . dF_i/dr_j for every
 * bead j, where F is the ik particle-mesh force of Eq. PMM plus the bond
 * force of Eq. bonds (charges included) at the current positions. dtheta
 * (NULL to skip) receives d(sum_i lam_i . F_i)/d(chi, kappa, a). Chained
 * through the integrator this gives derivatives of trajectories
 * (tild_trajectory_vjp). lam is spread onto the grid in 64-bit fixed
 * point with a power-of-two scale taken from max|lam|, so the result is
 * bitwise reproducible and exactly homogeneous under power-of-two scaling of
 * lam; a non-finite lam makes every output NaN. Returns
 * TILD_EUNSUPPORTED with the analytic force method or for grids whose
 * planes do not fit one CTA (FP32 above 128^3, FP64 above 64^3). */
tild_status tild_force_vjp(tild_ctx* ctx, const void* lam, void* out, int dtype, int where, double* dtheta);

/* Vector-Jacobian product of the density assignment (differentiable form;
 * Eq. rhohat with the spline weights of Sec. "Long-range interactions"
 * differentiated): for a grid adjoint dL_drho = dL/drho_K(g), [n_species]
 * [n][n][n] in [z][y][x] order (dtype/where), out [n_beads][3] receives
 * d/dr_i sum_{K,g} dL_drho_K(g) rho_K(g) = (1/dV) sum_g grad W(r_i - g)
 * dL_drho_{K_i}(g) at the current positions: the gradient of any loss on the
 * density grid (for example a density-profile loss) with respect to the
 * positions. Passed as r_bar to tild_trajectory_vjp it carries the loss back
 * through a trajectory. Three-dimensional boxes (else TILD_EUNSUPPORTED).
 * Allocates a context scratch of n_species n^3 + 3 n_beads values. */
tild_status tild_density_vjp(tild_ctx* ctx, const void* dL_drho, void* out, int dtype, int where);

/* Derivatives through a trajectory (differentiable form): runs n_steps
 * steps of the context's integrator scheme (GJF, EM or VV; TILD_FORCE_IK)
 * and returns the derivatives of a loss L(r^K, v^K) with respect to r^0
 * (r0_bar), v^0 (v0_bar) and, in dtheta (NULL to skip), chi, kappa and a,
 * given dL/dr^K = r_bar and dL/dv^K = v_bar (NULL: 0). The thermal noise is
 * held fixed (the same Philox counters). Every scheme advances the state
 * (r, u) in one linear form,
 *   h = su u + sf F(r) + sg xi,  r' = r + sd h + se xi,  u' = sh h + sk xi,
 * with v = vu u + vf F + vg xi and u^0 = wu v^0 + wf F(r^0) + wg xi, so the
 * reverse sweep is hb = sd rb' + sh ub', ub = su hb, rb = rb' + J^T(sf hb)
 * for every scheme (EM has no velocity: v0_bar is 0). Reverse mode
 * recomputes the states of each segment of checkpoint_every steps from a
 * device checkpoint (bit-identical), keeps each recomputed state binned as
 * it was (positions in slot order, slot arrays and the density grid, so no
 * re-binning before its VJP) and takes one force vector-Jacobian product per
 * state; the adjoint vectors are FP64. All arrays are [n_beads][3] by bead
 * id in dtype/where. The context ends at step n_steps. Device scratch, kept
 * with the context: n_steps/C + 2 states and C binned snapshots (3N values,
 * 3N ints, 2 n^3 64-bit grid points and the 4 n^3 complex values of that
 * state's fields each), C = min(checkpoint_every, n_steps). */
tild_status tild_trajectory_vjp(tild_ctx* ctx, int64_t n_steps, int checkpoint_every, const void* r_bar,
                                const void* v_bar, int dtype, int where, void* r0_bar, void* v0_bar, double* dtheta);

/* Current positions (wrapped into [0, L)), [n_beads][3]. */
tild_status tild_get_positions(tild_ctx* ctx, void* out, int dtype, int where);

/* Current velocities v^n, [n_beads][3]. */
tild_status tild_get_velocities(tild_ctx* ctx, void* out, int dtype, int where);

/* Species densities rho_K(g) on the grid (beads per unit volume) of the
 * current positions: [n_species][n][n][n] (two species: A then B),
 * [z][y][x] order. */
tild_status tild_get_density(tild_ctx* ctx, void* out, int dtype, int where);

/* Discrete Fourier transform Z(k) = sum_g (rho_A(g) + i rho_B(g)) e^{-i k.g}
 * of the current densities, as interleaved (re, im) pairs [n][n][n][2] in
 * [kz][ky][kx] FFT index order (index m < n/2 is frequency m, else m - n).
 * Three or four species: [2][n][n][n][2], the transforms of
 * rho_0 + i rho_1 and rho_2 + i rho_3 (rho_3 = 0 for three species). */
tild_status tild_get_spectrum(tild_ctx* ctx, void* out, int dtype, int where);

/* Gradients of the potential fields w_K = sum_K' eps_KK' u_G * rho_K' on
 * the grid, [3][n][n][n][2]: for direction d (x, y, z), point (z, y, x), the
 * pair (d w_A / d r_d, d w_B / d r_d). eps_KK = kappa/rho_0,
 * eps_AB = (chi_ab + kappa)/rho_0. Three or four species:
 * [2][3][n][n][n][2], species pairs (0, 1) and (2, 3). */
tild_status tild_get_field_gradient(tild_ctx* ctx, void* out, int dtype, int where);

/* Number of steps taken since velocities were set. */
tild_status tild_get_step(tild_ctx* ctx, int64_t* step);

/* Checkpoint: tild_state_bytes gives the size of the opaque blob that
 * tild_get_state writes (positions, carried velocities, step counter, seed,
 * in the context's precision) to host (where = TILD_HOST) or device
 * (TILD_DEVICE, 8-byte aligned) memory owned by the caller. tild_set_state
 * restores it into a context with the same chains and precision; continuing
 * from a restored state reproduces the original trajectory bit for bit. */
tild_status tild_state_bytes(tild_ctx* ctx, size_t* bytes);
tild_status tild_get_state(tild_ctx* ctx, void* blob, size_t bytes, int where);
tild_status tild_set_state(tild_ctx* ctx, const void* blob, size_t bytes, int where);

/* Time each kernel of the step: runs n_steps steps with CUDA events around
 * every kernel launch (no graph) and writes the mean device time in
 * milliseconds of the kernels of each stage to ms[5]:
 * [0] forward FFT passes (density in), [1] spectral z pass,
 * [2] inverse FFT passes (gradients out), [3] bead kernel (gather, bonds,
 * GJF, spread), [4] re-binning (per step, amortised). */
tild_status tild_profile_steps(tild_ctx* ctx, int n_steps, double* ms);

/* Number of kernel launches one tild_step(ctx, n) issues for this context. */
tild_status tild_launches_per_steps(tild_ctx* ctx, int64_t n_steps, int64_t* launches);

/* Autotuner: times whole re-binning cycles for re-binning periods 5, 10, 20
 * and 40 (each over about trial_steps steps after one untimed cycle, from
 * the same saved state) and keeps the fastest; then, at that period, times
 * the launch shapes of the step (tild_set_launch_shapes: every available
 * plane thread count and z column tile) and keeps the fastest. Trajectories
 * are bit-identical for every choice, so only speed changes; the context's
 * state is restored afterwards. sort_every (may be NULL) receives the chosen
 * period, ms_per_step (may be NULL) the four period timings in candidate
 * order; tild_get_launch_shapes reads the chosen shapes. Needs positions and
 * velocities; allocates one state-sized device buffer (cudaMalloc) for the
 * duration of the call. */
tild_status tild_autotune(tild_ctx* ctx, int64_t trial_steps, int* sort_every, double* ms_per_step);

/* Launch shapes of the step's FFT passes (results are bit-identical for
 * every choice; only speed changes):
 *   plane_threads  threads of each xy-plane CTA of the forward and inverse
 *                  passes: 512 (default), or 256 / 128 for planes small
 *                  enough that several CTAs share an SM (n <= 80 and n <= 64
 *                  respectively, when stage B of the line transform keeps at
 *                  most 32 complex values per thread), 1024 (FP32, n = 80 and
 *                  128: every thread has a unit of the line transform's
 *                  second stage), or 0 for separate x-row
 *                  and y-column passes through global memory (the passes of
 *                  grids whose planes do not fit shared memory; n a
 *                  multiple of 16 in FP32, of 8 (and at least 16) in FP64);
 *   z_columns      column tile of the z pass: the default (128 bytes of
 *                  complex values) or the alternative of half that width
 *                  (twice the CTAs).
 * tild_get_launch_shapes reports the current values; tild_set_launch_shapes
 * returns TILD_EINVAL for a value this grid does not have and
 * TILD_EUNSUPPORTED on the any-size grids. Batches launch every grid-size
 * group with the shapes of its first context. */
tild_status tild_get_launch_shapes(tild_ctx* ctx, int* plane_threads, int* z_columns);
tild_status tild_set_launch_shapes(tild_ctx* ctx, int plane_threads, int z_columns);

/*
 * Batched form (the paper's plan of several boxes per run, Sec.
 * "Conclusions"): step several independent systems ("replicas": contexts
 * with their own chains, box, grid, chi, kappa, a and seed; same precision
 * and device) together. When every replica is FP32 with pmeorder 1, the ik
 * force, no charges, two species and a grid of 24, 32, 40, 48 or 64 points
 * per edge, the steps between two re-binnings of all replicas are ONE
 * persistent cooperative launch: its CTAs walk a table of the work items of
 * every replica (xy planes, z-pass tiles, bead tiles), stage by stage, and
 * meet at grid-wide barriers whose waits are bounded
 * (tild_batch_set_wait_limit; a wait that runs out is reported as
 * TILD_ETIMEOUT by tild_batch_synchronize). Otherwise replicas with the same grid size and
 * assignment order share every kernel launch of a step (four per group),
 * reading their arguments from device tables, with each group's launch
 * shapes taken from its first context. Either way whole re-binning cycles
 * of all replicas are captured as one CUDA graph (re-binning and the
 * persistent launch, or the per-group launches). Each replica's trajectory
 * is bit-identical to stepping its context alone with the same re-binning
 * period (the batch uses the first context's sort_every).
 *
 * tild_batch_create: every context must have positions and velocities and a
 * grid of at most 128 points (FP32) or 64 (FP64) per edge. The contexts stay
 * owned by the caller and must outlive the batch; creating the batch
 * re-bins them. While the batch exists, change no context's chains,
 * interactions, integrator, positions or velocities (results would not
 * reflect the change); reading a context (positions, energies, state) is
 * fine after tild_batch_synchronize.
 * tild_batch_step: advance every replica n_steps (asynchronous on the
 * batch's own stream). tild_batch_synchronize waits for it and reports
 * TILD_ENAN if any replica flagged a non-finite force. Errors are described
 * by tild_last_error(NULL).
 */
typedef struct tild_batch tild_batch;
tild_status tild_batch_create(int n_replicas, tild_ctx* const* replicas, tild_batch** out);
tild_status tild_batch_step(tild_batch* batch, int64_t n_steps);
tild_status tild_batch_synchronize(tild_batch* batch);
tild_status tild_batch_launches_per_steps(tild_batch* batch, int64_t n_steps, int64_t* launches);
tild_status tild_batch_destroy(tild_batch* batch);

/* *persistent = 1 when the batch steps through the persistent kernel. */
tild_status tild_batch_is_persistent(tild_batch* batch, int* persistent);

/* Choose the persistent kernel (persistent != 0; TILD_EUNSUPPORTED when the
 * replicas do not allow it) or the per-group launches for the following
 * steps. Results do not depend on the choice. */
tild_status tild_batch_set_persistent(tild_batch* batch, int persistent);

/* Batch autotuner: times whole re-binning cycles of the batch (about
 * trial_steps steps each, after one untimed cycle, from the same saved
 * replica states) for 9 candidates: [0..2] the persistent kernel (when the
 * replicas allow it) with its registers allocated for 2, 3 and 4 resident
 * CTAs per SM, then the per-group launches with plane threads 512, 256, 128
 * (each group falls back to the largest its grid allows), each with the
 * default and the alternative z column tile; keeps the fastest. ms (may be
 * NULL) receives the 9 timings in ms per step (-1 for an unavailable
 * candidate), choice (may be NULL) the index kept. The replicas' states are
 * restored afterwards (results do not depend on the choice). Allocates one
 * state blob per replica (cudaMalloc) for the duration of the call. */
tild_status tild_batch_autotune(tild_batch* batch, int64_t trial_steps, double* ms, int* choice);

/* Time limit (wait_ns > 0; default 2 s) of one grid-barrier wait of the
 * persistent kernel, and extra >= 0 arrivals a barrier waits for beyond the
 * launch's CTAs. extra > 0 is a fault-injection hook for tests: no barrier
 * can complete, every wait runs out, the kernel returns and
 * tild_batch_synchronize reports TILD_ETIMEOUT (the replicas' states are
 * then undefined). TILD_EUNSUPPORTED without the persistent path. */
tild_status tild_batch_set_wait_limit(tild_batch* batch, int64_t wait_ns, int extra);

/* Description of the last error on this context (or, when ctx is NULL, of
 * the last failed tild_create, tild_batch_* call or
 * tild_spread_density_noalloc). Never NULL. */
const char* tild_last_error(tild_ctx* ctx);

/*
 * Allocation-free density assignment (the paper has no counterpart: this is
 * an interface for callers that cannot allocate device memory, such as code
 * running while a framework's caching allocator owns all device memory,
 * plug-ins held to a fixed memory budget, or loops where an allocation, which
 * can synchronise the device, is not acceptable).
 *
 * Computes the same species densities as tild_get_density, in FP32, for one
 * set of beads, without a context and without allocating: the 64-bit
 * fixed-point scratch grid is a static device array of 2 * 64^3 points
 * (4 MiB) that every GPU which loads this library holds until the process
 * exits.
 *   xyz      device, [n_beads][3] FP32 positions (wrapped into [0, L) here).
 *   species  device, [n_beads] bytes: 0 = A, anything else = B.
 *   L        cubic box edge (> 0).
 *   n        grid points per edge: a power of two in [8, 64]; larger grids
 *            return TILD_EINVAL (the scratch is sized for 64^3).
 *   pmeorder assignment order 1..4.
 *   rho_out  device, [2][n][n][n] FP32 output (species A then B, [z][y][x]).
 *   stream   cudaStream_t to order the work on (NULL = legacy default stream).
 * Work is asynchronous on `stream`. Every call looks up the device address
 * of the scratch array on the current device (a host-side lookup). CUDA
 * loads a library's device code lazily by default: the first call on each
 * device then places this file's code and the 4 MiB scratch array on that
 * device, which takes device memory once. Make that first call during
 * set-up, before any stream capture; later calls allocate nothing. Every
 * call shares the one
 * scratch array, which keeps the previous call's contents; each call clears
 * the part it uses first. Calls whose work overlaps on the GPU (other
 * streams, other host threads) race on the scratch and must be serialised
 * by the caller. Errors: TILD_EINVAL (NULL pointer, bad size or order),
 * TILD_EDEVICE (a CUDA call failed); text in tild_last_error(NULL).
 */
tild_status tild_spread_density_noalloc(const float* xyz, const unsigned char* species, int64_t n_beads, double L,
                                        int n, int pmeorder, float* rho_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TILD_H */
