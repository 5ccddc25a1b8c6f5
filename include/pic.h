/*
 * pic.h -- C ABI of the GB300 electrostatic PIC/MCC library (libpic_gb300.so).
 *
 * The library advances the plasma domain of the coupled cathode-plasma model of
 * Koitermaa et al. ("Coupled simulation of plasma-surface interactions during
 * early stages of vacuum arcing"): superparticles (electrons, Cu neutrals,
 * Cu+ ions) injected from the cathode, moved by the electric field of Poisson's
 * equation Eq. (1) with Dirichlet electrode potentials, colliding by Monte Carlo
 * collisions with probability Eq. (4), P = 1 - exp(-u n sigma(E) dt), and leaving
 * the domain at the electrodes (the PIC/MCC paragraph of the model description
 * and Appendix A, particle transfer).
 *
 * One step n -> n+1 of an instance runs, on the GPU, in this order:
 *   inject (surface sources)  -> cell sort (every sort_interval steps)
 *   -> cloud-in-cell deposit  -> Poisson solve (multigrid-preconditioned CG)
 *   -> field gather + leapfrog push + absorption + MCC -> ionization resolve
 *   -> compaction.
 *
 * Conventions
 *  - SI units throughout; cross-section energies in eV.
 *  - Grid: nx x ny x nz cells of side h. Nodes i in [0,nx) and j in [0,ny) are
 *    periodic, k in [0,nz]; k = 0 is the cathode (phi_cathode_V), k = nz the anode
 *    (phi_anode_V). Node and cell arrays are laid out [k][j][i] (i fastest):
 *    nodes (nz+1)*ny*nx, cells nz*ny*nx.
 *  - Every entry point returns a pic_status. Inputs are copied before return;
 *    the library owns all device memory of a handle. After an error the
 *    handle keeps its last consistent state where possible; otherwise it
 *    reports PIC_ESTATE until destroyed. pic_last_error() gives text.
 *  - All GPU work is enqueued on the stream given to pic_create (a
 *    cudaStream_t passed as void*, e.g. torch.cuda.current_stream().cuda_stream;
 *    NULL = legacy default stream). Calls that return data to host memory
 *    synchronise that stream.
 *  - A handle is not thread-safe; distinct handles are independent.
 *  - pids (superparticle identifiers) are 32-bit and assigned monotonically:
 *    preloaded particles in call order, then per step the injected particles
 *    in (source, k) order, then secondary electrons in parent-pid order.
 */
#ifndef PIC_GB300_H
#define PIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PIC_MAX_SPECIES 8
#define PIC_MAX_XSEC 8
#define PIC_MAX_SOURCES 16

typedef struct pic_handle pic_handle; /* opaque */

typedef enum {
  PIC_OK = 0,
  PIC_EINVAL = -1,     /* invalid argument or configuration */
  PIC_ENOMEM = -2,     /* device or host allocation failed */
  PIC_ECAPACITY = -3,  /* a species store (or the event buffer) overflowed; the step's
                          state is kept but the overflowing particles were dropped */
  PIC_ENOCONV = -4,    /* Poisson solve hit cg_maxit; non-fatal, phi is used */
  PIC_ECUDA = -5,      /* a CUDA call failed */
  PIC_ETIMEOUT = -6,   /* a bounded device-side wait gave up */
  PIC_ESTATE = -7      /* handle unusable after an earlier fatal error */
} pic_status;

enum { PIC_ELECTRON = 0, PIC_NEUTRAL = 1, PIC_ION = 2 };
enum { PIC_XS_IONIZATION = 0, PIC_XS_ELASTIC = 1, PIC_XS_CHARGE_EXCHANGE = 2 };
enum { PIC_FP64 = 0, PIC_MIXED = 1 };
/* PIC_WARM_UNET: the instance is meant to start its solves from the learned
 * warm start attached with pic_set_warm_unet (include/unet.h; a network handle
 * cannot live in this plain-data configuration); until one is attached it
 * starts from the previous potential, as PIC_WARM_PREV. */
enum { PIC_WARM_PREV = 0, PIC_WARM_ZERO = 1, PIC_WARM_UNET = 2 };
enum { PIC_FIELD_RHO = 0, PIC_FIELD_PHI = 1, PIC_FIELD_NCOUNT = 2 };

/* One species of superparticles (PIC/MCC paragraph: SPs of weight w_SP). */
typedef struct {
  double charge_C;  /* charge of one physical particle */
  double mass_kg;
  double weight;    /* physical particles per superparticle (> 0) */
  int32_t role;     /* PIC_ELECTRON | PIC_NEUTRAL | PIC_ION */
  int64_t capacity; /* maximum superparticles held; >= 1 */
} pic_species;

/* One collision channel of Eq. (4). The table is copied at pic_create.
 * sigma(E) = 0 for E <= threshold_eV; n == 1: constant sigma_m2[0];
 * n >= 2: E_eV strictly increasing, linear interpolation on E_i <= E < E_{i+1},
 * clamped to the end values outside [E_0, E_{n-1}].
 * IONIZATION: projectile (electron) + target (neutral) -> 2 projectiles + product
 *   (ion); the weights of projectile, target and product must be equal.
 * ELASTIC: projectile (electron) scattered isotropically by target, speed kept.
 * CHARGE_EXCHANGE: resonant charge exchange, one of the MCC collisions of the
 *   PIC/MCC paragraph with Eq. (4): projectile (ion) + target (neutral of the
 *   same element) -> the ion continues as a neutral of species `product` (which
 *   must be the target species), the neutral continues as an ion of the
 *   projectile species; both keep position and velocity. u in Eq. (4) is the
 *   ion speed (neutral at rest), E = m_ion u^2 / 2. Weights of projectile and
 *   target must be equal; threshold_eV >= 0. Ionization and charge exchange
 *   draw their victims from one pool: they must share the target species, and
 *   the exchange's projectile must be the ionization's product.
 * The victim of an event (ionization or charge exchange) is a target
 * superparticle in the primary's cell at x^n: per cell, events in increasing
 * primary pid take the targets in increasing Philox key; an event left without
 * one is suppressed. */
typedef struct {
  int32_t kind;
  int32_t projectile, target, product; /* species indices */
  double threshold_eV;
  int32_t n;
  const double* E_eV;
  const double* sigma_m2;
} pic_xsec;

/* One independent instance (grid, physics, species, collisions). */
typedef struct {
  int32_t nx, ny, nz;      /* cells; nx, ny >= 1, nz >= 2 */
  double h;                /* cell side (m) */
  double dt;               /* PIC time step (s) */
  double phi_cathode_V;    /* Dirichlet potential of the plane k = 0 */
  double phi_anode_V;      /* Dirichlet potential of the plane k = nz */
  double rho_background;   /* uniform background charge density (C/m^3) */
  int32_t sort_interval;   /* cell sort every this many steps (0 = never) */
  double cg_rtol;          /* stop when ||r||_2 <= cg_rtol ||b||_2 */
  int32_t cg_maxit;        /* iteration limit of the solve (PIC_ENOCONV beyond) */
  int32_t precision;       /* PIC_FP64 | PIC_MIXED */
  uint64_t seed;           /* Philox4x32-10 key */
  int32_t nspecies;        /* 1..PIC_MAX_SPECIES */
  const pic_species* species;
  int32_t nxsec;           /* 0..PIC_MAX_XSEC */
  const pic_xsec* xsec;
  int32_t warm_start;      /* PIC_WARM_PREV (previous phi) | PIC_WARM_ZERO | PIC_WARM_UNET */
  int32_t variable_weights; /* 0 | 1: superparticles carry integer multiplicities
                               (pic_inject_particles_m); see below */
} pic_instance_cfg;

/* Moments of one instance (a11). Cumulative counters run from pic_create. */
typedef struct {
  int64_t step;                                   /* steps completed */
  int64_t count[PIC_MAX_SPECIES];                 /* live superparticles */
  int64_t injected[PIC_MAX_SPECIES];              /* cumulative, by sources */
  int64_t absorbed_cathode[PIC_MAX_SPECIES];      /* cumulative, z < 0 */
  int64_t absorbed_anode[PIC_MAX_SPECIES];        /* cumulative, z >= Lz */
  double absorbed_energy_cathode_J[PIC_MAX_SPECIES]; /* cumulative, physical */
  double absorbed_energy_anode_J[PIC_MAX_SPECIES];
  int64_t ionizations, elastic, suppressed;       /* cumulative MCC events */
  int32_t cg_iters;                               /* last solve */
  double cg_resid_rel;                            /* last solve, true ||r||/||b|| */
  double total_charge_C;                          /* sum q w N over species */
  double kinetic_J[PIC_MAX_SPECIES];              /* sum (1/2) m w |v|^2 */
  double field_energy_J;                          /* (1/2) eps0 h sum_edges (dphi)^2 */
  double charge_to_cathode_C;                     /* absorbed in the last step */
  double charge_to_anode_C;
  uint32_t next_pid;
  int32_t error_flags;                            /* device-side error bits seen, and
                                                     PIC_FLAG_NONFINITE */
  int64_t pushed[PIC_MAX_SPECIES];                /* cumulative particle pushes (one per
                                                     live particle per step) */
  double anode_V;                                 /* anode potential of the next solve (moves
                                                     only with an external circuit) */
  int64_t charge_exchanges;                       /* cumulative (PIC_XS_CHARGE_EXCHANGE) */
} pic_moments_t;

/* error_flags bit set by pic_moments when a reduced moment (a species' kinetic
 * energy, the field energy, the anode potential or the last residual) is NaN
 * or Inf: some particle velocity or the potential is not finite. */
#define PIC_FLAG_NONFINITE 32

/* Phases of a step, for pic_get_phase_times. */
enum {
  PIC_PH_INJECT = 0,
  PIC_PH_SORT = 1,
  PIC_PH_DEPOSIT = 2,
  PIC_PH_SOLVE = 3,
  PIC_PH_EFIELD = 4,
  PIC_PH_PUSH_ELECTRON = 5, /* gather/push/absorb/MCC of electron species */
  PIC_PH_PUSH_ION = 6,
  PIC_PH_PUSH_NEUTRAL = 7,
  PIC_PH_RESOLVE = 8,
  PIC_NPHASES = 9
};

/* Create n_instances independent instances on the current CUDA device: the
 * plasma domain of the PIC/MCC paragraph (superparticles of the species in
 * cfgs[i].species, the collision channels of Eq. (4) in cfgs[i].xsec) between a
 * cathode and an anode held at the Dirichlet potentials of Eq. (1) (the setup
 * paragraph after Eq. (4): grounded cathode, anode at V0).
 * cfgs: array of n_instances configurations (copied). cuda_stream: the stream
 * all work is enqueued on. Errors: PIC_EINVAL (bad geometry, species, tables,
 * weights), PIC_ENOMEM, PIC_ECUDA. */
pic_status pic_create(const pic_instance_cfg* cfgs, int32_t n_instances, void* cuda_stream,
                      pic_handle** out);

/* Superparticle injection of the PIC/MCC paragraph (emitted electrons,
 * evaporated or sputtered neutrals entering the plasma at the surface).
 * Add (flux > 0) or remove (flux == 0) a persistent surface source of species
 * `species` on the cathode: a disk of radius radius_m centred at (cx, cy).
 * Every step it injects floor(acc) superparticles, acc += flux pi R^2 dt / w,
 * uniform on the disk with a half-Maxwellian velocity at temperature T_K
 * (vx, vy ~ N(0, kT/m), vz = |N(0, kT/m)|) and z = U vz dt. The carry
 * accumulator acc lives on the device, where each step updates it (in FP64,
 * the formula above); it is read back when the source list changes and by
 * pic_save. Up to
 * PIC_MAX_SOURCES sources per instance; a source with the same (species, cx,
 * cy, radius) is replaced and keeps its carry. */
pic_status pic_inject(pic_handle* h, int32_t inst, int32_t species, double cx, double cy,
                      double radius_m, double flux_m2s, double T_K);

/* Particle transfer into the plasma (Appendix A: atoms or clusters leaving the
 * surface model become superparticles of the PIC system); also the preload of
 * a population. Append n superparticles of `species` (host arrays x[n][3],
 * v[n][3], copied; v is taken as v^{n-1/2}). Positions must lie in [0,Lx) x [0,Ly) x [0,Lz).
 * pids continue from next_pid in array order. PIC_ECAPACITY if the store
 * would overflow (nothing is appended then). */
pic_status pic_inject_particles(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                                const double* x, const double* v);

/* Variable weights (the PIC/MCC paragraph's superparticles of weight w_SP,
 * with the weight per particle an integer multiple mw >= 1 of the species'
 * weight). Only for an instance created with variable_weights = 1.
 * The particle's deposit, neutral count, absorbed charge and energy,
 * kinetic energy and total charge are weighted by mw; the counts of
 * superparticles and events are not. An ionization or charge exchange moves
 * ms = min(mw of the primary, mw of the victim) physical multiples: the partner
 * with more keeps the rest in place, and the part that changes species
 * becomes a new superparticle of multiplicity ms with a pid of its own.
 * Successful events are numbered r: ionizations by primary pid, then
 * charge exchanges by primary pid. The secondary electron takes pid0 + r, the
 * victim's new ion pid0 + ns + 2r, and the exchanging ion's new neutral pid0 +
 * ns + 2r + 1, where pid0 is next_pid before the step and ns the successful
 * events. next_pid advances by 3 ns. A primary electron that moves less than
 * its whole multiplicity loses the ionization energy with probability ms / mw
 * (the second uniform of the ionization's second draw): energy is conserved on
 * average, charge and particle numbers exactly. Checkpoints (pic_save)
 * carry the multiplicities.
 * pic_inject_particles_m: as pic_inject_particles, with mw[n] (host, copied).
 * PIC_EINVAL if mw is NULL or an mw[i] is 0 or above 2^24, or above 1 on an
 * instance without variable weights. The multiplicities of the neutrals in one
 * cell must sum below 2^31 (the per-cell counts are int32). The call
 * synchronises the stream.
 * pic_get_multiplicity: the multiplicities of a species' live particles in the
 * order pic_get_particles gives (cap, *n and errors as there). */
pic_status pic_inject_particles_m(pic_handle* h, int32_t inst, int32_t species, int64_t n,
                                  const double* x, const double* v, const uint32_t* mw);
pic_status pic_get_multiplicity(pic_handle* h, int32_t inst, int32_t species, int64_t cap, int64_t* n,
                                uint32_t* mw);

/* Advance every instance by nsteps PIC steps of length dt (the PIC/MCC
 * paragraph: the field of Eq. (1) from the deposited charge, the push by
 * electric forces, collisions with the probability of Eq. (4), absorption at
 * the electrodes; the order is listed at the top of this file). Asynchronous on
 * the stream. The
 * returned status covers argument checks, launch errors and the device error
 * flags of earlier completed steps (PIC_ECAPACITY, PIC_ENOCONV, PIC_ETIMEOUT). */
pic_status pic_step(pic_handle* h, int32_t nsteps);

/* Fill *out (caller-owned) with the moments of instance inst: the counts,
 * collision events (Eq. 4), absorbed particles and energies, charge and energies
 * that the PIC/MCC paragraph's quantities are summed from. Synchronises. */
pic_status pic_moments(pic_handle* h, int32_t inst, pic_moments_t* out);

/* Release all device and host memory of the handle (NULL is accepted). Pure
 * resource management: the paper has no counterpart. */
pic_status pic_destroy(pic_handle* h);

/* Text of the last error on this handle (static storage, never NULL). */
const char* pic_last_error(pic_handle* h);

/* Device memory from the caller's allocator (a pool such as PyTorch's caching
 * allocator) instead of cudaMalloc / cudaFree. Resource management only: the
 * paper has no counterpart. Process-wide: every device buffer that a PIC or
 * U-Net handle created afterwards takes (stores, grids, solver, staging,
 * scratch) comes from alloc(bytes, ctx) and goes back through
 * free_fn(ptr, ctx); before each free_fn the library synchronises the device,
 * as cudaFree does. alloc must return memory of the current device aligned to
 * 256 bytes, or NULL (the library call then fails with PIC_ENOMEM or
 * PIC_ECUDA). Both NULL restores cudaMalloc / cudaFree. PIC_EINVAL if exactly
 * one is NULL; PIC_ESTATE while any PIC or U-Net handle is alive (memory must
 * return to the allocator it came from). Not thread-safe against concurrent
 * handle creation. */
typedef void* (*pic_alloc_fn)(size_t bytes, void* ctx);
typedef void (*pic_free_fn)(void* ptr, void* ctx);
pic_status pic_set_allocator(pic_alloc_fn alloc, pic_free_fn free_fn, void* ctx);

/* ---- inspection, test and tuning hooks (synchronous) -----------------------
 * These have no counterpart in the paper: they read or set the state that the
 * steps above work on, so that tests can compare it with the oracle and
 * callers can tune or observe a run. Each that returns a pic_status gives
 * PIC_EINVAL for a NULL handle, an instance or species index out of range, or
 * a NULL output where one is required, and PIC_ECUDA if a CUDA call fails. */

/* Number of live superparticles of a species. */
pic_status pic_get_count(pic_handle* h, int32_t inst, int32_t species, int64_t* n);

/* Copy a species out in store order: pid[n], x[n][3], v[n][3] (any may be
 * NULL). cap is the capacity of the caller's arrays; *n receives the count
 * (PIC_EINVAL if cap < count, nothing copied). Right after a cell sort the
 * store order is (cell, pid). Positions and velocities are FP64 in both
 * precisions (in PIC_MIXED they are converted from cell + FP32 offset). */
pic_status pic_get_particles(pic_handle* h, int32_t inst, int32_t species, int64_t cap, int64_t* n,
                             uint32_t* pid, double* x, double* v);

/* Copy a grid array to host memory: PIC_FIELD_RHO (double, nodes, the charge
 * density of the last deposit), PIC_FIELD_PHI (double, nodes, the last solve),
 * PIC_FIELD_NCOUNT (int32, cells, neutral counts of species `species` at the
 * last deposit; for RHO/PHI `species` is ignored). */
pic_status pic_get_field(pic_handle* h, int32_t inst, int32_t which, int32_t species, void* host_out);

/* Replace phi (double, nodes) of an instance, e.g. to set the warm start. */
pic_status pic_set_phi(pic_handle* h, int32_t inst, const double* host_phi);

/* Solve Eq. (1) for a given charge density with the instance's solver and
 * electrodes: rho and phi are host arrays over the nodes; phi's interior is
 * the initial guess on entry and the solution on exit. Does not touch the
 * instance's own phi. iters/resid_rel may be NULL. */
pic_status pic_solve(pic_handle* h, int32_t inst, const double* rho, double* phi, int32_t* iters,
                     double* resid_rel);

/* Sort every species of an instance by (cell, pid) now. */
pic_status pic_sort_now(pic_handle* h, int32_t inst);

/* Per-cell offsets of the last cell sort of a species: ncells + 1 int64. */
pic_status pic_get_cell_start(pic_handle* h, int32_t inst, int32_t species, int64_t* host_out);

/* Successful ionizations of the last step: rows (primary pid, victim pid,
 * secondary pid) in increasing primary pid; cap rows at most, *n receives the
 * number. Charge exchanges are not listed (their count is a moment). */
pic_status pic_get_ionization_log(pic_handle* h, int32_t inst, int64_t cap, int64_t* n, uint32_t* rows);

/* Philox4x32-10 on the device for n consecutive counters
 * (c0 + i, c1, c2, c3) with key (k0, k1); out[4 n] host array. */
pic_status pic_philox(pic_handle* h, int64_t n, const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t* out);

/* Test mode for the collision rates of Eq. (4): with density_m3 > 0 every
 * collision channel sees this fixed target density instead of the neutral
 * counts, and ionizations and charge exchanges are counted without consuming
 * neutrals, creating or converting particles. 0 restores the normal mode. */
pic_status pic_set_mcc_background(pic_handle* h, int32_t inst, double density_m3);

/* ---- external circuit -------------------------------------------------------
 * The paper puts a serial RC circuit (R = 1 kOhm, C = 1 pF) between the
 * electrodes and treats the voltage as constant on its time scale (the
 * paragraph describing the simulated system).
 * This call makes it dynamic: a source V0 charges the anode through R, the gap
 * holds capacitance C, and the charge the anode collects in a step (electrons
 * and ions absorbed there, pic_moments_t.charge_to_anode_C) flows onto it, once
 * per step after the push:
 *   V <- V + (dt (V0 - V) / R + Q_anode) / C.
 * The next step's Poisson solve uses V at the anode plane (pic_moments_t.anode_V
 * reports it); the cathode stays at phi_cathode_V. R <= 0 or C <= 0 switches the
 * circuit off, and the anode then keeps its current potential. PIC_EINVAL for a
 * NaN argument. */
pic_status pic_set_circuit(pic_handle* h, int32_t inst, double R_ohm, double C_farad, double V0);

/* ---- surface coupling: ions that bombard the cathode ----------------------
 * In the paper's coupled model ions that reach the cathode are handed to the
 * atomistic surface model, where they heat or sputter it (the PIC/MCC
 * paragraph after Eq. 4, and the particle transfer of Appendix A). These two
 * calls export them for such a model: every superparticle of an ion species
 * (PIC_ION) absorbed at the cathode (z^{n+1} < 0, step a7) is logged with its
 * pid, species, the step in which it crossed, the point where its straight
 * path from x^n to x^{n+1} meets the plane z = 0 (x and y wrapped into the
 * box), and v^{n+1/2}.
 *
 * pic_set_hit_log: log from the next step on, keeping at most `capacity` hits
 * between two reads (device memory allocated here; 0 switches the log off and
 * frees it). Synchronises the instance. PIC_EINVAL for capacity < 0,
 * PIC_ENOMEM if the log cannot be allocated (the log is then off). */
pic_status pic_set_hit_log(pic_handle* h, int32_t inst, int64_t capacity);

/* pic_get_hits: the hits logged since the previous call (or since the log was
 * switched on), ordered by (step, pid), after which the log is empty.
 * Synchronises the instance. Caller-owned outputs with room for `cap` hits:
 * pid[cap], species[cap], step[cap], x[3 cap] (crossing point, z = 0),
 * v[3 cap] (m/s), ke_eV[cap] (1/2 m |v|^2 of one physical ion, in eV).
 * *n receives the number of hits returned, *lost the number beyond the log's
 * capacity since the previous read (those are not kept; which hits are kept
 * when the capacity overflows is not specified). PIC_EINVAL if no log is on,
 * if an output pointer is null, or if more than `cap` hits are waiting (then
 * nothing is copied and the log is kept). */
pic_status pic_get_hits(pic_handle* h, int32_t inst, int64_t cap, int64_t* n, int64_t* lost, uint32_t* pid,
                        int32_t* species, int64_t* step, double* x, double* v, double* ke_eV);

/* Checkpoint and resume of one instance (no counterpart in the paper: the
 * state of a long run, kept so that it can stop and continue). pic_save writes
 * to `path` the live particles of every species in increasing pid (the store's
 * own representation: FP64 x, v; or cell, FP32 offsets and velocities of the
 * mixed store; with variable weights also the multiplicities), the potential
 * (and the mixed solver's FP32 state), the
 * cumulative counters, step and next pid, the surface sources with their carry
 * accumulators, the sort interval, the external circuit and the background
 * test mode. The hit log and the ionization log are outputs, not state, and
 * are not saved. pic_load reads such a file into an instance created with the
 * same grid, precision, electrode potentials, time step, seed, species and
 * variable-weights setting; it
 * checks the whole file first and leaves the instance unchanged on any error
 * (PIC_EINVAL: unreadable, not a checkpoint, a different configuration, or
 * truncated; PIC_ECAPACITY: more particles than a species holds). Draws are
 * counter-based, so a resumed run takes the same decisions as an
 * uninterrupted one; its first step deposits from scratch, so floating-point
 * sums may differ in the last bits. Both synchronise the caller's stream. */
pic_status pic_save(pic_handle* h, int32_t inst, const char* path);
pic_status pic_load(pic_handle* h, int32_t inst, const char* path);

/* Cell sort interval of one instance from now on (a2: the store is sorted when
 * the step index is a multiple of it; 0 never sorts). The sort only reorders
 * particles, so results do not depend on it beyond rounding; it trades the
 * sort's cost against the locality of the deposit and gather (the
 * autotuner in the Python package picks it per instance).
 * PIC_EINVAL for a negative interval or a bad instance. */
pic_status pic_set_sort_interval(pic_handle* h, int32_t inst, int32_t interval);

/* Launch shape of one instance's particle kernels (push, scratch deposit,
 * injection, resolve) from now on: blocks_per_sm thread blocks per SM (1..32,
 * default 8), each striding over the store. Like the sort interval it changes
 * no result beyond rounding (the order of compacted particles and of deposit
 * sums), only how the work is spread (the autotuner picks it with the sort
 * interval). PIC_EINVAL outside 1..32 or for a bad instance. */
pic_status pic_set_launch_shape(pic_handle* h, int32_t inst, int32_t blocks_per_sm);

/* Phase timing: with on != 0 every later step records CUDA events on the
 * handle's stream around each phase (and waits for them at the end of the step),
 * and marks each phase as an NVTX range for timeline profilers.
 * pic_get_phase_times adds up, per phase, the elapsed milliseconds (ms[PIC_NPHASES])
 * and the number of timed phase executions (count[PIC_NPHASES]) since profiling
 * was switched on; either pointer may be NULL. Switching on resets the sums. */
pic_status pic_set_profiling(pic_handle* h, int32_t on);
pic_status pic_get_phase_times(pic_handle* h, int32_t inst, double* ms, int64_t* count);

/* Launch operations the library issued to the GPU in this process so far: a
 * kernel launch counts one, and so does a graph launch (a recorded solve or a
 * recorded step), however many kernels the graph runs. */
uint64_t pic_launch_count(void);

/* Kernels run by those operations: a graph launch adds the kernel nodes it was
 * recorded with, the body of a device-side loop (the solver's iterations)
 * counted once, so this is a lower bound when a solve iterates. */
uint64_t pic_kernel_count(void);

/* ---- solve without allocating ----------------------------------------------
 * Not in the paper: an entry point for callers that cannot allocate device
 * memory while they run (programs that hand out all device memory from their
 * own pool at start-up, or that must keep a fixed footprint between coupling
 * steps). It solves the node-grid Poisson problem that pic_solve solves --
 * 7-point operator, periodic x/y, Dirichlet planes phi(k=0) = phi_cathode_V and
 * phi(k=nz) = phi_anode_V -- by unpreconditioned conjugate gradients,
 * with every work vector in one fixed array inside the library (file-scope
 * __device__ storage of PIC_STATIC_MAX_UNKNOWNS-sized vectors, about 8 MiB,
 * held by every GPU that loads the library until the process exits). It calls
 * no cudaMalloc, cudaFree or other allocating routine.
 *  rho_dev: device array of (nz+1)*ny*nx doubles, layout [k][j][i] (read only).
 *  phi_dev: device array of the same size; its interior (k = 1..nz-1) is the
 *           initial guess on entry; on return it holds the solution and the
 *           electrode planes hold their potentials. Caller-owned.
 *  Iterates until the recursive residual reaches rtol ||b|| or maxit
 *  iterations have run, then recomputes the true residual b - A phi; the status
 *  follows that true residual, which at very tight rtol can sit just above the
 *  recursive one. The true relative residual is reported in *resid_rel and the
 *  iteration count in *iters (either may be NULL). rho = 0 with both electrodes
 *  at 0 V gives the zero solution after 0 iterations.
 * Returns PIC_EINVAL for bad arguments or nx*ny*(nz-1) > PIC_STATIC_MAX_UNKNOWNS,
 * PIC_ENOCONV if the true residual is above rtol, PIC_ECUDA if a launch or copy
 * fails; pic_last_error(NULL) then says which. The first call on a device looks up the address of
 * the fixed array on that device (cudaGetSymbolAddress, with that device
 * current). No call can be captured into a CUDA graph: every iteration
 * synchronises the stream (below). All calls share
 * the array and it keeps the last call's contents (each call writes every
 * vector before reading it); calls that overlap on the GPU -- on different
 * streams or from different host threads on the same device -- race on it.
 * Work runs on cuda_stream; the call reads the residual back and synchronises
 * that stream once per iteration. */
#define PIC_STATIC_MAX_UNKNOWNS (1 << 18)
pic_status pic_poisson_solve_static(int32_t nx, int32_t ny, int32_t nz, double h, double phi_cathode_V,
                                    double phi_anode_V, const double* rho_dev, double* phi_dev, double rtol,
                                    int32_t maxit, void* cuda_stream, int32_t* iters, double* resid_rel);

/* Library version string. */
const char* pic_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PIC_GB300_H */
