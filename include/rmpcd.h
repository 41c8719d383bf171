/*
 * rmpcd.h -- C ABI of the GB300 (sm_103a) MPCD solvent collision-interval update.
 *
 * Method: Multiparticle Collision Dynamics solvent coupled to colloids by MD,
 * as described by de Buyl, Huang & Deprez, "RMPCDMD" (arXiv:1608.04904):
 * §1.1 (solvent + colloids in a cuboid, velocity-Verlet, no solvent-solvent
 * potential, bulk RMPCD reactions), §1.4 (SRD collision rule, Anderson
 * thermostat, random grid shift, body force, bounce-back walls with virtual
 * particles, WCA colloid-solvent potential, Verlet/cell lists sharing the MPCD
 * sort, exact RATTLE for the dimer, counter-based RNG, temperature estimator),
 * §1.5 (catalytic A -> B at the dimer's C sphere, the bead-built Janus
 * particle) and Appendix A (parameters).
 *
 * Conventions for every entry point:
 *   - Every call returns an rmpcd_status; no call prints or aborts.
 *   - Work is queued on the CUDA stream given to rmpcd_create and is
 *     asynchronous, except where a call says it synchronises.  Errors raised
 *     by kernels (bucket overflow, skin violation, a look-back that timed out)
 *     are latched on the device and returned by the next synchronising call
 *     (rmpcd_sync, rmpcd_get_state, rmpcd_observables, rmpcd_profile).
 *   - Host buffers passed in are copied before the call returns (or, for
 *     on_device = 0 outputs, filled before it returns); the library never keeps
 *     a caller's pointer.  All device memory of a system is owned by the
 *     library and released by rmpcd_destroy.
 *   - rmpcd_last_error() gives a one-line description of the last failure.
 *
 * Units: cell side a = 1, solvent mass m = 1.  Solvent flags: bit 0 = species
 * B (else A), bit 1 = catalytic tag (an A particle currently inside a
 * catalytic colloid's interaction range).
 */
#ifndef RMPCD_H
#define RMPCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmpcd_system rmpcd_system;

typedef enum {
    RMPCD_OK = 0,
    RMPCD_EINVAL = 1,     /* invalid argument or parameter combination          */
    RMPCD_ECUDA = 2,      /* a CUDA runtime call failed                          */
    RMPCD_ENOMEM = 3,     /* device allocation failed                            */
    RMPCD_EOVERFLOW = 4,  /* a cell beyond 1536 particles, or the overflow list full */
    RMPCD_ESKIN = 5,      /* a colloid moved further than skin in one interval   */
    RMPCD_ETIMEOUT = 6,   /* a bounded device wait ran out (state is invalid)    */
    RMPCD_ESTATE = 7      /* call not valid in the current state                 */
} rmpcd_status;

typedef enum { RMPCD_FP64 = 0, RMPCD_MIXED = 1 } rmpcd_precision;

/* Parameters of one replica (one independent system).  §1.4, Appendix A. */
typedef struct {
    int32_t L[3];          /* box sides in cells, each in [2, 1023]                      */
    int32_t walls;         /* 1: stick walls at z = 0 and z = L[2] (bounce-back + virtual particles) */
    int32_t rho_wall;      /* particles per cell that virtual particles fill wall cells up to */
    int32_t n_md;          /* velocity-Verlet sub-steps per collision interval (dt = tau / n_md) */
    int32_t n_slabs;       /* number of Anderson-thermostat (MPC-AT) slabs, 0..4          */
    int32_t n_solvent;     /* solvent particles of this replica                          */
    int32_t n_colloids;    /* colloids of this replica                                   */
    int32_t n_bonds;       /* rigid bonds (RATTLE) between this replica's colloids       */
    double kT;             /* solvent temperature                                        */
    double alpha;          /* SRD rotation angle in radians                              */
    double tau;            /* collision interval                                         */
    double g[3];           /* body acceleration on the solvent (g[2] must be 0 with walls) */
    double bulk_rate;      /* bulk B -> A rate k; 0 disables the bulk reaction            */
    double cat_prob;       /* probability of A -> B when a tagged A leaves catalytic range */
    double skin;           /* bound on colloid displacement per interval                 */
    double slab_x0[4], slab_x1[4], slab_kT[4];  /* MPC-AT slabs: cells with x0 <= cx < x1 */
    double cc_eps, cc_sigma, cc_rc;             /* colloid-colloid LJ; cc_rc = 0 disables  */
    uint64_t seed;         /* key of the counter-based RNG                               */
    int32_t res_y[4];      /* species reservoirs of the chemotactic set-up (§1.5
                            * chemotactic_cell): after every collision the particles of
                            * a cell whose y column on the collision grid lies in
                            * [res_y[0], res_y[1]) become A, in [res_y[2], res_y[3]) B
                            * (tags cleared); empty ranges (all 0) disable it          */
} rmpcd_params;

/* One colloid (§1.1: mass, position, velocity; §1.4: WCA sigma and per-species
 * epsilon).  x is kept unwrapped. */
typedef struct {
    double x[3], v[3];
    double mass, sigma, eps_A, eps_B;
    int32_t catalytic;     /* 1: converts A -> B (§1.5)                                */
    int32_t pad;
} rmpcd_colloid;

/* A rigid bond |x_a - x_b| = d held by exact RATTLE (§1.4, dimer motor).
 * a and b index the replica's own colloids. */
typedef struct {
    int32_t a, b;
    double d;
} rmpcd_bond;

/* A rigid composite colloid: the Janus particle of §1.5, a network of WCA
 * beads that moves as one rigid body (§1.4 holds the network together by
 * constraints; a rigid body keeps every bead distance exactly).  State: the
 * centre of mass x (unwrapped) and its velocity v, the unit quaternion
 * q = (w, x, y, z) taking the body frame to the space frame, and the angular
 * momentum l in the body frame.  Every bead has mass bead_mass and WCA sigma
 * `sigma` (cut-off 2^(1/6) sigma). */
typedef struct {
    double x[3], v[3];
    double q[4];
    double l[3];
    double bead_mass, sigma;
    int32_t n_beads;
    int32_t pad;
} rmpcd_body;

/* One bead: position relative to the centre of mass in the body's principal
 * frame, WCA epsilon towards A and B solvent, catalytic flag (§1.5). */
typedef struct {
    double b[3];
    double eps_A, eps_B;
    int32_t catalytic;
    int32_t pad;
} rmpcd_bead;

#define RMPCD_MAX_BEADS 1024

/* One bead of a bead network held by iterative RATTLE (the paper's Janus
 * integrator, §1.4): position (unwrapped, box frame) and velocity, mass, WCA
 * epsilon towards A and B solvent, catalytic flag (§1.5). */
typedef struct {
    double x[3], v[3];
    double mass, eps_A, eps_B;
    int32_t catalytic;
    int32_t pad;
} rmpcd_net_bead;

#define RMPCD_MAX_NET_BEADS 512

/* Observables of one replica after the last collision (§1.4 temperature
 * estimator; totals accumulated in FP64). */
typedef struct {
    double temperature;    /* 1/(3 N_c) sum_cells 1/(N-1) sum (v - v_cell)^2, cells with N >= 2 */
    double momentum[3];    /* total solvent momentum                                    */
    double kinetic;        /* total solvent kinetic energy                              */
    int64_t n_cells_used;  /* N_c                                                       */
    int64_t n_B;           /* solvent particles of species B                            */
    int64_t n_solvent;
    uint32_t step;         /* collision index the values belong to                      */
    uint32_t pad;
} rmpcd_obs;

/* Create a system of n_replicas independent replicas on the current CUDA
 * device.  params[n_replicas]; colloids and bonds are the replicas' lists
 * concatenated in replica order (params[r].n_colloids / n_bonds entries each;
 * may be NULL when all counts are 0).  precision: rmpcd_precision.
 * bucket_cap: width of a cell's bucket row (1..768), or 0: picked
 * automatically.  A cell's entries past the width go to an overflow list
 * (1024 + n_solvent/16 entries per buffer, read back by the cell pass of the
 * tiles that need it, in canonical order like the rest): a crowded cell is
 * not an error, though a width far below the typical count makes every tile
 * scan the list.  A cell may hold at most 1536 particles (what the cell pass
 * stages at once); beyond that, or with the list full, the run latches
 * EOVERFLOW.  The automatic width (the bucket-width autotuner:
 * 1.25x the count above which a Poisson cell count at the densest replica
 * occurs with probability < 1e-4 per collision, in multiples of 8, then
 * grown to 1.5x the largest count whenever a binning or a run comes within
 * 80 % of it).  stream: a cudaStream_t, or NULL for the legacy default
 * stream.  Solvent state is all zero until rmpcd_set_state.
 * Errors: EINVAL (bad sizes or parameters), ENOMEM, ECUDA. */
rmpcd_status rmpcd_create(rmpcd_system **out, int32_t precision, int32_t n_replicas,
                          const rmpcd_params *params, const rmpcd_colloid *colloids,
                          const rmpcd_bond *bonds, int32_t bucket_cap, void *stream);

/* Device memory that rmpcd_create would allocate for the same arguments: the
 * sum of its device buffers, each rounded up to 256 bytes (the CUDA allocator
 * may round further).  Not included: the CUDA context, captured CUDA graphs,
 * and the bead arrays and lookup grids that rmpcd_set_body adds later.
 * Validates the arguments exactly as rmpcd_create does (bucket_cap 0 is sized
 * by the same autotuner rule) and makes no CUDA call, so it works on a host
 * without a GPU.  bytes: host output.  Errors: EINVAL (same cases as
 * rmpcd_create, or bytes NULL). */
rmpcd_status rmpcd_workspace_size(int32_t precision, int32_t n_replicas, const rmpcd_params *params,
                                  const rmpcd_colloid *colloids, const rmpcd_bond *bonds, int32_t bucket_cap,
                                  size_t *bytes);

/* Release every device buffer of the system.  NULL is accepted. */
void rmpcd_destroy(rmpcd_system *sys);

/* Load the solvent of one replica: x[n][3] and v[n][3] FP64 (row-major,
 * x in [0, L) on periodic axes and [0, L[2]] with walls), flags[n] (may be
 * NULL = all A), n = params.n_solvent.  on_device = 1: the three pointers are
 * device pointers; 0: host pointers.  Particle ids are set to 0..n-1.  Any
 * pending fused-step state is discarded.  Errors: EINVAL, ECUDA. */
rmpcd_status rmpcd_set_state(rmpcd_system *sys, int32_t replica, const double *x, const double *v,
                             const uint8_t *flags, int64_t n, int32_t on_device);

/* Read the solvent of one replica in storage order (which, after any sort
 * or step, is the sorted-cell order of the last collision).  Any output
 * pointer may be NULL.  id[n]: particle ids; cell[n]: key of each particle's
 * cell on the grid of the last sort (-1 before any sort).  Synchronises and
 * returns latched device errors.  Errors: EINVAL, ECUDA, EOVERFLOW, ESKIN, ETIMEOUT. */
rmpcd_status rmpcd_get_state(rmpcd_system *sys, int32_t replica, double *x, double *v, uint8_t *flags,
                             uint32_t *id, int32_t *cell, int64_t n, int32_t on_device);

/* The solvent of every replica in one call: the arrays of rmpcd_set_state /
 * rmpcd_get_state concatenated in replica order (replica r's particles start
 * at the sum of params.n_solvent over the replicas before it; n = that sum
 * over all replicas).  Host arrays travel in one copy each way through a
 * staging area of n particles (allocated on the first host call, freed with
 * the system) with one synchronisation per call, where the per-replica calls
 * synchronise once per replica; device arrays are read or written in place.
 * The results are those of the per-replica calls, replica by replica.
 * rmpcd_set_state_all: flags may be NULL (all A); the host arrays may be
 * reused when it returns.  rmpcd_get_state_all: any output pointer may be
 * NULL; synchronises and returns latched device errors.  Errors: EINVAL (n
 * is not the system's total), ENOMEM (staging area), ECUDA, and for
 * rmpcd_get_state_all EOVERFLOW, ESKIN, ETIMEOUT. */
rmpcd_status rmpcd_set_state_all(rmpcd_system *sys, const double *x, const double *v, const uint8_t *flags,
                                 int64_t n, int32_t on_device);
rmpcd_status rmpcd_get_state_all(rmpcd_system *sys, double *x, double *v, uint8_t *flags, uint32_t *id,
                                 int32_t *cell, int64_t n, int32_t on_device);

/* Order of the cells in storage (§1.2 sorts the particles by cell; §1.4 puts
 * the cells in compact Hilbert order).  RMPCD_ORDER_LINEAR (the default):
 * cell key k = x + L0 (y + L1 z) on the collision grid (z over L[2] + 1
 * layers with walls) is also the cell's place.  RMPCD_ORDER_HILBERT: the
 * cells of each replica are placed by their index on the 3-D Hilbert curve
 * through the smallest enclosing cube of side 2^m (Skilling's transpose
 * method, x the most significant axis), ranked over the box's cells.  The
 * place decides the storage order of a sorted state (rmpcd_get_state), the
 * record rows and the tiles of the cell pass; a cell's draws, its geometry
 * and the cell keys reported keep the key, so every result is the same up to
 * the storage order.  rmpcd_set_cell_order moves a fused run's state back to
 * the flat layout first and drops captured graphs; the Hilbert tables (two
 * ints per cell) are allocated on first use.  rmpcd_cell_places: the place
 * of every key of a grid dims[3] (each in [1, 1023], at most 2^28 cells) in the given order
 * (host memory, dims[0] dims[1] dims[2] entries; no CUDA call).  Errors:
 * EINVAL, ENOMEM, ECUDA. */
#define RMPCD_ORDER_LINEAR 0
#define RMPCD_ORDER_HILBERT 1
rmpcd_status rmpcd_set_cell_order(rmpcd_system *sys, int32_t order);
rmpcd_status rmpcd_get_cell_order(rmpcd_system *sys, int32_t *order);
rmpcd_status rmpcd_cell_places(const int32_t dims[3], int32_t order, int64_t *place);

/* Colloids of one replica (host arrays of params.n_colloids entries). */
rmpcd_status rmpcd_set_colloids(rmpcd_system *sys, int32_t replica, const rmpcd_colloid *c, int32_t n);
rmpcd_status rmpcd_get_colloids(rmpcd_system *sys, int32_t replica, rmpcd_colloid *c, int32_t n);

/* Give one replica a rigid bead body, or replace its body (geometry and
 * state).  The replica must have been created with no colloids, no bonds and
 * no walls.  beads[body->n_beads], 1 <= n_beads <= RMPCD_MAX_BEADS, centred
 * (|sum b| <= 1e-9 n_beads max|b|) and in the principal frame (off-diagonal
 * inertia <= 1e-9 of its trace); bead_mass, sigma > 0; |q| = 1 within 1e-9;
 * the box must hold twice the body's reach (max|b| + 2^(1/6) sigma) plus
 * twice the skin.  M = n_beads bead_mass; principal moments
 * I_k = sum_j bead_mass (|b_j|^2 - b_jk^2).  The body moves by velocity
 * Verlet for x and the principal-axis splitting of the free rotation
 * (turns about axes 1, 2, 3, 2, 1 over dt/2, dt/2, dt, dt/2, dt/2, each by
 * the angle phi with tan(phi/2) = h l_k / (2 I_k)); solvent within
 * reach + |v| tau + |g| tau^2/2 + skin of x takes the MD sub-steps.  Discards
 * a primed fused pipeline; synchronises.  Errors: EINVAL, ENOMEM, ECUDA. */
rmpcd_status rmpcd_set_body(rmpcd_system *sys, int32_t replica, const rmpcd_body *body,
                            const rmpcd_bead *beads);

/* The body of one replica (state as of the last completed interval; beads
 * are not returned).  Synchronises and returns latched device errors.
 * Errors: EINVAL (no body), ECUDA, EOVERFLOW, ESKIN, ETIMEOUT. */
rmpcd_status rmpcd_get_body(rmpcd_system *sys, int32_t replica, rmpcd_body *body);

/* Give one replica a bead network held at fixed link lengths by iterative
 * RATTLE (§1.4: the paper's integrator of the Janus particle; every bead a
 * point mass), or replace it.  FP64 systems only; the replica must have been
 * created with no colloids, bonds or walls and hold no rigid body.
 * beads[n_beads], 1 <= n_beads <= RMPCD_MAX_NET_BEADS; links[n_links] join
 * beads a != b at length d > 0; colors[n_links] >= 0 with no bead twice in one
 * colour.  Each velocity-Verlet sub-step corrects positions (along the link
 * vectors of the sub-step's start) and then velocities (along the current
 * ones), sweeping the links colour by colour -- the links of a colour at once,
 * in the order given within a colour -- until every link holds within tol
 * (|d^2 - |x_a - x_b|^2| <= 2 tol d^2; |(v_a - v_b).(x_a - x_b)| <= tol d),
 * at most max_sweeps sweeps (more latches ESTATE).  Solvent within the beads'
 * reach (largest bead distance from the centre of mass plus 2^(1/6) sigma)
 * + |v| tau + |g| tau^2/2 + skin of the centre of mass takes the MD sub-steps.
 * Discards a primed fused pipeline; synchronises.  Errors: EINVAL, ENOMEM,
 * ECUDA. */
rmpcd_status rmpcd_set_network(rmpcd_system *sys, int32_t replica, const rmpcd_net_bead *beads, int32_t n_beads,
                               const rmpcd_bond *links, const int32_t *colors, int32_t n_links, double sigma,
                               double tol, int32_t max_sweeps);

/* Bead positions and velocities (host arrays of 3 n_beads doubles) of one
 * replica's network, as of the last completed interval.  Synchronises and
 * returns latched device errors.  Errors: EINVAL (no network, wrong count). */
rmpcd_status rmpcd_get_network(rmpcd_system *sys, int32_t replica, double *x, double *v, int32_t n_beads);

/* Collision counter that keys every random draw of the next interval. */
rmpcd_status rmpcd_set_step(rmpcd_system *sys, uint32_t step);
rmpcd_status rmpcd_get_step(const rmpcd_system *sys, uint32_t *step);

/* --- granular steps of one interval (§1.1, §1.4), all replicas ----------- */

/* Interval motion: solvent that may come within a colloid's cut-off during
 * the interval (distance < r_c + |v| tau + |g| tau^2 / 2 + skin) is integrated
 * with the colloids by n_md velocity-Verlet sub-steps under WCA forces, with
 * exact RATTLE on bonds and catalytic A -> B on leaving a catalytic colloid;
 * all other solvent flies freely over tau (body force, bounce-back walls).
 * Does not advance the step counter. */
rmpcd_status rmpcd_stream(rmpcd_system *sys);

/* One velocity-Verlet sub-step of the current interval (the interval of
 * rmpcd_stream, run one sub-step at a time; the paper's MD sub-step, §1.1,
 * dt = tau / n_md).  Sub-step 0 also flies the far particles over tau and
 * collects the particles near a colloid; sub-steps must run in order
 * 0, 1, ..., n_md - 1, and after the last one the state equals that of
 * rmpcd_stream bit for bit (same arithmetic; the colloid forces are exact
 * fixed-point sums).  Between sub-steps rmpcd_get_colloids reads the colloids
 * after sub-step k; the solvent is written back after the last sub-step, and
 * every call other than rmpcd_md_substep, rmpcd_get_colloids, rmpcd_sync and
 * the queries fails with ESTATE until then.  Replicas with fewer sub-steps
 * finish early.  Errors: EINVAL (k outside 0..n_md - 1, rigid bodies), ESTATE
 * (out of order), ECUDA. */
rmpcd_status rmpcd_md_substep(rmpcd_system *sys, int32_t k);

/* Random grid shift of the current step, cell keys and counting sort: storage
 * becomes sorted by cell, the particles of a cell in increasing id order. */
rmpcd_status rmpcd_shift_and_sort(rmpcd_system *sys);

/* Collision on the grid of the current step: SRD rotation by alpha about a
 * random axis per cell; MPC-AT inside slabs; virtual particles in wall cells.
 * Requires the state sorted on that grid (rmpcd_shift_and_sort). */
rmpcd_status rmpcd_collide(rmpcd_system *sys);

/* Bulk B -> A reaction per cell (one B with probability 1 - exp(-k N_B tau)),
 * then the species reservoirs (res_y) if any.  Requires the state sorted on
 * the current grid. */
rmpcd_status rmpcd_react(rmpcd_system *sys);

/* n_intervals full collision intervals (motion, shift, sort, collision,
 * bulk reaction), fused into two kernels per interval; the step counter
 * advances by n_intervals.  Equivalent to the granular sequence
 * stream, shift_and_sort, collide, react, step + 1. */
rmpcd_status rmpcd_step(rmpcd_system *sys, int32_t n_intervals);

/* Observables of one replica on the grid of the last collision (computed by
 * one extra cell pass over the stored state when requested).  Synchronises. */
rmpcd_status rmpcd_observables(rmpcd_system *sys, int32_t replica, rmpcd_obs *out);

/* One bin of a slab profile (rmpcd_profile). */
#define RMPCD_MAX_PROFILE_BINS 512
typedef struct {
    int64_t n;             /* solvent particles in the bin                                */
    int64_t n_B;           /* of which species B                                          */
    double v_sum[3];       /* sum of v_k over the bin, each term rounded to 2^-32         */
    double v2_sum[3];      /* sum of v_k^2 over the bin, each term rounded to 2^-24       */
} rmpcd_profile_bin;

/* Slab profile of one replica's solvent along one axis, for the flow profile
 * v_x(z) between the walls of a Poiseuille set-up and the slab temperatures and
 * species concentrations across a thermal or chemical gradient (paper,
 * §"Applications of RMPCDMD": poiseuille_flow, chemotactic_cell,
 * single_sphere_thermo_trap; the histogram routine of the `common` module).
 * The stored state is read as it is (the positions after the last step or
 * rmpcd_set_state).  Bin b holds the particles with
 * floor(x_axis * n_bins / L[axis]) == b, clamped to 0..n_bins-1 (a particle at
 * x = L[2] on a wall axis lands in the last bin).  The sums are fixed point:
 * every term is rounded to nearest-even on its grid (2^-32 for v_k, 2^-24 for
 * v_k^2) and summed as a 64-bit integer, so the result does not depend on the
 * summation order and is the same on every run; it is exact while
 * |sum v_k| < 2^31 and sum v_k^2 < 2^39 per bin.  Mean flow of a bin:
 * v_sum / n; slab temperature (mass 1, the bin's mean flow removed):
 * sum_k (v2_sum[k] - v_sum[k]^2 / n) / (3 (n - 1)).
 * axis: 0, 1 or 2.  n_bins: 1..RMPCD_MAX_PROFILE_BINS.  out[n_bins]: host
 * array owned by the caller.  Synchronises.
 * Errors: EINVAL (bad replica, axis or n_bins, NULL out), ECUDA, and any
 * latched device error. */
rmpcd_status rmpcd_profile(rmpcd_system *sys, int32_t replica, int32_t axis, int32_t n_bins, rmpcd_profile_bin *out);

/* Wait for all queued work and return latched device errors. */
rmpcd_status rmpcd_sync(rmpcd_system *sys);

/* Per-phase GPU timers (the paper's per-phase timers, §1.2 `timers`).  When
 * enabled, rmpcd_step records a CUDA event pair on the system's stream
 * around each kernel it launches; rmpcd_read_timers synchronises and returns,
 * per phase, the launches and their summed duration since the last reset.
 * Phases: 0 = first binning of a fused run, 1 = near-colloid MD,
 * 2 = cell pass (sort + collide + react + next flight/bin), 3 = unused. */
typedef struct {
    int64_t launches[4];
    double ms[4];
} rmpcd_timers;

rmpcd_status rmpcd_enable_timers(rmpcd_system *sys, int32_t on);
rmpcd_status rmpcd_read_timers(rmpcd_system *sys, rmpcd_timers *out, int32_t reset);

/* Launch tuning of the near-colloid MD kernel; the results are bit-identical
 * for every choice because the colloid forces are exact fixed-point sums.
 * md_cluster: CTAs per replica (one thread-block cluster): 1, 2, 4, 8, or 16
 *   for the few-colloid kernel where the device schedules 16-CTA clusters;
 *   0 (the default) times each candidate size three times on the first
 *   intervals of rmpcd_step (one synchronisation) and keeps the fastest.
 * md_kernel: 1 = general kernel; 2 = few-colloid kernel (every replica with at
 *   most 2 colloids, at most 1 bond and no colloid-colloid potential: every
 *   warp integrates the colloids itself, one CTA barrier per sub-step);
 *   3 = wide kernel (mixed path: one cooperative launch over all SMs per
 *   replica with colloids, one grid barrier per sub-step; md_cluster 0 or 1);
 *   0 (default) = 2 when allowed, else 3 for the mixed path with at most 4
 *   replicas with colloids, else 1.
 * rmpcd_get_tuning reports the cluster size in use (0 while tuning) and the
 * kernel.  Errors: EINVAL. */
rmpcd_status rmpcd_set_tuning(rmpcd_system *sys, int32_t md_cluster, int32_t md_kernel);
rmpcd_status rmpcd_get_tuning(const rmpcd_system *sys, int32_t *md_cluster, int32_t *md_kernel);

/* CUDA graphs for rmpcd_step (on by default): once the MD launch geometry is
 * settled (cluster size fixed or tuned) and timers are off, each fused
 * interval replays a captured graph of its launches (one per buffer parity;
 * the collision index is read and advanced on the device).  The legacy
 * default stream cannot be captured: a system created on it launches
 * directly.  Results are identical either way.  Errors: EINVAL. */
rmpcd_status rmpcd_set_graphs(rmpcd_system *sys, int32_t on);

/* Test hook of the bounded waits (the paper has no counterpart).  A sorting
 * pass of the flat layout (the granular calls, and the flattening of a fused
 * run's state that rmpcd_get_state, rmpcd_observables and rmpcd_profile do)
 * finds each tile's first output slot by waiting for its predecessors'
 * published prefixes; that wait gives up after max_polls polls (0 = the
 * default, 4,194,304: well over a second), latches RMPCD_ETIMEOUT (reported by
 * the next call that checks errors, e.g. rmpcd_sync) and leaves the tile's
 * writes out (every write is bounds-checked against the pushed-out base), so
 * the kernel returns and the CUDA context stays usable; the system's state is
 * then invalid.  stall != 0 makes every predecessor read as not ready, a flag
 * that nothing sets, so each wait with a predecessor runs out: a test of the
 * timeout path that involves no fault.  Applies to launches after the call
 * (captured graphs are dropped).  Errors: EINVAL (max_polls < 0). */
rmpcd_status rmpcd_set_wait_test(rmpcd_system *sys, int32_t max_polls, int32_t stall);

/* The bucket width in use (the automatic one when created with 0). */
rmpcd_status rmpcd_get_bucket_cap(const rmpcd_system *sys, int32_t *cap);

/* Count of this library's kernel launches since creation (for accounting). */
rmpcd_status rmpcd_launch_count(const rmpcd_system *sys, int64_t *count);

/* One-line description of the last failure of this system (or of the last
 * failed rmpcd_create when sys is NULL).  Never NULL. */
const char *rmpcd_last_error(const rmpcd_system *sys);

/* --- observables without device allocation --------------------------------
 * The paper has no counterpart of this entry point.  It computes what
 * rmpcd_observables reports (the temperature, momentum, kinetic energy and
 * counts) from caller-owned device arrays, and allocates no device memory: it reduces
 * through one static device array of fixed size per device.  It serves
 * callers that must not allocate where they measure: a monitor between the
 * steps of a run whose device memory is wholly reserved by another pool (an
 * allocation could fail), or a caller with work in flight on other streams
 * (cudaFree synchronises the whole device).
 *
 * Inputs (device pointers, n entries each): cell[n] int32 cell keys, e.g. the
 * `cell` output of rmpcd_get_state; entries outside [0, n_cells) are skipped
 * entirely.  v[n][3] FP64 velocities, row-major.  flags[n] (may be NULL = all
 * A): bit 0 = species B.  n_cells: number of cell keys, 1..RMPCD_NOALLOC_MAX_CELLS
 * (for rmpcd_get_state keys: L[0] L[1] L[2], or L[0] L[1] (L[2] + 1) with walls).
 * Output (device pointer, 8 doubles): out = {temperature, momentum x, y, z,
 * kinetic energy, N_c (cells with N >= 2), N_B, particles counted}.
 *
 * The work is queued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and is asynchronous; out is valid once that stream reaches it.
 * The scratch is zeroed by the call itself, so nothing needs to be cleared
 * between calls; `out` need not start at zero.  The first call on a device
 * resolves that device's scratch address and loads the kernels (setup); make
 * it before any stream capture begins.  Calls on one stream are ordered and
 * safe; calls whose work overlaps on one device (other streams or host
 * threads) share the scratch and race.  Sums use FP64 atomics: results agree
 * with rmpcd_observables to rounding, not bit for bit.
 * Errors (returned at once; rmpcd_last_error(NULL) describes them): EINVAL
 * (n < 0, n_cells beyond the limit, NULL or misaligned pointers), ECUDA (setup
 * or launch failed). */
#define RMPCD_NOALLOC_MAX_CELLS 65536
rmpcd_status rmpcd_observables_noalloc(const int32_t *cell, const double *v, const uint8_t *flags,
                                       int64_t n, int32_t n_cells, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RMPCD_H */
