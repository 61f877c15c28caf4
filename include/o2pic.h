/*
 * o2pic.h -- C ABI of libo2pic.so, a GB300 (sm_103a) implementation of the
 * per-time-step hot path of the particle-in-cell Monte-Carlo model of a
 * capacitively coupled RF discharge in O2 of Bronold, Matyash, Tskhakaya,
 * Schneider and Fehske, "Radio-frequency discharges in Oxygen. Part 1:
 * Modeling" (cited below as "the paper").
 *
 * What one pic_step() advances (paper Sec. II, "Method of simulation", and
 * Sec. III, "Scattering and reaction channels"):
 *   1. linear (cloud-in-cell) charge assignment of e, O- and O2+ (Sec. II (i));
 *   2. the 1D Poisson equation with the driven electrode x = 0 at
 *      U(t) = U_rf sin(2 pi f_rf t) and the grounded electrode x = L (Sec. II);
 *   3. linear force interpolation and the Newton (leapfrog) push (Sec. II (i));
 *   4. absorption at both electrodes, no secondary emission (Sec. II);
 *   5. collisions with the O2 reservoir n = p/(kT) for reactions (4)-(12) and
 *      (15)-(18) of Table I by the null-collision method, with the kinematic
 *      rules of Sec. III (Eq. 5, charge exchange, attachment, detachment,
 *      ionisation) and O2(a) at density C n_O2 for (17) (Sec. III C);
 *   6. births of new superparticles and removal of dead ones;
 *   7. every sort_interval steps a stable counting sort by cell that drops
 *      dead particles (Sec. II: particles are sorted into cells after the free
 *      flight);
 *   8. every n1 steps the per-cell particle-target reactions (13), (14), (19)
 *      with probability min(P, 1), P = n sigma u tau, tau = n1 dt (Eq. 1);
 *   9. diagnostics: cycle-averaged densities and potential, the electron
 *      energy distribution at L/2, the O- distribution f_-(E, x) (Sec. IV) and
 *      the O2+ energy distribution at each electrode.
 *
 * Units are SI unless a field name says otherwise.  Species indices:
 * 0 = electron, 1 = O-, 2 = O2+.  Several independent discharges can be
 * advanced together ("batched"): every entry point that takes a discharge
 * index refers to the order of the configurations given to pic_init().
 *
 * Memory: the caller allocates ONE device workspace of pic_workspace_size()
 * bytes (256-byte aligned) and keeps it alive until pic_destroy().  The
 * library never allocates device memory after pic_init(); host-side staging
 * for state and diagnostics copies uses ordinary host memory.  All work is
 * issued on the CUDA stream given to pic_init().
 *
 * Errors: every call returns a pic_status; nothing is thrown across the ABI.
 * After an error the handle stays valid and may be destroyed; pic_last_error()
 * returns a text.
 */
#ifndef O2PIC_H
#define O2PIC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,     /* invalid argument or configuration */
    PIC_ENOMEM = 2,     /* workspace too small */
    PIC_ECAPACITY = 3,  /* particle capacity or a birth buffer overflowed */
    PIC_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
    PIC_ECUDA = 5,      /* a CUDA runtime call failed */
    PIC_ENUMERIC = 6    /* collision-frequency bound or P <= 1 violated too often */
} pic_status;

typedef enum {
    PIC_FP64 = 0,       /* every particle quantity and all arithmetic in FP64 */
    PIC_FP32_MIXED = 1  /* particles and push/collisions in FP32; charge
                           accumulation (exact fixed point), Poisson, field
                           and diagnostics in FP64 */
} pic_precision;

/*
 * One cross-section table (one channel of Table I).  Nodes E_eV[0..n-1] are
 * strictly increasing; sigma is linear in E between nodes, equal to the first
 * node value below E_eV[0], equal to the last value above E_eV[n-1] (paper
 * Sec. III: the largest tabulated value is extended to higher energies), and
 * zero below threshold_eV.  threshold_eV is also the energy lost in the
 * inelastic channels (7)-(12), (15), (18), (19) (Eq. 5).  The energy argument
 * is the centre-of-mass energy (1/2) mu u^2 of the colliding pair.
 *
 * reaction: 4..19 in the numbering of Table I.  The projectile is the
 * electron for 4, 7-13, 15, 18, 19; O- for 5, 14, 16, 17; O2+ for 6.  The
 * target is O2 gas except 13, 14 (O2+) and 19 (O-).  The gas channels of one
 * projectile are tried in the order given here (null-collision walk) and must
 * share one node grid, which must be geometric (E_k = E_0 r^k).
 * sub: vibrational level for reaction 7 (informational), else 0.
 * The tables are copied by pic_init(); the caller keeps ownership.
 */
typedef struct {
    int reaction;
    int sub;
    int n;
    const double *E_eV;
    const double *sigma_m2;
    double threshold_eV;
} pic_xs_table;

/*
 * One discharge (paper Sec. II).  The driven electrode is x = 0.
 *   weight_m2      real particles per m^2 of electrode per superparticle (the
 *                  paper's lateral area A only enters through this number)
 *   C_delta        O2(a1Delta_g)/O2 density ratio for reaction (17) (Sec. III C)
 *   T0_eV          temperatures of the initial Maxwellian load per species
 *   ecap_eV        centre-of-mass energy up to which the collision-frequency
 *                  bound nu_max is taken: [0, ecap] is cut at every node and
 *                  threshold of the species' gas channels, and nu_max is the
 *                  largest sum_j n_j max(sigma_j(a), sigma_j(b)) sqrt(2b/mu)
 *                  over the pieces [a, b], times numax_safety (so no energy
 *                  up to the cap has a larger frequency)
 *   n_init         superparticles loaded uniformly in (0, L) per species
 *   capacity       slots per species (>= n_init; births beyond it fail with
 *                  PIC_ECAPACITY)
 *   n1             interval of the particle-target reactions (tau = n1 dt);
 *                  0 disables them
 *   sort_interval  cell-sort interval in steps (a sort also runs on every
 *                  particle-target step); 0 = only on those steps
 *   diag_every     diagnostics sampling interval in steps; 0 = none
 *   *_bins, *_emax histogram sizes and ranges [eV]; f_- uses fm_xbins equal
 *                  regions of (0, L) and fm_bins signed-energy bins over
 *                  (-fm_emax, fm_emax)
 *   cx_isotropic   reaction (6): 0 = the ion takes the gas molecule's velocity
 *                  (resonant exchange), 1 = isotropic elastic scattering
 *   numax_bins     electrons only, 0..64: the collision-frequency bound is
 *                  taken per bin of the electron's lab energy K after the push
 *                  (K = m 2^e with m in [1, 2): bin 4 (e + 6) + floor(4 (m - 1)),
 *                  clamped to [0, numax_bins - 1]); bin b < numax_bins - 1 uses
 *                  the bound up to the centre-of-mass energy of relative speed
 *                  (top electron speed of the bin + 10 sqrt(kT/M_O2), above
 *                  the fastest gas molecule the Box-Muller draws can give),
 *                  the last bin the species' bound; 0 = one bound for all
 *                  energies
 *   precision      pic_precision; all discharges of one handle share it
 *   n2             interval of the intra-species Coulomb collisions (1)-(3)
 *                  (Sec. III A): every n2 steps, after the cell sort of that
 *                  step and before a particle-target pass due in the same
 *                  step, the particles of each species in each cell are
 *                  paired by a random affine permutation (odd counts end in
 *                  a triangle with half the time) and scattered by the
 *                  binary model with <tan^2(chi/2)> = q^4 n lnGamma tau /
 *                  (8 pi eps0^2 mu^2 u^3) (Eq. 2), tau = n2 dt, mu = m/2, n
 *                  the species' density in the cell; 0 disables them; all
 *                  discharges of one handle share it.  A cell may hold at most
 *                  2^29 particles of a species.
 *   coulomb_log    ln Gamma of Eq. 2 (> 0 when n2 > 0)
 *   gas_scheme     gas-target channels: 0 = null-collision test every step
 *                  (one candidate draw against nu_max, then the channel walk);
 *                  1 = the paper's sequential scheme (Sec. II): no test
 *                  between particle-target steps; every n1 steps, after the
 *                  sort, the channels of Table I in order, each with Eq. 1's
 *                  P = n sigma u n1 dt (clamped at 1 and counted as a P > 1
 *                  clamp): gas channels below (13), (13), (14), gas channels
 *                  above (14) (a product of (15), (16), (17) meets the later
 *                  channels of the list), a new sort, (19).  Needs n1 > 0;
 *                  all discharges of one handle share it.
 *   ion_subcycle   k > 1: O- and O2+ are pushed, and tested for gas
 *                  collisions, only on steps n = 0 mod k, over k dt (null-
 *                  collision probability 1 - exp(-nu_max k dt)); in between
 *                  they rest and their charge stays in the grid.  Not in the
 *                  paper: a throughput variant.  0 or 1: every step.
 *                  diag_every must then be a multiple of k.
 *   coulomb_inter  1: inter-species Coulomb collisions as well, after the
 *                  intra-species ones of a Coulomb step (n2 > 0): pairs
 *                  e-O-, e-O2+, O- - O2+ in turn; per cell every particle of
 *                  the more numerous species collides once, those of the
 *                  other in turn; Eq. 2 with q_a^2 q_b^2, the pair's reduced
 *                  mass and the density of the less numerous species.
 */
typedef struct {
    double L_m, p_Pa, T_gas_K, U_rf_V, f_rf_Hz, rf_phase, dt_s;
    double weight_m2, C_delta;
    double T0_eV[3];
    double ecap_eV[3];
    double numax_safety;
    double eedf_emax_eV, iedf_emax_eV, fm_emax_eV;
    long long n_init[3];
    long long capacity[3];
    unsigned long long seed;
    int n_cells, n1, sort_interval, diag_every;
    int eedf_bins, iedf_bins, fm_bins, fm_xbins;
    int cx_isotropic;
    int numax_bins;
    int n2;
    int gas_scheme;
    int ion_subcycle;
    int coulomb_inter;
    int precision;
    double coulomb_log;
} pic_config;

typedef struct pic_handle pic_handle;

/*
 * Bytes of device workspace needed for the given discharges and tables.
 * Returns 0 if the configuration is invalid (pic_last_error(NULL) says why).
 */
size_t pic_workspace_size(const pic_config *cfgs, int n_discharges,
                          const pic_xs_table *xs, int n_xs);

/*
 * Validate, copy the tables to device look-up tables, compute nu_max per
 * species and discharge, carve the caller's workspace, load the particles
 * (uniform positions, Maxwellian velocities, counter-based Philox4x32-10 from
 * `seed`, so the load is reproducible) and deposit the initial charge.
 *   d_workspace  device pointer, >= pic_workspace_size() bytes, 256-aligned
 *   cuda_stream  a cudaStream_t (NULL = legacy default stream)
 *   out          receives the handle
 * Synchronises the stream before returning.
 */
pic_status pic_init(const pic_config *cfgs, int n_discharges,
                    const pic_xs_table *xs, int n_xs, void *d_workspace,
                    size_t ws_bytes, void *cuda_stream, pic_handle **out);

/*
 * Advance every discharge by n_steps time steps (each of length dt_s).
 * Work is queued on the handle's stream.  When one RF cycle, 1 / (f_rf dt),
 * is a whole number of time steps and of periods of the step schedule (the
 * least common multiple of 2, n1, n2, sort_interval and diag_every; taken
 * from the first discharge) and at most 8192 steps, the first full cycle a
 * call covers is captured as one CUDA graph and every full cycle from a
 * period-aligned step is one cudaGraphLaunch; what is left is replayed as
 * graphs of one period, then step by step.  (Timing mode launches step by
 * step.)  The call then synchronises and checks the device status word,
 * returning PIC_ECAPACITY, PIC_ETIMEOUT, PIC_ENUMERIC or PIC_EINVAL if the
 * device reported one.
 */
pic_status pic_step(pic_handle *h, long long n_steps);

/*
 * Diagnostics of one discharge, copied into caller-owned host arrays (any
 * pointer may be NULL to skip it).  Sizes: N = n_cells.  The densities and
 * the potential come back as sums over the n_samples samples of the window
 * (every diag_every steps since the last reset): dens_sum / n_samples and
 * phi_sum / n_samples are the cycle-averaged profiles of the paper's Sec. IV
 * when the window spans whole RF cycles.  Sums rather than averages let a
 * caller merge windows exactly (the FP32 path accumulates exact integers).
 *   dens_sum   [3][N+1]  sum over samples of the number density per species
 *   phi_sum    [N+1]     sum over samples of the potential
 *   eedf       [eedf_bins] electrons in the cell [L/2, L/2 + dx), E = m v^2/2
 *   iedf       [2][iedf_bins] O2+ absorbed at x = 0 and x = L, E = M v^2/2
 *   fm         [fm_xbins][fm_bins] O-, E = sign(vx) M vx^2 / 2
 *   counters   [40]: 0-5 absorbed (species*2 + wall), 6-25 events per
 *              reaction 0..19 (index 6 + reaction), 26 gas nu_max
 *              violations, 27 Eq. 1 P > 1 clamps (particle-target pass and
 *              sequential gas scheme), 28-30 slots per species
 *              (including dead slots not yet compacted), 31 steps taken,
 *              32 particle-steps (live particles pushed, summed over steps),
 *              33 null-collision candidates, 34 slots visited by the push,
 *              35 particles through the Coulomb pass (summed over passes),
 *              36 live slots through the sequential gas scheme (summed over
 *              its two parts and passes), 37 Eq. 1 probabilities evaluated
 *              (particle-target candidates and sequential-scheme tests below
 *              their bound), 38 time steps of the captured RF-cycle graph
 *              (0 when the cycle is not captured), 39 CUDA graph launches
 *              since pic_init (cycle and period graphs)
 *   n_samples  number of diagnostic samples accumulated
 * reset != 0 clears the sums and histograms after copying.
 */
pic_status pic_diagnostics(pic_handle *h, int discharge, double *dens_sum,
                           double *phi_sum, long long *eedf, long long *iedf,
                           long long *fm, long long *counters,
                           long long *n_samples, int reset);

/*
 * Particle state of one discharge and species, as host arrays of length
 * *n (slots in the device order, including not-yet-compacted dead slots):
 * x [m], vx, vy, vz [m/s] and alive (1/0).  Pass NULL arrays with a valid n
 * to query the count only; capacity_n is the length of the caller's arrays.
 */
pic_status pic_get_state(pic_handle *h, int discharge, int species,
                         double *x, double *vx, double *vy, double *vz,
                         int *alive, long long capacity_n, long long *n);

/*
 * Replace the particle state of one discharge and species (n slots, same
 * layout as pic_get_state; alive may be NULL = all alive) and recompute the
 * charge density of that discharge.  x must lie in [0, L) for live slots.
 */
pic_status pic_set_state(pic_handle *h, int discharge, int species, long long n,
                         const double *x, const double *vx, const double *vy,
                         const double *vz, const int *alive);

/* Set the step counter (which drives U(t) and the random counters). */
pic_status pic_set_step(pic_handle *h, long long step);

/*
 * Numerical budget of pic_step (paper Sec. II with reading R10/R11: the
 * null-collision bound nu_max is taken up to ecap_eV, and Eq. 1's linear
 * P = n sigma u tau is clamped at 1).  pic_step returns PIC_ENUMERIC when, in
 * a discharge, more than 10 and more than max_fraction of the null-collision
 * candidates met a total frequency above their bound (counters[26] against
 * counters[33]), or more than 10 and more than max_fraction of the Eq. 1
 * probabilities evaluated (particle-target candidates and sequential-scheme
 * tests, counters[37]) exceeded 1 (counters[27]).  Counts are cumulative
 * since pic_init.  Default 1e-6; a run that wants coarse n1 dt on purpose
 * raises it.  PIC_EINVAL for a fraction outside [0, 1].
 */
pic_status pic_set_numeric_budget(pic_handle *h, double max_fraction);

/* Potential, field and charge density of one discharge at the current state
 * (each [N+1], SI; NULL skips). */
pic_status pic_fields(pic_handle *h, int discharge, double *rho, double *phi,
                      double *E);

/* nu_max [1/s] of one discharge and species (after pic_init). */
double pic_numax(const pic_handle *h, int discharge, int species);

/*
 * Per-kernel timing: when on, pic_step launches kernels one by one with CUDA
 * events around each particle push and accumulates their device time;
 * pic_timing() returns (ms total of the push kernel, push launches, all
 * kernel launches, algorithmic bytes moved by the push kernel) since the last
 * reset.  Kernel launches are always counted.
 */
pic_status pic_set_timing(pic_handle *h, int on);
pic_status pic_timing(pic_handle *h, double *push_ms, long long *push_launches,
                      long long *launches, double *push_bytes, int reset);

/*
 * The same for one kernel kind (timing mode on): PIC_KERNEL_PUSH the push
 * launches of steps without diagnostics, PIC_KERNEL_PUSH_DIAG those of
 * diagnostics steps (pic_timing gives both together; their algorithmic
 * bytes are shared out by launches, reset clears both);
 * PIC_KERNEL_COULOMB the Coulomb pass of collisions
 * (1)-(3): device ms, launches and algorithmic bytes (vx, vy, vz read and
 * written for every particle of a cell holding at least two of its species)
 * since its last reset; PIC_KERNEL_SEQUENTIAL_GAS the two parts of the
 * sequential gas scheme (cell, offset, vx, vy, vz read and vx, vy, vz written
 * per live slot and part).  Unknown kinds return PIC_EINVAL.
 */
typedef enum {
    PIC_KERNEL_PUSH = 0,            /* push launches of steps without diagnostics */
    PIC_KERNEL_COULOMB = 1,
    PIC_KERNEL_SEQUENTIAL_GAS = 2,
    PIC_KERNEL_PUSH_DIAG = 3        /* push launches that also sample the diagnostics */
} pic_kernel;
pic_status pic_kernel_timing(pic_handle *h, int kernel, double *ms, long long *launches,
                             double *bytes, int reset);

/*
 * Launch shape of a kernel kind, for autotuning.  Only PIC_KERNEL_PUSH has
 * one: the particle push (steps 3 and 4 above, the charge assignment of
 * step 1 and the null-collision test of step 5) is a persistent grid of
 * blocks_per_sm blocks on every SM (of the current shape's threads, see
 * pic_launch_shapes below), each block taking tickets of tiles until none
 * are left.  pic_init sets the largest count that fits on
 * an SM (registers and shared memory); pic_set_launch may lower it to any
 * count in 1 .. that maximum.  Results do not depend on it: the charge sums
 * are exact integers and births are appended in parent order (FP32 mixed
 * state is bit for bit the same; the FP64 path adds each block's charge to
 * double accumulators, whose rounding can differ in the last bits).  The
 * call waits for the handle's stream and drops the captured graph of one
 * period, which the next pic_step records again.
 *   pic_get_launch  current and largest blocks per SM (either pointer may
 *                   be NULL)
 *   pic_set_launch  PIC_EINVAL for another kind or a count out of range, and
 *                   the shape is left unchanged
 */
pic_status pic_get_launch(pic_handle *h, int kernel, int *blocks_per_sm, int *max_blocks_per_sm);
pic_status pic_set_launch(pic_handle *h, int kernel, int blocks_per_sm);

/*
 * Launch shapes of the push (the same kernel work as above, for autotuning).
 * The push is compiled for a few shapes: threads per block and slots per
 * thread (each warp takes slots_per_thread / 4 consecutive sub-tiles of 128
 * slots at a time, each lane four consecutive slots of each: one 16-byte
 * vector per array and one Philox block).  The FP32 mixed path has several,
 * the FP64 path one.  Results do not depend on the shape (as for the blocks
 * per SM above).
 *   pic_launch_shapes     writes up to `capacity` shapes (threads per block,
 *                         slots per thread, largest blocks per SM; any
 *                         pointer may be NULL) and returns how many there
 *                         are; -1 for a NULL handle or another kind
 *   pic_get_launch_shape  the current shape index and blocks per SM
 *   pic_set_launch_shape  select a shape index and blocks per SM (1 .. that
 *                         shape's largest); PIC_EINVAL otherwise, leaving the
 *                         shape unchanged.  Waits for the stream and drops
 *                         the captured graph like pic_set_launch.
 */
int pic_launch_shapes(pic_handle *h, int kernel, int *threads, int *slots_per_thread,
                      int *max_blocks_per_sm, int capacity);
pic_status pic_get_launch_shape(pic_handle *h, int kernel, int *shape, int *blocks_per_sm);
pic_status pic_set_launch_shape(pic_handle *h, int kernel, int shape, int blocks_per_sm);

/*
 * pic_field_solve_static -- charge deposit, Poisson solve and field of ONE
 * discharge from particle arrays that the caller owns, without allocating
 * any memory.  The paper has no counterpart: this entry point serves callers
 * that cannot allocate device memory (code inside a host framework that
 * owns every allocation, code that must not call cudaMalloc in the middle of
 * its own GPU work because that call can synchronise the device, code with
 * a memory budget fixed up front) and so cannot use pic_init's workspace.
 * It computes what pic_fields() computes for a handle, from the same
 * particle representation.
 *   cfg        the discharge (L_m, n_cells, U_rf_V, f_rf_Hz, rf_phase, dt_s,
 *              weight_m2 and precision are used)
 *   step       time-step number n; phi(x = 0) = U_rf sin(2 pi f n dt + phase)
 *   d_cell[s]  device array of n[s] cell indices per species (< 0 = dead)
 *   d_off[s]   device array of n[s] offsets in [0, 1): float for
 *              PIC_FP32_MIXED, double for PIC_FP64; a value outside
 *              [0, 1] (or NaN) is clamped into it, so a bad offset moves
 *              that particle's charge within its cell but never corrupts
 *              the sums
 *   n[s]       host array of the three slot counts
 *   d_rho, d_phi, d_E  device outputs, n_cells + 1 doubles each (SI)
 *   cuda_stream  the work is queued on this stream (NULL = legacy default);
 *              the outputs are valid once the stream has reached this point
 * Limit: n_cells <= 4096 (larger grids fail with PIC_EINVAL).  Scratch: one
 * fixed array of 3 x 4097 x 8 bytes in device memory, which every GPU that
 * loads this library reserves until the process exits.  The first call on a
 * device looks up that array's device address with the device current, and
 * under CUDA's default lazy module loading that first call also loads this
 * library's kernels and the array onto the device (a driver-side
 * allocation): make one warm-up call per device before any region that must
 * not allocate and before any stream capture, or run with
 * CUDA_MODULE_LOADING=EAGER.  All calls on a
 * device share the array and clear it first: calls that can run at the same
 * time on the GPU (unordered streams) race and corrupt each other's output.
 */
pic_status pic_field_solve_static(const pic_config *cfg, long long step,
                                  const int *const *d_cell,
                                  const void *const *d_off, const long long *n,
                                  double *d_rho, double *d_phi, double *d_E,
                                  void *cuda_stream);

void pic_destroy(pic_handle *h);

/* Text of the last error on this handle (or of the calling thread's last
 * handle-less call when h == NULL). */
const char *pic_last_error(const pic_handle *h);

#ifdef __cplusplus
}
#endif
#endif /* O2PIC_H */
