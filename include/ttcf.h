/*
 * ttcf.h -- C ABI of the GB300 TTCF daughter-ensemble engine.
 *
 * The engine computes the transient-time correlation function (TTCF)
 * response of a sheared bulk WCA fluid (arXiv:2312.02990, Example 1):
 *
 *   <B(t)> = <B(0)> + int_0^t <Omega(0) B(s)> ds                      (Eq. 1)
 *   <Omega(0) B(s)> = (1/N) sum_i Omega(0)_i B(s)_i                   (Eq. 2)
 *
 * over daughter trajectories that start from the four phase-space mappings
 * (Eq. 3) of equilibrium mother states, follow the thermostatted SLLOD
 * equations of motion (Eq. 5) with the WCA pair potential (Eq. 6) under
 * Lees-Edwards sliding-brick boundaries, and measure B = P_xy with the
 * dissipation function Omega = -gamma V P_xy / (k_B T) (Eq. 7; the sign
 * follows from Omega = beta dH^ad/dt of the Mathematical Framework with the
 * standard pressure tensor).  The viscosity is eta = -<P_xy>/gamma (Eq. 8).
 *
 * Conventions shared by every call:
 *  - Reduced units: sigma = epsilon = m = k_B = 1.
 *  - A phase point is a C-contiguous float64 array [6][N]: rows x, y, z,
 *    px, py, pz.  Positions lie in the centred box [-L/2, L/2).  Momenta
 *    are peculiar (thermal) momenta; the streaming profile gamma*y of the
 *    daughter is carried by the equations of motion, never added to p.
 *  - The caller owns every array passed in or out.  Inputs are copied
 *    during the call.  The library owns all device memory it allocates,
 *    through the allocator given in ttcf_config (torch's caching allocator
 *    when created from Python) or cudaMalloc/cudaFree.
 *  - Every call returns a ttcf_status; no exception crosses the ABI and the
 *    process never aborts.  After an error, ttcf_last_error() holds a
 *    one-line description.
 *  - Work is queued on ttcf_config.stream; calls that return results to
 *    host memory synchronise that stream before returning.
 */
#ifndef TTCF_H
#define TTCF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttcf_ctx ttcf_ctx;

typedef enum {
    TTCF_OK = 0,
    TTCF_E_INVALID = 1,  /* bad argument or configuration                  */
    TTCF_E_CUDA = 2,     /* a CUDA runtime call failed                       */
    TTCF_E_OOM = 3,      /* device or host allocation failed                 */
    TTCF_E_NUMERIC = 4,  /* >= 1 daughter stopped: NaN/Inf, lost atom,
                            neighbour-list overflow; its group is excluded    */
    TTCF_E_TIMEOUT = 5,  /* ttcf_run exceeded timeout_s and was aborted      */
    TTCF_E_STATE = 6     /* call out of order (e.g. response before run)     */
} ttcf_status;

/* Systems.
 *  TTCF_BULK_WCA     Example 1: WCA fluid under SLLOD shear with
 *                    Lees-Edwards boundaries and a Nose-Hoover thermostat.
 *  TTCF_CONFINED_LJ  Example 2: Lennard-Jones fluid between two walls of
 *                    tethered atoms whose lattices slide at +-v in x
 *                    (Eq. 9, 10); MIXED precision only.
 *  TTCF_BULK_WCA_ELONG  the WCA fluid of Example 1 under planar
 *                    elongational flow, the other homogeneous field the
 *                    paper's introduction lists beside shear: the Eq. 5
 *                    equations with grad u = diag(eps, 0, -eps)
 *                    (stretching along x, compression along z) in a box
 *                    that deforms with the flow, Lx(t) = Lx e^{eps t},
 *                    Lz(t) = Lz e^{-eps t} (no periodic remapping: every
 *                    compressed edge must stay above 2 r_c up to the
 *                    daughter's end, which ttcf_spawn_daughters checks).
 *                    The per-group rates passed as shear_rates are the
 *                    elongation rates eps; the response is B = P_xx - P_zz,
 *                    Omega = -eps V B(0) / (k_B T), and ttcf_viscosity
 *                    returns eta_1 = -<P_xx - P_zz> / (4 eps), the shear
 *                    viscosity in the Newtonian limit.  Mapping codes as
 *                    for shear; the x <-> z exchange (bit 4) negates
 *                    Omega and time reversal keeps it, so the set
 *                    {0, 1, 16, 17} (mapping_mask 0x30003) cancels
 *                    <Omega(0)> per group.  One CTA per daughter with the
 *                    whole daughter in shared memory (N up to about 2200
 *                    in MIXED, 1900 in FP64) and its Verlet lists (skin
 *                    0.35, less where the compressed edge needs it) in a
 *                    global scratch; use_graph, skin, kernel_variant,
 *                    block_threads and cell_frac do not apply; the
 *                    control variate is not available.  The
 *                    equilibrium tools (ttcf_sample_mothers,
 *                    ttcf_mother_acf, ttcf_forces) work as in
 *                    TTCF_BULK_WCA.                                     */
enum { TTCF_BULK_WCA = 0, TTCF_CONFINED_LJ = 1, TTCF_BULK_WCA_ELONG = 2 };

/* Responses per sample of a confined daughter (TTCF_CONFINED_LJ):
 *  0              x force of the fluid on the bottom wall per wall area
 *  1              the same on the top wall
 *  2 + k          sum of fluid p_x in slab k (k < TTCF_CONF_NSLAB) of
 *                 equal slabs spanning y in [-Ly/2, Ly/2)
 *  2 + NSLAB + k  number of fluid atoms in slab k
 *  2 + 2 NSLAB    sum of p_x over the innermost layer of the bottom wall
 *                 (its atoms whose tether site lies within 0.1 sigma in y
 *                 of the wall's site plane nearest the channel)
 *  3 + 2 NSLAB    the same for the top wall
 * (slab velocity profile: response 2+k divided by response 2+NSLAB+k).  */
enum { TTCF_CONF_NSLAB = 40, TTCF_CONF_NOBS = 2 + 2 * 40 + 2 };

/* Arithmetic of the daughter integrator.
 *  TTCF_FP64:  every per-atom quantity in IEEE double (slow on GB300).
 *  TTCF_MIXED: FP32 pair forces and virial; positions and momenta kept as
 *              unevaluated float pairs (about 48 significand bits) updated
 *              on the FP32 pipe; alpha, the Lees-Edwards offset, Omega(0),
 *              B(0) and every accumulation in IEEE double.                  */
enum { TTCF_FP64 = 0, TTCF_MIXED = 1 };

/* Per-daughter flags reported by ttcf_group_status (bitwise OR per group). */
enum {
    TTCF_D_OK = 0,
    TTCF_D_NONFINITE = 1,      /* NaN or Inf in a reduced sum                 */
    TTCF_D_NBR_OVERFLOW = 2,   /* an atom had more Verlet neighbours than fit */
    TTCF_D_FAST_ATOM = 4,      /* an atom moved more than skin/2 in one step  */
    TTCF_D_ABORTED = 8,        /* stopped by the host (timeout)               */
    TTCF_D_ESCAPED = 16        /* confined system: an atom left the slab
                                  extent by more than Ly/2 (|y| > Ly) or
                                  became non-finite                            */
};

typedef void *(*ttcf_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*ttcf_free_fn)(void *ptr, void *stream, void *user);

/* Plain-old-data configuration; copied by ttcf_create. */
typedef struct {
    int system;             /* TTCF_BULK_WCA, TTCF_CONFINED_LJ or
                               TTCF_BULK_WCA_ELONG                           */
    int precision;          /* TTCF_FP64 or TTCF_MIXED                       */
    double dt;              /* time step h (Example 1: 0.0025)               */
    double T;               /* thermostat k_B T (Example 1: 0.722)           */
    double tau_T;           /* Nose-Hoover time: Q = g T tau_T^2             */
    int dof_mode;           /* 0: g = 3N as printed in Eq. 5; 1: g = 3N - 3  */
    int n_steps;            /* daughter length in steps                      */
    int sample_every;       /* B(s) recorded every sample_every steps;
                               n_steps must be a multiple of it              */
    unsigned mapping_mask;  /* bit m selects mapping code m (0xF = the four
                               mappings of Eq. 3).  Code m, applied as:
                               bit 4 exchange of x and z (positions and
                               momenta; needs Lx = Lz), bit 1/2/3
                               reflection of x/y/z with its momentum, bit 0
                               time reversal p -> -p (the further choices
                               listed after Eq. 3); codes 0..3 are Eq. 3.
                               Bulk only beyond 0..3; a set closed under the
                               x- or y-reflection keeps <Omega(0)> = 0 per
                               group, other sets call for the Eq. 4 form    */
    int reset_alpha;        /* 0: daughters inherit the mother's alpha,
                               negated by the time-reversing (odd) codes;
                               1: alpha = 0 at switch-on                     */
    int keep_state;         /* 1: keep every daughter's phase point on the
                               device after ttcf_run (ttcf_get_state)        */
    double skin;            /* Verlet skin (sigma); <= 0 selects autotuned   */
    int block_threads;      /* threads per daughter CTA; 0 = autotuned       */
    int kernel_variant;     /* 0 = automatic; k >= 1 selects launch variant
                               k-1 (atoms per thread, block size, register
                               budget): 1 (1,256,64r) 2 (2,512,64r)
                               3 (2,1024,64r) 4 (4,512,64r) 5 (4,512,128r)
                               6 (8,512,128r)                                 */
    int use_graph;          /* 1: ttcf_run captures its persistent launches
                               (one per size class, on forked streams) and
                               the reductions into one CUDA graph            */
    void *stream;           /* cudaStream_t; NULL = legacy default stream    */
    ttcf_alloc_fn dev_alloc;/* NULL: cudaMalloc                              */
    ttcf_free_fn dev_free;  /* NULL: cudaFree                                */
    void *alloc_user;       /* passed to dev_alloc / dev_free                */
    double timeout_s;       /* ttcf_run wall-clock limit; <= 0: none         */
    double cell_frac;       /* bulk list cells of width cell_frac (r_c+skin),
                               in [0.4, 1]; 0 = autotuned, else 2/3          */
} ttcf_config;

/* Fill *cfg with the Example 1 defaults: MIXED, dt 0.0025, T 0.722,
 * tau_T 0.25, g = 3N, 1000 steps, sample_every 1, all four mappings,
 * alpha carried, autotuned skin and block size, CUDA graph on.          */
void ttcf_config_default(ttcf_config *cfg);

/* Create a context.  *out receives an owned handle (ttcf_destroy frees it).
 * Errors: TTCF_E_INVALID (bad field), TTCF_E_CUDA (no device).             */
ttcf_status ttcf_create(const ttcf_config *cfg, ttcf_ctx **out);

/* Append one batch of daughters (Figure 1, Algorithm 2 "apply mapping",
 * "switch on ext. field"): for each of the n_mothers mother states g, one
 * daughter per mapping selected in mapping_mask, daughter index within the
 * batch d = g*M + k (k-th selected mapping, M = popcount(mask)).  Groups
 * stay contiguous so that <Omega(0)> = 0 holds per group (Eq. 3).
 *
 *  n_atoms       N of this batch (bulk WCA, 4 <= N <= 4096)
 *  box           [3] edge lengths Lx, Ly, Lz (each > 2 * (r_c + skin))
 *  mother_soa    [n_mothers][6][N] float64 phase points
 *  mother_alpha  [n_mothers] Nose-Hoover multipliers, or NULL for zeros
 *  shear_rates   [n_mothers] field gamma of each group (same for its M
 *                daughters); gamma = 0 is allowed (Omega = 0)
 *  ptr_is_device 1 if the three arrays are device pointers, else host
 *  batch_id      receives the batch index used by ttcf_response etc.
 *
 * Runs the spawn kernel: copies and maps the states and computes, in
 * IEEE double, B(0) = P_xy(0) and Omega(0) of every daughter.  Must be
 * called before the first ttcf_run.  Errors: TTCF_E_INVALID, TTCF_E_OOM,
 * TTCF_E_CUDA, TTCF_E_STATE (after ttcf_run).                              */
ttcf_status ttcf_spawn_daughters(ttcf_ctx *ctx, int n_atoms, const double box[3],
                                 int n_mothers, const double *mother_soa,
                                 const double *mother_alpha, const double *shear_rates,
                                 int ptr_is_device, int *batch_id);

/* Advance every daughter of every batch by n_steps steps (SLLOD + Nose-
 * Hoover, Eq. 5; pair forces, Eq. 6) in one persistent launch per size
 * class, recording B(s) on device.  May be called in chunks; chunks give
 * bitwise the same result as one call.  n_steps = 0 or more than remain:
 * runs the rest.  Returns after the stream is synchronised.  Confined
 * daughters (Eq. 10) run all n_steps in one call (a smaller n_steps is
 * TTCF_E_INVALID) and keep_state does not apply to them.
 * Errors: TTCF_E_STATE (nothing spawned), TTCF_E_NUMERIC (some daughters
 * failed; see ttcf_group_status), TTCF_E_TIMEOUT, TTCF_E_CUDA.             */
ttcf_status ttcf_run(ttcf_ctx *ctx, int n_steps);

/* Ensemble responses of one batch (Eq. 1, 2; Eq. 4 if corrected != 0),
 * reduced on the device in a fixed order in IEEE double, over the groups
 * whose daughters all finished.  Each output is [S] with S = n_steps /
 * sample_every + 1 samples at t = s * sample_every * dt; any output pointer
 * may be NULL.  Standard errors are taken over mother groups.
 *  t        sample times
 *  dav      direct average <B(t)>, dav_se its standard error
 *  corr     <Omega(0) B(s)>, corr_se
 *  ttcf     <B(0)> + trapezoid integral of corr, ttcf_se
 * capacity is the length of each caller array; *n_samples receives S.
 * Errors: TTCF_E_STATE (run not finished), TTCF_E_INVALID (capacity < S).  */
ttcf_status ttcf_response(ttcf_ctx *ctx, int batch_id, int corrected, double *t,
                          double *dav, double *dav_se, double *corr, double *corr_se,
                          double *ttcf, double *ttcf_se, int capacity, int *n_samples);

/* Shear viscosity of a batch whose groups share one shear rate gamma
 * (Eq. 8 with the standard pressure tensor): eta(t) = -<P_xy(t)>/gamma
 * from the TTCF and the direct averages, with standard errors.  For a
 * TTCF_BULK_WCA_ELONG batch, the planar elongational viscosity
 * eta_1(t) = -<P_xx(t) - P_zz(t)>/(4 eps).  Arrays as in ttcf_response.
 * Errors: as ttcf_response; TTCF_E_INVALID if the rate differs between
 * groups or is 0.                                                          */
ttcf_status ttcf_viscosity(ttcf_ctx *ctx, int batch_id, double *t, double *eta_ttcf,
                           double *eta_ttcf_se, double *eta_dav, double *eta_dav_se,
                           int capacity, int *n_samples);

/* <Omega(0)> of a finished batch, the mean of the dissipation function at
 * switch-on over the daughters of its valid mother groups, as used by the
 * Eq. 4 form of ttcf_response (corrected = 1); exactly 0 with all four
 * mappings of Eq. 3.  *n_valid receives the number of valid groups.  A
 * multi-rank merge folds (n_valid, omega_mean) of each rank into the global
 * <Omega(0)> that the Eq. 4 form of the merged ensemble needs.
 * Errors: TTCF_E_INVALID (bad batch), TTCF_E_STATE (run not finished).    */
ttcf_status ttcf_omega_mean(ttcf_ctx *ctx, int batch_id, double *omega_mean, double *n_valid);

/* Raw per-daughter outputs of a batch: B [D][n_obs][S] and Omega [D]
 * (host arrays, D = n_mothers * M; n_obs = 1 for the bulk system, so B is
 * [D][S] there, TTCF_CONF_NOBS for the confined one).  capacity_B is the
 * element count of B.                                                     */
ttcf_status ttcf_daughter_series(ttcf_ctx *ctx, int batch_id, double *B, double *Omega,
                                 size_t capacity_B);

/* Per-group status flags (TTCF_D_*, OR over the group's daughters) [G].   */
ttcf_status ttcf_group_status(ttcf_ctx *ctx, int batch_id, int *status, int capacity);

/* Phase point [6][N], alpha and Lees-Edwards offset of daughter d of a
 * batch after the last ttcf_run; requires keep_state = 1.  Positions are
 * wrapped into the box; for a TTCF_BULK_WCA_ELONG batch that is the box
 * of the last step run (Lx e^{eps t}, Ly, Lz e^{-eps t}) and the offset
 * is 0.                                                                    */
ttcf_status ttcf_get_state(ttcf_ctx *ctx, int batch_id, int daughter, double *soa,
                           double *alpha, double *delta);

/* Work counters of the last ttcf_run: device time of the persistent
 * launch(es) measured with CUDA events on the context's stream (ms), the
 * device time of the spawn kernels of the batches this run is the first
 * to cover and of the reductions (ms), the number of interacting ordered pairs
 * (r < r_c) summed over all atoms and steps, the number of Verlet-list
 * rebuilds, atom-steps, and kernel launches issued.                        */
typedef struct {
    double ms_run, ms_spawn, ms_reduce;
    double pairs_interacting;   /* ordered pairs (i,j), r_ij < r_c, summed
                                   over daughter steps (bulk: counted on the
                                   force passes that refresh the active
                                   lists, their mean times the steps run)   */
    double rebuilds;            /* neighbour-list builds, summed over daughters */
    double atom_steps;          /* sum over daughters of N * steps run       */
    int launches;               /* kernels launched by the last ttcf_run     */
    int block_threads;          /* block size used (largest class)          */
    double skin;                /* Verlet skin used                          */
} ttcf_stats;
ttcf_status ttcf_get_stats(ttcf_ctx *ctx, ttcf_stats *out);

/* Equilibrium mother states on the GPU (Algorithm 2, mother part): from
 * each of n_init initial phase points [n_init][6][N] (host), run n_eq
 * zero-field Nose-Hoover steps, then store n_states phase points `spacing`
 * steps apart.  out_soa [n_init][n_states][6][N] and out_alpha
 * [n_init][n_states] are host arrays.  Uses the context's precision and
 * kernels with gamma = 0.  Independent of any spawned batch.               */
ttcf_status ttcf_sample_mothers(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_init,
                                const double *init_soa, int n_eq, int n_states, int spacing,
                                double *out_soa, double *out_alpha);

/* Equilibrium correlations along GPU mother trajectories (the mother-side
 * tool for choosing the spacing of mother states, cf. Fig. 7, and the
 * Green-Kubo form of Eq. 8 at zero field): from each of n_init initial
 * phase points [n_init][6][N] (host), n_eq zero-field Nose-Hoover steps,
 * then n_steps steps recording B(s) = P_xy(s) every step.  Averaged over
 * trajectories and time origins, for lags k = 0 .. max_lag steps:
 *   acf_pxy[k]  = <P_xy(t) P_xy(t+k)>   (the correlation of Omega for the
 *                 shear field, Omega being proportional to P_xy),
 *   acf_pxy2[k] = autocovariance of P_xy^2 (that of Omega P_xy),
 *   eta_gk[k]   = (V/T) trapezoid integral of acf_pxy up to lag k.
 * series (may be NULL) receives P_xy [n_init][n_steps].  Host outputs of
 * length max_lag + 1 (any may be NULL).  Errors: TTCF_E_INVALID,
 * TTCF_E_NUMERIC (a trajectory failed), TTCF_E_OOM, TTCF_E_CUDA.          */
ttcf_status ttcf_mother_acf(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_init,
                            const double *init_soa, int n_eq, int n_steps, int max_lag,
                            double *acf_pxy, double *acf_pxy2, double *eta_gk, double *series);

/* Further mother states from one thermalised state (the thermalisation
 * workflow of the paper's computational section: further initial conditions
 * from a single equilibrated state by a small random kick to the
 * velocities; the dynamics is chaotic, so the copies decorrelate quickly).
 * Writes n_copies copies of the phase point state_soa [6][N] (x y z px py
 * pz) to out_soa [n_copies][6][N]: positions unchanged; copy c adds to
 * momentum component k of atom i the kick  kick * sqrt(T) * g  (T of the
 * context, unit masses), g standard normal from Philox-4x32-10 (Salmon et
 * al., SC'11) keyed by seed (low word first) with counter (i, c, b, 0),
 * b = 0, 1, and Box-Muller on the 53-bit uniforms of its word pairs (g0, g1
 * from b = 0, g2 the cosine branch of b = 1).  Every group of atoms (types
 * [N] with values 0, 1, 2, e.g. fluid and the two walls, or NULL for one
 * group) keeps its net momentum: the group mean of the kicks is removed.
 * keep_energy != 0: every group also keeps the kinetic energy of its
 * momenta relative to the group mean (the kicked relative momenta are
 * rescaled).  Inputs and outputs on the host (is_dev = 0) or on the
 * context's device (is_dev = 1, stream of the context); caller-owned.
 * IEEE double.  Errors: TTCF_E_INVALID (NULL, n_atoms or n_copies < 1,
 * kick < 0 or not finite, a type outside 0..2), TTCF_E_OOM, TTCF_E_CUDA. */
ttcf_status ttcf_kick_states(ttcf_ctx *ctx, int n_atoms, const double *state_soa, const int *types,
                             int n_copies, double kick, unsigned long long seed, int keep_energy,
                             double *out_soa, int is_dev);

/* Pair forces of n_states phase points [n_states][6][N] (host; rows 0-2
 * used) at Lees-Edwards offset delta, with the context's precision and the
 * same device code the daughters use: F [n_states][3][N] and virial
 * W [n_states][6] (xx yy zz xy xz yz, sum over pairs of r_a F_b), U
 * [n_states] (potential energy).  Host outputs.                            */
ttcf_status ttcf_forces(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_states,
                        double delta, const double *soa, double *F, double *W, double *U);

/* Autotuner (launch shape, Verlet skin and list-cell width).  Times
 * n_steps of the daughter kernel on n_states phase points [n_states][6][N]
 * (host; all four mappings, shear rate gamma) for every launch variant that
 * holds n_atoms, Verlet skins {0.3, 0.35, 0.4, 0.5, 0.6} and cell widths
 * {1/2, 2/3, 1} (r_c + skin), with CUDA events on the context's stream, and
 * remembers the fastest for batches of n_atoms spawned later on this
 * context (explicit kernel_variant / skin / cell_frac in the config still
 * win).  Returns the choice (1-based variant as in
 * ttcf_config.kernel_variant), the skin, the cell width and its time in
 * ms (any output may be NULL).  Errors: TTCF_E_INVALID if no variant can
 * run the system.                                                          */
ttcf_status ttcf_autotune(ttcf_ctx *ctx, int n_atoms, const double box[3], int n_states,
                          const double *soa, double shear_rate, int n_steps, int *best_variant,
                          double *best_skin, double *best_cell_frac, double *best_ms);

/* ------------------------------------------------------------------------
 * Confined system (Example 2; contexts created with system =
 * TTCF_CONFINED_LJ).  Pair potential 4[r^-12 - c_ij r^-6] cut at r_c
 * (Eq. 9) between fluid-fluid (c_ff), wall-fluid (c_wf) and wall-wall (c_ww,
 * optional) pairs.  Wall atoms are tethered to lattice
 * sites by springs k and carry a Nose-Hoover thermostat at cfg.T with
 * Q = 3 N_w T tau_T^2 (Eq. 10); during a daughter the bottom lattice moves
 * at -v and the top one at +v in x with v = gamma h / 2.  The dissipation
 * function is Omega = -(1/T) sum_w k (x_w - x_l) s_w v (Eq. 11; s_w = -1
 * bottom, +1 top).  x and z are periodic, y is open.
 * ------------------------------------------------------------------------ */
typedef struct {
    double k;               /* tether stiffness                              */
    double rc;              /* cut-off radius (Example 2: 2.5)                */
    double c_ff, c_wf;      /* wetting coefficients (Example 2: 1.2, 0.6325)  */
    double c_ww;            /* wall-wall coefficient (not given: 1, plain LJ) */
    double h;               /* channel width: v = gamma h / 2 (Example 2: 10) */
    int ww_on;              /* 1: wall-wall pairs interact; 0: tethers only   */
    int pad_;
} ttcf_confined_params;

/* Example 2 values: k 150, r_c 2.5, c_ff 1.2, c_wf 0.6325, h 10; wall-wall
 * pairs interact with c_ww = 1.                                           */
void ttcf_confined_params_default(ttcf_confined_params *p);

/* Append one batch of confined daughters (as ttcf_spawn_daughters, Eq. 3):
 *  n_atoms       N (4 <= N <= 12288, limited by shared memory)
 *  box           [3] Lx, Ly, Lz: x and z periodic (each >= 3 (r_c + skin));
 *                Ly is the extent of the slab profile (walls inside it)
 *  types         [N] 0 fluid, 1 bottom wall, 2 top wall (>= 1 wall atom)
 *  lattice       [3][N] tether sites at t = 0 (rows of fluid atoms unused)
 *  params        potential, tether and channel width; NULL = defaults
 *  mother_soa    [n_mothers][6][N] float64 phase points (x y z px py pz)
 *  mother_alpha  [n_mothers] wall thermostat multipliers, or NULL (zeros)
 *  shear_rates   [n_mothers] gamma of each group (v = gamma h / 2)
 *  ptr_is_device 1 if the five arrays are device pointers, else host
 * Computes, in IEEE double, Omega(0) and the TTCF_CONF_NOBS responses at
 * t = 0 of each mapped daughter.  The mappings reflect x (with the tether
 * sites) and the momenta as in Eq. 3.  Errors: TTCF_E_INVALID (also for a
 * TTCF_BULK_WCA context), TTCF_E_OOM, TTCF_E_CUDA, TTCF_E_STATE.            */
ttcf_status ttcf_spawn_confined(ttcf_ctx *ctx, int n_atoms, const double box[3], const int *types,
                                const double *lattice, const ttcf_confined_params *params,
                                int n_mothers, const double *mother_soa,
                                const double *mother_alpha, const double *shear_rates,
                                int ptr_is_device, int *batch_id);

/* Equilibrium mothers of the confined system on the GPU (lattice at rest):
 * from each of n_init initial phase points [n_init][6][N] (host), n_eq
 * steps, then n_states phase points `spacing` steps apart (x, z wrapped).
 * The thermostat starts from alpha = 0.  out_soa [n_init][n_states][6][N]
 * and out_alpha [n_init][n_states] are host arrays.  chain_status
 * [n_init] (host, may be NULL) receives each chain's TTCF_D_* flags: a
 * flagged chain stopped there and its unwritten states stay zero.  Errors: TTCF_E_NUMERIC if any chain
 * was flagged (the other chains' states are valid), as for ttcf_spawn_*. */
ttcf_status ttcf_sample_mothers_confined(ttcf_ctx *ctx, int n_atoms, const double box[3],
                                         const int *types, const double *lattice,
                                         const ttcf_confined_params *params, int n_init,
                                         const double *init_soa, int n_eq, int n_states,
                                         int spacing, double *out_soa, double *out_alpha,
                                         int *chain_status);

/* ttcf_response for response `observable` of a batch (0 for the bulk
 * system's P_xy; 0 .. TTCF_CONF_NOBS-1 for the confined system).          */
ttcf_status ttcf_response_obs(ttcf_ctx *ctx, int batch_id, int observable, int corrected,
                              double *t, double *dav, double *dav_se, double *corr,
                              double *corr_se, double *ttcf, double *ttcf_se, int capacity,
                              int *n_samples);

/* Slip velocity and friction coefficient at one wall of a confined batch
 * (Eq. 12, <F_x> = xi A <dv>), from its TTCF and direct-average responses,
 * with the slip velocity as the paper defines it (the velocity of the
 * innermost wall layer minus that of the outermost fluid layer):
 *   v_wall(t)  = <sum of p_x over the wall's innermost layer> / n_layer
 *                (response 82 + wall; n_layer atoms: the wall's atoms whose
 *                tether site lies within 0.1 sigma in y of its site plane
 *                nearest the channel),
 *   v_fluid(t) = sum_k <P_k(t)> / sum_k <n_k(t)> over the slabs whose
 *                centres lie within one sigma of the wall on the fluid side,
 *   slip(t) = v_wall(t) - v_fluid(t),
 *   xi(t)   = -<sigma_w(t)> / slip(t), sigma_w being the x force of the
 *             fluid on the wall per area (the wall's force on the fluid is
 *             its negative).
 * wall: 0 bottom, 1 top.  Arrays as in ttcf_response (any may be NULL).
 * Errors: TTCF_E_INVALID (not a confined batch, shear rate differing
 * between groups, bad wall, wall without atoms), TTCF_E_STATE (run not
 * done).                                                                   */
ttcf_status ttcf_friction(ttcf_ctx *ctx, int batch_id, int wall, double *t, double *slip_ttcf,
                          double *slip_dav, double *xi_ttcf, double *xi_dav, int capacity,
                          int *n_samples);

/* Checkpoints (the paper's runs restart from written states, Algorithm 1
 * "write_restart"/"read_restart"; here the whole ensemble).  ttcf_save
 * writes every batch of the context — mothers, shear rates, alphas, the
 * series B and Omega so far, statuses, the loop state of a chunked run —
 * and the step count to the file `path` (host file I/O; device data copied
 * through host memory).  ttcf_load fills a freshly created context (same
 * system, precision, dt, T, tau_T, dof_mode, n_steps, sample_every,
 * mapping_mask, reset_alpha) from such a file; ttcf_run then continues
 * where the saved run stopped, giving bitwise the same series as a run
 * never interrupted.  A finished run is reduced again on load.  The control
 * variate's network is not saved.  Errors: TTCF_E_INVALID (unreadable file,
 * other configuration, malformed contents), TTCF_E_STATE (ttcf_load on a
 * used context), TTCF_E_OOM, TTCF_E_CUDA.                                */
ttcf_status ttcf_save(ttcf_ctx *ctx, const char *path);
ttcf_status ttcf_load(ttcf_ctx *ctx, const char *path);

/* Spawn and run one small batch of daughters without allocating memory.
 *
 * The paper has no counterpart; this is a calling convention.  It is for
 * callers that cannot allocate device memory where they run the daughters:
 * a host application whose device memory is all owned by its own pool
 * allocator (a cudaMalloc there fails or fragments the pool), a
 * latency-critical loop that cannot pay for cudaMalloc/cudaFree (both may
 * synchronise the device), or a plugin whose host forbids allocation after
 * start-up.  It does what ttcf_spawn_daughters followed by ttcf_run does for
 * one batch, with the same kernels and the same results, but takes its
 * working buffers from one 32 MiB array compiled into the library (every
 * GPU that loads the library holds that array until the process exits).
 * No cudaMalloc, cudaFree or other allocating routine is called.
 *
 *  cfg            as for ttcf_create, system TTCF_BULK_WCA only (the
 *                 sheared bulk fluid); stream, precision, dt, T, tau_T,
 *                 dof_mode, n_steps, sample_every, mapping_mask,
 *                 reset_alpha, skin, kernel_variant, block_threads,
 *                 cell_frac are used (with the same defaults as a context
 *                 without autotuning, so the results equal those of
 *                 ttcf_spawn_daughters + ttcf_run bit for bit); allocator
 *                 hooks, keep_state, use_graph and timeout_s are ignored
 *  mother_soa     DEVICE [n_mothers][6][N] float64 phase points
 *  mother_alpha   DEVICE [n_mothers] or NULL (zeros)
 *  shear_rates    DEVICE [n_mothers]
 *  B              DEVICE output [D][S], D = n_mothers * M, S = n_steps /
 *                 sample_every + 1 (B(s) = P_xy(s) as in ttcf_daughter_series)
 *  Omega          DEVICE output [D]; status DEVICE output [D] (TTCF_D_*)
 *
 * Every array must be device (or managed) memory of the current device: a
 * host pointer is rejected with TTCF_E_INVALID (the library cannot check
 * the arrays' sizes, which are the caller's responsibility).
 * All arrays are the caller's.  The call only enqueues work on cfg->stream
 * and returns; results are valid once that stream has completed it.  The
 * first call on each device looks up the array's device address with that
 * device current (make it before any stream capture).  Every call uses the
 * same array, which keeps the previous call's contents (what must start at
 * zero is cleared by each call): calls whose work overlaps on the GPU race
 * and must be serialised by the caller.  A batch whose working buffers do
 * not fit (roughly 6*8*N*n_mothers + 60*D bytes plus one 64*N-byte
 * neighbour list) is rejected with TTCF_E_INVALID before any work is
 * queued.  Errors: TTCF_E_INVALID, TTCF_E_CUDA; the text is available from
 * ttcf_last_error(NULL).                                                   */
ttcf_status ttcf_run_noalloc(const ttcf_config *cfg, int n_atoms, const double box[3],
                             int n_mothers, const double *mother_soa, const double *mother_alpha,
                             const double *shear_rates, double *B, double *Omega, int *status);

/* Equilibrium friction coefficient xi_0 of Eq. 12 by the equilibrium method
 * the paper takes from its references (Hansen, Todd and Daivis 2011;
 * Varghese, Hansen and Todd 2021), at one wall of a finished confined batch
 * run at zero shear rate (its daughters are then equilibrium trajectories
 * with the lattices at rest; a single mapping, mapping_mask = 1, makes them
 * independent).  Per daughter and sample:
 *   dv(t) = slip velocity as in ttcf_friction (inner wall layer velocity
 *           minus the adjacent fluid slabs' velocity),
 *   F(t)  = -A sigma_w(t), the wall's x force on the fluid;
 * correlations over the valid daughters and all time origins, lags k =
 * 0 .. max_lag samples:  c_dvf[k] = <dv(t) F(t+k)>, c_dvdv[k] = <dv(t)
 * dv(t+k)>.  With F(t) = int_0^t zeta(t-u) dv(u) du + R(t), <dv(0)R(t)> = 0,
 * the friction kernel in the Laplace domain is zeta~(s) = C~_dvF(s) /
 * C~_dvdv(s) (trapezoid transforms over the lag window).  A Maxwell kernel
 * zeta~(s) = zeta_0 / (1 + s tau_M) is fitted as the least-squares line
 * 1/zeta~(s) = 1/zeta_0 + (tau_M/zeta_0) s over the n_s values s_grid.
 *   out[0] = xi_0 = zeta_0 / A,  out[1] = zeta_0,  out[2] = tau_M,
 *   out[3] = C~_dvF(0) / C~_dvdv(0) / A (the unfitted estimate).
 * c_dvf, c_dvdv [max_lag + 1] and zeta_s [n_s] (host, may be NULL).
 * Errors: TTCF_E_INVALID (not a confined batch, a nonzero shear rate, bad
 * wall, max_lag outside [1, samples - 2], fewer than 2 Laplace variables),
 * TTCF_E_STATE (run not finished), TTCF_E_OOM, TTCF_E_CUDA.                */
ttcf_status ttcf_friction_equilibrium(ttcf_ctx *ctx, int batch_id, int wall, int max_lag, int n_s,
                                      const double *s_grid, double out[4], double *c_dvf,
                                      double *c_dvdv, double *zeta_s);

/* ------------------------------------------------------------------------
 * Learned control variate.  The paper has no learned part; the estimator it
 * improves is Eq. 1.  A network f: 32 -> 128 -> 128 -> 1 (tanh) learns, from
 * the 32 features x of a mapped mother state, the per-daughter quantity
 * z = Omega(0) I(t_end) / gamma (I: trapezoid integral of B = P_xy), whose
 * group mean y_g = -(1/M) sum_m z is the group's TTCF viscosity at t_end.
 * With h_g = -(1/M) sum_m f(x), the estimate
 *     eta_cv = mean_D(y - c h) + c mean_aux(h)
 * over an evaluation batch D and an independent auxiliary set of mother
 * states is unbiased for any network and c.  Features (in order): kinetic
 * and configurational pressure tensors P^K_ab, P^C_ab (xx yy zz xy xz yz),
 * U/N, K/N, alpha, P_xy^2, then for q = 1..4 the (cos, sin) modes over 40
 * slabs in y of the density and of the x momentum (each / N).  The features
 * of every set of states (training, evaluation, auxiliary) come from one
 * FP32 kernel over the states themselves (cell list of width >= r_c, FP64
 * block sums), so the network is the same function on all sides of the
 * estimator.  Weights are FP32 masters used through their BF16 rounding;
 * FP32 accumulation.
 * ------------------------------------------------------------------------ */
typedef struct {
    int epochs;             /* passes over the training daughters            */
    int batch;              /* minibatch size (a multiple of 32)             */
    float lr, beta1, beta2, eps;   /* Adam                                   */
    float holdout;          /* fraction of groups held out to fit c          */
    unsigned long long seed;/* initialisation and shuffling                  */
} ttcf_cv_config;

/* Defaults: 40 epochs, batch 256, Adam(1e-3, 0.9, 0.999, 1e-8), hold-out
 * 0.2, seed 20231205.                                                      */
void ttcf_cv_config_default(ttcf_cv_config *cfg);

/* Features [D][32] (unstandardised, float) and targets z [D] (double) of
 * every daughter of a finished batch (host arrays; either may be NULL).     */
ttcf_status ttcf_cv_data(ttcf_ctx *ctx, int batch_id, float *X, double *z, size_t capacity);

/* Train the network on the daughters of a finished batch (all shear rates
 * allowed; targets are normalised by gamma).  The last `holdout` fraction
 * of its valid groups is held out: after every epoch the variance reduction
 * of the group control variate on them is measured, the weights of the best
 * epoch are kept (early stopping), and c is fitted on them.  Stores the
 * network in the context; loss_curve (may be NULL) receives the mean
 * training loss per epoch.                                                 */
ttcf_status ttcf_cv_train(ttcf_ctx *ctx, int batch_id, const ttcf_cv_config *cfg,
                          double *loss_curve, int capacity);

/* Control-variate estimate of eta(t_end) for a finished evaluation batch,
 * with n_aux auxiliary mother states [n_aux][6][N] (same N and box; alpha
 * may be NULL), host arrays or device arrays of the context's device (the
 * kind is read from aux_soa; aux_alpha must be of the same kind).  The
 * auxiliary states need their features only: no daughters are spawned for
 * them.  out[8]: eta_plain, se_plain, eta_cv, se_cv, c,
 * gain = se_plain^2 / se_cv^2, n_groups, n_aux.                             */
ttcf_status ttcf_cv_apply(ttcf_ctx *ctx, int batch_id, int n_aux, const double *aux_soa,
                          const double *aux_alpha, double out[8]);

/* The trained network: FP32 parameters [20865] (W1[128][32], b1, W2[128][128],
 * b2, W3[128], b3), feature standardisation [32][2] (mean, std), target
 * standardisation [2] and c.  Any pointer may be NULL.                      */
ttcf_status ttcf_cv_get_model(ttcf_ctx *ctx, float *params, double *feat_stats, double *z_stats,
                              double *c);

/* The network at given FP32 parameters on n standardised inputs X [n][32]
 * (host): outputs [n] (forward), or the mean-squared-loss gradient [20865]
 * and loss for targets y [n] (gradient; n <= 65536).                        */
ttcf_status ttcf_cv_forward(ttcf_ctx *ctx, const float *params, int n, const float *X, float *out);
ttcf_status ttcf_cv_gradient(ttcf_ctx *ctx, const float *params, int n, const float *X,
                             const float *y, float *grad, double *loss);

/* Release the context and all its device memory.  NULL is ignored.       */
void ttcf_destroy(ttcf_ctx *ctx);

/* Last error text of ctx (or of the last failed ttcf_create if ctx is
 * NULL).  Owned by the library; valid until the next call on ctx.         */
const char *ttcf_last_error(const ttcf_ctx *ctx);

/* Library version string (static storage).                                */
const char *ttcf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TTCF_H */
