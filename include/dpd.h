/*
 * libdpd — GB300 (sm_103a) simulator of self-propelled DPD dimers
 * (Hinz, Panchenko, Kim & Fried, arXiv:1310.0998).
 *
 * C ABI.  Every entry point returns an int status: DPD_OK (0) or a negative
 * DPD_ERR_* code; dpd_status_string() names it.  Pointers are plain host or
 * device addresses as stated per argument; nothing here takes a CUDA or torch
 * type (streams are passed as void*, a cudaStream_t; NULL makes the context
 * create and own a non-blocking stream).
 *
 * Model (Sec. 2): N beads of mass m in a periodic square of side L; beads 2k
 * and 2k+1 form agent k (2k = head).  Force on bead i:
 *   pair (Eqs. DPDf, DPDcdr, weightFunc01), r < r_c, bonded partner excluded:
 *     [A w - gamma w^2 (v_ij.e) + sqrt(2 gamma kBT) w alpha_ij dt^-1/2] e,
 *     w = 1 - r/r_c, e = (x_i - x_j)/r (minimum image);
 *   bond (Eq. stiffSpring): -kappa (r - r0) e toward the partner's side;
 *   propulsion (Eq. DPDnp): f_p n_k on each bead, n_k = head - tail, unit;
 *   Stokes drag (Eq. DPDnp): -zeta v.
 * Time stepping: standard velocity-Verlet (Sec. 5); the dissipative and drag
 * terms see the half-step velocity; the set-up force of a fresh state sees v.
 * alpha_ij: Philox4x32-10 (Salmon et al., SC'11), counter (min id, max id,
 * step lo, step hi), key (seed lo, seed hi ^ replica), word 0 mapped to
 * sqrt(3) (2 (w0 >> 8) + 1 - 2^24) 2^-24 (uniform, unit variance) or, with
 * noise = 1, Box-Muller on words 0 and 1.
 *
 * State on the ABI: positions x = double[N][2], velocities v = float[N][2],
 * forces f = float[N][2], all in id order.  Inside, positions are 32-bit
 * fixed point (x = X L / 2^32, uniform resolution L 2^-32, exact periodic
 * wrap); a position crosses the ABI as the exact double X L / 2^32 when L
 * has at most 21 significant bits (any L that is a multiple of 2^-8 below
 * 8192, say), so a state read back and set again is unchanged.  FP32
 * velocities and forces; FP64 reductions.
 *
 * Concurrency: a context is not thread-safe; all its work is ordered on its
 * stream.  Calls that return host data synchronise that stream.  Device-side
 * errors (non-finite state, a wait that timed out, an inconsistent cell list)
 * are latched in device memory and returned by the next synchronising call
 * (dpd_sync, any getter); dpd_step itself only reports launch errors.
 */
#ifndef DPD_H_
#define DPD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DPD_OK 0
#define DPD_ERR_INVALID_ARG (-1) /* a parameter or size failed validation      */
#define DPD_ERR_CUDA (-2)        /* a CUDA runtime call failed                 */
#define DPD_ERR_OOM (-3)         /* device allocation failed                   */
#define DPD_ERR_NONFINITE (-4)   /* a position or velocity became non-finite   */
#define DPD_ERR_TIMEOUT (-5)     /* a bounded device wait gave up              */
#define DPD_ERR_STATE (-6)       /* call not valid in the context's state      */
#define DPD_ERR_INTERNAL (-7)    /* cell list inconsistent (bounds check hit)  */

#define DPD_HOST 0   /* pointer argument is a host address   */
#define DPD_DEVICE 1 /* pointer argument is a device address */

/* Model and run parameters (Sec. 2; nondimensional groups of Sec. 3 map onto
 * them as A = Phi f0, kBT = f0 l0 / Pe, gamma = Gamma gamma0, zeta = Gamma_s
 * gamma0).  All lengths in the same unit as r_c. */
typedef struct dpd_params {
    double L;              /* box side, periodic square; L >= 3 r_c          */
    int64_t n_beads;       /* N, even, >= 2 (N/2 agents)                     */
    double a;              /* conservative amplitude A                       */
    double gamma;          /* pairwise friction gamma >= 0                   */
    double kBT;            /* k_B T >= 0                                     */
    double rc;             /* cutoff r_c > 0                                 */
    double k_bond;         /* spring stiffness kappa >= 0                    */
    double r0;             /* spring rest length l >= 0                      */
    double f_p;            /* propulsion per bead f_SP >= 0                  */
    double zeta;           /* Stokes friction gamma_s >= 0                   */
    double dt;             /* time step > 0                                  */
    double mass;           /* bead mass m > 0                                */
    uint64_t seed;         /* random-stream seed                             */
    uint32_t replica;      /* XORed into the high key word                   */
    int32_t exclude_bonded;/* 1 (paper): no pair force inside an agent       */
    int32_t noise;         /* 0: uniform alpha, 1: Gaussian alpha            */
    int32_t tile;          /* cell-block side in cells: 0 = default, else
                              one of 4, 8, 16                                */
    int32_t variant;       /* pair-kernel variant: 0 = default (fastest),
                              1 = thread-per-bead, 2 = pair queue,
                              3 = grid-order pair queue, 4 = flat range
                              enumeration, 5 = pair queue over merged
                              ranges.  tile = variant = 0 takes the
                              shape dpd_autotune cached for this workload,
                              else the built-in default.  Every shape gives
                              the same trajectory bits.                     */
    int32_t reserved;
    double wexp;           /* exponent s of w in the dissipative and random
                              forces (the changed weight exponent the closing
                              section proposes): w_D = w^s, w_R = w^(s/2), so
                              sigma^2 = 2 gamma kBT still sets the temperature;
                              0 or 2 = Eq. (DPDcdr) as printed; 0 <= s <= 8  */
} dpd_params;

typedef struct dpd_ctx dpd_ctx;

/* Geometry and counters of a context. */
typedef struct dpd_info {
    int64_t n_beads;
    int32_t n_cells_side;   /* n_c = floor(L / r_c); cell of x: floor(x n_c / L),
                               exact on the fixed-point grid                 */
    int32_t tile;           /* cell-block side B                             */
    int32_t n_tiles;        /* ceil(n_c/B)^2                                 */
    int32_t variant;        /* pair-kernel variant in use                    */
    int64_t step;           /* current step s of the canonical state         */
    int64_t overflow_tiles; /* tiles that took the global-memory path since
                               creation (tile + halo above shared capacity)  */
    int64_t device_bytes;   /* device memory held by the context             */
} dpd_info;

/* Result of a kernel-shape tuning run: every (tile, variant) timed, in ms per
 * step (-1: the shape did not fit in shared memory), and the fastest. */
typedef struct dpd_tune_report {
    int32_t n_shapes;
    int32_t best_tile, best_variant;
    int32_t reserved;
    double best_ms_per_step;
    int32_t tile[16], variant[16];
    double ms_per_step[16];
} dpd_tune_report;

/* Status text (static storage). */
const char *dpd_status_string(int status);

/* Create a context on the current CUDA device, ordered on `stream`.
 * Validates p (see field comments); allocates all device buffers (about
 * 130 bytes per bead plus 8 bytes per cell).  The state is undefined until
 * dpd_set_state or dpd_init_random.  *out receives the context. */
int dpd_create(const dpd_params *p, void *stream, dpd_ctx **out);

/* Release every resource of ctx; NULL is ignored. */
void dpd_destroy(dpd_ctx *ctx);

/* Replace the interaction/integration parameters.  n_beads, L and r_c must be
 * unchanged (DPD_ERR_STATE otherwise: they fix the cell geometry).  Takes
 * effect at the next step; forces of the current state are not recomputed. */
int dpd_set_params(dpd_ctx *ctx, const dpd_params *p);

/* Set the canonical state at step `step`.  x: [N][2] positions (anywhere;
 * wrapped into [0, L) and rounded to the nearest L 2^-32), v: [N][2]
 * velocities, f: [N][2] forces of that state, or NULL to compute the set-up
 * force F(x, v, step) (velocities v, the random stream of `step`).  where:
 * DPD_HOST or DPD_DEVICE for all pointers.  Non-finite input gives
 * DPD_ERR_NONFINITE.  Synchronises the stream. */
int dpd_set_state(dpd_ctx *ctx, const double *x, const float *v, const float *f, int64_t step, int where);

/* Paper's initial condition (Sec. 5): agent centres uniform in the box,
 * orientations uniform, bond at rest length r0, velocities zero; drawn on the
 * device from Philox4x32-10 (counter (k, 0, 0, 0) for agent k, key (seed lo,
 * seed hi ^ 0x1D17)) so it is reproducible; then the set-up force at step 0. */
int dpd_init_random(dpd_ctx *ctx, uint64_t seed);

/* Advance n >= 0 velocity-Verlet steps (asynchronous on the stream). */
int dpd_step(dpd_ctx *ctx, int64_t n);

/* Wait for the stream and return the latched device status. */
int dpd_sync(dpd_ctx *ctx);

/* Canonical state (x_s, v_s, f_s) and step s.  x: [N][2] (double), v, f:
 * [N][2] (float); any of x, v, f, step may be NULL.  where: DPD_HOST or
 * DPD_DEVICE.  Synchronises. */
int dpd_get_state(dpd_ctx *ctx, double *x, float *v, float *f, int64_t *step, int where);

/* FP64 reductions over the canonical state of the last completed step:
 * kinetic energy 1/2 sum m|v|^2, momentum sum m v, temperature
 * sum m|v|^2 / (2N - 2).  Host outputs.  Synchronise. */
int dpd_kinetic_energy(dpd_ctx *ctx, double *ke);
int dpd_momentum(dpd_ctx *ctx, double p[2]);
int dpd_temperature(dpd_ctx *ctx, double *T);

/* Per-step log of (KE, Px, Py, T) for steps [first, first + count), FP64,
 * host out [count][4].  The log keeps the last 65536 steps; older ones give
 * DPD_ERR_INVALID_ARG.  Synchronises. */
int dpd_thermo_log(dpd_ctx *ctx, int64_t first, int64_t count, double *out);

/* Sec. 5.4 filtered velocity field of the canonical state: agent COM
 * velocity averaged over a square window of side eps centred on the grid
 * point (i + 1/2) L/M (minimum image, closed window), 0 where the window is
 * empty.  eps <= 0 selects eps = L sqrt(10 / N_agents), Eq. (filterwidth).
 * u: host [M][M][2] (row = y), n_in: host [M][M] window counts or NULL.
 * 2 <= M <= 1024.  FP64 accumulation.  Synchronises. */
int dpd_velocity_field(dpd_ctx *ctx, int M, double eps, double *u, double *n_in);

/* Eqs. (fourierTrans01), (ESPf): E(k) = sum over modes with nint|k| = k of
 * (|uhat_x|^2 + |uhat_y|^2)/2 for k = 1..M/2 of the field above, with
 * uhat = M^-2 sum u exp(-2 pi i k.x / L).  M a power of two, 4 <= M <= 1024.
 * E: host [M/2] (E[0] is k = 1).  FP64 FFT on the device.  Synchronises. */
int dpd_energy_spectrum(dpd_ctx *ctx, int M, double eps, double *E);

/* The same E(k) as dpd_energy_spectrum (same arguments and output), computed
 * without allocating any memory.  The paper has no counterpart: this is a
 * property of this library, for callers that must not allocate mid-run (a
 * state sized to fill device memory, where a late cudaMalloc fails; a
 * pipelined run, where cudaMalloc / cudaFree would synchronise the device).
 * Scratch is one static device array per device of 2,622,464 bytes, so
 * M <= 256 (M > 256 gives DPD_ERR_INVALID_ARG); the per-agent staging of the
 * allocating path is fused into the deposit kernel.  The device current at
 * the call must be the one ctx was created on (DPD_ERR_INVALID_ARG
 * otherwise).  The first call on a device looks up the array's address; make
 * it before any stream capture.  The array is shared by every context on the
 * device: calls whose stream work overlaps race on it and return wrong
 * values, so serialise them.  Synchronises. */
int dpd_energy_spectrum_noalloc(dpd_ctx *ctx, int M, double eps, double *E);

/* Sec. 5.3: scalar vorticity omega = (curl u_M) . e_z of the filtered field
 * above (same M, eps), by second-order central differences on the periodic
 * grid: omega = (u_y[iy][ix+1] - u_y[iy][ix-1] - u_x[iy+1][ix] + u_x[iy-1][ix])
 * M / (2 L).  omega: host [M][M] (row = y).  3 <= M <= 1024.  FP64.
 * Synchronises. */
int dpd_vorticity(dpd_ctx *ctx, int M, double eps, double *omega);

/* Eqs. (VCF), (spatial01): all agent pairs with COM separation in
 * [b dr, (b+1) dr), b < nbins (nbins dr <= L/2 advised):
 *   g[b] = (<v_a.v_b>_b - |<v>|^2) / (<|v|^2> - |<v>|^2) (global means),
 * L_int = trapezoid of g over r = 0 (g = 1) and the non-empty bin centres.
 * Host outputs: g [nbins] (NaN for empty bins or a zero denominator), L_int
 * (may be NULL), num [nbins] pair sums and cnt [nbins] pair counts (either
 * may be NULL).  Pair pass on the device over the agent pairs within
 * r_max = nbins dr: a periodic cell grid of side >= r_max when at least three
 * such cells fit per side (O(N_agents rho r_max^2) work), else all agent
 * pairs (O(N_agents^2)); counts and sums are the same either way (FP64
 * minimum image, shells, products).  Synchronises. */
int dpd_velocity_correlation(dpd_ctx *ctx, double dr, int nbins, double *g, double *L_int,
                             double *num, int64_t *cnt);

/* Sec. 5.3 agent velocities: mean over agents of |v_COM|, v_COM = (v_head +
 * v_tail) / 2, of the canonical state (FP64 sum on the device).
 * Synchronises. */
int dpd_agent_speed(dpd_ctx *ctx, double *mean_speed);

/* Debug / parity: per-cell bead counts of the canonical state, row-major
 * [n_c][n_c] host; and per-bead interacting-neighbour counts (r < r_c,
 * bonded excluded) in id order, host [N], with the total pair count
 * (cnt or total may be NULL).  Synchronise. */
int dpd_cell_counts(dpd_ctx *ctx, uint32_t *counts);
int dpd_pair_counts(dpd_ctx *ctx, uint32_t *cnt, uint64_t *total);

int dpd_get_info(dpd_ctx *ctx, dpd_info *info);

/* The first device check that failed since the last set_state/init_random:
 * out[0] = site (0 none, 1 scatter slot or id out of range [values: bead,
 * slot, id], 2 bonded partner slot out of range [slot, id, partner slot],
 * 3 scan wait timed out [block, predecessor, 0]), out[1..3] = values.
 * Synchronises. */
int dpd_error_info(dpd_ctx *ctx, int64_t out[4]);

/* Measurement: advance one step exactly as dpd_step(ctx, 1) does, but with
 * the three kernels launched one by one between CUDA events on the context's
 * stream; ms[0..2] receive the device time of the scan, scatter and fused
 * force/integrate kernels.  Synchronises. */
int dpd_profile_step(dpd_ctx *ctx, double ms[3]);

/* ------------------------------------------------------------------------
 * Batched ensemble: R replicas (uneven box sizes, bead counts and parameters)
 * advanced together by one persistent kernel per call, captured into a CUDA
 * graph per step count.  Each replica is a full context reachable through
 * dpd_batch_replica, so states, observables and logs use the calls above;
 * replicas must not be passed to dpd_destroy (they belong to the batch).
 * All replicas share the tile side and pair-kernel variant of p[0].
 * ------------------------------------------------------------------------ */
typedef struct dpd_batch dpd_batch;

/* p: R parameter sets (1 <= R <= 1023), each validated as in dpd_create. */
int dpd_batch_create(const dpd_params *p, int R, void *stream, dpd_batch **out);
void dpd_batch_destroy(dpd_batch *b);

/* Borrowed handle of replica r (valid until dpd_batch_destroy). */
int dpd_batch_replica(dpd_batch *b, int r, dpd_ctx **view);

/* The paper's initial condition for every replica, replica r with seed + r. */
int dpd_batch_init_random(dpd_batch *b, uint64_t seed);

/* Advance every replica n steps in one persistent launch (asynchronous).
 * Every replica must hold a state.  Grid-wide waits inside the kernel are
 * bounded; a wait that gives up is reported as DPD_ERR_TIMEOUT by
 * dpd_batch_sync. */
int dpd_batch_step(dpd_batch *b, int64_t n);

/* Wait, then return the batch's latched status (the first error of the
 * batch or of any replica). */
int dpd_batch_sync(dpd_batch *b);

/* Failure-detection self-test: launches the grid barrier with one block that
 * never arrives; the others must give up after the bounded wait.  Returns
 * DPD_ERR_TIMEOUT when the timeout fired (the expected outcome) and leaves
 * the batch usable. */
int dpd_batch_barrier_selftest(dpd_batch *b);

/* Replica count, blocks of the persistent launch, (replica, cell block) items. */
int dpd_batch_info(dpd_batch *b, int *n_replicas, int *grid, int *n_work_tiles);

/* Profile of the persistent kernel (no counterpart in the paper): runs
 * nsteps (1..64) ordinary steps of every replica (they advance, as with
 * dpd_batch_step) with the kernel's phase log on.  out[0..2]: mean ms per step
 * of the scan, scatter and force/integrate phases between grid-barrier
 * releases; out[3..5]: the mean over blocks of the ms a block spent working in
 * that phase (the difference is time spent waiting at the barrier).
 * Allocates a small log buffer.  Synchronises. */
int dpd_batch_profile(dpd_batch *b, int nsteps, double out[6]);

/* Kernel-shape autotuner (no counterpart in the paper: its runs used a CPU
 * molecular-dynamics code).  The cell-block side B in {4, 8, 16} and the pair
 * walk variant (1-5) only change how the step's work is cut into CTAs and
 * lanes; all shapes give bit-identical trajectories.
 *
 * dpd_autotune creates a temporary context per shape on `stream` (device
 * memory of one context at a time), loads x, v (id order, [N][2]; `where`
 * says host or device; x = NULL: dpd_init_random(p->seed)), runs two warm-up
 * steps, times `steps` steps twice with CUDA events on the context's stream
 * and keeps the better time.  The fastest shape is returned in rep and cached
 * (process-wide, thread-safe) under the key (n_beads, L, r_c); dpd_create
 * with tile = variant = 0 then uses it.  dpd_batch_autotune does the same for
 * a batch of R replicas (variants 2-5; key: R, sum of N, sum of L^2, sum of
 * N^2) from dpd_batch_init_random(p[0].seed); dpd_batch_create with
 * p[0].tile = p[0].variant = 0 uses it.  Errors of a run are returned as is;
 * DPD_ERR_INVALID_ARG if no shape fits.  dpd_tune_store seeds the cache with a
 * known shape (R = 1: single system), dpd_tune_lookup reads it
 * (DPD_ERR_STATE: not cached), dpd_tune_clear empties it; these three are
 * host-only. */
int dpd_autotune(const dpd_params *p, const double *x, const float *v, int where, int steps, void *stream,
                 dpd_tune_report *rep);
int dpd_batch_autotune(const dpd_params *p, int R, int steps, void *stream, dpd_tune_report *rep);
int dpd_tune_store(const dpd_params *p, int R, int tile, int variant);
int dpd_tune_lookup(const dpd_params *p, int R, int *tile, int *variant);
void dpd_tune_clear(void);

/* ------------------------------------------------------------------------
 * Three-dimensional variant.  Sec. 2 states every force as a vector law; the
 * same pair force, bond, propulsion, drag and velocity-Verlet step (Sec. 5)
 * in a periodic cube of side p->L (fixed-point positions per axis, n_c^3
 * cells of side L / n_c >= r_c).  The paper itself simulates two dimensions.
 * All of dpd_params applies (tile and variant are ignored).  Host pointers.
 * Pair forces are summed in fixed point as in two dimensions, so a run
 * repeats bit for bit; the thermo sums are FP64.
 * ------------------------------------------------------------------------ */
typedef struct dpd3_ctx dpd3_ctx;

/* Create on the current device (about 220 bytes per bead plus 8 per cell). */
int dpd3_create(const dpd_params *p, void *stream, dpd3_ctx **out);
void dpd3_destroy(dpd3_ctx *ctx);

/* Set positions x [N][3] (any, wrapped into the cube and rounded to L 2^-32)
 * and velocities v [N][3] in id order at step `step`, and compute the set-up
 * force F(x, v, step).  Non-finite input gives DPD_ERR_NONFINITE.
 * Synchronises. */
int dpd3_set_state(dpd3_ctx *ctx, const double *x, const float *v, int64_t step);

/* Advance n velocity-Verlet steps (asynchronous; errors latched). */
int dpd3_step(dpd3_ctx *ctx, int64_t n);
int dpd3_sync(dpd3_ctx *ctx);

/* Canonical state in id order: x [N][3] (exact X L / 2^32), v, f [N][3].
 * Synchronises. */
int dpd3_get_state(dpd3_ctx *ctx, double *x, float *v, float *f, int64_t *step);

/* FP64 reductions of the current step: KE = m/2 sum |v|^2, P = m sum v,
 * T = m sum |v|^2 / (3N - 3); out = (KE, Px, Py, Pz, T).  Synchronises. */
int dpd3_thermo(dpd3_ctx *ctx, double out[5]);

/* Observables of Secs. 5.3-5.4 carried to the cube, FP64, from the canonical
 * state of the last call (agent k = beads 2k head, 2k+1 tail; centre of mass
 * c_k = x_tail + minimg(x_head - x_tail)/2 wrapped, v_k = (v_head + v_tail)/2).
 * Filter: cubic window of side eps (eps <= 0: L (10 / N_agents)^(1/3), the
 * window holding 10 agents on average) centred on (i + 1/2) L/M per axis,
 * closed, minimum image; an empty window gives u = 0; eps / (L / M) > 28 is
 * DPD_ERR_INVALID_ARG.  Grids are z-major [iz][iy][ix]; host outputs.
 * Scratch (about 64 M^3 + 64 N_agents bytes) is allocated on first use and
 * kept with the context.  Synchronise. */
/* u [M^3][3] = u_M (x, y, z); n_in [M^3] window counts (may be NULL); 2 <= M <= 256. */
int dpd3_velocity_field(dpd3_ctx *ctx, int M, double eps, double *u, double *n_in);
/* E [M/2]: E(k), k = 1..M/2, uhat = M^-3 sum u exp(-2 pi i k.x/L) per
 * component, E(k) = sum over nint|k| = k of (|uhat_x|^2+|uhat_y|^2+|uhat_z|^2)/2;
 * M a power of two in [4, 256]. */
int dpd3_energy_spectrum(dpd3_ctx *ctx, int M, double eps, double *E);
/* omega [M^3][3] = curl u_M by second-order central differences on the
 * periodic grid of spacing L/M; 3 <= M <= 256. */
int dpd3_vorticity(dpd3_ctx *ctx, int M, double eps, double *omega);
/* Velocity correlation over the agent pairs a < b with COM separation
 * r = sqrt((dx^2 + dy^2) + dz^2) (minimum image) in bin floor(r / dr) <
 * nbins (1 <= nbins <= 4096): g [nbins] as in dpd_velocity_correlation (NaN
 * for an empty bin), *L_int by the trapezoid rule, num / cnt the raw sums
 * and pair counts (may be NULL).  The pairs within r_max = nbins dr come from
 * a periodic cell grid of side >= r_max when at least three such cells fit
 * per side (at most 256), else from all agent pairs (O(N_agents^2)); counts
 * and sums are the same either way. */
int dpd3_velocity_correlation(dpd3_ctx *ctx, double dr, int nbins, double *g, double *L_int, double *num,
                              int64_t *cnt);

/* ------------------------------------------------------------------------
 * Learned surrogate of ensemble statistics (not part of the paper: a model
 * of this simulator's own outputs).  A deep ensemble of K MLPs
 * 4 -> 256 -> 256 -> 40 (SiLU hidden layers, linear output), BF16 weights and
 * activations, FP32 accumulation on the tensor cores, Adam on FP32 master
 * weights.  Input row: (area fraction, gamma, zeta, f_p) (gamma and zeta
 * enter as logarithms); output row: 40 statistics (see the binding's
 * documentation for their order).  Inputs and outputs are standardised with
 * the training set's mean and standard deviation.  Host pointers.
 * ------------------------------------------------------------------------ */
typedef struct sur_ctx sur_ctx;

/* n_members >= 1 MLPs with independent seeded initial weights; max_rows
 * bounds the rows of any later call. */
int sur_create(int n_members, int max_rows, uint64_t seed, void *stream, sur_ctx **out);
void sur_destroy(sur_ctx *s);

/* Replace member weights (FP32 masters; row-major, padded shapes):
 * W1 [256][16] (input columns 4..15 zero), b1 [256], W2 [256][256], b2 [256],
 * W3 [48][256] (rows 40..47 zero), b3 [48]. */
int sur_set_weights(sur_ctx *s, int member, const float *W1, const float *b1, const float *W2, const float *b2,
                    const float *W3, const float *b3);

/* Standardisation of inputs (after the logarithms) and outputs. */
int sur_set_scaling(sur_ctx *s, const float mu_x[4], const float sd_x[4], const float mu_y[40], const float sd_y[40]);

/* One forward and backward pass of one member on (X [n][4], Y [n][40]) with
 * the current scaling: mean squared error of the standardised outputs and
 * its gradients (shapes as in sur_set_weights; any output may be NULL). */
int sur_gradients(sur_ctx *s, int member, const float *X, const float *Y, int n, float *loss, float *gW1,
                  float *gb1, float *gW2, float *gb2, float *gW3, float *gb3);

/* Train every member with Adam (lr) for `epochs` passes over shuffled
 * minibatches of `batch` rows; sets the scaling from (X, Y) first.
 * final_loss: mean squared standardised error of the last epoch. */
int sur_train(sur_ctx *s, const float *X, const float *Y, int n, int epochs, int batch, float lr, float *final_loss);

/* Ensemble mean Y [n][40] and member standard deviation spread [n][40]
 * (may be NULL), in output units.  With n >= 128 rows and the tensor-core
 * backend (the default) the forward products run as tcgen05.mma (BF16 x BF16,
 * FP32 accumulator in tensor memory); a tensor-core wait that gives up
 * returns DPD_ERR_TIMEOUT. */
int sur_predict(sur_ctx *s, const float *X, int n, float *Y, float *spread);

/* Matrix products on tcgen05 (1, default: training products and the fused
 * forward pass of prediction) or on warp-level mma.sync (0). */
int sur_set_backend(sur_ctx *s, int use_tcgen05);

/* Device time of `reps` forward passes of every member over the first n rows
 * of the inputs the last sur_predict uploaded (inputs stay resident; no host
 * copies), between CUDA events; ms_per_pass: per pass of all members. */
int sur_bench_forward(sur_ctx *s, int n, int reps, double *ms_per_pass);

/* The 40 statistics a surrogate row holds, from the snapshots of one run:
 * E [n_snap][n_shells] (E(k), k = 1..n_shells, Sec. 5.4; n_shells >= 64),
 * g [n_snap][nbins] (velocity correlation, bin b centred at (b + 1/2) dr,
 * Sec. 5.3; NaN for an empty bin), T [n_snap], vcom [n_snap] (mean |v_COM|
 * of the agents).  With E and g averaged over the snapshots (g ignoring NaN;
 * a bin NaN in every snapshot counts as 0):
 *   out[0..31]  ln of E averaged over the shell pairs (2b+1, 2b+2)
 *   out[32]     first r with g(r) <= 1/e (linear interpolation from g(0) = 1
 *               over the bin centres), or the last centre when none
 *   out[33]     trapezoid of g over r = 0 and the bin centres
 *   out[34]     mean T
 *   out[35]     least-squares slope of ln(E/E_1) on ln k, k = 1..10
 *   out[36]     the same over k = 30..60
 *   out[37]     k of the largest E(k)
 *   out[38]     ln E_1
 *   out[39]     mean of vcom
 * (ln of a value below 1e-300 takes 1e-300.)  Host pointers; no device work. */
int sur_targets(int n_snap, int n_shells, int nbins, double dr, const double *E, const double *g, const double *T,
                const double *vcom, double out[40]);

/* Simulation protocol behind a surrogate row (phi, gamma, zeta, f_p): a
 * periodic box of side L with N_d = max(1, round(2 phi L^2)) agents
 * (A = 25, kBT = 1, r_c = 1, kappa = 100, r0 = 0.5, dt = 0.01, m = 1), the
 * paper's initial condition, `burn` steps, then `n_snap` snapshots `every`
 * steps apart, each giving E(k) on an M x M grid (M >= 128), g(r) in bins of
 * dr up to L/2, T and the mean |v_COM|. */
typedef struct sur_protocol {
    double L;          /* box side (48 in the training runs)               */
    double dr;         /* correlation bin width (0.25)                      */
    int32_t burn;      /* steps before the first snapshot (2000)           */
    int32_t n_snap;    /* snapshots (10)                                    */
    int32_t every;     /* steps between snapshots (200)                     */
    int32_t M;         /* velocity-field grid side, even, >= 128 (128)      */
    uint64_t seed;     /* row i runs with seed + i and replica i            */
} sur_protocol;

/* Prediction with simulation fallback (the deep ensemble's use): Y [n][40]
 * is the ensemble mean, spread [n][40] the member standard deviation (may be
 * NULL); a row whose largest relative spread max_t spread / (|mean| + 1)
 * exceeds `threshold` is answered instead by running the protocol on the
 * simulator (dpd_* on the surrogate's stream) and reducing it with
 * sur_targets, and used_fallback[i] = 1 (else 0).  n <= max_rows.  Host
 * pointers.  Synchronises. */
int sur_query(sur_ctx *s, const float *X, int n, float threshold, const sur_protocol *proto, float *Y,
              float *spread, int32_t *used_fallback);

#ifdef __cplusplus
}
#endif
#endif /* DPD_H_ */
