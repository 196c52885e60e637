/*
 * m2m.h -- C ABI of the GB300 chi^2 made-to-measure (M2M) particle step with
 * moving-prior regularisation (Morganti & Gerhard 2012, "Regularizing
 * made-to-measure particle models of galaxies", arXiv 1202.2355).
 *
 * One context holds one fit: N weighted test particles orbiting in a fixed
 * potential, a set of target observables, and the (E, x) grid of moving
 * priors. Every step advances the particles by leap-frog (Sec. 4.1), deposits
 * their weights into the model observables y_j = sum_i w_i K_j(z_i) (eq. obs),
 * smooths them in time (eq. myts), forms Delta_j and chi^2 (eqs. delta, chi),
 * bins the particles on the (E, L/Lc(E)) grid every `update_every` steps to
 * refresh the priors (Sec. 2.3.1), and applies the force of change
 * dw_i/dt = eps w_i (mu dS/dw_i - sum_j K_ij Delta_j / sigma_j) (eq. modFOC)
 * with the moving-prior entropy of eq. S+ or the global weight entropy of
 * eq. entropy.
 *
 * Conventions for every call:
 *  - Plain C types and pointers only. "host" pointers are ordinary CPU memory;
 *    "device" pointers are CUDA global memory of the context's device.
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes
 *    and of every output buffer it provides. The library owns the context and
 *    the device memory it allocates, released by m2m_destroy.
 *  - Every call returns an m2m_status. No exception or longjmp crosses the ABI.
 *    After an error, m2m_last_error(ctx) gives a one-line description.
 *  - m2m_step is asynchronous on the context's stream. Errors detected on the
 *    device (non-finite or negative weights, fixed-point range overflow) are
 *    latched in a device status word and returned by the next synchronising
 *    call (m2m_synchronize or any m2m_get_*).
 *  - Units are those of the potential descriptor (the workloads use G=M=a=1).
 */
#ifndef M2M_H
#define M2M_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct m2m_ctx m2m_ctx;

typedef enum {
    M2M_OK = 0,
    M2M_ERR_ARG = 1,          /* invalid argument or descriptor */
    M2M_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    M2M_ERR_OOM = 3,          /* device allocation failed */
    M2M_ERR_NONFINITE = 4,    /* a weight became NaN or infinite */
    M2M_ERR_NEG_WEIGHT = 5,   /* the explicit-Euler update made a weight <= 0 */
    M2M_ERR_OVERFLOW = 6,     /* a deposit left the fixed-point range (|v|^2 or total weight) */
    M2M_ERR_TIMEOUT = 7,      /* a bounded device wait expired */
    M2M_ERR_STATE = 8,        /* call not valid in the current state (e.g. no particles) */
    M2M_ERR_TARGET = 9        /* target construction failed (empty aperture for a GH kind) */
} m2m_status;

/* Potentials (all spherical ones are functions of r = |x|). */
enum {
    M2M_POT_HERNQUIST = 0,     /* phi = -G M/(r+a)                                  (eq. her) */
    M2M_POT_HERNQUIST_NFW = 1, /* Hernquist + NFW halo phi_h = -G Ms ln(1+r/rs)/r   */
    M2M_POT_LOG = 2,           /* phi = v0^2/2 ln(r0^2 + R^2 + z^2/q^2)             (eq. log_halo) */
    M2M_POT_SCF = 3            /* phi = Upsilon phi_star + the log halo (Sec. 6): phi_star from the
                                  particles themselves, see m2m_potential */
};

/* Aperture geometries: on the sky, or the 3-D radial grid of the density expansion. */
enum {
    M2M_GEOM_ANNULI = 0,       /* half-open annuli edges[p] <= R < edges[p+1] */
    M2M_GEOM_PIXELS = 1,       /* nx*ny pixels over [xlo,xhi) x [ylo,yhi); p = py*nx + px */
    M2M_GEOM_SHELLS = 2        /* grid radii r_p = edges[p], p < n_ap, of the 3-D radius r, with
                                  cloud-in-cell weights (eq. alm): r_{p-1} <= r < r_p gives
                                  (r_p - r)/(r_p - r_{p-1}) to point p-1 and (r - r_{p-1})/(r_p - r_{p-1})
                                  to point p; r < r_0 gives 1 to point 0; r >= r_{n_ap-1} nothing */
};

/* Observable kinds (kernel K_j of eq. obs, with the aperture selection delta_pi). */
enum {
    M2M_OBS_MASS = 0,          /* surface mass density: K = 1/area_p */
    M2M_OBS_V2 = 1,            /* luminosity-weighted second moment: K = v_los^2 */
    M2M_OBS_GH0 = 10,          /* b_n = l h_n: K = 2 sqrt(pi) u_n(nu), nu = (v_los - V_p)/sigma_p,
                                  kind M2M_OBS_GH0 + n for n = 0..6 (eq. lumghn) */
    M2M_OBS_ALM0 = 100         /* shells only: a_lm,p, K = gamma_p(r) Y_lm(theta, phi) (eq. alm), the total
                                  luminosity carried by the weights; kind M2M_OBS_ALM(l, m) */
};
/* Coefficient of the real spherical harmonic Y_lm, 0 <= l <= M2M_ALM_LMAX, |m| <= l: unit norm
 * over the sphere, without the Condon-Shortley phase; m = 0: N_l0 P_l(cos theta); m > 0:
 * sqrt2 N_lm P_l^m(cos theta) cos(m phi); m < 0: sqrt2 N_l|m| P_l^|m|(cos theta) sin(|m| phi);
 * N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!); theta from the z axis, phi = atan2(y, x). */
#define M2M_OBS_ALM(l, m) (M2M_OBS_ALM0 + (l) * ((l) + 1) + (m))
#define M2M_ALM_LMAX 6

enum { M2M_REG_GWR = 0, M2M_REG_MPR = 1 };            /* eq. entropy / eq. S+ with moving priors */
enum { M2M_E_LOGNEG = 0, M2M_E_EXP = 1, M2M_E_LINEAR = 2 }; /* E-axis bins uniform in ln(-E), exp(E), E */
enum { M2M_PREC_FP64 = 0, M2M_PREC_MIXED = 1 };
enum { M2M_UPDATE_EXP = 0, M2M_UPDATE_EULER = 1 };
/* Deposit strategy of the step kernel. SHARED: per-block fixed-point sums in
 * shared memory, flushed once per block; GLOBAL: every deposit added to the
 * global fixed-point sums (for observable sets too large for shared memory,
 * e.g. 64 x 64 maps of five moments). Both add the same integers, so results
 * are bit-identical. AUTO: SHARED when it fits. */
enum { M2M_DEPOSIT_AUTO = 0, M2M_DEPOSIT_SHARED = 1, M2M_DEPOSIT_GLOBAL = 2 };

#define M2M_MAX_GROUPS 4
#define M2M_MAX_KINDS 16

/* The potential. Unused fields are ignored.
 *
 * M2M_POT_SCF (Sec. 6): the particles move in phi = Upsilon phi_star + phi_D, phi_D the
 * flattened logarithmic halo (v0, r0, q; eq. log_halo) and phi_star the potential of the
 * particles' own light, estimated by a spherical-harmonic expansion with a constant
 * mass-to-light ratio Upsilon. The expansion lives on the grid radii scf_r[0..scf_n) with
 * real harmonics Y_lm (as M2M_OBS_ALM) for l <= scf_lmax: each particle's weight (its
 * luminosity) goes to its grid points with the cloud-in-cell weights of eq. alm, except
 * that r < r_0 goes wholly to r_0 and r >= r_{n-1} wholly to r_{n-1}, so the grid carries
 * thin shells of angular density sum_lm a_lm,k Y_lm, a_lm,k = sum_i w_i gamma_k Y_lm(theta_i,
 * phi_i), and
 *   phi_star(x) = -4 pi G sum_k sum_lm a_lm,k Y_lm(theta, phi) f_l(r, r_k) / (2l + 1),
 *   f_l = r^l / r_k^(l+1) inside the shell (r < r_k), r_k^l / r^(l+1) outside.
 * The expansion is rebuilt from the particles at the load and on the prior schedule (steps
 * 1, 1 + P, ..., after that step's binning) and held fixed in between. With eps_ups > 0 the
 * mass-to-light ratio is determined during the run (Sec. 6): at the same updates
 * d ln Upsilon/dt = -eps_ups sum_j Delta_j/sigma_j D_j over the P steps to the next update,
 * D_j = d y_j/d ln Upsilon when the velocities scale as Upsilon^(1/2) (the chi^2 gradient).
 * Not available in batches or checkpoints. */
typedef struct {
    int32_t kind;
    double G, M, a;        /* Hernquist mass and scale length */
    double Ms, rs;         /* NFW characteristic mass and scale radius */
    double v0, r0, q;      /* logarithmic halo: velocity scale, core radius, flattening */
    int32_t scf_n;         /* M2M_POT_SCF: number of grid radii, 1..64 */
    int32_t scf_lmax;      /* M2M_POT_SCF: highest harmonic degree, 0..6 */
    const double *scf_r;   /* M2M_POT_SCF, host: scf_n strictly increasing grid radii > 0 (copied) */
    double ups;            /* M2M_POT_SCF: initial mass-to-light ratio Upsilon > 0 */
    double eps_ups;        /* M2M_POT_SCF: rate of the mass-to-light update, >= 0 (0: Upsilon fixed) */
} m2m_potential;

/* One group of apertures sharing a geometry; each group carries n_kinds
 * observable kinds measured in every one of its n_ap apertures. */
typedef struct {
    int32_t geometry;              /* M2M_GEOM_* */
    int32_t n_ap;                  /* annuli: number of annuli; pixels: must equal nx*ny; shells:
                                      number of grid radii */
    const double *edges;           /* host: annuli, n_ap+1 strictly increasing radii >= 0; shells, n_ap
                                      strictly increasing grid radii > 0 */
    int32_t nx, ny;                /* pixels only */
    double xlo, xhi, ylo, yhi;     /* pixels only */
    int32_t n_kinds;               /* 1..M2M_MAX_KINDS */
    int32_t kinds[M2M_MAX_KINDS];  /* M2M_OBS_*, each at most once; shells take only
                                      M2M_OBS_ALM(l, m) kinds, the other geometries none of them */
    const double *Vp, *sp;         /* host, n_ap each: Gaussian parameters V_p, sigma_p of the target
                                      LOSVD per aperture (Sec. 3.3); required iff a GH kind is present */
} m2m_obs_group;

/* The observable set. Observable j is ordered group-major, then kind, then
 * aperture: j = offset(group) + kind_index * n_ap + p. J = sum n_kinds*n_ap. */
typedef struct {
    double incl_deg;               /* line of sight n = (0, sin i, cos i); sky axes e1 = (1,0,0),
                                      e2 = (0, cos i, -sin i); v_los = v . n */
    int32_t n_groups;              /* 1..M2M_MAX_GROUPS */
    m2m_obs_group groups[M2M_MAX_GROUPS];
    const double *Y;               /* host, J target values Y_j */
    const double *sigY;            /* host, J errors sigma(Y_j) > 0 */
} m2m_observables;

/* The (E, x) grid of moving priors (Sec. 2.3.1; signed L_z variant of Sec. 5).
 * Cell (k, l) = k*nx + l. k: E bin, uniform in s(E) = ln(-E), exp(E) or E between
 * Emin and Emax, clamped to [0, nE-1] (unbound E >= 0 goes to nE-1 with ln(-E)).
 * l: circularity bin of x = L/Lc(E) in [0,1], or x = Lz/Lc(E) in [-1,1] when
 * signed_lz, clamped; Lc(E) = 0 (no circular orbit) gives x = 0. For GWR the
 * grid is unused and the prior is the flat W0/N. */
typedef struct {
    int32_t mode;                  /* M2M_REG_GWR or M2M_REG_MPR */
    int32_t nE, nx;                /* grid shape, nE*nx <= 4096 */
    int32_t e_spacing;             /* M2M_E_* */
    int32_t signed_lz;
    int32_t update_every;          /* priors recomputed at steps t = 1, 1+P, 1+2P, ... */
    double Emin, Emax;
    int32_t smoothing;             /* M2M_SMOOTH_*: the priors are the raw cell means, or the penalised
                                      spline fit of the grid of cell means (Sec. 2.3.2, eq. smooth_grid) */
    double lambda;                 /* smoothing weight; 0: chosen at every update by generalized cross
                                      validation (golden-section search of log10 lambda in [-4, 6]) */
    int32_t window_E, window_x;    /* grid-less variant (Sec. 7 outlook): >= 0 half widths in cells.
                                      The prior of a particle in cell (k, l) is the mean weight of
                                      the particles in the cells |k'-k| <= window_E, |l'-l| <=
                                      window_x (cut at the grid's edges): a window centred on the
                                      particle's own cell instead of a fixed cell, which tends to
                                      the grid-less window mean as the grid is refined at a fixed
                                      window width. The window sums come from cumulative sums of
                                      the exact integer cell sums. 0, 0: the cell mean of Sec.
                                      2.3.1. Excludes smoothing. */
} m2m_prior_grid;

/* Prior smoothing (Sec. 2.3.2): f minimises |y - f|^2 + lambda sum_cells (f_EE^2 + 2 f_Ex^2
 * + f_xx^2) over the grid of raw cell means y, with second differences in bin units (f_EE,
 * f_xx over interior cells, f_Ex at cell corners): a plane as lambda -> infinity, the means
 * as lambda -> 0. Needs MPR, nE, nx >= 3 and nE*nx <= 4096; the library diagonalises the
 * grid penalty once per grid shape at creation (O((nE nx)^3) host work, about a second at
 * 1000 cells). Cells whose fitted prior is <= 0 exert no entropy force. Not available in
 * batches. */
enum { M2M_SMOOTH_NONE = 0, M2M_SMOOTH_SPLINE_GCV = 1 };

typedef struct {
    int32_t precision;             /* M2M_PREC_FP64: FP64 everywhere. M2M_PREC_MIXED: FP32 state,
                                      push and kernel values; exact int64 fixed-point bin sums;
                                      FP64 residuals, chi^2 and prior means */
    double dt;                     /* leap-frog step */
    int32_t renormalize;           /* 1: rescale weights to the initial total after each update */
    int32_t update_rule;           /* M2M_UPDATE_EXP: w <- w exp(eps dt F) (force held fixed over dt);
                                      M2M_UPDATE_EULER: w <- w (1 + eps dt F) */
    int64_t n_relax;               /* steps t <= n_relax update no weights (Sec. 4.1) */
    void *stream;                  /* cudaStream_t to run on; NULL: the library creates one */
    int32_t block;                 /* threads per block of the step kernel, a multiple of 32: at most
                                      256, or 1024 for the mixed-precision global-deposit kernel;
                                      0: 256 (512 for the global-deposit kernel) */
    int32_t blocks_per_sm;         /* resident blocks per SM; 0: as many as fit. With global
                                      deposits it also sizes the aperture window (a share of
                                      the SM's shared memory per block) */
    int32_t deposit;               /* M2M_DEPOSIT_*: where the step kernel accumulates y_j */
} m2m_options;

/* Create a fit context on the current CUDA device. eps, mu and alpha are the
 * force-of-change rate (eq. modFOC), the regularisation weight (eq. SF) and the
 * per-step temporal smoothing factor (eq. myts discretised as
 * ytil <- ytil + alpha (y - ytil)). All descriptors are copied.
 * Errors: M2M_ERR_ARG on an invalid descriptor, M2M_ERR_CUDA / M2M_ERR_OOM. */
m2m_status m2m_create(const m2m_potential *pot, const m2m_observables *obs,
                      const m2m_prior_grid *prior, double eps, double mu, double alpha,
                      const m2m_options *opt, m2m_ctx **out);

/* Load n particles from host FP64 arrays: pos = x[0..n) y[0..n) z[0..n) (3n
 * values, structure of arrays), vel likewise, w = n weights (> 0 or == 0).
 * Resets the step counter, computes y_0 and sets ytil_0 = y_0, W0 = sum w.
 * n may be 0. Synchronous. Errors: M2M_ERR_ARG (n < 0, null pointer, weight < 0
 * or non-finite), M2M_ERR_OOM, M2M_ERR_CUDA. */
m2m_status m2m_load_particles(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel,
                              const double *w);

/* Same as m2m_load_particles with device FP64 arrays of the same layout. */
m2m_status m2m_load_particles_device(m2m_ctx *ctx, int64_t n, const double *pos_dev,
                                     const double *vel_dev, const double *w_dev);

/* Advance nsteps >= 0 M2M steps, asynchronously on the context stream. */
m2m_status m2m_step(m2m_ctx *ctx, int64_t nsteps);

/* Wait for the context stream; report any latched device error. */
m2m_status m2m_synchronize(m2m_ctx *ctx);

/* Current weights (after the last completed step's update and renormalisation)
 * into the caller's host array of n values (n must equal the loaded count). */
m2m_status m2m_get_weights(m2m_ctx *ctx, double *w, int64_t n);

/* Current positions and velocities, FP64, same layout as m2m_load_particles. */
m2m_status m2m_get_state(m2m_ctx *ctx, double *pos, double *vel, int64_t n);

/* Smoothed (ytil) and raw (y) observables of the last step; either may be NULL. J must match. */
m2m_status m2m_get_observables(m2m_ctx *ctx, double *ytil, double *y, int32_t J);

/* chi^2 = sum Delta_j^2 of the last step (eq. chi) and the number of observables J;
 * delta (J values) receives Delta_j when not NULL. */
m2m_status m2m_get_chi2(m2m_ctx *ctx, double *chi2, int32_t *J, double *delta);

/* Moving priors of the last update: cell mean weights (nE*nx) and particle counts
 * (nE*nx); cells (n values) receives each particle's cell. Any may be NULL. */
m2m_status m2m_get_priors(m2m_ctx *ctx, double *grid_mean, int64_t *counts, int32_t *cells,
                          int64_t n);

/* Prior smoothing on: the raw cell means of the last update (nE*nx, may be NULL) and the
 * smoothing weight used (may be NULL). M2M_ERR_STATE when smoothing is off. */
m2m_status m2m_get_prior_smoothing(m2m_ctx *ctx, double *raw_means, double *lambda);

/* Self-consistent potential (M2M_POT_SCF): the current mass-to-light ratio (may be NULL) and
 * the coefficients a_lm,k of the last expansion (scf_n * (scf_lmax+1)^2 values, grid point
 * major, index l (l+1) + m within a point; may be NULL), the luminosity of the weights as
 * renormalised. M2M_ERR_STATE for other potentials. */
m2m_status m2m_get_scf(m2m_ctx *ctx, double *ups, double *coeffs, int32_t ncoeffs);

/* Number of steps taken since the last load. */
m2m_status m2m_get_step_count(m2m_ctx *ctx, int64_t *t);

/* Number of particles currently loaded (0 before the first load). */
m2m_status m2m_get_particle_count(m2m_ctx *ctx, int64_t *n);

/* Kernel timing. While on, every step-kernel launch (one per step: the
 * finalize runs inside it) is bracketed by CUDA events recorded on the
 * context stream (graph replay is off), and m2m_get_timing returns their
 * summed device time in milliseconds and the number of steps timed since
 * timing was switched on. Either output pointer may be NULL. */
m2m_status m2m_set_timing(m2m_ctx *ctx, int32_t on);
m2m_status m2m_get_timing(m2m_ctx *ctx, double *step_kernel_ms, int64_t *steps);

/* ---- Batches of independent fits ----
 *
 * A batch advances many independent fits (each with its own potential,
 * observable set and targets, prior grid, eps, mu, alpha and particle count)
 * with one kernel launch per step. Every fit of a batch is a full context: its
 * particles are loaded, and its weights, observables, chi^2, priors and state
 * read or checkpointed, through the fit handle m2m_batch_model returns, with the
 * single-fit calls above. m2m_step, m2m_synchronize and the timing calls take the
 * batch handle and act on all fits; the other single-fit calls reject it with
 * M2M_ERR_STATE. All fits share the precision and stream of `opt` and the
 * block-shared deposit (M2M_DEPOSIT_GLOBAL is rejected); a fit advanced in a batch
 * gives bit-identical results to the same fit advanced alone. */

/* Create a batch of nmodels >= 1 fits from arrays of nmodels descriptors and
 * parameters (copied; see m2m_create). Errors: M2M_ERR_ARG naming the first
 * invalid fit, M2M_ERR_CUDA / M2M_ERR_OOM. m2m_destroy(batch) releases every fit. */
m2m_status m2m_create_batch(int32_t nmodels, const m2m_potential *pots, const m2m_observables *obs,
                            const m2m_prior_grid *priors, const double *eps, const double *mu,
                            const double *alpha, const m2m_options *opt, m2m_ctx **out);

/* Number of fits in a batch. */
m2m_status m2m_batch_size(m2m_ctx *batch, int32_t *nmodels);

/* Handle of fit i (0 <= i < nmodels), owned by the batch (m2m_destroy on it does
 * nothing). Stepping it alone advances only that fit. */
m2m_status m2m_batch_model(m2m_ctx *batch, int32_t i, m2m_ctx **model);

/* chi^2 of the last step of every fit of the batch (eq. chi), nmodels values in fit
 * order, in one device-to-host copy; synchronises the batch's stream and reports the
 * first fit whose step flagged an error, like m2m_synchronize. The per-fit call
 * m2m_get_chi2 on each handle gives the same values with one copy per fit. */
m2m_status m2m_batch_get_chi2(m2m_ctx *batch, double *chi2, int32_t nmodels);

/* Times the batched step for a set of launch shapes (threads per block, resident
 * blocks per SM, particles per segment; a segment is a contiguous run of one
 * fit's particles that a block processes before flushing its sums), each over
 * `steps` steps after one warm-up step, and keeps the fastest, returned in the
 * optional outputs. The trial steps are real steps: every fit advances by
 * (steps + 1) times the number of shapes tried (at most 12). The sums are exact
 * integers, so results do not depend on the shape. Requires every fit loaded. */
m2m_status m2m_batch_autotune(m2m_ctx *batch, int32_t steps, int32_t *block, int32_t *blocks_per_sm,
                              int64_t *segment);

/* ---- One fit split over several processes ----
 *
 * The paper's fits run on "the parallel code NMAGIC" (Sec. 1, Sec. 2.1): every step is a
 * sum over particles (eq. obs) followed by work on the sums alone (eqs. myts, delta, chi,
 * the cell means of Sec. 2.3.1). A fit can therefore be split into shards, one per process
 * (typically one per GPU), each holding a contiguous range of the particles. Every shard
 * makes the pass over its own particles; the caller adds the shards' integer sums word by
 * word (an all-reduce: int64 addition, e.g. NCCL's sum over ncclInt64); then every shard
 * runs the same finalize on the same integers. The sums are exact integers, so the split
 * fit is bit-identical to the unsplit one whatever the number of shards: each shard's
 * observables, chi^2, priors and Delta are those of the whole fit, and the shards' weights
 * and particles, concatenated in shard order, are the whole fit's.
 *
 * Protocol, on every shard (all shards use the same descriptors and options):
 *   m2m_shard_bounds on the shard's particles; the caller sums w_sum and takes the maximum
 *     of v2_bound over the shards; m2m_shard_set with those and the total particle count;
 *   m2m_load_particles (its pass), exchange, m2m_step_end (completes the load);
 *   per step: m2m_step_begin, exchange, m2m_step_end;
 *   to read weights: m2m_shard_weights_begin, exchange, m2m_get_weights.
 * "exchange" = replace every shard's words (m2m_shard_exchange) by their sum over the
 * shards, ordered after the shard's stream work (on its stream, or synchronise first).
 * The words are zero outside an exchange. m2m_step and checkpoints are rejected on a shard
 * (M2M_ERR_STATE), and so are the diagnostics of the fit's own particles (pass them
 * explicitly). Device errors are latched per shard and reported by that shard's next
 * synchronising call. */

/* Bounds a shard contributes (host arrays of n particles, layout of m2m_load_particles):
 * the sum of its weights and the largest 2 (E - phi_min) of its particles in the fit's
 * potential, i.e. the largest v^2 it can reach. Synchronous. */
m2m_status m2m_shard_bounds(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel, const double *w,
                            double *w_sum, double *v2_bound);

/* Makes ctx one shard of a fit of n_total particles whose initial weights sum to w_total and
 * whose v2 bound (maximum over the shards of m2m_shard_bounds) is v2_bound. Call it before
 * loading; every shard must pass the same values. A shard whose own particles exceed
 * v2_bound is rejected at load (M2M_ERR_ARG). */
m2m_status m2m_shard_set(m2m_ctx *ctx, int64_t n_total, double w_total, double v2_bound);

/* The device array of int64 words a shard exchanges and their count: the fixed-point sums of
 * the observables, the total weight and the prior grid, one word of the deposited weight
 * for the overflow check, and two words of the weight total for read-outs. Owned by ctx. */
m2m_status m2m_shard_exchange(m2m_ctx *ctx, int64_t **words_dev, int64_t *count);

/* One step's pass over the shard's particles (pending force of change, push, deposit,
 * prior binning on update steps), asynchronous on the shard's stream; its sums are left in
 * the exchange words. With timing on, the pass is what is timed. */
m2m_status m2m_step_begin(m2m_ctx *ctx);

/* The finalize of the step (or of the load) from the summed words: smoothing, Delta_j,
 * chi^2, force-of-change coefficients and, on update steps, the priors. Asynchronous,
 * except after a load. */
m2m_status m2m_step_end(m2m_ctx *ctx);

/* Applies the pending force of change to the shard's weights and leaves their total in the
 * exchange words; after the exchange, m2m_get_weights renormalises them with the whole
 * fit's total and returns them. */
m2m_status m2m_shard_weights_begin(m2m_ctx *ctx);

/* Write / read the full fit state (particles, weights, priors, smoothed
 * observables, step counter, pending update) to / from a file. A context
 * resumed from a file continues bit-identically to an uninterrupted run with
 * the same descriptors; m2m_load_state rejects a file written for different
 * descriptors (M2M_ERR_ARG). */
m2m_status m2m_save_state(m2m_ctx *ctx, const char *path);
m2m_status m2m_load_state(m2m_ctx *ctx, const char *path);

/* Target observables from a target particle realisation (Sec. 3.3): for each
 * aperture the luminosity l_p, then V_p and sigma_p from the mean and rms
 * line-of-sight velocity, corrected with dh1 = -dV/(sqrt2 sigma) and
 * dh2 = -dsigma/(sqrt2 sigma) (eq. h1h2) until |h1|,|h2| <= 1e-12 (at most 200
 * iterations); then Y_j and sigma_j from the per-observable error err[j]
 * (relative on the surface density, relative on v_rms for M2M_OBS_V2, absolute
 * on h_n for GH kinds) with optional Gaussian noise noise[j] (standard normals,
 * may be NULL) added in the same variable. For a_lm kinds on shells (eq. alm)
 * sigma_j = err[j] sqrt(sum_i (w_i gamma_p(r_i))^2 / (4 pi)), the shot noise of the
 * coefficient of an isotropic realisation (the same for every l, m), and Y_j = y_j +
 * sigma_j noise[j]; shells have no V_p, sigma_p (0 and 1 are returned). obs->Y/sigY and the groups' Vp/sp are
 * ignored on input. Outputs are host arrays: Y, sigY (J), Vp, sp (sum of n_ap
 * over groups, group order). Runs on the device in FP64; synchronous.
 * Errors: M2M_ERR_TARGET for an empty aperture in a group with a GH kind. */
m2m_status m2m_build_targets(const m2m_observables *obs, int64_t n, const double *pos,
                             const double *vel, const double *w, const double *err,
                             const double *noise, double *Y, double *sigY, double *Vp,
                             double *sp, int32_t *iterations);

/* Observables without device allocation (annuli and pixels; shell groups are rejected).
 * The paper has no counterpart: this call
 * exists for callers that cannot call cudaMalloc, for example code running inside
 * another runtime's memory pool, under a policy that forbids allocation after
 * start-up, or next to a framework whose allocator owns the device. It computes
 * the raw observables y_j = sum_i w_i K_j(z_i) of n particles given as device FP64
 * arrays (pos, vel: 3n values each, x then y then z; w: n values) for the
 * observable set obs (obs->Y and obs->sigY are ignored), and writes the J values to
 * the device array y_dev, on `stream` (a cudaStream_t, NULL for the default
 * stream). Results agree with m2m_load_particles_device followed by the raw
 * observables of m2m_get_observables to FP64 rounding.
 *
 * It allocates nothing: all scratch lives in one static device array of about
 * 320 KiB that every GPU loading this library holds until the process exits. The
 * array limits J to 8192 observables, the apertures to 8192 and the annulus edges
 * to 8192 in total; larger sets are rejected with M2M_ERR_ARG. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and sets the
 * library's constant tables on that device. Every call copies the aperture tables
 * from host memory, reads its range statistics back into host memory and
 * synchronises `stream` before returning, so no call of it may be made while a
 * stream is being captured into a CUDA graph. Every call reuses the array (its sums
 * are cleared at the start of each call), so calls that overlap on the GPU, on any
 * streams, race: issue them one after another.
 * Errors go to m2m_last_error(NULL): M2M_ERR_ARG for invalid input, M2M_ERR_CUDA,
 * M2M_ERR_OVERFLOW if a deposit left the fixed-point range. */
m2m_status m2m_observe_static(const m2m_observables *obs, int64_t n, const double *pos_dev,
                              const double *vel_dev, const double *w_dev, double *y_dev, void *stream);

/* ------------------------------------------------------------------ diagnostics
 *
 * How well a fit recovers what the data do not show directly (Sec. 4.1): the target's
 * intrinsic kinematics, and its phase-space structure in the (E, x) grid of the priors
 * (Delta_grid); and how smooth the particle model is, as the rms of the weights about
 * their cell means (Sec. 5, Fig. res).
 *
 * The binning calls take either the fit's own particles (n = 0 and pos, vel, w all NULL:
 * the state in the fit's precision and the weights of m2m_get_weights), or n particles
 * from the caller's host arrays (pos, vel: 3n values each, x then y then z; w: n values),
 * for example a realisation of the target. Bins are decided in FP64. Sums are exact integer
 * sums in a two-word fixed point (the integer part and 32 fraction bits of v * 2^s, with s
 * set from the largest |w| and |v|^2 of the particles), converted to FP64 at the end: they
 * equal the FP64 sum to a relative 2^-90 of its bound and are bit-reproducible, whatever the
 * order of the particles. Non-finite particles are rejected (M2M_ERR_ARG). Outputs go to
 * caller-owned host buffers. The calls synchronise the fit's stream. */

/* Spherical polar bins of the intrinsic kinematics (Sec. 4.1): n_r shells, the first
 * [0, r_min) and n_r - 1 shells equally spaced in ln r from r_min to r_max; n_ct equal
 * bins of cos(theta) on [-1, 1], theta from the z axis; n_phi equal bins of the azimuth
 * phi = atan2(y, x) on [-pi, pi] (theta = 0 at the centre, phi = 0 on the z axis; upper
 * edges go to the last bin). Bin b = (i_r * n_ct + i_ct) * n_phi + i_phi. Particles with
 * r >= r_max are not binned. */
typedef struct {
    int32_t n_r, n_phi, n_ct;      /* n_r >= 2, n_phi >= 1, n_ct >= 1, at most 2^24 bins */
    double r_min, r_max;           /* 0 < r_min < r_max */
} m2m_sph_grid;

#define M2M_KIN_SUMS 7             /* per bin: sum w; sum w v_r, w v_theta, w v_phi;
                                      sum w v_r^2, w v_theta^2, w v_phi^2 */

/* Per-bin sums (nbins * M2M_KIN_SUMS doubles, bin-major) and particle counts (nbins,
 * may be NULL) of the particles in the spherical grid; nbins = n_r * n_phi * n_ct.
 * Errors: M2M_ERR_ARG (grid, sizes, arrays), M2M_ERR_STATE (no particles loaded, or a
 * batch handle), M2M_ERR_CUDA / M2M_ERR_OOM. */
m2m_status m2m_diag_kinematics(m2m_ctx *ctx, const m2m_sph_grid *grid, int64_t n, const double *pos,
                               const double *vel, const double *w, double *sums, int64_t *counts,
                               int64_t nbins);

/* Weights of the particles in an (E, x) grid with the fit's potential: per cell the sum of
 * weights wsum, the sum of squared deviations from the cell's mean weight wdev2 (two
 * passes; may be NULL) and the count (may be NULL); ncell = nE * nx. grid NULL: the fit's
 * own MPR grid (a GWR fit must pass one); its mode, update_every and smoothing are
 * ignored. Errors as m2m_diag_kinematics. */
m2m_status m2m_diag_grid(m2m_ctx *ctx, const m2m_prior_grid *grid, int64_t n, const double *pos,
                         const double *vel, const double *w, double *wsum, double *wdev2,
                         int64_t *counts, int32_t ncell);

/* Mean velocities and dispersions (3 per bin: r, theta, phi) from the per-bin sums; bins
 * with fewer than min_count particles or no mass get zeros and valid[b] = 0 (valid may
 * be NULL). Host arithmetic; errors go to m2m_last_error(NULL). */
m2m_status m2m_kin_moments(int64_t nbins, const double *sums, const int64_t *counts, int64_t min_count,
                           double *mean, double *disp, int32_t *valid);

/* Intrinsic-kinematics comparison (Sec. 4.1): over the bins valid in both (as in
 * m2m_kin_moments), the rms of model minus target of each moment: out[0..2] mean v_r,
 * v_theta, v_phi; out[3..5] sigma_r, sigma_theta, sigma_phi; out[6] the rms over all six.
 * bins_used (may be NULL) receives the number of bins compared. Host arithmetic. */
m2m_status m2m_delta_kin(int64_t nbins, const double *sums_model, const int64_t *counts_model,
                         const double *sums_target, const int64_t *counts_target, int64_t min_count,
                         double *out, int64_t *bins_used);

/* Delta_grid (Sec. 4.1): sqrt(sum_c wt_c ((wt_c - wm_c)/wt_c)^2 / sum_c wt_c) with the model's
 * and the target's cell weights each normalised to unit total first; cells without target
 * weight are left out; 0 if either total is not positive. Host arithmetic. */
m2m_status m2m_delta_grid(int32_t ncell, const double *w_model, const double *w_target, double *delta);

/* rms of the particle weights about their cell means (Sec. 5, Fig. res) over the cells
 * with more than min_count particles: sqrt(sum wdev2 / sum counts); 0 if there are none.
 * Host arithmetic. */
m2m_status m2m_weight_rms(int32_t ncell, const double *wdev2, const int64_t *counts, int64_t min_count,
                          double *rms);

/* One-line description of the last error on this context ("" if none); valid
 * until the next call on the context. ctx may be NULL for creation errors. */
const char *m2m_last_error(const m2m_ctx *ctx);

/* Release the context and all device memory it owns. NULL is ignored. */
void m2m_destroy(m2m_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* M2M_H */
