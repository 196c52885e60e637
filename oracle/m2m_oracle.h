/*
 * Plain single-threaded FP64 CPU oracle of the chi^2 made-to-measure step with
 * moving-prior regularisation (Morganti & Gerhard 2012, arXiv 1202.2355).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links or calls this
 * code: it exists so that tests, the smoke check and the CPU baseline of the
 * benchmark can compare the CUDA implementation against a slow, literal
 * transcription of the method. It shares no code, header or table with the
 * CUDA library.
 *
 * Units: G, M, a as given by the potential descriptor (the workloads use
 * G = M = a = 1). All arrays are caller-owned; nothing here allocates memory
 * that outlives a call, except where documented.
 */
#ifndef M2M_ORACLE_H
#define M2M_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_GROUPS 4
#define OR_MAX_KINDS 16

/* OR_POT_SCF: phi = Upsilon phi_star + phi_D (Sec. 6): phi_star the multipole expansion of the
 * particles' own luminosity (their weights) on a radial grid, phi_D the flattened log halo */
enum { OR_POT_HERNQUIST = 0, OR_POT_HERNQUIST_NFW = 1, OR_POT_LOG = 2, OR_POT_SCF = 3 };
/* apertures: annuli or pixels on the sky; or the 3-D radial grid of the spherical-harmonic
 * density coefficients (eq. alm), with cloud-in-cell weights between grid radii */
enum { OR_ANNULI = 0, OR_PIXELS = 1, OR_SHELLS = 2 };
/* observable kinds: surface mass density, luminosity-weighted v_los^2, Gauss-Hermite
 * b_n = l h_n for n = 0..6 (kind OR_GH0 + n), and on shells the coefficients a_lm of the
 * real spherical harmonic Y_lm, 0 <= l <= 6, |m| <= l (kind OR_ALM0 + l (l + 1) + m) */
enum { OR_MASS = 0, OR_V2 = 1, OR_GH0 = 10, OR_ALM0 = 100 };
#define OR_ALM_LMAX 6
enum { OR_GWR = 0, OR_MPR = 1 };
enum { OR_E_LOGNEG = 0, OR_E_EXP = 1, OR_E_LINEAR = 2 };
enum { OR_UPDATE_EXP = 0, OR_UPDATE_EULER = 1 };
enum { OR_OK = 0, OR_EARG = 1, OR_EWEIGHT = 2, OR_ETARGET = 3 };

typedef struct {
    int kind;
    double G, M, a;     /* Hernquist: phi = -G M/(r+a) (eq. her) */
    double Ms, rs;      /* NFW: phi = -G Ms ln(1+r/rs)/r */
    double v0, r0, q;   /* flattened log halo (eq. log_halo) */
    /* OR_POT_SCF: the expansion of the stellar potential on scf_n grid radii scf_r (increasing,
     * > 0) with harmonics l <= scf_lmax; scf_a (scf_n (scf_lmax+1)^2 values, caller-owned,
     * rewritten by or_run at every update) holds a_lm,k of the luminosity weights (see
     * or_scf_coeffs); *scf_ups is the mass-to-light ratio Upsilon (caller-owned, updated by
     * or_run when eps_ups > 0). */
    int scf_n, scf_lmax;
    const double *scf_r;
    double *scf_a;
    double *scf_ups;
} or_potential;

typedef struct {
    int geometry;       /* OR_ANNULI or OR_PIXELS */
    int n_ap;           /* number of apertures (annuli, nx*ny pixels, or shell grid radii) */
    const double *edges;/* annuli: n_ap+1 increasing projected radii; shells: n_ap increasing
                           3-D grid radii r_0 > 0 */
    int nx, ny;         /* pixels */
    double xlo, xhi, ylo, yhi;
    int n_kinds;
    int kinds[OR_MAX_KINDS];
    const double *Vp, *sp; /* per aperture: Gaussian parameters of the target LOSVD */
} or_group;

typedef struct {
    double incl_deg;    /* line of sight n = (0, sin i, cos i) */
    int n_groups;
    or_group g[OR_MAX_GROUPS];
} or_obs;

typedef struct {
    int mode;           /* OR_GWR or OR_MPR */
    int nE, nx;
    int e_spacing;      /* OR_E_LOGNEG, OR_E_EXP, OR_E_LINEAR */
    int signed_lz;      /* 0: x = L/Lc in [0,1]; 1: x = Lz/Lc in [-1,1] */
    int update_every;
    double Emin, Emax;
    int smoothing;      /* 0: raw cell means; 1: penalised spline fit of the grid (Sec. 2.3.2) */
    double lambda;      /* smoothing weight; <= 0: chosen by generalized cross validation */
    int window_E, window_x; /* grid-less variant (Sec. 7): half widths, in cells, of the window
                               centred on each particle's cell; 0, 0: the cell means */
} or_prior;

typedef struct {
    double dt, eps, mu, alpha;
    int renormalize;
    int update_rule;    /* OR_UPDATE_EXP or OR_UPDATE_EULER */
    long n_relax;
    double eps_ups;     /* OR_POT_SCF: rate of the mass-to-light update (0: Upsilon fixed) */
} or_params;

typedef struct {
    long n;
    double *x, *y, *z, *vx, *vy, *vz, *w;
} or_particles;

typedef struct {
    int *cell;          /* n: prior cell of each particle (MPR) */
    double *what;       /* n: prior weight of each particle */
    double *grid_mean;  /* nE*nx: cell mean weights at the last prior update */
    long *grid_count;   /* nE*nx */
    double *ytil;       /* J: temporally smoothed observables */
    double *yraw;       /* J: observables of the current snapshot */
    double *delta;      /* J: residuals */
    double chi2, W0;
    long t;
    double *grid_raw;   /* nE*nx: raw cell means before smoothing (may be NULL without smoothing) */
    double lambda;      /* smoothing weight of the last prior update */
} or_state;

int or_num_obs(const or_obs *o);
double or_phi(const or_potential *p, double x, double y, double z);
void or_accel(const or_potential *p, double x, double y, double z,
              double *ax, double *ay, double *az);
void or_leapfrog(const or_potential *p, or_particles *s, double dt);
double or_hermite(int n, double x);
double or_gh_kernel(int n, double nu);
/* Real spherical harmonic, unit norm over the sphere, without the Condon-Shortley phase:
 * m = 0: N_l0 P_l(cos t); m > 0: sqrt2 N_lm P_l^m(cos t) cos(m phi); m < 0: sqrt2 N_l|m|
 * P_l^|m|(cos t) sin(|m| phi); N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_m^m = (2m-1)!!
 * (1 - x^2)^(m/2) >= 0. */
double or_ylm(int l, int m, double cos_theta, double phi);
/* Cloud-in-cell weights of radius r on the grid of a shell group: r_{k-1} <= r < r_k gives
 * (r_k - r)/(r_k - r_{k-1}) to point k-1 and (r - r_{k-1})/(r_k - r_{k-1}) to point k; r < r_0
 * gives 1 to point 0; r >= r_{n-1} nothing. Returns the number of points (0..2). */
int or_cic(const or_group *G, double r, int *k_out, double *g_out);
/* Non-zero entries K_ij of one particle (at most 2 OR_MAX_GROUPS OR_MAX_KINDS): observable
 * index and value. */
int or_kernel_row(const or_obs *o, double x, double y, double z,
                  double vx, double vy, double vz, int *j_out, double *K_out);
void or_kernel_matrix(const or_obs *o, const or_particles *s, double *K);
void or_observe(const or_obs *o, const or_particles *s, double *y);
double or_circular_L(const or_potential *p, double E);

/* ---- Self-consistent stellar potential (Sec. 6) ----
 *
 * The stellar mass is Upsilon times the luminosity the weights carry. Its potential is
 * the multipole expansion on the grid radii r_0 < ... < r_{n-1}: every particle's
 * luminosity is shared between its grid points by the cloud-in-cell weights gamma_k of
 * eq. alm, except that r < r_0 goes wholly to point 0 and r >= r_{n-1} wholly to point
 * n-1 (all the mass counts in a potential), giving thin shells of angular density
 * sum_lm a_lm,k Y_lm with a_lm,k = sum_i w_i gamma_k(r_i) Y_lm(theta_i, phi_i). A shell of
 * radius r_k contributes -4 pi G a_lm,k Y_lm / (2l + 1) times r^l / r_k^(l+1) inside it and
 * r_k^l / r^(l+1) outside, so
 *   phi_star(x) = -4 pi G sum_k sum_lm a_lm,k Y_lm(theta, phi) f_l(r, r_k) / (2l + 1).
 * Index of (l, m): l (l + 1) + m. */
void or_scf_coeffs(const or_potential *p, const or_particles *s, double *a);
/* phi_star (without Upsilon) and its gradient at (x, y, z); grad may be NULL. */
double or_scf_phi(const or_potential *p, double x, double y, double z, double *grad);
/* Derivative of the raw observables with respect to ln Upsilon when the velocities scale
 * as Upsilon^(1/2) at fixed positions: D_j = 1/2 sum_i w_i v_los,i dK_j/dv_los (0 for the
 * surface mass and the a_lm). */
void or_observe_dlnups(const or_obs *o, const or_particles *s, double *D);
int or_cell(const or_potential *p, const or_prior *g, double x, double y, double z,
            double vx, double vy, double vz, double *E_out, double *xc_out);
double or_force(const or_obs *o, const or_params *par, int mode, double w_i, double what_i,
                double x, double y, double z, double vx, double vy, double vz,
                const double *delta, const double *sig);
void or_init(const or_obs *o, const double *Y, const double *sig, const or_prior *g,
             const or_particles *s, or_state *st);
int or_run(const or_potential *p, const or_obs *o, const double *Y, const double *sig,
           const or_prior *g, const or_params *par, or_particles *s, or_state *st, long nsteps);
/* Moving-window means (the grid-less cumulative variant of Sec. 7): for every cell (k, l) the
 * summed weight of the cells (k', l') with |k'-k| <= hE, |l'-l| <= hx (cut at the grid's edges)
 * over their summed particle count; 0 where that count is 0. hE = hx = 0 gives the cell means
 * of Sec. 2.3.1. */
void or_window_means(int nE, int nx, int hE, int hx, const double *sum, const long *count,
                     double *mean);
/* Finite-difference penalty of the prior grid (Sec. 2.3.2, eq. smooth_grid): P such that
 * f.P.f = sum of (f_EE)^2 + 2 (f_Ex)^2 + (f_xx)^2 with second differences in units of one
 * bin, f_EE at cells 1..nE-2 of each column, f_xx at cells 1..nx-2 of each row, f_Ex at the
 * (nE-1)(nx-1) cell corners. Cell (k, l) is k*nx + l; P is dense, n*n, n = nE*nx. */
void or_smooth_penalty(int nE, int nx, double *P);
/* Smoothed grid f minimising |y - f|^2 + lambda f.P.f, i.e. f = (I + lambda P)^-1 y. With
 * lambda <= 0 it is chosen by generalized cross validation: minimise n |(I-A) y|^2 / tr(I-A)^2,
 * A = (I + lambda P)^-1, by a plain golden-section search over log10 lambda in [-4, 6] (40 steps,
 * the middle of the last bracket). lambda_out receives the weight used. Needs nE, nx >= 3.
 * Returns OR_OK or OR_EARG. */
int or_smooth_grid(int nE, int nx, const double *y, double lambda, double *f, double *lambda_out);
/* The GCV score n |(I-A) y|^2 / tr(I-A)^2 at a given lambda > 0 (the quantity or_smooth_grid
 * minimises), so that another code's choice of lambda can be judged by its score. */
int or_smooth_gcv(int nE, int nx, const double *y, double lambda, double *score);

/* ---- Diagnostics of a fitted particle model (Sec. 4.1; Sec. 5, Fig. res) ---- */

/* Spherical polar bins of the intrinsic kinematics: n_r radial shells, the first [0, r_min)
 * and n_r - 1 shells equally spaced in ln r from r_min to r_max (quasi-logarithmic); n_ct
 * equal bins in cos(theta) on [-1, 1] (theta from the z axis); n_phi equal bins in the azimuth
 * phi = atan2(y, x) on [-pi, pi]. Bin (i_r * n_ct + i_ct) * n_phi + i_phi; r >= r_max: -1. */
typedef struct {
    int n_r, n_phi, n_ct;
    double r_min, r_max;
} or_sph_grid;

#define OR_KIN_SUMS 7  /* per bin: sum w, sum w v_r, w v_theta, w v_phi, w v_r^2, w v_theta^2, w v_phi^2 */

int or_sph_bin(const or_sph_grid *g, double x, double y, double z);
/* Velocity components along e_r, e_theta, e_phi. On the z axis phi = 0 is used; at r = 0,
 * e_r = e_z. */
void or_sph_velocity(double x, double y, double z, double vx, double vy, double vz,
                     double *vr, double *vth, double *vph);
/* Per-bin weighted sums (OR_KIN_SUMS per bin) and particle counts, zeroed first. */
void or_kin_sums(const or_sph_grid *g, const or_particles *s, double *sums, long *counts);
/* Mean velocities and dispersions of the bins with at least min_count particles and a
 * positive mass (others: 0 and valid[b] = 0). mean, disp: 3 per bin (r, theta, phi). */
void or_kin_moments(long nbins, const double *sums, const long *counts, long min_count,
                    double *mean, double *disp, int *valid);
/* rms over the bins valid in both models of the difference of each moment, model minus
 * target: out[0..2] mean v_r, v_theta, v_phi; out[3..5] sigma_r, sigma_theta, sigma_phi;
 * out[6] the rms over all six. Returns the number of bins used. */
long or_delta_kin(long nbins, const double *sums_m, const long *counts_m, const double *sums_t,
                  const long *counts_t, long min_count, double *out);
/* Weights of the fit in the (E, x) grid of the priors: per cell the sum of weights, the count,
 * and the sum of squared deviations from the cell's mean weight (two passes). */
void or_grid_weights(const or_potential *p, const or_prior *g, const or_particles *s,
                     double *wsum, double *wdev2, long *count);
/* Mass-weighted relative rms difference of model and target cell weights (Sec. 4.1, eq. of
 * Delta_grid), each normalised to unit total first; cells with no target weight are left out. */
double or_delta_grid(int ncell, const double *w_model, const double *w_target);
/* rms of the particle weights about their cell means over the cells with more than min_count
 * particles (Fig. res): sqrt(sum wdev2 / sum count) over those cells; 0 if there are none. */
double or_weight_rms(int ncell, const double *wdev2, const long *count, long min_count);

int or_build_targets(or_obs *o, const or_particles *tg, const double *err,
                     const double *noise, double *Vp_out, double *sp_out,
                     double *Y_out, double *sig_out, int *iters_out);

#ifdef __cplusplus
}
#endif
#endif
