// Device side of the M2M step: model description, per-particle arithmetic and
// the step kernel. Templated on the state type T: double (FP64 mode) or float
// (mixed mode: FP32 state, push and kernel values; exact integer bin sums).
//
// Method (arXiv 1202.2355): leap-frog push (Sec. 4.1), observables
// y_j = sum_i w_i K_j(z_i) (eq. obs) with the Gauss-Hermite kernels of
// eq. lumghn, temporal smoothing (eq. myts), residuals (eqs. delta, chi),
// (E, x) moving priors (Sec. 2.3.1) and the force of change (eq. modFOC) with
// the entropy of eq. S+ (moving priors) or eq. entropy (global).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "fp64_exp.cuh"

namespace m2m {

constexpr int kMaxGroups = 4;
constexpr int kMaxKinds = 16;
constexpr int kKindMass = 0;
constexpr int kKindV2 = 1;
constexpr int kKindV1 = 2;  // internal: first moment, used only to build targets
constexpr int kKindGH0 = 10;
constexpr int kKindAlm0 = 100;  // a_lm on shells: kKindAlm0 + l (l + 1) + m

enum : unsigned { kErrNonFinite = 1u, kErrNegWeight = 2u, kErrOverflow = 4u, kErrIndex = 8u };

struct GroupDesc {
    int geometry;   // 0 annuli, 1 pixels, 2 shells (3-D radial grid of the a_lm, eq. alm)
    int n_ap;
    int n_kinds;
    int obs_off;    // first observable index of the group
    int ap_off;     // first aperture index (into Vp / 1/sp arrays)
    int edge_off;   // first edge (annuli)
    int max_gh;     // highest Gauss-Hermite order used, -1 if none
    int has_v2;     // the group deposits v_los^2 (range-checked against v2max)
    int nx, ny;
    int kinds[kMaxKinds];
    double xlo, ylo, xw, yw;  // pixel box origin and widths (xhi - xlo, yhi - ylo)
    // FP32 versions: pixel origin and nx/xw, ny/yw; annulus lookup: bucket
    // b = floor((log2 R^2 - l0) lscale) -> first candidate annulus lut[lut_off + b]
    float xlo_f, ylo_f, ixw, iyw;
    int lut_off, lut_n;
    float l0, lscale;
    float e0sq_f, ensq_f;     // squared first and last edge (FP32 annuli)
    int lut_identity;         // edges uniform in log R: bucket b is annulus b (no table load)
    // plan: kind index (0..n_kinds-1) of each kernel in the group, or -1
    int k_mass, k_v2, k_v1;
    int k_gh[7];
    // shells: l and m of each kind, and the factor of the real Y_lm (N_lm, times sqrt2 for m != 0)
    signed char alm_l[kMaxKinds], alm_m[kMaxKinds];
    double alm_norm[kMaxKinds];
    float alm_norm_f[kMaxKinds];
};

struct Model {
    // potential
    int pot;                      // 0 Hernquist, 1 Hernquist + NFW, 2 log
    double G, M, a, Ms, rs, v0, r0, q;
    double phi_min;
    // projection
    double sin_i, cos_i;
    // observables
    int n_groups, J, n_ap_total, n_edges_total, n_lut;
    GroupDesc g[kMaxGroups];
    // priors
    int mode, nE, nx, e_spacing, signed_lz, update_every, ncell;
    double s_lo, s_den;           // E-axis map: f = (s(E) - s_lo) / s_den
    // circular orbits: closed form (Hernquist) or table of E_c(ln R)
    int lc_closed, lc_n;
    double lc_lnr0, lc_dlnr;
    // step
    double dt, eps, mu, alpha;
    int update_rule, renormalize;
    long long n_relax;
    // fixed point: value = words / scale
    double fx_w, fx_v2, fx_gh, v2max;
    int wps;                      // int64 words per sum in the global sums
    int hist_words, off_total, off_grid, off_count;
    int rec_len;                  // doubles per aperture record of the force of change
    // aperture cache: the deposit of a step stores each particle's apertures for the
    // force of change at the start of the next (same positions): 0 none, 1 two groups
    // of at most 255 apertures (8 bits each), 2 one group (16 bits)
    int ap_cache;
    // the acceleration at the current positions is kept between steps (always in FP64)
    int cache_accel;
    // FP64 mode with the aperture cache: exp(-nu^2/2) of this group's aperture (the
    // first group with Gauss-Hermite kernels, -1 none) is also kept from the deposit
    // for the next force of change (same nu, same value)
    int gx_group;
    // prior smoothing (Sec. 2.3.2): 0 off; lambda > 0 fixed, else chosen by GCV
    int smooth;
    double smooth_lambda;
    // grid-less moving priors (Sec. 7): half widths, in cells, of the window of cells
    // centred on each cell whose particles' mean weight is its prior; 0, 0: the cell mean
    int pwin_E, pwin_x;
    // global-deposit kernel: apertures [win_lo, win_lo + win_n) of group win_group keep
    // block-shared sums (the densest range, placed at load); the rest deposit globally
    int win_group, win_lo, win_n;
    // one shard of a fit split over processes: the step kernel leaves its integer sums for
    // the caller to add over the shards, and k_finalize runs the finalize afterwards;
    // n_all is the particle count of the whole fit (the local count when not sharded)
    int shard;
    long long n_all;
    // self-consistent stellar potential (pot 3, Sec. 6): phi = Upsilon phi_star + log halo,
    // phi_star the multipole expansion of the particles' luminosity on scf_n grid radii with
    // harmonics l <= scf_lmax (scf_nlm = (scf_lmax + 1)^2, index l (l + 1) + m). Its sums
    // are the slots [off_scf, off_scf + scf_n scf_nlm), deposited on update steps; with the
    // mass-to-light fit (eps_ups > 0) the derivatives D_j of the observables are the slots
    // [off_dups, off_dups + n_dups). nslots counts every slot of the sums.
    int scf_n, scf_lmax, scf_nlm, off_scf, off_dups, n_dups, nslots;
    double eps_ups, fx_dv;
    const double *scf_r;   // device: grid radii
    double *scf_tab;       // device: per interval j = 0..scf_n, (TA_lm, TB_lm), Upsilon and
                           // -4 pi G/(2l+1) folded in (see scf_field)
    float *scf_tabf;       // FP32 copy
    double *scf_coef;      // device: a_lm,k of the last expansion (scf_n x scf_nlm)
    double scf_norm[49];   // factor of Y_lm (N_lm, sqrt2 N_lm for m != 0) by index
    float scf_norm_f[49];
};

constexpr unsigned kApNone8 = 0xFFu, kApNone16 = 0xFFFFu;
constexpr unsigned kApUncached = 0xFFFFFFFFu;  // no cached code: locate the apertures

// Compile-time shape of an observable group, for step kernels specialised to a
// configuration: bits for the kernels it deposits and its geometry. kDyn: read the
// shape from the runtime GroupDesc (the generic kernel); 0: no such group.
constexpr unsigned kBitMass = 1u, kBitV2 = 2u, kBitV1 = 4u, kBitPix = 1u << 15, kBitShell = 1u << 16;
constexpr unsigned kDyn = 0xFFFFFFFFu;
__host__ __device__ constexpr unsigned bit_gh(int n) { return 8u << n; }
__host__ __device__ constexpr int mask_max_gh(unsigned m, int n = 6)
{
    return n < 0 ? -1 : ((m & bit_gh(n)) ? n : mask_max_gh(m, n - 1));
}

template <unsigned M>
struct GP {
    static constexpr unsigned mask = M;
    static constexpr bool dyn = M == kDyn;
    __device__ static bool present(const Model &m, int g)
    {
        if constexpr (dyn) return g < m.n_groups;
        else return M != 0u;
    }
    __device__ static bool pixels(const GroupDesc &G)
    {
        if constexpr (dyn) return G.geometry == 1;
        else return (M & kBitPix) != 0u;
    }
    __device__ static bool shells(const GroupDesc &G)
    {
        if constexpr (dyn) return G.geometry == 2;
        else return (M & kBitShell) != 0u;
    }
    __device__ static bool mass(const GroupDesc &G)
    {
        if constexpr (dyn) return G.k_mass >= 0;
        else return (M & kBitMass) != 0u;
    }
    __device__ static bool v2(const GroupDesc &G)
    {
        if constexpr (dyn) return G.k_v2 >= 0;
        else return (M & kBitV2) != 0u;
    }
    __device__ static bool v1(const GroupDesc &G)
    {
        if constexpr (dyn) return G.k_v1 >= 0;
        else return (M & kBitV1) != 0u;
    }
    __device__ static bool gh(const GroupDesc &G, int n)
    {
        if constexpr (dyn) return G.k_gh[n] >= 0;
        else return (M & bit_gh(n)) != 0u;
    }
    __device__ static int max_gh(const GroupDesc &G)
    {
        if constexpr (dyn) return G.max_gh;
        else return mask_max_gh(M);
    }
};

// Calls f(GP<M>{}, g) for each present group g, with g a compile-time constant.
template <int G0, unsigned M, unsigned... Rest, class F>
__device__ __forceinline__ void each_group(const Model &m, F &&f)
{
    if (GP<M>::present(m, G0)) f(GP<M>{}, G0);
    if constexpr (sizeof...(Rest) > 0) each_group<G0 + 1, Rest...>(m, f);
}

// Model constants in the state type, so that the FP32 path runs no FP64 operation. The
// batched kernel copies a fit's constants into shared memory in 8-byte words: the struct is
// kept a multiple of 16 bytes so that every element of an array of them is 8-byte aligned.
template <class T>
struct alignas(16) Cst {
    T GM, a, GMs, rs, v0sq, r0sq, q2, phi_min, hn_phi0, sin_i, cos_i;
    T dt, hdt, dteps, mu, v2max, fx_w, fx_v2, fx_gh, fx_dv;
    T s_lo, s_den, e_scale, nE, nx;
    T lc_lnr0, lc_dlnr, lc_r0, lc_rmax;
};

template <class T>
inline Cst<T> make_cst(const Model &m)
{
    Cst<T> k;
    k.GM = T(m.G * m.M); k.a = T(m.a); k.GMs = T(m.G * m.Ms); k.rs = T(m.rs);
    k.v0sq = T(m.v0 * m.v0); k.r0sq = T(m.r0 * m.r0); k.q2 = T(m.q * m.q);
    k.phi_min = T(m.phi_min); k.hn_phi0 = T(m.rs > 0 ? -m.G * m.Ms / m.rs : 0.0);
    k.sin_i = T(m.sin_i); k.cos_i = T(m.cos_i);
    k.dt = T(m.dt); k.hdt = T(0.5 * m.dt); k.dteps = T(m.dt * m.eps); k.mu = T(m.mu);
    k.v2max = T(m.v2max); k.fx_w = T(m.fx_w); k.fx_v2 = T(m.fx_v2); k.fx_gh = T(m.fx_gh); k.fx_dv = T(m.fx_dv);
    k.s_lo = T(m.s_lo); k.s_den = T(m.s_den);
    k.e_scale = T(m.G * m.M > 0 ? m.a / (m.G * m.M) : 0.0);
    k.nE = T(m.nE); k.nx = T(m.nx);
    k.lc_lnr0 = T(m.lc_lnr0); k.lc_dlnr = T(m.lc_dlnr);
    k.lc_r0 = T(exp(m.lc_lnr0)); k.lc_rmax = T(exp(m.lc_lnr0 + (m.lc_n - 1) * m.lc_dlnr));
    return k;
}

// Per-fit scalars living in device memory, written by the finalize.
struct Scalars {
    long long t;        // steps completed
    double wscale;      // current weight = wscale * stored weight (mixed mode)
    double lwscale;     // ln wscale: current ln w = stored ln w + lwscale (FP64 mode)
    double lwhat_flat;  // ln of the flat prior (-inf when it reads 0)
    double W0;          // initial total weight
    double what_flat;   // flat prior W0/N (global entropy)
    double chi2;
    double Wsum;        // total stored weight of the last deposit
    double Wcheck;      // floating-point sum of the deposited weights (range check only)
    double Wrange;      // largest total weight the fixed-point sums can hold
    int pending;        // the previous step's force of change is still to be applied
    unsigned err;       // latched kErr* bits
    unsigned blocks_done;  // blocks of the running step kernel that have flushed their sums
    int smooth_pending;    // new raw cell means wait for the prior smoothing kernels
    unsigned smooth_blocks;   // blocks of the running smoothing kernel that have finished
    double smooth_lambda;  // smoothing weight of the last prior update
    double ups;            // mass-to-light ratio of the self-consistent potential
};

template <class T>
struct State {
    T *x, *y, *z, *vx, *vy, *vz, *w;
    T *fa;            // force factor of the acceleration at the current positions (Model::cache_accel)
    uint16_t *cell;
    uint16_t *ap;     // cached apertures (Model::ap_cache), null without the cache
    T *gx;            // cached exp(-nu^2/2) of Model::gx_group (FP64 mode), else null
    long long n;
};

// FP64 mode stores ln w instead of w: the exponential force-of-change update is
// then an addition and the entropy term -ln(w/what) a subtraction, so the only
// transcendental left per particle for the weight is the exp that recovers w for
// the deposit (mixed mode keeps w: its FP32 ln w would lose ~1e-6 relative per step).
template <class T>
constexpr bool kLogWeights = sizeof(T) == 8;

// The step can keep a(x_t) from the closing half-kick of one step for the opening
// half-kick of the next (the same function of the same positions, so bit-identical
// to recomputing it). Every potential here has a = -f (x, y, z) (spherical) or
// f (x, y, z / q^2) (flattened log halo) with one scalar force factor f, so the factor
// is kept (one state array read and written) and the components are rebuilt from it
// with the same multiplications: bit-identical to keeping the three components, in a
// third of the traffic. FP64 mode always does (it is bound by the FP64 pipe, not by
// HBM); mixed mode does where the force is dear (Model::cache_accel: the Hernquist +
// NFW potential, whose halo term takes a logarithm and a division).
template <class T>
constexpr bool kCacheAccel = sizeof(T) == 8;

// The self-consistent potential is not of the force-factor form: its acceleration is
// evaluated at both ends of the step.
template <class T>
__host__ __device__ __forceinline__ bool keeps_accel(const Model &m)
{
    return m.pot != 3 && (kCacheAccel<T> || m.cache_accel);
}

struct Buffers {
    const double *edges, *Vp, *isp;  // per group edges, per aperture V_p and 1/sigma_p
    const float *Vpf, *ispf;         // FP32 copies of V_p and 1/sigma_p (read from global memory)
    const unsigned short *lut;       // annulus lookup tables (FP32 path)
    const double *lcE;               // E_c table
    const double *Y, *sig;
    const int *obs_kind;             // per observable: kind
    const double *obs_post;          // per observable: factor applied to the raw sum (1/area for mass)
    const double *obs_iscale;        // per observable: 1/fixed-point scale
    double *c;                       // per observable: coefficient of the force of change
    double *rec;                     // per aperture: the data term of eq. modFOC as polynomials in nu
    float *recf;                     // FP32 copy of rec (mixed mode reads it from global memory)
    double *prior;                   // per cell: prior (cell mean weight)
    double *iprior;                  // per cell: 1/prior (0 when the prior reads as 0)
    double *lprior;                  // per cell: ln prior (-inf when the prior reads as 0)
    long long *prior_count;          // per cell: particle count at the last update
    double *prior_raw;               // per cell: raw cell mean before smoothing (smoothing on)
    unsigned long long *pwin;        // window priors: (WPS + 1) x ncell words of cumulative sums
    const double *sV, *sVT, *sD;     // smoothing: eigenvectors of the grid penalty (V, V^T) and eigenvalues
    double *spart, *sz, *ss;         // smoothing scratch: chunk partial sums, V^T y, smoothed coefficients
    long long *hist;                 // global fixed-point sums
    double *ytil, *yraw, *delta;
    Scalars *sc;
};

// ---------------------------------------------------------------- math helpers
// FP32 (mixed mode) uses the hardware approximations on the device: exp and log
// through ex2/lg2 (relative error ~2^-21 |x| for exp), division through rcp. FP64
// keeps the correctly rounded functions.
__host__ __device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__host__ __device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float d_exp(float x)
{
#ifdef __CUDA_ARCH__
    return __expf(x);
#else
    return expf(x);
#endif
}
__host__ __device__ __forceinline__ double d_exp(double x) { return exp(x); }
__host__ __device__ __forceinline__ float d_log(float x)
{
#ifdef __CUDA_ARCH__
    return __logf(x);
#else
    return logf(x);
#endif
}
__host__ __device__ __forceinline__ double d_log(double x) { return log(x); }
__host__ __device__ __forceinline__ float d_div(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fdividef(a, b);
#else
    return a / b;
#endif
}
__host__ __device__ __forceinline__ double d_div(double a, double b) { return a / b; }
__host__ __device__ __forceinline__ float d_log1p(float x) { return log1pf(x); }
__host__ __device__ __forceinline__ double d_log1p(double x) { return log1p(x); }
__host__ __device__ __forceinline__ float d_floor(float x) { return floorf(x); }
__host__ __device__ __forceinline__ double d_floor(double x) { return floor(x); }
// Tests the FP64 step makes on bit patterns, so that they run on the integer pipe
// instead of the FP64 pipe (which bounds that step); FP32 keeps plain compares.
__host__ __device__ __forceinline__ bool is_zero(float v) { return v == 0.f; }
__host__ __device__ __forceinline__ bool is_zero(double v)
{
#ifdef __CUDA_ARCH__
    return (__double_as_longlong(v) << 1) == 0;  // +0 or -0
#else
    return v == 0.0;
#endif
}
// a > b for a, b >= 0 (FP64: a positive NaN counts as greater)
__device__ __forceinline__ bool gt_nonneg(float a, float b) { return a > b; }
__device__ __forceinline__ bool gt_nonneg(double a, double b)
{
    return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool is_neg_inf(double v)
{
    return __double_as_longlong(v) == static_cast<long long>(0xFFF0000000000000ull);
}

__host__ __device__ __forceinline__ bool d_finite(float x) { return isfinite(x); }
__host__ __device__ __forceinline__ bool d_finite(double x) { return isfinite(x); }

// ---------------------------------------------------------------- potentials

// NFW enclosed-mass factor mu(q) = ln(1+q) - q/(1+q), FP64. For small q the two terms
// cancel: below q = 1e-3 the alternating series sum_k (-1)^k (k-1)/k q^k (Horner).
template <class T>
__host__ __device__ __forceinline__ T nfw_mu(T qq)
{
    if (qq < T(1e-3)) {
        T s = T(-10.0 / 11.0);
        s = fma(qq, s, T(9.0 / 10.0));
        s = fma(qq, s, T(-8.0 / 9.0));
        s = fma(qq, s, T(7.0 / 8.0));
        s = fma(qq, s, T(-6.0 / 7.0));
        s = fma(qq, s, T(5.0 / 6.0));
        s = fma(qq, s, T(-4.0 / 5.0));
        s = fma(qq, s, T(3.0 / 4.0));
        s = fma(qq, s, T(-2.0 / 3.0));
        s = fma(qq, s, T(0.5));
        return qq * qq * s;
    }
    return d_log1p(qq) - d_div(qq, T(1) + qq);
}

// FP32: ln(1+q) and mu(q) together without the library log1p. Below q = 1 both come
// from the series in s = q/(2+q) <= 1/3: ln(1+q) = 2 atanh(s) = 2 s sum_{k>=0} s^(2k)/(2k+1),
// and, since 2s - q/(1+q) = s t exactly (t = q/(1+q)),
//   mu = ln(1+q) - t = s t + 2 s^3 P(s^2),  P(u) = sum_{k>=0} u^k/(2k+3),
// a sum of positive terms with no cancellation (8 terms of P, truncation below 1e-9
// relative). Above, ln(1+q) from the hardware log2 (__logf: a few ulp) and
// mu = ln(1+q) - t >= 0.19 without cancellation.
__host__ __device__ __forceinline__ void nfw_logs(float q, float &l1, float &mu)
{
    const float t = d_div(q, 1.f + q);
    if (q < 1.f) {
        const float s = d_div(q, 2.f + q), u = s * s;
        float P = 1.f / 17.f;
#pragma unroll
        for (int k = 6; k >= 0; --k) P = fmaf(u, P, 1.f / float(2 * k + 3));
        const float s3P2 = 2.f * (s * u) * P;
        l1 = fmaf(2.f, s, s3P2);
        mu = fmaf(s, t, s3P2);
    } else {
        l1 = d_log(1.f + q);
        mu = l1 - t;
    }
}

// ---------------------------------------------------------------- self-consistent potential
//
// The stellar potential of pot 3 (Sec. 6) is the multipole expansion of the particles'
// luminosity on grid radii r_0 < ... < r_{n-1} (thin shells, see the host's description
// at m2m_potential). At r in the interval j (r_{j-1} <= r < r_j, r_{-1} = 0, r_n = infinity):
//   phi_star(x) = sum_lm [TA_lm(j) r^-(2l+1) + TB_lm(j)] R_lm(x),
// with R_lm = r^l Y_lm the regular solid harmonic, TA_lm(j) = C_l sum_{k<j} a_lm,k r_k^l (the
// shells inside) and TB_lm(j) = C_l sum_{k>=j} a_lm,k r_k^-(l+1) (the shells outside),
// C_l = -4 pi G Upsilon/(2l+1); the finalize builds these tables on update steps. R_lm =
// N_lm T_lm(z, r^2) Re or Im (x + iy)^m, where T_mm = (2m-1)!!, T_{m+1,m} = (2m+1) z T_mm and
// (l-m) T_lm = (2l-1) z T_{l-1,m} - (l+m-1) r^2 T_{l-2,m} (the recurrences of the associated
// Legendre functions times r^(l-m)); the gradient follows the same recurrences, carried as
// derivatives in z and r^2, with d(x + iy)^m = m (x + iy)^(m-1) (dx + i dy).
constexpr int kScfLmax = 6;
constexpr int kScfMaxRadii = 64;

template <class T>
__device__ __forceinline__ const T *scf_table(const Model &m);
template <>
__device__ __forceinline__ const double *scf_table<double>(const Model &m) { return m.scf_tab; }
template <>
__device__ __forceinline__ const float *scf_table<float>(const Model &m) { return m.scf_tabf; }

// Number of grid radii with r_k^2 <= r2: the interval j of the point.
template <class T>
__device__ __forceinline__ int scf_interval(const Model &m, T r2)
{
    int lo = 0, hi = m.scf_n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const T rk = T(__ldg(m.scf_r + mid));
        if (rk * rk <= r2) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// phi_star (Upsilon included) at (x, y, z) and, if g is not null, its gradient.
template <class T>
__device__ T scf_field(const Model &m, T x, T y, T z, T *g)
{
    const T r2 = fma(x, x, fma(y, y, z * z));
    const int j = scf_interval(m, r2);
    const T *tab = scf_table<T>(m) + size_t(j) * m.scf_nlm * 2;
    const bool inner = j > 0;  // then r >= r_0 > 0
    const T ir2 = inner ? T(1) / r2 : T(0);
    const T ir = inner ? d_sqrt(ir2) : T(0);
    const int L = m.scf_lmax;
    T phi = T(0), gx = T(0), gy = T(0), gz = T(0);
    T cm = T(1), sm = T(0), cm1 = T(0), sm1 = T(0);  // (x + iy)^m and (x + iy)^(m-1)
    T dfac = T(1);                                  // (2m-1)!!
    T irm = ir;                                     // r^-(2m+1)
    for (int mm = 0; mm <= L; ++mm) {
        T t1 = dfac, t1z = T(0), t1r = T(0);  // T_l and its z, r^2 derivatives, l = mm
        T t0 = T(0), t0z = T(0), t0r = T(0);  // T_(l-1)
        T irl = irm;
        for (int l = mm; l <= L; ++l) {
            if (l > mm) {  // the recurrence in l
                const T a = T(2 * l - 1), bq = T(l + mm - 1), il = T(1) / T(l - mm);
                const T tn = (a * z * t1 - bq * r2 * t0) * il;
                const T tnz = (a * (t1 + z * t1z) - bq * r2 * t0z) * il;
                const T tnr = (a * z * t1r - bq * (t0 + r2 * t0r)) * il;
                t0 = t1; t0z = t1z; t0r = t1r;
                t1 = tn; t1z = tnz; t1r = tnr;
                irl *= ir2;
            }
            for (int v = 0; v < (mm > 0 ? 2 : 1); ++v) {
                const int idx = l * (l + 1) + (v == 0 ? mm : -mm);
                const T ta = tab[2 * idx], tb = tab[2 * idx + 1];
                const T N = sizeof(T) == 8 ? T(m.scf_norm[idx]) : T(m.scf_norm_f[idx]);
                const T P = v == 0 ? cm : sm;
                const T R = N * t1 * P;
                const T coef = fma(ta, irl, tb);
                phi = fma(coef, R, phi);
                if (g) {
                    // grad P: cos (m C_(m-1), -m S_(m-1), 0); sin (m S_(m-1), m C_(m-1), 0)
                    const T fm = T(mm);
                    const T px = v == 0 ? fm * cm1 : fm * sm1, py = v == 0 ? -fm * sm1 : fm * cm1;
                    const T gRx = N * fma(T(2) * x * t1r, P, t1 * px);
                    const T gRy = N * fma(T(2) * y * t1r, P, t1 * py);
                    const T gRz = N * (t1z + T(2) * z * t1r) * P;
                    const T rad = ta * T(2 * l + 1) * irl * ir2 * R;  // d r^-(2l+1) / dx_c = -(2l+1) r^-(2l+3) x_c
                    gx = fma(coef, gRx, gx) - rad * x;
                    gy = fma(coef, gRy, gy) - rad * y;
                    gz = fma(coef, gRz, gz) - rad * z;
                }
            }
        }
        cm1 = cm;
        sm1 = sm;
        const T cn = fma(cm, x, -(sm * y));
        sm = fma(cm, y, sm * x);
        cm = cn;
        dfac *= T(2 * mm + 1);
        irm *= ir2;
    }
    if (g) {
        g[0] = gx;
        g[1] = gy;
        g[2] = gz;
    }
    return phi;
}

// Potential and acceleration of the flattened logarithmic halo (eq. log_halo).
template <class T>
__host__ __device__ __forceinline__ T log_halo_phi(const Cst<T> &k, T x, T y, T z)
{
    const T D = fma(x, x, fma(y, y, k.r0sq)) + d_div(z * z, k.q2);
    return T(0.5) * k.v0sq * d_log(D);
}

template <class T>
__device__ __forceinline__ T scf_potential(const Model &m, const Cst<T> &k, T x, T y, T z)
{
#ifdef __CUDA_ARCH__
    return scf_field<T>(m, x, y, z, nullptr) + log_halo_phi(k, x, y, z);
#else
    return T(0);
#endif
}

template <class T>
__device__ __forceinline__ void scf_accel(const Model &m, const Cst<T> &k, T x, T y, T z, T &ax, T &ay, T &az)
{
    T g[3];
    scf_field<T>(m, x, y, z, g);
    const T D = fma(x, x, fma(y, y, k.r0sq)) + d_div(z * z, k.q2);
    const T f = -d_div(k.v0sq, D);
    ax = fma(f, x, -g[0]);
    ay = fma(f, y, -g[1]);
    az = d_div(f * z, k.q2) - g[2];
}

// SCF: whether the code of the self-consistent potential is compiled in (only the generic
// step kernel and the helpers around it need it; the kernels specialised to an observable
// shape run the other potentials without its registers).
template <class T, bool SCF = true>
__host__ __device__ __forceinline__ T potential(const Model &m, const Cst<T> &k, T x, T y, T z)
{
#ifdef __CUDA_ARCH__
    if constexpr (SCF) {
        if (m.pot == 3) return scf_potential(m, k, x, y, z);
    }
#endif
    if (m.pot == 2) {
        const T D = fma(x, x, fma(y, y, k.r0sq)) + d_div(z * z, k.q2);
        return T(0.5) * k.v0sq * d_log(D);
    }
    const T r = d_sqrt(fma(x, x, fma(y, y, z * z)));
    T phi = -d_div(k.GM, r + k.a);
    if (m.pot == 1) {
        if (!(r > T(0))) return phi + k.hn_phi0;
        T l1;
        if constexpr (sizeof(T) == 4) {
            T mu;
            nfw_logs(d_div(r, k.rs), l1, mu);
        } else {
            l1 = d_log1p(d_div(r, k.rs));
        }
        phi -= d_div(k.GMs * l1, r);
    }
    return phi;
}

// Force factor f of the acceleration at (x, y, z): a = -f (x, y, z) in the spherical
// potentials (f = g(r)/r with g = G M(<r)/r^2), a = f (x, y, z/q^2) in the flattened log
// halo (f = -v0^2/D).
template <class T>
__host__ __device__ __forceinline__ T accel_factor(const Model &m, const Cst<T> &k, T x, T y, T z)
{
    if (m.pot == 2) {
        const T D = fma(x, x, fma(y, y, k.r0sq)) + d_div(z * z, k.q2);
        return -d_div(k.v0sq, D);
    }
    const T r2 = fma(x, x, fma(y, y, z * z));
    if (is_zero(r2)) return T(0);
    const T r = d_sqrt(r2);
    const T ra = r + k.a;
    T f = d_div(k.GM, ra * ra * r);
    if (m.pot == 1) {
        T mu;
        if constexpr (sizeof(T) == 4) {
            T l1;
            nfw_logs(d_div(r, k.rs), l1, mu);
        } else {
            mu = nfw_mu(d_div(r, k.rs));
        }
        f += d_div(k.GMs * mu, r2 * r);
    }
    return f;
}

// The acceleration from its force factor (see accel_factor).
template <class T>
__host__ __device__ __forceinline__ void accel_from(const Model &m, const Cst<T> &k, T f, T x, T y, T z, T &ax,
                                                    T &ay, T &az)
{
    if (m.pot == 2) {
        ax = f * x;
        ay = f * y;
        az = d_div(f * z, k.q2);
        return;
    }
    ax = -f * x;
    ay = -f * y;
    az = -f * z;
}

template <class T, bool SCF = true>
__host__ __device__ __forceinline__ void accel(const Model &m, const Cst<T> &k, T x, T y, T z, T &ax, T &ay,
                                               T &az)
{
#ifdef __CUDA_ARCH__
    if constexpr (SCF) {
        if (m.pot == 3) {
            scf_accel(m, k, x, y, z, ax, ay, az);
            return;
        }
    }
#endif
    accel_from(m, k, accel_factor(m, k, x, y, z), x, y, z, ax, ay, az);
}

// One kick-drift-kick leap-frog step from the force factor f at the start position;
// returns the factor at the end position in f.
template <class T>
__device__ __forceinline__ void leapfrog_from(const Model &m, const Cst<T> &k, T &x, T &y, T &z, T &vx, T &vy, T &vz,
                                              T &f)
{
    T ax, ay, az;
    accel_from(m, k, f, x, y, z, ax, ay, az);
    vx = fma(k.hdt, ax, vx);
    vy = fma(k.hdt, ay, vy);
    vz = fma(k.hdt, az, vz);
    x = fma(k.dt, vx, x);
    y = fma(k.dt, vy, y);
    z = fma(k.dt, vz, z);
    f = accel_factor(m, k, x, y, z);
    accel_from(m, k, f, x, y, z, ax, ay, az);
    vx = fma(k.hdt, ax, vx);
    vy = fma(k.hdt, ay, vy);
    vz = fma(k.hdt, az, vz);
}

// One kick-drift-kick leap-frog step.
template <class T, bool SCF = true>
__device__ __forceinline__ void leapfrog(const Model &m, const Cst<T> &k, T &x, T &y, T &z, T &vx, T &vy, T &vz)
{
    T ax, ay, az;
    accel<T, SCF>(m, k, x, y, z, ax, ay, az);
    vx = fma(k.hdt, ax, vx);
    vy = fma(k.hdt, ay, vy);
    vz = fma(k.hdt, az, vz);
    x = fma(k.dt, vx, x);
    y = fma(k.dt, vy, y);
    z = fma(k.dt, vz, z);
    accel<T, SCF>(m, k, x, y, z, ax, ay, az);
    vx = fma(k.hdt, ax, vx);
    vy = fma(k.hdt, ay, vy);
    vz = fma(k.hdt, az, vz);
}

// ---------------------------------------------------------------- observables

// Sky coordinates for the line of sight n = (0, sin i, cos i): X = x (not
// returned), Y = y cos i - z sin i, v_los = vy sin i + vz cos i.
template <class T>
__device__ __forceinline__ void project(const Cst<T> &k, T y, T z, T vy, T vz, T &Y, T &vlos)
{
    Y = fma(y, k.cos_i, -(z * k.sin_i));
    vlos = fma(vy, k.sin_i, vz * k.cos_i);
}

// Aperture of sky point (X, Y) in group G, or -1: half-open annuli
// [edge_p, edge_p+1) in R = sqrt(X^2 + Y^2), decided on R^2 against squared edges
// (so the decision can differ from one made on R only within a few ulp of an
// edge), or pixel p = py nx + px with px = floor((X - xlo) nx / (xhi - xlo)).
// Annuli start from a candidate found from log2 R^2 in FP32 (the annulus itself
// for log-uniform edges, else a lookup table) and are corrected by exact
// comparisons; without a table (lut_n = 0) a binary search is used.
//
// FP64: for R^2 >= 0 the IEEE bit pattern orders like the value, so the
// comparisons run on the integer pipe.
template <unsigned M>
__device__ __forceinline__ int aperture(const GroupDesc &G, const double *esq, const unsigned short *lut,
                                        double X, double Y)
{
    if (!GP<M>::pixels(G)) {
        const double R2 = fma(X, X, Y * Y);
        const long long r = __double_as_longlong(R2);
        const double *e = esq + G.edge_off;
        if (r < __double_as_longlong(e[0]) || r >= __double_as_longlong(e[G.n_ap])) return -1;
        int p;
        if (G.lut_n > 0) {
            int b = __float2int_rd((__log2f(__double2float_rn(R2)) - G.l0) * G.lscale);
            b = b < 0 ? 0 : (b >= G.lut_n ? G.lut_n - 1 : b);
            p = G.lut_identity ? b : int(lut[G.lut_off + b]);
            // the candidate is right but within rounding of an edge or for crowded edges
            if (r < __double_as_longlong(e[p]) || r >= __double_as_longlong(e[p + 1])) {
                while (p > 0 && r < __double_as_longlong(e[p])) --p;
                while (r >= __double_as_longlong(e[p + 1])) ++p;
            }
        } else {
            int lo = 0, hi = G.n_ap;  // e[lo] <= R^2 < e[hi]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__double_as_longlong(e[mid]) <= r) lo = mid;
                else hi = mid;
            }
            p = lo;
        }
        return p;
    }
    const double fx = floor((X - G.xlo) * G.nx / G.xw);
    const double fy = floor((Y - G.ylo) * G.ny / G.yw);
    if (!(fx >= 0.0) || !(fx < G.nx) || !(fy >= 0.0) || !(fy < G.ny)) return -1;
    return int(fy) * G.nx + int(fx);
}

template <unsigned M>
__device__ __forceinline__ int aperture(const GroupDesc &G, const float *e2s, const unsigned short *lut, float X,
                                        float Y)
{
    if (!GP<M>::pixels(G)) {
        const float R2 = fmaf(X, X, Y * Y);
        if (!(R2 >= G.e0sq_f) || !(R2 < G.ensq_f)) return -1;
        int b = __float2int_rd((__log2f(R2) - G.l0) * G.lscale);
        b = b < 0 ? 0 : (b >= G.lut_n ? G.lut_n - 1 : b);
        int p = G.lut_identity ? b : int(lut[G.lut_off + b]);
        const float *e = e2s + G.edge_off;
        // the candidate is right but within rounding of an edge or for crowded edges
        if (R2 < e[p] || R2 >= e[p + 1]) {
            while (p > 0 && R2 < e[p]) --p;
            while (R2 >= e[p + 1]) ++p;
        }
        return p;
    }
    const float fx = floorf((X - G.xlo_f) * G.ixw);
    const float fy = floorf((Y - G.ylo_f) * G.iyw);
    if (!(fx >= 0.f) || !(fx < float(G.nx)) || !(fy >= 0.f) || !(fy < float(G.ny))) return -1;
    return int(fy) * G.nx + int(fx);
}

// ---------------------------------------------------------------- kernel values

// c_n = sqrt(2^(1-n)/n!): K_n = 2 sqrt(pi) u_n(nu) = c_n H_n(nu) exp(-nu^2/2) (eq. lumghn).
__host__ __device__ constexpr double gh_c(int n)
{
    return n == 0 ? 1.4142135623730950488
         : n == 1 ? 1.0
         : n == 2 ? 0.5
         : n == 3 ? 0.20412414523193150818
         : n == 4 ? 0.072168783648703220563
         : n == 5 ? 0.022821773229381921355
                  : 0.0065881721129167866018;
}

enum { kClassMass = 0, kClassVel = 1, kClassGH = 2 };  // fixed-point scale class

template <class T>
struct Tables {
    const T *esq;         // per group squared edges
    const unsigned short *lut;
    const T *vp, *isp;
    const double *e2;     // FP64 mode: 2^(j/32), j < 32 (exp_tab)
};

// exp of the kernel values and weights: the ex2-based approximation in mixed mode,
// the table-driven exp_tab in FP64 mode.
__device__ __forceinline__ float kexp(const Tables<float> &, float x) { return __expf(x); }
__device__ __forceinline__ double kexp(const Tables<double> &tb, double x) { return exp_tab(x, tb.e2); }

// Emits emit(slot, w K_slot, class, kind index in the group) for every kernel of group G
// at aperture p:
// surface mass (K = 1), v_los^2, v_los, and the Gauss-Hermite b_n with H_n from the
// recurrence H_{n+1} = 2 nu H_n - 2 n H_{n-1}, evaluated once up to the group's
// highest order.
template <unsigned M, class T, class F>
__device__ __forceinline__ void group_kernels(const GroupDesc &G, const Tables<T> &tb, int p, T vlos, T w, F &&emit,
                                              T *gexp_out = nullptr)
{
    using P = GP<M>;
    const int base = G.obs_off + p;
    if (P::mass(G)) emit(base + G.k_mass * G.n_ap, w, kClassMass, G.k_mass);
    if (P::v2(G)) emit(base + G.k_v2 * G.n_ap, w * vlos * vlos, kClassVel, G.k_v2);
    if (P::v1(G)) emit(base + G.k_v1 * G.n_ap, w * vlos, kClassVel, G.k_v1);
    const int nmax = P::max_gh(G);
    if (nmax >= 0) {
        const T nu = (vlos - tb.vp[G.ap_off + p]) * tb.isp[G.ap_off + p];
        const T ge = kexp(tb, T(-0.5) * nu * nu);
        if (gexp_out) *gexp_out = ge;
        const T we = w * ge;
        T hm1 = T(1), h = T(2) * nu;
        if (P::gh(G, 0)) emit(base + G.k_gh[0] * G.n_ap, T(gh_c(0)) * we, kClassGH, G.k_gh[0]);
        if (P::gh(G, 1)) emit(base + G.k_gh[1] * G.n_ap, h * we, kClassGH, G.k_gh[1]);
#pragma unroll
        for (int n = 1; n < 6; ++n) {
            if (n < nmax) {
                const T hn1 = fma(T(2) * nu, h, -(T(2 * n) * hm1));
                hm1 = h;
                h = hn1;
                if (P::gh(G, n + 1))
                    emit(base + G.k_gh[n + 1] * G.n_ap, T(gh_c(n + 1)) * h * we, kClassGH, G.k_gh[n + 1]);
            }
        }
    }
}

// The data term of eq. modFOC, sum_j K_j c_j, for one particle. In aperture p of a
// group every kernel is a polynomial in nu = (v_los - V_p)/sigma_p, the Gauss-
// Hermite ones times exp(-nu^2/2), so the finalize folds the coefficients c_j into
// one record per aperture, r = [V_p, 1/sigma_p, q0, q1, q2, p0 .. p_nmax], and
// sum_j K_j c_j = q0 + q1 nu + q2 nu^2 + exp(-nu^2/2) sum_n p_n nu^n
// (groups without Gauss-Hermite kernels use V = 0, 1/sigma = 1, i.e. nu = v_los).
// The first n values of a record (n <= 12), with 16-byte loads: records start on 16-byte
// boundaries (Model::rec_len is a multiple of 4).
__device__ __forceinline__ void load_record(const float *r, float *v, int n)
{
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (4 * q < n) {
            const float4 a = reinterpret_cast<const float4 *>(r)[q];
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
}
__device__ __forceinline__ void load_record(const double *r, double *v, int n)
{
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (2 * q < n) {
            const double2 a = reinterpret_cast<const double2 *>(r)[q];
            v[2 * q] = a.x;
            v[2 * q + 1] = a.y;
        }
}

template <unsigned M, class T>
__device__ __forceinline__ T group_data(const Model &m, const GroupDesc &G, const Tables<T> &tb, const T *rec, int p,
                                        T vlos, const T *gexp = nullptr)
{
    const T *rp = rec + (G.ap_off + p) * m.rec_len;
    const int nmax = GP<M>::max_gh(G);
    if (!GP<M>::v2(G) && !GP<M>::v1(G) && nmax < 0) return rp[2];  // surface mass only: a constant
    T r[12];
    load_record(rp, r, 6 + nmax);
    const T nu = (vlos - r[0]) * r[1];
    T d = fma(nu, fma(nu, r[4], r[3]), r[2]);
    if (nmax >= 0) {
        T poly = T(0);
#pragma unroll
        for (int n = 6; n >= 0; --n)
            if (n <= nmax) poly = fma(poly, nu, r[5 + n]);
        d = fma(gexp ? *gexp : kexp(tb, T(-0.5) * nu * nu), poly, d);
    }
    return d;
}

// ---- shells: the spherical-harmonic density coefficients of eq. alm
//
// a_lm,p = sum_i w_i gamma_p(r_i) Y_lm(theta_i, phi_i) on grid radii r_0 < ... < r_{n-1}
// (the total luminosity is carried by the weights). gamma is the cloud-in-cell weight:
// between r_{p-1} and r_p linear in r, inside r_0 all on point 0, none beyond r_{n-1}.
// Y_lm is the real spherical harmonic of unit norm without the Condon-Shortley phase,
// from the recurrences P_m^m = (2m-1)!! sin^m, P_{m+1}^m = (2m+1) cos P_m^m,
// (l-m) P_l^m = (2l-1) cos P_{l-1}^m - (l+m-1) P_{l-2}^m, and cos(m phi), sin(m phi) as the
// powers of cos phi + i sin phi.

// Grid points and cloud-in-cell weights of squared radius r2 (the group's squared grid
// radii at esq + edge_off): returns 0, 1 (point p0, weight 1) or 2 (p0 and p0 + 1).
template <class T>
__device__ __forceinline__ int shell_cic(const GroupDesc &G, const T *esq, T r2, int &p0, T &g0, T &g1)
{
    const T *e = esq + G.edge_off;
    const int n = G.n_ap;
    if (!(r2 < e[n - 1])) return 0;
    if (r2 < e[0]) {
        p0 = 0;
        g0 = T(1);
        g1 = T(0);
        return 1;
    }
    int lo = 0, hi = n - 1;  // e[lo] <= r2 < e[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= r2) lo = mid;
        else hi = mid;
    }
    const T r = d_sqrt(r2), ra = d_sqrt(e[lo]), rb = d_sqrt(e[hi]);
    const T d = rb - ra;
    p0 = lo;
    g0 = d_div(rb - r, d);
    g1 = d_div(r - ra, d);
    return 2;
}

// Direction cosines of (x, y, z): cos and sin of theta (from the z axis) and of phi;
// theta = 0 at the centre and phi = 0 on the z axis.
template <class T>
__device__ __forceinline__ void shell_angles(T x, T y, T z, T &ct, T &st, T &cp, T &sp)
{
    // explicit fused forms: the same rounding in every kernel that inlines this
    const T R2 = fma(x, x, y * y);
    const T R = d_sqrt(R2), r = d_sqrt(fma(z, z, R2));
    const bool c = r > T(0), a = R > T(0);
    ct = c ? d_div(z, r) : T(1);
    st = c ? d_div(R, r) : T(0);
    cp = a ? d_div(x, R) : T(1);
    sp = a ? d_div(y, R) : T(0);
}

// Y_lm of kind kk of a shell group.
template <class T>
__device__ __forceinline__ T shell_ylm(const GroupDesc &G, int kk, T ct, T st, T cp, T sp)
{
    const int l = G.alm_l[kk], m = G.alm_m[kk], am = m < 0 ? -m : m;
    T pmm = T(1);
    for (int i = 1; i <= am; ++i) pmm *= T(2 * i - 1) * st;
    T plm = pmm;
    if (l > am) {
        T p0 = pmm, p1 = ct * T(2 * am + 1) * pmm;
        for (int ll = am + 2; ll <= l; ++ll) {
            const T p2 = d_div(fma(ct * T(2 * ll - 1), p1, -(T(ll + am - 1) * p0)), T(ll - am));
            p0 = p1;
            p1 = p2;
        }
        plm = p1;
    }
    T c = T(1), s = T(0);
    for (int i = 0; i < am; ++i) {
        const T c2 = fma(c, cp, -(s * sp));
        s = fma(s, cp, c * sp);
        c = c2;
    }
    const T nrm = sizeof(T) == 8 ? T(G.alm_norm[kk]) : T(G.alm_norm_f[kk]);
    return nrm * plm * (m > 0 ? c : (m < 0 ? s : T(1)));
}

// emit(slot, w K_slot, class, kind index) for every a_lm of the group at the particle's
// one or two grid points.
template <class T, class F>
__device__ __forceinline__ void shell_kernels(const GroupDesc &G, const Tables<T> &tb, T x, T y, T z, T w, F &&emit)
{
    int p0 = 0;
    T g0 = T(0), g1 = T(0);
    const int np = shell_cic(G, tb.esq, fma(z, z, fma(x, x, y * y)), p0, g0, g1);
    if (np == 0) return;
    T ct, st, cp, sp;
    shell_angles(x, y, z, ct, st, cp, sp);
    for (int kk = 0; kk < G.n_kinds; ++kk) {
        const T v = w * shell_ylm(G, kk, ct, st, cp, sp);
        const int j = G.obs_off + kk * G.n_ap + p0;
        emit(j, g0 * v, kClassGH, kk);
        if (np == 2) emit(j + 1, g1 * v, kClassGH, kk);
    }
}

// sum_j K_j c_j over the group's a_lm: the records of a shell group hold c_j per kind.
template <class T>
__device__ __forceinline__ T shell_data(const Model &m, const GroupDesc &G, const Tables<T> &tb, const T *rec, T x,
                                        T y, T z)
{
    int p0 = 0;
    T g0 = T(0), g1 = T(0);
    const int np = shell_cic(G, tb.esq, fma(z, z, fma(x, x, y * y)), p0, g0, g1);
    if (np == 0) return T(0);
    T ct, st, cp, sp;
    shell_angles(x, y, z, ct, st, cp, sp);
    const T *r0 = rec + (G.ap_off + p0) * m.rec_len;
    T d0 = T(0), d1 = T(0);
    for (int kk = 0; kk < G.n_kinds; ++kk) {
        const T Y = shell_ylm(G, kk, ct, st, cp, sp);
        d0 = fma(Y, r0[kk], d0);
        if (np == 2) d1 = fma(Y, r0[m.rec_len + kk], d1);
    }
    return fma(g0, d0, g1 * d1);
}

template <unsigned... Ms, class T>
__device__ __forceinline__ T data_term(const Model &m, const Tables<T> &tb, const T *rec, T x, T y, T z, T X,
                                       T Y, T vlos)
{
    T data = T(0);
    each_group<0, Ms...>(m, [&](auto P, int g) {
        constexpr unsigned M = decltype(P)::mask;
        const GroupDesc &G = m.g[g];
        if (GP<M>::shells(G)) {
            data += shell_data(m, G, tb, rec, x, y, z);
            return;
        }
        const int p = aperture<M>(G, tb.esq, tb.lut, X, Y);
        if (p >= 0) data += group_data<M>(m, G, tb, rec, p, vlos);
    });
    return data;
}

// Aperture of group g in a cached code (Model::ap_cache), -1 outside.
__device__ __forceinline__ int ap_decode(const Model &m, unsigned code, int g)
{
    if (m.ap_cache == 2) return code == kApNone16 ? -1 : int(code);
    const unsigned a = (code >> (8 * g)) & 0xFFu;
    return a == kApNone8 ? -1 : int(a);
}

__device__ __forceinline__ unsigned ap_encode(const Model &m, unsigned code, int g, int p)
{
    if (m.ap_cache == 2) return p < 0 ? kApNone16 : unsigned(p);
    return (code & ~(0xFFu << (8 * g))) | ((p < 0 ? kApNone8 : unsigned(p)) << (8 * g));
}

// data_term with the apertures taken from a cached code.
template <unsigned... Ms, class T>
__device__ __forceinline__ T data_term_cached(const Model &m, const Tables<T> &tb, const T *rec, unsigned code,
                                              T vlos, const T *gexp)
{
    T data = T(0);
    each_group<0, Ms...>(m, [&](auto P, int g) {
        constexpr unsigned M = decltype(P)::mask;
        const int p = ap_decode(m, code, g);
        if (p >= 0) data += group_data<M>(m, m.g[g], tb, rec, p, vlos, g == m.gx_group ? gexp : nullptr);
    });
    return data;
}

// ---- deposits of the self-consistent potential

// emit(slot, w gamma_k Y_lm) of the expansion (Sec. 6): the particle's luminosity on its
// one or two grid points, cloud-in-cell weights as eq. alm except that r < r_0 goes wholly to
// point 0 and r >= r_{n-1} wholly to point n-1; Y_lm from the associated-Legendre recurrences
// in cos(theta) and the powers of cos(phi) + i sin(phi).
template <class T, class F>
__device__ __forceinline__ void scf_deposit(const Model &m, T x, T y, T z, T w, F &&emit)
{
    const T r2 = fma(x, x, fma(y, y, z * z));
    const int j = scf_interval(m, r2);
    int k0;
    T g0 = T(1), g1 = T(0);
    if (j == 0) {
        k0 = 0;
    } else if (j == m.scf_n) {
        k0 = m.scf_n - 1;
    } else {
        const T r = d_sqrt(r2), ra = T(__ldg(m.scf_r + j - 1)), rb = T(__ldg(m.scf_r + j));
        k0 = j - 1;
        g0 = d_div(rb - r, rb - ra);
        g1 = d_div(r - ra, rb - ra);
    }
    T ct, st, cp, sp;
    shell_angles(x, y, z, ct, st, cp, sp);
    const int L = m.scf_lmax, nlm = m.scf_nlm;
    const int s0 = m.off_scf + k0 * nlm;
    T cm = T(1), sm = T(0), pmm = T(1);
    for (int mm = 0; mm <= L; ++mm) {
        T p0 = T(0), p1 = pmm;
        for (int l = mm; l <= L; ++l) {
            if (l > mm) {
                const T p2 = d_div(fma(ct * T(2 * l - 1), p1, -(T(l + mm - 1) * p0)), T(l - mm));
                p0 = p1;
                p1 = p2;
            }
            for (int v = 0; v < (mm > 0 ? 2 : 1); ++v) {
                const int idx = l * (l + 1) + (v == 0 ? mm : -mm);
                const T N = sizeof(T) == 8 ? T(m.scf_norm[idx]) : T(m.scf_norm_f[idx]);
                const T Y = N * p1 * (v == 0 ? cm : sm);
                const T wy = w * Y;
                emit(s0 + idx, g0 * wy);
                if (g1 != T(0)) emit(s0 + nlm + idx, g1 * wy);
            }
        }
        const T cn = fma(cm, cp, -(sm * sp));
        sm = fma(sm, cp, cm * sp);
        cm = cn;
        pmm *= T(2 * mm + 1) * st;
    }
}

// emit(observable, D, class) of the derivatives of the kinematic kernels of group G at
// aperture p with respect to ln Upsilon when the velocities scale as Upsilon^(1/2):
// D = 1/2 w v_los dK/dv_los; w v_los^2 for v_los^2 (class kClassVel), and for b_n, with
// K_n = c_n H_n(nu) e^(-nu^2/2), 1/2 w v_los c_n (2n H_(n-1) - nu H_n) e^(-nu^2/2)/sigma_p
// (class kClassDv).
constexpr int kClassDv = 3;
template <unsigned M, class T, class F>
__device__ __forceinline__ void group_dkernels(const GroupDesc &G, const Tables<T> &tb, int p, T vlos, T w, F &&emit)
{
    using P = GP<M>;
    const int base = G.obs_off + p;
    if (P::v2(G)) emit(base + G.k_v2 * G.n_ap, w * vlos * vlos, kClassVel);
    const int nmax = P::max_gh(G);
    if (nmax >= 0) {
        const T is = tb.isp[G.ap_off + p];
        const T nu = (vlos - tb.vp[G.ap_off + p]) * is;
        const T half = T(0.5) * w * vlos * is * kexp(tb, T(-0.5) * nu * nu);
        T hm1 = T(0), h = T(1);  // H_(n-1), H_n at n = 0
#pragma unroll
        for (int n = 0; n <= 6; ++n) {
            if (n <= nmax) {
                if (P::gh(G, n)) emit(base + G.k_gh[n] * G.n_ap, T(gh_c(n)) * half * fma(T(2 * n), hm1, -(nu * h)),
                                      kClassDv);
                const T hn1 = fma(T(2) * nu, h, -(T(2 * n) * hm1));
                hm1 = h;
                h = hn1;
            }
        }
    }
}

// ---------------------------------------------------------------- priors

// v_c^2 = R |a(R)| and the potential at radius R on the x axis (R >= 0), for the
// spherical potentials without the square root of R^2 and with one logarithm for the
// NFW halo (shared by its potential and its enclosed mass); the flattened log halo
// through accel and potential.
template <class T, bool SCF = true>
__host__ __device__ __forceinline__ void circ_terms(const Model &m, const Cst<T> &k, T R, T &vc2, T &phi)
{
    if (m.pot >= 2) {
        T ax, ay, az;
        accel<T, SCF>(m, k, R, T(0), T(0), ax, ay, az);
        vc2 = -R * ax;
        phi = potential<T, SCF>(m, k, R, T(0), T(0));
        return;
    }
    const T ra = R + k.a;
    vc2 = d_div(k.GM * R, ra * ra);
    phi = -d_div(k.GM, ra);
    if (m.pot == 1) {
        if (R > T(0)) {
            const T q = d_div(R, k.rs);
            T l1, mu;
            if constexpr (sizeof(T) == 4) {
                nfw_logs(q, l1, mu);
            } else {
                // mu(q) = ln(1+q) - q/(1+q); its series where the two terms cancel
                l1 = d_log1p(q);
                mu = q < T(1e-3) ? nfw_mu(q) : l1 - d_div(q, T(1) + q);
            }
            vc2 += d_div(k.GMs * mu, R);
            phi -= d_div(k.GMs * l1, R);
        } else {
            phi += k.hn_phi0;
        }
    }
}

// Energy of the circular orbit of radius R in the equatorial plane: phi(R) + v_c^2/2.
template <class T, bool SCF = true>
__host__ __device__ __forceinline__ T circ_energy(const Model &m, const Cst<T> &k, T R)
{
    T vc2, phi;
    circ_terms<T, SCF>(m, k, R, vc2, phi);
    return phi + T(0.5) * vc2;
}

// Lc(E): closed form for the Hernquist potential (E_c = -(u+1)/(2u^2) GM/a with
// u = R/a + 1), otherwise the host table of E_c(ln R) bracketed by binary search,
// interpolated, and refined by secant steps on E_c(R) = E.
template <class T, bool SCF = true>
__device__ T circular_L(const Model &m, const Cst<T> &k, const double *lcE, T E)
{
    if (m.pot < 2 && !(E < T(0))) return T(0);
    if (m.lc_closed) {
        const T e = E * k.e_scale;
        if (!(e > T(-1))) return T(0);
        const T u = d_div(T(-1) - d_sqrt(T(1) - T(8) * e), T(4) * e);
        const T R = k.a * (u - T(1));
        const T ra = R + k.a;
        return d_div(R * d_sqrt(k.GM * R), ra);
    }
    if (!(E > k.phi_min)) return T(0);
    const int n = m.lc_n;
    int lo = 0, hi = n - 1;
    T R;
    if (SCF && m.pot == 3) {
        // The self-consistent potential need not be lowest at the centre (its l > 0 terms can
        // lower it off the axis), and its thin shells put kinks in E_c(R) at the grid radii,
        // so E_c(R) = E may have no root below phi(0) and is not smooth: Lc(E) by plain
        // bisection, from [0, 1] doubled until it brackets the root (no circular orbit
        // below E_c(0) = phi(0)).
        if (!(E > circ_energy<T, SCF>(m, k, T(0)))) return T(0);
        T hi = T(1), lo = T(0);
        while (hi < T(1e15) && circ_energy<T, SCF>(m, k, hi) <= E) hi *= T(2);
        for (int it = 0; it < 400; ++it) {
            const T mid = T(0.5) * (lo + hi);
            if (!(mid > lo) || !(mid < hi)) break;
            if (circ_energy<T, SCF>(m, k, mid) <= E) lo = mid;
            else hi = mid;
        }
        R = T(0.5) * (lo + hi);
        T vc2, phi;
        circ_terms<T, SCF>(m, k, R, vc2, phi);
        return R * d_sqrt(vc2);
    }
    if (!(E > T(__ldg(lcE)))) {
        R = k.lc_r0;
    } else if (!(E < T(__ldg(lcE + n - 1)))) {
        R = k.lc_rmax;
    } else {
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (T(__ldg(lcE + mid)) <= E) lo = mid;
            else hi = mid;
        }
        if constexpr (sizeof(T) == 4) {
            // FP32: inverse cubic interpolation of ln R in E through the four table
            // points around the bracket (Lagrange), clamped to the bracket. Its error,
            // of order (table step)^4 ~ 4e-9 in ln R, is below FP32 resolution, so no
            // refinement by the force is needed.
            int j0 = lo - 1;
            j0 = j0 < 0 ? 0 : (j0 > n - 4 ? n - 4 : j0);
            T xe[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) xe[q] = T(__ldg(lcE + j0 + q));
            T lnr = T(0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                T li = T(1);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q != i) li *= d_div(E - xe[q], xe[i] - xe[q]);
                lnr += li * (k.lc_lnr0 + T(j0 + i) * k.lc_dlnr);
            }
            const T ylo = k.lc_lnr0 + T(lo) * k.lc_dlnr;
            R = d_exp(fminf(fmaxf(lnr, ylo), ylo + k.lc_dlnr));
        } else {
            const T e0 = T(__ldg(lcE + lo)), e1 = T(__ldg(lcE + hi));
            const T fr = d_div(E - e0, e1 - e0);
            R = d_exp(k.lc_lnr0 + (T(lo) + fr) * k.lc_dlnr);
            // secant refinement, starting from the table segment's slope
            const T Ra = d_exp(k.lc_lnr0 + T(lo) * k.lc_dlnr);
            const T Rb = d_exp(k.lc_lnr0 + T(hi) * k.lc_dlnr);
            T r0 = R, f0 = circ_energy<T, SCF>(m, k, r0) - E;
            T r1 = r0 - f0 * d_div(Rb - Ra, e1 - e0);
            for (int it = 0; it < 3; ++it) {
                const T f1 = circ_energy<T, SCF>(m, k, r1) - E;
                if (f1 == f0) break;
                const T r2 = r1 - f1 * d_div(r1 - r0, f1 - f0);
                r0 = r1;
                f0 = f1;
                r1 = r2;
            }
            R = r1;
        }
    }
    T vc2, phi;
    circ_terms<T, SCF>(m, k, R, vc2, phi);
    return R * d_sqrt(vc2);
}

// Cell k*nx + l of a particle: E bin from the chosen spacing (clamped), circularity
// bin from x = L/Lc(E) (x = Lz/Lc(E) on [-1, 1] for the signed variant, clamped).
template <class T, bool SCF = true>
__device__ __forceinline__ int prior_cell(const Model &m, const Cst<T> &k, const double *lcE, T x, T y, T z,
                                          T vx, T vy, T vz)
{
    const T E = fma(T(0.5), fma(vx, vx, fma(vy, vy, vz * vz)), potential<T, SCF>(m, k, x, y, z));
    const T Lz = fma(x, vy, -(y * vx));
    T L;
    if (m.signed_lz) {
        L = Lz;
    } else {
        const T Lx = fma(y, vz, -(z * vy)), Ly = fma(z, vx, -(x * vz));
        L = d_sqrt(fma(Lx, Lx, fma(Ly, Ly, Lz * Lz)));
    }
    const T Lc = circular_L<T, SCF>(m, k, lcE, E);
    T xc = (Lc > T(0)) ? d_div(L, Lc) : T(0);
    const T xmin = m.signed_lz ? T(-1) : T(0);
    xc = xc < xmin ? xmin : (xc > T(1) ? T(1) : xc);
    T f;
    if (m.e_spacing == 0) f = (E >= T(0)) ? T(1) : d_div(d_log(-E) - k.s_lo, k.s_den);
    else if (m.e_spacing == 1) f = d_div(d_exp(E) - k.s_lo, k.s_den);
    else f = d_div(E - k.s_lo, k.s_den);
    const T fk = d_floor(f * k.nE);
    const int kb = !(fk >= T(0)) ? 0 : (fk >= k.nE ? m.nE - 1 : int(fk));
    const T fl = d_floor(d_div(xc - xmin, T(1) - xmin) * k.nx);
    const int lb = !(fl >= T(0)) ? 0 : (fl >= k.nx ? m.nx - 1 : int(fl));
    return kb * m.nx + lb;
}

// ---------------------------------------------------------------- fixed point
//
// Global sums are int64 words: FP64 mode uses two per slot (integer part and the
// next 32 fraction bits of v*scale), mixed mode one (round(v*scale)). Integer
// sums are exact, so the result does not depend on the order of the additions.

// FP64: v*scale = hi + lo 2^-32 with hi = floor and lo in [0, 2^32), computed with
// integer operations on the IEEE fields (scale is a power of two): the 53-bit
// significand m and exponent give T = round(v*scale*2^32) = m 2^k, split into its
// high and low 32-bit parts. |v*scale| < 2^62 keeps k <= 42, so m 2^(k-32) < 2^63.
__device__ __forceinline__ void fx2(double v, double scale, long long &hi, long long &lo)
{
    const long long bits = __double_as_longlong(v);
    const int e = int((bits >> 52) & 0x7FF);
    if (e == 0) {  // zero (and subnormals, below any resolution used here)
        hi = 0;
        lo = 0;
        return;
    }
    const int se = int((__double_as_longlong(scale) >> 52) & 0x7FF) - 1023;
    const unsigned long long m = (static_cast<unsigned long long>(bits) & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int k = e - 1075 + se + 32;
    unsigned long long th, tl;
    if (k >= 32) {
        th = m << (k - 32);
        tl = 0;
    } else if (k >= 0) {
        th = m >> (32 - k);
        tl = (m << k) & 0xFFFFFFFFull;
    } else if (k > -63) {
        const unsigned long long r = (m + (1ull << (-k - 1))) >> (-k);
        th = r >> 32;
        tl = r & 0xFFFFFFFFull;
    } else {
        th = 0;
        tl = 0;
    }
    if (bits < 0) {
        hi = tl ? -static_cast<long long>(th) - 1 : -static_cast<long long>(th);
        lo = tl ? 4294967296ll - static_cast<long long>(tl) : 0;
    } else {
        hi = static_cast<long long>(th);
        lo = static_cast<long long>(tl);
    }
}

// Mixed mode: round(v*scale) (the scaling by a power of two is exact) in one 64-bit
// conversion, added to the block sums as three 32-bit limbs (see Acc<float>).
__device__ __forceinline__ long long limbs_value(long long hi, long long mid, long long lo)
{
    return hi * 4294967296ll + mid * 65536ll + lo;
}

// Block-shared sums. FP64 mode: the two int64 words of each slot, added with
// 64-bit shared atomics. Mixed mode: three int32 limbs per slot added with native
// 32-bit shared atomics; at most kMaxParticlesPerBlock particles per block keep the
// sums of mid and lo (each term in [0, 2^16)) below 2^31, and |sum of hi| < 2^31
// follows from the fixed-point range. The block flush recombines the limbs into the
// int64 word exactly.
constexpr long long kMaxParticlesPerBlock = 32768;

template <class T>
struct Acc;

template <>
struct Acc<double> {
    static __host__ __device__ size_t bytes(const Model &m) { return sizeof(long long) * size_t(m.hist_words); }
    // the fixed-point value of v * scale (two words)
    struct Fx {
        long long hi, lo;
    };
    __device__ static Fx fx(double v, double scale)
    {
        Fx r;
        fx2(v, scale, r.hi, r.lo);
        return r;
    }
    __device__ static void put(void *base, int slot, const Fx &q)
    {
        long long *h = static_cast<long long *>(base);
        atomicAdd(reinterpret_cast<unsigned long long *>(h + 2 * slot), static_cast<unsigned long long>(q.hi));
        if (q.lo) atomicAdd(reinterpret_cast<unsigned long long *>(h + 2 * slot + 1), static_cast<unsigned long long>(q.lo));
    }
    __device__ static void add(void *base, const Model &, int slot, double v, double scale)
    {
        if (is_zero(v)) return;
        put(base, slot, fx(v, scale));
    }
    __device__ static void count(void *base, const Model &m, int c)
    {
        atomicAdd(reinterpret_cast<unsigned long long *>(static_cast<long long *>(base) + m.off_count + c), 1ull);
    }
    // global word k of the block's sums
    __device__ static long long word(const void *base, const Model &, int k) { return static_cast<const long long *>(base)[k]; }
};

template <>
struct Acc<float> {
    static __host__ __device__ size_t bytes(const Model &m)
    {
        return sizeof(int) * (3 * size_t(m.nslots) + size_t(m.ncell)) + 8;
    }
    // round(v*scale) as L = hi 2^32 + mid 2^16 + lo with mid, lo in [0, 2^16) and hi signed:
    // the two's-complement fields of one 64-bit conversion. Per block the lo and mid sums
    // stay below 32768 * 65535 < 2^31, and the hi sum within the fixed-point range.
    // the fixed-point value of v * scale (one 64-bit integer)
    struct Fx {
        long long L;
    };
    __device__ static Fx fx(float v, float scale) { return Fx{__float2ll_rn(v * scale)}; }
    __device__ static void put(void *base, int slot, const Fx &q)
    {
        int *h = static_cast<int *>(base) + 3 * slot;
        // the hi limb is added even when 0: cheaper than the branch around it
        atomicAdd(h, static_cast<int>(q.L >> 32));
        atomicAdd(h + 1, static_cast<int>((q.L >> 16) & 0xFFFF));
        atomicAdd(h + 2, static_cast<int>(q.L & 0xFFFF));
    }
    // a zero adds zeros: cheaper than the branch around it
    __device__ static void add(void *base, const Model &, int slot, float v, float scale)
    {
        put(base, slot, fx(v, scale));
    }
    __device__ static void count(void *base, const Model &m, int c)
    {
        atomicAdd(static_cast<int *>(base) + 3 * m.nslots + c, 1);
    }
    __device__ static long long word(const void *base, const Model &m, int k)
    {
        const int *h = static_cast<const int *>(base);
        if (k >= m.off_count) return static_cast<long long>(h[3 * m.nslots + (k - m.off_count)]);
        const int *q = h + 3 * k;
        return limbs_value(q[0], q[1], q[2]);
    }
};

// Per-thread running total of the deposited weight, in the same fixed point.
template <class T>
struct Total;

template <>
struct Total<double> {
    long long hi = 0, lo = 0;
    __device__ void add(double v, double scale)
    {
        long long a, b;
        fx2(v, scale, a, b);
        hi += a;
        lo += b;
    }
    __device__ void add_fx(const Acc<double>::Fx &q)
    {
        hi += q.hi;
        lo += q.lo;
    }
    __device__ long long word(int q, double) const { return q == 0 ? hi : lo; }
};

// Mixed mode: round(w * scale) of every weight summed in a 64-bit register, so the total
// is the exact integer sum and does not depend on how the particles are spread over
// threads and blocks.
template <>
struct Total<float> {
    long long s = 0;
    __device__ void add(float v, float scale) { s += __float2ll_rn(v * scale); }
    __device__ void add_fx(const Acc<float>::Fx &q) { s += q.L; }
    __device__ long long word(int, float) const { return s; }
};

template <int WPS>
__device__ __forceinline__ double fx_read(const long long *h, int slot)
{
    if (WPS == 1) return double(__ldcg(h + slot));
    return double(__ldcg(h + 2 * slot)) + double(__ldcg(h + 2 * slot + 1)) * (1.0 / 4294967296.0);
}

// ---------------------------------------------------------------- force of change

// The data term sum_j K_j c_j at the particle's position, with the apertures from
// the cached code of the last deposit when there is one.
template <unsigned... Ms, class T>
__device__ __forceinline__ T foc_data(const Model &m, const Cst<T> &k, const Tables<T> &tb, const T *rec,
                                      unsigned code, const T *gexp, T x, T y, T z, T vy, T vz)
{
    T Y, vlos;
    project(k, y, z, vy, vz, Y, vlos);
    if (code != kApUncached) return data_term_cached<Ms...>(m, tb, rec, code, vlos, gexp);
    return data_term<Ms...>(m, tb, rec, x, y, z, x, Y, vlos);
}

// Weight after the force of change of eq. modFOC over one step, the kernel
// values taken at the particle's current position and the priors held fixed:
// F = mu dS/dw - sum_j K_j c_j, c_j = Delta_j/sigma_j (times 1/area for mass),
// dS/dw = -ln(w/what) (eq. S+) or -ln(w/what) - 1 (eq. entropy).
template <unsigned... Ms, class T>
__device__ __forceinline__ T foc_update(const Model &m, const Cst<T> &k, const Tables<T> &tb, const T *rec,
                                        unsigned code, const T *gexp, T iprior, T w, T x, T y, T z, T vy, T vz,
                                        unsigned &err)
{
    if (w == T(0)) return w;  // w = 0 is a fixed point
    const T data = foc_data<Ms...>(m, k, tb, rec, code, gexp, x, y, z, vy, vz);
    // A cell mean below the resolution of the fixed-point cell sums reads as 0
    // (iprior = 0); the particle's weight is then unresolved too and the entropy
    // term is dropped.
    T dS = iprior > T(0) ? -d_log(w * iprior) : T(0);
    if (m.mode == 0) dS -= T(1);
    const T h = k.dteps * fma(k.mu, dS, -data);
    T wn;
    if (m.update_rule == 0) wn = w * d_exp(h);
    else wn = w * (T(1) + h);
    if (!d_finite(wn)) err |= kErrNonFinite;
    else if (wn < T(0) || (m.update_rule == 1 && !(wn > T(0)))) err |= kErrNegWeight;
    return wn;
}

// The same update on u = ln w (FP64 mode): u + eps dt F for the exponential rule,
// u + ln(1 + eps dt F) for explicit Euler, with dS/dw = ln(what) - u.
template <unsigned... Ms, class T>
__device__ __forceinline__ T foc_update_log(const Model &m, const Cst<T> &k, const Tables<T> &tb, const T *rec,
                                            unsigned code, const T *gexp, T lprior, T u, T x, T y, T z, T vy, T vz,
                                            unsigned &err)
{
    if (is_neg_inf(u)) return u;  // w = 0 is a fixed point
    const T data = foc_data<Ms...>(m, k, tb, rec, code, gexp, x, y, z, vy, vz);
    // a prior that reads 0 (below the resolution of the cell sums) drops the entropy term
    T dS = !is_neg_inf(lprior) ? lprior - u : T(0);
    if (m.mode == 0) dS -= T(1);
    const T h = k.dteps * fma(k.mu, dS, -data);
    T un;
    if (m.update_rule == 0) {
        un = u + h;
    } else {
        if (!(h > T(-1))) {
            err |= (h != h) ? kErrNonFinite : kErrNegWeight;
            return u;
        }
        un = u + log1p(h);
    }
    // exp_tab overflows above 709 (NaN of either sign is flagged too)
    const long long ub = __double_as_longlong(un);
    if ((ub & 0x7fffffffffffffffll) > 0x7ff0000000000000ll || ub > 0x4086280000000000ll) err |= kErrNonFinite;
    return un;
}

// ---------------------------------------------------------------- shared-memory layout

template <class T>
struct Smem {
    void *h;               // fixed-point sums of the block (layout of Acc<T>)
    T *c, *iprior, *esq, *vp, *isp;  // c: the force-of-change records; iprior: 1/prior, or ln prior (FP64)
    double *e2;            // 2^(j/32) for exp_tab
    unsigned short *lut;
};

// Block sums of the global-deposit kernel's aperture window: one slot per kind and
// window aperture, laid out as Acc<T> slots.
template <class T>
__host__ __device__ inline size_t window_bytes(const Model &m)
{
    const size_t slots = m.win_n > 0 ? size_t(m.g[m.win_group].n_kinds) * m.win_n : 0;
    return slots * (sizeof(T) == 8 ? 2 * sizeof(long long) : 3 * sizeof(int));
}

// hist: 0 no block sums, 1 all (Acc<T>), 2 the aperture window of the global deposit
template <class T>
__host__ __device__ inline size_t acc_bytes_padded(const Model &m, int hist = 1)
{
    const size_t b = hist == 2 ? window_bytes<T>(m) : Acc<T>::bytes(m);
    return (b + 15) / 16 * 16;
}

// Dynamic shared memory of a kernel holding the block sums (with_hist) and the
// force-of-change records (with_rec) in shared memory; the global-deposit step
// kernel keeps both in global memory.
template <class T>
__host__ __device__ inline size_t smem_bytes(const Model &m, int with_hist, int with_rec = 1, int with_vp = 1)
{
    size_t b = with_hist ? acc_bytes_padded<T>(m, with_hist) : 0;
    b += sizeof(T) * size_t((with_rec ? m.n_ap_total * m.rec_len : 0) + m.ncell + m.n_edges_total +
                            (with_vp ? 2 * m.n_ap_total : 0));
    b = (b + 7) / 8 * 8 + sizeof(double) * 32;
    b += sizeof(unsigned short) * size_t(m.n_lut) + 16;
    return b;
}

template <class T>
__device__ __forceinline__ Smem<T> carve(const Model &m, unsigned char *base, int with_hist, int with_rec = 1,
                                         int with_vp = 1)
{
    Smem<T> s;
    s.h = base;
    T *t = reinterpret_cast<T *>(base + (with_hist ? acc_bytes_padded<T>(m, with_hist) : 0));
    s.c = t;
    s.iprior = s.c + (with_rec ? m.n_ap_total * m.rec_len : 0);
    s.esq = s.iprior + m.ncell;
    s.vp = s.esq + m.n_edges_total;
    s.isp = s.vp + (with_vp ? m.n_ap_total : 0);
    unsigned char *e = reinterpret_cast<unsigned char *>(s.isp + (with_vp ? m.n_ap_total : 0));
    s.e2 = reinterpret_cast<double *>(base + (e - base + 7) / 8 * 8);
    s.lut = reinterpret_cast<unsigned short *>(s.e2 + 32);
    return s;
}

template <class T>
__device__ __forceinline__ void load_tables(const Model &m, const Buffers &b, const Smem<T> &s, int with_vp = 1)
{
    for (int k = threadIdx.x; k < m.n_edges_total; k += blockDim.x) s.esq[k] = T(b.edges[k] * b.edges[k]);
    for (int k = threadIdx.x; with_vp && k < m.n_ap_total; k += blockDim.x) {
        s.vp[k] = T(b.Vp[k]);
        s.isp[k] = T(b.isp[k]);
    }
    for (int k = threadIdx.x; k < m.n_lut; k += blockDim.x) s.lut[k] = b.lut[k];
    for (int k = threadIdx.x; k < 32; k += blockDim.x) s.e2[k] = kExp2j[k];
}

// ---------------------------------------------------------------- force-of-change records

// Folds the coefficients c_j of every aperture into its record (see data_term): with
// v_los = V + s nu (s = sigma_p), mass contributes c to q0, v_los^2 contributes
// c (V^2, 2 V s, s^2) and v_los contributes c (V, s) to (q0, q1, q2); b_n contributes
// c c_n H_n(nu) to the Hermite part, with the monomial coefficients of H_n from the
// recurrence H_{n+1} = 2 nu H_n - 2 n H_{n-1}. Called by every thread of one block.
// Coefficient of nu^q in the physicists' H_n, set on the host from the recurrence
// H_{n+1} = 2 nu H_n - 2 n H_{n-1} (see herm_table).
static __constant__ double kHerm[7][7];  // one copy per translation unit

inline void herm_table(double h[7][7])
{
    for (int n = 0; n < 7; ++n)
        for (int q = 0; q < 7; ++q) h[n][q] = 0.0;
    h[0][0] = 1.0;
    h[1][1] = 2.0;
    for (int n = 1; n < 6; ++n)
        for (int q = 0; q < 7; ++q) h[n + 1][q] = (q > 0 ? 2.0 * h[n][q - 1] : 0.0) - 2.0 * n * h[n - 1][q];
}

// Sets this translation unit's constant tables (kHerm, kExp2j) on the current device.
static inline cudaError_t upload_constants()
{
    double h[7][7];
    herm_table(h);
    cudaError_t e = cudaMemcpyToSymbol(kHerm, h, sizeof h);
    if (e != cudaSuccess) return e;
    double t[32];
    exp2_table(t);
    return cudaMemcpyToSymbol(kExp2j, t, sizeof t);
}

static __device__ void build_records(const Model &m, const Buffers &b)
{
    for (int g = 0; g < m.n_groups; ++g) {
        const GroupDesc &G = m.g[g];
        for (int p = threadIdx.x; p < G.n_ap; p += blockDim.x) {
            const int a = G.ap_off + p;
            double *r = b.rec + a * m.rec_len;
            if (G.geometry == 2) {  // shells: c_j of each a_lm
                float *rf = b.recf + a * m.rec_len;
                for (int q = 0; q < m.rec_len; ++q) {
                    r[q] = q < G.n_kinds ? b.c[G.obs_off + q * G.n_ap + p] : 0.0;
                    rf[q] = float(r[q]);
                }
                continue;
            }
            const bool gh = G.max_gh >= 0;
            const double V = gh ? b.Vp[a] : 0.0, is = gh ? b.isp[a] : 1.0, s = 1.0 / is;
            const int base = G.obs_off + p;
            double q0 = 0.0, q1 = 0.0, q2 = 0.0;
            if (G.k_mass >= 0) q0 += b.c[base + G.k_mass * G.n_ap];
            if (G.k_v2 >= 0) {
                const double c = b.c[base + G.k_v2 * G.n_ap];
                q0 += c * V * V;
                q1 += c * 2.0 * V * s;
                q2 += c * s * s;
            }
            if (G.k_v1 >= 0) {
                const double c = b.c[base + G.k_v1 * G.n_ap];
                q0 += c * V;
                q1 += c * s;
            }
            r[0] = V;
            r[1] = is;
            r[2] = q0;
            r[3] = q1;
            r[4] = q2;
            double pc[7] = {0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int n = 0; n < 7; ++n) {
                if (n <= G.max_gh && G.k_gh[n] >= 0) {
                    const double c = b.c[base + G.k_gh[n] * G.n_ap] * gh_c(n);
#pragma unroll
                    for (int q = 0; q <= n; ++q) pc[q] += c * kHerm[n][q];
                }
            }
#pragma unroll
            for (int q = 0; q < 7; ++q)
                if (5 + q < m.rec_len) r[5 + q] = pc[q];
            float *rf = b.recf + a * m.rec_len;
            for (int q = 0; q < m.rec_len; ++q) rf[q] = float(r[q]);
        }
    }
}

// ---------------------------------------------------------------- finalize (last block)
//
// Run by the last block of the step kernel once every block has added its sums:
// converts the fixed-point sums, renormalises, smooths (eq. myts), forms Delta_j,
// chi^2 (eqs. delta, chi) and the force-of-change coefficients, the prior means on
// Sums red[0 .. blockDim) into red[0] for any block size: the part above the largest
// power of two is folded in first. Called after red is written and synchronised.
__device__ __forceinline__ void block_fold(double *red)
{
    int p2 = 1;
    while (2 * p2 <= int(blockDim.x)) p2 *= 2;
    if (int(threadIdx.x) >= p2) red[threadIdx.x - p2] += red[threadIdx.x];
    __syncthreads();
    for (int s = p2 / 2; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
}

// The self-consistent potential at an update (Sec. 6), in the finalize: the mass-to-light
// ratio follows the chi^2 gradient, d ln Upsilon/dt = -eps_ups sum_j Delta_j/sigma_j D_j over
// the update_every steps to the next update (not at the load); then the interval tables
// TA, TB of scf_field from the new coefficients a_lm,k and Upsilon. red: blockDim doubles.
template <int WPS>
__device__ void scf_finalize(const Model &m, const Buffers &b, double s_ren, int init, double *red)
{
    Scalars &sc = *b.sc;
    if (!init && m.n_dups > 0) {
        double part = 0.0;
        for (int j = threadIdx.x; j < m.J; j += blockDim.x) {
            const int kind = b.obs_kind[j];
            const double sj = kind == kKindV2 ? m.fx_v2 : ((kind >= kKindGH0 && kind <= kKindGH0 + 6) ? m.fx_dv : 0.0);
            if (sj == 0.0) continue;
            const double D = fx_read<WPS>(b.hist, m.off_dups + j) / sj * s_ren;
            part += b.delta[j] / b.sig[j] * D;
        }
        red[threadIdx.x] = part;
        __syncthreads();
        block_fold(red);
        if (threadIdx.x == 0) sc.ups *= exp(-m.eps_ups * double(m.update_every) * m.dt * red[0]);
        __syncthreads();
    }
    const double ups = sc.ups;
    const int n = m.scf_n, nlm = m.scf_nlm;
    for (int idx = threadIdx.x; idx < nlm; idx += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= idx) ++l;
        const double C = -4.0 * 3.14159265358979323846 * m.G * ups / double(2 * l + 1);
        double A = 0.0;  // sum over the shells inside
        for (int j = 0; j <= n; ++j) {
            m.scf_tab[(size_t(j) * nlm + idx) * 2] = C * A;
            if (j < n) {
                const double a = fx_read<WPS>(b.hist, m.off_scf + j * nlm + idx) / m.fx_gh * s_ren;
                m.scf_coef[size_t(j) * nlm + idx] = a;
                A += a * pow(m.scf_r[j], l);
            }
        }
        double B = 0.0;  // sum over the shells outside
        for (int j = n; j >= 0; --j) {
            if (j < n) {
                const double a = fx_read<WPS>(b.hist, m.off_scf + j * nlm + idx) / m.fx_gh * s_ren;
                B += a * pow(m.scf_r[j], -(l + 1));
            }
            m.scf_tab[(size_t(j) * nlm + idx) * 2 + 1] = C * B;
        }
        for (int j = 0; j <= n; ++j) {
            const size_t q = (size_t(j) * nlm + idx) * 2;
            m.scf_tabf[q] = float(m.scf_tab[q]);
            m.scf_tabf[q + 1] = float(m.scf_tab[q + 1]);
        }
    }
    __syncthreads();
}

// update steps, and clears the sums for the next step. red: blockDim doubles.
// Priors of the grid-less variant (Sec. 7): the mean weight of the particles in the window of
// cells |k' - k| <= pwin_E, |l' - l| <= pwin_x around each cell (k, l), cut at the grid's
// edges. The window sums come from cumulative sums of the cells' integer words, first along
// x (into pwin), then, after the row windows are written back over the cell words, along E,
// so they equal the sums of the particles' own words in any order. q = 0 is the particle
// count, q = 1..WPS the words of the weight sum; all unsigned, wrapping like the deposits.
template <int WPS>
__device__ void window_priors(const Model &m, const Buffers &b, double s_ren)
{
    constexpr int NQ = WPS + 1;
    const int nE = m.nE, nx = m.nx, nc = m.ncell, hE = m.pwin_E, hx = m.pwin_x;
    unsigned long long *H = reinterpret_cast<unsigned long long *>(b.hist);
    unsigned long long *cum = b.pwin;
    auto at = [&](int q, int c) -> unsigned long long * {
        return q == 0 ? H + m.off_count + c : H + WPS * (m.J + 1 + c) + (q - 1);
    };
    for (int r = threadIdx.x; r < nE * NQ; r += blockDim.x) {  // cumulative sums along x
        const int k = r / NQ, q = r % NQ;
        unsigned long long acc = 0;
        for (int l = 0; l < nx; ++l) {
            const unsigned long long v = __ldcg(at(q, k * nx + l));
            if (q == 0) b.prior_count[k * nx + l] = (long long)v;
            acc += v;
            cum[size_t(q) * nc + k * nx + l] = acc;
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nc * NQ; r += blockDim.x) {  // row windows over the cell words
        const int q = r / nc, c = r % nc, k = c / nx, l = c % nx;
        const unsigned long long *row = cum + size_t(q) * nc + k * nx;
        *at(q, c) = __ldcg(row + min(l + hx, nx - 1)) - (l - hx - 1 >= 0 ? __ldcg(row + l - hx - 1) : 0ull);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nx * NQ; r += blockDim.x) {  // cumulative sums along E
        const int l = r / NQ, q = r % NQ;
        unsigned long long acc = 0;
        for (int k = 0; k < nE; ++k) {
            acc += __ldcg(at(q, k * nx + l));
            cum[size_t(q) * nc + k * nx + l] = acc;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        const int k = c / nx, l = c % nx, hi = min(k + hE, nE - 1), lo = k - hE - 1;
        unsigned long long box[NQ];
        for (int q = 0; q < NQ; ++q) {
            const unsigned long long *col = cum + size_t(q) * nc + l;
            box[q] = __ldcg(col + size_t(hi) * nx) - (lo >= 0 ? __ldcg(col + size_t(lo) * nx) : 0ull);
        }
        const long long cnt = (long long)box[0];
        double sum = double((long long)box[1]);
        if (WPS == 2) sum += double((long long)box[2]) * (1.0 / 4294967296.0);
        sum = sum / m.fx_w * s_ren;
        const double pr = cnt > 0 ? sum / double(cnt) : 0.0;
        b.prior[c] = pr;
        b.iprior[c] = pr > 0.0 ? 1.0 / pr : 0.0;
        b.lprior[c] = pr > 0.0 ? log(pr) : -HUGE_VAL;
    }
}

template <int WPS>
__device__ void finalize_block(const Model &m, const Buffers &b, long long n, int init, int prior_step,
                               double *red, int scf_step = 0)
{
    // other blocks updated the sums and scalars with atomics: read them from L2
    Scalars &sc = *b.sc;
    const long long t = init ? 0 : __ldcg(&sc.t) + 1;
    const double U = fx_read<WPS>(b.hist, m.J) / m.fx_w;
    double s_ren = 1.0;
    if (init) {
        if (threadIdx.x == 0) {
            sc.W0 = U;
            sc.what_flat = n > 0 ? U / double(n) : 0.0;
            sc.lwhat_flat = sc.what_flat > 0.0 ? log(sc.what_flat) : -HUGE_VAL;
        }
    } else if (m.renormalize && U > 0.0) {
        s_ren = __ldcg(&sc.W0) / U;
    }
    double part = 0.0;
    for (int j = threadIdx.x; j < m.J; j += blockDim.x) {
        const double raw = fx_read<WPS>(b.hist, j) * b.obs_iscale[j] * s_ren * b.obs_post[j];
        const double yt = init ? raw : b.ytil[j] + m.alpha * (raw - b.ytil[j]);
        const double d = (yt - b.Y[j]) / b.sig[j];
        b.yraw[j] = raw;
        b.ytil[j] = yt;
        b.delta[j] = d;
        b.c[j] = d / b.sig[j] * b.obs_post[j];
        part += d * d;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    build_records(m, b);
    block_fold(red);
    const double chi2 = red[0];
    __syncthreads();
    if (scf_step) scf_finalize<WPS>(m, b, s_ren, init, red);
    if (prior_step && (m.pwin_E > 0 || m.pwin_x > 0)) {
        window_priors<WPS>(m, b, s_ren);
    } else if (prior_step) {
        for (int c = threadIdx.x; c < m.ncell; c += blockDim.x) {
            const long long cnt = __ldcg(b.hist + m.off_count + c);
            const double sum = fx_read<WPS>(b.hist, m.J + 1 + c) / m.fx_w * s_ren;
            const double pr = cnt > 0 ? sum / double(cnt) : 0.0;  // mean weight of the cell
            b.prior_count[c] = cnt;
            if (m.smooth) {  // the smoothing kernels turn the raw means into the priors
                b.prior_raw[c] = pr;
                continue;
            }
            b.prior[c] = pr;
            b.iprior[c] = pr > 0.0 ? 1.0 / pr : 0.0;
            b.lprior[c] = pr > 0.0 ? log(pr) : -HUGE_VAL;
        }
    }
    __syncthreads();
    const int words = (prior_step || scf_step) ? m.hist_words : m.off_grid;
    for (int k = threadIdx.x; k < words; k += blockDim.x) b.hist[k] = 0;
    if (threadIdx.x == 0) {
        // the integer sums wrap beyond their range: the floating-point check sum catches it
        if (!(__ldcg(&sc.Wcheck) <= 0.5 * __ldcg(&sc.Wrange))) atomicOr(&sc.err, kErrOverflow);
        sc.Wcheck = 0.0;
        sc.Wsum = U;
        sc.chi2 = chi2;
        if (!init) sc.t = t;
        sc.wscale = s_ren;
        sc.lwscale = log(s_ren);
        sc.pending = init ? 0 : (t > m.n_relax ? 1 : 0);
        sc.blocks_done = 0;
        if (prior_step && m.smooth) sc.smooth_pending = 1;
    }
}

// ---------------------------------------------------------------- step kernel
//
// One M2M step over all particles, one read and one write of the particle state:
// (a) the previous step's force of change at the current position, (b) the
// kick-drift-kick push, (c) the deposit of w K_j into block-shared fixed-point
// sums, (d) on prior-update steps the (E, x) cell of every particle with per-cell
// weight sums and counts. Blocks add their sums to the global sums with integer
// atomics (exact, so order-independent); the last block to finish runs the
// finalize. Nothing waits on another block.
//
// GA (global deposit): for observable sets whose block sums or force-of-change
// records do not fit in shared memory (e.g. 64 x 64 pixel maps of five moments),
// every deposit goes straight to the global int64 sums with 64-bit atomics and the
// records are read from global memory (L1/L2 resident). The sums are the same
// integers in either mode, so both give bit-identical results.
template <class T>
__device__ __forceinline__ const T *global_records(const Buffers &b);
template <>
__device__ __forceinline__ const double *global_records<double>(const Buffers &b) { return b.rec; }
template <>
__device__ __forceinline__ const float *global_records<float>(const Buffers &b) { return b.recf; }

// V_p and 1/sigma_p per aperture in global memory (the global-deposit kernel keeps its
// shared memory for the aperture window)
template <class T>
__device__ __forceinline__ const T *global_vp(const Buffers &b);
template <>
__device__ __forceinline__ const double *global_vp<double>(const Buffers &b) { return b.Vp; }
template <>
__device__ __forceinline__ const float *global_vp<float>(const Buffers &b) { return b.Vpf; }
template <class T>
__device__ __forceinline__ const T *global_isp(const Buffers &b);
template <>
__device__ __forceinline__ const double *global_isp<double>(const Buffers &b) { return b.isp; }
template <>
__device__ __forceinline__ const float *global_isp<float>(const Buffers &b) { return b.ispf; }

// One deposit into the global sums (global-deposit mode): the fixed-point words of
// the block-shared path, added directly.
// Adds v to a 64-bit integer sum in global memory, without reading the result back.
__device__ __forceinline__ void red_add(long long *p, long long v)
{
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void global_add(long long *hist, int slot, double v, double scale)
{
    if (is_zero(v)) return;
    long long hi, lo;
    fx2(v, scale, hi, lo);
    red_add(hist + 2 * slot, hi);
    if (lo) red_add(hist + 2 * slot + 1, lo);
}
__device__ __forceinline__ void global_add(long long *hist, int slot, float v, float scale)
{
    if (v == 0.f) return;
    red_add(hist + slot, __float2ll_rn(v * scale));
}

// Per-step flags of one fit, read from its scalars at the start of the step.
template <class T>
struct StepFlags {
    int pending, prior_step, scf_step;
    T wscale, lwscale, iwhat_flat;
};

template <class T>
__device__ __forceinline__ StepFlags<T> step_flags(const Model &m, const Scalars &sc, int init)
{
    StepFlags<T> f;
    const long long t = sc.t + 1;
    f.pending = init ? 0 : sc.pending;
    f.prior_step = !init && m.mode == 1 && ((t - 1) % m.update_every) == 0;
    // the self-consistent potential is rebuilt at the load and on the prior schedule
    f.scf_step = m.pot == 3 && (init || ((t - 1) % m.update_every) == 0);
    f.wscale = init ? T(1) : T(sc.wscale);
    f.lwscale = init ? T(0) : T(sc.lwscale);
    f.iwhat_flat = kLogWeights<T> ? T(sc.lwhat_flat) : (sc.what_flat > 0.0 ? T(1.0 / sc.what_flat) : T(0));
    return f;
}

// Zeroes the block sums (block-shared deposit only).
template <class T, bool GA>
__device__ __forceinline__ void block_zero(const Model &m, const Smem<T> &S)
{
    int *z = static_cast<int *>(S.h);
    const int nw = int((GA ? window_bytes<T>(m) : Acc<T>::bytes(m)) / sizeof(int));
    for (int q = threadIdx.x; q < nw; q += blockDim.x) z[q] = 0;
}

// Copies a fit's records, priors and aperture tables into shared memory.
template <class T, bool GA>
__device__ __forceinline__ void block_tables(const Model &m, const Buffers &b, const Smem<T> &S, int pending)
{
    if (pending) {
        if (!GA)
            for (int q = threadIdx.x; q < m.n_ap_total * m.rec_len; q += blockDim.x) S.c[q] = global_records<T>(b)[q];
        if (m.mode == 1) {
            const double *pr = kLogWeights<T> ? b.lprior : b.iprior;
            for (int q = threadIdx.x; q < m.ncell; q += blockDim.x) S.iprior[q] = T(pr[q]);
        }
    }
    load_tables(m, b, S, GA ? 0 : 1);
}

// The per-particle part of one step for particles i0, i0 + stride, ... below i1:
// the pending force of change, the push, the deposit, the prior binning, and the
// write-back of the state.
template <class T, bool GA, unsigned M0, unsigned M1, unsigned M2, unsigned M3>
__device__ __forceinline__ void step_particles(const Model &m, const Model &mh, const Cst<T> &k, const State<T> &P,
                                               const Buffers &b,
                                               const Smem<T> &S, const StepFlags<T> &f, int push, long long i0,
                                               long long i1, long long stride, unsigned &err, Total<T> &wtot, T &wdep)
{
    // mh: the fields of the per-particle path (observable layout, regularisation and update
    // modes, potential kind). It is the fit's own Model, or in the batched kernel one Model
    // in the parameter space that every fit of the batch equals in those fields. m: the
    // fit's own Model, for the prior binning and the self-consistent potential.
    // the self-consistent potential runs in the generic kernel only (the host picks it)
    constexpr bool kScf = M0 == kDyn;
    const Tables<T> tb{S.esq, S.lut, GA ? global_vp<T>(b) : S.vp, GA ? global_isp<T>(b) : S.isp, S.e2};
    const T *rec = GA ? global_records<T>(b) : S.c;
    auto deposit = [&](int slot, T v, T scale) {
        if constexpr (GA) global_add(b.hist, slot, v, scale);
        else Acc<T>::add(S.h, mh, slot, v, scale);
    };
    // the next particle's state is loaded while the current one is processed
    const bool need_cell = f.pending && mh.mode == 1;
    const bool cache = mh.ap_cache != 0;
    const bool need_ap = cache && f.pending;
    const bool gxc = sizeof(T) == 8 && P.gx != nullptr;  // FP64, aperture cache, a Gauss-Hermite group
    const bool need_fa = keeps_accel<T>(mh) && push;
    T nx = T(0), ny = T(0), nz = T(0), nvx = T(0), nvy = T(0), nvz = T(0), nw = T(0), ngx = T(0), nfa = T(0);
    int ncell = 0;
    unsigned nap = kApUncached;
    auto fetch = [&](long long j) {
        nx = P.x[j]; ny = P.y[j]; nz = P.z[j];
        nvx = P.vx[j]; nvy = P.vy[j]; nvz = P.vz[j];
        nw = P.w[j];
        if (need_fa) nfa = P.fa[j];
        if (need_cell) ncell = P.cell[j];
        if (need_ap) nap = P.ap[j];
        if (need_ap && gxc) ngx = P.gx[j];
    };
    if (i0 < i1) fetch(i0);
    for (long long i = i0; i < i1; i += stride) {
        T x = nx, y = ny, z = nz;
        T vx = nvx, vy = nvy, vz = nvz;
        const T wst = nw;
        const int cell = ncell;
        const unsigned code = nap;
        const T gin = ngx;
        const T fa_in = nfa;
        const T *gp = gxc ? &gin : static_cast<const T *>(nullptr);
        if (i + stride < i1) fetch(i + stride);
        T w, u;
        if constexpr (kLogWeights<T>) {
            u = wst + f.lwscale;
            if (f.pending) {
                const T lp = mh.mode == 1 ? S.iprior[cell] : f.iwhat_flat;
                u = foc_update_log<M0, M1, M2, M3>(mh, k, tb, rec, code, gp, lp, u, x, y, z, vy, vz, err);
            }
            w = kexp(tb, u);
        } else {
            w = wst * f.wscale;
            if (f.pending) {
                const T pr = mh.mode == 1 ? S.iprior[cell] : f.iwhat_flat;
                w = foc_update<M0, M1, M2, M3>(mh, k, tb, rec, code, gp, pr, w, x, y, z, vy, vz, err);
            }
            u = w;
        }
        if (keeps_accel<T>(mh)) {
            T fa;
            if (push) {
                fa = fa_in;
                leapfrog_from(mh, k, x, y, z, vx, vy, vz, fa);
            } else {
                fa = accel_factor(mh, k, x, y, z);
            }
            P.fa[i] = fa;
        } else {
            if (push) leapfrog<T, kScf>(mh, k, x, y, z, vx, vy, vz);
        }
        if (!is_zero(w)) {
            T Y, vlos;
            project(k, y, z, vy, vz, Y, vlos);
            // the fixed-point weight, shared by the total and the surface-mass deposits
            const auto wfx = Acc<T>::fx(w, k.fx_w);
            unsigned code_out = 0;
            T gout = T(0);
            each_group<0, M0, M1, M2, M3>(mh, [&](auto Pl, int g) {
                constexpr unsigned M = decltype(Pl)::mask;
                const GroupDesc &G = mh.g[g];
                if (GP<M>::shells(G)) {  // never cached; never in the global-deposit kernel
                    shell_kernels(G, tb, x, y, z, w, [&](int j, T v, int, int) {
                        if constexpr (GA) global_add(b.hist, j, v, k.fx_gh);
                        else Acc<T>::add(S.h, mh, j, v, k.fx_gh);
                    });
                    return;
                }
                const int p = aperture<M>(G, tb.esq, tb.lut, x, Y);
                if (cache) code_out = ap_encode(mh, code_out, g, p);
                if (p >= 0) {
                    // the v^2 sums' range assumes v^2 <= v2max (energy bound with headroom)
                    if (GP<M>::v2(G) && gt_nonneg(vlos * vlos, k.v2max)) err |= kErrOverflow;
                    group_kernels<M>(
                        G, tb, p, vlos, w,
                        [&](int j, T v, int cls, int kk) {
                            const T scale = cls == kClassMass ? k.fx_w : (cls == kClassVel ? k.fx_v2 : k.fx_gh);
                            if constexpr (GA) {
                                const unsigned a = unsigned(p - mh.win_lo);
                                if (g == mh.win_group && a < unsigned(mh.win_n))
                                    Acc<T>::add(S.h, mh, kk * mh.win_n + int(a), v, scale);
                                else
                                    global_add(b.hist, j, v, scale);
                            } else if (cls == kClassMass) {  // v is w (the kernel is 1)
                                Acc<T>::put(S.h, j, wfx);
                            } else {
                                Acc<T>::add(S.h, mh, j, v, scale);
                            }
                        },
                        gxc && g == mh.gx_group ? &gout : nullptr);
                    if constexpr (kScf) {
                        if (f.scf_step && m.n_dups > 0)  // derivatives for the mass-to-light ratio (Sec. 6)
                            group_dkernels<M>(G, tb, p, vlos, w, [&](int j, T v, int cls) {
                                deposit(m.off_dups + j, v, cls == kClassVel ? k.fx_v2 : k.fx_dv);
                            });
                    }
                }
            });
            if constexpr (kScf) {
                if (f.scf_step)  // the particle's luminosity in the expansion of the stellar potential
                    scf_deposit(m, x, y, z, w, [&](int slot, T v) { deposit(slot, v, k.fx_gh); });
            }
            if (cache) P.ap[i] = static_cast<uint16_t>(code_out);
            if (gxc) P.gx[i] = gout;
            wtot.add_fx(wfx);
            wdep += w;
        }
        if (f.prior_step) {
            const int c = prior_cell<T, kScf>(m, k, b.lcE, x, y, z, vx, vy, vz);
            deposit(m.J + 1 + c, w, k.fx_w);
            if constexpr (GA) red_add(b.hist + m.off_count + c, 1);
            else Acc<T>::count(S.h, m, c);
            P.cell[i] = static_cast<uint16_t>(c);
        }
        P.x[i] = x; P.y[i] = y; P.z[i] = z;
        P.vx[i] = vx; P.vy[i] = vy; P.vz[i] = vz;
        P.w[i] = u;
    }
}

// Adds the block's sums, its total weight and its error bits to the fit's global
// sums and scalars. Called by every thread of the block.
template <class T, int WPS, bool GA>
__device__ __forceinline__ void block_flush(const Model &m, const Cst<T> &k, const Buffers &b, const Smem<T> &S,
                                            int prior_step, unsigned err, const Total<T> &wtot, T wdep,
                                            int scf_step = 0)
{
    if (err) atomicOr(&b.sc->err, err);
    // the total weight went into registers: one global atomic per warp and word
#pragma unroll
    for (int q = 0; q < WPS; ++q) {
        long long v = wtot.word(q, k.fx_w);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0)
            red_add(b.hist + WPS * m.J + q, v);
    }
    for (int o = 16; o > 0; o >>= 1) wdep += __shfl_xor_sync(0xffffffffu, wdep, o);
    if ((threadIdx.x & 31) == 0 && wdep != T(0)) atomicAdd(&b.sc->Wcheck, double(wdep));
    __syncthreads();
    if (GA) {  // the aperture window's sums go to their observables' global words
        const GroupDesc &G = m.g[m.win_group < 0 ? 0 : m.win_group];
        const int slots = m.win_n > 0 ? G.n_kinds * m.win_n : 0;
        for (int q = threadIdx.x; q < WPS * slots; q += blockDim.x) {
            const int slot = q / WPS, wd = q - slot * WPS;
            const int kk = slot / m.win_n, a = slot - kk * m.win_n;
            const long long v = Acc<T>::word(S.h, m, q);
            const int j = G.obs_off + kk * G.n_ap + m.win_lo + a;
            if (v != 0) red_add(b.hist + WPS * j + wd, v);
        }
    }
    const int words = GA ? 0 : ((prior_step || scf_step) ? m.hist_words : m.off_grid);
    for (int q = threadIdx.x; q < words; q += blockDim.x) {
        if (q >= WPS * m.J && q < WPS * (m.J + 1)) continue;  // the total is already global
        const long long v = Acc<T>::word(S.h, m, q);
        if (v != 0) red_add(b.hist + q, v);
    }
    __threadfence();
    __syncthreads();
}

// Threads per block the step kernel is compiled for. The mixed-precision global-deposit
// kernel runs up to 1024 threads in one block per SM, so that one aperture window takes
// the whole shared memory of the SM.
template <class T, bool GA>
constexpr int kStepMaxThreads = (GA && sizeof(T) == 4) ? 1024 : 256;

template <class T, int WPS, int MINB, bool GA, unsigned M0, unsigned M1, unsigned M2, unsigned M3>
__global__ void __launch_bounds__(kStepMaxThreads<T, GA>, (GA && sizeof(T) == 4) ? 1 : MINB) k_step(const Model m, const Cst<T> k, const State<T> P,
                                                    const Buffers b, int push, int init)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Smem<T> S = carve<T>(m, smem, GA ? 2 : 1, GA ? 0 : 1, GA ? 0 : 1);
    __shared__ bool am_last;

    const StepFlags<T> f = step_flags<T>(m, *b.sc, init);
    block_zero<T, GA>(m, S);
    block_tables<T, GA>(m, b, S, f.pending);
    __syncthreads();

    unsigned err = 0;
    Total<T> wtot;
    T wdep = T(0);  // floating-point twin of wtot, for the fixed-point range check
    step_particles<T, GA, M0, M1, M2, M3>(m, m, k, P, b, S, f, push, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                                          P.n, (long long)gridDim.x * blockDim.x, err, wtot, wdep);
    block_flush<T, WPS, GA>(m, k, b, S, f.prior_step, err, wtot, wdep, f.scf_step);
    if (m.shard) return;  // the sums of all shards are added by the caller; k_finalize follows
    // last block to finish runs the finalize
    if (threadIdx.x == 0) am_last = atomicAdd(&b.sc->blocks_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (am_last) {
        __threadfence();
        finalize_block<WPS>(m, b, P.n, init, f.prior_step, reinterpret_cast<double *>(smem), f.scf_step);
    }
}

// ---------------------------------------------------------------- shards of one fit
//
// A fit whose particles are split over several processes (contiguous ranges, one per
// shard) runs the per-particle pass of a step on every shard (k_step with Model::shard),
// then the caller adds the shards' integer sums word by word (an all-reduce), and every
// shard runs the same finalize on the same integers (k_finalize): the result is
// bit-identical to the unsplit fit. The exchanged words are the fixed-point sums of
// Model::hist_words, then one range word (the deposited weight in units of
// Wrange 2^-40, for the overflow check) and two words of the total weight that a
// weight read-out renormalises with.
constexpr double kRangeUnit = 1.0 / 1099511627776.0;  // 2^-40

// After a shard's pass: its floating-point deposited weight into the range word.
static __global__ void k_shard_pack(long long *hist, int hist_words, Scalars *sc)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        hist[hist_words] = llrint(ceil(sc->Wcheck / (sc->Wrange * kRangeUnit)));
        sc->Wcheck = 0.0;
    }
}

// The finalize of a shard from the exchanged (summed) words. red: blockDim doubles.
template <class T, int WPS>
__global__ void k_finalize(const Model m, const Buffers b, int init)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const StepFlags<T> f = step_flags<T>(m, *b.sc, init);
    __syncthreads();
    if (threadIdx.x == 0) {
        b.sc->Wcheck = double(b.hist[m.hist_words]) * (b.sc->Wrange * kRangeUnit);
        b.hist[m.hist_words] = 0;
    }
    __syncthreads();
    finalize_block<WPS>(m, b, m.n_all, init, f.prior_step, reinterpret_cast<double *>(smem), f.scf_step);
}

// ---------------------------------------------------------------- batched step kernel
//
// Many independent fits (their own potential, targets, priors and particle counts)
// advanced by one launch. The host cuts the fits' particles, taken in model order,
// into equal contiguous shares, one per block, and each share into segments
// (model, begin, end) of at most kMaxParticlesPerBlock particles. A block walks its
// segments: on a new model it loads the model's descriptors and tables into shared
// memory, it runs the per-particle step over the segment, and it flushes its sums
// into the model's global sums. The block that flushes a model's last segment runs
// that model's finalize. The sums are exact integers, so a fit advanced in a batch
// gives bit-identical results to the same fit advanced alone.
struct Segment {
    int model;
    int pad;
    long long begin, end;
};

template <class T>
struct BatchArgs {
    const Model *models;
    const Cst<T> *csts;
    const State<T> *states;
    const Buffers *bufs;
    const Segment *seg;
    const int *seg_off;      // block b walks seg[seg_off[b] .. seg_off[b+1])
    const unsigned *nseg;    // per model: its number of segments
};

// the batched kernel copies Model and Cst<T> into shared memory in 8-byte words
static_assert(sizeof(Model) % 8 == 0 && sizeof(Cst<float>) % 8 == 0 && sizeof(Cst<double>) % 8 == 0,
              "descriptor copies need whole 8-byte words");

// The per-fit constants of a batch in the kernel's parameter space (the constant bank): the
// per-particle loop reads them there, where no store can alias them, instead of from copies
// in shared memory that every shared-memory atomic of the deposit could have changed.
// shape: a Model that every fit of the batch equals in the fields of the per-particle path
// (see step_particles); cst[i]: the constants of fit i. With more fits than the bank holds,
// or fits that differ in those fields, the kernel runs from the shared-memory copies.
template <class T>
constexpr int kBankFits = sizeof(T) == 8 ? 112 : 224;

template <class T>
struct BatchBank {
    Model shape;
    Cst<T> cst[kBankFits<T>];
};
static_assert(sizeof(BatchBank<float>) + sizeof(BatchArgs<float>) <= 32764 &&
                  sizeof(BatchBank<double>) + sizeof(BatchArgs<double>) <= 32764,
              "kernel parameters are limited to 32764 bytes");

template <class T, int WPS, int MINB, bool BANK, unsigned M0, unsigned M1, unsigned M2, unsigned M3>
__global__ void __launch_bounds__(256, MINB) k_step_batch(const BatchArgs<T> a, const __grid_constant__ BatchBank<T> bank)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) unsigned long long mbuf[(sizeof(Model) + 7) / 8];
    __shared__ __align__(16) unsigned long long kbuf[(sizeof(Cst<T>) + 7) / 8];
    __shared__ Buffers sb;
    __shared__ State<T> sP;
    __shared__ bool am_last;
    const Model &m = *reinterpret_cast<const Model *>(mbuf);
    const Cst<T> &k = *reinterpret_cast<const Cst<T> *>(kbuf);

    int cur = -1;
    const int s1 = a.seg_off[blockIdx.x + 1];
    for (int s = a.seg_off[blockIdx.x]; s < s1; ++s) {
        const Segment sg = a.seg[s];
        const bool fresh = sg.model != cur;
        if (fresh) {
            __syncthreads();
            const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.models + sg.model);
            for (int q = threadIdx.x; q < int(sizeof(mbuf) / 8); q += blockDim.x) mbuf[q] = src[q];
            const unsigned long long *ks = reinterpret_cast<const unsigned long long *>(a.csts + sg.model);
            for (int q = threadIdx.x; q < int(sizeof(kbuf) / 8); q += blockDim.x) kbuf[q] = ks[q];
            if (threadIdx.x == 0) {
                sb = a.bufs[sg.model];
                sP = a.states[sg.model];
            }
            __syncthreads();
            cur = sg.model;
        }
        const Buffers &b = sb;
        const State<T> P = sP;
        const Smem<T> S = carve<T>(m, smem, 1, 1);
        const StepFlags<T> f = step_flags<T>(m, *b.sc, 0);
        block_zero<T, false>(m, S);
        if (fresh) block_tables<T, false>(m, b, S, f.pending);
        __syncthreads();
        unsigned err = 0;
        Total<T> wtot;
        T wdep = T(0);
        if constexpr (BANK)
            step_particles<T, false, M0, M1, M2, M3>(m, bank.shape, bank.cst[sg.model], P, b, S, f, 1,
                                                     sg.begin + threadIdx.x, sg.end, blockDim.x, err, wtot, wdep);
        else
            step_particles<T, false, M0, M1, M2, M3>(m, m, k, P, b, S, f, 1, sg.begin + threadIdx.x, sg.end,
                                                     blockDim.x, err, wtot, wdep);
        block_flush<T, WPS, false>(m, k, b, S, f.prior_step, err, wtot, wdep, f.scf_step);
        if (threadIdx.x == 0) am_last = atomicAdd(&b.sc->blocks_done, 1u) == a.nseg[cur] - 1;
        __syncthreads();
        if (am_last) {
            __threadfence();
            finalize_block<WPS>(m, b, P.n, 0, f.prior_step, reinterpret_cast<double *>(smem), f.scf_step);
            cur = -1;  // the finalize used the shared memory: reload before the next segment
        }
    }
}

// ---------------------------------------------------------------- helpers

// Weights as of the end of the last step: the pending force of change applied
// (without renormalisation) into out[], and the total added to acc (two words).
template <class T>
__global__ void k_materialize(const Model m, const Cst<T> k, const State<T> P, const Buffers b, double *out,
                              long long *acc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Smem<T> S = carve<T>(m, smem, 0, 0);
    const Scalars sc = *b.sc;
    if (m.mode == 1) {
        const double *pr = kLogWeights<T> ? b.lprior : b.iprior;
        for (int q = threadIdx.x; q < m.ncell; q += blockDim.x) S.iprior[q] = T(pr[q]);
    }
    load_tables(m, b, S);
    __syncthreads();
    const Tables<T> tb{S.esq, S.lut, S.vp, S.isp, S.e2};
    unsigned err = 0;
    Total<double> tot;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        T w;
        if constexpr (kLogWeights<T>) {
            T u = P.w[i] + T(sc.lwscale);
            if (sc.pending) {
                const T lp = (m.mode == 1) ? S.iprior[P.cell[i]] : T(sc.lwhat_flat);
                u = foc_update_log<kDyn, kDyn, kDyn, kDyn>(m, k, tb, global_records<T>(b), kApUncached,
                                                           static_cast<const T *>(nullptr), lp, u, P.x[i], P.y[i],
                                                           P.z[i], P.vy[i], P.vz[i], err);
            }
            w = kexp(tb, u);
        } else {
            w = P.w[i] * T(sc.wscale);
            if (sc.pending) {
                const T pr =
                    (m.mode == 1) ? S.iprior[P.cell[i]] : (sc.what_flat > 0.0 ? T(1.0 / sc.what_flat) : T(0));
                w = foc_update<kDyn, kDyn, kDyn, kDyn>(m, k, tb, global_records<T>(b), kApUncached,
                                                       static_cast<const T *>(nullptr), pr, w, P.x[i], P.y[i], P.z[i],
                                                       P.vy[i], P.vz[i], err);
            }
        }
        if (sc.pending && w != T(0)) tot.add(double(w), m.fx_w);
        out[i] = double(w);
    }
    if (err) atomicOr(&b.sc->err, err);
    for (int q = 0; q < 2; ++q) {
        long long s = tot.word(q, m.fx_w);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0 && s != 0)
            atomicAdd(reinterpret_cast<unsigned long long *>(acc + q), static_cast<unsigned long long>(s));
    }
}

static __global__ void k_scale(double *out, long long n, const long long *acc, const Model m, const Scalars *sc)
{
    const double U = (double(acc[0]) + double(acc[1]) * (1.0 / 4294967296.0)) / m.fx_w;
    if (!sc->pending || !m.renormalize || !(U > 0.0)) return;
    const double s = sc->W0 / U;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] *= s;
}

template <class T>
__global__ void k_convert_in(const double *src, T *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = T(src[i]);
}

// FP64 mode stores ln w (w = 0 gives -inf; load rejects negative weights first).
static __global__ void k_log_in(const double *src, double *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = log(src[i]);
}

template <class T>
__global__ void k_convert_out(const T *src, double *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = double(src[i]);
}

// Largest v^2 a particle can reach in the fixed potential (2 (E - phi_min)), and a
// flag for non-finite input or negative weights.
static __global__ void k_load_stats(const Model m, const Cst<double> k, const double *x, const double *y,
                             const double *z, const double *vx, const double *vy, const double *vz,
                             const double *w, long long n, unsigned long long *v2max_bits, unsigned *bad)
{
    double best = 0.0;
    unsigned flag = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
        // the self-consistent potential bounds only its halo here (its stellar well is added
        // on the host)
        const double pmin = m.pot == 3 ? m.v0 * m.v0 * log(m.r0) : m.phi_min;
        const double e = v2 + 2.0 * (potential<double>(m, k, x[i], y[i], z[i]) - pmin);
        const double val = e > v2 ? e : v2;
        if (!isfinite(val) || !isfinite(x[i] + y[i] + z[i]) || !isfinite(w[i]) || w[i] < 0.0) flag = 1;
        else if (val > best) best = val;
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    flag = __reduce_or_sync(0xffffffffu, flag);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(v2max_bits, static_cast<unsigned long long>(__double_as_longlong(best)));
        if (flag) atomicOr(bad, 1u);
    }
}

}  // namespace m2m
