// Device side of the M2M step: model description, per-particle arithmetic and
// the kernels. Templated on the state type T (double: FP64 mode; float: mixed
// mode) and on the number of int64 words per fixed-point sum (2 in FP64 mode,
// 1 in mixed mode).
//
// Method (arXiv 1202.2355): leap-frog push (Sec. 4.1), observables
// y_j = sum_i w_i K_j(z_i) (eq. obs) with the Gauss-Hermite kernels of
// eq. lumghn, temporal smoothing (eq. myts), residuals (eqs. delta, chi),
// (E, x) moving priors (Sec. 2.3.1) and the force of change (eq. modFOC) with
// the entropy of eq. S+ (moving priors) or eq. entropy (global).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace m2m {

constexpr int kMaxGroups = 4;
constexpr int kMaxKinds = 8;
constexpr int kKindMass = 0;
constexpr int kKindV2 = 1;
constexpr int kKindV1 = 2;  // internal: first moment, used only to build targets
constexpr int kKindGH0 = 10;

enum : unsigned { kErrNonFinite = 1u, kErrNegWeight = 2u, kErrOverflow = 4u, kErrIndex = 8u };

struct GroupDesc {
    int geometry;   // 0 annuli, 1 pixels
    int n_ap;
    int n_kinds;
    int obs_off;    // first observable index of the group
    int ap_off;     // first aperture index (into Vp / 1/sp arrays)
    int edge_off;   // first edge (annuli)
    int max_gh;     // highest Gauss-Hermite order used, -1 if none
    int nx, ny;
    int kinds[kMaxKinds];
    double xlo, ylo, xw, yw;  // pixel box origin and widths (xhi - xlo, yhi - ylo)
};

struct Model {
    // potential
    int pot;                      // 0 Hernquist, 1 Hernquist + NFW, 2 log
    double G, M, a, Ms, rs, v0, r0, q;
    double phi_min;
    // projection
    double sin_i, cos_i;
    // observables
    int n_groups, J, n_ap_total, n_edges_total;
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
    int wps;                      // int64 words per sum
    int hist_words, off_total, off_grid, off_count;
};

// Per-fit scalars living in device memory, written by the finalize kernel.
struct Scalars {
    long long t;        // steps completed
    double wscale;      // current weight = wscale * stored weight
    double W0;          // initial total weight
    double what_flat;   // flat prior W0/N (global entropy)
    double chi2;
    double Wsum;        // total stored weight of the last deposit
    double Wcheck;      // floating-point sum of the deposited weights (range check only)
    double Wrange;      // largest total weight the fixed-point sums can hold
    int pending;        // the previous step's force of change is still to be applied
    unsigned err;       // latched kErr* bits
};

template <class T>
struct State {
    T *x, *y, *z, *vx, *vy, *vz, *w;
    uint16_t *cell;
    long long n;
};

struct Buffers {
    const double *edges, *Vp, *isp;  // per group edges, per aperture V_p and 1/sigma_p
    const double *lcE;               // E_c table
    const double *Y, *sig;
    const int *obs_kind;             // per observable: kind
    const double *obs_post;          // per observable: factor applied to the raw sum (1/area for mass)
    const double *obs_iscale;        // per observable: 1/fixed-point scale
    double *c;                       // per observable: coefficient of the force of change
    double *prior;                   // per cell: prior (cell mean weight)
    long long *prior_count;          // per cell: particle count at the last update
    long long *hist;                 // fixed-point accumulators
    double *ytil, *yraw, *delta;
    Scalars *sc;
};

// ---------------------------------------------------------------- math helpers
__host__ __device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__host__ __device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float d_exp(float x) { return expf(x); }
__host__ __device__ __forceinline__ double d_exp(double x) { return exp(x); }
__host__ __device__ __forceinline__ float d_log(float x) { return logf(x); }
__host__ __device__ __forceinline__ double d_log(double x) { return log(x); }
__host__ __device__ __forceinline__ float d_log1p(float x) { return log1pf(x); }
__host__ __device__ __forceinline__ double d_log1p(double x) { return log1p(x); }
__host__ __device__ __forceinline__ float d_floor(float x) { return floorf(x); }
__host__ __device__ __forceinline__ double d_floor(double x) { return floor(x); }
__host__ __device__ __forceinline__ bool d_finite(float x) { return isfinite(x); }
__host__ __device__ __forceinline__ bool d_finite(double x) { return isfinite(x); }

// ---------------------------------------------------------------- potentials

// NFW enclosed-mass factor mu(q) = ln(1+q) - q/(1+q). For small q the two terms
// cancel. FP64: below q = 1e-3 the alternating series sum_k (-1)^k (k-1)/k q^k
// (Horner). FP32: below q = 0.3 the positive series sum_{k>=2} t^k/k in
// t = q/(1+q) (from ln(1+q) = -ln(1-t)), which has no cancellation.
template <class T>
__host__ __device__ __forceinline__ T nfw_mu(T qq)
{
    if (sizeof(T) == 8) {
        if (qq < T(1e-3)) {
            T s = T(-10.0 / 11.0);
            s = T(9.0 / 10.0) + qq * s;
            s = T(-8.0 / 9.0) + qq * s;
            s = T(7.0 / 8.0) + qq * s;
            s = T(-6.0 / 7.0) + qq * s;
            s = T(5.0 / 6.0) + qq * s;
            s = T(-4.0 / 5.0) + qq * s;
            s = T(3.0 / 4.0) + qq * s;
            s = T(-2.0 / 3.0) + qq * s;
            s = T(0.5) + qq * s;
            return qq * qq * s;
        }
    } else if (qq < T(0.3)) {
        const T t = qq / (T(1) + qq);
        T s = T(1.0 / 14.0);
        s = T(1.0 / 13.0) + t * s;
        s = T(1.0 / 12.0) + t * s;
        s = T(1.0 / 11.0) + t * s;
        s = T(1.0 / 10.0) + t * s;
        s = T(1.0 / 9.0) + t * s;
        s = T(1.0 / 8.0) + t * s;
        s = T(1.0 / 7.0) + t * s;
        s = T(1.0 / 6.0) + t * s;
        s = T(1.0 / 5.0) + t * s;
        s = T(1.0 / 4.0) + t * s;
        s = T(1.0 / 3.0) + t * s;
        s = T(0.5) + t * s;
        return t * t * s;
    }
    return d_log1p(qq) - qq / (T(1) + qq);
}

template <class T>
__host__ __device__ __forceinline__ T potential(const Model &m, T x, T y, T z)
{
    if (m.pot == 2) {
        const T q2 = T(m.q * m.q);
        const T D = T(m.r0 * m.r0) + x * x + y * y + z * z / q2;
        return T(0.5 * m.v0 * m.v0) * d_log(D);
    }
    const T r = d_sqrt(x * x + y * y + z * z);
    T phi = -T(m.G * m.M) / (r + T(m.a));
    if (m.pot == 1) phi += (r > T(0)) ? -T(m.G * m.Ms) * d_log1p(r / T(m.rs)) / r : -T(m.G * m.Ms / m.rs);
    return phi;
}

template <class T>
__host__ __device__ __forceinline__ void accel(const Model &m, T x, T y, T z, T &ax, T &ay, T &az)
{
    if (m.pot == 2) {
        const T q2 = T(m.q * m.q);
        const T D = T(m.r0 * m.r0) + x * x + y * y + z * z / q2;
        const T f = -T(m.v0 * m.v0) / D;
        ax = f * x;
        ay = f * y;
        az = f * z / q2;
        return;
    }
    const T r2 = x * x + y * y + z * z;
    const T r = d_sqrt(r2);
    if (r == T(0)) {
        ax = ay = az = T(0);
        return;
    }
    const T ra = r + T(m.a);
    // -g(r)/r with g = G M(<r) / r^2
    T f = T(m.G * m.M) / (ra * ra * r);
    if (m.pot == 1) f += T(m.G * m.Ms) * nfw_mu(r / T(m.rs)) / (r2 * r);
    ax = -f * x;
    ay = -f * y;
    az = -f * z;
}

// One kick-drift-kick leap-frog step.
template <class T>
__device__ __forceinline__ void leapfrog(const Model &m, T &x, T &y, T &z, T &vx, T &vy, T &vz)
{
    const T hdt = T(0.5 * m.dt), dt = T(m.dt);
    T ax, ay, az;
    accel(m, x, y, z, ax, ay, az);
    vx += hdt * ax;
    vy += hdt * ay;
    vz += hdt * az;
    x += dt * vx;
    y += dt * vy;
    z += dt * vz;
    accel(m, x, y, z, ax, ay, az);
    vx += hdt * ax;
    vy += hdt * ay;
    vz += hdt * az;
}

// ---------------------------------------------------------------- observables

template <class T>
__device__ __forceinline__ void project(const Model &m, T y, T z, T vy, T vz, T &Y, T &vlos)
{
    const T si = T(m.sin_i), ci = T(m.cos_i);
    Y = y * ci - z * si;
    vlos = vy * si + vz * ci;
}

// Aperture of sky point (X, Y) in group G, or -1. Annuli: binary search of the
// half-open intervals edges[p] <= R < edges[p+1].
template <class T>
__device__ __forceinline__ int aperture(const GroupDesc &G, const T *edges, T X, T Y)
{
    if (G.geometry == 0) {
        const T R = d_sqrt(X * X + Y * Y);
        const T *e = edges + G.edge_off;
        if (!(R >= e[0]) || !(R < e[G.n_ap])) return -1;
        int lo = 0, hi = G.n_ap;  // e[lo] <= R < e[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (e[mid] <= R) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    const T fx = d_floor((X - T(G.xlo)) * T(G.nx) / T(G.xw));
    const T fy = d_floor((Y - T(G.ylo)) * T(G.ny) / T(G.yw));
    if (!(fx >= T(0)) || !(fx < T(G.nx)) || !(fy >= T(0)) || !(fy < T(G.ny))) return -1;
    return int(fy) * G.nx + int(fx);
}

// Gauss-Hermite kernel values K_n = 2 sqrt(pi) u_n(nu) = sqrt(2^(1-n)/n!) H_n(nu) e^(-nu^2/2)
// for n = 0..nmax, with H_n by the three-term recurrence H_{n+1} = 2 nu H_n - 2 n H_{n-1}.
template <class T>
__device__ __forceinline__ void gh_values(T nu, int nmax, T *K)
{
    const T e = d_exp(T(-0.5) * nu * nu);
    T hm1 = T(1), h = T(2) * nu;
    K[0] = T(1.4142135623730950488) * e;
    if (nmax >= 1) K[1] = h * e;  // sqrt(2^0/1!) = 1
    // c_n = sqrt(2^(1-n)/n!)
    const T cn[7] = {T(1.4142135623730950488), T(1.0), T(0.5), T(0.20412414523193150818),
                     T(0.072168783648703220563), T(0.022821773229381921355),
                     T(0.0065881721129167866018)};
    for (int n = 1; n < nmax; ++n) {
        const T hn1 = T(2) * nu * h - T(2 * n) * hm1;
        hm1 = h;
        h = hn1;
        K[n + 1] = cn[n + 1] * h * e;
    }
}

// Calls f(j, K_j) for every observable j with K_j(z) != 0 for the particle with
// sky position (X, Y) and line-of-sight velocity vlos.
template <class T, class F>
__device__ __forceinline__ void for_each_kernel(const Model &m, const T *edges, const T *vp,
                                                const T *isp, T X, T Y, T vlos, F &&f)
{
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
        if (g >= m.n_groups) break;
        const GroupDesc &G = m.g[g];
        const int p = aperture(G, edges, X, Y);
        if (p < 0) continue;
        T gh[7];
        if (G.max_gh >= 0) {
            const T nu = (vlos - vp[G.ap_off + p]) * isp[G.ap_off + p];
            gh_values(nu, G.max_gh, gh);
        }
        for (int k = 0; k < G.n_kinds; ++k) {
            const int kind = G.kinds[k];
            T K;
            if (kind == kKindMass) K = T(1);
            else if (kind == kKindV2) K = vlos * vlos;
            else if (kind == kKindV1) K = vlos;
            else K = gh[kind - kKindGH0];
            f(G.obs_off + k * G.n_ap + p, kind, K);
        }
    }
}

// ---------------------------------------------------------------- priors

// Energy of the circular orbit of radius R in the equatorial plane.
template <class T>
__host__ __device__ __forceinline__ T circ_energy(const Model &m, T R)
{
    T ax, ay, az;
    accel(m, R, T(0), T(0), ax, ay, az);
    return potential(m, R, T(0), T(0)) - T(0.5) * R * ax;
}

// Lc(E): closed form for the Hernquist potential (E_c = -(u+1)/(2u^2) GM/a with
// u = R/a + 1), otherwise the host table of E_c(ln R) bracketed by binary search,
// interpolated, and refined by secant steps on E_c(R) = E.
template <class T>
__device__ T circular_L(const Model &m, const double *lcE, T E)
{
    if (m.pot != 2 && !(E < T(0))) return T(0);
    if (m.lc_closed) {
        const T e = E * T(m.a / (m.G * m.M));
        if (!(e > T(-1))) return T(0);
        const T u = (T(-1) - d_sqrt(T(1) - T(8) * e)) / (T(4) * e);
        const T R = T(m.a) * (u - T(1));
        const T ra = R + T(m.a);
        return R * d_sqrt(T(m.G * m.M) * R) / ra;
    }
    if (!(E > T(m.phi_min))) return T(0);
    const int n = m.lc_n;
    int lo = 0, hi = n - 1;
    T R;
    if (!(E > T(__ldg(lcE)))) {
        R = T(exp(m.lc_lnr0));
    } else if (!(E < T(__ldg(lcE + n - 1)))) {
        R = T(exp(m.lc_lnr0 + (n - 1) * m.lc_dlnr));
    } else {
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (T(__ldg(lcE + mid)) <= E) lo = mid;
            else hi = mid;
        }
        const T e0 = T(__ldg(lcE + lo)), e1 = T(__ldg(lcE + hi));
        const T fr = (E - e0) / (e1 - e0);
        R = d_exp(T(m.lc_lnr0) + (T(lo) + fr) * T(m.lc_dlnr));
        // secant refinement, starting from the table segment's slope
        const T Ra = d_exp(T(m.lc_lnr0) + T(lo) * T(m.lc_dlnr));
        const T Rb = d_exp(T(m.lc_lnr0) + T(hi) * T(m.lc_dlnr));
        T r0 = R, f0 = circ_energy(m, r0) - E;
        T r1 = r0 - f0 * (Rb - Ra) / (e1 - e0);
        for (int it = 0; it < 3; ++it) {
            const T f1 = circ_energy(m, r1) - E;
            if (f1 == f0) break;
            const T r2 = r1 - f1 * (r1 - r0) / (f1 - f0);
            r0 = r1;
            f0 = f1;
            r1 = r2;
        }
        R = r1;
    }
    T ax, ay, az;
    accel(m, R, T(0), T(0), ax, ay, az);
    return R * d_sqrt(-R * ax);
}

template <class T>
__device__ __forceinline__ int prior_cell(const Model &m, const double *lcE, T x, T y, T z, T vx,
                                          T vy, T vz)
{
    const T E = T(0.5) * (vx * vx + vy * vy + vz * vz) + potential(m, x, y, z);
    const T Lz = x * vy - y * vx;
    T L;
    if (m.signed_lz) {
        L = Lz;
    } else {
        const T Lx = y * vz - z * vy, Ly = z * vx - x * vz;
        L = d_sqrt(Lx * Lx + Ly * Ly + Lz * Lz);
    }
    const T Lc = circular_L(m, lcE, E);
    T xc = (Lc > T(0)) ? L / Lc : T(0);
    const T xmin = m.signed_lz ? T(-1) : T(0);
    xc = xc < xmin ? xmin : (xc > T(1) ? T(1) : xc);
    T f;
    if (m.e_spacing == 0) f = (E >= T(0)) ? T(1) : (d_log(-E) - T(m.s_lo)) / T(m.s_den);
    else if (m.e_spacing == 1) f = (d_exp(E) - T(m.s_lo)) / T(m.s_den);
    else f = (E - T(m.s_lo)) / T(m.s_den);
    const T fk = d_floor(f * T(m.nE));
    const int k = !(fk >= T(0)) ? 0 : (fk >= T(m.nE) ? m.nE - 1 : int(fk));
    const T fl = d_floor((xc - xmin) / (T(1) - xmin) * T(m.nx));
    const int l = !(fl >= T(0)) ? 0 : (fl >= T(m.nx) ? m.nx - 1 : int(fl));
    return k * m.nx + l;
}

// ---------------------------------------------------------------- fixed point

// Adds v * scale to a fixed-point sum. One word: round to nearest int64. Two
// words: integer part and the next 32 fraction bits, each summed exactly.
template <int WPS>
__device__ __forceinline__ void fx_add(long long *h, int slot, double v, double scale)
{
    const double s = v * scale;
    if (WPS == 1) {
        atomicAdd(reinterpret_cast<unsigned long long *>(h + slot),
                  static_cast<unsigned long long>(__double2ll_rn(s)));
    } else {
        const double hi = floor(s);
        const long long ihi = static_cast<long long>(hi);
        const long long ilo = __double2ll_rn((s - hi) * 4294967296.0);
        atomicAdd(reinterpret_cast<unsigned long long *>(h + 2 * slot), static_cast<unsigned long long>(ihi));
        atomicAdd(reinterpret_cast<unsigned long long *>(h + 2 * slot + 1), static_cast<unsigned long long>(ilo));
    }
}

template <int WPS>
__device__ __forceinline__ void fx_add_f(long long *h, int slot, float v, float scale)
{
    // mixed mode (WPS == 1): the product carries 24 significant bits
    atomicAdd(reinterpret_cast<unsigned long long *>(h + slot),
              static_cast<unsigned long long>(__float2ll_rn(v * scale)));
}

template <int WPS>
__device__ __forceinline__ double fx_read(const long long *h, int slot)
{
    if (WPS == 1) return double(h[slot]);
    return double(h[2 * slot]) + double(h[2 * slot + 1]) * (1.0 / 4294967296.0);
}

template <class T, int WPS>
__device__ __forceinline__ void deposit(long long *h, int slot, T v, double scale)
{
    if (v == T(0)) return;
    if (sizeof(T) == 4) fx_add_f<WPS>(h, slot, float(v), float(scale));
    else fx_add<WPS>(h, slot, double(v), scale);
}

// ---------------------------------------------------------------- force of change

// Weight after the force of change of eq. modFOC over one step, the kernel
// values taken at the particle's current position and the priors held fixed:
// F = mu dS/dw - sum_j K_j c_j, c_j = Delta_j/sigma_j (times 1/area for mass),
// dS/dw = -ln(w/what) (eq. S+) or -ln(w/what) - 1 (eq. entropy).
template <class T>
__device__ __forceinline__ T foc_update(const Model &m, const T *edges, const T *vp, const T *isp,
                                        const T *c, T prior, T w, T x, T y, T z, T vy, T vz,
                                        unsigned &err)
{
    if (w == T(0)) return w;  // w = 0 is a fixed point
    T Y, vlos;
    project(m, y, z, vy, vz, Y, vlos);
    T data = T(0);
    for_each_kernel(m, edges, vp, isp, x, Y, vlos, [&](int j, int, T K) { data += K * c[j]; });
    // A cell mean below the resolution of the fixed-point cell sums reads as 0;
    // the particle's weight is then unresolved too and the entropy term is dropped.
    T dS = prior > T(0) ? -d_log(w / prior) : T(0);
    if (m.mode == 0) dS -= T(1);
    const T h = T(m.dt * m.eps) * (T(m.mu) * dS - data);
    T wn;
    if (m.update_rule == 0) wn = w * d_exp(h);
    else wn = w * (T(1) + h);
    if (!d_finite(wn)) err |= kErrNonFinite;
    else if (wn < T(0) || (m.update_rule == 1 && !(wn > T(0)))) err |= kErrNegWeight;
    return wn;
}

// Loads the per-aperture tables (edges, V_p, 1/sigma_p) into shared memory.
template <class T>
__device__ __forceinline__ void load_tables(const Model &m, const Buffers &b, T *edges_s, T *vp_s,
                                            T *isp_s)
{
    for (int k = threadIdx.x; k < m.n_edges_total; k += blockDim.x) edges_s[k] = T(b.edges[k]);
    for (int k = threadIdx.x; k < m.n_ap_total; k += blockDim.x) {
        vp_s[k] = T(b.Vp[k]);
        isp_s[k] = T(b.isp[k]);
    }
}

// Shared-memory layout of the step kernel (bytes).
template <class T>
__host__ __device__ inline size_t step_smem_bytes(const Model &m)
{
    return sizeof(long long) * size_t(m.hist_words) +
           sizeof(T) * size_t(m.J + m.ncell + m.n_edges_total + 2 * m.n_ap_total);
}

// ---------------------------------------------------------------- step kernel
//
// One M2M step over all particles, one read and one write of the particle
// state: (a) the previous step's force of change at the current position,
// (b) kick-drift-kick push, (c) deposit of w K_j into block-local fixed-point
// sums, (d) on prior-update steps the (E, x) cell of every particle and the
// per-cell weight sums and counts. Block sums are added to the global sums
// with integer atomics, so the result does not depend on the order.
template <class T, int WPS>
__global__ void __launch_bounds__(256) k_step(const Model m, const State<T> P, const Buffers b,
                                              int push, int init)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *h = reinterpret_cast<long long *>(smem);
    T *c_s = reinterpret_cast<T *>(h + m.hist_words);
    T *pri_s = c_s + m.J;
    T *edges_s = pri_s + m.ncell;
    T *vp_s = edges_s + m.n_edges_total;
    T *isp_s = vp_s + m.n_ap_total;

    const Scalars sc = *b.sc;
    const long long t = sc.t + 1;
    const int pending = init ? 0 : sc.pending;
    const int prior_step = !init && m.mode == 1 && ((t - 1) % m.update_every) == 0;
    const T wscale = init ? T(1) : T(sc.wscale);
    const T what_flat = T(sc.what_flat);

    for (int k = threadIdx.x; k < m.hist_words; k += blockDim.x) h[k] = 0;
    if (pending) {
        for (int k = threadIdx.x; k < m.J; k += blockDim.x) c_s[k] = T(b.c[k]);
        if (m.mode == 1)
            for (int k = threadIdx.x; k < m.ncell; k += blockDim.x) pri_s[k] = T(b.prior[k]);
    }
    load_tables(m, b, edges_s, vp_s, isp_s);
    __syncthreads();

    unsigned err = 0;
    double wdep = 0.0;  // weight deposited by this thread, for the fixed-point range check
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        T x = P.x[i], y = P.y[i], z = P.z[i];
        T vx = P.vx[i], vy = P.vy[i], vz = P.vz[i];
        T w = P.w[i] * wscale;
        if (pending) {
            const T pr = (m.mode == 1) ? pri_s[P.cell[i]] : what_flat;
            w = foc_update(m, edges_s, vp_s, isp_s, c_s, pr, w, x, y, z, vy, vz, err);
        }
        if (push) leapfrog(m, x, y, z, vx, vy, vz);
        T Y, vlos;
        project(m, y, z, vy, vz, Y, vlos);
        if (w != T(0)) {
            for_each_kernel(m, edges_s, vp_s, isp_s, x, Y, vlos, [&](int j, int kind, T K) {
                double sc_ = kind == kKindMass ? m.fx_w : (kind == kKindV2 ? m.fx_v2 : m.fx_gh);
                if (kind == kKindV2 && K > T(m.v2max)) err |= kErrOverflow;
                if (kind == kKindV1) sc_ = m.fx_v2;
                deposit<T, WPS>(h, j, w * K, sc_);
            });
            deposit<T, WPS>(h, m.J, w, m.fx_w);
            wdep += double(w);
        }
        if (prior_step) {
            const int c = prior_cell(m, b.lcE, x, y, z, vx, vy, vz);
            if (w != T(0)) deposit<T, WPS>(h, m.J + 1 + c, w, m.fx_w);
            atomicAdd(reinterpret_cast<unsigned long long *>(h + m.off_count + c), 1ull);
            P.cell[i] = static_cast<uint16_t>(c);
        }
        P.x[i] = x;
        P.y[i] = y;
        P.z[i] = z;
        P.vx[i] = vx;
        P.vy[i] = vy;
        P.vz[i] = vz;
        P.w[i] = w;
    }
    if (err) atomicOr(&b.sc->err, err);
    // the check sum only guards the fixed-point range, so its summation order does not matter
    for (int o = 16; o > 0; o >>= 1) wdep += __shfl_xor_sync(0xffffffffu, wdep, o);
    if ((threadIdx.x & 31) == 0 && wdep != 0.0) atomicAdd(&b.sc->Wcheck, wdep);
    __syncthreads();
    const int words = prior_step ? m.hist_words : m.off_grid;
    for (int k = threadIdx.x; k < words; k += blockDim.x) {
        const long long v = h[k];
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long *>(b.hist + k), static_cast<unsigned long long>(v));
    }
}

// ---------------------------------------------------------------- finalize kernel
//
// One block: converts the fixed-point sums, renormalises, smooths (eq. myts),
// forms Delta_j, chi^2 (eqs. delta, chi) and the force-of-change coefficients,
// the prior means on update steps, and clears the sums for the next step.
template <int WPS>
__global__ void __launch_bounds__(1024) k_finalize(const Model m, const Buffers b, long long n, int init)
{
    __shared__ double red[1024];
    __shared__ double s_ren_s;
    __shared__ int prior_step_s;
    Scalars &sc = *b.sc;
    const long long t = init ? 0 : sc.t + 1;
    if (threadIdx.x == 0) {
        const double U = fx_read<WPS>(b.hist, m.J) / m.fx_w;
        double s_ren = 1.0;
        if (init) {
            sc.W0 = U;
            sc.what_flat = n > 0 ? U / double(n) : 0.0;
        } else if (m.renormalize && U > 0.0) {
            s_ren = sc.W0 / U;
        }
        // the integer sums wrap beyond the range: the floating-point check sum catches it
        if (!(sc.Wcheck <= 0.5 * sc.Wrange)) atomicOr(&sc.err, kErrOverflow);
        sc.Wcheck = 0.0;
        sc.Wsum = U;
        s_ren_s = s_ren;
        prior_step_s = !init && m.mode == 1 && ((t - 1) % m.update_every) == 0;
    }
    __syncthreads();
    const double s_ren = s_ren_s;
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
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (prior_step_s) {
        for (int c = threadIdx.x; c < m.ncell; c += blockDim.x) {
            const long long cnt = b.hist[m.off_count + c];
            const double sum = fx_read<WPS>(b.hist, m.J + 1 + c) / m.fx_w * s_ren;
            b.prior[c] = cnt > 0 ? sum / double(cnt) : 0.0;
            b.prior_count[c] = cnt;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m.hist_words; k += blockDim.x) b.hist[k] = 0;
    if (threadIdx.x == 0) {
        sc.chi2 = red[0];
        if (!init) sc.t = t;
        sc.wscale = s_ren;
        sc.pending = init ? 0 : (t > m.n_relax ? 1 : 0);
    }
}

// ---------------------------------------------------------------- helpers

// Weights as of the end of the last step: the pending force of change applied
// (without renormalisation) into out[], and the total added to acc (one sum).
template <class T, int WPS>
__global__ void k_materialize(const Model m, const State<T> P, const Buffers b, double *out,
                              long long *acc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *c_s = reinterpret_cast<T *>(smem);
    T *pri_s = c_s + m.J;
    T *edges_s = pri_s + m.ncell;
    T *vp_s = edges_s + m.n_edges_total;
    T *isp_s = vp_s + m.n_ap_total;
    const Scalars sc = *b.sc;
    for (int k = threadIdx.x; k < m.J; k += blockDim.x) c_s[k] = T(b.c[k]);
    if (m.mode == 1)
        for (int k = threadIdx.x; k < m.ncell; k += blockDim.x) pri_s[k] = T(b.prior[k]);
    load_tables(m, b, edges_s, vp_s, isp_s);
    __syncthreads();
    unsigned err = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        T w = P.w[i] * T(sc.wscale);
        if (sc.pending) {
            const T pr = (m.mode == 1) ? pri_s[P.cell[i]] : T(sc.what_flat);
            w = foc_update(m, edges_s, vp_s, isp_s, c_s, pr, w, P.x[i], P.y[i], P.z[i], P.vy[i],
                           P.vz[i], err);
            if (w != T(0)) fx_add<2>(acc, 0, double(w), m.fx_w);
        }
        out[i] = double(w);
    }
    if (err) atomicOr(&b.sc->err, err);
}

__global__ void k_scale(double *out, long long n, const long long *acc, const Model m, const Scalars *sc)
{
    const double U = fx_read<2>(acc, 0) / m.fx_w;
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

template <class T>
__global__ void k_convert_out(const T *src, double *dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = double(src[i]);
}

// Largest v^2 a particle can reach in the fixed potential (2 (E - phi_min)),
// and the total weight and smallest weight, for the fixed-point ranges.
__global__ void k_load_stats(const Model m, const double *x, const double *y, const double *z,
                             const double *vx, const double *vy, const double *vz, const double *w,
                             long long n, unsigned long long *v2max_bits, unsigned *bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
        const double e = v2 + 2.0 * (potential<double>(m, x[i], y[i], z[i]) - m.phi_min);
        const double val = e > v2 ? e : v2;
        if (!isfinite(val) || !isfinite(x[i] + y[i] + z[i]) || !isfinite(w[i]) || w[i] < 0.0) atomicOr(bad, 1u);
        else atomicMax(v2max_bits, static_cast<unsigned long long>(__double_as_longlong(val)));
    }
}

}  // namespace m2m
