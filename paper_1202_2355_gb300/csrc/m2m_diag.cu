// Diagnostics of a fitted particle model on the device.
//
// Sec. 4.1 assesses a fit by how well it recovers the target's intrinsic kinematics and
// its phase-space structure:
// - the intrinsic velocity moments (streaming velocities and dispersions along e_r,
//   e_theta, e_phi) in spherical polar bins: shells quasi-logarithmic in r, equal bins in
//   the azimuth phi and in cos(theta); the comparison with the target is the rms
//   difference of each moment over the bins both models populate;
// - Delta_grid, the mass-weighted relative rms difference of the model's and the
//   target's weights in the (E, x) cells of the prior grid.
// Sec. 5 (Fig. res) adds the rms of the particle weights about their cell means over the
// cells holding more than a minimum number of particles.
//
// The kernels bin either the fit's own particles (their state in the fit's precision,
// with the weights as of the end of the last step) or particles the caller passes from
// the host (a target realisation). Positions and velocities are taken to FP64 and every
// bin is decided in FP64. The per-bin sums are exact integer sums in the two-word fixed
// point of the step kernel (the integer part and the next 32 fraction bits of v * scale,
// scale a power of two): each term is converted to integers once, and integer addition
// does not depend on the order of the atomics, so the sums are bit-reproducible whatever
// the launch shape or the order of the particles. The scales come from a first pass that
// finds the largest |w| and |v|^2 (maxima, also order-independent), so that no bin sum
// can leave the range. The comparisons (moments, Delta_kin, Delta_grid, rms) are a few
// thousand bins of host arithmetic.
#include "m2m_ctx.h"

#include <cmath>
#include <cstring>
#include <vector>

using namespace m2m;

namespace {

constexpr int kKinSums = M2M_KIN_SUMS;
constexpr int kDiagThreads = 256;

// Spherical bins: shell 0 is [0, r_min); shells 1 .. n_r-1 are equal in ln r up to r_max.
struct SphBins {
    int n_r, n_phi, n_ct;
    double r_min, r_max, ln_rmin, ln_span;  // ln(r_max) - ln(r_min)
};

__device__ int sph_bin(const SphBins &g, double x, double y, double z)
{
    const double r = sqrt(x * x + y * y + z * z);
    if (!(r < g.r_max)) return -1;
    int ir = 0;
    if (r >= g.r_min) {
        const double f = (log(r) - g.ln_rmin) / g.ln_span;
        ir = 1 + int(floor(f * (g.n_r - 1)));
        if (ir > g.n_r - 1) ir = g.n_r - 1;
    }
    const double ct = r > 0.0 ? z / r : 1.0;
    int ic = int(floor((ct + 1.0) * 0.5 * g.n_ct));
    ic = ic < 0 ? 0 : (ic > g.n_ct - 1 ? g.n_ct - 1 : ic);
    const double ph = atan2(y, x);
    int ip = int(floor((ph + 3.14159265358979323846) / (2.0 * 3.14159265358979323846) * g.n_phi));
    ip = ip < 0 ? 0 : (ip > g.n_phi - 1 ? g.n_phi - 1 : ip);
    return (ir * g.n_ct + ic) * g.n_phi + ip;
}

// v along e_r, e_theta, e_phi; phi = 0 on the z axis and e_r = e_z at the centre.
__device__ void sph_velocity(double x, double y, double z, double vx, double vy, double vz, double v[3])
{
    const double R = sqrt(x * x + y * y);
    const double r = sqrt(R * R + z * z);
    const double cp = R > 0.0 ? x / R : 1.0, sp = R > 0.0 ? y / R : 0.0;
    const double ct = r > 0.0 ? z / r : 1.0, st = r > 0.0 ? R / r : 0.0;
    v[0] = vx * st * cp + vy * st * sp + vz * ct;
    v[1] = vx * ct * cp + vy * ct * sp - vz * st;
    v[2] = -vx * sp + vy * cp;
}

template <class T>
struct Particles {
    const T *x, *y, *z, *vx, *vy, *vz;
    const double *w;
    long long n;
};

// Fixed-point scales of the sums (powers of two): weights, w v and w v^2, and squared
// deviations from the cell means.
struct DiagScales {
    double w, wv, wv2, dev;
};

// Adds v to the two-word fixed-point sum at h[0], h[1].
__device__ __forceinline__ void fx_add(long long *h, double v, double scale)
{
    if (v == 0.0) return;
    long long hi, lo;
    fx2(v, scale, hi, lo);
    red_add(h, hi);
    if (lo) red_add(h + 1, lo);
}

// Largest |w| and |v|^2 (as ordered bit patterns of non-negative doubles) and a flag for
// non-finite input.
template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_diag_stats(const Particles<T> p, unsigned long long *mx,
                                                             unsigned *bad)
{
    double bw = 0.0, bv = 0.0;
    unsigned flag = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
         i += (long long)gridDim.x * blockDim.x) {
        const double vx = double(p.vx[i]), vy = double(p.vy[i]), vz = double(p.vz[i]);
        const double v2 = vx * vx + vy * vy + vz * vz, aw = fabs(p.w[i]);
        if (!isfinite(v2) || !isfinite(aw) || !isfinite(double(p.x[i]) + double(p.y[i]) + double(p.z[i]))) {
            flag = 1;
            continue;
        }
        bw = fmax(bw, aw);
        bv = fmax(bv, v2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        bw = fmax(bw, __shfl_xor_sync(0xffffffffu, bw, o));
        bv = fmax(bv, __shfl_xor_sync(0xffffffffu, bv, o));
    }
    flag = __reduce_or_sync(0xffffffffu, flag);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(mx, static_cast<unsigned long long>(__double_as_longlong(bw)));
        atomicMax(mx + 1, static_cast<unsigned long long>(__double_as_longlong(bv)));
        if (flag) atomicOr(bad, 1u);
    }
}

// Per bin: sum w; sum w v_c; sum w v_c^2 (c = r, theta, phi), each two int64 words.
template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_kin_sums(const SphBins g, const Particles<T> p, DiagScales sc,
                                                           long long *sums, unsigned long long *counts)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = double(p.x[i]), y = double(p.y[i]), z = double(p.z[i]);
        const int b = sph_bin(g, x, y, z);
        if (b < 0) continue;
        double v[3];
        sph_velocity(x, y, z, double(p.vx[i]), double(p.vy[i]), double(p.vz[i]), v);
        const double w = p.w[i];
        long long *o = sums + (long long)b * (2 * kKinSums);
        fx_add(o, w, sc.w);
        for (int c = 0; c < 3; ++c) {
            fx_add(o + 2 * (1 + c), w * v[c], sc.wv);
            fx_add(o + 2 * (4 + c), w * v[c] * v[c], sc.wv2);
        }
        atomicAdd(counts + b, 1ull);
    }
}

// First pass over the (E, x) grid: each particle's cell, the cell's weight and count.
template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_grid_sums(const Model m, const Cst<double> k, const double *lcE,
                                                            const Particles<T> p, DiagScales sc, int *cell,
                                                            long long *wsum, unsigned long long *counts)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = prior_cell<double>(m, k, lcE, double(p.x[i]), double(p.y[i]), double(p.z[i]),
                                         double(p.vx[i]), double(p.vy[i]), double(p.vz[i]));
        cell[i] = c;
        fx_add(wsum + 2 * c, p.w[i], sc.w);
        atomicAdd(counts + c, 1ull);
    }
}

// Value of a two-word fixed-point sum.
__host__ __device__ inline double fx_value(const long long *h, double scale)
{
    return (double(h[0]) + double(h[1]) * (1.0 / 4294967296.0)) / scale;
}

// Second pass: squared deviations from the cell means (the means from the exact sums).
__global__ void __launch_bounds__(kDiagThreads) k_grid_dev(long long n, const int *cell, const double *w,
                                                           const long long *wsum, const unsigned long long *counts,
                                                           DiagScales sc, long long *wdev2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = cell[i];
        const double d = w[i] - fx_value(wsum + 2 * c, sc.w) / double(counts[c]);
        fx_add(wdev2 + 2 * c, d * d, sc.dev);
    }
}

// Device copies of the particles the diagnostics bin, and the scratch they need; freed on
// destruction.
struct Scratch {
    std::vector<void *> blocks;
    ~Scratch()
    {
        for (void *p : blocks) cudaFree(p);
    }
    template <class U>
    cudaError_t get(U **p, size_t count)
    {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(U) * count);
        if (e == cudaSuccess) blocks.push_back(*p);
        return e;
    }
};

// The particles to bin: the caller's host arrays (copied to the device as FP64), or with
// n == 0 and no arrays the fit's own state and its current weights. kind: 0 = caller's
// (FP64), 1 = fit's FP64 state, 2 = fit's FP32 state.
struct Source {
    int kind = 0;
    Particles<double> d{};
    Particles<float> f{};
};

m2m_status source(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel, const double *w, Scratch &S,
                  Source &src)
{
    if (!ctx->sub.empty())
        return fail(ctx, M2M_ERR_STATE, "a batch context: per-fit calls take a fit handle from m2m_batch_model");
    if (n < 0) return fail(ctx, M2M_ERR_ARG, "n must be >= 0");
    if (n == 0 && !pos && !vel && !w) {
        if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
        m2m_status s = current_weights(ctx);
        if (s != M2M_OK) return s;
        if (ctx->precision == M2M_PREC_FP64) {
            src.kind = 1;
            const double *const *st = reinterpret_cast<const double *const *>(ctx->st);
            src.d = {st[0], st[1], st[2], st[3], st[4], st[5], ctx->d_wout, ctx->n};
        } else {
            src.kind = 2;
            const float *const *st = reinterpret_cast<const float *const *>(ctx->st);
            src.f = {st[0], st[1], st[2], st[3], st[4], st[5], ctx->d_wout, ctx->n};
        }
        return M2M_OK;
    }
    if (n > 0 && (!pos || !vel || !w))
        return fail(ctx, M2M_ERR_ARG, "pos, vel and w are required for n > 0 (or all NULL with n = 0)");
    double *d = nullptr;
    CU(S.get(&d, size_t(7) * size_t(n)));
    if (n > 0) {
        CU(cudaMemcpyAsync(d, pos, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(d + 3 * n, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
        CU(cudaMemcpyAsync(d + 6 * n, w, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    }
    src.kind = 0;
    src.d = {d, d + n, d + 2 * n, d + 3 * n, d + 4 * n, d + 5 * n, d + 6 * n, n};
    return M2M_OK;
}

int grid_of(const m2m_ctx *ctx, long long n)
{
    const long long want = (n + kDiagThreads - 1) / kDiagThreads;
    const long long cap = (long long)(ctx->nsm > 0 ? ctx->nsm : 1) * 8;
    return int(want < 1 ? 1 : (want < cap ? want : cap));
}

double pow2_floor(double x)
{
    int e;
    std::frexp(x, &e);  // x = f 2^e, f in [0.5, 1)
    return std::ldexp(1.0, e - 1);
}

// Scales that keep every bin sum of np particles below 2^62 in magnitude: |sum w| <=
// np max|w|, |sum w v| <= np max|w| max|v|, sum w v^2 <= np max|w| max v^2, sum of
// squared deviations <= np max|w|^2. Maxima, not sums, so the scales (and with them the
// results) do not depend on the order of the particles.
m2m_status diag_scales(m2m_ctx *ctx, const Source &src, long long np, Scratch &S, DiagScales &sc)
{
    unsigned long long *d_mx = nullptr;
    CU(S.get(&d_mx, 4));
    CU(cudaMemsetAsync(d_mx, 0, sizeof(unsigned long long) * 4, ctx->stream));
    unsigned *d_bad = reinterpret_cast<unsigned *>(d_mx + 2);
    if (np > 0) {
        if (src.kind == 2) k_diag_stats<float><<<grid_of(ctx, np), kDiagThreads, 0, ctx->stream>>>(src.f, d_mx, d_bad);
        else k_diag_stats<double><<<grid_of(ctx, np), kDiagThreads, 0, ctx->stream>>>(src.d, d_mx, d_bad);
        CU(cudaGetLastError());
    }
    unsigned long long h[3] = {0, 0, 0};
    CU(cudaMemcpyAsync(h, d_mx, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (h[2] & 0xFFFFFFFFull) return fail(ctx, M2M_ERR_ARG, "particles must be finite");
    double mw, mv2;
    std::memcpy(&mw, &h[0], sizeof mw);
    std::memcpy(&mv2, &h[1], sizeof mv2);
    const double two62 = 4611686018427387904.0, N = double(np > 0 ? np : 1);
    const double W = N * (mw > 0.0 ? mw : 1.0);
    const double v1 = mv2 > 1.0 ? std::sqrt(mv2) : 1.0, v2 = mv2 > 1.0 ? mv2 : 1.0;
    sc.w = pow2_floor(two62 / W);
    sc.wv = pow2_floor(two62 / (W * v1));
    sc.wv2 = pow2_floor(two62 / (W * v2));
    sc.dev = pow2_floor(two62 / (W * (mw > 0.0 ? mw : 1.0)));
    return M2M_OK;
}

}  // namespace

extern "C" m2m_status m2m_diag_kinematics(m2m_ctx *ctx, const m2m_sph_grid *grid, int64_t n, const double *pos,
                                          const double *vel, const double *w, double *sums, int64_t *counts,
                                          int64_t nbins)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!grid || !sums) return fail(ctx, M2M_ERR_ARG, "grid and sums are required");
    if (grid->n_r < 2 || grid->n_phi < 1 || grid->n_ct < 1 || !(grid->r_min > 0.0) ||
        !(grid->r_max > grid->r_min) || !std::isfinite(grid->r_max))
        return fail(ctx, M2M_ERR_ARG, "spherical grid needs n_r >= 2, n_phi, n_ct >= 1 and 0 < r_min < r_max");
    const long long nb = (long long)grid->n_r * grid->n_phi * grid->n_ct;
    if (nb > (1ll << 24)) return fail(ctx, M2M_ERR_ARG, "spherical grid has more than 2^24 bins");
    if (nbins != nb) return fail(ctx, M2M_ERR_ARG, "nbins must be n_r*n_phi*n_ct (%lld)", nb);
    Scratch S;
    Source src;
    m2m_status s = source(ctx, n, pos, vel, w, S, src);
    if (s != M2M_OK) return s;
    const long long np = src.kind == 2 ? src.f.n : src.d.n;
    DiagScales sc;
    s = diag_scales(ctx, src, np, S, sc);
    if (s != M2M_OK) return s;
    long long *d_sums = nullptr;
    unsigned long long *d_cnt = nullptr;
    CU(S.get(&d_sums, size_t(nb) * 2 * kKinSums));
    CU(S.get(&d_cnt, size_t(nb)));
    CU(cudaMemsetAsync(d_sums, 0, sizeof(long long) * nb * 2 * kKinSums, ctx->stream));
    CU(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * nb, ctx->stream));
    const SphBins g{grid->n_r, grid->n_phi, grid->n_ct, grid->r_min, grid->r_max, std::log(grid->r_min),
                    std::log(grid->r_max) - std::log(grid->r_min)};
    if (np > 0) {
        if (src.kind == 2) k_kin_sums<float><<<grid_of(ctx, np), kDiagThreads, 0, ctx->stream>>>(g, src.f, sc, d_sums, d_cnt);
        else k_kin_sums<double><<<grid_of(ctx, np), kDiagThreads, 0, ctx->stream>>>(g, src.d, sc, d_sums, d_cnt);
        CU(cudaGetLastError());
    }
    std::vector<long long> hs(size_t(nb) * 2 * kKinSums);
    CU(cudaMemcpyAsync(hs.data(), d_sums, sizeof(long long) * hs.size(), cudaMemcpyDeviceToHost, ctx->stream));
    if (counts)
        CU(cudaMemcpyAsync(counts, d_cnt, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    const double scl[kKinSums] = {sc.w, sc.wv, sc.wv, sc.wv, sc.wv2, sc.wv2, sc.wv2};
    for (long long b = 0; b < nb; ++b)
        for (int q = 0; q < kKinSums; ++q) sums[b * kKinSums + q] = fx_value(&hs[size_t(b * kKinSums + q) * 2], scl[q]);
    return src.kind == 0 ? M2M_OK : check_device_errors(ctx);
}

extern "C" m2m_status m2m_diag_grid(m2m_ctx *ctx, const m2m_prior_grid *grid, int64_t n, const double *pos,
                                    const double *vel, const double *w, double *wsum, double *wdev2,
                                    int64_t *counts, int32_t ncell)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!wsum) return fail(ctx, M2M_ERR_ARG, "wsum is required");
    if (!ctx->sub.empty())
        return fail(ctx, M2M_ERR_STATE, "a batch context: per-fit calls take a fit handle from m2m_batch_model");
    Model m = ctx->m;
    if (grid) {
        m2m_status gs = grid_fields(ctx, m, grid);
        if (gs != M2M_OK) return gs;
    } else if (m.mode != M2M_REG_MPR) {
        return fail(ctx, M2M_ERR_ARG, "a GWR fit has no (E, x) grid: pass one");
    }
    if (ncell != m.ncell) return fail(ctx, M2M_ERR_ARG, "ncell must be nE*nx (%d)", m.ncell);
    Scratch S;
    Source src;
    m2m_status s = source(ctx, n, pos, vel, w, S, src);
    if (s != M2M_OK) return s;
    const long long np = src.kind == 2 ? src.f.n : src.d.n;
    DiagScales sc;
    s = diag_scales(ctx, src, np, S, sc);
    if (s != M2M_OK) return s;
    long long *d_ws = nullptr, *d_wd = nullptr;
    unsigned long long *d_cnt = nullptr;
    int *d_cell = nullptr;
    CU(S.get(&d_ws, size_t(ncell) * 2));
    CU(S.get(&d_wd, size_t(ncell) * 2));
    CU(S.get(&d_cnt, size_t(ncell)));
    CU(S.get(&d_cell, size_t(np)));
    CU(cudaMemsetAsync(d_ws, 0, sizeof(long long) * 2 * ncell, ctx->stream));
    CU(cudaMemsetAsync(d_wd, 0, sizeof(long long) * 2 * ncell, ctx->stream));
    CU(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * ncell, ctx->stream));
    if (np > 0) {
        const Cst<double> kd = make_cst<double>(m);
        const int gr = grid_of(ctx, np);
        if (src.kind == 2) {
            k_grid_sums<float><<<gr, kDiagThreads, 0, ctx->stream>>>(m, kd, ctx->d_lcE, src.f, sc, d_cell, d_ws, d_cnt);
            k_grid_dev<<<gr, kDiagThreads, 0, ctx->stream>>>(np, d_cell, src.f.w, d_ws, d_cnt, sc, d_wd);
        } else {
            k_grid_sums<double><<<gr, kDiagThreads, 0, ctx->stream>>>(m, kd, ctx->d_lcE, src.d, sc, d_cell, d_ws, d_cnt);
            k_grid_dev<<<gr, kDiagThreads, 0, ctx->stream>>>(np, d_cell, src.d.w, d_ws, d_cnt, sc, d_wd);
        }
        CU(cudaGetLastError());
    }
    std::vector<long long> hw(size_t(ncell) * 2), hd(size_t(ncell) * 2);
    CU(cudaMemcpyAsync(hw.data(), d_ws, sizeof(long long) * hw.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaMemcpyAsync(hd.data(), d_wd, sizeof(long long) * hd.size(), cudaMemcpyDeviceToHost, ctx->stream));
    if (counts) CU(cudaMemcpyAsync(counts, d_cnt, sizeof(int64_t) * ncell, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < ncell; ++c) {
        wsum[c] = fx_value(&hw[size_t(c) * 2], sc.w);
        if (wdev2) wdev2[c] = fx_value(&hd[size_t(c) * 2], sc.dev);
    }
    return src.kind == 0 ? M2M_OK : check_device_errors(ctx);
}

// ------------------------------------------------------------------ host arithmetic

namespace {

// Mean velocity and dispersion of the three components of one bin; false if the bin has
// fewer than min_count particles or no mass.
bool moments(const double *o, int64_t count, int64_t min_count, double mean[3], double disp[3])
{
    if (count < min_count || count <= 0 || !(o[0] > 0.0)) return false;
    for (int c = 0; c < 3; ++c) {
        mean[c] = o[1 + c] / o[0];
        const double v2 = o[4 + c] / o[0] - mean[c] * mean[c];
        disp[c] = v2 > 0.0 ? std::sqrt(v2) : 0.0;
    }
    return true;
}

}  // namespace

extern "C" m2m_status m2m_kin_moments(int64_t nbins, const double *sums, const int64_t *counts, int64_t min_count,
                                      double *mean, double *disp, int32_t *valid)
{
    if (nbins < 0 || (nbins > 0 && (!sums || !counts || !mean || !disp)))
        return fail(nullptr, M2M_ERR_ARG, "m2m_kin_moments: null argument or nbins < 0");
    for (int64_t b = 0; b < nbins; ++b) {
        const bool ok = moments(sums + b * kKinSums, counts[b], min_count, mean + 3 * b, disp + 3 * b);
        if (!ok)
            for (int c = 0; c < 3; ++c) mean[3 * b + c] = disp[3 * b + c] = 0.0;
        if (valid) valid[b] = ok ? 1 : 0;
    }
    return M2M_OK;
}

extern "C" m2m_status m2m_delta_kin(int64_t nbins, const double *sums_model, const int64_t *counts_model,
                                    const double *sums_target, const int64_t *counts_target, int64_t min_count,
                                    double *out, int64_t *bins_used)
{
    if (nbins < 0 || !out || (nbins > 0 && (!sums_model || !counts_model || !sums_target || !counts_target)))
        return fail(nullptr, M2M_ERR_ARG, "m2m_delta_kin: null argument or nbins < 0");
    double acc[6] = {0, 0, 0, 0, 0, 0};
    int64_t used = 0;
    for (int64_t b = 0; b < nbins; ++b) {
        double mm[3], dm[3], mt[3], dt[3];
        if (!moments(sums_model + b * kKinSums, counts_model[b], min_count, mm, dm)) continue;
        if (!moments(sums_target + b * kKinSums, counts_target[b], min_count, mt, dt)) continue;
        for (int c = 0; c < 3; ++c) {
            acc[c] += (mm[c] - mt[c]) * (mm[c] - mt[c]);
            acc[3 + c] += (dm[c] - dt[c]) * (dm[c] - dt[c]);
        }
        ++used;
    }
    double all = 0.0;
    for (int q = 0; q < 6; ++q) {
        out[q] = used > 0 ? std::sqrt(acc[q] / double(used)) : 0.0;
        all += acc[q];
    }
    out[6] = used > 0 ? std::sqrt(all / (6.0 * double(used))) : 0.0;
    if (bins_used) *bins_used = used;
    return M2M_OK;
}

extern "C" m2m_status m2m_delta_grid(int32_t ncell, const double *w_model, const double *w_target, double *delta)
{
    if (ncell < 0 || !delta || (ncell > 0 && (!w_model || !w_target)))
        return fail(nullptr, M2M_ERR_ARG, "m2m_delta_grid: null argument or ncell < 0");
    double tm = 0.0, tt = 0.0;
    for (int c = 0; c < ncell; ++c) {
        tm += w_model[c];
        tt += w_target[c];
    }
    *delta = 0.0;
    if (!(tm > 0.0) || !(tt > 0.0)) return M2M_OK;
    double num = 0.0, den = 0.0;
    for (int c = 0; c < ncell; ++c) {
        const double wt = w_target[c] / tt;
        if (!(wt > 0.0)) continue;
        const double r = (wt - w_model[c] / tm) / wt;
        num += wt * r * r;
        den += wt;
    }
    *delta = std::sqrt(num / den);
    return M2M_OK;
}

extern "C" m2m_status m2m_weight_rms(int32_t ncell, const double *wdev2, const int64_t *counts, int64_t min_count,
                                     double *rms)
{
    if (ncell < 0 || !rms || (ncell > 0 && (!wdev2 || !counts)))
        return fail(nullptr, M2M_ERR_ARG, "m2m_weight_rms: null argument or ncell < 0");
    double s = 0.0;
    int64_t n = 0;
    for (int c = 0; c < ncell; ++c) {
        if (counts[c] <= min_count) continue;
        s += wdev2[c];
        n += counts[c];
    }
    *rms = n > 0 ? std::sqrt(s / double(n)) : 0.0;
    return M2M_OK;
}
