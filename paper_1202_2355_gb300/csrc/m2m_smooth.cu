// Smoothing of the grid of priors (Sec. 2.3.2, eq. smooth_grid) on the device.
//
// At a prior update the finalize leaves the raw cell means y (n = nE*nx cells). The
// priors are then the penalised least-squares fit f = (I + lambda P)^-1 y, where
// f.P.f = sum (f_EE^2 + 2 f_Ex^2 + f_xx^2) with second differences in bin units (f_EE,
// f_xx over the interior cells, f_Ex at the cell corners), and lambda is either fixed or
// chosen by generalized cross validation: the minimum of
// V(lambda) = n |(I - A) y|^2 / tr(I - A)^2, A = (I + lambda P)^-1, found by a
// golden-section search over log10 lambda in [-4, 6] (48 steps, a bracket of 1e-9
// decades; lambda is the middle of the last bracket). Where the minimum is flat to
// rounding any lambda in it is an equally good choice; 48 steps also bring a minimum at
// an end of the range to within 1e-9 decades of it.
//
// P depends on the grid shape only, so the host diagonalises it once per shape,
// P = V D V^T (Householder reduction to tridiagonal form, then implicit symmetric QR
// steps with Wilkinson shifts; Golub & Van Loan, Matrix Computations, Sec. 8.3). Then
//   f = V diag(1 / (1 + lambda d_k)) V^T y,
//   |(I - A) y|^2 = sum_k (lambda d_k / (1 + lambda d_k))^2 z_k^2,  z = V^T y,
//   tr(I - A) = sum_k lambda d_k / (1 + lambda d_k),
// so every GCV evaluation is O(n). Two kernels run after each step kernel and return at
// once unless the step updated the priors: k_smooth_a forms z with many blocks (partial
// sums over row chunks, added in a fixed order), its last block runs the search and
// forms s = z / (1 + lambda d); k_smooth_b forms f = V s the same way and writes the
// priors (cells whose fitted prior is <= 0 get no entropy force).
#include "m2m_ctx.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

using namespace m2m;

namespace {

constexpr int kSmoothThreads = 256;

// ------------------------------------------------------------------ host: penalty

// Dense penalty of the grid (row-major n x n) from its difference stencils.
std::vector<double> penalty(int nE, int nx)
{
    const int n = nE * nx;
    std::vector<double> P(size_t(n) * n, 0.0);
    auto add = [&](std::initializer_list<std::pair<int, double>> row, double w) {
        for (const auto &a : row)
            for (const auto &b : row) P[size_t(a.first) * n + b.first] += w * a.second * b.second;
    };
    for (int k = 1; k + 1 < nE; ++k)  // second difference along E
        for (int l = 0; l < nx; ++l)
            add({{(k - 1) * nx + l, 1.0}, {k * nx + l, -2.0}, {(k + 1) * nx + l, 1.0}}, 1.0);
    for (int k = 0; k < nE; ++k)  // along x
        for (int l = 1; l + 1 < nx; ++l)
            add({{k * nx + l - 1, 1.0}, {k * nx + l, -2.0}, {k * nx + l + 1, 1.0}}, 1.0);
    for (int k = 0; k + 1 < nE; ++k)  // mixed, at the cell corners, weighted 2
        for (int l = 0; l + 1 < nx; ++l)
            add({{(k + 1) * nx + l + 1, 1.0}, {(k + 1) * nx + l, -1.0}, {k * nx + l + 1, -1.0}, {k * nx + l, 1.0}},
                2.0);
    return P;
}

// ------------------------------------------------------------------ host: eigensolver

// Householder reduction of the symmetric A (row-major, destroyed) to tridiagonal form:
// A = Q T Q^T with T = tridiag(e, d, e), d the diagonal and e[i] the (i+1, i) entry.
// QT = Q^T is accumulated (row operations on contiguous rows).
void tridiagonalise(int n, std::vector<double> &A, std::vector<double> &QT, std::vector<double> &d,
                    std::vector<double> &e)
{
    QT.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; ++i) QT[size_t(i) * n + i] = 1.0;
    std::vector<double> v(n), p(n), w(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int m0 = k + 1;
        double xn = 0.0;
        for (int i = m0; i < n; ++i) xn += A[size_t(i) * n + k] * A[size_t(i) * n + k];
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        const double x0 = A[size_t(m0) * n + k];
        const double alpha = x0 > 0.0 ? -xn : xn;  // reflect x onto alpha e1, no cancellation
        for (int i = m0; i < n; ++i) v[i] = A[size_t(i) * n + k];
        v[m0] = x0 - alpha;
        double vv = 0.0;
        for (int i = m0; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        // H B H with B the trailing block, H = I - beta v v^T: B - v q^T - q v^T,
        // p = beta B v, K = beta (v.p) / 2, q = p - K v
        for (int i = m0; i < n; ++i) {
            double s = 0.0;
            const double *row = &A[size_t(i) * n];
            for (int j = m0; j < n; ++j) s += row[j] * v[j];
            p[i] = beta * s;
        }
        double vp = 0.0;
        for (int i = m0; i < n; ++i) vp += v[i] * p[i];
        const double K = 0.5 * beta * vp;
        for (int i = m0; i < n; ++i) p[i] -= K * v[i];  // p now holds q
        for (int i = m0; i < n; ++i) {
            double *row = &A[size_t(i) * n];
            for (int j = m0; j < n; ++j) row[j] -= v[i] * p[j] + p[i] * v[j];
        }
        A[size_t(m0) * n + k] = A[size_t(k) * n + m0] = alpha;
        for (int i = m0 + 1; i < n; ++i) A[size_t(i) * n + k] = A[size_t(k) * n + i] = 0.0;
        // Q <- Q H, i.e. QT <- H QT = QT - beta v (v^T QT) on rows m0..n-1
        std::fill(w.begin(), w.end(), 0.0);
        for (int j = m0; j < n; ++j) {
            const double *row = &QT[size_t(j) * n];
            const double vj = v[j];
            for (int c = 0; c < n; ++c) w[c] += vj * row[c];
        }
        for (int j = m0; j < n; ++j) {
            double *row = &QT[size_t(j) * n];
            const double f = beta * v[j];
            for (int c = 0; c < n; ++c) row[c] -= f * w[c];
        }
    }
    d.resize(n);
    e.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = A[size_t(i) * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[size_t(i + 1) * n + i];
}

// Implicit symmetric QR steps with Wilkinson shifts on tridiag(e, d, e), the Givens
// rotations accumulated into QT = Q^T (rows k, k+1). Returns false if a block fails to
// converge.
bool tridiagonal_qr(int n, std::vector<double> &d, std::vector<double> &e, std::vector<double> &QT)
{
    const double eps = 2.220446049250313e-16;
    int hi = n - 1, iter = 0;
    while (hi > 0) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            iter = 0;
            continue;
        }
        if (++iter > 60) return false;
        int lo = hi - 1;
        while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
        // shift: the eigenvalue of the trailing 2 x 2 block closer to its last diagonal entry
        const double dd = 0.5 * (d[hi - 1] - d[hi]), ee = e[hi - 1];
        const double mu = d[hi] - ee * ee / (dd + std::copysign(std::hypot(dd, ee), dd));
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = std::hypot(x, z);
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : z / r;
            if (k > lo) e[k - 1] = r;  // the bulge from the previous rotation is folded in
            const double a = d[k], b = e[k], dk1 = d[k + 1];
            d[k] = c * c * a + 2.0 * c * s * b + s * s * dk1;
            d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * dk1;
            e[k] = c * s * (dk1 - a) + (c * c - s * s) * b;
            if (k + 1 < hi) {
                x = e[k];
                z = s * e[k + 1];  // new bulge at (k+2, k)
                e[k + 1] *= c;
            }
            double *rk = &QT[size_t(k) * n], *rk1 = &QT[size_t(k + 1) * n];
            for (int j = 0; j < n; ++j) {
                const double a0 = rk[j], a1 = rk1[j];
                rk[j] = c * a0 + s * a1;
                rk1[j] = -s * a0 + c * a1;
            }
        }
    }
    return true;
}

struct Eigen {
    std::vector<double> V, VT, D;  // P = V diag(D) V^T; V row-major (cell, mode), VT = V^T
};

std::mutex g_eig_mu;
std::map<std::pair<int, int>, std::shared_ptr<const Eigen>> g_eig;

std::shared_ptr<const Eigen> eigen_of_grid(int nE, int nx)
{
    std::lock_guard<std::mutex> lock(g_eig_mu);
    auto it = g_eig.find({nE, nx});
    if (it != g_eig.end()) return it->second;
    const int n = nE * nx;
    std::vector<double> A = penalty(nE, nx), QT, d, e;
    tridiagonalise(n, A, QT, d, e);
    if (!tridiagonal_qr(n, d, e, QT)) return nullptr;
    auto E = std::make_shared<Eigen>();
    E->VT = QT;
    E->D = d;
    E->V.resize(size_t(n) * n);
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < n; ++i) E->V[size_t(i) * n + k] = QT[size_t(k) * n + i];
    g_eig[{nE, nx}] = E;
    return E;
}

// ------------------------------------------------------------------ device

__device__ double block_sum(double v, double *red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// GCV score at t = log10 lambda from z = V^T y and the eigenvalues D.
__device__ double gcv_score(double t, int n, const double *z, const double *D, double *red)
{
    const double lam = pow(10.0, t);
    double rss = 0.0, tr = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double q = lam * D[k] / (1.0 + lam * D[k]);
        rss += q * q * z[k] * z[k];
        tr += q;
    }
    rss = block_sum(rss, red);
    tr = block_sum(tr, red);
    return double(n) * rss / (tr * tr);
}

// Chunked product out_part[ch][r] = sum_{c in chunk ch} M[c][r] x[c] (M row-major n x n,
// coalesced over r); returns true in the last block to finish, which then holds all parts.
__device__ bool chunked_product(int n, const double *M, const double *x, double *part, unsigned *counter)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int cs = (n + gridDim.y - 1) / gridDim.y;
    const int c0 = blockIdx.y * cs, c1 = min(n, c0 + cs);
    if (r < n) {
        double acc = 0.0;
        for (int c = c0; c < c1; ++c) acc += M[size_t(c) * n + r] * __ldcg(x + c);
        part[size_t(blockIdx.y) * n + r] = acc;
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__global__ void __launch_bounds__(kSmoothThreads) k_smooth_a(const Model m, const Buffers b)
{
    Scalars &sc = *b.sc;
    if (!*reinterpret_cast<volatile int *>(&sc.smooth_pending)) return;
    const int n = m.ncell;
    if (!chunked_product(n, b.sV, b.prior_raw, b.spart, &sc.smooth_blocks)) return;
    __shared__ double red[kSmoothThreads];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double z = 0.0;
        for (int ch = 0; ch < int(gridDim.y); ++ch) z += __ldcg(b.spart + size_t(ch) * n + k);
        b.sz[k] = z;
    }
    __syncthreads();
    double lam = m.smooth_lambda;
    if (!(lam > 0.0)) {
        const double g = 0.5 * (sqrt(5.0) - 1.0);
        double a = -4.0, bb = 6.0;
        double c = bb - g * (bb - a), d = a + g * (bb - a);
        double vc = gcv_score(c, n, b.sz, b.sD, red), vd = gcv_score(d, n, b.sz, b.sD, red);
        for (int it = 0; it < 48; ++it) {
            if (vc <= vd) {
                bb = d;
                d = c;
                vd = vc;
                c = bb - g * (bb - a);
                vc = gcv_score(c, n, b.sz, b.sD, red);
            } else {
                a = c;
                c = d;
                vc = vd;
                d = a + g * (bb - a);
                vd = gcv_score(d, n, b.sz, b.sD, red);
            }
        }
        lam = pow(10.0, 0.5 * (a + bb));
    }
    for (int k = threadIdx.x; k < n; k += blockDim.x) b.ss[k] = b.sz[k] / (1.0 + lam * b.sD[k]);
    if (threadIdx.x == 0) {
        sc.smooth_lambda = lam;
        sc.smooth_blocks = 0;
    }
}

__global__ void __launch_bounds__(kSmoothThreads) k_smooth_b(const Model m, const Buffers b)
{
    Scalars &sc = *b.sc;
    if (!*reinterpret_cast<volatile int *>(&sc.smooth_pending)) return;
    const int n = m.ncell;
    if (!chunked_product(n, b.sVT, b.ss, b.spart, &sc.smooth_blocks)) return;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double f = 0.0;
        for (int ch = 0; ch < int(gridDim.y); ++ch) f += __ldcg(b.spart + size_t(ch) * n + c);
        b.prior[c] = f;
        b.iprior[c] = f > 0.0 ? 1.0 / f : 0.0;
        b.lprior[c] = f > 0.0 ? log(f) : -HUGE_VAL;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sc.smooth_blocks = 0;
        sc.smooth_pending = 0;
    }
}

}  // namespace

// Allocates the smoothing tables of a context with prior smoothing on.
m2m_status smooth_setup(m2m_ctx *ctx)
{
    const Model &m = ctx->m;
    if (!m.smooth) return M2M_OK;
    if (m.mode != 1 || m.nE < 3 || m.nx < 3)
        return fail(ctx, M2M_ERR_ARG, "prior smoothing needs the MPR grid with nE, nx >= 3");
    std::shared_ptr<const Eigen> E = eigen_of_grid(m.nE, m.nx);
    if (!E) return fail(ctx, M2M_ERR_ARG, "eigendecomposition of the %d x %d grid penalty failed", m.nE, m.nx);
    const int n = m.ncell;
    ctx->smooth_ch = std::max(1, std::min(n, (4 * ctx->nsm) / ((n + kSmoothThreads - 1) / kSmoothThreads)));
    CU(cudaMalloc(&ctx->d_sV, sizeof(double) * size_t(n) * n));
    CU(cudaMalloc(&ctx->d_sVT, sizeof(double) * size_t(n) * n));
    CU(cudaMalloc(&ctx->d_sD, sizeof(double) * n));
    CU(cudaMalloc(&ctx->d_spart, sizeof(double) * size_t(ctx->smooth_ch) * n));
    CU(cudaMalloc(&ctx->d_sz, sizeof(double) * n));
    CU(cudaMalloc(&ctx->d_ss, sizeof(double) * n));
    CU(cudaMalloc(&ctx->d_prior_raw, sizeof(double) * (n + 1)));
    CU(cudaMemcpy(ctx->d_sV, E->V.data(), sizeof(double) * size_t(n) * n, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_sVT, E->VT.data(), sizeof(double) * size_t(n) * n, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->d_sD, E->D.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CU(cudaMemset(ctx->d_prior_raw, 0, sizeof(double) * (n + 1)));
    return M2M_OK;
}

void smooth_free(m2m_ctx *ctx)
{
    free_dev(ctx->d_sV);
    free_dev(ctx->d_sVT);
    free_dev(ctx->d_sD);
    free_dev(ctx->d_spart);
    free_dev(ctx->d_sz);
    free_dev(ctx->d_ss);
    free_dev(ctx->d_prior_raw);
}

// The two smoothing kernels after a step kernel (both return at once on steps that did
// not update the priors).
void smooth_launch(m2m_ctx *ctx)
{
    if (!ctx->m.smooth) return;
    const Buffers b = buffers(ctx);
    const dim3 grid((ctx->m.ncell + kSmoothThreads - 1) / kSmoothThreads, ctx->smooth_ch);
    k_smooth_a<<<grid, kSmoothThreads, 0, ctx->stream>>>(ctx->m, b);
    k_smooth_b<<<grid, kSmoothThreads, 0, ctx->stream>>>(ctx->m, b);
}
