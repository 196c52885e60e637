// Batches of independent fits: m2m_create_batch and the batched step.
//
// A batch owns one complete fit context per model (its own potential,
// observables, targets, priors, particles and sums), so every per-fit call works
// on the handle m2m_batch_model returns. m2m_step on the batch advances every fit
// by one launch of k_step_batch per step: the fits' particles, taken in model
// order, are cut into one equal contiguous share per resident block, each share
// into segments (model, begin, end) of at most a set number of particles; a block
// walks its segments and the block that flushes a model's last segment runs that
// model's finalize. Launches are captured in a CUDA graph. The sums are exact
// integers, so neither batching nor the launch shape (threads per block, blocks,
// segment length) changes any result; m2m_batch_autotune times the shapes on real
// steps and keeps the fastest.
#include "m2m_ctx.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

using namespace m2m;

struct BatchState {
    int block = 256, bps = 0, grid = 0, nsm = 0, maxsm = 0;
    long long seg_cap = kMaxParticlesPerBlock;
    size_t smem = 0;
    void *kernel = nullptr;  // the k_step_batch instantiation for the fits' observable shape
    bool bank = false;       // the kernel reads the fits' constants from its parameter bank
    std::vector<unsigned char> h_bank;  // BatchBank<T> passed at every launch
    Model *d_models = nullptr;
    void *d_csts = nullptr, *d_states = nullptr;
    Buffers *d_bufs = nullptr;
    Segment *d_seg = nullptr;
    int *d_seg_off = nullptr;
    unsigned *d_nseg = nullptr;
    Scalars **d_scs = nullptr;    // the fits' scalars, for m2m_batch_get_chi2
    double *d_chi2 = nullptr;     // per fit: chi^2 and the error word (as a double)
    std::vector<long long> gens;  // the fits' load generations the arrays were built for
    bool ready = false;
    cudaGraphExec_t graph = nullptr;
    long long nseg_total = 0;
};

static const int kBatchGraphSteps = 16;

// ------------------------------------------------------------------ kernel choice

template <class T, int WPS, unsigned M0, unsigned M1, unsigned M2, unsigned M3>
static void *batch_fn(bool bank)
{
    if (bank) return reinterpret_cast<void *>(k_step_batch<T, WPS, kMinBlocksBatch<T>, true, M0, M1, M2, M3>);
    return reinterpret_cast<void *>(k_step_batch<T, WPS, kMinBlocksBatch<T>, false, M0, M1, M2, M3>);
}

template <class T>
using BatchFn = void (*)(const BatchArgs<T>, const BatchBank<T>);

static bool group_hot_equal(const GroupDesc &a, const GroupDesc &b)
{
    bool eq = a.geometry == b.geometry && a.n_ap == b.n_ap && a.n_kinds == b.n_kinds && a.obs_off == b.obs_off &&
              a.ap_off == b.ap_off && a.edge_off == b.edge_off && a.max_gh == b.max_gh && a.has_v2 == b.has_v2 &&
              a.nx == b.nx && a.ny == b.ny && a.xlo == b.xlo && a.ylo == b.ylo && a.xw == b.xw && a.yw == b.yw &&
              a.xlo_f == b.xlo_f && a.ylo_f == b.ylo_f && a.ixw == b.ixw && a.iyw == b.iyw && a.lut_off == b.lut_off &&
              a.lut_n == b.lut_n && a.l0 == b.l0 && a.lscale == b.lscale && a.e0sq_f == b.e0sq_f &&
              a.ensq_f == b.ensq_f && a.lut_identity == b.lut_identity && a.k_mass == b.k_mass && a.k_v2 == b.k_v2 &&
              a.k_v1 == b.k_v1;
    for (int n = 0; eq && n < 7; ++n) eq = a.k_gh[n] == b.k_gh[n];
    for (int q = 0; eq && q < a.n_kinds; ++q)
        eq = a.kinds[q] == b.kinds[q] && a.alm_l[q] == b.alm_l[q] && a.alm_m[q] == b.alm_m[q] &&
             a.alm_norm[q] == b.alm_norm[q] && a.alm_norm_f[q] == b.alm_norm_f[q];
    return eq;
}

// Whether two fits agree in every Model field that the per-particle path reads (the
// fields step_particles takes from its shape Model); the rest differ freely.
static bool hot_equal(const Model &a, const Model &b)
{
    bool eq = a.pot == b.pot && a.mode == b.mode && a.update_rule == b.update_rule && a.ap_cache == b.ap_cache &&
              a.cache_accel == b.cache_accel && a.gx_group == b.gx_group && a.J == b.J && a.nslots == b.nslots &&
              a.off_count == b.off_count && a.rec_len == b.rec_len && a.n_groups == b.n_groups &&
              a.win_group == b.win_group && a.win_lo == b.win_lo && a.win_n == b.win_n && a.n_dups == b.n_dups &&
              a.off_dups == b.off_dups;
    for (int g = 0; eq && g < a.n_groups; ++g) eq = group_hot_equal(a.g[g], b.g[g]);
    return eq;
}

// The specialised kernel when every fit has the same observable shape and it is
// one of the compiled ones, else the generic one; from the parameter bank when the
// fits fit in it and share the per-particle fields.
template <class T, int WPS>
static void *batch_pick(const std::vector<m2m_ctx *> &sub, bool &bank)
{
    bank = int(sub.size()) <= kBankFits<T>;
    for (const m2m_ctx *c : sub) bank = bank && hot_equal(sub[0]->m, c->m);
    const Model &m0 = sub[0]->m;
    unsigned mk[4] = {0, 0, 0, 0};
    for (int g = 0; g < m0.n_groups; ++g) mk[g] = group_mask(m0.g[g]);
    bool same = true;
    for (const m2m_ctx *c : sub) {
        if (c->m.n_groups != m0.n_groups) same = false;
        for (int g = 0; same && g < m0.n_groups; ++g)
            if (group_mask(c->m.g[g]) != mk[g]) same = false;
    }
    constexpr unsigned kin1 = kBitV2 | bit_gh(4), kin2 = kBitV2 | bit_gh(3) | bit_gh(4);
    constexpr unsigned map = kBitPix | kBitMass | bit_gh(1) | bit_gh(2) | bit_gh(3) | bit_gh(4);
    if (same && m0.n_groups == 2 && mk[0] == kBitMass && mk[1] == kin1)
        return batch_fn<T, WPS, kBitMass, kin1, 0u, 0u>(bank);
    if (same && m0.n_groups == 2 && mk[0] == kBitMass && mk[1] == kin2)
        return batch_fn<T, WPS, kBitMass, kin2, 0u, 0u>(bank);
    if (same && m0.n_groups == 1 && mk[0] == map) return batch_fn<T, WPS, map, 0u, 0u, 0u>(bank);
    return batch_fn<T, WPS, kDyn, kDyn, kDyn, kDyn>(bank);
}

// ------------------------------------------------------------------ segments

// Cuts the fits' particles (counts n, in model order) into `grid` equal contiguous
// shares and each share into segments of at most `cap` particles that do not cross
// a model boundary. A fit without particles gets one empty segment, so that its
// finalize still runs. nseg: segments per model.
static void build_segments(const std::vector<long long> &n, int grid, long long cap, std::vector<Segment> &seg,
                           std::vector<int> &off, std::vector<unsigned> &nseg)
{
    const int M = int(n.size());
    std::vector<long long> start(M + 1, 0);
    for (int m = 0; m < M; ++m) start[m + 1] = start[m] + n[m];
    const long long total = start[M];
    const long long share = total > 0 ? (total + grid - 1) / grid : 0;
    std::vector<std::vector<Segment>> per(grid);
    nseg.assign(M, 0);
    for (int b = 0; b < grid && share > 0; ++b) {
        long long lo = b * share;
        const long long hi = std::min(lo + share, total);
        while (lo < hi) {
            const int m = int(std::upper_bound(start.begin(), start.end(), lo) - start.begin()) - 1;
            const long long e = std::min(hi, start[m + 1]);
            for (long long a = lo; a < e; a += cap) {
                Segment s;
                s.model = m;
                s.pad = 0;
                s.begin = a - start[m];
                s.end = std::min(a + cap, e) - start[m];
                per[b].push_back(s);
                ++nseg[m];
            }
            lo = e;
        }
    }
    for (int m = 0; m < M; ++m)
        if (n[m] == 0) {
            per[m % grid].push_back(Segment{m, 0, 0, 0});
            ++nseg[m];
        }
    seg.clear();
    off.assign(grid + 1, 0);
    for (int b = 0; b < grid; ++b) {
        off[b] = int(seg.size());
        seg.insert(seg.end(), per[b].begin(), per[b].end());
    }
    off[grid] = int(seg.size());
}

// ------------------------------------------------------------------ device arrays

static void free_arrays(BatchState &B)
{
    free_dev(B.d_models);
    free_dev(B.d_csts);
    free_dev(B.d_states);
    free_dev(B.d_bufs);
    free_dev(B.d_seg);
    free_dev(B.d_seg_off);
    free_dev(B.d_nseg);
    free_dev(B.d_scs);
    free_dev(B.d_chi2);
    if (B.graph) cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
    B.ready = false;
}

template <class T>
static m2m_status upload(m2m_ctx *ctx, T *&d, const void *h, size_t bytes)
{
    free_dev(d);
    CU(cudaMalloc(&d, bytes > 0 ? bytes : 1));
    if (bytes) CU(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice));
    return M2M_OK;
}

// Builds the per-fit descriptor arrays and the segment list, unless they are
// current (no fit was reloaded and the launch shape is unchanged).
template <class T>
static m2m_status batch_prepare(m2m_ctx *ctx)
{
    BatchState &B = *ctx->bs;
    const int M = int(ctx->sub.size());
    std::vector<long long> gens(M), n(M);
    for (int i = 0; i < M; ++i) {
        m2m_ctx *c = ctx->sub[i];
        if (!c->loaded) return fail(ctx, M2M_ERR_STATE, "fit %d has no particles loaded", i);
        gens[i] = c->load_gen;
        n[i] = c->n;
    }
    if (B.ready && gens == B.gens) return M2M_OK;
    CU(cudaStreamSynchronize(ctx->stream));
    free_arrays(B);
    std::vector<Model> models(M);
    std::vector<Cst<T>> csts(M);
    std::vector<State<T>> states(M);
    std::vector<Buffers> bufs(M);
    for (int i = 0; i < M; ++i) {
        m2m_ctx *c = ctx->sub[i];
        models[i] = c->m;
        csts[i] = make_cst<T>(c->m);
        states[i] = state<T>(c);
        bufs[i] = buffers(c);
    }
    std::vector<Segment> seg;
    std::vector<int> off;
    std::vector<unsigned> nseg;
    build_segments(n, B.grid, B.seg_cap, seg, off, nseg);
    m2m_status s;
    if ((s = upload(ctx, B.d_models, models.data(), sizeof(Model) * M)) != M2M_OK) return s;
    if ((s = upload(ctx, B.d_csts, csts.data(), sizeof(Cst<T>) * M)) != M2M_OK) return s;
    B.h_bank.assign(sizeof(BatchBank<T>), 0);
    if (B.bank) {
        BatchBank<T> *bk = reinterpret_cast<BatchBank<T> *>(B.h_bank.data());
        bk->shape = models[0];
        for (int i = 0; i < M; ++i) bk->cst[i] = csts[i];
    }
    if ((s = upload(ctx, B.d_states, states.data(), sizeof(State<T>) * M)) != M2M_OK) return s;
    if ((s = upload(ctx, B.d_bufs, bufs.data(), sizeof(Buffers) * M)) != M2M_OK) return s;
    if ((s = upload(ctx, B.d_seg, seg.data(), sizeof(Segment) * seg.size())) != M2M_OK) return s;
    if ((s = upload(ctx, B.d_seg_off, off.data(), sizeof(int) * off.size())) != M2M_OK) return s;
    if ((s = upload(ctx, B.d_nseg, nseg.data(), sizeof(unsigned) * nseg.size())) != M2M_OK) return s;
    std::vector<Scalars *> scs(M);
    for (int i = 0; i < M; ++i) scs[i] = ctx->sub[i]->d_sc;
    if ((s = upload(ctx, B.d_scs, scs.data(), sizeof(Scalars *) * M)) != M2M_OK) return s;
    CU(cudaMalloc(&B.d_chi2, sizeof(double) * 2 * M));
    B.nseg_total = (long long)seg.size();
    B.gens = gens;
    B.ready = true;
    return M2M_OK;
}

template <class T>
static void batch_launch(m2m_ctx *ctx)
{
    const BatchState &B = *ctx->bs;
    BatchArgs<T> a;
    a.models = B.d_models;
    a.csts = static_cast<const Cst<T> *>(B.d_csts);
    a.states = static_cast<const State<T> *>(B.d_states);
    a.bufs = B.d_bufs;
    a.seg = B.d_seg;
    a.seg_off = B.d_seg_off;
    a.nseg = B.d_nseg;
    const BatchBank<T> &bank = *reinterpret_cast<const BatchBank<T> *>(B.h_bank.data());
    reinterpret_cast<BatchFn<T>>(B.kernel)<<<B.grid, B.block, B.smem, ctx->stream>>>(a, bank);
}

static m2m_status prepare(m2m_ctx *ctx)
{
    return ctx->precision == M2M_PREC_FP64 ? batch_prepare<double>(ctx) : batch_prepare<float>(ctx);
}

static void launch(m2m_ctx *ctx)
{
    if (ctx->precision == M2M_PREC_FP64) batch_launch<double>(ctx);
    else batch_launch<float>(ctx);
}

// ------------------------------------------------------------------ stepping

m2m_status batch_step(m2m_ctx *ctx, int64_t nsteps)
{
    if (nsteps < 0) return fail(ctx, M2M_ERR_ARG, "nsteps must be >= 0");
    m2m_status s = prepare(ctx);
    if (s != M2M_OK) return s;
    BatchState &B = *ctx->bs;
    if (ctx->timing) {
        for (int64_t k = 0; k < nsteps; ++k) {
            while (ctx->events.size() < 2 * (ctx->timed + 1)) {
                cudaEvent_t e;
                CU(cudaEventCreate(&e));
                ctx->events.push_back(e);
            }
            cudaEvent_t *ev = &ctx->events[2 * ctx->timed];
            cudaEventRecord(ev[0], ctx->stream);
            launch(ctx);
            cudaEventRecord(ev[1], ctx->stream);
            ++ctx->timed;
        }
        CU(cudaGetLastError());
        return M2M_OK;
    }
    int64_t left = nsteps;
    if (left >= kBatchGraphSteps && !B.graph) {
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kBatchGraphSteps; ++k) launch(ctx);
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        if (e != cudaSuccess) return fail(ctx, M2M_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&B.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            B.graph = nullptr;
            return fail(ctx, M2M_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    while (left >= kBatchGraphSteps) {
        CU(cudaGraphLaunch(B.graph, ctx->stream));
        left -= kBatchGraphSteps;
    }
    for (; left > 0; --left) launch(ctx);
    CU(cudaGetLastError());
    return M2M_OK;
}

m2m_status batch_synchronize(m2m_ctx *ctx)
{
    CU(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < ctx->sub.size(); ++i) {
        m2m_ctx *c = ctx->sub[i];
        if (!c->loaded) continue;
        const m2m_status s = check_device_errors(c);
        if (s != M2M_OK) return fail(ctx, s, "fit %zu: %s", i, c->err.c_str());
    }
    return M2M_OK;
}

// chi^2 and the error word of every fit, gathered for one copy to the host.
static __global__ void k_batch_chi2(Scalars *const *scs, double *out, int M)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        out[2 * i] = scs[i]->chi2;
        out[2 * i + 1] = double(scs[i]->err);
    }
}

extern "C" m2m_status m2m_batch_get_chi2(m2m_ctx *ctx, double *chi2, int32_t nmodels)
{
    if (!ctx) return M2M_ERR_ARG;
    if (ctx->sub.empty()) return fail(ctx, M2M_ERR_STATE, "not a batch context");
    const int M = int(ctx->sub.size());
    if (nmodels != M || !chi2) return fail(ctx, M2M_ERR_ARG, "chi2 must hold the batch's %d values", M);
    m2m_status s = prepare(ctx);
    if (s != M2M_OK) return s;
    BatchState &B = *ctx->bs;
    std::vector<double> h(2 * size_t(M));
    k_batch_chi2<<<(M + 127) / 128, 128, 0, ctx->stream>>>(B.d_scs, B.d_chi2, M);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(h.data(), B.d_chi2, sizeof(double) * 2 * M, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < M; ++i) {
        chi2[i] = h[2 * i];
        if (h[2 * i + 1] != 0.0) {  // the fit's own check decodes the error word
            s = check_device_errors(ctx->sub[i]);
            if (s != M2M_OK) return fail(ctx, s, "fit %d: %s", i, ctx->sub[i]->err.c_str());
        }
    }
    return M2M_OK;
}

void batch_destroy(m2m_ctx *ctx)
{
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->bs) {
        free_arrays(*ctx->bs);
        delete ctx->bs;
        ctx->bs = nullptr;
    }
    for (m2m_ctx *c : ctx->sub) destroy_impl(c);
    ctx->sub.clear();
}

// ------------------------------------------------------------------ creation

template <class T, int WPS>
static m2m_status batch_configure(m2m_ctx *ctx, const m2m_options *opt)
{
    BatchState &B = *ctx->bs;
    B.kernel = batch_pick<T, WPS>(ctx->sub, B.bank);
    size_t smem = size_t(256) * sizeof(double);  // the finalize's block reduction
    for (const m2m_ctx *c : ctx->sub) smem = std::max(smem, smem_bytes<T>(c->m, 1, 1));
    CU(cudaDeviceGetAttribute(&B.maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    CU(cudaDeviceGetAttribute(&B.nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    if (smem > size_t(B.maxsm))
        return fail(ctx, M2M_ERR_ARG, "the largest fit needs %zu B of shared memory (limit %d)", smem, B.maxsm);
    B.smem = smem;
    using Fn = BatchFn<T>;
    CU(cudaFuncSetAttribute(reinterpret_cast<Fn>(B.kernel), cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    B.block = opt->block > 0 ? opt->block : 256;
    if (B.block % 32 != 0 || B.block > 256) return fail(ctx, M2M_ERR_ARG, "block must be a multiple of 32, <= 256");
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<Fn>(B.kernel), B.block, smem));
    if (occ < 1) return fail(ctx, M2M_ERR_ARG, "batched step kernel cannot be resident with block %d", B.block);
    B.bps = (opt->blocks_per_sm > 0 && opt->blocks_per_sm < occ) ? opt->blocks_per_sm : occ;
    B.grid = B.nsm * B.bps;
    return M2M_OK;
}

extern "C" m2m_status m2m_create_batch(int32_t nmodels, const m2m_potential *pots, const m2m_observables *obs,
                                       const m2m_prior_grid *priors, const double *eps, const double *mu,
                                       const double *alpha, const m2m_options *opt, m2m_ctx **out)
{
    if (!out) return fail(nullptr, M2M_ERR_ARG, "out is null");
    *out = nullptr;
    if (nmodels < 1 || !pots || !obs || !priors || !eps || !mu || !alpha || !opt)
        return fail(nullptr, M2M_ERR_ARG, "nmodels >= 1 and non-null descriptor arrays required");
    if (opt->deposit == M2M_DEPOSIT_GLOBAL)
        return fail(nullptr, M2M_ERR_ARG, "batches use the block-shared deposit");
    for (int i = 0; i < nmodels; ++i) {
        if (priors[i].smoothing != M2M_SMOOTH_NONE)
            return fail(nullptr, M2M_ERR_ARG, "fit %d: prior smoothing is not available in batches", i);
        if (pots[i].kind == M2M_POT_SCF)
            return fail(nullptr, M2M_ERR_ARG, "fit %d: the self-consistent potential is not available in batches", i);
    }
    if (opt->precision != M2M_PREC_FP64 && opt->precision != M2M_PREC_MIXED)
        return fail(nullptr, M2M_ERR_ARG, "unknown precision %d", opt->precision);
    m2m_ctx *ctx = new (std::nothrow) m2m_ctx();
    if (!ctx) return fail(nullptr, M2M_ERR_OOM, "host allocation failed");
    ctx->precision = opt->precision;
    ctx->bs = new (std::nothrow) BatchState();
    m2m_status s = ctx->bs ? M2M_OK : fail(ctx, M2M_ERR_OOM, "host allocation failed");
    if (s == M2M_OK) {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess && opt->stream) {
            ctx->stream = static_cast<cudaStream_t>(opt->stream);
        } else if (e == cudaSuccess) {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = e == cudaSuccess;
        }
        if (e == cudaSuccess) e = upload_constants();
        if (e != cudaSuccess) s = fail(ctx, M2M_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    m2m_options so = *opt;
    so.stream = ctx->stream;
    so.deposit = M2M_DEPOSIT_SHARED;
    for (int i = 0; s == M2M_OK && i < nmodels; ++i) {
        m2m_ctx *c = nullptr;
        s = create_impl(&pots[i], &obs[i], &priors[i], eps[i], mu[i], alpha[i], &so, 0, &c);
        if (s != M2M_OK) {
            s = fail(ctx, s, "fit %d: %s", i, g_create_error.c_str());
            break;
        }
        c->parent = ctx;
        ctx->sub.push_back(c);
    }
    if (s == M2M_OK)
        s = ctx->precision == M2M_PREC_FP64 ? batch_configure<double, 2>(ctx, opt) : batch_configure<float, 1>(ctx, opt);
    if (s != M2M_OK) {
        g_create_error = ctx->err;
        batch_destroy(ctx);
        destroy_impl(ctx);
        return s;
    }
    *out = ctx;
    return M2M_OK;
}

extern "C" m2m_status m2m_batch_size(m2m_ctx *ctx, int32_t *nmodels)
{
    if (!ctx || !nmodels) return M2M_ERR_ARG;
    *nmodels = int32_t(ctx->sub.size());
    return M2M_OK;
}

extern "C" m2m_status m2m_batch_model(m2m_ctx *ctx, int32_t i, m2m_ctx **model)
{
    if (!ctx || !model) return M2M_ERR_ARG;
    *model = nullptr;
    if (ctx->sub.empty()) return fail(ctx, M2M_ERR_STATE, "not a batch context");
    if (i < 0 || i >= int32_t(ctx->sub.size())) return fail(ctx, M2M_ERR_ARG, "fit index %d out of range", i);
    *model = ctx->sub[i];
    return M2M_OK;
}

// ------------------------------------------------------------------ autotuner

extern "C" m2m_status m2m_batch_autotune(m2m_ctx *ctx, int32_t steps, int32_t *block, int32_t *blocks_per_sm,
                                         int64_t *segment)
{
    if (!ctx) return M2M_ERR_ARG;
    if (ctx->sub.empty()) return fail(ctx, M2M_ERR_STATE, "not a batch context");
    if (steps < 1) return fail(ctx, M2M_ERR_ARG, "steps must be >= 1");
    BatchState &B = *ctx->bs;
    m2m_status s = prepare(ctx);
    if (s != M2M_OK) return s;
    struct Shape {
        int block, bps;
        long long cap;
    };
    std::vector<Shape> cand;
    for (int blk : {256, 128}) {
        int occ = 0;
        if (ctx->precision == M2M_PREC_FP64) {
            using Fn = BatchFn<double>;
            CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<Fn>(B.kernel), blk, B.smem));
        } else {
            using Fn = BatchFn<float>;
            CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reinterpret_cast<Fn>(B.kernel), blk, B.smem));
        }
        std::vector<int> bl;
        for (int v : {occ, occ - 1, (occ + 1) / 2})
            if (v >= 1 && std::find(bl.begin(), bl.end(), v) == bl.end()) bl.push_back(v);
        for (int v : bl)
            for (long long cap : {kMaxParticlesPerBlock, kMaxParticlesPerBlock / 4}) cand.push_back({blk, v, cap});
    }
    const bool timing = ctx->timing;
    ctx->timing = false;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = -1.f;
    Shape pick = {B.block, B.bps, B.seg_cap};
    for (const Shape &sh : cand) {
        B.block = sh.block;
        B.bps = sh.bps;
        B.grid = B.nsm * sh.bps;
        B.seg_cap = sh.cap;
        B.ready = false;
        if ((s = prepare(ctx)) != M2M_OK) break;
        launch(ctx);  // warm-up
        cudaEventRecord(e0, ctx->stream);
        for (int k = 0; k < steps; ++k) launch(ctx);
        cudaEventRecord(e1, ctx->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            s = fail(ctx, M2M_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0.f || ms < best) {
            best = ms;
            pick = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->timing = timing;
    B.block = pick.block;
    B.bps = pick.bps;
    B.grid = B.nsm * pick.bps;
    B.seg_cap = pick.cap;
    B.ready = false;
    if (s == M2M_OK) s = prepare(ctx);
    if (s == M2M_OK) s = batch_synchronize(ctx);
    if (block) *block = pick.block;
    if (blocks_per_sm) *blocks_per_sm = pick.bps;
    if (segment) *segment = pick.cap;
    return s;
}
