// Internal to the library: the context behind the opaque m2m_ctx handle and the
// host helpers shared by the runtime's translation units (single fits in
// m2m_api.cu, batches of fits in m2m_batch.cu).
#pragma once

#include "m2m.h"
#include "m2m_device.cuh"

#include <string>
#include <vector>

struct BatchState;

struct m2m_ctx {
    m2m::Model m{};
    int precision = 0;
    int internal = 0;  // allows the internal first-moment kind (target construction)
    double eps = 0, mu = 0, alpha = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int block = 256, bps = 0, nsm = 0, grid = 0;
    int deposit = M2M_DEPOSIT_AUTO;  // requested; global_dep: the strategy in use
    bool global_dep = false;
    size_t smem_step = 0, smem_mat = 0;

    // host copies of the descriptors
    std::vector<double> edges, Vp, isp, Y, sig, obs_post, obs_iscale, area_of_obs, lcE, scf_r;
    std::vector<int> obs_kind;
    std::vector<unsigned short> lut;
    uint64_t config_hash = 0;

    // device buffers
    long long n = 0;
    long long capacity = 0;
    void *st[10] = {nullptr};  // x, y, z, vx, vy, vz, w, and where the step keeps it the force factor
    uint16_t *cell = nullptr;
    uint16_t *ap = nullptr;  // cached apertures (Model::ap_cache)
    double *gx = nullptr;    // cached exp(-nu^2/2) (Model::gx_group, FP64 mode)
    double *d_edges = nullptr, *d_Vp = nullptr, *d_isp = nullptr, *d_lcE = nullptr;
    float *d_Vpf = nullptr, *d_ispf = nullptr;
    unsigned short *d_lut = nullptr;
    double *d_Y = nullptr, *d_sig = nullptr, *d_post = nullptr, *d_iscale = nullptr;
    int *d_kind = nullptr;
    double *d_c = nullptr, *d_prior = nullptr, *d_ytil = nullptr, *d_yraw = nullptr, *d_delta = nullptr;
    double *d_rec = nullptr, *d_iprior = nullptr, *d_lprior = nullptr;
    float *d_recf = nullptr;
    long long *d_prior_count = nullptr, *d_hist = nullptr, *d_acc = nullptr;
    unsigned long long *d_pwin = nullptr;  // window priors: cumulative-sum scratch
    // prior smoothing (m2m_smooth.cu)
    double *d_prior_raw = nullptr, *d_sV = nullptr, *d_sVT = nullptr, *d_sD = nullptr;
    double *d_spart = nullptr, *d_sz = nullptr, *d_ss = nullptr;
    int smooth_ch = 1;
    m2m::Scalars *d_sc = nullptr;
    // self-consistent potential: grid radii, interval tables (FP64, FP32), coefficients
    double *d_scf_r = nullptr, *d_scf_tab = nullptr, *d_scf_coef = nullptr;
    float *d_scf_tabf = nullptr;
    double scf_ups0 = 1.0;
    double *d_wout = nullptr;
    long long wout_cap = 0;
    bool loaded = false;

    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    std::string err;
    void *kstep = nullptr;  // the step kernel picked for the observable shape

    // kernel timing (m2m_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;  // two per timed step
    size_t timed = 0;

    // batches (m2m_create_batch): the fits are full contexts owned by the batch
    std::vector<m2m_ctx *> sub;  // the batch's fits (empty for a single fit)
    m2m_ctx *parent = nullptr;   // the owning batch (a fit handle from m2m_batch_model)
    BatchState *bs = nullptr;    // launch configuration and device arrays of a batch
    long long load_gen = 0;      // incremented by every load of particles or state

    // one shard of a fit split over processes (m2m_shard_set): the whole fit's particle
    // count, total weight and v^2 bound; the phase waiting for the caller's exchange
    bool shard = false;
    long long shard_n = 0;
    double shard_w = 0.0, shard_v2 = 0.0;
    int shard_pending = 0;  // 0 none; 1 load pass, 2 step pass (m2m_step_end next); 3 weights
};

// int64 words a context exchanges (the fixed-point sums, the range word, two weight words)
inline long long exchange_words(const m2m_ctx *c) { return (long long)c->m.hist_words + 3; }

extern thread_local std::string g_create_error;

m2m_status fail(m2m_ctx *c, m2m_status s, const char *fmt, ...);

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? M2M_ERR_OOM : M2M_ERR_CUDA,       \
                        "%s: %s", #call, cudaGetErrorString(e_));                                  \
    } while (0)

template <class T>
inline void free_dev(T *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

m2m_status create_impl(const m2m_potential *pot, const m2m_observables *obs, const m2m_prior_grid *pg, double eps,
                       double mu, double alpha, const m2m_options *opt, int internal, m2m_ctx **out);
m2m_status check_device_errors(m2m_ctx *ctx);
m2m::Buffers buffers(m2m_ctx *c);
void destroy_impl(m2m_ctx *ctx);

// The (E, x) grid fields of a model (nE, nx, spacing, signed L_z, s_lo, s_den, ncell)
// from a grid descriptor, validated.
m2m_status grid_fields(m2m_ctx *ctx, m2m::Model &m, const m2m_prior_grid *pg);
// The fit's weights as of the end of its last step into ctx->d_wout (n doubles), queued
// on ctx->stream (the pending update applied, as m2m_get_weights).
m2m_status current_weights(m2m_ctx *ctx);

// prior smoothing (m2m_smooth.cu)
m2m_status smooth_setup(m2m_ctx *ctx);
void smooth_free(m2m_ctx *ctx);
void smooth_launch(m2m_ctx *ctx);

// batch runtime (m2m_batch.cu)
m2m_status batch_step(m2m_ctx *ctx, int64_t nsteps);
m2m_status batch_synchronize(m2m_ctx *ctx);
void batch_destroy(m2m_ctx *ctx);

template <class T>
inline m2m::State<T> state(m2m_ctx *c)
{
    m2m::State<T> s;
    s.x = (T *)c->st[0]; s.y = (T *)c->st[1]; s.z = (T *)c->st[2];
    s.vx = (T *)c->st[3]; s.vy = (T *)c->st[4]; s.vz = (T *)c->st[5]; s.w = (T *)c->st[6];
    s.fa = (T *)c->st[7];
    s.cell = c->cell;
    s.ap = c->ap;
    s.gx = sizeof(T) == 8 ? reinterpret_cast<T *>(c->gx) : nullptr;
    s.n = c->n;
    return s;
}

// Resident blocks per SM the step kernels are compiled for (register budget). The
// batched mixed-precision kernel runs best at 4 blocks of 256 (64 registers; 1.147 ms
// against 1.176 ms at 5 blocks on the 96-fit workload), the single-fit one at 5.
template <class T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 2 : 5;
template <class T>
constexpr int kMinBlocksBatch = sizeof(T) == 8 ? 2 : 4;

// Compile-time shape bits of a group (see m2m::GP), for picking a specialised kernel.
inline unsigned group_mask(const m2m::GroupDesc &G)
{
    unsigned mk = 0;
    if (G.k_mass >= 0) mk |= m2m::kBitMass;
    if (G.k_v2 >= 0) mk |= m2m::kBitV2;
    if (G.k_v1 >= 0) mk |= m2m::kBitV1;
    for (int n = 0; n < 7; ++n)
        if (G.k_gh[n] >= 0) mk |= m2m::bit_gh(n);
    if (G.geometry == 1) mk |= m2m::kBitPix;
    if (G.geometry == 2) mk |= m2m::kBitShell;
    return mk;
}
