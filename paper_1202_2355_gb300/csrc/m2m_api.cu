// Host runtime of the M2M library: the C ABI declared in include/m2m.h.
//
// A context owns the particle state (structure of arrays in HBM), the
// observable and prior tables, the fixed-point accumulators and a small block
// of per-step scalars in device memory. A step is one kernel, k_step: one pass
// over the particles, whose last block to finish runs the finalize over the
// observables and prior cells. Every per-step decision is read from device
// memory, so a chunk of steps is captured once in a CUDA graph and replayed.
#include "m2m_ctx.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace m2m;

thread_local std::string g_create_error;

m2m_status fail(m2m_ctx *c, m2m_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return s;
}

static m2m_status not_a_fit(m2m_ctx *ctx)
{
    return fail(ctx, M2M_ERR_STATE, "a batch context: per-fit calls take a fit handle from m2m_batch_model");
}

static double pow2_floor(double x)
{
    int e;
    std::frexp(x, &e);  // x = f 2^e, f in [0.5, 1)
    return std::ldexp(1.0, e - 1);
}

static uint64_t fnv(uint64_t h, const void *p, size_t n)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

static bool is_gh(int kind) { return kind >= kKindGH0 && kind <= kKindGH0 + 6; }

static void free_state(m2m_ctx *c)
{
    for (auto &p : c->st) free_dev(p);
    free_dev(c->cell);
    free_dev(c->ap);
    free_dev(c->gx);
    free_dev(c->d_wout);
    c->capacity = 0;
    c->wout_cap = 0;
}

// ------------------------------------------------------------------ creation

m2m_status grid_fields(m2m_ctx *ctx, Model &m, const m2m_prior_grid *pg)
{
    m.nE = pg->nE;
    m.nx = pg->nx;
    m.e_spacing = pg->e_spacing;
    m.signed_lz = pg->signed_lz ? 1 : 0;
    if (m.nE < 1 || m.nx < 1 || (long long)m.nE * m.nx > 65535)
        return fail(ctx, M2M_ERR_ARG, "the (E, x) grid needs nE, nx >= 1, nE*nx <= 65535");
    const double lo = pg->Emin, hi = pg->Emax;
    if (!(hi > lo)) return fail(ctx, M2M_ERR_ARG, "prior grid needs Emax > Emin");
    if (m.e_spacing == M2M_E_LOGNEG) {
        if (!(hi < 0)) return fail(ctx, M2M_ERR_ARG, "ln(-E) spacing needs Emin < Emax < 0");
        m.s_lo = std::log(-lo);
        m.s_den = std::log(-hi) - std::log(-lo);
    } else if (m.e_spacing == M2M_E_EXP) {
        m.s_lo = std::exp(lo);
        m.s_den = std::exp(hi) - std::exp(lo);
    } else if (m.e_spacing == M2M_E_LINEAR) {
        m.s_lo = lo;
        m.s_den = hi - lo;
    } else {
        return fail(ctx, M2M_ERR_ARG, "unknown E spacing");
    }
    m.ncell = m.nE * m.nx;
    return M2M_OK;
}

static m2m_status build_model(m2m_ctx *ctx, const m2m_potential *pot, const m2m_observables *obs,
                              const m2m_prior_grid *pg, const m2m_options *opt)
{
    Model &m = ctx->m;
    if (!pot || !obs || !pg || !opt) return fail(ctx, M2M_ERR_ARG, "null descriptor");
    if (pot->kind < 0 || pot->kind > 3) return fail(ctx, M2M_ERR_ARG, "unknown potential kind %d", pot->kind);
    m.pot = pot->kind;
    m.G = pot->G; m.M = pot->M; m.a = pot->a; m.Ms = pot->Ms; m.rs = pot->rs;
    m.v0 = pot->v0; m.r0 = pot->r0; m.q = pot->q;
    if (m.pot < 2 && !(m.a > 0 && m.G >= 0 && m.M >= 0))
        return fail(ctx, M2M_ERR_ARG, "Hernquist needs a > 0, G >= 0, M >= 0");
    if (m.pot == 1 && !(m.rs > 0 && m.Ms >= 0)) return fail(ctx, M2M_ERR_ARG, "NFW needs rs > 0, Ms >= 0");
    if (m.pot >= 2 && !(m.r0 > 0 && m.q > 0)) return fail(ctx, M2M_ERR_ARG, "log halo needs r0 > 0, q > 0");
    if (m.pot == 0) m.phi_min = -m.G * m.M / m.a;
    else if (m.pot == 1) m.phi_min = -m.G * m.M / m.a - m.G * m.Ms / m.rs;
    else if (m.pot == 2) m.phi_min = m.v0 * m.v0 * std::log(m.r0);
    else m.phi_min = -1e300;  // the stellar well is known only once the expansion is built
    m.scf_n = m.scf_lmax = m.scf_nlm = 0;
    m.eps_ups = 0.0;
    if (m.pot == 3) {
        if (pot->scf_n < 1 || pot->scf_n > kScfMaxRadii || pot->scf_lmax < 0 || pot->scf_lmax > kScfLmax ||
            !pot->scf_r)
            return fail(ctx, M2M_ERR_ARG, "the self-consistent potential needs 1..%d grid radii and 0 <= lmax <= %d",
                        kScfMaxRadii, kScfLmax);
        for (int k = 0; k < pot->scf_n; ++k)
            if (!std::isfinite(pot->scf_r[k]) || !(pot->scf_r[k] > 0) || (k > 0 && !(pot->scf_r[k] > pot->scf_r[k - 1])))
                return fail(ctx, M2M_ERR_ARG, "self-consistent potential: grid radii must be > 0 and increasing");
        if (!(pot->ups > 0) || !std::isfinite(pot->ups) || !(pot->eps_ups >= 0) || !std::isfinite(pot->eps_ups) ||
            !(m.G >= 0))
            return fail(ctx, M2M_ERR_ARG, "self-consistent potential: Upsilon > 0, eps_ups >= 0 and G >= 0 required");
        m.scf_n = pot->scf_n;
        m.scf_lmax = pot->scf_lmax;
        m.scf_nlm = (m.scf_lmax + 1) * (m.scf_lmax + 1);
        m.eps_ups = pot->eps_ups;
        ctx->scf_ups0 = pot->ups;
        ctx->scf_r.assign(pot->scf_r, pot->scf_r + m.scf_n);
        for (int l = 0; l <= m.scf_lmax; ++l)
            for (int mm = -l; mm <= l; ++mm) {
                const int am = mm < 0 ? -mm : mm;
                double ratio = 1.0;
                for (int i = l - am + 1; i <= l + am; ++i) ratio /= i;
                double nrm = std::sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * ratio);
                if (mm != 0) nrm *= std::sqrt(2.0);
                m.scf_norm[l * (l + 1) + mm] = nrm;
                m.scf_norm_f[l * (l + 1) + mm] = float(nrm);
            }
    }

    const double inc = obs->incl_deg * 3.14159265358979323846 / 180.0;
    m.sin_i = std::sin(inc);
    m.cos_i = std::cos(inc);
    if (obs->n_groups < 1 || obs->n_groups > kMaxGroups)
        return fail(ctx, M2M_ERR_ARG, "n_groups must be 1..%d", kMaxGroups);
    m.n_groups = obs->n_groups;
    int J = 0, nap = 0, ned = 0;
    ctx->edges.clear(); ctx->Vp.clear(); ctx->isp.clear(); ctx->lut.clear();
    ctx->obs_kind.clear(); ctx->obs_post.clear(); ctx->area_of_obs.clear();
    for (int g = 0; g < m.n_groups; ++g) {
        const m2m_obs_group &S = obs->groups[g];
        GroupDesc &G = m.g[g];
        G.geometry = S.geometry;
        G.n_ap = S.n_ap;
        G.n_kinds = S.n_kinds;
        if (S.n_ap < 1) return fail(ctx, M2M_ERR_ARG, "group %d: n_ap must be >= 1", g);
        if (S.n_kinds < 1 || S.n_kinds > kMaxKinds) return fail(ctx, M2M_ERR_ARG, "group %d: n_kinds must be 1..%d", g, kMaxKinds);
        G.obs_off = J;
        G.ap_off = nap;
        G.edge_off = ned;
        G.max_gh = -1;
        G.has_v2 = 0;
        G.k_mass = G.k_v2 = G.k_v1 = -1;
        for (int n = 0; n < 7; ++n) G.k_gh[n] = -1;
        std::vector<double> area(S.n_ap);
        if (S.geometry == M2M_GEOM_ANNULI) {
            if (!S.edges) return fail(ctx, M2M_ERR_ARG, "group %d: annuli need edges", g);
            for (int p = 0; p <= S.n_ap; ++p) {
                if (!std::isfinite(S.edges[p]) || S.edges[p] < 0 || (p > 0 && !(S.edges[p] > S.edges[p - 1])))
                    return fail(ctx, M2M_ERR_ARG, "group %d: edges must be finite, >= 0 and increasing", g);
                ctx->edges.push_back(S.edges[p]);
            }
            for (int p = 0; p < S.n_ap; ++p)
                area[p] = 3.14159265358979323846 * (S.edges[p + 1] * S.edges[p + 1] - S.edges[p] * S.edges[p]);
            ned += S.n_ap + 1;
            // FP32 lookup: buckets uniform in log2(R^2) over the group. With edges uniform
            // in log R (to 1e-9) bucket b is annulus b; otherwise each bucket holds a
            // candidate annulus from a table. The device corrects by exact comparisons.
            const double e0 = std::fmax(S.edges[0], 1e-30), e1 = S.edges[S.n_ap];
            bool logu = S.n_ap >= 2 && S.edges[0] > 0;
            for (int p = 1; logu && p < S.n_ap; ++p)
                logu = std::fabs(std::log(S.edges[p + 1] / S.edges[p]) - std::log(S.edges[1] / S.edges[0])) <
                       1e-9 * std::fabs(std::log(S.edges[1] / S.edges[0]));
            const int nb = logu ? S.n_ap : std::max(64, 4 * S.n_ap);
            G.lut_identity = logu ? 1 : 0;
            G.lut_off = int(ctx->lut.size());
            G.lut_n = nb;
            G.l0 = float(std::log2(e0 * e0));
            G.lscale = float(nb / (std::log2(e1 * e1) - std::log2(e0 * e0)));
            for (int b = 0; b < nb; ++b) {
                // annulus at the lower boundary of bucket b - 1: never above the true
                // annulus when the device's approximate log2 is off by one bucket
                const double R2 = std::exp2(double(G.l0) + (b - 1) / double(G.lscale)) * (1.0 - 1e-5);
                int p = 0;
                while (p + 1 < S.n_ap && float(S.edges[p + 1] * S.edges[p + 1]) <= float(R2)) ++p;
                ctx->lut.push_back((unsigned short)p);
            }
            G.e0sq_f = float(S.edges[0] * S.edges[0]);
            G.ensq_f = float(S.edges[S.n_ap] * S.edges[S.n_ap]);
        } else if (S.geometry == M2M_GEOM_SHELLS) {
            if (!S.edges) return fail(ctx, M2M_ERR_ARG, "group %d: shells need the grid radii in edges", g);
            for (int p = 0; p < S.n_ap; ++p) {
                if (!std::isfinite(S.edges[p]) || !(S.edges[p] > 0) || (p > 0 && !(S.edges[p] > S.edges[p - 1])))
                    return fail(ctx, M2M_ERR_ARG, "group %d: grid radii must be finite, > 0 and increasing", g);
                ctx->edges.push_back(S.edges[p]);
            }
            ned += S.n_ap;
            G.lut_off = int(ctx->lut.size());
            G.lut_n = 0;
            for (int p = 0; p < S.n_ap; ++p) area[p] = 1.0;
        } else if (S.geometry == M2M_GEOM_PIXELS) {
            if (S.nx < 1 || S.ny < 1 || (long long)S.nx * S.ny != S.n_ap || !(S.xhi > S.xlo) || !(S.yhi > S.ylo))
                return fail(ctx, M2M_ERR_ARG, "group %d: pixels need nx*ny == n_ap and a non-empty box", g);
            G.nx = S.nx; G.ny = S.ny;
            G.xlo = S.xlo; G.ylo = S.ylo; G.xw = S.xhi - S.xlo; G.yw = S.yhi - S.ylo;
            G.ixw = float(S.nx / (S.xhi - S.xlo));
            G.iyw = float(S.ny / (S.yhi - S.ylo));
            G.xlo_f = float(S.xlo);
            G.ylo_f = float(S.ylo);
            G.lut_off = int(ctx->lut.size());
            G.lut_n = 0;
            const double a_pix = (S.xhi - S.xlo) / S.nx * ((S.yhi - S.ylo) / S.ny);
            for (int p = 0; p < S.n_ap; ++p) area[p] = a_pix;
        } else {
            return fail(ctx, M2M_ERR_ARG, "group %d: unknown geometry %d", g, S.geometry);
        }
        bool has_gh = false;
        for (int k = 0; k < S.n_kinds; ++k) {
            const int kind = S.kinds[k];
            if (S.geometry == M2M_GEOM_SHELLS) {
                // eq. alm: the real Y_lm of each kind; N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
                const int lm = kind - kKindAlm0;
                int l = 0;
                while ((l + 1) * (l + 1) <= lm) ++l;
                const int mm = lm - l * (l + 1);
                if (lm < 0 || l > M2M_ALM_LMAX)
                    return fail(ctx, M2M_ERR_ARG, "group %d: shells take a_lm kinds with l <= %d only", g, M2M_ALM_LMAX);
                for (int k2 = 0; k2 < k; ++k2)
                    if (S.kinds[k2] == kind) return fail(ctx, M2M_ERR_ARG, "group %d: kind %d listed twice", g, kind);
                const int am = mm < 0 ? -mm : mm;
                double ratio = 1.0;
                for (int i = l - am + 1; i <= l + am; ++i) ratio /= double(i);
                double nrm = std::sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * ratio);
                if (mm != 0) nrm *= std::sqrt(2.0);
                G.kinds[k] = kind;
                G.alm_l[k] = (signed char)l;
                G.alm_m[k] = (signed char)mm;
                G.alm_norm[k] = nrm;
                G.alm_norm_f[k] = float(nrm);
                for (int p = 0; p < S.n_ap; ++p) {
                    ctx->obs_kind.push_back(kind);
                    ctx->obs_post.push_back(1.0);
                    ctx->area_of_obs.push_back(1.0);
                }
                continue;
            }
            const bool ok = kind == kKindMass || kind == kKindV2 || is_gh(kind) || (ctx->internal && kind == kKindV1);
            if (!ok) return fail(ctx, M2M_ERR_ARG, "group %d: unknown observable kind %d", g, kind);
            G.kinds[k] = kind;
            for (int k2 = 0; k2 < k; ++k2)
                if (S.kinds[k2] == kind) return fail(ctx, M2M_ERR_ARG, "group %d: kind %d listed twice", g, kind);
            if (kind == kKindMass) G.k_mass = k;
            if (kind == kKindV2) G.k_v2 = k;
            if (kind == kKindV1) G.k_v1 = k;
            if (is_gh(kind)) G.k_gh[kind - kKindGH0] = k;
            if (kind == kKindV2) G.has_v2 = 1;
            if (is_gh(kind)) {
                has_gh = true;
                if (kind - kKindGH0 > G.max_gh) G.max_gh = kind - kKindGH0;
            }
            for (int p = 0; p < S.n_ap; ++p) {
                ctx->obs_kind.push_back(kind);
                ctx->obs_post.push_back(kind == kKindMass ? 1.0 / area[p] : 1.0);
                ctx->area_of_obs.push_back(area[p]);
            }
        }
        for (int p = 0; p < S.n_ap; ++p) {
            double v = 0.0, s = 1.0;
            if (has_gh) {
                if (!S.Vp || !S.sp) return fail(ctx, M2M_ERR_ARG, "group %d: GH kinds need Vp and sp", g);
                v = S.Vp[p];
                s = S.sp[p];
                if (!std::isfinite(v) || !(s > 0) || !std::isfinite(s))
                    return fail(ctx, M2M_ERR_ARG, "group %d: sp must be finite and > 0", g);
            }
            ctx->Vp.push_back(v);
            ctx->isp.push_back(1.0 / s);
        }
        J += S.n_kinds * S.n_ap;
        nap += S.n_ap;
    }
    m.J = J;
    m.n_ap_total = nap;
    m.n_edges_total = ned;
    m.n_lut = int(ctx->lut.size());
    int max_gh = -1;
    for (int g = 0; g < m.n_groups; ++g) max_gh = std::max(max_gh, m.g[g].max_gh);
    m.rec_len = 5 + (max_gh + 1);
    for (int g = 0; g < m.n_groups; ++g)  // shell records hold c_j of each a_lm
        if (m.g[g].geometry == M2M_GEOM_SHELLS) m.rec_len = std::max(m.rec_len, m.g[g].n_kinds);
    m.rec_len = (m.rec_len + 3) / 4 * 4;  // 16-byte records in FP32 (vector loads in the force of change)
    ctx->Y.assign(J, 0.0);
    ctx->sig.assign(J, 1.0);
    if (obs->Y && obs->sigY) {
        for (int j = 0; j < J; ++j) {
            ctx->Y[j] = obs->Y[j];
            ctx->sig[j] = obs->sigY[j];
            if (!std::isfinite(ctx->Y[j]) || !(ctx->sig[j] > 0) || !std::isfinite(ctx->sig[j]))
                return fail(ctx, M2M_ERR_ARG, "observable %d: Y finite and sigY > 0 required", j);
        }
    } else if (!ctx->internal) {
        return fail(ctx, M2M_ERR_ARG, "obs->Y and obs->sigY are required");
    }

    // priors
    if (pg->mode != M2M_REG_GWR && pg->mode != M2M_REG_MPR) return fail(ctx, M2M_ERR_ARG, "unknown prior mode");
    m.mode = pg->mode;
    m.nE = pg->nE; m.nx = pg->nx;
    m.e_spacing = pg->e_spacing;
    m.signed_lz = pg->signed_lz ? 1 : 0;
    m.update_every = pg->update_every;
    if (m.mode == M2M_REG_MPR) {
        if (m.update_every < 1) return fail(ctx, M2M_ERR_ARG, "MPR grid needs update_every >= 1");
        m2m_status gs = grid_fields(ctx, m, pg);
        if (gs != M2M_OK) return gs;
    } else {
        m.ncell = 0;
        m.update_every = 1;
    }
    m.smooth = pg->smoothing;
    m.smooth_lambda = pg->lambda;
    m.pwin_E = m.mode == M2M_REG_MPR ? pg->window_E : 0;
    m.pwin_x = m.mode == M2M_REG_MPR ? pg->window_x : 0;
    if (m.pwin_E < 0 || m.pwin_x < 0) return fail(ctx, M2M_ERR_ARG, "prior window half widths must be >= 0");
    if ((m.pwin_E > 0 || m.pwin_x > 0) && pg->smoothing != M2M_SMOOTH_NONE)
        return fail(ctx, M2M_ERR_ARG, "the prior window and prior smoothing exclude each other");
    m.win_group = -1;
    m.win_lo = m.win_n = 0;
    if (m.smooth != M2M_SMOOTH_NONE) {
        if (m.smooth != M2M_SMOOTH_SPLINE_GCV) return fail(ctx, M2M_ERR_ARG, "unknown prior smoothing");
        if (m.mode != M2M_REG_MPR || m.nE < 3 || m.nx < 3 || m.ncell > 4096)
            return fail(ctx, M2M_ERR_ARG, "prior smoothing needs the MPR grid with nE, nx >= 3 and nE*nx <= 4096");
        if (!(m.smooth_lambda >= 0.0) || !std::isfinite(m.smooth_lambda))
            return fail(ctx, M2M_ERR_ARG, "prior smoothing lambda must be >= 0 (0: chosen by GCV)");
    }

    // circular orbits
    m.lc_closed = (m.pot == 0) ? 1 : 0;
    ctx->lcE.clear();
    if (m.pot == 3) {  // Lc(E) by bisection in the current expansion (see circular_L)
        m.lc_n = 0;
    } else if (!m.lc_closed) {
        const int n = 4096;
        m.lc_n = n;
        m.lc_lnr0 = std::log(1e-6);
        m.lc_dlnr = (std::log(1e8) - m.lc_lnr0) / (n - 1);
        ctx->lcE.resize(n);
        const Cst<double> kd = make_cst<double>(m);
        for (int k = 0; k < n; ++k) {
            ctx->lcE[k] = circ_energy<double>(m, kd, std::exp(m.lc_lnr0 + k * m.lc_dlnr));
            if (k > 0 && !(ctx->lcE[k] > ctx->lcE[k - 1]))
                return fail(ctx, M2M_ERR_ARG, "circular-orbit energy is not increasing with radius");
        }
    } else {
        m.lc_n = 0;
    }

    // step
    if (!std::isfinite(opt->dt) || opt->dt < 0) return fail(ctx, M2M_ERR_ARG, "dt must be finite and >= 0");
    m.dt = opt->dt;
    m.eps = ctx->eps;
    m.mu = ctx->mu;
    m.alpha = ctx->alpha;
    m.update_rule = opt->update_rule == M2M_UPDATE_EULER ? 1 : 0;
    m.renormalize = opt->renormalize ? 1 : 0;
    m.n_relax = opt->n_relax;
    if (opt->precision != M2M_PREC_FP64 && opt->precision != M2M_PREC_MIXED)
        return fail(ctx, M2M_ERR_ARG, "unknown precision");
    ctx->precision = opt->precision;
    m.wps = ctx->precision == M2M_PREC_FP64 ? 2 : 1;
    m.cache_accel = m.pot != 3 && (ctx->precision == M2M_PREC_FP64 || m.pot == 1) ? 1 : 0;
    m.off_total = m.J * m.wps;
    m.off_grid = (m.J + 1) * m.wps;
    // aperture cache: one 16-bit code per particle (two small groups or one group)
    m.ap_cache = 0;
    bool shells = false;
    for (int g = 0; g < m.n_groups; ++g) shells |= m.g[g].geometry == M2M_GEOM_SHELLS;
    if (shells) {
        // the a_lm are found from the 3-D position: nothing to cache
    } else if (m.n_groups == 1 && m.g[0].n_ap < int(kApNone16)) m.ap_cache = 2;
    else if (m.n_groups == 2 && m.g[0].n_ap < int(kApNone8) && m.g[1].n_ap < int(kApNone8)) m.ap_cache = 1;
    m.gx_group = -1;
    for (int g = 0; m.ap_cache && m.gx_group < 0 && g < m.n_groups; ++g)
        if (m.g[g].max_gh >= 0) m.gx_group = g;
    // slots of the sums: observables, total weight, prior grid, then (self-consistent
    // potential) the expansion and the derivatives for the mass-to-light ratio
    m.off_scf = m.J + 1 + m.ncell;
    m.off_dups = m.off_scf + m.scf_n * m.scf_nlm;
    m.n_dups = (m.pot == 3 && m.eps_ups > 0.0) ? m.J : 0;
    m.nslots = m.off_dups + m.n_dups;
    m.off_count = m.nslots * m.wps;
    m.hist_words = m.off_count + m.ncell;

    // descriptor hash (for checkpoint compatibility)
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &m, offsetof(Model, fx_w));
    h = fnv(h, ctx->edges.data(), ctx->edges.size() * 8);
    h = fnv(h, ctx->Vp.data(), ctx->Vp.size() * 8);
    h = fnv(h, ctx->isp.data(), ctx->isp.size() * 8);
    h = fnv(h, ctx->Y.data(), ctx->Y.size() * 8);
    h = fnv(h, ctx->sig.data(), ctx->sig.size() * 8);
    h = fnv(h, &ctx->precision, sizeof(int));
    h = fnv(h, &m.smooth, sizeof(int));
    h = fnv(h, &m.smooth_lambda, sizeof(double));
    h = fnv(h, &m.pwin_E, sizeof(int));
    h = fnv(h, &m.pwin_x, sizeof(int));
    ctx->config_hash = h;
    return M2M_OK;
}

// Step kernels: a generic one reading the observable shape at run time, and
// versions compiled for common shapes (mass annuli + kinematic annuli; one pixel
// group of mass and h1..h4), picked at creation by matching the group masks.
template <class T>
struct StepKernel {
    using Fn = void (*)(const Model, const Cst<T>, const State<T>, const Buffers, int, int);
};


template <class T, int WPS, bool GA, unsigned M0, unsigned M1, unsigned M2, unsigned M3>
static typename StepKernel<T>::Fn step_fn() { return k_step<T, WPS, kMinBlocks<T>, GA, M0, M1, M2, M3>; }

template <class T, int WPS, bool GA>
static typename StepKernel<T>::Fn pick_step(const Model &m)
{
    // the self-consistent potential is compiled into the generic kernel only
    if (m.pot == 3) return step_fn<T, WPS, GA, kDyn, kDyn, kDyn, kDyn>();
    unsigned mk[4] = {0, 0, 0, 0};
    for (int g = 0; g < m.n_groups; ++g) mk[g] = group_mask(m.g[g]);
    constexpr unsigned kin1 = kBitV2 | bit_gh(4), kin2 = kBitV2 | bit_gh(3) | bit_gh(4);
    constexpr unsigned map = kBitPix | kBitMass | bit_gh(1) | bit_gh(2) | bit_gh(3) | bit_gh(4);
    if (m.n_groups == 2 && mk[0] == kBitMass && mk[1] == kin1) return step_fn<T, WPS, GA, kBitMass, kin1, 0u, 0u>();
    if (m.n_groups == 2 && mk[0] == kBitMass && mk[1] == kin2) return step_fn<T, WPS, GA, kBitMass, kin2, 0u, 0u>();
    if (m.n_groups == 1 && mk[0] == map) return step_fn<T, WPS, GA, map, 0u, 0u, 0u>();
    return step_fn<T, WPS, GA, kDyn, kDyn, kDyn, kDyn>();
}

template <class T>
static typename StepKernel<T>::Fn step_kernel(const m2m_ctx *c)
{
    return reinterpret_cast<typename StepKernel<T>::Fn>(c->kstep);
}

template <class T, int WPS>
static m2m_status configure_kernels(m2m_ctx *ctx)
{
    Model &m = ctx->m;
    // the finalize reuses the start of the dynamic shared memory for a block reduction
    const size_t smem_shared = std::max(smem_bytes<T>(m, 1, 1), size_t(256) * sizeof(double));
    int maxsm = 0, smsm = 0;
    CU(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    CU(cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device));
    // block-shared sums while the sums and records fit in shared memory, else global deposits
    if (ctx->deposit == M2M_DEPOSIT_SHARED && smem_shared > size_t(maxsm))
        return fail(ctx, M2M_ERR_ARG, "shared deposit needs %zu B of shared memory (limit %d)", smem_shared, maxsm);
    ctx->global_dep = ctx->deposit == M2M_DEPOSIT_GLOBAL ||
                      (ctx->deposit == M2M_DEPOSIT_AUTO && smem_shared > size_t(maxsm));
    for (int g = 0; ctx->global_dep && g < m.n_groups; ++g)
        if (m.g[g].geometry == M2M_GEOM_SHELLS)
            return fail(ctx, M2M_ERR_ARG, "shell groups (a_lm) need the shared deposit (%zu B of shared memory, limit %d)",
                        smem_shared, maxsm);
    const int max_block = ctx->global_dep ? kStepMaxThreads<T, true> : kStepMaxThreads<T, false>;
    // 512 threads in two blocks per SM was the fastest shape of the mixed-precision
    // global-deposit kernel on 64x64 maps (1024 x 1 and 256 x 4 were 8-10 % slower)
    if (ctx->block == 0) ctx->block = std::min(max_block, 512);
    if (ctx->block % 32 != 0 || ctx->block < 32 || ctx->block > max_block)
        return fail(ctx, M2M_ERR_ARG, "block must be a multiple of 32, <= %d", max_block);
    ctx->kstep = reinterpret_cast<void *>(ctx->global_dep ? pick_step<T, WPS, true>(m) : pick_step<T, WPS, false>(m));
    const size_t red = size_t(ctx->block) * sizeof(double);
    m.win_group = 0;
    m.win_lo = m.win_n = 0;
    if (ctx->global_dep) {
        // an aperture window of the largest group keeps block-shared sums, as large as the
        // blocks that registers and threads allow on an SM (or blocks_per_sm) leave room for
        int rb = 0;
        const size_t base = std::max(smem_bytes<T>(m, 0, 0, 0), red);
        CU(cudaFuncSetAttribute(step_kernel<T>(ctx), cudaFuncAttributeMaxDynamicSharedMemorySize, int(base)));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rb, step_kernel<T>(ctx), ctx->block, base));
        if (rb < 1) return fail(ctx, M2M_ERR_ARG, "step kernel cannot be resident with block %d", ctx->block);
        if (ctx->bps > 0 && ctx->bps < rb) rb = ctx->bps;
        int best = 0;
        for (int g = 1; g < m.n_groups; ++g)
            if (m.g[g].n_kinds * m.g[g].n_ap > m.g[best].n_kinds * m.g[best].n_ap) best = g;
        m.win_group = best;
        // 1 KB per block is reserved by the runtime; 1 KB more covers the carve's alignment
        const long long per_block = std::min<long long>(smsm / rb, maxsm) - 2048 - (long long)smem_bytes<T>(m, 0, 0, 0);
        const long long slot_bytes = sizeof(T) == 8 ? 16 : 12;
        if (per_block > 0) m.win_n = int(std::min<long long>(m.g[best].n_ap, per_block / (slot_bytes * m.g[best].n_kinds)));
        m.win_lo = (m.g[best].n_ap - m.win_n) / 2;  // until the load places it
    }
    ctx->smem_step = ctx->global_dep ? std::max(smem_bytes<T>(m, 2, 0, 0), red) : smem_shared;
    ctx->smem_mat = smem_bytes<T>(m, 0, 0);
    if (ctx->smem_step > size_t(maxsm))
        return fail(ctx, M2M_ERR_ARG, "observable tables and prior grid need %zu B of shared memory (limit %d)",
                    ctx->smem_step, maxsm);
    CU(cudaFuncSetAttribute(step_kernel<T>(ctx), cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctx->smem_step)));
    CU(cudaFuncSetAttribute(k_materialize<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ctx->smem_mat)));
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_kernel<T>(ctx), ctx->block, ctx->smem_step));
    if (occ < 1) return fail(ctx, M2M_ERR_ARG, "step kernel cannot be resident with block %d", ctx->block);
    if (ctx->bps <= 0 || ctx->bps > occ) ctx->bps = occ;
    return M2M_OK;
}

static m2m_status upload_tables(m2m_ctx *ctx)
{
    const Model &m = ctx->m;
    auto up = [&](double *&d, const std::vector<double> &v) -> m2m_status {
        free_dev(d);
        if (v.empty()) return M2M_OK;
        CU(cudaMalloc(&d, v.size() * sizeof(double)));
        CU(cudaMemcpy(d, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        return M2M_OK;
    };
    m2m_status s;
    if ((s = up(ctx->d_edges, ctx->edges)) != M2M_OK) return s;
    if ((s = up(ctx->d_Vp, ctx->Vp)) != M2M_OK) return s;
    if ((s = up(ctx->d_isp, ctx->isp)) != M2M_OK) return s;
    {
        std::vector<float> vf(ctx->Vp.begin(), ctx->Vp.end()), sf(ctx->isp.begin(), ctx->isp.end());
        free_dev(ctx->d_Vpf);
        free_dev(ctx->d_ispf);
        if (!vf.empty()) {
            CU(cudaMalloc(&ctx->d_Vpf, vf.size() * sizeof(float)));
            CU(cudaMalloc(&ctx->d_ispf, sf.size() * sizeof(float)));
            CU(cudaMemcpy(ctx->d_Vpf, vf.data(), vf.size() * sizeof(float), cudaMemcpyHostToDevice));
            CU(cudaMemcpy(ctx->d_ispf, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    if ((s = up(ctx->d_lcE, ctx->lcE)) != M2M_OK) return s;
    if (m.pot == 3) {
        if ((s = up(ctx->d_scf_r, ctx->scf_r)) != M2M_OK) return s;
        const size_t nt = size_t(m.scf_n + 1) * m.scf_nlm * 2;
        free_dev(ctx->d_scf_tab);
        free_dev(ctx->d_scf_tabf);
        free_dev(ctx->d_scf_coef);
        CU(cudaMalloc(&ctx->d_scf_tab, sizeof(double) * nt));
        CU(cudaMalloc(&ctx->d_scf_tabf, sizeof(float) * nt));
        CU(cudaMalloc(&ctx->d_scf_coef, sizeof(double) * size_t(m.scf_n) * m.scf_nlm));
        CU(cudaMemset(ctx->d_scf_tab, 0, sizeof(double) * nt));
        CU(cudaMemset(ctx->d_scf_tabf, 0, sizeof(float) * nt));
        CU(cudaMemset(ctx->d_scf_coef, 0, sizeof(double) * size_t(m.scf_n) * m.scf_nlm));
        ctx->m.scf_r = ctx->d_scf_r;
        ctx->m.scf_tab = ctx->d_scf_tab;
        ctx->m.scf_tabf = ctx->d_scf_tabf;
        ctx->m.scf_coef = ctx->d_scf_coef;
    }
    if ((s = up(ctx->d_Y, ctx->Y)) != M2M_OK) return s;
    if ((s = up(ctx->d_sig, ctx->sig)) != M2M_OK) return s;
    if ((s = up(ctx->d_post, ctx->obs_post)) != M2M_OK) return s;
    free_dev(ctx->d_lut);
    CU(cudaMalloc(&ctx->d_lut, sizeof(unsigned short) * (ctx->lut.size() + 1)));
    if (!ctx->lut.empty())
        CU(cudaMemcpy(ctx->d_lut, ctx->lut.data(), sizeof(unsigned short) * ctx->lut.size(), cudaMemcpyHostToDevice));
    free_dev(ctx->d_kind);
    CU(cudaMalloc(&ctx->d_kind, sizeof(int) * m.J));
    CU(cudaMemcpy(ctx->d_kind, ctx->obs_kind.data(), sizeof(int) * m.J, cudaMemcpyHostToDevice));
    CU(cudaMalloc(&ctx->d_iscale, sizeof(double) * m.J));
    CU(cudaMalloc(&ctx->d_c, sizeof(double) * m.J));
    CU(cudaMalloc(&ctx->d_rec, sizeof(double) * m.n_ap_total * m.rec_len));
    CU(cudaMemset(ctx->d_rec, 0, sizeof(double) * m.n_ap_total * m.rec_len));
    CU(cudaMalloc(&ctx->d_recf, sizeof(float) * m.n_ap_total * m.rec_len));
    CU(cudaMemset(ctx->d_recf, 0, sizeof(float) * m.n_ap_total * m.rec_len));
    CU(cudaMalloc(&ctx->d_ytil, sizeof(double) * m.J));
    CU(cudaMalloc(&ctx->d_yraw, sizeof(double) * m.J));
    CU(cudaMalloc(&ctx->d_delta, sizeof(double) * m.J));
    CU(cudaMalloc(&ctx->d_prior, sizeof(double) * (m.ncell + 1)));
    CU(cudaMalloc(&ctx->d_iprior, sizeof(double) * (m.ncell + 1)));
    CU(cudaMemset(ctx->d_iprior, 0, sizeof(double) * (m.ncell + 1)));
    CU(cudaMalloc(&ctx->d_lprior, sizeof(double) * (m.ncell + 1)));
    CU(cudaMemset(ctx->d_lprior, 0, sizeof(double) * (m.ncell + 1)));
    CU(cudaMalloc(&ctx->d_prior_count, sizeof(long long) * (m.ncell + 1)));
    CU(cudaMalloc(&ctx->d_hist, sizeof(long long) * exchange_words(ctx)));
    if (m.pwin_E > 0 || m.pwin_x > 0) CU(cudaMalloc(&ctx->d_pwin, sizeof(unsigned long long) * 3 * m.ncell));
    CU(cudaMalloc(&ctx->d_acc, sizeof(long long) * 2));
    CU(cudaMalloc(&ctx->d_sc, sizeof(Scalars)));
    CU(cudaMemset(ctx->d_c, 0, sizeof(double) * m.J));
    CU(cudaMemset(ctx->d_ytil, 0, sizeof(double) * m.J));
    CU(cudaMemset(ctx->d_yraw, 0, sizeof(double) * m.J));
    CU(cudaMemset(ctx->d_delta, 0, sizeof(double) * m.J));
    CU(cudaMemset(ctx->d_prior, 0, sizeof(double) * (m.ncell + 1)));
    CU(cudaMemset(ctx->d_prior_count, 0, sizeof(long long) * (m.ncell + 1)));
    CU(cudaMemset(ctx->d_hist, 0, sizeof(long long) * exchange_words(ctx)));
    CU(cudaMemset(ctx->d_sc, 0, sizeof(Scalars)));
    return M2M_OK;
}

m2m_status create_impl(const m2m_potential *pot, const m2m_observables *obs,
                       const m2m_prior_grid *pg, double eps, double mu, double alpha,
                              const m2m_options *opt, int internal, m2m_ctx **out)
{
    if (!out) return fail(nullptr, M2M_ERR_ARG, "out is null");
    *out = nullptr;
    if (!std::isfinite(eps) || eps < 0 || !std::isfinite(mu) || mu < 0 || !std::isfinite(alpha) || alpha < 0 || alpha > 1)
        return fail(nullptr, M2M_ERR_ARG, "eps, mu >= 0 and 0 <= alpha <= 1 required");
    m2m_ctx *ctx = new (std::nothrow) m2m_ctx();
    if (!ctx) return fail(nullptr, M2M_ERR_OOM, "host allocation failed");
    ctx->internal = internal;
    ctx->eps = eps;
    ctx->mu = mu;
    ctx->alpha = alpha;
    m2m_status s = build_model(ctx, pot, obs, pg, opt);
    if (s == M2M_OK) {
        cudaError_t e = cudaGetDevice(&ctx->device);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        if (e != cudaSuccess) s = fail(ctx, M2M_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
    }
    if (s == M2M_OK) {
        ctx->block = opt->block > 0 ? opt->block : 0;  // checked once the deposit is known
        ctx->bps = opt->blocks_per_sm;
        ctx->deposit = opt->deposit;
        if (ctx->deposit < M2M_DEPOSIT_AUTO || ctx->deposit > M2M_DEPOSIT_GLOBAL)
            s = fail(ctx, M2M_ERR_ARG, "deposit must be M2M_DEPOSIT_AUTO, _SHARED or _GLOBAL");
    }
    if (s == M2M_OK) {
        s = ctx->precision == M2M_PREC_FP64 ? configure_kernels<double, 2>(ctx) : configure_kernels<float, 1>(ctx);
    }
    if (s == M2M_OK) {
        if (opt->stream) {
            ctx->stream = static_cast<cudaStream_t>(opt->stream);
        } else {
            cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) s = fail(ctx, M2M_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
            else ctx->own_stream = true;
        }
    }
    if (s == M2M_OK) {
        cudaError_t e = upload_constants();
        if (e != cudaSuccess) s = fail(ctx, M2M_ERR_CUDA, "constant tables: %s", cudaGetErrorString(e));
    }
    if (s == M2M_OK) s = upload_tables(ctx);
    if (s == M2M_OK) s = smooth_setup(ctx);
    if (s != M2M_OK) {
        g_create_error = ctx->err;
        m2m_destroy(ctx);
        return s;
    }
    *out = ctx;
    return M2M_OK;
}

extern "C" m2m_status m2m_create(const m2m_potential *pot, const m2m_observables *obs,
                                 const m2m_prior_grid *prior, double eps, double mu, double alpha,
                                 const m2m_options *opt, m2m_ctx **out)
{
    return create_impl(pot, obs, prior, eps, mu, alpha, opt, 0, out);
}

// ------------------------------------------------------------------ launches

Buffers buffers(m2m_ctx *c)
{
    Buffers b;
    b.edges = c->d_edges; b.Vp = c->d_Vp; b.isp = c->d_isp; b.Vpf = c->d_Vpf; b.ispf = c->d_ispf; b.lcE = c->d_lcE; b.lut = c->d_lut;
    b.Y = c->d_Y; b.sig = c->d_sig; b.obs_kind = c->d_kind; b.obs_post = c->d_post; b.obs_iscale = c->d_iscale;
    b.c = c->d_c; b.rec = c->d_rec; b.recf = c->d_recf; b.prior = c->d_prior; b.iprior = c->d_iprior;
    b.lprior = c->d_lprior; b.prior_count = c->d_prior_count; b.hist = c->d_hist;
    b.prior_raw = c->d_prior_raw; b.pwin = c->d_pwin; b.sV = c->d_sV; b.sVT = c->d_sVT; b.sD = c->d_sD;
    b.spart = c->d_spart; b.sz = c->d_sz; b.ss = c->d_ss;
    b.ytil = c->d_ytil; b.yraw = c->d_yraw; b.delta = c->d_delta; b.sc = c->d_sc;
    return b;
}

static int grid_for(m2m_ctx *c)
{
    long long need = (c->n + c->block - 1) / c->block;
    long long g = (long long)c->nsm * c->bps;
    if (need < g) g = need;
    // no block may process more than kMaxParticlesPerBlock particles (exact 32-bit sums)
    const long long floor_g = (c->n + kMaxParticlesPerBlock - 1) / kMaxParticlesPerBlock;
    if (g < floor_g) g = floor_g;
    return g < 1 ? 1 : int(g);
}

template <class T, int WPS>
static void launch_step(m2m_ctx *c, int push, int init)
{
    step_kernel<T>(c)<<<grid_for(c), c->block, c->smem_step, c->stream>>>(c->m, make_cst<T>(c->m), state<T>(c),
                                                                              buffers(c), push, init);
}

static void launch_one(m2m_ctx *c, int push, int init)
{
    if (c->precision == M2M_PREC_FP64) launch_step<double, 2>(c, push, init);
    else launch_step<float, 1>(c, push, init);
    // a shard's sums wait for the caller's exchange; the finalize and smoothing follow it
    if (c->m.shard) k_shard_pack<<<1, 32, 0, c->stream>>>(c->d_hist, c->m.hist_words, c->d_sc);
    else smooth_launch(c);
}

template <class T, int WPS>
static void launch_step_timed(m2m_ctx *c, cudaEvent_t *ev)
{
    cudaEventRecord(ev[0], c->stream);
    step_kernel<T>(c)<<<grid_for(c), c->block, c->smem_step, c->stream>>>(c->m, make_cst<T>(c->m), state<T>(c),
                                                                              buffers(c), 1, 0);
    smooth_launch(c);
    cudaEventRecord(ev[1], c->stream);
}

// ------------------------------------------------------------------ particles

static size_t elem_size(const m2m_ctx *c) { return c->precision == M2M_PREC_FP64 ? 8 : 4; }

// x, y, z, vx, vy, vz, w and, where the step keeps it, the force factor of the acceleration
static int state_arrays(const m2m_ctx *c) { return c->m.cache_accel ? 8 : 7; }

static m2m_status ensure_capacity(m2m_ctx *ctx, long long n)
{
    if (n <= ctx->capacity && ctx->st[0]) return M2M_OK;
    free_state(ctx);
    const long long cap = n > 0 ? n : 1;
    const int narr = state_arrays(ctx);
    for (int k = 0; k < narr; ++k) CU(cudaMalloc(&ctx->st[k], cap * elem_size(ctx)));
    CU(cudaMalloc(&ctx->cell, cap * sizeof(uint16_t)));
    if (ctx->m.ap_cache) CU(cudaMalloc(&ctx->ap, cap * sizeof(uint16_t)));
    if (ctx->precision == M2M_PREC_FP64 && ctx->m.gx_group >= 0) CU(cudaMalloc(&ctx->gx, cap * sizeof(double)));
    ctx->capacity = cap;
    return M2M_OK;
}

static m2m_status place_window(m2m_ctx *ctx);

// Sets the fixed-point scales from the loaded particles, then deposits y_0.
static m2m_status finish_load(m2m_ctx *ctx, const double *dx, const double *dy, const double *dz,
                              const double *dvx, const double *dvy, const double *dvz,
                              const double *dw, double W0_host)
{
    Model &m = ctx->m;
    unsigned long long *d_v2 = nullptr;
    unsigned *d_bad = nullptr;
    CU(cudaMalloc(&d_v2, sizeof(unsigned long long) + sizeof(unsigned)));
    d_bad = reinterpret_cast<unsigned *>(d_v2 + 1);
    CU(cudaMemsetAsync(d_v2, 0, sizeof(unsigned long long) + sizeof(unsigned), ctx->stream));
    if (ctx->n > 0)
        k_load_stats<<<ctx->nsm * 4, 256, 0, ctx->stream>>>(m, make_cst<double>(m), dx, dy, dz, dvx, dvy, dvz, dw,
                                                             ctx->n, d_v2, d_bad);
    unsigned long long v2bits = 0;
    unsigned bad = 0;
    cudaError_t e = cudaMemcpyAsync(&v2bits, d_v2, sizeof v2bits, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d_v2);
    if (e != cudaSuccess) return fail(ctx, M2M_ERR_CUDA, "load statistics: %s", cudaGetErrorString(e));
    if (bad) return fail(ctx, M2M_ERR_ARG, "particles must be finite with weights >= 0");
    double v2max;
    std::memcpy(&v2max, &v2bits, sizeof v2max);
    m.n_all = ctx->n;
    if (ctx->shard) {
        // every shard takes the whole fit's bounds, so that all shards add the same integers
        if (v2max > ctx->shard_v2)
            return fail(ctx, M2M_ERR_ARG, "this shard's particles reach v^2 = %g above the shard bound %g", v2max,
                        ctx->shard_v2);
        v2max = ctx->shard_v2;
        W0_host = ctx->shard_w;
        m.n_all = ctx->shard_n;
    }
    if (m.pot == 3) {
        // the particles' own well is not built yet: its depth is below G Upsilon W / r_0
        const double W = (ctx->shard ? ctx->shard_w : W0_host) > 0 ? (ctx->shard ? ctx->shard_w : W0_host) : 1.0;
        v2max += 2.0 * ctx->scf_ups0 * m.G * W / ctx->scf_r[0];
    }
    // fixed-point ranges. Weights are deposited before renormalisation, so the total
    // may exceed W0 by the largest single-step growth exp(eps dt F): FP64 mode keeps
    // 2^24 W0 of range (the second word still resolves 2^-70 W0), mixed mode 2^12 W0
    // (resolution 2^-50 W0). Beyond the range the step reports M2M_ERR_OVERFLOW.
    const double W = W0_host > 0 ? W0_host : 1.0;
    const double Wb = (ctx->precision == M2M_PREC_FP64 ? 16777216.0 : 4096.0) * W;
    m.v2max = 2.0 * (v2max > 0 ? v2max : 1.0);
    const double two62 = 4611686018427387904.0;
    m.fx_w = pow2_floor(two62 / Wb);
    m.fx_v2 = pow2_floor(two62 / (Wb * (m.v2max > 1.0 ? m.v2max : 1.0)));
    m.fx_gh = pow2_floor(two62 / (Wb * 1.5));  // |2 sqrt(pi) u_n| <= sqrt(2) (Cramer's inequality)
    // derivatives for the mass-to-light ratio: |1/2 v c_n (2n H_(n-1) - nu H_n) e^(-nu^2/2)/sigma_p|
    // <= 1.5 |v| / sigma_p (n <= 6)
    {
        double isp_max = 1.0;
        for (double v : ctx->isp) isp_max = std::max(isp_max, v);
        m.fx_dv = pow2_floor(two62 / (Wb * 1.5 * std::sqrt(m.v2max) * isp_max + Wb));
    }
    ctx->obs_iscale.resize(m.J);
    for (int j = 0; j < m.J; ++j) {
        const int k = ctx->obs_kind[j];
        const double s = k == kKindMass ? m.fx_w : ((k == kKindV2 || k == kKindV1) ? m.fx_v2 : m.fx_gh);
        ctx->obs_iscale[j] = 1.0 / s;
    }
    CU(cudaMemcpyAsync(ctx->d_iscale, ctx->obs_iscale.data(), sizeof(double) * m.J, cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_hist, 0, sizeof(long long) * exchange_words(ctx), ctx->stream));
    Scalars sc0{};
    sc0.Wrange = 9.2233720368547758e18 / m.fx_w;
    sc0.ups = ctx->scf_ups0;
    CU(cudaMemcpyAsync(ctx->d_sc, &sc0, sizeof(Scalars), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(ctx->d_prior, 0, sizeof(double) * (m.ncell + 1), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_iprior, 0, sizeof(double) * (m.ncell + 1), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_lprior, 0, sizeof(double) * (m.ncell + 1), ctx->stream));
    CU(cudaMemsetAsync(ctx->d_prior_count, 0, sizeof(long long) * (m.ncell + 1), ctx->stream));
    CU(cudaMemsetAsync(ctx->cell, 0, sizeof(uint16_t) * (ctx->n > 0 ? ctx->n : 1), ctx->stream));
    launch_one(ctx, 0, 1);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (ctx->shard) {  // y_0 needs every shard's sums: m2m_step_end completes the load
        ctx->shard_pending = 1;
        return M2M_OK;
    }
    return place_window(ctx);
}

// The aperture window of the global-deposit kernel on the densest range of the first
// deposit (any placement gives the same sums; this one keeps most deposits block-shared).
static m2m_status place_window(m2m_ctx *ctx)
{
    Model &m = ctx->m;
    if (ctx->global_dep && m.win_n > 0 && m.win_n < m.g[m.win_group].n_ap) {
        // place the aperture window on the densest range of the first deposit (any
        // placement gives the same sums; this one keeps most deposits block-shared)
        const GroupDesc &G = m.g[m.win_group];
        std::vector<double> y(G.n_ap);
        CU(cudaMemcpy(y.data(), ctx->d_yraw + G.obs_off, sizeof(double) * G.n_ap, cudaMemcpyDeviceToHost));
        double run = 0.0, best = -1.0;
        for (int p = 0; p < G.n_ap; ++p) {
            run += std::fabs(y[p]);
            if (p >= m.win_n) run -= std::fabs(y[p - m.win_n]);
            if (p + 1 >= m.win_n && run > best) {
                best = run;
                m.win_lo = p + 1 - m.win_n;
            }
        }
    }
    ctx->loaded = true;
    return M2M_OK;
}

static m2m_status load_common(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel,
                              const double *w, bool device)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (n < 0 || (n > 0 && (!pos || !vel || !w))) return fail(ctx, M2M_ERR_ARG, "n >= 0 and non-null arrays required");
    ++ctx->load_gen;
    if (n > 0x7fffffffll * 64) return fail(ctx, M2M_ERR_ARG, "too many particles");
    ctx->loaded = false;
    ctx->shard_pending = 0;
    m2m_status s = ensure_capacity(ctx, n);
    if (s != M2M_OK) return s;
    ctx->n = n;
    // stage FP64 inputs on the device
    double *stage = nullptr;
    const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    CU(cudaMalloc(&stage, bytes * 7));
    const double *src[7];
    double W0 = 0.0;
    if (device) {
        for (int k = 0; k < 3; ++k) src[k] = pos + k * n;
        for (int k = 0; k < 3; ++k) src[3 + k] = vel + k * n;
        src[6] = w;
        for (int k = 0; k < 7; ++k)
            if (n > 0) CU(cudaMemcpyAsync(stage + k * n, src[k], bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        std::vector<double> hw(n);
        if (n > 0) CU(cudaMemcpyAsync(hw.data(), w, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        for (long long i = 0; i < n; ++i) W0 += hw[i];
    } else {
        if (n > 0) {
            CU(cudaMemcpyAsync(stage, pos, bytes * 3, cudaMemcpyHostToDevice, ctx->stream));
            CU(cudaMemcpyAsync(stage + 3 * n, vel, bytes * 3, cudaMemcpyHostToDevice, ctx->stream));
            CU(cudaMemcpyAsync(stage + 6 * n, w, bytes, cudaMemcpyHostToDevice, ctx->stream));
        }
        for (long long i = 0; i < n; ++i) W0 += w[i];
    }
    if (n > 0) {
        if (ctx->precision == M2M_PREC_FP64) {
            for (int k = 0; k < 6; ++k)
                CU(cudaMemcpyAsync(ctx->st[k], stage + k * n, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
            k_log_in<<<ctx->nsm * 4, 256, 0, ctx->stream>>>(stage + 6 * n, (double *)ctx->st[6], n);
        } else {
            for (int k = 0; k < 7; ++k)
                k_convert_in<float><<<ctx->nsm * 4, 256, 0, ctx->stream>>>(stage + k * n, (float *)ctx->st[k], n);
        }
    }
    s = finish_load(ctx, stage, stage + n, stage + 2 * n, stage + 3 * n, stage + 4 * n, stage + 5 * n,
                    stage + 6 * n, W0);
    cudaFree(stage);
    return s;
}

extern "C" m2m_status m2m_load_particles(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel,
                                         const double *w)
{
    return load_common(ctx, n, pos, vel, w, false);
}

extern "C" m2m_status m2m_load_particles_device(m2m_ctx *ctx, int64_t n, const double *pos_dev,
                                                const double *vel_dev, const double *w_dev)
{
    return load_common(ctx, n, pos_dev, vel_dev, w_dev, true);
}

// ------------------------------------------------------------------ stepping

static const int kGraphSteps = 16;

static m2m_status build_graph(m2m_ctx *ctx)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < kGraphSteps; ++k) launch_one(ctx, 1, 0);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return fail(ctx, M2M_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->graph = nullptr;
        return fail(ctx, M2M_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    ctx->graph_steps = kGraphSteps;
    return M2M_OK;
}

extern "C" m2m_status m2m_step(m2m_ctx *ctx, int64_t nsteps)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return batch_step(ctx, nsteps);
    if (ctx->shard) return fail(ctx, M2M_ERR_STATE, "a shard steps with m2m_step_begin and m2m_step_end");
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    if (nsteps < 0) return fail(ctx, M2M_ERR_ARG, "nsteps must be >= 0");
    if (ctx->timing) {
        for (int64_t k = 0; k < nsteps; ++k) {
            while (ctx->events.size() < 2 * (ctx->timed + 1)) {
                cudaEvent_t e;
                CU(cudaEventCreate(&e));
                ctx->events.push_back(e);
            }
            cudaEvent_t *ev = &ctx->events[2 * ctx->timed];
            if (ctx->precision == M2M_PREC_FP64) launch_step_timed<double, 2>(ctx, ev);
            else launch_step_timed<float, 1>(ctx, ev);
            ++ctx->timed;
        }
        CU(cudaGetLastError());
        return M2M_OK;
    }
    int64_t left = nsteps;
    if (left >= kGraphSteps && !ctx->graph) {
        m2m_status s = build_graph(ctx);
        if (s != M2M_OK) return s;
    }
    while (left >= kGraphSteps) {
        CU(cudaGraphLaunch(ctx->graph, ctx->stream));
        left -= kGraphSteps;
    }
    for (; left > 0; --left) launch_one(ctx, 1, 0);
    CU(cudaGetLastError());
    return M2M_OK;
}

m2m_status check_device_errors(m2m_ctx *ctx)
{
    Scalars sc;
    CU(cudaMemcpyAsync(&sc, ctx->d_sc, sizeof sc, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (sc.err & kErrNegWeight) return fail(ctx, M2M_ERR_NEG_WEIGHT, "the force of change made a weight negative");
    if (sc.err & kErrOverflow) return fail(ctx, M2M_ERR_OVERFLOW, "a deposit left the fixed-point range");
    if (sc.err & kErrNonFinite) return fail(ctx, M2M_ERR_NONFINITE, "a weight became non-finite");
    if (sc.err) return fail(ctx, M2M_ERR_CUDA, "device error word %u", sc.err);
    return M2M_OK;
}

extern "C" m2m_status m2m_synchronize(m2m_ctx *ctx)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return batch_synchronize(ctx);
    CU(cudaStreamSynchronize(ctx->stream));
    if (!ctx->loaded) return M2M_OK;
    return check_device_errors(ctx);
}

// ------------------------------------------------------------------ getters

template <class T, int WPS>
static void launch_materialize(m2m_ctx *c)
{
    const int g = c->nsm * 4;
    cudaMemsetAsync(c->d_acc, 0, 2 * sizeof(long long), c->stream);
    k_materialize<T><<<g, 256, c->smem_mat, c->stream>>>(c->m, make_cst<T>(c->m), state<T>(c), buffers(c),
                                                         c->d_wout, c->d_acc);
    k_scale<<<g, 256, 0, c->stream>>>(c->d_wout, c->n, c->d_acc, c->m, c->d_sc);
}

// ------------------------------------------------------------------ shards of one fit

extern "C" m2m_status m2m_shard_bounds(m2m_ctx *ctx, int64_t n, const double *pos, const double *vel,
                                       const double *w, double *w_sum, double *v2_bound)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (n < 0 || (n > 0 && (!pos || !vel || !w)) || !w_sum || !v2_bound)
        return fail(ctx, M2M_ERR_ARG, "n >= 0 and non-null arrays required");
    double W = 0.0;
    for (long long i = 0; i < n; ++i) W += w[i];
    *w_sum = W;
    *v2_bound = 0.0;
    if (n == 0) return M2M_OK;
    double *d = nullptr;
    const size_t bytes = sizeof(double) * size_t(n);
    CU(cudaMalloc(&d, bytes * 7 + 16));
    unsigned long long *d_v2 = reinterpret_cast<unsigned long long *>(d + 7 * n);
    unsigned *d_bad = reinterpret_cast<unsigned *>(d_v2 + 1);
    cudaError_t e = cudaMemcpyAsync(d, pos, bytes * 3, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 3 * n, vel, bytes * 3, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + 6 * n, w, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_v2, 0, 16, ctx->stream);
    if (e == cudaSuccess) {
        k_load_stats<<<ctx->nsm * 4, 256, 0, ctx->stream>>>(ctx->m, make_cst<double>(ctx->m), d, d + n, d + 2 * n,
                                                            d + 3 * n, d + 4 * n, d + 5 * n, d + 6 * n, n, d_v2, d_bad);
        e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_v2, 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(ctx, M2M_ERR_CUDA, "shard bounds: %s", cudaGetErrorString(e));
    if (h[1] & 0xFFFFFFFFull) return fail(ctx, M2M_ERR_ARG, "particles must be finite with weights >= 0");
    std::memcpy(v2_bound, &h[0], sizeof(double));
    return M2M_OK;
}

extern "C" m2m_status m2m_shard_set(m2m_ctx *ctx, int64_t n_total, double w_total, double v2_bound)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (n_total < 0 || !(w_total > 0.0) || !std::isfinite(w_total) || !(v2_bound >= 0.0) || !std::isfinite(v2_bound))
        return fail(ctx, M2M_ERR_ARG, "n_total >= 0, w_total > 0 and a finite v2_bound >= 0 required");
    ctx->shard = true;
    ctx->shard_n = n_total;
    ctx->shard_w = w_total;
    ctx->shard_v2 = v2_bound;
    ctx->shard_pending = 0;
    ctx->loaded = false;
    ctx->m.shard = 1;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    return M2M_OK;
}

extern "C" m2m_status m2m_shard_exchange(m2m_ctx *ctx, int64_t **words_dev, int64_t *count)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->shard) return fail(ctx, M2M_ERR_STATE, "not a shard (m2m_shard_set)");
    if (!words_dev || !count) return fail(ctx, M2M_ERR_ARG, "null output");
    *words_dev = reinterpret_cast<int64_t *>(ctx->d_hist);
    *count = exchange_words(ctx);
    return M2M_OK;
}

extern "C" m2m_status m2m_step_begin(m2m_ctx *ctx)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->shard) return fail(ctx, M2M_ERR_STATE, "not a shard: use m2m_step");
    if (!ctx->loaded || ctx->shard_pending != 0)
        return fail(ctx, M2M_ERR_STATE, "m2m_step_begin needs a loaded shard with no exchange pending");
    cudaEvent_t *ev = nullptr;
    if (ctx->timing) {
        while (ctx->events.size() < 2 * (ctx->timed + 1)) {
            cudaEvent_t e;
            CU(cudaEventCreate(&e));
            ctx->events.push_back(e);
        }
        ev = &ctx->events[2 * ctx->timed];
        CU(cudaEventRecord(ev[0], ctx->stream));
    }
    if (ctx->precision == M2M_PREC_FP64) launch_step<double, 2>(ctx, 1, 0);
    else launch_step<float, 1>(ctx, 1, 0);
    if (ev) {
        CU(cudaEventRecord(ev[1], ctx->stream));
        ++ctx->timed;
    }
    k_shard_pack<<<1, 32, 0, ctx->stream>>>(ctx->d_hist, ctx->m.hist_words, ctx->d_sc);
    CU(cudaGetLastError());
    ctx->shard_pending = 2;
    return M2M_OK;
}

extern "C" m2m_status m2m_step_end(m2m_ctx *ctx)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->shard) return fail(ctx, M2M_ERR_STATE, "not a shard: use m2m_step");
    if (ctx->shard_pending != 1 && ctx->shard_pending != 2)
        return fail(ctx, M2M_ERR_STATE, "m2m_step_end follows a load or m2m_step_begin");
    const int init = ctx->shard_pending == 1;
    const int threads = ctx->block;  // the finalize block of m2m_step, so chi^2 adds in the same order
    if (ctx->precision == M2M_PREC_FP64)
        k_finalize<double, 2><<<1, threads, sizeof(double) * threads, ctx->stream>>>(ctx->m, buffers(ctx), init);
    else
        k_finalize<float, 1><<<1, threads, sizeof(double) * threads, ctx->stream>>>(ctx->m, buffers(ctx), init);
    smooth_launch(ctx);
    CU(cudaGetLastError());
    ctx->shard_pending = 0;
    if (!init) return M2M_OK;
    CU(cudaStreamSynchronize(ctx->stream));
    return place_window(ctx);
}

extern "C" m2m_status m2m_shard_weights_begin(m2m_ctx *ctx)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->shard) return fail(ctx, M2M_ERR_STATE, "not a shard");
    if (!ctx->loaded || ctx->shard_pending != 0)
        return fail(ctx, M2M_ERR_STATE, "m2m_shard_weights_begin needs a loaded shard with no exchange pending");
    if (ctx->wout_cap < ctx->n || !ctx->d_wout) {
        free_dev(ctx->d_wout);
        CU(cudaMalloc(&ctx->d_wout, sizeof(double) * (ctx->n > 0 ? ctx->n : 1)));
        ctx->wout_cap = ctx->n;
    }
    long long *acc = ctx->d_hist + ctx->m.hist_words + 1;
    CU(cudaMemsetAsync(acc, 0, 2 * sizeof(long long), ctx->stream));
    if (ctx->n > 0) {
        const int g = ctx->nsm * 4;
        if (ctx->precision == M2M_PREC_FP64)
            k_materialize<double><<<g, 256, ctx->smem_mat, ctx->stream>>>(ctx->m, make_cst<double>(ctx->m),
                                                                         state<double>(ctx), buffers(ctx), ctx->d_wout, acc);
        else
            k_materialize<float><<<g, 256, ctx->smem_mat, ctx->stream>>>(ctx->m, make_cst<float>(ctx->m),
                                                                        state<float>(ctx), buffers(ctx), ctx->d_wout, acc);
    }
    CU(cudaGetLastError());
    ctx->shard_pending = 3;
    return M2M_OK;
}

// The shard's weights after the exchange of m2m_shard_weights_begin: renormalised with the
// summed total of all shards.
static m2m_status shard_weights_end(m2m_ctx *ctx, double *w)
{
    if (ctx->shard_pending != 3)
        return fail(ctx, M2M_ERR_STATE, "a shard reads its weights after m2m_shard_weights_begin and the exchange");
    long long *acc = ctx->d_hist + ctx->m.hist_words + 1;
    if (ctx->n > 0) {
        k_scale<<<ctx->nsm * 4, 256, 0, ctx->stream>>>(ctx->d_wout, ctx->n, acc, ctx->m, ctx->d_sc);
        CU(cudaMemcpyAsync(w, ctx->d_wout, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CU(cudaMemsetAsync(acc, 0, 2 * sizeof(long long), ctx->stream));
    ctx->shard_pending = 0;
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_weights(m2m_ctx *ctx, double *w, int64_t n)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    if (n != ctx->n || (n > 0 && !w)) return fail(ctx, M2M_ERR_ARG, "n must equal the loaded count (%lld)", ctx->n);
    if (ctx->shard) return shard_weights_end(ctx, w);
    if (n == 0) return m2m_synchronize(ctx);
    m2m_status s = current_weights(ctx);
    if (s != M2M_OK) return s;
    CU(cudaMemcpyAsync(w, ctx->d_wout, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    return m2m_synchronize(ctx);
}

m2m_status current_weights(m2m_ctx *ctx)
{
    if (ctx->shard)
        return fail(ctx, M2M_ERR_STATE, "a shard's weights need the exchange of m2m_shard_weights_begin");
    if (ctx->wout_cap < ctx->n) {
        free_dev(ctx->d_wout);
        CU(cudaMalloc(&ctx->d_wout, sizeof(double) * ctx->n));
        ctx->wout_cap = ctx->n;
    }
    if (ctx->precision == M2M_PREC_FP64) launch_materialize<double, 2>(ctx);
    else launch_materialize<float, 1>(ctx);
    CU(cudaGetLastError());
    return M2M_OK;
}

extern "C" m2m_status m2m_get_state(m2m_ctx *ctx, double *pos, double *vel, int64_t n)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    if (n != ctx->n) return fail(ctx, M2M_ERR_ARG, "n must equal the loaded count");
    if (n == 0) return m2m_synchronize(ctx);
    double *tmp = nullptr;
    CU(cudaMalloc(&tmp, sizeof(double) * n));
    for (int k = 0; k < 6; ++k) {
        double *dst = k < 3 ? (pos ? pos + k * n : nullptr) : (vel ? vel + (k - 3) * n : nullptr);
        if (!dst) continue;
        if (ctx->precision == M2M_PREC_FP64) {
            CU(cudaMemcpyAsync(dst, ctx->st[k], sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
        } else {
            k_convert_out<float><<<ctx->nsm * 4, 256, 0, ctx->stream>>>((const float *)ctx->st[k], tmp, n);
            CU(cudaMemcpyAsync(dst, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
            CU(cudaStreamSynchronize(ctx->stream));
        }
    }
    CU(cudaStreamSynchronize(ctx->stream));
    cudaFree(tmp);
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_observables(m2m_ctx *ctx, double *ytil, double *y, int32_t J)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    if (J != ctx->m.J) return fail(ctx, M2M_ERR_ARG, "J must be %d", ctx->m.J);
    if (ytil) CU(cudaMemcpyAsync(ytil, ctx->d_ytil, sizeof(double) * J, cudaMemcpyDeviceToHost, ctx->stream));
    if (y) CU(cudaMemcpyAsync(y, ctx->d_yraw, sizeof(double) * J, cudaMemcpyDeviceToHost, ctx->stream));
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_chi2(m2m_ctx *ctx, double *chi2, int32_t *J, double *delta)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    Scalars sc;
    CU(cudaMemcpyAsync(&sc, ctx->d_sc, sizeof sc, cudaMemcpyDeviceToHost, ctx->stream));
    if (delta) CU(cudaMemcpyAsync(delta, ctx->d_delta, sizeof(double) * ctx->m.J, cudaMemcpyDeviceToHost, ctx->stream));
    m2m_status s = m2m_synchronize(ctx);
    if (chi2) *chi2 = sc.chi2;
    if (J) *J = ctx->m.J;
    return s;
}

extern "C" m2m_status m2m_get_priors(m2m_ctx *ctx, double *grid_mean, int64_t *counts, int32_t *cells, int64_t n)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    const int nc = ctx->m.ncell;
    if (grid_mean && nc) CU(cudaMemcpyAsync(grid_mean, ctx->d_prior, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    if (counts && nc) CU(cudaMemcpyAsync(counts, ctx->d_prior_count, sizeof(int64_t) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    if (cells) {
        if (n != ctx->n) return fail(ctx, M2M_ERR_ARG, "n must equal the loaded count");
        std::vector<uint16_t> c16(n);
        if (n > 0) CU(cudaMemcpyAsync(c16.data(), ctx->cell, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, ctx->stream));
        CU(cudaStreamSynchronize(ctx->stream));
        for (long long i = 0; i < n; ++i) cells[i] = c16[i];
    }
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_prior_smoothing(m2m_ctx *ctx, double *raw_means, double *lambda)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->m.smooth) return fail(ctx, M2M_ERR_STATE, "prior smoothing is off");
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    if (raw_means)
        CU(cudaMemcpyAsync(raw_means, ctx->d_prior_raw, sizeof(double) * ctx->m.ncell, cudaMemcpyDeviceToHost,
                           ctx->stream));
    if (lambda) CU(cudaMemcpyAsync(lambda, &ctx->d_sc->smooth_lambda, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_scf(m2m_ctx *ctx, double *ups, double *coeffs, int32_t ncoeffs)
{
    if (!ctx) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (ctx->m.pot != 3) return fail(ctx, M2M_ERR_STATE, "not a self-consistent potential");
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    const int nc = ctx->m.scf_n * ctx->m.scf_nlm;
    if (coeffs && ncoeffs != nc) return fail(ctx, M2M_ERR_ARG, "ncoeffs must be scf_n (lmax+1)^2 = %d", nc);
    if (coeffs) CU(cudaMemcpyAsync(coeffs, ctx->d_scf_coef, sizeof(double) * nc, cudaMemcpyDeviceToHost, ctx->stream));
    if (ups) CU(cudaMemcpyAsync(ups, &ctx->d_sc->ups, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return m2m_synchronize(ctx);
}

extern "C" m2m_status m2m_get_step_count(m2m_ctx *ctx, int64_t *t)
{
    if (!ctx || !t) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    Scalars sc;
    CU(cudaMemcpyAsync(&sc, ctx->d_sc, sizeof sc, cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    *t = sc.t;
    return M2M_OK;
}

extern "C" m2m_status m2m_get_particle_count(m2m_ctx *ctx, int64_t *n)
{
    if (!ctx || !n) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    *n = ctx->n;
    return M2M_OK;
}

extern "C" m2m_status m2m_set_timing(m2m_ctx *ctx, int32_t on)
{
    if (!ctx) return M2M_ERR_ARG;
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->timing = on != 0;
    ctx->timed = 0;
    return M2M_OK;
}

extern "C" m2m_status m2m_get_timing(m2m_ctx *ctx, double *step_ms, int64_t *steps)
{
    if (!ctx) return M2M_ERR_ARG;
    CU(cudaStreamSynchronize(ctx->stream));
    double a = 0.0;
    for (size_t k = 0; k < ctx->timed; ++k) {
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, ctx->events[2 * k], ctx->events[2 * k + 1]));
        a += t;
    }
    if (step_ms) *step_ms = a;
    if (steps) *steps = (int64_t)ctx->timed;
    return M2M_OK;
}

// ------------------------------------------------------------------ checkpoint

struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t precision;
    uint64_t config_hash;
    int64_t n;
    int32_t J, ncell;
    double fx_w, fx_v2, fx_gh, v2max;
};

extern "C" m2m_status m2m_save_state(m2m_ctx *ctx, const char *path)
{
    if (ctx && ctx->shard) return fail(ctx, M2M_ERR_STATE, "checkpoints of shards are not supported");
    if (ctx && ctx->m.pot == 3)
        return fail(ctx, M2M_ERR_STATE, "checkpoints of a self-consistent potential are not supported");
    if (!ctx || !path) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    if (!ctx->loaded) return fail(ctx, M2M_ERR_STATE, "no particles loaded");
    m2m_status s = m2m_synchronize(ctx);
    if (s != M2M_OK) return s;
    const Model &m = ctx->m;
    CkptHeader hd{};
    std::memcpy(hd.magic, "M2MSTATE", 8);
    hd.version = 6;
    hd.precision = ctx->precision;
    hd.config_hash = ctx->config_hash;
    hd.n = ctx->n;
    hd.J = m.J;
    hd.ncell = m.ncell;
    hd.fx_w = m.fx_w; hd.fx_v2 = m.fx_v2; hd.fx_gh = m.fx_gh; hd.v2max = m.v2max;
    const size_t es = elem_size(ctx), n = size_t(ctx->n);
    const int narr = state_arrays(ctx);
    const size_t apb = m.ap_cache ? 2 * n : 0, gxb = ctx->gx ? 8 * n : 0;
    std::vector<char> buf(es * n * narr + 2 * n + apb + gxb +
                          sizeof(double) * (4 * m.J + m.n_ap_total * m.rec_len + (m.smooth ? 4 : 3) * m.ncell) + 8 * m.ncell +
                          sizeof(Scalars));
    char *p = buf.data();
    for (int k = 0; k < narr; ++k) {
        if (n) CU(cudaMemcpy(p, ctx->st[k], es * n, cudaMemcpyDeviceToHost));
        p += es * n;
    }
    if (n) CU(cudaMemcpy(p, ctx->cell, 2 * n, cudaMemcpyDeviceToHost));
    p += 2 * n;
    if (n && apb) CU(cudaMemcpy(p, ctx->ap, apb, cudaMemcpyDeviceToHost));
    p += apb;
    if (n && gxb) CU(cudaMemcpy(p, ctx->gx, gxb, cudaMemcpyDeviceToHost));
    p += gxb;
    double *dv[4] = {ctx->d_c, ctx->d_ytil, ctx->d_yraw, ctx->d_delta};
    for (auto d : dv) {
        CU(cudaMemcpy(p, d, sizeof(double) * m.J, cudaMemcpyDeviceToHost));
        p += sizeof(double) * m.J;
    }
    CU(cudaMemcpy(p, ctx->d_rec, sizeof(double) * m.n_ap_total * m.rec_len, cudaMemcpyDeviceToHost));
    p += sizeof(double) * m.n_ap_total * m.rec_len;
    if (m.ncell) {
        CU(cudaMemcpy(p, ctx->d_prior, sizeof(double) * m.ncell, cudaMemcpyDeviceToHost));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(p, ctx->d_iprior, sizeof(double) * m.ncell, cudaMemcpyDeviceToHost));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(p, ctx->d_lprior, sizeof(double) * m.ncell, cudaMemcpyDeviceToHost));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(p, ctx->d_prior_count, 8 * m.ncell, cudaMemcpyDeviceToHost));
        p += 8 * m.ncell;
        if (m.smooth) CU(cudaMemcpy(p, ctx->d_prior_raw, sizeof(double) * m.ncell, cudaMemcpyDeviceToHost));
        if (m.smooth) p += sizeof(double) * m.ncell;
    }
    CU(cudaMemcpy(p, ctx->d_sc, sizeof(Scalars), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(ctx, M2M_ERR_ARG, "cannot open %s for writing", path);
    bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1 && std::fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(ctx, M2M_ERR_ARG, "short write to %s", path);
    return M2M_OK;
}

extern "C" m2m_status m2m_load_state(m2m_ctx *ctx, const char *path)
{
    if (ctx && ctx->shard) return fail(ctx, M2M_ERR_STATE, "checkpoints of shards are not supported");
    if (ctx && ctx->m.pot == 3)
        return fail(ctx, M2M_ERR_STATE, "checkpoints of a self-consistent potential are not supported");
    if (!ctx || !path) return M2M_ERR_ARG;
    if (!ctx->sub.empty()) return not_a_fit(ctx);
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(ctx, M2M_ERR_ARG, "cannot open %s", path);
    CkptHeader hd{};
    if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, "M2MSTATE", 8) != 0 || hd.version != 6) {
        std::fclose(f);
        return fail(ctx, M2M_ERR_ARG, "%s is not an M2M state file", path);
    }
    Model &m = ctx->m;
    if (hd.config_hash != ctx->config_hash || hd.precision != ctx->precision || hd.J != m.J || hd.ncell != m.ncell) {
        std::fclose(f);
        return fail(ctx, M2M_ERR_ARG, "%s was written for different descriptors", path);
    }
    const size_t es = elem_size(ctx), n = size_t(hd.n);
    const int narr = state_arrays(ctx);
    const size_t apb = m.ap_cache ? 2 * n : 0;
    const size_t gxb = (ctx->precision == M2M_PREC_FP64 && m.gx_group >= 0) ? 8 * n : 0;
    std::vector<char> buf(es * n * narr + 2 * n + apb + gxb +
                          sizeof(double) * (4 * m.J + m.n_ap_total * m.rec_len + (m.smooth ? 4 : 3) * m.ncell) + 8 * m.ncell +
                          sizeof(Scalars));
    const bool ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(ctx, M2M_ERR_ARG, "%s is truncated", path);
    CU(cudaStreamSynchronize(ctx->stream));
    ctx->loaded = false;
    ++ctx->load_gen;
    m2m_status s = ensure_capacity(ctx, hd.n);
    if (s != M2M_OK) return s;
    ctx->n = hd.n;
    m.fx_w = hd.fx_w; m.fx_v2 = hd.fx_v2; m.fx_gh = hd.fx_gh; m.v2max = hd.v2max;
    ctx->obs_iscale.resize(m.J);
    for (int j = 0; j < m.J; ++j) {
        const int k = ctx->obs_kind[j];
        ctx->obs_iscale[j] = 1.0 / (k == kKindMass ? m.fx_w : ((k == kKindV2 || k == kKindV1) ? m.fx_v2 : m.fx_gh));
    }
    CU(cudaMemcpy(ctx->d_iscale, ctx->obs_iscale.data(), sizeof(double) * m.J, cudaMemcpyHostToDevice));
    const char *p = buf.data();
    for (int k = 0; k < narr; ++k) {
        if (n) CU(cudaMemcpy(ctx->st[k], p, es * n, cudaMemcpyHostToDevice));
        p += es * n;
    }
    if (n) CU(cudaMemcpy(ctx->cell, p, 2 * n, cudaMemcpyHostToDevice));
    p += 2 * n;
    if (n && apb) CU(cudaMemcpy(ctx->ap, p, apb, cudaMemcpyHostToDevice));
    p += apb;
    if (n && gxb) CU(cudaMemcpy(ctx->gx, p, gxb, cudaMemcpyHostToDevice));
    p += gxb;
    double *dv[4] = {ctx->d_c, ctx->d_ytil, ctx->d_yraw, ctx->d_delta};
    for (auto d : dv) {
        CU(cudaMemcpy(d, p, sizeof(double) * m.J, cudaMemcpyHostToDevice));
        p += sizeof(double) * m.J;
    }
    CU(cudaMemcpy(ctx->d_rec, p, sizeof(double) * m.n_ap_total * m.rec_len, cudaMemcpyHostToDevice));
    k_convert_in<float><<<ctx->nsm, 256, 0, ctx->stream>>>(ctx->d_rec, ctx->d_recf, m.n_ap_total * m.rec_len);
    CU(cudaStreamSynchronize(ctx->stream));
    p += sizeof(double) * m.n_ap_total * m.rec_len;
    if (m.ncell) {
        CU(cudaMemcpy(ctx->d_prior, p, sizeof(double) * m.ncell, cudaMemcpyHostToDevice));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(ctx->d_iprior, p, sizeof(double) * m.ncell, cudaMemcpyHostToDevice));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(ctx->d_lprior, p, sizeof(double) * m.ncell, cudaMemcpyHostToDevice));
        p += sizeof(double) * m.ncell;
        CU(cudaMemcpy(ctx->d_prior_count, p, 8 * m.ncell, cudaMemcpyHostToDevice));
        p += 8 * m.ncell;
        if (m.smooth) CU(cudaMemcpy(ctx->d_prior_raw, p, sizeof(double) * m.ncell, cudaMemcpyHostToDevice));
        if (m.smooth) p += sizeof(double) * m.ncell;
    }
    CU(cudaMemcpy(ctx->d_sc, p, sizeof(Scalars), cudaMemcpyHostToDevice));
    CU(cudaMemset(ctx->d_hist, 0, sizeof(long long) * m.hist_words));
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    ctx->loaded = true;
    return M2M_OK;
}

// ------------------------------------------------------------------ targets

static m2m_status observe_now(m2m_ctx *c, std::vector<double> &y)
{
    m2m_ctx *ctx = c;
    CU(cudaMemcpyAsync(c->d_Vp, c->Vp.data(), sizeof(double) * c->Vp.size(), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_isp, c->isp.data(), sizeof(double) * c->isp.size(), cudaMemcpyHostToDevice, c->stream));
    Scalars sc0{};
    sc0.Wrange = 9.2233720368547758e18 / c->m.fx_w;
    CU(cudaMemcpyAsync(c->d_sc, &sc0, sizeof(Scalars), cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    launch_one(c, 0, 1);
    CU(cudaGetLastError());
    y.resize(c->m.J);
    CU(cudaMemcpyAsync(y.data(), c->d_yraw, sizeof(double) * c->m.J, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return check_device_errors(c);
}

extern "C" m2m_status m2m_build_targets(const m2m_observables *obs, int64_t n, const double *pos,
                                        const double *vel, const double *w, const double *err,
                                        const double *noise, double *Y, double *sigY, double *Vp,
                                        double *sp, int32_t *iterations)
{
    m2m_ctx *ctx = nullptr;
    if (!obs || !err || !Y || !sigY || !Vp || !sp || n < 0 || (n > 0 && (!pos || !vel || !w)))
        return fail(nullptr, M2M_ERR_ARG, "m2m_build_targets: null argument");
    if (obs->n_groups < 1 || obs->n_groups > kMaxGroups) return fail(nullptr, M2M_ERR_ARG, "n_groups must be 1..%d", kMaxGroups);
    m2m_potential pot{};
    pot.kind = M2M_POT_HERNQUIST;
    pot.G = 1; pot.M = 1; pot.a = 1;
    m2m_prior_grid pg{};
    pg.mode = M2M_REG_GWR;
    pg.update_every = 1;
    m2m_options opt{};
    opt.precision = M2M_PREC_FP64;
    // the line-of-sight groups (annuli, pixels) get V_p, sigma_p in passes 1 and 2; shell
    // groups get the sums of (w gamma)^2 of their grid points for the a_lm errors
    int nap_total = 0;
    std::vector<int> los, apoff(obs->n_groups);
    for (int g = 0; g < obs->n_groups; ++g) {
        apoff[g] = nap_total;
        nap_total += obs->groups[g].n_ap;
        if (obs->groups[g].geometry != M2M_GEOM_SHELLS) los.push_back(g);
    }
    std::vector<double> lum(nap_total, 0.0), V(nap_total, 0.0), S(nap_total, 1.0);
    std::vector<char> has_gh(obs->n_groups, 0);
    for (int g = 0; g < obs->n_groups; ++g) {
        const m2m_obs_group &Gs = obs->groups[g];
        if (Gs.geometry != M2M_GEOM_SHELLS) continue;
        if (!Gs.edges || Gs.n_ap < 1) return fail(nullptr, M2M_ERR_ARG, "group %d: shells need the grid radii", g);
        double *l2 = lum.data() + apoff[g];
        for (int64_t i = 0; i < n; ++i) {
            const double x = pos[i], yy = pos[n + i], z = pos[2 * n + i];
            const double r = std::sqrt(x * x + yy * yy + z * z);
            const double *e = Gs.edges;
            if (!(r < e[Gs.n_ap - 1])) continue;
            if (r < e[0]) {
                l2[0] += w[i] * w[i];
                continue;
            }
            int k = 1;
            while (!(r < e[k])) ++k;
            const double d = e[k] - e[k - 1], g0 = w[i] * (e[k] - r) / d, g1 = w[i] * (r - e[k - 1]) / d;
            l2[k - 1] += g0 * g0;
            l2[k] += g1 * g1;
        }
    }
    m2m_status s = M2M_OK;
    std::vector<double> y;
    int maxit = 0;
    if (!los.empty()) {
        // pass 1: luminosity, first and second moments per aperture
        m2m_observables o1 = *obs;
        o1.Y = o1.sigY = nullptr;
        o1.n_groups = int(los.size());
        for (size_t q = 0; q < los.size(); ++q) {
            o1.groups[q] = obs->groups[los[q]];
            o1.groups[q].n_kinds = 3;
            o1.groups[q].kinds[0] = kKindMass;
            o1.groups[q].kinds[1] = kKindV1;
            o1.groups[q].kinds[2] = kKindV2;
            o1.groups[q].Vp = o1.groups[q].sp = nullptr;
        }
        s = create_impl(&pot, &o1, &pg, 0, 0, 0, &opt, 1, &ctx);
        if (s != M2M_OK) return s;
        s = m2m_load_particles(ctx, n, pos, vel, w);
        if (s == M2M_OK) s = observe_now(ctx, y);
        if (s != M2M_OK) {
            g_create_error = ctx->err;
            m2m_destroy(ctx);
            return s;
        }
        for (size_t q = 0; q < los.size(); ++q) {
            const int g = los[q];
            const GroupDesc &G = ctx->m.g[q];
            for (int k = 0; k < obs->groups[g].n_kinds; ++k) has_gh[g] |= is_gh(obs->groups[g].kinds[k]);
            for (int p = 0; p < G.n_ap; ++p) {
                const int ap = apoff[g] + p;
                const int jm = G.obs_off + p;
                const double l = y[jm] * ctx->area_of_obs[jm];
                lum[ap] = l;
                if (l > 0) {
                    V[ap] = y[G.obs_off + G.n_ap + p] / l;
                    const double var = y[G.obs_off + 2 * G.n_ap + p] / l - V[ap] * V[ap];
                    S[ap] = var > 0 ? std::sqrt(var) : 0.0;
                } else {
                    V[ap] = 0.0;
                    S[ap] = 1.0;
                }
                if (has_gh[g] && !(l > 0 && S[ap] > 0)) {
                    m2m_destroy(ctx);
                    return fail(nullptr, M2M_ERR_TARGET, "group %d aperture %d is empty or has zero dispersion", g, p);
                }
            }
        }
        m2m_destroy(ctx);
        ctx = nullptr;
        // pass 2: correct V_p, sigma_p until h1 = h2 = 0 (eq. h1h2)
        m2m_observables o2 = o1;
        std::vector<std::vector<double>> vb(los.size()), sb(los.size());
        for (size_t q = 0; q < los.size(); ++q) {
            const int g = los[q], na = obs->groups[g].n_ap;
            vb[q].assign(V.begin() + apoff[g], V.begin() + apoff[g] + na);
            sb[q].assign(S.begin() + apoff[g], S.begin() + apoff[g] + na);
            for (int p = 0; p < na; ++p)
                if (!(sb[q][p] > 0)) sb[q][p] = 1.0;
            o2.groups[q].n_kinds = 2;
            o2.groups[q].kinds[0] = kKindGH0 + 1;
            o2.groups[q].kinds[1] = kKindGH0 + 2;
            o2.groups[q].Vp = vb[q].data();
            o2.groups[q].sp = sb[q].data();
        }
        s = create_impl(&pot, &o2, &pg, 0, 0, 0, &opt, 1, &ctx);
        if (s != M2M_OK) return s;
        s = m2m_load_particles(ctx, n, pos, vel, w);
        std::vector<char> active(los.size());
        for (size_t q = 0; q < los.size(); ++q) active[q] = has_gh[los[q]];
        for (int it = 0; s == M2M_OK && it < 200; ++it) {
            bool any = false;
            for (size_t q = 0; q < los.size(); ++q) any |= active[q] != 0;
            if (!any) break;
            s = observe_now(ctx, y);
            if (s != M2M_OK) break;
            int a0 = 0;  // apertures of ctx, in the order of the line-of-sight groups
            for (size_t q = 0; q < los.size(); ++q) {
                const GroupDesc &G = ctx->m.g[q];
                const int g = los[q];
                double worst = 0.0;
                for (int p = 0; active[q] && p < G.n_ap; ++p) {
                    const int a = a0 + p;
                    const double h1 = y[G.obs_off + p] / lum[apoff[g] + p];
                    const double h2 = y[G.obs_off + G.n_ap + p] / lum[apoff[g] + p];
                    worst = std::fmax(worst, std::fmax(std::fabs(h1), std::fabs(h2)));
                    const double s_old = 1.0 / ctx->isp[a];
                    ctx->Vp[a] += std::sqrt(2.0) * s_old * h1;
                    ctx->isp[a] = 1.0 / (s_old + std::sqrt(2.0) * s_old * h2);
                }
                if (active[q]) {
                    if (worst <= 1e-12) active[q] = 0;
                    maxit = it;
                }
                a0 += G.n_ap;
            }
        }
        int a0 = 0;
        for (size_t q = 0; q < los.size(); ++q) {
            const int g = los[q];
            for (int p = 0; p < obs->groups[g].n_ap; ++p) {
                V[apoff[g] + p] = ctx->Vp[a0 + p];
                S[apoff[g] + p] = 1.0 / ctx->isp[a0 + p];
            }
            a0 += obs->groups[g].n_ap;
        }
        if (s != M2M_OK) g_create_error = ctx->err;
        m2m_destroy(ctx);
        ctx = nullptr;
        if (s != M2M_OK) return s;
    }
    const std::vector<double> &Vfin = V, &Sfin = S;
    std::vector<std::vector<double>> vbuf(obs->n_groups), sbuf(obs->n_groups);
    int ap = 0;
    // pass 3: the requested observables with the fitted Gaussian parameters
    m2m_observables o3 = *obs;
    o3.Y = o3.sigY = nullptr;
    ap = 0;
    for (int g = 0; g < o3.n_groups; ++g) {
        const int na = obs->groups[g].n_ap;
        vbuf[g].assign(Vfin.begin() + ap, Vfin.begin() + ap + na);
        sbuf[g].assign(Sfin.begin() + ap, Sfin.begin() + ap + na);
        o3.groups[g].Vp = vbuf[g].data();
        o3.groups[g].sp = sbuf[g].data();
        ap += na;
    }
    s = create_impl(&pot, &o3, &pg, 0, 0, 0, &opt, 1, &ctx);
    if (s != M2M_OK) return s;
    s = m2m_load_particles(ctx, n, pos, vel, w);
    if (s == M2M_OK) s = observe_now(ctx, y);
    if (s != M2M_OK) {
        g_create_error = ctx->err;
        m2m_destroy(ctx);
        return s;
    }
    ap = 0;
    for (int g = 0; g < o3.n_groups; ++g) {
        const GroupDesc &G = ctx->m.g[g];
        for (int k = 0; k < G.n_kinds; ++k) {
            for (int p = 0; p < G.n_ap; ++p) {
                const int j = G.obs_off + k * G.n_ap + p;
                const int kind = G.kinds[k];
                const double gn = noise ? noise[j] : 0.0;
                const double l = lum[ap + p];
                if (kind >= kKindAlm0) {
                    // shot noise of a_lm of an isotropic realisation: sum (w gamma)^2 / (4 pi)
                    sigY[j] = err[j] * std::sqrt(l / (4.0 * 3.14159265358979323846));
                    Y[j] = y[j] + sigY[j] * gn;
                } else if (kind == kKindMass) {
                    sigY[j] = err[j] * y[j];
                    Y[j] = y[j] * (1.0 + err[j] * gn);
                } else if (kind == kKindV2) {
                    const double vrms = std::sqrt(y[j] / l);
                    const double vo = vrms * (1.0 + err[j] * gn);
                    sigY[j] = 2.0 * err[j] * y[j];
                    Y[j] = l * vo * vo;
                } else {
                    sigY[j] = l * err[j];
                    Y[j] = l * (y[j] / l + err[j] * gn);
                }
            }
        }
        ap += G.n_ap;
    }
    for (int a = 0; a < nap_total; ++a) {
        Vp[a] = Vfin[a];
        sp[a] = Sfin[a];
    }
    if (iterations) *iterations = maxit;
    m2m_destroy(ctx);
    return M2M_OK;
}

// ------------------------------------------------------------------ misc

extern "C" const char *m2m_last_error(const m2m_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" void m2m_destroy(m2m_ctx *ctx)
{
    if (!ctx || ctx->parent) return;  // a fit of a batch goes with its batch
    if (!ctx->sub.empty()) batch_destroy(ctx);
    destroy_impl(ctx);
}

void destroy_impl(m2m_ctx *ctx)
{
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    free_state(ctx);
    free_dev(ctx->d_edges); free_dev(ctx->d_Vp); free_dev(ctx->d_isp); free_dev(ctx->d_Vpf); free_dev(ctx->d_ispf); free_dev(ctx->d_lcE); free_dev(ctx->d_lut);
    free_dev(ctx->d_scf_r); free_dev(ctx->d_scf_tab); free_dev(ctx->d_scf_tabf); free_dev(ctx->d_scf_coef);
    free_dev(ctx->d_Y); free_dev(ctx->d_sig); free_dev(ctx->d_post); free_dev(ctx->d_iscale);
    free_dev(ctx->d_kind); free_dev(ctx->d_c); free_dev(ctx->d_rec); free_dev(ctx->d_recf); free_dev(ctx->d_prior); free_dev(ctx->d_iprior); free_dev(ctx->d_lprior);
    free_dev(ctx->d_ytil);
    free_dev(ctx->d_yraw); free_dev(ctx->d_delta); free_dev(ctx->d_prior_count);
    free_dev(ctx->d_hist); free_dev(ctx->d_acc); free_dev(ctx->d_sc); free_dev(ctx->d_pwin);
    smooth_free(ctx);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ------------------------------------------------------------------ observables without allocation
//
// m2m_observe_static serves callers that cannot allocate device memory: code
// running where cudaMalloc is unavailable or forbidden (inside a memory pool
// owned by another runtime, between captures that must not allocate, in
// processes whose allocator is reserved by a host framework). It computes the
// raw observables y_j = sum_i w_i K_j(z_i) of caller-provided device particles in
// FP64 with the same device code as a context's deposit, and keeps all its
// scratch (the fixed-point sums, the aperture tables, a few counters) in one
// file-scope device array of kStaticScratchBytes. Every GPU that loads this
// library holds that array until the process exits.

namespace {
constexpr int kStaticMaxObs = 8192;        // J
constexpr int kStaticMaxApertures = 8192;  // sum of n_ap over the groups
constexpr int kStaticMaxEdges = 8192;      // sum of n_ap + 1 over the annulus groups
constexpr size_t kOffHist = 0;             // 2 J int64 words
constexpr size_t kOffEdges = kOffHist + sizeof(long long) * 2 * kStaticMaxObs;
constexpr size_t kOffVp = kOffEdges + sizeof(double) * kStaticMaxEdges;
constexpr size_t kOffIsp = kOffVp + sizeof(double) * kStaticMaxApertures;
constexpr size_t kOffStats = kOffIsp + sizeof(double) * kStaticMaxApertures;
// stats: sum of weights (double), max v^2 (bits), input flag, error word, blocks done
constexpr size_t kStaticScratchBytes = kOffStats + 64;

struct StaticStats {
    double wsum;
    unsigned long long v2bits;
    unsigned bad, err, done;
};
}  // namespace

static __device__ __align__(256) unsigned char g_m2m_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void *g_static_addr[256];

// Device address of the scratch array for the current device. The first call on a
// device asks the runtime for it (cudaGetSymbolAddress) and sets the constant tables.
// (m2m_observe_static as a whole synchronises its stream and reads back to host
// memory, so it is never called inside a stream capture.)
static m2m_status static_scratch(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, M2M_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return fail(nullptr, M2M_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_m2m_scratch);
        if (e != cudaSuccess) return fail(nullptr, M2M_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        e = upload_constants();
        if (e != cudaSuccess) return fail(nullptr, M2M_ERR_CUDA, "constant tables: %s", cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_addr[dev]);
    return M2M_OK;
}

// Sum of weights, largest |v|^2, finiteness of the input, and 1/sigma_p in place.
__global__ void k_static_stats(const double *x, const double *y, const double *z, const double *vx,
                               const double *vy, const double *vz, const double *w, long long n, double *isp,
                               int nap, double *edges, int nedges, StaticStats *st)
{
    if (blockIdx.x == 0) {
        for (int a = threadIdx.x; a < nap; a += blockDim.x) isp[a] = 1.0 / isp[a];
        for (int a = threadIdx.x; a < nedges; a += blockDim.x) edges[a] = edges[a] * edges[a];  // squared
    }
    double s = 0.0, best = 0.0;
    unsigned flag = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
        if (!isfinite(v2) || !isfinite(x[i] + y[i] + z[i]) || !isfinite(w[i]) || w[i] < 0.0) {
            flag = 1;
        } else {
            s += w[i];
            best = fmax(best, v2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    }
    flag = __reduce_or_sync(0xffffffffu, flag);
    if ((threadIdx.x & 31) == 0) {
        if (s != 0.0) atomicAdd(&st->wsum, s);
        atomicMax(&st->v2bits, static_cast<unsigned long long>(__double_as_longlong(best)));
        if (flag) atomicOr(&st->bad, 1u);
    }
}

// The deposit of the step kernel (FP64, generic shape), without push or force of
// change, into block sums flushed to the scratch sums; the last block writes y.
__global__ void __launch_bounds__(256) k_static_observe(const Model m, const Cst<double> k, const double *x,
                                                        const double *y, const double *z, const double *vy,
                                                        const double *vz, const double *w, long long n,
                                                        const double *edges, const double *vp, const double *isp,
                                                        long long *hist, StaticStats *st, double *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    long long *h = reinterpret_cast<long long *>(smem);
    __shared__ bool am_last;
    for (int q = threadIdx.x; q < 2 * m.J; q += blockDim.x) h[q] = 0;
    __syncthreads();
    const Tables<double> tb{edges, nullptr, vp, isp, kExp2j};  // edges: squared
    unsigned err = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double wi = w[i];
        if (wi == 0.0) continue;
        double Y, vlos;
        project(k, y[i], z[i], vy[i], vz[i], Y, vlos);
        each_group<0, kDyn, kDyn, kDyn, kDyn>(m, [&](auto, int g) {
            const GroupDesc &G = m.g[g];
            const int p = aperture<kDyn>(G, tb.esq, nullptr, x[i], Y);
            if (p >= 0) {
                if (G.has_v2 && vlos * vlos > k.v2max) err |= kErrOverflow;
                group_kernels<kDyn>(G, tb, p, vlos, wi, [&](int j, double v, int cls, int) {
                    Acc<double>::add(h, m, j, v, cls == kClassMass ? m.fx_w : (cls == kClassVel ? m.fx_v2 : m.fx_gh));
                });
            }
        });
    }
    if (err) atomicOr(&st->err, err);
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * m.J; q += blockDim.x)
        if (h[q] != 0) atomicAdd(reinterpret_cast<unsigned long long *>(hist + q), static_cast<unsigned long long>(h[q]));
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int j = threadIdx.x; j < m.J; j += blockDim.x) {
        int g = 0;
        while (g + 1 < m.n_groups && j >= m.g[g + 1].obs_off) ++g;
        const GroupDesc &G = m.g[g];
        const int q = (j - G.obs_off) / G.n_ap, p = (j - G.obs_off) % G.n_ap;
        const int kind = G.kinds[q];
        const double scale = kind == kKindMass ? m.fx_w : (kind == kKindV2 ? m.fx_v2 : m.fx_gh);
        double post = 1.0;
        if (kind == kKindMass) {
            double area;
            if (G.geometry == 0) {  // edges holds the squared edges
                const double e0s = edges[G.edge_off + p], e1s = edges[G.edge_off + p + 1];
                area = __dmul_rn(3.14159265358979323846, __dsub_rn(e1s, e0s));
            } else {
                area = __dmul_rn(__ddiv_rn(G.xw, double(G.nx)), __ddiv_rn(G.yw, double(G.ny)));
            }
            post = 1.0 / area;
        }
        out[j] = fx_read<2>(hist, j) * (1.0 / scale) * post;
    }
}

extern "C" m2m_status m2m_observe_static(const m2m_observables *obs, int64_t n, const double *pos_dev,
                                         const double *vel_dev, const double *w_dev, double *y_dev, void *stream)
{
    // errors are reported through m2m_last_error(NULL)
    if (!obs || n < 0 || (n > 0 && (!pos_dev || !vel_dev || !w_dev)) || !y_dev)
        return fail(nullptr, M2M_ERR_ARG, "m2m_observe_static: null argument or n < 0");
    if (obs->n_groups < 1 || obs->n_groups > kMaxGroups)
        return fail(nullptr, M2M_ERR_ARG, "n_groups must be 1..%d", kMaxGroups);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *scr = nullptr;
    m2m_status status = static_scratch(&scr);
    if (status != M2M_OK) return status;
    double *d_edges = reinterpret_cast<double *>(scr + kOffEdges);
    double *d_vp = reinterpret_cast<double *>(scr + kOffVp);
    double *d_isp = reinterpret_cast<double *>(scr + kOffIsp);
    long long *d_hist = reinterpret_cast<long long *>(scr + kOffHist);
    StaticStats *d_st = reinterpret_cast<StaticStats *>(scr + kOffStats);

    // the model of the observable set (the fields the deposit reads), validated as m2m_create does
    Model m{};
    const double inc = obs->incl_deg * 3.14159265358979323846 / 180.0;
    m.sin_i = std::sin(inc);
    m.cos_i = std::cos(inc);
    m.n_groups = obs->n_groups;
    int J = 0, nap = 0, ned = 0;
    for (int g = 0; g < m.n_groups; ++g) {
        const m2m_obs_group &S = obs->groups[g];
        GroupDesc &G = m.g[g];
        G.geometry = S.geometry;
        G.n_ap = S.n_ap;
        G.n_kinds = S.n_kinds;
        G.obs_off = J;
        G.ap_off = nap;
        G.edge_off = ned;
        G.max_gh = -1;
        G.k_mass = G.k_v2 = G.k_v1 = -1;
        for (int q = 0; q < 7; ++q) G.k_gh[q] = -1;
        if (S.n_ap < 1 || S.n_kinds < 1 || S.n_kinds > kMaxKinds)
            return fail(nullptr, M2M_ERR_ARG, "group %d: n_ap >= 1 and 1 <= n_kinds <= %d required", g, kMaxKinds);
        if (S.geometry == M2M_GEOM_ANNULI) {
            if (!S.edges) return fail(nullptr, M2M_ERR_ARG, "group %d: annuli need edges", g);
            for (int p = 0; p <= S.n_ap; ++p)
                if (!std::isfinite(S.edges[p]) || S.edges[p] < 0 || (p > 0 && !(S.edges[p] > S.edges[p - 1])))
                    return fail(nullptr, M2M_ERR_ARG, "group %d: edges must be finite, >= 0 and increasing", g);
            ned += S.n_ap + 1;
        } else if (S.geometry == M2M_GEOM_PIXELS) {
            if (S.nx < 1 || S.ny < 1 || (long long)S.nx * S.ny != S.n_ap || !(S.xhi > S.xlo) || !(S.yhi > S.ylo))
                return fail(nullptr, M2M_ERR_ARG, "group %d: pixels need nx*ny == n_ap and a non-empty box", g);
            G.nx = S.nx; G.ny = S.ny;
            G.xlo = S.xlo; G.ylo = S.ylo; G.xw = S.xhi - S.xlo; G.yw = S.yhi - S.ylo;
        } else {
            return fail(nullptr, M2M_ERR_ARG, "group %d: unknown geometry %d", g, S.geometry);
        }
        for (int q = 0; q < S.n_kinds; ++q) {
            const int kind = S.kinds[q];
            if (!(kind == kKindMass || kind == kKindV2 || is_gh(kind)))
                return fail(nullptr, M2M_ERR_ARG, "group %d: unknown observable kind %d", g, kind);
            for (int q2 = 0; q2 < q; ++q2)
                if (S.kinds[q2] == kind) return fail(nullptr, M2M_ERR_ARG, "group %d: kind %d listed twice", g, kind);
            G.kinds[q] = kind;
            if (kind == kKindMass) G.k_mass = q;
            if (kind == kKindV2) G.k_v2 = q, G.has_v2 = 1;
            if (is_gh(kind)) G.k_gh[kind - kKindGH0] = q, G.max_gh = std::max(G.max_gh, kind - kKindGH0);
        }
        if (G.max_gh >= 0) {
            if (!S.Vp || !S.sp) return fail(nullptr, M2M_ERR_ARG, "group %d: GH kinds need Vp and sp", g);
            for (int p = 0; p < S.n_ap; ++p)
                if (!std::isfinite(S.Vp[p]) || !(S.sp[p] > 0) || !std::isfinite(S.sp[p]))
                    return fail(nullptr, M2M_ERR_ARG, "group %d: sp must be finite and > 0", g);
        }
        J += S.n_kinds * S.n_ap;
        nap += S.n_ap;
    }
    if (J > kStaticMaxObs || nap > kStaticMaxApertures || ned > kStaticMaxEdges)
        return fail(nullptr, M2M_ERR_ARG,
                    "m2m_observe_static holds at most %d observables, %d apertures and %d annulus edges "
                    "(got %d, %d, %d)", kStaticMaxObs, kStaticMaxApertures, kStaticMaxEdges, J, nap, ned);
    m.J = J;
    m.n_ap_total = nap;
    m.n_edges_total = ned;

#define CS(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(nullptr, M2M_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

    // tables into the scratch array; the sums and counters must start at zero
    for (int g = 0; g < m.n_groups; ++g) {
        const m2m_obs_group &S = obs->groups[g];
        const GroupDesc &G = m.g[g];
        if (G.geometry == 0)
            CS(cudaMemcpyAsync(d_edges + G.edge_off, S.edges, sizeof(double) * (S.n_ap + 1), cudaMemcpyHostToDevice, st));
        if (G.max_gh >= 0) {
            CS(cudaMemcpyAsync(d_vp + G.ap_off, S.Vp, sizeof(double) * S.n_ap, cudaMemcpyHostToDevice, st));
            CS(cudaMemcpyAsync(d_isp + G.ap_off, S.sp, sizeof(double) * S.n_ap, cudaMemcpyHostToDevice, st));
        } else {
            CS(cudaMemsetAsync(d_vp + G.ap_off, 0, sizeof(double) * S.n_ap, st));
            CS(cudaMemsetAsync(d_isp + G.ap_off, 0, sizeof(double) * S.n_ap, st));  // unused for such groups
        }
    }
    CS(cudaMemsetAsync(d_hist, 0, sizeof(long long) * 2 * J, st));
    CS(cudaMemsetAsync(d_st, 0, sizeof(StaticStats), st));
    int nsm = 0;
    int dev = 0;
    CS(cudaGetDevice(&dev));
    CS(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const double *px = pos_dev, *py = pos_dev + n, *pz = pos_dev + 2 * n;
    const double *vx = vel_dev, *vy = vel_dev + n, *vz = vel_dev + 2 * n;
    k_static_stats<<<nsm * 4, 256, 0, st>>>(px, py, pz, vx, vy, vz, w_dev, n, d_isp, nap, d_edges, ned, d_st);
    CS(cudaGetLastError());
    StaticStats hs{};
    CS(cudaMemcpyAsync(&hs, d_st, sizeof hs, cudaMemcpyDeviceToHost, st));
    CS(cudaStreamSynchronize(st));
    if (hs.bad) return fail(nullptr, M2M_ERR_ARG, "particles must be finite with weights >= 0");
    // groups without Gauss-Hermite kernels never read 1/sigma_p (zeros became inf above)
    double v2max;
    std::memcpy(&v2max, &hs.v2bits, sizeof v2max);
    const double W = hs.wsum > 0 ? hs.wsum : 1.0;
    const double Wb = 16777216.0 * W;  // the FP64-mode range of a context
    const double two62 = 4611686018427387904.0;
    m.v2max = 2.0 * (v2max > 0 ? v2max : 1.0);
    m.fx_w = pow2_floor(two62 / Wb);
    m.fx_v2 = pow2_floor(two62 / (Wb * (m.v2max > 1.0 ? m.v2max : 1.0)));
    m.fx_gh = pow2_floor(two62 / (Wb * 1.5));
    const size_t smem = sizeof(long long) * 2 * size_t(J);
    CS(cudaFuncSetAttribute(k_static_observe, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    int occ = 0;
    CS(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_static_observe, 256, smem));
    long long grid = std::min<long long>((n + 255) / 256, (long long)nsm * std::max(occ, 1));
    if (grid < 1) grid = 1;
    k_static_observe<<<int(grid), 256, smem, st>>>(m, make_cst<double>(m), px, py, pz, vy, vz, w_dev, n, d_edges, d_vp,
                                                    d_isp, d_hist, d_st, y_dev);
    CS(cudaGetLastError());
    CS(cudaMemcpyAsync(&hs, d_st, sizeof hs, cudaMemcpyDeviceToHost, st));
    CS(cudaStreamSynchronize(st));
#undef CS
    if (hs.err & kErrOverflow) return fail(nullptr, M2M_ERR_OVERFLOW, "a deposit left the fixed-point range");
    return M2M_OK;
}
