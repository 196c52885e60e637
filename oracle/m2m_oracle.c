/*
 * Plain single-threaded FP64 oracle of the chi^2 M2M step with moving-prior
 * regularisation (Morganti & Gerhard 2012, arXiv 1202.2355).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU baseline
 * leg of the benchmark; never by the product path. Written for obviousness,
 * not speed: every sum is a plain loop in particle order, every kernel value is
 * recomputed from its definition, the circular angular momentum is found by
 * bisection. Built with -ffp-contract=off so that x86 and Arm give the same
 * rounding.
 *
 * The step, in the order the method states it (Sec. 2.1, eqs. obs, myts,
 * delta, chi, modFOC; Sec. 2.3.1 for the priors; eq. S+ for the entropy):
 *   1. advance every particle by one leap-frog (kick-drift-kick) step (Sec. 4.1);
 *   2. observables y_j = sum_i w_i K_j(z_i)                            (eq. obs);
 *   3. temporal smoothing, discretised as ytil <- ytil + alpha (y - ytil) (eq. myts);
 *   4. residuals Delta_j = (ytil_j - Y_j)/sigma_j, chi^2 = sum Delta_j^2 (eqs. delta, chi);
 *   5. on prior-update steps: bin the particles on the (E, x = L/Lc(E))
 *      grid, prior of each cell = mean weight in the cell (Sec. 2.3.1);
 *   6. force of change dw_i/dt = eps w_i (mu dS/dw_i - sum_j K_ij Delta_j/sigma_j)
 *      (eq. modFOC) with dS/dw_i = -ln(w_i/what_i) for the moving-prior
 *      entropy (eq. S+) or -ln(w_i/what_i) - 1 for the global weight entropy
 *      (eq. entropy), integrated over dt with the force held fixed;
 *   7. optionally rescale the weights to the initial total weight (Sec. 3.2).
 */
#include "m2m_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static const double OR_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Potentials (eq. her; eq. log_halo; NFW halo)                        */
/* ------------------------------------------------------------------ */

/* Enclosed-mass factor of an NFW halo, ln(1+q) - q/(1+q), with its power
 * series for small q where the two terms cancel. */
static double nfw_mu(double q)
{
    if (q < 1e-3) {
        double s = 0.0, qk = q * q;
        for (int k = 2; k <= 9; ++k) {
            double term = (double)(k - 1) / (double)k * qk;
            s += (k % 2 == 0) ? term : -term;
            qk *= q;
        }
        return s;
    }
    return log1p(q) - q / (1.0 + q);
}

static double log_halo_phi(const or_potential *p, double x, double y, double z)
{
    double D = p->r0 * p->r0 + x * x + y * y + z * z / (p->q * p->q);
    return 0.5 * p->v0 * p->v0 * log(D);
}

static void log_halo_accel(const or_potential *p, double x, double y, double z, double *ax, double *ay,
                           double *az)
{
    double q2 = p->q * p->q;
    double D = p->r0 * p->r0 + x * x + y * y + z * z / q2;
    double v2 = p->v0 * p->v0;
    *ax = -v2 * x / D;
    *ay = -v2 * y / D;
    *az = -v2 * z / (q2 * D);
}

double or_phi(const or_potential *p, double x, double y, double z)
{
    if (p->kind == OR_POT_SCF)
        return *p->scf_ups * or_scf_phi(p, x, y, z, NULL) + log_halo_phi(p, x, y, z);
    if (p->kind == OR_POT_LOG) {
        double D = p->r0 * p->r0 + x * x + y * y + z * z / (p->q * p->q);
        return 0.5 * p->v0 * p->v0 * log(D);
    }
    double r = sqrt(x * x + y * y + z * z);
    double phi = -p->G * p->M / (r + p->a);
    if (p->kind == OR_POT_HERNQUIST_NFW) {
        if (r > 0.0)
            phi += -p->G * p->Ms * log1p(r / p->rs) / r;
        else
            phi += -p->G * p->Ms / p->rs;
    }
    return phi;
}

void or_accel(const or_potential *p, double x, double y, double z,
              double *ax, double *ay, double *az)
{
    if (p->kind == OR_POT_SCF) {
        double g[3];
        or_scf_phi(p, x, y, z, g);
        log_halo_accel(p, x, y, z, ax, ay, az);
        *ax -= *p->scf_ups * g[0];
        *ay -= *p->scf_ups * g[1];
        *az -= *p->scf_ups * g[2];
        return;
    }
    if (p->kind == OR_POT_LOG) {
        double q2 = p->q * p->q;
        double D = p->r0 * p->r0 + x * x + y * y + z * z / q2;
        double v2 = p->v0 * p->v0;
        *ax = -v2 * x / D;
        *ay = -v2 * y / D;
        *az = -v2 * z / (q2 * D);
        return;
    }
    double r = sqrt(x * x + y * y + z * z);
    if (r == 0.0) {
        *ax = *ay = *az = 0.0;
        return;
    }
    /* g(r) = G M(<r)/r^2; acceleration = -g(r) x/r */
    double g = p->G * p->M / ((r + p->a) * (r + p->a));
    if (p->kind == OR_POT_HERNQUIST_NFW)
        g += p->G * p->Ms * nfw_mu(r / p->rs) / (r * r);
    *ax = -g * x / r;
    *ay = -g * y / r;
    *az = -g * z / r;
}

void or_leapfrog(const or_potential *p, or_particles *s, double dt)
{
    for (long i = 0; i < s->n; ++i) {
        double ax, ay, az;
        or_accel(p, s->x[i], s->y[i], s->z[i], &ax, &ay, &az);
        s->vx[i] += 0.5 * dt * ax;
        s->vy[i] += 0.5 * dt * ay;
        s->vz[i] += 0.5 * dt * az;
        s->x[i] += dt * s->vx[i];
        s->y[i] += dt * s->vy[i];
        s->z[i] += dt * s->vz[i];
        or_accel(p, s->x[i], s->y[i], s->z[i], &ax, &ay, &az);
        s->vx[i] += 0.5 * dt * ax;
        s->vy[i] += 0.5 * dt * ay;
        s->vz[i] += 0.5 * dt * az;
    }
}

/* ------------------------------------------------------------------ */
/* Gauss-Hermite functions (Sec. 3.3, eq. lumghn)                      */
/* ------------------------------------------------------------------ */

/* Physicists' Hermite polynomial from its explicit sum:
 * H_n(x) = n! sum_{m=0}^{floor(n/2)} (-1)^m (2x)^(n-2m) / (m! (n-2m)!). */
double or_hermite(int n, double x)
{
    double fact[16];
    fact[0] = 1.0;
    for (int k = 1; k < 16; ++k) fact[k] = fact[k - 1] * k;
    double s = 0.0;
    for (int m = 0; 2 * m <= n; ++m) {
        double t = fact[n] / (fact[m] * fact[n - 2 * m]) * pow(2.0 * x, n - 2 * m);
        s += (m % 2 == 0) ? t : -t;
    }
    return s;
}

/* The kernel value of one particle for b_n, with L = 1:
 * 2 sqrt(pi) u_n(nu), u_n(nu) = (2^(n+1) pi n!)^(-1/2) H_n(nu) exp(-nu^2/2). */
double or_gh_kernel(int n, double nu)
{
    double nfact = 1.0;
    for (int k = 2; k <= n; ++k) nfact *= k;
    double norm = 1.0 / sqrt(pow(2.0, n + 1) * OR_PI * nfact);
    return 2.0 * sqrt(OR_PI) * norm * or_hermite(n, nu) * exp(-0.5 * nu * nu);
}

/* ------------------------------------------------------------------ */
/* Observables (eq. obs; surface density in apertures; eq. lumghn)     */
/* ------------------------------------------------------------------ */

int or_num_obs(const or_obs *o)
{
    int J = 0;
    for (int g = 0; g < o->n_groups; ++g) J += o->g[g].n_kinds * o->g[g].n_ap;
    return J;
}

/* Sky position (X, Y) and line-of-sight velocity for a line of sight
 * n = (0, sin i, cos i) with sky axes e1 = (1,0,0), e2 = (0, cos i, -sin i). */
static void project(double incl_deg, double x, double y, double z, double vy, double vz,
                    double *X, double *Y, double *vlos)
{
    double i = incl_deg * OR_PI / 180.0;
    double si = sin(i), ci = cos(i);
    *X = x;
    *Y = y * ci - z * si;
    *vlos = vy * si + vz * ci;
}

/* Aperture containing sky point (X, Y), or -1. Annuli are half-open
 * [edge_p, edge_p+1); pixel p = py*nx + px with px = floor((X-xlo) nx/(xhi-xlo)). */
static int aperture(const or_group *G, double X, double Y, double *area)
{
    if (G->geometry == OR_ANNULI) {
        double R = sqrt(X * X + Y * Y);
        for (int p = 0; p < G->n_ap; ++p) {
            if (G->edges[p] <= R && R < G->edges[p + 1]) {
                *area = OR_PI * (G->edges[p + 1] * G->edges[p + 1] - G->edges[p] * G->edges[p]);
                return p;
            }
        }
        return -1;
    }
    double fx = floor((X - G->xlo) * G->nx / (G->xhi - G->xlo));
    double fy = floor((Y - G->ylo) * G->ny / (G->yhi - G->ylo));
    if (fx < 0.0 || fx >= G->nx || fy < 0.0 || fy >= G->ny) return -1;
    *area = (G->xhi - G->xlo) / G->nx * ((G->yhi - G->ylo) / G->ny);
    return (int)fy * G->nx + (int)fx;
}

double or_ylm(int l, int m, double cos_theta, double phi)
{
    int am = m < 0 ? -m : m;
    double x = cos_theta;
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    /* P_am^am = (2 am - 1)!! s^am, then P_l^am by the recurrence in l */
    double pmm = 1.0;
    for (int i = 1; i <= am; ++i) pmm *= (2.0 * i - 1.0) * s;
    double plm = pmm;
    if (l > am) {
        double p1 = x * (2.0 * am + 1.0) * pmm, p0 = pmm;
        for (int ll = am + 2; ll <= l; ++ll) {
            double p2 = (x * (2.0 * ll - 1.0) * p1 - (ll + am - 1.0) * p0) / (ll - am);
            p0 = p1;
            p1 = p2;
        }
        plm = p1;
    }
    /* N_lm = sqrt((2l+1)/(4 pi) (l-am)!/(l+am)!) */
    double ratio = 1.0;
    for (int i = l - am + 1; i <= l + am; ++i) ratio /= i;
    double N = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * ratio);
    if (m == 0) return N * plm;
    if (m > 0) return sqrt(2.0) * N * plm * cos(am * phi);
    return sqrt(2.0) * N * plm * sin(am * phi);
}

int or_cic(const or_group *G, double r, int *k_out, double *g_out)
{
    const double *e = G->edges;
    int n = G->n_ap;
    if (r < e[0]) {
        k_out[0] = 0;
        g_out[0] = 1.0;
        return 1;
    }
    for (int k = 1; k < n; ++k) {
        if (e[k - 1] <= r && r < e[k]) {
            double d = e[k] - e[k - 1];
            k_out[0] = k - 1;
            g_out[0] = (e[k] - r) / d;
            k_out[1] = k;
            g_out[1] = (r - e[k - 1]) / d;
            return 2;
        }
    }
    return 0;
}

/* Non-zero entries K_ij of one particle: observable index and value. */
int or_kernel_row(const or_obs *o, double x, double y, double z,
                  double vx, double vy, double vz, int *j_out, double *K_out)
{
    (void)vx;
    double X, Y, vlos;
    project(o->incl_deg, x, y, z, vy, vz, &X, &Y, &vlos);
    int cnt = 0, off = 0;
    for (int g = 0; g < o->n_groups; ++g) {
        const or_group *G = &o->g[g];
        if (G->geometry == OR_SHELLS) {
            /* eq. alm: K = gamma_k^CIC(r) Y_lm(theta, phi), the total luminosity carried
             * by the weights */
            double r = sqrt(x * x + y * y + z * z);
            double ct = r > 0.0 ? z / r : 1.0;
            double phi = atan2(y, x);
            int kp[2];
            double gp[2];
            int np = or_cic(G, r, kp, gp);
            for (int a = 0; a < np; ++a) {
                for (int k = 0; k < G->n_kinds; ++k) {
                    int lm = G->kinds[k] - OR_ALM0;
                    int l = (int)floor(sqrt((double)lm));
                    int m = lm - l * (l + 1);
                    j_out[cnt] = off + k * G->n_ap + kp[a];
                    K_out[cnt] = gp[a] * or_ylm(l, m, ct, phi);
                    ++cnt;
                }
            }
            off += G->n_kinds * G->n_ap;
            continue;
        }
        double area = 0.0;
        int p = aperture(G, X, Y, &area);
        if (p >= 0) {
            for (int k = 0; k < G->n_kinds; ++k) {
                int kind = G->kinds[k];
                double K;
                if (kind == OR_MASS)
                    K = 1.0 / area;
                else if (kind == OR_V2)
                    K = vlos * vlos;
                else
                    K = or_gh_kernel(kind - OR_GH0, (vlos - G->Vp[p]) / G->sp[p]);
                j_out[cnt] = off + k * G->n_ap + p;
                K_out[cnt] = K;
                ++cnt;
            }
        }
        off += G->n_kinds * G->n_ap;
    }
    return cnt;
}

/* Dense N x J kernel matrix (row-major), for brute-force checks on tiny N. */
void or_kernel_matrix(const or_obs *o, const or_particles *s, double *K)
{
    int J = or_num_obs(o);
    int jj[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    double kk[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    memset(K, 0, sizeof(double) * (size_t)s->n * (size_t)J);
    for (long i = 0; i < s->n; ++i) {
        int c = or_kernel_row(o, s->x[i], s->y[i], s->z[i], s->vx[i], s->vy[i], s->vz[i], jj, kk);
        for (int e = 0; e < c; ++e) K[(size_t)i * J + jj[e]] = kk[e];
    }
}

/* y_j = sum_i w_i K_j(z_i) (eq. obs), summed in particle order. */
void or_observe(const or_obs *o, const or_particles *s, double *y)
{
    int J = or_num_obs(o);
    int jj[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    double kk[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    for (int j = 0; j < J; ++j) y[j] = 0.0;
    for (long i = 0; i < s->n; ++i) {
        int c = or_kernel_row(o, s->x[i], s->y[i], s->z[i], s->vx[i], s->vy[i], s->vz[i], jj, kk);
        for (int e = 0; e < c; ++e) y[jj[e]] += s->w[i] * kk[e];
    }
}

/* ------------------------------------------------------------------ */
/* Moving priors on the (E, x) grid (Sec. 2.3.1; signed L_z, Sec. 5)    */
/* ------------------------------------------------------------------ */

/* Energy of the circular orbit of radius R in the equatorial plane:
 * E_c(R) = phi(R,0,0) + R/2 dphi/dR. */
static double circ_energy(const or_potential *p, double R)
{
    double ax, ay, az;
    or_accel(p, R, 0.0, 0.0, &ax, &ay, &az);
    return or_phi(p, R, 0.0, 0.0) - 0.5 * R * ax;
}

/* Lc(E): angular momentum of the circular orbit of energy E, found by
 * bisection on E_c(R) = E. Returns 0 when no circular orbit has energy E
 * (E at or below the potential minimum, or E >= 0 in a potential that
 * vanishes at infinity). */
/* ------------------------------------------------------------------ */
/* Self-consistent stellar potential (Sec. 6)                          */
/* ------------------------------------------------------------------ */

/* Associated Legendre function without the Condon-Shortley phase, P_m^m = (2m-1)!!
 * (1-x^2)^(m/2); 0 outside 0 <= m <= l. */
static double plm(int l, int m, double x)
{
    if (l < 0 || m < 0 || m > l) return 0.0;
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double p0 = pmm, p1 = x * (2.0 * m + 1.0) * pmm;
    for (int ll = m + 2; ll <= l; ++ll) {
        double p2 = (x * (2.0 * ll - 1.0) * p1 - (ll + m - 1.0) * p0) / (ll - m);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

/* Factor of Y_lm: N_lm, times sqrt2 for m != 0. */
static double ylm_factor(int l, int m)
{
    int am = m < 0 ? -m : m;
    double ratio = 1.0;
    for (int i = l - am + 1; i <= l + am; ++i) ratio /= i;
    double N = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI) * ratio);
    return m == 0 ? N : sqrt(2.0) * N;
}

void or_scf_coeffs(const or_potential *p, const or_particles *s, double *a)
{
    int n = p->scf_n, nlm = (p->scf_lmax + 1) * (p->scf_lmax + 1);
    for (int q = 0; q < n * nlm; ++q) a[q] = 0.0;
    for (long i = 0; i < s->n; ++i) {
        double x = s->x[i], y = s->y[i], z = s->z[i];
        double r = sqrt(x * x + y * y + z * z);
        int k0;
        double g0, g1;
        if (r < p->scf_r[0]) {
            k0 = 0; g0 = 1.0; g1 = 0.0;
        } else if (r >= p->scf_r[n - 1]) {
            k0 = n - 1; g0 = 1.0; g1 = 0.0;
        } else {
            k0 = 0;
            while (!(r < p->scf_r[k0 + 1])) ++k0;
            double d = p->scf_r[k0 + 1] - p->scf_r[k0];
            g0 = (p->scf_r[k0 + 1] - r) / d;
            g1 = (r - p->scf_r[k0]) / d;
        }
        double ct = r > 0.0 ? z / r : 1.0;
        double ph = atan2(y, x);
        for (int l = 0; l <= p->scf_lmax; ++l)
            for (int m = -l; m <= l; ++m) {
                double Y = or_ylm(l, m, ct, ph);
                int idx = l * (l + 1) + m;
                a[k0 * nlm + idx] += s->w[i] * g0 * Y;
                if (g1 != 0.0) a[(k0 + 1) * nlm + idx] += s->w[i] * g1 * Y;
            }
    }
}

double or_scf_phi(const or_potential *p, double x, double y, double z, double *grad)
{
    int n = p->scf_n, L = p->scf_lmax, nlm = (L + 1) * (L + 1);
    double r = sqrt(x * x + y * y + z * z);
    double R = sqrt(x * x + y * y);
    double ct = r > 0.0 ? z / r : 1.0, st = r > 0.0 ? R / r : 0.0;
    double ph = atan2(y, x), cp = R > 0.0 ? x / R : 1.0, sp = R > 0.0 ? y / R : 0.0;
    double phi = 0.0, gr = 0.0, gt = 0.0, gp = 0.0;  /* dphi/dr, (1/r) dphi/dtheta, (1/(r sin)) dphi/dphi */
    for (int k = 0; k < n; ++k) {
        double rk = p->scf_r[k];
        for (int l = 0; l <= L; ++l) {
            /* radial function of a thin shell and its derivative */
            double f, df;
            if (r < rk) {
                f = pow(r, l) / pow(rk, l + 1);
                df = l > 0 ? l * pow(r, l - 1) / pow(rk, l + 1) : 0.0;
            } else {
                f = pow(rk, l) / pow(r, l + 1);
                df = -(l + 1) * pow(rk, l) / pow(r, l + 2);
            }
            double C = -4.0 * OR_PI * p->G / (2.0 * l + 1.0);
            for (int m = -l; m <= l; ++m) {
                double coef = C * p->scf_a[k * nlm + l * (l + 1) + m];
                if (coef == 0.0) continue;
                int am = m < 0 ? -m : m;
                double N = ylm_factor(l, m);
                double T = m > 0 ? cos(am * ph) : (m < 0 ? sin(am * ph) : 1.0);
                double dT = m > 0 ? -am * sin(am * ph) : (m < 0 ? am * cos(am * ph) : 0.0);
                double P = plm(l, am, ct);
                phi += coef * N * P * T * f;
                if (!grad || r == 0.0) continue;
                /* dP_l^m(cos t)/dt = ((l+m)(l-m+1) P_l^(m-1) - P_l^(m+1)) / 2, and -P_l^1 for m = 0 */
                double dP = am == 0 ? -plm(l, 1, ct)
                                    : 0.5 * ((l + am) * (l - am + 1.0) * plm(l, am - 1, ct) - plm(l, am + 1, ct));
                /* P_l^m / sin t = (P_(l-1)^(m+1) + (l+m-1)(l+m) P_(l-1)^(m-1)) / (2m), m >= 1 */
                double Ps = am == 0 ? 0.0
                                    : (plm(l - 1, am + 1, ct) + (l + am - 1.0) * (l + am) * plm(l - 1, am - 1, ct)) /
                                          (2.0 * am);
                gr += coef * N * P * T * df;
                gt += coef * N * dP * T * f / r;
                gp += coef * N * Ps * dT * f / r;
            }
        }
    }
    if (grad) {
        if (r == 0.0) {
            grad[0] = grad[1] = grad[2] = 0.0;
        } else {
            /* e_r = (st cp, st sp, ct), e_theta = (ct cp, ct sp, -st), e_phi = (-sp, cp, 0) */
            grad[0] = gr * st * cp + gt * ct * cp - gp * sp;
            grad[1] = gr * st * sp + gt * ct * sp + gp * cp;
            grad[2] = gr * ct - gt * st;
        }
    }
    (void)ph;
    return phi;
}

/* dK/dv_los of one kernel at line-of-sight velocity v in aperture p of group G (0 for the
 * surface mass and the a_lm). The Gauss-Hermite kernel is c_n H_n(nu) e^(-nu^2/2) with
 * c_n = 2 sqrt(pi) (2^(n+1) pi n!)^(-1/2) and nu = (v - V_p)/sigma_p, and
 * d/dnu [H_n e^(-nu^2/2)] = (2n H_(n-1) - nu H_n) e^(-nu^2/2). */
static double kernel_dv(const or_group *G, int kind, int p, double v)
{
    if (kind == OR_V2) return 2.0 * v;
    if (kind >= OR_GH0 && kind <= OR_GH0 + 6) {
        int nn = kind - OR_GH0;
        double nfact = 1.0;
        for (int k = 2; k <= nn; ++k) nfact *= k;
        double c = 2.0 * sqrt(OR_PI) / sqrt(pow(2.0, nn + 1) * OR_PI * nfact);
        double nu = (v - G->Vp[p]) / G->sp[p];
        double Hn = or_hermite(nn, nu), Hm = nn > 0 ? or_hermite(nn - 1, nu) : 0.0;
        return c * (2.0 * nn * Hm - nu * Hn) * exp(-0.5 * nu * nu) / G->sp[p];
    }
    return 0.0;
}

void or_observe_dlnups(const or_obs *o, const or_particles *s, double *D)
{
    int J = or_num_obs(o);
    for (int j = 0; j < J; ++j) D[j] = 0.0;
    for (long i = 0; i < s->n; ++i) {
        double X, Y, v;
        project(o->incl_deg, s->x[i], s->y[i], s->z[i], s->vy[i], s->vz[i], &X, &Y, &v);
        int off = 0;
        for (int g = 0; g < o->n_groups; ++g) {
            const or_group *G = &o->g[g];
            double area;
            int p = G->geometry == OR_SHELLS ? -1 : aperture(G, X, Y, &area);
            if (p >= 0)
                for (int q = 0; q < G->n_kinds; ++q)
                    D[off + q * G->n_ap + p] += 0.5 * s->w[i] * v * kernel_dv(G, G->kinds[q], p, v);
            off += G->n_kinds * G->n_ap;
        }
    }
}

double or_circular_L(const or_potential *p, double E)
{
    if (p->kind != OR_POT_LOG && p->kind != OR_POT_SCF && E >= 0.0) return 0.0;
    if (E <= circ_energy(p, 0.0)) return 0.0;
    double hi = 1.0;
    while (circ_energy(p, hi) <= E && hi < 1e15) hi *= 2.0;
    double lo = 0.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (circ_energy(p, mid) <= E)
            lo = mid;
        else
            hi = mid;
    }
    double R = 0.5 * (lo + hi);
    double ax, ay, az;
    or_accel(p, R, 0.0, 0.0, &ax, &ay, &az);
    double vc2 = -R * ax;
    return R * sqrt(vc2);
}

/* Cell (k, l) -> k*nx + l of one particle: E bin k from the chosen spacing
 * between Emin and Emax (clamped), circularity bin l from x = L/Lc(E)
 * (x = Lz/Lc(E) on [-1, 1] for the signed variant). */
int or_cell(const or_potential *p, const or_prior *g, double x, double y, double z,
            double vx, double vy, double vz, double *E_out, double *xc_out)
{
    double E = 0.5 * (vx * vx + vy * vy + vz * vz) + or_phi(p, x, y, z);
    double Lx = y * vz - z * vy, Ly = z * vx - x * vz, Lz = x * vy - y * vx;
    double L = g->signed_lz ? Lz : sqrt(Lx * Lx + Ly * Ly + Lz * Lz);
    double Lc = or_circular_L(p, E);
    double xc = (Lc > 0.0) ? L / Lc : 0.0;
    double xmin = g->signed_lz ? -1.0 : 0.0;
    if (xc < xmin) xc = xmin;
    if (xc > 1.0) xc = 1.0;

    double f;
    if (g->e_spacing == OR_E_LOGNEG) {
        if (E >= 0.0)
            f = 1.0;
        else
            f = (log(-E) - log(-g->Emin)) / (log(-g->Emax) - log(-g->Emin));
    } else if (g->e_spacing == OR_E_EXP) {
        f = (exp(E) - exp(g->Emin)) / (exp(g->Emax) - exp(g->Emin));
    } else {
        f = (E - g->Emin) / (g->Emax - g->Emin);
    }
    double fk = floor(f * g->nE);
    int k = fk < 0.0 ? 0 : (fk >= g->nE ? g->nE - 1 : (int)fk);
    double fl = floor((xc - xmin) / (1.0 - xmin) * g->nx);
    int l = fl < 0.0 ? 0 : (fl >= g->nx ? g->nx - 1 : (int)fl);
    if (E_out) *E_out = E;
    if (xc_out) *xc_out = xc;
    return k * g->nx + l;
}

/* ------------------------------------------------------------------ */
/* Force of change (eq. modFOC with eq. S+ or eq. entropy)             */
/* ------------------------------------------------------------------ */

/* The bracket of eq. modFOC for one particle:
 * mu dS/dw_i - sum_j K_ij Delta_j / sigma_j. */
double or_force(const or_obs *o, const or_params *par, int mode, double w_i, double what_i,
                double x, double y, double z, double vx, double vy, double vz,
                const double *delta, const double *sig)
{
    int jj[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    double kk[2 * OR_MAX_GROUPS * OR_MAX_KINDS];
    int c = or_kernel_row(o, x, y, z, vx, vy, vz, jj, kk);
    double data = 0.0;
    for (int e = 0; e < c; ++e) data += kk[e] * delta[jj[e]] / sig[jj[e]];
    /* a smoothed prior can be <= 0, where -ln(w/what) is undefined: no entropy force there */
    double dS = what_i > 0.0 ? -log(w_i / what_i) : 0.0;
    if (mode == OR_GWR) dS -= 1.0;
    return par->mu * dS - data;
}

static void residuals(int J, const double *Y, const double *sig, or_state *st)
{
    double c2 = 0.0;
    for (int j = 0; j < J; ++j) {
        st->delta[j] = (st->ytil[j] - Y[j]) / sig[j];
        c2 += st->delta[j] * st->delta[j];
    }
    st->chi2 = c2;
}

void or_window_means(int nE, int nx, int hE, int hx, const double *sum, const long *count,
                     double *mean)
{
    for (int k = 0; k < nE; ++k)
        for (int l = 0; l < nx; ++l) {
            double ws = 0.0;
            long nc = 0;
            for (int k2 = k - hE; k2 <= k + hE; ++k2)
                for (int l2 = l - hx; l2 <= l + hx; ++l2) {
                    if (k2 < 0 || k2 >= nE || l2 < 0 || l2 >= nx) continue;
                    ws += sum[k2 * nx + l2];
                    nc += count[k2 * nx + l2];
                }
            mean[k * nx + l] = nc > 0 ? ws / (double)nc : 0.0;
        }
}

void or_init(const or_obs *o, const double *Y, const double *sig, const or_prior *g,
             const or_particles *s, or_state *st)
{
    int J = or_num_obs(o);
    double W0 = 0.0;
    for (long i = 0; i < s->n; ++i) W0 += s->w[i];
    st->W0 = W0;
    or_observe(o, s, st->yraw);
    for (int j = 0; j < J; ++j) st->ytil[j] = st->yraw[j];
    residuals(J, Y, sig, st);
    for (long i = 0; i < s->n; ++i) {
        st->what[i] = W0 / (double)s->n;
        st->cell[i] = 0;
    }
    if (g->mode == OR_MPR) {
        for (int c = 0; c < g->nE * g->nx; ++c) {
            st->grid_mean[c] = 0.0;
            st->grid_count[c] = 0;
            if (st->grid_raw) st->grid_raw[c] = 0.0;
        }
    }
    st->lambda = 0.0;
    st->t = 0;
}

int or_run(const or_potential *p, const or_obs *o, const double *Y, const double *sig,
           const or_prior *g, const or_params *par, or_particles *s, or_state *st, long nsteps)
{
    int J = or_num_obs(o);
    int ncell = g->nE * g->nx;
    double *gsum = NULL;
    if (g->mode == OR_MPR) {
        gsum = (double *)malloc(sizeof(double) * (size_t)ncell);
        if (!gsum) return OR_EARG;
    }
    if (g->mode == OR_MPR && (g->window_E < 0 || g->window_x < 0 ||
                              (g->smoothing && (g->window_E > 0 || g->window_x > 0)))) {
        free(gsum);
        return OR_EARG;
    }
    int status = OR_OK;
    double *D = NULL;
    if (p->kind == OR_POT_SCF) {
        D = (double *)malloc(sizeof(double) * (size_t)(J > 0 ? J : 1));
        if (!D) {
            free(gsum);
            return OR_EARG;
        }
        /* the expansion of the initial particles moves them in the first step */
        if (st->t == 0) or_scf_coeffs(p, s, p->scf_a);
    }
    for (long step = 0; step < nsteps; ++step) {
        long t = st->t + 1;
        /* 1. push */
        or_leapfrog(p, s, par->dt);
        /* 2. observe */
        or_observe(o, s, st->yraw);
        /* 3. temporal smoothing */
        for (int j = 0; j < J; ++j) st->ytil[j] += par->alpha * (st->yraw[j] - st->ytil[j]);
        /* 4. residuals and chi^2 */
        residuals(J, Y, sig, st);
        /* 5. moving priors */
        if (g->mode == OR_MPR && (t - 1) % g->update_every == 0) {
            for (int c = 0; c < ncell; ++c) {
                gsum[c] = 0.0;
                st->grid_count[c] = 0;
            }
            for (long i = 0; i < s->n; ++i) {
                int c = or_cell(p, g, s->x[i], s->y[i], s->z[i], s->vx[i], s->vy[i], s->vz[i],
                                NULL, NULL);
                st->cell[i] = c;
                gsum[c] += s->w[i];
                st->grid_count[c] += 1;
            }
            /* Sec. 2.3.1: the mean weight of the cell; Sec. 7 (grid-less variant): the mean
             * weight of the particles in the window of cells centred on the particle's own */
            or_window_means(g->nE, g->nx, g->window_E, g->window_x, gsum, st->grid_count,
                            st->grid_mean);
            if (g->smoothing) {
                /* Sec. 2.3.2: the priors are the spline fit of the grid of cell means */
                if (st->grid_raw)
                    for (int c = 0; c < ncell; ++c) st->grid_raw[c] = st->grid_mean[c];
                memcpy(gsum, st->grid_mean, sizeof(double) * (size_t)ncell);
                if (or_smooth_grid(g->nE, g->nx, gsum, g->lambda, st->grid_mean, &st->lambda) != OR_OK) {
                    status = OR_EARG;
                    break;
                }
            }
            for (long i = 0; i < s->n; ++i) st->what[i] = st->grid_mean[st->cell[i]];
        }
        /* 5b. self-consistent potential (Sec. 6): on the same schedule as the priors, the
         * mass-to-light ratio follows the chi^2 gradient (velocities scaling as
         * Upsilon^(1/2)), d ln Upsilon/dt = -eps_ups sum_j Delta_j/sigma_j D_j, over the
         * update_every steps to the next update; then the expansion is rebuilt from the
         * particles as they are now. Both act from the next step on. */
        if (p->kind == OR_POT_SCF && (t - 1) % g->update_every == 0) {
            if (par->eps_ups > 0.0) {
                or_observe_dlnups(o, s, D);
                double G = 0.0;
                for (int j = 0; j < J; ++j) G += st->delta[j] / sig[j] * D[j];
                *p->scf_ups *= exp(-par->eps_ups * g->update_every * par->dt * G);
            }
            or_scf_coeffs(p, s, p->scf_a);
        }
        /* 6. force of change */
        if (t > par->n_relax) {
            for (long i = 0; i < s->n; ++i) {
                /* w = 0 (reachable by underflow) is a fixed point of eq. modFOC */
                if (s->w[i] == 0.0) continue;
                double F = or_force(o, par, g->mode, s->w[i], st->what[i], s->x[i], s->y[i],
                                    s->z[i], s->vx[i], s->vy[i], s->vz[i], st->delta, sig);
                double h = par->dt * par->eps * F;
                double wn = (par->update_rule == OR_UPDATE_EULER) ? s->w[i] * (1.0 + h)
                                                                  : s->w[i] * exp(h);
                if (!isfinite(wn) || wn < 0.0 ||
                    (par->update_rule == OR_UPDATE_EULER && wn <= 0.0))
                    status = OR_EWEIGHT;
                s->w[i] = wn;
            }
        }
        /* 7. renormalisation to the initial total weight */
        if (par->renormalize) {
            double W = 0.0;
            for (long i = 0; i < s->n; ++i) W += s->w[i];
            for (long i = 0; i < s->n; ++i) s->w[i] *= st->W0 / W;
        }
        st->t = t;
        if (status != OR_OK) break;
    }
    free(gsum);
    free(D);
    return status;
}

/* ------------------------------------------------------------------ */
/* Target observables from a target particle realisation (Sec. 3.3)    */
/* ------------------------------------------------------------------ */

/* For every aperture: luminosity l_p, then V_p and sigma_p from the mean and
 * rms line-of-sight velocity, corrected with dh1 = -dV/(sqrt2 sigma),
 * dh2 = -dsigma/(sqrt2 sigma) (eq. h1h2) until h1 = h2 = 0; then the target
 * values Y_j and errors sigma_j:
 *   mass:  Y = l/A,        sigma = err Y               (err relative)
 *   v2:    Y = l v_rms^2,  sigma = 2 err Y             (err relative on v_rms)
 *   GH n:  Y = l h_n,      sigma = l err               (err absolute on h_n)
 * with Gaussian noise sigma*noise added in the observable's own variable
 * (Y(1+err g), l (v_rms(1+err g))^2, l (h_n + err g)) when noise is given.
 * Vp_out/sp_out hold sum over groups of n_ap entries; the obs descriptor's
 * Vp/sp pointers are set to them. */
int or_build_targets(or_obs *o, const or_particles *tg, const double *err,
                     const double *noise, double *Vp_out, double *sp_out,
                     double *Y_out, double *sig_out, int *iters_out)
{
    int J = or_num_obs(o);
    int apoff = 0;
    int maxit = 0;
    int nap_total = 0;
    for (int g = 0; g < o->n_groups; ++g) nap_total += o->g[g].n_ap;
    double *lum = (double *)calloc((size_t)nap_total, sizeof(double));
    for (int g = 0; g < o->n_groups; ++g) {
        or_group *G = &o->g[g];
        int n_ap = G->n_ap;
        double *l = (double *)calloc((size_t)n_ap, sizeof(double));
        double *m1 = (double *)calloc((size_t)n_ap, sizeof(double));
        double *m2 = (double *)calloc((size_t)n_ap, sizeof(double));
        double *b1 = (double *)calloc((size_t)n_ap, sizeof(double));
        double *b2 = (double *)calloc((size_t)n_ap, sizeof(double));
        double *V = Vp_out + apoff, *S = sp_out + apoff;
        int has_gh = 0;
        for (int k = 0; k < G->n_kinds; ++k) has_gh |= G->kinds[k] >= OR_GH0 && G->kinds[k] < OR_ALM0;
        for (long i = 0; G->geometry != OR_SHELLS && i < tg->n; ++i) {
            double X, Y, v, area;
            project(o->incl_deg, tg->x[i], tg->y[i], tg->z[i], tg->vy[i], tg->vz[i], &X, &Y, &v);
            int p = aperture(G, X, Y, &area);
            if (p < 0) continue;
            l[p] += tg->w[i];
            m1[p] += tg->w[i] * v;
            m2[p] += tg->w[i] * v * v;
        }
        int bad = 0;
        for (int p = 0; p < n_ap; ++p) {
            if (l[p] > 0.0) {
                V[p] = m1[p] / l[p];
                double var = m2[p] / l[p] - V[p] * V[p];
                S[p] = var > 0.0 ? sqrt(var) : 0.0;
            } else {
                V[p] = 0.0;
                S[p] = 1.0;
            }
            if (has_gh && !(l[p] > 0.0 && S[p] > 0.0)) bad = 1;
            if (G->geometry == OR_SHELLS) {
                /* shells: l[p] = sum of (w gamma_p)^2, the shot noise of the coefficients */
                l[p] = 0.0;
            }
        }
        G->Vp = V;
        G->sp = S;
        if (G->geometry == OR_SHELLS) {
            for (long i = 0; i < tg->n; ++i) {
                double r = sqrt(tg->x[i] * tg->x[i] + tg->y[i] * tg->y[i] + tg->z[i] * tg->z[i]);
                int kp[2];
                double gp[2];
                int np = or_cic(G, r, kp, gp);
                for (int a = 0; a < np; ++a) l[kp[a]] += (tg->w[i] * gp[a]) * (tg->w[i] * gp[a]);
            }
        }
        for (int p = 0; p < n_ap; ++p) lum[apoff + p] = l[p];
        if (bad) {
            free(l); free(m1); free(m2); free(b1); free(b2); free(lum);
            return OR_ETARGET;
        }
        if (has_gh) {
            int it;
            for (it = 0; it < 200; ++it) {
                for (int p = 0; p < n_ap; ++p) b1[p] = b2[p] = 0.0;
                for (long i = 0; i < tg->n; ++i) {
                    double X, Y, v, area;
                    project(o->incl_deg, tg->x[i], tg->y[i], tg->z[i], tg->vy[i], tg->vz[i],
                            &X, &Y, &v);
                    int p = aperture(G, X, Y, &area);
                    if (p < 0) continue;
                    double nu = (v - V[p]) / S[p];
                    b1[p] += tg->w[i] * or_gh_kernel(1, nu);
                    b2[p] += tg->w[i] * or_gh_kernel(2, nu);
                }
                double worst = 0.0;
                for (int p = 0; p < n_ap; ++p) {
                    double h1 = b1[p] / l[p], h2 = b2[p] / l[p];
                    if (fabs(h1) > worst) worst = fabs(h1);
                    if (fabs(h2) > worst) worst = fabs(h2);
                    double s_old = S[p];
                    V[p] += sqrt(2.0) * s_old * h1;
                    S[p] += sqrt(2.0) * s_old * h2;
                }
                if (worst <= 1e-12) break;
            }
            if (it > maxit) maxit = it;
        }
        apoff += n_ap;
        free(m1); free(m2); free(b1); free(b2);
        free(l);
    }
    /* final observables with the fitted Gaussian parameters */
    double *y = (double *)calloc((size_t)J, sizeof(double));
    or_observe(o, tg, y);
    int off = 0;
    apoff = 0;
    for (int g = 0; g < o->n_groups; ++g) {
        const or_group *G = &o->g[g];
        for (int k = 0; k < G->n_kinds; ++k) {
            for (int p = 0; p < G->n_ap; ++p) {
                int j = off + k * G->n_ap + p;
                int kind = G->kinds[k];
                double gn = noise ? noise[j] : 0.0;
                if (kind >= OR_ALM0) {
                    /* shot noise of a_lm,k for an isotropic realisation, sum (w gamma)^2 / (4 pi),
                     * scaled by err */
                    sig_out[j] = err[j] * sqrt(lum[apoff + p] / (4.0 * OR_PI));
                    Y_out[j] = y[j] + sig_out[j] * gn;
                } else if (kind == OR_MASS) {
                    sig_out[j] = err[j] * y[j];
                    Y_out[j] = y[j] * (1.0 + err[j] * gn);
                } else {
                    double lp = lum[apoff + p]; /* luminosity of the aperture */
                    if (kind == OR_V2) {
                        double vrms = sqrt(y[j] / lp);
                        double vo = vrms * (1.0 + err[j] * gn);
                        sig_out[j] = 2.0 * err[j] * y[j];
                        Y_out[j] = lp * vo * vo;
                    } else {
                        double h = y[j] / lp;
                        sig_out[j] = lp * err[j];
                        Y_out[j] = lp * (h + err[j] * gn);
                    }
                }
            }
        }
        off += G->n_kinds * G->n_ap;
        apoff += G->n_ap;
    }
    free(y);
    free(lum);
    if (iters_out) *iters_out = maxit;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Smoothing of the grid of priors (Sec. 2.3.2)                        */

/* adds w r r^T to P for the stencil row r (nz entries idx[], coef[]) */
static void add_outer(double *P, int n, int nz, const int *idx, const double *coef, double w)
{
    for (int a = 0; a < nz; ++a)
        for (int b = 0; b < nz; ++b) P[(size_t)idx[a] * n + idx[b]] += w * coef[a] * coef[b];
}

void or_smooth_penalty(int nE, int nx, double *P)
{
    int n = nE * nx;
    for (size_t q = 0; q < (size_t)n * n; ++q) P[q] = 0.0;
    int idx[4];
    double coef[4];
    /* f_EE = f(k-1,l) - 2 f(k,l) + f(k+1,l) */
    for (int k = 1; k + 1 < nE; ++k)
        for (int l = 0; l < nx; ++l) {
            idx[0] = (k - 1) * nx + l; idx[1] = k * nx + l; idx[2] = (k + 1) * nx + l;
            coef[0] = 1.0; coef[1] = -2.0; coef[2] = 1.0;
            add_outer(P, n, 3, idx, coef, 1.0);
        }
    /* f_xx = f(k,l-1) - 2 f(k,l) + f(k,l+1) */
    for (int k = 0; k < nE; ++k)
        for (int l = 1; l + 1 < nx; ++l) {
            idx[0] = k * nx + l - 1; idx[1] = k * nx + l; idx[2] = k * nx + l + 1;
            coef[0] = 1.0; coef[1] = -2.0; coef[2] = 1.0;
            add_outer(P, n, 3, idx, coef, 1.0);
        }
    /* f_Ex at the corner between (k,l) and (k+1,l+1), weighted 2 */
    for (int k = 0; k + 1 < nE; ++k)
        for (int l = 0; l + 1 < nx; ++l) {
            idx[0] = (k + 1) * nx + l + 1; idx[1] = (k + 1) * nx + l; idx[2] = k * nx + l + 1; idx[3] = k * nx + l;
            coef[0] = 1.0; coef[1] = -1.0; coef[2] = -1.0; coef[3] = 1.0;
            add_outer(P, n, 4, idx, coef, 2.0);
        }
}

/* Cholesky factor L (lower) of the SPD matrix M in place; returns 0 on success */
static int cholesky(double *M, int n)
{
    for (int j = 0; j < n; ++j) {
        double d = M[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
        if (!(d > 0.0)) return 1;
        d = sqrt(d);
        M[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = M[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
            M[(size_t)i * n + j] = v / d;
        }
    }
    return 0;
}

/* solves L L^T x = b (x may alias b) */
static void chol_solve(const double *L, int n, const double *b, double *x)
{
    for (int i = 0; i < n; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * x[k];
        x[i] = v / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double v = x[i];
        for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * x[k];
        x[i] = v / L[(size_t)i * n + i];
    }
}

/* f = (I + lambda P)^-1 y and, when gcv is not NULL, the GCV score
 * n |y - f|^2 / (n - tr A)^2 with tr A from the diagonal of the explicit inverse */
static int smooth_at(const double *P, int n, const double *y, double lambda, double *f, double *gcv,
                     double *M, double *col)
{
    for (size_t q = 0; q < (size_t)n * n; ++q) M[q] = lambda * P[q];
    for (int i = 0; i < n; ++i) M[(size_t)i * n + i] += 1.0;
    if (cholesky(M, n)) return OR_EARG;
    chol_solve(M, n, y, f);
    if (gcv) {
        double tr = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < n; ++k) col[k] = (k == i) ? 1.0 : 0.0;
            chol_solve(M, n, col, col);
            tr += col[i];
        }
        double rss = 0.0;
        for (int i = 0; i < n; ++i) rss += (y[i] - f[i]) * (y[i] - f[i]);
        *gcv = (double)n * rss / ((n - tr) * (n - tr));
    }
    return OR_OK;
}

/* GCV choice of lambda (Sec. 2.3.2): the minimum of the GCV score over t = log10 lambda in
 * [-4, 6] by a plain golden-section search of 40 steps (interval 4e-8 decades), which
 * assumes the score is unimodal there. Any lambda whose score equals the minimum to rounding
 * is an equally valid choice: when the minimum is flat, codes that evaluate the score by
 * other means may pick a different one. */
int or_smooth_grid(int nE, int nx, const double *y, double lambda, double *f, double *lambda_out)
{
    if (nE < 3 || nx < 3) return OR_EARG;
    int n = nE * nx;
    double *P = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *M = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *col = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = OR_OK;
    if (!P || !M || !col) rc = OR_EARG;
    if (rc == OR_OK) {
        or_smooth_penalty(nE, nx, P);
        if (!(lambda > 0.0)) {
            const double g = 0.5 * (sqrt(5.0) - 1.0);
            double a = -4.0, b = 6.0;
            double c = b - g * (b - a), d = a + g * (b - a), vc, vd;
            rc = smooth_at(P, n, y, pow(10.0, c), f, &vc, M, col);
            if (rc == OR_OK) rc = smooth_at(P, n, y, pow(10.0, d), f, &vd, M, col);
            for (int it = 0; rc == OR_OK && it < 40; ++it) {
                if (vc <= vd) {
                    b = d; d = c; vd = vc;
                    c = b - g * (b - a);
                    rc = smooth_at(P, n, y, pow(10.0, c), f, &vc, M, col);
                } else {
                    a = c; c = d; vc = vd;
                    d = a + g * (b - a);
                    rc = smooth_at(P, n, y, pow(10.0, d), f, &vd, M, col);
                }
            }
            lambda = pow(10.0, 0.5 * (a + b));
        }
        if (rc == OR_OK) rc = smooth_at(P, n, y, lambda, f, NULL, M, col);
    }
    if (lambda_out) *lambda_out = lambda;
    free(P);
    free(M);
    free(col);
    return rc;
}

/* The GCV score n |y - f|^2 / (n - tr A)^2 of the fit f = A y = (I + lambda P)^-1 y. */
int or_smooth_gcv(int nE, int nx, const double *y, double lambda, double *score)
{
    if (nE < 3 || nx < 3 || !(lambda > 0.0)) return OR_EARG;
    int n = nE * nx;
    double *P = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *M = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *col = (double *)malloc(sizeof(double) * (size_t)n);
    double *f = (double *)malloc(sizeof(double) * (size_t)n);
    int rc = (P && M && col && f) ? OR_OK : OR_EARG;
    if (rc == OR_OK) {
        or_smooth_penalty(nE, nx, P);
        rc = smooth_at(P, n, y, lambda, f, score, M, col);
    }
    free(P);
    free(M);
    free(col);
    free(f);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Diagnostics (Sec. 4.1: Delta_grid, intrinsic kinematics in          */
/* spherical bins; Sec. 5, Fig. res: weight rms in the (E, x) cells)   */
/* ------------------------------------------------------------------ */

int or_sph_bin(const or_sph_grid *g, double x, double y, double z)
{
    double r = sqrt(x * x + y * y + z * z);
    if (!(r < g->r_max)) return -1;
    int ir;
    if (r < g->r_min) {
        ir = 0;
    } else {
        double f = (log(r) - log(g->r_min)) / (log(g->r_max) - log(g->r_min));
        ir = 1 + (int)floor(f * (g->n_r - 1));
        if (ir > g->n_r - 1) ir = g->n_r - 1;
    }
    double ct = r > 0.0 ? z / r : 1.0;
    int ic = (int)floor((ct + 1.0) * 0.5 * g->n_ct);
    if (ic < 0) ic = 0;
    if (ic > g->n_ct - 1) ic = g->n_ct - 1;
    double phi = atan2(y, x);
    int ip = (int)floor((phi + M_PI) / (2.0 * M_PI) * g->n_phi);
    if (ip < 0) ip = 0;
    if (ip > g->n_phi - 1) ip = g->n_phi - 1;
    return (ir * g->n_ct + ic) * g->n_phi + ip;
}

void or_sph_velocity(double x, double y, double z, double vx, double vy, double vz,
                     double *vr, double *vth, double *vph)
{
    double R = sqrt(x * x + y * y);
    double r = sqrt(R * R + z * z);
    double cp = 1.0, sp = 0.0;  /* azimuth 0 on the z axis */
    if (R > 0.0) {
        cp = x / R;
        sp = y / R;
    }
    double ct = 1.0, st = 0.0;  /* e_r = e_z at the centre */
    if (r > 0.0) {
        ct = z / r;
        st = R / r;
    }
    /* e_r = (st cp, st sp, ct), e_theta = (ct cp, ct sp, -st), e_phi = (-sp, cp, 0) */
    *vr = vx * st * cp + vy * st * sp + vz * ct;
    *vth = vx * ct * cp + vy * ct * sp - vz * st;
    *vph = -vx * sp + vy * cp;
}

void or_kin_sums(const or_sph_grid *g, const or_particles *s, double *sums, long *counts)
{
    long nb = (long)g->n_r * g->n_ct * g->n_phi;
    for (long b = 0; b < nb; ++b) {
        counts[b] = 0;
        for (int q = 0; q < OR_KIN_SUMS; ++q) sums[b * OR_KIN_SUMS + q] = 0.0;
    }
    for (long i = 0; i < s->n; ++i) {
        int b = or_sph_bin(g, s->x[i], s->y[i], s->z[i]);
        if (b < 0) continue;
        double v[3];
        or_sph_velocity(s->x[i], s->y[i], s->z[i], s->vx[i], s->vy[i], s->vz[i], &v[0], &v[1], &v[2]);
        double w = s->w[i];
        double *o = sums + (long)b * OR_KIN_SUMS;
        o[0] += w;
        for (int c = 0; c < 3; ++c) {
            o[1 + c] += w * v[c];
            o[4 + c] += w * v[c] * v[c];
        }
        counts[b] += 1;
    }
}

void or_kin_moments(long nbins, const double *sums, const long *counts, long min_count,
                    double *mean, double *disp, int *valid)
{
    for (long b = 0; b < nbins; ++b) {
        const double *o = sums + b * OR_KIN_SUMS;
        int ok = counts[b] >= min_count && counts[b] > 0 && o[0] > 0.0;
        valid[b] = ok;
        for (int c = 0; c < 3; ++c) {
            double m = ok ? o[1 + c] / o[0] : 0.0;
            double v2 = ok ? o[4 + c] / o[0] - m * m : 0.0;
            mean[3 * b + c] = m;
            disp[3 * b + c] = v2 > 0.0 ? sqrt(v2) : 0.0;
        }
    }
}

long or_delta_kin(long nbins, const double *sums_m, const long *counts_m, const double *sums_t,
                  const long *counts_t, long min_count, double *out)
{
    double *mm = malloc(sizeof(double) * 3 * nbins), *dm = malloc(sizeof(double) * 3 * nbins);
    double *mt = malloc(sizeof(double) * 3 * nbins), *dt = malloc(sizeof(double) * 3 * nbins);
    int *vm = malloc(sizeof(int) * nbins), *vt = malloc(sizeof(int) * nbins);
    or_kin_moments(nbins, sums_m, counts_m, min_count, mm, dm, vm);
    or_kin_moments(nbins, sums_t, counts_t, min_count, mt, dt, vt);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    long used = 0;
    for (long b = 0; b < nbins; ++b) {
        if (!(vm[b] && vt[b])) continue;
        for (int c = 0; c < 3; ++c) {
            double d1 = mm[3 * b + c] - mt[3 * b + c];
            double d2 = dm[3 * b + c] - dt[3 * b + c];
            acc[c] += d1 * d1;
            acc[3 + c] += d2 * d2;
        }
        used += 1;
    }
    double all = 0.0;
    for (int q = 0; q < 6; ++q) {
        out[q] = used > 0 ? sqrt(acc[q] / used) : 0.0;
        all += acc[q];
    }
    out[6] = used > 0 ? sqrt(all / (6.0 * used)) : 0.0;
    free(mm); free(dm); free(mt); free(dt); free(vm); free(vt);
    return used;
}

void or_grid_weights(const or_potential *p, const or_prior *g, const or_particles *s,
                     double *wsum, double *wdev2, long *count)
{
    int nc = g->nE * g->nx;
    int *cell = malloc(sizeof(int) * (s->n > 0 ? s->n : 1));
    for (int c = 0; c < nc; ++c) {
        wsum[c] = 0.0;
        wdev2[c] = 0.0;
        count[c] = 0;
    }
    for (long i = 0; i < s->n; ++i) {
        cell[i] = or_cell(p, g, s->x[i], s->y[i], s->z[i], s->vx[i], s->vy[i], s->vz[i], NULL, NULL);
        wsum[cell[i]] += s->w[i];
        count[cell[i]] += 1;
    }
    for (long i = 0; i < s->n; ++i) {
        int c = cell[i];
        double d = s->w[i] - wsum[c] / (double)count[c];
        wdev2[c] += d * d;
    }
    free(cell);
}

double or_delta_grid(int ncell, const double *w_model, const double *w_target)
{
    double tm = 0.0, tt = 0.0;
    for (int c = 0; c < ncell; ++c) {
        tm += w_model[c];
        tt += w_target[c];
    }
    if (!(tm > 0.0) || !(tt > 0.0)) return 0.0;
    double num = 0.0, den = 0.0;
    for (int c = 0; c < ncell; ++c) {
        double wt = w_target[c] / tt, wm = w_model[c] / tm;
        if (!(wt > 0.0)) continue;
        double r = (wt - wm) / wt;
        num += wt * r * r;
        den += wt;
    }
    return sqrt(num / den);
}

double or_weight_rms(int ncell, const double *wdev2, const long *count, long min_count)
{
    double s = 0.0;
    long n = 0;
    for (int c = 0; c < ncell; ++c) {
        if (count[c] <= min_count) continue;
        s += wdev2[c];
        n += count[c];
    }
    return n > 0 ? sqrt(s / (double)n) : 0.0;
}
