/*
 * etics_oracle.c -- plain FP64 CPU oracle of the SCF and MEX force
 * calculation (Meiron et al., "Expansion Techniques for Collisionless
 * Stellar Dynamical Simulations").
 *
 * TEST INFRASTRUCTURE ONLY: see etics_oracle.h.  Written for reading, not for
 * speed: every sum is the plain definition, summed serially in particle order
 * unless a comment says otherwise.  The only parallelism is over independent
 * evaluation points (each point's own sum is unchanged by it).
 *
 * Compile with -O2 -ffp-contract=off so that every product and sum is rounded
 * exactly as written.
 */
#include "etics_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Special functions                                                         */
/* ------------------------------------------------------------------------ */

/* Gegenbauer polynomials C_k^alpha(x), k = 0..n, by the textbook three-term
 * recursion  k C_k = 2 (k + alpha - 1) x C_{k-1} - (k + 2 alpha - 2) C_{k-2}. */
static void gegenbauer_all(int n, double alpha, double x, double *C)
{
    C[0] = 1.0;
    if (n >= 1) C[1] = 2.0 * alpha * x;
    for (int k = 2; k <= n; ++k)
        C[k] = (2.0 * (k + alpha - 1.0) * x * C[k - 1]
                - (k + 2.0 * alpha - 2.0) * C[k - 2]) / k;
}

/* Radial potential bases (Sec. 2.5), scale length 1.
 *
 * basis 0, Hernquist-Ostriker (HO92; the Hernquist model is the zeroth term):
 *   phi_nl(r) = - r^l / (1+r)^(2l+1) * C_n^(2l+3/2)(xi),  xi = (r-1)/(r+1),
 *   dxi/dr = 2/(1+r)^2.
 * basis 1, Clutton-Brock (CB73; the Plummer model is the zeroth term):
 *   phi_nl(r) = - r^l / (1+r^2)^(l+1/2) * C_n^(l+1)(xi),  xi = (r^2-1)/(r^2+1),
 *   dxi/dr = 4r/(1+r^2)^2.
 * Radial derivatives use d/dxi C_n^alpha = 2 alpha C_{n-1}^(alpha+1).  Fills
 * phi[0..n_max] (and dphi if non-NULL). */
static double basis_alpha(int basis, int l)
{
    return basis == 0 ? 2.0 * l + 1.5 : l + 1.0;
}

static void radial_all_b(int basis, int n_max, int l, double r, double *phi, double *dphi)
{
    double alpha = basis_alpha(basis, l);
    double xi, f, dfdr, dxidr;
    /* r^l with 0^0 = 1 */
    double rl = (l == 0) ? 1.0 : pow(r, (double)l);
    if (basis == 0) {
        xi = (r - 1.0) / (r + 1.0);
        f = -rl / pow(1.0 + r, 2.0 * l + 1.0);
        /* df/dr = -[l r^(l-1) (1+r)^-(2l+1) - (2l+1) r^l (1+r)^-(2l+2)] */
        dfdr = (2.0 * l + 1.0) * rl / pow(1.0 + r, 2.0 * l + 2.0);
        if (l > 0) dfdr -= l * pow(r, l - 1.0) / pow(1.0 + r, 2.0 * l + 1.0);
        dxidr = 2.0 / ((1.0 + r) * (1.0 + r));
    } else {
        double q = 1.0 + r * r;
        xi = (r * r - 1.0) / q;
        f = -rl / pow(q, l + 0.5);
        /* df/dr = -[l r^(l-1) q^-(l+1/2) - (2l+1) r^(l+1) q^-(l+3/2)] */
        dfdr = (2.0 * l + 1.0) * rl * r / pow(q, l + 1.5);
        if (l > 0) dfdr -= l * pow(r, l - 1.0) / pow(q, l + 0.5);
        dxidr = 4.0 * r / (q * q);
    }
    double C[64], Cp[64];
    gegenbauer_all(n_max, alpha, xi, C);
    for (int n = 0; n <= n_max; ++n) phi[n] = f * C[n];
    if (!dphi) return;
    gegenbauer_all(n_max, alpha + 1.0, xi, Cp);
    for (int n = 0; n <= n_max; ++n) {
        double dC = (n == 0) ? 0.0 : 2.0 * alpha * Cp[n - 1];
        dphi[n] = dfdr * C[n] + f * dC * dxidr;
    }
}

static void radial_all(int n_max, int l, double r, double *phi, double *dphi)
{
    radial_all_b(0, n_max, l, r, phi, dphi);
}

int etics_ref_phi_nl_b(int basis, int n, int l, double r, double *phi, double *dphi)
{
    if ((basis != 0 && basis != 1) || n < 0 || l < 0 || n > 60 || r < 0.0 || !phi) return -1;
    double p[64], dp[64];
    radial_all_b(basis, n, l, r, p, dphi ? dp : NULL);
    *phi = p[n];
    if (dphi) *dphi = dp[n];
    return 0;
}

int etics_ref_phi_nl(int n, int l, double r, double *phi, double *dphi)
{
    return etics_ref_phi_nl_b(0, n, l, r, phi, dphi);
}

/* J_nl = int rho_nl phi_nl r^2 dr for the density partner rho_nl of phi_nl
 * (laplacian phi_nl Y = 4 pi rho_nl Y), obtained with the Gegenbauer norm
 *   int (1-x^2)^(alpha-1/2) [C_n^alpha]^2 dx
 *       = pi 2^(1-2 alpha) Gamma(n + 2 alpha) / (n! (n + alpha) Gamma(alpha)^2).
 * HO92: rho_nl = K_nl/(2 pi) r^(l-1) (1+r)^-(2l+3) C_n^(2l+3/2)(xi),
 *   K_nl = n (n + 4l + 3)/2 + (l+1)(2l+1),
 *   J_nl = -K_nl 2^-(8l+6) Gamma(n+4l+3) / (n! (n+2l+3/2) Gamma(2l+3/2)^2)
 *   (J_00 = -1/(12 pi)).
 * CB73: rho_nl = K_nl/(4 pi) r^l (1+r^2)^-(l+5/2) C_n^(l+1)(xi),
 *   K_nl = 4n (n + 2l + 2) + (2l+1)(2l+3),
 *   J_nl = -K_nl 2^-(4l+6) Gamma(n+2l+2) / (n! (n+l+1) Gamma(l+1)^2)
 *   (J_00 = -3/64). */
double etics_ref_jnl_b(int basis, int n, int l)
{
    if (basis == 0) {
        double K = 0.5 * n * (n + 4.0 * l + 3.0) + (l + 1.0) * (2.0 * l + 1.0);
        double lg = lgamma(n + 4.0 * l + 3.0) - lgamma(n + 1.0)
                  - 2.0 * lgamma(2.0 * l + 1.5) - (8.0 * l + 6.0) * log(2.0);
        return -K * exp(lg) / (n + 2.0 * l + 1.5);
    }
    double K = 4.0 * n * (n + 2.0 * l + 2.0) + (2.0 * l + 1.0) * (2.0 * l + 3.0);
    double lg = lgamma(n + 2.0 * l + 2.0) - lgamma(n + 1.0)
              - 2.0 * lgamma(l + 1.0) - (4.0 * l + 6.0) * log(2.0);
    return -K * exp(lg) / (n + l + 1.0);
}

double etics_ref_jnl(int n, int l)
{
    return etics_ref_jnl_b(0, n, l);
}

/* Spherical coordinates of a point.  On the z axis phi = 0; at the origin
 * theta = phi = 0. */
typedef struct {
    double r, ct, st, ph;          /* r, cos theta, sin theta, phi       */
    double er[3], et[3], ep[3];    /* unit vectors e_r, e_theta, e_phi   */
} sph_t;

static void to_sph(double x, double y, double z, sph_t *s)
{
    double r2 = (x * x + y * y) + z * z;
    double r = sqrt(r2);
    double rho = sqrt(x * x + y * y);
    s->r = r;
    if (r > 0.0) { s->ct = z / r; s->st = rho / r; }
    else         { s->ct = 1.0;   s->st = 0.0; }
    s->ph = (rho > 0.0) ? atan2(y, x) : 0.0;
    double cp = cos(s->ph), sp = sin(s->ph);
    s->er[0] = s->st * cp; s->er[1] = s->st * sp; s->er[2] = s->ct;
    s->et[0] = s->ct * cp; s->et[1] = s->ct * sp; s->et[2] = -s->st;
    s->ep[0] = -sp;        s->ep[1] = cp;         s->ep[2] = 0.0;
}

/* Associated Legendre functions without the Condon-Shortley phase,
 * P_l^m(t) = s^m d^m/dt^m P_l(t) (s = sin theta, t = cos theta), by the
 * l-upward recursion (the stable direction; the paper's Sec. 4.2 explains why
 * the cot-theta recursion in m is not):
 *   P_m^m = (2m-1)!! s^m,  P_{m+1}^m = (2m+1) t P_m^m,
 *   (l-m) P_l^m = (2l-1) t P_{l-1}^m - (l+m-1) P_{l-2}^m.
 * Q_l^m = P_l^m / s (m >= 1) obeys the same recursion in l (every term shares
 * the factor s^m), started from Q_m^m = (2m-1)!! s^(m-1); it gives the
 * division-free angular derivatives
 *   dP_l^m/dtheta = m t Q_l^m - P_l^(m+1),   (m/s) P_l^m = m Q_l^m.
 * Tables are indexed [l*(L+2) + m] with m up to l+1 (P_l^(l+1) = 0). */
static void legendre_all(int L, double t, double s, double *P, double *Q)
{
    int W = L + 2;
    for (int i = 0; i < (L + 1) * W; ++i) { P[i] = 0.0; Q[i] = 0.0; }
    double pmm = 1.0, qmm = 1.0;   /* P_m^m and (m>=1) Q_m^m */
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            qmm = (m == 1) ? 1.0 : qmm * (2.0 * m - 1.0) * s;
            pmm = pmm * (2.0 * m - 1.0) * s;
        }
        P[m * W + m] = pmm;
        Q[m * W + m] = (m > 0) ? qmm : 0.0;
        if (m + 1 <= L) {
            P[(m + 1) * W + m] = (2.0 * m + 1.0) * t * P[m * W + m];
            Q[(m + 1) * W + m] = (2.0 * m + 1.0) * t * Q[m * W + m];
        }
        for (int l = m + 2; l <= L; ++l) {
            P[l * W + m] = ((2.0 * l - 1.0) * t * P[(l - 1) * W + m]
                            - (l + m - 1.0) * P[(l - 2) * W + m]) / (l - m);
            Q[l * W + m] = ((2.0 * l - 1.0) * t * Q[(l - 1) * W + m]
                            - (l + m - 1.0) * Q[(l - 2) * W + m]) / (l - m);
        }
    }
}

/* Real orthonormal harmonics Y_j, their theta derivative Yt_j and the
 * azimuthal term Yp_j = (1/sin theta) dY_j/dphi, j = l*l + l + m. */
static void ylm_all(int L, const sph_t *s, double *Y, double *Yt, double *Yp)
{
    int W = L + 2;
    double *P = (double *)malloc(sizeof(double) * (L + 1) * W);
    double *Q = (double *)malloc(sizeof(double) * (L + 1) * W);
    legendre_all(L, s->ct, s->st, P, Q);
    for (int l = 0; l <= L; ++l) {
        for (int m = 0; m <= l; ++m) {
            double N = sqrt((2.0 * l + 1.0) / (4.0 * PI)
                            * exp(lgamma(l - m + 1.0) - lgamma(l + m + 1.0)));
            double p  = P[l * W + m];
            double dp = m * s->ct * Q[l * W + m] - ((m + 1 <= l) ? P[l * W + m + 1] : 0.0);
            double mq = m * Q[l * W + m];
            if (m == 0) {
                int j = l * l + l;
                Y[j] = N * p;
                if (Yt) Yt[j] = N * dp;
                if (Yp) Yp[j] = 0.0;
            } else {
                double c = cos(m * s->ph), sn = sin(m * s->ph);
                double A = sqrt(2.0) * N;
                int jc = l * l + l + m, js = l * l + l - m;
                Y[jc] = A * p * c;
                Y[js] = A * p * sn;
                if (Yt) { Yt[jc] = A * dp * c; Yt[js] = A * dp * sn; }
                if (Yp) { Yp[jc] = -A * mq * sn; Yp[js] = A * mq * c; }
            }
        }
    }
    free(P);
    free(Q);
}

int etics_ref_ylm(int l_max, double x, double y, double z, double *Y)
{
    if (l_max < 0 || l_max > 80 || !Y) return -1;
    sph_t s;
    to_sph(x, y, z, &s);
    ylm_all(l_max, &s, Y, NULL, NULL);
    return 0;
}

/* Gradient of r*Y_1m (a constant vector): sqrt(3/4pi) times x-hat for m = 1,
 * y-hat for m = -1, z-hat for m = 0.  Used at the origin, where the l = 1 term
 * is the only one with a non-zero gradient. */
static void grad_rY1(int m, double g[3])
{
    double c = sqrt(3.0 / (4.0 * PI));
    g[0] = (m == 1) ? c : 0.0;
    g[1] = (m == -1) ? c : 0.0;
    g[2] = (m == 0) ? c : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Threading over independent points                                         */
/* ------------------------------------------------------------------------ */

int etics_ref_default_threads(void)
{
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

typedef void (*point_fn)(void *ctx, long begin, long end);
typedef struct { point_fn fn; void *ctx; long begin, end; } chunk_t;

static void *chunk_run(void *arg)
{
    chunk_t *c = (chunk_t *)arg;
    c->fn(c->ctx, c->begin, c->end);
    return NULL;
}

static void parallel_points(point_fn fn, void *ctx, long n, int nthreads)
{
    if (nthreads <= 0) nthreads = etics_ref_default_threads();
    if (nthreads > 256) nthreads = 256;
    if (n < 2 * nthreads) nthreads = 1;
    if (nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    chunk_t ch[256];
    for (int t = 0; t < nthreads; ++t) {
        ch[t].fn = fn; ch[t].ctx = ctx;
        ch[t].begin = n * t / nthreads;
        ch[t].end = n * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, chunk_run, &ch[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------------------ */
/* SCF                                                                       */
/* ------------------------------------------------------------------------ */

/* The sum over particles is split into fixed chunks of consecutive
 * particles, each summed serially in particle order into its own partial
 * array; the partial arrays are then added in chunk order.  The chunk length
 * depends on N alone (4096 particles, or N/1024 rounded up when that is
 * larger), so the result is the same whatever the number of threads that
 * sum the chunks. */
static long coeff_chunk(long n_part)
{
    long c = (n_part + 1023) / 1024;
    return c > 4096 ? c : 4096;
}

typedef struct {
    const double *pos, *mass;
    long n_part, chunk;
    int n_max, l_max, basis;
    double *part;   /* [nchunks][(n_max+1) * nj] */
} coef_ctx_t;

static void coef_chunks(void *vctx, long cbegin, long cend)
{
    coef_ctx_t *c = (coef_ctx_t *)vctx;
    int nj = (c->l_max + 1) * (c->l_max + 1);
    size_t ncoef = (size_t)(c->n_max + 1) * nj;
    double *Y = (double *)malloc(sizeof(double) * nj);
    double phi[64];
    for (long ch = cbegin; ch < cend; ++ch) {
        double *acc = c->part + (size_t)ch * ncoef;
        memset(acc, 0, sizeof(double) * ncoef);
        long k1 = (ch + 1) * c->chunk < c->n_part ? (ch + 1) * c->chunk : c->n_part;
        for (long k = ch * c->chunk; k < k1; ++k) {
            sph_t s;
            to_sph(c->pos[3 * k], c->pos[3 * k + 1], c->pos[3 * k + 2], &s);
            ylm_all(c->l_max, &s, Y, NULL, NULL);
            for (int l = 0; l <= c->l_max; ++l) {
                radial_all_b(c->basis, c->n_max, l, s.r, phi, NULL);
                for (int n = 0; n <= c->n_max; ++n)
                    for (int m = -l; m <= l; ++m) {
                        int j = l * l + l + m;
                        acc[(size_t)n * nj + j] += c->mass[k] * phi[n] * Y[j];
                    }
            }
        }
    }
    free(Y);
}

int etics_ref_scf_coeffs_bt(int basis, const double *pos, const double *mass, long n_part,
                            int n_max, int l_max, double *coeffs, int nthreads)
{
    if ((basis != 0 && basis != 1) || n_part < 0 || n_max < 0 || n_max > 60 || l_max < 0 ||
        l_max > 60 || (n_part > 0 && (!pos || !mass)) || !coeffs)
        return -1;
    int nj = (l_max + 1) * (l_max + 1);
    size_t ncoef = (size_t)(n_max + 1) * nj;
    memset(coeffs, 0, sizeof(double) * ncoef);
    if (n_part > 0) {
        long chunk = coeff_chunk(n_part);
        long nchunks = (n_part + chunk - 1) / chunk;
        double *part = (double *)malloc(sizeof(double) * ncoef * (size_t)nchunks);
        if (!part) return -2;
        coef_ctx_t ctx = {pos, mass, n_part, chunk, n_max, l_max, basis, part};
        parallel_points(coef_chunks, &ctx, nchunks, nthreads);
        for (long ch = 0; ch < nchunks; ++ch)
            for (size_t e = 0; e < ncoef; ++e) coeffs[e] += part[(size_t)ch * ncoef + e];
        free(part);
    }
    for (int n = 0; n <= n_max; ++n)
        for (int l = 0; l <= l_max; ++l) {
            double J = etics_ref_jnl_b(basis, n, l);
            for (int m = -l; m <= l; ++m) coeffs[(size_t)n * nj + l * l + l + m] /= J;
        }
    return 0;
}

int etics_ref_scf_coeffs_b(int basis, const double *pos, const double *mass, long n_part,
                           int n_max, int l_max, double *coeffs)
{
    return etics_ref_scf_coeffs_bt(basis, pos, mass, n_part, n_max, l_max, coeffs, 0);
}

int etics_ref_scf_coeffs(const double *pos, const double *mass, long n_part,
                         int n_max, int l_max, double *coeffs)
{
    return etics_ref_scf_coeffs_b(0, pos, mass, n_part, n_max, l_max, coeffs);
}

typedef struct {
    const double *pos, *coeffs;
    int n_max, l_max, basis;
    double *acc, *pot;
} scf_ctx_t;

static void scf_points(void *vctx, long begin, long end)
{
    scf_ctx_t *c = (scf_ctx_t *)vctx;
    int L = c->l_max, nj = (L + 1) * (L + 1);
    double *Y = (double *)malloc(sizeof(double) * nj);
    double *Yt = (double *)malloc(sizeof(double) * nj);
    double *Yp = (double *)malloc(sizeof(double) * nj);
    double phi[64], dphi[64];
    for (long i = begin; i < end; ++i) {
        sph_t s;
        to_sph(c->pos[3 * i], c->pos[3 * i + 1], c->pos[3 * i + 2], &s);
        double P = 0.0, g[3] = {0.0, 0.0, 0.0};
        if (s.r == 0.0) {
            /* Origin: phi_nl(0) = 0 for l >= 1, so only l = 0 enters the
             * potential.  The gradient of phi_nl Y_lm vanishes there for
             * l = 0 (by symmetry) and l >= 2; for l = 1,
             * phi_n1(r) Y_1m = (phi_n1/r) (r Y_1m) with phi_n1/r -> -C_n(-1). */
            radial_all_b(c->basis, c->n_max, 0, 0.0, phi, NULL);
            double Y00 = 1.0 / sqrt(4.0 * PI);
            for (int n = 0; n <= c->n_max; ++n) P += c->coeffs[(size_t)n * nj] * phi[n] * Y00;
            if (L >= 1) {
                /* both bases: phi_n1(r) / r -> -C_n^alpha_1(-1) as r -> 0 */
                double C[64];
                gegenbauer_all(c->n_max, basis_alpha(c->basis, 1), -1.0, C);
                for (int n = 0; n <= c->n_max; ++n)
                    for (int m = -1; m <= 1; ++m) {
                        double gv[3];
                        grad_rY1(m, gv);
                        double cf = c->coeffs[(size_t)n * nj + 2 + m] * (-C[n]);
                        for (int d = 0; d < 3; ++d) g[d] += cf * gv[d];
                    }
            }
        } else {
            ylm_all(L, &s, Y, Yt, Yp);
            double dr = 0.0, dt = 0.0, dp = 0.0;
            for (int l = 0; l <= L; ++l) {
                radial_all_b(c->basis, c->n_max, l, s.r, phi, dphi);
                for (int n = 0; n <= c->n_max; ++n)
                    for (int m = -l; m <= l; ++m) {
                        int j = l * l + l + m;
                        double cf = c->coeffs[(size_t)n * nj + j];
                        P  += cf * phi[n] * Y[j];
                        dr += cf * dphi[n] * Y[j];
                        dt += cf * phi[n] * Yt[j];
                        dp += cf * phi[n] * Yp[j];
                    }
            }
            for (int d = 0; d < 3; ++d)
                g[d] = dr * s.er[d] + (dt / s.r) * s.et[d] + (dp / s.r) * s.ep[d];
        }
        if (c->pot) c->pot[i] = P;
        if (c->acc) for (int d = 0; d < 3; ++d) c->acc[3 * i + d] = -g[d];
    }
    free(Y); free(Yt); free(Yp);
}

int etics_ref_scf_field_b(int basis, const double *pos, long n_part, int n_max, int l_max,
                          const double *coeffs, double *acc, double *pot, int nthreads)
{
    if ((basis != 0 && basis != 1) || n_part < 0 || n_max < 0 || n_max > 60 || l_max < 0 ||
        l_max > 60 || (n_part > 0 && !pos) || !coeffs)
        return -1;
    scf_ctx_t ctx = {pos, coeffs, n_max, l_max, basis, acc, pot};
    parallel_points(scf_points, &ctx, n_part, nthreads);
    return 0;
}

int etics_ref_scf_field(const double *pos, long n_part, int n_max, int l_max,
                        const double *coeffs, double *acc, double *pot,
                        int nthreads)
{
    return etics_ref_scf_field_b(0, pos, n_part, n_max, l_max, coeffs, acc, pot, nthreads);
}

/* ------------------------------------------------------------------------ */
/* MEX                                                                       */
/* ------------------------------------------------------------------------ */

/* MEX (Sec. 2.4 eqs. 15-17):
 *   Phi(r_i) = - sum_l 4pi/(2l+1) sum_m [q_lm(i) r_i^-(l+1) + p_lm(i) r_i^l] Y_lm(i)
 *   q_lm(i)  = sum_{j before i} m_j r_j^l      Y_lm(j)
 *   p_lm(i)  = sum_{j after i}  m_j r_j^-(l+1) Y_lm(j)
 * The ordering is by radius (Sec. 2.2: the cumulative sums need a sort);
 * exclusive on both sides, so a particle never acts on itself.  The
 * acceleration differentiates Phi at fixed q, p.  q is accumulated forward
 * and p backward (a true suffix sum), each serially in sorted order.
 * A particle at the origin sorts first: its own moment r^-(l+1) Y is taken as
 * zero, and its field uses the p terms of l = 0 (potential) and l = 1
 * (gradient of r Y_1m) only; q terms are skipped at the origin.
 *
 * Work order: the sorted list is taken in blocks, forward for q and then
 * backward for p.  In each block the particles' own moments are evaluated
 * (independent per particle, so over threads), the running sum is carried
 * through the block serially in sorted order (each particle keeps the sum
 * over the particles strictly before it, resp. after it), and the field
 * terms are evaluated from those kept sums (again per particle, over
 * threads).  Every sum is thus formed in exactly the serial order, and the
 * result does not depend on the number of threads. */

typedef struct { double r2; long idx; } key_t_;

static int key_cmp(const void *a, const void *b)
{
    const key_t_ *x = (const key_t_ *)a, *y = (const key_t_ *)b;
    if (x->r2 < y->r2) return -1;
    if (x->r2 > y->r2) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

#define MEX_BLOCK 65536

typedef struct {
    const double *pos, *mass;
    const key_t_ *key;
    int L, outer;      /* outer = 0: inner sums q (forward), 1: outer sums p */
    long k0;           /* first sorted position of the block */
    double *mom;       /* [block][nj]: own moments, then the exclusive sums */
    double *gP, *gG;   /* potential and grad Phi, by particle index */
} mex_ctx_t;

/* own moment of each particle of the block: m r^l Y (inner) or
 * m r^-(l+1) Y (outer; zero at the origin) */
static void mex_moments_pts(void *vctx, long begin, long end)
{
    mex_ctx_t *c = (mex_ctx_t *)vctx;
    int L = c->L, nj = (L + 1) * (L + 1);
    double *Y = (double *)malloc(sizeof(double) * nj);
    for (long b = begin; b < end; ++b) {
        long i = c->key[c->k0 + b].idx;
        double *mo = c->mom + (size_t)b * nj;
        sph_t s;
        to_sph(c->pos[3 * i], c->pos[3 * i + 1], c->pos[3 * i + 2], &s);
        ylm_all(L, &s, Y, NULL, NULL);
        for (int l = 0; l <= L; ++l) {
            double w;
            if (!c->outer) w = (l == 0) ? 1.0 : pow(s.r, (double)l);
            else w = (s.r > 0.0) ? pow(s.r, -(l + 1.0)) : 0.0;
            for (int m = -l; m <= l; ++m) {
                int j = l * l + l + m;
                mo[j] = c->mass[i] * w * Y[j];
            }
        }
    }
    free(Y);
}

/* field terms of each particle of the block from its exclusive sum */
static void mex_field_pts(void *vctx, long begin, long end)
{
    mex_ctx_t *c = (mex_ctx_t *)vctx;
    int L = c->L, nj = (L + 1) * (L + 1);
    double *Y = (double *)malloc(sizeof(double) * nj);
    double *Yt = (double *)malloc(sizeof(double) * nj);
    double *Yp = (double *)malloc(sizeof(double) * nj);
    for (long b = begin; b < end; ++b) {
        long i = c->key[c->k0 + b].idx;
        const double *qp = c->mom + (size_t)b * nj;   /* q (inner) or p (outer) */
        sph_t s;
        to_sph(c->pos[3 * i], c->pos[3 * i + 1], c->pos[3 * i + 2], &s);
        ylm_all(L, &s, Y, Yt, Yp);
        if (s.r > 0.0) {
            double P = 0.0, dr = 0.0, dt = 0.0, dp = 0.0;
            for (int l = 0; l <= L; ++l) {
                double w = 4.0 * PI / (2.0 * l + 1.0);
                double f, df;
                if (!c->outer) {
                    f = pow(s.r, -(l + 1.0));                 /* r^-(l+1) */
                    df = -(l + 1.0) * pow(s.r, -(l + 2.0));
                } else {
                    f = (l == 0) ? 1.0 : pow(s.r, (double)l); /* r^l */
                    df = (l == 0) ? 0.0 : l * pow(s.r, l - 1.0);
                }
                for (int m = -l; m <= l; ++m) {
                    int j = l * l + l + m;
                    P  += -w * qp[j] * f * Y[j];
                    dr += -w * qp[j] * df * Y[j];
                    dt += -w * qp[j] * f * Yt[j];
                    dp += -w * qp[j] * f * Yp[j];
                }
            }
            c->gP[i] += P;
            for (int d = 0; d < 3; ++d)
                c->gG[3 * i + d] += dr * s.er[d] + (dt / s.r) * s.et[d] + (dp / s.r) * s.ep[d];
        } else if (c->outer) {
            /* origin: Phi = -4pi p_00 Y_00; grad from l = 1 only */
            c->gP[i] += -4.0 * PI * qp[0] * (1.0 / sqrt(4.0 * PI));
            if (L >= 1)
                for (int m = -1; m <= 1; ++m) {
                    double gv[3];
                    grad_rY1(m, gv);
                    for (int d = 0; d < 3; ++d)
                        c->gG[3 * i + d] += -(4.0 * PI / 3.0) * qp[2 + m] * gv[d];
                }
        }
    }
    free(Y); free(Yt); free(Yp);
}

int etics_ref_mex_field_t(const double *pos, const double *mass, long n_part,
                          int l_max, double *acc, double *pot, long *order, int nthreads)
{
    if (n_part < 0 || l_max < 0 || l_max > 80 ||
        (n_part > 0 && (!pos || !mass)))
        return -1;
    if (n_part == 0) return 0;
    int L = l_max, nj = (L + 1) * (L + 1);
    key_t_ *key = (key_t_ *)malloc(sizeof(key_t_) * n_part);
    for (long i = 0; i < n_part; ++i) {
        double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        key[i].r2 = (x * x + y * y) + z * z;
        key[i].idx = i;
    }
    qsort(key, n_part, sizeof(key_t_), key_cmp);
    if (order) for (long k = 0; k < n_part; ++k) order[k] = key[k].idx;

    long blk = n_part < MEX_BLOCK ? n_part : MEX_BLOCK;
    double *run = (double *)calloc(nj, sizeof(double));          /* q, then p */
    double *mom = (double *)malloc(sizeof(double) * (size_t)blk * nj);
    double *gP = (double *)calloc(n_part, sizeof(double));       /* potential  */
    double *gG = (double *)calloc(3 * n_part, sizeof(double));   /* grad Phi   */
    mex_ctx_t ctx = {pos, mass, key, L, 0, 0, mom, gP, gG};

    /* forward: inner sums q over the particles before each one */
    for (long k0 = 0; k0 < n_part; k0 += blk) {
        long nb = (n_part - k0 < blk) ? n_part - k0 : blk;
        ctx.outer = 0;
        ctx.k0 = k0;
        parallel_points(mex_moments_pts, &ctx, nb, nthreads);
        for (long b = 0; b < nb; ++b)
            for (int j = 0; j < nj; ++j) {
                double own = mom[(size_t)b * nj + j];
                mom[(size_t)b * nj + j] = run[j];
                run[j] += own;
            }
        parallel_points(mex_field_pts, &ctx, nb, nthreads);
    }
    /* backward: outer sums p over the particles after each one (a true
     * suffix sum, from the outside in) */
    for (int j = 0; j < nj; ++j) run[j] = 0.0;
    for (long k1 = n_part; k1 > 0; k1 -= blk) {
        long k0 = (k1 - blk > 0) ? k1 - blk : 0;
        long nb = k1 - k0;
        ctx.outer = 1;
        ctx.k0 = k0;
        parallel_points(mex_moments_pts, &ctx, nb, nthreads);
        for (long b = nb - 1; b >= 0; --b) {
            int origin = key[k0 + b].r2 == 0.0;
            for (int j = 0; j < nj; ++j) {
                double own = mom[(size_t)b * nj + j];
                mom[(size_t)b * nj + j] = run[j];
                if (!origin) run[j] += own;
            }
        }
        parallel_points(mex_field_pts, &ctx, nb, nthreads);
    }
    for (long i = 0; i < n_part; ++i) {
        if (pot) pot[i] = gP[i];
        if (acc) for (int d = 0; d < 3; ++d) acc[3 * i + d] = -gG[3 * i + d];
    }
    free(key); free(run); free(mom); free(gP); free(gG);
    return 0;
}

int etics_ref_mex_field(const double *pos, const double *mass, long n_part,
                        int l_max, double *acc, double *pot, long *order)
{
    return etics_ref_mex_field_t(pos, mass, n_part, l_max, acc, pot, order, 0);
}

/* ------------------------------------------------------------------------ */
/* Direct summation (test use only)                                          */
/* ------------------------------------------------------------------------ */

/* Pairwise (cascade) summation of v[0..n). */
static double pairwise_sum(const double *v, long n)
{
    if (n <= 8) {
        double s = 0.0;
        for (long i = 0; i < n; ++i) s += v[i];
        return s;
    }
    long h = n / 2;
    return pairwise_sum(v, h) + pairwise_sum(v + h, n - h);
}

typedef struct {
    const double *pos, *mass;
    long n;
    double *acc, *pot;
} direct_ctx_t;

static void direct_points(void *vctx, long begin, long end)
{
    direct_ctx_t *c = (direct_ctx_t *)vctx;
    long n = c->n;
    double *t = (double *)malloc(sizeof(double) * 4 * (n > 0 ? n : 1));
    for (long i = begin; i < end; ++i) {
        long k = 0;
        for (long j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = c->pos[3 * i] - c->pos[3 * j];
            double dy = c->pos[3 * i + 1] - c->pos[3 * j + 1];
            double dz = c->pos[3 * i + 2] - c->pos[3 * j + 2];
            double d = sqrt((dx * dx + dy * dy) + dz * dz);
            double md3 = c->mass[j] / (d * d * d);
            t[k] = -c->mass[j] / d;
            t[n + k] = -md3 * dx;
            t[2 * n + k] = -md3 * dy;
            t[3 * n + k] = -md3 * dz;
            ++k;
        }
        if (c->pot) c->pot[i] = pairwise_sum(t, k);
        if (c->acc)
            for (int d = 0; d < 3; ++d) c->acc[3 * i + d] = pairwise_sum(t + (d + 1) * n, k);
    }
    free(t);
}

int etics_ref_direct(const double *pos, const double *mass, long n_part,
                     double *acc, double *pot, int nthreads)
{
    if (n_part < 0 || (n_part > 0 && (!pos || !mass))) return -1;
    direct_ctx_t ctx = {pos, mass, n_part, acc, pot};
    parallel_points(direct_points, &ctx, n_part, nthreads);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Leapfrog (kick-drift-kick)                                                */
/* ------------------------------------------------------------------------ */

int etics_ref_leapfrog_step(double *pos, double *vel, const double *mass,
                            double *acc, double *pot, long n_part, double dt,
                            int method, int n_max, int l_max, double *coeffs,
                            int nthreads)
{
    if (n_part < 0 || !pos || !vel || !mass || !acc || (method != 0 && method != 1))
        return -1;
    for (long i = 0; i < 3 * n_part; ++i) vel[i] += 0.5 * dt * acc[i];
    for (long i = 0; i < 3 * n_part; ++i) pos[i] += dt * vel[i];
    int rc;
    if (method == 0) {
        int nj = (l_max + 1) * (l_max + 1);
        double *c = coeffs ? coeffs
                           : (double *)malloc(sizeof(double) * (size_t)(n_max + 1) * nj);
        rc = etics_ref_scf_coeffs(pos, mass, n_part, n_max, l_max, c);
        if (rc == 0) rc = etics_ref_scf_field(pos, n_part, n_max, l_max, c, acc, pot, nthreads);
        if (!coeffs) free(c);
    } else {
        rc = etics_ref_mex_field(pos, mass, n_part, l_max, acc, pot, NULL);
    }
    if (rc) return rc;
    for (long i = 0; i < 3 * n_part; ++i) vel[i] += 0.5 * dt * acc[i];
    return 0;
}
