/*
 * fdtd_oracle.c -- plain, slow, FP64 CPU reference of the Bessel-antenna FDTD.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (normalised units: c = eps0 = mu0 = 1, eta = 1, lengths in
 * units of the source wavelength lambda, time in optical periods, omega = 2*pi):
 *
 *  - Analytic source fields: Hertz potentials Pi_x / Pi_y of Eq. 5 (read with
 *    the e^{+i beta z} e^{-i omega t} convention that the printed components of
 *    Eq. 6 and Eq. 7 follow), the Q and R vectors of Eq. 6 / Eq. 7, and the
 *    TE (Eq. 9a) / TM (Eq. 9b) normalisation.  The magnetic field carries the
 *    -i factor that Faraday's law gives for the e^{-i omega t} convention
 *    (H = curl E / (i omega mu0)); Eq. 12b prints H0 R without it.
 *  - The standard second-order Yee leapfrog (Section 4), z periodic, PEC outer
 *    x/y walls, convolutional PML on the x/y faces (Roden-Gedney CPML cited in
 *    Section 4; grading constants are a documented choice, the paper has none).
 *  - The soft source of Eq. 13: after the curl update, the analytic field of
 *    Eq. 12 is added at every Yee point of the hollow annulus; H at its own
 *    time (n+1/2) dt, E at (n+1) dt.
 *  - The fluence of Section 2 (time integral of |S|, S = E x H), taken at cell
 *    centres with H averaged in time: step n adds |E^n x (H^{n-1/2}+H^{n+1/2})/2| dt.
 *  - The reverse-time adjoint of the same discrete update (the paper is silent
 *    on gradients; this is the exact transpose of the steps above).
 *  - The analytic Bessel pulse of Eq. 11 (the Gaussian spectrum of Eq. 10
 *    integrated against J_m), by quadrature, as the reference of the
 *    Gaussian-pulse runs of Section 5.
 *
 * Loops are written out cell by cell in the order the method states; OpenMP
 * only splits the outer plane loop of each independent sub-step.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ types */

typedef struct {
    int nx, ny, nz, npml;
    double dx, dy, dz, dt;
    double pml_order;        /* m in sigma = sigma_max u^m                  */
    double pml_sigma_scale;  /* sigma_max = scale (m+1) / (eta dx)          */
    double pml_kappa_max;    /* kappa = 1 + (kappa_max - 1) u^m             */
    double pml_alpha_max;    /* alpha = alpha_max (1 - u)                   */
    int zbc;                 /* OR_Z_PERIODIC, or OR_Z_WALLS: PEC walls at z = 0 and
                                z = nz dz with npml_z CPML cells inside each      */
    int npml_z;
} or_grid;

enum { OR_Z_PERIODIC = 0, OR_Z_WALLS = 1 };

enum { OR_POL_Y = 0, OR_POL_X = 1, OR_POL_CIRC_PLUS = 2, OR_POL_CIRC_MINUS = 3, OR_POL_Z = 4 };
enum { OR_TE = 0, OR_TM = 1 };
enum { OR_ENV_CW_SIN2 = 0, OR_ENV_GAUSS = 1 };
enum { OR_INJ_ALL = 0, OR_INJ_TANGENTIAL = 1 };

typedef struct {
    int m;              /* Bessel order                                     */
    double theta;       /* cone angle, radians                              */
    int pol;            /* OR_POL_*: Y = Pi_x potential, X = Pi_y potential, Z = Pi_z potential */
    int mode;           /* OR_TE / OR_TM                                    */
    double E0;
    double r_center;    /* ring centre radius, in cells of dx               */
    double thickness;   /* ring thickness, in cells of dx                   */
    int envelope;       /* OR_ENV_*                                         */
    double ramp;        /* CW: sin^2 ramp length (periods)                  */
    double T, T0;       /* Gaussian: f = exp(-(t-T0)^2/T^2); phase uses t-T0 */
    int inject;         /* OR_INJ_*                                         */
    const double *w_amp;   /* nx*ny per-column amplitude weights or NULL    */
    const double *w_phase; /* nx*ny per-column phase weights or NULL        */
} or_source;

/* One antenna point of one component: its flat cell index, the column
 * (i + nx j) that selects its weight, and the unweighted analytic complex
 * amplitude A (so that the added value is f * Re{ w e^{i phi_w} A e^{-i Phi} }). */
typedef struct {
    long idx;
    long col;
    double are, aim;
} or_point;

typedef struct {
    or_point *pts[6];   /* 0..2: Ex,Ey,Ez ; 3..5: Hx,Hy,Hz */
    long npts[6];
    or_source src;
} or_antenna;

typedef struct {
    double *e[3], *h[3];
    double *psi_e[4];   /* Exy, Ezy, Eyx, Ezx  (full grid; nonzero in shells) */
    double *psi_h[4];   /* Hxy, Hzy, Hyx, Hzx                                 */
    double *fluence;    /* nx*ny*nz or NULL                                   */
    double *psi_ez[2];  /* Exz, Eyz (z shells of OR_Z_WALLS grids)           */
    double *psi_hz[2];  /* Hxz, Hyz                                           */
} or_state;

/* Wall source (the Bessel-Gauss reference of Section 2): a Gaussian beam,
 * polarised along x, with the axicon phase Phi(r) = -k r sin(theta), added
 * to E_x on the plane k = plane after each E update:
 *   E_x += f(t) Re{ E0 exp(-r^2 / w0^2) e^{-i k r sin(theta)} e^{-i omega t'} }
 * at the E_x point (r from the axis at nx dx/2, ny dy/2), t = (n+1) dt,
 * with f and t' as for the antenna (CW ramp or Gaussian).  The row j = 0
 * (on the y = 0 PEC wall) is left out, and on a z-walled grid the plane
 * may not be k = 0 (the z = 0 PEC wall). */
typedef struct {
    double theta, w0, E0;
    int envelope;
    double ramp, T, T0;
    int plane;
} or_wall;

/* ------------------------------------------------------------- helpers */

static inline long IDX(const or_grid *g, long i, long j, long k)
{
    return (k * g->ny + j) * g->nx + i;
}

double or_courant_dt(double dx, double dy, double dz, double courant)
{
    /* Yee stability limit in 3D, scaled by the Courant number (c = 1). */
    return courant / sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz));
}

/* J_n for any integer n, from the C library (J_{-n} = (-1)^n J_n). */
double or_jn(int n, double x)
{
    if (n < 0) {
        double v = jn(-n, x);
        return ((-n) & 1) ? -v : v;
    }
    return jn(n, x);
}

/* ---------------------------------------------------------------- CPML */

/* Profile at a physical coordinate `pos` along an axis of `n` cells of size d,
 * with a layer of npml cells at each end.  Roden-Gedney CFS-PML:
 *   u = depth / (npml d),  sigma = sigma_max u^m,  kappa = 1 + (kmax-1) u^m,
 *   alpha = alpha_max (1-u),  b = exp(-(sigma/kappa + alpha) dt),
 *   a = sigma (b-1) / (kappa (sigma + kappa alpha)).                          */
static void pml_profile_n(const or_grid *g, int n, int npml, double d, double pos,
                          double *b, double *a, double *kappa)
{
    *b = 1.0; *a = 0.0; *kappa = 1.0;
    if (npml <= 0) return;
    double L = n * d, w = npml * d;
    double depth = 0.0;
    if (pos < w) depth = w - pos;
    if (pos > L - w) depth = pos - (L - w);
    if (depth <= 0.0) return;
    double u = depth / w;
    double um = pow(u, g->pml_order);
    double sigma_max = g->pml_sigma_scale * (g->pml_order + 1.0) / d; /* eta = 1 */
    double sigma = sigma_max * um;
    double kap = 1.0 + (g->pml_kappa_max - 1.0) * um;
    double alpha = g->pml_alpha_max * (1.0 - u);
    *kappa = kap;
    *b = exp(-(sigma / kap + alpha) * g->dt);
    if (sigma > 0.0)
        *a = sigma * (*b - 1.0) / (kap * (sigma + kap * alpha));
}

void or_pml_profile(const or_grid *g, int n, double d, double pos,
                    double *b, double *a, double *kappa)
{
    pml_profile_n(g, n, g->npml, d, pos, b, a, kappa);
}

/* ------------------------------------------------ analytic source fields */

/* Complex amplitudes (re,im interleaved, 3 components) of E and H of the
 * order-m vector Bessel beam at (x,y,z) measured from the beam axis.
 * Physical field = Re{ A e^{-i omega t'} }.  Eq. 6 (Pi_x), Eq. 7 (Pi_y), Eq. 8 (Pi_z),
 * Eq. 9. */
typedef struct { double re, im; } cpx;
static inline cpx C(double r, double i) { cpx c = {r, i}; return c; }
static inline cpx cadd(cpx a, cpx b) { return C(a.re + b.re, a.im + b.im); }
static inline cpx csub(cpx a, cpx b) { return C(a.re - b.re, a.im - b.im); }
static inline cpx cmul(cpx a, cpx b) { return C(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static inline cpx cscale(cpx a, double s) { return C(a.re * s, a.im * s); }
static inline cpx cexpi(double p) { return C(cos(p), sin(p)); }
static const cpx CI = {0.0, 1.0};

/* Q and R of Eq. 6 (potential along x, which = 0) or Eq. 7 (along y, which = 1),
 * without the common factor e^{i m phi} e^{i beta z}. */
static void qr_linear(int which, int m, double K, double beta, double k,
                      double r, double phi, cpx Q[3], cpx R[3])
{
    double Kr = K * r;
    double jm = or_jn(m, Kr), jp1 = or_jn(m + 1, Kr), jm1 = or_jn(m - 1, Kr);
    double jp2 = or_jn(m + 2, Kr), jm2 = or_jn(m - 2, Kr);
    cpx e1 = cexpi(phi), e1m = cexpi(-phi), e2 = cexpi(2 * phi), e2m = cexpi(-2 * phi);
    cpx p1 = cscale(e1, jp1), m1 = cscale(e1m, jm1);   /* J_{m+1} e^{i phi}, J_{m-1} e^{-i phi} */
    cpx p2 = cscale(e2, jp2), m2 = cscale(e2m, jm2);   /* J_{m+2} e^{2i phi}, J_{m-2} e^{-2i phi} */
    double K2 = K * K;
    if (which == 0) {
        /* Eq. 6 */
        Q[0] = C(0, 0);
        Q[1] = C(0, beta * jm);                                   /* i beta J_m            */
        Q[2] = cmul(C(0, -K / 2.0), cadd(p1, m1));                /* K/(2i) [..+..]         */
        R[0] = cadd(C((k * k + beta * beta) / 2.0 * jm, 0), cscale(cadd(p2, m2), K2 / 4.0));
        R[1] = cmul(C(0, K2 / 4.0), csub(m2, p2));                /* i K^2/4 [J_{m-2}.. - J_{m+2}..] */
        R[2] = cmul(C(0, beta * K / 2.0), csub(m1, p1));          /* i beta K/2 [J_{m-1}.. - J_{m+1}..] */
    } else {
        /* Eq. 7 */
        Q[0] = C(0, -beta * jm);                                  /* -i beta J_m           */
        Q[1] = C(0, 0);
        Q[2] = cscale(csub(p1, m1), -K / 2.0);                    /* -K/2 [J_{m+1}.. - J_{m-1}..] */
        R[0] = cmul(C(0, K2 / 4.0), csub(m2, p2));
        R[1] = csub(C((k * k + beta * beta) / 2.0 * jm, 0), cscale(cadd(p2, m2), K2 / 4.0));
        R[2] = cscale(cadd(p1, m1), -beta * K / 2.0);
    }
}

/* Q and R of Eq. 8 (potential along z), without the common factor
 * e^{i m phi} e^{i beta z}: azimuthal (TE) or radial (TM) fields for m = 0. */
static void qr_axial(int m, double K, double beta, double r, double phi, cpx Q[3], cpx R[3])
{
    double Kr = K * r;
    double jm = or_jn(m, Kr), jp1 = or_jn(m + 1, Kr), jm1 = or_jn(m - 1, Kr);
    cpx p1 = cscale(cexpi(phi), jp1), m1 = cscale(cexpi(-phi), jm1);   /* J_{m+1} e^{i phi}, J_{m-1} e^{-i phi} */
    Q[0] = cmul(C(0, K / 2.0), cadd(p1, m1));                            /* i K/2 [..+..]          */
    Q[1] = cscale(csub(p1, m1), K / 2.0);                                /* K/2 [..-..]            */
    Q[2] = C(0, 0);
    R[0] = cmul(C(0, -beta * K / 2.0), csub(p1, m1));                    /* -i beta K/2 [..-..]    */
    R[1] = cscale(cadd(p1, m1), -beta * K / 2.0);                        /* -beta K/2 [..+..]      */
    R[2] = C(K * K * jm, 0);                                             /* K^2 J_m                */
}

void or_source_field(const or_source *s, double x, double y, double z,
                     double E[6], double H[6])
{
    double k = 2.0 * OR_PI;            /* k0 = omega / c with lambda = 1 */
    double K = k * sin(s->theta), beta = k * cos(s->theta);
    double r = sqrt(x * x + y * y);
    double phi = (r > 0.0) ? atan2(y, x) : 0.0;
    cpx Q[3], R[3];
    cpx Qa[3], Ra[3], Qb[3], Rb[3];
    if (s->pol == OR_POL_Y || s->pol == OR_POL_X) {
        qr_linear(s->pol == OR_POL_Y ? 0 : 1, s->m, K, beta, k, r, phi, Q, R);
    } else if (s->pol == OR_POL_Z) {
        qr_axial(s->m, K, beta, r, phi, Q, R);
    } else {
        /* (Pi_x +- i Pi_y) / sqrt 2 */
        double sg = (s->pol == OR_POL_CIRC_PLUS) ? 1.0 : -1.0;
        qr_linear(0, s->m, K, beta, k, r, phi, Qa, Ra);
        qr_linear(1, s->m, K, beta, k, r, phi, Qb, Rb);
        for (int c = 0; c < 3; ++c) {
            Q[c] = cscale(cadd(Qa[c], cmul(C(0, sg), Qb[c])), 1.0 / sqrt(2.0));
            R[c] = cscale(cadd(Ra[c], cmul(C(0, sg), Rb[c])), 1.0 / sqrt(2.0));
        }
    }
    cpx F = cmul(cexpi(s->m * phi), cexpi(beta * z));
    cpx e[3], h[3];
    for (int c = 0; c < 3; ++c) {
        if (s->mode == OR_TE) {
            /* Eq. 9a: E = k0^-2 E0 k0 Q ; H = -i k0^-2 H0 R, H0 = E0 / eta */
            e[c] = cscale(Q[c], s->E0 / k);
            h[c] = cmul(C(0, -1), cscale(R[c], s->E0 / (k * k)));
        } else {
            /* Eq. 9b: E = k0^-2 E0 R ; H = -i k0^-2 H0 k0 Q */
            e[c] = cscale(R[c], s->E0 / (k * k));
            h[c] = cmul(C(0, -1), cscale(Q[c], s->E0 / k));
        }
        e[c] = cmul(e[c], F);
        h[c] = cmul(h[c], F);
    }
    if (s->inject == OR_INJ_TANGENTIAL && r > 0.0) {
        /* remove the radial (x,y)-projection of the vector at this point */
        double cr = x / r, sr = y / r;
        cpx er = cadd(cscale(e[0], cr), cscale(e[1], sr));
        cpx hr = cadd(cscale(h[0], cr), cscale(h[1], sr));
        e[0] = csub(e[0], cscale(er, cr)); e[1] = csub(e[1], cscale(er, sr));
        h[0] = csub(h[0], cscale(hr, cr)); h[1] = csub(h[1], cscale(hr, sr));
    }
    for (int c = 0; c < 3; ++c) {
        E[2 * c] = e[c].re; E[2 * c + 1] = e[c].im;
        H[2 * c] = h[c].re; H[2 * c + 1] = h[c].im;
    }
}

/* Time factors of the soft source at time t: e^{-i Phi} with Phi = omega t',
 * t' = t (CW) or t - T0 (Gaussian), reduced modulo one period; envelope f(t). */
void or_source_time(const or_source *s, double t, double *cphi, double *sphi, double *f)
{
    double tp = (s->envelope == OR_ENV_GAUSS) ? t - s->T0 : t;
    double periods = tp;               /* period = lambda / c = 1 */
    double phase = 2.0 * OR_PI * (periods - floor(periods));
    *cphi = cos(phase);
    *sphi = sin(phase);
    if (s->envelope == OR_ENV_GAUSS) {
        double u = (t - s->T0) / s->T;
        *f = exp(-u * u);
    } else {
        if (t < s->ramp) {
            double sn = sin(OR_PI * t / (2.0 * s->ramp));
            *f = sn * sn;
        } else {
            *f = 1.0;
        }
    }
}

/* Staggered position offsets (in cells) of each component: Ex,Ey,Ez,Hx,Hy,Hz. */
static const double OFF[6][3] = {
    {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
    {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0},
};

/* Enumerate antenna points: every Yee point of each component whose distance
 * r (in cells) from the axis at (nx/2, ny/2) satisfies r_in <= r < r_out,
 * along the full z length (Fig. 3; Section 4).  Returns 0 on success. */
int or_antenna_build(const or_grid *g, const or_source *s, or_antenna *ant)
{
    memset(ant, 0, sizeof(*ant));
    ant->src = *s;
    double rin = s->r_center - 0.5 * s->thickness;
    double rout = s->r_center + 0.5 * s->thickness;
    double xc = 0.5 * g->nx, yc = 0.5 * g->ny;
    for (int c = 0; c < 6; ++c) {
        long cap = 0, n = 0;
        /* count */
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                double u = i + OFF[c][0] - xc, v = j + OFF[c][1] - yc;
                double r2 = u * u + v * v;
                if (r2 >= rin * rin && r2 < rout * rout) cap++;
            }
        cap *= g->nz;
        ant->pts[c] = (or_point *)malloc(sizeof(or_point) * (cap > 0 ? cap : 1));
        if (!ant->pts[c]) return -1;
        for (int k = 0; k < g->nz; ++k)
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    double u = i + OFF[c][0] - xc, v = j + OFF[c][1] - yc;
                    double r2 = u * u + v * v;
                    if (!(r2 >= rin * rin && r2 < rout * rout)) continue;
                    /* skip PEC-clamped tangential E on the walls */
                    if ((c == 1 || c == 2) && i == 0) continue;
                    if ((c == 0 || c == 2) && j == 0) continue;
                    double x = u * g->dx, y = v * g->dy, z = (k + OFF[c][2]) * g->dz;
                    double E[6], H[6];
                    or_source_field(s, x, y, z, E, H);
                    or_point *p = &ant->pts[c][n++];
                    p->idx = IDX(g, i, j, k);
                    p->col = (long)j * g->nx + i;
                    if (c < 3) { p->are = E[2 * c]; p->aim = E[2 * c + 1]; }
                    else       { p->are = H[2 * (c - 3)]; p->aim = H[2 * (c - 3) + 1]; }
                }
        ant->npts[c] = n;
    }
    return 0;
}

void or_antenna_free(or_antenna *ant)
{
    for (int c = 0; c < 6; ++c) { free(ant->pts[c]); ant->pts[c] = NULL; }
}

long or_antenna_count(const or_antenna *ant, int c) { return ant->npts[c]; }

/* Value added at one antenna point: f Re{ w e^{i phi_w} A e^{-i Phi} }. */
static inline double src_value(const or_source *s, const or_point *p,
                               double cphi, double sphi, double f)
{
    double wa = s->w_amp ? s->w_amp[p->col] : 1.0;
    double wp = s->w_phase ? s->w_phase[p->col] : 0.0;
    /* B = w e^{i phi_w} A */
    double bre = wa * (cos(wp) * p->are - sin(wp) * p->aim);
    double bim = wa * (cos(wp) * p->aim + sin(wp) * p->are);
    /* Re{ B (cphi - i sphi) } */
    return f * (bre * cphi + bim * sphi);
}

static void add_source(const or_antenna *ant, or_state *st, int first, double t)
{
    double cphi, sphi, f;
    or_source_time(&ant->src, t, &cphi, &sphi, &f);
    for (int c = first; c < first + 3; ++c) {
        double *fld = (c < 3) ? st->e[c] : st->h[c - 3];
        for (long p = 0; p < ant->npts[c]; ++p)
            fld[ant->pts[c][p].idx] += src_value(&ant->src, &ant->pts[c][p], cphi, sphi, f);
    }
}

/* ------------------------------------------- Bessel pulse (Eq. 10-11) */

/* E_y of the order-m Bessel pulse of Eq. 11 at n points (r, phi, z, t):
 *   E_y = -cos(theta) e^{i m phi} Int dw F(w) J_m(w sin(theta) r) e^{-i w tau},
 *   tau = t - T0 - z cos(theta),   F(w) = T / (2 sqrt(pi)) exp(-T^2 (w - w0)^2 / 4)
 * (Eq. 10, c = 1).  Eq. 11 prints the time factor as e^{+i w tau}; this
 * library's fields follow e^{-i w t} (the convention of Eq. 6-7's printed
 * components), so the conjugate time factor is used: the real part is the
 * same for m = 0 and the pattern of m > 0 turns the same way as the antenna's.
 * The integral is a trapezoid sum over w0 +- 12/T, where F has fallen to
 * e^{-36} of its peak, with nq >= 2 nodes.  out holds re, im per point. */
void or_bessel_pulse(int m, double theta, double T, double T0, double w0, long n, const double *r,
                     const double *phi, const double *z, const double *t, int nq, double *out)
{
    const double W = 12.0 / T, h = 2.0 * W / (nq - 1);
    const double norm = T / (2.0 * sqrt(OR_PI));
    const double st = sin(theta), ct = cos(theta);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        const double tau = t[p] - T0 - z[p] * ct;
        double sr = 0.0, si = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double w = w0 - W + q * h;
            const double wt = (q == 0 || q == nq - 1) ? 0.5 : 1.0;
            const double F = norm * exp(-0.25 * T * T * (w - w0) * (w - w0));
            const double a = wt * F * jn(m, w * st * r[p]);
            const double ph = m * phi[p] - w * tau;
            sr += a * cos(ph);
            si += a * sin(ph);
        }
        out[2 * p] = -ct * h * sr;
        out[2 * p + 1] = -ct * h * si;
    }
}

/* ------------------------------------------------------------ Yee step */

/* Field value with the PEC / periodic boundary reading: indices past the
 * +x / +y walls (i == nx, j == ny) are the wall itself, where tangential E
 * and normal H are zero; z wraps, or (OR_Z_WALLS) reads zero past the z
 * walls in the same way. */
static inline double at(const or_grid *g, const double *f, long i, long j, long k)
{
    if (i >= g->nx || j >= g->ny || i < 0 || j < 0) return 0.0;
    if (g->zbc == OR_Z_WALLS) {
        if (k < 0 || k >= g->nz) return 0.0;
    } else {
        k = ((k % g->nz) + g->nz) % g->nz;
    }
    return f[IDX(g, i, j, k)];
}

/* CPML profiles at every position of one axis (half = 1: the (i+1/2)
 * positions of H's transverse derivatives; half = 0: integer positions). */
typedef struct { double *b, *a, *kappa; } or_prof;

/* axis 0, 1, 2 = x, y, z; the z axis has a CPML only on OR_Z_WALLS grids */
static void prof_build(const or_grid *g, int axis, int half, or_prof *p)
{
    int n = axis == 0 ? g->nx : (axis == 1 ? g->ny : g->nz);
    double d = axis == 0 ? g->dx : (axis == 1 ? g->dy : g->dz);
    int npml = axis < 2 ? g->npml : (g->zbc == OR_Z_WALLS ? g->npml_z : 0);
    p->b = (double *)malloc(sizeof(double) * n);
    p->a = (double *)malloc(sizeof(double) * n);
    p->kappa = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i)
        pml_profile_n(g, n, npml, d, (i + 0.5 * half) * d, &p->b[i], &p->a[i], &p->kappa[i]);
}

static void prof_free(or_prof *p) { free(p->b); free(p->a); free(p->kappa); }

static void update_h(const or_grid *g, or_state *s)
{
    double *Ex = s->e[0], *Ey = s->e[1], *Ez = s->e[2];
    double *Hx = s->h[0], *Hy = s->h[1], *Hz = s->h[2];
    double dt = g->dt;
    or_prof px, py, pz;
    prof_build(g, 0, 1, &px);
    prof_build(g, 1, 1, &py);
    prof_build(g, 2, 1, &pz);
    const int zw = g->zbc == OR_Z_WALLS;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j) {
            double byh = py.b[j], ayh = py.a[j], kyh = py.kappa[j];
            double bzh = pz.b[k], azh = pz.a[k], kzh = pz.kappa[k];
            for (long i = 0; i < g->nx; ++i) {
                double bxh = px.b[i], axh = px.a[i], kxh = px.kappa[i];
                long id = IDX(g, i, j, k);
                /* Hx at (i, j+1/2, k+1/2): dEz/dy - dEy/dz */
                double dEz_dy = (at(g, Ez, i, j + 1, k) - at(g, Ez, i, j, k)) / g->dy;
                double dEy_dz = (at(g, Ey, i, j, k + 1) - at(g, Ey, i, j, k)) / g->dz;
                s->psi_h[0][id] = byh * s->psi_h[0][id] + ayh * dEz_dy;
                double zx = dEy_dz;
                if (zw) {
                    s->psi_hz[0][id] = bzh * s->psi_hz[0][id] + azh * dEy_dz;
                    zx = dEy_dz / kzh + s->psi_hz[0][id];
                }
                Hx[id] -= dt * (dEz_dy / kyh + s->psi_h[0][id] - zx);
                /* Hy at (i+1/2, j, k+1/2): dEx/dz - dEz/dx */
                double dEx_dz = (at(g, Ex, i, j, k + 1) - at(g, Ex, i, j, k)) / g->dz;
                double dEz_dx = (at(g, Ez, i + 1, j, k) - at(g, Ez, i, j, k)) / g->dx;
                s->psi_h[2][id] = bxh * s->psi_h[2][id] + axh * dEz_dx;
                double zy = dEx_dz;
                if (zw) {
                    s->psi_hz[1][id] = bzh * s->psi_hz[1][id] + azh * dEx_dz;
                    zy = dEx_dz / kzh + s->psi_hz[1][id];
                }
                Hy[id] -= dt * (zy - (dEz_dx / kxh + s->psi_h[2][id]));
                /* Hz at (i+1/2, j+1/2, k): dEy/dx - dEx/dy */
                double dEy_dx = (at(g, Ey, i + 1, j, k) - at(g, Ey, i, j, k)) / g->dx;
                double dEx_dy = (at(g, Ex, i, j + 1, k) - at(g, Ex, i, j, k)) / g->dy;
                s->psi_h[3][id] = bxh * s->psi_h[3][id] + axh * dEy_dx;
                s->psi_h[1][id] = byh * s->psi_h[1][id] + ayh * dEx_dy;
                Hz[id] -= dt * ((dEy_dx / kxh + s->psi_h[3][id]) - (dEx_dy / kyh + s->psi_h[1][id]));
            }
        }
    prof_free(&px);
    prof_free(&py);
    prof_free(&pz);
}

static void update_e(const or_grid *g, or_state *s)
{
    double *Ex = s->e[0], *Ey = s->e[1], *Ez = s->e[2];
    double *Hx = s->h[0], *Hy = s->h[1], *Hz = s->h[2];
    double dt = g->dt;
    or_prof px, py, pz;
    prof_build(g, 0, 0, &px);
    prof_build(g, 1, 0, &py);
    prof_build(g, 2, 0, &pz);
    const int zw = g->zbc == OR_Z_WALLS;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j) {
            double bye = py.b[j], aye = py.a[j], kye = py.kappa[j];
            double bze = pz.b[k], aze = pz.a[k], kze = pz.kappa[k];
            for (long i = 0; i < g->nx; ++i) {
                double bxe = px.b[i], axe = px.a[i], kxe = px.kappa[i];
                long id = IDX(g, i, j, k);
                /* Ex at (i+1/2, j, k): dHz/dy - dHy/dz ; tangential to the y = 0 wall at j = 0
                 * (and to the z = 0 wall at k = 0 on OR_Z_WALLS grids) */
                if (j > 0 && !(zw && k == 0)) {
                    double dHz_dy = (at(g, Hz, i, j, k) - at(g, Hz, i, j - 1, k)) / g->dy;
                    double dHy_dz = (at(g, Hy, i, j, k) - at(g, Hy, i, j, k - 1)) / g->dz;
                    s->psi_e[0][id] = bye * s->psi_e[0][id] + aye * dHz_dy;
                    double zx = dHy_dz;
                    if (zw) {
                        s->psi_ez[0][id] = bze * s->psi_ez[0][id] + aze * dHy_dz;
                        zx = dHy_dz / kze + s->psi_ez[0][id];
                    }
                    Ex[id] += dt * ((dHz_dy / kye + s->psi_e[0][id]) - zx);
                } else {
                    Ex[id] = 0.0;   /* PEC: tangential E on the y = 0 (z = 0) wall */
                }
                /* Ey at (i, j+1/2, k): dHx/dz - dHz/dx ; tangential to x = 0 at i = 0 (and z = 0) */
                if (i > 0 && !(zw && k == 0)) {
                    double dHx_dz = (at(g, Hx, i, j, k) - at(g, Hx, i, j, k - 1)) / g->dz;
                    double dHz_dx = (at(g, Hz, i, j, k) - at(g, Hz, i - 1, j, k)) / g->dx;
                    s->psi_e[2][id] = bxe * s->psi_e[2][id] + axe * dHz_dx;
                    double zy = dHx_dz;
                    if (zw) {
                        s->psi_ez[1][id] = bze * s->psi_ez[1][id] + aze * dHx_dz;
                        zy = dHx_dz / kze + s->psi_ez[1][id];
                    }
                    Ey[id] += dt * (zy - (dHz_dx / kxe + s->psi_e[2][id]));
                } else {
                    Ey[id] = 0.0;   /* PEC: tangential E on the x = 0 (z = 0) wall */
                }
                /* Ez at (i, j, k+1/2): dHy/dx - dHx/dy ; tangential to both walls */
                if (i > 0 && j > 0) {
                    double dHy_dx = (at(g, Hy, i, j, k) - at(g, Hy, i - 1, j, k)) / g->dx;
                    double dHx_dy = (at(g, Hx, i, j, k) - at(g, Hx, i, j - 1, k)) / g->dy;
                    s->psi_e[3][id] = bxe * s->psi_e[3][id] + axe * dHy_dx;
                    s->psi_e[1][id] = bye * s->psi_e[1][id] + aye * dHx_dy;
                    Ez[id] += dt * ((dHy_dx / kxe + s->psi_e[3][id]) - (dHx_dy / kye + s->psi_e[1][id]));
                } else {
                    Ez[id] = 0.0;   /* PEC: tangential on both walls */
                }
            }
        }
    prof_free(&px);
    prof_free(&py);
    prof_free(&pz);
}

/* |E_c x Hbar_c| at the centre of cell (i,j,k): E averaged over the four
 * edges of each component around the centre, H over the two faces. */
static double poynting_mag(const or_grid *g, const or_state *s, double *const hold[3],
                           long i, long j, long k)
{
    const double *Ex = s->e[0], *Ey = s->e[1], *Ez = s->e[2];
    double ex = 0.25 * (at(g, Ex, i, j, k) + at(g, Ex, i, j + 1, k) + at(g, Ex, i, j, k + 1) + at(g, Ex, i, j + 1, k + 1));
    double ey = 0.25 * (at(g, Ey, i, j, k) + at(g, Ey, i + 1, j, k) + at(g, Ey, i, j, k + 1) + at(g, Ey, i + 1, j, k + 1));
    double ez = 0.25 * (at(g, Ez, i, j, k) + at(g, Ez, i + 1, j, k) + at(g, Ez, i, j + 1, k) + at(g, Ez, i + 1, j + 1, k));
    double hb[3];
    hb[0] = 0.25 * (at(g, s->h[0], i, j, k) + at(g, hold[0], i, j, k) + at(g, s->h[0], i + 1, j, k) + at(g, hold[0], i + 1, j, k));
    hb[1] = 0.25 * (at(g, s->h[1], i, j, k) + at(g, hold[1], i, j, k) + at(g, s->h[1], i, j + 1, k) + at(g, hold[1], i, j + 1, k));
    hb[2] = 0.25 * (at(g, s->h[2], i, j, k) + at(g, hold[2], i, j, k) + at(g, s->h[2], i, j, k + 1) + at(g, hold[2], i, j, k + 1));
    double sx = ey * hb[2] - ez * hb[1];
    double sy = ez * hb[0] - ex * hb[2];
    double sz = ex * hb[1] - ey * hb[0];
    return sqrt(sx * sx + sy * sy + sz * sz);
}

/* The wall source at time t (E time (n+1) dt): E_x on the plane w->plane. */
static void add_wall(const or_grid *g, const or_wall *w, or_state *st, double t)
{
    or_source tsrc;
    memset(&tsrc, 0, sizeof(tsrc));
    tsrc.envelope = w->envelope;
    tsrc.ramp = w->ramp;
    tsrc.T = w->T;
    tsrc.T0 = w->T0;
    double cphi, sphi, f;
    or_source_time(&tsrc, t, &cphi, &sphi, &f);
    const double k = 2.0 * OR_PI, ks = k * sin(w->theta);
    const double xc = 0.5 * g->nx * g->dx, yc = 0.5 * g->ny * g->dy;
    for (long j = 1; j < g->ny; ++j)   /* j = 0: E_x is tangential to the y = 0 PEC wall */
        for (long i = 0; i < g->nx; ++i) {
            const double x = (i + 0.5) * g->dx - xc, y = j * g->dy - yc;   /* E_x point */
            const double r = sqrt(x * x + y * y);
            const double a = w->E0 * exp(-(r * r) / (w->w0 * w->w0));
            /* Re{ a e^{-i k r sin(theta)} e^{-i Phi} } = a cos(k r sin(theta) + Phi) */
            const double ph = ks * r;
            st->e[0][IDX(g, i, j, w->plane)] += f * a * (cos(ph) * cphi - sin(ph) * sphi);
        }
}

/* Advance `nsteps` full Yee steps starting at step index n0 (E at n0 dt,
 * H at (n0 - 1/2) dt).  Order in each step: H curl update (with CPML psi),
 * H soft source at (n+1/2) dt, fluence term n, E curl update (with CPML psi),
 * E soft source at (n+1) dt, wall source at (n+1) dt.  Returns 0 on success. */
static int or_step_all(const or_grid *g, const or_antenna *ant, const or_wall *wall, or_state *s, long n0,
                       int nsteps)
{
    long ncell = (long)g->nx * g->ny * g->nz;
    double *hold[3] = {NULL, NULL, NULL};
    if (s->fluence) {
        for (int c = 0; c < 3; ++c) {
            hold[c] = (double *)malloc(sizeof(double) * ncell);
            if (!hold[c]) { for (int q = 0; q < c; ++q) free(hold[q]); return -1; }
        }
    }
    for (long n = n0; n < n0 + nsteps; ++n) {
        if (s->fluence)
            for (int c = 0; c < 3; ++c) memcpy(hold[c], s->h[c], sizeof(double) * ncell);
        update_h(g, s);
        if (ant) add_source(ant, s, 3, (n + 0.5) * g->dt);
        if (s->fluence) {
#pragma omp parallel for schedule(static)
            for (long k = 0; k < g->nz; ++k)
                for (long j = 0; j < g->ny; ++j)
                    for (long i = 0; i < g->nx; ++i)
                        s->fluence[IDX(g, i, j, k)] += poynting_mag(g, s, hold, i, j, k) * g->dt;
        }
        update_e(g, s);
        if (ant) add_source(ant, s, 0, (n + 1.0) * g->dt);
        if (wall) add_wall(g, wall, s, (n + 1.0) * g->dt);
    }
    for (int c = 0; c < 3; ++c) free(hold[c]);
    return 0;
}

int or_step(const or_grid *g, const or_antenna *ant, or_state *s, long n0, int nsteps)
{
    return or_step_all(g, ant, NULL, s, n0, nsteps);
}

/* Convenience for callers that only hold flat arrays: build the antenna,
 * run, free.  src may be NULL (source-free run). */
int or_run_wall(const or_grid *g, const or_source *src, const or_wall *wall, or_state *s, long n0, int nsteps)
{
    or_antenna ant;
    int rc;
    if (wall && (wall->plane < 0 || wall->plane >= g->nz)) return -1;
    if (wall && g->zbc == OR_Z_WALLS && wall->plane == 0) return -1;   /* the z = 0 PEC wall */
    if (src && g->zbc == OR_Z_WALLS) return -1;   /* the antenna boxes are z-periodic (Section 4) */
    if (src) {
        if (or_antenna_build(g, src, &ant) != 0) { or_antenna_free(&ant); return -1; }
        rc = or_step_all(g, &ant, wall, s, n0, nsteps);
        or_antenna_free(&ant);
    } else {
        rc = or_step_all(g, NULL, wall, s, n0, nsteps);
    }
    return rc;
}

int or_run(const or_grid *g, const or_source *src, or_state *s, long n0, int nsteps)
{
    return or_run_wall(g, src, NULL, s, n0, nsteps);
}

/* Threads of the OpenMP loops (timing of the oracle on the host cores). */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of antenna points per component for a source (for tests). */
int or_antenna_counts(const or_grid *g, const or_source *src, long counts[6])
{
    or_antenna ant;
    if (or_antenna_build(g, src, &ant) != 0) { or_antenna_free(&ant); return -1; }
    for (int c = 0; c < 6; ++c) counts[c] = ant.npts[c];
    or_antenna_free(&ant);
    return 0;
}

/* ------------------------------------------------------------- adjoint */

/* Derivatives of the value added at one antenna point with respect to its
 * column's amplitude and phase weights (s = f Re{ w e^{i phi_w} A e^{-i Phi} }). */
static void src_dweights(const or_source *s, const or_point *p, double cphi, double sphi, double f,
                         double *ds_damp, double *ds_dphase)
{
    double wa = s->w_amp ? s->w_amp[p->col] : 1.0;
    double wp = s->w_phase ? s->w_phase[p->col] : 0.0;
    double zre = cos(wp) * p->are - sin(wp) * p->aim;   /* e^{i phi_w} A */
    double zim = cos(wp) * p->aim + sin(wp) * p->are;
    *ds_damp = f * (zre * cphi + zim * sphi);
    *ds_dphase = f * wa * (-zim * cphi + zre * sphi);
}

static void source_grad(const or_antenna *ant, const or_state *adj, int first, double t,
                        double *grad_amp, double *grad_phase)
{
    double cphi, sphi, f;
    or_source_time(&ant->src, t, &cphi, &sphi, &f);
    for (int c = first; c < first + 3; ++c) {
        const double *lam = (c < 3) ? adj->e[c] : adj->h[c - 3];
        for (long q = 0; q < ant->npts[c]; ++q) {
            const or_point *p = &ant->pts[c][q];
            double da, dp;
            src_dweights(&ant->src, p, cphi, sphi, f, &da, &dp);
            if (grad_amp) grad_amp[p->col] += lam[p->idx] * da;
            if (grad_phase) grad_phase[p->col] += lam[p->idx] * dp;
        }
    }
}

/* add v at (i, j, k) unless (i, j) lies on the virtual +x / +y wall; k wraps */
static inline void acc(const or_grid *g, double *f, long i, long j, long k, double v)
{
    if (i >= g->nx || j >= g->ny || i < 0 || j < 0) return;
    k = ((k % g->nz) + g->nz) % g->nz;
    f[IDX(g, i, j, k)] += v;
}

/* Transpose of update_e: adjoint of E^{n+1} (adj->e), of psi_E^{n+1}
 * (adj->psi_e) -> contributions to the adjoint of H^{n+1/2} (adj->h); psi_E
 * adjoint carried back to step n.  The adjoint of E passes through unchanged. */
static void adjoint_update_e(const or_grid *g, or_state *adj)
{
    double dt = g->dt;
    or_prof px, py;
    prof_build(g, 0, 0, &px);
    prof_build(g, 1, 0, &py);
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long id = IDX(g, i, j, k);
                double bye = py.b[j], aye = py.a[j], kye = py.kappa[j];
                double bxe = px.b[i], axe = px.a[i], kxe = px.kappa[i];
                if (j > 0) {   /* Ex */
                    double e = adj->e[0][id];
                    double ps = adj->psi_e[0][id] + dt * e;
                    double gzy = dt / kye * e + aye * ps;   /* on dHz/dy */
                    double gyz = -dt * e;                  /* on dHy/dz */
                    acc(g, adj->h[2], i, j, k, gzy / g->dy);
                    acc(g, adj->h[2], i, j - 1, k, -gzy / g->dy);
                    acc(g, adj->h[1], i, j, k, gyz / g->dz);
                    acc(g, adj->h[1], i, j, k - 1, -gyz / g->dz);
                    adj->psi_e[0][id] = bye * ps;
                }
                if (i > 0) {   /* Ey */
                    double e = adj->e[1][id];
                    double ps = adj->psi_e[2][id] - dt * e;
                    double gzx = -dt / kxe * e + axe * ps;  /* on dHz/dx */
                    double gxz = dt * e;                    /* on dHx/dz */
                    acc(g, adj->h[2], i, j, k, gzx / g->dx);
                    acc(g, adj->h[2], i - 1, j, k, -gzx / g->dx);
                    acc(g, adj->h[0], i, j, k, gxz / g->dz);
                    acc(g, adj->h[0], i, j, k - 1, -gxz / g->dz);
                    adj->psi_e[2][id] = bxe * ps;
                }
                if (i > 0 && j > 0) {   /* Ez */
                    double e = adj->e[2][id];
                    double psx = adj->psi_e[3][id] + dt * e;
                    double psy = adj->psi_e[1][id] - dt * e;
                    double gyx = dt / kxe * e + axe * psx;   /* on dHy/dx */
                    double gxy = -dt / kye * e + aye * psy;  /* on dHx/dy */
                    acc(g, adj->h[1], i, j, k, gyx / g->dx);
                    acc(g, adj->h[1], i - 1, j, k, -gyx / g->dx);
                    acc(g, adj->h[0], i, j, k, gxy / g->dy);
                    acc(g, adj->h[0], i, j - 1, k, -gxy / g->dy);
                    adj->psi_e[3][id] = bxe * psx;
                    adj->psi_e[1][id] = bye * psy;
                }
            }
    prof_free(&px);
    prof_free(&py);
}

/* Transpose of update_h: adjoint of H^{n+1/2} and psi_H^{n+1/2} ->
 * contributions to the adjoint of E^n; psi_H adjoint carried back. */
static void adjoint_update_h(const or_grid *g, or_state *adj)
{
    double dt = g->dt;
    or_prof px, py;
    prof_build(g, 0, 1, &px);
    prof_build(g, 1, 1, &py);
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long id = IDX(g, i, j, k);
                double byh = py.b[j], ayh = py.a[j], kyh = py.kappa[j];
                double bxh = px.b[i], axh = px.a[i], kxh = px.kappa[i];
                {   /* Hx */
                    double h = adj->h[0][id];
                    double ps = adj->psi_h[0][id] - dt * h;
                    double gzy = -dt / kyh * h + ayh * ps;   /* on dEz/dy */
                    double gyz = dt * h;                    /* on dEy/dz */
                    acc(g, adj->e[2], i, j + 1, k, gzy / g->dy);
                    acc(g, adj->e[2], i, j, k, -gzy / g->dy);
                    acc(g, adj->e[1], i, j, k + 1, gyz / g->dz);
                    acc(g, adj->e[1], i, j, k, -gyz / g->dz);
                    adj->psi_h[0][id] = byh * ps;
                }
                {   /* Hy */
                    double h = adj->h[1][id];
                    double ps = adj->psi_h[2][id] + dt * h;
                    double gzx = dt / kxh * h + axh * ps;    /* on dEz/dx */
                    double gxz = -dt * h;                   /* on dEx/dz */
                    acc(g, adj->e[2], i + 1, j, k, gzx / g->dx);
                    acc(g, adj->e[2], i, j, k, -gzx / g->dx);
                    acc(g, adj->e[0], i, j, k + 1, gxz / g->dz);
                    acc(g, adj->e[0], i, j, k, -gxz / g->dz);
                    adj->psi_h[2][id] = bxh * ps;
                }
                {   /* Hz */
                    double h = adj->h[2][id];
                    double psx = adj->psi_h[3][id] - dt * h;
                    double psy = adj->psi_h[1][id] + dt * h;
                    double gyx = -dt / kxh * h + axh * psx;  /* on dEy/dx */
                    double gxy = dt / kyh * h + ayh * psy;   /* on dEx/dy */
                    acc(g, adj->e[1], i + 1, j, k, gyx / g->dx);
                    acc(g, adj->e[1], i, j, k, -gyx / g->dx);
                    acc(g, adj->e[0], i, j + 1, k, gxy / g->dy);
                    acc(g, adj->e[0], i, j, k, -gxy / g->dy);
                    adj->psi_h[3][id] = bxh * psx;
                    adj->psi_h[1][id] = byh * psy;
                }
            }
    prof_free(&px);
    prof_free(&py);
}

/* One reverse step: the exact transpose of forward step n (E^n, H^{n-1/2},
 * psi -> E^{n+1}, H^{n+1/2}, psi), applied to the adjoint state `adj`
 * (adjoints of E^{n+1}, H^{n+1/2} and psi on entry; of E^n, H^{n-1/2} and
 * psi on return), accumulating dL/dw_amp and dL/dw_phase (nx*ny each, may be
 * NULL) from the source terms of step n.  The caller adds dL/dE^{n+1} to
 * adj->e before the call. */
int or_adjoint_step(const or_grid *g, const or_source *src, or_state *adj, long n,
                    double *grad_amp, double *grad_phase)
{
    or_antenna ant;
    int have = src != NULL;
    if (g->zbc != OR_Z_PERIODIC) return -1;   /* the adjoint covers z-periodic grids only */
    if (have && or_antenna_build(g, src, &ant) != 0) { or_antenna_free(&ant); return -1; }
    /* PEC: E^{n+1} on the walls is forced to zero, so nothing flows back from it */
    for (long k = 0; k < g->nz; ++k)
        for (long j = 0; j < g->ny; ++j)
            for (long i = 0; i < g->nx; ++i) {
                long id = IDX(g, i, j, k);
                if (j == 0) { adj->e[0][id] = 0.0; adj->e[2][id] = 0.0; }
                if (i == 0) { adj->e[1][id] = 0.0; adj->e[2][id] = 0.0; }
            }
    if (have) source_grad(&ant, adj, 0, (n + 1.0) * g->dt, grad_amp, grad_phase);
    adjoint_update_e(g, adj);
    if (have) source_grad(&ant, adj, 3, (n + 0.5) * g->dt, grad_amp, grad_phase);
    adjoint_update_h(g, adj);
    if (have) or_antenna_free(&ant);
    return 0;
}
