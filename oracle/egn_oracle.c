/*
 * egn_oracle.c -- plain, slow FP64 CPU oracle for the ISRS EGN island integral
 * of arXiv 2412.11614 ("Acceleration and Parallelization Methods for ISRS EGN
 * Model").
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference leg may load this library.  The product path
 * (paper_2412_11614_gb300/) never links, imports or executes it, and it shares
 * no source, header, table or helper with the CUDA path.
 *
 * Every routine follows the paper's equations literally, in FP64, with libm:
 *   - SI -> internal unit conversion (THz, ps, km, W)  [Sec. III-A, Table I]
 *   - L_eff(z), rho(z,f), SRS_G(z,f), Delta rho          [Eq. 12-14, 25]
 *   - FWM efficiency mu_s: integral form (adaptive quadrature) [Eq. 23-25],
 *     Maclaurin closed form [Eq. 2-6], segment closed form [Eq. 7-10]
 *   - link function Upsilon as an explicit sum over spans        [Eq. 22]
 *   - islands (kappa1, kappa2, l) / (n1, n2, n3)                [Eq. 15-16]
 *   - the island integrals D, E, F, G, H on a Gauss-Legendre node rule
 *     and on a brute-force midpoint grid                         [Eq. 17-21]
 *   - sigma^2_NLI and eta                                        [Eq. 11, 15]
 *   - modulation-format moments Phi, Psi (enumerated constellations)
 *
 * Readings taken where the paper is silent or garbled:
 *   - the NLI PSD is evaluated at the COI centre and integrated over the COI
 *     as R times that value (2-D islands in f1, f2; white NLI);
 *   - |S(f)|^2 = h(f) / R^2 with h the raised-cosine shape of roll-off beta;
 *   - Phi = mu4 - 2, Psi = mu6 - 9 mu4 + 12 from the moments of the
 *     equiprobable unit-energy constellation (Gaussian: 0, 0);
 *   - every amplifier restores its span exactly (the gain/ISRS products of
 *     Eq. 22 are 1);
 *   - the ISRS profile (Eq. 25) and beta2/beta3 are taken about the spectral
 *     centre (f_min + f_max) / 2, with B_tot = (f_max - f_min) N / (N - 1);
 *   - beta2, beta3 follow from D, S at the reference wavelength, beta2 shifted
 *     by 2 pi beta3 (f_c - f_ref);
 *   - at Cr = 0 (0/0 in Eq. 25) C_k takes its limit 1;
 *   - an island exists only if its overlap has positive area (strict
 *     inequality); E and F coefficients 16/27 and 32/81 as printed.
 *
 * Internal units: frequency THz, time ps, length km, power W.  Then
 * beta2 [ps^2/km] * f^2 [THz^2] is rad/km and zeta = Ptot*Cr*Leff is 1/THz.
 *
 * Parity pins: see tests/test_oracle_*.py.  Absolute eta values are not printed
 * by the paper ("parity unpinned by the paper" for the absolute scale beyond the
 * closed-form and geometric pins listed there).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.141592653589793238462643383279502884
#define OR_C_M_PER_S 299792458.0

/* ------------------------------------------------------------------------- */
/* Data model (internal units)                                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    double alpha;  /* power attenuation [1/km] */
    double beta2;  /* GVD at the spectral centre [ps^2/km] */
    double beta3;  /* dispersion slope [ps^3/km] */
    double gamma;  /* nonlinear coefficient [1/W/km] */
    double cr;     /* Raman gain slope [1/W/km/THz] */
    double L;      /* span length [km] */
} or_span;

enum { OR_MU_SEGMENT = 0, OR_MU_MACLAURIN = 1, OR_MU_INTEGRAL = 2 };

typedef struct {
    int n_ch;
    const double* nu;   /* channel centre relative to the spectral centre [THz] */
    const double* R;    /* symbol rate [THz] */
    const double* P;    /* launch power [W] */
    const double* phi;  /* EGN Phi per channel */
    const double* psi;  /* EGN Psi per channel */
    double rolloff;     /* raised-cosine roll-off */
    double ptot;        /* total launch power [W] */
    double btot;        /* total WDM bandwidth [THz] */
    int n_spans;
    const or_span* spans;
    int gl_order;       /* Gauss-Legendre order n per island (n x n rule) */
    int mu_form;        /* OR_MU_* */
    double dz;          /* segment step Delta z [km] (segment form) */
    double int_tol;     /* relative tolerance of the adaptive integral form */
    int terms;          /* 0 = GN (D only), 1 = EGN (D + corrections) */
    const double* f_off; /* per channel: offset of the frequency f at which the
                            channel is evaluated as COI, from its centre [THz];
                            NULL = 0 (the white-NLI reading) */
} or_problem;

/* ------------------------------------------------------------------------- */
/* Units (Sec. III-A parameter tables)                                        */
/* ------------------------------------------------------------------------- */

/* alpha [dB/km] -> power attenuation [1/km]; D [ps/nm/km], S [ps/nm^2/km] at
 * lambda_ref [m] -> beta2, beta3; beta2 moved from f_ref = c/lambda_ref to the
 * spectral centre fc_hz using beta2(f) = beta2(f_ref) + 2 pi beta3 (f - f_ref). */
void or_units(double alpha_db_km, double D_ps_nm_km, double S_ps_nm2_km,
              double lambda_ref_m, double fc_hz,
              double* alpha, double* beta2, double* beta3)
{
    *alpha = alpha_db_km * log(10.0) / 10.0;
    double D_si = D_ps_nm_km * 1e-6;   /* s/m^2 */
    double S_si = S_ps_nm2_km * 1e3;   /* s/m^3 */
    double lam = lambda_ref_m;
    double a = lam * lam / (2.0 * OR_PI * OR_C_M_PER_S); /* s*m */
    double b2_si = -D_si * a;                            /* s^2/m */
    double b3_si = a * a * (S_si + 2.0 * D_si / lam);    /* s^3/m */
    double b2 = b2_si * 1e27;                            /* ps^2/km */
    double b3 = b3_si * 1e39;                            /* ps^3/km */
    double f_ref_thz = OR_C_M_PER_S / lam * 1e-12;
    double fc_thz = fc_hz * 1e-12;
    *beta2 = b2 + 2.0 * OR_PI * b3 * (fc_thz - f_ref_thz);
    *beta3 = b3;
}

/* ------------------------------------------------------------------------- */
/* ISRS power profile (Appendix A, Eq. 12-14, 25)                             */
/* ------------------------------------------------------------------------- */

/* Effective length L_eff(z) = (1 - e^{-alpha z}) / alpha. */
double or_leff(double alpha, double z)
{
    return -expm1(-alpha * z) / alpha;
}

/* SRS gain, Eq. 14: B P Cr Leff e^{-P Cr Leff f} / (2 sinh(P B Cr Leff / 2)).
 * At Cr = 0 the expression is 0/0; its limit is 1. */
double or_srs_gain(double z, double f, double alpha, double ptot, double cr, double btot)
{
    double zeta = ptot * cr * or_leff(alpha, z);
    double x = btot * zeta;
    if (x == 0.0) return 1.0;
    return x * exp(-zeta * f) / (2.0 * sinh(x / 2.0));
}

/* Normalised signal power profile, Eq. 25 (= Eq. 13): SRS_G * e^{-alpha z}. */
double or_rho(double z, double f, double alpha, double ptot, double cr, double btot)
{
    return or_srs_gain(z, f, alpha, ptot, cr, btot) * exp(-alpha * z);
}

/* Edge-channel power transfer, Eq. 12, with the paper's "4.3" read as 10 log10(e). */
double or_delta_rho_db(double alpha, double L, double ptot, double cr, double btot)
{
    return 10.0 * log10(exp(1.0)) * ptot * cr * or_leff(alpha, L) * btot;
}

/* Phase mismatch per unit length, Eq. 5 / Eq. 24 without z. */
double or_chi(double f1, double f2, double f, double beta2, double beta3)
{
    return 4.0 * OR_PI * OR_PI * (f1 - f) * (f2 - f) * (beta2 + OR_PI * beta3 * (f1 + f2));
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre nodes on [-1, 1] (Newton iteration on P_n)                  */
/* ------------------------------------------------------------------------- */

void or_gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double t = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-15) break;
        }
        /* recompute derivative at the converged node */
        {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        /* ascending order */
        x[n - 1 - i] = t;
        w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* ------------------------------------------------------------------------- */
/* FWM efficiency factor mu_s(f1, f2, f)                                      */
/* ------------------------------------------------------------------------- */

/* Eq. 6 (the paper's "eta", called mu_lin here): (e^{(i chi - alpha) L} - 1)/(i chi - alpha). */
cplx or_mu_lin(double chi, double alpha, double L)
{
    cplx g = I * chi - alpha;
    return (cexp(g * L) - 1.0) / g;
}

/* Segment count K = ceil(L / dz) (Sec. II-C-2). */
int or_segments(double L, double dz)
{
    int K = (int)ceil(L / dz);
    return K < 1 ? 1 : K;
}

/* Segment closed form, Eq. 8-10, term by term. */
cplx or_mu_segment(double chi, double f3, const or_span* s, double ptot, double btot, int K)
{
    cplx g = I * chi - s->alpha;
    cplx sum = 0.0;
    for (int k = 0; k < K; ++k) {
        double zk = (k + 0.5) / K * s->L;                                  /* Eq. 10 */
        double srsg = or_srs_gain(zk, f3, s->alpha, ptot, s->cr, btot);    /* Eq. 14 */
        double za = (double)(k + 1) / K * s->L;
        double zb = (double)k / K * s->L;
        cplx Ik = (cexp(g * za) - cexp(g * zb)) / g;                       /* Eq. 9 */
        sum += srsg * Ik;                                                  /* Eq. 8 */
    }
    return sum;
}

/* Maclaurin closed form, Eq. 4-6. */
cplx or_mu_maclaurin(double chi, double f3, const or_span* s, double ptot)
{
    cplx g1 = I * chi - s->alpha;
    cplx g2 = I * chi - 2.0 * s->alpha;
    cplx eta = (cexp(g1 * s->L) - 1.0) / g1;
    cplx second = (cexp(g2 * s->L) - 1.0) / g2;
    return eta - (ptot * s->cr * f3 / s->alpha) * (eta - second);
}

/* Integral form, Eq. 23 with Eq. 24-25: adaptive Gauss-Legendre quadrature.
 * [0, L] is first cut into pieces no longer than a quarter period of the phase
 * factor; each piece is refined by bisection until the 10-point rule on the
 * piece agrees with the sum over its two halves. */
typedef struct {
    double chi, f3, alpha, ptot, cr, btot;
    const double* gx;
    const double* gw;
    int gn;
} or_int_ctx;

static cplx or_int_f(const or_int_ctx* c, double z)
{
    return or_rho(z, c->f3, c->alpha, c->ptot, c->cr, c->btot) * cexp(I * c->chi * z);
}

static cplx or_int_gl(const or_int_ctx* c, double a, double b)
{
    double m = 0.5 * (a + b), h = 0.5 * (b - a);
    cplx s = 0.0;
    for (int i = 0; i < c->gn; ++i) s += c->gw[i] * or_int_f(c, m + h * c->gx[i]);
    return s * h;
}

static cplx or_int_adapt(const or_int_ctx* c, double a, double b, cplx whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    cplx left = or_int_gl(c, a, m);
    cplx right = or_int_gl(c, m, b);
    cplx both = left + right;
    if (depth >= 30 || cabs(both - whole) <= tol) return both;
    return or_int_adapt(c, a, m, left, 0.5 * tol, depth + 1) +
           or_int_adapt(c, m, b, right, 0.5 * tol, depth + 1);
}

cplx or_mu_integral(double chi, double f3, const or_span* s, double ptot, double btot, double rel_tol)
{
    double gx[10], gw[10];
    or_gauss_legendre(10, gx, gw);
    or_int_ctx c = {chi, f3, s->alpha, ptot, s->cr, btot, gx, gw, 10};
    double quarter = (chi != 0.0) ? OR_PI / (2.0 * fabs(chi)) : s->L;
    long npieces = (long)ceil(s->L / quarter);
    if (npieces < 1) npieces = 1;
    double h = s->L / (double)npieces;
    double tol = rel_tol * or_leff(s->alpha, s->L) / (double)npieces;
    cplx sum = 0.0;
    for (long p = 0; p < npieces; ++p) {
        double a = p * h, b = (p + 1 == npieces) ? s->L : (p + 1) * h;
        cplx whole = or_int_gl(&c, a, b);
        sum += or_int_adapt(&c, a, b, whole, tol, 0);
    }
    return sum;
}

/* mu_s for span s, with f1, f2, f total frequencies relative to the spectral centre. */
cplx or_mu(const or_problem* pb, const or_span* s, double f1, double f2, double f)
{
    double chi = or_chi(f1, f2, f, s->beta2, s->beta3);
    double f3 = f1 + f2 - f;
    switch (pb->mu_form) {
    case OR_MU_MACLAURIN:
        return or_mu_maclaurin(chi, f3, s, pb->ptot);
    case OR_MU_INTEGRAL:
        return or_mu_integral(chi, f3, s, pb->ptot, pb->btot, pb->int_tol);
    default:
        return or_mu_segment(chi, f3, s, pb->ptot, pb->btot, or_segments(s->L, pb->dz));
    }
}

/* ------------------------------------------------------------------------- */
/* Link function, Eq. 22: explicit coherent sum over spans                    */
/* ------------------------------------------------------------------------- */

/* Upsilon(f1, f2, f) = sum_s gamma_s mu_s e^{i sum_{s'<s} chi_{s'} L_{s'}} with
 * the gain/ISRS products equal to 1 under ideal per-span power restoration.
 * mu_s is recomputed for every span except when the span's parameters equal
 * the previous span's (then mu_s is the same number). */
cplx or_upsilon(const or_problem* pb, double f1, double f2, double f)
{
    cplx Y = 0.0;
    double acc = 0.0;
    cplx mu = 0.0;
    const or_span* prev = NULL;
    for (int s = 0; s < pb->n_spans; ++s) {
        const or_span* sp = &pb->spans[s];
        if (!prev || memcmp(prev, sp, sizeof(or_span)) != 0) mu = or_mu(pb, sp, f1, f2, f);
        prev = sp;
        Y += sp->gamma * mu * cexp(I * acc);
        acc += 4.0 * OR_PI * OR_PI * (f1 - f) * (f2 - f) *
               (sp->beta2 * sp->L + OR_PI * (f1 + f2) * sp->beta3 * sp->L);
    }
    return Y;
}

/* ------------------------------------------------------------------------- */
/* Spectra and islands                                                        */
/* ------------------------------------------------------------------------- */

/* Raised-cosine power shape h(x) (unit in band), support |x| <= (1+beta) R / 2. */
double or_rc(double x, double R, double beta)
{
    double ax = fabs(x);
    double a = 0.5 * (1.0 - beta) * R, b = 0.5 * (1.0 + beta) * R;
    if (ax <= a) return 1.0;
    if (ax >= b) return 0.0;
    return 0.5 * (1.0 + cos(OR_PI / (beta * R) * (ax - a)));
}

static double or_width(const or_problem* pb, int n) { return pb->R[n] * (1.0 + pb->rolloff); }

/* The frequency f at which COI n is evaluated: its centre, plus f_off[n]. */
static double or_fcoi(const or_problem* pb, int n)
{
    return pb->nu[n] + (pb->f_off ? pb->f_off[n] : 0.0);
}

/* Frequency offset of the island: d = (nu_n1 - f) + (nu_n2 - nu_n3), with f the
 * COI's evaluation frequency (its centre unless f_off is set). */
static double or_offset(const or_problem* pb, int n, int n1, int n2, int n3)
{
    return (pb->nu[n1] - or_fcoi(pb, n)) + (pb->nu[n2] - pb->nu[n3]);
}

/* Node rule.  Outer variable o with |o| <= A, inner variable t with |t| <= B,
 * coupled by |t - (s*o + c)| <= C.  Writes the outer panel edges (2..4 values)
 * and returns the number of panels, 0 if the island has zero area. */
static int or_panels(double A, double B, double s, double c, double C, double* e)
{
    double p = s * (-(B + C) - c), q = s * ((B + C) - c);
    double lo = fmax(-A, fmin(p, q));
    double hi = fmin(A, fmax(p, q));
    if (!(hi > lo)) return 0;
    double k1 = s * ((C - B) - c);
    double k2 = s * ((B - C) - c);
    if (k1 > k2) { double t = k1; k1 = k2; k2 = t; }
    int n = 0;
    e[n++] = lo;
    if (k1 > lo && k1 < hi) e[n++] = k1;
    if (k2 > lo && k2 < hi && k2 != k1) e[n++] = k2;
    e[n++] = hi;
    return n - 1;
}

static void or_inner(double B, double s, double c, double C, double o, double* lo, double* hi)
{
    double m = s * o + c;
    *lo = fmax(-B, m - C);
    *hi = fmin(B, m + C);
}

/* Island existence: the (outer w, inner u) region of Eq. 17 has positive area. */
int or_island_exists(const or_problem* pb, int n, int n1, int n2, int n3)
{
    double e[4];
    double d = or_offset(pb, n, n1, n2, n3);
    return or_panels(0.5 * or_width(pb, n3), 0.5 * or_width(pb, n1), 1.0, -d,
                     0.5 * or_width(pb, n2), e) > 0;
}

/* All islands of COI n by brute force over (n1, n2, n3), lexicographic order.
 * Writes up to max triples; returns the count. */
long or_islands(const or_problem* pb, int n, int* out, long max)
{
    long cnt = 0;
    for (int n1 = 0; n1 < pb->n_ch; ++n1)
        for (int n2 = 0; n2 < pb->n_ch; ++n2)
            for (int n3 = 0; n3 < pb->n_ch; ++n3)
                if (or_island_exists(pb, n, n1, n2, n3)) {
                    if (out && cnt < max) {
                        out[3 * cnt + 0] = n1;
                        out[3 * cnt + 1] = n2;
                        out[3 * cnt + 2] = n3;
                    }
                    ++cnt;
                }
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Island integrals, Eq. 17-21, on the Gauss-Legendre node rule               */
/* ------------------------------------------------------------------------- */

enum { OR_T_D = 0, OR_T_E = 1, OR_T_F = 2, OR_T_G = 3, OR_T_H = 4 };

/* Coefficients of D..H after |S|^2 = h/R^2 and int df -> R (value at f = 0). */
static void or_coefs(const or_problem* pb, int n, int n1, int n2, int n3, double* cf)
{
    double R = pb->R[n];
    cf[OR_T_D] = (16.0 / 27.0) * R / (pb->R[n1] * pb->R[n2] * pb->R[n3]);
    cf[OR_T_E] = (16.0 / 27.0) / (R * R * R);
    cf[OR_T_F] = (32.0 / 81.0) / (R * R * R);
    cf[OR_T_G] = (16.0 / 81.0) / (R * R * R);
    cf[OR_T_H] = (16.0 / 81.0) / (R * R * R * R);
}

/* Walk the node rule of one ordering and evaluate
 *   outer sum  sum_i wo_i * ho(o_i) * |sum_j wi_j * a(t_j, o_i) * Y|^2   (mode 1)
 * or the plain D / H sums (mode 0, DW ordering only).
 * ordering: 0 = (outer w, inner u), 1 = (outer v, inner u), 2 = (outer u, inner v). */
static void or_walk(const or_problem* pb, int n, int n1, int n2, int n3, int ordering,
                    const double* gx, const double* gw, int gn,
                    double* D, double* corr, cplx* Hsum)
{
    double W1 = or_width(pb, n1), W2 = or_width(pb, n2), W3 = or_width(pb, n3);
    double R1 = pb->R[n1], R2 = pb->R[n2], R3 = pb->R[n3];
    double beta = pb->rolloff;
    double d = or_offset(pb, n, n1, n2, n3);
    double A, B, s, c, C;
    if (ordering == 0) { A = 0.5 * W3; B = 0.5 * W1; s = 1.0; c = -d; C = 0.5 * W2; }
    else if (ordering == 1) { A = 0.5 * W2; B = 0.5 * W1; s = -1.0; c = -d; C = 0.5 * W3; }
    else { A = 0.5 * W1; B = 0.5 * W2; s = -1.0; c = -d; C = 0.5 * W3; }
    double e[4];
    int np = or_panels(A, B, s, c, C, e);
    double dsum = 0.0, csum = 0.0;
    cplx hsum = 0.0;
    if (np == 0) { *D = 0; *corr = 0; *Hsum = 0; return; }
    int no = (gn + np - 1) / np;
    double* ox = (double*)malloc(sizeof(double) * no);
    double* ow = (double*)malloc(sizeof(double) * no);
    or_gauss_legendre(no, ox, ow);
    double f = or_fcoi(pb, n);
    for (int p = 0; p < np; ++p) {
        double pm = 0.5 * (e[p] + e[p + 1]), ph = 0.5 * (e[p + 1] - e[p]);
        for (int i = 0; i < no; ++i) {
            double o = pm + ph * ox[i];
            double wo = ph * ow[i];
            double lo, hi;
            or_inner(B, s, c, C, o, &lo, &hi);
            double im = 0.5 * (lo + hi), ih = 0.5 * (hi - lo);
            cplx inner = 0.0;
            for (int j = 0; j < gn; ++j) {
                double t = im + ih * gx[j];
                double wi = ih * gw[j];
                double u, v, w;
                if (ordering == 0) { w = o; u = t; v = w - u - d; }
                else if (ordering == 1) { v = o; u = t; w = u + v + d; }
                else { u = o; v = t; w = u + v + d; }
                double h1 = or_rc(u, R1, beta), h2 = or_rc(v, R2, beta), h3 = or_rc(w, R3, beta);
                cplx Y = or_upsilon(pb, pb->nu[n1] + u, pb->nu[n2] + v, f);
                if (ordering == 0) {
                    dsum += wo * wi * h1 * h2 * h3 * creal(Y * conj(Y));
                    inner += wi * sqrt(h1 * h2) * Y;          /* G inner (along w = const) */
                    hsum += wo * wi * sqrt(h1 * h2 * h3) * Y;  /* H */
                } else if (ordering == 1) {
                    inner += wi * sqrt(h1 * h3) * Y;          /* E inner (over u at fixed v) */
                } else {
                    inner += wi * sqrt(h2 * h3) * Y;          /* F inner (over v at fixed u) */
                }
            }
            double outer_shape;
            if (ordering == 0) outer_shape = or_rc(o, R3, beta);       /* h3(w) */
            else if (ordering == 1) outer_shape = or_rc(o, R2, beta);  /* h2(v) */
            else outer_shape = or_rc(o, R1, beta);                     /* h1(u) */
            csum += wo * outer_shape * creal(inner * conj(inner));
        }
    }
    free(ox);
    free(ow);
    *D = dsum;
    *corr = csum;
    *Hsum = hsum;
}

/* D, E, F, G, H of island (n1, n2, n3) for COI n (Eq. 17-21 with the readings
 * in the header of this file).  With all = 0 only the terms selected by the Kronecker deltas of
 * Eq. 15 are evaluated (others set to 0); with all = 1 every term is evaluated. */
void or_island_terms(const or_problem* pb, int n, int n1, int n2, int n3, int all, double* out)
{
    int gn = pb->gl_order;
    double* gx = (double*)malloc(sizeof(double) * 2 * (size_t)gn);
    double* gw = gx + gn;
    or_gauss_legendre(gn, gx, gw);
    double cf[5];
    or_coefs(pb, n, n1, n2, n3, cf);
    for (int t = 0; t < 5; ++t) out[t] = 0.0;
    double D, corr;
    cplx H;
    int egn = pb->terms != 0;
    or_walk(pb, n, n1, n2, n3, 0, gx, gw, gn, &D, &corr, &H);
    out[OR_T_D] = cf[OR_T_D] * D;
    if (all || (egn && n1 == n2)) out[OR_T_G] = cf[OR_T_G] * corr;
    if (all || (egn && n1 == n2 && n2 == n3)) out[OR_T_H] = cf[OR_T_H] * creal(H * conj(H));
    if (all || (egn && n1 == n3)) {
        double dd;
        cplx hh;
        or_walk(pb, n, n1, n2, n3, 1, gx, gw, gn, &dd, &corr, &hh);
        out[OR_T_E] = cf[OR_T_E] * corr;
    }
    if (all || (egn && n2 == n3)) {
        double dd;
        cplx hh;
        or_walk(pb, n, n1, n2, n3, 2, gx, gw, gn, &dd, &corr, &hh);
        out[OR_T_F] = cf[OR_T_F] * corr;
    }
    free(gx);
}

/* Brute force: the same five integrals on a dense midpoint grid of M x M cells
 * over the bounding rectangle of each ordering, with the channel supports
 * entering only through the spectral shapes (no panels, no kinks). */
void or_island_terms_midpoint(const or_problem* pb, int n, int n1, int n2, int n3, int M, double* out)
{
    double W1 = or_width(pb, n1), W2 = or_width(pb, n2), W3 = or_width(pb, n3);
    double R1 = pb->R[n1], R2 = pb->R[n2], R3 = pb->R[n3];
    double beta = pb->rolloff;
    double d = or_offset(pb, n, n1, n2, n3);
    double f = or_fcoi(pb, n);
    double cf[5];
    or_coefs(pb, n, n1, n2, n3, cf);
    /* (w, u) grid: D, G, H */
    double dw = W3 / M, du = W1 / M, dv = W2 / M;
    double Dsum = 0.0, Gsum = 0.0;
    cplx Hsum = 0.0;
    for (int i = 0; i < M; ++i) {
        double w = -0.5 * W3 + (i + 0.5) * dw;
        cplx inner = 0.0;
        for (int j = 0; j < M; ++j) {
            double u = -0.5 * W1 + (j + 0.5) * du;
            double v = w - u - d;
            double h1 = or_rc(u, R1, beta), h2 = or_rc(v, R2, beta), h3 = or_rc(w, R3, beta);
            if (h1 * h2 * h3 == 0.0) continue;
            cplx Y = or_upsilon(pb, pb->nu[n1] + u, pb->nu[n2] + v, f);
            Dsum += dw * du * h1 * h2 * h3 * creal(Y * conj(Y));
            inner += du * sqrt(h1 * h2) * Y;
            Hsum += dw * du * sqrt(h1 * h2 * h3) * Y;
        }
        Gsum += dw * or_rc(w, R3, beta) * creal(inner * conj(inner));
    }
    /* (v, u) grid: E */
    double Esum = 0.0;
    for (int i = 0; i < M; ++i) {
        double v = -0.5 * W2 + (i + 0.5) * dv;
        cplx inner = 0.0;
        for (int j = 0; j < M; ++j) {
            double u = -0.5 * W1 + (j + 0.5) * du;
            double w = u + v + d;
            double h1 = or_rc(u, R1, beta), h3 = or_rc(w, R3, beta);
            if (h1 * h3 == 0.0) continue;
            cplx Y = or_upsilon(pb, pb->nu[n1] + u, pb->nu[n2] + v, f);
            inner += du * sqrt(h1 * h3) * Y;
        }
        Esum += dv * or_rc(v, R2, beta) * creal(inner * conj(inner));
    }
    /* (u, v) grid: F */
    double Fsum = 0.0;
    for (int i = 0; i < M; ++i) {
        double u = -0.5 * W1 + (i + 0.5) * du;
        cplx inner = 0.0;
        for (int j = 0; j < M; ++j) {
            double v = -0.5 * W2 + (j + 0.5) * dv;
            double w = u + v + d;
            double h2 = or_rc(v, R2, beta), h3 = or_rc(w, R3, beta);
            if (h2 * h3 == 0.0) continue;
            cplx Y = or_upsilon(pb, pb->nu[n1] + u, pb->nu[n2] + v, f);
            inner += dv * sqrt(h2 * h3) * Y;
        }
        Fsum += du * or_rc(u, R1, beta) * creal(inner * conj(inner));
    }
    out[OR_T_D] = cf[OR_T_D] * Dsum;
    out[OR_T_E] = cf[OR_T_E] * Esum;
    out[OR_T_F] = cf[OR_T_F] * Fsum;
    out[OR_T_G] = cf[OR_T_G] * Gsum;
    out[OR_T_H] = cf[OR_T_H] * creal(Hsum * conj(Hsum));
}

/* Contribution of one island to sigma^2_NLI of COI n, Eq. 15. */
static double or_island_pnli(const or_problem* pb, int n, int n1, int n2, int n3, const double* t)
{
    double s = t[OR_T_D];
    if (pb->terms != 0) {
        if (n1 == n3) s += pb->phi[n1] * t[OR_T_E];
        if (n2 == n3) s += pb->phi[n2] * t[OR_T_F];
        if (n1 == n2) s += pb->phi[n1] * t[OR_T_G];
        if (n1 == n2 && n2 == n3) s += pb->psi[n1] * t[OR_T_H];
    }
    return pb->P[n1] * pb->P[n2] * pb->P[n3] * s;
}

/* sigma^2_NLI (= P_NLI [W]) and eta = P_NLI / P_n^3 [1/W^2] (Eq. 11, 15) for the
 * listed COIs (all if coi == NULL).  Islands run in parallel; their
 * contributions are stored and summed serially in island order. */
int or_eta(const or_problem* pb, const int* coi, int n_coi, double* eta, double* pnli)
{
    int total = coi ? n_coi : pb->n_ch;
    int* tri = (int*)malloc(sizeof(int) * 3 * (size_t)pb->n_ch * pb->n_ch * 3 + 3);
    if (!tri) return -1;
    for (int q = 0; q < total; ++q) {
        int n = coi ? coi[q] : q;
        long cap = (long)pb->n_ch * pb->n_ch * 3;
        long ni = or_islands(pb, n, tri, cap);
        if (ni > cap) { free(tri); return -2; }
        double* contrib = (double*)malloc(sizeof(double) * (ni > 0 ? ni : 1));
        long i;
#pragma omp parallel for schedule(dynamic, 1)
        for (i = 0; i < ni; ++i) {
            double t[5];
            or_island_terms(pb, n, tri[3 * i], tri[3 * i + 1], tri[3 * i + 2], 0, t);
            contrib[i] = or_island_pnli(pb, n, tri[3 * i], tri[3 * i + 1], tri[3 * i + 2], t);
        }
        double s = 0.0;
        for (i = 0; i < ni; ++i) s += contrib[i];
        free(contrib);
        pnli[q] = s;
        eta[q] = s / (pb->P[n] * pb->P[n] * pb->P[n]);
    }
    free(tri);
    return 0;
}

/* Per-island contributions (Eq. 15 summand) for COI n in island order. */
long or_island_contribs(const or_problem* pb, int n, int* tri, double* contrib, long max)
{
    long ni = or_islands(pb, n, tri, max);
    if (ni > max) return -ni;
    long i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < ni; ++i) {
        double t[5];
        or_island_terms(pb, n, tri[3 * i], tri[3 * i + 1], tri[3 * i + 2], 0, t);
        contrib[i] = or_island_pnli(pb, n, tri[3 * i], tri[3 * i + 1], tri[3 * i + 2], t);
    }
    return ni;
}

/* Outer/inner node coordinates of island (n1, n2, n3) in the (w, u) ordering:
 * writes (u, v, weight) per node, returns the node count (<= max). */
long or_island_nodes(const or_problem* pb, int n, int n1, int n2, int n3, double* uvw, long max)
{
    int gn = pb->gl_order;
    double W1 = or_width(pb, n1), W2 = or_width(pb, n2), W3 = or_width(pb, n3);
    double d = or_offset(pb, n, n1, n2, n3);
    double e[4];
    int np = or_panels(0.5 * W3, 0.5 * W1, 1.0, -d, 0.5 * W2, e);
    if (np == 0) return 0;
    int no = (gn + np - 1) / np;
    double* gx = (double*)malloc(sizeof(double) * 2 * (size_t)(gn + no));
    double *gw = gx + gn, *ox = gw + gn, *ow = ox + no;
    or_gauss_legendre(gn, gx, gw);
    or_gauss_legendre(no, ox, ow);
    long cnt = 0;
    for (int p = 0; p < np; ++p) {
        double pm = 0.5 * (e[p] + e[p + 1]), ph = 0.5 * (e[p + 1] - e[p]);
        for (int i = 0; i < no; ++i) {
            double w = pm + ph * ox[i];
            double lo, hi;
            or_inner(0.5 * W1, 1.0, -d, 0.5 * W2, w, &lo, &hi);
            double im = 0.5 * (lo + hi), ih = 0.5 * (hi - lo);
            for (int j = 0; j < gn; ++j) {
                double u = im + ih * gx[j];
                if (cnt < max) {
                    uvw[3 * cnt + 0] = u;
                    uvw[3 * cnt + 1] = w - u - d;
                    uvw[3 * cnt + 2] = ph * ow[i] * ih * gw[j];
                }
                ++cnt;
            }
        }
    }
    free(gx);
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Modulation-format moments                                                  */
/* ------------------------------------------------------------------------- */

/* Phi = mu4 - 2, Psi = mu6 - 9 mu4 + 12 with mu_k = E|a|^k / (E|a|^2)^{k/2} of the
 * equiprobable square constellation with m points per dimension (m = 2: QPSK,
 * 4: 16QAM, 8: 64QAM), enumerated point by point; m = 0 is the complex Gaussian
 * limit (mu4 = 2, mu6 = 6). */
int or_format_moments(int m, double* phi, double* psi)
{
    if (m == 0) { *phi = 0.0; *psi = 0.0; return 0; }
    if (m < 2 || m > 64) return -1;
    double e2 = 0.0, e4 = 0.0, e6 = 0.0;
    int cnt = 0;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            double re = 2.0 * a - (m - 1), im = 2.0 * b - (m - 1);
            double r2 = re * re + im * im;
            e2 += r2;
            e4 += r2 * r2;
            e6 += r2 * r2 * r2;
            ++cnt;
        }
    e2 /= cnt;
    e4 /= cnt;
    e6 /= cnt;
    double mu4 = e4 / (e2 * e2), mu6 = e6 / (e2 * e2 * e2);
    *phi = mu4 - 2.0;
    *psi = mu6 - 9.0 * mu4 + 12.0;
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Out-pointer wrappers for the complex-valued routines (ctypes has no complex) */
/* ------------------------------------------------------------------------- */

static void or_put(cplx z, double* out) { out[0] = creal(z); out[1] = cimag(z); }

void or_mu_lin_out(double chi, double alpha, double L, double* out) { or_put(or_mu_lin(chi, alpha, L), out); }

void or_mu_segment_out(double chi, double f3, const or_span* s, double ptot, double btot, int K, double* out)
{
    or_put(or_mu_segment(chi, f3, s, ptot, btot, K), out);
}

void or_mu_maclaurin_out(double chi, double f3, const or_span* s, double ptot, double* out)
{
    or_put(or_mu_maclaurin(chi, f3, s, ptot), out);
}

void or_mu_integral_out(double chi, double f3, const or_span* s, double ptot, double btot, double rel_tol, double* out)
{
    or_put(or_mu_integral(chi, f3, s, ptot, btot, rel_tol), out);
}

void or_upsilon_out(const or_problem* pb, double f1, double f2, double f, double* out)
{
    or_put(or_upsilon(pb, f1, f2, f), out);
}

/* Batched evaluation of Upsilon at n points (f1[i], f2[i], f) in parallel. */
void or_upsilon_many(const or_problem* pb, long n, const double* f1, const double* f2, double f, double* out)
{
    long i;
#pragma omp parallel for schedule(dynamic, 64)
    for (i = 0; i < n; ++i) or_put(or_upsilon(pb, f1[i], f2[i], f), out + 2 * i);
}
