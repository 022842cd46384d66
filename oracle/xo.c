/*
 * xo.c -- plain, slow FP64 CPU oracle for the line-list -> cross-section path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the only thing
 * both sides share is the seeded input generator (xcsynth), which holds none
 * of the method's arithmetic.
 *
 * Everything here is written from the ExoCross paper (Yurchenko, Al-Refaie &
 * Tennyson 2018, arXiv:1801.09803), in its notation, in the order it gives:
 *   Q(T)          Eq. (e:pf)   direct state sum
 *   I_fi          Eq. (e:int)  LTE absorption intensity, upper degeneracy
 *   eps_fi        Eq. (e:emiss) LTE emissivity from the upper state (E' = E'' + nu),
 *                 with the photon energy h c nu so that it comes out in the unit the
 *                 text gives (erg/s/sr per molecule; the printed formula omits h c)
 *   VV / VVN      Sec. "Vectorized Voigt approximation", Eq. (e:fast-v), (e:beta): the w4
 *                 Voigt within `split` (4 cm^-1) of the centre, beyond it the reference
 *                 profile -- the Voigt of a line at 1 cm^-1 (alpha_ref = alpha / nu), same
 *                 gamma -- times beta (1, or the ratio that makes it continuous at split),
 *                 at the line's own offsets; VVN (Sec. "Binned Vectorized Voigt") divides
 *                 I by Sigma = h sum_k f(nu_k - nu), the sum over the line's cut window on
 *                 the grid's lattice (also past the grid ends), so that each line's area is I
 *   broadening    Sec. "Broadening parameters" (.broad): per broadener a constant
 *                 (gamma_0, n_L), or a table by J'' (a0) or by (J'', J') (a1), with the
 *                 broadener's defaults for a line whose quantum numbers it does not
 *                 list; Sec. "Mixtures of broadeners": gamma_L = sum_i rho_i gamma_i
 *   thresholds    Sec. "Intensity thresholds": constant, or HITRAN's dynamic
 *                 I_crit (nu/nu_crit) tanh(c2 nu / 2T) below nu_crit, I_crit above;
 *                 a line whose intensity (or emissivity) is below it is left out
 *   alpha_D       Eq. (e:alphaD)
 *   gamma_L       Eq. (e:gamma_L)
 *   Gauss         Eq. (e:Gauss)        Lorentz  Eq. (e:lor)
 *   Voigt         Eq. (e:Voigt), read as the unit-area convolution
 *                 V = sqrt(ln2/pi)/alpha * Re w(x+iy), x = sqrt(ln2) D/alpha,
 *                 y = sqrt(ln2) gamma/alpha  (the printed prefactor is garbled)
 *   w(z)          Humlicek's four-region rational approximation "w4"
 *                 (J. Humlicek, JQSRT 27 (1982) 437), restated below
 *   GH sampled    Eq. (e:V-quad) with the node shift alpha*x_j/sqrt(ln2)
 *   GH binned     Eq. (e:sigma:quad), y^+- = (nu_k +- dnu/2 - nu_fi - alpha x_j/sqrt(ln2))/gamma
 *   Gauss binned  Eq. (eqn:sig_ij), bin average by the erf difference, Sec. "Binned Gaussian"
 *   Lorentz binned Eq. (eqn:sig_lor-2), bin average by the arctan difference, with
 *                 y^+- = (nu_k +- dnu/2 - nu_fi)/gamma (Eq. e:y_k^pm read with its lost minus)
 *   sampling      sigma(nu_k) = sum_fi I_fi f(nu_k)  (Sec. 3.1), lines outer,
 *                 grid points inner, within the cutoff ("Off-set", Sec. 3.10)
 *   grid          nu_k = nu_A + k * dnu, N points including both ends, Eq. (e:Ngrid)
 *
 * Readings where the paper is silent: the cutoff test is inclusive,
 * |nu_k - nu_fi| <= cut; accumulation is FP64 with Neumaier compensation;
 * OpenMP threads (the paper's own design, Sec. 5.3) each own a private grid
 * over a contiguous block of lines and are combined in thread order.
 *
 * The adjoint (vector-Jacobian product) is not in the paper; it is the
 * analytic chain rule of the same expressions (see xo_cross_section_vjp).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -shared -fPIC xo.c -lm
 * (-ffp-contract=off keeps a*b+c as two roundings on every host.)
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 exact SI values */
static const double XO_H = 6.62607015e-34;      /* J s */
static const double XO_C_SI = 2.99792458e8;     /* m/s */
static const double XO_KB = 1.380649e-23;       /* J/K */
static const double XO_DALTON = 1.66053906660e-27; /* kg */

static const double XO_PI = 3.14159265358979323846;
static const double XO_LN2 = 0.69314718055994530942;

double xo_c2(void) { return XO_H * (XO_C_SI * 100.0) / XO_KB; } /* cm K */

enum { XO_DOPPLER = 0, XO_LORENTZ = 1, XO_VOIGT_W4 = 2, XO_GH_BINNED = 3, XO_GH_SAMPLED = 4,
       XO_DOPPLER_BINNED = 5, XO_LORENTZ_BINNED = 6, XO_VOIGT_VV = 7 };

/* ---------------------------------------------------------------------- */
/* Partition function, Eq. (e:pf), and its temperature derivative          */
/* ---------------------------------------------------------------------- */
void xo_partition_function(const double *E, const int32_t *g, size_t n, double T,
                           double *Q, double *dQdT)
{
    const double c2 = xo_c2();
    double q = 0.0, dq = 0.0;
    for (size_t i = 0; i < n; ++i) {
        double b = exp(-c2 * E[i] / T);
        q += (double)g[i] * b;
        dq += (double)g[i] * (c2 * E[i] / (T * T)) * b;
    }
    *Q = q;
    if (dQdT) *dQdT = dq;
}

/* ---------------------------------------------------------------------- */
/* Per-line parameters for one condition                                  */
/* ---------------------------------------------------------------------- */
typedef struct {
    double T, P, Q, dQdT;       /* K, units of P_ref, -, 1/K */
    double mass_da, T_ref, P_ref;
    double gamma_scale, n_shift;
    double abundance;
} xo_condition;

typedef struct {
    int profile;                 /* XO_* */
    double cutoff;               /* cm^-1 */
    double width_mult;           /* > 0: cut_l = min(cutoff, width_mult*max(alpha, gamma)) */
    int n_gh;
    int quantity;                /* 0: absorption, Eq. (e:int); 1: emission, Eq. (e:emiss) */
    int thr_mode;                /* 0: none; 1: constant I_cut; 2: HITRAN dynamic (nu_crit, I_crit) */
    double I_cut, nu_crit, I_crit;
    double vv_split;             /* XO_VOIGT_VV: the exact-Voigt zone |nu - nu_fi| <= vv_split */
    int vv_beta;                 /* 1: beta of Eq. (e:beta), 0: beta = 1 */
    int vv_norm;                 /* 1: VVN, the line area renormalised to I */
} xo_opts;

/* Eq. (e:int): I = g' A / (8 pi c nu^2) * exp(-c2 E''/T) * (1 - exp(-c2 nu/T)) / Q(T) */
double xo_intensity(double nu, double elower, double A, double g_up, const xo_condition *c)
{
    const double c2 = xo_c2();
    const double c_cm = XO_C_SI * 100.0;
    double boltz = exp(-c2 * elower / c->T);
    double stim = -expm1(-c2 * nu / c->T);
    return c->abundance * g_up * A / (8.0 * XO_PI * c_cm * nu * nu) * boltz * stim / c->Q;
}

/* Eq. (e:emiss): emissivity of the line from its upper state, E' = E'' + nu, times the
 * photon energy h c nu (erg): g' A h c nu / (4 pi) * exp(-c2 E'/T) / Q(T) */
double xo_emissivity(double nu, double elower, double A, double g_up, const xo_condition *c)
{
    const double c2 = xo_c2();
    const double c_cm = XO_C_SI * 100.0;
    const double h_erg = XO_H * 1e7;
    double boltz = exp(-c2 * (elower + nu) / c->T);
    return c->abundance * g_up * A * (h_erg * c_cm * nu) / (4.0 * XO_PI) * boltz / c->Q;
}

/* Intensity threshold at wavenumber nu (Sec. "Intensity thresholds"): 0 = none */
double xo_threshold(double nu, double T, const xo_opts *o)
{
    if (o->thr_mode == 1) return o->I_cut;
    if (o->thr_mode == 2) {
        if (nu > o->nu_crit) return o->I_crit;
        return o->I_crit * (nu / o->nu_crit) * tanh(xo_c2() * nu / (2.0 * T));
    }
    return 0.0;
}

/* the line's strength for the chosen quantity, or -1 if the threshold leaves it out */
static double line_strength(const xo_opts *o, double nu, double elower, double A, double g_up,
                            const xo_condition *c)
{
    double S = o->quantity == 1 ? xo_emissivity(nu, elower, A, g_up, c)
                                : xo_intensity(nu, elower, A, g_up, c);
    if (o->thr_mode != 0 && S < xo_threshold(nu, c->T, o)) return -1.0;
    return S;
}

/* Eq. (e:alphaD): Doppler HWHM */
double xo_alpha_doppler(double nu, const xo_condition *c)
{
    double m = c->mass_da * XO_DALTON;
    return sqrt(2.0 * XO_KB * c->T * XO_LN2 / m) * nu / XO_C_SI;
}

/* Eq. (e:gamma_L): Lorentz HWHM, with a global scale and exponent shift */
double xo_gamma_lorentz(double gamma_ref, double n_T, const xo_condition *c)
{
    return c->gamma_scale * gamma_ref * pow(c->T_ref / c->T, n_T + c->n_shift) * (c->P / c->P_ref);
}

/* One broadener of a mixture (Sec. "Broadening parameters", "Mixtures of broadeners") */
typedef struct {
    int type;                    /* 0: constant, 1: a0 (by J''), 2: a1 (by J'' and J') */
    double fraction;             /* rho_i */
    double gamma0, n;            /* the constant values, and the default for unlisted lines */
    long long n_entries;
    const int32_t *j_lo, *j_up;  /* table keys (j_up for a1 only) */
    const double *gamma0_j, *n_j;
} xo_broadener;

/* gamma_0 and n_L of broadener b for a line with lower / upper J */
static void broad_lookup(const xo_broadener *b, int jl, int ju, double *g0, double *n)
{
    *g0 = b->gamma0;
    *n = b->n;
    if (b->type == 0) return;
    for (long long i = 0; i < b->n_entries; ++i) {
        if (b->j_lo[i] != jl) continue;
        if (b->type == 2 && b->j_up[i] != ju) continue;
        *g0 = b->gamma0_j[i];
        *n = b->n_j[i];
        return;
    }
}

/* Lorentz HWHM of a line under a mixture: sum_i rho_i gamma_0,i (T_ref/T)^(n_i + n_shift)
 * P/P_ref, times the global gamma_scale (the single-broadener form of Eq. e:gamma_L per term) */
double xo_gamma_mixture(int jl, int ju, const xo_broadener *b, int nb, const xo_condition *c)
{
    double g = 0.0;
    for (int i = 0; i < nb; ++i) {
        double g0, n;
        broad_lookup(&b[i], jl, ju, &g0, &n);
        g += b[i].fraction * g0 * pow(c->T_ref / c->T, n + c->n_shift);
    }
    return c->gamma_scale * g * (c->P / c->P_ref);
}

/* where a line's Lorentz HWHM comes from: its own (gamma_ref, n_T), or a mixture */
typedef struct {
    const float *gamma_ref, *n_T;
    const int16_t *j_lo, *j_up;
    const xo_broadener *b;
    int nb;
} xo_gsrc;

static double line_gamma(const xo_gsrc *g, size_t l, const xo_condition *c)
{
    if (g->nb > 0) return xo_gamma_mixture(g->j_lo[l], g->j_up ? g->j_up[l] : 0, g->b, g->nb, c);
    return xo_gamma_lorentz(g->gamma_ref[l], g->n_T[l], c);
}

/* ---------------------------------------------------------------------- */
/* Humlicek w4: w(z) ~ F(t), t = y - i x, four regions by s = |x| + y      */
/* F'(t) is the exact derivative of the same rational (and exp) forms.     */
/* ---------------------------------------------------------------------- */
static int w4_region(double x, double y)
{
    double s = fabs(x) + y;
    if (s >= 15.0) return 1;
    if (s >= 5.5) return 2;
    if (y >= 0.195 * fabs(x) - 0.176) return 3;
    return 4;
}

/* region III numerator / denominator polynomials in t (Horner form) */
static const double R3P[5] = {16.4955, 20.20933, 11.96482, 3.778987, 0.5642236};
static const double R3Q[6] = {16.4955, 38.82363, 39.27121, 21.69274, 6.699398, 1.0};
/* region IV: w = exp(u) - t*N(u)/D(u), u = t^2; N and D alternate in sign */
static const double R4N[7] = {36183.31, 3321.9905, 1540.787, 219.0313, 35.76683, 1.320522, 0.56419};
static const double R4D[8] = {32066.6, 24322.84, 9022.228, 2186.181, 364.2191, 61.57037, 1.841439, 1.0};

static double complex poly(const double *a, int n, double complex t)
{   /* a[0] + a[1] t + ... + a[n-1] t^(n-1) */
    double complex r = a[n - 1];
    for (int i = n - 2; i >= 0; --i) r = r * t + a[i];
    return r;
}
static double complex dpoly(const double *a, int n, double complex t)
{
    double complex r = (n - 1) * a[n - 1];
    for (int i = n - 2; i >= 1; --i) r = r * t + i * a[i];
    return r;
}
static double complex altpoly(const double *a, int n, double complex u)
{   /* a[0] - u (a[1] - u (a[2] - ...)) = sum_i (-1)^i a[i] u^i */
    double complex r = a[n - 1];
    for (int i = n - 2; i >= 0; --i) r = a[i] - u * r;
    return r;
}
static double complex daltpoly(const double *a, int n, double complex u)
{
    double complex r = 0.0;
    for (int i = n - 1; i >= 1; --i) r = r * u + ((i & 1) ? -1.0 : 1.0) * i * a[i];
    return r;
}

void xo_w4_deriv(double x, double y, double *wre, double *wim, double *dre, double *dim)
{
    double complex t = y - I * x;
    double complex w, d;
    switch (w4_region(x, y)) {
    case 1: {
        double complex den = 0.5 + t * t;
        w = t * 0.5641896 / den;
        d = 0.5641896 * (0.5 - t * t) / (den * den);
        break;
    }
    case 2: {
        double complex u = t * t;
        double complex N = t * (1.410474 + u * 0.5641896);
        double complex Np = 1.410474 + 3.0 * 0.5641896 * u;
        double complex D = 0.75 + u * (3.0 + u);
        double complex Dp = 6.0 * t + 4.0 * t * u;
        w = N / D;
        d = (Np * D - N * Dp) / (D * D);
        break;
    }
    case 3: {
        double complex N = poly(R3P, 5, t), D = poly(R3Q, 6, t);
        w = N / D;
        d = (dpoly(R3P, 5, t) * D - N * dpoly(R3Q, 6, t)) / (D * D);
        break;
    }
    default: {
        double complex u = t * t;
        double complex N = altpoly(R4N, 7, u), D = altpoly(R4D, 8, u);
        double complex Nu = daltpoly(R4N, 7, u), Du = daltpoly(R4D, 8, u);
        double complex e = cexp(u);
        double complex r = N / D;
        double complex ru = (Nu * D - N * Du) / (D * D);
        w = e - t * r;
        d = 2.0 * t * e - (r + t * ru * 2.0 * t);
        break;
    }
    }
    *wre = creal(w); *wim = cimag(w);
    if (dre) *dre = creal(d);
    if (dim) *dim = cimag(d);
}

void xo_w4(double x, double y, double *wre, double *wim)
{
    xo_w4_deriv(x, y, wre, wim, NULL, NULL);
}

/* ---------------------------------------------------------------------- */
/* Gauss-Hermite nodes and weights for weight exp(-x^2)                   */
/* Roots of H_N bracketed by sign changes on a fine mesh, refined by       */
/* bisection; weights are Christoffel numbers 1 / sum_k p_k(x)^2 with the  */
/* orthonormal Hermite polynomials p_k (three-term recurrence).            */
/* ---------------------------------------------------------------------- */
static void orthonormal_hermite(int N, double x, double *pN, double *sumsq)
{
    double pm1 = 0.0, p = pow(XO_PI, -0.25), s = p * p;
    for (int k = 0; k < N; ++k) {
        double pn = x * sqrt(2.0 / (k + 1)) * p - sqrt((double)k / (k + 1)) * pm1;
        pm1 = p; p = pn;
        if (k + 1 < N) s += p * p;
    }
    *pN = p;
    if (sumsq) *sumsq = s;
}

int xo_gauss_hermite(int N, double *x, double *w)
{
    if (N < 1 || N > 200) return -1;
    double L = sqrt(2.0 * N + 1.0) + 1.0;
    int M = 200 * N + 1, found = 0;
    double a = -L, fa; orthonormal_hermite(N, a, &fa, NULL);
    for (int i = 1; i < M && found < N; ++i) {
        double b = -L + 2.0 * L * i / (M - 1), fb;
        orthonormal_hermite(N, b, &fb, NULL);
        if (fa == 0.0) { x[found++] = a; }
        else if (fa * fb < 0.0) {
            double lo = a, hi = b, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), fm;
                if (mid == lo || mid == hi) break;
                orthonormal_hermite(N, mid, &fm, NULL);
                if (flo * fm <= 0.0) hi = mid; else { lo = mid; flo = fm; }
            }
            x[found++] = 0.5 * (lo + hi);
        }
        a = b; fa = fb;
    }
    if (found != N) return -2;
    for (int j = 0; j < N; ++j) {
        double pN, s;
        orthonormal_hermite(N, x[j], &pN, &s);
        w[j] = 1.0 / s;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Line profiles (unit area), D = nu - nu_fi                              */
/* ---------------------------------------------------------------------- */
double xo_gauss(double D, double alpha)        /* Eq. (e:Gauss) */
{
    return sqrt(XO_LN2 / XO_PI) / alpha * exp(-D * D * XO_LN2 / (alpha * alpha));
}

double xo_lorentz(double D, double gamma)      /* Eq. (e:lor) */
{
    return gamma / (XO_PI * (D * D + gamma * gamma));
}

double xo_voigt_w4(double D, double alpha, double gamma)
{
    double sl = sqrt(XO_LN2);
    double wr, wi;
    xo_w4(sl * D / alpha, sl * gamma / alpha, &wr, &wi);
    return sqrt(XO_LN2 / XO_PI) / alpha * wr;
}

double xo_voigt_gh(double D, double alpha, double gamma, int n, const double *xg, const double *wg)
{
    double s = 0.0, sl = sqrt(XO_LN2);
    for (int j = 0; j < n; ++j) {
        double d = D - alpha * xg[j] / sl;
        s += wg[j] * gamma / (d * d + gamma * gamma);
    }
    return s / pow(XO_PI, 1.5);
}

/* bin average over [D - h/2, D + h/2], Eq. (e:sigma:quad) without I */
double xo_voigt_gh_binned(double D, double h, double alpha, double gamma,
                          int n, const double *xg, const double *wg)
{
    double s = 0.0, sl = sqrt(XO_LN2);
    for (int j = 0; j < n; ++j) {
        double yp = (D + 0.5 * h - alpha * xg[j] / sl) / gamma;
        double ym = (D - 0.5 * h - alpha * xg[j] / sl) / gamma;
        s += wg[j] * (atan(yp) - atan(ym));
    }
    return s / (pow(XO_PI, 1.5) * h);
}

/* bin average of the Gaussian over [D - h/2, D + h/2], Eq. (eqn:sig_ij) without I:
 * (erf(x+) - erf(x-)) / (2h), x+- = sqrt(ln2)/alpha (D +- h/2).  When both limits lie
 * on one side of the centre the same difference is taken as erfc(x-) - erfc(x+) (on the
 * mirrored side), which is the identical quantity without the cancellation of two
 * values near 1. */
double xo_gauss_binned(double D, double h, double alpha)
{
    double sl = sqrt(XO_LN2);
    double xp = sl * (D + 0.5 * h) / alpha, xm = sl * (D - 0.5 * h) / alpha;
    double d;
    if (xm >= 0.0) d = erfc(xm) - erfc(xp);
    else if (xp <= 0.0) d = erfc(-xp) - erfc(-xm);
    else d = erf(xp) - erf(xm);
    return d / (2.0 * h);
}

/* bin average of the Lorentzian, Eq. (eqn:sig_lor-2) without I:
 * (atan(y+) - atan(y-)) / (pi h), y+- = (D +- h/2)/gamma */
double xo_lorentz_binned(double D, double h, double gamma)
{
    return (atan((D + 0.5 * h) / gamma) - atan((D - 0.5 * h) / gamma)) / (XO_PI * h);
}

/* profile value and its partial derivatives w.r.t. alpha and gamma */
static double profile_eval(int prof, double D, double h, double alpha, double gamma,
                           int ngh, const double *xg, const double *wg,
                           double *dVda, double *dVdg)
{
    double sl = sqrt(XO_LN2);
    double V, da = 0.0, dg = 0.0;
    switch (prof) {
    case XO_DOPPLER:
        V = xo_gauss(D, alpha);
        da = V * (-1.0 / alpha + 2.0 * XO_LN2 * D * D / (alpha * alpha * alpha));
        break;
    case XO_LORENTZ: {
        double q = D * D + gamma * gamma;
        V = gamma / (XO_PI * q);
        dg = (D * D - gamma * gamma) / (XO_PI * q * q);
        break;
    }
    case XO_VOIGT_W4: {
        double wr, wi, dr, di;
        xo_w4_deriv(sl * D / alpha, sl * gamma / alpha, &wr, &wi, &dr, &di);
        V = sqrt(XO_LN2 / XO_PI) / alpha * wr;
        double dVdD = XO_LN2 / (sqrt(XO_PI) * alpha * alpha) * di;   /* Re(-i F') = Im F' */
        dg = XO_LN2 / (sqrt(XO_PI) * alpha * alpha) * dr;
        da = -(V + D * dVdD + gamma * dg) / alpha;
        break;
    }
    case XO_GH_SAMPLED: {
        double s = 0.0;
        for (int j = 0; j < ngh; ++j) {
            double d = D - alpha * xg[j] / sl, q = d * d + gamma * gamma;
            s += wg[j] * gamma / q;
            dg += wg[j] * (d * d - gamma * gamma) / (q * q);
            da += wg[j] * gamma * 2.0 * d * (xg[j] / sl) / (q * q);
        }
        double k = pow(XO_PI, -1.5);
        V = s * k; dg *= k; da *= k;
        break;
    }
    case XO_DOPPLER_BINNED: {
        /* d/dalpha erf(x) = 2/sqrt(pi) e^{-x^2} (-x/alpha) */
        double xp = sl * (D + 0.5 * h) / alpha, xm = sl * (D - 0.5 * h) / alpha;
        V = xo_gauss_binned(D, h, alpha);
        da = (-xp * exp(-xp * xp) + xm * exp(-xm * xm)) / (sqrt(XO_PI) * alpha * h);
        break;
    }
    case XO_LORENTZ_BINNED: {
        /* d/dgamma atan(s/gamma) = -s/(s^2 + gamma^2) */
        double sp = D + 0.5 * h, sm = D - 0.5 * h;
        V = xo_lorentz_binned(D, h, gamma);
        dg = (-sp / (sp * sp + gamma * gamma) + sm / (sm * sm + gamma * gamma)) / (XO_PI * h);
        break;
    }
    case XO_GH_BINNED:
    default: {
        double s = 0.0;
        for (int j = 0; j < ngh; ++j) {
            double sp = D + 0.5 * h - alpha * xg[j] / sl, sm = D - 0.5 * h - alpha * xg[j] / sl;
            s += wg[j] * (atan(sp / gamma) - atan(sm / gamma));
            dg += wg[j] * (-sp / (sp * sp + gamma * gamma) + sm / (sm * sm + gamma * gamma));
            da += wg[j] * (xg[j] / sl) * (-gamma / (sp * sp + gamma * gamma) + gamma / (sm * sm + gamma * gamma));
        }
        double k = 1.0 / (pow(XO_PI, 1.5) * h);
        V = s * k; dg *= k; da *= k;
        break;
    }
    }
    if (dVda) *dVda = da;
    if (dVdg) *dVdg = dg;
    return V;
}

double xo_profile(int prof, double D, double h, double alpha, double gamma, int ngh,
                  const double *xg, const double *wg, double *dVda, double *dVdg)
{
    return profile_eval(prof, D, h, alpha, gamma, ngh, xg, wg, dVda, dVdg);
}

/* ---------------------------------------------------------------------- */
/* Cross section by sampling (Sec. 3.1): lines outer, grid points inner    */
/* ---------------------------------------------------------------------- */
static double line_cut(const xo_opts *o, double alpha, double gamma)
{
    if (o->width_mult > 0.0) {
        double w = o->width_mult * (alpha > gamma ? alpha : gamma);
        return w < o->cutoff ? w : o->cutoff;
    }
    return o->cutoff;
}

static void neumaier_add(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else *c += (v - t) + *s;
    *s = t;
}

/* first grid index k with nu_A + k*h >= x  (a window start; exact test done per point) */
static long long grid_floor_index(double x, double nu_A, double h)
{
    return (long long)floor((x - nu_A) / h);
}

static int cross_section_impl(const double *nu, const float *elower, const float *A, const xo_gsrc *gsrc,
                              const int16_t *g_up, size_t n_lines, const xo_condition *cond, double nu_A,
                              double h, long long n_pts, const xo_opts *o, double *sigma, int nthreads);

/* Eq. (e:fast-v): the Vectorized Voigt of a line at nu_l, offset D */
double xo_voigt_vv(double D, double alpha, double gamma, double nu_l, double split, int beta_mode)
{
    if (fabs(D) <= split) return xo_voigt_w4(D, alpha, gamma);
    double a_ref = alpha / nu_l;   /* alpha_D is proportional to nu: its value at 1 cm^-1 */
    double beta = beta_mode ? xo_voigt_w4(split, alpha, gamma) / xo_voigt_w4(split, a_ref, gamma) : 1.0;
    return beta * xo_voigt_w4(D, a_ref, gamma);
}

/* the profile value of a line (every profile; VV needs the line position) */
static double line_value(const xo_opts *o, double D, double h, double al, double ga, double nul, int ngh,
                         const double *xg, const double *wg)
{
    if (o->profile == XO_VOIGT_VV) return xo_voigt_vv(D, al, ga, nul, o->vv_split, o->vv_beta);
    return profile_eval(o->profile, D, h, al, ga, ngh, xg, wg, NULL, NULL);
}

/* VVN: Sigma = h sum_k f(nu_k - nu) over the lattice points nu_A + k h within the cut */
static double vv_norm(const xo_opts *o, double nul, double al, double ga, double cut, double nu_A, double h)
{
    long long k0 = (long long)floor((nul - cut - nu_A) / h) - 1;
    long long k1 = (long long)floor((nul + cut - nu_A) / h) + 1;
    double s = 0.0, c = 0.0;
    for (long long k = k0; k <= k1; ++k) {
        double D = (nu_A + (double)k * h) - nul;
        if (fabs(D) > cut) continue;
        neumaier_add(&s, &c, xo_voigt_vv(D, al, ga, nul, o->vv_split, o->vv_beta));
    }
    return (s + c) * h;
}

int xo_cross_section(const double *nu, const float *elower, const float *A, const float *gamma_ref,
                     const float *n_T, const int16_t *g_up, size_t n_lines,
                     const xo_condition *cond, double nu_A, double h, long long n_pts,
                     const xo_opts *o, double *sigma, int nthreads)
{
    xo_gsrc g = {gamma_ref, n_T, NULL, NULL, NULL, 0};
    return cross_section_impl(nu, elower, A, &g, g_up, n_lines, cond, nu_A, h, n_pts, o, sigma, nthreads);
}

/* the same with every line's Lorentz HWHM from a mixture of .broad broadeners */
int xo_cross_section_broad(const double *nu, const float *elower, const float *A, const int16_t *j_lo,
                           const int16_t *j_up, const int16_t *g_up, size_t n_lines, const xo_broadener *b,
                           int nb, const xo_condition *cond, double nu_A, double h, long long n_pts,
                           const xo_opts *o, double *sigma, int nthreads)
{
    xo_gsrc g = {NULL, NULL, j_lo, j_up, b, nb};
    return cross_section_impl(nu, elower, A, &g, g_up, n_lines, cond, nu_A, h, n_pts, o, sigma, nthreads);
}

static int cross_section_impl(const double *nu, const float *elower, const float *A, const xo_gsrc *gsrc,
                              const int16_t *g_up, size_t n_lines, const xo_condition *cond, double nu_A,
                              double h, long long n_pts, const xo_opts *o, double *sigma, int nthreads)
{
    if (n_pts <= 0) return 0;
    double xg[200], wg[200];
    int ngh = 0;
    if (o->profile == XO_GH_BINNED || o->profile == XO_GH_SAMPLED) {
        ngh = o->n_gh;
        if (xo_gauss_hermite(ngh, xg, wg) != 0) return -1;
    }
    if (nthreads < 1) nthreads = 1;
    double *acc = (double *)calloc((size_t)nthreads * 2 * (size_t)n_pts, sizeof(double));
    if (!acc) return -2;

#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static, 1)
#endif
    for (int t = 0; t < nthreads; ++t) {
        double *s = acc + (size_t)t * 2 * (size_t)n_pts, *c = s + n_pts;
        size_t l0 = n_lines * (size_t)t / (size_t)nthreads;
        size_t l1 = n_lines * (size_t)(t + 1) / (size_t)nthreads;
        for (size_t l = l0; l < l1; ++l) {
            double nul = nu[l];
            double Ifi = line_strength(o, nul, elower[l], A[l], g_up[l], cond);
            if (Ifi < 0.0) continue;   /* below the intensity threshold */
            double al = xo_alpha_doppler(nul, cond);
            double ga = line_gamma(gsrc, l, cond);
            double cut = line_cut(o, al, ga);
            if (o->profile == XO_VOIGT_VV && o->vv_norm) {
                double sn = vv_norm(o, nul, al, ga, cut, nu_A, h);
                Ifi = sn > 0.0 ? Ifi / sn : 0.0;
            }
            long long k0 = grid_floor_index(nul - cut, nu_A, h) - 1;
            long long k1 = grid_floor_index(nul + cut, nu_A, h) + 1;
            if (k0 < 0) k0 = 0;
            if (k1 > n_pts - 1) k1 = n_pts - 1;
            for (long long k = k0; k <= k1; ++k) {
                double xk = nu_A + (double)k * h;
                double D = xk - nul;
                if (fabs(D) > cut) continue;
                double v = line_value(o, D, h, al, ga, nul, ngh, xg, wg);
                neumaier_add(&s[k], &c[k], Ifi * v);
            }
        }
    }
    for (long long k = 0; k < n_pts; ++k) {
        double s = 0.0, c = 0.0;
        for (int t = 0; t < nthreads; ++t) {
            double *st = acc + (size_t)t * 2 * (size_t)n_pts;
            neumaier_add(&s, &c, st[k]);
            neumaier_add(&s, &c, st[n_pts + k]);
        }
        sigma[k] = s + c;
    }
    free(acc);
    return 0;
}

/* Cross section at selected grid points k_list[0..m-1] (same definition as
 * xo_cross_section, evaluated one point at a time).  nu must be sorted
 * ascending: the lines within the largest possible cut of x_k are found by
 * binary search, then each is tested against its own cut exactly as above.
 * Sum per point over lines in list order, Neumaier-compensated. */
static size_t first_geq(const double *a, size_t n, double x)
{
    size_t lo = 0, hi = n;
    while (lo < hi) { size_t mid = lo + (hi - lo) / 2; if (a[mid] < x) lo = mid + 1; else hi = mid; }
    return lo;
}

int xo_cross_section_points(const double *nu, const float *elower, const float *A, const float *gamma_ref,
                            const float *n_T, const int16_t *g_up, size_t n_lines,
                            const xo_condition *cond, double nu_A, double h, const long long *k_list,
                            long long m, const xo_opts *o, double *out, int nthreads)
{
    double xg[200], wg[200];
    int ngh = 0;
    if (o->profile == XO_GH_BINNED || o->profile == XO_GH_SAMPLED) {
        ngh = o->n_gh;
        if (xo_gauss_hermite(ngh, xg, wg) != 0) return -1;
    }
    for (size_t l = 1; l < n_lines; ++l)
        if (nu[l] < nu[l - 1]) return -3;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
    for (long long i = 0; i < m; ++i) {
        double xk = nu_A + (double)k_list[i] * h;
        size_t l0 = first_geq(nu, n_lines, xk - o->cutoff * (1.0 + 1e-12) - 1e-9);
        double s = 0.0, c = 0.0;
        for (size_t l = l0; l < n_lines && nu[l] <= xk + o->cutoff * (1.0 + 1e-12) + 1e-9; ++l) {
            double al = xo_alpha_doppler(nu[l], cond);
            double ga = xo_gamma_lorentz(gamma_ref[l], n_T[l], cond);
            double cut = line_cut(o, al, ga);
            double D = xk - nu[l];
            if (fabs(D) > cut) continue;
            double Ifi = line_strength(o, nu[l], elower[l], A[l], g_up[l], cond);
            if (Ifi < 0.0) continue;   /* below the intensity threshold */
            if (o->profile == XO_VOIGT_VV && o->vv_norm) {
                double sn = vv_norm(o, nu[l], al, ga, cut, nu_A, h);
                Ifi = sn > 0.0 ? Ifi / sn : 0.0;
            }
            neumaier_add(&s, &c, Ifi * line_value(o, D, h, al, ga, nu[l], ngh, xg, wg));
        }
        out[i] = s + c;
    }
    return 0;
}

/* number of (line, grid point) pairs inside the cutoff: the algorithmic work (every
 * line counts, whatever an intensity threshold would leave out) */
long long xo_count_evals(const double *nu, const float *gamma_ref, const float *n_T, size_t n_lines,
                         const xo_condition *cond, double nu_A, double h, long long n_pts,
                         const xo_opts *o)
{
    long long cnt = 0;
    for (size_t l = 0; l < n_lines; ++l) {
        double al = xo_alpha_doppler(nu[l], cond);
        double ga = xo_gamma_lorentz(gamma_ref[l], n_T[l], cond);
        double cut = line_cut(o, al, ga);
        long long k0 = grid_floor_index(nu[l] - cut, nu_A, h) - 1;
        long long k1 = grid_floor_index(nu[l] + cut, nu_A, h) + 1;
        if (k0 < 0) k0 = 0;
        if (k1 > n_pts - 1) k1 = n_pts - 1;
        for (long long k = k0; k <= k1; ++k) {
            double D = (nu_A + (double)k * h) - nu[l];
            if (fabs(D) <= cut) ++cnt;
        }
    }
    return cnt;
}

/* ---------------------------------------------------------------------- */
/* Adjoint: given g_k = dL/dsigma_k for each condition, the chain rule     */
/*   dL/dT_c, dL/dP_c                         per condition               */
/*   dL/d(gamma_scale), dL/d(n_shift)         global                      */
/*   dL/d(gamma_ref_l), dL/d(n_l)             per line (summed over c)    */
/* and, with a mixture of broadeners (gamma = sum_i gamma_i, each term of   */
/* the form of Eq. e:gamma_L), per broadener i:                            */
/*   dL/d(scale of all its gamma_0 values, at 1):   dgamma/d = gamma_i      */
/*   dL/d(shift of all its n values, at 0):  dgamma/d = gamma_i ln(T_ref/T) */
/* The cutoff is held fixed (its boundary terms are measure-zero).         */
/* ---------------------------------------------------------------------- */
static int cross_section_vjp_impl(const double *nu, const float *elower, const float *A, const xo_gsrc *gsrc,
                                  const int16_t *g_up, size_t n_lines,
                                  const xo_condition *conds, int n_cond, double nu_A, double h, long long n_pts,
                                  const xo_opts *o, const double *grad_sigma,
                                  double *dT, double *dP, double *d_gscale, double *d_nshift,
                                  double *d_gref_line, double *d_n_line, double *d_g0_broad, double *d_n_broad)
{
    const double c2 = xo_c2();
    double xg[200], wg[200];
    int ngh = 0;
    if (o->quantity != 0 || o->thr_mode != 0 || o->profile == XO_VOIGT_VV) return -4;   /* absorption, no threshold */
    if (o->profile == XO_GH_BINNED || o->profile == XO_GH_SAMPLED) {
        ngh = o->n_gh;
        if (xo_gauss_hermite(ngh, xg, wg) != 0) return -1;
    }
    const int nb = gsrc->nb;
    if (nb > 8) return -1;
    double gs = 0.0, gn = 0.0;
    if (d_gref_line) memset(d_gref_line, 0, n_lines * sizeof(double));
    if (d_n_line) memset(d_n_line, 0, n_lines * sizeof(double));
    if (d_g0_broad) memset(d_g0_broad, 0, (size_t)nb * sizeof(double));
    if (d_n_broad) memset(d_n_broad, 0, (size_t)nb * sizeof(double));
    for (int c = 0; c < n_cond; ++c) {
        const xo_condition *cd = &conds[c];
        const double *g = grad_sigma + (size_t)c * (size_t)n_pts;
        double T = cd->T;
        double sT = 0.0, sP = 0.0;
        for (size_t l = 0; l < n_lines; ++l) {
            double nul = nu[l];
            double Ifi = xo_intensity(nul, elower[l], A[l], g_up[l], cd);
            double al = xo_alpha_doppler(nul, cd);
            /* Lorentz HWHM and dgamma/dT: the line's own (gamma_ref, n_T), or the sum of the
             * mixture's terms gamma_i = s rho_i gamma_0,i (T_ref/T)^(n_i + n_shift) P/P_ref */
            double ga, dgdT, gi[8];
            if (nb > 0) {
                ga = 0.0;
                dgdT = 0.0;
                for (int b = 0; b < nb; ++b) {
                    double g0, nn;
                    broad_lookup(&gsrc->b[b], gsrc->j_lo[l], gsrc->j_up ? gsrc->j_up[l] : 0, &g0, &nn);
                    gi[b] = cd->gamma_scale * gsrc->b[b].fraction * g0 * pow(cd->T_ref / T, nn + cd->n_shift)
                            * (cd->P / cd->P_ref);
                    ga += gi[b];
                    dgdT += -(nn + cd->n_shift) * gi[b] / T;
                }
            } else {
                ga = xo_gamma_lorentz(gsrc->gamma_ref[l], gsrc->n_T[l], cd);
                dgdT = -(gsrc->n_T[l] + cd->n_shift) * ga / T;
            }
            double cut = line_cut(o, al, ga);
            long long k0 = grid_floor_index(nul - cut, nu_A, h) - 1;
            long long k1 = grid_floor_index(nul + cut, nu_A, h) + 1;
            if (k0 < 0) k0 = 0;
            if (k1 > n_pts - 1) k1 = n_pts - 1;
            double SI = 0.0, Sa = 0.0, Sg = 0.0;
            for (long long k = k0; k <= k1; ++k) {
                double D = (nu_A + (double)k * h) - nul;
                if (fabs(D) > cut) continue;
                double dVa, dVg;
                double V = profile_eval(o->profile, D, h, al, ga, ngh, xg, wg, &dVa, &dVg);
                SI += g[k] * V;
                Sa += g[k] * Ifi * dVa;
                Sg += g[k] * Ifi * dVg;
            }
            /* d ln I / dT = c2 E''/T^2 - (c2 nu/T^2)/(exp(c2 nu/T) - 1) - Q'/Q */
            double dlnI = c2 * elower[l] / (T * T) - (c2 * nul / (T * T)) / expm1(c2 * nul / T)
                          - cd->dQdT / cd->Q;
            double dIdT = Ifi * dlnI;
            double dadT = al / (2.0 * T);
            sT += SI * dIdT + Sa * dadT + Sg * dgdT;
            sP += Sg * ga / cd->P;
            gs += Sg * ga / cd->gamma_scale;
            double lnTr = log(cd->T_ref / T);
            gn += Sg * ga * lnTr;
            if (nb > 0) {
                for (int b = 0; b < nb; ++b) {
                    if (d_g0_broad) d_g0_broad[b] += Sg * gi[b];
                    if (d_n_broad) d_n_broad[b] += Sg * gi[b] * lnTr;
                }
            } else {
                if (d_gref_line) d_gref_line[l] += Sg * ga / gsrc->gamma_ref[l];
                if (d_n_line) d_n_line[l] += Sg * ga * lnTr;
            }
        }
        dT[c] = sT;
        dP[c] = sP;
    }
    if (d_gscale) *d_gscale = gs;
    if (d_nshift) *d_nshift = gn;
    return 0;
}

int xo_cross_section_vjp(const double *nu, const float *elower, const float *A, const float *gamma_ref,
                         const float *n_T, const int16_t *g_up, size_t n_lines,
                         const xo_condition *conds, int n_cond, double nu_A, double h, long long n_pts,
                         const xo_opts *o, const double *grad_sigma,
                         double *dT, double *dP, double *d_gscale, double *d_nshift,
                         double *d_gref_line, double *d_n_line)
{
    xo_gsrc g = {gamma_ref, n_T, NULL, NULL, NULL, 0};
    return cross_section_vjp_impl(nu, elower, A, &g, g_up, n_lines, conds, n_cond, nu_A, h, n_pts, o, grad_sigma,
                                  dT, dP, d_gscale, d_nshift, d_gref_line, d_n_line, NULL, NULL);
}

/* the adjoint with every line's Lorentz HWHM from a mixture of .broad broadeners; per
 * broadener, dL/d(scale of its gamma_0 values) and dL/d(shift of its n values) */
int xo_cross_section_vjp_broad(const double *nu, const float *elower, const float *A, const int16_t *j_lo,
                               const int16_t *j_up, const int16_t *g_up, size_t n_lines, const xo_broadener *b,
                               int nb, const xo_condition *conds, int n_cond, double nu_A, double h,
                               long long n_pts, const xo_opts *o, const double *grad_sigma,
                               double *dT, double *dP, double *d_gscale, double *d_nshift,
                               double *d_g0_broad, double *d_n_broad)
{
    if (nb < 1) return -1;
    xo_gsrc g = {NULL, NULL, j_lo, j_up, b, nb};
    return cross_section_vjp_impl(nu, elower, A, &g, g_up, n_lines, conds, n_cond, nu_A, h, n_pts, o, grad_sigma,
                                  dT, dP, d_gscale, d_nshift, NULL, NULL, d_g0_broad, d_n_broad);
}
