// xc_internal.cuh -- internals shared by the libxc translation units.
//
// Physics follows the ExoCross paper (arXiv:1801.09803): Eq. (e:int) intensity,
// Eq. (e:alphaD) Doppler HWHM, Eq. (e:gamma_L) Lorentz HWHM, Eq. (e:pf) Q(T),
// Eqs. (e:Gauss), (e:lor), (e:Voigt) profiles with w(z) from Humlicek's w4,
// Eqs. (e:V-quad), (e:sigma:quad) Gauss-Hermite Voigt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/xc.h"

namespace xc {

// CODATA 2018 exact SI values
constexpr double kPlanck = 6.62607015e-34;     // J s
constexpr double kLightSI = 2.99792458e8;      // m/s
constexpr double kBoltzmann = 1.380649e-23;    // J/K
constexpr double kDalton = 1.66053906660e-27;  // kg
constexpr double kPi = 3.141592653589793238;
constexpr double kLn2 = 0.6931471805599453094;
constexpr double kSqrtLn2 = 0.8325546111576977563;
constexpr double kSqrtPi = 1.772453850905516027;
constexpr double kC2 = kPlanck * (kLightSI * 100.0) / kBoltzmann;  // second radiation constant, cm K
constexpr double kLightCm = kLightSI * 100.0;
constexpr double kPlanckErg = kPlanck * 1e7;                       // erg s

// What a line contributes (absorption or emission) and the intensity threshold
struct StrengthSel {
    int quantity = XC_ABSORPTION, threshold = XC_THRESHOLD_NONE;
    double I_cut = 0.0, nu_crit = 0.0, I_crit = 0.0;
};
inline StrengthSel strength_sel(const xc_opts &o) {
    StrengthSel s;
    s.quantity = o.quantity;
    s.threshold = o.threshold;
    s.I_cut = o.I_cut;
    s.nu_crit = o.nu_crit;
    s.I_crit = o.I_crit;
    return s;
}

// Stage slots of the timing table (see xc_last_timings)
enum Stage { ST_SORT = 0, ST_GATHER, ST_Q, ST_PARAMS, ST_RANGES, ST_PROFILE, ST_VJP, ST_FINISH, ST_COUNT };

struct LinesDev {
    const double *nu;
    const float *elower, *A, *gamma_ref, *n_T;
    const int16_t *g_up, *j_lo;
    // intensity-threshold decisions of the FP32 kernels: bit c of word l * keep_words + c / 32
    // set when line l is kept for condition c (in the order the launch's CParam rows name);
    // nullptr: every line is kept
    const uint32_t *keep = nullptr;
    int keep_words = 0;
    // broadener mixture (xc_set_broadening): per broadener i and line l, rho_i gamma_0,i at
    // bgam[i * bstride + l] and n_L,i at bn[i * bstride + l]; n_broad = 0: the line's own
    // gamma_ref and n_T
    const double *bgam = nullptr, *bn = nullptr;
    size_t bstride = 0;
    int n_broad = 0;
    // FP32 kernels under a mixture: the Lorentz HWHM (cm^-1) of line l for condition row c
    // at gamma_lc[l * gamma_stride + c], computed in FP64
    const float *gamma_lc = nullptr;
    int gamma_stride = 0;
    // FP32 kernels with VVN: intensity factor of line l, condition row c at vv_scale[l * nc + c]
    const float *vv_scale = nullptr;
    int vv_stride = 0;
};

struct CondDev {  // mirrors xc_condition plus resolved Q
    double T, P, Q, dQdT, mass_da, T_ref, P_ref, gamma_scale, n_shift, abundance;
};

__host__ __device__ inline int64_t i64min(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ inline int64_t i64max(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Per-line physics in FP64
// ---------------------------------------------------------------------------
__host__ __device__ inline double alpha_coef(double T, double mass_da) {
    // alpha_D / nu = sqrt(2 k T ln2 / m) / c   (Eq. e:alphaD)
    return sqrt(2.0 * kBoltzmann * T * kLn2 / (mass_da * kDalton)) / kLightSI;
}

// Line strength in FP64: the absorption intensity of Eq. (e:int), or with XC_EMISSION the
// emissivity of Eq. (e:emiss) (upper state E' = E'' + nu) times the photon energy h c nu;
// -1 when the intensity threshold leaves the line out.  pref_abs = abundance / (8 pi c Q).
__device__ inline double line_strength64(double nu, double elower, double gA, const CondDev &c,
                                         const StrengthSel &s) {
    const double inv_T = 1.0 / c.T;
    double S;
    if (s.quantity == XC_EMISSION) {
        S = c.abundance * gA * (kPlanckErg * kLightCm * nu) / (4.0 * kPi) * exp(-kC2 * (elower + nu) * inv_T) / c.Q;
    } else {
        const double boltz = exp(-kC2 * elower * inv_T);
        const double stim = -expm1(-kC2 * nu * inv_T);
        S = c.abundance / (8.0 * kPi * kLightCm * c.Q) * gA / (nu * nu) * boltz * stim;
    }
    if (s.threshold != XC_THRESHOLD_NONE) {
        double thr = s.I_cut;
        if (s.threshold == XC_THRESHOLD_HITRAN)
            thr = nu > s.nu_crit ? s.I_crit : s.I_crit * (nu / s.nu_crit) * tanh(kC2 * nu * inv_T * 0.5);
        if (S < thr) return -1.0;
    }
    return S;
}

// Lorentz HWHM of line l under the broadener mixture (Sec. "Mixtures of broadeners"):
// gamma_scale P/P_ref sum_i rho_i gamma_0,i (T_ref/T)^(n_i + n_shift), each term Eq. (e:gamma_L)
__device__ inline double mixture_gamma64(const LinesDev &L, size_t l, const CondDev &c) {
    const double lnTr = log(c.T_ref / c.T);
    double g = 0.0;
    for (int i = 0; i < L.n_broad; ++i)
        g += L.bgam[(size_t)i * L.bstride + l] * exp((L.bn[(size_t)i * L.bstride + l] + c.n_shift) * lnTr);
    return c.gamma_scale * g * (c.P / c.P_ref);
}

// grid point nu_k = nu_A + k * step, rounded exactly as two separate operations
__device__ inline double grid_x(double nu_A, double step, int64_t k) {
    return __dadd_rn(nu_A, __dmul_rn((double)k, step));
}

// Inclusive k-range of grid points with |x_k - nu| <= cut, using the same
// rounding as grid_x; empty range gives ka > kb.
// inv_step = 1 / step, computed once by the caller: the first estimates only need to be
// close (the loops below settle them on the exact predicate), and an FP64 division per
// call costs more than the rest of the function on a GPU with a low FP64 rate
__device__ inline void line_k_range(double nu, double cut, double nu_A, double step, double inv_step, int64_t n,
                                    int64_t *ka_out, int64_t *kb_out) {
    double fa = ceil((nu - cut - nu_A) * inv_step);
    double fb = floor((nu + cut - nu_A) * inv_step);
    fa = fmax(fa, -1.0);
    fb = fmin(fb, (double)n);
    int64_t ka, kb;
    if (fa > (double)n || fb < -1.0) { *ka_out = 1; *kb_out = 0; return; }
    ka = (int64_t)fa;
    kb = (int64_t)fb;
    // adjust to the exact predicate (monotone in k)
    while (ka > 0 && __dsub_rn(grid_x(nu_A, step, ka - 1), nu) >= -cut) --ka;
    while (ka <= kb && __dsub_rn(grid_x(nu_A, step, ka), nu) < -cut) ++ka;
    while (kb < n - 1 && __dsub_rn(grid_x(nu_A, step, kb + 1), nu) <= cut) ++kb;
    while (kb >= ka && __dsub_rn(grid_x(nu_A, step, kb), nu) > cut) --kb;
    if (ka < 0) ka = 0;
    if (kb > n - 1) kb = n - 1;
    *ka_out = ka;
    *kb_out = kb;
}

// ---------------------------------------------------------------------------
// Small complex type (FP64 and FP32)
// ---------------------------------------------------------------------------
template <typename R>
struct Cx {
    R re, im;
};
template <typename R>
__device__ inline Cx<R> cx(R a, R b) { return Cx<R>{a, b}; }
template <typename R>
__device__ inline Cx<R> operator+(Cx<R> a, Cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ inline Cx<R> operator-(Cx<R> a, Cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__device__ inline Cx<R> operator*(Cx<R> a, Cx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ inline Cx<R> operator*(R s, Cx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__device__ inline Cx<R> operator+(R s, Cx<R> a) { return {s + a.re, a.im}; }
// reciprocal: IEEE in FP64; the hardware approximation (about 1 ulp) in FP32
__device__ inline double recip(double x) { return 1.0 / x; }
__device__ inline float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <typename R>
__device__ inline Cx<R> cdiv(Cx<R> a, Cx<R> b) {
    R d = recip(b.re * b.re + b.im * b.im);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}

// ---------------------------------------------------------------------------
// Humlicek w4 (JQSRT 27, 1982, 437): w(x+iy) ~ F(t), t = y - ix, by region of
// s = |x| + y.  Region I: s >= 15; II: s >= 5.5; III: y >= 0.195|x| - 0.176;
// IV otherwise.  F'(t) is the exact derivative of the same forms, used by the
// adjoint (dF/dx = -i F', dF/dy = F').
// ---------------------------------------------------------------------------
__device__ inline void sincos_(double a, double *s, double *c) { sincos(a, s, c); }
__device__ inline void sincos_(float a, float *s, float *c) { sincosf(a, s, c); }

template <typename R>
__device__ inline int w4_region(R ax, R y) {
    R s = ax + y;
    if (s >= R(15)) return 1;
    if (s >= R(5.5)) return 2;
    if (y >= R(0.195) * ax - R(0.176)) return 3;
    return 4;
}

template <typename R>
__device__ inline Cx<R> w4_eval(R x, R y, Cx<R> *dF) {
    Cx<R> t = cx<R>(y, -x);
    R ax = x < R(0) ? -x : x;
    switch (w4_region<R>(ax, y)) {
    case 1: {
        Cx<R> t2 = t * t;
        Cx<R> den = R(0.5) + t2;
        Cx<R> w = cdiv(R(0.5641896) * t, den);
        if (dF) *dF = cdiv(R(0.5641896) * cx<R>(R(0.5) - t2.re, -t2.im), den * den);
        return w;
    }
    case 2: {
        Cx<R> u = t * t;
        Cx<R> N = t * (R(1.410474) + R(0.5641896) * u);
        Cx<R> D = R(0.75) + u * (R(3) + u);
        Cx<R> w = cdiv(N, D);
        if (dF) {
            Cx<R> Np = R(1.410474) + R(3.0 * 0.5641896) * u;
            Cx<R> Dp = t * (R(6) + R(4) * u);
            *dF = cdiv(Np * D - N * Dp, D * D);
        }
        return w;
    }
    case 3: {
        Cx<R> N = R(16.4955) + t * (R(20.20933) + t * (R(11.96482) + t * (R(3.778987) + R(0.5642236) * t)));
        Cx<R> D = R(16.4955) + t * (R(38.82363) + t * (R(39.27121) + t * (R(21.69274) + t * (R(6.699398) + t))));
        Cx<R> w = cdiv(N, D);
        if (dF) {
            Cx<R> Np = R(20.20933) + t * (R(2 * 11.96482) + t * (R(3 * 3.778987) + R(4 * 0.5642236) * t));
            Cx<R> Dp = R(38.82363) + t * (R(2 * 39.27121) + t * (R(3 * 21.69274) + t * (R(4 * 6.699398) + R(5) * t)));
            *dF = cdiv(Np * D - N * Dp, D * D);
        }
        return w;
    }
    default: {
        Cx<R> u = t * t;
        Cx<R> m = cx<R>(-u.re, -u.im);  // -u: the alternating Horner form in u becomes plain Horner in -u
        Cx<R> N = R(36183.31) + m * (R(3321.9905) + m * (R(1540.787) + m * (R(219.0313) +
                   m * (R(35.76683) + m * (R(1.320522) + R(0.56419) * m)))));
        Cx<R> D = R(32066.6) + m * (R(24322.84) + m * (R(9022.228) + m * (R(2186.181) +
                   m * (R(364.2191) + m * (R(61.57037) + m * (R(1.841439) + m))))));
        R eu = exp(u.re);
        R sn, cs;
        sincos_(u.im, &sn, &cs);
        Cx<R> e = cx<R>(eu * cs, eu * sn);
        Cx<R> r = cdiv(N, D);
        Cx<R> w = e - t * r;
        if (dF) {
            // dN/du = -dN/dm, with N as a polynomial in m = -u
            Cx<R> Nm = R(3321.9905) + m * (R(2 * 1540.787) + m * (R(3 * 219.0313) + m * (R(4 * 35.76683) +
                        m * (R(5 * 1.320522) + R(6 * 0.56419) * m))));
            Cx<R> Dm = R(24322.84) + m * (R(2 * 9022.228) + m * (R(3 * 2186.181) + m * (R(4 * 364.2191) +
                        m * (R(5 * 61.57037) + m * (R(6 * 1.841439) + R(7) * m)))));
            Cx<R> ru = cdiv(Dm * N - Nm * D, D * D);  // dr/du = -(Nm D - N Dm)/D^2
            Cx<R> tt2 = R(2) * (t * t);
            *dF = R(2) * (t * e) - (r + tt2 * ru);
        }
        return w;
    }
    }
}

// unit-area Voigt by w4: sqrt(ln2/pi)/alpha Re w(x + iy), x = sqrt(ln2) D/alpha, y = sqrt(ln2) gamma/alpha
__device__ inline double voigt64(double D, double al, double ga) {
    double ia = kSqrtLn2 / al;
    Cx<double> w = w4_eval<double>(D * ia, ga * ia, nullptr);
    return 0.46971863934982566 / al * w.re;
}

// Eq. (e:fast-v): the Voigt within split of the centre, beyond it the Voigt of a line at 1 cm^-1
// (Doppler HWHM alpha / nu) times beta (Eq. e:beta, or 1)
__device__ inline double voigt_vv64(double D, double al, double ga, double nul, double split, int beta) {
    if (fabs(D) <= split) return voigt64(D, al, ga);
    const double ar = al / nul;
    const double b = beta ? voigt64(split, al, ga) / voigt64(split, ar, ga) : 1.0;
    return b * voigt64(D, ar, ga);
}



// ---------------------------------------------------------------------------
// Host-side helpers
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);

// Reads one byte of every page of a host buffer (host code; a no-op below 1 MB).  On a
// CPU-GPU coherent system (Grace + Blackwell) a copy-engine transfer from or to host pages
// that no CPU core has touched for a few seconds runs about 15x slower (measured on the
// GB300 machine: 2.8 GB in 205-250 ms instead of 13 ms); one read per page first (about 1 ms
// for 2.8 GB with 64 KB pages) restores the full rate.
void warm_host_pages(const void *p, size_t bytes);

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t need) {
        if (need <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, need ? need : 16);
        if (e == cudaSuccess) bytes = need;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// kernel launchers implemented in the other translation units
cudaError_t launch_partition_function(const double *E, const int32_t *g, size_t n, const double *T, int nT,
                                      double *Q, double *dQ, cudaStream_t s);
cudaError_t launch_sort_lines(const LinesDev &in, size_t n, bool assume_sorted, DevBuf *tmp, double *nu,
                              float *elower, float *A, float *gref, float *nT, int16_t *g, int16_t *j,
                              uint32_t *perm, int *d_flag, cudaStream_t s, cudaEvent_t *ev, int64_t *launches,
                              bool *bad_input, bool *unsorted);
cudaError_t launch_line_params64(const LinesDev &L, size_t n, const CondDev *cond_dev, int cut_mode,
                                 double cutoff, double width_mult, double *I, double *alpha, double *gamma,
                                 double *cut, cudaStream_t s, const StrengthSel &sel = StrengthSel());
// per-line mixture parameters from broadener tables (keys sorted on the host): for broadener
// i, type[i] 0 constant, 1 a0 (key J''), 2 a1 (key J'' * 65536 + J'); rows [row0[i], row0[i+1])
cudaError_t launch_apply_broadening(const int16_t *j_lo, const int16_t *j_up, size_t n, int nb, const int *type,
                                    const double *frac, const double *g0_def, const double *n_def,
                                    const int *row0, const int64_t *keys, const double *g0, const double *nl,
                                    double *bgam, double *bn, cudaStream_t s);
// out[i] = in[perm[i]]: a per-line int16 field given in input order -> sorted order
cudaError_t launch_permute_i16(const int16_t *in, const uint32_t *perm, size_t n, int16_t *out, cudaStream_t s);
// FP32 kernels under a mixture: gamma_lc[l * nc + c] and the per-condition maximum (float bits)
cudaError_t launch_line_gamma(const LinesDev &L, size_t n, const CondDev *conds, int nc, float *gamma_lc,
                              unsigned *gmax_bits, cudaStream_t s);
// per (line, condition) threshold decisions for the FP32 kernels (see LinesDev::keep)
cudaError_t launch_line_keep(const LinesDev &L, size_t n, const CondDev *conds, int nc, const StrengthSel &sel,
                             uint32_t *keep, int words, cudaStream_t s);
cudaError_t launch_window_ranges(const double *nu, size_t n, double nu_A, double step, int64_t n_pts,
                                 int64_t W, double cutmax, int64_t n_win, int64_t *lo, int64_t *hi,
                                 cudaStream_t s);
cudaError_t launch_count_evals(const LinesDev &L, size_t n, const CondDev *conds_dev, int n_cond,
                               double nu_A, double step, int64_t n_pts, double cutoff, double width_mult,
                               unsigned long long *count, cudaStream_t s);
cudaError_t launch_gather_f64(int profile, const double *nu, const double *I, const double *alpha,
                              const double *gamma, const double *cut, const int64_t *win_lo,
                              const int64_t *win_hi, int64_t n_win, double nu_A, double step, int64_t n_pts,
                              const double *ghx, const double *ghw, int ngh, double *sigma, cudaStream_t s,
                              double vv_split = 4.0, int vv_beta = 0);
// VVN: I[l] /= h sum_k f_VV(nu_k - nu_l) over the line's cut window on the grid lattice
cudaError_t launch_vv_norm64(const double *nu, double *I, const double *alpha, const double *gamma,
                             const double *cut, size_t n, double nu_A, double step, double vv_split, int vv_beta,
                             cudaStream_t s);
// VVN for the FP32 kernels: scale[l * nc + c] = 1 / (h sum_k f_VV) of line l, condition c
cudaError_t launch_vv_norm32(const LinesDev &L, size_t n, const CondDev *conds, int nc, double nu_A, double step,
                             double cutoff, double width_mult, double vv_split, int vv_beta, float *scale,
                             cudaStream_t s);
cudaError_t launch_gh_nodes(int n, double *x, double *w, cudaStream_t s);

}  // namespace xc
