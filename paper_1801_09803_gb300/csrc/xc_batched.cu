// xc_batched.cu -- FP32 gather-form profile kernel over many (T, P) conditions.
//
// Work unit ("tile") = (window of W consecutive grid points, group of CG
// conditions).  A persistent grid pulls tiles from an atomic work counter in
// descending order of cost (lines in range x conditions; ranked on the device).
// For its window a CTA walks the lines whose cut can reach the window (binary
// search on the sorted wavenumbers), staging SCH lines at a time in shared
// memory together with their per-condition constants, which are computed while
// staging (the fused intensity / half-width step: Eq. e:int, e:alphaD, e:gamma_L).
//
// Thread layout: warp w owns the 32*R consecutive points [w*32R, (w+1)*32R) of
// the window, lane j the points j + 32 r; every thread keeps R x CG FP32
// accumulators in registers.  Offsets from line centre to grid point are
// formed exactly: delta = (k - n_l) - f_l with n_l the integer and f_l the
// fractional grid position of the line computed in FP64.
//
// Voigt (w4): Humlicek's region I (|x| + y >= 15), written in grid units as
//     V = P (u + C) / (u (u + E) + F),   u = delta^2,
// covers all but a few points next to each line centre.  Two lines that cover
// the whole warp span with no region II-IV point are summed over one shared
// reciprocal:  q1/D1 + q2/D2 = (q1 D2 + q2 D1) / (D1 D2).  Lines that straddle
// the span edge of their cut, or whose centre zone (region II-IV for some
// condition) reaches the span, take a masked single-line path that evaluates
// region I there; the centre zones are left to the centre-zone kernel.
//
// Accumulation: FP32 in registers over FOLD_CHUNKS chunks of lines, then folded
// into the FP64 output, which each thread owns exclusively (no atomics, fixed
// order: bitwise reproducible).  Intensities are carried in FP32 multiplied by
// a per-condition power of two that keeps the strongest possible line near
// 1e10 (bound from max g A / nu^2 and max g A / nu over the list).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "xc_batched.cuh"
#include "xc_tcgen05.cuh"

namespace xc {

constexpr int GT = 256;          // threads per CTA
constexpr int SCH = 64;          // lines per staged chunk
constexpr int FOLD_CHUNKS = 8;   // FP32 -> FP64 fold period, in chunks (512 lines)
constexpr float kPiM32 = 0.17958712212516656f;          // pi^(-3/2)
constexpr float kFarU3 = 1.f / 0.003f;                   // 3-term far-wing series from u >= C / 0.003
constexpr float kFarU4 = 1.f / 0.012f;                   // 4-term far-wing series from u >= C / 0.012

struct GatherParams {
    LinesDev L;
    const int *n_abs;          // per line: integer grid position (clamped)
    const float *f_frac;       // per line: fractional grid position
    const int *ka_abs, *kb_abs;// per line: inclusive grid-index range inside the cut
    const CParam *cp;          // per condition
    const unsigned *win_lo, *win_hi;
    const int *tile_order;
    int *counter;
    int n_tiles, n_groups, n_cond;
    int W;
    int64_t n_pts;
    float h, inv_h;
    int max_lines_per_tile;    // autotune probe: stop early (0 = all)
    const float *ghx, *ghw;    // Gauss-Hermite nodes (float), device
    int ngh;
    int tc_far;                // Voigt w4: the far-wing kernel has written the (line, condition,
                               // 128-point block) pairs with span_far; evaluate the rest, add
    double *sigma;
};

// Two FP32 values in one 64-bit register pair, for the packed f32x2 arithmetic of
// sm_100-class GPUs: one instruction issue performs two FP32 adds / multiplies /
// FMAs (the FMA pipe throughput is unchanged; the issue slots are halved).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float lo2(f32x2 v) { float a, b; upk2(v, a, b); return a; }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f32x2 rcp2(f32x2 a) {
    float x, y;
    upk2(a, x, y);
    return pk2(rcp_approx(x), rcp_approx(y));
}
// ---------------------------------------------------------------------------
// per-condition constants
// ---------------------------------------------------------------------------
// width of a condition's profiles at a representative line (nu = 5000 cm^-1, n = 0.6):
// C = alpha^2 / (2 ln 2) + gamma^2, the scale of the far-wing radius
__device__ double cond_width_key(const CondDev &d) {
    const double al = alpha_coef(d.T, d.mass_da) * 5000.0;
    const double ga = d.gamma_scale * (d.P / d.P_ref) * pow(d.T_ref / d.T, 0.6 + d.n_shift);
    return al * al * (0.5 / 0.6931471805599453) + ga * ga;
}

// Per-condition constants, stored in order of increasing profile width (stable), so that
// the conditions sharing a tile have similar far-wing radii; row keeps the caller's index.
__global__ void k_cparams(const CondDev *conds, int n_cond, const GeomStats *gs, CParam *cp, double step,
                          int quantity, const unsigned *gmax_bits, float vv_split, int vv_beta) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cond) return;
    const CondDev d = conds[c];
    const double key = cond_width_key(d);
    int rank = 0;
    for (int j = 0; j < n_cond; ++j) {
        const double kj = cond_width_key(conds[j]);
        rank += (kj < key) || (kj == key && j < c);
    }
    const double log2e = 1.4426950408889634;
    double kT = kC2 * log2e / d.T;
    float hi = (float)kT;
    float lo = (float)(kT - (double)hi);
    const bool emis = quantity == XC_EMISSION;
    double pref = emis ? d.abundance * kPlanckErg * kLightCm / (4.0 * kPi * d.Q)
                       : d.abundance / (8.0 * kPi * kLightCm * d.Q);
    double s1 = (double)__uint_as_float(gs->gA_nu2_bits);
    double s2 = (double)__uint_as_float(gs->gA_nu_bits);
    const double numax = (double)__uint_as_float(gs->nu_bits);
    // bound on the largest intensity (absorption), or emissivity: g A nu <= max(g A / nu) nu_max^2
    double ib = emis ? pref * s2 * numax * numax : pref * fmin(s1, kC2 / d.T * s2);
    int e2 = 0;
    if (ib > 0.0 && isfinite(ib)) {
        e2 = (int)floor(log2(1e10 / ib));
        e2 = max(-120, min(120, e2));
    }
    double scale = ldexp(1.0, e2);
    CParam p;
    p.inv_scale = ldexp(1.0, -e2);
    p.kT_hi = hi;
    p.kT_lo = lo;
    p.c2T = (float)(kC2 / d.T);
    p.pref = (float)(pref * scale);
    p.acoef = (float)alpha_coef(d.T, d.mass_da);
    p.log2Tr = (float)log2(d.T_ref / d.T);
    p.pscale = (float)(d.gamma_scale * d.P / d.P_ref);
    p.nshift = (float)d.n_shift;
    p.row = c;
    p.emis = emis ? 1.f : 0.f;
    p.vv_split = vv_split;
    p.vv_beta = vv_beta;
    {
        // D4 <= ceil(sqrt(max(C k4, t2))) + 1 grows with both widths; t2 <= (15 a_h / sqrt ln2)^2.
        // Upper bounds of the widths from the line statistics (|n| <= nT_max), with margin.
        const double num = (double)__uint_as_float(gs->nu_bits);
        const double grm = (double)__uint_as_float(gs->gref_bits);
        const double ntm = (double)__uint_as_float(gs->nT_bits);
        const double lr = log(d.T_ref / d.T);
        const double tf = fmax(exp((ntm + d.n_shift) * lr), exp((-ntm + d.n_shift) * lr));
        const double ah = alpha_coef(d.T, d.mass_da) * num / step;
        // under a broadener mixture the largest width of this condition over all lines
        const double gh = gmax_bits ? (double)__uint_as_float(gmax_bits[c]) / step
                                    : fabs(d.gamma_scale * d.P / d.P_ref) * grm * tf / step;
        const double C = ah * ah * (0.5 / 0.6931471805599453) + gh * gh;
        const double t2 = 225.0 * ah * ah / 0.6931471805599453;
        const double uf = fmax(C * (1.0 / 0.012), t2);
        const double db = ceil(sqrt(uf) * 1.001) + 3.0;
        p.dbound = (isfinite(db) && db < 1e9) ? (float)db : 1e9f;
    }
    cp[rank] = p;
}

// (window, condition-group) tile -> line range for the CUDA-core kernel when the
// tensor-core kernel takes the far wings: only lines within the group's largest far
// radius of the window (or within the cut, if that is smaller) have work there
__global__ void k_win_ranges_near(const double *__restrict__ nu, int64_t n, double nu_A, double step,
                                  int64_t n_pts, int W, double cutoff, int n_win, int n_groups, int CG,
                                  const CParam *cp, int n_cond, unsigned *lo, unsigned *hi) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_win * n_groups) return;
    const int w = t / n_groups, g = t % n_groups;
    float db = 0.f;
    for (int c = g * CG; c < min(n_cond, (g + 1) * CG); ++c) db = fmaxf(db, cp[c].dbound);
    const double cutmax = fmin(cutoff, ((double)db + 2.0) * step);
    // the nominal window, also past the last grid point: both kernels test far-ness on
    // whole nominal 128-point blocks, so a line within its radius of a block's nominal
    // end but farther from the last grid point is left out by the far-wing kernel and
    // must be staged here (its far wing still reaches the grid)
    int64_t k0 = (int64_t)w * W;
    int64_t k1 = k0 + W - 1;
    (void)n_pts;
    double x0 = grid_x(nu_A, step, k0), x1 = grid_x(nu_A, step, k1);
    double margin = cutmax * (1.0 + 1e-12) + 1e-12 * (fabs(x0) + fabs(x1)) + 1e-300;
    int64_t a = 0, b = n;
    double x = x0 - margin;
    while (a < b) { int64_t m = a + ((b - a) >> 1); if (nu[m] < x) a = m + 1; else b = m; }
    lo[t] = (unsigned)a;
    int64_t a2 = a, b2 = n;
    x = x1 + margin;
    while (a2 < b2) { int64_t m = a2 + ((b2 - a2) >> 1); if (nu[m] <= x) a2 = m + 1; else b2 = m; }
    hi[t] = (unsigned)a2;
}

// ---------------------------------------------------------------------------
// per-line grid geometry (and the intensity bound statistics)
// cond >= 0: per-line cut min(cutoff, width_mult * max(alpha, gamma)) of that condition
// ---------------------------------------------------------------------------
__global__ void k_line_geom(LinesDev L, size_t n, double nu_A, double step, int64_t n_pts, double cutoff,
                            double width_mult, const CondDev *cond, int *n_abs, float *f_frac, int *ka_abs,
                            int *kb_abs, GeomStats *gs, float4 *tc_geo, float4 *tc_phys) {
    const double inv_h = 1.0 / step;
    float m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f, m5 = 0.f;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        double nu = L.nu[l];
        m3 = fmaxf(m3, __double2float_ru(fabs(nu)));
        m4 = fmaxf(m4, fabsf(L.gamma_ref[l]));
        m5 = fmaxf(m5, fabsf(L.n_T[l]));
        double cut = cutoff;
        if (width_mult > 0.0 && cond) {
            const CondDev c = *cond;
            double al = alpha_coef(c.T, c.mass_da) * nu;
            double ga = L.n_broad > 0 ? mixture_gamma64(L, l, c)
                                      : c.gamma_scale * (double)L.gamma_ref[l] *
                                            exp(((double)L.n_T[l] + c.n_shift) * log(c.T_ref / c.T)) * (c.P / c.P_ref);
            cut = fmin(width_mult * fmax(al, ga), cutoff);
        }
        double d = (nu - nu_A) * inv_h;
        double fl = floor(d);
        double flc = fmin(fmax(fl, -1073741824.0), 1073741824.0);
        n_abs[l] = (int)flc;
        f_frac[l] = (float)(d - fl);
        int64_t ka, kb;
        line_k_range(nu, cut, nu_A, step, inv_h, n_pts, &ka, &kb);
        if (kb < ka) { ka = 1; kb = 0; }
        ka_abs[l] = (int)i64min(i64max(ka, -1), (int64_t)0x7fffffff);
        kb_abs[l] = (int)i64min(i64max(kb, -1), (int64_t)0x7fffffff);
        float gA = (float)L.g_up[l] * L.A[l];
        float nuf = (float)nu;
        m1 = fmaxf(m1, gA / (nuf * nuf));
        m2 = fmaxf(m2, gA / nuf);
        if (tc_geo) {
            // the far-wing kernel's line records: position, cut range (exact integers
            // as floats) and the condition-independent physics
            tc_geo[l] = make_float4((float)n_abs[l], f_frac[l], (float)ka_abs[l], (float)kb_abs[l]);
            tc_phys[l] = make_float4(nuf, L.elower[l], gA / (nuf * nuf), L.gamma_ref[l]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
        m3 = fmaxf(m3, __shfl_xor_sync(0xffffffffu, m3, o));
        m4 = fmaxf(m4, __shfl_xor_sync(0xffffffffu, m4, o));
        m5 = fmaxf(m5, __shfl_xor_sync(0xffffffffu, m5, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (isfinite(m1)) atomicMax(&gs->gA_nu2_bits, __float_as_uint(m1));
        if (isfinite(m2)) atomicMax(&gs->gA_nu_bits, __float_as_uint(m2));
        atomicMax(&gs->nu_bits, __float_as_uint(m3));   // non-negative floats: integer order
        atomicMax(&gs->gref_bits, __float_as_uint(m4));
        atomicMax(&gs->nT_bits, __float_as_uint(m5));
    }
}

cudaError_t launch_fp32_setup(const LinesDev &L, size_t n, const CondDev *conds, int nc, const xc_grid &grid,
                              double cutoff, int *n_abs, float *f, int *ka, int *kb, GeomStats *gs, CParam *cp,
                              cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gs, 0, sizeof(GeomStats), s);
    if (e != cudaSuccess) return e;
    if (n) {
        const unsigned gb = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16));
        k_line_geom<<<gb, 256, 0, s>>>(L, n, grid.nu_A, grid.step, grid.n, cutoff, 0.0, nullptr, n_abs, f, ka, kb,
                                       gs, nullptr, nullptr);
    }
    if (nc) k_cparams<<<(nc + 63) / 64, 64, 0, s>>>(conds, nc, gs, cp, grid.step, XC_ABSORPTION, nullptr, 4.f, 0);
    return cudaGetLastError();
}

// window -> line range for a fixed maximum cut
__global__ void k_win_ranges32(const double *__restrict__ nu, int64_t n, double nu_A, double step, int64_t n_pts,
                               int W, double cutmax, int n_win, unsigned *lo, unsigned *hi) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_win) return;
    int64_t k0 = (int64_t)w * W;
    int64_t k1 = i64min(k0 + W, n_pts) - 1;
    double x0 = grid_x(nu_A, step, k0), x1 = grid_x(nu_A, step, k1);
    double margin = cutmax * (1.0 + 1e-12) + 1e-12 * (fabs(x0) + fabs(x1)) + 1e-300;
    int64_t a = 0, b = n;
    double t = x0 - margin;
    while (a < b) { int64_t m = a + ((b - a) >> 1); if (nu[m] < t) a = m + 1; else b = m; }
    lo[w] = (unsigned)a;
    int64_t a2 = a, b2 = n;
    t = x1 + margin;
    while (a2 < b2) { int64_t m = a2 + ((b2 - a2) >> 1); if (nu[m] <= t) a2 = m + 1; else b2 = m; }
    hi[w] = (unsigned)a2;
}

// rank tiles by decreasing cost (ties by index): order[rank] = tile
__global__ void k_rank_tiles(const unsigned *lo, const unsigned *hi, int n_win, int n_groups, int n_tiles,
                             int *order, bool do_rank, bool per_tile) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    if (!do_rank) {  // very many tiles: keep index order
        order[t] = t;
        return;
    }
    const int rt = per_tile ? t : t / n_groups;
    unsigned ct = hi[rt] - lo[rt];
    int rank = 0;
    for (int u = 0; u < n_tiles; ++u) {
        const int ru = per_tile ? u : u / n_groups;
        unsigned cu = hi[ru] - lo[ru];
        rank += (cu > ct) || (cu == ct && u < t);
    }
    order[rank] = t;
}

__global__ void k_nodes_to_float(const double *x, const double *w, int n, float *xf, float *wf) {
    int j = threadIdx.x;
    if (j < n) {
        xf[j] = (float)x[j];
        wf[j] = (float)w[j];
    }
}

// ---------------------------------------------------------------------------
// per-(line, condition) constants, by profile
//   W4 : A = {E', F', P', P'C'}   B = {a, y, Pv, thr^2}   (grid units)
//   VV : A = reference wing {E', F', P', P'C'} (or {a, -1, P, y} where it is not region I
//        throughout)   B = {a, y, Pv, exact-zone half-width}
//   LOR: A = {G', P', 0, 0}
//   DOP: A = {qd, Pd, 0, 0}
//   GHS: A = {sh, G', P, 0}
//   GHB: A = {sh, g', G' - 1/4, P}
// ---------------------------------------------------------------------------
// Voigt w4 zones of a (line, condition) from its widths in grid steps: x = a |delta|,
// y, the region-I threshold u >= t2 (t2 < 0: region I everywhere) and the far radius D.
// Explicitly rounded operations: every kernel that splits work by these gets the same bits.
//   Far wing: the region-I rational P (u + C)/(u^2 + E u + F) equals its series
//   P r (1 + c1 r + c2 r^2 + ...) in r = 1/u, c1 = C - E = 3b - g^2, c2 = E^2 - C E - F =
//   (g^2 - 5b)^2 - 20 b^2.  u^2 + E u + F has its two roots on |u| = C, so |c_n| <=
//   (2n + 1) C^n and the terms dropped beyond r^2 stay below 7 x^3 / (1 - 9x/7), x = C r:
//   at u >= C / 0.003 that is < 2e-7 of the value, below FP32 rounding of the rational;
//   with four terms (c3 = -E c2 - F c1) the bound is 9 x^4 / (1 - 11x/9) < 2e-7 from
//   u >= C / 0.012.
//   D3, D4: integer radii (grid steps) beyond which every point is in the 3- or 4-term
//   far zone and in region I; a block [t0, t1] with n - D > t1 or n + D < t0 (n =
//   integer part of the line position) qualifies.
struct W4Zone {
    float a, y, t2, D3, D4;
};
__device__ __forceinline__ W4Zone w4_zone(float ah, float gh) {
    W4Zone z;
    const float rah = rcp_approx(ah);
    z.a = __fmul_rn(kSqrtLn2f, rah);
    z.y = __fmul_rn(z.a, gh);
    const float thr = __fmul_rn(__fmul_rn(__fsub_rn(15.f, z.y), ah), 1.f / kSqrtLn2f);
    z.t2 = z.y < 15.f ? __fmul_rn(thr, thr) : -1.f;
    const float Crn = __fadd_rn(__fmul_rn(__fmul_rn(ah, ah), (float)(0.5 / 0.6931471805599453)), __fmul_rn(gh, gh));
    // any D >= sqrt(uf) is valid: approximate square root (one MUFU op), scaled up by
    // more than its error bound
    float sq3, sq4;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq3) : "f"(fmaxf(__fmul_rn(Crn, kFarU3), z.t2)));
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(sq4) : "f"(fmaxf(__fmul_rn(Crn, kFarU4), z.t2)));
    z.D3 = ceilf(__fmul_rn(sq3, 1.000001f)) + 1.f;
    z.D4 = ceilf(__fmul_rn(sq4, 1.000001f)) + 1.f;
    return z;
}

// S = (p0, p1, p2, D) of the 3-term far-wing series; D = D4 (the tensor-core kernel's
// radius) when that kernel takes the far wings (d4), else D3
__device__ __noinline__ float w4_value_f32(float delta, const float4 &B);

// EXT: the options that change a line's constants per (line, condition) -- emission,
// intensity thresholds, broadener mixtures, VVN -- are honoured; without them (EXT = false)
// the Voigt-w4 hot kernels carry none of their checks
template <int PROF, bool EXT = true>
__device__ __forceinline__ void line_consts(const LinesDev &L, size_t l, const CParam &c, float h, float inv_h,
                                            float4 *A, float4 *B, float *thr2, float4 *S, bool d4 = false) {
    const float nu = (float)L.nu[l];
    const float E = L.elower[l];
    // Boltzmann factor exp(-c2 E/T) = 2^-(E c2 log2e / T), product kept to ~1 ulp
    float z = fmaf(E, c.kT_hi, E * c.kT_lo);
    float boltz = exp2_neg(z);
    float I;
    if (EXT && c.emis != 0.f) {
        // Eq. (e:emiss) times h c nu: the upper state's Boltzmann factor as exp(-c2 E''/T)
        // exp(-c2 nu/T), each to ~1 ulp
        I = c.pref * ((float)L.g_up[l] * L.A[l]) * nu * boltz * exp2_neg(fmaf(nu, c.kT_hi, nu * c.kT_lo));
    } else {
        float stim = -expm1f(-c.c2T * nu);
        I = c.pref * ((float)L.g_up[l] * L.A[l]) * rcp_approx(nu * nu) * boltz * stim;
    }
    // left out by the intensity threshold for this condition (decided in FP64)
    if (EXT && L.keep && !((L.keep[l * (size_t)L.keep_words + (c.row >> 5)] >> (c.row & 31)) & 1u)) I = 0.f;
    // VVN: this (line, condition)'s area normalisation (computed in FP64)
    if (EXT && L.vv_scale) I *= L.vv_scale[l * (size_t)L.vv_stride + c.row];
    float al = c.acoef * nu;                                                   // Eq. e:alphaD
    float ah, gh;                                                              // widths in grid steps
    if (EXT && L.gamma_lc) {
        // broadener mixture: the width of this (line, condition), computed in FP64
        ah = __fmul_rn(c.acoef * nu, inv_h);
        gh = __fmul_rn(L.gamma_lc[l * (size_t)L.gamma_stride + c.row], inv_h);
    } else {
        line_widths(nu, L.gamma_ref[l], L.n_T[l], c, inv_h, &ah, &gh);
    }
    *thr2 = -1.f;
    *S = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
    if (PROF == XC_VOIGT_W4) {
        float b = ah * ah * (float)(0.5 / 0.6931471805599453);
        float g2 = gh * gh;
        float C = b + g2;
        float P = I * kKappa * gh * inv_h;
        *A = make_float4(2.f * (g2 - b), C * C, P, P * C);
        // a, y and the region-I threshold decide which kernel evaluates a point (the
        // main kernel: |x| + y >= 15; the centre-zone kernel: the rest); the far radius
        // which points the tensor-core kernel takes (see w4_zone)
        const W4Zone z = w4_zone(ah, gh);
        float Pv = I * kSqrtLn2OverPi * rcp_approx(al);
        *B = make_float4(z.a, z.y, Pv, z.t2);
        *thr2 = z.t2;
        float e5 = g2 - 5.f * b;
        *S = make_float4(P, P * (3.f * b - g2), P * fmaf(e5, e5, -20.f * b * b), d4 ? z.D4 : z.D3);
    } else if (PROF == XC_LORENTZ) {
        *A = make_float4(fmaxf(gh * gh, 1e-30f), I * gh * inv_h * (float)(1.0 / 3.141592653589793), 0.f, 0.f);
    } else if (PROF == XC_DOPPLER) {
        float qd = rcp_approx(ah * ah);
        *A = make_float4(qd, I * kSqrtLn2OverPi * rcp_approx(al), 0.f, 0.f);
    } else if (PROF == XC_VOIGT_GH_SAMPLED) {
        *A = make_float4(ah / kSqrtLn2f, fmaxf(gh * gh, 1e-30f), I * kPiM32 * gh * inv_h, 0.f);
    } else if (PROF == XC_VOIGT_VV) {
        // B: the line's own w4 Voigt (a, y, Pv) and the exact zone's half-width in grid steps;
        // A: the reference wing -- the Voigt of a line at 1 cm^-1, Doppler HWHM alpha / nu:
        // a_ref = a nu, y_ref = a_ref g, amplitude Pv nu, times beta (Eq. e:beta) when asked
        const float a = kSqrtLn2f * rcp_approx(ah), y = a * gh;
        const float Pv = I * kSqrtLn2OverPi * rcp_approx(al);
        const float ar = a * nu, yr = ar * gh;
        const float sp = c.vv_split * inv_h;
        float Pw = Pv * nu;
        if (c.vv_beta) {
            const float rw = w4_value_f32(sp, make_float4(ar, yr, 1.f, 0.f));
            Pw = rw > 0.f ? w4_value_f32(sp, make_float4(a, y, Pv, 0.f)) / rw : 0.f;
        }
        if (ar * (sp + gh) >= 15.f) {
            // beyond the exact zone the reference Voigt is in w4's region I everywhere
            // (x_ref + y_ref > a_ref (sp + g) >= 15): its rational in u = delta^2, as the
            // Voigt w4 constants A (with b_ref = 1 / (2 a_ref^2), C = b_ref + g^2).
            // a_ref = sqrt(ln 2) h / (alpha / nu) does not depend on nu (thousands for common
            // steps), so only a split and a Lorentz width both far below a grid step fail it
            const float br = 0.5f * rcp_approx(ar * ar), g2 = gh * gh, Cr = br + g2;
            const float Pr = Pw * 0.5641896f * gh * rcp_approx(ar);
            *A = make_float4(2.f * (g2 - br), Cr * Cr, Pr, Pr * Cr);
        } else {
            *A = make_float4(ar, -1.f, Pw, yr);   // flagged by A.y < 0: the complex w4 where needed
        }
        *B = make_float4(a, y, Pv, sp);
    } else if (PROF == XC_DOPPLER_BINNED) {
        // Eq. (eqn:sig_ij) in grid steps: x+- = (sqrt(ln2)/ah) (delta +- 1/2), I/(2h)
        *A = make_float4(kSqrtLn2f * rcp_approx(ah), 0.5f * I * inv_h, 0.f, 0.f);
    } else if (PROF == XC_LORENTZ_BINNED) {
        // Eq. (eqn:sig_lor-2) in grid steps: y+- = (delta +- 1/2)/gh, I/(pi h)
        *A = make_float4(gh, gh * gh - 0.25f, I * inv_h * (float)(1.0 / 3.141592653589793), 0.f);
    } else {
        *A = make_float4(ah / kSqrtLn2f, gh, gh * gh - 0.25f, I * kPiM32 * inv_h);
    }
}

// Re w in w4's region II (5.5 <= |x| + y < 15) in real arithmetic.  The region-II
// rational t(a + b t^2)/(t^4 + 3 t^2 + 3/4) has denominator (t^2 + Q1)(t^2 + Q2) with
// Q1,2 = (3 -+ sqrt 6)/2, so it splits into two partial fractions A_m t/(t^2 + Q_m),
// A_m = (a - b Q_m)/(Q_other - Q_m); each is a pair of Lorentzians in x at +-sqrt(Q_m):
//   Re w = y sum_m A_m (X + Y + Q_m) / ((X + Y - Q_m)^2 + 4 Q_m Y),  X = x^2, Y = y^2.
// (The nodes +-sqrt(Q_m) are those of 4-point Gauss-Hermite quadrature.)
__device__ __forceinline__ float w4_region2_re(float x, float y) {
    constexpr double a = 1.410474, b = 0.5641896, s6 = 2.449489742783178098;
    constexpr float Q1 = (float)((3.0 - s6) / 2.0), Q2 = (float)((3.0 + s6) / 2.0);
    constexpr float A1 = (float)((a - b * ((3.0 - s6) / 2.0)) / s6);
    constexpr float A2 = (float)(-(a - b * ((3.0 + s6) / 2.0)) / s6);
    float X = x * x, Y = y * y;
    float t1 = X + Y - Q1, t2 = X + Y - Q2;
    float D1 = fmaf(t1, t1, 4.f * Q1 * Y), D2 = fmaf(t2, t2, 4.f * Q2 * Y);
    float N1 = A1 * (X + Y + Q1), N2 = A2 * (X + Y + Q2);
    return y * fmaf(N1, D2, N2 * D1) * rcp_approx(D1 * D2);
}

// full FP32 w4 Voigt value (all regions) times Pv, at grid offset delta
// (kept out of line: only the few points with |x| + y < 5.5 reach it, and inlining
// its four regions into every unrolled (point, condition) slot bloats the kernel)
__device__ __noinline__ float w4_value_f32(float delta, const float4 &B) {
    float x = B.x * fabsf(delta);
    Cx<float> w = w4_eval<float>(x, B.y, nullptr);
    return B.z * w.re;
}

// Re w in w4's region I from (x, y): 0.5641896 y (0.5 + X + Y) / ((X + Y - 0.5)^2 + 2Y)
__device__ __forceinline__ float w4_region1_re(float x, float y) {
    float X = x * x, Y = y * y;
    float t = X + Y - 0.5f;
    return 0.5641896f * y * (0.5f + X + Y) * rcp_approx(fmaf(t, t, 2.f * Y));
}

template <int PROF>
__device__ __forceinline__ float contrib_single(float u, float delta, const float4 &A, const float4 &B,
                                                const float *s_x, const float *s_w, int ngh) {
    if (PROF == XC_VOIGT_W4) {
        // region I only; points with |x| + y < 15 belong to the centre-zone kernel
        float D = fmaf(u, u + A.x, A.y);
        float q = fmaf(A.z, u, A.w);
        return u >= B.w ? q * rcp_approx(D) : 0.f;
    } else if (PROF == XC_LORENTZ) {
        return A.y * rcp_approx(u + A.x);
    } else if (PROF == XC_DOPPLER) {
        return A.y * ex2_approx(-A.x * u);
    } else if (PROF == XC_VOIGT_GH_SAMPLED) {
        float s = 0.f;
        for (int j = 0; j < ngh; ++j) {
            float e = fmaf(-A.x, s_x[j], delta);
            s = fmaf(s_w[j], rcp_approx(fmaf(e, e, A.y)), s);
        }
        return A.z * s;
    } else if (PROF == XC_VOIGT_VV) {
        // Eq. (e:fast-v): the line's own Voigt in the exact zone, the reference wing beyond it.
        // Both are w4 Voigts.  The reference wing (most of the points) is region I throughout
        // for almost every line: its rational in u with the line's constants, as Voigt w4's
        // main kernel evaluates it; in the exact zone w4 is its region-I rational in real
        // form where |x| + y >= 15 and the full w4 only for the few points nearer the centre
        const float ad = fabsf(delta);
        if (ad > B.w) {
            if (A.y >= 0.f) return fmaf(A.z, u, A.w) * rcp_approx(fmaf(u, u + A.x, A.y));
            const float x = A.x * ad;
            return x + A.w >= 15.f ? A.z * w4_region1_re(x, A.w) : w4_value_f32(delta, make_float4(A.x, A.w, A.z, 0.f));
        }
        const float x = B.x * ad;
        return x + B.y >= 15.f ? B.z * w4_region1_re(x, B.y) : w4_value_f32(delta, make_float4(B.x, B.y, B.z, 0.f));
    } else if (PROF == XC_DOPPLER_BINNED) {
        // erf(x+) - erf(x-) on the side |delta| of the (symmetric) profile, as
        // erfc(x-) - erfc(x+): no difference of two numbers near 1 in the wings
        const float t = fabsf(delta);
        return A.y * (erfcf(A.x * (t - 0.5f)) - erfcf(A.x * (t + 0.5f)));
    } else if (PROF == XC_LORENTZ_BINNED) {
        // atan(y+) - atan(y-) = atan2(y+ - y-, 1 + y+ y-), both arguments scaled by gh^2 > 0
        return A.z * atan2_ypos(A.x, u + A.y);
    } else {
        float s = 0.f;
        for (int j = 0; j < ngh; ++j) {
            float e = fmaf(-A.x, s_x[j], delta);
            s = fmaf(s_w[j], atan2_ypos(A.y, fmaf(e, e, A.z)), s);
        }
        return A.w * s;
    }
}

// FP32 register partials -> FP64 output (each thread owns its points)
template <int R, int CG>
__device__ __forceinline__ void fold_acc(f32x2 (&acc)[R / 2][CG], const int (&ji)[R], int64_t kw, int grp,
                                         const GatherParams &p, const double *sScale, const int *sRow, bool first) {
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
#pragma unroll
        for (int c = 0; c < CG; ++c) {
            float v2[2];
            upk2(acc[q][c], v2[0], v2[1]);
            int cc = grp * CG + c;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int64_t k = kw + ji[2 * q + h];
                if (k < p.n_pts && cc < p.n_cond) {
                    double *dst = p.sigma + (size_t)sRow[c] * (size_t)p.n_pts + (size_t)k;
                    double v = (double)v2[h] * sScale[c];
                    if (first) *dst = v; else *dst += v;
                }
            }
            acc[q][c] = 0ull;
        }
    }
}

// per-(line, condition) constants in shared memory: Voigt w4 and Lorentz keep them
// duplicated in packed pairs ((E,E),(F,F),(P,P),(PC,PC) / (G,G),(P,P)) for the f32x2 path
template <int PROF>
struct ConstLayout {
    // Voigt w4: 48 B = packed (E,E),(F,F),(P,P),(PC,PC) for the rational, then
    // {p0, p1, p2, u_far} of the far-wing series
    static constexpr size_t kBytes = (PROF == XC_VOIGT_W4) ? 48 : 16;
};

template <int PROF>
__device__ __forceinline__ void store_consts(unsigned char *base, int idx, const float4 &A, const float4 &S) {
    if (PROF == XC_VOIGT_W4) {
        ulonglong2 *q = reinterpret_cast<ulonglong2 *>(base + (size_t)48 * idx);
        q[0] = make_ulonglong2(pk2(A.x, A.x), pk2(A.y, A.y));
        q[1] = make_ulonglong2(pk2(A.z, A.z), pk2(A.w, A.w));
        reinterpret_cast<float4 *>(q)[2] = S;
    } else if (PROF == XC_LORENTZ) {
        reinterpret_cast<ulonglong2 *>(base)[idx] = make_ulonglong2(pk2(A.x, A.x), pk2(A.y, A.y));
    } else {
        reinterpret_cast<float4 *>(base)[idx] = A;
    }
}

template <int PROF>
__device__ __forceinline__ float4 load_consts(const unsigned char *base, int idx) {
    if (PROF == XC_VOIGT_W4) {
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(base + (size_t)48 * idx);
        ulonglong2 a = q[0], b = q[1];
        return make_float4(lo2(a.x), lo2(a.y), lo2(b.x), lo2(b.y));
    } else if (PROF == XC_LORENTZ) {
        ulonglong2 a = reinterpret_cast<const ulonglong2 *>(base)[idx];
        return make_float4(lo2(a.x), lo2(a.y), 0.f, 0.f);
    } else {
        return reinterpret_cast<const float4 *>(base)[idx];
    }
}

template <int PROF, int R, int CG>
struct SmemLayout {
    static constexpr bool kHasB = (PROF == XC_VOIGT_W4 || PROF == XC_VOIGT_VV);
    static constexpr size_t kA = (size_t)SCH * CG * ConstLayout<PROF>::kBytes;
    static constexpr size_t kB = kHasB ? (size_t)SCH * CG * sizeof(float4) : 0;
    static constexpr size_t kMetaI = (size_t)SCH * sizeof(int4);
    static constexpr size_t kMetaF = (size_t)SCH * sizeof(float2);
    static constexpr size_t kScale = (size_t)CG * sizeof(double);
    static constexpr size_t kNodes = 2 * 64 * sizeof(float);
    static constexpr size_t total = kA + kB + kMetaI + kMetaF + kScale + kNodes + 16;
};

// the far radius D of (line, condition) idx among the staged Voigt w4 constants
__device__ __forceinline__ float sfar_radius(const unsigned char *smem, int idx) {
    return reinterpret_cast<const float4 *>(smem + (size_t)48 * idx)[2].w;
}

// every point of [t0, t1] lies beyond the far radius D of a line at integer position n
// (all integers well below 2^24, so the float comparisons are exact; D = inf: never)
__device__ __forceinline__ bool span_far(int n, float D, int t0, int t1) {
    return (float)(n - t1) > D || (float)(t0 - n) > D;
}

// far-wing series of two lines (constants e1, e2) at R points, condition c:
//   acc += r1 (p0 + r1 (p1 + r1 p2)) + r2 (...), two points per packed operation
template <int R, int CG>
__device__ __forceinline__ void w4_series_pair(f32x2 (&acc)[R / 2][CG], int c, const unsigned char *e1,
                                               const unsigned char *e2, const f32x2 (&ra)[R / 2],
                                               const f32x2 (&rb)[R / 2]) {
    const float4 s1 = reinterpret_cast<const float4 *>(e1)[2];
    const float4 s2 = reinterpret_cast<const float4 *>(e2)[2];
    const f32x2 p01 = pk2(s1.x, s1.x), p11 = pk2(s1.y, s1.y), p21 = pk2(s1.z, s1.z);
    const f32x2 p02 = pk2(s2.x, s2.x), p12 = pk2(s2.y, s2.y), p22 = pk2(s2.z, s2.z);
#pragma unroll
    for (int q = 0; q < R / 2; ++q) {
        f32x2 t1 = fma2(fma2(p21, ra[q], p11), ra[q], p01);
        f32x2 t2 = fma2(fma2(p22, rb[q], p12), rb[q], p02);
        acc[q][c] = fma2(t2, rb[q], fma2(t1, ra[q], acc[q][c]));
    }
}

// TCN: compiled for the near pairs of the tensor-core sweep only (p.tc_far set): the code
// of the other modes is left out, which frees registers for more resident warps
// CTAs per SM the register allocation is held to: more resident warps hide the latency of
// these kernels' dependent chains, as long as the allocation does not spill in the point
// loops (ptxas: the near-pair kernel 84 bytes at 4; the one-condition Voigt w4 shape 6 bytes
// at 3; the other Voigt w4 shapes and Lorentz at 8 conditions hundreds of bytes at 3, so
// they keep 2)
template <int PROF, int CG, bool TCN>
constexpr int gather_min_ctas() {
    return TCN ? (CG >= 16 ? 2 : 4)
               : (CG >= 16 ? 1 : ((PROF == XC_VOIGT_W4 ? CG == 1 : CG <= 4) ? 3 : 2));
}

template <int PROF, int R, int CG, bool EXT = true, bool TCN = false>
__global__ void __launch_bounds__(GT, (gather_min_ctas<PROF, CG, TCN>())) k_gather_f32(GatherParams p) {
    constexpr unsigned kAllConds = CG >= 32 ? 0xffffffffu : ((1u << CG) - 1u);
    using Lay = SmemLayout<PROF, R, CG>;
    extern __shared__ __align__(16) unsigned char smem[];
    // per-(line, condition) constants start at smem (see store_consts / load_consts)
    float4 *sB = reinterpret_cast<float4 *>(smem + Lay::kA);
    int4 *sMi = reinterpret_cast<int4 *>(smem + Lay::kA + Lay::kB);
    float2 *sMf = reinterpret_cast<float2 *>(smem + Lay::kA + Lay::kB + Lay::kMetaI);
    double *sScale = reinterpret_cast<double *>(smem + Lay::kA + Lay::kB + Lay::kMetaI + Lay::kMetaF);
    float *sX = reinterpret_cast<float *>(smem + Lay::kA + Lay::kB + Lay::kMetaI + Lay::kMetaF + Lay::kScale);
    float *sW = sX + 64;
    __shared__ int s_tile;
    __shared__ int sRow[CG];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = p.W;
    const int span0 = warp * 32 * R, span1 = span0 + 32 * R - 1;
    if (PROF == XC_VOIGT_GH_BINNED || PROF == XC_VOIGT_GH_SAMPLED) {
        if (tid < p.ngh) {
            sX[tid] = p.ghx[tid];
            sW[tid] = p.ghw[tid];
        }
    }
    float jf[R];
    int ji[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ji[r] = span0 + r * 32 + lane;
        jf[r] = (float)ji[r];
    }
    f32x2 jf2[R / 2];
#pragma unroll
    for (int q = 0; q < R / 2; ++q) jf2[q] = pk2(jf[2 * q], jf[2 * q + 1]);

    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(p.counter, 1);
        __syncthreads();
        const int t = s_tile;
        if (t >= p.n_tiles) break;
        const int tile = p.tile_order[t];
        const int win = tile / p.n_groups, grp = tile % p.n_groups;
        const int64_t kw = (int64_t)win * W;
        const unsigned lo = p.win_lo[p.tc_far ? tile : win];   // near mode: a range per tile
        const unsigned hi = p.win_hi[p.tc_far ? tile : win];
        if (tid < CG) {
            int c = grp * CG + tid;
            sScale[tid] = c < p.n_cond ? p.cp[c].inv_scale : 0.0;
            sRow[tid] = c < p.n_cond ? p.cp[c].row : 0;
        }
        __syncthreads();
        f32x2 acc[R / 2][CG];
#pragma unroll
        for (int q = 0; q < R / 2; ++q)
#pragma unroll
            for (int c = 0; c < CG; ++c) acc[q][c] = 0ull;
        bool first_fold = true;
        int chunk = 0;

        // Chunk ci holds lines lo + ci + j * nch (j < SCH): every chunk samples the whole
        // wavenumber range of the window, so the centre-zone (w4 region II-IV) work of a
        // chunk falls on all warps instead of on the one warp that owns those centres.
        const unsigned nl = hi - lo;
        const unsigned nch = (nl + SCH - 1) / SCH;
        // autotune probe: the first chunks only; each samples the whole line range, so
        // the probe sees the same mix of line positions as the full tile
        const unsigned nch_run = p.max_lines_per_tile > 0 ? min(nch, (unsigned)(p.max_lines_per_tile / SCH)) : nch;
        for (unsigned ci = 0; ci < nch_run; ++ci) {
            const int cnt = (int)((nl - ci + nch - 1) / nch);
            __syncthreads();
            // ---- stage: per-line geometry and per-(line, condition) constants
            if (tid < cnt) {
                size_t l = (size_t)lo + ci + (size_t)tid * nch;
                int na = p.n_abs[l];
                int ka = p.ka_abs[l], kb = p.kb_abs[l];
                int64_t kaw = (int64_t)ka - kw, kbw = (int64_t)kb - kw;
                if (kb < ka) { kaw = 1; kbw = 0; }
                kaw = i64max(-1, i64min(kaw, W));
                kbw = i64max(-1, i64min(kbw, W));
                // .w (largest far radius) is written by another thread in the loop below,
                // before the next barrier: leave it alone here
                sMi[tid].x = (int)((int64_t)na - kw);
                sMi[tid].y = (int)kaw;
                sMi[tid].z = (int)kbw;
                sMf[tid].x = p.f_frac[l];
            }
#pragma unroll 1
            for (int pb = 0; pb < SCH * CG; pb += GT) {
                int q = pb + tid;
                int i = q / CG, c = q % CG;
                int cc = grp * CG + c;
                bool v = (i < cnt);
                float t2 = -1.f;
                if (v) {
                    float4 A, B = make_float4(0.f, 0.f, 0.f, -1.f);
                    float4 S = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
                    if (cc < p.n_cond) {
                        line_consts<PROF, EXT>(p.L, (size_t)lo + ci + (size_t)i * nch, p.cp[cc], p.h, p.inv_h, &A, &B,
                                          &t2, &S, TCN || p.tc_far != 0);
                    } else {  // padding condition: contributes exactly 0
                        if (PROF == XC_VOIGT_W4 || PROF == XC_VOIGT_VV) A = make_float4(1.f, 1.f, 0.f, 0.f);   // 0 / (u^2 + u + 1)
                        else if (PROF == XC_VOIGT_GH_SAMPLED) A = make_float4(0.f, 1.f, 0.f, 0.f);
                        else if (PROF == XC_VOIGT_GH_BINNED) A = make_float4(0.f, 1.f, 1.f, 0.f);
                        else A = make_float4(1.f, 0.f, 0.f, 0.f);
                    }
                    store_consts<PROF>(smem, i * CG + c, A, S);
                    if (Lay::kHasB) sB[i * CG + c] = B;
                }
                // the largest far radius over the group's real conditions (Voigt w4)
                float dm = (PROF == XC_VOIGT_W4 && v && cc < p.n_cond) ? sfar_radius(smem, i * CG + c) : -1.f;
                if (CG > 1) {
#pragma unroll
                    for (int o = CG / 2; o > 0; o >>= 1) {
                        t2 = fmaxf(t2, __shfl_xor_sync(0xffffffffu, t2, o));
                        dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
                    }
                }
                if (v && c == 0) {
                    sMf[i].y = t2;
                    sMi[i].w = (int)fminf(dm, 1.0e9f);
                }
            }
            __syncthreads();

            // ---- evaluate: classify lines for this warp's span, then accumulate
            for (int ib = 0; ib < cnt; ib += 32) {
                int i = ib + lane;
                if (PROF == XC_VOIGT_W4 && (TCN || p.tc_far)) {
                    // The far-wing kernel took every (line, condition) with span_far on this
                    // 128-point span; the rest here, region I only: pairs of lines that cover
                    // the span with no centre-zone point (packed, shared reciprocal), the
                    // others as masked single lines.  Per condition, a line that is far
                    // drops out of the pair (its numerator constants are zero).
                    bool fq = false, sq = false;
                    if (i < cnt) {
                        const int4 mi = sMi[i];
                        const float2 mf = sMf[i];
                        const bool none = (mi.z < span0) || (mi.y > span1) || (mi.y > mi.z);
                        const bool nr = !none && !span_far(mi.x, (float)mi.w, span0, span1);
                        const bool full = (mi.y <= span0) && (mi.z >= span1);
                        bool core = false;
                        if (mf.y > 0.f) {
                            const float cpos = (float)mi.x + mf.x;
                            const float thr = sqrtf(mf.y) + 1.f;
                            core = (cpos + thr >= (float)span0) && (cpos - thr <= (float)span1);
                        }
                        fq = nr && full && !core;
                        sq = nr && !fq;
                    }
                    unsigned fm = __ballot_sync(0xffffffffu, fq);
                    unsigned nm = __ballot_sync(0xffffffffu, sq);
                    if (__popc(fm) & 1) {  // odd count: the last fast line joins the single lines
                        const unsigned top = 1u << (31 - __clz(fm));
                        fm &= ~top;
                        nm |= top;
                    }
                    while (fm) {
                        const int i1 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int i2 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int4 m1 = sMi[i1], m2 = sMi[i2];
                        const float f1 = sMf[i1].x, n1 = (float)m1.x, f2 = sMf[i2].x, n2 = (float)m2.x;
                        const f32x2 nn1 = pk2(n1, n1), ff1 = pk2(f1, f1), nn2 = pk2(n2, n2), ff2 = pk2(f2, f2);
                        f32x2 ua[R / 2], ub[R / 2];
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) {
                            f32x2 da = sub2(sub2(jf2[q], nn1), ff1), db = sub2(sub2(jf2[q], nn2), ff2);
                            ua[q] = mul2(da, da);
                            ub[q] = mul2(db, db);
                        }
                        bool g1 = false, g2 = false;
                        if (lane < CG) {
                            g1 = span_far(m1.x, sfar_radius(smem, i1 * CG + lane), span0, span1);
                            g2 = span_far(m2.x, sfar_radius(smem, i2 * CG + lane), span0, span1);
                        }
                        const unsigned t1 = __ballot_sync(0xffffffffu, g1), t2 = __ballot_sync(0xffffffffu, g2);
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const bool x1 = (t1 >> c) & 1u, x2 = (t2 >> c) & 1u;
                            if (x1 && x2) continue;
                            const ulonglong2 *e1 = reinterpret_cast<const ulonglong2 *>(smem + (size_t)48 * (i1 * CG + c));
                            const ulonglong2 *e2 = reinterpret_cast<const ulonglong2 *>(smem + (size_t)48 * (i2 * CG + c));
                            const ulonglong2 a0 = e1[0], b0 = e2[0];
                            // a line that is far for c contributes nothing here: numerator 0
                            const ulonglong2 a1 = x1 ? make_ulonglong2(0ull, 0ull) : e1[1];
                            const ulonglong2 b1 = x2 ? make_ulonglong2(0ull, 0ull) : e2[1];
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                f32x2 D1 = fma2(ua[q], add2(ua[q], a0.x), a0.y);
                                f32x2 D2 = fma2(ub[q], add2(ub[q], b0.x), b0.y);
                                f32x2 q1 = fma2(a1.x, ua[q], a1.y);
                                f32x2 q2 = fma2(b1.x, ub[q], b1.y);
                                f32x2 num = fma2(q1, D2, mul2(q2, D1));
                                acc[q][c] = fma2(num, rcp2(mul2(D1, D2)), acc[q][c]);
                            }
                        }
                    }
                    while (nm) {
                        const int i1 = ib + __ffs(nm) - 1;
                        nm &= nm - 1;
                        const int4 m1 = sMi[i1];
                        const float f1 = sMf[i1].x, n1 = (float)m1.x;
                        float d1[R], u1[R];
                        bool in1[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            d1[r] = (jf[r] - n1) - f1;
                            u1[r] = d1[r] * d1[r];
                            in1[r] = (ji[r] >= m1.y) && (ji[r] <= m1.z);
                        }
                        bool fl = false;
                        if (lane < CG) fl = span_far(m1.x, sfar_radius(smem, i1 * CG + lane), span0, span1);
                        const unsigned tcm = __ballot_sync(0xffffffffu, fl);
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            if ((tcm >> c) & 1u) continue;
                            const float4 A1 = load_consts<PROF>(smem, i1 * CG + c);
                            const float4 B1 = sB[i1 * CG + c];
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                float a0, a1;
                                upk2(acc[q][c], a0, a1);
                                if (in1[2 * q]) a0 += contrib_single<PROF>(u1[2 * q], d1[2 * q], A1, B1, sX, sW, p.ngh);
                                if (in1[2 * q + 1])
                                    a1 += contrib_single<PROF>(u1[2 * q + 1], d1[2 * q + 1], A1, B1, sX, sW, p.ngh);
                                acc[q][c] = pk2(a0, a1);
                            }
                        }
                    }
                    continue;
                }
                bool fast = false, slow = false;
                if (i < cnt) {
                    int4 mi = sMi[i];
                    float2 mf = sMf[i];
                    bool none = (mi.z < span0) || (mi.y > span1) || (mi.y > mi.z);
                    bool full = (mi.y <= span0) && (mi.z >= span1);
                    bool core = false;
                    if (PROF == XC_VOIGT_W4 && mf.y > 0.f) {
                        float cpos = (float)mi.x + mf.x;
                        float thr = sqrtf(mf.y) + 1.f;
                        core = (cpos + thr >= (float)span0) && (cpos - thr <= (float)span1);
                    }
                    bool pairable = (PROF == XC_VOIGT_W4 || PROF == XC_LORENTZ);
                    fast = !none && full && !core && pairable;
                    slow = !none && !fast;
                }
                unsigned fm = __ballot_sync(0xffffffffu, fast);
                unsigned sm = __ballot_sync(0xffffffffu, slow);
                if (PROF == XC_VOIGT_W4 || PROF == XC_LORENTZ) {
                    // lines covering the whole span with no centre-zone point in it:
                    // unmasked, two grid points per packed f32x2 operation
                    const ulonglong2 *cq = reinterpret_cast<const ulonglong2 *>(smem);
                    // Voigt w4 region I: two lines share one reciprocal,
                    //   q1/D1 + q2/D2 = (q1 D2 + q2 D1) / (D1 D2),
                    // 5 FMA-pipe ops + 0.5 reciprocal per eval; the unpaired form (4 + 1) is
                    // bound by the MUFU reciprocal rate instead
                    while (PROF == XC_VOIGT_W4 && __popc(fm) >= 2) {
                        const int i1 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int i2 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int4 m1 = sMi[i1], m2 = sMi[i2];
                        const float f1 = sMf[i1].x, n1 = (float)m1.x, f2 = sMf[i2].x, n2 = (float)m2.x;
                        const f32x2 nn1 = pk2(n1, n1), ff1 = pk2(f1, f1), nn2 = pk2(n2, n2), ff2 = pk2(f2, f2);
                        f32x2 ua[R / 2], ub[R / 2];
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) {
                            f32x2 da = sub2(sub2(jf2[q], nn1), ff1), db = sub2(sub2(jf2[q], nn2), ff2);
                            ua[q] = mul2(da, da);
                            ub[q] = mul2(db, db);
                        }
                        // conditions for which every point of the span lies in the far wing of
                        // both lines (u >= u_far): series in r = 1/u, with r shared by them all
                        unsigned far = 0;
                        {
                            bool fl = false;
                            if (lane < CG) {
                                const float D1 = reinterpret_cast<const float4 *>(smem + (size_t)48 * (i1 * CG + lane))[2].w;
                                const float D2 = reinterpret_cast<const float4 *>(smem + (size_t)48 * (i2 * CG + lane))[2].w;
                                fl = span_far(m1.x, D1, span0, span1) && span_far(m2.x, D2, span0, span1);
                            }
                            far = __ballot_sync(0xffffffffu, fl);
                        }
                        f32x2 ra[R / 2], rb[R / 2];
                        if (far) {
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                ra[q] = rcp2(ua[q]);
                                rb[q] = rcp2(ub[q]);
                            }
                        }
                        if (far == kAllConds) {  // the common case: no per-condition branch
#pragma unroll
                            for (int c = 0; c < CG; ++c)
                                w4_series_pair<R, CG>(acc, c, smem + (size_t)48 * (i1 * CG + c),
                                                      smem + (size_t)48 * (i2 * CG + c), ra, rb);
                            continue;
                        }
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const unsigned char *e1 = smem + (size_t)48 * (i1 * CG + c);
                            const unsigned char *e2 = smem + (size_t)48 * (i2 * CG + c);
                            if ((far >> c) & 1u) {
                                w4_series_pair<R, CG>(acc, c, e1, e2, ra, rb);
                                continue;
                            }
                            const ulonglong2 a0 = reinterpret_cast<const ulonglong2 *>(e1)[0];
                            const ulonglong2 a1 = reinterpret_cast<const ulonglong2 *>(e1)[1];
                            const ulonglong2 b0 = reinterpret_cast<const ulonglong2 *>(e2)[0];
                            const ulonglong2 b1 = reinterpret_cast<const ulonglong2 *>(e2)[1];
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                f32x2 D1 = fma2(ua[q], add2(ua[q], a0.x), a0.y);
                                f32x2 D2 = fma2(ub[q], add2(ub[q], b0.x), b0.y);
                                f32x2 q1 = fma2(a1.x, ua[q], a1.y);
                                f32x2 q2 = fma2(b1.x, ub[q], b1.y);
                                f32x2 num = fma2(q1, D2, mul2(q2, D1));
                                acc[q][c] = fma2(num, rcp2(mul2(D1, D2)), acc[q][c]);
                            }
                        }
                    }
                    // Lorentz: two lines share one reciprocal, (P1 D2 + P2 D1) / (D1 D2): its
                    // unpaired form would be bound by the MUFU pipe (1/4 of the FMA rate)
                    while (PROF == XC_LORENTZ && __popc(fm) >= 2) {
                        const int i1 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int i2 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int4 m1 = sMi[i1], m2 = sMi[i2];
                        const float f1 = sMf[i1].x, n1 = (float)m1.x, f2 = sMf[i2].x, n2 = (float)m2.x;
                        const f32x2 nn1 = pk2(n1, n1), ff1 = pk2(f1, f1), nn2 = pk2(n2, n2), ff2 = pk2(f2, f2);
                        f32x2 ua[R / 2], ub[R / 2];
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) {
                            f32x2 da = sub2(sub2(jf2[q], nn1), ff1), db = sub2(sub2(jf2[q], nn2), ff2);
                            ua[q] = mul2(da, da);
                            ub[q] = mul2(db, db);
                        }
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const ulonglong2 a = cq[i1 * CG + c], b = cq[i2 * CG + c];
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                f32x2 D1 = add2(ua[q], a.x), D2 = add2(ub[q], b.x);
                                f32x2 num = fma2(a.y, D2, mul2(b.y, D1));
                                acc[q][c] = fma2(num, rcp2(mul2(D1, D2)), acc[q][c]);
                            }
                        }
                    }
                    while (fm) {
                        const int i1 = ib + __ffs(fm) - 1;
                        fm &= fm - 1;
                        const int4 m1 = sMi[i1];
                        const float f1 = sMf[i1].x, n1 = (float)m1.x;
                        const f32x2 nn = pk2(n1, n1), ff = pk2(f1, f1);
                        f32x2 u2[R / 2];
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) {
                            f32x2 d2 = sub2(sub2(jf2[q], nn), ff);
                            u2[q] = mul2(d2, d2);
                        }
#pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            if (PROF == XC_VOIGT_W4) {
                                const ulonglong2 *e1 = reinterpret_cast<const ulonglong2 *>(smem + (size_t)48 * (i1 * CG + c));
                                const ulonglong2 a0 = e1[0], a1 = e1[1];
#pragma unroll
                                for (int q = 0; q < R / 2; ++q) {
                                    f32x2 D = fma2(u2[q], add2(u2[q], a0.x), a0.y);
                                    f32x2 num = fma2(a1.x, u2[q], a1.y);
                                    acc[q][c] = fma2(num, rcp2(D), acc[q][c]);
                                }
                            } else {
                                const ulonglong2 a0 = cq[i1 * CG + c];
#pragma unroll
                                for (int q = 0; q < R / 2; ++q)
                                    acc[q][c] = fma2(a0.y, rcp2(add2(u2[q], a0.x)), acc[q][c]);
                            }
                        }
                    }
                }
                while (sm) {
                    int i1 = ib + __ffs(sm) - 1;
                    sm &= sm - 1;
                    const int4 m1 = sMi[i1];
                    const float f1 = sMf[i1].x;
                    const float n1 = (float)m1.x;
                    float d1[R], u1[R];
                    bool in1[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        d1[r] = (jf[r] - n1) - f1;
                        u1[r] = d1[r] * d1[r];
                        in1[r] = (ji[r] >= m1.y) && (ji[r] <= m1.z);
                    }
                    // Voigt w4: far-wing series where the whole span is far for a condition
                    // (typically the spans holding a cut edge)
                    unsigned far = 0;
                    float rr[R];
                    if (PROF == XC_VOIGT_W4) {
                        bool fl = false;
                        if (lane < CG)
                            fl = span_far(m1.x, reinterpret_cast<const float4 *>(smem + (size_t)48 * (i1 * CG + lane))[2].w,
                                          span0, span1);
                        far = __ballot_sync(0xffffffffu, fl);
                        if (far) {
#pragma unroll
                            for (int r = 0; r < R; ++r) rr[r] = in1[r] ? rcp_approx(u1[r]) : 0.f;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < CG; ++c) {
                        if (PROF == XC_VOIGT_W4 && ((far >> c) & 1u)) {
                            const float4 s1 = reinterpret_cast<const float4 *>(smem + (size_t)48 * (i1 * CG + c))[2];
#pragma unroll
                            for (int q = 0; q < R / 2; ++q) {
                                float a0, a1;
                                upk2(acc[q][c], a0, a1);
                                const float r0 = rr[2 * q], r1 = rr[2 * q + 1];
                                a0 = fmaf(fmaf(fmaf(s1.z, r0, s1.y), r0, s1.x), r0, a0);
                                a1 = fmaf(fmaf(fmaf(s1.z, r1, s1.y), r1, s1.x), r1, a1);
                                acc[q][c] = pk2(a0, a1);
                            }
                            continue;
                        }
                        const float4 A1 = load_consts<PROF>(smem, i1 * CG + c);
                        const float4 B1 = Lay::kHasB ? sB[i1 * CG + c] : make_float4(0.f, 0.f, 0.f, -1.f);
#pragma unroll
                        for (int q = 0; q < R / 2; ++q) {
                            float a0, a1;
                            upk2(acc[q][c], a0, a1);
                            if (in1[2 * q]) a0 += contrib_single<PROF>(u1[2 * q], d1[2 * q], A1, B1, sX, sW, p.ngh);
                            if (in1[2 * q + 1])
                                a1 += contrib_single<PROF>(u1[2 * q + 1], d1[2 * q + 1], A1, B1, sX, sW, p.ngh);
                            acc[q][c] = pk2(a0, a1);
                        }
                    }
                }
            }
            if (++chunk == FOLD_CHUNKS) {
                fold_acc<R, CG>(acc, ji, kw, grp, p, sScale, sRow, first_fold && !TCN && !p.tc_far);
                first_fold = false;
                chunk = 0;
            }
        }
        fold_acc<R, CG>(acc, ji, kw, grp, p, sScale, sRow, first_fold && !TCN && !p.tc_far);
    }
}

// ---------------------------------------------------------------------------
// Far-wing kernel on the tensor cores (Voigt w4, FP32, fixed cut, many conditions).
//
// For a block of 128 grid points and a line l far from all of them (integer
// radius D4(l, c), see w4_zone), the region-I rational of condition c equals its
// series r (p0 + p1 r + p2 r^2 + p3 r^3), r = 1/u, to < 2e-7.  Summed over lines,
//   F[k, c] = sum_l sum_j r_kl^(j+1) p_j(l, c)
// is a matrix product: A[k, (j, l)] = r_kl^(j+1) depends on the point and the
// line only, B[(j, l), c] = p_j(l, c) on the line and the condition only.  A CTA
// owns TC_BLK blocks of 128 points (one TMEM lane per point, one warp quadrant
// per 32 points) and 32 conditions (the MMA's N), walks the lines whose cut reaches
// its points in chunks of TC_L, and per chunk: computes the series coefficients of
// every (line, condition) once, stores per block a B operand in shared memory (zero
// where (l, c) is not far from that block: the CUDA-core kernel evaluates those),
// writes A to tensor memory, and per block one thread issues tcgen05.mma kind::tf32
// (M = 128, N = 32, K = 8): a CTA keeps one MMA chain per block in flight.  Operand
// precision follows each term's weight (four terms, x = C r <= 0.012): for j = 0 (the
// value itself) and j = 1 (<= 3x = 0.036 of it) r^(j+1) and p_j are split x = hi + lo
// with hi exact in TF32, D += Ahi Bhi + Ahi Blo + Alo Bhi (the dropped Alo Blo is
// < 2^-20 of the product; hi is x with its low 13 mantissa bits cleared, a bias
// toward zero below 5e-7); the j = 2 term (<= 5x^2 = 7e-4 of the value) and the j = 3
// term (<= 7x^3 = 1.3e-5) take r^3, r^4, p2, p3 as the MMA reads them (TF32: relative
// error <= 2^-10 of a term that small, < 7e-7).  Eight MMAs per chunk and block.  A
// and B are double buffered (the next chunk is built while the MMAs of this one run).
// The tensor
// core adds in FP32 with truncation, a bias that grows with the number of MMAs
// summed into one accumulator, so D is restarted every TC_FOLD chunks after its
// value is added into compensated (Kahan) FP32 sums in shared memory; the blocks
// are written (not added) to the output at the end.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;                 // points per block = MMA M = TMEM lanes
constexpr int TC_BLK = 2;                 // blocks per CTA (one MMA issuer each)
constexpr int TC_T = TC_M * TC_BLK;       // threads per CTA: one per point
constexpr int TC_N = 32;                  // conditions per tile = MMA N
constexpr int TC_L = 8;                   // lines per chunk
constexpr int TC_J = 4;                   // series terms
constexpr int TC_ACOLS = 5 * TC_L;        // A columns per chunk: r hi, r lo, r^2, r^3, r^4
constexpr int TC_ASTRIDE = 48;            // TMEM columns between the two A buffers
constexpr int TC_BT = 5;                  // B tiles (K = 8 each): p0 hi, p0 lo, p1, p2, p3
constexpr int TC_MMAS = 6;                // MMAs per chunk and block
constexpr int TC_FOLD = 16;               // chunks per tensor-memory accumulation period
constexpr uint32_t TC_COLS = 128 * TC_BLK;// TMEM columns: per block D 32 + 2 buffers x 48
constexpr int TC_BTILE = TC_N * TC_L;     // one B tile: 8 K x 32 N = 256 floats (1 KB)
constexpr size_t TC_SMEM_B = (size_t)TC_BLK * 2 * TC_BT * TC_BTILE * sizeof(float);  // [blk][buf][tile]
constexpr size_t TC_SMEM_ACC = (size_t)2 * TC_N * TC_T * sizeof(float);           // compensated FP32 sums
constexpr size_t TC_SMEM = 100 * 1024;    // B + sums + barriers; sized so that 2 CTAs (2 x 256 TMEM
                                          // columns) and never 3 share an SM
static_assert(TC_N + 2 * TC_ASTRIDE <= 128 && TC_ACOLS <= TC_ASTRIDE, "far-wing kernel tensor-memory columns");
static_assert(TC_SMEM_B + TC_SMEM_ACC + 128 + 4 * TC_L * 16 + 2 * TC_L * 4 + 12 <= TC_SMEM, "far-wing kernel shared memory");

// a chunk line with a cut covering the whole super-block [t0, t0 + TC_T) and its centre
// at least one step outside it: no range test and no guard against u < 1 needed
__device__ __forceinline__ bool tc_line_plain(const float4 &g, int t0) {
    return g.z <= (float)t0 && g.w >= (float)(t0 + TC_T - 1) &&
           (g.x <= (float)(t0 - 2) || g.x >= (float)(t0 + TC_T + 1));
}
constexpr int TC_NB = TC_N * TC_L;        // (line, condition) pairs per chunk
static_assert(TC_NB == TC_T, "one (line, condition) pair per thread and chunk");
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

struct TcParams {
    const float4 *geo;                 // per line: integer position n, fraction f, ka, kb (floats)
    const float4 *phys;                // per line: nu, E'', g A / nu^2, gamma_ref (float)
    const float *n_T;                  // per line: temperature exponent
    const CParam *cp;
    const uint32_t *keep;              // intensity-threshold decisions (see LinesDev::keep), or nullptr
    int keep_words;
    const float *gamma_lc;             // widths under a broadener mixture (see LinesDev::gamma_lc), or nullptr
    int gamma_stride;
    const unsigned *blk_lo, *blk_hi;   // per TC_T-point super-block: line range
    int *counter;
    int *status;                       // set to 1 if a wait ran out
    int n_tiles, n_groups, n_cond;
    int64_t n_pts;
    float h, inv_h;
    double *sigma;
};

// element (n, k) of an 8 (K) x 32 (N) B tile, K-major with 8 x 16-byte core matrices:
// core (n / 8, k / 4) at ((n / 8) * 2 + k / 4) * 128 bytes (LBO 128, SBO 256)
__device__ __forceinline__ int tc_b_index(int n, int k) {
    return (((n >> 3) * 2 + (k >> 2)) * 128 + (n & 7) * 16 + (k & 3) * 4) >> 2;
}

// series coefficients (p0, p1, p2) and far radius D4 of a (line, condition), p3 in *p3;
// D4 is the same value line_consts gives (same inputs, same rounded operations)
template <bool EXT>
__device__ __forceinline__ float4 tc_series_consts(const float4 &ph, float nT, const CParam &c, float inv_h,
                                                   float *p3, float ga_lc) {
    const float nu = ph.x, E = ph.y;
    const float z = fmaf(E, c.kT_hi, E * c.kT_lo);
    float I;
    if (EXT && c.emis != 0.f)
        I = c.pref * (ph.z * (nu * nu * nu)) * exp2_neg(z) * exp2_neg(fmaf(nu, c.kT_hi, nu * c.kT_lo));
    else
        I = c.pref * ph.z * exp2_neg(z) * (-expm1f(-c.c2T * nu));
    float ah, gh;
    if (EXT && ga_lc >= 0.f) {   // broadener mixture: this (line, condition)'s width (see line_consts)
        ah = __fmul_rn(c.acoef * nu, inv_h);
        gh = __fmul_rn(ga_lc, inv_h);
    } else {
        line_widths(nu, ph.w, nT, c, inv_h, &ah, &gh);
    }
    const W4Zone zn = w4_zone(ah, gh);
    const float b = ah * ah * (float)(0.5 / 0.6931471805599453), g2 = gh * gh;
    const float P = I * kKappa * gh * inv_h;
    const float e5 = g2 - 5.f * b;
    const float c1 = 3.f * b - g2, c2 = fmaf(e5, e5, -20.f * b * b);
    const float Cw = b + g2, Ew = 2.f * (g2 - b);
    *p3 = P * -fmaf(Ew, c2, Cw * Cw * c1);   // c3 = -E c2 - F c1
    return make_float4(P, P * c1, P * c2, zn.D4);
}

template <bool EXT>
__global__ void __launch_bounds__(TC_T, 2) k_far_tc(TcParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *sB = reinterpret_cast<float *>(smem);                           // [blk][buf][tile][256]
    float *sSum = reinterpret_cast<float *>(smem + TC_SMEM_B);             // [c][point]
    float *sCmp = sSum + TC_N * TC_T;                                       // Kahan compensation
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + TC_SMEM_B + TC_SMEM_ACC);  // [blk][buf]
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(mbar + 2 * TC_BLK);
    int *sTile = reinterpret_cast<int *>(sTmem + 1);
    // the chunk's line records, double buffered: loaded into registers by TC_L threads one
    // chunk ahead and stored before the chunk's barrier, so their latency is hidden
    float4 *sGeo = reinterpret_cast<float4 *>(smem + TC_SMEM_B + TC_SMEM_ACC + 128);   // [2][TC_L]
    float4 *sPhys = sGeo + 2 * TC_L;                                                     // [2][TC_L]
    float *sNT = reinterpret_cast<float *>(sPhys + 2 * TC_L);                            // [2][TC_L]
    int *sFast = reinterpret_cast<int *>(sNT + 2 * TC_L);                                // [2]
    volatile int *sAbort = sFast + 2;                                                    // a wait ran out

    const int tid = threadIdx.x, warp = tid >> 5;
    const int blkh = tid / TC_M;                 // this thread's block within the CTA
    if (tid == 0) {
        for (int i = 0; i < 2 * TC_BLK; ++i) tc::mbar_init(&mbar[i], 1);
        tc::mbar_init_fence();
        *sAbort = 0;
    }
    if (warp == 0) tc::tmem_alloc(sTmem, TC_COLS);
    for (int c = 0; c < TC_N; ++c) sSum[c * TC_T + tid] = sCmp[c * TC_T + tid] = 0.f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *sTmem;
    const uint32_t tblk = tbase + 128u * blkh;                                // this block's columns
    const uint32_t t_lane = tblk + ((uint32_t)((warp & 3) * 32) << 16);       // this warp's lanes
    constexpr uint32_t kIdesc = tc::idesc_tf32(128, TC_N);
    const uint32_t sB_addr = tc::smem_u32(sB);
    // One MMA-issuing thread per block, in a warp of that block.  MMA issue from one
    // SM sub-partition is serialised, so the two issuers sit on different sub-partitions
    // (warp % 4), and CTAs of odd index use the other two (two CTAs share an SM).
    // (One CTA of four blocks and four issuers per SM measured slower.)
    const bool odd_cta = (blockIdx.x & 1) != 0;
    const bool issuer = (tid & 31) == 0 && (warp == (odd_cta ? 2 : 0) || warp == (odd_cta ? 7 : 5));
    // descriptor of this block's B operand (buffer 0, hi); the whole region lies below
    // 256 KB, so the start field never carries into the next one
    const uint64_t desc_b0 = tc::smem_desc(sB_addr + (uint32_t)(blkh * 2 * TC_BT * TC_BTILE * 4), 128u, 256u);

    uint32_t uses[2] = {0u, 0u};   // commits per buffer (each block's barrier of it) so far
    // `ok` is per thread (its own bounded waits).  A thread whose wait ran out raises the
    // shared flag before the next barrier; after that barrier every thread sees it (`stop`):
    // no further MMA is issued and no further output is written.
    bool ok = true, stop = false;
    // The (line, condition) pair whose coefficients this thread computes each chunk, chosen
    // so that a warp's B entries of one term fill one 8 x 4 core matrix (32 consecutive
    // floats: conflict-free stores): conditions 8 (w % 4) .. + 7, lines 4 (w / 4) .. + 3.
    const int lane = tid & 31;
    const int cB = (warp & 3) * 8 + (lane >> 2), lB = (warp >> 2) * 4 + (lane & 3);
    const int bix = tc_b_index(cB, lB);   // the same slot in each of the five B tiles

    for (;;) {
        if (tid == 0) *sTile = atomicAdd(p.counter, 1);
        __syncthreads();
        const int t = *sTile;
        __syncthreads();
        if (t >= p.n_tiles) break;
        const int sblk = t / p.n_groups, grp = t % p.n_groups;
        const int t0 = sblk * TC_T;               // first point of the super-block
        const float kf = (float)(t0 + tid);       // this thread's point (exact: < 2^23)
        const unsigned lo = p.blk_lo[sblk], hi = p.blk_hi[sblk];
        const int nl = (int)(hi - lo);
        const int nch = (nl + TC_L - 1) / TC_L;
        const float4 *geo = p.geo + lo;
        const float4 *phys = p.phys + lo;
        const float *nT = p.n_T + lo;
        const int cc = grp * TC_N + cB;
        CParam cpr;
        if (cc < p.n_cond) cpr = p.cp[cc];
        if (warp == 0 && nch > 0) {
            bool plain = true;
            if (tid < TC_L) {
                const int li = tid < nl ? tid : 0;
                const float4 g = geo[li];
                sGeo[tid] = g;
                sPhys[tid] = phys[li];
                sNT[tid] = nT[li];
                plain = tid < nl && tc_line_plain(g, t0);
            }
            const unsigned all = __ballot_sync(0xffffffffu, plain);
            if (tid == 0) sFast[0] = all == 0xffffffffu;
        }
        __syncthreads();
        int in_fold = 0;
        for (int ci = 0; ci < nch; ++ci) {
            const int b = ci & 1;
            // next chunk's records: issue the loads now, store them before this chunk's barrier
            float4 nGeo, nPhys;
            float nNT = 0.f;
            const bool pre = tid < TC_L && ci + 1 < nch;
            if (pre) {
                const int li = min((ci + 1) * TC_L + tid, nl - 1);
                nGeo = geo[li];
                nPhys = phys[li];
                nNT = nT[li];
            }
            const bool fast = sFast[b] != 0;
            const float4 *cGeo = sGeo + b * TC_L;
            // buffer b of every block is free once the MMAs of its previous chunk completed
            if (uses[b] > 0u) {
#pragma unroll
                for (int hb = 0; hb < TC_BLK; ++hb)
                    ok &= tc::mbar_wait(&mbar[hb * 2 + b], (uses[b] - 1u) & 1u, TC_WAIT_LIMIT);
                tc::fence_after_sync();
            }
            const int l0 = ci * TC_L;
            // ---- B: series coefficients of this thread's (line, condition), per block zero
            // unless far from all of that block's points, split hi + lo
            {
                float4 S = make_float4(0.f, 0.f, 0.f, __int_as_float(0x7f800000));
                float p3 = 0.f;
                float na = 0.f;
                bool live = false;
                if (l0 + lB < nl && cc < p.n_cond) {
                    const float4 g = cGeo[lB];
                    live = g.w >= g.z;   // non-empty cut range
                    na = g.x;
                    const size_t lg = (size_t)lo + (size_t)(l0 + lB);
                    const float ga_lc =
                        (EXT && p.gamma_lc) ? p.gamma_lc[lg * (size_t)p.gamma_stride + cpr.row] : -1.f;
                    S = tc_series_consts<EXT>(sPhys[b * TC_L + lB], sNT[b * TC_L + lB], cpr, p.inv_h, &p3, ga_lc);
                    if (EXT && p.keep && !((p.keep[lg * (size_t)p.keep_words + (cpr.row >> 5)] >> (cpr.row & 31)) & 1u)) {
                        S.x = S.y = S.z = 0.f;   // left out by the intensity threshold
                        p3 = 0.f;
                    }
                }
                // p0 as hi + lo; p1 rounded to the nearest TF32 value (where the series is
                // used its term is at most 3.6 % of p0's, so one unbiased TF32 rounding of each
                // factor stays below 4e-5 of the sum)
                const float p0h = tc::tf32_trunc(S.x);
                const float p0l = S.x - p0h, p1r = tc::tf32_round(S.y), p2h = S.z;
#pragma unroll
                for (int hb = 0; hb < TC_BLK; ++hb) {
                    // span_far in float: na and the block ends are exact integers below 2^24,
                    // so the differences are exact and the test is the same
                    const float b0 = (float)(t0 + hb * TC_M);
                    const bool far = live && ((na - (b0 + (float)(TC_M - 1)) > S.w) || (b0 - na > S.w));
                    float *bt = sB + (size_t)(hb * 2 + b) * TC_BT * TC_BTILE + bix;
                    bt[0 * TC_BTILE] = far ? p0h : 0.f;
                    bt[1 * TC_BTILE] = far ? p0l : 0.f;
                    bt[2 * TC_BTILE] = far ? p1r : 0.f;
                    bt[3 * TC_BTILE] = far ? p2h : 0.f;
                    bt[4 * TC_BTILE] = far ? p3 : 0.f;
                }
            }
            // ---- A: r^(j+1) of this thread's point for the chunk's lines (r split hi + lo,
            // r^2 rounded to the nearest TF32 value)
            {
                float av[TC_ACOLS];   // [r hi | r lo | r^2 | r^3 | r^4], TC_L lines each
#pragma unroll
                for (int l8 = 0; l8 < TC_L; ++l8) {
                    float r;
                    const float4 g = cGeo[l8];
                    const float d = (kf - g.x) - g.y;
                    if (fast) {
                        // every line covers the super-block, no centre in it
                        r = rcp_approx(d * d);
                    } else {
                        // inside the cut; points within one step of the centre only ever
                        // meet zero B entries (not far), r is kept finite there
                        r = (l0 + l8 < nl && kf >= g.z && kf <= g.w) ? rcp_approx(fmaxf(d * d, 1.f)) : 0.f;
                    }
                    const float r2 = r * r;
                    const float rh = tc::tf32_trunc(r);
                    av[l8] = rh;
                    av[TC_L + l8] = r - rh;
                    av[2 * TC_L + l8] = tc::tf32_round(r2);
                    av[3 * TC_L + l8] = r2 * r;    // the MMA reads r^3, r^4, p2, p3 as TF32
                    av[4 * TC_L + l8] = r2 * r2;
                }
                const uint32_t ta = t_lane + 32u + (uint32_t)b * TC_ASTRIDE;
                static_assert(TC_ACOLS == 2 * 16 + 8, "A stores: two 16-column and one 8-column store");
                float v16[16];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v16[i] = av[16 * q + i];
                    tc::tmem_st16(ta + 16u * q, v16);
                }
                float v8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) v8[i] = av[32 + i];
                tc::tmem_st8(ta + 32u, v8);
                tc::tmem_st_wait();
            }
            if (warp == 0 && ci + 1 < nch) {
                bool plain = true;
                if (pre) {
                    const int nb = (b ^ 1) * TC_L;
                    sGeo[nb + tid] = nGeo;
                    sPhys[nb + tid] = nPhys;
                    sNT[nb + tid] = nNT;
                    plain = (ci + 1) * TC_L + tid < nl && tc_line_plain(nGeo, t0);
                }
                const unsigned all = __ballot_sync(0xffffffffu, plain);
                if (tid == 0) sFast[b ^ 1] = all == 0xffffffffu;
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            if (!ok) *sAbort = 1;
            __syncthreads();
            if (*sAbort) {   // a buffer may still be in use: issue nothing more
                stop = true;
                break;
            }
            if (issuer) {
                tc::fence_after_sync();
                const uint32_t a0 = tblk + 32u + (uint32_t)b * TC_ASTRIDE;
                // descriptors differ only in the start address field (bits 0-13, 16-byte units):
                // tile t of buffer b at + (b * TC_BT + t) KB
                const uint64_t d0 = desc_b0 + (uint64_t)(b * TC_BT * (TC_BTILE * 4 / 16));
                constexpr uint64_t kT = TC_BTILE * 4 / 16;
                static_assert(TC_MMAS == 6, "the issue sequence below");
                tc::mma_tf32_ts(tblk, a0 + 0u * TC_L, d0 + 0 * kT, kIdesc, in_fold > 0 ? 1u : 0u);  // rhi p0hi
                tc::mma_tf32_ts(tblk, a0 + 0u * TC_L, d0 + 1 * kT, kIdesc, 1u);                    // rhi p0lo
                tc::mma_tf32_ts(tblk, a0 + 1u * TC_L, d0 + 0 * kT, kIdesc, 1u);                    // rlo p0hi
                tc::mma_tf32_ts(tblk, a0 + 2u * TC_L, d0 + 2 * kT, kIdesc, 1u);                    // r^2 p1
                tc::mma_tf32_ts(tblk, a0 + 3u * TC_L, d0 + 3 * kT, kIdesc, 1u);                    // r^3 p2
                tc::mma_tf32_ts(tblk, a0 + 4u * TC_L, d0 + 4 * kT, kIdesc, 1u);                    // r^4 p3
                tc::mma_commit(&mbar[blkh * 2 + b]);
            }
            ++uses[b];
            if (++in_fold == TC_FOLD || ci == nch - 1) {
                // this block's tensor-memory sums -> compensated FP32 sums (one row per thread)
                ok &= tc::mbar_wait(&mbar[blkh * 2 + b], (uses[b] - 1u) & 1u, TC_WAIT_LIMIT);
                tc::fence_after_sync();
                float v[32];
                tc::tmem_ld32(t_lane, v);
#pragma unroll
                for (int c = 0; c < TC_N; ++c) {
                    const float sm = sSum[c * TC_T + tid];
                    const float y = __fsub_rn(v[c], sCmp[c * TC_T + tid]);
                    const float tt = __fadd_rn(sm, y);
                    sCmp[c * TC_T + tid] = __fsub_rn(__fsub_rn(tt, sm), y);
                    sSum[c * TC_T + tid] = tt;
                }
                tc::fence_before_sync();
                in_fold = 0;
            }
        }
        if (stop) break;
        // ---- the super-block's far-wing sums: first writer of these outputs.  A thread's
        // sums come from its own block's MMAs only, all covered by its own last wait: it
        // writes them only if every wait of its own succeeded
        const int64_t k = (int64_t)t0 + tid;
        for (int c = 0; c < TC_N; ++c) {
            const int c2 = grp * TC_N + c;
            if (ok && k < p.n_pts && c2 < p.n_cond)
                p.sigma[(size_t)p.cp[c2].row * (size_t)p.n_pts + (size_t)k] =
                    ((double)sSum[c * TC_T + tid] - (double)sCmp[c * TC_T + tid]) * p.cp[c2].inv_scale;
            sSum[c * TC_T + tid] = sCmp[c * TC_T + tid] = 0.f;
        }
    }
    if (!ok) *sAbort = 1;
    tc::fence_before_sync();
    __syncthreads();
    if (*sAbort) {
        // a wait ran out: before the tensor memory is released, wait (bounded again) for the
        // last commit of each block's buffers, which covers every MMA issued before it; the
        // status flag tells the host that this launch's output is not valid
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (uses[b] > 0u)
#pragma unroll
                for (int hb = 0; hb < TC_BLK; ++hb)
                    (void)tc::mbar_wait(&mbar[hb * 2 + b], (uses[b] - 1u) & 1u, TC_WAIT_LIMIT);
        if (tid == 0) atomicExch(p.status, 1);
        tc::fence_before_sync();
        __syncthreads();
    }
    if (warp == 0) tc::tmem_dealloc(tbase, TC_COLS);
}

// The far-wing kernel's algorithmic work: for every (line, condition), the grid points
// inside the line's cut that lie in a 128-point block far from it -- the same test on the
// same rounded values as k_far_tc (the radius D4 from the line's widths, the integer line
// position n): a block [b0, b0 + 127] is far when n - (b0 + 127) > D4 or b0 - n > D4.  The
// far blocks are those wholly below n - D4 or above n + D4, so the count is two interval
// lengths per pair.  Run on request (xc_count_far_evals), not inside the sweep.
__global__ void k_far_count(const float4 *__restrict__ geo, const float4 *__restrict__ phys,
                            const float *__restrict__ n_T, const CParam *__restrict__ cp, int nc,
                            const float *gamma_lc, int gamma_stride, size_t n, float inv_h,
                            unsigned long long *count) {
    unsigned long long acc = 0;
    const size_t total = n * (size_t)nc;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t l = i / (size_t)nc;
        const CParam c = cp[i % (size_t)nc];
        const float4 g = geo[l];
        if (!(g.w >= g.z)) continue;   // empty cut range
        const float4 ph = phys[l];
        float ah, gh;
        if (gamma_lc) {
            ah = __fmul_rn(c.acoef * ph.x, inv_h);
            gh = __fmul_rn(gamma_lc[l * (size_t)gamma_stride + c.row], inv_h);
        } else {
            line_widths(ph.x, ph.w, n_T[l], c, inv_h, &ah, &gh);
        }
        const double D = (double)w4_zone(ah, gh).D4;
        const double na = (double)g.x, ka = (double)g.z, kb = (double)g.w;
        double cnt = 0.0;
        const double X = na - D - (double)(TC_M - 1);   // far-left: TC_M j < X
        if (X > 0.0) {
            const double KL = (double)TC_M * (ceil(X / TC_M) - 1.0) + (double)(TC_M - 1);
            cnt += fmax(0.0, fmin(kb, KL) - ka + 1.0);
        }
        const double KR = (double)TC_M * (floor((na + D) / TC_M) + 1.0);   // far-right: TC_M j > n + D
        cnt += fmax(0.0, kb - fmax(ka, KR) + 1.0);
        acc += (unsigned long long)cnt;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(count, acc);
}

// ---------------------------------------------------------------------------
// Centre-zone kernel (Voigt w4): the points with |x| + y < 15, which the main
// kernel skips.  Gather form again: a CTA owns CORE_T consecutive grid points
// (one per thread) and a group of conditions, walks the lines whose centre zone
// can reach its window (|nu - x| < 18.02 alpha_max, a range of the sorted list),
// and for each of its points sums, in line order, Re w by region: I (rounding
// cases at the boundary), II (real two-Lorentzian-pair form) or III/IV (complex
// w4).  It runs after the main kernel and adds its FP32 sums into the FP64
// output each thread owns (every CORE_FLUSH chunks), so the result stays
// deterministic.  Which kernel evaluates a (line, point, condition) is decided by
// the same test u < thr^2 on bit-identical values, so every contribution is
// counted exactly once.
// ---------------------------------------------------------------------------
constexpr int CORE_T = 256;
constexpr int CORE_CG = 32;
constexpr int CORE_SCH = 16;
// The FP32 sums of a thread's point are added into the FP64 output every CORE_FLUSH chunks
// (1024 lines) and restarted: at the largest line densities tens of thousands of centre
// zones cover a point, and a single FP32 sum over all of them would round away its
// smallest terms (a systematic loss that grows with the density)
constexpr int CORE_FLUSH = 64;

struct CoreParams {
    LinesDev L;
    const int *n_abs;
    const float *f_frac;
    const int *ka_abs, *kb_abs;
    const CParam *cp;
    const unsigned *win_lo, *win_hi;
    int n_cond;
    int64_t n_pts;
    float h, inv_h;
    double *sigma;
};

// Re w in w4's regions III and IV (|x| + y < 5.5), the same forms as w4_eval with only
// the real part formed: region III the real part of the quotient; region IV needs
// cos(Im u) of exp(u), u = t^2, and no sine
__device__ __forceinline__ float w4_region34_re(float x, float y) {
    const Cx<float> t = cx<float>(y, -x);
    const float ax = fabsf(x);
    if (y >= 0.195f * ax - 0.176f) {
        const Cx<float> N = 16.4955f + t * (20.20933f + t * (11.96482f + t * (3.778987f + 0.5642236f * t)));
        const Cx<float> D = 16.4955f + t * (38.82363f + t * (39.27121f + t * (21.69274f + t * (6.699398f + t))));
        return (N.re * D.re + N.im * D.im) * recip(D.re * D.re + D.im * D.im);
    }
    const Cx<float> u = t * t;
    const Cx<float> m = cx<float>(-u.re, -u.im);
    const Cx<float> N = 36183.31f + m * (3321.9905f + m * (1540.787f + m * (219.0313f +
                        m * (35.76683f + m * (1.320522f + 0.56419f * m)))));
    const Cx<float> D = 32066.6f + m * (24322.84f + m * (9022.228f + m * (2186.181f +
                        m * (364.2191f + m * (61.57037f + m * (1.841439f + m))))));
    const Cx<float> r = cdiv(N, D);
    return expf(u.re) * cosf(u.im) - (t.re * r.re - t.im * r.im);
}

__global__ void __launch_bounds__(CORE_T) k_core_w4_f32(CoreParams p) {
    __shared__ float4 sB[CORE_SCH][CORE_CG];
    __shared__ int4 sMi[CORE_SCH];
    __shared__ float2 sMf[CORE_SCH];
    __shared__ double sScale[CORE_CG];
    __shared__ float sAcc[CORE_CG][CORE_T];  // per-thread column: the thread's point, every condition
    __shared__ float sThr[CORE_SCH][CORE_CG];         // per line: thresholds u < thr^2, descending
    __shared__ unsigned char sOrd[CORE_SCH][CORE_CG]; // ... and their conditions
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t kw = (int64_t)blockIdx.x * CORE_T;
    const int grp = blockIdx.y;
    const float jf = (float)tid;
    __shared__ int sRow[CORE_CG];
    if (tid < CORE_CG) {
        int c = grp * CORE_CG + tid;
        sScale[tid] = c < p.n_cond ? p.cp[c].inv_scale : 0.0;
        sRow[tid] = c < p.n_cond ? p.cp[c].row : 0;
    }
#pragma unroll
    for (int c = 0; c < CORE_CG; ++c) sAcc[c][tid] = 0.f;
    const unsigned lo = p.win_lo[blockIdx.x], hi = p.win_hi[blockIdx.x];
    const int64_t k_out = kw + tid;
    // add this thread's FP32 sums into the FP64 output (after the other kernels' values)
    auto flush = [&]() {
        if (k_out >= p.n_pts) return;
#pragma unroll
        for (int c = 0; c < CORE_CG; ++c) {
            const int cc = grp * CORE_CG + c;
            const float a = sAcc[c][tid];
            if (cc < p.n_cond && a != 0.f)
                p.sigma[(size_t)sRow[c] * (size_t)p.n_pts + (size_t)k_out] += (double)a * sScale[c];
            sAcc[c][tid] = 0.f;
        }
    };
    // strided chunks (lines lo + ci + j * nch): the centre zones of one chunk spread
    // over the whole window instead of piling onto the threads of one spot
    const unsigned nl = hi - lo;
    const unsigned nch = (nl + CORE_SCH - 1) / CORE_SCH;
    for (unsigned ci = 0; ci < nch; ++ci) {
        const int cnt = (int)((nl - ci + nch - 1) / nch);
        __syncthreads();
        if (tid < cnt) {
            size_t l = (size_t)lo + ci + (size_t)tid * nch;
            int ka = p.ka_abs[l], kb = p.kb_abs[l];
            int64_t kaw = (int64_t)ka - kw, kbw = (int64_t)kb - kw;
            if (kb < ka) { kaw = 1; kbw = 0; }
            kaw = i64max(-1, i64min(kaw, CORE_T));
            kbw = i64max(-1, i64min(kbw, CORE_T));
            sMi[tid] = make_int4((int)((int64_t)p.n_abs[l] - kw), (int)kaw, (int)kbw, 0);
            sMf[tid].x = p.f_frac[l];
        }
#pragma unroll 1
        for (int pb = 0; pb < CORE_SCH * CORE_CG; pb += CORE_T) {
            int q = pb + tid;
            int i = q / CORE_CG, c = q % CORE_CG;
            int cc = grp * CORE_CG + c;
            float t2 = -1.f;
            float4 A, S, B = make_float4(0.f, 0.f, 0.f, -1.f);
            if (i < cnt && cc < p.n_cond)
                line_consts<XC_VOIGT_W4>(p.L, (size_t)lo + ci + (size_t)i * nch, p.cp[cc], p.h, p.inv_h, &A, &B,
                                         &t2, &S);
            if (i < cnt) sB[i][c] = B;
            // one line per warp (CORE_CG == 32 lanes = conditions): bitonic sort of the
            // thresholds, largest first, so the point loop can stop at the first
            // condition whose centre zone does not reach the point
            float key = -t2;
            int val = c;
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int j = k >> 1; j > 0; j >>= 1) {
                    float pkey = __shfl_xor_sync(0xffffffffu, key, j);
                    int pval = __shfl_xor_sync(0xffffffffu, val, j);
                    bool asc = (lane & k) == 0, low = (lane & j) == 0;
                    bool take = low ? (asc ? pkey < key : pkey > key) : (asc ? pkey > key : pkey < key);
                    if (take) {
                        key = pkey;
                        val = pval;
                    }
                }
            }
            if (i < cnt) {
                sThr[i][lane] = -key;
                sOrd[i][lane] = (unsigned char)val;
                if (lane == 0) sMf[i].y = -key;  // the largest threshold of the line
            }
        }
        __syncthreads();
        // the chunk's lines whose widest centre zone can reach this warp's 32 points
        unsigned wl = 0;
        {
            bool hit = false;
            if (lane < cnt) {
                const int4 m = sMi[lane];
                const float2 mf = sMf[lane];
                if (mf.y > 0.f) {
                    const float cpos = (float)m.x + mf.x, thr = sqrtf(mf.y) + 2.f;
                    const float w0 = (float)(tid - lane), w1 = w0 + 31.f;
                    hit = cpos + thr >= w0 && cpos - thr <= w1 && m.y <= (int)w1 && m.z >= (int)w0;
                }
            }
            wl = __ballot_sync(0xffffffffu, hit);
        }
        while (wl) {
            const int i = __ffs(wl) - 1;
            wl &= wl - 1;
            const int4 m = sMi[i];
            const float2 mf = sMf[i];
            const float d = (jf - (float)m.x) - mf.x;
            const float u = d * d;
            if (!(u < mf.y) || tid < m.y || tid > m.z) continue;
            const float ad = fabsf(d);
#pragma unroll 1
            for (int kk = 0; kk < CORE_CG; ++kk) {
                if (!(u < sThr[i][kk])) break;
                const int c = sOrd[i][kk];
                const float4 B = sB[i][c];
                float x = B.x * ad, y = B.y, s = x + y;
                float w = s >= 15.f ? w4_region1_re(x, y)
                                    : (s >= 5.5f ? w4_region2_re(x, y) : w4_region34_re(x, y));
                sAcc[c][tid] = fmaf(B.z, w, sAcc[c][tid]);
            }
        }
        if ((ci + 1) % CORE_FLUSH == 0) flush();   // this thread's own column: no barrier needed
    }
    flush();
}

// window -> line range for the centre zone: |nu - x| < K nu with K = 18.02 alpha_max/nu
__global__ void k_core_ranges(const double *__restrict__ nu, int64_t n, double nu_A, double step, int64_t n_pts,
                              double K, int n_win, unsigned *lo, unsigned *hi) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_win) return;
    int64_t k0 = (int64_t)w * CORE_T;
    int64_t k1 = i64min(k0 + CORE_T, n_pts) - 1;
    double x0 = grid_x(nu_A, step, k0), x1 = grid_x(nu_A, step, k1);
    double a0 = x0 > 0.0 ? x0 / (1.0 + K) : x0, a1 = x1 > 0.0 ? x1 / (1.0 - K) : x1;
    a0 -= 1e-9 * (fabs(x0) + 1.0);
    a1 += 1e-9 * (fabs(x1) + 1.0);
    int64_t a = 0, b = n;
    while (a < b) { int64_t m = a + ((b - a) >> 1); if (nu[m] < a0) a = m + 1; else b = m; }
    lo[w] = (unsigned)a;
    int64_t a2 = a, b2 = n;
    while (a2 < b2) { int64_t m = a2 + ((b2 - a2) >> 1); if (nu[m] <= a1) a2 = m + 1; else b2 = m; }
    hi[w] = (unsigned)(a2 < a ? a : a2);
}

// ---------------------------------------------------------------------------
// kernel table
// ---------------------------------------------------------------------------
typedef void (*GatherFn)(GatherParams);
struct Variant {
    int profile, R, CG;
    GatherFn fn;
    size_t smem;
    bool ext;   // honours the per-(line, condition) options (see line_consts)
    bool tcn;   // the near-pair kernel of the tensor-core sweep (and nothing else)
};

#define XC_VARIANT(P, R, CG) {P, R, CG, k_gather_f32<P, R, CG, true>, SmemLayout<P, R, CG>::total, true, false}
#define XC_VARIANT_PLAIN(P, R, CG) {P, R, CG, k_gather_f32<P, R, CG, false>, SmemLayout<P, R, CG>::total, false, false}
#define XC_VARIANT_TCN(P, R, CG) {P, R, CG, k_gather_f32<P, R, CG, true, true>, SmemLayout<P, R, CG>::total, true, true}
#define XC_VARIANT_PLAIN_TCN(P, R, CG) \
    {P, R, CG, k_gather_f32<P, R, CG, false, true>, SmemLayout<P, R, CG>::total, false, true}
static const Variant kVariants[] = {
    // Voigt w4: the plain hot kernels, and the shapes that carry the per-(line, condition) options
    XC_VARIANT_PLAIN(XC_VOIGT_W4, 4, 16), XC_VARIANT_PLAIN(XC_VOIGT_W4, 2, 32), XC_VARIANT_PLAIN(XC_VOIGT_W4, 4, 8),
    XC_VARIANT_PLAIN(XC_VOIGT_W4, 8, 8),  XC_VARIANT_PLAIN(XC_VOIGT_W4, 8, 4),  XC_VARIANT_PLAIN(XC_VOIGT_W4, 8, 2),
    XC_VARIANT_PLAIN(XC_VOIGT_W4, 8, 1),
    XC_VARIANT(XC_VOIGT_W4, 4, 16), XC_VARIANT(XC_VOIGT_W4, 4, 8), XC_VARIANT(XC_VOIGT_W4, 8, 4),
    XC_VARIANT(XC_VOIGT_W4, 8, 1),
    // the near pairs of the tensor-core sweep (128-point spans: R = 4)
    XC_VARIANT_PLAIN_TCN(XC_VOIGT_W4, 4, 16), XC_VARIANT_PLAIN_TCN(XC_VOIGT_W4, 4, 8),
    XC_VARIANT_TCN(XC_VOIGT_W4, 4, 16), XC_VARIANT_TCN(XC_VOIGT_W4, 4, 8),
    XC_VARIANT(XC_LORENTZ, 4, 16),  XC_VARIANT(XC_LORENTZ, 8, 8),   XC_VARIANT(XC_LORENTZ, 8, 4),
    XC_VARIANT(XC_LORENTZ, 8, 1),
    XC_VARIANT(XC_DOPPLER, 4, 16),  XC_VARIANT(XC_DOPPLER, 8, 4),   XC_VARIANT(XC_DOPPLER, 8, 1),
    XC_VARIANT(XC_VOIGT_GH_SAMPLED, 4, 16), XC_VARIANT(XC_VOIGT_GH_SAMPLED, 8, 4),
    XC_VARIANT(XC_VOIGT_GH_SAMPLED, 8, 1),
    XC_VARIANT(XC_VOIGT_GH_BINNED, 4, 16), XC_VARIANT(XC_VOIGT_GH_BINNED, 8, 4),
    XC_VARIANT(XC_VOIGT_GH_BINNED, 8, 1),
    XC_VARIANT(XC_DOPPLER_BINNED, 4, 16), XC_VARIANT(XC_DOPPLER_BINNED, 8, 4),
    XC_VARIANT(XC_DOPPLER_BINNED, 8, 1),
    XC_VARIANT(XC_LORENTZ_BINNED, 4, 16), XC_VARIANT(XC_LORENTZ_BINNED, 8, 4),
    XC_VARIANT(XC_LORENTZ_BINNED, 8, 1),
    XC_VARIANT(XC_VOIGT_VV, 4, 16), XC_VARIANT(XC_VOIGT_VV, 8, 4),
    XC_VARIANT(XC_VOIGT_VV, 8, 1),
};
static const int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
static_assert(sizeof(kVariants) / sizeof(kVariants[0]) <= 64, "configure_variant tracks at most 64 variants");

// the call uses an option that changes constants per (line, condition)
bool needs_ext(const BatchedArgs &a) {
    return a.opts.quantity != XC_ABSORPTION || a.opts.threshold != XC_THRESHOLD_NONE || a.L.n_broad > 0 ||
           (a.opts.profile == XC_VOIGT_VV && (a.opts.vv_flags & XC_VV_NORMALISE));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

#define BT_TRY(call)                                                                            \
    do {                                                                                        \
        cudaError_t _e = (call);                                                                \
        if (_e == cudaErrorMemoryAllocation) {                                                  \
            cudaGetLastError();                                                                 \
            set_error("device allocation failed: %s", #call);                                   \
            return XC_ENOMEM;                                                                   \
        }                                                                                       \
        if (_e != cudaSuccess) {                                                                \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
            return XC_ECUDA;                                                                    \
        }                                                                                       \
    } while (0)

int num_sms(int dev) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

// Everything the persistent kernel needs, carved out of the state's buffers.
struct Plan {
    const Variant *v = nullptr;
    int W = 0, n_win = 0, n_groups = 0, n_tiles = 0, grid = 0, n_ranges = 0;
    int *n_abs = nullptr, *ka = nullptr, *kb = nullptr;
    float *f = nullptr;
    CParam *cp = nullptr;
    unsigned *lo = nullptr, *hi = nullptr;
    int *order = nullptr, *counter = nullptr;
    GeomStats *gs = nullptr;
    float *gx = nullptr, *gw = nullptr;
    int n_win_core = 0;                         // centre-zone kernel windows (Voigt w4)
    unsigned *core_lo = nullptr, *core_hi = nullptr;
    bool tc = false;                            // far wings on the tensor cores (Voigt w4)
    int n_blk = 0, n_tc_tiles = 0;              // TC_T-point super-blocks, (super-block, group) tiles
    unsigned *blk_lo = nullptr, *blk_hi = nullptr;
    int *tc_counter = nullptr, *tc_status = nullptr;
    float4 *tc_geo = nullptr, *tc_phys = nullptr;
    uint32_t *keep = nullptr;                   // intensity-threshold decisions (with a threshold)
    float *gamma_lc = nullptr;                  // widths per (line, condition) (broadener mixture)
    float *vv_scale = nullptr;                  // VVN factors per (line, condition)
    unsigned *gmax = nullptr;                   // their per-condition maxima (float bits)
};

xc_status make_plan(BatchedState *st, const BatchedArgs &a, const Variant *v, int n_cond_call, Plan *pl,
                    bool tc) {
    const size_t n = a.n_lines;
    pl->v = v;
    pl->tc = tc;
    pl->W = GT * v->R;
    pl->n_win = (int)((a.grid.n + pl->W - 1) / pl->W);
    pl->n_groups = (n_cond_call + v->CG - 1) / v->CG;
    pl->n_tiles = pl->n_win * pl->n_groups;
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    size_t o_n = carve(n * 4), o_f = carve(n * 4), o_ka = carve(n * 4), o_kb = carve(n * 4);
    size_t o_cp = carve((size_t)n_cond_call * sizeof(CParam));
    pl->n_ranges = tc ? pl->n_tiles : pl->n_win;   // near mode: one line range per tile
    size_t o_lo = carve((size_t)pl->n_ranges * 4), o_hi = carve((size_t)pl->n_ranges * 4);
    size_t o_ord = carve((size_t)pl->n_tiles * 4), o_ctr = carve(64), o_gs = carve(64), o_nodes = carve(512);
    pl->n_win_core = (int)((a.grid.n + CORE_T - 1) / CORE_T);
    size_t o_clo = carve((size_t)pl->n_win_core * 4), o_chi = carve((size_t)pl->n_win_core * 4);
    size_t o_blo = 0, o_bhi = 0, o_tcc = 0, o_geo = 0, o_phys = 0, o_keep = 0;
    if (a.opts.threshold != XC_THRESHOLD_NONE) o_keep = carve(n * (size_t)((n_cond_call + 31) / 32) * 4);
    size_t o_glc = 0, o_gmax = 0, o_vvs = 0;
    const bool vvn = a.opts.profile == XC_VOIGT_VV && (a.opts.vv_flags & XC_VV_NORMALISE);
    if (vvn) o_vvs = carve(n * (size_t)n_cond_call * 4);
    if (a.L.n_broad > 0) {
        o_glc = carve(n * (size_t)n_cond_call * 4);
        o_gmax = carve((size_t)n_cond_call * 4);
    }
    if (tc) {
        pl->n_blk = (int)((a.grid.n + TC_T - 1) / TC_T);
        pl->n_tc_tiles = pl->n_blk * ((n_cond_call + TC_N - 1) / TC_N);
        o_blo = carve((size_t)pl->n_blk * 4);
        o_bhi = carve((size_t)pl->n_blk * 4);
        o_tcc = carve(64);
        o_geo = carve(n * sizeof(float4));
        o_phys = carve(n * sizeof(float4));
    }
    BT_TRY(st->tiles.ensure(off));
    char *b = st->tiles.as<char>();
    pl->n_abs = (int *)(b + o_n);
    pl->f = (float *)(b + o_f);
    pl->ka = (int *)(b + o_ka);
    pl->kb = (int *)(b + o_kb);
    pl->cp = (CParam *)(b + o_cp);
    pl->lo = (unsigned *)(b + o_lo);
    pl->hi = (unsigned *)(b + o_hi);
    pl->order = (int *)(b + o_ord);
    pl->counter = (int *)(b + o_ctr);
    pl->gs = (GeomStats *)(b + o_gs);
    pl->gx = (float *)(b + o_nodes);
    pl->gw = pl->gx + 64;
    pl->core_lo = (unsigned *)(b + o_clo);
    pl->core_hi = (unsigned *)(b + o_chi);
    if (a.opts.threshold != XC_THRESHOLD_NONE) pl->keep = (uint32_t *)(b + o_keep);
    if (vvn) pl->vv_scale = (float *)(b + o_vvs);
    if (a.L.n_broad > 0) {
        pl->gamma_lc = (float *)(b + o_glc);
        pl->gmax = (unsigned *)(b + o_gmax);
    }
    if (tc) {
        pl->blk_lo = (unsigned *)(b + o_blo);
        pl->blk_hi = (unsigned *)(b + o_bhi);
        pl->tc_counter = (int *)(b + o_tcc);
        pl->tc_status = pl->tc_counter + 1;
        st->tc_blk_lo = pl->blk_lo;
        st->tc_blk_hi = pl->blk_hi;
        st->tc_n_blk = pl->n_blk;
        st->tc_groups = (n_cond_call + TC_N - 1) / TC_N;
        pl->tc_geo = (float4 *)(b + o_geo);
        pl->tc_phys = (float4 *)(b + o_phys);
        st->tc_status = pl->tc_status;
    }
    return XC_OK;
}

int tc_grid_size(int n_tiles);

// A timing event inside the sweep: while the sweep is captured into a graph it must be an
// external event node (a plain record would become an internal dependency); on a stream
// that is not capturing (the per-condition sweeps of a width-limited cut) the external
// flag is refused, and a plain record is the same thing.
static cudaError_t record_timing_event(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                               : cudaEventRecord(ev, s);
}

// enqueue the whole sweep for conditions [c0, c0 + nc) on the stream
xc_status enqueue(const BatchedArgs &a, const Plan &pl, int c0, int nc, int grid, int max_lines, int64_t *launches,
                  bool per_cond_cut) {
    cudaStream_t s = a.stream;
    const size_t n = a.n_lines;
    unsigned gblocks = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16);
    if (gblocks == 0) gblocks = 1;
    BT_TRY(cudaMemsetAsync(pl.gs, 0, sizeof(GeomStats), s));
    LinesDev L = a.L;   // the lines as the profile kernels see them (threshold decisions, mixture widths)
    if (pl.gamma_lc) {
        BT_TRY(cudaMemsetAsync(pl.gmax, 0, (size_t)nc * 4, s));
        BT_TRY(launch_line_gamma(a.L, n, a.conds_dev + c0, nc, pl.gamma_lc, pl.gmax, s));
        L.gamma_lc = pl.gamma_lc;
        L.gamma_stride = nc;
        *launches += 1;
    }
    k_line_geom<<<gblocks, 256, 0, s>>>(a.L, n, a.grid.nu_A, a.grid.step, a.grid.n, a.opts.cutoff,
                                        per_cond_cut ? a.opts.width_mult : 0.0,
                                        per_cond_cut ? a.conds_dev + c0 : nullptr, pl.n_abs, pl.f, pl.ka, pl.kb,
                                        pl.gs, pl.tc ? pl.tc_geo : nullptr, pl.tc ? pl.tc_phys : nullptr);
    const double vv_split = a.opts.vv_split > 0.0 ? a.opts.vv_split : 4.0;
    const int vv_beta = (a.opts.vv_flags & XC_VV_BETA) ? 1 : 0;
    k_cparams<<<(nc + 63) / 64, 64, 0, s>>>(a.conds_dev + c0, nc, pl.gs, pl.cp, a.grid.step, a.opts.quantity,
                                            pl.gmax, (float)vv_split, vv_beta);
    if (pl.vv_scale) {
        BT_TRY(launch_vv_norm32(L, n, a.conds_dev + c0, nc, a.grid.nu_A, a.grid.step, a.opts.cutoff,
                                per_cond_cut ? a.opts.width_mult : 0.0, vv_split, vv_beta, pl.vv_scale, s));
        L.vv_scale = pl.vv_scale;
        L.vv_stride = nc;
        *launches += 1;
    }
    if (pl.keep) {
        const int words = (nc + 31) / 32;
        BT_TRY(launch_line_keep(a.L, n, a.conds_dev + c0, nc, strength_sel(a.opts), pl.keep, words, s));
        L.keep = pl.keep;
        L.keep_words = words;
        *launches += 1;
    }
    if (pl.tc)
        k_win_ranges_near<<<(pl.n_tiles + 127) / 128, 128, 0, s>>>(a.L.nu, (int64_t)n, a.grid.nu_A, a.grid.step,
                                                                  a.grid.n, pl.W, a.opts.cutoff, pl.n_win,
                                                                  pl.n_groups, pl.v->CG, pl.cp, nc, pl.lo, pl.hi);
    else
        k_win_ranges32<<<(pl.n_win + 127) / 128, 128, 0, s>>>(a.L.nu, (int64_t)n, a.grid.nu_A, a.grid.step,
                                                               a.grid.n, pl.W, a.opts.cutoff, pl.n_win, pl.lo, pl.hi);
    k_rank_tiles<<<(pl.n_tiles + 127) / 128, 128, 0, s>>>(pl.lo, pl.hi, pl.n_win, pl.n_groups, pl.n_tiles,
                                                          pl.order, pl.n_tiles <= 16384, pl.tc);
    *launches += 4;
    if (a.ghx) {
        k_nodes_to_float<<<1, 64, 0, s>>>(a.ghx, a.ghw, a.opts.n_gh, pl.gx, pl.gw);
        *launches += 1;
    }
    BT_TRY(cudaMemsetAsync(pl.counter, 0, sizeof(int), s));
    GatherParams gp;
    gp.L = L;
    gp.n_abs = pl.n_abs;
    gp.f_frac = pl.f;
    gp.ka_abs = pl.ka;
    gp.kb_abs = pl.kb;
    gp.cp = pl.cp;
    gp.win_lo = pl.lo;
    gp.win_hi = pl.hi;
    gp.tile_order = pl.order;
    gp.counter = pl.counter;
    gp.n_tiles = pl.n_tiles;
    gp.n_groups = pl.n_groups;
    gp.n_cond = nc;
    gp.W = pl.W;
    gp.n_pts = a.grid.n;
    gp.h = (float)a.grid.step;
    gp.inv_h = (float)(1.0 / a.grid.step);
    gp.max_lines_per_tile = max_lines;
    gp.ghx = pl.gx;
    gp.ghw = pl.gw;
    gp.ngh = a.opts.n_gh;
    gp.tc_far = pl.tc ? 1 : 0;
    gp.sigma = a.sigma + (size_t)c0 * (size_t)a.grid.n;
    const bool ev = a.timing && a.ev_main0 && max_lines == 0;
    if (ev) BT_TRY(record_timing_event(a.ev_main0, s));
    if (pl.tc && max_lines == 0) {
        // far wings on the tensor cores: first writer of every output of the sweep
        k_win_ranges32<<<(pl.n_blk + 127) / 128, 128, 0, s>>>(a.L.nu, (int64_t)n, a.grid.nu_A, a.grid.step, a.grid.n,
                                                              TC_T, a.opts.cutoff, pl.n_blk, pl.blk_lo, pl.blk_hi);
        BT_TRY(cudaMemsetAsync(pl.tc_counter, 0, 2 * sizeof(int), s));
        TcParams tp;
        tp.geo = pl.tc_geo;
        tp.phys = pl.tc_phys;
        tp.n_T = a.L.n_T;
        tp.cp = pl.cp;
        tp.keep = L.keep;
        tp.keep_words = L.keep_words;
        tp.gamma_lc = L.gamma_lc;
        tp.gamma_stride = L.gamma_stride;
        tp.blk_lo = pl.blk_lo;
        tp.blk_hi = pl.blk_hi;
        tp.counter = pl.tc_counter;
        tp.status = pl.tc_status;
        tp.n_tiles = pl.n_tc_tiles;
        tp.n_groups = (nc + TC_N - 1) / TC_N;
        tp.n_cond = nc;
        tp.n_pts = a.grid.n;
        tp.h = gp.h;
        tp.inv_h = gp.inv_h;
        tp.sigma = gp.sigma;
        if (needs_ext(a))
            k_far_tc<true><<<tc_grid_size(pl.n_tc_tiles), TC_T, TC_SMEM, s>>>(tp);
        else
            k_far_tc<false><<<tc_grid_size(pl.n_tc_tiles), TC_T, TC_SMEM, s>>>(tp);
        if (ev && a.ev_tc1) BT_TRY(record_timing_event(a.ev_tc1, s));
        *launches += 2;
    }
    pl.v->fn<<<grid, GT, pl.v->smem, s>>>(gp);
    if (ev) BT_TRY(record_timing_event(a.ev_main1, s));
    *launches += 1;
    if (a.opts.profile == XC_VOIGT_W4 && max_lines == 0) {
        // centre zone: |x| + y < 15, |nu - x| < 18.02 alpha <= K nu
        double amax = 0.0;
        for (int c = 0; c < nc; ++c)
            amax = std::max(amax, alpha_coef(a.conds_host[c0 + c].T, a.conds_host[c0 + c].mass_da));
        const double K = 18.05 * amax;
        k_core_ranges<<<(pl.n_win_core + 127) / 128, 128, 0, s>>>(a.L.nu, (int64_t)n, a.grid.nu_A, a.grid.step,
                                                                   a.grid.n, K, pl.n_win_core, pl.core_lo,
                                                                   pl.core_hi);
        CoreParams cp;
        cp.L = L;
        cp.n_abs = pl.n_abs;
        cp.f_frac = pl.f;
        cp.ka_abs = pl.ka;
        cp.kb_abs = pl.kb;
        cp.cp = pl.cp;
        cp.win_lo = pl.core_lo;
        cp.win_hi = pl.core_hi;
        cp.n_cond = nc;
        cp.n_pts = a.grid.n;
        cp.h = gp.h;
        cp.inv_h = gp.inv_h;
        cp.sigma = gp.sigma;
        dim3 cg(pl.n_win_core, (nc + CORE_CG - 1) / CORE_CG);
        k_core_w4_f32<<<cg, CORE_T, 0, s>>>(cp);
        *launches += 2;
    }
    if (ev) BT_TRY(record_timing_event(a.ev_core1, s));
    BT_TRY(cudaGetLastError());
    return XC_OK;
}

bool use_tc(const BatchedArgs &a, int nc);

std::string shape_key(const BatchedArgs &a, int nc) {
    char buf[384];
    snprintf(buf, sizeof(buf), "p%d n%zu c%d g%lld/%.17g/%.17g cut%.17g wm%.17g gh%d f%d tc%d q%d t%d/%.17g/%.17g/%.17g",
             a.opts.profile, a.n_lines, nc, (long long)a.grid.n, a.grid.nu_A, a.grid.step, a.opts.cutoff,
             a.opts.width_mult, a.opts.n_gh, a.opts.flags, use_tc(a, nc) ? 1 : 0, a.opts.quantity,
             a.opts.threshold, a.opts.I_cut, a.opts.nu_crit, a.opts.I_crit);
    if (a.opts.profile == XC_VOIGT_VV) {
        char vb[64];
        snprintf(vb, sizeof(vb), " vv%.17g/%d", a.opts.vv_split, a.opts.vv_flags);
        std::string r = std::string(buf) + vb;
        if (a.L.n_broad > 0) {
            snprintf(vb, sizeof(vb), " b%d@%p", a.L.n_broad, (const void *)a.L.bgam);
            r += vb;
        }
        return r;
    }
    if (a.L.n_broad > 0) {
        char bb[64];
        snprintf(bb, sizeof(bb), " b%d@%p", a.L.n_broad, (const void *)a.L.bgam);
        return std::string(buf) + bb;
    }
    return buf;
}

// A kernel attribute set by cudaFuncSetAttribute holds for the current device's context
// only, so the "already configured" flags are kept per device (and per variant), under a
// lock because calls may come from several host threads.
constexpr int kMaxDevices = 64;
static std::mutex g_attr_mu;

xc_status configure_variant(const Variant *v, int dev) {
    static bool done[kMaxDevices][64] = {};
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d this library tracks", dev, kMaxDevices);
        return XC_EINVAL;
    }
    const int idx = (int)(v - kVariants);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (done[dev][idx]) return XC_OK;
    BT_TRY(cudaFuncSetAttribute((const void *)v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem));
    done[dev][idx] = true;
    return XC_OK;
}

// far-wing kernel residency per SM and its diagnosis, per device (-1: not yet set up)
static int g_tc_per_sm[kMaxDevices] = {};
static bool g_tc_ready[kMaxDevices] = {};
static char g_tc_diag[kMaxDevices][160] = {};

int tc_per_sm(int dev) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    return (dev >= 0 && dev < kMaxDevices && g_tc_ready[dev]) ? g_tc_per_sm[dev] : 0;
}

std::string tc_diag(int dev) {
    std::lock_guard<std::mutex> lk(g_attr_mu);
    return (dev >= 0 && dev < kMaxDevices && g_tc_ready[dev]) ? std::string(g_tc_diag[dev]) : std::string();
}

int tc_grid_size(int n_tiles) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;   // rejected earlier by configure_variant
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (!g_tc_ready[dev]) {
        int ps = 0;
        cudaError_t e1 = cudaFuncSetAttribute((const void *)k_far_tc<false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        if (e1 == cudaSuccess)
            e1 = cudaFuncSetAttribute((const void *)k_far_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TC_SMEM);
        cudaError_t e2 = e1 == cudaSuccess ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                                 &ps, (const void *)k_far_tc<false>, TC_T, TC_SMEM)
                                           : e1;
        // The occupancy query answers 1 for this kernel (it does not model tensor-memory
        // allocation); residency is bounded by shared memory (TC_SMEM admits 2 CTAs), by
        // registers, and by the 512 TMEM columns of an SM (2 x 256).  Extra CTAs would
        // only wait: the work queue is shared.
        cudaFuncAttributes fa;
        int smem_sm = 0;
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        int by_regs = 1, by_smem = 1, regs = 0;
        if (cudaFuncGetAttributes(&fa, (const void *)k_far_tc<false>) == cudaSuccess) regs = fa.numRegs;
        if (cudaFuncGetAttributes(&fa, (const void *)k_far_tc<true>) == cudaSuccess) regs = std::max(regs, fa.numRegs);
        if (regs > 0) by_regs = 65536 / (regs * TC_T);
        if (smem_sm > 0) by_smem = smem_sm / (int)(TC_SMEM + 1024);
        const int mine = std::max(1, std::min((int)(512 / TC_COLS), std::min(by_regs, by_smem)));
        snprintf(g_tc_diag[dev], sizeof(g_tc_diag[dev]), "query %d (%s), registers %d, shared memory %d", ps,
                 cudaGetErrorString(e2), by_regs, by_smem);
        cudaGetLastError();
        g_tc_per_sm[dev] = mine;
        g_tc_ready[dev] = true;
    }
    return std::max(1, std::min(num_sms(dev) * g_tc_per_sm[dev], n_tiles));
}

int grid_size(const Variant *v, int dev, int n_tiles) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)v->fn, GT, v->smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    int g = num_sms(dev) * per_sm;
    return std::max(1, std::min(g, n_tiles));
}

// Autotune: time each candidate variant on a probe (every tile, first 4096 lines)
// and predict the full run from the measured time per (tile line x condition);
// the prediction includes the wave quantisation of the tile count.
// far wings of the Voigt w4 sweep on the tensor cores: many conditions (the MMA's N is
// 32, so a handful of conditions would waste it), one fixed cut, grids of < 2^30 points
bool use_tc(const BatchedArgs &a, int nc) {
    return a.allow_tc && a.opts.profile == XC_VOIGT_W4 && a.opts.width_mult <= 0.0 && nc >= 16 &&
           !(a.opts.flags & XC_OPT_NO_TENSOR_CORES) && a.grid.n < ((int64_t)1 << 23);
}

std::string tuned_key(const BatchedState *st, const BatchedArgs &a, int nc) {
    std::string key = shape_key(a, nc);
    if (st->force_R > 0) {
        char fb[48];
        snprintf(fb, sizeof(fb), " fixed R%d CG%d", st->force_R, st->force_CG);
        key += fb;
    }
    return key;
}

xc_status autotune(BatchedState *st, const BatchedArgs &a, int nc, TileCfg *out, int64_t *launches) {
    const std::string key = tuned_key(st, a, nc);
    const bool tc = use_tc(a, nc);
    if (tc) tc_grid_size(1);   // kernel attributes set outside any graph capture
    auto it = st->tuned.find(key);
    if (it != st->tuned.end()) {
        *out = it->second;
        return XC_OK;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int> cands;
    // the shape heuristics first; if they leave no variant of this profile (e.g. 5 to 7
    // conditions where only groups of 1, 4 and 16 exist), every admissible shape
    for (int pass = 0; pass < 2 && cands.empty(); ++pass) {
        for (int i = 0; i < kNumVariants; ++i) {
            const Variant &v = kVariants[i];
            if (v.profile != a.opts.profile) continue;
            if (v.profile == XC_VOIGT_W4 && v.ext != needs_ext(a)) continue;
            if (a.opts.width_mult > 0.0 && v.CG != 1) continue;  // per-condition cut: one condition per tile
            if (pass == 0 && a.opts.width_mult <= 0.0 && st->force_R == 0) {
                if (v.CG > 1 && v.CG > 2 * nc) continue;          // no more than half the group padded
                if (v.CG < std::min(nc, 8)) continue;              // enough conditions share each staged line
            }
            if (v.tcn != tc) continue;     // with the far wings on the tensor cores: the near-pair kernels
            if (st->force_R > 0 && (v.R != st->force_R || v.CG != st->force_CG)) continue;
            cands.push_back(i);
        }
    }
    if (cands.empty()) {
        set_error("no FP32 kernel variant for profile %d", a.opts.profile);
        return XC_EUNSUPPORTED;
    }
    TileCfg best;
    best.variant = cands[0];
    best.points = GT * kVariants[cands[0]].R;
    best.cgroup = kVariants[cands[0]].CG;
    best.ms = 0.f;
    if (cands.size() > 1) {
        cudaEvent_t e0, e1;
        BT_TRY(cudaEventCreate(&e0));
        BT_TRY(cudaEventCreate(&e1));
        float best_pred = 1e30f;
        for (int vi : cands) {
            const Variant *v = &kVariants[vi];
            xc_status s = configure_variant(v, dev);
            if (s) return s;
            Plan pl;
            int ncv = a.opts.width_mult > 0.0 ? 1 : nc;
            if ((s = make_plan(st, a, v, ncv, &pl, tc))) return s;
            int grid = grid_size(v, dev, pl.n_tiles);
            const int probe_lines = 4096;
            if ((s = enqueue(a, pl, 0, ncv, grid, probe_lines, launches, a.opts.width_mult > 0.0))) return s;
            BT_TRY(cudaEventRecord(e0, a.stream));
            if ((s = enqueue(a, pl, 0, ncv, grid, probe_lines, launches, a.opts.width_mult > 0.0))) return s;
            BT_TRY(cudaEventRecord(e1, a.stream));
            BT_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            BT_TRY(cudaEventElapsedTime(&ms, e0, e1));
            // measured: all tiles, <= probe_lines lines each. Predict for the full line count:
            std::vector<unsigned> lo(pl.n_ranges), hi(pl.n_ranges);
            BT_TRY(cudaMemcpy(lo.data(), pl.lo, pl.n_ranges * 4, cudaMemcpyDeviceToHost));
            BT_TRY(cudaMemcpy(hi.data(), pl.hi, pl.n_ranges * 4, cudaMemcpyDeviceToHost));
            double probe_max = 0.0, full_work = 0.0, max_tile = 0.0, probe_sum = 0.0;
            for (int w = 0; w < pl.n_ranges; ++w) {
                double cntl = (double)(hi[w] - lo[w]);
                double pc = std::min(cntl, (double)probe_lines);
                probe_sum += pc;
                probe_max = std::max(probe_max, pc);
                full_work += cntl;
                max_tile = std::max(max_tile, cntl);
            }
            // time per tile-line for one slot, from waves x mean probe tile
            double waves = std::ceil((double)pl.n_tiles / grid);
            double probe_avg = probe_sum / pl.n_ranges;
            double t_line = (probe_avg > 0 && waves > 0) ? ms / (waves * probe_avg) : 0.0;
            double avg_tile = full_work / pl.n_ranges;
            double pred = t_line * std::max(waves * avg_tile, max_tile);
            {
                char lb[160];
                snprintf(lb, sizeof(lb), "[R=%d CG=%d W=%d grid=%d probe %.3f ms pred %.1f ms] ", v->R, v->CG,
                         pl.W, grid, ms, pred);
                st->tune_log[key] += lb;
            }
            if (pred < best_pred) {
                best_pred = (float)pred;
                best.variant = vi;
                best.points = pl.W;
                best.cgroup = v->CG;
                best.ms = (float)pred;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    st->tuned[key] = best;
    *out = best;
    return XC_OK;
}

}  // namespace

xc_status batched_run(BatchedState *st, const BatchedArgs &a, int64_t *launches) {
    if (a.grid.n >= ((int64_t)1 << 31) - (1 << 20)) {
        set_error("the FP32 path needs fewer than 2^31 grid points");
        return XC_EINVAL;
    }
    // the status word lives in the plan's scratch, which a later plan may reallocate:
    // it is valid only for the run that set it
    st->tc_status = nullptr;
    st->tc_blk_lo = st->tc_blk_hi = nullptr;
    st->tc_n_blk = st->tc_groups = 0;
    if (a.n_lines == 0 || a.n_cond == 0 || a.grid.n == 0) return XC_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    TileCfg cfg;
    xc_status s = autotune(st, a, a.n_cond, &cfg, launches);
    if (s) return s;
    const Variant *v = &kVariants[cfg.variant];
    if ((s = configure_variant(v, dev))) return s;
    {
        char lb[256];
        if (use_tc(a, a.n_cond)) {
            const std::string dg = tc_diag(dev);
            snprintf(lb, sizeof(lb), "profile %d R=%d CG=%d W=%d points, far wings on tensor cores (%d CTAs/SM%s%s); ",
                     v->profile, v->R, v->CG, GT * v->R, tc_per_sm(dev), dg.empty() ? "" : ", ", dg.c_str());
        }
        else
            snprintf(lb, sizeof(lb), "profile %d R=%d CG=%d W=%d points; ", v->profile, v->R, v->CG, GT * v->R);
        st->last_tuning = std::string(lb) + st->tune_log[tuned_key(st, a, a.n_cond)];
    }
    const bool per_cond = a.opts.width_mult > 0.0;
    if (per_cond) {
        // per-condition cut: one launch sequence per condition
        if (a.timing) cudaEventRecord(a.ev_begin, a.stream);
        for (int c = 0; c < a.n_cond; ++c) {
            Plan pl;
            if ((s = make_plan(st, a, v, 1, &pl, false))) return s;
            if ((s = enqueue(a, pl, c, 1, grid_size(v, dev, pl.n_tiles), 0, launches, true))) return s;
        }
        if (a.timing) cudaEventRecord(a.ev_end, a.stream);
        return XC_OK;
    }
    Plan pl;
    if ((s = make_plan(st, a, v, a.n_cond, &pl, use_tc(a, a.n_cond)))) return s;
    const int grid = grid_size(v, dev, pl.n_tiles);
    // graph cache: the sweep (geometry, constants, ranges, tile ranking, counter
    // reset, persistent kernel) is captured once per shape and buffer set, then replayed
    char kb[512];
    snprintf(kb, sizeof(kb), "%s v%d t%d L%p C%p S%p T%p", shape_key(a, a.n_cond).c_str(), cfg.variant,
             a.timing ? 1 : 0,
             (const void *)a.L.nu, (const void *)a.conds_dev, (void *)a.sigma, (void *)st->tiles.p);
    std::string gkey = kb;
    auto it = st->graphs.find(gkey);
    if (it == st->graphs.end()) {
        GraphEntry ge;
        cudaStream_t cs;
        BT_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        BatchedArgs ac = a;
        ac.stream = cs;
        int64_t nl = 0;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            BT_TRY(e);
        }
        xc_status se = enqueue(ac, pl, 0, a.n_cond, grid, 0, &nl, false);
        e = cudaStreamEndCapture(cs, &ge.graph);
        cudaStreamDestroy(cs);
        if (se) return se;
        BT_TRY(e);
        BT_TRY(cudaGraphInstantiate(&ge.exec, ge.graph, 0));
        it = st->graphs.emplace(gkey, ge).first;
    }
    if (a.timing) cudaEventRecord(a.ev_begin, a.stream);
    BT_TRY(cudaGraphLaunch(it->second.exec, a.stream));
    if (a.timing) cudaEventRecord(a.ev_end, a.stream);
    *launches += a.ghx ? 6 : 5;
    return XC_OK;
}

xc_status batched_check(BatchedState *st) {
    if (!st->tc_status) return XC_OK;
    int v = 0;
    if (cudaMemcpy(&v, st->tc_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("reading the tensor-core kernel status failed: %s", cudaGetErrorString(cudaGetLastError()));
        return XC_ECUDA;
    }
    if (v) {
        set_error("tensor-core far-wing kernel: an MMA completion wait ran out; results are not valid");
        return XC_ETIMEOUT;
    }
    return XC_OK;
}

int64_t batched_tc_mma_count(BatchedState *st) {
    if (!st->tc_blk_lo || st->tc_n_blk <= 0) return 0;
    std::vector<unsigned> lo(st->tc_n_blk), hi(st->tc_n_blk);
    if (cudaMemcpy(lo.data(), st->tc_blk_lo, lo.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hi.data(), st->tc_blk_hi, hi.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    int64_t chunks = 0;
    for (int i = 0; i < st->tc_n_blk; ++i) chunks += (int64_t)((hi[i] - lo[i] + TC_L - 1) / TC_L);
    // per chunk and 128-point block: TC_MMAS MMAs (M = 128, N = 32, K = 8)
    return chunks * st->tc_groups * TC_BLK * TC_MMAS;
}

xc_status batched_count_far(BatchedState *st, const BatchedArgs &a, int64_t *count) {
    *count = 0;
    const int nc = a.n_cond;
    if (a.n_lines == 0 || nc == 0 || a.grid.n == 0 || !use_tc(a, nc)) return XC_OK;
    const Variant *v = nullptr;
    for (int i = 0; i < kNumVariants && !v; ++i)
        if (kVariants[i].profile == XC_VOIGT_W4 && kVariants[i].R == 4) v = &kVariants[i];
    Plan pl;
    xc_status s = make_plan(st, a, v, nc, &pl, true);
    if (s) return s;
    cudaStream_t cs = a.stream;
    const size_t n = a.n_lines;
    unsigned gblocks = (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 16));
    BT_TRY(cudaMemsetAsync(pl.gs, 0, sizeof(GeomStats), cs));
    if (pl.gamma_lc) {
        BT_TRY(cudaMemsetAsync(pl.gmax, 0, (size_t)nc * 4, cs));
        BT_TRY(launch_line_gamma(a.L, n, a.conds_dev, nc, pl.gamma_lc, pl.gmax, cs));
    }
    k_line_geom<<<gblocks, 256, 0, cs>>>(a.L, n, a.grid.nu_A, a.grid.step, a.grid.n, a.opts.cutoff, 0.0, nullptr,
                                         pl.n_abs, pl.f, pl.ka, pl.kb, pl.gs, pl.tc_geo, pl.tc_phys);
    k_cparams<<<(nc + 63) / 64, 64, 0, cs>>>(a.conds_dev, nc, pl.gs, pl.cp, a.grid.step, a.opts.quantity, pl.gmax,
                                             4.f, 0);
    unsigned long long *dcount = reinterpret_cast<unsigned long long *>(pl.tc_counter + 2);   // 8-byte aligned
    BT_TRY(cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), cs));
    int dev = 0;
    cudaGetDevice(&dev);
    k_far_count<<<num_sms(dev) * 8, 256, 0, cs>>>(pl.tc_geo, pl.tc_phys, a.L.n_T, pl.cp, nc, pl.gamma_lc, nc, n,
                                                (float)(1.0 / a.grid.step), dcount);
    BT_TRY(cudaGetLastError());
    unsigned long long hc = 0;
    BT_TRY(cudaMemcpyAsync(&hc, dcount, sizeof(hc), cudaMemcpyDeviceToHost, cs));
    BT_TRY(cudaStreamSynchronize(cs));
    *count = (int64_t)hc;
    return XC_OK;
}

void batched_invalidate(BatchedState *st) {
    for (auto &kv : st->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
    }
    st->graphs.clear();
    st->tuned.clear();
}

void batched_release(BatchedState *st) {
    batched_invalidate(st);
    st->tiles.release();
    st->cparams.release();
    st->counter.release();
    st->vjp_buf.release();
    st->gsig32.release();
    st->staging.release();
}

// ---------------------------------------------------------------------------
// Allocation-free variant (xc_cross_section_batched_static).
//
// Some callers cannot allocate device memory while they run: code that executes
// inside another framework's memory pool or a pre-planned memory budget, real-time
// loops that must not call cudaMalloc/cudaFree (both can synchronise the device),
// or hosts that hand this library nothing but the buffers they already own.  For
// them, the per-call scratch of the FP32 batched kernel (per-line grid geometry,
// per-condition constants, window ranges, tile order, work counter) lives in the
// fixed-size array below, which every GPU that loads the library holds until the
// process exits.  Host code must not take the array's address directly (the name
// is only a host-side stand-in); it asks the runtime for the device address once
// per device and passes that pointer to the kernels.
// ---------------------------------------------------------------------------
constexpr size_t kStaticMaxLines = (size_t)1 << 20;      // 1,048,576 lines
constexpr int kStaticMaxCond = 64;
constexpr int64_t kStaticMaxPoints = (int64_t)1 << 22;   // 4,194,304 grid points
constexpr int kStaticR = 4;                               // tile shape used by this entry point
constexpr int kStaticMinW = GT * kStaticR;
constexpr int kStaticMaxWin = (int)((kStaticMaxPoints + kStaticMinW - 1) / kStaticMinW);
constexpr int kStaticMaxTiles = kStaticMaxWin * kStaticMaxCond;
constexpr int kStaticMaxCoreWin = (int)((kStaticMaxPoints + CORE_T - 1) / CORE_T);

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct StaticLayout {
    static constexpr size_t o_n = 0;
    static constexpr size_t o_f = o_n + al256(kStaticMaxLines * 4);
    static constexpr size_t o_ka = o_f + al256(kStaticMaxLines * 4);
    static constexpr size_t o_kb = o_ka + al256(kStaticMaxLines * 4);
    static constexpr size_t o_cp = o_kb + al256(kStaticMaxLines * 4);
    static constexpr size_t o_cd = o_cp + al256(kStaticMaxCond * sizeof(CParam));
    static constexpr size_t o_q = o_cd + al256(kStaticMaxCond * sizeof(CondDev));
    static constexpr size_t o_lo = o_q + al256(kStaticMaxCond * 3 * sizeof(double) + kStaticMaxCond * sizeof(int));
    static constexpr size_t o_hi = o_lo + al256((size_t)kStaticMaxWin * 4);
    static constexpr size_t o_ord = o_hi + al256((size_t)kStaticMaxWin * 4);
    static constexpr size_t o_clo = o_ord + al256((size_t)kStaticMaxTiles * 4);
    static constexpr size_t o_chi = o_clo + al256((size_t)kStaticMaxCoreWin * 4);
    static constexpr size_t o_ctr = o_chi + al256((size_t)kStaticMaxCoreWin * 4);
    static constexpr size_t o_gs = o_ctr + 256;
    static constexpr size_t o_nodes = o_gs + 256;
    static constexpr size_t o_flag = o_nodes + 512;
    static constexpr size_t total = o_flag + 256;
};

static __device__ __align__(256) unsigned char g_static_scratch[StaticLayout::total];

// per device: the device address of g_static_scratch, looked up once
static std::mutex g_static_mu;
static void *g_static_ptr[256] = {};

__global__ void k_static_fill_conds(CondDev *c, int n, const int *tix, const double *Q, const double *dQ) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tix[i] < 0) return;
    c[i].Q = Q[tix[i]];
    c[i].dQdT = dQ[tix[i]];
}

__global__ void k_static_check_lines(LinesDev L, size_t n, int *flag) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double v = L.nu[i];
        bool ok = isfinite(v) && v > 0.0 && isfinite(L.elower[i]) && L.elower[i] >= 0.f && L.A[i] >= 0.f &&
                  L.gamma_ref[i] >= 0.f && isfinite(L.n_T[i]) && L.g_up[i] >= 0;
        if (!ok) atomicOr(flag, 1);
        if (i + 1 < n && !(v <= L.nu[i + 1])) atomicOr(flag, 2);
    }
}

}  // namespace xc

extern "C" xc_status xc_cross_section_batched_static(const xc_lines *lines, size_t n_lines, const double *E,
                                                     const int32_t *g, size_t n_states, const xc_condition *conds,
                                                     size_t n_cond, const xc_grid *grid, const xc_opts *opts,
                                                     double *sigma_out, void *stream) {
    using namespace xc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!lines || !conds || !grid || !opts || (!sigma_out && n_cond && grid->n)) {
        set_error("NULL argument");
        return XC_EINVAL;
    }
    if (lines->mem != XC_MEM_DEVICE) { set_error("lines must be device arrays (sorted by nu)"); return XC_EINVAL; }
    if (n_lines > kStaticMaxLines) {
        set_error("n_lines = %zu exceeds the static scratch limit of %zu lines", n_lines, kStaticMaxLines);
        return XC_EINVAL;
    }
    if (n_cond > (size_t)kStaticMaxCond) {
        set_error("n_cond = %zu exceeds the static scratch limit of %d conditions", n_cond, kStaticMaxCond);
        return XC_EINVAL;
    }
    if (grid->n < 0 || grid->n > kStaticMaxPoints) {
        set_error("grid n = %lld exceeds the static scratch limit of %lld points", (long long)grid->n,
                  (long long)kStaticMaxPoints);
        return XC_EINVAL;
    }
    if (!(grid->step > 0.0) || !isfinite(grid->step) || !isfinite(grid->nu_A)) { set_error("bad grid"); return XC_EINVAL; }
    if (opts->precision != XC_FP32 || opts->width_mult != 0.0) {
        set_error("the allocation-free entry point computes the FP32 kernel with a fixed cut");
        return XC_EUNSUPPORTED;
    }
    if (opts->profile < XC_DOPPLER || opts->profile > XC_VOIGT_VV || !(opts->cutoff > 0.0)) {
        set_error("bad opts");
        return XC_EINVAL;
    }
    if (opts->profile == XC_VOIGT_GH_BINNED || opts->profile == XC_VOIGT_GH_SAMPLED) {
        set_error("Gauss-Hermite profiles need node tables: use xc_cross_section_batched");
        return XC_EUNSUPPORTED;
    }
    if (opts->profile == XC_DOPPLER_BINNED || opts->profile == XC_LORENTZ_BINNED) {
        set_error("binned profiles: use xc_cross_section_batched");
        return XC_EUNSUPPORTED;
    }
    if (opts->quantity != XC_ABSORPTION || opts->threshold != XC_THRESHOLD_NONE) {
        set_error("emission and intensity thresholds: use xc_cross_section_batched");
        return XC_EUNSUPPORTED;
    }
    if (opts->profile == XC_VOIGT_VV) {
        set_error("the Vectorized Voigt: use xc_cross_section_batched");
        return XC_EUNSUPPORTED;
    }
    for (size_t i = 0; i < n_cond; ++i) {
        const xc_condition &c = conds[i];
        if (!(c.T > 0.0) || !(c.P >= 0.0) || !(c.mass_da > 0.0) || !(c.T_ref > 0.0) || !(c.P_ref > 0.0)) {
            set_error("condition %zu: bad T/P/mass/reference values", i);
            return XC_EINVAL;
        }
        if (c.Q <= 0.0 && (!E || !g || !n_states)) {
            set_error("condition %zu: Q <= 0 needs a device state list (E, g)", i);
            return XC_EINVAL;
        }
    }
    if (n_cond == 0 || grid->n == 0) return XC_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) { set_error("cudaGetDevice failed"); return XC_ECUDA; }
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p) {
                set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
                cudaGetLastError();
                return XC_ECUDA;
            }
            g_static_ptr[dev] = p;
        }
        base = static_cast<char *>(g_static_ptr[dev]);
    }
    const int nc = (int)n_cond;
    const Variant *v = nullptr;
    int want_cg = nc >= 16 ? 16 : (nc >= 8 ? 8 : (nc >= 4 ? 4 : 1));
    for (int i = 0; i < kNumVariants && !v; ++i)
        if (kVariants[i].profile == opts->profile && kVariants[i].CG == want_cg && !kVariants[i].tcn &&
            (kVariants[i].profile != XC_VOIGT_W4 || !kVariants[i].ext))   // no per-(line, condition) options here
            v = &kVariants[i];
    for (int i = 0; i < kNumVariants && !v; ++i)  // profiles compiled with fewer group sizes
        if (kVariants[i].profile == opts->profile && kVariants[i].CG <= want_cg && !kVariants[i].tcn) v = &kVariants[i];
    if (!v) { set_error("no kernel variant for this profile"); return XC_EUNSUPPORTED; }
    xc_status st = configure_variant(v, dev);
    if (st) return st;
    // carve the static scratch
    Plan pl;
    pl.v = v;
    pl.W = GT * v->R;
    pl.n_win = (int)((grid->n + pl.W - 1) / pl.W);
    pl.n_groups = (nc + v->CG - 1) / v->CG;
    pl.n_tiles = pl.n_win * pl.n_groups;
    if (pl.n_win > kStaticMaxWin || pl.n_tiles > kStaticMaxTiles) { set_error("tile table too large"); return XC_EINVAL; }
    pl.n_abs = (int *)(base + StaticLayout::o_n);
    pl.f = (float *)(base + StaticLayout::o_f);
    pl.ka = (int *)(base + StaticLayout::o_ka);
    pl.kb = (int *)(base + StaticLayout::o_kb);
    pl.cp = (CParam *)(base + StaticLayout::o_cp);
    pl.lo = (unsigned *)(base + StaticLayout::o_lo);
    pl.hi = (unsigned *)(base + StaticLayout::o_hi);
    pl.order = (int *)(base + StaticLayout::o_ord);
    pl.counter = (int *)(base + StaticLayout::o_ctr);
    pl.gs = (GeomStats *)(base + StaticLayout::o_gs);
    pl.gx = (float *)(base + StaticLayout::o_nodes);
    pl.gw = pl.gx + 64;
    pl.n_win_core = (int)((grid->n + CORE_T - 1) / CORE_T);
    pl.core_lo = (unsigned *)(base + StaticLayout::o_clo);
    pl.core_hi = (unsigned *)(base + StaticLayout::o_chi);
    CondDev *dc = (CondDev *)(base + StaticLayout::o_cd);
    double *qT = (double *)(base + StaticLayout::o_q), *qQ = qT + kStaticMaxCond, *qD = qQ + kStaticMaxCond;
    int *tix_d = (int *)(qD + kStaticMaxCond);
    int *flag = (int *)(base + StaticLayout::o_flag);
    LinesDev L{lines->nu, lines->elower, lines->A, lines->gamma_ref, lines->n_T, lines->g_up, lines->j_lo};
    // conditions: host -> static scratch, Q(T) for those that need it
    CondDev hc[kStaticMaxCond];
    double uT[kStaticMaxCond];
    int tix[kStaticMaxCond];
    int nT = 0;
    for (int i = 0; i < nc; ++i) {
        const xc_condition &c = conds[i];
        hc[i] = CondDev{c.T, c.P, c.Q, c.dQdT, c.mass_da, c.T_ref, c.P_ref, c.gamma_scale, c.n_shift, c.abundance};
        tix[i] = -1;
        if (c.Q <= 0.0) {
            int j = 0;
            while (j < nT && uT[j] != c.T) ++j;
            if (j == nT) uT[nT++] = c.T;
            tix[i] = j;
        }
    }
#define ST_TRY(call)                                                                             \
    do {                                                                                         \
        cudaError_t _e = (call);                                                                 \
        if (_e != cudaSuccess) {                                                                 \
            set_error("%s failed: %s", #call, cudaGetErrorString(_e));                            \
            return XC_ECUDA;                                                                     \
        }                                                                                        \
    } while (0)
    ST_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    if (n_lines) {
        k_static_check_lines<<<(unsigned)std::max<size_t>(1, std::min<size_t>((n_lines + 255) / 256, 152 * 8)), 256, 0, s>>>(
            L, n_lines, flag);
    }
    int hflag = 0;
    ST_TRY(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    ST_TRY(cudaMemcpyAsync(dc, hc, nc * sizeof(CondDev), cudaMemcpyHostToDevice, s));
    ST_TRY(cudaStreamSynchronize(s));  // host arrays above are on this stack frame
    if (hflag & 1) { set_error("invalid line values"); return XC_EINVAL; }
    if (hflag & 2) { set_error("lines must be sorted by nu"); return XC_EINVAL; }
    if (nT) {
        ST_TRY(cudaMemcpyAsync(qT, uT, nT * sizeof(double), cudaMemcpyHostToDevice, s));
        ST_TRY(cudaMemcpyAsync(tix_d, tix, nc * sizeof(int), cudaMemcpyHostToDevice, s));
        ST_TRY(launch_partition_function(E, g, n_states, qT, nT, qQ, qD, s));
        k_static_fill_conds<<<1, 64, 0, s>>>(dc, nc, tix_d, qQ, qD);
        ST_TRY(cudaStreamSynchronize(s));  // uT and tix live on this stack frame
    }
    if (n_lines == 0) {
        ST_TRY(cudaMemsetAsync(sigma_out, 0, (size_t)nc * grid->n * sizeof(double), s));
        return XC_OK;
    }
    BatchedArgs a;
    a.L = L;
    a.n_lines = n_lines;
    a.conds_dev = dc;
    a.conds_host = conds;
    a.n_cond = nc;
    a.grid = *grid;
    a.opts = *opts;
    a.sigma = sigma_out;
    a.stream = s;
    int64_t nl = 0;
    st = enqueue(a, pl, 0, nc, grid_size(v, dev, pl.n_tiles), 0, &nl, false);
#undef ST_TRY
    return st;
}
