// xc_lines.cu -- per-line and per-state kernels:
//   Q(T) and dQ/dT (Eq. e:pf) in FP64, one CTA per temperature;
//   FP64 line parameters I (Eq. e:int), alpha_D (Eq. e:alphaD), gamma_L (Eq. e:gamma_L);
//   window -> line range by binary search on the sorted wavenumbers;
//   exact count of (line, grid point) pairs inside the cutoff;
//   Gauss-Hermite nodes and weights on the device.
#include <math.h>

#include "xc_internal.cuh"

namespace xc {

// ---------------------------------------------------------------------------
// Q(T) = sum_n g_n exp(-c2 E_n / T) and dQ/dT = sum_n g_n (c2 E_n / T^2) exp(-c2 E_n / T)
// One CTA per temperature; fixed-order tree reduction (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_partition_function(const double *__restrict__ E,
                                                            const int32_t *__restrict__ g, size_t n,
                                                            const double *__restrict__ T, double *Q,
                                                            double *dQ) {
    __shared__ double sq[256], sd[256];
    const double t = T[blockIdx.x];
    const double a = kC2 / t;
    double q = 0.0, d = 0.0;
    for (size_t i = threadIdx.x; i < n; i += 256) {
        double b = exp(-a * E[i]);
        double gb = (double)g[i] * b;
        q += gb;
        d += gb * (a * E[i] / t);
    }
    sq[threadIdx.x] = q;
    sd[threadIdx.x] = d;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sq[threadIdx.x] += sq[threadIdx.x + s];
            sd[threadIdx.x] += sd[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        Q[blockIdx.x] = sq[0];
        if (dQ) dQ[blockIdx.x] = sd[0];
    }
}

cudaError_t launch_partition_function(const double *E, const int32_t *g, size_t n, const double *T, int nT,
                                      double *Q, double *dQ, cudaStream_t s) {
    if (nT <= 0) return cudaSuccess;
    k_partition_function<<<nT, 256, 0, s>>>(E, g, n, T, Q, dQ);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 line parameters for one condition (fused: reads nu, E'', A, g', gamma_ref, n
// once; writes I, alpha, gamma and the per-line cut)
// ---------------------------------------------------------------------------
__device__ inline double line_cut(int cut_mode, double cutoff, double width_mult, double al, double ga) {
    if (cut_mode) {
        double w = width_mult * fmax(al, ga);
        return fmin(w, cutoff);
    }
    return cutoff;
}

__global__ void __launch_bounds__(256) k_line_params64(LinesDev L, size_t n, const CondDev *__restrict__ cd,
                                                       int cut_mode, double cutoff, double width_mult,
                                                       double *I, double *alpha, double *gamma, double *cut,
                                                       StrengthSel sel) {
    const CondDev c = *cd;
    const double inv_T = 1.0 / c.T;
    const double acoef = alpha_coef(c.T, c.mass_da);
    const double lnTr = log(c.T_ref * inv_T);
    const double pscale = c.gamma_scale * (c.P / c.P_ref);
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        double nu = L.nu[l];
        double Il = line_strength64(nu, (double)L.elower[l], (double)L.g_up[l] * (double)L.A[l], c, sel);
        double al = acoef * nu;
        double ga = L.n_broad > 0 ? mixture_gamma64(L, l, c)
                                  : pscale * (double)L.gamma_ref[l] * exp(((double)L.n_T[l] + c.n_shift) * lnTr);
        double cl = line_cut(cut_mode, cutoff, width_mult, al, ga);
        if (Il < 0.0) {   // left out by the intensity threshold: no grid point is within a negative cut
            Il = 0.0;
            cl = -1.0;
        }
        if (I) I[l] = Il;
        if (alpha) alpha[l] = al;
        if (gamma) gamma[l] = ga;
        if (cut) cut[l] = cl;
    }
}

__global__ void __launch_bounds__(256) k_line_keep(LinesDev L, size_t n, const CondDev *__restrict__ conds, int nc,
                                                   StrengthSel sel, uint32_t *keep, int words) {
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        const double nu = L.nu[l], E = (double)L.elower[l], gA = (double)L.g_up[l] * (double)L.A[l];
        for (int w = 0; w < words; ++w) {
            uint32_t bits = 0u;
            for (int b = 0; b < 32 && w * 32 + b < nc; ++b)
                if (line_strength64(nu, E, gA, conds[w * 32 + b], sel) >= 0.0) bits |= 1u << b;
            keep[l * (size_t)words + w] = bits;
        }
    }
}

__global__ void __launch_bounds__(256) k_apply_broadening(const int16_t *j_lo, const int16_t *j_up, size_t n, int nb,
                                                          const int *type, const double *frac, const double *g0_def,
                                                          const double *n_def, const int *row0, const int64_t *keys,
                                                          const double *g0, const double *nl, double *bgam,
                                                          double *bn) {
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        const int jl = j_lo ? j_lo[l] : 0, ju = j_up ? j_up[l] : 0;
        for (int i = 0; i < nb; ++i) {
            double g = g0_def[i], m = n_def[i];
            if (type[i] != XC_BROAD_CONSTANT && row0[i + 1] > row0[i]) {
                const int64_t key = type[i] == XC_BROAD_A1 ? (int64_t)jl * 65536 + ju : (int64_t)jl;
                int lo = row0[i], hi = row0[i + 1];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (keys[mid] < key) lo = mid + 1; else hi = mid;
                }
                if (lo < row0[i + 1] && keys[lo] == key) {
                    g = g0[lo];
                    m = nl[lo];
                }
            }
            bgam[(size_t)i * n + l] = frac[i] * g;
            bn[(size_t)i * n + l] = m;
        }
    }
}

cudaError_t launch_apply_broadening(const int16_t *j_lo, const int16_t *j_up, size_t n, int nb, const int *type,
                                    const double *frac, const double *g0_def, const double *n_def,
                                    const int *row0, const int64_t *keys, const double *g0, const double *nl,
                                    double *bgam, double *bn, cudaStream_t s) {
    if (n == 0 || nb == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_apply_broadening<<<(unsigned)blocks, 256, 0, s>>>(j_lo, j_up, n, nb, type, frac, g0_def, n_def, row0, keys, g0,
                                                        nl, bgam, bn);
    return cudaGetLastError();
}

__global__ void k_permute_i16(const int16_t *__restrict__ in, const uint32_t *__restrict__ perm, size_t n,
                              int16_t *__restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[perm[i]];
}

cudaError_t launch_permute_i16(const int16_t *in, const uint32_t *perm, size_t n, int16_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_permute_i16<<<(unsigned)blocks, 256, 0, s>>>(in, perm, n, out);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_line_gamma(LinesDev L, size_t n, const CondDev *__restrict__ conds, int nc,
                                                    float *gamma_lc, unsigned *gmax_bits) {
    for (int c = 0; c < nc; ++c) {
        const CondDev cd = conds[c];
        float m = 0.f;
        for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
            const float g = (float)mixture_gamma64(L, l, cd);
            gamma_lc[l * (size_t)nc + c] = g;
            m = fmaxf(m, g);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        // non-negative floats order as their bit patterns; rounded up so that the bound holds
        if ((threadIdx.x & 31) == 0) atomicMax(&gmax_bits[c], __float_as_uint(m) + 1u);
    }
}

cudaError_t launch_line_gamma(const LinesDev &L, size_t n, const CondDev *conds, int nc, float *gamma_lc,
                              unsigned *gmax_bits, cudaStream_t s) {
    if (n == 0 || nc == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_line_gamma<<<(unsigned)blocks, 256, 0, s>>>(L, n, conds, nc, gamma_lc, gmax_bits);
    return cudaGetLastError();
}

// VVN for the FP32 kernels, one warp per (line, condition): 1 / (h sum_k f_VV) over the
// lattice points within the line's cut (fixed, or width-limited as the kernels take it)
__global__ void __launch_bounds__(256) k_vv_norm32(LinesDev L, size_t n, const CondDev *__restrict__ conds, int nc,
                                                   double nu_A, double step, double cutoff, double width_mult,
                                                   double split, int beta, float *scale) {
    const int lane = threadIdx.x & 31;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    const size_t pairs = n * (size_t)nc;
    for (size_t q = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < pairs; q += warps) {
        const size_t l = q / (size_t)nc;
        const int c = (int)(q % (size_t)nc);
        const CondDev cd = conds[c];
        const double nul = L.nu[l];
        const double al = alpha_coef(cd.T, cd.mass_da) * nul;
        const double ga = L.n_broad > 0 ? mixture_gamma64(L, l, cd)
                                        : cd.gamma_scale * (double)L.gamma_ref[l] *
                                              exp(((double)L.n_T[l] + cd.n_shift) * log(cd.T_ref / cd.T)) *
                                              (cd.P / cd.P_ref);
        const double cut = width_mult > 0.0 ? fmin(width_mult * fmax(al, ga), cutoff) : cutoff;
        const int64_t k0 = (int64_t)floor((nul - cut - nu_A) / step) - 1;
        const int64_t k1 = (int64_t)floor((nul + cut - nu_A) / step) + 1;
        double sum = 0.0;
        for (int64_t k = k0 + lane; k <= k1; k += 32) {
            const double D = __dsub_rn(grid_x(nu_A, step, k), nul);
            if (fabs(D) <= cut) sum += voigt_vv64(D, al, ga, nul, split, beta);
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) scale[q] = sum > 0.0 ? (float)(1.0 / (sum * step)) : 0.f;
    }
}

cudaError_t launch_vv_norm32(const LinesDev &L, size_t n, const CondDev *conds, int nc, double nu_A, double step,
                             double cutoff, double width_mult, double vv_split, int vv_beta, float *scale,
                             cudaStream_t s) {
    if (n == 0 || nc == 0) return cudaSuccess;
    size_t blocks = (n * (size_t)nc + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_vv_norm32<<<(unsigned)blocks, 256, 0, s>>>(L, n, conds, nc, nu_A, step, cutoff, width_mult, vv_split, vv_beta,
                                                 scale);
    return cudaGetLastError();
}

cudaError_t launch_line_keep(const LinesDev &L, size_t n, const CondDev *conds, int nc, const StrengthSel &sel,
                             uint32_t *keep, int words, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_line_keep<<<(unsigned)blocks, 256, 0, s>>>(L, n, conds, nc, sel, keep, words);
    return cudaGetLastError();
}

cudaError_t launch_line_params64(const LinesDev &L, size_t n, const CondDev *cond_dev, int cut_mode,
                                 double cutoff, double width_mult, double *I, double *alpha, double *gamma,
                                 double *cut, cudaStream_t s, const StrengthSel &sel) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_line_params64<<<(unsigned)blocks, 256, 0, s>>>(L, n, cond_dev, cut_mode, cutoff, width_mult, I, alpha,
                                                     gamma, cut, sel);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Window -> line range: lo = first l with nu_l >= x_first - cutmax,
// hi = first l with nu_l > x_last + cutmax (sorted nu).  A small relative
// margin keeps every line whose exact cut test could pass.
// ---------------------------------------------------------------------------
__device__ inline int64_t lower_bound_d(const double *a, int64_t n, double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ inline int64_t upper_bound_d(const double *a, int64_t n, double x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_window_ranges(const double *__restrict__ nu, int64_t n, double nu_A, double step, int64_t n_pts,
                                int64_t W, double cutmax, int64_t n_win, int64_t *lo, int64_t *hi) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_win) return;
    int64_t k0 = w * W;
    int64_t k1 = i64min(k0 + W, n_pts) - 1;
    double x0 = grid_x(nu_A, step, k0), x1 = grid_x(nu_A, step, k1);
    double margin = cutmax * (1.0 + 1e-12) + 1e-12 * (fabs(x0) + fabs(x1));
    lo[w] = lower_bound_d(nu, n, x0 - margin);
    hi[w] = upper_bound_d(nu, n, x1 + margin);
}

cudaError_t launch_window_ranges(const double *nu, size_t n, double nu_A, double step, int64_t n_pts,
                                 int64_t W, double cutmax, int64_t n_win, int64_t *lo, int64_t *hi,
                                 cudaStream_t s) {
    if (n_win <= 0) return cudaSuccess;
    k_window_ranges<<<(unsigned)((n_win + 127) / 128), 128, 0, s>>>(nu, (int64_t)n, nu_A, step, n_pts, W, cutmax,
                                                                     n_win, lo, hi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Algorithmic work: sum over conditions and lines of the number of grid
// points with |x_k - nu_l| <= cut_l.  Warp-reduced, one 64-bit atomic per warp
// (an integer sum, so the order does not matter).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_count_evals(LinesDev L, size_t n, const CondDev *__restrict__ conds,
                                                     int n_cond, double nu_A, double step, int64_t n_pts,
                                                     double cutoff, double width_mult,
                                                     unsigned long long *count) {
    unsigned long long local = 0;
    const double inv_step = 1.0 / step;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
        double nu = L.nu[l];
        for (int c = 0; c < n_cond; ++c) {
            double cut = cutoff;
            if (width_mult > 0.0) {
                const CondDev &cd = conds[c];
                double al = alpha_coef(cd.T, cd.mass_da) * nu;
                double ga = L.n_broad > 0 ? mixture_gamma64(L, l, cd)
                                          : cd.gamma_scale * (double)L.gamma_ref[l] *
                                                exp(((double)L.n_T[l] + cd.n_shift) * log(cd.T_ref / cd.T)) *
                                                (cd.P / cd.P_ref);
                cut = fmin(width_mult * fmax(al, ga), cutoff);
            }
            int64_t ka, kb;
            line_k_range(nu, cut, nu_A, step, inv_step, n_pts, &ka, &kb);
            if (kb >= ka) local += (unsigned long long)(kb - ka + 1);
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(count, local);
}

cudaError_t launch_count_evals(const LinesDev &L, size_t n, const CondDev *conds_dev, int n_cond,
                               double nu_A, double step, int64_t n_pts, double cutoff, double width_mult,
                               unsigned long long *count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_count_evals<<<(unsigned)blocks, 256, 0, s>>>(L, n, conds_dev, n_cond, nu_A, step, n_pts, cutoff, width_mult,
                                                   count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gauss-Hermite nodes/weights for weight exp(-x^2), n <= 64, on the device.
// Thread j finds root j (ascending): a WKB phase estimate
//   (2n+1)/2 (phi + sin(2 phi)/2) = pi (j - (n-1)/2),  x0 = sqrt(2n+1) sin(phi),
// then Newton's method on the orthonormal Hermite polynomial p_n, whose
// derivative is sqrt(2n) p_{n-1}.  At a root, the Christoffel-Darboux identity
// gives sum_{k<n} p_k^2 = n p_{n-1}^2, so the weight is 1 / (n p_{n-1}^2).
// ---------------------------------------------------------------------------
__device__ inline void herm_norm(int n, double x, double *pn, double *pn1) {
    // orthonormal recurrence: p_{k+1} = x sqrt(2/(k+1)) p_k - sqrt(k/(k+1)) p_{k-1}
    double pm = 0.0, p = 0.75112554446494248286;  // pi^(-1/4)
    for (int k = 0; k < n; ++k) {
        double q = x * sqrt(2.0 / (k + 1)) * p - sqrt((double)k / (k + 1)) * pm;
        pm = p;
        p = q;
    }
    *pn = p;
    *pn1 = pm;
}

__global__ void k_gh_nodes(int n, double *x, double *w) {
    int j = threadIdx.x;
    if (j >= n) return;
    const double m = 2.0 * n + 1.0;
    const double target = kPi * (j - 0.5 * (n - 1));
    double phi = 0.0;
    for (int it = 0; it < 60; ++it) {
        double F = 0.5 * m * (phi + 0.5 * sin(2.0 * phi));
        double c = cos(phi);
        phi -= (F - target) / (m * c * c);
        phi = fmin(fmax(phi, -1.5), 1.5);
    }
    double r = sqrt(m) * sin(phi);
    for (int it = 0; it < 100; ++it) {
        double pn, pn1;
        herm_norm(n, r, &pn, &pn1);
        double st = pn / (sqrt(2.0 * n) * pn1);
        r -= st;
        if (fabs(st) < 1e-15 * fmax(1.0, fabs(r))) break;
    }
    double pn, pn1;
    herm_norm(n, r, &pn, &pn1);
    x[j] = r;
    w[j] = 1.0 / (n * pn1 * pn1);
}

cudaError_t launch_gh_nodes(int n, double *x, double *w, cudaStream_t s) {
    if (n < 1 || n > 64) return cudaErrorInvalidValue;
    k_gh_nodes<<<1, 64, 0, s>>>(n, x, w);
    return cudaGetLastError();
}

}  // namespace xc
