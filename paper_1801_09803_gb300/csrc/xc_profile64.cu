// xc_profile64.cu -- the plain FP64 gather-form profile kernel.
//
// Each CTA owns a window of 256 consecutive grid points (one per thread) and
// walks the lines whose cut can reach the window (range found by binary search
// on the sorted wavenumbers), staging 256 line records at a time in shared
// memory.  Every thread evaluates the profile of each staged line at its own
// grid point when |nu_k - nu_l| <= cut_l (paper Sec. 3.1 sampling, Sec. 3.10
// cutoff) and accumulates I_l f_l(nu_k) in FP64 in line order.  No atomics:
// each output is written once by its owner thread.
#include "xc_internal.cuh"

namespace xc {

constexpr int G64_THREADS = 256;

template <int PROF>
__device__ inline double profile64(double D, double step, double al, double ga, const double *ghx,
                                   const double *ghw, int ngh) {
    if (PROF == XC_DOPPLER) {
        // Eq. (e:Gauss): sqrt(ln2/pi)/alpha exp(-D^2 ln2/alpha^2)
        double r = D / al;
        return 0.46971863934982566 / al * exp(-kLn2 * r * r);
    } else if (PROF == XC_LORENTZ) {
        // Eq. (e:lor)
        return ga / (kPi * (D * D + ga * ga));
    } else if (PROF == XC_VOIGT_W4) {
        // unit-area Voigt: sqrt(ln2/pi)/alpha Re w(x + iy), x = sqrt(ln2) D/alpha, y = sqrt(ln2) gamma/alpha
        double ia = kSqrtLn2 / al;
        Cx<double> w = w4_eval<double>(D * ia, ga * ia, nullptr);
        return 0.46971863934982566 / al * w.re;
    } else if (PROF == XC_DOPPLER_BINNED) {
        // Eq. (eqn:sig_ij) without I: (erf(x+) - erf(x-)) / (2h), x+- = sqrt(ln2)/alpha (D +- h/2),
        // taken on the side |D| as erfc(x-) - erfc(x+) (the profile is symmetric)
        double t = fabs(D), c = kSqrtLn2 / al;
        return (erfc(c * (t - 0.5 * step)) - erfc(c * (t + 0.5 * step))) / (2.0 * step);
    } else if (PROF == XC_LORENTZ_BINNED) {
        // Eq. (eqn:sig_lor-2) without I: (atan(y+) - atan(y-)) / (pi h), y+- = (D +- h/2)/gamma,
        // as one atan2 with both arguments scaled by gamma^2 > 0
        double hh = 0.5 * step;
        return atan2(step * ga, (D + hh) * (D - hh) + ga * ga) / (kPi * step);
    } else if (PROF == XC_VOIGT_GH_SAMPLED) {
        // Eq. (e:V-quad) with node shift alpha x_j / sqrt(ln2)
        double s = 0.0, g2 = ga * ga, sh = al / kSqrtLn2;
        for (int j = 0; j < ngh; ++j) {
            double d = D - sh * ghx[j];
            s += ghw[j] * ga / (d * d + g2);
        }
        return s * 0.17958712212516656;  // pi^(-3/2)
    } else {
        // Eq. (e:sigma:quad) without I: pi^(-3/2)/h sum_j w_j [atan(y+) - atan(y-)],
        // with atan(a) - atan(b) = atan2(a - b, 1 + ab) for a > b
        double s = 0.0, sh = al / kSqrtLn2, hh = 0.5 * step;
        for (int j = 0; j < ngh; ++j) {
            double d = D - sh * ghx[j];
            double q = (d + hh) * (d - hh) + ga * ga;  // gamma^2 (1 + y+ y-)
            s += ghw[j] * atan2(step * ga, q);          // scaled by gamma^2 > 0 in both arguments
        }
        return s * 0.17958712212516656 / step;
    }
}

template <int PROF>
__global__ void __launch_bounds__(G64_THREADS) k_gather_f64(const double *__restrict__ nu,
                                                            const double *__restrict__ I,
                                                            const double *__restrict__ alpha,
                                                            const double *__restrict__ gamma,
                                                            const double *__restrict__ cut,
                                                            const int64_t *__restrict__ win_lo,
                                                            const int64_t *__restrict__ win_hi, double nu_A,
                                                            double step, int64_t n_pts,
                                                            const double *__restrict__ ghx_g,
                                                            const double *__restrict__ ghw_g, int ngh,
                                                            double *__restrict__ sigma) {
    __shared__ double s_nu[G64_THREADS], s_I[G64_THREADS], s_a[G64_THREADS], s_g[G64_THREADS],
        s_c[G64_THREADS];
    __shared__ double s_ghx[64], s_ghw[64];
    const int tid = threadIdx.x;
    if (tid < ngh) {
        s_ghx[tid] = ghx_g[tid];
        s_ghw[tid] = ghw_g[tid];
    }
    const int64_t w = blockIdx.x;
    const int64_t k = w * G64_THREADS + tid;
    const bool active = k < n_pts;
    const double xk = grid_x(nu_A, step, k);
    const int64_t lo = win_lo[w], hi = win_hi[w];
    double acc = 0.0;
    for (int64_t l0 = lo; l0 < hi; l0 += G64_THREADS) {
        const int cnt = (int)i64min(G64_THREADS, hi - l0);
        __syncthreads();
        if (tid < cnt) {
            s_nu[tid] = nu[l0 + tid];
            s_I[tid] = I[l0 + tid];
            s_a[tid] = alpha[l0 + tid];
            s_g[tid] = gamma[l0 + tid];
            s_c[tid] = cut[l0 + tid];
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < cnt; ++i) {
                double D = __dsub_rn(xk, s_nu[i]);
                if (fabs(D) <= s_c[i]) acc += s_I[i] * profile64<PROF>(D, step, s_a[i], s_g[i], s_ghx, s_ghw, ngh);
            }
        }
    }
    if (active) sigma[k] = acc;
}

cudaError_t launch_gather_f64(int profile, const double *nu, const double *I, const double *alpha,
                              const double *gamma, const double *cut, const int64_t *win_lo,
                              const int64_t *win_hi, int64_t n_win, double nu_A, double step, int64_t n_pts,
                              const double *ghx, const double *ghw, int ngh, double *sigma, cudaStream_t s) {
    if (n_win <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_win), block(G64_THREADS);
    switch (profile) {
    case XC_DOPPLER:
        k_gather_f64<XC_DOPPLER><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A, step,
                                                       n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_LORENTZ:
        k_gather_f64<XC_LORENTZ><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A, step,
                                                       n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_VOIGT_W4:
        k_gather_f64<XC_VOIGT_W4><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A, step,
                                                        n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_VOIGT_GH_BINNED:
        k_gather_f64<XC_VOIGT_GH_BINNED><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A,
                                                               step, n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_VOIGT_GH_SAMPLED:
        k_gather_f64<XC_VOIGT_GH_SAMPLED><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A,
                                                                step, n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_DOPPLER_BINNED:
        k_gather_f64<XC_DOPPLER_BINNED><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A,
                                                              step, n_pts, ghx, ghw, ngh, sigma);
        break;
    case XC_LORENTZ_BINNED:
        k_gather_f64<XC_LORENTZ_BINNED><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A,
                                                              step, n_pts, ghx, ghw, ngh, sigma);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace xc
