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
                                   const double *ghw, int ngh, double nul = 0.0, double split = 4.0,
                                   int beta = 0) {
    if (PROF == XC_VOIGT_VV) {
        return voigt_vv64(D, al, ga, nul, split, beta);
    } else if (PROF == XC_DOPPLER) {
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
                                                            double *__restrict__ sigma, double vv_split,
                                                            int vv_beta) {
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
                if (fabs(D) <= s_c[i])
                    acc += s_I[i] * profile64<PROF>(D, step, s_a[i], s_g[i], s_ghx, s_ghw, ngh, s_nu[i], vv_split,
                                                    vv_beta);
            }
        }
    }
    if (active) sigma[k] = acc;
}

cudaError_t launch_gather_f64(int profile, const double *nu, const double *I, const double *alpha,
                              const double *gamma, const double *cut, const int64_t *win_lo,
                              const int64_t *win_hi, int64_t n_win, double nu_A, double step, int64_t n_pts,
                              const double *ghx, const double *ghw, int ngh, double *sigma, cudaStream_t s,
                              double vv_split, int vv_beta) {
    if (n_win <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_win), block(G64_THREADS);
#define XC_G64(P) k_gather_f64<P><<<grid, block, 0, s>>>(nu, I, alpha, gamma, cut, win_lo, win_hi, nu_A, step, \
                                                        n_pts, ghx, ghw, ngh, sigma, vv_split, vv_beta)
    switch (profile) {
    case XC_DOPPLER: XC_G64(XC_DOPPLER); break;
    case XC_LORENTZ: XC_G64(XC_LORENTZ); break;
    case XC_VOIGT_W4: XC_G64(XC_VOIGT_W4); break;
    case XC_VOIGT_GH_BINNED: XC_G64(XC_VOIGT_GH_BINNED); break;
    case XC_VOIGT_GH_SAMPLED: XC_G64(XC_VOIGT_GH_SAMPLED); break;
    case XC_DOPPLER_BINNED: XC_G64(XC_DOPPLER_BINNED); break;
    case XC_LORENTZ_BINNED: XC_G64(XC_LORENTZ_BINNED); break;
    case XC_VOIGT_VV: XC_G64(XC_VOIGT_VV); break;
    default:
        return cudaErrorInvalidValue;
    }
#undef XC_G64
    return cudaGetLastError();
}

// VVN normalisation, one warp per line: Sigma = h sum_k f_VV over the lattice points
// nu_A + k h within the line's cut (the grid extended past its ends), summed in FP64 in a
// fixed order (strided lanes, then a butterfly), then I /= Sigma
__global__ void __launch_bounds__(256) k_vv_norm64(const double *__restrict__ nu, double *__restrict__ I,
                                                   const double *__restrict__ alpha,
                                                   const double *__restrict__ gamma, const double *__restrict__ cut,
                                                   size_t n, double nu_A, double step, double split, int beta) {
    const int lane = threadIdx.x & 31;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t l = (size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < n; l += warps) {
        const double nul = nu[l], al = alpha[l], ga = gamma[l], c = cut[l];
        if (!(c >= 0.0)) continue;   // a line the intensity threshold left out
        const int64_t k0 = (int64_t)floor((nul - c - nu_A) / step) - 1;
        const int64_t k1 = (int64_t)floor((nul + c - nu_A) / step) + 1;
        double sum = 0.0;
        for (int64_t k = k0 + lane; k <= k1; k += 32) {
            const double D = __dsub_rn(grid_x(nu_A, step, k), nul);
            if (fabs(D) <= c) sum += voigt_vv64(D, al, ga, nul, split, beta);
        }
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) I[l] = sum > 0.0 ? I[l] / (sum * step) : 0.0;
    }
}

cudaError_t launch_vv_norm64(const double *nu, double *I, const double *alpha, const double *gamma,
                             const double *cut, size_t n, double nu_A, double step, double vv_split, int vv_beta,
                             cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t blocks = (n + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_vv_norm64<<<(unsigned)blocks, 256, 0, s>>>(nu, I, alpha, gamma, cut, n, nu_A, step, vv_split, vv_beta);
    return cudaGetLastError();
}

}  // namespace xc
