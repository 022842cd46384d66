// xc_vjp.cu -- adjoint (vector-Jacobian product) of the cross section.
//
// Not in the paper: the chain rule of Eq. (e:int) (intensity), Eq. (e:alphaD),
// Eq. (e:gamma_L) and the profile, applied to sigma_k = sum_l I_l V(nu_k - nu_l;
// alpha_l, gamma_l).  For every line and condition the kernel gathers, over
// the grid points inside the cut,
//     S_I = sum_k g_k V,   S_a = sum_k g_k dV/dalpha,   S_g = sum_k g_k dV/dgamma
// (g = dL/dsigma), recomputing the profile instead of storing it, and then
//     dL/dT_c += I S_I dlnI/dT + I S_a alpha/(2T) - I S_g n gamma/T
//     dL/dP_c += I S_g dgamma/dP,  dL/ds += I S_g dgamma/ds,  dL/dn += I S_g gamma ln(T_ref/T)
//     dL/dgamma_ref_l += I S_g dgamma/dgamma_ref,  dL/dn_l += I S_g gamma ln(T_ref/T)
// with dlnI/dT = c2 E''/T^2 - (c2 nu/T^2)/(exp(c2 nu/T) - 1) - Q'/Q.
//
// Layout: one warp per line (grid-stride), lanes stride over the line's grid
// points, lane c holds the FP64 constants of condition c (<= 32 per launch).
// Per-condition scalars are reduced warp -> block in fixed order, written as
// block partials and summed in block order by a second kernel, so the result
// is deterministic.  Region I of w4 uses its rational form and closed-form
// derivatives; points in regions II-IV evaluate the complex w4 and its exact
// derivative F'(t).
#include <math.h>

#include <algorithm>

#include "xc_batched.cuh"

namespace xc {

constexpr int VT = 256;
constexpr int VW = VT / 32;
constexpr int VMAXC = 32;
constexpr double kKappa64 = 0.5641896 / 1.772453850905516027;

struct VjpLineCond {  // per (line, condition), FP64
    double I, al, ga, dlnI, dga_dP, dga_ds, dga_dgr, lnTr, T;
};

__device__ inline VjpLineCond line_cond64(const LinesDev &L, size_t l, const CondDev &c) {
    VjpLineCond r;
    double nu = L.nu[l];
    double inv_T = 1.0 / c.T;
    double x = kC2 * nu * inv_T;
    double boltz = exp(-kC2 * (double)L.elower[l] * inv_T);
    double stim = -expm1(-x);
    r.I = c.abundance / (8.0 * kPi * kLightCm * c.Q) * (double)L.g_up[l] * (double)L.A[l] / (nu * nu) * boltz * stim;
    r.al = alpha_coef(c.T, c.mass_da) * nu;
    r.lnTr = log(c.T_ref * inv_T);
    double tn = exp(((double)L.n_T[l] + c.n_shift) * r.lnTr);  // (T_ref/T)^n
    double gr = (double)L.gamma_ref[l];
    r.ga = c.gamma_scale * gr * tn * (c.P / c.P_ref);
    r.dga_dP = c.gamma_scale * gr * tn / c.P_ref;
    r.dga_ds = gr * tn * (c.P / c.P_ref);
    r.dga_dgr = c.gamma_scale * tn * (c.P / c.P_ref);
    r.dlnI = kC2 * (double)L.elower[l] * inv_T * inv_T - (x * inv_T) / expm1(x) - c.dQdT / c.Q;
    r.T = c.T;
    return r;
}

__device__ inline double shfl64(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Re w and its partial derivatives d/dx, d/dy (x >= 0) in w4's regions I and II,
// from their real forms: region I is one pair of Lorentzians (nodes +-1/sqrt2),
// region II two pairs (nodes +-sqrt(Q_m), Q_m = (3 -+ sqrt 6)/2):
//   Re w = y sum_m A_m (X + Y + Q_m) / ((X + Y - Q_m)^2 + 4 Q_m Y),  X = x^2, Y = y^2.
__device__ inline float w4_re_grad_12(float x, float y, float *dx, float *dy) {
    constexpr double a = 1.410474, b = 0.5641896, s6 = 2.449489742783178098;
    const bool r1 = x + y >= 15.f;
    const float Qm[2] = {r1 ? 0.5f : (float)((3.0 - s6) / 2.0), (float)((3.0 + s6) / 2.0)};
    const float Am[2] = {r1 ? 0.5641896f : (float)((a - b * ((3.0 - s6) / 2.0)) / s6),
                         r1 ? 0.f : (float)(-(a - b * ((3.0 + s6) / 2.0)) / s6)};
    const float X = x * x, Y = y * y;
    float S = 0.f, SX = 0.f, SY = 0.f;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        float N = X + Y + Qm[m], t = X + Y - Qm[m];
        float D = fmaf(t, t, 4.f * Qm[m] * Y);
        float rD = 1.f / D, rD2 = rD * rD;
        S = fmaf(Am[m] * N, rD, S);
        SX = fmaf(Am[m], (D - 2.f * N * t) * rD2, SX);                    // d(N/D)/dX
        SY = fmaf(Am[m], (D - N * (2.f * t + 4.f * Qm[m])) * rD2, SY);    // d(N/D)/dY
    }
    *dx = y * SX * 2.f * x;
    *dy = S + y * SY * 2.f * y;
    return y * S;
}

// compensated FP32 sum (Kahan): the running compensation keeps the rounding of every
// addition, so the sum is good to a few FP32 ulps of its terms whatever its length
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// value and derivatives of the profile (FP64 reference form, all w4 regions)
template <int PROF>
__device__ inline void prof_deriv64(double D, double al, double ga, double *V, double *dVa, double *dVg) {
    if (PROF == XC_DOPPLER) {
        double r = D / al;
        double v = 0.46971863934982566 / al * exp(-kLn2 * r * r);
        *V = v;
        *dVa = v * (-1.0 / al + 2.0 * kLn2 * D * D / (al * al * al));
        *dVg = 0.0;
    } else if (PROF == XC_LORENTZ) {
        double q = D * D + ga * ga;
        *V = ga / (kPi * q);
        *dVa = 0.0;
        *dVg = (D * D - ga * ga) / (kPi * q * q);
    } else {
        double ia = kSqrtLn2 / al;
        Cx<double> dF;
        Cx<double> w = w4_eval<double>(D * ia, ga * ia, &dF);
        double v = 0.46971863934982566 / al * w.re;
        double k2 = kLn2 / (kSqrtPi * al * al);
        double dVD = k2 * dF.im;  // dF/dx = -i F'  ->  Re = Im F'
        double dg = k2 * dF.re;
        *V = v;
        *dVg = dg;
        *dVa = -(v + D * dVD + ga * dg) / al;
    }
}

template <int PROF, bool F64>
__global__ void __launch_bounds__(VT) k_vjp_lines(LinesDev L, size_t n, const CondDev *__restrict__ conds, int nc,
                                                  double nu_A, double step, int64_t n_pts, double cutoff,
                                                  double width_mult, const double *__restrict__ g64,
                                                  const float *__restrict__ g32, double *block_part /*[blk][nc][4]*/,
                                                  double *d_gref_line, double *d_n_line, int accumulate) {
    __shared__ double s_part[VW][VMAXC][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double accT = 0.0, accP = 0.0, accS = 0.0, accN = 0.0;  // lane c: condition c
    const CondDev cme = conds[lane < nc ? lane : 0];
    for (size_t l = (size_t)blockIdx.x * VW + warp; l < n; l += (size_t)gridDim.x * VW) {
        const double nu = L.nu[l];
        VjpLineCond mine = line_cond64(L, l, cme);
        double line_gr = 0.0, line_n = 0.0;
        // grid position of the line
        const double dpos = (nu - nu_A) / step;
        const double fl = floor(dpos);
        const float ff = (float)(dpos - fl);
        const int64_t nabs = (int64_t)fl;
        int64_t ka0 = 0, kb0 = -1;
        if (!(width_mult > 0.0)) line_k_range(nu, cutoff, nu_A, step, n_pts, &ka0, &kb0);
        for (int c = 0; c < nc; ++c) {
            const double I = shfl64(mine.I, c), al = shfl64(mine.al, c), ga = shfl64(mine.ga, c);
            int64_t ka = ka0, kb = kb0;
            if (width_mult > 0.0) line_k_range(nu, fmin(width_mult * fmax(al, ga), cutoff), nu_A, step, n_pts, &ka, &kb);
            double SI = 0.0, Sa = 0.0, Sg = 0.0;
            if (F64) {
                for (int64_t k = ka + lane; k <= kb; k += 32) {
                    double D = __dsub_rn(grid_x(nu_A, step, k), nu);
                    double V, dVa, dVg;
                    prof_deriv64<PROF>(D, al, ga, &V, &dVa, &dVg);
                    double g = g64[(size_t)c * n_pts + k];
                    SI += g * V;
                    Sa += g * dVa;
                    Sg += g * dVg;
                }
            } else {
                const float h = (float)step;
                const float alf = (float)al, gaf = (float)ga;
                const float g2 = gaf * gaf;
                const float b = alf * alf * (float)(0.5 / 0.6931471805599453);
                const float bg = b + g2;
                const float a_sc = (float)kSqrtLn2 / alf;      // x = a |D|
                const float yv = a_sc * gaf;
                const float thr = yv < 15.f ? (15.f - yv) / a_sc : -1.f;  // region I iff |D| >= thr
                const float thr2 = thr > 0.f ? thr * thr : -1.f;
                // FP32 terms in compensated (Kahan) FP32 sums: as accurate as folding them into
                // FP64 and free of FP64 instructions, which run at a small fraction of the FP32
                // rate on this GPU.  Centre points of w4 regions III/IV, which carry the largest
                // terms of sums that cancel (the derivatives of a unit-area profile integrate to
                // zero), are evaluated and added in FP64.
                double C0 = 0.0, C1 = 0.0, C2 = 0.0;
                KahanF s0, s1, s2, c0, c1, c2;
                const float *gc = g32 + (size_t)c * n_pts;
                for (int64_t kb8 = ka + lane; kb8 <= kb; kb8 += 32 * 8) {
#pragma unroll 4
                    for (int j = 0; j < 8; ++j) {
                        const int64_t k = kb8 + 32 * j;
                        if (k > kb) break;
                        float D = ((float)(k - nabs) - ff) * h;
                        float u = D * D;
                        float g = gc[k];
                        if (PROF == XC_VOIGT_W4) {
                            if (u >= thr2) {
                                float t = bg - u;
                                float Dn = fmaf(t, t, 4.f * g2 * u);
                                float N = u + bg;
                                float rD = 1.f / Dn;
                                float rD2 = rD * rD;
                                s0.add(g * (N * rD));
                                s1.add(g * (fmaf(-2.f * N, t, Dn) * rD2));
                                float q = fmaf(Dn, N + 2.f * g2, -4.f * g2 * N * N);
                                s2.add(g * (q * rD2));
                            } else if (a_sc * fabsf(D) + yv >= 5.5f) {
                                // region II (or I by rounding at its edge): real form, FP32
                                float rx, ry;
                                float w = w4_re_grad_12(a_sc * fabsf(D), yv, &rx, &ry);
                                float v = (float)0.46971863934982566 / alf * w;
                                float k2 = (float)(0.6931471805599453 / 1.772453850905516027) / (alf * alf);
                                float dVD = k2 * (D < 0.f ? -rx : rx), dg = k2 * ry;
                                c0.add(g * v);
                                c1.add(g * (-(v + D * dVD + gaf * dg) / alf));
                                c2.add(g * dg);
                            } else {
                                // regions III/IV: complex rationals whose derivative cancels in
                                // FP32; evaluated in FP64 (a narrow band around the centre)
                                double D64 = __dsub_rn(grid_x(nu_A, step, k), nu);
                                double V, dVa, dVg;
                                prof_deriv64<XC_VOIGT_W4>(D64, al, ga, &V, &dVa, &dVg);
                                double gd = (double)g;
                                C0 += gd * V;
                                C1 += gd * dVa;
                                C2 += gd * dVg;
                            }
                        } else if (PROF == XC_DOPPLER) {
                            float e = expf(-(float)kLn2 * u / (alf * alf));
                            c0.add(g * e);
                            c1.add(g * (e * u));
                        } else {
                            float r = 1.f / (u + g2);
                            c0.add(g * r);
                            c2.add(g * ((u - g2) * r * r));
                        }
                    }
                }
                const double S0 = s0.value(), S1 = s1.value(), S2 = s2.value();
                C0 += c0.value();
                C1 += c1.value();
                C2 += c2.value();
                if (PROF == XC_VOIGT_W4) {
                    double kg = kKappa64 * ga;
                    SI = kg * S0 + C0;
                    Sa = kg * S1 * (al / kLn2) + C1;  // dV/dalpha = dV/db * alpha/ln2
                    Sg = kKappa64 * S2 + C2;
                } else if (PROF == XC_DOPPLER) {
                    double pd = 0.46971863934982566 / al;
                    SI = pd * C0;
                    Sa = pd * (-C0 / al + 2.0 * kLn2 / (al * al * al) * C1);
                    Sg = 0.0;
                } else {
                    SI = ga / kPi * C0;
                    Sa = 0.0;
                    Sg = C2 / kPi;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                SI += __shfl_xor_sync(0xffffffffu, SI, o);
                Sa += __shfl_xor_sync(0xffffffffu, Sa, o);
                Sg += __shfl_xor_sync(0xffffffffu, Sg, o);
            }
            // every lane holds the sums; lane c owns condition c's scalars
            if (lane == c) {
                const double T = mine.T;
                accT += I * (SI * mine.dlnI + Sa * al / (2.0 * T) - Sg * (double)(L.n_T[l] + cme.n_shift) * ga / T);
                accP += I * Sg * mine.dga_dP;
                accS += I * Sg * mine.dga_ds;
                accN += I * Sg * ga * mine.lnTr;
            }
            line_gr += I * Sg * shfl64(mine.dga_dgr, c);
            line_n += I * Sg * ga * shfl64(mine.lnTr, c);
        }
        if (lane == 0) {
            if (d_gref_line) d_gref_line[l] = accumulate ? d_gref_line[l] + line_gr : line_gr;
            if (d_n_line) d_n_line[l] = accumulate ? d_n_line[l] + line_n : line_n;
        }
    }
    if (lane < nc) {
        s_part[warp][lane][0] = accT;
        s_part[warp][lane][1] = accP;
        s_part[warp][lane][2] = accS;
        s_part[warp][lane][3] = accN;
    }
    __syncthreads();
    if (threadIdx.x < nc * 4) {
        int c = threadIdx.x >> 2, q = threadIdx.x & 3;
        double s = 0.0;
        for (int w = 0; w < VW; ++w) s += s_part[w][c][q];
        block_part[((size_t)blockIdx.x * nc + c) * 4 + q] = s;
    }
}

// sum block partials in block order; conditions c0.. of this chunk
__global__ void k_vjp_finish(const double *block_part, int n_blocks, int nc, int c0, double *dT, double *dP,
                             double *dS_acc, double *dN_acc) {
    int c = threadIdx.x;
    if (c >= nc) return;
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < n_blocks; ++b)
        for (int q = 0; q < 4; ++q) s[q] += block_part[((size_t)b * nc + c) * 4 + q];
    dT[c0 + c] = s[0];
    dP[c0 + c] = s[1];
    dS_acc[c0 + c] = s[2];
    dN_acc[c0 + c] = s[3];
}

// global scalars: sum over conditions in order
__global__ void k_vjp_scalars(const double *dS_acc, const double *dN_acc, int nc, double *ds, double *dn) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < nc; ++c) {
        a += dS_acc[c];
        b += dN_acc[c];
    }
    if (ds) *ds = a;
    if (dn) *dn = b;
}

__global__ void k_to_f32(const double *in, float *out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

typedef void (*VjpFn)(LinesDev, size_t, const CondDev *, int, double, double, int64_t, double, double,
                      const double *, const float *, double *, double *, double *, int);

static VjpFn pick(int prof, bool f64) {
    switch (prof) {
    case XC_DOPPLER: return f64 ? k_vjp_lines<XC_DOPPLER, true> : k_vjp_lines<XC_DOPPLER, false>;
    case XC_LORENTZ: return f64 ? k_vjp_lines<XC_LORENTZ, true> : k_vjp_lines<XC_LORENTZ, false>;
    default: return f64 ? k_vjp_lines<XC_VOIGT_W4, true> : k_vjp_lines<XC_VOIGT_W4, false>;
    }
}

#define VJ_TRY(call)                                                                            \
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

xc_status vjp_run(BatchedState *st, const VjpArgs &a, int64_t *launches) {
    cudaStream_t s = a.stream;
    const int nc = a.n_cond;
    const size_t n = a.n_lines, N = (size_t)a.grid.n;
    const bool f64 = a.opts.precision == XC_FP64_PLAIN;
    const bool host = a.mem == XC_MEM_HOST;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = (int)std::max<size_t>(1, std::min<size_t>((n + VW - 1) / VW, (size_t)nsm * 8));
    // scratch: [grad sigma in device memory][f32 copy][block partials][per-cond acc][outputs]
    size_t off = 0;
    auto carve = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    size_t o_g = host ? carve((size_t)nc * N * 8) : 0;
    size_t o_g32 = f64 ? 0 : carve((size_t)nc * N * 4);
    size_t o_bp = carve((size_t)blocks * VMAXC * 4 * 8);
    size_t o_acc = carve((size_t)nc * 2 * 8);
    size_t o_out = host ? carve((size_t)(2 * nc + 2) * 8 + 2 * n * 8) : 0;
    VJ_TRY(st->vjp_buf.ensure(off + 256));
    char *base = st->vjp_buf.as<char>();
    const double *g64 = a.grad_sigma;
    if (host && nc && N) {
        VJ_TRY(cudaMemcpyAsync(base + o_g, a.grad_sigma, (size_t)nc * N * 8, cudaMemcpyHostToDevice, s));
        g64 = (const double *)(base + o_g);
    }
    float *g32 = f64 ? nullptr : (float *)(base + o_g32);
    double *bp = (double *)(base + o_bp);
    double *dS = (double *)(base + o_acc), *dN = dS + nc;
    double *dT = a.dT, *dP = a.dP, *ds = a.d_gamma_scale, *dn = a.d_n_shift;
    double *dgl = a.d_gamma_ref_line, *dnl = a.d_n_line;
    if (host) {
        double *o = (double *)(base + o_out);
        dT = o;
        dP = o + nc;
        ds = a.d_gamma_scale ? o + 2 * nc : nullptr;
        dn = a.d_n_shift ? o + 2 * nc + 1 : nullptr;
        dgl = a.d_gamma_ref_line ? o + 2 * nc + 2 : nullptr;
        dnl = a.d_n_line ? o + 2 * nc + 2 + n : nullptr;
    }
    if (a.timing) cudaEventRecord(a.ev_begin, s);
    if (nc == 0 || n == 0) {
        if (nc) {
            VJ_TRY(cudaMemsetAsync(dT, 0, nc * 8, s));
            VJ_TRY(cudaMemsetAsync(dP, 0, nc * 8, s));
        }
        if (ds) VJ_TRY(cudaMemsetAsync(ds, 0, 8, s));
        if (dn) VJ_TRY(cudaMemsetAsync(dn, 0, 8, s));
    } else {
        if (!f64 && N) {
            k_to_f32<<<nsm * 4, 256, 0, s>>>(g64, g32, (size_t)nc * N);
            ++*launches;
        }
        for (int c0 = 0; c0 < nc; c0 += VMAXC) {
            int cc = std::min(VMAXC, nc - c0);
            VjpFn fn = pick(a.opts.profile, f64);
            fn<<<blocks, VT, 0, s>>>(a.L, n, a.conds_dev + c0, cc, a.grid.nu_A, a.grid.step, a.grid.n, a.opts.cutoff,
                                     a.opts.width_mult, g64 ? g64 + (size_t)c0 * N : nullptr,
                                     g32 ? g32 + (size_t)c0 * N : nullptr, bp, dgl, dnl, c0 > 0 ? 1 : 0);
            k_vjp_finish<<<1, 32, 0, s>>>(bp, blocks, cc, c0, dT, dP, dS, dN);
            *launches += 2;
        }
        k_vjp_scalars<<<1, 32, 0, s>>>(dS, dN, nc, ds, dn);
        ++*launches;
        VJ_TRY(cudaGetLastError());
    }
    if (a.timing) cudaEventRecord(a.ev_end, s);
    if (host) {
        if (nc) {
            VJ_TRY(cudaMemcpyAsync(a.dT, dT, nc * 8, cudaMemcpyDeviceToHost, s));
            VJ_TRY(cudaMemcpyAsync(a.dP, dP, nc * 8, cudaMemcpyDeviceToHost, s));
        }
        if (a.d_gamma_scale) VJ_TRY(cudaMemcpyAsync(a.d_gamma_scale, ds, 8, cudaMemcpyDeviceToHost, s));
        if (a.d_n_shift) VJ_TRY(cudaMemcpyAsync(a.d_n_shift, dn, 8, cudaMemcpyDeviceToHost, s));
        if (a.d_gamma_ref_line && n) VJ_TRY(cudaMemcpyAsync(a.d_gamma_ref_line, dgl, n * 8, cudaMemcpyDeviceToHost, s));
        if (a.d_n_line && n) VJ_TRY(cudaMemcpyAsync(a.d_n_line, dnl, n * 8, cudaMemcpyDeviceToHost, s));
        VJ_TRY(cudaStreamSynchronize(s));
    }
    return XC_OK;
}

}  // namespace xc
