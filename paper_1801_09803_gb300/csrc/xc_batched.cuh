// xc_batched.cuh -- interface of the FP32 / batched profile kernels and the adjoint.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "xc_internal.cuh"

namespace xc {

constexpr float kKappa = (float)(0.5641896 / 1.772453850905516027);  // w4 region-I constant / sqrt(pi)
constexpr float kSqrtLn2f = 0.8325546111576977f;
constexpr float kSqrtLn2OverPi = 0.46971863934982566f;  // sqrt(ln2/pi)

// Per-condition constants of the FP32 kernels (and the FP32 adjoint), in grid units
struct CParam {
    double inv_scale;   // 1 / scale (power of two)
    float kT_hi, kT_lo; // c2 log2(e) / T as a float pair
    float c2T;          // c2 / T
    float pref;         // abundance / (8 pi c Q) * scale
    float acoef;        // alpha / nu
    float log2Tr;       // log2(T_ref / T)
    float pscale;       // gamma_scale * P / P_ref
    float nshift;
    int row;            // output row (the caller's condition index)
    float dbound;       // upper bound of the far radius D4 over all lines (grid steps)
    float emis;         // 1: emission (pref = abundance h c / (4 pi Q) * scale), 0: absorption
    float vv_split;     // Vectorized Voigt: half-width of the exact zone (cm^-1)
    int vv_beta;        // Vectorized Voigt: 1 = continuity factor beta, 0 = beta 1
};

struct GeomStats {
    unsigned int gA_nu2_bits;  // max g A / nu^2 (float bits; values >= 0)
    unsigned int gA_nu_bits;   // max g A / nu
    unsigned int nu_bits;      // max nu (float, rounded up)
    unsigned int gref_bits;    // max |gamma_ref|
    unsigned int nT_bits;      // max |n_T|
};

__device__ __forceinline__ float rcp_approx(float x) { return recip(x); }

__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// atan2(y, x) for y >= 0 (in [0, pi]), the arctangent of the binned Lorentzian and of the
// binned Gauss-Hermite Voigt (Eqs. eqn:sig_lor-2, e:sigma:quad), whose first argument is
// gamma >= 0.  t = min(|x|, y) / max(|x|, y) in [0, 1]; atan(t) = t q(t^2) with q the
// degree-8 polynomial interpolating atan(sqrt(s)) / sqrt(s) at the 9 Chebyshev nodes of
// s in [0, 1] (derived here in FP64, relative error 1.8e-8); then atan2 = pi/2 - atan(t)
// where y > |x| and pi minus that where x < 0.  In FP32 with the approximate reciprocal
// the result is within a few units in the last place of atan2 (2e-7 relative over
// y in [1e-6, 1e3], |x| in [1e-6, 1e7]); about 20 instructions against ~50 for the
// general library function.  atan2(0, 0) = 0.
__device__ __forceinline__ float atan2_ypos(float y, float x) {
    const float ax = fabsf(x);
    const float mx = fmaxf(ax, y), mn = fminf(ax, y);
    const float t = mx > 0.f ? mn * rcp_approx(mx) : 0.f;
    const float s = t * t;
    float q = 2.766283504e-03f;
    q = fmaf(q, s, -1.573124913e-02f);
    q = fmaf(q, s, 4.213762360e-02f);
    q = fmaf(q, s, -7.456854827e-02f);
    q = fmaf(q, s, 1.061837064e-01f);
    q = fmaf(q, s, -1.419779779e-01f);
    q = fmaf(q, s, 1.999187203e-01f);
    q = fmaf(q, s, -3.333303671e-01f);
    q = fmaf(q, s, 9.999999818e-01f);
    float p = q * t;
    if (y > ax) p = 1.5707963267948966f - p;
    if (x < 0.f) p = 3.141592653589793f - p;
    return p;
}

// 2^(-z) for z >= 0 with the argument split into integer and fraction
__device__ __forceinline__ float exp2_neg(float z) {
    float zi = rintf(z);
    float zf = z - zi;
    if (zi > 125.f) return 0.f;
    float b = ex2_approx(-zf);
    return b * __int_as_float((127 - (int)zi) << 23);
}

// Doppler and Lorentz half-widths in grid steps (Eqs. e:alphaD, e:gamma_L)
__device__ __forceinline__ void line_widths(float nu, float gref, float nT, const CParam &c, float inv_h, float *ah,
                                            float *gh) {
    float al = c.acoef * nu;
    float ga = c.pscale * gref * ex2_approx((nT + c.nshift) * c.log2Tr);
    *ah = __fmul_rn(al, inv_h);
    *gh = __fmul_rn(ga, inv_h);
}

struct BatchedArgs {
    LinesDev L{};
    size_t n_lines = 0;
    const CondDev *conds_dev = nullptr;     // resolved conditions (Q filled) on the device
    const xc_condition *conds_host = nullptr;
    int n_cond = 0;
    xc_grid grid{};
    xc_opts opts{};
    double *sigma = nullptr;                // device, [n_cond][grid.n]
    cudaStream_t stream = nullptr;
    bool timing = false;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
    // with timing: events recorded (as graph event nodes when captured) before the main
    // kernel, after it, and after the centre-zone kernel
    cudaEvent_t ev_main0 = nullptr, ev_main1 = nullptr, ev_core1 = nullptr;
    cudaEvent_t ev_tc1 = nullptr;            // after the tensor-core far-wing kernel (when it runs)
    const double *ghx = nullptr, *ghw = nullptr;  // device Gauss-Hermite nodes/weights
    bool allow_tc = true;                   // far wings may use the tensor-core kernel
};

struct VjpArgs {
    LinesDev L{};
    size_t n_lines = 0;
    const CondDev *conds_dev = nullptr;
    const xc_condition *conds_host = nullptr;
    int n_cond = 0;
    xc_grid grid{};
    xc_opts opts{};
    cudaStream_t stream = nullptr;
    int mem = XC_MEM_DEVICE;
    const double *grad_sigma = nullptr;
    double *dT = nullptr, *dP = nullptr, *d_gamma_scale = nullptr, *d_n_shift = nullptr;
    double *d_gamma_ref_line = nullptr, *d_n_line = nullptr;
    double *d_gamma0_broad = nullptr, *d_n_broad = nullptr;   // per broadener of a mixture (nullable)
    const double *ghx = nullptr, *ghw = nullptr;               // Gauss-Hermite nodes (binned GH), device
    bool timing = false;
    cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
};

// Tile shape of the FP32 gather kernel, chosen by the autotuner.
struct TileCfg {
    int variant = 0;   // index into the compiled kernel table
    int points = 0;    // grid points per window
    int cgroup = 0;    // conditions per tile
    float ms = 0.f;    // autotune measurement
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct BatchedState {
    DevBuf tiles;      // tile table (window, group, line range, cost order)
    DevBuf cparams;    // per-condition constants
    DevBuf counter;    // work-queue counter
    DevBuf vjp_buf;    // adjoint scratch
    DevBuf gsig32;     // grad sigma as float
    DevBuf staging;    // host <-> device staging for the adjoint
    std::map<std::string, TileCfg> tuned;       // autotune cache: shape key -> config
    std::map<std::string, GraphEntry> graphs;   // graph cache: shape key + pointers -> graph
    std::map<std::string, std::string> tune_log; // shape key -> candidate predictions
    std::string last_tuning;                     // description of the last batched configuration
    int *tc_status = nullptr;                    // device word: a tensor-core wait ran out
    // the last run's tensor-core work: super-block line ranges (device) and shape
    const unsigned *tc_blk_lo = nullptr, *tc_blk_hi = nullptr;
    int tc_n_blk = 0, tc_groups = 0;
    int force_R = 0, force_CG = 0;               // fixed CUDA-core tile shape (0: autotune)
};

xc_status batched_run(BatchedState *st, const BatchedArgs &a, int64_t *launches);
// per-line grid geometry for a fixed cut (integer position n_abs, fraction f, inclusive
// cut range [ka, kb]) and the per-condition FP32 constants (in order of increasing
// profile width, each with its caller's row), as the batched FP32 kernels make them
cudaError_t launch_fp32_setup(const LinesDev &L, size_t n, const CondDev *conds, int nc, const xc_grid &grid,
                              double cutoff, int *n_abs, float *f, int *ka, int *kb, GeomStats *gs, CParam *cp,
                              cudaStream_t s);
xc_status vjp_run(BatchedState *st, const VjpArgs &a, int64_t *launches);
// after the stream has synchronised: XC_ETIMEOUT if the tensor-core kernel reported a
// wait that ran out (its results are then not valid), else XC_OK
xc_status batched_check(BatchedState *st);
// after the stream has synchronised: tcgen05.mma instructions the last run's tensor-core
// kernel issued (0 if it did not run), from its super-block line ranges
int64_t batched_tc_mma_count(BatchedState *st);
// (line, grid point, condition) evaluations the tensor-core far-wing kernel takes in a
// batched call with these arguments (0 when that kernel would not run); synchronises
xc_status batched_count_far(BatchedState *st, const BatchedArgs &a, int64_t *count);
void batched_invalidate(BatchedState *st);
void batched_release(BatchedState *st);

}  // namespace xc
