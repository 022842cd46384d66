// xc_api.cu -- the extern "C" boundary of libxc (declared in include/xc.h).
//
// Host code only validates arguments, moves data across the host/device
// boundary, resolves conditions (Q(T) from the states when not given) and
// enqueues kernels; every step of the cross-section path runs in kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "xc_internal.cuh"
#include "xc_batched.cuh"

#include <unistd.h>

#ifndef XC_VERSION_STRING
#define XC_VERSION_STRING "xc 0.1 (sm_103a)"
#endif

namespace xc {

static thread_local std::string g_last_error;

void warm_host_pages(const void *p, size_t bytes) {
    if (!p || bytes < ((size_t)1 << 20)) return;
    static const size_t page = [] {
        const long v = sysconf(_SC_PAGESIZE);
        return v > 0 ? (size_t)v : (size_t)4096;
    }();
    const volatile unsigned char *c = static_cast<const volatile unsigned char *>(p);
    unsigned acc = 0;
    for (size_t o = 0; o < bytes; o += page) acc += c[o];
    acc += c[bytes - 1];
    (void)acc;
}

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

}  // namespace xc

using namespace xc;

struct xc_handle {
    int device = 0;
    size_t n_lines = 0, cap_lines = 0;
    double *nu = nullptr;
    float *elower = nullptr, *A = nullptr, *gamma_ref = nullptr, *n_T = nullptr;
    int16_t *g_up = nullptr, *j_lo = nullptr;
    uint32_t *perm = nullptr;
    double *st_E = nullptr;
    int32_t *st_g = nullptr;
    size_t n_states = 0;
    int *d_flag = nullptr;
    DevBuf sort_tmp[5];
    DevBuf stage_in;         // unsorted host lines copied to the device
    DevBuf params;           // FP64 per-line I, alpha, gamma, cut
    DevBuf ranges;           // window line ranges
    DevBuf conds;            // CondDev[]
    DevBuf qtab;             // T, Q, dQ for unique temperatures
    DevBuf out;              // device staging of outputs for host destinations
    DevBuf gh;               // Gauss-Hermite nodes (x then w)
    DevBuf misc;             // counters
    DevBuf vjp;              // adjoint scratch
    DevBuf broad;            // broadener mixture: per broadener rho gamma_0 and n_L per line, tables
    int n_broad = 0;         // broadeners in use (0: the line list's gamma_ref, n_T)
    int gh_n = 0;
    bool timing = false;
    cudaEvent_t ev[2 * ST_COUNT + 4] = {};
    float last_ms[ST_COUNT] = {};
    double kernel_ms[3] = {-1.0, -1.0, -1.0};   // last FP32 sweep: far-wing (tensor), main, centre zone
    int64_t tc_mma = 0;
    int64_t launches = 0;
    BatchedState batched;
};

namespace {

#define XC_TRY(call)                                                                           \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) {                                                               \
            set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
            return XC_ECUDA;                                                                   \
        }                                                                                      \
    } while (0)

#define XC_TRY_MEM(call)                                                                       \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e == cudaErrorMemoryAllocation) {                                                 \
            cudaGetLastError();                                                                \
            set_error("device allocation failed: %s", #call);                                  \
            return XC_ENOMEM;                                                                  \
        }                                                                                      \
        if (_e != cudaSuccess) {                                                               \
            set_error("%s failed: %s", #call, cudaGetErrorString(_e));                         \
            return XC_ECUDA;                                                                   \
        }                                                                                      \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

void stage_begin(xc_handle *h, int st, cudaStream_t s) {
    if (h->timing) cudaEventRecord(h->ev[2 * st], s);
}
void stage_end(xc_handle *h, int st, cudaStream_t s) {
    if (h->timing) cudaEventRecord(h->ev[2 * st + 1], s);
}

void reset_timing(xc_handle *h) {
    for (int i = 0; i < ST_COUNT; ++i) h->last_ms[i] = 0.f;
    h->launches = 0;
}

// called after the stream was synchronised
void collect_timing(xc_handle *h, const bool *used) {
    if (!h->timing) return;
    for (int i = 0; i < ST_COUNT; ++i) {
        if (!used[i]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) h->last_ms[i] = ms;
        else cudaGetLastError();
    }
}

xc_status check_handle(const xc_handle *h) {
    if (!h) {
        set_error("NULL handle");
        return XC_EINVAL;
    }
    return XC_OK;
}

xc_status check_grid(const xc_grid *g) {
    if (!g) { set_error("NULL grid"); return XC_EINVAL; }
    if (g->n < 0) { set_error("grid n < 0"); return XC_EINVAL; }
    if (!(g->step > 0.0) || !isfinite(g->step) || !isfinite(g->nu_A)) {
        set_error("grid step must be > 0 and finite");
        return XC_EINVAL;
    }
    if (g->n > ((int64_t)1 << 40)) { set_error("grid too large"); return XC_EINVAL; }
    return XC_OK;
}

xc_status check_opts(const xc_opts *o) {
    if (!o) { set_error("NULL opts"); return XC_EINVAL; }
    if (o->profile < XC_DOPPLER || o->profile > XC_VOIGT_VV) {
        set_error("unknown profile %d", o->profile);
        return XC_EUNSUPPORTED;
    }
    if (o->precision != XC_FP64_PLAIN && o->precision != XC_FP32) {
        set_error("unknown precision %d", o->precision);
        return XC_EUNSUPPORTED;
    }
    if (!(o->cutoff > 0.0) || !isfinite(o->cutoff)) { set_error("cutoff must be > 0"); return XC_EINVAL; }
    if (o->width_mult < 0.0 || !isfinite(o->width_mult)) { set_error("width_mult must be >= 0"); return XC_EINVAL; }
    if (o->flags & ~XC_OPT_NO_TENSOR_CORES) { set_error("unknown opts flags 0x%x", (unsigned)o->flags); return XC_EINVAL; }
    if ((o->profile == XC_VOIGT_GH_BINNED || o->profile == XC_VOIGT_GH_SAMPLED) && (o->n_gh < 1 || o->n_gh > 64)) {
        set_error("n_gh must be in 1..64");
        return XC_EINVAL;
    }
    if (o->quantity != XC_ABSORPTION && o->quantity != XC_EMISSION) {
        set_error("unknown quantity %d", o->quantity);
        return XC_EINVAL;
    }
    if (o->threshold < XC_THRESHOLD_NONE || o->threshold > XC_THRESHOLD_HITRAN) {
        set_error("unknown threshold mode %d", o->threshold);
        return XC_EINVAL;
    }
    if (o->threshold == XC_THRESHOLD_CONSTANT && !(o->I_cut >= 0.0 && isfinite(o->I_cut))) {
        set_error("I_cut must be finite and >= 0");
        return XC_EINVAL;
    }
    if (!(o->vv_split >= 0.0) || !isfinite(o->vv_split) || (o->vv_flags & ~(XC_VV_BETA | XC_VV_NORMALISE))) {
        set_error("vv_split must be finite and >= 0, vv_flags XC_VV_* bits");
        return XC_EINVAL;
    }
    if (o->threshold == XC_THRESHOLD_HITRAN &&
        !(o->nu_crit > 0.0 && isfinite(o->nu_crit) && o->I_crit >= 0.0 && isfinite(o->I_crit))) {
        set_error("the HITRAN threshold needs nu_crit > 0 and a finite I_crit >= 0");
        return XC_EINVAL;
    }
    return XC_OK;
}

xc_status check_conds(const xc_condition *c, size_t n, const xc_handle *h) {
    if (!c && n) { set_error("NULL conditions"); return XC_EINVAL; }
    for (size_t i = 0; i < n; ++i) {
        const xc_condition &d = c[i];
        if (!(d.T > 0.0) || !isfinite(d.T)) { set_error("condition %zu: T must be > 0", i); return XC_EINVAL; }
        if (!(d.P >= 0.0) || !isfinite(d.P)) { set_error("condition %zu: P must be >= 0", i); return XC_EINVAL; }
        if (!(d.mass_da > 0.0) || !(d.T_ref > 0.0) || !(d.P_ref > 0.0)) {
            set_error("condition %zu: mass_da, T_ref, P_ref must be > 0", i);
            return XC_EINVAL;
        }
        if (!(d.gamma_scale >= 0.0) || !isfinite(d.n_shift) || !(d.abundance >= 0.0)) {
            set_error("condition %zu: bad gamma_scale / n_shift / abundance", i);
            return XC_EINVAL;
        }
        if (d.Q <= 0.0 && (!h || h->n_states == 0)) {
            set_error("condition %zu: Q <= 0 needs states (xc_set_states)", i);
            return XC_EINVAL;
        }
    }
    return XC_OK;
}

// Upload conditions and fill Q, dQ/dT for those with Q <= 0 from the states,
// one Q(T) evaluation per distinct temperature.  Returns the device CondDev array.
__global__ void k_fill_conds(CondDev *c, int n, const int *tix, const double *Q, const double *dQ) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || tix[i] < 0) return;
    c[i].Q = Q[tix[i]];
    c[i].dQdT = dQ[tix[i]];
}

xc_status resolve_conds(xc_handle *h, const xc_condition *conds, size_t n, cudaStream_t s, CondDev **out) {
    std::vector<CondDev> hc(n);
    std::vector<double> uT;
    std::vector<int> tix(n, -1);
    for (size_t i = 0; i < n; ++i) {
        const xc_condition &c = conds[i];
        hc[i] = CondDev{c.T, c.P, c.Q, c.dQdT, c.mass_da, c.T_ref, c.P_ref, c.gamma_scale, c.n_shift, c.abundance};
        if (c.Q <= 0.0) {
            auto it = std::find(uT.begin(), uT.end(), c.T);
            if (it == uT.end()) {
                tix[i] = (int)uT.size();
                uT.push_back(c.T);
            } else {
                tix[i] = (int)(it - uT.begin());
            }
        }
    }
    size_t nT = uT.size();
    size_t bytes_c = n * sizeof(CondDev);
    size_t off_q = (bytes_c + 255) & ~size_t(255);
    size_t need = off_q + 3 * nT * sizeof(double) + n * sizeof(int) + 64;
    XC_TRY_MEM(h->conds.ensure(need));
    char *base = h->conds.as<char>();
    CondDev *dc = reinterpret_cast<CondDev *>(base);
    double *dT = reinterpret_cast<double *>(base + off_q);
    double *dQ = dT + nT, *ddQ = dQ + nT;
    int *dtix = reinterpret_cast<int *>(ddQ + nT);
    // pageable host -> device copies of small parameter blocks (stream-ordered)
    XC_TRY(cudaMemcpyAsync(dc, hc.data(), bytes_c, cudaMemcpyHostToDevice, s));
    if (nT) {
        XC_TRY(cudaMemcpyAsync(dT, uT.data(), nT * sizeof(double), cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(dtix, tix.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
        stage_begin(h, ST_Q, s);
        XC_TRY(launch_partition_function(h->st_E, h->st_g, h->n_states, dT, (int)nT, dQ, ddQ, s));
        k_fill_conds<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(dc, (int)n, dtix, dQ, ddQ);
        XC_TRY(cudaGetLastError());
        stage_end(h, ST_Q, s);
        h->launches += 2;
    }
    *out = dc;
    return XC_OK;
}

LinesDev lines_of(const xc_handle *h) {
    LinesDev L{h->nu, h->elower, h->A, h->gamma_ref, h->n_T, h->g_up, h->j_lo};
    if (h->n_broad > 0) {
        L.bgam = h->broad.as<double>();
        L.bn = L.bgam + (size_t)h->n_broad * h->n_lines;
        L.bstride = h->n_lines;
        L.n_broad = h->n_broad;
    }
    return L;
}

xc_status ensure_gh(xc_handle *h, int n, cudaStream_t s) {
    if (h->gh_n == n) return XC_OK;
    XC_TRY_MEM(h->gh.ensure(2 * 64 * sizeof(double)));
    XC_TRY(launch_gh_nodes(n, h->gh.as<double>(), h->gh.as<double>() + 64, s));
    h->launches += 1;
    h->gh_n = n;
    return XC_OK;
}

// FP64 plain cross section of one (already resolved) condition into device memory
xc_status cross_section_f64(xc_handle *h, const CondDev *dcond, const xc_grid *g, const xc_opts *o, double *sig,
                            cudaStream_t s) {
    const size_t n = h->n_lines;
    const int64_t W = 256;
    const int64_t n_win = (g->n + W - 1) / W;
    if (g->n == 0) return XC_OK;
    if (n == 0) {
        XC_TRY(cudaMemsetAsync(sig, 0, g->n * sizeof(double), s));
        return XC_OK;
    }
    XC_TRY_MEM(h->params.ensure(n * 4 * sizeof(double)));
    XC_TRY_MEM(h->ranges.ensure(n_win * 2 * sizeof(int64_t)));
    double *I = h->params.as<double>(), *al = I + n, *ga = al + n, *cut = ga + n;
    int64_t *lo = h->ranges.as<int64_t>(), *hi = lo + n_win;
    stage_begin(h, ST_PARAMS, s);
    XC_TRY(launch_line_params64(lines_of(h), n, dcond, o->width_mult > 0.0 ? 1 : 0, o->cutoff, o->width_mult, I, al,
                                ga, cut, s, strength_sel(*o)));
    stage_end(h, ST_PARAMS, s);
    stage_begin(h, ST_RANGES, s);
    XC_TRY(launch_window_ranges(h->nu, n, g->nu_A, g->step, g->n, W, o->cutoff, n_win, lo, hi, s));
    stage_end(h, ST_RANGES, s);
    const double *ghx = nullptr, *ghw = nullptr;
    if (o->profile == XC_VOIGT_GH_BINNED || o->profile == XC_VOIGT_GH_SAMPLED) {
        xc_status st = ensure_gh(h, o->n_gh, s);
        if (st != XC_OK) return st;
        ghx = h->gh.as<double>();
        ghw = ghx + 64;
    }
    const double vv_split = o->vv_split > 0.0 ? o->vv_split : 4.0;
    const int vv_beta = (o->vv_flags & XC_VV_BETA) ? 1 : 0;
    if (o->profile == XC_VOIGT_VV && (o->vv_flags & XC_VV_NORMALISE)) {
        XC_TRY(launch_vv_norm64(h->nu, I, al, ga, cut, n, g->nu_A, g->step, vv_split, vv_beta, s));
        h->launches += 1;
    }
    stage_begin(h, ST_PROFILE, s);
    XC_TRY(launch_gather_f64(o->profile, h->nu, I, al, ga, cut, lo, hi, n_win, g->nu_A, g->step, g->n, ghx, ghw,
                             ghx ? o->n_gh : 0, sig, s, vv_split, vv_beta));
    stage_end(h, ST_PROFILE, s);
    h->launches += 3;
    return XC_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char *xc_version(void) { return XC_VERSION_STRING; }

const char *xc_last_error(void) { return g_last_error.c_str(); }

xc_status xc_create(xc_handle **out, int device) {
    if (!out) { set_error("NULL out"); return XC_EINVAL; }
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        set_error("cudaGetDeviceCount: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return XC_ECUDA;
    }
    if (device < 0 || device >= ndev) { set_error("device %d out of range (%d devices)", device, ndev); return XC_EINVAL; }
    DeviceGuard dg(device);
    xc_handle *h = new (std::nothrow) xc_handle();
    if (!h) { set_error("host allocation failed"); return XC_ENOMEM; }
    h->device = device;
    for (auto &ev : h->ev) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            set_error("cudaEventCreate failed");
            xc_destroy(h);
            return XC_ECUDA;
        }
    }
    if (cudaMalloc(&h->d_flag, 64) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc failed");
        xc_destroy(h);
        return XC_ENOMEM;
    }
    *out = h;
    return XC_OK;
}

static void free_lines(xc_handle *h) {
    cudaFree(h->nu);
    cudaFree(h->elower);
    cudaFree(h->A);
    cudaFree(h->gamma_ref);
    cudaFree(h->n_T);
    cudaFree(h->g_up);
    cudaFree(h->j_lo);
    cudaFree(h->perm);
    h->nu = nullptr; h->elower = h->A = h->gamma_ref = h->n_T = nullptr;
    h->g_up = h->j_lo = nullptr; h->perm = nullptr;
    h->cap_lines = h->n_lines = 0;
}

xc_status xc_destroy(xc_handle *h) {
    if (!h) return XC_OK;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    free_lines(h);
    cudaFree(h->st_E);
    cudaFree(h->st_g);
    cudaFree(h->d_flag);
    for (auto &b : h->sort_tmp) b.release();
    h->stage_in.release();
    h->params.release();
    h->ranges.release();
    h->conds.release();
    h->qtab.release();
    h->out.release();
    h->gh.release();
    h->misc.release();
    h->vjp.release();
    h->broad.release();
    batched_release(&h->batched);
    for (auto &ev : h->ev)
        if (ev) cudaEventDestroy(ev);
    delete h;
    cudaGetLastError();
    return XC_OK;
}

xc_status xc_load_lines(xc_handle *h, const xc_lines *L, size_t n, unsigned flags, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!L) { set_error("NULL lines"); return XC_EINVAL; }
    if (n >= ((size_t)1 << 32)) { set_error("at most 2^32 - 1 lines"); return XC_EINVAL; }
    if (n && (!L->nu || !L->elower || !L->A || !L->gamma_ref || !L->n_T || !L->g_up)) {
        set_error("NULL line array");
        return XC_EINVAL;
    }
    if (L->mem != XC_MEM_HOST && L->mem != XC_MEM_DEVICE) { set_error("bad mem flag"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    reset_timing(h);
    if (n > h->cap_lines) {
        free_lines(h);
        XC_TRY_MEM(cudaMalloc(&h->nu, n * 8));
        XC_TRY_MEM(cudaMalloc(&h->elower, n * 4));
        XC_TRY_MEM(cudaMalloc(&h->A, n * 4));
        XC_TRY_MEM(cudaMalloc(&h->gamma_ref, n * 4));
        XC_TRY_MEM(cudaMalloc(&h->n_T, n * 4));
        XC_TRY_MEM(cudaMalloc(&h->g_up, n * 2));
        XC_TRY_MEM(cudaMalloc(&h->j_lo, n * 2));
        XC_TRY_MEM(cudaMalloc(&h->perm, n * 4));
        h->cap_lines = n;
    }
    h->n_lines = 0;
    h->n_broad = 0;   // a broadener mixture belongs to the lines it was set for
    // graphs and tuning stay valid: they key on shapes and buffer addresses, and read the
    // line data when replayed
    if (n == 0) return XC_OK;
    LinesDev in{L->nu, L->elower, L->A, L->gamma_ref, L->n_T, L->g_up, L->j_lo};
    bool used[ST_COUNT] = {};
    if (L->mem == XC_MEM_HOST) {
        // host -> device copy of the unsorted list (the host/device boundary)
        XC_TRY_MEM(h->stage_in.ensure(n * 28 + 7 * 256));
        char *p = h->stage_in.as<char>();
        auto take = [&](size_t bytes) { char *q = p; p += (bytes + 255) & ~size_t(255); return q; };
        double *nu = (double *)take(n * 8);
        float *e = (float *)take(n * 4), *a = (float *)take(n * 4), *gr = (float *)take(n * 4),
              *nt = (float *)take(n * 4);
        int16_t *g = (int16_t *)take(n * 2), *j = (int16_t *)take(n * 2);
        const void *src[7] = {L->nu, L->elower, L->A, L->gamma_ref, L->n_T, L->g_up, L->j_lo};
        const size_t sz[7] = {n * 8, n * 4, n * 4, n * 4, n * 4, n * 2, n * 2};
        for (int f = 0; f < 7; ++f) warm_host_pages(src[f], sz[f]);
        stage_begin(h, ST_FINISH, s);
        XC_TRY(cudaMemcpyAsync(nu, L->nu, n * 8, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(e, L->elower, n * 4, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(a, L->A, n * 4, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(gr, L->gamma_ref, n * 4, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(nt, L->n_T, n * 4, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(g, L->g_up, n * 2, cudaMemcpyHostToDevice, s));
        if (L->j_lo) XC_TRY(cudaMemcpyAsync(j, L->j_lo, n * 2, cudaMemcpyHostToDevice, s));
        stage_end(h, ST_FINISH, s);
        used[ST_FINISH] = true;
        in = LinesDev{nu, e, a, gr, nt, g, L->j_lo ? j : nullptr};
    }
    bool bad = false, unsorted = false;
    cudaEvent_t ev3[3] = {h->ev[2 * ST_SORT], h->ev[2 * ST_SORT + 1], h->ev[2 * ST_GATHER + 1]};
    cudaError_t e = launch_sort_lines(in, n, (flags & XC_ASSUME_SORTED) != 0, h->sort_tmp, h->nu, h->elower, h->A,
                                      h->gamma_ref, h->n_T, h->g_up, h->j_lo, h->perm, h->d_flag, s,
                                      h->timing ? ev3 : nullptr, &h->launches, &bad, &unsorted);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        set_error("sort scratch allocation failed");
        return XC_ENOMEM;
    }
    if (e != cudaSuccess) { set_error("sort failed: %s", cudaGetErrorString(e)); return XC_ECUDA; }
    if (h->timing) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev3[0], ev3[1]) == cudaSuccess) h->last_ms[ST_SORT] = ms;
        if (cudaEventElapsedTime(&ms, ev3[1], ev3[2]) == cudaSuccess) h->last_ms[ST_GATHER] = ms;
        cudaGetLastError();
    }
    collect_timing(h, used);
    if (bad) {
        set_error("invalid line values (need finite nu > 0, A >= 0, gamma_ref >= 0, finite E'' >= 0 and n_T, g >= 0)");
        return XC_EINVAL;
    }
    if (unsorted) { set_error("XC_ASSUME_SORTED given but nu is not sorted"); return XC_EINVAL; }
    h->n_lines = n;
    return XC_OK;
}

xc_status xc_num_lines(const xc_handle *h, size_t *n_out) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!n_out) { set_error("NULL out"); return XC_EINVAL; }
    *n_out = h->n_lines;
    return XC_OK;
}

xc_status xc_get_lines(xc_handle *h, double *nu, float *elower, float *A, float *gamma_ref, float *n_T,
                       int16_t *g_up, int16_t *j_lo, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    cudaMemcpyKind k = mem == XC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    size_t n = h->n_lines;
    if (n == 0) return XC_OK;
    if (nu) XC_TRY(cudaMemcpyAsync(nu, h->nu, n * 8, k, s));
    if (elower) XC_TRY(cudaMemcpyAsync(elower, h->elower, n * 4, k, s));
    if (A) XC_TRY(cudaMemcpyAsync(A, h->A, n * 4, k, s));
    if (gamma_ref) XC_TRY(cudaMemcpyAsync(gamma_ref, h->gamma_ref, n * 4, k, s));
    if (n_T) XC_TRY(cudaMemcpyAsync(n_T, h->n_T, n * 4, k, s));
    if (g_up) XC_TRY(cudaMemcpyAsync(g_up, h->g_up, n * 2, k, s));
    if (j_lo) XC_TRY(cudaMemcpyAsync(j_lo, h->j_lo, n * 2, k, s));
    if (mem == XC_MEM_HOST) XC_TRY(cudaStreamSynchronize(s));
    return XC_OK;
}

xc_status xc_set_broadening(xc_handle *h, const xc_broadener *b, int n_broadeners, const int16_t *j_up, int mem,
                            void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (n_broadeners < 0 || n_broadeners > 8) { set_error("0..8 broadeners"); return XC_EINVAL; }
    if (n_broadeners > 0 && !b) { set_error("NULL broadeners"); return XC_EINVAL; }
    if (mem != XC_MEM_HOST && mem != XC_MEM_DEVICE) { set_error("bad mem flag"); return XC_EINVAL; }
    // host tables: per broadener its rows sorted by key (a0: J'', a1: J'' * 65536 + J')
    const int nb = n_broadeners;
    std::vector<int> type(nb), row0(nb + 1, 0);
    std::vector<double> frac(nb), gdef(nb), ndef(nb);
    std::vector<int64_t> keys;
    std::vector<double> g0, nl;
    bool need_jup = false;
    for (int i = 0; i < nb; ++i) {
        const xc_broadener &x = b[i];
        if (x.type != XC_BROAD_CONSTANT && x.type != XC_BROAD_A0 && x.type != XC_BROAD_A1) {
            set_error("broadener %d: unknown type %d", i, x.type);
            return XC_EINVAL;
        }
        if (!(x.fraction >= 0.0) || !isfinite(x.fraction) || !(x.gamma0 >= 0.0) || !isfinite(x.gamma0) ||
            !isfinite(x.n)) {
            set_error("broadener %d: fraction and gamma0 must be finite and >= 0, n finite", i);
            return XC_EINVAL;
        }
        type[i] = x.type;
        frac[i] = x.fraction;
        gdef[i] = x.gamma0;
        ndef[i] = x.n;
        std::vector<std::pair<int64_t, int64_t>> rows;   // (key, row)
        if (x.type != XC_BROAD_CONSTANT) {
            if (x.n_entries < 0 || x.n_entries > (1 << 20)) { set_error("broadener %d: 0..2^20 rows", i); return XC_EINVAL; }
            if (x.n_entries > 0 && (!x.j_lo || !x.gamma0_j || !x.n_j || (x.type == XC_BROAD_A1 && !x.j_up))) {
                set_error("broadener %d: NULL table array", i);
                return XC_EINVAL;
            }
            for (int64_t r = 0; r < x.n_entries; ++r) {
                if (!(x.gamma0_j[r] >= 0.0) || !isfinite(x.gamma0_j[r]) || !isfinite(x.n_j[r]) ||
                    x.j_lo[r] < 0 || x.j_lo[r] > 32767 || (x.type == XC_BROAD_A1 && (x.j_up[r] < 0 || x.j_up[r] > 32767))) {
                    set_error("broadener %d row %lld: bad values", i, (long long)r);
                    return XC_EINVAL;
                }
                const int64_t key = x.type == XC_BROAD_A1 ? (int64_t)x.j_lo[r] * 65536 + x.j_up[r] : (int64_t)x.j_lo[r];
                rows.emplace_back(key, r);
            }
            std::sort(rows.begin(), rows.end());
            for (size_t r = 1; r < rows.size(); ++r)
                if (rows[r].first == rows[r - 1].first) { set_error("broadener %d: duplicate key", i); return XC_EINVAL; }
            need_jup |= x.type == XC_BROAD_A1 && x.n_entries > 0;
        }
        for (auto &kr : rows) {
            keys.push_back(kr.first);
            g0.push_back(x.gamma0_j[kr.second]);
            nl.push_back(x.n_j[kr.second]);
        }
        row0[i + 1] = (int)keys.size();
    }
    if (need_jup && !j_up && h->n_lines) { set_error("an a1 broadener needs j_up"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    h->n_broad = 0;
    const size_t n = h->n_lines;
    if (nb == 0 || n == 0) return XC_OK;
    // device layout: bgam [nb][n], bn [nb][n], J' sorted [n], then the tables
    const size_t nr = keys.size();
    // bn follows bgam with no gap (lines_of finds it there)
    const size_t o_bg = 0, o_bn = (size_t)nb * n * 8;
    size_t off = 2 * (size_t)nb * n * 8;
    auto carve = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        size_t o = off;
        off += bytes;
        return o;
    };
    const size_t o_ju = carve(n * 2),
                 o_jin = carve(n * 2), o_type = carve(nb * 4), o_row0 = carve((nb + 1) * 4), o_frac = carve(nb * 8),
                 o_gdef = carve(nb * 8), o_ndef = carve(nb * 8), o_keys = carve(nr * 8 + 8), o_g0 = carve(nr * 8 + 8),
                 o_nl = carve(nr * 8 + 8);
    XC_TRY_MEM(h->broad.ensure(off));
    char *d = h->broad.as<char>();
    int16_t *jus = nullptr;
    if (j_up) {
        const int16_t *jin = j_up;
        if (mem == XC_MEM_HOST) {
            XC_TRY(cudaMemcpyAsync(d + o_jin, j_up, n * 2, cudaMemcpyHostToDevice, s));
            jin = (const int16_t *)(d + o_jin);
        }
        jus = (int16_t *)(d + o_ju);
        XC_TRY(launch_permute_i16(jin, h->perm, n, jus, s));
    }
    XC_TRY(cudaMemcpyAsync(d + o_type, type.data(), nb * 4, cudaMemcpyHostToDevice, s));
    XC_TRY(cudaMemcpyAsync(d + o_row0, row0.data(), (nb + 1) * 4, cudaMemcpyHostToDevice, s));
    XC_TRY(cudaMemcpyAsync(d + o_frac, frac.data(), nb * 8, cudaMemcpyHostToDevice, s));
    XC_TRY(cudaMemcpyAsync(d + o_gdef, gdef.data(), nb * 8, cudaMemcpyHostToDevice, s));
    XC_TRY(cudaMemcpyAsync(d + o_ndef, ndef.data(), nb * 8, cudaMemcpyHostToDevice, s));
    if (nr) {
        XC_TRY(cudaMemcpyAsync(d + o_keys, keys.data(), nr * 8, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(d + o_g0, g0.data(), nr * 8, cudaMemcpyHostToDevice, s));
        XC_TRY(cudaMemcpyAsync(d + o_nl, nl.data(), nr * 8, cudaMemcpyHostToDevice, s));
    }
    XC_TRY(launch_apply_broadening(h->j_lo, jus, n, nb, (const int *)(d + o_type), (const double *)(d + o_frac),
                                   (const double *)(d + o_gdef), (const double *)(d + o_ndef),
                                   (const int *)(d + o_row0), (const int64_t *)(d + o_keys),
                                   (const double *)(d + o_g0), (const double *)(d + o_nl), (double *)(d + o_bg),
                                   (double *)(d + o_bn), s));
    h->launches += j_up ? 2 : 1;
    XC_TRY(cudaStreamSynchronize(s));   // the host tables above live on this stack frame
    h->n_broad = nb;
    return XC_OK;
}

xc_status xc_get_permutation(xc_handle *h, uint32_t *perm_out, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!perm_out && h->n_lines) { set_error("NULL out"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    if (h->n_lines == 0) return XC_OK;
    XC_TRY(cudaMemcpyAsync(perm_out, h->perm, h->n_lines * 4,
                           mem == XC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    if (mem == XC_MEM_HOST) XC_TRY(cudaStreamSynchronize(s));
    return XC_OK;
}

xc_status xc_set_states(xc_handle *h, const double *E, const int32_t *g, size_t n_states, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (n_states && (!E || !g)) { set_error("NULL states"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    cudaFree(h->st_E);
    cudaFree(h->st_g);
    h->st_E = nullptr;
    h->st_g = nullptr;
    h->n_states = 0;
    if (!n_states) return XC_OK;
    XC_TRY_MEM(cudaMalloc(&h->st_E, n_states * 8));
    XC_TRY_MEM(cudaMalloc(&h->st_g, n_states * 4));
    cudaMemcpyKind k = mem == XC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    XC_TRY(cudaMemcpyAsync(h->st_E, E, n_states * 8, k, s));
    XC_TRY(cudaMemcpyAsync(h->st_g, g, n_states * 4, k, s));
    XC_TRY(cudaStreamSynchronize(s));
    h->n_states = n_states;
    return XC_OK;
}

xc_status xc_partition_function(const double *E, const int32_t *g, size_t n_states, const double *T, size_t nT,
                                double *Q_out, double *dQdT_out, int mem, void *stream) {
    if (nT && (!T || !Q_out)) { set_error("NULL T or Q_out"); return XC_EINVAL; }
    if (n_states && (!E || !g)) { set_error("NULL states"); return XC_EINVAL; }
    if (nT > (1u << 20)) { set_error("too many temperatures"); return XC_EINVAL; }
    if (nT == 0) return XC_OK;
    cudaStream_t s = S(stream);
    if (mem == XC_MEM_HOST) {
        for (size_t i = 0; i < nT; ++i)
            if (!(T[i] > 0.0) || !isfinite(T[i])) { set_error("T[%zu] must be > 0", i); return XC_EINVAL; }
        void *buf = nullptr;
        size_t bytes = n_states * 12 + nT * 24 + 64;
        XC_TRY_MEM(cudaMalloc(&buf, bytes));
        double *dE = (double *)buf;
        double *dT = dE + n_states, *dQ = dT + nT, *ddQ = dQ + nT;
        int32_t *dg = (int32_t *)(ddQ + nT);
        cudaError_t e = cudaSuccess;
        if (n_states) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(dE, E, n_states * 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dg, g, n_states * 4, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(dT, T, nT * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_partition_function(dE, dg, n_states, dT, (int)nT, dQ, ddQ, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Q_out, dQ, nT * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && dQdT_out) e = cudaMemcpyAsync(dQdT_out, ddQ, nT * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(buf);
        if (e != cudaSuccess) { set_error("partition function: %s", cudaGetErrorString(e)); return XC_ECUDA; }
        return XC_OK;
    }
    XC_TRY(launch_partition_function(E, g, n_states, T, (int)nT, Q_out, dQdT_out, s));
    return XC_OK;
}

xc_status xc_line_params(xc_handle *h, const xc_condition *cond, double *I_out, double *alpha_out,
                         double *gamma_out, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if ((st = check_conds(cond, 1, h))) return st;
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    reset_timing(h);
    const size_t n = h->n_lines;
    if (n == 0) return XC_OK;
    CondDev *dc = nullptr;
    if ((st = resolve_conds(h, cond, 1, s, &dc))) return st;
    double *I = I_out, *al = alpha_out, *ga = gamma_out;
    if (mem == XC_MEM_HOST) {
        XC_TRY_MEM(h->out.ensure(n * 3 * sizeof(double)));
        I = h->out.as<double>();
        al = I + n;
        ga = al + n;
    }
    bool used[ST_COUNT] = {};
    used[ST_PARAMS] = true;
    used[ST_Q] = cond->Q <= 0.0;
    stage_begin(h, ST_PARAMS, s);
    XC_TRY(launch_line_params64(lines_of(h), n, dc, 0, 25.0, 0.0, I_out ? I : nullptr, alpha_out ? al : nullptr,
                                gamma_out ? ga : nullptr, nullptr, s));
    stage_end(h, ST_PARAMS, s);
    h->launches += 1;
    if (mem == XC_MEM_HOST) {
        if (I_out) XC_TRY(cudaMemcpyAsync(I_out, I, n * 8, cudaMemcpyDeviceToHost, s));
        if (alpha_out) XC_TRY(cudaMemcpyAsync(alpha_out, al, n * 8, cudaMemcpyDeviceToHost, s));
        if (gamma_out) XC_TRY(cudaMemcpyAsync(gamma_out, ga, n * 8, cudaMemcpyDeviceToHost, s));
    }
    XC_TRY(cudaStreamSynchronize(s));
    collect_timing(h, used);
    return XC_OK;
}

xc_status xc_count_evals(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                         const xc_opts *opts, int64_t *count_out, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if ((st = check_grid(grid)) || (st = check_opts(opts)) || (st = check_conds(conds, n_cond, h))) return st;
    if (!count_out) { set_error("NULL out"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    *count_out = 0;
    if (h->n_lines == 0 || n_cond == 0 || grid->n == 0) return XC_OK;
    CondDev *dc = nullptr;
    if ((st = resolve_conds(h, conds, n_cond, s, &dc))) return st;
    XC_TRY_MEM(h->misc.ensure(64));
    unsigned long long *cnt = h->misc.as<unsigned long long>();
    XC_TRY(launch_count_evals(lines_of(h), h->n_lines, dc, (int)n_cond, grid->nu_A, grid->step, grid->n,
                              opts->cutoff, opts->width_mult, cnt, s));
    unsigned long long hc = 0;
    XC_TRY(cudaMemcpyAsync(&hc, cnt, 8, cudaMemcpyDeviceToHost, s));
    XC_TRY(cudaStreamSynchronize(s));
    *count_out = (int64_t)hc;
    return XC_OK;
}

xc_status xc_cross_section(xc_handle *h, const xc_condition *cond, const xc_grid *grid, const xc_opts *opts,
                           double *sigma_out, int mem, void *stream) {
    return xc_cross_section_batched(h, cond, 1, grid, opts, sigma_out, mem, stream);
}

xc_status xc_cross_section_batched(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                                   const xc_opts *opts, double *sigma_out, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if ((st = check_grid(grid)) || (st = check_opts(opts)) || (st = check_conds(conds, n_cond, h))) return st;
    if (n_cond > 4096) { set_error("at most 4096 conditions per call"); return XC_EINVAL; }
    if (grid->n > 0 && n_cond > 0 && !sigma_out) { set_error("NULL sigma_out"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    reset_timing(h);
    if (grid->n == 0 || n_cond == 0) return XC_OK;
    const size_t total = (size_t)n_cond * (size_t)grid->n;
    double *sig = sigma_out;
    if (mem == XC_MEM_HOST) {
        XC_TRY_MEM(h->out.ensure(total * sizeof(double)));
        sig = h->out.as<double>();
    }
    bool used[ST_COUNT] = {};
    bool anyQ = false;
    for (size_t c = 0; c < n_cond; ++c) anyQ |= conds[c].Q <= 0.0;
    used[ST_Q] = anyQ;
    CondDev *dc = nullptr;
    if ((st = resolve_conds(h, conds, n_cond, s, &dc))) return st;
    if (opts->precision == XC_FP64_PLAIN || h->n_lines == 0) {
        for (size_t c = 0; c < n_cond; ++c) {
            if ((st = cross_section_f64(h, dc + c, grid, opts, sig + c * grid->n, s))) return st;
        }
        used[ST_PARAMS] = used[ST_RANGES] = used[ST_PROFILE] = h->n_lines > 0;
    } else {
        BatchedArgs a;
        a.L = lines_of(h);
        a.n_lines = h->n_lines;
        a.conds_dev = dc;
        a.conds_host = conds;
        a.n_cond = (int)n_cond;
        a.grid = *grid;
        a.opts = *opts;
        a.sigma = sig;
        a.stream = s;
        a.timing = h->timing;
        a.ev_begin = h->ev[2 * ST_PARAMS];          // whole sweep (setup + kernels)
        a.ev_end = h->ev[2 * ST_PARAMS + 1];
        a.ev_main0 = h->ev[2 * ST_PROFILE];         // main kernel
        a.ev_main1 = h->ev[2 * ST_PROFILE + 1];
        a.ev_core1 = h->ev[2 * ST_RANGES + 1];      // centre-zone kernel: main end -> core end
        a.ev_tc1 = h->ev[2 * ST_COUNT];             // tensor-core far-wing kernel: main start -> here
        if (opts->profile == XC_VOIGT_GH_BINNED || opts->profile == XC_VOIGT_GH_SAMPLED) {
            if ((st = ensure_gh(h, opts->n_gh, s))) return st;
            a.ghx = h->gh.as<double>();
            a.ghw = a.ghx + 64;
        }
        int64_t nl = 0;
        if ((st = batched_run(&h->batched, a, &nl))) return st;
        h->launches += nl;
        used[ST_PARAMS] = true;  // whole sweep; per-kernel times are read below
    }
    if (mem == XC_MEM_HOST) {
        warm_host_pages(sigma_out, total * sizeof(double));
        stage_begin(h, ST_FINISH, s);
        XC_TRY(cudaMemcpyAsync(sigma_out, sig, total * sizeof(double), cudaMemcpyDeviceToHost, s));
        stage_end(h, ST_FINISH, s);
        used[ST_FINISH] = true;
    }
    XC_TRY(cudaStreamSynchronize(s));
    if (opts->precision == XC_FP32 && h->n_lines > 0 && (st = batched_check(&h->batched))) return st;
    collect_timing(h, used);
    if (h->timing && opts->precision == XC_FP32 && h->n_lines > 0 && opts->width_mult <= 0.0) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * ST_PROFILE], h->ev[2 * ST_PROFILE + 1]) == cudaSuccess)
            h->last_ms[ST_PROFILE] = ms;
        if (opts->profile == XC_VOIGT_W4 &&
            cudaEventElapsedTime(&ms, h->ev[2 * ST_PROFILE + 1], h->ev[2 * ST_RANGES + 1]) == cudaSuccess)
            h->last_ms[ST_RANGES] = ms;
        // per kernel: far wings on the tensor cores (if they ran), CUDA-core kernel, centre zone
        h->tc_mma = batched_tc_mma_count(&h->batched);
        h->kernel_ms[0] = h->kernel_ms[1] = h->kernel_ms[2] = -1.0;
        if (h->tc_mma > 0) {
            if (cudaEventElapsedTime(&ms, h->ev[2 * ST_PROFILE], h->ev[2 * ST_COUNT]) == cudaSuccess)
                h->kernel_ms[0] = ms;
            if (cudaEventElapsedTime(&ms, h->ev[2 * ST_COUNT], h->ev[2 * ST_PROFILE + 1]) == cudaSuccess)
                h->kernel_ms[1] = ms;
        } else {
            h->kernel_ms[1] = h->last_ms[ST_PROFILE];
        }
        if (opts->profile == XC_VOIGT_W4) h->kernel_ms[2] = h->last_ms[ST_RANGES];
        cudaGetLastError();
    }
    return XC_OK;
}

static xc_status vjp_common(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                            const xc_opts *opts, const double *grad_sigma, double *dT, double *dP,
                            double *d_gamma_scale, double *d_n_shift, double *d_gamma_ref_line, double *d_n_line,
                            double *d_gamma0_broad, double *d_n_broad, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if ((st = check_grid(grid)) || (st = check_opts(opts)) || (st = check_conds(conds, n_cond, h))) return st;
    if (opts->profile != XC_DOPPLER && opts->profile != XC_LORENTZ && opts->profile != XC_VOIGT_W4 &&
        opts->profile != XC_VOIGT_GH_BINNED) {
        set_error("the adjoint supports Doppler, Lorentz, Voigt-w4 and binned Gauss-Hermite profiles");
        return XC_EUNSUPPORTED;
    }
    if (opts->quantity != XC_ABSORPTION || opts->threshold != XC_THRESHOLD_NONE) {
        set_error("the adjoint supports absorption without an intensity threshold");
        return XC_EUNSUPPORTED;
    }
    if (h->n_broad > 0 && (d_gamma_ref_line || d_n_line)) {
        set_error("under a broadener mixture the line list's gamma_ref and n_T are not used: pass NULL per-line "
                  "outputs (per-broadener gradients: xc_cross_section_vjp_broadening)");
        return XC_EINVAL;
    }
    if (n_cond && (!grad_sigma || !dT || !dP)) { set_error("NULL grad_sigma / dT / dP"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    reset_timing(h);
    VjpArgs a;
    a.L = lines_of(h);
    a.n_lines = h->n_lines;
    a.n_cond = (int)n_cond;
    a.grid = *grid;
    a.opts = *opts;
    a.stream = s;
    CondDev *dc = nullptr;
    if (n_cond) {
        if ((st = resolve_conds(h, conds, n_cond, s, &dc))) return st;
    }
    a.conds_dev = dc;
    a.conds_host = conds;
    a.mem = mem;
    a.grad_sigma = grad_sigma;
    a.dT = dT;
    a.dP = dP;
    a.d_gamma_scale = d_gamma_scale;
    a.d_n_shift = d_n_shift;
    a.d_gamma_ref_line = d_gamma_ref_line;
    a.d_n_line = d_n_line;
    a.d_gamma0_broad = d_gamma0_broad;
    a.d_n_broad = d_n_broad;
    if (opts->profile == XC_VOIGT_GH_BINNED) {
        if ((st = ensure_gh(h, opts->n_gh, s))) return st;
        a.ghx = h->gh.as<double>();
        a.ghw = a.ghx + 64;
    }
    a.timing = h->timing;
    a.ev_begin = h->ev[2 * ST_VJP];
    a.ev_end = h->ev[2 * ST_VJP + 1];
    int64_t nl = 0;
    if ((st = vjp_run(&h->batched, a, &nl))) return st;
    h->launches += nl;
    bool used[ST_COUNT] = {};
    used[ST_VJP] = true;
    XC_TRY(cudaStreamSynchronize(s));
    collect_timing(h, used);
    return XC_OK;
}

xc_status xc_cross_section_vjp(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                               const xc_opts *opts, const double *grad_sigma, double *dT, double *dP,
                               double *d_gamma_scale, double *d_n_shift, double *d_gamma_ref_line,
                               double *d_n_line, int mem, void *stream) {
    return vjp_common(h, conds, n_cond, grid, opts, grad_sigma, dT, dP, d_gamma_scale, d_n_shift, d_gamma_ref_line,
                      d_n_line, nullptr, nullptr, mem, stream);
}

xc_status xc_cross_section_vjp_broadening(xc_handle *h, const xc_condition *conds, size_t n_cond,
                                          const xc_grid *grid, const xc_opts *opts, const double *grad_sigma,
                                          double *dT, double *dP, double *d_gamma_scale, double *d_n_shift,
                                          double *d_gamma0_broad, double *d_n_broad, int mem, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (h->n_broad <= 0) {
        set_error("no broadener mixture is set (xc_set_broadening)");
        return XC_EINVAL;
    }
    return vjp_common(h, conds, n_cond, grid, opts, grad_sigma, dT, dP, d_gamma_scale, d_n_shift, nullptr, nullptr,
                      d_gamma0_broad, d_n_broad, mem, stream);
}

xc_status xc_set_timing(xc_handle *h, int enable) {
    xc_status st = check_handle(h);
    if (st) return st;
    h->timing = enable != 0;
    return XC_OK;
}

xc_status xc_last_timings(xc_handle *h, float *ms_out8) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!ms_out8) { set_error("NULL out"); return XC_EINVAL; }
    for (int i = 0; i < ST_COUNT; ++i) ms_out8[i] = h->last_ms[i];
    return XC_OK;
}

xc_status xc_get_tuning(xc_handle *h, char *buf, size_t len) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!buf || !len) { set_error("NULL buffer"); return XC_EINVAL; }
    snprintf(buf, len, "%s", h->batched.last_tuning.c_str());
    return XC_OK;
}

xc_status xc_last_sweep_kernels(xc_handle *h, double *ms_out, int64_t *mma_out) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!ms_out || !mma_out) { set_error("NULL out"); return XC_EINVAL; }
    for (int i = 0; i < 3; ++i) ms_out[i] = h->kernel_ms[i];
    *mma_out = h->tc_mma;
    return XC_OK;
}

xc_status xc_count_far_evals(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                             const xc_opts *opts, int64_t *count_out, void *stream) {
    xc_status st = check_handle(h);
    if (st) return st;
    if ((st = check_grid(grid)) || (st = check_opts(opts)) || (st = check_conds(conds, n_cond, h))) return st;
    if (!count_out) { set_error("NULL out"); return XC_EINVAL; }
    if (n_cond > 4096) { set_error("at most 4096 conditions per call"); return XC_EINVAL; }
    DeviceGuard dg(h->device);
    cudaStream_t s = S(stream);
    *count_out = 0;
    if (h->n_lines == 0 || n_cond == 0 || grid->n == 0 || opts->precision != XC_FP32) return XC_OK;
    CondDev *dc = nullptr;
    if ((st = resolve_conds(h, conds, n_cond, s, &dc))) return st;
    BatchedArgs a;
    a.L = lines_of(h);
    a.n_lines = h->n_lines;
    a.conds_dev = dc;
    a.conds_host = conds;
    a.n_cond = (int)n_cond;
    a.grid = *grid;
    a.opts = *opts;
    a.stream = s;
    return batched_count_far(&h->batched, a, count_out);
}

xc_status xc_set_tile_shape(xc_handle *h, int R, int CG) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (R < 0 || CG < 0 || (R == 0) != (CG == 0)) { set_error("tile shape (%d, %d): both 0 or both > 0", R, CG); return XC_EINVAL; }
    h->batched.force_R = R;
    h->batched.force_CG = CG;
    return XC_OK;
}

xc_status xc_last_launch_count(xc_handle *h, int64_t *count_out) {
    xc_status st = check_handle(h);
    if (st) return st;
    if (!count_out) { set_error("NULL out"); return XC_EINVAL; }
    *count_out = h->launches;
    return XC_OK;
}

}  // extern "C"
