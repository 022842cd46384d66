/*
 * xc.h -- C ABI of libxc, a GB300 (sm_103a) engine that turns a molecular
 * line list into absorption cross sections on a wavenumber grid, following
 * the ExoCross method (Yurchenko, Al-Refaie & Tennyson 2018, arXiv:1801.09803).
 *
 * Conventions for every entry point
 *   - All functions return xc_status (XC_OK = 0).  They never throw, abort or
 *     exit; on failure xc_last_error() gives a message (thread-local, valid
 *     until the next call on the same thread).
 *   - Pointers passed in are borrowed for the duration of the call.  Outputs
 *     are allocated by the caller.  A `mem` argument says whether the arrays
 *     it covers are host (XC_MEM_HOST) or device (XC_MEM_DEVICE) memory; host
 *     outputs are complete when the call returns, device outputs are complete
 *     in stream order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; calls with host inputs or outputs
 *     synchronise that stream before returning.
 *   - Units (paper Table t:units): wavenumber cm^-1, temperature K, pressure
 *     in units of P_ref, intensity cm/molecule, cross section
 *     cm^2/molecule = cm/(molecule cm^-1); with XC_EMISSION the line strength is
 *     an emissivity (erg/s/sr per molecule) and sigma its emission spectrum
 *     (erg/s/sr per molecule per cm^-1).
 *   - Per-line arrays that the library returns are in the library's sorted
 *     order (ascending wavenumber, ties by input position);
 *     xc_get_permutation() maps sorted position -> input position.
 */
#ifndef XC_H
#define XC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int xc_status;
enum {
    XC_OK = 0,
    XC_EINVAL = 1,        /* bad argument or invalid input values */
    XC_ENOMEM = 2,        /* device or pinned host allocation failed */
    XC_ECUDA = 3,         /* a CUDA runtime call failed */
    XC_ETIMEOUT = 4,      /* a bounded device wait gave up */
    XC_EUNSUPPORTED = 5   /* valid request this build does not implement */
};

enum { XC_MEM_HOST = 0, XC_MEM_DEVICE = 1 };

/* line profiles (paper Sec. 3) */
enum {
    XC_DOPPLER = 0,          /* Eq. (e:Gauss) with alpha_D of Eq. (e:alphaD) */
    XC_LORENTZ = 1,          /* Eq. (e:lor) with gamma_L of Eq. (e:gamma_L) */
    XC_VOIGT_W4 = 2,         /* Eq. (e:Voigt), w(z) by Humlicek's w4 */
    XC_VOIGT_GH_BINNED = 3,  /* Eq. (e:sigma:quad): bin-averaged Gauss-Hermite (area-conserving) */
    XC_VOIGT_GH_SAMPLED = 4, /* Eq. (e:V-quad): Gauss-Hermite sum sampled at the grid point */
    XC_DOPPLER_BINNED = 5,   /* Eq. (eqn:sig_ij): Gaussian averaged over each grid bin (erf) */
    XC_LORENTZ_BINNED = 6,   /* Eq. (eqn:sig_lor-2): Lorentzian averaged over each grid bin (arctan) */
    XC_VOIGT_VV = 7          /* Eq. (e:fast-v): Vectorized Voigt -- the w4 Voigt within vv_split of the
                                centre, beyond it the Voigt of a line at 1 cm^-1 (Doppler HWHM
                                alpha / nu, the same gamma) times beta, at the line's own offsets */
};

/* xc_opts.vv_flags (XC_VOIGT_VV) */
enum {
    XC_VV_BETA = 1,      /* beta of Eq. (e:beta): the wing scaled to be continuous at vv_split (else 1) */
    XC_VV_NORMALISE = 2  /* VVN (Sec. "Binned Vectorized Voigt"): each line's intensity divided by
                            h sum_k f(nu_k - nu), the sum over its cut window on the grid's lattice
                            (also past the grid ends), so that every line's area is I */
};

/* arithmetic of the profile evaluation */
enum {
    XC_FP64_PLAIN = 0,  /* every step in FP64 */
    XC_FP32 = 1         /* FP32 profile math and window accumulators; FP64 grid offsets,
                           Q(T) and final accumulation */
};

/* xc_load_lines flags */
enum { XC_ASSUME_SORTED = 1u };

/* xc_opts.flags.  With XC_FP32, Voigt w4, a fixed cut and 16 or more conditions,
 * the far wings (points at least D(l, c) grid steps from a line, D chosen so that
 * the region-I rational equals its three-term series in 1/u to < 2e-7) are summed
 * on the tensor cores as a matrix product (TF32 operands split hi + lo, FP32
 * accumulation); XC_OPT_NO_TENSOR_CORES keeps every evaluation on the CUDA cores. */
enum { XC_OPT_NO_TENSOR_CORES = 1 };

/* xc_opts.quantity: what each line contributes, times its profile */
enum {
    XC_ABSORPTION = 0,  /* absorption intensity I, Eq. (e:int): cm/molecule */
    XC_EMISSION = 1     /* emissivity, Eq. (e:emiss), from the upper state E' = E'' + nu, times
                           the photon energy h c nu so that it is in erg/s/sr per molecule (the
                           unit the paper states; its printed formula leaves out h c) */
};

/* xc_opts.threshold (Sec. "Intensity thresholds"): lines whose strength (I, or the
 * emissivity with XC_EMISSION) is below the threshold at their wavenumber are left out.
 * The decision is taken in FP64 for every precision. */
enum {
    XC_THRESHOLD_NONE = 0,
    XC_THRESHOLD_CONSTANT = 1,  /* I_cut */
    XC_THRESHOLD_HITRAN = 2     /* I_crit (nu/nu_crit) tanh(c2 nu / 2T) for nu <= nu_crit, else I_crit */
};

typedef struct xc_handle xc_handle;

/* Line list, structure of arrays, n entries each (28 bytes per line).
 * nu: transition wavenumber (float64, > 0, finite); elower: lower-state term
 * value E'' (float32, finite, >= 0); A: Einstein coefficient (float32, >= 0);
 * gamma_ref: Lorentz HWHM at T_ref, P_ref (float32, >= 0); n_T: temperature
 * exponent (float32, finite); g_up: upper total degeneracy g_ns(2J'+1)
 * (int16, >= 0); j_lo: lower J'' (int16, may be NULL: stored as 0).
 * Paper: Eq. (e:int), Eq. (e:gamma_L), ExoMol .trans/.states fields (Sec. 5.1). */
typedef struct {
    const double *nu;
    const float *elower;
    const float *A;
    const float *gamma_ref;
    const float *n_T;
    const int16_t *g_up;
    const int16_t *j_lo;
    int mem;  /* XC_MEM_HOST or XC_MEM_DEVICE, for all seven arrays */
} xc_lines;

/* One (T, P) condition.  gamma = gamma_scale * gamma_ref * (T_ref/T)^(n_T + n_shift)
 * * P/P_ref (Eq. e:gamma_L); alpha from Eq. (e:alphaD) with m = mass_da daltons;
 * I from Eq. (e:int) times `abundance`.  Q <= 0 means "compute Q(T) and dQ/dT
 * from the states given to xc_set_states" (Eq. e:pf); otherwise Q and dQdT are
 * used as given (dQdT only matters for the adjoint). */
typedef struct {
    double T, P, Q, dQdT;
    double mass_da, T_ref, P_ref;
    double gamma_scale, n_shift;
    double abundance;
} xc_condition;

/* Equidistant grid nu_k = nu_A + k*step, k = 0..n-1 (Eq. e:Ngrid: n counts both ends). */
typedef struct {
    double nu_A;
    double step;
    int64_t n;
} xc_grid;

/* Profile options.  Each line contributes to grid points with |nu_k - nu_l| <= cut_l
 * (inclusive), cut_l = cutoff, or min(cutoff, width_mult * max(alpha_l, gamma_l))
 * when width_mult > 0 (Sec. 3.10 "Off-set").  n_gh: Gauss-Hermite nodes (1..64). */
typedef struct {
    int profile;        /* XC_DOPPLER .. XC_VOIGT_VV */
    int precision;      /* XC_FP64_PLAIN or XC_FP32 */
    double cutoff;      /* cm^-1, > 0 */
    double width_mult;  /* 0 = fixed cut */
    int n_gh;
    int flags;          /* XC_OPT_* bits, 0 by default */
    int quantity;       /* XC_ABSORPTION (default) or XC_EMISSION */
    int threshold;      /* XC_THRESHOLD_* */
    double I_cut;       /* constant threshold, >= 0, in the unit of the quantity */
    double nu_crit;     /* HITRAN threshold: > 0, cm^-1 (the paper's default 2000) */
    double I_crit;      /* HITRAN threshold: >= 0, in the unit of the quantity (default 1e-29) */
    double vv_split;    /* XC_VOIGT_VV: half-width of the exact zone, cm^-1 (0: the paper's 4) */
    int vv_flags;       /* XC_VV_* bits */
} xc_opts;

/* Library version string (static storage). */
const char *xc_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *xc_last_error(void);

/* Create a handle bound to CUDA device `device`; it owns the sorted line
 * arrays, the states, scratch buffers, the autotune cache and CUDA graphs.
 * EINVAL: bad device or NULL out pointer.  ENOMEM / ECUDA on failure. */
xc_status xc_create(xc_handle **out, int device);

/* Release everything the handle owns (NULL is accepted).  Synchronises the device. */
xc_status xc_destroy(xc_handle *h);

/* Copy n lines into the handle and sort them by wavenumber on the device
 * (LSD radix sort on the float64 bit pattern; stable, so equal wavenumbers keep
 * input order), then gather every field into sorted order.  Replaces any lines
 * loaded before.  flags & XC_ASSUME_SORTED skips the sort but still checks the
 * order (EINVAL if unsorted).  EINVAL: n >= 2^32, NULL arrays (except j_lo),
 * nu <= 0 or non-finite, A < 0, gamma_ref < 0, non-finite elower/n_T.
 * Paper: chunked reading of .trans lines (Sec. 5.3); ExoMol transitions are
 * stored in wavenumber order (Table tab:trans). */
xc_status xc_load_lines(xc_handle *h, const xc_lines *lines, size_t n, unsigned flags, void *stream);

/* Number of lines held by the handle. */
xc_status xc_num_lines(const xc_handle *h, size_t *n_out);

/* Copy the sorted line arrays out (any pointer may be NULL to skip that field). */
xc_status xc_get_lines(xc_handle *h, double *nu, float *elower, float *A, float *gamma_ref,
                       float *n_T, int16_t *g_up, int16_t *j_lo, int mem, void *stream);

/* Sorted position -> input position (uint32, n entries). */
xc_status xc_get_permutation(xc_handle *h, uint32_t *perm_out, int mem, void *stream);

/* .broad broadening schemes of one broadener (Sec. "Broadening parameters") */
enum { XC_BROAD_CONSTANT = 0, XC_BROAD_A0 = 1, XC_BROAD_A1 = 2 };

/* One broadener of a mixture (Secs. "Broadening parameters", "Mixtures of broadeners").
 * All table arrays are host memory, n_entries rows each. */
typedef struct {
    int type;                 /* XC_BROAD_CONSTANT, XC_BROAD_A0 (key J'') or XC_BROAD_A1 (J'', J') */
    double fraction;          /* rho_i >= 0: the broadener's share of the mixture */
    double gamma0, n;         /* gamma_0 at T_ref, P_ref (cm^-1) and n_L: the constant values,
                                 and the defaults for lines the table does not list */
    int64_t n_entries;        /* table rows (a0, a1), <= 2^20 */
    const int32_t *j_lo;      /* J'' of each row */
    const int32_t *j_up;      /* J' of each row (a1; may be NULL otherwise) */
    const double *gamma0_j;   /* gamma_0 of each row (>= 0, finite) */
    const double *n_j;        /* n_L of each row (finite) */
} xc_broadener;

/* Lorentz widths from a mixture of .broad broadeners instead of the line list's gamma_ref
 * and n_T: gamma_L = gamma_scale P/P_ref sum_i rho_i gamma_0,i (T_ref/T)^(n_L,i + n_shift),
 * each term Eq. (e:gamma_L) of the paper, the sum its Sec. "Mixtures of broadeners".
 * a0 finds a line's row by its J'' (j_lo of the loaded lines), a1 by J'' and J'
 * (j_up: one int16 per line in the order given to xc_load_lines, host or device per mem;
 * may be NULL when no broadener is a1); a line without a row takes gamma0 and n.
 * At most 8 broadeners; duplicate table keys, negative widths or fractions: EINVAL.
 * n_broadeners = 0 returns to the line list's widths, as does the next xc_load_lines.
 * Synchronises `stream`.  Under a mixture the adjoint returns dT, dP, dgamma_scale and dn_shift
 * (xc_cross_section_vjp, per-line outputs NULL) and per-broadener gradients
 * (xc_cross_section_vjp_broadening). */
xc_status xc_set_broadening(xc_handle *h, const xc_broadener *b, int n_broadeners, const int16_t *j_up, int mem,
                            void *stream);

/* Give the handle a state list (E term values cm^-1 float64, total degeneracy
 * g int32 >= 0) for conditions with Q <= 0.  Paper Eq. (e:pf). */
xc_status xc_set_states(xc_handle *h, const double *E, const int32_t *g, size_t n_states,
                        int mem, void *stream);

/* Partition function Q(T) = sum_n g_n exp(-c2 E_n / T) and dQ/dT for nT
 * temperatures, in FP64 on the device (Eq. e:pf; Sec. 2.6).  E, g, T, Q_out,
 * dQdT_out (nullable) all live in `mem`.  EINVAL: T <= 0, NULL E/g with
 * n_states > 0.  No handle needed; uses the current device. */
xc_status xc_partition_function(const double *E, const int32_t *g, size_t n_states,
                                const double *T, size_t nT, double *Q_out, double *dQdT_out,
                                int mem, void *stream);

/* Per-line parameters for one condition, in FP64, in sorted order:
 * I (Eq. e:int), alpha_D (Eq. e:alphaD), gamma_L (Eq. e:gamma_L).
 * Any output may be NULL. */
xc_status xc_line_params(xc_handle *h, const xc_condition *cond, double *I_out,
                         double *alpha_out, double *gamma_out, int mem, void *stream);

/* Number of (line, grid point) pairs inside the cutoff for these conditions:
 * the algorithmic work of a cross section (host int64 output). */
xc_status xc_count_evals(xc_handle *h, const xc_condition *conds, size_t n_cond,
                         const xc_grid *grid, const xc_opts *opts, int64_t *count_out, void *stream);

/* Cross section of one condition on the grid: sigma_k = sum_l I_l f_l(nu_k)
 * over |nu_k - nu_l| <= cut_l (paper Sec. 3.1 "sampling method", Eq. e:cross;
 * XC_VOIGT_GH_BINNED gives the bin average of Eq. e:sigma:quad).  Gather form:
 * each CTA owns a window of grid points and visits only the lines whose cut
 * reaches it; no global atomics, so results are bitwise reproducible.
 * sigma_out: float64[grid->n] in `mem`.  EINVAL on bad grid/opts/condition,
 * EUNSUPPORTED for an unknown profile/precision. */
xc_status xc_cross_section(xc_handle *h, const xc_condition *cond, const xc_grid *grid,
                           const xc_opts *opts, double *sigma_out, int mem, void *stream);

/* n_cond conditions in one persistent launch that shares every staged line
 * across conditions (sigma_out: float64[n_cond][grid->n], condition-major).
 * opts->precision XC_FP32 uses the batched FP32 kernel (window size picked by
 * the autotuner and cached per shape; the sweep is captured once into a CUDA
 * graph and replayed); XC_FP64_PLAIN runs the FP64 kernel per condition. */
xc_status xc_cross_section_batched(xc_handle *h, const xc_condition *conds, size_t n_cond,
                                   const xc_grid *grid, const xc_opts *opts, double *sigma_out,
                                   int mem, void *stream);

/* Vector-Jacobian product of the batched cross section.  Given
 * grad_sigma = dL/dsigma (float64[n_cond][grid->n], in `mem`), returns
 *   dT[c], dP[c]                      dL/dT_c, dL/dP_c          (n_cond each)
 *   d_gamma_scale, d_n_shift          dL/d(gamma_scale), dL/d(n_shift), summed over conditions
 *   d_gamma_ref_line, d_n_line        dL/d(gamma_ref_l), dL/d(n_l), sorted order (nullable)
 * all float64 in `mem`.  dT includes dQ/dT through Q (from the states, or the
 * condition's dQdT).  Profiles are recomputed, not stored; the cut is held
 * fixed.  opts->precision selects FP32 (default) or FP64 recomputation; the
 * per-condition and per-line reductions are FP64 and deterministic.  XC_DOPPLER,
 * XC_LORENTZ, XC_VOIGT_W4 only (EUNSUPPORTED otherwise).  Under a broadener mixture
 * (xc_set_broadening) the line list's gamma_ref and n_T are not used: d_gamma_ref_line
 * and d_n_line must then be NULL (EINVAL otherwise).  Not in the paper: the chain rule
 * of Eqs. (e:int), (e:alphaD), (e:gamma_L) and the profile. */
xc_status xc_cross_section_vjp(xc_handle *h, const xc_condition *conds, size_t n_cond,
                               const xc_grid *grid, const xc_opts *opts, const double *grad_sigma,
                               double *dT, double *dP, double *d_gamma_scale, double *d_n_shift,
                               double *d_gamma_ref_line, double *d_n_line, int mem, void *stream);

/* The adjoint under the handle's mixture of broadeners (xc_set_broadening; EINVAL if none
 * is set): gamma_L = gamma_scale P/P_ref sum_i gamma_i, gamma_i = rho_i gamma_0,i
 * (T_ref/T)^(n_L,i + n_shift), each term Eq. (e:gamma_L), the sum Sec. "Mixtures of
 * broadeners".  Besides dT, dP (n_cond each), d_gamma_scale and d_n_shift (scalars, each
 * nullable) as in xc_cross_section_vjp, per broadener i (in the order given to
 * xc_set_broadening; n_broadeners entries each, nullable):
 *   d_gamma0_broad[i]  dL/d(a factor on all of broadener i's gamma_0 values, its table rows
 *                      and its default, at 1) -- d gamma_L = gamma_i; dL/d rho_i is this / rho_i
 *   d_n_broad[i]       dL/d(a shift of all its n_L values, at 0) -- d gamma_L = gamma_i ln(T_ref/T)
 * Summed over broadeners they give gamma_scale dL/d(gamma_scale) and dL/d(n_shift).
 * All arrays in `mem`; profiles, precisions and errors as xc_cross_section_vjp. */
xc_status xc_cross_section_vjp_broadening(xc_handle *h, const xc_condition *conds, size_t n_cond,
                                          const xc_grid *grid, const xc_opts *opts, const double *grad_sigma,
                                          double *dT, double *dP, double *d_gamma_scale, double *d_n_shift,
                                          double *d_gamma0_broad, double *d_n_broad, int mem, void *stream);

/* Stage timing: when enabled, the library records CUDA events on the launch
 * stream around its kernels (as event nodes inside its CUDA graphs); xc_last_timings
 * returns the milliseconds of the most recent call per stage: [0] sort,
 * [1] gather/load, [2] Q(T), [3] line parameters (FP64 path) or the whole FP32
 * sweep (setup kernels + profile kernels), [4] window ranges (FP64 path) or the
 * FP32 centre-zone kernel (Voigt w4), [5] the main profile kernel, [6] adjoint,
 * [7] host<->device copies.  Stages not run read 0. */
xc_status xc_set_timing(xc_handle *h, int enable);
xc_status xc_last_timings(xc_handle *h, float *ms_out8);

/* Allocation-free FP32 batched cross section.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory while
 * they run -- code inside another framework's memory pool or a fixed memory
 * budget, real-time loops where cudaMalloc/cudaFree (which can synchronise the
 * device) are not allowed, or hosts that can only hand over buffers they own.
 * It needs no handle and allocates nothing: its scratch (per-line grid
 * geometry, per-condition constants, window ranges, tile order, work counter)
 * is one fixed array of about 18 MB (17.9e6 bytes) in device memory that every GPU loading
 * the library holds until the process exits.
 *   lines      device arrays (lines->mem == XC_MEM_DEVICE), already sorted by
 *              ascending nu (checked: EINVAL if not), n_lines <= 1,048,576.
 *   E, g       device state list for conditions with Q <= 0 (else may be NULL).
 *   conds      host array, n_cond <= 64.   grid->n <= 4,194,304 points.
 *   opts       precision XC_FP32, width_mult 0, profile Doppler, Lorentz or
 *              Voigt-w4 (EUNSUPPORTED otherwise).
 *   sigma_out  device float64[n_cond][grid->n].
 * Sizes beyond these limits return XC_EINVAL with a message naming the limit.
 * The first call on each device looks up the scratch array's device address
 * (with that device current); make that first call before any stream capture.
 * Every call on a device shares the same scratch array, which keeps the last
 * call's contents (the parts that must start at zero are cleared by each call):
 * calls whose work overlaps on the GPU (different streams or threads) race and
 * must be serialised by the caller.  The call synchronises `stream` while it
 * uploads the conditions. */
xc_status xc_cross_section_batched_static(const xc_lines *lines, size_t n_lines, const double *E,
                                          const int32_t *g, size_t n_states, const xc_condition *conds,
                                          size_t n_cond, const xc_grid *grid, const xc_opts *opts,
                                          double *sigma_out, void *stream);

/* Description of the FP32 kernel configuration the autotuner chose for the most
 * recent batched call (tile shape and the prediction of every candidate), as a
 * NUL-terminated string truncated to `len` bytes. */
xc_status xc_get_tuning(xc_handle *h, char *buf, size_t len);

/* Kernel launches issued by the last call (for launch accounting). */
xc_status xc_last_launch_count(xc_handle *h, int64_t *count_out);

/* Per-kernel times (ms, CUDA events; needs xc_set_timing(h, 1)) of the last FP32
 * batched call with a fixed cut: ms_out[0] the tensor-core far-wing kernel, ms_out[1]
 * the CUDA-core profile kernel, ms_out[2] the Voigt w4 centre-zone kernel; -1 where a
 * kernel did not run or was not timed.  *mma_out: tcgen05.mma instructions (M = 128,
 * N = 32, K = 8, kind::tf32) the tensor-core kernel issued, 0 if it did not run. */
xc_status xc_last_sweep_kernels(xc_handle *h, double *ms_out, int64_t *mma_out);

/* Algorithmic work of the tensor-core far-wing kernel: the number of (line, grid point,
 * condition) evaluations inside the cut (each one region-I w4 evaluation of Eq. e:Voigt)
 * that xc_cross_section_batched with the same arguments sums on the tensor cores, found
 * by a separate kernel that applies the far-wing kernel's own test to the same rounded
 * values.  0 when the tensor-core kernel would not run (FP64, fewer than 16 conditions,
 * a width-limited cut, another profile).  Host int64 output; synchronises `stream`. */
xc_status xc_count_far_evals(xc_handle *h, const xc_condition *conds, size_t n_cond, const xc_grid *grid,
                             const xc_opts *opts, int64_t *count_out, void *stream);

/* Fix the tile shape of the FP32 CUDA-core kernel for later batched calls on this
 * handle: R grid points per thread and CG conditions per tile, one of the compiled
 * shapes of the profile (R in {2, 4, 8}; CG in {1, 2, 4, 8, 16, 32}); (0, 0) restores
 * the autotuner.  A call whose profile has no such shape fails with XC_EUNSUPPORTED.
 * For testing every compiled kernel and for reproducible timing. */
xc_status xc_set_tile_shape(xc_handle *h, int R, int CG);

#ifdef __cplusplus
}
#endif

#endif /* XC_H */
