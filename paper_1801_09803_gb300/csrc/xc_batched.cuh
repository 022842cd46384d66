// xc_batched.cuh -- interface of the FP32 / batched profile kernels and the adjoint.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "xc_internal.cuh"

namespace xc {

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
