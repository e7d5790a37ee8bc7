// fs_internal.h - the simulation object behind the opaque fs_sim handle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/flatspin_b300.h"
#include "fs_common.cuh"

namespace fs {

// A caller's device buffer that a simulation's allocations are carved from:
// the state from the bottom (lo bytes used), a build's temporaries from the top
// (hi bytes used).
struct Workspace {
    char* base = nullptr;
    size_t cap = 0, lo = 0, hi = 0;
};

// Device allocations owned by one object: stream-ordered from the pool, or, bound
// to a workspace (ws), carved from its bottom or its top end with nothing freed.
struct Arena {
    std::vector<void*> blocks;
    int64_t bytes = 0;
    Workspace* ws = nullptr;
    bool top = false;
    cudaError_t alloc(void** out, size_t n, cudaStream_t st);
    void release(cudaStream_t st);
};

// Arrays of at least this many islands relax in multi-flip rounds unless the
// simulation chooses otherwise (fs_set_relax_mode).
constexpr int64_t kMultiAutoIslands = 32768;
bool relax_multi(const fs_sim* sim);

int choose_lanes(double avg_groups);
int relax_smem_levels(int64_t n);  // bytes of upper tree levels kept in shared memory
int relax_smem_max();              // largest dynamic shared memory of any relax launch
// Queues K field steps (external-field table, sweep, relax) of one simulation on
// `st`; the descriptor and state must already be on the device.
cudaError_t enqueue_steps(fs_sim* sim, int64_t K, int resweep, cudaStream_t st);

}  // namespace fs

struct fs_sim {
    // geometry (canonical order)
    int64_t n = 0;
    double a = 1.0;
    std::vector<double> x, y, theta;
    std::vector<uint16_t> cls;
    std::vector<double> cls_cos, cls_sin;
    // parameters
    fs_params p{};
    std::vector<double> hk;
    std::vector<float2> rbc32;
    std::vector<double2> rbc64;
    bool built = false;
    int device = -1;  // the CUDA device current when the parameters were set
    bool fields_valid = false;
    // current external field and thermal step
    double hx = 0.0, hy = 0.0;
    uint32_t step = 0;
    // device
    cudaStream_t stream = nullptr;
    fs::Workspace ws;  // caller's buffer (fs_bind_workspace), else unused
    fs::Arena mem;     // everything that lives as long as the parameters
    fs::Arena run;  // per-call protocol buffers
    fs::Arena ext_mem;  // local or spatial external-field series and per-island projections
    fs::Arena sig_mem;  // thermal standard deviation series
    fs::Inst inst{};      // descriptor (host copy)
    fs::Inst inst_run{};  // descriptor of the queued call (host staging)
    fs::InstState state_host{};
    fs::Inst* d_inst = nullptr;
    fs::InstState* d_state = nullptr;
    int64_t* d_task_start = nullptr;
    unsigned** d_tcnts = nullptr;
    unsigned* tcnt = nullptr;
    int32_t* d_work = nullptr;
    double* d_field = nullptr;
    double* d_eval = nullptr;
    int64_t nnzp = 0;
    int32_t max_deg = 0;
    int32_t e64 = 0, e32 = 0;
    int lanes = 16;
    int sweep_occ = 4;  // resident sweep CTAs per SM (4 or 5), set by the autotuner
    int relax_mode = 0; // FS_RELAX_AUTO, FS_RELAX_SINGLE, FS_RELAX_MULTI or FS_RELAX_MULTI_CTA
    int64_t rechecks = 0, fallbacks = 0;
    int64_t rounds = 0, idle_rounds = 0;  // multi-flip relax
    int64_t round_flips = 0, handoffs = 0;
    cudaGraphExec_t graph_exec = nullptr;
    // profiling: CUDA events around each sweep and relax launch
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    double prof_sweep_ms = 0.0, prof_relax_ms = 0.0;
    int64_t prof_sweeps = 0, prof_relaxes = 0;
    std::string err;
};

fs_status fs_build_sim(fs_sim* sim);
