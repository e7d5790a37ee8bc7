// fs_kernels.h - launch interfaces of the sweep and relax kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"

namespace fs {

struct SweepLaunch {
    const Inst* tab;            // device table of simulations
    const int64_t* task_start;  // device [n_inst + 1]: first 32-island task of each
    int n_inst;
    int64_t total_tasks;
    unsigned* const* tcnts;     // device [n_inst]: per-simulation tree counters
    int prec;
    int resweep;                // 0 margins only, 1 recompute the dipolar sums
    int lanes_per_row;          // 4, 8, 16 or 32
    int occupancy = 4;          // resident CTAs per SM the kernel is built for: 4 or 5
};

// The relax keeps the tree's levels up to the first one with at most this many
// nodes (one warp reduces it, 8 nodes a lane, in place of the levels above).
constexpr int kRelaxTopNodes = 256;

struct RelaxLaunch {
    const Inst* tab;
    const int32_t* work;  // device [n_work]: simulation of each CTA
    int n_work;
    int prec;
    int smem_levels;      // dynamic shared memory for the upper tree levels
    int min_blocks = 1;   // 2: the build for two resident CTAs per SM (shared GPU)
    int multi = 0;        // 1: multi-flip rounds (fs_relax_multi.cu) first, then the
                          // single-flip kernel for what they hand off; 2: the same,
                          // the rounds on one CTA
};

// The work queue of the persistent batch kernel: one entry per member, in the
// order of `work` (largest members first), in device memory.
struct PersistLaunch {
    const Inst* tab;
    const int32_t* work;        // [n]: member at each queue position
    const int64_t* task_start;  // [members + 1]: first 32-island task of each member
    unsigned* const* tcnts;     // [members]: tree arrival counters
    int n;                      // queue positions (members)
    int prec, resweep, lanes_per_row;
    int smem_levels;            // dynamic shared memory of the relax's upper tree levels
    int32_t* state;             // [n]: kQ* below
    uint32_t* chunk;            // [n]: next sweep chunk of the member's current field step
    uint32_t* nchunk;           // [n]: sweep chunks per field step
    int32_t* ctl;               // [4]: members done, fault, progress beat, (unused)
};
constexpr int32_t kQSweep = 0;  // the field step's sweep: chunks to claim
constexpr int32_t kQReady = 1;  // swept: the relax is next
constexpr int32_t kQRelax = 2;  // relaxing
constexpr int32_t kQDone = 3;   // protocol finished (or stopped by a status)

// Queues the persistent batch protocol (state initialised from the members'
// device states; the first step's external-field table must be queued before).
// Returns cudaErrorInvalidConfiguration when the kernel cannot be resident with
// this much shared memory (the caller then uses per-step launches).
cudaError_t launch_batch_persist(const PersistLaunch& L, cudaStream_t st);

cudaError_t launch_ext_table(const SweepLaunch& L, cudaStream_t st);
cudaError_t launch_sweep(const SweepLaunch& L, cudaStream_t st);
cudaError_t launch_relax(const RelaxLaunch& L, cudaStream_t st);
cudaError_t launch_relax_multi(const RelaxLaunch& L, cudaStream_t st);
cudaError_t prepare_relax(int prec, int smem);
// out5 = [h_par | h_perp | lhs | lo | hi], 5 n doubles
cudaError_t launch_eval_all(const Inst* tab, int64_t n, double hx, double hy, uint32_t step,
                            double* out5, cudaStream_t st);
int relax_threads();
size_t relax_static_smem(int prec);

}  // namespace fs
