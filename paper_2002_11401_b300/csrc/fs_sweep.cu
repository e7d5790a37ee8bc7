// fs_sweep.cu - the full field-and-margin sweep (Sec. "Dynamics": at each
// simulation step the total field on every island is calculated; Eq. 2, 3, 5, 6).
//
// One warp owns 32 consecutive islands (one node of the first tree level); the
// task itself (row sums, evaluation, keys, the tree above it) is sweep_task in
// fs_sweep_task.cuh. One launch covers every task of every simulation of a table,
// so the whole max-tree is ready when the kernel ends.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"
#include "fs_kernels.h"
#include "fs_sweep_task.cuh"

namespace fs {

namespace {

// OCC resident CTAs per SM: 4 (registers as needed) or 5 (at most 51 registers a
// thread, some spilled): the latter puts 5920 warps on the 148 SMs, one wave for
// an array of up to 189,000 islands. The autotuner picks. MODE as sweep_task.
template <int PREC, int W, int MODE, int OCC>
__global__ void __launch_bounds__(kSweepThreads, OCC)
    k_sweep(const Inst* __restrict__ tab, const int64_t* __restrict__ task_start, int n_inst,
            int64_t total_tasks, unsigned* const* __restrict__ tcnts) {
    __shared__ int sums32[PREC == 1 ? kSweepWarps : 1][32][2];
    __shared__ long long sums64[kSweepWarps][32][2];
    const int wib = threadIdx.x >> 5;
    const int64_t gw = (blockIdx.x * (int64_t)kSweepThreads + threadIdx.x) >> 5;
    if (gw >= total_tasks) return;
    const int inst = find_inst(task_start, n_inst, gw);
    const Inst& I = tab[inst];
    const InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;
    const int64_t lt = gw - task_start[inst];
    sweep_task<PREC, W, MODE, false>(I, tcnts[inst], t, lt, st->init != 0,
                                     sums32[PREC == 1 ? wib : 0], sums64[wib]);
}

// Projections of the current step's external field on every angle class of every
// active simulation (FP64, and rounded once to FP32), one block per simulation.
__global__ void k_ext_table(const Inst* __restrict__ tab, int n_inst) {
    const Inst& I = tab[blockIdx.x];
    const InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;
    const double hx = I.phx[t], hy = I.phy[t];
    for (int c = threadIdx.x; c < I.nclass; c += blockDim.x) {
        const double2 e = ext_proj(hx, hy, I.cs64[c]);
        I.ext64[c] = e;
        I.ext32[c] = make_float2(__double2float_rn(e.x), __double2float_rn(e.y));
    }
}

template <int PREC, int MODE, int W>
cudaError_t launch_wo(unsigned blocks, const SweepLaunch& L, cudaStream_t st) {
    if (L.occupancy == 5)
        k_sweep<PREC, W, MODE, 5><<<blocks, kSweepThreads, 0, st>>>(
            L.tab, L.task_start, L.n_inst, L.total_tasks, L.tcnts);
    else
        k_sweep<PREC, W, MODE, 4><<<blocks, kSweepThreads, 0, st>>>(
            L.tab, L.task_start, L.n_inst, L.total_tasks, L.tcnts);
    return cudaGetLastError();
}

template <int PREC, int MODE>
cudaError_t launch_w(const SweepLaunch& L, cudaStream_t st) {
    const unsigned blocks = (unsigned)((L.total_tasks + kSweepWarps - 1) / kSweepWarps);
    if (blocks == 0) return cudaSuccess;
    switch (L.lanes_per_row) {
        case 2:
            return launch_wo<PREC, MODE, 2>(blocks, L, st);
        case 4:
            return launch_wo<PREC, MODE, 4>(blocks, L, st);
        case 8:
            return launch_wo<PREC, MODE, 8>(blocks, L, st);
        case 16:
            return launch_wo<PREC, MODE, 16>(blocks, L, st);
        default:
            return launch_wo<PREC, MODE, 32>(blocks, L, st);
    }
}

}  // namespace

cudaError_t launch_ext_table(const SweepLaunch& L, cudaStream_t st) {
    if (L.n_inst == 0) return cudaSuccess;
    k_ext_table<<<L.n_inst, 128, 0, st>>>(L.tab, L.n_inst);
    return cudaGetLastError();
}

// The sweep proper; launch_ext_table must have run for the same step.
cudaError_t launch_sweep(const SweepLaunch& L, cudaStream_t st) {
    if (L.n_inst == 0) return cudaSuccess;
    if (L.prec == 1)
        return L.resweep ? launch_w<1, 1>(L, st) : launch_w<1, 0>(L, st);
    return L.resweep ? launch_w<0, 1>(L, st) : launch_w<0, 0>(L, st);
}

}  // namespace fs
