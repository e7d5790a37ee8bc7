// fs_batch.h - device table of simulations advanced together (batches, server).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fs_common.cuh"
#include "fs_internal.h"

namespace fs {

struct BatchTable {
    Arena mem;
    int cap = 0;
    Inst* tab = nullptr;
    int64_t* task_start = nullptr;
    unsigned** tcnts = nullptr;
    int32_t* work = nullptr;
    int n_inst = 0;
    int64_t total_tasks = 0;
    int lanes = 16;
    int occ = 4;  // sweep build: resident CTAs per SM
    std::vector<Inst> h_tab;
    std::vector<int64_t> h_task;
    std::vector<unsigned*> h_tcnt;
    std::vector<int32_t> h_work;
    // the persistent schedule's work queue (one entry per member) and its counters
    int32_t* q_state = nullptr;
    uint32_t* q_chunk = nullptr;
    uint32_t* q_nchunk = nullptr;
    int32_t* q_ctl = nullptr;  // [4]: members done, fault, progress beat, (unused)

    cudaError_t upload(const std::vector<fs_sim*>& sims, const std::vector<Inst>& descs,
                       cudaStream_t st);
    // one field step of every member: a sweep over all rows, then one relax CTA each
    cudaError_t enqueue_step(int prec, int resweep, int levels, cudaStream_t st) const;
    // the whole protocol in one persistent launch (members advance independently);
    // cudaErrorInvalidConfiguration when it cannot be resident
    cudaError_t enqueue_persistent(int prec, int resweep, int levels, cudaStream_t st) const;
    // times the batched sweep's builds (lanes per row x resident CTAs per SM) on
    // the batch's own rows and keeps the fastest; every build gives the same bits
    cudaError_t autotune(int prec, int resweep, cudaStream_t st);
};

cudaError_t prepare_relax(int prec, int smem);

}  // namespace fs
