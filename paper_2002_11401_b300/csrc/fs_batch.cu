// fs_batch.cu - many independent simulations advanced together (ensembles of
// disorder realisations, parameter sweeps; Sec. "Simulation framework", runner).
//
// Two schedules, each captured in a CUDA graph and launched once: a persistent
// kernel in which every member advances its own field steps (a free CTA takes a
// swept member's relax, else a chunk of some member's sweep; fs_relax.cu), or per
// field step one sweep launch over the rows of every member (one warp per 32
// islands of any member, so the whole device streams the CSR at once) and one
// relax launch giving every member its own CTA. Each member's arithmetic is
// exactly that of a solo run: integer field sums and per-island evaluations do not
// depend on what else is in flight.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/flatspin_b300.h"
#include "fs_batch.h"
#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_kernels.h"

namespace fs {

cudaError_t BatchTable::upload(const std::vector<fs_sim*>& sims,
                               const std::vector<Inst>& descs, cudaStream_t st) {
    const int n = (int)sims.size();
    cudaError_t e;
    if (n > cap) {
        mem.release(st);
        cap = std::max(n, 2 * cap);
        if ((e = mem.alloc((void**)&tab, sizeof(Inst) * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&task_start, 8 * (cap + 1), st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&tcnts, 8 * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&work, 4 * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&q_state, 4 * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&q_chunk, 4 * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&q_nchunk, 4 * cap, st)) != cudaSuccess) return e;
        if ((e = mem.alloc((void**)&q_ctl, 16, st)) != cudaSuccess) return e;
    }
    h_tab = descs;
    h_task.assign((size_t)n + 1, 0);
    h_tcnt.resize((size_t)n);
    h_work.resize((size_t)n);
    double deg = 0.0, rows = 0.0;
    for (int i = 0; i < n; ++i) {
        h_task[(size_t)i + 1] = h_task[(size_t)i] + (sims[(size_t)i]->n + 31) / 32;
        h_tcnt[(size_t)i] = sims[(size_t)i]->tcnt;
        deg += (double)sims[(size_t)i]->nnzp;
        rows += (double)sims[(size_t)i]->n;
    }
    // largest members first, so that long relaxes start early
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return sims[(size_t)a]->n > sims[(size_t)b]->n; });
    for (int i = 0; i < n; ++i) h_work[(size_t)i] = order[(size_t)i];
    total_tasks = h_task[(size_t)n];
    n_inst = n;
    lanes = choose_lanes(rows > 0 ? deg / rows / 4.0 : 4.0);
    if (n == 0) return cudaSuccess;
    if ((e = cudaMemcpyAsync(tab, h_tab.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(task_start, h_task.data(), 8 * (n + 1), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(tcnts, h_tcnt.data(), 8 * n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return e;
    return cudaMemcpyAsync(work, h_work.data(), 4 * n, cudaMemcpyHostToDevice, st);
}

cudaError_t BatchTable::enqueue_step(int prec, int resweep, int levels, cudaStream_t st) const {
    if (n_inst == 0) return cudaSuccess;
    SweepLaunch S;
    S.tab = tab;
    S.task_start = task_start;
    S.n_inst = n_inst;
    S.total_tasks = total_tasks;
    S.tcnts = tcnts;
    S.prec = prec;
    S.resweep = resweep;
    S.lanes_per_row = lanes;
    S.occupancy = occ;
    cudaError_t e = launch_ext_table(S, st);
    if (e != cudaSuccess) return e;
    e = launch_sweep(S, st);
    if (e != cudaSuccess) return e;
    RelaxLaunch R;
    R.tab = tab;
    R.work = work;
    R.n_work = n_inst;
    R.prec = prec;
    R.smem_levels = levels;
    // more members than SMs: two latency-bound relaxes per SM
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    R.min_blocks = n_inst > std::max(nsm, 1) ? 2 : 1;
    return launch_relax(R, st);
}

cudaError_t BatchTable::enqueue_persistent(int prec, int resweep, int levels,
                                          cudaStream_t st) const {
    if (n_inst == 0) return cudaSuccess;
    SweepLaunch S;
    S.tab = tab;
    S.task_start = task_start;
    S.n_inst = n_inst;
    S.total_tasks = total_tasks;
    S.tcnts = tcnts;
    S.prec = prec;
    S.resweep = resweep;
    cudaError_t e = cudaMemsetAsync(q_ctl, 0, 16, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_ext_table(S, st)) != cudaSuccess) return e;  // the first step's table
    PersistLaunch P;
    P.tab = tab;
    P.work = work;
    P.task_start = task_start;
    P.tcnts = tcnts;
    P.n = n_inst;
    P.prec = prec;
    P.resweep = resweep;
    P.lanes_per_row = lanes;
    P.smem_levels = levels;
    P.state = q_state;
    P.chunk = q_chunk;
    P.nchunk = q_nchunk;
    P.ctl = q_ctl;
    return launch_batch_persist(P, st);
}

cudaError_t BatchTable::autotune(int prec, int resweep, cudaStream_t st) {
    // The trial sweeps compute what the protocol's first sweep computes (the same
    // field step of the same states): they change nothing the protocol reads.
    SweepLaunch S;
    S.tab = tab;
    S.task_start = task_start;
    S.n_inst = n_inst;
    S.total_tasks = total_tasks;
    S.tcnts = tcnts;
    S.prec = prec;
    S.resweep = resweep;
    cudaError_t e = launch_ext_table(S, st);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    const int cands[5] = {2, 4, 8, 16, 32};
    float best_ms = 1e30f;
    for (int c = 0; c < 10 && e == cudaSuccess; ++c) {
        S.lanes_per_row = cands[c % 5];
        S.occupancy = c < 5 ? 4 : 5;
        if ((e = launch_sweep(S, st)) != cudaSuccess) break;  // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, st);
            e = launch_sweep(S, st);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            lanes = S.lanes_per_row;
            occ = S.occupancy;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace fs

using namespace fs;

extern "C" fs_status fs_batch_run_protocol_ex(fs_sim* const* sims, int32_t n, const double* hx,
                                              const double* hy, int64_t K, int32_t resweep,
                                              int32_t schedule, int64_t* n_flips,
                                              uint64_t* seq_hash, int32_t* status,
                                              int64_t* flips_per_step) {
    if (!sims || n <= 0 || !sims[0]) return FS_ERR_INVALID;
    fs_sim* lead = sims[0];
    if (K < 0 || (K > 0 && (!hx || !hy)) || !n_flips || !seq_hash || !status ||
        schedule < FS_BATCH_AUTO || schedule > FS_BATCH_TWO_CHAINS) {
        lead->err = "bad batch arguments";
        return FS_ERR_INVALID;
    }
    bool local = false;  // a member with a local or spatial field
    std::vector<fs_sim*> v((size_t)n);
    for (int i = 0; i < n; ++i) {
        if (!sims[i] || !sims[i]->built) {
            lead->err = "batch member " + std::to_string(i) + " has no parameters";
            return FS_ERR_STATE;
        }
        if (sims[i]->p.precision != lead->p.precision) {
            lead->err = "batch members must share one precision";
            return FS_ERR_INVALID;
        }
        const Inst& M = sims[i]->inst;
        if ((M.exti64 && K > M.ext_K) || (M.sig && K > M.sig_K)) {
            lead->err = "batch member " + std::to_string(i) +
                        ": its local, spatial or thermal series is shorter than the protocol";
            return FS_ERR_INVALID;
        }
        local = local || M.exti64 != nullptr;
        v[(size_t)i] = sims[i];
    }
    if (schedule == FS_BATCH_PERSISTENT && local) {
        lead->err = "the persistent schedule takes no member with a local or spatial field";
        return FS_ERR_INVALID;
    }
    // FS_BATCH_AUTO takes the per-step launches: on the 512-member ensemble they
    // measured 1.26 s against 1.42 s for the persistent kernel (FP32; 1.62 s against
    // 1.68 s on FP64), whose relax CTAs (128 registers a thread, two per SM) leave a
    // sweeping CTA a fraction of the SM's warps and share its L1 with the chains
    const bool persist = schedule == FS_BATCH_PERSISTENT;
    // FS_BATCH_AUTO: two chains from twice as many members as SMs (512-member
    // ensemble: 1.252 s against 1.265 s in one chain, FP32; 1.601 s against 1.623 s,
    // FP64), else one
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const bool two = n >= 2 && (schedule == FS_BATCH_TWO_CHAINS ||
                                (schedule == FS_BATCH_AUTO && n >= 2 * nsm));
    // graphs cannot be captured on the legacy default stream: run the batch on a
    // stream of its own, ordered after the lead's queued work
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
        lead->err = "could not create a stream";
        return FS_ERR_CUDA;
    }
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    } guard{st};
    Arena tmp;
    double *dhx = nullptr, *dhy = nullptr;
    int64_t* dfps = nullptr;
    cudaError_t e;
    auto bail = [&](cudaError_t err, const char* where) {
        tmp.release(st);
        cudaStreamSynchronize(st);
        lead->err = std::string(where) + ": " + cudaGetErrorString(err);
        return FS_ERR_CUDA;
    };
    // members' own work must be finished before the batch reuses their buffers
    for (int i = 0; i < n; ++i)
        if ((e = cudaStreamSynchronize(v[(size_t)i]->stream)) != cudaSuccess)
            return bail(e, "sync");
    if ((e = tmp.alloc((void**)&dhx, 8 * std::max<int64_t>(K, 1), st)) != cudaSuccess)
        return bail(e, "alloc");
    if ((e = tmp.alloc((void**)&dhy, 8 * std::max<int64_t>(K, 1), st)) != cudaSuccess)
        return bail(e, "alloc");
    if (flips_per_step &&
        (e = tmp.alloc((void**)&dfps, 8 * std::max<int64_t>(K * n, 1), st)) != cudaSuccess)
        return bail(e, "alloc");
    if (K > 0) {
        if ((e = cudaMemcpyAsync(dhx, hx, 8 * K, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(e, "upload");
        if ((e = cudaMemcpyAsync(dhy, hy, 8 * K, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(e, "upload");
    }
    std::vector<Inst> descs((size_t)n);
    std::vector<InstState> states((size_t)n);
    for (int i = 0; i < n; ++i) {
        Inst I = v[(size_t)i]->inst;
        I.phx = dhx;
        I.phy = dhy;
        I.K = K;
        I.step0 = 0;
        I.resweep = resweep;
        I.log_step = nullptr;
        I.log_spin = nullptr;
        I.log_cap = 0;
        I.flips_per_step = dfps ? dfps + (int64_t)i * K : nullptr;
        descs[(size_t)i] = I;
        memset(&states[(size_t)i], 0, sizeof(InstState));
        states[(size_t)i].hash = seq_hash[i];
        states[(size_t)i].init = v[(size_t)i]->fields_valid ? 0 : 1;
        if ((e = cudaMemcpyAsync(v[(size_t)i]->d_state, &states[(size_t)i], sizeof(InstState),
                                 cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return bail(e, "upload");
    }
    BatchTable B;
    if ((e = B.upload(v, descs, st)) != cudaSuccess) return bail(e, "upload");
    // a batch whose sweep is long enough to matter times its own sweep builds
    // (about 20 sweeps); smaller ones keep the row-length rule
    if (K >= 16 && B.total_tasks >= 8192 &&
        (e = B.autotune(lead->p.precision, resweep ? 1 : 0, st)) != cudaSuccess)
        return bail(e, "autotune");
    const int prec = lead->p.precision;
    int levels = 1024;
    for (int i = 0; i < n; ++i) levels = std::max(levels, relax_smem_levels(v[(size_t)i]->n));
    if ((e = prepare_relax(prec, levels)) != cudaSuccess) return bail(e, "relax setup");
    // two chains: the members alternately by size into two tables, each with its
    // own field steps, forked from and joined to st in the graph
    BatchTable half[2];
    cudaStream_t st2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    struct ChainGuard {
        cudaStream_t* s;
        cudaEvent_t* a;
        cudaEvent_t* b;
        ~ChainGuard() {
            if (*s) {
                cudaStreamSynchronize(*s);
                cudaStreamDestroy(*s);
            }
            if (*a) cudaEventDestroy(*a);
            if (*b) cudaEventDestroy(*b);
        }
    } chain_guard{&st2, &ev_fork, &ev_join};
    if (two) {
        std::vector<fs_sim*> vs[2];
        std::vector<Inst> ds[2];
        for (int q = 0; q < n; ++q) {
            const int m = B.h_work[(size_t)q];  // (largest first)
            vs[q & 1].push_back(v[(size_t)m]);
            ds[q & 1].push_back(descs[(size_t)m]);
        }
        for (int c = 0; c < 2; ++c) {
            if ((e = half[c].upload(vs[c], ds[c], st)) != cudaSuccess) return bail(e, "upload");
            half[c].lanes = B.lanes;
            half[c].occ = B.occ;
        }
        if ((e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "streams");
    }
    // capture the whole protocol in one graph: one persistent launch, or the field
    // steps' launches (in one chain or two)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return bail(e, "capture");
    cudaError_t le = cudaSuccess;
    if (persist && K > 0) {
        le = B.enqueue_persistent(prec, resweep ? 1 : 0, levels, st);
    } else if (two) {
        le = cudaEventRecord(ev_fork, st);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(st2, ev_fork, 0);
        for (int64_t t = 0; t < K && le == cudaSuccess; ++t) {
            le = half[0].enqueue_step(prec, resweep ? 1 : 0, levels, st);
            if (le == cudaSuccess) le = half[1].enqueue_step(prec, resweep ? 1 : 0, levels, st2);
        }
        if (le == cudaSuccess) le = cudaEventRecord(ev_join, st2);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(st, ev_join, 0);
    } else {
        for (int64_t t = 0; t < K && le == cudaSuccess; ++t)
            le = B.enqueue_step(prec, resweep ? 1 : 0, levels, st);
    }
    e = cudaStreamEndCapture(st, &graph);
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bail(le, "launch");
    }
    if (e != cudaSuccess) return bail(e, "capture");
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return bail(e, "instantiate");
    }
    e = cudaGraphLaunch(exec, st);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return bail(e, "graph launch");
    }
    for (int i = 0; i < n; ++i)
        if ((e = cudaMemcpyAsync(&states[(size_t)i], v[(size_t)i]->d_state, sizeof(InstState),
                                 cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return bail(e, "download");
    if (flips_per_step && K > 0 &&
        (e = cudaMemcpyAsync(flips_per_step, dfps, 8 * K * n, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
        return bail(e, "download");
    int32_t ctl[4] = {0, 0, 0, 0};
    if (persist && K > 0 &&
        (e = cudaMemcpyAsync(ctl, B.q_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
        return bail(e, "download");
    e = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return bail(e, "protocol");
    tmp.release(st);
    B.mem.release(st);
    half[0].mem.release(st);
    half[1].mem.release(st);
    fs_status worst = FS_OK;
    for (int i = 0; i < n; ++i) {
        const InstState& S = states[(size_t)i];
        n_flips[i] = S.n_flips;
        seq_hash[i] = S.hash;
        status[i] = S.status;
        v[(size_t)i]->rechecks += S.rechecks;
        v[(size_t)i]->fields_valid = K > 0 ? true : v[(size_t)i]->fields_valid;
        if (S.status != ST_OK && worst == FS_OK) worst = (fs_status)S.status;
    }
    cudaStreamSynchronize(st);
    if (ctl[1] != 0) {
        lead->err = "persistent batch: no progress for 10 s";
        return FS_ERR_BOUNDS;
    }
    if (worst != FS_OK) lead->err = "a batch member stopped early (see status[])";
    return worst;
}

extern "C" fs_status fs_batch_run_protocol(fs_sim* const* sims, int32_t n, const double* hx,
                                           const double* hy, int64_t K, int32_t resweep,
                                           int64_t* n_flips, uint64_t* seq_hash,
                                           int32_t* status, int64_t* flips_per_step) {
    return fs_batch_run_protocol_ex(sims, n, hx, hy, K, resweep, FS_BATCH_AUTO, n_flips, seq_hash,
                                    status, flips_per_step);
}
