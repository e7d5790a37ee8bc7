// fs_server.cu - continuous-batching server for simulation requests.
//
// Three parties:
//   - callers submit requests (geometry, parameters, field protocol) and poll;
//   - a builder thread admits pending requests while their estimated device
//     footprint fits the budget, and builds each (geometry, h_k draw, neighbour
//     tensors) on its own stream, overlapping the running iterations;
//   - a worker thread owns the active set and advances it one field step per
//     iteration (one batched sweep launch over every active member's rows, one
//     relax CTA per member), re-uploading the batch table only when members join
//     or leave. Finished members are retired between iterations: final state
//     read back, memory freed, budget returned.
// Device waits are all host-side stream synchronisations; no kernel waits on the
// host.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/flatspin_b300.h"
#include "fs_batch.h"
#include "fs_common.cuh"
#include "fs_internal.h"
#include "fs_kernels.h"

using namespace fs;

namespace {

struct Job {
    uint64_t ticket = 0;
    fs_request req{};
    std::vector<double> hx, hy;
    int8_t* spins_out = nullptr;
    fs_sim* sim = nullptr;
    size_t reserved = 0;
    fs_result res{};
    double* d_hx = nullptr;
    double* d_hy = nullptr;
};

// Device bytes of one request before it is built: per island ~80 B of state and,
// per neighbour pair, the CSR entry (4 B), both coefficient widths and the
// transposed copies (44 B); the degree is the cutoff disc's area times the
// array's island density, with 25% slack.
size_t estimate_bytes(const fs_request& r) {
    const double rc = r.params.cutoff;
    double n, density;
    if (r.kind == FS_KAGOME) {
        n = 3.0 * r.nx * r.ny + 2.0 * r.nx + 2.0 * r.ny;
        density = 3.0 / (1.5 * std::sqrt(3.0));
    } else {
        n = 2.0 * r.nx * r.ny + r.nx + r.ny;
        density = 2.0;
    }
    const double deg = 1.25 * M_PI * rc * rc * density + 8.0;
    return (size_t)(n * (deg * 44.0 + 96.0) + 8.0 * r.K * 2.0 + (1 << 20));
}

}  // namespace

struct fs_server {
    size_t budget = 0;
    int max_active = 256;
    std::atomic<size_t> used{0};
    std::chrono::steady_clock::time_point t0;
    cudaStream_t main_st = nullptr, build_st = nullptr;
    std::mutex mu;
    std::condition_variable cv_build, cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::deque<std::shared_ptr<Job>> ready;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    int64_t outstanding = 0;
    bool stop = false;
    std::thread builder, worker;
    std::string err;
    int device = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

void finish(fs_server* S, const std::shared_ptr<Job>& j, int32_t status) {
    std::lock_guard<std::mutex> g(S->mu);
    j->res.status = status;
    j->res.done = 1;
    j->res.t_done = S->now();
    --S->outstanding;
    S->cv_done.notify_all();
}

void builder_loop(fs_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::shared_ptr<Job> j;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_build.wait(lk, [&] {
                if (S->stop) return true;
                if (S->pending.empty()) return false;
                const size_t need = estimate_bytes(S->pending.front()->req);
                // admit when it fits, or when nothing else holds memory
                return S->used.load() + need <= S->budget || S->used.load() == 0;
            });
            if (S->stop) return;
            j = S->pending.front();
            S->pending.pop_front();
            j->reserved = estimate_bytes(j->req);
            S->used += j->reserved;
        }
        j->res.t_admit = S->now();
        fs_sim* sim = nullptr;
        fs_status st = fs_create_geometry(j->req.kind, j->req.nx, j->req.ny, j->req.a, &sim);
        if (st == FS_OK) {
            fs_set_stream(sim, S->build_st);
            st = fs_set_params(sim, &j->req.params);
        }
        if (st == FS_OK) {
            // protocol buffers live in the simulation's per-call arena
            Arena& A = sim->run;
            const int64_t K = std::max<int64_t>(j->req.K, 1);
            if (A.alloc((void**)&j->d_hx, 8 * K, S->build_st) != cudaSuccess ||
                A.alloc((void**)&j->d_hy, 8 * K, S->build_st) != cudaSuccess)
                st = FS_ERR_OOM;
            else if (j->req.K > 0 &&
                     (cudaMemcpyAsync(j->d_hx, j->hx.data(), 8 * j->req.K, cudaMemcpyHostToDevice,
                                      S->build_st) != cudaSuccess ||
                      cudaMemcpyAsync(j->d_hy, j->hy.data(), 8 * j->req.K, cudaMemcpyHostToDevice,
                                      S->build_st) != cudaSuccess))
                st = FS_ERR_CUDA;
            if (cudaStreamSynchronize(S->build_st) != cudaSuccess) st = FS_ERR_CUDA;
        }
        if (st != FS_OK) {
            if (sim) fs_destroy(sim);
            S->used -= j->reserved;
            j->res.n = 0;
            finish(S, j, st);
            S->cv_build.notify_all();
            continue;
        }
        // account the real footprint
        const size_t real = (size_t)(sim->mem.bytes + sim->run.bytes);
        S->used += real;
        S->used -= j->reserved;
        j->reserved = real;
        sim->stream = S->main_st;
        j->sim = sim;
        j->res.n = sim->n;
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->ready.push_back(j);
        }
        S->cv_work.notify_all();
    }
}

void worker_loop(fs_server* S) {
    cudaSetDevice(S->device);
    std::vector<std::shared_ptr<Job>> active[2];  // by precision
    BatchTable table[2];
    bool dirty[2] = {false, false};
    std::vector<InstState> states;
    const int smem = relax_smem_budget(0);
    prepare_relax(0, smem);
    prepare_relax(1, smem);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                return S->stop || !S->ready.empty() || !active[0].empty() || !active[1].empty();
            });
            if (S->stop) break;
            while (!S->ready.empty() &&
                   (int)(active[0].size() + active[1].size()) < S->max_active) {
                auto j = S->ready.front();
                S->ready.pop_front();
                const int p = j->req.params.precision == FS_FP32_RECHECK ? 1 : 0;
                // fresh protocol state of the joining member
                Inst I = j->sim->inst;
                I.phx = j->d_hx;
                I.phy = j->d_hy;
                I.K = j->req.K;
                I.step0 = 0;
                I.resweep = 1;
                I.log_step = nullptr;
                I.log_spin = nullptr;
                I.log_cap = 0;
                I.flips_per_step = nullptr;
                j->sim->inst_run = I;
                InstState st0;
                memset(&st0, 0, sizeof(st0));
                st0.hash = fs_hash_init();
                st0.init = 1;
                j->sim->state_host = st0;
                cudaMemcpyAsync(j->sim->d_state, &j->sim->state_host, sizeof(InstState),
                                cudaMemcpyHostToDevice, S->main_st);
                active[p].push_back(j);
                dirty[p] = true;
            }
        }
        // a chunk of iterations on both precision groups
        for (int p = 0; p < 2; ++p) {
            if (!dirty[p]) continue;
            std::vector<fs_sim*> sims;
            std::vector<Inst> descs;
            for (auto& j : active[p]) {
                sims.push_back(j->sim);
                descs.push_back(j->sim->inst_run);
            }
            table[p].upload(sims, descs, S->main_st);
            dirty[p] = false;
        }
        int64_t left = 0;
        for (int p = 0; p < 2; ++p)
            for (auto& j : active[p]) {
                (void)j;
                ++left;
            }
        const int chunk = 4;
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < chunk && e == cudaSuccess; ++it)
            for (int p = 0; p < 2 && e == cudaSuccess; ++p)
                e = table[p].enqueue_step(p, 1, smem, S->main_st);
        // read every member's progress
        for (int p = 0; p < 2; ++p) {
            states.resize(active[p].size());
            for (size_t q = 0; q < active[p].size(); ++q)
                cudaMemcpyAsync(&states[q], active[p][q]->sim->d_state, sizeof(InstState),
                                cudaMemcpyDeviceToHost, S->main_st);
            if (cudaStreamSynchronize(S->main_st) != cudaSuccess) e = cudaErrorUnknown;
            std::vector<std::shared_ptr<Job>> keep;
            for (size_t q = 0; q < active[p].size(); ++q) {
                auto& j = active[p][q];
                const InstState& s = states[q];
                if (e == cudaSuccess && s.t < j->req.K && s.status == ST_OK) {
                    keep.push_back(j);
                    continue;
                }
                j->res.n_flips = s.n_flips;
                j->res.seq_hash = s.hash;
                if (j->spins_out)
                    cudaMemcpy(j->spins_out, j->sim->inst.s, j->sim->n, cudaMemcpyDeviceToHost);
                const size_t bytes = j->reserved;
                fs_destroy(j->sim);
                j->sim = nullptr;
                S->used -= bytes;
                S->cv_build.notify_all();
                finish(S, j, e != cudaSuccess ? FS_ERR_CUDA : s.status);
                dirty[p] = true;
            }
            active[p].swap(keep);
        }
        (void)left;
    }
    for (int p = 0; p < 2; ++p) {
        for (auto& j : active[p]) {
            if (j->sim) fs_destroy(j->sim);
            finish(S, j, FS_ERR_STATE);
        }
        table[p].mem.release(S->main_st);
    }
    cudaStreamSynchronize(S->main_st);
}

}  // namespace

extern "C" fs_status fs_server_create(size_t hbm_budget, int32_t max_active, fs_server** out) {
    if (!out || hbm_budget == 0 || max_active <= 0) return FS_ERR_INVALID;
    fs_server* S = new fs_server();
    S->budget = hbm_budget;
    S->max_active = max_active;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    if (cudaStreamCreateWithFlags(&S->main_st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->build_st, cudaStreamNonBlocking) != cudaSuccess) {
        delete S;
        return FS_ERR_CUDA;
    }
    S->builder = std::thread(builder_loop, S);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return FS_OK;
}

extern "C" fs_status fs_server_submit(fs_server* S, const fs_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return FS_ERR_INVALID;
    if (req->K < 0 || (req->K > 0 && (!req->hx || !req->hy))) {
        std::lock_guard<std::mutex> g(S->mu);
        S->err = "bad protocol";
        return FS_ERR_INVALID;
    }
    auto j = std::make_shared<Job>();
    j->req = *req;
    j->hx.assign(req->hx, req->hx + req->K);
    j->hy.assign(req->hy, req->hy + req->K);
    j->req.hx = nullptr;
    j->req.hy = nullptr;
    j->spins_out = req->spins_out;
    {
        std::lock_guard<std::mutex> g(S->mu);
        j->ticket = S->next_ticket++;
        j->res.t_submit = S->now();
        S->jobs[j->ticket] = j;
        S->pending.push_back(j);
        ++S->outstanding;
        *ticket = j->ticket;
    }
    S->cv_build.notify_all();
    return FS_OK;
}

extern "C" fs_status fs_server_poll(fs_server* S, uint64_t ticket, fs_result* out) {
    if (!S || !out) return FS_ERR_INVALID;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) {
        S->err = "unknown ticket";
        return FS_ERR_INVALID;
    }
    if (!it->second->res.done) return FS_ERR_STATE;
    *out = it->second->res;
    S->jobs.erase(it);
    return FS_OK;
}

extern "C" fs_status fs_server_drain(fs_server* S) {
    if (!S) return FS_ERR_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->outstanding == 0; });
    return FS_OK;
}

extern "C" double fs_server_now(const fs_server* S) { return S ? S->now() : 0.0; }

extern "C" const char* fs_server_last_error(const fs_server* S) {
    return S ? S->err.c_str() : "";
}

extern "C" void fs_server_destroy(fs_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_build.notify_all();
    S->cv_work.notify_all();
    if (S->builder.joinable()) S->builder.join();
    if (S->worker.joinable()) S->worker.join();
    for (auto& j : S->pending) (void)j;
    for (auto& j : S->ready)
        if (j->sim) fs_destroy(j->sim);
    cudaStreamDestroy(S->main_st);
    cudaStreamDestroy(S->build_st);
    delete S;
}
