// fs_server.cu - continuous-batching server for simulation requests.
//
// Three parties:
//   - callers submit requests (geometry, parameters, field protocol) and poll;
//   - builder threads admit pending requests while their estimated device
//     footprint fits the budget, and build each (geometry, h_k draw, neighbour
//     tensors) on their own streams, overlapping the running iterations;
//   - the builder also captures a few field steps of the request's protocol (per
//     field step: external-field table, sweep, relax) as one CUDA graph; the
//     kernels take the step index from the simulation's device state, so the
//     same graph, launched again, runs the next steps;
//   - a worker thread launches every admitted request's graph on a stream of its
//     own, at most two launches in flight per request and the next one as soon as
//     one ends, so requests advance independently and their sweeps and relaxes
//     overlap on the device (requests that arrive while others run start as soon
//     as they are built), while the device's queues hold only a few steps of each
//     request (a whole protocol queued at once held up every later launch, the
//     builds' included, until it had run); finished requests are retired as
//     their last launch ends: final state read back, memory freed, budget
//     returned.
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
    cudaGraphExec_t exec = nullptr;  // kChunk field steps of the request's protocol
    int64_t launches = 0;            // launches of it that run the whole protocol
};

// Device bytes of one request before it is built: per island ~156 B of state
// and, per neighbour pair, the CSR entry and both coefficient widths with their
// transposed copies (40 B: on the FS_FP64 path the 32-bit ones are the build's
// scratch) and the FS_FP32_RECHECK path's 16-bit column offset (2 B); the degree
// is the cutoff disc's area times the array's island density, plus a margin for
// the rounding of the rows to multiples of 4.
double islands_of(const fs_request& r) {
    const double x = r.nx, y = r.ny;
    switch (r.kind) {
        case FS_KAGOME:
            return 3.0 * x * y + 2.0 * x + 2.0 * y;
        case FS_ISING:
            return x * y;
        case FS_PINWHEEL_DIAMOND:
            return 2.0 * x * y;
        case FS_SQUARE_OPEN:
        case FS_PINWHEEL_LUCKY_KNOT:
            return 2.0 * x * y - x - y;
        default:
            return 2.0 * x * y + x + y;
    }
}

size_t estimate_bytes(const fs_request& r) {
    const double rc = r.params.cutoff;
    const double n = islands_of(r);
    const double density = r.kind == FS_KAGOME ? 3.0 / (1.5 * std::sqrt(3.0))
                           : r.kind == FS_ISING ? 1.0
                                                : 2.0;
    const double deg = 1.05 * M_PI * rc * rc * density + 8.0;
    return (size_t)(n * (deg * 42.0 + 156.0) + 16.0 * r.K + (1 << 20));
}

// Admission order: a request that has waited longer than kAgeS goes first (oldest
// first), else the one with the least estimated work (islands x field steps), so
// that short requests are not queued behind long ones and long ones still start.
constexpr double kAgeS = 10.0;

// Field steps a request's graph holds; the worker keeps at most kInFlight launches
// of it queued.
constexpr int64_t kChunk = 8;
constexpr int kInFlight = 2;

double work_of(const fs_request& r) { return islands_of(r) * (double)std::max<int64_t>(r.K, 1); }

}  // namespace

struct fs_server {
    size_t budget = 0;
    int max_active = 256;
    std::atomic<size_t> used{0};
    std::chrono::steady_clock::time_point t0;
    cudaStream_t main_st = nullptr;
    std::vector<cudaStream_t> build_st;
    std::mutex mu;
    std::condition_variable cv_build, cv_work, cv_done;
    std::deque<std::shared_ptr<Job>> pending;
    std::deque<std::shared_ptr<Job>> ready;
    std::map<uint64_t, std::shared_ptr<Job>> jobs;
    uint64_t next_ticket = 1;
    int64_t outstanding = 0;
    bool stop = false;
    std::vector<std::thread> builders;
    std::thread worker;
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

// The pending request to admit next (index into S->pending; call with S->mu held).
size_t next_pending(const fs_server* S) {
    const double now = S->now();
    size_t best = 0;
    for (size_t q = 0; q < S->pending.size(); ++q) {
        const Job& j = *S->pending[q];
        if (now - j.res.t_submit > kAgeS) return q;  // the oldest aged request
        if (work_of(j.req) < work_of(S->pending[best]->req)) best = q;
    }
    return best;
}

void builder_loop(fs_server* S, int which) {
    cudaSetDevice(S->device);
    cudaStream_t bst = S->build_st[(size_t)which];
    for (;;) {
        std::shared_ptr<Job> j;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            size_t pick = 0;
            S->cv_build.wait_for(lk, std::chrono::milliseconds(100), [&] {
                if (S->stop) return true;
                if (S->pending.empty()) return false;
                pick = next_pending(S);
                const size_t need = estimate_bytes(S->pending[pick]->req);
                // admit when it fits, or when nothing else holds memory
                return S->used.load() + need <= S->budget || S->used.load() == 0;
            });
            if (S->stop) return;
            if (S->pending.empty()) continue;
            pick = next_pending(S);
            const size_t need = estimate_bytes(S->pending[pick]->req);
            if (!(S->used.load() + need <= S->budget || S->used.load() == 0)) continue;
            j = S->pending[pick];
            S->pending.erase(S->pending.begin() + (std::ptrdiff_t)pick);
            j->reserved = estimate_bytes(j->req);
            S->used += j->reserved;
        }
        j->res.t_admit = S->now();
        fs_sim* sim = nullptr;
        fs_status st = fs_create_geometry(j->req.kind, j->req.nx, j->req.ny, j->req.a, &sim);
        if (st == FS_OK) {
            fs_set_stream(sim, bst);
            // one CTA per request: a shared device does the most flips per SM this way
            // (a multi-flip cluster holds 8 SMs and waits for them to empty)
            fs_set_relax_mode(sim, FS_RELAX_SINGLE);
            st = fs_set_params(sim, &j->req.params);
        }
        if (st == FS_OK) {
            // protocol buffers live in the simulation's per-call arena
            Arena& A = sim->run;
            const int64_t K = std::max<int64_t>(j->req.K, 1);
            if (A.alloc((void**)&j->d_hx, 8 * K, bst) != cudaSuccess ||
                A.alloc((void**)&j->d_hy, 8 * K, bst) != cudaSuccess)
                st = FS_ERR_OOM;
            else if (j->req.K > 0 &&
                     (cudaMemcpyAsync(j->d_hx, j->hx.data(), 8 * j->req.K, cudaMemcpyHostToDevice,
                                      bst) != cudaSuccess ||
                      cudaMemcpyAsync(j->d_hy, j->hy.data(), 8 * j->req.K, cudaMemcpyHostToDevice,
                                      bst) != cudaSuccess))
                st = FS_ERR_CUDA;
            if (cudaStreamSynchronize(bst) != cudaSuccess) st = FS_ERR_CUDA;
        }
        if (st != FS_OK) {
            if (sim) fs_destroy(sim);
            S->used -= j->reserved;
            j->res.n = 0;
            finish(S, j, st);
            S->cv_build.notify_all();
            continue;
        }
        // descriptor and fresh state on the device, then kChunk field steps captured
        // as one graph (external-field table, sweep, relax per step; a kernel whose
        // step lies past K returns at once)
        if (st == FS_OK) {
            Inst I = sim->inst;
            I.phx = j->d_hx;
            I.phy = j->d_hy;
            I.K = j->req.K;
            I.step0 = 0;
            I.resweep = 1;
            I.log_step = nullptr;
            I.log_spin = nullptr;
            I.log_cap = 0;
            I.flips_per_step = nullptr;
            sim->inst_run = I;
            memset(&sim->state_host, 0, sizeof(InstState));
            sim->state_host.hash = fs_hash_init();
            sim->state_host.init = 1;
            cudaGraph_t graph = nullptr;
            bool ok = cudaMemcpy(sim->d_inst, &sim->inst_run, sizeof(Inst),
                                 cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(sim->d_state, &sim->state_host, sizeof(InstState),
                                 cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaStreamBeginCapture(bst, cudaStreamCaptureModeThreadLocal) ==
                          cudaSuccess;
            if (ok) {
                const int64_t c = std::min<int64_t>(std::max<int64_t>(j->req.K, 1), kChunk);
                j->launches = std::max<int64_t>((j->req.K + c - 1) / c, 1);
                const cudaError_t le = enqueue_steps(sim, j->req.K > 0 ? c : 0, 1, bst);
                const cudaError_t ce = cudaStreamEndCapture(bst, &graph);
                ok = le == cudaSuccess && ce == cudaSuccess && graph &&
                     cudaGraphInstantiate(&j->exec, graph, 0) == cudaSuccess;
            }
            if (graph) cudaGraphDestroy(graph);
            if (!ok) {
                if (j->exec) cudaGraphExecDestroy(j->exec);
                j->exec = nullptr;
                st = FS_ERR_CUDA;
            }
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

// The worker: every admitted request's graph is launched on a stream of its own,
// each launch followed by an event, kInFlight at most queued; requests therefore
// advance independently and their kernels overlap on the device. Progress and
// completion are found by polling the events.
void worker_loop(fs_server* S) {
    cudaSetDevice(S->device);
    struct Active {
        std::shared_ptr<Job> job;
        cudaStream_t stream = nullptr;
        int prio = 0;
        cudaEvent_t ev[kInFlight] = {};
        int64_t launched = 0, ended = 0;  // launches queued, launches ended
        cudaError_t err = cudaSuccess;
    };
    std::vector<Active> active;
    std::map<int, std::vector<cudaStream_t>> free_streams;  // by priority
    std::vector<cudaEvent_t> free_events;
    // Smaller requests run at higher stream priorities (the builders' level excepted):
    // their kernels are short, and taking SMs first they finish and leave the device to
    // the long flip chains of the large requests (measured on the 40-request stream, in
    // three pairs of runs: 0.75/0.95/0.83M flips/s against 0.68/0.92/0.73M with the
    // larger requests first).
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    auto prio_of = [&](int64_t n) {
        const int levels = std::max(0, prio_lo - prio_hi - 1);  // below the builders'
        const double lg = std::log2((double)std::max<int64_t>(n, 1));
        const int big = std::min(levels, std::max(0, (int)(lg - 14.0) / 2));
        return prio_lo - (levels - big);
    };
    auto take_event = [&](cudaEvent_t* e) {
        if (!free_events.empty()) {
            *e = free_events.back();
            free_events.pop_back();
            return true;
        }
        return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    };
    auto give_back = [&](Active& a) {
        if (a.stream) free_streams[a.prio].push_back(a.stream);
        for (cudaEvent_t& e : a.ev)
            if (e) free_events.push_back(e);
    };
    // queues launches until kInFlight are in flight or all are queued
    auto top_up = [&](Active& a) {
        const Job& j = *a.job;
        while (a.err == cudaSuccess && a.launched < j.launches &&
               a.launched - a.ended < kInFlight) {
            cudaError_t e = cudaGraphLaunch(j.exec, a.stream);
            if (e == cudaSuccess) e = cudaEventRecord(a.ev[a.launched % kInFlight], a.stream);
            if (e != cudaSuccess) a.err = e;
            ++a.launched;
        }
    };
    for (;;) {
        std::vector<std::shared_ptr<Job>> joining;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (active.empty())
                S->cv_work.wait(lk, [&] { return S->stop || !S->ready.empty(); });
            else
                S->cv_work.wait_for(lk, std::chrono::microseconds(200),
                                    [&] { return S->stop || !S->ready.empty(); });
            if (S->stop) break;
            while (!S->ready.empty() &&
                   (int)(active.size() + joining.size()) < S->max_active) {
                joining.push_back(S->ready.front());
                S->ready.pop_front();
            }
        }
        for (auto& j : joining) {
            Active a;
            a.job = j;
            a.prio = prio_of(j->sim->n);
            auto& pool = free_streams[a.prio];
            if (!pool.empty()) {
                a.stream = pool.back();
                pool.pop_back();
            } else if (cudaStreamCreateWithPriority(&a.stream, cudaStreamNonBlocking, a.prio) !=
                       cudaSuccess) {
                a.stream = nullptr;
            }
            bool ok = a.stream != nullptr;
            for (cudaEvent_t& e : a.ev) ok = ok && take_event(&e);
            fs_sim* sim = j->sim;
            if (ok) {
                sim->stream = a.stream;
                top_up(a);
                ok = a.err == cudaSuccess;
            }
            if (!ok) {
                if (a.stream) cudaStreamSynchronize(a.stream);
                if (j->exec) cudaGraphExecDestroy(j->exec);
                j->exec = nullptr;
                fs_destroy(sim);
                j->sim = nullptr;
                S->used -= j->reserved;
                S->cv_build.notify_all();
                finish(S, j, FS_ERR_CUDA);
                give_back(a);
                continue;
            }
            active.push_back(a);
        }
        // advance every request; retire the finished ones
        std::vector<Active> keep;
        for (auto& a : active) {
            while (a.err == cudaSuccess && a.ended < a.launched) {
                const cudaError_t q = cudaEventQuery(a.ev[a.ended % kInFlight]);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) a.err = q;
                ++a.ended;
            }
            top_up(a);
            if (a.err == cudaSuccess && a.ended < a.job->launches) {
                keep.push_back(a);
                continue;
            }
            auto& j = a.job;
            // the request's work has ended: read its state (and spins) back now; a
            // copy into pageable memory queued earlier would have blocked this thread
            cudaError_t e = a.err;
            if (e != cudaSuccess) cudaStreamSynchronize(a.stream);
            InstState& st = j->sim->state_host;
            if (e == cudaSuccess)
                e = cudaMemcpy(&st, j->sim->d_state, sizeof(InstState), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && j->spins_out)
                e = cudaMemcpy(j->spins_out, j->sim->inst.s, j->sim->n, cudaMemcpyDeviceToHost);
            j->res.n_flips = st.n_flips;
            j->res.seq_hash = st.hash;
            const int32_t status = e != cudaSuccess ? FS_ERR_CUDA : st.status;
            const size_t bytes = j->reserved;
            cudaGraphExecDestroy(j->exec);
            j->exec = nullptr;
            fs_destroy(j->sim);
            j->sim = nullptr;
            S->used -= bytes;
            S->cv_build.notify_all();
            finish(S, j, status);
            give_back(a);
        }
        active.swap(keep);
    }
    for (auto& a : active) {
        cudaStreamSynchronize(a.stream);
        if (a.job->exec) cudaGraphExecDestroy(a.job->exec);
        fs_destroy(a.job->sim);
        a.job->sim = nullptr;
        finish(S, a.job, FS_ERR_STATE);
        give_back(a);
    }
    for (auto& pool : free_streams)
        for (cudaStream_t st : pool.second) cudaStreamDestroy(st);
    for (cudaEvent_t e : free_events) cudaEventDestroy(e);
}

}  // namespace

extern "C" fs_status fs_server_create(size_t hbm_budget, int32_t max_active, fs_server** out) {
    if (!out || hbm_budget == 0 || max_active <= 0) return FS_ERR_INVALID;
    fs_server* S = new fs_server();
    S->budget = hbm_budget;
    S->max_active = max_active;
    S->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&S->device);
    // the relax kernel's shared-memory limit is set before any capture
    if (prepare_relax(0, relax_smem_max()) != cudaSuccess ||
        prepare_relax(1, relax_smem_max()) != cudaSuccess) {
        delete S;
        return FS_ERR_CUDA;
    }
    const int nb = 8;  // builder threads, each with its own stream
    S->build_st.resize(nb, nullptr);
    bool ok = cudaStreamCreateWithFlags(&S->main_st, cudaStreamNonBlocking) == cudaSuccess;
    // builds run at the highest stream priority: their kernels and copies are short
    // steps between host synchronisations, which would otherwise wait behind the
    // running requests' sweeps for every SM they need
    int prio_lo = 0, prio_hi = 0;
    if (ok) ok = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) == cudaSuccess;
    for (int b = 0; b < nb && ok; ++b)
        ok = cudaStreamCreateWithPriority(&S->build_st[(size_t)b], cudaStreamNonBlocking,
                                          prio_hi) == cudaSuccess;
    if (!ok) {
        delete S;
        return FS_ERR_CUDA;
    }
    for (int b = 0; b < nb; ++b) S->builders.emplace_back(builder_loop, S, b);
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
    for (auto& t : S->builders)
        if (t.joinable()) t.join();
    if (S->worker.joinable()) S->worker.join();
    for (auto& j : S->ready) {
        if (j->exec) cudaGraphExecDestroy(j->exec);
        if (j->sim) fs_destroy(j->sim);
    }
    cudaStreamDestroy(S->main_st);
    for (cudaStream_t b : S->build_st) cudaStreamDestroy(b);
    delete S;
}
