// fs_api.cu - the C ABI of include/flatspin_b300.h: simulation objects, device
// memory, the neighbour build, the field-step protocol driver and batches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "../../include/flatspin_b300.h"
#include "fs_build.h"
#include "fs_common.cuh"
#include "fs_host.h"
#include "fs_internal.h"
#include "fs_kernels.h"

using namespace fs;

namespace {

thread_local std::string g_last_error;

const char* cuda_msg(cudaError_t e) { return cudaGetErrorString(e); }

}  // namespace

// ---------------------------------------------------------------------------
// Device arena
// ---------------------------------------------------------------------------

namespace fs {

void Arena::release(cudaStream_t st) {
    for (void* p : blocks) cudaFreeAsync(p, st);
    blocks.clear();
    if (ws) (top ? ws->hi : ws->lo) = 0;
    bytes = 0;
}

cudaError_t Arena::alloc(void** out, size_t n, cudaStream_t st) {
    *out = nullptr;
    if (n == 0) n = 16;
    n = (n + 255) & ~(size_t)255;
    if (ws) {  // carved from the caller's buffer (its base and size are 256-aligned)
        if (ws->lo + ws->hi + n > ws->cap) return cudaErrorMemoryAllocation;
        if (top) {
            ws->hi += n;
            *out = ws->base + (ws->cap - ws->hi);
        } else {
            *out = ws->base + ws->lo;
            ws->lo += n;
        }
        bytes += (int64_t)n;
        return cudaSuccess;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, n, st);
    if (e != cudaSuccess) return e;
    blocks.push_back(p);
    bytes += (int64_t)n;
    *out = p;
    return cudaSuccess;
}

// Bound on |th32 - th64| / (|th_par| + |th_perp|) of the FP32 and FP64 thermal
// draws of one Philox block (the sum is at least sigma times the Box-Muller
// radius), from the maximum ulp errors the CUDA Math API documents for the FP32
// functions (an error of k ulp against the correctly rounded value is within
// k + 1/2 ulp, i.e. (2k + 1) u, of the exact one; u = 2^-24):
//  - u1 (or 1 - u1, formed exactly in integers) rounded to FP32 twice: 2u;
//  - ln u1: logf (1 ulp, 3u) plus 2u / ln 2 from u1's error, |ln u1| >= ln 2 when
//    u1 < 1/2; log1pf(-(1 - u1)) (1 ulp, 3u) plus 2u / (1 - om) <= 4u from the
//    argument's error, |ln(1 - om)| >= om: at most 7u;
//  - the radius sqrt(-2 ln u1): half of that plus sqrtf's rounding (correctly
//    rounded without fast-math): 4.5u;
//  - cos and sin of the angle: sincospif (1 ulp, 3u relative) of the exactly split
//    high part, the first-order correction's truncation (below 1e-13) and its
//    product (|pi x_lo| < 4e-7), one subtraction: 4u of the value plus 1e-6 u;
//  - the product with the radius (u), sigma rounded to FP32 (u) and the product
//    with it (u); the FP64 draw's own error (log, sqrt, sincos: a few 1e-16).
// 4.5u + 4u + 3u = 11.5u and change, taken as 12u.
const double kThermalRel = 12.0 * std::ldexp(1.0, -24);

// The smallest float at least v (v >= 0).
float up_float(double v) {
    float f = (float)v;
    if ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

int choose_lanes(double avg_groups) {
    if (avg_groups <= 4.5) return 4;
    if (avg_groups <= 8.5) return 8;
    if (avg_groups <= 16.5) return 16;
    return 8;
}

}  // namespace fs

static fs_status fail(fs_sim* s, fs_status code, const std::string& msg) {
    if (s)
        s->err = msg;
    else
        g_last_error = msg;
    return code;
}

static fs_status cfail(fs_sim* s, cudaError_t e, const char* where) {
    return fail(s, e == cudaErrorMemoryAllocation ? FS_ERR_OOM : FS_ERR_CUDA,
                std::string(where) + ": " + cuda_msg(e));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cfail(sim, e_, where); \
    } while (0)

extern "C" const char* fs_last_error(const fs_sim* sim) {
    return sim ? sim->err.c_str() : g_last_error.c_str();
}

extern "C" uint64_t fs_hash_init(void) { return 0xcbf29ce484222325ull; }

// ---------------------------------------------------------------------------
// Creation
// ---------------------------------------------------------------------------

static fs_status init_sim(fs_sim* sim, std::vector<double>&& x, std::vector<double>&& y,
                          std::vector<double>&& th, double a) {
    sim->n = (int64_t)x.size();
    sim->a = a;
    sim->x = std::move(x);
    sim->y = std::move(y);
    sim->theta = std::move(th);
    // angle classes: exact dedup of the angle values; (cos, sin) from the host libm
    std::map<uint64_t, uint16_t> seen;
    sim->cls.resize((size_t)sim->n);
    for (int64_t i = 0; i < sim->n; ++i) {
        uint64_t bits;
        memcpy(&bits, &sim->theta[(size_t)i], 8);
        auto it = seen.find(bits);
        if (it == seen.end()) {
            if (seen.size() >= 65536)
                return fail(sim, FS_ERR_INVALID, "more than 65536 distinct island angles");
            const uint16_t c = (uint16_t)seen.size();
            seen.emplace(bits, c);
            sim->cls_cos.push_back(std::cos(sim->theta[(size_t)i]));
            sim->cls_sin.push_back(std::sin(sim->theta[(size_t)i]));
            sim->cls[(size_t)i] = c;
        } else {
            sim->cls[(size_t)i] = it->second;
        }
    }
    return FS_OK;
}

extern "C" fs_status fs_create_geometry(int32_t kind, int32_t nx, int32_t ny, double a,
                                        fs_sim** out) {
    if (!out) return fail(nullptr, FS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (kind < FS_SQUARE || kind > FS_ISING)
        return fail(nullptr, FS_ERR_INVALID, "unknown geometry kind");
    if (nx <= 0 || ny <= 0 || nx > 100000 || ny > 100000 || !(a > 0.0))
        return fail(nullptr, FS_ERR_INVALID, "bad geometry size or spacing");
    Geometry g;
    if (!make_geometry(kind, nx, ny, a, g)) return fail(nullptr, FS_ERR_INVALID, "bad geometry");
    if ((int64_t)g.x.size() >= (1ll << 31) - 64)
        return fail(nullptr, FS_ERR_INVALID, "too many islands");
    fs_sim* sim = new fs_sim();
    const fs_status r = init_sim(sim, std::move(g.x), std::move(g.y), std::move(g.theta), a);
    if (r != FS_OK) {
        g_last_error = sim->err;
        delete sim;
        return r;
    }
    *out = sim;
    return FS_OK;
}

extern "C" fs_status fs_create_custom(int64_t n, const double* x, const double* y,
                                      const double* theta, double a, fs_sim** out) {
    if (!out) return fail(nullptr, FS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n <= 0 || n >= (1ll << 31) - 64 || !x || !y || !theta || !(a > 0.0))
        return fail(nullptr, FS_ERR_INVALID, "bad custom geometry arguments");
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i]) || !std::isfinite(y[i]) || !std::isfinite(theta[i]))
            return fail(nullptr, FS_ERR_INVALID, "non-finite position or angle");
    fs_sim* sim = new fs_sim();
    const fs_status r =
        init_sim(sim, std::vector<double>(x, x + n), std::vector<double>(y, y + n),
                 std::vector<double>(theta, theta + n), a);
    if (r != FS_OK) {
        g_last_error = sim->err;
        delete sim;
        return r;
    }
    *out = sim;
    return FS_OK;
}

extern "C" void fs_destroy(fs_sim* sim) {
    if (!sim) return;
    if (sim->graph_exec) cudaGraphExecDestroy(sim->graph_exec);
    cudaStreamSynchronize(sim->stream);
    for (cudaEvent_t e : sim->ev_pool) cudaEventDestroy(e);
    sim->run.release(sim->stream);
    sim->ext_mem.release(sim->stream);
    sim->sig_mem.release(sim->stream);
    sim->mem.release(sim->stream);
    cudaStreamSynchronize(sim->stream);
    delete sim;
}

extern "C" fs_status fs_set_relax_mode(fs_sim* sim, int32_t mode) {
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    if (mode != FS_RELAX_AUTO && mode != FS_RELAX_SINGLE && mode != FS_RELAX_MULTI &&
        mode != FS_RELAX_MULTI_CTA)
        return fail(sim, FS_ERR_INVALID, "unknown relax mode");
    sim->relax_mode = mode;
    return FS_OK;
}

extern "C" fs_status fs_set_stream(fs_sim* sim, void* stream) {
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    sim->stream = (cudaStream_t)stream;
    return FS_OK;
}

// ---------------------------------------------------------------------------
// Parameters and the neighbour build
// ---------------------------------------------------------------------------

static bool bad_double(double v) { return !std::isfinite(v); }

// Per-island scales of the evaluations: 1 / (b h_k) and 1 / (c h_k) in double (the
// FP64 astroid's), each rounded once more to FP32 (the FP32 one's).
static void fill_rbc(fs_sim* sim) {
    sim->rbc32.resize((size_t)sim->n);
    sim->rbc64.resize((size_t)sim->n);
    // (the parallel-only criterion compares |h_par| with h_k itself: b = 1)
    const double b = sim->p.criterion == FS_CRITERION_PARALLEL ? 1.0 : sim->p.b;
    for (int64_t i = 0; i < sim->n; ++i) {
        const double h = sim->hk[(size_t)i];
        const double rb = 1.0 / (b * h), rc = 1.0 / (sim->p.c * h);
        sim->rbc64[(size_t)i] = make_double2(rb, rc);
        sim->rbc32[(size_t)i] = make_float2((float)rb, (float)rc);
    }
}

// Size of one Arena allocation of b bytes (as Arena::alloc rounds it).
static size_t arena_round(size_t b) {
    if (b == 0) b = 16;
    return (b + 255) & ~(size_t)255;
}

// Nodes of the max-tree above the leaves: fan-out 32, every level up to the root.
static int64_t tree_nodes(int64_t n) {
    int64_t cnt = (n + 31) / 32, total = 0;
    for (;;) {
        total += cnt;
        if (cnt == 1) return total;
        cnt = (cnt + 31) / 32;
    }
}

// Device bytes of one build: the simulation's state (kept until the next build or
// fs_destroy) and the build's temporaries (released when it returns), every
// allocation rounded as Arena::alloc rounds it. fs_build_sim checks its arenas
// against this after allocating, so the two cannot drift apart.
struct PlanBytes {
    size_t state = 0, temps = 0;
};

static PlanBytes plan_bytes(int64_t n, size_t ncls, int64_t ncell, int64_t nnzp, bool fp32,
                            bool thermal) {
    PlanBytes b;
    auto T = [&](int64_t x) { b.temps += arena_round((size_t)x); };
    auto S = [&](int64_t x) { b.state += arena_round((size_t)x); };
    const int64_t nc = (int64_t)ncls;
    const int64_t scr = std::max(scan_scratch_elems(ncell + 1), scan_scratch_elems(n + 1)) + 8;
    // count phase: positions, classes, cell grid, degrees, scan, rows
    T(8 * n), T(8 * n), T(2 * n), T(16 * nc);
    T(4 * n), T(4 * ncell), T(4 * (ncell + 1)), T(4 * n), T(8 * (ncell + 1)), T(8 * (ncell + 1));
    T(8 * n), T(8 * scr), T((int64_t)sizeof(BuildStats)), T(8 * (n + 1));
    // neighbour tensors (the 32-bit ones are scratch on the FP64 path)
    S(8 * (n + 1)), S(4 * nnzp), S(16 * nnzp), S(8 * nnzp);
    if (fp32)
        S(8 * nnzp), S(4 * nnzp), S(2 * nnzp);  // (with the 16-bit column offsets)
    else
        T(8 * nnzp), T(4 * nnzp);
    // islands, classes, relax state
    S(n), S(16 * n), S(8 * n), S(2 * n), S(16 * nc), S(8 * nc);
    S(16 * n), S(8 * n), S((int64_t)sizeof(IslandRec) * n), S(8 * n), S(16 * nc), S(8 * nc);
    S(16 * n);  // island centres
    if (thermal) S(8 * n), S(16 * n), S(4 * n);
    const int64_t total = tree_nodes(n);
    S(8 * total), S(4 * total);
    S((int64_t)sizeof(InstState)), S((int64_t)sizeof(Inst)), S(16), S(8), S(16), S(16);
    S(8 * 5 * n);
    return b;
}

// The neighbour build's cell grid for cutoff rc: cells of at least rc, doubled
// while there are more than 4 n + 4096 of them.
static void grid_of(const fs_sim* sim, double rc, BuildWork& w) {
    const int64_t n = sim->n;
    double xmin = sim->x[0], xmax = sim->x[0], ymin = sim->y[0], ymax = sim->y[0];
    for (int64_t i = 1; i < n; ++i) {
        xmin = std::min(xmin, sim->x[i]);
        xmax = std::max(xmax, sim->x[i]);
        ymin = std::min(ymin, sim->y[i]);
        ymax = std::max(ymax, sim->y[i]);
    }
    double cell = rc * 1.0001;
    auto dims = [&](double c, int64_t& gx, int64_t& gy) {
        gx = (int64_t)std::floor((xmax - xmin) / c) + 1;
        gy = (int64_t)std::floor((ymax - ymin) / c) + 1;
    };
    dims(cell, w.gx, w.gy);
    while ((double)w.gx * (double)w.gy > 4.0 * (double)n + 4096.0) {
        cell *= 2.0;
        dims(cell, w.gx, w.gy);
    }
    w.xmin = xmin;
    w.ymin = ymin;
    w.cell = cell;
}

// First phase of the build: positions and classes uploaded, the cell grid, every
// island's padded degree and the row pointers (*rp_out), with temporaries from
// `tmp` on `st`. Fills in, w and stats; returns the padded pair count in *nnzp.
static fs_status count_pairs(fs_sim* sim, const fs_params& p, Arena& tmp, cudaStream_t st,
                             BuildIn& in, BuildWork& w, int64_t** rp_out, BuildStats& stats,
                             int64_t* nnzp) {
    const int64_t n = sim->n;
    auto talloc = [&](void** q, size_t b) { return tmp.alloc(q, b, st); };
    double *dx = nullptr, *dy = nullptr;
    uint16_t* dcls = nullptr;
    double2* dcs = nullptr;
    const size_t ncls = sim->cls_cos.size();
    std::vector<double2> cs64(ncls);
    for (size_t c = 0; c < ncls; ++c) cs64[c] = make_double2(sim->cls_cos[c], sim->cls_sin[c]);
    CK(talloc((void**)&dx, 8 * n), "alloc");
    CK(talloc((void**)&dy, 8 * n), "alloc");
    CK(talloc((void**)&dcls, 2 * n), "alloc");
    CK(talloc((void**)&dcs, 16 * ncls), "alloc");
    CK(cudaMemcpyAsync(dx, sim->x.data(), 8 * n, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(dy, sim->y.data(), 8 * n, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(dcls, sim->cls.data(), 2 * n, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(dcs, cs64.data(), 16 * ncls, cudaMemcpyHostToDevice, st), "upload");

    in.n = n;
    in.x = dx;
    in.y = dy;
    in.cls = dcls;
    in.cs = dcs;
    const double rc = p.cutoff * sim->a;
    in.rc2 = rc * rc * (1.0 + 1e-9);
    in.alpha = p.alpha;

    grid_of(sim, rc, w);
    const int64_t ncell = w.gx * w.gy;
    CK(talloc((void**)&w.cell_of, 4 * n), "alloc");
    CK(talloc((void**)&w.cell_cnt, 4 * ncell), "alloc");
    CK(talloc((void**)&w.cell_start, 4 * (ncell + 1)), "alloc");
    CK(talloc((void**)&w.items, 4 * n), "alloc");
    CK(talloc((void**)&w.tmp64, 8 * (ncell + 1)), "alloc");
    CK(talloc((void**)&w.tmp64b, 8 * (ncell + 1)), "alloc");
    CK(talloc((void**)&w.deg_pad, 8 * n), "alloc");
    const int64_t scr = std::max(scan_scratch_elems(ncell + 1), scan_scratch_elems(n + 1)) + 8;
    CK(talloc((void**)&w.scratch, 8 * scr), "alloc");
    CK(talloc((void**)&w.stats, sizeof(BuildStats)), "alloc");
    int64_t* rp_tmp = nullptr;
    CK(talloc((void**)&rp_tmp, 8 * (n + 1)), "alloc");

    CK(build_cells(in, w, st), "cell grid");
    CK(build_degrees(in, w, st), "degrees");
    CK(build_rows(in, w, rp_tmp, st), "row scan");
    *nnzp = 0;
    CK(cudaMemcpyAsync(&stats, w.stats, sizeof(stats), cudaMemcpyDeviceToHost, st), "stats");
    CK(cudaMemcpyAsync(nnzp, rp_tmp + n, 8, cudaMemcpyDeviceToHost, st), "stats");
    CK(cudaStreamSynchronize(st), "build sync");
    *rp_out = rp_tmp;
    return FS_OK;
}

fs_status fs_build_sim(fs_sim* sim) {
    cudaStream_t st = sim->stream;
    const int64_t n = sim->n;
    const fs_params& p = sim->p;
    sim->mem.release(st);
    sim->fields_valid = false;

    // ---- temporaries of the build (the top of a bound workspace)
    Arena tmp;
    if (sim->ws.base) {
        sim->ws.hi = 0;
        tmp.ws = &sim->ws;
        tmp.top = true;
    }
    auto talloc = [&](void** q, size_t b) { return tmp.alloc(q, b, st); };
    const size_t ncls = sim->cls_cos.size();
    std::vector<double2> cs64(ncls);
    for (size_t c = 0; c < ncls; ++c) cs64[c] = make_double2(sim->cls_cos[c], sim->cls_sin[c]);
    BuildIn in;
    BuildWork w;
    BuildStats stats;
    int64_t* rp_tmp = nullptr;
    int64_t nnzp = 0;
    {
        const fs_status r = count_pairs(sim, p, tmp, st, in, w, &rp_tmp, stats, &nnzp);
        if (r != FS_OK) {
            tmp.release(st);
            return r;
        }
    }
    const uint16_t* dcls = in.cls;
    if (stats.max_deg > kMaxPaddedDegree) {
        tmp.release(st);
        return fail(sim, FS_ERR_INVALID,
                    "neighbourhood too large: " + std::to_string(stats.max_deg) +
                        " neighbours (max " + std::to_string(kMaxPaddedDegree) +
                        "); reduce the cutoff");
    }
    double bound;
    memcpy(&bound, &stats.bound_bits, 8);
    bound *= 1.000001;
    int e64 = 0, e32 = 0;
    if (bound > 0.0) {
        e64 = (int)std::floor(62.0 - std::log2(bound));
        e32 = (int)std::floor(30.0 - std::log2(bound));
    }
    e64 = std::max(-900, std::min(e64, 900));
    e32 = std::max(-900, std::min(e32, 900));
    sim->e64 = e64;
    sim->e32 = e32;
    sim->nnzp = nnzp;
    sim->max_deg = stats.max_deg;

    // ---- persistent arrays
    Inst& I = sim->inst;
    memset(&I, 0, sizeof(I));
    I.n = n;
    I.nnzp = nnzp;
    I.prec = p.precision;
    auto palloc = [&](void** q, size_t b) { return sim->mem.alloc(q, b, st); };
    int64_t* rp = nullptr;
    int32_t* col = nullptr;
    longlong2* pq64 = nullptr;
    long long* qt64 = nullptr;
    int2* pq32 = nullptr;
    int* qt32 = nullptr;
    CK(palloc((void**)&rp, 8 * (n + 1)), "alloc");
    CK(palloc((void**)&col, 4 * nnzp), "alloc");
    CK(palloc((void**)&pq64, 16 * nnzp), "alloc");
    CK(palloc((void**)&qt64, 8 * nnzp), "alloc");
    if (p.precision == FS_FP32_RECHECK) {
        CK(palloc((void**)&pq32, 8 * nnzp), "alloc");
        CK(palloc((void**)&qt32, 4 * nnzp), "alloc");
    } else {
        // the fill kernel writes both widths; the 32-bit ones go to scratch
        CK(talloc((void**)&pq32, 8 * nnzp), "alloc");
        CK(talloc((void**)&qt32, 4 * nnzp), "alloc");
    }
    CK(cudaMemcpyAsync(rp, rp_tmp, 8 * (n + 1), cudaMemcpyDeviceToDevice, st), "copy");
    BuildOut o;
    o.scale64 = std::ldexp(1.0, e64);
    o.scale32 = std::ldexp(1.0, e32);
    o.rp = rp;
    o.col = col;
    o.pq64 = pq64;
    o.qt64 = qt64;
    o.pq32 = pq32;
    o.qt32 = qt32;
    CK(build_fill(in, w, o, st), "fill");
    // The FP32 sweeps read 16-bit column offsets instead of col when every one fits
    // (lattice orderings keep neighbours close in index); read back below.
    int16_t* dcol = nullptr;
    int32_t dcol_over = 1;
    if (p.precision == FS_FP32_RECHECK) {
        CK(palloc((void**)&dcol, 2 * nnzp), "alloc");
        CK(build_dcol(n, rp, col, dcol, &w.stats->dcol_over, st), "offsets");
        CK(cudaMemcpyAsync(&dcol_over, &w.stats->dcol_over, 4, cudaMemcpyDeviceToHost, st),
           "stats");
    }
    I.rp = rp;
    I.col = col;
    I.pq64 = pq64;
    I.qt64 = qt64;
    I.pq32 = p.precision == FS_FP32_RECHECK ? pq32 : nullptr;
    I.qt32 = p.precision == FS_FP32_RECHECK ? qt32 : nullptr;

    // islands
    int8_t* s = nullptr;
    double2* rbc64 = nullptr;
    float2* rbc32 = nullptr;
    uint16_t* cls = nullptr;
    double2* c64 = nullptr;
    float2* c32 = nullptr;
    CK(palloc((void**)&s, n), "alloc");
    CK(palloc((void**)&rbc64, 16 * n), "alloc");
    CK(palloc((void**)&rbc32, 8 * n), "alloc");
    CK(palloc((void**)&cls, 2 * n), "alloc");
    CK(palloc((void**)&c64, 16 * ncls), "alloc");
    CK(palloc((void**)&c32, 8 * ncls), "alloc");
    std::vector<float2> cs32(ncls);
    for (size_t c = 0; c < ncls; ++c)
        cs32[c] = make_float2((float)sim->cls_cos[c], (float)sim->cls_sin[c]);
    CK(cudaMemsetAsync(s, 1, n, st), "init spins");
    CK(cudaMemcpyAsync(cls, dcls, 2 * n, cudaMemcpyDeviceToDevice, st), "copy");
    CK(cudaMemcpyAsync(c64, cs64.data(), 16 * ncls, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(c32, cs32.data(), 8 * ncls, cudaMemcpyHostToDevice, st), "upload");
    I.s = s;
    I.rbc64 = rbc64;
    I.rbc32 = rbc32;
    I.cls = cls;
    I.cs64 = c64;
    I.cs32 = c32;

    CK(palloc((void**)&I.h64, 16 * n), "alloc");
    CK(palloc((void**)&I.key32, 8 * n), "alloc");
    CK(palloc((void**)&I.rec, sizeof(IslandRec) * n), "alloc");
    CK(palloc((void**)&I.key64, 8 * n), "alloc");
    CK(palloc((void**)&I.ext64, 16 * ncls), "alloc");
    CK(palloc((void**)&I.ext32, 8 * ncls), "alloc");
    I.nclass = (int32_t)ncls;
    {
        double2* pos = nullptr;
        CK(palloc((void**)&pos, 16 * n), "alloc");
        std::vector<double2> hp((size_t)n);
        for (int64_t i = 0; i < n; ++i)
            hp[(size_t)i] = make_double2(sim->x[(size_t)i], sim->y[(size_t)i]);
        CK(cudaMemcpyAsync(pos, hp.data(), 16 * n, cudaMemcpyHostToDevice, st), "upload");
        CK(cudaStreamSynchronize(st), "upload");  // (the host copy goes out of scope)
        I.pos = pos;
        I.dcol = dcol_over == 0 ? dcol : nullptr;
        const double rc = 2.0 * p.cutoff * sim->a;
        I.rconf2 = rc * rc * (1.0 + 1e-6);
        // the same test on FP32 centres: each coordinate is within ext 2^-24 of its
        // double (ext: the largest magnitude), a difference within 3 ext 2^-24 more
        // (its own rounding included), so a squared distance below (rc + d)^2 with
        // d = 2 sqrt(2) 3 ext 2^-24 plus the FP32 sum's roundings covers every pair
        // within rc in double; widened further to be safe
        double ext = 1.0;
        for (int64_t i = 0; i < n; ++i)
            ext = std::max(ext, std::max(std::fabs(sim->x[(size_t)i]), std::fabs(sim->y[(size_t)i])));
        const double d = 10.0 * ext * std::ldexp(1.0, -24);
        I.rconf2f = up_float((rc + d) * (rc + d) * (1.0 + 1e-5) + 1e-6);
    }
    if (p.sigma_th > 0.0) {
        CK(palloc((void**)&I.th32, 8 * n), "alloc");
        CK(palloc((void**)&I.th64, 16 * n), "alloc");
        CK(palloc((void**)&I.th_step, 4 * n), "alloc");
        CK(cudaMemsetAsync(I.th_step, 0xFF, 4 * n, st), "init");
    }

    // max-tree levels above the leaves, fan-out 32
    int nlev = 0;
    int64_t cnt = (n + 31) / 32, total = 0;
    for (;;) {
        if (nlev >= kMaxLevels) return fail(sim, FS_ERR_INVALID, "system too large for the tree");
        I.lvl_n[nlev] = (int32_t)cnt;
        I.lvl_off[nlev] = total;
        total += cnt;
        ++nlev;
        if (cnt == 1) break;
        cnt = (cnt + 31) / 32;
    }
    I.nlev = nlev;
    CK(palloc((void**)&I.tree, 8 * total), "alloc");
    CK(palloc((void**)&sim->tcnt, 4 * total), "alloc");
    CK(cudaMemsetAsync(sim->tcnt, 0, 4 * total, st), "init");
    CK(palloc((void**)&sim->d_state, sizeof(InstState)), "alloc");
    CK(palloc((void**)&sim->d_inst, sizeof(Inst)), "alloc");
    CK(palloc((void**)&sim->d_task_start, 16), "alloc");
    CK(palloc((void**)&sim->d_tcnts, 8), "alloc");
    CK(palloc((void**)&sim->d_work, 16), "alloc");
    CK(palloc((void**)&sim->d_field, 16), "alloc");
    CK(palloc((void**)&sim->d_eval, 8 * 5 * n), "alloc");
    {
        const PlanBytes pb = plan_bytes(n, ncls, w.gx * w.gy, nnzp,
                                        p.precision == FS_FP32_RECHECK, p.sigma_th > 0.0);
        if ((size_t)sim->mem.bytes != pb.state || (size_t)tmp.bytes != pb.temps) {
            tmp.release(st);
            return fail(sim, FS_ERR_STATE, "internal: the build's device bytes differ from its plan");
        }
    }
    const int64_t ts[2] = {0, (n + 31) / 32};
    CK(cudaMemcpyAsync(sim->d_task_start, ts, 16, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(sim->d_tcnts, &sim->tcnt, 8, cudaMemcpyHostToDevice, st), "upload");
    const int32_t wk = 0;
    CK(cudaMemcpyAsync(sim->d_work, &wk, 4, cudaMemcpyHostToDevice, st), "upload");

    // parameters; the parallel-only criterion is the astroid's first term with
    // b = 1 and the exponent 1, without the second
    const bool parallel = p.criterion == FS_CRITERION_PARALLEL;
    I.perp = parallel ? 0 : 1;
    I.b = parallel ? 1.0 : p.b;
    I.c = p.c;
    I.pexp = parallel ? 1.0 : 2.0 / p.gamma;
    I.qexp = parallel ? 1.0 : 2.0 / p.beta;
    I.sigma = p.sigma_th;
    I.bf = (float)p.b;
    I.cf = (float)p.c;
    I.pexpf = (float)I.pexp;
    I.qexpf = (float)I.qexp;
    I.sigmaf = (float)p.sigma_th;
    I.inv64 = std::ldexp(1.0, -e64);
    I.inv64f = (float)std::ldexp(1.0, -e64);
    I.inv32 = (float)std::ldexp(1.0, -e32);
    I.seed = p.seed;
    I.instance = p.instance;
    I.max_flips = p.max_flips_per_step > 0 ? p.max_flips_per_step : 16 * n;
    I.st = sim->d_state;
    // FP32 error model, bounds on |FP32 evaluation - FS_FP64 evaluation| (u = 2^-24):
    //  - dh_abs: both fixed-point roundings over the longest row;
    //  - th_rel: the FP32 Box-Muller draw against the FP64 one, relative to the
    //    draw's radius (kThermalRel, from the documented ulp bounds);
    //  - dh_rel: three roundings of the field pieces (int to float, the external
    //    field to FP32, two sums: u |dp| + u |ext| + u |dp + ext| + u |h|, at most
    //    3u (|dp| + |ext| + |th|) and change), widened by 2^-20 for the FP64 sums'
    //    own roundings;
    //  - div_rel: 1 / (b h_k) rounded to FP32 (u) and the FP32 product (u) against
    //    the FP64 product with the FP64 reciprocal (2^-53), 2u + 2^-50;
    //  - pow_rel_*: the power. For the exponent 2/3, x rcbrtf(x): rcbrtf's
    //    documented 1 ulp (3u against the exact value) and the product's rounding,
    //    (1 + 3u)(1 + u) - 1 < 4.01u; otherwise powf at the FP32-rounded exponent,
    //    taken as 8 ulp (17u; no less than its documented maximum) plus the exponent's rounding
    //    |p - pf| |ln x| (lnk_*, applied per argument in pow_err). Both include
    //    2^-40 for the FP64 power's own error (pow: 2 ulp; the 2/3 power: 1.6 ulp).
    //    The bound arithmetic itself rounds outward.
    const double u = std::ldexp(1.0, -24);
    const double quant = (double)stats.max_deg * (std::ldexp(1.0, -e32 - 1) +
                                                  std::ldexp(1.0, -e64 - 1));
    I.dh_abs = up_float(quant * 1.5 + 1e-30);
    I.th_rel = up_float(kThermalRel);
    I.dh_rel = up_float(3.0 * u * (1.0 + std::ldexp(1.0, -20)));
    I.div_rel = up_float(2.0 * u + std::ldexp(1.0, -50));
    auto pmode = [](double e) { return e == 2.0 / 3.0 ? kPowCube : e == 1.0 ? kPowOne : kPowF; };
    I.pmode_p = pmode(I.pexp);
    I.pmode_q = pmode(I.qexp);
    auto prel = [&](int32_t m) {
        return up_float(m == kPowCube ? 4.01 * u + std::ldexp(1.0, -40)
                                      : m == kPowOne ? std::ldexp(1.0, -40)
                                                     : 17.0 * u + std::ldexp(1.0, -40));
    };
    const double ln2 = 0.69314718055994530942;
    I.pow_rel_p = prel(I.pmode_p);
    I.pow_rel_q = prel(I.pmode_q);
    I.lnk_p = I.pmode_p != kPowF
                  ? 0.0f
                  : up_float(std::fabs(I.pexp - (double)I.pexpf) * ln2 * (1.0 + 1e-6));
    I.lnk_q = I.pmode_q != kPowF
                  ? 0.0f
                  : up_float(std::fabs(I.qexp - (double)I.qexpf) * ln2 * (1.0 + 1e-6));
    sim->lanes = choose_lanes((double)nnzp / (double)n / 4.0);

    // coercive fields
    fill_rbc(sim);
    CK(cudaMemcpyAsync(rbc64, sim->rbc64.data(), 16 * n, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(rbc32, sim->rbc32.data(), 8 * n, cudaMemcpyHostToDevice, st), "upload");
    CK(cudaMemcpyAsync(sim->d_inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st), "upload");
    tmp.release(st);
    CK(cudaStreamSynchronize(st), "build");
    CK(cudaGetDevice(&sim->device), "device");
    sim->built = true;
    return FS_OK;
}

static fs_status check_params(fs_sim* sim, const fs_params* p) {
    if (!sim || !p) return fail(sim, FS_ERR_INVALID, "NULL argument");
    if (bad_double(p->alpha) || bad_double(p->hk) || bad_double(p->k_disorder) ||
        bad_double(p->b) || bad_double(p->c) || bad_double(p->beta) || bad_double(p->gamma) ||
        bad_double(p->cutoff) || bad_double(p->sigma_th))
        return fail(sim, FS_ERR_INVALID, "non-finite parameter");
    if (!(p->hk > 0.0) || !(p->b > 0.0) || !(p->c > 0.0) || !(p->beta > 0.0) ||
        !(p->gamma > 0.0) || !(p->cutoff > 0.0) || p->sigma_th < 0.0 || p->k_disorder < 0.0 ||
        p->alpha < 0.0)
        return fail(sim, FS_ERR_INVALID, "parameter out of range");
    if (p->precision != FS_FP64 && p->precision != FS_FP32_RECHECK)
        return fail(sim, FS_ERR_INVALID, "unknown precision");
    if (p->criterion != FS_CRITERION_ASTROID && p->criterion != FS_CRITERION_PARALLEL)
        return fail(sim, FS_ERR_INVALID, "unknown switching criterion");
    return FS_OK;
}

extern "C" fs_status fs_workspace_bytes(const fs_sim* csim, const fs_params* p, size_t* bytes) {
    fs_sim* sim = const_cast<fs_sim*>(csim);  // (only its error message is written)
    if (!bytes) return fail(sim, FS_ERR_INVALID, "NULL argument");
    *bytes = 0;
    fs_status r = check_params(sim, p);
    if (r != FS_OK) return r;
    // the build's neighbour count, with its temporaries from the pool
    cudaStream_t st = sim->stream;
    Arena tmp;
    BuildIn in;
    BuildWork w;
    BuildStats stats;
    int64_t* rp_tmp = nullptr;
    int64_t nnzp = 0;
    r = count_pairs(sim, *p, tmp, st, in, w, &rp_tmp, stats, &nnzp);
    tmp.release(st);
    if (r != FS_OK) return r;
    if (stats.max_deg > kMaxPaddedDegree)
        return fail(sim, FS_ERR_INVALID,
                    "neighbourhood too large: " + std::to_string(stats.max_deg) +
                        " neighbours (max " + std::to_string(kMaxPaddedDegree) +
                        "); reduce the cutoff");
    const PlanBytes pb = plan_bytes(sim->n, sim->cls_cos.size(), w.gx * w.gy, nnzp,
                                    p->precision == FS_FP32_RECHECK, p->sigma_th > 0.0);
    *bytes = pb.state + pb.temps;
    return FS_OK;
}

extern "C" fs_status fs_bind_workspace(fs_sim* sim, void* dev_ptr, size_t bytes,
                                       void* cuda_stream) {
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    if (sim->built) return fail(sim, FS_ERR_STATE, "bind the workspace before fs_set_params");
    if (dev_ptr && ((uintptr_t)dev_ptr & 255u) != 0)
        return fail(sim, FS_ERR_INVALID, "workspace must start on a 256-byte boundary");
    if (dev_ptr) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, dev_ptr) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();  // (clear the lookup's error)
            return fail(sim, FS_ERR_INVALID, "workspace is not device memory");
        }
    }
    if (cuda_stream) sim->stream = (cudaStream_t)cuda_stream;
    sim->mem.release(sim->stream);  // (what a failed build left)
    sim->ws = Workspace{};
    sim->mem.ws = nullptr;
    if (dev_ptr) {
        sim->ws.base = (char*)dev_ptr;
        sim->ws.cap = bytes & ~(size_t)255;
        sim->mem.ws = &sim->ws;
        sim->mem.top = false;
    }
    return FS_OK;
}

extern "C" fs_status fs_set_params(fs_sim* sim, const fs_params* p) {
    const fs_status r = check_params(sim, p);
    if (r != FS_OK) return r;
    sim->p = *p;
    draw_hk(sim->n, p->hk, p->k_disorder, p->seed, p->instance, sim->hk);
    sim->built = false;
    // (new parameters drop any local, spatial or thermal series)
    sim->ext_mem.release(sim->stream);
    sim->sig_mem.release(sim->stream);
    const fs_status b = fs_build_sim(sim);
    // a failed build's queued work ends before the caller may reuse its buffer
    if (b != FS_OK) cudaStreamSynchronize(sim->stream);
    return b;
}

static fs_status need_built(fs_sim* sim) {
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    if (!sim->built) return fail(sim, FS_ERR_STATE, "parameters not set");
    return FS_OK;
}

extern "C" fs_status fs_set_hk(fs_sim* sim, const double* hk, int64_t n) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!hk || n != sim->n) return fail(sim, FS_ERR_INVALID, "hk must have n values");
    for (int64_t i = 0; i < n; ++i)
        if (!(hk[i] > 0.0) || !std::isfinite(hk[i]))
            return fail(sim, FS_ERR_INVALID, "hk values must be positive and finite");
    sim->hk.assign(hk, hk + n);
    fill_rbc(sim);
    CK(cudaMemcpyAsync((void*)sim->inst.rbc64, sim->rbc64.data(), 16 * n, cudaMemcpyHostToDevice,
                       sim->stream),
       "upload");
    CK(cudaMemcpyAsync((void*)sim->inst.rbc32, sim->rbc32.data(), 8 * n, cudaMemcpyHostToDevice,
                       sim->stream),
       "upload");
    CK(cudaStreamSynchronize(sim->stream), "sync");
    return FS_OK;
}

extern "C" fs_status fs_set_spins(fs_sim* sim, const int8_t* s, int64_t n) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!s || n != sim->n) return fail(sim, FS_ERR_INVALID, "spins must have n values");
    for (int64_t i = 0; i < n; ++i)
        if (s[i] != 1 && s[i] != -1) return fail(sim, FS_ERR_INVALID, "spins must be +1 or -1");
    CK(cudaMemcpyAsync(sim->inst.s, s, n, cudaMemcpyHostToDevice, sim->stream), "upload");
    CK(cudaStreamSynchronize(sim->stream), "sync");
    sim->fields_valid = false;
    return FS_OK;
}

extern "C" fs_status fs_set_field(fs_sim* sim, double hx, double hy, uint32_t step) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (bad_double(hx) || bad_double(hy)) return fail(sim, FS_ERR_INVALID, "non-finite field");
    sim->hx = hx;
    sim->hy = hy;
    sim->step = step;
    return FS_OK;
}

// ---------------------------------------------------------------------------
// Protocol driver
// ---------------------------------------------------------------------------

namespace fs {

// Dynamic shared memory of a relax CTA: the tree levels above the keys that the
// relax keeps (up to the first with at most kRelaxTopNodes nodes) and that fit in
// 96 KiB, counted from the top down (the kernel places them the same way). Small
// systems take little, so several relax CTAs share an SM.
int relax_smem_levels(int64_t n) {
    const int64_t cap = 96 * 1024;
    std::vector<int64_t> lv;
    int64_t cnt = (n + 31) / 32;
    for (;;) {
        lv.push_back(8 * cnt);
        if (cnt <= kRelaxTopNodes) break;
        cnt = (cnt + 31) / 32;
    }
    int64_t used = 0;
    for (size_t q = lv.size(); q-- > 0;) {
        if (used + lv[q] > cap) break;
        used += lv[q];
    }
    return (int)std::max<int64_t>(8 * kRelaxTopNodes, used);
}

int relax_smem_max() { return 96 * 1024; }

// Queues K field steps of one simulation (sweep + relax per step). The
// descriptor's protocol fields must already point at device buffers.
static cudaError_t next_event(fs_sim* sim, cudaEvent_t* ev) {
    if (sim->ev_used == sim->ev_pool.size()) {
        cudaEvent_t e;
        const cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        sim->ev_pool.push_back(e);
    }
    *ev = sim->ev_pool[sim->ev_used++];
    return cudaSuccess;
}

// Accumulates the durations of the recorded (ext, sweep, relax) launch triples.
cudaError_t collect_profile(fs_sim* sim) {
    if (sim->ev_used == 0) return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(sim->ev_pool[sim->ev_used - 1]);
    if (e != cudaSuccess) return e;
    for (size_t q = 0; q + 2 < sim->ev_used; q += 3) {
        float a = 0.0f, b = 0.0f;
        cudaEventElapsedTime(&a, sim->ev_pool[q], sim->ev_pool[q + 1]);
        cudaEventElapsedTime(&b, sim->ev_pool[q + 1], sim->ev_pool[q + 2]);
        sim->prof_sweep_ms += a;
        sim->prof_relax_ms += b;
        ++sim->prof_sweeps;
        ++sim->prof_relaxes;
    }
    sim->ev_used = 0;
    return cudaSuccess;
}

// Queues K field steps of one simulation: per step the external-field table,
// the sweep and the relax. With profiling on, events bracket the sweep and the
// relax of every step.
// Whether the simulation's relaxes run as multi-flip rounds: by choice, or (auto)
// for arrays large enough that many of the largest keys lie far apart.
bool relax_multi(const fs_sim* sim) {
    if (sim->relax_mode == FS_RELAX_MULTI || sim->relax_mode == FS_RELAX_MULTI_CTA) return true;
    if (sim->relax_mode == FS_RELAX_SINGLE) return false;
    return sim->n >= kMultiAutoIslands;
}

cudaError_t enqueue_steps(fs_sim* sim, int64_t K, int resweep, cudaStream_t st) {
    SweepLaunch S;
    S.tab = sim->d_inst;
    S.task_start = sim->d_task_start;
    S.n_inst = 1;
    S.total_tasks = (sim->n + 31) / 32;
    S.tcnts = sim->d_tcnts;
    S.prec = sim->p.precision;
    S.lanes_per_row = sim->lanes;
    S.occupancy = sim->sweep_occ;
    S.resweep = resweep ? 1 : 0;
    RelaxLaunch R;
    R.tab = sim->d_inst;
    R.work = sim->d_work;
    R.n_work = 1;
    R.prec = sim->p.precision;
    R.smem_levels = relax_smem_levels(sim->n);
    R.multi = !relax_multi(sim) ? 0 : sim->relax_mode == FS_RELAX_MULTI_CTA ? 2 : 1;
    cudaError_t e;
    if (sim->profiling && sim->ev_used + 3 * (size_t)K > 30000 &&
        (e = collect_profile(sim)) != cudaSuccess)
        return e;
    for (int64_t t = 0; t < K; ++t) {
        if ((e = launch_ext_table(S, st)) != cudaSuccess) return e;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        if (sim->profiling) {
            if ((e = next_event(sim, &e0)) != cudaSuccess) return e;
            if ((e = next_event(sim, &e1)) != cudaSuccess) return e;
            if ((e = next_event(sim, &e2)) != cudaSuccess) return e;
            cudaEventRecord(e0, st);
        }
        if ((e = launch_sweep(S, st)) != cudaSuccess) return e;
        if (sim->profiling) cudaEventRecord(e1, st);
        if ((e = launch_relax(R, st)) != cudaSuccess) return e;
        if (sim->profiling) cudaEventRecord(e2, st);
    }
    return cudaSuccess;
}

}  // namespace fs

struct RunBufs {
    double* hx = nullptr;
    double* hy = nullptr;
    uint32_t* ls = nullptr;
    uint32_t* lk = nullptr;
    int64_t* fps = nullptr;
};

// A protocol's field steps step0 .. step0 + K - 1 must lie inside the simulation's
// local, spatial and thermal series, when it has them.
static fs_status check_series(fs_sim* sim, uint64_t step0, int64_t K) {
    const uint64_t end = step0 + (uint64_t)std::max<int64_t>(K, 1);
    if (sim->inst.exti64 && end > (uint64_t)sim->inst.ext_K)
        return fail(sim, FS_ERR_INVALID, "field step beyond the local or spatial field series");
    if (sim->inst.sig && end > (uint64_t)sim->inst.sig_K)
        return fail(sim, FS_ERR_INVALID, "field step beyond the thermal series");
    return FS_OK;
}

static fs_status run_device(fs_sim* sim, const double* d_hx, const double* d_hy, int64_t K,
                            uint32_t step0, int32_t resweep, uint32_t* d_ls, uint32_t* d_lk,
                            int64_t log_cap, int64_t* d_fps, uint64_t hash0) {
    const fs_status rs = check_series(sim, step0, K);
    if (rs != FS_OK) return rs;
    cudaStream_t st = sim->stream;
    Inst I = sim->inst;
    I.phx = d_hx;
    I.phy = d_hy;
    I.K = K;
    I.step0 = step0;
    I.resweep = resweep;
    I.log_step = d_ls;
    I.log_spin = d_lk;
    I.log_cap = (d_ls && d_lk) ? log_cap : 0;
    I.flips_per_step = d_fps;
    InstState S;
    memset(&S, 0, sizeof(S));
    S.hash = hash0;
    S.init = sim->fields_valid ? 0 : 1;
    sim->inst_run = I;
    CK(cudaMemcpyAsync(sim->d_inst, &sim->inst_run, sizeof(Inst), cudaMemcpyHostToDevice, st),
       "upload");
    sim->state_host = S;
    CK(cudaMemcpyAsync(sim->d_state, &sim->state_host, sizeof(S), cudaMemcpyHostToDevice, st),
       "upload");
    CK(enqueue_steps(sim, K, resweep, st), "launch");
    if (K > 0) sim->fields_valid = true;
    return FS_OK;
}

static fs_status finish_run(fs_sim* sim, InstState* out) {
    CK(cudaMemcpyAsync(&sim->state_host, sim->d_state, sizeof(InstState), cudaMemcpyDeviceToHost,
                       sim->stream),
       "download");
    CK(cudaStreamSynchronize(sim->stream), "protocol");
    *out = sim->state_host;
    sim->rechecks += out->rechecks;
    sim->fallbacks += out->fallbacks;
    sim->rounds += out->rounds;
    sim->idle_rounds += out->idle;
    sim->round_flips += out->round_flips;
    sim->handoffs += out->handoffs;
    if (out->status == ST_NOT_CONVERGED)
        return fail(sim, FS_ERR_NOT_CONVERGED, "a relax exceeded max_flips_per_step");
    if (out->status == ST_BOUNDS)
        return fail(sim, FS_ERR_BOUNDS, "FP64 recheck did not settle (internal error)");
    if (out->status != ST_OK) return fail(sim, FS_ERR_CUDA, "device status " +
                                                                std::to_string(out->status));
    return FS_OK;
}

extern "C" fs_status fs_run_protocol(fs_sim* sim, const double* hx, const double* hy, int64_t K,
                                     uint32_t step0, int32_t resweep, uint32_t* log_step,
                                     uint32_t* log_spin, int64_t log_cap,
                                     int64_t* flips_per_step, uint64_t* seq_hash,
                                     int64_t* n_flips) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (K < 0 || (K > 0 && (!hx || !hy)) || !seq_hash || !n_flips)
        return fail(sim, FS_ERR_INVALID, "bad protocol arguments");
    if (log_cap < 0) return fail(sim, FS_ERR_INVALID, "log_cap < 0");
    for (int64_t t = 0; t < K; ++t)
        if (bad_double(hx[t]) || bad_double(hy[t]))
            return fail(sim, FS_ERR_INVALID, "non-finite field value");
    const bool want_log = log_step && log_spin && log_cap > 0;
    cudaStream_t st = sim->stream;
    sim->run.release(st);
    RunBufs b;
    auto ralloc = [&](void** q, size_t n) { return sim->run.alloc(q, n, st); };
    CK(ralloc((void**)&b.hx, 8 * std::max<int64_t>(K, 1)), "alloc");
    CK(ralloc((void**)&b.hy, 8 * std::max<int64_t>(K, 1)), "alloc");
    if (want_log) {
        CK(ralloc((void**)&b.ls, 4 * log_cap), "alloc");
        CK(ralloc((void**)&b.lk, 4 * log_cap), "alloc");
    }
    if (flips_per_step) CK(ralloc((void**)&b.fps, 8 * std::max<int64_t>(K, 1)), "alloc");
    if (K > 0) {
        CK(cudaMemcpyAsync(b.hx, hx, 8 * K, cudaMemcpyHostToDevice, st), "upload");
        CK(cudaMemcpyAsync(b.hy, hy, 8 * K, cudaMemcpyHostToDevice, st), "upload");
    }
    r = run_device(sim, b.hx, b.hy, K, step0, resweep, b.ls, b.lk, log_cap, b.fps, *seq_hash);
    if (r != FS_OK) return r;
    InstState S;
    r = finish_run(sim, &S);
    const int64_t m = std::min<int64_t>(S.n_flips, want_log ? log_cap : 0);
    if (m > 0) {
        CK(cudaMemcpyAsync(log_step, b.ls, 4 * m, cudaMemcpyDeviceToHost, st), "download");
        CK(cudaMemcpyAsync(log_spin, b.lk, 4 * m, cudaMemcpyDeviceToHost, st), "download");
    }
    if (flips_per_step && K > 0)
        CK(cudaMemcpyAsync(flips_per_step, b.fps, 8 * K, cudaMemcpyDeviceToHost, st), "download");
    CK(cudaStreamSynchronize(st), "download");
    *seq_hash = S.hash;
    *n_flips = S.n_flips;
    if (K > 0) {
        sim->hx = hx[K - 1];
        sim->hy = hy[K - 1];
        sim->step = step0 + (uint32_t)(K - 1);
    }
    return r;
}

// d_out: {status, n_flips, hash, rechecks}
__global__ void k_copy_out(const InstState* st, uint64_t* out) {
    out[0] = (uint64_t)(int64_t)st->status;
    out[1] = (uint64_t)st->n_flips;
    out[2] = st->hash;
    out[3] = (uint64_t)st->rechecks;
}

extern "C" fs_status fs_run_protocol_dev(fs_sim* sim, const double* d_hx, const double* d_hy,
                                         int64_t K, uint32_t step0, int32_t resweep,
                                         uint32_t* d_log_step, uint32_t* d_log_spin,
                                         int64_t log_cap, int64_t* d_flips_per_step,
                                         uint64_t* d_out) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (K < 0 || (K > 0 && (!d_hx || !d_hy)) || !d_out || log_cap < 0)
        return fail(sim, FS_ERR_INVALID, "bad protocol arguments");
    r = run_device(sim, d_hx, d_hy, K, step0, resweep, d_log_step, d_log_spin, log_cap,
                   d_flips_per_step, fs_hash_init());
    if (r != FS_OK) return r;
    k_copy_out<<<1, 1, 0, sim->stream>>>(sim->d_state, d_out);
    CK(cudaGetLastError(), "launch");
    return FS_OK;
}

extern "C" fs_status fs_relax(fs_sim* sim, uint32_t* log_spin, int64_t log_cap,
                              int64_t* n_flips) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!n_flips || log_cap < 0) return fail(sim, FS_ERR_INVALID, "bad arguments");
    std::vector<uint32_t> ls((size_t)std::max<int64_t>(log_cap, 0));
    uint64_t h = fs_hash_init();
    const double hx = sim->hx, hy = sim->hy;
    return fs_run_protocol(sim, &hx, &hy, 1, sim->step, 1, log_cap > 0 ? ls.data() : nullptr,
                           log_cap > 0 ? log_spin : nullptr, log_cap, nullptr, &h, n_flips);
}

// ---------------------------------------------------------------------------
// Read-back
// ---------------------------------------------------------------------------

extern "C" fs_status fs_get_spins(const fs_sim* csim, int8_t* out, int64_t n) {
    fs_sim* sim = const_cast<fs_sim*>(csim);
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!out || n != sim->n) return fail(sim, FS_ERR_INVALID, "out must hold n values");
    CK(cudaMemcpyAsync(out, sim->inst.s, n, cudaMemcpyDeviceToHost, sim->stream), "download");
    CK(cudaStreamSynchronize(sim->stream), "sync");
    return FS_OK;
}

// Brings the dipolar sums up to date for the current spins (one resweep).
static fs_status refresh_fields(fs_sim* sim) {
    if (sim->fields_valid) return FS_OK;
    cudaStream_t st = sim->stream;
    double f[2] = {sim->hx, sim->hy};
    CK(cudaMemcpyAsync(sim->d_field, f, 16, cudaMemcpyHostToDevice, st), "upload");
    Inst I = sim->inst;
    I.phx = sim->d_field;
    I.phy = sim->d_field + 1;
    I.K = 1;
    I.step0 = sim->step;
    sim->inst_run = I;
    CK(cudaMemcpyAsync(sim->d_inst, &sim->inst_run, sizeof(Inst), cudaMemcpyHostToDevice, st),
       "upload");
    memset(&sim->state_host, 0, sizeof(InstState));
    sim->state_host.init = 1;
    CK(cudaMemcpyAsync(sim->d_state, &sim->state_host, sizeof(InstState), cudaMemcpyHostToDevice,
                       st),
       "upload");
    SweepLaunch S;
    S.tab = sim->d_inst;
    S.task_start = sim->d_task_start;
    S.n_inst = 1;
    S.total_tasks = (sim->n + 31) / 32;
    S.tcnts = sim->d_tcnts;
    S.prec = sim->p.precision;
    S.resweep = 1;
    S.lanes_per_row = sim->lanes;
    S.occupancy = sim->sweep_occ;
    CK(launch_ext_table(S, st), "sweep");
    CK(launch_sweep(S, st), "sweep");
    CK(cudaStreamSynchronize(st), "sweep");
    sim->fields_valid = true;
    return FS_OK;
}

static fs_status eval_into(fs_sim* sim, double* hpar, double* hperp, double* lhs, double* lo,
                           double* hi, int64_t n) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (n != sim->n) return fail(sim, FS_ERR_INVALID, "outputs must hold n values");
    r = check_series(sim, sim->step, 1);
    if (r != FS_OK) return r;
    r = refresh_fields(sim);
    if (r != FS_OK) return r;
    cudaStream_t st = sim->stream;
    Inst I = sim->inst;
    sim->inst_run = I;
    CK(cudaMemcpyAsync(sim->d_inst, &sim->inst_run, sizeof(Inst), cudaMemcpyHostToDevice, st),
       "upload");
    double* d = sim->d_eval;
    CK(launch_eval_all(sim->d_inst, n, sim->hx, sim->hy, sim->step, d, st), "eval");
    double* outs[5] = {hpar, hperp, lhs, lo, hi};
    for (int q = 0; q < 5; ++q)
        if (outs[q])
            CK(cudaMemcpyAsync(outs[q], d + q * n, 8 * n, cudaMemcpyDeviceToHost, st), "download");
    CK(cudaStreamSynchronize(st), "download");
    return FS_OK;
}

extern "C" fs_status fs_get_fields(fs_sim* sim, double* h_par, double* h_perp, int64_t n) {
    return eval_into(sim, h_par, h_perp, nullptr, nullptr, nullptr, n);
}

extern "C" fs_status fs_get_lhs(fs_sim* sim, double* lhs, double* lo, double* hi, int64_t n) {
    return eval_into(sim, nullptr, nullptr, lhs, lo, hi, n);
}

extern "C" fs_status fs_get_hk(const fs_sim* csim, double* out, int64_t n) {
    fs_sim* sim = const_cast<fs_sim*>(csim);
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!out || n != sim->n) return fail(sim, FS_ERR_INVALID, "out must hold n values");
    memcpy(out, sim->hk.data(), 8 * n);
    return FS_OK;
}

extern "C" fs_status fs_get_geometry(const fs_sim* csim, double* x, double* y, double* theta,
                                     int64_t n) {
    fs_sim* sim = const_cast<fs_sim*>(csim);
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    if (n != sim->n) return fail(sim, FS_ERR_INVALID, "outputs must hold n values");
    if (x) memcpy(x, sim->x.data(), 8 * n);
    if (y) memcpy(y, sim->y.data(), 8 * n);
    if (theta) memcpy(theta, sim->theta.data(), 8 * n);
    return FS_OK;
}

extern "C" fs_status fs_get_info(const fs_sim* csim, fs_info* out) {
    fs_sim* sim = const_cast<fs_sim*>(csim);
    if (!sim || !out) return fail(sim, FS_ERR_INVALID, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->n = sim->n;
    if (!sim->built) return FS_OK;
    out->nnz_padded = sim->nnzp;
    out->max_degree = sim->max_deg;
    out->e64 = sim->e64;
    out->e32 = sim->e32;
    out->device_bytes = sim->mem.bytes;
    out->band_rel = std::max(sim->inst.pow_rel_p, sim->inst.pow_rel_q) + sim->inst.div_rel +
                    sim->inst.dh_rel;
    out->band_abs = sim->inst.dh_abs;
    out->col_offsets16 = sim->inst.dcol != nullptr ? 1 : 0;
    // unpadded nnz: count non-self entries
    std::vector<int64_t> rp((size_t)sim->n + 1);
    std::vector<int32_t> col((size_t)sim->nnzp);
    CK(cudaMemcpyAsync(rp.data(), sim->inst.rp, 8 * (sim->n + 1), cudaMemcpyDeviceToHost,
                       sim->stream),
       "download");
    CK(cudaMemcpyAsync(col.data(), sim->inst.col, 4 * sim->nnzp, cudaMemcpyDeviceToHost,
                       sim->stream),
       "download");
    CK(cudaStreamSynchronize(sim->stream), "sync");
    int64_t nnz = 0;
    for (int64_t i = 0; i < sim->n; ++i)
        for (int64_t e = rp[(size_t)i]; e < rp[(size_t)i + 1]; ++e) nnz += col[(size_t)e] != i;
    out->nnz = nnz;
    return FS_OK;
}

extern "C" fs_status fs_get_csr(const fs_sim* csim, int64_t* row_ptr, int32_t* col_out,
                                double* P, double* Q) {
    fs_sim* sim = const_cast<fs_sim*>(csim);
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    const int64_t n = sim->n, nnzp = sim->nnzp;
    std::vector<int64_t> rp((size_t)n + 1);
    std::vector<int32_t> col((size_t)nnzp);
    std::vector<longlong2> pq((size_t)nnzp);
    cudaStream_t st = sim->stream;
    CK(cudaMemcpyAsync(rp.data(), sim->inst.rp, 8 * (n + 1), cudaMemcpyDeviceToHost, st),
       "download");
    CK(cudaMemcpyAsync(col.data(), sim->inst.col, 4 * nnzp, cudaMemcpyDeviceToHost, st),
       "download");
    CK(cudaMemcpyAsync(pq.data(), sim->inst.pq64, 16 * nnzp, cudaMemcpyDeviceToHost, st),
       "download");
    CK(cudaStreamSynchronize(st), "sync");
    const double inv = std::ldexp(1.0, -sim->e64);
    int64_t q = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = rp[(size_t)i]; e < rp[(size_t)i + 1]; ++e) {
            if (col[(size_t)e] == i) continue;
            if (col_out) col_out[q] = col[(size_t)e];
            if (P) P[q] = (double)pq[(size_t)e].x * inv;
            if (Q) Q[q] = (double)pq[(size_t)e].y * inv;
            ++q;
        }
        if (row_ptr) row_ptr[i + 1] = q;
    }
    return FS_OK;
}

extern "C" fs_status fs_set_spins_dev(fs_sim* sim, const int8_t* d_s, int64_t n) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    if (!d_s || n != sim->n) return fail(sim, FS_ERR_INVALID, "spins must have n values");
    CK(cudaMemcpyAsync(sim->inst.s, d_s, n, cudaMemcpyDeviceToDevice, sim->stream), "copy");
    sim->fields_valid = false;
    return FS_OK;
}

extern "C" fs_status fs_set_profiling(fs_sim* sim, int32_t on) {
    if (!sim) return fail(nullptr, FS_ERR_INVALID, "sim is NULL");
    CK(collect_profile(sim), "profile");
    sim->profiling = on != 0;
    sim->prof_sweep_ms = sim->prof_relax_ms = 0.0;
    sim->prof_sweeps = sim->prof_relaxes = 0;
    return FS_OK;
}

extern "C" fs_status fs_get_profile(fs_sim* sim, fs_profile* out) {
    if (!sim || !out) return fail(sim, FS_ERR_INVALID, "NULL argument");
    CK(collect_profile(sim), "profile");
    out->sweep_ms = sim->prof_sweep_ms;
    out->relax_ms = sim->prof_relax_ms;
    out->sweep_launches = sim->prof_sweeps;
    out->relax_launches = sim->prof_relaxes;
    out->rechecks = sim->rechecks;
    out->fallbacks = sim->fallbacks;
    out->rounds = sim->rounds;
    out->idle_rounds = sim->idle_rounds;
    out->round_flips = sim->round_flips;
    out->handoffs = sim->handoffs;
    return FS_OK;
}

// Sweep autotuner: times the sweep with 4, 8, 16 and 32 lanes per CSR row (CUDA
// events, best of three after one warm-up each) at the current spins and field and
// keeps the fastest. Every choice gives bit-identical results (integer sums).
extern "C" fs_status fs_autotune(fs_sim* sim, int32_t* lanes_out) {
    fs_status r = need_built(sim);
    if (r != FS_OK) return r;
    r = check_series(sim, sim->step, 1);
    if (r != FS_OK) return r;
    r = refresh_fields(sim);
    if (r != FS_OK) return r;
    cudaStream_t st = sim->stream;
    double f[2] = {sim->hx, sim->hy};
    CK(cudaMemcpyAsync(sim->d_field, f, 16, cudaMemcpyHostToDevice, st), "upload");
    Inst I = sim->inst;
    I.phx = sim->d_field;
    I.phy = sim->d_field + 1;
    I.K = 1;
    I.step0 = sim->step;
    sim->inst_run = I;
    CK(cudaMemcpyAsync(sim->d_inst, &sim->inst_run, sizeof(Inst), cudaMemcpyHostToDevice, st),
       "upload");
    memset(&sim->state_host, 0, sizeof(InstState));
    CK(cudaMemcpyAsync(sim->d_state, &sim->state_host, sizeof(InstState), cudaMemcpyHostToDevice,
                       st),
       "upload");
    SweepLaunch S;
    S.tab = sim->d_inst;
    S.task_start = sim->d_task_start;
    S.n_inst = 1;
    S.total_tasks = (sim->n + 31) / 32;
    S.tcnts = sim->d_tcnts;
    S.prec = sim->p.precision;
    S.resweep = 1;
    CK(launch_ext_table(S, st), "sweep");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const int cands[5] = {2, 4, 8, 16, 32};
    int best = sim->lanes, best_occ = sim->sweep_occ;
    float best_ms = 1e30f;
    for (int c = 0; c < 10; ++c) {
        S.lanes_per_row = cands[c % 5];
        S.occupancy = c < 5 ? 4 : 5;
        CK(launch_sweep(S, st), "sweep");
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            CK(launch_sweep(S, st), "sweep");
            cudaEventRecord(e1, st);
            CK(cudaEventSynchronize(e1), "sweep");
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cands[c % 5];
            best_occ = S.occupancy;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sim->lanes = best;
    sim->sweep_occ = best_occ;
    if (lanes_out) *lanes_out = best;
    return FS_OK;
}
