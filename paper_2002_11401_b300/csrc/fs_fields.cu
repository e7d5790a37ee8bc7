// fs_fields.cu - external fields beyond the global one and thermal protocols
// (Sec. "External field", Sec. "Thermal field"), the input encoders (Sec.
// "Simulation framework"), and the spin-spin correlation against separation
// (Sec. "Domain size in square ASI").
//
// Local and spatial fields are kept on the device as series indexed by the field
// step (the index that also keys the thermal draw); the sweep adds the island's
// entry to the global field of the step, projects the sum on the island's frame
// and keeps it for the relax (fs_common.cuh: ext_lab, ext64_at, ext32_at).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/flatspin_b300.h"
#include "fs_common.cuh"
#include "fs_internal.h"

using namespace fs;

namespace {

fs_status ffail(fs_sim* sim, fs_status code, const std::string& msg) {
    if (sim) sim->err = msg;
    return code;
}

fs_status need_params(fs_sim* sim) {
    if (!sim) return FS_ERR_INVALID;
    if (!sim->built) return ffail(sim, FS_ERR_STATE, "parameters not set");
    return FS_OK;
}

bool all_finite(const double* v, int64_t m) {
    for (int64_t q = 0; q < m; ++q)
        if (!std::isfinite(v[q])) return false;
    return true;
}

// Drops the local or spatial field (the relax goes back to the per-class table).
void clear_ext(fs_sim* sim) {
    sim->ext_mem.release(sim->stream);
    Inst& I = sim->inst;
    I.lx = I.ly = I.gx = I.gy = nullptr;
    I.gcell = nullptr;
    I.exti64 = nullptr;
    I.exti32 = nullptr;
    I.ext_K = 0;
    I.grid_G = 0;
}

// Allocates and uploads `count` doubles of each component.
fs_status upload_pair(fs_sim* sim, const double* a, const double* b, int64_t count, double** da,
                      double** db) {
    cudaStream_t st = sim->stream;
    if (sim->ext_mem.alloc((void**)da, 8 * (size_t)count, st) != cudaSuccess ||
        sim->ext_mem.alloc((void**)db, 8 * (size_t)count, st) != cudaSuccess)
        return ffail(sim, FS_ERR_OOM, "out of device memory for the field series");
    if (cudaMemcpyAsync(*da, a, 8 * (size_t)count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(*db, b, 8 * (size_t)count, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ffail(sim, FS_ERR_CUDA, "upload of the field series failed");
    return FS_OK;
}

fs_status alloc_projections(fs_sim* sim) {
    Inst& I = sim->inst;
    if (sim->ext_mem.alloc((void**)&I.exti64, 16 * (size_t)sim->n, sim->stream) != cudaSuccess ||
        sim->ext_mem.alloc((void**)&I.exti32, 8 * (size_t)sim->n, sim->stream) != cudaSuccess)
        return ffail(sim, FS_ERR_OOM, "out of device memory for the per-island fields");
    return FS_OK;
}

}  // namespace

extern "C" fs_status fs_set_field_local(fs_sim* sim, const double* hx, const double* hy,
                                        int64_t K, int64_t n) {
    fs_status r = need_params(sim);
    if (r != FS_OK) return r;
    if (K < 0 || (K > 0 && (!hx || !hy)) || (K > 0 && n != sim->n))
        return ffail(sim, FS_ERR_INVALID, "local field: K x n values per component");
    if (K > 0 && (!all_finite(hx, K * n) || !all_finite(hy, K * n)))
        return ffail(sim, FS_ERR_INVALID, "local field: non-finite value");
    clear_ext(sim);
    if (K == 0) return FS_OK;
    Inst& I = sim->inst;
    double *dx = nullptr, *dy = nullptr;
    r = upload_pair(sim, hx, hy, K * n, &dx, &dy);
    if (r == FS_OK) r = alloc_projections(sim);
    if (r != FS_OK) {
        cudaStreamSynchronize(sim->stream);
        clear_ext(sim);
        return r;
    }
    I.lx = dx;
    I.ly = dy;
    I.ext_K = K;
    if (cudaStreamSynchronize(sim->stream) != cudaSuccess)
        return ffail(sim, FS_ERR_CUDA, "local field: upload failed");
    return FS_OK;
}

extern "C" fs_status fs_set_field_spatial(fs_sim* sim, const double* hx, const double* hy,
                                          int64_t K, int32_t gw, int32_t gh, double x0,
                                          double y0, double dx, double dy) {
    fs_status r = need_params(sim);
    if (r != FS_OK) return r;
    if (K < 0 || (K > 0 && (!hx || !hy || gw <= 0 || gh <= 0 || !(dx > 0.0) || !(dy > 0.0) ||
                            !std::isfinite(x0) || !std::isfinite(y0) || !std::isfinite(dx) ||
                            !std::isfinite(dy))))
        return ffail(sim, FS_ERR_INVALID, "spatial field: bad grid or series");
    const int64_t G = (int64_t)gw * gh;
    if (K > 0 && (G > (int64_t)1 << 30 || !all_finite(hx, K * G) || !all_finite(hy, K * G)))
        return ffail(sim, FS_ERR_INVALID, "spatial field: grid too large or non-finite value");
    clear_ext(sim);
    if (K == 0) return FS_OK;
    // the cell of each island centre, clamped to the grid
    std::vector<int32_t> cell((size_t)sim->n);
    for (int64_t i = 0; i < sim->n; ++i) {
        int64_t cx = (int64_t)std::floor((sim->x[(size_t)i] - x0) / dx);
        int64_t cy = (int64_t)std::floor((sim->y[(size_t)i] - y0) / dy);
        cx = std::min<int64_t>(std::max<int64_t>(cx, 0), gw - 1);
        cy = std::min<int64_t>(std::max<int64_t>(cy, 0), gh - 1);
        cell[(size_t)i] = (int32_t)(cy * gw + cx);
    }
    Inst& I = sim->inst;
    double *gxd = nullptr, *gyd = nullptr;
    int32_t* dcell = nullptr;
    r = upload_pair(sim, hx, hy, K * G, &gxd, &gyd);
    if (r == FS_OK) {
        if (sim->ext_mem.alloc((void**)&dcell, 4 * (size_t)sim->n, sim->stream) != cudaSuccess)
            r = ffail(sim, FS_ERR_OOM, "out of device memory for the cell map");
        else if (cudaMemcpyAsync(dcell, cell.data(), 4 * (size_t)sim->n, cudaMemcpyHostToDevice,
                                 sim->stream) != cudaSuccess)
            r = ffail(sim, FS_ERR_CUDA, "upload of the cell map failed");
    }
    if (r == FS_OK) r = alloc_projections(sim);
    // (the host vector must outlive the copy)
    const cudaError_t e = cudaStreamSynchronize(sim->stream);
    if (r == FS_OK && e != cudaSuccess) r = ffail(sim, FS_ERR_CUDA, "spatial field: upload failed");
    if (r != FS_OK) {
        clear_ext(sim);
        return r;
    }
    I.gx = gxd;
    I.gy = gyd;
    I.gcell = dcell;
    I.grid_G = G;
    I.ext_K = K;
    return FS_OK;
}

extern "C" fs_status fs_set_sigma_series(fs_sim* sim, const double* sigma, int64_t K) {
    fs_status r = need_params(sim);
    if (r != FS_OK) return r;
    if (K < 0 || (K > 0 && !sigma)) return ffail(sim, FS_ERR_INVALID, "thermal series: bad arguments");
    if (K > 0 && !(sim->p.sigma_th > 0.0))
        return ffail(sim, FS_ERR_STATE,
                     "thermal series: set parameters with sigma_th > 0 first (thermal buffers)");
    for (int64_t q = 0; q < K; ++q)
        if (!std::isfinite(sigma[q]) || sigma[q] < 0.0)
            return ffail(sim, FS_ERR_INVALID, "thermal series: values must be finite and >= 0");
    cudaStream_t st = sim->stream;
    sim->sig_mem.release(st);
    Inst& I = sim->inst;
    I.sig = nullptr;
    I.sig_K = 0;
    // FP64 draws kept for a step were drawn with that step's old deviation
    if (I.th_step && cudaMemsetAsync(I.th_step, 0xFF, 4 * (size_t)sim->n, st) != cudaSuccess)
        return ffail(sim, FS_ERR_CUDA, "thermal series: reset of the kept draws failed");
    if (K > 0) {
        double* d = nullptr;
        if (sim->sig_mem.alloc((void**)&d, 8 * (size_t)K, st) != cudaSuccess)
            return ffail(sim, FS_ERR_OOM, "out of device memory for the thermal series");
        if (cudaMemcpyAsync(d, sigma, 8 * (size_t)K, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return ffail(sim, FS_ERR_CUDA, "upload of the thermal series failed");
        I.sig = d;
        I.sig_K = K;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return ffail(sim, FS_ERR_CUDA, "thermal series: upload failed");
    return FS_OK;
}

// ---------------------------------------------------------------------------
// Input encoders
// ---------------------------------------------------------------------------

extern "C" fs_status fs_encode(int32_t kind, const double* inputs, int64_t m, int32_t period,
                               double h_lo, double h_hi, double angle_deg, double* hx,
                               double* hy) {
    if (m < 0 || period < 1 || (m > 0 && (!inputs || !hx || !hy)) ||
        (kind != FS_ENCODE_SINUSOID && kind != FS_ENCODE_SAWTOOTH &&
         kind != FS_ENCODE_ROTATION) ||
        (kind == FS_ENCODE_SAWTOOTH && period < 2))
        return FS_ERR_INVALID;
    const double dir = (angle_deg * M_PI) / 180.0;
    const double cd = std::cos(dir), sd = std::sin(dir);
    for (int64_t k = 0; k < m; ++k) {
        const double amp = h_lo + (h_hi - h_lo) * inputs[k];
        double* ox = hx + k * period;
        double* oy = hy + k * period;
        for (int32_t j = 0; j < period; ++j) {
            if (kind == FS_ENCODE_ROTATION) {
                const double a = ((angle_deg + (360.0 * (double)j) / (double)period) * M_PI) / 180.0;
                ox[j] = amp * std::cos(a);
                oy[j] = amp * std::sin(a);
                continue;
            }
            const double h = kind == FS_ENCODE_SINUSOID
                                 ? amp * std::sin((2.0 * M_PI * (double)j) / (double)period)
                                 : amp * ((2.0 * (double)j) / (double)(period - 1) - 1.0);
            ox[j] = h * cd;
            oy[j] = h * sd;
        }
    }
    return FS_OK;
}

// ---------------------------------------------------------------------------
// Spin-spin correlation against separation
// ---------------------------------------------------------------------------

namespace {

constexpr int kCorrThreads = 256;
constexpr int kCorrMaxBins = 2048;

// One thread per island i (islands in cell order): every island j > i in the 3 x 3
// cells around i's (cells no smaller than rmax) within rmax goes to its separation
// bin with the sign of s_i s_j v_ij, v_ij = 3 (mhat_i . rhat)(mhat_j . rhat) -
// mhat_i . mhat_j (the sign that makes the pair's dipolar energy, Eq. 3, negative).
// Every floating-point step is an explicit IEEE operation in a fixed order, so a
// pair's bin and sign are the same wherever they are evaluated in double. Bins are
// summed in shared memory per block, then into global memory.
__global__ void __launch_bounds__(kCorrThreads)
    k_correlation(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                  const int8_t* __restrict__ s, const uint16_t* __restrict__ cls,
                  const double2* __restrict__ cs, const int32_t* __restrict__ items,
                  const int32_t* __restrict__ cell_of, const int64_t* __restrict__ cstart,
                  int64_t gx, int64_t gy, double r2max, double w, int nbins,
                  unsigned long long* __restrict__ count, unsigned long long* __restrict__ sum) {
    __shared__ unsigned long long hc[kCorrMaxBins];
    __shared__ unsigned long long hs[kCorrMaxBins];
    for (int b = threadIdx.x; b < nbins; b += kCorrThreads) {
        hc[b] = 0ull;
        hs[b] = 0ull;
    }
    __syncthreads();
    const int64_t q = blockIdx.x * (int64_t)kCorrThreads + threadIdx.x;
    if (q < n) {
        const int64_t i = items[q];
        const double xi = x[i], yi = y[i];
        const double2 mi = cs[cls[i]];
        const int si = s[i];
        const int64_t c = cell_of[i];
        const int64_t cx = c % gx, cy = c / gx;
        for (int64_t uy = max(cy - 1, (int64_t)0); uy <= min(cy + 1, gy - 1); ++uy) {
            for (int64_t ux = max(cx - 1, (int64_t)0); ux <= min(cx + 1, gx - 1); ++ux) {
                const int64_t cc = uy * gx + ux;
                for (int64_t e = cstart[cc]; e < cstart[cc + 1]; ++e) {
                    const int64_t j = items[e];
                    if (j <= i) continue;
                    const double rx = __dsub_rn(xi, x[j]), ry = __dsub_rn(yi, y[j]);
                    const double r2 = __dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry));
                    if (r2 > r2max) continue;
                    const double r = __dsqrt_rn(r2);
                    const int64_t b = (int64_t)floor(__dadd_rn(__ddiv_rn(r, w), 1e-7));
                    if (b >= nbins) continue;
                    const double2 mj = cs[cls[j]];
                    const double ui = __ddiv_rn(__dadd_rn(__dmul_rn(mi.x, rx), __dmul_rn(mi.y, ry)), r);
                    const double uj = __ddiv_rn(__dadd_rn(__dmul_rn(mj.x, rx), __dmul_rn(mj.y, ry)), r);
                    const double v = __dsub_rn(__dmul_rn(__dmul_rn(3.0, ui), uj),
                                               __dadd_rn(__dmul_rn(mi.x, mj.x), __dmul_rn(mi.y, mj.y)));
                    if (fabs(v) <= 1e-9) continue;
                    const long long sv = (v > 0.0 ? 1 : -1) * si * (int)s[j];
                    atomicAdd(&hc[b], 1ull);
                    atomicAdd(&hs[b], (unsigned long long)sv);
                }
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kCorrThreads) {
        if (hc[b]) {
            atomicAdd(&count[b], hc[b]);
            atomicAdd(&sum[b], hs[b]);
        }
    }
}

struct DevFree {
    std::vector<void*> p;
    cudaStream_t st;
    ~DevFree() {
        for (void* q : p) cudaFreeAsync(q, st);
        cudaStreamSynchronize(st);
    }
};

}  // namespace

extern "C" fs_status fs_correlation(fs_sim* sim, double rmax, double bin_width, int32_t nbins,
                                    int64_t* pair_count, int64_t* corr_sum) {
    fs_status r = need_params(sim);
    if (r != FS_OK) return r;
    if (!(rmax > 0.0) || !std::isfinite(rmax) || !(bin_width > 0.0) || !std::isfinite(bin_width) ||
        nbins < 1 || nbins > kCorrMaxBins || !pair_count || !corr_sum)
        return ffail(sim, FS_ERR_INVALID, "correlation: bad arguments (1 <= nbins <= 2048)");
    const int64_t n = sim->n;
    double xmin = sim->x[0], xmax = xmin, ymin = sim->y[0], ymax = ymin;
    for (int64_t i = 1; i < n; ++i) {
        xmin = std::min(xmin, sim->x[(size_t)i]);
        xmax = std::max(xmax, sim->x[(size_t)i]);
        ymin = std::min(ymin, sim->y[(size_t)i]);
        ymax = std::max(ymax, sim->y[(size_t)i]);
    }
    const double cell = rmax * 1.0001;
    const int64_t gx = (int64_t)std::floor((xmax - xmin) / cell) + 1;
    const int64_t gy = (int64_t)std::floor((ymax - ymin) / cell) + 1;
    if (gx * gy > ((int64_t)1 << 26))
        return ffail(sim, FS_ERR_INVALID, "correlation: rmax too small for the array's extent");
    // counting sort of the islands by cell (ascending index within a cell)
    std::vector<int32_t> cell_of((size_t)n), items((size_t)n);
    std::vector<int64_t> cstart((size_t)(gx * gy + 1), 0);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t cx = std::min<int64_t>((int64_t)std::floor((sim->x[(size_t)i] - xmin) / cell), gx - 1);
        const int64_t cy = std::min<int64_t>((int64_t)std::floor((sim->y[(size_t)i] - ymin) / cell), gy - 1);
        cell_of[(size_t)i] = (int32_t)(cy * gx + cx);
        ++cstart[(size_t)(cy * gx + cx) + 1];
    }
    for (int64_t c = 0; c < gx * gy; ++c) cstart[(size_t)c + 1] += cstart[(size_t)c];
    {
        std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t i = 0; i < n; ++i) items[(size_t)fill[(size_t)cell_of[(size_t)i]]++] = (int32_t)i;
    }
    cudaStream_t st = sim->stream;
    DevFree tmp{{}, st};
    auto dalloc = [&](void** q, size_t b) {
        const cudaError_t e = cudaMallocAsync(q, b ? b : 16, st);
        if (e == cudaSuccess) tmp.p.push_back(*q);
        return e;
    };
    double *dx = nullptr, *dy = nullptr;
    int32_t *ditems = nullptr, *dcell = nullptr;
    int64_t* dstart = nullptr;
    unsigned long long *dcount = nullptr, *dsum = nullptr;
    if (dalloc((void**)&dx, 8 * (size_t)n) || dalloc((void**)&dy, 8 * (size_t)n) ||
        dalloc((void**)&ditems, 4 * (size_t)n) || dalloc((void**)&dcell, 4 * (size_t)n) ||
        dalloc((void**)&dstart, 8 * cstart.size()) || dalloc((void**)&dcount, 8 * (size_t)nbins) ||
        dalloc((void**)&dsum, 8 * (size_t)nbins))
        return ffail(sim, FS_ERR_OOM, "correlation: out of device memory");
    if (cudaMemcpyAsync(dx, sim->x.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(dy, sim->y.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(ditems, items.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(dcell, cell_of.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, st) ||
        cudaMemcpyAsync(dstart, cstart.data(), 8 * cstart.size(), cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(dcount, 0, 8 * (size_t)nbins, st) ||
        cudaMemsetAsync(dsum, 0, 8 * (size_t)nbins, st))
        return ffail(sim, FS_ERR_CUDA, "correlation: upload failed");
    const double r2max = rmax * rmax * (1.0 + 1e-9);
    const unsigned blocks = (unsigned)((n + kCorrThreads - 1) / kCorrThreads);
    k_correlation<<<blocks, kCorrThreads, 0, st>>>(n, dx, dy, sim->inst.s, sim->inst.cls,
                                                   sim->inst.cs64, ditems, dcell, dstart, gx, gy,
                                                   r2max, bin_width, nbins, dcount, dsum);
    if (cudaGetLastError() != cudaSuccess)
        return ffail(sim, FS_ERR_CUDA, "correlation: launch failed");
    if (cudaMemcpyAsync(pair_count, dcount, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, st) ||
        cudaMemcpyAsync(corr_sum, dsum, 8 * (size_t)nbins, cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return ffail(sim, FS_ERR_CUDA, "correlation: kernel or download failed");
    return FS_OK;
}
