// fs_build.cu - neighbour tensors on the device (Sec. "Magnetic dipole-dipole
// interactions"): a uniform cell grid no finer than the cutoff, per-island
// degree counts, an exclusive scan into padded CSR row pointers, and a fill pass
// that sorts each row by neighbour index and stores the per-pair coefficients
//   P_ij = mhat_i . T_ij mhat_j,  Q_ij = mhat_perp_i . T_ij mhat_j,
//   T_ij = alpha (3 rhat rhat^T - I) / |r_ij|^3,  r_ij = r_i - r_j        (Eq. 3)
// together with the transposed Q_ji, in 64-bit and 32-bit fixed point.
//
// The field on island i is sum_j s_j (P_ij, Q_ij) in i's frame. P_ij = P_ji
// holds bit for bit: T depends on r only through rx^2, ry^2, rx*ry and r^2, and
// every product is formed in an order that does not depend on which island is
// the row, with no contraction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_build.h"
#include "fs_common.cuh"

namespace fs {

namespace {

__device__ __forceinline__ double sq_dist(double xi, double yi, double xj, double yj) {
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

struct Tensor {
    double xx, xy, yy;
};

// T_ij of Eq. 3 (alpha included); symmetric under r -> -r bit for bit.
__device__ __forceinline__ Tensor dipole_tensor(double rx, double ry, double alpha) {
    const double rxrx = __dmul_rn(rx, rx), ryry = __dmul_rn(ry, ry), rxry = __dmul_rn(rx, ry);
    const double r2 = __dadd_rn(rxrx, ryry);
    const double r = __dsqrt_rn(r2);
    const double a = __ddiv_rn(alpha, __dmul_rn(r2, r));
    Tensor T;
    T.xx = __dmul_rn(a, __dsub_rn(__ddiv_rn(__dmul_rn(3.0, rxrx), r2), 1.0));
    T.xy = __dmul_rn(a, __ddiv_rn(__dmul_rn(3.0, rxry), r2));
    T.yy = __dmul_rn(a, __dsub_rn(__ddiv_rn(__dmul_rn(3.0, ryry), r2), 1.0));
    return T;
}

// mhat_a . T mhat_b; symmetric in (a, b).
__device__ __forceinline__ double p_coeff(const Tensor& T, double ca, double sa, double cb,
                                          double sb) {
    const double cc = __dmul_rn(ca, cb), ss = __dmul_rn(sa, sb);
    const double mix = __dadd_rn(__dmul_rn(ca, sb), __dmul_rn(sa, cb));
    return __dadd_rn(__dadd_rn(__dmul_rn(T.xx, cc), __dmul_rn(T.xy, mix)), __dmul_rn(T.yy, ss));
}

// mhat_perp_a . T mhat_b with mhat_perp_a = (-sa, ca).
__device__ __forceinline__ double q_coeff(const Tensor& T, double ca, double sa, double cb,
                                          double sb) {
    const double t1 = __dmul_rn(T.xx, -__dmul_rn(sa, cb));
    const double t2 = __dmul_rn(T.xy, __dsub_rn(__dmul_rn(ca, cb), __dmul_rn(sa, sb)));
    const double t3 = __dmul_rn(T.yy, __dmul_rn(ca, sb));
    return __dadd_rn(__dadd_rn(t1, t2), t3);
}

__global__ void k_cell_count(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                             double xmin, double ymin, double inv_cell, int64_t gx, int64_t gy,
                             int32_t* __restrict__ cell_of, int32_t* __restrict__ cell_cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t cx = (int64_t)floor((x[i] - xmin) * inv_cell);
    int64_t cy = (int64_t)floor((y[i] - ymin) * inv_cell);
    cx = cx < 0 ? 0 : (cx >= gx ? gx - 1 : cx);
    cy = cy < 0 ? 0 : (cy >= gy ? gy - 1 : cy);
    const int32_t c = (int32_t)(cy * gx + cx);
    cell_of[i] = c;
    atomicAdd(&cell_cnt[c], 1);
}

__global__ void k_cell_fill(int64_t n, const int32_t* __restrict__ cell_of,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ items) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t pos = atomicAdd(&cursor[cell_of[i]], 1);
    items[pos] = (int32_t)i;
}

// One warp per island: neighbours within the inclusive cutoff, and the bound
// sum_j 2 alpha / r^3 on |sum_j s_j P_ij| and |sum_j s_j Q_ij|.
__global__ void k_degree(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                         const int32_t* __restrict__ cell_of, const int32_t* __restrict__ cell_start,
                         const int32_t* __restrict__ items, int64_t gx, int64_t gy, double rc2,
                         double alpha, int64_t* __restrict__ deg_pad,
                         unsigned long long* __restrict__ bound_bits, int32_t* __restrict__ max_deg) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const double xi = x[i], yi = y[i];
    const int32_t c = cell_of[i];
    const int64_t cx = c % gx, cy = c / gx;
    int cnt = 0;
    double bsum = 0.0;
    for (int64_t dy = -1; dy <= 1; ++dy) {
        const int64_t uy = cy + dy;
        if (uy < 0 || uy >= gy) continue;
        for (int64_t dx = -1; dx <= 1; ++dx) {
            const int64_t ux = cx + dx;
            if (ux < 0 || ux >= gx) continue;
            const int32_t cc = (int32_t)(uy * gx + ux);
            for (int32_t q = cell_start[cc] + lane; q < cell_start[cc + 1]; q += 32) {
                const int32_t j = items[q];
                if (j == i) continue;
                const double d2 = sq_dist(xi, yi, x[j], y[j]);
                if (d2 <= rc2) {
                    ++cnt;
                    bsum += 2.0 * alpha / (d2 * sqrt(d2));
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        bsum += __shfl_xor_sync(0xffffffffu, bsum, o);
    }
    if (lane == 0) {
        const int64_t dp = ((int64_t)cnt + kRowPad - 1) / kRowPad * kRowPad;
        deg_pad[i] = dp;
        atomicMax(max_deg, (int32_t)dp);
        atomicMax(bound_bits, (unsigned long long)__double_as_longlong(bsum));
    }
}

constexpr int kFillWarps = 4;

// One warp per island: gather the neighbours, place each at its rank among the
// row's indices (rows ascending in j), and store the coefficients.
__global__ void __launch_bounds__(kFillWarps * 32)
    k_fill(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
           const uint16_t* __restrict__ cls, const double2* __restrict__ cs,
           const int32_t* __restrict__ cell_of, const int32_t* __restrict__ cell_start,
           const int32_t* __restrict__ items, int64_t gx, int64_t gy, double rc2, double alpha,
           double scale64, double scale32, const int64_t* __restrict__ rp,
           int32_t* __restrict__ col, longlong2* __restrict__ pq64, long long* __restrict__ qt64,
           int2* __restrict__ pq32, int* __restrict__ qt32) {
    __shared__ int32_t buf[kFillWarps][kMaxPaddedDegree];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const double xi = x[i], yi = y[i];
    const int32_t c = cell_of[i];
    const int64_t cx = c % gx, cy = c / gx;
    int cnt = 0;
    for (int64_t dy = -1; dy <= 1; ++dy) {
        const int64_t uy = cy + dy;
        if (uy < 0 || uy >= gy) continue;
        for (int64_t dx = -1; dx <= 1; ++dx) {
            const int64_t ux = cx + dx;
            if (ux < 0 || ux >= gx) continue;
            const int32_t cc = (int32_t)(uy * gx + ux);
            const int32_t q0 = cell_start[cc], q1 = cell_start[cc + 1];
            for (int32_t base = q0; base < q1; base += 32) {
                const int32_t q = base + lane;
                bool hit = false;
                int32_t j = -1;
                if (q < q1) {
                    j = items[q];
                    hit = (j != i) && sq_dist(xi, yi, x[j], y[j]) <= rc2;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) {
                    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (pos < kMaxPaddedDegree) buf[w][pos] = j;
                }
                cnt += __popc(m);
            }
        }
    }
    __syncwarp();
    const int64_t e0 = rp[i];
    const int64_t dp = rp[i + 1] - e0;
    if (cnt > kMaxPaddedDegree) cnt = kMaxPaddedDegree;  // unreachable: degree checked on host
    const uint16_t ci_cls = cls[i];
    const double ci = cs[ci_cls].x, si = cs[ci_cls].y;
    for (int q = lane; q < cnt; q += 32) {
        const int32_t j = buf[w][q];
        int rank = 0;
        for (int u = 0; u < cnt; ++u) rank += buf[w][u] < j;
        const double2 mj = cs[cls[j]];
        const Tensor T = dipole_tensor(__dsub_rn(xi, x[j]), __dsub_rn(yi, y[j]), alpha);
        const double P = p_coeff(T, ci, si, mj.x, mj.y);
        const double Qij = q_coeff(T, ci, si, mj.x, mj.y);
        const double Qji = q_coeff(T, mj.x, mj.y, ci, si);
        const int64_t e = e0 + rank;
        col[e] = j;
        pq64[e] = make_longlong2(__double2ll_rn(__dmul_rn(P, scale64)),
                                 __double2ll_rn(__dmul_rn(Qij, scale64)));
        qt64[e] = __double2ll_rn(__dmul_rn(Qji, scale64));
        pq32[e] = make_int2(__double2int_rn(__dmul_rn(P, scale32)),
                            __double2int_rn(__dmul_rn(Qij, scale32)));
        qt32[e] = __double2int_rn(__dmul_rn(Qji, scale32));
    }
    for (int64_t q = cnt + lane; q < dp; q += 32) {
        const int64_t e = e0 + q;
        col[e] = (int32_t)i;  // zero-weight self entry (row padding)
        pq64[e] = make_longlong2(0, 0);
        qt64[e] = 0;
        pq32[e] = make_int2(0, 0);
        qt32[e] = 0;
    }
}

// ---- exclusive scan of int64 (three phases) ----------------------------------

constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += t;
        }
        warp_sums[lane] = ws;
    }
    __syncthreads();
    const int64_t before = (w > 0 ? warp_sums[w - 1] : 0) + incl - v;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanBlock)
    k_scan_local(int64_t n, const int64_t* __restrict__ in, int64_t* __restrict__ out,
                 int64_t* __restrict__ block_sums) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const int64_t v = i < n ? in[i] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(v, &total);
    if (i < n) out[i] = ex;
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums, chunk by chunk.
__global__ void __launch_bounds__(kScanBlock)
    k_scan_sums(int64_t nb, int64_t* __restrict__ sums, int64_t* __restrict__ grand) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exclusive_scan(v, &total);
        if (i < nb) sums[i] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ sums) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < n) out[i] += sums[blockIdx.x];
}

__global__ void k_scan_i32_to_i32(int64_t n, const int32_t* __restrict__ cnt,
                                  int64_t* __restrict__ tmp) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) tmp[i] = cnt[i];
}

__global__ void k_i64_to_i32(int64_t n, const int64_t* __restrict__ in, int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

}  // namespace

// Exclusive scan of in[0..n) into out[0..n], out[n] = total. Scratch: block sums.
cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch,
                     cudaStream_t st) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    k_scan_local<<<(unsigned)nb, kScanBlock, 0, st>>>(n, in, out, scratch);
    k_scan_sums<<<1, kScanBlock, 0, st>>>(nb, scratch, out + n);
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(n, out, scratch);
    return cudaGetLastError();
}

int64_t scan_scratch_elems(int64_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

cudaError_t build_cells(const BuildIn& in, BuildWork& w, cudaStream_t st) {
    cudaError_t e;
    const int64_t n = in.n;
    const int64_t ncell = w.gx * w.gy;
    if ((e = cudaMemsetAsync(w.cell_cnt, 0, sizeof(int32_t) * ncell, st)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_cell_count<<<nb, 256, 0, st>>>(n, in.x, in.y, w.xmin, w.ymin, 1.0 / w.cell, w.gx, w.gy,
                                     w.cell_of, w.cell_cnt);
    const unsigned cb = (unsigned)((ncell + 255) / 256);
    k_scan_i32_to_i32<<<cb, 256, 0, st>>>(ncell, w.cell_cnt, w.tmp64);
    if ((e = scan_i64(w.tmp64, w.tmp64b, ncell, w.scratch, st)) != cudaSuccess) return e;
    k_i64_to_i32<<<(unsigned)((ncell + 1 + 255) / 256), 256, 0, st>>>(ncell + 1, w.tmp64b,
                                                                      w.cell_start);
    if ((e = cudaMemcpyAsync(w.cell_cnt, w.cell_start, sizeof(int32_t) * ncell,
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    k_cell_fill<<<nb, 256, 0, st>>>(n, w.cell_of, w.cell_cnt, w.items);
    return cudaGetLastError();
}

cudaError_t build_degrees(const BuildIn& in, BuildWork& w, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(w.stats, 0, sizeof(BuildStats), st)) != cudaSuccess) return e;
    const int64_t threads = in.n * 32;
    k_degree<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        in.n, in.x, in.y, w.cell_of, w.cell_start, w.items, w.gx, w.gy, in.rc2, in.alpha,
        w.deg_pad, &w.stats->bound_bits, &w.stats->max_deg);
    return cudaGetLastError();
}

cudaError_t build_rows(const BuildIn& in, BuildWork& w, int64_t* rp, cudaStream_t st) {
    return scan_i64(w.deg_pad, rp, in.n, w.scratch, st);
}

cudaError_t build_fill(const BuildIn& in, BuildWork& w, const BuildOut& o, cudaStream_t st) {
    const int64_t threads = in.n * 32;
    k_fill<<<(unsigned)((threads + kFillWarps * 32 - 1) / (kFillWarps * 32)), kFillWarps * 32, 0,
             st>>>(in.n, in.x, in.y, in.cls, in.cs, w.cell_of, w.cell_start, w.items, w.gx, w.gy,
                   in.rc2, in.alpha, o.scale64, o.scale32, o.rp, o.col, o.pq64, o.qt64, o.pq32,
                   o.qt32);
    return cudaGetLastError();
}

// One warp per row: the row's column offsets from its own island, 16 bits each.
__global__ void k_dcol(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                       int16_t* __restrict__ dcol, int32_t* __restrict__ over) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    bool bad = false;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
        const int64_t d = (int64_t)col[e] - i;
        bad = bad || d < -32768 || d > 32767;
        dcol[e] = (int16_t)d;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(over, 1);
}

cudaError_t build_dcol(int64_t n, const int64_t* rp, const int32_t* col, int16_t* dcol,
                       int32_t* over, cudaStream_t st) {
    const int64_t threads = n * 32;
    k_dcol<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rp, col, dcol, over);
    return cudaGetLastError();
}

}  // namespace fs
