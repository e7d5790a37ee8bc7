// fs_build.h - host-side interface of the device neighbour build.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

struct BuildStats {
    unsigned long long bound_bits;  // max_i sum_j 2 alpha / r_ij^3 (double bits)
    int32_t max_deg;                // max padded degree
    int32_t dcol_over;              // some col[e] - i does not fit 16 bits
};

struct BuildIn {
    int64_t n;
    const double* x;        // device, [n]
    const double* y;        // device, [n]
    const uint16_t* cls;    // device, [n]
    const double2* cs;      // device, per class (cos, sin)
    double rc2;             // (cutoff * a)^2 (1 + 1e-9)
    double alpha;
};

struct BuildWork {
    double xmin, ymin, cell;
    int64_t gx, gy;
    int32_t* cell_of;     // [n]
    int32_t* cell_cnt;    // [gx*gy]
    int32_t* cell_start;  // [gx*gy + 1]
    int32_t* items;       // [n]
    int64_t* tmp64;       // [gx*gy + 1]
    int64_t* tmp64b;      // [gx*gy + 1]
    int64_t* deg_pad;     // [n]
    int64_t* scratch;     // scan block sums
    BuildStats* stats;    // device
};

struct BuildOut {
    double scale64, scale32;  // 2^e64, 2^e32
    int64_t* rp;              // [n+1]
    int32_t* col;             // [nnz_padded]
    longlong2* pq64;
    long long* qt64;
    int2* pq32;
    int* qt32;
};

cudaError_t scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* scratch,
                     cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);
cudaError_t build_cells(const BuildIn& in, BuildWork& w, cudaStream_t st);
cudaError_t build_degrees(const BuildIn& in, BuildWork& w, cudaStream_t st);
cudaError_t build_rows(const BuildIn& in, BuildWork& w, int64_t* rp, cudaStream_t st);
cudaError_t build_fill(const BuildIn& in, BuildWork& w, const BuildOut& o, cudaStream_t st);
// dcol[e] = col[e] - i for every entry e of row i; sets *over when one does not fit
// 16 bits (those entries are then left truncated and dcol is not to be used).
cudaError_t build_dcol(int64_t n, const int64_t* rp, const int32_t* col, int16_t* dcol,
                       int32_t* over, cudaStream_t st);

}  // namespace fs
