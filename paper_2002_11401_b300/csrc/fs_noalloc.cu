// fs_noalloc.cu - a field-and-margin sweep with argmax that allocates nothing.
//
// For callers that cannot allocate device memory at the time of the call (a
// control loop that must not block on the allocator, or a process whose device
// memory is wholly reserved by another framework's pool): the caller passes the
// spins and the output buffers, and the sweep's max-tree lives in one fixed
// static device array of this file instead of a per-call allocation.
//
// The arithmetic is that of the FS_FP64 path: exact 64-bit dipolar sums over the
// simulation's neighbour tensors, the external and thermal fields, Eq. 5 and 6,
// and the flippable island with the largest LHS (lowest index on ties).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/flatspin_b300.h"
#include "fs_common.cuh"
#include "fs_internal.h"

using namespace fs;

namespace {

// Largest system this entry point accepts, and the static scratch that holds its
// max-tree: every tree node (16 B) and an arrival counter (4 B) per node above
// the leaves, for up to kStaticMaxIslands islands (about 1.4 MB, rounded up).
constexpr int64_t kStaticMaxIslands = int64_t(1) << 21;
constexpr size_t kStaticScratchBytes = size_t(2) << 20;

// Every GPU that loads the library holds this array until the process exits.
// Host code must not use its name as a device address; fs_eval_argmax_static
// looks the address up with cudaGetSymbolAddress once per device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

constexpr int kThreads = 256;

__device__ __forceinline__ ulonglong2 best_of(ulonglong2 a, ulonglong2 b) {
    return better64(a.x, a.y, b.x, b.y) ? a : b;
}

__device__ __forceinline__ ulonglong2 warp_best(ulonglong2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ulonglong2 u;
        u.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        u.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = best_of(v, u);
    }
    return v;
}

// One warp per 32 islands: the exact sums of each row (sub-warp of 8 lanes per
// row), then one island per lane: FP64 evaluation, key = LHS when flippable,
// else 0. The warp's best becomes a first-level tree node; the last of 32
// sibling nodes to arrive builds their parent (fenced counter), up to the root,
// whose island index is the result.
__global__ void __launch_bounds__(kThreads)
    k_static_sweep(Inst I, const int8_t* __restrict__ s, double hx, double hy, uint32_t step,
                   double* __restrict__ lhs_out, int64_t* __restrict__ best_out,
                   ulonglong2* __restrict__ tree, unsigned* __restrict__ cnt) {
    constexpr int W = 8;
    __shared__ long long sums[kThreads / 32][32][2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t task = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
    if (task >= I.lvl_n[0]) return;
    const int64_t r0 = task << 5;
    const int sub = lane / W, sl = lane % W;
    for (int q = sub; q < 32; q += 32 / W) {
        const int64_t i = r0 + q;
        long long ap = 0, aq = 0;
        if (i < I.n) {
            for (int64_t e = I.rp[i] + sl; e < I.rp[i + 1]; e += W) {
                const int sj = s[I.col[e]];
                const longlong2 v = I.pq64[e];
                ap += sj > 0 ? v.x : -v.x;
                aq += sj > 0 ? v.y : -v.y;
            }
        }
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            ap += __shfl_xor_sync(0xffffffffu, ap, o);
            aq += __shfl_xor_sync(0xffffffffu, aq, o);
        }
        if (sl == 0) {
            sums[wib][q][0] = ap;
            sums[wib][q][1] = aq;
        }
    }
    __syncwarp();
    const int64_t i = r0 + lane;
    ulonglong2 node = make_ulonglong2(0ull, 0xFFFFFFFFFFFFFFFFull);
    if (i < I.n) {
        double tp = 0.0, tq = 0.0;
        if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
        const uint16_t ci = I.cls[i];
        const Eval64 e = eval64(I, s[i], sums[wib][lane][0], sums[wib][lane][1], I.rbc64[i],
                                ext_proj(hx, hy, I.cs64[ci]), tp, tq);
        const double key = e.flippable ? e.lhs : 0.0;
        lhs_out[i] = key;
        node = make_ulonglong2((unsigned long long)__double_as_longlong(key),
                               (unsigned long long)i);
    }
    node = warp_best(node);
    if (lane == 0) tree[I.lvl_off[0] + task] = node;
    int lev = 0;
    int64_t idx = task;
    while (lev + 1 < I.nlev) {
        const int64_t parent = idx >> 5, first = parent << 5;
        const int64_t last = min((int64_t)I.lvl_n[lev], first + 32);
        __threadfence();
        unsigned old = 0;
        if (lane == 0) old = atomicAdd(&cnt[I.lvl_off[lev + 1] + parent], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old + 1 != (unsigned)(last - first)) return;
        if (lane == 0) cnt[I.lvl_off[lev + 1] + parent] = 0u;
        __threadfence();
        ulonglong2 v = make_ulonglong2(0ull, 0xFFFFFFFFFFFFFFFFull);
        if (first + lane < last) v = __ldcg(&tree[I.lvl_off[lev] + first + lane]);
        v = warp_best(v);
        if (lane == 0) tree[I.lvl_off[lev + 1] + parent] = v;
        ++lev;
        idx = parent;
    }
    // only the warp that completed the root gets here
    if (lane == 0) {
        const ulonglong2 root = tree[I.lvl_off[I.nlev - 1]];
        *best_out = root.x != 0ull ? (int64_t)root.y : -1;
    }
}

}  // namespace

extern "C" fs_status fs_eval_argmax_static(const fs_sim* sim, const int8_t* d_spins, double hx,
                                           double hy, uint32_t step, double* d_lhs,
                                           int64_t* d_best, void* stream) {
    if (!sim || !d_spins || !d_lhs || !d_best) return FS_ERR_INVALID;
    if (!sim->built) return FS_ERR_STATE;
    if (sim->n > kStaticMaxIslands) return FS_ERR_INVALID;
    const Inst& I = sim->inst;
    const int64_t nodes = I.lvl_off[I.nlev - 1] + I.lvl_n[I.nlev - 1];
    const size_t tree_bytes = (size_t)nodes * sizeof(ulonglong2);
    const size_t cnt_bytes = (size_t)nodes * sizeof(unsigned);
    if (tree_bytes + cnt_bytes > kStaticScratchBytes) return FS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FS_ERR_CUDA;
    // the simulation's buffers live on the device it was built on; the scratch
    // address looked up below is that of the current device
    if (dev != sim->device) return FS_ERR_STATE;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_addr[dev]) {
            // one-time set-up on this device, with this device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p)
                return FS_ERR_CUDA;
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    ulonglong2* tree = reinterpret_cast<ulonglong2*>(base);
    unsigned* cnt = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(base) + tree_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's contents: the counters must start at zero
    if (cudaMemsetAsync(cnt, 0, cnt_bytes, st) != cudaSuccess) return FS_ERR_CUDA;
    const unsigned blocks = (unsigned)((I.lvl_n[0] + kThreads / 32 - 1) / (kThreads / 32));
    k_static_sweep<<<blocks, kThreads, 0, st>>>(I, d_spins, hx, hy, step, d_lhs, d_best, tree,
                                                cnt);
    return cudaGetLastError() == cudaSuccess ? FS_OK : FS_ERR_CUDA;
}
