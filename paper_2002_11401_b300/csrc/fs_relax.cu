// fs_relax.cu - the greedy single-flip relaxation (Sec. "Dynamics"), one CTA per
// simulation, entirely on the device.
//
// Keys: one 64-bit key per island, (FP32 upper bound of its Eq. 5 LHS) << 32 |
// (2^32 - 1 - index), 0 when the island cannot be flippable; a max-tree of fan-out
// 32 over the keys up to the first level of at most 256 nodes (the top), its upper
// levels in shared memory. The root is not stored: warp 0 reduces the top level
// when it picks. The largest key is the island with the largest bound, lowest
// index first.
//
// Per flip, two phases and two barriers:
//  - Warp 0 repairs the tree (nodes whose maximum was a key that shrank are
//    rebuilt from their children, level by level), reads the root's island w and
//    the largest other key (w's sibling sets at every level), and takes w when its
//    certified lower bound exceeds one and that runner-up's upper bound; otherwise
//    the islands whose bounds reach the threshold are compared exactly (FS_FP64
//    values) and the exact best is taken. It flips the pick k.
//  - Meanwhile warps 1..7 compute the neighbour updates of the predicted pick
//    (loads and arithmetic only): every neighbour i of it (its CSR row, whose
//    transposed coefficients give the field it puts on i in i's frame) gets
//    2 s(new) (P, Q) added to its exact fixed-point sums and a new key.
//  - After the barrier the precomputed updates are committed when k is the
//    predicted island and no key changed on the way; otherwise k's updates are
//    computed and committed now. A key that grows is pushed up the tree with
//    atomic maxima; one that shrank queues its node for the next repair. The
//    prediction for the next flip is the largest of the untouched runner-up and
//    the neighbours' new keys.
// Fields are held constant over the relax, as the paper states.
//
// FS_FP32_RECHECK computes keys from FP32 bounds and its exact values in FP64;
// FS_FP64 computes every candidate's exact value when its key is set, and its keys
// are that value rounded out to FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "fs_common.cuh"
#include "fs_kernels.h"
#include "fs_sweep_task.cuh"
#include "fs_update.cuh"

namespace fs {

namespace {

constexpr int kT = 256;  // threads per relax CTA
constexpr int kNW = kT / 32;
constexpr int kDirtyCap = kMaxPaddedDegree + 8;
// Thread that folds each flip into the sequence hash, during the commit phase (off
// warp 0's chain; it holds no update unless a row has kT - 34 entries).
constexpr int kHashThread = kT - 2;
// Levels the relax keeps: fewer than 2^31 islands need at most five (the fifth
// has at most 64 nodes).
constexpr int kRelaxLevels = 5;
constexpr int kTopPerLane = kRelaxTopNodes / 32;

// The tree's levels above the leaves. Held in registers: every access goes through
// lp()/ln(), which select with compile-time indices (a run-time index into these
// arrays would put them in local memory, one more dependent load per level step).
struct Levels {
    unsigned long long* p[kRelaxLevels];  // base of each level
    int32_t n[kRelaxLevels];              // nodes per level
    int nlev;                             // level nlev - 1 is the top
    int first_sm;  // levels first_sm.. are in shared memory, those below in global
};

__device__ __forceinline__ unsigned long long* lp(const Levels& L, int lev) {
    unsigned long long* r = L.p[0];
#pragma unroll
    for (int q = 1; q < kRelaxLevels; ++q) r = lev == q ? L.p[q] : r;
    return r;
}

__device__ __forceinline__ int64_t ln(const Levels& L, int lev) {
    int32_t r = L.n[0];
#pragma unroll
    for (int q = 1; q < kRelaxLevels; ++q) r = lev == q ? L.n[q] : r;
    return r;
}

// Node `node` of level `lev` from its 32 children (leaves when lev == 0).
__device__ __forceinline__ unsigned long long warp_node(const Inst& I, const Levels& L, int lev,
                                                        int64_t node) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (node << 5) + lane;
    unsigned long long v = 0ull;
    if (lev == 0) {
        if (c < I.n) v = I.key32[c];
    } else if (c < ln(L, lev - 1)) {
        v = lp(L, lev - 1)[c];
    }
    return warp_max_key(v);
}

// The top level's nodes, lane + 32 u in tv[u] (0 past its end).
__device__ __forceinline__ void load_top(const Levels& L, unsigned long long (&tv)[kTopPerLane]) {
    const int lane = threadIdx.x & 31;
    const unsigned long long* top = lp(L, L.nlev - 1);
    const int ntop = (int)ln(L, L.nlev - 1);
#pragma unroll
    for (int u = 0; u < kTopPerLane; ++u) tv[u] = lane + 32 * u < ntop ? top[lane + 32 * u] : 0ull;
}

// The largest key other than island w's: w's fellow leaves, at every level below
// the top the siblings of w's ancestor, and every top node but w's ancestor (from
// tv, the top as loaded by the caller). Warp-wide.
__device__ unsigned long long runner_up(const Inst& I, const Levels& L, int64_t w,
                                        const unsigned long long (&tv)[kTopPerLane]) {
    const int lane = threadIdx.x & 31;
    unsigned long long m = 0ull;
    {
        const int64_t c = ((w >> 5) << 5) + lane;
        if (c != w && c < I.n) m = I.key32[c];
    }
    // every level's load in flight at once (unrolled; the levels are independent)
#pragma unroll
    for (int lev = 1; lev < kRelaxLevels; ++lev) {
        const int64_t anc = w >> (5 * lev);
        const int64_t c = ((anc >> 5) << 5) + lane;
        if (lev < L.nlev && c != anc && c < L.n[lev - 1]) {
            const unsigned long long v = L.p[lev - 1][c];
            m = v > m ? v : m;
        }
    }
    const int64_t at = w >> (5 * L.nlev);
#pragma unroll
    for (int u = 0; u < kTopPerLane; ++u)
        if (lane + 32 * u != at) m = tv[u] > m ? tv[u] : m;
    return warp_max_key(m);
}

// An upper bound of every key other than islands w's and r's (r != w): the groups
// of leaves, at every level below the top the sibling sets, and the top, that hold
// w's or r's ancestors, less those ancestors. Warp-wide.
__device__ unsigned long long third_key(const Inst& I, const Levels& L, int64_t w, int64_t r,
                                        const unsigned long long (&tv)[kTopPerLane]) {
    const int lane = threadIdx.x & 31;
    unsigned long long m = 0ull;
    {
        const int64_t c = ((w >> 5) << 5) + lane, c2 = ((r >> 5) << 5) + lane;
        if (c != w && c != r && c < I.n) m = I.key32[c];
        if ((r >> 5) != (w >> 5) && c2 != r && c2 != w && c2 < I.n) {
            const unsigned long long v = I.key32[c2];
            m = v > m ? v : m;
        }
    }
#pragma unroll
    for (int lev = 1; lev < kRelaxLevels; ++lev) {
        if (lev >= L.nlev) break;
        const int64_t aw = w >> (5 * lev), ar = r >> (5 * lev);
        const int64_t c = ((aw >> 5) << 5) + lane, c2 = ((ar >> 5) << 5) + lane;
        const int64_t lim = L.n[lev - 1];
        if (c != aw && c != ar && c < lim) {
            const unsigned long long v = L.p[lev - 1][c];
            m = v > m ? v : m;
        }
        if ((ar >> 5) != (aw >> 5) && c2 != ar && c2 != aw && c2 < lim) {
            const unsigned long long v = L.p[lev - 1][c2];
            m = v > m ? v : m;
        }
    }
    const int64_t tw = w >> (5 * L.nlev), tr = r >> (5 * L.nlev);
#pragma unroll
    for (int u = 0; u < kTopPerLane; ++u)
        if (lane + 32 * u != tw && lane + 32 * u != tr) m = tv[u] > m ? tv[u] : m;
    return warp_max_key(m);
}

struct Dirty {
    int32_t lv0[kDirtyCap];    // first-level nodes to rebuild
    int32_t up[2][kDirtyCap];  // upper-level nodes, ping-pong by level parity
    int32_t n0;
};

// A leaf's key went from `old` to `nk`: a larger key is pushed up with atomic
// maxima on its ancestors, up to the first shared-memory one that already holds at
// least nk (nodes only grow while leaves change, so a stale read costs at most one
// more atomic; stopping early keeps most of the flip's keys off the few upper
// nodes, where same-address atomics serialise); if the leaf held its first-level
// node's maximum and shrank, that node is queued for a rebuild.
__device__ __forceinline__ void leaf_changed(const Inst& I, const Levels& L, Dirty& D, int64_t i,
                                             unsigned long long old, unsigned long long nk) {
    if (nk > old) {
        int64_t node = i;
#pragma unroll
        for (int lev = 0; lev < kRelaxLevels; ++lev) {  // (compile-time level indices)
            if (lev >= L.nlev) break;
            node >>= 5;
            unsigned long long* a = L.p[lev] + node;
            if (lev >= L.first_sm) {  // shared-memory instructions, not generic ones
                const unsigned sa = (unsigned)__cvta_generic_to_shared(a);
                unsigned long long cur;
                asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(cur) : "r"(sa));
                if (cur >= nk) break;
                asm volatile("red.shared.max.u64 [%0], %1;" ::"r"(sa), "l"(nk) : "memory");
            } else {  // (not read first: the read would wait for L2)
                atomicMax(a, nk);
            }
        }
    } else if (nk < old) {
        const int64_t node = i >> 5;
        if (lp(L, 0)[node] == old) {
            const int q = atomicAdd(&D.n0, 1);
            if (q < kDirtyCap) D.lv0[q] = (int32_t)node;
        }
    }
}

// The prediction of the next pick: the larger of the largest key the flip left
// untouched (the runner-up, when the flip was certified from bounds) and the
// largest new key among the flip's neighbours, folded into best[parity] with
// atomic maxima during the neighbour updates. Double-buffered by flip parity.
struct Prediction {
    unsigned long long best[2];
};

// Warp 0 after the neighbour updates: rebuilds the queued first-level nodes (their
// leaves loaded four nodes at a time) and then, level by level, every node above
// whose maximum was a key that shrank. Every lane reads the same node values, so
// the decision to queue a parent is warp-uniform and the queues' lengths stay in
// registers. Empties the first-level queue.
__device__ void repair_warp(const Inst& I, const Levels& L, Dirty& D) {
    constexpr int kBatch = 4;
    const int lane = threadIdx.x & 31;
    const int n0 = min(D.n0, kDirtyCap);
    int32_t* qout = D.up[1];
    int nout = 0;
    for (int q0 = 0; q0 < n0; q0 += kBatch) {
        unsigned long long v[kBatch];
        int64_t node[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            node[u] = q0 + u < n0 ? (int64_t)D.lv0[q0 + u] : -1;
            const int64_t c = (node[u] << 5) + lane;
            v[u] = node[u] >= 0 && c < I.n ? I.key32[c] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (node[u] < 0) break;
            const unsigned long long old = lp(L, 0)[node[u]];
            const unsigned long long nv = warp_max_key(v[u]);
            if (lane == 0) lp(L, 0)[node[u]] = nv;
            if (nv < old && L.nlev > 1 && lp(L, 1)[node[u] >> 5] == old) {
                if (lane == 0 && nout < kDirtyCap) qout[nout] = (int32_t)(node[u] >> 5);
                ++nout;
            }
            __syncwarp();
        }
    }
    int nn = min(nout, kDirtyCap);
    __syncwarp();
#pragma unroll
    for (int lev = 1; lev < kRelaxLevels; ++lev) {  // (compile-time level indices)
        if (lev >= L.nlev || nn <= 0) break;
        const int32_t* qin = D.up[lev & 1];
        qout = D.up[(lev + 1) & 1];
        const int64_t nchild = L.n[lev - 1];
        nout = 0;
        unsigned long long* const here = L.p[lev];
        const unsigned long long* const below = L.p[lev - 1];
        unsigned long long* const above =
            lev + 1 < kRelaxLevels && lev + 1 < L.nlev ? L.p[lev + 1 < kRelaxLevels ? lev + 1 : lev] : nullptr;
        for (int q = 0; q < nn; ++q) {
            const int64_t node = qin[q];
            const int64_t c = (node << 5) + lane;
            // the node, its children and its parent, loaded together
            const unsigned long long old = here[node];
            const unsigned long long cv = c < nchild ? below[c] : 0ull;
            const unsigned long long pv = above ? above[node >> 5] : 0ull;
            const unsigned long long nv = warp_max_key(cv);
            if (lane == 0) here[node] = nv;
            if (nv < old && above && pv == old) {
                if (lane == 0 && nout < kDirtyCap) qout[nout] = (int32_t)(node >> 5);
                ++nout;
            }
        }
        __syncwarp();
        nn = min(nout, kDirtyCap);
    }
    if (lane == 0) D.n0 = 0;
    __syncwarp();
}

// Whole tree from the leaves (after a full rescan).
__device__ void rebuild_tree(const Inst& I, const Levels& L) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int lev = 0; lev < L.nlev; ++lev) {
        for (int64_t node = wid; node < ln(L, lev); node += kNW) {
            const unsigned long long v = warp_node(I, L, lev, node);
            if (lane == 0) lp(L, lev)[node] = v;
        }
        __syncthreads();
    }
}

// Asks L2 for bytes [p, p + n) ahead of their use (TMA bulk prefetch: p 16-byte
// aligned, n a multiple of 16; no completion to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, uint32_t n) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n) : "memory");
}

// Column indices of row [a0, a1), which a flip of its island reads first. Rows
// start and end on multiples of 4 entries, so the range is 16-byte aligned with a
// length that is a multiple of 16 bytes. (The coefficient arrays are left to the
// speculating warps' own loads: asking for all five arrays queues five bulk
// requests per candidate on the flip's critical path, which measured slower.)
template <int PREC>
__device__ __forceinline__ void prefetch_row(const Inst& I, int64_t a0, int64_t a1) {
    const uint32_t m = (uint32_t)(a1 - a0);
    if (m != 0u) bulk_prefetch_l2(I.col + a0, 4u * m);
}

// Island j (key kj), whose row is [a0, a1), may be the next pick: its row's column
// indices are asked into L2 now and its key enters the prediction.
template <int PREC>
__device__ __forceinline__ void predict_candidate(const Inst& I, Prediction& P, int par,
                                                  unsigned long long kj, int64_t a0,
                                                  int64_t a1) {
    prefetch_row<PREC>(I, a0, a1);
    if (*(volatile unsigned long long*)&P.best[par] < kj) atomicMax(&P.best[par], kj);
}

// The update's effects: new sums, key, bounds and kept value; the tree told; and,
// when the new key exceeds `pf_above` (the largest key the flip did not touch),
// the island enters the prediction of the next pick.
template <int PREC>
__device__ __forceinline__ void commit_update(const Inst& I, const Levels& L, Dirty& D,
                                              Prediction& P, int par, const Upd& u,
                                              unsigned long long pf_above) {
    I.h64[u.i] = u.h;
    rec_store_dyn(I, u.i, u.g, u.lo, u.s);
    I.key64[u.i] = u.x;
    I.key32[u.i] = u.nk;
    leaf_changed(I, L, D, u.i, u.old, u.nk);
    if (u.nk > pf_above) predict_candidate<PREC>(I, P, par, u.nk, u.r0, u.r1);
}

struct RecheckShared {
    int32_t front[2][kRecheckCap];
    unsigned long long leaf_key[kRecheckCap];  // candidates' keys when collected
    unsigned long long new_key[kRecheckCap];
    int32_t result;
    float tau;
};

// Rebuilds every node on island w's path up to the top level from its children. Warp-wide.
__device__ void rebuild_path(const Inst& I, const Levels& L, int64_t w) {
    int64_t node = w;
    for (int lev = 0; lev < L.nlev; ++lev) {
        node >>= 5;
        const unsigned long long v = warp_node(I, L, lev, node);
        if ((threadIdx.x & 31) == 0) lp(L, lev)[node] = v;
        __syncwarp();
    }
}

// Exact comparison of the islands whose key bound reaches tau, by warp 0 alone.
// Returns the winner (its exact value is at least tau, so nothing outside the set
// can beat it) with its spin and row in *sk, *a0, *a1 on every lane and the largest
// new key among the other candidates in *next; -2 with R.tau
// lowered to widen the set; -1 when none of them is flippable; -3 when the set
// overflowed (nothing changed then). The candidates' keys become their exact
// values rounded out; the first-level nodes that held a lowered key are queued for
// the rebuild after the flip (the tree keeps upper bounds meanwhile, which every
// later comparison tolerates), except on -1, when their paths are repaired at once
// for the next look at the root.
template <int PREC>
__device__ int64_t recheck_warp(const Inst& I, const Levels& L, RecheckShared& R, Dirty& D,
                                float tau, uint32_t step, int* sk, int64_t* a0, int64_t* a1,
                                unsigned long long* next) {
    constexpr int kBatch = 4;  // frontier nodes whose children are loaded together
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned long long tkey = (unsigned long long)__float_as_uint(tau) << 32;
    // descent from the top through every node whose maximum reaches tau
    int cur = 0, nf = 0;
    {
        unsigned long long tv[kTopPerLane];
        load_top(L, tv);
#pragma unroll
        for (int u = 0; u < kTopPerLane; ++u) {
            const bool hit = tv[u] != 0ull && tv[u] >= tkey;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            const int pos = nf + __popc(m & lt);
            if (hit && pos < kRecheckCap) R.front[0][pos] = lane + 32 * u;
            nf += __popc(m);
        }
        __syncwarp();
        if (nf > kRecheckCap) return -3;
    }
    for (int lev = L.nlev - 1; lev >= 0; --lev) {
        const unsigned long long* src = lev > 0 ? lp(L, lev - 1) : I.key32;
        const int64_t lim = lev > 0 ? ln(L, lev - 1) : I.n;
        int nn = 0;
        for (int f0 = 0; f0 < nf; f0 += kBatch) {
            unsigned long long k[kBatch];
            int64_t child[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                child[u] = f0 + u < nf ? ((int64_t)R.front[cur][f0 + u] << 5) + lane : lim;
                k[u] = child[u] < lim ? src[child[u]] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const bool hit = k[u] != 0ull && k[u] >= tkey;
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                const int pos = nn + __popc(m & lt);
                if (hit && pos < kRecheckCap) {
                    R.front[cur ^ 1][pos] = (int32_t)child[u];
                    if (lev == 0) R.leaf_key[pos] = k[u];
                }
                nn += __popc(m);
            }
        }
        __syncwarp();
        if (nn > kRecheckCap) return -3;
        cur ^= 1;
        nf = nn;
    }
    const int nc = nf;
    // Per candidate, one lane each: the exact value, best by (value, lowest index);
    // the new key (exact value rounded out: only ever lower), queued rebuild.
    unsigned long long bv = 0ull;
    int64_t bi = -1;
    int bs = 0;
    int64_t b0 = 0, b1 = 0;
    for (int c = lane; c < nc; c += 32) {
        const int64_t i = R.front[cur][c];
        const IslandRec rc = rec_load(I, i);
        const int si = rc.s;
        const int64_t r0 = (int64_t)rc.rowq << 2, r1 = r0 + ((int64_t)rc.rowlenq << 2);
        const double v = exact_value<PREC>(I, i, step);
        const unsigned long long vb = v > 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull;
        if (vb > 0ull && (bi < 0 || vb > bv || (vb == bv && i < bi))) {
            bv = vb;
            bi = i;
            bs = si;
            b0 = r0;
            b1 = r1;
        }
        const unsigned long long old = R.leaf_key[c];
        const unsigned long long nk = v > 0.0 ? key32_of(__double2float_ru(v), i) : 0ull;
        I.key32[i] = nk;
        I.rec[i].lo = v > 0.0 ? __double2float_rd(v) : -1.0f;
        R.new_key[c] = nk;
        if (nk < old && lp(L, 0)[i >> 5] == old) {
            const int q = atomicAdd(&D.n0, 1);
            if (q < kDirtyCap) D.lv0[q] = (int32_t)(i >> 5);
        }
    }
    const int64_t my_bi = bi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
    }
    __syncwarp();
    const double bl = __longlong_as_double((long long)bv);
    if (bi >= 0 && bl >= (double)tau) {
        const int src = __ffs(__ballot_sync(0xffffffffu, my_bi == bi)) - 1;
        *sk = __shfl_sync(0xffffffffu, bs, src);
        *a0 = __shfl_sync(0xffffffffu, b0, src);
        *a1 = __shfl_sync(0xffffffffu, b1, src);
        // the largest new key among the other candidates: the next pick's likeliest
        unsigned long long nx = 0ull;
        for (int c = lane; c < nc; c += 32)
            if (R.front[cur][c] != bi && R.new_key[c] > nx) nx = R.new_key[c];
        *next = warp_max_key(nx);
        return bi;
    }
    if (bi >= 0) {
        if (lane == 0) R.tau = __double2float_rd(bl);  // something outside might beat it
        __syncwarp();
        return -2;
    }
    // none flippable: rebuild the nodes whose maximum was a lowered key, bottom-up
    for (int c = 0; c < nc; ++c) {
        const unsigned long long old = R.leaf_key[c];
        if (R.new_key[c] >= old) continue;
        int64_t node = (int64_t)R.front[cur][c];
        for (int lev = 0; lev < L.nlev; ++lev) {
            node >>= 5;
            if (lp(L, lev)[node] != old) break;
            const unsigned long long nv = warp_node(I, L, lev, node);
            if (lane == 0) lp(L, lev)[node] = nv;
            __syncwarp();
        }
    }
    return -1;
}

// Fallback when the candidate set overflows: every island whose key reaches tau
// is compared exactly, one thread each; the tree is rebuilt afterwards.
template <int PREC>
__device__ int64_t recheck_scan(const Inst& I, const Levels& L, RecheckShared& R, float tau,
                                uint32_t step) {
    __shared__ double sbl[kT];
    __shared__ int64_t sbi[kT];
    const unsigned long long tkey = (unsigned long long)__float_as_uint(tau) << 32;
    double bl = 0.0;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < I.n; i += kT) {
        const unsigned long long k = I.key32[i];
        if (k == 0ull || k < tkey) continue;
        const double v = exact_value<PREC>(I, i, step);
        I.key32[i] = v > 0.0 ? key32_of(__double2float_ru(v), i) : 0ull;
        I.rec[i].lo = v > 0.0 ? __double2float_rd(v) : -1.0f;
        if (v > 0.0 && (bi < 0 || v > bl || (v == bl && i < bi))) {
            bl = v;
            bi = i;
        }
    }
    sbl[threadIdx.x] = bl;
    sbi[threadIdx.x] = bi;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < kT; ++t) {
            if (sbi[t] < 0) continue;
            if (bi < 0 || sbl[t] > bl || (sbl[t] == bl && sbi[t] < bi)) {
                bl = sbl[t];
                bi = sbi[t];
            }
        }
        if (bi >= 0 && bl >= (double)tau) {
            R.result = (int32_t)bi;
        } else if (bi >= 0) {
            R.result = -2;
            R.tau = __double2float_rd(bl);
        } else {
            R.result = -1;
        }
    }
    __syncthreads();
    rebuild_tree(I, L);
    return R.result;
}

// Exact comparison of islands w and r when no other key reaches tau <= x(w) (the
// caller has checked): the exact best of the two is the pick. Both get keys from
// their exact values (lowered; their first-level nodes queued for the repair when
// they held the old key). Warp-wide; returns the pick with its spin and row, and
// the other one's new key in *kother.
template <int PREC>
__device__ int64_t pair_compare(const Inst& I, const Levels& L, Dirty& D, int64_t w, int64_t r,
                                unsigned long long kw, unsigned long long kr, uint32_t step,
                                int* sk, int64_t* a0, int64_t* a1,
                                unsigned long long* kother) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    int si = 0;
    int64_t r0 = 0, r1 = 0;
    unsigned long long nk = 0ull;
    if (lane < 2) {
        const int64_t i = lane == 0 ? w : r;
        const unsigned long long old = lane == 0 ? kw : kr;
        const IslandRec rc = rec_load(I, i);
        si = rc.s;
        r0 = (int64_t)rc.rowq << 2;
        r1 = r0 + ((int64_t)rc.rowlenq << 2);
        v = exact_value<PREC>(I, i, step);
        nk = v > 0.0 ? key32_of(__double2float_ru(v), i) : 0ull;
        I.key32[i] = nk;
        I.rec[i].lo = v > 0.0 ? __double2float_rd(v) : -1.0f;
        if (nk < old && lp(L, 0)[i >> 5] == old) {
            const int q = atomicAdd(&D.n0, 1);
            if (q < kDirtyCap) D.lv0[q] = (int32_t)(i >> 5);
        }
    }
    const double vw = __shfl_sync(0xffffffffu, v, 0), vr = __shfl_sync(0xffffffffu, v, 1);
    // w is flippable (its lower bound exceeds one); r wins on a larger value, or an
    // equal one with a lower index
    const int src = (vr > vw || (vr == vw && r < w)) ? 1 : 0;
    *sk = __shfl_sync(0xffffffffu, si, src);
    *a0 = __shfl_sync(0xffffffffu, r0, src);
    *a1 = __shfl_sync(0xffffffffu, r1, src);
    *kother = __shfl_sync(0xffffffffu, nk, src ^ 1);
    __syncwarp();
    return src == 1 ? r : w;
}

// Pick codes besides an island index.
constexpr int64_t kPickNone = -1;      // no flippable island: the relax is done
constexpr int64_t kPickOverflow = -3;  // exact comparison needs the CTA-wide scan
constexpr int64_t kPickBounds = -4;    // the comparison did not settle
constexpr int64_t kPickMaxFlips = -6;  // flip budget of the step spent

// Warp 0: the island to flip next. Reads the root's island w and the largest other
// key; takes w when its certified lower bound exceeds one and that key's upper
// bound, else compares the contenders exactly. On return lane 0 holds the pick's
// spin and row, `ru` the largest key other than the pick's when it was certified
// from bounds, or after an exact comparison of two the larger of the other one's
// new key and the third key, or after a wider comparison the largest new key
// among its other candidates (the next pick's likeliest island), and `clean`
// whether no key changed on the way (no exact comparison ran).
template <int PREC>
__device__ int64_t pick_warp(const Inst& I, const Levels& L, RecheckShared& R, Dirty& D,
                             InstState* st, uint32_t step, int* sk, int64_t* a0, int64_t* a1,
                             unsigned long long* ru_out, float* tau_out, bool* clean) {
    const int lane = threadIdx.x & 31;
    *ru_out = ~0ull;
    *clean = true;
    for (int guard = 0; guard < 4 * kRecheckCap + 64; ++guard) {
        unsigned long long tv[kTopPerLane];
        load_top(L, tv);
        unsigned long long tm = tv[0];
#pragma unroll
        for (int u = 1; u < kTopPerLane; ++u) tm = tv[u] > tm ? tv[u] : tm;
        const unsigned long long root = warp_max_key(tm);
        if (root == 0ull) return kPickNone;
        const int64_t w = key32_idx(root);
        unsigned long long kw = 0ull;
        float lo = 0.0f;
        if (lane == 0) {  // independent loads, in flight during the runner-up scan
            kw = I.key32[w];
            const IslandRec r = rec_load(I, w);
            lo = r.lo;
            *sk = r.s;
            *a0 = (int64_t)r.rowq << 2;
            *a1 = *a0 + ((int64_t)r.rowlenq << 2);
        }
        const unsigned long long ru = runner_up(I, L, w, tv);
        kw = __shfl_sync(0xffffffffu, kw, 0);
        lo = __shfl_sync(0xffffffffu, lo, 0);
        if (kw != root) {  // a lowered key still held by its ancestors
            rebuild_path(I, L, w);
            continue;
        }
        const float hi2 = ru ? key32_hi(ru) : 0.0f;
        if (lo > 1.0f && lo > hi2) {
            *ru_out = ru;
            return w;
        }
        // With tau = lo(w) > 1 the set holds w, whose exact value is at least tau,
        // so one round settles it; at the threshold, start from the runner-up.
        float tau = lo > 1.0f ? lo : fmaxf(hi2, lo);
        if (lo > 1.0f && ru != 0ull && (int64_t)key32_idx(ru) != w) {
            // When no key but w's and the runner-up's reaches tau, those two alone are
            // compared exactly (no descent through the tree).
            const int64_t r = key32_idx(ru);
            const unsigned long long k3 = third_key(I, L, w, r, tv);
            if (k3 < ((unsigned long long)__float_as_uint(tau) << 32)) {
                *clean = false;
                if (lane == 0) atomicAdd((unsigned long long*)&st->rechecks, 1ull);
                unsigned long long ko;
                const int64_t k = pair_compare<PREC>(I, L, D, w, r, kw, ru, step, sk, a0, a1, &ko);
                *ru_out = ko > k3 ? ko : k3;
                return k;
            }
        }
        int64_t k = -2;
        unsigned long long nx = ~0ull;
        for (int rounds = 0; k == -2;) {
            if (++rounds > 64) return kPickBounds;
            *clean = false;
            k = recheck_warp<PREC>(I, L, R, D, tau, step, sk, a0, a1, &nx);
            if (lane == 0) atomicAdd((unsigned long long*)&st->rechecks, 1ull);
            if (k == -2) tau = R.tau;
        }
        if (k == -1) continue;  // every contender was demoted: look at the root again
        if (k == kPickOverflow) {
            *tau_out = tau;
            return k;
        }
        *ru_out = nx;
        return k;
    }
    return kPickBounds;
}

// The relax of one simulation's field step by the whole CTA (the body of k_relax,
// and a work item of the persistent batch kernel). sm_levels: the dynamic shared
// memory for the upper tree levels, smem_levels bytes. beat (or NULL): a counter
// raised every 256 flips, so that CTAs waiting for work see that this one is
// still making progress.
template <int PREC>
__device__ __forceinline__ void relax_sim(const Inst& I, int smem_levels, int cont,
                                          unsigned long long* sm_levels, unsigned* beat) {
    __shared__ int64_t sh_k;
    __shared__ Prediction P;
    __shared__ int64_t sh_e0, sh_e1;
    __shared__ unsigned long long sh_ru;
    __shared__ int32_t sh_snew;
    __shared__ int32_t sh_clean;
    __shared__ float sh_tau;
    __shared__ int32_t sh_spec_snew[kNW];  // spin after the flip each speculating warp assumed
    __shared__ int32_t sh_spec_len;
    __shared__ RecheckShared R;
    __shared__ Dirty D;

    InstState* st = I.st;
    // cont: launched after the multi-flip relax of the same step, which either
    // finished it (nothing to do) or handed the rest over (continue from its flips)
    if (cont && st->handoff == 0) return;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;
    const int64_t prior = cont ? st->step_flips : 0;  // the step's flips before the hand-off
    const uint32_t step = I.step0 + (uint32_t)t;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    // The levels up to the top (the first with at most kRelaxTopNodes nodes); the
    // upper ones in shared memory while they fit.
    int nl = 1;
    while (nl < I.nlev && I.lvl_n[nl - 1] > kRelaxTopNodes) ++nl;
    if (nl > kRelaxLevels) {  // (more islands than the indices allow; not reached)
        if (threadIdx.x == 0) st->status = ST_BOUNDS;
        return;
    }
    Levels L;
    {
        int64_t used = 0;
        int first_sm = nl;
        for (int lev = nl - 1; lev >= 0; --lev) {
            const int64_t b = (int64_t)I.lvl_n[lev] * (int64_t)sizeof(unsigned long long);
            if (used + b > smem_levels) break;
            used += b;
            first_sm = lev;
        }
        L.first_sm = first_sm;
        L.nlev = nl;
        // (static indices only: the descriptor stays in registers)
        int64_t off = 0;
#pragma unroll
        for (int lev = kRelaxLevels - 1; lev >= 0; --lev) {
            L.n[lev] = lev < nl ? I.lvl_n[lev] : 0;
            if (lev < nl && lev >= first_sm) {
                L.p[lev] = sm_levels + off;
                off += I.lvl_n[lev];
            } else {
                L.p[lev] = lev < nl ? I.tree + I.lvl_off[lev] : nullptr;
            }
        }
        for (int lev = first_sm; lev < L.nlev; ++lev)
            for (int64_t q = threadIdx.x; q < ln(L, lev); q += kT)
                lp(L, lev)[q] = I.tree[I.lvl_off[lev] + q];
        if (threadIdx.x == 0) {
            D.n0 = 0;
            P.best[0] = 0ull;
            P.best[1] = 0ull;
        }
    }
    __syncthreads();

    int64_t flips = 0;
    int32_t status = ST_OK;
    uint64_t hash = threadIdx.x == kHashThread ? st->hash : 0ull;
    const int64_t flips_before = threadIdx.x == 0 ? st->n_flips : 0;
    const int64_t max_flips = I.max_flips;
    int par = 0;  // parity of the flip whose neighbour updates ran last
    // Full-scan comparisons that demoted every contender without a flip, since the
    // last flip. Each one lowers at least one key to zero, so a relax needs at most
    // n of them in a row; the cap turns a failure of that argument into ST_BOUNDS
    // instead of an endless loop.
    int64_t demotions = 0;
    const int64_t kMaxDemotions = I.n + 64;

    // Thread 0: flip island k, log it, publish its row.
    auto do_flip = [&](int64_t k, int sk, int64_t a0, int64_t a1) {
        const int snew = -sk;
        I.s[k] = (int8_t)snew;
        I.rec[k].s = snew;
        sh_snew = snew;
        sh_e0 = a0;
        sh_e1 = a1;
        const int64_t q = flips_before + flips;
        if (I.log_spin && q < I.log_cap) {
            I.log_step[q] = step;
            I.log_spin[q] = (uint32_t)k;
        }
    };

    for (;;) {
        // Predicted next pick (from the last neighbour updates), read by every thread.
        const unsigned long long pk = P.best[par];
        const int64_t pred = pk != 0ull ? (int64_t)key32_idx(pk) : -1;
        Upd spec;
        spec.i = -1;
        if (wid == 0) {
            // repair the tree, pick, and flip
            repair_warp(I, L, D);
            int sk = 0;
            int64_t a0 = 0, a1 = 0;
            unsigned long long ru = ~0ull;
            float tau = 0.0f;
            bool clean = true;
            int64_t k =
                pick_warp<PREC>(I, L, R, D, st, step, &sk, &a0, &a1, &ru, &tau, &clean);
            if (lane == 0) {
                if (k >= 0) {
                    if (prior + flips < max_flips)
                        do_flip(k, sk, a0, a1);
                    else
                        k = kPickMaxFlips;
                }
                sh_k = k;
                sh_ru = ru;
                sh_tau = tau;
                sh_clean = clean ? 1 : 0;
                P.best[par ^ 1] = 0ull;  // the next updates' prediction
            }
        } else if (pred >= 0) {
            // Meanwhile warps 1..7 compute the predicted flip's neighbour updates
            // (loads and arithmetic only), one entry of its row per thread.
            const IslandRec rpr = rec_load(I, pred);
            const int sp = rpr.s;
            const int64_t a0 = (int64_t)rpr.rowq << 2;
            const int len = (int)rpr.rowlenq << 2;
            if (lane == 0) sh_spec_snew[wid] = -sp;
            if (threadIdx.x == 32) sh_spec_len = len;
            const int q = threadIdx.x - 32;
            if (len < kT - 32 && q < len) {
                const int64_t e = a0 + q;
                const int32_t i = __ldg(&I.col[e]);
                const long long dp = __ldg(&I.pq64[e].x), dq = __ldg(&I.qt64[e]);
                int dp32 = 0, dq32 = 0;
                if constexpr (PREC == 1) {
                    dp32 = __ldg(&I.pq32[e].x);
                    dq32 = __ldg(&I.qt32[e]);
                }
                if (i != (int32_t)pred)  // not row padding
                    spec = compute_update<PREC, false>(I, i, -sp, dp, dq, dp32, dq32, step);
            } else if (len < kT - 32 && q == len) {
                // the predicted island itself: its field unchanged, its spin flipped
                spec = compute_update<PREC, false>(I, pred, -sp, 0, 0, 0, 0, step, -sp);
            }
        }
        __syncthreads();
        int64_t k = sh_k;
        if (k == kPickOverflow) {
            // too many contenders for one warp: every thread compares exactly
            float tau = sh_tau;
            int64_t r = -2;
            for (int rounds = 0; r == -2 && rounds < 64; ++rounds) {
                if (threadIdx.x == 0) atomicAdd((unsigned long long*)&st->fallbacks, 1ull);
                r = recheck_scan<PREC>(I, L, R, tau, step);
                tau = R.tau;
            }
            if (r == -1 && ++demotions <= kMaxDemotions) {
                __syncthreads();
                continue;  // everything examined was demoted: look at the root again
            }
            if (r == -1) r = -2;  // (the retries' cap: reported as a bounds failure)
            if (r == -2) {
                k = kPickBounds;
            } else {
                if (threadIdx.x == 0) {
                    if (prior + flips < max_flips) {
                        const IslandRec rr = rec_load(I, r);
                        const int64_t ra = (int64_t)rr.rowq << 2;
                        do_flip(r, rr.s, ra, ra + ((int64_t)rr.rowlenq << 2));
                        sh_k = r;
                    } else {
                        sh_k = kPickMaxFlips;
                    }
                    sh_ru = ~0ull;
                    sh_clean = 0;
                }
                __syncthreads();
                k = sh_k;
            }
        }
        if (k == kPickBounds) {
            status = ST_BOUNDS;
            break;
        }
        if (k == kPickMaxFlips) {
            status = ST_NOT_CONVERGED;
            break;
        }
        if (k < 0) break;
        ++flips;
        demotions = 0;
        par ^= 1;
        if (beat != nullptr && threadIdx.x == 0 && (flips & 255) == 0) atomicAdd(beat, 1u);
        if (threadIdx.x == kHashThread) hash = fnv_flip(hash, step, (uint32_t)k);
        // every neighbour i of k: add 2 s_k(new) (P_ik, Q_ik), new key, tree update
        const int snew = sh_snew;
        const unsigned long long ru = sh_ru;
        // An exact comparison during the pick changes keys, bounds, kept values and
        // kept thermal draws (published so that a concurrent reader sees a whole draw
        // or none, and a draw is the same value either way), never sums or spins, so
        // the precomputed updates stay valid once each takes its island's current key
        // as the old one.
        const bool clean = sh_clean != 0;
        bool use_spec = k == pred && sh_spec_len < kT - 32;
#pragma unroll
        for (int w = 1; w < kNW; ++w) use_spec = use_spec && sh_spec_snew[w] == snew;
        if (use_spec) {
            if (spec.i >= 0) {
                if (!clean) spec.old = I.key32[spec.i];
                commit_update<PREC>(I, L, D, P, par, spec, spec.i == k ? ~0ull : ru);
            }
        } else {
            const int64_t e0 = sh_e0;
            const int len = (int)(sh_e1 - e0);
            for (int q = threadIdx.x; q < len; q += kT) {
                const int64_t e = e0 + q;
                // the row's entries (read-only), all issued before the padding test
                const int32_t i = __ldg(&I.col[e]);
                const long long dp = __ldg(&I.pq64[e].x), dq = __ldg(&I.qt64[e]);
                int dp32 = 0, dq32 = 0;
                if constexpr (PREC == 1) {
                    dp32 = __ldg(&I.pq32[e].x);
                    dq32 = __ldg(&I.qt32[e]);
                }
                if (i == (int32_t)k) continue;  // row padding
                const Upd u = compute_update<PREC, true>(I, i, snew, dp, dq, dp32, dq32, step);
                commit_update<PREC>(I, L, D, P, par, u, ru);
            }
        }
        // k's own field is unchanged; its key is not (already computed ahead on the
        // speculative path; on the other, the last thread seldom holds an entry).
        if (!use_spec && threadIdx.x == kT - 1) {
            const Upd u = compute_update<PREC, true>(I, k, snew, 0, 0, 0, 0, step);
            commit_update<PREC>(I, L, D, P, par, u, ~0ull);
        }
        // the runner-up is the next pick unless a neighbour rises above it
        if (threadIdx.x == 0 && ru != ~0ull && ru != 0ull) atomicMax(&P.best[par], ru);
        __syncthreads();
    }
    if (threadIdx.x == kHashThread) st->hash = hash;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (I.flips_per_step) I.flips_per_step[t] = prior + flips;
        st->n_flips = flips_before + flips;
        st->handoff = 0;
        if (status != ST_OK) st->status = status;
        st->init = 0;
        st->t = t + 1;
    }
}

// MINB: resident CTAs per SM the build is made for. One CTA per SM (registers as
// needed) for a relax that has the GPU to itself; two (at most 128 registers a
// thread) for a batch with more members than SMs, so that each SM interleaves two
// latency-bound chains (measured: 24.3M vs 20.9M flips/s on the 512-member FP32
// ensemble; the server's requests, fewer at a time, run faster with one).
template <int PREC, int MINB>
__global__ void __launch_bounds__(kT, MINB)
    k_relax(const Inst* __restrict__ tab, const int32_t* __restrict__ work, int n_work,
            int smem_levels, int cont) {
    extern __shared__ unsigned long long sm_levels[];
    relax_sim<PREC>(tab[work[blockIdx.x]], smem_levels, cont, sm_levels, nullptr);
}

// Total field, LHS and its bounds for every island at the current state (FS_FP64
// values for prec 0 with lo = hi = LHS; the FP32 evaluation and its bounds for
// prec 1).
__global__ void k_eval_all(const Inst* __restrict__ tab, double hx, double hy, uint32_t step,
                           double* __restrict__ hpar, double* __restrict__ hperp,
                           double* __restrict__ lhs, double* __restrict__ lo,
                           double* __restrict__ hi) {
    const Inst& I = tab[0];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= I.n) return;
    const IslandRec r = rec_load(I, i);
    const int si = r.s;
    const uint16_t ci = r.cls;
    const double2 lab = ext_lab(I, i, step, hx, hy);
    const double2 ext = ext_proj(lab.x, lab.y, I.cs64[ci]);
    if (I.prec == 1) {
        const int2 h = r.h32;
        const float2 th = I.sigma > 0.0 ? thermal32(I, i, step) : make_float2(0.0f, 0.0f);
        const Eval32 e = eval32(I, si, __fmul_rn(__int2float_rn(h.x), I.inv32),
                                __fmul_rn(__int2float_rn(h.y), I.inv32), r.rbc,
                                make_float2(__double2float_rn(ext.x), __double2float_rn(ext.y)),
                                th.x, th.y);
        hpar[i] = e.hpar;
        hperp[i] = e.hperp;
        lhs[i] = e.lhs;
        lo[i] = e.lo;
        hi[i] = e.hi;
    } else {
        const longlong2 h = I.h64[i];
        double tp = 0.0, tq = 0.0;
        if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
        const Eval64 e = eval64(I, si, h.x, h.y, I.rbc64[i], ext, tp, tq);
        hpar[i] = e.hpar;
        hperp[i] = e.hperp;
        lhs[i] = e.lhs;
        lo[i] = e.lhs;
        hi[i] = e.lhs;
    }
}

// ---- Persistent batch kernel ------------------------------------------------
// Every member of a batch advances its own protocol (Sec. "Simulation framework":
// ensembles and parameter sweeps), inside one launch: a CTA takes whatever work is
// ready — first the relax of a member whose field step has been swept (members in
// queue order, largest first), else a chunk of a member's sweep — so that one
// member's relax (a latency-bound chain on one SM) overlaps other members' sweeps
// (bandwidth-bound), and no member waits for another's field step. A member's
// steps are the same kernels' work as in per-step launches (the sweep task, the
// single-flip relax), in the same order, so its results are those of a solo run.
//
// Hand-offs between CTAs: the warp that completes a sweep's tree marks the member
// ready; the CTA that relaxed it computes the next step's external-field table,
// resets its chunk counter and marks it sweeping; claims are atomics, each side
// fenced, so that the claimer sees everything the previous owner wrote. The spins
// are read through the coherent path (other CTAs flip them within this launch).
// A CTA that finds no work sleeps and looks again; it stops when every member is
// done, or, having seen no progress anywhere (no item finished, no relax's
// 256-flip beat) for kIdleLimitNs, it sets the fault word and stops (the host
// reports FS_ERR_BOUNDS).
constexpr int kChunkPerWarp = 4;               // tasks a warp sweeps per claimed chunk
constexpr int kChunkTasks = kNW * kChunkPerWarp;
constexpr unsigned long long kIdleLimitNs = 10000000000ull;  // 10 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int32_t ld_volatile(const int32_t* p) {
    return *reinterpret_cast<const volatile int32_t*>(p);
}
__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

__global__ void k_persist_init(PersistLaunch A) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= A.n) return;
    const int m = A.work[p];
    const Inst& I = A.tab[m];
    const InstState* st = I.st;
    const int64_t tasks = A.task_start[m + 1] - A.task_start[m];
    A.nchunk[p] = (uint32_t)((tasks + kChunkTasks - 1) / kChunkTasks);
    A.chunk[p] = 0u;
    const bool done = st->status != ST_OK || st->t >= I.K;
    A.state[p] = done ? kQDone : kQSweep;
    if (done) atomicAdd(&A.ctl[0], 1);
}

template <int PREC, int W, int MODE>
__global__ void __launch_bounds__(kT, 2) k_batch_persist(PersistLaunch A) {
    extern __shared__ unsigned long long sm_levels[];
    __shared__ int sums32[PREC == 1 ? kNW : 1][32][2];
    __shared__ long long sums64[kNW][32][2];
    __shared__ int32_t q_kind, q_pos, q_best, q_stop;
    __shared__ uint32_t q_chunk;
    __shared__ int64_t q_t;
    __shared__ int32_t q_init, q_next;
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    int32_t* const n_done = &A.ctl[0];
    int32_t* const fault = &A.ctl[1];
    unsigned* const beat = reinterpret_cast<unsigned*>(&A.ctl[2]);
    unsigned seen = 0u;                     // (thread 0) the progress beat last seen
    unsigned long long quiet_since = 0ull;  // (thread 0) when it last changed
    unsigned nap = 64u;                     // ns to sleep after a pass without work
    int aff = -1;   // the member this CTA last relaxed or swept: its work is tried first
    for (;;) {
        // The next item: the member this CTA worked on last (its relax when its sweep
        // is done, else a chunk of its sweep), else the first member in queue order
        // (largest first) with either: the longest chains are kept moving first.
        if (tid == 0) {
            q_kind = 0;
            if (aff >= 0) {
                const int32_t sa = ld_volatile(&A.state[aff]);
                if (sa == kQReady && atomicCAS(&A.state[aff], kQReady, kQRelax) == kQReady) {
                    q_kind = 1;
                    q_pos = aff;
                } else if (sa == kQSweep && ld_volatile(&A.chunk[aff]) < A.nchunk[aff]) {
                    const uint32_t c = atomicAdd(&A.chunk[aff], 1u);
                    if (c < A.nchunk[aff]) {
                        q_kind = 2;
                        q_pos = aff;
                        q_chunk = c;
                    }
                }
            }
            q_best = 0x7fffffff;
        }
        __syncthreads();
        if (q_kind == 0) {
            for (int p = tid; p < A.n; p += kT) {
                const int32_t sp = ld_volatile(&A.state[p]);
                if (sp == kQReady || (sp == kQSweep && ld_volatile(&A.chunk[p]) < A.nchunk[p])) {
                    atomicMin(&q_best, p);
                    break;
                }
            }
            __syncthreads();
            if (tid == 0 && q_best != 0x7fffffff) {
                const int p = q_best;
                if (ld_volatile(&A.state[p]) == kQReady) {
                    if (atomicCAS(&A.state[p], kQReady, kQRelax) == kQReady) {
                        q_kind = 1;
                        q_pos = p;
                    }
                } else {
                    const uint32_t c = atomicAdd(&A.chunk[p], 1u);
                    if (c < A.nchunk[p]) {
                        q_kind = 2;
                        q_pos = p;
                        q_chunk = c;
                    }
                }
                if (q_kind == 0) q_kind = -1;  // lost a race for it: look again at once
            }
            __syncthreads();
        }
        if (q_kind == -1) continue;
        if (q_kind == 0) {
            aff = -1;
            // nothing to take: finished, faulted, or wait
            if (tid == 0) {
                q_stop = 0;
                if (ld_volatile(n_done) >= A.n || ld_volatile(fault) != 0) {
                    q_stop = 1;
                } else {
                    const unsigned b = ld_volatile(reinterpret_cast<const uint32_t*>(beat));
                    const unsigned long long now = global_ns();
                    if (b != seen || quiet_since == 0ull) {
                        seen = b;
                        quiet_since = now;
                    } else if (now - quiet_since > kIdleLimitNs) {
                        atomicExch(fault, 1);
                        q_stop = 1;
                    }
                }
            }
            __syncthreads();
            if (q_stop) return;
            __nanosleep(nap);
            nap = min(nap * 2u, 4096u);
            continue;
        }
        nap = 64u;
        aff = q_pos;
        if (tid == 0) {
            __threadfence();  // (acquire: the claim observed the previous owner's release)
            const Inst& I = A.tab[A.work[q_pos]];
            q_t = I.st->t;
            q_init = I.st->init;
        }
        __syncthreads();
        __threadfence();  // (every thread, before it reads the member's state)
        const int m = A.work[q_pos];
        const Inst& I = A.tab[m];
        if (q_kind == 2) {
            // a chunk of the member's sweep: warp w takes tasks chunk * kChunkTasks +
            // u * kNW + w, so that the CTA streams neighbouring rows together
            const int64_t tasks = A.task_start[m + 1] - A.task_start[m];
            for (int u = 0; u < kChunkPerWarp; ++u) {
                const int64_t lt = (int64_t)q_chunk * kChunkTasks + u * kNW + wid;
                if (lt >= tasks) break;
                const bool root = sweep_task<PREC, W, MODE, true>(
                    I, A.tcnts[m], q_t, lt, q_init != 0, sums32[PREC == 1 ? wid : 0], sums64[wid]);
                if (root && lane == 0) {  // the tree is complete: the relax is next
                    __threadfence();
                    atomicExch(&A.state[q_pos], kQReady);
                    atomicAdd(beat, 1u);
                }
            }
            __syncthreads();
            continue;  // (a completed tree: this CTA tries the member's relax first)
        }
        // the member's relax, then its next field step
        relax_sim<PREC>(I, A.smem_levels, 0, sm_levels, beat);
        __threadfence();  // (every thread's stores, before the member changes hands)
        __syncthreads();
        if (tid == 0) {
            const InstState* st = I.st;
            q_next = st->status == ST_OK && st->t < I.K ? 1 : 0;
            q_t = st->t;
        }
        __syncthreads();
        if (q_next) {
            // the next step's external field on every angle class
            const double hx = I.phx[q_t], hy = I.phy[q_t];
            for (int c = tid; c < I.nclass; c += kT) {
                const double2 e = ext_proj(hx, hy, I.cs64[c]);
                I.ext64[c] = e;
                I.ext32[c] = make_float2(__double2float_rn(e.x), __double2float_rn(e.y));
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            if (q_next) {
                atomicExch(&A.chunk[q_pos], 0u);
                __threadfence();
                atomicExch(&A.state[q_pos], kQSweep);
            } else {
                atomicExch(&A.state[q_pos], kQDone);
                atomicAdd(n_done, 1);
            }
            atomicAdd(beat, 1u);
        }
        __syncthreads();
    }
}

template <int PREC, int MODE>
void* persist_fn(int W) {
    switch (W) {
        case 2:
            return (void*)k_batch_persist<PREC, 2, MODE>;
        case 4:
            return (void*)k_batch_persist<PREC, 4, MODE>;
        case 8:
            return (void*)k_batch_persist<PREC, 8, MODE>;
        case 16:
            return (void*)k_batch_persist<PREC, 16, MODE>;
        default:
            return (void*)k_batch_persist<PREC, 32, MODE>;
    }
}

}  // namespace

int relax_threads() { return kT; }

size_t relax_static_smem(int prec) {
    cudaFuncAttributes a{};
    if (prec == 1)
        cudaFuncGetAttributes(&a, k_relax<1, 1>);
    else
        cudaFuncGetAttributes(&a, k_relax<0, 1>);
    return a.sharedSizeBytes;
}

// Sets the dynamic shared-memory limit of the relax kernels once per size (a
// no-op afterwards, so launches can be captured in graphs). Thread-safe: the
// server's builder threads reach it concurrently.
cudaError_t prepare_relax(int prec, int smem) {
    static std::atomic<int> set_bytes[2] = {{-1}, {-1}};
    static std::mutex mu;
    const int k = prec == 1 ? 1 : 0;
    if (set_bytes[k].load() >= smem) return cudaSuccess;
    std::lock_guard<std::mutex> g(mu);
    if (set_bytes[k].load() >= smem) return cudaSuccess;
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if (prec == 1) {
        e = cudaFuncSetAttribute(k_relax<1, 1>, A, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_relax<1, 2>, A, smem);
    } else {
        e = cudaFuncSetAttribute(k_relax<0, 1>, A, smem);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_relax<0, 2>, A, smem);
    }
    if (e == cudaSuccess) set_bytes[k].store(smem);
    return e;
}

cudaError_t launch_relax(const RelaxLaunch& L, cudaStream_t st) {
    if (L.n_work == 0) return cudaSuccess;
    // multi-flip rounds first; the single-flip kernel then takes over a step they
    // handed off (and returns at once otherwise)
    if (L.multi) {
        const cudaError_t e = launch_relax_multi(L, st);
        if (e != cudaSuccess) return e;
    }
    const int cont = L.multi ? 1 : 0;
    const cudaError_t e = prepare_relax(L.prec, L.smem_levels);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)L.n_work;
    const int sm = L.smem_levels;
    if (L.prec == 1) {
        if (L.min_blocks == 2)
            k_relax<1, 2><<<g, kT, sm, st>>>(L.tab, L.work, L.n_work, sm, cont);
        else
            k_relax<1, 1><<<g, kT, sm, st>>>(L.tab, L.work, L.n_work, sm, cont);
    } else {
        if (L.min_blocks == 2)
            k_relax<0, 2><<<g, kT, sm, st>>>(L.tab, L.work, L.n_work, sm, cont);
        else
            k_relax<0, 1><<<g, kT, sm, st>>>(L.tab, L.work, L.n_work, sm, cont);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_persist(const PersistLaunch& L, cudaStream_t st) {
    if (L.n == 0) return cudaSuccess;
    void* fn = L.prec == 1 ? (L.resweep ? persist_fn<1, 1>(L.lanes_per_row)
                                        : persist_fn<1, 0>(L.lanes_per_row))
                           : (L.resweep ? persist_fn<0, 1>(L.lanes_per_row)
                                        : persist_fn<0, 0>(L.lanes_per_row));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         L.smem_levels);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kT,
                                                           (size_t)L.smem_levels)) != cudaSuccess)
        return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    k_persist_init<<<(L.n + 255) / 256, 256, 0, st>>>(L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // every CTA resident at once (no CTA waits for a particular other one, so this
    // is for speed, not for progress)
    void* args[] = {(void*)&L};
    return cudaLaunchKernel(fn, dim3((unsigned)(per_sm * nsm)), dim3(kT), args,
                            (size_t)L.smem_levels, st);
}

cudaError_t launch_eval_all(const Inst* tab, int64_t n, double hx, double hy, uint32_t step,
                            double* out5, cudaStream_t st) {
    k_eval_all<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tab, hx, hy, step, out5, out5 + n,
                                                           out5 + 2 * n, out5 + 3 * n,
                                                           out5 + 4 * n);
    return cudaGetLastError();
}

}  // namespace fs
