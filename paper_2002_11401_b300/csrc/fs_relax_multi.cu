// fs_relax_multi.cu - the greedy relax of Sec. "Dynamics" in rounds of several
// flips, each round exactly the next flips of the single-flip order.
//
// The single-flip relax flips the flippable island with the largest Eq. 5 LHS
// (lowest index on ties), updates its neighbours, and repeats. A round here takes
// the islands with the largest keys in the order of their exact (FS_FP64) values,
// v_0 > v_1 > ... (lowest index first on ties), and flips the longest prefix
// c_0 .. c_{p-1} of that order that the single-flip relax would flip next, in the
// same order. c_i is the next single flip after c_0 .. c_{i-1} when
//  (a) it beats every island outside the candidate set: the candidates are all
//      islands whose key (an upper bound of the exact value) reaches a threshold,
//      and c_i's exact value reaches that threshold too;
//  (b) no earlier pick changed its field or shares a neighbour with it: picks are
//      more than twice the cutoff apart, so each island's field changes by at most
//      one pick of the round and every neighbour's new value is that of one flip;
//  (c) no neighbour of an earlier pick got a new value that beats it (the flipped
//      islands themselves are no longer flippable: their field is unchanged and
//      their spin now opposes h_par's sign).
// (a) and (b) are checked before the round's flips; all picks that pass them are
// flipped at once (their neighbourhoods are disjoint), (c) is checked on the new
// values, and the picks after the first that fails are flipped back (the exact
// integer sums return to their old values and every key is evaluated again from
// them). A round therefore always flips at least one island, and the flip
// sequence, the flips per field step and the hash equal the single-flip relax's.
//
// The max-tree over the keys is kept as an upper bound: keys that grow are pushed
// up with atomic maxima, keys that shrink leave their ancestors stale, and the
// candidate descent rebuilds every node it expands from its children.
//
// One thread-block cluster of NC CTAs per simulation and field step. The leader
// (rank 0) holds the round's state and the upper tree levels in its shared memory,
// chooses the threshold, descends the upper levels, sorts and tests the candidates
// and finds the prefix; all CTAs together expand the lowest level into candidate
// islands, evaluate their exact values, flip the picks and flip back the rest
// (the others reach the leader's shared memory as distributed shared memory).
// Cluster barriers separate the phases; every decision that steers the control
// flow is read from the leader after a barrier, so all CTAs take the same path.
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "fs_common.cuh"
#include "fs_kernels.h"
#include "fs_update.cuh"

namespace fs {

namespace {

constexpr int kMT = 512;          // threads of a multi-flip relax CTA
constexpr int kMW = kMT / 32;
constexpr int kCandCap = 1024;    // candidate islands per round
constexpr int kPickCap = 256;     // picks tested per round
constexpr int kSelMax = 8192;     // threshold chosen on the lowest level with at most this many nodes
constexpr int kSelPer = kSelMax / kMT;
constexpr int kM0 = 256;          // rank of the threshold node
constexpr int kHashT = kMT - 1;   // thread that folds the flips into the sequence hash
constexpr int kMaxIdle = 1024;    // consecutive iterations without a flip before ST_BOUNDS
constexpr int kCarry = 160;       // candidates carried below a round's last flip
// A step is handed to the single-flip relax after kLowRounds consecutive rounds of
// fewer than kPMin flips (a chain of flips that each make a neighbour the largest).
constexpr int kPMin = 8;
constexpr int kLowRounds = 4;

struct MultiShared {
    unsigned long long cv[kCandCap];  // candidates' exact values (double bits; 0 = none)
    int32_t ci[kCandCap];             // candidates' islands
    int32_t front[2][kCandCap];       // descent frontier
    float2 cpos[kPickCap];            // the first candidates' centres (FP32)
    unsigned long long xv[kPickCap];  // per pick: the best new value among its neighbours
    int32_t xi[kPickCap];             //   and its island
    int32_t cs[kPickCap];             // the picks' spins before the round
    int32_t hist[256];
    int32_t nf[2];
    int32_t nc, q, p, overflow, conflict_at, eligible;
    unsigned long long sel;
    int32_t sel_rem;
    int32_t lsh;                             // levels lsh.. are in shared memory
    unsigned long long* lp[kMaxLevels];      // base of each tree level (as this CTA sees it)
    // the leader's decisions for the whole cluster
    unsigned long long tkey;                 // this round's threshold
    int32_t cmd;                             // what the round does next (kCmd*)
    int32_t f0;                              // buffer of the level-0 nodes to expand
    int32_t nl;                              // candidate islands found
    int32_t stop;                            // 1: the relax of this launch ends after the round
};

constexpr int32_t kCmdExpand = 0;  // expand the level-0 nodes in front[f0]
constexpr int32_t kCmdCommit = 1;  // the picks are ready (q in S.q)
constexpr int32_t kCmdRetry = 2;   // nothing to flip yet: the leader starts again
constexpr int32_t kCmdStop = 3;    // the relax of this launch is over

// Tree levels: the upper ones (from lsh up) are copied into shared memory for the
// whole launch (the next sweep rebuilds the tree in global memory), the lower ones
// stay in global memory and are read through L2.
__device__ __forceinline__ unsigned long long lvl_load(const MultiShared& S, int lev,
                                                       int64_t idx) {
    return lev >= S.lsh ? S.lp[lev][idx] : __ldcg(S.lp[lev] + idx);
}

__device__ __forceinline__ bool before(unsigned long long va, int32_t ia, unsigned long long vb,
                                       int32_t ib) {
    return va > vb || (va == vb && ia < ib);
}

// The M-th largest key among the nodes of level `lev` (all nodes, stale ones too),
// by a radix selection over the 64-bit values, eight bits a pass. CTA-wide.
__device__ unsigned long long select_threshold(const Inst& I, int lev, int M, MultiShared& S) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int cnt = I.lvl_n[lev];
    unsigned long long v[kSelPer];
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        const int c = tid + u * kMT;
        v[u] = c < cnt ? lvl_load(S, lev, c) : 0ull;
    }
    if (M > cnt) M = cnt;
    if (tid == 0) {
        S.sel = 0ull;
        S.sel_rem = M;
    }
    unsigned long long mask = 0ull;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = tid; b < 256; b += kMT) S.hist[b] = 0;
        __syncthreads();
        const unsigned long long pre = S.sel;
#pragma unroll
        for (int u = 0; u < kSelPer; ++u)
            if (tid + u * kMT < cnt && (v[u] & mask) == pre)
                atomicAdd(&S.hist[(int)((v[u] >> shift) & 255ull)], 1);
        __syncthreads();
        if (tid < 32) {
            // lane l holds digits 255 - 8l .. 248 - 8l (descending)
            int h[8], sum = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                h[u] = S.hist[255 - 8 * lane - u];
                sum += h[u];
            }
            int incl = sum;  // inclusive prefix over lanes (from the top digit down)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - sum;
            const int rem = S.sel_rem;
            const bool here = excl < rem && rem <= incl;
            const unsigned who = __ballot_sync(0xffffffffu, here);
            if (here) {
                int acc = excl, d = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (acc + h[u] >= rem) {
                        d = 255 - 8 * lane - u;
                        break;
                    }
                    acc += h[u];
                }
                S.sel = pre | ((unsigned long long)d << shift);
                S.sel_rem = rem - acc;
            }
            if (who == 0u && lane == 0) S.sel_rem = 0;  // (fewer values than M: keep the prefix)
        }
        mask |= 255ull << shift;
        __syncthreads();
    }
    return S.sel;
}

// A key that grew is pushed up with atomic maxima, on every level below the root
// (the descent always expands the root's children, so the root is never read and
// every key needs no atomic on its one node): reductions that do not wait for the
// old value on the global levels; on the levels in shared memory (the one-CTA
// launch) the old value the atomic returns stops the push at the first node that
// already held the key (its ancestors hold it too once the phase's pushes are done).
__device__ __forceinline__ void push_up(const MultiShared& S, int nlev, int64_t i,
                                        unsigned long long nk) {
    const int top = nlev > 1 ? nlev - 1 : 1;  // levels 0 .. top - 1
    int64_t node = i;
    for (int lev = 0; lev < top; ++lev) {
        node >>= 5;
        unsigned long long* a = S.lp[lev] + node;
        if (lev < S.lsh) {
            atomicMax(a, nk);
        } else if (atomicMax(a, nk) >= nk) {
            break;
        }
    }
}

// The leader descends from the root to the level-0 nodes (the parents of the
// keys) whose value reaches tkey (>= 1), rebuilding each expanded node from its
// children; the nodes go to S.front[result] (S.nf[result] of them). Returns the
// buffer, or -1 when more than kCandCap nodes of a level reach tkey. With a single
// level the root is the one level-0 node. CTA-wide.
__device__ int descend_upper(const Inst& I, unsigned long long tkey, MultiShared& S) {
    constexpr int kB = 4;  // frontier nodes whose children a warp loads together
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int r = I.nlev - 1;
    if (tid == 0) {  // (the root's value is not kept: its children are always expanded)
        S.front[0][0] = 0;
        S.nf[0] = 1;
    }
    __syncthreads();
    int cur = 0;
    for (int lev = r; lev >= 1; --lev) {
        const int nf = S.nf[cur];
        if (tid == 0) S.nf[cur ^ 1] = 0;
        __syncthreads();
        const int64_t lim = I.lvl_n[lev - 1];
        for (int f0 = wid * kB; f0 < nf; f0 += kMW * kB) {
            int64_t node[kB];
            unsigned long long v[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {  // every load in flight together
                node[u] = f0 + u < nf ? (int64_t)S.front[cur][f0 + u] : -1;
                const int64_t c = (node[u] << 5) + lane;
                v[u] = node[u] >= 0 && c < lim ? lvl_load(S, lev - 1, c) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                if (node[u] < 0) break;
                const int64_t c = (node[u] << 5) + lane;
                // (a node is never below its children: pushes raise every ancestor,
                // repairs set a node to its children's maximum; so the maximum can
                // be stored without reading the node first)
                const unsigned long long m = warp_max_key(v[u]);
                if (lane == 0) S.lp[lev][node[u]] = m;
                const bool hit = v[u] != 0ull && v[u] >= tkey;
                const unsigned msk = __ballot_sync(0xffffffffu, hit);
                int base = 0;
                if (lane == 0 && msk) base = atomicAdd(&S.nf[cur ^ 1], __popc(msk));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int pos = base + __popc(msk & lt);
                if (hit && pos < kCandCap) S.front[cur ^ 1][pos] = (int32_t)c;
            }
        }
        __syncthreads();
        if (S.nf[cur ^ 1] > kCandCap) return -1;
        cur ^= 1;
    }
    return cur;
}

// Every CTA of the cluster: the level-0 nodes L->front[L->f0] expanded into the
// keys that reach L->tkey, appended to L->ci (L->nl counts them, past kCandCap
// too); each node is rebuilt from its keys. Warps of all CTAs share the nodes.
template <int NC>
__device__ void expand_leaves(const Inst& I, MultiShared* L, const MultiShared& S, int rank) {
    constexpr int kB = 8;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int gw = rank * kMW + wid;
    const int f0 = L->f0;
    const int nf = L->nf[f0];
    const unsigned long long tkey = L->tkey;
    for (int fb = gw * kB; fb < nf; fb += NC * kMW * kB) {
        int64_t node[kB];
        unsigned long long v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            node[u] = fb + u < nf ? (int64_t)L->front[f0][fb + u] : -1;
            const int64_t c = (node[u] << 5) + lane;
            v[u] = node[u] >= 0 && c < I.n ? __ldcg(&I.key32[c]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (node[u] < 0) break;
            const int64_t c = (node[u] << 5) + lane;
            const unsigned long long m = warp_max_key(v[u]);
            if (lane == 0) S.lp[0][node[u]] = m;
            const bool hit = v[u] != 0ull && v[u] >= tkey;
            const unsigned msk = __ballot_sync(0xffffffffu, hit);
            int base = 0;
            if (lane == 0 && msk) base = atomicAdd(&L->nl, __popc(msk));
            base = __shfl_sync(0xffffffffu, base, 0);
            const int pos = base + __popc(msk & lt);
            if (hit && pos < kCandCap) L->ci[pos] = (int32_t)c;
        }
    }
}

// Sorts S.cv / S.ci[0 .. n) into "before" order: up to kRankMax entries by rank
// (every entry counts those that go before it; keys are distinct), more by a
// bitonic network over the next power of two (padding entries sort last).
constexpr int kRankMax = 256;
__device__ void sort_candidates(MultiShared& S, int n, int n2) {
    if (n <= kRankMax) {
        unsigned long long v[kRankMax / kMT + 1];
        int32_t ix[kRankMax / kMT + 1], rk[kRankMax / kMT + 1];
        int m = 0;
        for (int t = threadIdx.x; t < n; t += kMT, ++m) {
            v[m] = S.cv[t];
            ix[m] = S.ci[t];
            int r = 0;
            for (int u = 0; u < n; ++u) r += before(S.cv[u], S.ci[u], v[m], ix[m]) ? 1 : 0;
            rk[m] = r;
        }
        __syncthreads();
        for (int u = 0; u < m; ++u) {
            S.cv[rk[u]] = v[u];
            S.ci[rk[u]] = ix[u];
        }
        __syncthreads();
        return;
    }
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < n2; t += kMT) {
                const int o = t ^ j;
                if (o > t) {
                    const bool up = (t & k) == 0;
                    const unsigned long long va = S.cv[t], vb = S.cv[o];
                    const int32_t ia = S.ci[t], ib = S.ci[o];
                    const bool swap = up ? before(vb, ib, va, ia) : before(va, ia, vb, ib);
                    if (swap) {
                        S.cv[t] = vb;
                        S.cv[o] = va;
                        S.ci[t] = ib;
                        S.ci[o] = ia;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Flips island k to spin snew (its neighbours' exact sums change by 2 snew times
// their coefficients) with every new value stored; warp-wide. Returns, on every
// lane, the best new value among the neighbours (FS_FP64: exact; FP32 path: the
// upper bound of the key) and its island.
template <int PREC>
__device__ void flip_warp(const Inst& I, const MultiShared& S, int64_t k, int snew, uint32_t step,
                          unsigned long long* xv, int32_t* xi) {
    const int lane = threadIdx.x & 31;
    const IslandRec rk = rec_load(I, k);
    const int64_t r0 = (int64_t)rk.rowq << 2, r1 = r0 + ((int64_t)rk.rowlenq << 2);
    unsigned long long bv = 0ull;
    int32_t bi = 0x7fffffff;
    // two entries a lane at a time: both updates are computed (loads in flight
    // together) before either is stored
    // k's own update (its field unchanged, its spin flipped) takes the slot of the
    // row's last entry when that is padding (a self-entry of zero weight, which
    // gives exactly that update), else it follows the row
    const bool own_in_row = r1 > r0 && __ldg(&I.col[r1 - 1]) == (int32_t)k;
    for (int64_t e0 = r0 + lane; e0 < r1; e0 += 64) {
        Upd u[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t e = e0 + 32 * h;
            u[h].i = -1;
            if (e < r1) {
                const int32_t i = __ldg(&I.col[e]);
                const long long dp = __ldg(&I.pq64[e].x), dq = __ldg(&I.qt64[e]);
                int dp32 = 0, dq32 = 0;
                if constexpr (PREC == 1) {
                    dp32 = __ldg(&I.pq32[e].x);
                    dq32 = __ldg(&I.qt32[e]);
                }
                if (i != (int32_t)k)
                    u[h] = compute_update<PREC, true>(I, i, snew, dp, dq, dp32, dq32, step);
                else if (e == r1 - 1)
                    u[h] = compute_update<PREC, true>(I, k, snew, 0, 0, 0, 0, step, snew);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (u[h].i < 0) continue;
            const int64_t i = u[h].i;
            if (i == k) I.s[k] = (int8_t)snew;
            I.h64[i] = u[h].h;
            rec_store_dyn(I, i, u[h].g, u[h].lo, u[h].s);
            I.key64[i] = u[h].x;
            I.key32[i] = u[h].nk;
            if (u[h].nk > u[h].old) push_up(S, I.nlev, i, u[h].nk);
            unsigned long long val = 0ull;
            if constexpr (PREC == 0) {
                val = u[h].x > 0.0 ? (unsigned long long)__double_as_longlong(u[h].x) : 0ull;
            } else {
                val = u[h].nk ? (unsigned long long)__double_as_longlong((double)key32_hi(u[h].nk))
                              : 0ull;
            }
            if (i != k && val && before(val, (int32_t)i, bv, bi)) {
                bv = val;
                bi = (int32_t)i;
            }
        }
    }
    if (!own_in_row && lane == 0) {  // k itself: its field is unchanged, its spin is not
        I.s[k] = (int8_t)snew;
        const Upd u = compute_update<PREC, true>(I, k, snew, 0, 0, 0, 0, step, snew);
        I.h64[k] = u.h;
        rec_store_dyn(I, k, u.g, u.lo, u.s);
        I.key64[k] = u.x;
        I.key32[k] = u.nk;
        if (u.nk > u.old) push_up(S, I.nlev, k, u.nk);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov && before(ov, oi, bv, bi)) {
            bv = ov;
            bi = oi;
        }
    }
    *xv = bv;
    *xi = bi;
}

// The exact best flippable island of the whole array by a full scan (every key
// above zero evaluated exactly), for rounds whose candidate set cannot be held;
// S.ci[0] / S.cv[0] receive it (S.nc = 0 when none). CTA-wide.
template <int PREC>
__device__ void scan_best(const Inst& I, uint32_t step, MultiShared& S) {
    const int tid = threadIdx.x;
    unsigned long long bv = 0ull;
    int32_t bi = 0x7fffffff;
    for (int64_t i = tid; i < I.n; i += kMT) {
        if (__ldcg(&I.key32[i]) == 0ull) continue;
        const double v = exact_value<PREC>(I, i, step);
        if (!(v > 0.0)) {
            I.key32[i] = 0ull;
            continue;
        }
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        if (before(b, (int32_t)i, bv, bi)) {
            bv = b;
            bi = (int32_t)i;
        }
    }
    S.cv[tid] = bv;
    S.ci[tid] = bi;
    __syncthreads();
    for (int w = kMT / 2; w > 0; w >>= 1) {
        if (tid < w && S.cv[tid + w] && before(S.cv[tid + w], S.ci[tid + w], S.cv[tid], S.ci[tid])) {
            S.cv[tid] = S.cv[tid + w];
            S.ci[tid] = S.ci[tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) S.nc = S.cv[0] ? 1 : 0;
    __syncthreads();
}

template <int PREC, int NC>
__global__ void __launch_bounds__(kMT, 1)
    k_relax_multi(const Inst* __restrict__ tab, const int32_t* __restrict__ work, int n_work,
                  int smem_levels) {
    namespace cg = cooperative_groups;
    __shared__ MultiShared S;
    extern __shared__ unsigned long long sm_levels[];
    int rank = 0;
    MultiShared* L = &S;  // the leader's state, as this CTA reaches it
    unsigned long long* lead_levels = sm_levels;
    if constexpr (NC > 1) {
        cg::cluster_group cl = cg::this_cluster();
        rank = (int)cl.block_rank();
        if (rank != 0) {
            L = cl.map_shared_rank(&S, 0);
            lead_levels = cl.map_shared_rank(sm_levels, 0);
        }
    }
    auto csync = [&]() {
        if constexpr (NC > 1)
            cg::this_cluster().sync();
        else
            __syncthreads();
    };
    const bool leader = rank == 0;
    const Inst& I = tab[work[blockIdx.x / NC]];
    InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;  // (the same for every CTA)
    const uint32_t step = I.step0 + (uint32_t)t;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    // the upper tree levels that fit smem_levels bytes, from the top down, in the
    // leader's shared memory (the host sizes the launch by the same rule)
    if (tid == 0) {
        int64_t used = 0;
        int lsh = I.nlev;
        for (int lev = I.nlev - 1; lev >= 0; --lev) {
            const int64_t b = 8 * (int64_t)I.lvl_n[lev];
            if (used + b > smem_levels) break;
            used += b;
            lsh = lev;
        }
        S.lsh = lsh;
        int64_t off = 0;
        for (int lev = kMaxLevels - 1; lev >= 0; --lev) {
            if (lev >= I.nlev) {
                S.lp[lev] = nullptr;
            } else if (lev >= lsh) {
                S.lp[lev] = lead_levels + off;
                off += I.lvl_n[lev];
            } else {
                S.lp[lev] = I.tree + I.lvl_off[lev];
            }
        }
    }
    __syncthreads();
    if (leader)
        for (int lev = S.lsh; lev < I.nlev; ++lev)
            for (int q = tid; q < I.lvl_n[lev]; q += kMT)
                S.lp[lev][q] = __ldcg(&I.tree[I.lvl_off[lev] + q]);
    csync();

    int lsel = 0;
    while (lsel < I.nlev - 1 && I.lvl_n[lsel] > kSelMax) ++lsel;

    // the leader's round state (the same in every leader thread)
    int64_t flips = 0;
    int32_t status = ST_OK;
    uint64_t hash = leader && tid == kHashT ? st->hash : 0ull;
    const int64_t flips_before = st->n_flips;
    const int64_t max_flips = I.max_flips;
    const int m0 = max(1, min(kM0, I.lvl_n[lsel] / 8));  // rank of the threshold node
    int M = m0;
    int idle = 0;
    int64_t rounds = 0, idle_total = 0;
    int low = 0;
    bool handoff = false;
    bool need_scan = false;
    bool was_carried = false, was_forced = false;
    unsigned long long carry = 0ull;   // a threshold from the previous round's candidates
    unsigned long long forced = 0ull;  // a threshold set by the previous iteration

    for (;;) {
        // ---- A (leader): the threshold and the level-0 nodes that reach it --------
        if (leader) {
            int32_t cmd = kCmdExpand;
            if (++idle > kMaxIdle) {
                status = ST_BOUNDS;
                cmd = kCmdStop;
            } else if (need_scan) {  // a candidate set too large for any threshold
                need_scan = false;
                M = m0;
                scan_best<PREC>(I, step, S);
                if (S.nc == 0) {
                    cmd = kCmdStop;
                } else {
                    const int64_t allowed = max_flips - flips;
                    if (allowed <= 0) {
                        status = ST_NOT_CONVERGED;
                        cmd = kCmdStop;
                    } else {
                        if (tid == 0) {
                            S.q = 1;
                            S.cs[0] = rec_load(I, S.ci[0]).s;
                        }
                        cmd = kCmdCommit;
                    }
                }
            } else {
                ++idle_total;
                unsigned long long tkey = 1ull;
                was_forced = forced != 0ull;
                was_carried = !was_forced && carry != 0ull;
                if (was_forced) {
                    tkey = forced;
                    forced = 0ull;
                } else if (was_carried) {
                    tkey = carry;
                    carry = 0ull;
                } else {
                    const unsigned long long sel = select_threshold(I, lsel, M, S);
                    // lowered by 2^-18 (relative) so that the node's own island, whose
                    // exact value lies within its key's band, counts as reaching it
                    const float hi = __uint_as_float((uint32_t)(sel >> 32));
                    const float lo = __fmul_rd(hi, 1.0f - 0x1.0p-18f);
                    tkey = sel ? ((unsigned long long)__float_as_uint(lo) << 32) : 1ull;
                    if (tkey == 0ull) tkey = 1ull;
                }
                const int buf = descend_upper(I, tkey, S);
                if (buf < 0) {  // too many nodes reach it: a higher threshold, or a scan
                    if (!was_carried) {
                        if (M > 1 && !was_forced)
                            M >>= 1;
                        else
                            need_scan = true;
                    }
                    cmd = kCmdRetry;
                } else if (S.nf[buf] == 0) {
                    if (tkey == 1ull) {
                        cmd = kCmdStop;  // no key above zero: the relax is done
                    } else {
                        M = m0;  // the threshold came from stale nodes, repaired on the way
                        cmd = kCmdRetry;
                    }
                } else if (tid == 0) {
                    S.f0 = buf;
                    S.tkey = tkey;
                    S.nl = 0;
                }
            }
            if (tid == 0) S.cmd = cmd;
        }
        csync();
        int32_t cmd = L->cmd;
        if (cmd == kCmdStop) break;
        if (cmd == kCmdRetry) continue;
        if (cmd == kCmdExpand) {
            // ---- B (all): the candidate islands ------------------------------------
            expand_leaves<NC>(I, L, S, rank);
            csync();
            const int nl = L->nl;
            if (nl > kCandCap) {
                if (leader && !was_carried) {
                    if (M > 1 && !was_forced)
                        M >>= 1;
                    else
                        need_scan = true;
                }
                continue;
            }
            if (nl == 0) {
                if (L->tkey == 1ull) break;  // (cannot happen: its parent reached it)
                if (leader) M = m0;
                continue;
            }
            // ---- C (all): exact values; islands found not flippable are demoted ----
            int n2 = 1;
            while (n2 < nl) n2 <<= 1;
            for (int c = rank * kMT + tid; c < n2; c += NC * kMT) {
                if (c < nl) {
                    const int32_t i = L->ci[c];
                    const double v = exact_value<PREC>(I, i, step);
                    if (v > 0.0) {
                        if constexpr (PREC == 1) I.key32[i] = key32_of(__double2float_ru(v), i);
                        L->cv[c] = (unsigned long long)__double_as_longlong(v);
                    } else {
                        I.key32[i] = 0ull;
                        L->cv[c] = 0ull;
                    }
                } else {
                    L->cv[c] = 0ull;
                    L->ci[c] = 0x7fffffff;
                }
            }
            csync();
            // ---- D (leader): order, threshold test, independence ---------------------
            if (leader) {
                if (tid == 0) S.nc = nl;
                sort_candidates(S, nl, n2);
                // (a) a pick must beat every island below the threshold: (v, i) no
                // later than (tau, tau_index) in "before" order
                const unsigned long long tkey = S.tkey;
                const double tau = (double)__uint_as_float((uint32_t)(tkey >> 32));
                const uint32_t tau_i = key32_idx(tkey);
                const unsigned long long tb = (unsigned long long)__double_as_longlong(tau);
                if (tid == 0) {
                    S.eligible = 0;
                    S.conflict_at = kPickCap;
                }
                __syncthreads();
                for (int c = tid; c < min(nl, kPickCap); c += kMT) {
                    const unsigned long long v = S.cv[c];
                    const bool ok = v != 0ull && (v > tb || (v == tb && (uint32_t)S.ci[c] <= tau_i));
                    if (ok) atomicMax(&S.eligible, c + 1);  // eligibility is a prefix of the order
                }
                __syncthreads();
                int q = S.eligible;
                int32_t c2 = kCmdCommit;
                if (q == 0) {
                    if (S.cv[0] == 0ull) {  // none of them is flippable (all demoted)
                        M = m0;
                    } else {
                        // every candidate lies below the threshold: the next iteration
                        // takes the best one's value (rounded down) as the threshold, so
                        // that every island that could beat it is a candidate
                        const float v0 =
                            __double2float_rd(__longlong_as_double((long long)S.cv[0]));
                        const unsigned long long tk = (unsigned long long)__float_as_uint(v0) << 32;
                        forced = tk > 0ull ? tk : 1ull;
                    }
                    c2 = kCmdRetry;
                } else {
                    // (b) picks more than twice the cutoff apart
                    for (int c = tid; c < q; c += kMT) {
                        const double2 pc = __ldg(&I.pos[S.ci[c]]);
                        S.cpos[c] = make_float2(__double2float_rn(pc.x), __double2float_rn(pc.y));
                    }
                    __syncthreads();
                    // pair (c, j), j < c: warp per row c, lanes over j; in FP32 against a
                    // radius widened by the rounding of the centres (I.rconf2f)
                    for (int c = 1 + wid; c < q; c += kMW) {
                        if (c >= S.conflict_at) break;
                        const float2 a = S.cpos[c];
                        bool hit = false;
                        for (int j = lane; j < c; j += 32) {
                            const float dx = __fsub_rn(a.x, S.cpos[j].x);
                            const float dy = __fsub_rn(a.y, S.cpos[j].y);
                            hit = hit || __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= I.rconf2f;
                        }
                        if (__any_sync(0xffffffffu, hit)) {
                            if (lane == 0) atomicMin(&S.conflict_at, c);
                            break;
                        }
                    }
                    __syncthreads();
                    q = min(q, S.conflict_at);
                    // the step's flip budget
                    const int64_t allowed = max_flips - flips;
                    if (allowed <= 0) {
                        status = ST_NOT_CONVERGED;
                        c2 = kCmdStop;
                    } else if (q > allowed) {
                        q = (int)allowed;
                    }
                    for (int c = tid; c < q; c += kMT) S.cs[c] = rec_load(I, S.ci[c]).s;
                    if (tid == 0) S.q = q;
                }
                if (tid == 0) S.cmd = c2;
            }
            csync();
            cmd = L->cmd;
            if (cmd == kCmdStop) break;
            if (cmd == kCmdRetry) continue;
        }
        // ---- E (all): flip the picks together (disjoint neighbourhoods) --------------
        {
            const int q = L->q;
            for (int j = rank + NC * wid; j < q; j += NC * kMW) {
                unsigned long long xv;
                int32_t xi;
                flip_warp<PREC>(I, S, L->ci[j], -L->cs[j], step, &xv, &xi);
                if (lane == 0) {
                    L->xv[j] = xv;
                    L->xi[j] = xi;
                }
            }
        }
        csync();
        // ---- F (leader): the longest prefix no earlier pick's neighbour overtakes ----
        if (leader) {
            const int q = S.q;
            // warp 0, 32 picks at a time: the best of the earlier picks' neighbour
            // values (an exclusive prefix maximum), carried between chunks
            if (wid == 0) {
                unsigned long long cv_ = 0ull;  // carried maximum
                int32_t ci_ = 0x7fffffff;
                int p = q;
                for (int j0 = 0; j0 < q; j0 += 32) {
                    const int j = j0 + lane;
                    unsigned long long xv = j < q ? S.xv[j] : 0ull;
                    int32_t xi = j < q ? S.xi[j] : 0x7fffffff;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {  // inclusive prefix maximum
                        const unsigned long long ov = __shfl_up_sync(0xffffffffu, xv, o);
                        const int32_t oi = __shfl_up_sync(0xffffffffu, xi, o);
                        if (lane >= o && ov && (!xv || before(ov, oi, xv, xi))) {
                            xv = ov;
                            xi = oi;
                        }
                    }
                    unsigned long long ev = __shfl_up_sync(0xffffffffu, xv, 1);
                    int32_t ei = __shfl_up_sync(0xffffffffu, xi, 1);
                    if (lane == 0) {
                        ev = 0ull;
                        ei = 0x7fffffff;
                    }
                    if (cv_ && (!ev || before(cv_, ci_, ev, ei))) {
                        ev = cv_;
                        ei = ci_;
                    }
                    const bool fail = j < q && j > 0 && ev && !before(S.cv[j], S.ci[j], ev, ei);
                    const unsigned fm = __ballot_sync(0xffffffffu, fail);
                    if (fm) {
                        p = j0 + __ffs(fm) - 1;
                        break;
                    }
                    const unsigned long long lv = __shfl_sync(0xffffffffu, xv, 31);
                    const int32_t li = __shfl_sync(0xffffffffu, xi, 31);
                    if (lv && (!cv_ || before(lv, li, cv_, ci_))) {
                        cv_ = lv;
                        ci_ = li;
                    }
                }
                if (lane == 0) S.p = p;
            }
            __syncthreads();
            const int p = S.p;
            // log and hash, in the order of the picks
            for (int j = tid; j < p; j += kMT) {
                const int64_t qq = flips_before + flips + j;
                if (I.log_spin && qq < I.log_cap) {
                    I.log_step[qq] = step;
                    I.log_spin[qq] = (uint32_t)S.ci[j];
                }
            }
            if (tid == kHashT)
                for (int j = 0; j < p; ++j) hash = fnv_flip(hash, step, (uint32_t)S.ci[j]);
            flips += p;
            idle = 0;
            --idle_total;
            ++rounds;
            M = m0;
            low = p < kPMin ? low + 1 : 0;
            if (low >= kLowRounds) handoff = true;
            // the next round's threshold: the value kCarry places below this round's
            // last flip among its candidates (most of them are still unflipped), so
            // that the next candidate set is about that large
            {
                const int nc = S.nc;
                const int r = min(nc - 1, p + kCarry);
                const unsigned long long vr = r > p ? S.cv[r] : 0ull;
                if (vr) {
                    const float f = __fmul_rd(__double2float_rd(__longlong_as_double((long long)vr)),
                                              1.0f - 0x1.0p-18f);
                    carry = (unsigned long long)__float_as_uint(f) << 32;
                }
            }
            if (tid == 0) S.stop = handoff ? 1 : 0;
        }
        csync();
        // ---- G (all): flip the rest back ---------------------------------------------
        {
            const int q = L->q, p = L->p;
            for (int j = p + rank + NC * wid; j < q; j += NC * kMW) {
                unsigned long long xv;
                int32_t xi;
                flip_warp<PREC>(I, S, L->ci[j], L->cs[j], step, &xv, &xi);
            }
        }
        csync();
        if (L->stop) break;
    }
    csync();  // (no CTA leaves while another may still reach the leader's memory)
    if (!leader) return;
    if (tid == kHashT) st->hash = hash;
    if (handoff && status == ST_OK) {
        // the single-flip relax reads the whole tree from global memory: the levels
        // kept here (raised by this launch's pushes) go back there
        for (int lev = S.lsh; lev < I.nlev; ++lev)
            for (int q = tid; q < I.lvl_n[lev]; q += kMT) I.tree[I.lvl_off[lev] + q] = S.lp[lev][q];
    }
    __syncthreads();
    if (tid == 0) {
        st->rounds += rounds;
        st->idle += idle_total;
        st->n_flips = flips_before + flips;
        if (status != ST_OK) st->status = status;
        if (handoff && status == ST_OK) {  // the single-flip relax finishes step t
            st->handoff = 1;
            st->step_flips = flips;
        } else {
            if (I.flips_per_step) I.flips_per_step[t] = flips;
            st->init = 0;
            st->t = t + 1;
        }
    }
}

}  // namespace

// Dynamic shared memory of a multi-flip relax CTA: the tree levels above the keys
// that fit 128 KiB, counted from the top down (the kernel places them the same way).
int relax_multi_smem(int64_t n) {
    const int64_t cap = 128 * 1024;
    std::vector<int64_t> lv;
    for (int64_t cnt = (n + 31) / 32;; cnt = (cnt + 31) / 32) {
        lv.push_back(cnt);
        if (cnt == 1) break;
    }
    int64_t used = 0;
    for (size_t q = lv.size(); q-- > 0;) {
        if (used + 8 * lv[q] > cap) break;
        used += 8 * lv[q];
    }
    return (int)used;
}

namespace {

constexpr int kNC = 8;  // CTAs of a multi-flip relax cluster

template <int PREC, int NC>
cudaError_t launch_multi(const RelaxLaunch& L, int smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(L.n_work * NC));
    cfg.blockDim = dim3(kMT);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_relax_multi<PREC, NC>, L.tab, L.work, L.n_work, smem);
}

template <int PREC, int NC>
cudaError_t set_multi_smem(int smem) {
    return cudaFuncSetAttribute(k_relax_multi<PREC, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem);
}

// Whether a cluster of kNC CTAs with this much dynamic shared memory fits the GPU.
template <int PREC>
bool cluster_fits(int smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kNC);
    cfg.blockDim = dim3(kMT);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kNC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, k_relax_multi<PREC, kNC>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters >= 1;
}

}  // namespace

cudaError_t launch_relax_multi(const RelaxLaunch& L, cudaStream_t st) {
    if (L.n_work == 0) return cudaSuccess;
    // per precision: the dynamic shared memory set so far, and whether the cluster
    // of that size fits (checked once per size, before any launch is captured)
    static std::atomic<int> set_bytes[2] = {{-1}, {-1}};
    static std::atomic<int> use_cluster[2] = {{0}, {0}};
    static std::mutex mu;
    const int k = L.prec == 1 ? 1 : 0;
    const int smem = L.smem_multi;
    if (set_bytes[k].load() < smem) {
        std::lock_guard<std::mutex> g(mu);
        if (set_bytes[k].load() < smem) {
            cudaError_t e = k ? set_multi_smem<1, 1>(smem) : set_multi_smem<0, 1>(smem);
            if (e == cudaSuccess) e = k ? set_multi_smem<1, kNC>(smem) : set_multi_smem<0, kNC>(smem);
            if (e != cudaSuccess) return e;
            use_cluster[k].store((k ? cluster_fits<1>(0) : cluster_fits<0>(0)) ? 1 : 0);
            set_bytes[k].store(smem);
        }
    }
    // A cluster keeps the whole tree in global memory (every CTA pushes keys into
    // it); the one-CTA launch keeps the upper levels in its shared memory.
    if (use_cluster[k].load())
        return k ? launch_multi<1, kNC>(L, 0, st) : launch_multi<0, kNC>(L, 0, st);
    return k ? launch_multi<1, 1>(L, smem, st) : launch_multi<0, 1>(L, smem, st);
}

}  // namespace fs
