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
// (a) and (b) are checked before the round's flips; the updates of all picks that
// pass them are computed together (their neighbourhoods are disjoint), (c) is
// checked on the new values, and only the prefix before the first pick that fails
// is stored. A round therefore always flips at least one island, and the flip
// sequence, the flips per field step and the hash equal the single-flip relax's.
//
// The max-tree over the keys is kept as an upper bound: keys that grow are pushed
// up with atomic maxima (also those of picks that are not stored), keys that
// shrink leave their ancestors stale, and every node the candidate search expands
// is rebuilt from its children.
//
// One thread-block cluster of NC CTAs per simulation and field step. A round is
// three cluster-wide phases, each ended by a cluster barrier:
//   expand:  all CTAs expand the frontier the leader chose into the candidate
//            islands and evaluate each one exactly (value, spin, row, centre);
//   compute: all CTAs compute the picks' neighbour updates into shared memory, one
//            warp a pick, and push the keys that grow up the tree;
//   store:   the updates of the picks before the prefix are stored.
// The leader (rank 0) holds the round's state in its shared memory and does the
// serial work alone between the phases: after an expansion it orders and tests the
// candidates and chooses the picks; after the computation it finds the prefix and
// plans the next round (its threshold from one tree level, loaded whole, and the
// frontier of nodes that reach it). The other CTAs reach the leader's shared memory
// as distributed shared memory; every decision that steers the control flow is read
// from the leader after a barrier, so all CTAs take the same path.
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "fs_common.cuh"
#include "fs_kernels.h"
#include "fs_update.cuh"

namespace fs {

namespace {

constexpr int kMT = 512;          // threads of a multi-flip relax CTA
constexpr int kMW = kMT / 32;
constexpr int kCandCap = 1024;    // candidate islands per round
constexpr int kPickCap = 240;     // picks tested per round (one a warp of the cluster's 15
                                  // CTAs besides the leader, a cluster of 16)
constexpr int kSelMax = 4096;     // thresholds are chosen on the lowest level with at most this many nodes
constexpr int kSelPer = kSelMax / kMT;
constexpr int kM0 = 512;          // rank of the threshold node
constexpr int kHashT = kMT - 1;   // thread that folds the flips into the sequence hash
constexpr int kMaxIdle = 1024;    // consecutive iterations without a flip before ST_BOUNDS
constexpr int kCarry = 160;       // candidates carried below a round's last flip
// A step is handed to the single-flip relax after kLowRounds consecutive rounds of
// fewer than kPMin flips (a chain of flips that each make a neighbour the largest).
constexpr int kPMin = 4;
constexpr int kLowRounds = 4;
constexpr int kClsSh = 32;        // angle classes whose external field is read from shared memory
constexpr int kRankMax = kMT / 2;  // candidates sorted by rank (more: by merging)
constexpr int kHashQ = 2 * kPickCap;  // flips waiting to be folded into the sequence hash

// One candidate island as its exact evaluation found it.
struct __align__(16) Cand {
    unsigned long long v;  // exact value (double bits; 0 = not flippable)
    int32_t i;
    uint32_t rowq;         // its neighbour row (first entry / 4, entries / 4)
    float2 pos;            // centre (FP32)
    uint16_t rowlenq;
    int16_t s;             // spin
    int32_t pad;
};

// One pick of a round: the island, its spin before the round and its row.
struct __align__(16) Pick {
    int32_t i;
    uint32_t rowq;
    uint16_t rowlenq;
    int16_t s;
    int32_t eager;  // 1: flipped (stored) at once, to be flipped back if after the prefix
};

struct MultiShared {
    Cand cand[kCandCap];              // candidates in the order found
    unsigned long long sv[kCandCap];  // candidates in "before" order: value,
    int32_t si[kCandCap];             //   island,
    int16_t so[kCandCap];             //   and slot in cand
    unsigned long long mv[kCandCap];  // the merge sort's second buffer
    int32_t mi[kCandCap];
    int16_t mo[kCandCap];
    float2 sp[kPickCap];              // the first candidates' centres, in that order
    int32_t front[2][kCandCap];       // frontier of the tree search
    int32_t loc[kCandCap];            // the candidate islands this CTA found
    Pick pk[kPickCap];                // the round's picks
    unsigned long long xv[kPickCap];  // per pick: the best new value among its neighbours
    int32_t xi[kPickCap];             //   and its island
    int32_t hist[256];
    unsigned long long wv[kMW];       // per warp: a prefix maximum and its island
    int32_t wi[kMW];
    int32_t hq[kHashQ];               // flips not yet in the hash, in order (leader)
    int32_t hq_n;
    double2 ext64[kClsSh];            // the step's external field per angle class
    float2 ext32[kClsSh];
    Inst inst;                        // this CTA's copy of the simulation's descriptor
    unsigned long long* lp[kMaxLevels];  // base of each tree level (global memory)
    int32_t nf[2];
    int32_t nloc, lbase;              // this CTA's candidates; their first slot
    int32_t nl;                       // candidate islands found (leader; past kCandCap too)
    int32_t nc, nz, q, p, conflict_at;
    int32_t sel_n, sel_d, sel_r;      // threshold selection: values, digit, rank left
    unsigned dmin[4], dmax[4];        //   digit range of each pass
    // the leader's decisions for the whole cluster
    unsigned long long tkey;          // this round's threshold
    int32_t cmd;                      // what the cluster does next (kCmd*)
    int32_t f_lev;                    // level of the frontier nodes to expand (0 or 1)
    int32_t f_buf;                    // their buffer in front
    int32_t next;                     // the command that follows the stores (kCmdPlan: the
                                      //   leader chooses it after them)
};

// Dynamic shared memory of a CTA: its state, then every warp's staging slots.
constexpr int kStageOff = (int)((sizeof(MultiShared) + 15) & ~(size_t)15);

constexpr int32_t kCmdExpand = 0;   // expand the frontier into candidates
constexpr int32_t kCmdCompute = 1;  // compute the picks' flips (q in S.q), then store the
                                    // prefix's (p in S.p)
constexpr int32_t kCmdStop = 2;     // the relax of this launch is over

__device__ __forceinline__ bool before(unsigned long long va, int32_t ia, unsigned long long vb,
                                       int32_t ib) {
    return va > vb || (va == vb && ia < ib);
}

// The two halves of a cluster barrier: this thread's writes so far are released to
// the cluster (arrive), and it waits until every thread of the cluster has arrived
// (wait, acquiring their writes). A thread waits before it arrives again.
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Appends the lanes' hits (island or node `c` where `hit`) to list[*cnt ...) (the
// count runs on past cap; entries past it are dropped). Warp-wide.
__device__ __forceinline__ void warp_append(bool hit, int32_t c, int32_t* list, int32_t* cnt,
                                            int cap) {
    const int lane = threadIdx.x & 31;
    const unsigned msk = __ballot_sync(0xffffffffu, hit);
    int base = 0;
    if (lane == 0 && msk) base = atomicAdd(cnt, __popc(msk));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int pos = base + __popc(msk & ((1u << lane) - 1u));
    if (hit && pos < cap) list[pos] = c;
}

// The upper half (the FP32 bound) of the M-th largest nonzero value v[u] (node
// tid + u kMT, cnt nodes; stale ones too), by a radix selection over those 32 bits,
// eight a pass; a pass in which every value still in the running has the same digit
// takes that digit without a histogram. Returns 0 when no value is nonzero.
// CTA-wide.
__device__ uint32_t select_threshold(const unsigned long long (&v)[kSelPer], int cnt, int M,
                                     MultiShared& S) {
    const int tid = threadIdx.x, lane = tid & 31;
    uint32_t h[kSelPer];
    int nn = 0;
#pragma unroll
    for (int u = 0; u < kSelPer; ++u) {
        h[u] = tid + u * kMT < cnt ? (uint32_t)(v[u] >> 32) : 0u;
        nn += h[u] != 0u ? 1 : 0;
    }
    if (tid == 0) {
        S.sel_n = 0;
        for (int q = 0; q < 4; ++q) {
            S.dmin[q] = 255u;
            S.dmax[q] = 0u;
        }
    }
    __syncthreads();
    nn = __reduce_add_sync(0xffffffffu, nn);
    if (lane == 0 && nn) atomicAdd(&S.sel_n, nn);
    __syncthreads();
    const int total = S.sel_n;
    if (total == 0) return 0u;
    int rem = min(M, total);  // the rank still to find among the values in the running
    uint32_t pre = 0u, mask = 0u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        unsigned dmin = 255u, dmax = 0u;
#pragma unroll
        for (int u = 0; u < kSelPer; ++u)
            if (h[u] != 0u && (h[u] & mask) == pre) {
                const unsigned d = (h[u] >> shift) & 255u;
                dmin = min(dmin, d);
                dmax = max(dmax, d);
            }
        dmin = __reduce_min_sync(0xffffffffu, dmin);
        dmax = __reduce_max_sync(0xffffffffu, dmax);
        if (lane == 0) {
            atomicMin(&S.dmin[pass], dmin);
            atomicMax(&S.dmax[pass], dmax);
        }
        for (int q = tid; q < 256; q += kMT) S.hist[q] = 0;
        __syncthreads();
        const unsigned gmin = S.dmin[pass], gmax = S.dmax[pass];
        if (gmin == gmax) {
            pre |= gmin << shift;
        } else {
#pragma unroll
            for (int u = 0; u < kSelPer; ++u)
                if (h[u] != 0u && (h[u] & mask) == pre) atomicAdd(&S.hist[(h[u] >> shift) & 255u], 1);
            __syncthreads();
            if (tid < 32) {
                // lane l holds digits 255 - 8l .. 248 - 8l (descending)
                int hh[8], sum = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    hh[u] = S.hist[255 - 8 * lane - u];
                    sum += hh[u];
                }
                int incl = sum;  // inclusive prefix over lanes (from the top digit down)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = incl - sum;
                if (excl < rem && rem <= incl) {  // (one lane: rem <= the values in the running)
                    int acc = excl, d = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (acc + hh[u] >= rem) {
                            d = 255 - 8 * lane - u;
                            break;
                        }
                        acc += hh[u];
                    }
                    S.sel_d = d;
                    S.sel_r = rem - acc;
                }
            }
            __syncthreads();
            pre |= (uint32_t)S.sel_d << shift;
            rem = S.sel_r;
        }
        mask |= 255u << shift;
    }
    return pre;
}

// A key that grew is pushed up with atomic maxima (reductions that do not wait for
// the old value) on every level below the root: the search never reads the root,
// and the single-flip relax that may take over reads only levels below it.
__device__ __forceinline__ void push_up(unsigned long long* const* lp, int nlev, int64_t i,
                                        unsigned long long nk) {
    const int top = nlev > 1 ? nlev - 1 : 1;  // levels 0 .. top - 1
    int64_t node = i;
    for (int lev = 0; lev < top; ++lev) {
        node >>= 5;
        atomicMax(lp[lev] + node, nk);
    }
}

// What one neighbour update writes: the island's exact sums, the changing half of
// its record and its keys, and whether its key grew (then it is pushed up the tree).
struct __align__(16) Stage {
    longlong2 h;
    unsigned long long nk;
    double x;
    int2 g;
    int32_t i;  // -1: none
    float lo;
    int32_t s;
    int32_t push;
};

constexpr int kSlots = 2;                 // slots a lane takes per pass (rows of up to 64 staged)
constexpr int kStageSlots = 32 * kSlots;  // a warp's staging slots (one pass)

// One pass over the slots e0, e0 + 32, ... (e0 = first + lane) of the flip of
// island k (row [.., r1)) to spin snew: each neighbour's exact sums change by
// 2 snew times their coefficients and its key is evaluated again; with `own`, k's
// own update (its field unchanged, its spin snew) takes the slot r1, just past the
// row; the row's padding (self-entries of zero weight) is skipped. Every load of
// the pass is in flight before any result is used; nothing is stored.
template <int PREC>
__device__ __forceinline__ void pass_compute(const Inst& I, int64_t k, int snew, int64_t e0,
                                             int64_t r1, bool own, uint32_t step,
                                             Stage (&t)[kSlots]) {
#pragma unroll
    for (int h = 0; h < kSlots; ++h) {
        const int64_t e = e0 + 32 * h;
        Upd u;
        u.i = -1;
        if (e < r1) {
            // (the FP32 path reads the 16-bit column offsets the sweep streams)
            const int32_t i = PREC == 1 && I.dcol != nullptr
                                  ? (int32_t)k + (int32_t)__ldg(&I.dcol[e])
                                  : __ldg(&I.col[e]);
            const long long dp = __ldg(&I.pq64[e].x), dq = __ldg(&I.qt64[e]);
            int dp32 = 0, dq32 = 0;
            if constexpr (PREC == 1) {
                dp32 = __ldg(&I.pq32[e].x);
                dq32 = __ldg(&I.qt32[e]);
            }
            if (i != (int32_t)k) u = compute_update<PREC, true>(I, i, snew, dp, dq, dp32, dq32, step);
        } else if (own && e == r1) {
            u = compute_update<PREC, true>(I, k, snew, 0, 0, 0, 0, step, snew);
        }
        t[h].i = (int32_t)u.i;
        t[h].h = u.h;
        t[h].nk = u.nk;
        t[h].x = u.x;
        t[h].g = u.g;
        t[h].lo = u.lo;
        t[h].s = u.s;
        t[h].push = u.nk > u.old ? 1 : 0;
    }
}

// Stores one update (t.i == k: the flipped island itself, whose spin goes too), the
// tree aside.
__device__ __forceinline__ void stage_store(const Inst& I, int64_t k, int snew, const Stage& t) {
    const int64_t i = t.i;
    if (i == k) I.s[k] = (int8_t)snew;
    I.h64[i] = t.h;
    rec_store_dyn(I, i, t.g, t.lo, t.s);
    I.key64[i] = t.x;
    I.key32[i] = t.nk;
}

// Stores one update and pushes its key up the tree when it grew.
__device__ __forceinline__ void stage_commit(const Inst& I, unsigned long long* const* lp,
                                             int64_t k, int snew, const Stage& t) {
    stage_store(I, k, snew, t);
    if (t.push) push_up(lp, I.nlev, t.i, t.nk);
}

// The own update of a pick flipped forward: island k keeps its field and its spin
// now points along h_par, so by Eq. 6 it is not flippable (its evaluation always
// gives key 0, exact value 0 and no lower bound); the 32-bit sums in its record
// stay as they are, so only the record's lower bound and spin are written.
__device__ __forceinline__ void own_flipped(const Inst& I, int64_t k, int snew) {
    I.s[k] = (int8_t)snew;
    *reinterpret_cast<int2*>(reinterpret_cast<int*>(I.rec + k) + 2) =
        make_int2(__float_as_int(-1.0f), snew);
    I.key64[k] = 0.0;
    I.key32[k] = 0ull;
}

// The best new value among a pick's neighbours, (*bv, *bi) so far: FS_FP64 the
// exact value, the FP32 path the upper bound of the key.
template <int PREC>
__device__ __forceinline__ void stage_best(const Stage& t, int64_t k, unsigned long long* bv,
                                           int32_t* bi) {
    if (t.i < 0 || t.i == k) return;
    unsigned long long val = 0ull;
    if constexpr (PREC == 0) {
        val = t.x > 0.0 ? (unsigned long long)__double_as_longlong(t.x) : 0ull;
    } else {
        val = t.nk ? (unsigned long long)__double_as_longlong((double)key32_hi(t.nk)) : 0ull;
    }
    if (val && before(val, t.i, *bv, *bi)) {
        *bv = val;
        *bi = t.i;
    }
}

__device__ __forceinline__ void warp_best(unsigned long long* bv, int32_t* bi) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, *bv, o);
        const int32_t oi = __shfl_xor_sync(0xffffffffu, *bi, o);
        if (ov && before(ov, oi, *bv, *bi)) {
            *bv = ov;
            *bi = oi;
        }
    }
}

// Flips island k (row [r0, r1)) to spin snew with every update stored, pass by
// pass; `forward`: a flip of the round (k's own update is own_flipped), else a flip
// back (k's own update evaluated like a neighbour's). Warp-wide; returns, on every
// lane, the best new value among the neighbours and its island.
template <int PREC>
__device__ void flip_warp(const Inst& I, unsigned long long* const* lp, int64_t k, int snew,
                          int64_t r0, int64_t r1, bool forward, uint32_t step,
                          unsigned long long* xv, int32_t* xi) {
    const int lane = threadIdx.x & 31;
    unsigned long long bv = 0ull;
    int32_t bi = 0x7fffffff;
    if (forward && lane == 0) own_flipped(I, k, snew);
    const int64_t last = forward ? r1 - 1 : r1;  // the last slot
    for (int64_t e0 = r0 + lane; e0 <= last; e0 += kStageSlots) {
        Stage t[kSlots];
        pass_compute<PREC>(I, k, snew, e0, r1, !forward, step, t);
#pragma unroll
        for (int h = 0; h < kSlots; ++h) {
            if (t[h].i < 0) continue;
            stage_commit(I, lp, k, snew, t[h]);
            stage_best<PREC>(t[h], k, &bv, &bi);
        }
    }
    warp_best(&bv, &bi);
    *xv = bv;
    *xi = bi;
}

// The forward flip of island k (row [r0, r1) of at most kStageSlots entries): the
// neighbours' updates computed into the warp's staging slots stg[0 .. kStageSlots)
// and the keys that grow pushed up the tree, nothing else stored; returns the best
// new neighbour value as flip_warp does. Warp-wide.
template <int PREC>
__device__ void compute_pick(const Inst& I, unsigned long long* const* lp, int64_t k, int snew,
                             int64_t r0, int64_t r1, uint32_t step, Stage* stg,
                             unsigned long long* xv, int32_t* xi) {
    const int lane = threadIdx.x & 31;
    unsigned long long bv = 0ull;
    int32_t bi = 0x7fffffff;
    Stage t[kSlots];
    pass_compute<PREC>(I, k, snew, r0 + lane, r1, false, step, t);
#pragma unroll
    for (int h = 0; h < kSlots; ++h) {
        stg[lane + 32 * h] = t[h];
        // (the keys that grow go up the tree now: a pick that is not stored leaves
        // the tree an upper bound still, and the next threshold can be chosen before
        // the stores)
        if (t[h].i >= 0 && t[h].push) push_up(lp, I.nlev, t[h].i, t[h].nk);
        stage_best<PREC>(t[h], k, &bv, &bi);
    }
    warp_best(&bv, &bi);
    *xv = bv;
    *xi = bi;
}

// Stores the flip compute_pick staged (its keys are up the tree already), and k's
// own update. Warp-wide.
__device__ void store_pick(const Inst& I, int64_t k, int snew, const Stage* stg) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) own_flipped(I, k, snew);
#pragma unroll
    for (int h = 0; h < kSlots; ++h) {
        const Stage t = stg[lane + 32 * h];
        if (t.i >= 0) stage_store(I, k, snew, t);
    }
}

// The exact FS_FP64 value of candidate island i, with what a round needs of it
// (spin, row, centre). An island found not flippable gets key 0 (no candidate until
// a flip raises it again); on the FP32 path a flippable one gets the key of its
// exact value (an upper bound no higher than the one it had). The FP32 path
// evaluates the exact sums in FP64 unless its current fields already were
// (key64 >= 0); the step's thermal draw is the kept one, or drawn and kept (no
// other thread evaluates island i meanwhile; *nfp64 counts the FP64 evaluations).
// Every load is issued up front.
template <int PREC>
__device__ __forceinline__ Cand eval_cand(const Inst& I, int64_t i, uint32_t step, int* nfp64) {
    const IslandRec r = rec_load(I, i);
    const double2 pc = __ldg(&I.pos[i]);
    const double kept = I.key64[i];
    double v = kept;
    if constexpr (PREC == 1) {
        const longlong2 h = I.h64[i];
        const double2 rb64 = __ldg(&I.rbc64[i]);
        const bool th = I.sigma > 0.0;
        uint32_t ts = 0u;
        double2 tv = make_double2(0.0, 0.0);
        if (th) {
            ts = I.th_step[i];
            tv = I.th64[i];
        }
        if (kept < 0.0) {
            ++*nfp64;
            if (th && ts != step) {
                thermal64(I, i, step, &tv.x, &tv.y);
                I.th64[i] = tv;
                __threadfence_block();
                *(volatile uint32_t*)&I.th_step[i] = step;
            }
            const Eval64 e = eval64(I, r.s, h.x, h.y, rb64, ext64_at(I, i, r.cls), tv.x, tv.y);
            v = e.flippable ? e.lhs : 0.0;
            I.key64[i] = v;
        }
    }
    if (v > 0.0) {
        if constexpr (PREC == 1) I.key32[i] = key32_of(__double2float_ru(v), i);
    } else {
        I.key32[i] = 0ull;
    }
    Cand c;
    c.v = v > 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull;
    c.i = (int32_t)i;
    c.rowq = r.rowq;
    c.pos = make_float2(__double2float_rn(pc.x), __double2float_rn(pc.y));
    c.rowlenq = r.rowlenq;
    c.s = (int16_t)r.s;
    c.pad = 0;
    return c;
}

// The exact best flippable island of the whole array by a full scan (every key
// above zero evaluated exactly), for rounds whose candidate set cannot be held;
// S.si[0] / S.sv[0] receive it (S.nc = 0 when none). CTA-wide.
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
    S.sv[tid] = bv;
    S.si[tid] = bi;
    __syncthreads();
    for (int w = kMT / 2; w > 0; w >>= 1) {
        if (tid < w && S.sv[tid + w] && before(S.sv[tid + w], S.si[tid + w], S.sv[tid], S.si[tid])) {
            S.sv[tid] = S.sv[tid + w];
            S.si[tid] = S.si[tid + w];
        }
        __syncthreads();
    }
    if (tid == 0) S.nc = S.sv[0] ? 1 : 0;
    __syncthreads();
}

// S.cand[0 .. n) into "before" order in S.sv / S.si / S.so. Up to kRankMax entries
// by rank (each entry counts those that go before it, kMT / n threads an entry;
// islands are distinct). More by merging: every warp sorts runs of 32 in registers
// (a bitonic network over its lanes), then pairs of runs merge until one run holds
// everything, each entry's place being its place in its own run plus the number of
// entries of the other run that go before it (a binary search; the left run wins
// ties, which only padding entries, past n up to a power of two, can have: they
// sort last). CTA-wide.
__device__ void sort_candidates(MultiShared& S, int n) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (n <= kRankMax) {
        // kMT / n consecutive threads count for one entry (at least two), each over
        // every tpc-th other, their counts summed in S.mi
        const int tpc = kMT / n;
        const int e = tid / tpc, part = tid - e * tpc;
        for (int c = tid; c < n; c += kMT) S.mi[c] = 0;
        __syncthreads();
        unsigned long long v = 0ull;
        int32_t ix = 0;
        if (e < n) {
            v = S.cand[e].v;
            ix = S.cand[e].i;
            int r = 0;
            int u = part;
            for (; u + 7 * tpc < n; u += 8 * tpc) {  // (eight loads in flight)
                unsigned long long w[8];
                int32_t wi[8];
#pragma unroll
                for (int z = 0; z < 8; ++z) {
                    w[z] = S.cand[u + z * tpc].v;
                    wi[z] = S.cand[u + z * tpc].i;
                }
#pragma unroll
                for (int z = 0; z < 8; ++z) r += before(w[z], wi[z], v, ix) ? 1 : 0;
            }
            for (; u < n; u += tpc) r += before(S.cand[u].v, S.cand[u].i, v, ix) ? 1 : 0;
            if (r) atomicAdd(&S.mi[e], r);
        }
        __syncthreads();
        if (e < n && part == 0) {
            const int r = S.mi[e];
            S.sv[r] = v;
            S.si[r] = ix;
            S.so[r] = (int16_t)e;
        }
        __syncthreads();
        return;
    }
    int n2 = 32;
    while (n2 < n) n2 <<= 1;  // (<= kCandCap)
    // runs of 32 in registers, into (sv, si, so)
    for (int base = wid * 32; base < n2; base += kMT) {
        const int t = base + lane;
        unsigned long long v = t < n ? S.cand[t].v : 0ull;
        int32_t ix = t < n ? S.cand[t].i : 0x7fffffff;
        int32_t so = t < n ? t : -1;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, j);
                const int32_t oi = __shfl_xor_sync(0xffffffffu, ix, j);
                const int32_t os = __shfl_xor_sync(0xffffffffu, so, j);
                // the pair's lower lane keeps the entry that goes first in a block
                // sorted forwards, the later one in a block sorted backwards
                const bool fwd = (lane & k) == 0 || k == 32;
                const bool lower = (lane & j) == 0;
                const bool take = fwd == lower ? before(ov, oi, v, ix) : before(v, ix, ov, oi);
                if (take) {
                    v = ov;
                    ix = oi;
                    so = os;
                }
            }
        }
        S.sv[t] = v;
        S.si[t] = ix;
        S.so[t] = (int16_t)so;
    }
    __syncthreads();
    // pairwise merges, between (sv, si, so) and (mv, mi, mo)
    bool in_m = false;
    for (int r = 32; r < n2; r <<= 1) {
        const unsigned long long* fv = in_m ? S.mv : S.sv;
        const int32_t* fi = in_m ? S.mi : S.si;
        const int16_t* fo = in_m ? S.mo : S.so;
        unsigned long long* tv = in_m ? S.sv : S.mv;
        int32_t* ti = in_m ? S.si : S.mi;
        int16_t* to = in_m ? S.so : S.mo;
        for (int t = tid; t < n2; t += kMT) {
            const unsigned long long v = fv[t];
            const int32_t ix = fi[t];
            const int16_t so = fo[t];
            const int run = t / r, k = t % r;
            const bool left = (run & 1) == 0;
            const int other = (run ^ 1) * r;
            // entries of the other run that go before this one (ties: the left run first)
            int lo = 0, hi = r;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                const unsigned long long w = fv[other + mid];
                const int32_t wi = fi[other + mid];
                const bool goes_before = left ? before(w, wi, v, ix) : !before(v, ix, w, wi);
                if (goes_before)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int dst = (run >> 1) * 2 * r + k + lo;
            tv[dst] = v;
            ti[dst] = ix;
            to[dst] = so;
        }
        __syncthreads();
        in_m = !in_m;
    }
    if (in_m) {
        for (int t = tid; t < n; t += kMT) {
            S.sv[t] = S.mv[t];
            S.si[t] = S.mi[t];
            S.so[t] = S.mo[t];
        }
        __syncthreads();
    }
}

constexpr int32_t kCmdPlan = 3;  // (the leader's own step: choose the next threshold)

// The leader's round state (the same in every leader thread; the hash on kHashT).
struct Lead {
    int64_t flips, rounds, idle_total, max_flips, flips_before;
    uint64_t hash;
    unsigned long long carry;   // a threshold from the previous round's candidates
    unsigned long long forced;  // a threshold set by the previous iteration
    int32_t status;
    int M, m0, idle, low, lsel;
    bool need_scan, was_carried, was_forced, handoff;
};

// The leader: the next threshold and the frontier of tree nodes that reach it (on
// level 1, or level 0 for a one-level selection), or, for a candidate set too large
// at every threshold, the one best island by a full scan. The threshold is chosen
// on level lsel, loaded whole (its M-th largest node, unless the previous round
// carried one or forced one). `early`: the round's stores are still to come (the
// tree holds their keys already); a scan then waits for them (returns kCmdPlan).
// Returns the cluster's next command. Leader CTA-wide.
template <int PREC>
__device__ int32_t plan(const Inst& I, MultiShared& S, Lead& G, uint32_t step, bool early) {
    constexpr int kB = 4;  // frontier nodes whose children a warp loads together
    const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
    for (;;) {
        if (++G.idle > kMaxIdle) {
            G.status = ST_BOUNDS;
            return kCmdStop;
        }
        if (G.need_scan && early) return kCmdPlan;  // (a scan reads the stored keys)
        if (G.need_scan) {  // a candidate set too large for any threshold
            G.need_scan = false;
            G.M = G.m0;
            scan_best<PREC>(I, step, S);
            if (S.nc == 0) return kCmdStop;
            if (G.max_flips - G.flips <= 0) {
                G.status = ST_NOT_CONVERGED;
                return kCmdStop;
            }
            if (tid == 0) {
                const IslandRec r = rec_load(I, S.si[0]);
                Pick pk;
                pk.i = S.si[0];
                pk.rowq = r.rowq;
                pk.rowlenq = r.rowlenq;
                pk.s = (int16_t)r.s;
                pk.eager = 0;
                S.pk[0] = pk;
                S.q = 1;
                S.nz = 1;
            }
            __syncthreads();
            return kCmdCompute;
        }
        ++G.idle_total;
        const int lsel = G.lsel;
        const int cnt = I.lvl_n[lsel];
        unsigned long long v[kSelPer];
#pragma unroll
        for (int u = 0; u < kSelPer; ++u) {
            const int c = tid + u * kMT;
            v[u] = c < cnt ? __ldcg(S.lp[lsel] + c) : 0ull;
        }
        unsigned long long tkey = 1ull;
        G.was_forced = G.forced != 0ull;
        G.was_carried = !G.was_forced && G.carry != 0ull;
        if (G.was_forced) {
            tkey = G.forced;
            G.forced = 0ull;
        } else if (G.was_carried) {
            tkey = G.carry;
            G.carry = 0ull;
        } else {
            const uint32_t sel = select_threshold(v, cnt, G.M, S);
            // lowered by 2^-18 (relative) so that the node's own island, whose exact
            // value lies within its key's band, counts as reaching it
            const float lo = __fmul_rd(__uint_as_float(sel), 1.0f - 0x1.0p-18f);
            tkey = sel ? ((unsigned long long)__float_as_uint(lo) << 32) : 1ull;
            if (tkey == 0ull) tkey = 1ull;
        }
        // the nodes of level lsel that reach it
        if (tid == 0) S.nf[0] = 0;
        __syncthreads();
        {  // (each thread's hits as a mask; one reservation a warp)
            unsigned hm = 0u;
#pragma unroll
            for (int u = 0; u < kSelPer; ++u)
                if (tid + u * kMT < cnt && v[u] != 0ull && v[u] >= tkey) hm |= 1u << u;
            const int nh = __popc(hm);
            int incl = nh;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            int base = 0;
            if (lane == 31 && incl) base = atomicAdd(&S.nf[0], incl);
            int pos = __shfl_sync(0xffffffffu, base, 31) + incl - nh;
#pragma unroll
            for (int u = 0; u < kSelPer; ++u)
                if ((hm >> u) & 1u) {
                    if (pos < kCandCap) S.front[0][pos] = tid + u * kMT;
                    ++pos;
                }
        }
        __syncthreads();
        int cur = 0;
        bool over = S.nf[0] > kCandCap;
        // down to level 1, every expanded node rebuilt from its children (a node is
        // never below its children: pushes raise every ancestor, rebuilds set a node
        // to its children's maximum; so it is stored without being read first)
        for (int lev = lsel; lev >= 2 && !over; --lev) {
            const int nf = S.nf[cur];
            if (tid == 0) S.nf[cur ^ 1] = 0;
            __syncthreads();
            const int64_t lim = I.lvl_n[lev - 1];
            for (int f0 = wid * kB; f0 < nf; f0 += kMW * kB) {
                int64_t node[kB];
                unsigned long long w[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    node[u] = f0 + u < nf ? (int64_t)S.front[cur][f0 + u] : -1;
                    const int64_t c = (node[u] << 5) + lane;
                    w[u] = node[u] >= 0 && c < lim ? __ldcg(S.lp[lev - 1] + c) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    if (node[u] < 0) break;
                    const int64_t c = (node[u] << 5) + lane;
                    const unsigned long long m = warp_max_key(w[u]);
                    if (lane == 0) S.lp[lev][node[u]] = m;
                    warp_append(w[u] != 0ull && w[u] >= tkey, (int32_t)c, S.front[cur ^ 1],
                                &S.nf[cur ^ 1], kCandCap);
                }
            }
            __syncthreads();
            over = S.nf[cur ^ 1] > kCandCap;
            cur ^= 1;
        }
        if (over) {  // too many nodes reach it: a higher threshold, or a scan
            if (!G.was_carried) {
                if (G.M > 1 && !G.was_forced)
                    G.M >>= 1;
                else
                    G.need_scan = true;
            }
            continue;
        }
        if (S.nf[cur] == 0) {
            if (tkey == 1ull) return kCmdStop;  // no key above zero: the relax is done
            G.M = G.m0;  // the threshold came from stale nodes, rebuilt on the way
            continue;
        }
        if (tid == 0) {
            S.f_lev = lsel >= 1 ? 1 : 0;
            S.f_buf = cur;
            S.tkey = tkey;
            S.nl = 0;
        }
        __syncthreads();
        return kCmdExpand;
    }
}

// The leader after an expansion: the candidates in order, the eligible prefix (a),
// the cut at the first pick too close to an earlier one (b) and the step's flip
// budget give the picks. Returns the cluster's next command (kCmdPlan when there
// is nothing to flip at this threshold). Leader CTA-wide.
__device__ int32_t decide(const Inst& I, MultiShared& S, Lead& G) {
    const int tid = threadIdx.x;
    const int nl = S.nl;
    if (nl > kCandCap) {  // too many candidates: a higher threshold, or a scan
        if (!G.was_carried) {
            if (G.M > 1 && !G.was_forced)
                G.M >>= 1;
            else
                G.need_scan = true;
        }
        return kCmdPlan;
    }
    if (nl == 0) {
        if (S.tkey == 1ull) return kCmdStop;  // no key above zero
        G.M = G.m0;  // stale nodes, rebuilt by the expansion
        return kCmdPlan;
    }
    sort_candidates(S, nl);
    // (a) a pick must beat every island below the threshold: (v, i) no later than
    // (tau, tau_index) in "before" order; eligibility is a prefix of the order
    const unsigned long long tkey = S.tkey;
    const double tau = (double)__uint_as_float((uint32_t)(tkey >> 32));
    const uint32_t tau_i = key32_idx(tkey);
    const unsigned long long tb = (unsigned long long)__double_as_longlong(tau);
    if (tid == 0) S.conflict_at = kPickCap;
    // flippable candidates and eligible ones are prefixes of the order: their counts
    // are their lengths
    int nz = 0, q = 0;
    for (int c0 = 0; c0 < nl; c0 += kMT) {  // (uniform: nl <= kCandCap)
        const int c = c0 + tid;
        const unsigned long long v = c < nl ? S.sv[c] : 0ull;
        if (c < kPickCap && c < nl) S.sp[c] = S.cand[S.so[c]].pos;
        const bool ok =
            c < kPickCap && v != 0ull && (v > tb || (v == tb && (uint32_t)S.si[c] <= tau_i));
        nz += __syncthreads_count(v != 0ull);
        q += __syncthreads_count(ok);
    }
    if (tid == 0) S.nz = nz;
    if (q == 0) {
        if (S.sv[0] != 0ull) {
            // every candidate lies below the threshold: the next iteration takes the
            // best one's value (rounded down) as the threshold, so that every island
            // that could beat it is a candidate
            const float v0 = __double2float_rd(__longlong_as_double((long long)S.sv[0]));
            const unsigned long long tk = (unsigned long long)__float_as_uint(v0) << 32;
            G.forced = tk > 0ull ? tk : 1ull;
        } else {
            G.M = G.m0;  // none of them is flippable (all demoted)
        }
        return kCmdPlan;
    }
    // (b) picks more than twice the cutoff apart: threads 2c and 2c + 1 test pick c
    // against the even and the odd j < c, in FP32 against a radius widened by the
    // rounding of the centres
    {
        const int c = tid >> 1;  // (q <= kPickCap <= kMT / 2)
        bool hit = false;
        if (c >= 1 && c < q) {
            const float2 a = S.sp[c];
            const float r2 = I.rconf2f;
            int j = tid & 1;
            for (; j + 6 < c; j += 8) {
#pragma unroll
                for (int z = 0; z < 4; ++z) {
                    const float2 b = S.sp[j + 2 * z];
                    const float dx = __fsub_rn(a.x, b.x);
                    const float dy = __fsub_rn(a.y, b.y);
                    hit |= __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= r2;
                }
            }
            for (; j < c; j += 2) {
                const float2 b = S.sp[j];
                const float dx = __fsub_rn(a.x, b.x);
                const float dy = __fsub_rn(a.y, b.y);
                hit |= __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) <= r2;
            }
        }
        if (hit) atomicMin(&S.conflict_at, c);
    }
    __syncthreads();
    q = min(q, S.conflict_at);
    // the step's flip budget
    const int64_t allowed = G.max_flips - G.flips;
    if (allowed <= 0) {
        G.status = ST_NOT_CONVERGED;
        return kCmdStop;
    }
    if (q > allowed) q = (int)allowed;
    for (int c = tid; c < q; c += kMT) {
        const Cand& cd = S.cand[S.so[c]];
        Pick pk;
        pk.i = cd.i;
        pk.rowq = cd.rowq;
        pk.rowlenq = cd.rowlenq;
        pk.s = cd.s;
        pk.eager = 0;
        S.pk[c] = pk;
    }
    if (tid == 0) {
        S.q = q;
        S.nc = nl;
    }
    __syncthreads();
    return kCmdCompute;
}

// The hash thread folds the first n queued flips into the sequence hash, in order.
__device__ __forceinline__ void hash_queue(const MultiShared& S, Lead& G, uint32_t step, int n) {
    for (int j = 0; j < n; ++j) G.hash = fnv_flip(G.hash, step, (uint32_t)S.hq[j]);
}

// The leader after the picks are computed: the longest prefix of the picks that no
// earlier pick's neighbour overtakes (c); the eager picks after it flipped back (a
// warp a pick); the prefix logged and queued for the hash in order; the threshold
// carried to the next round, and the next round planned (S.next: what follows the
// stores). In a cluster it arrives at a cluster barrier once the prefix is known, so
// that the other CTAs store the prefix meanwhile. Leader CTA-wide.
template <int PREC, int NC>
__device__ void prefix_step(const Inst& I, MultiShared& S, Lead& G, uint32_t step) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int q = S.q;
    // the best of the earlier picks' neighbour values, an exclusive prefix maximum
    // over the picks in order (thread j: pick j; within warps, then across them)
    if (tid == 0) S.p = q;
    {
        const int j = tid;  // (q <= kPickCap <= kMT)
        unsigned long long xv = j < q ? S.xv[j] : 0ull;
        int32_t xi = j < q ? S.xi[j] : 0x7fffffff;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {  // inclusive prefix maximum within the warp
            const unsigned long long ov = __shfl_up_sync(0xffffffffu, xv, o);
            const int32_t oi = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o && ov && (!xv || before(ov, oi, xv, xi))) {
                xv = ov;
                xi = oi;
            }
        }
        if (lane == 31) {
            S.wv[wid] = xv;
            S.wi[wid] = xi;
        }
        unsigned long long ev = __shfl_up_sync(0xffffffffu, xv, 1);
        int32_t ei = __shfl_up_sync(0xffffffffu, xi, 1);
        if (lane == 0) {
            ev = 0ull;
            ei = 0x7fffffff;
        }
        __syncthreads();
        for (int w = 0; w < wid && w * 32 < q; ++w) {  // the earlier warps' maxima
            const unsigned long long wv = S.wv[w];
            const int32_t wi = S.wi[w];
            if (wv && (!ev || before(wv, wi, ev, ei))) {
                ev = wv;
                ei = wi;
            }
        }
        if (j < q && j > 0 && ev && !before(S.sv[j], S.si[j], ev, ei)) atomicMin(&S.p, j);
    }
    __syncthreads();
    const int p = S.p;
    // the prefix is out: the other CTAs store their picks' updates while the leader
    // goes on (it waits for that barrier before the next one)
    if constexpr (NC > 1) cluster_arrive();
    // the eager ones among the rest flipped back (the staged ones are dropped)
    for (int j = p + wid; j < q; j += kMW) {
        const Pick pk = S.pk[j];
        if (!pk.eager) continue;
        const int64_t r0 = (int64_t)pk.rowq << 2;
        unsigned long long xv;
        int32_t xi;
        flip_warp<PREC>(I, S.lp, pk.i, pk.s, r0, r0 + ((int64_t)pk.rowlenq << 2), false, step, &xv,
                        &xi);
    }
    // log and hash, in the order of the picks
    for (int j = tid; j < p; j += kMT) {
        const int64_t qq = G.flips_before + G.flips + j;
        if (I.log_spin && qq < I.log_cap) {
            I.log_step[qq] = step;
            I.log_spin[qq] = (uint32_t)S.si[j];
        }
    }
    // the flips join the hash queue (folded in by the hash thread while the next
    // picks are computed, or here when the queue is full)
    const int hn = S.hq_n;  // (rewritten below only after a barrier)
    int h0 = hn;
    if (hn + p > kHashQ) {
        if (tid == kHashT) hash_queue(S, G, step, hn);
        __syncthreads();
        h0 = 0;
    }
    for (int j = tid; j < p; j += kMT) S.hq[h0 + j] = S.si[j];
    G.flips += p;
    G.idle = 0;
    --G.idle_total;
    ++G.rounds;
    G.M = G.m0;
    G.low = p < kPMin ? G.low + 1 : 0;
    if (G.low >= kLowRounds) G.handoff = true;
    // the next round's threshold: the value kCarry places below this round's last
    // flip among its flippable candidates (most of them are still unflipped), so
    // that the next candidate set is about that large
    {
        const int r = min(S.nz - 1, p + kCarry);
        const unsigned long long vr = r > p ? S.sv[r] : 0ull;
        G.carry = 0ull;
        if (vr) {
            const float f = __fmul_rd(__double2float_rd(__longlong_as_double((long long)vr)),
                                      1.0f - 0x1.0p-18f);
            G.carry = (unsigned long long)__float_as_uint(f) << 32;
        }
    }
    __syncthreads();
    if (tid == 0) S.hq_n = h0 + p;
    // the next threshold and frontier now (the tree holds the round's keys)
    const int32_t next = G.handoff ? kCmdStop : plan<PREC>(I, S, G, step, true);
    if (tid == 0) S.next = next;
}

// Every CTA of the cluster: the frontier nodes L->front[L->f_buf] expanded into the
// keys that reach L->tkey (level-1 nodes first into their level-0 children that
// reach it), each expanded node rebuilt from its children; the candidate islands
// this CTA found are then evaluated exactly into the leader's list (L->nl counts
// them, past kCandCap too). Warps of all CTAs share the nodes.
template <int PREC, int NC>
__device__ void expand_eval(const Inst& I, MultiShared* L, MultiShared& S, int rank,
                            uint32_t step, int* nfp64) {
    constexpr int kB = 8;
    constexpr int kW = NC * kMW;  // warps that expand
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int gw = rank * kMW + wid;
    if (tid == 0) S.nloc = 0;
    __syncthreads();
    {
        const int f_lev = L->f_lev, buf = L->f_buf;
        const int nf = L->nf[buf];
        const unsigned long long tkey = L->tkey;
        if (f_lev == 0) {
            for (int fb = gw * kB; fb < nf; fb += kW * kB) {
                int64_t node[kB];
                unsigned long long v[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    node[u] = fb + u < nf ? (int64_t)L->front[buf][fb + u] : -1;
                    const int64_t c = (node[u] << 5) + lane;
                    v[u] = node[u] >= 0 && c < I.n ? __ldcg(&I.key32[c]) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    if (node[u] < 0) break;
                    const int64_t c = (node[u] << 5) + lane;
                    const unsigned long long m = warp_max_key(v[u]);
                    if (lane == 0) S.lp[0][node[u]] = m;
                    warp_append(v[u] != 0ull && v[u] >= tkey, (int32_t)c, S.loc, &S.nloc,
                                kCandCap);
                }
            }
        } else {
            const int64_t n0 = I.lvl_n[0];
            for (int f = gw; f < nf; f += kW) {
                const int64_t node1 = L->front[buf][f];
                const int64_t c1 = (node1 << 5) + lane;
                const unsigned long long w = c1 < n0 ? __ldcg(S.lp[0] + c1) : 0ull;
                const unsigned long long m1 = warp_max_key(w);
                if (lane == 0) S.lp[1][node1] = m1;
                unsigned hm = __ballot_sync(0xffffffffu, w != 0ull && w >= tkey);
                while (hm) {  // the children that reach it, kB at a time
                    int64_t node[kB];
                    unsigned long long v[kB];
#pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        node[u] = -1;
                        if (hm) {
                            node[u] = (node1 << 5) + (__ffs(hm) - 1);
                            hm &= hm - 1u;
                        }
                        const int64_t c = (node[u] << 5) + lane;
                        v[u] = node[u] >= 0 && c < I.n ? __ldcg(&I.key32[c]) : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        if (node[u] < 0) break;
                        const int64_t c = (node[u] << 5) + lane;
                        const unsigned long long m = warp_max_key(v[u]);
                        if (lane == 0) S.lp[0][node[u]] = m;
                        warp_append(v[u] != 0ull && v[u] >= tkey, (int32_t)c, S.loc, &S.nloc,
                                    kCandCap);
                    }
                }
            }
        }
    }
    __syncthreads();
    // one block of slots in the leader's list for this CTA's candidates
    const int nloc = S.nloc;
    if (tid == 0) S.lbase = nloc ? atomicAdd(&L->nl, nloc) : 0;
    __syncthreads();
    const int base = S.lbase;
    const int lim = min(nloc, kCandCap - base);  // (an overflowing set is dropped by the leader)
    for (int k = tid; k < lim; k += kMT)
        L->cand[base + k] = eval_cand<PREC>(I, S.loc[k], step, nfp64);
}

// Every CTA of the cluster: the round's picks (their neighbourhoods are disjoint), a
// warp a pick. A warp's first pick whose row fits one pass is computed into the
// warp's staging slots, to be stored once the prefix is known (returns true, with
// the pick's index, island and new spin); any other pick is flipped at once and
// marked eager. Each pick's best new neighbour value goes to the leader.
template <int PREC, int NC>
__device__ bool compute_picks(const Inst& I, MultiShared* L, MultiShared& S, Lead& G, Stage* stg,
                              int rank, uint32_t step, int* held_j, int64_t* held_k,
                              int* held_s) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int q = L->q;
    bool held = false;
    // in a cluster the leader takes no pick (it plans the next round while the other
    // CTAs store theirs): pick j goes to CTA 1 + j % (NC - 1)
    constexpr int kPR = NC > 1 ? NC - 1 : 1;  // CTAs that take picks
    const int prank = NC > 1 ? rank - 1 : 0;
    for (int j = prank + kPR * wid; prank >= 0 && j < q; j += kPR * kMW) {
        const Pick pk = L->pk[j];
        const int64_t r0 = (int64_t)pk.rowq << 2, r1 = r0 + ((int64_t)pk.rowlenq << 2);
        unsigned long long xv;
        int32_t xi;
        if (!held && r1 - r0 <= kStageSlots) {
            compute_pick<PREC>(I, S.lp, pk.i, -pk.s, r0, r1, step, stg, &xv, &xi);
            held = true;
            *held_j = j;
            *held_k = pk.i;
            *held_s = -pk.s;
        } else {
            flip_warp<PREC>(I, S.lp, pk.i, -pk.s, r0, r1, true, step, &xv, &xi);
            if (lane == 0) L->pk[j].eager = 1;
        }
        if (lane == 0) {
            L->xv[j] = xv;
            L->xi[j] = xi;
        }
    }
    // the leader's hash thread (in a cluster its warp has no pick; alone, its first
    // pick, kMW - 1, lies past most rounds' picks): the queued flips of the earlier
    // rounds into the hash
    if (rank == 0 && threadIdx.x == kHashT) {
        hash_queue(S, G, step, S.hq_n);
        S.hq_n = 0;
    }
    return held;
}

template <int PREC, int NC>
__global__ void __launch_bounds__(kMT, 1)
    k_relax_multi(const Inst* __restrict__ tab, const int32_t* __restrict__ work, int n_work) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char multi_smem[];
    MultiShared& S = *reinterpret_cast<MultiShared*>(multi_smem);
    Stage* const stg = reinterpret_cast<Stage*>(multi_smem + kStageOff) +
                       (threadIdx.x >> 5) * kStageSlots;  // this warp's staging slots
    int rank = 0;
    MultiShared* L = &S;  // the leader's state, as this CTA reaches it
    if constexpr (NC > 1) {
        cg::cluster_group cl = cg::this_cluster();
        rank = (int)cl.block_rank();
        if (rank != 0) L = cl.map_shared_rank(&S, 0);
    }
    auto csync = [&]() {
        if constexpr (NC > 1)
            cg::this_cluster().sync();
        else
            __syncthreads();
    };
    const bool leader = rank == 0;
    const int tid = threadIdx.x;

    // this CTA's copy of the descriptor, read from shared memory from here on; with
    // a global external field, the step's per-class table is copied too
    {
        const unsigned long long* src =
            reinterpret_cast<const unsigned long long*>(&tab[work[blockIdx.x / NC]]);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&S.inst);
        for (int w = tid; w < (int)(sizeof(Inst) / 8); w += kMT) dst[w] = src[w];
    }
    __syncthreads();
    const Inst& I = S.inst;
    InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;  // (the same for every CTA)
    const uint32_t step = I.step0 + (uint32_t)t;
    const bool cls_sh = I.exti64 == nullptr && I.nclass <= kClsSh;
    if (cls_sh)
        for (int c = tid; c < I.nclass; c += kMT) {
            S.ext64[c] = I.ext64[c];
            S.ext32[c] = I.ext32[c];
        }
    __syncthreads();
    if (tid == 0) {
        if (cls_sh) {
            S.inst.ext64 = S.ext64;
            S.inst.ext32 = S.ext32;
        }
        for (int lev = 0; lev < kMaxLevels; ++lev)
            S.lp[lev] = lev < I.nlev ? I.tree + I.lvl_off[lev] : nullptr;
        S.hq_n = 0;
    }
    __syncthreads();

    Lead G;
    G.lsel = 0;
    while (G.lsel < I.nlev - 1 && I.lvl_n[G.lsel] > kSelMax) ++G.lsel;
    G.flips = 0;
    G.rounds = 0;
    G.idle_total = 0;
    G.max_flips = I.max_flips;
    G.flips_before = st->n_flips;
    G.hash = leader && tid == kHashT ? st->hash : 0ull;
    G.carry = 0ull;
    G.forced = 0ull;
    G.status = ST_OK;
    G.m0 = max(1, min(kM0, I.lvl_n[G.lsel] / 8));  // rank of the threshold node
    G.M = G.m0;
    G.idle = 0;
    G.low = 0;
    G.need_scan = G.was_carried = G.was_forced = G.handoff = false;

    int32_t cmd = kCmdPlan;  // (the leader's next step)
    int nfp64 = 0;           // this thread's FP64 evaluations of candidates
    bool ready = false;      // every CTA has the next command already (S.next)
    bool held = false;       // this warp holds a staged pick:
    int held_j = 0, held_s = 0;  // its index and new spin,
    int64_t held_k = 0;      // its island
    for (;;) {
        if (ready) {
            ready = false;
        } else {
            if (leader) {
                if (cmd == kCmdPlan) cmd = plan<PREC>(I, S, G, step, false);
                if (tid == 0) S.cmd = cmd;
            }
            csync();  // the leader's command is out
            cmd = L->cmd;
        }
        if (cmd == kCmdStop) break;
        if (cmd == kCmdExpand) {
            expand_eval<PREC, NC>(I, L, S, rank, step, &nfp64);
            csync();  // the candidates are in
            if (leader) cmd = decide(I, S, G);
        } else {  // kCmdCompute
            held = compute_picks<PREC, NC>(I, L, S, G, stg, rank, step, &held_j, &held_k, &held_s);
            csync();  // the picks are computed
            if constexpr (NC > 1) {
                if (leader) {
                    prefix_step<PREC, NC>(I, S, G, step);  // (arrives once the prefix is out)
                    cluster_wait();
                } else {
                    // the picks before the prefix stored while the leader plans
                    cluster_arrive();
                    cluster_wait();  // the prefix is out
                    if (held && held_j < L->p) store_pick(I, held_k, held_s, stg);
                }
            } else {
                prefix_step<PREC, NC>(I, S, G, step);
                if (held && held_j < S.p) store_pick(I, held_k, held_s, stg);
            }
            held = false;
            csync();  // the prefix is stored, the next round planned
            cmd = L->next;
            ready = cmd != kCmdPlan;  // (a plan that waited for the stores comes next)
        }
    }
    csync();  // (no CTA leaves while another may still reach the leader's memory)
    // the FP64 evaluations of the candidates count as the FP32 path's exact work
    nfp64 = __reduce_add_sync(0xffffffffu, nfp64);
    if ((threadIdx.x & 31) == 0 && nfp64)
        atomicAdd((unsigned long long*)&st->rechecks, (unsigned long long)nfp64);
    if (!leader) return;
    if (tid == kHashT) {
        hash_queue(S, G, step, S.hq_n);
        st->hash = G.hash;
    }
    if (tid == 0) {
        st->rounds += G.rounds;
        st->idle += G.idle_total;
        st->round_flips += G.flips;
        st->n_flips = G.flips_before + G.flips;
        if (G.status != ST_OK) st->status = G.status;
        if (G.handoff && G.status == ST_OK) {  // the single-flip relax finishes step t
            st->handoff = 1;
            st->step_flips = G.flips;
            ++st->handoffs;
        } else {
            if (I.flips_per_step) I.flips_per_step[t] = G.flips;
            st->init = 0;
            st->t = t + 1;
        }
    }
}

constexpr int kNC = 16;  // CTAs of a multi-flip relax cluster (a non-portable size)

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
    return cudaLaunchKernelEx(&cfg, k_relax_multi<PREC, NC>, L.tab, L.work, L.n_work);
}

template <int PREC, int NC>
cudaError_t set_multi_smem(int smem) {
    if (NC > 8) {  // (more than the portable 8 CTAs a cluster)
        const cudaError_t e = cudaFuncSetAttribute(
            k_relax_multi<PREC, NC>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
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
    // per precision: whether the attributes are set, and whether a cluster fits
    // (checked once, before any launch is captured)
    static std::atomic<int> ready[2] = {{0}, {0}};
    static std::atomic<int> use_cluster[2] = {{0}, {0}};
    static std::mutex mu;
    const int k = L.prec == 1 ? 1 : 0;
    const int smem = kStageOff + kMW * kStageSlots * (int)sizeof(Stage);
    if (!ready[k].load()) {
        std::lock_guard<std::mutex> g(mu);
        if (!ready[k].load()) {
            cudaError_t e = k ? set_multi_smem<1, 1>(smem) : set_multi_smem<0, 1>(smem);
            if (e == cudaSuccess) e = k ? set_multi_smem<1, kNC>(smem) : set_multi_smem<0, kNC>(smem);
            if (e != cudaSuccess) return e;
            use_cluster[k].store((k ? cluster_fits<1>(smem) : cluster_fits<0>(smem)) ? 1 : 0);
            ready[k].store(1);
        }
    }
    if (use_cluster[k].load() && L.multi != 2)
        return k ? launch_multi<1, kNC>(L, smem, st) : launch_multi<0, kNC>(L, smem, st);
    return k ? launch_multi<1, 1>(L, smem, st) : launch_multi<0, 1>(L, smem, st);
}

}  // namespace fs
