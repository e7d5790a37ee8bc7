// fs_relax.cu - the greedy single-flip relaxation (Sec. "Dynamics"), one CTA per
// simulation, entirely on the device.
//
// Keys: one 64-bit key per island, (FP32 upper bound of its Eq. 5 LHS) << 32 |
// (2^32 - 1 - index), 0 when the island cannot be flippable; a max-tree of fan-out
// 32 over the keys, its upper levels in shared memory. The largest key is the
// island with the largest bound, lowest index first.
//
// Per flip: warp 0 reads the root's island w and the largest other key (w's
// sibling sets at every level). w is taken when its certified lower bound exceeds
// one and that runner-up's upper bound; otherwise the islands whose bounds reach
// the threshold are compared exactly (FS_FP64 values), non-flippable ones are
// demoted, and the exact best is taken once no island outside the set can beat
// it. Then island k is flipped and every neighbour i of k (row k of the CSR,
// whose transposed coefficients give the field k puts on i in i's frame) gets
// 2 s_k(new) (P_ik, Q_ik) added to its exact fixed-point sums and a new key. A key
// that grows is pushed up the tree with atomic maxima; a node whose maximum was a
// key that shrank is rebuilt from its children, level by level. Fields are held
// constant over the relax, as the paper states.
//
// FS_FP32_RECHECK computes keys from FP32 bounds and its exact values in FP64;
// FS_FP64 computes every candidate's exact value when its key is set, and its keys
// are that value rounded out to FP32.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"
#include "fs_kernels.h"

namespace fs {

namespace {

constexpr int kT = 256;  // threads per relax CTA
constexpr int kNW = kT / 32;
constexpr int kDirtyCap = kMaxPaddedDegree + 8;

struct Levels {
    unsigned long long* p[kMaxLevels];
};

// Warp maximum of 64-bit keys (every lane gets it): the largest upper half, then
// among those the largest lower half.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

// Node `node` of level `lev` from its 32 children (leaves when lev == 0).
__device__ __forceinline__ unsigned long long warp_node(const Inst& I, const Levels& L, int lev,
                                                        int64_t node) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (node << 5) + lane;
    unsigned long long v = 0ull;
    if (lev == 0) {
        if (c < I.n) v = I.key32[c];
    } else if (c < I.lvl_n[lev - 1]) {
        v = L.p[lev - 1][c];
    }
    return warp_max_key(v);
}

// The largest key other than island w's: w's fellow leaves and, at every level,
// the siblings of w's ancestor. Warp-wide.
__device__ unsigned long long runner_up(const Inst& I, const Levels& L, int64_t w) {
    const int lane = threadIdx.x & 31;
    unsigned long long m = 0ull;
    {
        const int64_t c = ((w >> 5) << 5) + lane;
        if (c != w && c < I.n) m = I.key32[c];
    }
    for (int lev = 1; lev < I.nlev; ++lev) {
        const int64_t anc = w >> (5 * lev);
        const int64_t c = ((anc >> 5) << 5) + lane;
        if (c != anc && c < I.lvl_n[lev - 1]) {
            const unsigned long long v = L.p[lev - 1][c];
            m = v > m ? v : m;
        }
    }
    return warp_max_key(m);
}

struct Dirty {
    int32_t lv0[kDirtyCap];        // first-level nodes to rebuild
    int32_t up[2][kDirtyCap];      // upper-level nodes, one level at a time
    int32_t n0, nup[2];
};

// A leaf's key went from `old` to `nk`: a larger key is pushed up with atomic
// maxima on every ancestor; if the leaf held its
// first-level node's maximum and shrank, that node is queued for a rebuild.
__device__ __forceinline__ void leaf_changed(const Inst& I, const Levels& L, Dirty& D, int64_t i,
                                             unsigned long long old, unsigned long long nk) {
    if (nk > old) {
        int64_t node = i;
        for (int lev = 0; lev < I.nlev; ++lev) {
            node >>= 5;
            atomicMax(&L.p[lev][node], nk);
        }
    } else if (nk < old) {
        const int64_t node = i >> 5;
        if (L.p[0][node] == old) {
            const int q = atomicAdd(&D.n0, 1);
            if (q < kDirtyCap) D.lv0[q] = (int32_t)node;
        }
    }
}

// Rebuilds the queued nodes: all warps the first level, then warp 0 the levels
// above (few nodes), each queueing its parent when its maximum shrank and the
// parent held it. Call with every thread; returns with warp 0 possibly still
// working on the upper levels when `wait` is false.
__device__ void rebuild_dirty(const Inst& I, const Levels& L, Dirty& D, bool wait) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n0 = min(D.n0, kDirtyCap);
    for (int q = wid; q < n0; q += kNW) {
        const int64_t node = D.lv0[q];
        const unsigned long long old = L.p[0][node];
        const unsigned long long nv = warp_node(I, L, 0, node);
        if (lane == 0) {
            L.p[0][node] = nv;
            if (nv < old && I.nlev > 1 && L.p[1][node >> 5] == old) {
                const int r = atomicAdd(&D.nup[0], 1);
                if (r < kDirtyCap) D.up[0][r] = (int32_t)(node >> 5);
            }
        }
    }
    __syncthreads();
    if (wid == 0) {
        int cur = 0;
        for (int lev = 1; lev < I.nlev; ++lev) {
            const int nn = min(D.nup[cur], kDirtyCap);
            if (lane == 0) D.nup[cur ^ 1] = 0;
            __syncwarp();
            for (int q = 0; q < nn; ++q) {
                const int64_t node = D.up[cur][q];
                const unsigned long long old = L.p[lev][node];
                const unsigned long long nv = warp_node(I, L, lev, node);
                if (lane == 0) {
                    L.p[lev][node] = nv;
                    if (nv < old && lev + 1 < I.nlev && L.p[lev + 1][node >> 5] == old) {
                        const int r = D.nup[cur ^ 1]++;
                        if (r < kDirtyCap) D.up[cur ^ 1][r] = (int32_t)(node >> 5);
                    }
                }
                __syncwarp();
            }
            cur ^= 1;
        }
        if (lane == 0) {
            D.n0 = 0;
            D.nup[0] = 0;
            D.nup[1] = 0;
        }
    }
    if (wait) __syncthreads();
}

// Whole tree from the leaves (after a full rescan).
__device__ void rebuild_tree(const Inst& I, const Levels& L) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int lev = 0; lev < I.nlev; ++lev) {
        for (int64_t node = wid; node < I.lvl_n[lev]; node += kNW) {
            const unsigned long long v = warp_node(I, L, lev, node);
            if (lane == 0) L.p[lev][node] = v;
        }
        __syncthreads();
    }
}

// Key of island i from its current state (already loaded): returns the new key
// and writes lo (and, on the FP64 path, the exact value x).
template <int PREC>
__device__ __forceinline__ unsigned long long key_of(const Inst& I, int64_t i, uint32_t step,
                                                     int si, longlong2 h64, int2 h32,
                                                     float2 rbc, float2 e32, float2 th,
                                                     double hk, double2 e64, float* lo,
                                                     double* x64) {
    if constexpr (PREC == 1) {
        const float dp = __fmul_rn(__int2float_rn(h32.x), I.inv32);
        const float dq = __fmul_rn(__int2float_rn(h32.y), I.inv32);
        const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
        if (e.possible && !e.certain) {
            // within its band of the threshold or of the sign change: FP64 now
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
            const Eval64 f = eval64(I, si, h64.x, h64.y, hk, e64, tp, tq);
            const double x = f.flippable ? f.lhs : 0.0;
            *lo = x > 0.0 ? __double2float_rd(x) : -1.0f;
            return x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
        }
        *lo = e.certain ? e.lo : -1.0f;
        return e.possible ? key32_of(e.hi, i) : 0ull;
    } else {
        const float dp = __fmul_rn(__ll2float_rn(h64.x), I.inv64f);
        const float dq = __fmul_rn(__ll2float_rn(h64.y), I.inv64f);
        const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
        double x = 0.0;
        if (e.possible) {
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
            const Eval64 f = eval64(I, si, h64.x, h64.y, hk, e64, tp, tq);
            if (f.flippable) x = f.lhs;
        }
        *x64 = x;
        *lo = x > 0.0 ? __double2float_rd(x) : -1.0f;
        return x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
    }
}

// Island i's field changes by 2 s_new (dp, dq) (exact 64-bit sums; dp32, dq32 the
// 32-bit ones); its key is re-evaluated and the tree told. Every load is issued
// before the first store so that they overlap.
template <int PREC>
__device__ __forceinline__ void update_island(const Inst& I, const Levels& L, Dirty& D,
                                              int64_t i, int snew, long long dp, long long dq,
                                              int dp32, int dq32, uint32_t step) {
    longlong2 h = I.h64[i];
    int2 g = make_int2(0, 0);
    if constexpr (PREC == 1) g = I.h32[i];
    const unsigned long long old = I.key32[i];
    const int si = I.s[i];
    const uint16_t ci = __ldg(&I.cls[i]);
    const float2 rbc = __ldg(&I.rbc32[i]);
    float2 th = make_float2(0.0f, 0.0f);
    if (I.sigma > 0.0) th = I.th32[i];
    const double hk = __ldg(&I.hk64[i]);
    const double2 e64 = I.ext64[ci];
    const float2 e32 = I.ext32[ci];
    const unsigned long long up = 2ull * (unsigned long long)dp;
    const unsigned long long uq = 2ull * (unsigned long long)dq;
    h.x = (long long)(snew > 0 ? (unsigned long long)h.x + up : (unsigned long long)h.x - up);
    h.y = (long long)(snew > 0 ? (unsigned long long)h.y + uq : (unsigned long long)h.y - uq);
    if constexpr (PREC == 1) {
        const unsigned vp = 2u * (unsigned)dp32, vq = 2u * (unsigned)dq32;
        g.x = (int)(snew > 0 ? (unsigned)g.x + vp : (unsigned)g.x - vp);
        g.y = (int)(snew > 0 ? (unsigned)g.y + vq : (unsigned)g.y - vq);
    }
    float lo;
    double x = 0.0;
    const unsigned long long nk = key_of<PREC>(I, i, step, si, h, g, rbc, e32, th, hk, e64, &lo, &x);
    I.h64[i] = h;
    if constexpr (PREC == 1) I.h32[i] = g;
    if constexpr (PREC == 0) I.key64[i] = x;
    I.key32[i] = nk;
    I.lo32[i] = lo;
    leaf_changed(I, L, D, i, old, nk);
}

// Exact FP64 value of island i (0 when not flippable): on the FP64 path the value
// kept with its key, on the FP32 path a fresh FP64 evaluation of its exact sums.
template <int PREC>
__device__ __forceinline__ double exact_value(const Inst& I, int64_t i, uint32_t step) {
    if constexpr (PREC == 0) {
        return I.key64[i];
    } else {
        double tp = 0.0, tq = 0.0;
        if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
        const longlong2 h = I.h64[i];
        const Eval64 e = eval64(I, I.s[i], h.x, h.y, I.hk64[i], I.ext64[I.cls[i]], tp, tq);
        return e.flippable ? e.lhs : 0.0;
    }
}

struct RecheckShared {
    int32_t front[2][kRecheckCap];
    int32_t cand[kRecheckCap];
    double cand_val[kRecheckCap];
    unsigned long long cand_old[kRecheckCap];
    unsigned long long cand_new[kRecheckCap];
    int32_t result;
    float tau;
};

// Exact comparison of the islands whose key bound reaches tau, by warp 0 alone.
// Returns the winner (its exact value is at least tau, so nothing outside the set
// can beat it), -2 with R.tau lowered to widen the set, -1 when all of them were
// demoted, -3 when the set overflowed (nothing changed then).
template <int PREC>
__device__ int64_t recheck_warp(const Inst& I, const Levels& L, RecheckShared& R, float tau,
                                uint32_t step) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned long long tkey = (unsigned long long)__float_as_uint(tau) << 32;
    // descent from the root through every node whose maximum reaches tau
    if (lane == 0) R.front[0][0] = 0;
    __syncwarp();
    int cur = 0, nf = 1;
    for (int lev = I.nlev - 1; lev >= 0; --lev) {
        int nn = 0;
        for (int f = 0; f < nf; ++f) {
            const int64_t child = ((int64_t)R.front[cur][f] << 5) + lane;
            unsigned long long k = 0ull;
            if (lev > 0) {
                if (child < I.lvl_n[lev - 1]) k = L.p[lev - 1][child];
            } else if (child < I.n) {
                k = I.key32[child];
            }
            const bool hit = k != 0ull && k >= tkey;
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            const int pos = nn + __popc(m & lt);
            if (hit && pos < kRecheckCap) R.front[cur ^ 1][pos] = (int32_t)child;
            nn += __popc(m);
        }
        __syncwarp();
        if (nn > kRecheckCap) return -3;
        cur ^= 1;
        nf = nn;
    }
    const int nc = nf;
    // exact values, one lane per candidate; best by (value, lowest index)
    unsigned long long bv = 0ull;
    int64_t bi = -1;
    for (int c = lane; c < nc; c += 32) {
        const int64_t i = R.front[cur][c];
        const double v = exact_value<PREC>(I, i, step);
        R.cand[c] = (int32_t)i;
        R.cand_val[c] = v;
        const unsigned long long vb = v > 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull;
        if (vb > 0ull && (bi < 0 || vb > bv || (vb == bv && i < bi))) {
            bv = vb;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ov > bv || (ov == bv && oi < bi))) {
            bv = ov;
            bi = oi;
        }
    }
    // Demote what proved non-flippable; give the flippable ones keys from their
    // exact values (valid until their field changes). Both only lower keys.
    for (int c = lane; c < nc; c += 32) {
        const int64_t i = R.cand[c];
        const double v = R.cand_val[c];
        const unsigned long long old = I.key32[i];
        const unsigned long long nk = v > 0.0 ? key32_of(__double2float_ru(v), i) : 0ull;
        I.key32[i] = nk;
        I.lo32[i] = v > 0.0 ? __double2float_rd(v) : -1.0f;
        R.cand_old[c] = old;
        R.cand_new[c] = nk;
    }
    __syncwarp();
    // rebuild the nodes whose maximum was a lowered key, bottom-up
    for (int c = 0; c < nc; ++c) {
        const unsigned long long old = R.cand_old[c];
        if (R.cand_new[c] >= old) continue;
        int64_t node = (int64_t)R.cand[c];
        for (int lev = 0; lev < I.nlev; ++lev) {
            node >>= 5;
            if (L.p[lev][node] != old) break;
            const unsigned long long nv = warp_node(I, L, lev, node);
            if (lane == 0) L.p[lev][node] = nv;
            __syncwarp();
        }
    }
    const double bl = __longlong_as_double((long long)bv);
    if (bi >= 0 && bl >= (double)tau) return bi;
    if (bi >= 0) {
        if (lane == 0) R.tau = __double2float_rd(bl);  // something outside might beat it
        __syncwarp();
        return -2;
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
        I.lo32[i] = v > 0.0 ? __double2float_rd(v) : -1.0f;
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

template <int PREC>
__global__ void __launch_bounds__(kT, 1)
    k_relax(const Inst* __restrict__ tab, const int32_t* __restrict__ work, int n_work,
            int smem_budget) {
    extern __shared__ unsigned long long sm_levels[];
    __shared__ int64_t sh_k;
    __shared__ int64_t sh_e0, sh_e1;
    __shared__ int32_t sh_snew;
    __shared__ float sh_tau;
    __shared__ RecheckShared R;
    __shared__ Dirty D;

    const Inst& I = tab[work[blockIdx.x]];
    InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;
    const uint32_t step = I.step0 + (uint32_t)t;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    // Place the upper tree levels in shared memory while they fit.
    Levels L;
    {
        int64_t used = 0;
        int first_sm = I.nlev;
        for (int lev = I.nlev - 1; lev >= 0; --lev) {
            const int64_t b = (int64_t)I.lvl_n[lev] * (int64_t)sizeof(unsigned long long);
            if (used + b > smem_budget) break;
            used += b;
            first_sm = lev;
        }
        int64_t off = 0;
        for (int lev = I.nlev - 1; lev >= 0; --lev) {
            if (lev >= first_sm) {
                L.p[lev] = sm_levels + off;
                off += I.lvl_n[lev];
            } else {
                L.p[lev] = I.tree + I.lvl_off[lev];
            }
        }
        for (int lev = first_sm; lev < I.nlev; ++lev)
            for (int64_t q = threadIdx.x; q < I.lvl_n[lev]; q += kT)
                L.p[lev][q] = I.tree[I.lvl_off[lev] + q];
        if (threadIdx.x == 0) {
            D.n0 = 0;
            D.nup[0] = 0;
            D.nup[1] = 0;
        }
    }
    __syncthreads();

    int64_t flips = 0;
    int32_t status = ST_OK;
    int rounds = 0;
    uint64_t hash = threadIdx.x == 0 ? st->hash : 0ull;
    const int64_t flips_before = threadIdx.x == 0 ? st->n_flips : 0;
    const int64_t max_flips = I.max_flips;

    // Thread 0: flip island k, log it, fold it into the hash, publish its row.
    auto do_flip = [&](int64_t k, int sk, int64_t a0, int64_t a1) {
        const int snew = -sk;
        I.s[k] = (int8_t)snew;
        sh_snew = snew;
        sh_e0 = a0;
        sh_e1 = a1;
        const int64_t q = flips_before + flips;
        if (I.log_spin && q < I.log_cap) {
            I.log_step[q] = step;
            I.log_spin[q] = (uint32_t)k;
        }
        hash = fnv_flip(hash, step, (uint32_t)k);
    };

    for (;;) {
        // pick, and flip when the pick is certain: warp 0
        if (wid == 0) {
            const unsigned long long root = L.p[I.nlev - 1][0];
            int64_t k = -1;
            if (root != 0ull) {
                const int64_t w = key32_idx(root);
                float lo = 0.0f;
                int sw = 0;
                int64_t a0 = 0, a1 = 0;
                if (lane == 0) {  // independent loads, in flight during the runner-up scan
                    lo = I.lo32[w];
                    sw = I.s[w];
                    a0 = I.rp[w];
                    a1 = I.rp[w + 1];
                }
                const unsigned long long ru = runner_up(I, L, w);
                if (lane == 0) {
                    const float hi2 = ru ? key32_hi(ru) : 0.0f;
                    if (lo > 1.0f && lo > hi2) {
                        if (flips < max_flips) {
                            do_flip(w, sw, a0, a1);
                            k = w;
                        } else {
                            k = -6;
                        }
                    } else {
                        k = -2;
                        sh_tau = fmaxf(hi2, lo);
                    }
                }
            }
            if (lane == 0) sh_k = k;
        }
        __syncthreads();
        int64_t k = sh_k;
        if (k == -2) {
            float tau = sh_tau;
            while (k == -2) {
                if (++rounds > 64) {
                    k = -4;
                    break;
                }
                if (wid == 0) {
                    const int64_t r = recheck_warp<PREC>(I, L, R, tau, step);
                    if (lane == 0) {
                        R.result = (int32_t)r;
                        atomicAdd((unsigned long long*)&st->rechecks, 1ull);
                    }
                }
                __syncthreads();
                int64_t r = R.result;
                if (r == -3) {
                    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&st->fallbacks, 1ull);
                    r = recheck_scan<PREC>(I, L, R, tau, step);
                }
                tau = R.tau;
                if (r == -1) {
                    k = -5;  // everything examined was demoted: look at the root again
                    rounds = 0;
                } else {
                    k = r;  // the winner, or -2 to widen
                }
                __syncthreads();
            }
            if (k == -5) continue;
            if (k == -4) {
                status = ST_BOUNDS;
                break;
            }
            if (k >= 0) {
                if (threadIdx.x == 0) {
                    if (flips < max_flips)
                        do_flip(k, I.s[k], I.rp[k], I.rp[k + 1]);
                    else
                        sh_k = -6;
                }
                __syncthreads();
                if (sh_k == -6) k = -6;
            }
        }
        rounds = 0;
        if (k == -6) {
            status = ST_NOT_CONVERGED;
            break;
        }
        if (k < 0) break;
        ++flips;
        // every neighbour i of k: add 2 s_k(new) (P_ik, Q_ik), new key, tree update
        const int snew = sh_snew;
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
            update_island<PREC>(I, L, D, i, snew, dp, dq, dp32, dq32, step);
        }
        if (threadIdx.x == kT - 1)  // k's own field is unchanged; its key is not
            update_island<PREC>(I, L, D, k, snew, 0, 0, 0, 0, step);
        __syncthreads();
        rebuild_dirty(I, L, D, false);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (I.flips_per_step) I.flips_per_step[t] = flips;
        st->n_flips = flips_before + flips;
        st->hash = hash;
        if (status != ST_OK) st->status = status;
        st->init = 0;
        st->t = t + 1;
    }
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
    const int si = I.s[i];
    const uint16_t ci = I.cls[i];
    const double2 ext = ext_proj(hx, hy, I.cs64[ci]);
    if (I.prec == 1) {
        const int2 h = I.h32[i];
        const float2 th = I.sigma > 0.0 ? thermal32(I, i, step) : make_float2(0.0f, 0.0f);
        const Eval32 e = eval32(I, si, __fmul_rn(__int2float_rn(h.x), I.inv32),
                                __fmul_rn(__int2float_rn(h.y), I.inv32), I.rbc32[i],
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
        const Eval64 e = eval64(I, si, h.x, h.y, I.hk64[i], ext, tp, tq);
        hpar[i] = e.hpar;
        hperp[i] = e.hperp;
        lhs[i] = e.lhs;
        lo[i] = e.lhs;
        hi[i] = e.lhs;
    }
}

}  // namespace

int relax_threads() { return kT; }

size_t relax_static_smem(int prec) {
    cudaFuncAttributes a{};
    if (prec == 1)
        cudaFuncGetAttributes(&a, k_relax<1>);
    else
        cudaFuncGetAttributes(&a, k_relax<0>);
    return a.sharedSizeBytes;
}

// Sets the dynamic shared-memory limit of the relax kernel once per size (a
// no-op afterwards, so launches can be captured in graphs).
cudaError_t prepare_relax(int prec, int smem) {
    static int set_bytes[2] = {-1, -1};
    const int k = prec == 1 ? 1 : 0;
    if (set_bytes[k] >= smem) return cudaSuccess;
    const cudaError_t e =
        prec == 1 ? cudaFuncSetAttribute(k_relax<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem)
                  : cudaFuncSetAttribute(k_relax<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e == cudaSuccess) set_bytes[k] = smem;
    return e;
}

cudaError_t launch_relax(const RelaxLaunch& L, cudaStream_t st) {
    if (L.n_work == 0) return cudaSuccess;
    const cudaError_t e = prepare_relax(L.prec, L.smem_budget);
    if (e != cudaSuccess) return e;
    if (L.prec == 1)
        k_relax<1><<<L.n_work, kT, L.smem_budget, st>>>(L.tab, L.work, L.n_work, L.smem_budget);
    else
        k_relax<0><<<L.n_work, kT, L.smem_budget, st>>>(L.tab, L.work, L.n_work, L.smem_budget);
    return cudaGetLastError();
}

cudaError_t launch_eval_all(const Inst* tab, int64_t n, double hx, double hy, uint32_t step,
                            double* out5, cudaStream_t st) {
    k_eval_all<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tab, hx, hy, step, out5, out5 + n,
                                                           out5 + 2 * n, out5 + 3 * n,
                                                           out5 + 4 * n);
    return cudaGetLastError();
}

}  // namespace fs
