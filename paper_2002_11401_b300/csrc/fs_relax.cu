// fs_relax.cu - the greedy single-flip relaxation (Sec. "Dynamics"), one CTA per
// simulation, entirely on the device.
//
// Per flip: read the root of the max-tree (largest Eq. 5 LHS among flippable
// islands, lowest index on ties); flip that island k; for every neighbour i of k
// (row k of the CSR, whose transposed coefficients give the field k puts on i in
// i's frame) add 2 s_k(new) (P_ik, Q_ik) to i's exact fixed-point dipolar sums and
// re-evaluate i's key; then rebuild only the tree nodes above the changed leaves,
// level by level. The fields stay constant over the relax, as the paper states.
//
// FS_FP32_RECHECK: keys are FP32 upper bounds of the LHS, nodes keep the best two
// keys. The root's island is accepted when its certified lower bound exceeds one
// and the runner-up's upper bound; otherwise every island whose upper bound
// reaches the threshold is re-evaluated with the FS_FP64 arithmetic (exact
// 64-bit sum of its CSR row), non-flippable ones are demoted, and the FP64 best
// is taken once no island outside the set can beat it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"
#include "fs_kernels.h"

namespace fs {

namespace {

constexpr int kT = 512;  // threads per relax CTA

struct Levels {
    ulonglong2* p[kMaxLevels];
};

__device__ __forceinline__ ulonglong2 best64n(ulonglong2 a, ulonglong2 b) {
    return better64(a.x, a.y, b.x, b.y) ? a : b;
}

template <int PREC>
__device__ __forceinline__ ulonglong2 empty_node() {
    if constexpr (PREC == 1)
        return make_ulonglong2(0ull, 0ull);
    else
        return make_ulonglong2(0ull, 0xFFFFFFFFFFFFFFFFull);
}

template <int PREC>
__device__ __forceinline__ ulonglong2 merge_node(ulonglong2 a, ulonglong2 b) {
    if constexpr (PREC == 1)
        return top2(a, b);
    else
        return best64n(a, b);
}

// Node `node` of level `lev` from its 32 children (leaves when lev == 0), one
// child per lane and a shuffle butterfly; every lane returns the node.
template <int PREC>
__device__ __forceinline__ ulonglong2 warp_children(const Inst& I, const Levels& L, int lev,
                                                    int64_t node) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (node << 5) + lane;
    ulonglong2 v = empty_node<PREC>();
    if (lev == 0) {
        if (c < I.n) {
            if constexpr (PREC == 1)
                v = make_ulonglong2(I.key32[c], 0ull);
            else
                v = make_ulonglong2((unsigned long long)__double_as_longlong(I.key64[c]),
                                    (unsigned long long)c);
        }
    } else if (c < I.lvl_n[lev - 1]) {
        v = L.p[lev - 1][c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ulonglong2 u;
        u.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        u.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = merge_node<PREC>(v, u);
    }
    return v;
}

// Warp-wide: the distinct parents (x >> 5) of in[0..nin) in order, written to
// out. Entries < 0 are skipped. `in` is ascending except that its last entry may
// be out of place; that entry's parent is checked against all others.
__device__ int warp_parents(const int32_t* in, int nin, int32_t* out) {
    const int lane = threadIdx.x & 31;
    int cnt = 0;
    int carry = -1;
    for (int base = 0; base < nin; base += 32) {
        const int t = base + lane;
        const int p = (t < nin && in[t] >= 0) ? (in[t] >> 5) : -1;
        int up = __shfl_up_sync(0xffffffffu, p, 1);
        if (lane == 0) up = carry;
        const bool first = p >= 0 && p != up;
        const unsigned m = __ballot_sync(0xffffffffu, first);
        if (first) out[cnt + __popc(m & ((1u << lane) - 1u))] = p;
        cnt += __popc(m);
        carry = __shfl_sync(0xffffffffu, p, 31);
    }
    __syncwarp();
    if (cnt >= 2) {
        const int last = out[cnt - 1];
        bool dup = false;
        for (int base = 0; base < cnt - 1; base += 32) {
            const int t = base + lane;
            dup |= __any_sync(0xffffffffu, t < cnt - 1 && out[t] == last);
        }
        if (dup) --cnt;
    }
    __syncwarp();
    return cnt;
}

struct TreeScratch {
    int32_t nodes[2][kMaxPaddedDegree + 2];
    int32_t n1;
};

// Re-derives the tree above the changed leaves list[0..len) (ascending except the
// last entry; entries < 0 skipped): all warps rebuild the first level, one warp
// per node; then warp 0 alone climbs the few upper levels. Ends with warp 0 still
// working; the caller's next block barrier orders it before any reader.
template <int PREC>
__device__ void tree_update_sorted(const Inst& I, const Levels& L, TreeScratch& T,
                                   const int32_t* list, int len) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid == 0) {
        const int n1 = warp_parents(list, len, T.nodes[0]);
        if (lane == 0) T.n1 = n1;
    }
    __syncthreads();
    const int n1 = T.n1;
    for (int q = wid; q < n1; q += kT / 32) {
        const int64_t node = T.nodes[0][q];
        const ulonglong2 v = warp_children<PREC>(I, L, 0, node);
        if (lane == 0) L.p[0][node] = v;
    }
    __syncthreads();
    if (wid == 0) {
        int cur = 0, ncur = n1;
        for (int lev = 1; lev < I.nlev; ++lev) {
            const int nn = warp_parents(T.nodes[cur], ncur, T.nodes[cur ^ 1]);
            for (int q = 0; q < nn; ++q) {
                const int64_t node = T.nodes[cur ^ 1][q];
                const ulonglong2 v = warp_children<PREC>(I, L, lev, node);
                if (lane == 0) L.p[lev][node] = v;
                __syncwarp();
            }
            cur ^= 1;
            ncur = nn;
        }
    }
}

// Whole tree from the leaves (after a full rescan).
template <int PREC>
__device__ void rebuild_tree(const Inst& I, const Levels& L) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int lev = 0; lev < I.nlev; ++lev) {
        for (int64_t node = wid; node < I.lvl_n[lev]; node += kT / 32) {
            const ulonglong2 v = warp_children<PREC>(I, L, lev, node);
            if (lane == 0) L.p[lev][node] = v;
        }
        __syncthreads();
    }
}

// Key of island i at the current spins and fields (FP32 path writes key32/lo32,
// FP64 path key64).
template <int PREC>
__device__ __forceinline__ void rekey(const Inst& I, int64_t i, uint32_t step) {
    const int si = I.s[i];
    const uint16_t ci = I.cls[i];
    float2 th = make_float2(0.0f, 0.0f);
    if (I.sigma > 0.0) th = I.th32[i];
    const float2 e32 = I.ext32[ci];
    if constexpr (PREC == 1) {
        const int2 h = I.h32[i];
        const float dp = __fmul_rn(__int2float_rn(h.x), I.inv32);
        const float dq = __fmul_rn(__int2float_rn(h.y), I.inv32);
        const Eval32 e = eval32(I, si, dp, dq, I.hk32[i], e32, th.x, th.y);
        I.key32[i] = e.possible ? key32_of(e.hi, i) : 0ull;
        I.lo32[i] = e.certain ? e.lo : -1.0f;
    } else {
        const longlong2 h = I.h64[i];
        const float dp = __fmul_rn(__ll2float_rn(h.x), I.inv64f);
        const float dq = __fmul_rn(__ll2float_rn(h.y), I.inv64f);
        const Eval32 e = eval32(I, si, dp, dq, I.hk32[i], e32, th.x, th.y);
        double key = 0.0;
        if (e.possible) {
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
            const Eval64 f = eval64(I, si, h.x, h.y, I.hk64[i], I.ext64[ci], tp, tq);
            if (f.flippable) key = f.lhs;
        }
        I.key64[i] = key;
    }
}

// Exact FP64 evaluation of island i from its exact 64-bit sums.
__device__ __forceinline__ Eval64 exact_eval(const Inst& I, int64_t i, uint32_t step) {
    double tp = 0.0, tq = 0.0;
    if (I.sigma > 0.0) thermal64(I, i, step, &tp, &tq);
    const longlong2 h = I.h64[i];
    return eval64(I, I.s[i], h.x, h.y, I.hk64[i], I.ext64[I.cls[i]], tp, tq);
}

struct RecheckShared {
    int32_t front[2][kRecheckCap];
    int32_t nfront[2];
    int32_t cand[kRecheckCap];
    double cand_lhs[kRecheckCap];
    int32_t cand_ok[kRecheckCap];
    int32_t sorted[kRecheckCap];
    int32_t nsorted;
    int32_t overflow;
    int32_t result;
    float tau;
};

// Finds the FP64 winner among islands whose FP32 upper bound reaches tau, or
// demotes what it proves non-flippable. Returns the winner, -1 when the caller
// should look at the root again, -3 on a recheck-round overflow (fallback used).
__device__ int64_t recheck_round(const Inst& I, const Levels& L, RecheckShared& R,
                                 TreeScratch& T, float tau, uint32_t step) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long tkey = (unsigned long long)__float_as_uint(tau) << 32;
    if (threadIdx.x == 0) {
        R.front[0][0] = 0;
        R.nfront[0] = 1;
        R.nfront[1] = 0;
        R.overflow = 0;
    }
    __syncthreads();
    int cur = 0;
    for (int lev = I.nlev - 1; lev >= 0; --lev) {
        const int nf = R.nfront[cur];
        for (int f = wid; f < nf; f += kT / 32) {
            const int64_t node = R.front[cur][f];
            const int64_t child = (node << 5) + lane;
            bool hit = false;
            if (lev > 0) {
                if (child < I.lvl_n[lev - 1]) hit = L.p[lev - 1][child].x >= tkey;
            } else {
                if (child < I.n) {
                    const unsigned long long k = I.key32[child];
                    hit = k != 0ull && k >= tkey;
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&R.nfront[cur ^ 1], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (hit) {
                const int pos = base + __popc(m & ((1u << lane) - 1u));
                if (pos < kRecheckCap)
                    R.front[cur ^ 1][pos] = (int32_t)child;
                else
                    R.overflow = 1;
            }
        }
        __syncthreads();
        if (R.overflow) break;
        if (threadIdx.x == 0) R.nfront[cur] = 0;
        cur ^= 1;
        __syncthreads();
    }
    if (R.overflow) return -3;
    const int nc = R.nfront[cur];
    // exact evaluation, one thread per candidate
    for (int c = threadIdx.x; c < nc; c += kT) {
        const int64_t i = R.front[cur][c];
        const Eval64 e = exact_eval(I, i, step);
        R.cand[c] = (int32_t)i;
        R.cand_lhs[c] = e.lhs;
        R.cand_ok[c] = e.flippable;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t best = -1;
        double bl = 0.0;
        for (int c = 0; c < nc; ++c) {
            if (!R.cand_ok[c]) continue;
            const int64_t i = R.cand[c];
            if (best < 0 || R.cand_lhs[c] > bl || (R.cand_lhs[c] == bl && i < best)) {
                best = i;
                bl = R.cand_lhs[c];
            }
        }
        if (best >= 0 && bl >= (double)tau) {
            R.result = (int32_t)best;
        } else if (best >= 0) {
            // something outside the set might beat it: widen to its value
            R.result = -2;
            R.tau = __double2float_rd(bl);
        } else {
            R.result = -1;
        }
    }
    __syncthreads();
    // Demote proven non-flippable candidates; give the flippable ones the tight
    // bounds of their exact value (valid until their field changes). Then refresh
    // the tree above them.
    for (int c = threadIdx.x; c < nc; c += kT) {
        const int64_t i = R.cand[c];
        if (!R.cand_ok[c]) {
            I.key32[i] = 0ull;
            I.lo32[i] = -1.0f;
        } else {
            I.key32[i] = key32_of(__double2float_ru(R.cand_lhs[c]), i);
            I.lo32[i] = __double2float_rd(R.cand_lhs[c]);
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nc; c += kT) {
        const int32_t v = R.cand[c];
        int rank = 0;
        for (int u = 0; u < nc; ++u) rank += R.cand[u] < v;
        R.sorted[rank] = v;
    }
    if (threadIdx.x == 0) R.nsorted = nc;
    __syncthreads();
    tree_update_sorted<1>(I, L, T, R.sorted, R.nsorted);
    __syncthreads();
    return R.result;
}

// Fallback when the candidate set overflows: every island with a key at or above
// tau is evaluated exactly, by one thread each.
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
        const Eval64 e = exact_eval(I, i, step);
        if (!e.flippable) {
            I.key32[i] = 0ull;
            I.lo32[i] = -1.0f;
        } else {
            I.key32[i] = key32_of(__double2float_ru(e.lhs), i);
            I.lo32[i] = __double2float_rd(e.lhs);
            if (bi < 0 || e.lhs > bl || (e.lhs == bl && i < bi)) {
                bl = e.lhs;
                bi = i;
            }
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
    rebuild_tree<1>(I, L);
    return R.result;
}

template <int PREC>
__global__ void __launch_bounds__(kT, 1)
    k_relax(const Inst* __restrict__ tab, const int32_t* __restrict__ work, int n_work,
            int smem_budget) {
    extern __shared__ ulonglong2 sm_levels[];
    __shared__ int32_t list[kMaxPaddedDegree + 1];
    __shared__ int64_t sh_k;
    __shared__ int64_t sh_e0, sh_e1;
    __shared__ int32_t sh_snew;
    __shared__ float sh_tau;
    __shared__ RecheckShared R;
    __shared__ TreeScratch T;

    const Inst& I = tab[work[blockIdx.x]];
    InstState* st = I.st;
    const int64_t t = st->t;
    if (st->status != ST_OK || t >= I.K) return;
    const uint32_t step = I.step0 + (uint32_t)t;

    // Place the upper tree levels in shared memory while they fit.
    Levels L;
    {
        int64_t used = 0;
        int first_sm = I.nlev;
        for (int lev = I.nlev - 1; lev >= 0; --lev) {
            const int64_t b = (int64_t)I.lvl_n[lev] * (int64_t)sizeof(ulonglong2);
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
    }
    __syncthreads();

    int64_t flips = 0;
    int32_t status = ST_OK;
    int rounds = 0;
    uint64_t hash = threadIdx.x == 0 ? st->hash : 0ull;
    const int64_t flips_before = threadIdx.x == 0 ? st->n_flips : 0;
    const int64_t max_flips = I.max_flips;

    // Thread 0: flip island k (Sec. "Dynamics"), log it, fold it into the hash and
    // publish its CSR row for the neighbour update.
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
        // pick (and, when the pick is certain, flip) in one step of thread 0
        if (threadIdx.x == 0) {
            const ulonglong2 root = L.p[I.nlev - 1][0];
            int64_t k = -1;
            if (root.x != 0ull) {
                const int64_t w = PREC == 1 ? (int64_t)key32_idx(root.x) : (int64_t)root.y;
                // independent loads, issued together
                const int sw = I.s[w];
                const int64_t a0 = I.rp[w], a1 = I.rp[w + 1];
                if constexpr (PREC == 1) {
                    const float lo = I.lo32[w];
                    const float hi2 = root.y ? key32_hi(root.y) : 0.0f;
                    if (lo > 1.0f && lo > hi2) {
                        k = w;
                    } else {
                        k = -2;
                        sh_tau = fmaxf(hi2, lo);
                    }
                } else {
                    k = w;
                }
                if (k >= 0) {
                    if (flips < max_flips)
                        do_flip(k, sw, a0, a1);
                    else
                        k = -6;
                }
            }
            sh_k = k;
        }
        __syncthreads();
        int64_t k = sh_k;
        if constexpr (PREC == 1) {
            if (k == -2) {
                float tau = sh_tau;
                while (k == -2) {
                    if (++rounds > 64) {
                        k = -4;
                        break;
                    }
                    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&st->rechecks, 1ull);
                    int64_t r = recheck_round(I, L, R, T, tau, step);
                    if (r == -3) {
                        if (threadIdx.x == 0)
                            atomicAdd((unsigned long long*)&st->fallbacks, 1ull);
                        r = recheck_scan(I, L, R, tau, step);
                    }
                    __syncthreads();
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
        }
        rounds = 0;
        if (k == -6) {
            status = ST_NOT_CONVERGED;
            break;
        }
        if (k < 0) break;
        ++flips;
        // every neighbour i of k: add 2 s_k(new) (P_ik, Q_ik) and re-evaluate i
        const int snew = sh_snew;
        const int64_t e0 = sh_e0;
        const int len = (int)(sh_e1 - e0);
        for (int q = threadIdx.x; q < len; q += kT) {
            const int64_t e = e0 + q;
            const int32_t i = I.col[e];
            if (i == (int32_t)k) {
                list[q] = -1;  // row padding
                continue;
            }
            {
                longlong2 h = I.h64[i];
                const unsigned long long up = 2ull * (unsigned long long)I.pq64[e].x;
                const unsigned long long uq = 2ull * (unsigned long long)I.qt64[e];
                h.x = (long long)(snew > 0 ? (unsigned long long)h.x + up
                                           : (unsigned long long)h.x - up);
                h.y = (long long)(snew > 0 ? (unsigned long long)h.y + uq
                                           : (unsigned long long)h.y - uq);
                I.h64[i] = h;
            }
            if constexpr (PREC == 1) {
                int2 h = I.h32[i];
                const unsigned up = 2u * (unsigned)I.pq32[e].x, uq = 2u * (unsigned)I.qt32[e];
                h.x = (int)(snew > 0 ? (unsigned)h.x + up : (unsigned)h.x - up);
                h.y = (int)(snew > 0 ? (unsigned)h.y + uq : (unsigned)h.y - uq);
                I.h32[i] = h;
            }
            rekey<PREC>(I, i, step);
            list[q] = i;
        }
        if (threadIdx.x == kT - 1) {
            rekey<PREC>(I, k, step);
            list[len] = (int32_t)k;
        }
        __syncthreads();
        tree_update_sorted<PREC>(I, L, T, list, len + 1);
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
                                __fmul_rn(__int2float_rn(h.y), I.inv32), I.hk32[i],
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
