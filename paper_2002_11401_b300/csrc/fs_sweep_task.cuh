// fs_sweep_task.cuh - one task of the field-and-margin sweep (Sec. "Dynamics": at
// each simulation step the total field on every island is calculated; Eq. 2, 3,
// 5, 6): the 32 consecutive islands of one first-level tree node, swept by one
// warp. Shared by the sweep kernel (every task of a field step in one launch) and
// the persistent batch kernel (tasks claimed by whichever CTA is free).
//
// Sub-warps of W lanes stream one CSR row each: every lane reads a group of four
// entries with 16-byte loads (column indices, or on the FP32 path their 16-bit
// offsets from the row's island in 8 bytes, then the fixed-point (P, Q)
// coefficients), gathers the four spins, and accumulates the exact integer sums
// s_j P_ij and s_j Q_ij; a shuffle butterfly inside the sub-warp finishes the row.
// The per-row sums are staged in shared memory so that lane q then evaluates
// island q: external and thermal fields, Eq. 5/6, the argmax key. A warp max
// gives the first tree level; the last warp to finish a group of 32 sibling
// nodes builds their parent (fenced counter), up to the root.
//
// With resweep off, the exact sums kept up to date by the flips are read instead
// of recomputed; integer sums make both modes bit-identical.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"
#include "fs_update.cuh"

namespace fs {
namespace {

constexpr int kSweepThreads = 256;
constexpr int kSweepWarps = kSweepThreads / 32;

__device__ __forceinline__ int find_inst(const int64_t* __restrict__ start, int n_inst,
                                         int64_t task) {
    int lo = 0, hi = n_inst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= task)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int sgn_sel(int8_t s, int v) { return s > 0 ? v : -v; }
__device__ __forceinline__ long long sgn_sel(int8_t s, long long v) { return s > 0 ? v : -v; }

// Called by a full warp after lane 0 wrote node `idx` of level `lev`: the last
// of its siblings to arrive builds the parent, and so on up to the root. Returns
// true on the warp that built (or, for a one-node tree, wrote) the root.
__device__ bool propagate_up(const Inst& I, unsigned* __restrict__ tcnt, int lev, int64_t idx) {
    const int lane = threadIdx.x & 31;
    while (lev + 1 < I.nlev) {
        const int64_t parent = idx >> 5;
        const int64_t first = parent << 5;
        const int64_t last = min((int64_t)I.lvl_n[lev], first + 32);
        const unsigned nchild = (unsigned)(last - first);
        __threadfence();
        unsigned old = 0;
        if (lane == 0) old = atomicAdd(&tcnt[I.lvl_off[lev + 1] + parent], 1u);
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old + 1 != nchild) return false;
        if (lane == 0) tcnt[I.lvl_off[lev + 1] + parent] = 0u;
        __threadfence();
        unsigned long long v = 0ull;
        if (first + lane < last) v = __ldcg(&I.tree[I.lvl_off[lev] + first + lane]);
        v = warp_max_key(v);
        if (lane == 0) I.tree[I.lvl_off[lev + 1] + parent] = v;
        ++lev;
        idx = parent;
    }
    return true;
}

// The FP32 sums alone (the FP32 path's sweeps after the first) for the 32 rows from
// r0: a sub-warp's rows two at a time (q and q + R; the sub-warp holds W rows, an
// even number), their groups loaded side by side so that twice a lane's loads are
// in flight; a row past its end contributes zero coefficients. D16: the columns
// come from the 16-bit offsets (I.dcol, 8 bytes a group of four) instead of col
// (16 bytes). Results to s32[q] by the sub-warp's first lane.
template <int W, bool COHERENT, bool D16>
__device__ __forceinline__ void sum32_rows(const Inst& I, int64_t r0, int (*s32)[2]) {
    constexpr int R = 32 / W;
    const int lane = threadIdx.x & 31;
    const int sub = lane / W, sl = lane % W;
    const int4* __restrict__ col4 = reinterpret_cast<const int4*>(I.col);
    const int2* __restrict__ dcol4 = reinterpret_cast<const int2*>(I.dcol);
    for (int q = sub; q < 32; q += 2 * R) {
        const int64_t ia = r0 + q, ib = r0 + q + R;
        int64_t ga = 0, ea = 0, gb = 0, eb = 0;
        if (ia < I.n) {
            ga = (__ldg(&I.rp[ia]) >> 2) + sl;
            ea = __ldg(&I.rp[ia + 1]) >> 2;
        }
        if (ib < I.n) {
            gb = (__ldg(&I.rp[ib]) >> 2) + sl;
            eb = __ldg(&I.rp[ib + 1]) >> 2;
        }
        int bpa = 0, bqa = 0, bpb = 0, bqb = 0;
        for (; ga < ea || gb < eb; ga += W, gb += W) {
            const bool va = ga < ea, vb = gb < eb;
            const int4 z4 = make_int4(0, 0, 0, 0);
            int4 ca = z4, cb = z4;
            if constexpr (D16) {
                // four offsets in 8 bytes, added to the row's island
                const int2 da = va ? __ldg(&dcol4[ga]) : make_int2(0, 0);
                const int2 db = vb ? __ldg(&dcol4[gb]) : make_int2(0, 0);
                ca = make_int4((int)ia + (int)(short)(da.x & 0xffff), (int)ia + (da.x >> 16),
                               (int)ia + (int)(short)(da.y & 0xffff), (int)ia + (da.y >> 16));
                cb = make_int4((int)ib + (int)(short)(db.x & 0xffff), (int)ib + (db.x >> 16),
                               (int)ib + (int)(short)(db.y & 0xffff), (int)ib + (db.y >> 16));
            } else {
                ca = va ? __ldg(&col4[ga]) : z4;
                cb = vb ? __ldg(&col4[gb]) : z4;
            }
            const int4* pa = reinterpret_cast<const int4*>(I.pq32) + 2 * ga;
            const int4* pb = reinterpret_cast<const int4*>(I.pq32) + 2 * gb;
            const int4 xa = va ? __ldg(pa) : z4, ya = va ? __ldg(pa + 1) : z4;
            const int4 xb = vb ? __ldg(pb) : z4, yb = vb ? __ldg(pb + 1) : z4;
            int8_t a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
            if constexpr (COHERENT) {
                if (va) {
                    a0 = I.s[ca.x];
                    a1 = I.s[ca.y];
                    a2 = I.s[ca.z];
                    a3 = I.s[ca.w];
                }
                if (vb) {
                    b0 = I.s[cb.x];
                    b1 = I.s[cb.y];
                    b2 = I.s[cb.z];
                    b3 = I.s[cb.w];
                }
            } else {
                if (va) {
                    a0 = __ldg(&I.s[ca.x]);
                    a1 = __ldg(&I.s[ca.y]);
                    a2 = __ldg(&I.s[ca.z]);
                    a3 = __ldg(&I.s[ca.w]);
                }
                if (vb) {
                    b0 = __ldg(&I.s[cb.x]);
                    b1 = __ldg(&I.s[cb.y]);
                    b2 = __ldg(&I.s[cb.z]);
                    b3 = __ldg(&I.s[cb.w]);
                }
            }
            bpa += sgn_sel(a0, xa.x) + sgn_sel(a1, xa.z) + sgn_sel(a2, ya.x) +
                   sgn_sel(a3, ya.z);
            bqa += sgn_sel(a0, xa.y) + sgn_sel(a1, xa.w) + sgn_sel(a2, ya.y) +
                   sgn_sel(a3, ya.w);
            bpb += sgn_sel(b0, xb.x) + sgn_sel(b1, xb.z) + sgn_sel(b2, yb.x) +
                   sgn_sel(b3, yb.z);
            bqb += sgn_sel(b0, xb.y) + sgn_sel(b1, xb.w) + sgn_sel(b2, yb.y) +
                   sgn_sel(b3, yb.w);
        }
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            bpa += __shfl_xor_sync(0xffffffffu, bpa, o);
            bqa += __shfl_xor_sync(0xffffffffu, bqa, o);
            bpb += __shfl_xor_sync(0xffffffffu, bpb, o);
            bqb += __shfl_xor_sync(0xffffffffu, bqb, o);
        }
        if (sl == 0) {
            s32[q][0] = bpa;
            s32[q][1] = bqa;
            s32[q + R][0] = bpb;
            s32[q + R][1] = bqb;
        }
    }
}

// One warp's task: islands 32 lt .. 32 lt + 31 of simulation I at protocol step t
// (its state's `init`: the sums are set up from scratch). MODE 0: margins only
// (exact sums kept by the flips); MODE 1: resweep the sums of the simulation's
// width. A simulation whose state says `init` is swept in any mode, and on the
// FP32 path both widths are summed. COHERENT: the spins are read through the
// coherent path (a kernel in which other CTAs flip them between tasks), else
// through the read-only cache. s32 / s64: this warp's staging rows in shared
// memory. Returns true on the warp that completed the whole tree (see
// propagate_up).
template <int PREC, int W, int MODE, bool COHERENT>
__device__ __forceinline__ bool sweep_task(const Inst& I, unsigned* __restrict__ tcnt,
                                           int64_t t, int64_t lt, bool init,
                                           int (*s32)[2], long long (*s64)[2]) {
    const int lane = threadIdx.x & 31;
    const int64_t r0 = lt << 5;
    const bool SUM32 = PREC == 1 && (MODE == 1 || init);
    const bool SUM64 = PREC == 0 ? (MODE == 1 || init) : init;

    if (SUM32 || SUM64) {
        constexpr int R = 32 / W;
        const int sub = lane / W, sl = lane % W;
        const int4* __restrict__ col4 = reinterpret_cast<const int4*>(I.col);
        // The FP32 sums alone two rows at a time (sum32_rows); with 64-bit sums one
        // row at a time (registers).
        if (!SUM64) {
            if (I.dcol)
                sum32_rows<W, COHERENT, true>(I, r0, s32);
            else
                sum32_rows<W, COHERENT, false>(I, r0, s32);
        } else {
            for (int q = sub; q < 32; q += R) {
                const int64_t i = r0 + q;
                int bp = 0, bq = 0;
                long long ap = 0, aq = 0;
                if (i < I.n) {
                    const int64_t g0 = __ldg(&I.rp[i]) >> 2, g1 = __ldg(&I.rp[i + 1]) >> 2;
                    for (int64_t g = g0 + sl; g < g1; g += W) {
                        const int4 c = __ldg(&col4[g]);
                        int8_t s0, s1, s2, s3;
                        if constexpr (COHERENT) {
                            s0 = I.s[c.x];
                            s1 = I.s[c.y];
                            s2 = I.s[c.z];
                            s3 = I.s[c.w];
                        } else {
                            s0 = __ldg(&I.s[c.x]);
                            s1 = __ldg(&I.s[c.y]);
                            s2 = __ldg(&I.s[c.z]);
                            s3 = __ldg(&I.s[c.w]);
                        }
                        if (PREC == 1 && SUM32) {
                            const int4* p4 = reinterpret_cast<const int4*>(I.pq32) + 2 * g;
                            const int4 a = __ldg(p4), b = __ldg(p4 + 1);
                            bp += sgn_sel(s0, a.x) + sgn_sel(s1, a.z) + sgn_sel(s2, b.x) +
                                  sgn_sel(s3, b.z);
                            bq += sgn_sel(s0, a.y) + sgn_sel(s1, a.w) + sgn_sel(s2, b.y) +
                                  sgn_sel(s3, b.w);
                        }
                        if (SUM64) {
                            const longlong2* p = I.pq64 + 4 * g;
                            const longlong2 v0 = __ldg(p), v1 = __ldg(p + 1);
                            const longlong2 v2 = __ldg(p + 2), v3 = __ldg(p + 3);
                            ap += sgn_sel(s0, v0.x) + sgn_sel(s1, v1.x) + sgn_sel(s2, v2.x) +
                                  sgn_sel(s3, v3.x);
                            aq += sgn_sel(s0, v0.y) + sgn_sel(s1, v1.y) + sgn_sel(s2, v2.y) +
                                  sgn_sel(s3, v3.y);
                        }
                    }
                }
    #pragma unroll
                for (int o = W / 2; o > 0; o >>= 1) {
                    if (SUM32) {
                        bp += __shfl_xor_sync(0xffffffffu, bp, o);
                        bq += __shfl_xor_sync(0xffffffffu, bq, o);
                    }
                    if (SUM64) {
                        ap += __shfl_xor_sync(0xffffffffu, ap, o);
                        aq += __shfl_xor_sync(0xffffffffu, aq, o);
                    }
                }
                if (sl == 0) {
                    if (PREC == 1 && SUM32) {
                        s32[q][0] = bp;
                        s32[q][1] = bq;
                    }
                    if (SUM64) {
                        s64[q][0] = ap;
                        s64[q][1] = aq;
                    }
                }
            }
        }
        __syncwarp();
    }

    const int64_t i = r0 + lane;
    unsigned long long node = 0ull;
    if (i < I.n) {
        const uint32_t step = I.step0 + (uint32_t)t;
        const int si = I.s[i];
        const uint16_t ci = I.cls[i];
        const float2 rbc = I.rbc32[i];
        const int64_t ra = __ldg(&I.rp[i]), rb = __ldg(&I.rp[i + 1]);
        // the external field on the island's frame: the class table of the global
        // field, or with a local or spatial field the island's own projection,
        // kept for the relax
        double2 e64 = I.ext64[ci];
        float2 e32 = I.ext32[ci];
        if (I.exti64) {
            const double2 lab = ext_lab(I, i, step, I.phx[t], I.phy[t]);
            e64 = ext_proj(lab.x, lab.y, I.cs64[ci]);
            e32 = make_float2(__double2float_rn(e64.x), __double2float_rn(e64.y));
            I.exti64[i] = e64;
            I.exti32[i] = e32;
        }
        float2 th = make_float2(0.0f, 0.0f);
        if (I.sigma > 0.0) {
            th = thermal32(I, i, step);
            I.th32[i] = th;
        }
        longlong2 h64;
        if (SUM64) {
            h64 = make_longlong2(s64[lane][0], s64[lane][1]);
            I.h64[i] = h64;
        }
        if constexpr (PREC == 1) {
            // (without the resweep, the 32-bit sums kept by the flips)
            const int2 h = SUM32 ? make_int2(s32[lane][0], s32[lane][1]) : rec_load(I, i).h32;
            const float dp = __fmul_rn(__int2float_rn(h.x), I.inv32);
            const float dq = __fmul_rn(__int2float_rn(h.y), I.inv32);
            const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
            float lo = e.certain ? e.lo : -1.0f;
            node = e.possible ? key32_of(e.hi, i) : 0ull;
            double x = e.possible ? -1.0 : 0.0;
            // An island that may be flippable may meet an exact comparison in the
            // relax: its FP64 thermal draw is taken and kept here, off the flip chain.
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0 && e.possible) thermal64_kept(I, i, step, &tp, &tq);
            if (e.possible && !e.certain) {
                // within its band of the threshold or of the sign change: FP64 now
                if (!SUM64) h64 = I.h64[i];
                const Eval64 f = eval64(I, si, h64.x, h64.y, I.rbc64[i], e64, tp, tq);
                x = f.flippable ? f.lhs : 0.0;
                node = x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
                lo = x > 0.0 ? __double2float_rd(x) : -1.0f;
            }
            I.key32[i] = node;
            I.key64[i] = x;
            rec_store(I, i, h, lo, si, rbc, ra, rb, ci);
        } else {
            if (!SUM64) h64 = I.h64[i];
            const float dp = __fmul_rn(__ll2float_rn(h64.x), I.inv64f);
            const float dq = __fmul_rn(__ll2float_rn(h64.y), I.inv64f);
            const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
            double x = 0.0;
            if (e.possible) {
                double tp = 0.0, tq = 0.0;
                if (I.sigma > 0.0) thermal64_kept(I, i, step, &tp, &tq);
                const Eval64 f = eval64(I, si, h64.x, h64.y, I.rbc64[i], e64, tp, tq);
                if (f.flippable) x = f.lhs;
            }
            I.key64[i] = x;
            node = x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
            I.key32[i] = node;
            rec_store(I, i, make_int2(0, 0), x > 0.0 ? __double2float_rd(x) : -1.0f, si, rbc, ra,
                      rb, ci);
        }
    }
    node = warp_max_key(node);
    if (lane == 0) I.tree[I.lvl_off[0] + lt] = node;
    return propagate_up(I, tcnt, 0, lt);
}

}  // namespace
}  // namespace fs
