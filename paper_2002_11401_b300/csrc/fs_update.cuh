// fs_update.cuh - per-island key evaluation and neighbour updates shared by the
// relax kernels (the single-flip chain and the multi-flip rounds): the key of an
// island from its current state (Eq. 2, 5, 6 in FP32 with bounds, FP64 where the
// bounds do not decide), the update of a neighbour's exact sums after a flip, and
// the exact FP64 value of an island.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_common.cuh"

namespace fs {
namespace {

// Warp maximum of 64-bit keys (every lane gets it): the largest upper half, then
// among those the largest lower half.
__device__ __forceinline__ unsigned long long warp_max_key(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32), lo = (unsigned)v;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

// Key of island i from its current state (already loaded): returns the new key
// and writes lo and the exact value x (the FS_FP64 LHS when flippable, 0 when
// not; on the FP32 path -1 when only the FP32 bounds were taken). KEEP: an FP64
// thermal draw taken here is kept for later evaluations; without it the kept
// draws are only read (for evaluations ahead of the pick, which store nothing).
template <int PREC, bool KEEP>
__device__ __forceinline__ unsigned long long key_of(const Inst& I, int64_t i, uint32_t step,
                                                     int si, uint16_t ci, longlong2 h64, int2 h32,
                                                     float2 rbc, float2 e32, float2 th,
                                                     double2 rb64, double2 e64, float* lo,
                                                     double* x64) {
    if constexpr (PREC == 1) {
        const float dp = __fmul_rn(__int2float_rn(h32.x), I.inv32);
        const float dq = __fmul_rn(__int2float_rn(h32.y), I.inv32);
        const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
        if (e.possible && !e.certain) {
            // within its band of the threshold or of the sign change: FP64 now
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0) thermal64_at<KEEP>(I, i, step, &tp, &tq);
            const Eval64 f =
                eval64(I, si, h64.x, h64.y, __ldg(&I.rbc64[i]), ext64_at(I, i, ci), tp, tq);
            const double x = f.flippable ? f.lhs : 0.0;
            *x64 = x;
            *lo = x > 0.0 ? __double2float_rd(x) : -1.0f;
            return x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
        }
        *x64 = e.possible ? -1.0 : 0.0;
        *lo = e.certain ? e.lo : -1.0f;
        return e.possible ? key32_of(e.hi, i) : 0ull;
    } else {
        const float dp = __fmul_rn(__ll2float_rn(h64.x), I.inv64f);
        const float dq = __fmul_rn(__ll2float_rn(h64.y), I.inv64f);
        const Eval32 e = eval32(I, si, dp, dq, rbc, e32, th.x, th.y);
        double x = 0.0;
        if (e.possible) {
            double tp = 0.0, tq = 0.0;
            if (I.sigma > 0.0) thermal64_at<KEEP>(I, i, step, &tp, &tq);
            const Eval64 f = eval64(I, si, h64.x, h64.y, rb64, e64, tp, tq);
            if (f.flippable) x = f.lhs;
        }
        *x64 = x;
        *lo = x > 0.0 ? __double2float_rd(x) : -1.0f;
        return x > 0.0 ? key32_of(__double2float_ru(x), i) : 0ull;
    }
}

// One neighbour update: island i's field changes by 2 s_new (dp, dq) (exact 64-bit
// sums; dp32, dq32 the 32-bit ones) and its key is re-evaluated. Computing it
// (loads and arithmetic) is kept apart from its effects (stores, tree, prediction)
// so that it can be computed ahead of the pick and committed once the pick is
// known; both ways run the same code.
struct Upd {
    int64_t i;  // -1: none
    longlong2 h;
    int2 g;
    unsigned long long old, nk;
    float lo;
    double x;
    int64_t r0, r1;  // island i's row, for the prediction
    int s;           // island i's spin (written back with the sums)
};

// Every load is issued before any result is needed so that they overlap. `own`:
// island i's spin when given (nonzero), else read from memory.
template <int PREC, bool KEEP>
__device__ __forceinline__ Upd compute_update(const Inst& I, int64_t i, int snew, long long dp,
                                              long long dq, int dp32, int dq32, uint32_t step,
                                              int own = 0) {
    Upd u;
    u.i = i;
    longlong2 h = I.h64[i];
    const IslandRec r = rec_load(I, i);
    int2 g = make_int2(0, 0);
    if constexpr (PREC == 1) g = r.h32;
    u.old = I.key32[i];
    const int si = own != 0 ? own : r.s;
    u.s = si;
    const uint16_t ci = r.cls;
    const float2 rbc = r.rbc;
    float2 th = make_float2(0.0f, 0.0f);
    if (I.sigma > 0.0) th = I.th32[i];
    u.r0 = (int64_t)r.rowq << 2;
    u.r1 = u.r0 + ((int64_t)r.rowlenq << 2);
    double2 rb64 = make_double2(0.0, 0.0);
    double2 e64 = make_double2(0.0, 0.0);
    if constexpr (PREC == 0) {
        rb64 = __ldg(&I.rbc64[i]);
        e64 = ext64_at(I, i, ci);
    }
    const float2 e32 = ext32_at(I, i, ci);
    const unsigned long long up = 2ull * (unsigned long long)dp;
    const unsigned long long uq = 2ull * (unsigned long long)dq;
    h.x = (long long)(snew > 0 ? (unsigned long long)h.x + up : (unsigned long long)h.x - up);
    h.y = (long long)(snew > 0 ? (unsigned long long)h.y + uq : (unsigned long long)h.y - uq);
    if constexpr (PREC == 1) {
        const unsigned vp = 2u * (unsigned)dp32, vq = 2u * (unsigned)dq32;
        g.x = (int)(snew > 0 ? (unsigned)g.x + vp : (unsigned)g.x - vp);
        g.y = (int)(snew > 0 ? (unsigned)g.y + vq : (unsigned)g.y - vq);
    }
    u.h = h;
    u.g = g;
    u.x = 0.0;
    u.nk = key_of<PREC, KEEP>(I, i, step, si, ci, h, g, rbc, e32, th, rb64, e64, &u.lo, &u.x);
    return u;
}

// Exact FP64 value of island i (0 when not flippable): the value kept with its
// key when its current fields were evaluated in FP64, else (FP32 path) a fresh
// FP64 evaluation of its exact sums, which is then kept. The island's state is
// loaded before the kept value is looked at, so that a miss costs no extra trip.
template <int PREC>
__device__ __forceinline__ double exact_value(const Inst& I, int64_t i, uint32_t step) {
    const double kept = I.key64[i];
    if constexpr (PREC == 0) {
        return kept;
    } else {
        const longlong2 h = I.h64[i];
        const IslandRec r = rec_load(I, i);
        const int si = r.s;
        const double2 rb64 = __ldg(&I.rbc64[i]);
        const uint16_t ci = r.cls;
        if (kept >= 0.0) return kept;
        double tp = 0.0, tq = 0.0;
        if (I.sigma > 0.0) thermal64_kept(I, i, step, &tp, &tq);
        const Eval64 e = eval64(I, si, h.x, h.y, rb64, ext64_at(I, i, ci), tp, tq);
        const double v = e.flippable ? e.lhs : 0.0;
        I.key64[i] = v;
        return v;
    }
}

}  // namespace
}  // namespace fs
