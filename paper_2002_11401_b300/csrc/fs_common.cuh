// fs_common.cuh - device-visible instance descriptor and the per-island
// arithmetic shared by every kernel: Philox4x32-10, Box-Muller, the total field
// in the island's frame (Eq. 2), the astroid left-hand side (Eq. 5) and the
// anti-alignment test (Eq. 6), in FP64 and in FP32 with rigorous error bounds.
//
// Every floating-point expression that decides a flip is written with explicit
// round-to-nearest intrinsics so that no compiler contraction can make two
// kernels evaluate the same island differently.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fs {

constexpr int kRowPad = 4;                // CSR rows padded to multiples of 4 entries
constexpr int kMaxPaddedDegree = 1024;    // neighbours per island after padding
constexpr int kFan = 32;                  // max-tree fan-out (one warp)
constexpr int kMaxLevels = 8;             // tree levels above the leaves
constexpr int kRecheckCap = 256;          // FP64 recheck candidates per round

// Device status codes (mirror fs_status).
enum : int32_t {
    ST_OK = 0,
    ST_NOT_CONVERGED = 4,
    ST_TIMEOUT = 5,
    ST_BOUNDS = 6,
};

// Mutable per-simulation state in device memory.
struct InstState {
    int64_t t;          // next protocol step (0..K)
    int64_t n_flips;    // flips so far in this protocol call
    uint64_t hash;      // FNV-1a of (step, island) so far
    int32_t status;     // ST_*
    int32_t init;       // 1: the dipolar sums must be computed from scratch this step
    double hx, hy;      // external field of the current step
    uint32_t step;      // thermal step index of the current step
    uint32_t pad;
    int64_t rechecks;   // FP32 path: FP64 recheck rounds (single-flip relax), FP64
                        // evaluations of candidates (multi-flip relax)
    int64_t fallbacks;  // full-scan rechecks (candidate overflow)
    int64_t rounds;     // multi-flip relax: rounds that flipped, and iterations without a flip
    int64_t idle;
    int32_t handoff;    // 1: the multi-flip relax left the rest of step t to the single-flip one
    int32_t pad2;
    int64_t step_flips; // flips of step t before the hand-off
    int64_t round_flips;  // multi-flip relax: flips made in its rounds,
    int64_t handoffs;     //   and field steps it handed to the single-flip relax
};

// Read-only descriptor of one simulation (one entry of a batch table).
// Per-island state that the relax reads and writes together, 32 bytes (one sector):
// the first half (32-bit sums, lower bound, spin) is written by the flips; the
// second half (FP32 1/(b h_k), 1/(c h_k), row, angle class) is constant over a
// relax. Every field-and-margin sweep rewrites the whole record from the
// per-island arrays, so a relax always starts from a fresh one.
struct __align__(32) IslandRec {
    int2 h32;          // dipolar (par, perp), 32-bit fixed-point sums (FP32 path; else 0)
    float lo;          // certified lower bound of the LHS, -1 if none
    int32_t s;         // spin
    float2 rbc;        // 1 / (b h_k), 1 / (c h_k)
    uint32_t rowq;     // first entry of the island's CSR row / 4
    uint16_t cls;      // angle class
    uint16_t rowlenq;  // entries of the row / 4
};
static_assert(sizeof(IslandRec) == 32, "one 32-byte sector per island");

struct Inst {
    int64_t n;       // islands
    int64_t nnzp;    // padded CSR entries
    int32_t prec;    // 0 = FP64, 1 = FP32 + FP64 recheck
    int32_t nlev;    // tree levels above the leaves; level nlev-1 is the root
    int32_t nclass;  // distinct island angles
    int32_t pad1;
    int32_t lvl_n[kMaxLevels];
    int64_t lvl_off[kMaxLevels];  // node offset of each level in `tree`
    // neighbour tensors (rows padded with self-entries of zero weight)
    const int64_t* rp;
    const int32_t* col;
    const longlong2* pq64;  // (P, Q) in 2^-e64 fixed point
    const long long* qt64;  // transposed Q: field of the row island on col, col's frame
    const int2* pq32;       // (P, Q) in 2^-e32 fixed point
    const int* qt32;
    // col[e] - i for row i as 16-bit offsets (FP32 path, when every offset fits;
    // else null): what the FP32 sweeps read instead of col
    const int16_t* dcol;
    // islands
    int8_t* s;
    const double2* rbc64;   // (1 / (b h_k), 1 / (c h_k)) per island, FP64
    const float2* rbc32;    // the same, FP32
    const uint16_t* cls;    // angle class
    const double2* cs64;    // (cos, sin) per class
    const float2* cs32;
    double2* ext64;         // external field projected on each class, current step
    float2* ext32;
    // fields and keys
    longlong2* h64;         // dipolar (par, perp), exact 64-bit sums (both paths)
    IslandRec* rec;         // the relax's per-island record (see IslandRec)
    float2* th32;           // thermal (par, perp) of the current step (sigma > 0)
    double2* th64;          // FP64 thermal (par, perp) drawn for step th_step[i]
    uint32_t* th_step;      // (sigma > 0; all ones before the first draw)
    unsigned long long* key32;  // (bits(upper bound) << 32) | ~i, 0 = not a candidate
    double* key64;              // exact LHS when flippable, 0 when not; FP32 path: -1
                                // while the current fields have not been evaluated in FP64
    unsigned long long* tree;   // max-tree nodes above the keys
    // protocol
    const double* phx;
    const double* phy;
    int64_t K;
    uint32_t step0;
    int32_t resweep;
    uint32_t* log_step;
    uint32_t* log_spin;
    int64_t log_cap;
    int64_t* flips_per_step;
    // parameters
    double b, c, pexp, qexp, sigma;
    float bf, cf, pexpf, qexpf, sigmaf;
    double inv64;   // 2^-e64
    float inv64f;   // 2^-e64 as a float
    float inv32;    // 2^-e32
    uint64_t seed;
    uint32_t instance;
    int32_t pad0;
    int64_t max_flips;
    // FP32 error model: |h32 - h64| <= dh_abs + th_rel * |h_th| + dh_rel * (|h_dip| +
    // |h_ext| + |h_th|); div_rel bounds the relative error of |h| / (b h_k) against
    // the FP64 product |h| (1 / (b h_k)); the FP32 power of each astroid term is
    // within pow_rel_* + lnk_* (|e| + 2) of x^p (e the binary exponent of x, p the
    // FP64 exponent), see pow_err.
    float dh_abs, dh_rel, div_rel;
    float th_rel;   // |th32 - th64| <= th_rel (|th_par| + |th_perp|)
    float pow_rel_p, pow_rel_q;  // the FP32 power's own error (documented ulp bound)
    float lnk_p, lnk_q;          // |p - (float)p| ln 2, rounded up (0 unless powf)
    int32_t pmode_p, pmode_q;    // power: kPowF, kPowCube (x rcbrtf(x)) or kPowOne (x)
    int32_t perp;                // 1: Eq. 5 has its perpendicular term; 0: the parallel-only criterion
    int32_t pad3;
    // External field of each island beyond the global one (Sec. "External field"):
    // a local series lx[step n + i] or a spatial one gx[step G + gcell[i]] (lab frame),
    // step < ext_K; the sweep writes the step's projected total into exti64/exti32,
    // which the relax reads in place of the per-class table. NULL: global field only.
    const double* lx;
    const double* ly;
    const double* gx;
    const double* gy;
    const int32_t* gcell;
    int64_t ext_K, grid_G;
    double2* exti64;
    float2* exti32;
    // Thermal standard deviation per field step (a thermal protocol, e.g. annealing):
    // sig[step], step < sig_K; NULL: sigma.
    const double* sig;
    int64_t sig_K;
    // Island centres (the multi-flip relax's independence test) and the square of
    // the distance below which two islands may share a neighbour: (2 cutoff)^2,
    // widened by 1e-6 beyond the inclusive cutoff.
    const double2* pos;
    double rconf2;
    float rconf2f;  // the same, for FP32 centres: widened by their rounding
    int32_t pad4;
    InstState* st;
};

// Powers of the astroid terms.
constexpr int32_t kPowF = 0;     // powf at the FP32-rounded exponent
constexpr int32_t kPowCube = 1;  // exponent 2/3: x rcbrtf(x)
constexpr int32_t kPowOne = 2;   // exponent 1: x itself

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
#else
    const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c[0]) >> 32);
    const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c[2]) >> 32);
#endif
    const uint32_t lo0 = 0xD2511F53u * c[0];
    const uint32_t lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

// Ten rounds, key advanced by the Weyl constants between rounds.
__host__ __device__ __forceinline__ void philox10(uint32_t c[4], uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        philox_round(c, k0, k1);
    }
}

// The 53-bit uniforms in (0,1): ((w_hi:w_lo) >> 11) + 1/2, times 2^-53.
__host__ __device__ __forceinline__ uint64_t u53(uint32_t hi, uint32_t lo) {
    return (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
}

// FP64 Box-Muller of one Philox output block.
__device__ __forceinline__ void box_muller64(const uint32_t w[4], double* z0, double* z1) {
    const double u1 = __dmul_rn(__dadd_rn((double)u53(w[0], w[1]), 0.5), 0x1.0p-53);
    const double u2 = __dmul_rn(__dadd_rn((double)u53(w[2], w[3]), 0.5), 0x1.0p-53);
    const double rad = sqrt(__dmul_rn(-2.0, log(u1)));
    const double ang = __dmul_rn(2.0 * 3.14159265358979323846, u2);
    double sn, cs;
    sincos(ang, &sn, &cs);
    *z0 = __dmul_rn(rad, cs);
    *z1 = __dmul_rn(rad, sn);
}

// FP32 Box-Muller of the same block, with an error relative to the radius.
// ln(u1) is taken from u1 itself when u1 < 1/2 and from log1p(-(1 - u1))
// otherwise, with 1 - u1 formed exactly in integers. The angle 2 pi u2 = pi x,
// x = (2b + 1) 2^-53, is split exactly in integers into x_hi (24 bits) + x_lo, and
// sincospi(x_hi) is corrected to first order in pi x_lo (|pi x_lo| < 4e-7), so the
// 53-bit uniform is not rounded to 24 bits first.
__device__ __forceinline__ void box_muller32(const uint32_t w[4], float* z0, float* z1) {
    const uint64_t a = u53(w[0], w[1]);
    const uint64_t b = u53(w[2], w[3]);
    float l;
    if (a < (1ull << 52)) {
        const float u1 = __fmul_rn(__ull2float_rn(a) + 0.5f, 0x1.0p-53f);
        l = logf(u1);
    } else {
        // 1 - u1 = (2^53 - a - 1/2) 2^-53
        const uint64_t v = (1ull << 53) - a;
        const float om = __fmul_rn(__fsub_rn(__ull2float_rn(v), 0.5f), 0x1.0p-53f);
        l = log1pf(-om);
    }
    const float rad = sqrtf(__fmul_rn(-2.0f, l));
    const uint64_t x = 2 * b + 1;  // < 2^54
    const float xh = __fmul_rn(__uint2float_rn((uint32_t)(x >> 30)), 0x1.0p-23f);
    const float xl = __fmul_rn(__uint2float_rn((uint32_t)(x & ((1u << 30) - 1u))), 0x1.0p-53f);
    float sn, cs;
    sincospif(xh, &sn, &cs);
    const float d = __fmul_rn(3.14159265f, xl);
    const float c2 = __fsub_rn(cs, __fmul_rn(sn, d));
    const float s2 = __fadd_rn(sn, __fmul_rn(cs, d));
    *z0 = __fmul_rn(rad, c2);
    *z1 = __fmul_rn(rad, s2);
}

// Thermal field (par, perp) of island i at thermal step `step`: counter
// (i, step, instance, 1).
// Thermal standard deviation of field step `step`.
__device__ __forceinline__ double sigma_at(const Inst& I, uint32_t step) {
    return I.sig ? I.sig[step] : I.sigma;
}

__device__ __forceinline__ void thermal64(const Inst& I, int64_t i, uint32_t step, double* tp,
                                          double* tq) {
    uint32_t c[4] = {(uint32_t)i, step, I.instance, 1u};
    philox10(c, I.seed);
    double z0, z1;
    box_muller64(c, &z0, &z1);
    const double sg = sigma_at(I, step);
    *tp = __dmul_rn(sg, z0);
    *tq = __dmul_rn(sg, z1);
}

// The kept draw of island i for `step`, when there is one. The draw is published
// after its value (a block-scope fence between the two stores, the step number
// written and read as a volatile, strong access, and a fence between reading it
// and reading the value), so that a thread of the same block that sees the step
// also sees the value written before it, even while another thread keeps a draw.
__device__ __forceinline__ bool kept_draw(const Inst& I, int64_t i, uint32_t step, double* tp,
                                          double* tq) {
    if (*(volatile uint32_t*)&I.th_step[i] != step) return false;
    __threadfence_block();
    const double2 v = I.th64[i];
    *tp = v.x;
    *tq = v.y;
    return true;
}

// thermal64 of island i, drawn once per island and step: the draw is kept with
// its step number, and later evaluations of the same step reuse it. One island
// is never kept by two threads at the same time; others may read it meanwhile.
__device__ __forceinline__ void thermal64_kept(const Inst& I, int64_t i, uint32_t step, double* tp,
                                               double* tq) {
    if (kept_draw(I, i, step, tp, tq)) return;
    thermal64(I, i, step, tp, tq);
    I.th64[i] = make_double2(*tp, *tq);
    __threadfence_block();
    *(volatile uint32_t*)&I.th_step[i] = step;
}

// thermal64 of island i at `step`, kept (KEEP) or only looked up among the kept
// draws (otherwise drawn afresh without keeping it; the value is the same).
template <bool KEEP>
__device__ __forceinline__ void thermal64_at(const Inst& I, int64_t i, uint32_t step, double* tp,
                                             double* tq) {
    if constexpr (KEEP) {
        thermal64_kept(I, i, step, tp, tq);
    } else if (!kept_draw(I, i, step, tp, tq)) {
        thermal64(I, i, step, tp, tq);
    }
}

__device__ __forceinline__ float2 thermal32(const Inst& I, int64_t i, uint32_t step) {
    uint32_t c[4] = {(uint32_t)i, step, I.instance, 1u};
    philox10(c, I.seed);
    float z0, z1;
    box_muller32(c, &z0, &z1);
    const float sg = I.sig ? __double2float_rn(I.sig[step]) : I.sigmaf;
    return make_float2(__fmul_rn(sg, z0), __fmul_rn(sg, z1));
}

// ---------------------------------------------------------------------------
// Eq. 2 in the island's frame, Eq. 5 and Eq. 6
// ---------------------------------------------------------------------------

// Projection of the external field on an island's frame (h_ext . mhat,
// h_ext . mhat_perp), in FP64. Both evaluations below take this same value (the
// FP32 one rounded once), so its error is relative to the projection itself.
__device__ __forceinline__ double2 ext_proj(double hx, double hy, double2 cs) {
    return make_double2(__dadd_rn(__dmul_rn(hx, cs.x), __dmul_rn(hy, cs.y)),
                        __dadd_rn(__dmul_rn(-hx, cs.y), __dmul_rn(hy, cs.x)));
}

// The external field of island i (class ci) projected on its frame at the current
// field step: the per-island values the sweep wrote when a local or spatial field
// is set, else the per-class table of the global field (read with plain loads: a
// kernel may point the descriptor's table at a copy in its shared memory).
__device__ __forceinline__ double2 ext64_at(const Inst& I, int64_t i, uint16_t ci) {
    return I.exti64 ? __ldg(&I.exti64[i]) : I.ext64[ci];
}
__device__ __forceinline__ float2 ext32_at(const Inst& I, int64_t i, uint16_t ci) {
    return I.exti32 ? __ldg(&I.exti32[i]) : I.ext32[ci];
}

// The lab-frame external field of island i at field step `step`: the global
// (hx, hy) plus its local or spatial part (the sum in this order, as the reference
// evaluation takes it).
__device__ __forceinline__ double2 ext_lab(const Inst& I, int64_t i, uint32_t step, double hx,
                                           double hy) {
    if (I.lx) {
        const int64_t q = (int64_t)step * I.n + i;
        return make_double2(__dadd_rn(hx, I.lx[q]), __dadd_rn(hy, I.ly[q]));
    }
    if (I.gx) {
        const int64_t q = (int64_t)step * I.grid_G + I.gcell[i];
        return make_double2(__dadd_rn(hx, I.gx[q]), __dadd_rn(hy, I.gy[q]));
    }
    return make_double2(hx, hy);
}

// x^(2/3) for x > 0 as x r, r = x^(-1/3). The seed r0 is the FP32 reciprocal cube
// root of x (relative error below 2^-22); one FP64 step of the binomial series
// (1 - e)^(-1/3) = 1 + e/3 + 2e^2/9 + O(e^3) with e = 1 - x r0^3 (Householder's
// method of order 2 for r^-3 = x) leaves a truncation error near 2^-66, so the
// result is within a few ulps of x^(2/3). Eight FP64 operations (each a long
// issue on this GPU's FP64 pipe) instead of a cube root. Outside [2^-100, 2^100],
// where the FP32 seed could over- or underflow, the cube root of x^2 is taken.
__device__ __forceinline__ double pow23(double x) {
    if (!(x >= 0x1p-100 && x <= 0x1p100)) return cbrt(__dmul_rn(x, x));
    const double r0 = (double)rcbrtf(__double2float_rn(x));
    const double r03 = __dmul_rn(__dmul_rn(r0, r0), r0);
    const double e = __fma_rn(-x, r03, 1.0);
    const double t = __fma_rn(2.0 / 9.0, e, 1.0 / 3.0);
    const double r = __fma_rn(__dmul_rn(r0, e), t, r0);
    return __dmul_rn(x, r);
}

// x^p for x >= 0 in FP64. p = 2/3 (gamma or beta = 3, the Stoner-Wohlfarth value)
// takes pow23, several times cheaper than pow on this GPU.
__device__ __forceinline__ double pow_pos(double x, double p) {
    if (x <= 0.0) return 0.0;
    if (p == 2.0 / 3.0) return pow23(x);
    if (p == 1.0) return x;
    return pow(x, p);
}

// Exact FP64 evaluation from the 64-bit fixed-point dipolar sums.
struct Eval64 {
    double hpar, hperp, lhs;
    bool flippable;
};

// rb: the island's (1 / (b h_k), 1 / (c h_k)) in FP64, so that the astroid's
// arguments take a product where a quotient would cost a division (a long FP64
// sequence on this GPU); each differs from the quotient by at most one rounding.
__device__ __forceinline__ Eval64 eval64(const Inst& I, int s, long long dp, long long dq,
                                         double2 rb, double2 ext, double tp, double tq) {
    Eval64 e;
    e.hpar = __dadd_rn(__dadd_rn(__dmul_rn((double)dp, I.inv64), ext.x), tp);
    e.hperp = __dadd_rn(__dadd_rn(__dmul_rn((double)dq, I.inv64), ext.y), tq);
    const double x = __dmul_rn(fabs(e.hpar), rb.x);
    const double y = __dmul_rn(fabs(e.hperp), rb.y);
    // (the parallel-only criterion: |h_par| / h_k alone, exponent 1, no second term)
    e.lhs = I.perp ? __dadd_rn(pow_pos(x, I.pexp), pow_pos(y, I.qexp)) : pow_pos(x, I.pexp);
    e.flippable = ((double)s * e.hpar < 0.0) && (e.lhs > 1.0);
    return e;
}

// FP32 evaluation with bounds: [lo, hi] contains the FS_FP64 value of the LHS;
// `possible` = the island may be flippable in FP64, `certain` = it surely is.
struct Eval32 {
    float hpar, hperp, lhs, hi, lo;
    bool possible, certain;
};

// x^p in FP32 for x >= 0 (0 for x <= 0). kPowCube (p = 2/3, the Stoner-Wohlfarth
// exponent): x rcbrtf(x), the exponent exact and the error that of rcbrtf plus one
// rounding; kPowOne (p = 1): x, exact; otherwise powf at the FP32-rounded exponent.
__device__ __forceinline__ float pow32(float x, float p, int mode) {
    if (!(x > 0.0f)) return 0.0f;
    if (mode == kPowCube) return __fmul_rn(x, rcbrtf(x));
    if (mode == kPowOne) return x;
    return powf(x, p);
}

// Bound on the relative error of pow32(x) against x^p with the FP64 exponent p:
// rel (the function's own error, from its documented maximum ulp error) plus the
// exponent's rounding, x^pf / x^p = exp((pf - p) ln x) with |ln x| <= (|e| + 1) ln 2
// for the binary exponent e of x (|e| + 2 leaves room for exp(t) - 1 <= t e^t; a
// subnormal x counts as e = -150); the sum is widened by 2^-16 so that the bound
// also covers 1 / (1 - r) - 1 where callers divide by 1 - r.
__device__ __forceinline__ float pow_err(float x, float rel, float lnk) {
    float r = rel;
    if (lnk > 0.0f) {
        const int bexp = (int)((__float_as_uint(x) >> 23) & 0xFFu);
        const int e = bexp == 0 ? 150 : abs(bexp - 127);
        r = __fadd_ru(r, __fmul_ru(lnk, (float)(e + 2)));
    }
    return __fmul_ru(r, 1.0f + 0x1.0p-16f);
}

// Bounds of one astroid term a^p, a = |h| / (b h_k), whose FP32 value t = pow32(x)
// was taken at x; u bounds the relative error of x. For p <= 1 the concave power
// gives (x(1+u))^p <= x^p (1 + p u) and (x(1-u))^p >= x^p (1 - p u / (1 - u)), and
// 1 / (1 - u) <= 1 + 2u on u <= 1/4; for 1 < p <= 3, (1 + u)^(p-1) <= 2 on u <= 1/4
// gives the factors 1 + 2 p u and 1 - p u. Outside u <= 1/4 the monotone bounds
// are evaluated directly. The power's own error comes from pow_err at the argument
// it was taken at. Upper bounds are formed with round-up and lower bounds with
// round-down arithmetic.
__device__ __forceinline__ void term_bounds(float t, float x, float u, float p, int mode,
                                            float rel, float lnk, float* hi, float* lo) {
    if (u <= 0.25f && p <= 3.0f) {
        const float r = pow_err(x, rel, lnk);
        const float pu = __fmul_ru(p, u);
        const float g_hi = p <= 1.0f ? pu : __fmul_ru(2.0f, pu);
        const float g_lo = p <= 1.0f ? __fmul_ru(pu, __fadd_ru(1.0f, __fmul_ru(2.0f, u))) : pu;
        *hi = __fmul_ru(__fmul_ru(t, __fadd_ru(1.0f, r)), __fadd_ru(1.0f, g_hi));
        *lo = __fmul_rd(__fmul_rd(t, __fsub_rd(1.0f, r)), fmaxf(__fsub_rd(1.0f, g_lo), 0.0f));
    } else {
        const float xh = __fmul_ru(x, __fadd_ru(1.0f, u));
        *hi = __fmul_ru(pow32(xh, p, mode), __fadd_ru(1.0f, pow_err(xh, rel, lnk)));
        if (u < 1.0f) {
            const float xl = __fmul_rd(x, __fsub_rd(1.0f, u));
            *lo = __fmul_rd(pow32(xl, p, mode), __fsub_rd(1.0f, pow_err(xl, rel, lnk)));
        } else {
            *lo = 0.0f;
        }
    }
}

// An upper bound of 1 / x for x > 0: the hardware reciprocal (at most 1 ulp off,
// PTX ISA rcp.approx.f32) widened by 2^-22 and rounded up. A denormal x gives
// +inf, which the callers treat as "no useful bound".
__device__ __forceinline__ float rcp_up(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmul_ru(r, 1.0f + 0x1.0p-22f);
}

// rbc = (1 / (b h_k), 1 / (c h_k)) of the island, each rounded once to FP32.
__device__ __forceinline__ Eval32 eval32(const Inst& I, int s, float dp, float dq, float2 rbc,
                                         float2 ext, float tp, float tq) {
    Eval32 e;
    e.hpar = __fadd_rn(__fadd_rn(dp, ext.x), tp);
    e.hperp = __fadd_rn(__fadd_rn(dq, ext.y), tq);
    // field error bound: fixed point + thermal draw (absolute), float roundings
    // thermal draw: its FP32 error is relative to the radius |th| <= |tp| + |tq|
    const float dth = __fmul_ru(I.th_rel, __fadd_ru(fabsf(tp), fabsf(tq)));
    const float dpar = __fadd_ru(__fadd_ru(I.dh_abs, dth),
                                 __fmul_ru(I.dh_rel, __fadd_ru(__fadd_ru(fabsf(dp), fabsf(ext.x)),
                                                               fabsf(tp))));
    const float dperp = __fadd_ru(__fadd_ru(I.dh_abs, dth),
                                  __fmul_ru(I.dh_rel, __fadd_ru(__fadd_ru(fabsf(dq), fabsf(ext.y)),
                                                                fabsf(tq))));
    const float ap = fabsf(e.hpar), aq = fabsf(e.hperp);
    const float x = __fmul_rn(ap, rbc.x), y = __fmul_rn(aq, rbc.y);
    const float tx = pow32(x, I.pexpf, I.pmode_p);
    const float ty = I.perp ? pow32(y, I.qexpf, I.pmode_q) : 0.0f;
    e.lhs = __fadd_rn(tx, ty);
    // relative error of x and y: the field bound (times 1 + 2^-22, which covers its
    // product with the scaling's error) plus the scaling roundings
    const float ux = ap > 0.0f ? __fadd_ru(__fmul_ru(__fmul_ru(dpar, rcp_up(ap)), 1.0f + 0x1.0p-22f),
                                           I.div_rel)
                               : 2.0f;
    const float uy = aq > 0.0f ? __fadd_ru(__fmul_ru(__fmul_ru(dperp, rcp_up(aq)), 1.0f + 0x1.0p-22f),
                                           I.div_rel)
                               : 2.0f;
    float hx_, lx_, hy_, ly_;
    if (ap > 0.0f) {
        term_bounds(tx, x, ux, I.pexpf, I.pmode_p, I.pow_rel_p, I.lnk_p, &hx_, &lx_);
    } else {  // |h_par| <= dpar
        const float xm = __fmul_ru(__fmul_ru(dpar, rbc.x), __fadd_ru(1.0f, I.div_rel));
        hx_ = __fmul_ru(pow32(xm, I.pexpf, I.pmode_p),
                        __fadd_ru(1.0f, pow_err(xm, I.pow_rel_p, I.lnk_p)));
        lx_ = 0.0f;
    }
    if (!I.perp) {
        hy_ = 0.0f;
        ly_ = 0.0f;
    } else if (aq > 0.0f) {
        term_bounds(ty, y, uy, I.qexpf, I.pmode_q, I.pow_rel_q, I.lnk_q, &hy_, &ly_);
    } else {
        const float ym = __fmul_ru(__fmul_ru(dperp, rbc.y), __fadd_ru(1.0f, I.div_rel));
        hy_ = __fmul_ru(pow32(ym, I.qexpf, I.pmode_q),
                        __fadd_ru(1.0f, pow_err(ym, I.pow_rel_q, I.lnk_q)));
        ly_ = 0.0f;
    }
    e.hi = __fadd_ru(hx_, hy_);
    e.lo = __fadd_rd(lx_, ly_);
    const float sp = (float)s * e.hpar;
    e.possible = (sp < dpar) && (e.hi > 1.0f);
    e.certain = (sp < -dpar) && (e.lo > 1.0f);
    return e;
}

// FP32 key: the upper bound of the LHS (order) with the lowest index winning ties.
__device__ __forceinline__ unsigned long long key32_of(float hi, int64_t i) {
    return ((unsigned long long)__float_as_uint(hi) << 32) |
           (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
}
__device__ __forceinline__ float key32_hi(unsigned long long k) {
    return __uint_as_float((uint32_t)(k >> 32));
}
__device__ __forceinline__ uint32_t key32_idx(unsigned long long k) {
    return 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
}

// FP64 node order: larger LHS first, then lower index. (v, idx) packed in a
// ulonglong2 as (double bits, index). Keys are non-negative doubles, whose bit
// patterns order like their values, so the compare is integer-only.
__device__ __forceinline__ bool better64(unsigned long long va, unsigned long long ia,
                                         unsigned long long vb, unsigned long long ib) {
    return va > vb || (va == vb && ia < ib);
}

// IslandRec access in 16-byte halves.
__device__ __forceinline__ IslandRec rec_load(const Inst& I, int64_t i) {
    const int4* p = reinterpret_cast<const int4*>(I.rec + i);
    const int4 a = p[0], b = p[1];
    IslandRec r;
    r.h32 = make_int2(a.x, a.y);
    r.lo = __int_as_float(a.z);
    r.s = a.w;
    r.rbc = make_float2(__int_as_float(b.x), __int_as_float(b.y));
    r.rowq = (uint32_t)b.z;
    r.cls = (uint16_t)((uint32_t)b.w & 0xFFFFu);
    r.rowlenq = (uint16_t)((uint32_t)b.w >> 16);
    return r;
}

// The half the flips change: 32-bit sums, lower bound, spin.
__device__ __forceinline__ void rec_store_dyn(const Inst& I, int64_t i, int2 h32, float lo,
                                              int s) {
    *reinterpret_cast<int4*>(I.rec + i) = make_int4(h32.x, h32.y, __float_as_int(lo), s);
}

// The whole record; row [ra, rb) (multiples of 4 entries).
__device__ __forceinline__ void rec_store(const Inst& I, int64_t i, int2 h32, float lo, int s,
                                          float2 rbc, int64_t ra, int64_t rb, uint16_t cls) {
    int4* p = reinterpret_cast<int4*>(I.rec + i);
    p[0] = make_int4(h32.x, h32.y, __float_as_int(lo), s);
    p[1] = make_int4(__float_as_int(rbc.x), __float_as_int(rbc.y), (int)(uint32_t)(ra >> 2),
                     (int)((uint32_t)cls | ((uint32_t)((rb - ra) >> 2) << 16)));
}

// FNV-1a over the 8 little-endian bytes of (step, island).
__device__ __forceinline__ uint64_t fnv_flip(uint64_t h, uint32_t step, uint32_t spin) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h ^= (step >> (8 * q)) & 0xFFu;
        h *= 0x100000001b3ull;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        h ^= (spin >> (8 * q)) & 0xFFu;
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace fs
