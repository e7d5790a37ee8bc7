/*
 * flatspin_b300.h - C ABI of the flatspin relax loop on B300 (sm_103a).
 *
 * The model is the dipole model of Jensen et al., "flatspin: A Large-Scale
 * Artificial Spin Ice Simulator" (arXiv 2002.11401):
 *   - islands are point dipoles with Ising spins s_i in {-1,+1} at fixed
 *     positions r_i and angles theta_i (Sec. "Magnets as dipoles", Eq. 1);
 *   - the total field is dipolar + external + thermal (Eq. 2); the dipolar
 *     field sums Eq. 3 over the neighbours inside a cutoff (Sec. "Magnetic
 *     dipole-dipole interactions");
 *   - an island may switch when the left-hand side (LHS) of the generalised
 *     Stoner-Wohlfarth astroid, Eq. 5, exceeds one and h_i . m_i < 0, Eq. 6;
 *   - coercive fields h_k^(i) ~ N(h_k, k_disorder h_k) (Sec. "Imperfections and
 *     disorder");
 *   - dynamics: flip the flippable island with the largest LHS (ties: lowest
 *     index), repeat until none is flippable, then move to the next field value
 *     (Sec. "Dynamics").
 *
 * Conventions for every call:
 *   - Host buffers belong to the caller and are copied in or out before the
 *     call returns. Device buffers passed to *_dev calls belong to the caller
 *     and must stay valid until the work queued on the simulation's stream ends.
 *   - The library owns every device allocation it makes for a simulation and
 *     frees it in fs_destroy; a buffer bound with fs_bind_workspace stays the
 *     caller's.
 *   - Calls are synchronous on the simulation's stream unless named *_dev.
 *   - A fs_sim is not thread-safe; distinct fs_sim objects are independent.
 *   - Island order is the canonical order: ascending y, then ascending x, for
 *     generated arrays; the caller's order for custom arrays. Every index in and
 *     out of the library uses it.
 *   - On error nothing is committed and fs_last_error() explains.
 *   - A device fault is reported as FS_ERR_CUDA; the CUDA context is then
 *     unusable and the process should exit.
 */
#ifndef FLATSPIN_B300_H
#define FLATSPIN_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_ERR_INVALID = 1,       /* bad argument or unsupported size */
    FS_ERR_OOM = 2,           /* device or host allocation failed */
    FS_ERR_CUDA = 3,          /* a CUDA call failed */
    FS_ERR_NOT_CONVERGED = 4, /* a relax exceeded max_flips_per_step */
    FS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    FS_ERR_BOUNDS = 6,        /* an index check on device failed */
    FS_ERR_STATE = 8          /* call out of order (e.g. relax before params) */
} fs_status;

/* Geometries (Sec. "Geometries", Fig. "geometries"); see fs_create_geometry. */
typedef enum {
    FS_SQUARE = 0,
    FS_PINWHEEL = 1,
    FS_KAGOME = 2,
    FS_SQUARE_OPEN = 3,
    FS_PINWHEEL_DIAMOND = 4,
    FS_PINWHEEL_LUCKY_KNOT = 5,
    FS_ISING = 6
} fs_geom;

/* Switching criterion. FS_CRITERION_ASTROID: Eq. 5 > 1 and Eq. 6 (Sec.
 * "Switching"). FS_CRITERION_PARALLEL: the simpler criterion the pinwheel section
 * contrasts with it (only the field component along the magnet counts): an island
 * may switch when the component opposing its magnetisation exceeds its coercive
 * field, -s h_par > h_k; its LHS, the ranked quantity, is |h_par| / h_k (b, c,
 * beta and gamma are not used). */
typedef enum { FS_CRITERION_ASTROID = 0, FS_CRITERION_PARALLEL = 1 } fs_criterion;

/* Arithmetic of the relax loop.
 * FS_FP64: dipolar sums in 64-bit fixed point (exact integer sums of per-pair
 *   coefficients rounded to 2^-e64, e64 chosen per system), the astroid in FP64.
 * FS_FP32_RECHECK: dipolar sums in 32-bit fixed point, the astroid in FP32 with
 *   rigorous error bounds; a pick whose FP32 margin is within its error band of
 *   one, of another candidate, or of the sign change of Eq. 6 is re-evaluated
 *   in the FS_FP64 arithmetic. Both yield the same flip sequence. */
typedef enum { FS_FP64 = 0, FS_FP32_RECHECK = 1 } fs_precision;

/* Model parameters (Sec. "The flatspin magnetic model"). */
typedef struct {
    double alpha;       /* dipolar coupling, Eq. 3 */
    double hk;          /* mean coercive field h_k */
    double k_disorder;  /* relative std of h_k^(i) */
    double b, c;        /* astroid height and width, Eq. 5 */
    double beta, gamma; /* astroid exponents: 2/gamma on h_par, 2/beta on h_perp (Eq. 5) */
    double cutoff;      /* neighbourhood radius in lattice spacings (inclusive) */
    double sigma_th;    /* thermal field std, Sec. "Thermal field" (0 = none) */
    uint64_t seed;      /* Philox key of the h_k and thermal draws */
    uint32_t instance;  /* third Philox counter word (ensemble member) */
    int32_t precision;  /* fs_precision */
    int64_t max_flips_per_step; /* guard; <= 0 means 16 * n */
    int32_t criterion;  /* fs_criterion (0: Eq. 5 and 6) */
    int32_t reserved;   /* 0 */
} fs_params;

typedef struct fs_sim fs_sim;

/* Read-only facts about a built system. */
typedef struct {
    int64_t n;         /* islands */
    int64_t nnz;       /* neighbour pairs (ordered) */
    int64_t nnz_padded;/* stored entries (rows padded to multiples of 4) */
    int32_t max_degree;
    int32_t e64, e32;  /* fixed-point exponents: value = integer * 2^-e */
    int64_t device_bytes;
    double band_rel, band_abs; /* FP32 error band of the LHS: rel * LHS + abs */
    int32_t col_offsets16; /* 1: the FP32 path's sweeps and multi-flip rounds read
                            * each neighbour as its row island plus a 16-bit offset
                            * (every offset fits), 0: the 32-bit column indices */
    int32_t reserved_info;  /* 0 */
} fs_info;

/* Last error message of `sim` (or of the last failed create call when sim is
 * NULL). Valid until the next call on the same object / thread. */
const char* fs_last_error(const fs_sim* sim);

/* FNV-1a (64-bit) offset basis: the value a fresh flip-sequence hash starts
 * from. The hash folds the 8 little-endian bytes (u32 step, u32 island) of
 * every flip, in order. */
uint64_t fs_hash_init(void);

/* Generated arrays (Sec. "Geometries", Fig. "geometries"): nx x ny cells of
 * spacing a.
 * FS_SQUARE: closed edges, islands at 0 and 90 degrees, 2 nx ny + nx + ny islands.
 * FS_PINWHEEL: the square's islands turned 45 degrees about their centres.
 * FS_KAGOME: nx x ny flat-top hexagons of edge a, islands at 0/60/120 degrees on
 *   the edge midpoints, 3 nx ny + 2 nx + 2 ny - 1 islands.
 * The figure names further edge forms without defining them; these readings:
 * FS_SQUARE_OPEN: open edges, the closed square without the islands on its outer
 *   boundary, 2 nx ny - nx - ny islands (needs nx + ny > 2).
 * FS_PINWHEEL_DIAMOND: nx x ny unit cells of one horizontal island at
 *   (x + 1/2, y) and one vertical at (x, y + 1/2), turned 45 degrees: 2 nx ny
 *   islands (the pinwheel section's 25 x 25 array has 1250).
 * FS_PINWHEEL_LUCKY_KNOT: the open-edged square's islands turned 45 degrees.
 * FS_ISING: one island at every lattice point (x, y), all at 0 degrees.
 * Angles are (deg * pi) / 180 in double. *out receives a new simulation. */
fs_status fs_create_geometry(int32_t kind, int32_t nx, int32_t ny, double a, fs_sim** out);

/* Any 2D set of identical islands (Sec. "Geometries", last paragraph):
 * positions x, y and angles theta (radians), n islands, caller's order.
 * At most 65536 distinct angles. `a` is the unit of the cutoff. */
fs_status fs_create_custom(int64_t n, const double* x, const double* y, const double* theta,
                           double a, fs_sim** out);

void fs_destroy(fs_sim* sim);

/* CUDA stream (cudaStream_t) for all later work of `sim`; NULL = legacy default. */
fs_status fs_set_stream(fs_sim* sim, void* stream);

/* How a relax (Sec. "Dynamics") runs on the device; every mode flips the same
 * islands in the same order.
 * FS_RELAX_SINGLE: one flip at a time, by one CTA: the flippable island with the
 *   largest LHS, then its neighbours' updates.
 * FS_RELAX_MULTI: rounds of several flips: the islands with the largest LHS, in
 *   order, as long as each is the one the single-flip order takes next: its exact
 *   value beats everything outside the round, it lies more than twice the cutoff
 *   from every earlier island of the round (so that no flip of the round changes
 *   its field or a neighbour shared with it), and no earlier flip's neighbour got a
 *   value that beats it. Faster on large arrays, where many of the largest values
 *   lie far apart. A field step whose rounds stay below 4 flips for 4 rounds in a
 *   row (a chain of flips that each make a neighbour the largest) is finished by
 *   the single-flip chain. The rounds run on a cluster of 16 CTAs (16 SMs), or on
 *   one CTA where a cluster of 16 does not fit.
 * FS_RELAX_MULTI_CTA: the same rounds on one CTA (one SM), e.g. beside other work.
 * FS_RELAX_AUTO (default): multi-flip rounds from 32,768 islands on.
 * Batches always use single flips. Errors: FS_ERR_INVALID. */
typedef enum {
    FS_RELAX_AUTO = 0,
    FS_RELAX_SINGLE = 1,
    FS_RELAX_MULTI = 2,
    FS_RELAX_MULTI_CTA = 3
} fs_relax_mode;
fs_status fs_set_relax_mode(fs_sim* sim, int32_t mode);

/* Device bytes fs_set_params(sim, p) would allocate: the simulation's state (the
 * neighbour tensors of Eq. 3, the island arrays, the relax's records and keys, the
 * max-tree) plus the build's temporaries, every allocation rounded up to 256
 * bytes. Exact (fs_set_params checks its allocations against the same plan), for
 * admission and for sizing a workspace. Runs the build's neighbour count on the
 * simulation's stream (cell grid and degrees, with temporary pool memory freed
 * before it returns) and changes nothing in `sim`. Not included: the per-call
 * buffers of fs_run_protocol (16 B per field step, 8 B more with per-step flip
 * counts, 8 B per logged flip), which come from the pool.
 * Errors: FS_ERR_INVALID (NULL argument, a parameter out of range, a
 * neighbourhood above the degree limit), FS_ERR_OOM, FS_ERR_CUDA. */
fs_status fs_workspace_bytes(const fs_sim* sim, const fs_params* p, size_t* bytes);

/* Carves the simulation's device state from the caller's buffer (memory a
 * framework's allocator owns, say) instead of the library's stream-ordered pool.
 * dev_ptr: device or managed memory, 256-byte aligned, `bytes` long; the state
 * takes the buffer's bottom, the build's temporaries its top while fs_set_params
 * runs (fs_workspace_bytes gives the need of a parameter set). The caller keeps
 * the buffer alive and otherwise unused until fs_destroy or the next bind; the
 * library never frees it. dev_ptr NULL returns to the pool. cuda_stream, when not
 * NULL, becomes the simulation's stream (as fs_set_stream). Call before
 * fs_set_params; a build that does not fit returns FS_ERR_OOM (after the work it
 * queued has ended) and leaves the simulation without parameters, to be bound
 * again. Per-call buffers still come from the pool.
 * Errors: FS_ERR_INVALID (NULL sim; a misaligned or non-device pointer),
 * FS_ERR_STATE (parameters already set). */
fs_status fs_bind_workspace(fs_sim* sim, void* dev_ptr, size_t bytes, void* cuda_stream);

/* Sets the parameters, draws h_k^(i) (Philox4x32-10 counter (i, r, instance, 0),
 * Box-Muller, redrawn while <= 0; Sec. "Imperfections and disorder") and builds
 * the neighbour tensors on the device (cell grid, CSR rows ascending, per-pair
 * coefficients P_ij = mhat_i . T_ij mhat_j and Q_ij = mhat_perp_i . T_ij mhat_j,
 * T_ij = alpha (3 rhat rhat^T - I) / r^3, Eq. 3). Resets spins to +1. */
fs_status fs_set_params(fs_sim* sim, const fs_params* p);

/* Replaces the drawn coercive fields with the caller's (n values, > 0). */
fs_status fs_set_hk(fs_sim* sim, const double* hk, int64_t n);

/* Spins (n values in {-1,+1}); default after fs_set_params is all +1. */
fs_status fs_set_spins(fs_sim* sim, const int8_t* s, int64_t n);

/* External field (Sec. "External field", global form) and the field-step index
 * that keys the thermal draw (Philox counter (i, step, instance, 1)). */
fs_status fs_set_field(fs_sim* sim, double hx, double hy, uint32_t step);

/* One relax at the current field (Sec. "Dynamics"): recompute every field,
 * then flip the flippable island with the largest Eq. 5 LHS (lowest index on
 * ties) until none is flippable. The first log_cap flipped islands go to
 * log_spin (may be NULL). *n_flips receives the number of flips. */
fs_status fs_relax(fs_sim* sim, uint32_t* log_spin, int64_t log_cap, int64_t* n_flips);

/* K field steps; step t applies (hx[t], hy[t]) with thermal step index
 * step0 + t, then relaxes. Host buffers. log_step/log_spin receive the first
 * log_cap flips (may be NULL), flips_per_step[K] may be NULL, *seq_hash is
 * updated in place (start from fs_hash_init()), *n_flips receives the total.
 * resweep != 0 recomputes every dipolar sum from the neighbour tensors at every
 * field step (the paper's order); resweep == 0 keeps the exact fixed-point sums
 * that the flips maintain and only re-evaluates Eq. 5/6. Both give identical
 * results because integer sums are exact. */
fs_status fs_run_protocol(fs_sim* sim, const double* hx, const double* hy, int64_t K,
                          uint32_t step0, int32_t resweep, uint32_t* log_step,
                          uint32_t* log_spin, int64_t log_cap, int64_t* flips_per_step,
                          uint64_t* seq_hash, int64_t* n_flips);

/* As fs_run_protocol with device buffers, queued on the simulation's stream
 * without waiting: d_hx/d_hy [K] in; d_log_step/d_log_spin [log_cap] (or NULL),
 * d_flips_per_step [K] (or NULL), d_out[4] receives {status, n_flips,
 * seq_hash, 0} as int64/uint64 when the queued work ends (seq_hash starts from
 * fs_hash_init()). Returns an error only for bad arguments or launch failures. */
fs_status fs_run_protocol_dev(fs_sim* sim, const double* d_hx, const double* d_hy, int64_t K,
                              uint32_t step0, int32_t resweep, uint32_t* d_log_step,
                              uint32_t* d_log_spin, int64_t log_cap,
                              int64_t* d_flips_per_step, uint64_t* d_out);

/* Spins from a device buffer (n int8 values in {-1,+1}, not checked), queued on
 * the simulation's stream; the next protocol call recomputes every dipolar sum. */
fs_status fs_set_spins_dev(fs_sim* sim, const int8_t* d_s, int64_t n);

/* Per-kernel timing (profiling subsystem): with profiling on, every field step
 * of fs_run_protocol / fs_run_protocol_dev brackets its sweep and its relax
 * launch with CUDA events on the simulation's stream. fs_set_profiling resets
 * the totals; fs_get_profile waits for the recorded events and returns them. */
typedef struct {
    double sweep_ms, relax_ms;  /* summed device time of the sweeps and relaxes */
    int64_t sweep_launches, relax_launches;
    int64_t rechecks;           /* FP32 path: FP64 recheck rounds (single-flip relax) and
                                   FP64 evaluations of candidates (multi-flip relax) so far */
    int64_t fallbacks;          /* rechecks that overflowed into a full scan */
    int64_t rounds;             /* multi-flip relax: rounds that flipped so far */
    int64_t idle_rounds;        /* multi-flip relax: candidate passes that flipped nothing */
    int64_t round_flips;        /* multi-flip relax: flips made in its rounds */
    int64_t handoffs;           /* multi-flip relax: field steps handed to the single-flip one */
} fs_profile;
fs_status fs_set_profiling(fs_sim* sim, int32_t on);
fs_status fs_get_profile(fs_sim* sim, fs_profile* out);

/* Sweep autotuner: times the field-and-margin sweep with 2, 4, 8, 16 and 32 lanes per
 * CSR row, each built for 4 and for 5 resident blocks per SM, on this system and
 * keeps the fastest for later calls; *lanes_out (may be NULL) receives the lanes
 * per row of the choice. Every choice gives bit-identical results. */
fs_status fs_autotune(fs_sim* sim, int32_t* lanes_out);

/* Current spins, n values. */
fs_status fs_get_spins(const fs_sim* sim, int8_t* out, int64_t n);

/* Total field (Eq. 2) of every island in its own frame at the current spins,
 * external field and thermal step: h_par = h . mhat_i, h_perp = h . mhat_perp_i.
 * In FS_FP32_RECHECK the values are those of the FP32 evaluation. */
fs_status fs_get_fields(fs_sim* sim, double* h_par, double* h_perp, int64_t n);

/* Eq. 5 LHS of every island at the current state, in the simulation's precision,
 * with bounds lo <= LHS(FS_FP64) <= hi (for FS_FP64, lo = hi = lhs). Any output
 * may be NULL. */
fs_status fs_get_lhs(fs_sim* sim, double* lhs, double* lo, double* hi, int64_t n);

fs_status fs_get_hk(const fs_sim* sim, double* out, int64_t n);
fs_status fs_get_geometry(const fs_sim* sim, double* x, double* y, double* theta, int64_t n);
fs_status fs_get_info(const fs_sim* sim, fs_info* out);

/* Neighbour CSR (unpadded): row_ptr[n+1], col[nnz] ascending per row, and the
 * FP64-path coefficients P[nnz], Q[nnz] (fixed point converted back to double;
 * field at i per unit spin of j, in i's frame). Any output may be NULL. */
fs_status fs_get_csr(const fs_sim* sim, int64_t* row_ptr, int32_t* col, double* P, double* Q);

/* ---- External fields beyond the global one; thermal protocols ----------------
 * Sec. "External field": besides the global field, a field set per island
 * (local) or given as a spatial vector field, each a discrete time series. Both
 * are lab-frame vectors added to the global field of the field step. Series are
 * indexed by the field-step index, the one that keys the thermal draw (step0 + t
 * in fs_run_protocol, `step` in fs_set_field); a call that reaches a step at or
 * beyond a series' length fails with FS_ERR_INVALID. At most one local or spatial
 * series is set at a time (setting one replaces the other); K = 0 clears it.
 * Series are copied to device memory from the library's pool (not from a bound
 * workspace) and freed by fs_destroy, by fs_set_params (new parameters drop every
 * series) or by the next call. Batches accept members with series as long as
 * they cover the protocol; the allocation-free entry point applies the global
 * field only.
 * Errors: FS_ERR_STATE (parameters not set), FS_ERR_INVALID (bad sizes, a
 * non-finite value), FS_ERR_OOM, FS_ERR_CUDA. */

/* Local field: hx[t*n + i], hy[t*n + i] at field step t for island i (canonical
 * order), t < K; n must be the island count. Device bytes: 16 K n + 24 n. */
fs_status fs_set_field_local(fs_sim* sim, const double* hx, const double* hy, int64_t K,
                             int64_t n);

/* Spatial field h_ext(r) on a grid of gw x gh cells, cell (cx, cy) covering
 * [x0 + cx dx, x0 + (cx + 1) dx) x [y0 + cy dy, y0 + (cy + 1) dy): at field step
 * t the cell holds (hx, hy)[(t gh + cy) gw + cx]. An island takes the value of the
 * cell that contains its centre (an island outside the grid, the nearest edge
 * cell's). Device bytes: 16 K gw gh + 28 n. */
fs_status fs_set_field_spatial(fs_sim* sim, const double* hx, const double* hy, int64_t K,
                               int32_t gw, int32_t gh, double x0, double y0, double dx,
                               double dy);

/* Thermal protocol (Sec. "Thermal field"; the annealing of Sec. "Domain size in
 * square ASI" lowers sigma_th step by step): field step t draws its thermal field
 * with standard deviation sigma[t] (>= 0) instead of sigma_th, t < K. The
 * simulation's parameters must have sigma_th > 0 (which sets up the thermal
 * buffers). Resets the FP64 draws kept from earlier calls. K = 0 clears it. */
fs_status fs_set_sigma_series(fs_sim* sim, const double* sigma, int64_t K);

/* ---- Input encoders (Sec. "Simulation framework") -----------------------------
 * The encoder turns input values into a series of global external fields. Input
 * u_k (k < m) becomes one period of `period` values, amplitude
 * A_k = h_lo + (h_hi - h_lo) u_k, at j = 0 .. period - 1:
 *   FS_ENCODE_SINUSOID: A_k sin(2 pi j / period) along angle_deg;
 *   FS_ENCODE_SAWTOOTH: A_k (2 j / (period - 1) - 1) along angle_deg, a linear rise
 *     from -A_k to +A_k (period >= 2);
 *   FS_ENCODE_ROTATION: magnitude A_k at the angle angle_deg + 360 j / period.
 * Writes hx, hy[k period + j] (host buffers of m period values; host arithmetic,
 * no device work). Angles in degrees, (deg pi) / 180. FS_ERR_INVALID on bad
 * arguments. */
typedef enum { FS_ENCODE_SINUSOID = 0, FS_ENCODE_SAWTOOTH = 1, FS_ENCODE_ROTATION = 2 } fs_encoder;
fs_status fs_encode(int32_t kind, const double* inputs, int64_t m, int32_t period, double h_lo,
                    double h_hi, double angle_deg, double* hx, double* hy);

/* ---- Spin-spin correlation (Sec. "Domain size in square ASI") -----------------
 * The correlation of two spins is +1 when their dipolar interaction is at its
 * minimum and -1 at its maximum: sign(s_i s_j v_ij), v_ij = 3 (mhat_i . rhat_ij)
 * (mhat_j . rhat_ij) - mhat_i . mhat_j (the pair energy of Eq. 3 is
 * -alpha s_i s_j v_ij / r^3). Over the current spins, every unordered pair with
 * |r_ij|^2 <= rmax^2 (1 + 1e-9) falls into bin floor(|r_ij| / bin_width + 1e-7)
 * (whole multiples of bin_width, up to rounding, go to the upper bin); pairs with
 * |v_ij| <= 1e-9 and bins >= nbins are left out. Host outputs, nbins values each
 * (1 <= nbins <= 2048): pair_count[b] pairs, corr_sum[b] the sum of their
 * correlations (the mean correlation is corr_sum / pair_count). Positions in units
 * of the array's spacing a as generated. Runs one GPU pass over a cell grid of
 * cells rmax wide; synchronous on the simulation's stream.
 * Errors: FS_ERR_STATE (parameters not set), FS_ERR_INVALID, FS_ERR_OOM,
 * FS_ERR_CUDA. */
fs_status fs_correlation(fs_sim* sim, double rmax, double bin_width, int32_t nbins,
                         int64_t* pair_count, int64_t* corr_sum);

/* ---- Allocation-free evaluation ----------------------------------------------
 * The paper has no counterpart; this is a service for callers that cannot
 * allocate device memory when they call (a control loop that must not block on
 * the CUDA allocator, or a process whose device memory is wholly reserved by
 * another framework's pool).
 *
 * One field-and-margin sweep in the FS_FP64 arithmetic (exact 64-bit dipolar sums
 * over sim's neighbour tensors, external field (hx, hy), thermal draw of `step`,
 * the same astroid and alignment test as fs_get_lhs) for the caller's spins, and
 * the argmax of the relax rule.
 *   sim      built simulation (fs_set_params done); its spins are not used or
 *            changed; n = its island count, at most 2,097,152 (2^21)
 *   d_spins  device, n int8 in {-1,+1} (values are not checked)
 *   d_lhs    device output, n doubles: the astroid left-hand side (the value
 *            fs_get_lhs reports) of every flippable island, 0 for the others
 *   d_best   device output, one int64: the flippable island with the largest
 *            LHS (lowest index on ties), or -1 when none is flippable
 *   stream   cudaStream_t to queue on (NULL = legacy default); the call returns
 *            without waiting, the outputs are valid once the stream gets there
 * It calls no allocator: its scratch (the max-tree and its arrival counters) is
 * one static device array of 2 MiB in the library, which every GPU that loads the
 * library holds until the process exits. The first call on a device looks up that
 * array's address (once per device, with that device current); later calls only
 * queue a memset of the counters and one kernel. All calls share the array, so
 * calls whose work overlaps on the GPU race and give undefined results.
 * The device current at the call must be the one that was current when the
 * simulation's parameters were set (its buffers live there).
 * Returns FS_ERR_INVALID (NULL pointer or n above the limit), FS_ERR_STATE
 * (parameters not set, or another device current) or FS_ERR_CUDA (lookup or
 * launch failed); no message is recorded for fs_last_error. */
fs_status fs_eval_argmax_static(const fs_sim* sim, const int8_t* d_spins, double hx, double hy,
                                uint32_t step, double* d_lhs, int64_t* d_best, void* stream);

/* ---- Batched ensembles ------------------------------------------------------
 * Advances n independent simulations (an ensemble of disorder realisations or a
 * parameter sweep, Sec. "Simulation framework") through the same protocol
 * together, all members in flight at once, the protocol captured in one CUDA
 * graph on a stream of the batch's own, ordered after sims[0]'s queued work.
 * Every member must have parameters set and the same precision. Per member i:
 * n_flips[i], seq_hash[i] (in/out, start from fs_hash_init()), status[i]
 * (fs_status), flips_per_step[i*K + t] (or NULL). Results equal those of running
 * each member alone.
 *
 * Schedules:
 * FS_BATCH_PERSISTENT: one persistent kernel (two CTAs per SM) in which every
 *   member advances its own field steps: a free CTA takes the relax of a member
 *   whose step has been swept (largest members first), else a chunk of a member's
 *   sweep, so that relaxes (latency-bound chains) overlap other members' sweeps
 *   (bandwidth-bound) and no member waits for another's step. Not for members
 *   with a local or spatial field (FS_ERR_INVALID).
 * FS_BATCH_PER_STEP: per field step one sweep launch over every member's rows,
 *   then one relax launch with a CTA per member.
 * FS_BATCH_TWO_CHAINS: the same launches for two halves of the members (taken
 *   alternately by size), each half with its own chain of field steps, so that one
 *   half's relaxes may overlap the other's sweeps.
 * FS_BATCH_AUTO: per step, in two chains from twice as many members as SMs
 *   (measured faster on the 512-member ensemble: 1.25 s in two chains, 1.26 s in
 *   one, 1.42 s persistent, FP32; a relax CTA holds half an SM's registers, so a
 *   CTA sweeping beside it has a fraction of the warps the sweep kernel runs with).
 * The sweep's lanes per CSR row are timed on the batch's own rows first (for a
 * batch whose sweep is long enough).
 *   hx, hy   host, K doubles each: the external field of every field step
 *   resweep  1: the dipolar sums recomputed in every field step's sweep; 0: the
 *            exact sums the flips keep are used (the same bits)
 * Errors: FS_ERR_INVALID (NULL arrays, n <= 0, an unknown schedule, members of
 * different precisions, a local, spatial or thermal series shorter than K, or the
 * persistent schedule with a local or spatial field), FS_ERR_STATE (a member
 * without parameters), FS_ERR_CUDA, FS_ERR_BOUNDS (a persistent run in which no
 * work finished anywhere for 10 s), else the first member's failing status (each
 * member's own in status[]). */
typedef enum {
    FS_BATCH_AUTO = 0,
    FS_BATCH_PERSISTENT = 1,
    FS_BATCH_PER_STEP = 2,
    FS_BATCH_TWO_CHAINS = 3
} fs_batch_schedule;

fs_status fs_batch_run_protocol_ex(fs_sim* const* sims, int32_t n, const double* hx,
                                   const double* hy, int64_t K, int32_t resweep,
                                   int32_t schedule, int64_t* n_flips, uint64_t* seq_hash,
                                   int32_t* status, int64_t* flips_per_step);

/* fs_batch_run_protocol_ex with FS_BATCH_AUTO. */
fs_status fs_batch_run_protocol(fs_sim* const* sims, int32_t n, const double* hx,
                                const double* hy, int64_t K, int32_t resweep, int64_t* n_flips,
                                uint64_t* seq_hash, int32_t* status, int64_t* flips_per_step);

/* ---- Continuous-batching server ---------------------------------------------
 * Builder threads admit requests while their estimated device footprint fits the
 * budget and build them on side streams; every admitted request then gets a
 * stream of its own on which a graph of a few field steps of its protocol is
 * launched again and again (two launches queued at most) until the protocol is
 * done, so requests that arrive while others run start as soon as they are built
 * and all of them overlap on the device. Builds run at the highest stream
 * priority and smaller requests (short kernels) at higher priorities than larger
 * ones. Admission order: a request waiting longer than 10 s first (oldest
 * first), else the least estimated work (islands x field steps). Every request
 * relaxes with the single-flip chain (FS_RELAX_SINGLE: one CTA, one SM), which
 * makes the most flips per SM on a shared device. Results equal those of running
 * each request alone. */
typedef struct fs_server fs_server;

typedef struct {
    int32_t kind;          /* fs_geom */
    int32_t nx, ny;
    double a;
    fs_params params;
    int64_t K;             /* field steps */
    const double* hx;      /* [K], copied at submit */
    const double* hy;      /* [K], copied at submit */
    int8_t* spins_out;     /* optional host buffer [n] for the final spins (written before done) */
} fs_request;

typedef struct {
    int32_t status;        /* fs_status of the simulation */
    int32_t done;          /* 1 when finished */
    int64_t n;             /* islands */
    int64_t n_flips;
    uint64_t seq_hash;
    double t_submit, t_admit, t_done; /* seconds on the server's monotonic clock */
} fs_result;

/* hbm_budget: bytes of device memory the server may hold for admitted requests. */
fs_status fs_server_create(size_t hbm_budget, int32_t max_active, fs_server** out);
fs_status fs_server_submit(fs_server* srv, const fs_request* req, uint64_t* ticket);
/* FS_ERR_STATE while the request is not done; FS_OK with *out filled when done. A
 * result is handed out once: the ticket is then forgotten (FS_ERR_INVALID after). */
fs_status fs_server_poll(fs_server* srv, uint64_t ticket, fs_result* out);
/* Blocks until every submitted request is done. */
fs_status fs_server_drain(fs_server* srv);
/* Seconds on the server's clock (for arrival schedules). */
double fs_server_now(const fs_server* srv);
void fs_server_destroy(fs_server* srv);
const char* fs_server_last_error(const fs_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* FLATSPIN_B300_H */
