/*
 * flatspin_oracle.c - plain, slow FP64 CPU oracle of the flatspin dipole model
 * and its greedy relax loop (Jensen et al., "flatspin: A Large-Scale Artificial
 * Spin Ice Simulator", arXiv 2002.11401).
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the benchmark's
 * CPU-baseline leg are the only users. The library's product path never loads,
 * links or calls this code, and this code includes nothing from the library.
 *
 * Everything is evaluated straight from the paper's definitions, in double
 * precision, in the order the paper states them:
 *   - Sec. "Magnets as dipoles", Eq. (1): m_i = s_i * mhat_i, mhat_i = (cos t_i, sin t_i).
 *   - Sec. "Magnetic Fields and Temperature", Eq. (2): h_i = h_dip + h_ext + h_th.
 *   - Sec. "Magnetic dipole-dipole interactions", Eq. (3) and the neighbourhood
 *     cutoff paragraph: h_dip is evaluated from positions for every neighbour j
 *     (ascending j) at every evaluation; no precomputed tensor is stored.
 *   - Sec. "Thermal field": two orthogonal components ~ N(0, sigma_th^2).
 *   - Sec. "Switching", Eq. (5) "esw" and Eq. (6) "sw2".
 *   - Sec. "Imperfections and disorder": h_k^(i) ~ N(h_k, k_disorder * h_k), > 0.
 *   - Sec. "Dynamics": flip the flippable spin with the largest left-hand side of
 *     Eq. (5), repeat until none is flippable, fields held constant over a relax.
 *   - Sec. "Geometries" and Fig. "geometries": square (closed edges), pinwheel
 *     (square islands rotated 45 degrees about their centres, Sec. "Superferro-
 *     magnetism in pinwheel ASI") and kagome.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - fractional powers act on |h_par| and |h_perp|; Eq. (6) supplies the sign;
 *   - both inequalities are strict;
 *   - ties in the largest left-hand side go to the lowest spin index;
 *   - the cutoff is inclusive: |r_ij|^2 <= (cutoff*a)^2 * (1 + 1e-9);
 *   - random numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     SC'11, "Parallel random numbers: as easy as 1, 2, 3") and Box-Muller.
 *
 * Variants, with the readings they take where the paper gives only a figure or a
 * name (all listed in the design notes): the open-edged square, the pinwheel
 * "diamond" and "lucky-knot" edge forms and the ising array (Fig. "geometries");
 * the parallel-only switching criterion the pinwheel section contrasts with
 * Eq. (5); per-island and spatial external fields and the sinusoid, sawtooth and
 * rotation input encoders (Sec. "External field", Sec. "Simulation framework");
 * per-step thermal standard deviations (annealing) and the spin-spin correlation
 * against separation (Sec. "Domain size in square ASI").
 *
 * Parity pins (tests/test_oracle_*.py): the pair field against the closed-form
 * field of a point dipole; Eq. (5) against the Stoner-Wohlfarth astroid's closed
 * form; the relax against a brute-force state table and the energy invariant;
 * geometry counts against the paper's printed count (29x29 kagome = 2638) and
 * the 8-neighbour square neighbourhood of the performance section; Philox
 * against an independent third-party implementation; the variants against the
 * paper's 25 x 25 = 1250 pinwheel count, closed-form switching fields and switching
 * times, uniform local and spatial fields against the global field, constant
 * thermal series against sigma_th, and the correlation against closed-form pair
 * counts and the sign of the Eq. (3) pair energy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_INVALID 1
#define OR_ERR_OOM 2
#define OR_ERR_NOT_CONVERGED 4

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */
/* ------------------------------------------------------------------------ */

static int g_threads = 1;

void or_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int or_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and Box-Muller                                              */
/* ------------------------------------------------------------------------ */

/* One Philox4x32 round: two 32x32->64 multiplies, the high halves xored with
 * the other counter words and the key (Salmon et al. SC'11, Sec. 4). */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

/* Philox4x32 with 10 rounds; the key is bumped by the Weyl constants between
 * rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* Two uniforms in (0,1) from the four output words (53-bit mantissas, offset by
 * half a step so that 0 and 1 are never produced), then the Box-Muller pair. */
void or_box_muller(const uint32_t w[4], double* z0, double* z1) {
    const uint64_t a = ((uint64_t)w[0] << 32) | (uint64_t)w[1];
    const uint64_t b = ((uint64_t)w[2] << 32) | (uint64_t)w[3];
    const double u1 = ((double)(a >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = ((double)(b >> 11) + 0.5) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    const double ang = (2.0 * M_PI) * u2;
    *z0 = rad * cos(ang);
    *z1 = rad * sin(ang);
}

static void normal_pair(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                        double* z0, double* z1) {
    const uint32_t ctr[4] = {w0, w1, w2, w3};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    or_box_muller(out, z0, z1);
}

/* Sec. "Imperfections and disorder": h_k^(i) = h_k (1 + k_disorder z), z from
 * counter (i, r, instance, 0); a non-positive draw is redrawn with r = 1, 2, ... */
void or_draw_hk(int64_t n, double hk, double kdis, uint64_t seed, uint32_t instance, double* out) {
    for (int64_t i = 0; i < n; ++i) {
        double v = 0.0;
        for (uint32_t r = 0;; ++r) {
            double z0, z1;
            normal_pair(seed, (uint32_t)i, r, instance, 0u, &z0, &z1);
            v = hk * (1.0 + kdis * z0);
            if (v > 0.0) break;
        }
        out[i] = v;
    }
}

/* Sec. "Thermal field": (th_par, th_perp) = sigma_th (z0, z1) in the magnet's
 * frame, counter (i, step, instance, 1). */
void or_thermal(int64_t n, double sigma, uint64_t seed, uint32_t instance, uint32_t step,
                double* th_par, double* th_perp) {
    for (int64_t i = 0; i < n; ++i) {
        double z0, z1;
        normal_pair(seed, (uint32_t)i, step, instance, 1u, &z0, &z1);
        th_par[i] = sigma * z0;
        th_perp[i] = sigma * z1;
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. "Geometries", Fig. "geometries")                           */
/* ------------------------------------------------------------------------ */

enum {
    OR_SQUARE = 0,
    OR_PINWHEEL = 1,
    OR_KAGOME = 2,
    OR_SQUARE_OPEN = 3,
    OR_PINWHEEL_DIAMOND = 4,
    OR_PINWHEEL_LUCKY_KNOT = 5,
    OR_ISING = 6
};

typedef struct {
    int64_t X, Y; /* integer lattice coordinates (see or_geometry) */
    int deg;      /* island angle in degrees */
} site;

static int site_cmp(const void* pa, const void* pb) {
    const site* a = (const site*)pa;
    const site* b = (const site*)pb;
    if (a->Y != b->Y) return a->Y < b->Y ? -1 : 1;
    if (a->X != b->X) return a->X < b->X ? -1 : 1;
    return 0;
}

/* Upper bound on the number of islands, for the caller's buffers. */
int64_t or_geometry_capacity(int kind, int32_t nx, int32_t ny) {
    if (nx <= 0 || ny <= 0) return 0;
    if (kind == OR_KAGOME) return 6 * (int64_t)nx * ny;
    if (kind == OR_ISING) return (int64_t)nx * ny;
    return (int64_t)nx * (ny + 1) + (int64_t)ny * (nx + 1);
}

/* Island centres and angles, in the canonical order (ascending y, then x).
 *
 * Square, nx x ny cells, lattice spacing a: horizontal islands (0 degrees) at
 * (x + 1/2, y) for x < nx, y <= ny, and vertical islands (90 degrees) at
 * (x, y + 1/2) for x <= nx, y < ny: closed edges, every cell has four islands.
 * Integer coordinates are in half spacings: (X, Y) -> (X * 0.5 * a, Y * 0.5 * a).
 *
 * Pinwheel: the square's centres, each island turned 45 degrees about its
 * centre (45 and 135 degrees).
 *
 * The figure of the geometries names more edge forms without defining them; the
 * readings here (stated in the design notes) are:
 * - square, open edges: the closed square without the islands on its outer
 *   boundary (horizontal islands at y = 0 and y = ny, vertical ones at x = 0 and
 *   x = nx): 2 nx ny - nx - ny islands;
 * - pinwheel "diamond": nx x ny unit cells of one horizontal island at
 *   (x + 1/2, y) and one vertical at (x, y + 1/2), each turned 45 degrees:
 *   2 nx ny islands (the pinwheel section's 25 x 25 array has 1250);
 * - pinwheel "lucky-knot": the open-edged square's islands turned 45 degrees;
 * - ising: one island at every lattice point (x, y), x < nx, y < ny, all along
 *   x (0 degrees), a single sublattice.
 *
 * Kagome, nx x ny flat-top hexagons with edge length a: hexagon (c, r) centred
 * at (1.5 c, sqrt(3) r + (c odd ? sqrt(3)/2 : 0)); one island on the midpoint
 * of each edge, along the edge; shared edges are kept once. Integer coordinates
 * are in quarter edges along x and sqrt(3)/4 along y:
 * (X, Y) -> (X * 0.25 * a, Y * (sqrt(3)/4) * a).
 *
 * Angles are converted as (deg * M_PI) / 180. Returns the number of islands. */
int64_t or_geometry(int kind, int32_t nx, int32_t ny, double a, double* x, double* y,
                    double* theta) {
    const int64_t cap = or_geometry_capacity(kind, nx, ny);
    if (cap <= 0 || !(a > 0.0)) return -1;
    site* s = (site*)malloc(sizeof(site) * (size_t)cap);
    if (!s) return -2;
    int64_t m = 0;
    double sx, sy;
    if (kind == OR_SQUARE || kind == OR_PINWHEEL || kind == OR_SQUARE_OPEN ||
        kind == OR_PINWHEEL_DIAMOND || kind == OR_PINWHEEL_LUCKY_KNOT) {
        const int rot = (kind == OR_PINWHEEL || kind == OR_PINWHEEL_DIAMOND ||
                         kind == OR_PINWHEEL_LUCKY_KNOT) ? 45 : 0;
        const int open = kind == OR_SQUARE_OPEN || kind == OR_PINWHEEL_LUCKY_KNOT;
        const int cells = kind == OR_PINWHEEL_DIAMOND;
        /* horizontal islands: rows y = 0..ny (closed), 1..ny-1 (open), 0..ny-1 (cells) */
        const int64_t hy0 = open ? 1 : 0, hy1 = (open || cells) ? ny - 1 : ny;
        /* vertical islands: columns x = 0..nx (closed), 1..nx-1 (open), 0..nx-1 (cells) */
        const int64_t vx0 = open ? 1 : 0, vx1 = (open || cells) ? nx - 1 : nx;
        for (int64_t yy = hy0; yy <= hy1; ++yy)
            for (int64_t xx = 0; xx < nx; ++xx) {
                s[m].X = 2 * xx + 1;
                s[m].Y = 2 * yy;
                s[m].deg = 0 + rot;
                ++m;
            }
        for (int64_t yy = 0; yy < ny; ++yy)
            for (int64_t xx = vx0; xx <= vx1; ++xx) {
                s[m].X = 2 * xx;
                s[m].Y = 2 * yy + 1;
                s[m].deg = 90 + rot;
                ++m;
            }
        sx = 0.5;
        sy = 0.5;
    } else if (kind == OR_ISING) {
        for (int64_t yy = 0; yy < ny; ++yy)
            for (int64_t xx = 0; xx < nx; ++xx) {
                s[m].X = 2 * xx;
                s[m].Y = 2 * yy;
                s[m].deg = 0;
                ++m;
            }
        sx = 0.5;
        sy = 0.5;
    } else if (kind == OR_KAGOME) {
        /* edge k midpoint offset from the centre, in (quarter, sqrt(3)/4) units,
         * for the directions 30 + 60k degrees; the island lies along the edge,
         * at (120 + 60k) mod 180 degrees. */
        static const int off[6][2] = {{3, 1}, {0, 2}, {-3, 1}, {-3, -1}, {0, -2}, {3, -1}};
        for (int64_t c = 0; c < nx; ++c)
            for (int64_t r = 0; r < ny; ++r) {
                const int64_t CX = 6 * c;
                const int64_t CY = 4 * r + ((c & 1) ? 2 : 0);
                for (int k = 0; k < 6; ++k) {
                    s[m].X = CX + off[k][0];
                    s[m].Y = CY + off[k][1];
                    s[m].deg = (120 + 60 * k) % 180;
                    ++m;
                }
            }
        sx = 0.25;
        sy = sqrt(3.0) / 4.0;
    } else {
        free(s);
        return -1;
    }
    qsort(s, (size_t)m, sizeof(site), site_cmp);
    int64_t n = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (n > 0 && s[n - 1].X == s[i].X && s[n - 1].Y == s[i].Y) continue;
        s[n++] = s[i];
    }
    for (int64_t i = 0; i < n; ++i) {
        x[i] = ((double)s[i].X * sx) * a;
        y[i] = ((double)s[i].Y * sy) * a;
        theta[i] = ((double)s[i].deg * M_PI) / 180.0;
    }
    free(s);
    return n > 0 ? n : -1;
}

/* ------------------------------------------------------------------------ */
/* Eq. (3): the field of dipole j at the position of dipole i                */
/* ------------------------------------------------------------------------ */

/* h = alpha * [ 3 r (m . r) / |r|^5 - m / |r|^3 ] with r = r_i - r_j (reduced
 * units of the lattice spacing) and m the moment of j. */
void or_dipole_field(double rx, double ry, double mx, double my, double alpha, double* hx,
                     double* hy) {
    const double r2 = rx * rx + ry * ry;
    const double r = sqrt(r2);
    const double r3 = r2 * r;
    const double r5 = r3 * r2;
    const double mr = mx * rx + my * ry;
    *hx = alpha * (3.0 * rx * mr / r5 - mx / r3);
    *hy = alpha * (3.0 * ry * mr / r5 - my / r3);
}

/* ------------------------------------------------------------------------ */
/* Eq. (5) "esw" and Eq. (6) "sw2"                                            */
/* ------------------------------------------------------------------------ */

/* Left-hand side of Eq. (5): (|h_par| / (b h_k))^(2/gamma) + (|h_perp| / (c h_k))^(2/beta). */
double or_astroid_lhs(double hpar, double hperp, double hk, double b, double c, double beta,
                      double gamma) {
    return pow(fabs(hpar) / (b * hk), 2.0 / gamma) + pow(fabs(hperp) / (c * hk), 2.0 / beta);
}

/* Eq. (5) > 1 and Eq. (6): h . m_i < 0, i.e. s_i h_par < 0. */
int or_flippable(int s, double hpar, double lhs) { return ((double)s * hpar < 0.0) && (lhs > 1.0); }

/* The simpler switching criterion the pinwheel section contrasts with Eq. (5):
 * only the field component along the magnet counts. Read as: the island may switch
 * when the component opposing its magnetisation exceeds its coercive field,
 * -s h_par > h_k; its "left-hand side" is |h_par| / h_k, so that the same rule
 * (LHS > 1 and Eq. (6)) and the same ranking (largest LHS first) apply. */
double or_parallel_lhs(double hpar, double hk) { return fabs(hpar) / hk; }

/* ------------------------------------------------------------------------ */
/* Neighbourhoods (Sec. "Magnetic dipole-dipole interactions", cutoff)       */
/* ------------------------------------------------------------------------ */

static int within_cutoff(double dx, double dy, double rc2) { return dx * dx + dy * dy <= rc2; }

static int cmp_i32(const void* a, const void* b) {
    const int32_t u = *(const int32_t*)a, v = *(const int32_t*)b;
    return (u > v) - (u < v);
}

/* All pairs j != i with |r_i - r_j| inside the cutoff, each row ascending in j.
 * brute != 0 compares every pair; otherwise a uniform grid of cells no smaller
 * than the cutoff limits the candidates to the 3x3 surrounding cells. Returns nnz,
 * or -1 on bad input, -2 when out of memory. rowptr/col may be NULL (count only). */
int64_t or_neighbors(int64_t n, const double* x, const double* y, double rc, int brute,
                     int64_t* rowptr, int32_t* col, int64_t cap) {
    if (n < 0 || !(rc > 0.0)) return -1;
    const double rc2 = rc * rc * (1.0 + 1e-9);
    int64_t nnz = 0;
    if (rowptr) rowptr[0] = 0;
    if (brute || n < 2) {
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                if (within_cutoff(x[i] - x[j], y[i] - y[j], rc2)) {
                    if (col && nnz < cap) col[nnz] = (int32_t)j;
                    ++nnz;
                }
            }
            if (rowptr) rowptr[i + 1] = nnz;
        }
        return nnz;
    }
    double xmin = x[0], xmax = x[0], ymin = y[0], ymax = y[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < xmin) xmin = x[i];
        if (x[i] > xmax) xmax = x[i];
        if (y[i] < ymin) ymin = y[i];
        if (y[i] > ymax) ymax = y[i];
    }
    const double cell = rc * 1.0001;
    const int64_t gx = (int64_t)floor((xmax - xmin) / cell) + 1;
    const int64_t gy = (int64_t)floor((ymax - ymin) / cell) + 1;
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(gx * gy));
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!head || !next || !cand) {
        free(head);
        free(next);
        free(cand);
        return -2;
    }
    for (int64_t c = 0; c < gx * gy; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        const int64_t cx = (int64_t)floor((x[i] - xmin) / cell);
        const int64_t cy = (int64_t)floor((y[i] - ymin) / cell);
        next[i] = head[cy * gx + cx];
        head[cy * gx + cx] = i;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int64_t cx = (int64_t)floor((x[i] - xmin) / cell);
        const int64_t cy = (int64_t)floor((y[i] - ymin) / cell);
        int64_t nc = 0;
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                const int64_t ux = cx + dx, uy = cy + dy;
                if (ux < 0 || uy < 0 || ux >= gx || uy >= gy) continue;
                for (int64_t j = head[uy * gx + ux]; j >= 0; j = next[j]) {
                    if (j == i) continue;
                    if (within_cutoff(x[i] - x[j], y[i] - y[j], rc2)) cand[nc++] = (int32_t)j;
                }
            }
        qsort(cand, (size_t)nc, sizeof(int32_t), cmp_i32);
        for (int64_t q = 0; q < nc; ++q) {
            if (col && nnz < cap) col[nnz] = cand[q];
            ++nnz;
        }
        if (rowptr) rowptr[i + 1] = nnz;
    }
    free(head);
    free(next);
    free(cand);
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* The simulated system                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double alpha, b, c, beta, gamma, sigma_th, cutoff_abs;
    uint64_t seed;
    uint32_t instance;
    int criterion; /* 0: Eq. (5) and (6); 1: parallel component only (or_parallel_lhs) */
} or_params;

typedef struct {
    int64_t n, nnz;
    double *x, *y, *mx, *my; /* positions, mhat_i = (cos theta_i, sin theta_i) */
    double* hk;              /* per-island coercive field h_k^(i) */
    int64_t* rowptr;
    int32_t* col;
    or_params p;
} or_sim;

void or_sim_destroy(or_sim* s) {
    if (!s) return;
    free(s->x);
    free(s->y);
    free(s->mx);
    free(s->my);
    free(s->hk);
    free(s->rowptr);
    free(s->col);
    free(s);
}

/* cutoff_abs is the neighbourhood radius in the positions' units. */
or_sim* or_sim_create(int64_t n, const double* x, const double* y, const double* theta,
                      const double* hk, double alpha, double b, double c, double beta,
                      double gamma, double sigma_th, double cutoff_abs, uint64_t seed,
                      uint32_t instance, int brute_neighbors) {
    if (n <= 0) return NULL;
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    if (!s) return NULL;
    s->n = n;
    s->x = (double*)malloc(sizeof(double) * (size_t)n);
    s->y = (double*)malloc(sizeof(double) * (size_t)n);
    s->mx = (double*)malloc(sizeof(double) * (size_t)n);
    s->my = (double*)malloc(sizeof(double) * (size_t)n);
    s->hk = (double*)malloc(sizeof(double) * (size_t)n);
    s->rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!s->x || !s->y || !s->mx || !s->my || !s->hk || !s->rowptr) {
        or_sim_destroy(s);
        return NULL;
    }
    for (int64_t i = 0; i < n; ++i) {
        s->x[i] = x[i];
        s->y[i] = y[i];
        s->mx[i] = cos(theta[i]);
        s->my[i] = sin(theta[i]);
        s->hk[i] = hk[i];
    }
    s->p.alpha = alpha;
    s->p.b = b;
    s->p.c = c;
    s->p.beta = beta;
    s->p.gamma = gamma;
    s->p.sigma_th = sigma_th;
    s->p.cutoff_abs = cutoff_abs;
    s->p.seed = seed;
    s->p.instance = instance;
    const int64_t nnz = or_neighbors(n, x, y, cutoff_abs, brute_neighbors, NULL, NULL, 0);
    if (nnz < 0) {
        or_sim_destroy(s);
        return NULL;
    }
    s->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!s->col) {
        or_sim_destroy(s);
        return NULL;
    }
    s->nnz = or_neighbors(n, x, y, cutoff_abs, brute_neighbors, s->rowptr, s->col, nnz);
    return s;
}

/* Switching criterion: 0 = Eq. (5) and (6) (the default), 1 = parallel only. */
void or_sim_set_criterion(or_sim* s, int criterion) { s->p.criterion = criterion; }

int64_t or_sim_n(const or_sim* s) { return s->n; }
int64_t or_sim_nnz(const or_sim* s) { return s->nnz; }

void or_sim_neighbors(const or_sim* s, int64_t* rowptr, int32_t* col) {
    memcpy(rowptr, s->rowptr, sizeof(int64_t) * (size_t)(s->n + 1));
    memcpy(col, s->col, sizeof(int32_t) * (size_t)s->nnz);
}

/* Eq. (3) for island i: alpha * sum over neighbours j (ascending) of the bracket,
 * with m_j = s_j mhat_j, from positions. Lab-frame vector. */
static void dip_field_at(const or_sim* S, const int8_t* s, int64_t i, double* hx, double* hy) {
    double sx = 0.0, sy = 0.0;
    for (int64_t e = S->rowptr[i]; e < S->rowptr[i + 1]; ++e) {
        const int64_t j = S->col[e];
        const double rx = S->x[i] - S->x[j];
        const double ry = S->y[i] - S->y[j];
        const double mx = (double)s[j] * S->mx[j];
        const double my = (double)s[j] * S->my[j];
        const double r2 = rx * rx + ry * ry;
        const double r = sqrt(r2);
        const double r3 = r2 * r;
        const double r5 = r3 * r2;
        const double mr = mx * rx + my * ry;
        sx += 3.0 * rx * mr / r5 - mx / r3;
        sy += 3.0 * ry * mr / r5 - my / r3;
    }
    *hx = S->p.alpha * sx;
    *hy = S->p.alpha * sy;
}

/* Full recomputation of every island's dipolar field (lab frame). */
void or_sim_dip_fields(const or_sim* S, const int8_t* s, double* hdx, double* hdy) {
    const int64_t n = S->n;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t i = 0; i < n; ++i) dip_field_at(S, s, i, &hdx[i], &hdy[i]);
}

/* Eq. (2) projected on the island's frame: h_par = h . mhat_i, h_perp = h . mhat_perp_i,
 * mhat_perp_i = (-sin theta_i, cos theta_i); the thermal field enters as th_par mhat_i +
 * th_perp mhat_perp_i. */
static void project_total(const or_sim* S, int64_t i, double hdx, double hdy, double hex,
                          double hey, double thp, double tht, double* hpar, double* hperp) {
    const double c = S->mx[i], sn = S->my[i];
    const double hx = hdx + hex + (thp * c - tht * sn);
    const double hy = hdy + hey + (thp * sn + tht * c);
    *hpar = hx * c + hy * sn;
    *hperp = -hx * sn + hy * c;
}

/* Total field of every island in its own frame, for spin state s, external field
 * (hex, hey) plus the per-island field (lx[i], ly[i]) when given (Sec. "External
 * field": local or spatial form; lab frame, added to the global field), and the
 * thermal draw of field step `step` with standard deviation sigma. */
void or_sim_fields_ext(const or_sim* S, const int8_t* s, double hex, double hey, const double* lx,
                       const double* ly, double sigma, uint32_t step, double* hpar,
                       double* hperp) {
    const int64_t n = S->n;
    double* hdx = (double*)malloc(sizeof(double) * (size_t)n);
    double* hdy = (double*)malloc(sizeof(double) * (size_t)n);
    double* tp = (double*)calloc((size_t)n, sizeof(double));
    double* tq = (double*)calloc((size_t)n, sizeof(double));
    or_sim_dip_fields(S, s, hdx, hdy);
    if (S->p.sigma_th > 0.0) or_thermal(n, sigma, S->p.seed, S->p.instance, step, tp, tq);
    for (int64_t i = 0; i < n; ++i)
        project_total(S, i, hdx[i], hdy[i], lx ? hex + lx[i] : hex, ly ? hey + ly[i] : hey,
                      tp[i], tq[i], &hpar[i], &hperp[i]);
    free(hdx);
    free(hdy);
    free(tp);
    free(tq);
}

/* As or_sim_fields_ext with the global field only and the system's sigma_th. */
void or_sim_fields(const or_sim* S, const int8_t* s, double hex, double hey, uint32_t step,
                   double* hpar, double* hperp) {
    or_sim_fields_ext(S, s, hex, hey, NULL, NULL, S->p.sigma_th, step, hpar, hperp);
}

/* The LHS the switching rule ranks by, for the system's criterion. */
double or_sim_lhs(const or_sim* S, int64_t i, double hpar, double hperp) {
    if (S->p.criterion == 1) return or_parallel_lhs(hpar, S->hk[i]);
    return or_astroid_lhs(hpar, hperp, S->hk[i], S->p.b, S->p.c, S->p.beta, S->p.gamma);
}

/* ------------------------------------------------------------------------ */
/* Argmax over flippable islands (Sec. "Dynamics")                            */
/* ------------------------------------------------------------------------ */

/* Key of island i: its Eq. (5) left-hand side when flippable, else -1. The
 * larger key wins; equal keys go to the lower index. */
static int better(double va, int64_t ia, double vb, int64_t ib) {
    return va > vb || (va == vb && ia < ib);
}

typedef struct {
    int64_t size; /* power of two >= n */
    double* v;
    int64_t* id;
} maxtree;

static int tree_init(maxtree* t, int64_t n) {
    t->size = 1;
    while (t->size < n) t->size <<= 1;
    t->v = (double*)malloc(sizeof(double) * (size_t)(2 * t->size));
    t->id = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * t->size));
    if (!t->v || !t->id) return -1;
    for (int64_t q = 0; q < 2 * t->size; ++q) {
        t->v[q] = -1.0;
        t->id[q] = INT64_MAX;
    }
    return 0;
}

static void tree_pull(maxtree* t, int64_t q) {
    const int64_t a = 2 * q, b = 2 * q + 1;
    if (better(t->v[a], t->id[a], t->v[b], t->id[b])) {
        t->v[q] = t->v[a];
        t->id[q] = t->id[a];
    } else {
        t->v[q] = t->v[b];
        t->id[q] = t->id[b];
    }
}

static void tree_set(maxtree* t, int64_t i, double key) {
    int64_t q = t->size + i;
    t->v[q] = key;
    t->id[q] = i;
    for (q >>= 1; q >= 1; q >>= 1) tree_pull(t, q);
}

static void tree_build(maxtree* t, const double* key, int64_t n) {
    for (int64_t i = 0; i < t->size; ++i) {
        t->v[t->size + i] = i < n ? key[i] : -1.0;
        t->id[t->size + i] = i < n ? i : INT64_MAX;
    }
    for (int64_t q = t->size - 1; q >= 1; --q) tree_pull(t, q);
}

static void tree_free(maxtree* t) {
    free(t->v);
    free(t->id);
}

/* ------------------------------------------------------------------------ */
/* Protocol: field steps, each followed by a relax (Sec. "Dynamics")          */
/* ------------------------------------------------------------------------ */

/* FNV-1a (64 bit) over the eight little-endian bytes of each (step, spin). */
static uint64_t fnv_flip(uint64_t h, uint32_t step, uint32_t spin) {
    const uint8_t b[8] = {(uint8_t)step,         (uint8_t)(step >> 8), (uint8_t)(step >> 16),
                          (uint8_t)(step >> 24), (uint8_t)spin,        (uint8_t)(spin >> 8),
                          (uint8_t)(spin >> 16), (uint8_t)(spin >> 24)};
    for (int q = 0; q < 8; ++q) {
        h ^= b[q];
        h *= 0x100000001b3ull;
    }
    return h;
}

uint64_t or_hash_init(void) { return 0xcbf29ce484222325ull; }
uint64_t or_hash_flip(uint64_t h, uint32_t step, uint32_t spin) { return fnv_flip(h, step, spin); }

#define OR_MODE_DEFINITION 1 /* recompute every field after every flip */
#define OR_MODE_LINEAR 2     /* linear-scan argmax even for large systems */

/* Near-tie counters: [0] picks whose runner-up is within 1e-12 (relative) of the
 * winner; [1] evaluations of an anti-aligned island with |LHS - 1| <= 1e-12;
 * [2] evaluations of an island with LHS > 1 and |h_par| <= 1e-12 * max_i h_k^(i).
 * A counted event is a place where a different but equally valid rounding order
 * could change the flip sequence. */

typedef struct {
    const or_sim* S;
    const int8_t* s;
    double hex, hey;
    const double *lx, *ly; /* this step's per-island external field, or NULL */
    const double *tp, *tq;
    double* hdx;
    double* hdy;
    double* hpar;
    double* lhs;
    double* key;
    double hscale;
    int64_t* ties;
} relax_ctx;

static void eval_island(relax_ctx* c, int64_t i) {
    const or_sim* S = c->S;
    double hpar, hperp;
    project_total(S, i, c->hdx[i], c->hdy[i], c->lx ? c->hex + c->lx[i] : c->hex,
                  c->ly ? c->hey + c->ly[i] : c->hey, c->tp ? c->tp[i] : 0.0,
                  c->tq ? c->tq[i] : 0.0, &hpar, &hperp);
    const double L = or_sim_lhs(S, i, hpar, hperp);
    c->hpar[i] = hpar;
    c->lhs[i] = L;
    const int fl = or_flippable(c->s[i], hpar, L);
    c->key[i] = fl ? L : -1.0;
    if (c->ties) {
        if ((double)c->s[i] * hpar < 0.0 && fabs(L - 1.0) <= 1e-12) c->ties[1]++;
        if (L > 1.0 && fabs(hpar) <= 1e-12 * c->hscale) c->ties[2]++;
    }
}

/* Runs K field steps. Step t uses the external field (hx[t], hy[t]), plus, when
 * lhx/lhy are given, the per-island field (lhx[t n + i], lhy[t n + i]) (Sec.
 * "External field": local, or spatial sampled at the island centres; lab frame),
 * and the thermal draw keyed by step index step0 + t with standard deviation
 * sig[t] when sig is given (a thermal protocol such as the annealing of Sec.
 * "Domain size in square ASI"), else sigma_th. `s` holds the spins on entry and
 * receives the final state. The first log_cap flips are written to
 * log_step/log_spin (may be NULL); flips_per_step[K] may be NULL; *hash is
 * updated in place (start from or_hash_init()). max_flips_per_step <= 0 means
 * 16 * n. Returns OR_OK or OR_ERR_NOT_CONVERGED. */
int or_sim_run_ext(const or_sim* S, int8_t* s, const double* hx, const double* hy,
                   const double* lhx, const double* lhy, const double* sig, int64_t K,
                   uint32_t step0, uint32_t* log_step, uint32_t* log_spin, int64_t log_cap,
                   int64_t* flips_per_step, uint64_t* hash, int64_t* n_flips,
                   int64_t max_flips_per_step, int mode, int64_t* ties) {
    const int64_t n = S->n;
    int status = OR_OK;
    if (max_flips_per_step <= 0) max_flips_per_step = 16 * n;
    relax_ctx c;
    memset(&c, 0, sizeof(c));
    c.S = S;
    c.s = s;
    c.ties = ties;
    c.hdx = (double*)malloc(sizeof(double) * (size_t)n);
    c.hdy = (double*)malloc(sizeof(double) * (size_t)n);
    c.hpar = (double*)malloc(sizeof(double) * (size_t)n);
    c.lhs = (double*)malloc(sizeof(double) * (size_t)n);
    c.key = (double*)malloc(sizeof(double) * (size_t)n);
    double* tp = NULL;
    double* tq = NULL;
    if (S->p.sigma_th > 0.0) {
        tp = (double*)malloc(sizeof(double) * (size_t)n);
        tq = (double*)malloc(sizeof(double) * (size_t)n);
    }
    c.tp = tp;
    c.tq = tq;
    c.hscale = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (S->hk[i] > c.hscale) c.hscale = S->hk[i];
    const int use_tree = !(mode & OR_MODE_LINEAR) && n > 4096;
    maxtree T;
    memset(&T, 0, sizeof(T));
    if (use_tree && tree_init(&T, n) != 0) status = OR_ERR_OOM;
    int64_t total = 0;
    uint64_t h = *hash;
    for (int64_t t = 0; t < K && status == OR_OK; ++t) {
        const uint32_t step = step0 + (uint32_t)t;
        c.hex = hx[t];
        c.hey = hy[t];
        c.lx = lhx ? lhx + t * n : NULL;
        c.ly = lhy ? lhy + t * n : NULL;
        if (tp) or_thermal(n, sig ? sig[t] : S->p.sigma_th, S->p.seed, S->p.instance, step, tp, tq);
        /* "At each simulation step, we calculate the total magnetic field". */
        or_sim_dip_fields(S, s, c.hdx, c.hdy);
        for (int64_t i = 0; i < n; ++i) eval_island(&c, i);
        if (use_tree) tree_build(&T, c.key, n);
        int64_t fl = 0;
        for (;;) {
            int64_t k = -1;
            double best = -1.0, second = -1.0;
            if (use_tree) {
                if (T.v[1] > 0.0) {
                    k = T.id[1];
                    best = T.v[1];
                    if (ties) {
                        tree_set(&T, k, -1.0);
                        second = T.v[1];
                        tree_set(&T, k, best);
                    }
                }
            } else {
                for (int64_t i = 0; i < n; ++i) {
                    if (c.key[i] < 0.0) continue;
                    if (k < 0 || better(c.key[i], i, best, k)) {
                        second = best;
                        best = c.key[i];
                        k = i;
                    } else if (c.key[i] > second) {
                        second = c.key[i];
                    }
                }
            }
            if (k < 0) break;
            if (ties && second > 0.0 && best - second <= 1e-12 * best) ties[0]++;
            if (fl >= max_flips_per_step) {
                status = OR_ERR_NOT_CONVERGED;
                break;
            }
            /* Flip k; m_k changes by 2 s_k(new) mhat_k. */
            s[k] = (int8_t)-s[k];
            if (log_step && total < log_cap) {
                log_step[total] = step;
                log_spin[total] = (uint32_t)k;
            }
            h = fnv_flip(h, step, (uint32_t)k);
            ++total;
            ++fl;
            if (mode & OR_MODE_DEFINITION) {
                or_sim_dip_fields(S, s, c.hdx, c.hdy);
                for (int64_t i = 0; i < n; ++i) eval_island(&c, i);
                if (use_tree) tree_build(&T, c.key, n);
            } else {
                const double dm = 2.0 * (double)s[k];
                for (int64_t e = S->rowptr[k]; e < S->rowptr[k + 1]; ++e) {
                    const int64_t i = S->col[e];
                    double dx, dy;
                    or_dipole_field(S->x[i] - S->x[k], S->y[i] - S->y[k], dm * S->mx[k],
                                    dm * S->my[k], S->p.alpha, &dx, &dy);
                    c.hdx[i] += dx;
                    c.hdy[i] += dy;
                    eval_island(&c, i);
                    if (use_tree) tree_set(&T, i, c.key[i]);
                }
                eval_island(&c, k);
                if (use_tree) tree_set(&T, k, c.key[k]);
            }
        }
        if (flips_per_step) flips_per_step[t] = fl;
    }
    if (use_tree) tree_free(&T);
    *hash = h;
    *n_flips = total;
    free(c.hdx);
    free(c.hdy);
    free(c.hpar);
    free(c.lhs);
    free(c.key);
    free(tp);
    free(tq);
    return status;
}

/* The global-field form of or_sim_run_ext. */
int or_sim_run(const or_sim* S, int8_t* s, const double* hx, const double* hy, int64_t K,
               uint32_t step0, uint32_t* log_step, uint32_t* log_spin, int64_t log_cap,
               int64_t* flips_per_step, uint64_t* hash, int64_t* n_flips,
               int64_t max_flips_per_step, int mode, int64_t* ties) {
    return or_sim_run_ext(S, s, hx, hy, NULL, NULL, NULL, K, step0, log_step, log_spin, log_cap,
                          flips_per_step, hash, n_flips, max_flips_per_step, mode, ties);
}

/* ------------------------------------------------------------------------ */
/* Spatial external field h_ext(r) (Sec. "External field")                   */
/* ------------------------------------------------------------------------ */

/* A spatial field given on a grid of gw x gh cells, cell (cx, cy) covering
 * [x0 + cx dx, x0 + (cx + 1) dx) x [y0 + cy dy, y0 + (cy + 1) dy), K time steps of
 * lab-frame vectors grid[t][cy][cx] (row-major), sampled at each island's centre:
 * the island takes the value of the cell that contains it (a centre outside the
 * grid takes the nearest edge cell). Writes out[t n + i]. */
void or_sample_grid(int64_t n, const double* x, const double* y, int64_t K, int32_t gw,
                    int32_t gh, double x0, double y0, double dx, double dy, const double* gx,
                    const double* gy, double* outx, double* outy) {
    for (int64_t i = 0; i < n; ++i) {
        int64_t cx = (int64_t)floor((x[i] - x0) / dx);
        int64_t cy = (int64_t)floor((y[i] - y0) / dy);
        if (cx < 0) cx = 0;
        if (cx > gw - 1) cx = gw - 1;
        if (cy < 0) cy = 0;
        if (cy > gh - 1) cy = gh - 1;
        for (int64_t t = 0; t < K; ++t) {
            outx[t * n + i] = gx[(t * gh + cy) * gw + cx];
            outy[t * n + i] = gy[(t * gh + cy) * gw + cx];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Input encoders (Sec. "Simulation framework": sinusoidal, sawtooth and      */
/* rotational fields)                                                         */
/* ------------------------------------------------------------------------ */

/* Each input value u_k (k < m) becomes one period of `period` field values with
 * amplitude A_k = h_lo + (h_hi - h_lo) u_k:
 *   kind 0, sinusoid:  A_k sin(2 pi j / period) along the angle `angle_deg`;
 *   kind 1, sawtooth:  A_k (2 j / (period - 1) - 1) along the angle, a linear rise
 *                      from -A_k to +A_k;
 *   kind 2, rotation:  magnitude A_k at the angle angle_deg + 360 j / period;
 * for j = 0 .. period - 1, written to hx, hy[k period + j]. Angles in degrees,
 * converted as (deg pi) / 180. Returns m period, or -1 on bad arguments. */
int64_t or_encode(int kind, int64_t m, const double* u, int32_t period, double h_lo, double h_hi,
                  double angle_deg, double* hx, double* hy) {
    if (m < 0 || period < 1 || (kind == 1 && period < 2) || kind < 0 || kind > 2) return -1;
    const double phi = (angle_deg * M_PI) / 180.0;
    for (int64_t k = 0; k < m; ++k) {
        const double A = h_lo + (h_hi - h_lo) * u[k];
        for (int32_t j = 0; j < period; ++j) {
            double h = 0.0, ang = phi;
            if (kind == 0) {
                h = A * sin((2.0 * M_PI * (double)j) / (double)period);
            } else if (kind == 1) {
                h = A * ((2.0 * (double)j) / (double)(period - 1) - 1.0);
            } else {
                h = A;
                ang = ((angle_deg + (360.0 * (double)j) / (double)period) * M_PI) / 180.0;
            }
            hx[k * period + j] = h * cos(ang);
            hy[k * period + j] = h * sin(ang);
        }
    }
    return m * period;
}

/* ------------------------------------------------------------------------ */
/* Spin-spin correlation against separation (Sec. "Domain size in square ASI") */
/* ------------------------------------------------------------------------ */

/* The correlation of two spins is +1 when their dipolar interaction is at its
 * minimum and -1 at its maximum. The pair energy of islands i, j is
 * -alpha s_i s_j v_ij / r^3 with v_ij = 3 (mhat_i . rhat)(mhat_j . rhat) - mhat_i . mhat_j
 * (Eq. 3), so the correlation is sign(s_i s_j v_ij). For every unordered pair
 * i < j with |r_ij|^2 <= rmax^2 (1 + 1e-9) it goes to bin floor(|r_ij| / w + 1e-7)
 * (the small offset keeps separations that are whole multiples of w, up to
 * rounding, in the upper bin); pairs with |v_ij| <= 1e-9 (no preferred relative
 * orientation) and bins >= nbins are left out. count[b] receives the pairs of bin
 * b and sum[b] the sum of their correlations: the mean is sum / count. */
void or_correlation(int64_t n, const double* x, const double* y, const double* theta,
                    const int8_t* s, double rmax, double w, int32_t nbins, int64_t* count,
                    int64_t* sum) {
    for (int32_t b = 0; b < nbins; ++b) {
        count[b] = 0;
        sum[b] = 0;
    }
    const double r2max = rmax * rmax * (1.0 + 1e-9);
    for (int64_t i = 0; i < n; ++i) {
        const double mix = cos(theta[i]), miy = sin(theta[i]);
        for (int64_t j = i + 1; j < n; ++j) {
            const double rx = x[i] - x[j], ry = y[i] - y[j];
            const double r2 = rx * rx + ry * ry;
            if (r2 > r2max) continue;
            const double r = sqrt(r2);
            const int64_t b = (int64_t)floor(r / w + 1e-7);
            if (b >= nbins) continue;
            const double mjx = cos(theta[j]), mjy = sin(theta[j]);
            const double ui = (mix * rx + miy * ry) / r, uj = (mjx * rx + mjy * ry) / r;
            const double v = 3.0 * ui * uj - (mix * mjx + miy * mjy);
            if (fabs(v) <= 1e-9) continue;
            const int sv = v > 0.0 ? 1 : -1;
            count[b] += 1;
            sum[b] += (int64_t)s[i] * (int64_t)s[j] * sv;
        }
    }
}
