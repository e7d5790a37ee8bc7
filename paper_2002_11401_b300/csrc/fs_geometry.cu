// fs_geometry.cpp - host-side generators: island arrays (Sec. "Geometries") and
// coercive-field disorder (Sec. "Imperfections and disorder").
#include "fs_host.h"

#include <algorithm>
#include <cmath>
#include <tuple>

#include "fs_common.cuh"

namespace fs {

namespace {

struct Site {
    int64_t X, Y;  // integer lattice coordinates
    int deg;       // island angle in degrees
};

}  // namespace

// Square / pinwheel: centres on a half-spacing grid, (X, Y) -> (X/2, Y/2) * a.
// Horizontal islands at odd X, even Y (x < nx, y <= ny); vertical islands at even
// X, odd Y (x <= nx, y < ny): closed edges. Pinwheel turns each island by 45
// degrees about its centre.
// Kagome: flat-top hexagons of edge a, hexagon (c, r) centred at
// (1.5 c, sqrt(3) r + (c odd) sqrt(3)/2); islands on the six edge midpoints, along
// the edges; integer coordinates in units of (a/4, a sqrt(3)/4); shared edges
// appear once.
// Edge forms of the square lattice (the figure of the geometries names them; these
// are the readings): open edges drop the closed square's boundary islands
// (horizontal rows y = 0 and y = ny, vertical columns x = 0 and x = nx); the
// pinwheel "diamond" keeps one horizontal and one vertical island per unit cell
// (rows y < ny, columns x < nx: 2 nx ny islands); "lucky-knot" is the open square
// turned 45 degrees. Ising: one island at every lattice point, all at 0 degrees.
// Order: ascending Y, then ascending X (ascending y, then x).
bool make_geometry(int kind, int32_t nx, int32_t ny, double a, Geometry& g) {
    if (nx <= 0 || ny <= 0 || !(a > 0.0)) return false;
    std::vector<Site> s;
    double ux, uy;
    if (kind == 0 || kind == 1 || (kind >= 3 && kind <= 5)) {
        const int rot = (kind == 1 || kind == 4 || kind == 5) ? 45 : 0;
        // rows of horizontal islands [h_lo, h_hi] and columns of vertical ones [v_lo, v_hi]
        int64_t h_lo = 0, h_hi = ny, v_lo = 0, v_hi = nx;
        if (kind == 3 || kind == 5) {
            h_lo = 1;
            h_hi = ny - 1;
            v_lo = 1;
            v_hi = nx - 1;
        } else if (kind == 4) {
            h_hi = ny - 1;
            v_hi = nx - 1;
        }
        s.reserve((size_t)nx * (ny + 1) + (size_t)ny * (nx + 1));
        for (int64_t y = h_lo; y <= h_hi; ++y)
            for (int64_t x = 0; x < nx; ++x) s.push_back({2 * x + 1, 2 * y, rot});
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = v_lo; x <= v_hi; ++x) s.push_back({2 * x, 2 * y + 1, 90 + rot});
        ux = 0.5;
        uy = 0.5;
    } else if (kind == 6) {
        s.reserve((size_t)nx * ny);
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) s.push_back({x, y, 0});
        ux = 1.0;
        uy = 1.0;
    } else if (kind == 2) {
        // midpoint of edge k (direction 30 + 60k degrees) and the island's angle
        const int ox[6] = {3, 0, -3, -3, 0, 3};
        const int oy[6] = {1, 2, 1, -1, -2, -1};
        s.reserve((size_t)6 * nx * ny);
        for (int64_t c = 0; c < nx; ++c)
            for (int64_t r = 0; r < ny; ++r)
                for (int k = 0; k < 6; ++k)
                    s.push_back({6 * c + ox[k], 4 * r + ((c & 1) ? 2 : 0) + oy[k],
                                 (120 + 60 * k) % 180});
        ux = 0.25;
        uy = std::sqrt(3.0) / 4.0;
    } else {
        return false;
    }
    std::sort(s.begin(), s.end(), [](const Site& p, const Site& q) {
        return std::tie(p.Y, p.X) < std::tie(q.Y, q.X);
    });
    s.erase(std::unique(s.begin(), s.end(),
                        [](const Site& p, const Site& q) { return p.X == q.X && p.Y == q.Y; }),
            s.end());
    const size_t n = s.size();
    if (n == 0) return false;
    g.x.resize(n);
    g.y.resize(n);
    g.theta.resize(n);
    for (size_t i = 0; i < n; ++i) {
        g.x[i] = ((double)s[i].X * ux) * a;
        g.y[i] = ((double)s[i].Y * uy) * a;
        g.theta[i] = ((double)s[i].deg * M_PI) / 180.0;
    }
    return true;
}

// h_k^(i) = h_k (1 + k_disorder z), z the first Box-Muller normal of Philox block
// (i, r, instance, 0), r = 0, 1, ... until the value is positive.
void draw_hk(int64_t n, double hk, double kdis, uint64_t seed, uint32_t instance,
             std::vector<double>& out) {
    out.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double v = 0.0;
        for (uint32_t r = 0;; ++r) {
            uint32_t c[4] = {(uint32_t)i, r, instance, 0u};
            philox10(c, seed);
            const double u1 = ((double)u53(c[0], c[1]) + 0.5) * 0x1.0p-53;
            const double u2 = ((double)u53(c[2], c[3]) + 0.5) * 0x1.0p-53;
            const double z0 = std::sqrt(-2.0 * std::log(u1)) * std::cos((2.0 * M_PI) * u2);
            v = hk * (1.0 + kdis * z0);
            if (v > 0.0) break;
        }
        out[(size_t)i] = v;
    }
}

}  // namespace fs
