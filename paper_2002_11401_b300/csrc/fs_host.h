// fs_host.h - host-side helpers shared by the C ABI implementation.
#pragma once

#include <stdint.h>

#include <vector>

namespace fs {

struct Geometry {
    std::vector<double> x, y, theta;
};

bool make_geometry(int kind, int32_t nx, int32_t ny, double a, Geometry& g);
void draw_hk(int64_t n, double hk, double kdis, uint64_t seed, uint32_t instance,
             std::vector<double>& out);

}  // namespace fs
