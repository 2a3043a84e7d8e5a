// Velocity sets of the GPU library (Section 2: D2Q9 / D3Q19, T = 1/3).
//
// Internal axes: populations are stored on an (NX, NY, NZ) grid, x fastest,
// and every step kernel marches along z.  A D2Q9 grid of user size (nx, ny)
// is stored as (nx, 1, ny): its velocities lie in the internal x-z plane, so
// the 2-D and 3-D paths are the same kernel with a one-plane-deep y axis.
//
// Order: velocities with the same (c_y, c_z) are consecutive, c_x = 0, +1, -1
// within a group.  A pull of a whole group reads the same rows and plane,
// shifted only in x, so one bulk tensor copy fetches a group (groups[]:
// first index, size, c_y, c_z).
#pragma once

namespace lbm {

constexpr double kT = 1.0 / 3.0;

template <int LAT>
struct Lattice;

template <>
struct Lattice<0> {   // D2Q9 in the internal x-z plane
    static constexpr int Q = 9;
    static constexpr bool kHasY = false;
    static constexpr int cx[Q] = {0, 1, -1, 0, 1, -1, 0, 1, -1};
    static constexpr int cy[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    static constexpr int cz[Q] = {0, 0, 0, 1, 1, 1, -1, -1, -1};
    static constexpr double w[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36,
                                    1.0 / 9, 1.0 / 36, 1.0 / 36};
    static constexpr int op[Q] = {0, 2, 1, 6, 8, 7, 3, 5, 4};
    static constexpr int NG = 3;
    static constexpr int groups[NG][4] = {{0, 3, 0, 0}, {3, 3, 0, 1}, {6, 3, 0, -1}};
    __host__ __device__ static constexpr int opp(int i) { return op[i]; }
};

template <>
struct Lattice<1> {   // D3Q19
    static constexpr int Q = 19;
    static constexpr bool kHasY = true;
    static constexpr int cx[Q] = {0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 0, 0, 0};
    static constexpr int cy[Q] = {0, 0, 0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1};
    static constexpr int cz[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, -1, -1, -1, 1, -1, -1, 1};
    static constexpr double w[Q] = {1.0 / 3,
                                    1.0 / 18, 1.0 / 18,
                                    1.0 / 18, 1.0 / 36, 1.0 / 36,
                                    1.0 / 18, 1.0 / 36, 1.0 / 36,
                                    1.0 / 18, 1.0 / 36, 1.0 / 36,
                                    1.0 / 18, 1.0 / 36, 1.0 / 36,
                                    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    static constexpr int op[Q] = {0, 2, 1, 6, 8, 7, 3, 5, 4, 12, 14, 13, 9, 11, 10, 16, 15, 18, 17};
    static constexpr int NG = 9;
    static constexpr int groups[NG][4] = {{0, 3, 0, 0},  {3, 3, 1, 0},   {6, 3, -1, 0},
                                          {9, 3, 0, 1},  {12, 3, 0, -1}, {15, 1, 1, 1},
                                          {16, 1, -1, -1}, {17, 1, 1, -1}, {18, 1, -1, 1}};
    __host__ __device__ static constexpr int opp(int i) { return op[i]; }
};

}  // namespace lbm
