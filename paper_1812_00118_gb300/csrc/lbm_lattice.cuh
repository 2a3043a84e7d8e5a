// Velocity sets of the GPU library (Section 2: D2Q9 / D3Q19, T = 1/3).
//
// Internal axes: populations are stored on an (NX, NY, NZ) grid, x fastest,
// and every step kernel marches along z.  A D2Q9 grid of user size (nx, ny)
// is stored as (nx, 1, ny): its velocities lie in the internal x-z plane, so
// the 2-D and 3-D paths are the same kernel with a one-plane-deep y axis.
// Opposite velocities are adjacent: c[2k] = -c[2k-1] for k >= 1.
#pragma once

namespace lbm {

constexpr double kT = 1.0 / 3.0;

template <int LAT>
struct Lattice;

template <>
struct Lattice<0> {   // D2Q9 in the internal x-z plane
    static constexpr int Q = 9;
    static constexpr bool kHasY = false;
    static constexpr int cx[Q] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    static constexpr int cy[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    static constexpr int cz[Q] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    static constexpr double w[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                                    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

template <>
struct Lattice<1> {   // D3Q19
    static constexpr int Q = 19;
    static constexpr bool kHasY = true;
    static constexpr int cx[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    static constexpr int cy[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    static constexpr int cz[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    static constexpr double w[Q] = {1.0 / 3,
                                    1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

}  // namespace lbm
