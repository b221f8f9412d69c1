// D3Q19 velocity set of the library (Sec. II.A of the paper: D3Q19, c_s^2 = 1/3).
// Order: rest, +-x, +-y, +-z, then the 12 edge diagonals in opposite pairs;
// this is the population order documented in include/stg_lbm.h.  Written as
// constexpr functions so that fully unrolled loops over i fold to constants.
#pragma once

namespace stg {

__host__ __device__ constexpr int cx_of(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz_of(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
// opposite direction: pairs (1,2), (3,4), ..., (17,18)
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// weights: 1/3 rest, 1/18 axis, 1/36 edge
__host__ __device__ constexpr float w_of(int i) { return i == 0 ? (1.0f / 3.0f) : (i <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }
__host__ __device__ constexpr double w_of_d(int i) { return i == 0 ? (1.0 / 3.0) : (i <= 6 ? (1.0 / 18.0) : (1.0 / 36.0)); }

constexpr int Q = 19;

}  // namespace stg
