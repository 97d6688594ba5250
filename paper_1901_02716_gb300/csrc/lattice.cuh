// lattice.cuh -- D2Q9 and D3Q19 velocity sets and weights for the CUDA kernels.
//
// Velocities in lattice units c_a = e_a / e, in the order the paper lists them
// (D2Q9 after Eq. (1), D3Q19 with the description of the five simulations);
// weights as given after Eq. (2) and with the D3Q19 list.  Every accessor is
// constexpr so that, inside fully unrolled direction loops, each c_a and w_a
// is an immediate.
#pragma once

namespace maclab {

enum : int { kD2Q9 = 0, kD3Q19 = 1 };

template <int LAT>
struct Lattice;

template <>
struct Lattice<kD2Q9> {
  static constexpr int D = 2;
  static constexpr int Q = 9;
  __host__ __device__ static constexpr int c(int a, int i) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},   {0, 1, 0},  {-1, 0, 0}, {0, -1, 0},
                             {1, 1, 0},  {-1, 1, 0},  {-1, -1, 0}, {1, -1, 0}};
    return t[a][i];
  }
  // weight in units of 1/36
  __host__ __device__ static constexpr int w36(int a) { return a == 0 ? 16 : (a <= 4 ? 4 : 1); }
};

template <>
struct Lattice<kD3Q19> {
  static constexpr int D = 3;
  static constexpr int Q = 19;
  __host__ __device__ static constexpr int c(int a, int i) {
    constexpr int t[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                              {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {-1, 1, 0},
                              {1, -1, 0}, {0, 1, 1},   {0, -1, -1}, {0, -1, 1}, {0, 1, -1},
                              {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1}, {1, 0, -1}};
    return t[a][i];
  }
  __host__ __device__ static constexpr int w36(int a) { return a == 0 ? 12 : (a <= 6 ? 2 : 1); }
};

}  // namespace maclab
