// adjoint_tiled.cuh -- tiled reverse step for domains stored with interleaved
// row halves (nx % 4 == 0).  Same arithmetic as adjoint.cu:
//   L_r(x) = lam_rho'(x) - lam_u'(x) . (u'(x) - force) / rho'(x),  L_m(x) = lam_u'(x) / rho'(x),
//   g_a(x) = L_r(x) + c_a . L_m(x),
//   G0(y) = sum_a w_a g_a(y + c_a), G1 = sum_a w_a c_a g_a(y + c_a), G2 = sum_a w_a c_a c_a^T g_a(y + c_a),
//   lam_rho(y) = G0 (1 - 3/2 u.u) + 3 u.G1 + 9/2 u^T G2 u,
//   lam_u(y)   = rho (3 G1 + 9 G2 u - 3 u G0),
// plus lam' passed through at wall nodes.
//
// One launch.  Blocks span the x extent and TY rows (+ a halo row on each
// side) and march the slowest axis.  Every thread forms (L_r, L_m) of its own
// quad (4 stored nodes = node pairs a, b) on paired FP32 lanes from the
// post-step state and lam', and writes them into a ring of four staged planes
// in shared memory; the destination pairs then pull their 19 neighbours'
// records from the three planes around them and accumulate the moments with
// the integer weights w36 (divided out at the end).  The loads of plane q + 2
// are issued before the gather of plane q and staged after it, so one barrier
// per plane suffices.
//
// Shared layout: [stage][row][pair][unit][column] of 16-byte units, a unit
// holding two components (FP32) or one (FP64) of a pair's record, so that the
// threads of a warp read consecutive units.  Across the seam between the two
// half rows the lanes swap: the end threads of each row also write a
// lane-swapped copy of their edge pair into two extra columns.
#pragma once
#include "step_tiled.cuh"

namespace maclab {

struct AdjArgs {
  int nx, ny, nplanes;   // ny = 1 in 2D
  int64_t n;             // nodes
  int64_t plane_stride;  // nx * ny
  int ty, nzc;
  int px, py, pz;
  int wall_mode;
  const uint8_t* mask;
  double force[3];
  int overlap;           // host side: launch with programmatic dependent launch
};

// a - b as fma(b, -1, a): the same correctly rounded difference, written
// without inline assembly so the compiler schedules it freely
template <typename C>
__device__ __forceinline__ typename Pair<C>::P adj_sub(typename Pair<C>::P a, typename Pair<C>::P b) {
  return Pair<C>::fma(b, Pair<C>::splat(C(-1)), a);
}

// 16-byte unit <-> lane pairs
template <typename P>
struct AdjUnit;
template <>
struct AdjUnit<float2> {
  static constexpr int G = 2;
  __device__ __forceinline__ static void st(uint4* u, const float2* v) {
    *reinterpret_cast<float4*>(u) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  }
  __device__ __forceinline__ static void st_swapped(uint4* u, const float2* v) {
    *reinterpret_cast<float4*>(u) = make_float4(v[0].y, v[0].x, v[1].y, v[1].x);
  }
  __device__ __forceinline__ static void ld(const uint4* u, float2* v) {
    const float4 t = *reinterpret_cast<const float4*>(u);
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
  }
};
template <>
struct AdjUnit<double2> {
  static constexpr int G = 1;
  __device__ __forceinline__ static void st(uint4* u, const double2* v) { *reinterpret_cast<double2*>(u) = v[0]; }
  __device__ __forceinline__ static void st_swapped(uint4* u, const double2* v) {
    *reinterpret_cast<double2*>(u) = make_double2(v[0].y, v[0].x);
  }
  __device__ __forceinline__ static void ld(const uint4* u, double2* v) { v[0] = *reinterpret_cast<const double2*>(u); }
};

template <int LAT, typename S, int BXC, int RY>
struct AdjTile {
  using C = typename Store<S>::C;
  using P = typename Pair<C>::P;
  static constexpr int D = Lattice<LAT>::D;
  static constexpr int K = D + 1;                 // record components: L_r, L_m
  static constexpr int G = AdjUnit<P>::G;         // components per unit
  static constexpr int NU = (K + G - 1) / G;      // units per pair record
  static constexpr int W = BXC + 2;               // columns, with the two seam copies
  static constexpr int SEAM_L = BXC, SEAM_R = BXC + 1;
  static constexpr int STAGES = 4;
  static constexpr int STAGE = RY * 2 * NU * W;   // units per stage
  static constexpr int THREADS = BXC * RY;
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 2 : 1;
  __host__ __device__ static constexpr size_t smem_bytes() { return (size_t)16 * STAGES * STAGE; }
  __device__ __forceinline__ static constexpr int unit(int k, int rr, int pr, int u, int col) {
    return (((k * RY + rr) * 2 + pr) * NU + u) * W + col;
  }
};

template <int LAT, typename S, int BXC, int RY>
__global__ void __launch_bounds__(BXC * RY, (AdjTile<LAT, S, BXC, RY>::MIN_BLOCKS))
    adj_step_tiled(AdjArgs A, const S* __restrict__ in_state, const S* __restrict__ out_state,
                   const typename Store<S>::C* __restrict__ lam1, typename Store<S>::C* __restrict__ lam0,
                   double* __restrict__ grad_force) {
  using T = AdjTile<LAT, S, BXC, RY>;
  using C = typename T::C;
  using O = Pair<C>;
  using P = typename O::P;
  using U = AdjUnit<P>;
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  constexpr int D = T::D, K = T::K, G = T::G, NU = T::NU;
  extern __shared__ __align__(16) uint4 units[];
  pdl_wait();  // the previous kernel's writes are visible from here on
  pdl_launch_next();
  const int tx = threadIdx.x, r = threadIdx.y;
  const int bxr = A.nx >> 2;
  const bool active = tx < bxr;

  int row = 0, row_mem = 0;
  bool row_exists = true, interior = true;
  if (D == 3) {
    row = blockIdx.y * A.ty + r - 1;
    interior = r >= 1 && r <= RY - 2 && row < A.ny;
    row_mem = row;
    if (row < 0 || row >= A.ny) {
      if (A.py) row_mem = (row + A.ny) % A.ny;
      else row_exists = false;
    }
  }
  interior = interior && active;
  const bool stages_own = active && row_exists;
  const int64_t row_off = (int64_t)row_mem * A.nx + 4 * tx;  // storage index of the quad in a plane

  const int z0 = (int)(((int64_t)blockIdx.x * A.nplanes) / A.nzc);
  const int z1 = (int)(((int64_t)(blockIdx.x + 1) * A.nplanes) / A.nzc);
  auto plane_exists = [&](int p) { return (p >= 0 && p < A.nplanes) || A.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + A.nplanes : (p >= A.nplanes ? p - A.nplanes : p); };

  // wall lanes (a.x, a.y, b.x, b.y) as bits 0..3; box walls off the march axis are fixed per thread
  uint32_t box_bits = 0;
  if (A.wall_mode == kWallBox) {
    if (!A.px) box_bits |= (tx == 0 ? 1u : 0u) | (tx == bxr - 1 ? 8u : 0u);
    if (D == 3 && !A.py && (row_mem == 0 || row_mem == A.ny - 1)) box_bits = 15u;
  }

  P force[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) force[i] = O::splat(C(A.force[i]));
  C gfp[3] = {C(0), C(0), C(0)};
  double gfd[3] = {0.0, 0.0, 0.0};

  // post-step state and lam' of this thread's quad in one plane
  struct Raw {
    P st[K][2], lm[K][2];
    uint32_t wall;
    bool have;
  };
  auto load_raw = [&](int p, Raw& R) {
    R.have = stages_own && plane_exists(p);
    R.wall = 0;
    if (R.have) {
      const int pm = plane_mem(p);
      const int64_t off = (int64_t)pm * A.plane_stride + row_off;
#pragma unroll
      for (int f = 0; f < K; ++f) {
        Quad<S>::ld(out_state + f * A.n + off, R.st[f][0], R.st[f][1]);
        Quad<C>::ld(lam1 + f * A.n + off, R.lm[f][0], R.lm[f][1]);
      }
      if (A.wall_mode == kWallMask) {
        const uchar4 mk = *reinterpret_cast<const uchar4*>(A.mask + off);
        R.wall = (mk.x ? 1u : 0u) | (mk.y ? 2u : 0u) | (mk.z ? 4u : 0u) | (mk.w ? 8u : 0u);
      } else if (A.wall_mode == kWallBox) {
        R.wall = (!A.pz && (pm == 0 || pm == A.nplanes - 1)) ? 15u : box_bits;
      }
    }
  };

  uint32_t wq = 0;  // wall bits of the last three staged planes, newest in bits 0..3
  // records of plane p into stage p & 3 (zeros where the row or plane is absent)
  auto stage = [&](int p, const Raw& R) {
    wq = (wq << 4) | R.wall;
    if (!active) return;
    const int k = p & (T::STAGES - 1);
    P rec[2][NU * G];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int c = 0; c < NU * G; ++c) rec[q][c] = O::splat(C(0));
    if (R.have) {
      const bool counted = interior && p >= z0 && p < z1 && grad_force;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const P inv = O::rcp(O::add(O::splat(C(1)), R.st[0][q]));
        P lr = R.lm[0][q];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const P um = adj_sub<C>(R.st[1 + i][q], force[i]);  // m' / rho'
          lr = adj_sub<C>(lr, O::mul(O::mul(R.lm[1 + i][q], um), inv));
          rec[q][1 + i] = O::mul(R.lm[1 + i][q], inv);
        }
        rec[q][0] = lr;
        const bool w0 = (R.wall >> (2 * q)) & 1u, w1 = (R.wall >> (2 * q + 1)) & 1u;
#pragma unroll
        for (int c = 0; c < K; ++c) {  // walls carry no (L_r, L_m)
          if (w0) rec[q][c].x = C(0);
          if (w1) rec[q][c].y = C(0);
        }
        if (counted)
#pragma unroll
          for (int i = 0; i < D; ++i)
            gfp[i] += (w0 ? C(0) : R.lm[1 + i][q].x) + (w1 ? C(0) : R.lm[1 + i][q].y);
      }
      if (counted && ((p - z0) & 7) == 7)
#pragma unroll
        for (int i = 0; i < D; ++i) {
          gfd[i] += (double)gfp[i];
          gfp[i] = C(0);
        }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int u = 0; u < NU; ++u) U::st(&units[T::unit(k, r, q, u, tx)], &rec[q][u * G]);
    if (tx == bxr - 1)  // swapped pair b: left neighbour of thread 0's pair a
#pragma unroll
      for (int u = 0; u < NU; ++u) U::st_swapped(&units[T::unit(k, r, 1, u, T::SEAM_L)], &rec[1][u * G]);
    if (tx == 0)        // swapped pair a: right neighbour of the last thread's pair b
#pragma unroll
      for (int u = 0; u < NU; ++u) U::st_swapped(&units[T::unit(k, r, 0, u, T::SEAM_R)], &rec[0][u * G]);
  };

  const int col_l = tx == 0 ? T::SEAM_L : tx - 1;
  const int col_r = tx == bxr - 1 ? T::SEAM_R : tx + 1;

  {
    Raw R0, R1;
    load_raw(z0 - 1, R0);
    load_raw(z0, R1);
    stage(z0 - 1, R0);
    load_raw(z0 + 1, R0);
    stage(z0, R1);
    stage(z0 + 1, R0);
  }
  Raw R;
  for (int q = z0; q < z1; ++q) {
    const bool next = q + 2 <= z1;
    if (next) load_raw(q + 2, R);
    const int64_t off = (int64_t)q * A.plane_stride + row_off;
    const uint32_t wd = (wq >> 4) & 15u;  // wall lanes of plane q
    P st[K][2], l1[K][2];
    if (interior) {
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<S>::ld(in_state + f * A.n + off, st[f][0], st[f][1]);
      if (wd)
#pragma unroll
        for (int f = 0; f < K; ++f) Quad<C>::ld(lam1 + f * A.n + off, l1[f][0], l1[f][1]);
    }
    __syncthreads();  // stages of planes q - 1, q, q + 1 are complete
    if (interior) {
      P res[K][2];
#pragma unroll
      for (int qp = 0; qp < 2; ++qp) {
        P G0 = O::splat(C(0)), G1[3], G2[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          G1[i] = O::splat(C(0));
#pragma unroll
          for (int j = 0; j < 3; ++j) G2[i][j] = O::splat(C(0));
        }
        static_for<0, L::Q>([&](auto Ia) {
          constexpr int a = decltype(Ia)::value;
          constexpr int cx = F::fx(a), cy = F::fy(a), cz = F::fz(a);
          // neighbour y + c_a: stage of plane q + cz, row r + cy, column and pair by cx
          const int k = (q + cz) & (T::STAGES - 1);
          const int rr = r + cy;
          int col, pr;
          if constexpr (cx == 0) { col = tx; pr = qp; }
          else if constexpr (cx == 1) { if (qp == 0) { col = tx; pr = 1; } else { col = col_r; pr = 0; } }
          else { if (qp == 1) { col = tx; pr = 0; } else { col = col_l; pr = 1; } }
          P v[NU * G];
#pragma unroll
          for (int u = 0; u < NU; ++u) U::ld(&units[T::unit(k, rr, pr, u, col)], &v[u * G]);
          P g = v[0];
          static_for<0, D>([&](auto Ii) {
            constexpr int i = decltype(Ii)::value;
            constexpr int c = L::c(a, i);
            if constexpr (c == 1) g = O::add(g, v[1 + i]);
            else if constexpr (c == -1) g = adj_sub<C>(g, v[1 + i]);
          });
          constexpr int w = L::w36(a);
          const P wg = w == 1 ? g : O::mul(g, O::splat(C(w)));
          G0 = O::add(G0, wg);
          static_for<0, D>([&](auto Ii) {
            constexpr int i = decltype(Ii)::value;
            constexpr int ci = L::c(a, i);
            if constexpr (ci != 0) {
              G1[i] = ci > 0 ? O::add(G1[i], wg) : adj_sub<C>(G1[i], wg);
              G2[i][i] = O::add(G2[i][i], wg);
              static_for<i + 1, D>([&](auto Ij) {
                constexpr int j = decltype(Ij)::value;
                constexpr int cj = L::c(a, j);
                if constexpr (cj != 0) G2[i][j] = ci * cj > 0 ? O::add(G2[i][j], wg) : adj_sub<C>(G2[i][j], wg);
              });
            }
          });
        });
        // equilibrium Jacobian at the destination (its own state)
        const P rho = O::add(O::splat(C(1)), st[0][qp]);
        P u[3], G2u[3];
        P uu = O::splat(C(0)), uG1 = O::splat(C(0)), uG2u = O::splat(C(0));
#pragma unroll
        for (int i = 0; i < D; ++i) {
          u[i] = st[1 + i][qp];
          uu = O::fma(u[i], u[i], uu);
          uG1 = O::fma(u[i], G1[i], uG1);
        }
#pragma unroll
        for (int i = 0; i < D; ++i) {
          G2u[i] = O::splat(C(0));
#pragma unroll
          for (int j = 0; j < D; ++j) G2u[i] = O::fma(i <= j ? G2[i][j] : G2[j][i], u[j], G2u[i]);
          uG2u = O::fma(u[i], G2u[i], uG2u);
        }
        // sums carry the factor 36 of the integer weights
        const P k36 = O::splat(C(1.0 / 36.0));
        P lr = O::fma(O::fma(uu, O::splat(C(-1.5)), O::splat(C(1))), G0,
                      O::fma(uG1, O::splat(C(3)), O::mul(uG2u, O::splat(C(4.5)))));
        res[0][qp] = O::mul(lr, k36);
        const P rk = O::mul(rho, k36);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          P t = O::fma(G2u[i], O::splat(C(9)), O::mul(G1[i], O::splat(C(3))));
          t = adj_sub<C>(t, O::mul(O::mul(u[i], G0), O::splat(C(3))));
          res[1 + i][qp] = O::mul(rk, t);
        }
      }
      if (wd) {  // a wall node's output is its input: pass lam' through
#pragma unroll
        for (int f = 0; f < K; ++f) {
          if (wd & 1u) res[f][0].x += l1[f][0].x;
          if (wd & 2u) res[f][0].y += l1[f][0].y;
          if (wd & 4u) res[f][1].x += l1[f][1].x;
          if (wd & 8u) res[f][1].y += l1[f][1].y;
        }
      }
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<C>::st(lam0 + f * A.n + off, res[f][0], res[f][1]);
    }
    if (next) stage(q + 2, R);  // stage (q + 2) & 3 was last read in the gather of plane q - 1
  }

  if (grad_force) {
    // block sum of the force gradient: warp shuffles, then one value per warp
    __shared__ double red[3][32];
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double v = gfd[i] + (double)gfp[i];
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) v += __shfl_down_sync(0xffffffffu, v, s);
      if (lane == 0) red[i][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0)
      for (int i = 0; i < D; ++i) {
        double s = 0.0;
        for (int w = 0; w < nwarps; ++w) s += red[i][w];
        atomicAdd(grad_force + i, s);
      }
  }
}

// Launch helper (instantiated in adjoint_tiled.cu).  Returns the number of
// blocks of this shape one SM holds through *resident.
template <int LAT, typename S, int BXC, int RY>
cudaError_t launch_adj_tiled(const AdjArgs& A, const void* in_state, const void* out_state,
                             const void* lam1, void* lam0, double* grad_force, cudaStream_t st,
                             int ytiles, int* resident_out) {
  using T = AdjTile<LAT, S, BXC, RY>;
  using C = typename T::C;
  auto kern = adj_step_tiled<LAT, S, BXC, RY>;
  constexpr size_t smem = T::smem_bytes();
  static int resident_dev[64] = {};  // per instantiation and device
  int dev = 0;
  cudaError_t e0 = cudaGetDevice(&dev);
  if (e0 != cudaSuccess) return e0;
  int& resident = resident_dev[dev & 63];
  if (!resident) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, T::THREADS, smem);
    if (e != cudaSuccess) return e;
    resident = nb < 1 ? 1 : nb;
  }
  if (resident_out) {  // sizing query only
    *resident_out = resident;
    return cudaSuccess;
  }
  return launch_kernel(kern, dim3(A.nzc, ytiles), dim3(BXC, RY), smem, st, A.overlap, A,
                       static_cast<const S*>(in_state), static_cast<const S*>(out_state),
                       static_cast<const C*>(lam1), static_cast<C*>(lam0), grad_force);
}

}  // namespace maclab
