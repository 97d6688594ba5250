// adjoint_tiled.cuh -- tiled reverse step for domains stored with interleaved
// row halves (nx % 4 == 0).  Same arithmetic as adjoint.cu:
//   L_r(x) = lam_rho'(x) - lam_u'(x) . (u'(x) - force) / rho'(x),  L_m(x) = lam_u'(x) / rho'(x),
//   g_a(x) = L_r(x) + c_a . L_m(x),
//   G0(y) = sum_a w_a g_a(y + c_a), G1 = sum_a w_a c_a g_a(y + c_a), G2 = sum_a w_a c_a c_a^T g_a(y + c_a),
//   lam_rho(y) = G0 (1 - 3/2 u.u) + 3 u.G1 + 9/2 u^T G2 u,
//   lam_u(y)   = rho (3 G1 + 9 G2 u - 3 u G0),
// plus lam' passed through at wall nodes.
//
//  * adj_records: one thread per quad (4 stored nodes = node pairs a, b) forms
//    (L_r, L_m) on paired FP32 lanes and writes them pair-major: per quad,
//    pair a's (L_r, L_mx, L_my, L_mz) as four lane pairs, then pair b's
//    (64 bytes in FP32).
//  * adj_gather_tiled: blocks span the x extent and TY rows (+ a halo row on
//    each side) and march the slowest axis; the records of three planes are
//    staged in shared memory with per-thread cp.async copies (one barrier per
//    plane); each destination pair pulls its 19 neighbours' records (two
//    16-byte loads each) and accumulates the moments on lane pairs with the
//    integer weights w36 (divided out at the end).  Across the seam between
//    the two half rows the lanes swap: the end threads of each row stage a
//    lane-swapped copy of their edge pair in two extra columns.
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
};

// ------------------------------------------------------------------ records

template <int LAT, typename S>
__global__ void __launch_bounds__(256) adj_records(AdjArgs A, const S* __restrict__ out_state,
                                                   const typename Store<S>::C* __restrict__ lam1,
                                                   typename Store<S>::C* __restrict__ rec,
                                                   double* __restrict__ grad_force) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int D = Lattice<LAT>::D;
  const int64_t nquads = A.n >> 2;
  double gf[3] = {0.0, 0.0, 0.0};
  P force[3];
  for (int i = 0; i < 3; ++i) force[i] = O::splat(C(A.force[i]));
  for (int64_t qd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qd < nquads;
       qd += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = qd << 2;
    // wall flags of the quad's lanes (a.x, a.y, b.x, b.y)
    bool wall[4] = {false, false, false, false};
    if (A.wall_mode == kWallMask) {
      const uchar4 mk = *reinterpret_cast<const uchar4*>(A.mask + m);
      wall[0] = mk.x != 0; wall[1] = mk.y != 0; wall[2] = mk.z != 0; wall[3] = mk.w != 0;
    } else if (A.wall_mode == kWallBox) {
      const int64_t row = m / A.nx;
      const int t = (int)(m - row * A.nx) >> 2;
      const int y = (int)(row % A.ny), z = (int)(row / A.ny);
      bool rw = false;
      if (D == 3) {
        if (!A.py) rw |= (y == 0) | (y == A.ny - 1);
        if (!A.pz) rw |= (z == 0) | (z == A.nplanes - 1);
      } else {
        if (!A.pz) rw |= (z == 0) | (z == A.nplanes - 1);  // 2D: rows along the march axis
      }
      for (int k = 0; k < 4; ++k) wall[k] = rw;
      if (!A.px) {
        wall[0] |= t == 0;                       // x = 0
        wall[3] |= t == (A.nx >> 2) - 1;         // x = nx - 1
      }
    }
    P st[D + 1][2], lm[D + 1][2];
#pragma unroll
    for (int f = 0; f <= D; ++f) {
      Quad<S>::ld(out_state + f * A.n + m, st[f][0], st[f][1]);
      Quad<C>::ld(lam1 + f * A.n + m, lm[f][0], lm[f][1]);
    }
    P out[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const P inv = O::rcp(O::add(O::splat(C(1)), st[0][q]));
      P lr = lm[0][q];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const P um = O::sub(st[1 + i][q], force[i]);           // m' / rho'
        lr = O::sub(lr, O::mul(O::mul(lm[1 + i][q], um), inv));
        out[q][1 + i] = O::mul(lm[1 + i][q], inv);
      }
      out[q][0] = lr;
      if (D == 2) out[q][3] = O::splat(C(0));
      // walls carry no (L_r, L_m)
      const bool w0 = wall[2 * q], w1 = wall[2 * q + 1];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (w0) out[q][k].x = C(0);
        if (w1) out[q][k].y = C(0);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (!w0) gf[i] += (double)lm[1 + i][q].x;
        if (!w1) gf[i] += (double)lm[1 + i][q].y;
      }
    }
    C* dst = rec + qd * 16;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 4; k += 2) Quad<C>::st(dst + q * 8 + 2 * k, out[q][k], out[q][k + 1]);
  }
  if (grad_force) {
    __shared__ double red[3][256];
    for (int i = 0; i < 3; ++i) red[i][threadIdx.x] = gf[i];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s)
        for (int i = 0; i < 3; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      for (int i = 0; i < D; ++i) atomicAdd(grad_force + i, red[i][0]);
  }
}

// ------------------------------------------------------------------ gather

// Stage layout: [kAdjStages][RY][W = BXC + 2][2 pairs][4 components] lane pairs.
constexpr int kAdjStages = 4;

template <typename C, int BXC, int RY>
__host__ __device__ constexpr size_t adj_stage_bytes() {
  return sizeof(typename Pair<C>::P) * (size_t)kAdjStages * RY * (BXC + 2) * 2 * 4;
}

template <int LAT, typename S, int BXC, int RY>
__global__ void __launch_bounds__(BXC * RY) adj_gather_tiled(AdjArgs A, const S* __restrict__ in_state,
                                                             const typename Store<S>::C* __restrict__ lam1,
                                                             const typename Store<S>::C* __restrict__ rec,
                                                             typename Store<S>::C* __restrict__ lam0) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  constexpr int D = L::D;
  constexpr int K = D + 1;
  constexpr int W = BXC + 2;
  constexpr int SEAM_L = BXC, SEAM_R = BXC + 1;
  constexpr int PAIR = 4;                 // lane pairs per node-pair record
  constexpr int COL = 2 * PAIR;           // lane pairs per column (pairs a and b)
  constexpr int ROW = W * COL;
  constexpr int STAGE = RY * ROW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  P* stg = reinterpret_cast<P*>(smem_raw);
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
  const bool stages_own = active && (D == 2 || r < RY) && row_exists;
  const int64_t row_off = (int64_t)row_mem * A.nx + 4 * tx;     // storage index of the quad
  const int64_t rec_row = (int64_t)row_mem * (A.nx >> 2) + tx;  // record (quad) index

  const int z0 = (int)(((int64_t)blockIdx.x * A.nplanes) / A.nzc);
  const int z1 = (int)(((int64_t)(blockIdx.x + 1) * A.nplanes) / A.nzc);
  auto plane_exists = [&](int p) { return (p >= 0 && p < A.nplanes) || A.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + A.nplanes : (p >= A.nplanes ? p - A.nplanes : p); };
  const int64_t rec_plane = (int64_t)(A.nx >> 2) * (D == 3 ? A.ny : 1);

  // this thread's column in stage k
  auto col_ptr = [&](int k, int rr, int col) { return stg + k * STAGE + rr * ROW + col * COL; };
  const uint32_t own_sh = (uint32_t)__cvta_generic_to_shared(col_ptr(0, r, tx));
  constexpr uint32_t kStageBytes = STAGE * sizeof(P);

  // start copying plane p into stage p & 3 (or zero it when the plane/row is absent)
  auto fetch = [&](int p) {
    const int k = p & (kAdjStages - 1);
    if (active) {
      if (stages_own && plane_exists(p)) {
        const C* src = rec + ((int64_t)plane_mem(p) * rec_plane + rec_row) * 16;
        const uint32_t sh = own_sh + k * kStageBytes;
#pragma unroll
        for (int j = 0; j < 16 * (int)sizeof(C) / 16; ++j) cp_async16(sh + 16 * j, src + j * (16 / sizeof(C)));
      } else {
        P* d = col_ptr(k, r, tx);
#pragma unroll
        for (int j = 0; j < COL; ++j) d[j] = O::splat(C(0));
      }
    }
    cp_async_commit();
  };
  // after the copies of plane p landed: lane-swapped seam copies
  auto seam = [&](int p) {
    const int k = p & (kAdjStages - 1);
    if (!active) return;
    if (tx == bxr - 1) {  // swapped pair b -> SEAM_L (left neighbour of thread 0's pair a)
      const P* s = col_ptr(k, r, tx) + PAIR;
      P* d = col_ptr(k, r, SEAM_L) + PAIR;
#pragma unroll
      for (int j = 0; j < PAIR; ++j) d[j] = O::swap(s[j]);
    }
    if (tx == 0) {        // swapped pair a -> SEAM_R (right neighbour of the last pair b)
      const P* s = col_ptr(k, r, tx);
      P* d = col_ptr(k, r, SEAM_R);
#pragma unroll
      for (int j = 0; j < PAIR; ++j) d[j] = O::swap(s[j]);
    }
  };
  const int col_l = tx == 0 ? SEAM_L : tx - 1;
  const int col_r = tx == bxr - 1 ? SEAM_R : tx + 1;

  // destination state and lam' (walls) of plane q for this quad
  const bool x_lo_wall = A.wall_mode == kWallBox && !A.px && tx == 0;
  const bool x_hi_wall = A.wall_mode == kWallBox && !A.px && tx == bxr - 1;
  const bool row_wall = D == 3 && !A.py && (row == 0 || row == A.ny - 1);

  fetch(z0 - 1);
  fetch(z0);
  for (int q = z0; q < z1; ++q) {
    fetch(q + 1);
    cp_async_wait<0>();
    seam(q - 1);
    seam(q);
    seam(q + 1);
    __syncthreads();
    if (interior) {
      const int64_t off = (int64_t)q * A.plane_stride + row_off;
      P st[K][2];
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<S>::ld(in_state + f * A.n + off, st[f][0], st[f][1]);
      bool wall[4] = {x_lo_wall, false, false, x_hi_wall};
      const bool plane_wall = !A.pz && (q == 0 || q == A.nplanes - 1);
      if (row_wall || plane_wall) wall[0] = wall[1] = wall[2] = wall[3] = true;
      if (A.wall_mode == kWallMask) {
        const uchar4 mk = *reinterpret_cast<const uchar4*>(A.mask + off);
        wall[0] = mk.x != 0; wall[1] = mk.y != 0; wall[2] = mk.z != 0; wall[3] = mk.w != 0;
      }
      const bool any_wall = wall[0] || wall[1] || wall[2] || wall[3];
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
          // neighbour y + c_a: stage of plane q + cz, row r + cy, pair by cx
          const int k = (q + cz) & (kAdjStages - 1);
          const int rr = r + cy;
          int col, pr;
          if constexpr (cx == 0) { col = tx; pr = qp; }
          else if constexpr (cx == 1) { if (qp == 0) { col = tx; pr = 1; } else { col = col_r; pr = 0; } }
          else { if (qp == 1) { col = tx; pr = 0; } else { col = col_l; pr = 1; } }
          const P* rp = col_ptr(k, rr, col) + pr * PAIR;
          P g = rp[0];
          static_for<0, D>([&](auto Ii) {
            constexpr int i = decltype(Ii)::value;
            constexpr int c = L::c(a, i);
            if constexpr (c == 1) g = O::add(g, rp[1 + i]);
            else if constexpr (c == -1) g = O::sub(g, rp[1 + i]);
          });
          constexpr int w = L::w36(a);
          const P wg = w == 1 ? g : O::mul(g, O::splat(C(w)));
          G0 = O::add(G0, wg);
          static_for<0, D>([&](auto Ii) {
            constexpr int i = decltype(Ii)::value;
            constexpr int ci = L::c(a, i);
            if constexpr (ci != 0) {
              G1[i] = ci > 0 ? O::add(G1[i], wg) : O::sub(G1[i], wg);
              G2[i][i] = O::add(G2[i][i], wg);
              static_for<i + 1, D>([&](auto Ij) {
                constexpr int j = decltype(Ij)::value;
                constexpr int cj = L::c(a, j);
                if constexpr (cj != 0) G2[i][j] = ci * cj > 0 ? O::add(G2[i][j], wg) : O::sub(G2[i][j], wg);
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
          t = O::sub(t, O::mul(O::mul(u[i], G0), O::splat(C(3))));
          res[1 + i][qp] = O::mul(rk, t);
        }
      }
      if (any_wall) {  // a wall node's output is its input: pass lam' through
        P l1[K][2];
#pragma unroll
        for (int f = 0; f < K; ++f) Quad<C>::ld(lam1 + f * A.n + off, l1[f][0], l1[f][1]);
#pragma unroll
        for (int f = 0; f < K; ++f) {
          if (wall[0]) res[f][0].x += l1[f][0].x;
          if (wall[1]) res[f][0].y += l1[f][0].y;
          if (wall[2]) res[f][1].x += l1[f][1].x;
          if (wall[3]) res[f][1].y += l1[f][1].y;
        }
      }
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<C>::st(lam0 + f * A.n + off, res[f][0], res[f][1]);
    }
    __syncthreads();  // stage of plane q - 1 is refilled by the next iteration's fetch
  }
  cp_async_wait<0>();
}

// Launch helpers (instantiated in adjoint_tiled.cu).
template <int LAT, typename S, int BXC, int RY>
cudaError_t launch_adj_gather(const AdjArgs& A, const void* in_state, const void* lam1,
                              const void* rec, void* lam0, cudaStream_t st, dim3 grid) {
  using C = typename Store<S>::C;
  auto kern = adj_gather_tiled<LAT, S, BXC, RY>;
  constexpr size_t smem = adj_stage_bytes<C, BXC, RY>();
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, dim3(BXC, RY), smem, st>>>(A, static_cast<const S*>(in_state),
                                          static_cast<const C*>(lam1), static_cast<const C*>(rec),
                                          static_cast<C*>(lam0));
  return cudaGetLastError();
}

}  // namespace maclab
