// step_block.cu -- block-resident temporal blocking of the D2Q9 step
// (Eqs. (2), (4), (5)): one launch advances the state K steps.
//
// Storage is the interleaved order of the tiled kernel (nx % 4 == 0): pair j
// of row y holds nodes x = j and x = j + H, H = nx / 2.  In these pair
// coordinates every stencil neighbour of pair j is pair j - 1, j or j + 1 of a
// neighbouring row, and pair j + H (j - H) is pair j with its two nodes
// swapped, so a tile is a plain rectangle of pairs whatever its position.
//
//  * A block loads a tile of 32 x BY pairs into registers: an output tile of
//    (32 - 2K) x (BY - 2K) pairs with a halo of K pairs and K rows on every
//    side (wrapped where the axis is periodic; zero rows beyond a closed y
//    boundary).  FP64 storage: 32 x 16 pairs, one per thread (step_block_d2q9).
//    FP32 storage: 32 x 32 pairs, 2 x 2 per thread (step_block2_d2q9, below),
//    which keeps most of the exchange in registers and warp shuffles.
//  * Each step, every thread forms the nine equilibrium terms T_a of its pair
//    once (Eq. (2), factored as in the tiled kernel), multiplies them by the
//    integer weights 36 w_a (powers of two: exact) and publishes those other
//    pairs need; after one barrier every thread of the valid region, which
//    shrinks by one pair and one row per step, gathers the nine terms that
//    reach it (Eq. (4)), divides and adds the force (Eq. (5)).  Wall nodes
//    keep their values; beyond a closed boundary only wall nodes are reached.
//  * The sums run in the order of the tiled and segment kernels: source rows
//    y - 1, y, y + 1, and within a row the sources x, x + 1, x - 1 for even x
//    and x - 1, x, x + 1 for odd x.  With the weights folded in, each add is
//    the same rounding as those kernels' fma(w, T, acc), so every step gives
//    the same bits as one step of the tiled kernel.
//  * The term buffers alternate between steps, so one barrier per step
//    suffices: a thread writes buffer s & 1 only after every thread has
//    passed the barrier of step s - 1, i.e. finished its reads of step s - 2.
//  * After K steps the output tile is stored (wall nodes are never written;
//    their values are in both buffers).  Global memory is touched once per K
//    steps: the tile's state once in and once out.

#include "step_tiled.cuh"

namespace maclab {
namespace {

constexpr int kBlockBX = 32;  // pairs per tile row: one warp

// D2Q9 direction with velocity (cx, cy)
__host__ __device__ constexpr int d2q9_dir(int cx, int cy) {
  int r = -1;
  for (int a = 0; a < 9; ++a)
    if (Lattice<kD2Q9>::c(a, 0) == cx && Lattice<kD2Q9>::c(a, 1) == cy) r = a;
  return r;
}

struct BlockArgs {
  const void* in;
  void* out;
  const uint8_t* mask;  // node types in storage order (kWallMask)
  int64_t n;            // nodes (field stride)
  int nx, ny, hx;       // hx = nx / 2
  int px, py;           // periodic flags
  int wall_mode;
  double force[2];      // lattice-unit force increment
};

template <typename S>
struct PairIO;
template <>
struct PairIO<float> {
  __device__ __forceinline__ static float2 ld(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
  __device__ __forceinline__ static void st(float* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
};
template <>
struct PairIO<double> {
  __device__ __forceinline__ static double2 ld(const double* p) {
    return __ldg(reinterpret_cast<const double2*>(p));
  }
  __device__ __forceinline__ static void st(double* p, double2 v) { *reinterpret_cast<double2*>(p) = v; }
};

// The three sources of one source row (velocity cy) in summation order: for
// position k the term slot and pair offset, as an element offset from the
// thread's own pair in the term buffer; sx[k] = cx of that source.
template <int BY, int CY>
__device__ __forceinline__ void row_offsets(bool even, int (&off)[3]) {
  constexpr int PLANE = kBlockBX * BY;
  // even x: cx = 0, -1, +1; odd x: cx = +1, 0, -1
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int cx = even ? (k == 0 ? 0 : (k == 1 ? -1 : 1)) : (k == 0 ? 1 : (k == 1 ? 0 : -1));
    const int a = cx == 0 ? d2q9_dir(0, CY) : (cx > 0 ? d2q9_dir(1, CY) : d2q9_dir(-1, CY));
    off[k] = a * PLANE - CY * kBlockBX - cx;
  }
}

// acc += the three terms of one source row (velocity CY) reaching this pair,
// in summation order: R and M_y from each, M_x through the sources' cx (an
// fma with +-1 rounds as the add / subtract, with 0 it leaves the sum as is).
template <typename C, int CY>
__device__ __forceinline__ void gather_row(const typename Pair<C>::P* v, const int (&off)[3],
                                           const typename Pair<C>::P (&sx)[3], typename Pair<C>::P (&acc)[3]) {
  using O = Pair<C>;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const typename O::P t = v[off[k]];
    acc[0] = O::add(acc[0], t);
    acc[1] = O::fma(sx[k], t, acc[1]);
    if constexpr (CY == 1) acc[2] = O::add(acc[2], t);
    else if constexpr (CY == -1) acc[2] = O::sub(acc[2], t);
  }
}

template <typename S, int K, int BY>
__global__ void __launch_bounds__(kBlockBX * BY, 1) step_block_d2q9(BlockArgs a) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int BX = kBlockBX, TX = BX - 2 * K, TY = BY - 2 * K, PLANE = BX * BY;
  static_assert(TX > 0 && TY > 0, "tile smaller than its halo");
  extern __shared__ __align__(16) unsigned char block_smem[];
  P* const vbuf = reinterpret_cast<P*>(block_smem);  // [2][9][BY][BX] weighted terms
  const int ix = threadIdx.x, iy = threadIdx.y, me = iy * BX + ix;
  const int H = a.hx;
  const int jj = blockIdx.x * TX - K + ix;  // pair column, possibly outside [0, H)
  const int yy = blockIdx.y * TY - K + iy;
  int wraps = jj / H;
  if (jj % H < 0) --wraps;
  const int p = jj - wraps * H;              // stored pair, 0 <= p < H
  const bool swapped = (wraps & 1) != 0;     // its nodes in the other order
  bool row_ok = true;
  int ym = yy;
  if (yy < 0 || yy >= a.ny) {
    if (a.py) ym = ((yy % a.ny) + a.ny) % a.ny;
    else row_ok = false;
  }
  const int64_t off = (int64_t)(row_ok ? ym : 0) * a.nx + 2 * p;

  P st[3];
  uint32_t keep = 3u;  // bit 0 / 1: lane x / y holds a wall node (kept) or a node beyond a closed boundary
  pdl_wait();  // the previous step's writes are visible from here on
  if (row_ok) {
    const S* in = static_cast<const S*>(a.in);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      st[f] = PairIO<S>::ld(in + f * a.n + off);
      if (swapped) st[f] = O::swap(st[f]);
    }
    if (a.wall_mode == kWallMask) {
      const uchar2 m = *reinterpret_cast<const uchar2*>(a.mask + off);
      const uint32_t m0 = m.x != 0 ? 1u : 0u, m1 = m.y != 0 ? 1u : 0u;
      keep = swapped ? (m1 | (m0 << 1)) : (m0 | (m1 << 1));
    } else if (a.wall_mode == kWallBox) {
      const int x0 = swapped ? p + H : p, x1 = swapped ? p : p + H;
      const bool yw = !a.py && (ym == 0 || ym == a.ny - 1);
      const bool w0 = yw || (!a.px && (x0 == 0 || x0 == a.nx - 1));
      const bool w1 = yw || (!a.px && (x1 == 0 || x1 == a.nx - 1));
      keep = (w0 ? 1u : 0u) | (w1 ? 2u : 0u);
    } else {
      keep = 0u;
    }
  } else {
#pragma unroll
    for (int f = 0; f < 3; ++f) st[f] = O::splat(C(0));
  }
  pdl_launch_next();

  const bool even = (jj & 1) == 0;  // x parity of both nodes of the pair (H is even)
  int off_p[3], off_0[3], off_m[3];
  row_offsets<BY, 1>(even, off_p);
  row_offsets<BY, 0>(even, off_0);
  row_offsets<BY, -1>(even, off_m);
  const P sx[3] = {O::splat(even ? C(0) : C(1)), O::splat(even ? C(-1) : C(0)), O::splat(even ? C(1) : C(-1))};
  P force[2];
  force[0] = O::splat(C(a.force[0]));
  force[1] = O::splat(C(a.force[1]));

#pragma unroll 1
  for (int s = 1; s <= K; ++s) {
    P* const vb = vbuf + (s & 1) * 9 * PLANE;
    // sources: the pairs the region of step s reads (rows s - 1 .. BY - s)
    if (iy >= s - 1 && iy <= BY - s) {
      Terms<2, C> tm;
      const P u[3] = {st[1], st[2], O::splat(C(0))};
      make_terms<2, C>(st[0], u, tm);
      static_for<0, 9>([&](auto I) {
        constexpr int d = decltype(I)::value;
        constexpr int w = Lattice<kD2Q9>::w36(d);
        P t = term<kD2Q9, C, d>(tm);
        if constexpr (w != 1) t = O::mul(O::splat(C(w)), t);
        vb[d * PLANE + me] = t;
      });
    }
    __syncthreads();
    if (iy >= s && iy < BY - s && ix >= s && ix < BX - s) {
      P acc[3] = {O::splat(C(0)), O::splat(C(0)), O::splat(C(0))};
      const P* v = vb + me;
      gather_row<C, 1>(v, off_p, sx, acc);   // source row y - 1
      gather_row<C, 0>(v, off_0, sx, acc);   // row y
      gather_row<C, -1>(v, off_m, sx, acc);  // row y + 1
      const P inv = O::rcp(O::add(O::splat(C(36)), acc[0]));
      const P nv[3] = {O::mul(acc[0], O::splat(C(1.0 / 36.0))), O::fma(acc[1], inv, force[0]),
                       O::fma(acc[2], inv, force[1])};
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        if (!(keep & 1u)) st[f].x = nv[f].x;
        if (!(keep & 2u)) st[f].y = nv[f].y;
      }
    }
  }

  // the output tile: pairs 0 <= jj < H of rows 0 <= yy < ny (never swapped)
  if (ix >= K && ix < BX - K && iy >= K && iy < BY - K && jj < H && yy >= 0 && yy < a.ny && keep != 3u) {
    S* out = static_cast<S*>(a.out);
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      S* q = out + f * a.n + off;
      if (keep == 0u) {
        PairIO<S>::st(q, st[f]);
      } else if (keep == 2u) {
        q[0] = st[f].x;
      } else {
        q[1] = st[f].y;
      }
    }
  }
}

// ------------------------------------------------------------------ 2 x 2 pairs per thread
//
// The same tile of 32 x 32 pairs and the same K steps, with 256 threads: a
// thread owns the 2 x 2 pairs (columns 2 tx, 2 tx + 1; rows 2 ty, 2 ty + 1),
// lane tx + 16 (ty & 1) of warp ty / 2.  Of each pair's nine terms, the rest
// term and the three that reach the thread's other pairs stay in registers;
// those crossing into the left or right neighbour's columns within the same
// rows move by warp shuffle; only those crossing into the thread-row above or
// below go through shared memory, three directions per pair, stored at the
// source's column (rows of 36 with two pad columns on each side, thread-rows
// -1 .. 16).  The x parity of a column is fixed by the tile origin (K & 1),
// so the summation order is resolved at compile time.

// a pair from lane - 1 / lane + 1 (a lane at the warp's end gets its own)
template <typename P>
__device__ __forceinline__ P b2_from_left(P v, int d) {
  P r;
  r.x = __shfl_up_sync(0xffffffffu, v.x, d);
  r.y = __shfl_up_sync(0xffffffffu, v.y, d);
  return r;
}
template <typename P>
__device__ __forceinline__ P b2_from_right(P v, int d) {
  P r;
  r.x = __shfl_down_sync(0xffffffffu, v.x, d);
  r.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return r;
}

constexpr int kB2RowStride = 36;                 // columns -2 .. 33
constexpr int kB2Plane = 18 * kB2RowStride;      // thread-rows -1 .. 16

// Terms entering dest (R, CC) from source row R + DY (DY = -1: the row below,
// velocity c_y = +1; 0: the same row; +1: the row above, c_y = -1): vc from the
// same column, vl from the column to the left (c_x = +1), vr from the right
// (c_x = -1).  Rows -1 and 2 are the neighbouring thread-rows' shared terms.
template <typename P, int R, int CC, int DY>
__device__ __forceinline__ void b2_sources(const P (&V)[2][2][9], const P (&fl)[4], const P (&fr)[4],
                                           const P* up, const P* dn, int sb_lo, int sb_hi, P& vc, P& vl,
                                           P& vr) {
  constexpr int RS = R + DY, CY = -DY;
  constexpr int A0 = d2q9_dir(0, CY), AL = d2q9_dir(1, CY), AR = d2q9_dir(-1, CY);
  // shared slots: up (c_y = +1) holds a(0,1), a(1,1), a(-1,1); down holds a(0,-1), a(-1,-1), a(1,-1)
  constexpr int SLOT0 = 0, SLOTL = CY > 0 ? 1 : 2, SLOTR = CY > 0 ? 2 : 1;
  if constexpr (RS == 0 || RS == 1) {
    vc = V[RS][CC][A0];
  } else {
    const P* b = RS < 0 ? up + sb_lo : dn + sb_hi;
    vc = b[SLOT0 * kB2Plane + CC];
  }
  if constexpr (CC == 1) {
    if constexpr (RS == 0 || RS == 1) vl = V[RS][0][AL];
    else vl = (RS < 0 ? up + sb_lo : dn + sb_hi)[SLOTL * kB2Plane + 0];
  } else {
    if constexpr (RS == 0 || RS == 1) {
      // from the left neighbour: a(1,0) of (0,1) / (1,1), a(1,1) of (0,1), a(1,-1) of (1,1)
      vl = CY == 0 ? fl[RS] : (CY > 0 ? fl[2] : fl[3]);
    } else {
      vl = (RS < 0 ? up + sb_lo : dn + sb_hi)[SLOTL * kB2Plane - 1];
    }
  }
  if constexpr (CC == 0) {
    if constexpr (RS == 0 || RS == 1) vr = V[RS][1][AR];
    else vr = (RS < 0 ? up + sb_lo : dn + sb_hi)[SLOTR * kB2Plane + 1];
  } else {
    if constexpr (RS == 0 || RS == 1) {
      // from the right neighbour: a(-1,0) of (0,0) / (1,0), a(-1,1) of (0,0), a(-1,-1) of (1,0)
      vr = CY == 0 ? fr[RS] : (CY > 0 ? fr[2] : fr[3]);
    } else {
      vr = (RS < 0 ? up + sb_lo : dn + sb_hi)[SLOTR * kB2Plane + 2];
    }
  }
}

// acc += one source row's three terms in the order of dest parity EVEN
// (even x: c_x = 0, -1, +1; odd x: +1, 0, -1)
template <typename O, int DY, bool EVEN>
__device__ __forceinline__ void b2_row(typename O::P vc, typename O::P vl, typename O::P vr,
                                       typename O::P (&acc)[3]) {
  auto y = [&](typename O::P t) {
    if constexpr (DY < 0) acc[2] = O::add(acc[2], t);
    else if constexpr (DY > 0) acc[2] = O::sub(acc[2], t);
  };
  if constexpr (EVEN) {
    acc[0] = O::add(acc[0], vc); y(vc);
    acc[0] = O::add(acc[0], vr); acc[1] = O::sub(acc[1], vr); y(vr);
    acc[0] = O::add(acc[0], vl); acc[1] = O::add(acc[1], vl); y(vl);
  } else {
    acc[0] = O::add(acc[0], vl); acc[1] = O::add(acc[1], vl); y(vl);
    acc[0] = O::add(acc[0], vc); y(vc);
    acc[0] = O::add(acc[0], vr); acc[1] = O::sub(acc[1], vr); y(vr);
  }
}

template <typename S, int K>
__global__ void __launch_bounds__(256, 2) step_block2_d2q9(BlockArgs a) {  // FP32: 128 registers
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int TW = kBlockBX, TX = TW - 2 * K;  // tile and output width (and height) in pairs
  extern __shared__ __align__(16) unsigned char block_smem[];
  P* const xb = reinterpret_cast<P*>(block_smem);  // [2 buffers][up, down][3 slots][18][36]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = lane & 15, ty = 2 * warp + (lane >> 4);
  const int H = a.hx;
  const int j0 = blockIdx.x * TX - K, y0 = blockIdx.y * TX - K;

  P st[2][2][3];
  uint32_t keep[2][2];
  int64_t goff[2][2];
  bool out_ok[2][2];
  pdl_wait();  // the previous step's writes are visible from here on
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int ix = 2 * tx + c, iy = 2 * ty + r;
      const int jj = j0 + ix, yy = y0 + iy;
      int wraps = jj / H;
      if (jj % H < 0) --wraps;
      const int p = jj - wraps * H;
      const bool swapped = (wraps & 1) != 0;
      bool row_ok = true;
      int ym = yy;
      if (yy < 0 || yy >= a.ny) {
        if (a.py) ym = ((yy % a.ny) + a.ny) % a.ny;
        else row_ok = false;
      }
      const int64_t off = (int64_t)(row_ok ? ym : 0) * a.nx + 2 * p;
      goff[r][c] = off;
      uint32_t kp = 3u;
      if (row_ok) {
        const S* in = static_cast<const S*>(a.in);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          st[r][c][f] = PairIO<S>::ld(in + f * a.n + off);
          if (swapped) st[r][c][f] = O::swap(st[r][c][f]);
        }
        if (a.wall_mode == kWallMask) {
          const uchar2 m = *reinterpret_cast<const uchar2*>(a.mask + off);
          const uint32_t m0 = m.x != 0 ? 1u : 0u, m1 = m.y != 0 ? 1u : 0u;
          kp = swapped ? (m1 | (m0 << 1)) : (m0 | (m1 << 1));
        } else if (a.wall_mode == kWallBox) {
          const int x0 = swapped ? p + H : p, x1 = swapped ? p : p + H;
          const bool yw = !a.py && (ym == 0 || ym == a.ny - 1);
          const bool w0 = yw || (!a.px && (x0 == 0 || x0 == a.nx - 1));
          const bool w1 = yw || (!a.px && (x1 == 0 || x1 == a.nx - 1));
          kp = (w0 ? 1u : 0u) | (w1 ? 2u : 0u);
        } else {
          kp = 0u;
        }
      } else {
#pragma unroll
        for (int f = 0; f < 3; ++f) st[r][c][f] = O::splat(C(0));
      }
      keep[r][c] = kp;
      out_ok[r][c] = ix >= K && ix < TW - K && iy >= K && iy < TW - K && jj < H && yy >= 0 && yy < a.ny &&
                     kp != 3u;
    }
  pdl_launch_next();

  P force[2];
  force[0] = O::splat(C(a.force[0]));
  force[1] = O::splat(C(a.force[1]));
  const int sb_me = (ty + 1) * kB2RowStride + 2 + 2 * tx;  // (this thread-row, column 2 tx)
  const int sb_lo = sb_me - kB2RowStride, sb_hi = sb_me + kB2RowStride;

#pragma unroll 1
  for (int s = 1; s <= K; ++s) {
    P* const up = xb + (s & 1) * 6 * kB2Plane;
    P* const dn = up + 3 * kB2Plane;
    // the warp's pair rows 4 warp .. 4 warp + 3 against the rows step s reads (s - 1 .. TW - s)
    const bool active = 4 * warp + 3 >= s - 1 && 4 * warp <= TW - s;
    P V[2][2][9];
    P fl[4], fr[4];
    if (active) {
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          Terms<2, C> tm;
          const P u[3] = {st[r][c][1], st[r][c][2], O::splat(C(0))};
          make_terms<2, C>(st[r][c][0], u, tm);
          static_for<0, 9>([&](auto I) {
            constexpr int d = decltype(I)::value;
            constexpr int w = Lattice<kD2Q9>::w36(d);
            P t = term<kD2Q9, C, d>(tm);
            if constexpr (w != 1) t = O::mul(O::splat(C(w)), t);
            V[r][c][d] = t;
          });
        }
      // into the thread-row above: a(0,1), a(1,1), a(-1,1) of row 1; below: a(0,-1), a(-1,-1), a(1,-1) of row 0
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        up[0 * kB2Plane + sb_me + c] = V[1][c][d2q9_dir(0, 1)];
        up[1 * kB2Plane + sb_me + c] = V[1][c][d2q9_dir(1, 1)];
        up[2 * kB2Plane + sb_me + c] = V[1][c][d2q9_dir(-1, 1)];
        dn[0 * kB2Plane + sb_me + c] = V[0][c][d2q9_dir(0, -1)];
        dn[1 * kB2Plane + sb_me + c] = V[0][c][d2q9_dir(-1, -1)];
        dn[2 * kB2Plane + sb_me + c] = V[0][c][d2q9_dir(1, -1)];
      }
      // across columns within the rows (lanes 0 / 15 and 16 / 31 receive
      // values for the tile's edge columns, which no step's region contains)
      fl[0] = b2_from_left(V[0][1][d2q9_dir(1, 0)], 1);
      fl[1] = b2_from_left(V[1][1][d2q9_dir(1, 0)], 1);
      fl[2] = b2_from_left(V[0][1][d2q9_dir(1, 1)], 1);
      fl[3] = b2_from_left(V[1][1][d2q9_dir(1, -1)], 1);
      fr[0] = b2_from_right(V[0][0][d2q9_dir(-1, 0)], 1);
      fr[1] = b2_from_right(V[1][0][d2q9_dir(-1, 0)], 1);
      fr[2] = b2_from_right(V[0][0][d2q9_dir(-1, 1)], 1);
      fr[3] = b2_from_right(V[1][0][d2q9_dir(-1, -1)], 1);
    }
    __syncthreads();
    if (active) {
      // every pair is updated; those outside the step's region hold values
      // that no later step of the valid region reads
      static_for<0, 4>([&](auto Q) {
        constexpr int R = decltype(Q)::value >> 1, CC = decltype(Q)::value & 1;
        constexpr bool EVEN = ((K + CC) & 1) == 0;  // x parity of column 2 tx + CC
        P acc[3] = {O::splat(C(0)), O::splat(C(0)), O::splat(C(0))};
        P vc, vl, vr;
        b2_sources<P, R, CC, -1>(V, fl, fr, up, dn, sb_lo, sb_hi, vc, vl, vr);
        b2_row<O, -1, EVEN>(vc, vl, vr, acc);
        b2_sources<P, R, CC, 0>(V, fl, fr, up, dn, sb_lo, sb_hi, vc, vl, vr);
        b2_row<O, 0, EVEN>(vc, vl, vr, acc);
        b2_sources<P, R, CC, 1>(V, fl, fr, up, dn, sb_lo, sb_hi, vc, vl, vr);
        b2_row<O, 1, EVEN>(vc, vl, vr, acc);
        const P inv = O::rcp(O::add(O::splat(C(36)), acc[0]));
        const P nv[3] = {O::mul(acc[0], O::splat(C(1.0 / 36.0))), O::fma(acc[1], inv, force[0]),
                         O::fma(acc[2], inv, force[1])};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
          if (!(keep[R][CC] & 1u)) st[R][CC][f].x = nv[f].x;
          if (!(keep[R][CC] & 2u)) st[R][CC][f].y = nv[f].y;
        }
      });
    }
  }

  S* out = static_cast<S*>(a.out);
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!out_ok[r][c]) continue;
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        S* q = out + f * a.n + goff[r][c];
        if (keep[r][c] == 0u) PairIO<S>::st(q, st[r][c][f]);
        else if (keep[r][c] == 2u) q[0] = st[r][c][f].x;
        else q[1] = st[r][c][f].y;
      }
    }
}

template <typename S, int K, int BY>
cudaError_t launch_block_t(const StepLaunch& s, cudaStream_t stream) {
  using P = typename Pair<typename Store<S>::C>::P;
  constexpr int TX = kBlockBX - 2 * K, TY = BY - 2 * K;
  constexpr size_t smem = 2 * 9 * (size_t)kBlockBX * BY * sizeof(P);
  auto kern = step_block_d2q9<S, K, BY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BlockArgs a;
  a.in = s.in;
  a.out = s.out;
  a.mask = s.g.mask;
  a.n = s.g.n;
  a.nx = s.g.nx;
  a.ny = s.g.ny;
  a.hx = s.g.nx / 2;
  a.px = (s.g.periodic & 1u) ? 1 : 0;
  a.py = (s.g.periodic & 2u) ? 1 : 0;
  a.wall_mode = s.g.wall_mode;
  a.force[0] = s.force[0];
  a.force[1] = s.force[1];
  const dim3 grid((unsigned)((a.hx + TX - 1) / TX), (unsigned)((a.ny + TY - 1) / TY));
  return launch_kernel(kern, grid, dim3(kBlockBX, BY), smem, stream, s.overlap, a);
}

template <typename S, int K>
cudaError_t launch_block2_t(const StepLaunch& s, cudaStream_t stream) {
  using P = typename Pair<typename Store<S>::C>::P;
  constexpr int TX = kBlockBX - 2 * K;
  constexpr size_t smem = 2 * 6 * (size_t)kB2Plane * sizeof(P);
  auto kern = step_block2_d2q9<S, K>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  BlockArgs a;
  a.in = s.in;
  a.out = s.out;
  a.mask = s.g.mask;
  a.n = s.g.n;
  a.nx = s.g.nx;
  a.ny = s.g.ny;
  a.hx = s.g.nx / 2;
  a.px = (s.g.periodic & 1u) ? 1 : 0;
  a.py = (s.g.periodic & 2u) ? 1 : 0;
  a.wall_mode = s.g.wall_mode;
  a.force[0] = s.force[0];
  a.force[1] = s.force[1];
  const dim3 grid((unsigned)((a.hx + TX - 1) / TX), (unsigned)((a.ny + TX - 1) / TX));
  return launch_kernel(kern, grid, dim3(256), smem, stream, s.overlap, a);
}

// FP32: the 2 x 2 form (256 threads, two blocks per SM); FP64: one pair per
// thread on tiles of 32 x 16 pairs (512 threads; the 2 x 2 form needs 224
// registers in FP64 and measured 1.7x slower), which leaves no output rows at
// 8 steps.
constexpr int kBlockRowsF64 = 16;

}  // namespace

// Steps per launch for the tile setting ty; default (ty = 0, measured on a
// GB300 with cavities of 128^2 to 1024^2): FP32 8 up to 65,536 pairs, 4
// above; FP64 4 up to 16,384 pairs, 2 above.
int block_steps(const Geometry& g, int precision, int ty) {
  if (precision != MACLAB_F32 && precision != MACLAB_F64) return 0;
  const int64_t pairs = (int64_t)(g.nx / 2) * g.ny;
  if (ty == 0) return precision == MACLAB_F32 ? (pairs <= 65536 ? 8 : 4) : (pairs <= 16384 ? 4 : 2);
  if (ty == 1 || ty == 2 || ty == 4) return ty;
  if (ty == 8 && precision == MACLAB_F32) return 8;
  return 0;
}

bool block_supported(const Geometry& g, int precision, int ty) {
  const int k = block_steps(g, precision, ty);
  if (g.lattice != kD2Q9 || !g.ilv || k == 0) return false;
  const int rows = (precision == MACLAB_F32 ? kBlockBX : kBlockRowsF64) - 2 * k;
  return (g.ny + rows - 1) / rows <= 65535;
}

int block_threads(int precision) { return precision == MACLAB_F64 ? kBlockBX * kBlockRowsF64 : 256; }

// One launch of `steps` steps (1, 2, 4, or 8 with FP32 storage) from s.in to s.out.
cudaError_t launch_block(const StepLaunch& s, cudaStream_t stream, int steps) {
  if (!block_supported(s.g, s.precision, steps)) return cudaErrorInvalidValue;
  if (s.precision == MACLAB_F32) {
    switch (steps) {
      case 1: return launch_block2_t<float, 1>(s, stream);
      case 2: return launch_block2_t<float, 2>(s, stream);
      case 4: return launch_block2_t<float, 4>(s, stream);
      case 8: return launch_block2_t<float, 8>(s, stream);
    }
  } else {
    switch (steps) {
      case 1: return launch_block_t<double, 1, kBlockRowsF64>(s, stream);
      case 2: return launch_block_t<double, 2, kBlockRowsF64>(s, stream);
      case 4: return launch_block_t<double, 4, kBlockRowsF64>(s, stream);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace maclab
