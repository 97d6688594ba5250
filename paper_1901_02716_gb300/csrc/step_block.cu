// step_block.cu -- block-resident temporal blocking of the D2Q9 step
// (Eqs. (2), (4), (5)): one launch advances the state K steps.
//
// Storage is the interleaved order of the tiled kernel (nx % 4 == 0): pair j
// of row y holds nodes x = j and x = j + H, H = nx / 2.  In these pair
// coordinates every stencil neighbour of pair j is pair j - 1, j or j + 1 of a
// neighbouring row, and pair j + H (j - H) is pair j with its two nodes
// swapped, so a tile is a plain rectangle of pairs whatever its position.
//
//  * A block of 32 x BY threads loads a tile of 32 x BY pairs, one per thread,
//    into registers: an output tile of (32 - 2K) x (BY - 2K) pairs with a
//    halo of K pairs and K rows on every side (wrapped where the axis is
//    periodic; zero rows beyond a closed y boundary).
//  * Each step, every thread forms the nine equilibrium terms T_a of its pair
//    once (Eq. (2), factored as in the tiled kernel), multiplies them by the
//    integer weights 36 w_a (powers of two: exact) and publishes them in
//    shared memory; after one barrier every thread of the valid region, which
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

// FP32 tiles are 32 x 32 pairs (1024 threads); FP64 ones 32 x 16 (the same
// 144 KB of terms), which leaves no output rows at 8 steps.
constexpr int kBlockRowsF32 = 32, kBlockRowsF64 = 16;

}  // namespace

// Steps per launch for the tile setting ty; default (ty = 0, measured on a
// GB300 with cavities of 128^2 to 2048^2): FP32 8 up to 65,536 pairs, 4
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
  const int rows = (precision == MACLAB_F32 ? kBlockRowsF32 : kBlockRowsF64) - 2 * k;
  return (g.ny + rows - 1) / rows <= 65535;
}

int block_threads(int precision) {
  return kBlockBX * (precision == MACLAB_F64 ? kBlockRowsF64 : kBlockRowsF32);
}

// One launch of `steps` steps (1, 2, 4, or 8 with FP32 storage) from s.in to s.out.
cudaError_t launch_block(const StepLaunch& s, cudaStream_t stream, int steps) {
  if (!block_supported(s.g, s.precision, steps)) return cudaErrorInvalidValue;
  if (s.precision == MACLAB_F32) {
    switch (steps) {
      case 1: return launch_block_t<float, 1, kBlockRowsF32>(s, stream);
      case 2: return launch_block_t<float, 2, kBlockRowsF32>(s, stream);
      case 4: return launch_block_t<float, 4, kBlockRowsF32>(s, stream);
      case 8: return launch_block_t<float, 8, kBlockRowsF32>(s, stream);
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
