// step_tiled.cu -- the tiled MacLAB step kernel (Eqs. (2), (4), (5)).
//
// Same update as step_naive (see step.cu for the drho form), organised so that
// every stored value is read from memory once per step and every equilibrium
// F_a(y) is evaluated once, at its source node y, then moved to the node that
// gathers it (y + c_a):
//
//  * A thread owns a strip of 4 consecutive x nodes (one 16-byte load per field
//    in FP32).  A block spans the whole x extent, so wrap in x is an index
//    wrap in shared memory.
//  * The block marches along the slowest axis (z in 3D, y in 2D) over a chunk
//    of TZ planes, plus one halo plane on each side.  The momentum sums of
//    three destination planes (p - 1, p, p + 1) live in registers; after
//    source plane p, plane p - 1 is complete and is written out.
//  * In 3D a block holds TY rows of y plus a halo row on each side; halo rows
//    only publish the equilibria that cross into the tile.
//  * Equilibria that stay in the thread's strip are added in registers; those
//    that leave it (x edge, or another row in 3D) go through shared memory.
//    The shared arrays are laid out [slot][row][node-in-strip][thread] so that
//    every access of a warp is 32 consecutive words (no bank conflicts).
//  * The equilibrium is factored once per node: with rho = 1 + drho and
//    everything scaled by 1/36,
//       B_i = rho/12 u_i,  P_ii = 3/2 B_i u_i,  P_ij = 3 B_i u_j,
//       A = drho/36 - (P_xx + P_yy + P_zz)/3,
//    36 w_a f_a^eq-minus-w_a = w36_a (A + c.B + sum_i c_i^2 P_ii
//    + sum_{i<j} c_i c_j P_ij), and the constant part cancels as in step.cu.
//  * Wall nodes are never written (their values are in both buffers).

#include "common.cuh"
#include "lattice.cuh"

namespace maclab {

// ------------------------------------------------------------------ frame
// Frame axes: x (threads), the in-plane row axis (3D: y; 2D: none) and the
// march axis (3D: z; 2D: y).
template <int LAT>
struct Frame {
  using L = Lattice<LAT>;
  static constexpr int D = L::D;
  static constexpr int Q = L::Q;
  __host__ __device__ static constexpr int fx(int a) { return L::c(a, 0); }
  __host__ __device__ static constexpr int fy(int a) { return D == 3 ? L::c(a, 1) : 0; }
  __host__ __device__ static constexpr int fz(int a) { return D == 3 ? L::c(a, 2) : L::c(a, 1); }
  __host__ __device__ static constexpr bool xcross(int a) { return fy(a) == 0 && fx(a) != 0; }
  __host__ __device__ static constexpr bool ycross(int a) { return fy(a) != 0; }
  __host__ __device__ static constexpr int xslot(int a) {
    int s = 0;
    for (int b = 0; b < a; ++b) s += xcross(b) ? 1 : 0;
    return s;
  }
  __host__ __device__ static constexpr int yslot(int a) {
    int s = 0;
    for (int b = 0; b < a; ++b) s += ycross(b) ? 1 : 0;
    return s;
  }
  __host__ __device__ static constexpr int count_x() { return xslot(Q); }
  __host__ __device__ static constexpr int count_y() { return yslot(Q); }
};

struct TiledArgs {
  int nx, ny, nplanes;     // ny = 1 in 2D; nplanes = extent of the march axis
  int64_t n;               // nodes per field
  int64_t plane_stride;    // nx * ny
  int ty, tz;              // rows per tile (3D), planes per chunk
  int px, py, pz;          // periodic flags of the frame axes
  int wall_mode;
  const uint8_t* mask;
  double force[3];
};

// ------------------------------------------------------------------ vector I/O

template <typename S>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ __forceinline__ static void ld(const float* p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec4<double> {
  __device__ __forceinline__ static void ld(const double* p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ static void st(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};
template <>
struct Vec4<__nv_bfloat16> {
  __device__ __forceinline__ static void ld(const __nv_bfloat16* p, float (&v)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&t.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&t.y);
    const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, const float (&v)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&a);
    t.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
  }
};
template <>
struct Vec4<__half> {
  __device__ __forceinline__ static void ld(const __half* p, float (&v)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    const __half2 a = *reinterpret_cast<const __half2*>(&t.x);
    const __half2 b = *reinterpret_cast<const __half2*>(&t.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
  }
  __device__ __forceinline__ static void st(__half* p, const float (&v)[4]) {
    const __half2 a = __floats2half2_rn(v[0], v[1]);
    const __half2 b = __floats2half2_rn(v[2], v[3]);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&a);
    t.y = *reinterpret_cast<const unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = t;
  }
};

// ------------------------------------------------------------------ per-node terms

template <int D, typename C>
struct Terms {
  C A;
  C B[3];
  C S[3];           // A + P_ii
  C Ep[3], Em[3];   // pair k = (i, j): S_i + P_jj +- P_ij
  C Op[3], Om[3];   // B_i +- B_j
};

__host__ __device__ constexpr int pair_index(int i, int j) { return i + j - 1; }  // (0,1)->0 (0,2)->1 (1,2)->2

template <int D, typename C>
__device__ __forceinline__ void make_terms(C r, const C (&u)[3], Terms<D, C>& t) {
  const C g = (C(1) + r) * C(1.0 / 12.0);
  C P[3];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    t.B[i] = g * u[i];
    P[i] = C(1.5) * t.B[i] * u[i];
  }
  C psum = P[0] + P[1];
  if (D == 3) psum += P[2];
  t.A = r * C(1.0 / 36.0) - psum * C(1.0 / 3.0);
#pragma unroll
  for (int i = 0; i < D; ++i) t.S[i] = t.A + P[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i + 1; j < D; ++j) {
      const int k = pair_index(i, j);
      const C pij = C(3) * t.B[i] * u[j];
      const C base = t.S[i] + P[j];
      t.Ep[k] = base + pij;
      t.Em[k] = base - pij;
      t.Op[k] = t.B[i] + t.B[j];
      t.Om[k] = t.B[i] - t.B[j];
    }
}

// T_a = A + c.B + sum c_i^2 P_ii + sum_{i<j} c_i c_j P_ij (all / 36)
template <int LAT, typename C>
__device__ __forceinline__ C term(const Terms<Lattice<LAT>::D, C>& t, int a) {
  using L = Lattice<LAT>;
  int nzc = 0, i0 = -1, i1 = -1;
  for (int i = 0; i < L::D; ++i)
    if (L::c(a, i) != 0) {
      if (nzc == 0) i0 = i; else i1 = i;
      ++nzc;
    }
  if (nzc == 0) return t.A;
  if (nzc == 1) return L::c(a, i0) > 0 ? t.S[i0] + t.B[i0] : t.S[i0] - t.B[i0];
  const int k = pair_index(i0, i1);
  const int s0 = L::c(a, i0), s1 = L::c(a, i1);
  if (s0 == s1) return s0 > 0 ? t.Ep[k] + t.Op[k] : t.Ep[k] - t.Op[k];
  return s0 > 0 ? t.Em[k] + t.Om[k] : t.Em[k] - t.Om[k];
}

// acc[0] += w36 T; acc[1 + i] += c_i w36 T
template <int LAT, typename C>
__device__ __forceinline__ void accum(C (&acc)[Lattice<LAT>::D + 1], C T, int a) {
  using L = Lattice<LAT>;
  const int w = L::w36(a);
  acc[0] = (w == 1) ? acc[0] + T : fma(C(w), T, acc[0]);
#pragma unroll
  for (int i = 0; i < L::D; ++i) {
    const int c = L::c(a, i);
    if (c == 1) acc[1 + i] = (w == 1) ? acc[1 + i] + T : fma(C(w), T, acc[1 + i]);
    if (c == -1) acc[1 + i] = (w == 1) ? acc[1 + i] - T : fma(C(-w), T, acc[1 + i]);
  }
}

enum PlaneMode { kFirst = 0, kMid = 1, kLast = 2 };

template <int LAT, int MODE>
__device__ __forceinline__ constexpr bool mode_allows(int a) {
  return MODE == kMid || (MODE == kFirst && Frame<LAT>::fz(a) == 1) ||
         (MODE == kLast && Frame<LAT>::fz(a) == -1);
}

// One source plane: publish outgoing equilibria, gather incoming ones.
// st: the plane's state for the thread's 4 nodes (field-major).
// ap/ac/an: momentum sums of destination planes p-1, p, p+1 (node-major).
template <int LAT, typename C, int MODE>
__device__ __forceinline__ void plane_update(const C (&st)[Lattice<LAT>::D + 1][4],
                                             C (&ap)[4][Lattice<LAT>::D + 1],
                                             C (&ac)[4][Lattice<LAT>::D + 1],
                                             C (&an)[4][Lattice<LAT>::D + 1], C* __restrict__ Xe,
                                             C* __restrict__ Ye, int tx, int r, int BX, int RY,
                                             bool interior, bool halo_lo, bool halo_hi) {
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  constexpr int D = L::D;
  constexpr int NXS = F::count_x();
  // Xe: [NXS][RY][BX]; Ye: [NYS][RY][4][BX]
  (void)NXS;
  const bool publish_any = interior || halo_lo || halo_hi;
  if (publish_any) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      Terms<D, C> t;
      C u[3] = {st[1][j], st[2][j], D == 3 ? st[3][j] : C(0)};
      make_terms<D, C>(st[0][j], u, t);
#pragma unroll
      for (int a = 0; a < L::Q; ++a) {
        if (!mode_allows<LAT, MODE>(a)) continue;
        const int fz = F::fz(a);
        if (F::ycross(a)) {
          const int fy = F::fy(a);
          if (interior || (halo_lo && fy == 1) || (halo_hi && fy == -1))
            Ye[((F::yslot(a) * RY + r) * 4 + j) * BX + tx] = term<LAT, C>(t, a);
        } else if (interior) {
          const C T = term<LAT, C>(t, a);
          const int jd = j + F::fx(a);
          if (jd >= 0 && jd < 4) {
            if (fz == 1) accum<LAT, C>(an[jd], T, a);
            else if (fz == 0) accum<LAT, C>(ac[jd], T, a);
            else accum<LAT, C>(ap[jd], T, a);
          } else {
            Xe[(F::xslot(a) * RY + r) * BX + tx] = T;
          }
        }
      }
    }
  }
  __syncthreads();
  if (interior) {
    const int txl = tx == 0 ? BX - 1 : tx - 1;   // thread owning x0 - 1 (wrapped)
    const int txr = tx == BX - 1 ? 0 : tx + 1;   // thread owning x0 + 4 (wrapped)
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      if (!mode_allows<LAT, MODE>(a)) continue;
      const int fz = F::fz(a);
      const int fx = F::fx(a);
      C(&dst)[4][D + 1] = fz == 1 ? an : (fz == 0 ? ac : ap);
      if (F::xcross(a)) {
        // from the neighbouring strip's edge node
        const C v = Xe[(F::xslot(a) * RY + r) * BX + (fx == 1 ? txl : txr)];
        accum<LAT, C>(dst[fx == 1 ? 0 : 3], v, a);
      } else if (F::ycross(a)) {
        const int rs = r - F::fy(a);
        const C* row = Ye + (F::yslot(a) * RY + rs) * 4 * BX;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // source node x0 + j - fx
          const int js = j - fx;
          C v;
          if (js < 0) v = row[3 * BX + txl];
          else if (js > 3) v = row[0 * BX + txr];
          else v = row[js * BX + tx];
          accum<LAT, C>(dst[j], v, a);
        }
      }
    }
  }
  __syncthreads();
}

template <int LAT, typename S>
__device__ __forceinline__ void load_plane(const S* __restrict__ in, const TiledArgs& ta,
                                           int64_t off, bool exists,
                                           typename Store<S>::C (&st)[Lattice<LAT>::D + 1][4]) {
  using C = typename Store<S>::C;
  constexpr int K = Lattice<LAT>::D + 1;
#pragma unroll
  for (int f = 0; f < K; ++f) {
    if (exists) {
      Vec4<S>::ld(in + f * ta.n + off, st[f]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) st[f][j] = C(0);
    }
  }
}

template <int LAT, typename S>
__device__ __forceinline__ void store_plane(S* __restrict__ out, const TiledArgs& ta, int64_t off,
                                            int x0, bool plane_wall, bool row_wall,
                                            typename Store<S>::C (&a)[4][Lattice<LAT>::D + 1]) {
  using C = typename Store<S>::C;
  constexpr int D = Lattice<LAT>::D;
  if (plane_wall || row_wall) return;
  bool wall[4] = {false, false, false, false};
  bool any = false;
  if (ta.wall_mode == kWallBox) {
    if (!ta.px) {
      wall[0] = x0 == 0;
      wall[3] = x0 + 3 == ta.nx - 1;
      any = wall[0] || wall[3];
    }
  } else if (ta.wall_mode == kWallMask) {
    const uchar4 m = *reinterpret_cast<const uchar4*>(ta.mask + off);
    wall[0] = m.x != 0; wall[1] = m.y != 0; wall[2] = m.z != 0; wall[3] = m.w != 0;
    any = wall[0] || wall[1] || wall[2] || wall[3];
  }
  C v[D + 1][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const C rho = C(1) + a[j][0];
    C inv;
    if constexpr (sizeof(C) == 4) inv = __frcp_rn(rho);
    else inv = C(1) / rho;
    v[0][j] = a[j][0];
#pragma unroll
    for (int i = 0; i < D; ++i) v[1 + i][j] = a[j][1 + i] * inv + C(ta.force[i]);
  }
  if (!any) {
#pragma unroll
    for (int f = 0; f <= D; ++f) Vec4<S>::st(out + f * ta.n + off, v[f]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (!wall[j])
#pragma unroll
        for (int f = 0; f <= D; ++f) Store<S>::st(out + f * ta.n + off + j, v[f][j]);
  }
}

template <int LAT, typename S>
__global__ void __launch_bounds__(512) step_tiled(TiledArgs ta, const S* __restrict__ in,
                                                  S* __restrict__ out) {
  using C = typename Store<S>::C;
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  constexpr int D = L::D;
  constexpr int K = D + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int BX = blockDim.x, RY = blockDim.y;
  const int tx = threadIdx.x, r = threadIdx.y;
  C* Xe = reinterpret_cast<C*>(smem_raw);
  C* Ye = Xe + F::count_x() * RY * BX;
  const int x0 = 4 * tx;

  // in-plane row (3D) of this thread
  int row = 0, row_mem = 0;
  bool row_exists = true, interior = true, halo_lo = false, halo_hi = false;
  if (D == 3) {
    row = blockIdx.y * ta.ty + r - 1;
    halo_lo = r == 0;
    halo_hi = r == RY - 1;
    interior = !halo_lo && !halo_hi && row < ta.ny;
    row_mem = row;
    if (row < 0 || row >= ta.ny) {
      if (ta.py) row_mem = (row + ta.ny) % ta.ny;
      else row_exists = false;
    }
  }
  const bool row_wall = D == 3 && !ta.py && (row == 0 || row == ta.ny - 1);
  const int64_t row_off = (int64_t)row_mem * ta.nx + x0;

  const int z0 = blockIdx.x * ta.tz;
  const int z1 = min(z0 + ta.tz, ta.nplanes);
  auto plane_exists = [&](int p) { return (p >= 0 && p < ta.nplanes) || ta.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + ta.nplanes : (p >= ta.nplanes ? p - ta.nplanes : p); };
  auto plane_wall = [&](int q) { return !ta.pz && (q == 0 || q == ta.nplanes - 1); };

  C ap[4][K], ac[4][K], an[4][K];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < K; ++k) ap[j][k] = ac[j][k] = an[j][k] = C(0);

  C st[K][4], nxt[K][4];
  // first (halo) plane z0 - 1: only the equilibria moving up the march axis
  {
    const int p = z0 - 1;
    const bool ex = plane_exists(p);
    load_plane<LAT, S>(in, ta, (int64_t)plane_mem(p) * ta.plane_stride + row_off,
                       ex && row_exists, st);
    load_plane<LAT, S>(in, ta, (int64_t)z0 * ta.plane_stride + row_off, row_exists, nxt);
    if (ex) plane_update<LAT, C, kFirst>(st, ap, ac, an, Xe, Ye, tx, r, BX, RY, interior, halo_lo, halo_hi);
  }
  // rotate: dest z0 becomes "current"
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      ac[j][k] = an[j][k];
      an[j][k] = C(0);
    }
  for (int p = z0; p < z1; ++p) {
#pragma unroll
    for (int f = 0; f < K; ++f)
#pragma unroll
      for (int j = 0; j < 4; ++j) st[f][j] = nxt[f][j];
    {
      const int pn = p + 1;
      const bool exn = plane_exists(pn) && row_exists;
      load_plane<LAT, S>(in, ta, (int64_t)plane_mem(pn) * ta.plane_stride + row_off, exn, nxt);
    }
    plane_update<LAT, C, kMid>(st, ap, ac, an, Xe, Ye, tx, r, BX, RY, interior, halo_lo, halo_hi);
    if (p - 1 >= z0 && interior)
      store_plane<LAT, S>(out, ta, (int64_t)(p - 1) * ta.plane_stride + row_off, x0,
                          plane_wall(p - 1), row_wall, ap);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        ap[j][k] = ac[j][k];
        ac[j][k] = an[j][k];
        an[j][k] = C(0);
      }
  }
  // last (halo) plane z1: only the equilibria moving down the march axis
  {
    const int p = z1;
    if (plane_exists(p)) {
#pragma unroll
      for (int f = 0; f < K; ++f)
#pragma unroll
        for (int j = 0; j < 4; ++j) st[f][j] = nxt[f][j];
      plane_update<LAT, C, kLast>(st, ap, ac, an, Xe, Ye, tx, r, BX, RY, interior, halo_lo, halo_hi);
    }
    if (interior)
      store_plane<LAT, S>(out, ta, (int64_t)(z1 - 1) * ta.plane_stride + row_off, x0,
                          plane_wall(z1 - 1), row_wall, ap);
  }
}

// ------------------------------------------------------------------ host side

struct TiledShape {
  int ty, tz, bx, ry;
  size_t smem;
};

static TiledShape tiled_shape(const Geometry& g, int precision, int ty_req, int tz_req) {
  TiledShape s{};
  const size_t cb = precision == MACLAB_F64 ? 8 : 4;
  s.bx = g.nx / 4;
  if (g.d == 3) {
    s.ty = ty_req > 0 ? ty_req : 4;
    s.ry = s.ty + 2;
    s.tz = tz_req > 0 ? tz_req : 8;
    s.smem = cb * ((size_t)6 * s.ry * s.bx + (size_t)10 * s.ry * 4 * s.bx);
  } else {
    s.ty = 1;
    s.ry = 1;
    s.tz = tz_req > 0 ? tz_req : 8;
    s.smem = cb * (size_t)6 * s.bx;
  }
  return s;
}

bool tiled_supported(const Geometry& g, int precision, int ty, int tz) {
  if (g.nx % 4 != 0 || g.nx < 4) return false;
  const TiledShape s = tiled_shape(g, precision, ty, tz);
  if (s.bx * s.ry > 512) return false;
  if (s.smem > 200 * 1024) return false;
  if (g.d == 3 && (g.periodic & 2u) && g.ny % s.ty != 0) return false;
  if (g.d == 2 && g.ny < 1) return false;
  return true;
}

template <int LAT, typename S>
static cudaError_t launch_tiled_t(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  const Geometry& g = sl.g;
  const TiledShape s = tiled_shape(g, sl.precision, ty, tz);
  TiledArgs ta{};
  ta.nx = g.nx;
  ta.ny = g.d == 3 ? g.ny : 1;
  ta.nplanes = g.d == 3 ? g.nz : g.ny;
  ta.n = g.n;
  ta.plane_stride = (int64_t)g.nx * ta.ny;
  ta.ty = s.ty;
  ta.tz = s.tz;
  ta.px = (g.periodic & 1u) ? 1 : 0;
  ta.py = g.d == 3 ? ((g.periodic & 2u) ? 1 : 0) : 0;
  ta.pz = g.d == 3 ? ((g.periodic & 4u) ? 1 : 0) : ((g.periodic & 2u) ? 1 : 0);
  ta.wall_mode = g.wall_mode;
  ta.mask = g.mask;
  for (int i = 0; i < 3; ++i) ta.force[i] = sl.force[i];
  const dim3 block(s.bx, s.ry);
  const dim3 grid((ta.nplanes + s.tz - 1) / s.tz, g.d == 3 ? (ta.ny + s.ty - 1) / s.ty : 1);
  auto kern = step_tiled<LAT, S>;
  if (s.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, s.smem, stream>>>(ta, static_cast<const S*>(sl.in), static_cast<S*>(sl.out));
  return cudaGetLastError();
}

template <int LAT>
static cudaError_t launch_tiled_lat(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  switch (sl.precision) {
    case MACLAB_F64: return launch_tiled_t<LAT, double>(sl, stream, ty, tz);
    case MACLAB_F32: return launch_tiled_t<LAT, float>(sl, stream, ty, tz);
    case MACLAB_BF16_STORE: return launch_tiled_t<LAT, __nv_bfloat16>(sl, stream, ty, tz);
    case MACLAB_F16_STORE: return launch_tiled_t<LAT, __half>(sl, stream, ty, tz);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tiled(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  return sl.g.lattice == kD2Q9 ? launch_tiled_lat<kD2Q9>(sl, stream, ty, tz)
                               : launch_tiled_lat<kD3Q19>(sl, stream, ty, tz);
}

int tiled_threads(const Geometry& g, int precision, int ty, int tz) {
  const TiledShape s = tiled_shape(g, precision, ty, tz);
  return s.bx * s.ry;
}

}  // namespace maclab
