// step_tiled.cuh -- the tiled MacLAB step kernel (Eqs. (2), (4), (5)).
//
// Same update as step_naive (see step.cu for the drho form), organised so that
// every stored value is read from memory once per step, every equilibrium
// F_a(y) is evaluated once, at its source node y, and then moved to the node
// that gathers it (y + c_a), and the FP32 arithmetic runs on the paired FP32
// datapath (one add.f32x2 / fma.f32x2 does two nodes).
//
//  * Storage order (set up by the library when nx % 4 == 0): within each x
//    row the two halves are interleaved, node x at position
//    2 (x mod H) + [x >= H], H = nx / 2.  One 16-byte load at position 4t
//    then gives the two node pairs a = (2t, 2t + H) and b = (2t + 1, 2t + 1 + H)
//    of thread t, already in aligned register pairs, and a shift by one node
//    in x maps pair a onto pair b of the same thread and pair b onto pair a of
//    thread t + 1: every lane-wise operation stays lane-wise.
//  * A block spans the whole x extent.  The seam between the two half rows
//    (x = H - 1 -> H, and the periodic wrap nx - 1 -> 0) swaps lanes; the
//    threads at the ends of the row publish a lane-swapped copy for it.
//  * The block marches along the slowest axis (z in 3D, y in 2D) over a chunk
//    of TZ planes plus a halo plane on each side.  The momentum sums of three
//    destination planes (p - 1, p, p + 1) stay in registers; after source
//    plane p, plane p - 1 is complete and is written out.
//  * In 3D a block holds TY rows of y plus a halo row on each side; halo rows
//    only publish the equilibria that cross into the tile.
//  * Equilibria that stay in the thread go straight into its sums; the others
//    go through shared memory laid out so a warp touches 32 consecutive pairs.
//  * The equilibrium is factored once per node: with rho = 1 + drho,
//    f_a^eq - w_a = w_a T_a,  T_a = A + c.B + sum_i c_i^2 P_ii + sum_{i<j} c_i c_j P_ij,
//    B_i = 3 rho u_i,  P_ii = 9/2 rho u_i^2,  P_ij = 9 rho u_i u_j,
//    A = drho - 3/2 rho u.u.  The sums are gathered with the integer weights
//    w36_a = 36 w_a: R = sum w36 T = 36 drho', M = sum w36 c T = 36 m'.
//  * Wall nodes are never written (their values are in both buffers).
#pragma once
#include <type_traits>

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
  int ty, nzc;             // rows per tile (3D), number of chunks of the march axis
  int px, py, pz;          // periodic flags of the frame axes
  int wall_mode;
  const uint8_t* mask;     // node types in storage order (kWallMask)
  double force[3];
  int overlap;             // host side: launch with programmatic dependent launch
  BoundsLog* bounds;       // debug builds: where bad indices are recorded (bounds_ok)
  const float* lam;        // viscosity-term launches: the adjoint of the state after the step
  double* nu_acc;          // viscosity-term launches: the sum's accumulator (one double)
  unsigned* status;        // bit 0 set when a bounded wait on a copy ran out (step_status())
};

// ------------------------------------------------------------------ lane pairs

template <typename C>
struct Pair;

template <>
struct Pair<float> {
  using P = float2;
  __device__ __forceinline__ static unsigned long long pk(P v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
  }
  __device__ __forceinline__ static P upk(unsigned long long r) {
    P v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
  }
  __device__ __forceinline__ static P make(float a, float b) { return make_float2(a, b); }
  __device__ __forceinline__ static P splat(float a) { return make_float2(a, a); }
  __device__ __forceinline__ static P add(P a, P b) { return __fadd2_rn(a, b); }
  __device__ __forceinline__ static P sub(P a, P b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
    return upk(d);
  }
  __device__ __forceinline__ static P mul(P a, P b) { return __fmul2_rn(a, b); }
  __device__ __forceinline__ static P fma(P a, P b, P c) { return __ffma2_rn(a, b, c); }
  // 1/a on both lanes: the hardware approximation r0 (rcp.approx, relative
  // error below 2^-22) refined by one Newton-Raphson step for f(r) = 1/r - a,
  // r1 = r0 + r0 (1 - a r0), on the paired FMA datapath.  The residual
  // 1 - a r0 is formed exactly by the FMA, so r1 is within about half an ulp
  // of 1/a (checked by maclab_check_reciprocal).  The arguments here are
  // 36 + R and 1 + drho, far from zero, infinities and subnormals.
  __device__ __forceinline__ static P rcp(P a) {
    float r0, r1;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(a.y));
    const P r = make_float2(r0, r1);
    const P e = __ffma2_rn(make_float2(-a.x, -a.y), r, make_float2(1.f, 1.f));
    return __ffma2_rn(r, e, r);
  }
  __device__ __forceinline__ static P swap(P a) { return make_float2(a.y, a.x); }
};

template <>
struct Pair<double> {
  using P = double2;
  __device__ __forceinline__ static P make(double a, double b) { return make_double2(a, b); }
  __device__ __forceinline__ static P splat(double a) { return make_double2(a, a); }
  __device__ __forceinline__ static P add(P a, P b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ __forceinline__ static P sub(P a, P b) { return make_double2(a.x - b.x, a.y - b.y); }
  __device__ __forceinline__ static P mul(P a, P b) { return make_double2(a.x * b.x, a.y * b.y); }
  __device__ __forceinline__ static P fma(P a, P b, P c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
  }
  __device__ __forceinline__ static P rcp(P a) { return make_double2(1.0 / a.x, 1.0 / a.y); }
  __device__ __forceinline__ static P swap(P a) { return make_double2(a.y, a.x); }
};

// ------------------------------------------------------------------ storage I/O
// Four consecutive stored values <-> the thread's pairs a = (v0, v1), b = (v2, v3).

__device__ __forceinline__ void cp_async16(uint32_t smem, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t smem, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename S>
struct Quad;
template <>
struct Quad<float> {
  using P = float2;
  static constexpr int BYTES = 16;
  __device__ __forceinline__ static void copy(uint32_t smem, const float* g) { cp_async16(smem, g); }
  __device__ __forceinline__ static void lds(const float* p, P& a, P& b) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
  }
  __device__ __forceinline__ static void ld(const float* p, P& a, P& b) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    a = make_float2(t.x, t.y);
    b = make_float2(t.z, t.w);
  }
  __device__ __forceinline__ static void st(float* p, P a, P b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ __forceinline__ static void st1(float* p, float v) { *p = v; }
};
template <>
struct Quad<double> {
  using P = double2;
  static constexpr int BYTES = 32;
  __device__ __forceinline__ static void copy(uint32_t smem, const double* g) {
    cp_async16(smem, g);
    cp_async16(smem + 16, g + 2);
  }
  __device__ __forceinline__ static void lds(const double* p, P& a, P& b) {
    a = reinterpret_cast<const double2*>(p)[0];
    b = reinterpret_cast<const double2*>(p)[1];
  }
  __device__ __forceinline__ static void ld(const double* p, P& a, P& b) {
    a = __ldg(reinterpret_cast<const double2*>(p));
    b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  }
  __device__ __forceinline__ static void st(double* p, P a, P b) {
    reinterpret_cast<double2*>(p)[0] = a;
    reinterpret_cast<double2*>(p)[1] = b;
  }
  __device__ __forceinline__ static void st1(double* p, double v) { *p = v; }
};
template <>
struct Quad<__nv_bfloat16> {
  using P = float2;
  static constexpr int BYTES = 8;
  __device__ __forceinline__ static void copy(uint32_t smem, const __nv_bfloat16* g) { cp_async8(smem, g); }
  __device__ __forceinline__ static void lds(const __nv_bfloat16* p, P& a, P& b) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.y));
  }
  __device__ __forceinline__ static void ld(const __nv_bfloat16* p, P& a, P& b) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&t.y));
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, P a, P b) {
    const __nv_bfloat162 x = __float22bfloat162_rn(a), y = __float22bfloat162_rn(b);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&x);
    t.y = *reinterpret_cast<const unsigned*>(&y);
    *reinterpret_cast<uint2*>(p) = t;
  }
  __device__ __forceinline__ static void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct Quad<__half> {
  using P = float2;
  static constexpr int BYTES = 8;
  __device__ __forceinline__ static void copy(uint32_t smem, const __half* g) { cp_async8(smem, g); }
  __device__ __forceinline__ static void lds(const __half* p, P& a, P& b) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
  }
  __device__ __forceinline__ static void ld(const __half* p, P& a, P& b) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
  }
  __device__ __forceinline__ static void st(__half* p, P a, P b) {
    const __half2 x = __float22half2_rn(a), y = __float22half2_rn(b);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&x);
    t.y = *reinterpret_cast<const unsigned*>(&y);
    *reinterpret_cast<uint2*>(p) = t;
  }
  __device__ __forceinline__ static void st1(__half* p, float v) { *p = __float2half_rn(v); }
};

// ------------------------------------------------------------------ per-pair terms

template <int D, typename C>
struct Terms {
  using P = typename Pair<C>::P;
  P A;
  P B[3];
  P S[3];          // A + P_ii (D3Q19: 2 (A + P_ii), see kAxisScale)
  P Ep[3], Em[3];  // pair k = (i, j): S_i + P_jj +- P_ij
  P Op[3], Om[3];  // B_i +- B_j
  P B2[3];         // D3Q19: 2 B_i (axis directions carry their weight 2)
};

// D3Q19 axis directions have weight w36 = 2; their T_a is formed already
// doubled (2 S_i +- 2 B_i), so they are accumulated with a plain add.
template <int LAT>
struct AxisScale {
  static constexpr int value = LAT == kD3Q19 ? 2 : 1;
};

__host__ __device__ constexpr int pair_index(int i, int j) { return i + j - 1; }  // (0,1)->0 (0,2)->1 (1,2)->2

// Terms in units where the weights are the integers w36_a = 36 w_a (exact):
//   B_i = 3 rho u_i, P_ii = 9/2 rho u_i^2 = 3/2 B_i u_i, P_ij = 9 rho u_i u_j = 3 B_i u_j,
//   A = drho - 3/2 rho u.u = drho - (P_xx + P_yy + P_zz) / 3.
// Every constant that multiplies a first-order quantity (3, 3/2) is exact in
// binary, so no rounding bias enters the momentum; the sums are divided by 36
// only at the end (u' = M / (36 + R)).
template <int D, typename C>
__device__ __forceinline__ void make_terms(typename Pair<C>::P r, const typename Pair<C>::P (&u)[3],
                                           Terms<D, C>& t) {
  using O = Pair<C>;
  using P = typename O::P;
  const P g = O::fma(r, O::splat(C(3)), O::splat(C(3)));  // 3 (1 + drho)
  P Pd[3];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    t.B[i] = O::mul(g, u[i]);
    Pd[i] = O::mul(O::mul(t.B[i], u[i]), O::splat(C(1.5)));
  }
  P psum = O::add(Pd[0], Pd[1]);
  if (D == 3) psum = O::add(psum, Pd[2]);
  t.A = O::fma(psum, O::splat(C(-1.0 / 3.0)), r);
#pragma unroll
  for (int i = 0; i < D; ++i) t.S[i] = O::add(t.A, Pd[i]);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i + 1; j < D; ++j) {
      const int k = pair_index(i, j);
      const P pij = O::mul(O::mul(t.B[i], u[j]), O::splat(C(3)));
      const P base = O::add(t.S[i], Pd[j]);
      t.Ep[k] = O::add(base, pij);
      t.Em[k] = O::sub(base, pij);
      t.Op[k] = O::add(t.B[i], t.B[j]);
      t.Om[k] = O::sub(t.B[i], t.B[j]);
    }
  if (D == 3) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
      t.B2[i] = O::add(t.B[i], t.B[i]);
      t.S[i] = O::add(t.S[i], t.S[i]);  // S is used by the axis directions only
    }
  }
}

// Compile-time loop over directions: fn(std::integral_constant<int, a>) for
// a = I .. N - 1, so every direction-dependent choice below is an
// if constexpr on a constant.
template <int I, int N, typename Fn>
__device__ __forceinline__ void static_for(Fn&& fn) {
  if constexpr (I < N) {
    fn(std::integral_constant<int, I>{});
    static_for<I + 1, N>(fn);
  }
}

template <int LAT>
struct Dir {
  using L = Lattice<LAT>;
  __host__ __device__ static constexpr int nz(int a) {
    int n = 0;
    for (int i = 0; i < L::D; ++i) n += L::c(a, i) != 0 ? 1 : 0;
    return n;
  }
  __host__ __device__ static constexpr int first(int a) {
    for (int i = 0; i < L::D; ++i)
      if (L::c(a, i) != 0) return i;
    return 0;
  }
  __host__ __device__ static constexpr int second(int a) {
    int seen = 0;
    for (int i = 0; i < L::D; ++i)
      if (L::c(a, i) != 0) {
        if (seen) return i;
        seen = 1;
      }
    return 0;
  }
};

// T_a of both lanes
template <int LAT, typename C, int A>
__device__ __forceinline__ typename Pair<C>::P term(const Terms<Lattice<LAT>::D, C>& t) {
  using L = Lattice<LAT>;
  using O = Pair<C>;
  constexpr int nzc = Dir<LAT>::nz(A);
  constexpr int i0 = Dir<LAT>::first(A), i1 = Dir<LAT>::second(A);
  if constexpr (nzc == 0) {
    return t.A;
  } else if constexpr (nzc == 1) {
    // D3Q19: already doubled (AxisScale)
    if constexpr (LAT == kD3Q19) {
      if constexpr (L::c(A, i0) > 0) return O::add(t.S[i0], t.B2[i0]);
      else return O::sub(t.S[i0], t.B2[i0]);
    } else {
      if constexpr (L::c(A, i0) > 0) return O::add(t.S[i0], t.B[i0]);
      else return O::sub(t.S[i0], t.B[i0]);
    }
  } else {
    constexpr int k = pair_index(i0, i1);
    constexpr int s0 = L::c(A, i0), s1 = L::c(A, i1);
    if constexpr (s0 == s1) {
      if constexpr (s0 > 0) return O::add(t.Ep[k], t.Op[k]);
      else return O::sub(t.Ep[k], t.Op[k]);
    } else {
      if constexpr (s0 > 0) return O::add(t.Em[k], t.Om[k]);
      else return O::sub(t.Em[k], t.Om[k]);
    }
  }
}

// acc[0] += w36 T; acc[1 + i] += c_i w36 T (both lanes)
template <int LAT, typename C, int A>
__device__ __forceinline__ void accum(typename Pair<C>::P (&acc)[Lattice<LAT>::D + 1],
                                      typename Pair<C>::P T) {
  using L = Lattice<LAT>;
  using O = Pair<C>;
  constexpr int w = Dir<LAT>::nz(A) == 1 ? L::w36(A) / AxisScale<LAT>::value : L::w36(A);
  if constexpr (w == 1) acc[0] = O::add(acc[0], T);
  else acc[0] = O::fma(O::splat(C(w)), T, acc[0]);
  static_for<0, L::D>([&](auto I) {
    constexpr int i = decltype(I)::value;
    constexpr int c = L::c(A, i);
    if constexpr (c == 1) {
      if constexpr (w == 1) acc[1 + i] = O::add(acc[1 + i], T);
      else acc[1 + i] = O::fma(O::splat(C(w)), T, acc[1 + i]);
    } else if constexpr (c == -1) {
      if constexpr (w == 1) acc[1 + i] = O::sub(acc[1 + i], T);
      else acc[1 + i] = O::fma(O::splat(C(-w)), T, acc[1 + i]);
    }
  });
}

// the sums of the destination plane reached by c_z = FZ
template <int FZ, typename T>
__device__ __forceinline__ T& pick(T& prev, T& cur, T& next) {
  if constexpr (FZ == 1) return next;
  else if constexpr (FZ == 0) return cur;
  else return prev;
}

enum PlaneMode { kFirst = 0, kMid = 1, kLast = 2 };

template <int LAT, int MODE>
__device__ __forceinline__ constexpr bool mode_allows(int a) {
  return MODE == kMid || (MODE == kFirst && Frame<LAT>::fz(a) == 1) ||
         (MODE == kLast && Frame<LAT>::fz(a) == -1);
}

// Depth of the per-thread copy pipeline: planes in flight (global -> shared)
// while one plane is computed.
constexpr int kStages = 2;
// Exchange arrays: double buffered (one barrier per plane, twice the shared
// memory) or single buffered (two barriers per plane).
constexpr bool kDoubleBuffer = false;

// Shared-memory columns: BXC thread columns, then two seam columns holding
// lane-swapped copies: column BXC is read by thread 0 as its left neighbour
// (written by the last thread), column BXC + 1 by the last thread as its
// right neighbour (written by thread 0).
template <int BXC>
struct Cols {
  static constexpr int W = BXC + 2;
  static constexpr int SEAM_L = BXC;
  static constexpr int SEAM_R = BXC + 1;
};

// Per-thread shared-memory bases (pairs).  Xe: [NXS][RY][W]; Ye: [NYS][RY][2][W].
template <typename P>
struct SmemBase {
  P* x_own;        // Xe + r*W + tx
  const P* x_l;    // Xe + r*W + (left column: tx - 1, or SEAM_L for thread 0)
  const P* x_r;    // Xe + r*W + (right column: tx + 1, or SEAM_R for the last thread)
  P* x_sl;         // Xe + r*W + SEAM_L
  P* x_sr;         // Xe + r*W + SEAM_R
  P* y_own;        // Ye + r*2W + tx
  const P* y_l;
  const P* y_r;
  P* y_sl;
  P* y_sr;
  bool wl;         // this thread writes the SEAM_L copies (last thread of the row)
  bool wr;         // this thread writes the SEAM_R copies (thread 0)
  // the same bases in exchange buffer B (each buffer holds E pairs)
  template <int B, int E>
  __device__ __forceinline__ SmemBase buffer() const {
    SmemBase s = *this;
    if (B) {
      s.x_own += E; s.x_l += E; s.x_r += E; s.x_sl += E; s.x_sr += E;
      s.y_own += E; s.y_l += E; s.y_r += E; s.y_sl += E; s.y_sr += E;
    }
    return s;
  }
};

// A halo row (3D) only publishes the equilibria that move into the tile: those
// with c_y = FY.
template <int LAT, typename C, int MODE, int BXC, int RY, int FY>
__device__ __forceinline__ void halo_publish(const typename Pair<C>::P (&st)[Lattice<LAT>::D + 1][2],
                                             const SmemBase<typename Pair<C>::P>& sb) {
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int D = L::D;
  constexpr int W = Cols<BXC>::W;
  constexpr int YS = RY * 2 * W;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Terms<D, C> t;
    const P u[3] = {st[1][q], st[2][q], D == 3 ? st[3][q] : O::splat(C(0))};
    make_terms<D, C>(st[0][q], u, t);
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<LAT, MODE>(a) && F::ycross(a) && F::fy(a) == FY) {
        constexpr int fx = F::fx(a);
        const P T = term<LAT, C, a>(t);
        constexpr int off = F::yslot(a) * YS;
        sb.y_own[off + q * W] = T;
        if constexpr (fx == 1) {
          if (q == 1 && sb.wl) sb.y_sl[off + W] = O::swap(T);
        } else if constexpr (fx == -1) {
          if (q == 0 && sb.wr) sb.y_sr[off] = O::swap(T);
        }
      }
    });
  }
}

// One source plane: publish outgoing equilibria, gather incoming ones.
// st: the plane's state (field, pair); ap/ac/an: sums (pair, component) of
// destination planes p - 1, p, p + 1.
// role: 0 = interior row, 1 = lower halo row (publishes +y), 2 = upper halo row.
template <int LAT, typename C, int MODE, int BXC, int RY, int BUF>
__device__ __forceinline__ void plane_update(
    const typename Pair<C>::P (&st)[Lattice<LAT>::D + 1][2],
    typename Pair<C>::P (&ap)[2][Lattice<LAT>::D + 1], typename Pair<C>::P (&ac)[2][Lattice<LAT>::D + 1],
    typename Pair<C>::P (&an)[2][Lattice<LAT>::D + 1], const SmemBase<typename Pair<C>::P>& sb0,
    int role, bool active) {
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int D = L::D;
  constexpr int W = Cols<BXC>::W;
  constexpr int XS = RY * W;      // stride between x slots
  constexpr int YR = 2 * W;       // stride between rows of a y slot
  constexpr int YS = RY * YR;     // stride between y slots
  const SmemBase<P> sb = sb0.template buffer<kDoubleBuffer ? BUF : 0,
                                             Frame<LAT>::count_x() * RY * W +
                                                 Frame<LAT>::count_y() * RY * 2 * W>();
  if (active) {
    if (role == 0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        Terms<D, C> t;
        const P u[3] = {st[1][q], st[2][q], D == 3 ? st[3][q] : O::splat(C(0))};
        make_terms<D, C>(st[0][q], u, t);
        static_for<0, L::Q>([&](auto I) {
          constexpr int a = decltype(I)::value;
          if constexpr (mode_allows<LAT, MODE>(a)) {
            constexpr int fx = F::fx(a);
            const P T = term<LAT, C, a>(t);
            if constexpr (F::ycross(a)) {
              constexpr int off = F::yslot(a) * YS;
              sb.y_own[off + q * W] = T;
              // the lane-swapped copy read across the seam (diagonal directions)
              if constexpr (fx == 1) {
                if (q == 1 && sb.wl) sb.y_sl[off + W] = O::swap(T);
              } else if constexpr (fx == -1) {
                if (q == 0 && sb.wr) sb.y_sr[off] = O::swap(T);
              }
            } else {
              constexpr int fz = F::fz(a);
              // destination pair within the thread: a -> b for +x, b -> a for -x
              const int qd = q + fx;
              if (qd >= 0 && qd < 2) {
                accum<LAT, C, a>(pick<fz>(ap, ac, an)[qd], T);
              } else {
                constexpr int off = F::xslot(a) * XS;
                sb.x_own[off] = T;
                if constexpr (fx == 1) {
                  if (sb.wl) sb.x_sl[off] = O::swap(T);
                } else {
                  if (sb.wr) sb.x_sr[off] = O::swap(T);
                }
              }
            }
          }
        });
      }
    } else if (D == 3 && role == 1) {
      halo_publish<LAT, C, MODE, BXC, RY, 1>(st, sb);
    } else if (D == 3 && role == 2) {
      halo_publish<LAT, C, MODE, BXC, RY, -1>(st, sb);
    }
  }
  __syncthreads();
  if (active && role == 0) {
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<LAT, MODE>(a)) {
        constexpr int fz = F::fz(a);
        constexpr int fx = F::fx(a);
        auto& dst = pick<fz>(ap, ac, an);
        if constexpr (F::xcross(a)) {
          // +x: pair a receives the left neighbour's pair b; -x: pair b gets the right one's a
          constexpr int off = F::xslot(a) * XS;
          if constexpr (fx == 1) accum<LAT, C, a>(dst[0], sb.x_l[off]);
          else accum<LAT, C, a>(dst[1], sb.x_r[off]);
        } else if constexpr (F::ycross(a)) {
          constexpr int off = F::yslot(a) * YS - F::fy(a) * YR;  // source row r - fy
          if constexpr (fx == 0) {
            accum<LAT, C, a>(dst[0], sb.y_own[off]);
            accum<LAT, C, a>(dst[1], sb.y_own[off + W]);
          } else if constexpr (fx == 1) {
            accum<LAT, C, a>(dst[0], sb.y_l[off + W]);   // left neighbour's pair b
            accum<LAT, C, a>(dst[1], sb.y_own[off]);     // own pair a
          } else {
            accum<LAT, C, a>(dst[0], sb.y_own[off + W]); // own pair b
            accum<LAT, C, a>(dst[1], sb.y_r[off]);       // right neighbour's pair a
          }
        }
      }
    });
  }
  if constexpr (!kDoubleBuffer) __syncthreads();
}

// fp: per-field pointers at the thread's quad of plane 0; mrow: the node-type
// mask at the same quad; off: offset of the destination plane.  Lane order of
// the quad: (a.x, a.y, b.x, b.y) = nodes (x0, x0 + H, x0 + 1, x0 + 1 + H).
template <int LAT, typename S>
__device__ __forceinline__ void store_plane(S* const (&fp)[4], const uint8_t* mrow,
                                            const TiledArgs& ta, int64_t off, bool x_lo_wall,
                                            bool x_hi_wall, bool skip,
                                            typename Quad<S>::P (&acc)[2][Lattice<LAT>::D + 1],
                                            const typename Quad<S>::P (&force)[3]) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int D = Lattice<LAT>::D;
  if (skip) return;
  bool wall[4] = {x_lo_wall, false, false, x_hi_wall};
  bool any = x_lo_wall || x_hi_wall;
  if (ta.wall_mode == kWallMask) {
    const uchar4 m = *reinterpret_cast<const uchar4*>(mrow + off);
    wall[0] = m.x != 0; wall[1] = m.y != 0; wall[2] = m.z != 0; wall[3] = m.w != 0;
    any = wall[0] || wall[1] || wall[2] || wall[3];
  }
  P v[D + 1][2];
  // sums are 36 x (drho', m'): u' = m' / (1 + drho') = M / (36 + R)
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const P inv = O::rcp(O::add(O::splat(C(36)), acc[q][0]));
    v[0][q] = O::mul(acc[q][0], O::splat(C(1.0 / 36.0)));
#pragma unroll
    for (int i = 0; i < D; ++i) v[1 + i][q] = O::fma(acc[q][1 + i], inv, force[i]);
  }
  if (!any) {
#pragma unroll
    for (int f = 0; f <= D; ++f) Quad<S>::st(fp[f] + off, v[f][0], v[f][1]);
  } else {
#pragma unroll
    for (int f = 0; f <= D; ++f) {
      if (!wall[0]) Quad<S>::st1(fp[f] + off + 0, v[f][0].x);
      if (!wall[1]) Quad<S>::st1(fp[f] + off + 1, v[f][0].y);
      if (!wall[2]) Quad<S>::st1(fp[f] + off + 2, v[f][1].x);
      if (!wall[3]) Quad<S>::st1(fp[f] + off + 3, v[f][1].y);
    }
  }
}


// Bytes of shared memory one block uses: exchange arrays (pairs) then the
// stage buffers [kStages][K][RY][BXC] of 4-value quads.
template <int LAT, typename S, int BXC, int RY>
__host__ __device__ constexpr size_t tiled_exchange_bytes() {
  return (kDoubleBuffer ? 2 : 1) * sizeof(typename Quad<S>::P) * (size_t)RY * (BXC + 2) *
         (Frame<LAT>::count_x() + 2 * Frame<LAT>::count_y());
}
template <int LAT, typename S, int BXC, int RY>
__host__ __device__ constexpr size_t tiled_smem_bytes() {
  return ((tiled_exchange_bytes<LAT, S, BXC, RY>() + 15) / 16) * 16 +
         (size_t)kStages * (Lattice<LAT>::D + 1) * RY * BXC * Quad<S>::BYTES;
}

// Resident blocks per SM asked of the register allocator, matched to what the
// shared-memory footprint allows.
template <int BXC, int RY>
struct TiledMinBlocks {
  static constexpr int value =
      (BXC * RY) >= 512 ? 1 : (kDoubleBuffer ? 2 : ((BXC * RY) <= 192 ? 3 : 512 / (BXC * RY)));
};

template <int LAT, typename S, int BXC, int RY>
__global__ void __launch_bounds__(BXC * RY, TiledMinBlocks<BXC, RY>::value)
    step_tiled(TiledArgs ta, const S* __restrict__ in, S* __restrict__ out) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<LAT>;
  using F = Frame<LAT>;
  constexpr int D = L::D;
  constexpr int K = D + 1;
  constexpr int W = Cols<BXC>::W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();  // the previous step's writes are visible from here on
  pdl_launch_next();
  const int tx = threadIdx.x, r = threadIdx.y;
  const int bxr = ta.nx >> 2;                  // threads per row actually used
  const bool active = tx < bxr;
  P* Xe = reinterpret_cast<P*>(smem_raw);
  P* Ye = Xe + F::count_x() * RY * W;
  const int col_l = tx == 0 ? Cols<BXC>::SEAM_L : tx - 1;
  const int col_r = tx == bxr - 1 ? Cols<BXC>::SEAM_R : tx + 1;
  SmemBase<P> sb;
  sb.wl = tx == bxr - 1;
  sb.wr = tx == 0;
  sb.x_own = Xe + r * W + tx;
  sb.x_l = Xe + r * W + col_l;
  sb.x_r = Xe + r * W + col_r;
  sb.x_sl = Xe + r * W + Cols<BXC>::SEAM_L;
  sb.x_sr = Xe + r * W + Cols<BXC>::SEAM_R;
  sb.y_own = Ye + r * 2 * W + tx;
  sb.y_l = Ye + r * 2 * W + col_l;
  sb.y_r = Ye + r * 2 * W + col_r;
  sb.y_sl = Ye + r * 2 * W + Cols<BXC>::SEAM_L;
  sb.y_sr = Ye + r * 2 * W + Cols<BXC>::SEAM_R;

  // in-plane row (3D) of this thread and its role
  int row = 0, row_mem = 0, role = 0;
  bool row_exists = true;
  if (D == 3) {
    row = blockIdx.y * ta.ty + r - 1;
    role = r == 0 ? 1 : (r == RY - 1 ? 2 : 0);
    if (role == 0 && row >= ta.ny) role = 3;  // beyond a ragged last tile: idle
    row_mem = row;
    if (row < 0 || row >= ta.ny) {
      if (ta.py) row_mem = (row + ta.ny) % ta.ny;
      else row_exists = false;
    }
  }
  const bool row_wall = D == 3 && !ta.py && (row == 0 || row == ta.ny - 1);
  const int64_t row_off = (int64_t)row_mem * ta.nx + 4 * tx;
  const bool loads = active && row_exists && role != 3;
  // box walls at x = 0 (lane a.x of thread 0) and x = nx - 1 (lane b.y of the last)
  const bool x_lo_wall = ta.wall_mode == kWallBox && !ta.px && tx == 0;
  const bool x_hi_wall = ta.wall_mode == kWallBox && !ta.px && tx == bxr - 1;

  const S* ip[4];
  S* op[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    ip[f] = in + (int64_t)f * ta.n + row_off;
    op[f] = out + (int64_t)f * ta.n + row_off;
  }
  const uint8_t* mrow = ta.wall_mode == kWallMask ? ta.mask + row_off : nullptr;
  P force[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) force[i] = O::splat(C(ta.force[i]));

  // chunk c of nzc covers planes [c * nplanes / nzc, (c + 1) * nplanes / nzc)
  const int z0 = (int)(((int64_t)blockIdx.x * ta.nplanes) / ta.nzc);
  const int z1 = (int)(((int64_t)(blockIdx.x + 1) * ta.nplanes) / ta.nzc);
  const int64_t ps = ta.plane_stride;
  auto plane_exists = [&](int p) { return (p >= 0 && p < ta.nplanes) || ta.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + ta.nplanes : (p >= ta.nplanes ? p - ta.nplanes : p); };
  auto store_skip = [&](int q) {
    return role != 0 || !active || row_wall || (!ta.pz && (q == 0 || q == ta.nplanes - 1));
  };

  // stage buffers: thread's own quad of field f for plane slot k at
  // stage_base + (k * K + f) * RY * BXC quads
  constexpr int QW = Quad<S>::BYTES;
  constexpr uint32_t kFieldStride = RY * BXC * QW;
  constexpr uint32_t kSlotStride = K * kFieldStride;
  S* stage_gen = reinterpret_cast<S*>(smem_raw + ((tiled_exchange_bytes<LAT, S, BXC, RY>() + 15) / 16) * 16 +
                                      (size_t)(r * BXC + tx) * QW);
  const uint32_t stage_sh = (uint32_t)__cvta_generic_to_shared(stage_gen);
  const int np = z1 - z0 + 2;  // planes z0 - 1 .. z1
  auto fetch = [&](int i) {    // start copying plane z0 - 1 + i into its stage
    const int p = z0 - 1 + i;
    if (i < np && loads && plane_exists(p)) {
      const int64_t off = (int64_t)plane_mem(p) * ps;
      const uint32_t sh = stage_sh + (uint32_t)(i & (kStages - 1)) * kSlotStride;
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<S>::copy(sh + f * kFieldStride, ip[f] + off);
    }
    cp_async_commit();
  };
  P st[K][2];
  auto take = [&](int i) {     // wait for plane z0 - 1 + i and read it
    cp_async_wait<kStages - 1>();
    const int p = z0 - 1 + i;
    const bool ok = loads && plane_exists(p);
    const unsigned char* base = reinterpret_cast<const unsigned char*>(stage_gen) +
                                (size_t)(i & (kStages - 1)) * kSlotStride;
#pragma unroll
    for (int f = 0; f < K; ++f) {
      if (ok) {
        Quad<S>::lds(reinterpret_cast<const S*>(base + f * kFieldStride), st[f][0], st[f][1]);
      } else {
        st[f][0] = P{0, 0};
        st[f][1] = P{0, 0};
      }
    }
  };

  P R0[2][K], R1[2][K], R2[2][K];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < K; ++k) R0[q][k] = R1[q][k] = R2[q][k] = O::splat(C(0));

#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) fetch(i);
  // first (halo) plane z0 - 1 (plane index 0, buffer 0): only the equilibria
  // moving up the march axis, into destination plane z0 = R1 of the first step
  fetch(kStages - 1);
  take(0);
  if (plane_exists(z0 - 1))
    plane_update<LAT, C, kFirst, BXC, RY, 0>(st, R0, R2, R1, sb, role, active);

  // full plane p (plane index i = p - z0 + 1, buffer i & 1): contributions to
  // the sums A (dest p - 1), B (dest p), N (dest p + 1); then A is complete.
  auto step = [&](const int buf, int p, P(&A)[2][K], P(&B)[2][K], P(&N)[2][K]) {
    const int i = p - z0 + 1;
    fetch(i + kStages - 1);
    take(i);
    if (buf) plane_update<LAT, C, kMid, BXC, RY, 1>(st, A, B, N, sb, role, active);
    else plane_update<LAT, C, kMid, BXC, RY, 0>(st, A, B, N, sb, role, active);
    if (p - 1 >= z0)
      store_plane<LAT, S>(op, mrow, ta, (int64_t)(p - 1) * ps, x_lo_wall, x_hi_wall,
                          store_skip(p - 1), A, force);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) A[q][k] = O::splat(C(0));
  };
  // last (halo) plane z1: only the equilibria moving down, into plane z1 - 1 (= B)
  auto last = [&](const int buf, P(&B)[2][K]) {
    const int i = np - 1;
    fetch(i + kStages - 1);
    take(i);
    if (plane_exists(z1)) {
      if (buf) plane_update<LAT, C, kLast, BXC, RY, 1>(st, B, R0, R0, sb, role, active);
      else plane_update<LAT, C, kLast, BXC, RY, 0>(st, B, R0, R0, sb, role, active);
    }
    store_plane<LAT, S>(op, mrow, ta, (int64_t)(z1 - 1) * ps, x_lo_wall, x_hi_wall,
                        store_skip(z1 - 1), B, force);
  };
  // roles rotate with period 3 (and, double buffered, the exchange arrays alternate)
  if constexpr (kDoubleBuffer) {
    for (int p = z0;; p += 6) {
      step(1, p, R0, R1, R2);
      if (p + 1 >= z1) { last(0, R1); break; }
      step(0, p + 1, R1, R2, R0);
      if (p + 2 >= z1) { last(1, R2); break; }
      step(1, p + 2, R2, R0, R1);
      if (p + 3 >= z1) { last(0, R0); break; }
      step(0, p + 3, R0, R1, R2);
      if (p + 4 >= z1) { last(1, R1); break; }
      step(1, p + 4, R1, R2, R0);
      if (p + 5 >= z1) { last(0, R2); break; }
      step(0, p + 5, R2, R0, R1);
      if (p + 6 >= z1) { last(1, R0); break; }
    }
  } else {  // one exchange array: unroll by 3 only (half the code of the loop above)
    for (int p = z0;; p += 3) {
      step(0, p, R0, R1, R2);
      if (p + 1 >= z1) { last(0, R1); break; }
      step(0, p + 1, R1, R2, R0);
      if (p + 2 >= z1) { last(0, R2); break; }
      step(0, p + 2, R2, R0, R1);
      if (p + 3 >= z1) { last(0, R0); break; }
    }
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------ launch

struct TiledShape {
  int bxc, ry, ty, tz;
  size_t smem;
};

// Launch one instance; explicit instantiations live in step_tiled_*.cu.
template <int LAT, typename S, int BXC, int RY>
cudaError_t launch_shape(const TiledArgs& ta, const TiledShape& s, const void* in, void* out,
                         cudaStream_t stream, dim3 grid);

#define MACLAB_TILED_LAUNCH_DEF                                                               \
  template <int LAT, typename S, int BXC, int RY>                                             \
  cudaError_t launch_shape(const TiledArgs& ta, const TiledShape& s, const void* in,          \
                           void* out, cudaStream_t stream, dim3 grid) {                       \
    auto kern = step_tiled<LAT, S, BXC, RY>;                                                  \
    constexpr size_t smem = tiled_smem_bytes<LAT, S, BXC, RY>();                              \
    (void)s;                                                                                  \
    if (smem > 48 * 1024) {                                                                   \
      cudaError_t e =                                                                         \
          cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                         \
    }                                                                                         \
    return launch_kernel(kern, grid, dim3(BXC, RY), smem, stream, ta.overlap, ta,            \
                         static_cast<const S*>(in), static_cast<S*>(out));                    \
  }

#define MACLAB_TILED_INST(LAT, S, BXC, RY)                                                     \
  template cudaError_t launch_shape<LAT, S, BXC, RY>(const TiledArgs&, const TiledShape&,     \
                                                     const void*, void*, cudaStream_t, dim3);

}  // namespace maclab
