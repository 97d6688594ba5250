// adjoint.cu -- reverse mode of one MacLAB step, and the gradient assembly.
//
// Forward step (step.cu): for a fluid node x, rho'(x) = sum_a F_a(x - c_a),
// m'(x) = sum_a c_a F_a(x - c_a), u'(x) = m' / rho' + force, with
// F_a = f_a^eq(rho, u) of Eq. (2); wall nodes keep their values.  Given the
// adjoints (lam_rho', lam_u') of the outputs, the chain rule gives, for fluid x,
//   L_r(x) = lam_rho'(x) - lam_u'(x) . (u'(x) - force) / rho'(x)   (dL/drho' through both outputs)
//   L_m(x) = lam_u'(x) / rho'(x)                                    (dL/dm')
// and every source y receives from each downstream fluid node x = y + c_a the
// weight g_a = L_r(x) + c_a . L_m(x) of dF_a/d(rho, u) at y.  With the moments
// G0 = sum_a w_a g_a, G1 = sum_a w_a g_a c_a, G2 = sum_a w_a g_a c_a c_a^T and
// dF_a/drho = w_a (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
// dF_a/du   = w_a rho (3 c + 9 (c.u) c - 3 u),
//   lam_rho(y) = G0 (1 - 3/2 u.u) + 3 u.G1 + 9/2 u^T G2 u
//   lam_u(y)   = rho (3 G1 + 9 G2 u - 3 u G0).
// A wall node's output equals its input, so its lam' is passed straight
// through.  d(output)/d(force) is the identity on fluid nodes, so the force
// gradient is the sum of lam_u' over fluid nodes.
//
// Two kernels: adj_lambda forms (L_r, L_m) at every node (zero at walls) into a
// scratch array of one 4-value record per node (L_r, L_m x, L_m y, L_m z), so
// that adj_gather reads each downstream neighbour with one vector load.  Arithmetic in FP64
// for FP64 storage, FP32 otherwise; adjoint arrays are in that arithmetic
// type, in the library's storage order.

#include "common.cuh"
#include "lattice.cuh"

namespace maclab {

template <int LAT>
__device__ __forceinline__ bool wall_at(const Geometry& g, int x, int y, int z, int64_t m) {
  if (g.wall_mode == kWallNone) return false;
  if (g.wall_mode == kWallMask) return g.mask[m] != 0;
  bool w = false;
  if (!(g.periodic & 1u)) w |= (x == 0) | (x == g.nx - 1);
  if (!(g.periodic & 2u)) w |= (y == 0) | (y == g.ny - 1);
  if (Lattice<LAT>::D == 3 && !(g.periodic & 4u)) w |= (z == 0) | (z == g.nz - 1);
  return w;
}

// one 4-value record (16 bytes in FP32, 32 in FP64) read with vector loads
template <typename C>
struct Rec4;
template <>
struct Rec4<float> {
  __device__ __forceinline__ static void ld(const float* p, float (&r)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&r)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  }
};
template <>
struct Rec4<double> {
  __device__ __forceinline__ static void ld(const double* p, double (&r)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  }
  __device__ __forceinline__ static void st(double* p, const double (&r)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(r[2], r[3]);
  }
};

template <int LAT, typename S>
__global__ void __launch_bounds__(256) adj_lambda(Geometry g, const S* __restrict__ out_state,
                                                  const typename Store<S>::C* __restrict__ lam1,
                                                  typename Store<S>::C* __restrict__ Lam,
                                                  double f0, double f1, double f2,
                                                  double* __restrict__ grad_force) {
  using C = typename Store<S>::C;
  constexpr int D = Lattice<LAT>::D;
  const int64_t N = g.n;
  const C force[3] = {C(f0), C(f1), C(f2)};
  double gf[3] = {0.0, 0.0, 0.0};
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < N;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int x = log_x(g, (int)(m % g.nx));
    const int y = (int)((m / g.nx) % g.ny);
    const int z = (int)(m / ((int64_t)g.nx * g.ny));
    C rec[4] = {C(0), C(0), C(0), C(0)};
    if (!wall_at<LAT>(g, x, y, z, m)) {
      const C rho = C(1) + (C)Store<S>::from(out_state[m]);
      const C inv = C(1) / rho;
      C lr = lam1[m];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const C lu = lam1[(1 + i) * N + m];
        const C um = (C)Store<S>::from(out_state[(1 + i) * N + m]) - force[i];  // m' / rho'
        lr -= lu * um * inv;
        rec[1 + i] = lu * inv;
        gf[i] += (double)lu;
      }
      rec[0] = lr;
    }
    Rec4<C>::st(Lam + 4 * m, rec);
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

template <int LAT, typename S>
__global__ void __launch_bounds__(256) adj_gather(Geometry g, const S* __restrict__ in_state,
                                                  const typename Store<S>::C* __restrict__ lam1,
                                                  const typename Store<S>::C* __restrict__ Lam,
                                                  typename Store<S>::C* __restrict__ lam0) {
  using C = typename Store<S>::C;
  using L = Lattice<LAT>;
  constexpr int D = L::D;
  const int64_t N = g.n;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < N;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int x = log_x(g, (int)(m % g.nx));
    const int y = (int)((m / g.nx) % g.ny);
    const int z = (int)(m / ((int64_t)g.nx * g.ny));
    C G0 = 0, G1[3] = {0, 0, 0}, G2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      // downstream node x + c_a (it gathered F_a from this node)
      int xs = x + L::c(a, 0), ys = y + L::c(a, 1), zs = D == 3 ? z + L::c(a, 2) : 0;
      if (xs < 0 || xs >= g.nx) {
        if (!(g.periodic & 1u)) continue;
        xs = xs < 0 ? xs + g.nx : xs - g.nx;
      }
      if (ys < 0 || ys >= g.ny) {
        if (!(g.periodic & 2u)) continue;
        ys = ys < 0 ? ys + g.ny : ys - g.ny;
      }
      if (D == 3 && (zs < 0 || zs >= g.nz)) {
        if (!(g.periodic & 4u)) continue;
        zs = zs < 0 ? zs + g.nz : zs - g.nz;
      }
      const int64_t s = ((int64_t)zs * g.ny + ys) * g.nx + mem_x(g, xs);
      C rec[4];
      Rec4<C>::ld(Lam + 4 * s, rec);
      C ga = rec[0];
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (L::c(a, i) != 0) ga += C(L::c(a, i)) * rec[1 + i];
      const C wg = ga * (C(L::w36(a)) / C(36));
      G0 += wg;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (L::c(a, i) == 0) continue;
        G1[i] += C(L::c(a, i)) * wg;
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (L::c(a, j) != 0) G2[i][j] += C(L::c(a, i) * L::c(a, j)) * wg;
      }
    }
    const C rho = C(1) + (C)Store<S>::from(in_state[m]);
    C u[3] = {0, 0, 0};
    C uu = 0, uG1 = 0, uG2u = 0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      u[i] = (C)Store<S>::from(in_state[(1 + i) * N + m]);
      uu += u[i] * u[i];
      uG1 += u[i] * G1[i];
    }
    C G2u[3] = {0, 0, 0};
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int j = 0; j < D; ++j) G2u[i] += G2[i][j] * u[j];
      uG2u += u[i] * G2u[i];
    }
    C lr = G0 * (C(1) - C(1.5) * uu) + C(3) * uG1 + C(4.5) * uG2u;
    C lu[3];
#pragma unroll
    for (int i = 0; i < D; ++i) lu[i] = rho * (C(3) * G1[i] + C(9) * G2u[i] - C(3) * u[i] * G0);
    if (wall_at<LAT>(g, x, y, z, m)) {  // identity pass-through of a wall node's output
      lr += lam1[m];
#pragma unroll
      for (int i = 0; i < D; ++i) lu[i] += lam1[(1 + i) * N + m];
    }
    lam0[m] = lr;
#pragma unroll
    for (int i = 0; i < D; ++i) lam0[(1 + i) * N + m] = lu[i];
  }
}

// ------------------------------------------------------------------ the viscosity term
//
// nu enters a rollout only through e = 6 nu / dx (Eq. (6)): the initial and
// wall velocities are u / e in lattice units, the force increment is
// g dt / e = g dx / e^2, the output is u = e ut, and the lattice update itself
// does not depend on e.  With the tangent tau_n = e d(state_n)/de and
// s_n = tau_n + (0, ut_n) (zero at t = 0 and on wall nodes), s follows
// s_(n+1) = J_n s_n + D_n with the defect of one step at a fluid node
//   D_n^u   = ut'_nf - J (0, ut) |_u - F,        D_n^drho = -J (0, ut) |_drho,
// where ut'_nf = m' / rho' is the step's output without the force F and
// J (0, ut) the step's derivative along ut scaled by (1 + eps):
//   dF_a = w_a rho (3 c.u + 9 (c.u)^2 - 3 u.u),  drho' = sum dF_a,
//   dut' = (sum c dF_a - ut'_nf drho') / rho'.
// Then e dL/de = lam_T . s_T = sum_n sum_x lam_(n+1)(x) . D_n(x): every term is
// formed directly (ut'_nf - dut' = (m' - dm') / rho' + ut'_nf drho' / rho', with
// m' - dm' = sum c w rho (1 - 9/2 (c.u)^2 + 3/2 u.u)), not as the difference of
// the end-point products lam_T . ut_T and lam_0 . ut_0, which nearly cancel.
// Sums use the integer weights 36 w_a and drop their constant parts exactly
// (sum 36 w_a = 36, sum 36 w_a c_a = 0).
// Running sum of one thread: FP64 for FP64 storage; float-float (Knuth's
// two-sum, the error of every FP32 addition kept in lo) otherwise, so the
// per-node terms, formed in FP32, are added without FP64 arithmetic.
template <typename C>
struct NuAcc {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct NuAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// One thread per node along the grid stride; the node's storage coordinates
// advance with the stride (no division per node), and the storage offsets of
// its 3 x 3 x 3 upstream neighbourhood are formed once per node.
template <int LAT, typename S>
__global__ void __launch_bounds__(256) adj_nu_term(Geometry g, const S* __restrict__ state,
                                                   const typename Store<S>::C* __restrict__ lam1,
                                                   double f0, double f1, double f2,
                                                   double* __restrict__ acc) {
  using C = typename Store<S>::C;
  using L = Lattice<LAT>;
  constexpr int D = L::D;
  const int64_t N = g.n;
  const C force[3] = {C(f0), C(f1), C(f2)};
  NuAcc<C> sum;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int mx, y, sx, sy;
  int64_t z, sz;
  if (N < (int64_t)INT32_MAX && stride < (int64_t)INT32_MAX) {
    const unsigned nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned m32 = (unsigned)(m < N ? m : 0), q32 = m32 / nx, s32 = (unsigned)stride, sq32 = s32 / nx;
    mx = (int)(m32 - q32 * nx);
    y = (int)(q32 % ny);
    z = q32 / ny;
    sx = (int)(s32 - sq32 * nx);
    sy = (int)(sq32 % ny);
    sz = sq32 / ny;
  } else {
    const int64_t q = m / g.nx, sq = stride / g.nx;
    mx = (int)(m - q * g.nx);
    y = (int)(q % g.ny);
    z = q / g.ny;
    sx = (int)(stride - sq * g.nx);
    sy = (int)(sq % g.ny);
    sz = sq / g.ny;
  }
  const int64_t plane = (int64_t)g.nx * g.ny;
  for (; m < N; m += stride) {
    const int x = log_x(g, mx);
    const int yy = y;
    const int64_t zz = z;
    mx += sx;
    const int carry = mx >= g.nx ? 1 : 0;
    mx -= carry * g.nx;
    y += sy + carry;
    if (y >= g.ny) {
      y -= g.ny;
      z += 1;
    }
    z += sz;
    if (wall_at<LAT>(g, x, yy, (int)zz, m)) continue;
    // storage offsets of the source x - c: index k = c + 1 along each axis
    int xo[3];
    int64_t yo[3], zo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int xs = x - (k - 1), ys = yy - (k - 1);
      xs = xs < 0 ? xs + g.nx : (xs >= g.nx ? xs - g.nx : xs);
      ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
      xo[k] = mem_x(g, xs);
      yo[k] = (int64_t)ys * g.nx;
      int64_t zs = zz;
      if (D == 3) {
        zs = zz - (k - 1);
        zs = zs < 0 ? zs + g.nz : (zs >= g.nz ? zs - g.nz : zs);
      }
      zo[k] = zs * plane;
    }
    C R = 0, dR = 0, M[3] = {0, 0, 0}, Md[3] = {0, 0, 0};  // all x 36
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      const int64_t sidx = zo[(D == 3 ? L::c(a, 2) : 0) + 1] + yo[L::c(a, 1) + 1] + xo[L::c(a, 0) + 1];
      const C dr = (C)Store<S>::from(state[sidx]);
      const C rho = C(1) + dr;
      C cu = 0, uu = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const C u = (C)Store<S>::from(state[(1 + i) * N + sidx]);
        cu += C(L::c(a, i)) * u;
        uu += u * u;
      }
      const C w = C(L::w36(a));
      const C p = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;   // f = w rho (1 + p)
      const C q = C(1.5) * uu - C(4.5) * cu * cu;               // f - df = w rho (1 + q)
      const C fv = w * (dr + rho * p);                          // f - w (the constant part)
      const C gv = w * (dr + rho * q);                          // f - df - w
      R += fv;
      dR += w * rho * (C(3) * cu + C(9) * cu * cu - C(3) * uu);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        if (L::c(a, i) == 0) continue;
        M[i] += C(L::c(a, i)) * fv;
        Md[i] += C(L::c(a, i)) * gv;
      }
    }
    const C R36 = C(36) + R;                 // 36 rho'
    C t = -lam1[m] * (dR / C(36));
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const C unf = M[i] / R36;              // m' / rho'
      const C du = Md[i] / R36 + unf * (dR / R36) - force[i];
      t += lam1[(1 + i) * N + m] * du;
    }
    sum.add(t);
  }
  // block sum: warp shuffles, one value per warp, one FP64 atomic per block
  double v = sum.value();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s2 += red[w];
    atomicAdd(acc, s2);
  }
}

// Blocks of the viscosity-term kernel: four 256-thread blocks per SM at most.
static unsigned nu_blocks(int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  int64_t b = (n + 255) / 256;
  if (b > 4 * sms) b = 4 * sms;
  return (unsigned)(b < 1 ? 1 : b);
}

static unsigned grid256(int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  int64_t b = (n + 255) / 256;
  if (b > 8 * sms) b = 8 * sms;
  return (unsigned)(b < 1 ? 1 : b);
}

template <int LAT, typename S>
static cudaError_t adjoint_t(const Geometry& g, const void* sn, const void* sn1, const void* lam1,
                             void* lam0, void* scratch, const double* force, double* gf,
                             cudaStream_t st) {
  using C = typename Store<S>::C;
  adj_lambda<LAT, S><<<grid256(g.n), 256, 0, st>>>(g, (const S*)sn1, (const C*)lam1, (C*)scratch,
                                                   force[0], force[1], force[2], gf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_gather<LAT, S><<<grid256(g.n), 256, 0, st>>>(g, (const S*)sn, (const C*)lam1,
                                                   (const C*)scratch, (C*)lam0);
  return cudaGetLastError();
}

template <int LAT>
static cudaError_t adjoint_lat(const Geometry& g, int precision, const void* sn, const void* sn1,
                               const void* lam1, void* lam0, void* scratch, const double* force,
                               double* gf, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return adjoint_t<LAT, double>(g, sn, sn1, lam1, lam0, scratch, force, gf, st);
    case MACLAB_F32: return adjoint_t<LAT, float>(g, sn, sn1, lam1, lam0, scratch, force, gf, st);
    case MACLAB_BF16_STORE:
      return adjoint_t<LAT, __nv_bfloat16>(g, sn, sn1, lam1, lam0, scratch, force, gf, st);
    case MACLAB_F16_STORE: return adjoint_t<LAT, __half>(g, sn, sn1, lam1, lam0, scratch, force, gf, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_step(const Geometry& g, int precision, const void* state_n,
                                const void* state_np1, const void* lam_np1, void* lam_n,
                                void* scratch, const double force_lat[3], double* grad_force,
                                cudaStream_t st) {
  return g.lattice == kD2Q9
             ? adjoint_lat<kD2Q9>(g, precision, state_n, state_np1, lam_np1, lam_n, scratch,
                                  force_lat, grad_force, st)
             : adjoint_lat<kD3Q19>(g, precision, state_n, state_np1, lam_np1, lam_n, scratch,
                                   force_lat, grad_force, st);
}

template <int LAT>
static cudaError_t nu_term_lat(const Geometry& g, int precision, const void* sn, const void* lam1,
                               const double* f, double* acc, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64:
      adj_nu_term<LAT, double><<<nu_blocks(g.n), 256, 0, st>>>(g, (const double*)sn, (const double*)lam1, f[0], f[1],
                                                            f[2], acc);
      break;
    case MACLAB_F32:
      adj_nu_term<LAT, float><<<nu_blocks(g.n), 256, 0, st>>>(g, (const float*)sn, (const float*)lam1, f[0], f[1],
                                                           f[2], acc);
      break;
    case MACLAB_BF16_STORE:
      adj_nu_term<LAT, __nv_bfloat16><<<nu_blocks(g.n), 256, 0, st>>>(g, (const __nv_bfloat16*)sn, (const float*)lam1,
                                                                   f[0], f[1], f[2], acc);
      break;
    case MACLAB_F16_STORE:
      adj_nu_term<LAT, __half><<<nu_blocks(g.n), 256, 0, st>>>(g, (const __half*)sn, (const float*)lam1, f[0], f[1],
                                                            f[2], acc);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_nu_term(const Geometry& g, int precision, const void* state_n, const void* lam_np1,
                                   const double force_lat[3], double* acc, cudaStream_t st) {
  return g.lattice == kD2Q9 ? nu_term_lat<kD2Q9>(g, precision, state_n, lam_np1, force_lat, acc, st)
                            : nu_term_lat<kD3Q19>(g, precision, state_n, lam_np1, force_lat, acc, st);
}

// ------------------------------------------------------------------ seeds and gradients
//
// Physical output gradients (logical order) -> adjoint of the stored state
// (storage order): rho = rho0 (1 + drho) and u = e ut, so dL/ddrho = rho0 dL/drho
// and dL/dut = e dL/du.  Also sums lam_ut . ut over all nodes (the output's
// dependence on e, for dL/de).
template <typename S, typename T>
__global__ void adj_seed(Geometry g, const T* __restrict__ grho, const T* __restrict__ gu,
                         const S* __restrict__ state, double rho0, double e,
                         typename Store<S>::C* __restrict__ lam, double* __restrict__ dot) {
  using C = typename Store<S>::C;
  const int64_t N = g.n;
  double acc = 0.0;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < N;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = m / g.nx;
    const int64_t j = row * g.nx + log_x(g, (int)(m - row * g.nx));
    lam[m] = grho ? C(rho0 * (double)grho[j]) : C(0);
    for (int i = 0; i < g.d; ++i) {
      const double l = gu ? e * (double)gu[i * N + j] : 0.0;
      lam[(1 + i) * N + m] = C(l);
      acc += l * (double)Store<S>::from(state[(1 + i) * N + m]);
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(dot, red[0]);
}

// Adjoint of the initial stored state -> gradients of the physical inputs.
// Fluid nodes: dL/drho0 = lam_drho / rho0, dL/du0 = lam_ut / e (logical order);
// wall nodes get 0 there (their initial values come from the wall tables) and
// their adjoint is summed per wall id into wall[k * 4 + (0: rho, 1..3: u)].
// dot += sum over all nodes of lam_ut . ut (the inputs' dependence on e).
template <typename S, typename T>
__global__ void adj_finish(Geometry g, const typename Store<S>::C* __restrict__ lam,
                           const S* __restrict__ state, const uint8_t* __restrict__ node_type,
                           int n_wall_ids, double rho0, double e, T* __restrict__ grho,
                           T* __restrict__ gu, double* __restrict__ wall, double* __restrict__ dot) {
  const int64_t N = g.n;
  double acc = 0.0;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < N;
       m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = m / g.nx;
    const int64_t j = row * g.nx + log_x(g, (int)(m - row * g.nx));
    const int k = node_type ? (int)node_type[m] : 0;
    const double lr = (double)lam[m];
    for (int i = 0; i < g.d; ++i)
      acc += (double)lam[(1 + i) * N + m] * (double)Store<S>::from(state[(1 + i) * N + m]);
    if (k > 0 && k <= n_wall_ids) {
      if (grho) grho[j] = T(0);
      if (wall) atomicAdd(wall + 4 * (k - 1), lr / rho0);
      for (int i = 0; i < g.d; ++i) {
        if (gu) gu[i * N + j] = T(0);
        if (wall) atomicAdd(wall + 4 * (k - 1) + 1 + i, (double)lam[(1 + i) * N + m] / e);
      }
    } else {
      if (grho) grho[j] = T(lr / rho0);
      for (int i = 0; i < g.d; ++i)
        if (gu) gu[i * N + j] = T((double)lam[(1 + i) * N + m] / e);
    }
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(dot, red[0]);
}

template <typename S>
static cudaError_t seed_t(const Geometry& g, const void* grho, const void* gu, int dtype,
                          const void* state, double rho0, double e, void* lam, double* dot,
                          cudaStream_t st) {
  if (dtype == MACLAB_DTYPE_F64)
    adj_seed<S, double><<<grid256(g.n), 256, 0, st>>>(g, (const double*)grho, (const double*)gu,
                                                      (const S*)state, rho0, e,
                                                      (typename Store<S>::C*)lam, dot);
  else
    adj_seed<S, float><<<grid256(g.n), 256, 0, st>>>(g, (const float*)grho, (const float*)gu,
                                                     (const S*)state, rho0, e,
                                                     (typename Store<S>::C*)lam, dot);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t finish_t(const Geometry& g, const void* lam, const void* state, const uint8_t* nt,
                            int nw, double rho0, double e, void* grho, void* gu, int dtype,
                            double* wall, double* dot, cudaStream_t st) {
  using C = typename Store<S>::C;
  if (dtype == MACLAB_DTYPE_F64)
    adj_finish<S, double><<<grid256(g.n), 256, 0, st>>>(g, (const C*)lam, (const S*)state, nt, nw,
                                                        rho0, e, (double*)grho, (double*)gu, wall, dot);
  else
    adj_finish<S, float><<<grid256(g.n), 256, 0, st>>>(g, (const C*)lam, (const S*)state, nt, nw,
                                                       rho0, e, (float*)grho, (float*)gu, wall, dot);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(const Geometry& g, int precision, const void* grho, const void* gu,
                                int dtype, const void* state, double rho0, double e, void* lam,
                                double* dot, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return seed_t<double>(g, grho, gu, dtype, state, rho0, e, lam, dot, st);
    case MACLAB_F32: return seed_t<float>(g, grho, gu, dtype, state, rho0, e, lam, dot, st);
    case MACLAB_BF16_STORE: return seed_t<__nv_bfloat16>(g, grho, gu, dtype, state, rho0, e, lam, dot, st);
    case MACLAB_F16_STORE: return seed_t<__half>(g, grho, gu, dtype, state, rho0, e, lam, dot, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_finish(const Geometry& g, int precision, const void* lam, const void* state,
                                  const uint8_t* nt, int nw, double rho0, double e, void* grho,
                                  void* gu, int dtype, double* wall, double* dot, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return finish_t<double>(g, lam, state, nt, nw, rho0, e, grho, gu, dtype, wall, dot, st);
    case MACLAB_F32: return finish_t<float>(g, lam, state, nt, nw, rho0, e, grho, gu, dtype, wall, dot, st);
    case MACLAB_BF16_STORE:
      return finish_t<__nv_bfloat16>(g, lam, state, nt, nw, rho0, e, grho, gu, dtype, wall, dot, st);
    case MACLAB_F16_STORE:
      return finish_t<__half>(g, lam, state, nt, nw, rho0, e, grho, gu, dtype, wall, dot, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace maclab
