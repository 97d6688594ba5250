// reduce.cu -- FP64 diagnostics of the stored state.
//
// Sums over fluid nodes (walls excluded), in nine slots:
//   slot 0  sum drho                      (mass = rho0 (n_fluid + slot 0))
//   slot 1  sum rho |u|^2                 (kinetic energy = rho0 e^2 slot 1 / 2)
//   slot 2..4  sum rho u_i                (momentum = rho0 e slot)
//   slot 5  sum |u - u_prev|^2            (steady residual numerator)
//   slot 6  sum |u|^2                     (steady residual denominator)
//   slot 7  max |u|                       (lattice Mach number of the fastest node)
//   slot 8  number of non-finite values
// Each node's products are formed in the storage's arithmetic type (FP32 for
// FP32 and 16-bit storage) and added in float-float (FP64 for FP64 storage)
// by threads, warps, blocks and the grid; only the nine results become FP64.
// Mass and momentum are the quantities the equilibrium conserves (Eq. (15));
// the residual ||u^n - u^(n-1)||_2 / ||u^n||_2 is the steady-state measure.
// One kernel: block records into a scratch array, folded by the last block to
// finish.

#include <mutex>

#include "common.cuh"
#include "lattice.cuh"
#include "step_tiled.cuh"  // Quad<S>: four stored values in one vector load

namespace maclab {

constexpr int kDiagSlots = 9;

// Running sum of one thread.  FP64 storage sums in FP64.  FP32 and 16-bit
// storage form each node's products in FP32 and add them in float-float: a
// pair (hi, lo) updated with Knuth's error-free two-sum, so the rounding error
// of every FP32 addition is kept in lo and the pair carries about 46 bits.
// Threads, warps and blocks combine their pairs the same way (two-sum of the
// hi parts, the lo parts and that error added), and only the nine final
// values become FP64.  All of this runs on the FP32 pipe: GB300's FP64 rate is
// a small fraction of it, and a reduction that folded its partial sums in FP64
// spent much of its time there.
template <typename C>
struct DiagAcc;
template <>
struct DiagAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void merge(const DiagAcc& o) { v += o.v; }
  __device__ __forceinline__ DiagAcc shfl_down(int o) const {
    DiagAcc r;
    r.v = __shfl_down_sync(0xffffffffu, v, o);
    return r;
  }
  __device__ __forceinline__ void store(double* w) const { *w = v; }
  template <bool kGlobal>
  __device__ __forceinline__ static DiagAcc load(const double* w) {
    DiagAcc r;
    r.v = kGlobal ? __ldcg(w) : *w;
    return r;
  }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct DiagAcc<float> {
  float hi = 0.f, lo = 0.f;
  // s + err == a + b exactly (Knuth's two-sum; no FMA contraction in these
  // steps: each is an explicitly rounded add or subtract)
  __device__ __forceinline__ static float two_sum(float a, float b, float* err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    *err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
  }
  __device__ __forceinline__ void add(float x) {
    float err;
    hi = two_sum(hi, x, &err);
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void merge(const DiagAcc& o) {
    float err;
    hi = two_sum(hi, o.hi, &err);
    lo = __fadd_rn(lo, __fadd_rn(o.lo, err));
  }
  __device__ __forceinline__ DiagAcc shfl_down(int o) const {
    DiagAcc r;
    r.hi = __shfl_down_sync(0xffffffffu, hi, o);
    r.lo = __shfl_down_sync(0xffffffffu, lo, o);
    return r;
  }
  // one 8-byte word of a record holds the pair
  __device__ __forceinline__ void store(double* w) const { *reinterpret_cast<float2*>(w) = make_float2(hi, lo); }
  template <bool kGlobal>
  __device__ __forceinline__ static DiagAcc load(const double* w) {
    const float2* p = reinterpret_cast<const float2*>(w);
    const float2 v = kGlobal ? __ldcg(p) : *p;
    DiagAcc r;
    r.hi = v.x;
    r.lo = v.y;
    return r;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Everything one thread, warp or block has gathered: the seven sums, the
// largest |u|^2 and the count of non-finite nodes.  A record of it is nine
// 8-byte words (the slots of the output; word 7 holds max |u|^2 in the
// arithmetic type, word 8 the count as an unsigned 64-bit integer).
template <typename C>
struct DiagPart {
  DiagAcc<C> sum[kDiagSlots - 2];
  C umax2 = C(0);
  unsigned nonfinite = 0;

  __device__ __forceinline__ void merge(const DiagPart& o) {
#pragma unroll
    for (int k = 0; k < kDiagSlots - 2; ++k) sum[k].merge(o.sum[k]);
    umax2 = fmax(umax2, o.umax2);
    nonfinite += o.nonfinite;
  }
  __device__ __forceinline__ DiagPart shfl_down(int o) const {
    DiagPart r;
#pragma unroll
    for (int k = 0; k < kDiagSlots - 2; ++k) r.sum[k] = sum[k].shfl_down(o);
    r.umax2 = __shfl_down_sync(0xffffffffu, umax2, o);
    r.nonfinite = __shfl_down_sync(0xffffffffu, nonfinite, o);
    return r;
  }
  __device__ __forceinline__ void store(double* rec) const {
#pragma unroll
    for (int k = 0; k < kDiagSlots - 2; ++k) sum[k].store(rec + k);
    *reinterpret_cast<C*>(rec + 7) = umax2;
    *reinterpret_cast<unsigned long long*>(rec + 8) = nonfinite;
  }
  template <bool kGlobal>
  __device__ __forceinline__ static DiagPart load(const double* rec) {
    DiagPart r;
#pragma unroll
    for (int k = 0; k < kDiagSlots - 2; ++k) r.sum[k] = DiagAcc<C>::template load<kGlobal>(rec + k);
    const C* m = reinterpret_cast<const C*>(rec + 7);
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(rec + 8);
    r.umax2 = kGlobal ? __ldcg(m) : *m;
    r.nonfinite = (unsigned)(kGlobal ? __ldcg(c) : *c);
    return r;
  }
  // the nine output values; the root of max |u|^2 is taken once, here
  __device__ __forceinline__ void output(double* out) const {
#pragma unroll
    for (int k = 0; k < kDiagSlots - 2; ++k) out[k] = sum[k].value();
    out[7] = sqrt((double)umax2);
    out[8] = (double)nonfinite;
  }
};

// Folds the parts of a block's threads (blockDim.x a multiple of 32, at most
// 1024) into one, held by thread 0.  Warps fold by shuffles; one record per
// warp goes through shared memory and warp 0 folds those.
template <typename C>
__device__ __forceinline__ DiagPart<C> block_fold(DiagPart<C> t) {
  __shared__ double red[32][kDiagSlots];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t.merge(t.shfl_down(o));
  if (lane == 0) t.store(red[warp]);
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    t = lane < nw ? DiagPart<C>::template load<false>(red[lane]) : DiagPart<C>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t.merge(t.shfl_down(o));
  }
  __syncthreads();  // red may be reused by a second fold
  return t;
}

// The end of a diagnostics kernel.  Each block writes its record to
// partial[blockIdx.x]; the last block to finish (a ticket counter that the
// last one also returns to zero, atomicInc wrapping at gridDim.x - 1) reads
// all the records and writes the nine output values.  No block waits for
// another.  ticket must hold 0 before the launch; every launch leaves it 0.
template <typename C>
__device__ __forceinline__ void grid_fold(const DiagPart<C>& mine, double* __restrict__ partial,
                                          unsigned* __restrict__ ticket, double* __restrict__ out) {
  __shared__ bool last;
  const DiagPart<C> b = block_fold(mine);
  if (threadIdx.x == 0) {
    b.store(partial + (int64_t)blockIdx.x * kDiagSlots);
    __threadfence();  // the record is visible to every block before the ticket is taken
    last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  DiagPart<C> t;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x)
    t.merge(DiagPart<C>::template load<true>(partial + (int64_t)k * kDiagSlots));
  t = block_fold(t);
  if (threadIdx.x == 0) {
    double v[kDiagSlots];
    t.output(v);
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) out[k] = v[k];
  }
}

template <typename S>
__global__ void __launch_bounds__(256) diag_partial(Geometry g, const S* __restrict__ cur,
                                                    const S* __restrict__ prev,
                                                    double* __restrict__ partial,
                                                    unsigned* __restrict__ ticket,
                                                    double* __restrict__ out) {
  using C = typename Store<S>::C;
  pdl_wait();  // the step before this kernel has completed and its writes are visible
  pdl_launch_next();  // the next step may be scheduled; it waits for this kernel before writing
  DiagPart<C> t;
  const int64_t N = g.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // storage position (mx, y, z) of m, advanced by the stride without dividing
  // (32-bit divisions where the node count allows: 64-bit ones are emulated)
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
  for (; m < N; m += stride) {
    bool wall = false;
    if (g.wall_mode == kWallMask) {
      wall = g.mask[m] != 0;
    } else if (g.wall_mode == kWallBox) {
      const int x = log_x(g, mx);
      if (!(g.periodic & 1u)) wall |= (x == 0) | (x == g.nx - 1);
      if (!(g.periodic & 2u)) wall |= (y == 0) | (y == g.ny - 1);
      if (g.d == 3 && !(g.periodic & 4u)) wall |= (z == 0) | (z == g.nz - 1);
    }
    mx += sx;
    const int carry = mx >= g.nx ? 1 : 0;
    mx -= carry * g.nx;
    y += sy + carry;
    if (y >= g.ny) {
      y -= g.ny;
      z += 1;
    }
    z += sz;
    if (wall) continue;
    // per-node products in the storage's arithmetic type
    const C dr = Store<S>::from(cur[m]);
    const C rho = C(1) + dr;
    C uu = C(0), du = C(0);
    bool finite = isfinite(dr);
    t.sum[0].add(dr);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i >= g.d) break;
      const C u = Store<S>::from(cur[(1 + i) * N + m]);
      finite = finite && isfinite(u);
      uu = fma(u, u, uu);
      t.sum[2 + i].add(rho * u);
      if (prev) {
        const C d = u - Store<S>::from(prev[(1 + i) * N + m]);
        du = fma(d, d, du);
      }
    }
    t.sum[1].add(rho * uu);
    t.sum[5].add(du);
    t.sum[6].add(uu);
    t.umax2 = fmax(t.umax2, uu);  // max |u|^2 here, its root at the end (the root is monotonic)
    if (!finite) ++t.nonfinite;
  }
  grid_fold(t, partial, ticket, out);
}

// Rows of x (nx % 4 == 0): a warp takes whole rows, each lane 16-byte quads of
// the four stored values of a node quad (vector loads, many in flight); rows on
// a closed y or z boundary are wall rows and skipped as a whole, and in box
// mode only the storage positions 0 and nx - 1 of a row (x = 0, nx - 1) are
// x-walls.  The stored density deviations are exact inputs and enter the
// float-float sum node by node, as in diag_partial.  The per-node products
// (rho |u|^2, rho u_i, |u - u_prev|^2, |u|^2) are formed on the quad's two node
// pairs with paired arithmetic, each rounded to the arithmetic type; a quad's
// four are added in that type and the quad's sum enters the float-float sum
// (one two-sum per quad and slot instead of one per node: three more
// roundings of the same size per quad, not an error that grows with the node
// count; the sums differ from diag_partial's by at most 5 units of 2^-24 of
// the sum of the terms' magnitudes).  Wall nodes of a quad enter as zeros.  A
// quad whose summed density and |u|^2 are not finite holds a non-finite value
// (or overflows) and is checked node by node.
template <typename S>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 1 : 2) diag_rows(Geometry g, const S* __restrict__ cur,
                                                    const S* __restrict__ prev,
                                                    double* __restrict__ partial,
                                                    unsigned* __restrict__ ticket,
                                                    double* __restrict__ out) {
  using C = typename Store<S>::C;
  using P = typename Quad<S>::P;
  using O = Pair<C>;
  pdl_wait();  // the step before this kernel has completed and its writes are visible
  pdl_launch_next();  // the next step may be scheduled; it waits for this kernel before writing
  DiagPart<C> t;
  const int64_t N = g.n;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = N / g.nx;
  const int quads = g.nx >> 2;
  const bool xw = g.wall_mode == kWallBox && !(g.periodic & 1u);
  const bool yw = g.wall_mode == kWallBox && !(g.periodic & 2u);
  const bool zw = g.wall_mode == kWallBox && g.d == 3 && !(g.periodic & 4u);
  // (y, z) of the warp's row, advanced by nwarps rows a turn without dividing
  int y = (int)(warp % g.ny);
  int64_t z = warp / g.ny;
  const int dy = (int)(nwarps % g.ny);
  const int64_t dz = nwarps / g.ny;
  for (int64_t row = warp; row < rows; row += nwarps) {
    const bool wall_row = (yw && (y == 0 || y == g.ny - 1)) || (zw && (z == 0 || z == g.nz - 1));
    y += dy;
    z += dz;
    if (y >= g.ny) {
      y -= g.ny;
      ++z;
    }
    if (wall_row) continue;
    for (int q = lane; q < quads; q += 32) {
      const int64_t m = row * g.nx + 4 * q;
      bool wall[4] = {false, false, false, false};
      if (g.wall_mode == kWallMask) {
        const uchar4 mk = *reinterpret_cast<const uchar4*>(g.mask + m);
        wall[0] = mk.x != 0; wall[1] = mk.y != 0; wall[2] = mk.z != 0; wall[3] = mk.w != 0;
      } else if (xw) {
        wall[0] = q == 0;
        wall[3] = q == quads - 1;
      }
      P r[2], u[3][2], v[3][2];
      Quad<S>::ld(cur + m, r[0], r[1]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (i >= g.d) break;
        Quad<S>::ld(cur + (1 + i) * N + m, u[i][0], u[i][1]);
        if (prev) Quad<S>::ld(prev + (1 + i) * N + m, v[i][0], v[i][1]);
      }
      // wall nodes of the quad enter as zeros (their values are not summed)
      if (wall[0] | wall[1] | wall[2] | wall[3]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const bool w0 = wall[2 * h], w1 = wall[2 * h + 1];
          r[h].x = w0 ? C(0) : r[h].x;
          r[h].y = w1 ? C(0) : r[h].y;
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            if (i >= g.d) break;
            u[i][h].x = w0 ? C(0) : u[i][h].x;
            u[i][h].y = w1 ? C(0) : u[i][h].y;
            v[i][h].x = w0 ? C(0) : v[i][h].x;
            v[i][h].y = w1 ? C(0) : v[i][h].y;
          }
        }
      }
      // the quad's sums on its two node pairs: drho, rho |u|^2, rho u_i,
      // |u - u_prev|^2, |u|^2; the density deviations also node by node
      P qs[kDiagSlots - 2];
#pragma unroll
      for (int k = 0; k < kDiagSlots - 2; ++k) qs[k] = O::splat(C(0));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const P dr = r[h];
        t.sum[0].add(dr.x);
        t.sum[0].add(dr.y);
        const P rho = O::add(O::splat(C(1)), dr);
        P uu = O::splat(C(0)), du = O::splat(C(0));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i >= g.d) break;
          const P ui = u[i][h];
          uu = O::fma(ui, ui, uu);
          qs[2 + i] = O::fma(rho, ui, qs[2 + i]);
          if (prev) {
            const P dd = O::sub(ui, v[i][h]);
            du = O::fma(dd, dd, du);
          }
        }
        qs[0] = O::add(qs[0], dr);
        qs[1] = O::fma(rho, uu, qs[1]);
        qs[5] = O::add(qs[5], du);
        qs[6] = O::add(qs[6], uu);
        t.umax2 = fmax(t.umax2, fmax(uu.x, uu.y));
      }
#pragma unroll
      for (int k = 1; k < kDiagSlots - 2; ++k) {
        if (k >= 2 && k < 5 && k - 2 >= g.d) continue;
        t.sum[k].add(qs[k].x + qs[k].y);
      }
      if (!isfinite(qs[0].x + qs[0].y + qs[6].x + qs[6].y)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (wall[k]) continue;
          const int h = k >> 1;
          const auto pick = [&](const P& p) { return (k & 1) ? p.y : p.x; };
          bool finite = isfinite(pick(r[h]));
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            if (i >= g.d) break;
            finite = finite && isfinite(pick(u[i][h]));
          }
          if (!finite) ++t.nonfinite;
        }
      }
    }
  }
  grid_fold(t, partial, ticket, out);
}

// Blocks of one launch: two 256-thread blocks per SM (the row kernel's paired
// sums need more than the 85 registers three blocks would leave), fewer on
// small grids.
int diag_blocks(int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  int64_t b = (n + 255) / 256;
  if (b > 2 * sms) b = 2 * sms;
  return (int)(b < 1 ? 1 : b);
}

template <typename S>
static cudaError_t diag_t(const Geometry& g, const void* cur, const void* prev, double* partial,
                          unsigned* ticket, int nblocks, double* out, cudaStream_t st, int overlap) {
  if (g.nx % 4 == 0)
    return launch_kernel(diag_rows<S>, dim3(nblocks), dim3(256), 0, st, overlap, g, (const S*)cur,
                         (const S*)prev, partial, ticket, out);
  return launch_kernel(diag_partial<S>, dim3(nblocks), dim3(256), 0, st, overlap, g, (const S*)cur,
                       (const S*)prev, partial, ticket, out);
}

// One kernel: per-block records in partial (nblocks * kDiagSlots doubles), the
// last block's fold into out (kDiagSlots doubles, device).  ticket: one
// counter on the device that holds 0 and that no other launch uses at the
// same time; the launch leaves it 0.  overlap: launched with programmatic
// dependent launch after a step kernel.
cudaError_t launch_diagnostics(const Geometry& g, int precision, const void* cur, const void* prev,
                               double* partial, unsigned* ticket, int nblocks, double* out,
                               cudaStream_t st, int overlap) {
  switch (precision) {
    case MACLAB_F64: return diag_t<double>(g, cur, prev, partial, ticket, nblocks, out, st, overlap);
    case MACLAB_F32: return diag_t<float>(g, cur, prev, partial, ticket, nblocks, out, st, overlap);
    case MACLAB_BF16_STORE:
      return diag_t<__nv_bfloat16>(g, cur, prev, partial, ticket, nblocks, out, st, overlap);
    case MACLAB_F16_STORE: return diag_t<__half>(g, cur, prev, partial, ticket, nblocks, out, st, overlap);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ allocation-free variant
//
// For callers that cannot allocate device memory while they run (for example a
// host loop that reserved all device memory for its own pool up front, or code
// that may not block on an allocation): the same kernels, with the per-block
// records and the ticket counter in a fixed array that the module holds,
// instead of a buffer owned by a handle.
//
// A call launches ceil(n / kNoAllocNodesPerBlock) blocks, so each block folds
// about kNoAllocNodesPerBlock nodes (interleaved with the other blocks' by the
// grid stride); the array holds kNoAllocMaxBlocks records, which bounds one
// call to kNoAllocMaxNodes nodes.

constexpr int64_t kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocNodesPerBlock = 8192;
constexpr int64_t kNoAllocMaxNodes = kNoAllocMaxBlocks * kNoAllocNodesPerBlock;  // 33,554,432

// Held by every GPU that loads this module, until the process exits
// (4096 x 9 records and one word for the ticket: 288 KiB).  Every call
// overwrites the records it reads before reading them and sets the ticket to
// 0 before its reduction starts, so nothing here has to start at zero; calls
// that overlap on the GPU share it and race.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kDiagSlots + 1];

__global__ void diag_ticket_reset(unsigned* ticket) { *ticket = 0u; }

namespace {
using CtxGetCurrent = int (*)(void**);  // cuCtxGetCurrent(CUcontext*), through the runtime
std::mutex g_noalloc_mutex;
struct NoAllocSlot {
  void* ctx = nullptr;     // context the address below belongs to
  double* ptr = nullptr;   // device address of g_noalloc_partials in that context
};
NoAllocSlot g_noalloc_slot[64];  // per device
CtxGetCurrent g_ctx_get = nullptr;
bool g_ctx_get_looked_up = false;
}  // namespace

// Set-up on the current device, once per device and context: load the
// reduction kernels (with lazy module loading a kernel's code is otherwise
// loaded, and may take device memory, at its first launch) and look up the
// array's address with that device current.  A context that replaces the
// device's previous one (cudaDeviceReset) has another handle and gets the
// set-up again; a recreated context that happened to reuse the old handle
// would not be told apart.
static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_ctx_get_looked_up) {
    g_ctx_get_looked_up = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      g_ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
    cudaGetLastError();
  }
  void* ctx = nullptr;
  if (g_ctx_get) g_ctx_get(&ctx);
  NoAllocSlot& slot = g_noalloc_slot[dev];
  if (!slot.ptr || slot.ctx != ctx) {
    cudaFuncAttributes fa{};
    const void* kernels[] = {(const void*)diag_partial<double>, (const void*)diag_partial<float>,
                             (const void*)diag_partial<__nv_bfloat16>, (const void*)diag_partial<__half>,
                             (const void*)diag_rows<double>, (const void*)diag_rows<float>,
                             (const void*)diag_rows<__nv_bfloat16>, (const void*)diag_rows<__half>,
                             (const void*)diag_ticket_reset};
    for (const void* k : kernels) {
      e = cudaFuncGetAttributes(&fa, k);
      if (e != cudaSuccess) return e;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    slot.ptr = static_cast<double*>(p);
    slot.ctx = ctx;
  }
  *out = slot.ptr;
  return cudaSuccess;
}

// True if p is device (or managed) memory that the current device can use.
static bool noalloc_device_pointer(const void* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace maclab

using namespace maclab;

extern "C" maclab_status maclab_diagnostics_noalloc(int32_t lattice, int32_t precision,
                                                    int64_t n_nodes, const void* state,
                                                    const void* prev_state,
                                                    const uint8_t* exclude, double* out_sums,
                                                    void* stream) {
  auto err = [](maclab_status s, const char* m) {
    record_error(m);
    return s;
  };
  if (lattice != MACLAB_D2Q9 && lattice != MACLAB_D3Q19) return err(MACLAB_ERR_INVALID, "unknown lattice");
  if (precision < MACLAB_F64 || precision > MACLAB_F16_STORE)
    return err(MACLAB_ERR_INVALID, "unknown precision");
  if (!state || !out_sums) return err(MACLAB_ERR_INVALID, "state and out_sums are required");
  if (n_nodes < 1) return err(MACLAB_ERR_INVALID, "n_nodes must be >= 1");
  if (n_nodes > kNoAllocMaxNodes)
    return err(MACLAB_ERR_INVALID,
               "n_nodes exceeds the 33554432 nodes the fixed scratch of "
               "maclab_diagnostics_noalloc can reduce in one call");
  if (!noalloc_device_pointer(state) || (prev_state && !noalloc_device_pointer(prev_state)) ||
      (exclude && !noalloc_device_pointer(exclude)) || !noalloc_device_pointer(out_sums))
    return err(MACLAB_ERR_INVALID,
               "state, prev_state, exclude and out_sums must be device memory of the current device");
  double* partials = nullptr;
  cudaError_t e = noalloc_scratch(&partials);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(MACLAB_ERR_CUDA, "cudaGetSymbolAddress of the fixed scratch failed");
  }
  Geometry g{};
  g.lattice = lattice == MACLAB_D2Q9 ? kD2Q9 : kD3Q19;
  g.d = lattice == MACLAB_D2Q9 ? 2 : 3;
  g.nx = 1;
  g.ny = 1;
  g.nz = 1;
  g.n = n_nodes;
  g.wall_mode = exclude ? kWallMask : kWallNone;
  g.mask = exclude;
  const int nblocks = (int)((n_nodes + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
  unsigned* ticket = reinterpret_cast<unsigned*>(partials + kNoAllocMaxBlocks * kDiagSlots);
  diag_ticket_reset<<<1, 1, 0, (cudaStream_t)stream>>>(ticket);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_diagnostics(g, precision, state, prev_state, partials, ticket, nblocks, out_sums,
                           (cudaStream_t)stream, 0);
  if (e != cudaSuccess) return err(MACLAB_ERR_CUDA, cudaGetErrorString(e));
  return MACLAB_OK;
}
