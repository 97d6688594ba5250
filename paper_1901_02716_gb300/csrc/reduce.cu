// reduce.cu -- FP64 diagnostics of the stored state.
//
// Sums over fluid nodes (walls excluded), to FP64 accuracy whatever the
// storage type (each node's products are formed in the storage's arithmetic
// type, FP32 for FP32 and 16-bit storage, and added in float-float within a
// thread, where FP64 arithmetic is slow; FP64 across threads):
//   slot 0  sum drho                      (mass = rho0 (n_fluid + slot 0))
//   slot 1  sum rho |u|^2                 (kinetic energy = rho0 e^2 slot 1 / 2)
//   slot 2..4  sum rho u_i                (momentum = rho0 e slot)
//   slot 5  sum |u - u_prev|^2            (steady residual numerator)
//   slot 6  sum |u|^2                     (steady residual denominator)
//   slot 7  max |u|                       (lattice Mach number of the fastest node)
//   slot 8  number of non-finite values
// Mass and momentum are the quantities the equilibrium conserves (Eq. (15));
// the residual ||u^n - u^(n-1)||_2 / ||u^n||_2 is the steady-state measure.
// Two kernels: per-block partials into a scratch array, then one block folds
// the partials.

#include <mutex>

#include "common.cuh"
#include "lattice.cuh"
#include "step_tiled.cuh"  // Quad<S>: four stored values in one vector load

namespace maclab {

constexpr int kDiagSlots = 9;

// Running sum of one thread.  FP64 storage sums in FP64.  FP32 and 16-bit
// storage form each node's products in FP32, and a thread adds them in
// float-float: a pair (hi, lo) updated with Knuth's error-free two-sum, so the
// rounding error of every FP32 addition is kept in lo and the pair carries
// about 46 bits; it becomes one FP64 value at the end of the thread's loop.
// All of this runs on the FP32 pipe (GB300's FP64 rate is a small fraction
// of it), and the per-thread sums stay accurate to about 2^-46 of their size.
template <typename C>
struct DiagAcc;
template <>
struct DiagAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double value() const { return v; }
};
template <>
struct DiagAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename S>
__global__ void __launch_bounds__(256) diag_partial(Geometry g, const S* __restrict__ cur,
                                                    const S* __restrict__ prev,
                                                    double* __restrict__ partial) {
  using C = typename Store<S>::C;
  DiagAcc<C> sum[kDiagSlots - 2];  // slots 0-6
  float nonfinite = 0.f;
  C umax2 = C(0);
  const int64_t N = g.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // storage position (mx, y, z) of m, advanced by the stride without dividing
  // (32-bit divisions where the node count allows: 64-bit ones are emulated)
  int64_t q, sq;
  int mx, y, sx, sy;
  int64_t z, sz;
  if (N < (int64_t)INT32_MAX && stride < (int64_t)INT32_MAX) {
    const unsigned nx = (unsigned)g.nx, ny = (unsigned)g.ny;
    const unsigned m32 = (unsigned)(m < N ? m : 0), q32 = m32 / nx, s32 = (unsigned)stride, sq32 = s32 / nx;
    q = q32;
    mx = (int)(m32 - q32 * nx);
    y = (int)(q32 % ny);
    z = q32 / ny;
    sq = sq32;
    sx = (int)(s32 - sq32 * nx);
    sy = (int)(sq32 % ny);
    sz = sq32 / ny;
  } else {
    q = m / g.nx;
    mx = (int)(m - q * g.nx);
    y = (int)(q % g.ny);
    z = q / g.ny;
    sq = stride / g.nx;
    sx = (int)(stride - sq * g.nx);
    sy = (int)(sq % g.ny);
    sz = sq / g.ny;
  }
  (void)q;
  (void)sq;
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
    sum[0].add(dr);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (i >= g.d) break;
      const C u = Store<S>::from(cur[(1 + i) * N + m]);
      finite = finite && isfinite(u);
      uu = fma(u, u, uu);
      sum[2 + i].add(rho * u);
      if (prev) {
        const C d = u - Store<S>::from(prev[(1 + i) * N + m]);
        du = fma(d, d, du);
      }
    }
    sum[1].add(rho * uu);
    sum[5].add(du);
    sum[6].add(uu);
    umax2 = fmax(umax2, uu);  // max |u|^2 here, its root below (the root is monotonic)
    if (!finite) nonfinite += 1.f;
  }
  double acc[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots - 2; ++k) acc[k] = sum[k].value();
  acc[7] = sqrt((double)umax2);
  acc[8] = (double)nonfinite;
  // block reduction: warp shuffles, then one value per warp through shared memory
  __shared__ double red[kDiagSlots][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = k == 7 ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) {
      double v = lane < nw ? red[k][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = k == 7 ? fmax(v, w) : v + w;
      }
      if (lane == 0) partial[(int64_t)blockIdx.x * kDiagSlots + k] = v;
    }
  }
}

// Rows of x (nx % 4 == 0): a warp takes whole rows, each lane 16-byte quads of
// the four stored values of a node quad (vector loads, many in flight); rows on
// a closed y or z boundary are wall rows and skipped as a whole, and in box
// mode only the storage positions 0 and nx - 1 of a row (x = 0, nx - 1) are
// x-walls.  Same per-node products and sums as diag_partial.
template <typename S>
__global__ void __launch_bounds__(256) diag_rows(Geometry g, const S* __restrict__ cur,
                                                 const S* __restrict__ prev, double* __restrict__ partial) {
  using C = typename Store<S>::C;
  using P = typename Quad<S>::P;
  DiagAcc<C> sum[kDiagSlots - 2];
  float nonfinite = 0.f;
  C umax2 = C(0);
  const int64_t N = g.n;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = N / g.nx;
  const int quads = g.nx >> 2;
  const bool xw = g.wall_mode == kWallBox && !(g.periodic & 1u);
  const bool yw = g.wall_mode == kWallBox && !(g.periodic & 2u);
  const bool zw = g.wall_mode == kWallBox && g.d == 3 && !(g.periodic & 4u);
  for (int64_t row = warp; row < rows; row += nwarps) {
    const int y = (int)(row % g.ny);
    const int64_t z = row / g.ny;
    if ((yw && (y == 0 || y == g.ny - 1)) || (zw && (z == 0 || z == g.nz - 1))) continue;
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
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (wall[k]) continue;
        const int h = k >> 1;
        const auto pick = [&](const P& p) { return (k & 1) ? p.y : p.x; };
        const C dr = pick(r[h]);
        const C rho = C(1) + dr;
        C uu = C(0), du = C(0);
        bool finite = isfinite(dr);
        sum[0].add(dr);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (i >= g.d) break;
          const C ui = pick(u[i][h]);
          finite = finite && isfinite(ui);
          uu = fma(ui, ui, uu);
          sum[2 + i].add(rho * ui);
          if (prev) {
            const C d = ui - pick(v[i][h]);
            du = fma(d, d, du);
          }
        }
        sum[1].add(rho * uu);
        sum[5].add(du);
        sum[6].add(uu);
        umax2 = fmax(umax2, uu);
        if (!finite) nonfinite += 1.f;
      }
    }
  }
  double acc[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots - 2; ++k) acc[k] = sum[k].value();
  acc[7] = sqrt((double)umax2);
  acc[8] = (double)nonfinite;
  __shared__ double red[kDiagSlots][32];
  const int wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) {
    double v = acc[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = k == 7 ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[k][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) {
      double v = lane < nw ? red[k][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = k == 7 ? fmax(v, w) : v + w;
      }
      if (lane == 0) partial[(int64_t)blockIdx.x * kDiagSlots + k] = v;
    }
  }
}

// One block folds the partials: strided sums per thread, then warp shuffles
// and one value per warp through shared memory.
__global__ void __launch_bounds__(256) diag_final(const double* __restrict__ partial, int nblocks,
                                                  double* __restrict__ out) {
  __shared__ double red[kDiagSlots][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double w = partial[(int64_t)b * kDiagSlots + k];
      v = k == 7 ? fmax(v, w) : v + w;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = k == 7 ? fmax(v, w) : v + w;
    }
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < kDiagSlots; ++k) {
      double v = lane < 8 ? red[k][lane] : 0.0;
      for (int o = 4; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, v, o);
        v = k == 7 ? fmax(v, w) : v + w;
      }
      if (lane == 0) out[k] = v;
    }
  }
}

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
                          int nblocks, double* out, cudaStream_t st) {
  if (g.nx % 4 == 0)
    diag_rows<S><<<nblocks, 256, 0, st>>>(g, (const S*)cur, (const S*)prev, partial);
  else
    diag_partial<S><<<nblocks, 256, 0, st>>>(g, (const S*)cur, (const S*)prev, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final<<<1, 256, 0, st>>>(partial, nblocks, out);
  return cudaGetLastError();
}

// partial: scratch of nblocks * kDiagSlots doubles; out: kDiagSlots doubles (device).
cudaError_t launch_diagnostics(const Geometry& g, int precision, const void* cur, const void* prev,
                               double* partial, int nblocks, double* out, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return diag_t<double>(g, cur, prev, partial, nblocks, out, st);
    case MACLAB_F32: return diag_t<float>(g, cur, prev, partial, nblocks, out, st);
    case MACLAB_BF16_STORE: return diag_t<__nv_bfloat16>(g, cur, prev, partial, nblocks, out, st);
    case MACLAB_F16_STORE: return diag_t<__half>(g, cur, prev, partial, nblocks, out, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ allocation-free variant
//
// For callers that cannot allocate device memory while they run (for example a
// host loop that reserved all device memory for its own pool up front, or code
// that may not block on an allocation): the same two kernels, with the
// per-block partial sums in a fixed array that the module holds, instead of a
// buffer owned by a handle.
//
// A call launches ceil(n / kNoAllocNodesPerBlock) blocks, so each block folds
// about kNoAllocNodesPerBlock nodes (interleaved with the other blocks' by the
// grid stride); the array holds kNoAllocMaxBlocks partials, which bounds one
// call to kNoAllocMaxNodes nodes.

constexpr int64_t kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocNodesPerBlock = 8192;
constexpr int64_t kNoAllocMaxNodes = kNoAllocMaxBlocks * kNoAllocNodesPerBlock;  // 33,554,432

// Held by every GPU that loads this module, until the process exits
// (4096 x 9 doubles = 288 KiB).  Every call overwrites the entries it reads
// before reading them, so nothing here has to start at zero; calls that
// overlap on the GPU share it and race.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kDiagSlots];

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
                             (const void*)diag_final};
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
  e = launch_diagnostics(g, precision, state, prev_state, partials, nblocks, out_sums,
                         (cudaStream_t)stream);
  if (e != cudaSuccess) return err(MACLAB_ERR_CUDA, cudaGetErrorString(e));
  return MACLAB_OK;
}
