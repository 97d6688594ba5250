// reduce.cu -- FP64 diagnostics of the stored state.
//
// Sums over fluid nodes (walls excluded), accumulated in FP64 whatever the
// storage type (each node's products are formed in the storage's arithmetic
// type, FP32 for FP32 and 16-bit storage, where FP64 arithmetic is slow):
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

namespace maclab {

constexpr int kDiagSlots = 9;

template <typename S>
__global__ void __launch_bounds__(256) diag_partial(Geometry g, const S* __restrict__ cur,
                                                    const S* __restrict__ prev,
                                                    double* __restrict__ partial) {
  using C = typename Store<S>::C;
  double acc[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) acc[k] = 0.0;
  C umax2 = C(0);
  const int64_t N = g.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // storage position (mx, y, z) of m, advanced by the stride without dividing
  int64_t q = m / g.nx;
  int mx = (int)(m - q * g.nx), y = (int)(q % g.ny);
  int64_t z = q / g.ny;
  const int64_t sq = stride / g.nx;
  const int sx = (int)(stride - sq * g.nx), sy = (int)(sq % g.ny);
  const int64_t sz = sq / g.ny;
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
    // per-node products in the storage's arithmetic type, sums in FP64
    const C dr = Store<S>::from(cur[m]);
    const C rho = C(1) + dr;
    C uu = C(0), du = C(0);
    bool finite = isfinite(dr);
    acc[0] += (double)dr;
    for (int i = 0; i < g.d; ++i) {
      const C u = Store<S>::from(cur[(1 + i) * N + m]);
      finite = finite && isfinite(u);
      uu = fma(u, u, uu);
      acc[2 + i] += (double)(rho * u);
      if (prev) {
        const C d = u - Store<S>::from(prev[(1 + i) * N + m]);
        du = fma(d, d, du);
      }
    }
    acc[1] += (double)(rho * uu);
    acc[5] += (double)du;
    acc[6] += (double)uu;
    umax2 = fmax(umax2, uu);  // max |u|^2 here, its root below (the root is monotonic)
    if (!finite) acc[8] += 1.0;
  }
  acc[7] = sqrt((double)umax2);
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

__global__ void __launch_bounds__(256) diag_final(const double* __restrict__ partial, int nblocks,
                                                  double* __restrict__ out) {
  __shared__ double red[kDiagSlots][256];
  for (int k = 0; k < kDiagSlots; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
      const double w = partial[(int64_t)b * kDiagSlots + k];
      v = k == 7 ? fmax(v, w) : v + w;
    }
    red[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
      for (int k = 0; k < kDiagSlots; ++k)
        red[k][threadIdx.x] = k == 7 ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + s])
                                     : red[k][threadIdx.x] + red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < kDiagSlots) out[threadIdx.x] = red[threadIdx.x][0];
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
