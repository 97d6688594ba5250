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
// per-block partial sums in a fixed array that the library reserves when it is
// loaded, instead of a buffer owned by a handle.
//
// Each block folds a fixed run of kNoAllocNodesPerBlock nodes, so the partials
// a call needs grow with the node count; the array holds kNoAllocMaxBlocks of
// them, which bounds one call to kNoAllocMaxNodes nodes.

constexpr int64_t kNoAllocMaxBlocks = 4096;
constexpr int64_t kNoAllocNodesPerBlock = 8192;
constexpr int64_t kNoAllocMaxNodes = kNoAllocMaxBlocks * kNoAllocNodesPerBlock;  // 33,554,432

// Held by every GPU that loads the library, until the process exits
// (4096 x 9 doubles = 288 KiB).  Every call overwrites the entries it reads
// before reading them, so nothing here has to start at zero; calls that
// overlap on the GPU share it and race.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocMaxBlocks * kDiagSlots];

namespace {
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[64] = {};  // device address of g_noalloc_partials, per device
}  // namespace

// Address of the array on the current device: looked up once per device (the
// first call on a device does it) with that device current.
static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
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
