// reduce.cu -- FP64 diagnostics of the stored state.
//
// Sums over fluid nodes (walls excluded), accumulated in FP64 whatever the
// storage type:
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

#include "common.cuh"
#include "lattice.cuh"

namespace maclab {

constexpr int kDiagSlots = 9;

template <typename S>
__global__ void __launch_bounds__(256) diag_partial(Geometry g, const S* __restrict__ cur,
                                                    const S* __restrict__ prev,
                                                    double* __restrict__ partial) {
  double acc[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) acc[k] = 0.0;
  const int64_t N = g.n;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < N;
       m += (int64_t)gridDim.x * blockDim.x) {
    bool wall = false;
    if (g.wall_mode == kWallMask) {
      wall = g.mask[m] != 0;
    } else if (g.wall_mode == kWallBox) {
      const int x = log_x(g, (int)(m % g.nx));
      const int y = (int)((m / g.nx) % g.ny);
      const int z = (int)(m / ((int64_t)g.nx * g.ny));
      if (!(g.periodic & 1u)) wall |= (x == 0) | (x == g.nx - 1);
      if (!(g.periodic & 2u)) wall |= (y == 0) | (y == g.ny - 1);
      if (g.d == 3 && !(g.periodic & 4u)) wall |= (z == 0) | (z == g.nz - 1);
    }
    if (wall) continue;
    const double dr = (double)Store<S>::from(cur[m]);
    const double rho = 1.0 + dr;
    double uu = 0.0, du = 0.0;
    bool finite = isfinite(dr);
    acc[0] += dr;
    for (int i = 0; i < g.d; ++i) {
      const double u = (double)Store<S>::from(cur[(1 + i) * N + m]);
      finite = finite && isfinite(u);
      uu += u * u;
      acc[2 + i] += rho * u;
      if (prev) {
        const double d = u - (double)Store<S>::from(prev[(1 + i) * N + m]);
        du += d * d;
      }
    }
    acc[1] += rho * uu;
    acc[5] += du;
    acc[6] += uu;
    acc[7] = fmax(acc[7], sqrt(uu));
    if (!finite) acc[8] += 1.0;
  }
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

}  // namespace maclab
