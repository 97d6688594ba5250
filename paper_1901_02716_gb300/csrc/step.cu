// step.cu -- the MacLAB time step (Eqs. (2), (4), (5)) on the GPU.
//
// Stored state: drho = rho / rho0 - 1 and ut = u / e, structure of arrays in
// storage order (see mem_x in common.cuh).
// With rho = 1 + drho and P_a = 3 c_a.ut + 9/2 (c_a.ut)^2 - 3/2 ut.ut, the
// equilibrium of Eq. (2) is f_a^eq = w_a (1 + drho + (1 + drho) P_a).  The
// constant w_a sums to 1 over a and w_a c_a sums to 0, so Eqs. (4)-(5) become
//   drho'(x) = sum_a w_a T_a(x - c_a),   m'(x) = sum_a w_a c_a T_a(x - c_a),
//   ut'(x)   = m'(x) / (1 + drho'(x)) + force,   T_a = drho + (1 + drho) P_a,
// in which every term is small: this is what keeps FP32 (and 16-bit storage)
// accurate.  Wall nodes are never written: both ping-pong buffers hold their
// values.  Periodic axes wrap; on closed axes a fluid node's upstream
// neighbours always exist because the outer layers are walls (checked on the
// host at create time).
//
// Kernels here:
//  * step_naive: one thread per node, the Q upstream states read straight from
//    global memory.  Any size; the reference the faster kernel is tested on.
//  * step_tiled (step_tiled.cu): strips of 4 nodes per thread, a march along
//    the slowest axis, equilibria exchanged through shared memory.

#include "common.cuh"
#include "lattice.cuh"

namespace maclab {

template <typename C>
struct Force {
  C f[3];
};

template <int LAT>
__device__ __forceinline__ bool is_wall_node(const Geometry& g, int x, int y, int z, int64_t node) {
  if (g.wall_mode == kWallNone) return false;
  if (g.wall_mode == kWallMask) return g.mask[node] != 0;
  bool w = false;
  if (!(g.periodic & 1u)) w |= (x == 0) | (x == g.nx - 1);
  if (!(g.periodic & 2u)) w |= (y == 0) | (y == g.ny - 1);
  if (Lattice<LAT>::D == 3 && !(g.periodic & 4u)) w |= (z == 0) | (z == g.nz - 1);
  return w;
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// ------------------------------------------------------------------ naive kernel

template <int LAT, typename S>
__global__ void __launch_bounds__(256) step_naive(Geometry g, const S* __restrict__ in,
                                                  S* __restrict__ out,
                                                  Force<typename Store<S>::C> force) {
  using C = typename Store<S>::C;
  using L = Lattice<LAT>;
  constexpr int D = L::D;
  const int64_t N = g.n;
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < N;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int x = log_x(g, (int)(node % g.nx));
    const int y = (int)((node / g.nx) % g.ny);
    const int z = (int)(node / ((int64_t)g.nx * g.ny));
    if (is_wall_node<LAT>(g, x, y, z, node)) continue;
    C dr = 0, m[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      const int xs = wrap(x - L::c(a, 0), g.nx);
      const int ys = wrap(y - L::c(a, 1), g.ny);
      const int zs = D == 3 ? wrap(z - L::c(a, 2), g.nz) : 0;
      const int64_t s = ((int64_t)zs * g.ny + ys) * g.nx + mem_x(g, xs);
      const C r = Store<S>::ld(in + s);
      C u[3] = {Store<S>::ld(in + N + s), Store<S>::ld(in + 2 * N + s),
                D == 3 ? Store<S>::ld(in + 3 * N + s) : C(0)};
      C cu = 0, uu = 0;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        cu += C(L::c(a, i)) * u[i];
        uu += u[i] * u[i];
      }
      const C P = C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu;
      const C T = (r + (C(1) + r) * P) * (C(L::w36(a)) / C(36));
      dr += T;
#pragma unroll
      for (int i = 0; i < D; ++i)
        if (L::c(a, i) != 0) m[i] += C(L::c(a, i)) * T;
    }
    const C inv = C(1) / (C(1) + dr);
    Store<S>::st(out + node, dr);
#pragma unroll
    for (int i = 0; i < D; ++i) Store<S>::st(out + (1 + i) * N + node, m[i] * inv + force.f[i]);
  }
}

// ------------------------------------------------------------------ dispatch

template <int LAT, typename S>
static cudaError_t launch_naive_t(const StepLaunch& s, cudaStream_t stream) {
  using C = typename Store<S>::C;
  Force<C> f{{C(s.force[0]), C(s.force[1]), C(s.force[2])}};
  const int threads = 256;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (s.g.n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  step_naive<LAT, S><<<(unsigned)blocks, threads, 0, stream>>>(
      s.g, static_cast<const S*>(s.in), static_cast<S*>(s.out), f);
  return cudaGetLastError();
}

template <int LAT>
static cudaError_t launch_naive_lat(const StepLaunch& s, cudaStream_t stream) {
  switch (s.precision) {
    case MACLAB_F64: return launch_naive_t<LAT, double>(s, stream);
    case MACLAB_F32: return launch_naive_t<LAT, float>(s, stream);
    case MACLAB_BF16_STORE: return launch_naive_t<LAT, __nv_bfloat16>(s, stream);
    case MACLAB_F16_STORE: return launch_naive_t<LAT, __half>(s, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Time steps per launch of the segment kernel for the tile setting ty (2 asks
// for two steps per launch: FP32 or FP64 storage and nx >= 8; otherwise 1).
// Segment kernel defaults (measured on a GB300, FP32 cavities of 64^2 to
// 8192^2): two steps per launch below 200,000 quads (small grids are bound by
// the launches) and, with FP32 storage, above 524,288 quads (large grids are
// bound by memory traffic, which two steps halve: 1.57x at 2048^2, 1.8x at
// 8192^2; FP64 is bound by its arithmetic, which the halo rows only add to),
// one step in between (1024^2); rows per work item 2 up to 65,536 quads, 4
// above, and 32 for two steps above 524,288 quads (the two halo rows each
// side of an item then cost an eighth of its rows).
static bool segment_large(const Geometry& g) { return (int64_t)(g.nx / 4) * g.ny > 524288; }

int segment_depth(const Geometry& g, int precision, int ty) {
  const bool two_ok = (precision == MACLAB_F32 || precision == MACLAB_F64) && g.nx >= 8;
  if (ty == 0)
    return two_ok && ((int64_t)(g.nx / 4) * g.ny < 200000 || (segment_large(g) && precision == MACLAB_F32)) ? 2
                                                                                                             : 1;
  return (ty == 2 || ty == 3) && two_ok ? 2 : 1;  // 3: two steps, runs in one persistent launch
}

int segment_rows(const Geometry& g, int precision, int ty, int tz) {
  if (tz > 0) return tz;
  if (segment_large(g) && segment_depth(g, precision, ty) == 2) return 32;
  return (int64_t)(g.nx / 4) * g.ny <= 65536 ? 2 : 4;
}

bool step_kernel_supported(const Geometry& g, int precision, int kernel) {
  if (kernel == MACLAB_KERNEL_REFERENCE) return true;
  if (kernel == MACLAB_KERNEL_TILED) return tiled_supported(g, precision, 0, 0);
  if (kernel == MACLAB_KERNEL_FOLDED) return fold_supported(g, precision, 0);
  if (kernel == MACLAB_KERNEL_SEGMENT) return g.lattice == kD2Q9 && g.ilv == 1;
  if (kernel == MACLAB_KERNEL_ROWS2) return rows2_supported(g, precision, 0);
  if (kernel == MACLAB_KERNEL_BLOCK) return block_supported(g, precision, 0);
  return false;
}

// D3Q19 with FP32 storage: the two-rows-per-thread kernel where it applies
// (rows of up to 128 nodes), else the folded one where it is built (ny a
// multiple of its tile rows); for D2Q9 grids with nx % 4 == 0 the block kernel
// with FP32 or FP64 storage up to 131,072 node pairs (512^2; measured on a
// GB300, FP32: 1.9x the segment kernel at 128^2 and 256^2, 1.16x at 512^2;
// FP64: 1.9x to 2.4x), else the segment
// kernel (faster than the tiled one from 64^2 to 1024^2 with its size
// defaults, and than the block kernel above 512^2); else the tiled one, else
// the reference kernel.
int pick_step_kernel(const Geometry& g, int precision) {
  if (precision == MACLAB_F32 && step_kernel_supported(g, precision, MACLAB_KERNEL_ROWS2))
    return MACLAB_KERNEL_ROWS2;
  if (step_kernel_supported(g, precision, MACLAB_KERNEL_FOLDED)) return MACLAB_KERNEL_FOLDED;
  if ((int64_t)(g.nx / 2) * g.ny <= 131072 && step_kernel_supported(g, precision, MACLAB_KERNEL_BLOCK))
    return MACLAB_KERNEL_BLOCK;
  if (step_kernel_supported(g, precision, MACLAB_KERNEL_SEGMENT)) return MACLAB_KERNEL_SEGMENT;
  return step_kernel_supported(g, precision, MACLAB_KERNEL_TILED) ? MACLAB_KERNEL_TILED
                                                                 : MACLAB_KERNEL_REFERENCE;
}

static const char* kernel_name(const Geometry& g, int precision, int kernel) {
  if (kernel == MACLAB_KERNEL_ROWS2) {
    static const char* rows2[4] = {"step_rows2<D3Q19,f64>", "step_rows2<D3Q19,f32>", "step_rows2<D3Q19,bf16>",
                                   "step_rows2<D3Q19,f16>"};
    return rows2[precision & 3];
  }
  if (kernel == MACLAB_KERNEL_FOLDED) {
    static const char* fold[4] = {"step_fold<D3Q19,f64>", "step_fold<D3Q19,f32>", "step_fold<D3Q19,bf16>",
                                  "step_fold<D3Q19,f16>"};
    return fold[precision & 3];
  }
  if (kernel == MACLAB_KERNEL_BLOCK) {
    static const char* blk[4] = {"step_block<D2Q9,f64>", "step_block<D2Q9,f32>", "step_block<D2Q9,bf16>",
                                 "step_block<D2Q9,f16>"};
    return blk[precision & 3];
  }
  if (kernel == MACLAB_KERNEL_SEGMENT) {
    static const char* seg[4] = {"segment<D2Q9,f64>", "segment<D2Q9,f32>", "segment<D2Q9,bf16>",
                                 "segment<D2Q9,f16>"};
    return seg[precision & 3];
  }
  static const char* names[2][2][4] = {
      {{"step_naive<D2Q9,f64>", "step_naive<D2Q9,f32>", "step_naive<D2Q9,bf16>",
        "step_naive<D2Q9,f16>"},
       {"step_naive<D3Q19,f64>", "step_naive<D3Q19,f32>", "step_naive<D3Q19,bf16>",
        "step_naive<D3Q19,f16>"}},
      {{"step_tiled<D2Q9,f64>", "step_tiled<D2Q9,f32>", "step_tiled<D2Q9,bf16>",
        "step_tiled<D2Q9,f16>"},
       {"step_tiled<D3Q19,f64>", "step_tiled<D3Q19,f32>", "step_tiled<D3Q19,bf16>",
        "step_tiled<D3Q19,f16>"}}};
  return names[kernel == MACLAB_KERNEL_TILED ? 1 : 0][g.lattice == kD2Q9 ? 0 : 1][precision & 3];
}

KernelInfo describe_step_kernel(const Geometry& g, int precision, int kernel, int ty, int tz) {
  if (kernel == MACLAB_KERNEL_TILED)
    return KernelInfo{MACLAB_KERNEL_TILED, 1, 1, tiled_threads(g, precision, ty, tz),
                      kernel_name(g, precision, kernel)};
  if (kernel == MACLAB_KERNEL_FOLDED)
    return KernelInfo{MACLAB_KERNEL_FOLDED, 1, 1, fold_threads(g, precision, ty),
                      kernel_name(g, precision, kernel)};
  if (kernel == MACLAB_KERNEL_ROWS2)
    return KernelInfo{MACLAB_KERNEL_ROWS2, 1, 1, rows2_threads(g, precision, ty), kernel_name(g, precision, kernel)};
  if (kernel == MACLAB_KERNEL_BLOCK)
    return KernelInfo{MACLAB_KERNEL_BLOCK, block_steps(g, precision, ty), 1, block_threads(precision),
                      kernel_name(g, precision, kernel)};

  if (kernel == MACLAB_KERNEL_SEGMENT) {
    const int depth = segment_depth(g, precision, ty);
    return KernelInfo{MACLAB_KERNEL_SEGMENT, depth, 1, depth == 2 ? 128 : 256, kernel_name(g, precision, kernel)};
  }
  return KernelInfo{MACLAB_KERNEL_REFERENCE, 1, 1, 256, kernel_name(g, precision, kernel)};
}

cudaError_t launch_step(const StepLaunch& s, cudaStream_t stream, int kernel) {
  switch (kernel) {
    case MACLAB_KERNEL_REFERENCE:
      return s.g.lattice == kD2Q9 ? launch_naive_lat<kD2Q9>(s, stream)
                                  : launch_naive_lat<kD3Q19>(s, stream);
    case MACLAB_KERNEL_TILED:
      return launch_tiled(s, stream, s.ty, s.tz);
    case MACLAB_KERNEL_FOLDED:
      return launch_fold(s, stream, s.ty, s.tz);
    case MACLAB_KERNEL_ROWS2:
      return launch_rows2(s, stream, s.ty, s.tz);
    case MACLAB_KERNEL_BLOCK:
      return launch_block(s, stream, s.seg_steps);
    case MACLAB_KERNEL_SEGMENT:
      if (!s.seg_inst || !s.seg_items) return cudaErrorInvalidValue;
      if (s.seg_steps == 2)
        return launch_batch_step2(s.precision, s.seg_inst, s.seg_items, s.seg_n_items, s.cur, s.seg_blocks,
                                  stream, s.overlap);
      return launch_batch_step(s.precision, s.seg_inst, s.seg_items, s.seg_n_items, s.cur, s.seg_blocks,
                               s.seg_depth == 2 ? kBatchSegW2 : kBatchSegW1, stream, s.overlap);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace maclab
