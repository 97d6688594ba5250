// lbm.cu -- the stream-and-collide comparator (maclab_lbm_*): the single-
// relaxation-time lattice Boltzmann method of Eq. (1) with the BGK collision,
// on fully periodic D2Q9 grids, storing the nine distributions per node.
//
// State: f[a][y][x] (x fastest) of the post-collision distributions, two
// buffers.  One kernel per step, one thread per node: gather the streamed
// values f_a(x - c_a) (Eq. (1): what left the upstream node along c_a arrives
// here), form rho and u (Eq. (3)) and the equilibria (Eq. (2)), relax by
// omega = 1 / tau and store the nine post-collision values (9 reads and 9
// writes per update).  The collision conserves rho and rho u, so the moments
// of the stored post-collision values are those of the step's distributions.

#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "lattice.cuh"

struct maclab_lbm_ctx {
  int nx = 0, ny = 0, precision = MACLAB_F32;
  double tau = 1.0;
  cudaStream_t stream = nullptr;
  int device = 0;
  void* f[2] = {nullptr, nullptr};
  int cur = 0;
  double* d_stage = nullptr;  // 3 n doubles: rho, u_x, u_y
  int64_t steps = 0;
  int graph_steps = 32;       // steps per captured graph (even)
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
};

namespace maclab {
namespace {

using L9 = Lattice<kD2Q9>;

template <typename C>
__device__ __forceinline__ C lbm_feq(int a, C rho, C ux, C uy, C uu) {
  const C cu = C(L9::c(a, 0)) * ux + C(L9::c(a, 1)) * uy;
  return (C(L9::w36(a)) / C(36)) * rho * (C(1) + C(3) * cu + C(4.5) * cu * cu - C(1.5) * uu);
}

template <typename C>
__global__ void __launch_bounds__(256) lbm_step_k(const C* __restrict__ fin, C* __restrict__ fout, int nx,
                                                  int ny, C omega) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(node / nx);
    const int x = (int)(node - (int64_t)y * nx);
    C f[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      int xs = x - L9::c(a, 0), ys = y - L9::c(a, 1);
      xs += xs < 0 ? nx : (xs >= nx ? -nx : 0);
      ys += ys < 0 ? ny : (ys >= ny ? -ny : 0);
      f[a] = fin[a * n + (int64_t)ys * nx + xs];
    }
    C rho = C(0), mx = C(0), my = C(0);
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      rho += f[a];
      mx += C(L9::c(a, 0)) * f[a];
      my += C(L9::c(a, 1)) * f[a];
    }
    const C ux = mx / rho, uy = my / rho;
    const C uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) fout[a * n + node] = f[a] + omega * (lbm_feq<C>(a, rho, ux, uy, uu) - f[a]);
  }
}

// f = f^eq(rho, u) from the staged doubles
template <typename C>
__global__ void lbm_set_k(const double* __restrict__ stage, C* __restrict__ f, int64_t n) {
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    const C rho = C(stage[node]), ux = C(stage[n + node]), uy = C(stage[2 * n + node]);
    const C uu = ux * ux + uy * uy;
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a * n + node] = lbm_feq<C>(a, rho, ux, uy, uu);
  }
}

// moments of f into the staged doubles
template <typename C>
__global__ void lbm_get_k(const C* __restrict__ f, double* __restrict__ stage, int64_t n) {
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < n;
       node += (int64_t)gridDim.x * blockDim.x) {
    double rho = 0.0, mx = 0.0, my = 0.0;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double fa = (double)f[a * n + node];
      rho += fa;
      mx += L9::c(a, 0) * fa;
      my += L9::c(a, 1) * fa;
    }
    stage[node] = rho;
    stage[n + node] = mx / rho;
    stage[2 * n + node] = my / rho;
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 65536) b = 65536;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t lbm_launch(const maclab_lbm_ctx* h, int from, cudaStream_t st) {
  const int64_t n = (int64_t)h->nx * h->ny;
  if (h->precision == MACLAB_F64)
    lbm_step_k<double><<<grid_for(n), 256, 0, st>>>(static_cast<const double*>(h->f[from]),
                                                     static_cast<double*>(h->f[from ^ 1]), h->nx, h->ny,
                                                     1.0 / h->tau);
  else
    lbm_step_k<float><<<grid_for(n), 256, 0, st>>>(static_cast<const float*>(h->f[from]),
                                                    static_cast<float*>(h->f[from ^ 1]), h->nx, h->ny,
                                                    (float)(1.0 / h->tau));
  return cudaGetLastError();
}

void lbm_drop_graphs(maclab_lbm_ctx* h) {
  for (int c = 0; c < 2; ++c)
    if (h->graph_exec[c]) {
      cudaGraphExecDestroy(h->graph_exec[c]);
      h->graph_exec[c] = nullptr;
    }
}

void lbm_free(maclab_lbm_ctx* h) {
  lbm_drop_graphs(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  cudaFree(h->f[0]);
  cudaFree(h->f[1]);
  cudaFree(h->d_stage);
  delete h;
}

maclab_status lbm_fail(maclab_status s, const char* msg) {
  record_error(msg);
  return s;
}

maclab_status lbm_cuda(cudaError_t e, const char* where) {
  record_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  return MACLAB_ERR_CUDA;
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace maclab

using namespace maclab;

extern "C" {

maclab_status maclab_lbm_create(int32_t nx, int32_t ny, double tau, int32_t precision, void* stream,
                                maclab_lbm* out) {
  if (!out) return lbm_fail(MACLAB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || (int64_t)nx * ny > ((int64_t)1 << 31))
    return lbm_fail(MACLAB_ERR_INVALID, "bad grid size");
  if (!(tau > 0.5) || !(tau < 1e6)) return lbm_fail(MACLAB_ERR_INVALID, "tau must exceed 1/2");
  if (precision != MACLAB_F32 && precision != MACLAB_F64)
    return lbm_fail(MACLAB_ERR_INVALID, "precision must be MACLAB_F32 or MACLAB_F64");
  maclab_lbm_ctx* h = new (std::nothrow) maclab_lbm_ctx();
  if (!h) return lbm_fail(MACLAB_ERR_OOM, "host allocation failed");
  h->nx = nx;
  h->ny = ny;
  h->tau = tau;
  h->precision = precision;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  const int64_t n = (int64_t)nx * ny;
  const size_t fb = (size_t)9 * n * (precision == MACLAB_F64 ? 8 : 4);
  if (cudaMalloc(&h->f[0], fb) != cudaSuccess || cudaMalloc(&h->f[1], fb) != cudaSuccess ||
      cudaMalloc(&h->d_stage, sizeof(double) * 3 * n) != cudaSuccess) {
    cudaGetLastError();
    lbm_free(h);
    return lbm_fail(MACLAB_ERR_OOM, "device allocation failed");
  }
  *out = h;
  return MACLAB_OK;
}

maclab_status maclab_lbm_destroy(maclab_lbm h) {
  if (!h) return MACLAB_OK;
  DeviceScope ds(h->device);
  cudaStreamSynchronize(h->stream);
  lbm_free(h);
  return MACLAB_OK;
}

maclab_status maclab_lbm_set_state(maclab_lbm h, const double* rho, const double* u) {
  if (!h || !rho || !u) return lbm_fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceScope ds(h->device);
  const int64_t n = (int64_t)h->nx * h->ny;
  cudaError_t e = cudaMemcpyAsync(h->d_stage, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_stage + n, u, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return lbm_cuda(e, "lbm set_state upload");
  if (h->precision == MACLAB_F64)
    lbm_set_k<double><<<grid_for(n), 256, 0, h->stream>>>(h->d_stage, static_cast<double*>(h->f[h->cur]), n);
  else
    lbm_set_k<float><<<grid_for(n), 256, 0, h->stream>>>(h->d_stage, static_cast<float*>(h->f[h->cur]), n);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return lbm_cuda(e, "lbm set_state");
  h->steps = 0;
  return MACLAB_OK;
}

maclab_status maclab_lbm_step(maclab_lbm h, int64_t n) {
  if (!h) return lbm_fail(MACLAB_ERR_INVALID, "NULL handle");
  if (n < 0) return lbm_fail(MACLAB_ERR_INVALID, "n must be >= 0");
  DeviceScope ds(h->device);
  // runs of graph_steps steps replay a captured graph (even length: it ends on
  // the buffer it started from)
  while (n >= h->graph_steps) {
    cudaGraphExec_t& ge = h->graph_exec[h->cur];
    if (!ge) {
      if (!h->capture_stream &&
          cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        return lbm_cuda(cudaGetLastError(), "lbm capture stream");
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return lbm_cuda(e, "lbm begin capture");
      cudaError_t err = cudaSuccess;
      for (int k = 0; k < h->graph_steps && err == cudaSuccess; ++k)
        err = lbm_launch(h, h->cur ^ (k & 1), h->capture_stream);
      e = cudaStreamEndCapture(h->capture_stream, &graph);
      if (err != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return lbm_cuda(err != cudaSuccess ? err : e, "lbm graph capture");
      }
      e = cudaGraphInstantiate(&ge, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        ge = nullptr;
        return lbm_cuda(e, "lbm graph instantiate");
      }
    }
    cudaError_t e = cudaGraphLaunch(ge, h->stream);
    if (e != cudaSuccess) return lbm_cuda(e, "lbm graph launch");
    n -= h->graph_steps;
    h->steps += h->graph_steps;
  }
  for (; n > 0; --n) {
    cudaError_t e = lbm_launch(h, h->cur, h->stream);
    if (e != cudaSuccess) return lbm_cuda(e, "lbm step launch");
    h->cur ^= 1;
    h->steps += 1;
  }
  return MACLAB_OK;
}

maclab_status maclab_lbm_get_state(maclab_lbm h, double* rho, double* u) {
  if (!h || !rho || !u) return lbm_fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceScope ds(h->device);
  const int64_t n = (int64_t)h->nx * h->ny;
  if (h->precision == MACLAB_F64)
    lbm_get_k<double><<<grid_for(n), 256, 0, h->stream>>>(static_cast<const double*>(h->f[h->cur]), h->d_stage, n);
  else
    lbm_get_k<float><<<grid_for(n), 256, 0, h->stream>>>(static_cast<const float*>(h->f[h->cur]), h->d_stage, n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(rho, h->d_stage, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(u, h->d_stage + n, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return lbm_cuda(e, "lbm get_state");
  return MACLAB_OK;
}

maclab_status maclab_lbm_info(maclab_lbm h, int64_t out[4]) {
  if (!h || !out) return lbm_fail(MACLAB_ERR_INVALID, "NULL argument");
  const int64_t n = (int64_t)h->nx * h->ny;
  const int64_t b = h->precision == MACLAB_F64 ? 8 : 4;
  out[0] = n;
  out[1] = 2 * 9 * n * b;
  out[2] = 2 * 9 * b;
  out[3] = h->steps;
  return MACLAB_OK;
}

}  // extern "C"
