// api.cu -- the C ABI of libmaclab (declared in include/maclab.h).
//
// Host-side only: validation, the unit conversion of procedure step (i)
// (e = 6 nu / dx, Eq. (6); dt = dx / e), buffer ownership and launches.  All
// arithmetic on fields happens in the kernels of step.cu / convert.cu.

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <map>
#include <mutex>
#include <new>
#include <iterator>
#include <string>

#include "common.cuh"
#include "lattice.cuh"

namespace {

// Scoped NVTX range (shows the C-ABI calls on a profiler's timeline; no cost
// without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace

using namespace maclab;

namespace {

thread_local std::string g_last_error;

maclab_status fail(maclab_status s, const char* msg) {
  g_last_error = msg;
  return s;
}

maclab_status cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return MACLAB_ERR_CUDA;
}

#define CUDA_TRY(call, where)                       \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool on_closed_boundary(const Geometry& g, int64_t x, int64_t y, int64_t z) {
  if (!(g.periodic & 1u) && (x == 0 || x == g.nx - 1)) return true;
  if (!(g.periodic & 2u) && (y == 0 || y == g.ny - 1)) return true;
  if (g.d == 3 && !(g.periodic & 4u) && (z == 0 || z == g.nz - 1)) return true;
  return false;
}

void drop_graphs(maclab_ctx* h) {
  for (int c = 0; c < 2; ++c)
    if (h->graph_exec[c]) {
      cudaGraphExecDestroy(h->graph_exec[c]);
      h->graph_exec[c] = nullptr;
    }
}

void free_ctx(maclab_ctx* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  cudaFree(h->d_partial);
  cudaFree(h->d_diag);
  if (h->h_diag) cudaFreeHost(h->h_diag);
  cudaFree(h->d_adj_scratch);
  cudaFree(h->d_adj_red);
  cudaFree(h->d_seg_inst);
  cudaFree(h->d_seg_items);
  cudaFree(h->d_seg_deps);
  cudaFree(h->d_seg_done);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->d_node_type);
  cudaFree(h->d_wall_lat);
  cudaFree(h->d_staging);
  delete h;
}

maclab_status ensure_staging(maclab_ctx* h, size_t bytes) {
  if (h->staging_cap >= bytes) return MACLAB_OK;
  cudaFree(h->d_staging);
  h->d_staging = nullptr;
  h->staging_cap = 0;
  if (cudaMalloc(&h->d_staging, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(MACLAB_ERR_OOM, "staging allocation failed");
  }
  h->staging_cap = bytes;
  return MACLAB_OK;
}

size_t state_bytes(const maclab_ctx* h) { return (size_t)(h->g.d + 1) * (size_t)h->g.n * h->elem; }

// Copy the current buffer onto the other one so that both hold the same wall
// values (wall nodes are never written by the step kernels).
maclab_status mirror_buffers(maclab_ctx* h) {
  CUDA_TRY(cudaMemcpyAsync(h->buf[h->cur ^ 1], h->buf[h->cur], state_bytes(h),
                           cudaMemcpyDeviceToDevice, h->stream),
           "mirror state");
  return MACLAB_OK;
}

}  // namespace

void maclab::record_error(const char* msg) { g_last_error = msg; }

extern "C" {

const char* maclab_status_string(maclab_status s) {
  switch (s) {
    case MACLAB_OK: return "MACLAB_OK";
    case MACLAB_WARN_RLE: return "MACLAB_WARN_RLE: lattice Reynolds number above 1";
    case MACLAB_ERR_INVALID: return "MACLAB_ERR_INVALID: invalid argument";
    case MACLAB_ERR_CUDA: return "MACLAB_ERR_CUDA: CUDA error";
    case MACLAB_ERR_NONFINITE: return "MACLAB_ERR_NONFINITE: non-finite value in the state";
    case MACLAB_ERR_TIMEOUT: return "MACLAB_ERR_TIMEOUT: bounded device wait expired";
    case MACLAB_ERR_OOM: return "MACLAB_ERR_OOM: allocation failed";
    case MACLAB_ERR_UNSUPPORTED: return "MACLAB_ERR_UNSUPPORTED: not supported by this library";
  }
  return "unknown maclab_status";
}

const char* maclab_version(void) { return "maclab sm_103a"; }

maclab_status maclab_check_reciprocal(float lo, float hi, int32_t n, double* max_rel_err) {
  if (!max_rel_err) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (!(lo > 0.0f) || !(hi > lo) || !isfinite(hi) || n < 1 || n > (1 << 24))
    return fail(MACLAB_ERR_INVALID, "need 0 < lo < hi (finite) and 1 <= n <= 2^24");
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MACLAB_ERR_OOM, "reciprocal check allocation failed");
  }
  unsigned long long bits = 0;
  cudaError_t e = cudaMemset(d, 0, sizeof(bits));
  if (e == cudaSuccess) e = launch_check_reciprocal(lo, hi, n, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "reciprocal check");
  double v;
  memcpy(&v, &bits, sizeof(v));
  *max_rel_err = v;
  return MACLAB_OK;
}

maclab_status maclab_measure_fp32_peak(double* tflops) {
  if (!tflops) return fail(MACLAB_ERR_INVALID, "NULL argument");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return cuda_fail(cudaGetLastError(), "device query");
  float2* sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MACLAB_ERR_OOM, "peak measurement allocation failed");
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double flops = 0, best = 0;
  cudaError_t e = cudaSuccess;
  // 8 blocks of 256 threads per SM (full occupancy); warm-up, then the best of 3
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, nullptr);
    e = launch_fp32_peak(8 * sms, 256, 1 << 14, sink, nullptr, &flops);
    cudaEventRecord(b, nullptr);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && rep > 0 && ms > 0) best = fmax(best, flops / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "peak measurement");
  *tflops = best;
  return MACLAB_OK;
}

const char* maclab_last_error(void) { return g_last_error.c_str(); }

maclab_status maclab_create(const maclab_config* cfg, maclab_handle* out) {
  if (!out) return fail(MACLAB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(MACLAB_ERR_INVALID, "cfg is NULL");
  if (cfg->lattice != MACLAB_D2Q9 && cfg->lattice != MACLAB_D3Q19)
    return fail(MACLAB_ERR_INVALID, "unknown lattice");
  if (cfg->precision < MACLAB_F64 || cfg->precision > MACLAB_F16_STORE)
    return fail(MACLAB_ERR_INVALID, "unknown precision");
  const int d = cfg->lattice == MACLAB_D2Q9 ? 2 : 3;
  const int64_t nx = cfg->dims[0], ny = cfg->dims[1], nz = cfg->dims[2];
  if (nx < 1 || ny < 1 || nz < 1) return fail(MACLAB_ERR_INVALID, "dims must be >= 1");
  if (d == 2 && nz != 1) return fail(MACLAB_ERR_INVALID, "D2Q9 needs dims[2] == 1");
  if (nx > (1 << 30) || ny > (1 << 30) || nz > (1 << 30))
    return fail(MACLAB_ERR_INVALID, "dimension too large");
  const int64_t N = nx * ny * nz;
  if (N > ((int64_t)1 << 40)) return fail(MACLAB_ERR_INVALID, "too many nodes");
  if (!(cfg->dx > 0) || !(cfg->nu > 0) || !isfinite(cfg->dx) || !isfinite(cfg->nu))
    return fail(MACLAB_ERR_INVALID, "dx and nu must be finite and > 0");
  if (cfg->n_wall_ids < 0 || cfg->n_wall_ids > 255)
    return fail(MACLAB_ERR_INVALID, "n_wall_ids must be in 0..255");
  if (cfg->n_wall_ids > 0 && !cfg->wall_u)
    return fail(MACLAB_ERR_INVALID, "wall_u is NULL");
  for (int i = 0; i < 3; ++i)
    if (!isfinite(cfg->body_force[i])) return fail(MACLAB_ERR_INVALID, "body_force not finite");

  maclab_ctx* h = new (std::nothrow) maclab_ctx();
  if (!h) return fail(MACLAB_ERR_OOM, "host allocation failed");
  Geometry& g = h->g;
  g.lattice = cfg->lattice == MACLAB_D2Q9 ? kD2Q9 : kD3Q19;
  g.d = d;
  g.nx = (int)nx;
  g.ny = (int)ny;
  g.nz = (int)nz;
  g.n = N;
  g.periodic = cfg->periodic & (d == 2 ? 3u : 7u);
  g.ilv = (nx % 4 == 0) ? 1 : 0;
  g.hx = (int)(nx / 2);
  h->precision = cfg->precision;
  h->elem = storage_bytes(cfg->precision);
  h->dx = cfg->dx;
  h->nu = cfg->nu;
  h->rho0 = cfg->rho0 > 0 ? cfg->rho0 : 1.0;
  h->e = 6.0 * cfg->nu / cfg->dx;  // Eq. (6)
  h->dt = cfg->dx / h->e;
  h->stream = (cudaStream_t)cfg->stream;
  cudaGetDevice(&h->device);
  for (int i = 0; i < 3; ++i) {
    h->force_phys[i] = i < d ? cfg->body_force[i] : 0.0;
    h->force_lat[i] = h->force_phys[i] * h->dt / h->e;
  }

  // wall tables
  h->n_wall_ids = cfg->n_wall_ids;
  double umax = 0;
  for (int k = 0; k < h->n_wall_ids; ++k) {
    const double r = cfg->wall_rho ? cfg->wall_rho[k] : h->rho0;
    if (!(r > 0) || !isfinite(r)) { free_ctx(h); return fail(MACLAB_ERR_INVALID, "wall_rho must be > 0"); }
    h->wall_rho.push_back(r);
    h->wall_lat.push_back(r / h->rho0 - 1.0);
    double s = 0;
    for (int i = 0; i < 3; ++i) {
      const double v = cfg->wall_u[3 * k + i];
      if (!isfinite(v)) { free_ctx(h); return fail(MACLAB_ERR_INVALID, "wall_u not finite"); }
      h->wall_u.push_back(v);
      h->wall_lat.push_back(i < d ? v / h->e : 0.0);
      if (i < d) s += v * v;
    }
    umax = fmax(umax, sqrt(s));
  }
  h->rle = umax * cfg->dx / cfg->nu;

  // node types: validate, classify (none / box / mask)
  int64_t n_wall = 0;
  bool box = true;
  if (cfg->node_type) {
    for (int64_t z = 0, i = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x, ++i) {
          const int k = cfg->node_type[i];
          if (k > h->n_wall_ids) { free_ctx(h); return fail(MACLAB_ERR_INVALID, "node_type id out of range"); }
          const bool closed = on_closed_boundary(g, x, y, z);
          if (closed && k == 0) {
            free_ctx(h);
            return fail(MACLAB_ERR_INVALID,
                        "fluid node on the outer layer of a non-periodic axis (needs a wall)");
          }
          if ((k != 0) != closed) box = false;
          n_wall += k != 0;
        }
  } else {
    for (int i = 0; i < d; ++i)
      if (!((g.periodic >> i) & 1u)) {
        free_ctx(h);
        return fail(MACLAB_ERR_INVALID, "non-periodic axis without a node_type mask");
      }
  }
  h->n_fluid = N - n_wall;
  g.wall_mode = n_wall == 0 ? kWallNone : (box ? kWallBox : kWallMask);

  DeviceGuard dg(h->device);
  const size_t sb = state_bytes(h);
  h->diag_nblocks = diag_blocks(N);
  if (cudaMalloc(&h->buf[0], sb) != cudaSuccess || cudaMalloc(&h->buf[1], sb) != cudaSuccess ||
      cudaMalloc(&h->d_partial, sizeof(double) * (kDiagOut * h->diag_nblocks + 1)) != cudaSuccess ||
      cudaMalloc(&h->d_diag, sizeof(double) * kDiagOut) != cudaSuccess ||
      cudaHostAlloc(&h->h_diag, sizeof(double) * kDiagOut, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(h);
    return fail(MACLAB_ERR_OOM, "state allocation failed");
  }
  // the step kernels' status word exists before any launch or graph capture
  if (!step_status()) {
    free_ctx(h);
    return fail(MACLAB_ERR_OOM, "status word allocation failed");
  }
  // the diagnostics kernel's ticket counter (after the block records) starts at 0
  if (cudaMemsetAsync(h->d_partial + kDiagOut * h->diag_nblocks, 0, sizeof(double), h->stream) != cudaSuccess) {
    cudaGetLastError();
    free_ctx(h);
    return fail(MACLAB_ERR_CUDA, "diagnostics scratch initialisation failed");
  }
  if (n_wall > 0) {
    if (cudaMalloc(&h->d_node_type, (size_t)N) != cudaSuccess ||
        cudaMalloc(&h->d_wall_lat, sizeof(double) * h->wall_lat.size()) != cudaSuccess) {
      cudaGetLastError();
      free_ctx(h);
      return fail(MACLAB_ERR_OOM, "mask allocation failed");
    }
    // device copy in storage order
    std::vector<uint8_t> nt_mem((size_t)N);
    for (int64_t row = 0; row < N / nx; ++row)
      for (int64_t x = 0; x < nx; ++x)
        nt_mem[(size_t)(row * nx + mem_x(g, (int)x))] = cfg->node_type[row * nx + x];
    cudaError_t e1 = cudaMemcpy(h->d_node_type, nt_mem.data(), (size_t)N, cudaMemcpyHostToDevice);
    cudaError_t e2 = cudaMemcpy(h->d_wall_lat, h->wall_lat.data(),
                                sizeof(double) * h->wall_lat.size(), cudaMemcpyHostToDevice);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      free_ctx(h);
      return cuda_fail(e1 != cudaSuccess ? e1 : e2, "mask upload");
    }
  }
  g.mask = g.wall_mode == kWallMask ? h->d_node_type : nullptr;

  // rest state with the wall values in place, in both buffers
  cudaError_t e = cudaMemsetAsync(h->buf[0], 0, sb, h->stream);
  if (e == cudaSuccess)
    e = launch_fill_walls(g, h->precision, h->d_node_type, h->d_wall_lat, h->n_wall_ids, h->buf[0],
                          h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->buf[1], h->buf[0], sb, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    free_ctx(h);
    return cuda_fail(e, "initial state");
  }
  h->kernel = pick_step_kernel(g, h->precision);
  *out = h;
  return h->rle > 1.0 ? MACLAB_WARN_RLE : MACLAB_OK;
}

maclab_status maclab_destroy(maclab_handle h) {
  if (!h) return MACLAB_OK;
  DeviceGuard dg(h->device);
  cudaStreamSynchronize(h->stream);
  free_ctx(h);
  return MACLAB_OK;
}

maclab_status maclab_params(maclab_handle h, double out[8]) {
  if (!h || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  out[0] = h->e;
  out[1] = h->dt;
  out[2] = h->rle;
  out[3] = h->force_lat[0];
  out[4] = h->force_lat[1];
  out[5] = h->force_lat[2];
  out[6] = (double)h->n_fluid;
  out[7] = (double)h->steps;
  return MACLAB_OK;
}

maclab_status maclab_state_bytes(maclab_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(MACLAB_ERR_INVALID, "NULL argument");
  *bytes = state_bytes(h);
  return MACLAB_OK;
}

// Device address of page-locked host memory mapped for this device (pinned
// with cudaHostAlloc or cudaHostRegister), else nullptr: the conversion
// kernels then read or write the caller's buffer directly over the host link
// instead of going through the staging buffer and a copy.
static void* pinned_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || a.device != device) return nullptr;
  return a.devicePointer;
}

maclab_status maclab_set_state(maclab_handle h, const void* rho, const void* u, int32_t where,
                               int32_t dtype) {
  NvtxRange nvtx_range("maclab_set_state");
  if (!h || !rho || !u) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (dtype != MACLAB_DTYPE_F64 && dtype != MACLAB_DTYPE_F32)
    return fail(MACLAB_ERR_INVALID, "dtype must be F64 or F32");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  DeviceGuard dg(h->device);
  const size_t es = dtype == MACLAB_DTYPE_F64 ? 8 : 4;
  const size_t nb = (size_t)h->g.n * es;
  const void* r = rho;
  const void* v = u;
  const void* pr = where == MACLAB_HOST ? pinned_device_ptr(rho, h->device) : nullptr;
  const void* pu = pr ? pinned_device_ptr(u, h->device) : nullptr;
  if (pr && pu) {
    r = pr;
    v = pu;
  } else if (where == MACLAB_HOST) {
    maclab_status s = ensure_staging(h, nb * (h->g.d + 1));
    if (s != MACLAB_OK) return s;
    char* st = (char*)h->d_staging;
    CUDA_TRY(cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, h->stream), "set_state H2D");
    CUDA_TRY(cudaMemcpyAsync(st + nb, u, nb * h->g.d, cudaMemcpyHostToDevice, h->stream),
             "set_state H2D");
    r = st;
    v = st + nb;
  }
  CUDA_TRY(launch_set_physical(h->g, h->precision, r, v, dtype, h->rho0, h->e, h->d_node_type,
                               h->d_wall_lat, h->n_wall_ids, h->buf[h->cur], h->stream),
           "set_state kernel");
  maclab_status s = mirror_buffers(h);
  if (s != MACLAB_OK) return s;
  h->steps = 0;
  h->prev_valid = false;
  if (where == MACLAB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream), "set_state sync");
  return MACLAB_OK;
}

maclab_status maclab_set_wall_state(maclab_handle h, const void* rho, const void* u, int32_t where,
                                    int32_t dtype) {
  NvtxRange nvtx_range("maclab_set_wall_state");
  if (!h || !rho || !u) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (dtype != MACLAB_DTYPE_F64 && dtype != MACLAB_DTYPE_F32)
    return fail(MACLAB_ERR_INVALID, "dtype must be F64 or F32");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  if (!h->d_node_type) return MACLAB_OK;  // no wall nodes
  DeviceGuard dg(h->device);
  const size_t es = dtype == MACLAB_DTYPE_F64 ? 8 : 4;
  const size_t nb = (size_t)h->g.n * es;
  const void* r = rho;
  const void* v = u;
  const void* pr = where == MACLAB_HOST ? pinned_device_ptr(rho, h->device) : nullptr;
  const void* pu = pr ? pinned_device_ptr(u, h->device) : nullptr;
  if (pr && pu) {
    r = pr;
    v = pu;
  } else if (where == MACLAB_HOST) {
    maclab_status s = ensure_staging(h, nb * (h->g.d + 1));
    if (s != MACLAB_OK) return s;
    char* st = (char*)h->d_staging;
    CUDA_TRY(cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, h->stream), "set_wall_state H2D");
    CUDA_TRY(cudaMemcpyAsync(st + nb, u, nb * h->g.d, cudaMemcpyHostToDevice, h->stream),
             "set_wall_state H2D");
    r = st;
    v = st + nb;
  }
  CUDA_TRY(launch_set_wall_values(h->g, h->precision, r, v, dtype, h->rho0, h->e, h->d_node_type,
                                  h->buf[0], h->buf[1], h->stream),
           "set_wall_state kernel");
  if (where == MACLAB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream), "set_wall_state sync");
  return MACLAB_OK;
}

maclab_status maclab_get_state(maclab_handle h, void* rho, void* u, int32_t where, int32_t dtype) {
  NvtxRange nvtx_range("maclab_get_state");
  if (!h || !rho || !u) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (dtype != MACLAB_DTYPE_F64 && dtype != MACLAB_DTYPE_F32)
    return fail(MACLAB_ERR_INVALID, "dtype must be F64 or F32");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  DeviceGuard dg(h->device);
  const size_t es = dtype == MACLAB_DTYPE_F64 ? 8 : 4;
  const size_t nb = (size_t)h->g.n * es;
  void* pr = where == MACLAB_HOST ? pinned_device_ptr(rho, h->device) : nullptr;
  void* pu = pr ? pinned_device_ptr(u, h->device) : nullptr;
  if (where == MACLAB_DEVICE || (pr && pu)) {
    CUDA_TRY(launch_get_physical(h->g, h->precision, h->buf[h->cur], pr ? pr : rho, pu ? pu : u, dtype,
                                 h->rho0, h->e, h->stream),
             "get_state kernel");
  } else {
    maclab_status s = ensure_staging(h, nb * (h->g.d + 1));
    if (s != MACLAB_OK) return s;
    char* st = (char*)h->d_staging;
    CUDA_TRY(launch_get_physical(h->g, h->precision, h->buf[h->cur], st, st + nb, dtype, h->rho0,
                                 h->e, h->stream),
             "get_state kernel");
    CUDA_TRY(cudaMemcpyAsync(rho, st, nb, cudaMemcpyDeviceToHost, h->stream), "get_state D2H");
    CUDA_TRY(cudaMemcpyAsync(u, st + nb, nb * h->g.d, cudaMemcpyDeviceToHost, h->stream),
             "get_state D2H");
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream), "get_state sync");
  return MACLAB_OK;
}

maclab_status maclab_get_lattice_state(maclab_handle h, void* state, int32_t where) {
  if (!h || !state) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  DeviceGuard dg(h->device);
  CUDA_TRY(cudaMemcpyAsync(state, h->buf[h->cur], state_bytes(h),
                           where == MACLAB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           h->stream),
           "get_lattice_state");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "get_lattice_state sync");
  return MACLAB_OK;
}

maclab_status maclab_set_lattice_state(maclab_handle h, const void* state, int32_t where) {
  if (!h || !state) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  DeviceGuard dg(h->device);
  CUDA_TRY(cudaMemcpyAsync(h->buf[h->cur], state, state_bytes(h),
                           where == MACLAB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           h->stream),
           "set_lattice_state");
  maclab_status s = mirror_buffers(h);
  if (s != MACLAB_OK) return s;
  h->prev_valid = false;
  if (where == MACLAB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream), "set_lattice_state sync");
  return MACLAB_OK;
}

// The diagnostics kernel's ticket counter: the word after the handle's block records.
static unsigned* diag_ticket(const maclab_ctx* h) {
  return reinterpret_cast<unsigned*>(h->d_partial + kDiagOut * h->diag_nblocks);
}

static StepLaunch step_launch(const maclab_ctx* h, int from) {
  StepLaunch s;
  s.g = h->g;
  s.precision = h->precision;
  for (int i = 0; i < 3; ++i) s.force[i] = h->force_lat[i];
  s.ty = h->ty;
  s.tz = h->tz;
  s.in = h->buf[from];
  s.out = h->buf[from ^ 1];
  s.seg_inst = h->d_seg_inst;
  s.seg_items = h->d_seg_items;
  s.seg_n_items = h->seg_n_items;
  s.seg_blocks = h->seg_blocks;
  s.cur = from;
  s.seg_depth = h->seg_depth;
  s.seg_steps = h->kernel == MACLAB_KERNEL_SEGMENT ? h->seg_depth
                : h->kernel == MACLAB_KERNEL_BLOCK ? block_steps(h->g, h->precision, h->ty)
                                                   : 1;
  s.overlap = h->overlap;
  return s;
}

// Time steps one launch of the handle's kernel advances.
static int launch_depth(const maclab_ctx* h) {
  if (h->kernel == MACLAB_KERNEL_BLOCK) return block_steps(h->g, h->precision, h->ty);
  return h->kernel == MACLAB_KERNEL_SEGMENT ? h->seg_depth : 1;
}

static int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  }
  return sms;
}

// The segment kernel's descriptor of this domain and its work list for the
// current rows per item (tz, default 4) and steps per launch (ty: 2 for two,
// else one), built on first use and after a change of either; graphs captured
// with the old list are dropped.  Synchronises the handle's stream when it
// uploads.
// The persistent form's wait lists (segment kernel, ty 3): as many blocks as
// fit at once, each with the list of blocks it waits for between sweeps.
// Built on first use for the current work list.
static maclab_status segment_persist_prepare(maclab_ctx* h) {
  if (h->seg_persist_blocks > 0 || h->seg_depth != 2) return MACLAB_OK;
  int capacity = 0;
  if (batch_persist_capacity(h->precision, &capacity) != cudaSuccess || capacity < 1) {
    cudaGetLastError();
    return MACLAB_OK;  // the form is unavailable; stepping uses graphs of launches
  }
  const int want = (h->seg_n_items + 3) / 4;
  const int pb = want < capacity ? (want > 0 ? want : 1) : capacity;
  std::vector<int> deps;
  batch_persist_deps(h->seg_items_host, {(int)h->g.ny}, {(h->g.periodic & 2u) != 0 ? 1 : 0}, pb, deps);
  if (cudaMalloc(&h->d_seg_deps, deps.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->d_seg_done, (size_t)pb * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->d_seg_deps);
    h->d_seg_deps = nullptr;
    return fail(MACLAB_ERR_OOM, "persistent segment lists allocation failed");
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_seg_deps, deps.data(), deps.size() * sizeof(int), cudaMemcpyHostToDevice,
                           h->stream),
           "persistent segment lists upload");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "persistent segment lists sync");
  h->seg_persist_blocks = pb;
  return MACLAB_OK;
}

// The segment kernel's descriptor and work list for the current tile setting
// (rows per item and steps per launch), rebuilt when they change, and for the
// persistent form (ty 3) its wait lists.
static maclab_status segment_prepare(maclab_ctx* h) {
  if (h->kernel != MACLAB_KERNEL_SEGMENT) return MACLAB_OK;
  const int rows = segment_rows(h->g, h->precision, h->ty, h->tz);
  const int depth = segment_depth(h->g, h->precision, h->ty);
  if (!(h->d_seg_inst && h->d_seg_items && h->seg_rows == rows && h->seg_depth == depth)) {
    if (!h->d_seg_inst) {
      if (cudaMalloc(&h->d_seg_inst, batch_inst_bytes()) != cudaSuccess) {
        cudaGetLastError();
        h->d_seg_inst = nullptr;
        return fail(MACLAB_ERR_OOM, "segment descriptor allocation failed");
      }
    }
    std::vector<unsigned char> inst(batch_inst_bytes());
    batch_fill_inst(inst.data(), h->g, h->buf[0], h->buf[1], h->force_lat);
    std::vector<int> items;
    batch_items(0, h->g, rows, depth, items);
    void* d = nullptr;
    if (cudaMalloc(&d, items.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(MACLAB_ERR_OOM, "segment work list allocation failed");
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_seg_inst, inst.data(), inst.size(), cudaMemcpyHostToDevice, h->stream),
             "segment descriptor upload");
    CUDA_TRY(cudaMemcpyAsync(d, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream),
             "segment work list upload");
    CUDA_TRY(cudaStreamSynchronize(h->stream), "segment upload sync");
    cudaFree(h->d_seg_items);
    h->d_seg_items = d;
    h->seg_n_items = (int)(items.size() / 4);
    h->seg_items_host.swap(items);
    h->seg_rows = rows;
    h->seg_depth = depth;
    // one step per launch: 256-thread blocks, two per SM; two: 128-thread blocks, three per SM
    const int warps = depth == 2 ? 4 : 8, per_sm = depth == 2 ? 3 : 2;
    const int want = (h->seg_n_items + warps - 1) / warps;
    h->seg_blocks = want < per_sm * device_sms() ? (want > 0 ? want : 1) : per_sm * device_sms();
    drop_graphs(h);
    cudaFree(h->d_seg_deps);
    cudaFree(h->d_seg_done);
    h->d_seg_deps = nullptr;
    h->d_seg_done = nullptr;
    h->seg_persist_blocks = 0;
  }
  return h->ty == 3 ? segment_persist_prepare(h) : MACLAB_OK;
}

// Capture graph_steps / depth launches (graph_steps steps) starting from
// buffer c; with an odd number of launches the graph ends on buffer c ^ 1.
static maclab_status build_graph(maclab_ctx* h, int c) {
  if (!h->capture_stream) {
    if (cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "capture stream");
  }
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed), "begin capture");
  cudaError_t err = cudaSuccess;
  const int launches = h->graph_steps / launch_depth(h);
  for (int k = 0; k < launches && err == cudaSuccess; ++k)
    err = launch_step(step_launch(h, c ^ (k & 1)), h->capture_stream, h->kernel);
  cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(err != cudaSuccess ? err : e2, "graph capture");
  }
  err = cudaGraphInstantiate(&h->graph_exec[c], graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    h->graph_exec[c] = nullptr;
    return cuda_fail(err, "graph instantiate");
  }
  return MACLAB_OK;
}

maclab_status maclab_step(maclab_handle h, int64_t n) {
  NvtxRange nvtx_range("maclab_step");
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  if (n < 0) return fail(MACLAB_ERR_INVALID, "n must be >= 0");
  DeviceGuard dg(h->device);
  maclab_status ps = segment_prepare(h);
  if (ps != MACLAB_OK) return ps;
  // With two steps per launch the last step is a one-step launch, so that the
  // other buffer holds step n - 1 (the steady residual reads it).
  const int k = launch_depth(h);
  const int64_t bulk = k > 1 && n > 0 ? n - 1 : n;
  const int launches = h->graph_steps / k;
  const int64_t gsteps = (int64_t)launches * k;
  int64_t done = 0;
  // the persistent segment form (ty 3): the bulk's step pairs in one
  // cooperative launch per call instead of graphs of launches
  const bool persist = h->kernel == MACLAB_KERNEL_SEGMENT && h->ty == 3 && k == 2 && h->seg_persist_blocks > 0;
  for (int64_t pairs = persist ? bulk / 2 : 0; pairs > 0;) {
    const int sweeps = pairs > (1 << 30) ? (1 << 30) : (int)pairs;
    CUDA_TRY(launch_batch_step2_persist(h->precision, h->d_seg_inst, h->d_seg_items, h->seg_n_items, h->cur,
                                        h->seg_persist_blocks, sweeps, h->d_seg_deps, h->d_seg_done,
                                        step_status(), h->wait_limit, h->stream),
             "persistent step launch");
    if (sweeps & 1) h->cur ^= 1;
    done += 2 * (int64_t)sweeps;
    pairs -= sweeps;
  }
  while (!persist && gsteps > 0 && bulk - done >= gsteps) {
    if (!h->graph_exec[h->cur]) {
      maclab_status s = build_graph(h, h->cur);
      if (s != MACLAB_OK) return s;
    }
    CUDA_TRY(cudaGraphLaunch(h->graph_exec[h->cur], h->stream), "graph launch");
    if (launches & 1) h->cur ^= 1;
    done += gsteps;
  }
  for (; bulk - done >= k; done += k) {
    CUDA_TRY(launch_step(step_launch(h, h->cur), h->stream, h->kernel), "step launch");
    h->cur ^= 1;
  }
  for (; done < n; ++done) {
    StepLaunch sl = step_launch(h, h->cur);
    sl.seg_steps = 1;
    CUDA_TRY(launch_step(sl, h->stream, h->kernel), "step launch");
    h->cur ^= 1;
  }
  h->steps += n;
  if (n > 0) h->prev_valid = true;
  return MACLAB_OK;
}

maclab_status maclab_set_graph(maclab_handle h, int32_t steps) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  if (steps < 0 || steps > (1 << 20)) return fail(MACLAB_ERR_INVALID, "bad graph length");
  DeviceGuard dg(h->device);
  drop_graphs(h);
  h->graph_steps = steps + (steps & 1);
  return MACLAB_OK;
}

static size_t adjoint_bytes(const maclab_ctx* h) {
  return (size_t)(h->g.d + 1) * (size_t)h->g.n * (h->precision == MACLAB_F64 ? 8 : 4);
}

// records: the per-node (L_r, L_m) buffer that only the reference kernels use
static maclab_status ensure_adjoint(maclab_ctx* h, bool records = false) {
  if (records && !h->d_adj_scratch) {
    // one 4-value record per node
    const size_t rec = 4 * (size_t)h->g.n * (h->precision == MACLAB_F64 ? 8 : 4);
    if (cudaMalloc(&h->d_adj_scratch, rec) != cudaSuccess) {
      cudaGetLastError();
      h->d_adj_scratch = nullptr;
      return fail(MACLAB_ERR_OOM, "adjoint scratch allocation failed");
    }
  }
  if (!h->d_adj_red) {
    if (cudaMalloc(&h->d_adj_red, sizeof(double) * (1 + 4 * (size_t)h->n_wall_ids)) != cudaSuccess) {
      cudaGetLastError();
      h->d_adj_red = nullptr;
      return fail(MACLAB_ERR_OOM, "adjoint scratch allocation failed");
    }
  }
  return MACLAB_OK;
}

maclab_status maclab_adjoint_bytes(maclab_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(MACLAB_ERR_INVALID, "NULL argument");
  *bytes = adjoint_bytes(h);
  return MACLAB_OK;
}

maclab_status maclab_adjoint_step(maclab_handle h, const void* state_n, const void* state_np1,
                                  const void* lam_np1, void* lam_n, double* grad_force) {
  NvtxRange nvtx_range("maclab_adjoint_step");
  if (!h || !state_n || !state_np1 || !lam_np1 || !lam_n) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (lam_n == lam_np1) return fail(MACLAB_ERR_INVALID, "lam_n must not alias lam_np1");
  DeviceGuard dg(h->device);
  // the tiled reverse step where it is built (unless the reference kernel was chosen)
  const bool tiled = h->kernel != MACLAB_KERNEL_REFERENCE && tiled_adjoint_supported(h->g, h->precision);
  maclab_status s = ensure_adjoint(h, !tiled);
  if (s != MACLAB_OK) return s;
  if (tiled) {
    CUDA_TRY(launch_tiled_adjoint(h->g, h->precision, state_n, state_np1, lam_np1, lam_n,
                                  h->force_lat, grad_force, h->overlap, h->stream),
             "adjoint step");
  } else {
    CUDA_TRY(launch_adjoint_step(h->g, h->precision, state_n, state_np1, lam_np1, lam_n,
                                 h->d_adj_scratch, h->force_lat, grad_force, h->stream),
             "adjoint step");
  }
  return MACLAB_OK;
}

maclab_status maclab_adjoint_nu_term(maclab_handle h, const void* state_n, const void* state_np1,
                                     const void* lam_np1, double* acc) {
  NvtxRange nvtx_range("maclab_adjoint_nu_term");
  if (!h || !state_n || !lam_np1 || !acc) return fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceGuard dg(h->device);
  auto aligned = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
  if (state_np1 && h->kernel != MACLAB_KERNEL_REFERENCE && rows2_nu_supported(h->g, h->precision) &&
      aligned(state_n) && aligned(state_np1) && aligned(lam_np1)) {
    CUDA_TRY(launch_rows2_nu(h->g, state_n, state_np1, static_cast<const float*>(lam_np1), h->force_lat, acc,
                             h->overlap, h->stream),
             "adjoint nu term (two-rows kernel)");
    return MACLAB_OK;
  }
  CUDA_TRY(launch_adjoint_nu_term(h->g, h->precision, state_n, lam_np1, h->force_lat, acc, h->stream),
           "adjoint nu term");
  return MACLAB_OK;
}

maclab_status maclab_adjoint_seed(maclab_handle h, const void* grad_rho, const void* grad_u,
                                  int32_t dtype, const void* state_T, void* lam_T, double* dot_T) {
  if (!h || !state_T || !lam_T) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (dtype != MACLAB_DTYPE_F64 && dtype != MACLAB_DTYPE_F32) return fail(MACLAB_ERR_INVALID, "bad dtype");
  DeviceGuard dg(h->device);
  maclab_status s = ensure_adjoint(h);
  if (s != MACLAB_OK) return s;
  CUDA_TRY(cudaMemsetAsync(h->d_adj_red, 0, sizeof(double), h->stream), "adjoint seed");
  CUDA_TRY(launch_adjoint_seed(h->g, h->precision, grad_rho, grad_u, dtype, state_T, h->rho0, h->e,
                               lam_T, h->d_adj_red, h->stream),
           "adjoint seed");
  double dot = 0;
  CUDA_TRY(cudaMemcpyAsync(&dot, h->d_adj_red, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "adjoint seed D2H");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "adjoint seed sync");
  if (dot_T) *dot_T = dot;
  return MACLAB_OK;
}

maclab_status maclab_adjoint_finish(maclab_handle h, const void* lam_0, const void* state_0,
                                    void* grad_rho0, void* grad_u0, int32_t dtype, double dot_T,
                                    const double* grad_force_lat, double* grad_wall,
                                    double* grad_scalars) {
  if (!h || !lam_0 || !state_0) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (dtype != MACLAB_DTYPE_F64 && dtype != MACLAB_DTYPE_F32) return fail(MACLAB_ERR_INVALID, "bad dtype");
  DeviceGuard dg(h->device);
  maclab_status s = ensure_adjoint(h);
  if (s != MACLAB_OK) return s;
  const size_t nred = 1 + 4 * (size_t)h->n_wall_ids;
  CUDA_TRY(cudaMemsetAsync(h->d_adj_red, 0, sizeof(double) * nred, h->stream), "adjoint finish");
  CUDA_TRY(launch_adjoint_finish(h->g, h->precision, lam_0, state_0, h->d_node_type, h->n_wall_ids,
                                 h->rho0, h->e, grad_rho0, grad_u0, dtype,
                                 h->n_wall_ids ? h->d_adj_red + 1 : nullptr, h->d_adj_red, h->stream),
           "adjoint finish");
  std::vector<double> red(nred);
  CUDA_TRY(cudaMemcpyAsync(red.data(), h->d_adj_red, sizeof(double) * nred, cudaMemcpyDeviceToHost,
                           h->stream),
           "adjoint finish D2H");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "adjoint finish sync");
  if (grad_wall)
    for (size_t k = 0; k < 4 * (size_t)h->n_wall_ids; ++k) grad_wall[k] = red[1 + k];
  if (grad_scalars) {
    // e enters through ut0 = u0 / e (inputs and walls), the output u = e ut and
    // the force increment force * dt / e = force * dx / e^2.
    double lf = 0;
    for (int i = 0; i < h->g.d; ++i)
      lf += (grad_force_lat ? grad_force_lat[i] : 0.0) * h->force_lat[i];
    const double dLde = (dot_T - red[0] - 2.0 * lf) / h->e;
    grad_scalars[0] = dLde * 6.0 / h->dx;  // e = 6 nu / dx
    grad_scalars[1] = dLde;
    for (int i = 0; i < 3; ++i)
      grad_scalars[2 + i] =
          (i < h->g.d && grad_force_lat) ? grad_force_lat[i] * h->dt / h->e : 0.0;
  }
  return MACLAB_OK;
}

maclab_status maclab_diagnostics(maclab_handle h, double out[8]) {
  NvtxRange nvtx_range("maclab_diagnostics");
  if (!h || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceGuard dg(h->device);
  CUDA_TRY(launch_diagnostics(h->g, h->precision, h->buf[h->cur],
                              h->prev_valid ? h->buf[h->cur ^ 1] : nullptr, h->d_partial,
                              diag_ticket(h), h->diag_nblocks, h->d_diag, h->stream, h->overlap),
           "diagnostics kernel");
  CUDA_TRY(cudaMemcpyAsync(h->h_diag, h->d_diag, kDiagOut * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "diagnostics D2H");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "diagnostics sync");
  double r[kDiagOut];
  for (int k = 0; k < kDiagOut; ++k) r[k] = h->h_diag[k];
  const double nf = (double)h->n_fluid;
  out[0] = h->rho0 * (nf + r[0]);
  out[1] = 0.5 * h->rho0 * h->e * h->e * r[1];
  out[2] = h->rho0 * h->e * r[2];
  out[3] = h->rho0 * h->e * r[3];
  out[4] = h->rho0 * h->e * r[4];
  out[5] = h->prev_valid ? (r[6] > 0 ? sqrt(r[5] / r[6]) : 0.0) : -1.0;
  out[6] = r[7];
  out[7] = r[8];
  if (r[8] > 0) return fail(MACLAB_ERR_NONFINITE, "non-finite values in the state");
  return MACLAB_OK;
}

maclab_status maclab_diagnostics_device(maclab_handle h, double* out) {
  NvtxRange nvtx_range("maclab_diagnostics_device");
  if (!h || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceGuard dg(h->device);
  CUDA_TRY(launch_diagnostics(h->g, h->precision, h->buf[h->cur],
                              h->prev_valid ? h->buf[h->cur ^ 1] : nullptr, h->d_partial,
                              diag_ticket(h), h->diag_nblocks, out, h->stream, h->overlap),
           "diagnostics kernel");
  return MACLAB_OK;
}

maclab_status maclab_diagnostics_sums(maclab_handle h, double out[9]) {
  NvtxRange nvtx_range("maclab_diagnostics_sums");
  if (!h || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  DeviceGuard dg(h->device);
  CUDA_TRY(launch_diagnostics(h->g, h->precision, h->buf[h->cur],
                              h->prev_valid ? h->buf[h->cur ^ 1] : nullptr, h->d_partial,
                              diag_ticket(h), h->diag_nblocks, h->d_diag, h->stream, h->overlap),
           "diagnostics kernel");
  CUDA_TRY(cudaMemcpyAsync(h->h_diag, h->d_diag, kDiagOut * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
           "diagnostics D2H");
  CUDA_TRY(cudaStreamSynchronize(h->stream), "diagnostics sync");
  for (int k = 0; k < kDiagOut; ++k) out[k] = h->h_diag[k];
  if (!h->prev_valid) out[5] = out[6] = -1.0;
  return MACLAB_OK;
}

// Planes of the march axis (z in 3D, y in 2D) of the current state: plane p of
// field f is the contiguous run of plane_size stored values at f * N + p * plane_size.
static maclab_status planes_args(maclab_ctx* h, int64_t p0, int64_t count, const void* buf, int32_t where,
                                 size_t* plane_bytes) {
  if (!h || !buf) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (where != MACLAB_HOST && where != MACLAB_DEVICE) return fail(MACLAB_ERR_INVALID, "bad where");
  const int64_t np = h->g.d == 3 ? h->g.nz : h->g.ny;
  if (count < 1 || p0 < 0 || p0 + count > np) return fail(MACLAB_ERR_INVALID, "plane range outside the domain");
  *plane_bytes = (size_t)(h->g.n / np) * h->elem;
  return MACLAB_OK;
}

maclab_status maclab_get_planes(maclab_handle h, int64_t p0, int64_t count, void* dst, int32_t where) {
  NvtxRange nvtx_range("maclab_get_planes");
  size_t pb = 0;
  maclab_status s = planes_args(h, p0, count, dst, where, &pb);
  if (s != MACLAB_OK) return s;
  DeviceGuard dg(h->device);
  const size_t field = (size_t)h->g.n * h->elem;
  for (int f = 0; f <= h->g.d; ++f)
    CUDA_TRY(cudaMemcpyAsync((char*)dst + f * count * pb, (const char*)h->buf[h->cur] + f * field + p0 * pb,
                             count * pb, cudaMemcpyDefault, h->stream),
             "get_planes copy");
  if (where == MACLAB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream), "get_planes sync");
  return MACLAB_OK;
}

maclab_status maclab_set_planes(maclab_handle h, int64_t p0, int64_t count, const void* src, int32_t where) {
  NvtxRange nvtx_range("maclab_set_planes");
  size_t pb = 0;
  maclab_status s = planes_args(h, p0, count, src, where, &pb);
  if (s != MACLAB_OK) return s;
  DeviceGuard dg(h->device);
  const size_t field = (size_t)h->g.n * h->elem;
  for (int f = 0; f <= h->g.d; ++f)
    CUDA_TRY(cudaMemcpyAsync((char*)h->buf[h->cur] + f * field + p0 * pb, (const char*)src + f * count * pb,
                             count * pb, cudaMemcpyDefault, h->stream),
             "set_planes copy");
  if (where == MACLAB_HOST) CUDA_TRY(cudaStreamSynchronize(h->stream), "set_planes sync");
  return MACLAB_OK;
}

}  // extern "C"

namespace maclab {
unsigned* step_status() {
  static std::mutex m;
  static unsigned* words[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(m);
  if (!words[dev]) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess || cudaMemset(p, 0, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    words[dev] = static_cast<unsigned*>(p);
  }
  return words[dev];
}

BoundsLog* bounds_log() {
#ifdef MACLAB_BOUNDS_CHECK
  static std::mutex m;
  static BoundsLog* logs[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(m);
  if (!logs[dev]) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(BoundsLog)) != cudaSuccess || cudaMemset(p, 0, sizeof(BoundsLog)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    logs[dev] = static_cast<BoundsLog*>(p);
  }
  return logs[dev];
#else
  return nullptr;
#endif
}
}  // namespace maclab

extern "C" {

maclab_status maclab_debug_bounds(int64_t out[2]) {
  if (!out) return fail(MACLAB_ERR_INVALID, "NULL argument");
#ifdef MACLAB_BOUNDS_CHECK
  BoundsLog* log = bounds_log();
  if (!log) return fail(MACLAB_ERR_CUDA, "bounds log unavailable");
  BoundsLog h{};
  CUDA_TRY(cudaDeviceSynchronize(), "debug_bounds sync");
  CUDA_TRY(cudaMemcpy(&h, log, sizeof(h), cudaMemcpyDeviceToHost), "debug_bounds read");
  CUDA_TRY(cudaMemset(log, 0, sizeof(h)), "debug_bounds clear");
  out[0] = (int64_t)h.count;
  out[1] = (int64_t)h.first;
  return MACLAB_OK;
#else
  out[0] = out[1] = 0;
  return fail(MACLAB_ERR_UNSUPPORTED, "library built without MACLAB_BOUNDS_CHECK");
#endif
}

maclab_status maclab_set_kernel(maclab_handle h, int32_t kernel) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  drop_graphs(h);
  if (kernel == MACLAB_KERNEL_AUTO) {
    h->kernel = pick_step_kernel(h->g, h->precision);
    return MACLAB_OK;
  }
  if (kernel != MACLAB_KERNEL_REFERENCE && kernel != MACLAB_KERNEL_TILED && kernel != MACLAB_KERNEL_FOLDED &&
      kernel != MACLAB_KERNEL_SEGMENT && kernel != MACLAB_KERNEL_ROWS2 && kernel != MACLAB_KERNEL_BLOCK)
    return fail(MACLAB_ERR_INVALID, "unknown kernel id");
  if (!step_kernel_supported(h->g, h->precision, kernel))
    return fail(MACLAB_ERR_UNSUPPORTED, "kernel does not support this domain");
  h->kernel = kernel;
  // a tile shape the new kernel lacks falls back to its default
  if (kernel == MACLAB_KERNEL_FOLDED && !fold_supported(h->g, h->precision, h->ty)) h->ty = 0;
  if (kernel == MACLAB_KERNEL_ROWS2 && !rows2_supported(h->g, h->precision, h->ty)) h->ty = 0;
  if (kernel == MACLAB_KERNEL_BLOCK && !block_supported(h->g, h->precision, h->ty)) h->ty = 0;
  if (kernel == MACLAB_KERNEL_TILED && !tiled_supported(h->g, h->precision, h->ty, h->tz)) h->ty = 0;
  return MACLAB_OK;
}

maclab_status maclab_set_launch_overlap(maclab_handle h, int32_t on) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  if (on != 0 && on != 1) return fail(MACLAB_ERR_INVALID, "on must be 0 or 1");
  drop_graphs(h);
  h->overlap = on;
  return MACLAB_OK;
}

maclab_status maclab_get_launch_overlap(maclab_handle h, int32_t* on) {
  if (!h || !on) return fail(MACLAB_ERR_INVALID, "NULL argument");
  *on = h->overlap;
  return MACLAB_OK;
}

maclab_status maclab_set_tile(maclab_handle h, int32_t ty, int32_t tz) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  if (ty < 0 || tz < 0 || tz > (1 << 20)) return fail(MACLAB_ERR_INVALID, "bad tile shape");
  const bool ok = h->kernel == MACLAB_KERNEL_FOLDED    ? fold_supported(h->g, h->precision, ty)
                  : h->kernel == MACLAB_KERNEL_ROWS2   ? rows2_supported(h->g, h->precision, ty)
                  : h->kernel == MACLAB_KERNEL_BLOCK   ? block_supported(h->g, h->precision, ty)  // ty: steps
                  : h->kernel == MACLAB_KERNEL_SEGMENT
                      ? (ty <= 1 || segment_depth(h->g, h->precision, ty) == 2)  // ty: steps per launch, tz: rows
                                                       : tiled_supported(h->g, h->precision, ty, tz);
  if (!ok) return fail(MACLAB_ERR_UNSUPPORTED, "no built tiled instance has this shape");
  drop_graphs(h);
  h->ty = ty;
  h->tz = tz;
  return MACLAB_OK;
}

maclab_status maclab_kernel_info(maclab_handle h, int32_t out[4], const char** name) {
  if (!h || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  const KernelInfo k = describe_step_kernel(h->g, h->precision, h->kernel, h->ty, h->tz);
  out[0] = k.id;
  out[1] = k.steps_per_launch;
  out[2] = k.launches;
  out[3] = k.threads;
  if (name) *name = k.name;
  return MACLAB_OK;
}

maclab_status maclab_sync(maclab_handle h) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  DeviceGuard dg(h->device);
  CUDA_TRY(cudaStreamSynchronize(h->stream), "sync");
  if (unsigned* st = step_status()) {
    unsigned v = 0;
    CUDA_TRY(cudaMemcpy(&v, st, sizeof(v), cudaMemcpyDeviceToHost), "sync status read");
    if (v) {
      CUDA_TRY(cudaMemset(st, 0, sizeof(v)), "sync status clear");
      return fail(MACLAB_ERR_TIMEOUT, "a step kernel's bounded wait (for a tile copy or another block) ran out");
    }
  }
  return MACLAB_OK;
}

maclab_status maclab_debug_segment_waits(int32_t nx, int32_t ny, int32_t periodic_y, int32_t rows,
                                         int32_t blocks, int32_t* items, int64_t items_cap, int32_t* waits,
                                         int64_t waits_cap, int64_t lens[2]) {
  if (!lens) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (nx < 8 || nx % 4 != 0 || ny < 1 || rows < 1 || blocks < 1)
    return fail(MACLAB_ERR_INVALID, "bad segment shape");
  Geometry g{};
  g.lattice = kD2Q9;
  g.d = 2;
  g.nx = nx;
  g.ny = ny;
  g.nz = 1;
  g.n = (int64_t)nx * ny;
  std::vector<int> it, w;
  batch_items(0, g, rows, 2, it);
  batch_persist_deps(it, {ny}, {periodic_y != 0 ? 1 : 0}, blocks, w);
  lens[0] = (int64_t)it.size();
  lens[1] = (int64_t)w.size();
  if (items_cap < lens[0] || waits_cap < lens[1] || (lens[0] && !items) || (lens[1] && !waits))
    return fail(MACLAB_ERR_INVALID, "output arrays too small (lens holds the sizes)");
  std::copy(it.begin(), it.end(), items);
  std::copy(w.begin(), w.end(), waits);
  return MACLAB_OK;
}

maclab_status maclab_debug_batch_waits(int32_t count, const int32_t* nx, const int32_t* ny,
                                       const int32_t* periodic_y, int32_t rows, int32_t blocks, int32_t* items,
                                       int64_t items_cap, int32_t* waits, int64_t waits_cap, int64_t lens[2]) {
  if (!lens || !nx || !ny || !periodic_y) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (count < 1 || rows < 1 || blocks < 1) return fail(MACLAB_ERR_INVALID, "bad batch shape");
  std::vector<int> it, w, nys, pys;
  for (int i = 0; i < count; ++i) {
    if (nx[i] < 8 || nx[i] % 4 != 0 || ny[i] < 1) return fail(MACLAB_ERR_INVALID, "bad domain shape");
    Geometry g{};
    g.lattice = kD2Q9;
    g.d = 2;
    g.nx = nx[i];
    g.ny = ny[i];
    g.nz = 1;
    g.n = (int64_t)nx[i] * ny[i];
    batch_items(i, g, rows, 2, it);
    nys.push_back(ny[i]);
    pys.push_back(periodic_y[i] != 0 ? 1 : 0);
  }
  batch_persist_deps(it, nys, pys, blocks, w);
  lens[0] = (int64_t)it.size();
  lens[1] = (int64_t)w.size();
  if (items_cap < lens[0] || waits_cap < lens[1] || (lens[0] && !items) || (lens[1] && !waits))
    return fail(MACLAB_ERR_INVALID, "output arrays too small (lens holds the sizes)");
  std::copy(it.begin(), it.end(), items);
  std::copy(w.begin(), w.end(), waits);
  return MACLAB_OK;
}

maclab_status maclab_set_wait_limit(maclab_handle h, int64_t polls) {
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  if (polls > (int64_t)0xffffffffu) return fail(MACLAB_ERR_INVALID, "wait limit above 2^32 - 1");
  h->wait_limit = polls < 0 ? kWaitLimit : (unsigned)polls;
  return MACLAB_OK;
}

}  // extern "C"

// ====================================================================== batches

struct maclab_batch_ctx {
  std::vector<maclab_ctx*> members;
  int lattice = 0, precision = 0;
  bool one_launch = false;     // all D2Q9 with nx % 4 == 0: one launch per step
  void* d_insts = nullptr;
  void* d_items = nullptr;
  int n_items = 0;
  int rows = 0;                // rows per work item
  int depth = 1;               // time steps per launch (1 or 2)
  int blocks = 0;
  // the persistent form (depth 3 in maclab_batch_set_depth): the two-step
  // work list, and every step pair of a call in one cooperative launch whose
  // blocks wait only for the blocks owning rows next to theirs
  bool persist = false;
  std::vector<int> items_host;  // the work list (4 ints per item) the wait lists are built from
  int* d_deps = nullptr;        // each block's wait list (batch_persist_deps)
  unsigned* d_done = nullptr;   // the blocks' finished-sweep counters
  int persist_blocks = 0;
  unsigned wait_limit = maclab::kWaitLimit;  // polls before a wait between blocks gives up
  int overlap = 1;             // programmatic dependent launch
  int cur = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  int graph_steps = 32;
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
};

namespace {

void batch_drop_graphs(maclab_batch_ctx* b) {
  for (int c = 0; c < 2; ++c)
    if (b->graph_exec[c]) {
      cudaGraphExecDestroy(b->graph_exec[c]);
      b->graph_exec[c] = nullptr;
    }
}

void batch_free(maclab_batch_ctx* b) {
  if (!b) return;
  batch_drop_graphs(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  cudaFree(b->d_insts);
  cudaFree(b->d_items);
  cudaFree(b->d_deps);
  cudaFree(b->d_done);
  for (maclab_ctx* m : b->members) maclab_destroy(m);
  delete b;
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  return sms;
}

// Two steps per launch need FP32 or FP64 storage and rows of at least two quads.
bool batch_depth2_ok(const maclab_batch_ctx* b) {
  if (!b->one_launch || (b->precision != MACLAB_F32 && b->precision != MACLAB_F64)) return false;
  for (const maclab_ctx* m : b->members)
    if (m->g.nx < 8) return false;
  return true;
}

// (Re)build the work list for `rows` rows per item and `depth` steps per launch.
maclab_status batch_build_items(maclab_batch_ctx* b, int rows, int depth) {
  if (!b->one_launch) {
    b->rows = rows;
    b->depth = 1;
    return MACLAB_OK;
  }
  std::vector<int> items;
  for (size_t i = 0; i < b->members.size(); ++i) batch_items((int)i, b->members[i]->g, rows, depth, items);
  void* d = nullptr;
  if (cudaMalloc(&d, items.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(MACLAB_ERR_OOM, "batch work list allocation failed");
  }
  cudaError_t e = cudaMemcpy(d, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_fail(e, "batch work list upload");
  }
  cudaFree(b->d_items);
  b->d_items = d;
  b->n_items = (int)(items.size() / 4);
  b->items_host.swap(items);
  b->rows = rows;
  b->depth = depth;
  cudaFree(b->d_deps);
  cudaFree(b->d_done);
  b->d_deps = nullptr;
  b->d_done = nullptr;
  b->persist_blocks = 0;
  // resident warps: two 256-thread blocks per SM (one step per launch) or
  // three 128-thread blocks (two steps)
  const int warps_per_block = depth == 2 ? 4 : 8, per_sm = depth == 2 ? 3 : 2;
  const int want = (b->n_items + warps_per_block - 1) / warps_per_block;
  b->blocks = want < per_sm * sm_count() ? (want > 0 ? want : 1) : per_sm * sm_count();
  batch_drop_graphs(b);
  return MACLAB_OK;
}

// The persistent form's wait lists for the current (two-step) work list: as
// many blocks as fit at once.  Returns MACLAB_ERR_UNSUPPORTED when the device
// cannot hold even one block of the cooperative launch.
maclab_status batch_persist_prepare(maclab_batch_ctx* b) {
  if (b->persist_blocks > 0) return MACLAB_OK;
  if (b->depth != 2) return fail(MACLAB_ERR_INVALID, "the persistent form needs the two-step work list");
  int capacity = 0;
  if (batch_persist_capacity(b->precision, &capacity) != cudaSuccess || capacity < 1) {
    cudaGetLastError();
    return fail(MACLAB_ERR_UNSUPPORTED, "the persistent launch does not fit on this device");
  }
  const int want = (b->n_items + 3) / 4;
  const int pb = want < capacity ? (want > 0 ? want : 1) : capacity;
  std::vector<int> ny, py;
  for (const maclab_ctx* m : b->members) {
    ny.push_back(m->g.ny);
    py.push_back((m->g.periodic & 2u) != 0 ? 1 : 0);
  }
  std::vector<int> deps;
  batch_persist_deps(b->items_host, ny, py, pb, deps);
  if (cudaMalloc(&b->d_deps, deps.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_done, (size_t)pb * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->d_deps);
    b->d_deps = nullptr;
    b->d_done = nullptr;
    return fail(MACLAB_ERR_OOM, "persistent batch lists allocation failed");
  }
  CUDA_TRY(cudaMemcpyAsync(b->d_deps, deps.data(), deps.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream),
           "persistent batch lists upload");
  CUDA_TRY(cudaStreamSynchronize(b->stream), "persistent batch lists sync");
  b->persist_blocks = pb;
  return MACLAB_OK;
}

// `sweeps` two-step sweeps from buffer c in one persistent launch.
cudaError_t batch_launch_persist(maclab_batch_ctx* b, int c, int sweeps, cudaStream_t st) {
  return launch_batch_step2_persist(b->precision, b->d_insts, b->d_items, b->n_items, c, b->persist_blocks, sweeps,
                                    b->d_deps, b->d_done, step_status(), b->wait_limit, st);
}

// One launch of `steps` time steps (1, or b->depth) from buffer c.
cudaError_t batch_launch_steps(maclab_batch_ctx* b, int c, int steps, cudaStream_t st) {
  if (b->one_launch && steps == 2)
    return launch_batch_step2(b->precision, b->d_insts, b->d_items, b->n_items, c, b->blocks, st,
                              b->overlap);
  if (b->one_launch)
    return launch_batch_step(b->precision, b->d_insts, b->d_items, b->n_items, c, b->blocks,
                             b->depth == 2 ? kBatchSegW2 : kBatchSegW1, st, b->overlap);
  for (maclab_ctx* m : b->members) {
    StepLaunch sl = step_launch(m, c);
    sl.seg_steps = 1;  // one step per member launch (the block kernel's one-step form)
    cudaError_t e = launch_step(sl, st, m->kernel);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One launch of b->depth steps.
cudaError_t batch_launch_one(maclab_batch_ctx* b, int c, cudaStream_t st) {
  return batch_launch_steps(b, c, b->one_launch ? b->depth : 1, st);
}

// Launches in one graph: graph_steps / depth, each of depth steps.
int batch_graph_launches(const maclab_batch_ctx* b) { return b->graph_steps / b->depth; }

maclab_status batch_build_graph(maclab_batch_ctx* b, int c) {
  if (!b->capture_stream &&
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "capture stream");
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed), "begin capture");
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < batch_graph_launches(b) && err == cudaSuccess; ++k)
    err = batch_launch_one(b, c ^ (k & 1), b->capture_stream);
  cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &graph);
  if (err != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(err != cudaSuccess ? err : e2, "batch graph capture");
  }
  err = cudaGraphInstantiate(&b->graph_exec[c], graph, 0);
  cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    b->graph_exec[c] = nullptr;
    return cuda_fail(err, "batch graph instantiate");
  }
  return MACLAB_OK;
}

}  // namespace

extern "C" {

maclab_status maclab_batch_create(const maclab_config* cfgs, int32_t count, maclab_batch* out) {
  if (!out) return fail(MACLAB_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfgs || count < 1) return fail(MACLAB_ERR_INVALID, "need at least one configuration");
  maclab_batch_ctx* b = new (std::nothrow) maclab_batch_ctx();
  if (!b) return fail(MACLAB_ERR_OOM, "host allocation failed");
  b->lattice = cfgs[0].lattice;
  b->precision = cfgs[0].precision;
  b->stream = (cudaStream_t)cfgs[0].stream;
  maclab_status warn = MACLAB_OK;
  for (int i = 0; i < count; ++i) {
    if (cfgs[i].lattice != b->lattice || cfgs[i].precision != b->precision ||
        cfgs[i].stream != cfgs[0].stream) {
      batch_free(b);
      return fail(MACLAB_ERR_INVALID, "batch members must share lattice, precision and stream");
    }
    maclab_handle h = nullptr;
    maclab_status s = maclab_create(&cfgs[i], &h);
    if (s < 0) {
      batch_free(b);
      return s;
    }
    if (s > 0) warn = s;
    b->members.push_back(h);
  }
  b->device = b->members[0]->device;
  for (maclab_ctx* m : b->members)
    if (m->device != b->device) {
      batch_free(b);
      return fail(MACLAB_ERR_INVALID, "batch members must be on one device");
    }
  DeviceGuard dg(b->device);
  b->one_launch = b->lattice == MACLAB_D2Q9;
  for (maclab_ctx* m : b->members) b->one_launch = b->one_launch && m->g.ilv == 1;
  // one launch per member and step: the segment kernel's work list is not
  // built, and the block kernel would take one step per launch
  if (!b->one_launch)
    for (maclab_ctx* m : b->members)
      if (m->kernel == MACLAB_KERNEL_SEGMENT || m->kernel == MACLAB_KERNEL_BLOCK)
        m->kernel = tiled_supported(m->g, m->precision, 0, 0) ? MACLAB_KERNEL_TILED : MACLAB_KERNEL_REFERENCE;
  if (b->one_launch) {
    std::vector<unsigned char> insts(batch_inst_bytes() * b->members.size());
    for (size_t i = 0; i < b->members.size(); ++i) {
      maclab_ctx* m = b->members[i];
      batch_fill_inst(insts.data() + i * batch_inst_bytes(), m->g, m->buf[0], m->buf[1], m->force_lat);
    }
    if (cudaMalloc(&b->d_insts, insts.size()) != cudaSuccess) {
      cudaGetLastError();
      batch_free(b);
      return fail(MACLAB_ERR_OOM, "batch descriptor allocation failed");
    }
    cudaError_t e = cudaMemcpy(b->d_insts, insts.data(), insts.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      batch_free(b);
      return cuda_fail(e, "batch descriptor upload");
    }
  }
  maclab_status s = batch_build_items(b, 16, 1);
  if (s != MACLAB_OK) {
    batch_free(b);
    return s;
  }
  *out = b;
  return warn;
}

maclab_status maclab_batch_destroy(maclab_batch b) {
  if (!b) return MACLAB_OK;
  DeviceGuard dg(b->device);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return MACLAB_OK;
}

maclab_status maclab_batch_member(maclab_batch b, int32_t i, maclab_handle* out) {
  if (!b || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  if (i < 0 || i >= (int)b->members.size()) return fail(MACLAB_ERR_INVALID, "member index out of range");
  *out = b->members[i];
  return MACLAB_OK;
}

maclab_status maclab_batch_step(maclab_batch b, int64_t n) {
  NvtxRange nvtx_range("maclab_batch_step");
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  if (n < 0) return fail(MACLAB_ERR_INVALID, "n must be >= 0");
  for (maclab_ctx* m : b->members)
    if (m->cur != b->cur) return fail(MACLAB_ERR_INVALID, "a member was stepped outside the batch");
  DeviceGuard dg(b->device);
  // With two steps per launch the last step is a one-step launch, so that the
  // other buffer holds step n - 1 as after single steps (the residual reads it).
  const int k = b->one_launch ? b->depth : 1;
  const int64_t bulk = k > 1 && n > 0 ? n - 1 : n;
  const int launches = batch_graph_launches(b);
  const int64_t gsteps = (int64_t)launches * k;
  int64_t done = 0;
  // the persistent form: the bulk's step pairs in one cooperative launch
  const bool persist = b->persist && k == 2 && b->persist_blocks > 0;
  for (int64_t pairs = persist ? bulk / 2 : 0; pairs > 0;) {
    const int sweeps = pairs > (1 << 30) ? (1 << 30) : (int)pairs;
    CUDA_TRY(batch_launch_persist(b, b->cur, sweeps, b->stream), "persistent batch launch");
    if (sweeps & 1) b->cur ^= 1;
    done += 2 * (int64_t)sweeps;
    pairs -= sweeps;
  }
  while (!persist && gsteps > 0 && bulk - done >= gsteps) {
    if (!b->graph_exec[b->cur]) {
      maclab_status s = batch_build_graph(b, b->cur);
      if (s != MACLAB_OK) return s;
    }
    CUDA_TRY(cudaGraphLaunch(b->graph_exec[b->cur], b->stream), "batch graph launch");
    if (launches & 1) b->cur ^= 1;
    done += gsteps;
  }
  for (; bulk - done >= k; done += k) {
    CUDA_TRY(batch_launch_one(b, b->cur, b->stream), "batch step launch");
    b->cur ^= 1;
  }
  for (; done < n; ++done) {
    CUDA_TRY(batch_launch_steps(b, b->cur, 1, b->stream), "batch step launch");
    b->cur ^= 1;
  }
  for (maclab_ctx* m : b->members) {
    m->cur = b->cur;
    m->steps += n;
    if (n > 0) m->prev_valid = true;
  }
  return MACLAB_OK;
}

maclab_status maclab_batch_set_rows(maclab_batch b, int32_t rows) {
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  if (rows < 0 || rows > (1 << 20)) return fail(MACLAB_ERR_INVALID, "bad row count");
  DeviceGuard dg(b->device);
  maclab_status s = batch_build_items(b, rows ? rows : 16, b->depth);
  return s == MACLAB_OK && b->persist ? batch_persist_prepare(b) : s;
}

maclab_status maclab_batch_set_depth(maclab_batch b, int32_t depth) {
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  if (depth < 0 || depth > 3) return fail(MACLAB_ERR_INVALID, "depth must be 0, 1, 2 or 3");
  if (depth == 0) depth = 1;
  if (depth >= 2 && !batch_depth2_ok(b))
    return fail(MACLAB_ERR_UNSUPPORTED,
                "two steps per launch need one launch per step, FP32 or FP64 storage and nx >= 8");
  DeviceGuard dg(b->device);
  const bool persist = depth == 3;
  maclab_status s = batch_build_items(b, b->rows ? b->rows : 16, persist ? 2 : depth);
  if (s != MACLAB_OK) return s;
  b->persist = false;
  if (persist) {
    s = batch_persist_prepare(b);
    if (s != MACLAB_OK) return s;
    b->persist = true;
  }
  return MACLAB_OK;
}

maclab_status maclab_batch_set_wait_limit(maclab_batch b, int64_t polls) {
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  if (polls > (int64_t)0xffffffffu) return fail(MACLAB_ERR_INVALID, "wait limit above 2^32 - 1");
  b->wait_limit = polls < 0 ? kWaitLimit : (unsigned)polls;
  return MACLAB_OK;
}

maclab_status maclab_batch_set_launch_overlap(maclab_batch b, int32_t on) {
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  if (on != 0 && on != 1) return fail(MACLAB_ERR_INVALID, "on must be 0 or 1");
  batch_drop_graphs(b);
  b->overlap = on;
  for (maclab_ctx* m : b->members) {
    drop_graphs(m);
    m->overlap = on;
  }
  return MACLAB_OK;
}

maclab_status maclab_batch_info(maclab_batch b, int64_t out[7]) {
  if (!b || !out) return fail(MACLAB_ERR_INVALID, "NULL argument");
  int64_t nodes = 0, fluid = 0;
  for (maclab_ctx* m : b->members) {
    nodes += m->g.n;
    fluid += m->n_fluid;
  }
  out[0] = (int64_t)b->members.size();
  out[1] = nodes;
  out[2] = fluid;
  out[3] = b->one_launch ? b->n_items : 0;
  out[4] = b->rows;
  out[5] = b->one_launch ? 1 : (int64_t)b->members.size();
  out[6] = !b->one_launch ? 1 : (b->persist ? 3 : b->depth);
  return MACLAB_OK;
}

}  // extern "C"

// ====================================================================== tuning

namespace {

std::mutex g_tune_mutex;
struct TuneChoice {
  int kernel, ty, tz;
  int overlap = 1;  // programmatic dependent launch on (1) or off (0)
};
std::map<std::string, TuneChoice> g_tune_cache;

bool shape_supported(const maclab_ctx* h, int kernel, int ty, int tz) {
  if (kernel == MACLAB_KERNEL_SEGMENT)
    return step_kernel_supported(h->g, h->precision, MACLAB_KERNEL_SEGMENT) &&
           (ty <= 1 || segment_depth(h->g, h->precision, ty) == 2);
  if (kernel == MACLAB_KERNEL_ROWS2) return rows2_supported(h->g, h->precision, ty);
  if (kernel == MACLAB_KERNEL_BLOCK) return block_supported(h->g, h->precision, ty);
  return kernel == MACLAB_KERNEL_FOLDED ? fold_supported(h->g, h->precision, ty)
                                        : tiled_supported(h->g, h->precision, ty, tz);
}

// Device model as a key part: its name (spaces as '_') and SM count.
std::string device_tag(int device) {
  static std::mutex m;
  static std::map<int, std::string> tags;
  std::lock_guard<std::mutex> lock(m);
  auto it = tags.find(device);
  if (it != tags.end()) return it->second;
  cudaDeviceProp prop;
  std::string tag = "unknown";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
    tag = prop.name;
    for (char& c : tag)
      if (c == ' ' || c == '\t') c = '_';
    tag += "/" + std::to_string(prop.multiProcessorCount);
  } else {
    cudaGetLastError();
  }
  tags[device] = tag;
  return tag;
}

std::string tune_key(const maclab_ctx* h) {
  char buf[160];
  snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/%u/%d/", h->g.lattice, h->precision, h->g.nx, h->g.ny,
           h->g.nz, h->g.periodic, h->g.wall_mode);
  return buf + device_tag(h->device);
}

// Tuning results kept across processes: MACLAB_TUNE_CACHE names a text file
// of lines "<key> <kernel> <ty> <tz> [<overlap>]".  A shape not tuned in this
// process is looked up there first; a newly tuned one is appended.  Malformed
// lines and an unreadable file are ignored.
const char* tune_cache_path() {
  const char* p = getenv("MACLAB_TUNE_CACHE");
  return p && *p ? p : nullptr;
}

bool tune_cache_find(const std::string& key, TuneChoice* out) {
  const char* path = tune_cache_path();
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[512], k[400];
  int kern = 0, ty = 0, tz = 0, ov = 1;
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    ov = 1;
    const int got = sscanf(line, "%399s %d %d %d %d", k, &kern, &ty, &tz, &ov);
    if (got >= 4 && key == k && (ov == 0 || ov == 1)) {
      *out = TuneChoice{kern, ty, tz, ov};  // the last line for a key wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_append(const std::string& key, const TuneChoice& c) {
  const char* path = tune_cache_path();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %d\n", key.c_str(), c.kernel, c.ty, c.tz, c.overlap);
  fclose(f);
}

template <typename Fn>
// Milliseconds per call of fn: the best of three runs of k calls, after three
// warm-up calls.
float time_ms(cudaStream_t st, int k, Fn fn) {
  for (int i = 0; i < 3; ++i) fn();
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a, st);
    for (int i = 0; i < k; ++i) fn();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best / k;
}

}  // namespace

extern "C" {

maclab_status maclab_tune(maclab_handle h, int32_t out[2]) {
  NvtxRange nvtx_range("maclab_tune");
  if (!h) return fail(MACLAB_ERR_INVALID, "NULL handle");
  DeviceGuard dg(h->device);
  const std::string key = tune_key(h);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    TuneChoice stored;
    if (it == g_tune_cache.end() && tune_cache_find(key, &stored)) it = g_tune_cache.emplace(key, stored).first;
    if (it != g_tune_cache.end()) {
      if (shape_supported(h, it->second.kernel, it->second.ty, it->second.tz)) {
        drop_graphs(h);
        h->kernel = it->second.kernel;
        h->ty = it->second.ty;
        h->tz = it->second.tz;
        h->overlap = it->second.overlap;
      }
      if (out) { out[0] = h->ty; out[1] = h->tz; }
      return MACLAB_OK;
    }
  }
  bool any = false;
  for (int kernel : {MACLAB_KERNEL_TILED, MACLAB_KERNEL_FOLDED, MACLAB_KERNEL_SEGMENT, MACLAB_KERNEL_ROWS2,
                     MACLAB_KERNEL_BLOCK})
    any = any || step_kernel_supported(h->g, h->precision, kernel);
  if (!any) {
    if (out) { out[0] = 0; out[1] = 0; }
    return MACLAB_OK;  // only the reference kernel serves this domain
  }
  // save the state
  void* saved = nullptr;
  const size_t sb = state_bytes(h);
  if (cudaMalloc(&saved, sb) != cudaSuccess) {
    cudaGetLastError();
    return fail(MACLAB_ERR_OOM, "tuning buffer allocation failed");
  }
  CUDA_TRY(cudaMemcpyAsync(saved, h->buf[h->cur], sb, cudaMemcpyDeviceToDevice, h->stream), "tune save");
  const int64_t steps0 = h->steps;
  const bool prev0 = h->prev_valid;
  const int kernel0 = h->kernel, ty0 = h->ty, tz0 = h->tz;
  const int tys3[] = {2, 4, 8};
  const int tzs[] = {0, 4, 8, 16, 32};
  float best = 1e30f;
  int bkernel = MACLAB_KERNEL_TILED, bty = 0, btz = 0;
  drop_graphs(h);
  const int n_ty = h->g.d == 3 ? 3 : 1;
  // each candidate timed on a captured graph of 8 launches, or 64 where 8 take
  // under 0.5 ms (stepping runs in graphs, where the launch gaps that separate
  // launches would add are absent)
  if (!h->capture_stream && cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(saved);
    return cuda_fail(cudaGetLastError(), "capture stream");
  }
  auto graph_ms = [&](int launches) -> float {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return 1e30f;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < launches && err == cudaSuccess; ++k)
      err = launch_step(step_launch(h, h->cur ^ (k & 1)), h->capture_stream, h->kernel);
    cudaError_t e2 = cudaStreamEndCapture(h->capture_stream, &graph);
    if (err != cudaSuccess || e2 != cudaSuccess || !graph ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return 1e30f;
    }
    cudaGraphDestroy(graph);
    const float ms = time_ms(h->stream, 1, [&]() { cudaGraphLaunch(exec, h->stream); });
    cudaGraphExecDestroy(exec);
    return ms;
  };
  // candidates (kernel, ty, tz): tiled and folded shapes; the segment kernel
  // with one or two steps per launch (ty) and 2, 4 or 8 rows per work item (tz)
  struct Cand {
    int kernel, ty, tz;
  };
  std::vector<Cand> cands;
  for (int kernel : {MACLAB_KERNEL_TILED, MACLAB_KERNEL_FOLDED})
    for (int a = 0; a < n_ty; ++a)
      for (int tz : tzs) cands.push_back(Cand{kernel, h->g.d == 3 ? tys3[a] : 0, tz});
  for (int ty : {1, 2, 3})  // 3: two steps per sweep, runs in one persistent launch
    for (int tz : {2, 4, 8, 16, 32}) cands.push_back(Cand{MACLAB_KERNEL_SEGMENT, ty, tz});
  // the block kernel up to 131,072 node pairs (512^2), where it was measured
  // to win; above it the segment kernel is faster in sustained runs (1024^2:
  // 5.5 against 5.6-5.7 us/step), though a short timing can rank them the
  // other way
  if ((int64_t)(h->g.nx / 2) * h->g.ny <= 131072)
    for (int ty : {1, 2, 4, 8}) cands.push_back(Cand{MACLAB_KERNEL_BLOCK, ty, 0});  // ty: steps per launch
  if (h->g.d == 3)
    for (int ty : {4, 8})
      for (int tz : tzs) cands.push_back(Cand{MACLAB_KERNEL_ROWS2, ty, tz});
  for (const Cand& c : cands) {
    if (!shape_supported(h, c.kernel, c.ty, c.tz)) continue;
    h->kernel = c.kernel;
    h->ty = c.ty;
    h->tz = c.tz;
    if (segment_prepare(h) != MACLAB_OK) continue;
    // per time step; graphs of 64 launches where 8 take under 0.5 ms, so that
    // the launch of the graph itself does not decide between close shapes
    float ms;
    if (c.kernel == MACLAB_KERNEL_SEGMENT && c.ty == 3) {
      // the persistent form: one launch of 32 sweeps (64 steps)
      if (h->seg_persist_blocks < 1 || h->seg_depth != 2) continue;
      ms = time_ms(h->stream, 1, [&]() {
             launch_batch_step2_persist(h->precision, h->d_seg_inst, h->d_seg_items, h->seg_n_items, h->cur,
                                        h->seg_persist_blocks, 32, h->d_seg_deps, h->d_seg_done, step_status(),
                                        kWaitLimit, h->stream);
           }) / 64.f;
    } else {
      ms = graph_ms(8);
      if (ms < 0.5f) ms = graph_ms(64) / 8.f;
      ms /= 8 * launch_depth(h);
    }
    if (ms < best) {
      best = ms;
      bkernel = c.kernel;
      bty = c.ty;
      btz = c.tz;
    }
  }
  // launch overlap for the chosen shape: kept on unless plain launches are
  // faster by more than 0.5 %
  const int overlap0 = h->overlap;
  int bover = overlap0;
  if (best < 1e29f) {
    h->kernel = bkernel;
    h->ty = bty;
    h->tz = btz;
    if (segment_prepare(h) == MACLAB_OK) {
      float t[2];
      for (int ov = 0; ov < 2; ++ov) {
        h->overlap = ov;
        t[ov] = graph_ms(8);
        if (t[ov] < 0.5f) t[ov] = graph_ms(64) / 8.f;
      }
      bover = t[0] < 0.995f * t[1] ? 0 : 1;
    }
  }
  h->overlap = bover;
  cudaError_t e = cudaGetLastError();
  // restore
  h->cur = 0;
  cudaMemcpyAsync(h->buf[0], saved, sb, cudaMemcpyDeviceToDevice, h->stream);
  cudaMemcpyAsync(h->buf[1], saved, sb, cudaMemcpyDeviceToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  cudaFree(saved);
  h->steps = steps0;
  h->prev_valid = false;  // both buffers now hold the restored state
  (void)prev0;
  if (e != cudaSuccess) {
    h->kernel = kernel0;
    h->ty = ty0;
    h->tz = tz0;
    h->overlap = overlap0;
    return cuda_fail(e, "tuning launch");
  }
  drop_graphs(h);
  h->kernel = bkernel;
  h->ty = bty;
  h->tz = btz;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneChoice{bkernel, bty, btz, h->overlap};
    tune_cache_append(key, TuneChoice{bkernel, bty, btz, h->overlap});
  }
  if (out) { out[0] = bty; out[1] = btz; }
  return MACLAB_OK;
}

maclab_status maclab_batch_tune(maclab_batch b, int32_t* rows_out) {
  NvtxRange nvtx_range("maclab_batch_tune");
  if (!b) return fail(MACLAB_ERR_INVALID, "NULL batch");
  DeviceGuard dg(b->device);
  if (!b->one_launch) {
    for (maclab_ctx* m : b->members) {
      maclab_status s = maclab_tune(m, nullptr);
      if (s != MACLAB_OK) return s;
    }
    batch_drop_graphs(b);
    if (rows_out) *rows_out = 0;
    return MACLAB_OK;
  }
  // save every member's state
  std::vector<void*> saved(b->members.size(), nullptr);
  for (size_t i = 0; i < b->members.size(); ++i) {
    maclab_ctx* m = b->members[i];
    if (cudaMalloc(&saved[i], state_bytes(m)) != cudaSuccess) {
      cudaGetLastError();
      for (void* p : saved) cudaFree(p);
      return fail(MACLAB_ERR_OOM, "tuning buffer allocation failed");
    }
    cudaMemcpyAsync(saved[i], m->buf[m->cur], state_bytes(m), cudaMemcpyDeviceToDevice, b->stream);
  }
  // rows per work item x time steps per launch, compared per time step on a
  // captured graph of 8 launches, or 64 where 8 take under 0.5 ms (stepping
  // runs in graphs, where the launch gaps that separate launches would add
  // are absent)
  if (!b->capture_stream &&
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "capture stream");
  auto graph_ms = [&](int launches) -> float {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) return 1e30f;
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < launches && err == cudaSuccess; ++k)
      err = batch_launch_one(b, b->cur ^ (k & 1), b->capture_stream);
    cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &graph);
    if (err != cudaSuccess || e2 != cudaSuccess || !graph ||
        cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return 1e30f;
    }
    cudaGraphDestroy(graph);
    const float ms = time_ms(b->stream, 1, [&]() { cudaGraphLaunch(exec, b->stream); });
    cudaGraphExecDestroy(exec);
    return ms;
  };
  const int candidates[] = {2, 4, 8, 16, 32, 64};
  float best = 1e30f;
  int best_rows = 16, best_depth = 1;
  bool best_persist = false;
  b->persist = false;
  const int max_depth = batch_depth2_ok(b) ? 2 : 1;
  for (int depth = 1; depth <= max_depth; ++depth)
    for (int rows : candidates) {
      if (batch_build_items(b, rows, depth) != MACLAB_OK) continue;
      float ms = graph_ms(8);
      if (ms < 0.5f) ms = graph_ms(64) / 8.f;  // short steps: a longer graph
      ms /= 8 * depth;
      if (ms < best) {
        best = ms;
        best_rows = rows;
        best_depth = depth;
        best_persist = false;
      }
      // the persistent form of the same work list: one launch of 32 sweeps (64 steps)
      if (depth == 2 && batch_persist_prepare(b) == MACLAB_OK) {
        // the default wait budget: a smaller one set by the caller could cut
        // the sweeps short and time less than the work
        const unsigned limit = b->wait_limit;
        b->wait_limit = kWaitLimit;
        const float pms = time_ms(b->stream, 1, [&]() { batch_launch_persist(b, b->cur, 32, b->stream); }) / 64.f;
        b->wait_limit = limit;
        if (pms < best) {
          best = pms;
          best_rows = rows;
          best_depth = depth;
          best_persist = true;
        }
      }
    }
  // launch overlap for the chosen work list: kept on unless plain launches
  // are faster by more than 0.5 %
  if (best < 1e29f && batch_build_items(b, best_rows, best_depth) == MACLAB_OK) {
    float t[2];
    for (int ov = 0; ov < 2; ++ov) {
      b->overlap = ov;
      t[ov] = graph_ms(8);
      if (t[ov] < 0.5f) t[ov] = graph_ms(64) / 8.f;
    }
    const int bover = t[0] < 0.995f * t[1] ? 0 : 1;
    b->overlap = bover;
    for (maclab_ctx* m : b->members) m->overlap = bover;
  }
  cudaError_t e = cudaGetLastError();
  b->cur = 0;
  for (size_t i = 0; i < b->members.size(); ++i) {
    maclab_ctx* m = b->members[i];
    cudaMemcpyAsync(m->buf[0], saved[i], state_bytes(m), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(m->buf[1], saved[i], state_bytes(m), cudaMemcpyDeviceToDevice, b->stream);
    m->cur = 0;
    m->prev_valid = false;
  }
  cudaStreamSynchronize(b->stream);
  for (void* p : saved) cudaFree(p);
  if (e != cudaSuccess) return cuda_fail(e, "batch tuning launch");
  maclab_status s = batch_build_items(b, best_rows, best_depth);
  if (s == MACLAB_OK && best_persist) {
    s = batch_persist_prepare(b);
    b->persist = s == MACLAB_OK;
  }
  if (rows_out) *rows_out = best_rows;
  return s;
}

}  // extern "C"
