// convert.cu -- unit maps at the boundary of the library.
//
// Physical (rho, u) <-> stored lattice state (drho = rho / rho0 - 1, ut = u / e)
// with e = 6 nu / dx (Eq. (6)).  Wall nodes take their wall id's values
// (procedure step (iv): physical variables are retained on walls).  The maps
// are computed in FP64 and rounded once to the storage type.  User arrays are
// in logical order; the state and the device node-type copy in storage order.

#include "common.cuh"

namespace maclab {

template <typename T>
__device__ __forceinline__ double ld_user(const T* p, int64_t i) {
  return (double)p[i];
}

// User arrays are in logical order (x fastest); the state in storage order.
// The maps walk the user arrays in order (a warp touches one contiguous run of
// each user array, which may be page-locked host memory read or written over
// the host link) and place each node at its storage index.
__device__ __forceinline__ int64_t storage_index(const Geometry& g, int64_t j) {
  const int64_t row = j / g.nx;
  return row * g.nx + mem_x(g, (int)(j - row * g.nx));
}

template <typename S, typename T>
__global__ void set_physical_k(Geometry g, int d, int64_t N, const T* __restrict__ rho, const T* __restrict__ u,
                               double inv_rho0, double inv_e, const uint8_t* __restrict__ node_type,
                               const double* __restrict__ wall_lat, int n_wall_ids,
                               S* __restrict__ state) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = storage_index(g, j);
    const int k = node_type ? (int)node_type[i] : 0;
    if (k > 0 && k <= n_wall_ids) {
      const double* w = wall_lat + 4 * (k - 1);
      state[i] = Store<S>::to(typename Store<S>::C(w[0]));
      for (int c = 0; c < d; ++c) state[(1 + c) * N + i] = Store<S>::to(typename Store<S>::C(w[1 + c]));
    } else {
      state[i] = Store<S>::to(typename Store<S>::C(ld_user(rho, j) * inv_rho0 - 1.0));
      for (int c = 0; c < d; ++c)
        state[(1 + c) * N + i] = Store<S>::to(typename Store<S>::C(ld_user(u, c * N + j) * inv_e));
    }
  }
}

template <typename S>
__global__ void fill_walls_k(int d, int64_t N, const uint8_t* __restrict__ node_type,
                             const double* __restrict__ wall_lat, int n_wall_ids,
                             S* __restrict__ state) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)node_type[i];
    if (k > 0 && k <= n_wall_ids) {
      const double* w = wall_lat + 4 * (k - 1);
      state[i] = Store<S>::to(typename Store<S>::C(w[0]));
      for (int c = 0; c < d; ++c) state[(1 + c) * N + i] = Store<S>::to(typename Store<S>::C(w[1 + c]));
    }
  }
}

// Per-node wall values: every wall node (node type > 0) takes the given
// physical (rho, u), in both state buffers (the step kernels never write a
// wall node, so whichever buffer is current reads them); fluid entries of the
// arrays are not read.
template <typename S, typename T>
__global__ void set_walls_k(Geometry g, int d, int64_t N, const T* __restrict__ rho, const T* __restrict__ u,
                            double inv_rho0, double inv_e, const uint8_t* __restrict__ node_type,
                            S* __restrict__ s0, S* __restrict__ s1) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = storage_index(g, j);
    if (node_type[i] == 0) continue;
    const S r = Store<S>::to(typename Store<S>::C(ld_user(rho, j) * inv_rho0 - 1.0));
    s0[i] = r;
    s1[i] = r;
    for (int c = 0; c < d; ++c) {
      const S v = Store<S>::to(typename Store<S>::C(ld_user(u, c * N + j) * inv_e));
      s0[(1 + c) * N + i] = v;
      s1[(1 + c) * N + i] = v;
    }
  }
}

template <typename S, typename T>
__global__ void get_physical_k(Geometry g, int d, int64_t N, const S* __restrict__ state, double rho0,
                               double e, T* __restrict__ rho, T* __restrict__ u) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = storage_index(g, j);
    rho[j] = (T)(rho0 * (1.0 + (double)Store<S>::from(state[i])));
    for (int c = 0; c < d; ++c) u[c * N + j] = (T)(e * (double)Store<S>::from(state[(1 + c) * N + i]));
  }
}

static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename S>
static cudaError_t set_t(const Geometry& g, const void* rho, const void* u, int dtype, double rho0,
                         double e, const uint8_t* nt, const double* wl, int nw, void* state,
                         cudaStream_t st) {
  if (dtype == MACLAB_DTYPE_F64)
    set_physical_k<S, double><<<grid_for(g.n), 256, 0, st>>>(
        g, g.d, g.n, (const double*)rho, (const double*)u, 1.0 / rho0, 1.0 / e, nt, wl, nw, (S*)state);
  else
    set_physical_k<S, float><<<grid_for(g.n), 256, 0, st>>>(
        g, g.d, g.n, (const float*)rho, (const float*)u, 1.0 / rho0, 1.0 / e, nt, wl, nw, (S*)state);
  return cudaGetLastError();
}

template <typename S>
static cudaError_t get_t(const Geometry& g, const void* state, void* rho, void* u, int dtype,
                         double rho0, double e, cudaStream_t st) {
  if (dtype == MACLAB_DTYPE_F64)
    get_physical_k<S, double><<<grid_for(g.n), 256, 0, st>>>(g, g.d, g.n, (const S*)state, rho0, e,
                                                            (double*)rho, (double*)u);
  else
    get_physical_k<S, float><<<grid_for(g.n), 256, 0, st>>>(g, g.d, g.n, (const S*)state, rho0, e,
                                                           (float*)rho, (float*)u);
  return cudaGetLastError();
}

cudaError_t launch_set_physical(const Geometry& g, int precision, const void* rho, const void* u,
                                int dtype, double rho0, double e, const uint8_t* nt,
                                const double* wl, int nw, void* state, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return set_t<double>(g, rho, u, dtype, rho0, e, nt, wl, nw, state, st);
    case MACLAB_F32: return set_t<float>(g, rho, u, dtype, rho0, e, nt, wl, nw, state, st);
    case MACLAB_BF16_STORE:
      return set_t<__nv_bfloat16>(g, rho, u, dtype, rho0, e, nt, wl, nw, state, st);
    case MACLAB_F16_STORE: return set_t<__half>(g, rho, u, dtype, rho0, e, nt, wl, nw, state, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_get_physical(const Geometry& g, int precision, const void* state, void* rho,
                                void* u, int dtype, double rho0, double e, cudaStream_t st) {
  switch (precision) {
    case MACLAB_F64: return get_t<double>(g, state, rho, u, dtype, rho0, e, st);
    case MACLAB_F32: return get_t<float>(g, state, rho, u, dtype, rho0, e, st);
    case MACLAB_BF16_STORE: return get_t<__nv_bfloat16>(g, state, rho, u, dtype, rho0, e, st);
    case MACLAB_F16_STORE: return get_t<__half>(g, state, rho, u, dtype, rho0, e, st);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
static cudaError_t walls_t(const Geometry& g, const void* rho, const void* u, int dtype, double rho0,
                           double e, const uint8_t* nt, void* s0, void* s1, cudaStream_t st) {
  if (dtype == MACLAB_DTYPE_F64)
    set_walls_k<S, double><<<grid_for(g.n), 256, 0, st>>>(g, g.d, g.n, (const double*)rho, (const double*)u,
                                                         1.0 / rho0, 1.0 / e, nt, (S*)s0, (S*)s1);
  else
    set_walls_k<S, float><<<grid_for(g.n), 256, 0, st>>>(g, g.d, g.n, (const float*)rho, (const float*)u,
                                                        1.0 / rho0, 1.0 / e, nt, (S*)s0, (S*)s1);
  return cudaGetLastError();
}

cudaError_t launch_set_wall_values(const Geometry& g, int precision, const void* rho, const void* u,
                                   int dtype, double rho0, double e, const uint8_t* nt, void* s0,
                                   void* s1, cudaStream_t st) {
  if (!nt) return cudaSuccess;
  switch (precision) {
    case MACLAB_F64: return walls_t<double>(g, rho, u, dtype, rho0, e, nt, s0, s1, st);
    case MACLAB_F32: return walls_t<float>(g, rho, u, dtype, rho0, e, nt, s0, s1, st);
    case MACLAB_BF16_STORE: return walls_t<__nv_bfloat16>(g, rho, u, dtype, rho0, e, nt, s0, s1, st);
    case MACLAB_F16_STORE: return walls_t<__half>(g, rho, u, dtype, rho0, e, nt, s0, s1, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_fill_walls(const Geometry& g, int precision, const uint8_t* nt, const double* wl,
                              int nw, void* state, cudaStream_t st) {
  if (!nt) return cudaSuccess;
  switch (precision) {
    case MACLAB_F64:
      fill_walls_k<double><<<grid_for(g.n), 256, 0, st>>>(g.d, g.n, nt, wl, nw, (double*)state);
      break;
    case MACLAB_F32:
      fill_walls_k<float><<<grid_for(g.n), 256, 0, st>>>(g.d, g.n, nt, wl, nw, (float*)state);
      break;
    case MACLAB_BF16_STORE:
      fill_walls_k<__nv_bfloat16><<<grid_for(g.n), 256, 0, st>>>(g.d, g.n, nt, wl, nw,
                                                                 (__nv_bfloat16*)state);
      break;
    case MACLAB_F16_STORE:
      fill_walls_k<__half><<<grid_for(g.n), 256, 0, st>>>(g.d, g.n, nt, wl, nw, (__half*)state);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace maclab
