// common.cuh -- storage types, loads/stores and the solver context shared by the
// CUDA translation units of libmaclab.  Internal: not part of the C ABI.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "maclab.h"

namespace maclab {

// ------------------------------------------------------------------ launch overlap
// Programmatic dependent launch.  A kernel queued by launch_kernel with
// overlap set may be scheduled onto the SMs while the kernel before it in the
// stream is still running.  Every such kernel calls pdl_wait() before it
// touches global memory: it returns once the previous kernel has completed
// and its writes are visible, so results do not depend on the overlap.
// pdl_launch_next() then lets the following kernel be scheduled.  Launched
// without the attribute (overlap 0), both are no-ops and the stream
// serialises the kernels as usual.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                          int overlap, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ------------------------------------------------------------------ bulk tensor copies
// One thread issues a TMA copy of a tile of a tensor map into shared memory;
// its completion is counted in bytes on an mbarrier that the consumers wait
// on.  Waits are bounded: a wait that runs out returns false (the caller
// records it in the device status word, step_status(), and carries on, so no
// thread leaves the block's barriers early).
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// mbarrier initialisation visible to the copy engine before the first copy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// shared memory the block has read made safe to overwrite by the copy engine
__device__ __forceinline__ void proxy_async_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds before a wait gives up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// tile at coordinates (x, y, z, w) of a 4-D tensor map into shared memory at dst
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void* map, int x, int y, int z, int w,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------------ bounds checks
// Debug builds (compiled with -DMACLAB_BOUNDS_CHECK; _build.build(bounds_check=True)
// makes libmaclab_bounds.so): the kernels that take a BoundsLog check each
// global and shared-memory index against the size of its buffer before the
// access; a bad index is counted, the first one recorded, and the access
// skipped (a load gives 0).  Nothing traps.  maclab_debug_bounds reads and
// clears the log.  In normal builds bounds_ok is the constant true and the
// checks compile away.
struct BoundsLog {
  unsigned long long count;
  long long first;
};
#ifdef MACLAB_BOUNDS_CHECK
__device__ __forceinline__ bool bounds_ok(BoundsLog* log, long long idx, long long limit) {
  if (idx >= 0 && idx < limit) return true;
  if (log && atomicAdd(&log->count, 1ull) == 0ull) log->first = idx;
  return false;
}
#else
__device__ __forceinline__ bool bounds_ok(BoundsLog*, long long, long long) { return true; }
#endif
// Device log of the current device (debug builds; nullptr otherwise).  Defined in api.cu.
BoundsLog* bounds_log();
// Defined in api.cu: the device status word of the current device (bit 0: a
// bounded wait on a copy ran out), allocated and zeroed on first use;
// maclab_sync reads and clears it.
unsigned* step_status();

// ------------------------------------------------------------------ storage

template <typename S>
struct Store;  // S = storage type; C = arithmetic type

template <>
struct Store<double> {
  using C = double;
  __device__ __forceinline__ static double ld(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static void st(double* p, double v) { *p = v; }
  __device__ __forceinline__ static double from(double v) { return v; }
  __device__ __forceinline__ static double to(double v) { return v; }
};
template <>
struct Store<float> {
  using C = float;
  __device__ __forceinline__ static float ld(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static void st(float* p, float v) { *p = v; }
  __device__ __forceinline__ static float from(float v) { return v; }
  __device__ __forceinline__ static float to(float v) { return v; }
};
template <>
struct Store<__nv_bfloat16> {
  using C = float;
  __device__ __forceinline__ static float ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  __device__ __forceinline__ static void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ __forceinline__ static float from(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static __nv_bfloat16 to(float v) { return __float2bfloat16_rn(v); }
};
template <>
struct Store<__half> {
  using C = float;
  __device__ __forceinline__ static float ld(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static void st(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ __forceinline__ static float from(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half to(float v) { return __float2half_rn(v); }
};

inline size_t storage_bytes(int precision) {
  switch (precision) {
    case MACLAB_F64: return 8;
    case MACLAB_F32: return 4;
    case MACLAB_BF16_STORE:
    case MACLAB_F16_STORE: return 2;
    default: return 0;
  }
}

// ------------------------------------------------------------------ geometry

// How wall nodes are identified inside the step kernels.
enum WallMode : int {
  kWallNone = 0,  // all nodes are fluid (fully periodic)
  kWallBox = 1,   // exactly the first/last layers of every non-periodic axis
  kWallMask = 2,  // explicit per-node byte mask (nonzero = wall)
};

struct Geometry {
  int lattice;        // kD2Q9 / kD3Q19
  int d;              // 2 or 3
  int nx, ny, nz;     // nz = 1 for D2Q9
  int64_t n;          // nx * ny * nz
  uint32_t periodic;  // bit0 x, bit1 y, bit2 z
  int wall_mode;      // WallMode
  const uint8_t* mask;  // device node types in storage order (kWallMask), else unused
  int ilv;            // 1: the two halves of every x row are interleaved in storage
  int hx;             // nx / 2 (used when ilv)
};

// Storage position within an x row of logical x, and its inverse.  With ilv
// (nx % 4 == 0) node x is stored at 2 (x mod H) + [x >= H], H = nx / 2, so that
// four consecutive stored values are the node pairs (x, x + H), (x + 1, x + 1 + H)
// the tiled kernel computes on; otherwise storage order is x itself.
__host__ __device__ inline int mem_x(const Geometry& g, int x) {
  return g.ilv ? (x < g.hx ? 2 * x : 2 * (x - g.hx) + 1) : x;
}
__host__ __device__ inline int log_x(const Geometry& g, int m) {
  return g.ilv ? (m >> 1) + (m & 1) * g.hx : m;
}

// Arguments of one step launch (device pointers to whole stored states).
struct StepLaunch {
  Geometry g;
  int precision;
  const void* in;
  void* out;
  double force[3];  // lattice-unit increment added after the division of Eq. (5)
  int ty = 0, tz = 0;  // tile shape of the tiled kernel (0 = default)
  // segment kernel: the domain's batch descriptor and work list on the device,
  // and the buffer the step reads (in = buf[cur] of the descriptor)
  const void* seg_inst = nullptr;
  const void* seg_items = nullptr;
  int seg_n_items = 0, seg_blocks = 0, cur = 0;
  int seg_depth = 1;  // steps per launch the work list was cut for (1 or 2)
  int seg_steps = 1;  // steps this launch advances (segment: 1, or 2 with seg_depth 2; block: 1 to 8)
  int overlap = 0;    // programmatic dependent launch (launch_kernel)
};

// Defined in step.cu.  Kernel ids follow MACLAB_KERNEL_* of maclab.h.
struct KernelInfo {
  int id;                // MACLAB_KERNEL_REFERENCE / _TILED / _FOLDED / _SEGMENT / _ROWS2 / _BLOCK
  int steps_per_launch;  // time steps one launch group advances
  int launches;          // kernel launches in one group
  int threads;           // threads per block
  const char* name;      // static name of the instance
};
bool step_kernel_supported(const Geometry& g, int precision, int kernel);
// Defined in step_block.cu: the block-resident D2Q9 kernel (ty = steps per
// launch: 1, 2, 4 or, with FP32 storage, 8; 0 = by size; FP32 / FP64 storage, nx % 4 == 0).
int block_steps(const Geometry& g, int precision, int ty);
bool block_supported(const Geometry& g, int precision, int ty);
int block_threads(int precision);
cudaError_t launch_block(const StepLaunch& s, cudaStream_t stream, int steps);
int segment_depth(const Geometry& g, int precision, int ty);
// Defined in batch.cu: `sweeps` two-step launches of the segment kernel in one
// persistent cooperative launch of `blocks` blocks, each waiting between sweeps
// (at most wait_limit polls; status bit 1 on a timeout) for the blocks on its
// list in deps (from batch_persist_deps); done: `blocks` device counters.
// batch_persist_capacity: the most blocks that can be resident at once.
cudaError_t launch_batch_step2_persist(int precision, const void* insts, const void* items, int n_items, int cur,
                                       int blocks, int sweeps, const int* deps, unsigned* done, unsigned* status,
                                       unsigned wait_limit, cudaStream_t st);
cudaError_t batch_persist_capacity(int precision, int* capacity);
// ny[i], py[i]: rows and y periodicity of domain i of the work list.
void batch_persist_deps(const std::vector<int>& items4, const std::vector<int>& ny, const std::vector<int>& py,
                        int blocks, std::vector<int>& out);
int segment_rows(const Geometry& g, int precision, int ty, int tz);
int pick_step_kernel(const Geometry& g, int precision);
KernelInfo describe_step_kernel(const Geometry& g, int precision, int kernel, int ty, int tz);
// Queue one launch group of `kernel` (advances steps_per_launch steps).
cudaError_t launch_step(const StepLaunch& s, cudaStream_t stream, int kernel);

// Defined in step_tiled.cu.
bool tiled_supported(const Geometry& g, int precision, int ty, int tz);
cudaError_t launch_tiled(const StepLaunch& s, cudaStream_t stream, int ty, int tz);
int tiled_threads(const Geometry& g, int precision, int ty, int tz);

// Defined in step_fold.cu (D3Q19 FP32 without halo-row threads).
bool fold_supported(const Geometry& g, int precision, int ty);
int fold_threads(const Geometry& g, int precision, int ty);
cudaError_t launch_fold(const StepLaunch& s, cudaStream_t stream, int ty, int tz);
// Chunks of the march axis for a grid of ytiles tiles per plane with per_sm
// resident blocks per SM (tz_req > 0: planes per chunk as asked).
int fold_chunks(int nplanes, int ytiles, int tz_req, int per_sm);

// Defined in step_rows2.cu (D3Q19, two rows per thread; FP32 arithmetic).
bool rows2_supported(const Geometry& g, int precision, int ty);
int rows2_threads(const Geometry& g, int precision, int ty);
cudaError_t launch_rows2(const StepLaunch& s, cudaStream_t stream, int ty, int tz);
// The viscosity term of one reverse step (maclab_adjoint_nu_term) on the two-rows
// kernel: FP32 storage where the step kernel is built; acc += the sum.
bool rows2_nu_supported(const Geometry& g, int precision);
cudaError_t launch_rows2_nu(const Geometry& g, const void* state_n, const void* state_np1, const float* lam,
                            const double force[3], double* acc, int overlap, cudaStream_t stream);

// Defined in api.cu: message returned by maclab_last_error on this thread.
void record_error(const char* msg);

// Defined in reduce.cu.
constexpr int kDiagOut = 9;
int diag_blocks(int64_t n);
cudaError_t launch_diagnostics(const Geometry& g, int precision, const void* cur, const void* prev,
                               double* partial, unsigned* ticket, int nblocks, double* out,
                               cudaStream_t st, int overlap);

// Defined in adjoint.cu.
cudaError_t launch_adjoint_step(const Geometry& g, int precision, const void* state_n,
                                const void* state_np1, const void* lam_np1, void* lam_n,
                                void* scratch, const double force_lat[3], double* grad_force,
                                cudaStream_t st);
// Defined in selfcheck.cu: the largest relative error of the FP32 pair
// reciprocal over n points in [lo, hi], as double bits, into *d_worst.
cudaError_t launch_check_reciprocal(float lo, float hi, int n, unsigned long long* d_worst,
                                    cudaStream_t st);
// Defined in selfcheck.cu: one launch of the paired-FP32 FMA rate kernel;
// *flops receives the floating-point operations it performs.
cudaError_t launch_fp32_peak(int blocks, int threads, int iters, float2* sink, cudaStream_t st,
                             double* flops);
// Defined in adjoint_tiled.cu (domains with interleaved rows).
bool tiled_adjoint_supported(const Geometry& g, int precision);
cudaError_t launch_tiled_adjoint(const Geometry& g, int precision, const void* state_n,
                                 const void* state_np1, const void* lam_np1, void* lam_n,
                                 const double force_lat[3], double* grad_force, int overlap, cudaStream_t st);
// sum over fluid x of lam_np1(x) . D_n(x), the viscosity term of one reverse step, into *acc
cudaError_t launch_adjoint_nu_term(const Geometry& g, int precision, const void* state_n, const void* lam_np1,
                                   const double force_lat[3], double* acc, cudaStream_t st);
cudaError_t launch_adjoint_seed(const Geometry& g, int precision, const void* grho, const void* gu,
                                int dtype, const void* state, double rho0, double e, void* lam,
                                double* dot, cudaStream_t st);
cudaError_t launch_adjoint_finish(const Geometry& g, int precision, const void* lam, const void* state,
                                  const uint8_t* nt, int nw, double rho0, double e, void* grho,
                                  void* gu, int dtype, double* wall, double* dot, cudaStream_t st);

// Defined in batch.cu.
// segw: quads per segment of the work list (30 when it was cut for one step per launch)
cudaError_t launch_batch_step(int precision, const void* insts, const void* items, int n_items,
                              int cur, int blocks, int segw, cudaStream_t st, int overlap);
constexpr int kBatchSegW1 = 30, kBatchSegW2 = 28;
// two time steps per launch (FP32 / FP64 storage, every nx >= 8), 128-thread blocks
cudaError_t launch_batch_step2(int precision, const void* insts, const void* items, int n_items,
                               int cur, int blocks, cudaStream_t st, int overlap);
size_t batch_inst_bytes();
size_t batch_item_bytes();
void batch_fill_inst(void* dst, const Geometry& g, void* buf0, void* buf1, const double force[3]);
void batch_items(int inst, const Geometry& g, int rows, int depth, std::vector<int>& out4);

// Defined in convert.cu.
cudaError_t launch_set_physical(const Geometry& g, int precision, const void* rho,
                                const void* u, int dtype, double rho0, double e,
                                const uint8_t* node_type, const double* wall_lat,
                                int n_wall_ids, void* state, cudaStream_t stream);
cudaError_t launch_get_physical(const Geometry& g, int precision, const void* state,
                                void* rho, void* u, int dtype, double rho0, double e,
                                cudaStream_t stream);
cudaError_t launch_set_wall_values(const Geometry& g, int precision, const void* rho, const void* u,
                                   int dtype, double rho0, double e, const uint8_t* node_type, void* s0,
                                   void* s1, cudaStream_t stream);
cudaError_t launch_fill_walls(const Geometry& g, int precision, const uint8_t* node_type,
                              const double* wall_lat, int n_wall_ids, void* state,
                              cudaStream_t stream);

}  // namespace maclab

// ------------------------------------------------------------------ the handle

struct maclab_ctx {
  maclab::Geometry g{};
  int precision = MACLAB_F32;
  double dx = 0, nu = 0, rho0 = 1, e = 0, dt = 0, rle = 0;
  double force_phys[3] = {0, 0, 0};
  double force_lat[3] = {0, 0, 0};
  int n_wall_ids = 0;
  std::vector<double> wall_rho, wall_u;  // physical, n_wall_ids and n_wall_ids * 3
  std::vector<double> wall_lat;          // lattice units, n_wall_ids * 4 (drho, u0, u1, u2)
  int64_t n_fluid = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  uint8_t* d_node_type = nullptr;  // device copy of the node types (if any walls)
  double* d_wall_lat = nullptr;    // device copy of wall_lat
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;                     // buf[cur] holds the current state
  size_t elem = 4;                 // bytes per stored value
  int64_t steps = 0;
  int kernel = MACLAB_KERNEL_REFERENCE;
  int ty = 0, tz = 0;              // tiled-kernel shape (0 = default)
  int overlap = 1;                 // programmatic dependent launch of the step kernels
  void* d_staging = nullptr;       // device staging for host set/get
  size_t staging_cap = 0;
  bool prev_valid = false;         // buf[cur ^ 1] holds the state one step back
  double* d_partial = nullptr;     // diagnostics scratch (per-block partial sums)
  double* d_diag = nullptr;        // diagnostics result (kDiagOut doubles)
  double* h_diag = nullptr;        // page-locked host copy of it
  int diag_nblocks = 0;
  // CUDA graphs of graph_steps steps, one per starting buffer
  int graph_steps = 32;
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  // segment kernel (a batch of this one domain): descriptor, work list
  void* d_seg_inst = nullptr;
  void* d_seg_items = nullptr;
  int* d_seg_deps = nullptr;       // persistent segment launches: each block's wait list
  unsigned* d_seg_done = nullptr;  // and the blocks' finished-sweep counters
  int seg_n_items = 0, seg_blocks = 0, seg_rows = 0, seg_depth = 1, seg_persist_blocks = 0;
  std::vector<int> seg_items_host;  // the work list (4 ints per item) the wait lists are built from
  unsigned wait_limit = maclab::kWaitLimit;  // polls before a wait between blocks gives up
  void* d_adj_scratch = nullptr;   // reference adjoint: (L_r, L_m) at every node
  double* d_adj_red = nullptr;     // adjoint: reductions (1 + 4 * n_wall_ids doubles)
};
