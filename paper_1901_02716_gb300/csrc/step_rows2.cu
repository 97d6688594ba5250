// step_rows2.cu -- host side of the D3Q19 step with two rows per thread
// (step_rows2.cuh): block shapes, chunking of the march axis, instances.

#include <cudaTypedefs.h>  // the driver's cuTensorMapEncodeTiled signature

#include "step_rows2.cuh"

namespace maclab {

namespace {

// (BXC, TYT) in order of preference for each row width (the first whose tile
// of 2 TYT rows divides ny is the default); 16-bit storage: TYT = 4 only.
struct Rows2Shape {
  int bxc, tyt;
};
constexpr Rows2Shape kRows2Shapes[] = {{16, 4}, {32, 4}, {32, 2}};

bool rows2_precision(int precision) {
  return precision == MACLAB_F32 || precision == MACLAB_BF16_STORE || precision == MACLAB_F16_STORE;
}

// ty: rows per tile asked (0 = default), i.e. 2 TYT
bool rows2_shape(const Geometry& g, int precision, int ty, Rows2Shape* out) {
  if (g.d != 3 || g.lattice != kD3Q19 || !g.ilv || !rows2_precision(precision)) return false;
  const int bx = g.nx / 4;
  int bxc = 0;
  for (int c : {16, 32})
    if (bx <= c) { bxc = c; break; }
  if (!bxc) return false;
  for (const Rows2Shape& s : kRows2Shapes) {
    if (s.bxc != bxc || (ty > 0 && 2 * s.tyt != ty)) continue;
    if (precision != MACLAB_F32 && s.tyt != 4) continue;
    // a tile copy's row is nx stored values: a multiple of 16 bytes
    if (precision != MACLAB_F32 && g.nx % 8 != 0) continue;
    if (g.ny % (2 * s.tyt) != 0) continue;
    *out = s;
    return true;
  }
  return false;
}

// The driver's tensor-map encoder, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// Tile copies of the state at `base` (layout [4 fields][nz][ny][nx], storage
// type of `precision`): a box of ty rows of every field, and one of a single row.
cudaError_t rows2_maps(const Geometry& g, int precision, int ty, const void* base, CUtensorMap* own,
                       CUtensorMap* halo) {
  const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0) return cudaErrorMisalignedAddress;
  const CUtensorMapDataType dt = precision == MACLAB_F32         ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : precision == MACLAB_BF16_STORE ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t es = precision == MACLAB_F32 ? 4 : 2;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 4};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es, (cuuint64_t)g.n * es};
  const cuuint32_t box_own[4] = {(cuuint32_t)g.nx, (cuuint32_t)ty, 1, 4};
  const cuuint32_t box_row[4] = {(cuuint32_t)g.nx, 1, 1, 4};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  void* gp = const_cast<void*>(base);
  if (encode(own, dt, 4, gp, dims, strides, box_own, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      encode(halo, dt, 4, gp, dims, strides, box_row, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

}  // namespace

template <typename S>
cudaError_t rows2_dispatch(int bxc, int tyt, const TiledArgs& ta, const void* in, void* out,
                           const CUtensorMap& tm_own, const CUtensorMap& tm_halo, cudaStream_t st, dim3 grid,
                           int* resident) {
  switch (bxc * 100 + tyt) {
    case 1604: return launch_rows2_shape<S, 16, 4>(ta, in, out, tm_own, tm_halo, st, grid, resident);
    case 3202: return launch_rows2_shape<S, 32, 2>(ta, in, out, tm_own, tm_halo, st, grid, resident);
    case 3204: return launch_rows2_shape<S, 32, 4>(ta, in, out, tm_own, tm_halo, st, grid, resident);
  }
  return cudaErrorInvalidValue;
}
template cudaError_t rows2_dispatch<float>(int, int, const TiledArgs&, const void*, void*, const CUtensorMap&,
                                          const CUtensorMap&, cudaStream_t, dim3, int*);

bool rows2_supported(const Geometry& g, int precision, int ty) {
  Rows2Shape s;
  return rows2_shape(g, precision, ty, &s);
}

int rows2_threads(const Geometry& g, int precision, int ty) {
  Rows2Shape s;
  return rows2_shape(g, precision, ty, &s) ? s.bxc * s.tyt : 0;
}

cudaError_t launch_rows2(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  const Geometry& g = sl.g;
  Rows2Shape s;
  if (!rows2_shape(g, sl.precision, ty, &s)) return cudaErrorInvalidValue;
  TiledArgs ta{};
  ta.nx = g.nx;
  ta.ny = g.ny;
  ta.nplanes = g.nz;
  ta.n = g.n;
  ta.plane_stride = (int64_t)g.nx * g.ny;
  ta.ty = 2 * s.tyt;
  const int ytiles = g.ny / ta.ty;
  CUtensorMap tm_own{}, tm_halo{};
  auto dispatch = [&](const void* in, void* out, dim3 grid, int* resident) {
    switch (sl.precision) {
      case MACLAB_F32:
        return rows2_dispatch<float>(s.bxc, s.tyt, ta, in, out, tm_own, tm_halo, stream, grid, resident);
      case MACLAB_BF16_STORE:
        return rows2_dispatch<__nv_bfloat16>(s.bxc, s.tyt, ta, in, out, tm_own, tm_halo, stream, grid, resident);
      case MACLAB_F16_STORE:
        return rows2_dispatch<__half>(s.bxc, s.tyt, ta, in, out, tm_own, tm_halo, stream, grid, resident);
    }
    return cudaErrorInvalidValue;
  };
  int resident = 0;
  cudaError_t e = dispatch(nullptr, nullptr, dim3(), &resident);
  if (e != cudaSuccess) return e;
  e = rows2_maps(g, sl.precision, ta.ty, sl.in, &tm_own, &tm_halo);
  if (e != cudaSuccess) return e;
  ta.nzc = fold_chunks(ta.nplanes, ytiles, tz, resident);
  ta.px = (g.periodic & 1u) ? 1 : 0;
  ta.py = (g.periodic & 2u) ? 1 : 0;
  ta.pz = (g.periodic & 4u) ? 1 : 0;
  ta.wall_mode = g.wall_mode;
  ta.mask = g.mask;
  for (int i = 0; i < 3; ++i) ta.force[i] = sl.force[i];
  ta.overlap = sl.overlap;
  ta.bounds = bounds_log();
  ta.status = step_status();
  return dispatch(sl.in, sl.out, dim3(ta.nzc, ytiles), nullptr);
}

bool rows2_nu_supported(const Geometry& g, int precision) {
  Rows2Shape s;
  return precision == MACLAB_F32 && rows2_shape(g, precision, 0, &s);
}

cudaError_t launch_rows2_nu(const Geometry& g, const void* state_n, const void* state_np1, const float* lam,
                            const double force[3], double* acc, int overlap, cudaStream_t stream) {
  Rows2Shape s;
  if (!rows2_nu_supported(g, MACLAB_F32) || !rows2_shape(g, MACLAB_F32, 0, &s)) return cudaErrorInvalidValue;
  TiledArgs ta{};
  ta.nx = g.nx;
  ta.ny = g.ny;
  ta.nplanes = g.nz;
  ta.n = g.n;
  ta.plane_stride = (int64_t)g.nx * g.ny;
  ta.ty = 2 * s.tyt;
  const int ytiles = g.ny / ta.ty;
  CUtensorMap tm_own{}, tm_halo{};
  int resident = 0;
  cudaError_t e = rows2_nu_dispatch(s.bxc, s.tyt, ta, nullptr, nullptr, tm_own, tm_halo, stream, dim3(), &resident);
  if (e != cudaSuccess) return e;
  e = rows2_maps(g, MACLAB_F32, ta.ty, state_n, &tm_own, &tm_halo);
  if (e != cudaSuccess) return e;
  ta.nzc = fold_chunks(ta.nplanes, ytiles, 0, resident);
  ta.px = (g.periodic & 1u) ? 1 : 0;
  ta.py = (g.periodic & 2u) ? 1 : 0;
  ta.pz = (g.periodic & 4u) ? 1 : 0;
  ta.wall_mode = g.wall_mode;
  ta.mask = g.mask;
  for (int i = 0; i < 3; ++i) ta.force[i] = force[i];
  ta.overlap = overlap;  // waits for the previous kernel before reading (pdl_wait)
  ta.bounds = bounds_log();
  ta.lam = lam;
  ta.nu_acc = acc;
  ta.status = step_status();
  return rows2_nu_dispatch(s.bxc, s.tyt, ta, state_n, state_np1, tm_own, tm_halo, stream, dim3(ta.nzc, ytiles),
                           nullptr);
}

}  // namespace maclab
