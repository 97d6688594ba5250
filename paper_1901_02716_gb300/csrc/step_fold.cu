// step_fold.cu -- host side of the D3Q19 step without halo-row threads
// (step_fold.cuh): block shapes, chunking of the march axis, instances.

#include "step_fold.cuh"

namespace maclab {

namespace {

// Instantiated (BXC, TY) in order of preference for each width (the first whose
// TY divides ny is the default): FP32 all of them, 16-bit storage (32, 8),
// (32, 4), (64, 4) and (128, 4).
constexpr FoldShape kFoldShapes[] = {{16, 8}, {32, 8}, {32, 4}, {64, 4}, {64, 8}, {128, 4}};

bool fold_shape_built(const FoldShape& s, int precision) {
  if (precision == MACLAB_F32) return true;
  if (precision == MACLAB_BF16_STORE || precision == MACLAB_F16_STORE)
    return (s.bxc == 32 && (s.ty == 8 || s.ty == 4)) || ((s.bxc == 64 || s.bxc == 128) && s.ty == 4);
  return false;
}

bool fold_shape(const Geometry& g, int precision, int ty_req, FoldShape* out) {
  if (g.d != 3 || g.lattice != kD3Q19 || !g.ilv || precision == MACLAB_F64) return false;
  const int bx = g.nx / 4;
  int bxc = 0;
  for (int c : {16, 32, 64, 128})
    if (bx <= c) { bxc = c; break; }
  if (!bxc) return false;
  for (const FoldShape& s : kFoldShapes) {
    if (s.bxc != bxc || (ty_req > 0 && s.ty != ty_req) || !fold_shape_built(s, precision)) continue;
    if (g.ny % s.ty != 0) continue;  // every row of a tile exists
    *out = s;
    return true;
  }
  return false;
}

template <typename S>
cudaError_t fold_dispatch(const FoldShape& s, const TiledArgs& ta, const void* in, void* out,
                          cudaStream_t st, dim3 grid, int* resident) {
  switch (s.bxc * 100 + s.ty) {
    case 1608: return launch_fold_shape<S, 16, 8>(ta, in, out, st, grid, resident);
    case 3204: return launch_fold_shape<S, 32, 4>(ta, in, out, st, grid, resident);
    case 3208: return launch_fold_shape<S, 32, 8>(ta, in, out, st, grid, resident);
    case 6404: return launch_fold_shape<S, 64, 4>(ta, in, out, st, grid, resident);
    case 6408: return launch_fold_shape<S, 64, 8>(ta, in, out, st, grid, resident);
    case 12804: return launch_fold_shape<S, 128, 4>(ta, in, out, st, grid, resident);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

static int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
  }
  return sms;
}

// Chunks of the march axis: an explicit tz gives ceil(nplanes / tz).  By
// default the chunks are as long as possible (every chunk re-reads and
// half-processes a plane at each end) while the grid still fills two waves of
// resident blocks: 32 planes, halved down to 8 until it does; then the block
// count is rounded up to whole waves and chunks are kept to at least 4 planes.
int fold_chunks(int nplanes, int ytiles, int tz_req, int per_sm) {
  if (tz_req > 0) return (nplanes + tz_req - 1) / tz_req;
  const long slots = (long)sm_count() * (per_sm < 1 ? 1 : per_sm);
  int tz = 32;
  while (tz > 8 && (long)((nplanes + tz - 1) / tz) * ytiles < 2 * slots) tz /= 2;
  const long blocks = (long)((nplanes + tz - 1) / tz) * ytiles;
  const long waves = (blocks + slots - 1) / slots;
  int nzc = (int)((waves * slots) / ytiles);
  const int max_chunks = nplanes / 4 > 0 ? nplanes / 4 : 1;
  if (nzc > max_chunks) nzc = max_chunks;
  if (nzc < 1) nzc = 1;
  return nzc;
}


bool fold_supported(const Geometry& g, int precision, int ty) {
  FoldShape s;
  return fold_shape(g, precision, ty, &s);
}

int fold_threads(const Geometry& g, int precision, int ty) {
  FoldShape s;
  return fold_shape(g, precision, ty, &s) ? s.bxc * s.ty : 0;
}

cudaError_t launch_fold(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  const Geometry& g = sl.g;
  FoldShape s;
  if (!fold_shape(g, sl.precision, ty, &s)) return cudaErrorInvalidValue;
  TiledArgs ta{};
  ta.nx = g.nx;
  ta.ny = g.ny;
  ta.nplanes = g.nz;
  ta.n = g.n;
  ta.plane_stride = (int64_t)g.nx * g.ny;
  ta.ty = s.ty;
  const int ytiles = g.ny / s.ty;
  auto dispatch = [&](const void* in, void* out, dim3 grid, int* resident) {
    return sl.precision == MACLAB_F32 ? fold_dispatch<float>(s, ta, in, out, stream, grid, resident)
                                      : fold_dispatch_s16(sl.precision, s, ta, in, out, stream, grid, resident);
  };
  int resident = 0;
  cudaError_t e = dispatch(nullptr, nullptr, dim3(), &resident);
  if (e != cudaSuccess) return e;
  ta.nzc = fold_chunks(ta.nplanes, ytiles, tz, resident);
  ta.px = (g.periodic & 1u) ? 1 : 0;
  ta.py = (g.periodic & 2u) ? 1 : 0;
  ta.pz = (g.periodic & 4u) ? 1 : 0;
  ta.wall_mode = g.wall_mode;
  ta.mask = g.mask;
  for (int i = 0; i < 3; ++i) ta.force[i] = sl.force[i];
  ta.overlap = sl.overlap;
  return dispatch(sl.in, sl.out, dim3(ta.nzc, ytiles), nullptr);
}

}  // namespace maclab
