// step_tiled.cu -- host side of the tiled step kernel (see step_tiled.cuh):
// picks the block shape for a domain and dispatches to the instantiated
// kernels (step_tiled_d2q9.cu, step_tiled_d3q19_*.cu).

#include "step_tiled.cuh"

namespace maclab {

namespace {

// Instantiated shapes.  2D: (BXC, 1) for every storage type.  3D: (BXC, TY + 2)
// with the rows per tile TY; not every width is built for every storage type.
struct Shape3 {
  int bxc, ty;
  bool f64, f32, s16;
};
constexpr Shape3 kShapes3[] = {
    {16, 8, true, true, false},  {32, 4, true, true, true}, {32, 8, false, true, false},
    {64, 4, false, true, true},  {128, 2, false, true, false},
};

bool built3(const Shape3& s, int precision) {
  if (precision == MACLAB_F64) return s.f64;
  if (precision == MACLAB_F32) return s.f32;
  return s.s16;
}

}  // namespace

static bool tiled_shape(const Geometry& g, int precision, int ty_req, int tz_req, TiledShape* s) {
  const int bx = g.nx / 4;
  if (g.nx % 4 != 0 || bx < 1) return false;
  const size_t cb = precision == MACLAB_F64 ? 8 : 4;
  if (g.d == 2) {
    int bxc = 0;
    for (int c : {16, 32, 64, 128, 256})
      if (bx <= c) { bxc = c; break; }
    if (!bxc) return false;
    s->bxc = bxc;
    s->ry = 1;
    s->ty = 1;
    s->tz = tz_req > 0 ? tz_req : 8;
    s->smem = (kDoubleBuffer ? 2 : 1) * 2 * cb * (size_t)6 * (bxc + 2) + (size_t)kStages * 3 * bxc * 4 * cb;
    return g.ilv == 1;
  }
  int bxc = 0;
  for (int c : {16, 32, 64, 128})
    if (bx <= c) { bxc = c; break; }
  if (!bxc) return false;
  int ty = 0;
  for (const Shape3& sh : kShapes3) {
    if (sh.bxc != bxc || !built3(sh, precision)) continue;
    if (ty_req > 0 && sh.ty != ty_req) continue;
    if ((g.periodic & 2u) && g.ny % sh.ty != 0) continue;
    ty = sh.ty;
    break;
  }
  if (!ty) return false;
  s->bxc = bxc;
  s->ty = ty;
  s->ry = ty + 2;
  s->tz = tz_req > 0 ? tz_req : 8;
  s->smem = (kDoubleBuffer ? 2 : 1) * 2 * cb * ((size_t)6 * s->ry * (bxc + 2) + (size_t)10 * s->ry * 2 * (bxc + 2)) +
            (size_t)kStages * 4 * s->ry * bxc * 4 * cb;
  return g.ilv == 1 && s->smem <= 200 * 1024;
}

bool tiled_supported(const Geometry& g, int precision, int ty, int tz) {
  TiledShape s;
  return tiled_shape(g, precision, ty, tz, &s);
}

int tiled_threads(const Geometry& g, int precision, int ty, int tz) {
  TiledShape s;
  if (!tiled_shape(g, precision, ty, tz, &s)) return 0;
  return s.bxc * s.ry;
}

// Chunks of the march axis.  An explicit tz gives ceil(nplanes / tz) chunks.
// By default the block count is rounded to whole waves of the GPU (SMs x
// resident blocks), so no SM idles in the last wave, with chunks of at least
// 4 planes.
static int chunk_count(int nplanes, int ytiles, int tz_req, const TiledShape& s) {
  if (tz_req > 0) return (nplanes + tz_req - 1) / tz_req;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 148;
  }
  // resident blocks per SM from the shared-memory footprint (registers allow at
  // least two blocks of these shapes)
  int per_sm = (int)((227u * 1024u) / (s.smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 4) per_sm = 4;
  const long slots = (long)sms * per_sm;
  const int base = (nplanes + 7) / 8;  // ~8 planes per chunk
  const long blocks = (long)base * ytiles;
  const long waves = (blocks + slots - 1) / slots;
  int nzc = (int)((waves * slots) / ytiles);
  const int max_chunks = nplanes / 4 > 0 ? nplanes / 4 : 1;
  if (nzc > max_chunks) nzc = max_chunks;
  if (nzc < 1) nzc = 1;
  return nzc;
}

template <int LAT, typename S>
static cudaError_t dispatch(const TiledArgs& ta, const TiledShape& s, const void* in, void* out,
                            cudaStream_t st, dim3 grid) {
  if (LAT == kD2Q9) {
    switch (s.bxc) {
      case 16: return launch_shape<LAT, S, 16, 1>(ta, s, in, out, st, grid);
      case 32: return launch_shape<LAT, S, 32, 1>(ta, s, in, out, st, grid);
      case 64: return launch_shape<LAT, S, 64, 1>(ta, s, in, out, st, grid);
      case 128: return launch_shape<LAT, S, 128, 1>(ta, s, in, out, st, grid);
      case 256: return launch_shape<LAT, S, 256, 1>(ta, s, in, out, st, grid);
    }
    return cudaErrorInvalidValue;
  }
  const int key = s.bxc * 100 + s.ry;
  constexpr bool is64 = sizeof(S) == 8, is32 = sizeof(S) == 4;
  switch (key) {
    case 1610:
      if (is64 || is32) return launch_shape<LAT, S, 16, 10>(ta, s, in, out, st, grid);
      break;
    case 3206: return launch_shape<LAT, S, 32, 6>(ta, s, in, out, st, grid);
    case 3210:
      if (is32) return launch_shape<LAT, S, 32, 10>(ta, s, in, out, st, grid);
      break;
    case 6406:
      if (!is64) return launch_shape<LAT, S, 64, 6>(ta, s, in, out, st, grid);
      break;
    case 12804:
      if (is32) return launch_shape<LAT, S, 128, 4>(ta, s, in, out, st, grid);
      break;
  }
  return cudaErrorInvalidValue;
}

template <int LAT, typename S>
static cudaError_t launch_tiled_t(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  const Geometry& g = sl.g;
  TiledShape s;
  if (!tiled_shape(g, sl.precision, ty, tz, &s)) return cudaErrorInvalidValue;
  TiledArgs ta{};
  ta.nx = g.nx;
  ta.ny = g.d == 3 ? g.ny : 1;
  ta.nplanes = g.d == 3 ? g.nz : g.ny;
  ta.n = g.n;
  ta.plane_stride = (int64_t)g.nx * ta.ny;
  ta.ty = s.ty;
  const int ytiles = g.d == 3 ? (ta.ny + s.ty - 1) / s.ty : 1;
  ta.nzc = chunk_count(ta.nplanes, ytiles, tz, s);
  ta.px = (g.periodic & 1u) ? 1 : 0;
  ta.py = g.d == 3 ? ((g.periodic & 2u) ? 1 : 0) : 0;
  ta.pz = g.d == 3 ? ((g.periodic & 4u) ? 1 : 0) : ((g.periodic & 2u) ? 1 : 0);
  ta.wall_mode = g.wall_mode;
  ta.mask = g.mask;
  for (int i = 0; i < 3; ++i) ta.force[i] = sl.force[i];
  ta.overlap = sl.overlap;
  const dim3 grid(ta.nzc, ytiles);
  return dispatch<LAT, S>(ta, s, sl.in, sl.out, stream, grid);
}

template <int LAT>
static cudaError_t launch_tiled_lat(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  switch (sl.precision) {
    case MACLAB_F64: return launch_tiled_t<LAT, double>(sl, stream, ty, tz);
    case MACLAB_F32: return launch_tiled_t<LAT, float>(sl, stream, ty, tz);
    case MACLAB_BF16_STORE: return launch_tiled_t<LAT, __nv_bfloat16>(sl, stream, ty, tz);
    case MACLAB_F16_STORE: return launch_tiled_t<LAT, __half>(sl, stream, ty, tz);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tiled(const StepLaunch& sl, cudaStream_t stream, int ty, int tz) {
  return sl.g.lattice == kD2Q9 ? launch_tiled_lat<kD2Q9>(sl, stream, ty, tz)
                               : launch_tiled_lat<kD3Q19>(sl, stream, ty, tz);
}

}  // namespace maclab
