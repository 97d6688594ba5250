// adjoint_tiled.cu -- host side of the tiled reverse step (adjoint_tiled.cuh):
// block shapes, instantiations and the launch.

#include "adjoint_tiled.cuh"

namespace maclab {

namespace {

struct AdjShape {
  int bxc, ry, ty;
};

// Widths built: D2Q9 (BXC, 1); D3Q19 (BXC, TY + 2).  FP64 up to 64 quads per row in 3D,
// 128 in 2D.
bool adj_shape(const Geometry& g, int precision, AdjShape* s) {
  if (!g.ilv || precision == MACLAB_BF16_STORE || precision == MACLAB_F16_STORE) return false;
  const int bx = g.nx / 4;
  int bxc = 0;
  for (int c : {16, 32, 64, 128, 256})
    if (bx <= c) { bxc = c; break; }
  if (!bxc) return false;
  if (g.d == 2) {
    if (precision == MACLAB_F64 && bxc > 128) return false;
    *s = AdjShape{bxc, 1, 1};
    return true;
  }
  int ty = 0;
  switch (bxc) {
    case 16: ty = 8; break;
    case 32: ty = 4; break;
    case 64: ty = 4; break;
    case 128: ty = 2; break;
    default: return false;
  }
  if (precision == MACLAB_F64 && bxc > 64) return false;
  if ((g.periodic & 2u) && g.ny % ty != 0) return false;  // a periodic y needs whole tiles
  *s = AdjShape{bxc, ty + 2, ty};
  return true;
}

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 148;
  }
  return n;
}

template <int LAT, typename S>
cudaError_t tiled_dispatch(const AdjShape& s, const AdjArgs& A, const void* sn, const void* sn1,
                           const void* lam1, void* lam0, double* gf, cudaStream_t st, int ytiles,
                           int* resident) {
#define MACLAB_ADJ_LAUNCH(BXC, RY) \
  launch_adj_tiled<LAT, S, BXC, RY>(A, sn, sn1, lam1, lam0, gf, st, ytiles, resident)
  if (LAT == kD2Q9) {
    switch (s.bxc) {
      case 16: return MACLAB_ADJ_LAUNCH(16, 1);
      case 32: return MACLAB_ADJ_LAUNCH(32, 1);
      case 64: return MACLAB_ADJ_LAUNCH(64, 1);
      case 128: return MACLAB_ADJ_LAUNCH(128, 1);
      case 256:
        if constexpr (sizeof(S) == 4) return MACLAB_ADJ_LAUNCH(256, 1);
        break;
    }
    return cudaErrorInvalidValue;
  }
  switch (s.bxc * 100 + s.ry) {
    case 1610: return MACLAB_ADJ_LAUNCH(16, 10);
    case 3206: return MACLAB_ADJ_LAUNCH(32, 6);
    case 6406: return MACLAB_ADJ_LAUNCH(64, 6);
    case 12804:
      if constexpr (sizeof(S) == 4) return MACLAB_ADJ_LAUNCH(128, 4);
      break;
  }
#undef MACLAB_ADJ_LAUNCH
  return cudaErrorInvalidValue;
}

template <int LAT, typename S>
cudaError_t tiled_adjoint_t(const Geometry& g, const AdjShape& s, const void* sn, const void* sn1,
                            const void* lam1, void* lam0, const double* force, double* gf,
                            int overlap, cudaStream_t st) {
  AdjArgs A{};
  A.overlap = overlap;
  A.nx = g.nx;
  A.ny = g.d == 3 ? g.ny : 1;
  A.nplanes = g.d == 3 ? g.nz : g.ny;
  A.n = g.n;
  A.plane_stride = (int64_t)g.nx * A.ny;
  A.ty = s.ty;
  A.px = (g.periodic & 1u) ? 1 : 0;
  A.py = g.d == 3 ? ((g.periodic & 2u) ? 1 : 0) : 0;
  A.pz = g.d == 3 ? ((g.periodic & 4u) ? 1 : 0) : ((g.periodic & 2u) ? 1 : 0);
  A.wall_mode = g.wall_mode;
  A.mask = g.mask;
  for (int i = 0; i < 3; ++i) A.force[i] = force[i];
  const int ytiles = g.d == 3 ? (A.ny + s.ty - 1) / s.ty : 1;
  int resident = 0;
  cudaError_t e = tiled_dispatch<LAT, S>(s, A, sn, sn1, lam1, lam0, gf, st, ytiles, &resident);
  if (e != cudaSuccess) return e;
  // about 8 planes per block, rounded up to whole waves of resident blocks
  int nzc = (A.nplanes + 7) / 8;
  const long slots = (long)resident * sms();
  const long blocks = (long)nzc * ytiles;
  const long waves = (blocks + slots - 1) / slots;
  nzc = (int)((waves * slots) / ytiles);
  if (nzc > A.nplanes / 2) nzc = A.nplanes / 2 > 0 ? A.nplanes / 2 : 1;
  if (nzc < 1) nzc = 1;
  A.nzc = nzc;
  return tiled_dispatch<LAT, S>(s, A, sn, sn1, lam1, lam0, gf, st, ytiles, nullptr);
}

}  // namespace

bool tiled_adjoint_supported(const Geometry& g, int precision) {
  AdjShape s;
  return adj_shape(g, precision, &s);
}

cudaError_t launch_tiled_adjoint(const Geometry& g, int precision, const void* state_n,
                                 const void* state_np1, const void* lam_np1, void* lam_n,
                                 const double force_lat[3], double* grad_force, int overlap, cudaStream_t st) {
  AdjShape s;
  if (!adj_shape(g, precision, &s)) return cudaErrorInvalidValue;
  if (g.lattice == kD2Q9) {
    if (precision == MACLAB_F64)
      return tiled_adjoint_t<kD2Q9, double>(g, s, state_n, state_np1, lam_np1, lam_n, force_lat, grad_force, overlap, st);
    return tiled_adjoint_t<kD2Q9, float>(g, s, state_n, state_np1, lam_np1, lam_n, force_lat, grad_force, overlap, st);
  }
  if (precision == MACLAB_F64)
    return tiled_adjoint_t<kD3Q19, double>(g, s, state_n, state_np1, lam_np1, lam_n, force_lat, grad_force, overlap, st);
  return tiled_adjoint_t<kD3Q19, float>(g, s, state_n, state_np1, lam_np1, lam_n, force_lat, grad_force, overlap, st);
}

}  // namespace maclab
