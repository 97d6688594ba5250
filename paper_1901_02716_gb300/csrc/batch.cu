// batch.cu -- many independent D2Q9 domains advanced by one persistent launch.
//
// Same update as step_naive / step_tiled (Eqs. (2), (4), (5) in the drho form
// of step.cu, the factored equilibrium and exact integer weights of
// step_tiled.cuh), organised for a batch of domains of different sizes:
//
//  * Work item = (domain, x segment, chunk of rows).  A warp takes items from
//    a work list (item = warp id + k * warps in the grid); items of all
//    domains are in one list, so one launch advances the whole batch.
//  * A warp covers 30 quads of its row segment (lanes 1..30) plus the quad on
//    each side (lanes 0 and 31, the halo), and marches over the rows of its
//    chunk plus a halo row on each side.  Storage rows interleave their two
//    halves (see common.cuh), so quad t holds the node pairs
//    a = (2t, 2t + H) and b = (2t + 1, 2t + 1 + H); a halo quad that wraps
//    around the row end is lane-swapped on load, which is what the seam
//    between the half rows needs.
//  * Equilibria moving +x leave pair b for the next lane's pair a, those moving
//    -x leave pair a for the previous lane's pair b: warp shuffles, no shared
//    memory, no block barrier.  The halo lanes' own sums are discarded.
//  * The three destination rows of momentum sums live in registers, as in
//    step_tiled.

#include <vector>

#include "step_tiled.cuh"

namespace maclab {

struct BatchInst {
  const void* buf[2];    // ping-pong state buffers (storage type, storage order)
  const uint8_t* mask;   // node types in storage order (kWallMask)
  int64_t n;             // nodes
  int nx, ny;            // nx % 4 == 0
  int px, py;            // periodic flags
  int wall_mode;
  float force[2];        // lattice-unit force increment (FP32 arithmetic)
  double force64[2];     // the same for FP64 storage
};

struct BatchItem {
  int inst, seg, y0, y1;
};

template <typename P>
__device__ __forceinline__ P shfl_up_pair(P v, int d) {
  P r;
  r.x = __shfl_up_sync(0xffffffffu, v.x, d);
  r.y = __shfl_up_sync(0xffffffffu, v.y, d);
  return r;
}
template <typename P>
__device__ __forceinline__ P shfl_down_pair(P v, int d) {
  P r;
  r.x = __shfl_down_sync(0xffffffffu, v.x, d);
  r.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return r;
}

// index of direction a among the directions with the same x component
template <int LAT>
__host__ __device__ constexpr int same_fx_index(int a) {
  int s = 0;
  for (int b = 0; b < a; ++b) s += Frame<LAT>::fx(b) == Frame<LAT>::fx(a) ? 1 : 0;
  return s;
}

// Contributions of one source row (state st of this lane's two pairs) to the
// sums of destination rows y - 1 (ap), y (ac), y + 1 (an); MODE as in step_tiled.
template <typename C, int MODE>
__device__ __forceinline__ void batch_row_update(const typename Pair<C>::P (&st)[3][2],
                                                 typename Pair<C>::P (&ap)[2][3],
                                                 typename Pair<C>::P (&ac)[2][3],
                                                 typename Pair<C>::P (&an)[2][3]) {
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<kD2Q9>;
  using F = Frame<kD2Q9>;
  P out_b[3], out_a[3];  // equilibria leaving pair b (+x) / pair a (-x)
#pragma unroll
  for (int k = 0; k < 3; ++k) out_b[k] = out_a[k] = O::splat(C(0));
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Terms<2, C> tm;
    const P u[3] = {st[1][q], st[2][q], O::splat(C(0))};
    make_terms<2, C>(st[0][q], u, tm);
    static_for<0, L::Q>([&](auto Ia) {
      constexpr int a = decltype(Ia)::value;
      if constexpr (mode_allows<kD2Q9, MODE>(a)) {
        constexpr int fx = F::fx(a), fz = F::fz(a);
        const P T = term<kD2Q9, C, a>(tm);
        const int qd = q + fx;
        if (qd >= 0 && qd < 2) {
          accum<kD2Q9, C, a>(pick<fz>(ap, ac, an)[qd], T);
        } else {
          if constexpr (fx == 1) out_b[same_fx_index<kD2Q9>(a)] = T;
          else if constexpr (fx == -1) out_a[same_fx_index<kD2Q9>(a)] = T;
        }
      }
    });
  }
  // +x: lane l - 1's pair b feeds lane l's pair a; -x: lane l + 1's pair a feeds pair b
  static_for<0, L::Q>([&](auto Ia) {
    constexpr int a = decltype(Ia)::value;
    if constexpr (mode_allows<kD2Q9, MODE>(a) && F::fx(a) != 0) {
      constexpr int fx = F::fx(a), fz = F::fz(a);
      if constexpr (fx == 1) {
        const P v = shfl_up_pair(out_b[same_fx_index<kD2Q9>(a)], 1);
        accum<kD2Q9, C, a>(pick<fz>(ap, ac, an)[0], v);
      } else {
        const P v = shfl_down_pair(out_a[same_fx_index<kD2Q9>(a)], 1);
        accum<kD2Q9, C, a>(pick<fz>(ap, ac, an)[1], v);
      }
    }
  });
}

template <typename S>
__global__ void __launch_bounds__(256) batch_step_d2q9(const BatchInst* __restrict__ insts,
                                                       const BatchItem* __restrict__ items,
                                                       int n_items, int cur) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<kD2Q9>;
  using F = Frame<kD2Q9>;
  constexpr int K = 3;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;

  for (int it = warp; it < n_items; it += nwarps) {
    const BatchItem item = items[it];
    const BatchInst& I = insts[item.inst];
    const S* in = static_cast<const S*>(I.buf[cur]);
    S* out = const_cast<S*>(static_cast<const S*>(I.buf[cur ^ 1]));
    const int nq = I.nx >> 2;
    const int n_int = min(30, nq - 30 * item.seg);
    int t = 30 * item.seg - 1 + lane;              // quad of this lane
    const bool interior = lane >= 1 && lane <= n_int;
    const bool active = lane <= n_int + 1;          // interior or halo
    bool swapped = false;
    if (t < 0) { t += nq; swapped = true; }
    if (t >= nq) { t -= nq; swapped = true; }
    const int64_t n = I.n;
    P force[2];
    if constexpr (sizeof(C) == 8) {
      force[0] = O::splat(C(I.force64[0]));
      force[1] = O::splat(C(I.force64[1]));
    } else {
      force[0] = O::splat(C(I.force[0]));
      force[1] = O::splat(C(I.force[1]));
    }
    const bool x_lo_wall = I.wall_mode == kWallBox && !I.px && t == 0 && interior;
    const bool x_hi_wall = I.wall_mode == kWallBox && !I.px && t == nq - 1 && interior;

    auto row_exists = [&](int y) { return (y >= 0 && y < I.ny) || I.py; };
    auto row_mem = [&](int y) { return y < 0 ? y + I.ny : (y >= I.ny ? y - I.ny : y); };
    auto load = [&](int y, P (&st)[K][2]) {
      const bool ok = active && row_exists(y);
      const int64_t off = (int64_t)row_mem(y) * I.nx + 4 * t;
#pragma unroll
      for (int f = 0; f < K; ++f) {
        if (ok) {
          Quad<S>::ld(in + f * n + off, st[f][0], st[f][1]);
          if (swapped) {
            st[f][0] = O::swap(st[f][0]);
            st[f][1] = O::swap(st[f][1]);
          }
        } else {
          st[f][0] = O::splat(C(0));
          st[f][1] = O::splat(C(0));
        }
      }
    };
    auto store = [&](int y, P (&acc)[2][K]) {
      if (!interior) return;
      if (!I.py && (y == 0 || y == I.ny - 1)) return;
      const int64_t off = (int64_t)y * I.nx + 4 * t;
      bool wall[4] = {x_lo_wall, false, false, x_hi_wall};
      bool any = x_lo_wall || x_hi_wall;
      if (I.wall_mode == kWallMask) {
        const uchar4 m = *reinterpret_cast<const uchar4*>(I.mask + off);
        wall[0] = m.x != 0; wall[1] = m.y != 0; wall[2] = m.z != 0; wall[3] = m.w != 0;
        any = wall[0] || wall[1] || wall[2] || wall[3];
      }
      P v[K][2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const P inv = O::rcp(O::add(O::splat(C(36)), acc[q][0]));
        v[0][q] = O::mul(acc[q][0], O::splat(C(1.0 / 36.0)));
        v[1][q] = O::fma(acc[q][1], inv, force[0]);
        v[2][q] = O::fma(acc[q][2], inv, force[1]);
      }
      if (!any) {
#pragma unroll
        for (int f = 0; f < K; ++f) Quad<S>::st(out + f * n + off, v[f][0], v[f][1]);
      } else {
#pragma unroll
        for (int f = 0; f < K; ++f) {
          if (!wall[0]) Quad<S>::st1(out + f * n + off + 0, v[f][0].x);
          if (!wall[1]) Quad<S>::st1(out + f * n + off + 1, v[f][0].y);
          if (!wall[2]) Quad<S>::st1(out + f * n + off + 2, v[f][1].x);
          if (!wall[3]) Quad<S>::st1(out + f * n + off + 3, v[f][1].y);
        }
      }
    };

    P R0[2][K], R1[2][K], R2[2][K];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) R0[q][k] = R1[q][k] = R2[q][k] = O::splat(C(0));
    P st[K][2], nxt[K][2];
    const int y0 = item.y0, y1 = item.y1;
    load(y0 - 1, st);
    load(y0, nxt);
    if (row_exists(y0 - 1))
      batch_row_update<C, kFirst>(st, R0, R2, R1);
    for (int y = y0; y < y1; ++y) {
#pragma unroll
      for (int f = 0; f < K; ++f) {
        st[f][0] = nxt[f][0];
        st[f][1] = nxt[f][1];
      }
      load(y + 1, nxt);
      batch_row_update<C, kMid>(st, R0, R1, R2);
      if (y - 1 >= y0) store(y - 1, R0);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          R0[q][k] = R1[q][k];
          R1[q][k] = R2[q][k];
          R2[q][k] = O::splat(C(0));
        }
    }
    if (row_exists(y1)) {
#pragma unroll
      for (int f = 0; f < K; ++f) {
        st[f][0] = nxt[f][0];
        st[f][1] = nxt[f][1];
      }
      batch_row_update<C, kLast>(st, R0, R1, R2);
    }
    store(y1 - 1, R0);
  }
}

template <typename S>
static cudaError_t launch_batch_t(const BatchInst* insts, const BatchItem* items, int n_items,
                                  int cur, int blocks, cudaStream_t st) {
  batch_step_d2q9<S><<<blocks, 256, 0, st>>>(insts, items, n_items, cur);
  return cudaGetLastError();
}

cudaError_t launch_batch_step(int precision, const void* insts, const void* items, int n_items,
                              int cur, int blocks, cudaStream_t st) {
  const BatchInst* I = static_cast<const BatchInst*>(insts);
  const BatchItem* T = static_cast<const BatchItem*>(items);
  switch (precision) {
    case MACLAB_F64: return launch_batch_t<double>(I, T, n_items, cur, blocks, st);
    case MACLAB_F32: return launch_batch_t<float>(I, T, n_items, cur, blocks, st);
    case MACLAB_BF16_STORE: return launch_batch_t<__nv_bfloat16>(I, T, n_items, cur, blocks, st);
    case MACLAB_F16_STORE: return launch_batch_t<__half>(I, T, n_items, cur, blocks, st);
  }
  return cudaErrorInvalidValue;
}

size_t batch_inst_bytes() { return sizeof(BatchInst); }
size_t batch_item_bytes() { return sizeof(BatchItem); }

// Host-side descriptor of one domain (filled by the API from a handle).
void batch_fill_inst(void* dst, const Geometry& g, void* buf0, void* buf1, const double force[3]) {
  BatchInst* b = static_cast<BatchInst*>(dst);
  b->buf[0] = buf0;
  b->buf[1] = buf1;
  b->mask = g.mask;
  b->n = g.n;
  b->nx = g.nx;
  b->ny = g.ny;
  b->px = (g.periodic & 1u) ? 1 : 0;
  b->py = (g.periodic & 2u) ? 1 : 0;
  b->wall_mode = g.wall_mode;
  b->force[0] = (float)force[0];
  b->force[1] = (float)force[1];
  b->force64[0] = force[0];
  b->force64[1] = force[1];
}

// Work items of one domain with `rows` rows per chunk.
void batch_items(int inst, const Geometry& g, int rows, std::vector<int>& out4) {
  const int nq = g.nx / 4;
  const int nseg = (nq + 29) / 30;
  for (int y0 = 0; y0 < g.ny; y0 += rows) {
    const int y1 = y0 + rows < g.ny ? y0 + rows : g.ny;
    for (int s = 0; s < nseg; ++s) {
      out4.push_back(inst);
      out4.push_back(s);
      out4.push_back(y0);
      out4.push_back(y1);
    }
  }
}

}  // namespace maclab
