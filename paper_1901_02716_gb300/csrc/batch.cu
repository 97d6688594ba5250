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
//    -x leave pair a for the previous lane's pair b: warp shuffles, no block
//    barrier.  The halo lanes' own sums are discarded.
//  * Input rows are prefetched one row ahead in registers (the two-step
//    kernel below stages them four rows ahead through shared memory).
//  * The three destination rows of momentum sums live in registers, as in
//    step_tiled.

#include <algorithm>
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


// Store of one final row (Eq. (5): u' = M / (36 + R) + F).  In box mode every
// lane stores its whole quad: a lane whose quad holds one x-wall node (a.x at
// x = 0, b.y at x = nx - 1) puts that node's unchanged fields wk in place of
// the computed ones, so the warp never splits into per-node stores.  Masks,
// and a quad holding both x-walls (nx = 4), store node by node.
template <typename S>
__device__ __forceinline__ void batch_store(S* out, int64_t n, int64_t off, const uint8_t* mask, int wall_mode,
                                            bool x_lo_wall, bool x_hi_wall,
                                            const typename Store<S>::C (&wk)[3],
                                            const typename Pair<typename Store<S>::C>::P (&acc)[2][3],
                                            const typename Pair<typename Store<S>::C>::P (&force)[2]) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int K = 3;
  P v[K][2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const P inv = O::rcp(O::add(O::splat(C(36)), acc[q][0]));
    v[0][q] = O::mul(acc[q][0], O::splat(C(1.0 / 36.0)));
    v[1][q] = O::fma(acc[q][1], inv, force[0]);
    v[2][q] = O::fma(acc[q][2], inv, force[1]);
  }
  if (wall_mode == kWallMask || (x_lo_wall && x_hi_wall)) {
    bool wall[4] = {x_lo_wall, false, false, x_hi_wall};
    if (wall_mode == kWallMask) {
      const uchar4 m = *reinterpret_cast<const uchar4*>(mask + off);
      wall[0] = m.x != 0; wall[1] = m.y != 0; wall[2] = m.z != 0; wall[3] = m.w != 0;
    }
    if (!(wall[0] || wall[1] || wall[2] || wall[3])) {
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<S>::st(out + f * n + off, v[f][0], v[f][1]);
      return;
    }
#pragma unroll
    for (int f = 0; f < K; ++f) {
      if (!wall[0]) Quad<S>::st1(out + f * n + off + 0, v[f][0].x);
      if (!wall[1]) Quad<S>::st1(out + f * n + off + 1, v[f][0].y);
      if (!wall[2]) Quad<S>::st1(out + f * n + off + 2, v[f][1].x);
      if (!wall[3]) Quad<S>::st1(out + f * n + off + 3, v[f][1].y);
    }
    return;
  }
#pragma unroll
  for (int f = 0; f < K; ++f) {
    if (x_lo_wall) v[f][0].x = wk[f];
    if (x_hi_wall) v[f][1].y = wk[f];
    Quad<S>::st(out + f * n + off, v[f][0], v[f][1]);
  }
}

// segw: quads per work item's segment (30, or fewer when the work list was cut
// for two steps per launch)
template <typename S>
__global__ void __launch_bounds__(256) batch_step_d2q9(const BatchInst* __restrict__ insts,
                                                       const BatchItem* __restrict__ items,
                                                       int n_items, int cur, int segw) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<kD2Q9>;
  using F = Frame<kD2Q9>;
  constexpr int K = 3;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  pdl_wait();  // the previous step's writes are visible from here on
  pdl_launch_next();

  for (int it = warp; it < n_items; it += nwarps) {
    const BatchItem item = items[it];
    const BatchInst& I = insts[item.inst];
    const S* in = static_cast<const S*>(I.buf[cur]);
    S* out = const_cast<S*>(static_cast<const S*>(I.buf[cur ^ 1]));
    // the descriptor's fields, read once per work item
    const int d_nx = I.nx, d_ny = I.ny, d_px = I.px, d_py = I.py, d_wall = I.wall_mode;
    const uint8_t* const d_mask = I.mask;
    const int nq = d_nx >> 2;
    const int n_int = min(segw, nq - segw * item.seg);
    int t = segw * item.seg - 1 + lane;            // quad of this lane
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
    const bool x_lo_wall = d_wall == kWallBox && !d_px && t == 0 && interior;
    const bool x_hi_wall = d_wall == kWallBox && !d_px && t == nq - 1 && interior;
    C wk[K] = {C(0), C(0), C(0)};  // x-wall lanes: the wall node's fields in the row stored next

    auto row_exists = [&](int y) { return (y >= 0 && y < d_ny) || d_py; };
    auto row_mem = [&](int y) { return y < 0 ? y + d_ny : (y >= d_ny ? y - d_ny : y); };
    auto load = [&](int y, P (&st)[K][2]) {
      const bool ok = active && row_exists(y);
      const int64_t off = (int64_t)row_mem(y) * d_nx + 4 * t;
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
      if (!d_py && (y == 0 || y == d_ny - 1)) return;
      const int64_t off = (int64_t)y * d_nx + 4 * t;
      batch_store<S>(out, n, off, d_mask, d_wall, x_lo_wall, x_hi_wall, wk, acc, force);
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
    // source row y: sums A, B, N of destination rows y - 1, y, y + 1; then row
    // y - 1 is complete
    auto row = [&](int y, P(&A)[2][K], P(&B)[2][K], P(&N)[2][K]) {
#pragma unroll
      for (int f = 0; f < K; ++f) {
        st[f][0] = nxt[f][0];
        st[f][1] = nxt[f][1];
      }
      load(y + 1, nxt);
      batch_row_update<C, kMid>(st, A, B, N);
      if (y - 1 >= y0) store(y - 1, A);
#pragma unroll
      for (int f = 0; f < K; ++f) wk[f] = x_lo_wall ? st[f][0].x : st[f][1].y;  // row y, stored next
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < K; ++k) A[q][k] = O::splat(C(0));
    };
    // source row y1 (beyond the chunk): its contributions to row y1 - 1 (= B)
    auto last = [&](P(&B)[2][K]) {
      if (row_exists(y1)) {
#pragma unroll
        for (int f = 0; f < K; ++f) {
          st[f][0] = nxt[f][0];
          st[f][1] = nxt[f][1];
        }
        batch_row_update<C, kLast>(st, B, R0, R0);
      }
      store(y1 - 1, B);
    };
    // the three row sums rotate with period 3
    for (int y = y0;;) {
      if (y >= y1) { last(R0); break; }
      row(y++, R0, R1, R2);
      if (y >= y1) { last(R1); break; }
      row(y++, R1, R2, R0);
      if (y >= y1) { last(R2); break; }
      row(y++, R2, R0, R1);
    }
  }
}

// ------------------------------------------------------------------ two steps per launch
//
// Temporal blocking of depth 2: the warp's work item covers 28 quads of its row
// segment with two halo quads on each side (lanes 0-1 and 30-31) and marches
// the rows y0 - 2 .. y1 + 1 of the input.  A first update turns each input row
// into the intermediate state of rows y0 - 1 .. y1 (kept in registers, never
// stored); a second update, fed row by row as they complete, gives the state
// two steps on for rows y0 .. y1 - 1.  Every value of the intermediate state
// the second update reads is what a single step would have stored (its
// dependence reaches one quad and one row per step), walls keep their input
// values and rows beyond a closed y boundary are zero, and both updates sum in
// the order of batch_step_d2q9: the results are bit-identical to two launches
// of it.  FP32 and FP64 storage (16-bit storage would round the intermediate
// state on its way through memory).

constexpr int kSegW2 = kBatchSegW2;  // output quads per warp at depth 2

// Per-warp ring of kRowRing staged input rows in shared memory: each lane's
// quad of every field, copied with cp.async kRowRing rows ahead of its use.  A
// lane reads back only what it copied itself, so the ring needs no barrier.
constexpr int kRowRing = 4;
template <typename S, int K>
struct RowRing {
  static constexpr int QW = Quad<S>::BYTES;
  static constexpr size_t warp_bytes = (size_t)kRowRing * K * 32 * QW;
  unsigned char* base;  // this lane's quad of slot 0, field 0
  uint32_t sh;          // its shared-space address
  __device__ __forceinline__ RowRing(unsigned char* smem, int warp_in_block, int lane) {
    base = smem + (size_t)warp_in_block * warp_bytes + (size_t)lane * QW;
    sh = (uint32_t)__cvta_generic_to_shared(base);
  }
  __device__ __forceinline__ uint32_t slot_sh(int slot, int f) const {
    return sh + (uint32_t)((slot * K + f) * 32 * QW);
  }
  __device__ __forceinline__ const S* slot_ptr(int slot, int f) const {
    return reinterpret_cast<const S*>(base + (size_t)(slot * K + f) * 32 * QW);
  }
};

// Intermediate state of one row from its sums (the arithmetic of the store of
// batch_step_d2q9), with wall lanes (bits a.x, a.y, b.x, b.y) keeping the
// row's input state `in`; zero for a row that does not exist.
template <typename C>
__device__ __forceinline__ void batch_emit(const typename Pair<C>::P (&acc)[2][3],
                                           const typename Pair<C>::P (&in)[3][2], uint32_t wall,
                                           bool exists, const typename Pair<C>::P (&force)[2],
                                           typename Pair<C>::P (&out)[3][2]) {
  using O = Pair<C>;
  using P = typename O::P;
  if (!exists) {
#pragma unroll
    for (int f = 0; f < 3; ++f) out[f][0] = out[f][1] = O::splat(C(0));
    return;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const P inv = O::rcp(O::add(O::splat(C(36)), acc[q][0]));
    out[0][q] = O::mul(acc[q][0], O::splat(C(1.0 / 36.0)));
    out[1][q] = O::fma(acc[q][1], inv, force[0]);
    out[2][q] = O::fma(acc[q][2], inv, force[1]);
  }
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    if (wall & 1u) out[f][0].x = in[f][0].x;
    if (wall & 2u) out[f][0].y = in[f][0].y;
    if (wall & 4u) out[f][1].x = in[f][1].x;
    if (wall & 8u) out[f][1].y = in[f][1].y;
  }
}

template <typename P>
__device__ __forceinline__ void zero_sums(P (&a)[2][3]) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) a[q][k] = P{0, 0};
}

// Two updates of every work item, reading buffer cur and writing cur ^ 1:
// the work of one launch of batch_step2_d2q9 (and of one sweep of the
// persistent kernel below).
template <typename S>
__device__ __forceinline__ void batch2_sweep(const BatchInst* __restrict__ insts,
                                             const BatchItem* __restrict__ items, int n_items, int cur,
                                             const RowRing<S, 3>& ring, int lane, int warp, int nwarps) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int K = 3;
  for (int it = warp; it < n_items; it += nwarps) {
    const BatchItem item = items[it];
    const BatchInst& I = insts[item.inst];
    const S* in = static_cast<const S*>(I.buf[cur]);
    S* out = const_cast<S*>(static_cast<const S*>(I.buf[cur ^ 1]));
    // the descriptor's fields, read once per work item
    const int d_nx = I.nx, d_ny = I.ny, d_px = I.px, d_py = I.py, d_wall = I.wall_mode;
    const uint8_t* const d_mask = I.mask;
    const int nq = d_nx >> 2;                        // >= 2 (checked by the host)
    const int n_int = min(kSegW2, nq - kSegW2 * item.seg);
    int t = kSegW2 * item.seg - 2 + lane;            // quad of this lane
    const bool interior = lane >= 2 && lane <= n_int + 1;
    const bool active = lane <= n_int + 3;           // interior or halo
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
    // box walls at x = 0 and x = nx - 1 in lane order (a wrapped quad is lane-swapped)
    uint32_t xwall = 0;
    if (d_wall == kWallBox && !d_px) {
      if (t == 0) xwall |= swapped ? 2u : 1u;
      if (t == nq - 1) xwall |= swapped ? 4u : 8u;
    }
    const bool x_lo_wall = d_wall == kWallBox && !d_px && t == 0 && interior;
    const bool x_hi_wall = d_wall == kWallBox && !d_px && t == nq - 1 && interior;
    // x-wall lanes: the wall node's fields in the final row stored next (walls
    // keep their values, so the intermediate row's are the input's)
    C wk[K] = {C(0), C(0), C(0)};

    auto row_exists = [&](int y) { return (y >= 0 && y < d_ny) || d_py; };
    auto row_mem = [&](int y) { return y < 0 ? y + d_ny : (y >= d_ny ? y - d_ny : y); };
    // input rows y0 - 2 .. y1 + 1 (index i = y - y0 + 2) through the ring:
    // issue(i) starts copying row i, load(y) waits for row y and reads it
    // (zeros where absent) with the wall lanes of this quad in it
    const int y0 = item.y0, y1 = item.y1;
    const int nr = y1 - y0 + 4;
    auto issue = [&](int i) {
      const int y = y0 - 2 + i;
      if (i < nr && active && row_exists(y)) {
        const int64_t off = (int64_t)row_mem(y) * d_nx + 4 * t;
#pragma unroll
        for (int f = 0; f < K; ++f) Quad<S>::copy(ring.slot_sh(i % kRowRing, f), in + f * n + off);
      }
      cp_async_commit();
    };
    auto load = [&](int y, P (&st)[K][2], uint32_t& wall) {
      const int i = y - y0 + 2;
      cp_async_wait<kRowRing - 1>();
      const bool ok = active && row_exists(y);
      const int ym = row_mem(y);
      const int64_t off = (int64_t)ym * d_nx + 4 * t;
      wall = 0;
#pragma unroll
      for (int f = 0; f < K; ++f) {
        if (ok) {
          Quad<S>::lds(ring.slot_ptr(i % kRowRing, f), st[f][0], st[f][1]);
          if (swapped) {
            st[f][0] = O::swap(st[f][0]);
            st[f][1] = O::swap(st[f][1]);
          }
        } else {
          st[f][0] = O::splat(C(0));
          st[f][1] = O::splat(C(0));
        }
      }
      if (ok) {
        if (d_wall == kWallMask) {
          const uchar4 m = *reinterpret_cast<const uchar4*>(d_mask + off);
          wall = swapped ? ((m.y ? 1u : 0u) | (m.x ? 2u : 0u) | (m.w ? 4u : 0u) | (m.z ? 8u : 0u))
                         : ((m.x ? 1u : 0u) | (m.y ? 2u : 0u) | (m.z ? 4u : 0u) | (m.w ? 8u : 0u));
        } else if (d_wall == kWallBox) {
          wall = (!d_py && (ym == 0 || ym == d_ny - 1)) ? 15u : xwall;
        }
      }
    };
    // final rows: the store of batch_step_d2q9
    auto store = [&](int y, P (&acc)[2][K]) {
      if (!interior) return;
      if (!d_py && (y == 0 || y == d_ny - 1)) return;
      const int64_t off = (int64_t)y * d_nx + 4 * t;
      batch_store<S>(out, n, off, d_mask, d_wall, x_lo_wall, x_hi_wall, wk, acc, force);
    };

    // sums of the first update for row d in A[(d - y0 + 3) % 3], of the second in B[...]
    P A0[2][K], A1[2][K], A2[2][K], B0[2][K], B1[2][K], B2[2][K];
    zero_sums(A0); zero_sums(A1); zero_sums(A2);
    zero_sums(B0); zero_sums(B1); zero_sums(B2);
    P st[K][2], prev[K][2], mid[K][2];
    uint32_t w_st = 0, w_prev = 0;
    auto advance = [&](int y) {  // st <- input row y; start copying row y + kRowRing
      load(y, st, w_st);
      issue(y - y0 + 2 + kRowRing);
    };
    auto keep_wall = [&]() {  // wk <- intermediate row just emitted, the final row stored next
#pragma unroll
      for (int f = 0; f < K; ++f) wk[f] = x_lo_wall ? mid[f][0].x : mid[f][1].y;
    };
    auto keep = [&]() {  // prev <- st: the input of the row the next emission completes
#pragma unroll
      for (int f = 0; f < K; ++f) {
        prev[f][0] = st[f][0];
        prev[f][1] = st[f][1];
      }
      w_prev = w_st;
    };

    // input row y0 - 2: only its sums into row y0 - 1
#pragma unroll
    for (int i = 0; i < kRowRing; ++i) issue(i);
    advance(y0 - 2);
    if (row_exists(y0 - 2)) batch_row_update<C, kFirst>(st, A0, A1, A2);
    // input row y0 - 1 (row y0 - 2 of the first update is not needed)
    advance(y0 - 1);
    batch_row_update<C, kMid>(st, A1, A2, A0);
    zero_sums(A1);
    keep();
    // input row y0 completes intermediate row y0 - 1, the second update's first source
    advance(y0);
    batch_row_update<C, kMid>(st, A2, A0, A1);
    batch_emit<C>(A2, prev, w_prev, row_exists(y0 - 1), force, mid);
    zero_sums(A2);
    keep();
    keep_wall();
    if (row_exists(y0 - 1)) batch_row_update<C, kFirst>(mid, B1, B2, B0);

    // input row ys: intermediate row ys - 1 complete, fed to the second update,
    // which completes final row ys - 2.  Ap/Ac/An: first-update sums of rows
    // ys - 1, ys, ys + 1; Bp/Bc/Bn: second-update sums of rows ys - 2, ys - 1, ys.
    auto body = [&](int ys, P(&Ap)[2][K], P(&Ac)[2][K], P(&An)[2][K], P(&Bp)[2][K], P(&Bc)[2][K],
                    P(&Bn)[2][K]) {
      advance(ys);
      batch_row_update<C, kMid>(st, Ap, Ac, An);
      batch_emit<C>(Ap, prev, w_prev, row_exists(ys - 1), force, mid);
      zero_sums(Ap);
      keep();
      batch_row_update<C, kMid>(mid, Bp, Bc, Bn);
      if (ys - 2 >= y0) store(ys - 2, Bp);
      keep_wall();
      zero_sums(Bp);
    };
    // input row y1 + 1: completes intermediate row y1 and final row y1 - 1
    auto last = [&](P(&Ap)[2][K], P(&Ac)[2][K], P(&An)[2][K], P(&Bp)[2][K], P(&Bc)[2][K],
                    P(&Bn)[2][K]) {
      if (row_exists(y1 + 1)) {
        advance(y1 + 1);
        batch_row_update<C, kLast>(st, Ap, Ac, An);
      }
      batch_emit<C>(Ap, prev, w_prev, row_exists(y1), force, mid);
      if (row_exists(y1)) batch_row_update<C, kLast>(mid, Bp, Bc, Bn);
      store(y1 - 1, Bp);
    };
    // the sums rotate with period 3
    for (int ys = y0 + 1;;) {
      if (ys > y1) { last(A0, A1, A2, B2, B0, B1); break; }
      body(ys++, A0, A1, A2, B2, B0, B1);
      if (ys > y1) { last(A1, A2, A0, B0, B1, B2); break; }
      body(ys++, A1, A2, A0, B0, B1, B2);
      if (ys > y1) { last(A2, A0, A1, B1, B2, B0); break; }
      body(ys++, A2, A0, A1, B1, B2, B0);
    }
  }
}

// FP32: three blocks per SM; FP64 needs more registers (two blocks)
template <typename S>
__global__ void __launch_bounds__(128, sizeof(S) == 8 ? 2 : 3) batch_step2_d2q9(const BatchInst* __restrict__ insts,
                                                           const BatchItem* __restrict__ items,
                                                           int n_items, int cur) {
  extern __shared__ __align__(16) unsigned char batch_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const RowRing<S, 3> ring(batch_smem, threadIdx.x >> 5, lane);
  pdl_wait();  // the previous step's writes are visible from here on
  pdl_launch_next();
  batch2_sweep<S>(insts, items, n_items, cur, ring, lane, warp, nwarps);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Persistent form for small domains: `sweeps` launches' worth of
// batch_step2_d2q9 (2 sweeps steps) in one cooperative launch, the buffers
// alternating.  Between sweeps a block waits only for the blocks that own rows
// within two of its own (deps[deps[b] .. deps[b + 1]), block b's list): after
// sweep k it sets done[b] = k + 1 and starts sweep k + 1 once those blocks'
// counters reach k + 1.  Their new rows are then written (its input) and their
// reads of its rows ended (its output overwrites them).  All blocks are
// resident, so every wait ends; each is bounded all the same (wait_limit polls),
// and one that runs out sets bit 1 of *status and ends the block's sweeps (its
// neighbours' waits then run out in turn).  The state is read through the row ring only
// (cp.async.cg, from L2), so a block never sees another block's stale values.
template <typename S>
__global__ void __launch_bounds__(128, sizeof(S) == 8 ? 2 : 3)
    batch_step2_persist(const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items, int n_items,
                        int cur, int sweeps, const int* __restrict__ deps, unsigned* __restrict__ done,
                        unsigned* __restrict__ status, unsigned wait_limit) {
  extern __shared__ __align__(16) unsigned char batch_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const RowRing<S, 3> ring(batch_smem, threadIdx.x >> 5, lane);
  const int d0 = deps[blockIdx.x], d1 = deps[blockIdx.x + 1];
  for (int k = 0; k < sweeps; ++k) {
    batch2_sweep<S>(insts, items, n_items, cur ^ (k & 1), ring, lane, warp, nwarps);
    if (k + 1 == sweeps) break;
    cp_async_wait<0>();  // no row copy of this sweep lands after the next one starts
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this block's stores are visible before its counter
      st_release_gpu(&done[blockIdx.x], (unsigned)(k + 1));
    }
    int ok = 1;
    for (int j = d0 + (int)threadIdx.x; ok && j < d1; j += blockDim.x) {
      const unsigned* f = &done[deps[j]];
      ok = 0;
      for (uint32_t it = 0; it < wait_limit; ++it) {
        if (ld_acquire_gpu(f) >= (unsigned)(k + 1)) {
          ok = 1;
          break;
        }
      }
    }
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0 && status) atomicOr(status, 2u);
      break;
    }
  }
}

template <typename S>
static cudaError_t launch_batch2_t(const BatchInst* insts, const BatchItem* items, int n_items,
                                   int cur, int blocks, cudaStream_t st, int overlap) {
  constexpr size_t smem = 4 * RowRing<S, 3>::warp_bytes;  // 4 warps
  return launch_kernel(batch_step2_d2q9<S>, dim3(blocks), dim3(128), smem, st, overlap, insts, items,
                       n_items, cur);
}

template <typename S>
static cudaError_t launch_batch_t(const BatchInst* insts, const BatchItem* items, int n_items,
                                  int cur, int blocks, int segw, cudaStream_t st, int overlap) {
  return launch_kernel(batch_step_d2q9<S>, dim3(blocks), dim3(256), 0, st, overlap, insts, items, n_items,
                       cur, segw);
}

cudaError_t launch_batch_step(int precision, const void* insts, const void* items, int n_items,
                              int cur, int blocks, int segw, cudaStream_t st, int overlap) {
  const BatchInst* I = static_cast<const BatchInst*>(insts);
  const BatchItem* T = static_cast<const BatchItem*>(items);
  if (segw < 1 || segw > 30) return cudaErrorInvalidValue;
  switch (precision) {
    case MACLAB_F64: return launch_batch_t<double>(I, T, n_items, cur, blocks, segw, st, overlap);
    case MACLAB_F32: return launch_batch_t<float>(I, T, n_items, cur, blocks, segw, st, overlap);
    case MACLAB_BF16_STORE: return launch_batch_t<__nv_bfloat16>(I, T, n_items, cur, blocks, segw, st, overlap);
    case MACLAB_F16_STORE: return launch_batch_t<__half>(I, T, n_items, cur, blocks, segw, st, overlap);
  }
  return cudaErrorInvalidValue;
}

// Two steps per launch: FP32 and FP64 storage only.
cudaError_t launch_batch_step2(int precision, const void* insts, const void* items, int n_items,
                               int cur, int blocks, cudaStream_t st, int overlap) {
  const BatchInst* I = static_cast<const BatchInst*>(insts);
  const BatchItem* T = static_cast<const BatchItem*>(items);
  switch (precision) {
    case MACLAB_F64: return launch_batch2_t<double>(I, T, n_items, cur, blocks, st, overlap);
    case MACLAB_F32: return launch_batch2_t<float>(I, T, n_items, cur, blocks, st, overlap);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
static cudaError_t persist_setup(int* capacity) {
  constexpr size_t smem = 4 * RowRing<S, 3>::warp_bytes;  // 4 warps
  auto kern = batch_step2_persist<S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  *capacity = per_sm * sms;
  return cudaSuccess;
}

// Blocks of the persistent launch that can be resident at once (its limit).
cudaError_t batch_persist_capacity(int precision, int* capacity) {
  *capacity = 0;
  switch (precision) {
    case MACLAB_F64: return persist_setup<double>(capacity);
    case MACLAB_F32: return persist_setup<float>(capacity);
  }
  return cudaErrorInvalidValue;
}

template <typename S>
static cudaError_t launch_batch2_persist_t(const BatchInst* insts, const BatchItem* items, int n_items, int cur,
                                           int blocks, int sweeps, const int* deps, unsigned* done,
                                           unsigned* status, unsigned wait_limit, cudaStream_t st) {
  constexpr size_t smem = 4 * RowRing<S, 3>::warp_bytes;
  int capacity = 0;
  cudaError_t e = persist_setup<S>(&capacity);
  if (e != cudaSuccess) return e;
  // a cooperative launch: every block resident at once (the waits need it);
  // the dependency lists were built for exactly this block count
  if (blocks < 1 || blocks > capacity) return cudaErrorCooperativeLaunchTooLarge;
  if ((e = cudaMemsetAsync(done, 0, (size_t)blocks * sizeof(unsigned), st)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_step2_persist<S>, insts, items, n_items, cur, sweeps, deps, done, status,
                            wait_limit);
}

// `sweeps` two-step launches in one persistent cooperative launch (FP32 and
// FP64 storage).  deps: the lists of batch_persist_deps for `blocks` blocks;
// done: `blocks` counters (zeroed here); wait_limit: polls before a wait gives up.
cudaError_t launch_batch_step2_persist(int precision, const void* insts, const void* items, int n_items, int cur,
                                       int blocks, int sweeps, const int* deps, unsigned* done, unsigned* status,
                                       unsigned wait_limit, cudaStream_t st) {
  const BatchInst* I = static_cast<const BatchInst*>(insts);
  const BatchItem* T = static_cast<const BatchItem*>(items);
  if (sweeps < 1 || !deps || !done) return cudaErrorInvalidValue;
  switch (precision) {
    case MACLAB_F64:
      return launch_batch2_persist_t<double>(I, T, n_items, cur, blocks, sweeps, deps, done, status, wait_limit, st);
    case MACLAB_F32:
      return launch_batch2_persist_t<float>(I, T, n_items, cur, blocks, sweeps, deps, done, status, wait_limit, st);
  }
  return cudaErrorInvalidValue;
}

// The wait lists of the persistent launch: with `blocks` blocks of four warps,
// warp w takes the items w, w + 4 blocks, ...; an item (domain i, rows y0, y1)
// reads rows y0 - 2 .. y1 + 1 of domain i (wrapped where its y is periodic,
// py[i]; domain i has ny[i] rows) in every x segment and writes rows
// y0 .. y1 - 1.  Block b waits for every other block owning a row that one of
// its items reads; the relation is symmetric, so these are also the blocks
// that read b's rows.  Rows of different domains never meet.  out: blocks + 1
// offsets (relative to the array's start), then the lists.
void batch_persist_deps(const std::vector<int>& items4, const std::vector<int>& ny, const std::vector<int>& py,
                        int blocks, std::vector<int>& out) {
  const int n = (int)(items4.size() / 4), nwarps = 4 * blocks;
  std::vector<size_t> base(ny.size() + 1, 0);  // first row of domain i in `owners`
  for (size_t i = 0; i < ny.size(); ++i) base[i + 1] = base[i] + (size_t)ny[i];
  std::vector<std::vector<int>> owners(base.back());  // blocks owning a row (ascending, no repeats)
  for (int i = 0; i < n; ++i) {
    const int b = (i % nwarps) / 4, d = items4[4 * i];
    for (int y = items4[4 * i + 2]; y < items4[4 * i + 3]; ++y) {
      std::vector<int>& o = owners[base[d] + y];
      if (o.empty() || o.back() != b) o.push_back(b);
    }
  }
  std::vector<std::vector<int>> dep(blocks);
  for (int i = 0; i < n; ++i) {
    const int b = (i % nwarps) / 4, d = items4[4 * i];
    for (int y = items4[4 * i + 2] - 2; y < items4[4 * i + 3] + 2; ++y) {
      int r = y;
      if (r < 0 || r >= ny[d]) {
        if (!py[d]) continue;
        r = ((r % ny[d]) + ny[d]) % ny[d];
      }
      for (int c : owners[base[d] + r])
        if (c != b) dep[b].push_back(c);
    }
  }
  out.assign(blocks + 1, 0);
  for (int b = 0; b < blocks; ++b) {
    std::sort(dep[b].begin(), dep[b].end());
    dep[b].erase(std::unique(dep[b].begin(), dep[b].end()), dep[b].end());
    out[b] = (int)out.size();
    out.insert(out.end(), dep[b].begin(), dep[b].end());
  }
  out[blocks] = (int)out.size();
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

// Work items of one domain with `rows` rows per chunk; segments of 30 quads
// (one step per launch) or 28 (two steps per launch).
void batch_items(int inst, const Geometry& g, int rows, int depth, std::vector<int>& out4) {
  const int nq = g.nx / 4;
  const int segw = depth == 2 ? kBatchSegW2 : kBatchSegW1;
  const int nseg = (nq + segw - 1) / segw;
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
