// step_fold.cuh -- D3Q19 variant of the tiled step (step_tiled.cuh) without
// halo-row threads (Eqs. (2), (4), (5); the same terms, summed in another
// order, so results agree with step_tiled to rounding).
//
// step_tiled gives every block TY rows of y plus one halo row on each side,
// and the halo rows' threads only publish the five equilibria that cross into
// the tile, then wait at both barriers of every plane.  Here a block holds
// only its TY rows: the threads of the first and last row also load the halo
// row next to them and fold its inward equilibria directly into their own
// sums (c_x = 0 and the moves within the thread's quad), or through the x
// exchange (two extra slots) for the pair that crosses to the neighbouring
// thread.  Equilibria of the tile's own rows that leave the tile in y are
// dropped: the neighbouring tile forms them from its halo row.  Every warp
// then does the full update and a block needs two fewer warps for the same
// rows, so more blocks fit on an SM.
//
// Requires ny % TY == 0 and TY >= 2 (the first and last rows are distinct).
#pragma once
#include "step_tiled.cuh"

namespace maclab {

// A block shape: BXC quads of a row by TY rows.
struct FoldShape {
  int bxc, ty;
};

// Launch dispatch for 16-bit storage (step_fold_s16.cu): shapes (32, 8),
// (32, 4), (64, 4) and (128, 4); with resident set, only the blocks one SM holds.
cudaError_t fold_dispatch_s16(int precision, const FoldShape& s, const TiledArgs& ta, const void* in,
                              void* out, cudaStream_t st, dim3 grid, int* resident);

template <typename S, int BXC, int TY>
struct FoldLayout {
  using C = typename Store<S>::C;
  using P = typename Pair<C>::P;
  using F = Frame<kD3Q19>;
  static constexpr int W = Cols<BXC>::W;
  static constexpr int NXO = F::count_x();       // x-crossing slots of the own rows
  static constexpr int NXS = NXO + 2;            // + the halo row's (+x, -x) slots
  static constexpr int NYS = F::count_y();
  static constexpr int RS = TY + 2;              // staged rows: lower halo, TY own, upper halo
  // Rows that fit in a warp (BXC <= 32) exchange x-crossing equilibria by
  // shuffles and double-buffer the y exchange (one barrier per plane); wider
  // rows use the shared x exchange and one y buffer (two barriers).
  static constexpr bool XSH = BXC <= 32;
  static constexpr int YROW = 2 * BXC + 1;       // XSH y row: pairs a, pairs b, one seam copy
  static constexpr size_t ye_buf_pairs = (size_t)NYS * (TY - 1) * YROW;
  static constexpr size_t xe_pairs = XSH ? 0 : (size_t)NXS * TY * W;
  static constexpr size_t ye_pairs = XSH ? 2 * ye_buf_pairs : (size_t)NYS * TY * 2 * W;
  static constexpr size_t exch_bytes = ((sizeof(P) * (xe_pairs + ye_pairs) + 15) / 16) * 16;
  static constexpr size_t stage_bytes = (size_t)kStages * 4 * RS * BXC * Quad<S>::BYTES;
  // box walls at x = 0 and x = nx - 1: each row's two wall lanes keep the four
  // fields of their wall node for the last two planes taken (walls never change)
  static constexpr size_t wall_bytes = (size_t)TY * 2 * kStages * 16;
  static constexpr size_t smem = exch_bytes + stage_bytes + wall_bytes;
  static constexpr int THREADS = BXC * TY;
  static constexpr int MIN_BLOCKS = THREADS <= 128 ? 4 : (THREADS <= 256 ? 2 : 1);
};

// The halo directions: the lower halo row (source y - 1) sends c_y = +1, the
// upper one c_y = -1.  HX: index of the direction (c_x, c_y, c_z) = (FX, FY, 0).
template <int FX, int FY>
__host__ __device__ constexpr int fold_dir() {
  using F = Frame<kD3Q19>;
  for (int a = 0; a < Lattice<kD3Q19>::Q; ++a)
    if (F::fx(a) == FX && F::fy(a) == FY && F::fz(a) == 0) return a;
  return -1;
}

// Halo row (FY = +1: lower, -1: upper): its equilibria moving into the
// thread's row, folded into the sums or published in the halo x slots.
template <typename C, int MODE, int BXC, int TY, int FY>
__device__ __forceinline__ void fold_halo(const typename Pair<C>::P (&hs)[4][2],
                                          typename Pair<C>::P (&ap)[2][4], typename Pair<C>::P (&ac)[2][4],
                                          typename Pair<C>::P (&an)[2][4],
                                          const SmemBase<typename Pair<C>::P>& sb) {
  using L = Lattice<kD3Q19>;
  using F = Frame<kD3Q19>;
  using O = Pair<C>;
  using P = typename O::P;
  using Lay = FoldLayout<float, BXC, TY>;  // slot geometry only (independent of S)
  constexpr int XS = TY * Cols<BXC>::W;
  constexpr int HP = Lay::NXO, HM = Lay::NXO + 1;  // halo +x and -x slots
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Terms<3, C> t;
    const P u[3] = {hs[1][q], hs[2][q], hs[3][q]};
    make_terms<3, C>(hs[0][q], u, t);
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == FY) {
        constexpr int fx = F::fx(a), fz = F::fz(a);
        const P T = term<kD3Q19, C, a>(t);
        const int qd = q + fx;
        if (qd >= 0 && qd < 2) {
          accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[qd], T);
        } else if constexpr (fx == 1) {  // pair b -> the next thread's pair a
          sb.x_own[HP * XS] = T;
          if (sb.wl) sb.x_sl[HP * XS] = O::swap(T);
        } else if constexpr (fx == -1) { // pair a -> the previous thread's pair b
          sb.x_own[HM * XS] = T;
          if (sb.wr) sb.x_sr[HM * XS] = O::swap(T);
        }
      }
    });
  }
}

// One source plane.  st: the thread's own quad; hsrc: its staged halo quad
// (first and last row only, halo = +1 lower / -1 upper / 0 none; field f at
// hsrc + f * fstride bytes), read only where it is folded in; ap/ac/an: sums
// of the destination planes p - 1, p, p + 1.
template <typename S, typename C, int MODE, int BXC, int TY>
__device__ __forceinline__ void fold_update(const typename Pair<C>::P (&st)[4][2],
                                            const unsigned char* hsrc, uint32_t fstride, int halo,
                                            typename Pair<C>::P (&ap)[2][4], typename Pair<C>::P (&ac)[2][4],
                                            typename Pair<C>::P (&an)[2][4],
                                            const SmemBase<typename Pair<C>::P>& sb, int r, bool live) {
  using L = Lattice<kD3Q19>;
  using F = Frame<kD3Q19>;
  using O = Pair<C>;
  using P = typename O::P;
  using Lay = FoldLayout<float, BXC, TY>;
  constexpr int W = Cols<BXC>::W;
  constexpr int XS = TY * W;       // stride between x slots
  constexpr int YR = 2 * W;        // stride between rows of a y slot
  constexpr int YS = TY * YR;      // stride between y slots
  constexpr int HP = Lay::NXO, HM = Lay::NXO + 1;
  if (live) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      Terms<3, C> t;
      const P u[3] = {st[1][q], st[2][q], st[3][q]};
      make_terms<3, C>(st[0][q], u, t);
      static_for<0, L::Q>([&](auto I) {
        constexpr int a = decltype(I)::value;
        if constexpr (mode_allows<kD3Q19, MODE>(a)) {
          constexpr int fx = F::fx(a);
          if constexpr (F::ycross(a)) {
            // rows of the tile only: what leaves it is formed by the next tile's halo
            constexpr int fy = F::fy(a);
            if (fy == 1 ? r < TY - 1 : r > 0) {
              const P T = term<kD3Q19, C, a>(t);
              constexpr int off = F::yslot(a) * YS;
              sb.y_own[off + q * W] = T;
              if constexpr (fx == 1) {
                if (q == 1 && sb.wl) sb.y_sl[off + W] = O::swap(T);
              } else if constexpr (fx == -1) {
                if (q == 0 && sb.wr) sb.y_sr[off] = O::swap(T);
              }
            }
          } else {
            constexpr int fz = F::fz(a);
            const P T = term<kD3Q19, C, a>(t);
            const int qd = q + fx;
            if (qd >= 0 && qd < 2) {
              accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[qd], T);
            } else {
              constexpr int off = F::xslot(a) * XS;
              sb.x_own[off] = T;
              if constexpr (fx == 1) {
                if (sb.wl) sb.x_sl[off] = O::swap(T);
              } else {
                if (sb.wr) sb.x_sr[off] = O::swap(T);
              }
            }
          }
        }
      });
    }
    if (halo != 0) {
      P hs[4][2];
#pragma unroll
      for (int f = 0; f < 4; ++f)
        Quad<S>::lds(reinterpret_cast<const S*>(hsrc + f * fstride), hs[f][0], hs[f][1]);
      if (halo == 1) fold_halo<C, MODE, BXC, TY, 1>(hs, ap, ac, an, sb);
      else fold_halo<C, MODE, BXC, TY, -1>(hs, ap, ac, an, sb);
    }
  }
  __syncthreads();
  if (live) {
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a)) {
        constexpr int fz = F::fz(a);
        constexpr int fx = F::fx(a);
        auto& dst = pick<fz>(ap, ac, an);
        if constexpr (F::xcross(a)) {
          // +x: pair a receives the left neighbour's pair b; -x: pair b gets the right one's a
          constexpr int off = F::xslot(a) * XS;
          if constexpr (fx == 1) accum<kD3Q19, C, a>(dst[0], sb.x_l[off]);
          else accum<kD3Q19, C, a>(dst[1], sb.x_r[off]);
        } else if constexpr (F::ycross(a)) {
          constexpr int fy = F::fy(a);
          // source row r - fy: a row of the tile (the halo rows were folded in already)
          if (fy == 1 ? r > 0 : r < TY - 1) {
            constexpr int off = F::yslot(a) * YS - fy * YR;
            if constexpr (fx == 0) {
              accum<kD3Q19, C, a>(dst[0], sb.y_own[off]);
              accum<kD3Q19, C, a>(dst[1], sb.y_own[off + W]);
            } else if constexpr (fx == 1) {
              accum<kD3Q19, C, a>(dst[0], sb.y_l[off + W]);   // left neighbour's pair b
              accum<kD3Q19, C, a>(dst[1], sb.y_own[off]);     // own pair a
            } else {
              accum<kD3Q19, C, a>(dst[0], sb.y_own[off + W]); // own pair b
              accum<kD3Q19, C, a>(dst[1], sb.y_r[off]);       // right neighbour's pair a
            }
          }
        }
      }
    });
    if constexpr (MODE == kMid) {  // the halo row's x-crossing pairs
      if (halo == 1) {
        accum<kD3Q19, C, fold_dir<1, 1>()>(ac[0], sb.x_l[HP * XS]);
        accum<kD3Q19, C, fold_dir<-1, 1>()>(ac[1], sb.x_r[HM * XS]);
      } else if (halo == -1) {
        accum<kD3Q19, C, fold_dir<1, -1>()>(ac[0], sb.x_l[HP * XS]);
        accum<kD3Q19, C, fold_dir<-1, -1>()>(ac[1], sb.x_r[HM * XS]);
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ rows within a warp
// Per-thread constants of the shuffle x exchange and the compact y exchange.
template <typename P>
struct FoldXs {
  P* ye;               // y exchange buffer of the current plane
  int tx;
  int li, ri;          // y-row column of the left neighbour's pair b / right one's pair a (or the seam copy)
  int src_l, src_r;    // lanes (within the row's segment) of the left / right neighbour
  bool swap_l, swap_r; // receiving across the seam: thread 0 from the left, the last thread from the right
  bool wl, wr;         // writing the seam copy: the last thread (+x), thread 0 (-x)
};

template <int WIDTH, typename P>
__device__ __forceinline__ P fold_shfl(P v, int src) {
  P r;
  r.x = __shfl_sync(0xffffffffu, v.x, src, WIDTH);
  r.y = __shfl_sync(0xffffffffu, v.y, src, WIDTH);
  return r;
}

// index of an x-crossing direction among those with the same c_x (c_y = 0)
__host__ __device__ constexpr int fold_xidx(int a) {
  using F = Frame<kD3Q19>;
  int k = 0;
  for (int b = 0; b < a; ++b) k += (F::fy(b) == 0 && F::fx(b) == F::fx(a)) ? 1 : 0;
  return k;
}

// Halo row (FY = +1 lower, -1 upper) with the shuffle exchange: in-thread
// moves go into the sums, the pair crossing to a neighbour into hb (+x) / ha (-x).
template <typename C, int MODE, int FY>
__device__ __forceinline__ void fold_halo_xs(const typename Pair<C>::P (&hs)[4][2],
                                             typename Pair<C>::P (&ap)[2][4], typename Pair<C>::P (&ac)[2][4],
                                             typename Pair<C>::P (&an)[2][4], typename Pair<C>::P& hb,
                                             typename Pair<C>::P& ha) {
  using L = Lattice<kD3Q19>;
  using F = Frame<kD3Q19>;
  using P = typename Pair<C>::P;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    Terms<3, C> t;
    const P u[3] = {hs[1][q], hs[2][q], hs[3][q]};
    make_terms<3, C>(hs[0][q], u, t);
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == FY) {
        constexpr int fx = F::fx(a), fz = F::fz(a);
        const P T = term<kD3Q19, C, a>(t);
        const int qd = q + fx;
        if (qd >= 0 && qd < 2) accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[qd], T);
        else if constexpr (fx == 1) hb = T;
        else if constexpr (fx == -1) ha = T;
      }
    });
  }
}

// One source plane, rows within a warp.  Every lane runs the first phase and
// the shuffles (lanes past the row end hold zeros and are never read); the y
// exchange goes through this plane's buffer, and the one barrier suffices
// because consecutive planes use different buffers.
template <typename S, typename C, int MODE, int BXC, int TY>
__device__ __forceinline__ void fold_update_xs(const typename Pair<C>::P (&st)[4][2],
                                               const unsigned char* hsrc, uint32_t fstride, int halo,
                                               typename Pair<C>::P (&ap)[2][4], typename Pair<C>::P (&ac)[2][4],
                                               typename Pair<C>::P (&an)[2][4], const FoldXs<typename Pair<C>::P>& xs,
                                               int r, bool live) {
  using L = Lattice<kD3Q19>;
  using F = Frame<kD3Q19>;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int YROW = 2 * BXC + 1;
  constexpr int SEAM = 2 * BXC;
  P xb[3], xa[3];  // x-crossing equilibria leaving pair b (+x) and pair a (-x)
#pragma unroll
  for (int k = 0; k < 3; ++k) xb[k] = xa[k] = O::splat(C(0));
  // y rows of this plane's buffer: row r carries the c_y = +1 equilibria of
  // source row r (read by row r + 1), row r - 1 the c_y = -1 ones (read by r - 1)
  P* const y_up = xs.ye + r * YROW;
  P* const y_dn = y_up - YROW;
  // equilibria of pair q with c_y = FY into the y rows (rows of the tile only:
  // what leaves it is formed by the next tile's halo)
  auto publish_y = [&](auto fyc, const Terms<3, C>& t, auto qc) {
    constexpr int FY = decltype(fyc)::value;
    constexpr int q = decltype(qc)::value;
    P* const base = FY == 1 ? y_up : y_dn;
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == FY) {
        constexpr int fx = F::fx(a);
        const P T = term<kD3Q19, C, a>(t);
        P* const row = base + F::yslot(a) * (TY - 1) * YROW;
        row[q * BXC + xs.tx] = T;
        if constexpr (fx == 1 && q == 1) {
          if (xs.wl) row[SEAM] = O::swap(T);
        } else if constexpr (fx == -1 && q == 0) {
          if (xs.wr) row[SEAM] = O::swap(T);
        }
      }
    });
  };
  static_for<0, 2>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    Terms<3, C> t;
    const P u[3] = {st[1][q], st[2][q], st[3][q]};
    make_terms<3, C>(st[0][q], u, t);
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a) && !F::ycross(a)) {
        constexpr int fx = F::fx(a), fz = F::fz(a);
        const P T = term<kD3Q19, C, a>(t);
        constexpr int qd = q + fx;
        if constexpr (qd >= 0 && qd < 2) accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[qd], T);
        else if constexpr (fx == 1) xb[fold_xidx(a)] = T;
        else if constexpr (fx == -1) xa[fold_xidx(a)] = T;
      }
    });
    if (r < TY - 1) publish_y(std::integral_constant<int, 1>{}, t, qc);
    if (r > 0) publish_y(std::integral_constant<int, -1>{}, t, qc);
  });
  P hb = O::splat(C(0)), ha = O::splat(C(0));
  if (live && halo != 0) {
    P hs[4][2];
#pragma unroll
    for (int f = 0; f < 4; ++f) Quad<S>::lds(reinterpret_cast<const S*>(hsrc + f * fstride), hs[f][0], hs[f][1]);
    if (halo == 1) fold_halo_xs<C, MODE, 1>(hs, ap, ac, an, hb, ha);
    else fold_halo_xs<C, MODE, -1>(hs, ap, ac, an, hb, ha);
  }
  // x exchange: +x from the left neighbour's pair b into pair a, -x from the
  // right neighbour's pair a into pair b (lane-swapped across the seam)
  static_for<0, L::Q>([&](auto I) {
    constexpr int a = decltype(I)::value;
    if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == 0 && F::fx(a) != 0) {
      constexpr int fx = F::fx(a), fz = F::fz(a);
      if constexpr (fx == 1) {
        P v = fold_shfl<BXC>(xb[fold_xidx(a)], xs.src_l);
        if (xs.swap_l) v = O::swap(v);
        accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[0], v);
      } else {
        P v = fold_shfl<BXC>(xa[fold_xidx(a)], xs.src_r);
        if (xs.swap_r) v = O::swap(v);
        accum<kD3Q19, C, a>(pick<fz>(ap, ac, an)[1], v);
      }
    }
  });
  if constexpr (MODE == kMid) {  // the halo row's crossing pairs (c_z = 0 only)
    P v = fold_shfl<BXC>(hb, xs.src_l);
    P w = fold_shfl<BXC>(ha, xs.src_r);
    if (xs.swap_l) v = O::swap(v);
    if (xs.swap_r) w = O::swap(w);
    if (halo == 1) {
      accum<kD3Q19, C, fold_dir<1, 1>()>(ac[0], v);
      accum<kD3Q19, C, fold_dir<-1, 1>()>(ac[1], w);
    } else if (halo == -1) {
      accum<kD3Q19, C, fold_dir<1, -1>()>(ac[0], v);
      accum<kD3Q19, C, fold_dir<-1, -1>()>(ac[1], w);
    }
  }
  __syncthreads();
  // gather the equilibria with c_y = FY from source row r - FY, a row of the
  // tile (the halo rows were folded in already)
  auto gather_y = [&](auto fyc) {
    constexpr int FY = decltype(fyc)::value;
    const P* const base = FY == 1 ? y_dn : y_up;
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == FY) {
        constexpr int fz = F::fz(a), fx = F::fx(a);
        auto& dst = pick<fz>(ap, ac, an);
        const P* const row = base + F::yslot(a) * (TY - 1) * YROW;
        if constexpr (fx == 0) {
          accum<kD3Q19, C, a>(dst[0], row[xs.tx]);
          accum<kD3Q19, C, a>(dst[1], row[BXC + xs.tx]);
        } else if constexpr (fx == 1) {
          accum<kD3Q19, C, a>(dst[0], row[xs.li]);          // left neighbour's pair b
          accum<kD3Q19, C, a>(dst[1], row[xs.tx]);          // own pair a
        } else {
          accum<kD3Q19, C, a>(dst[0], row[BXC + xs.tx]);    // own pair b
          accum<kD3Q19, C, a>(dst[1], row[xs.ri]);          // right neighbour's pair a
        }
      }
    });
  };
  if (live) {
    if (r > 0) gather_y(std::integral_constant<int, 1>{});
    if (r < TY - 1) gather_y(std::integral_constant<int, -1>{});
  }
}

// Store of one destination plane (Eq. (5): u' = M / (36 + R) + F) for box
// walls, every lane with the same instructions: the lane whose quad holds one
// x-wall node (a.x at x = 0, b.y at x = nx - 1) puts that node's unchanged
// value, wv (its four fields, kept when the plane was taken), in place of the
// computed one and stores the whole quad.  Masks, and a quad holding both
// x-walls (nx = 4), take store_plane's per-node path.
template <typename S>
__device__ __forceinline__ void fold_store(S* const (&fp)[4], const uint8_t* mrow, const TiledArgs& ta,
                                           int64_t off, bool x_lo_wall, bool x_hi_wall, const float4& wv,
                                           bool skip, typename Quad<S>::P (&acc)[2][4],
                                           const typename Quad<S>::P (&force)[3]) {
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  if (ta.wall_mode == kWallMask || (x_lo_wall && x_hi_wall)) {
    store_plane<kD3Q19, S>(fp, mrow, ta, off, x_lo_wall, x_hi_wall, skip, acc, force);
    return;
  }
  if (skip) return;
  P v[4][2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const P inv = O::rcp(O::add(O::splat(C(36)), acc[q][0]));
    v[0][q] = O::mul(acc[q][0], O::splat(C(1.0 / 36.0)));
#pragma unroll
    for (int i = 0; i < 3; ++i) v[1 + i][q] = O::fma(acc[q][1 + i], inv, force[i]);
  }
  const float w[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (x_lo_wall) v[f][0].x = C(w[f]);
    if (x_hi_wall) v[f][1].y = C(w[f]);
    Quad<S>::st(fp[f] + off, v[f][0], v[f][1]);
  }
}

template <typename S, int BXC, int TY>
__global__ void __launch_bounds__(BXC * TY, FoldLayout<S, BXC, TY>::MIN_BLOCKS)
    step_fold(TiledArgs ta, const S* __restrict__ in, S* __restrict__ out) {
  using Lay = FoldLayout<S, BXC, TY>;
  using C = typename Store<S>::C;
  using O = Pair<C>;
  using P = typename O::P;
  constexpr int K = 4;
  constexpr int W = Cols<BXC>::W;
  constexpr int RS = Lay::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pdl_wait();  // the previous step's writes are visible from here on
  pdl_launch_next();
  const int tx = threadIdx.x, r = threadIdx.y;
  const int bxr = ta.nx >> 2;  // threads per row actually used
  const bool active = tx < bxr;
  P* Xe = reinterpret_cast<P*>(smem_raw);
  P* Ye = Xe + Lay::xe_pairs;
  const int col_l = tx == 0 ? Cols<BXC>::SEAM_L : tx - 1;
  const int col_r = tx == bxr - 1 ? Cols<BXC>::SEAM_R : tx + 1;
  SmemBase<P> sb;
  sb.wl = tx == bxr - 1;
  sb.wr = tx == 0;
  sb.x_own = Xe + r * W + tx;
  sb.x_l = Xe + r * W + col_l;
  sb.x_r = Xe + r * W + col_r;
  sb.x_sl = Xe + r * W + Cols<BXC>::SEAM_L;
  sb.x_sr = Xe + r * W + Cols<BXC>::SEAM_R;
  sb.y_own = Ye + r * 2 * W + tx;
  sb.y_l = Ye + r * 2 * W + col_l;
  sb.y_r = Ye + r * 2 * W + col_r;
  sb.y_sl = Ye + r * 2 * W + Cols<BXC>::SEAM_L;
  sb.y_sr = Ye + r * 2 * W + Cols<BXC>::SEAM_R;
  FoldXs<P> xs;  // rows within a warp: shuffle x exchange, alternating y buffers
  xs.ye = Ye;
  xs.tx = tx;
  xs.li = tx == 0 ? 2 * BXC : BXC + tx - 1;
  xs.ri = tx == bxr - 1 ? 2 * BXC : tx + 1;
  xs.src_l = tx == 0 ? bxr - 1 : tx - 1;
  xs.src_r = tx == bxr - 1 ? 0 : tx + 1;
  xs.swap_l = tx == 0;
  xs.swap_r = tx == bxr - 1;
  xs.wl = tx == bxr - 1;
  xs.wr = tx == 0;
  int ybuf = 0;

  // own row (every row of the tile exists: ny % TY == 0) and the halo row of
  // the first (+1: row - 1) and last (-1: row + 1) rows
  const int row = blockIdx.y * TY + r;
  int halo = r == 0 ? 1 : (r == TY - 1 ? -1 : 0);
  int hrow = row - halo;
  if (halo != 0 && (hrow < 0 || hrow >= ta.ny)) {
    if (ta.py) hrow = (hrow + ta.ny) % ta.ny;
    else halo = 0;  // no row beyond a closed y boundary: nothing to fold in
  }
  const bool row_wall = !ta.py && (row == 0 || row == ta.ny - 1);
  const int64_t row_off = (int64_t)row * ta.nx + 4 * tx;
  const int64_t halo_delta = (int64_t)(hrow - row) * ta.nx;  // halo quad - own quad
  // box walls at x = 0 (lane a.x of thread 0) and x = nx - 1 (lane b.y of the last)
  const bool x_lo_wall = ta.wall_mode == kWallBox && !ta.px && tx == 0;
  const bool x_hi_wall = ta.wall_mode == kWallBox && !ta.px && tx == bxr - 1;

  const S* ip[4];
  S* op[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    ip[f] = in + (int64_t)f * ta.n + row_off;
    op[f] = out + (int64_t)f * ta.n + row_off;
  }
  const uint8_t* mrow = ta.wall_mode == kWallMask ? ta.mask + row_off : nullptr;
  P force[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) force[i] = O::splat(C(ta.force[i]));

  // chunk c of nzc covers planes [c * nplanes / nzc, (c + 1) * nplanes / nzc)
  const int z0 = (int)(((int64_t)blockIdx.x * ta.nplanes) / ta.nzc);
  const int z1 = (int)(((int64_t)(blockIdx.x + 1) * ta.nplanes) / ta.nzc);
  const int64_t ps = ta.plane_stride;
  auto plane_exists = [&](int p) { return (p >= 0 && p < ta.nplanes) || ta.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + ta.nplanes : (p >= ta.nplanes ? p - ta.nplanes : p); };
  auto store_skip = [&](int q) {
    return !active || row_wall || (!ta.pz && (q == 0 || q == ta.nplanes - 1));
  };

  // stage buffers [kStages][K][RS][BXC] quads: own quad at staged row r + 1,
  // the halo quad at row 0 (lower) or TY + 1 (upper)
  constexpr int QW = Quad<S>::BYTES;
  constexpr uint32_t kFieldStride = RS * BXC * QW;
  constexpr uint32_t kSlotStride = K * kFieldStride;
  unsigned char* stage0 = smem_raw + Lay::exch_bytes + (size_t)tx * QW;
  const uint32_t own_off = (uint32_t)(r + 1) * BXC * QW;
  const uint32_t halo_off = (uint32_t)(halo == 1 ? 0 : TY + 1) * BXC * QW;
  const uint32_t stage_sh = (uint32_t)__cvta_generic_to_shared(stage0);
  // this lane's wall ring (lanes with exactly one x-wall node only)
  const bool xwall1 = x_lo_wall != x_hi_wall;
  float4* const wring = reinterpret_cast<float4*>(smem_raw + Lay::exch_bytes + Lay::stage_bytes) +
                        (r * 2 + (x_hi_wall ? 1 : 0)) * kStages;
  const int np = z1 - z0 + 2;  // planes z0 - 1 .. z1
  auto fetch = [&](int i) {    // start copying plane z0 - 1 + i into its stage
    const int p = z0 - 1 + i;
    if (i < np && active && plane_exists(p)) {
      const int64_t off = (int64_t)plane_mem(p) * ps;
      const uint32_t sh = stage_sh + (uint32_t)(i & (kStages - 1)) * kSlotStride;
#pragma unroll
      for (int f = 0; f < K; ++f) Quad<S>::copy(sh + f * kFieldStride + own_off, ip[f] + off);
      if (halo != 0)
#pragma unroll
        for (int f = 0; f < K; ++f) Quad<S>::copy(sh + f * kFieldStride + halo_off, ip[f] + off + halo_delta);
    }
    cp_async_commit();
  };
  P st[K][2];
  const unsigned char* hsrc = stage0 + halo_off;  // the halo quad of the plane taken last
  auto take = [&](int i) {     // wait for plane z0 - 1 + i and read the own quad
    cp_async_wait<kStages - 1>();
    const int p = z0 - 1 + i;
    const bool ok = active && plane_exists(p);
    const unsigned char* base = stage0 + (size_t)(i & (kStages - 1)) * kSlotStride;
    hsrc = base + halo_off;
#pragma unroll
    for (int f = 0; f < K; ++f) {
      if (ok) {
        Quad<S>::lds(reinterpret_cast<const S*>(base + f * kFieldStride + own_off), st[f][0], st[f][1]);
      } else {
        st[f][0] = st[f][1] = O::splat(C(0));
      }
    }
    if (xwall1 && ok)
      wring[i & (kStages - 1)] = x_lo_wall ? make_float4(st[0][0].x, st[1][0].x, st[2][0].x, st[3][0].x)
                                           : make_float4(st[0][1].y, st[1][1].y, st[2][1].y, st[3][1].y);
  };

  // one source plane into the sums of destination planes p - 1, p, p + 1
  auto update = [&](auto mode, P(&ap)[2][K], P(&ac)[2][K], P(&an)[2][K]) {
    constexpr int MODE = decltype(mode)::value;
    if constexpr (Lay::XSH) {
      xs.ye = Ye + ybuf * Lay::ye_buf_pairs;
      ybuf ^= 1;
      fold_update_xs<S, C, MODE, BXC, TY>(st, hsrc, kFieldStride, halo, ap, ac, an, xs, r, active);
    } else {
      fold_update<S, C, MODE, BXC, TY>(st, hsrc, kFieldStride, halo, ap, ac, an, sb, r, active);
    }
  };

  P R0[2][K], R1[2][K], R2[2][K];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < K; ++k) R0[q][k] = R1[q][k] = R2[q][k] = O::splat(C(0));

#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) fetch(i);
  // first (halo) plane z0 - 1: only the equilibria moving up the march axis,
  // into destination plane z0 (= R1 of the first step)
  fetch(kStages - 1);
  take(0);
  if (plane_exists(z0 - 1)) update(std::integral_constant<int, kFirst>{}, R0, R2, R1);

  auto store = [&](int q, P(&acc)[2][K]) {
    float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (xwall1) wv = wring[(q - z0 + 1) & (kStages - 1)];  // kept when plane q was taken
    fold_store<S>(op, mrow, ta, (int64_t)q * ps, x_lo_wall, x_hi_wall, wv, store_skip(q), acc, force);
  };

  // full plane p: contributions to the sums A (dest p - 1), B (dest p), N (dest
  // p + 1); then A is complete
  auto step = [&](int p, P(&A)[2][K], P(&B)[2][K], P(&N)[2][K]) {
    const int i = p - z0 + 1;
    fetch(i + kStages - 1);
    take(i);
    update(std::integral_constant<int, kMid>{}, A, B, N);
    if (p - 1 >= z0) store(p - 1, A);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k) A[q][k] = O::splat(C(0));
  };
  // last (halo) plane z1: only the equilibria moving down, into plane z1 - 1 (= B)
  auto last = [&](P(&B)[2][K]) {
    const int i = np - 1;
    fetch(i + kStages - 1);
    take(i);
    if (plane_exists(z1)) update(std::integral_constant<int, kLast>{}, B, R0, R0);
    store(z1 - 1, B);
  };
  // the three plane sums rotate with period 3
  for (int p = z0;; p += 3) {
    step(p, R0, R1, R2);
    if (p + 1 >= z1) { last(R1); break; }
    step(p + 1, R1, R2, R0);
    if (p + 2 >= z1) { last(R2); break; }
    step(p + 2, R2, R0, R1);
    if (p + 3 >= z1) { last(R0); break; }
  }
  cp_async_wait<0>();
}

// Launch one instance (the instances are in step_fold.cu).  With resident_out
// set, only report the blocks of this shape one SM holds.
template <typename S, int BXC, int TY>
cudaError_t launch_fold_shape(const TiledArgs& ta, const void* in, void* out, cudaStream_t stream, dim3 grid,
                              int* resident_out) {
  auto kern = step_fold<S, BXC, TY>;
  constexpr size_t smem = FoldLayout<S, BXC, TY>::smem;
  static int resident_dev[64] = {};  // per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& resident = resident_dev[dev & 63];
  if (!resident) {
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BXC * TY, smem);
    if (e != cudaSuccess) return e;
    resident = nb < 1 ? 1 : nb;
  }
  if (resident_out) {
    *resident_out = resident;
    return cudaSuccess;
  }
  return launch_kernel(kern, grid, dim3(BXC, TY), smem, stream, ta.overlap, ta, static_cast<const S*>(in),
                       static_cast<S*>(out));
}

}  // namespace maclab
