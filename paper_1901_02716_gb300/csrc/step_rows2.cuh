// step_rows2.cuh -- D3Q19 MacLAB step with two rows per thread (Eqs. (2),
// (4), (5); the same update as step_naive, summed in another order).
//
// Layout and march as in step_tiled.cuh: storage rows interleaved in halves
// (a thread's 16-byte quad is the node pairs a = (2t, 2t + H), b = (2t + 1,
// 2t + 1 + H)), a block marches z over a chunk of planes keeping the sums of
// the destination planes p - 1, p, p + 1 in registers.  What differs:
//
//  * Each thread owns the quads of two adjacent rows (r0 = 2 tr, r1 = r0 + 1)
//    of a tile of TY = 2 TYT rows.  Equilibria moving between its two rows
//    stay in registers (or go to a neighbouring lane by a warp shuffle when
//    they also move in x); only those leaving the thread's row pair in y go
//    through shared memory: half the exchange of one row per thread.  The
//    terms of one node pair are formed at a time, and each row's x-crossing
//    values go by shuffle as soon as its two pairs are done, which keeps the
//    register footprint near what two blocks per SM allow without spilling.
//  * The y exchange is laid out for the receiver: for each direction and each
//    receiving thread-row there is one 16-byte unit per column holding the two
//    values its pairs a and b gather, so a receiver reads a direction with one
//    16-byte load.  Senders of the diagonal directions write their pair-b (+x)
//    or pair-a (-x) value into the neighbouring column; at the seam between
//    the row's halves the lane-swapped value is written, chosen per lane with
//    selects (no divergent stores).
//  * The halo rows next to the tile are loaded by the first and last
//    thread-rows, which publish the halo's inward equilibria into the same
//    exchange units a neighbouring thread-row would have filled: every thread
//    then gathers the same way, with no branch on its position.
//  * Terms of Eq. (2) per node: B_i = 3 rho u_i, P_ii = 3/2 B_i u_i,
//    A = drho - (P_xx + P_yy + P_zz) / 3, S_i = A + P_ii, and for each axis
//    pair (i, j) the sums S_i + P_jj +- 3 B_i u_j and B_i +- B_j.  A direction
//    along an axis has T = S_i +- B_i and is added with its integer weight 2 by
//    a fused multiply-add; the rest direction adds 12 A; the diagonals add 1 T.
//    The sums are R = 36 drho' and M = 36 m', u' = M / (36 + R) + F.
//  * Box x-walls: the lanes holding x = 0 or x = nx - 1 store the wall node's
//    unchanged values in place of the computed ones, with selects, so every
//    lane stores whole quads.  The values come from the staged plane: when a
//    plane is taken from its stage slot, these lanes copy their wall node's
//    four values of both rows into a small per-thread shared-memory slot
//    (two, by plane parity), which the store of that plane reads a plane
//    later.  (A global load at the store exposed its latency, and registers
//    held across a plane's update do not fit.)
//
// Requires: D3Q19, FP32 arithmetic (FP32, BF16 or FP16 storage), nx % 4 == 0,
// nx / 4 <= BXC, ny % TY == 0, TYT >= 2.
//
// Viscosity-term mode (NU, FP32 storage): the same march and exchanges gather
// the moments of g_a = w_a (drho + rho (3/2 u.u - 9/2 (c.u)^2)) (the
// equilibrium less its derivative along u and its constant: Eq. (2) with no
// linear part and the quadratic part negated) instead of Eq. (2) itself, and
// the store becomes a sum: with R and u' of the stored state after the step,
// drho' along u is dR = R - G0, and each fluid node adds
//   lam_rho (-dR / 36) + sum_i lam_u_i (Md_i / (36 + R) + (u'_i - F_i) dR / (36 + R) - F_i),
// Md = the first moments of g, into the accumulator (the term of
// maclab_adjoint_nu_term, per node as in adj_nu_term).

#pragma once
#include "step_fold.cuh"

namespace maclab {

// ------------------------------------------------------------------ terms

template <typename C>
struct Terms3 {
  using P = typename Pair<C>::P;
  P A;      // drho - 3/2 rho u.u
  P B[3];   // 3 rho u_i
  P S[3];   // A + 9/2 rho u_i^2
  P Ep[3], Em[3];  // pair k = (i, j): S_i + 9/2 rho u_j^2 +- 9 rho u_i u_j
  P Op[3], Om[3];  // B_i +- B_j
};

template <typename C>
__device__ __forceinline__ void make_terms3(typename Pair<C>::P r, const typename Pair<C>::P (&u)[3],
                                            Terms3<C>& t) {
  using O = Pair<C>;
  using P = typename O::P;
  const P g = O::fma(r, O::splat(C(3)), O::splat(C(3)));  // 3 (1 + drho)
  P Pd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    t.B[i] = O::mul(g, u[i]);
    Pd[i] = O::mul(O::mul(t.B[i], u[i]), O::splat(C(1.5)));
  }
  const P psum = O::add(O::add(Pd[0], Pd[1]), Pd[2]);
  t.A = O::fma(psum, O::splat(C(-1.0 / 3.0)), r);
#pragma unroll
  for (int i = 0; i < 3; ++i) t.S[i] = O::add(t.A, Pd[i]);
  // 9 rho u_i u_j = (3 B_i) u_j, formed inside the fused multiply-adds
  const P B30 = O::mul(t.B[0], O::splat(C(3)));
  const P B31 = O::mul(t.B[1], O::splat(C(3)));
  const P nu1 = O::sub(O::splat(C(0)), u[1]);
  const P nu2 = O::sub(O::splat(C(0)), u[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i + 1; j < 3; ++j) {
      const int k = pair_index(i, j);
      const P base = O::add(t.S[i], Pd[j]);
      const P b3 = i == 0 ? B30 : B31;
      t.Ep[k] = O::fma(b3, u[j], base);
      t.Em[k] = O::fma(b3, j == 1 ? nu1 : nu2, base);
      t.Op[k] = O::add(t.B[i], t.B[j]);
      t.Om[k] = O::sub(t.B[i], t.B[j]);
    }
}

// Terms of g_a / w_a = drho + rho (3/2 u.u - 9/2 (c.u)^2) in the same slots:
// A = drho + 3/2 rho u.u, S_i = A - 9/2 rho u_i^2, and for the pair (i, j)
// Ep = S_i - 9/2 rho u_j^2 - 9 rho u_i u_j, Em = ... + 9 rho u_i u_j; no B, O.
template <typename C>
__device__ __forceinline__ void make_terms3_nu(typename Pair<C>::P r, const typename Pair<C>::P (&u)[3],
                                               Terms3<C>& t) {
  using O = Pair<C>;
  using P = typename O::P;
  const P g = O::fma(r, O::splat(C(3)), O::splat(C(3)));  // 3 (1 + drho)
  P B[3], Pd[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    B[i] = O::mul(g, u[i]);
    Pd[i] = O::mul(O::mul(B[i], u[i]), O::splat(C(1.5)));  // 9/2 rho u_i^2
  }
  const P psum = O::add(O::add(Pd[0], Pd[1]), Pd[2]);
  t.A = O::fma(psum, O::splat(C(1.0 / 3.0)), r);
#pragma unroll
  for (int i = 0; i < 3; ++i) t.S[i] = O::sub(t.A, Pd[i]);
  const P B30 = O::mul(B[0], O::splat(C(3)));
  const P B31 = O::mul(B[1], O::splat(C(3)));
  const P nu1 = O::sub(O::splat(C(0)), u[1]);
  const P nu2 = O::sub(O::splat(C(0)), u[2]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i + 1; j < 3; ++j) {
      const int k = pair_index(i, j);
      const P base = O::sub(t.S[i], Pd[j]);
      const P b3 = i == 0 ? B30 : B31;
      t.Ep[k] = O::fma(b3, j == 1 ? nu1 : nu2, base);
      t.Em[k] = O::fma(b3, u[j], base);
    }
}

// T_a of both lanes (axis directions undoubled: they carry the weight 2)
template <typename C, int A, bool NU = false>
__device__ __forceinline__ typename Pair<C>::P term3(const Terms3<C>& t) {
  using L = Lattice<kD3Q19>;
  using O = Pair<C>;
  constexpr int nzc = Dir<kD3Q19>::nz(A);
  constexpr int i0 = Dir<kD3Q19>::first(A), i1 = Dir<kD3Q19>::second(A);
  if constexpr (nzc == 0) {
    return t.A;
  } else if constexpr (nzc == 1) {
    if constexpr (NU) return t.S[i0];
    else if constexpr (L::c(A, i0) > 0) return O::add(t.S[i0], t.B[i0]);
    else return O::sub(t.S[i0], t.B[i0]);
  } else {
    constexpr int k = pair_index(i0, i1);
    constexpr int s0 = L::c(A, i0), s1 = L::c(A, i1);
    if constexpr (NU) {
      return s0 == s1 ? t.Ep[k] : t.Em[k];
    } else if constexpr (s0 == s1) {
      if constexpr (s0 > 0) return O::add(t.Ep[k], t.Op[k]);
      else return O::sub(t.Ep[k], t.Op[k]);
    } else {
      if constexpr (s0 > 0) return O::add(t.Em[k], t.Om[k]);
      else return O::sub(t.Em[k], t.Om[k]);
    }
  }
}

// Constants of the weighted sums, held in registers once.
template <typename C>
struct Weights3 {
  using P = typename Pair<C>::P;
  P w12, w2, wm2;
};

// acc[0] += w36 T; acc[1 + i] += c_i w36 T
template <typename C, int A>
__device__ __forceinline__ void accum3(typename Pair<C>::P (&acc)[4], typename Pair<C>::P T,
                                       const Weights3<C>& w) {
  using L = Lattice<kD3Q19>;
  using O = Pair<C>;
  constexpr int wt = L::w36(A);
  if constexpr (wt == 1) {
    acc[0] = O::add(acc[0], T);
    static_for<0, 3>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (L::c(A, i) == 1) acc[1 + i] = O::add(acc[1 + i], T);
      else if constexpr (L::c(A, i) == -1) acc[1 + i] = O::sub(acc[1 + i], T);
    });
  } else if constexpr (wt == 2) {
    acc[0] = O::fma(w.w2, T, acc[0]);
    static_for<0, 3>([&](auto I) {
      constexpr int i = decltype(I)::value;
      if constexpr (L::c(A, i) == 1) acc[1 + i] = O::fma(w.w2, T, acc[1 + i]);
      else if constexpr (L::c(A, i) == -1) acc[1 + i] = O::fma(w.wm2, T, acc[1 + i]);
    });
  } else {
    acc[0] = O::fma(w.w12, T, acc[0]);
  }
}

// index of direction a among the five with the same c_y (c_y != 0)
__host__ __device__ constexpr int rows2_ykey(int a) {
  using F = Frame<kD3Q19>;
  int k = 0;
  for (int b = 0; b < a; ++b) k += F::fy(b) == F::fy(a) ? 1 : 0;
  return k;
}

// ------------------------------------------------------------------ layout

template <typename S, int BXC, int TYT>
struct Rows2Layout {
  static constexpr int TY = 2 * TYT;
  static constexpr int RS = TY + 2;       // staged rows: lower halo, TY own, upper halo
  static constexpr int YC = BXC + 1;      // units per slot row (+1: the idle lanes' column)
  static constexpr int NSLOT = TYT + 1;   // receiving rows per sign (see step_rows2)
  static constexpr int DIR_UNITS = NSLOT * YC;
  static constexpr int SIGN_UNITS = 5 * DIR_UNITS;
  static constexpr int BUF_UNITS = 2 * SIGN_UNITS;
  static constexpr size_t y_bytes = (size_t)2 * BUF_UNITS * 16;  // two buffers of 16-byte units
  // a stage slot: the TY own rows [4 fields][TY][row], then the halo rows
  // below and above, [4 fields][row] each, as the tile copies lay them out
  // (a row is nx stored values); offsets are multiples of 128 bytes
  static constexpr size_t QB = (size_t)BXC * Quad<S>::BYTES;  // the widest row
  static constexpr size_t slot_bytes = 4 * RS * QB;
  static constexpr size_t halo_lo = 4 * TY * QB;
  static constexpr size_t halo_hi = halo_lo + 4 * QB;
  static constexpr size_t stage_bytes = (size_t)kStages * slot_bytes;
  static constexpr size_t mbar_off = stage_bytes;        // one mbarrier per slot
  static constexpr size_t y_off = stage_bytes + 16;
  // box x-wall values of the two planes in flight, [plane parity][TYT][side]
  // [2 rows x 4 fields] floats, each slot written and read by its own thread
  static constexpr size_t wall_off = y_off + y_bytes;
  static constexpr size_t wall_bytes = (size_t)2 * TYT * 2 * 8 * sizeof(float);
  // + 128: the base is rounded up to a 128-byte boundary at run time
  static constexpr size_t smem = 128 + wall_off + wall_bytes;
  static constexpr int THREADS = BXC * TYT;
  // at least eight warps per SM where shared memory allows
  static constexpr int SMEM_BLOCKS = (int)((220 * 1024) / smem) < 1 ? 1 : (int)((220 * 1024) / smem);
  static constexpr int WANT = 256 / THREADS < 1 ? 1 : 256 / THREADS;
  static constexpr int MIN_BLOCKS = WANT < SMEM_BLOCKS ? WANT : SMEM_BLOCKS;
};

// ------------------------------------------------------------------ kernel

// Running float-float sum of one thread (viscosity-term mode): Knuth's two-sum
// keeps the rounding error of every FP32 addition.
struct Rows2Sum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
    hi = s;
  }
};

// NU: viscosity-term mode (see the top of this file); `out` is then the state
// after the step, read only.
// Tile copies: tm_own maps the state as [4 fields][nz][ny][nx] with a box of the
// tile's TY own rows of every field; tm_halo the same tensor with a box of one
// row of every field.
template <typename S, int BXC, int TYT, bool NU = false>
__global__ void __launch_bounds__(BXC * TYT, Rows2Layout<S, BXC, TYT>::MIN_BLOCKS)
    step_rows2(TiledArgs ta, const S* __restrict__ in, S* __restrict__ out,
               const __grid_constant__ CUtensorMap tm_own, const __grid_constant__ CUtensorMap tm_halo) {
  using Lay = Rows2Layout<S, BXC, TYT>;
  using C = float;
  using O = Pair<C>;
  using P = typename O::P;
  using L = Lattice<kD3Q19>;
  using F = Frame<kD3Q19>;
  constexpr int TY = Lay::TY;
  constexpr int RS = Lay::RS;
  constexpr int YC = Lay::YC;
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // stage slots at a 128-byte boundary (tile copies land on it), then the
  // mbarriers, then the y exchange
  unsigned char* const smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
  const int tx = threadIdx.x, tr = threadIdx.y;
  // issues the tile copies: a thread of a middle thread-row, which forms no
  // halo row, where there is one
  const bool leader = tx == 0 && tr == (TYT > 2 ? 1 : 0);
  const uint32_t mbar0 = smem_u32(smem_raw + Lay::mbar_off);
  if (leader) {
    mbar_init(mbar0, 1);
    mbar_init(mbar0 + 8, 1);
    mbar_init_fence();
  }
  __syncthreads();
  pdl_wait();  // the previous step's writes are visible from here on
  pdl_launch_next();

  const int bxr = ta.nx >> 2;  // threads per row actually used
  const bool active = tx < bxr;
  float4* const Y = reinterpret_cast<float4*>(smem_raw + Lay::y_off);

  // columns: own, the right neighbour's (the unit a +x diagonal value goes to)
  // and the left one's (-x); idle lanes write into the spare column BXC
  const int col = tx;
  const int col_r = !active ? BXC : (tx + 1 == bxr ? 0 : tx + 1);
  const int col_l = !active ? BXC : (tx == 0 ? bxr - 1 : tx - 1);
  const bool seam_r = tx == bxr - 1;  // +x across the seam: send lane-swapped
  const bool seam_l = tx == 0;        // -x across the seam
  // shuffle sources and lane swaps of the x exchange (width BXC)
  const int src_l = tx == 0 ? bxr - 1 : tx - 1;
  const int src_r = tx == bxr - 1 ? 0 : tx + 1;

  // rows: own rows 2 tr, 2 tr + 1 of the tile; the first thread-row also
  // forms the equilibria of the row below the tile, the last one those of the
  // row above (staged with the tile)
  const int row0 = blockIdx.y * TY + 2 * tr;
  int halo = tr == 0 ? 1 : (tr == TYT - 1 ? -1 : 0);
  {
    const int hrow = halo == 1 ? row0 - 1 : row0 + 2;
    if (halo != 0 && (hrow < 0 || hrow >= ta.ny) && !ta.py)
      halo = 0;  // beyond a closed y boundary: the row next to it is a wall row
  }
  bool row_wall[2];
  row_wall[0] = !ta.py && row0 == 0;
  row_wall[1] = !ta.py && row0 + 1 == ta.ny - 1;
  const int64_t row_off = (int64_t)row0 * ta.nx + 4 * tx;
  const bool x_lo_wall = ta.wall_mode == kWallBox && !ta.px && tx == 0;
  const bool x_hi_wall = ta.wall_mode == kWallBox && !ta.px && tx == bxr - 1;
  const bool box_x = ta.wall_mode == kWallBox && !ta.px;
  const bool per_node_store = ta.wall_mode == kWallMask || (x_lo_wall && x_hi_wall);
  // box x-walls: the lanes holding x = 0 or nx - 1 keep the wall node's values
  // of a staged plane (walls never change) in their own shared-memory slot
  // until the plane is stored, a plane later, instead of registers or a
  // global load at the store
  const bool keep_walls = !NU && box_x && (x_lo_wall || x_hi_wall) && !per_node_store;
  float* const WV = reinterpret_cast<float*>(smem_raw + Lay::wall_off);
  auto wall_slot = [&](int parity) { return ((parity * TYT + tr) * 2 + (x_hi_wall ? 1 : 0)) * 8; };

  S* op[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) op[f] = out + (int64_t)f * ta.n + row_off;
  const uint8_t* mrow = ta.wall_mode == kWallMask ? ta.mask + row_off : nullptr;
  P force[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) force[i] = O::splat(C(ta.force[i]));
  Weights3<C> wts;
  wts.w12 = O::splat(C(12));
  wts.w2 = O::splat(C(2));
  wts.wm2 = O::splat(C(-2));

  const int z0 = (int)(((int64_t)blockIdx.x * ta.nplanes) / ta.nzc);
  const int z1 = (int)(((int64_t)(blockIdx.x + 1) * ta.nplanes) / ta.nzc);
  const int64_t ps = ta.plane_stride;
  const int64_t nx64 = ta.nx;
  auto plane_exists = [&](int p) { return (p >= 0 && p < ta.nplanes) || ta.pz; };
  auto plane_mem = [&](int p) { return p < 0 ? p + ta.nplanes : (p >= ta.nplanes ? p - ta.nplanes : p); };
  const bool zwall = !ta.pz;

  // stage slots (Lay): own row j of this thread at row 2 tr + j of the own
  // block, the halo row below or above in its block; rows are nx values
  // (rowB bytes) as the tile copies write them
  constexpr int QW = Quad<S>::BYTES;
  static_assert(kStages == 2, "two stage slots, two mbarriers");
  const uint32_t rowB = (uint32_t)bxr * QW;
  const uint32_t fieldB = (uint32_t)TY * rowB;  // own block: [4 fields][TY rows]
  const uint32_t own_off = (uint32_t)(2 * tr) * rowB + (uint32_t)tx * QW;
  const uint32_t halo_off = (uint32_t)(halo == 1 ? Lay::halo_lo : Lay::halo_hi) + (uint32_t)tx * QW;
  const uint32_t stage_sh = smem_u32(smem_raw);
  const int np = z1 - z0 + 2;  // planes z0 - 1 .. z1
  // halo rows of the tile (wrapped on a periodic y axis; none beyond a closed one)
  const int tile_row0 = blockIdx.y * TY;
  int lo_row = tile_row0 - 1, hi_row = tile_row0 + TY;
  bool lo_ok = true, hi_ok = true;
  if (lo_row < 0) {
    if (ta.py) lo_row += ta.ny;
    else lo_ok = false;
  }
  if (hi_row >= ta.ny) {
    if (ta.py) hi_row -= ta.ny;
    else hi_ok = false;
  }
  const uint32_t tile_bytes = 4 * fieldB + (lo_ok ? 4 * rowB : 0u) + (hi_ok ? 4 * rowB : 0u);
  // debug builds: a quad copy or load of 4 values at element offset e (from
  // `in` or `out`) and a stage byte offset b must lie in bounds
  const int64_t n4 = 4 * ta.n;
  const int64_t in_off = row_off;
  // plane z0 - 1 + i into slot i & 1: one thread copies the tile's own rows
  // and its halo rows of the four fields; a plane that does not exist (beyond
  // a closed march axis) completes the slot's phase with no bytes
  auto fetch = [&](int i) {
    if (!leader || i >= np) return;
    const int p = z0 - 1 + i;
    const uint32_t s = (uint32_t)(i & 1);
    const uint32_t bar = mbar0 + 8 * s;
    const uint32_t dst = stage_sh + s * (uint32_t)Lay::slot_bytes;
    if (plane_exists(p)) {
      const int pm = plane_mem(p);
      proxy_async_fence();  // the block's reads of this slot (before its last barrier) come first
      mbar_arrive_expect_tx(bar, tile_bytes);
      tma_load_4d(dst, &tm_own, 0, tile_row0, pm, 0, bar);
      if (lo_ok) tma_load_4d(dst + (uint32_t)Lay::halo_lo, &tm_halo, 0, lo_row, pm, 0, bar);
      if (hi_ok) tma_load_4d(dst + (uint32_t)Lay::halo_hi, &tm_halo, 0, hi_row, pm, 0, bar);
    } else {
      mbar_arrive(bar);
    }
  };
  P st[2][4][2];
  const unsigned char* slot_base = smem_raw;
  auto take = [&](int i) {
    const int p = z0 - 1 + i;
    const uint32_t s = (uint32_t)(i & 1);
    if (!mbar_wait(mbar0 + 8 * s, (uint32_t)(i >> 1) & 1u) && ta.status) atomicOr(ta.status, 1u);
    const bool ok = active && plane_exists(p);
    slot_base = smem_raw + (size_t)s * Lay::slot_bytes;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int64_t b = (int64_t)s * Lay::slot_bytes + own_off + j * rowB + f * fieldB;
        if (ok && bounds_ok(ta.bounds, b, (int64_t)Lay::stage_bytes - QW + 1)) {
          Quad<S>::lds(reinterpret_cast<const S*>(smem_raw + b), st[j][f][0], st[j][f][1]);
        } else {
          st[j][f][0] = st[j][f][1] = O::splat(C(0));
        }
      }
    if (keep_walls) {
      const int w = wall_slot(i & 1);
#pragma unroll
      for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (bounds_ok(ta.bounds, w + 4 * j + f, (int64_t)(Lay::wall_bytes / sizeof(float))))
            WV[w + 4 * j + f] = x_lo_wall ? st[j][f][0].x : st[j][f][1].y;
    }
  };

  // ---------------------------------------------------------------- one plane
  int ybuf = 0;
  // publish the equilibria of pair values (Ta, Tb) of direction A into the
  // units of slot row `slot` of sign FY (receivers: the thread-row that owns
  // that slot)
  auto publish = [&](float4* ybase, auto dir, int slot, P Ta, P Tb) {
    constexpr int A = decltype(dir)::value;
    constexpr int FY = F::fy(A), FX = F::fx(A);
    float4* const u = ybase + (FY == 1 ? 0 : Lay::SIGN_UNITS) + rows2_ykey(A) * Lay::DIR_UNITS + slot * YC;
    auto unit_ok = [&](int c) { return bounds_ok(ta.bounds, (u + c) - Y, 2 * Lay::BUF_UNITS); };
    if constexpr (FX == 0) {
      if (unit_ok(col)) u[col] = make_float4(Ta.x, Ta.y, Tb.x, Tb.y);
    } else if constexpr (FX == 1) {
      // receiver column c gathers (left neighbour's b, own a)
      if (unit_ok(col)) reinterpret_cast<float2*>(u + col)[1] = Ta;
      const P b = seam_r ? O::swap(Tb) : Tb;
      if (unit_ok(col_r)) reinterpret_cast<float2*>(u + col_r)[0] = b;
    } else {
      // receiver column c gathers (own b, right neighbour's a)
      if (unit_ok(col)) reinterpret_cast<float2*>(u + col)[0] = Tb;
      const P a = seam_l ? O::swap(Ta) : Ta;
      if (unit_ok(col_l)) reinterpret_cast<float2*>(u + col_l)[1] = a;
    }
  };

  // the value of one pair (q) of direction A into its half of the receiver's unit
  auto publish_half = [&](float4* ybase, auto dir, auto qc, int slot, P T) {
    constexpr int A = decltype(dir)::value;
    constexpr int q = decltype(qc)::value;
    constexpr int FY = F::fy(A), FX = F::fx(A);
    float4* const u = ybase + (FY == 1 ? 0 : Lay::SIGN_UNITS) + rows2_ykey(A) * Lay::DIR_UNITS + slot * YC;
    auto unit_ok = [&](int c) { return bounds_ok(ta.bounds, (u + c) - Y, 2 * Lay::BUF_UNITS); };
    if constexpr (FX == 0) {
      if (unit_ok(col)) reinterpret_cast<float2*>(u + col)[q] = T;
    } else if constexpr (FX == 1) {
      if constexpr (q == 0) {
        if (unit_ok(col)) reinterpret_cast<float2*>(u + col)[1] = T;
      } else {
        const P b = seam_r ? O::swap(T) : T;
        if (unit_ok(col_r)) reinterpret_cast<float2*>(u + col_r)[0] = b;
      }
    } else {
      if constexpr (q == 1) {
        if (unit_ok(col)) reinterpret_cast<float2*>(u + col)[0] = T;
      } else {
        const P a = seam_l ? O::swap(T) : T;
        if (unit_ok(col_l)) reinterpret_cast<float2*>(u + col_l)[1] = a;
      }
    }
  };
  auto update = [&](auto mode, P(&ap)[2][2][4], P(&ac)[2][2][4], P(&an)[2][2][4]) {
    constexpr int MODE = decltype(mode)::value;
    const int ybuf_units = ybuf * Lay::BUF_UNITS;
    float4* const ybase = Y + ybuf_units;
    ybuf ^= 1;
    // one pair at a time (terms of one pair live at once); each row's x-crossing
    // values go by shuffle as soon as the row is done
    auto shuffle_in = [&](auto dir, auto jdc, P vb_or_va) {
      constexpr int a = decltype(dir)::value;
      constexpr int jd = decltype(jdc)::value;
      constexpr int fx = F::fx(a), fz = F::fz(a);
      auto& dst = pick<fz>(ap, ac, an)[jd];
      if constexpr (fx == 1) {
        P v = fold_shfl<BXC>(vb_or_va, src_l);
        if (seam_l) v = O::swap(v);
        accum3<C, a>(dst[0], v, wts);
      } else {
        P v = fold_shfl<BXC>(vb_or_va, src_r);
        if (seam_r) v = O::swap(v);
        accum3<C, a>(dst[1], v, wts);
      }
    };
    static_for<0, 2>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      constexpr int jd = 1 - j;
      P xb[4], xa[4];  // [k]: k < 3 own c_y = 0 directions, 3: the diagonal into row jd
#pragma unroll
      for (int k = 0; k < 4; ++k) xb[k] = xa[k] = O::splat(C(0));
      static_for<0, 2>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        Terms3<C> t;
        {
          const P u[3] = {st[j][1][q], st[j][2][q], st[j][3][q]};
          if constexpr (NU) make_terms3_nu<C>(st[j][0][q], u, t);
          else make_terms3<C>(st[j][0][q], u, t);
        }
        static_for<0, L::Q>([&](auto I) {
          constexpr int a = decltype(I)::value;
          if constexpr (mode_allows<kD3Q19, MODE>(a)) {
            constexpr int fx = F::fx(a), fy = F::fy(a), fz = F::fz(a);
            const P T = term3<C, a, NU>(t);
            if constexpr (fy == 0) {
              auto& dst = pick<fz>(ap, ac, an)[j];
              constexpr int qd = q + fx;
              if constexpr (qd >= 0 && qd < 2) accum3<C, a>(dst[qd], T, wts);
              else if constexpr (fx == 1) xb[fold_xidx(a)] = T;
              else xa[fold_xidx(a)] = T;
            } else if constexpr ((j == 0 && fy == 1) || (j == 1 && fy == -1)) {
              auto& dst = pick<fz>(ap, ac, an)[jd];
              constexpr int qd = q + fx;
              if constexpr (qd >= 0 && qd < 2) accum3<C, a>(dst[qd], T, wts);
              else if constexpr (fx == 1) xb[3] = T;
              else xa[3] = T;
            } else {
              publish_half(ybase, I, qc, j == 1 ? tr + 1 : tr, T);
            }
          }
        });
      });
      static_for<0, L::Q>([&](auto I) {
        constexpr int a = decltype(I)::value;
        constexpr int fx = F::fx(a), fy = F::fy(a), fz = F::fz(a);
        if constexpr (mode_allows<kD3Q19, MODE>(a) && fy == 0 && fx != 0)
          shuffle_in(I, jc, fx == 1 ? xb[fold_xidx(a)] : xa[fold_xidx(a)]);
        if constexpr (mode_allows<kD3Q19, MODE>(a) && fz == 0 && fx != 0 &&
                      ((j == 0 && fy == 1) || (j == 1 && fy == -1)))
          shuffle_in(I, std::integral_constant<int, jd>{}, fx == 1 ? xb[3] : xa[3]);
      });
    });
    // ---- halo row: its inward equilibria into the slot its neighbour reads
    if (halo != 0) {  // idle lanes publish into their own or the spare column
      P hs[4][2];
      const int64_t hb = (int64_t)(slot_base - smem_raw) + halo_off;
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        if (bounds_ok(ta.bounds, hb + f * rowB, (int64_t)Lay::stage_bytes - QW + 1))
          Quad<S>::lds(reinterpret_cast<const S*>(smem_raw + hb + f * rowB), hs[f][0], hs[f][1]);
        else
          hs[f][0] = hs[f][1] = O::splat(C(0));
      }
      Terms3<C> t[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const P u[3] = {hs[1][q], hs[2][q], hs[3][q]};
        if constexpr (NU) make_terms3_nu<C>(hs[0][q], u, t[q]);
        else make_terms3<C>(hs[0][q], u, t[q]);
      }
      if (halo == 1) {
        static_for<0, L::Q>([&](auto I) {
          constexpr int a = decltype(I)::value;
          if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == 1)
            publish(ybase, I, 0, term3<C, a, NU>(t[0]), term3<C, a, NU>(t[1]));
        });
      } else {
        static_for<0, L::Q>([&](auto I) {
          constexpr int a = decltype(I)::value;
          if constexpr (mode_allows<kD3Q19, MODE>(a) && F::fy(a) == -1)
            publish(ybase, I, TYT, term3<C, a, NU>(t[0]), term3<C, a, NU>(t[1]));
        });
      }
    }
    __syncthreads();
    // ---- gather: row 0 the +y units of slot tr, row 1 the -y units of slot tr + 1
    static_for<0, L::Q>([&](auto I) {
      constexpr int a = decltype(I)::value;
      constexpr int fy = F::fy(a), fz = F::fz(a);
      if constexpr (mode_allows<kD3Q19, MODE>(a) && fy != 0) {
        constexpr int j = fy == 1 ? 0 : 1;
        const int slot = fy == 1 ? tr : tr + 1;
        const int64_t unit = (int64_t)ybuf_units + (fy == 1 ? 0 : Lay::SIGN_UNITS) + rows2_ykey(a) * Lay::DIR_UNITS +
                             slot * YC + col;
        const float4 v = bounds_ok(ta.bounds, unit, 2 * Lay::BUF_UNITS) ? Y[unit] : make_float4(0.f, 0.f, 0.f, 0.f);
        auto& dst = pick<fz>(ap, ac, an)[j];
        accum3<C, a>(dst[0], O::make(v.x, v.y), wts);
        accum3<C, a>(dst[1], O::make(v.z, v.w), wts);
      }
    });
  };

  // ---------------------------------------------------------------- store
  Rows2Sum nus;  // viscosity-term mode: this thread's sum
  // viscosity-term mode: the stored state after the step and lam of the plane
  // q the next store sums, loaded early so their latency overlaps the update
  P nsn[2][4][2], nlm[2][4][2];
  auto nu_prefetch = [&](int q) {
    if constexpr (NU) {
      const bool zskip = zwall && (q == 0 || q == ta.nplanes - 1);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const bool skip = !active || row_wall[j] || zskip || q < 0 || q >= ta.nplanes;
        const int64_t off = (int64_t)q * ps + j * nx64;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const int64_t e = f * ta.n + in_off + off;
          if (!skip && bounds_ok(ta.bounds, e, n4 - 3)) {
            Quad<S>::ld(out + e, nsn[j][f][0], nsn[j][f][1]);
            Quad<float>::ld(ta.lam + e, nlm[j][f][0], nlm[j][f][1]);
          } else {
            nsn[j][f][0] = nsn[j][f][1] = nlm[j][f][0] = nlm[j][f][1] = O::splat(C(0));
          }
        }
      }
    }
  };
  auto store = [&](int q, P(&acc)[2][2][4]) {
    const bool zskip = zwall && (q == 0 || q == ta.nplanes - 1);
    if constexpr (NU) {
      // the viscosity term of the fluid nodes of the two rows: R and u' of the
      // stored state after the step and lam, loaded by nu_prefetch(q) before
      // the plane update that precedes this store
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        if (!active || row_wall[j] || zskip) continue;
        const int64_t off = (int64_t)q * ps + j * nx64;
        const P(&sn)[4][2] = nsn[j];
        const P(&lm)[4][2] = nlm[j];
        // fluid lanes: (pair a.x, a.y, b.x, b.y) = storage positions 4 tx .. 4 tx + 3
        bool fl[4] = {!x_lo_wall, true, true, !x_hi_wall};
        if (ta.wall_mode == kWallMask && bounds_ok(ta.bounds, in_off + off, ta.n - 3)) {
          const uchar4 mk = *reinterpret_cast<const uchar4*>(mrow + off);
          fl[0] = mk.x == 0; fl[1] = mk.y == 0; fl[2] = mk.z == 0; fl[3] = mk.w == 0;
        }
        float part = 0.f;
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          const P R = O::mul(sn[0][qq], O::splat(C(36)));
          const P inv = O::rcp(O::add(O::splat(C(36)), R));
          const P dR = O::sub(R, acc[j][qq][0]);
          const P dRi = O::mul(dR, inv);
          P t = O::mul(lm[0][qq], O::mul(dR, O::splat(C(-1.0 / 36.0))));
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const P unf = O::sub(sn[1 + i][qq], force[i]);
            const P du = O::sub(O::fma(unf, dRi, O::mul(acc[j][qq][1 + i], inv)), force[i]);
            t = O::fma(lm[1 + i][qq], du, t);
          }
          part += (fl[2 * qq] ? t.x : 0.f) + (fl[2 * qq + 1] ? t.y : 0.f);
        }
        nus.add(part);
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const bool skip = !active || row_wall[j] || zskip;
      const int64_t off = (int64_t)q * ps + j * nx64;
      if (per_node_store) {
        S* const fp[4] = {op[0], op[1], op[2], op[3]};
        store_plane<kD3Q19, S>(fp, mrow, ta, off, x_lo_wall, x_hi_wall, skip, acc[j], force);
        continue;
      }
      if (skip) continue;
      // box x-walls: the values kept when plane q was staged (take index q - z0 + 1)
      float wv[4] = {0.f, 0.f, 0.f, 0.f};
      if (keep_walls) {
        const int w = wall_slot((q - z0 + 1) & 1) + 4 * j;
#pragma unroll
        for (int f = 0; f < 4; ++f)
          if (bounds_ok(ta.bounds, w + f, (int64_t)(Lay::wall_bytes / sizeof(float)))) wv[f] = WV[w + f];
      }
      P v[4][2];
#pragma unroll
      for (int qq = 0; qq < 2; ++qq) {
        const P inv = O::rcp(O::add(O::splat(C(36)), acc[j][qq][0]));
        v[0][qq] = O::mul(acc[j][qq][0], O::splat(C(1.0 / 36.0)));
#pragma unroll
        for (int i = 0; i < 3; ++i) v[1 + i][qq] = O::fma(acc[j][qq][1 + i], inv, force[i]);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        v[f][0].x = x_lo_wall ? wv[f] : v[f][0].x;
        v[f][1].y = x_hi_wall ? wv[f] : v[f][1].y;
        if (bounds_ok(ta.bounds, f * ta.n + in_off + off, n4 - 3)) Quad<S>::st(op[f] + off, v[f][0], v[f][1]);
      }
    }
  };

  P R0[2][2][4], R1[2][2][4], R2[2][2][4];
  auto zero = [&](P(&A)[2][2][4]) {
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) A[j][q][k] = O::splat(C(0));
  };
  zero(R0);
  zero(R1);
  zero(R2);

#pragma unroll
  for (int i = 0; i < kStages - 1; ++i) fetch(i);
  // first (halo) plane z0 - 1: only the equilibria moving up the march axis
  fetch(kStages - 1);
  take(0);
  // (the barrier inside update, or this one, keeps slot 0's next copy behind
  // every thread's wait for its current one)
  if (plane_exists(z0 - 1)) update(std::integral_constant<int, kFirst>{}, R0, R2, R1);
  else __syncthreads();

  // full planes: R0, R1, R2 hold the sums of planes p - 1, p, p + 1; after
  // plane p, p - 1 is complete and the sums move down by one plane.  The
  // loop body is not unrolled: one copy of the two-row update keeps the code
  // within the instruction cache (the moves cost less than the misses of a
  // three-way unrolled body, whose copies would rename the sums instead).
#pragma unroll 1
  for (int p = z0; p < z1; ++p) {
    const int i = p - z0 + 1;
    fetch(i + kStages - 1);
    nu_prefetch(p - 1);
    take(i);
    update(std::integral_constant<int, kMid>{}, R0, R1, R2);
    if (p - 1 >= z0) store(p - 1, R0);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          R0[j][q][k] = R1[j][q][k];
          R1[j][q][k] = R2[j][q][k];
          R2[j][q][k] = O::splat(C(0));
        }
  }
  // last (halo) plane z1: only the equilibria moving down, into plane z1 - 1 (R0)
  {
    const int i = np - 1;
    fetch(i + kStages - 1);
    nu_prefetch(z1 - 1);
    take(i);
    if (plane_exists(z1)) update(std::integral_constant<int, kLast>{}, R0, R1, R1);
    store(z1 - 1, R0);
  }
  if constexpr (NU) {
    // block sum: warp shuffles, one value per warp, one FP64 atomic per block
    double v = (double)nus.hi + (double)nus.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double red[32];
    const int lid = tr * BXC + tx;
    if ((lid & 31) == 0) red[lid >> 5] = v;
    __syncthreads();
    if (lid == 0) {
      double sum = 0.0;
      for (int w = 0; w < (BXC * TYT) / 32; ++w) sum += red[w];
      atomicAdd(ta.nu_acc, sum);
    }
  }
}

// Launch of the instance (bxc, tyt) for storage type S (FP32 instances in
// step_rows2.cu, 16-bit storage in step_rows2_s16.cu).
template <typename S>
cudaError_t rows2_dispatch(int bxc, int tyt, const TiledArgs& ta, const void* in, void* out,
                           const CUtensorMap& tm_own, const CUtensorMap& tm_halo, cudaStream_t st, dim3 grid,
                           int* resident);
// The viscosity-term mode, FP32 storage (instances in step_rows2_nu.cu).
cudaError_t rows2_nu_dispatch(int bxc, int tyt, const TiledArgs& ta, const void* in, const void* out,
                              const CUtensorMap& tm_own, const CUtensorMap& tm_halo, cudaStream_t st, dim3 grid,
                              int* resident);

// Launch one instance.  With resident_out set,
// only report the blocks of this shape one SM holds.
template <typename S, int BXC, int TYT, bool NU = false>
cudaError_t launch_rows2_shape(const TiledArgs& ta, const void* in, void* out, const CUtensorMap& tm_own,
                               const CUtensorMap& tm_halo, cudaStream_t stream, dim3 grid, int* resident_out) {
  auto kern = step_rows2<S, BXC, TYT, NU>;
  constexpr size_t smem = Rows2Layout<S, BXC, TYT>::smem;
  static int resident_dev[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int& resident = resident_dev[dev & 63];
  if (!resident) {
    // set whatever the size: static shared memory counts against the 48 KB
    // default as well
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, BXC * TYT, smem);
    if (e != cudaSuccess) return e;
    resident = nb < 1 ? 1 : nb;
  }
  if (resident_out) {
    *resident_out = resident;
    return cudaSuccess;
  }
  return launch_kernel(kern, grid, dim3(BXC, TYT), smem, stream, ta.overlap, ta, static_cast<const S*>(in),
                       static_cast<S*>(out), tm_own, tm_halo);
}

}  // namespace maclab
